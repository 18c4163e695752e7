// Fq = GF(p), p the 377-bit BLS12-377 base-field prime, on sm_103a.
//
// Representation in registers: 15 digits of radix 2^26 (390 bits), each held in
// a 32-bit register with headroom, Montgomery form x * R mod p with R = 2^390.
// This is the paper's element format idea (Sec. III-B/III-D: 25-bit elements in
// 32-bit lanes, up to 26 bits per element, carries propagated coarsely instead
// of exactly) carried over to the GPU: a product of two 26-bit digits is one
// mad.wide.u32 (32x32 + 64 -> 64) into a 64-bit column sum, and 30 such terms
// fit in 64 bits, so the 29 columns of a*b accumulate with no carry chains at
// all; the 15 Montgomery steps (m_i = -c_i mod 2^26, because p = 1 mod 2^46)
// add m_i * p into the columns the same way; and the result leaves in two
// rounds of coarse carry propagation (mask, shift, add), the paper's step0 /
// step1, not an exact serial carry.
//
// Invariants (checked by the bound analysis in ec.cuh and by the tests):
//  * digits of any multiplication input are < 2^29, its value < 2^383;
//    then every column sum stays below 15*2^58 + 15*2^52 < 2^62 and the
//    Montgomery output value is < a*b/R + p < 2p.
//  * multiplication outputs are "normal": digits 0..13 <= 2^26 + 2^10,
//    digit 14 < 2^14 (value < 2p).
//  * add() is digit-wise (no carries); sub<K>(a, b) is a - b + K*p digit-wise
//    with K*p written in a redundant form whose digits 0..13 are >= 2^28 - 4,
//    so it never goes negative as long as b < (K - 1) p and b's digits are
//    below 2^28 - 4.
// Memory formats stay the packed 12 x 32-bit little-endian limbs (pack/unpack).
#pragma once
#include <stdint.h>

namespace fq {

constexpr int N = 15;      // digits per element
constexpr int NW = 12;     // 32-bit words per packed element
constexpr uint32_t MASK = (1u << 26) - 1u;

struct fe {
    uint32_t d[N];
};

// radix-2^26 digits of p
__host__ __device__ constexpr uint32_t p26(int i) {
    switch (i) {
        case 0: return 0x1u;
        case 1: return 0x2300000u;
        case 2: return 0x850u;
        case 3: return 0x110c000u;
        case 4: return 0x170b5du;
        case 5: return 0x2825200u;
        case 6: return 0x33622fbu;
        case 7: return 0x4e3c7bu;
        case 8: return 0x1f300f5u;
        case 9: return 0x2c688b6u;
        case 10: return 0x2ca1493u;
        case 11: return 0xec1701u;
        case 12: return 0x110eac6u;
        case 13: return 0x29185f1u;
        default: return 0x1ae3u;
    }
}

// canonical radix-2^26 digit i of K*p (the top digit keeps any carry)
__host__ __device__ constexpr uint32_t kp_digit(int K, int i) {
    uint64_t c = 0;
    uint32_t out = 0;
    for (int j = 0; j <= i; ++j) {
        uint64_t t = (uint64_t)K * p26(j) + c;
        out = (j == N - 1) ? (uint32_t)t : (uint32_t)(t & MASK);
        c = t >> 26;
    }
    return out;
}

// digit i of K*p in the redundant form used by sub<K>: 2^28 is added to digits
// 0..13 and 4 is borrowed from each next digit (2^28 = 4 * 2^26), value unchanged.
__host__ __device__ constexpr uint32_t sub_digit(int K, int i) {
    return kp_digit(K, i) + (i < N - 1 ? (1u << 28) : 0u) - (i > 0 ? 4u : 0u);
}

// 2^390 mod p (Montgomery one) and 2^780 mod p (to-Montgomery factor), radix 2^26.
__host__ __device__ constexpr uint32_t one26(int i) {
    switch (i) {
        case 0: return 0x3ffd9ebu;
        case 1: return 0x20fffffu;
        case 2: return 0x2c35c9cu;
        case 3: return 0x1203fffu;
        case 4: return 0x26c393au;
        case 5: return 0x3234524u;
        case 6: return 0x35dc785u;
        case 7: return 0x9aa955u;
        case 8: return 0xec8afeu;
        case 9: return 0x16bb283u;
        case 10: return 0x25e6384u;
        case 11: return 0x137dc5cu;
        case 12: return 0x2c350fau;
        case 13: return 0x2e3314u;
        default: return 0xedu;
    }
}

__host__ __device__ constexpr uint32_t r2_26(int i) {
    switch (i) {
        case 0: return 0xd21be9u;
        case 1: return 0x3625003u;
        case 2: return 0x19584fbu;
        case 3: return 0x7fcc6cu;
        case 4: return 0x605039u;
        case 5: return 0x3d455f5u;
        case 6: return 0x2a84fb8u;
        case 7: return 0x30f4b26u;
        case 8: return 0x34ef1e7u;
        case 9: return 0x184d1b5u;
        case 10: return 0x91d1b4u;
        case 11: return 0x329f86du;
        case 12: return 0x58072du;
        case 13: return 0x34f7770u;
        default: return 0x3c5u;
    }
}

__device__ __forceinline__ void set_zero(fe& r) {
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = 0;
}

__device__ __forceinline__ void set_one(fe& r) {
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = one26(k);
}

__device__ __forceinline__ void set_r2(fe& r) {
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = r2_26(k);
}

// Montgomery step i on the column window c[i .. i+15]: column i is complete
// (every a_k b_{i-k} and m_k p_{i-k} with k < i is in), so m_i = -c_i mod 2^26
// zeroes its low 26 bits (p_0 = 1), m_i p_j goes into columns i + j and the
// column's high part carries into column i + 1. Columns below i are dead, so
// only 16 column sums are live at a time.
#define FQ_REDUCE_STEP(c, i)                                                  \
    {                                                                         \
        const uint32_t m_ = (0u - (uint32_t)c[(i)]) & MASK;                   \
        c[(i)] += m_;                                                         \
        _Pragma("unroll") for (int j_ = 1; j_ < N; ++j_) c[(i) + j_] +=       \
            (uint64_t)m_ * p26(j_);                                           \
        c[(i) + 1] += c[(i)] >> 26;                                           \
    }

// Two rounds of coarse carry propagation over the result columns c[N .. 2N-1]
// (Sec. III-D step0 / step1); digits 0..13 end <= 2^26 + 2^10.
#define FQ_FINISH(r, c)                                                                     \
    {                                                                                       \
        uint64_t e_[N];                                                                     \
        e_[0] = c[N] & MASK;                                                                \
        _Pragma("unroll") for (int k_ = 1; k_ < N; ++k_) e_[k_] =                           \
            (c[N + k_] & MASK) + (c[N + k_ - 1] >> 26); /* c[2N-1] = 0 */                  \
        r.d[0] = (uint32_t)e_[0];                                                           \
        _Pragma("unroll") for (int k_ = 1; k_ < N - 1; ++k_) r.d[k_] =                      \
            (uint32_t)((e_[k_] & MASK) + (e_[k_ - 1] >> 26));                               \
        r.d[N - 1] = (uint32_t)(e_[N - 1] + (e_[N - 2] >> 26)); /* value bound: < 2^14 */  \
    }

// r = a * b * 2^-390 mod p, result normal (value < 2p).
__device__ __forceinline__ void mul(fe& r, const fe& a, const fe& b) {
    uint64_t c[2 * N];
#pragma unroll
    for (int k = 0; k < 2 * N; ++k) c[k] = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) c[i + j] += (uint64_t)a.d[i] * b.d[j];
        FQ_REDUCE_STEP(c, i)
    }
    FQ_FINISH(r, c)
}

// r = a^2 * 2^-390 mod p: the symmetric products once, doubled. Row i adds
// a_i^2 and 2 a_i a_j (j > i); column i is complete after row i as in mul().
__device__ __forceinline__ void sqr(fe& r, const fe& a) {
    uint64_t c[2 * N];
#pragma unroll
    for (int k = 0; k < 2 * N; ++k) c[k] = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        c[2 * i] += (uint64_t)a.d[i] * a.d[i];
        const uint32_t a2 = a.d[i] << 1;
#pragma unroll
        for (int j = i + 1; j < N; ++j) c[i + j] += (uint64_t)a2 * a.d[j];
        FQ_REDUCE_STEP(c, i)
    }
    FQ_FINISH(r, c)
}

// r = a + b, digit-wise (no carries).
__device__ __forceinline__ void add(fe& r, const fe& a, const fe& b) {
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
}

// r = a - b + K p, digit-wise. Needs b < (K - 1) p and b's digits 0..13 < 2^28 - 4.
template <int K>
__device__ __forceinline__ void sub(fe& r, const fe& a, const fe& b) {
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + sub_digit(K, k) - b.d[k];
}

// Two rounds of coarse carry propagation (Sec. III-D step0/step1): value unchanged,
// digits 0..13 <= 2^26 afterwards for input digits < 2^31; the top digit keeps its excess.
__device__ __forceinline__ void settle(fe& a) {
    uint32_t t[N];
    t[0] = a.d[0] & MASK;
#pragma unroll
    for (int k = 1; k < N - 1; ++k) t[k] = (a.d[k] & MASK) + (a.d[k - 1] >> 26);
    t[N - 1] = a.d[N - 1] + (a.d[N - 2] >> 26);
    a.d[0] = t[0];
#pragma unroll
    for (int k = 1; k < N - 1; ++k) a.d[k] = (t[k] & MASK) + (t[k - 1] >> 26);
    a.d[N - 1] = t[N - 1] + (t[N - 2] >> 26);
}

// Exact digits (each < 2^26 except the top one) by a serial carry pass.
__device__ __forceinline__ void exact(fe& a) {
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < N - 1; ++k) {
        uint32_t t = a.d[k] + c;
        a.d[k] = t & MASK;
        c = t >> 26;
    }
    a.d[N - 1] += c;
}

// a >= p for exact digits
__device__ __forceinline__ bool geq_p(const fe& a) {
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
        if (a.d[k] != p26(k)) return a.d[k] > p26(k);
    }
    return true;
}

// a -= p for exact digits with a >= p (result exact)
__device__ __forceinline__ void sub_p_exact(fe& a) {
    int32_t borrow = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int32_t t = (int32_t)a.d[k] - (int32_t)p26(k) - borrow;
        borrow = t < 0;
        a.d[k] = (uint32_t)(t + (borrow ? (1 << 26) : 0));
    }
}

// Canonical exact digits in [0, p) from any value < 64 p.
__device__ __forceinline__ void canon(fe& a) {
    exact(a);
    while (geq_p(a)) sub_p_exact(a);
}

// value == 0 mod p, for a normal value (< 2p): exact digits are 0 or p.
__device__ __forceinline__ bool is_zero_normal(fe a) {
    exact(a);
    uint32_t z = 0, q = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        z |= a.d[k];
        q |= a.d[k] ^ p26(k);
    }
    return z == 0 || q == 0;
}

// value == 0 mod p for any value < 64 p (slow path).
__device__ __forceinline__ bool is_zero_any(fe a) {
    canon(a);
    uint32_t z = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) z |= a.d[k];
    return z == 0;
}

__device__ __forceinline__ bool is_zero_raw(const fe& a) {
    uint32_t z = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) z |= a.d[k];
    return z == 0;
}

// ---- packed 12 x 32-bit limbs <-> digits

__device__ __forceinline__ void unpack(fe& r, const uint32_t (&w)[NW]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int bit = 26 * i, k = bit >> 5, off = bit & 31;
        uint32_t lo = w[k] >> off;
        uint32_t hi = (off > 6 && k + 1 < NW) ? (w[k + 1] << (32 - off)) : 0u;
        r.d[i] = (lo | hi) & MASK;
    }
}

// Needs exact digits (< 2^26) and a value < 2^384.
__device__ __forceinline__ void pack(uint32_t (&w)[NW], const fe& a) {
#pragma unroll
    for (int k = 0; k < NW; ++k) w[k] = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int bit = 26 * i, k = bit >> 5, off = bit & 31;
        w[k] |= a.d[i] << off;
        if (off > 6 && k + 1 < NW) w[k + 1] |= a.d[i] >> (32 - off);
    }
}

__device__ __forceinline__ void load_packed(fe& r, const uint32_t* p) {
    uint32_t w[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) w[k] = p[k];
    unpack(r, w);
}

// Stores canonical [0, p) packed limbs.
__device__ __forceinline__ void store_canonical(uint32_t* p, fe a) {
    canon(a);
    uint32_t w[NW];
    pack(w, a);
#pragma unroll
    for (int k = 0; k < NW; ++k) p[k] = w[k];
}

// Strided (structure-of-arrays) packed access: limb k of element i at base[k * stride + i].
__device__ __forceinline__ void load_soa(fe& r, const uint32_t* base, size_t i, size_t stride) {
    uint32_t w[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) w[k] = base[k * stride + i];
    unpack(r, w);
}

__device__ __forceinline__ void store_soa(uint32_t* base, size_t i, size_t stride, fe a) {
    canon(a);
    uint32_t w[NW];
    pack(w, a);
#pragma unroll
    for (int k = 0; k < NW; ++k) base[k * stride + i] = w[k];
}

}  // namespace fq
