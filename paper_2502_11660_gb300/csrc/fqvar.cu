// Alternative Fq multiplications, measured against the library's Montgomery CIOS
// (fq_mul_batch_variant). None of them is used by the MSM; they exist to compare
// the designs the paper uses or proposes with the one this library chose:
//
//  * BARRETT   -- the paper's modular multiplication (Sec. III-C): the 754-bit
//                 product a*b, then Barrett reduction by three multiplications with
//                 k = bitlen(p) = 377, mu = floor(2^754 / p): q1 = x >> (k - 1),
//                 q3 = (q1 mu) >> (k + 1), r = x - q3 p mod 2^(k + 1) in [0, 3p),
//                 then at most two subtractions of p. Standard-form operands.
//  * KARATSUBA -- Montgomery, with a*b by one Karatsuba level over 192-bit halves
//                 and schoolbook leaves (Sec. V-C proposes Karatsuba at the top
//                 level); then word-by-word Montgomery reduction of the 24-word product.
//  * CARRYSAVE -- Montgomery on 16 digits of 24 bits in 32-bit registers, 64-bit
//                 column sums and two rounds of coarse carry propagation (the
//                 element format of Sec. III-B / III-D carried to the GPU).
//  * CIOS_DOUBLEROW -- the library's double-row steps with the plain digit
//                 m = -t (mul_doublerow): the compiler folds that negation into
//                 the m p multiplications, which then do not fuse into 64-bit
//                 multiply-adds (the library negates through a mask it reads
//                 with a volatile load).
//  * CIOS_SINGLEROW -- the library's earlier form: one row and one digit per step
//                 (fq::mul_singlerow_inl).
//  * CIOS_TWOPASS -- the library's word-serial Montgomery product with each row
//                 as one chain of low halves followed by one chain of high halves
//                 (the library's multiplication runs each row as two independent
//                 chains of adjacent low/high halves instead).
//
// Every variant reads 12 x 32-bit limbs in structure-of-arrays layout and writes the
// canonical result in [0, p), so all five are bit-comparable.
#include <cuda_runtime.h>

#include "common.cuh"
#include "wfq.cuh"
#include "fq.cuh"

namespace {

using fq::fe;
constexpr int N = 12;

__device__ __constant__ static const uint32_t kPv[N] = {FQ_P_LIMBS};
// mu = floor(2^754 / p), 378 bits
__device__ __constant__ static const uint32_t kMuB[N] = {
    0x5e4daffcu, 0x1f9fd58cu, 0x89c42a59u, 0xd0ed6877u, 0xd85a6d02u, 0x6af2d488u,
    0x6776b1a0u, 0x3bbad0deu, 0x582ef4f7u, 0x976c3ca0u, 0x0cc4060eu, 0x0261508du};

// acc[0..12] += ai * b[0..11]: low halves at acc[j], high halves at acc[j + 1];
// the final carry lands in acc[12] (the caller bounds the window so none leaves it).
__device__ __forceinline__ void row(uint32_t& t0, uint32_t& t1, uint32_t& t2, uint32_t& t3, uint32_t& t4,
                                    uint32_t& t5, uint32_t& t6, uint32_t& t7, uint32_t& t8, uint32_t& t9,
                                    uint32_t& t10, uint32_t& t11, uint32_t& t12, uint32_t ai, const uint32_t* b) {
    asm("mad.lo.cc.u32 %0, %13, %14, %0;\n\t"
        "madc.lo.cc.u32 %1, %13, %15, %1;\n\t"
        "madc.lo.cc.u32 %2, %13, %16, %2;\n\t"
        "madc.lo.cc.u32 %3, %13, %17, %3;\n\t"
        "madc.lo.cc.u32 %4, %13, %18, %4;\n\t"
        "madc.lo.cc.u32 %5, %13, %19, %5;\n\t"
        "madc.lo.cc.u32 %6, %13, %20, %6;\n\t"
        "madc.lo.cc.u32 %7, %13, %21, %7;\n\t"
        "madc.lo.cc.u32 %8, %13, %22, %8;\n\t"
        "madc.lo.cc.u32 %9, %13, %23, %9;\n\t"
        "madc.lo.cc.u32 %10, %13, %24, %10;\n\t"
        "madc.lo.cc.u32 %11, %13, %25, %11;\n\t"
        "addc.u32 %12, %12, 0;\n\t"
        "mad.hi.cc.u32 %1, %13, %14, %1;\n\t"
        "madc.hi.cc.u32 %2, %13, %15, %2;\n\t"
        "madc.hi.cc.u32 %3, %13, %16, %3;\n\t"
        "madc.hi.cc.u32 %4, %13, %17, %4;\n\t"
        "madc.hi.cc.u32 %5, %13, %18, %5;\n\t"
        "madc.hi.cc.u32 %6, %13, %19, %6;\n\t"
        "madc.hi.cc.u32 %7, %13, %20, %7;\n\t"
        "madc.hi.cc.u32 %8, %13, %21, %8;\n\t"
        "madc.hi.cc.u32 %9, %13, %22, %9;\n\t"
        "madc.hi.cc.u32 %10, %13, %23, %10;\n\t"
        "madc.hi.cc.u32 %11, %13, %24, %11;\n\t"
        "madc.hi.u32 %12, %13, %25, %12;"
        : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8), "+r"(t9),
          "+r"(t10), "+r"(t11), "+r"(t12)
        : "r"(ai), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]),
          "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]));
}

#define ROW_AT(x, i, ai, b)                                                                                  \
    row(x[(i) + 0], x[(i) + 1], x[(i) + 2], x[(i) + 3], x[(i) + 4], x[(i) + 5], x[(i) + 6], x[(i) + 7],      \
        x[(i) + 8], x[(i) + 9], x[(i) + 10], x[(i) + 11], x[(i) + 12], ai, b)

// x[0..23] = a * b (x has 25 words; x[24] stays 0).
__device__ __forceinline__ void mul_wide(uint32_t (&x)[25], const uint32_t* a, const uint32_t* b) {
#pragma unroll
    for (int k = 0; k < 25; ++k) x[k] = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) ROW_AT(x, i, a[i], b);
}

// a - b over n words; returns the borrow.
template <int W>
__device__ __forceinline__ uint32_t sub_words(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    uint32_t borrow = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        uint64_t t = (uint64_t)a[k] - b[k] - borrow;
        r[k] = (uint32_t)t;
        borrow = (uint32_t)(t >> 63);
    }
    return borrow;
}

// r in [0, 2^384) -> r - p while r >= p (at most `times` subtractions)
template <int TIMES>
__device__ __forceinline__ void reduce_p(uint32_t* r) {
#pragma unroll
    for (int s = 0; s < TIMES; ++s) {
        uint32_t d[N];
        const uint32_t borrow = sub_words<N>(d, r, kPv);
        if (!borrow) {
#pragma unroll
            for (int k = 0; k < N; ++k) r[k] = d[k];
        }
    }
}

// ---------------------------------------------------------------- Barrett (Sec. III-C)

__device__ __forceinline__ void mul_barrett(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    uint32_t x[25];
    mul_wide(x, a, b);  // x < p^2 < 2^754
    // q1 = x >> 376: words 11.. shifted by 24 bits (x < 2^754, so q1 < 2^378)
    uint32_t q1[N];
#pragma unroll
    for (int i = 0; i < N; ++i) q1[i] = (x[11 + i] >> 24) | (x[12 + i] << 8);
    // q2 = q1 * mu, q3 = q2 >> 378: words 11.. shifted by 26 bits
    uint32_t q2[25];
    mul_wide(q2, q1, kMuB);
    uint32_t q3[N];
#pragma unroll
    for (int i = 0; i < N; ++i) q3[i] = (q2[11 + i] >> 26) | (q2[12 + i] << 6);
    // r2 = q3 * p mod 2^378 (only the 12 low words are needed)
    uint32_t r2[25];
#pragma unroll
    for (int k = 0; k < 25; ++k) r2[k] = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) ROW_AT(r2, i, q3[i], kPv);
    // r = (x - r2) mod 2^378, in [0, 3p)
    uint32_t rr[N];
    sub_words<N>(rr, x, r2);
    rr[N - 1] &= (1u << 26) - 1u;
    reduce_p<2>(rr);
#pragma unroll
    for (int k = 0; k < N; ++k) r[k] = rr[k];
}

// ---------------------------------------------------------------- Karatsuba + Montgomery

// x[0..12] = a[0..5] * b[0..5] (6 x 6 words; x has 13 words, x[12] = 0)
__device__ __forceinline__ void mul6(uint32_t (&x)[13], const uint32_t* a, const uint32_t* b) {
#pragma unroll
    for (int k = 0; k < 13; ++k) x[k] = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        uint64_t carry = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            uint64_t t = (uint64_t)a[i] * b[j] + x[i + j] + carry;
            x[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        x[i + 6] = (uint32_t)carry;
    }
}

__device__ __forceinline__ void mul_karatsuba(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    // a = a0 + a1 2^192, b = b0 + b1 2^192
    uint32_t z0[13], z2[13], z1[13];
    mul6(z0, a, b);
    mul6(z2, a + 6, b + 6);
    uint32_t sa[6], sb[6];
    uint32_t ca = 0, cb = 0;
    {
        uint64_t c1 = 0, c2 = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            uint64_t t = (uint64_t)a[k] + a[k + 6] + c1;
            sa[k] = (uint32_t)t;
            c1 = t >> 32;
            uint64_t u = (uint64_t)b[k] + b[k + 6] + c2;
            sb[k] = (uint32_t)u;
            c2 = u >> 32;
        }
        ca = (uint32_t)c1;
        cb = (uint32_t)c2;
    }
    mul6(z1, sa, sb);
    // (sa + ca 2^192)(sb + cb 2^192) = sa sb + (ca sb + cb sa) 2^192 + ca cb 2^384
    uint32_t mid[14];
#pragma unroll
    for (int k = 0; k < 13; ++k) mid[k] = z1[k];
    mid[13] = 0;
    {
        uint64_t c = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            uint64_t t = (uint64_t)mid[6 + k] + (ca ? sb[k] : 0u) + (cb ? sa[k] : 0u) + c;
            mid[6 + k] = (uint32_t)t;
            c = t >> 32;
        }
        uint64_t t = (uint64_t)mid[12] + c + (ca & cb);
        mid[12] = (uint32_t)t;
        mid[13] = (uint32_t)(t >> 32);
    }
    // mid -= z0 + z2 (mid >= z0 + z2, the middle Karatsuba term is non-negative)
    {
        uint64_t borrow = 0;
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            uint64_t t = (uint64_t)mid[k] - (k < 13 ? z0[k] : 0u) - (k < 13 ? z2[k] : 0u) - borrow;
            mid[k] = (uint32_t)t;
            borrow = (uint32_t)(0u - (uint32_t)(t >> 32));  // 0, 1 or 2
        }
    }
    // x = z0 + mid 2^192 + z2 2^384 (25 words)
    uint32_t x[26];
#pragma unroll
    for (int k = 0; k < 26; ++k) x[k] = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) x[k] = z0[k];
#pragma unroll
    for (int k = 0; k < 12; ++k) x[12 + k] = z2[k];
    {
        uint64_t c = 0;
#pragma unroll
        for (int k = 0; k < 20; ++k) {
            uint64_t t = (uint64_t)x[6 + k] + (k < 14 ? mid[k] : 0u) + c;
            x[6 + k] = (uint32_t)t;
            c = t >> 32;
        }
    }
    // Montgomery reduction, word by word: m = -x_i (since -p^-1 = 0xffffffff mod 2^32)
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const uint32_t m = 0u - x[i];
        uint32_t top = 0;
        row(x[i + 0], x[i + 1], x[i + 2], x[i + 3], x[i + 4], x[i + 5], x[i + 6], x[i + 7], x[i + 8], x[i + 9],
            x[i + 10], x[i + 11], top, m, kPv);
        // top holds the carry into word i + 12 (< 2^32); add it with a full carry chain
        uint64_t c = top;
#pragma unroll
        for (int k = i + 12; k < 26; ++k) {
            uint64_t t = (uint64_t)x[k] + c;
            x[k] = (uint32_t)t;
            c = t >> 32;
        }
    }
    // result = x >> 384 < 2p
    uint32_t rr[N];
#pragma unroll
    for (int k = 0; k < N; ++k) rr[k] = x[12 + k];
    reduce_p<1>(rr);
#pragma unroll
    for (int k = 0; k < N; ++k) r[k] = rr[k];
}

// ---------------------------------------------------------------- carry-save radix 2^24 Montgomery

constexpr int ND = 16;  // digits of 24 bits
constexpr uint32_t DMASK = (1u << 24) - 1u;

__host__ __device__ constexpr uint32_t pdig(int i) {
    return i == 0 ? 0x1u : i == 1 ? 0xc00000u : i == 2 ? 0x8508u : i == 3 ? 0x300000u : i == 4 ? 0xb5d44u
         : i == 5 ? 0x480017u : i == 6 ? 0x2fba09u : i == 7 ? 0x1ef362u : i == 8 ? 0xf5138fu
         : i == 9 ? 0xd9f300u : i == 10 ? 0x3b1a22u : i == 11 ? 0x6ca149u : i == 12 ? 0x3b05c0u
         : i == 13 ? 0x10eac6u : i == 14 ? 0x4617c5u : 0x1ae3au;
}

__device__ __forceinline__ void unpack24(uint32_t (&d)[ND], const uint32_t* w) {
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const uint32_t w0 = w[3 * g], w1 = w[3 * g + 1], w2 = w[3 * g + 2];
        d[4 * g + 0] = w0 & DMASK;
        d[4 * g + 1] = ((w0 >> 24) | (w1 << 8)) & DMASK;
        d[4 * g + 2] = ((w1 >> 16) | (w2 << 16)) & DMASK;
        d[4 * g + 3] = w2 >> 8;
    }
}

// r = a b 2^-384 mod p on 24-bit digits: row i adds a_i b into 64-bit column sums;
// column i is then complete, m_i = -c_i mod 2^24 (p = 1 mod 2^24) zeroes its low
// 24 bits and m_i p is added the same way; the column's high part carries into
// column i + 1. Two rounds of coarse carries settle the result columns.
__device__ __forceinline__ void mul_carrysave(uint32_t* r, const uint32_t* aw, const uint32_t* bw) {
    uint32_t a[ND], b[ND];
    unpack24(a, aw);
    unpack24(b, bw);
    uint64_t c[2 * ND];
#pragma unroll
    for (int k = 0; k < 2 * ND; ++k) c[k] = 0;
#pragma unroll
    for (int i = 0; i < ND; ++i) {
#pragma unroll
        for (int j = 0; j < ND; ++j) c[i + j] += (uint64_t)a[i] * b[j];
        const uint32_t m = (0u - (uint32_t)c[i]) & DMASK;
        c[i] += m;
#pragma unroll
        for (int j = 1; j < ND; ++j) c[i + j] += (uint64_t)m * pdig(j);
        c[i + 1] += c[i] >> 24;
    }
    // exact digits of the result columns c[16..31] by one serial carry pass
    uint32_t d[ND];
    uint64_t carry = 0;
#pragma unroll
    for (int k = 0; k < ND; ++k) {
        uint64_t t = c[ND + k] + carry;
        d[k] = k < ND - 1 ? (uint32_t)(t & DMASK) : (uint32_t)t;
        carry = t >> 24;
    }
    uint32_t w[N];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        w[3 * g] = d[4 * g] | (d[4 * g + 1] << 24);
        w[3 * g + 1] = (d[4 * g + 1] >> 8) | (d[4 * g + 2] << 16);
        w[3 * g + 2] = (d[4 * g + 2] >> 16) | (d[4 * g + 3] << 8);
    }
    reduce_p<1>(w);
#pragma unroll
    for (int k = 0; k < N; ++k) r[k] = w[k];
}

// CIOS with one low-half chain and one high-half chain per row (the form the
// library used before its even/odd chains): same quotient digits, same lazy result
// in [0, 2p).
__device__ __forceinline__ void mul_cios_twopass(fe& r, const fe& a, const fe& bb) {
    const uint32_t* b = bb.v;
    uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0, t8 = 0, t9 = 0,
             t10 = 0, t11 = 0, t12 = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        asm(
        "mad.lo.cc.u32 %0, %13, %14, %0;\n\t"
        "madc.lo.cc.u32 %1, %13, %15, %1;\n\t"
        "madc.lo.cc.u32 %2, %13, %16, %2;\n\t"
        "madc.lo.cc.u32 %3, %13, %17, %3;\n\t"
        "madc.lo.cc.u32 %4, %13, %18, %4;\n\t"
        "madc.lo.cc.u32 %5, %13, %19, %5;\n\t"
        "madc.lo.cc.u32 %6, %13, %20, %6;\n\t"
        "madc.lo.cc.u32 %7, %13, %21, %7;\n\t"
        "madc.lo.cc.u32 %8, %13, %22, %8;\n\t"
        "madc.lo.cc.u32 %9, %13, %23, %9;\n\t"
        "madc.lo.cc.u32 %10, %13, %24, %10;\n\t"
        "madc.lo.cc.u32 %11, %13, %25, %11;\n\t"
        "addc.u32 %12, %12, 0;\n\t"
        "mad.hi.cc.u32 %1, %13, %14, %1;\n\t"
        "madc.hi.cc.u32 %2, %13, %15, %2;\n\t"
        "madc.hi.cc.u32 %3, %13, %16, %3;\n\t"
        "madc.hi.cc.u32 %4, %13, %17, %4;\n\t"
        "madc.hi.cc.u32 %5, %13, %18, %5;\n\t"
        "madc.hi.cc.u32 %6, %13, %19, %6;\n\t"
        "madc.hi.cc.u32 %7, %13, %20, %7;\n\t"
        "madc.hi.cc.u32 %8, %13, %21, %8;\n\t"
        "madc.hi.cc.u32 %9, %13, %22, %9;\n\t"
        "madc.hi.cc.u32 %10, %13, %23, %10;\n\t"
        "madc.hi.cc.u32 %11, %13, %24, %11;\n\t"
        "madc.hi.u32 %12, %13, %25, %12;"
            : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8), "+r"(t9), "+r"(t10), "+r"(t11), "+r"(t12)
            : "r"(a.v[i]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]));
        uint32_t m = 0u - t0;
        asm(
        "add.cc.u32 %0, %0, %13;\n\t"
        "madc.lo.cc.u32 %1, %13, 0x8508c000, %1;\n\t"
        "madc.lo.cc.u32 %2, %13, 0x30000000, %2;\n\t"
        "madc.lo.cc.u32 %3, %13, 0x170b5d44, %3;\n\t"
        "madc.lo.cc.u32 %4, %13, 0xba094800, %4;\n\t"
        "madc.lo.cc.u32 %5, %13, 0x1ef3622f, %5;\n\t"
        "madc.lo.cc.u32 %6, %13, 0x00f5138f, %6;\n\t"
        "madc.lo.cc.u32 %7, %13, 0x1a22d9f3, %7;\n\t"
        "madc.lo.cc.u32 %8, %13, 0x6ca1493b, %8;\n\t"
        "madc.lo.cc.u32 %9, %13, 0xc63b05c0, %9;\n\t"
        "madc.lo.cc.u32 %10, %13, 0x17c510ea, %10;\n\t"
        "madc.lo.cc.u32 %11, %13, 0x01ae3a46, %11;\n\t"
        "addc.u32 %12, %12, 0;\n\t"
        "mad.hi.cc.u32 %2, %13, 0x8508c000, %2;\n\t"
        "madc.hi.cc.u32 %3, %13, 0x30000000, %3;\n\t"
        "madc.hi.cc.u32 %4, %13, 0x170b5d44, %4;\n\t"
        "madc.hi.cc.u32 %5, %13, 0xba094800, %5;\n\t"
        "madc.hi.cc.u32 %6, %13, 0x1ef3622f, %6;\n\t"
        "madc.hi.cc.u32 %7, %13, 0x00f5138f, %7;\n\t"
        "madc.hi.cc.u32 %8, %13, 0x1a22d9f3, %8;\n\t"
        "madc.hi.cc.u32 %9, %13, 0x6ca1493b, %9;\n\t"
        "madc.hi.cc.u32 %10, %13, 0xc63b05c0, %10;\n\t"
        "madc.hi.cc.u32 %11, %13, 0x17c510ea, %11;\n\t"
        "madc.hi.u32 %12, %13, 0x01ae3a46, %12;"
            : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8), "+r"(t9), "+r"(t10), "+r"(t11), "+r"(t12)
            : "r"(m));
        t0 = t1; t1 = t2; t2 = t3; t3 = t4; t4 = t5; t5 = t6; t6 = t7; t7 = t8; t8 = t9;
        t9 = t10; t10 = t11; t11 = t12; t12 = 0;
    }
    r.v[0] = t0; r.v[1] = t1; r.v[2] = t2; r.v[3] = t3; r.v[4] = t4; r.v[5] = t5;
    r.v[6] = t6; r.v[7] = t7; r.v[8] = t8; r.v[9] = t9; r.v[10] = t10; r.v[11] = t11;
}

// ---- CIOS_DOUBLEROW: two rows and two quotient digits per step, accumulators
// shifted by two limbs, so the register pair holding the low and high half of one
// partial product keeps its alignment from step to step; here with the digits
// formed as plain negations, which the compiler folds into the m p products (they
// then split into a low and a high multiply). fq::mont_dstep is the same step with
// the digits formed through an opaque all-ones mask.
//
// The running value is E + 2^32 O: E[k] at limb k holds the partial products that
// start at an even limb (a low half at 2j, its high half at 2j + 1), O[k] at limb
// k + 1 those that start at an odd limb. One step, for x0 = a_2s, x1 = a_2s+1:
//   E += x0 b_even,  O += x0 b_odd,  O += x1 b_even,  E += 2^64 x1 b_odd (E[2..]),
//   m0 = -E[0];  O += m0 p_odd;  E += m0 p_even, where p_0 = 1 leaves the high
//   half of m0 p_0 zero and that slot adds O[0] (so limb 1 is held by E alone);
//   m1 = -E[1];  E += 2^32 m1 (at limb 1) + 2^64 m1 p_odd (E[2..]);
//   O += m1 p_even without its p_0 term (O[2..], limbs 3 up);
//   then O[1] (limb 2) and the carry of limb 1 move into E, E[0] = E[1] = 0, and
//   both accumulators drop two limbs.
// The quotient digits are those of the word-serial form (the pair (m0, m1) is the
// two-limb digit -t p^-1 mod 2^64), so the lazy result in [0, 2p) is the same.
// Bounds: E stays below 2^444 and O below 2^413 within a step, so E[0..13] and
// O[0..13] hold them and the top carries are zero.
struct MontAcc2 {
    uint32_t e[14], o[14];
};

__device__ __forceinline__ void mont_step2(MontAcc2& t, uint32_t x0, uint32_t x1, const uint32_t* b) {
    uint32_t* E = t.e;
    uint32_t* O = t.o;
    // E[0..11] += x0 b_even, carry into E[12..13]
    asm("mad.lo.cc.u32 %0, %14, %15, %0;\n\t"
        "madc.hi.cc.u32 %1, %14, %15, %1;\n\t"
        "madc.lo.cc.u32 %2, %14, %16, %2;\n\t"
        "madc.hi.cc.u32 %3, %14, %16, %3;\n\t"
        "madc.lo.cc.u32 %4, %14, %17, %4;\n\t"
        "madc.hi.cc.u32 %5, %14, %17, %5;\n\t"
        "madc.lo.cc.u32 %6, %14, %18, %6;\n\t"
        "madc.hi.cc.u32 %7, %14, %18, %7;\n\t"
        "madc.lo.cc.u32 %8, %14, %19, %8;\n\t"
        "madc.hi.cc.u32 %9, %14, %19, %9;\n\t"
        "madc.lo.cc.u32 %10, %14, %20, %10;\n\t"
        "madc.hi.cc.u32 %11, %14, %20, %11;\n\t"
        "addc.cc.u32 %12, %12, 0;\n\t"
        "addc.u32 %13, %13, 0;"
        : "+r"(E[0]), "+r"(E[1]), "+r"(E[2]), "+r"(E[3]), "+r"(E[4]), "+r"(E[5]), "+r"(E[6]), "+r"(E[7]),
          "+r"(E[8]), "+r"(E[9]), "+r"(E[10]), "+r"(E[11]), "+r"(E[12]), "+r"(E[13])
        : "r"(x0), "r"(b[0]), "r"(b[2]), "r"(b[4]), "r"(b[6]), "r"(b[8]), "r"(b[10]));
    // O[0..11] += x0 b_odd, carry into O[12..13]
    asm("mad.lo.cc.u32 %0, %14, %15, %0;\n\t"
        "madc.hi.cc.u32 %1, %14, %15, %1;\n\t"
        "madc.lo.cc.u32 %2, %14, %16, %2;\n\t"
        "madc.hi.cc.u32 %3, %14, %16, %3;\n\t"
        "madc.lo.cc.u32 %4, %14, %17, %4;\n\t"
        "madc.hi.cc.u32 %5, %14, %17, %5;\n\t"
        "madc.lo.cc.u32 %6, %14, %18, %6;\n\t"
        "madc.hi.cc.u32 %7, %14, %18, %7;\n\t"
        "madc.lo.cc.u32 %8, %14, %19, %8;\n\t"
        "madc.hi.cc.u32 %9, %14, %19, %9;\n\t"
        "madc.lo.cc.u32 %10, %14, %20, %10;\n\t"
        "madc.hi.cc.u32 %11, %14, %20, %11;\n\t"
        "addc.cc.u32 %12, %12, 0;\n\t"
        "addc.u32 %13, %13, 0;"
        : "+r"(O[0]), "+r"(O[1]), "+r"(O[2]), "+r"(O[3]), "+r"(O[4]), "+r"(O[5]), "+r"(O[6]), "+r"(O[7]),
          "+r"(O[8]), "+r"(O[9]), "+r"(O[10]), "+r"(O[11]), "+r"(O[12]), "+r"(O[13])
        : "r"(x0), "r"(b[1]), "r"(b[3]), "r"(b[5]), "r"(b[7]), "r"(b[9]), "r"(b[11]));
    // O[0..11] += x1 b_even (limbs 1..12), carry into O[12..13]
    asm("mad.lo.cc.u32 %0, %14, %15, %0;\n\t"
        "madc.hi.cc.u32 %1, %14, %15, %1;\n\t"
        "madc.lo.cc.u32 %2, %14, %16, %2;\n\t"
        "madc.hi.cc.u32 %3, %14, %16, %3;\n\t"
        "madc.lo.cc.u32 %4, %14, %17, %4;\n\t"
        "madc.hi.cc.u32 %5, %14, %17, %5;\n\t"
        "madc.lo.cc.u32 %6, %14, %18, %6;\n\t"
        "madc.hi.cc.u32 %7, %14, %18, %7;\n\t"
        "madc.lo.cc.u32 %8, %14, %19, %8;\n\t"
        "madc.hi.cc.u32 %9, %14, %19, %9;\n\t"
        "madc.lo.cc.u32 %10, %14, %20, %10;\n\t"
        "madc.hi.cc.u32 %11, %14, %20, %11;\n\t"
        "addc.cc.u32 %12, %12, 0;\n\t"
        "addc.u32 %13, %13, 0;"
        : "+r"(O[0]), "+r"(O[1]), "+r"(O[2]), "+r"(O[3]), "+r"(O[4]), "+r"(O[5]), "+r"(O[6]), "+r"(O[7]),
          "+r"(O[8]), "+r"(O[9]), "+r"(O[10]), "+r"(O[11]), "+r"(O[12]), "+r"(O[13])
        : "r"(x1), "r"(b[0]), "r"(b[2]), "r"(b[4]), "r"(b[6]), "r"(b[8]), "r"(b[10]));
    // E[2..13] += x1 b_odd (limbs 2..13); no carry leaves E[13]
    asm("mad.lo.cc.u32 %0, %12, %13, %0;\n\t"
        "madc.hi.cc.u32 %1, %12, %13, %1;\n\t"
        "madc.lo.cc.u32 %2, %12, %14, %2;\n\t"
        "madc.hi.cc.u32 %3, %12, %14, %3;\n\t"
        "madc.lo.cc.u32 %4, %12, %15, %4;\n\t"
        "madc.hi.cc.u32 %5, %12, %15, %5;\n\t"
        "madc.lo.cc.u32 %6, %12, %16, %6;\n\t"
        "madc.hi.cc.u32 %7, %12, %16, %7;\n\t"
        "madc.lo.cc.u32 %8, %12, %17, %8;\n\t"
        "madc.hi.cc.u32 %9, %12, %17, %9;\n\t"
        "madc.lo.cc.u32 %10, %12, %18, %10;\n\t"
        "madc.hi.u32 %11, %12, %18, %11;"
        : "+r"(E[2]), "+r"(E[3]), "+r"(E[4]), "+r"(E[5]), "+r"(E[6]), "+r"(E[7]), "+r"(E[8]), "+r"(E[9]),
          "+r"(E[10]), "+r"(E[11]), "+r"(E[12]), "+r"(E[13])
        : "r"(x1), "r"(b[1]), "r"(b[3]), "r"(b[5]), "r"(b[7]), "r"(b[9]), "r"(b[11]));
    const uint32_t m0 = 0u - E[0];
    // O[0..11] += m0 p_odd (limbs 1..12), carry into O[12..13]
    asm("mad.lo.cc.u32 %0, %14, 0x8508c000, %0;\n\t"
        "madc.hi.cc.u32 %1, %14, 0x8508c000, %1;\n\t"
        "madc.lo.cc.u32 %2, %14, 0x170b5d44, %2;\n\t"
        "madc.hi.cc.u32 %3, %14, 0x170b5d44, %3;\n\t"
        "madc.lo.cc.u32 %4, %14, 0x1ef3622f, %4;\n\t"
        "madc.hi.cc.u32 %5, %14, 0x1ef3622f, %5;\n\t"
        "madc.lo.cc.u32 %6, %14, 0x1a22d9f3, %6;\n\t"
        "madc.hi.cc.u32 %7, %14, 0x1a22d9f3, %7;\n\t"
        "madc.lo.cc.u32 %8, %14, 0xc63b05c0, %8;\n\t"
        "madc.hi.cc.u32 %9, %14, 0xc63b05c0, %9;\n\t"
        "madc.lo.cc.u32 %10, %14, 0x01ae3a46, %10;\n\t"
        "madc.hi.cc.u32 %11, %14, 0x01ae3a46, %11;\n\t"
        "addc.cc.u32 %12, %12, 0;\n\t"
        "addc.u32 %13, %13, 0;"
        : "+r"(O[0]), "+r"(O[1]), "+r"(O[2]), "+r"(O[3]), "+r"(O[4]), "+r"(O[5]), "+r"(O[6]), "+r"(O[7]),
          "+r"(O[8]), "+r"(O[9]), "+r"(O[10]), "+r"(O[11]), "+r"(O[12]), "+r"(O[13])
        : "r"(m0));
    // E[0..11] += m0 p_even: limb 0 takes m0 (p_0 = 1), limb 1 takes O[0] in the
    // zero high half of m0 p_0; carry into E[12..13]
    asm("add.cc.u32 %0, %0, %15;\n\t"
        "addc.cc.u32 %1, %1, %14;\n\t"
        "madc.lo.cc.u32 %2, %15, 0x30000000, %2;\n\t"
        "madc.hi.cc.u32 %3, %15, 0x30000000, %3;\n\t"
        "madc.lo.cc.u32 %4, %15, 0xba094800, %4;\n\t"
        "madc.hi.cc.u32 %5, %15, 0xba094800, %5;\n\t"
        "madc.lo.cc.u32 %6, %15, 0x00f5138f, %6;\n\t"
        "madc.hi.cc.u32 %7, %15, 0x00f5138f, %7;\n\t"
        "madc.lo.cc.u32 %8, %15, 0x6ca1493b, %8;\n\t"
        "madc.hi.cc.u32 %9, %15, 0x6ca1493b, %9;\n\t"
        "madc.lo.cc.u32 %10, %15, 0x17c510ea, %10;\n\t"
        "madc.hi.cc.u32 %11, %15, 0x17c510ea, %11;\n\t"
        "addc.cc.u32 %12, %12, 0;\n\t"
        "addc.u32 %13, %13, 0;"
        : "+r"(E[0]), "+r"(E[1]), "+r"(E[2]), "+r"(E[3]), "+r"(E[4]), "+r"(E[5]), "+r"(E[6]), "+r"(E[7]),
          "+r"(E[8]), "+r"(E[9]), "+r"(E[10]), "+r"(E[11]), "+r"(E[12]), "+r"(E[13])
        : "r"(O[0]), "r"(m0));
    const uint32_t m1 = 0u - E[1];
    // E[1..13] += m1 (limb 1, p_0 = 1) + 2^64 m1 p_odd (limbs 2..13): E[1] becomes 0
    asm("add.cc.u32 %0, %0, %13;\n\t"
        "madc.lo.cc.u32 %1, %13, 0x8508c000, %1;\n\t"
        "madc.hi.cc.u32 %2, %13, 0x8508c000, %2;\n\t"
        "madc.lo.cc.u32 %3, %13, 0x170b5d44, %3;\n\t"
        "madc.hi.cc.u32 %4, %13, 0x170b5d44, %4;\n\t"
        "madc.lo.cc.u32 %5, %13, 0x1ef3622f, %5;\n\t"
        "madc.hi.cc.u32 %6, %13, 0x1ef3622f, %6;\n\t"
        "madc.lo.cc.u32 %7, %13, 0x1a22d9f3, %7;\n\t"
        "madc.hi.cc.u32 %8, %13, 0x1a22d9f3, %8;\n\t"
        "madc.lo.cc.u32 %9, %13, 0xc63b05c0, %9;\n\t"
        "madc.hi.cc.u32 %10, %13, 0xc63b05c0, %10;\n\t"
        "madc.lo.cc.u32 %11, %13, 0x01ae3a46, %11;\n\t"
        "madc.hi.u32 %12, %13, 0x01ae3a46, %12;"
        : "+r"(E[1]), "+r"(E[2]), "+r"(E[3]), "+r"(E[4]), "+r"(E[5]), "+r"(E[6]), "+r"(E[7]), "+r"(E[8]),
          "+r"(E[9]), "+r"(E[10]), "+r"(E[11]), "+r"(E[12]), "+r"(E[13])
        : "r"(m1));
    // O[2..11] += m1 (p_2 .. p_10) at limbs 3..12, carry into O[12..13]
    asm("mad.lo.cc.u32 %0, %12, 0x30000000, %0;\n\t"
        "madc.hi.cc.u32 %1, %12, 0x30000000, %1;\n\t"
        "madc.lo.cc.u32 %2, %12, 0xba094800, %2;\n\t"
        "madc.hi.cc.u32 %3, %12, 0xba094800, %3;\n\t"
        "madc.lo.cc.u32 %4, %12, 0x00f5138f, %4;\n\t"
        "madc.hi.cc.u32 %5, %12, 0x00f5138f, %5;\n\t"
        "madc.lo.cc.u32 %6, %12, 0x6ca1493b, %6;\n\t"
        "madc.hi.cc.u32 %7, %12, 0x6ca1493b, %7;\n\t"
        "madc.lo.cc.u32 %8, %12, 0x17c510ea, %8;\n\t"
        "madc.hi.cc.u32 %9, %12, 0x17c510ea, %9;\n\t"
        "addc.cc.u32 %10, %10, 0;\n\t"
        "addc.u32 %11, %11, 0;"
        : "+r"(O[2]), "+r"(O[3]), "+r"(O[4]), "+r"(O[5]), "+r"(O[6]), "+r"(O[7]), "+r"(O[8]), "+r"(O[9]),
          "+r"(O[10]), "+r"(O[11]), "+r"(O[12]), "+r"(O[13])
        : "r"(m1));
    // limb 1 is zero overall (E[1] = 0 now; O[0] was added into it); O[1] (limb 2)
    // moves into E[2] with the carry up E
    asm("add.cc.u32 %0, %0, %12;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.cc.u32 %4, %4, 0;\n\t"
        "addc.cc.u32 %5, %5, 0;\n\t"
        "addc.cc.u32 %6, %6, 0;\n\t"
        "addc.cc.u32 %7, %7, 0;\n\t"
        "addc.cc.u32 %8, %8, 0;\n\t"
        "addc.cc.u32 %9, %9, 0;\n\t"
        "addc.cc.u32 %10, %10, 0;\n\t"
        "addc.u32 %11, %11, 0;"
        : "+r"(E[2]), "+r"(E[3]), "+r"(E[4]), "+r"(E[5]), "+r"(E[6]), "+r"(E[7]), "+r"(E[8]), "+r"(E[9]),
          "+r"(E[10]), "+r"(E[11]), "+r"(E[12]), "+r"(E[13])
        : "r"(O[1]));
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        E[k] = E[k + 2];
        O[k] = O[k + 2];
    }
    E[12] = E[13] = 0;
    O[12] = O[13] = 0;
}

__device__ __forceinline__ void mul_doublerow(fe& r, const fe& a, const fe& b) {
    MontAcc2 t = {};
#pragma unroll
    for (int i = 0; i < N; i += 2) mont_step2(t, a.v[i], a.v[i + 1], b.v);
    const uint32_t* e = t.e;
    const uint32_t* o = t.o;
    r.v[0] = e[0];
    asm("add.cc.u32 %0, %11, %22;\n\t"
        "addc.cc.u32 %1, %12, %23;\n\t"
        "addc.cc.u32 %2, %13, %24;\n\t"
        "addc.cc.u32 %3, %14, %25;\n\t"
        "addc.cc.u32 %4, %15, %26;\n\t"
        "addc.cc.u32 %5, %16, %27;\n\t"
        "addc.cc.u32 %6, %17, %28;\n\t"
        "addc.cc.u32 %7, %18, %29;\n\t"
        "addc.cc.u32 %8, %19, %30;\n\t"
        "addc.cc.u32 %9, %20, %31;\n\t"
        "addc.u32 %10, %21, %32;"
        : "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]), "=r"(r.v[6]), "=r"(r.v[7]),
          "=r"(r.v[8]), "=r"(r.v[9]), "=r"(r.v[10]), "=r"(r.v[11])
        : "r"(e[1]), "r"(e[2]), "r"(e[3]), "r"(e[4]), "r"(e[5]), "r"(e[6]), "r"(e[7]), "r"(e[8]), "r"(e[9]),
          "r"(e[10]), "r"(e[11]), "r"(o[0]), "r"(o[1]), "r"(o[2]), "r"(o[3]), "r"(o[4]), "r"(o[5]), "r"(o[6]),
          "r"(o[7]), "r"(o[8]), "r"(o[9]), "r"(o[10]));
}

// ---------------------------------------------------------------- kernel

// Product scanning (column by column) with the Montgomery reduction folded in
// (finely integrated product scanning): column k of a b + m p is summed into one
// three-word accumulator (t0, t1, t2), the quotient digit m_k = -t0 is taken when
// column k < 12 is complete (t0 + m_k p_0 = t0 + m_k = 0 mod 2^32), and columns
// 12..23 give the result words. Every product is added as one low/high pair into
// the same two accumulator words, so each is one wide multiply-add (no product
// lands on a register pair shifted by one limb, as the rows of CIOS do), and the
// modulus limbs are register operands rather than immediates. 144 + 132 products;
// with a b < p R the result is below 2p, as for CIOS.
__device__ __forceinline__ void fips_acc(uint32_t& t0, uint32_t& t1, uint32_t& t2, uint32_t x, uint32_t y) {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(t0), "+r"(t1), "+r"(t2)
        : "r"(x), "r"(y));
}

__device__ __forceinline__ void mul_fips(fe& r, const fe& a, const fe& b) {
    uint32_t p[N], m[N];
#pragma unroll
    for (int j = 0; j < N; ++j) p[j] = fq::kP[j];
    uint32_t t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
#pragma unroll
        for (int i = 0; i <= k; ++i) fips_acc(t0, t1, t2, a.v[i], b.v[k - i]);
#pragma unroll
        for (int i = 0; i < k; ++i) fips_acc(t0, t1, t2, m[i], p[k - i]);
        m[k] = 0u - t0;
        // t0 + m_k p_0 = t0 + m_k = 0 (mod 2^32), carrying 1 unless t0 = 0
        asm("add.cc.u32 %0, %0, %3;\n\t"
            "addc.cc.u32 %1, %1, 0;\n\t"
            "addc.u32 %2, %2, 0;"
            : "+r"(t0), "+r"(t1), "+r"(t2)
            : "r"(m[k]));
        t0 = t1;
        t1 = t2;
        t2 = 0;
    }
#pragma unroll
    for (int k = N; k < 2 * N - 1; ++k) {
#pragma unroll
        for (int i = k - N + 1; i < N; ++i) fips_acc(t0, t1, t2, a.v[i], b.v[k - i]);
#pragma unroll
        for (int i = k - N + 1; i < N; ++i) fips_acc(t0, t1, t2, m[i], p[k - i]);
        r.v[k - N] = t0;
        t0 = t1;
        t1 = t2;
        t2 = 0;
    }
    r.v[N - 1] = t0;
}

template <int V>
__global__ void k_fq_mul_variant(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                                 uint32_t* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t x[N], y[N], r[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            x[k] = a[k * n + i];
            y[k] = b[k * n + i];
        }
        if (V == MSM377_FQMUL_CIOS || V == MSM377_FQMUL_FIPS || V == MSM377_FQMUL_CIOS_SINGLEROW) {
            fe fa, fb, fr;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                fa.v[k] = x[k];
                fb.v[k] = y[k];
            }
            if (V == MSM377_FQMUL_FIPS)
                mul_fips(fr, fa, fb);
            else if (V == MSM377_FQMUL_CIOS_SINGLEROW)
                fq::mul_singlerow_inl(fr, fa, fb);
            else
                fq::mul_inl(fr, fa, fb);
            fq::canon(fr, fr);
#pragma unroll
            for (int k = 0; k < N; ++k) r[k] = fr.v[k];
        } else if (V == MSM377_FQMUL_CIOS_DOUBLEROW) {
            fe fa, fb, fr;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                fa.v[k] = x[k];
                fb.v[k] = y[k];
            }
            mul_doublerow(fr, fa, fb);
            fq::canon(fr, fr);
#pragma unroll
            for (int k = 0; k < N; ++k) r[k] = fr.v[k];
        } else if (V == MSM377_FQMUL_CIOS_TWOPASS) {
            fe fa, fb, fr;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                fa.v[k] = x[k];
                fb.v[k] = y[k];
            }
            mul_cios_twopass(fr, fa, fb);
            fq::canon(fr, fr);
#pragma unroll
            for (int k = 0; k < N; ++k) r[k] = fr.v[k];
        } else if (V == MSM377_FQMUL_BARRETT) {
            mul_barrett(r, x, y);
        } else if (V == MSM377_FQMUL_KARATSUBA) {
            mul_karatsuba(r, x, y);
        } else {
            mul_carrysave(r, x, y);
        }
#pragma unroll
        for (int k = 0; k < N; ++k) out[k * n + i] = r[k];
    }
}

// ---- the paper's own format (Sec. III-B .. III-E): 16 elements of 25 bits in 32-bit
// registers, schoolbook products summed per column, the two-round coarse carry, and
// the looser Barrett step for operands below 6p (k = 378): q1 = x >> 377,
// mu = floor(2^756 / p), q3 = (q1 mu) >> 379, r = (x - q3 p) mod 2^379, which lies
// in [0, 4p) (for operands below 6p the error bound is 3.33 p on this p).
constexpr int kEl = 16;
constexpr uint32_t kMask25 = 0x1ffffffu;
__device__ __constant__ static const uint32_t kPEl[kEl] = {
    0x0000001u, 0x0600000u, 0x0002142u, 0x0860000u, 0x170b5d4u, 0x04a4000u, 0x188bee8u, 0x11e3de6u,
    0x100f513u, 0x1116cf9u, 0x0524ec6u, 0x0b80d94u, 0x0ac63b0u, 0x0be2887u, 0x0b8e918u, 0x0000003u};
__device__ __constant__ static const uint32_t kMuEl[kEl] = {   // floor(2^756 / p), 380 bits
    0x136bff3u, 0x1ab18bcu, 0x0591f9fu, 0x1c4e215u, 0x03b5a1du, 0x14da05au, 0x1488d85u, 0x1035796u,
    0x19ddac6u, 0x175a1bcu, 0x0f4f73bu, 0x0502c17u, 0x1a5db0fu, 0x19880c1u, 0x01508d0u, 0x0000013u};

// 12 x 32-bit words -> 16 x 25-bit elements (values below 2^400)
__device__ __forceinline__ void to_el(uint32_t (&e)[kEl], const uint32_t (&w)[N]) {
#pragma unroll
    for (int i = 0; i < kEl; ++i) {
        const int bit = 25 * i, word = bit >> 5, off = bit & 31;
        uint32_t v = w[word] >> off;
        if (off > 7 && word + 1 < N) v |= w[word + 1] << (32 - off);
        e[i] = v & kMask25;
    }
}

// Column sums of x y: c[k] = sum_{i + j = k} x_i y_j (each product < 2^52 with
// elements below 2^26, at most 16 per column: below 2^56).
template <int NC>
__device__ __forceinline__ void el_columns(uint64_t (&c)[NC], const uint32_t (&x)[kEl], const uint32_t (&y)[kEl]) {
#pragma unroll
    for (int k = 0; k < NC; ++k) c[k] = 0;
#pragma unroll
    for (int i = 0; i < kEl; ++i)
#pragma unroll
        for (int j = 0; j < kEl; ++j)
            if (i + j < NC) c[i + j] += (uint64_t)x[i] * y[j];
}

// Sec. III-D coarse carry, two rounds over the whole column vector: o = in & 0x1ffffff
// (taken as in - ((in >> 25) << 25), as on the AIE), c = in >> 25, o += carry of the
// element below. Afterwards every element is below 2^26 (the value is unchanged; the
// carry out of the top element is dropped, the caller's width covers the value).
template <int NC>
__device__ __forceinline__ void coarse_carry(uint64_t (&c)[NC]) {
#pragma unroll
    for (int round = 0; round < 2; ++round) {
        uint64_t carry = 0;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const uint64_t hi = c[k] >> 25;
            c[k] = c[k] - (hi << 25) + carry;
            carry = hi;
        }
    }
}

// Accurate carry propagation: every element below 2^25.
template <int NC>
__device__ __forceinline__ void exact_carry(uint64_t (&c)[NC]) {
    uint64_t carry = 0;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const uint64_t v = c[k] + carry;
        c[k] = v & kMask25;
        carry = v >> 25;
    }
}

// Elements lo .. lo + 15 of v >> (25 lo + s) for 0 < s < 25 (v normalised).
template <int NC>
__device__ __forceinline__ void el_shift(uint32_t (&q)[kEl], const uint64_t (&v)[NC], int lo, int s) {
#pragma unroll
    for (int i = 0; i < kEl; ++i) {
        const uint32_t a = lo + i < NC ? (uint32_t)v[lo + i] : 0u;
        const uint32_t b = lo + i + 1 < NC ? (uint32_t)v[lo + i + 1] : 0u;
        q[i] = ((a >> s) | (b << (25 - s))) & kMask25;
    }
}

__device__ __forceinline__ void mul_paper25(uint32_t (&r)[N], const uint32_t (&aw)[N], const uint32_t (&bw)[N]) {
    uint32_t a[kEl], b[kEl], q[kEl], mu[kEl], pe[kEl];
    to_el(a, aw);
    to_el(b, bw);
#pragma unroll
    for (int i = 0; i < kEl; ++i) {
        mu[i] = kMuEl[i];
        pe[i] = kPEl[i];
    }
    uint64_t x[31];
    el_columns(x, a, b);                  // mul_in: x = a b < 36 p^2 < 2^759
    coarse_carry(x);
    exact_carry(x);                       // the MSBs must be exact for q1
    el_shift(q, x, 15, 2);                // q1 = x >> 377
    uint64_t y[31];
    el_columns(y, q, mu);                 // mul_mu
    coarse_carry(y);
    exact_carry(y);
    el_shift(q, y, 15, 4);                // q3 = (q1 mu) >> 379
    uint64_t z[kEl];
    el_columns(z, q, pe);                 // mul_m, low 400 bits only
    coarse_carry(z);
    exact_carry(z);
    // r = (x - q3 p) mod 2^379: 25-bit elements with a borrow, top element 4 bits
    uint32_t re[kEl];
    int64_t borrow = 0;
#pragma unroll
    for (int k = 0; k < kEl; ++k) {
        const int64_t d = (int64_t)x[k] - (int64_t)z[k] - borrow;
        borrow = d < 0 ? 1 : 0;
        re[k] = (uint32_t)(d + (borrow << 25)) & kMask25;
    }
    re[kEl - 1] &= 0xfu;                  // bits 375..378
#pragma unroll
    for (int w = 0; w < N; ++w) r[w] = 0;
#pragma unroll
    for (int i = 0; i < kEl; ++i) {
        const int bit = 25 * i, word = bit >> 5, off = bit & 31;
        r[word] |= re[i] << off;
        if (off > 7 && word + 1 < N) r[word + 1] |= re[i] >> (32 - off);
    }
}

__global__ void k_fq_mul_paper25(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                                 uint32_t* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t x[N], y[N], r[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            x[k] = a[k * n + i];
            y[k] = b[k * n + i];
        }
        mul_paper25(r, x, y);
#pragma unroll
        for (int k = 0; k < N; ++k) out[k * n + i] = r[k];
    }
}

// One warp per product (the chains' latency form, wfq.cuh): lanes hold the limbs,
// three column products and warp-wide carry resolution. Operands below 8p.
__global__ void __launch_bounds__(128) k_fq_mul_warp(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                                                     uint32_t* __restrict__ out, size_t n) {
    __shared__ __align__(16) uint32_t scratch[4 * wfq::kScratchWords];
    wfq::Consts K;
    wfq::init(K, scratch + (threadIdx.x >> 5) * wfq::kScratchWords);
    const int l = wfq::lane();
    const size_t warps = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t i = blockIdx.x * (size_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const uint32_t x = l < 12 ? a[(size_t)l * n + i] : 0u;
        const uint32_t y = l < 12 ? b[(size_t)l * n + i] : 0u;
        const uint32_t r = wfq::canon(wfq::mul(x, y, K), K);
        if (l < 12) out[(size_t)l * n + i] = r;
    }
}

}  // namespace

using namespace msm377;

extern "C" int fq_mul_batch_variant(const uint32_t* a, const uint32_t* b, uint32_t* out, size_t n, int variant,
                                    void* stream) {
    if (variant < MSM377_FQMUL_CIOS || variant > MSM377_FQMUL_CIOS_SINGLEROW)
        return set_error(MSM377_EINVAL, "fq_mul_batch_variant: unknown variant %d", variant);
    if (n == 0) return MSM377_OK;
    if (!a || !b || !out) return set_error(MSM377_EINVAL, "fq_mul_batch_variant: NULL pointer");
    cudaStream_t s = as_stream(stream);
    int sms = 0, dev = 0;
    MSM_CUDA_TRY(cudaGetDevice(&dev));
    MSM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    size_t blocks = (n + 255) / 256;
    const size_t cap = (size_t)sms * 16;
    if (blocks > cap) blocks = cap;
    switch (variant) {
        case MSM377_FQMUL_CIOS:
            k_fq_mul_variant<MSM377_FQMUL_CIOS><<<(unsigned)blocks, 256, 0, s>>>(a, b, out, n);
            break;
        case MSM377_FQMUL_BARRETT:
            k_fq_mul_variant<MSM377_FQMUL_BARRETT><<<(unsigned)blocks, 256, 0, s>>>(a, b, out, n);
            break;
        case MSM377_FQMUL_KARATSUBA:
            k_fq_mul_variant<MSM377_FQMUL_KARATSUBA><<<(unsigned)blocks, 256, 0, s>>>(a, b, out, n);
            break;
        case MSM377_FQMUL_CARRYSAVE:
            k_fq_mul_variant<MSM377_FQMUL_CARRYSAVE><<<(unsigned)blocks, 256, 0, s>>>(a, b, out, n);
            break;
        case MSM377_FQMUL_CIOS_TWOPASS:
            k_fq_mul_variant<MSM377_FQMUL_CIOS_TWOPASS><<<(unsigned)blocks, 256, 0, s>>>(a, b, out, n);
            break;
        case MSM377_FQMUL_FIPS:
            k_fq_mul_variant<MSM377_FQMUL_FIPS><<<(unsigned)blocks, 256, 0, s>>>(a, b, out, n);
            break;
        case MSM377_FQMUL_CIOS_SINGLEROW:
            k_fq_mul_variant<MSM377_FQMUL_CIOS_SINGLEROW><<<(unsigned)blocks, 256, 0, s>>>(a, b, out, n);
            break;
        case MSM377_FQMUL_PAPER:
            k_fq_mul_paper25<<<(unsigned)blocks, 256, 0, s>>>(a, b, out, n);
            break;
        case MSM377_FQMUL_WARP: {
            size_t wb = (n + 3) / 4;   // four warps (products) per block
            if (wb > cap * 4) wb = cap * 4;
            k_fq_mul_warp<<<(unsigned)wb, 128, 0, s>>>(a, b, out, n);
            break;
        }
        default:
            k_fq_mul_variant<MSM377_FQMUL_CIOS_DOUBLEROW><<<(unsigned)blocks, 256, 0, s>>>(a, b, out, n);
    }
    note_launches(1);
    return check_launch("fq_mul_batch_variant");
}
