// Fq arithmetic spread over a warp, for latency-bound chains of point operations.
//
// A field element is held by a whole warp: lane j < 12 holds limb j, lanes 12..31
// hold 0. Values are in Montgomery form (x 2^384 mod p), in [0, 2p) as in fq.cuh,
// or a few multiples of p for the unfolded add / subtract that feed products.
//
// Multiplication (Montgomery, R = 2^384) takes three column products instead of
// twelve sequential rows:
//   T = a b,   m = (T mod R) p' mod R  (p' = -p^-1 mod R),   U = (T + m p) / R.
// In a column product lane k (< 24) sums its own column,
//   sum_i lo(x_i y_{k-i}) + sum_i hi(x_i y_{k-1-i}),
// with every limb x_i of the broadcast operand read by all lanes from the warp's
// shared-memory scratch (three 16-byte loads of one address) and y_{k-d} either
// fetched per lane by shuffles (the operand b) or, for the constants p' and p of
// the two reduction products, kept per lane in registers -- so the twelve rows run
// in parallel across lanes and a product costs about thirty shared-memory and
// shuffle operations, the resource the four warps of a group share. The column sums (below 2^37) are then turned into words
// in constant time: after adding the previous column's high part, each lane
// either generates a carry, propagates one (its word is 2^32 - 1) or neither; with
// G and P the warp's ballots of those flags, the carries into the lanes are the
// bits of ((G | P) + G) ^ P (the carry vector of the binary sum (G | P) + G, a
// carry-lookahead adder across the warp). With a, b below 8p, T < 64 p^2 < p R,
// so U < 2p (R / p > 152). Latency: three column products and three carry
// resolutions instead of twelve dependent Montgomery rows on one thread.
#pragma once
#include <stdint.h>

#include "fq.cuh"

namespace wfq {

constexpr unsigned kFull = 0xffffffffu;

// p' = -p^-1 mod 2^384 (so that T + ((T mod R) p' mod R) p = 0 mod R).
__device__ __constant__ static const uint32_t kPInvNeg[12] = {
    0xffffffffu, 0x8508bfffu, 0xa0000000u, 0xd1e94577u, 0x970debffu, 0x35ed1347u,
    0xcced7a13u, 0x5b245b86u, 0x806a3cecu, 0x22f80141u, 0xeec82e3du, 0xbfa5205fu};

__device__ __forceinline__ int lane() { return threadIdx.x & 31; }

// Words of the per-warp shared-memory scratch a multiplication uses: the broadcast
// operand, T mod R and the quotient m (12 words each, 16-byte aligned).
constexpr int kScratchWords = 36;

// Per-lane values: limb `lane` of p, 2p and 4p, the column operands p_{lane - d} and
// p'_{lane - d} for d = 0..12 (0 outside the twelve limbs), and the shared-memory
// address of this warp's scratch.
struct Consts {
    uint32_t p, p2, p4, p6;
    uint32_t pc[13], qc[13];
    uint32_t scratch;
};

__device__ __forceinline__ uint32_t limb_of(const uint32_t (&c)[12]) {
    const int l = lane();
    return l < 12 ? c[l] : 0u;
}

__device__ __forceinline__ uint32_t normalize(uint32_t lo, uint32_t hi);
__device__ __forceinline__ uint32_t keep12(uint32_t v);

// scratch: this warp's kScratchWords words of shared memory, 16-byte aligned.
__device__ __forceinline__ void init(Consts& K, uint32_t* scratch) {
    const int l = lane();
    K.p = limb_of(fq::kP);
    K.p2 = limb_of(fq::k2P);
    const uint32_t q = limb_of(kPInvNeg);
    // 4p = 2 (2p): limbs of 2p shifted left by one bit across lanes
    const uint32_t below = __shfl_up_sync(kFull, K.p2, 1);
    K.p4 = l < 12 ? (K.p2 << 1) | (l ? below >> 31 : 0u) : 0u;
    {   // 6p = 4p + 2p
        const uint32_t s = K.p4 + K.p2;
        K.p6 = keep12(normalize(s, (uint32_t)(s < K.p4)));
    }
#pragma unroll
    for (int d = 0; d < 13; ++d) {
        K.pc[d] = __shfl_sync(kFull, K.p, (l - d) & 31);   // negative sources wrap to lanes >= 20: zero
        K.qc[d] = __shfl_sync(kFull, q, (l - d) & 31);
    }
    K.scratch = (uint32_t)__cvta_generic_to_shared(scratch);
}

// All twelve limbs of a distributed value in every lane, through the scratch slot
// at byte offset `off` (written by lanes 0..11, then three 16-byte broadcast loads).
__device__ __forceinline__ void broadcast(uint32_t (&x)[12], uint32_t v, const Consts& K, int off) {
    const uint32_t a = K.scratch + off;
    __syncwarp();                                   // earlier readers of the slot are done
    if (lane() < 12) asm volatile("st.shared.u32 [%0], %1;" ::"r"(a + 4 * lane()), "r"(v) : "memory");
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 3; ++q)
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(x[4 * q]), "=r"(x[4 * q + 1]), "=r"(x[4 * q + 2]), "=r"(x[4 * q + 3])
                     : "r"(a + 16 * q)
                     : "memory");
}

// y[d] = y_{lane - d} for d = 0..12 (y distributed; lanes past the twelve limbs and
// negative indices, which wrap to lanes 20..31, read 0).
__device__ __forceinline__ void spread(uint32_t y, uint32_t (&yc)[13]) {
    const int l = lane();
#pragma unroll
    for (int d = 0; d < 13; ++d) yc[d] = __shfl_sync(kFull, y, (l - d) & 31);
}

// Lane k: sum_i lo(x_i y[i]) + hi(x_i y[i + 1]) for y[d] = y_{k-d}, as lo + 2^32 hi
// (x in every lane's registers).
__device__ __forceinline__ void columns(const uint32_t (&x)[12], const uint32_t (&y)[13], uint32_t& lo,
                                        uint32_t& hi) {
    uint64_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
    for (int i = 0; i < 12; i += 2) {
        s0 += x[i] * y[i];
        s1 += __umulhi(x[i], y[i + 1]);
        s2 += x[i + 1] * y[i + 1];
        s3 += __umulhi(x[i + 1], y[i + 2]);
    }
    const uint64_t s = (s0 + s1) + (s2 + s3);
    lo = (uint32_t)s;
    hi = (uint32_t)(s >> 32);
}

// s + (carry into this lane), where `gen` says this lane's own addition overflowed
// (then s != 2^32 - 1) and a lane with s = 2^32 - 1 passes an incoming carry on.
__device__ __forceinline__ uint32_t propagate(uint32_t s, bool gen) {
    const uint32_t G = __ballot_sync(kFull, gen);
    const uint32_t P = __ballot_sync(kFull, s == 0xffffffffu);
    const uint32_t C = ((G | P) + G) ^ P;
    return s + ((C >> lane()) & 1u);
}

// Words of sum_k (lo_k + 2^32 hi_k) 2^(32 k) (hi_k small).
__device__ __forceinline__ uint32_t normalize(uint32_t lo, uint32_t hi) {
    uint32_t h = __shfl_up_sync(kFull, hi, 1);
    if (lane() == 0) h = 0;
    const uint32_t s = lo + h;
    return propagate(s, s < lo);
}

__device__ __forceinline__ uint32_t keep12(uint32_t v) { return lane() < 12 ? v : 0u; }

// a b R^-1 mod p in [0, 2p) for a, b below 8p (distributed).
__device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b, const Consts& K) {
    uint32_t x[12], yc[13], lo, hi;
    spread(b, yc);
    broadcast(x, a, K, 0);
    columns(x, yc, lo, hi);
    const uint32_t t = normalize(lo, hi);           // T, lanes 0..23
    broadcast(x, keep12(t), K, 48);
    columns(x, K.qc, lo, hi);
    const uint32_t m = keep12(normalize(lo, hi));   // T p' mod R
    broadcast(x, m, K, 96);
    columns(x, K.pc, lo, hi);
    const uint64_t v = (uint64_t)lo + t;            // + T
    const uint32_t u = normalize((uint32_t)v, hi + (uint32_t)(v >> 32));
    return keep12(__shfl_down_sync(kFull, u, 12));  // (T + m p) / R
}

// a + b (no reduction; for values that feed products).
__device__ __forceinline__ uint32_t add_nr(uint32_t a, uint32_t b) {
    const uint32_t s = a + b;
    return keep12(normalize(s, (uint32_t)(s < a)));
}

// a - b + K p with K p given per lane (kp = K.p2 or K.p4): a + kp + (2^384 - 1 - b) + 1
// taken mod 2^384 (needs b <= a + K p).
__device__ __forceinline__ uint32_t sub_kp(uint32_t a, uint32_t b, uint32_t kp) {
    const int l = lane();
    const uint64_t v = (uint64_t)a + kp + (l < 12 ? ~b : 0u) + (l == 0 ? 1u : 0u);
    return keep12(normalize((uint32_t)v, (uint32_t)(v >> 32)));
}

// sum of the P positive terms - sum of the Q negative terms + k p (kp = k p's limb
// `lane`), with one carry resolution: each subtraction is a two's complement over
// the twelve limbs, so the per-lane sum stays below 2^35 and its high part flows up.
// Needs the result to be non-negative (the caller's k p covers the negative terms).
template <int P, int Q>
__device__ __forceinline__ uint32_t lincomb(const uint32_t (&pos)[P], const uint32_t (&neg)[Q], uint32_t kp) {
    const int l = lane();
    uint64_t v = (uint64_t)kp + (l == 0 ? (uint32_t)Q : 0u);
#pragma unroll
    for (int i = 0; i < P; ++i) v += pos[i];
#pragma unroll
    for (int i = 0; i < Q; ++i) v += l < 12 ? ~neg[i] : 0u;
    return keep12(normalize((uint32_t)v, (uint32_t)(v >> 32)));
}

__device__ __forceinline__ uint32_t sub_nr2(uint32_t a, uint32_t b, const Consts& K) { return sub_kp(a, b, K.p2); }
__device__ __forceinline__ uint32_t sub_nr4(uint32_t a, uint32_t b, const Consts& K) { return sub_kp(a, b, K.p4); }

// Folded forms for [0, 2p) operands and results. The two candidates are formed in
// parallel; word 12 of the 13-word sum says which one is in range.
__device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b, const Consts& K) {
    const int l = lane();
    const uint32_t s = a + b;
    const uint32_t sum = normalize(s, (uint32_t)(s < a));                 // a + b
    const uint64_t v = (uint64_t)a + b + (l < 12 ? ~K.p2 : 0u) + (l == 0 ? 1u : 0u);
    const uint32_t red = normalize((uint32_t)v, (uint32_t)(v >> 32));    // a + b - 2p + 2^384
    const bool ge = __shfl_sync(kFull, red, 12) != 0;                     // a + b >= 2p
    return keep12(ge ? red : sum);
}

__device__ __forceinline__ uint32_t sub(uint32_t a, uint32_t b, const Consts& K) {
    const int l = lane();
    const uint64_t v = (uint64_t)a + (l < 12 ? ~b : 0u) + (l == 0 ? 1u : 0u);
    const uint32_t d = normalize((uint32_t)v, (uint32_t)(v >> 32));      // a - b + 2^384
    const uint32_t e = sub_kp(a, b, K.p2);                                // a - b + 2p
    const bool ge = __shfl_sync(kFull, d, 12) != 0;                       // a >= b
    return keep12(ge ? d : e);
}

// [0, 2p) -> [0, p).
__device__ __forceinline__ uint32_t canon(uint32_t x, const Consts& K) {
    const int l = lane();
    const uint64_t v = (uint64_t)x + (l < 12 ? ~K.p : 0u) + (l == 0 ? 1u : 0u);
    const uint32_t d = normalize((uint32_t)v, (uint32_t)(v >> 32));      // x - p + 2^384
    return keep12(__shfl_sync(kFull, d, 12) != 0 ? d : x);
}

// x in [0, 2p) is zero mod p (x = 0 or x = p); the same answer in every lane.
__device__ __forceinline__ bool is_zero(uint32_t x, const Consts& K) {
    const int l = lane();
    const uint32_t nz = __ballot_sync(kFull, l < 12 && x != 0u);
    const uint32_t np = __ballot_sync(kFull, l < 12 && x != K.p);
    return nz == 0u || np == 0u;
}

// Every limb zero (a raw all-zero value in memory).
__device__ __forceinline__ bool is_zero_raw(uint32_t x) { return __ballot_sync(kFull, lane() < 12 && x != 0u) == 0u; }

// A 12-word slot (shared or global memory): lane j < 12 takes word j.
__device__ __forceinline__ uint32_t load(const uint32_t* slot) { return lane() < 12 ? slot[lane()] : 0u; }
__device__ __forceinline__ void store(uint32_t* slot, uint32_t v) {
    if (lane() < 12) slot[lane()] = v;
}

}  // namespace wfq
