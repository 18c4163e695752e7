// Fq = GF(p), p the 377-bit BLS12-377 base-field prime, on sm_103a.
//
// Elements are 12 little-endian 32-bit limbs in Montgomery form x*R mod p with
// R = 2^384. Multiplication is word-serial Montgomery (CIOS) taken two words at a
// time: each step adds the rows a_2s*b and a_2s+1*b, then the two quotient digits
// m0 = -t_0 and m1 = -t_1 (-p^-1 = 0xffffffff mod 2^32 because p = 1 mod 2^46)
// with their rows m*p, and the accumulator drops two words (mont_dstep). Every row
// runs as mad.lo.cc / madc.hi.cc carry chains of adjacent low/high halves (the
// products with the even- and with the odd-indexed limbs in two accumulators);
// every chain sits in one asm statement so the carry flag never crosses
// statements.
//
// Two facts about how these chains compile on sm_103a, measured with ncu opcode
// counts (a chain pair compiles either to one fused 64-bit multiply-add, four
// cycles of the multiply pipe, or to a low and a high multiply, six cycles):
//  * A pair fuses only when its 64-bit accumulator sits in an aligned register
//    pair. Dropping one word per row misaligns every other row (the compiler then
//    inserts a move per product); dropping two words per step keeps every pair
//    aligned.
//  * The compiler folds a negation into the multiplications it feeds, and a
//    folded m*p_j does not fuse. So the digits are formed as (t_k ^ mask) + 1 with
//    the all-ones mask read through a volatile constant load (neg_one), which the
//    compiler cannot see through: two ALU operations per digit (t_k * (-1) with the
//    same opaque -1 also works, but takes the multiply pipe), and all 276 products
//    per multiplication fuse.
// Against one word per row with m = -t_0 (mul_singlerow_inl, the earlier form):
// 1104 instead of 1368 multiply-pipe cycles per multiplication, and the MSM's
// accumulation 4.63 -> 4.22 ms at 2^20 points.
//
// mul() is one out-of-line function. A point operation makes 10-14 calls; with
// the body inlined at every call site the code of one point addition is about
// 100 KB, which thrashes the instruction cache: measured on GB300, one thread's
// XYZZ doubling takes 63k cycles inlined and 27k out of line, and a full grid of
// doublings runs 1.1-1.6 G/s inlined and 1.8-1.9 G/s out of line. mul_inl() is the
// inlined body for kernels with a single multiplication per element.
//
// Lazy reduction (the GPU form of the paper's skipped fine reduction and
// unreduced intermediate additions, Sec. III-E): a product of inputs a, b with
// a*b < p*R leaves mul() in [0, 2p) without the final conditional subtraction.
// All values kept in registers or memory by the curve code live in [0, 2p);
// add/sub fold back into [0, 2p) with one masked correction of 2p, so every
// product satisfies a*b < 4p^2 < p*R (R/p > 152). canon() maps [0, 2p) to [0, p).
// Accumulator bounds: see mont_dstep.
//
// (A carry-save variant in the style of the paper's Sec. III-D -- 16 digits of
// 24 bits, 64-bit mad.wide column sums, two coarse carry rounds -- was built and
// measured: 2.7x lower multiplication latency than inlined CIOS but, at the
// quarter-rate 64-bit mad.wide, 1.3x lower throughput in full point operations,
// and slower than out-of-line CIOS in both; it is not used.)
#pragma once
#include <stdint.h>

namespace fq {

constexpr int N = 12;

struct fe {
    uint32_t v[N];
};

// p, 2p, R mod p (Montgomery one), R^2 mod p (to-Montgomery factor), R^3 mod p.
__device__ __constant__ static const uint32_t kP[N] = {
    0x00000001u, 0x8508c000u, 0x30000000u, 0x170b5d44u, 0xba094800u, 0x1ef3622fu,
    0x00f5138fu, 0x1a22d9f3u, 0x6ca1493bu, 0xc63b05c0u, 0x17c510eau, 0x01ae3a46u};
__device__ __constant__ static const uint32_t k2P[N] = {
    0x00000002u, 0x0a118000u, 0x60000001u, 0x2e16ba88u, 0x74129000u, 0x3de6c45fu,
    0x01ea271eu, 0x3445b3e6u, 0xd9429276u, 0x8c760b80u, 0x2f8a21d5u, 0x035c748cu};
__device__ __constant__ static const uint32_t kOne[N] = {
    0xffffff68u, 0x02cdffffu, 0x7fffffb1u, 0x51409f83u, 0x8a7d3ff2u, 0x9f7db3a9u,
    0x6e7c6305u, 0x7b4e97b7u, 0x803c84e8u, 0x4cf495bfu, 0xe2fdf49au, 0x008d6661u};
__device__ __constant__ static const uint32_t kR2[N] = {
    0x9400cd22u, 0xb786686cu, 0xb00431b1u, 0x0329fcaau, 0x62d6b46du, 0x22a5f111u,
    0x827dc3acu, 0xbfdf7d03u, 0x41790bf9u, 0x837e92f0u, 0x1e914b88u, 0x006dfccbu};
__device__ __constant__ static const uint32_t kR3[N] = {
    0x8815de20u, 0x581f532fu, 0xbe329585u, 0xe50f4148u, 0x0449f513u, 0x2be8b118u,
    0xc804a20eu, 0x6a2a9516u, 0x13590cb9u, 0x3f725407u, 0xc0e7dda5u, 0x01065ab4u};

// 2p limbs as compile-time values for masked corrections.
#define FQ_2P_LIMBS 0x00000002u, 0x0a118000u, 0x60000001u, 0x2e16ba88u, 0x74129000u, \
    0x3de6c45fu, 0x01ea271eu, 0x3445b3e6u, 0xd9429276u, 0x8c760b80u, 0x2f8a21d5u, 0x035c748cu
#define FQ_P_LIMBS 0x00000001u, 0x8508c000u, 0x30000000u, 0x170b5d44u, 0xba094800u, \
    0x1ef3622fu, 0x00f5138fu, 0x1a22d9f3u, 0x6ca1493bu, 0xc63b05c0u, 0x17c510eau, 0x01ae3a46u

__device__ __forceinline__ void set_zero(fe& r) {
#pragma unroll
    for (int k = 0; k < N; ++k) r.v[k] = 0;
}

__device__ __forceinline__ void set_one(fe& r) {
    const uint32_t one[N] = {0xffffff68u, 0x02cdffffu, 0x7fffffb1u, 0x51409f83u, 0x8a7d3ff2u,
                             0x9f7db3a9u, 0x6e7c6305u, 0x7b4e97b7u, 0x803c84e8u, 0x4cf495bfu,
                             0xe2fdf49au, 0x008d6661u};
#pragma unroll
    for (int k = 0; k < N; ++k) r.v[k] = one[k];
}

// r = a*b*R^-1 mod p, result in [0, 2p) when a*b < p*R. Inlined body.
// Word-serial Montgomery (one row per limb a_i: t += a_i b, m = -t_0, t += m p,
// t >>= 32) with each row's partial products split into two independent carry
// chains: the even-indexed limbs of the multiplicand accumulate in e (low half of
// a_i b_j at e[j], high half at e[j + 1]) and the odd-indexed ones in o, held one
// limb up (a_i b_j for odd j at o[j - 1], o[j]); so each chain is one run of
// lo/hi multiply-adds of the same product, with no second pass for the high
// halves (on GB300 this shape runs 1.4x faster than a low-half chain followed by
// a high-half chain, in throughput and in latency). The running value is
// e + 2^32 o, so the quotient digit is m = -e[0] (-p^-1 = -1 mod 2^32). m p is
// split the same way; since p_0 = 1, the high half of m p_0 is zero, and that
// slot of the even chain adds o[0] instead, after which both chains shift down
// one limb and e + 2^32 o again has o one limb above e. After the 12 rows the
// result is e + 2^32 o (one carry chain).
struct MontAcc {
    uint32_t e[13], o[13];
};

// One row: t += x b, m = -e[0], t += m p, shift (mul_singlerow_inl). Within a row
// the two accumulators e (even-indexed limbs of b) and o (odd, one word up) are
// independent chains; with a, b < 2p a row adds less than 2^411 to each, whose
// values stay below 2^380 after the shift and below 2^412 before it (13 words).
__device__ __forceinline__ void mont_row(MontAcc& t, uint32_t x, const uint32_t* b) {
    uint32_t* e = t.e;
    uint32_t* o = t.o;
    asm("mad.lo.cc.u32 %0, %13, %14, %0;\n\t"
        "madc.hi.cc.u32 %1, %13, %14, %1;\n\t"
        "madc.lo.cc.u32 %2, %13, %15, %2;\n\t"
        "madc.hi.cc.u32 %3, %13, %15, %3;\n\t"
        "madc.lo.cc.u32 %4, %13, %16, %4;\n\t"
        "madc.hi.cc.u32 %5, %13, %16, %5;\n\t"
        "madc.lo.cc.u32 %6, %13, %17, %6;\n\t"
        "madc.hi.cc.u32 %7, %13, %17, %7;\n\t"
        "madc.lo.cc.u32 %8, %13, %18, %8;\n\t"
        "madc.hi.cc.u32 %9, %13, %18, %9;\n\t"
        "madc.lo.cc.u32 %10, %13, %19, %10;\n\t"
        "madc.hi.cc.u32 %11, %13, %19, %11;\n\t"
        "addc.u32 %12, %12, 0;"
        : "+r"(e[0]), "+r"(e[1]), "+r"(e[2]), "+r"(e[3]), "+r"(e[4]), "+r"(e[5]), "+r"(e[6]), "+r"(e[7]),
          "+r"(e[8]), "+r"(e[9]), "+r"(e[10]), "+r"(e[11]), "+r"(e[12])
        : "r"(x), "r"(b[0]), "r"(b[2]), "r"(b[4]), "r"(b[6]), "r"(b[8]), "r"(b[10]));
    asm("mad.lo.cc.u32 %0, %13, %14, %0;\n\t"
        "madc.hi.cc.u32 %1, %13, %14, %1;\n\t"
        "madc.lo.cc.u32 %2, %13, %15, %2;\n\t"
        "madc.hi.cc.u32 %3, %13, %15, %3;\n\t"
        "madc.lo.cc.u32 %4, %13, %16, %4;\n\t"
        "madc.hi.cc.u32 %5, %13, %16, %5;\n\t"
        "madc.lo.cc.u32 %6, %13, %17, %6;\n\t"
        "madc.hi.cc.u32 %7, %13, %17, %7;\n\t"
        "madc.lo.cc.u32 %8, %13, %18, %8;\n\t"
        "madc.hi.cc.u32 %9, %13, %18, %9;\n\t"
        "madc.lo.cc.u32 %10, %13, %19, %10;\n\t"
        "madc.hi.cc.u32 %11, %13, %19, %11;\n\t"
        "addc.u32 %12, %12, 0;"
        : "+r"(o[0]), "+r"(o[1]), "+r"(o[2]), "+r"(o[3]), "+r"(o[4]), "+r"(o[5]), "+r"(o[6]), "+r"(o[7]),
          "+r"(o[8]), "+r"(o[9]), "+r"(o[10]), "+r"(o[11]), "+r"(o[12])
        : "r"(x), "r"(b[1]), "r"(b[3]), "r"(b[5]), "r"(b[7]), "r"(b[9]), "r"(b[11]));
    const uint32_t m = 0u - e[0];
    asm("mad.lo.cc.u32 %0, %13, 0x8508c000, %0;\n\t"
        "madc.hi.cc.u32 %1, %13, 0x8508c000, %1;\n\t"
        "madc.lo.cc.u32 %2, %13, 0x170b5d44, %2;\n\t"
        "madc.hi.cc.u32 %3, %13, 0x170b5d44, %3;\n\t"
        "madc.lo.cc.u32 %4, %13, 0x1ef3622f, %4;\n\t"
        "madc.hi.cc.u32 %5, %13, 0x1ef3622f, %5;\n\t"
        "madc.lo.cc.u32 %6, %13, 0x1a22d9f3, %6;\n\t"
        "madc.hi.cc.u32 %7, %13, 0x1a22d9f3, %7;\n\t"
        "madc.lo.cc.u32 %8, %13, 0xc63b05c0, %8;\n\t"
        "madc.hi.cc.u32 %9, %13, 0xc63b05c0, %9;\n\t"
        "madc.lo.cc.u32 %10, %13, 0x01ae3a46, %10;\n\t"
        "madc.hi.cc.u32 %11, %13, 0x01ae3a46, %11;\n\t"
        "addc.u32 %12, %12, 0;"
        : "+r"(o[0]), "+r"(o[1]), "+r"(o[2]), "+r"(o[3]), "+r"(o[4]), "+r"(o[5]), "+r"(o[6]), "+r"(o[7]),
          "+r"(o[8]), "+r"(o[9]), "+r"(o[10]), "+r"(o[11]), "+r"(o[12])
        : "r"(m));
    asm("add.cc.u32 %0, %0, %14;\n\t"
        "addc.cc.u32 %1, %1, %13;\n\t"
        "madc.lo.cc.u32 %2, %14, 0x30000000, %2;\n\t"
        "madc.hi.cc.u32 %3, %14, 0x30000000, %3;\n\t"
        "madc.lo.cc.u32 %4, %14, 0xba094800, %4;\n\t"
        "madc.hi.cc.u32 %5, %14, 0xba094800, %5;\n\t"
        "madc.lo.cc.u32 %6, %14, 0x00f5138f, %6;\n\t"
        "madc.hi.cc.u32 %7, %14, 0x00f5138f, %7;\n\t"
        "madc.lo.cc.u32 %8, %14, 0x6ca1493b, %8;\n\t"
        "madc.hi.cc.u32 %9, %14, 0x6ca1493b, %9;\n\t"
        "madc.lo.cc.u32 %10, %14, 0x17c510ea, %10;\n\t"
        "madc.hi.cc.u32 %11, %14, 0x17c510ea, %11;\n\t"
        "addc.u32 %12, %12, 0;"
        : "+r"(e[0]), "+r"(e[1]), "+r"(e[2]), "+r"(e[3]), "+r"(e[4]), "+r"(e[5]), "+r"(e[6]), "+r"(e[7]),
          "+r"(e[8]), "+r"(e[9]), "+r"(e[10]), "+r"(e[11]), "+r"(e[12])
        : "r"(o[0]), "r"(m));
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        e[k] = e[k + 1];
        o[k] = o[k + 1];
    }
    e[12] = 0;
    o[12] = 0;
}

// r = e + 2^32 o after the last row (the words from 12 up cancel).
__device__ __forceinline__ void mont_final(fe& r, const MontAcc& t) {
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

// Two rows and two quotient digits per step, accumulators shifted by two limbs, so
// the register pair holding the low and high half of one partial product keeps its
// alignment from step to step.
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
struct MontAccD {
    uint32_t e[14], o[14];
};

__device__ __forceinline__ void mont_dstep(MontAccD& t, uint32_t x0, uint32_t x1, const uint32_t* b, uint32_t neg1) {
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
    const uint32_t m0 = (E[0] ^ neg1) + 1u;   // -E[0], through the opaque mask (neg_one)
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
    const uint32_t m1 = (E[1] ^ neg1) + 1u;
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

// r = E + 2^32 O after the last step (the words from 12 up cancel).
__device__ __forceinline__ void mont_dfinal(fe& r, const MontAccD& t) {
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

// All ones (-1), read through a volatile constant load so the compiler cannot fold it.
__device__ __constant__ static volatile uint32_t kNegOne = 0xffffffffu;
__device__ __forceinline__ uint32_t neg_one() { return kNegOne; }

__device__ __forceinline__ void mul_inl(fe& r, const fe& a, const fe& b) {
    MontAccD t = {};
    const uint32_t neg1 = neg_one();
#pragma unroll
    for (int i = 0; i < N; i += 2) mont_dstep(t, a.v[i], a.v[i + 1], b.v, neg1);
    mont_dfinal(r, t);
}

// The earlier form: one row and one digit m = -t_0 per step (the variant
// MSM377_FQMUL_CIOS_SINGLEROW of fq_mul_batch_variant).
__device__ __forceinline__ void mul_singlerow_inl(fe& r, const fe& a, const fe& b) {
    MontAcc t = {};
#pragma unroll
    for (int i = 0; i < N; ++i) mont_row(t, a.v[i], b.v);
    mont_final(r, t);
}

// Two independent products with their rows interleaved: four independent carry
// chains in flight instead of two.
__device__ __forceinline__ void mul2_inl(fe& r1, const fe& a1, const fe& b1, fe& r2, const fe& a2, const fe& b2) {
    MontAccD t1 = {}, t2 = {};
    const uint32_t neg1 = neg_one();
#pragma unroll
    for (int i = 0; i < N; i += 2) {
        mont_dstep(t1, a1.v[i], a1.v[i + 1], b1.v, neg1);
        mont_dstep(t2, a2.v[i], a2.v[i + 1], b2.v, neg1);
    }
    mont_dfinal(r1, t1);
    mont_dfinal(r2, t2);
}

// Out-of-line multiplication used by the point arithmetic (one copy of the code).
// Operands and result pass by value so the call keeps them in registers (a
// by-reference signature forces them through the stack in local memory).
static __device__ __noinline__ fe mul_v(fe a, fe b) {
    fe r;
    mul_inl(r, a, b);
    return r;
}
__device__ __forceinline__ void mul(fe& r, const fe& a, const fe& b) { r = mul_v(a, b); }

struct fe2 {
    fe a, b;
};
static __device__ __noinline__ fe2 mul2_v(fe a1, fe b1, fe a2, fe b2) {
    fe2 r;
    mul2_inl(r.a, a1, b1, r.b, a2, b2);
    return r;
}
// r1 = a1 b1, r2 = a2 b2 (R^-1 mod p each) in one call.
__device__ __forceinline__ void mul2(fe& r1, const fe& a1, const fe& b1, fe& r2, const fe& a2, const fe& b2) {
    const fe2 r = mul2_v(a1, b1, a2, b2);
    r1 = r.a;
    r2 = r.b;
}

__device__ __forceinline__ void sqr(fe& r, const fe& a) { mul(r, a, a); }

// r = a + b, inputs in [0, 2p); result folded into [0, 2p).
__device__ __forceinline__ void add(fe& rr, const fe& a, const fe& bb) {
    uint32_t r[N];
    const uint32_t* b = bb.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r[k] = a.v[k];
    asm(
        "add.cc.u32 %0, %0, %12;\n\t"
        "addc.cc.u32 %1, %1, %13;\n\t"
        "addc.cc.u32 %2, %2, %14;\n\t"
        "addc.cc.u32 %3, %3, %15;\n\t"
        "addc.cc.u32 %4, %4, %16;\n\t"
        "addc.cc.u32 %5, %5, %17;\n\t"
        "addc.cc.u32 %6, %6, %18;\n\t"
        "addc.cc.u32 %7, %7, %19;\n\t"
        "addc.cc.u32 %8, %8, %20;\n\t"
        "addc.cc.u32 %9, %9, %21;\n\t"
        "addc.cc.u32 %10, %10, %22;\n\t"
        "addc.u32 %11, %11, %23;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]));
    uint32_t u[N], mask;
    asm(
        "sub.cc.u32 %0, %13, 0x00000002;\n\t"
        "subc.cc.u32 %1, %14, 0x0a118000;\n\t"
        "subc.cc.u32 %2, %15, 0x60000001;\n\t"
        "subc.cc.u32 %3, %16, 0x2e16ba88;\n\t"
        "subc.cc.u32 %4, %17, 0x74129000;\n\t"
        "subc.cc.u32 %5, %18, 0x3de6c45f;\n\t"
        "subc.cc.u32 %6, %19, 0x01ea271e;\n\t"
        "subc.cc.u32 %7, %20, 0x3445b3e6;\n\t"
        "subc.cc.u32 %8, %21, 0xd9429276;\n\t"
        "subc.cc.u32 %9, %22, 0x8c760b80;\n\t"
        "subc.cc.u32 %10, %23, 0x2f8a21d5;\n\t"
        "subc.cc.u32 %11, %24, 0x035c748c;\n\t"
        "subc.u32 %12, 0, 0;"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
          "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(mask)
        : "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
          "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]));
    // mask = ~0 when a + b < 2p (keep the sum), 0 otherwise (take the difference)
#pragma unroll
    for (int k = 0; k < N; ++k) rr.v[k] = (r[k] & mask) | (u[k] & ~mask);
}

// r = a - b, inputs in [0, 2p); adds 2p when the difference is negative.
__device__ __forceinline__ void sub(fe& rr, const fe& a, const fe& bb) {
    uint32_t r[N], mask;
    const uint32_t* b = bb.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r[k] = a.v[k];
    asm(
        "sub.cc.u32 %0, %0, %13;\n\t"
        "subc.cc.u32 %1, %1, %14;\n\t"
        "subc.cc.u32 %2, %2, %15;\n\t"
        "subc.cc.u32 %3, %3, %16;\n\t"
        "subc.cc.u32 %4, %4, %17;\n\t"
        "subc.cc.u32 %5, %5, %18;\n\t"
        "subc.cc.u32 %6, %6, %19;\n\t"
        "subc.cc.u32 %7, %7, %20;\n\t"
        "subc.cc.u32 %8, %8, %21;\n\t"
        "subc.cc.u32 %9, %9, %22;\n\t"
        "subc.cc.u32 %10, %10, %23;\n\t"
        "subc.cc.u32 %11, %11, %24;\n\t"
        "subc.u32 %12, 0, 0;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "=r"(mask)
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]));
    const uint32_t twop[N] = {FQ_2P_LIMBS};
    uint32_t c[N];
#pragma unroll
    for (int k = 0; k < N; ++k) c[k] = twop[k] & mask;
    asm(
        "add.cc.u32 %0, %0, %12;\n\t"
        "addc.cc.u32 %1, %1, %13;\n\t"
        "addc.cc.u32 %2, %2, %14;\n\t"
        "addc.cc.u32 %3, %3, %15;\n\t"
        "addc.cc.u32 %4, %4, %16;\n\t"
        "addc.cc.u32 %5, %5, %17;\n\t"
        "addc.cc.u32 %6, %6, %18;\n\t"
        "addc.cc.u32 %7, %7, %19;\n\t"
        "addc.cc.u32 %8, %8, %20;\n\t"
        "addc.cc.u32 %9, %9, %21;\n\t"
        "addc.cc.u32 %10, %10, %22;\n\t"
        "addc.u32 %11, %11, %23;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11])
        : "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(c[5]), "r"(c[6]),
          "r"(c[7]), "r"(c[8]), "r"(c[9]), "r"(c[10]), "r"(c[11]));
#pragma unroll
    for (int k = 0; k < N; ++k) rr.v[k] = r[k];
}

__device__ __forceinline__ void dbl(fe& r, const fe& a) { add(r, a, a); }

// Unfolded add / subtract for values that only feed multiplications. mul() stays
// exact and lands in [0, 2p) for a b < p R (R / p > 152), so an operand may be a
// few multiples of p: add_nr of two values below 2p is below 4p, sub_nr<K> of
// a, b is a - b + K p (needs b <= a + K p), and the callers keep every product
// below 152 p^2 (ed.cuh states the ranges per formula). One carry chain (add_nr)
// or two (sub_nr) instead of the folded forms' chains, masks and selects.
__device__ __forceinline__ void add_nr(fe& rr, const fe& a, const fe& bb) {
    uint32_t r[N];
    const uint32_t* b = bb.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r[k] = a.v[k];
    asm(
        "add.cc.u32 %0, %0, %12;\n\t"
        "addc.cc.u32 %1, %1, %13;\n\t"
        "addc.cc.u32 %2, %2, %14;\n\t"
        "addc.cc.u32 %3, %3, %15;\n\t"
        "addc.cc.u32 %4, %4, %16;\n\t"
        "addc.cc.u32 %5, %5, %17;\n\t"
        "addc.cc.u32 %6, %6, %18;\n\t"
        "addc.cc.u32 %7, %7, %19;\n\t"
        "addc.cc.u32 %8, %8, %20;\n\t"
        "addc.cc.u32 %9, %9, %21;\n\t"
        "addc.cc.u32 %10, %10, %22;\n\t"
        "addc.u32 %11, %11, %23;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]));
#pragma unroll
    for (int k = 0; k < N; ++k) rr.v[k] = r[k];
}

template <int K>
__device__ __forceinline__ void sub_nr(fe& rr, const fe& a, const fe& bb) {
    static_assert(K == 2 || K == 4, "sub_nr adds 2p or 4p");
    uint32_t r[N];
    const uint32_t* b = bb.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r[k] = a.v[k];
    if constexpr (K == 2) {
        asm(
        "add.cc.u32 %0, %0, 0x00000002;\n\t"
        "addc.cc.u32 %1, %1, 0x0a118000;\n\t"
        "addc.cc.u32 %2, %2, 0x60000001;\n\t"
        "addc.cc.u32 %3, %3, 0x2e16ba88;\n\t"
        "addc.cc.u32 %4, %4, 0x74129000;\n\t"
        "addc.cc.u32 %5, %5, 0x3de6c45f;\n\t"
        "addc.cc.u32 %6, %6, 0x01ea271e;\n\t"
        "addc.cc.u32 %7, %7, 0x3445b3e6;\n\t"
        "addc.cc.u32 %8, %8, 0xd9429276;\n\t"
        "addc.cc.u32 %9, %9, 0x8c760b80;\n\t"
        "addc.cc.u32 %10, %10, 0x2f8a21d5;\n\t"
        "addc.u32 %11, %11, 0x035c748c;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]));
    } else {
        asm(
        "add.cc.u32 %0, %0, 0x00000004;\n\t"
        "addc.cc.u32 %1, %1, 0x14230000;\n\t"
        "addc.cc.u32 %2, %2, 0xc0000002;\n\t"
        "addc.cc.u32 %3, %3, 0x5c2d7510;\n\t"
        "addc.cc.u32 %4, %4, 0xe8252000;\n\t"
        "addc.cc.u32 %5, %5, 0x7bcd88be;\n\t"
        "addc.cc.u32 %6, %6, 0x03d44e3c;\n\t"
        "addc.cc.u32 %7, %7, 0x688b67cc;\n\t"
        "addc.cc.u32 %8, %8, 0xb28524ec;\n\t"
        "addc.cc.u32 %9, %9, 0x18ec1701;\n\t"
        "addc.cc.u32 %10, %10, 0x5f1443ab;\n\t"
        "addc.u32 %11, %11, 0x06b8e918;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]));
    }
    asm(
        "sub.cc.u32 %0, %0, %12;\n\t"
        "subc.cc.u32 %1, %1, %13;\n\t"
        "subc.cc.u32 %2, %2, %14;\n\t"
        "subc.cc.u32 %3, %3, %15;\n\t"
        "subc.cc.u32 %4, %4, %16;\n\t"
        "subc.cc.u32 %5, %5, %17;\n\t"
        "subc.cc.u32 %6, %6, %18;\n\t"
        "subc.cc.u32 %7, %7, %19;\n\t"
        "subc.cc.u32 %8, %8, %20;\n\t"
        "subc.cc.u32 %9, %9, %21;\n\t"
        "subc.cc.u32 %10, %10, %22;\n\t"
        "subc.u32 %11, %11, %23;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]));
#pragma unroll
    for (int k = 0; k < N; ++k) rr.v[k] = r[k];
}

// [0, 2p) -> [0, p)
__device__ __forceinline__ void canon(fe& rr, const fe& a) {
    uint32_t u[N], mask;
    asm(
        "sub.cc.u32 %0, %13, 0x00000001;\n\t"
        "subc.cc.u32 %1, %14, 0x8508c000;\n\t"
        "subc.cc.u32 %2, %15, 0x30000000;\n\t"
        "subc.cc.u32 %3, %16, 0x170b5d44;\n\t"
        "subc.cc.u32 %4, %17, 0xba094800;\n\t"
        "subc.cc.u32 %5, %18, 0x1ef3622f;\n\t"
        "subc.cc.u32 %6, %19, 0x00f5138f;\n\t"
        "subc.cc.u32 %7, %20, 0x1a22d9f3;\n\t"
        "subc.cc.u32 %8, %21, 0x6ca1493b;\n\t"
        "subc.cc.u32 %9, %22, 0xc63b05c0;\n\t"
        "subc.cc.u32 %10, %23, 0x17c510ea;\n\t"
        "subc.cc.u32 %11, %24, 0x01ae3a46;\n\t"
        "subc.u32 %12, 0, 0;"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
          "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(mask)
        : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
          "r"(a.v[6]), "r"(a.v[7]), "r"(a.v[8]), "r"(a.v[9]), "r"(a.v[10]), "r"(a.v[11]));
#pragma unroll
    for (int k = 0; k < N; ++k) rr.v[k] = (a.v[k] & mask) | (u[k] & ~mask);
}

// r = -a for a in [0, 2p): 2p - a, then folded into [0, 2p) (maps 0 to 0).
__device__ __forceinline__ void neg(fe& r, const fe& a) {
    fe z;
    set_zero(z);
    sub(r, z, a);
}

__device__ __forceinline__ bool is_zero_raw(const fe& a) {
    uint32_t o = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) o |= a.v[k];
    return o == 0;
}

// a in [0, 2p) represents zero iff a == 0 or a == p.
__device__ __forceinline__ bool is_zero(const fe& a) {
    const uint32_t p[N] = {FQ_P_LIMBS};
    uint32_t o = 0, q = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        o |= a.v[k];
        q |= a.v[k] ^ p[k];
    }
    return o == 0 || q == 0;
}

// a == b as field elements, both in [0, 2p).
__device__ __forceinline__ bool equal(const fe& a, const fe& b) {
    fe d;
    sub(d, a, b);
    return is_zero(d);
}

__device__ __forceinline__ void to_mont(fe& r, const fe& a_std) {
    fe r2;
#pragma unroll
    for (int k = 0; k < N; ++k) r2.v[k] = kR2[k];
    mul(r, a_std, r2);
    canon(r, r);
}

__device__ __forceinline__ void from_mont(fe& r, const fe& a) {
    fe one;
    set_zero(one);
    one.v[0] = 1;
    mul(r, a, one);
    canon(r, r);
}

__device__ __forceinline__ void load(fe& r, const uint32_t* p) {
#pragma unroll
    for (int k = 0; k < N; ++k) r.v[k] = p[k];
}

__device__ __forceinline__ void store(uint32_t* p, const fe& a) {
#pragma unroll
    for (int k = 0; k < N; ++k) p[k] = a.v[k];
}

// Strided (structure-of-arrays) access: limb k of element i at base[k * stride + i].
__device__ __forceinline__ void load_soa(fe& r, const uint32_t* base, size_t i, size_t stride) {
#pragma unroll
    for (int k = 0; k < N; ++k) r.v[k] = base[k * stride + i];
}

__device__ __forceinline__ void store_soa(uint32_t* base, size_t i, size_t stride, const fe& a) {
#pragma unroll
    for (int k = 0; k < N; ++k) base[k * stride + i] = a.v[k];
}

// a < p for a standard-form input (used to validate boundary data).
__device__ __forceinline__ bool lt_p(const fe& a) {
    const uint32_t p[N] = {FQ_P_LIMBS};
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
        if (a.v[k] != p[k]) return a.v[k] < p[k];
    }
    return false;
}

}  // namespace fq
