// Point operations of both curve models run by four warps together, each warp
// computing one product of a formula level with the warp-spread multiplication of
// wfq.cuh; the warps exchange values through shared memory slots of 12 words and
// meet at block barriers (one group of four warps per 128-thread block). For the
// dependent chains of an MSM (window combination, per-window sums, the paper's
// dependent-chain latency experiment, Sec. V-A), where one accumulator is updated
// again and again: a doubling costs two (Edwards) or three (XYZZ) latencies of the
// warp multiplication instead of as many sequential Montgomery multiplications on
// one lane.
//
// The accumulator lives in slots 0..3 (Edwards X, Y, Z, T; XYZZ X, Y, ZZ, ZZZ);
// slots 4..17 are temporaries. Every thread of the block calls every function
// (the branches taken on point values are block-uniform: every warp reads the same
// shared or global words), so each __syncthreads is reached by all.
// Formulas and value ranges are those of ed.cuh and ec.cuh.
#pragma once
#include "ec.cuh"
#include "ed.cuh"
#include "wfq.cuh"

namespace wpt {

using wfq::Consts;

constexpr int kSlots = 18;
// Shared words a group needs: the slots, then each warp's multiplication scratch.
constexpr int kSharedWords = kSlots * 12 + 4 * wfq::kScratchWords;
enum : int { X = 0, Y = 1, Z = 2, T = 3, ZZ = 2, ZZZ = 3 };

struct Group {
    uint32_t* s;   // kSlots x 12 words of shared memory (then the warps' scratch)
    int w;         // warp index within the group, 0..3
    Consts K;
    uint32_t k;    // limb `lane` of the Edwards constant k = 2d (Montgomery form)
    uint32_t one;  // limb `lane` of 1 (Montgomery form)

    __device__ __forceinline__ uint32_t ld(int i) const { return wfq::load(s + 12 * i); }
    __device__ __forceinline__ void st(int i, uint32_t v) const { wfq::store(s + 12 * i, v); }
    __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) const { return wfq::mul(a, b, K); }
};

// slots: kSharedWords words of shared memory, 16-byte aligned.
__device__ __forceinline__ void init(Group& g, uint32_t* slots) {
    g.s = slots;
    g.w = threadIdx.x >> 5;
    wfq::init(g.K, slots + kSlots * 12 + g.w * wfq::kScratchWords);
    g.k = wfq::limb_of(ed::kK);
    g.one = wfq::limb_of(fq::kOne);
}

// Accumulator <- point in memory (four coordinates of 12 words: 12 uint4).
__device__ __forceinline__ void load_acc(const Group& g, const uint32_t* p) {
    g.st(g.w, wfq::load(p + 12 * g.w));
    __syncthreads();
}

__device__ __forceinline__ void store_acc(const Group& g, uint32_t* p) {
    wfq::store(p + 12 * g.w, g.ld(g.w));
}

// ------------------------------------------------------------------ Edwards

__device__ __forceinline__ void ed_set_inf(const Group& g) {   // (0, 1, 1, 0)
    g.st(g.w, (g.w == Y || g.w == Z) ? g.one : 0u);
    __syncthreads();
}

// P = 2P (a = -1): level 1 {A = X^2, B = Y^2, C = Z^2, X Y}; E = 2 X Y (= (X + Y)^2 -
// A - B), G = B - A, H = -A - B, F = G - 2C, each one linear combination with a
// single carry resolution; level 2 {E F, G H, E H, F G}. Ranges: E < 4p, G, H < 4p,
// F = B - A - 2C + 6p < 8p.
__device__ __forceinline__ void ed_dbl(const Group& g) {
    const Consts& K = g.K;
    switch (g.w) {
        case 0: g.st(4, g.mul(g.ld(X), g.ld(X))); break;
        case 1: g.st(5, g.mul(g.ld(Y), g.ld(Y))); break;
        case 2: g.st(6, g.mul(g.ld(Z), g.ld(Z))); break;
        default: g.st(7, g.mul(g.ld(X), g.ld(Y)));
    }
    __syncthreads();
    const uint32_t A = g.ld(4), B = g.ld(5);
    switch (g.w) {
        case 0: {
            const uint32_t xy = g.ld(7);
            g.st(8, wfq::add_nr(xy, xy));                                            // E
            break;
        }
        case 1: g.st(9, wfq::lincomb<1, 1>({B}, {A}, K.p2)); break;                  // G
        case 2: g.st(10, wfq::lincomb<1, 2>({0u}, {A, B}, K.p4)); break;             // H
        default: {
            const uint32_t C = g.ld(6);
            g.st(11, wfq::lincomb<1, 3>({B}, {A, C, C}, K.p6));                      // F
        }
    }
    __syncthreads();
    switch (g.w) {
        case 0: g.st(X, g.mul(g.ld(8), g.ld(11))); break;
        case 1: g.st(Y, g.mul(g.ld(9), g.ld(10))); break;
        case 2: g.st(T, g.mul(g.ld(8), g.ld(10))); break;
        default: g.st(Z, g.mul(g.ld(11), g.ld(9)));
    }
    __syncthreads();
}

// E, H from A (slot 4), B (5) and F, G from D (7), C (6); then level {E F, G H, E H, F G}.
__device__ __forceinline__ void ed_finish(const Group& g) {
    const Consts& K = g.K;
    switch (g.w) {
        case 0: g.st(8, wfq::sub_nr2(g.ld(5), g.ld(4), K)); break;    // E = B - A
        case 1: g.st(9, wfq::add_nr(g.ld(5), g.ld(4))); break;        // H = B + A
        case 2: g.st(10, wfq::sub_nr2(g.ld(7), g.ld(6), K)); break;   // F = D - C
        default: g.st(11, wfq::add_nr(g.ld(7), g.ld(6)));             // G = D + C
    }
    __syncthreads();
    switch (g.w) {
        case 0: g.st(X, g.mul(g.ld(8), g.ld(10))); break;
        case 1: g.st(Y, g.mul(g.ld(11), g.ld(9))); break;
        case 2: g.st(T, g.mul(g.ld(8), g.ld(9))); break;
        default: g.st(Z, g.mul(g.ld(10), g.ld(11)));
    }
    __syncthreads();
}

// A point operand held by every warp of the group: limb `lane` of each coordinate
// (read once from memory, so the loads of the next operand can overlap the current
// operation).
struct Operand {
    uint32_t c[4];
};

__device__ __forceinline__ Operand load_operand(const uint32_t* q, int ncoord) {
    Operand o;
#pragma unroll
    for (int i = 0; i < 4; ++i) o.c[i] = i < ncoord ? wfq::load(q + 12 * i) : 0u;
    return o;
}

// P += Q, Q stored (x, y, u = k x y) as loaded by load_operand(q, 3): level 1
// {A, B, C = T1 u2} (the sums of Q's coordinates formed alongside those of P's),
// D = 2 Z1.
__device__ __forceinline__ void ed_madd(const Group& g, const Operand& q) {
    const Consts& K = g.K;
    switch (g.w) {
        case 0: g.st(4, g.mul(wfq::sub_nr2(g.ld(Y), g.ld(X), K), wfq::sub_nr2(q.c[1], q.c[0], K))); break;
        case 1: g.st(5, g.mul(wfq::add_nr(g.ld(Y), g.ld(X)), wfq::add_nr(q.c[1], q.c[0]))); break;
        case 2: g.st(6, g.mul(g.ld(T), q.c[2])); break;
        default: g.st(7, wfq::add_nr(g.ld(Z), g.ld(Z)));
    }
    __syncthreads();
    ed_finish(g);
}

// P += Q, Q extended (X, Y, Z, T); an all-zero Q (an empty bucket) is skipped.
// Level 1 {A, B, T1 T2, Z1 Z2}, level 2 {C = k T1 T2}, D = 2 Z1 Z2.
__device__ __forceinline__ void ed_add(const Group& g, const Operand& q) {
    if (wfq::is_zero_raw(q.c[2])) return;
    const Consts& K = g.K;
    switch (g.w) {
        case 0: g.st(4, g.mul(wfq::sub_nr2(g.ld(Y), g.ld(X), K), wfq::sub_nr2(q.c[1], q.c[0], K))); break;
        case 1: g.st(5, g.mul(wfq::add_nr(g.ld(Y), g.ld(X)), wfq::add_nr(q.c[1], q.c[0]))); break;
        case 2: g.st(12, g.mul(g.ld(T), q.c[3])); break;
        default: g.st(13, g.mul(g.ld(Z), q.c[2]));
    }
    __syncthreads();
    if (g.w == 2) g.st(6, g.mul(g.ld(12), g.k));                      // C = k T1 T2
    if (g.w == 3) g.st(7, wfq::add_nr(g.ld(13), g.ld(13)));           // D = 2 Z1 Z2
    __syncthreads();
    ed_finish(g);
}

// ------------------------------------------------------------------ XYZZ

__device__ __forceinline__ void xyzz_set_inf(const Group& g) {
    g.st(g.w, 0u);
    __syncthreads();
}

// P = 2P: U = 2Y, V = U^2, W = U V, S = X V, M = 3 X^2, X3 = M^2 - 2S,
// Y3 = M (S - X3) - W Y, ZZ3 = V ZZ, ZZZ3 = W ZZZ; levels {V, X^2}, {W, S, V ZZ, M^2},
// {M (S - X3), W Y, W ZZZ}. The identity (ZZ = 0) stays the identity (ZZ3 = 0).
__device__ __forceinline__ void xyzz_dbl(const Group& g) {
    const Consts& K = g.K;
    if (g.w == 0) {
        const uint32_t U = wfq::add(g.ld(Y), g.ld(Y), K);
        g.st(8, U);
        g.st(4, g.mul(U, U));
    }
    if (g.w == 1) g.st(5, g.mul(g.ld(X), g.ld(X)));
    __syncthreads();
    switch (g.w) {
        case 0: g.st(6, g.mul(g.ld(8), g.ld(4))); break;      // W
        case 1: g.st(7, g.mul(g.ld(X), g.ld(4))); break;      // S
        case 2: g.st(ZZ, g.mul(g.ld(4), g.ld(ZZ))); break;    // ZZ3
        default: {
            const uint32_t xx = g.ld(5);
            const uint32_t M = wfq::add(xx, wfq::add(xx, xx, K), K);
            g.st(9, M);
            g.st(10, g.mul(M, M));
        }
    }
    __syncthreads();
    if (g.w == 0) g.st(X, wfq::sub(wfq::sub(g.ld(10), g.ld(7), K), g.ld(7), K));   // X3
    __syncthreads();
    switch (g.w) {
        case 0: g.st(11, g.mul(g.ld(9), wfq::sub(g.ld(7), g.ld(X), K))); break;
        case 1: g.st(12, g.mul(g.ld(6), g.ld(Y))); break;
        case 2: g.st(ZZZ, g.mul(g.ld(6), g.ld(ZZZ))); break;
        default: break;
    }
    __syncthreads();
    if (g.w == 0) g.st(Y, wfq::sub(g.ld(11), g.ld(12), K));
    __syncthreads();
}

// P += Q, Q XYZZ (ZZ = 0 or all-zero words: the identity). Every case: Q = O,
// P = O, Q = P (doubling), Q = -P (the identity).
__device__ __forceinline__ void xyzz_add(const Group& g, const Operand& q) {
    const Consts& K = g.K;
    if (wfq::is_zero(q.c[2], K)) return;
    if (wfq::is_zero(g.ld(ZZ), K)) {
        __syncthreads();                                  // every warp has read ZZ
        g.st(g.w, q.c[g.w & 3]);
        __syncthreads();
        return;
    }
    switch (g.w) {
        case 0: g.st(4, g.mul(g.ld(X), q.c[2])); break;       // U1
        case 1: g.st(5, g.mul(q.c[0], g.ld(ZZ))); break;      // U2
        case 2: g.st(6, g.mul(g.ld(Y), q.c[3])); break;       // S1
        default: g.st(7, g.mul(q.c[1], g.ld(ZZZ)));          // S2
    }
    __syncthreads();
    if (g.w == 0) g.st(8, wfq::sub(g.ld(5), g.ld(4), K));              // P = U2 - U1
    if (g.w == 1) g.st(9, wfq::sub(g.ld(7), g.ld(6), K));              // R = S2 - S1
    __syncthreads();
    if (wfq::is_zero(g.ld(8), K)) {
        const bool same = wfq::is_zero(g.ld(9), K);
        __syncthreads();                                  // every warp has decided
        if (same)
            xyzz_dbl(g);
        else
            xyzz_set_inf(g);
        return;
    }
    switch (g.w) {
        case 0: g.st(10, g.mul(g.ld(8), g.ld(8))); break;     // PP
        case 1: g.st(11, g.mul(g.ld(9), g.ld(9))); break;     // RR
        case 2: g.st(12, g.mul(g.ld(ZZ), q.c[2])); break;     // ZZ1 ZZ2
        default: g.st(13, g.mul(g.ld(ZZZ), q.c[3]));        // ZZZ1 ZZZ2
    }
    __syncthreads();
    switch (g.w) {
        case 0: g.st(14, g.mul(g.ld(8), g.ld(10))); break;    // PPP
        case 1: g.st(15, g.mul(g.ld(4), g.ld(10))); break;    // Q = U1 PP
        case 2: g.st(ZZ, g.mul(g.ld(12), g.ld(10))); break;   // ZZ3
        default: break;
    }
    __syncthreads();
    if (g.w == 0) {
        const uint32_t q2 = wfq::add(g.ld(15), g.ld(15), K);
        g.st(X, wfq::sub(wfq::sub(g.ld(11), g.ld(14), K), q2, K));    // X3 = RR - PPP - 2Q
    }
    __syncthreads();
    switch (g.w) {
        case 0: g.st(16, g.mul(g.ld(9), wfq::sub(g.ld(15), g.ld(X), K))); break;   // R (Q - X3)
        case 1: g.st(17, g.mul(g.ld(6), g.ld(14))); break;                         // S1 PPP
        case 2: g.st(ZZZ, g.mul(g.ld(13), g.ld(14))); break;                       // ZZZ3
        default: break;
    }
    __syncthreads();
    if (g.w == 0) g.st(Y, wfq::sub(g.ld(16), g.ld(17), K));
    __syncthreads();
}

// Full 12-word values of the accumulator for one thread (after a barrier).
__device__ __forceinline__ void read_acc(const Group& g, fq::fe (&c)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 12; ++k) c[i].v[k] = g.s[12 * i + k];
}

}  // namespace wpt
