// BLS12-377 G1 point arithmetic on sm_103a: E: y^2 = x^3 + 1 over Fq.
//
// The paper's PADD (Sec. II-D) is a mixed addition for bucket accumulation and
// a complete addition for bucket aggregation; it works on a twisted Edwards
// model, whose PADD graph (its Fig. 1) is not reproducible from the text. Here
// the same two operations run on the short Weierstrass model in XYZZ
// coordinates (x = X/ZZ, y = Y/ZZZ, ZZ^3 = ZZZ^2; Bernstein-Lange), which give
// the same group elements:
//   madd: XYZZ += affine     8M + 2S
//   add : XYZZ += XYZZ      12M + 2S
//   dbl : 2 * XYZZ           6M + 3S (a = 0)
//   mdbl: 2 * affine -> XYZZ 4M + 3S
// XYZZ formulas are not complete, so every special case is branched on:
// O operands, P + P (falls through to doubling), P + (-P) (gives O).
// The identity is ZZ = ZZZ = 0; the affine identity is (0, 0), which is not on
// the curve. Every coordinate is in Montgomery form and in [0, 2p).
#pragma once
#include "fq.cuh"

namespace ec {

using fq::fe;

struct xyzz {
    fe X, Y, ZZ, ZZZ;
};

struct affine {
    fe x, y;
};

__device__ __forceinline__ void set_inf(xyzz& P) {
    fq::set_zero(P.X);
    fq::set_zero(P.Y);
    fq::set_zero(P.ZZ);
    fq::set_zero(P.ZZZ);
}

__device__ __forceinline__ bool is_inf(const xyzz& P) { return fq::is_zero(P.ZZ); }

__device__ __forceinline__ bool is_inf(const affine& Q) {
    return fq::is_zero_raw(Q.x) && fq::is_zero_raw(Q.y);
}

__device__ __forceinline__ void from_affine(xyzz& P, const affine& Q) {
    if (is_inf(Q)) {
        set_inf(P);
        return;
    }
    P.X = Q.x;
    P.Y = Q.y;
    fq::set_one(P.ZZ);
    fq::set_one(P.ZZZ);
}

__device__ __forceinline__ void neg(affine& Q) {
    if (!is_inf(Q)) fq::neg(Q.y, Q.y);
}

// R = 2 * Q for affine Q: U = 2y, V = U^2, W = U V, S = x V, M = 3x^2,
// X3 = M^2 - 2S, Y3 = M (S - X3) - W y, ZZ3 = V, ZZZ3 = W.
__device__ __forceinline__ void mdbl(xyzz& R, const affine& Q) {
    if (is_inf(Q) || fq::is_zero(Q.y)) {
        set_inf(R);
        return;
    }
    fe U, V, W, S, M, t;
    fq::dbl(U, Q.y);
    fq::sqr(V, U);
    fq::mul(W, U, V);
    fq::mul(S, Q.x, V);
    fq::sqr(t, Q.x);
    fq::dbl(M, t);
    fq::add(M, M, t);
    fq::sqr(R.X, M);
    fq::dbl(t, S);
    fq::sub(R.X, R.X, t);
    fq::sub(t, S, R.X);
    fq::mul(t, M, t);
    fq::mul(R.Y, W, Q.y);
    fq::sub(R.Y, t, R.Y);
    R.ZZ = V;
    R.ZZZ = W;
}

// P = 2 P: U = 2Y, V = U^2, W = U V, S = X V, M = 3X^2,
// X3 = M^2 - 2S, Y3 = M (S - X3) - W Y, ZZ3 = V ZZ, ZZZ3 = W ZZZ.
// Y = 0 gives V = 0 and so ZZ3 = 0 (the identity) without a branch.
// Independent products go in pairs through fq::mul2 (four carry chains in flight).
__device__ __forceinline__ void dbl(xyzz& P) {
    if (is_inf(P)) return;
    fe U, V, W, M, t;
    fq::dbl(U, P.Y);
    fq::mul2(V, U, U, t, P.X, P.X);          // V = U^2, X^2
    fq::dbl(M, t);
    fq::add(M, M, t);                        // M = 3 X^2
    fq::mul2(W, U, V, U, P.X, V);            // W = U V, S = X V (in U's slot)
    fq::mul2(P.ZZ, P.ZZ, V, t, M, M);        // ZZ3 = ZZ V, M^2
    fq::mul2(P.ZZZ, P.ZZZ, W, P.Y, W, P.Y);  // ZZZ3 = ZZZ W, W Y
    fq::dbl(V, U);                           // 2S
    fq::sub(P.X, t, V);                      // X3
    fq::sub(t, U, P.X);                      // S - X3
    fq::mul(t, M, t);
    fq::sub(P.Y, t, P.Y);                    // Y3
}

// P += Q (Q affine). `p_inf` says P is the identity (kept by the caller).
// U2 = x2 ZZ1, S2 = y2 ZZZ1, Pd = U2 - X1, R = S2 - Y1, PP = Pd^2, PPP = Pd PP,
// Q1 = X1 PP, X3 = R^2 - PPP - 2 Q1, Y3 = R (Q1 - X3) - Y1 PPP,
// ZZ3 = ZZ1 PP, ZZZ3 = ZZZ1 PPP.
__device__ __forceinline__ void madd(xyzz& P, bool& p_inf, const affine& Q) {
    if (is_inf(Q)) return;
    if (p_inf) {
        from_affine(P, Q);
        p_inf = false;
        return;
    }
    fe U2, S2, Pd, R;
    fq::mul2(U2, Q.x, P.ZZ, S2, Q.y, P.ZZZ);
    fq::sub(Pd, U2, P.X);
    fq::sub(R, S2, P.Y);
    if (fq::is_zero(Pd)) {
        if (fq::is_zero(R)) {
            mdbl(P, Q);
            p_inf = is_inf(P);
        } else {
            set_inf(P);
            p_inf = true;
        }
        return;
    }
    fe PP, PPP, Q1, t;
    fq::mul2(PP, Pd, Pd, t, R, R);              // PP, R^2
    fq::mul2(PPP, Pd, PP, Q1, P.X, PP);
    fq::mul2(P.ZZ, P.ZZ, PP, P.ZZZ, P.ZZZ, PPP);
    fq::sub(P.X, t, PPP);
    fq::dbl(t, Q1);
    fq::sub(P.X, P.X, t);       // X3
    fq::sub(t, Q1, P.X);
    fq::mul2(PPP, P.Y, PPP, t, R, t);           // Y1 PPP, R (Q1 - X3)
    fq::sub(P.Y, t, PPP);
}

__device__ __forceinline__ void madd(xyzz& P, const affine& Q) {
    bool inf = is_inf(P);
    madd(P, inf, Q);
}

// Second operand of add_q() held in registers.
struct RegQ {
    const xyzz* q;
    __device__ __forceinline__ void X(fe& r) const { r = q->X; }
    __device__ __forceinline__ void Y(fe& r) const { r = q->Y; }
    __device__ __forceinline__ void ZZ(fe& r) const { r = q->ZZ; }
    __device__ __forceinline__ void ZZZ(fe& r) const { r = q->ZZZ; }
    __device__ __forceinline__ void all(xyzz& r) const { r = *q; }
};

// P += Q (both XYZZ); Q's coordinates are fetched through `q` when needed, so a
// Q in memory never occupies registers, and P's slots are reused once X1, Y1 die.
// U1 = X1 ZZ2, U2 = X2 ZZ1, S1 = Y1 ZZZ2, S2 = Y2 ZZZ1, Pd = U2 - U1,
// R = S2 - S1, PP = Pd^2, PPP = Pd PP, Q1 = U1 PP, X3 = R^2 - PPP - 2 Q1,
// Y3 = R (Q1 - X3) - S1 PPP, ZZ3 = ZZ1 ZZ2 PP, ZZZ3 = ZZZ1 ZZZ2 PPP.
template <class QL>
__device__ __forceinline__ void add_q(xyzz& P, const QL& q) {
    fe t, u, Pd, R;
    q.ZZ(t);
    if (fq::is_zero(t)) return;     // Q = O
    if (is_inf(P)) {
        q.all(P);
        return;
    }
    fq::mul(P.X, P.X, t);           // U1
    q.X(u);
    fq::mul(u, u, P.ZZ);            // U2
    fq::sub(Pd, u, P.X);
    q.ZZZ(t);
    fq::mul(P.Y, P.Y, t);           // S1
    q.Y(u);
    fq::mul(u, u, P.ZZZ);           // S2
    fq::sub(R, u, P.Y);
    if (fq::is_zero(Pd)) {
        if (fq::is_zero(R)) {
            q.all(P);               // P = Q: the sum is 2Q
            dbl(P);
        } else {
            set_inf(P);
        }
        return;
    }
    fq::sqr(u, Pd);                 // PP
    fq::mul(Pd, Pd, u);             // PPP in Pd's slot
    fq::mul(P.X, P.X, u);           // Q1 in X's slot
    q.ZZ(t);
    fq::mul(P.ZZ, P.ZZ, t);
    fq::mul(P.ZZ, P.ZZ, u);         // ZZ3
    q.ZZZ(t);
    fq::mul(P.ZZZ, P.ZZZ, t);
    fq::mul(P.ZZZ, P.ZZZ, Pd);      // ZZZ3
    fq::dbl(u, P.X);
    fq::add(u, u, Pd);              // 2 Q1 + PPP
    fq::mul(Pd, P.Y, Pd);           // S1 PPP
    fq::sqr(t, R);
    fq::sub(t, t, u);               // X3
    fq::sub(u, P.X, t);             // Q1 - X3
    P.X = t;
    fq::mul(u, R, u);
    fq::sub(P.Y, u, Pd);            // Y3
}

__device__ __forceinline__ void add(xyzz& P, const xyzz& Q) { add_q(P, RegQ{&Q}); }

// ---- four lanes per point operation (latency-bound chains)
//
// A dependent chain of point operations (the window combination, the per-window
// Horner sums) runs at the latency of one thread's multiplications. The
// multiplications inside one formula fall into a few levels of independent
// products, so four lanes of a warp that hold the same point each compute one
// product of a level and exchange the results through shared memory. Every lane
// of the warp calls these functions (lanes of the same group of four hold the same
// values, so every branch is uniform within a group); `sh` is the group's
// four-element shared slot and `l` = lane % 4.

__device__ __forceinline__ void xchg4(fe (&v)[4], const fe& mine, fe* sh, int l, bool writer) {
    if (writer) sh[l] = mine;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = sh[k];
    __syncwarp();
}

// Word-wise select by lane role (no addresses taken, so everything stays in registers).
__device__ __forceinline__ fe pick4(int l, const fe& a, const fe& b, const fe& c, const fe& d) {
    fe r;
#pragma unroll
    for (int k = 0; k < fq::N; ++k)
        r.v[k] = l == 0 ? a.v[k] : (l == 1 ? b.v[k] : (l == 2 ? c.v[k] : d.v[k]));
    return r;
}

// P = 2P in three levels: {U^2 (U = 2Y), X^2}, {U V, X V, ZZ V, M^2 (M = 3X^2)},
// {ZZZ W, W Y, M (S - X3)}: three multiplication latencies instead of nine. The
// identity (ZZ = 0) and Y = 0 give ZZ3 = ZZ V = 0 without a branch.
__device__ __forceinline__ void dbl4(xyzz& P, fe* sh, int l, bool writer) {
    fe U, r, v[4];
    fq::dbl(U, P.Y);
    fe x = pick4(l, U, P.X, U, P.X);
    fq::sqr(r, x);
    xchg4(v, r, sh, l, writer);     // V, X^2
    fe V = v[0], M, t;
    fq::dbl(M, v[1]);
    fq::add(M, M, v[1]);            // M = 3 X^2
    x = pick4(l, U, P.X, P.ZZ, M);
    fe y = pick4(l, V, V, V, M);
    fq::mul(r, x, y);
    xchg4(v, r, sh, l, writer);     // W, S, ZZ3, M^2
    fe W = v[0], S = v[1];
    P.ZZ = v[2];
    fq::dbl(t, S);
    fq::sub(P.X, v[3], t);          // X3 = M^2 - 2S
    fq::sub(t, S, P.X);             // S - X3
    x = pick4(l, P.ZZZ, W, M, M);
    y = pick4(l, W, P.Y, t, t);
    fq::mul(r, x, y);
    xchg4(v, r, sh, l, writer);     // ZZZ3, W Y, M (S - X3)
    P.ZZZ = v[0];
    fq::sub(P.Y, v[2], v[1]);       // Y3
}

// P += Q (both XYZZ, Q through a loader) in four levels: {U1, U2, S1, S2},
// {PP = Pd^2, R^2, ZZ1 ZZ2, ZZZ1 ZZZ2}, {PPP, Q1 = U1 PP, ZZ3}, {ZZZ3, S1 PPP,
// R (Q1 - X3)}. Groups of one warp may hold different points, so every group runs
// the same exchanges (a __syncwarp is warp-wide): the special cases (Q = O, P = O,
// P = -Q, P = Q) are computed alongside and chosen by selects, and the doubling
// that P = Q needs runs, for every group, only when some group of the warp needs it.
__device__ __forceinline__ void select(xyzz& P, bool take, const xyzz& Q) {
#pragma unroll
    for (int k = 0; k < fq::N; ++k) {
        P.X.v[k] = take ? Q.X.v[k] : P.X.v[k];
        P.Y.v[k] = take ? Q.Y.v[k] : P.Y.v[k];
        P.ZZ.v[k] = take ? Q.ZZ.v[k] : P.ZZ.v[k];
        P.ZZZ.v[k] = take ? Q.ZZZ.v[k] : P.ZZZ.v[k];
    }
}

template <class QL>
__device__ __forceinline__ void add4(xyzz& P, const QL& q, fe* sh, int l, bool writer) {
    xyzz Q;
    q.all(Q);
    const bool q_inf = fq::is_zero(Q.ZZ), p_inf = is_inf(P);
    fe r, v[4];
    fe x = pick4(l, P.X, Q.X, P.Y, Q.Y);
    fe y = pick4(l, Q.ZZ, P.ZZ, Q.ZZZ, P.ZZZ);
    fq::mul(r, x, y);
    xchg4(v, r, sh, l, writer);     // U1, U2, S1, S2
    const fe U1 = v[0], S1 = v[2];
    fe Pd, R;
    fq::sub(Pd, v[1], U1);
    fq::sub(R, v[3], S1);
    const bool same_x = !q_inf && !p_inf && fq::is_zero(Pd);
    const bool doubling = same_x && fq::is_zero(R);     // P = Q
    const bool cancel = same_x && !doubling;            // P = -Q
    xyzz D = Q;
    if (__any_sync(0xffffffffu, doubling)) dbl4(D, sh, l, writer);  // warp-uniform branch
    xyzz S = P;
    x = pick4(l, Pd, R, P.ZZ, P.ZZZ);
    y = pick4(l, Pd, R, Q.ZZ, Q.ZZZ);
    fq::mul(r, x, y);
    xchg4(v, r, sh, l, writer);     // PP, R^2, ZZ1 ZZ2, ZZZ1 ZZZ2
    const fe PP = v[0], RR = v[1], Z12 = v[2], ZZZ12 = v[3];
    x = pick4(l, Pd, U1, Z12, Z12);
    y = pick4(l, PP, PP, PP, PP);
    fq::mul(r, x, y);
    xchg4(v, r, sh, l, writer);     // PPP, Q1, ZZ3
    const fe PPP = v[0], Q1 = v[1];
    S.ZZ = v[2];
    fe t;
    fq::sub(S.X, RR, PPP);
    fq::dbl(t, Q1);
    fq::sub(S.X, S.X, t);           // X3 = R^2 - PPP - 2 Q1
    fq::sub(t, Q1, S.X);            // Q1 - X3
    x = pick4(l, ZZZ12, S1, R, R);
    y = pick4(l, PPP, PPP, t, t);
    fq::mul(r, x, y);
    xchg4(v, r, sh, l, writer);     // ZZZ3, S1 PPP, R (Q1 - X3)
    S.ZZZ = v[0];
    fq::sub(S.Y, v[2], v[1]);       // Y3
    xyzz O;
    set_inf(O);
    select(S, doubling, D);
    select(S, cancel, O);
    select(S, p_inf, Q);
    select(S, q_inf, P);
    P = S;
}

// Inverse by the optimized binary GCD of T. Pornin ("Optimized Binary GCD for
// Modular Inversion", 2020): the binary extended GCD on (a, b) = (y, p), but 31
// steps at a time on 64-bit approximations of a and b (their top 33 and low 31
// bits), which fix an update matrix (f0 g0; f1 g1) with entries of at most 2^31
// in magnitude; the matrix is then applied once to the full a, b and to the
// Bezout coefficients u, v (a = u y, b = v y mod p), dividing by 2^31 (exact for
// a, b; mod p for u, v, where x / 2^31 = (x + m p) / 2^31 with m = -x mod 2^31
// because p = 1 mod 2^31). ceil((2 * 377 - 1) / 31) = 25 rounds bring a to 0 and
// b to 1 = gcd, and then v = y^-1. For u = aR (Montgomery form) that is
// a^-1 R^-1, and one Montgomery multiplication by R^3 mod p turns it into a^-1 R.
// Variable time (MSM results are public); every loop has a fixed trip count.
namespace detail {
constexpr int W = 12;

// r (13 words, two's complement) = f x + g y for |f|, |g| <= 2^31 and x, y < 2^384.
__device__ __forceinline__ void lin_comb(uint32_t (&r)[W + 1], const uint32_t (&x)[W], const uint32_t (&y)[W],
                                         int64_t f, int64_t g) {
    const uint32_t fa = (uint32_t)(f < 0 ? -f : f), ga = (uint32_t)(g < 0 ? -g : g);
    uint32_t px[W + 1], py[W + 1];
    uint64_t cx = 0, cy = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        uint64_t t = (uint64_t)fa * x[k] + cx;
        px[k] = (uint32_t)t;
        cx = t >> 32;
        uint64_t u = (uint64_t)ga * y[k] + cy;
        py[k] = (uint32_t)u;
        cy = u >> 32;
    }
    px[W] = (uint32_t)cx;
    py[W] = (uint32_t)cy;
    // r = (+-px) + (+-py) in 13-word two's complement (|r| < 2^416 fits)
    const uint32_t nx = f < 0 ? 0xffffffffu : 0u, ny = g < 0 ? 0xffffffffu : 0u;
    uint64_t carry = (nx ? 1u : 0u) + (ny ? 1u : 0u);  // two's complement: ~v + 1
#pragma unroll
    for (int k = 0; k <= W; ++k) {
        uint64_t t = (uint64_t)(px[k] ^ nx) + (py[k] ^ ny) + carry;
        r[k] = (uint32_t)t;
        carry = t >> 32;
    }
}

// x = r >> 31 (r's low 31 bits are zero), made non-negative; returns true if r < 0.
__device__ __forceinline__ bool shift31_abs(uint32_t (&x)[W], uint32_t (&r)[W + 1]) {
    const bool neg = (r[W] >> 31) != 0;
    if (neg) {
        uint64_t carry = 1;
#pragma unroll
        for (int k = 0; k <= W; ++k) {
            uint64_t t = (uint64_t)(~r[k]) + carry;
            r[k] = (uint32_t)t;
            carry = t >> 32;
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) x[k] = (r[k] >> 31) | (r[k + 1] << 1);
    return neg;
}

// u = (f u0 + g v0) / 2^31 mod p in [0, p), for u0, v0 in [0, p) and |f|, |g| <= 2^31.
__device__ __forceinline__ void lin_comb_mod(uint32_t (&u)[W], const uint32_t (&u0)[W], const uint32_t (&v0)[W],
                                             int64_t f, int64_t g) {
    uint32_t r[W + 1];
    lin_comb(r, u0, v0, f, g);          // |r| < 2^32 p
    // + 2^32 p: r > 0, below 2^33 p < 2^411 (words 1..12 of 2^32 p are p's words)
    uint64_t carry = 0;
#pragma unroll
    for (int k = 0; k <= W; ++k) {
        uint64_t t = (uint64_t)r[k] + (k >= 1 ? fq::kP[k - 1] : 0u) + carry;
        r[k] = (uint32_t)t;
        carry = t >> 32;
    }
    // + m p with m = -r mod 2^31 makes the low 31 bits zero (p = 1 mod 2^31)
    const uint32_t m = (0u - r[0]) & 0x7fffffffu;
    uint32_t s[W + 2];
    carry = 0;
#pragma unroll
    for (int k = 0; k <= W; ++k) {
        uint64_t t = (uint64_t)r[k] + (k < W ? (uint64_t)m * fq::kP[k] : 0u) + carry;
        s[k] = (uint32_t)t;
        carry = t >> 32;
    }
    s[W + 1] = (uint32_t)carry;
    // / 2^31: below (2^33 p + 2^31 p) / 2^31 = 5 p
#pragma unroll
    for (int k = 0; k < W; ++k) u[k] = (s[k] >> 31) | (s[k + 1] << 1);
    // subtract 4p, 2p, p where possible
#pragma unroll
    for (int mult = 4; mult >= 1; mult >>= 1) {
        uint32_t d[W];
        uint64_t borrow = 0, cm = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            uint64_t pk = (uint64_t)fq::kP[k] * mult + cm;
            cm = pk >> 32;
            uint64_t t = (uint64_t)u[k] - (uint32_t)pk - borrow;
            d[k] = (uint32_t)t;
            borrow = (t >> 63) & 1u;
        }
        if (!borrow && cm == 0) {
#pragma unroll
            for (int k = 0; k < W; ++k) u[k] = d[k];
        }
    }
}
}  // namespace detail

__device__ __noinline__ static void inv(fe& r, const fe& a_in) {
    using namespace detail;
    fe a;
    fq::canon(a, a_in);
    uint32_t A[W], B[W], U[W], V[W];
    uint32_t z = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        A[k] = a.v[k];
        B[k] = fq::kP[k];
        U[k] = 0;
        V[k] = 0;
        z |= a.v[k];
    }
    U[0] = 1;
    if (z == 0) {
        fq::set_zero(r);
        return;
    }
    for (int round = 0; round < 25; ++round) {
        // bit length n = max(len A, len B, 64) and the 64-bit approximations
        int top = 0;
#pragma unroll
        for (int k = 0; k < W; ++k)
            if (A[k] | B[k]) top = k;
        const uint32_t hiw = A[top] | B[top];
        const int n = 32 * top + (32 - __clz(hiw));
        uint64_t ah, bh;
        if (n <= 64) {
            ah = ((uint64_t)A[1] << 32) | A[0];
            bh = ((uint64_t)B[1] << 32) | B[0];
        } else {
            const int sbit = n - 33, idx = sbit >> 5, sh = sbit & 31;
            uint32_t alo = 0, ahi = 0, blo = 0, bhi = 0;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (k == idx) { alo = A[k]; blo = B[k]; }
                if (k == idx + 1) { ahi = A[k]; bhi = B[k]; }
            }
            const uint64_t at = ((((uint64_t)ahi << 32) | alo) >> sh) & 0x1ffffffffull;
            const uint64_t bt = ((((uint64_t)bhi << 32) | blo) >> sh) & 0x1ffffffffull;
            ah = (at << 31) | (A[0] & 0x7fffffffu);
            bh = (bt << 31) | (B[0] & 0x7fffffffu);
        }
        int64_t f0 = 1, g0 = 0, f1 = 0, g1 = 1;
#pragma unroll 1
        for (int i = 0; i < 31; ++i) {
            if (ah & 1) {
                if (ah < bh) {
                    uint64_t t = ah; ah = bh; bh = t;
                    int64_t tf = f0; f0 = f1; f1 = tf;
                    int64_t tg = g0; g0 = g1; g1 = tg;
                }
                ah -= bh;
                f0 -= f1;
                g0 -= g1;
            }
            ah >>= 1;
            f1 <<= 1;
            g1 <<= 1;
        }
        uint32_t ra[W + 1], rb[W + 1];
        lin_comb(ra, A, B, f0, g0);
        lin_comb(rb, A, B, f1, g1);
        if (shift31_abs(A, ra)) { f0 = -f0; g0 = -g0; }
        if (shift31_abs(B, rb)) { f1 = -f1; g1 = -g1; }
        uint32_t U2[W], V2[W];
        lin_comb_mod(U2, U, V, f0, g0);
        lin_comb_mod(V2, U, V, f1, g1);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            U[k] = U2[k];
            V[k] = V2[k];
        }
    }
    fe x, r3;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        x.v[k] = V[k];
        r3.v[k] = fq::kR3[k];
    }
    fq::mul(r, x, r3);  // a^-1 R^-1 * R^3 * R^-1 = a^-1 R
}

// Affine result in Montgomery form, canonical [0, p); O gives (0, 0).
// One inversion: I = (ZZ ZZZ)^-1, x = X ZZZ I, y = Y ZZ I.
__device__ __forceinline__ void to_affine(affine& A, const xyzz& P) {
    if (is_inf(P)) {
        fq::set_zero(A.x);
        fq::set_zero(A.y);
        return;
    }
    fe I, t;
    fq::mul(t, P.ZZ, P.ZZZ);
    inv(I, t);
    fq::mul(t, P.ZZZ, I);
    fq::mul(A.x, P.X, t);
    fq::canon(A.x, A.x);
    fq::mul(t, P.ZZ, I);
    fq::mul(A.y, P.Y, t);
    fq::canon(A.y, A.y);
}

}  // namespace ec
