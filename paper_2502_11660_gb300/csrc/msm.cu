// Pippenger multi-scalar multiplication over BLS12-377 G1 (Sec. II-C of the
// paper: windows, bucket accumulation, bucket aggregation, group aggregation),
// laid out for one GB300.
//
// Stages:
//  1. prepare     standard affine -> Montgomery affine (96 B per point, AoS, so a
//                 random gather of one point reads three full 32 B sectors)
//  2. digits      c-bit window digits per scalar (signed or unsigned);
//                 key = |digit|, value = point index | sign << 31, window-major
//  3. sort        bucket order within each window: a counting sort over (window,
//                 key) bins (count, scan, scatter with warp-aggregated atomics) for
//                 few windows or wide keys, else a stable LSD radix sort with 8-bit
//                 digits per pass (histogram, scans, ranked scatter)
//  4. accumulate  per window, the sorted stream is cut into equal chunks of K
//                 items, one per thread, so heavy buckets spread over threads;
//                 runs inside a chunk are summed with mixed PADDs and written
//                 to their bucket, runs
//                 crossing a chunk edge leave partial sums
//  5. merge       partial sums of runs that cross chunk edges are added up
//  6. reduce      per window sum_b b * B_b: segments of L buckets by running sums
//                 in-thread, then sum_g g * Y_g split by the bits of g into
//                 independent sums, recombined by Horner
//  7. combine     sum_j 2^(c j) S_j by Horner over windows, one inversion,
//                 affine standard form
//
// Everything runs on the caller's stream, one launch per stage over all windows.
//
// Two curve models run the same pipeline (a template parameter of every point
// kernel): short Weierstrass XYZZ (default; any points on the curve) and the
// paper's twisted Edwards model in extended coordinates (MSM377_EDWARDS; 7M
// mixed additions, points of the order-r subgroup). MSM377_GLV splits every
// scalar k = k1 + lambda k2 (lambda = x0^2 - 1, 127-bit halves) and runs the
// pipeline over the 2n points P_i, phi(P_i) = (beta x_i, y_i) with half the
// windows (subgroup points); stored rows 2i and 2i + 1 are P_i and phi(P_i).
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "common.cuh"
#include "ec.cuh"
#include "ed.cuh"
#include "wpt.cuh"

namespace {

using ec::affine;
using ec::xyzz;
using fq::fe;

constexpr uint32_t kNone = 0xffffffffu;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048
constexpr int kXyzzVec = 12;                // XYZZ in memory: 4 x 12 packed words = 12 uint4
constexpr size_t kXyzzBytes = kXyzzVec * 16;

// ---------------------------------------------------------------- memory I/O

__device__ __forceinline__ void load_affine(affine& Q, const uint4* __restrict__ pts, uint32_t idx) {
    const uint4* p = pts + 6 * (size_t)idx;
    uint4 a = __ldg(p + 0), b = __ldg(p + 1), c = __ldg(p + 2);
    uint4 d = __ldg(p + 3), e = __ldg(p + 4), f = __ldg(p + 5);
    Q.x.v[0] = a.x; Q.x.v[1] = a.y; Q.x.v[2] = a.z; Q.x.v[3] = a.w;
    Q.x.v[4] = b.x; Q.x.v[5] = b.y; Q.x.v[6] = b.z; Q.x.v[7] = b.w;
    Q.x.v[8] = c.x; Q.x.v[9] = c.y; Q.x.v[10] = c.z; Q.x.v[11] = c.w;
    Q.y.v[0] = d.x; Q.y.v[1] = d.y; Q.y.v[2] = d.z; Q.y.v[3] = d.w;
    Q.y.v[4] = e.x; Q.y.v[5] = e.y; Q.y.v[6] = e.z; Q.y.v[7] = e.w;
    Q.y.v[8] = f.x; Q.y.v[9] = f.y; Q.y.v[10] = f.z; Q.y.v[11] = f.w;
}

__device__ __forceinline__ void load_fe(fe& a, const uint4* p) {
    uint4 u0 = p[0], u1 = p[1], u2 = p[2];
    a.v[0] = u0.x; a.v[1] = u0.y; a.v[2] = u0.z; a.v[3] = u0.w;
    a.v[4] = u1.x; a.v[5] = u1.y; a.v[6] = u1.z; a.v[7] = u1.w;
    a.v[8] = u2.x; a.v[9] = u2.y; a.v[10] = u2.z; a.v[11] = u2.w;
}

__device__ __forceinline__ void store_fe(uint4* p, const fe& a) {
    p[0] = make_uint4(a.v[0], a.v[1], a.v[2], a.v[3]);
    p[1] = make_uint4(a.v[4], a.v[5], a.v[6], a.v[7]);
    p[2] = make_uint4(a.v[8], a.v[9], a.v[10], a.v[11]);
}

// XYZZ point in memory: 12 uint4 (X, Y, ZZ, ZZZ), each coordinate in [0, 2p).
__device__ __forceinline__ void load_xyzz(xyzz& P, const uint4* p) {
    load_fe(P.X, p);
    load_fe(P.Y, p + 3);
    load_fe(P.ZZ, p + 6);
    load_fe(P.ZZZ, p + 9);
}

__device__ __forceinline__ void store_xyzz(uint4* p, const xyzz& P) {
    store_fe(p, P.X);
    store_fe(p + 3, P.Y);
    store_fe(p + 6, P.ZZ);
    store_fe(p + 9, P.ZZZ);
}

// Second operand of ec::add_q() read from memory coordinate by coordinate.
struct MemQ {
    const uint4* p;
    __device__ __forceinline__ void X(fe& r) const { load_fe(r, p); }
    __device__ __forceinline__ void Y(fe& r) const { load_fe(r, p + 3); }
    __device__ __forceinline__ void ZZ(fe& r) const { load_fe(r, p + 6); }
    __device__ __forceinline__ void ZZZ(fe& r) const { load_fe(r, p + 9); }
    __device__ __forceinline__ void all(xyzz& r) const { load_xyzz(r, p); }
};

// Second operand of ed::add_q() read from memory: (X, Y, Z, T) as 12 uint4.
struct MemQE {
    const uint4* p;
    __device__ __forceinline__ void X(fe& r) const { load_fe(r, p); }
    __device__ __forceinline__ void Y(fe& r) const { load_fe(r, p + 3); }
    __device__ __forceinline__ void Z(fe& r) const { load_fe(r, p + 6); }
    __device__ __forceinline__ void T(fe& r) const { load_fe(r, p + 9); }
};

// ---------------------------------------------------------------- curve models
//
// What the pipeline needs from a curve model: the stored form of an input point
// (kStored uint4 per point), a mixed addition of a gathered stored point, a full
// addition from memory or registers, a doubling, and the affine Weierstrass
// result. Accumulators of both models are four 12-word coordinates, 12 uint4 in
// memory. A bucket that received no point is all-zero words in memory: XYZZ
// reads that as its identity (ZZ = 0); the Edwards loader skips it.

struct ModelXyzz {
    using acc = xyzz;
    static constexpr int kDblDepth = 3, kAddDepth = 4;  // multiplication levels of dbl4 / add4
    static constexpr int kAccBlocks = 3;  // accumulation blocks of 128 per SM (<= 168 registers)
    static constexpr int kStored = 6;  // affine (x, y)
    static __device__ __forceinline__ void set_inf(acc& P) { ec::set_inf(P); }
    static __device__ __forceinline__ void load(acc& P, const uint4* p) { load_xyzz(P, p); }
    static __device__ __forceinline__ void store(uint4* p, const acc& P) { store_xyzz(p, P); }
    static __device__ __forceinline__ void madd_at(acc& P, bool& inf, const uint4* pts, uint32_t idx, bool negate) {
        affine Q;
        load_affine(Q, pts, idx);
        if (negate) ec::neg(Q);
        ec::madd(P, inf, Q);
    }
    static __device__ __forceinline__ void add_mem(acc& P, const uint4* q) { ec::add_q(P, MemQ{q}); }
    static __device__ __forceinline__ void add(acc& P, const acc& Q) { ec::add(P, Q); }
    static __device__ __forceinline__ void dbl(acc& P) { ec::dbl(P); }
    static __device__ __forceinline__ void to_affine(affine& A, const acc& P) { ec::to_affine(A, P); }
    static __device__ __forceinline__ void dbl4(acc& P, fe* sh, int l) { ec::dbl4(P, sh, l, true); }
    static __device__ __forceinline__ void add4_mem(acc& P, const uint4* q, fe* sh, int l) {
        ec::add4(P, MemQ{q}, sh, l, true);
    }
    // four-warp group operations (wpt.cuh)
    static __device__ __forceinline__ void gset_inf(const wpt::Group& g) { wpt::xyzz_set_inf(g); }
    static __device__ __forceinline__ void gdbl(const wpt::Group& g) { wpt::xyzz_dbl(g); }
    static __device__ __forceinline__ void gadd(const wpt::Group& g, const wpt::Operand& q) { wpt::xyzz_add(g, q); }
    static __device__ __forceinline__ void to_affine4(affine& A, const fe (&c)[4]) {
        xyzz P;
        P.X = c[0];
        P.Y = c[1];
        P.ZZ = c[2];
        P.ZZZ = c[3];
        ec::to_affine(A, P);
    }
};

struct ModelEdwards {
    using acc = ed::ext;
    static constexpr int kDblDepth = 2, kAddDepth = 3;  // multiplication levels of dbl4 / add4
    static constexpr int kAccBlocks = 4;  // accumulation blocks of 128 per SM (<= 128 registers)
    static constexpr int kStored = 9;  // (x, y, u = k x y), the paper's (X, Y, U) with Z = 1
    static __device__ __forceinline__ void set_inf(acc& P) { ed::set_inf(P); }
    static __device__ __forceinline__ void load(acc& P, const uint4* p) {
        load_fe(P.X, p);
        load_fe(P.Y, p + 3);
        load_fe(P.Z, p + 6);
        load_fe(P.T, p + 9);
    }
    static __device__ __forceinline__ void store(uint4* p, const acc& P) {
        store_fe(p, P.X);
        store_fe(p + 3, P.Y);
        store_fe(p + 6, P.Z);
        store_fe(p + 9, P.T);
    }
    static __device__ __forceinline__ void madd_at(acc& P, bool& inf, const uint4* pts, uint32_t idx, bool negate) {
        ed::stored Q;
        const uint4* q = pts + (size_t)kStored * idx;
        load_fe(Q.x, q);
        load_fe(Q.y, q + 3);
        load_fe(Q.u, q + 6);
        if (negate) ed::neg(Q);
        ed::madd(P, inf, Q);
    }
    static __device__ __forceinline__ void add_mem(acc& P, const uint4* q) {
        fe z;
        load_fe(z, q + 6);
        if (fq::is_zero_raw(z)) return;  // empty bucket
        ed::add_q(P, MemQE{q});
    }
    static __device__ __forceinline__ void add(acc& P, const acc& Q) { ed::add(P, Q); }
    static __device__ __forceinline__ void dbl(acc& P) { ed::dbl(P); }
    static __device__ __forceinline__ void to_affine(affine& A, const acc& P) { ed::to_weierstrass(A, P); }
    static __device__ __forceinline__ void dbl4(acc& P, fe* sh, int l) { ed::dbl4(P, sh, l, true); }
    static __device__ __forceinline__ void add4_mem(acc& P, const uint4* q, fe* sh, int l) {
        ed::add4(P, MemQE{q}, sh, l, true);
    }
    static __device__ __forceinline__ void gset_inf(const wpt::Group& g) { wpt::ed_set_inf(g); }
    static __device__ __forceinline__ void gdbl(const wpt::Group& g) { wpt::ed_dbl(g); }
    static __device__ __forceinline__ void gadd(const wpt::Group& g, const wpt::Operand& q) { wpt::ed_add(g, q); }
    static __device__ __forceinline__ void to_affine4(affine& A, const fe (&c)[4]) {
        ed::ext P;
        P.X = c[0];
        P.Y = c[1];
        P.Z = c[2];
        P.T = c[3];
        ed::to_weierstrass(A, P);
    }
};

// ---------------------------------------------------------------- stage 1

// beta, a primitive cube root of unity in Fq with (beta x, y) = lambda (x, y) on
// the order-r subgroup (Montgomery form).
__device__ __constant__ static const uint32_t kBeta[fq::N] = {
    0xa5847973u, 0xdacd106du, 0xbac2a79au, 0xd8fe2454u, 0xfd832edcu, 0x1ada4fd6u,
    0x9d150908u, 0xfb986844u, 0xea32285eu, 0xd63eb8aeu, 0x6f873fd0u, 0x0167d6a3u};

// Stored point i of np in Montgomery form: input point i when np = n; with GLV
// (np = 2n) rows 2j and 2j + 1 are P_j and phi(P_j) = (beta x_j, y_j), so any
// contiguous range of input points is a contiguous range of stored rows. The
// affine identity (0, 0) stays (0, 0).
__device__ __forceinline__ void glv_source(fe& x, fe& y, const uint4* __restrict__ in, size_t i, size_t n,
                                           size_t np) {
    const bool split = np != n;
    const size_t src = split ? i >> 1 : i;
    load_fe(x, in + 6 * src);
    load_fe(y, in + 6 * src + 3);
    fq::to_mont(x, x);
    fq::to_mont(y, y);
    if (split && (i & 1)) {
        fe b;
        ed::load_const(b, kBeta);
        fq::mul(x, x, b);
        fq::canon(x, x);
    }
}

// Stored rows [lo, hi) of np (the whole set: lo = 0, hi = np).
__global__ void k_prepare(const uint4* __restrict__ in, uint4* __restrict__ out, size_t n, size_t np, size_t lo,
                          size_t hi) {
    size_t i = lo + blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= hi) return;
    fe x, y;
    glv_source(x, y, in, i, n, np);
    store_fe(out + 6 * i, x);
    store_fe(out + 6 * i + 3, y);
}

// Weierstrass -> Edwards stored form. For (x_w, y_w), with a = x_w + 1:
//   D = y_w (a + s),  x = c1 a (a + s) / D,  y = (a - s) y_w / D,  u = k x y.
// The affine identity, and points outside the map's domain (D = 0: order 2 or 4,
// never in the subgroup), become the Edwards identity (0, 1, 0).
//
// ed_affine_chunk (used by the fixed-base precomputation) takes kEdChunk points
// per lane in registers: one inversion per warp (Montgomery's trick twice: each
// thread multiplies the D of its kEdChunk points, a warp scan multiplies the
// threads' products, lane 0 inverts the warp's total, and prefix and suffix
// products hand every thread the inverse of its own product, from which it walks
// back through its chunk). k_prepare_ed, below, is the same map arranged for the
// preparation of whole sets.
constexpr int kEdChunk = 8;
// The GLV pair path of ed_affine_chunk needs every lane's first row and row count
// even (pairs P, phi(P) never straddle two lanes).
static_assert(kEdChunk % 2 == 0, "kEdChunk must be even");

__device__ __forceinline__ fe shfl_fe_up(const fe& a, int off) {
    fe r;
#pragma unroll
    for (int k = 0; k < fq::N; ++k) r.v[k] = __shfl_up_sync(0xffffffffu, a.v[k], off);
    return r;
}

__device__ __forceinline__ fe shfl_fe_down(const fe& a, int off) {
    fe r;
#pragma unroll
    for (int k = 0; k < fq::N; ++k) r.v[k] = __shfl_down_sync(0xffffffffu, a.v[k], off);
    return r;
}

__device__ __forceinline__ fe shfl_fe(const fe& a, int src) {
    fe r;
#pragma unroll
    for (int k = 0; k < fq::N; ++k) r.v[k] = __shfl_sync(0xffffffffu, a.v[k], src);
    return r;
}

// The inverse of every lane's acc (nonzero on every lane) with one field inversion
// for the warp: prefix products P_l = acc_0 ... acc_l and suffix products
// S_l = acc_{l+1} ... acc_31 over the lanes give acc_l^-1 = total^-1 P_{l-1} S_l.
// Every lane of the warp must call it.
__device__ __forceinline__ fe warp_lane_inverse(const fe& acc) {
    const int lane = threadIdx.x & 31;
    fe one;
    fq::set_one(one);
    fe pre = acc, y;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {  // P_l
        y = shfl_fe_up(pre, off);
        if (lane >= off) fq::mul(pre, pre, y);
    }
    fe sacc = acc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {  // acc_l ... acc_31
        y = shfl_fe_down(sacc, off);
        if (lane + off < 32) fq::mul(sacc, sacc, y);
    }
    fe suf = shfl_fe_down(sacc, 1);           // S_l
    if (lane == 31) suf = one;
    const fe total = shfl_fe(pre, 31);
    fe tinv = one;
    if (lane == 0) ec::inv(tinv, total);
    tinv = shfl_fe(tinv, 0);
    fe before = shfl_fe_up(pre, 1);           // P_{l-1}
    if (lane == 0) before = one;
    fe inv;
    fq::mul(inv, tinv, before);
    fq::mul(inv, inv, suf);
    return inv;
}

// Replaces den[j] (j < m, where ok[j]) by its inverse, with one inversion for
// the whole warp: each lane multiplies its chunk, warp_lane_inverse hands it the
// inverse of that product, from which it walks back through its chunk. Every lane
// of the warp must call it (m may be 0; lanes carry 1 then).
template <int K>
__device__ __forceinline__ void warp_batch_inverse(fe (&den)[K], const bool (&ok)[K], int m) {
    fe prefix[K];
    fe acc;
    fq::set_one(acc);
    for (int j = 0; j < m; ++j) {
        prefix[j] = acc;                   // product of the valid den[0..j-1]
        if (ok[j]) fq::mul(acc, acc, den[j]);
    }
    fe inv = warp_lane_inverse(acc);
    for (int j = m - 1; j >= 0; --j) {
        if (!ok[j]) continue;
        fe dj;
        fq::mul(dj, inv, prefix[j]);
        fq::mul(inv, inv, den[j]);
        den[j] = dj;
    }
}

__device__ __forceinline__ void store_ed_identity(uint4* o) {
    fe z, one;
    fq::set_zero(z);
    fq::set_one(one);
    fq::canon(one, one);
    store_fe(o, z);
    store_fe(o + 3, one);
    store_fe(o + 6, z);
}

// Edwards affine (x, y) of the chunk's stored points i0 .. i0 + m - 1 (from the
// standard-form input, GLV rows included); ok[j] is false for the affine identity
// and points outside the map's domain, whose (x, y) is then left unset. Every lane
// of the warp must call it (one inversion per warp).
// pairs: GLV rows taken as (P, phi(P)) pairs. The caller decides it for the whole
// launch (every lane must reach the same warp_batch_inverse): a GLV row range with
// an even start and end, so every lane's i0 and m are even.
__device__ __forceinline__ void ed_affine_chunk(const uint4* __restrict__ in, size_t n, size_t np, size_t i0, int m,
                                                bool pairs, fe (&xe)[kEdChunk], fe (&ye)[kEdChunk],
                                                bool (&ok)[kEdChunk]) {
    fe one, sp;
    fq::set_one(one);
    ed::load_const(sp, ed::kS);
    if (pairs) {
        // GLV rows in pairs (P, phi(P)) = ((x, y), (beta x, y)): the pair shares y, so
        // it inverts y, a + s and a' + s (a = x + 1, a' = beta x + 1) instead of the
        // two products y (a + s), y (a' + s); x_e = c1 a / y, y_e = (a - s) / (a + s).
        constexpr int kPairs = kEdChunk / 2;
        fe xs[kEdChunk], inv[3 * kPairs];
        bool okv[3 * kPairs];
        fe y[kPairs];
        for (int q = 0; q < m / 2; ++q) {
            fe x0;
            glv_source(x0, y[q], in, i0 + 2 * q, n, np);
            const bool id = fq::is_zero_raw(x0) && fq::is_zero_raw(y[q]);
            fe b;
            ed::load_const(b, kBeta);
            fq::mul(xs[2 * q + 1], x0, b);
            fq::canon(xs[2 * q + 1], xs[2 * q + 1]);
            xs[2 * q] = x0;
            inv[3 * q] = y[q];
            fq::add(inv[3 * q + 1], xs[2 * q], one);
            fq::add(inv[3 * q + 1], inv[3 * q + 1], sp);
            fq::add(inv[3 * q + 2], xs[2 * q + 1], one);
            fq::add(inv[3 * q + 2], inv[3 * q + 2], sp);
            okv[3 * q] = !id && !fq::is_zero(inv[3 * q]);
            okv[3 * q + 1] = !id && !fq::is_zero(inv[3 * q + 1]);
            okv[3 * q + 2] = !id && !fq::is_zero(inv[3 * q + 2]);
        }
        warp_batch_inverse(inv, okv, 3 * (m / 2));
        fe c1;
        ed::load_const(c1, ed::kC1);
        for (int q = 0; q < m / 2; ++q) {
            fe cy;
            if (okv[3 * q]) fq::mul(cy, c1, inv[3 * q]);   // c1 / y
            for (int h = 0; h < 2; ++h) {
                const int j = 2 * q + h;
                ok[j] = okv[3 * q] && okv[3 * q + 1 + h];
                if (!ok[j]) continue;
                fe a, d;
                fq::add(a, xs[j], one);
                fq::mul(xe[j], a, cy);                        // c1 a / y
                fq::sub(d, a, sp);
                fq::mul(ye[j], d, inv[3 * q + 1 + h]);        // (a - s) / (a + s)
            }
        }
        return;
    }
    fe xs[kEdChunk], ys[kEdChunk], den[kEdChunk];
    for (int j = 0; j < m; ++j) {
        glv_source(xs[j], ys[j], in, i0 + j, n, np);
        ok[j] = !(fq::is_zero_raw(xs[j]) && fq::is_zero_raw(ys[j]));
        fe a, apl;
        fq::add(a, xs[j], one);
        fq::add(apl, a, sp);
        fq::mul(den[j], ys[j], apl);
        ok[j] = ok[j] && !fq::is_zero(den[j]);
    }
    warp_batch_inverse(den, ok, m);
    for (int j = 0; j < m; ++j) {
        if (!ok[j]) continue;
        fe c, a;
        fq::add(a, xs[j], one);
        fq::add(c, a, sp);                  // a + s
        fq::mul(xe[j], a, c);
        ed::load_const(c, ed::kC1);
        fq::mul(xe[j], xe[j], c);
        fq::mul(xe[j], xe[j], den[j]);      // c1 a (a + s) / D
        fq::sub(c, a, sp);                  // a - s
        fq::mul(ye[j], c, ys[j]);
        fq::mul(ye[j], ye[j], den[j]);      // (a - s) y / D
    }
}

__device__ __forceinline__ void store_ed_stored(uint4* o, fe x, fe y) {
    fe u, k;
    ed::load_const(k, ed::kK);
    fq::mul(u, x, y);
    fq::mul(u, u, k);
    fq::canon(x, x);
    fq::canon(y, y);
    fq::canon(u, u);
    store_fe(o, x);
    store_fe(o + 3, y);
    store_fe(o + 6, u);
}

__device__ __forceinline__ void load_fe_cg(fe& a, const uint4* p) {   // through L2 (written by this thread)
    const uint4 u0 = __ldcg(p), u1 = __ldcg(p + 1), u2 = __ldcg(p + 2);
    a.v[0] = u0.x; a.v[1] = u0.y; a.v[2] = u0.z; a.v[3] = u0.w;
    a.v[4] = u1.x; a.v[5] = u1.y; a.v[6] = u1.z; a.v[7] = u1.w;
    a.v[8] = u2.x; a.v[9] = u2.y; a.v[10] = u2.z; a.v[11] = u2.w;
}

// s in standard form (the integer s, which is s / R as a Montgomery residue).
__device__ __constant__ static const uint32_t kSStd[fq::N] = {
    0xd09adc01u, 0x9c05824au, 0x0e1c7a7cu, 0x2e6bb28fu, 0xfc166427u, 0x2fe2cb65u,
    0x183465a4u, 0x86ef0d33u, 0x15ccbf8eu, 0x59416eceu, 0x062d349eu, 0x0032d756u};

__device__ __forceinline__ void add_one_raw(fe& r, const fe& a) {  // a + the integer 1
    fe o;
    fq::set_zero(o);
    o.v[0] = 1;
    fq::add(r, a, o);
}

__device__ __forceinline__ fe cst(const uint32_t (&c)[fq::N]) {
    fe r;
    ed::load_const(r, c);
    return r;
}

__device__ __forceinline__ fe mont_one() {
    fe r;
    fq::set_one(r);
    return r;
}

// Blocks of 128 per SM for the Edwards preparation: the GLV form at four (128
// registers, a few spills), the single-row form at two (its measured best: 0.54 ms for
// 2^20 points against 0.60 at four).
constexpr int prep_blocks_per_sm(bool glv) { return glv ? 4 : 2; }

// Stored Edwards rows of input points [a, b): row i, or rows 2i and 2i + 1 (P_i and
// phi(P_i) = (beta x_i, y_i)) with GLV. Same map as above, arranged to cost fewer
// multiplications and no local memory:
//  * The inputs stay in standard form. Read as Montgomery residues, x and y stand
//    for x / R and y / R; with the additive constants 1 and s entered in that same
//    scale (the integers 1 and s) every quantity the map divides is scaled by the
//    same power of R in numerator and denominator, so the Edwards coordinates come
//    out exact, in Montgomery form, with no conversion multiplications.
//  * GLV pair (P, phi(P)): one denominator t = y (a + s)(a' + s), a' = beta x + 1;
//    from t^-1 and u = y (a + s): 1/(a' + s) = t^-1 u, w = t^-1 (a' + s) = 1/u,
//    1/y = w (a + s), 1/(a + s) = w y; then x_e = c1 a / y, y_e = (a - s)/(a + s)
//    per row. Single row: t = y (a + s), x_e = c1 a (a + s) / t,
//    y_e = (a - s) y / t.
//  * A warp takes batches of 32 K consecutive points (lane l: points
//    base + 32 q + l, q < K) and inverts all their t with one field inversion
//    (Montgomery's trick over the lane's K points, warp_lane_inverse over the
//    lanes). Pass 1 writes each point's prefix product and the values pass 2
//    needs into that point's own output rows; pass 2 reads them back (through
//    L2) and overwrites the rows with the stored form.
// A zero factor of t (the identity, or a point outside the map's domain) is
// replaced by 1 and the rows it feeds become the Edwards identity.
template <bool kGlv>
__global__ void __launch_bounds__(128, prep_blocks_per_sm(kGlv))
    k_prepare_ed(const uint4* __restrict__ in, uint4* out, size_t a, size_t b, int K) {
    const int lane = threadIdx.x & 31;
    const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
    const size_t warps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t per = 32 * (size_t)K;
    const size_t nb = (b - a + per - 1) / per;
    constexpr int kRows = kGlv ? 2 : 1;
    constexpr int kVec = ModelEdwards::kStored;  // uint4 per stored row
    for (size_t bt = warp; bt < nb; bt += warps) {
        const size_t base = a + bt * per + lane;
        fe acc = mont_one();
        for (int q = 0; q < K; ++q) {            // pass 1
            const size_t i = base + 32 * (size_t)q;
            if (i >= b) break;
            fe X, Y, A, D1, t;
            load_fe(X, in + 6 * i);
            load_fe(Y, in + 6 * i + 3);
            const bool id = fq::is_zero_raw(X) && fq::is_zero_raw(Y);
            add_one_raw(A, X);
            fq::add(D1, A, cst(kSStd));
            const bool okY = !id && !fq::is_zero(Y), ok1 = !id && !fq::is_zero(D1);
            const fe Yf = okY ? Y : mont_one(), D1f = ok1 ? D1 : mont_one();
            uint4* o = out + (size_t)kVec * kRows * i;
            fq::mul(t, Yf, D1f);
            if (kGlv) {
                fe BX, D2;
                fq::mul(BX, cst(kBeta), X);
                add_one_raw(D2, BX);
                fq::add(D2, D2, cst(kSStd));
                const bool ok2 = !id && !fq::is_zero(D2);
                store_fe(o + 6, t);              // u = y (a + s)
                store_fe(o + 9, BX);
                fq::mul(t, t, ok2 ? D2 : mont_one());
            }
            store_fe(o, acc);                    // prefix product
            store_fe(o + 3, t);
            fq::mul(acc, acc, t);
        }
        fe inv = warp_lane_inverse(acc);         // acc^-1 on every lane
        for (int q = K - 1; q >= 0; --q) {       // pass 2
            const size_t i = base + 32 * (size_t)q;
            if (i >= b) continue;
            uint4* o = out + (size_t)kVec * kRows * i;
            fe X, Y, A, D1, pre, t, tinv;
            load_fe(X, in + 6 * i);
            load_fe(Y, in + 6 * i + 3);
            load_fe_cg(pre, o);
            load_fe_cg(t, o + 3);
            fq::mul(tinv, inv, pre);             // t^-1
            fq::mul(inv, inv, t);                // (prefix)^-1 for the next q down
            const bool id = fq::is_zero_raw(X) && fq::is_zero_raw(Y);
            add_one_raw(A, X);
            fq::add(D1, A, cst(kSStd));
            const bool okY = !id && !fq::is_zero(Y), ok1 = !id && !fq::is_zero(D1);
            if (kGlv) {
                fe u, BX, A2, D2, i2, w, iy, i1, cy;
                load_fe_cg(u, o + 6);
                load_fe_cg(BX, o + 9);
                add_one_raw(A2, BX);
                fq::add(D2, A2, cst(kSStd));
                const bool ok2 = !id && !fq::is_zero(D2);
                fq::mul(i2, tinv, u);                        // 1 / (a' + s)
                fq::mul(w, tinv, ok2 ? D2 : mont_one());     // 1 / (y (a + s))
                fq::mul(iy, w, ok1 ? D1 : mont_one());       // 1 / y
                fq::mul(i1, w, okY ? Y : mont_one());        // 1 / (a + s)
                fq::mul(cy, cst(ed::kC1), iy);               // c1 / y
                fe xe, ye, d;
                if (okY && ok1) {
                    fq::mul(xe, A, cy);
                    fq::sub(d, A, cst(kSStd));
                    fq::mul(ye, d, i1);
                    store_ed_stored(o, xe, ye);
                } else {
                    store_ed_identity(o);
                }
                if (okY && ok2) {
                    fq::mul(xe, A2, cy);
                    fq::sub(d, A2, cst(kSStd));
                    fq::mul(ye, d, i2);
                    store_ed_stored(o + kVec, xe, ye);
                } else {
                    store_ed_identity(o + kVec);
                }
            } else {
                if (okY && ok1) {
                    fe ct, xe, ye, d;
                    fq::mul(ct, cst(ed::kC1), tinv);         // c1 / t
                    fq::mul(xe, A, D1);
                    fq::mul(xe, xe, ct);                     // c1 a (a + s) / t
                    fq::sub(d, A, cst(kSStd));
                    fq::mul(ye, d, Y);
                    fq::mul(ye, ye, tinv);                   // (a - s) y / t
                    store_ed_stored(o, xe, ye);
                } else {
                    store_ed_identity(o);
                }
            }
        }
    }
}

// Fixed-base precomputation for resident Edwards sets: row q Wd + j of out is the
// stored form of 2^(c j) P'_q for j < Wd, P' the np stored points of the
// standard-form input (point-major, so the rows of a contiguous range of points are
// contiguous). Each lane maps its chunk to Edwards, then doubles it c times per
// window and normalises it with one inversion per warp and window. With these,
// every window of an MSM adds into the same buckets:
// sum_j 2^(cj) sum_b b B_jb = sum_b b sum_j B'_jb with B' over the shifted points.
__global__ void __launch_bounds__(128, 3) k_precompute_ed(const uint4* __restrict__ in, uint4* __restrict__ out,
                                                       size_t n, size_t np, int c, int Wd) {
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t i0 = t * kEdChunk;
    const int m = i0 >= np ? 0 : (int)(np - i0 < (size_t)kEdChunk ? np - i0 : (size_t)kEdChunk);
    fe den[kEdChunk];
    bool ok[kEdChunk];
    ed::ext P[kEdChunk];
    {
        fe xe[kEdChunk], ye[kEdChunk];
        ed_affine_chunk(in, n, np, i0, m, np != n && (np & 1) == 0, xe, ye, ok);  // rows [0, np): launch-wide
        for (int q = 0; q < m; ++q) {
            uint4* o = out + (size_t)ModelEdwards::kStored * ((i0 + q) * (size_t)Wd);
            if (ok[q]) {
                ed::stored Q;
                Q.x = xe[q];
                Q.y = ye[q];
                ed::from_stored(P[q], Q);   // u unused by from_stored
                store_ed_stored(o, xe[q], ye[q]);
            } else {
                ed::set_inf(P[q]);          // the identity stays the identity
                store_ed_identity(o);
            }
        }
    }
    for (int j = 1; j < Wd; ++j) {
        for (int q = 0; q < m; ++q) {
            for (int d = 0; d < c; ++d) ed::dbl(P[q]);
            den[q] = P[q].Z;
            ok[q] = !fq::is_zero(P[q].Z);
        }
        warp_batch_inverse(den, ok, m);
        for (int q = 0; q < m; ++q) {
            uint4* o = out + (size_t)ModelEdwards::kStored * ((i0 + q) * (size_t)Wd + j);
            if (!ok[q]) {
                store_ed_identity(o);
                continue;
            }
            fe x, y;
            fq::mul(x, P[q].X, den[q]);
            fq::mul(y, P[q].Y, den[q]);
            store_ed_stored(o, x, y);
        }
    }
}

// ---------------------------------------------------------------- stage 2

// Window digits of one scalar (8 words, little-endian) for point index `idx`:
// key = |digit| (0 = no contribution), value = point | sign << 31, window-major
// ([W][np]). The point is idx, or with precomputed shifted points (`pre`) the
// copy 2^(c j) P_idx at row idx W + j, so the W windows form one bucket problem.
__device__ __forceinline__ void emit_digits(const uint32_t (&s)[8], int c, int W, int sgn, size_t idx,
                                            size_t np, int pre, uint32_t* __restrict__ keys,
                                            uint32_t* __restrict__ vals) {
    const uint32_t cmask = (1u << c) - 1u, half = 1u << (c - 1);
    uint32_t carry = 0;
    for (int j = 0; j < W; ++j) {
        int b0 = j * c, w = b0 >> 5, off = b0 & 31;
        uint32_t raw = 0;
        if (w < 8) {
            raw = s[w] >> off;
            if (off + c > 32 && w + 1 < 8) raw |= s[w + 1] << (32 - off);
            raw &= cmask;
        }
        uint32_t key, neg = 0;
        if (sgn) {
            uint32_t v = raw + carry;
            if (v > half) {
                key = (1u << c) - v;  // |v - 2^c|
                neg = 1;
                carry = 1;
            } else {
                key = v;
                carry = 0;
            }
        } else {
            key = raw;
        }
        keys[(size_t)j * np + idx] = key;
        vals[(size_t)j * np + idx] = (uint32_t)(pre ? idx * (size_t)W + j : idx) | (neg << 31);
    }
}

// GLV split of a scalar k < 2^256: k mod r = k1 + lambda k2 with 0 <= k1 < lambda
// and k2 <= lambda + 1 (both below 2^127), lambda = x0^2 - 1 and
// lambda^2 + lambda + 1 = r. k is first reduced below r by conditional
// subtraction of 8r, 4r, 2r, r (2^256 < 16 r). Then q = floor(k mu / 2^256) with
// mu = floor(2^256 / lambda) is k2 or k2 - 1 (k mu / 2^256 > k / lambda - 1 since
// k < 2^256), fixed by one conditional subtraction of lambda.
__device__ __constant__ static const uint32_t kR8[4][8] = {
    {0x00000008u, 0x508c0000u, 0x80000008u, 0xcd53b7f6u, 0xe1bd800au, 0x05a268f2u, 0xd1652ab3u, 0x955b2af4u},
    {0x00000004u, 0x28460000u, 0x40000004u, 0x66a9dbfbu, 0x70dec005u, 0x82d13479u, 0x68b29559u, 0x4aad957au},
    {0x00000002u, 0x14230000u, 0xa0000002u, 0xb354edfdu, 0xb86f6002u, 0xc1689a3cu, 0x34594aacu, 0x2556cabdu},
    {0x00000001u, 0x0a118000u, 0xd0000001u, 0x59aa76feu, 0x5c37b001u, 0x60b44d1eu, 0x9a2ca556u, 0x12ab655eu}};
__device__ __constant__ static const uint32_t kLambda[4] = {0x00000000u, 0x0a118000u, 0x90000001u, 0x452217ccu};
__device__ __constant__ static const uint32_t kMu[5] = {0xaf90182cu, 0x7f72ed32u, 0x9fd37160u, 0xb3f7aa96u,
                                                        0x00000003u};

__device__ __forceinline__ void glv_split(uint32_t (&k)[8], uint32_t (&k1)[8], uint32_t (&k2)[8]) {
    for (int m = 0; m < 4; ++m) {  // k -= 8r, 4r, 2r, r where k is at least that
        uint32_t d[8];
        uint64_t borrow = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            uint64_t t = (uint64_t)k[w] - kR8[m][w] - borrow;
            d[w] = (uint32_t)t;
            borrow = (t >> 63) & 1u;
        }
        if (!borrow) {
#pragma unroll
            for (int w = 0; w < 8; ++w) k[w] = d[w];
        }
    }
    // q = floor(k mu / 2^256): columns 8..12 of the 8 x 5 word product
    uint32_t prod[13];
#pragma unroll
    for (int w = 0; w < 13; ++w) prod[w] = 0;
    for (int i = 0; i < 8; ++i) {
        uint64_t carry = 0;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            uint64_t t = (uint64_t)k[i] * kMu[j] + prod[i + j] + carry;
            prod[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        for (int w = i + 5; w < 13 && carry; ++w) {
            uint64_t t = (uint64_t)prod[w] + carry;
            prod[w] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    uint32_t q[4] = {prod[8], prod[9], prod[10], prod[11]};  // k mu < 2^383, so prod[12] = 0
    // rem = k - q lambda (fits in 5 words: rem < 2 lambda < 2^128)
    uint32_t ql[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) ql[w] = 0;
    for (int i = 0; i < 4; ++i) {
        uint64_t carry = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint64_t t = (uint64_t)q[i] * kLambda[j] + ql[i + j] + carry;
            ql[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        ql[i + 4] = (uint32_t)carry;
    }
    uint32_t rem[8];
    uint64_t borrow = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        uint64_t t = (uint64_t)k[w] - ql[w] - borrow;
        rem[w] = (uint32_t)t;
        borrow = (t >> 63) & 1u;
    }
    // rem >= lambda ? (rem < 2^128 here, so words 4..7 are zero)
    bool ge = true;
    for (int w = 3; w >= 0; --w) {
        if (rem[w] != kLambda[w]) {
            ge = rem[w] > kLambda[w];
            break;
        }
    }
    if (rem[4] | rem[5] | rem[6] | rem[7]) ge = true;
    if (ge) {
        uint64_t br = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            uint64_t t = (uint64_t)rem[w] - (w < 4 ? kLambda[w] : 0u) - br;
            rem[w] = (uint32_t)t;
            br = (t >> 63) & 1u;
        }
        uint64_t cy = 1;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            uint64_t t = (uint64_t)q[w] + cy;
            q[w] = (uint32_t)t;
            cy = t >> 32;
        }
    }
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        k1[w] = w < 4 ? rem[w] : 0u;
        k2[w] = w < 4 ? q[w] : 0u;
    }
}

__global__ void k_digits(const uint4* __restrict__ scalars, size_t n, int c, int W, int sgn,
                         int bits, int glv, int pre, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                         int* __restrict__ status) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint4 lo = scalars[2 * i], hi = scalars[2 * i + 1];
    uint32_t s[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    if (bits < 256) {
        uint32_t over = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int lo_bit = 32 * k;
            uint32_t m = lo_bit >= bits ? 0xffffffffu
                         : (bits - lo_bit >= 32 ? 0u : ~((1u << (bits - lo_bit)) - 1u));
            over |= s[k] & m;
        }
        if (over) atomicCAS(status, 0, MSM377_ERANGE);   // the first error of the call stays
    }
    if (!glv) {
        emit_digits(s, c, W, sgn, i, n, pre, keys, vals);
        return;
    }
    uint32_t k1[8], k2[8];
    glv_split(s, k1, k2);
    emit_digits(k1, c, W, sgn, 2 * i, 2 * n, pre, keys, vals);      // P_i
    emit_digits(k2, c, W, sgn, 2 * i + 1, 2 * n, pre, keys, vals);  // phi(P_i)
}

// ---------------------------------------------------------------- stage 3: radix sort

// Digits of RB bits per pass, R = 2^RB bins (the library sorts 8 bits per pass).
template <int RB>
__global__ void k_sort_hist(const uint32_t* __restrict__ keys, size_t n, int shift, size_t tiles,
                            uint32_t* __restrict__ hist) {
    constexpr int R = 1 << RB;
    __shared__ uint32_t cnt[R];
    const size_t t = blockIdx.x, w = blockIdx.y;
    for (int d = threadIdx.x; d < R; d += kSortThreads) cnt[d] = 0;
    __syncthreads();
    const uint32_t* seg = keys + w * n;
    const size_t start = t * kSortTile;
#pragma unroll
    for (int e = 0; e < kSortItems; ++e) {
        size_t idx = start + (size_t)e * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(seg[idx] >> shift) & (R - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < R; d += kSortThreads) hist[(w * R + d) * tiles + t] = cnt[d];
}

// Exclusive block-wide scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sums[kSortThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < kSortThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kSortThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t before = wid ? warp_sums[wid - 1] : 0;
    if (total) *total = warp_sums[kSortThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

// For each (window, digit): exclusive scan over tiles in place; the digit total goes to dtot.
template <int RB>
__global__ void k_sort_scan_tiles(uint32_t* __restrict__ hist, size_t tiles, uint32_t* __restrict__ dtot) {
    constexpr int R = 1 << RB;
    const size_t d = blockIdx.x, w = blockIdx.y;
    uint32_t* row = hist + (w * R + d) * tiles;
    const size_t per = (tiles + kSortThreads - 1) / kSortThreads;
    const size_t lo = threadIdx.x * per;
    uint32_t local = 0;
    for (size_t k = 0; k < per; ++k)
        if (lo + k < tiles) local += row[lo + k];
    uint32_t total;
    uint32_t run = block_exclusive_scan(local, &total);
    for (size_t k = 0; k < per; ++k) {
        if (lo + k < tiles) {
            uint32_t c = row[lo + k];
            row[lo + k] = run;
            run += c;
        }
    }
    if (threadIdx.x == 0) dtot[w * R + d] = total;
}

// Exclusive scan of the R digit totals of a window (R / 256 consecutive digits per thread).
template <int RB>
__global__ void k_sort_scan_digits(uint32_t* __restrict__ dtot) {
    constexpr int R = 1 << RB, PER = R / kSortThreads;
    uint32_t* row = dtot + blockIdx.x * R + threadIdx.x * PER;
    uint32_t v[PER], local = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = row[k];
        local += v[k];
    }
    uint32_t run = block_exclusive_scan(local, nullptr);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        row[k] = run;
        run += v[k];
    }
}

template <int RB>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, uint2* __restrict__ kvout, size_t n, int shift, size_t tiles,
    const uint32_t* __restrict__ hist, const uint32_t* __restrict__ doff) {
    constexpr int R = 1 << RB;
    __shared__ uint32_t wcnt[kSortThreads / 32][R];
    __shared__ uint32_t base[R];
    const size_t t = blockIdx.x, w = blockIdx.y;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < (kSortThreads / 32) * R; k += kSortThreads)
        (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    const size_t seg = w * n;
    const size_t sub = t * kSortTile + (size_t)wid * (32 * kSortItems);
    uint32_t key[kSortItems], val[kSortItems], dig[kSortItems], rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        size_t idx = sub + (size_t)r * 32 + lane;
        bool valid = idx < n;
        key[r] = valid ? kin[seg + idx] : 0u;
        val[r] = valid ? vin[seg + idx] : 0u;
        // Items past the end sort last in the tile and are never written.
        dig[r] = valid ? ((key[r] >> shift) & (R - 1)) : (R - 1);
        uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
        uint32_t before = wcnt[wid][dig[r]];
        __syncwarp();
        if (lane == __ffs(peers) - 1) wcnt[wid][dig[r]] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < R; d += kSortThreads) {
        uint32_t run = 0;
#pragma unroll
        for (int k = 0; k < kSortThreads / 32; ++k) {
            uint32_t c = wcnt[k][d];
            wcnt[k][d] = run;
            run += c;
        }
        base[d] = doff[w * R + d] + hist[(w * R + d) * tiles + t];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        size_t idx = sub + (size_t)r * 32 + lane;
        if (idx < n) {
            size_t pos = (size_t)base[dig[r]] + wcnt[wid][dig[r]] + rank[r];
            if (pos < n) {  // always true when the counts agree; keeps writes in bounds
                if (kvout) {    // last pass: (key, value) pairs, one 8-byte store
                    kvout[seg + pos] = make_uint2(key[r], val[r]);
                } else {
                    kout[seg + pos] = key[r];
                    vout[seg + pos] = val[r];
                }
            }
        }
    }
}

// ---------------------------------------------------------------- stage 3 (counting sort)
//
// Bucket order by counting: every (window, key) is a bin; one pass counts the
// items of each bin with warp-aggregated atomics, a scan turns the counts into
// bin offsets (window w's bins start at w np, since each window holds np items),
// and one pass scatters every item to its bin's next free slot. The order inside
// a bin is not kept -- it does not matter, since a bucket's sum is the same group
// element in any order. Two passes over the (key, value) pairs instead of a
// histogram and a scatter pass per 8 key bits.
constexpr int kScanBlock = 1024, kScanPer = 4, kScanTile = kScanBlock * kScanPer;

// Grid (items of a window / 256, windows): item i = w np + j of window w = blockIdx.y.
// Counts per (window, key) bin; each item keeps its rank among the items of its bin
// (the warp's share from one atomic per distinct bin, then the lanes' order), so the
// scatter needs no atomics. This global-counter form serves key ranges too wide for
// the shared-memory tiles below (c >= 18 with signed digits, c >= 17 unsigned).
__global__ void k_bin_count(const uint32_t* __restrict__ keys, size_t np, uint32_t nb,
                            uint32_t* __restrict__ counts, uint32_t* __restrict__ rank) {
    const size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const bool valid = j < np;
    const size_t i = (size_t)blockIdx.y * np + j;
    const uint32_t bin = valid ? blockIdx.y * nb + keys[i] : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, bin);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid && lane == leader) base = atomicAdd(&counts[bin], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) rank[i] = base + __popc(peers & ((1u << lane) - 1u));
}
__global__ void __launch_bounds__(kScanBlock) k_scan_tiles(uint32_t* __restrict__ x, size_t m,
                                                           uint32_t* __restrict__ bsum) {
    __shared__ uint32_t warp_tot[kScanBlock / 32];
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer], local = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < m ? x[base + k] : 0u;
        local += v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    uint32_t run = inc - local + (wid ? warp_tot[wid - 1] : 0u);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < m) x[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = warp_tot[kScanBlock / 32 - 1];
}

// Exclusive scan of the tile totals in one block (any count: a serial run per thread).
__global__ void __launch_bounds__(kScanBlock) k_scan_totals(uint32_t* __restrict__ bsum, size_t nb) {
    __shared__ uint32_t warp_tot[kScanBlock / 32];
    const size_t per = (nb + kScanBlock - 1) / kScanBlock;
    const size_t lo = threadIdx.x * per;
    uint32_t local = 0;
    for (size_t k = lo; k < lo + per && k < nb; ++k) local += bsum[k];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    uint32_t run = inc - local + (wid ? warp_tot[wid - 1] : 0u);
    for (size_t k = lo; k < lo + per && k < nb; ++k) {
        const uint32_t c = bsum[k];
        bsum[k] = run;
        run += c;
    }
}

__global__ void k_scan_add(uint32_t* __restrict__ x, size_t m, const uint32_t* __restrict__ bsum) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < m) x[i] += bsum[i / kScanTile];
}

// Each item to the next free slot of its bin (cursor = the bins' offsets, advanced
// with one warp-aggregated atomic per bin and warp).
__global__ void k_bin_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                              const uint32_t* __restrict__ rank, uint2* __restrict__ kvout, size_t total,
                              size_t np, uint32_t nb, const uint32_t* __restrict__ start) {
    const size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    const size_t i = (size_t)blockIdx.y * np + j;
    const uint32_t key = kin[i];
    const size_t pos = (size_t)start[blockIdx.y * nb + key] + rank[i];
    if (pos < total) kvout[pos] = make_uint2(key, vin[i]);  // in bounds when the counts agree
}

// The same counting sort with the counts taken per tile in shared memory, for key
// ranges whose counters fit there (no global atomics at all). Tile t of window w
// holds items [t T, (t + 1) T); its block counts the tile's keys in 16-bit shared
// counters packed two to a word (T < 2^16, so no count reaches the neighbour's
// half) and gives each item its rank among the tile's items of the same key. The
// tile counts go to cnt[w][t][key]; a column pass sums them into the bin totals, the
// bin scan gives each (window, key) its offset, a second column pass turns cnt into
// each tile's first slot per key (offset + counts of the earlier tiles), and an
// item's slot is that plus its rank.
constexpr int kTileThreads = 1024;
constexpr uint32_t kTileItemsMax = 65535;
constexpr size_t kTileSmemMax = 200 * 1024;    // packed counters of one block (GB300: 227 KB opt-in)

// Grid (tiles, windows). Plain shared atomics: with random keys the counters rarely
// collide. Measured on GB300 (n = 2^20, c = 16): one atomic per distinct key and
// warp (found with match.any) made the head 0.09 ms slower with random scalars, and a
// one-atomic path for warps whose keys are all equal moved it by at most 0.02 ms
// with all-equal scalars.
__global__ void __launch_bounds__(kTileThreads) k_tile_count(const uint32_t* __restrict__ keys, size_t np,
                                                             uint32_t nb, uint32_t T, uint32_t ntiles,
                                                             uint32_t* __restrict__ cnt, uint32_t* __restrict__ rank) {
    extern __shared__ uint32_t h[];
    const uint32_t hw = (nb + 1) / 2;
    for (uint32_t k = threadIdx.x; k < hw; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const size_t w = blockIdx.y;
    const size_t lo = (size_t)blockIdx.x * T;
    const size_t hi = lo + T < np ? lo + T : np;
    const uint32_t* kw = keys + w * np;
    uint32_t* rw = rank + w * np;
    for (size_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const uint32_t key = kw[j];
        if (key >= nb) continue;   // keys are below nb by construction
        const uint32_t sh = (key & 1u) << 4;
        const uint32_t old = atomicAdd(&h[key >> 1], 1u << sh);
        rw[j] = (old >> sh) & 0xffffu;
    }
    __syncthreads();
    uint32_t* cw = cnt + (w * ntiles + blockIdx.x) * nb;
    for (uint32_t k = threadIdx.x; k < nb; k += blockDim.x) cw[k] = (h[k >> 1] >> ((k & 1u) << 4)) & 0xffffu;
}

// Thread (w, key): bins[w][key] <- the count over the window's tiles.
__global__ void k_tile_totals(const uint32_t* __restrict__ cnt, uint32_t nb, uint32_t ntiles, uint32_t W,
                              uint32_t* __restrict__ bins) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)W * nb) return;
    const size_t w = id / nb, k = id % nb;
    const uint32_t* c = cnt + w * ntiles * nb + k;
    uint32_t run = 0;
    for (uint32_t t = 0; t < ntiles; ++t) run += c[(size_t)t * nb];
    bins[id] = run;
}

// Thread (w, key), after the bin scan: cnt[w][t][key] <- the slot of the tile's first
// item of that key, start[w][key] plus the counts of tiles t' < t.
__global__ void k_tile_offsets(uint32_t* __restrict__ cnt, uint32_t nb, uint32_t ntiles, uint32_t W,
                               const uint32_t* __restrict__ start) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)W * nb) return;
    const size_t w = id / nb, k = id % nb;
    uint32_t* c = cnt + w * ntiles * nb + k;
    uint32_t run = start[id];
    constexpr uint32_t kStep = 16;   // loads in flight per thread
    for (uint32_t t0 = 0; t0 < ntiles; t0 += kStep) {
        uint32_t v[kStep];
#pragma unroll
        for (uint32_t u = 0; u < kStep; ++u) v[u] = t0 + u < ntiles ? c[(size_t)(t0 + u) * nb] : 0u;
#pragma unroll
        for (uint32_t u = 0; u < kStep; ++u) {
            if (t0 + u < ntiles) c[(size_t)(t0 + u) * nb] = run;
            run += v[u];
        }
    }
}

// Grid (items of a window / 256, windows): each item to its tile's slot for the key
// plus its rank.
__global__ void k_tile_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                               const uint32_t* __restrict__ rank, uint2* __restrict__ kvout, size_t total,
                               size_t np, uint32_t nb, uint32_t T, uint32_t ntiles, const uint32_t* __restrict__ cnt) {
    const size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    const size_t w = blockIdx.y;
    const size_t i = w * np + j;
    const uint32_t key = kin[i];
    if (key >= nb) return;
    const size_t t = j / T;
    const size_t pos = (size_t)cnt[(w * ntiles + t) * nb + key] + rank[i];
    if (pos < total) kvout[pos] = make_uint2(key, vin[i]);
}

// ---------------------------------------------------------------- stages 4-5

struct AccArgs {
    const uint2* kv;       // [W][n] sorted (bucket key, point index | sign << 31)
    const uint4* pts;
    uint4* buckets;        // [W][Bp] XYZZ
    uint4* head;           // [W][cpw] XYZZ
    uint4* tail;           // [W][cpw] XYZZ
    uint32_t* headflag;    // 0 none, 1 run ends here, 2 run continues past this chunk
    uint32_t* tailkey;     // key of the run leaving this chunk, or kNone
    size_t n;              // items per window
    uint32_t cpw;          // chunks per window
    uint32_t Bp;
    int K;
    int w0, nwin;          // window range of this launch
    const uint32_t* bin;   // counting sort: first kv slot of each (window, key) bin (else null)
    uint32_t nb;           // keys per window (Bp + 1)
};

// Mixed additions of chunk t of window w. Flushes each run to its bucket, or to
// the chunk's head / tail partial when it crosses a chunk edge.
template <class M>
__device__ __forceinline__ void accumulate_chunk(const AccArgs& a, int w, uint32_t t) {
    const size_t ci = (size_t)w * a.cpw + t;
    const uint2* kv = a.kv + (size_t)w * a.n;
    const size_t start = (size_t)t * a.K;
    const size_t end = start + a.K < a.n ? start + a.K : a.n;
    const uint32_t prev = start > 0 ? kv[start - 1].x : kNone;
    const uint32_t next = end < a.n ? kv[end].x : kNone;
    a.tailkey[ci] = kNone;
    a.headflag[ci] = 0;
    typename M::acc acc;
    M::set_inf(acc);
    bool inf = true;
    uint32_t cur = kv[start].x;
    bool first = true;
    for (size_t g = start; g <= end; ++g) {
        const uint2 e = g < end ? kv[g] : make_uint2(kNone, 0u);
        const uint32_t key = e.x;
        if (key != cur) {
            if (cur != 0) {  // key 0 = zero digit, contributes nothing
                const bool sb = first && prev == cur;
                const bool ea = (g == end) && next == cur;
                if (!sb && !ea) {
                    M::store(a.buckets + ((size_t)w * a.Bp + (cur - 1)) * kXyzzVec, acc);
                } else if (sb) {
                    M::store(a.head + ci * kXyzzVec, acc);
                    a.headflag[ci] = ea ? 2u : 1u;
                } else {
                    M::store(a.tail + ci * kXyzzVec, acc);
                    a.tailkey[ci] = cur;
                }
            }
            if (g == end) break;
            M::set_inf(acc);
            inf = true;
            cur = key;
            first = false;
        }
        if (key != 0) {
            const uint32_t v = e.y;
            if ((v & 0x7fffffffu) >= a.n) continue;  // cannot happen for sorted digit output
            M::madd_at(acc, inf, a.pts, v & 0x7fffffffu, (v >> 31) != 0);
        }
    }
}

// Register caps per curve model (M::kAccBlocks blocks of 128 resident per SM), each
// the faster of the caps measured at n = 2^20, c = 16: XYZZ at 168 registers, three
// blocks (4 blocks: 5.75 vs 5.74 ms per accumulation; uncapped, 190 registers and two
// blocks, slower still); Edwards at 128 registers, four blocks, with a few spills
// (4.14 vs 4.24 ms at three blocks).
template <class M>
__global__ void __launch_bounds__(128, M::kAccBlocks) k_accumulate(AccArgs a) {
    const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (uint32_t)a.nwin * a.cpw) return;
    accumulate_chunk<M>(a, a.w0 + (int)(id / a.cpw), id % a.cpw);
}

// Batched MSMs: one persistent kernel drains a queue of (job, window, chunk)
// items of all jobs. Each warp takes 32 consecutive items with one atomic.
constexpr int kMaxBatch = 128;
struct BatchAcc {
    AccArgs job[kMaxBatch];
    uint32_t prefix[kMaxBatch + 1];  // cumulative W * cpw over jobs
    int njobs;
    uint32_t* counter;
};

template <class M>
__global__ void __launch_bounds__(128, M::kAccBlocks) k_accumulate_batched(const __grid_constant__ BatchAcc b) {
    const uint32_t total = b.prefix[b.njobs];
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(b.counter, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        const uint32_t item = base + lane;
        if (item < total) {
            int lo = 0, hi = b.njobs - 1;   // last job with prefix <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (b.prefix[mid] <= item) lo = mid; else hi = mid - 1;
            }
            const AccArgs& a = b.job[lo];
            const uint32_t local = item - b.prefix[lo];
            accumulate_chunk<M>(a, (int)(local / a.cpw), local % a.cpw);
        }
    }
}

// Partial sums of runs that cross chunk edges. When a bucket's run is expected to be
// no longer than a chunk (items per bucket <= K), a run that continues into at most
// kWalkHeads later chunks (every run of random scalars then) is finished by the
// thread of its tail chunk, which adds the run's head partials in order
// (k_merge_walk). With longer runs, serial additions on one thread would cost more
// than the rounds below (measured at n = 2^22, c = 16: 256 items per bucket, chunks
// of 64, 1 ms slower), so the walk is skipped and every run takes the log-depth path.
// Longer runs are combined in log depth, so a bucket holding a large share of the
// window (all-equal scalars, a nearly empty top window) costs O(log) serial additions,
// not O(chunks); those kernels return at once unless the walk left such a run:
//  * k_merge_start: for a chunk u whose first run continues an earlier chunk's
//    run, start[u] = the chunk t0 where that run begins (its tail): the run's key
//    first occurs at lower_bound(keys, key) in the sorted window, so t0 is that
//    position / K (one binary search per chunk, no scan);
//  * k_merge_round(d): for heads at offset j = u - start[u] - 1 with j % 2d == 0,
//    head[u] += head[u + d] when u + d continues the same run; ceil(log2 cpw) rounds
//    leave each run's sum of heads at its first head;
//  * k_merge_long: the rounds above are launched for d < kMergeRounds only (enough for
//    the runs of random scalars, which cross a few chunk edges); a run with more heads
//    is finished by one block that runs the remaining rounds (d = kMergeRounds,
//    2 kMergeRounds, ...) over that run alone between block barriers. When no run is
//    that long the launch returns at once: one launch instead of a dozen idle rounds;
//  * k_merge_final: bucket = tail[start] + that sum.
constexpr uint32_t kWalkHeads = 4;

template <class M>
__global__ void k_merge_walk(AccArgs a, uint32_t H, int* __restrict__ longrun) {
    const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (uint32_t)a.nwin * a.cpw) return;
    const int w = a.w0 + (int)(id / a.cpw);
    const uint32_t t = id % a.cpw;
    const size_t ci = (size_t)w * a.cpw + t;
    const uint32_t key = a.tailkey[ci];
    if (key == kNone) return;
    typename M::acc acc;
    M::load(acc, a.tail + ci * kXyzzVec);
    // The run starts in chunk t (a run that began earlier would make chunk t a head);
    // it ends where its bin ends, so it has nh = (last item) / K - t heads. Without the
    // bin table (radix sort) the heads' flags are counted instead.
    uint32_t nh = H + 1;
    if (a.bin) {
        const size_t b = (size_t)w * a.nb + key;
        const size_t end = key + 1 < a.nb ? (size_t)a.bin[b + 1] - (size_t)w * a.n : a.n;   // within the window
        nh = (uint32_t)((end - 1) / (size_t)a.K) - t;
    } else {
        for (uint32_t h = H + 1; h >= 1; --h) {
            const uint32_t f = t + h < a.cpw ? a.headflag[ci + h] : 0u;
            if (f == 0) nh = h - 1;      // the run ended before chunk t + h
            if (f == 1) nh = h;          // the run ends in chunk t + h
        }
    }
    if (nh > H) {                        // tail key and all, for k_merge_start .. k_merge_final
        *longrun = 1;
        return;
    }
    for (uint32_t h = 1;; ++h) {       // the heads up to the one with flag 1
        const uint32_t f = t + h < a.cpw ? a.headflag[ci + h] : 0u;
        if (f == 0 || h > nh) break;     // the run ended before chunk t + h
        M::add_mem(acc, a.head + (ci + h) * kXyzzVec);
        if (f == 1) break;               // the run ends in chunk t + h
    }
    M::store(a.buckets + ((size_t)w * a.Bp + (key - 1)) * kXyzzVec, acc);
    a.tailkey[ci] = kNone;
}

// longrun: the walk's flag (null when no walk ran: every run is merged here).
__global__ void k_merge_start(AccArgs a, const int* __restrict__ longrun, int32_t* __restrict__ start,
                              int* __restrict__ maxspan) {
    if (longrun && *longrun == 0) return;  // every run was finished by the walk
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)a.nwin * a.cpw) return;
    const int w = a.w0 + (int)(id / a.cpw);
    const uint32_t u = (uint32_t)(id % a.cpw);
    const size_t ci = (size_t)w * a.cpw + u;
    if (a.headflag[ci] == 0) {
        start[ci] = -1;
        return;
    }
    const uint2* kv = a.kv + (size_t)w * a.n;
    const size_t first = (size_t)u * a.K;   // u > 0 here: chunk 0 has no earlier run
    const uint32_t key = kv[first].x;
    size_t lo = 0, hi = first;              // first index in [0, first] with keys[i] >= key
    while (lo < hi) {
        const size_t mid = (lo + hi) >> 1;
        if (kv[mid].x < key) lo = mid + 1; else hi = mid;
    }
    const int32_t t0 = (int32_t)(lo / (size_t)a.K);
    start[ci] = t0;
    atomicMax(maxspan, (int)(u - (uint32_t)t0));  // heads of this run up to u
}

template <class M>
__global__ void k_merge_round(AccArgs a, const int32_t* __restrict__ start, uint32_t d,
                              const int* __restrict__ maxspan) {
    if (d >= (uint32_t)*maxspan) return;  // no run has heads this far apart: nothing to pair
    const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (uint32_t)a.nwin * a.cpw) return;
    const int w = a.w0 + (int)(id / a.cpw);
    const uint32_t u = id % a.cpw;
    const size_t base = (size_t)w * a.cpw;
    if (a.headflag[base + u] == 0) return;
    const int32_t t0 = start[base + u];
    if (t0 < 0) return;
    const uint32_t j = u - (uint32_t)t0 - 1;
    if (j % (2 * d) != 0) return;
    const uint32_t v = u + d;
    if (v >= a.cpw || a.headflag[base + v] == 0 || start[base + v] != t0) return;
    typename M::acc acc;
    M::load(acc, a.head + (base + u) * kXyzzVec);
    M::add_mem(acc, a.head + (base + v) * kXyzzVec);
    M::store(a.head + (base + u) * kXyzzVec, acc);
}

constexpr uint32_t kMergeRounds = 8;   // rounds d = 1, 2, 4 launched one by one
constexpr int kMergeLongThreads = 128;

template <class M>
__global__ void __launch_bounds__(kMergeLongThreads) k_merge_long(AccArgs a, const int32_t* __restrict__ start,
                                                                  const int* __restrict__ maxspan) {
    if ((uint32_t)*maxspan <= kMergeRounds) return;  // every run is complete already
    __shared__ uint32_t first[kMergeLongThreads], span[kMergeLongThreads];
    __shared__ uint32_t nfound;
    const uint32_t nchunks = (uint32_t)a.nwin * a.cpw;
    for (uint32_t tile = blockIdx.x * kMergeLongThreads; tile < nchunks; tile += gridDim.x * kMergeLongThreads) {
        if (threadIdx.x == 0) nfound = 0;
        __syncthreads();
        // the first head (j = 0) of every run with more than kMergeRounds heads in this tile
        const uint32_t id = tile + threadIdx.x;
        if (id < nchunks) {
            const int w = a.w0 + (int)(id / a.cpw);
            const uint32_t u = id % a.cpw;
            const size_t ci = (size_t)w * a.cpw + u;
            const int32_t t0 = a.headflag[ci] != 0 ? start[ci] : -1;
            if (t0 >= 0 && u == (uint32_t)t0 + 1) {
                // the run's last item: the last index with this key (upper bound - 1)
                const uint2* kv = a.kv + (size_t)w * a.n;
                const uint32_t key = kv[(size_t)u * a.K].x;
                size_t lo = (size_t)u * a.K, hi = a.n;
                while (lo < hi) {
                    const size_t mid = (lo + hi) >> 1;
                    if (kv[mid].x <= key) lo = mid + 1; else hi = mid;
                }
                const uint32_t heads = (uint32_t)((lo - 1) / (size_t)a.K) - (uint32_t)t0;
                if (heads > kMergeRounds) {
                    const uint32_t k = atomicAdd(&nfound, 1u);
                    first[k] = id;
                    span[k] = heads;
                }
            }
        }
        __syncthreads();
        const uint32_t nf = nfound;
        for (uint32_t r = 0; r < nf; ++r) {
            const uint32_t f = first[r], S = span[r];
            const int w = a.w0 + (int)(f / a.cpw);
            const size_t h0 = (size_t)w * a.cpw + f % a.cpw;   // head j = 0 of the run
            for (uint32_t d = kMergeRounds; d < S; d <<= 1) {
                const uint32_t pairs = (S - d + 2 * d - 1) / (2 * d);   // j = 0, 2d, ... with j + d < S
                for (uint32_t q = threadIdx.x; q < pairs; q += blockDim.x) {
                    const size_t j = (size_t)q * 2 * d;
                    typename M::acc acc;
                    M::load(acc, a.head + (h0 + j) * kXyzzVec);
                    M::add_mem(acc, a.head + (h0 + j + d) * kXyzzVec);
                    M::store(a.head + (h0 + j) * kXyzzVec, acc);
                }
                __syncthreads();   // this level's sums are visible to the next level
            }
        }
        __syncthreads();   // the list is read before the next tile overwrites it
    }
}

template <class M>
__global__ void k_merge_final(AccArgs a, const int* __restrict__ longrun) {
    if (longrun && *longrun == 0) return;  // every run was finished by the walk
    const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (uint32_t)a.nwin * a.cpw) return;
    const int w = a.w0 + (int)(id / a.cpw);
    const uint32_t t = id % a.cpw;
    const size_t ci = (size_t)w * a.cpw + t;
    const uint32_t key = a.tailkey[ci];
    if (key == kNone) return;
    typename M::acc acc;
    M::load(acc, a.tail + ci * kXyzzVec);
    if (t + 1 < a.cpw && a.headflag[ci + 1] != 0) M::add_mem(acc, a.head + (ci + 1) * kXyzzVec);
    M::store(a.buckets + ((size_t)w * a.Bp + (key - 1)) * kXyzzVec, acc);
}

// ---------------------------------------------------------------- stage 6

// Thread (wi, g): Y = sum_{i=1..L} B[gL+i], V = sum_{i=1..L} i * B[gL+i] (bucket b at index b-1).
template <class M>
__global__ void __launch_bounds__(128) k_reduce_segments(const uint4* __restrict__ buckets, uint32_t Bp, uint32_t L, int w0, int nwin,
                                  uint32_t G, uint4* __restrict__ Y, uint4* __restrict__ V) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (id >= (size_t)nwin * G) return;
    const size_t wi = id / G, g = id % G;
    const uint4* seg = buckets + ((size_t)(w0 + wi) * Bp + g * L) * kXyzzVec;
    typename M::acc T, S;
    M::set_inf(T);
    M::set_inf(S);
    for (int i = (int)L; i >= 1; --i) {
        M::add_mem(T, seg + (size_t)(i - 1) * kXyzzVec);   // T += B
        M::add(S, T);                                       // S += T
    }
    M::store(Y + id * kXyzzVec, T);
    M::store(V + id * kXyzzVec, S);
}

// Thread (wi, k, q): partial of Z_k = sum_{g: bit k of g set} Y_g over the q-th of Q
// equal slices of those G/2 indices, or for k == logG the partial of sum_g V_g over
// the q-th slice of all G indices. The j-th index with bit k set is j with a one
// inserted at bit k, so the threads of a warp (same k) run the same additions.
template <class M>
__global__ void k_bitsums(const uint4* __restrict__ Y, const uint4* __restrict__ V, int nwin, uint32_t G,
                          int logG, uint32_t Q, uint4* __restrict__ P) {
    const size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t per_w = (size_t)(logG + 1) * Q;
    if (id >= (size_t)nwin * per_w) return;
    const size_t wi = id / per_w;
    const int kk = (int)((id % per_w) / Q);
    const int k = kk == 0 ? logG : kk - 1;  // the V slices (twice as long) are scheduled first
    const uint32_t q = (uint32_t)(id % Q);
    typename M::acc acc;
    M::set_inf(acc);
    if (k == logG) {
        const uint32_t span = G / Q, g0 = q * span;
        for (uint32_t g = g0; g < g0 + span; ++g) M::add_mem(acc, V + (wi * G + g) * kXyzzVec);
    } else {
        const uint32_t span = (G / 2) / Q, j0 = q * span, low = (1u << k) - 1u;
        for (uint32_t j = j0; j < j0 + span; ++j) {
            const uint32_t g = ((j & ~low) << 1) | (1u << k) | (j & low);
            M::add_mem(acc, Y + (wi * G + g) * kXyzzVec);
        }
    }
    M::store(P + (wi * per_w + (size_t)k * Q + q) * kXyzzVec, acc);
}

// Block (s, b) sums in[s][F 32 b .. F 32 (b + 1) - 1] (within the segment's m points)
// into out[s][b] with four lanes per addition: group j of the block's 32 groups sums
// in[F 32 b + j + 32 f] for f < F in sequence, then a tree over the groups in shared
// memory (depth F - 1 + 5 four-lane additions; a segment of m points needs
// log_(32 F) m launches; F is chosen so that a launch fills about one wave of
// blocks). Every group of a warp runs the same additions (a missing operand is the
// identity; idle groups of warp 0 add and discard), so each __syncwarp inside them
// is warp-wide; a warp with no active group skips a level as a whole.
constexpr int kTreeThreads = 128;
constexpr int kTreeGroups = kTreeThreads / 4;
constexpr size_t kTreeWave = 152 * 3;  // blocks resident at once (3 per SM)

template <class M>
__global__ void __launch_bounds__(kTreeThreads) k_sum_tree(const uint4* __restrict__ in, size_t nseg, uint32_t m,
                                                          uint32_t F, uint4* __restrict__ out) {
    __shared__ uint4 pub[kTreeGroups * kXyzzVec];
    __shared__ uint4 idn[kXyzzVec];
    __shared__ fe sh[kTreeGroups][4];
    const uint32_t per = kTreeGroups * F;
    const uint32_t nb = (m + per - 1) / per;
    const size_t seg = blockIdx.x / nb;
    const uint32_t b = blockIdx.x % nb;
    if (seg >= nseg) return;  // whole block
    const int t = threadIdx.x, g = t >> 2, l = t & 3, warp = t >> 5;
    if (t == 0) {
        typename M::acc e;
        M::set_inf(e);
        M::store(idn, e);
    }
    __syncthreads();
    const uint32_t i0 = b * per + g;
    typename M::acc acc;
    if (i0 < m)
        M::load(acc, in + (seg * m + i0) * kXyzzVec);
    else
        M::set_inf(acc);
    for (uint32_t f = 1; f < F; ++f) {
        const uint32_t i = i0 + f * kTreeGroups;
        M::add4_mem(acc, i < m ? in + (seg * m + i) * kXyzzVec : idn, sh[g], l);
    }
    // level h: groups [h, 2h) publish, groups [0, h) add them. The slots read at
    // level h, [h, 2h), are never written at a later level (those write [h', 2h')
    // with 2h' <= h), so one barrier per level orders every access.
    for (int h = kTreeGroups / 2; h >= 1; h >>= 1) {
        if (g >= h && g < 2 * h && l == 0) M::store(pub + g * kXyzzVec, acc);
        __syncthreads();
        if (warp * 8 < h) {
            typename M::acc r = acc;
            M::add4_mem(r, pub + (g + h) * kXyzzVec, sh[g], l);  // g + h < 32: g < h for h >= 8, g <= 7 below
            if (g < h) acc = r;
        }
    }
    if (t == 0) M::store(out + (seg * nb + b) * kXyzzVec, acc);
}

// ---------------------------------------------------------------- stage 7

// The two latency-bound chains run on one group of four warps per block: each
// point operation's products are spread over the warps (one product per warp and
// formula level) and each product over the lanes of its warp (wpt.cuh, wfq.cuh).
// The next operand's loads are issued before the current operation, so they
// overlap it.

// Block w: S_w = L sum_{k < logG} 2^k Z_k + Z_logG for window w, by Horner from the
// top term.
template <class M>
__global__ void __launch_bounds__(128, 1) k_window_horner_w(const uint4* __restrict__ Z, int nwin, int logG, int log2L,
                                                         uint4* __restrict__ S) {
    __shared__ __align__(16) uint32_t slots[wpt::kSharedWords];
    wpt::Group g;
    wpt::init(g, slots);
    const int w = blockIdx.x;
    if (w >= nwin) return;  // whole block
    const uint32_t* z = reinterpret_cast<const uint32_t*>(Z + (size_t)w * (logG + 1) * kXyzzVec);
    constexpr size_t kWords = 4 * kXyzzVec;
    M::gset_inf(g);
    wpt::Operand next = wpt::load_operand(z + (size_t)(logG > 0 ? logG - 1 : logG) * kWords, 4);
    for (int k = logG - 1; k >= 0; --k) {
        const wpt::Operand q = next;   // Z_k
        next = wpt::load_operand(z + (size_t)(k > 0 ? k - 1 : logG) * kWords, 4);
        if (k < logG - 1) M::gdbl(g);
        M::gadd(g, q);
    }
    for (int t = 0; t < log2L; ++t) M::gdbl(g);
    M::gadd(g, next);                  // Z_logG
    wpt::store_acc(g, reinterpret_cast<uint32_t*>(S + (size_t)w * kXyzzVec));
}

// sum_w 2^(c w) S_w by Horner over the windows, then the affine result in standard
// form (thread 0 writes it after the inversion).
template <class M>
__global__ void __launch_bounds__(128, 1) k_chain_w(const uint4* __restrict__ S, int W, int c, uint32_t* __restrict__ out) {
    __shared__ __align__(16) uint32_t slots[wpt::kSharedWords];
    wpt::Group g;
    wpt::init(g, slots);
    const uint32_t* s = reinterpret_cast<const uint32_t*>(S);
    constexpr size_t kWords = 4 * kXyzzVec;
    M::gset_inf(g);
    wpt::Operand next = wpt::load_operand(s + (size_t)(W - 1) * kWords, 4);
    for (int j = W - 1; j >= 0; --j) {
        const wpt::Operand q = next;   // S_j
        if (j > 0) next = wpt::load_operand(s + (size_t)(j - 1) * kWords, 4);
        if (j < W - 1)
            for (int t = 0; t < c; ++t) M::gdbl(g);
        M::gadd(g, q);
    }
    if (threadIdx.x != 0) return;
    fe acc[4];
    wpt::read_acc(g, acc);
    affine A;
    M::to_affine4(A, acc);
    if (!ec::is_inf(A)) {
        fq::from_mont(A.x, A.x);
        fq::from_mont(A.y, A.y);
    }
    fq::store(out, A.x);
    fq::store(out + 12, A.y);
}

// ---------------------------------------------------------------- planning

struct Plan {
    size_t n;        // scalars (and input points)
    size_t np;       // stored points = items per window: n, or 2n with GLV
    int edw, glv;    // curve model (0 XYZZ, 1 Edwards); GLV split
    int pre;         // precomputed shifted points: the Wd digit windows share one bucket set
    int Wd;          // digit windows per scalar (W = 1 when pre, else W = Wd)
    size_t items;    // items per pipeline window: np, or Wd np when pre
    int stored_vec;  // uint4 per stored point
    int user_bits;   // scalar range checked against opts.scalar_bits
    int c, sgn, bits, W;
    uint32_t B, Bp;
    int passes, rb;  // radix-sort passes of rb-bit digits
    size_t tiles;
    int K;
    uint32_t cpw;   // chunks per window
    int gw;         // windows per group
    int ngroups;
    uint32_t L, G, Q;
    int logG, log2L;
    size_t off_status, off_points, off_keys0, off_vals0, off_keys1, off_vals1, off_kv, off_rank, off_hist, off_dtot;
    int counting;                      // counting sort (else LSD radix sort)
    size_t nbins, off_bins, off_bsum;  // counting sort: bins (window, key) and scan tile totals
    uint32_t ttiles, tT;               // counting sort in shared-memory tiles: tiles per window, items per
                                       // tile (ttiles = 0: global counters)
    size_t off_tcnt;                   // per-tile counts and prefixes [W][ttiles][Bp + 1]
    uint32_t walk;                     // heads a run's tail thread adds itself (0: no walk)
    size_t off_buckets, off_head, off_tail, off_headflag, off_tailkey, off_Y, off_V, off_P0, off_P1;
    size_t off_S, off_start, total;
};

constexpr uint64_t kReduceThreads = 32768;

int ilog2(uint64_t v) {
    int r = 0;
    while ((1ull << (r + 1)) <= v) ++r;
    return r;
}

// Tuned schedules for signed digits by floor(log2 n), one table per mode (Edwards,
// GLV, fixed-base), set from measured tables by msm_g1_set_window_table (window
// widths) and msm_g1_set_schedule (every field); 0 = the built-in rule.
std::atomic<int> g_ctable[8][32];      // window width c
std::atomic<int> g_ktable[8][32];      // items per accumulation chunk K
std::atomic<int> g_sorttable[8][32];   // 1 counting sort, 2 LSD radix sort
std::atomic<int> g_rtable[8][32];      // log2 of the level-1 reduction threads
std::atomic<int> g_gtable[8][32];      // window groups (1 = no overlap of tails with accumulation)

int table_mode(uint32_t flags) {
    return ((flags & MSM377_EDWARDS) ? 1 : 0) | ((flags & MSM377_GLV) ? 2 : 0) |
           ((flags & MSM377_PRECOMPUTED) ? 4 : 0);
}

int default_c(size_t n, int sgn, uint32_t flags) {
    int lg = n > 1 ? ilog2(n) : 0;
    if (sgn && lg < 32) {
        const int t = g_ctable[table_mode(flags)][lg].load(std::memory_order_relaxed);
        if (t > 0) return t;
    }
    if (flags & MSM377_GLV) ++lg;  // 2n points per window
    if (flags & MSM377_PRECOMPUTED) lg += 2;  // one bucket set for all windows: wider windows pay
    int c = lg - 4;
    if (!sgn) c = lg - 3;
    if (c < 4) c = 4;
    if (c > 17) c = 17;
    return c;
}

constexpr int kMaxGroups = 8;
// status words: the call's status, then per window group the longest run's head count
// (k_merge_start) and whether a run outgrew the walk (k_merge_walk)
constexpr int kStatusWords = 1 + 2 * kMaxGroups;

// allow_groups = false: one window group (batched calls overlap whole jobs instead).
bool make_plan(size_t n, const msm_opts* o, Plan* p, bool allow_groups = true) {
    if (!o) return false;
    p->n = n;
    p->edw = (o->flags & MSM377_EDWARDS) ? 1 : 0;
    p->glv = (o->flags & MSM377_GLV) ? 1 : 0;
    p->pre = (o->flags & MSM377_PRECOMPUTED) ? 1 : 0;
    // precomputed sets are Edwards stored points made for one explicit c
    if (p->pre && (!p->edw || !(o->flags & MSM377_POINTS_PREPARED) || o->c == 0)) return false;
    p->stored_vec = p->edw ? ModelEdwards::kStored : ModelXyzz::kStored;
    p->sgn = o->signed_digits ? 1 : 0;
    p->user_bits = o->scalar_bits ? o->scalar_bits : 256;
    if (p->user_bits < 1 || p->user_bits > 256) return false;
    p->bits = p->glv ? 127 : p->user_bits;  // GLV halves are below 2^127
    p->c = o->c ? o->c : default_c(n, p->sgn, o->flags);
    if (p->c < 2 || p->c > 20) return false;
    if (n >= (1ull << 30)) return false;
    const size_t np = p->glv ? 2 * n : n;
    p->np = np;
    p->Wd = p->sgn ? (p->bits + 1 + p->c - 1) / p->c : (p->bits + p->c - 1) / p->c;
    p->W = p->pre ? 1 : p->Wd;
    p->items = p->pre ? (size_t)p->Wd * np : np;
    if (p->items >= (1ull << 31)) return false;
    if ((uint64_t)p->W * p->items >= (1ull << 32)) return false;   // bin offsets are 32-bit
    const size_t items = p->items;
    p->B = p->sgn ? (1u << (p->c - 1)) : ((1u << p->c) - 1u);
    p->Bp = p->sgn ? p->B : (1u << p->c);
    // keys are |digit| <= 2^(c-1) (signed) or < 2^c: c bits, sorted 8 bits per pass
    // (10-bit digits would save a pass at c = 17..20 but measured slower on GB300:
    // the 1024-bin scatter's shared-memory counters cost more than the pass)
    p->rb = 8;
    p->passes = (p->c + p->rb - 1) / p->rb;
    // Measured on GB300: the counting sort (ranks taken in the counting pass, no
    // atomics in the scatter) beats the radix passes for every plan; the radix sort
    // stays available for comparison.
    const int lgn = n > 1 ? ilog2(n) : 0;
    const int tmode = table_mode(o->flags);
    const int tsort = (p->sgn && lgn < 32) ? g_sorttable[tmode][lgn].load(std::memory_order_relaxed) : 0;
    const int tk = (p->sgn && lgn < 32) ? g_ktable[tmode][lgn].load(std::memory_order_relaxed) : 0;
    const int tr = (p->sgn && lgn < 32) ? g_rtable[tmode][lgn].load(std::memory_order_relaxed) : 0;
    const int tg = (p->sgn && lgn < 32) ? g_gtable[tmode][lgn].load(std::memory_order_relaxed) : 0;
    p->counting = ((o->flags & MSM377_RADIX_SORT) || tsort == 2) ? 0 : 1;
    p->tiles = (items + kSortTile - 1) / kSortTile;
    // Counting in shared-memory tiles when a block's packed counters fit: tiles of
    // fewer than 2^16 items, about one wave of 1024-thread blocks (two per SM when
    // the counters take at most 100 KB), and at least ~1024 items a tile.
    p->ttiles = 0;
    p->tT = 0;
    {
        const size_t smem = (size_t)((p->Bp + 2) / 2) * 4;
        if (p->counting && items > 0 && smem <= kTileSmemMax) {
            const size_t per_sm = smem <= 100 * 1024 ? 2 : 1;
            const size_t fewest = (items + kTileItemsMax - 1) / kTileItemsMax;
            size_t tl = (152 * per_sm + p->W - 1) / p->W;
            const size_t cap = (items + 1023) / 1024;
            if (tl > cap) tl = cap;
            if (tl < fewest) tl = fewest;
            if (tl < 1) tl = 1;
            p->ttiles = (uint32_t)tl;
            p->tT = (uint32_t)((items + tl - 1) / tl);
        }
    }
    // Window groups (a schedule option): the accumulation runs group by group on the
    // caller's stream and each group's merges, bucket reduction and per-window sums
    // run on a higher-priority helper stream as soon as its accumulation is done,
    // overlapping the next group's accumulation. Built-in rule: one group. Measured
    // on GB300 (Edwards + GLV, c = 16): 2^20 one group 6.17 ms, two 6.55, four 7.28;
    // 2^22 20.7 / 22.0 / 22.6 ms -- the overlapped tails slow the accumulation more
    // than they save, so the autotuner keeps one group at every size measured.
    int groups = 1;
    if (allow_groups && !p->pre) {
        groups = tg > 0 ? tg : 1;
        if (groups > p->W) groups = p->W;
        if (groups > kMaxGroups) groups = kMaxGroups;
    }
    p->gw = (p->W + groups - 1) / groups;
    p->ngroups = (p->W + p->gw - 1) / p->gw;
    // Chunks of K <= 64 items, one per thread, sized so that the chunks of one
    // accumulation launch (one window group) fill whole waves of resident threads
    // (152 SMs x kAccBlocks blocks of 128 on a GB300): m waves of K items rather than
    // a last, partly idle wave.
    const size_t kWave = (size_t)152 * 128 * (p->edw ? ModelEdwards::kAccBlocks : ModelXyzz::kAccBlocks);
    const size_t total = (size_t)p->gw * items;
    size_t waves = (total + 64 * kWave - 1) / (64 * kWave);
    if (waves < 1) waves = 1;
    size_t K = (total + waves * kWave - 1) / (waves * kWave);
    if (K < 2) K = 2;
    if (K > 64) K = 64;
    if (tk > 0) K = (size_t)tk;        // measured choice (2..256)
    p->K = (int)K;
    p->cpw = (uint32_t)((items + K - 1) / K);
    p->walk = (items + p->Bp - 1) / p->Bp <= K ? kWalkHeads : 0u;   // runs about a chunk long at most
    if (p->cpw == 0) p->cpw = 1;
    // bucket reduction geometry: segments of L buckets, the longest L that still
    // leaves kReduceThreads level-1 threads over all windows (longer segments mean
    // fewer segment sums for the bit-sum stage, but fewer threads for the running sums)
    uint64_t group_buckets = (uint64_t)p->W * p->Bp;
    uint32_t L = 2;
    const uint64_t reduce_threads = tr > 0 ? (1ull << tr) : kReduceThreads;
    while (L < p->Bp && group_buckets / (2 * L) >= reduce_threads) L <<= 1;
    if (L > p->Bp) L = p->Bp;
    p->L = L;
    p->G = p->Bp / L;
    p->logG = ilog2(p->G);
    p->log2L = ilog2(L);
    p->Q = p->G >= 8 ? p->G / 8 : 1;
    // workspace layout, 256-byte aligned pieces
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o2 = off;
        off = msm377::align_up(off + bytes, 256);
        return o2;
    };
    const size_t XY = kXyzzBytes;
    const size_t chunks = (size_t)p->W * p->cpw;
    p->off_status = take(256);
    p->off_points = take(o->flags & MSM377_POINTS_PREPARED ? 0 : np * 16 * (size_t)p->stored_vec);
    p->off_keys0 = take((size_t)p->W * items * 4);
    p->off_vals0 = take((size_t)p->W * items * 4);
    // the sort's ping-pong buffers (radix passes before the last); the last pass, or
    // the counting scatter, writes (key, value) pairs to kv
    const bool pingpong = !p->counting && p->passes > 1;
    p->off_keys1 = take(pingpong ? (size_t)p->W * items * 4 : 0);
    p->off_vals1 = take(pingpong ? (size_t)p->W * items * 4 : 0);
    p->off_kv = take((size_t)p->W * items * 8);
    p->off_rank = take(p->counting ? (size_t)p->W * items * 4 : 0);  // counting sort: rank within the bin
    p->off_hist = take((size_t)p->W * (1u << p->rb) * (p->tiles ? p->tiles : 1) * 4);
    p->off_dtot = take((size_t)p->W * (1u << p->rb) * 4);
    p->nbins = (size_t)p->W * (p->Bp + 1);  // keys 0 .. Bp of every window
    p->off_bins = take(p->nbins * 4);
    p->off_bsum = take(((p->nbins + kScanTile - 1) / kScanTile) * 4);
    p->off_tcnt = take((size_t)p->W * p->ttiles * (p->Bp + 1) * 4);
    p->off_buckets = take((size_t)p->W * p->Bp * XY);
    p->off_head = take(chunks * XY);
    p->off_tail = take(chunks * XY);
    p->off_headflag = take(chunks * 4);
    p->off_tailkey = take(chunks * 4);
    p->off_start = take(chunks * 4);
    p->off_Y = take((size_t)p->ngroups * p->gw * p->G * XY);    // per group
    p->off_V = take((size_t)p->ngroups * p->gw * p->G * XY);
    const size_t zs = (size_t)p->gw * (p->logG + 1) * p->Q;
    p->off_P0 = take((size_t)p->ngroups * zs * XY);
    p->off_P1 = take((size_t)p->ngroups * zs * XY);
    p->off_S = take((size_t)p->W * XY);
    p->total = off;
    return true;
}

// Stored points of a set: the form the pipeline gathers from (XYZZ: Montgomery
// affine, 96 B; Edwards: (x, y, k x y), 144 B), for n input points or, with GLV,
// for the 2n points P_0, phi(P_0), P_1, phi(P_1), ...
size_t stored_count(size_t n, uint32_t flags) { return (flags & MSM377_GLV) ? 2 * n : n; }
int stored_vec(uint32_t flags) { return (flags & MSM377_EDWARDS) ? ModelEdwards::kStored : ModelXyzz::kStored; }

// Stored rows of input points [a, b) (rows [a, b), or [2a, 2b) with GLV). The
// Edwards kernel's points per lane are sized for `sizing` points (0: b - a), so the
// launches of the chunks of one set, on separate streams, fill the GPU together.
void launch_prepare_range(const uint4* in, uint4* out, size_t n, size_t a, size_t b, uint32_t flags,
                          cudaStream_t s, size_t sizing = 0) {
    const size_t np = stored_count(n, flags);
    const size_t lo = stored_count(a, flags), hi = stored_count(b, flags);
    if (hi <= lo) return;
    if (flags & MSM377_EDWARDS) {
        // K points per lane: enough batches to give every resident warp (per_sm blocks
        // of 4 warps per SM) about one, at least 2 and at most 32 points per lane
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = prep_blocks_per_sm((flags & MSM377_GLV) != 0);
        const size_t items = b - a, slots = (size_t)sms * per_sm * 4;
        const size_t basis = sizing ? sizing : items;
        size_t K = (basis + 32 * slots - 1) / (32 * slots);
        K = K < 2 ? 2 : (K > 32 ? 32 : K);
        const size_t batches = (items + 32 * K - 1) / (32 * K);
        const size_t blocks = (batches + 3) / 4;
        const size_t cap = (size_t)sms * per_sm;
        const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
        if (flags & MSM377_GLV)
            k_prepare_ed<true><<<grid, 128, 0, s>>>(in, out, a, b, (int)K);
        else
            k_prepare_ed<false><<<grid, 128, 0, s>>>(in, out, a, b, (int)K);
    } else {
        k_prepare<<<msm377::grid_for(hi - lo, 256), 256, 0, s>>>(in, out, n, np, lo, hi);
    }
    msm377::note_launches(1);
}

void launch_prepare(const uint4* in, uint4* out, size_t n, uint32_t flags, cudaStream_t s) {
    launch_prepare_range(in, out, n, 0, n, flags, s);
}

template <typename T>
T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

}  // namespace

using namespace msm377;

extern "C" int msm_g1_default_c(size_t n, int signed_digits, uint32_t flags) {
    return default_c(n, signed_digits ? 1 : 0, flags);
}

extern "C" int msm_g1_set_window_table(const int32_t* c_by_log2n, int len, uint32_t flags) {
    if (len < 0 || len > 32 || (len > 0 && !c_by_log2n))
        return set_error(MSM377_EINVAL, "msm_g1_set_window_table: bad table (len %d)", len);
    if (flags & ~(MSM377_EDWARDS | MSM377_GLV | MSM377_PRECOMPUTED))
        return set_error(MSM377_EINVAL,
                         "msm_g1_set_window_table: flags 0x%x (only EDWARDS, GLV and PRECOMPUTED select a table)",
                         flags);
    for (int k = 0; k < len; ++k)
        if (c_by_log2n[k] != 0 && (c_by_log2n[k] < 2 || c_by_log2n[k] > 20))
            return set_error(MSM377_EINVAL, "msm_g1_set_window_table: c = %d at log2 n = %d", c_by_log2n[k], k);
    const int mode = table_mode(flags);
    for (int k = 0; k < 32; ++k)
        g_ctable[mode][k].store(k < len ? c_by_log2n[k] : 0, std::memory_order_relaxed);
    return MSM377_OK;
}

extern "C" int msm_g1_set_schedule(uint32_t flags, int log2n, int c, int chunk, int sort, int reduce_log2,
                                   int groups) {
    if (flags & ~(MSM377_EDWARDS | MSM377_GLV | MSM377_PRECOMPUTED))
        return set_error(MSM377_EINVAL, "msm_g1_set_schedule: flags 0x%x (only EDWARDS, GLV and PRECOMPUTED)",
                         flags);
    if (log2n < 0 || log2n >= 32 || (c && (c < 2 || c > 20)) || (chunk && (chunk < 2 || chunk > 256)) ||
        sort < 0 || sort > 2 || (reduce_log2 && (reduce_log2 < 8 || reduce_log2 > 20)) || groups < 0 ||
        groups > kMaxGroups)
        return set_error(MSM377_EINVAL, "msm_g1_set_schedule: log2n %d c %d chunk %d sort %d reduce_log2 %d groups %d",
                         log2n, c, chunk, sort, reduce_log2, groups);
    const int mode = table_mode(flags);
    g_ctable[mode][log2n].store(c, std::memory_order_relaxed);
    g_ktable[mode][log2n].store(chunk, std::memory_order_relaxed);
    g_sorttable[mode][log2n].store(sort, std::memory_order_relaxed);
    g_rtable[mode][log2n].store(reduce_log2, std::memory_order_relaxed);
    g_gtable[mode][log2n].store(groups, std::memory_order_relaxed);
    return MSM377_OK;
}

extern "C" int msm_g1_schedule(size_t n, const msm_opts* opts, int32_t* out5) {
    if (!opts || !out5) return set_error(MSM377_EINVAL, "msm_g1_schedule: NULL argument");
    Plan p;
    if (!make_plan(n, opts, &p)) return set_error(MSM377_EINVAL, "msm_g1_schedule: bad options");
    out5[0] = p.c;
    out5[1] = p.K;
    out5[2] = p.counting ? 1 : 2;
    out5[3] = ilog2((uint64_t)p.W * p.G);
    out5[4] = p.ngroups;
    return MSM377_OK;
}

extern "C" size_t msm_g1_workspace_bytes(size_t n, const msm_opts* opts) {
    Plan p;
    if (!make_plan(n, opts, &p)) return 0;
    return p.total;
}

extern "C" size_t msm_points_prepared_bytes(size_t n, uint32_t flags) {
    if (flags & ~(MSM377_EDWARDS | MSM377_GLV)) return 0;
    if (n >= (1ull << 30)) return 0;
    return stored_count(n, flags) * 16 * (size_t)stored_vec(flags);
}

extern "C" int msm_points_prepare_ex(const uint32_t* points_std, size_t n, uint32_t* out, uint32_t flags,
                                     void* stream) {
    if (flags & ~(MSM377_EDWARDS | MSM377_GLV))
        return set_error(MSM377_EINVAL, "msm_points_prepare_ex: flags 0x%x (only EDWARDS and GLV)", flags);
    if (n >= (1ull << 30)) return set_error(MSM377_EINVAL, "msm_points_prepare_ex: n = %zu too large", n);
    if (n == 0) return MSM377_OK;
    if (!points_std || !out || !aligned(points_std, 16) || !aligned(out, 16))
        return set_error(MSM377_EINVAL, "msm_points_prepare_ex: null or non-16-byte-aligned pointer");
    launch_prepare(reinterpret_cast<const uint4*>(points_std), reinterpret_cast<uint4*>(out), n, flags,
                   as_stream(stream));
    return check_launch("msm_points_prepare_ex");
}

extern "C" int msm_points_prepare(const uint32_t* points_std, size_t n, uint32_t* out, void* stream) {
    return msm_points_prepare_ex(points_std, n, out, 0, stream);
}

extern "C" size_t msm_points_precomputed_bytes(size_t n, const msm_opts* opts) {
    if (!opts || !(opts->flags & MSM377_PRECOMPUTED)) return 0;
    msm_opts o = *opts;
    o.flags |= MSM377_POINTS_PREPARED;
    Plan p;
    if (!make_plan(n, &o, &p)) return 0;
    return p.items * 16 * (size_t)ModelEdwards::kStored;
}

extern "C" int msm_points_precompute(const uint32_t* points_std, size_t n, uint32_t* out, const msm_opts* opts) {
    if (!opts) return set_error(MSM377_EINVAL, "msm_points_precompute: opts is NULL");
    if (msm_points_precomputed_bytes(n > 0 ? n : 1, opts) == 0)  // options valid (n = 0 needs 0 bytes)
        return set_error(MSM377_EINVAL,
                         "msm_points_precompute: needs MSM377_EDWARDS | MSM377_PRECOMPUTED, an explicit c and "
                         "valid options (c=%d scalar_bits=%d)", opts->c, opts->scalar_bits);
    if (n == 0) return MSM377_OK;
    if (!points_std || !out || !aligned(points_std, 16) || !aligned(out, 16))
        return set_error(MSM377_EINVAL, "msm_points_precompute: null or non-16-byte-aligned pointer");
    msm_opts o = *opts;
    o.flags |= MSM377_POINTS_PREPARED;
    Plan p;
    make_plan(n, &o, &p);
    cudaStream_t s = as_stream(opts->stream);
    const size_t threads = (p.np + kEdChunk - 1) / kEdChunk;  // whole warps: grid_for rounds up to 128
    k_precompute_ed<<<grid_for(threads, 128), 128, 0, s>>>(reinterpret_cast<const uint4*>(points_std),
                                                           reinterpret_cast<uint4*>(out), n, p.np, p.c, p.Wd);
    note_launches(1);
    return check_launch("msm_points_precompute");
}

namespace {

// Phase 1-3 of one MSM on stream s: status reset, preparation, digits, sort,
// bucket reset. Fills `a` with the job's accumulation arguments.
// reset_status = false: the caller has cleared the status word and the merge
// counter already (msm_g1_host validates point chunks on a helper stream first).
int enqueue_head(const Plan& p, const uint32_t* points, const uint32_t* scalars, void* workspace,
                 const msm_opts* opts, cudaStream_t s, AccArgs* a_out, bool reset_status = true) {
    const size_t n = p.n;
    int* status = at<int>(workspace, p.off_status);
    if (reset_status)
        MSM_CUDA_TRY(cudaMemsetAsync(status, 0, kStatusWords * sizeof(int), s));  // status, longest runs
    const uint4* pts = reinterpret_cast<const uint4*>(points);
    if ((opts->flags & MSM377_VALIDATE) && !(opts->flags & MSM377_POINTS_PREPARED)) {
        const int r = launch_validate(points, n, (opts->flags & (MSM377_EDWARDS | MSM377_GLV)) != 0, status, s);
        if (r) return r;
    }
    if (!(opts->flags & MSM377_POINTS_PREPARED)) {
        uint4* prep = at<uint4>(workspace, p.off_points);
        launch_prepare(pts, prep, n, opts->flags, s);
        pts = prep;
    }
    const size_t np = p.items;  // items per pipeline window
    uint32_t* keys[2] = {at<uint32_t>(workspace, p.off_keys0), at<uint32_t>(workspace, p.off_keys1)};
    uint32_t* vals[2] = {at<uint32_t>(workspace, p.off_vals0), at<uint32_t>(workspace, p.off_vals1)};
    uint2* kv = at<uint2>(workspace, p.off_kv);
    k_digits<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const uint4*>(scalars), n, p.c, p.Wd,
                                              p.sgn, p.user_bits, p.glv, p.pre, keys[0], vals[0], status);
    note_launches(1);
    int cur = 0;
    if (p.counting) {
        // counting sort: count, scan, scatter (window-major bins, window w at w np)
        const size_t total = (size_t)p.W * np;
        const uint32_t nb = p.Bp + 1;
        uint32_t* bins = at<uint32_t>(workspace, p.off_bins);
        uint32_t* bsum = at<uint32_t>(workspace, p.off_bsum);
        uint32_t* rank = at<uint32_t>(workspace, p.off_rank);
        const size_t ntiles = (p.nbins + kScanTile - 1) / kScanTile;
        const dim3 gw(grid_for(np, 256), (unsigned)p.W);
        uint32_t* tcnt = at<uint32_t>(workspace, p.off_tcnt);
        if (p.ttiles) {
            // the counters of one block exceed the default 48 KB of dynamic shared memory
            const size_t smem = (size_t)((nb + 1) / 2) * 4;
            MSM_CUDA_TRY(cudaFuncSetAttribute(k_tile_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kTileSmemMax));
            k_tile_count<<<dim3(p.ttiles, (unsigned)p.W), kTileThreads, smem, s>>>(keys[0], np, nb, p.tT, p.ttiles,
                                                                                  tcnt, rank);
            k_tile_totals<<<grid_for(p.nbins, 256), 256, 0, s>>>(tcnt, nb, p.ttiles, (uint32_t)p.W, bins);
        } else {
            MSM_CUDA_TRY(cudaMemsetAsync(bins, 0, p.nbins * 4, s));
            k_bin_count<<<gw, 256, 0, s>>>(keys[0], np, nb, bins, rank);
        }
        k_scan_tiles<<<(unsigned)ntiles, kScanBlock, 0, s>>>(bins, p.nbins, bsum);
        k_scan_totals<<<1, kScanBlock, 0, s>>>(bsum, ntiles);
        k_scan_add<<<grid_for(p.nbins, 256), 256, 0, s>>>(bins, p.nbins, bsum);
        if (p.ttiles) {
            k_tile_offsets<<<grid_for(p.nbins, 256), 256, 0, s>>>(tcnt, nb, p.ttiles, (uint32_t)p.W, bins);
            k_tile_scatter<<<gw, 256, 0, s>>>(keys[0], vals[0], rank, kv, total, np, nb, p.tT, p.ttiles, tcnt);
        } else {
            k_bin_scatter<<<gw, 256, 0, s>>>(keys[0], vals[0], rank, kv, total, np, nb, bins);
        }
        note_launches(p.ttiles ? 7 : 5);
    } else {
        uint32_t* hist = at<uint32_t>(workspace, p.off_hist);
        uint32_t* dtot = at<uint32_t>(workspace, p.off_dtot);
        for (int pass = 0; pass < p.passes; ++pass) {
            const int shift = p.rb * pass;
            const dim3 g((unsigned)p.tiles, (unsigned)p.W);
            k_sort_hist<8><<<g, kSortThreads, 0, s>>>(keys[cur], np, shift, p.tiles, hist);
            k_sort_scan_tiles<8><<<dim3(1u << 8, p.W), kSortThreads, 0, s>>>(hist, p.tiles, dtot);
            k_sort_scan_digits<8><<<p.W, kSortThreads, 0, s>>>(dtot);
            uint2* last = pass == p.passes - 1 ? kv : nullptr;
            k_sort_scatter<8><<<g, kSortThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], last,
                                                         np, shift, p.tiles, hist, dtot);
            note_launches(4);
            cur ^= 1;
        }
    }
    uint4* buckets = at<uint4>(workspace, p.off_buckets);
    MSM_CUDA_TRY(cudaMemsetAsync(buckets, 0, (size_t)p.W * p.Bp * kXyzzBytes, s));
    AccArgs& a = *a_out;
    a.kv = kv;
    a.pts = pts;
    a.buckets = buckets;
    a.head = at<uint4>(workspace, p.off_head);
    a.tail = at<uint4>(workspace, p.off_tail);
    a.headflag = at<uint32_t>(workspace, p.off_headflag);
    a.tailkey = at<uint32_t>(workspace, p.off_tailkey);
    a.n = np;
    a.cpw = p.cpw;
    a.Bp = p.Bp;
    a.K = p.K;
    a.w0 = 0;
    a.nwin = p.W;
    a.bin = p.counting ? at<uint32_t>(workspace, p.off_bins) : nullptr;
    a.nb = p.Bp + 1;
    return check_launch("msm head");
}

// Phase 5-6 and the per-window sums of stage 7 for the windows of one group
// (a.w0 .. a.w0 + a.nwin - 1) on stream s: partial merges, bucket reduction, and
// S_w for each window, in group g's buffers.
template <class M>
int enqueue_group_tail_m(const Plan& p, const AccArgs& a, int g, void* workspace, cudaStream_t s) {
    const size_t yv = (size_t)p.gw * p.G * kXyzzVec;
    const size_t zs = (size_t)p.gw * (p.logG + 1) * p.Q * kXyzzVec;
    uint4* Y = at<uint4>(workspace, p.off_Y) + (size_t)g * yv;
    uint4* V = at<uint4>(workspace, p.off_V) + (size_t)g * yv;
    uint4* P0 = at<uint4>(workspace, p.off_P0) + (size_t)g * zs;
    uint4* P1 = at<uint4>(workspace, p.off_P1) + (size_t)g * zs;
    uint4* S = at<uint4>(workspace, p.off_S);
    const size_t nchunks = (size_t)a.nwin * p.cpw;
    // 5. merge partial sums of runs crossing chunk edges (log depth)
    int32_t* start = at<int32_t>(workspace, p.off_start);
    int* maxspan = at<int>(workspace, p.off_status) + 1 + g;
    // the walk's flag, or null without a walk (a one-byte memset in its place made 64
    // graph-captured batched MSMs 37 -> 52 ms on GB300)
    int* longrun = p.walk ? at<int>(workspace, p.off_status) + 1 + kMaxGroups + g : nullptr;
    if (p.walk) {
        k_merge_walk<M><<<grid_for(nchunks, 128), 128, 0, s>>>(a, p.walk, longrun);
        note_launches(1);
    }
    k_merge_start<<<grid_for(nchunks, 128), 128, 0, s>>>(a, longrun, start, maxspan);
    note_launches(1);
    for (uint32_t d = 1; d < p.cpw && d < kMergeRounds; d <<= 1) {
        k_merge_round<M><<<grid_for(nchunks, 128), 128, 0, s>>>(a, start, d, maxspan);
        note_launches(1);
    }
    if (p.cpw > kMergeRounds) {
        int dev = 0, sms = 152;
        MSM_CUDA_TRY(cudaGetDevice(&dev));
        MSM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const size_t want = (nchunks + kMergeLongThreads - 1) / kMergeLongThreads, cap = (size_t)sms * 4;
        k_merge_long<M><<<(unsigned)(want < cap ? want : cap), kMergeLongThreads, 0, s>>>(a, start, maxspan);
        note_launches(1);
    }
    k_merge_final<M><<<grid_for(nchunks, 128), 128, 0, s>>>(a, longrun);
    note_launches(1);
    // 6. bucket reduction of the group's windows
    const size_t WG = (size_t)a.nwin * p.G;
    k_reduce_segments<M><<<grid_for(WG, 128), 128, 0, s>>>(a.buckets, p.Bp, p.L, a.w0, a.nwin, p.G, Y, V);
    const size_t nseg = (size_t)a.nwin * (p.logG + 1);
    k_bitsums<M><<<grid_for(nseg * p.Q, 128), 128, 0, s>>>(Y, V, a.nwin, p.G, p.logG, p.Q, P0);
    note_launches(2);
    uint32_t m = p.Q;
    uint4* zin = P0;
    uint4* zout = P1;
    while (m > 1) {
        uint32_t F = 2;  // per-group fan-in: about one wave of blocks, at most 8 sequential additions
        while (F < 8 && nseg * ((m + kTreeGroups * F - 1) / (kTreeGroups * F)) > kTreeWave) F <<= 1;
        const uint32_t nb = (m + kTreeGroups * F - 1) / (kTreeGroups * F);
        k_sum_tree<M><<<(unsigned)(nseg * nb), kTreeThreads, 0, s>>>(zin, nseg, m, F, zout);
        note_launches(1);
        m = nb;
        uint4* tmp = zin;
        zin = zout;
        zout = tmp;
    }
    // 7a. the per-window sums S_w
    k_window_horner_w<M><<<(unsigned)a.nwin, 128, 0, s>>>(zin, a.nwin, p.logG, p.log2L, S + (size_t)a.w0 * kXyzzVec);
    note_launches(1);
    return check_launch("msm tail");
}

int enqueue_group_tail(const Plan& p, const AccArgs& a, int g, void* workspace, cudaStream_t s) {
    return p.edw ? enqueue_group_tail_m<ModelEdwards>(p, a, g, workspace, s)
                 : enqueue_group_tail_m<ModelXyzz>(p, a, g, workspace, s);
}

// 7b. the window combination and normalisation into out.
int enqueue_chain(const Plan& p, void* workspace, uint32_t* out, cudaStream_t s) {
    const uint4* S = at<uint4>(workspace, p.off_S);
    if (p.edw)
        k_chain_w<ModelEdwards><<<1, 128, 0, s>>>(S, p.W, p.c, out);
    else
        k_chain_w<ModelXyzz><<<1, 128, 0, s>>>(S, p.W, p.c, out);
    note_launches(1);
    return check_launch("msm chain");
}

// Phase 5-7 of one MSM as a single window group on stream s (batched calls).
int enqueue_tail(const Plan& p, const AccArgs& a, void* workspace, uint32_t* out, cudaStream_t s) {
    int r = enqueue_group_tail(p, a, 0, workspace, s);
    if (r) return r;
    return enqueue_chain(p, workspace, out, s);
}

// Accumulation of the windows a.w0 .. a.w0 + a.nwin - 1.
int enqueue_accumulate(const Plan& p, const AccArgs& a, cudaStream_t s) {
    const unsigned grid = grid_for((size_t)a.nwin * p.cpw, 128);
    if (p.edw)
        k_accumulate<ModelEdwards><<<grid, 128, 0, s>>>(a);
    else
        k_accumulate<ModelXyzz><<<grid, 128, 0, s>>>(a);
    note_launches(1);
    return check_launch("msm accumulate");
}

// A helper stream of the highest priority and events, one set per caller stream
// (so calls on different streams never share them), created on first use.
struct Overlap {
    cudaStream_t hi;
    cudaEvent_t ev[kMaxGroups + 1];
};
constexpr int kOverlapSlots = 32;
struct OverlapSlot {
    bool used = false;
    int dev = -1;
    cudaStream_t caller = nullptr;
    Overlap ov;
};
OverlapSlot g_overlap[kOverlapSlots];
std::mutex g_overlap_mu;

// nullptr when every slot is taken: the groups then run in sequence on s.
const Overlap* overlap_for(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(g_overlap_mu);
    for (auto& sl : g_overlap)
        if (sl.used && sl.dev == dev && sl.caller == s) return &sl.ov;
    for (auto& sl : g_overlap) {
        if (sl.used) continue;
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return nullptr;
        if (cudaStreamCreateWithPriority(&sl.ov.hi, cudaStreamNonBlocking, greatest) != cudaSuccess) return nullptr;
        for (int i = 0; i <= kMaxGroups; ++i)
            if (cudaEventCreateWithFlags(&sl.ov.ev[i], cudaEventDisableTiming) != cudaSuccess) return nullptr;
        sl.used = true;
        sl.dev = dev;
        sl.caller = s;
        return &sl.ov;
    }
    return nullptr;
}

// Phase 4-7 on stream s: the accumulation group by group, each group's tail on the
// high-priority helper as soon as its accumulation is done (overlapping the next
// group's accumulation), then the window chain on s. Without a helper (ov null, or
// one group) everything runs in order on s. prof: stage marks after the last
// accumulation and after the chain.
int enqueue_body(const Plan& p, const AccArgs& a, void* workspace, uint32_t* out, cudaStream_t s, const Overlap* ov,
                 bool prof) {
    int r;
    if (p.ngroups <= 1 || !ov) {
        for (int g = 0; g < p.ngroups; ++g) {
            AccArgs ag = a;
            ag.w0 = g * p.gw;
            ag.nwin = (p.W - ag.w0) < p.gw ? (p.W - ag.w0) : p.gw;
            if ((r = enqueue_accumulate(p, ag, s))) return r;
        }
        if (prof) profile_mark(s);
        for (int g = 0; g < p.ngroups; ++g) {
            AccArgs ag = a;
            ag.w0 = g * p.gw;
            ag.nwin = (p.W - ag.w0) < p.gw ? (p.W - ag.w0) : p.gw;
            if ((r = enqueue_group_tail(p, ag, g, workspace, s))) return r;
        }
    } else {
        for (int g = 0; g < p.ngroups; ++g) {
            AccArgs ag = a;
            ag.w0 = g * p.gw;
            ag.nwin = (p.W - ag.w0) < p.gw ? (p.W - ag.w0) : p.gw;
            if ((r = enqueue_accumulate(p, ag, s))) return r;
            MSM_CUDA_TRY(cudaEventRecord(ov->ev[g], s));
            MSM_CUDA_TRY(cudaStreamWaitEvent(ov->hi, ov->ev[g], 0));
            if ((r = enqueue_group_tail(p, ag, g, workspace, ov->hi))) return r;
        }
        if (prof) profile_mark(s);
        MSM_CUDA_TRY(cudaEventRecord(ov->ev[kMaxGroups], ov->hi));
        MSM_CUDA_TRY(cudaStreamWaitEvent(s, ov->ev[kMaxGroups], 0));
    }
    if ((r = enqueue_chain(p, workspace, out, s))) return r;
    if (prof) profile_mark(s);
    return MSM377_OK;
}

// Library-owned helper streams for batched calls, per device, created once.
constexpr int kMaxDevices = 64;
constexpr int kAuxStreams = 16;
constexpr int kHostChunks = 4;  // the copy (about 200 GB/s) is shorter than the preparation; small first chunk
constexpr size_t kSplitPrepMin = size_t(1) << 15;  // msm_g1: prepare beside the head from this size on
static_assert(1 + kHostChunks <= kAuxStreams, "msm_g1_host needs a copy stream and one stream per chunk");
struct DeviceAux {
    bool ready = false;
    int sms = 0, acc_blocks_per_sm[2] = {0, 0};  // k_accumulate_batched per model
    cudaStream_t st[kAuxStreams];
    cudaEvent_t fork, done[kAuxStreams];
    cudaEvent_t chunk[kHostChunks];  // msm_g1_host: point chunk k has arrived
};
DeviceAux g_aux[kMaxDevices];
std::mutex g_aux_mu;

int device_aux(DeviceAux** out) {
    int dev = 0;
    MSM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(MSM377_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_aux_mu);
    DeviceAux& a = g_aux[dev];
    if (!a.ready) {
        MSM_CUDA_TRY(cudaDeviceGetAttribute(&a.sms, cudaDevAttrMultiProcessorCount, dev));
        MSM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a.acc_blocks_per_sm[0],
                                                                   k_accumulate_batched<ModelXyzz>, 128, 0));
        MSM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a.acc_blocks_per_sm[1],
                                                                   k_accumulate_batched<ModelEdwards>, 128, 0));
        for (int m = 0; m < 2; ++m)
            if (a.acc_blocks_per_sm[m] < 1) a.acc_blocks_per_sm[m] = 1;
        for (int i = 0; i < kAuxStreams; ++i) {
            MSM_CUDA_TRY(cudaStreamCreateWithFlags(&a.st[i], cudaStreamNonBlocking));
            MSM_CUDA_TRY(cudaEventCreateWithFlags(&a.done[i], cudaEventDisableTiming));
        }
        MSM_CUDA_TRY(cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming));
        for (int k = 0; k < kHostChunks; ++k) MSM_CUDA_TRY(cudaEventCreateWithFlags(&a.chunk[k], cudaEventDisableTiming));
        a.ready = true;
    }
    *out = &a;
    return MSM377_OK;
}

// Helper streams wait for work already on s; then s waits for the helpers.
int fork_from(DeviceAux* aux, cudaStream_t s, int k) {
    MSM_CUDA_TRY(cudaEventRecord(aux->fork, s));
    for (int i = 0; i < k; ++i) MSM_CUDA_TRY(cudaStreamWaitEvent(aux->st[i], aux->fork, 0));
    return MSM377_OK;
}
int join_into(DeviceAux* aux, cudaStream_t s, int k) {
    for (int i = 0; i < k; ++i) {
        MSM_CUDA_TRY(cudaEventRecord(aux->done[i], aux->st[i]));
        MSM_CUDA_TRY(cudaStreamWaitEvent(s, aux->done[i], 0));
    }
    return MSM377_OK;
}

}  // namespace

namespace msm377 {

int msm_g1_run(const uint32_t* points, const uint32_t* scalars, size_t n, uint32_t* out, void* workspace,
               size_t workspace_bytes, const msm_opts* opts, bool overlap) {
    if (!opts) return set_error(MSM377_EINVAL, "msm_g1: opts is NULL");
    if (!out) return set_error(MSM377_EINVAL, "msm_g1: out is NULL");
    cudaStream_t s = as_stream(opts->stream);
    Plan p;
    if (!make_plan(n, opts, &p))
        return set_error(MSM377_EINVAL, "msm_g1: bad options (c=%d scalar_bits=%d) or n too large",
                         opts->c, opts->scalar_bits);
    if (!workspace || !aligned(workspace, 256))
        return set_error(MSM377_EINVAL, "msm_g1: workspace NULL or not 256-byte aligned");
    if (workspace_bytes < p.total)
        return set_error(MSM377_ENOMEM, "msm_g1: workspace %zu bytes, need %zu", workspace_bytes, p.total);
    if ((opts->flags & MSM377_VALIDATE) && (opts->flags & MSM377_POINTS_PREPARED))
        return set_error(MSM377_EINVAL, "msm_g1: MSM377_VALIDATE checks standard-form input points; stored "
                         "(prepared) points are validated when the set is made (msm_points_create)");
    const bool prof = (opts->flags & MSM377_PROFILE) != 0;
    if (prof) {
        int pr = profile_begin(s);
        if (pr) return pr;
    }
    if (n == 0) {
        MSM_CUDA_TRY(cudaMemsetAsync(at<int>(workspace, p.off_status), 0, sizeof(int), s));
        MSM_CUDA_TRY(cudaMemsetAsync(out, 0, 24 * sizeof(uint32_t), s));
        return MSM377_OK;
    }
    if (!points || !scalars || !aligned(points, 16) || !aligned(scalars, 16))
        return set_error(MSM377_EINVAL, "msm_g1: points/scalars NULL or not 16-byte aligned");
    AccArgs a;
    // Standard-form points: their preparation (and validation) runs on the caller
    // stream's high-priority helper while the digits and the sort, which need only
    // the scalars, run on s; the accumulation waits for both.
    const bool split = overlap && !prof && !(opts->flags & MSM377_POINTS_PREPARED) && n >= kSplitPrepMin;
    const Overlap* ov = (overlap && (p.ngroups > 1 || split)) ? overlap_for(s) : nullptr;
    int r;
    if (split && ov) {
        int* status = at<int>(workspace, p.off_status);
        MSM_CUDA_TRY(cudaMemsetAsync(status, 0, kStatusWords * sizeof(int), s));
        MSM_CUDA_TRY(cudaEventRecord(ov->ev[0], s));
        MSM_CUDA_TRY(cudaStreamWaitEvent(ov->hi, ov->ev[0], 0));
        if (opts->flags & MSM377_VALIDATE) {
            r = launch_validate(points, n, (opts->flags & (MSM377_EDWARDS | MSM377_GLV)) != 0, status, ov->hi);
            if (r) return r;
        }
        uint4* prep = at<uint4>(workspace, p.off_points);
        launch_prepare(reinterpret_cast<const uint4*>(points), prep, n, opts->flags, ov->hi);
        MSM_CUDA_TRY(cudaEventRecord(ov->ev[1], ov->hi));
        msm_opts op = *opts;
        op.flags |= MSM377_POINTS_PREPARED;  // the plan keeps the prepared region in the workspace
        r = enqueue_head(p, reinterpret_cast<const uint32_t*>(prep), scalars, workspace, &op, s, &a, false);
        if (r) return r;
        MSM_CUDA_TRY(cudaStreamWaitEvent(s, ov->ev[1], 0));
    } else {
        r = enqueue_head(p, points, scalars, workspace, opts, s, &a);
        if (r) return r;
    }
    if (prof) profile_mark(s);
    return enqueue_body(p, a, workspace, out, s, p.ngroups > 1 ? ov : nullptr, prof);
}

}  // namespace msm377

extern "C" int msm_g1(const uint32_t* points, const uint32_t* scalars, size_t n, uint32_t* out,
                      void* workspace, size_t workspace_bytes, const msm_opts* opts) {
    return msm_g1_run(points, scalars, n, out, workspace, workspace_bytes, opts, true);
}

namespace {
constexpr size_t kBatchHeader = 256;

// c for job i of a batch: the job's own, else the options', else the size default.
bool batch_plans(const msm_job* jobs, size_t njobs, const msm_opts* opts, Plan* plans, size_t* total) {
    size_t off = kBatchHeader;
    for (size_t i = 0; i < njobs; ++i) {
        msm_opts o = *opts;
        if (jobs[i].c) o.c = jobs[i].c;
        if (!make_plan(jobs[i].n, &o, &plans[i], false)) return false;
        off += align_up(plans[i].total, 256);
    }
    *total = off;
    return true;
}
}  // namespace

extern "C" size_t msm_g1_batched_workspace_bytes(const msm_job* jobs, size_t njobs, const msm_opts* opts) {
    if (!jobs || !opts || njobs == 0 || njobs > (size_t)kMaxBatch) return 0;
    Plan plans[kMaxBatch];
    size_t total = 0;
    if (!batch_plans(jobs, njobs, opts, plans, &total)) return 0;
    return total;
}

extern "C" int msm_g1_batched(const msm_job* jobs, size_t njobs, void* workspace, size_t workspace_bytes,
                              const msm_opts* opts) {
    if (!jobs || !opts) return set_error(MSM377_EINVAL, "msm_g1_batched: NULL argument");
    if (njobs == 0) return MSM377_OK;
    if (njobs > (size_t)kMaxBatch)
        return set_error(MSM377_EINVAL, "msm_g1_batched: %zu jobs, at most %d per call", njobs, kMaxBatch);
    if (opts->flags & (MSM377_PROFILE | MSM377_VALIDATE))
        return set_error(MSM377_EINVAL, "msm_g1_batched: MSM377_PROFILE and MSM377_VALIDATE are not supported "
                         "(validate point sets once with msm_points_validate or msm_points_create)");
    Plan plans[kMaxBatch];
    size_t total = 0;
    if (!batch_plans(jobs, njobs, opts, plans, &total))
        return set_error(MSM377_EINVAL, "msm_g1_batched: bad options or n too large in some job");
    if (!workspace || !aligned(workspace, 256))
        return set_error(MSM377_EINVAL, "msm_g1_batched: workspace NULL or not 256-byte aligned");
    if (workspace_bytes < total)
        return set_error(MSM377_ENOMEM, "msm_g1_batched: workspace %zu bytes, need %zu", workspace_bytes, total);
    for (size_t i = 0; i < njobs; ++i) {
        if (!jobs[i].out) return set_error(MSM377_EINVAL, "msm_g1_batched: job %zu has no output", i);
        if (jobs[i].n && (!jobs[i].points || !jobs[i].scalars || !aligned(jobs[i].points, 16) ||
                          !aligned(jobs[i].scalars, 16)))
            return set_error(MSM377_EINVAL, "msm_g1_batched: job %zu points/scalars NULL or misaligned", i);
    }
    DeviceAux* aux = nullptr;
    int r = device_aux(&aux);
    if (r) return r;
    cudaStream_t s = as_stream(opts->stream);
    const int nst = njobs < (size_t)kAuxStreams ? (int)njobs : kAuxStreams;

    // heads of all jobs on the helper streams
    BatchAcc b;
    b.njobs = 0;
    b.prefix[0] = 0;
    uint32_t* counter = static_cast<uint32_t*>(workspace);
    MSM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(uint32_t), s));
    r = fork_from(aux, s, nst);
    if (r) return r;
    char* base = static_cast<char*>(workspace) + kBatchHeader;
    void* ws[kMaxBatch];
    for (size_t i = 0; i < njobs; ++i) {
        ws[i] = base;
        base += align_up(plans[i].total, 256);
        cudaStream_t si = aux->st[i % nst];
        if (jobs[i].n == 0) {
            MSM_CUDA_TRY(cudaMemsetAsync(jobs[i].out, 0, 24 * sizeof(uint32_t), si));
            continue;
        }
        r = enqueue_head(plans[i], jobs[i].points, jobs[i].scalars, ws[i], opts, si, &b.job[b.njobs]);
        if (r) return r;
        b.prefix[b.njobs + 1] = b.prefix[b.njobs] + (uint32_t)(plans[i].W * plans[i].cpw);
        ++b.njobs;
    }
    r = join_into(aux, s, nst);
    if (r) return r;

    // every job's bucket accumulation in one persistent launch
    if (b.njobs > 0) {
        b.counter = counter;
        const int edw = (opts->flags & MSM377_EDWARDS) ? 1 : 0;
        const unsigned grid = (unsigned)(aux->sms * aux->acc_blocks_per_sm[edw]);
        if (edw)
            k_accumulate_batched<ModelEdwards><<<grid, 128, 0, s>>>(b);
        else
            k_accumulate_batched<ModelXyzz><<<grid, 128, 0, s>>>(b);
        note_launches(1);
        r = check_launch("msm_g1_batched accumulate");
        if (r) return r;
    }

    // tails of all jobs on the helper streams
    r = fork_from(aux, s, nst);
    if (r) return r;
    for (size_t i = 0, k = 0; i < njobs; ++i) {
        if (jobs[i].n == 0) continue;
        r = enqueue_tail(plans[i], b.job[k], ws[i], jobs[i].out, aux->st[i % nst]);
        if (r) return r;
        ++k;
    }
    return join_into(aux, s, nst);
}

extern "C" int msm_g1_status(const void* workspace, const msm_opts* opts) {
    if (!workspace || !opts) return set_error(MSM377_EINVAL, "msm_g1_status: NULL argument");
    int st = 0;
    cudaStream_t s = as_stream(opts->stream);
    MSM_CUDA_TRY(cudaMemcpyAsync(&st, workspace, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st == MSM377_ERANGE) return set_error(MSM377_ERANGE, "msm_g1: a scalar exceeds scalar_bits");
    if (st == MSM377_ENOTONCURVE)
        return set_error(MSM377_ENOTONCURVE, "msm_g1: an input point is not on the curve (or, with "
                         "MSM377_EDWARDS / MSM377_GLV, not in the order-r subgroup)");
    return st;
}

extern "C" size_t msm_g1_host_workspace_bytes(size_t n, const msm_opts* opts) {
    if (!opts) return 0;
    msm_opts o = *opts;
    o.flags &= ~MSM377_POINTS_PREPARED;
    size_t core = msm_g1_workspace_bytes(n, &o);
    if (!core) return 0;
    return core + align_up(n * 96, 256) + align_up(n * 32, 256) + 256;
}

extern "C" int msm_g1_host(const uint32_t* points_host, const uint32_t* scalars_host, size_t n,
                           uint32_t* out_host, void* workspace, size_t workspace_bytes,
                           const msm_opts* opts) {
    if (!opts || !out_host || !workspace) return set_error(MSM377_EINVAL, "msm_g1_host: NULL argument");
    if (n && (!points_host || !scalars_host)) return set_error(MSM377_EINVAL, "msm_g1_host: NULL inputs");
    size_t need = msm_g1_host_workspace_bytes(n, opts);
    if (!need) return set_error(MSM377_EINVAL, "msm_g1_host: bad options");
    if (workspace_bytes < need)
        return set_error(MSM377_ENOMEM, "msm_g1_host: workspace %zu bytes, need %zu", workspace_bytes, need);
    if (!aligned(workspace, 256)) return set_error(MSM377_EINVAL, "msm_g1_host: workspace not 256-byte aligned");
    msm_opts o = *opts;
    o.flags &= ~(MSM377_POINTS_PREPARED | MSM377_PROFILE);
    Plan p;
    if (!make_plan(n, &o, &p)) return set_error(MSM377_EINVAL, "msm_g1_host: bad options");
    const size_t core = p.total;
    char* base = static_cast<char*>(workspace);
    uint32_t* d_pts = reinterpret_cast<uint32_t*>(base + core);
    uint32_t* d_sc = reinterpret_cast<uint32_t*>(base + core + align_up(n * 96, 256));
    uint32_t* d_out = reinterpret_cast<uint32_t*>(base + core + align_up(n * 96, 256) + align_up(n * 32, 256));
    cudaStream_t s = as_stream(o.stream);
    if (n == 0) {
        int r = msm_g1(d_pts, d_sc, 0, d_out, workspace, core, &o);
        if (r) return r;
        MSM_CUDA_TRY(cudaMemcpyAsync(out_host, d_out, 24 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        return msm_g1_status(workspace, &o);
    }
    // The points travel in chunks on one helper stream and each chunk is prepared
    // on a helper stream of its own as soon as it has arrived (the chunks' launches
    // are sized to fill the GPU together), while the scalars' copy, digits and
    // bucket sort run on the caller's stream; the accumulation waits for them all.
    DeviceAux* aux = nullptr;
    int r = device_aux(&aux);
    if (r) return r;
    cudaStream_t sc = aux->st[0];
    MSM_CUDA_TRY(cudaMemsetAsync(at<int>(workspace, p.off_status), 0, kStatusWords * sizeof(int), s));  // before the fork
    r = fork_from(aux, s, 1 + kHostChunks);
    if (r) return r;
    uint4* prep = at<uint4>(workspace, p.off_points);
    const size_t per = (n + kHostChunks - 1) / kHostChunks;
    for (int k = 0; k < kHostChunks; ++k) {
        const size_t a = (size_t)k * per, b = a + per < n ? a + per : n;
        if (a >= b) break;
        cudaStream_t sp = aux->st[1 + k];
        MSM_CUDA_TRY(cudaMemcpyAsync(d_pts + 24 * a, points_host + 24 * a, (b - a) * 96, cudaMemcpyHostToDevice, sc));
        MSM_CUDA_TRY(cudaEventRecord(aux->chunk[k], sc));
        MSM_CUDA_TRY(cudaStreamWaitEvent(sp, aux->chunk[k], 0));
        if (o.flags & MSM377_VALIDATE) {
            r = launch_validate(d_pts + 24 * a, b - a, (o.flags & (MSM377_EDWARDS | MSM377_GLV)) != 0,
                                at<int>(workspace, p.off_status), sp);
            if (r) return r;
        }
        launch_prepare_range(reinterpret_cast<const uint4*>(d_pts), prep, n, a, b, o.flags, sp, n);
    }
    MSM_CUDA_TRY(cudaMemcpyAsync(d_sc, scalars_host, n * 32, cudaMemcpyHostToDevice, s));
    msm_opts op = o;
    op.flags |= MSM377_POINTS_PREPARED;  // the plan above keeps the prepared region in the workspace
    AccArgs acc;
    r = enqueue_head(p, reinterpret_cast<const uint32_t*>(prep), d_sc, workspace, &op, s, &acc, false);
    if (r) return r;
    r = join_into(aux, s, 1 + kHostChunks);
    if (r) return r;
    r = enqueue_body(p, acc, workspace, d_out, s, p.ngroups > 1 ? overlap_for(s) : nullptr, false);
    if (r) return r;
    MSM_CUDA_TRY(cudaMemcpyAsync(out_host, d_out, 24 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    return msm_g1_status(workspace, &o);
}
