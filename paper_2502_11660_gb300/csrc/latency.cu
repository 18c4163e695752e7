// The dependent-chain latency experiment of the paper (Sec. V-A): the points of a
// stream are summed strictly in order, P_0 + P_1 + ... + P_{n-1}, so every mixed
// PADD waits for the previous one and the time per PADD is its latency, not a
// throughput. The paper lowers that latency by spreading one PADD over several
// AIE tiles (its med-ind mapping); here the analogue is spreading the independent
// multiplications of one Edwards PADD over four lanes of a warp (ed::madd4: two
// multiplication latencies per addition instead of seven).
//
// Variants (padd_chain): XYZZ on one thread (10 multiplications in sequence per
// mixed addition, with the special-case branches), Edwards on one thread, Edwards
// on four lanes, and Edwards on four warps (128 threads: each product of an
// addition on its own warp and spread over that warp's lanes, wpt.cuh). Inputs are
// stored points (msm_points_prepare_ex), so the timed kernel is the chain alone.
#include <cuda_runtime.h>

#include "common.cuh"
#include "ec.cuh"
#include "ed.cuh"
#include "wpt.cuh"

namespace {

using ec::affine;
using fq::fe;

__device__ __forceinline__ void load_fe16(fe& a, const uint4* p) {
    uint4 u0 = p[0], u1 = p[1], u2 = p[2];
    a.v[0] = u0.x; a.v[1] = u0.y; a.v[2] = u0.z; a.v[3] = u0.w;
    a.v[4] = u1.x; a.v[5] = u1.y; a.v[6] = u1.z; a.v[7] = u1.w;
    a.v[8] = u2.x; a.v[9] = u2.y; a.v[10] = u2.z; a.v[11] = u2.w;
}

__device__ __forceinline__ void load_stored(ed::stored& Q, const uint4* pts, size_t i) {
    load_fe16(Q.x, pts + 9 * i);
    load_fe16(Q.y, pts + 9 * i + 3);
    load_fe16(Q.u, pts + 9 * i + 6);
}

__device__ __forceinline__ void store_affine_std(uint32_t* out, affine A) {
    if (!ec::is_inf(A)) {
        fq::from_mont(A.x, A.x);
        fq::from_mont(A.y, A.y);
    }
    fq::store(out, A.x);
    fq::store(out + 12, A.y);
}

// One thread: XYZZ accumulator += Montgomery affine points in order.
__global__ void k_chain_xyzz1(const uint4* __restrict__ pts, size_t n, uint32_t* __restrict__ out) {
    if (threadIdx.x != 0) return;
    ec::xyzz acc;
    ec::set_inf(acc);
    bool inf = true;
    affine next;
    if (n) {
        load_fe16(next.x, pts);
        load_fe16(next.y, pts + 3);
    }
    for (size_t i = 0; i < n; ++i) {
        const affine Q = next;          // the next point's loads overlap this addition
        if (i + 1 < n) {
            load_fe16(next.x, pts + 6 * (i + 1));
            load_fe16(next.y, pts + 6 * (i + 1) + 3);
        }
        ec::madd(acc, inf, Q);
    }
    affine A;
    ec::to_affine(A, acc);
    store_affine_std(out, A);
}

// One thread: Edwards accumulator += stored points (x, y, k x y) in order.
__global__ void k_chain_ed1(const uint4* __restrict__ pts, size_t n, uint32_t* __restrict__ out) {
    if (threadIdx.x != 0) return;
    ed::ext acc;
    ed::set_inf(acc);
    ed::stored next;
    if (n) load_stored(next, pts, 0);
    for (size_t i = 0; i < n; ++i) {
        const ed::stored Q = next;      // the next point's loads overlap this addition
        if (i + 1 < n) load_stored(next, pts, i + 1);
        ed::madd(acc, Q);
    }
    affine A;
    ed::to_weierstrass(A, acc);
    store_affine_std(out, A);
}

// Four lanes per addition; the eight groups of a warp compute the same chain (so
// every __syncwarp is warp-wide) and lane 0 writes the result.
__global__ void __launch_bounds__(32) k_chain_ed4(const uint4* __restrict__ pts, size_t n, uint32_t* __restrict__ out) {
    __shared__ fe sh[8][4];
    const int lane = threadIdx.x & 31, g = lane >> 2, l = lane & 3;
    ed::ext acc;
    ed::set_inf(acc);
    ed::stored next;
    if (n) load_stored(next, pts, 0);
    for (size_t i = 0; i < n; ++i) {
        const ed::stored Q = next;      // the next point's loads overlap this addition
        if (i + 1 < n) load_stored(next, pts, i + 1);
        ed::madd4(acc, Q, sh[g], l, true);
    }
    if (lane != 0) return;
    affine A;
    ed::to_weierstrass(A, acc);
    store_affine_std(out, A);
}

// Four warps per addition: level 1 {A, B, C} and level 2 {X3, Y3, T3, Z3} on one
// warp each, every product spread over the lanes of its warp.
__global__ void __launch_bounds__(128, 1) k_chain_edw(const uint4* __restrict__ pts, size_t n, uint32_t* __restrict__ out) {
    __shared__ __align__(16) uint32_t slots[wpt::kSharedWords];
    wpt::Group g;
    wpt::init(g, slots);
    wpt::ed_set_inf(g);
    const uint32_t* p = reinterpret_cast<const uint32_t*>(pts);
    wpt::Operand next = {};
    if (n) next = wpt::load_operand(p, 3);
    for (size_t i = 0; i < n; ++i) {
        const wpt::Operand q = next;    // the next point's loads overlap this addition
        if (i + 1 < n) next = wpt::load_operand(p + 36 * (i + 1), 3);
        wpt::ed_madd(g, q);
    }
    if (threadIdx.x != 0) return;
    fe c[4];
    wpt::read_acc(g, c);
    ed::ext P;
    P.X = c[0];
    P.Y = c[1];
    P.Z = c[2];
    P.T = c[3];
    affine A;
    ed::to_weierstrass(A, P);
    store_affine_std(out, A);
}

}  // namespace

using namespace msm377;

extern "C" int padd_chain(const uint32_t* points, size_t n, uint32_t* out, uint32_t flags, int lanes, void* stream) {
    if (flags & ~(uint32_t)MSM377_EDWARDS)
        return set_error(MSM377_EINVAL, "padd_chain: flags 0x%x (0 or MSM377_EDWARDS)", flags);
    if (lanes != 1 && lanes != 4 && lanes != 128)
        return set_error(MSM377_EINVAL, "padd_chain: lanes = %d (1, 4 or 128)", lanes);
    if (lanes != 1 && !(flags & MSM377_EDWARDS))
        return set_error(MSM377_EINVAL, "padd_chain: %d lanes need the Edwards model", lanes);
    if (!out || (n && (!points || !aligned(points, 16))))
        return set_error(MSM377_EINVAL, "padd_chain: NULL or non-16-byte-aligned pointer");
    cudaStream_t s = as_stream(stream);
    const uint4* p = reinterpret_cast<const uint4*>(points);
    if (flags & MSM377_EDWARDS) {
        if (lanes == 128)
            k_chain_edw<<<1, 128, 0, s>>>(p, n, out);
        else if (lanes == 4)
            k_chain_ed4<<<1, 32, 0, s>>>(p, n, out);
        else
            k_chain_ed1<<<1, 32, 0, s>>>(p, n, out);
    } else {
        k_chain_xyzz1<<<1, 32, 0, s>>>(p, n, out);
    }
    note_launches(1);
    return check_launch("padd_chain");
}
