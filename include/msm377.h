/*
 * msm377 — BLS12-377 G1 multi-scalar multiplication on NVIDIA sm_103a (GB300).
 *
 * C-ABI of the library libmsm377.so. The operation is the one arXiv:2502.11660
 * accelerates: MSM, sum_i s_i * P_i over the BLS12-377 curve with a 377-bit
 * base field (Abstract; Sec. II-C), computed by Pippenger's bucket method as a
 * stream of elliptic-curve point additions (PADDs, Sec. II-D).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Field elements: 12 little-endian 32-bit limbs. STANDARD form is the integer
 *   x in [0, p); MONTGOMERY form is x * 2^384 mod p in [0, p).
 * - Affine points: x then y (24 u32). The identity O is (0, 0), which is not on
 *   y^2 = x^3 + 1.
 * - XYZZ points (x = X/ZZ, y = Y/ZZZ): X, Y, ZZ, ZZZ; the identity has ZZ = 0.
 * - Scalars: 8 little-endian 32-bit limbs (any 256-bit value is accepted).
 * - Ownership: the caller allocates and frees every buffer. Pointers are device
 *   pointers unless the name ends in _host. No call keeps a pointer after it
 *   returns. The exception is a resident set (msm_points_create): a copy of the
 *   caller's points in the library's own device memory until msm_points_destroy.
 * - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream). Calls only enqueue work on it and return, except those marked
 *   "synchronous".
 * - Inputs out of their stated range (coordinates >= p, points off the curve)
 *   produce unspecified output values but never out-of-bounds accesses, unless
 *   the call is asked to check them (MSM377_VALIDATE, msm_points_validate).
 * - Every call returns a status code below; on MSM377_ECUDA and MSM377_EINVAL,
 *   msm377_last_error() holds a message.
 */
#ifndef MSM377_H
#define MSM377_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSM377_OK 0
#define MSM377_EINVAL (-1)   /* bad argument: null pointer, misalignment, size, option */
#define MSM377_ENOMEM (-2)   /* the workspace passed is smaller than required */
#define MSM377_ECUDA (-3)    /* a CUDA runtime call failed */
#define MSM377_ETIMEOUT (-4) /* a bounded device-side wait gave up */
#define MSM377_ENOTONCURVE (-5) /* MSM377_VALIDATE: an input point is not on y^2 = x^3 + 1 (or has a
                                   coordinate >= p), or, where the curve model needs it, is not in the
                                   order-r subgroup */
#define MSM377_ERANGE (-6)   /* a scalar had bits at or above opts.scalar_bits */

#define MSM377_FORM_STANDARD 0
#define MSM377_FORM_MONTGOMERY 1

/* Copies the last error message of the calling thread into buf (NUL-terminated,
 * truncated to len). Returns the length of the full message. */
int msm377_last_error(char *buf, size_t len);

/* Library version, major * 10000 + minor * 100 + patch. */
int msm377_version(void);

/* ------------------------------------------------------------------------
 * Batched field multiplication (the modular multiplication of Sec. III-C;
 * here Montgomery's method in place of Barrett's, as Sec. V-C proposes).
 * out_i = a_i * b_i mod p for i < n.
 * a, b, out: device, structure-of-arrays [12][n] u32 (limb k of element i at
 *   k * n + i), 4-byte aligned; out may alias a or b.
 * form: MSM377_FORM_STANDARD (inputs and result in standard form) or
 *   MSM377_FORM_MONTGOMERY (inputs and result in Montgomery form).
 * Results are fully reduced into [0, p). n = 0 is a no-op.
 */
int fq_mul_batch(const uint32_t *a, const uint32_t *b, uint32_t *out, size_t n, int form,
                 void *stream);

/* Standard <-> Montgomery conversion of n elements, SoA [12][n]; out may alias in. */
int fq_to_montgomery(const uint32_t *in, uint32_t *out, size_t n, void *stream);
/* Alternative multiplications, for comparison with fq_mul_batch's Montgomery CIOS
 * (same layout: structure-of-arrays [12][n], 16-byte aligned device arrays,
 * operands in [0, p), result canonical in [0, p)). The MSM does not use them.
 *   MSM377_FQMUL_CIOS      a b 2^-384 mod p, word-serial Montgomery two words per step
 *                          with the quotient digits formed out of the compiler's
 *                          sight (the library's)
 *   MSM377_FQMUL_BARRETT   a b mod p on standard-form operands: the paper's Barrett
 *                          reduction (Sec. III-C), k = 377, mu = floor(2^754 / p),
 *                          remainder in [0, 3p) then at most two subtractions of p
 *   MSM377_FQMUL_KARATSUBA a b 2^-384 mod p, a b by one Karatsuba level over 192-bit
 *                          halves with schoolbook leaves (Sec. V-C), then
 *                          word-by-word Montgomery reduction
 *   MSM377_FQMUL_CARRYSAVE a b 2^-384 mod p on 16 digits of 24 bits with 64-bit
 *                          column sums and deferred carries (Sec. III-B, III-D)
 *   MSM377_FQMUL_CIOS_TWOPASS a b 2^-384 mod p, the same CIOS product with each
 *                          row as a chain of low halves followed by a chain of
 *                          high halves (the library's multiplication runs each
 *                          row as two independent chains of adjacent low/high
 *                          halves of the even- and odd-indexed limbs' products)
 *   MSM377_FQMUL_CIOS_DOUBLEROW a b 2^-384 mod p, the library's double-row steps with
 *                          the digits written as plain negations (which the compiler
 *                          folds into the digit products)
 *   MSM377_FQMUL_CIOS_SINGLEROW a b 2^-384 mod p, one row and one digit per step, the
 *                          library's earlier form
 *   MSM377_FQMUL_WARP      a b 2^-384 mod p with one warp per product: lane j holds
 *                          limb j, three column products (a b, the Montgomery
 *                          quotient, its multiple of p) with warp-wide carry
 *                          resolution; the low-latency form the MSM's window chains
 *                          use. Operands may be any values below 8p here.
 *   MSM377_FQMUL_PAPER     the paper's own format and reduction (Sec. III-B .. III-E)
 *                          on standard-form operands below 6p (the unreduced operands
 *                          of its final multiplications): 16 elements of 25 bits,
 *                          schoolbook column sums, the two-round coarse carry
 *                          (Sec. III-D), and the looser Barrett step with k = 378
 *                          (q1 = x >> 377, mu = floor(2^756 / p), q3 = q1 mu >> 379,
 *                          r = (x - q3 p) mod 2^379). The result is that remainder,
 *                          r = a b (mod p) with 0 <= r < 4p, not reduced further.
 *   MSM377_FQMUL_FIPS      a b 2^-384 mod p by product scanning with the Montgomery
 *                          reduction folded in: column k of a b + m p summed into one
 *                          three-word accumulator, quotient digit m_k = -t0 when
 *                          column k < 12 completes, columns 12..23 the result.
 * MSM377_EINVAL for another variant. */
#define MSM377_FQMUL_CIOS 0
#define MSM377_FQMUL_BARRETT 1
#define MSM377_FQMUL_KARATSUBA 2
#define MSM377_FQMUL_CARRYSAVE 3
#define MSM377_FQMUL_CIOS_TWOPASS 4
#define MSM377_FQMUL_CIOS_DOUBLEROW 5
#define MSM377_FQMUL_WARP 6
#define MSM377_FQMUL_PAPER 7
#define MSM377_FQMUL_FIPS 8
#define MSM377_FQMUL_CIOS_SINGLEROW 9
int fq_mul_batch_variant(const uint32_t *a, const uint32_t *b, uint32_t *out, size_t n, int variant,
                         void *stream);

int fq_from_montgomery(const uint32_t *in, uint32_t *out, size_t n, void *stream);

/* ------------------------------------------------------------------------
 * Batched mixed point addition (the bucket-accumulation PADD, Sec. II-D and
 * the throughput experiment of Sec. V-A): out_i = acc_i + q_i.
 * acc, out: device, XYZZ in SoA [4][12][n] (coordinate c, limb k, element i at
 *   (c * 12 + k) * n + i). q: device, affine SoA [2][12][n], (0, 0) = O.
 * Every case is handled: acc = O, q = O, q = acc (doubling), q = -acc (O).
 * form: coordinates of acc, q and out in STANDARD or MONTGOMERY form. The output
 *   is one valid XYZZ representative of the sum (compare after normalising to
 *   affine: x = X / ZZ, y = Y / ZZZ), fully reduced limbs.
 * out may alias acc. n = 0 is a no-op.
 */
int padd_batch(const uint32_t *acc, const uint32_t *q, uint32_t *out, size_t n, int form,
               void *stream);

/* Affine normalisation of n XYZZ points (SoA [4][12][n]) into affine SoA [2][12][n],
 * same form in and out; O maps to (0, 0). */
int xyzz_to_affine_batch(const uint32_t *xyzz, uint32_t *aff, size_t n, int form, void *stream);

/* ------------------------------------------------------------------------
 * Fixed-base scalar multiplication by the standard G1 generator G:
 * out_i = seeds_i * G as affine points, array-of-structures (24 u32 per point,
 * standard form). seeds: device, 8 u32 per scalar. Used to build synthetic
 * point sets P_i = s_i * G on the device.
 */
int g1_generator_mul(const uint32_t *seeds, size_t n, uint32_t *out, void *stream);

/* ------------------------------------------------------------------------
 * Multi-scalar multiplication (Sec. II-C): out = sum_{i < n} scalars_i * points_i.
 */

/* opts.flags */
#define MSM377_POINTS_PREPARED 1u /* points are in the stored form of msm_points_prepare_ex
                                     for the same EDWARDS / GLV flags */
#define MSM377_PROFILE 2u         /* record CUDA events between stages (see msm377_profile_last) */
/* Curve model of the pipeline: the paper's twisted Edwards curve
 * -x^2 + y^2 = 1 + (k/2) x^2 y^2 in extended coordinates (Sec. II-D): input points
 * stored as (x, y, u = k x y) with Z = 1 (144 bytes each), buckets as (X, Y, Z, T);
 * 7 multiplications per mixed addition instead of XYZZ's 10, no special cases.
 * PRECONDITION: every point lies in the order-r subgroup of G1 (all points a
 * BLS12-377 prover commits to do). For other points on y^2 = x^3 + 1 the result
 * is unspecified (no fault: such points may become the identity). */
#define MSM377_EDWARDS 4u
/* GLV split (not in the paper): phi(x, y) = (beta x, y) acts on the order-r
 * subgroup as multiplication by lambda = x0^2 - 1, lambda^2 + lambda + 1 = r. Each
 * scalar is reduced mod r and split as k1 + lambda k2 with halves below 2^127;
 * the MSM runs over the 2n points P_i, phi(P_i) with half the windows.
 * PRECONDITION: every point lies in the order-r subgroup (same as MSM377_EDWARDS);
 * scalars may be any 256-bit values (reduced mod r). */
#define MSM377_GLV 8u
/* Fixed-base precomputation for resident sets (with MSM377_EDWARDS and
 * MSM377_POINTS_PREPARED, GLV optional): points is msm_points_precompute output,
 * the stored forms of 2^(c j) P_i for every digit window j, made for this same c
 * (explicit, nonzero), scalar_bits, signed_digits and GLV choice. All windows then
 * add into one bucket set: the bucket reduction shrinks by the window count and the
 * window chain has no doublings; the mixed additions are the same in number. */
#define MSM377_PRECOMPUTED 16u
/* Sort the (bucket, point) pairs by 8-bit LSD radix passes instead of the default
 * counting sort over (window, bucket) bins (counts and each item's rank per tile of
 * items in shared-memory counters, a scan of the bin totals, one scatter). Same
 * result; kept for comparison (the counting sort measured faster for every plan on
 * GB300). */
#define MSM377_RADIX_SORT 32u
/* Check the input points before using them (Sec. I / II-C: the problem is a sum over
 * points of the BLS12-377 G1 group): every coordinate below p, every point on
 * y^2 = x^3 + 1 ((0, 0) is O), and with MSM377_EDWARDS or MSM377_GLV (whose maps are
 * exact on the order-r subgroup only) also r P = O, by double-and-add per point (about
 * 3,200 field multiplications per point: opt-in, for data of unknown origin).
 * msm_g1 (standard-form points only; with MSM377_POINTS_PREPARED the call fails with
 * MSM377_EINVAL) and msm_g1_host report MSM377_ENOTONCURVE through the device status;
 * msm_points_create returns it. Not accepted by msm_g1_batched and msm_g1_noalloc. */
#define MSM377_VALIDATE 64u

typedef struct msm_opts {
    int32_t c;             /* window width in bits, 2..20; 0 = chosen from n */
    int32_t signed_digits; /* 1: digits in (-2^(c-1), 2^(c-1)], buckets 1..2^(c-1);
                              0: unsigned digits in [0, 2^c), buckets 1..2^c-1 */
    int32_t scalar_bits;   /* caller's bound: every scalar < 2^scalar_bits (1..256);
                              0 = 256. A larger scalar makes the call fail with
                              MSM377_ERANGE (reported through the workspace status). */
    uint32_t flags;        /* MSM377_POINTS_PREPARED | MSM377_PROFILE | MSM377_EDWARDS | MSM377_GLV |
                              MSM377_PRECOMPUTED | MSM377_RADIX_SORT | MSM377_VALIDATE */
    void *stream;          /* cudaStream_t */
} msm_opts;

/* Workspace bytes msm_g1 needs for n points with these options (0 on bad options). */
size_t msm_g1_workspace_bytes(size_t n, const msm_opts *opts);

/* Window width msm_g1 uses for n points when opts.c == 0 (flags: the options'
 * MSM377_EDWARDS / MSM377_GLV bits). */
int msm_g1_default_c(size_t n, int signed_digits, uint32_t flags);

/* Installs measured window widths for signed digits: c_by_log2n[k] is used for
 * n in [2^k, 2^(k+1)) when opts.c == 0 (0 keeps the built-in rule). One table per
 * combination of MSM377_EDWARDS, MSM377_GLV and MSM377_PRECOMPUTED, chosen by flags
 * (other bits: MSM377_EINVAL; with PRECOMPUTED the table only advises which c to
 * precompute for, since those calls need an explicit c). len <= 32; len = 0 clears that table. Process-wide; written by
 * the autotuner. */
int msm_g1_set_window_table(const int32_t *c_by_log2n, int len, uint32_t flags);

/* Installs one measured schedule entry for signed digits and n in [2^log2n, 2^(log2n+1))
 * in the table of the mode named by flags (MSM377_EDWARDS / MSM377_GLV /
 * MSM377_PRECOMPUTED): c (window width, used when opts.c == 0), chunk (items per
 * accumulation thread, 2..256), sort (1 counting sort, 2 LSD radix sort),
 * reduce_log2 (log2 of the level-1 bucket-reduction threads, 8..20) and groups
 * (window groups, 1..8: the accumulation runs group by group and each group's
 * merges and bucket reduction run on a high-priority helper stream of the caller's
 * stream, overlapping the next group's accumulation); 0 in a field keeps the
 * built-in rule. Process-wide, like the window tables (written by the autotuner);
 * workspace sizes depend on it, so install before sizing workspaces. */
int msm_g1_set_schedule(uint32_t flags, int log2n, int c, int chunk, int sort, int reduce_log2, int groups);

/* The schedule msm_g1 would use for n points with these options: out5 = {c, chunk,
 * sort (1 counting, 2 radix), log2 of the level-1 reduction threads, window groups}. */
int msm_g1_schedule(size_t n, const msm_opts *opts, int32_t *out5);

/* Bytes of the stored form of n points for flags (a combination of MSM377_EDWARDS
 * and MSM377_GLV; 0 for other bits): XYZZ 96 per stored point, Edwards 144;
 * n stored points, or 2n with GLV, interleaved: P_0, phi(P_0), P_1, phi(P_1), ...
 * so the stored rows of input points [a, b) are rows [2a, 2b): a resident set can
 * be sliced without copying. */
size_t msm_points_prepared_bytes(size_t n, uint32_t flags);

/* Converts n affine points in standard form (array-of-structures, 24 u32 per point,
 * 16-byte aligned; (0, 0) = O) into the stored form that msm_g1 reads with
 * MSM377_POINTS_PREPARED and the same EDWARDS / GLV flags: out (16-byte aligned)
 * holds msm_points_prepared_bytes(n, flags). XYZZ: Montgomery affine (x, y).
 * Edwards: (x, y, k x y) in Montgomery form, one field inversion per warp batch of
 * points (Montgomery's trick); the kernel uses out's rows as scratch between its
 * two passes. out must not overlap points_std unless flags == 0. */
int msm_points_prepare_ex(const uint32_t *points_std, size_t n, uint32_t *out, uint32_t flags,
                          void *stream);

/* msm_points_prepare_ex with flags = 0 (XYZZ, no GLV; 96 bytes per point). out
 * may alias in. */
int msm_points_prepare(const uint32_t *points_std, size_t n, uint32_t *out, void *stream);

/* Bytes of the precomputed set for n points and these options (flags must hold
 * MSM377_EDWARDS | MSM377_PRECOMPUTED, GLV optional; c explicit): Wd * n' stored
 * points of 144 bytes, Wd = the digit windows of scalar_bits at width c, n' = n or
 * 2n with GLV. 0 on other options. */
size_t msm_points_precomputed_bytes(size_t n, const msm_opts *opts);

/* Fills out (device, 16-byte aligned, msm_points_precomputed_bytes; it must not
 * overlap points_std) from n affine standard-form points: row i Wd + j is the
 * Edwards stored form of 2^(c j) P'_i, P' the (GLV-interleaved) stored points, so
 * the rows of input points [a, b) are rows [a Wd', b Wd') (Wd' = Wd, or 2 Wd with
 * GLV) and a resident set slices without copies. Asynchronous on opts->stream;
 * one-time work per resident set (c doublings per point and window, one inversion
 * per 256 points and window). Subgroup points only, as MSM377_EDWARDS. */
int msm_points_precompute(const uint32_t *points_std, size_t n, uint32_t *out, const msm_opts *opts);

/* With more than one window group (a schedule option, msm_g1_set_schedule; one by
 * default), the first msm_g1 call on a stream creates a helper stream of the highest
 * priority and a few events for that stream (kept until the process exits; up to 32
 * caller streams, beyond that the groups run in order on the caller's stream): make
 * that first call outside stream capture.
 * points: device, 24 u32 per point in standard form, or with MSM377_POINTS_PREPARED
 *   the stored form of msm_points_prepare_ex for the same flags; 16-byte aligned. scalars: device, 8 u32 per scalar, 16-byte aligned.
 * out: device, 24 u32: the affine sum in standard form, (0, 0) for O.
 * workspace: device, >= msm_g1_workspace_bytes(n, opts), 256-byte aligned; the
 *   first 4 bytes hold the call's device status (0 or a negative code), readable
 *   with msm_g1_status once the stream has reached the end of the call.
 * Asynchronous on opts->stream. n = 0 writes O.
 */
int msm_g1(const uint32_t *points, const uint32_t *scalars, size_t n, uint32_t *out,
           void *workspace, size_t workspace_bytes, const msm_opts *opts);

/* ------------------------------------------------------------------------
 * Point validation and resident point sets. A prover commits to the same point
 * set (the "bases" of the sum of Sec. I / II-C) over and over with fresh scalars;
 * a resident set holds their stored form in library-owned device memory.
 */

/* Checks n affine standard-form points (device, 24 u32 each, 16-byte aligned) as
 * MSM377_VALIDATE describes; flags: MSM377_EDWARDS / MSM377_GLV / MSM377_PRECOMPUTED
 * ask for the subgroup check as well (MSM377_VALIDATE itself is allowed and ignored).
 * Synchronous on stream. Returns MSM377_OK or MSM377_ENOTONCURVE. */
int msm_points_validate(const uint32_t *points_std, size_t n, uint32_t flags, void *stream);

/* Opaque handle of a resident set. */
typedef struct msm_points_set *msm_points_t;

/* Makes a resident set from n >= 1 affine standard-form points (device, 24 u32 per
 * point, 16-byte aligned; read during the call only). opts->flags: the curve model
 * (MSM377_EDWARDS, MSM377_GLV; MSM377_PRECOMPUTED with MSM377_EDWARDS and an explicit
 * opts->c makes a fixed-base set for that c, opts->scalar_bits and digit kind) and
 * optionally MSM377_VALIDATE (then the points are checked first, synchronously, and
 * a failing set returns MSM377_ENOTONCURVE and no handle). The set owns device
 * memory (cudaMalloc) for the stored rows until msm_points_destroy; the stored
 * form is filled asynchronously on opts->stream. *handle is NULL on failure. */
int msm_points_create(const uint32_t *points_std, size_t n, const msm_opts *opts, msm_points_t *handle);

/* Frees the set's device memory (cudaFree: waits for the device). NULL is a no-op. */
int msm_points_destroy(msm_points_t handle);

/* Number of input points the set holds (0 for NULL). */
size_t msm_points_count(msm_points_t handle);

/* Device pointer to the stored rows of input point `offset` (offset <= count), for
 * msm_job.points of a batched call with MSM377_POINTS_PREPARED and the set's own
 * model flags; NULL for a bad handle or offset. Valid until msm_points_destroy. */
const uint32_t *msm_points_data(msm_points_t handle, size_t offset);

/* Workspace bytes of msm_g1_resident for n points of the set (0 on bad options). */
size_t msm_g1_resident_workspace_bytes(msm_points_t handle, size_t n, const msm_opts *opts);

/* msm_g1 over the set's input points [offset, offset + n) (Sec. II-C):
 * out = sum_{i < n} scalars_i * P_{offset + i}. The set supplies the curve model
 * (opts->flags may repeat it or leave it out; another model is MSM377_EINVAL); a
 * fixed-base set also fixes c, scalar_bits and the digit kind (opts->c and
 * opts->scalar_bits 0 or equal). Allowed extra flags: MSM377_PROFILE,
 * MSM377_RADIX_SORT. scalars, out, workspace and the status word as for msm_g1.
 * Asynchronous on opts->stream. */
int msm_g1_resident(msm_points_t handle, size_t offset, size_t n, const uint32_t *scalars, uint32_t *out,
                    void *workspace, size_t workspace_bytes, const msm_opts *opts);

/* End-to-end variant over a resident set (synchronous): copies scalars_host (8 u32
 * per scalar, pageable or pinned) into the workspace, runs msm_g1_resident over
 * points [offset, offset + n) and copies the 24-u32 affine result into out_host.
 * This is a prover's step: the points (the committed bases) stay on the device,
 * each step brings fresh scalars. workspace (device, 256-byte aligned) must hold
 * msm_g1_resident_host_workspace_bytes(handle, n, opts). Returns the device status. */
size_t msm_g1_resident_host_workspace_bytes(msm_points_t handle, size_t n, const msm_opts *opts);
int msm_g1_resident_host(msm_points_t handle, size_t offset, size_t n, const uint32_t *scalars_host,
                         uint32_t *out_host, void *workspace, size_t workspace_bytes, const msm_opts *opts);

/* ------------------------------------------------------------------------
 * Batched MSM: many independent MSMs of uneven size in one call. The per-job
 * preparation, digits and sort run on library-owned helper streams; the bucket
 * accumulation of all jobs is one persistent kernel that drains a queue of
 * (job, window, chunk) items; the jobs' reductions and window combinations run
 * on the helper streams again, so the serial tails overlap each other. Every
 * step forks from and joins back into opts->stream through events, so the call
 * can be captured into a CUDA graph once the first call on the device has
 * created the helper streams (make one uncaptured call first).
 */
typedef struct msm_job {
    const uint32_t *points;  /* device, 24 u32 per point (standard, or prepared with the flag) */
    const uint32_t *scalars; /* device, 8 u32 per scalar */
    size_t n;
    uint32_t *out;           /* device, 24 u32: affine result in standard form */
    int32_t c;               /* window bits for this job, 0 = opts->c or the size default */
    int32_t reserved;
} msm_job;

/* Workspace for a batch (0 on bad options or more than 128 jobs). */
size_t msm_g1_batched_workspace_bytes(const msm_job *jobs, size_t njobs, const msm_opts *opts);

/* Runs njobs <= 128 MSMs; opts applies to all jobs (except c, see msm_job).
 * Asynchronous on opts->stream. The per-job device status words are not
 * reported; leave scalar_bits at 0 (256) to rule the range error out. */
int msm_g1_batched(const msm_job *jobs, size_t njobs, void *workspace, size_t workspace_bytes,
                   const msm_opts *opts);

/* Synchronous: waits for opts->stream and returns the device status word of the
 * last msm_g1 / msm_g1_batched that used this workspace. */
int msm_g1_status(const void *workspace, const msm_opts *opts);

/* End-to-end variant on host buffers (synchronous): copies points_host (24 u32
 * per point, standard form) and scalars_host (8 u32 per scalar) into the
 * workspace, runs the MSM and copies the 24-u32 result into out_host. The points
 * travel in 2 chunks on a library helper stream and each chunk is prepared (the
 * options' curve model / GLV form) on a second helper stream as soon as it has
 * arrived, while the scalars' copy, digits and bucket sort run on opts->stream;
 * the accumulation starts when the last chunk is prepared. Host buffers may be
 * pageable; pinned buffers copy faster and overlap. workspace (device, 256-byte
 * aligned) must hold msm_g1_host_workspace_bytes(n, opts) bytes;
 * MSM377_POINTS_PREPARED, MSM377_PRECOMPUTED and MSM377_PROFILE are not used here.
 * The helper streams are shared per device: calls from several host threads on
 * one device must not overlap (the same holds for msm_g1_batched).
 * Returns the device status. */
size_t msm_g1_host_workspace_bytes(size_t n, const msm_opts *opts);
int msm_g1_host(const uint32_t *points_host, const uint32_t *scalars_host, size_t n,
                uint32_t *out_host, void *workspace, size_t workspace_bytes,
                const msm_opts *opts);

/* msm_g1 for callers that cannot allocate device memory. No counterpart in the
 * paper. Some callers of an MSM library cannot call cudaMalloc or accept a
 * caller-sized workspace: a plugin loaded into a host program whose device
 * memory is owned by that program's pooling allocator, a latency-critical
 * request path on which allocation calls (which can synchronise the device) are
 * forbidden, or a deployment whose device-memory budget is fixed when the
 * library is loaded. This entry point takes the same inputs, output and options
 * as msm_g1 but uses a fixed scratch array of MSM377_NOALLOC_SCRATCH_BYTES
 * (64 MiB) that the library holds on every GPU that loads it, until the process
 * exits; it calls no cudaMalloc, cudaFree or other allocating routine.
 * - Size limit: n and the options must need at most MSM377_NOALLOC_SCRATCH_BYTES
 *   of workspace (msm_g1_workspace_bytes); with the default options that holds
 *   up to n = 2^15. Larger requests fail with MSM377_EINVAL and a message.
 * - The first call on each device (and in each CUDA context: a driver-API
 *   context, or the primary context again after cudaDeviceReset) looks up the
 *   scratch address (a one-time set-up there); make that first call before any
 *   stream capture.
 * - Every call on a device shares the one scratch array and it keeps the last
 *   call's contents (each call clears what must start at zero). Calls whose
 *   work overlaps on the GPU (different streams, or different host threads)
 *   race on it and give wrong results: serialise them.
 * - The device status word (MSM377_ERANGE for scalars at or above
 *   opts->scalar_bits) is not reported here; leave scalar_bits at 0 (256) to
 *   rule that error out. MSM377_PROFILE and MSM377_VALIDATE are rejected.
 * Asynchronous on opts->stream, like msm_g1. */
#define MSM377_NOALLOC_SCRATCH_BYTES (64u << 20)
int msm_g1_noalloc(const uint32_t *points, const uint32_t *scalars, size_t n, uint32_t *out,
                   const msm_opts *opts);

/* ------------------------------------------------------------------------
 * Dependent-chain latency (Sec. V-A, the sequential sum of a point stream):
 * out = P_0 + P_1 + ... + P_{n-1} added strictly in order, each mixed PADD waiting
 * for the previous one, so time / n is the latency of one PADD.
 * points: device, the stored form of msm_points_prepare_ex(points, n, ., flags)
 *   with flags = 0 (XYZZ model, Montgomery affine) or MSM377_EDWARDS (no GLV).
 * lanes: 1 (one thread performs every multiplication), 4 (Edwards only: the
 *   independent multiplications of each addition run on four lanes of a warp, the
 *   analogue of the paper's multi-tile med-ind mapping) or 128 (Edwards only: four
 *   warps, one product of each level per warp, every product spread over the 32
 *   lanes of its warp).
 * out: device, 24 u32, affine standard form, (0, 0) for O. Asynchronous on stream.
 * MSM377_EINVAL for other flags or lanes. The Edwards model needs subgroup points. */
int padd_chain(const uint32_t *points, size_t n, uint32_t *out, uint32_t flags, int lanes, void *stream);

/* Stage timings of the most recent msm_g1 call made with MSM377_PROFILE, in
 * milliseconds, from CUDA events recorded on the caller's stream:
 * [0] head: preparation, digits, sort, bucket reset; [1] bucket accumulation;
 * [2] tail: partial merges, bucket reduction, window combination and
 * normalisation. Synchronous (waits for the last event). Writes min(cap, 3) values and returns
 * the number of stages, or a negative status. Not thread-safe: one profiled
 * call at a time per process. */
int msm377_profile_last(float *ms, int cap);

/* Number of kernels this library has launched in the process so far (host-side
 * counter, all entry points). */
uint64_t msm377_launch_count(void);

/* ------------------------------------------------------------------------
 * Micro-benchmark for the roofline denominator: runs `iters` rounds of
 * Montgomery-row-shaped carry chains (mad.lo.cc / madc.hi.cc of one product
 * adjacent, even- and odd-indexed limbs in two chains, two independent rows; every
 * operand different in every thread) on every SM and writes the measured count of
 * 32x32->64 limb products per second into *products_per_s. Synchronous.
 */
int msm377_imad_probe(int iters, double *products_per_s, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MSM377_H */
