/*
 * Plain C big-integer oracle for BLS12-377 G1 MSM — TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark load this library. It shares no code, header or constant with the
 * CUDA library: the modulus, the Barrett constant and the generator are handed
 * in at run time by the Python oracle, which derives them from the BLS12 seed.
 *
 * Field: GF(p) with 6 x 64-bit words; a*b by the schoolbook product and reduction
 * by Barrett's method (the modular multiplication of Sec. III-C of the paper:
 * product, high part times mu, high part times M, subtract, then at most two
 * corrections out of [0, 3M)). Inverse by Fermat, a^(p-2).
 * Group: Jacobian coordinates (x = X/Z^2, y = Y/Z^3) on y^2 = x^3 + 1; the mixed
 * addition adds an affine point (Sec. II-D: mixed PADD in bucket accumulation,
 * complete PADD in aggregation).
 * MSM: textbook Pippenger with unsigned c-bit windows (Sec. II-C), windows spread
 * over POSIX threads; point generation P_i = s_i*G with a fixed-base comb.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef unsigned __int128 u128;
#define NW 6

static uint64_t MOD[NW];
static uint64_t MU[NW + 1];   /* floor(2^754 / p): 378 bits */
static uint64_t ONE[NW] = {1, 0, 0, 0, 0, 0};
static uint64_t GEN_X[NW], GEN_Y[NW];
static int g_inited = 0;
static const int KBITS = 377; /* bit length of p */

/* ------------------------------------------------------------------ bigint */

static void mul_n(const uint64_t *a, int na, const uint64_t *b, int nb, uint64_t *out) {
    memset(out, 0, sizeof(uint64_t) * (size_t)(na + nb));
    for (int i = 0; i < na; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < nb; j++) {
            u128 t = (u128)a[i] * b[j] + out[i + j] + carry;
            out[i + j] = (uint64_t)t;
            carry = (uint64_t)(t >> 64);
        }
        out[i + nb] = carry;
    }
}

/* out = in >> shift (bits), keeping nout words */
static void shr_bits(const uint64_t *in, int nin, int shift, uint64_t *out, int nout) {
    int ws = shift / 64, bs = shift % 64;
    for (int k = 0; k < nout; k++) {
        int s = k + ws;
        uint64_t lo = s < nin ? in[s] : 0;
        uint64_t hi = s + 1 < nin ? in[s + 1] : 0;
        out[k] = bs ? (lo >> bs) | (hi << (64 - bs)) : lo;
    }
}

/* a -= b over n words; returns borrow */
static uint64_t sub_n(uint64_t *a, const uint64_t *b, int n) {
    uint64_t borrow = 0;
    for (int k = 0; k < n; k++) {
        u128 t = (u128)a[k] - b[k] - borrow;
        a[k] = (uint64_t)t;
        borrow = (uint64_t)(t >> 64) & 1;
    }
    return borrow;
}

static uint64_t add_n(uint64_t *a, const uint64_t *b, int n) {
    uint64_t carry = 0;
    for (int k = 0; k < n; k++) {
        u128 t = (u128)a[k] + b[k] + carry;
        a[k] = (uint64_t)t;
        carry = (uint64_t)(t >> 64);
    }
    return carry;
}

/* compare a (na words) with b (nb words): -1, 0, 1 */
static int cmp_n(const uint64_t *a, int na, const uint64_t *b, int nb) {
    int n = na > nb ? na : nb;
    for (int k = n - 1; k >= 0; k--) {
        uint64_t x = k < na ? a[k] : 0, y = k < nb ? b[k] : 0;
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}

static int is_zero(const uint64_t *a) {
    uint64_t o = 0;
    for (int k = 0; k < NW; k++) o |= a[k];
    return o == 0;
}

/* ------------------------------------------------------------------ field */

static void fq_add(const uint64_t *a, const uint64_t *b, uint64_t *r) {
    uint64_t t[NW + 1];
    memcpy(t, a, sizeof(uint64_t) * NW);
    t[NW] = add_n(t, b, NW);
    if (cmp_n(t, NW + 1, MOD, NW) >= 0) {
        uint64_t m[NW + 1];
        memcpy(m, MOD, sizeof(uint64_t) * NW);
        m[NW] = 0;
        sub_n(t, m, NW + 1);
    }
    memcpy(r, t, sizeof(uint64_t) * NW);
}

static void fq_sub(const uint64_t *a, const uint64_t *b, uint64_t *r) {
    uint64_t t[NW];
    memcpy(t, a, sizeof(t));
    if (sub_n(t, b, NW)) add_n(t, MOD, NW);
    memcpy(r, t, sizeof(t));
}

/* Barrett reduction of x < p^2 (12 words) into [0, p). */
static void fq_reduce(const uint64_t *x, uint64_t *r) {
    uint64_t q1[NW + 1], q2[2 * NW + 2], q3[NW + 1], qm[2 * NW + 2], t[2 * NW + 2];
    shr_bits(x, 2 * NW, KBITS - 1, q1, NW + 1);      /* high part of the product */
    mul_n(q1, NW + 1, MU, NW + 1, q2);               /* times mu */
    shr_bits(q2, 2 * NW + 2, KBITS + 1, q3, NW + 1); /* high part of that */
    mul_n(q3, NW + 1, MOD, NW, qm);                  /* times the modulus */
    memset(t, 0, sizeof(t));
    memcpy(t, x, sizeof(uint64_t) * 2 * NW);
    sub_n(t, qm, 2 * NW + 1);                        /* now in [0, 3p) */
    while (cmp_n(t, 2 * NW + 1, MOD, NW) >= 0) {
        uint64_t m[2 * NW + 1];
        memset(m, 0, sizeof(m));
        memcpy(m, MOD, sizeof(uint64_t) * NW);
        sub_n(t, m, 2 * NW + 1);
    }
    memcpy(r, t, sizeof(uint64_t) * NW);
}

static void fq_mul(const uint64_t *a, const uint64_t *b, uint64_t *r) {
    uint64_t x[2 * NW];
    mul_n(a, NW, b, NW, x);
    fq_reduce(x, r);
}

static void fq_inv(const uint64_t *a, uint64_t *r) {
    /* a^(p-2), left to right */
    uint64_t e[NW], two[NW] = {2, 0, 0, 0, 0, 0}, acc[NW];
    memcpy(e, MOD, sizeof(e));
    sub_n(e, two, NW);
    memcpy(acc, ONE, sizeof(acc));
    for (int bit = 64 * NW - 1; bit >= 0; bit--) {
        fq_mul(acc, acc, acc);
        if ((e[bit / 64] >> (bit % 64)) & 1) fq_mul(acc, a, acc);
    }
    memcpy(r, acc, sizeof(acc));
}

/* ------------------------------------------------------------------ group */

typedef struct { uint64_t x[NW], y[NW]; int inf; } aff_t;
typedef struct { uint64_t X[NW], Y[NW], Z[NW]; } jac_t;   /* Z = 0 is the identity */

static void jac_set_inf(jac_t *p) {
    memset(p, 0, sizeof(*p));
    p->X[0] = 1;
    p->Y[0] = 1;
}

static void jac_from_aff(const aff_t *a, jac_t *p) {
    if (a->inf) { jac_set_inf(p); return; }
    memcpy(p->X, a->x, sizeof(p->X));
    memcpy(p->Y, a->y, sizeof(p->Y));
    memcpy(p->Z, ONE, sizeof(p->Z));
}

static void jac_dbl(const jac_t *p, jac_t *r) {
    if (is_zero(p->Z) || is_zero(p->Y)) { jac_set_inf(r); return; }
    uint64_t A[NW], B[NW], C[NW], D[NW], E[NW], F[NW], t[NW], X3[NW], Y3[NW], Z3[NW];
    fq_mul(p->X, p->X, A);
    fq_mul(p->Y, p->Y, B);
    fq_mul(B, B, C);
    fq_add(p->X, B, t);
    fq_mul(t, t, D);
    fq_sub(D, A, D);
    fq_sub(D, C, D);
    fq_add(D, D, D);                 /* D = 4 X Y^2 */
    fq_add(A, A, E);
    fq_add(E, A, E);                 /* E = 3 X^2 */
    fq_mul(E, E, F);
    fq_sub(F, D, X3);
    fq_sub(X3, D, X3);               /* X3 = F - 2D */
    fq_sub(D, X3, t);
    fq_mul(E, t, Y3);
    fq_add(C, C, t);
    fq_add(t, t, t);
    fq_add(t, t, t);                 /* 8C */
    fq_sub(Y3, t, Y3);
    fq_mul(p->Y, p->Z, Z3);
    fq_add(Z3, Z3, Z3);
    memcpy(r->X, X3, sizeof(X3));
    memcpy(r->Y, Y3, sizeof(Y3));
    memcpy(r->Z, Z3, sizeof(Z3));
}

/* r = p + q, q affine */
static void jac_add_aff(const jac_t *p, const aff_t *q, jac_t *r) {
    if (q->inf) { *r = *p; return; }
    if (is_zero(p->Z)) { jac_from_aff(q, r); return; }
    uint64_t Z1Z1[NW], U2[NW], S2[NW], H[NW], Rr[NW], HH[NW], HHH[NW], V[NW], t[NW];
    uint64_t X3[NW], Y3[NW], Z3[NW];
    fq_mul(p->Z, p->Z, Z1Z1);
    fq_mul(q->x, Z1Z1, U2);
    fq_mul(q->y, p->Z, S2);
    fq_mul(S2, Z1Z1, S2);
    fq_sub(U2, p->X, H);
    fq_sub(S2, p->Y, Rr);
    if (is_zero(H)) {
        if (is_zero(Rr)) { jac_dbl(p, r); return; }
        jac_set_inf(r);
        return;
    }
    fq_mul(H, H, HH);
    fq_mul(H, HH, HHH);
    fq_mul(p->X, HH, V);
    fq_mul(Rr, Rr, X3);
    fq_sub(X3, HHH, X3);
    fq_sub(X3, V, X3);
    fq_sub(X3, V, X3);
    fq_sub(V, X3, t);
    fq_mul(Rr, t, Y3);
    fq_mul(p->Y, HHH, t);
    fq_sub(Y3, t, Y3);
    fq_mul(p->Z, H, Z3);
    memcpy(r->X, X3, sizeof(X3));
    memcpy(r->Y, Y3, sizeof(Y3));
    memcpy(r->Z, Z3, sizeof(Z3));
}

static void jac_add(const jac_t *p, const jac_t *q, jac_t *r) {
    if (is_zero(p->Z)) { *r = *q; return; }
    if (is_zero(q->Z)) { *r = *p; return; }
    uint64_t Z1Z1[NW], Z2Z2[NW], U1[NW], U2[NW], S1[NW], S2[NW], H[NW], Rr[NW];
    uint64_t HH[NW], HHH[NW], V[NW], t[NW], X3[NW], Y3[NW], Z3[NW];
    fq_mul(p->Z, p->Z, Z1Z1);
    fq_mul(q->Z, q->Z, Z2Z2);
    fq_mul(p->X, Z2Z2, U1);
    fq_mul(q->X, Z1Z1, U2);
    fq_mul(p->Y, q->Z, S1);
    fq_mul(S1, Z2Z2, S1);
    fq_mul(q->Y, p->Z, S2);
    fq_mul(S2, Z1Z1, S2);
    fq_sub(U2, U1, H);
    fq_sub(S2, S1, Rr);
    if (is_zero(H)) {
        if (is_zero(Rr)) { jac_dbl(p, r); return; }
        jac_set_inf(r);
        return;
    }
    fq_mul(H, H, HH);
    fq_mul(H, HH, HHH);
    fq_mul(U1, HH, V);
    fq_mul(Rr, Rr, X3);
    fq_sub(X3, HHH, X3);
    fq_sub(X3, V, X3);
    fq_sub(X3, V, X3);
    fq_sub(V, X3, t);
    fq_mul(Rr, t, Y3);
    fq_mul(S1, HHH, t);
    fq_sub(Y3, t, Y3);
    fq_mul(p->Z, q->Z, Z3);
    fq_mul(Z3, H, Z3);
    memcpy(r->X, X3, sizeof(X3));
    memcpy(r->Y, Y3, sizeof(Y3));
    memcpy(r->Z, Z3, sizeof(Z3));
}

static void jac_to_aff(const jac_t *p, aff_t *a) {
    if (is_zero(p->Z)) { memset(a, 0, sizeof(*a)); a->inf = 1; return; }
    uint64_t zi[NW], zi2[NW], zi3[NW];
    fq_inv(p->Z, zi);
    fq_mul(zi, zi, zi2);
    fq_mul(zi2, zi, zi3);
    fq_mul(p->X, zi2, a->x);
    fq_mul(p->Y, zi3, a->y);
    a->inf = 0;
}

/* Montgomery's simultaneous inversion over a run of Jacobian points. */
static void jac_to_aff_batch(const jac_t *p, aff_t *a, size_t n) {
    uint64_t (*pre)[NW] = malloc(sizeof(uint64_t[NW]) * (n + 1));
    uint64_t acc[NW], inv[NW], t[NW], zi2[NW], zi3[NW];
    memcpy(acc, ONE, sizeof(acc));
    for (size_t i = 0; i < n; i++) {
        memcpy(pre[i], acc, sizeof(acc));
        if (!is_zero(p[i].Z)) fq_mul(acc, p[i].Z, acc);
    }
    fq_inv(acc, inv);
    for (size_t i = n; i-- > 0;) {
        if (is_zero(p[i].Z)) { memset(&a[i], 0, sizeof(aff_t)); a[i].inf = 1; continue; }
        fq_mul(inv, pre[i], t);          /* 1 / Z_i */
        fq_mul(inv, p[i].Z, inv);
        fq_mul(t, t, zi2);
        fq_mul(zi2, t, zi3);
        fq_mul(p[i].X, zi2, a[i].x);
        fq_mul(p[i].Y, zi3, a[i].y);
        a[i].inf = 0;
    }
    free(pre);
}

/* ------------------------------------------------------------------ format */

static void fq_from_u32(const uint32_t *w, uint64_t *v) {
    for (int k = 0; k < NW; k++) v[k] = (uint64_t)w[2 * k] | ((uint64_t)w[2 * k + 1] << 32);
}

static void fq_to_u32(const uint64_t *v, uint32_t *w) {
    for (int k = 0; k < NW; k++) {
        w[2 * k] = (uint32_t)v[k];
        w[2 * k + 1] = (uint32_t)(v[k] >> 32);
    }
}

static void aff_from_u32(const uint32_t *w, aff_t *a) {
    fq_from_u32(w, a->x);
    fq_from_u32(w + 12, a->y);
    a->inf = is_zero(a->x) && is_zero(a->y);
}

static void aff_to_u32(const aff_t *a, uint32_t *w) {
    if (a->inf) { memset(w, 0, 24 * sizeof(uint32_t)); return; }
    fq_to_u32(a->x, w);
    fq_to_u32(a->y, w + 12);
}

static int scalar_bit(const uint32_t *s, int bit) { return (s[bit / 32] >> (bit % 32)) & 1; }

static uint32_t scalar_window(const uint32_t *s, int lo, int c) {
    uint32_t v = 0;
    for (int b = 0; b < c && lo + b < 256; b++) v |= (uint32_t)scalar_bit(s, lo + b) << b;
    return v;
}

static int nthreads_or_default(int nt) {
    if (nt > 0) return nt;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* ------------------------------------------------------------------ API */

int orc_init(const uint64_t *p, const uint64_t *mu, const uint64_t *gx, const uint64_t *gy) {
    memcpy(MOD, p, sizeof(MOD));
    memcpy(MU, mu, sizeof(MU));
    memcpy(GEN_X, gx, sizeof(GEN_X));
    memcpy(GEN_Y, gy, sizeof(GEN_Y));
    g_inited = 1;
    return 0;
}

int orc_fq_mul(const uint64_t *a, const uint64_t *b, uint64_t *r) {
    if (!g_inited) return -1;
    fq_mul(a, b, r);
    return 0;
}

int orc_fq_inv(const uint64_t *a, uint64_t *r) {
    if (!g_inited || is_zero(a)) return -1;
    fq_inv(a, r);
    return 0;
}

/* out = k * P (k: 8 u32 little-endian), double-and-add; points as 24 u32 */
int orc_scalar_mul(const uint32_t *pt, const uint32_t *k, uint32_t *out) {
    if (!g_inited) return -1;
    aff_t a, res;
    jac_t acc;
    aff_from_u32(pt, &a);
    jac_set_inf(&acc);
    for (int bit = 255; bit >= 0; bit--) {
        jac_dbl(&acc, &acc);
        if (scalar_bit(k, bit)) jac_add_aff(&acc, &a, &acc);
    }
    jac_to_aff(&acc, &res);
    aff_to_u32(&res, out);
    return 0;
}

/* sum of two affine points (the chord/tangent result via Jacobian) */
int orc_padd(const uint32_t *p1, const uint32_t *p2, uint32_t *out) {
    if (!g_inited) return -1;
    aff_t a, b, res;
    jac_t j;
    aff_from_u32(p1, &a);
    aff_from_u32(p2, &b);
    jac_from_aff(&a, &j);
    jac_add_aff(&j, &b, &j);
    jac_to_aff(&j, &res);
    aff_to_u32(&res, out);
    return 0;
}

/* --- fixed-base comb for P_i = s_i * G: T[j][d] = d * 2^(8j) * G --- */

static aff_t *g_comb = NULL;   /* 32 x 256 */

static void build_comb(void) {
    if (g_comb) return;
    jac_t *tmp = malloc(sizeof(jac_t) * 32 * 256);
    aff_t base;
    memcpy(base.x, GEN_X, sizeof(base.x));
    memcpy(base.y, GEN_Y, sizeof(base.y));
    base.inf = 0;
    jac_t bj;
    jac_from_aff(&base, &bj);
    for (int j = 0; j < 32; j++) {
        jac_set_inf(&tmp[j * 256]);
        for (int d = 1; d < 256; d++) jac_add(&tmp[j * 256 + d - 1], &bj, &tmp[j * 256 + d]);
        for (int k = 0; k < 8; k++) jac_dbl(&bj, &bj);
    }
    aff_t *tab = malloc(sizeof(aff_t) * 32 * 256);
    jac_to_aff_batch(tmp, tab, 32 * 256);
    free(tmp);
    g_comb = tab;
}

typedef struct {
    const uint32_t *seeds;
    uint32_t *out;
    size_t lo, hi;
} gen_job_t;

static void *gen_worker(void *arg) {
    gen_job_t *job = (gen_job_t *)arg;
    const size_t CH = 1024;
    jac_t *acc = malloc(sizeof(jac_t) * CH);
    aff_t *aff = malloc(sizeof(aff_t) * CH);
    for (size_t base = job->lo; base < job->hi; base += CH) {
        size_t m = job->hi - base < CH ? job->hi - base : CH;
        for (size_t i = 0; i < m; i++) {
            const uint32_t *s = job->seeds + 8 * (base + i);
            jac_set_inf(&acc[i]);
            for (int j = 0; j < 32; j++) {
                uint32_t d = scalar_window(s, 8 * j, 8);
                if (d) jac_add_aff(&acc[i], &g_comb[j * 256 + d], &acc[i]);
            }
        }
        jac_to_aff_batch(acc, aff, m);
        for (size_t i = 0; i < m; i++) aff_to_u32(&aff[i], job->out + 24 * (base + i));
    }
    free(acc);
    free(aff);
    return NULL;
}

int orc_gen_points(const uint32_t *seeds, size_t n, uint32_t *out, int nthreads) {
    if (!g_inited) return -1;
    build_comb();
    int nt = nthreads_or_default(nthreads);
    if ((size_t)nt > n / 1024 + 1) nt = (int)(n / 1024 + 1);
    pthread_t th[256];
    gen_job_t jobs[256];
    if (nt > 256) nt = 256;
    for (int t = 0; t < nt; t++) {
        jobs[t].seeds = seeds;
        jobs[t].out = out;
        jobs[t].lo = n * (size_t)t / (size_t)nt;
        jobs[t].hi = n * (size_t)(t + 1) / (size_t)nt;
        pthread_create(&th[t], NULL, gen_worker, &jobs[t]);
    }
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
    return 0;
}

/* --- textbook Pippenger, unsigned c-bit windows, windows over threads --- */

typedef struct {
    const aff_t *pts;
    const uint32_t *sc;
    size_t n;
    int c, nwin, next;
    jac_t *wsum;
    pthread_mutex_t *mu;
} pip_job_t;

static void *pip_worker(void *arg) {
    pip_job_t *job = (pip_job_t *)arg;
    size_t nb = ((size_t)1 << job->c) - 1;
    jac_t *bk = malloc(sizeof(jac_t) * (nb + 1));
    for (;;) {
        pthread_mutex_lock(job->mu);
        int j = job->next++;
        pthread_mutex_unlock(job->mu);
        if (j >= job->nwin) break;
        for (size_t b = 0; b <= nb; b++) jac_set_inf(&bk[b]);
        for (size_t i = 0; i < job->n; i++) {
            uint32_t d = scalar_window(job->sc + 8 * i, job->c * j, job->c);
            if (d) jac_add_aff(&bk[d], &job->pts[i], &bk[d]);
        }
        jac_t run, tot;
        jac_set_inf(&run);
        jac_set_inf(&tot);
        for (size_t b = nb; b >= 1; b--) {
            jac_add(&run, &bk[b], &run);
            jac_add(&tot, &run, &tot);
        }
        job->wsum[j] = tot;
    }
    free(bk);
    return NULL;
}

int orc_msm(const uint32_t *points, const uint32_t *scalars, size_t n, int c, int nthreads,
            uint32_t *out) {
    if (!g_inited || c < 1 || c > 24) return -1;
    aff_t res;
    if (n == 0) {
        res.inf = 1;
        aff_to_u32(&res, out);
        return 0;
    }
    aff_t *pts = malloc(sizeof(aff_t) * n);
    for (size_t i = 0; i < n; i++) aff_from_u32(points + 24 * i, &pts[i]);
    int nwin = (256 + c - 1) / c;
    jac_t *wsum = malloc(sizeof(jac_t) * (size_t)nwin);
    pthread_mutex_t mu;
    pthread_mutex_init(&mu, NULL);
    pip_job_t job = {pts, scalars, n, c, nwin, 0, wsum, &mu};
    int nt = nthreads_or_default(nthreads);
    if (nt > nwin) nt = nwin;
    if (nt > 256) nt = 256;
    pthread_t th[256];
    for (int t = 0; t < nt; t++) pthread_create(&th[t], NULL, pip_worker, &job);
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&mu);
    jac_t acc;
    jac_set_inf(&acc);
    for (int j = nwin - 1; j >= 0; j--) {
        for (int k = 0; k < c; k++) jac_dbl(&acc, &acc);
        jac_add(&acc, &wsum[j], &acc);
    }
    jac_to_aff(&acc, &res);
    aff_to_u32(&res, out);
    free(wsum);
    free(pts);
    return 0;
}

/* --- sum_i s_i P_i by double-and-add per term (the definition) --- */
int orc_msm_naive(const uint32_t *points, const uint32_t *scalars, size_t n, uint32_t *out) {
    if (!g_inited) return -1;
    jac_t acc, term;
    aff_t a, res;
    jac_set_inf(&acc);
    for (size_t i = 0; i < n; i++) {
        aff_from_u32(points + 24 * i, &a);
        jac_set_inf(&term);
        for (int bit = 255; bit >= 0; bit--) {
            jac_dbl(&term, &term);
            if (scalar_bit(scalars + 8 * i, bit)) jac_add_aff(&term, &a, &term);
        }
        jac_add(&acc, &term, &acc);
    }
    jac_to_aff(&acc, &res);
    aff_to_u32(&res, out);
    return 0;
}

/* Affine sums acc_i + q_i for a stream of pairs (the mixed-PADD task rate). */
int orc_padd_stream(const uint32_t *acc, const uint32_t *q, size_t n, uint32_t *out) {
    if (!g_inited) return -1;
    for (size_t i = 0; i < n; i++) orc_padd(acc + 24 * i, q + 24 * i, out + 24 * i);
    return 0;
}
