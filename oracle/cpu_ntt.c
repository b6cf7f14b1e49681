/*
 * cpu_ntt.c -- independent CPU statement of the NTT (arxiv 2509.22684,
 * Section II-B: A_k = sum_j a_j w^(jk); radix-2 Cooley-Tukey of Fig. 3(b)).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py load this library.  It shares no code, header,
 * table or constant generator with the CUDA path: it uses 4 x 64-bit limbs
 * and unsigned __int128 where the GPU path uses 8 x 32-bit limbs, and it
 * derives every constant (R mod r, R^2 mod r, -r^-1 mod 2^64, the 2-adicity,
 * the roots of unity, n^-1) from the modulus and the generator at start-up.
 *
 * Representation: values are kept in Montgomery form X = x * 2^256 mod r,
 * which is also the boundary layout (8 little-endian u32 limbs == 4
 * little-endian u64 limbs, packed explicitly below).  A product in that
 * domain is mont(X, Y) = X * Y * 2^-256 mod r (CIOS, one pass per 64-bit word
 * of Y).  The transform is the textbook iterative radix-2 decimation-in-time
 * algorithm: bit-reversal permutation, then log2 n stages of n/2 butterflies
 * (x, y) -> (x + w y, x - w y); each stage is split across threads.
 *
 * Readings of the paper: the inverse applies n^-1 (round trip = identity);
 * the coset forward transform scales a_j by g^j first; the coset inverse
 * scales output j by g^-j after the inverse transform; Groth16 H is
 * iNTT x3, coset NTT x3, (A B - C) * (g^n - 1)^-1, coset iNTT (Fig. 2).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef unsigned __int128 u128;
typedef uint64_t u64;

typedef struct {
    u64 r[4];      /* modulus, little-endian words */
    u64 rp;        /* -r^-1 mod 2^64 */
    u64 one[4];    /* R mod r: Montgomery form of 1 */
    u64 r2[4];     /* R^2 mod r */
    u64 g;         /* multiplicative generator (plain) */
    int s;         /* 2-adicity of r - 1 */
    u64 wmax[4];   /* Montgomery form of g^((r-1)/2^s) */
} field_t;

#define NFIELDS 3
static field_t FIELDS[NFIELDS];
static int fields_ready = 0;
static pthread_mutex_t init_lock = PTHREAD_MUTEX_INITIALIZER;

/* ---------------- 256-bit helpers ---------------- */
static int geq(const u64 a[4], const u64 b[4]) {
    for (int i = 3; i >= 0; i--) {
        if (a[i] != b[i]) return a[i] > b[i];
    }
    return 1;
}

static u64 sub4(u64 out[4], const u64 a[4], const u64 b[4]) {
    u64 borrow = 0;
    for (int i = 0; i < 4; i++) {
        u128 d = (u128)a[i] - b[i] - borrow;
        out[i] = (u64)d;
        borrow = (u64)(d >> 64) ? 1 : 0;
    }
    return borrow;
}

static u64 add4(u64 out[4], const u64 a[4], const u64 b[4]) {
    u128 c = 0;
    for (int i = 0; i < 4; i++) {
        c = (u128)a[i] + b[i] + (u64)(c >> 64);
        out[i] = (u64)c;
    }
    return (u64)(c >> 64);
}

static void fadd(u64 out[4], const u64 a[4], const u64 b[4], const field_t *F) {
    u64 t[4];
    u64 carry = add4(t, a, b);
    if (carry || geq(t, F->r)) sub4(t, t, F->r);
    memcpy(out, t, sizeof t);
}

static void fsub(u64 out[4], const u64 a[4], const u64 b[4], const field_t *F) {
    u64 t[4];
    if (sub4(t, a, b)) add4(t, t, F->r);
    memcpy(out, t, sizeof t);
}

/* Montgomery product a * b * 2^-256 mod r (CIOS, 64-bit words). */
static void mont(u64 out[4], const u64 a[4], const u64 b[4], const field_t *F) {
    u64 t[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 4; i++) {
        u128 c = 0;
        for (int j = 0; j < 4; j++) {
            c = (u128)a[j] * b[i] + t[j] + (u64)(c >> 64);
            t[j] = (u64)c;
        }
        c = (u128)t[4] + (u64)(c >> 64);
        t[4] = (u64)c;
        t[5] = (u64)(c >> 64);
        u64 m = t[0] * F->rp;
        c = (u128)m * F->r[0] + t[0];
        for (int j = 1; j < 4; j++) {
            c = (u128)m * F->r[j] + t[j] + (u64)(c >> 64);
            t[j - 1] = (u64)c;
        }
        c = (u128)t[4] + (u64)(c >> 64);
        t[3] = (u64)c;
        t[4] = t[5] + (u64)(c >> 64);
    }
    u64 res[4] = {t[0], t[1], t[2], t[3]};
    if (t[4] || geq(res, F->r)) sub4(res, res, F->r);
    memcpy(out, res, sizeof res);
}

/* base^e for an exponent given as 4 words; base and result in Montgomery form */
static void fpow(u64 out[4], const u64 base[4], const u64 e[4], const field_t *F) {
    u64 acc[4], b[4];
    memcpy(acc, F->one, sizeof acc);
    memcpy(b, base, sizeof b);
    for (int i = 0; i < 256; i++) {
        if ((e[i / 64] >> (i % 64)) & 1) mont(acc, acc, b, F);
        mont(b, b, b, F);
    }
    memcpy(out, acc, sizeof acc);
}

static void fpow_u64(u64 out[4], const u64 base[4], u64 e, const field_t *F) {
    u64 ee[4] = {e, 0, 0, 0};
    fpow(out, base, ee, F);
}

static void finv(u64 out[4], const u64 a[4], const field_t *F) {
    u64 e[4], two[4] = {2, 0, 0, 0};
    sub4(e, F->r, two); /* Fermat: a^(r-2) */
    fpow(out, a, e, F);
}

/* plain value v (< 2^64) -> Montgomery form: mont(v, R^2) */
static void to_mont_u64(u64 out[4], u64 v, const field_t *F) {
    u64 x[4] = {v, 0, 0, 0};
    mont(out, x, F->r2, F);
}

static void field_setup(field_t *F, const u64 r[4], u64 g) {
    memcpy(F->r, r, sizeof F->r);
    /* -r^-1 mod 2^64 by Newton iteration: x <- x (2 - r0 x) doubles the bits. */
    u64 inv = 1;
    for (int i = 0; i < 7; i++) inv *= 2 - r[0] * inv;
    F->rp = (u64)0 - inv;
    /* R mod r and R^2 mod r by repeated doubling of 1 modulo r. */
    u64 x[4] = {1, 0, 0, 0};
    for (int i = 0; i < 512; i++) {
        u64 t[4];
        u64 carry = add4(t, x, x);
        if (carry || geq(t, r)) sub4(t, t, r);
        memcpy(x, t, sizeof x);
        if (i == 255) memcpy(F->one, x, sizeof x);
    }
    memcpy(F->r2, x, sizeof x);
    F->g = g;
    /* 2-adicity of r - 1 */
    u64 rm1[4], one_plain[4] = {1, 0, 0, 0};
    sub4(rm1, r, one_plain);
    int s = 0;
    while (((rm1[s / 64] >> (s % 64)) & 1) == 0) s++;
    F->s = s;
    /* (r - 1) >> s */
    u64 e[4] = {0, 0, 0, 0};
    for (int i = 0; i < 256 - s; i++) {
        int src = i + s;
        if ((rm1[src / 64] >> (src % 64)) & 1) e[i / 64] |= (u64)1 << (i % 64);
    }
    u64 gm[4];
    to_mont_u64(gm, g, F);
    fpow(F->wmax, gm, e, F);
}

static void fields_init(void) {
    pthread_mutex_lock(&init_lock);
    if (!fields_ready) {
        /* BLS12-381, BN254 and BLS12-377 scalar fields (standard moduli). */
        static const u64 bls[4] = {0xffffffff00000001ULL, 0x53bda402fffe5bfeULL,
                                   0x3339d80809a1d805ULL, 0x73eda753299d7d48ULL};
        static const u64 bn[4] = {0x43e1f593f0000001ULL, 0x2833e84879b97091ULL,
                                  0xb85045b68181585dULL, 0x30644e72e131a029ULL};
        static const u64 bls377[4] = {0x0a11800000000001ULL, 0x59aa76fed0000001ULL,
                                      0x60b44d1e5c37b001ULL, 0x12ab655e9a2ca556ULL};
        field_setup(&FIELDS[0], bls, 7);
        field_setup(&FIELDS[1], bn, 5);
        field_setup(&FIELDS[2], bls377, 22);
        fields_ready = 1;
    }
    pthread_mutex_unlock(&init_lock);
}

static void load(u64 out[4], const uint32_t *src) {
    for (int i = 0; i < 4; i++) out[i] = (u64)src[2 * i] | ((u64)src[2 * i + 1] << 32);
}

static void store(uint32_t *dst, const u64 v[4]) {
    for (int i = 0; i < 4; i++) {
        dst[2 * i] = (uint32_t)v[i];
        dst[2 * i + 1] = (uint32_t)(v[i] >> 32);
    }
}

/* omega_n (or its inverse) for n = 2^log_n, Montgomery form: the primitive
 * n-th root the transform of Section II-B needs, w_max^(2^(s - log_n)) */
static void root_of_unity(u64 out[4], const field_t *F, int log_n, int inverse) {
    u64 w[4];
    memcpy(w, F->wmax, sizeof w);
    for (int i = 0; i < F->s - log_n; i++) mont(w, w, w, F);
    if (inverse) finv(w, w, F);
    memcpy(out, w, sizeof w);
}

/* ---------------- tiny parallel-for ---------------- */
typedef void (*range_fn)(void *ctx, u64 lo, u64 hi);
typedef struct { range_fn fn; void *ctx; u64 lo, hi; } task_t;

static void *run_task(void *p) {
    task_t *t = (task_t *)p;
    t->fn(t->ctx, t->lo, t->hi);
    return NULL;
}

static void parallel_for(int threads, u64 count, range_fn fn, void *ctx) {
    if (threads < 1) threads = 1;
    if (count < 4096 || threads == 1) { fn(ctx, 0, count); return; }
    if ((u64)threads > count) threads = (int)count;
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * threads);
    task_t *tasks = (task_t *)malloc(sizeof(task_t) * threads);
    char *live = (char *)calloc((size_t)threads, 1);
    if (!tid || !tasks || !live) {
        free(tid); free(tasks); free(live);
        fn(ctx, 0, count);
        return;
    }
    for (int i = 0; i < threads; i++) {
        tasks[i].fn = fn;
        tasks[i].ctx = ctx;
        tasks[i].lo = count * i / threads;
        tasks[i].hi = count * (i + 1) / threads;
    }
    /* tasks 0..threads-2 on new threads (inline if creation fails), the last here */
    for (int i = 0; i < threads - 1; i++) {
        if (pthread_create(&tid[i], NULL, run_task, &tasks[i]) == 0) live[i] = 1;
        else fn(ctx, tasks[i].lo, tasks[i].hi);
    }
    fn(ctx, tasks[threads - 1].lo, tasks[threads - 1].hi);
    for (int i = 0; i < threads - 1; i++)
        if (live[i]) pthread_join(tid[i], NULL);
    free(tid);
    free(tasks);
    free(live);
}

/* ---------------- the transform ---------------- */
typedef struct {
    const field_t *F;
    u64 (*x)[4];
    u64 (*tw)[4];
    const u64 (*src)[4];
    u64 n;
    int log_n;
    u64 half;
    u64 w[4];
    const u64 *scale;
} job_t;

static u64 bitrev(u64 i, int bits) {
    u64 o = 0;
    for (int b = 0; b < bits; b++) { o = (o << 1) | (i & 1); i >>= 1; }
    return o;
}

static void do_twiddles(void *p, u64 lo, u64 hi) {
    job_t *J = (job_t *)p;
    u64 cur[4];
    fpow_u64(cur, J->w, lo, J->F);
    for (u64 j = lo; j < hi; j++) {
        memcpy(J->tw[j], cur, sizeof cur);
        mont(cur, cur, J->w, J->F);
    }
}

static void do_bitrev(void *p, u64 lo, u64 hi) {
    job_t *J = (job_t *)p;
    for (u64 i = lo; i < hi; i++) memcpy(J->x[i], J->src[bitrev(i, J->log_n)], sizeof J->x[i]);
}

static void do_stage(void *p, u64 lo, u64 hi) {
    job_t *J = (job_t *)p;
    u64 half = J->half, stride = J->n / (2 * half);
    for (u64 b = lo; b < hi; b++) {
        u64 grp = b / half, j = b % half;
        u64 i0 = grp * 2 * half + j, i1 = i0 + half;
        u64 v[4];
        mont(v, J->x[i1], J->tw[j * stride], J->F);
        u64 u[4];
        memcpy(u, J->x[i0], sizeof u);
        fadd(J->x[i0], u, v, J->F);
        fsub(J->x[i1], u, v, J->F);
    }
}

/* x_j <- x_j * c * s^j  (s, c Montgomery form) */
typedef struct { const field_t *F; u64 (*x)[4]; u64 s[4]; u64 c[4]; } scale_t;

static void do_scale(void *p, u64 lo, u64 hi) {
    scale_t *S = (scale_t *)p;
    u64 cur[4];
    fpow_u64(cur, S->s, lo, S->F);
    mont(cur, cur, S->c, S->F);
    for (u64 j = lo; j < hi; j++) {
        mont(S->x[j], S->x[j], cur, S->F);
        mont(cur, cur, S->s, S->F);
    }
}

static void scale_powers(const field_t *F, u64 (*x)[4], u64 n, const u64 s[4], const u64 c[4], int threads) {
    scale_t S;
    S.F = F;
    S.x = x;
    memcpy(S.s, s, sizeof S.s);
    memcpy(S.c, c, sizeof S.c);
    parallel_for(threads, n, do_scale, &S);
}

/* transform in the Montgomery domain, natural order in and out: radix-2
 * decimation in time (Section II-B, Fig. 3(b)), with the inverse's n^-1 and
 * the coset scales (Fig. 2) applied as separate passes */
static int ntt_core(const field_t *F, int log_n, int inverse, const u64 *shift,
                    const u64 (*in)[4], u64 (*out)[4], int threads) {
    u64 n = (u64)1 << log_n;
    u64 (*x)[4] = (u64(*)[4])malloc(sizeof(u64[4]) * n);
    u64 (*tw)[4] = (u64(*)[4])malloc(sizeof(u64[4]) * (n / 2 + 1));
    if (!x || !tw) { free(x); free(tw); return 2; }
    u64 (*src)[4] = (u64(*)[4])in;
    u64 (*pre)[4] = NULL;
    if (!inverse && shift) {
        pre = (u64(*)[4])malloc(sizeof(u64[4]) * n);
        if (!pre) { free(x); free(tw); return 2; }
        memcpy(pre, in, sizeof(u64[4]) * n);
        scale_powers(F, pre, n, shift, F->one, threads);
        src = pre;
    }
    job_t J;
    memset(&J, 0, sizeof J);
    J.F = F;
    J.x = x;
    J.tw = tw;
    J.src = (const u64(*)[4])src;
    J.n = n;
    J.log_n = log_n;
    root_of_unity(J.w, F, log_n, inverse);
    if (n >= 2) parallel_for(threads, n / 2, do_twiddles, &J);
    parallel_for(threads, n, do_bitrev, &J);
    for (J.half = 1; J.half < n; J.half *= 2) parallel_for(threads, n / 2, do_stage, &J);
    if (inverse) {
        u64 nm[4], ninv[4];
        to_mont_u64(nm, n, F);
        finv(ninv, nm, F);
        if (shift) {
            u64 sinv[4];
            finv(sinv, shift, F);
            scale_powers(F, x, n, sinv, ninv, threads);
        } else {
            scale_powers(F, x, n, F->one, ninv, threads);
        }
    }
    memcpy(out, x, sizeof(u64[4]) * n);
    free(x);
    free(tw);
    free(pre);
    return 0;
}

static int check_args(int field, int log_n) {
    if (field < 0 || field >= NFIELDS) return 1;
    fields_init();
    if (log_n < 0 || log_n > FIELDS[field].s || log_n > 30) return 1;
    return 0;
}

static u64 (*load_vec(const uint32_t *src, u64 n))[4] {
    u64 (*v)[4] = (u64(*)[4])malloc(sizeof(u64[4]) * (n ? n : 1));
    if (!v) return NULL;
    for (u64 i = 0; i < n; i++) load(v[i], src + 8 * i);
    return v;
}

static void store_vec(uint32_t *dst, u64 (*v)[4], u64 n) {
    for (u64 i = 0; i < n; i++) store(dst + 8 * i, v[i]);
}

/* ---------------- exported API (Montgomery-form u32 limbs) ---------------- */

int zo_threads_default(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* 2-adicity s of r - 1: the largest transform is 2^s (Section II-B) */
int zo_two_adicity(int field) {
    if (field < 0 || field >= NFIELDS) return -1;
    fields_init();
    return FIELDS[field].s;
}

/* the primitive 2^log_n-th root (or its inverse), Montgomery form (Section II-B) */
int zo_root(int field, int log_n, int inverse, uint32_t *out) {
    if (field < 0 || field >= NFIELDS) return 1;
    fields_init();
    if (log_n < 0 || log_n > FIELDS[field].s) return 1;
    u64 w[4];
    root_of_unity(w, &FIELDS[field], log_n, inverse);
    store(out, w);
    return 0;
}

/* Montgomery product a b 2^-256 mod r (FF_mul, Section IV-B) */
int zo_mont_mul(int field, const uint32_t *a, const uint32_t *b, uint32_t *out) {
    if (field < 0 || field >= NFIELDS) return 1;
    fields_init();
    u64 x[4], y[4], z[4];
    load(x, a);
    load(y, b);
    mont(z, x, y, &FIELDS[field]);
    store(out, z);
    return 0;
}

/* forward / inverse / coset transform of n = 2^log_n Montgomery-form elements
 * (Section II-B; coset and inverse readings as in the file header) */
int zo_ntt(int field, int log_n, int inverse, const uint32_t *shift_mont,
           const uint32_t *in, uint32_t *out, int threads) {
    if (check_args(field, log_n)) return 1;
    u64 n = (u64)1 << log_n;
    u64 (*v)[4] = load_vec(in, n);
    if (!v) return 2;
    u64 sh[4];
    if (shift_mont) load(sh, shift_mont);
    int rc = ntt_core(&FIELDS[field], log_n, inverse, shift_mont ? sh : NULL,
                      (const u64(*)[4])v, v, threads);
    if (rc == 0) store_vec(out, v, n);
    free(v);
    return rc;
}

/* out = sum_j c_j x^j (Horner), all Montgomery form: one output A_k of the
 * Section II-B definition when x = w^k */
int zo_eval(int field, uint64_t n, const uint32_t *coeffs, const uint32_t *x_mont, uint32_t *out) {
    if (field < 0 || field >= NFIELDS) return 1;
    fields_init();
    const field_t *F = &FIELDS[field];
    u64 x[4], acc[4] = {0, 0, 0, 0}, c[4];
    load(x, x_mont);
    for (u64 i = n; i-- > 0;) {
        mont(acc, acc, x, F);
        load(c, coeffs + 8 * i);
        fadd(acc, acc, c, F);
    }
    store(out, acc);
    return 0;
}

typedef struct { const field_t *F; u64 (*A)[4]; u64 (*B)[4]; u64 (*C)[4]; u64 z[4]; } pw_t;

static void do_pointwise(void *p, u64 lo, u64 hi) {
    pw_t *P = (pw_t *)p;
    for (u64 i = lo; i < hi; i++) {
        u64 t[4];
        mont(t, P->A[i], P->B[i], P->F);
        fsub(t, t, P->C[i], P->F);
        mont(P->A[i], t, P->z, P->F);
    }
}

/* the Groth16 H sequence (Fig. 2, Section IV-A) */
int zo_groth16_h(int field, int log_n, const uint32_t *a, const uint32_t *b,
                 const uint32_t *c, uint32_t *h, int threads) {
    if (check_args(field, log_n)) return 1;
    const field_t *F = &FIELDS[field];
    u64 n = (u64)1 << log_n;
    u64 (*A)[4] = load_vec(a, n), (*B)[4] = load_vec(b, n), (*C)[4] = load_vec(c, n);
    if (!A || !B || !C) { free(A); free(B); free(C); return 2; }
    u64 g[4];
    to_mont_u64(g, F->g, F);
    int rc = 0;
    u64 (*vs[3])[4] = {A, B, C};
    for (int k = 0; k < 3 && !rc; k++) {
        rc |= ntt_core(F, log_n, 1, NULL, (const u64(*)[4])vs[k], vs[k], threads);
        rc |= ntt_core(F, log_n, 0, g, (const u64(*)[4])vs[k], vs[k], threads);
    }
    if (!rc) {
        pw_t P;
        P.F = F; P.A = A; P.B = B; P.C = C;
        u64 gn[4], one[4];
        fpow_u64(gn, g, n, F);
        memcpy(one, F->one, sizeof one);
        fsub(gn, gn, one, F);
        finv(P.z, gn, F);
        parallel_for(threads, n, do_pointwise, &P);
        rc = ntt_core(F, log_n, 1, g, (const u64(*)[4])A, A, threads);
    }
    if (!rc) store_vec(h, A, n);
    free(A); free(B); free(C);
    return rc;
}
