/*
 * spdz_oracle.c -- plain, slow CPU oracle for the SPDZ online phase.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the bench's CPU
 * baseline leg may load this library.  It shares no code with the CUDA path:
 * the field, the counter PRG, the dealer and every protocol step are written
 * here again, from their definitions, for a generic odd prime p < 2^127.
 *
 * Arithmetic: every value is an integer in [0, p) held in an unsigned
 * __int128.  Products use the plain `%` operator when p < 2^64 and
 * double-and-add otherwise; there is no Mersenne-specific reduction.
 *
 * External element format (all arrays): w 64-bit little-endian words per
 * element, w = 1 when p < 2^64 and w = 2 otherwise.  Party-major share arrays
 * are laid out [n][count][w].
 *
 * Where each function comes from (An LLVM-Based Optimization Pipeline for
 * SPDZ, arXiv 2512.11112):
 *   - additive sharing and the MAC relation ........ Sec. II-A.2
 *   - local addition / linear gates ................. Sec. II-A.3 (Addition)
 *   - Beaver multiplication and the triple identity . Sec. II-A.3 (Multiplication)
 *   - batched MAC check (abort on failure) .......... Sec. II-A.2, II-A.4, III-D.3
 *   - matrix (tile) Beaver triples .................. Sec. III-D.3
 *   - LinearLayer y = W x + b, row tiles, one
 *     matrix-vector triple per tile ................ Sec. III-D.3, Sec. IV
 *   - input sharing and the checked reveal of
 *     outputs .................................... Sec. I (sharing sketch),
 *                                                   Sec. II-A.2, Sec. IV ("all
 *                                                   inputs are secret-shared")
 *   - ReduceAdd (horizontal sum, inner products) .... Sec. III-B (vectorization)
 *   - fake preprocessing (dealer) ................... Sec. IV-A
 * The paper gives no formula for the MAC-share updates, for which party adds
 * the public d*e term, or for the MAC-check algorithm; the readings used are:
 * only party 0 adds d*e to its value share, every party adds alpha_i*d*e to
 * its MAC share, public-constant add goes to party 0's value and alpha_i*k to
 * every MAC share, and the check is the SPDZ random-linear-combination check
 * (sigma_i = S_i - alpha_i * A, accept iff sum sigma_i == 0).
 *
 * Parity status: every protocol function is pinned by the tests in
 * tests/test_oracle_*.py against closed forms (reconstruct(z) == x*y mod p,
 * sum gamma_i(v) == alpha*v, linearity, cleartext circuit evaluation,
 * X*Y for matrices), brute force over tiny primes, and deterministic tamper
 * detection.  The dealer's individual share values are fixed only by the PRG
 * specification (SplitMix64 counter form), which the CUDA side implements
 * independently.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef unsigned __int128 u128;
typedef uint64_t u64;

/* ------------------------------------------------------------------ field */

static inline u128 f_add(u128 a, u128 b, u128 p) {
    u128 s = a + b;               /* a, b < p < 2^127: no overflow */
    return s >= p ? s - p : s;
}

static inline u128 f_sub(u128 a, u128 b, u128 p) {
    return a >= b ? a - b : p - (b - a);
}

static inline u128 f_mul(u128 a, u128 b, u128 p) {
    if ((p >> 64) == 0)
        return ((u128)(u64)a * (u128)(u64)b) % p;
    /* double-and-add over the bits of b, most significant first */
    u128 r = 0;
    for (int bit = 127; bit >= 0; --bit) {
        r = f_add(r, r, p);
        if ((b >> bit) & 1) r = f_add(r, a, p);
    }
    return r;
}

static inline int words_of(u128 p) { return (p >> 64) ? 2 : 1; }

static inline u128 ld(const u64 *a, int64_t idx, int w) {
    if (w == 1) return (u128)a[idx];
    return ((u128)a[2 * idx + 1] << 64) | (u128)a[2 * idx];
}

static inline void st(u64 *a, int64_t idx, int w, u128 v) {
    if (w == 1) { a[idx] = (u64)v; return; }
    a[2 * idx] = (u64)v;
    a[2 * idx + 1] = (u64)(v >> 64);
}

static inline u128 mkp(u64 plo, u64 phi) { return ((u128)phi << 64) | plo; }

static int bitlen(u128 p) {
    int b = 0;
    while (p) { ++b; p >>= 1; }
    return b;
}

/* Exported scalar field ops, so the tests can pin them against Python ints. */
void orc_fadd(u64 plo, u64 phi, const u64 *a, const u64 *b, u64 *out) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    st(out, 0, w, f_add(ld(a, 0, w), ld(b, 0, w), p));
}
void orc_fsub(u64 plo, u64 phi, const u64 *a, const u64 *b, u64 *out) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    st(out, 0, w, f_sub(ld(a, 0, w), ld(b, 0, w), p));
}
void orc_fmul(u64 plo, u64 phi, const u64 *a, const u64 *b, u64 *out) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    st(out, 0, w, f_mul(ld(a, 0, w), ld(b, 0, w), p));
}

/* ---------------------------------------------------------- counter PRG
 * SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), in counter form: output i of a generator whose
 * state starts at `key` is mix(key + (i + 1) * GAMMA).
 *   stream key      K(seed, stream) = sm64(seed, stream)
 *   element j of a stream: b = bitlen(p); if b <= 64 take the top b bits of
 *   sm64(K, j); else take sm64(K, 2j) as the low word and the top b-64 bits of
 *   sm64(K, 2j+1) as the high word; subtract p once if the value is >= p.
 *   stream id = kind << 56 | role << 48 | party << 40 | sub (sub < 2^40).
 */
#define SM_GAMMA 0x9E3779B97F4A7C15ULL

static inline u64 sm_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

u64 orc_sm64(u64 key, u64 i) { return sm_mix(key + (i + 1) * SM_GAMMA); }

u64 orc_stream_id(u64 kind, u64 role, u64 party, u64 sub) {
    return (kind << 56) | (role << 48) | (party << 40) | (sub & ((1ULL << 40) - 1));
}

u64 orc_stream_key(u64 seed, u64 stream) { return orc_sm64(seed, stream); }

static u128 draw_elem(u64 key, u64 j, u128 p) {
    int b = bitlen(p);
    u128 v;
    if (b <= 64) {
        v = (u128)(orc_sm64(key, j) >> (64 - b));
    } else {
        u64 lo = orc_sm64(key, 2 * j);
        u64 hi = orc_sm64(key, 2 * j + 1) >> (128 - b);
        v = ((u128)hi << 64) | lo;
    }
    return v >= p ? v - p : v;
}

void orc_draw(u64 plo, u64 phi, u64 seed, u64 stream, u64 j0, int64_t count, u64 *out) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    u64 key = orc_stream_key(seed, stream);
    for (int64_t j = 0; j < count; ++j) st(out, j, w, draw_elem(key, j0 + (u64)j, p));
}

enum { K_ALPHA = 1, K_TRIPLE_A = 2, K_TRIPLE_B = 3, K_TRIPLE_C = 4, K_INPUT = 5,
       K_CHECK = 6, K_MTRIPLE_A = 7, K_MTRIPLE_B = 8, K_MTRIPLE_C = 9, K_INPUT_MASK = 10 };
enum { R_SECRET = 0, R_VAL_SHARE = 1, R_MAC_SHARE = 2 };

/* ------------------------------------------------------------- threading */

typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void *ctx; int64_t lo, hi; } range_job;

static void *range_thread(void *arg) {
    range_job *j = (range_job *)arg;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static int g_threads = 1;
void orc_set_threads(int t) { g_threads = t < 1 ? 1 : (t > 256 ? 256 : t); }
int orc_get_threads(void) { return g_threads; }

/* Runs fn over [0, count) split into contiguous chunks, one per thread. */
static void parallel_for(int64_t count, range_fn fn, void *ctx) {
    int t = g_threads;
    if (t <= 1 || count < 4096) { fn(ctx, 0, count); return; }
    pthread_t th[256];
    range_job jobs[256];
    int64_t chunk = (count + t - 1) / t;
    int used = 0;
    for (int k = 0; k < t; ++k) {
        int64_t lo = (int64_t)k * chunk, hi = lo + chunk;
        if (lo >= count) break;
        if (hi > count) hi = count;
        jobs[k] = (range_job){fn, ctx, lo, hi};
        pthread_create(&th[k], NULL, range_thread, &jobs[k]);
        ++used;
    }
    for (int k = 0; k < used; ++k) pthread_join(th[k], NULL);
}

/* ---------------------------------------------------------------- dealer
 * "Fake preprocessing" (Sec. IV-A): a trusted dealer samples alpha, the
 * secrets and all but the last party's shares from the PRG; the last party's
 * share makes the sum come out right (additive sharing, Sec. II-A.2).
 */

void orc_deal_alpha(u64 plo, u64 phi, int n, u64 seed, u64 *alpha_out, u64 *shares_out) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    u128 alpha = draw_elem(orc_stream_key(seed, orc_stream_id(K_ALPHA, R_SECRET, 0, 0)), 0, p);
    u128 sum = 0;
    for (int i = 0; i < n - 1; ++i) {
        u128 s = draw_elem(orc_stream_key(seed, orc_stream_id(K_ALPHA, R_VAL_SHARE, (u64)i, 0)), 0, p);
        st(shares_out, i, w, s);
        sum = f_add(sum, s, p);
    }
    st(shares_out, n - 1, w, f_sub(alpha, sum, p));
    st(alpha_out, 0, w, alpha);
}


/* Derives the per-party PRG keys of one shared array (kind, sub). */
typedef struct {
    u64 key_secret;
    u64 key_v[64];
    u64 key_m[64];
} share_keys;

static void make_share_keys(share_keys *k, u64 seed, int n, u64 kind, u64 sub) {
    k->key_secret = orc_stream_key(seed, orc_stream_id(kind, R_SECRET, 0, sub));
    for (int i = 0; i < n - 1; ++i) {
        k->key_v[i] = orc_stream_key(seed, orc_stream_id(kind, R_VAL_SHARE, (u64)i, sub));
        k->key_m[i] = orc_stream_key(seed, orc_stream_id(kind, R_MAC_SHARE, (u64)i, sub));
    }
}

/* Shares secret v (and its MAC alpha*v) of global index gj into slot j of
 * the [n][count] output arrays. */
static void share_one(const share_keys *k, int n, u128 p, int w, u128 alpha, u64 gj,
                      u128 v, int64_t j, int64_t count, u64 *val, u64 *mac) {
    u128 m = f_mul(alpha, v, p);
    u128 sv = 0, sm = 0;
    for (int i = 0; i < n - 1; ++i) {
        u128 vi = draw_elem(k->key_v[i], gj, p);
        u128 mi = draw_elem(k->key_m[i], gj, p);
        st(val, (int64_t)i * count + j, w, vi);
        st(mac, (int64_t)i * count + j, w, mi);
        sv = f_add(sv, vi, p);
        sm = f_add(sm, mi, p);
    }
    st(val, (int64_t)(n - 1) * count + j, w, f_sub(v, sv, p));
    st(mac, (int64_t)(n - 1) * count + j, w, f_sub(m, sm, p));
}

typedef struct {
    u128 p, alpha; int w, n; u64 j0; int64_t count;
    share_keys k;
    const u64 *secret_in; u64 *val, *mac, *secret_out;
} deal_shared_ctx;

static void deal_shared_range(void *vc, int64_t lo, int64_t hi) {
    deal_shared_ctx *c = (deal_shared_ctx *)vc;
    for (int64_t j = lo; j < hi; ++j) {
        u64 gj = c->j0 + (u64)j;
        u128 v = c->secret_in ? ld(c->secret_in, j, c->w) : draw_elem(c->k.key_secret, gj, c->p);
        if (c->secret_out) st(c->secret_out, j, c->w, v);
        share_one(&c->k, c->n, c->p, c->w, c->alpha, gj, v, j, c->count, c->val, c->mac);
    }
}

/* Elements j0 .. j0+count-1 of the secret-shared array (kind, sub): the
 * secret is drawn from the PRG unless secret_in is given; value shares and
 * MAC shares of alpha*secret go to val/mac [n][count]. */
void orc_deal_shared(u64 plo, u64 phi, int n, u64 seed, u64 kind, u64 sub, u64 j0,
                     int64_t count, const u64 *alpha, const u64 *secret_in,
                     u64 *val, u64 *mac, u64 *secret_out) {
    deal_shared_ctx c;
    c.p = mkp(plo, phi); c.w = words_of(c.p); c.n = n; c.j0 = j0; c.count = count;
    c.alpha = ld(alpha, 0, c.w);
    make_share_keys(&c.k, seed, n, kind, sub);
    c.secret_in = secret_in; c.val = val; c.mac = mac; c.secret_out = secret_out;
    parallel_for(count, deal_shared_range, &c);
}

typedef struct {
    u128 p, alpha; int w, n; u64 j0; int64_t count;
    share_keys ka, kb, kc;
    u64 *av, *am, *bv, *bm, *cv, *cm;
} deal_triple_ctx;

static void deal_triple_range(void *vc, int64_t lo, int64_t hi) {
    deal_triple_ctx *c = (deal_triple_ctx *)vc;
    for (int64_t j = lo; j < hi; ++j) {
        u64 gj = c->j0 + (u64)j;
        u128 a = draw_elem(c->ka.key_secret, gj, c->p);
        u128 b = draw_elem(c->kb.key_secret, gj, c->p);
        u128 cc = f_mul(a, b, c->p);
        share_one(&c->ka, c->n, c->p, c->w, c->alpha, gj, a, j, c->count, c->av, c->am);
        share_one(&c->kb, c->n, c->p, c->w, c->alpha, gj, b, j, c->count, c->bv, c->bm);
        share_one(&c->kc, c->n, c->p, c->w, c->alpha, gj, cc, j, c->count, c->cv, c->cm);
    }
}

/* Beaver triples j0 .. j0+count-1: a, b uniform, c = a*b (Sec. II-A.3), each
 * shared with MACs (kinds TRIPLE_A/B/C, sub 0). */
void orc_deal_triples(u64 plo, u64 phi, int n, u64 seed, u64 j0, int64_t count,
                      const u64 *alpha, u64 *av, u64 *am, u64 *bv, u64 *bm, u64 *cv, u64 *cm) {
    deal_triple_ctx c;
    c.p = mkp(plo, phi); c.w = words_of(c.p); c.n = n; c.j0 = j0; c.count = count;
    c.alpha = ld(alpha, 0, c.w);
    make_share_keys(&c.ka, seed, n, K_TRIPLE_A, 0);
    make_share_keys(&c.kb, seed, n, K_TRIPLE_B, 0);
    make_share_keys(&c.kc, seed, n, K_TRIPLE_C, 0);
    c.av = av; c.am = am; c.bv = bv; c.bm = bm; c.cv = cv; c.cm = cm;
    parallel_for(count, deal_triple_range, &c);
}

/* ------------------------------------------------------------ linear gates
 * Sec. II-A.3 (Addition): z_i = x_i + y_i, MAC shares added the same way.
 * Subtraction likewise.  Public-constant multiply scales value and MAC
 * shares by k.  Public-constant add: party 0 adds k to its value share and
 * every party adds alpha_i * k to its MAC share (so sum gamma_i = alpha*(x+k)).
 */
enum { OP_ADD = 0, OP_SUB = 1, OP_CMUL = 2, OP_CADD = 3, OP_MUL = 4 };

typedef struct {
    u128 p; int w, n, op; int64_t count; u128 k;
    const u64 *xv, *xm, *yv, *ym, *alpha_sh; u64 *zv, *zm;
} linear_ctx;

static void linear_range(void *vc, int64_t lo, int64_t hi) {
    linear_ctx *c = (linear_ctx *)vc;
    u128 p = c->p; int w = c->w;
    for (int64_t j = lo; j < hi; ++j) {
        for (int i = 0; i < c->n; ++i) {
            int64_t e = (int64_t)i * c->count + j;
            u128 x = ld(c->xv, e, w), gx = ld(c->xm, e, w), z, gz;
            switch (c->op) {
            case OP_ADD:
                z = f_add(x, ld(c->yv, e, w), p); gz = f_add(gx, ld(c->ym, e, w), p); break;
            case OP_SUB:
                z = f_sub(x, ld(c->yv, e, w), p); gz = f_sub(gx, ld(c->ym, e, w), p); break;
            case OP_CMUL:
                z = f_mul(c->k, x, p); gz = f_mul(c->k, gx, p); break;
            default: /* OP_CADD */
                z = (i == 0) ? f_add(x, c->k, p) : x;
                gz = f_add(gx, f_mul(ld(c->alpha_sh, i, w), c->k, p), p);
                break;
            }
            st(c->zv, e, w, z);
            st(c->zm, e, w, gz);
        }
    }
}

/* Arrays [n][count]; y may be NULL for CMUL/CADD; k is one field element. */
void orc_linear(u64 plo, u64 phi, int n, int op, int64_t count,
                const u64 *xv, const u64 *xm, const u64 *yv, const u64 *ym,
                const u64 *k, const u64 *alpha_sh, u64 *zv, u64 *zm) {
    linear_ctx c;
    c.p = mkp(plo, phi); c.w = words_of(c.p); c.n = n; c.op = op; c.count = count;
    c.k = (op == OP_CMUL || op == OP_CADD) ? ld(k, 0, c.w) : 0;
    c.xv = xv; c.xm = xm; c.yv = yv; c.ym = ym; c.alpha_sh = alpha_sh; c.zv = zv; c.zm = zm;
    parallel_for(count, linear_range, &c);
}

/* ------------------------------------------------------------------- open
 * Sec. II-A.3: the public value is the sum of all parties' shares. */
void orc_open(u64 plo, u64 phi, int n, int64_t count, const u64 *xv, u64 *out) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    for (int64_t j = 0; j < count; ++j) {
        u128 s = 0;
        for (int i = 0; i < n; ++i) s = f_add(s, ld(xv, (int64_t)i * count + j, w), p);
        st(out, j, w, s);
    }
}

/* ------------------------------------------------------------------ Beaver
 * Sec. II-A.3 (Multiplication).  For each j:
 *   d_i = x_i - a_i,  e_i = y_i - b_i;  d = sum d_i,  e = sum e_i  (opened)
 *   z_i = c_i + d*b_i + e*a_i + [i == 0] d*e
 *   gamma(z)_i = gamma(c)_i + d*gamma(b)_i + e*gamma(a)_i + alpha_i*d*e
 * The opened d (= eps) carries MAC shares gamma(x)_i - gamma(a)_i and e
 * (= delta) carries gamma(y)_i - gamma(b)_i; they are returned for the check.
 */
typedef struct {
    u128 p; int w, n; int64_t count;
    const u64 *xv, *xm, *yv, *ym, *av, *am, *bv, *bm, *cv, *cm, *alpha_sh;
    u64 *zv, *zm, *eps, *dlt, *eps_mac, *dlt_mac;
} mul_ctx;

static void mul_range(void *vc, int64_t lo, int64_t hi) {
    mul_ctx *c = (mul_ctx *)vc;
    u128 p = c->p; int w = c->w, n = c->n;
    for (int64_t j = lo; j < hi; ++j) {
        u128 d = 0, e = 0;
        for (int i = 0; i < n; ++i) {
            int64_t q = (int64_t)i * c->count + j;
            d = f_add(d, f_sub(ld(c->xv, q, w), ld(c->av, q, w), p), p);
            e = f_add(e, f_sub(ld(c->yv, q, w), ld(c->bv, q, w), p), p);
        }
        u128 de = f_mul(d, e, p);
        for (int i = 0; i < n; ++i) {
            int64_t q = (int64_t)i * c->count + j;
            u128 z = f_add(ld(c->cv, q, w),
                           f_add(f_mul(d, ld(c->bv, q, w), p), f_mul(e, ld(c->av, q, w), p), p), p);
            if (i == 0) z = f_add(z, de, p);
            u128 gz = f_add(ld(c->cm, q, w),
                            f_add(f_mul(d, ld(c->bm, q, w), p), f_mul(e, ld(c->am, q, w), p), p), p);
            gz = f_add(gz, f_mul(ld(c->alpha_sh, i, w), de, p), p);
            st(c->zv, q, w, z);
            st(c->zm, q, w, gz);
            if (c->eps_mac) st(c->eps_mac, q, w, f_sub(ld(c->xm, q, w), ld(c->am, q, w), p));
            if (c->dlt_mac) st(c->dlt_mac, q, w, f_sub(ld(c->ym, q, w), ld(c->bm, q, w), p));
        }
        if (c->eps) st(c->eps, j, w, d);
        if (c->dlt) st(c->dlt, j, w, e);
    }
}

/* All share arrays [n][count]; the triple arrays start at the triple this
 * batch consumes first.  eps/dlt [count], eps_mac/dlt_mac [n][count]: NULL
 * to skip. */
void orc_mul(u64 plo, u64 phi, int n, int64_t count,
             const u64 *xv, const u64 *xm, const u64 *yv, const u64 *ym,
             const u64 *av, const u64 *am, const u64 *bv, const u64 *bm,
             const u64 *cv, const u64 *cm, const u64 *alpha_sh,
             u64 *zv, u64 *zm, u64 *eps, u64 *dlt, u64 *eps_mac, u64 *dlt_mac) {
    mul_ctx c;
    c.p = mkp(plo, phi); c.w = words_of(c.p); c.n = n; c.count = count;
    c.xv = xv; c.xm = xm; c.yv = yv; c.ym = ym; c.av = av; c.am = am; c.bv = bv; c.bm = bm;
    c.cv = cv; c.cm = cm; c.alpha_sh = alpha_sh;
    c.zv = zv; c.zm = zm; c.eps = eps; c.dlt = dlt; c.eps_mac = eps_mac; c.dlt_mac = dlt_mac;
    parallel_for(count, mul_range, &c);
}

/* --------------------------------------------------------------- MAC check
 * Random linear combination over opened values v_j (public) with MAC shares
 * gamma_i(v_j):  r_j = element j0+j of stream (CHECK, 0, 0, epoch) under
 * check_seed;  A = sum r_j v_j;  S_i = sum r_j gamma_i(v_j).  orc_rlc returns
 * A and S for one chunk of the opened log; chunks add mod p.
 */
void orc_check_coeffs(u64 plo, u64 phi, u64 check_seed, u64 epoch, u64 j0, int64_t m, u64 *r) {
    orc_draw(plo, phi, check_seed, orc_stream_id(K_CHECK, 0, 0, epoch), j0, m, r);
}

void orc_rlc(u64 plo, u64 phi, int n, int64_t m, const u64 *vals, const u64 *macs,
             u64 check_seed, u64 epoch, u64 j0, u64 *A_out, u64 *S_out) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    u64 key = orc_stream_key(check_seed, orc_stream_id(K_CHECK, 0, 0, epoch));
    u128 A = 0, S[64];
    for (int i = 0; i < n; ++i) S[i] = 0;
    for (int64_t j = 0; j < m; ++j) {
        u128 r = draw_elem(key, j0 + (u64)j, p);
        A = f_add(A, f_mul(r, ld(vals, j, w), p), p);
        for (int i = 0; i < n; ++i)
            S[i] = f_add(S[i], f_mul(r, ld(macs, (int64_t)i * m + j, w), p), p);
    }
    st(A_out, 0, w, A);
    for (int i = 0; i < n; ++i) st(S_out, i, w, S[i]);
}

/* sigma_i = S_i - alpha_i * A; the check passes iff sum_i sigma_i == 0
 * (then sum_i S_i == alpha * A, the MAC relation of Sec. II-A.2). */
int orc_check_finish(u64 plo, u64 phi, int n, const u64 *A, const u64 *S,
                     const u64 *alpha_sh, u64 *sigma_out) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    u128 a = ld(A, 0, w), tot = 0;
    for (int i = 0; i < n; ++i) {
        u128 s = f_sub(ld(S, i, w), f_mul(ld(alpha_sh, i, w), a, p), p);
        st(sigma_out, i, w, s);
        tot = f_add(tot, s, p);
    }
    return tot == 0;
}

/* ---------------------------------------------------------- inner products
 * P products of length L (ReduceAdd over a MultBatch, Sec. III-B): each term
 * is a Beaver product, opened in one batch; the products' shares and MAC
 * shares are summed locally, z_t = sum_k x_{t,k} * y_{t,k}.  Term arrays are
 * [n][P*L] with term (t, k) at t*L + k; outputs are [n][P]; the opened
 * values and their MAC shares of the terms are returned like orc_mul's.
 */
void orc_innerprod(u64 plo, u64 phi, int n, int64_t P, int64_t L,
                   const u64 *xv, const u64 *xm, const u64 *yv, const u64 *ym,
                   const u64 *av, const u64 *am, const u64 *bv, const u64 *bm,
                   const u64 *cv, const u64 *cm, const u64 *alpha_sh,
                   u64 *zv, u64 *zm, u64 *eps, u64 *dlt, u64 *eps_mac, u64 *dlt_mac) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    int64_t T = P * L;
    u64 *tv = (u64 *)malloc(sizeof(u64) * (size_t)(n * T * w));
    u64 *tm = (u64 *)malloc(sizeof(u64) * (size_t)(n * T * w));
    orc_mul(plo, phi, n, T, xv, xm, yv, ym, av, am, bv, bm, cv, cm, alpha_sh,
            tv, tm, eps, dlt, eps_mac, dlt_mac);
    for (int i = 0; i < n; ++i)
        for (int64_t t = 0; t < P; ++t) {
            u128 sv = 0, sm = 0;
            for (int64_t k = 0; k < L; ++k) {
                sv = f_add(sv, ld(tv, (int64_t)i * T + t * L + k, w), p);
                sm = f_add(sm, ld(tm, (int64_t)i * T + t * L + k, w), p);
            }
            st(zv, (int64_t)i * P + t, w, sv);
            st(zm, (int64_t)i * P + t, w, sm);
        }
    free(tv); free(tm);
}

/* ----------------------------------------------------------- matrix Beaver
 * Sec. III-D.3: with a matrix triple (A, B, C = A*B), open E = X - A (M x K)
 * and F = Y - B (K x N); then
 *   Z_i = C_i + E*B_i + A_i*F + [i == 0] E*F
 *   gamma(Z)_i = gamma(C)_i + E*gamma(B)_i + gamma(A)_i*F + alpha_i * E*F
 * orc_mat_open returns E, F and their MAC shares; orc_mat_entries computes
 * chosen entries of every party's Z and gamma(Z) by the plain triple loop.
 */
void orc_mat_open(u64 plo, u64 phi, int n, int64_t M, int64_t K, int64_t N,
                  const u64 *Xv, const u64 *Xm, const u64 *Yv, const u64 *Ym,
                  const u64 *Av, const u64 *Am, const u64 *Bv, const u64 *Bm,
                  u64 *E, u64 *F, u64 *E_mac, u64 *F_mac) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    int64_t mk = M * K, kn = K * N;
    for (int64_t j = 0; j < mk; ++j) {
        u128 s = 0;
        for (int i = 0; i < n; ++i) {
            int64_t q = (int64_t)i * mk + j;
            s = f_add(s, f_sub(ld(Xv, q, w), ld(Av, q, w), p), p);
            if (E_mac) st(E_mac, q, w, f_sub(ld(Xm, q, w), ld(Am, q, w), p));
        }
        st(E, j, w, s);
    }
    for (int64_t j = 0; j < kn; ++j) {
        u128 s = 0;
        for (int i = 0; i < n; ++i) {
            int64_t q = (int64_t)i * kn + j;
            s = f_add(s, f_sub(ld(Yv, q, w), ld(Bv, q, w), p), p);
            if (F_mac) st(F_mac, q, w, f_sub(ld(Ym, q, w), ld(Bm, q, w), p));
        }
        st(F, j, w, s);
    }
}

typedef struct {
    u128 p; int w, n; int64_t M, K, N, nidx;
    const u64 *E, *F, *Av, *Am, *Bv, *Bm, *Cv, *Cm, *alpha_sh;
    const int64_t *rows, *cols;
    u64 *Zv, *Zm;
} mat_ctx;

static void mat_range(void *vc, int64_t lo, int64_t hi) {
    mat_ctx *c = (mat_ctx *)vc;
    u128 p = c->p; int w = c->w;
    int64_t M = c->M, K = c->K, N = c->N;
    for (int64_t t = lo; t < hi; ++t) {
        int64_t r = c->rows[t], col = c->cols[t];
        u128 ef = 0;
        for (int64_t k = 0; k < K; ++k)
            ef = f_add(ef, f_mul(ld(c->E, r * K + k, w), ld(c->F, k * N + col, w), p), p);
        for (int i = 0; i < c->n; ++i) {
            const int64_t oa = (int64_t)i * M * K, ob = (int64_t)i * K * N, oc = (int64_t)i * M * N;
            u128 z = ld(c->Cv, oc + r * N + col, w);
            u128 gz = ld(c->Cm, oc + r * N + col, w);
            for (int64_t k = 0; k < K; ++k) {
                u128 e = ld(c->E, r * K + k, w), f = ld(c->F, k * N + col, w);
                z = f_add(z, f_mul(e, ld(c->Bv, ob + k * N + col, w), p), p);
                z = f_add(z, f_mul(ld(c->Av, oa + r * K + k, w), f, p), p);
                gz = f_add(gz, f_mul(e, ld(c->Bm, ob + k * N + col, w), p), p);
                gz = f_add(gz, f_mul(ld(c->Am, oa + r * K + k, w), f, p), p);
            }
            if (i == 0) z = f_add(z, ef, p);
            gz = f_add(gz, f_mul(ld(c->alpha_sh, i, w), ef, p), p);
            st(c->Zv, (int64_t)i * c->nidx + t, w, z);
            st(c->Zm, (int64_t)i * c->nidx + t, w, gz);
        }
    }
}

void orc_mat_entries(u64 plo, u64 phi, int n, int64_t M, int64_t K, int64_t N,
                     const u64 *E, const u64 *F,
                     const u64 *Av, const u64 *Am, const u64 *Bv, const u64 *Bm,
                     const u64 *Cv, const u64 *Cm, const u64 *alpha_sh,
                     int64_t nidx, const int64_t *rows, const int64_t *cols,
                     u64 *Zv, u64 *Zm) {
    mat_ctx c;
    c.p = mkp(plo, phi); c.w = words_of(c.p); c.n = n; c.M = M; c.K = K; c.N = N; c.nidx = nidx;
    c.E = E; c.F = F; c.Av = Av; c.Am = Am; c.Bv = Bv; c.Bm = Bm; c.Cv = Cv; c.Cm = Cm;
    c.alpha_sh = alpha_sh; c.rows = rows; c.cols = cols; c.Zv = Zv; c.Zm = Zm;
    parallel_for(nidx, mat_range, &c);
}

/* Matrix triples: A (M x K) and B (K x N) uniform, C = A*B computed by the
 * plain triple loop, each shared with MACs (kinds MTRIPLE_A/B/C, element
 * index = row-major position).  sub selects the triple. */
typedef struct {
    u128 p; int w; int64_t M, K, N;
    const u64 *a, *b; u64 *c;
} matprod_ctx;

static void matprod_range(void *vc, int64_t lo, int64_t hi) {
    matprod_ctx *c = (matprod_ctx *)vc;
    for (int64_t t = lo; t < hi; ++t) {
        int64_t r = t / c->N, col = t % c->N;
        u128 s = 0;
        for (int64_t k = 0; k < c->K; ++k)
            s = f_add(s, f_mul(ld(c->a, r * c->K + k, c->w), ld(c->b, k * c->N + col, c->w), c->p), c->p);
        st(c->c, t, c->w, s);
    }
}

void orc_deal_matrix_triple(u64 plo, u64 phi, int n, u64 seed, u64 sub,
                            int64_t M, int64_t K, int64_t N, const u64 *alpha,
                            u64 *Av, u64 *Am, u64 *Bv, u64 *Bm, u64 *Cv, u64 *Cm) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    u64 *a = (u64 *)malloc(sizeof(u64) * (size_t)(M * K * w));
    u64 *b = (u64 *)malloc(sizeof(u64) * (size_t)(K * N * w));
    u64 *c = (u64 *)malloc(sizeof(u64) * (size_t)(M * N * w));
    orc_deal_shared(plo, phi, n, seed, K_MTRIPLE_A, sub, 0, M * K, alpha, NULL, Av, Am, a);
    orc_deal_shared(plo, phi, n, seed, K_MTRIPLE_B, sub, 0, K * N, alpha, NULL, Bv, Bm, b);
    matprod_ctx mc = {p, w, M, K, N, a, b, c};
    parallel_for(M * N, matprod_range, &mc);
    orc_deal_shared(plo, phi, n, seed, K_MTRIPLE_C, sub, 0, M * N, alpha, c, Cv, Cm, NULL);
    free(a); free(b); free(c);
}

/* ------------------------------------------------------------ LinearLayer
 * y = W x + b (Sec. III-D.3 "Data slicing" and "MPC-specific optimization";
 * the workload of Sec. IV): W is dout x din, row-major; its rows are cut into
 * tiles of R consecutive rows (the last tile may be shorter), T = ceil(dout/R).
 * Tile t has its own triple: A_t = rows of a dout x din matrix A (kind
 * MTRIPLE_A, element index row*din + col), B_t = din values (kind MTRIPLE_B,
 * index t*din + k) and C_t = A_t B_t (kind MTRIPLE_C, index = row).  The tile
 * opens E_t = x - B_t and D_t = W_t - A_t and every party computes
 *   z_i = C_i + D_t B_{t,i} + A_{t,i} E_t + [i = 0] D_t E_t
 *   gamma(z)_i = gamma(C)_i + D_t gamma(B)_{t,i} + gamma(A)_{t,i} E_t + alpha_i D_t E_t
 * and y_i = z_i + b_i (MAC shares likewise).  Opening order of the check log:
 * for t = 0..T-1, E_t (din values), then D_t row by row.  Shares are [n][.]:
 * W, A [n][dout*din], x [n][din], b, C, y [n][dout], B [n][T*din]. */
void orc_deal_matvec_triples(u64 plo, u64 phi, int n, u64 seed, u64 sub, int64_t dout, int64_t din, int64_t R,
                             const u64 *alpha, u64 *Av, u64 *Am, u64 *Bv, u64 *Bm, u64 *Cv, u64 *Cm) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    int64_t T = (dout + R - 1) / R;
    u64 *a = (u64 *)malloc(sizeof(u64) * (size_t)(dout * din * w));
    u64 *b = (u64 *)malloc(sizeof(u64) * (size_t)(T * din * w));
    u64 *c = (u64 *)malloc(sizeof(u64) * (size_t)(dout * w));
    orc_deal_shared(plo, phi, n, seed, K_MTRIPLE_A, sub, 0, dout * din, alpha, NULL, Av, Am, a);
    orc_deal_shared(plo, phi, n, seed, K_MTRIPLE_B, sub, 0, T * din, alpha, NULL, Bv, Bm, b);
    for (int64_t r = 0; r < dout; ++r) {
        int64_t t = r / R;
        u128 s = 0;
        for (int64_t k = 0; k < din; ++k)
            s = f_add(s, f_mul(ld(a, r * din + k, w), ld(b, t * din + k, w), p), p);
        st(c, r, w, s);
    }
    orc_deal_shared(plo, phi, n, seed, K_MTRIPLE_C, sub, 0, dout, alpha, c, Cv, Cm, NULL);
    free(a); free(b); free(c);
}

typedef struct {
    u128 p; int w, n; int64_t dout, din, R;
    const u64 *Wv, *Wm, *xv, *xm, *bv, *bm, *Av, *Am, *Bv, *Bm, *Cv, *Cm, *alpha_sh;
    const int64_t *rows; int64_t nrows;
    u64 *yv, *ym;                       /* [n][nrows] */
    u64 check_key; u64 j0;              /* rlc: coefficient key and index of the first opened value */
    u64 *rowA, *rowS;                   /* rlc partials: [dout], [n][dout] */
} ll_ctx;

/* E_t[k] (one opened value) and its MAC shares */
static u128 ll_e(const ll_ctx *c, int64_t t, int64_t k) {
    u128 e = 0;
    for (int i = 0; i < c->n; ++i)
        e = f_add(e, f_sub(ld(c->xv, (int64_t)i * c->din + k, c->w),
                           ld(c->Bv, (int64_t)i * ((c->dout + c->R - 1) / c->R) * c->din + t * c->din + k, c->w), c->p), c->p);
    return e;
}
static u128 ll_d(const ll_ctx *c, int64_t r, int64_t k) {
    u128 d = 0;
    const int64_t q = r * c->din + k, S = c->dout * c->din;
    for (int i = 0; i < c->n; ++i)
        d = f_add(d, f_sub(ld(c->Wv, (int64_t)i * S + q, c->w), ld(c->Av, (int64_t)i * S + q, c->w), c->p), c->p);
    return d;
}

static void ll_rows_range(void *vc, int64_t lo, int64_t hi) {
    const ll_ctx *c = (const ll_ctx *)vc;
    u128 p = c->p; int w = c->w, n = c->n;
    const int64_t din = c->din, S = c->dout * din, T = (c->dout + c->R - 1) / c->R;
    for (int64_t q = lo; q < hi; ++q) {
        const int64_t r = c->rows[q], t = r / c->R;
        u128 de = 0;
        for (int64_t k = 0; k < din; ++k) de = f_add(de, f_mul(ll_d(c, r, k), ll_e(c, t, k), p), p);
        for (int i = 0; i < n; ++i) {
            u128 z = ld(c->Cv, (int64_t)i * c->dout + r, w), gz = ld(c->Cm, (int64_t)i * c->dout + r, w);
            for (int64_t k = 0; k < din; ++k) {
                const u128 d = ll_d(c, r, k), e = ll_e(c, t, k);
                const int64_t qb = (int64_t)i * T * din + t * din + k, qa = (int64_t)i * S + r * din + k;
                z = f_add(z, f_add(f_mul(d, ld(c->Bv, qb, w), p), f_mul(ld(c->Av, qa, w), e, p), p), p);
                gz = f_add(gz, f_add(f_mul(d, ld(c->Bm, qb, w), p), f_mul(ld(c->Am, qa, w), e, p), p), p);
            }
            if (i == 0) z = f_add(z, de, p);
            gz = f_add(gz, f_mul(ld(c->alpha_sh, i, w), de, p), p);
            z = f_add(z, ld(c->bv, (int64_t)i * c->dout + r, w), p);
            gz = f_add(gz, ld(c->bm, (int64_t)i * c->dout + r, w), p);
            st(c->yv, (int64_t)i * c->nrows + q, w, z);
            st(c->ym, (int64_t)i * c->nrows + q, w, gz);
        }
    }
}

/* y for the listed rows only: yv, ym are [n][nrows]. */
void orc_linear_layer(u64 plo, u64 phi, int n, int64_t dout, int64_t din, int64_t R,
                      const u64 *Wv, const u64 *Wm, const u64 *xv, const u64 *xm, const u64 *bv, const u64 *bm,
                      const u64 *Av, const u64 *Am, const u64 *Bv, const u64 *Bm, const u64 *Cv, const u64 *Cm,
                      const u64 *alpha_sh, int64_t nrows, const int64_t *rows, u64 *yv, u64 *ym) {
    ll_ctx c = {0};
    c.p = mkp(plo, phi); c.w = words_of(c.p); c.n = n; c.dout = dout; c.din = din; c.R = R;
    c.Wv = Wv; c.Wm = Wm; c.xv = xv; c.xm = xm; c.bv = bv; c.bm = bm;
    c.Av = Av; c.Am = Am; c.Bv = Bv; c.Bm = Bm; c.Cv = Cv; c.Cm = Cm; c.alpha_sh = alpha_sh;
    c.rows = rows; c.nrows = nrows; c.yv = yv; c.ym = ym;
    parallel_for(nrows, ll_rows_range, &c);
}

/* The opened values in log order with their MAC shares: vals [m], macs
 * [n][m], m = T*din + dout*din (small layers: the whole log is stored). */
void orc_linear_open(u64 plo, u64 phi, int n, int64_t dout, int64_t din, int64_t R,
                     const u64 *Wv, const u64 *Wm, const u64 *xv, const u64 *xm,
                     const u64 *Av, const u64 *Am, const u64 *Bv, const u64 *Bm, u64 *vals, u64 *macs) {
    ll_ctx c = {0};
    c.p = mkp(plo, phi); c.w = words_of(c.p); c.n = n; c.dout = dout; c.din = din; c.R = R;
    c.Wv = Wv; c.Wm = Wm; c.xv = xv; c.xm = xm; c.Av = Av; c.Am = Am; c.Bv = Bv; c.Bm = Bm;
    const int64_t T = (dout + R - 1) / R, S = dout * din, m = T * din + S;
    int w = c.w;
    int64_t pos = 0;
    for (int64_t t = 0; t < T; ++t) {
        for (int64_t k = 0; k < din; ++k, ++pos) {
            st(vals, pos, w, ll_e(&c, t, k));
            for (int i = 0; i < n; ++i)
                st(macs, (int64_t)i * m + pos, w, f_sub(ld(xm, (int64_t)i * din + k, w),
                                                        ld(Bm, (int64_t)i * T * din + t * din + k, w), c.p));
        }
        const int64_t r1 = (t + 1) * R < dout ? (t + 1) * R : dout;
        for (int64_t r = t * R; r < r1; ++r)
            for (int64_t k = 0; k < din; ++k, ++pos) {
                st(vals, pos, w, ll_d(&c, r, k));
                for (int i = 0; i < n; ++i)
                    st(macs, (int64_t)i * m + pos, w, f_sub(ld(Wm, (int64_t)i * S + r * din + k, w),
                                                            ld(Am, (int64_t)i * S + r * din + k, w), c.p));
            }
    }
}

static void ll_rlc_range(void *vc, int64_t lo, int64_t hi) {
    const ll_ctx *c = (const ll_ctx *)vc;
    u128 p = c->p; int w = c->w, n = c->n;
    const int64_t din = c->din, R = c->R, S = c->dout * din, T = (c->dout + R - 1) / R;
    for (int64_t r = lo; r < hi; ++r) {
        /* row r of the log: position of D[r][0]; the tile's E precedes its rows */
        const int64_t t = r / R;
        const int64_t pos0 = t * (din + R * din) + din + (r - t * R) * din;
        u128 A = 0, Sv[64];
        for (int i = 0; i < n; ++i) Sv[i] = 0;
        for (int64_t k = 0; k < din; ++k) {
            const u128 rr = draw_elem(c->check_key, c->j0 + (u64)(pos0 + k), p);
            A = f_add(A, f_mul(rr, ll_d(c, r, k), p), p);
            for (int i = 0; i < n; ++i)
                Sv[i] = f_add(Sv[i], f_mul(rr, f_sub(ld(c->Wm, (int64_t)i * S + r * din + k, w),
                                                     ld(c->Am, (int64_t)i * S + r * din + k, w), p), p), p);
        }
        if (r == t * R) {   /* the first row of a tile also carries the tile's E */
            for (int64_t k = 0; k < din; ++k) {
                const u128 rr = draw_elem(c->check_key, c->j0 + (u64)(t * (din + R * din) + k), p);
                A = f_add(A, f_mul(rr, ll_e(c, t, k), p), p);
                for (int i = 0; i < n; ++i)
                    Sv[i] = f_add(Sv[i], f_mul(rr, f_sub(ld(c->xm, (int64_t)i * din + k, w),
                                                         ld(c->Bm, (int64_t)i * T * din + t * din + k, w), p), p), p);
            }
        }
        st(c->rowA, r, w, A);
        for (int i = 0; i < n; ++i) st(c->rowS, (int64_t)i * c->dout + r, w, Sv[i]);
    }
}

/* The check sums of the layer's log without storing it: A = sum r_j v_j and
 * S_i = sum r_j gamma_i(v_j), with r_j the epoch's coefficient of opened
 * value j0 + j (j in log order). */
void orc_linear_rlc(u64 plo, u64 phi, int n, int64_t dout, int64_t din, int64_t R,
                    const u64 *Wv, const u64 *Wm, const u64 *xv, const u64 *xm,
                    const u64 *Av, const u64 *Am, const u64 *Bv, const u64 *Bm,
                    u64 check_seed, u64 epoch, u64 j0, u64 *A_out, u64 *S_out) {
    ll_ctx c = {0};
    c.p = mkp(plo, phi); c.w = words_of(c.p); c.n = n; c.dout = dout; c.din = din; c.R = R;
    c.Wv = Wv; c.Wm = Wm; c.xv = xv; c.xm = xm; c.Av = Av; c.Am = Am; c.Bv = Bv; c.Bm = Bm;
    c.check_key = orc_stream_key(check_seed, orc_stream_id(K_CHECK, 0, 0, epoch));
    c.j0 = j0;
    int w = c.w;
    c.rowA = (u64 *)malloc(sizeof(u64) * (size_t)(dout * w));
    c.rowS = (u64 *)malloc(sizeof(u64) * (size_t)(n * dout * w));
    parallel_for(dout, ll_rlc_range, &c);
    u128 A = 0, Sv[64];
    for (int i = 0; i < n; ++i) Sv[i] = 0;
    for (int64_t r = 0; r < dout; ++r) {
        A = f_add(A, ld(c.rowA, r, w), c.p);
        for (int i = 0; i < n; ++i) Sv[i] = f_add(Sv[i], ld(c.rowS, (int64_t)i * dout + r, w), c.p);
    }
    st(A_out, 0, w, A);
    for (int i = 0; i < n; ++i) st(S_out, i, w, Sv[i]);
    free(c.rowA); free(c.rowS);
}

/* --------------------------------------------------------- input sharing
 * The owner of a private input x holds a dealer mask r in the clear, and the
 * parties hold a sharing [r] with MACs (kind INPUT_MASK, sub = the owner).
 * The owner publishes eps = x - r; every party sets [x] = [r] + eps: party 0
 * adds eps to its value share and every party adds alpha_i * eps to its MAC
 * share (the public-constant addition).  eps is public and is returned. */
void orc_input(u64 plo, u64 phi, int n, int64_t count, const u64 *x, const u64 *r_clear,
               const u64 *rv, const u64 *rm, const u64 *alpha_sh, u64 *outv, u64 *outm, u64 *eps) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    for (int64_t j = 0; j < count; ++j) {
        u128 e = f_sub(ld(x, j, w), ld(r_clear, j, w), p);
        st(eps, j, w, e);
        for (int i = 0; i < n; ++i) {
            int64_t q = (int64_t)i * count + j;
            u128 v = ld(rv, q, w);
            st(outv, q, w, i == 0 ? f_add(v, e, p) : v);
            st(outm, q, w, f_add(ld(rm, q, w), f_mul(ld(alpha_sh, i, w), e, p), p));
        }
    }
}

/* --------------------------------------------------------------------- DAG
 * A straight-line arithmetic circuit: gate g reads wires in0[g], in1[g] and
 * writes wire n_in + g.  Gates are evaluated in gate order; the t-th MUL gate
 * (in gate order) consumes triple t of the given triple arrays, and opens
 * eps_t and delta_t (log slots 2t and 2t+1 of the run's check).  Wires are
 * [n][W] with W = n_in + n_gates; the triple arrays are [n][T].  kconst holds
 * one field element per gate (used by CMUL and CADD).  eps/dlt are [n_mul]
 * and eps_mac/dlt_mac [n][n_mul], n_mul = number of MUL gates.
 */
typedef struct {
    u128 p; int w, n;
    int64_t n_in, W, T, n_mul;
    const uint8_t *ops; const uint32_t *in0, *in1;
    const u64 *kconst, *alpha_sh;
    u64 *wv, *wm;
    const u64 *av, *am, *bv, *bm, *cv, *cm;
    u64 *eps, *dlt, *eps_mac, *dlt_mac;
    const int64_t *mul_rank;     /* layer-parallel form: MUL rank of each gate */
    int64_t g0;                  /* layer-parallel form: first gate of the layer */
} dag_ctx;

/* Gate g; t = its MUL rank (the triple it consumes when it is a MUL gate). */
static void dag_gate(const dag_ctx *c, int64_t g, int64_t t) {
    u128 p = c->p; int w = c->w, n = c->n;
    int64_t W = c->W, T = c->T, n_mul = c->n_mul;
    int64_t out = c->n_in + g, a0 = c->in0[g], a1 = c->in1[g];
    int op = c->ops[g];
    u64 *wv = c->wv, *wm = c->wm;
    if (op == OP_MUL) {
        u128 d = 0, e = 0;
        for (int i = 0; i < n; ++i) {
            d = f_add(d, f_sub(ld(wv, i * W + a0, w), ld(c->av, i * T + t, w), p), p);
            e = f_add(e, f_sub(ld(wv, i * W + a1, w), ld(c->bv, i * T + t, w), p), p);
        }
        u128 de = f_mul(d, e, p);
        for (int i = 0; i < n; ++i) {
            int64_t q = i * T + t;
            u128 z = f_add(ld(c->cv, q, w), f_add(f_mul(d, ld(c->bv, q, w), p), f_mul(e, ld(c->av, q, w), p), p), p);
            if (i == 0) z = f_add(z, de, p);
            u128 gz = f_add(ld(c->cm, q, w), f_add(f_mul(d, ld(c->bm, q, w), p), f_mul(e, ld(c->am, q, w), p), p), p);
            gz = f_add(gz, f_mul(ld(c->alpha_sh, i, w), de, p), p);
            if (c->eps_mac) st(c->eps_mac, (int64_t)i * n_mul + t, w, f_sub(ld(wm, i * W + a0, w), ld(c->am, q, w), p));
            if (c->dlt_mac) st(c->dlt_mac, (int64_t)i * n_mul + t, w, f_sub(ld(wm, i * W + a1, w), ld(c->bm, q, w), p));
            st(wv, i * W + out, w, z);
            st(wm, i * W + out, w, gz);
        }
        if (c->eps) st(c->eps, t, w, d);
        if (c->dlt) st(c->dlt, t, w, e);
    } else {
        u128 k = ld(c->kconst, g, w);
        for (int i = 0; i < n; ++i) {
            u128 x = ld(wv, i * W + a0, w), gx = ld(wm, i * W + a0, w), z, gz;
            if (op == OP_ADD) {
                z = f_add(x, ld(wv, i * W + a1, w), p); gz = f_add(gx, ld(wm, i * W + a1, w), p);
            } else if (op == OP_SUB) {
                z = f_sub(x, ld(wv, i * W + a1, w), p); gz = f_sub(gx, ld(wm, i * W + a1, w), p);
            } else if (op == OP_CMUL) {
                z = f_mul(k, x, p); gz = f_mul(k, gx, p);
            } else {
                z = (i == 0) ? f_add(x, k, p) : x;
                gz = f_add(gx, f_mul(ld(c->alpha_sh, i, w), k, p), p);
            }
            st(wv, i * W + out, w, z);
            st(wm, i * W + out, w, gz);
        }
    }
}

static dag_ctx dag_ctx_make(u64 plo, u64 phi, int n, int64_t n_in, int64_t n_gates,
                            const uint8_t *ops, const uint32_t *in0, const uint32_t *in1,
                            const u64 *kconst, const u64 *alpha_sh, u64 *wv, u64 *wm,
                            int64_t T, const u64 *av, const u64 *am, const u64 *bv, const u64 *bm,
                            const u64 *cv, const u64 *cm, u64 *eps, u64 *dlt, u64 *eps_mac, u64 *dlt_mac) {
    dag_ctx c;
    c.p = mkp(plo, phi); c.w = words_of(c.p); c.n = n;
    c.n_in = n_in; c.W = n_in + n_gates; c.T = T;
    c.n_mul = 0;
    for (int64_t g = 0; g < n_gates; ++g) c.n_mul += (ops[g] == OP_MUL);
    c.ops = ops; c.in0 = in0; c.in1 = in1; c.kconst = kconst; c.alpha_sh = alpha_sh;
    c.wv = wv; c.wm = wm; c.av = av; c.am = am; c.bv = bv; c.bm = bm; c.cv = cv; c.cm = cm;
    c.eps = eps; c.dlt = dlt; c.eps_mac = eps_mac; c.dlt_mac = dlt_mac;
    c.mul_rank = NULL; c.g0 = 0;
    return c;
}

void orc_dag_eval(u64 plo, u64 phi, int n, int64_t n_in, int64_t n_gates,
                  const uint8_t *ops, const uint32_t *in0, const uint32_t *in1,
                  const u64 *kconst, const u64 *alpha_sh,
                  u64 *wv, u64 *wm,
                  int64_t T, const u64 *av, const u64 *am, const u64 *bv, const u64 *bm,
                  const u64 *cv, const u64 *cm,
                  u64 *eps, u64 *dlt, u64 *eps_mac, u64 *dlt_mac) {
    dag_ctx c = dag_ctx_make(plo, phi, n, n_in, n_gates, ops, in0, in1, kconst, alpha_sh, wv, wm, T,
                             av, am, bv, bm, cv, cm, eps, dlt, eps_mac, dlt_mac);
    int64_t t = 0;
    for (int64_t g = 0; g < n_gates; ++g) {
        dag_gate(&c, g, t);
        if (ops[g] == OP_MUL) ++t;
    }
}

static void dag_layer_range(void *ctx, int64_t lo, int64_t hi) {
    const dag_ctx *c = (const dag_ctx *)ctx;
    for (int64_t k = lo; k < hi; ++k) dag_gate(c, c->g0 + k, c->mul_rank[c->g0 + k]);
}

/* The same evaluation, layer by layer, with the gates of a layer spread over
 * the oracle's threads (layer l = gates [off[l], off[l+1])): a gate's triple
 * is still its MUL rank in gate order, so every share equals orc_dag_eval's.
 * Every operand of a layer's gates must be written before the layer (an
 * input or an earlier layer's output); returns -1 (nothing evaluated) when
 * one is not, 0 otherwise. */
int orc_dag_eval_layers(u64 plo, u64 phi, int n, int64_t n_in, int64_t n_gates, int depth,
                        const int64_t *layer_offsets,
                        const uint8_t *ops, const uint32_t *in0, const uint32_t *in1,
                        const u64 *kconst, const u64 *alpha_sh,
                        u64 *wv, u64 *wm,
                        int64_t T, const u64 *av, const u64 *am, const u64 *bv, const u64 *bm,
                        const u64 *cv, const u64 *cm,
                        u64 *eps, u64 *dlt, u64 *eps_mac, u64 *dlt_mac) {
    if (depth < 0 || layer_offsets[0] != 0 || layer_offsets[depth] != n_gates) return -1;
    for (int l = 0; l < depth; ++l) {
        if (layer_offsets[l + 1] < layer_offsets[l]) return -1;
        for (int64_t g = layer_offsets[l]; g < layer_offsets[l + 1]; ++g) {
            int binary = ops[g] == OP_ADD || ops[g] == OP_SUB || ops[g] == OP_MUL;
            if ((int64_t)in0[g] >= n_in + layer_offsets[l] || (binary && (int64_t)in1[g] >= n_in + layer_offsets[l]))
                return -1;
        }
    }
    int64_t *rank = (int64_t *)malloc((size_t)(n_gates > 0 ? n_gates : 1) * sizeof(int64_t));
    if (!rank) return -1;
    int64_t t = 0;
    for (int64_t g = 0; g < n_gates; ++g) {
        rank[g] = t;
        if (ops[g] == OP_MUL) ++t;
    }
    dag_ctx c = dag_ctx_make(plo, phi, n, n_in, n_gates, ops, in0, in1, kconst, alpha_sh, wv, wm, T,
                             av, am, bv, bm, cv, cm, eps, dlt, eps_mac, dlt_mac);
    c.mul_rank = rank;
    for (int l = 0; l < depth; ++l) {
        c.g0 = layer_offsets[l];
        parallel_for(layer_offsets[l + 1] - layer_offsets[l], dag_layer_range, &c);
    }
    free(rank);
    return 0;
}

/* Cleartext evaluation of the same circuit on the secrets, for the
 * end-to-end closed-form check reconstruct(outputs) == circuit(inputs). */
void orc_dag_clear(u64 plo, u64 phi, int64_t n_in, int64_t n_gates,
                   const uint8_t *ops, const uint32_t *in0, const uint32_t *in1,
                   const u64 *kconst, u64 *wires) {
    u128 p = mkp(plo, phi); int w = words_of(p);
    for (int64_t g = 0; g < n_gates; ++g) {
        u128 x = ld(wires, in0[g], w), y = ld(wires, in1[g], w), k = ld(kconst, g, w), z;
        switch (ops[g]) {
        case OP_ADD: z = f_add(x, y, p); break;
        case OP_SUB: z = f_sub(x, y, p); break;
        case OP_CMUL: z = f_mul(k, x, p); break;
        case OP_CADD: z = f_add(x, k, p); break;
        default: z = f_mul(x, y, p); break;
        }
        st(wires, n_in + g, w, z);
    }
}
