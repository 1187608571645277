/*
 * msat_oracle.c -- CPU oracle for the torchmSAT objective (arXiv 2402.03640).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * GPU library is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline / reference arm may load it.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only
 * through the seeded instance generator (synth/) and the arrays it returns.
 *
 * What it computes (paper section 4, "The Neural Network Architecture",
 * "Unsatisfiable Cores", "The Solving Process", Algorithm 1; setup in
 * section 5):
 *
 *   x in R^n                       relaxed variables, random start      (Sec. 4)
 *   t = tanh(e * x)                e is all-ones, so t = tanh(x)         (Sec. 4)
 *   f = t . W,  W[i][j] = +1 if x_i in c_j, -1 if not-x_i in c_j        (Sec. 4)
 *   x'_i = [x_i > 0]                de-relaxation                        (Sec. 4)
 *   clause j unsatisfied  <=>  no literal of c_j is true under x'       (Sec. 4,
 *       "Unsatisfiable Cores"; the printed test x'.W == s is read with
 *       x' mapped to +-1, see orc_cost_identity in the tests)
 *   cost = sum_j w_j [j unsat]     (w = 1: number of unsat clauses)     (Sec. 2)
 *   L = sum_{j in U} w_j f_j^2 / sum_{j in U} w_j                       (Sec. 4,
 *       MSE of f against zero over the unsatisfied clauses)
 *   Adam step on x (lr from the caller; the paper uses 1e-4)            (Sec. 5)
 *   Algorithm 1: evaluate x, keep the best assignment, loss, backprop,
 *       one optimizer step; a restart whose cost reaches 0 stops.
 *
 * Two arithmetic modes:
 *   mode 0 (FP64)       the plain definition in double precision, libm tanh,
 *                       sequential sums in clause order.  Tolerance anchor.
 *   mode 1 (FP32-canon) the same steps in float with a fixed, stated
 *                       rounding contract so a GPU trajectory can be
 *                       compared bit for bit:
 *       - tanh: own float routine (Cody-Waite range reduction of exp with a
 *         Taylor polynomial, tanh(a) = em1/(em1+2), em1 = e^{2|a|}-1).
 *       - every sum over clause literals or variable occurrences: terms
 *         in stored order, 32-term leaves summed left to right, leaves
 *         combined by the dyadic tree (split at the largest power of two
 *         below the leaf count).
 *       - g_j = ((float)w_j * f_j) * (2 / (float)N) for unsat j, else 0,
 *         N = W_U unless another normaliser is selected (orc_set_loss_norm).
 *       - grad_i = S_i * fmaf(-t_i, t_i, 1) with S_i the occurrence sum of
 *         +-g_j.
 *       - Adam per element: m = b1*m + (1-b1)*g; v = b2*v + ((1-b2)*g)*g;
 *         x = x - (a_t*m) / (sqrtf(v)*r_t + eps), a_t = lr/(1-b1^t),
 *         r_t = 1/sqrt(1-b2^t), b^t by repeated multiplication in double,
 *         every per-step scalar rounded once from double to float.
 *     Built with -ffp-contract=off: no multiply-add is fused unless written
 *     as fmaf().
 *
 * Initial x: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014; the constants of
 * the published splitmix64 generator), output number c = b*n + i of the
 * stream seeded with seed_x, k = top 24 bits, x = k * 2^-23 - 1 (exact in
 * float, in [-1, 1)).
 *
 * Literal input format: DIMACS integers, +(i+1) for x_i and -(i+1) for
 * not-x_i.  Clauses are canonicalised by dropping a literal equal to an
 * earlier literal of the same clause (W holds one entry per variable and
 * clause, Sec. 4); a clause with x and not-x is kept as is and can never be
 * unsatisfied.  Weights must be >= 1 (NULL means all 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------ CNF */

typedef struct {
    int32_t n;
    int64_t m;
    int64_t nnz;
    int64_t *off; /* m+1 */
    int32_t *var; /* nnz, 0-based variable */
    uint8_t *neg; /* nnz, 1 = negated literal */
    int64_t *w;   /* m, >= 1 */
    /* variable -> occurrence lists, occurrences in (clause, position) order */
    int64_t *voff; /* n+1 */
    int64_t *occ_clause;
    uint8_t *occ_neg;
} ocnf;

static void ocnf_free(ocnf *c)
{
    free(c->off);
    free(c->var);
    free(c->neg);
    free(c->w);
    free(c->voff);
    free(c->occ_clause);
    free(c->occ_neg);
    memset(c, 0, sizeof(*c));
}

/* Copy the clause set, drop repeated literals inside a clause, build the
 * per-variable occurrence lists. */
static int ocnf_build(ocnf *c, int32_t n, int64_t m, const int64_t *off, const int32_t *lits,
                      const int64_t *w)
{
    memset(c, 0, sizeof(*c));
    if (n < 0 || m < 0 || !off) return ORC_EINVAL;
    if (off[0] != 0) return ORC_EINVAL;
    for (int64_t j = 0; j < m; ++j)
        if (off[j + 1] < off[j]) return ORC_EINVAL;
    int64_t raw = off[m];
    if (raw > 0 && !lits) return ORC_EINVAL;
    for (int64_t q = 0; q < raw; ++q) {
        int32_t l = lits[q];
        if (l == 0 || l > n || l < -n) return ORC_EINVAL;
    }
    if (w)
        for (int64_t j = 0; j < m; ++j)
            if (w[j] < 1) return ORC_EINVAL;

    c->n = n;
    c->m = m;
    c->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    c->var = (int32_t *)malloc(sizeof(int32_t) * (size_t)(raw > 0 ? raw : 1));
    c->neg = (uint8_t *)malloc((size_t)(raw > 0 ? raw : 1));
    c->w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    c->voff = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!c->off || !c->var || !c->neg || !c->w || !c->voff) {
        ocnf_free(c);
        return ORC_ENOMEM;
    }
    int64_t q = 0;
    c->off[0] = 0;
    for (int64_t j = 0; j < m; ++j) {
        int64_t start = q;
        for (int64_t p = off[j]; p < off[j + 1]; ++p) {
            int32_t l = lits[p];
            int32_t v = (l > 0 ? l : -l) - 1;
            uint8_t ng = (uint8_t)(l < 0);
            int dup = 0;
            for (int64_t r = start; r < q; ++r)
                if (c->var[r] == v && c->neg[r] == ng) dup = 1;
            if (dup) continue;
            c->var[q] = v;
            c->neg[q] = ng;
            ++q;
        }
        c->off[j + 1] = q;
        c->w[j] = w ? w[j] : 1;
    }
    c->nnz = q;
    /* occurrence lists: count, prefix, fill in clause order */
    for (int64_t r = 0; r < q; ++r) c->voff[c->var[r] + 1] += 1;
    for (int32_t i = 0; i < n; ++i) c->voff[i + 1] += c->voff[i];
    c->occ_clause = (int64_t *)malloc(sizeof(int64_t) * (size_t)(q > 0 ? q : 1));
    c->occ_neg = (uint8_t *)malloc((size_t)(q > 0 ? q : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!c->occ_clause || !c->occ_neg || !fill) {
        free(fill);
        ocnf_free(c);
        return ORC_ENOMEM;
    }
    for (int32_t i = 0; i < n; ++i) fill[i] = c->voff[i];
    for (int64_t j = 0; j < m; ++j)
        for (int64_t r = c->off[j]; r < c->off[j + 1]; ++r) {
            int64_t slot = fill[c->var[r]]++;
            c->occ_clause[slot] = j;
            c->occ_neg[slot] = c->neg[r];
        }
    free(fill);
    return ORC_OK;
}

/* ------------------------------------------------------------ SplitMix64 */

static uint64_t sm64_output(uint64_t seed, uint64_t c)
{
    /* output number c (0-based) of the splitmix64 stream started at seed */
    uint64_t z = seed + (c + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t seed, uint64_t c) { return sm64_output(seed, c); }

/* Random start of Algorithm 1: uniform on the 2^24-point grid of [-1, 1).
 * Column b of x is restart b0 + b: output number (b0 + b) * n + i. */
static void init_x_from(int32_t n, int32_t B, int32_t b0, uint64_t seed, float *x)
{
    for (int32_t b = 0; b < B; ++b)
        for (int32_t i = 0; i < n; ++i) {
            uint64_t u = sm64_output(seed, (uint64_t)(b0 + b) * (uint64_t)n + (uint64_t)i);
            float k = (float)(uint32_t)(u >> 40);
            x[(int64_t)i * B + b] = k * 0x1p-23f - 1.0f;
        }
}

int orc_init_x(int32_t n, int32_t B, uint64_t seed, float *x /* [n][B] */)
{
    if (n < 0 || B < 1 || (n > 0 && !x)) return ORC_EINVAL;
    init_x_from(n, B, 0, seed, x);
    return ORC_OK;
}

/* ------------------------------------------------------- FP32-canon tanh */

/* e^y - 1 for 0 <= y <= 18, float, Cody-Waite reduction y = k ln2 + r,
 * |r| <= ln2/2, e^r - 1 = r + r^2 * sum_{i>=2} r^{i-2}/i! (Taylor to r^8). */
static float canon_expm1(float y)
{
    const float inv_ln2 = 1.44269504088896341f;
    const float ln2_hi = 0.693145751953125f;         /* 0x3F317200: 16 trailing zero bits */
    const float ln2_lo = 1.428606820309417232e-06f;  /* ln2 - ln2_hi */
    float kf = rintf(y * inv_ln2);
    float r = fmaf(-kf, ln2_hi, y);
    r = fmaf(-kf, ln2_lo, r);
    /* Taylor coefficients 1/i!, i = 2..8, Horner from the top */
    float q = 1.0f / 40320.0f;
    q = fmaf(q, r, 1.0f / 5040.0f);
    q = fmaf(q, r, 1.0f / 720.0f);
    q = fmaf(q, r, 1.0f / 120.0f);
    q = fmaf(q, r, 1.0f / 24.0f);
    q = fmaf(q, r, 1.0f / 6.0f);
    q = fmaf(q, r, 0.5f);
    float rr = r * r;
    float pm1 = fmaf(rr, q, r); /* e^r - 1 */
    int k = (int)kf;
    if (k == 0) return pm1;
    /* 2^k as float from its exponent field; k in [1, 26] here */
    uint32_t bits = (uint32_t)(127 + k) << 23;
    float scale;
    memcpy(&scale, &bits, sizeof(scale));
    return fmaf(scale, pm1, scale - 1.0f);
}

float orc_tanh32(float a)
{
    float s = fabsf(a);
    float r;
    if (!(s < 9.0f)) {
        r = (s != s) ? s : 1.0f; /* NaN stays NaN */
    } else {
        float em1 = canon_expm1(s + s);
        r = em1 / (em1 + 2.0f);
    }
    return copysignf(r, a);
}

/* ------------------------------------------------- FP32-canon summation */

/* Terms in order; 32-term leaves summed left to right; leaves combined by
 * the dyadic tree (a leaf count K splits into the largest power of two
 * below K and the rest).  The stack below holds finished dyadic blocks;
 * what is left at the end is combined right to left, which is the same
 * tree. */
static float canon_sum(const float *a, int64_t L)
{
    if (L <= 0) return 0.0f;
    float blk[64];
    int64_t sz[64];
    int top = 0;
    for (int64_t lo = 0; lo < L; lo += 32) {
        int64_t hi = lo + 32 < L ? lo + 32 : L;
        float s = a[lo];
        for (int64_t k = lo + 1; k < hi; ++k) s = s + a[k];
        blk[top] = s;
        sz[top] = 1;
        ++top;
        while (top >= 2 && sz[top - 1] == sz[top - 2]) {
            blk[top - 2] = blk[top - 2] + blk[top - 1];
            sz[top - 2] *= 2;
            --top;
        }
    }
    float r = blk[top - 1];
    for (int q = top - 2; q >= 0; --q) r = blk[q] + r;
    return r;
}

float orc_canon_sum(const float *a, int64_t L) { return canon_sum(a, L); }

/* -------------------------------------------------------- exact cost */

/* literal true under the 0/1 assignment a */
static int lit_true(uint8_t neg, uint8_t a) { return (a != 0) != (neg != 0); }

/* cost_b = sum_j w_j [no literal of c_j is true under assign[b]] */
int orc_cost(int32_t n, int64_t m, const int64_t *off, const int32_t *lits, const int64_t *w,
             int32_t B, const uint8_t *assign /* [B][n] 0/1 */, int64_t *cost /* [B] */)
{
    ocnf c;
    int rc = ocnf_build(&c, n, m, off, lits, w);
    if (rc) return rc;
    for (int32_t b = 0; b < B; ++b) {
        const uint8_t *a = assign + (int64_t)b * n;
        int64_t total = 0;
        for (int64_t j = 0; j < c.m; ++j) {
            int sat = 0;
            for (int64_t r = c.off[j]; r < c.off[j + 1]; ++r)
                if (lit_true(c.neg[r], a[c.var[r]])) sat = 1;
            if (!sat) total += c.w[j];
        }
        cost[b] = total;
    }
    ocnf_free(&c);
    return ORC_OK;
}

/* ------------------------------------------------- loss normaliser */

/* Normaliser N of L = sum_{j in U} w_j f_j^2 / N and g_j = 2 w_j f_j / N.
 * Sec. 4 takes the MSE of f against zero over the unsatisfied clauses, read
 * as N = W_U = sum_{j in U} w_j (mode 0, the default).  Mode 1 (N = 1, the
 * sum) and mode 2 (N = total weight, the mean over all clauses) are the
 * other readings, for the ablation.  Set by orc_set_loss_norm. */
static int g_loss_norm = 0;

int orc_set_loss_norm(int32_t mode)
{
    if (mode < 0 || mode > 2) return ORC_EINVAL;
    g_loss_norm = mode;
    return ORC_OK;
}

static int64_t total_weight(const ocnf *c)
{
    int64_t s = 0;
    for (int64_t j = 0; j < c->m; ++j) s += c->w[j];
    return s;
}

/* N in double (FP64 mode) and in float (FP32-canon: (float) of the integer) */
static double norm_f64(int64_t wu, int64_t wsum)
{
    return g_loss_norm == 1 ? 1.0 : (double)(g_loss_norm == 2 ? wsum : wu);
}

static float norm_f32(int64_t wu, int64_t wsum)
{
    return g_loss_norm == 1 ? 1.0f : (float)(g_loss_norm == 2 ? wsum : wu);
}

/* ------------------------------------------------------ FP64 objective */

/* One evaluation of the relaxed objective at x (double, [n][B]):
 * f [m][B], unsat [m][B], cost [B], loss [B], grad [n][B] (any may be NULL
 * except cost and loss). */
static void objective_f64(const ocnf *c, int32_t B, const double *x, double *f_out,
                          uint8_t *unsat_out, int64_t *cost, double *loss, double *grad,
                          double *t, double *f, uint8_t *u)
{
    const int32_t n = c->n;
    const int64_t wsum = total_weight(c);
    for (int64_t q = 0; q < (int64_t)n * B; ++q) t[q] = tanh(x[q]);
    for (int32_t b = 0; b < B; ++b) {
        int64_t wu = 0;
        double num = 0.0;
        for (int64_t j = 0; j < c->m; ++j) {
            double fj = 0.0;
            int sat = 0;
            for (int64_t r = c->off[j]; r < c->off[j + 1]; ++r) {
                int64_t q = (int64_t)c->var[r] * B + b;
                fj += c->neg[r] ? -t[q] : t[q];
                if (lit_true(c->neg[r], (uint8_t)(x[q] > 0.0))) sat = 1;
            }
            f[j * B + b] = fj;
            u[j * B + b] = (uint8_t)!sat;
            if (!sat) {
                wu += c->w[j];
                num += (double)c->w[j] * fj * fj;
            }
        }
        cost[b] = wu;
        loss[b] = wu > 0 ? num / norm_f64(wu, wsum) : 0.0;
        if (grad) {
            for (int32_t i = 0; i < n; ++i) grad[(int64_t)i * B + b] = 0.0;
            if (wu > 0) {
                /* dL/dt_i = sum over unsat j containing i of sign * 2 w_j f_j / N */
                for (int64_t j = 0; j < c->m; ++j) {
                    if (!u[j * B + b]) continue;
                    double g = 2.0 * (double)c->w[j] * f[j * B + b] / norm_f64(wu, wsum);
                    for (int64_t r = c->off[j]; r < c->off[j + 1]; ++r) {
                        int64_t q = (int64_t)c->var[r] * B + b;
                        grad[q] += c->neg[r] ? -g : g;
                    }
                }
                for (int32_t i = 0; i < n; ++i) {
                    int64_t q = (int64_t)i * B + b;
                    grad[q] *= 1.0 - t[q] * t[q];
                }
            }
        }
    }
    if (f_out) memcpy(f_out, f, sizeof(double) * (size_t)(c->m * B));
    if (unsat_out) memcpy(unsat_out, u, (size_t)(c->m * B));
}

int orc_objective_f64(int32_t n, int64_t m, const int64_t *off, const int32_t *lits,
                      const int64_t *w, int32_t B, const double *x, double *f_out,
                      uint8_t *unsat_out, int64_t *cost, double *loss, double *grad)
{
    if (B < 1 || !cost || !loss) return ORC_EINVAL;
    ocnf c;
    int rc = ocnf_build(&c, n, m, off, lits, w);
    if (rc) return rc;
    double *t = (double *)malloc(sizeof(double) * (size_t)((int64_t)n * B + 1));
    double *f = (double *)malloc(sizeof(double) * (size_t)(c.m * B + 1));
    uint8_t *u = (uint8_t *)malloc((size_t)(c.m * B + 1));
    if (!t || !f || !u) {
        free(t);
        free(f);
        free(u);
        ocnf_free(&c);
        return ORC_ENOMEM;
    }
    objective_f64(&c, B, x, f_out, unsat_out, cost, loss, grad, t, f, u);
    free(t);
    free(f);
    free(u);
    ocnf_free(&c);
    return ORC_OK;
}

/* ------------------------------------------------ FP32-canon objective */

typedef struct {
    float *t;      /* [n][B] */
    float *f;      /* [m][B] */
    uint8_t *u;    /* [m][B] */
    float *terms;  /* max(max clause length, max degree) */
    float *g;      /* [m][B] */
} work32;

static int work32_alloc(work32 *wk, const ocnf *c, int32_t B)
{
    int64_t maxlen = 1;
    for (int64_t j = 0; j < c->m; ++j)
        if (c->off[j + 1] - c->off[j] > maxlen) maxlen = c->off[j + 1] - c->off[j];
    for (int32_t i = 0; i < c->n; ++i)
        if (c->voff[i + 1] - c->voff[i] > maxlen) maxlen = c->voff[i + 1] - c->voff[i];
    wk->t = (float *)malloc(sizeof(float) * (size_t)((int64_t)c->n * B + 1));
    wk->f = (float *)malloc(sizeof(float) * (size_t)(c->m * B + 1));
    wk->u = (uint8_t *)malloc((size_t)(c->m * B + 1));
    wk->terms = (float *)malloc(sizeof(float) * (size_t)maxlen);
    wk->g = (float *)malloc(sizeof(float) * (size_t)(c->m * B + 1));
    if (!wk->t || !wk->f || !wk->u || !wk->terms || !wk->g) return ORC_ENOMEM;
    return ORC_OK;
}

static void work32_free(work32 *wk)
{
    free(wk->t);
    free(wk->f);
    free(wk->u);
    free(wk->terms);
    free(wk->g);
}

/* Evaluate x (float): t, f, unsat, cost, and loss (reported in double from
 * the float f).  Then, if grad is non-NULL, the canonical float gradient. */
static void objective_f32(const ocnf *c, int32_t B, const float *x, work32 *wk, int64_t *cost,
                          double *loss, float *grad)
{
    const int32_t n = c->n;
    const int64_t wsum = total_weight(c);
    for (int64_t q = 0; q < (int64_t)n * B; ++q) wk->t[q] = orc_tanh32(x[q]);
    for (int32_t b = 0; b < B; ++b) {
        int64_t wu = 0;
        double num = 0.0;
        for (int64_t j = 0; j < c->m; ++j) {
            int64_t L = 0;
            int sat = 0;
            for (int64_t r = c->off[j]; r < c->off[j + 1]; ++r) {
                int64_t q = (int64_t)c->var[r] * B + b;
                float tv = wk->t[q];
                wk->terms[L++] = c->neg[r] ? -tv : tv;
                if (lit_true(c->neg[r], (uint8_t)(x[q] > 0.0f))) sat = 1;
            }
            float fj = canon_sum(wk->terms, L);
            wk->f[j * B + b] = fj;
            wk->u[j * B + b] = (uint8_t)!sat;
            if (!sat) {
                wu += c->w[j];
                num += (double)c->w[j] * (double)fj * (double)fj;
            }
        }
        cost[b] = wu;
        loss[b] = wu > 0 ? num / norm_f64(wu, wsum) : 0.0;
        if (!grad) continue;
        float cb = wu > 0 ? 2.0f / norm_f32(wu, wsum) : 0.0f;
        for (int64_t j = 0; j < c->m; ++j)
            wk->g[j * B + b] = wk->u[j * B + b] ? ((float)c->w[j] * wk->f[j * B + b]) * cb : 0.0f;
        for (int32_t i = 0; i < n; ++i) {
            int64_t L = 0;
            for (int64_t s = c->voff[i]; s < c->voff[i + 1]; ++s) {
                int64_t j = c->occ_clause[s];
                float g = wk->u[j * B + b] ? wk->g[j * B + b] : 0.0f;
                wk->terms[L++] = (wk->u[j * B + b] && c->occ_neg[s]) ? -g : g;
            }
            float S = canon_sum(wk->terms, L);
            float tv = wk->t[(int64_t)i * B + b];
            grad[(int64_t)i * B + b] = S * fmaf(-tv, tv, 1.0f);
        }
    }
}

int orc_objective_f32(int32_t n, int64_t m, const int64_t *off, const int32_t *lits,
                      const int64_t *w, int32_t B, const float *x, float *f_out,
                      uint8_t *unsat_out, int64_t *cost, double *loss, float *grad)
{
    if (B < 1 || !cost || !loss) return ORC_EINVAL;
    ocnf c;
    int rc = ocnf_build(&c, n, m, off, lits, w);
    if (rc) return rc;
    work32 wk;
    memset(&wk, 0, sizeof(wk));
    rc = work32_alloc(&wk, &c, B);
    if (!rc) {
        objective_f32(&c, B, x, &wk, cost, loss, grad);
        if (f_out) memcpy(f_out, wk.f, sizeof(float) * (size_t)(c.m * B));
        if (unsat_out) memcpy(unsat_out, wk.u, (size_t)(c.m * B));
    }
    work32_free(&wk);
    ocnf_free(&c);
    return rc;
}

/* ------------------------------------------------------- Algorithm 1 */

typedef struct {
    double lr, beta1, beta2, eps;
} orc_adam;

/* Per-step float scalars of the canonical Adam update for step t >= 1. */
static void adam_scalars(const orc_adam *h, int64_t t, float *a_t, float *r_t)
{
    double p1 = 1.0, p2 = 1.0;
    for (int64_t s = 0; s < t; ++s) {
        p1 *= h->beta1;
        p2 *= h->beta2;
    }
    *a_t = (float)(h->lr / (1.0 - p1));
    *r_t = (float)(1.0 / sqrt(1.0 - p2));
}

/*
 * One iteration of Algorithm 1 in FP32-canon arithmetic, on the state
 * (x, mom, vel) [n][B] with `steps_done` optimizer steps already taken:
 *   evaluate x (cost, loss)            Algorithm 1, evaluation
 *   best update (strict <)             Algorithm 1, best kept
 *   if cost == 0 the restart has stopped: no update (Algorithm 1 stops at zero)
 *   else gradient + one Adam step      Algorithm 1, backpropagation and update
 * If `update` is 0 only the evaluation and best update run (the final
 * evaluation after the last step).  best_assign may be NULL.
 */
int orc_step32(int32_t n, int64_t m, const int64_t *off, const int32_t *lits, const int64_t *w,
               int32_t B, float *x, float *mom, float *vel, int64_t steps_done, double lr,
               double beta1, double beta2, double eps, int32_t update, int64_t *best_cost,
               uint8_t *best_assign, int64_t *cost, double *loss, float *grad_out)
{
    if (B < 1 || !x || !cost || !loss || !best_cost) return ORC_EINVAL;
    ocnf c;
    int rc = ocnf_build(&c, n, m, off, lits, w);
    if (rc) return rc;
    work32 wk;
    memset(&wk, 0, sizeof(wk));
    float *grad = (float *)malloc(sizeof(float) * (size_t)((int64_t)n * B + 1));
    rc = work32_alloc(&wk, &c, B);
    if (!rc && !grad) rc = ORC_ENOMEM;
    if (!rc) {
        objective_f32(&c, B, x, &wk, cost, loss, update ? grad : NULL);
        for (int32_t b = 0; b < B; ++b) {
            if (cost[b] < best_cost[b]) {
                best_cost[b] = cost[b];
                if (best_assign)
                    for (int32_t i = 0; i < n; ++i)
                        best_assign[(int64_t)b * n + i] = (uint8_t)(x[(int64_t)i * B + b] > 0.0f);
            }
        }
        if (update) {
            orc_adam h = {lr, beta1, beta2, eps};
            float a_t, r_t;
            adam_scalars(&h, steps_done + 1, &a_t, &r_t);
            const float b1 = (float)beta1, b2 = (float)beta2;
            const float omb1 = (float)(1.0 - beta1), omb2 = (float)(1.0 - beta2);
            const float epsf = (float)eps;
            for (int32_t b = 0; b < B; ++b) {
                if (cost[b] == 0) continue; /* stopped restart */
                for (int32_t i = 0; i < n; ++i) {
                    int64_t q = (int64_t)i * B + b;
                    float g = grad[q];
                    float mq = b1 * mom[q] + omb1 * g;
                    float vq = b2 * vel[q] + (omb2 * g) * g;
                    float den = sqrtf(vq) * r_t + epsf;
                    mom[q] = mq;
                    vel[q] = vq;
                    x[q] = x[q] - (a_t * mq) / den;
                }
            }
            if (grad_out) memcpy(grad_out, grad, sizeof(float) * (size_t)((int64_t)n * B));
        }
    }
    free(grad);
    work32_free(&wk);
    ocnf_free(&c);
    return rc;
}

/*
 * Algorithm 1 with a fixed number of steps in place of the time limit T,
 * followed by one evaluation of the final x.
 *   mode 0: FP64 definition;  mode 1: FP32-canon.
 * Outputs (each may be NULL except best_cost):
 *   cost_hist [steps+1][B]   cost of x_0 .. x_steps
 *   loss_hist [steps][B]     loss at x_0 .. x_{steps-1}
 *   best_cost [B], best_assign [B][n]
 *   x_final [n][B] (as double)
 */
static int solve_from(int32_t n, int64_t m, const int64_t *off, const int32_t *lits, const int64_t *w,
                      int32_t B, int32_t b0, uint64_t seed_x, double lr, double beta1, double beta2,
                      double eps, int32_t steps, int32_t mode, int64_t *cost_hist, double *loss_hist,
                      int64_t *best_cost, uint8_t *best_assign, double *x_final);

int orc_solve(int32_t n, int64_t m, const int64_t *off, const int32_t *lits, const int64_t *w,
              int32_t B, uint64_t seed_x, double lr, double beta1, double beta2, double eps,
              int32_t steps, int32_t mode, int64_t *cost_hist, double *loss_hist,
              int64_t *best_cost, uint8_t *best_assign, double *x_final)
{
    return solve_from(n, m, off, lits, w, B, 0, seed_x, lr, beta1, beta2, eps, steps, mode,
                      cost_hist, loss_hist, best_cost, best_assign, x_final);
}

/* The same for restarts b0 .. b0 + B - 1 of a larger run: restarts never
 * interact (each has its own x, moments, cost and best), so a run of B'
 * restarts equals the column-wise union of runs over any split of them. */
int orc_solve_from(int32_t n, int64_t m, const int64_t *off, const int32_t *lits, const int64_t *w,
                   int32_t B, int32_t b0, uint64_t seed_x, double lr, double beta1, double beta2,
                   double eps, int32_t steps, int32_t mode, int64_t *cost_hist, double *loss_hist,
                   int64_t *best_cost, uint8_t *best_assign, double *x_final)
{
    if (b0 < 0) return ORC_EINVAL;
    return solve_from(n, m, off, lits, w, B, b0, seed_x, lr, beta1, beta2, eps, steps, mode,
                      cost_hist, loss_hist, best_cost, best_assign, x_final);
}

static int solve_from(int32_t n, int64_t m, const int64_t *off, const int32_t *lits, const int64_t *w,
                      int32_t B, int32_t b0, uint64_t seed_x, double lr, double beta1, double beta2,
                      double eps, int32_t steps, int32_t mode, int64_t *cost_hist, double *loss_hist,
                      int64_t *best_cost, uint8_t *best_assign, double *x_final)
{
    if (B < 1 || steps < 0 || !best_cost || (mode != 0 && mode != 1)) return ORC_EINVAL;
    ocnf c;
    int rc = ocnf_build(&c, n, m, off, lits, w);
    if (rc) return rc;
    const int64_t nb = (int64_t)n * B;
    int64_t wsum = 0;
    for (int64_t j = 0; j < c.m; ++j) wsum += c.w[j];
    for (int32_t b = 0; b < B; ++b) best_cost[b] = wsum; /* Algorithm 1 starts from the total weight */
    int64_t *cost = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    double *loss = (double *)malloc(sizeof(double) * (size_t)B);
    float *x0 = (float *)malloc(sizeof(float) * (size_t)(nb + 1));
    if (!cost || !loss || !x0) {
        rc = ORC_ENOMEM;
        goto done;
    }
    init_x_from(n, B, b0, seed_x, x0);

    if (mode == 0) {
        double *x = (double *)malloc(sizeof(double) * (size_t)(nb + 1));
        double *mo = (double *)calloc((size_t)(nb + 1), sizeof(double));
        double *ve = (double *)calloc((size_t)(nb + 1), sizeof(double));
        double *gr = (double *)malloc(sizeof(double) * (size_t)(nb + 1));
        double *t = (double *)malloc(sizeof(double) * (size_t)(nb + 1));
        double *f = (double *)malloc(sizeof(double) * (size_t)(c.m * B + 1));
        uint8_t *u = (uint8_t *)malloc((size_t)(c.m * B + 1));
        if (!x || !mo || !ve || !gr || !t || !f || !u) {
            rc = ORC_ENOMEM;
        } else {
            for (int64_t q = 0; q < nb; ++q) x[q] = (double)x0[q];
            double p1 = 1.0, p2 = 1.0;
            for (int32_t s = 0; s <= steps; ++s) {
                int upd = s < steps;
                objective_f64(&c, B, x, NULL, NULL, cost, loss, upd ? gr : NULL, t, f, u);
                if (cost_hist)
                    for (int32_t b = 0; b < B; ++b) cost_hist[(int64_t)s * B + b] = cost[b];
                if (loss_hist && upd)
                    for (int32_t b = 0; b < B; ++b) loss_hist[(int64_t)s * B + b] = loss[b];
                for (int32_t b = 0; b < B; ++b)
                    if (cost[b] < best_cost[b]) {
                        best_cost[b] = cost[b];
                        if (best_assign)
                            for (int32_t i = 0; i < n; ++i)
                                best_assign[(int64_t)b * n + i] = (uint8_t)(x[(int64_t)i * B + b] > 0.0);
                    }
                if (!upd) break;
                p1 *= beta1;
                p2 *= beta2;
                for (int32_t b = 0; b < B; ++b) {
                    if (cost[b] == 0) continue;
                    for (int32_t i = 0; i < n; ++i) {
                        int64_t q = (int64_t)i * B + b;
                        double g = gr[q];
                        mo[q] = beta1 * mo[q] + (1.0 - beta1) * g;
                        ve[q] = beta2 * ve[q] + (1.0 - beta2) * g * g;
                        double mh = mo[q] / (1.0 - p1);
                        double vh = ve[q] / (1.0 - p2);
                        x[q] -= lr * mh / (sqrt(vh) + eps);
                    }
                }
            }
            if (x_final) memcpy(x_final, x, sizeof(double) * (size_t)nb);
        }
        free(x);
        free(mo);
        free(ve);
        free(gr);
        free(t);
        free(f);
        free(u);
    } else {
        float *mo = (float *)calloc((size_t)(nb + 1), sizeof(float));
        float *ve = (float *)calloc((size_t)(nb + 1), sizeof(float));
        float *gr = (float *)malloc(sizeof(float) * (size_t)(nb + 1));
        work32 wk;
        memset(&wk, 0, sizeof(wk));
        int arc = work32_alloc(&wk, &c, B);
        if (!mo || !ve || !gr || arc) {
            rc = ORC_ENOMEM;
        } else {
            const float b1 = (float)beta1, b2 = (float)beta2;
            const float omb1 = (float)(1.0 - beta1), omb2 = (float)(1.0 - beta2);
            const float epsf = (float)eps;
            orc_adam h = {lr, beta1, beta2, eps};
            for (int32_t s = 0; s <= steps; ++s) {
                int upd = s < steps;
                objective_f32(&c, B, x0, &wk, cost, loss, upd ? gr : NULL);
                if (cost_hist)
                    for (int32_t b = 0; b < B; ++b) cost_hist[(int64_t)s * B + b] = cost[b];
                if (loss_hist && upd)
                    for (int32_t b = 0; b < B; ++b) loss_hist[(int64_t)s * B + b] = loss[b];
                for (int32_t b = 0; b < B; ++b)
                    if (cost[b] < best_cost[b]) {
                        best_cost[b] = cost[b];
                        if (best_assign)
                            for (int32_t i = 0; i < n; ++i)
                                best_assign[(int64_t)b * n + i] = (uint8_t)(x0[(int64_t)i * B + b] > 0.0f);
                    }
                if (!upd) break;
                float a_t, r_t;
                adam_scalars(&h, (int64_t)s + 1, &a_t, &r_t);
                for (int32_t b = 0; b < B; ++b) {
                    if (cost[b] == 0) continue;
                    for (int32_t i = 0; i < n; ++i) {
                        int64_t q = (int64_t)i * B + b;
                        float g = gr[q];
                        float mq = b1 * mo[q] + omb1 * g;
                        float vq = b2 * ve[q] + (omb2 * g) * g;
                        float den = sqrtf(vq) * r_t + epsf;
                        mo[q] = mq;
                        ve[q] = vq;
                        x0[q] = x0[q] - (a_t * mq) / den;
                    }
                }
            }
            if (x_final)
                for (int64_t q = 0; q < nb; ++q) x_final[q] = (double)x0[q];
        }
        free(mo);
        free(ve);
        free(gr);
        work32_free(&wk);
    }
done:
    free(cost);
    free(loss);
    free(x0);
    ocnf_free(&c);
    return rc;
}
