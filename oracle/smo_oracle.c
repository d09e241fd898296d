/*
 * FP64 reference implementation of the SVM training method of
 * "Fast Support Vector Machines Using Parallel Adaptive Shrinking on
 * Distributed Systems" (arXiv:1406.5161).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the oracle that the CUDA library is
 * checked against. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it; the library itself never does. It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Everything is plain, sequential-order FP64 arithmetic on the float32 input
 * values. Threads (OpenMP) only split independent per-row loops; every
 * reduction is merged in a fixed order, so results do not depend on the
 * thread count.
 *
 * Contents and the passage each function follows:
 *   or_dot            Algorithm 2 (merge-style inner product of two CSR rows)
 *   or_kernel         RBF kernel exp(-gamma * ||x - z||^2), distance from
 *                     ||x||^2 + ||z||^2 - 2<x,z> (Section IV-E, Eq. for the
 *                     Gaussian kernel in Section V-A, gamma = 1/(2 sigma^2));
 *                     or, selected by or_set_kernel, one of the other standard
 *                     kernels that Section V calls straightforward to use:
 *                     linear <x,z>, polynomial (gamma <x,z> + coef0)^degree,
 *                     sigmoid tanh(gamma <x,z> + coef0)
 *   or_smo            Algorithm 1: Keerthi's modification 2 SMO without
 *                     shrinking; Eqs. (fcache), (fup), (setinfo), (bminmax),
 *                     (kktterm), (alphaup), (rho); threshold beta of Sec. III-A
 *   or_smo_wss2       or_smo with a second-order choice of i_low (the
 *                     working-set selection the paper leaves to future work,
 *                     Section VI): i_up as in Eq. (bminmax); i_low maximises
 *                     (f_t - f_up)^2 / (K_uu + K_tt - 2 K_ut) over t in I_low
 *                     with f_t > f_up (Fan, Chen and Lin, JMLR 2005); same
 *                     stopping rule (kktterm)
 *   or_smo_shrink     Algorithms 4 and 5 (adaptive shrinking, Eq. (shrink),
 *                     shrink counter heuristics of Sec. III-C and Table 3)
 *                     with single or multiple gradient reconstructions
 *                     (Algorithm 6); wss = 2 takes i_low by the
 *                     second-order rule over the active rows (the future
 *                     work of Section VI) while the shrink rule and the
 *                     stopping tests keep the first-order b_up / b_low
 *   or_reconstruct    Algorithm 6 (gradient reconstruction of given samples)
 *   or_gradient       Eq. (fcache) evaluated from scratch
 *   or_decision       Eq. (classi) without the sign: sum_j a_j y_j K(x_j,z) - b
 *
 * Readings of the paper that the code takes where it is silent or garbled
 * (kept identical in the CUDA path, which implements them independently):
 *   - pair selection follows Eq. (bminmax): i_up = argmin f over
 *     I0 u I1 u I2, i_low = argmax f over I0 u I3 u I4, lowest index on ties;
 *     the initial pair falls out of this rule at alpha = 0.
 *   - the alpha step (Eq. alphaup with rho = -eta) is clipped jointly to the
 *     segment [L, H] that keeps sum y alpha = 0 and 0 <= alpha <= C; when
 *     eta <= 1e-12 the end point with the larger objective is taken
 *     (Platt's rule for a flat curvature, Sec. III-A).
 *   - alpha within 1e-12*C of 0 or C is set exactly to the bound, so the
 *     index sets of Eq. (setinfo) are decided by exact comparisons.
 *   - Eq. (fup) sums both terms (its '+' is missing in the text).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n, d;
    const int64_t *indptr;  /* n + 1 */
    const int32_t *indices; /* nnz, sorted within a row */
    const float *values;    /* nnz */
} or_csr;

enum { OR_SET_I0 = 0, OR_SET_I1 = 1, OR_SET_I2 = 2, OR_SET_I3 = 3, OR_SET_I4 = 4 };

/* ---------------------------------------------------------------- kernel */

/* Algorithm 2: walk both sorted index lists, multiply values where the
 * column indices are equal (the garbled test "|x[s1]-y[s2]| < 0" read as
 * equality), advance the list with the smaller index otherwise. */
double or_dot(const or_csr *A, int64_t i, const or_csr *B, int64_t j)
{
    int64_t s1 = A->indptr[i], e1 = A->indptr[i + 1];
    int64_t s2 = B->indptr[j], e2 = B->indptr[j + 1];
    double dp = 0.0;
    while (s1 < e1 && s2 < e2) {
        int32_t c1 = A->indices[s1], c2 = B->indices[s2];
        if (c1 == c2) {
            dp += (double)A->values[s1] * (double)B->values[s2];
            ++s1;
            ++s2;
        } else if (c1 < c2) {
            ++s1;
        } else {
            ++s2;
        }
    }
    return dp;
}

double or_sqnorm(const or_csr *A, int64_t i)
{
    double s = 0.0;
    for (int64_t k = A->indptr[i]; k < A->indptr[i + 1]; ++k)
        s += (double)A->values[k] * (double)A->values[k];
    return s;
}

/* The kernel in use (one per process; set before a call, read-only during
 * it). kind: 0 RBF, 1 linear, 2 polynomial, 3 sigmoid. */
static int g_kind = 0;
static double g_coef0 = 0.0;
static int g_degree = 3;

void or_set_kernel(int kind, double coef0, int degree)
{
    g_kind = kind;
    g_coef0 = coef0;
    g_degree = degree;
}

/* RBF: K(x,z) = exp(-gamma * ||x-z||^2), ||x-z||^2 = ||x||^2 + ||z||^2 - 2<x,z>
 * (the "simple linear algebra trick"), clamped at 0 against rounding.
 * Polynomial: the power by repeated multiplication, degree >= 1. */
double or_kernel(double gamma, double nx, double nz, double dot)
{
    if (g_kind == 1) return dot;
    if (g_kind == 2) {
        const double b = gamma * dot + g_coef0;
        double r = b;
        for (int k = 1; k < g_degree; ++k) r *= b;
        return r;
    }
    if (g_kind == 3) return tanh(gamma * dot + g_coef0);
    double d2 = nx + nz - 2.0 * dot;
    if (d2 < 0.0) d2 = 0.0;
    return exp(-gamma * d2);
}

static double kern(const or_csr *X, const double *nrm, double gamma, int64_t i, int64_t j)
{
    return or_kernel(gamma, nrm[i], nrm[j], or_dot(X, i, X, j));
}

/* Eq. (setinfo) */
static int set_of(int8_t y, double a, double C)
{
    if (a > 0.0 && a < C) return OR_SET_I0;
    if (a == 0.0) return y > 0 ? OR_SET_I1 : OR_SET_I4;
    return y > 0 ? OR_SET_I3 : OR_SET_I2; /* a == C */
}
static int in_up(int s) { return s == OR_SET_I0 || s == OR_SET_I1 || s == OR_SET_I2; }
static int in_low(int s) { return s == OR_SET_I0 || s == OR_SET_I3 || s == OR_SET_I4; }

/* ------------------------------------------------------- pair selection */

typedef struct {
    double b_up, b_low;     /* min f over I_up, max f over I_low */
    int64_t i_up, i_low;    /* arg, lowest index on ties; -1 if the set is empty */
    double up2, low2;       /* second smallest / second largest value */
} or_sel;

static void sel_init(or_sel *s)
{
    s->b_up = INFINITY; s->b_low = -INFINITY;
    s->i_up = -1; s->i_low = -1;
    s->up2 = INFINITY; s->low2 = -INFINITY;
}

static void sel_add(or_sel *s, int64_t i, double fi, int set)
{
    if (in_up(set)) {
        if (fi < s->b_up || (fi == s->b_up && (s->i_up < 0 || i < s->i_up))) {
            if (s->i_up >= 0 && s->b_up < s->up2) s->up2 = s->b_up;
            s->b_up = fi; s->i_up = i;
        } else if (fi < s->up2) {
            s->up2 = fi;
        }
    }
    if (in_low(set)) {
        if (fi > s->b_low || (fi == s->b_low && (s->i_low < 0 || i < s->i_low))) {
            if (s->i_low >= 0 && s->b_low > s->low2) s->low2 = s->b_low;
            s->b_low = fi; s->i_low = i;
        } else if (fi > s->low2) {
            s->low2 = fi;
        }
    }
}

/* merge b into a; b covers higher indices than a (thread order) */
static void sel_merge(or_sel *a, const or_sel *b)
{
    if (b->i_up >= 0) {
        if (b->b_up < a->b_up || a->i_up < 0) {
            double old = a->b_up;
            a->up2 = fmin(fmin(old, a->up2), b->up2);
            a->b_up = b->b_up; a->i_up = b->i_up;
        } else {
            /* a wins (ties go to the lower index, which is in a) */
            a->up2 = fmin(a->up2, fmin(b->b_up, b->up2));
        }
    }
    if (b->i_low >= 0) {
        if (b->b_low > a->b_low || a->i_low < 0) {
            double old = a->b_low;
            a->low2 = fmax(fmax(old, a->low2), b->low2);
            a->b_low = b->b_low; a->i_low = b->i_low;
        } else {
            a->low2 = fmax(a->low2, fmax(b->b_low, b->low2));
        }
    }
}

/* Eq. (bminmax) over the rows listed in idx[0..m) (or all rows if idx is
 * NULL). Deterministic for any thread count. */
static or_sel select_pair(int64_t m, const int64_t *idx, const double *f, const uint8_t *set)
{
    or_sel res;
    sel_init(&res);
#ifdef _OPENMP
    int nt = omp_get_max_threads();
    if (m < 4096) nt = 1;
    or_sel part[256];
    if (nt > 256) nt = 256;
#pragma omp parallel num_threads(nt)
    {
        int t = omp_get_thread_num(), T = omp_get_num_threads();
        int64_t lo = m * t / T, hi = m * (t + 1) / T;
        or_sel s;
        sel_init(&s);
        for (int64_t k = lo; k < hi; ++k) {
            int64_t i = idx ? idx[k] : k;
            sel_add(&s, i, f[i], set[i]);
        }
        part[t] = s;
#pragma omp barrier
#pragma omp single
        {
            for (int u = 0; u < T; ++u) sel_merge(&res, &part[u]);
        }
    }
#else
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        sel_add(&res, i, f[i], set[i]);
    }
#endif
    return res;
}

/* ----------------------------------------------------------- alpha step */

typedef struct {
    double au, al;     /* new alpha of i_up, i_low */
    double du, dl;     /* y_up*(au'-au), y_low*(al'-al): the (fup) coefficients */
} or_step;

/* Eq. (alphaup) with rho = 2K_ul - K_uu - K_ll = -eta, jointly clipped to the
 * feasible segment; Platt's end-point rule when eta <= 1e-12. */
static or_step alpha_step(double C, int8_t yu, int8_t yl, double au, double al,
                          double fu, double fl, double kuu, double kll, double kul)
{
    double eta = kuu + kll - 2.0 * kul;
    double s = (double)(yu * yl);
    double L, H;
    if (s < 0) {
        L = fmax(0.0, al - au);
        H = fmin(C, C + al - au);
    } else {
        L = fmax(0.0, al + au - C);
        H = fmin(C, al + au);
    }
    double slope = (double)yl * (fu - fl); /* dW/d alpha_low along the segment */
    double aln;
    if (eta > 1e-12) {
        double t = al + slope / eta;
        aln = t < L ? L : (t > H ? H : t);
    } else {
        aln = slope > 0.0 ? H : L;
    }
    double aun = au + s * (al - aln);
    double snap = 1e-12 * C;
    if (aln < snap) aln = 0.0;
    if (aln > C - snap) aln = C;
    if (aun < snap) aun = 0.0;
    if (aun > C - snap) aun = C;
    or_step r;
    r.au = aun; r.al = aln;
    r.du = (double)yu * (aun - au);
    r.dl = (double)yl * (aln - al);
    return r;
}

/* ------------------------------------------------------------- helpers */

static double *row_norms(const or_csr *X)
{
    double *nrm = (double *)malloc(sizeof(double) * (size_t)(X->n > 0 ? X->n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < X->n; ++i) nrm[i] = or_sqnorm(X, i);
    return nrm;
}

static double threshold_b(int64_t n, const double *f, const uint8_t *set, double b_up, double b_low)
{
    double s = 0.0;
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        if (set[i] == OR_SET_I0) { s += f[i]; ++c; }
    return c ? s / (double)c : 0.5 * (b_up + b_low);
}

/* W = sum a - 1/2 sum a_i y_i (f_i + y_i)  (Eq. lagdual using Eq. fcache) */
static double objective(int64_t n, const int8_t *y, const double *a, const double *f)
{
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        s1 += a[i];
        s2 += a[i] * (double)y[i] * (f[i] + (double)y[i]);
    }
    return s1 - 0.5 * s2;
}

/* Eq. (fup) over the listed rows */
static void update_f(const or_csr *X, const double *nrm, double gamma, int64_t m,
                     const int64_t *idx, double *f, int64_t u, int64_t l, double du, double dl)
{
#pragma omp parallel for schedule(static) if (m >= 4096)
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        double ku = kern(X, nrm, gamma, u, i);
        double kl = kern(X, nrm, gamma, l, i);
        f[i] = f[i] + du * ku + dl * kl;
    }
}

/* ---------------------------------------------------------- public API */

typedef struct {
    int64_t iters;
    double b, b_up, b_low, objective;
    int64_t n_shrink, n_recon, final_active;
    int32_t status;  /* 0 converged, 1 max_iter reached */
} or_result;

void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Algorithm 1 (no shrinking). alpha and f are outputs of length n.
 * trace (2*trace_len int64: i_up, i_low per iteration) and margin
 * (2*trace_len: second-best minus best violation value on each side) may be
 * NULL. objs (trace_len) records the objective after each step when non-NULL
 * (O(n) per iteration).
 */
int or_smo(const or_csr *X, const int8_t *y, double C, double gamma, double tau,
           int64_t max_iter, double *alpha, double *f, or_result *res,
           int64_t *trace, double *margin, double *objs, int64_t trace_len)
{
    int64_t n = X->n;
    double *nrm = row_norms(X);
    uint8_t *set = (uint8_t *)malloc((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        alpha[i] = 0.0;
        f[i] = -(double)y[i];
        set[i] = (uint8_t)set_of(y[i], 0.0, C);
    }
    int64_t it = 0;
    or_sel s = select_pair(n, NULL, f, set);
    int status = 0;
    while (s.b_low - s.b_up > 2.0 * tau) {
        if (it >= max_iter) { status = 1; break; }
        int64_t u = s.i_up, l = s.i_low;
        if (trace && it < trace_len) {
            trace[2 * it] = u;
            trace[2 * it + 1] = l;
            if (margin) {
                margin[2 * it] = s.up2 - s.b_up;
                margin[2 * it + 1] = s.b_low - s.low2;
            }
        }
        double kuu = kern(X, nrm, gamma, u, u), kll = kern(X, nrm, gamma, l, l);
        double kul = kern(X, nrm, gamma, u, l);
        or_step st = alpha_step(C, y[u], y[l], alpha[u], alpha[l], f[u], f[l], kuu, kll, kul);
        alpha[u] = st.au;
        alpha[l] = st.al;
        set[u] = (uint8_t)set_of(y[u], alpha[u], C);
        set[l] = (uint8_t)set_of(y[l], alpha[l], C);
        update_f(X, nrm, gamma, n, NULL, f, u, l, st.du, st.dl);
        if (objs && it < trace_len) objs[it] = objective(n, y, alpha, f);
        ++it;
        s = select_pair(n, NULL, f, set);
    }
    res->iters = it;
    res->b_up = s.b_up;
    res->b_low = s.b_low;
    res->b = threshold_b(n, f, set, s.b_up, s.b_low);
    res->objective = objective(n, y, alpha, f);
    res->n_shrink = 0;
    res->n_recon = 0;
    res->final_active = n;
    res->status = status;
    free(set);
    free(nrm);
    return status;
}

/* Eq. (fcache) from scratch for all i: f_i = sum_j a_j y_j K_ij - y_i. */
void or_gradient(const or_csr *X, const int8_t *y, const double *alpha, double gamma, double *f)
{
    int64_t n = X->n;
    double *nrm = row_norms(X);
    int64_t nsv = 0;
    int64_t *sv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j)
        if (alpha[j] > 0.0) sv[nsv++] = j;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = 0; k < nsv; ++k) {
            int64_t j = sv[k];
            s += alpha[j] * (double)y[j] * kern(X, nrm, gamma, i, j);
        }
        f[i] = s - (double)y[i];
    }
    free(sv);
    free(nrm);
}

/* Algorithm 6 for the rows listed in rows[0..m): f_a = sum_{b: a_b > 0}
 * a_b y_b K(a,b) - y_a, summed over b in ascending index order. */
void or_reconstruct(const or_csr *X, const int8_t *y, const double *alpha, double gamma,
                    int64_t m, const int64_t *rows, double *f)
{
    int64_t n = X->n;
    double *nrm = row_norms(X);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < m; ++k) {
        int64_t a = rows[k];
        double s = 0.0;
        for (int64_t b = 0; b < n; ++b)
            if (alpha[b] > 0.0) s += alpha[b] * (double)y[b] * kern(X, nrm, gamma, a, b);
        f[a] = s - (double)y[a];
    }
    free(nrm);
}

/* KKT check over all samples from a given alpha (recomputes f from scratch):
 * returns b_up, b_low (Eq. bminmax), the objective and the threshold b. */
void or_kkt(const or_csr *X, const int8_t *y, const double *alpha, double C, double gamma,
            double *f_out, or_result *res)
{
    int64_t n = X->n;
    or_gradient(X, y, alpha, gamma, f_out);
    uint8_t *set = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) set[i] = (uint8_t)set_of(y[i], alpha[i], C);
    or_sel s = select_pair(n, NULL, f_out, set);
    res->b_up = s.b_up;
    res->b_low = s.b_low;
    res->b = threshold_b(n, f_out, set, s.b_up, s.b_low);
    res->objective = objective(n, y, alpha, f_out);
    res->iters = 0;
    res->status = 0;
    free(set);
}

/* Eq. (classi) before the sign: out_k = sum_{j: a_j > 0} a_j y_j K(x_j, z_k) - b */
void or_decision(const or_csr *X, const int8_t *y, const double *alpha, double b, double gamma,
                 const or_csr *Z, double *out)
{
    int64_t n = X->n;
    double *nx = row_norms(X);
    double *nz = row_norms(Z);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < Z->n; ++k) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j)
            if (alpha[j] > 0.0)
                s += alpha[j] * (double)y[j] * or_kernel(gamma, nx[j], nz[k], or_dot(X, j, Z, k));
        out[k] = s - b;
    }
    free(nz);
    free(nx);
}

/* ----------------------------------------------- shrinking (Alg. 4 / 5) */

enum { OR_SHRINK_NONE = 0, OR_SHRINK_FIXED = 1, OR_SHRINK_FRACTION = 2 };
enum { OR_RECON_SINGLE = 0, OR_RECON_MULTI = 1 };

/*
 * Adaptive shrinking with gradient reconstruction.
 *
 * Shrink counter (Sec. III-C, Table 3): h = value (kind FIXED, the "random: k"
 * rows, read as a fixed constant) or ceil(value * N) (kind FRACTION, the
 * "numsamples" rows). The counter counts down once per iteration; when it
 * reaches 0 the iteration applies Eq. (shrink) to every active row after its
 * f update, using the b_up/b_low that selected the iteration's pair
 * (Algorithm 4 tests the rule before the global b values are updated); the
 * counter is then reset to min(h, |active|).
 *
 * Phases (Algorithm 5): iterate with shrinking while the active-set gap
 * exceeds first_factor*tau (20 tau in the paper); then reconstruct f of every
 * shrunk row (Algorithm 6) and take b_up/b_low over all rows. If the gap is
 * <= 2 tau, stop. Otherwise:
 *   SINGLE: reset the active set to all rows and continue without shrinking
 *           until the gap is <= 2 tau.
 *   MULTI : reset the active set to all rows, restart the counter at h and
 *           keep shrinking; every later reconstruction is triggered at 2 tau.
 * Rows removed in an iteration take no part in that iteration's selection.
 * With wss = 2 the pair is (i_up, the second-order i_low over the active
 * rows); b_up and b_low stay the first-order extremes of Eq. (bminmax), so
 * Eq. (shrink) and Eq. (kktterm) read the same values as without it.
 */
/* i_low of the second-order rule: the largest gain (f_t - f_u)^2 / a_ut over
 * t in I_low with f_t > f_u, a_ut = K_uu + K_tt - 2 K_ut floored at 1e-12;
 * lowest index on ties. Candidates t are act[0 .. m) (increasing sample
 * indices), or 0 .. m-1 when act is NULL. *gap2 = the gain's relative lead
 * over the runner-up. */
static int64_t select_low2(const or_csr *X, const double *nrm, double gamma, int64_t m,
                           const int64_t *act, const double *f, const uint8_t *set, int64_t u,
                           double *gap2)
{
    const double kuu = kern(X, nrm, gamma, u, u);
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    double *bg = (double *)malloc(sizeof(double) * 2 * (size_t)nt);
    int64_t *bi = (int64_t *)malloc(sizeof(int64_t) * (size_t)nt);
    for (int t = 0; t < nt; ++t) { bg[2 * t] = -1.0; bg[2 * t + 1] = -1.0; bi[t] = -1; }
#pragma omp parallel if (m >= 4096)
    {
        int me = 0;
#ifdef _OPENMP
        me = omp_get_thread_num();
#endif
        double g1 = -1.0, g2 = -1.0;
        int64_t i1 = -1;
#pragma omp for schedule(static)
        for (int64_t k = 0; k < m; ++k) {
            const int64_t t = act ? act[k] : k;
            if (!in_low(set[t]) || !(f[t] > f[u])) continue;
            const double b = f[t] - f[u];
            double a = kuu + kern(X, nrm, gamma, t, t) - 2.0 * kern(X, nrm, gamma, u, t);
            if (a <= 0.0) a = 1e-12;
            const double g = (b * b) / a;
            if (g > g1) { g2 = g1; g1 = g; i1 = t; }
            else if (g > g2) g2 = g;
        }
        bg[2 * me] = g1;
        bg[2 * me + 1] = g2;
        bi[me] = i1;
    }
    /* merge in thread order: threads hold increasing index ranges */
    double g1 = -1.0, g2 = -1.0;
    int64_t i1 = -1;
    for (int t = 0; t < nt; ++t) {
        if (bi[t] < 0) continue;
        if (bg[2 * t] > g1) { g2 = g1 > bg[2 * t + 1] ? g1 : bg[2 * t + 1]; g1 = bg[2 * t]; i1 = bi[t]; }
        else { const double c = bg[2 * t] > bg[2 * t + 1] ? bg[2 * t] : bg[2 * t + 1]; if (c > g2) g2 = c; }
    }
    free(bg);
    free(bi);
    *gap2 = g1 > 0.0 ? (g1 - g2) / g1 : 0.0;
    return i1;
}

int or_smo_wss2(const or_csr *X, const int8_t *y, double C, double gamma, double tau,
                int64_t max_iter, double *alpha, double *f, or_result *res,
                int64_t *trace, double *margin, int64_t trace_len)
{
    int64_t n = X->n;
    double *nrm = row_norms(X);
    uint8_t *set = (uint8_t *)malloc((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        alpha[i] = 0.0;
        f[i] = -(double)y[i];
        set[i] = (uint8_t)set_of(y[i], 0.0, C);
    }
    int64_t it = 0;
    or_sel s = select_pair(n, NULL, f, set);
    int status = 0;
    while (s.b_low - s.b_up > 2.0 * tau) {
        if (it >= max_iter) { status = 1; break; }
        int64_t u = s.i_up;
        double gap2 = 0.0;
        int64_t l = select_low2(X, nrm, gamma, n, NULL, f, set, u, &gap2);
        if (trace && it < trace_len) {
            trace[2 * it] = u;
            trace[2 * it + 1] = l;
            if (margin) {
                margin[2 * it] = s.up2 - s.b_up;
                margin[2 * it + 1] = gap2;
            }
        }
        double kuu = kern(X, nrm, gamma, u, u), kll = kern(X, nrm, gamma, l, l);
        double kul = kern(X, nrm, gamma, u, l);
        or_step st = alpha_step(C, y[u], y[l], alpha[u], alpha[l], f[u], f[l], kuu, kll, kul);
        alpha[u] = st.au;
        alpha[l] = st.al;
        set[u] = (uint8_t)set_of(y[u], alpha[u], C);
        set[l] = (uint8_t)set_of(y[l], alpha[l], C);
        update_f(X, nrm, gamma, n, NULL, f, u, l, st.du, st.dl);
        ++it;
        s = select_pair(n, NULL, f, set);
    }
    res->iters = it;
    res->b_up = s.b_up;
    res->b_low = s.b_low;
    res->b = threshold_b(n, f, set, s.b_up, s.b_low);
    res->objective = objective(n, y, alpha, f);
    res->n_shrink = 0;
    res->n_recon = 0;
    res->final_active = n;
    res->status = status;
    free(set);
    free(nrm);
    return status;
}

/*
 * Algorithms 4 and 5 with Algorithm 6. Optional records (each may be NULL):
 *   trace / active_trace (trace_len): pair and active-set size of each step;
 *   gap_trace (trace_len): b_low - b_up of the selection that chose each
 *     step's pair, over the active rows (the quantity the phase threshold of
 *     Algorithm 5 is tested on);
 *   ev (3 * ev_cap) and ev_gap (2 * ev_cap): the events of the schedule in
 *     order, (steps completed, kind, active rows after) with kind 1 = shrink
 *     (Algorithm 4) and 2 = reconstruction (Algorithm 6); ev_gap holds the
 *     active-set gap that triggered the event and, for a reconstruction, the
 *     gap over all rows after it (Algorithm 5's stopping test). *n_ev receives
 *     the number of events (it may exceed ev_cap; only ev_cap are stored).
 */
int or_smo_shrink(const or_csr *X, const int8_t *y, double C, double gamma, double tau,
                  int64_t max_iter, int kind, double value, int recon, double first_factor,
                  double *alpha, double *f, or_result *res,
                  int64_t *trace, int64_t trace_len, int64_t *active_trace, int wss,
                  double *gap_trace, int64_t *ev, double *ev_gap, int64_t ev_cap, int64_t *n_ev)
{
    int64_t n = X->n;
    double *nrm = row_norms(X);
    uint8_t *set = (uint8_t *)malloc((size_t)n);
    int64_t *act = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    uint8_t *live = (uint8_t *)malloc((size_t)n);
    int64_t *shr = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        alpha[i] = 0.0;
        f[i] = -(double)y[i];
        set[i] = (uint8_t)set_of(y[i], 0.0, C);
        act[i] = i;
        live[i] = 1;
    }
    int64_t m = n;
    int64_t h = 0;
    if (kind == OR_SHRINK_FIXED) h = (int64_t)value;
    if (kind == OR_SHRINK_FRACTION) h = (int64_t)ceil(value * (double)n);
    if (kind != OR_SHRINK_NONE && h < 1) h = 1;
    int shrinking = kind != OR_SHRINK_NONE;
    int64_t counter = h;
    double thr = shrinking ? first_factor * tau : 2.0 * tau;
    int64_t it = 0, n_shrink = 0, n_recon = 0, ne = 0;
    int status = 0;
    or_sel s = select_pair(m, act, f, set);
    for (;;) {
        while (s.b_low - s.b_up > thr) {
            if (it >= max_iter) { status = 1; break; }
            int64_t u = s.i_up, l = s.i_low;
            if (wss == 2) {
                double gap2;
                l = select_low2(X, nrm, gamma, m, act, f, set, u, &gap2);
            }
            if (trace && it < trace_len) { trace[2 * it] = u; trace[2 * it + 1] = l; }
            if (active_trace && it < trace_len) active_trace[it] = m;
            if (gap_trace && it < trace_len) gap_trace[it] = s.b_low - s.b_up;
            double kuu = kern(X, nrm, gamma, u, u), kll = kern(X, nrm, gamma, l, l);
            double kul = kern(X, nrm, gamma, u, l);
            or_step st = alpha_step(C, y[u], y[l], alpha[u], alpha[l], f[u], f[l], kuu, kll, kul);
            alpha[u] = st.au;
            alpha[l] = st.al;
            set[u] = (uint8_t)set_of(y[u], alpha[u], C);
            set[l] = (uint8_t)set_of(y[l], alpha[l], C);
            update_f(X, nrm, gamma, m, act, f, u, l, st.du, st.dl);
            int shrink_now = 0;
            if (shrinking) {
                counter -= 1;
                shrink_now = counter <= 0;
            }
            if (shrink_now) {
                /* Eq. (shrink) with the b values that selected this pair */
                int64_t w = 0;
                for (int64_t k = 0; k < m; ++k) {
                    int64_t i = act[k];
                    int st_i = set[i];
                    int drop = ((st_i == OR_SET_I3 || st_i == OR_SET_I4) && f[i] < s.b_up) ||
                               ((st_i == OR_SET_I1 || st_i == OR_SET_I2) && f[i] > s.b_low);
                    if (drop) live[i] = 0; else act[w++] = i;
                }
                m = w;
                counter = h < m ? h : m;
                if (counter < 1) counter = 1;
                ++n_shrink;
                if (ev && ne < ev_cap) {
                    ev[3 * ne] = it + 1; ev[3 * ne + 1] = 1; ev[3 * ne + 2] = m;
                    if (ev_gap) { ev_gap[2 * ne] = s.b_low - s.b_up; ev_gap[2 * ne + 1] = NAN; }
                }
                ++ne;
            }
            ++it;
            s = select_pair(m, act, f, set);
        }
        if (status) break;
        if (!shrinking) break;
        /* Algorithm 6 on every shrunk row, then b over all rows */
        int64_t ns = 0;
        for (int64_t i = 0; i < n; ++i)
            if (!live[i]) shr[ns++] = i;
        if (ns > 0) {
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t k = 0; k < ns; ++k) {
                int64_t a = shr[k];
                double acc = 0.0;
                for (int64_t b = 0; b < n; ++b)
                    if (alpha[b] > 0.0) acc += alpha[b] * (double)y[b] * kern(X, nrm, gamma, a, b);
                f[a] = acc - (double)y[a];
            }
        }
        ++n_recon;
        const double gap_active = s.b_low - s.b_up;
        for (int64_t i = 0; i < n; ++i) { act[i] = i; live[i] = 1; }
        m = n;
        s = select_pair(m, act, f, set);
        if (ev && ne < ev_cap) {
            ev[3 * ne] = it; ev[3 * ne + 1] = 2; ev[3 * ne + 2] = m;
            if (ev_gap) { ev_gap[2 * ne] = gap_active; ev_gap[2 * ne + 1] = s.b_low - s.b_up; }
        }
        ++ne;
        if (s.b_low - s.b_up <= 2.0 * tau) break;
        if (recon == OR_RECON_SINGLE) {
            shrinking = 0;
        } else {
            counter = h;
        }
        thr = 2.0 * tau;
    }
    res->iters = it;
    res->b_up = s.b_up;
    res->b_low = s.b_low;
    res->b = threshold_b(n, f, set, s.b_up, s.b_low);
    res->objective = objective(n, y, alpha, f);
    res->n_shrink = n_shrink;
    res->n_recon = n_recon;
    res->final_active = m;
    res->status = status;
    if (n_ev) *n_ev = ne;
    free(shr);
    free(live);
    free(act);
    free(set);
    free(nrm);
    return status;
}
