/* Memory- and UB-safety driver for the FP64 oracle (test infrastructure).
 *
 * Built together with oracle/mf_oracle.c under AddressSanitizer and
 * UndefinedBehaviorSanitizer by tests/test_oracle_sanitizers.py; it calls
 * every exported oracle function once or twice on small grid, sparse and
 * dense models (including the one-variable and one-label edge cases) so that
 * an out-of-bounds read or write, a leak or an undefined operation in the
 * oracle makes the process exit non-zero.  It checks no values: the pins do.
 *
 * Inputs come from a fixed 64-bit LCG; nothing here depends on the CUDA
 * library.  The oracle has no header, so the prototypes are restated here.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct orc_model orc_model;

int orc_num_threads(void);
void orc_model_free(orc_model *m);
orc_model *orc_model_sparse(int64_t n, int32_t L, const double *U, const double *mu, int64_t ne,
                            const int64_t *ei, const int64_t *ej, const double *ew);
orc_model *orc_model_dense(int64_t n, int32_t L, const double *U, const double *mu, const double *K);
int64_t orc_grid_edge_count(int64_t H, int64_t W, int32_t conn);
void orc_grid_edges(int64_t H, int64_t W, int32_t conn, const double *w, int64_t *ei, int64_t *ej, double *ew);
void orc_dense_gauss_kernel(int64_t n, const double *f, double theta_pos, double theta_rgb, double *K);
void orc_hess_vec(const orc_model *m, const double *v, double *out);
void orc_grad(const orc_model *m, const double *q, double *g);
double orc_energy(const orc_model *m, const double *q);
double orc_neg_entropy(const orc_model *m, const double *q);
double orc_free_energy(const orc_model *m, const double *q);
void orc_init_logq(const orc_model *m, double *s);
void orc_prox_step(const orc_model *m, double eta, const double *s_in, double *s_out);
void orc_prox_step_rows(const orc_model *m, double eta, const double *s_in, const int64_t *rows, int64_t nrows,
                        double *out);
void orc_parallel_prox(const orc_model *m, double eta, int32_t iters, double *s, double *F_trace);
int32_t orc_prox_step_adaptive(const orc_model *m, double d, const double *s_in, double *s_out);
int32_t orc_parallel_prox_adaptive(const orc_model *m, double d, int32_t iters, double *s, double *F_trace);
void orc_parallel_prox_momentum(const orc_model *m, double eta, double gamma1, int32_t iters, double *s,
                                double *F_trace);
void orc_parallel_prox_adam(const orc_model *m, double d0, double gamma1, double gamma2, double eps,
                            int32_t iters, double *s, double *F_trace);
void orc_parallel_adhoc(const orc_model *m, double eta, int32_t iters, double *s, double *F_trace);
void orc_sweep(const orc_model *m, int32_t sweeps, double *s);
double orc_unrolled_loss_grad(const orc_model *m, double eta, int32_t K, const int32_t *y, double *dU,
                              double *dmu, double *dw);
double orc_unrolled_loss(const orc_model *m, double eta, int32_t K, const int32_t *y);
double orc_state_energy(const orc_model *m, const int32_t *x);
int orc_brute_force(const orc_model *m, double *logZ, double *marg);
double orc_brute_free_energy(const orc_model *m, const double *q);
int orc_brute_cond_energy(const orc_model *m, const double *q, double *out);
void orc_jacobi_eigenvalues(int64_t n, double *A, double *ev);
int orc_hessian_eigenvalues(const orc_model *m, int projected, double *ev);
int32_t orc_lanczos_tangent(const orc_model *m, int32_t iters, const double *v0, double *lmin, double *lmax);
double orc_step_size(double Lambda);

static uint64_t g_state = 0x9E3779B97F4A7C15ull;

static double urand(void)   /* [0, 1) */
{
    g_state = g_state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(g_state >> 11) * (1.0 / 9007199254740992.0);
}

static double *rnd(size_t n, double lo, double hi)
{
    double *p = (double *)malloc(sizeof(double) * (n ? n : 1));
    for (size_t k = 0; k < n; ++k) p[k] = lo + (hi - lo) * urand();
    return p;
}

static double *zeros(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

static int g_fail = 0;

static void check_finite(const char *what, const double *v, size_t n)
{
    for (size_t k = 0; k < n; ++k)
        if (!isfinite(v[k])) {
            fprintf(stderr, "%s: non-finite entry %zu\n", what, k);
            g_fail = 1;
            return;
        }
}

/* Every state-level call on one model with n variables and L labels;
 * ne edges (0 for dense models). */
static void exercise(orc_model *m, int64_t n, int32_t L, int64_t ne)
{
    const size_t nl = (size_t)(n * L);
    const int32_t iters = 4;
    double *s = zeros(nl), *t = zeros(nl), *q = zeros(nl), *g = zeros(nl), *F = zeros(iters + 1);
    orc_init_logq(m, s);
    for (size_t k = 0; k < nl; ++k) q[k] = exp(s[k]);
    orc_grad(m, q, g);
    orc_hess_vec(m, q, t);
    double e = orc_energy(m, q) + orc_neg_entropy(m, q) + orc_free_energy(m, q);
    check_finite("energies", &e, 1);

    orc_prox_step(m, 0.5, s, t);
    check_finite("prox_step", t, nl);
    int64_t rows[3] = {0, n - 1, n / 2};
    double *out = zeros((size_t)3 * L);
    orc_prox_step_rows(m, 0.5, s, rows, 3, out);
    free(out);

    orc_parallel_prox(m, 0.5, iters, s, F);
    check_finite("parallel_prox", F, iters + 1);
    orc_parallel_prox(m, 0.5, 1, s, NULL);
    orc_init_logq(m, s);
    orc_parallel_prox_momentum(m, 0.5, 0.9, iters, s, F);
    orc_init_logq(m, s);
    orc_parallel_prox_adam(m, 0.5, 0.9, 0.999, 1e-8, iters, s, F);
    orc_init_logq(m, s);
    orc_parallel_adhoc(m, 0.5, iters, s, F);
    orc_init_logq(m, s);
    if (orc_prox_step_adaptive(m, 2.0, s, t) == 0) {
        orc_parallel_prox_adaptive(m, 2.0, iters, s, F);
        check_finite("adaptive", s, nl);
    }
    orc_init_logq(m, s);
    orc_sweep(m, 2, s);
    check_finite("sweep", s, nl);

    int32_t *y = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) y[i] = (int32_t)(urand() * L) % L;
    double *dU = zeros(nl), *dmu = zeros((size_t)L * L), *dw = zeros((size_t)ne);
    double lg = orc_unrolled_loss_grad(m, 0.4, 3, y, dU, dmu, dw) + orc_unrolled_loss(m, 0.4, 3, y);
    check_finite("unrolled", &lg, 1);
    check_finite("unrolled dU", dU, nl);
    double es = orc_state_energy(m, y);
    check_finite("state_energy", &es, 1);

    double lmin = 0.0, lmax = 0.0;
    double *v0 = rnd(nl, -1.0, 1.0);
    if (nl > 1) orc_lanczos_tangent(m, 8, v0, &lmin, &lmax);
    double eta = orc_step_size(lmax) + orc_step_size(-1.0);
    check_finite("step_size", &eta, 1);
    if (nl <= 2048) {
        double *ev = zeros(nl);
        orc_hessian_eigenvalues(m, 1, ev);
        orc_hessian_eigenvalues(m, 0, ev);
        check_finite("hessian eigenvalues", ev, nl);
        free(ev);
    }
    double logZ = 0.0;
    double *marg = zeros(nl), *ce = zeros(nl);
    if (orc_brute_force(m, &logZ, marg) == 0) {
        double bf = orc_brute_free_energy(m, q);
        check_finite("brute free energy", &bf, 1);
        orc_brute_cond_energy(m, q, ce);
        check_finite("brute marginals", marg, nl);
    }
    free(marg); free(ce); free(v0); free(y); free(dU); free(dmu); free(dw);
    free(s); free(t); free(q); free(g); free(F);
}

static void grid_case(int64_t H, int64_t W, int32_t L, int32_t conn, int sym)
{
    const int nd = conn == 8 ? 4 : 2;
    const int64_t n = H * W;
    double *U = rnd((size_t)(n * L), 0.0, 2.0), *mu = rnd((size_t)L * L, -1.0, 1.0);
    if (sym)
        for (int a = 0; a < L; ++a)
            for (int b = 0; b < a; ++b) mu[a * L + b] = mu[b * L + a];
    double *w = rnd((size_t)(nd * n), 0.0, 1.0);
    const int64_t ne = orc_grid_edge_count(H, W, conn);
    int64_t *ei = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ne ? ne : 1));
    int64_t *ej = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ne ? ne : 1));
    double *ew = zeros((size_t)ne);
    orc_grid_edges(H, W, conn, w, ei, ej, ew);
    orc_model *m = orc_model_sparse(n, L, U, mu, ne, ei, ej, ew);
    if (!m) { fprintf(stderr, "grid model allocation failed\n"); g_fail = 1; return; }
    exercise(m, n, L, ne);
    orc_model_free(m);
    free(U); free(mu); free(w); free(ei); free(ej); free(ew);
}

static void sparse_case(int64_t n, int32_t L, int64_t ne)
{
    double *U = rnd((size_t)(n * L), 0.0, 2.0), *mu = rnd((size_t)L * L, -1.0, 1.0);
    int64_t *ei = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ne ? ne : 1));
    int64_t *ej = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ne ? ne : 1));
    double *ew = rnd((size_t)ne, -0.5, 0.5);
    for (int64_t e = 0; e < ne; ++e) {
        ei[e] = (int64_t)(urand() * n) % n;
        ej[e] = (ei[e] + 1 + (int64_t)(urand() * (n - 1))) % n;   /* no self loops */
    }
    orc_model *m = orc_model_sparse(n, L, U, mu, ne, ei, ej, ew);
    if (!m) { fprintf(stderr, "sparse model allocation failed\n"); g_fail = 1; return; }
    exercise(m, n, L, ne);
    orc_model_free(m);
    free(U); free(mu); free(ei); free(ej); free(ew);
}

static void dense_case(int64_t n, int32_t L)
{
    double *U = rnd((size_t)(n * L), 0.0, 2.0), *mu = rnd((size_t)L * L, 0.0, 1.0);
    for (int a = 0; a < L; ++a)
        for (int b = 0; b < a; ++b) mu[a * L + b] = mu[b * L + a];
    double *f = rnd((size_t)n * 5, 0.0, 10.0), *K = zeros((size_t)(n * n));
    orc_dense_gauss_kernel(n, f, 3.0, 5.0, K);
    orc_model *m = orc_model_dense(n, L, U, mu, K);
    if (!m) { fprintf(stderr, "dense model allocation failed\n"); g_fail = 1; return; }
    exercise(m, n, L, 0);
    orc_model_free(m);
    free(U); free(mu); free(f); free(K);
}

int main(void)
{
    if (orc_num_threads() < 1) g_fail = 1;
    grid_case(5, 7, 3, 8, 1);
    grid_case(4, 6, 2, 4, 0);
    grid_case(1, 1, 4, 8, 1);     /* one variable, no edges */
    grid_case(3, 1, 1, 4, 1);     /* one label */
    grid_case(2, 3, 2, 8, 0);     /* small enough for brute force */
    sparse_case(9, 3, 20);
    sparse_case(6, 2, 0);         /* no edges */
    dense_case(12, 3);
    dense_case(4, 2);

    double A[9] = {2.0, 1.0, 0.0, 1.0, 3.0, 1.0, 0.0, 1.0, 4.0}, ev[3];
    orc_jacobi_eigenvalues(3, A, ev);
    check_finite("jacobi", ev, 3);

    if (g_fail) return 1;
    printf("oracle sanitizer driver: ok\n");
    return 0;
}
