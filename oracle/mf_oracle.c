/*
 * mf_oracle.c -- plain FP64 CPU oracle for parallel proximal mean-field
 * inference on pairwise discrete random fields (Baque, Bagautdinov, Fleuret,
 * Fua, "Principled Parallel Mean-Field Inference for Discrete Random Fields").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Everything is written for a reader checking it against the paper by eye:
 * FP64 throughout, libm exp/log, no blocking or fusion beyond what the
 * definitions state.  The only parallelism is an OpenMP loop over variables
 * where every variable's result is computed independently, in a fixed order,
 * so results do not depend on the thread count.
 *
 * Conventions (the paper writes potentials phi inside exp(+...), Sec. 2.1):
 *   U[i*L+l]    unary energy (cost) of x_i = l, i.e. U = -phi_i;
 *   mu[l*L+m]   pairwise cost of (x_i=l, x_j=m) on an edge oriented i->j;
 *   E(x)        = sum_i U[i,x_i] + sum_{edges i->j} w_ij mu[x_i,x_j],
 *               each unordered pair counted once (Eq. related:pairwise-mrf);
 *   q[i*L+l]    mean parameters on the simplex (Eq. related:definition_q);
 *   s = log q   the log-domain state; q_il ∝ exp(-theta_il) (Eq. naturalParam),
 *               so s is the natural parameter negated and normalised.
 *
 * Dense ("fully connected") models keep an explicit symmetric N x N weight
 * matrix K with zero diagonal; the pair (i,j), i<j, is oriented i->j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct orc_model {
    int64_t n;          /* variables */
    int32_t L;          /* labels */
    double *U;          /* [n][L] */
    double *mu;         /* [L][L] */
    /* sparse mode: oriented edge list plus incidence lists */
    int64_t ne;
    int64_t *ei, *ej;
    double *ew;
    int64_t *out_ptr, *out_e;   /* edges leaving variable i  */
    int64_t *in_ptr, *in_e;     /* edges entering variable i */
    /* dense mode: K != NULL, [n][n] */
    double *K;
} orc_model;

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* model construction                                                  */
/* ------------------------------------------------------------------ */

static void *xcalloc(size_t n, size_t sz)
{
    void *p = calloc(n ? n : 1, sz);
    return p;
}

void orc_model_free(orc_model *m)
{
    if (!m) return;
    free(m->U); free(m->mu);
    free(m->ei); free(m->ej); free(m->ew);
    free(m->out_ptr); free(m->out_e); free(m->in_ptr); free(m->in_e);
    free(m->K);
    free(m);
}

static orc_model *model_common(int64_t n, int32_t L, const double *U, const double *mu)
{
    orc_model *m = (orc_model *)xcalloc(1, sizeof(orc_model));
    if (!m) return NULL;
    m->n = n;
    m->L = L;
    m->U = (double *)xcalloc((size_t)(n * L), sizeof(double));
    m->mu = (double *)xcalloc((size_t)L * L, sizeof(double));
    if (!m->U || !m->mu) { orc_model_free(m); return NULL; }
    memcpy(m->U, U, sizeof(double) * (size_t)(n * L));
    memcpy(m->mu, mu, sizeof(double) * (size_t)L * L);
    return m;
}

/* Pairwise model on an arbitrary graph: edge e is oriented ei[e] -> ej[e]
 * with weight ew[e] (Eq. related:pairwise-mrf with phi_ij = -ew*mu). */
orc_model *orc_model_sparse(int64_t n, int32_t L, const double *U, const double *mu,
                            int64_t ne, const int64_t *ei, const int64_t *ej,
                            const double *ew)
{
    orc_model *m = model_common(n, L, U, mu);
    if (!m) return NULL;
    m->ne = ne;
    m->ei = (int64_t *)xcalloc((size_t)ne, sizeof(int64_t));
    m->ej = (int64_t *)xcalloc((size_t)ne, sizeof(int64_t));
    m->ew = (double *)xcalloc((size_t)ne, sizeof(double));
    m->out_ptr = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    m->in_ptr = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    m->out_e = (int64_t *)xcalloc((size_t)ne, sizeof(int64_t));
    m->in_e = (int64_t *)xcalloc((size_t)ne, sizeof(int64_t));
    if (!m->ei || !m->ej || !m->ew || !m->out_ptr || !m->in_ptr || !m->out_e || !m->in_e) {
        orc_model_free(m);
        return NULL;
    }
    memcpy(m->ei, ei, sizeof(int64_t) * (size_t)ne);
    memcpy(m->ej, ej, sizeof(int64_t) * (size_t)ne);
    memcpy(m->ew, ew, sizeof(double) * (size_t)ne);
    /* incidence lists, edges kept in their original order */
    for (int64_t e = 0; e < ne; ++e) {
        m->out_ptr[ei[e] + 1]++;
        m->in_ptr[ej[e] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) {
        m->out_ptr[i + 1] += m->out_ptr[i];
        m->in_ptr[i + 1] += m->in_ptr[i];
    }
    int64_t *fo = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
    int64_t *fi = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
    if (!fo || !fi) { free(fo); free(fi); orc_model_free(m); return NULL; }
    for (int64_t e = 0; e < ne; ++e) {
        m->out_e[m->out_ptr[ei[e]] + fo[ei[e]]++] = e;
        m->in_e[m->in_ptr[ej[e]] + fi[ej[e]]++] = e;
    }
    free(fo); free(fi);
    return m;
}

/* Fully connected model: K[i*n+j] = K[j*n+i] is the weight of the pair
 * {i,j}; the diagonal is ignored (pairs are i != j only, Sec. 2.1). */
orc_model *orc_model_dense(int64_t n, int32_t L, const double *U, const double *mu,
                           const double *K)
{
    orc_model *m = model_common(n, L, U, mu);
    if (!m) return NULL;
    m->K = (double *)malloc(sizeof(double) * (size_t)(n * n));
    if (!m->K) { orc_model_free(m); return NULL; }
    memcpy(m->K, K, sizeof(double) * (size_t)(n * n));
    for (int64_t i = 0; i < n; ++i) m->K[i * n + i] = 0.0;
    return m;
}

/* ------------------------------------------------------------------ */
/* grid and dense-kernel geometry                                      */
/* ------------------------------------------------------------------ */

/* Grid neighbourhood: pixel p = y*W + x.  Direction k (forward edges only):
 *   k=0 right (y, x+1), k=1 down (y+1, x), k=2 down-right (y+1, x+1),
 *   k=3 down-left (y+1, x-1).  4-connected grids use k=0,1; 8-connected
 *   grids use k=0..3.  w[k][y][x] is the weight of the edge leaving (y,x)
 *   in direction k; edges that leave the image do not exist. */
static const int DY[4] = {0, 1, 1, 1};
static const int DX[4] = {1, 0, 1, -1};

int64_t orc_grid_edge_count(int64_t H, int64_t W, int32_t conn)
{
    int nd = conn == 8 ? 4 : 2;
    int64_t c = 0;
    for (int k = 0; k < nd; ++k)
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                int64_t yy = y + DY[k], xx = x + DX[k];
                if (yy >= 0 && yy < H && xx >= 0 && xx < W) c++;
            }
    return c;
}

void orc_grid_edges(int64_t H, int64_t W, int32_t conn, const double *w,
                    int64_t *ei, int64_t *ej, double *ew)
{
    int nd = conn == 8 ? 4 : 2;
    int64_t c = 0;
    for (int k = 0; k < nd; ++k)
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                int64_t yy = y + DY[k], xx = x + DX[k];
                if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                    ei[c] = y * W + x;
                    ej[c] = yy * W + xx;
                    ew[c] = w[(k * H + y) * W + x];
                    c++;
                }
            }
}

/* Gaussian appearance kernel over (x, y, r, g, b) features, as used by
 * fully connected segmentation CRFs (Sec. 4.2, semantic segmentation):
 *   K_ij = exp(-|p_i-p_j|^2 / (2 theta_pos^2) - |c_i-c_j|^2 / (2 theta_rgb^2)),
 * K_ii = 0. */
void orc_dense_gauss_kernel(int64_t n, const double *f, double theta_pos,
                            double theta_rgb, double *K)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (i == j) { K[i * n + j] = 0.0; continue; }
            double dx = f[i * 5 + 0] - f[j * 5 + 0];
            double dy = f[i * 5 + 1] - f[j * 5 + 1];
            double dr = f[i * 5 + 2] - f[j * 5 + 2];
            double dg = f[i * 5 + 3] - f[j * 5 + 3];
            double db = f[i * 5 + 4] - f[j * 5 + 4];
            double p2 = dx * dx + dy * dy;
            double c2 = dr * dr + dg * dg + db * db;
            K[i * n + j] = exp(-p2 / (2.0 * theta_pos * theta_pos)
                               - c2 / (2.0 * theta_rgb * theta_rgb));
        }
    }
}

/* ------------------------------------------------------------------ */
/* energy, gradient, free energy  (Sec. 2.2.1, Eq. related:mf-objective) */
/* ------------------------------------------------------------------ */

/* sum_{l,m} a_l mu[l][m] b_m */
static double bilinear(const double *a, const double *mu, const double *b, int L)
{
    double t = 0.0;
    for (int l = 0; l < L; ++l) {
        double r = 0.0;
        for (int k = 0; k < L; ++k) r += mu[l * L + k] * b[k];
        t += a[l] * r;
    }
    return t;
}

/* Pairwise part of the gradient of the expected energy for variable i:
 *   out_l = sum_{i->j} w_ij sum_m mu[l][m] v_j,m + sum_{k->i} w_ki sum_m v_k,m mu[m][l].
 * Because E(q) is multilinear, this is the Hessian (the "potential
 * matrix" of Sec. 3.2) applied to v. */
static void pair_grad_var(const orc_model *m, const double *v, int64_t i, double *out)
{
    const int L = m->L;
    for (int l = 0; l < L; ++l) out[l] = 0.0;
    if (m->K) {
        const int64_t n = m->n;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double kij = m->K[i * n + j];
            const double *vj = v + j * L;
            if (j > i) {           /* pair oriented i -> j */
                for (int l = 0; l < L; ++l) {
                    double r = 0.0;
                    for (int k = 0; k < L; ++k) r += m->mu[l * L + k] * vj[k];
                    out[l] += kij * r;
                }
            } else {               /* pair oriented j -> i */
                for (int l = 0; l < L; ++l) {
                    double r = 0.0;
                    for (int k = 0; k < L; ++k) r += vj[k] * m->mu[k * L + l];
                    out[l] += kij * r;
                }
            }
        }
        return;
    }
    for (int64_t p = m->out_ptr[i]; p < m->out_ptr[i + 1]; ++p) {
        int64_t e = m->out_e[p];
        const double *vj = v + m->ej[e] * L;
        for (int l = 0; l < L; ++l) {
            double r = 0.0;
            for (int k = 0; k < L; ++k) r += m->mu[l * L + k] * vj[k];
            out[l] += m->ew[e] * r;
        }
    }
    for (int64_t p = m->in_ptr[i]; p < m->in_ptr[i + 1]; ++p) {
        int64_t e = m->in_e[p];
        const double *vk = v + m->ei[e] * L;
        for (int l = 0; l < L; ++l) {
            double r = 0.0;
            for (int k = 0; k < L; ++k) r += vk[k] * m->mu[k * L + l];
            out[l] += m->ew[e] * r;
        }
    }
}

/* Dense models: the vectors mu v_j (P) and mu^T v_j (PT) of every variable,
 * each entry summed over k in ascending order exactly as pair_grad_var sums
 * it.  A dense model pairs every variable with all others, so these vectors
 * are formed once per call instead of once per pair; the terms and their
 * order are those of pair_grad_var, so the results are the same bit for bit. */
static void dense_mu_vectors(const orc_model *m, const double *v, double *P, double *PT)
{
    const int L = m->L;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < m->n; ++j) {
        const double *vj = v + j * L;
        for (int l = 0; l < L; ++l) {
            double r = 0.0, rt = 0.0;
            for (int k = 0; k < L; ++k) {
                r += m->mu[l * L + k] * vj[k];
                rt += vj[k] * m->mu[k * L + l];
            }
            P[j * L + l] = r;
            PT[j * L + l] = rt;
        }
    }
}

/* pair_grad_var of a dense model from the vectors of dense_mu_vectors:
 * out_l = sum_{j>i} K_ij (mu v_j)_l + sum_{j<i} K_ij (mu^T v_j)_l, over j in
 * ascending order. */
static void dense_pair_grad_var(const orc_model *m, const double *P, const double *PT, int64_t i, double *out)
{
    const int L = m->L;
    const int64_t n = m->n;
    for (int l = 0; l < L; ++l) out[l] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const double kij = m->K[i * n + j];
        const double *pj = (j > i ? P : PT) + j * L;
        for (int l = 0; l < L; ++l) out[l] += kij * pj[l];
    }
}

/* The pairwise gradient of every variable: pair_grad_var for each i (dense
 * models through the per-variable vectors above). */
static void pair_grad_all(const orc_model *m, const double *v, double *out)
{
    if (m->K) {
        const size_t nl = (size_t)(m->n * m->L);
        double *P = (double *)malloc(sizeof(double) * nl);
        double *PT = (double *)malloc(sizeof(double) * nl);
        dense_mu_vectors(m, v, P, PT);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m->n; ++i) dense_pair_grad_var(m, P, PT, i, out + i * m->L);
        free(P);
        free(PT);
        return;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m->n; ++i) pair_grad_var(m, v, i, out + i * m->L);
}

/* Hessian-vector product H v (no unary term). */
void orc_hess_vec(const orc_model *m, const double *v, double *out)
{
    pair_grad_all(m, v, out);
}

/* g = grad E(q): g_il = U_il + (H q)_il.  By multilinearity this equals the
 * conditional expectation E_{Q(X\X_i)}[E(x) | x_i = l] (Eq. related:sweep-update,
 * Eq. method:update_natural: theta* = grad E). */
void orc_grad(const orc_model *m, const double *q, double *g)
{
    const int L = m->L;
    pair_grad_all(m, q, g);
    for (int64_t i = 0; i < m->n; ++i)
        for (int l = 0; l < L; ++l) g[i * L + l] += m->U[i * L + l];
}

/* E(q) = E_Q[E(x)] = sum_i q_i.U_i + sum_{pairs i->j} w_ij q_i^T mu q_j. */
double orc_energy(const orc_model *m, const double *q)
{
    const int L = m->L;
    const int64_t n = m->n;
    double *term = (double *)xcalloc((size_t)n, sizeof(double));
    /* dense: mu q_j once per variable; q_i^T (mu q_j) then sums exactly as
     * bilinear() does */
    double *P = NULL, *PT = NULL;
    if (m->K) {
        P = (double *)malloc(sizeof(double) * (size_t)(n * L));
        PT = (double *)malloc(sizeof(double) * (size_t)(n * L));
        dense_mu_vectors(m, q, P, PT);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double t = 0.0;
        for (int l = 0; l < L; ++l) t += q[i * L + l] * m->U[i * L + l];
        if (m->K) {
            for (int64_t j = i + 1; j < n; ++j) {
                double b = 0.0;
                for (int l = 0; l < L; ++l) b += q[i * L + l] * P[j * L + l];
                t += m->K[i * n + j] * b;
            }
        } else {
            for (int64_t p = m->out_ptr[i]; p < m->out_ptr[i + 1]; ++p) {
                int64_t e = m->out_e[p];
                t += m->ew[e] * bilinear(q + i * L, m->mu, q + m->ej[e] * L, L);
            }
        }
        term[i] = t;
    }
    double E = 0.0;
    for (int64_t i = 0; i < n; ++i) E += term[i];
    free(term);
    free(P);
    free(PT);
    return E;
}

/* -H(q) = sum q log q, with 0 log 0 = 0. */
double orc_neg_entropy(const orc_model *m, const double *q)
{
    double h = 0.0;
    const int64_t nl = m->n * m->L;
    for (int64_t k = 0; k < nl; ++k)
        if (q[k] > 0.0) h += q[k] * log(q[k]);
    return h;
}

/* F(q) = E(q) - H(q)  (Eq. related:mf-objective). */
double orc_free_energy(const orc_model *m, const double *q)
{
    return orc_energy(m, q) + orc_neg_entropy(m, q);
}

/* ------------------------------------------------------------------ */
/* the parallel proximal step  (Sec. 3.1-3.2)                          */
/* ------------------------------------------------------------------ */

static void log_softmax(const double *a, double *s, int L)
{
    double mx = a[0];
    for (int l = 1; l < L; ++l) if (a[l] > mx) mx = a[l];
    double z = 0.0;
    for (int l = 0; l < L; ++l) z += exp(a[l] - mx);
    double lse = mx + log(z);
    for (int l = 0; l < L; ++l) s[l] = a[l] - lse;
}

/* q^0 = softmax(-U): the unary-only marginals. */
void orc_init_logq(const orc_model *m, double *s)
{
    const int L = m->L;
    double *a = (double *)xcalloc((size_t)L, sizeof(double));
    for (int64_t i = 0; i < m->n; ++i) {
        for (int l = 0; l < L; ++l) a[l] = -m->U[i * L + l];
        log_softmax(a, s + i * L, L);
    }
    free(a);
}

/* One parallel proximal step with fixed step size (Eq. method:update_mean,
 * Eq. method:update_natural, Eq. fixedStepSize):
 *   theta^{t+1} = eta theta* + (1-eta) theta^t,  theta* = grad E(q^t),
 * written for the normalised log-domain state s = log q:
 *   a_il = -eta g_il + (1-eta) s_il,  s^{t+1}_i = a_i - logsumexp(a_i).
 * eta = 1 is the undamped FULL-PARALLEL update. */
void orc_prox_step(const orc_model *m, double eta, const double *s_in, double *s_out)
{
    const int L = m->L;
    const int64_t nl = m->n * L;
    double *q = (double *)malloc(sizeof(double) * (size_t)nl);
    double *g = (double *)malloc(sizeof(double) * (size_t)nl);
    for (int64_t k = 0; k < nl; ++k) q[k] = exp(s_in[k]);
    orc_grad(m, q, g);
#pragma omp parallel
    {
        double *a = (double *)xcalloc((size_t)L, sizeof(double));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m->n; ++i) {
            for (int l = 0; l < L; ++l)
                a[l] = -eta * g[i * L + l] + (1.0 - eta) * s_in[i * L + l];
            log_softmax(a, s_out + i * L, L);
        }
        free(a);
    }
    free(q);
    free(g);
}

/* The same step for the listed variables only (rows[r] in 0..n-1): out gets
 * log q^{t+1} of those variables, one row of L values each. */
void orc_prox_step_rows(const orc_model *m, double eta, const double *s_in, const int64_t *rows,
                        int64_t nrows, double *out)
{
    const int L = m->L;
    const int64_t nl = m->n * L;
    double *q = (double *)malloc(sizeof(double) * (size_t)nl);
    for (int64_t k = 0; k < nl; ++k) q[k] = exp(s_in[k]);
#pragma omp parallel
    {
        double *g = (double *)xcalloc((size_t)L, sizeof(double));
        double *a = (double *)xcalloc((size_t)L, sizeof(double));
#pragma omp for schedule(static)
        for (int64_t r = 0; r < nrows; ++r) {
            const int64_t i = rows[r];
            pair_grad_var(m, q, i, g);
            for (int l = 0; l < L; ++l)
                a[l] = -eta * (g[l] + m->U[i * L + l]) + (1.0 - eta) * s_in[i * L + l];
            log_softmax(a, out + r * L, L);
        }
        free(g);
        free(a);
    }
    free(q);
}

/* iters parallel proximal steps on s (in place).  F_trace, if given, gets
 * F(q^t) for t = 0..iters (iters+1 values). */
void orc_parallel_prox(const orc_model *m, double eta, int32_t iters, double *s,
                       double *F_trace)
{
    const int64_t nl = m->n * m->L;
    double *q = (double *)malloc(sizeof(double) * (size_t)nl);
    double *t = (double *)malloc(sizeof(double) * (size_t)nl);
    for (int32_t it = 0; it <= iters; ++it) {
        if (F_trace) {
            for (int64_t k = 0; k < nl; ++k) q[k] = exp(s[k]);
            F_trace[it] = orc_free_energy(m, q);
        }
        if (it == iters) break;
        orc_prox_step(m, eta, s, t);
        memcpy(s, t, sizeof(double) * (size_t)nl);
    }
    free(q);
    free(t);
}

/* Adaptive step for binary models (Sec. 3.3, Eq. hessian): the proximal
 * weights are d_{i,0} = d_{i,1} = d q_{i,0} q_{i,1}, taken from q^t, and
 * the update is Eq. method:update_mean with eta_i = 1/(1 + d_{i,l}).
 * Returns -1 (nothing written) unless L == 2. */
int32_t orc_prox_step_adaptive(const orc_model *m, double d, const double *s_in, double *s_out)
{
    if (m->L != 2) return -1;
    const int64_t nl = m->n * 2;
    double *q = (double *)malloc(sizeof(double) * (size_t)nl);
    double *g = (double *)malloc(sizeof(double) * (size_t)nl);
    for (int64_t k = 0; k < nl; ++k) q[k] = exp(s_in[k]);
    orc_grad(m, q, g);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m->n; ++i) {
        const double di = d * q[2 * i] * q[2 * i + 1];
        const double eta = 1.0 / (1.0 + di);
        double a[2];
        for (int l = 0; l < 2; ++l) a[l] = -eta * g[2 * i + l] + (1.0 - eta) * s_in[2 * i + l];
        log_softmax(a, s_out + 2 * i, 2);
    }
    free(q);
    free(g);
    return 0;
}

/* iters adaptive steps on s (in place); F_trace as in orc_parallel_prox. */
int32_t orc_parallel_prox_adaptive(const orc_model *m, double d, int32_t iters, double *s, double *F_trace)
{
    if (m->L != 2) return -1;
    const int64_t nl = m->n * 2;
    double *q = (double *)malloc(sizeof(double) * (size_t)nl);
    double *t = (double *)malloc(sizeof(double) * (size_t)nl);
    for (int32_t it = 0; it <= iters; ++it) {
        if (F_trace) {
            for (int64_t k = 0; k < nl; ++k) q[k] = exp(s[k]);
            F_trace[it] = orc_free_energy(m, q);
        }
        if (it == iters) break;
        orc_prox_step_adaptive(m, d, s, t);
        memcpy(s, t, sizeof(double) * (size_t)nl);
    }
    free(q);
    free(t);
    return 0;
}

/* OURS-MOMENTUM (Sec. 3.4, Eq. momentumUpdate): the gradient of Eq.
 * method:update_natural is replaced by its exponentially weighted average
 *   m^{t+1} = gamma1 m^t + (1 - gamma1) grad E(q^t),
 *   theta^{t+1} = eta m^{t+1} + (1 - eta) theta^t,
 * using the freshly formed m^{t+1}; the average starts from the first
 * gradient (m^1 = grad E(q^0)).  iters steps on s in place; F_trace as in
 * orc_parallel_prox. */
void orc_parallel_prox_momentum(const orc_model *m, double eta, double gamma1, int32_t iters, double *s,
                                double *F_trace)
{
    const int L = m->L;
    const int64_t nl = m->n * L;
    double *q = (double *)malloc(sizeof(double) * (size_t)nl);
    double *g = (double *)malloc(sizeof(double) * (size_t)nl);
    double *mom = (double *)malloc(sizeof(double) * (size_t)nl);
    double *a = (double *)malloc(sizeof(double) * (size_t)L);
    for (int32_t it = 0; it <= iters; ++it) {
        for (int64_t k = 0; k < nl; ++k) q[k] = exp(s[k]);
        if (F_trace) F_trace[it] = orc_free_energy(m, q);
        if (it == iters) break;
        orc_grad(m, q, g);
        for (int64_t k = 0; k < nl; ++k) mom[k] = it == 0 ? g[k] : gamma1 * mom[k] + (1.0 - gamma1) * g[k];
        for (int64_t i = 0; i < m->n; ++i) {
            for (int l = 0; l < L; ++l) a[l] = -eta * mom[i * L + l] + (1.0 - eta) * s[i * L + l];
            log_softmax(a, s + i * L, L);
        }
    }
    free(q);
    free(g);
    free(mom);
    free(a);
}

/* OURS-ADAM (Sec. 3.5, Eq. adamStepSize) with the momentum average above and
 * a per-(variable, label) proximal weight from the second moment of the
 * natural gradient.  Readings: the natural gradient is grad E + log q
 * centred over each variable's labels (zero exactly at a mean-field fixed
 * point, where log q = -grad E + const); v starts at 1 (the paper asks for a
 * strictly positive start) and is averaged as
 *   v^{t+1} = gamma2 v^t + (1 - gamma2) r^2;
 * d_{i,l} = sqrt(v^{t+1}) d0 + eps - 1, floored at 0 so that eta <= 1;
 * eta_{i,l} = 1/(1 + d_{i,l}) in Eq. method:update_natural with m^{t+1}. */
void orc_parallel_prox_adam(const orc_model *m, double d0, double gamma1, double gamma2, double eps,
                            int32_t iters, double *s, double *F_trace)
{
    const int L = m->L;
    const int64_t nl = m->n * L;
    double *q = (double *)malloc(sizeof(double) * (size_t)nl);
    double *g = (double *)malloc(sizeof(double) * (size_t)nl);
    double *mom = (double *)malloc(sizeof(double) * (size_t)nl);
    double *v = (double *)malloc(sizeof(double) * (size_t)nl);
    double *a = (double *)malloc(sizeof(double) * (size_t)L);
    for (int64_t k = 0; k < nl; ++k) v[k] = 1.0;
    for (int32_t it = 0; it <= iters; ++it) {
        for (int64_t k = 0; k < nl; ++k) q[k] = exp(s[k]);
        if (F_trace) F_trace[it] = orc_free_energy(m, q);
        if (it == iters) break;
        orc_grad(m, q, g);
        for (int64_t i = 0; i < m->n; ++i) {
            double mean = 0.0;
            for (int l = 0; l < L; ++l) mean += g[i * L + l] + s[i * L + l];
            mean /= L;
            for (int l = 0; l < L; ++l) {
                const int64_t k = i * L + l;
                const double r = g[k] + s[k] - mean;
                mom[k] = it == 0 ? g[k] : gamma1 * mom[k] + (1.0 - gamma1) * g[k];
                v[k] = gamma2 * v[k] + (1.0 - gamma2) * r * r;
                double dk = sqrt(v[k]) * d0 + eps - 1.0;
                if (dk < 0.0) dk = 0.0;
                const double eta = 1.0 / (1.0 + dk);
                a[l] = -eta * mom[k] + (1.0 - eta) * s[k];
            }
            log_softmax(a, s + i * L, L);
        }
    }
    free(q);
    free(g);
    free(mom);
    free(v);
    free(a);
}

/* ADHOC damping (Sec. 2.2.2, Eq. related:parallel-update): every variable
 * moves towards the solution of its own coordinate update,
 *   q^{t+1} = (1 - eta) q^t + eta softmax(-grad E(q^t)),
 * the damping applied to mean parameters (the paper's baseline).  iters
 * steps on s = log q in place; F_trace as in orc_parallel_prox. */
void orc_parallel_adhoc(const orc_model *m, double eta, int32_t iters, double *s, double *F_trace)
{
    const int L = m->L;
    const int64_t nl = m->n * L;
    double *q = (double *)malloc(sizeof(double) * (size_t)nl);
    double *g = (double *)malloc(sizeof(double) * (size_t)nl);
    double *a = (double *)malloc(sizeof(double) * (size_t)L);
    double *st = (double *)malloc(sizeof(double) * (size_t)L);
    for (int32_t it = 0; it <= iters; ++it) {
        for (int64_t k = 0; k < nl; ++k) q[k] = exp(s[k]);
        if (F_trace) F_trace[it] = orc_free_energy(m, q);
        if (it == iters) break;
        orc_grad(m, q, g);
        for (int64_t i = 0; i < m->n; ++i) {
            for (int l = 0; l < L; ++l) a[l] = -g[i * L + l];
            log_softmax(a, st, L);
            for (int l = 0; l < L; ++l)
                s[i * L + l] = log((1.0 - eta) * q[i * L + l] + eta * exp(st[l]));
        }
    }
    free(q);
    free(g);
    free(a);
    free(st);
}

/* SWEEP coordinate descent (Sec. 2.2.1, Eq. related:sweep-update): variables
 * in index (raster) order, each set to softmax(-grad E) computed from the
 * current values of all the others.  One call = sweeps full passes. */
void orc_sweep(const orc_model *m, int32_t sweeps, double *s)
{
    const int L = m->L;
    const int64_t nl = m->n * L;
    double *q = (double *)malloc(sizeof(double) * (size_t)nl);
    double *g = (double *)xcalloc((size_t)L, sizeof(double));
    for (int64_t k = 0; k < nl; ++k) q[k] = exp(s[k]);
    for (int32_t sw = 0; sw < sweeps; ++sw) {
        for (int64_t i = 0; i < m->n; ++i) {
            pair_grad_var(m, q, i, g);
            for (int l = 0; l < L; ++l) g[l] = -(g[l] + m->U[i * L + l]);
            log_softmax(g, s + i * L, L);
            for (int l = 0; l < L; ++l) q[i * L + l] = exp(s[i * L + l]);
        }
    }
    free(q);
    free(g);
}

/* ------------------------------------------------------------------ */
/* reverse-mode gradient of K unrolled steps                           */
/* ------------------------------------------------------------------ */

/* Loss of K unrolled parallel proximal steps from q^0 = softmax(-U), with a
 * fixed step eta: loss = -(1/n) sum_i log q^K_{i, y_i} (cross-entropy against
 * the label map y).  Returns the loss; fills dU [n][L], dmu [L][L] and dw
 * [n_edges] with its gradient, by the chain rule through every step taken
 * backwards in time (the step constant is held fixed).  Each step is
 *   q = exp(s),  m = H q (pairwise part of grad E),  a = -eta (U + m) + (1-eta) s,
 *   s' = a - logsumexp(a). */
double orc_unrolled_loss_grad(const orc_model *m, double eta, int32_t K, const int32_t *y,
                              double *dU, double *dmu, double *dw)
{
    const int L = m->L;
    const int64_t n = m->n, nl = n * L;
    double *S = (double *)malloc(sizeof(double) * (size_t)nl * (size_t)(K + 1));   /* s^0..s^K */
    double *q = (double *)malloc(sizeof(double) * (size_t)nl);
    double *gs = (double *)xcalloc((size_t)nl, sizeof(double));    /* d loss / d s^t */
    double *ga = (double *)xcalloc((size_t)nl, sizeof(double));
    double *gm = (double *)xcalloc((size_t)nl, sizeof(double));
    double *hq = (double *)xcalloc((size_t)nl, sizeof(double));
    double *qt = (double *)malloc(sizeof(double) * (size_t)nl);
    double *mq = (double *)malloc(sizeof(double) * (size_t)L);
    memset(dU, 0, sizeof(double) * (size_t)nl);
    memset(dmu, 0, sizeof(double) * (size_t)L * L);
    if (!m->K) memset(dw, 0, sizeof(double) * (size_t)m->ne);
    /* forward, keeping every state */
    orc_init_logq(m, S);
    for (int32_t t = 0; t < K; ++t) orc_prox_step(m, eta, S + (size_t)t * nl, S + (size_t)(t + 1) * nl);
    double loss = 0.0;
    for (int64_t i = 0; i < n; ++i) loss -= S[(size_t)K * nl + i * L + y[i]] / (double)n;
    for (int64_t i = 0; i < n; ++i) gs[i * L + y[i]] = -1.0 / (double)n;
    /* backward */
    for (int32_t t = K - 1; t >= 0; --t) {
        const double *st = S + (size_t)t * nl, *sn = S + (size_t)(t + 1) * nl;
        /* through s^{t+1} = a - logsumexp(a): ga = gs - q^{t+1} sum_l gs */
        for (int64_t i = 0; i < n; ++i) {
            double sum = 0.0;
            for (int l = 0; l < L; ++l) sum += gs[i * L + l];
            for (int l = 0; l < L; ++l) ga[i * L + l] = gs[i * L + l] - exp(sn[i * L + l]) * sum;
        }
        /* through a = -eta (U + m) + (1-eta) s */
        for (int64_t k = 0; k < nl; ++k) {
            dU[k] += -eta * ga[k];
            gm[k] = -eta * ga[k];
        }
        for (int64_t k = 0; k < nl; ++k) q[k] = exp(st[k]);
        /* through m = H q: H is symmetric, so dq = H gm; parameters by product rule */
        orc_hess_vec(m, gm, hq);
        if (m->K) {
            for (int64_t i = 0; i < n; ++i)
                for (int64_t j = i + 1; j < n; ++j) {
                    const double kij = m->K[i * n + j];
                    for (int a = 0; a < L; ++a)
                        for (int b = 0; b < L; ++b)
                            dmu[a * L + b] += kij * (gm[i * L + a] * q[j * L + b] + q[i * L + a] * gm[j * L + b]);
                }
        } else {
            for (int64_t e = 0; e < m->ne; ++e) {
                const int64_t i = m->ei[e], j = m->ej[e];
                const double *qi = q + i * L, *qj = q + j * L, *gi = gm + i * L, *gj = gm + j * L;
                /* edge energy w q_i^T mu q_j enters m_i as w mu q_j and m_j as w mu^T q_i */
                dw[e] += bilinear(gi, m->mu, qj, L) + bilinear(qi, m->mu, gj, L);
                for (int a = 0; a < L; ++a)
                    for (int b = 0; b < L; ++b)
                        dmu[a * L + b] += m->ew[e] * (gi[a] * qj[b] + qi[a] * gj[b]);
            }
        }
        /* through q = exp(s) and the direct (1-eta) s term */
        for (int64_t k = 0; k < nl; ++k) gs[k] = (1.0 - eta) * ga[k] + q[k] * hq[k];
    }
    /* through s^0 = logsoftmax(-U) */
    for (int64_t i = 0; i < n; ++i) {
        double sum = 0.0;
        for (int l = 0; l < L; ++l) sum += gs[i * L + l];
        for (int l = 0; l < L; ++l) {
            const double q0 = exp(S[i * L + l]);
            dU[i * L + l] += -(gs[i * L + l] - q0 * sum);
        }
    }
    (void)qt; (void)mq;
    free(S); free(q); free(gs); free(ga); free(gm); free(hq); free(qt); free(mq);
    return loss;
}

/* The loss alone (for finite differences). */
double orc_unrolled_loss(const orc_model *m, double eta, int32_t K, const int32_t *y)
{
    const int L = m->L;
    const int64_t nl = m->n * L;
    double *s = (double *)malloc(sizeof(double) * (size_t)nl);
    double *t = (double *)malloc(sizeof(double) * (size_t)nl);
    orc_init_logq(m, s);
    for (int32_t k = 0; k < K; ++k) {
        orc_prox_step(m, eta, s, t);
        memcpy(s, t, sizeof(double) * (size_t)nl);
    }
    double loss = 0.0;
    for (int64_t i = 0; i < m->n; ++i) loss -= s[i * L + y[i]] / (double)m->n;
    free(s); free(t);
    return loss;
}

/* ------------------------------------------------------------------ */
/* brute-force enumeration (tiny models only)                          */
/* ------------------------------------------------------------------ */

/* E(x) of a full labelling x (Eq. related:pairwise-mrf, energy = -log P + const). */
double orc_state_energy(const orc_model *m, const int32_t *x)
{
    const int L = m->L;
    double E = 0.0;
    for (int64_t i = 0; i < m->n; ++i) E += m->U[i * L + x[i]];
    if (m->K) {
        for (int64_t i = 0; i < m->n; ++i)
            for (int64_t j = i + 1; j < m->n; ++j)
                E += m->K[i * m->n + j] * m->mu[x[i] * L + x[j]];
    } else {
        for (int64_t e = 0; e < m->ne; ++e)
            E += m->ew[e] * m->mu[x[m->ei[e]] * L + x[m->ej[e]]];
    }
    return E;
}

static int64_t n_states(const orc_model *m)
{
    double c = pow((double)m->L, (double)m->n);
    if (c > (double)(1 << 22)) return -1;
    return (int64_t)llround(c);
}

static void next_state(int32_t *x, int64_t n, int L)
{
    for (int64_t i = 0; i < n; ++i) {
        if (++x[i] < L) return;
        x[i] = 0;
    }
}

/* Exact log Z and marginals P(x_i = l) by enumerating all L^n labellings.
 * Returns -1 if there are more than 2^22 states. */
int orc_brute_force(const orc_model *m, double *logZ, double *marg)
{
    int64_t ns = n_states(m);
    if (ns < 0) return -1;
    const int L = m->L;
    int32_t *x = (int32_t *)xcalloc((size_t)m->n, sizeof(int32_t));
    double *E = (double *)malloc(sizeof(double) * (size_t)ns);
    double mn = INFINITY;
    for (int64_t c = 0; c < ns; ++c) {
        E[c] = orc_state_energy(m, x);
        if (E[c] < mn) mn = E[c];
        next_state(x, m->n, L);
    }
    double z = 0.0;
    for (int64_t c = 0; c < ns; ++c) z += exp(-(E[c] - mn));
    *logZ = -mn + log(z);
    if (marg) {
        memset(marg, 0, sizeof(double) * (size_t)(m->n * L));
        memset(x, 0, sizeof(int32_t) * (size_t)m->n);
        for (int64_t c = 0; c < ns; ++c) {
            double p = exp(-E[c] - *logZ);
            for (int64_t i = 0; i < m->n; ++i) marg[i * L + x[i]] += p;
            next_state(x, m->n, L);
        }
    }
    free(x);
    free(E);
    return 0;
}

/* F(q) = sum_x Q(x) [E(x) + log Q(x)] by enumeration (Eq. related:mf-objective
 * taken literally), Q(x) = prod_i q_{i,x_i}.  NAN if too many states. */
double orc_brute_free_energy(const orc_model *m, const double *q)
{
    int64_t ns = n_states(m);
    if (ns < 0) return NAN;
    const int L = m->L;
    int32_t *x = (int32_t *)xcalloc((size_t)m->n, sizeof(int32_t));
    double F = 0.0;
    for (int64_t c = 0; c < ns; ++c) {
        double Q = 1.0;
        for (int64_t i = 0; i < m->n; ++i) Q *= q[i * L + x[i]];
        if (Q > 0.0) F += Q * (orc_state_energy(m, x) + log(Q));
        next_state(x, m->n, L);
    }
    free(x);
    return F;
}

/* out_il = E_{Q(X\X_i)}[E(x) | x_i = l] = sum_{x: x_i=l} prod_{j!=i} q_{j,x_j} E(x),
 * by enumeration (the quantity inside Eq. related:sweep-update). */
int orc_brute_cond_energy(const orc_model *m, const double *q, double *out)
{
    int64_t ns = n_states(m);
    if (ns < 0) return -1;
    const int L = m->L;
    int32_t *x = (int32_t *)xcalloc((size_t)m->n, sizeof(int32_t));
    memset(out, 0, sizeof(double) * (size_t)(m->n * L));
    for (int64_t c = 0; c < ns; ++c) {
        double E = orc_state_energy(m, x);
        for (int64_t i = 0; i < m->n; ++i) {
            double w = 1.0;
            for (int64_t j = 0; j < m->n; ++j)
                if (j != i) w *= q[j * L + x[j]];
            out[i * L + x[i]] += w * E;
        }
        next_state(x, m->n, L);
    }
    free(x);
    return 0;
}

/* ------------------------------------------------------------------ */
/* step-size constant  (Sec. 3.2)                                      */
/* ------------------------------------------------------------------ */

/* Cyclic Jacobi eigenvalue iteration on a symmetric n x n matrix A (row-major,
 * destroyed).  Eigenvalues go to ev, ascending. */
static void sort_asc(double *v, int64_t n)
{
    for (int64_t i = 1; i < n; ++i) {
        double t = v[i];
        int64_t j = i - 1;
        while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; --j; }
        v[j + 1] = t;
    }
}

void orc_jacobi_eigenvalues(int64_t n, double *A, double *ev)
{
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) {
                double a2 = A[i * n + j] * A[i * n + j];
                tot += a2;
                if (i != j) off += a2;
            }
        if (off <= 1e-30 * (tot > 0 ? tot : 1.0)) break;
        for (int64_t p = 0; p < n; ++p)
            for (int64_t r = p + 1; r < n; ++r) {
                double apr = A[p * n + r];
                if (fabs(apr) < 1e-300) continue;
                double app = A[p * n + p], arr = A[r * n + r];
                double theta = (arr - app) / (2.0 * apr);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J, J the rotation in the (p, r) plane */
                for (int64_t k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akr = A[k * n + r];
                    A[k * n + p] = c * akp - s * akr;
                    A[k * n + r] = s * akp + c * akr;
                }
                for (int64_t k = 0; k < n; ++k) {
                    double apk = A[p * n + k], ark = A[r * n + k];
                    A[p * n + k] = c * apk - s * ark;
                    A[r * n + k] = s * apk + c * ark;
                }
            }
    }
    for (int64_t i = 0; i < n; ++i) ev[i] = A[i * n + i];
    sort_asc(ev, n);
}

/* Project onto the tangent space of the simplex product:
 * (C v)_il = v_il - mean_l v_i. */
static void center(const orc_model *m, double *v)
{
    const int L = m->L;
    for (int64_t i = 0; i < m->n; ++i) {
        double s = 0.0;
        for (int l = 0; l < L; ++l) s += v[i * L + l];
        s /= L;
        for (int l = 0; l < L; ++l) v[i * L + l] -= s;
    }
}

/* All eigenvalues of the potential matrix H (the constant Hessian of E for a
 * pairwise model, Sec. 3.2), either as is (projected = 0) or restricted to
 * the tangent space, H_T = C H C (projected = 1).  The matrix is formed
 * column by column from Hessian-vector products.  n*L <= 2048. */
int orc_hessian_eigenvalues(const orc_model *m, int projected, double *ev)
{
    const int64_t nl = m->n * m->L;
    if (nl > 2048) return -1;
    double *A = (double *)xcalloc((size_t)(nl * nl), sizeof(double));
    double *e = (double *)xcalloc((size_t)nl, sizeof(double));
    double *h = (double *)xcalloc((size_t)nl, sizeof(double));
    for (int64_t c = 0; c < nl; ++c) {
        memset(e, 0, sizeof(double) * (size_t)nl);
        e[c] = 1.0;
        if (projected) center(m, e);
        orc_hess_vec(m, e, h);
        if (projected) center(m, h);
        for (int64_t r = 0; r < nl; ++r) A[r * nl + c] = h[r];
    }
    /* symmetrise away rounding */
    for (int64_t r = 0; r < nl; ++r)
        for (int64_t c = r + 1; c < nl; ++c) {
            double v = 0.5 * (A[r * nl + c] + A[c * nl + r]);
            A[r * nl + c] = A[c * nl + r] = v;
        }
    orc_jacobi_eigenvalues(nl, A, ev);
    free(A); free(e); free(h);
    return 0;
}

/* Extreme eigenvalues of H_T by the Lanczos method with full
 * re-orthogonalisation (the paper obtains the constant "by the power
 * method", Sec. 4.3; Lanczos is the Krylov refinement of it).  v0 is the
 * start vector (the caller's random draw).  Returns the iteration count. */
int32_t orc_lanczos_tangent(const orc_model *m, int32_t iters, const double *v0,
                            double *lmin, double *lmax)
{
    const int64_t nl = m->n * m->L;
    double *V = (double *)malloc(sizeof(double) * (size_t)nl * (size_t)(iters + 1));
    double *w = (double *)malloc(sizeof(double) * (size_t)nl);
    double *alpha = (double *)xcalloc((size_t)iters + 1, sizeof(double));
    double *beta = (double *)xcalloc((size_t)iters + 1, sizeof(double));
    if (!V || !w) { free(V); free(w); free(alpha); free(beta); return -1; }
    memcpy(V, v0, sizeof(double) * (size_t)nl);
    center(m, V);
    double nrm = 0.0;
    for (int64_t k = 0; k < nl; ++k) nrm += V[k] * V[k];
    nrm = sqrt(nrm);
    for (int64_t k = 0; k < nl; ++k) V[k] /= nrm;
    int32_t kdone = 0;
    for (int32_t it = 0; it < iters; ++it) {
        double *v = V + (size_t)it * nl;
        orc_hess_vec(m, v, w);
        center(m, w);
        double a = 0.0;
        for (int64_t k = 0; k < nl; ++k) a += v[k] * w[k];
        alpha[it] = a;
        kdone = it + 1;
        /* full re-orthogonalisation against all previous vectors, twice */
        for (int pass = 0; pass < 2; ++pass)
            for (int32_t j = 0; j <= it; ++j) {
                double *vj = V + (size_t)j * nl;
                double d = 0.0;
                for (int64_t k = 0; k < nl; ++k) d += vj[k] * w[k];
                for (int64_t k = 0; k < nl; ++k) w[k] -= d * vj[k];
            }
        double b = 0.0;
        for (int64_t k = 0; k < nl; ++k) b += w[k] * w[k];
        b = sqrt(b);
        beta[it] = b;
        if (b < 1e-13 || it + 1 == iters) break;
        double *vn = V + (size_t)(it + 1) * nl;
        for (int64_t k = 0; k < nl; ++k) vn[k] = w[k] / b;
    }
    /* eigenvalues of the tridiagonal Lanczos matrix */
    double *T = (double *)xcalloc((size_t)kdone * kdone, sizeof(double));
    double *ev = (double *)xcalloc((size_t)kdone, sizeof(double));
    for (int32_t i = 0; i < kdone; ++i) {
        T[i * kdone + i] = alpha[i];
        if (i + 1 < kdone) T[i * kdone + i + 1] = T[(i + 1) * kdone + i] = beta[i];
    }
    orc_jacobi_eigenvalues(kdone, T, ev);
    *lmin = ev[0];
    *lmax = ev[kdone - 1];
    free(T); free(ev); free(V); free(w); free(alpha); free(beta);
    return kdone;
}

/* eta = 1/(1+d) with d = max(Lambda, 0) (Eq. fixedStepSize; a non-positive
 * constant -- a negative semi-definite potential matrix -- gives the
 * undamped update, Sec. 3.2). */
double orc_step_size(double Lambda)
{
    double d = Lambda > 0.0 ? Lambda : 0.0;
    return 1.0 / (1.0 + d);
}
