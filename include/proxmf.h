/*
 * proxmf.h -- C ABI of the GB300 parallel proximal mean-field library.
 *
 * The library minimises the variational free energy
 *     F(q) = E_Q[E(x)] + sum_i sum_l q_il log q_il          (Sec. 2.2.1, Eq. related:mf-objective)
 * of a pairwise discrete random field (Sec. 2.1, Eq. related:pairwise-mrf)
 * over factorised distributions Q(x) = prod_i q_{i,x_i} (Eq. related:q-factorized),
 * with the fully parallel KL-proximal update of Sec. 3.1-3.2
 * (Eq. method:update_mean / method:update_natural, Eq. fixedStepSize):
 *     theta^{t+1} = eta grad E(q^t) + (1 - eta) theta^t,   q_il ∝ exp(-theta_il),
 *     eta = 1/(1+d), d = max(Lambda, 0),
 * where Lambda bounds the curvature of E on the simplex (Sec. 3.2).
 *
 * Energy convention (costs; the paper's potentials are phi = -cost):
 *     E(x) = sum_i U[i, x_i] + sum_{edges i->j} w_ij mu[x_i, x_j].
 *
 * Conventions shared by every call:
 *   - Every call returns a crf_status; nothing aborts or throws across the ABI.
 *   - A handle owns all of its device memory; inputs are copied when set; the
 *     caller owns every output buffer.
 *   - Work is ordered on the handle's stream (crf_desc.stream).  Calls that
 *     return host values synchronise that stream before returning.
 *   - Pointers flagged is_device = 1 are device pointers of the current CUDA
 *     device; is_device = 0 means host memory (pinned or pageable).
 *   - External layout of per-variable arrays is [batch][N][L] row-major, N =
 *     height*width, variable p = y*width + x.  The internal device layout is
 *     private (pixel-major, label count padded) and converted when data is
 *     set or read.
 *   - A handle is used by one host thread at a time.
 *   - A CUDA error is reported as CRF_E_CUDA and makes the handle unusable
 *     (later calls return CRF_E_STATE).
 *   - Every wait inside a kernel is bounded (about 2 s).  When a step
 *     kernel's wait runs out, the call returns CRF_E_TIMEOUT and the handle
 *     becomes unusable as well (copies or tensor-core operations it waited
 *     for may still have been in flight): destroy it and create a new one.
 *     The Lanczos grid barriers of mf_lipschitz are the exception (below).
 */
#ifndef PROXMF_H
#define PROXMF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct crf_s *crf_t;

typedef enum {
    CRF_OK = 0,
    CRF_E_INVALID = -1,     /* bad argument, size or call order              */
    CRF_E_OOM = -2,         /* device allocation failed                      */
    CRF_E_CUDA = -3,        /* a CUDA call failed; the handle is now broken  */
    CRF_E_STATE = -4,       /* handle broken by an earlier CUDA error        */
    CRF_E_TIMEOUT = -5,     /* a bounded wait ran out                        */
    CRF_E_NUMERIC = -6,     /* a non-finite free energy was produced         */
    CRF_E_UNSUPPORTED = -7  /* valid request outside what this build covers  */
} crf_status;

typedef enum {
    CRF_GRID4 = 0,          /* 4-connected H x W grid                         */
    CRF_GRID8 = 1,          /* 8-connected H x W grid                         */
    CRF_DENSE_GAUSS = 2,    /* fully connected, Gaussian kernel over features */
    CRF_SPARSE = 3          /* general pairwise graph from an edge list       */
                            /* (crf_set_graph); N = height*width variables    */
} crf_topology;

typedef enum {
    CRF_FP32 = 0,           /* FP32 messages, FP32 state                     */
    CRF_BF16 = 1            /* BF16 tensor-core messages, FP32 state: dense  */
                            /* N x N product (fully connected) or the L x L  */
                            /* product (grids); FP32 accumulation.  The F    */
                            /* trace of a BF16 step uses its BF16 messages;  */
                            /* mf_free_energy and final_free_energy always   */
                            /* use FP32 messages                             */
} crf_precision;

typedef struct {
    int32_t topology;       /* crf_topology                                   */
    int32_t n_labels;       /* L: 1..32 (grids, sparse), 1..24 (fully connected) */
    int32_t batch;          /* independent instances with the same shape, >= 1 */
    int32_t precision;      /* crf_precision                                  */
    int64_t height;         /* grid rows; dense: N = height*width variables   */
    int64_t width;          /* grid columns                                   */
    void *stream;           /* cudaStream_t; NULL = the legacy default stream */
} crf_desc;

/* crf_create -- allocate a handle and its device storage for desc.
 * Defines the model of Sec. 2.1 (Eq. related:pairwise-mrf) on the given
 * topology.  Fails with CRF_E_INVALID for sizes out of range, CRF_E_OOM if
 * the device storage cannot be allocated.  *out is NULL on failure. */
crf_status crf_create(const crf_desc *desc, crf_t *out);

/* crf_destroy -- synchronise the handle's stream and free everything.
 * NULL is accepted. */
crf_status crf_destroy(crf_t h);

/* crf_set_unary -- unary energies U = -phi_i of Eq. related:pairwise-mrf,
 * [batch][N][L] float32.  Copied into the handle; the mean-field state is
 * reset to q^0 = softmax(-U) (the unary-only marginals). */
crf_status crf_set_unary(crf_t h, const float *U, int is_device);

/* crf_set_pairwise -- the pairwise term phi_ij = -w_ij mu[x_i, x_j].
 *   mu   [L][L] float32, shared by all instances; mu[l*L+m] is the cost of
 *        (x_i = l, x_j = m) on an edge oriented i -> j.
 *   grid: w_or_feats = w [batch][n_dirs][H][W] float32 (n_dirs = 2 for GRID4:
 *        right, down; 4 for GRID8: right, down, down-right, down-left); the
 *        entry at (y, x) weights the edge leaving (y, x) in that direction;
 *        entries whose edge would leave the image are ignored.  theta unused.
 *   dense: w_or_feats = features [batch][N][5] (x, y, r, g, b) and theta[2] =
 *        {theta_pos, theta_rgb}; w_ij = exp(-|dp|^2/(2 theta_pos^2)
 *        - |dc|^2/(2 theta_rgb^2)) for i != j; mu must be symmetric.
 * Invalidates the cached step-size constant (recomputed on demand). */
crf_status crf_set_pairwise(crf_t h, const float *mu, const float *w_or_feats,
                            const float *theta, int is_device);

/* crf_set_state -- import a mean-field state as log q, [batch][N][L] float32
 * (each row should be a normalised log-distribution; it is used as given).
 * Checkpoint / resume, and identical starting points for parity checks. */
crf_status crf_set_state(crf_t h, const float *logq, int is_device);

/* crf_set_graph -- pairwise term of a CRF_SPARSE handle (Sec. 2.1, Eq.
 * related:pairwise-mrf on an arbitrary edge set): n_edges oriented edges
 * src[e] -> dst[e] (0 <= index < N, src != dst) with weights w[e] (finite)
 * and mu [L][L] (cost of x_src = l, x_dst = l'), shared by all instances of
 * the batch.  Arrays are device pointers if is_device = 1, else host.  The
 * step-size constant of a sparse graph is replaced by a bound on it (no
 * Lanczos): Lambda <= D max|eig(C mu C)| for symmetric mu, D the largest
 * summed |w| of a variable's edges; (D_out + D_in) ||mu||_F otherwise.  The
 * bound is >= Lambda, so eta = 1/(1+bound) keeps the descent guarantee.
 * CRF_E_INVALID for a handle of another topology or a bad index. */
crf_status crf_set_graph(crf_t h, const float *mu, int64_t n_edges, const int32_t *src, const int32_t *dst,
                         const float *w, int32_t is_device);

typedef struct {
    double eta;             /* > 0: fixed step eta (1 = FULL-PARALLEL);        */
                            /* <= 0: eta = 1/(1+max(Lambda,0)) (Sec. 3.2)       */
    int32_t max_iters;      /* iterations to run (>= 0)                         */
    int32_t reset;          /* 1: restart from q^0 = softmax(-U) first          */
    double rel_tol;         /* > 0: instance b stops after the step at which    */
                            /* |F^t - F^{t-1}| <= rel_tol |F^t| (stopping rule  */
                            /* on the objective, Sec. 3.1); 0: fixed count      */
    int32_t refine_fp32;    /* BF16 form: FP32 iterations run after max_iters   */
                            /* (counted in iters_done and the F trace)          */
    int32_t final_free_energy; /* 1: also evaluate F(q^K) on the device at the */
                            /* end (mf_free_energy then returns it without a    */
                            /* recomputation); no host synchronisation          */
    int32_t rule;           /* MF_RULE_FIXED (0): one eta for all variables     */
                            /* (Eq. fixedStepSize); MF_RULE_ADAPTIVE (1):        */
                            /* binary grids only, per-variable                   */
                            /* eta_i = 1/(1 + d q_i0 q_i1) from q^t (Sec. 3.3,   */
                            /* Eq. hessian), eta ignored; MF_RULE_MOMENTUM (2):  */
                            /* the gradient replaced by its running average      */
                            /* m' = gamma1 m + (1-gamma1) grad E, started at the */
                            /* first gradient (Sec. 3.4, Eq. momentumUpdate);    */
                            /* MF_RULE_ADAM (3): momentum plus a per-label eta   */
                            /* = 1/(1 + max(sqrt(v') d + epsilon - 1, 0)) from   */
                            /* v' = gamma2 v + (1-gamma2) r^2, r the natural     */
                            /* gradient grad E + log q centred over labels, v    */
                            /* starting at 1 (Sec. 3.5, Eq. adamStepSize), eta   */
                            /* ignored; MF_RULE_ADHOC (4): the paper's baseline  */
                            /* damping of the mean parameters,                   */
                            /* q' = (1-eta) q + eta softmax(-grad E) (Sec. 2.2.2,*/
                            /* Eq. related:parallel-update).  Rules 2-4: FP32    */
                            /* grids only; each mf_iterate call starts a new run */
                            /* (no history).                                     */
    double d;               /* MF_RULE_ADAPTIVE, MF_RULE_ADAM: d > 0 as given;   */
                            /* d <= 0: the step-size constant max(Lambda, 0)     */
    double gamma1;          /* MF_RULE_MOMENTUM, MF_RULE_ADAM: in [0, 1]         */
    double gamma2;          /* MF_RULE_ADAM: in [0, 1]                           */
    double epsilon;         /* MF_RULE_ADAM: >= 0                                */
} mf_params;

enum { MF_RULE_FIXED = 0, MF_RULE_ADAPTIVE = 1, MF_RULE_MOMENTUM = 2, MF_RULE_ADAM = 3, MF_RULE_ADHOC = 4 };

/* mf_iterate -- run the parallel proximal iteration of Eq. method:update_natural.
 * rule = MF_RULE_ADAPTIVE on a model that is not a binary grid, and rules
 * MF_RULE_MOMENTUM / MF_RULE_ADAM / MF_RULE_ADHOC on a fully connected or
 * BF16 handle, return CRF_E_UNSUPPORTED.
 * Each step computes grad E(q^t) (expected pairwise energy plus unaries),
 * takes the log-domain proximal step, renormalises every variable, and
 * records F(q^t).  iters_done (host, [batch], may be NULL) receives the
 * number of steps each instance actually took.  Requires unary and pairwise
 * terms to be set. */
crf_status mf_iterate(crf_t h, const mf_params *p, int32_t *iters_done);

/* mf_free_energy -- F(q) of the current state per instance (Eq.
 * related:mf-objective), FP64, host array [batch]. */
crf_status mf_free_energy(crf_t h, double *F);

/* mf_free_energy_trace -- F(q^t), t = 0 .. n-1, recorded by the last
 * mf_iterate call, host array [batch][n]; n <= that call's max_iters.
 * Entries after an instance stopped early are left as recorded (stale). */
crf_status mf_free_energy_trace(crf_t h, double *F, int32_t n);

/* mf_marginals -- q (Eq. related:definition_q), [batch][N][L] float32. */
crf_status mf_marginals(crf_t h, float *q, int is_device);

/* mf_log_marginals -- log q, [batch][N][L] float32 (the log-domain state). */
crf_status mf_log_marginals(crf_t h, float *logq, int is_device);

/* mf_lipschitz -- the step-size constant Lambda (largest eigenvalue of the
 * constant Hessian of E restricted to the tangent space of the simplex
 * product, Sec. 3.2) and eta = 1/(1+max(Lambda,0)), one per instance: host
 * arrays [batch] (either may be NULL).  Computed on the device by a Lanczos
 * iteration on first use after crf_set_pairwise (also by mf_iterate with
 * eta <= 0); synchronises the stream.  On grids with symmetric mu the
 * Lanczos chain runs as cooperative launches whose grid barriers wait at
 * most ~2 s each: a wait that runs out returns CRF_E_TIMEOUT, leaves the
 * constant unset and the handle usable. */
crf_status mf_lipschitz(crf_t h, double *Lambda, double *eta);

/* mf_profile -- enable (1) or disable (0) event timing of the iteration
 * loop: while enabled, mf_iterate, mf_unrolled_forward and
 * mf_unrolled_backward bracket their step launches (K forward steps; K
 * reverse steps of two kernels each) with two CUDA events on the handle's
 * stream.  No synchronisation. */
crf_status mf_profile(crf_t h, int32_t enable);

/* mf_profile_read -- device time of the last profiled iteration loop in ms
 * and the number of step launches it contained (host scalars).  Waits for
 * the loop's end event. */
crf_status mf_profile_read(crf_t h, double *loop_ms, int32_t *launches);

/* mf_use_resident -- 1 (the default): mf_iterate on a grid handle whose
 * iterates fit in the shared memory of a thread-block cluster (up to 8 CTAs
 * per instance, each holding a slab of rows: 4 x rows x W x L_stored floats
 * <= 200 KB per CTA, L <= 16), FP32 form, fixed rule and at least two steps
 * runs the whole loop in one launch (a cluster barrier between steps) and
 * records it as one launch; 0: one launch per step.  Same traces, stopping
 * rule and final state, up to FP32 rounding.  Returns CRF_E_INVALID for a
 * null handle. */
crf_status mf_use_resident(crf_t h, int32_t enable);

/* mf_dense_on_the_fly -- dense handles of precision CRF_BF16 only: 1 makes
 * the tensor-core steps compute the Gaussian weights w_ij of the fully
 * connected model (crf_set_pairwise, dense) inside the kernel from the
 * features instead of reading the BF16 copy of them made at crf_set_pairwise;
 * 0 (the default) reads the copy.  Both round K to BF16 and
 * accumulate the message in FP32; the weights agree to the rounding of the
 * exponential.  FP32 steps (refinement) and the step constant keep using the
 * FP32 K.  Returns CRF_E_UNSUPPORTED for other handles.  No synchronisation. */
crf_status mf_dense_on_the_fly(crf_t h, int32_t enable);

/* mf_use_graphs -- 1: mf_iterate records its step launches into a CUDA
 * graph the first time a configuration (max_iters, refine_fp32, rel_tol, the
 * step-size source, the parity of the state buffers) is seen and replays the
 * graph afterwards, which removes the host launch cost per step (small
 * problems are launch-bound); 0 (default): launches are issued one by one.
 * Graphs hold the handle's device buffers and are dropped when the free-
 * energy trace is regrown or the handle is destroyed.  Results are identical
 * either way. */
crf_status mf_use_graphs(crf_t h, int32_t enable);

/* crf_launch_count -- number of kernels this handle has launched so far. */
crf_status crf_launch_count(crf_t h, int64_t *n);

/* Differentiable unrolled inference (reverse mode through K steps).
 *
 * The paper derives the forward iteration only (Sec. 3.1-3.2); the reverse
 * pass is the chain rule through K parallel proximal steps (Eq.
 * method:update_natural) taken from q^0 = softmax(-U) with a step eta that is
 * held constant (not differentiated through Lambda).  Grid topologies only,
 * n_labels <= 24; other handles return CRF_E_UNSUPPORTED.
 *
 * mf_unrolled_checkpoint_floats -- number of floats (4 bytes each) the
 *   checkpoint buffer of a K-step forward needs: (K+1) states s^0..s^K in
 *   the private padded layout.  The caller owns that device buffer (for
 *   autograd it lives as long as the saved tensors).
 *
 * mf_unrolled_forward -- reset to s^0 = log softmax(-U), take K steps
 *   (1 <= K <= 4096) with step eta (0 < eta <= 1: the same eta for every
 *   instance; eta <= 0: each instance's 1/(1+max(Lambda,0)), computed once
 *   as in mf_iterate), write s^0..s^K into ckpt (device, at least
 *   mf_unrolled_checkpoint_floats(K) floats, 16-byte aligned), and leave
 *   the handle's state at s^K (mf_marginals / mf_log_marginals read it;
 *   mf_free_energy_trace(K) gives F(q^0..q^{K-1})).  The handle's unary and
 *   pairwise terms must be set.  A CRF_BF16 handle takes the K steps with
 *   BF16 tensor-core messages; the reverse pass is then the FP32 adjoint of
 *   the step map evaluated along that trajectory.
 *
 * mf_unrolled_backward -- gradients of a scalar loss given dlogq = d loss /
 *   d log q^K ([batch][N][L], external layout).  Needs the ckpt of a forward
 *   with the same K and eta on this handle, with unary and pairwise terms
 *   unchanged since.  Writes
 *     dU   [batch][N][L]            d loss / d U
 *     dmu  [L][L]                   d loss / d mu (summed over the batch,
 *                                   since mu is shared)
 *     dw   [batch][n_dirs][H][W]    d loss / d w, layout of crf_set_pairwise
 *                                   (zero for edges that leave the grid).
 *   Any output may be NULL (not written).  All four arrays are device
 *   pointers if is_device = 1, else host.  Accumulation order is fixed, so
 *   results repeat bit for bit.  Scratch memory (about 3 states, the
 *   weights and (B*N/128) L x L partials) is allocated on first use and kept
 *   by the handle.
 */
crf_status mf_unrolled_checkpoint_floats(crf_t h, int32_t K, int64_t *n_floats);
crf_status mf_unrolled_forward(crf_t h, int32_t K, double eta, float *ckpt);
crf_status mf_unrolled_backward(crf_t h, int32_t K, double eta, const float *ckpt, const float *dlogq,
                                float *dU, float *dmu, float *dw, int32_t is_device);

/* mf_grid_step_noalloc -- one parallel proximal step of a single grid
 * instance on caller-owned device buffers, for callers that cannot allocate
 * device memory (an allocator or memory pool that owns the device, a region
 * where cudaMalloc is forbidden or would synchronise).  The paper has no
 * counterpart: this is an integration entry point, not a step of the method.
 *   topology   CRF_GRID4 or CRF_GRID8; n_labels L in 1..32.
 *   U, logq_in, logq_out  pixel-major [height][width][Lp] float32, device,
 *              with Lp = L rounded up to a multiple of 4 (2 when L <= 2);
 *              padding entries must hold U = 0 and log q = -1e30, and the
 *              step writes -1e30 there.
 *   w          pixel-major [height][width][n_dirs] float32, device, same
 *              directions as crf_set_pairwise; entries whose edge leaves the
 *              image must be 0.
 *   mu         [L][L] float32, HOST memory.
 *   eta        step in (0, 1].
 *   F_out      device double: receives F(q_in); NaN when the step reports
 *              an error or F is not finite (inf or NaN).
 *   stream     cudaStream_t (NULL = legacy default stream).
 * Allocates nothing: its scratch (tile partials, counter, status, step, mu
 * table) is a 512 KiB static device array, held on every GPU that loads the
 * library until exit, which limits one call to 64480 tiles of 32 x 8 pixels
 * (CRF_E_INVALID beyond).  The first call on a device looks up that array's address (make it
 * before any stream capture).  All calls share the array: calls that overlap
 * on the GPU race and must be serialised by the caller.  logq_in and logq_out
 * must not alias.  mu is read before the call returns (it travels to the
 * device as kernel parameters; no host buffer is copied asynchronously).
 * Asynchronous: three kernel launches on the stream (set-up, step, finish);
 * errors of the launches are CRF_E_CUDA. */
crf_status mf_grid_step_noalloc(int32_t topology, int32_t n_labels, int64_t height,
                                int64_t width, const float *U, const float *w,
                                const float *mu, const float *logq_in, float *logq_out,
                                double eta, double *F_out, void *stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of many grid CRFs on one GPU (the request loop of a
 * serving deployment).  A server owns one device pool of budget_bytes; each
 * request (one grid CRF: batch 1, FP32) is copied on submit and queued.
 * mf_server_step retires finished requests (q copied to the request's q_out,
 * slot and pool memory returned), admits queued requests in arrival order as
 * slots and pool memory allow, and then advances every in-flight request by
 * `iters` proximal steps -- one persistent launch per label class per step,
 * replayed from a CUDA graph.  A request stops after max_iters steps or when
 * |F^t - F^{t-1}| <= rel_tol |F^t| (Sec. 3.1), exactly as mf_iterate would
 * stop it, and its arithmetic does not depend on the other requests.
 * eta <= 0 asks for eta = 1/(1 + D max|nu|) with D the largest weighted degree
 * and nu the eigenvalues of C mu C: an upper bound of the step-size constant
 * of Sec. 3.2 (so the descent guarantee holds) that costs no iteration; it
 * needs a symmetric mu.  One server is driven by one host thread. */
typedef struct mf_server_s *mf_server_t;

/* mf_server_create -- max_slots in 1..256 requests in flight; stream as in
 * crf_desc.  CRF_E_OOM if the pool cannot be allocated. */
crf_status mf_server_create(int64_t budget_bytes, int32_t max_slots, void *stream, mf_server_t *out);

/* mf_server_destroy -- waits for the stream, frees the pool. */
crf_status mf_server_destroy(mf_server_t s);

/* mf_server_submit -- queue one request.  d: GRID4/GRID8, batch 1, FP32.
 * U [N][L], mu [L][L], w [n_dirs][H][W]: host arrays, copied now.  q_out:
 * host [N][L] receiving the marginals when the request finishes (may be
 * NULL), must stay valid until then.  *ticket identifies the request.
 * CRF_E_OOM if the request alone exceeds the pool; CRF_E_UNSUPPORTED for a
 * rule other than MF_RULE_FIXED. */
crf_status mf_server_submit(mf_server_t s, const crf_desc *d, const float *U, const float *mu, const float *w,
                            const mf_params *p, float *q_out, uint64_t *ticket);

/* mf_server_step -- retire, admit, then run `iters` steps of every in-flight
 * request (asynchronous on the stream).  Reports the requests in flight and
 * still queued. */
crf_status mf_server_step(mf_server_t s, int32_t iters, int32_t *in_flight, int32_t *queued);

/* mf_server_poll -- state of a request: 0 queued, 1 running, 2 done (its q_out
 * written); F is F(q^{K-1}) of its last step and iters the steps it took. */
crf_status mf_server_poll(mf_server_t s, uint64_t ticket, int32_t *state, double *F, int32_t *iters);

/* mf_server_sync -- wait for the server's stream. */
crf_status mf_server_sync(mf_server_t s);

/* crf_error_string -- static description of a status code. */
const char *crf_error_string(crf_status s);

/* crf_version -- library version string. */
const char *crf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PROXMF_H */
