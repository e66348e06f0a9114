/*
 * vomt.h -- C ABI of the GB300 (sm_103a) solver for vector- and matrix-valued
 * L1 optimal mass transport by the primal-dual hybrid gradient (PDHG) method of
 * Ryu, Chen, Li and Osher, "Vector and Matrix Optimal Mass Transport: Theory,
 * Algorithm, and Applications" (arXiv:1712.10279).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.  An n x n grid on [0,1]^2 with spacing h = 1/(n-1) (Section 7 and
 *   Appendix A).  Every grid field is FP32, stored plane by plane as
 *   [plane][j][i] with the x index i fastest: element (i, j) of plane p sits at
 *   (p*n + j)*pitch + i, with the row pitch given by vomt_params.pitch (or the
 *   pitch argument of vomt_backward) and n (dense) by default.
 * Densities.  Cell masses (the finite-volume averages of Appendix A).  For the
 *   vector problem rho0 and rho1 are [k][n][n] and must be nonnegative with
 *   equal totals over all cells and channels (the constraint of eq. (vomt)
 *   sums to zero because div_x and div_G do).
 * Flux and potential.  u is [2][k][n][n]: the x components u_x (plane c) then
 *   the y components u_y (plane k + c).  Entries u_x(n-1, j) and u_y(i, n-1)
 *   are the ghost cells of Appendix A: they are ignored on input and are zero
 *   on output.  w is [l][n][n] (one plane per graph edge, in the order the
 *   edges are given).  phi is [k][n][n].
 * Memory.  "device" pointers are CUDA global memory of the context's device,
 *   owned by the caller (for example torch tensors); the library never frees
 *   or keeps them after the call returns.  "host" pointers are ordinary host
 *   memory (pageable or pinned).
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  All device work of a call is ordered on that stream.  A solve
 *   that stops on a tolerance reads its stopping flag back while it runs and
 *   returns only after its last kernel finished, so outputs and *result are
 *   valid when the call returns.
 * Status.  Every entry point returns an int: VOMT_OK (0), VOMT_NOT_CONVERGED
 *   (1, outputs valid, iteration cap reached before the tolerance) or a
 *   negative VOMT_ERR_* code.  No entry point aborts the process or lets an
 *   exception escape.  vomt_last_error() gives a message for the last error
 *   on a context.
 * Threads.  A context may be used by one host thread at a time.
 */
#ifndef VOMT_H
#define VOMT_H

#ifdef __cplusplus
extern "C" {
#endif

#define VOMT_OK                      0
#define VOMT_NOT_CONVERGED           1
#define VOMT_ERR_BAD_ARG            -1   /* a size, pointer or parameter is invalid */
#define VOMT_ERR_MASS_MISMATCH      -2   /* |sum rho0 - sum rho1| > 1e-6 max(sum rho0, sum rho1) */
#define VOMT_ERR_NEGATIVE_DENSITY   -3   /* some density entry < 0 */
#define VOMT_ERR_GRAPH              -4   /* channel graph not connected, self loop or repeated edge */
#define VOMT_ERR_L_KERNEL           -5   /* ker grad_L on symmetric matrices is larger than span{I} */
#define VOMT_ERR_STEP_CONDITION     -6   /* user step sizes break 1 > tau mu 8(n-1)^2 + tau nu lmax */
#define VOMT_ERR_NONFINITE          -7   /* an input or an iterate became NaN / Inf */
#define VOMT_ERR_BARRIER_TIMEOUT    -8   /* a device-side wait ran out of its iteration budget */
#define VOMT_ERR_CUDA               -9   /* a CUDA runtime call failed (see vomt_last_error) */
#define VOMT_ERR_TOO_LARGE         -10   /* the problem exceeds a documented size limit */

/* Norm choices (Section 6.2).  u: per-channel Euclidean summed over channels
 * (||u||_{1,2}, the Table 1 setting), joint Euclidean (||u||_2) or entrywise
 * (||u||_1).  w: entrywise (||w||_1) or joint Euclidean (||w||_2). */
#define VOMT_U_L12 0
#define VOMT_U_L2  1
#define VOMT_U_L1  2
#define VOMT_W_L1  0
#define VOMT_W_L2  1
#define VOMT_U_NUC 3   /* matrix OMT: ||U||_{1,nuc} = ||U_x||_nuc + ||U_y||_nuc (Section 6.2) */
#define VOMT_W_NUC 2   /* matrix OMT: ||W||_{1,nuc} = sum_s ||W_s||_nuc (Section 6.2) */

/* Engines.  AUTO picks RESIDENT when the whole state fits in the SMs'
 * registers and shared memory, else STREAM. */
#define VOMT_ENGINE_AUTO      0
#define VOMT_ENGINE_STREAM    1   /* one fused stencil launch per iteration, state in HBM */
#define VOMT_ENGINE_RESIDENT  2   /* one persistent launch, state on chip for the whole solve */

#define VOMT_MAX_CHANNELS 8        /* k <= 8, so l <= 28 */

typedef struct vomt_ctx vomt_ctx;

/* The channel graph of Section 3.1: k nodes, l undirected edges {tail[e], head[e]}
 * (0-based, any order inside a pair; each edge is oriented from its smaller to
 * its larger node).  cost[e] > 0 is the cost c_e of changing along edge e
 * (edge weight 1/c_e^2); cost == NULL means every c_e = 1.  Host memory. */
typedef struct {
    int k;
    int n_edges;
    const int *tail;
    const int *head;
    const double *cost;
} vomt_graph;

typedef struct {
    double tau;          /* dual step; <= 0 picks Table 1's value: 1 for n <= 64, else 3 */
    double mu, nu;       /* primal steps; <= 0 picks Section 7.2's rule
                            mu = 1/(32 tau (n-1)^2), nu = 1/(4 tau lambda_max(-Delta_G));
                            for l = 0 the scalar rule mu = 1/(16 tau (n-1)^2) of Section 7.1 */
    int u_norm, w_norm;  /* VOMT_U_*, VOMT_W_* */
    int max_iters;       /* iteration cap (>= 0) */
    int check_every;     /* iterations between FP64 convergence checks (>= 1) */
    double tol_gap;      /* stop when rel_gap <= tol_gap and rel_res <= tol_res; tol_gap <= 0
                            runs exactly max_iters iterations */
    double tol_res;
    int warm_start;      /* 1: u, w, phi hold the initial iterate; 0: start from zero (Section 7
                            leaves the initial guess open; zero is this library's default) */
    int engine;          /* VOMT_ENGINE_* */
    int halo;            /* resident engine: iterations between halo exchanges, 1..16 (0 = the
                            plan's estimate; a one-tile grid never exchanges) */
    double eps;          /* >= 0: quadratic regularisation of the paper's concluding section,
                            eps (||u(x)||_2^2 + ||w(x)||_2^2) added at every point (Euclidean
                            norms, so the problem is strictly convex); each primal step is then
                            the shrink of v / (1 + 2 t eps) with threshold t / (1 + 2 t eps), P
                            includes the term and D subtracts sum dist_2(., dual ball)^2 /
                            (4 eps).  0 (default) is the plain problem.  Vector OMT, forward
                            solves (vomt_unrolled_grad and momt_solve take eps = 0 only). */
    int pitch;           /* row pitch in floats of every grid array of vomt_solve, vomt_solve_host
                            and momt_solve: element (i, j) of plane p at (p*n + j)*pitch + i,
                            so that rows may be padded (e.g. to 16 bytes, or views of larger
                            arrays).  0 (default) means pitch = n (dense); else pitch >= n.
                            Pitched arrays are staged densely by the library (one 2-D copy per
                            array in, one per output array out), so the solve itself is the
                            same.  The other entry points take dense arrays. */
} vomt_params;

typedef struct {
    double primal;       /* P = sum_ij ||u_ij||_u + alpha sum_ij ||w_ij||_w (Appendix A), plus the
                            eps term when regularised */
    double dual;         /* D = sum_ij <phi_ij, rho1_ij - rho0_ij> (eq. vomt-dual), minus the
                            conjugate terms of the regulariser when eps > 0 */
    double rel_gap;      /* |P - D| / |P|, the measure of Section 8.1 */
    double rel_res;      /* ||div_x u + div_G w - (rho0 - rho1)||_2 / ||rho0 - rho1||_2 */
    double fp_resid;     /* R of Section 6.1 between the last two iterates, weights 1/mu, 1/nu, 1/tau */
    double dual_infeas;  /* max_ij max(||grad phi||_{u*} - 1, ||grad_G phi||_{w*} - alpha, 0) */
    double mu, nu, tau;  /* step sizes used */
    int iters;           /* iterations run */
    int status;          /* VOMT_OK or VOMT_NOT_CONVERGED */
    int engine;          /* engine that ran */
    int checks;          /* convergence checks run */
    int launches;        /* CUDA kernels this call launched */
    int blocks;          /* thread blocks of the main launch (resident: one tile each) */
    int halo;            /* resident engine: iterations between halo exchanges (0 otherwise) */
    int variant;         /* form of the main step kernel: 1 = inputs staged by TMA tiles,
                            0 = per-thread loads (streaming and 3-D solves); for
                            vomt_solve_batched: 1 = the solve ran as one CUDA graph launch */
} vomt_result;

/* Create a context on CUDA device `device`.  The context owns the solver's
 * scratch memory (double-buffered iterates, FP64 partial sums, status words),
 * grown on demand and freed by vomt_destroy.  Returns VOMT_OK or an error. */
int vomt_create(vomt_ctx **out, int device);
void vomt_destroy(vomt_ctx *ctx);
const char *vomt_status_str(int status);
const char *vomt_last_error(const vomt_ctx *ctx);

/* Fill *p with the defaults: tau, mu, nu from the paper's rules, ||u||_{1,2},
 * ||w||_1, max_iters 2000, check_every 100, tol_gap = tol_res = 0, cold start,
 * engine AUTO, halo 0. */
void vomt_default_params(vomt_params *p);

/* Step sizes of Section 7.2 for an n x n grid and graph g (host only, no GPU):
 * lambda_max(-Delta_G) by Householder tridiagonalisation and Sturm bisection,
 * then mu, nu from tau (tau <= 0 picks the Table 1 value).  Any output pointer
 * may be NULL.  Errors: VOMT_ERR_BAD_ARG, VOMT_ERR_GRAPH. */
int vomt_step_sizes(int n, const vomt_graph *g, double tau,
                    double *mu, double *nu, double *tau_used, double *lmax_graph);

/* Solve vector OMT (eq. (vomt)) by the V-OMT iteration of Section 7.2:
 *   u <- shrink_u(u + mu grad phi; mu), w <- shrink_w(w + nu grad_G phi; alpha nu),
 *   phi <- phi + tau (div_x(2u' - u) + div_G(2w' - w) + rho1 - rho0).
 * n >= 2.  rho0, rho1: device [k][n][n].  u, w, phi: device outputs (inputs too
 * when p->warm_start).  alpha > 0.  p == NULL uses the defaults.  *result
 * (host) receives the metrics of the last check; every run ends with a check.
 * Errors: BAD_ARG, MASS_MISMATCH, NEGATIVE_DENSITY, GRAPH, STEP_CONDITION,
 * NONFINITE, TOO_LARGE, CUDA. */
int vomt_solve(vomt_ctx *ctx, int n, const float *rho0, const float *rho1,
               const vomt_graph *g, double alpha, const vomt_params *p,
               float *u, float *w, float *phi, vomt_result *result, void *stream);

/* The same solve with every array in host memory: the call copies rho0, rho1
 * (and the warm-start iterate) to the context's device memory, solves, and
 * copies u, w, phi back before it returns. */
int vomt_solve_host(vomt_ctx *ctx, int n, const float *rho0, const float *rho1,
                    const vomt_graph *g, double alpha, const vomt_params *p,
                    float *u, float *w, float *phi, vomt_result *result, void *stream);

/* Vector OMT on an n x n x n grid: the finite-volume discretization of
 * Appendix A with a third direction (gradient, backward-difference divergence
 * and ghost faces in z as in x and y), iterated as in Section 7.2 with one
 * fused launch per iteration.  2 <= n <= 1024.
 *   rho0, rho1: device [k][n][n][n] cell masses (x fastest).
 *   u: device [3][k][n][n][n], the planes u_x, u_y, u_z; each component's
 *      ghost face (last index in its own direction) stays zero.
 *   w: device [l][n][n][n]; phi: device [k][n][n][n].
 * Outputs (inputs too when p->warm_start), like vomt_solve.  Norms: u_norm in
 * {L12, L2, L1} (the 2-norm over the three directions at a point), w_norm in
 * {L1, L2}; p->eps must be 0; p->engine is ignored; p->halo > 0 sets the
 * number of z planes each thread block marches through (0: the library's
 * choice, about four blocks per SM).  result->variant tells whether the TMA
 * form of the step ran (n a multiple of 4, n >= 40, k <= 4).  Default mu
 * is 1/(48 tau (n-1)^2) (1/(24 tau (n-1)^2) without edges), since
 * ||grad||^2 <= 12 (n-1)^2 in 3-D; user mu, nu must satisfy
 * tau mu 12 (n-1)^2 + tau nu lambda_max(-Delta_G) < 1.  The history is that of
 * vomt_history().  Errors: those of vomt_solve. */
int vomt_solve3d(vomt_ctx *ctx, int n, const float *rho0, const float *rho1,
                 const vomt_graph *g, double alpha, const vomt_params *p,
                 float *u, float *w, float *phi, vomt_result *result, void *stream);

/* Metrics of every convergence check of the last solve on ctx, 8 doubles per
 * row: primal, dual, rel_gap, rel_res, fp_resid, dual_infeas, iteration,
 * converged flag.  Writes min(cap, checks) rows to host `out`; returns the
 * number of rows available, or a negative error. */
int vomt_history(vomt_ctx *ctx, double *out, int cap);

/* Bounded waits of the resident engine (no counterpart in the paper; a test
 * and tuning hook).  In the resident engine one thread block waits on another
 * (halo words, check rows); every such wait gives up after a time limit, then
 * all blocks return and the solve reports VOMT_ERR_BARRIER_TIMEOUT with the
 * context still usable (the output arrays are not written).
 *   budget_ms      limit of one wait in milliseconds; 0 restores the default
 *                  (2000 ms).
 *   drop_exchange  > 0: in the following resident solves on ctx, block 0 does
 *                  not publish halo exchange number drop_exchange, so that its
 *                  neighbours' waits run out (a message dropped on purpose);
 *                  0 turns this off.
 * Applies to later calls on ctx.  Returns VOMT_OK, or VOMT_ERR_BAD_ARG for a
 * null ctx or a negative or non-finite argument. */
int vomt_set_wait_policy(vomt_ctx *ctx, double budget_ms, int drop_exchange);

/* ------------------------------------------------------------------------ */
/* Gradients of the transport cost                                            */
/* ------------------------------------------------------------------------ */

/* Envelope gradient of V (the optimal value of eq. (vomt) / eq. (vomt-dual))
 * for `batch` problems of one shape: the dual is a maximum over a feasible set
 * independent of the densities of <phi, rho1 - rho0>, so dV/drho1 = phi* and
 * dV/drho0 = -phi*, with the constant the dual leaves free fixed by making phi*
 * zero-mean over all cells and channels; the primal is linear in alpha, so
 * dV/dalpha = sum_ij ||w*_ij||_w.  phi: device [batch][k][n][pitch], w: device
 * [batch][l][n][pitch] (a converged iterate, e.g. from vomt_solve), rows of n
 * floats at a row pitch of `pitch` floats (0 means n).  grad_scale: device
 * [batch] factors (the upstream gradient) or NULL for 1.  Outputs (any may be
 * NULL): d_rho0, d_rho1 device [batch][k][n][pitch] (the padding is not
 * written), d_alpha device [batch].  Asynchronous on `stream`.  Errors:
 * BAD_ARG (also pitch in (0, n)), CUDA. */
int vomt_backward(vomt_ctx *ctx, int batch, int n, int pitch, int k, int n_edges, int w_norm, const float *phi,
                  const float *w, const float *grad_scale, float *d_rho0, float *d_rho1, float *d_alpha,
                  void *stream);

/* Unrolled gradient: J_T = P(u^T, w^T), the primal objective after T
 * iterations of Section 7.2 from the zero iterate (tau, mu, nu, norms from p;
 * p->u_norm must be VOMT_U_L12), and its exact gradient by reverse mode through
 * the T iterations.  The forward pass keeps the iterate every `ckpt`
 * iterations; the reverse pass recomputes each segment from its checkpoint.
 * rho0, rho1: device [k][n][n].  Outputs: d_rho0, d_rho1 device [k][n][n]
 * (either may be NULL), *d_alpha and *J host (either may be NULL); every
 * derivative is multiplied by `scale`.  Returns after the work finished.
 * Errors: as vomt_solve. */
int vomt_unrolled_grad(vomt_ctx *ctx, int n, const float *rho0, const float *rho1, const vomt_graph *g,
                       double alpha, const vomt_params *p, int T, int ckpt, double scale, float *d_rho0,
                       float *d_rho1, double *d_alpha, double *J, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched vector OMT: many independent problems in one persistent launch     */
/* ------------------------------------------------------------------------ */
/* Each instance is a vector-OMT problem of its own grid side, channel count,
 * channel graph and alpha (Section 7.2).  Its data lives in one FP32 arena in
 * device memory, starting at float `offset`:
 *   rho0 [k][n][n], rho1 [k][n][n], u [2][k][n][n], w [l][n][n], phi [k][n][n]
 * i.e. (5k + l) n^2 floats.  rho0 / rho1 are inputs, u / w / phi outputs (and
 * inputs when p->warm_start).  vomt_batch_layout assigns consecutive 64-byte
 * aligned offsets. */
typedef struct {
    int n;               /* grid side (>= 2) */
    vomt_graph graph;    /* channel graph (host memory) */
    double alpha;        /* > 0 */
    double tau;          /* <= 0: p->tau if > 0, else Table 1's value for this n */
    size_t offset;       /* first float of this instance in the arena */
} vomt_instance;

#define VOMT_ENGINE_BATCHED 3   /* reported in vomt_result.engine by vomt_solve_batched */

/* Fill inst[q].offset for consecutive, 16-float aligned instance blocks and
 * return the arena size in floats.  Host only. */
int vomt_batch_layout(int count, vomt_instance *inst, size_t *total_floats);

/* Solve every instance by the iteration of Section 7.2, each to its own
 * stopping point (tolerance or p->max_iters, checked every p->check_every
 * iterations, as in vomt_solve).  mu and nu follow the paper's rule per
 * instance; p->mu, p->nu and p->halo are ignored.  Both paths run as one CUDA
 * graph launch per call where they can (results[q].variant = 1).  Two paths:
 *   one block per instance (p->engine == VOMT_ENGINE_STREAM): one persistent
 *     launch; thread blocks take instances from a device queue (largest first)
 *     and run the fused streaming step on each.  When `stream` is not the
 *     legacy default stream (NULL), the launch (queue reset, kernel, status
 *     read-back) is captured into a CUDA graph on the first call and replayed
 *     by later calls with the same instances, arena and parameters.
 *   grouped (p->engine == VOMT_ENGINE_RESIDENT): instances of equal channel
 *     count and side form a wave; one cooperative launch per wave splits the
 *     SMs into groups of T tiles and each group runs the resident algorithm on
 *     its share of the wave, one instance after another.  The waves' launches
 *     are captured into one CUDA graph (on `stream`, or on a private stream of
 *     the context when `stream` is the legacy default stream) on the first call
 *     and replayed by later calls with the same instances, arena and
 *     parameters.  Needs k <= 5 and
 *     p->max_iters < 2^20 - 2 (else VOMT_ERR_TOO_LARGE).
 * VOMT_ENGINE_AUTO or VOMT_ENGINE_BATCHED: the path vomt_batch_tune found
 * faster on ctx, else the one a cost model estimates faster.
 * results: host array of `count` (may be NULL); results[q].blocks is the
 * number of tiles instance q ran on and .halo its ring width.  Returns
 * VOMT_OK, VOMT_NOT_CONVERGED if some instance hit the cap, or the first error
 * (the message names the instance).  The context keeps the scratch between
 * calls. */
int vomt_solve_batched(vomt_ctx *ctx, int count, const vomt_instance *inst, float *arena,
                       const vomt_params *p, vomt_result *results, void *stream);

/* Tuner of the batched engine: runs the batch for sample_iters iterations (no
 * tolerance) on the one-block-per-instance path with 128, 256 and 512 threads
 * per block, and on the grouped path where it applies; keeps the fastest
 * thread count and the faster path for later vomt_solve_batched calls on ctx
 * with VOMT_ENGINE_AUTO / VOMT_ENGINE_BATCHED.  Returns the best thread count
 * in *best_threads and the times (milliseconds) in ms[0..3] (128, 256, 512
 * threads, then the grouped path or -1); either pointer may be NULL.
 * Overwrites the arena's u, w, phi. */
int vomt_batch_tune(vomt_ctx *ctx, int count, const vomt_instance *inst, float *arena,
                    const vomt_params *p, int sample_iters, int *best_threads, double *ms);

/* Set the batched engine's threads per block (128, 256 or 512; 0 restores the
 * default, 512), e.g. from a tuning result cached by the caller. */
int vomt_batch_set_threads(vomt_ctx *ctx, int threads);

/* ------------------------------------------------------------------------ */
/* Matrix OMT (Section 4, eq. (momt); algorithm of Section 7.3)               */
/* ------------------------------------------------------------------------ */
/* Densities are real symmetric k x k matrices per cell (k = 2 or 3), stored as
 * full matrices: plane a*k + b of a [k*k][n][n] array holds entry (a, b).
 * The quantum gradient of Section 4.1 is built from N real symmetric k x k
 * matrices L (host, row-major, N*k*k doubles): grad_L X = (L_s X - X L_s)_s, and
 * div_L = -grad_L^*.  The standing assumption ker grad_L = span{I} (Section 4.1)
 * is checked; a violation returns VOMT_ERR_L_KERNEL.
 *
 * Norms (Section 6.2): u_norm VOMT_U_L2 is ||U||_2 (joint Frobenius over both
 * directions) and VOMT_U_L1 is ||U||_1 (entrywise); the per-channel code
 * VOMT_U_L12 (the vomt_default_params value) selects ||U||_2 here; VOMT_U_NUC
 * is ||U||_{1,nuc} = ||U_x||_nuc + ||U_y||_nuc.  w_norm VOMT_W_L1 is ||W||_1
 * (entrywise), VOMT_W_L2 is ||W||_2 (joint Frobenius), VOMT_W_NUC is
 * ||W||_{1,nuc} = sum_s ||W_s||_nuc.  The nuclear shrink soft-thresholds the
 * singular values (Appendix B): for symmetric U through a per-point
 * eigen-decomposition (one Jacobi rotation at 2 x 2, a closed form at 3 x 3);
 * for 3 x 3 skew W_s, whose two nonzero singular values
 * are equal, it scales W_s by max(0, 1 - t / sigma).
 * Step sizes: tau <= 0 picks Table 3's value (10 for n <= 64, 30 for n <= 128,
 * else 60); mu = 1/(32 tau (n-1)^2), nu = 1/(4 tau lambda_max(-Delta_L)) with
 * lambda_max taken over all k x k matrices, as Section 7.3 forms it.
 *
 * Internally symmetric fields are stored as their k(k+1)/2 upper entries and
 * skew ones as their k(k-1)/2 entries above the diagonal, with the off-diagonal
 * entries weighted 2 in every inner product and norm, which reproduces the
 * Hilbert-Schmidt geometry exactly (the shrinks stay exact by the Lemma of
 * Appendix B and its entrywise analogue). */

/* lambda_max(-Delta_L) over all k x k matrices, the second-smallest eigenvalue
 * of -Delta_L on symmetric matrices (positive iff ker grad_L = span{I}), and the
 * step sizes (host only).  Any output pointer may be NULL.
 * Errors: BAD_ARG (k, N, L not symmetric), L_KERNEL. */
int momt_step_sizes(int n, int k, int N, const double *L, double tau, double *mu, double *nu,
                    double *tau_used, double *lmax, double *sym_gap);

/* Solve matrix OMT by the M-OMT iteration of Section 7.3:
 *   U <- shrink_u(U + mu grad Phi; mu), W <- shrink_w(W + nu grad_L Phi; alpha nu),
 *   Phi <- Phi + tau (div_x(2U' - U) + div_L(2W' - W) + Lam1 - Lam0).
 * Lam0, Lam1: device [k*k][n][n], symmetric (|X_ab - X_ba| <= 1e-5 max|X|),
 * nonnegative diagonals, equal total trace.  U: device [2][k*k][n][n] (x then y
 * components), W: device [N][k*k][n][n] (skew), Phi: device [k*k][n][n]
 * (symmetric); outputs, and inputs when p->warm_start (symmetrised / made skew
 * on the way in).  Metrics in *result use the Hilbert-Schmidt inner product.
 * Errors: as vomt_solve, plus L_KERNEL. */
int momt_solve(vomt_ctx *ctx, int n, int k, const float *Lam0, const float *Lam1, int N, const double *L,
               double alpha, const vomt_params *p, float *U, float *W, float *Phi, vomt_result *result,
               void *stream);

/* Complex Hermitian matrix OMT: Section 4's complex setting (Hermitian densities
 * and L_l, skew-Hermitian W, the Hilbert-Schmidt product Re tr(X Y*)), iterated
 * as in Section 7.3.  Norms (Section 6.2, per point): p->u_norm VOMT_U_L2 (or
 * the default) is the Frobenius norm ||U||_2 of (U_x, U_y), VOMT_U_L1 the
 * entrywise ||U||_1 = sum of the moduli |U_ab| of both directions' entries;
 * p->w_norm VOMT_W_L2 is ||W||_2, VOMT_W_L1 the entrywise ||W||_1 (anything else
 * is BAD_ARG).  The entrywise shrink scales each complex entry by
 * max(0, 1 - t / |z|) (Appendix B's shrink_2 on the entry as a point of the plane).
 *   k = 2 (a Hermitian 2 x 2 field is 4 real coordinates), 1 <= N <= 9; or
 *   k = 3 (9 real coordinates), 1 <= N <= 4.  3 x 3 fields and the entrywise
 *   norms run on the resident engine only: VOMT_ENGINE_STREAM is BAD_ARG, and a
 *   grid beyond the resident engine's reach is VOMT_ERR_TOO_LARGE.
 *   L: host, N complex k x k Hermitian matrices as (re, im) double pairs,
 *      row-major: L[((s*k + a)*k + b)*2 + {0, 1}].
 *   Lam0, Lam1: device [2][k*k][n][n] floats, the real parts then the imaginary
 *      parts of the k*k entries (entry (a, b) at plane a*k + b); Hermitian
 *      (|X_ab - conj X_ba| and |Im X_aa| <= 1e-5 max|X|), nonnegative real
 *      diagonals, equal total trace.
 *   U: device [2][2][k*k][n][n] (direction x, y; then re, im), W: device
 *      [N][2][k*k][n][n] (skew-Hermitian), Phi: device [2][k*k][n][n]; outputs,
 *      and inputs when p->warm_start.
 * Step sizes as momt_solve, with lambda_max(-Delta_L) over C^{k x k}; the
 * kernel condition is checked on Hermitian matrices (L_KERNEL).  Internally a
 * Hermitian field is its real diagonal and the real and imaginary parts of the
 * entries above it (weights 1, 2, 2), a skew-Hermitian one the imaginary
 * diagonal and the entries above it, which reproduces Re tr(X Y*) exactly.
 * Errors: as momt_solve. */
int momt_solve_complex(vomt_ctx *ctx, int n, int k, const float *Lam0, const float *Lam1, int N,
                       const double *L, double alpha, const vomt_params *p, float *U, float *W, float *Phi,
                       vomt_result *result, void *stream);

/* Matrix OMT on an n x n x n grid (2 <= n <= 1024): the iteration of momt_solve
 * with a third spatial direction (the discretization of vomt_solve3d), for
 * volumes of matrix densities such as 3-D DTI.
 *   Lam0, Lam1: device [k*k][n][n][n] (x fastest), the checks of momt_solve.
 *   U: device [3][k*k][n][n][n] (U_x, U_y, U_z; ghost faces zero),
 *   W: device [N][k*k][n][n][n], Phi: device [k*k][n][n][n].
 * Norms: u_norm L2 (Frobenius over the three directions jointly), L1 or NUC
 * (sum of the three directions' nuclear norms); w_norm as momt_solve.  Default
 * mu = 1/(48 tau (n-1)^2); user steps must satisfy tau mu 12 (n-1)^2 + tau nu
 * lambda_max(-Delta_L) < 1.  p->engine is ignored; p->halo > 0 sets the z planes
 * each block marches through.  k = 2 runs the TMA form of the step where the
 * grid allows (result->variant), k = 3 the per-thread form.
 * Errors: as momt_solve. */
int momt_solve3d(vomt_ctx *ctx, int n, int k, const float *Lam0, const float *Lam1, int N, const double *L,
                 double alpha, const vomt_params *p, float *U, float *W, float *Phi, vomt_result *result,
                 void *stream);

/* ------------------------------------------------------------------------ */
/* Tuning the dual step tau                                                   */
/* ------------------------------------------------------------------------ */
/* Sections 7.1-7.3 tie the primal steps to tau (mu = 1/(32 tau (n-1)^2),
 * nu = 1/(4 tau lambda_max)), so that every tau > 0 meets the convergence
 * condition, and tune tau per experiment "for the fastest convergence" (Tables 1
 * and 3 list the values).  The best tau scales with the densities and with how
 * far mass moves, so these calls measure it: runs of the solve itself from the
 * zero iterate over the grid tau_j = tau_paper * 10^((j - 1) / 2),
 * j = 0 .. VOMT_TAU_GRID - 1 (tau_paper: Table 1's or Table 3's value for n),
 * scored by max(rel_gap, rel_res) at the end of the run. */
#define VOMT_TAU_GRID 10

/* Vector OMT: successive halving on the grid (every tau runs sample_iters
 * iterations, the best 4 twice as many, the best 2 four times as many), then
 * the winner's neighbours tau * 10^(+-1/4) at that length; about 34 sample_iters
 * iterations in all.  Arguments as vomt_solve; p supplies norms, engine and eps
 * (its tau, mu, nu, iteration and tolerance fields are ignored).  u, w, phi are
 * device scratch of vomt_solve's shapes, overwritten.  Outputs (host, any may be
 * NULL): *best_tau, *best_score (its score at the longest run),
 * grid_scores[VOMT_TAU_GRID] (the score of every grid point after sample_iters).
 * Returns after the work finished.  Errors: those of vomt_solve (a candidate
 * whose iterate became non-finite only scores +infinity). */
int vomt_tune_tau(vomt_ctx *ctx, int n, const float *rho0, const float *rho1, const vomt_graph *g,
                  double alpha, const vomt_params *p, int sample_iters, float *u, float *w, float *phi,
                  double *best_tau, double *best_score, double *grid_scores, void *stream);

/* Matrix OMT: the same search through momt_solve (arguments as momt_solve). */
int momt_tune_tau(vomt_ctx *ctx, int n, int k, const float *Lam0, const float *Lam1, int N, const double *L,
                  double alpha, const vomt_params *p, int sample_iters, float *U, float *W, float *Phi,
                  double *best_tau, double *best_score, double *grid_scores, void *stream);

/* Batched vector OMT: every grid point is run once for the whole batch
 * (vomt_solve_batched, sample_iters iterations, instance q at tau_j of its own
 * n), and each instance keeps its best: taus[q] (host, count entries, required)
 * receives it, ready for inst[q].tau; scores[q] (host, may be NULL) its score.
 * Overwrites the arena's u, w, phi.  Errors: those of vomt_solve_batched. */
int vomt_batch_tune_tau(vomt_ctx *ctx, int count, const vomt_instance *inst, float *arena,
                        const vomt_params *p, int sample_iters, double *taus, double *scores);

/* ------------------------------------------------------------------------ */
/* Allocation-free solve.  The paper has no counterpart: this is a            */
/* deployment feature of this library.                                        */
/* ------------------------------------------------------------------------ */

/* Size of the fixed device scratch array behind vomt_solve_noalloc: 16 MiB,
 * enough for n = 256 with k = 3 channels and 3 edges (the solve needs
 * 4 (7k + 2l) n^2 bytes, plus 80 bytes per 256 grid points and 11 KB). */
#define VOMT_NOALLOC_SCRATCH_BYTES (16u << 20)

/* The vomt_solve computation (streaming engine) for callers that cannot
 * allocate device memory: applications whose device memory belongs to one
 * custom pool or allocator, which a cudaMalloc behind its back would fragment
 * or overcommit; plug-ins and long-running services that must not grow the
 * process footprint, or meet an out-of-memory failure, after start-up.  It
 * needs no context and never allocates or frees memory: its scratch is one
 * fixed array of VOMT_NOALLOC_SCRATCH_BYTES in the library's device image,
 * which every GPU that loads the library holds until the process exits.
 *   - Runs on the calling thread's current CUDA device; `stream` must belong
 *     to it.  The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress), a one-time set-up per device.
 *   - The call reads its stopping flag and results back and synchronises
 *     `stream` while it runs, so it cannot be recorded into a CUDA graph: a
 *     stream under capture is refused with VOMT_ERR_BAD_ARG before any GPU
 *     work, leaving the capture intact.
 *   - Every call shares the one array and overwrites it (the status block is
 *     cleared at the start of each call), so calls that overlap on the GPU --
 *     from other streams or host threads -- race and give wrong results.
 *     Serialise them.
 *   - Arguments, layouts, step-size rules, checks and results are those of
 *     vomt_solve; p->engine and p->halo are ignored (always the streaming
 *     engine), and vomt_history() does not see these solves.
 *   - Problems whose scratch would exceed the array return VOMT_ERR_TOO_LARGE
 *     before any GPU work.  `error` (may be NULL) receives a message, valid
 *     until the next call on the same host thread.
 */
int vomt_solve_noalloc(int n, const float *rho0, const float *rho1, const vomt_graph *g,
                       double alpha, const vomt_params *p, float *u, float *w, float *phi,
                       vomt_result *result, void *stream, const char **error);

#ifdef __cplusplus
}
#endif
#endif /* VOMT_H */
