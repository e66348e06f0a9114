// Internal declarations shared by the translation units of libvomt.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "vomt.h"

namespace vomt {

// Channels and flux entries of the per-point operator: up to VOMT_MAX_CHANNELS (8)
// colour channels for vector OMT, up to 9 real coordinates for a complex
// Hermitian 3 x 3 field; the flux bound is K(K-1)/2.
constexpr int KMAX = 9;
constexpr int LMAX = KMAX * (KMAX - 1) / 2;
constexpr int KVEC = VOMT_MAX_CHANNELS;            // vector OMT: k <= 8
constexpr int LVEC = KVEC * (KVEC - 1) / 2;

// Internal norm codes beyond the public ones: the entrywise ||.||_1 of complex
// Hermitian / skew-Hermitian fields (Section 6.2, sum of the entries' moduli), whose
// shrink acts jointly on the (Re, Im) coordinate pairs the operator marks (OpDev
// upair / wpair) and entrywise on the other coordinates.
constexpr int U_CL1 = 4;
constexpr int W_CL1 = 3;

// Channel graph as the kernels see it (passed by value as a kernel argument).
// Edge e runs from node lo[e] to node hi[e] (lo < hi), scaled by inv_c[e] = 1/c_e.
struct GraphDev {
    int k, l;
    int8_t lo[LMAX], hi[LMAX];
    float inv_c[LMAX];
};

// Per-point linear structure as the kernels see it (a kernel argument).  A
// point carries k "channels" (vector OMT: the k colour channels; matrix OMT:
// the k(k+1)/2 entries of a symmetric matrix, diagonal first) and l flux
// entries (vector OMT: the graph edges; matrix OMT: the k(k-1)/2 entries above
// the diagonal of each skew-symmetric W_s).  Inner products weigh channel c by
// wc[c] and flux entry e by we[e] (2 for an off-diagonal entry, which stands for
// itself and its mirror), so the compact coordinates reproduce the
// Hilbert-Schmidt products of Section 4.
struct OpDev {
    int k, l;
    // complex fields: bit c of upair (bit e of wpair) marks coordinate c (flux entry e)
    // as the real part of an entry whose imaginary part is coordinate c + 1
    uint32_t upair;
    uint32_t wpair[2];
    float wc[KMAX];
    float we[LMAX];
    float G[LMAX][KMAX];     // (grad phi)_e = sum_c G[e][c] phi_c   (grad_G or grad_L)
    float Dv[KMAX][LMAX];    // (div y)_c = -sum_e Dv[c][e] y_e,  Dv = (we / wc) G^T (div = -grad^*)
};

// Per-solve scalars.
struct StepDev {
    int n;          // grid side
    float ih;       // 1/h = n - 1
    float mu, nu, tau, alpha;
    // quadratic regularisation eps (||u||_2^2 + ||w||_2^2): the primal steps shrink
    // su * v with threshold su * mu (u) and sw * v with threshold sw * alpha * nu (w),
    // su = 1 / (1 + 2 mu eps), sw = 1 / (1 + 2 nu eps); reg = 0 when eps = 0
    int reg;
    float eps, su, sw;
};

// Reduction slots of one convergence check (FP64).
enum {
    RED_P = 0,      // primal objective
    RED_D,          // dual objective
    RED_RR,         // ||residual||^2
    RED_BB,         // ||rho0 - rho1||^2
    RED_DU,         // ||u^t - u^{t-1}||^2
    RED_DW,         // ||w^t - w^{t-1}||^2
    RED_DP,         // ||phi^t - phi^{t-1}||^2
    RED_X,          // <phi^t - phi^{t-1}, div(u^t - u^{t-1}) + div_G(w^t - w^{t-1})>
    RED_DIST,       // sum of squared distances of grad phi, grad_G phi to the dual balls (eps > 0)
    RED_NSUM,       // number of summed slots
    RED_MAX = RED_NSUM,  // dual infeasibility (max)
    NRED
};

constexpr int NMET = 8;

// Solve status kept in device memory and written by the finalize kernels.
struct DevStatus {
    int stop;       // 1 once the tolerance is met or an error was found
    int iter;       // iteration of the last check
    int checks;     // checks run
    int error;      // 0 or VOMT_ERR_NONFINITE / VOMT_ERR_BARRIER_TIMEOUT
    int raw;        // 1: met[2], met[3] hold ||r||^2 and ||rho0 - rho1||^2 (finish_raw_row)
    int reserved;
    double met[NMET];
};

// The resident engine's checks decide on the device with products and comparisons
// only (FP64 division and square root are slow on this GPU and would sit on the
// grid-wide critical path) and store each row as (P, D, ||r||^2, ||rho0 - rho1||^2,
// R, dual infeasibility, t, converged); the host then forms the two ratios.
inline void finish_raw_row(double *m)
{
    const double P = m[0], D = m[1], RR = m[2], BB = m[3];
    m[2] = fabs(P - D) / fmax(fabs(P), 1e-300);
    m[3] = sqrt(RR) / (BB > 0.0 ? sqrt(BB) : 1.0);
}

struct SolveCfg {
    double tol_gap, tol_res;
    double mu, nu, tau;
    int has_w;
    double eps;     // regularisation weight (0: none)
};

// Fill the regularisation fields of the step constants and the check settings.
inline void set_regularisation(StepDev *s, SolveCfg *cfg, double eps, double mu, double nu)
{
    s->reg = eps > 0.0 ? 1 : 0;
    s->eps = (float)eps;
    s->su = (float)(1.0 / (1.0 + 2.0 * mu * eps));
    s->sw = (float)(1.0 / (1.0 + 2.0 * nu * eps));
    cfg->eps = eps;
}

// Relative tolerance of the equal-mass check of the densities (the constraint of
// eq. (vomt) sums to zero over all cells and channels, so the totals must agree).
constexpr double kMassRelTol = 1e-6;

// ----------------------------------------------------------------- host setup
int graph_to_dev(const vomt_graph *g, GraphDev *out, std::string *err);
double sym_lmax(int m, const double *A);     // largest eigenvalue of a symmetric m x m matrix
double sym_eig(int m, const double *A, int idx);   // idx-th smallest eigenvalue (0-based)
double graph_lmax(const GraphDev &g, const double *cost);
void graph_to_op(const GraphDev &g, OpDev *op);
// Quantum operator of Section 4.1 for N real symmetric k x k matrices L (row-major,
// host): compact grad / div, lambda_max(-Delta_L) over all k x k matrices (the
// k^2 x k^2 matrix of Section 7.3) and the second-smallest eigenvalue of -Delta_L on
// symmetric matrices (positive iff ker grad_L = span{I}, the standing assumption).
int quantum_to_op(int k, int N, const double *L, OpDev *op, double *lmax, double *sym_gap, std::string *err);
// complex Hermitian fields (k = 2); L: N complex k x k matrices, (re, im) pairs row-major
int hermitian_to_op(int k, int N, const double *L, OpDev *op, double *lmax, double *sym_gap, std::string *err);

}  // namespace vomt

namespace vomt {
struct BatchState;
void batch_state_free(BatchState *b);
}  // namespace vomt

// The opaque context.
struct vomt_ctx {
    int device = 0;
    int sm_count = 0;
    std::string err;
    // streaming-engine workspace
    float *ws = nullptr;
    size_t ws_floats = 0;
    double *partials = nullptr;
    size_t partials_cap = 0;
    vomt::DevStatus *dstatus = nullptr;
    vomt::DevStatus *hstatus = nullptr;      // pinned, 2 slots
    double *dhist = nullptr;
    int hist_cap = 0;
    bool hist_raw = false;                   // the last solve's history rows need finish_raw_row
    std::vector<double> last_hist;
    int last_checks = 0;
    // host-API staging buffers (device)
    float *stage = nullptr;
    size_t stage_floats = 0;
    // dense copies of pitched device arrays (vomt_params.pitch)
    float *pstage = nullptr;
    size_t pstage_bytes = 0;
    int launches = 0;                        // kernels launched by the current call
    int last_blocks = 0, last_halo = 0, last_variant = 0;      // launch shape of the current call
    // matrix-OMT compact staging (device)
    float *mstage = nullptr;
    size_t mstage_bytes = 0;
    // gradient scratch (unrolled adjoint checkpoints, adjoints, partial sums)
    float *gbuf = nullptr;
    size_t gbuf_bytes = 0;
    double *gpart = nullptr;
    size_t gpart_bytes = 0;
    // batched engine (tables, scratch, captured graph)
    vomt::BatchState *batch = nullptr;
    // resident-engine scratch
    void *rscratch = nullptr;
    size_t rscratch_bytes = 0;
    // stream on which the streaming engine captures its iteration graphs
    cudaStream_t cap_stream = nullptr;
    // bounded waits of the resident engine: limit (0 = default) and the test hook
    unsigned long long wait_ns = 0;
    int drop_exchange = 0;
};

namespace vomt {
int set_cuda_error(vomt_ctx *ctx, cudaError_t e, const char *what);
int fail(vomt_ctx *ctx, int code, const char *msg);
// 2-D copy of `planes` planes of n rows of n floats between row pitches (in floats).
cudaError_t copy_planes(float *dst, int dst_pitch, const float *src, int src_pitch, int n, size_t planes,
                        cudaMemcpyKind kind, cudaStream_t st);
int prepare_vector(vomt_ctx *ctx, int n, const vomt_graph *graph, double alpha, const vomt_params *pin, OpDev *op,
                   StepDev *s, SolveCfg *cfg, vomt_params *p);
// Argument checks and step sizes of a vector solve, shared by the entry points with a
// context and the allocation-free one: parameter ranges, the channel graph (checked and
// converted), tau (Table 1's value when p->tau <= 0), mu and nu by Section 7.2's rule
// unless given (user steps must satisfy its condition), the step constants and the
// check settings.  On error *err holds the message.
struct VectorSetup {
    GraphDev gd;
    OpDev g;
    StepDev s;
    SolveCfg cfg;
    vomt_params p;
    double lmax;
};
int setup_vector(int n, const vomt_graph *graph, double alpha, const vomt_params *pin, VectorSetup *out,
                 std::string *err);
int check_vector_densities(vomt_ctx *ctx, int k, int n, const float *rho0, const float *rho1, cudaStream_t st);
// 3-D solve after validation and step sizes (vector3d.cu); compact channels of g
int solve3d_core(vomt_ctx *ctx, int n, const OpDev &g, const StepDev &s, const SolveCfg &cfg, const vomt_params &p,
                 int zc_user, const float *rho0, const float *rho1, float *u, float *w, float *phi, cudaStream_t st);
void fill_result(vomt_ctx *ctx, const SolveCfg &cfg, int engine, vomt_result *r, int *status);
int run_engine(vomt_ctx *ctx, const OpDev &op, const StepDev &s, const SolveCfg &cfg, const vomt_params &p,
               const float *rho0, const float *rho1, float *u, float *w, float *phi, cudaStream_t st, int *engine);
int ensure_buffer(vomt_ctx *ctx, void **p, size_t *cap, size_t bytes, const char *what);

// streaming engine (vector_stream.cu)
int stream_solve(vomt_ctx *ctx, const OpDev &g, const StepDev &s, const SolveCfg &cfg,
                 const vomt_params &p, const float *rho0, const float *rho1,
                 float *u, float *w, float *phi, cudaStream_t st);
// resident engine (vector_resident.cu)
struct ResidentPlan {
    int Gx, Gy, TXm, TYm, H, threads, P;
    double est_ns;      // estimated ns per iteration (a wave plan: of the whole wave, all its rounds)
    int lb;             // launch bound of the single-problem kernel (0: res_threads(k))
};
// Launch as a programmatic dependent of the previous kernel on the stream: the
// kernel's blocks may be scheduled while that kernel drains, and each of the
// streaming kernels (2-D and 3-D steps, checks, k_finalize) waits in
// cudaGridDependencySynchronize() before it reads what the previous one wrote.
// An iteration is a chain of short kernels, so this hides part of the gap
// between them.
template <typename... Exp, typename... Act>
inline cudaError_t launch_pdl(void (*kern)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Act... args)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Blocks of a streaming check (k_metrics, k_metrics3): the check's kernel loops
// over the grid with at most this many blocks (four per SM on a GB300), which
// bounds the FP64 rows k_finalize sums.
constexpr int kMetricBlocks = 608;
// Fixed-order sum of per-block FP64 partials (NRED per block), the stopping
// decision and the history row (one block of kFinThreads threads, one warp per
// slot; vector_stream.cu).  t < 0: the iteration is the last check's plus -t
// (replayed graphs).
constexpr int kFinThreads = 32 * NRED;
__global__ void k_finalize(const double *__restrict__ partials, int nblocks, SolveCfg cfg, int t, DevStatus *st,
                           double *hist, int hist_cap);

bool resident_plan(int n, int k, int max_blocks, int force_H, ResidentPlan *out);
bool resident_plan_wave(int n, int k, int count, int max_blocks, ResidentPlan *out);
int resident_solve(vomt_ctx *ctx, const OpDev &g, const StepDev &s, const SolveCfg &cfg, const vomt_params &p,
                   const ResidentPlan &plan, const float *rho0, const float *rho1, float *u, float *w, float *phi,
                   cudaStream_t st);
void launch_step(const OpDev &g, const StepDev &s, int un, int wn, const float *in, float *out, const float *b,
                 const DevStatus *st, cudaStream_t stream);
int validate_densities(vomt_ctx *ctx, int planes, int n, const float *rho0, const float *rho1,
                       cudaStream_t st, double *sums /* s0, s1, min0, min1, nonfinite */);
}  // namespace vomt
