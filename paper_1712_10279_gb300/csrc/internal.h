// Internal declarations shared by the translation units of libvomt.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "vomt.h"

namespace vomt {

constexpr int KMAX = VOMT_MAX_CHANNELS;
constexpr int LMAX = KMAX * (KMAX - 1) / 2;

// Channel graph as the kernels see it (passed by value as a kernel argument).
// Edge e runs from node lo[e] to node hi[e] (lo < hi), scaled by inv_c[e] = 1/c_e.
struct GraphDev {
    int k, l;
    int8_t lo[LMAX], hi[LMAX];
    float inv_c[LMAX];
};

// Per-solve scalars.
struct StepDev {
    int n;          // grid side
    float ih;       // 1/h = n - 1
    float mu, nu, tau, alpha;
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
    double met[NMET];
};

struct SolveCfg {
    double tol_gap, tol_res;
    double mu, nu, tau;
    int has_w;
};

// ----------------------------------------------------------------- host setup
int graph_to_dev(const vomt_graph *g, GraphDev *out, std::string *err);
double sym_lmax(int m, const double *A);     // largest eigenvalue of a symmetric m x m matrix
double graph_lmax(const GraphDev &g, const double *cost);

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
    std::vector<double> last_hist;
    int last_checks = 0;
    // host-API staging buffers (device)
    float *stage = nullptr;
    size_t stage_floats = 0;
    int launches = 0;                        // kernels launched by the current call
    // resident-engine scratch
    void *rscratch = nullptr;
    size_t rscratch_bytes = 0;
};

namespace vomt {
int set_cuda_error(vomt_ctx *ctx, cudaError_t e, const char *what);
int ensure_buffer(vomt_ctx *ctx, void **p, size_t *cap, size_t bytes, const char *what);

// streaming engine (vector_stream.cu)
int stream_solve(vomt_ctx *ctx, const GraphDev &g, const StepDev &s, const SolveCfg &cfg,
                 const vomt_params &p, const float *rho0, const float *rho1,
                 float *u, float *w, float *phi, cudaStream_t st);
// resident engine (vector_resident.cu)
struct ResidentPlan {
    int Gx, Gy, TXm, TYm, H, threads, P;
    double est_ns;
};
bool resident_plan(int n, int k, int max_blocks, int force_H, ResidentPlan *out);
int resident_solve(vomt_ctx *ctx, const GraphDev &g, const StepDev &s, const SolveCfg &cfg, const vomt_params &p,
                   const ResidentPlan &plan, const float *rho0, const float *rho1, float *u, float *w, float *phi,
                   cudaStream_t st);
int validate_densities(vomt_ctx *ctx, int planes, int n, const float *rho0, const float *rho1,
                       cudaStream_t st, double *sums /* s0, s1, min0, min1, nonfinite */);
}  // namespace vomt
