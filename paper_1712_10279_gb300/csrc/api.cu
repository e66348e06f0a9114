// C ABI of libvomt: argument checks, step sizes, engine choice and the host
// side of every solve.  Kernels live in the engine translation units.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "internal.h"

namespace vomt {

int set_cuda_error(vomt_ctx *ctx, cudaError_t e, const char *what)
{
    // clear a non-sticky error from the thread's last-error slot, so that it does not
    // surface in the caller's next unrelated CUDA call
    (void)cudaGetLastError();
    if (ctx) {
        char buf[256];
        snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
        ctx->err = buf;
    }
    return VOMT_ERR_CUDA;
}

int ensure_buffer(vomt_ctx *ctx, void **p, size_t *cap, size_t bytes, const char *what)
{
    if (*cap >= bytes && *p) return VOMT_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, what);
    *cap = bytes;
    return VOMT_OK;
}

cudaError_t copy_planes(float *dst, int dst_pitch, const float *src, int src_pitch, int n, size_t planes,
                        cudaMemcpyKind kind, cudaStream_t st)
{
    if (planes == 0) return cudaSuccess;
    return cudaMemcpy2DAsync(dst, sizeof(float) * (size_t)dst_pitch, src, sizeof(float) * (size_t)src_pitch,
                             sizeof(float) * (size_t)n, planes * (size_t)n, kind, st);
}

int fail(vomt_ctx *ctx, int code, const char *msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

// Table 1's tuned tau (1 for the 32^2 and 64^2 grids, 3 for 128^2 and 256^2).
static double default_tau(int n) { return n <= 64 ? 1.0 : 3.0; }

int setup_vector(int n, const vomt_graph *graph, double alpha, const vomt_params *pin, VectorSetup *out,
                 std::string *err)
{
    if (n < 2 || n > 32768) { *err = "n must be in [2, 32768]"; return VOMT_ERR_BAD_ARG; }
    if (!(alpha > 0.0) || !isfinite(alpha)) { *err = "alpha must be positive"; return VOMT_ERR_BAD_ARG; }
    vomt_params p;
    vomt_default_params(&p);
    if (pin) p = *pin;
    if (p.max_iters < 0 || p.check_every < 1) { *err = "max_iters >= 0, check_every >= 1"; return VOMT_ERR_BAD_ARG; }
    if (p.u_norm < 0 || p.u_norm > 2 || p.w_norm < 0 || p.w_norm > 1) { *err = "bad norm code"; return VOMT_ERR_BAD_ARG; }
    if (!(p.eps >= 0.0) || !isfinite(p.eps)) { *err = "eps must be finite and >= 0"; return VOMT_ERR_BAD_ARG; }
    if (p.pitch != 0 && p.pitch < n) { *err = "pitch must be 0 or >= n"; return VOMT_ERR_BAD_ARG; }
    int rc = graph_to_dev(graph, &out->gd, err);
    if (rc) return rc;
    graph_to_op(out->gd, &out->g);
    const double tau = p.tau > 0.0 ? p.tau : default_tau(n);
    const double lmax = graph_lmax(out->gd, graph->cost);
    const double n1 = (double)(n - 1);
    double mu = p.mu, nu = p.nu;
    const bool user = mu > 0.0 || nu > 0.0;
    if (!(mu > 0.0)) mu = out->g.l > 0 ? 1.0 / (32.0 * tau * n1 * n1) : 1.0 / (16.0 * tau * n1 * n1);
    if (!(nu > 0.0)) nu = out->g.l > 0 ? 1.0 / (4.0 * tau * lmax) : 1.0;
    if (user && !(tau * mu * 8.0 * n1 * n1 + (out->g.l > 0 ? tau * nu * lmax : 0.0) < 1.0)) {
        *err = "step sizes break 1 > tau mu 8(n-1)^2 + tau nu lambda_max(-Delta_G)";
        return VOMT_ERR_STEP_CONDITION;
    }
    out->s.n = n;
    out->s.ih = (float)n1;
    out->s.mu = (float)mu;
    out->s.nu = (float)nu;
    out->s.tau = (float)tau;
    out->s.alpha = (float)alpha;
    set_regularisation(&out->s, &out->cfg, p.eps, mu, nu);
    out->cfg.tol_gap = p.tol_gap;
    out->cfg.tol_res = p.tol_res;
    out->cfg.mu = mu;
    out->cfg.nu = nu;
    out->cfg.tau = tau;
    out->cfg.has_w = out->g.l > 0;
    out->p = p;
    out->p.tau = tau;
    out->p.mu = mu;
    out->p.nu = nu;
    out->lmax = lmax;
    return VOMT_OK;
}

static int prepare(vomt_ctx *ctx, int n, const vomt_graph *graph, double alpha, const vomt_params *pin,
                   VectorSetup *out)
{
    if (!ctx) return VOMT_ERR_BAD_ARG;
    ctx->err.clear();
    if (pin && (pin->engine < 0 || pin->engine > 2)) return fail(ctx, VOMT_ERR_BAD_ARG, "bad engine code");
    if (pin && (pin->halo < 0 || pin->halo > 16)) return fail(ctx, VOMT_ERR_BAD_ARG, "halo must be in [0, 16]");
    return setup_vector(n, graph, alpha, pin, out, &ctx->err);
}

static int check_densities(vomt_ctx *ctx, int planes, int n, const float *rho0, const float *rho1, cudaStream_t st)
{
    double sums[5];
    int rc = validate_densities(ctx, planes, n, rho0, rho1, st, sums);
    if (rc) return rc;
    if (sums[4] > 0.0) return fail(ctx, VOMT_ERR_NONFINITE, "density has NaN or Inf entries");
    if (sums[2] < 0.0 || sums[3] < 0.0) return fail(ctx, VOMT_ERR_NEGATIVE_DENSITY, "density has negative entries");
    if (fabs(sums[0] - sums[1]) > kMassRelTol * fmax(fabs(sums[0]), fabs(sums[1])))
        return fail(ctx, VOMT_ERR_MASS_MISMATCH, "rho0 and rho1 have different total mass");
    return VOMT_OK;
}

int prepare_vector(vomt_ctx *ctx, int n, const vomt_graph *graph, double alpha, const vomt_params *pin, OpDev *op,
                   StepDev *s, SolveCfg *cfg, vomt_params *p)
{
    VectorSetup P;
    const int rc = prepare(ctx, n, graph, alpha, pin, &P);
    if (rc) return rc;
    *op = P.g;
    *s = P.s;
    *cfg = P.cfg;
    *p = P.p;
    return VOMT_OK;
}

int check_vector_densities(vomt_ctx *ctx, int k, int n, const float *rho0, const float *rho1, cudaStream_t st)
{
    return check_densities(ctx, k, n, rho0, rho1, st);
}

void fill_result(vomt_ctx *ctx, const SolveCfg &cfg, int engine, vomt_result *r, int *status)
{
    const DevStatus &h = ctx->hstatus[0];
    ctx->last_checks = h.checks;
    double met[NMET];
    for (int q = 0; q < NMET; ++q) met[q] = h.met[q];
    if (h.raw) finish_raw_row(met);
    if (h.error) {
        *status = h.error;
        ctx->err = h.error == VOMT_ERR_NONFINITE ? "iterate became non-finite" : "device wait timed out";
    } else if (cfg.tol_gap > 0.0) {
        *status = met[7] != 0.0 ? VOMT_OK : VOMT_NOT_CONVERGED;
    } else {
        *status = VOMT_OK;
    }
    if (r) {
        r->primal = met[0];
        r->dual = met[1];
        r->rel_gap = met[2];
        r->rel_res = met[3];
        r->fp_resid = met[4];
        r->dual_infeas = met[5];
        r->iters = h.iter;
        r->mu = cfg.mu;
        r->nu = cfg.nu;
        r->tau = cfg.tau;
        r->status = *status;
        r->engine = engine;
        r->checks = h.checks;
        r->launches = ctx->launches;
        r->blocks = ctx->last_blocks;
        r->halo = ctx->last_halo;
        r->variant = ctx->last_variant;
    }
}

// Resident engine when the plan fits (AUTO / RESIDENT), else the streaming engine.
int run_engine(vomt_ctx *ctx, const OpDev &op, const StepDev &s, const SolveCfg &cfg, const vomt_params &p,
               const float *rho0, const float *rho1, float *u, float *w, float *phi, cudaStream_t st, int *engine)
{
    *engine = VOMT_ENGINE_STREAM;
    ctx->last_blocks = 0;
    ctx->last_halo = 0;
    ctx->last_variant = 0;
    int rc;
    if (p.engine != VOMT_ENGINE_STREAM) {
        ResidentPlan plan;
        if (resident_plan(s.n, op.k, ctx->sm_count, p.halo, &plan)) {
            rc = resident_solve(ctx, op, s, cfg, p, plan, rho0, rho1, u, w, phi, st);
            if (rc == VOMT_OK) {
                *engine = VOMT_ENGINE_RESIDENT;
                return VOMT_OK;
            }
            if (!(rc == VOMT_ERR_TOO_LARGE && p.engine == VOMT_ENGINE_AUTO)) return rc;
        } else if (p.engine == VOMT_ENGINE_RESIDENT) {
            return fail(ctx, VOMT_ERR_TOO_LARGE, "grid too large for the resident engine");
        }
    }
    // the streaming kernels exist for up to VOMT_MAX_CHANNELS channels and the public norms
    if (op.k > KVEC || p.u_norm == U_CL1 || p.w_norm == W_CL1)
        return fail(ctx, VOMT_ERR_TOO_LARGE,
                    "complex 3 x 3 fields and the complex entrywise norm run on the resident engine only, and the "
                    "grid does not fit it");
    return stream_solve(ctx, op, s, cfg, p, rho0, rho1, u, w, phi, st);
}

static int solve_device(vomt_ctx *ctx, int n, const float *rho0, const float *rho1, const vomt_graph *graph,
                        double alpha, const vomt_params *pin, float *u, float *w, float *phi, vomt_result *result,
                        cudaStream_t st)
{
    VectorSetup P;
    int rc = prepare(ctx, n, graph, alpha, pin, &P);
    if (rc) return rc;
    if (!rho0 || !rho1 || !u || !phi || (P.g.l > 0 && !w)) return fail(ctx, VOMT_ERR_BAD_ARG, "null array");
    ctx->launches = 0;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaSetDevice");
    const int pitch = P.p.pitch;
    if (pitch != 0 && pitch != n) {
        // stage the pitched arrays densely, solve, copy the outputs back
        const size_t nn = (size_t)n * n, k = P.g.k, l = P.g.l;
        rc = ensure_buffer(ctx, (void **)&ctx->pstage, &ctx->pstage_bytes, sizeof(float) * (5 * k + l) * nn,
                           "pitch staging");
        if (rc) return rc;
        float *d0 = ctx->pstage, *d1 = d0 + k * nn, *du = d1 + k * nn, *dw = du + 2 * k * nn, *dp = dw + l * nn;
        e = copy_planes(d0, n, rho0, pitch, n, k, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = copy_planes(d1, n, rho1, pitch, n, k, cudaMemcpyDeviceToDevice, st);
        if (P.p.warm_start) {
            if (e == cudaSuccess) e = copy_planes(du, n, u, pitch, n, 2 * k, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess && l) e = copy_planes(dw, n, w, pitch, n, l, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = copy_planes(dp, n, phi, pitch, n, k, cudaMemcpyDeviceToDevice, st);
        }
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "pitched copy in");
        vomt_params dense = P.p;
        dense.pitch = 0;
        dense.tau = pin && pin->tau > 0.0 ? pin->tau : 0.0;
        dense.mu = pin ? pin->mu : 0.0;
        dense.nu = pin ? pin->nu : 0.0;
        const int status = solve_device(ctx, n, d0, d1, graph, alpha, &dense, du, dw, dp, result, st);
        if (status < 0) return status;
        e = copy_planes(u, pitch, du, n, n, 2 * k, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && l) e = copy_planes(w, pitch, dw, n, n, l, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = copy_planes(phi, pitch, dp, n, n, k, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "pitched copy out");
        return status;
    }
    rc = check_densities(ctx, P.g.k, n, rho0, rho1, st);
    if (rc) return rc;
    int engine = 0;
    rc = run_engine(ctx, P.g, P.s, P.cfg, P.p, rho0, rho1, u, w, phi, st, &engine);
    if (rc) return rc;
    int status = 0;
    fill_result(ctx, P.cfg, engine, result, &status);
    return status;
}

}  // namespace vomt

using namespace vomt;

extern "C" {

int vomt_create(vomt_ctx **out, int device)
{
    if (!out) return VOMT_ERR_BAD_ARG;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device < 0 || device >= count) return VOMT_ERR_CUDA;
    vomt_ctx *c = new (std::nothrow) vomt_ctx();
    if (!c) return VOMT_ERR_BAD_ARG;
    c->device = device;
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&c->dstatus, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost(&c->hstatus, 2 * sizeof(DevStatus));
    if (e != cudaSuccess) {
        vomt_destroy(c);
        return VOMT_ERR_CUDA;
    }
    memset(c->hstatus, 0, 2 * sizeof(DevStatus));
    *out = c;
    return VOMT_OK;
}

void vomt_destroy(vomt_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->ws) cudaFree(c->ws);
    if (c->partials) cudaFree(c->partials);
    if (c->dstatus) cudaFree(c->dstatus);
    if (c->hstatus) cudaFreeHost(c->hstatus);
    if (c->dhist) cudaFree(c->dhist);
    if (c->stage) cudaFree(c->stage);
    if (c->pstage) cudaFree(c->pstage);
    if (c->mstage) cudaFree(c->mstage);
    if (c->batch) batch_state_free(c->batch);
    if (c->gbuf) cudaFree(c->gbuf);
    if (c->gpart) cudaFree(c->gpart);
    if (c->rscratch) cudaFree(c->rscratch);
    delete c;
}

const char *vomt_status_str(int s)
{
    switch (s) {
        case VOMT_OK: return "ok";
        case VOMT_NOT_CONVERGED: return "iteration cap reached before the tolerance";
        case VOMT_ERR_BAD_ARG: return "invalid argument";
        case VOMT_ERR_MASS_MISMATCH: return "densities have different total mass";
        case VOMT_ERR_NEGATIVE_DENSITY: return "negative density entry";
        case VOMT_ERR_GRAPH: return "invalid or disconnected channel graph";
        case VOMT_ERR_L_KERNEL: return "ker grad_L on symmetric matrices is larger than span{I}";
        case VOMT_ERR_STEP_CONDITION: return "step sizes violate the PDHG convergence condition";
        case VOMT_ERR_NONFINITE: return "non-finite input or iterate";
        case VOMT_ERR_BARRIER_TIMEOUT: return "device-side wait timed out";
        case VOMT_ERR_CUDA: return "CUDA runtime error";
        case VOMT_ERR_TOO_LARGE: return "problem exceeds a size limit";
        default: return "unknown status";
    }
}

const char *vomt_last_error(const vomt_ctx *c) { return c ? c->err.c_str() : "null context"; }

void vomt_default_params(vomt_params *p)
{
    if (!p) return;
    p->tau = 0.0;
    p->mu = 0.0;
    p->nu = 0.0;
    p->u_norm = VOMT_U_L12;
    p->w_norm = VOMT_W_L1;
    p->max_iters = 2000;
    p->check_every = 100;
    p->tol_gap = 0.0;
    p->tol_res = 0.0;
    p->warm_start = 0;
    p->engine = VOMT_ENGINE_AUTO;
    p->halo = 0;
    p->eps = 0.0;
    p->pitch = 0;
}

int vomt_step_sizes(int n, const vomt_graph *g, double tau, double *mu, double *nu, double *tau_used, double *lmax_graph)
{
    if (n < 2) return VOMT_ERR_BAD_ARG;
    GraphDev gd;
    std::string err;
    int rc = graph_to_dev(g, &gd, &err);
    if (rc) return rc;
    const double t = tau > 0.0 ? tau : default_tau(n);
    const double lm = graph_lmax(gd, g->cost);
    const double n1 = (double)(n - 1);
    if (mu) *mu = gd.l > 0 ? 1.0 / (32.0 * t * n1 * n1) : 1.0 / (16.0 * t * n1 * n1);
    if (nu) *nu = gd.l > 0 ? 1.0 / (4.0 * t * lm) : 0.0;
    if (tau_used) *tau_used = t;
    if (lmax_graph) *lmax_graph = lm;
    return VOMT_OK;
}

int vomt_solve(vomt_ctx *ctx, int n, const float *rho0, const float *rho1, const vomt_graph *g, double alpha,
               const vomt_params *p, float *u, float *w, float *phi, vomt_result *result, void *stream)
{
    try {
        return solve_device(ctx, n, rho0, rho1, g, alpha, p, u, w, phi, result, (cudaStream_t)stream);
    } catch (...) {
        return fail(ctx, VOMT_ERR_BAD_ARG, "internal exception");
    }
}

int vomt_solve_host(vomt_ctx *ctx, int n, const float *rho0, const float *rho1, const vomt_graph *g, double alpha,
                    const vomt_params *p, float *u, float *w, float *phi, vomt_result *result, void *stream)
{
    try {
        if (!ctx || !g || n < 2 || g->k < 1 || g->k > KVEC || g->n_edges < 0 || g->n_edges > LVEC)
            return fail(ctx, VOMT_ERR_BAD_ARG, "bad arguments");
        if (!rho0 || !rho1 || !u || !phi || (g->n_edges > 0 && !w)) return fail(ctx, VOMT_ERR_BAD_ARG, "null array");
        cudaStream_t st = (cudaStream_t)stream;
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaSetDevice");
        const size_t nn = (size_t)n * n, k = g->k, l = g->n_edges;
        const int pitch = p && p->pitch ? p->pitch : n;
        if (pitch < n) return fail(ctx, VOMT_ERR_BAD_ARG, "pitch must be 0 or >= n");
        const size_t need = (2 * k + 2 * k + l + k) * nn;
        int rc = ensure_buffer(ctx, (void **)&ctx->stage, &ctx->stage_floats, need * sizeof(float), "staging");
        if (rc) return rc;
        float *d0 = ctx->stage, *d1 = d0 + k * nn, *du = d1 + k * nn, *dw = du + 2 * k * nn, *dp = dw + l * nn;
        const bool warm = p && p->warm_start;
        const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
        e = copy_planes(d0, n, rho0, pitch, n, k, h2d, st);
        if (e == cudaSuccess) e = copy_planes(d1, n, rho1, pitch, n, k, h2d, st);
        if (warm && e == cudaSuccess) e = copy_planes(du, n, u, pitch, n, 2 * k, h2d, st);
        if (warm && l && e == cudaSuccess) e = copy_planes(dw, n, w, pitch, n, l, h2d, st);
        if (warm && e == cudaSuccess) e = copy_planes(dp, n, phi, pitch, n, k, h2d, st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "host to device copy");
        vomt_params dense;
        vomt_default_params(&dense);
        if (p) dense = *p;
        dense.pitch = 0;
        int status = solve_device(ctx, n, d0, d1, g, alpha, &dense, du, dw, dp, result, st);
        if (status < 0) return status;
        e = copy_planes(u, pitch, du, n, n, 2 * k, d2h, st);
        if (l && e == cudaSuccess) e = copy_planes(w, pitch, dw, n, n, l, d2h, st);
        if (e == cudaSuccess) e = copy_planes(phi, pitch, dp, n, n, k, d2h, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "device to host copy");
        return status;
    } catch (...) {
        return fail(ctx, VOMT_ERR_BAD_ARG, "internal exception");
    }
}

extern "C" int vomt_set_wait_policy(vomt_ctx *ctx, double budget_ms, int drop_exchange)
{
    if (!ctx) return VOMT_ERR_BAD_ARG;
    if (!(budget_ms >= 0.0) || !isfinite(budget_ms) || budget_ms > 3.6e6 || drop_exchange < 0)
        return fail(ctx, VOMT_ERR_BAD_ARG, "budget_ms must be in [0, 3.6e6] and drop_exchange >= 0");
    ctx->wait_ns = (unsigned long long)(budget_ms * 1e6);
    ctx->drop_exchange = drop_exchange;
    return VOMT_OK;
}

int vomt_history(vomt_ctx *ctx, double *out, int cap)
{
    if (!ctx) return VOMT_ERR_BAD_ARG;
    int rows = ctx->last_checks < ctx->hist_cap ? ctx->last_checks : ctx->hist_cap;
    if (out && cap > 0 && rows > 0 && ctx->dhist) {
        int m = rows < cap ? rows : cap;
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e == cudaSuccess) e = cudaMemcpy(out, ctx->dhist, sizeof(double) * NMET * (size_t)m, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "history copy");
        if (ctx->hist_raw)
            for (int q = 0; q < m; ++q) finish_raw_row(out + (size_t)q * NMET);
    }
    return rows;
}

}  // extern "C"
