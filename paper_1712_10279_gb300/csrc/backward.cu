// Gradients of the vector-OMT cost.
//
// Envelope gradient.  V(rho0, rho1) is the value of the dual problem (eq.
// vomt-dual): a maximum over a feasible set that does not depend on the
// densities of the linear function <phi, rho1 - rho0>.  At a solution phi*,
// dV/drho1 = phi* and dV/drho0 = -phi*, up to the constant the dual leaves free
// (grad and grad_G vanish on a constant shared by all channels), fixed here by
// making phi* zero-mean.  V is also the value of the primal (eq. vomt), linear
// in alpha for fixed (u, w), so dV/dalpha = sum_ij ||w*_ij||_w.  One block per
// problem: an FP64 mean, then the scaled, centred copy.
//
// Unrolled gradient.  J_T = P(u^T, w^T), the primal objective after T
// iterations of Section 7.2 from the zero iterate, is differentiated by reverse
// mode through the T iterations.  The forward pass keeps the iterate every
// `ckpt` iterations; the reverse pass recomputes one segment at a time from its
// checkpoint and applies the transposed Jacobian of one iteration per step
// (k_adj_step): the chain rule through phi' = phi + tau(div_x ubar + div_G wbar +
// rho1 - rho0), through u' = shrink(u + mu grad phi; mu) and through
// w' = shrink_w(w + nu grad_G phi; alpha nu), with div_x^T = -grad_x
// (Appendix A) and div_G = -grad_G^* (Section 3.1).
#include <math.h>
#include <string.h>

#include <vector>

#include "internal.h"

namespace vomt {
namespace {

constexpr int AX = 32, AY = 8, AT = AX * AY;

__global__ void __launch_bounds__(1024) k_envelope(int n, int pitch, int k, int l, int wn, const float *__restrict__ phi,
                                                   const float *__restrict__ w, const float *__restrict__ gscale,
                                                   float *__restrict__ d_rho0, float *__restrict__ d_rho1,
                                                   float *__restrict__ d_alpha)
{
    // logical element q = (plane * n + j) * n + i sits at (plane * n + j) * pitch + i
    const size_t nn = (size_t)n * n, cnt = (size_t)k * nn;
    const size_t pcnt = (size_t)k * n * pitch, pw = (size_t)n * pitch;
    const float *P = phi + blockIdx.x * pcnt;
    const float *Wb = w + blockIdx.x * (size_t)l * pw;
    auto at = [n, pitch](size_t q) { return (q / (size_t)n) * (size_t)pitch + q % (size_t)n; };
    double s = 0.0, sw = 0.0;
    for (size_t q = threadIdx.x; q < cnt; q += blockDim.x) s += P[at(q)];
    for (size_t q = threadIdx.x; q < nn && l > 0; q += blockDim.x) {
        double a = 0.0;
        const size_t o = at(q);
        for (int e = 0; e < l; ++e) {
            const double x = Wb[e * pw + o];
            a += (wn == VOMT_W_L1) ? fabs(x) : x * x;
        }
        sw += (wn == VOMT_W_L1) ? a : sqrt(a);
    }
    __shared__ double sh[2][1024];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = sw;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + off];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + off];
        }
        __syncthreads();
    }
    const double mean = sh[0][0] / (double)cnt;
    const float g = gscale ? gscale[blockIdx.x] : 1.0f;
    for (size_t q = threadIdx.x; q < cnt; q += blockDim.x) {
        const size_t o = at(q);
        const float v = g * (float)((double)P[o] - mean);
        if (d_rho1) d_rho1[blockIdx.x * pcnt + o] = v;
        if (d_rho0) d_rho0[blockIdx.x * pcnt + o] = -v;
    }
    if (threadIdx.x == 0 && d_alpha) d_alpha[blockIdx.x] = (float)(g * sh[1][0]);
}

// transpose of the Jacobian of shrink_2(.; t) at v (a 2-vector), applied to H:
// (1 - t/s) H + t (v.H) v / s^3 for s = |v| > t, else 0
__device__ __forceinline__ void vjp_shrink2(float vx, float vy, float t, float hx, float hy, float &ox, float &oy)
{
    const float s2 = vx * vx + vy * vy;
    if (s2 > t * t) {
        const float r = rsqrtf(s2), s = s2 * r;
        const float a = 1.0f - t * r, c = t * (vx * hx + vy * hy) * r * r * r;
        (void)s;
        ox = a * hx + c * vx;
        oy = a * hy + c * vy;
    } else {
        ox = 0.0f;
        oy = 0.0f;
    }
}

template <int K>
struct ALK {
    static constexpr int v = K * (K - 1) / 2 > 0 ? K * (K - 1) / 2 : 1;
};

// Adjoint of J_T = P(u^T, w^T) with respect to the final iterate (||u||_{1,2},
// ||w||_1 or ||w||_2); per-block partial sums of J_T and of sum ||w^T|| go to
// part[blk][0..1].
template <int K>
__global__ void __launch_bounds__(AT) k_adj_init(int n, int l, int wn, float alpha, const float *__restrict__ S,
                                                  float *__restrict__ A, double *__restrict__ part)
{
    const int i = blockIdx.x * AX + threadIdx.x, j = blockIdx.y * AY + threadIdx.y;
    const size_t nn = (size_t)n * n;
    double jp = 0.0, wp = 0.0;
    if (i < n && j < n) {
        const size_t p = (size_t)j * n + i;
        for (int c = 0; c < K; ++c) {
            const float x = S[(K + c) * nn + p], y = S[(2 * K + c) * nn + p];
            const float s = sqrtf(x * x + y * y);
            jp += s;
            A[c * nn + p] = 0.0f;                                  // adjoint of phi^T
            A[(K + c) * nn + p] = s > 0.0f ? x / s : 0.0f;         // adjoint of u^T
            A[(2 * K + c) * nn + p] = s > 0.0f ? y / s : 0.0f;
        }
        float ws = 0.0f;
        for (int e = 0; e < l; ++e) {
            const float x = S[(3 * K + e) * nn + p];
            ws += (wn == VOMT_W_L1) ? fabsf(x) : x * x;
        }
        if (wn == VOMT_W_L2) ws = sqrtf(ws);
        for (int e = 0; e < l; ++e) {
            const float x = S[(3 * K + e) * nn + p];
            float gdir = (wn == VOMT_W_L1) ? (x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f)) : (ws > 0.0f ? x / ws : 0.0f);
            A[(3 * K + e) * nn + p] = alpha * gdir;
        }
        jp += (double)alpha * ws;
        wp = ws;
    }
    __shared__ double sh[2][AT];
    const int t = threadIdx.y * AX + threadIdx.x;
    sh[0][t] = jp;
    sh[1][t] = wp;
    __syncthreads();
    for (int off = AT / 2; off > 0; off >>= 1) {
        if (t < off) { sh[0][t] += sh[0][t + off]; sh[1][t] += sh[1][t + off]; }
        __syncthreads();
    }
    if (t == 0) {
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        part[blk * 2 + 0] = sh[0][0];
        part[blk * 2 + 1] = sh[1][0];
    }
}

// One reverse step: given the iterate s^t (S) and the adjoint of s^{t+1} (A1),
// write the adjoint of s^t (A0), add tau * (adjoint of phi^{t+1}) to grho (the
// derivative with respect to rho1; rho0 gets its negative) and add this block's
// contribution to dJ/dalpha to apart[blk].  ||u||_{1,2} (per channel shrink_2).
template <int K>
__global__ void __launch_bounds__(AT) k_adj_step(OpDev g, StepDev s, int wn, const float *__restrict__ S,
                                                 const float *__restrict__ A1, float *__restrict__ A0,
                                                 float *__restrict__ grho, double *__restrict__ apart)
{
    constexpr int LK = ALK<K>::v;
    const int n = s.n, l = g.l;
    const int i = blockIdx.x * AX + threadIdx.x, j = blockIdx.y * AY + threadIdx.y;
    double ga = 0.0;
    if (i < n && j < n) {
        const size_t nn = (size_t)n * n, p = (size_t)j * n + i;
        const bool hR = i < n - 1, hU = j < n - 1, hL = i > 0, hD = j > 0;
        const float mu = s.mu, nu = s.nu, tau = s.tau, ih = s.ih, muih = mu * ih;
        const float *phi = S, *ux = S + (size_t)K * nn, *uy = S + (size_t)2 * K * nn, *w = S + (size_t)3 * K * nn;
        const float *Gp = A1, *Gx = A1 + (size_t)K * nn, *Gy = A1 + (size_t)2 * K * nn, *Gw = A1 + (size_t)3 * K * nn;
        float qc[K], dvg[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const size_t o = c * nn + p;
            const float pc = phi[o], pr = hR ? phi[o + 1] : 0.0f, pu = hU ? phi[o + n] : 0.0f;
            const float pl = hL ? phi[o - 1] : 0.0f, plu = (hL && hU) ? phi[o - 1 + n] : 0.0f;
            const float pd = hD ? phi[o - n] : 0.0f, prd = (hR && hD) ? phi[o + 1 - n] : 0.0f;
            qc[c] = Gp[o];
            const float qr = hR ? Gp[o + 1] : 0.0f, qu = hU ? Gp[o + n] : 0.0f;
            const float ql = hL ? Gp[o - 1] : 0.0f, qlu = (hL && hU) ? Gp[o - 1 + n] : 0.0f;
            const float qd = hD ? Gp[o - n] : 0.0f, qrd = (hR && hD) ? Gp[o + 1 - n] : 0.0f;
            // at p
            const float ax = hR ? ih * (qr - qc[c]) : 0.0f, ay = hU ? ih * (qu - qc[c]) : 0.0f;
            const float vx = ux[o] + (hR ? muih * (pr - pc) : 0.0f), vy = uy[o] + (hU ? muih * (pu - pc) : 0.0f);
            float gvx, gvy;
            vjp_shrink2(vx, vy, mu, Gx[o] - 2.0f * tau * ax, Gy[o] - 2.0f * tau * ay, gvx, gvy);
            A0[(K + c) * nn + p] = gvx + tau * ax;
            A0[(2 * K + c) * nn + p] = gvy + tau * ay;
            // x component of the same quantity at (i-1, j)
            float glx = 0.0f;
            if (hL) {
                const float lax = ih * (qc[c] - ql), lay = hU ? ih * (qlu - ql) : 0.0f;
                const float lvx = ux[o - 1] + muih * (pc - pl), lvy = uy[o - 1] + (hU ? muih * (plu - pl) : 0.0f);
                float t_;
                vjp_shrink2(lvx, lvy, mu, Gx[o - 1] - 2.0f * tau * lax, Gy[o - 1] - 2.0f * tau * lay, glx, t_);
            }
            // y component at (i, j-1)
            float gdy = 0.0f;
            if (hD) {
                const float dax = hR ? ih * (qrd - qd) : 0.0f, day = ih * (qc[c] - qd);
                const float dvx = ux[o - n] + (hR ? muih * (prd - pd) : 0.0f), dvy = uy[o - n] + muih * (pc - pd);
                float t_;
                vjp_shrink2(dvx, dvy, mu, Gx[o - n] - 2.0f * tau * dax, Gy[o - n] - 2.0f * tau * day, t_, gdy);
            }
            dvg[c] = ih * ((gvx - glx) + (gvy - gdy));      // div of the shrink adjoint at p
        }
        // graph part at p
        float xw[LK], hw[LK], gxw[LK];
#pragma unroll
        for (int e = 0; e < LK; ++e) {
            float ge = 0.0f, dq = 0.0f;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                ge += g.G[e][c] * phi[c * nn + p];
                dq += g.Dv[c][e] * qc[c];
            }
            xw[e] = (e < l) ? w[e * nn + p] + nu * ge : 0.0f;
            hw[e] = (e < l) ? Gw[e * nn + p] - 2.0f * tau * dq : 0.0f;
            gxw[e] = 0.0f;
            if (e < l) A0[(3 * K + e) * nn + p] = tau * dq;
        }
        const float th = s.alpha * nu;
        if (wn == VOMT_W_L1) {
#pragma unroll
            for (int e = 0; e < LK; ++e)
                if (e < l && fabsf(xw[e]) > th) {
                    gxw[e] = hw[e];
                    ga += -(double)nu * (xw[e] > 0.0f ? 1.0 : -1.0) * (double)hw[e];
                }
        } else {
            float s2 = 0.0f, xh = 0.0f;
#pragma unroll
            for (int e = 0; e < LK; ++e) { s2 += xw[e] * xw[e]; xh += xw[e] * hw[e]; }
            if (s2 > th * th) {
                const float r = rsqrtf(s2);
                const float a = 1.0f - th * r, c3 = th * xh * r * r * r;
#pragma unroll
                for (int e = 0; e < LK; ++e) gxw[e] = a * hw[e] + c3 * xw[e];
                ga += -(double)nu * (double)(xh * r);
            }
        }
#pragma unroll
        for (int e = 0; e < LK; ++e)
            if (e < l) A0[(3 * K + e) * nn + p] += gxw[e];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            float gg = 0.0f;
#pragma unroll
            for (int e = 0; e < LK; ++e) gg += g.G[e][c] * gxw[e];
            A0[c * nn + p] = qc[c] - mu * dvg[c] + nu * gg;
            grho[c * nn + p] += tau * qc[c];
        }
    }
    __shared__ double sh[AT];
    const int t = threadIdx.y * AX + threadIdx.x;
    sh[t] = ga;
    __syncthreads();
    for (int off = AT / 2; off > 0; off >>= 1) {
        if (t < off) sh[t] += sh[t + off];
        __syncthreads();
    }
    if (t == 0) apart[blockIdx.y * gridDim.x + blockIdx.x] += sh[0];
}

__global__ void k_sub(size_t cnt, const float *__restrict__ r0, const float *__restrict__ r1, float *__restrict__ b)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < cnt; q += (size_t)gridDim.x * blockDim.x)
        b[q] = r1[q] - r0[q];
}

__global__ void k_finish_grad(size_t cnt, float scale, const float *__restrict__ grho, float *__restrict__ d_rho0,
                              float *__restrict__ d_rho1)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < cnt; q += (size_t)gridDim.x * blockDim.x) {
        if (d_rho1) d_rho1[q] = scale * grho[q];
        if (d_rho0) d_rho0[q] = -scale * grho[q];
    }
}

using AdjInit = void (*)(int, int, int, float, const float *, float *, double *);
using AdjStep = void (*)(OpDev, StepDev, int, const float *, const float *, float *, float *, double *);

template <int K>
void pick_adj_k(AdjInit *ai, AdjStep *as)
{
    *ai = k_adj_init<K>;
    *as = k_adj_step<K>;
}

void pick_adj(int k, AdjInit *ai, AdjStep *as)
{
    switch (k) {
        case 1: pick_adj_k<1>(ai, as); break;
        case 2: pick_adj_k<2>(ai, as); break;
        case 3: pick_adj_k<3>(ai, as); break;
        case 4: pick_adj_k<4>(ai, as); break;
        case 5: pick_adj_k<5>(ai, as); break;
        case 6: pick_adj_k<6>(ai, as); break;
        case 7: pick_adj_k<7>(ai, as); break;
        default: pick_adj_k<8>(ai, as); break;
    }
}

}  // namespace
}  // namespace vomt

using namespace vomt;

extern "C" int vomt_backward(vomt_ctx *ctx, int batch, int n, int pitch, int k, int n_edges, int w_norm,
                             const float *phi, const float *w, const float *grad_scale, float *d_rho0, float *d_rho1,
                             float *d_alpha, void *stream)
{
    if (!ctx) return VOMT_ERR_BAD_ARG;
    ctx->err.clear();
    if (batch < 1 || n < 2 || k < 1 || k > KVEC || n_edges < 0 || n_edges > LVEC || w_norm < 0 || w_norm > 1)
        return fail(ctx, VOMT_ERR_BAD_ARG, "backward: bad sizes");
    if (pitch == 0) pitch = n;
    if (pitch < n) return fail(ctx, VOMT_ERR_BAD_ARG, "backward: pitch must be 0 or >= n");
    if (!phi || (n_edges > 0 && !w)) return fail(ctx, VOMT_ERR_BAD_ARG, "backward: null array");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaSetDevice");
    k_envelope<<<batch, 1024, 0, (cudaStream_t)stream>>>(n, pitch, k, n_edges, w_norm, phi, w, grad_scale, d_rho0,
                                                         d_rho1, d_alpha);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "backward launch");
    return VOMT_OK;
}

extern "C" int vomt_unrolled_grad(vomt_ctx *ctx, int n, const float *rho0, const float *rho1, const vomt_graph *graph,
                                  double alpha, const vomt_params *pin, int T, int ckpt, double scale, float *d_rho0,
                                  float *d_rho1, double *d_alpha, double *J, void *stream)
{
    try {
        if (!ctx) return VOMT_ERR_BAD_ARG;
        OpDev op;
        StepDev s;
        SolveCfg cfg;
        vomt_params p;
        int rc = prepare_vector(ctx, n, graph, alpha, pin, &op, &s, &cfg, &p);
        if (rc) return rc;
        if (p.eps != 0.0) return fail(ctx, VOMT_ERR_BAD_ARG, "the unrolled gradient takes eps = 0");
        if (p.u_norm != VOMT_U_L12) return fail(ctx, VOMT_ERR_BAD_ARG, "unrolled gradient: u_norm must be VOMT_U_L12");
        if (T < 1 || ckpt < 1) return fail(ctx, VOMT_ERR_BAD_ARG, "unrolled gradient: T >= 1 and ckpt >= 1");
        if (!rho0 || !rho1) return fail(ctx, VOMT_ERR_BAD_ARG, "null array");
        cudaStream_t st = (cudaStream_t)stream;
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaSetDevice");
        ctx->launches = 0;
        rc = check_vector_densities(ctx, op.k, n, rho0, rho1, st);
        if (rc) return rc;
        const int K = op.k, l = op.l;
        const size_t nn = (size_t)n * n, SZ = (size_t)(3 * K + l) * nn;
        const int nck = T / ckpt + 1;
        const size_t floats = (size_t)2 * K * nn + ((size_t)nck + ckpt + 1 + 2) * SZ;
        rc = ensure_buffer(ctx, (void **)&ctx->gbuf, &ctx->gbuf_bytes, floats * sizeof(float), "gradient scratch");
        if (rc) return rc;
        const dim3 blk(AX, AY), grd((n + AX - 1) / AX, (n + AY - 1) / AY);
        const int nb = (int)(grd.x * grd.y);
        rc = ensure_buffer(ctx, (void **)&ctx->gpart, &ctx->gpart_bytes, sizeof(double) * 3 * (size_t)nb, "gradient sums");
        if (rc) return rc;
        float *b = ctx->gbuf, *grho = b + (size_t)K * nn;
        float *ck = grho + (size_t)K * nn;                  // nck checkpoints
        float *seg = ck + (size_t)nck * SZ;                 // ckpt + 1 recompute slots
        float *adj = seg + (size_t)(ckpt + 1) * SZ;         // 2 adjoint states
        double *part = ctx->gpart, *apart = part + 2 * (size_t)nb;
        const int pb = (int)(((size_t)K * nn + 255) / 256 < 2048 ? ((size_t)K * nn + 255) / 256 : 2048);
        e = cudaMemsetAsync(ctx->dstatus, 0, sizeof(DevStatus), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ck, 0, SZ * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(grho, 0, (size_t)K * nn * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(apart, 0, sizeof(double) * nb, st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "gradient reset");
        k_sub<<<pb, 256, 0, st>>>((size_t)K * nn, rho0, rho1, b);
        ++ctx->launches;
        // forward, keeping every ckpt-th iterate
        const float *cur = ck;
        for (int t = 1; t <= T; ++t) {
            float *out = (t % ckpt == 0) ? ck + (size_t)(t / ckpt) * SZ : seg + (size_t)(t & 1) * SZ;
            launch_step(op, s, p.u_norm, p.w_norm, cur, out, b, ctx->dstatus, st);
            ++ctx->launches;
            cur = out;
        }
        AdjInit ai;
        AdjStep as;
        pick_adj(K, &ai, &as);
        ai<<<grd, blk, 0, st>>>(n, l, p.w_norm, s.alpha, cur, adj, part);
        ++ctx->launches;
        // reverse, one checkpoint segment at a time
        int a_in = 0;
        for (int sg = (T - 1) / ckpt; sg >= 0; --sg) {
            const int t0 = sg * ckpt, t1 = (t0 + ckpt < T) ? t0 + ckpt : T;
            const float *base = ck + (size_t)sg * SZ;
            for (int m = 1; m < t1 - t0; ++m) {
                const float *in = (m == 1) ? base : seg + (size_t)(m - 1) * SZ;
                launch_step(op, s, p.u_norm, p.w_norm, in, seg + (size_t)m * SZ, b, ctx->dstatus, st);
                ++ctx->launches;
            }
            for (int t = t1 - 1; t >= t0; --t) {
                const float *St = (t == t0) ? base : seg + (size_t)(t - t0) * SZ;
                as<<<grd, blk, 0, st>>>(op, s, p.w_norm, St, adj + (size_t)a_in * SZ, adj + (size_t)(1 - a_in) * SZ,
                                        grho, apart);
                ++ctx->launches;
                a_in = 1 - a_in;
            }
        }
        k_finish_grad<<<pb, 256, 0, st>>>((size_t)K * nn, (float)scale, grho, d_rho0, d_rho1);
        ++ctx->launches;
        std::vector<double> hp((size_t)3 * nb);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "unrolled gradient");
        double jv = 0.0, ws = 0.0, ga = 0.0;
        for (int q = 0; q < nb; ++q) {
            jv += hp[2 * q];
            ws += hp[2 * q + 1];
            ga += hp[2 * nb + q];
        }
        if (J) *J = jv;
        if (d_alpha) *d_alpha = scale * (ws + ga);
        if (!isfinite(jv)) return fail(ctx, VOMT_ERR_NONFINITE, "unrolled objective is not finite");
        return VOMT_OK;
    } catch (...) {
        return fail(ctx, VOMT_ERR_BAD_ARG, "internal exception");
    }
}
