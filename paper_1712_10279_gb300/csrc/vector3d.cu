// Vector OMT on 3-D grids: the discretization of Appendix A with a third
// direction (the extension to volumes that the paper points to for 3-D DTI,
// Section 8.2), solved by the streaming engine's scheme: one fused launch per
// PDHG iteration (Section 7.2), FP64 convergence checks.
//
// Grid n x n x n on [0,1]^3, h = 1/(n-1); every field is planar [c][z][y][x]
// with x fastest; the flux has three components u_x, u_y, u_z per channel, with
// ghost entries at the last index of their own direction (kept zero).  One
// thread per point computes u' at its point and at its three upwind neighbours
// (their components enter the backward-difference divergence at the point), w'
// and phi'.  Step rule: ||grad||^2 <= 12 / h^2 in 3-D, so mu = 1/(48 tau (n-1)^2)
// (1/(24 tau (n-1)^2) without edges) keeps the 2-D rule's share of the bound.
#include <math.h>
#include <string.h>

#include "internal.h"
#include "pdhg_device.cuh"

namespace vomt {
namespace {

using dev::shrink2_factor;
using dev::soft;

constexpr int T3 = 256;

struct S3In {
    const float *phi, *ux, *uy, *uz, *w;
};
struct S3Out {
    float *phi, *ux, *uy, *uz, *w;
};

template <int K>
struct LK3 {
    static constexpr int v = K * (K - 1) / 2 > 0 ? K * (K - 1) / 2 : 1;
};

template <int K, int UN>
__device__ __forceinline__ void shrink_u3(float (&a)[K], float (&b)[K], float (&c)[K], float t, const float *wc)
{
    if (UN == VOMT_U_L12) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const float f = shrink2_factor(a[q] * a[q] + b[q] * b[q] + c[q] * c[q], t);
            a[q] *= f;
            b[q] *= f;
            c[q] *= f;
        }
    } else if (UN == VOMT_U_L2) {
        float s2 = 0.0f;
#pragma unroll
        for (int q = 0; q < K; ++q) s2 += wc[q] * (a[q] * a[q] + b[q] * b[q] + c[q] * c[q]);
        const float f = shrink2_factor(s2, t);
#pragma unroll
        for (int q = 0; q < K; ++q) { a[q] *= f; b[q] *= f; c[q] *= f; }
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) { a[q] = soft(a[q], t); b[q] = soft(b[q], t); c[q] = soft(c[q], t); }
    }
}

template <int LK, int WN>
__device__ __forceinline__ void shrink_w3(float (&x)[LK], int l, float t, const float *we)
{
    if (WN == VOMT_W_L1) {
#pragma unroll
        for (int e = 0; e < LK; ++e)
            if (e < l) x[e] = soft(x[e], t);
    } else {
        float s2 = 0.0f;
#pragma unroll
        for (int e = 0; e < LK; ++e)
            if (e < l) s2 += we[e] * x[e] * x[e];
        const float f = shrink2_factor(s2, t);
#pragma unroll
        for (int e = 0; e < LK; ++e) x[e] *= f;
    }
}

template <int K, int UN, int WN>
__global__ void __launch_bounds__(T3) k_step3(S3In in, S3Out out, const float *__restrict__ b, OpDev g, StepDev s,
                                              const DevStatus *__restrict__ st)
{
    if (st->stop) return;
    constexpr int LK = LK3<K>::v;
    const int n = s.n;
    const size_t m = (size_t)n * n * n;
    const size_t p = (size_t)blockIdx.x * T3 + threadIdx.x;
    if (p >= m) return;
    const int x = (int)(p % n), y = (int)((p / n) % n), z = (int)(p / ((size_t)n * n));
    const long SX = 1, SY = n, SZ = (long)n * n;
    const bool hx = x < n - 1, hy = y < n - 1, hz = z < n - 1, lx = x > 0, ly = y > 0, lz = z > 0;
    const float mi = s.mu * s.ih;
    float pc[K], px[K], py[K], pz[K], mx[K], mxy[K], mxz[K], my[K], myx[K], myz[K], mz[K], mzx[K], mzy[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const float *P = in.phi + c * m + p;
        pc[c] = __ldg(P);
        px[c] = hx ? __ldg(P + SX) : 0.0f;
        py[c] = hy ? __ldg(P + SY) : 0.0f;
        pz[c] = hz ? __ldg(P + SZ) : 0.0f;
        mx[c] = lx ? __ldg(P - SX) : 0.0f;
        mxy[c] = (lx && hy) ? __ldg(P - SX + SY) : 0.0f;
        mxz[c] = (lx && hz) ? __ldg(P - SX + SZ) : 0.0f;
        my[c] = ly ? __ldg(P - SY) : 0.0f;
        myx[c] = (ly && hx) ? __ldg(P - SY + SX) : 0.0f;
        myz[c] = (ly && hz) ? __ldg(P - SY + SZ) : 0.0f;
        mz[c] = lz ? __ldg(P - SZ) : 0.0f;
        mzx[c] = (lz && hx) ? __ldg(P - SZ + SX) : 0.0f;
        mzy[c] = (lz && hy) ? __ldg(P - SZ + SY) : 0.0f;
    }
    // u' at the point
    float ux0[K], uy0[K], uz0[K], vx[K], vy[K], vz[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const size_t q = c * m + p;
        ux0[c] = __ldg(in.ux + q);
        uy0[c] = __ldg(in.uy + q);
        uz0[c] = __ldg(in.uz + q);
        vx[c] = ux0[c] + (hx ? mi * (px[c] - pc[c]) : 0.0f);
        vy[c] = uy0[c] + (hy ? mi * (py[c] - pc[c]) : 0.0f);
        vz[c] = uz0[c] + (hz ? mi * (pz[c] - pc[c]) : 0.0f);
    }
    shrink_u3<K, UN>(vx, vy, vz, s.mu, g.wc);
    // u' at (x-1): its x component enters div at the point
    float ax[K], ay[K], az[K], ax0[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const size_t q = c * m + p;
        ax0[c] = lx ? __ldg(in.ux + q - SX) : 0.0f;
        const float ay0 = lx ? __ldg(in.uy + q - SX) : 0.0f, az0 = lx ? __ldg(in.uz + q - SX) : 0.0f;
        ax[c] = ax0[c] + (lx ? mi * (pc[c] - mx[c]) : 0.0f);
        ay[c] = ay0 + ((lx && hy) ? mi * (mxy[c] - mx[c]) : 0.0f);
        az[c] = az0 + ((lx && hz) ? mi * (mxz[c] - mx[c]) : 0.0f);
    }
    shrink_u3<K, UN>(ax, ay, az, s.mu, g.wc);
    // u' at (y-1): its y component
    float bx[K], by[K], bz[K], by0[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const size_t q = c * m + p;
        by0[c] = ly ? __ldg(in.uy + q - SY) : 0.0f;
        const float bx0 = ly ? __ldg(in.ux + q - SY) : 0.0f, bz0 = ly ? __ldg(in.uz + q - SY) : 0.0f;
        bx[c] = bx0 + ((ly && hx) ? mi * (myx[c] - my[c]) : 0.0f);
        by[c] = by0[c] + (ly ? mi * (pc[c] - my[c]) : 0.0f);
        bz[c] = bz0 + ((ly && hz) ? mi * (myz[c] - my[c]) : 0.0f);
    }
    shrink_u3<K, UN>(bx, by, bz, s.mu, g.wc);
    // u' at (z-1): its z component
    float cx[K], cy[K], cz[K], cz0[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const size_t q = c * m + p;
        cz0[c] = lz ? __ldg(in.uz + q - SZ) : 0.0f;
        const float cx0 = lz ? __ldg(in.ux + q - SZ) : 0.0f, cy0 = lz ? __ldg(in.uy + q - SZ) : 0.0f;
        cx[c] = cx0 + ((lz && hx) ? mi * (mzx[c] - mz[c]) : 0.0f);
        cy[c] = cy0 + ((lz && hy) ? mi * (mzy[c] - mz[c]) : 0.0f);
        cz[c] = cz0[c] + (lz ? mi * (pc[c] - mz[c]) : 0.0f);
    }
    shrink_u3<K, UN>(cx, cy, cz, s.mu, g.wc);
    // w' at the point
    float w0[LK], wx[LK];
#pragma unroll
    for (int e = 0; e < LK; ++e) {
        if (e < g.l) {
            w0[e] = __ldg(in.w + e * m + p);
            float ge = 0.0f;
#pragma unroll
            for (int c = 0; c < K; ++c) ge += g.G[e][c] * pc[c];
            wx[e] = w0[e] + s.nu * ge;
        } else {
            w0[e] = 0.0f;
            wx[e] = 0.0f;
        }
    }
    shrink_w3<LK, WN>(wx, g.l, s.alpha * s.nu, g.we);
    // phi' = phi + tau (div ubar + div_G wbar + rho1 - rho0)
    float r[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const float bxc = 2.0f * vx[c] - ux0[c], byc = 2.0f * vy[c] - uy0[c], bzc = 2.0f * vz[c] - uz0[c];
        const float bxl = lx ? 2.0f * ax[c] - ax0[c] : 0.0f;
        const float byl = ly ? 2.0f * by[c] - by0[c] : 0.0f;
        const float bzl = lz ? 2.0f * cz[c] - cz0[c] : 0.0f;
        r[c] = s.ih * ((bxc - bxl) + (byc - byl) + (bzc - bzl)) + __ldg(b + c * m + p);
    }
#pragma unroll
    for (int e = 0; e < LK; ++e) {
        const float v = 2.0f * wx[e] - w0[e];
#pragma unroll
        for (int c = 0; c < K; ++c) r[c] -= g.Dv[c][e] * v;
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const size_t q = c * m + p;
        out.phi[q] = pc[c] + s.tau * r[c];
        out.ux[q] = vx[c];
        out.uy[q] = vy[c];
        out.uz[q] = vz[c];
    }
#pragma unroll
    for (int e = 0; e < LK; ++e)
        if (e < g.l) out.w[e * m + p] = wx[e];
}

// FP64 block partials of one convergence check (slots RED_*): per-point terms in
// FP32 (the constraint residual in FP64), summed per block in FP64.
template <int K, int UN, int WN>
__global__ void __launch_bounds__(T3) k_metrics3(S3In cur, S3In prv, const float *__restrict__ b, OpDev g,
                                                 StepDev s, double *__restrict__ partials,
                                                 const DevStatus *__restrict__ st)
{
    if (st->stop) return;
    constexpr int LK = LK3<K>::v;
    const int n = s.n;
    const size_t m = (size_t)n * n * n;
    const size_t p = (size_t)blockIdx.x * T3 + threadIdx.x;
    double v[NRED];
#pragma unroll
    for (int q = 0; q < NRED; ++q) v[q] = 0.0;
    if (p < m) {
        const int x = (int)(p % n), y = (int)((p / n) % n), z = (int)(p / ((size_t)n * n));
        const long SX = 1, SY = n, SZ = (long)n * n;
        const bool hx = x < n - 1, hy = y < n - 1, hz = z < n - 1, lx = x > 0, ly = y > 0, lz = z > 0;
        const float ih = s.ih, alpha = s.alpha;
        const double dih = (double)(n - 1);
        float ph[K], dph[K], ddiv[K], gwb[K];
        double rdiv[K];
        float nu_pt = 0.0f, dn_u = 0.0f, fdu = 0.0f, fdp = 0.0f, fd = 0.0f, fbb = 0.0f, fdw = 0.0f, fx = 0.0f;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const size_t q = c * m + p;
            const float a = cur.ux[q], bq = cur.uy[q], cq = cur.uz[q], bc = b[q], wgt = g.wc[c];
            ph[c] = cur.phi[q];
            dph[c] = ph[c] - prv.phi[q];
            const float al = lx ? cur.ux[q - SX] : 0.0f, bl = ly ? cur.uy[q - SY] : 0.0f,
                        cl = lz ? cur.uz[q - SZ] : 0.0f;
            rdiv[c] = dih * ((((double)a - (double)al) + ((double)bq - (double)bl)) + ((double)cq - (double)cl));
            gwb[c] = bc;
            const float da = a - prv.ux[q], db = bq - prv.uy[q], dc = cq - prv.uz[q];
            const float dal = lx ? cur.ux[q - SX] - prv.ux[q - SX] : 0.0f;
            const float dbl = ly ? cur.uy[q - SY] - prv.uy[q - SY] : 0.0f;
            const float dcl = lz ? cur.uz[q - SZ] - prv.uz[q - SZ] : 0.0f;
            ddiv[c] = ih * ((da - dal) + (db - dbl) + (dc - dcl));
            fdu += wgt * (da * da + db * db + dc * dc);
            fdp += wgt * dph[c] * dph[c];
            fd += wgt * ph[c] * bc;
            fbb += wgt * bc * bc;
            const float gx = hx ? ih * (cur.phi[q + SX] - ph[c]) : 0.0f;
            const float gy = hy ? ih * (cur.phi[q + SY] - ph[c]) : 0.0f;
            const float gz = hz ? ih * (cur.phi[q + SZ] - ph[c]) : 0.0f;
            if (UN == VOMT_U_L12) {
                nu_pt += sqrtf(a * a + bq * bq + cq * cq);
                dn_u = fmaxf(dn_u, sqrtf(gx * gx + gy * gy + gz * gz));
            } else if (UN == VOMT_U_L2) {
                nu_pt += wgt * (a * a + bq * bq + cq * cq);
                dn_u += wgt * (gx * gx + gy * gy + gz * gz);
            } else {
                nu_pt += wgt * (fabsf(a) + fabsf(bq) + fabsf(cq));
                dn_u = fmaxf(dn_u, fmaxf(fabsf(gx), fmaxf(fabsf(gy), fabsf(gz))));
            }
        }
        if (UN == VOMT_U_L2) { nu_pt = sqrtf(nu_pt); dn_u = sqrtf(dn_u); }
        float nw_pt = 0.0f, dn_w = 0.0f;
#pragma unroll
        for (int e = 0; e < LK; ++e) {
            if (e < g.l) {
                const size_t q = e * m + p;
                const float we = cur.w[q], dwe = we - prv.w[q], wgt = g.we[e];
                fdw += wgt * dwe * dwe;
                float ge = 0.0f;
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    ge += g.G[e][c] * ph[c];
                    gwb[c] -= g.Dv[c][e] * we;
                    ddiv[c] -= g.Dv[c][e] * dwe;
                }
                if (WN == VOMT_W_L1) { nw_pt += wgt * fabsf(we); dn_w = fmaxf(dn_w, fabsf(ge)); }
                else { nw_pt += wgt * we * we; dn_w += wgt * ge * ge; }
            }
        }
        if (WN == VOMT_W_L2) { nw_pt = sqrtf(nw_pt); dn_w = sqrtf(dn_w); }
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const double rc = rdiv[c] + (double)gwb[c];
            v[RED_RR] += (double)g.wc[c] * rc * rc;
            fx += g.wc[c] * dph[c] * ddiv[c];
        }
        v[RED_P] = (double)(nu_pt + alpha * nw_pt);
        v[RED_D] = (double)fd;
        v[RED_BB] = (double)fbb;
        v[RED_DU] = (double)fdu;
        v[RED_DW] = (double)fdw;
        v[RED_DP] = (double)fdp;
        v[RED_X] = (double)fx;
        float di = fmaxf(dn_u - 1.0f, 0.0f);
        if (g.l > 0) di = fmaxf(di, dn_w - alpha);
        v[RED_MAX] = (double)di;
    }
    // fixed-order block reduction
    __shared__ double sh[T3 / 32][NRED];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NRED; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_down_sync(0xffffffffu, v[q], off);
            v[q] = (q == RED_MAX) ? fmax(v[q], o) : v[q] + o;
        }
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NRED; ++q) sh[wid][q] = v[q];
    __syncthreads();
    if (wid == 0 && lane < NRED) {
        double a = sh[0][lane];
        for (int w2 = 1; w2 < T3 / 32; ++w2) a = (lane == RED_MAX) ? fmax(a, sh[w2][lane]) : a + sh[w2][lane];
        partials[(size_t)blockIdx.x * NRED + lane] = a;
    }
}

__global__ void k_prepare3(size_t m, int k, int l, const float *__restrict__ rho0, const float *__restrict__ rho1,
                           float *__restrict__ b, int warm, const float *__restrict__ u_in,
                           const float *__restrict__ w_in, const float *__restrict__ phi_in, S3Out s0)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < m; q += (size_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < k; ++c) {
            b[c * m + q] = rho1[c * m + q] - rho0[c * m + q];
            s0.phi[c * m + q] = warm ? phi_in[c * m + q] : 0.0f;
            s0.ux[c * m + q] = warm ? u_in[c * m + q] : 0.0f;
            s0.uy[c * m + q] = warm ? u_in[(k + c) * m + q] : 0.0f;
            s0.uz[c * m + q] = warm ? u_in[(2 * k + c) * m + q] : 0.0f;
        }
        for (int e = 0; e < l; ++e) s0.w[e * m + q] = warm ? w_in[e * m + q] : 0.0f;
    }
}

__global__ void k_copy_out3(size_t m, int k, int l, S3In s0, S3In s1, const DevStatus *st, float *u, float *w,
                            float *phi)
{
    const S3In &s = (st->iter & 1) ? s1 : s0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < m; q += (size_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < k; ++c) {
            phi[c * m + q] = s.phi[c * m + q];
            u[c * m + q] = s.ux[c * m + q];
            u[(k + c) * m + q] = s.uy[c * m + q];
            u[(2 * k + c) * m + q] = s.uz[c * m + q];
        }
        for (int e = 0; e < l; ++e) w[e * m + q] = s.w[e * m + q];
    }
}

struct L3 {
    void (*step)(S3In, S3Out, const float *, OpDev, StepDev, const DevStatus *);
    void (*metrics)(S3In, S3In, const float *, OpDev, StepDev, double *, const DevStatus *);
};

template <int K, int UN, int WN>
L3 make3()
{
    return L3{k_step3<K, UN, WN>, k_metrics3<K, UN, WN>};
}

template <int K>
L3 pick3_norms(int un, int wn)
{
    if (un == VOMT_U_L12) return wn == VOMT_W_L1 ? make3<K, 0, 0>() : make3<K, 0, 1>();
    if (un == VOMT_U_L2) return wn == VOMT_W_L1 ? make3<K, 1, 0>() : make3<K, 1, 1>();
    return wn == VOMT_W_L1 ? make3<K, 2, 0>() : make3<K, 2, 1>();
}

L3 pick3(int k, int un, int wn)
{
    switch (k) {
        case 1: return pick3_norms<1>(un, wn);
        case 2: return pick3_norms<2>(un, wn);
        case 3: return pick3_norms<3>(un, wn);
        case 4: return pick3_norms<4>(un, wn);
        case 5: return pick3_norms<5>(un, wn);
        case 6: return pick3_norms<6>(un, wn);
        case 7: return pick3_norms<7>(un, wn);
        default: return pick3_norms<8>(un, wn);
    }
}

}  // namespace
}  // namespace vomt

using namespace vomt;

extern "C" int vomt_solve3d(vomt_ctx *ctx, int n, const float *rho0, const float *rho1, const vomt_graph *graph,
                            double alpha, const vomt_params *pin, float *u, float *w, float *phi,
                            vomt_result *result, void *stream)
{
    try {
        if (!ctx) return VOMT_ERR_BAD_ARG;
        ctx->err.clear();
        ctx->launches = 0;
        ctx->last_blocks = 0;
        ctx->last_halo = 0;
        if (n < 2 || n > 1024) return fail(ctx, VOMT_ERR_BAD_ARG, "3-D grids: n must be in [2, 1024]");
        if (!rho0 || !rho1 || !u || !phi || !graph || (graph->n_edges > 0 && !w))
            return fail(ctx, VOMT_ERR_BAD_ARG, "null array");
        if (pin && pin->eps != 0.0) return fail(ctx, VOMT_ERR_BAD_ARG, "3-D grids take eps = 0");
        cudaStream_t st = (cudaStream_t)stream;
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaSetDevice");
        OpDev g;
        StepDev s;
        SolveCfg cfg;
        vomt_params p;
        int rc = prepare_vector(ctx, n, graph, alpha, pin, &g, &s, &cfg, &p);
        if (rc) return rc;
        // the 3-D step rule: ||grad||^2 <= 12 (n-1)^2, so mu takes 1/(48 tau (n-1)^2)
        // (1/(24 ...) without edges), the 2-D rule's share of the bound
        const double n1 = (double)(n - 1), tau = cfg.tau;
        const bool user = pin && (pin->mu > 0.0 || pin->nu > 0.0);
        const double mu = pin && pin->mu > 0.0 ? pin->mu
                                               : (g.l > 0 ? 1.0 / (48.0 * tau * n1 * n1) : 1.0 / (24.0 * tau * n1 * n1));
        double lmax = 0.0;
        if (g.l > 0) {
            rc = vomt_step_sizes(n, graph, tau, nullptr, nullptr, nullptr, &lmax);
            if (rc) return fail(ctx, rc, "bad graph");
        }
        if (user && !(tau * mu * 12.0 * n1 * n1 + (g.l > 0 ? tau * cfg.nu * lmax : 0.0) < 1.0))
            return fail(ctx, VOMT_ERR_STEP_CONDITION,
                        "step sizes break 1 > tau mu 12(n-1)^2 + tau nu lambda_max(-Delta_G)");
        s.mu = (float)mu;
        cfg.mu = mu;
        p.mu = mu;
        const int k = g.k, l = g.l;
        const size_t m = (size_t)n * n * n;
        rc = check_vector_densities(ctx, k * n, n, rho0, rho1, st);
        if (rc) return rc;
        // workspace: b, then two states {phi, u_x, u_y, u_z, w}
        const size_t per_state = (size_t)(4 * k + l) * m;
        rc = ensure_buffer(ctx, (void **)&ctx->ws, &ctx->ws_floats, ((size_t)k * m + 2 * per_state) * sizeof(float),
                           "workspace");
        if (rc) return rc;
        float *b = ctx->ws;
        S3Out so[2];
        S3In si[2];
        for (int q = 0; q < 2; ++q) {
            float *base = ctx->ws + (size_t)k * m + q * per_state;
            so[q] = S3Out{base, base + (size_t)k * m, base + (size_t)2 * k * m, base + (size_t)3 * k * m,
                          base + (size_t)4 * k * m};
            si[q] = S3In{so[q].phi, so[q].ux, so[q].uy, so[q].uz, so[q].w};
        }
        const int nblocks = (int)((m + T3 - 1) / T3);
        ctx->last_blocks = nblocks;
        rc = ensure_buffer(ctx, (void **)&ctx->partials, &ctx->partials_cap, sizeof(double) * (size_t)nblocks * NRED,
                           "partials");
        if (rc) return rc;
        const int max_checks = p.max_iters / p.check_every + 2;
        if (ctx->hist_cap < max_checks) {
            if (ctx->dhist) cudaFree(ctx->dhist);
            ctx->dhist = nullptr;
            ctx->hist_cap = 0;
            e = cudaMalloc(&ctx->dhist, sizeof(double) * NMET * (size_t)max_checks);
            if (e != cudaSuccess) return set_cuda_error(ctx, e, "history");
            ctx->hist_cap = max_checks;
        }
        e = cudaMemsetAsync(ctx->dstatus, 0, sizeof(DevStatus), st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "status reset");
        const int pblocks = (int)std::min<size_t>((m + 255) / 256, 4096);
        k_prepare3<<<pblocks, 256, 0, st>>>(m, k, l, rho0, rho1, b, p.warm_start, u, w, phi, so[0]);
        ctx->launches += 1;
        L3 L = pick3(k, p.u_norm, p.w_norm);
        auto check = [&](int t, int cur) {
            L.metrics<<<nblocks, T3, 0, st>>>(si[cur], si[cur ^ 1], b, g, s, ctx->partials, ctx->dstatus);
            k_finalize<<<1, 256, 0, st>>>(ctx->partials, nblocks, cfg, t, ctx->dstatus, ctx->dhist, ctx->hist_cap);
            ctx->launches += 2;
        };
        if (p.max_iters == 0) check(0, 0);
        const bool tol_mode = cfg.tol_gap > 0.0;
        const int chunk = p.check_every * ((2048 + p.check_every - 1) / p.check_every);
        int t = 0, nchunk = 0;
        bool stopped = false;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        if (tol_mode)
            for (int q = 0; q < 2; ++q) cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming);
        while (t < p.max_iters && !stopped) {
            const int end = std::min(t + chunk, p.max_iters);
            for (int tt = t + 1; tt <= end; ++tt) {
                const int cur = tt & 1;
                L.step<<<nblocks, T3, 0, st>>>(si[cur ^ 1], so[cur], b, g, s, ctx->dstatus);
                ctx->launches += 1;
                if (tt % p.check_every == 0 || tt == p.max_iters) check(tt, cur);
            }
            t = end;
            if (tol_mode) {
                const int slot = nchunk & 1;
                cudaMemcpyAsync(&ctx->hstatus[slot], ctx->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
                cudaEventRecord(ev[slot], st);
                if (nchunk >= 1) {
                    cudaEventSynchronize(ev[slot ^ 1]);
                    if (ctx->hstatus[slot ^ 1].stop) stopped = true;
                }
                ++nchunk;
            }
        }
        k_copy_out3<<<pblocks, 256, 0, st>>>(m, k, l, si[0], si[1], ctx->dstatus, u, w, phi);
        ctx->launches += 1;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ctx->hstatus[0], ctx->dstatus, sizeof(DevStatus),
                                                  cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        for (int q = 0; q < 2; ++q)
            if (ev[q]) cudaEventDestroy(ev[q]);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "3-D solve");
        int status = VOMT_OK;
        fill_result(ctx, cfg, VOMT_ENGINE_STREAM, result, &status);
        return status;
    } catch (...) {
        return fail(ctx, VOMT_ERR_BAD_ARG, "internal exception");
    }
}
