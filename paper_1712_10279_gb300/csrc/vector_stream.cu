// Streaming engine for vector OMT: one fused launch per PDHG iteration
// (Section 7.2), state double-buffered in HBM, FP64 convergence checks.
//
// One thread owns one grid point (i, j) and all k channels of it.  The phi
// update at (i, j) needs ubar = 2u' - u at (i, j), (i-1, j) and (i, j-1); the
// thread recomputes the two neighbouring shrinks from phi and u instead of
// waiting for the threads that own them, so one launch does a whole iteration
// and no grid-wide barrier is needed between the u/w and phi halves
// (Section 7.4 puts a synchronisation there).
#include <math.h>

#include "internal.h"
#include "matrix_norms.cuh"
#include "pdhg_device.cuh"
#include "stream_tma.h"

namespace vomt {
namespace {

constexpr int BX = 32, BY = 8, NT = BX * BY;

struct StateIn {
    const float *phi, *ux, *uy, *w;
};
struct StateOut {
    float *phi, *ux, *uy, *w;
};

// shrink_2 factor and soft threshold of Appendix B (pdhg_device.cuh)
using dev::shrink2_factor;
using dev::soft;
using dev::CheckAcc;
using dev::block_sum_store;

template <int K>
__device__ __forceinline__ float pick(const float (&a)[K], int idx)
{
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < K; ++c) r = (c == idx) ? a[c] : r;
    return r;
}

// shrink_u on one point, all channels, in place (Section 7.2, u-update)
// (channel weights wc enter the joint norm ||u||_2: 2 for an off-diagonal matrix entry)
template <int K, int UN>
__device__ __forceinline__ void shrink_u(float (&vx)[K], float (&vy)[K], float t, const float *wc)
{
    if (UN == VOMT_U_L12) {
#pragma unroll
        for (int c = 0; c < K; ++c) {
            float f = shrink2_factor(vx[c] * vx[c] + vy[c] * vy[c], t);
            vx[c] *= f;
            vy[c] *= f;
        }
    } else if (UN == VOMT_U_L2) {
        float s2 = 0.0f;
#pragma unroll
        for (int c = 0; c < K; ++c) s2 += wc[c] * (vx[c] * vx[c] + vy[c] * vy[c]);
        float f = shrink2_factor(s2, t);
#pragma unroll
        for (int c = 0; c < K; ++c) { vx[c] *= f; vy[c] *= f; }
    } else if (UN == VOMT_U_NUC) {
        mat::sym_shrink_nuc<K>(vx, t);
        mat::sym_shrink_nuc<K>(vy, t);
    } else {
#pragma unroll
        for (int c = 0; c < K; ++c) { vx[c] = soft(vx[c], t); vy[c] = soft(vy[c], t); }
    }
}

// shrink_w on one point (Section 7.2, w-update), l <= LK flux entries with weights we
template <int LK, int WN>
__device__ __forceinline__ void shrink_w(float (&x)[LK], int l, float t, const float *we)
{
    if (WN == VOMT_W_L1) {
#pragma unroll
        for (int e = 0; e < LK; ++e)
            if (e < l) x[e] = soft(x[e], t);
    } else if (WN == VOMT_W_NUC) {
        if constexpr (LK % 3 == 0) {
#pragma unroll
            for (int g = 0; g < LK; g += 3) {
                if (g < l) {
                    const float f = shrink2_factor(x[g] * x[g] + x[g + 1] * x[g + 1] + x[g + 2] * x[g + 2], t);
                    x[g] *= f;
                    x[g + 1] *= f;
                    x[g + 2] *= f;
                }
            }
        }
    } else {
        float s2 = 0.0f;
#pragma unroll
        for (int e = 0; e < LK; ++e)
            if (e < l) s2 += we[e] * x[e] * x[e];
        float f = shrink2_factor(s2, t);
#pragma unroll
        for (int e = 0; e < LK; ++e) x[e] *= f;
    }
}

template <int K>
struct LKOf {
    static constexpr int v = K * (K - 1) / 2 > 0 ? K * (K - 1) / 2 : 1;
};

// ----------------------------------------------------------------- iteration
template <int K, int UN, int WN>
__global__ void __launch_bounds__(NT) k_step(StateIn in, StateOut out, const float *__restrict__ b,
                                              OpDev g, StepDev s, const DevStatus *__restrict__ st)
{
    cudaGridDependencySynchronize();      // after the previous kernel (no-op for a normal launch)
    if (st->stop) return;
    constexpr int LK = LKOf<K>::v;
    const int n = s.n;
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= n || j >= n) return;
    const size_t nn = (size_t)n * n;
    const size_t p = (size_t)j * n + i;
    const bool hR = i < n - 1, hU = j < n - 1, hL = i > 0, hD = j > 0;
    const float mu = s.mu, ih = s.ih;
    // regularised prox (eps > 0): shrink su * v by su * mu, su = 1 / (1 + 2 mu eps)
    const float su = s.reg ? s.su : 1.0f, tu = s.reg ? mu * s.su : mu;

    float pc[K], pr[K], pu[K], pl[K], plu[K], pd[K], prd[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const float *P = in.phi + c * nn + p;
        pc[c] = __ldg(P);
        pr[c] = hR ? __ldg(P + 1) : 0.0f;
        pu[c] = hU ? __ldg(P + n) : 0.0f;
        pl[c] = hL ? __ldg(P - 1) : 0.0f;
        plu[c] = (hL && hU) ? __ldg(P - 1 + n) : 0.0f;
        pd[c] = hD ? __ldg(P - n) : 0.0f;
        prd[c] = (hR && hD) ? __ldg(P + 1 - n) : 0.0f;
    }
    // u' at (i, j)
    float ux0[K], uy0[K], vx[K], vy[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        ux0[c] = __ldg(in.ux + c * nn + p);
        uy0[c] = __ldg(in.uy + c * nn + p);
        vx[c] = ux0[c] + (hR ? mu * (ih * (pr[c] - pc[c])) : 0.0f);
        vy[c] = uy0[c] + (hU ? mu * (ih * (pu[c] - pc[c])) : 0.0f);
        if (s.reg) { vx[c] *= su; vy[c] *= su; }
    }
    shrink_u<K, UN>(vx, vy, tu, g.wc);
    // u' at (i-1, j): only its x component enters div at (i, j)
    float lx[K], ly[K], lx0[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        lx0[c] = hL ? __ldg(in.ux + c * nn + p - 1) : 0.0f;
        float ly0 = hL ? __ldg(in.uy + c * nn + p - 1) : 0.0f;
        lx[c] = lx0[c] + (hL ? mu * (ih * (pc[c] - pl[c])) : 0.0f);
        ly[c] = ly0 + ((hL && hU) ? mu * (ih * (plu[c] - pl[c])) : 0.0f);
        if (s.reg) { lx[c] *= su; ly[c] *= su; }
    }
    shrink_u<K, UN>(lx, ly, tu, g.wc);
    // u' at (i, j-1): only its y component enters div at (i, j)
    float dx[K], dy[K], dy0[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        float dx0 = hD ? __ldg(in.ux + c * nn + p - n) : 0.0f;
        dy0[c] = hD ? __ldg(in.uy + c * nn + p - n) : 0.0f;
        dx[c] = dx0 + ((hR && hD) ? mu * (ih * (prd[c] - pd[c])) : 0.0f);
        dy[c] = dy0[c] + (hD ? mu * (ih * (pc[c] - pd[c])) : 0.0f);
        if (s.reg) { dx[c] *= su; dy[c] *= su; }
    }
    shrink_u<K, UN>(dx, dy, tu, g.wc);
    // w' at (i, j)
    float w0[LK], wx[LK];
#pragma unroll
    for (int e = 0; e < LK; ++e) {
        if (e < g.l) {
            w0[e] = __ldg(in.w + e * nn + p);
            float ge = 0.0f;
#pragma unroll
            for (int c = 0; c < K; ++c) ge += g.G[e][c] * pc[c];
            wx[e] = w0[e] + s.nu * ge;
            if (s.reg) wx[e] *= s.sw;
        } else {
            w0[e] = 0.0f;
            wx[e] = 0.0f;
        }
    }
    shrink_w<LK, WN>(wx, g.l, s.reg ? s.alpha * s.nu * s.sw : s.alpha * s.nu, g.we);
    // phi' = phi + tau (div_x ubar + div_G wbar + rho1 - rho0)
    float r[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        float bxc = 2.0f * vx[c] - ux0[c];
        float byc = 2.0f * vy[c] - uy0[c];
        float bxl = hL ? 2.0f * lx[c] - lx0[c] : 0.0f;
        float byd = hD ? 2.0f * dy[c] - dy0[c] : 0.0f;
        r[c] = ih * ((bxc - bxl) + (byc - byd)) + __ldg(b + c * nn + p);
    }
#pragma unroll
    for (int e = 0; e < LK; ++e) {
        const float v = 2.0f * wx[e] - w0[e];     // zero for e >= l
#pragma unroll
        for (int c = 0; c < K; ++c) r[c] -= g.Dv[c][e] * v;
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
        out.phi[c * nn + p] = pc[c] + s.tau * r[c];
        out.ux[c * nn + p] = vx[c];
        out.uy[c * nn + p] = vy[c];
    }
#pragma unroll
    for (int e = 0; e < LK; ++e)
        if (e < g.l) out.w[e * nn + p] = wx[e];
}

// ----------------------------------------------------------------- metrics
template <int K, int UN, int WN>
__global__ void __launch_bounds__(NT) k_metrics(StateIn cur, StateIn prv, const float *__restrict__ b,
                                                 OpDev g, StepDev s, double *__restrict__ partials,
                                                 const DevStatus *__restrict__ st)
{
    cudaGridDependencySynchronize();
    if (st->stop) return;
    constexpr int LK = LKOf<K>::v;
    const int n = s.n;
    // the grid's BX x BY tiles, visited by the blocks in turn (at most kMetricBlocks
    // blocks, so that k_finalize sums few rows)
    const int gxb = (n + BX - 1) / BX, ntile = gxb * ((n + BY - 1) / BY);
    CheckAcc acc;
    acc.zero();
    for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int i = (tile % gxb) * BX + threadIdx.x;
    const int j = (tile / gxb) * BY + threadIdx.y;
    if (i < n && j < n) {
        // Per-point terms in FP32 (each rounding is relative 2^-24), converted once
        // per point and accumulated in FP64 (FP64 arithmetic is scarce on this
        // GPU).  The spatial part of the constraint residual, which cancels
        // several digits, is formed in FP64.
        const size_t nn = (size_t)n * n, p = (size_t)j * n + i;
        const bool hR = i < n - 1, hU = j < n - 1, hL = i > 0, hD = j > 0;
        const float ih = s.ih, alpha = s.alpha;
        const double dih = (double)(n - 1);
        float ph[K], dph[K], ddiv[K], gwb[K];
        double rdiv[K];
        float nu_pt = 0.0f, dn_u = 0.0f, fdu = 0.0f, fdp = 0.0f, fd = 0.0f, fbb = 0.0f, fdw = 0.0f, fx = 0.0f;
        float q2 = 0.0f, dist = 0.0f;     // regularisation: squared norms, squared distances to the dual balls
        float gxs[K], gys[K], uxs[K], uys[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const size_t q = c * nn + p;
            const float uxc = cur.ux[q], uyc = cur.uy[q], bc = b[q], wgt = g.wc[c];
            ph[c] = cur.phi[q];
            dph[c] = ph[c] - prv.phi[q];
            const float xl = hL ? cur.ux[q - 1] : 0.0f, yd = hD ? cur.uy[q - n] : 0.0f;
            rdiv[c] = dih * (((double)uxc - (double)xl) + ((double)uyc - (double)yd));
            gwb[c] = bc;
            const float dux = uxc - prv.ux[q], duy = uyc - prv.uy[q];
            const float dxl = hL ? cur.ux[q - 1] - prv.ux[q - 1] : 0.0f;
            const float dyd = hD ? cur.uy[q - n] - prv.uy[q - n] : 0.0f;
            ddiv[c] = ih * ((dux - dxl) + (duy - dyd));
            fdu += wgt * (dux * dux + duy * duy);
            fdp += wgt * dph[c] * dph[c];
            fd += wgt * ph[c] * bc;
            fbb += wgt * bc * bc;
            q2 += wgt * (uxc * uxc + uyc * uyc);
            const float gx = hR ? ih * (cur.phi[q + 1] - ph[c]) : 0.0f;
            const float gy = hU ? ih * (cur.phi[q + n] - ph[c]) : 0.0f;
            gxs[c] = gx;
            gys[c] = gy;
            uxs[c] = uxc;
            uys[c] = uyc;
            if (UN == VOMT_U_NUC) {
                // after the loop
            } else if (UN == VOMT_U_L12) {
                nu_pt += sqrtf(uxc * uxc + uyc * uyc);
                const float gn = sqrtf(gx * gx + gy * gy);
                dn_u = fmaxf(dn_u, gn);
                const float o = fmaxf(gn - 1.0f, 0.0f);
                dist += o * o;
            } else if (UN == VOMT_U_L2) {
                nu_pt += wgt * (uxc * uxc + uyc * uyc);
                dn_u += wgt * (gx * gx + gy * gy);
            } else {
                nu_pt += wgt * (fabsf(uxc) + fabsf(uyc));
                dn_u = fmaxf(dn_u, fmaxf(fabsf(gx), fabsf(gy)));
                const float ox = fmaxf(fabsf(gx) - 1.0f, 0.0f), oy = fmaxf(fabsf(gy) - 1.0f, 0.0f);
                dist += wgt * (ox * ox + oy * oy);
            }
        }
        if (UN == VOMT_U_L2) {
            nu_pt = sqrtf(nu_pt);
            dn_u = sqrtf(dn_u);
            const float o = fmaxf(dn_u - 1.0f, 0.0f);
            dist += o * o;
        }
        if constexpr (UN == VOMT_U_NUC) {        // sum of the nuclear norms, larger spectral norm
            float n1, s1, n2, s2;
            mat::sym_nuc_spec<K>(uxs, n1, s1);
            mat::sym_nuc_spec<K>(uys, n2, s2);
            nu_pt = n1 + n2;
            mat::sym_nuc_spec<K>(gxs, n1, s1);
            mat::sym_nuc_spec<K>(gys, n2, s2);
            dn_u = fmaxf(s1, s2);
        }
        float nw_pt = 0.0f, dn_w = 0.0f, wg2 = 0.0f, gg2 = 0.0f;
#pragma unroll
        for (int e = 0; e < LK; ++e) {
            if (e < g.l) {
                const size_t q = e * nn + p;
                const float we = cur.w[q], dwe = we - prv.w[q], wgt = g.we[e];
                fdw += wgt * dwe * dwe;
                q2 += wgt * we * we;
                float ge = 0.0f;
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    ge += g.G[e][c] * ph[c];
                    gwb[c] -= g.Dv[c][e] * we;      // div y = -Dv y
                    ddiv[c] -= g.Dv[c][e] * dwe;
                }
                if (WN == VOMT_W_L1) {
                    nw_pt += wgt * fabsf(we);
                    dn_w = fmaxf(dn_w, fabsf(ge));
                    const float o = fmaxf(fabsf(ge) - alpha, 0.0f);
                    dist += wgt * o * o;
                } else if (WN == VOMT_W_NUC) {
                    // 3 x 3 skew components (a, b, c): ||W_s||_nuc = 2 |(a,b,c)|, spectral |(a,b,c)|
                    wg2 += we * we;
                    gg2 += ge * ge;
                    if (e % 3 == 2) {
                        nw_pt += 2.0f * sqrtf(wg2);
                        dn_w = fmaxf(dn_w, sqrtf(gg2));
                        wg2 = gg2 = 0.0f;
                    }
                } else {
                    nw_pt += wgt * we * we;
                    dn_w += wgt * ge * ge;
                }
            }
        }
        if (WN == VOMT_W_L2) {
            nw_pt = sqrtf(nw_pt);
            dn_w = sqrtf(dn_w);
            const float o = fmaxf(dn_w - alpha, 0.0f);
            if (g.l > 0) dist += o * o;
        }
        double rr = 0.0;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const double rc = rdiv[c] + (double)gwb[c];
            rr += (double)g.wc[c] * rc * rc;
            fx += g.wc[c] * dph[c] * ddiv[c];
        }
        acc.add_d(RED_RR, rr);
        acc.add(RED_P, nu_pt + alpha * nw_pt);
        if (s.reg) {
            acc.add(RED_P, s.eps * q2);
            acc.add(RED_DIST, dist);
        }
        acc.add(RED_D, fd);
        acc.add(RED_BB, fbb);
        acc.add(RED_DU, fdu);
        acc.add(RED_DW, fdw);
        acc.add(RED_DP, fdp);
        acc.add(RED_X, fx);
        float di = fmaxf(dn_u - 1.0f, 0.0f);
        if (g.l > 0) di = fmaxf(di, dn_w - alpha);
        acc.max(RED_MAX, di);
    }
    }
    block_sum_store<NT>(acc, partials + (size_t)blockIdx.x * NRED);
}

// ----------------------------------------------------------------- setup / copy
__global__ void k_prepare(int n, int k, int l, const float *__restrict__ rho0, const float *__restrict__ rho1,
                          float *__restrict__ b, int warm, const float *__restrict__ u_in,
                          const float *__restrict__ w_in, const float *__restrict__ phi_in, StateOut s0)
{
    const size_t nn = (size_t)n * n;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % n), j = (int)(q / n);
        for (int c = 0; c < k; ++c) {
            b[c * nn + q] = rho1[c * nn + q] - rho0[c * nn + q];
            s0.phi[c * nn + q] = warm ? phi_in[c * nn + q] : 0.0f;
            s0.ux[c * nn + q] = (warm && i < n - 1) ? u_in[c * nn + q] : 0.0f;
            s0.uy[c * nn + q] = (warm && j < n - 1) ? u_in[(k + c) * nn + q] : 0.0f;
        }
        for (int e = 0; e < l; ++e) s0.w[e * nn + q] = warm ? w_in[e * nn + q] : 0.0f;
    }
}

__global__ void k_copy_out(int n, int k, int l, StateIn s0, StateIn s1, const DevStatus *__restrict__ st,
                           float *__restrict__ u, float *__restrict__ w, float *__restrict__ phi)
{
    const StateIn s = (st->iter & 1) ? s1 : s0;
    const size_t nn = (size_t)n * n;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < k; ++c) {
            phi[c * nn + q] = s.phi[c * nn + q];
            u[c * nn + q] = s.ux[c * nn + q];
            u[(k + c) * nn + q] = s.uy[c * nn + q];
        }
        for (int e = 0; e < l; ++e) w[e * nn + q] = s.w[e * nn + q];
    }
}

// density validation: per block sum0, sum1, min0, min1, nonfinite count
__global__ void k_validate(size_t count, const float *__restrict__ r0, const float *__restrict__ r1,
                           double *__restrict__ out)
{
    double s0 = 0.0, s1 = 0.0, m0 = 1e300, m1 = 1e300, bad = 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count; q += (size_t)gridDim.x * blockDim.x) {
        float a = r0[q], c = r1[q];
        if (!isfinite(a) || !isfinite(c)) { bad += 1.0; continue; }
        s0 += a; s1 += c;
        m0 = fmin(m0, (double)a);
        m1 = fmin(m1, (double)c);
    }
    __shared__ double sh[5][256];
    sh[0][threadIdx.x] = s0; sh[1][threadIdx.x] = s1; sh[2][threadIdx.x] = m0; sh[3][threadIdx.x] = m1;
    sh[4][threadIdx.x] = bad;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + off];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + off];
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + off]);
            sh[3][threadIdx.x] = fmin(sh[3][threadIdx.x], sh[3][threadIdx.x + off]);
            sh[4][threadIdx.x] += sh[4][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x < 5) out[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

// ----------------------------------------------------------------- dispatch
struct Launchers {
    void (*step)(StateIn, StateOut, const float *, OpDev, StepDev, const DevStatus *);
    void (*metrics)(StateIn, StateIn, const float *, OpDev, StepDev, double *, const DevStatus *);
};

template <int K, int UN, int WN>
Launchers make_launchers()
{
    return Launchers{k_step<K, UN, WN>, k_metrics<K, UN, WN>};
}

template <int K>
Launchers pick_norms(int un, int wn)
{
    if constexpr (K == 3 || K == 6) {          // nuclear norms: compact 2 x 2 and 3 x 3 matrices
        if (un == VOMT_U_NUC)
            return wn == VOMT_W_L1 ? make_launchers<K, 3, 0>()
                                   : (wn == VOMT_W_L2 ? make_launchers<K, 3, 1>() : make_launchers<K, 3, 2>());
        if (wn == VOMT_W_NUC) return un == VOMT_U_L2 ? make_launchers<K, 1, 2>() : make_launchers<K, 2, 2>();
    }
    if (un == VOMT_U_L12) return wn == VOMT_W_L1 ? make_launchers<K, 0, 0>() : make_launchers<K, 0, 1>();
    if (un == VOMT_U_L2) return wn == VOMT_W_L1 ? make_launchers<K, 1, 0>() : make_launchers<K, 1, 1>();
    return wn == VOMT_W_L1 ? make_launchers<K, 2, 0>() : make_launchers<K, 2, 1>();
}

Launchers pick(int k, int un, int wn)
{
    switch (k) {
        case 1: return pick_norms<1>(un, wn);
        case 2: return pick_norms<2>(un, wn);
        case 3: return pick_norms<3>(un, wn);
        case 4: return pick_norms<4>(un, wn);
        case 5: return pick_norms<5>(un, wn);
        case 6: return pick_norms<6>(un, wn);
        case 7: return pick_norms<7>(un, wn);
        default: return pick_norms<8>(un, wn);
    }
}

}  // namespace

// Fixed-order sum of the per-block partials, the stopping decision and the
// history row.  One block of 256 threads.
__global__ void k_finalize(const double *__restrict__ partials, int nblocks, SolveCfg cfg, int t,
                           DevStatus *st, double *hist, int hist_cap)
{
    cudaGridDependencySynchronize();
    if (st->stop) return;
    __shared__ double S[NRED];
    // warp q sums slot q: lane j takes rows j, j + 32, ..., then a butterfly over
    // the lanes (a fixed order, so the same sum on every run)
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    if (q < NRED) {
        double a = 0.0;
        for (int bk = lane; bk < nblocks; bk += 32) {
            const double x = partials[(size_t)bk * NRED + q];
            a = (q == RED_MAX) ? fmax(a, x) : a + x;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_xor_sync(0xffffffffu, a, off);
            a = (q == RED_MAX) ? fmax(a, o) : a + o;
        }
        if (lane == 0) S[q] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (t < 0) t = st->iter - t;       // in a replayed graph: the last check's iteration plus -t
        double P = S[RED_P], D = S[RED_D] - (cfg.eps > 0.0 ? S[RED_DIST] / (4.0 * cfg.eps) : 0.0);
        double m[NMET];
        m[0] = P;
        m[1] = D;
        m[2] = fabs(P - D) / fmax(fabs(P), 1e-300);
        m[3] = sqrt(S[RED_RR]) / (S[RED_BB] > 0.0 ? sqrt(S[RED_BB]) : 1.0);
        m[4] = S[RED_DU] / cfg.mu + (cfg.has_w ? S[RED_DW] / cfg.nu : 0.0) + S[RED_DP] / cfg.tau - 2.0 * S[RED_X];
        m[5] = S[RED_MAX];
        m[6] = (double)t;
        bool finite = true;
        for (int q = 0; q < 6; ++q) finite = finite && isfinite(m[q]);
        bool conv = cfg.tol_gap > 0.0 && m[2] <= cfg.tol_gap && m[3] <= cfg.tol_res;
        m[7] = conv ? 1.0 : 0.0;
        for (int q = 0; q < NMET; ++q) st->met[q] = m[q];
        if (hist && st->checks < hist_cap)
            for (int q = 0; q < NMET; ++q) hist[(size_t)st->checks * NMET + q] = m[q];
        st->checks += 1;
        st->iter = t;
        if (!finite) { st->error = VOMT_ERR_NONFINITE; st->stop = 1; }
        if (conv) st->stop = 1;
    }
}

// One fused iteration (Section 7.2) from the state at `in` to the state at
// `out`; each state is contiguous planes phi [k], u_x [k], u_y [k], w [l].
void launch_step(const OpDev &g, const StepDev &s, int un, int wn, const float *in, float *out, const float *b,
                 const DevStatus *st, cudaStream_t stream)
{
    const size_t nn = (size_t)s.n * s.n;
    const int k = g.k;
    const StateIn si{in, in + (size_t)k * nn, in + (size_t)2 * k * nn, in + (size_t)3 * k * nn};
    const StateOut so{out, out + (size_t)k * nn, out + (size_t)2 * k * nn, out + (size_t)3 * k * nn};
    const dim3 blk(BX, BY), grd((s.n + BX - 1) / BX, (s.n + BY - 1) / BY);
    pick(k, un, wn).step<<<grd, blk, 0, stream>>>(si, so, b, g, s, st);
}

int validate_densities(vomt_ctx *ctx, int planes, int n, const float *rho0, const float *rho1,
                       cudaStream_t st, double *sums)
{
    const size_t count = (size_t)planes * n * n;
    const int blocks = (int)((count + 255) / 256 < 1024 ? (count + 255) / 256 : 1024);
    int rc = ensure_buffer(ctx, (void **)&ctx->partials, &ctx->partials_cap,
                           sizeof(double) * (size_t)blocks * 5, "partials");
    if (rc) return rc;
    k_validate<<<blocks, 256, 0, st>>>(count, rho0, rho1, ctx->partials);
    ctx->launches += 1;
    std::vector<double> h((size_t)blocks * 5);
    cudaError_t e = cudaMemcpyAsync(h.data(), ctx->partials, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "validate");
    sums[0] = sums[1] = sums[4] = 0.0;
    sums[2] = sums[3] = 1e300;
    for (int q = 0; q < blocks; ++q) {
        sums[0] += h[q * 5 + 0];
        sums[1] += h[q * 5 + 1];
        sums[2] = fmin(sums[2], h[q * 5 + 2]);
        sums[3] = fmin(sums[3], h[q * 5 + 3]);
        sums[4] += h[q * 5 + 4];
    }
    return VOMT_OK;
}

int stream_solve(vomt_ctx *ctx, const OpDev &g, const StepDev &s, const SolveCfg &cfg,
                 const vomt_params &p, const float *rho0, const float *rho1,
                 float *u, float *w, float *phi, cudaStream_t st)
{
    ctx->hist_raw = false;           // k_finalize writes finished rows
    const int n = s.n, k = g.k, l = g.l;
    const size_t nn = (size_t)n * n;
    // workspace: b, then two states {phi, ux, uy, w}
    const size_t per_state = (size_t)(3 * k + l) * nn;
    const size_t need = (size_t)k * nn + 2 * per_state;
    int rc = ensure_buffer(ctx, (void **)&ctx->ws, &ctx->ws_floats, need * sizeof(float), "workspace");
    if (rc) return rc;
    float *b = ctx->ws;
    StateOut so[2];
    StateIn si[2];
    for (int q = 0; q < 2; ++q) {
        float *base = ctx->ws + (size_t)k * nn + q * per_state;
        so[q] = StateOut{base, base + (size_t)k * nn, base + (size_t)2 * k * nn, base + (size_t)3 * k * nn};
        si[q] = StateIn{so[q].phi, so[q].ux, so[q].uy, so[q].w};
    }
    const dim3 blk(BX, BY), grd((n + BX - 1) / BX, (n + BY - 1) / BY);
    const int nblocks = (int)(grd.x * grd.y);
    const int mblocks = nblocks < kMetricBlocks ? nblocks : kMetricBlocks;     // blocks of a check
    ctx->last_blocks = nblocks;
    rc = ensure_buffer(ctx, (void **)&ctx->partials, &ctx->partials_cap, sizeof(double) * (size_t)nblocks * NRED,
                       "partials");
    if (rc) return rc;
    const int max_checks = p.max_iters / p.check_every + 2;
    if (ctx->hist_cap < max_checks) {
        if (ctx->dhist) cudaFree(ctx->dhist);
        ctx->dhist = nullptr;
        ctx->hist_cap = 0;
        cudaError_t e = cudaMalloc(&ctx->dhist, sizeof(double) * NMET * (size_t)max_checks);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "history");
        ctx->hist_cap = max_checks;
    }
    cudaError_t e = cudaMemsetAsync(ctx->dstatus, 0, sizeof(DevStatus), st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "status reset");
    const int pblocks = (int)((nn + 255) / 256 < 2048 ? (nn + 255) / 256 : 2048);
    k_prepare<<<pblocks, 256, 0, st>>>(n, k, l, rho0, rho1, b, p.warm_start, u, w, phi, so[0]);
    ctx->launches += 1;

    Launchers L = pick(k, p.u_norm, p.w_norm);
    // TMA tiles for the iteration where they apply (n a multiple of 4, k <= 4)
    TmaPlan *tp = tma_step_supported(n, k, l, p.u_norm, p.w_norm)
                      ? tma_plan_create(n, k, l, p.u_norm, p.w_norm, so[0].phi, so[1].phi, b)
                      : nullptr;
    if (tp) {
        ctx->last_blocks = ((n + 63) / 64) * ((n + 15) / 16);    // the step's 64 x 16 tiles
        ctx->last_variant = 1;
    }
    auto check = [&](int t, int cur) {
        launch_pdl(L.metrics, dim3(mblocks), blk, 0, st, si[cur], si[cur ^ 1], (const float *)b, g, s, ctx->partials,
                   (const DevStatus *)ctx->dstatus);
        launch_pdl(k_finalize, dim3(1), dim3(kFinThreads), 0, st, (const double *)ctx->partials, mblocks, cfg, t,
                   ctx->dstatus, ctx->dhist, ctx->hist_cap);
        ctx->launches += 2;
    };
    if (p.max_iters == 0) {
        L.metrics<<<mblocks, blk, 0, st>>>(si[0], si[0], b, g, s, ctx->partials, ctx->dstatus);
        k_finalize<<<1, kFinThreads, 0, st>>>(ctx->partials, mblocks, cfg, 0, ctx->dstatus, ctx->dhist, ctx->hist_cap);
        ctx->launches += 2;
    }
    const bool tol_mode = cfg.tol_gap > 0.0;
    int chunk = p.check_every * ((2048 + p.check_every - 1) / p.check_every);
    // Long solves replay a captured CUDA graph of G iterations (G = check_every, made
    // even so that the ping-pong parity repeats, and its checks), cutting the launch
    // gaps between the short kernels of mid-size grids.  Captured on the context's
    // own stream, launched on the caller's.
    const int G = (p.check_every % 2 == 0) ? p.check_every : 2 * p.check_every;
    cudaGraphExec_t gexec = nullptr;
    if (G <= 512 && p.max_iters >= 4 * G) {
        if (!ctx->cap_stream) cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
        cudaGraph_t graph = nullptr;
        if (ctx->cap_stream && cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            for (int tt = 1; tt <= G; ++tt) {
                const int cur = tt & 1;
                if (tp)
                    tma_launch_step(tp, cur ^ 1, so[cur].phi, g, s, ctx->dstatus, ctx->cap_stream, true);
                else
                    launch_pdl(L.step, grd, blk, 0, ctx->cap_stream, si[cur ^ 1], so[cur], (const float *)b, g, s,
                               (const DevStatus *)ctx->dstatus);
                if (tt % p.check_every == 0) {
                    launch_pdl(L.metrics, dim3(mblocks), blk, 0, ctx->cap_stream, si[cur], si[cur ^ 1], (const float *)b, g,
                               s, ctx->partials, (const DevStatus *)ctx->dstatus);
                    launch_pdl(k_finalize, dim3(1), dim3(kFinThreads), 0, ctx->cap_stream, (const double *)ctx->partials,
                               mblocks, cfg, -p.check_every, ctx->dstatus, ctx->dhist, ctx->hist_cap);
                }
            }
            if (cudaStreamEndCapture(ctx->cap_stream, &graph) != cudaSuccess ||
                cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess)
                gexec = nullptr;
            if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();          // a failed capture leaves the plain launches below
    }
    const int per_graph_launches = G + 2 * (G / p.check_every);
    // graph replays need an even starting iteration: chunks are whole multiples of G
    if (gexec) chunk = G * ((2048 + G - 1) / G);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (tol_mode) {
        for (int q = 0; q < 2; ++q) cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming);
    }
    int t = 0, nchunk = 0;
    bool stopped = false;
    while (t < p.max_iters && !stopped) {
        const int end = t + chunk < p.max_iters ? t + chunk : p.max_iters;
        if (gexec) {
            while (t + G <= end) {
                cudaGraphLaunch(gexec, st);
                ctx->launches += per_graph_launches;
                t += G;
            }
        }
        for (int tt = t + 1; tt <= end; ++tt) {
            const int cur = tt & 1;
            if (tp)
                tma_launch_step(tp, cur ^ 1, so[cur].phi, g, s, ctx->dstatus, st, true);
            else
                launch_pdl(L.step, grd, blk, 0, st, si[cur ^ 1], so[cur], (const float *)b, g, s,
                           (const DevStatus *)ctx->dstatus);
            ctx->launches += 1;
            if (tt % p.check_every == 0 || tt == p.max_iters) check(tt, cur);
        }
        t = end;
        if (tol_mode) {
            const int slot = nchunk & 1;
            cudaMemcpyAsync(&ctx->hstatus[slot], ctx->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
            cudaEventRecord(ev[slot], st);
            if (nchunk >= 1) {
                // the previous chunk's flag: the GPU keeps running the chunk just queued
                cudaEventSynchronize(ev[slot ^ 1]);
                if (ctx->hstatus[slot ^ 1].stop) stopped = true;
            }
            ++nchunk;
        }
    }
    k_copy_out<<<pblocks, 256, 0, st>>>(n, k, l, si[0], si[1], ctx->dstatus, u, w, phi);
    ctx->launches += 1;
    if (gexec) {
        cudaStreamSynchronize(st);
        cudaGraphExecDestroy(gexec);
    }
    tma_plan_destroy(tp);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        for (int q = 0; q < 2; ++q) if (ev[q]) cudaEventDestroy(ev[q]);
        return set_cuda_error(ctx, e, "launch");
    }
    e = cudaMemcpyAsync(&ctx->hstatus[0], ctx->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int q = 0; q < 2; ++q) if (ev[q]) cudaEventDestroy(ev[q]);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "solve");
    return VOMT_OK;
}

}  // namespace vomt

// ---------------------------------------------------------------------------
// Allocation-free variant of the streaming solve (vomt_solve_noalloc).
//
// Some callers cannot allocate device memory: applications whose device memory
// is owned by one custom pool or allocator (a cudaMalloc behind its back would
// fragment or overcommit it), and plug-ins or long-running services that must
// not grow the process's footprint, or risk an out-of-memory failure, after
// start-up.  For them this entry point takes its scratch (double-buffered
// iterates, b = rho1 - rho0, FP64 partial sums, the status block) from one
// fixed array of VOMT_NOALLOC_SCRATCH_BYTES bytes that is part of the library
// image: every GPU that loads the library holds it until the process exits,
// and no call ever allocates or frees memory.  Every call shares the array, so
// calls that overlap on the GPU (other streams, other host threads) race with
// each other.  The call reads its stopping flag and results back while it
// runs, so it refuses a stream that is being captured into a CUDA graph.
// ---------------------------------------------------------------------------
#include <mutex>

static __device__ __align__(256) unsigned char g_noalloc_scratch[VOMT_NOALLOC_SCRATCH_BYTES];

namespace vomt {
namespace {

constexpr int kNoAllocMaxDevices = 256;
std::mutex g_noalloc_mu;
void *g_noalloc_base[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per
// device (the first call on a device does this set-up).
int noalloc_base(void **out, const char **why)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) { *why = "cudaGetDevice failed"; return VOMT_ERR_CUDA; }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) { *why = "cudaGetSymbolAddress failed for the scratch array"; return VOMT_ERR_CUDA; }
        g_noalloc_base[dev] = p;
    }
    *out = g_noalloc_base[dev];
    return VOMT_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace vomt

namespace vomt {
namespace {

// Messages of failed calls outlive the call: one per host thread.
thread_local std::string t_noalloc_msg;

int noalloc_solve(int n, const float *rho0, const float *rho1, const vomt_graph *graph, double alpha,
                  const vomt_params *pin, float *u, float *w, float *phi, vomt_result *result, cudaStream_t st,
                  const char **why);

}  // namespace
}  // namespace vomt

extern "C" int vomt_solve_noalloc(int n, const float *rho0, const float *rho1, const vomt_graph *graph, double alpha,
                                  const vomt_params *pin, float *u, float *w, float *phi, vomt_result *result,
                                  void *stream, const char **error)
{
    const char *dummy = nullptr;
    const char **why = error ? error : &dummy;
    *why = "";
    try {
        return vomt::noalloc_solve(n, rho0, rho1, graph, alpha, pin, u, w, phi, result, (cudaStream_t)stream, why);
    } catch (...) {
        *why = "internal exception";
        return VOMT_ERR_BAD_ARG;
    }
}

namespace vomt {
namespace {

int noalloc_solve(int n, const float *rho0, const float *rho1, const vomt_graph *graph, double alpha,
                  const vomt_params *pin, float *u, float *w, float *phi, vomt_result *result, cudaStream_t st,
                  const char **why)
{
    // The call reads results back and synchronises `st` while it runs, which a stream
    // under CUDA graph capture does not allow: refuse before any GPU work, so that the
    // caller's capture stays intact.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) { *why = "cudaStreamIsCapturing failed"; return VOMT_ERR_CUDA; }
    if (cap != cudaStreamCaptureStatusNone) {
        *why = "the stream is being captured into a CUDA graph; this call synchronises its stream";
        return VOMT_ERR_BAD_ARG;
    }
    VectorSetup S;
    int rc = setup_vector(n, graph, alpha, pin, &S, &t_noalloc_msg);
    if (rc) { *why = t_noalloc_msg.c_str(); return rc; }
    const OpDev &g = S.g;
    const StepDev &s = S.s;
    const SolveCfg &cfg = S.cfg;
    const vomt_params &p = S.p;
    const double mu = cfg.mu, nu = cfg.nu, tau = cfg.tau;
    if (!rho0 || !rho1 || !u || !phi || (g.l > 0 && !w)) { *why = "null array"; return VOMT_ERR_BAD_ARG; }

    // carve the scratch array
    const int k = g.k, l = g.l;
    const size_t nn = (size_t)n * n;
    const dim3 blk(BX, BY), grd((n + BX - 1) / BX, (n + BY - 1) / BY);
    const int nblocks = (int)(grd.x * grd.y);
    const int mblocks = nblocks < kMetricBlocks ? nblocks : kMetricBlocks;     // blocks of a check
    const size_t count = (size_t)k * nn;
    const int vblocks = (int)((count + 255) / 256 < 256 ? (count + 255) / 256 : 256);
    const size_t off_status = 0;
    const size_t off_vpart = align256(off_status + sizeof(DevStatus));
    const size_t off_part = align256(off_vpart + sizeof(double) * 5 * (size_t)vblocks);
    const size_t off_b = align256(off_part + sizeof(double) * NRED * (size_t)nblocks);
    const size_t per_state = (size_t)(3 * k + l) * nn;
    const size_t off_s0 = align256(off_b + sizeof(float) * (size_t)k * nn);
    const size_t off_s1 = align256(off_s0 + sizeof(float) * per_state);
    const size_t total = align256(off_s1 + sizeof(float) * per_state);
    if (total > (size_t)VOMT_NOALLOC_SCRATCH_BYTES) {
        *why = "problem needs more scratch than VOMT_NOALLOC_SCRATCH_BYTES";
        return VOMT_ERR_TOO_LARGE;
    }
    void *basev = nullptr;
    rc = noalloc_base(&basev, why);
    if (rc) return rc;
    unsigned char *base = (unsigned char *)basev;
    DevStatus *dstatus = (DevStatus *)(base + off_status);
    double *vpart = (double *)(base + off_vpart);
    double *partials = (double *)(base + off_part);
    float *b = (float *)(base + off_b);
    StateOut so[2];
    StateIn si[2];
    for (int q = 0; q < 2; ++q) {
        float *sb = (float *)(base + (q ? off_s1 : off_s0));
        so[q] = StateOut{sb, sb + (size_t)k * nn, sb + (size_t)2 * k * nn, sb + (size_t)3 * k * nn};
        si[q] = StateIn{so[q].phi, so[q].ux, so[q].uy, so[q].w};
    }
    int launches = 0;

    // density checks (the scratch keeps the previous call's contents: every slot read below is written first)
    k_validate<<<vblocks, 256, 0, st>>>(count, rho0, rho1, vpart);
    ++launches;
    double hv[5 * 256];
    e = cudaMemcpyAsync(hv, vpart, sizeof(double) * 5 * (size_t)vblocks, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { *why = cudaGetErrorString(e); return VOMT_ERR_CUDA; }
    double s0 = 0.0, s1 = 0.0, m0 = 1e300, m1 = 1e300, bad = 0.0;
    for (int q = 0; q < vblocks; ++q) {
        s0 += hv[q * 5 + 0];
        s1 += hv[q * 5 + 1];
        m0 = fmin(m0, hv[q * 5 + 2]);
        m1 = fmin(m1, hv[q * 5 + 3]);
        bad += hv[q * 5 + 4];
    }
    if (bad > 0.0) { *why = "density has NaN or Inf entries"; return VOMT_ERR_NONFINITE; }
    if (m0 < 0.0 || m1 < 0.0) { *why = "density has negative entries"; return VOMT_ERR_NEGATIVE_DENSITY; }
    if (fabs(s0 - s1) > kMassRelTol * fmax(fabs(s0), fabs(s1))) { *why = "rho0 and rho1 have different total mass"; return VOMT_ERR_MASS_MISMATCH; }

    // the status block must start at zero; iterates and b are written by k_prepare
    e = cudaMemsetAsync(dstatus, 0, sizeof(DevStatus), st);
    if (e != cudaSuccess) { *why = cudaGetErrorString(e); return VOMT_ERR_CUDA; }
    const int pblocks = (int)((nn + 255) / 256 < 2048 ? (nn + 255) / 256 : 2048);
    k_prepare<<<pblocks, 256, 0, st>>>(n, k, l, rho0, rho1, b, p.warm_start, u, w, phi, so[0]);
    ++launches;
    Launchers L = pick(k, p.u_norm, p.w_norm);
    if (p.max_iters == 0) {
        L.metrics<<<mblocks, blk, 0, st>>>(si[0], si[0], b, g, s, partials, dstatus);
        k_finalize<<<1, kFinThreads, 0, st>>>(partials, mblocks, cfg, 0, dstatus, nullptr, 0);
        launches += 2;
    }
    const bool tol_mode = cfg.tol_gap > 0.0;
    const int chunk = p.check_every * ((2048 + p.check_every - 1) / p.check_every);
    DevStatus hs;
    int t = 0;
    while (t < p.max_iters) {
        const int end = t + chunk < p.max_iters ? t + chunk : p.max_iters;
        for (int tt = t + 1; tt <= end; ++tt) {
            const int cur = tt & 1;
            L.step<<<grd, blk, 0, st>>>(si[cur ^ 1], so[cur], b, g, s, dstatus);
            ++launches;
            if (tt % p.check_every == 0 || tt == p.max_iters) {
                L.metrics<<<mblocks, blk, 0, st>>>(si[cur], si[cur ^ 1], b, g, s, partials, dstatus);
                k_finalize<<<1, kFinThreads, 0, st>>>(partials, mblocks, cfg, tt, dstatus, nullptr, 0);
                launches += 2;
            }
        }
        t = end;
        if (tol_mode && t < p.max_iters) {
            e = cudaMemcpyAsync(&hs, dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { *why = cudaGetErrorString(e); return VOMT_ERR_CUDA; }
            if (hs.stop) break;
        }
    }
    k_copy_out<<<pblocks, 256, 0, st>>>(n, k, l, si[0], si[1], dstatus, u, w, phi);
    ++launches;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { *why = cudaGetErrorString(e); return VOMT_ERR_CUDA; }
    int status = VOMT_OK;
    if (hs.error) { status = hs.error; *why = "iterate became non-finite"; }
    else if (cfg.tol_gap > 0.0 && hs.met[7] == 0.0) status = VOMT_NOT_CONVERGED;
    if (result) {
        result->primal = hs.met[0];
        result->dual = hs.met[1];
        result->rel_gap = hs.met[2];
        result->rel_res = hs.met[3];
        result->fp_resid = hs.met[4];
        result->dual_infeas = hs.met[5];
        result->mu = mu;
        result->nu = nu;
        result->tau = tau;
        result->iters = hs.iter;
        result->status = status;
        result->engine = VOMT_ENGINE_STREAM;
        result->checks = hs.checks;
        result->launches = launches;
        result->blocks = nblocks;
        result->halo = 0;
        result->variant = 0;
    }
    return status;
}

}  // namespace
}  // namespace vomt
