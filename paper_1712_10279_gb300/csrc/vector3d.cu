// Vector OMT on 3-D grids: the discretization of Appendix A with a third
// direction (the extension to volumes that the paper points to for 3-D DTI,
// Section 8.2), solved by the streaming engine's scheme: one fused launch per
// PDHG iteration (Section 7.2), FP64 convergence checks.
//
// Grid n x n x n on [0,1]^3, h = 1/(n-1); every field is planar [c][z][y][x]
// with x fastest; the flux has three components u_x, u_y, u_z per channel, with
// ghost entries at the last index of their own direction (kept zero).  The
// backward-difference divergence at a point takes 2u' - u of its three upwind
// neighbours, so the step marches blocks up z: u' is computed once per point,
// the x and y components meet their neighbours through shared memory and the z
// component is carried to the next plane.  Two forms of that step: inputs staged
// by TMA tiles (vector3d_tma.cu; n a multiple of 4, n >= 40, k <= 6) and, for
// every other case, the form below with per-thread loads.  Step rule:
// ||grad||^2 <= 12 / h^2 in 3-D, so mu = 1/(48 tau (n-1)^2) (1/(24 tau (n-1)^2)
// without edges) keeps the 2-D rule's share of the bound.
#include <math.h>
#include <string.h>

#include "internal.h"
#include "pdhg_device.cuh"
#include "vector3d.cuh"
#include "vector3d_tma.h"

namespace vomt {
namespace {

using namespace v3;

constexpr int T3 = 256;

// z-marching form of the same iteration (2.5-D blocking).  A block owns a
// TX x TY column of the grid over a chunk of z; per z plane it stages phi of
// planes z and z+1 (with a one-cell halo in x and y) in shared memory, prefetches
// plane z+2 into registers, computes u' once per point, and publishes the
// x and y components of 2u' - u through shared memory (the tile's x0-1 column and
// y0-1 row are recomputed by the block).  The z component of 2u' - u at z-1 is the
// thread's own value from the previous plane, carried in a register; the chunk's
// first plane recomputes it.
constexpr int HX = MX + 2, HY = MY + 2, HP = HX * HY;

template <int K>
struct MarchSmem {
    static constexpr int phi = 3 * K * HP;              // three plane slots
    static constexpr int bx = K * MY * (MX + 1);        // 2u'_x - u_x, column 0 = x0-1
    static constexpr int by = K * (MY + 1) * MX;        // 2u'_y - u_y, row 0 = y0-1
    static constexpr size_t bytes = sizeof(float) * (phi + bx + by);
};

template <int K>
__device__ __forceinline__ void load_plane(float *slot, const float *__restrict__ phi, size_t m, int n, int x0,
                                           int y0, int zp)
{
    const bool zin = zp >= 0 && zp < n;
    for (int e = threadIdx.x; e < HP; e += MT) {
        const int j = e / HX, i = e - j * HX;
        const int x = x0 + i - 1, y = y0 + j - 1;
        const bool in = zin && x >= 0 && x < n && y >= 0 && y < n;
        const size_t q = in ? ((size_t)zp * n + y) * n + x : 0;
#pragma unroll
        for (int c = 0; c < K; ++c) slot[c * HP + e] = in ? __ldg(phi + c * m + q) : 0.0f;
    }
}

template <int K, int UN, int WN>
__global__ void __launch_bounds__(MT, K <= 4 ? 2 : 1) k_step3m(S3In in, S3Out out, const float *__restrict__ b, OpDev g,
                                                 StepDev s, const DevStatus *__restrict__ st, int zc)
{
    cudaGridDependencySynchronize();      // after the previous kernel (no-op for a normal launch)
    if (st->stop) return;
    constexpr int LK = LK3<K>::v;
    constexpr int PF = (HP + MT - 1) / MT;
    extern __shared__ float smem[];
    float *sphi = smem;
    float *sbx = smem + MarchSmem<K>::phi;
    float *sby = sbx + MarchSmem<K>::bx;
    const int n = s.n;
    const size_t m = (size_t)n * n * n, nn = (size_t)n * n;
    const int tid = threadIdx.x, tx = tid % MX, ty = tid / MX;
    const int x0 = blockIdx.x * MX, y0 = blockIdx.y * MY;
    const int z0 = blockIdx.z * zc, z1 = min(n, z0 + zc);
    const int x = x0 + tx, y = y0 + ty;
    const bool inb = x < n && y < n;
    const bool hx = x < n - 1, hy = y < n - 1, lx = x > 0, ly = y > 0;
    const float mi = s.mu * s.ih;
    auto S = [&](int zp, int c, int j, int i) -> float & { return sphi[((zp % 3) * K + c) * HP + j * HX + i]; };

    load_plane<K>(&S(z0, 0, 0, 0), in.phi, m, n, x0, y0, z0);
    load_plane<K>(&S(z0 + 1, 0, 0, 0), in.phi, m, n, x0, y0, z0 + 1);
    // 2u'_z - u_z at (x, y, z0 - 1)
    float cz[K];
#pragma unroll
    for (int c = 0; c < K; ++c) cz[c] = 0.0f;
    if (z0 > 0 && inb) {
        const size_t p = (size_t)(z0 - 1) * nn + (size_t)y * n + x;
        float ax[K], ay[K], az[K], az0[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const float *P = in.phi + c * m + p;
            const float pc = __ldg(P), px = hx ? __ldg(P + 1) : 0.0f, py = hy ? __ldg(P + n) : 0.0f;
            const float pz = __ldg(P + nn);
            const size_t q = c * m + p;
            az0[c] = __ldg(in.uz + q);
            ax[c] = upre(__ldg(in.ux + q), px, pc, hx, mi);
            ay[c] = upre(__ldg(in.uy + q), py, pc, hy, mi);
            az[c] = upre(az0[c], pz, pc, true, mi);
        }
        shrink_u3<K, UN>(ax, ay, az, s.mu, g.wc);
#pragma unroll
        for (int c = 0; c < K; ++c) cz[c] = 2.0f * az[c] - az0[c];
    }
    __syncthreads();

    for (int z = z0; z < z1; ++z) {
        const bool hz = z < n - 1, lz = z > 0;
        const size_t p = (size_t)z * nn + (size_t)(inb ? y : 0) * n + (inb ? x : 0);
        // prefetch plane z + 2 (needed as the "+1" plane of step z + 1)
        float pf[PF][K];
        const int zn = z + 2;
        const bool want = zn < n && zn <= z1;
#pragma unroll
        for (int r = 0; r < PF; ++r) {
            const int e = tid + r * MT;
            const int j = e / HX, i = e - j * HX;
            const int xx = x0 + i - 1, yy = y0 + j - 1;
            const bool ok = want && e < HP && xx >= 0 && xx < n && yy >= 0 && yy < n;
            const size_t q = ok ? ((size_t)zn * n + yy) * n + xx : 0;
#pragma unroll
            for (int c = 0; c < K; ++c) pf[r][c] = ok ? __ldg(in.phi + c * m + q) : 0.0f;
        }
        // own u' and 2u' - u
        float pc[K], vx[K], vy[K], vz[K], ux0[K], uy0[K], uz0[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const size_t q = c * m + p;
            ux0[c] = inb ? __ldg(in.ux + q) : 0.0f;
            uy0[c] = inb ? __ldg(in.uy + q) : 0.0f;
            uz0[c] = inb ? __ldg(in.uz + q) : 0.0f;
            pc[c] = S(z, c, ty + 1, tx + 1);
            vx[c] = upre(ux0[c], S(z, c, ty + 1, tx + 2), pc[c], hx, mi);
            vy[c] = upre(uy0[c], S(z, c, ty + 2, tx + 1), pc[c], hy, mi);
            vz[c] = upre(uz0[c], S(z + 1, c, ty + 1, tx + 1), pc[c], hz, mi);
        }
        shrink_u3<K, UN>(vx, vy, vz, s.mu, g.wc);
#pragma unroll
        for (int c = 0; c < K; ++c) {
            sbx[(c * MY + ty) * (MX + 1) + tx + 1] = 2.0f * vx[c] - ux0[c];
            sby[(c * (MY + 1) + ty + 1) * MX + tx] = 2.0f * vy[c] - uy0[c];
        }
        // the tile's y0-1 row (threads 0..MX-1) and x0-1 column (threads MX..MX+MY-1)
        {
            int hxp = -1, hyp = -1, j = 0, i = 0;
            if (tid < MX) {
                if (y0 > 0 && x0 + tid < n) { hxp = x0 + tid; hyp = y0 - 1; j = 0; i = tid + 1; }
            } else if (tid < MX + MY) {
                if (x0 > 0 && y0 + tid - MX < n) { hxp = x0 - 1; hyp = y0 + tid - MX; j = tid - MX + 1; i = 0; }
            }
            if (hxp >= 0) {
                const bool ax_in = hxp < n - 1, ay_in = hyp < n - 1;
                const size_t ph = (size_t)z * nn + (size_t)hyp * n + hxp;
                float ax[K], ay[K], az[K], a0x[K], a0y[K];
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const size_t q = c * m + ph;
                    a0x[c] = __ldg(in.ux + q);
                    a0y[c] = __ldg(in.uy + q);
                    const float here = S(z, c, j, i);
                    ax[c] = upre(a0x[c], S(z, c, j, i + 1), here, ax_in, mi);
                    ay[c] = upre(a0y[c], S(z, c, j + 1, i), here, ay_in, mi);
                    az[c] = upre(__ldg(in.uz + q), S(z + 1, c, j, i), here, hz, mi);
                }
                shrink_u3<K, UN>(ax, ay, az, s.mu, g.wc);
                if (tid < MX) {
#pragma unroll
                    for (int c = 0; c < K; ++c) sby[(c * (MY + 1)) * MX + tid] = 2.0f * ay[c] - a0y[c];
                } else {
#pragma unroll
                    for (int c = 0; c < K; ++c) sbx[(c * MY + (tid - MX)) * (MX + 1)] = 2.0f * ax[c] - a0x[c];
                }
            }
        }
        // w' at the point
        float w0[LK], wx[LK];
#pragma unroll
        for (int e = 0; e < LK; ++e) {
            if (e < g.l) {
                w0[e] = inb ? __ldg(in.w + e * m + p) : 0.0f;
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
        __syncthreads();
        // phi' = phi + tau (div ubar + div_G wbar + rho1 - rho0)
        float r[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const float bxc = 2.0f * vx[c] - ux0[c], byc = 2.0f * vy[c] - uy0[c], bzc = 2.0f * vz[c] - uz0[c];
            const float bxl = lx ? sbx[(c * MY + ty) * (MX + 1) + tx] : 0.0f;
            const float byl = ly ? sby[(c * (MY + 1) + ty) * MX + tx] : 0.0f;
            const float bzl = lz ? cz[c] : 0.0f;
            r[c] = s.ih * ((bxc - bxl) + (byc - byl) + (bzc - bzl)) + (inb ? __ldg(b + c * m + p) : 0.0f);
            cz[c] = bzc;
        }
#pragma unroll
        for (int e = 0; e < LK; ++e) {
            const float v = 2.0f * wx[e] - w0[e];
#pragma unroll
            for (int c = 0; c < K; ++c) r[c] -= g.Dv[c][e] * v;
        }
        if (inb) {
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
        // plane z + 2 into the slot of plane z - 1 (every thread is past step z - 1)
#pragma unroll
        for (int r2 = 0; r2 < PF; ++r2) {
            const int e = tid + r2 * MT;
            if (e < HP)
#pragma unroll
                for (int c = 0; c < K; ++c) sphi[((zn % 3) * K + c) * HP + e] = pf[r2][c];
        }
        __syncthreads();
    }
}

// FP64 block partials of one convergence check (slots RED_*): per-point terms in
// FP32 (the constraint residual in FP64), summed per thread and warp in pairs of
// FP32 numbers with TwoSum and per block in FP64 (CheckAcc, block_sum_store).
// At most kMetricBlocks blocks loop over the volume's points.
template <int K, int UN, int WN>
__global__ void __launch_bounds__(T3) k_metrics3(S3In cur, S3In prv, const float *__restrict__ b, OpDev g,
                                                 StepDev s, double *__restrict__ partials,
                                                 const DevStatus *__restrict__ st)
{
    cudaGridDependencySynchronize();      // after the previous kernel (no-op for a normal launch)
    if (st->stop) return;
    constexpr int LK = LK3<K>::v;
    const int n = s.n;
    const size_t m = (size_t)n * n * n;
    CheckAcc acc;
    acc.zero();
    for (size_t p = (size_t)blockIdx.x * T3 + threadIdx.x; p < m; p += (size_t)gridDim.x * T3) {
        const int x = (int)(p % n), y = (int)((p / n) % n), z = (int)(p / ((size_t)n * n));
        const long SX = 1, SY = n, SZ = (long)n * n;
        const bool hx = x < n - 1, hy = y < n - 1, hz = z < n - 1, lx = x > 0, ly = y > 0, lz = z > 0;
        const float ih = s.ih, alpha = s.alpha;
        const double dih = (double)(n - 1);
        float ph[K], dph[K], ddiv[K], gwb[K];
        float uxs[K], uys[K], uzs[K], gxs[K], gys[K], gzs[K];     // nuclear norms only
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
            if (UN == VOMT_U_NUC) {
                uxs[c] = a; uys[c] = bq; uzs[c] = cq;
                gxs[c] = gx; gys[c] = gy; gzs[c] = gz;
            } else if (UN == VOMT_U_L12) {
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
        if constexpr (UN == VOMT_U_NUC) {        // sum of the nuclear norms, largest spectral norm
            float n1, s1, n2, s2, n3, s3;
            mat::sym_nuc_spec<K>(uxs, n1, s1);
            mat::sym_nuc_spec<K>(uys, n2, s2);
            mat::sym_nuc_spec<K>(uzs, n3, s3);
            nu_pt = n1 + n2 + n3;
            mat::sym_nuc_spec<K>(gxs, n1, s1);
            mat::sym_nuc_spec<K>(gys, n2, s2);
            mat::sym_nuc_spec<K>(gzs, n3, s3);
            dn_u = fmaxf(s1, fmaxf(s2, s3));
        }
        float nw_pt = 0.0f, dn_w = 0.0f, wg2 = 0.0f, gg2 = 0.0f;
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
                if (WN == VOMT_W_L1) {
                    nw_pt += wgt * fabsf(we);
                    dn_w = fmaxf(dn_w, fabsf(ge));
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
        if (WN == VOMT_W_L2) { nw_pt = sqrtf(nw_pt); dn_w = sqrtf(dn_w); }
        double rr = 0.0;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const double rc = rdiv[c] + (double)gwb[c];
            rr += (double)g.wc[c] * rc * rc;
            fx += g.wc[c] * dph[c] * ddiv[c];
        }
        acc.add_d(RED_RR, rr);
        acc.add(RED_P, nu_pt + alpha * nw_pt);
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
    block_sum_store<T3>(acc, partials + (size_t)blockIdx.x * NRED);
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
    void (*step)(S3In, S3Out, const float *, OpDev, StepDev, const DevStatus *, int);
    void (*metrics)(S3In, S3In, const float *, OpDev, StepDev, double *, const DevStatus *);
    size_t smem;
};

template <int K, int UN, int WN>
L3 make3()
{
    return L3{k_step3m<K, UN, WN>, k_metrics3<K, UN, WN>, MarchSmem<K>::bytes};
}

template <int K>
L3 pick3_norms(int un, int wn)
{
    if constexpr (K == 3 || K == 6) {          // nuclear norms: compact 2 x 2 and 3 x 3 matrices
        if (un == VOMT_U_NUC)
            return wn == VOMT_W_L1 ? make3<K, 3, 0>() : (wn == VOMT_W_L2 ? make3<K, 3, 1>() : make3<K, 3, 2>());
        if (wn == VOMT_W_NUC) return un == VOMT_U_L2 ? make3<K, 1, 2>() : make3<K, 2, 2>();
    }
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

namespace vomt {

// The 3-D solve after validation and step sizes: workspace, the z-marching
// iterations with their checks, the copy-out; ctx->hstatus[0] holds the final
// status block.  rho0, rho1, u, w, phi are [c][z][y][x] volumes (u: u_x, u_y,
// u_z runs of k volumes each) in the compact channels of g.
int solve3d_core(vomt_ctx *ctx, int n, const OpDev &g, const StepDev &s, const SolveCfg &cfg, const vomt_params &p,
                 int zc_user, const float *rho0, const float *rho1, float *u, float *w, float *phi, cudaStream_t st)
{
    ctx->hist_raw = false;           // k_finalize writes finished rows
    const int k = g.k, l = g.l;
    const size_t m = (size_t)n * n * n;
    cudaError_t e;
    int rc;
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
    const int mblocks = nblocks < kMetricBlocks ? nblocks : kMetricBlocks;     // blocks of a check
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
    e = cudaFuncSetAttribute((const void *)L.step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "3-D step shared memory");
    // inputs by TMA tiles where they apply (n a multiple of 4, n >= 40, k <= 6)
    Tma3Plan *tp = tma3_supported(n, k, l, p.u_norm, p.w_norm)
                       ? tma3_plan_create(n, k, l, p.u_norm, p.w_norm, so[0].phi, so[1].phi, b)
                       : nullptr;
    ctx->last_variant = tp ? 1 : 0;
    // z chunk: the longest of 32, 16, 8, 4 planes that still gives 1.5 blocks per SM
    // (TMA form; longer chunks amortise the pipeline fill, but fewer blocks than SMs
    // leave HBM idle; 32 measured best at 128^3 and 256^3) or four blocks per SM
    // (per-thread form, which needs the warps)
    const int tiles = ((n + MX - 1) / MX) * ((n + MY - 1) / MY);
    const size_t want = tp ? (size_t)(3 * ctx->sm_count / 2) : (size_t)(4 * ctx->sm_count);
    int zc = 4;
    for (int c : {32, 16, 8})
        if ((size_t)tiles * ((n + c - 1) / c) >= want) { zc = c; break; }
    if (zc_user > 0) zc = std::min(zc_user, n);
    const dim3 mgrid((n + MX - 1) / MX, (n + MY - 1) / MY, (n + zc - 1) / zc);
    ctx->last_blocks = (int)(mgrid.x * mgrid.y * mgrid.z);
    auto check = [&](int t, int cur) {
        launch_pdl(L.metrics, dim3(mblocks), dim3(T3), 0, st, si[cur], si[cur ^ 1], (const float *)b, g, s,
                   ctx->partials, (const DevStatus *)ctx->dstatus);
        launch_pdl(k_finalize, dim3(1), dim3(kFinThreads), 0, st, (const double *)ctx->partials, mblocks, cfg, t,
                   ctx->dstatus, ctx->dhist, ctx->hist_cap);
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
            if (tp)
                tma3_launch_step(tp, cur ^ 1, so[cur], g, s, ctx->dstatus, zc, st);
            else
                launch_pdl(L.step, mgrid, dim3(MT), (size_t)L.smem, st, si[cur ^ 1], so[cur], (const float *)b, g, s,
                           (const DevStatus *)ctx->dstatus, zc);
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
    tma3_plan_destroy(tp);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "3-D solve");
    return VOMT_OK;
}

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
        ctx->last_variant = 0;
        if (n < 2 || n > 1024) return fail(ctx, VOMT_ERR_BAD_ARG, "3-D grids: n must be in [2, 1024]");
        if (!rho0 || !rho1 || !u || !phi || !graph || (graph->n_edges > 0 && !w))
            return fail(ctx, VOMT_ERR_BAD_ARG, "null array");
        if (pin && pin->eps != 0.0) return fail(ctx, VOMT_ERR_BAD_ARG, "3-D grids take eps = 0");
        if (pin && pin->pitch != 0 && pin->pitch != n) return fail(ctx, VOMT_ERR_BAD_ARG, "3-D grids take dense arrays");
        cudaStream_t st = (cudaStream_t)stream;
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaSetDevice");
        OpDev g;
        StepDev s;
        SolveCfg cfg;
        vomt_params p, p3;
        vomt_default_params(&p3);
        if (pin) p3 = *pin;
        const int zc_user = p3.halo;       // 3-D: planes each block marches through (0: the library's choice)
        if (zc_user < 0) return fail(ctx, VOMT_ERR_BAD_ARG, "halo (the 3-D z chunk) must be >= 0");
        p3.halo = 0;
        int rc = prepare_vector(ctx, n, graph, alpha, &p3, &g, &s, &cfg, &p);
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
        rc = check_vector_densities(ctx, g.k * n, n, rho0, rho1, st);
        if (rc) return rc;
        rc = solve3d_core(ctx, n, g, s, cfg, p, zc_user, rho0, rho1, u, w, phi, st);
        if (rc) return rc;
        int status = VOMT_OK;
        fill_result(ctx, cfg, VOMT_ENGINE_STREAM, result, &status);
        return status;
    } catch (...) {
        return fail(ctx, VOMT_ERR_BAD_ARG, "internal exception");
    }
}
