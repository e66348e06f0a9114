// Resident engine for vector OMT: one cooperative launch runs the whole PDHG
// solve (Section 7.2) with the state on chip.
//
// The n x n grid is cut into Gx x Gy rectangular tiles, one per thread block
// (one block per SM).  Each thread owns one grid point and keeps its iterate
// (phi, u_x, u_y, w for all channels and edges) and b = rho1 - rho0 in
// registers for the whole solve; HBM is touched only to load the densities and
// the initial iterate and to store the final iterate.  Within a tile the
// stencils of Appendix A go through shared memory.  Across tiles, the values a
// neighbour needs (phi on the four tile edges, u on the right column and top
// row) are written to L2 as 64-bit words tagged with the iteration number;
// the reader polls the words themselves, so one L2 round trip replaces the
// grid-wide barrier that Section 7.4 places around the phi update.  The two
// neighbouring shrinks that the divergence at a tile's left / bottom edge needs
// are recomputed from the received u and phi (the halo recompute of the
// streaming engine).
//
// Convergence checks (every check_every iterations and at the end) reduce
// the FP64 metric terms per block, publish one row per block, and every block
// sums all rows in the same fixed order, so all blocks take the same stopping
// decision without a further exchange.
#include <math.h>

#include "internal.h"
#include "pdhg_device.cuh"

namespace vomt {
namespace {

using namespace dev;

constexpr int EMAX = 64;              // longest tile side
constexpr int RES_THREADS = 512;      // most points per tile (one thread each)
constexpr int NE = 8;                 // exchange edges: phi L,R,D,U; u_x,u_y right; u_x,u_y top

struct ResGeom {
    int n, Gx, Gy, TXm, TYm;
};

struct ResArgs {
    ResGeom geo;
    GraphDev g;
    StepDev s;
    SolveCfg cfg;
    int un, wn, max_iters, check_every, warm;
    const float *rho0, *rho1;
    float *u, *w, *phi;
    unsigned long long *xch;
    double *rows;          // [2][G][NRED]
    uint32_t *flags;       // [G]
    ResCtl *ctl;
    DevStatus *st;
    double *hist;
    int hist_cap;
    int recv_max;          // receive-table capacity per block
};

template <int K>
struct LK {
    static constexpr int v = K * (K - 1) / 2 > 0 ? K * (K - 1) / 2 : 1;
};

// Shared-memory layout (bytes), computed identically on host and device.
struct SmemLayout {
    int red, S, dec, tsrc, tdst, sphi, sux, suy, sdx, sdy, hux, huy, hdx, hdy, phux, phuy, phdx, phdy, total;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SmemLayout smem_layout(int K, int TXm, int TYm, int recv_max)
{
    SmemLayout L;
    int o = 0;
    L.red = o; o += align16((RES_THREADS / 32) * NRED * 8);
    L.S = o; o += align16(NRED * 8);
    L.dec = o; o += 16;
    L.tsrc = o; o += align16(recv_max * 4);
    L.tdst = o; o += align16(recv_max * 4);
    L.sphi = o; o += align16(K * (TYm + 2) * (TXm + 2) * 4);
    L.sux = o; o += align16(K * TYm * (TXm + 1) * 4);
    L.suy = o; o += align16(K * (TYm + 1) * TXm * 4);
    L.sdx = o; o += align16(K * TYm * (TXm + 1) * 4);
    L.sdy = o; o += align16(K * (TYm + 1) * TXm * 4);
    L.hux = o; o += align16(K * TYm * 4);
    L.huy = o; o += align16(K * TYm * 4);
    L.hdx = o; o += align16(K * TXm * 4);
    L.hdy = o; o += align16(K * TXm * 4);
    L.phux = o; o += align16(K * TYm * 4);
    L.phuy = o; o += align16(K * TYm * 4);
    L.phdx = o; o += align16(K * TXm * 4);
    L.phdy = o; o += align16(K * TXm * 4);
    L.total = o;
    return L;
}

// number of words a tile receives per iteration (upper bound for a TXm x TYm tile)
__host__ __device__ inline int recv_words(int K, int TX, int TY)
{
    return 3 * K * TY + K * TY + 3 * K * TX + K * TX + 2 * K;
}

template <int K>
__global__ void __launch_bounds__(RES_THREADS, 1) k_resident(ResArgs a)
{
    constexpr int LKv = LK<K>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    const ResGeom G = a.geo;
    const int n = G.n;
    const size_t nn = (size_t)n * n;
    const SmemLayout SL = smem_layout(K, G.TXm, G.TYm, a.recv_max);
    double *red = (double *)(smem + SL.red);
    double *S = (double *)(smem + SL.S);
    int *dec = (int *)(smem + SL.dec);
    uint32_t *tsrc = (uint32_t *)(smem + SL.tsrc);
    uint32_t *tdst = (uint32_t *)(smem + SL.tdst);
    float *sphi = (float *)(smem + SL.sphi), *sux = (float *)(smem + SL.sux), *suy = (float *)(smem + SL.suy);
    float *sdx = (float *)(smem + SL.sdx), *sdy = (float *)(smem + SL.sdy);
    float *hux = (float *)(smem + SL.hux), *huy = (float *)(smem + SL.huy);
    float *hdx = (float *)(smem + SL.hdx), *hdy = (float *)(smem + SL.hdy);
    float *phux = (float *)(smem + SL.phux), *phuy = (float *)(smem + SL.phuy);
    float *phdx = (float *)(smem + SL.phdx), *phdy = (float *)(smem + SL.phdy);
    const int PW = G.TXm + 2, PH = G.TYm + 2, XW = G.TXm + 1, YW = G.TXm;
#define SPHI(c, r, q) sphi[((c) * PH + (r)) * PW + (q)]
#define SUX(c, r, q) sux[((c) * G.TYm + (r)) * XW + (q)]
#define SUY(c, r, q) suy[((c) * (G.TYm + 1) + (r)) * YW + (q)]
#define SDX(c, r, q) sdx[((c) * G.TYm + (r)) * XW + (q)]
#define SDY(c, r, q) sdy[((c) * (G.TYm + 1) + (r)) * YW + (q)]

    const int tile = blockIdx.x, gx = tile % G.Gx, gy = tile / G.Gx;
    const int x0 = gx * n / G.Gx, x1 = (gx + 1) * n / G.Gx;
    const int y0 = gy * n / G.Gy, y1 = (gy + 1) * n / G.Gy;
    const int TXa = x1 - x0, TYa = y1 - y0;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lx = tid % TXa, ly = tid / TXa;
    const bool act = ly < TYa;
    const int x = x0 + lx, y = y0 + ly;
    const bool hasL = gx > 0, hasR = gx < G.Gx - 1, hasD = gy > 0, hasU = gy < G.Gy - 1;
    const bool hasUL = hasL && hasU, hasDR = hasR && hasD;
    const int k = a.g.k, l = a.g.l;
    const float mu = a.s.mu, nu = a.s.nu, tau = a.s.tau, ih = a.s.ih, alpha = a.s.alpha;
    const float muih = mu * ih;
    const int T = a.max_iters, CE = a.check_every;
    const size_t SLOT = (size_t)NE * K * EMAX;       // words per (tile, parity)
    auto word = [&](int t_, int par, int E, int c, int idx) -> unsigned long long * {
        return a.xch + ((size_t)t_ * 2 + par) * SLOT + ((size_t)E * K + c) * EMAX + idx;
    };

    // ---- receive table: every halo word this tile reads, with its shared-memory destination
    // destinations: index into the float pool starting at sphi (all halo arrays follow it)
    int nrecv = 0;
    if (tid == 0) {
        auto add = [&](int t_, int E, int c, int idx, float *dst) {
            tsrc[nrecv] = (uint32_t)(((size_t)t_ * 2) * SLOT + ((size_t)E * K + c) * EMAX + idx);
            tdst[nrecv] = (uint32_t)(dst - sphi);
            ++nrecv;
        };
        for (int c = 0; c < K; ++c) {
            if (hasL)
                for (int r = 0; r < TYa; ++r) {
                    add(tile - 1, 1, c, r, &SPHI(c, r + 1, 0));
                    add(tile - 1, 4, c, r, &hux[c * G.TYm + r]);
                    add(tile - 1, 5, c, r, &huy[c * G.TYm + r]);
                }
            if (hasR)
                for (int r = 0; r < TYa; ++r) add(tile + 1, 0, c, r, &SPHI(c, r + 1, TXa + 1));
            if (hasD)
                for (int q = 0; q < TXa; ++q) {
                    add(tile - G.Gx, 3, c, q, &SPHI(c, 0, q + 1));
                    add(tile - G.Gx, 6, c, q, &hdx[c * G.TXm + q]);
                    add(tile - G.Gx, 7, c, q, &hdy[c * G.TXm + q]);
                }
            if (hasU)
                for (int q = 0; q < TXa; ++q) add(tile + G.Gx, 2, c, q, &SPHI(c, TYa + 1, q + 1));
            if (hasUL) add(tile + G.Gx - 1, 1, c, 0, &SPHI(c, TYa + 1, 0));
            if (hasDR) add(tile - G.Gx + 1, 3, c, 0, &SPHI(c, 0, TXa + 1));
        }
        dec[0] = 0;          // abort seen by a thread of this block
        dec[1] = nrecv;
        dec[2] = 0;          // stop decision of the last check
    }
    __syncthreads();
    nrecv = dec[1];

    // ---- own state
    float ph[K], ux[K], uy[K], bb[K], w[LKv];
    const size_t p = (size_t)y * n + x;
#pragma unroll
    for (int c = 0; c < K; ++c) {
        ph[c] = ux[c] = uy[c] = bb[c] = 0.0f;
        if (act) {
            bb[c] = a.rho1[c * nn + p] - a.rho0[c * nn + p];
            if (a.warm) {
                ph[c] = a.phi[c * nn + p];
                ux[c] = (x < n - 1) ? a.u[c * nn + p] : 0.0f;
                uy[c] = (y < n - 1) ? a.u[(k + c) * nn + p] : 0.0f;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < LKv; ++e) w[e] = (act && a.warm && e < l) ? a.w[e * nn + p] : 0.0f;

    auto publish = [&](int t) {
        if (!act) return;
        const uint32_t tag = (uint32_t)t + 1u;
        const int par = t & 1;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            if (lx == 0 && hasL) st_tagged(word(tile, par, 0, c, ly), ph[c], tag);
            if (lx == TXa - 1 && hasR) {
                st_tagged(word(tile, par, 1, c, ly), ph[c], tag);
                st_tagged(word(tile, par, 4, c, ly), ux[c], tag);
                st_tagged(word(tile, par, 5, c, ly), uy[c], tag);
            }
            if (ly == 0 && hasD) st_tagged(word(tile, par, 2, c, lx), ph[c], tag);
            if (ly == TYa - 1 && hasU) {
                st_tagged(word(tile, par, 3, c, lx), ph[c], tag);
                st_tagged(word(tile, par, 6, c, lx), ux[c], tag);
                st_tagged(word(tile, par, 7, c, lx), uy[c], tag);
            }
        }
    };
    // Load every halo word this thread owns, keep re-polling the ones whose tag is
    // not there yet (all of them per round, so a round costs one L2 round trip);
    // false if the wait ran out of time or another block aborted.
    auto receive = [&](int t) -> bool {
        const uint32_t tag = (uint32_t)t + 1u;
        const size_t par_off = (size_t)(t & 1) * SLOT;
        for (int base = 0; base < nrecv; base += 4 * nthr) {
            unsigned pending = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (base + tid + r * nthr < nrecv) pending |= 1u << r;
            uint64_t t0 = 0;
            for (uint32_t round = 0; pending; ++round) {
                unsigned long long v[4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    v[r] = (pending >> r & 1u) ? ld_relaxed64(a.xch + tsrc[base + tid + r * nthr] + par_off) : 0ull;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if ((pending >> r & 1u) && (uint32_t)(v[r] >> 32) == tag) {
                        sphi[tdst[base + tid + r * nthr]] = __uint_as_float((uint32_t)v[r]);
                        pending &= ~(1u << r);
                    }
                }
                if (pending && (round & 63u) == 63u) {
                    if (t0 == 0) t0 = global_ns();
                    if (ld_relaxed32(&a.ctl->abort)) return false;
                    if (global_ns() - t0 > kWaitBudgetNs) {
                        atomicExch(&a.ctl->abort, 1u);
                        atomicExch(&a.ctl->where, 1u);
                        return false;
                    }
                }
            }
        }
        return true;
    };

    // ---- initial halo exchange (state 0, tag 1)
    publish(0);
    if (act)
#pragma unroll
        for (int c = 0; c < K; ++c) SPHI(c, ly + 1, lx + 1) = ph[c];
    if (!receive(0)) dec[0] = 1;
    __syncthreads();
    bool aborted = dec[0] != 0;

    float oph[K], oux[K], ouy[K], ow[LKv];
    int checks = 0;
    bool stop = false;
    for (int t = (T == 0 ? 0 : 1); t <= T && !aborted && !stop; ++t) {
        const bool is_check = (T == 0) || (t % CE == 0) || (t == T);
        if (t > 0) {
            // ---- u', w' and ubar (Section 7.2, first two lines of the loop)
            float vx[K], vy[K], wx[LKv];
            if (act) {
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const float pc = SPHI(c, ly + 1, lx + 1);
                    vx[c] = ux[c] + ((x < n - 1) ? muih * (SPHI(c, ly + 1, lx + 2) - pc) : 0.0f);
                    vy[c] = uy[c] + ((y < n - 1) ? muih * (SPHI(c, ly + 2, lx + 1) - pc) : 0.0f);
                }
                shrink_u<K>(vx, vy, mu, a.un);
#pragma unroll
                for (int e = 0; e < LKv; ++e) {
                    if (e < l) {
                        const float ge = a.g.inv_c[e] * (pick<K>(ph, a.g.lo[e]) - pick<K>(ph, a.g.hi[e]));
                        wx[e] = w[e] + nu * ge;
                    } else {
                        wx[e] = 0.0f;
                    }
                }
                shrink_w<LKv>(wx, l, alpha * nu, a.wn);
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    SUX(c, ly, lx + 1) = 2.0f * vx[c] - ux[c];
                    SUY(c, ly + 1, lx) = 2.0f * vy[c] - uy[c];
                }
                if (lx == 0 && hasL) {           // u' at (x0-1, y) from the received halo
                    float hx[K], hy[K];
#pragma unroll
                    for (int c = 0; c < K; ++c) {
                        const float pl = SPHI(c, ly + 1, 0);
                        hx[c] = hux[c * G.TYm + ly] + muih * (SPHI(c, ly + 1, 1) - pl);
                        hy[c] = huy[c * G.TYm + ly] + ((y < n - 1) ? muih * (SPHI(c, ly + 2, 0) - pl) : 0.0f);
                    }
                    shrink_u<K>(hx, hy, mu, a.un);
#pragma unroll
                    for (int c = 0; c < K; ++c) SUX(c, ly, 0) = 2.0f * hx[c] - hux[c * G.TYm + ly];
                }
                if (ly == 0 && hasD) {           // u' at (x, y0-1)
                    float hx[K], hy[K];
#pragma unroll
                    for (int c = 0; c < K; ++c) {
                        const float pd = SPHI(c, 0, lx + 1);
                        hx[c] = hdx[c * G.TXm + lx] + ((x < n - 1) ? muih * (SPHI(c, 0, lx + 2) - pd) : 0.0f);
                        hy[c] = hdy[c * G.TXm + lx] + muih * (SPHI(c, 1, lx + 1) - pd);
                    }
                    shrink_u<K>(hx, hy, mu, a.un);
#pragma unroll
                    for (int c = 0; c < K; ++c) SUY(c, 0, lx) = 2.0f * hy[c] - hdy[c * G.TXm + lx];
                }
                if (is_check) {
                    if (lx == 0 && hasL)
#pragma unroll
                        for (int c = 0; c < K; ++c) {
                            phux[c * G.TYm + ly] = hux[c * G.TYm + ly];
                            phuy[c * G.TYm + ly] = huy[c * G.TYm + ly];
                        }
                    if (ly == 0 && hasD)
#pragma unroll
                        for (int c = 0; c < K; ++c) {
                            phdx[c * G.TXm + lx] = hdx[c * G.TXm + lx];
                            phdy[c * G.TXm + lx] = hdy[c * G.TXm + lx];
                        }
                }
            }
            __syncthreads();
            // ---- phi' = phi + tau (div_x ubar + div_G wbar + rho1 - rho0)
            if (act) {
                float r[K];
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const float xl = (x > 0) ? SUX(c, ly, lx) : 0.0f;
                    const float yd = (y > 0) ? SUY(c, ly, lx) : 0.0f;
                    r[c] = ih * ((SUX(c, ly, lx + 1) - xl) + (SUY(c, ly + 1, lx) - yd)) + bb[c];
                }
#pragma unroll
                for (int e = 0; e < LKv; ++e) {
                    if (e < l) {
                        const float v = a.g.inv_c[e] * (2.0f * wx[e] - w[e]);
                        const int lo = a.g.lo[e], hi = a.g.hi[e];
#pragma unroll
                        for (int c = 0; c < K; ++c) r[c] += (c == hi ? v : 0.0f) - (c == lo ? v : 0.0f);
                    }
                }
                if (is_check) {
#pragma unroll
                    for (int c = 0; c < K; ++c) { oph[c] = ph[c]; oux[c] = ux[c]; ouy[c] = uy[c]; }
#pragma unroll
                    for (int e = 0; e < LKv; ++e) ow[e] = w[e];
                }
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    ph[c] = ph[c] + tau * r[c];
                    ux[c] = vx[c];
                    uy[c] = vy[c];
                }
#pragma unroll
                for (int e = 0; e < LKv; ++e) w[e] = wx[e];
            }
            // nothing reads the phi tile again before the barrier below, so the own
            // value and the received halo can be written right away
            publish(t);
            if (act)
#pragma unroll
                for (int c = 0; c < K; ++c) SPHI(c, ly + 1, lx + 1) = ph[c];
            if (!receive(t)) dec[0] = 1;
            __syncthreads();
            if (dec[0]) { aborted = true; break; }
        } else {
            // zero iterations: metrics of the initial state, no change
#pragma unroll
            for (int c = 0; c < K; ++c) { oph[c] = ph[c]; oux[c] = ux[c]; ouy[c] = uy[c]; }
#pragma unroll
            for (int e = 0; e < LKv; ++e) ow[e] = w[e];
            if (act && lx == 0 && hasL)
                for (int c = 0; c < K; ++c) { phux[c * G.TYm + ly] = hux[c * G.TYm + ly]; phuy[c * G.TYm + ly] = huy[c * G.TYm + ly]; }
            if (act && ly == 0 && hasD)
                for (int c = 0; c < K; ++c) { phdx[c * G.TXm + lx] = hdx[c * G.TXm + lx]; phdy[c * G.TXm + lx] = hdy[c * G.TXm + lx]; }
        }
        if (!is_check) continue;

        // ---- FP64 convergence check on the state after iteration t
        if (act) {
#pragma unroll
            for (int c = 0; c < K; ++c) {
                SUX(c, ly, lx + 1) = ux[c];
                SUY(c, ly + 1, lx) = uy[c];
                SDX(c, ly, lx + 1) = ux[c] - oux[c];
                SDY(c, ly + 1, lx) = uy[c] - ouy[c];
            }
            if (lx == 0 && hasL)
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    SUX(c, ly, 0) = hux[c * G.TYm + ly];
                    SDX(c, ly, 0) = hux[c * G.TYm + ly] - phux[c * G.TYm + ly];
                }
            if (ly == 0 && hasD)
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    SUY(c, 0, lx) = hdy[c * G.TXm + lx];
                    SDY(c, 0, lx) = hdy[c * G.TXm + lx] - phdy[c * G.TXm + lx];
                }
        }
        __syncthreads();
        double v[NRED];
#pragma unroll
        for (int q = 0; q < NRED; ++q) v[q] = 0.0;
        if (act) {
            const double dih = (double)(n - 1);
            double rdiv[K], ddiv[K], dph[K];
            double nu_pt = 0.0, dn_u = 0.0;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const double uxc = ux[c], uyc = uy[c], phc = ph[c], bc = bb[c];
                dph[c] = phc - (double)oph[c];
                const double xl = (x > 0) ? (double)SUX(c, ly, lx) : 0.0;
                const double yd = (y > 0) ? (double)SUY(c, ly, lx) : 0.0;
                rdiv[c] = dih * ((uxc - xl) + (uyc - yd));
                const double dux = uxc - (double)oux[c], duy = uyc - (double)ouy[c];
                const double dxl = (x > 0) ? (double)SDX(c, ly, lx) : 0.0;
                const double dyd = (y > 0) ? (double)SDY(c, ly, lx) : 0.0;
                ddiv[c] = dih * ((dux - dxl) + (duy - dyd));
                v[RED_DU] += dux * dux + duy * duy;
                v[RED_DP] += dph[c] * dph[c];
                v[RED_D] += phc * bc;
                v[RED_BB] += bc * bc;
                const double gxx = (x < n - 1) ? dih * ((double)SPHI(c, ly + 1, lx + 2) - phc) : 0.0;
                const double gyy = (y < n - 1) ? dih * ((double)SPHI(c, ly + 2, lx + 1) - phc) : 0.0;
                if (a.un == VOMT_U_L12) {
                    nu_pt += sqrt(uxc * uxc + uyc * uyc);
                    dn_u = fmax(dn_u, sqrt(gxx * gxx + gyy * gyy));
                } else if (a.un == VOMT_U_L2) {
                    nu_pt += uxc * uxc + uyc * uyc;
                    dn_u += gxx * gxx + gyy * gyy;
                } else {
                    nu_pt += fabs(uxc) + fabs(uyc);
                    dn_u = fmax(dn_u, fmax(fabs(gxx), fabs(gyy)));
                }
            }
            if (a.un == VOMT_U_L2) { nu_pt = sqrt(nu_pt); dn_u = sqrt(dn_u); }
            double nw_pt = 0.0, dn_w = 0.0;
#pragma unroll
            for (int e = 0; e < LKv; ++e) {
                if (e < l) {
                    const int lo = a.g.lo[e], hi = a.g.hi[e];
                    const double ic = (double)a.g.inv_c[e];
                    const double we = w[e], dwe = we - (double)ow[e];
                    v[RED_DW] += dwe * dwe;
                    double ge = 0.0;
#pragma unroll
                    for (int c = 0; c < K; ++c) {
                        const double sgn = (c == lo) ? 1.0 : (c == hi ? -1.0 : 0.0);
                        ge += sgn * (double)ph[c];
                        rdiv[c] -= sgn * ic * we;
                        ddiv[c] -= sgn * ic * dwe;
                    }
                    ge *= ic;
                    if (a.wn == VOMT_W_L1) { nw_pt += fabs(we); dn_w = fmax(dn_w, fabs(ge)); }
                    else { nw_pt += we * we; dn_w += ge * ge; }
                }
            }
            if (a.wn == VOMT_W_L2) { nw_pt = sqrt(nw_pt); dn_w = sqrt(dn_w); }
            v[RED_P] = nu_pt + (double)alpha * nw_pt;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const double rc = rdiv[c] + (double)bb[c];
                v[RED_RR] += rc * rc;
                v[RED_X] += dph[c] * ddiv[c];
            }
            double di = fmax(dn_u - 1.0, 0.0);
            if (l > 0) di = fmax(di, dn_w - (double)alpha);
            v[RED_MAX] = di;
        }
        // block reduction in a fixed order
        const int lane = tid & 31, wid = tid >> 5, nw = (nthr + 31) >> 5;
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
            for (int q = 0; q < NRED; ++q) red[wid * NRED + q] = v[q];
        __syncthreads();
        const int cpar = checks & 1;
        const uint32_t cflag = (uint32_t)checks + 1u;
        if (tid < NRED) {
            double acc = red[tid];
            for (int q = 1; q < nw; ++q) acc = (tid == RED_MAX) ? fmax(acc, red[q * NRED + tid]) : acc + red[q * NRED + tid];
            a.rows[((size_t)cpar * gridDim.x + tile) * NRED + tid] = acc;
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) st_release32(&a.flags[tile], cflag);
        // every block sums every row in block order (identical in all blocks)
        if (tid < NRED) {
            bool ok = true;
            for (int b = 0; b < (int)gridDim.x && ok; ++b) ok = wait_flag(&a.flags[b], cflag, a.ctl, 2);
            double acc = 0.0;
            if (ok)
                for (int b = 0; b < (int)gridDim.x; ++b) {
                    const double x_ = ld_relaxed_f64(&a.rows[((size_t)cpar * gridDim.x + b) * NRED + tid]);
                    acc = (tid == RED_MAX) ? fmax(acc, x_) : acc + x_;
                }
            S[tid] = acc;
            if (!ok) dec[0] = 1;
        }
        __syncthreads();
        if (dec[0]) { aborted = true; break; }
        if (tid == 0) {
            double m[NMET];
            m[0] = S[RED_P];
            m[1] = S[RED_D];
            m[2] = fabs(m[0] - m[1]) / fmax(fabs(m[0]), 1e-300);
            m[3] = sqrt(S[RED_RR]) / (S[RED_BB] > 0.0 ? sqrt(S[RED_BB]) : 1.0);
            m[4] = S[RED_DU] / a.cfg.mu + (a.cfg.has_w ? S[RED_DW] / a.cfg.nu : 0.0) + S[RED_DP] / a.cfg.tau -
                   2.0 * S[RED_X];
            m[5] = S[RED_MAX];
            m[6] = (double)t;
            bool finite = true;
            for (int q = 0; q < 6; ++q) finite = finite && isfinite(m[q]);
            const bool conv = a.cfg.tol_gap > 0.0 && m[2] <= a.cfg.tol_gap && m[3] <= a.cfg.tol_res;
            m[7] = conv ? 1.0 : 0.0;
            if (tile == 0) {
                for (int q = 0; q < NMET; ++q) a.st->met[q] = m[q];
                if (a.hist && checks < a.hist_cap)
                    for (int q = 0; q < NMET; ++q) a.hist[(size_t)checks * NMET + q] = m[q];
                a.st->checks = checks + 1;
                a.st->iter = t;
                if (!finite) a.st->error = VOMT_ERR_NONFINITE;
                if (conv || !finite) a.st->stop = 1;
            }
            dec[2] = (conv || !finite) ? 1 : 0;
        }
        __syncthreads();
        ++checks;
        stop = dec[2] != 0;
        if (T == 0) break;
    }
    if (aborted) {
        if (tid == 0 && tile == 0) {
            a.st->error = VOMT_ERR_BARRIER_TIMEOUT;
            a.st->stop = 1;
        }
        return;
    }
    // ---- final iterate to the caller's arrays
    if (act) {
#pragma unroll
        for (int c = 0; c < K; ++c) {
            a.phi[c * nn + p] = ph[c];
            a.u[c * nn + p] = ux[c];
            a.u[(k + c) * nn + p] = uy[c];
        }
#pragma unroll
        for (int e = 0; e < LKv; ++e)
            if (e < l) a.w[e * nn + p] = w[e];
    }
#undef SPHI
#undef SUX
#undef SUY
#undef SDX
#undef SDY
}

using ResKernel = void (*)(ResArgs);

ResKernel pick_kernel(int k)
{
    switch (k) {
        case 1: return k_resident<1>;
        case 2: return k_resident<2>;
        case 3: return k_resident<3>;
        case 4: return k_resident<4>;
        case 5: return k_resident<5>;
        case 6: return k_resident<6>;
        case 7: return k_resident<7>;
        default: return k_resident<8>;
    }
}

}  // namespace

// Tile plan.  Cost of a plan in point-equivalents: the points of the largest
// tile (one thread each, so proportional to the time of one iteration's
// arithmetic) plus, when there is more than one tile, the L2 exchange between
// tiles (about 1000 points' worth of time per iteration).  Every grid of at
// most `max_blocks` tiles with sides <= 64 and <= 512 points per tile is tried.
bool resident_plan(int n, int k, int max_blocks, ResidentPlan *out)
{
    (void)k;
    long best = -1, best_per = 0;
    for (int Gx = 1; Gx <= n && Gx <= max_blocks; ++Gx) {
        const int TX = (n + Gx - 1) / Gx;
        if (TX > EMAX) continue;
        for (int Gy = 1; Gy <= n && Gx * Gy <= max_blocks; ++Gy) {
            const int TY = (n + Gy - 1) / Gy;
            if (TY > EMAX || TX * TY > RES_THREADS) continue;
            const long cost = (long)TX * TY + (Gx * Gy > 1 ? 1000 : 0), per = TX + TY;
            if (best < 0 || cost < best || (cost == best && per < best_per)) {
                best = cost;
                best_per = per;
                out->Gx = Gx;
                out->Gy = Gy;
                out->TXm = TX;
                out->TYm = TY;
            }
        }
    }
    if (best < 0) return false;
    out->threads = ((out->TXm * out->TYm + 31) / 32) * 32;
    return true;
}

int resident_solve(vomt_ctx *ctx, const GraphDev &g, const StepDev &s, const SolveCfg &cfg, const vomt_params &p,
                   const ResidentPlan &plan, const float *rho0, const float *rho1, float *u, float *w, float *phi,
                   cudaStream_t st)
{
    const int K = g.k;
    const int G = plan.Gx * plan.Gy;
    const int recv_max = recv_words(K, plan.TXm, plan.TYm);
    const SmemLayout SL = smem_layout(K, plan.TXm, plan.TYm, recv_max);
    // scratch: exchange words, check rows, flags, control words
    const size_t xch_bytes = (size_t)G * 2 * NE * K * EMAX * sizeof(unsigned long long);
    const size_t rows_bytes = (size_t)2 * G * NRED * sizeof(double);
    const size_t flag_bytes = ((size_t)G * sizeof(uint32_t) + 255) & ~(size_t)255;
    const size_t need = xch_bytes + rows_bytes + flag_bytes + 256;
    int rc = ensure_buffer(ctx, &ctx->rscratch, &ctx->rscratch_bytes, need, "resident scratch");
    if (rc) return rc;
    unsigned char *base = (unsigned char *)ctx->rscratch;
    ResArgs a;
    a.geo = ResGeom{s.n, plan.Gx, plan.Gy, plan.TXm, plan.TYm};
    a.g = g;
    a.s = s;
    a.cfg = cfg;
    a.un = p.u_norm;
    a.wn = p.w_norm;
    a.max_iters = p.max_iters;
    a.check_every = p.check_every;
    a.warm = p.warm_start;
    a.rho0 = rho0;
    a.rho1 = rho1;
    a.u = u;
    a.w = w;
    a.phi = phi;
    a.xch = (unsigned long long *)base;
    a.rows = (double *)(base + xch_bytes);
    a.flags = (uint32_t *)(base + xch_bytes + rows_bytes);
    a.ctl = (ResCtl *)(base + xch_bytes + rows_bytes + flag_bytes);
    a.st = ctx->dstatus;
    a.recv_max = recv_max;
    const int max_checks = p.max_iters / p.check_every + 2;
    if (ctx->hist_cap < max_checks) {
        if (ctx->dhist) cudaFree(ctx->dhist);
        ctx->dhist = nullptr;
        ctx->hist_cap = 0;
        cudaError_t e = cudaMalloc(&ctx->dhist, sizeof(double) * NMET * (size_t)max_checks);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "history");
        ctx->hist_cap = max_checks;
    }
    a.hist = ctx->dhist;
    a.hist_cap = ctx->hist_cap;

    ResKernel kern = pick_kernel(K);
    cudaError_t e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SL.total);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "resident smem attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)kern, plan.threads, SL.total);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "resident occupancy");
    if (per_sm < 1 || G > per_sm * ctx->sm_count) {
        ctx->err = "resident plan does not fit on the device";
        return VOMT_ERR_TOO_LARGE;
    }
    e = cudaMemsetAsync(base, 0, need, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dstatus, 0, sizeof(DevStatus), st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "resident reset");
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(plan.threads), args, SL.total, st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "resident launch");
    ctx->launches += 1;
    e = cudaMemcpyAsync(&ctx->hstatus[0], ctx->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "resident solve");
    return VOMT_OK;
}

}  // namespace vomt
