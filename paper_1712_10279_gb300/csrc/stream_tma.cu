// Streaming engine, tensor-memory-accelerator form of the fused iteration.
//
// One launch runs one PDHG iteration of Section 7.2 over the whole grid, like
// k_step in vector_stream.cu, but each 64 x 16 tile's inputs arrive in shared
// memory by TMA (cp.async.bulk.tensor) instead of per-thread loads: one thread
// issues five 3-D tile copies (phi with a one-cell halo on every side, u_x and
// u_y with a halo to the left and below, w and b without halo) that complete on
// one mbarrier; the whole block then computes from shared memory.  The copies
// keep the tile's bytes in flight without tying up registers, which is what the
// per-thread loads lacked at large grids (their warps waited on DRAM latency).
//
// TMA rules honoured here: the tensors are 3-D (x, y, plane) with row and plane
// strides of 4n and 4n^2 bytes, so n must be a multiple of 4 (16-byte strides);
// every box starts at an x that is a multiple of 4 (the tile's x0 - 4 for the
// halo boxes, x0 for the others); loads may start at negative or out-of-range
// coordinates and then read zeros, which the stencil masks away anyway.  The
// wait on the mbarrier is bounded: a wait that runs out marks the solve failed
// (status error) instead of hanging.
#include <math.h>
#include <string.h>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>

#include "internal.h"
#include "matrix_norms.cuh"
#include "pdhg_device.cuh"
#include "stream_tma.h"

namespace vomt {
namespace {

constexpr int TX = 64, TY = 16, TXP = TX + 8, NTH = 256;
constexpr int ROWS = TY / (NTH / TX);    // rows per thread (4)

__host__ __device__ inline int align128(int x) { return (x + 127) & ~127; }

struct TmaSmem {
    int phi, ux, uy, w, b, total;
    unsigned bytes;                       // bytes the five copies deliver
};

__host__ __device__ inline TmaSmem tma_smem(int K, int l)
{
    TmaSmem S;
    int o = 0;
    S.phi = o; o += align128(K * (TY + 2) * TXP * 4);
    S.ux = o; o += align128(K * (TY + 1) * TXP * 4);
    S.uy = o; o += align128(K * (TY + 1) * TXP * 4);
    S.w = o; o += align128((l > 0 ? l : 1) * TY * TX * 4);
    S.b = o; o += align128(K * TY * TX * 4);
    S.total = o;
    S.bytes = (unsigned)(K * (TY + 2) * TXP * 4 + 2 * K * (TY + 1) * TXP * 4 + l * TY * TX * 4 + K * TY * TX * 4);
    return S;
}

// shrink_2 factor and soft threshold of Appendix B (pdhg_device.cuh)
using dev::shrink2_factor;
using dev::soft;

template <int K, int UN>
__device__ __forceinline__ void shrink_u(float (&vx)[K], float (&vy)[K], float t, const float *wc)
{
    if (UN == VOMT_U_L12) {
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const float f = shrink2_factor(vx[c] * vx[c] + vy[c] * vy[c], t);
            vx[c] *= f;
            vy[c] *= f;
        }
    } else if (UN == VOMT_U_L2) {
        float s2 = 0.0f;
#pragma unroll
        for (int c = 0; c < K; ++c) s2 += wc[c] * (vx[c] * vx[c] + vy[c] * vy[c]);
        const float f = shrink2_factor(s2, t);
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
        const float f = shrink2_factor(s2, t);
#pragma unroll
        for (int e = 0; e < LK; ++e) x[e] *= f;
    }
}

template <int K>
struct LKT {
    static constexpr int v = K * (K - 1) / 2 > 0 ? K * (K - 1) / 2 : 1;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}

struct TmaMapsDev {
    CUtensorMap phi;    // state, box TXP x (TY + 2) x K at plane 0
    CUtensorMap u;      // state, box TXP x (TY + 1) x K at planes K (u_x) and 2K (u_y)
    CUtensorMap w;      // state, box TX x TY x l at plane 3K
    CUtensorMap b;      // rho1 - rho0, box TX x TY x K
};

template <int K, int UN, int WN>
__global__ void __launch_bounds__(NTH) k_step_tma(const __grid_constant__ TmaMapsDev maps, float *__restrict__ out,
                                                  OpDev g, StepDev s, DevStatus *st)
{
    constexpr int LK = LKT<K>::v;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar;
    const int n = s.n, l = g.l;
    const TmaSmem SL = tma_smem(K, l);
    float *sphi = (float *)(smem + SL.phi), *sux = (float *)(smem + SL.ux), *suy = (float *)(smem + SL.uy);
    float *sw = (float *)(smem + SL.w), *sb = (float *)(smem + SL.b);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.x;
    const uint32_t mb = smem_u32(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // launched as a programmatic dependent of the previous step or check: everything
    // above ran while that kernel drained; from here on its writes are complete and
    // visible (a no-op for a normal launch)
    cudaGridDependencySynchronize();
    if (st->stop) return;
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(SL.bytes) : "memory");
        tma_load_3d(smem_u32(sphi), &maps.phi, x0 - 4, y0 - 1, 0, mb);
        tma_load_3d(smem_u32(sux), &maps.u, x0 - 4, y0 - 1, K, mb);
        tma_load_3d(smem_u32(suy), &maps.u, x0 - 4, y0 - 1, 2 * K, mb);
        if (l > 0) tma_load_3d(smem_u32(sw), &maps.w, x0, y0, 3 * K, mb);
        tma_load_3d(smem_u32(sb), &maps.b, x0, y0, 0, mb);
    }
    // bounded wait for the copies (phase 0)
    {
        uint32_t done = 0;
        for (uint32_t it = 0; !done; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(done)
                : "r"(mb), "r"(0u)
                : "memory");
            if (!done && it >= (1u << 22)) {
                st->error = VOMT_ERR_BARRIER_TIMEOUT;
                st->stop = 1;
                return;          // this block's output is not written; the solve reports the error
            }
        }
    }
    const size_t nn = (size_t)n * n;
    const int PL = (TY + 2) * TXP, UL = (TY + 1) * TXP, WL = TY * TX;
    const float mu = s.mu, ih = s.ih;
    const float su = s.reg ? s.su : 1.0f, tu = s.reg ? mu * s.su : mu;
    const int tx = tid % TX, tyb = tid / TX;
#pragma unroll 1
    for (int r = 0; r < ROWS; ++r) {
        const int ty = tyb + r * (NTH / TX);
        const int i = x0 + tx, j = y0 + ty;
        if (i >= n || j >= n) continue;
        const bool hR = i < n - 1, hU = j < n - 1, hL = i > 0, hD = j > 0;
        // shared-array offsets of (i, j): phi / u tiles start at (x0 - 4, y0 - 1)
        const int oP = (ty + 1) * TXP + tx + 4;
        float pc[K], pr[K], pu[K], pl[K], plu[K], pd[K], prd[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const float *P = sphi + c * PL + oP;
            pc[c] = P[0];
            pr[c] = hR ? P[1] : 0.0f;
            pu[c] = hU ? P[TXP] : 0.0f;
            pl[c] = hL ? P[-1] : 0.0f;
            plu[c] = (hL && hU) ? P[TXP - 1] : 0.0f;
            pd[c] = hD ? P[-TXP] : 0.0f;
            prd[c] = (hR && hD) ? P[1 - TXP] : 0.0f;
        }
        float ux0[K], uy0[K], vx[K], vy[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            ux0[c] = sux[c * UL + oP];
            uy0[c] = suy[c * UL + oP];
            vx[c] = ux0[c] + (hR ? mu * (ih * (pr[c] - pc[c])) : 0.0f);
            vy[c] = uy0[c] + (hU ? mu * (ih * (pu[c] - pc[c])) : 0.0f);
            if (s.reg) { vx[c] *= su; vy[c] *= su; }
        }
        shrink_u<K, UN>(vx, vy, tu, g.wc);
        float lx[K], ly[K], lx0[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            lx0[c] = hL ? sux[c * UL + oP - 1] : 0.0f;
            const float ly0 = hL ? suy[c * UL + oP - 1] : 0.0f;
            lx[c] = lx0[c] + (hL ? mu * (ih * (pc[c] - pl[c])) : 0.0f);
            ly[c] = ly0 + ((hL && hU) ? mu * (ih * (plu[c] - pl[c])) : 0.0f);
            if (s.reg) { lx[c] *= su; ly[c] *= su; }
        }
        shrink_u<K, UN>(lx, ly, tu, g.wc);
        float dx[K], dy[K], dy0[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const float dx0 = hD ? sux[c * UL + oP - TXP] : 0.0f;
            dy0[c] = hD ? suy[c * UL + oP - TXP] : 0.0f;
            dx[c] = dx0 + ((hR && hD) ? mu * (ih * (prd[c] - pd[c])) : 0.0f);
            dy[c] = dy0[c] + (hD ? mu * (ih * (pc[c] - pd[c])) : 0.0f);
            if (s.reg) { dx[c] *= su; dy[c] *= su; }
        }
        shrink_u<K, UN>(dx, dy, tu, g.wc);
        const int oW = ty * TX + tx;
        float w0[LK], wx[LK];
#pragma unroll
        for (int e = 0; e < LK; ++e) {
            if (e < l) {
                w0[e] = sw[e * WL + oW];
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
        shrink_w<LK, WN>(wx, l, s.reg ? s.alpha * s.nu * s.sw : s.alpha * s.nu, g.we);
        float rr[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const float bxc = 2.0f * vx[c] - ux0[c];
            const float byc = 2.0f * vy[c] - uy0[c];
            const float bxl = hL ? 2.0f * lx[c] - lx0[c] : 0.0f;
            const float byd = hD ? 2.0f * dy[c] - dy0[c] : 0.0f;
            rr[c] = ih * ((bxc - bxl) + (byc - byd)) + sb[c * WL + oW];
        }
#pragma unroll
        for (int e = 0; e < LK; ++e) {
            const float v = 2.0f * wx[e] - w0[e];
#pragma unroll
            for (int c = 0; c < K; ++c) rr[c] -= g.Dv[c][e] * v;
        }
        const size_t p = (size_t)j * n + i;
        float *ophi = out, *oux = out + (size_t)K * nn, *ouy = out + (size_t)2 * K * nn, *ow = out + (size_t)3 * K * nn;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            ophi[c * nn + p] = pc[c] + s.tau * rr[c];
            oux[c * nn + p] = vx[c];
            ouy[c * nn + p] = vy[c];
        }
#pragma unroll
        for (int e = 0; e < LK; ++e)
            if (e < l) ow[e * nn + p] = wx[e];
    }
}

using TmaKernel = void (*)(TmaMapsDev, float *, OpDev, StepDev, DevStatus *);

template <int K>
TmaKernel pick_norms_tma(int un, int wn)
{
    if constexpr (K == 3) {
        if (un == VOMT_U_NUC)
            return wn == VOMT_W_L1 ? k_step_tma<K, 3, 0> : (wn == VOMT_W_L2 ? k_step_tma<K, 3, 1> : k_step_tma<K, 3, 2>);
        if (wn == VOMT_W_NUC) return un == VOMT_U_L2 ? k_step_tma<K, 1, 2> : k_step_tma<K, 2, 2>;
    }
    if (un == VOMT_U_L12) return wn == VOMT_W_L1 ? k_step_tma<K, 0, 0> : k_step_tma<K, 0, 1>;
    if (un == VOMT_U_L2) return wn == VOMT_W_L1 ? k_step_tma<K, 1, 0> : k_step_tma<K, 1, 1>;
    return wn == VOMT_W_L1 ? k_step_tma<K, 2, 0> : k_step_tma<K, 2, 1>;
}

TmaKernel pick_tma(int k, int un, int wn)
{
    switch (k) {
        case 1: return pick_norms_tma<1>(un, wn);
        case 2: return pick_norms_tma<2>(un, wn);
        case 3: return pick_norms_tma<3>(un, wn);
        case 4: return pick_norms_tma<4>(un, wn);
        default: return nullptr;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

bool encode(CUtensorMap *m, const float *base, int n, int planes, int bx, int by, int bz)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)n * 4, (cuuint64_t)n * n * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct TmaPlan {
    TmaMapsDev maps[2];        // reading state 0 / state 1
    TmaKernel kern;
    int smem;
};

bool tma_step_supported(int n, int k, int l, int un, int wn)
{
    if (n < 64 || n % 4 != 0 || n >= (1 << 20) || k > 4) return false;
    // Below about 16 MB of iterate the plain step (four times the blocks) is as fast;
    // so it is while the 64 x 16 tiles fill fewer than two blocks on each of the 152
    // SMs (512^2 at k = 3: 256 tiles).  Measured on GB300, 3000 iterations: 1024^2 at
    // k = 1 10.7 -> 10.0 us, 768^2 at k = 3 15.2 -> 14.2 us with TMA; 512^2 at k = 3
    // 7.9 us either way.
    if ((double)n * n * (7 * k + 2 * l) * 4.0 < 16.0 * 1024 * 1024) return false;
    if (((n + TX - 1) / TX) * ((n + TY - 1) / TY) < 2 * 152) return false;
    if (tma_smem(k, l).total > 110 * 1024) return false;     // two blocks per SM at least
    if (!pick_tma(k, un, wn)) return false;
    return encode_fn() != nullptr;
}

TmaPlan *tma_plan_create(int n, int k, int l, int un, int wn, const float *state0, const float *state1, const float *b)
{
    TmaPlan *pl = new TmaPlan();
    const float *st[2] = {state0, state1};
    const int planes = 3 * k + l;
    bool ok = true;
    for (int q = 0; q < 2 && ok; ++q) {
        ok = encode(&pl->maps[q].phi, st[q], n, planes, TXP, TY + 2, k) &&
             encode(&pl->maps[q].u, st[q], n, planes, TXP, TY + 1, k) &&
             (l == 0 || encode(&pl->maps[q].w, st[q], n, planes, TX, TY, l)) &&
             encode(&pl->maps[q].b, b, n, k, TX, TY, k);
        if (l == 0) memset(&pl->maps[q].w, 0, sizeof(CUtensorMap));
    }
    pl->kern = pick_tma(k, un, wn);
    pl->smem = tma_smem(k, l).total;
    if (ok && pl->kern)
        ok = cudaFuncSetAttribute((const void *)pl->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pl->smem) ==
             cudaSuccess;
    if (!ok || !pl->kern) {
        delete pl;
        return nullptr;
    }
    return pl;
}

void tma_plan_destroy(TmaPlan *pl) { delete pl; }

void tma_launch_step(const TmaPlan *pl, int in_state, float *out_state, const OpDev &g, const StepDev &s,
                     DevStatus *st, cudaStream_t stream, bool pdl)
{
    const dim3 grd((s.n + TX - 1) / TX, (s.n + TY - 1) / TY);
    if (!pdl) {
        pl->kern<<<grd, NTH, pl->smem, stream>>>(pl->maps[in_state], out_state, g, s, st);
        return;
    }
    launch_pdl(pl->kern, grd, dim3(NTH), pl->smem, stream, pl->maps[in_state], out_state, g, s, st);
}

}  // namespace vomt
