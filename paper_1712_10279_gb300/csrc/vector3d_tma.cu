// 3-D fused iteration (Appendix A's discretization with a third direction,
// the step of Section 7.2) with its inputs staged by the tensor memory
// accelerator.
//
// A block owns a 32 x 8 column of the grid and marches up a chunk of z.  Each
// plane's inputs arrive in a ring of NS shared-memory stages by six 4-D
// cp.async.bulk.tensor copies issued by one thread on the stage's mbarrier:
// phi with a one-cell halo on every side (x0-4 .. x0+35 so that the box starts
// on a 16-byte boundary, y0-1 .. y0+8), u_x, u_y and u_z with the x0-1 column
// and the y0-1 row (x0-4 .. x0+31, the tile's upwind neighbours), w and b on the
// tile.  Plane z + NS - 1 is issued while plane z is computed, so NS - 2 planes
// are in flight per block without tying up registers.  Per plane each thread computes
// u' at its point once; the tile's x0-1 column and y0-1 row are recomputed;
// the x and y components of 2u' - u meet their downwind neighbours through
// shared memory, the z component is carried in a register to the next plane
// (the chunk's first plane recomputes it from global memory).
//
// TMA rules honoured here: the tensors are 4-D (x, y, z, volume) with strides
// 4n, 4n^2, 4n^3 bytes, so n must be a multiple of 4; every box starts at an x
// that is a multiple of 4; loads may start at negative or out-of-range
// coordinates and then read zeros, which the stencil masks anyway.  Every wait
// on an mbarrier is bounded: one that runs out marks the solve failed, the
// block drains its copies in flight (again bounded) and returns.
#include <math.h>
#include <string.h>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>

#include "internal.h"
#include "pdhg_device.cuh"
#include "vector3d.cuh"
#include "vector3d_tma.h"

namespace vomt {
namespace {

using namespace v3;

constexpr int BXH = MX + 8;          // phi box columns x0-4 .. x0+35 (x0+32 is the last x+1)
constexpr int BXU = MX + 4;          // u box columns x0-4 .. x0+31 (x0-1 is the upwind column)
constexpr int BYP = MY + 2;          // phi rows y0-1 .. y0+8
constexpr int BYU = MY + 1;          // u rows y0-1 .. y0+7
constexpr uint32_t kSpins = 1u << 22;

__host__ __device__ inline int al128(int x) { return (x + 127) & ~127; }

struct Stage3 {
    int phi, ux, uy, uz, w, b, size;
    unsigned bytes_all, bytes_phi;     // bytes a full plane / a phi-only plane delivers
};

__host__ __device__ inline Stage3 stage3(int K, int l)
{
    Stage3 S;
    int o = 0;
    S.phi = o; o += al128(K * BYP * BXH * 4);
    S.ux = o; o += al128(K * BYU * BXU * 4);
    S.uy = o; o += al128(K * BYU * BXU * 4);
    S.uz = o; o += al128(K * BYU * BXU * 4);
    S.w = o; o += al128((l > 0 ? l : 1) * MY * MX * 4);
    S.b = o; o += al128(K * MY * MX * 4);
    S.size = o;
    S.bytes_phi = (unsigned)(K * BYP * BXH * 4);
    S.bytes_all = S.bytes_phi + (unsigned)(3 * K * BYU * BXU * 4 + l * MY * MX * 4 + K * MY * MX * 4);
    return S;
}

// stages: planes z and z+1 in use, the rest in flight.  Four for K <= 3 channels
// (two blocks per SM; three stages would fit three blocks per SM but measured
// slower, the copies then land too late), three for K = 4 (two blocks per SM),
// four for K = 5, 6 (one block per SM: 3 x 3 matrix fields are 6 channels).
__host__ __device__ constexpr int nstages(int K) { return K == 4 ? 3 : 4; }
__host__ __device__ constexpr int blocks_per_sm(int K) { return K <= 4 ? 2 : 1; }
// double-buffered exchange arrays (one barrier per plane) where they fit: not at K = 4,
// whose two blocks per SM leave no room
__host__ __device__ constexpr bool dbuf(int K) { return K != 4; }
// the tile's MT threads plus two halo warps: the y0-1 row (32 lanes) and the x0-1
// column (MY lanes) of 2u' - u, computed beside the tile instead of by tile warps
constexpr int HT = 64, NT3 = MT + HT;

__host__ __device__ inline int sb_floats(int K) { return K * MY * (MX + 1) + K * (MY + 1) * MX; }

__host__ __device__ inline int smem3(int K, int l)
{
    return nstages(K) * stage3(K, l).size + 4 * sb_floats(K) * (dbuf(K) ? 2 : 1);
}

struct Maps3 {
    CUtensorMap phi;    // state volumes, box BXH x BYP x 1 x K
    CUtensorMap u;      // state volumes, box BXU x BYU x 1 x K (at volumes K, 2K, 3K)
    CUtensorMap w;      // state volumes, box MX x MY x 1 x l (at volume 4K)
    CUtensorMap b;      // rho1 - rho0, box MX x MY x 1 x K
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int v,
                                            uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(v), "r"(mbar)
        : "memory");
}

// bounded wait for the completion of phase `parity` of the mbarrier at `mb`
__device__ __forceinline__ bool wait_phase(uint32_t mb, uint32_t parity, uint32_t spins)
{
    for (uint32_t it = 0; it < spins; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mb), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int K, int UN, int WN>
__global__ void __launch_bounds__(NT3, blocks_per_sm(K)) k_step3t(const __grid_constant__ Maps3 maps, const float *__restrict__ in,
                                                 S3Out out, OpDev g, StepDev s, DevStatus *st, int zc)
{
    constexpr int NS = nstages(K), LK = LK3<K>::v;
    constexpr int PL = BYP * BXH, UL = BYU * BXU, WL = MY * MX;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar[NS];
    __shared__ int abort_flag;
    const int n = s.n, l = g.l;
    const Stage3 SL = stage3(K, l);
    float *const sb0 = (float *)(smem + NS * SL.size);
    const size_t m = (size_t)n * n * n, nn = (size_t)n * n;
    const int tid = threadIdx.x, tx = tid % MX, ty = tid / MX;
    const bool tile = tid < MT;                 // else a halo thread: ht < MX row, < MX + MY column
    const int ht = tid - MT;
    const int x0 = blockIdx.x * MX, y0 = blockIdx.y * MY;
    const int z0 = blockIdx.z * zc, z1 = min(n, z0 + zc), zlast = min(z1, n - 1);
    const int x = x0 + tx, y = y0 + ty;
    const bool inb = tile && x < n && y < n;
    const bool hx = x < n - 1, hy = y < n - 1, lx = x > 0, ly = y > 0;
    const float mi = s.mu * s.ih;
    if (tid == 0) {
        for (int q = 0; q < NS; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[q])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    // launched as a programmatic dependent of the previous step or check: the setup
    // above ran while that kernel drained; from here on its writes are complete and
    // visible (a no-op for a normal launch)
    cudaGridDependencySynchronize();
    if (st->stop) return;
    // plane p lives in stage (p - z0) % NS; its use of that stage has phase parity ((p - z0) / NS) & 1
    auto issue = [&](int p) {
        const int q = (p - z0) % NS;
        unsigned char *base = smem + q * SL.size;
        const uint32_t mb = smem_u32(&mbar[q]);
        const bool phi_only = p == z1;        // plane z1 serves only as the z+1 plane of step z1-1
        const unsigned bytes = phi_only ? SL.bytes_phi : SL.bytes_all;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
        tma_load_4d(smem_u32(base + SL.phi), &maps.phi, x0 - 4, y0 - 1, p, 0, mb);
        if (!phi_only) {
            tma_load_4d(smem_u32(base + SL.ux), &maps.u, x0 - 4, y0 - 1, p, K, mb);
            tma_load_4d(smem_u32(base + SL.uy), &maps.u, x0 - 4, y0 - 1, p, 2 * K, mb);
            tma_load_4d(smem_u32(base + SL.uz), &maps.u, x0 - 4, y0 - 1, p, 3 * K, mb);
            if (l > 0) tma_load_4d(smem_u32(base + SL.w), &maps.w, x0, y0, p, 4 * K, mb);
            tma_load_4d(smem_u32(base + SL.b), &maps.b, x0, y0, p, 0, mb);
        }
    };
    auto wait_plane = [&](int p, uint32_t spins) {
        return wait_phase(smem_u32(&mbar[(p - z0) % NS]), (uint32_t)(((p - z0) / NS) & 1), spins);
    };
    if (tid == 0)
        for (int p = z0; p < z0 + NS - 1 && p <= zlast; ++p) issue(p);

    // 2u'_z - u_z at (x, y, z0 - 1), from global memory
    float cz[K];
#pragma unroll
    for (int c = 0; c < K; ++c) cz[c] = 0.0f;
    if (z0 > 0 && inb) {
        const size_t p = (size_t)(z0 - 1) * nn + (size_t)y * n + x;
        float ax[K], ay[K], az[K], az0[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const float *P = in + c * m + p;
            const float pc = __ldg(P), px = hx ? __ldg(P + 1) : 0.0f, py = hy ? __ldg(P + n) : 0.0f;
            const float pz = __ldg(P + nn);
            az0[c] = __ldg(in + (3 * K + c) * m + p);
            ax[c] = upre(__ldg(in + (K + c) * m + p), px, pc, hx, mi);
            ay[c] = upre(__ldg(in + (2 * K + c) * m + p), py, pc, hy, mi);
            az[c] = upre(az0[c], pz, pc, true, mi);
        }
        shrink_u3<K, UN>(ax, ay, az, s.mu, g.wc);
#pragma unroll
        for (int c = 0; c < K; ++c) cz[c] = 2.0f * az[c] - az0[c];
    }

    const int oP = (ty + 1) * BXH + tx + 4;     // (x, y) in the phi box
    const int oU = (ty + 1) * BXU + tx + 4;     // (x, y) in the u boxes
    const int oT = ty * MX + tx;                // (x, y) in the w and b boxes
    for (int z = z0; z < z1; ++z) {
        const bool hz = z < n - 1, lz = z > 0;
        float *sbx = sb0 + (dbuf(K) ? (z & 1) * sb_floats(K) : 0);
        float *sby = sbx + K * MY * (MX + 1);
        bool ok = wait_plane(z, kSpins);
        if (ok && hz) ok = wait_plane(z + 1, kSpins);
        if (!ok) abort_flag = 1;
        const unsigned char *S0 = smem + ((z - z0) % NS) * SL.size;
        const unsigned char *S1 = smem + ((z + 1 - z0) % NS) * SL.size;
        const float *P0 = (const float *)(S0 + SL.phi), *P1 = (const float *)(S1 + SL.phi);
        const float *Ux = (const float *)(S0 + SL.ux), *Uy = (const float *)(S0 + SL.uy);
        const float *Uz = (const float *)(S0 + SL.uz);
        const float *W0 = (const float *)(S0 + SL.w), *B0 = (const float *)(S0 + SL.b);
        // tile threads: own u', 2u' - u and w'; halo threads: the upwind row and column
        float pc[K], vx[K], vy[K], vz[K], ux0[K], uy0[K], uz0[K], bb[K];
        float w0[LK], wx[LK];
        if (tile) {
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const float *P = P0 + c * PL + oP;
            pc[c] = P[0];
            ux0[c] = Ux[c * UL + oU];
            uy0[c] = Uy[c * UL + oU];
            uz0[c] = Uz[c * UL + oU];
            vx[c] = upre(ux0[c], P[1], pc[c], hx, mi);
            vy[c] = upre(uy0[c], P[BXH], pc[c], hy, mi);
            vz[c] = upre(uz0[c], P1[c * PL + oP], pc[c], hz, mi);
            bb[c] = B0[c * WL + oT];
        }
        shrink_u3<K, UN>(vx, vy, vz, s.mu, g.wc);
#pragma unroll
        for (int c = 0; c < K; ++c) {
            sbx[(c * MY + ty) * (MX + 1) + tx + 1] = 2.0f * vx[c] - ux0[c];
            sby[(c * (MY + 1) + ty + 1) * MX + tx] = 2.0f * vy[c] - uy0[c];
        }
        // w' at the point
#pragma unroll
        for (int e = 0; e < LK; ++e) {
            if (e < l) {
                w0[e] = W0[e * WL + oT];
                float ge = 0.0f;
#pragma unroll
                for (int c = 0; c < K; ++c) ge += g.G[e][c] * pc[c];
                wx[e] = w0[e] + s.nu * ge;
            } else {
                w0[e] = 0.0f;
                wx[e] = 0.0f;
            }
        }
        shrink_w3<LK, WN>(wx, l, s.alpha * s.nu, g.we);
        } else {
            // the tile's y0-1 row (halo lanes 0..MX-1) and x0-1 column (lanes MX..MX+MY-1)
            int hxp = -1, hyp = -1, o = 0, ou = 0;
            if (ht < MX) {
                if (y0 > 0 && x0 + ht < n) { hxp = x0 + ht; hyp = y0 - 1; o = ht + 4; ou = ht + 4; }
            } else if (ht < MX + MY) {
                if (x0 > 0 && y0 + ht - MX < n) {
                    hxp = x0 - 1;
                    hyp = y0 + ht - MX;
                    o = (ht - MX + 1) * BXH + 3;
                    ou = (ht - MX + 1) * BXU + 3;
                }
            }
            if (hxp >= 0) {
                const bool ax_in = hxp < n - 1, ay_in = hyp < n - 1;
                float ax[K], ay[K], az[K], a0x[K], a0y[K];
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const float *P = P0 + c * PL + o;
                    a0x[c] = Ux[c * UL + ou];
                    a0y[c] = Uy[c * UL + ou];
                    ax[c] = upre(a0x[c], P[1], P[0], ax_in, mi);
                    ay[c] = upre(a0y[c], P[BXH], P[0], ay_in, mi);
                    az[c] = upre(Uz[c * UL + ou], P1[c * PL + o], P[0], hz, mi);
                }
                shrink_u3<K, UN>(ax, ay, az, s.mu, g.wc);
                if (ht < MX) {
#pragma unroll
                    for (int c = 0; c < K; ++c) sby[(c * (MY + 1)) * MX + ht] = 2.0f * ay[c] - a0y[c];
                } else {
#pragma unroll
                    for (int c = 0; c < K; ++c) sbx[(c * MY + (ht - MX)) * (MX + 1)] = 2.0f * ax[c] - a0x[c];
                }
            }
        }
        __syncthreads();
        if (abort_flag) {
            if (tid == 0) {
                st->error = VOMT_ERR_BARRIER_TIMEOUT;
                st->stop = 1;
                for (int p = z; p <= min(z + NS - 2, zlast); ++p) wait_plane(p, 1u << 16);   // drain
            }
            return;
        }
        // every thread is past plane z - 1: its stage takes plane z + NS - 1
        if (tid == 0 && z + NS - 1 <= zlast) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(z + NS - 1);
        }
        if (tile) {
        // phi' = phi + tau (div ubar + div_G wbar + rho1 - rho0)
        float r[K];
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const float bxc = 2.0f * vx[c] - ux0[c], byc = 2.0f * vy[c] - uy0[c], bzc = 2.0f * vz[c] - uz0[c];
            const float bxl = lx ? sbx[(c * MY + ty) * (MX + 1) + tx] : 0.0f;
            const float byl = ly ? sby[(c * (MY + 1) + ty) * MX + tx] : 0.0f;
            const float bzl = lz ? cz[c] : 0.0f;
            r[c] = s.ih * ((bxc - bxl) + (byc - byl) + (bzc - bzl)) + bb[c];
            cz[c] = bzc;
        }
#pragma unroll
        for (int e = 0; e < LK; ++e) {
            const float v = 2.0f * wx[e] - w0[e];
#pragma unroll
            for (int c = 0; c < K; ++c) r[c] -= g.Dv[c][e] * v;
        }
        if (inb) {
            const size_t p = (size_t)z * nn + (size_t)y * n + x;
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
                if (e < l) out.w[e * m + p] = wx[e];
        }
        }
        // with one exchange buffer the next plane's writes wait for this plane's reads
        if constexpr (!dbuf(K)) __syncthreads();
    }
}

using Kern3 = void (*)(const Maps3, const float *, S3Out, OpDev, StepDev, DevStatus *, int);

template <int K>
Kern3 pick_norms3t(int un, int wn)
{
    if constexpr (K == 3 || K == 6) {          // nuclear norms: compact 2 x 2 and 3 x 3 matrices
        if (un == VOMT_U_NUC)
            return wn == VOMT_W_L1 ? k_step3t<K, 3, 0> : (wn == VOMT_W_L2 ? k_step3t<K, 3, 1> : k_step3t<K, 3, 2>);
        if (wn == VOMT_W_NUC) return un == VOMT_U_L2 ? k_step3t<K, 1, 2> : k_step3t<K, 2, 2>;
    }
    if (un == VOMT_U_L12) return wn == VOMT_W_L1 ? k_step3t<K, 0, 0> : k_step3t<K, 0, 1>;
    if (un == VOMT_U_L2) return wn == VOMT_W_L1 ? k_step3t<K, 1, 0> : k_step3t<K, 1, 1>;
    return wn == VOMT_W_L1 ? k_step3t<K, 2, 0> : k_step3t<K, 2, 1>;
}

Kern3 pick3t(int k, int un, int wn)
{
    if (un < 0 || un > 3 || wn < 0 || wn > 2) return nullptr;
    if ((un == VOMT_U_NUC || wn == VOMT_W_NUC) && k != 3 && k != 6) return nullptr;
    switch (k) {
        case 1: return pick_norms3t<1>(un, wn);
        case 2: return pick_norms3t<2>(un, wn);
        case 3: return pick_norms3t<3>(un, wn);
        case 4: return pick_norms3t<4>(un, wn);
        case 5: return pick_norms3t<5>(un, wn);
        case 6: return pick_norms3t<6>(un, wn);
        default: return nullptr;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn3()
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

// 4-D map (x, y, z, volume) over `vols` n^3 volumes at base; box bx x by x 1 x bv
bool encode4(CUtensorMap *map, const float *base, int n, int vols, int bx, int by, int bv)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn3();
    if (!fn) return false;
    const cuuint64_t nn = (cuuint64_t)n;
    const cuuint64_t dims[4] = {nn, nn, nn, (cuuint64_t)vols};
    const cuuint64_t strides[3] = {nn * 4, nn * nn * 4, nn * nn * nn * 4};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)bv};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct Tma3Plan {
    Maps3 maps[2];       // reading state 0 / state 1
    const float *in[2];
    Kern3 kern;
    int smem;
};

bool tma3_supported(int n, int k, int l, int un, int wn)
{
    if (n < BXH || n % 4 != 0 || n > 1024) return false;
    if (!pick3t(k, un, wn)) return false;
    // the ring fits blocks_per_sm blocks of one SM's 228 KB (1 KB reserved per block)
    if (smem3(k, l) > (k <= 4 ? 110 : 224) * 1024) return false;
    return encode_fn3() != nullptr;
}

Tma3Plan *tma3_plan_create(int n, int k, int l, int un, int wn, const float *state0, const float *state1,
                           const float *b)
{
    Tma3Plan *pl = new Tma3Plan();
    const float *st[2] = {state0, state1};
    const int vols = 4 * k + l;
    bool ok = true;
    for (int q = 0; q < 2 && ok; ++q) {
        pl->in[q] = st[q];
        ok = encode4(&pl->maps[q].phi, st[q], n, vols, BXH, BYP, k) &&
             encode4(&pl->maps[q].u, st[q], n, vols, BXU, BYU, k) &&
             (l == 0 || encode4(&pl->maps[q].w, st[q], n, vols, MX, MY, l)) &&
             encode4(&pl->maps[q].b, b, n, k, MX, MY, k);
        if (l == 0) memset(&pl->maps[q].w, 0, sizeof(CUtensorMap));
    }
    pl->kern = pick3t(k, un, wn);
    pl->smem = smem3(k, l);
    if (ok && pl->kern)
        ok = cudaFuncSetAttribute((const void *)pl->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pl->smem) ==
             cudaSuccess;
    if (!ok || !pl->kern) {
        delete pl;
        return nullptr;
    }
    return pl;
}

void tma3_plan_destroy(Tma3Plan *pl) { delete pl; }

void tma3_launch_step(const Tma3Plan *pl, int in_state, S3Out out, const OpDev &g, const StepDev &s, DevStatus *st,
                      int zc, cudaStream_t stream)
{
    const int n = s.n;
    const dim3 grd((n + MX - 1) / MX, (n + MY - 1) / MY, (n + zc - 1) / zc);
    launch_pdl(pl->kern, grd, dim3(NT3), pl->smem, stream, pl->maps[in_state], pl->in[in_state], out, g, s, st, zc);
}

}  // namespace vomt
