// Matrix OMT (Section 4, algorithm of Section 7.3) on the vector engines.
//
// In compact coordinates a real symmetric k x k field is k(k+1)/2 channels
// (diagonal first, then the entries above it) and a skew one is k(k-1)/2 flux
// entries per L_s.  With off-diagonal entries weighted 2 in every inner product,
// the Hilbert-Schmidt geometry of Section 4 is reproduced exactly, the spatial
// gradient and divergence act channel by channel, and grad_L / div_L become one
// per-point linear map and its weighted adjoint (built on the host by
// quantum_to_op).  The iteration is then the one the vector engines run, so the
// matrix path adds only the conversions between full and compact storage and
// the input checks.
#include <math.h>
#include <string.h>

#include <vector>

#include "internal.h"

namespace vomt {
namespace {

// entry (a, b) of compact channel c (symmetric) / flux entry j (skew, a < b)
struct PairTable {
    int k, K, ks;
    int sa[KMAX], sb[KMAX];
    int ka[3], kb[3];
};

PairTable make_pairs(int k)
{
    PairTable t;
    memset(&t, 0, sizeof t);
    t.k = k;
    t.K = k * (k + 1) / 2;
    t.ks = k * (k - 1) / 2;
    for (int a = 0; a < k; ++a) { t.sa[a] = a; t.sb[a] = a; }
    int c = k, j = 0;
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b) {
            t.sa[c] = a; t.sb[c] = b; ++c;
            t.ka[j] = a; t.kb[j] = b; ++j;
        }
    return t;
}

// per block: sum tr Lam0, sum tr Lam1, min diagonal entry, max |X_ab - X_ba|,
// max |X_ab|, count of non-finite entries
__global__ void k_mat_validate(size_t nn, int k, const float *__restrict__ L0, const float *__restrict__ L1,
                               double *__restrict__ out)
{
    double t0 = 0.0, t1 = 0.0, mind = 1e300, asym = 0.0, mabs = 0.0, bad = 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x) {
        for (int side = 0; side < 2; ++side) {
            const float *X = side ? L1 : L0;
            for (int a = 0; a < k; ++a)
                for (int b = 0; b < k; ++b) {
                    const float v = X[(a * k + b) * nn + q];
                    if (!isfinite(v)) { bad += 1.0; continue; }
                    mabs = fmax(mabs, (double)fabsf(v));
                    if (a == b) {
                        if (side) t1 += v; else t0 += v;
                        mind = fmin(mind, (double)v);
                    } else if (a < b) {
                        asym = fmax(asym, (double)fabsf(v - X[(b * k + a) * nn + q]));
                    }
                }
        }
    }
    __shared__ double sh[6][256];
    sh[0][threadIdx.x] = t0; sh[1][threadIdx.x] = t1; sh[2][threadIdx.x] = mind;
    sh[3][threadIdx.x] = asym; sh[4][threadIdx.x] = mabs; sh[5][threadIdx.x] = bad;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            const int o = threadIdx.x + off;
            sh[0][threadIdx.x] += sh[0][o];
            sh[1][threadIdx.x] += sh[1][o];
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][o]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][o]);
            sh[4][threadIdx.x] = fmax(sh[4][threadIdx.x], sh[4][o]);
            sh[5][threadIdx.x] += sh[5][o];
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) out[blockIdx.x * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

// full symmetric planes -> compact channels (the symmetric part), `groups` fields
// of k*k planes each (e.g. 2 for U = (U_x, U_y))
__global__ void k_sym_to_compact(size_t nn, PairTable t, int groups, const float *__restrict__ full,
                                 float *__restrict__ comp)
{
    const int kk = t.k * t.k;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x)
        for (int g = 0; g < groups; ++g)
            for (int c = 0; c < t.K; ++c) {
                const int a = t.sa[c], b = t.sb[c];
                const float *F = full + (size_t)g * kk * nn;
                comp[((size_t)g * t.K + c) * nn + q] = 0.5f * (F[(a * t.k + b) * nn + q] + F[(b * t.k + a) * nn + q]);
            }
}

// full planes of N skew matrices -> compact entries above the diagonal (the skew part)
__global__ void k_skew_to_compact(size_t nn, PairTable t, int N, const float *__restrict__ full, float *__restrict__ comp)
{
    const int kk = t.k * t.k;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x)
        for (int s = 0; s < N; ++s)
            for (int j = 0; j < t.ks; ++j) {
                const int a = t.ka[j], b = t.kb[j];
                const float *F = full + (size_t)s * kk * nn;
                comp[((size_t)s * t.ks + j) * nn + q] = 0.5f * (F[(a * t.k + b) * nn + q] - F[(b * t.k + a) * nn + q]);
            }
}

__global__ void k_compact_to_sym(size_t nn, PairTable t, int groups, const float *__restrict__ comp, float *__restrict__ full)
{
    const int kk = t.k * t.k;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x)
        for (int g = 0; g < groups; ++g)
            for (int c = 0; c < t.K; ++c) {
                const int a = t.sa[c], b = t.sb[c];
                const float v = comp[((size_t)g * t.K + c) * nn + q];
                float *F = full + (size_t)g * kk * nn;
                F[(a * t.k + b) * nn + q] = v;
                F[(b * t.k + a) * nn + q] = v;
            }
}

__global__ void k_compact_to_skew(size_t nn, PairTable t, int N, const float *__restrict__ comp, float *__restrict__ full)
{
    const int kk = t.k * t.k;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x)
        for (int s = 0; s < N; ++s) {
            float *F = full + (size_t)s * kk * nn;
            for (int a = 0; a < t.k; ++a) F[(a * t.k + a) * nn + q] = 0.0f;
            for (int j = 0; j < t.ks; ++j) {
                const int a = t.ka[j], b = t.kb[j];
                const float v = comp[((size_t)s * t.ks + j) * nn + q];
                F[(a * t.k + b) * nn + q] = v;
                F[(b * t.k + a) * nn + q] = -v;
            }
        }
}

// Table 3's tuned tau: 10 for the 32^2 and 64^2 grids, 30 for 128^2, 60 for 256^2
double default_tau_matrix(int n) { return n <= 64 ? 10.0 : (n <= 128 ? 30.0 : 60.0); }

// ---- complex Hermitian fields (k = 2): planar (re, im) arrays <-> real compact
// coordinates of hermitian_to_op (diagonal; Re, Im above it), padded to K
// channels with zeros.  `full` holds `groups` fields of [re: k*k planes][im: k*k planes].

// per block: sum Re tr Lam0, sum Re tr Lam1, min Re diagonal, max |X_ab - conj X_ba|
// (and |Im X_aa|), max |X|, count of non-finite entries
__global__ void k_herm_validate(size_t nn, int k, const float *__restrict__ L0, const float *__restrict__ L1,
                                double *__restrict__ out)
{
    const int kk = k * k;
    double t0 = 0.0, t1 = 0.0, mind = 1e300, asym = 0.0, mabs = 0.0, bad = 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x) {
        for (int side = 0; side < 2; ++side) {
            const float *re = side ? L1 : L0, *im = re + (size_t)kk * nn;
            for (int a = 0; a < k; ++a)
                for (int b = 0; b < k; ++b) {
                    const float xr = re[(a * k + b) * nn + q], xi = im[(a * k + b) * nn + q];
                    if (!isfinite(xr) || !isfinite(xi)) { bad += 1.0; continue; }
                    mabs = fmax(mabs, (double)fmaxf(fabsf(xr), fabsf(xi)));
                    if (a == b) {
                        if (side) t1 += xr; else t0 += xr;
                        mind = fmin(mind, (double)xr);
                        asym = fmax(asym, (double)fabsf(xi));
                    } else if (a < b) {
                        const float yr = re[(b * k + a) * nn + q], yi = im[(b * k + a) * nn + q];
                        asym = fmax(asym, (double)fmaxf(fabsf(xr - yr), fabsf(xi + yi)));
                    }
                }
        }
    }
    __shared__ double sh[6][256];
    sh[0][threadIdx.x] = t0; sh[1][threadIdx.x] = t1; sh[2][threadIdx.x] = mind;
    sh[3][threadIdx.x] = asym; sh[4][threadIdx.x] = mabs; sh[5][threadIdx.x] = bad;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            const int o = threadIdx.x + off;
            sh[0][threadIdx.x] += sh[0][o];
            sh[1][threadIdx.x] += sh[1][o];
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][o]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][o]);
            sh[4][threadIdx.x] = fmax(sh[4][threadIdx.x], sh[4][o]);
            sh[5][threadIdx.x] += sh[5][o];
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) out[blockIdx.x * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

// Hermitian part of full complex fields -> compact channels
__global__ void k_herm_to_compact(size_t nn, int k, int K, int groups, const float *__restrict__ full,
                                  float *__restrict__ comp)
{
    const int kk = k * k;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x)
        for (int g = 0; g < groups; ++g) {
            const float *re = full + (size_t)g * 2 * kk * nn, *im = re + (size_t)kk * nn;
            float *o = comp + (size_t)g * K * nn;
            int c = 0;
            for (int a = 0; a < k; ++a) o[(size_t)(c++) * nn + q] = re[(a * k + a) * nn + q];
            for (int a = 0; a < k; ++a)
                for (int b = a + 1; b < k; ++b) {
                    o[(size_t)(c++) * nn + q] = 0.5f * (re[(a * k + b) * nn + q] + re[(b * k + a) * nn + q]);
                    o[(size_t)(c++) * nn + q] = 0.5f * (im[(a * k + b) * nn + q] - im[(b * k + a) * nn + q]);
                }
            for (; c < K; ++c) o[(size_t)c * nn + q] = 0.0f;
        }
}

__global__ void k_compact_to_herm(size_t nn, int k, int K, int groups, const float *__restrict__ comp,
                                  float *__restrict__ full)
{
    const int kk = k * k;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x)
        for (int g = 0; g < groups; ++g) {
            float *re = full + (size_t)g * 2 * kk * nn, *im = re + (size_t)kk * nn;
            const float *o = comp + (size_t)g * K * nn;
            int c = 0;
            for (int a = 0; a < k; ++a) {
                re[(a * k + a) * nn + q] = o[(size_t)(c++) * nn + q];
                im[(a * k + a) * nn + q] = 0.0f;
            }
            for (int a = 0; a < k; ++a)
                for (int b = a + 1; b < k; ++b) {
                    const float xr = o[(size_t)(c++) * nn + q], xi = o[(size_t)(c++) * nn + q];
                    re[(a * k + b) * nn + q] = xr;
                    im[(a * k + b) * nn + q] = xi;
                    re[(b * k + a) * nn + q] = xr;
                    im[(b * k + a) * nn + q] = -xi;
                }
        }
}

// skew-Hermitian part of N full complex fields -> compact flux entries (Im of the
// diagonal, then Re and Im above it), and back
__global__ void k_skewh_to_compact(size_t nn, int k, int N, const float *__restrict__ full, float *__restrict__ comp)
{
    const int kk = k * k;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x)
        for (int s = 0; s < N; ++s) {
            const float *re = full + (size_t)s * 2 * kk * nn, *im = re + (size_t)kk * nn;
            float *o = comp + (size_t)s * kk * nn;
            int e = 0;
            for (int a = 0; a < k; ++a) o[(size_t)(e++) * nn + q] = im[(a * k + a) * nn + q];
            for (int a = 0; a < k; ++a)
                for (int b = a + 1; b < k; ++b) {
                    o[(size_t)(e++) * nn + q] = 0.5f * (re[(a * k + b) * nn + q] - re[(b * k + a) * nn + q]);
                    o[(size_t)(e++) * nn + q] = 0.5f * (im[(a * k + b) * nn + q] + im[(b * k + a) * nn + q]);
                }
        }
}

__global__ void k_compact_to_skewh(size_t nn, int k, int N, const float *__restrict__ comp, float *__restrict__ full)
{
    const int kk = k * k;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x)
        for (int s = 0; s < N; ++s) {
            float *re = full + (size_t)s * 2 * kk * nn, *im = re + (size_t)kk * nn;
            const float *o = comp + (size_t)s * kk * nn;
            int e = 0;
            for (int a = 0; a < k; ++a) {
                re[(a * k + a) * nn + q] = 0.0f;
                im[(a * k + a) * nn + q] = o[(size_t)(e++) * nn + q];
            }
            for (int a = 0; a < k; ++a)
                for (int b = a + 1; b < k; ++b) {
                    const float zr = o[(size_t)(e++) * nn + q], zi = o[(size_t)(e++) * nn + q];
                    re[(a * k + b) * nn + q] = zr;
                    im[(a * k + b) * nn + q] = zi;
                    re[(b * k + a) * nn + q] = -zr;
                    im[(b * k + a) * nn + q] = zi;
                }
        }
}

}  // namespace
}  // namespace vomt

using namespace vomt;

extern "C" int momt_step_sizes(int n, int k, int N, const double *L, double tau, double *mu, double *nu,
                               double *tau_used, double *lmax, double *sym_gap)
{
    if (n < 2) return VOMT_ERR_BAD_ARG;
    OpDev op;
    double lm = 0.0, gap = 0.0;
    std::string err;
    const int rc = quantum_to_op(k, N, L, &op, &lm, &gap, &err);
    if (sym_gap) *sym_gap = gap;
    if (lmax) *lmax = lm;
    if (rc) return rc;
    const double t = tau > 0.0 ? tau : default_tau_matrix(n);
    const double n1 = (double)(n - 1);
    if (mu) *mu = 1.0 / (32.0 * t * n1 * n1);
    if (nu) *nu = 1.0 / (4.0 * t * lm);
    if (tau_used) *tau_used = t;
    return VOMT_OK;
}

// Matrix OMT on a 2-D (dim 2) or 3-D (dim 3) grid: checks, compaction, the vector
// engines (2-D) or the 3-D march, expansion.
static int momt_any(int dim, vomt_ctx *ctx, int n, int k, const float *Lam0, const float *Lam1, int N,
                    const double *L, double alpha, const vomt_params *pin, float *U, float *W, float *Phi,
                    vomt_result *result, void *stream)
{
    try {
        if (!ctx) return VOMT_ERR_BAD_ARG;
        ctx->err.clear();
        cudaStream_t st = (cudaStream_t)stream;
        if (dim == 2 && (n < 2 || n > 32768)) return fail(ctx, VOMT_ERR_BAD_ARG, "n must be in [2, 32768]");
        if (dim == 3 && (n < 2 || n > 1024)) return fail(ctx, VOMT_ERR_BAD_ARG, "3-D grids: n must be in [2, 1024]");
        if (!(alpha > 0.0) || !isfinite(alpha)) return fail(ctx, VOMT_ERR_BAD_ARG, "alpha must be positive");
        if (!Lam0 || !Lam1 || !U || !W || !Phi) return fail(ctx, VOMT_ERR_BAD_ARG, "null array");
        vomt_params p;
        vomt_default_params(&p);
        if (pin) p = *pin;
        if (p.u_norm == VOMT_U_L12) p.u_norm = VOMT_U_L2;
        if (p.max_iters < 0 || p.check_every < 1) return fail(ctx, VOMT_ERR_BAD_ARG, "max_iters >= 0, check_every >= 1");
        if (p.u_norm < 1 || p.u_norm > 3 || p.w_norm < 0 || p.w_norm > 2) return fail(ctx, VOMT_ERR_BAD_ARG, "bad norm code");
        // 2 x 2 skew components have one entry a and ||W_s||_nuc = 2 |a|, the weighted ||.||_1
        if (k == 2 && p.w_norm == VOMT_W_NUC) p.w_norm = VOMT_W_L1;
        if (p.engine < 0 || p.engine > 2 || p.halo < 0 || (dim == 2 && p.halo > 16))
            return fail(ctx, VOMT_ERR_BAD_ARG, "bad engine / halo");
        if (p.eps != 0.0) return fail(ctx, VOMT_ERR_BAD_ARG, "matrix OMT takes eps = 0 (regularisation is for vector OMT)");
        if (p.pitch != 0 && (p.pitch < n || (dim == 3 && p.pitch != n)))
            return fail(ctx, VOMT_ERR_BAD_ARG, dim == 2 ? "pitch must be 0 or >= n" : "3-D grids take dense arrays");
        if (p.pitch != 0 && p.pitch != n) {
            // pitched full matrices: stage them densely, solve, copy the outputs back
            const size_t nn = (size_t)n * n, kk = (size_t)k * k;
            if (k < 1 || k > 8 || N < 1 || N * kk > 512) return fail(ctx, VOMT_ERR_BAD_ARG, "bad k or N");
            int rc = ensure_buffer(ctx, (void **)&ctx->pstage, &ctx->pstage_bytes,
                                   sizeof(float) * (5 + (size_t)N) * kk * nn, "pitch staging");
            if (rc) return rc;
            cudaError_t e = cudaSetDevice(ctx->device);
            float *d0 = ctx->pstage, *d1 = d0 + kk * nn, *dU = d1 + kk * nn, *dW = dU + 2 * kk * nn;
            float *dP = dW + (size_t)N * kk * nn;
            const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
            const int pitch = p.pitch;
            if (e == cudaSuccess) e = copy_planes(d0, n, Lam0, pitch, n, kk, d2d, st);
            if (e == cudaSuccess) e = copy_planes(d1, n, Lam1, pitch, n, kk, d2d, st);
            if (p.warm_start) {
                if (e == cudaSuccess) e = copy_planes(dU, n, U, pitch, n, 2 * kk, d2d, st);
                if (e == cudaSuccess) e = copy_planes(dW, n, W, pitch, n, (size_t)N * kk, d2d, st);
                if (e == cudaSuccess) e = copy_planes(dP, n, Phi, pitch, n, kk, d2d, st);
            }
            if (e != cudaSuccess) return set_cuda_error(ctx, e, "pitched copy in");
            vomt_params dense = *pin;
            dense.pitch = 0;
            const int status = momt_any(dim, ctx, n, k, d0, d1, N, L, alpha, &dense, dU, dW, dP, result, stream);
            if (status < 0) return status;
            e = copy_planes(U, pitch, dU, n, n, 2 * kk, d2d, st);
            if (e == cudaSuccess) e = copy_planes(W, pitch, dW, n, n, (size_t)N * kk, d2d, st);
            if (e == cudaSuccess) e = copy_planes(Phi, pitch, dP, n, n, kk, d2d, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return set_cuda_error(ctx, e, "pitched copy out");
            return status;
        }
        OpDev op;
        double lmax = 0.0, gap = 0.0;
        int rc = quantum_to_op(k, N, L, &op, &lmax, &gap, &ctx->err);
        if (rc) return rc;
        const double tau = p.tau > 0.0 ? p.tau : default_tau_matrix(n);
        const double n1 = (double)(n - 1);
        // ||grad||^2 <= 4 dim (n-1)^2; the default mu keeps tau mu ||grad||^2 at 1/4
        const double gsq = 4.0 * dim;
        double mu = p.mu, nu = p.nu;
        const bool user = mu > 0.0 || nu > 0.0;
        if (!(mu > 0.0)) mu = 1.0 / (4.0 * gsq * tau * n1 * n1);
        if (!(nu > 0.0)) nu = 1.0 / (4.0 * tau * lmax);
        if (user && !(tau * mu * gsq * n1 * n1 + tau * nu * lmax < 1.0))
            return fail(ctx, VOMT_ERR_STEP_CONDITION,
                        dim == 2 ? "step sizes break 1 > tau mu 8(n-1)^2 + tau nu lambda_max(-Delta_L)"
                                 : "step sizes break 1 > tau mu 12(n-1)^2 + tau nu lambda_max(-Delta_L)");
        p.tau = tau;
        p.mu = mu;
        p.nu = nu;
        StepDev s{n, (float)n1, (float)mu, (float)nu, (float)tau, (float)alpha};
        SolveCfg cfg{p.tol_gap, p.tol_res, mu, nu, tau, 1};

        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaSetDevice");
        ctx->launches = 0;
        const size_t nn = dim == 2 ? (size_t)n * n : (size_t)n * n * n;
        const PairTable t = make_pairs(k);
        const int K = t.K, l = op.l, kk = k * k;
        // input checks
        const int vb = (int)((nn + 255) / 256 < 512 ? (nn + 255) / 256 : 512);
        rc = ensure_buffer(ctx, (void **)&ctx->partials, &ctx->partials_cap, sizeof(double) * 6 * (size_t)vb, "partials");
        if (rc) return rc;
        k_mat_validate<<<vb, 256, 0, st>>>(nn, k, Lam0, Lam1, ctx->partials);
        ++ctx->launches;
        std::vector<double> hv((size_t)vb * 6);
        e = cudaMemcpyAsync(hv.data(), ctx->partials, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "matrix validate");
        double tr0 = 0.0, tr1 = 0.0, mind = 1e300, asym = 0.0, mabs = 0.0, bad = 0.0;
        for (int q = 0; q < vb; ++q) {
            tr0 += hv[q * 6 + 0];
            tr1 += hv[q * 6 + 1];
            mind = fmin(mind, hv[q * 6 + 2]);
            asym = fmax(asym, hv[q * 6 + 3]);
            mabs = fmax(mabs, hv[q * 6 + 4]);
            bad += hv[q * 6 + 5];
        }
        if (bad > 0.0) return fail(ctx, VOMT_ERR_NONFINITE, "density has NaN or Inf entries");
        if (mind < 0.0) return fail(ctx, VOMT_ERR_NEGATIVE_DENSITY, "density has a negative diagonal entry");
        if (asym > 1e-5 * mabs) return fail(ctx, VOMT_ERR_BAD_ARG, "densities must be symmetric matrices");
        if (fabs(tr0 - tr1) > kMassRelTol * fmax(fabs(tr0), fabs(tr1)))
            return fail(ctx, VOMT_ERR_MASS_MISMATCH, "Lam0 and Lam1 have different total trace");
        // compact staging: rho0, rho1 (K), u (dim K), w (l), phi (K)
        const size_t need = sizeof(float) * (size_t)((3 + dim) * K + l) * nn;
        rc = ensure_buffer(ctx, (void **)&ctx->mstage, &ctx->mstage_bytes, need, "matrix staging");
        if (rc) return rc;
        float *c0 = ctx->mstage, *c1 = c0 + (size_t)K * nn, *cu = c1 + (size_t)K * nn;
        float *cw = cu + (size_t)dim * K * nn, *cp = cw + (size_t)l * nn;
        const int pb = (int)((nn + 255) / 256 < 2048 ? (nn + 255) / 256 : 2048);
        k_sym_to_compact<<<pb, 256, 0, st>>>(nn, t, 1, Lam0, c0);
        k_sym_to_compact<<<pb, 256, 0, st>>>(nn, t, 1, Lam1, c1);
        ctx->launches += 2;
        if (p.warm_start) {
            k_sym_to_compact<<<pb, 256, 0, st>>>(nn, t, dim, U, cu);
            k_skew_to_compact<<<pb, 256, 0, st>>>(nn, t, N, W, cw);
            k_sym_to_compact<<<pb, 256, 0, st>>>(nn, t, 1, Phi, cp);
            ctx->launches += 3;
        }
        int engine = VOMT_ENGINE_STREAM;
        if (dim == 2) {
            rc = run_engine(ctx, op, s, cfg, p, c0, c1, cu, cw, cp, st, &engine);
        } else {
            ctx->last_blocks = ctx->last_halo = ctx->last_variant = 0;
            vomt_params p3 = p;
            p3.halo = 0;
            rc = solve3d_core(ctx, n, op, s, cfg, p3, p.halo, c0, c1, cu, cw, cp, st);
        }
        if (rc) return rc;
        k_compact_to_sym<<<pb, 256, 0, st>>>(nn, t, dim, cu, U);
        k_compact_to_skew<<<pb, 256, 0, st>>>(nn, t, N, cw, W);
        k_compact_to_sym<<<pb, 256, 0, st>>>(nn, t, 1, cp, Phi);
        ctx->launches += 3;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "matrix expand");
        (void)kk;
        int status = 0;
        fill_result(ctx, cfg, engine, result, &status);
        return status;
    } catch (...) {
        return fail(ctx, VOMT_ERR_BAD_ARG, "internal exception");
    }
}

extern "C" int momt_solve(vomt_ctx *ctx, int n, int k, const float *Lam0, const float *Lam1, int N, const double *L,
                          double alpha, const vomt_params *pin, float *U, float *W, float *Phi, vomt_result *result,
                          void *stream)
{
    return momt_any(2, ctx, n, k, Lam0, Lam1, N, L, alpha, pin, U, W, Phi, result, stream);
}

extern "C" int momt_solve3d(vomt_ctx *ctx, int n, int k, const float *Lam0, const float *Lam1, int N,
                            const double *L, double alpha, const vomt_params *pin, float *U, float *W, float *Phi,
                            vomt_result *result, void *stream)
{
    return momt_any(3, ctx, n, k, Lam0, Lam1, N, L, alpha, pin, U, W, Phi, result, stream);
}

// Complex Hermitian matrix OMT (Section 4's complex setting, iteration of Section
// 7.3) with the Frobenius norms, on the vector engines through hermitian_to_op.
extern "C" int momt_solve_complex(vomt_ctx *ctx, int n, int k, const float *Lam0, const float *Lam1, int N,
                                  const double *L, double alpha, const vomt_params *pin, float *U, float *W,
                                  float *Phi, vomt_result *result, void *stream)
{
    try {
        if (!ctx) return VOMT_ERR_BAD_ARG;
        ctx->err.clear();
        cudaStream_t st = (cudaStream_t)stream;
        if (n < 2 || n > 32768) return fail(ctx, VOMT_ERR_BAD_ARG, "n must be in [2, 32768]");
        if (!(alpha > 0.0) || !isfinite(alpha)) return fail(ctx, VOMT_ERR_BAD_ARG, "alpha must be positive");
        if (!Lam0 || !Lam1 || !U || !W || !Phi) return fail(ctx, VOMT_ERR_BAD_ARG, "null array");
        vomt_params p;
        vomt_default_params(&p);
        if (pin) p = *pin;
        if (p.pitch != 0 && p.pitch != n) return fail(ctx, VOMT_ERR_BAD_ARG, "complex matrix OMT takes dense arrays");
        if (p.u_norm == VOMT_U_L12) p.u_norm = VOMT_U_L2;
        if ((p.u_norm != VOMT_U_L2 && p.u_norm != VOMT_U_L1) || (p.w_norm != VOMT_W_L2 && p.w_norm != VOMT_W_L1))
            return fail(ctx, VOMT_ERR_BAD_ARG,
                        "complex matrix OMT takes the Frobenius norms (L2) or the entrywise norms (L1) for U and W");
        // the entrywise norms of complex fields are the modulus kind (internal codes)
        const bool entrywise = p.u_norm == VOMT_U_L1 || p.w_norm == VOMT_W_L1;
        if (p.u_norm == VOMT_U_L1) p.u_norm = U_CL1;
        if (p.w_norm == VOMT_W_L1) p.w_norm = W_CL1;
        if ((entrywise || k == 3) && p.engine == VOMT_ENGINE_STREAM)
            return fail(ctx, VOMT_ERR_BAD_ARG, "complex 3 x 3 fields and the entrywise norms run on the resident engine");
        if (p.max_iters < 0 || p.check_every < 1) return fail(ctx, VOMT_ERR_BAD_ARG, "max_iters >= 0, check_every >= 1");
        if (p.engine < 0 || p.engine > 2 || p.halo < 0 || p.halo > 16) return fail(ctx, VOMT_ERR_BAD_ARG, "bad engine / halo");
        if (p.eps != 0.0) return fail(ctx, VOMT_ERR_BAD_ARG, "complex matrix OMT takes eps = 0");
        OpDev op;
        double lmax = 0.0, gap = 0.0;
        int rc = hermitian_to_op(k, N, L, &op, &lmax, &gap, &ctx->err);
        if (rc) return rc;
        const double tau = p.tau > 0.0 ? p.tau : default_tau_matrix(n);
        const double n1 = (double)(n - 1);
        double mu = p.mu, nu = p.nu;
        const bool user = mu > 0.0 || nu > 0.0;
        if (!(mu > 0.0)) mu = 1.0 / (32.0 * tau * n1 * n1);
        if (!(nu > 0.0)) nu = 1.0 / (4.0 * tau * lmax);
        if (user && !(tau * mu * 8.0 * n1 * n1 + tau * nu * lmax < 1.0))
            return fail(ctx, VOMT_ERR_STEP_CONDITION, "step sizes break 1 > tau mu 8(n-1)^2 + tau nu lambda_max(-Delta_L)");
        p.tau = tau;
        p.mu = mu;
        p.nu = nu;
        StepDev s{n, (float)n1, (float)mu, (float)nu, (float)tau, (float)alpha};
        SolveCfg cfg{p.tol_gap, p.tol_res, mu, nu, tau, 1};
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "cudaSetDevice");
        ctx->launches = 0;
        const size_t nn = (size_t)n * n;
        const int K = op.k, l = op.l, kk = k * k;
        const int vb = (int)((nn + 255) / 256 < 512 ? (nn + 255) / 256 : 512);
        rc = ensure_buffer(ctx, (void **)&ctx->partials, &ctx->partials_cap, sizeof(double) * 6 * (size_t)vb, "partials");
        if (rc) return rc;
        k_herm_validate<<<vb, 256, 0, st>>>(nn, k, Lam0, Lam1, ctx->partials);
        ++ctx->launches;
        std::vector<double> hv((size_t)vb * 6);
        e = cudaMemcpyAsync(hv.data(), ctx->partials, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "complex validate");
        double tr0 = 0.0, tr1 = 0.0, mind = 1e300, asym = 0.0, mabs = 0.0, bad = 0.0;
        for (int q = 0; q < vb; ++q) {
            tr0 += hv[q * 6 + 0];
            tr1 += hv[q * 6 + 1];
            mind = fmin(mind, hv[q * 6 + 2]);
            asym = fmax(asym, hv[q * 6 + 3]);
            mabs = fmax(mabs, hv[q * 6 + 4]);
            bad += hv[q * 6 + 5];
        }
        if (bad > 0.0) return fail(ctx, VOMT_ERR_NONFINITE, "density has NaN or Inf entries");
        if (mind < 0.0) return fail(ctx, VOMT_ERR_NEGATIVE_DENSITY, "density has a negative diagonal entry");
        if (asym > 1e-5 * mabs) return fail(ctx, VOMT_ERR_BAD_ARG, "densities must be Hermitian matrices");
        if (fabs(tr0 - tr1) > kMassRelTol * fmax(fabs(tr0), fabs(tr1)))
            return fail(ctx, VOMT_ERR_MASS_MISMATCH, "Lam0 and Lam1 have different total trace");
        // compact staging: rho0, rho1 (K), u (2K), w (l), phi (K)
        const size_t need = sizeof(float) * (size_t)(5 * K + l) * nn;
        rc = ensure_buffer(ctx, (void **)&ctx->mstage, &ctx->mstage_bytes, need, "matrix staging");
        if (rc) return rc;
        float *c0 = ctx->mstage, *c1 = c0 + (size_t)K * nn, *cu = c1 + (size_t)K * nn;
        float *cw = cu + (size_t)2 * K * nn, *cp = cw + (size_t)l * nn;
        const int pb = (int)((nn + 255) / 256 < 2048 ? (nn + 255) / 256 : 2048);
        k_herm_to_compact<<<pb, 256, 0, st>>>(nn, k, K, 1, Lam0, c0);
        k_herm_to_compact<<<pb, 256, 0, st>>>(nn, k, K, 1, Lam1, c1);
        ctx->launches += 2;
        if (p.warm_start) {
            k_herm_to_compact<<<pb, 256, 0, st>>>(nn, k, K, 2, U, cu);
            k_skewh_to_compact<<<pb, 256, 0, st>>>(nn, k, N, W, cw);
            k_herm_to_compact<<<pb, 256, 0, st>>>(nn, k, K, 1, Phi, cp);
            ctx->launches += 3;
        }
        int engine = 0;
        rc = run_engine(ctx, op, s, cfg, p, c0, c1, cu, cw, cp, st, &engine);
        if (rc) return rc;
        k_compact_to_herm<<<pb, 256, 0, st>>>(nn, k, K, 2, cu, U);
        k_compact_to_skewh<<<pb, 256, 0, st>>>(nn, k, N, cw, W);
        k_compact_to_herm<<<pb, 256, 0, st>>>(nn, k, K, 1, cp, Phi);
        ctx->launches += 3;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "complex expand");
        (void)kk;
        int status = 0;
        fill_result(ctx, cfg, engine, result, &status);
        return status;
    } catch (...) {
        return fail(ctx, VOMT_ERR_BAD_ARG, "internal exception");
    }
}
