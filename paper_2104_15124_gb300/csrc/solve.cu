// Leading eigenpairs of the discrete Kolmogorov operator and the spectral
// solve of L f = g (Sec. 2.2 eigen-decomposition, Sec. 3.1 Eqs. LS minimiser
// and f_LS, Sec. 4 steps 3-4).
//
// The solver works on L = S^-1 L-hat S, whose eigenvectors phi = S^-1 phi-hat are
// the ones the paper uses, with the inner product <f, g>_S = f^T S^2 g / n under
// which L is self-adjoint.  In these coordinates
//     (L z)_i = sum_{j != i} w_ij (z_j - z_i),   w_ij = L-hat_ij S_j / S_i >= 0,
// so every difference z_j - z_i of FP32 values is exact when it cancels
// (Sterbenz) and smooth vectors keep full accuracy without FP64 arithmetic.
//
// Method: block Chebyshev-filtered subspace iteration (GPU: a fused SpMM with a
// three-term update per filter step, Gram matrices in FP32 blocks carried to
// FP64, block rotations) with Rayleigh-Ritz on the host in FP64 (cyclic
// Jacobi).  A block of B >= ell + 1 vectors captures clusters and near-equal
// pairs (the circle's +-k pairs, the 2l + 1 groups on S^2) that a
// single-vector Lanczos would resolve slowly.  Spectrum bounds: L's
// eigenvalues lie in [-2 max_i sum_j w_ij, 0] (Gershgorin on the weights).
#include "vb_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace vb {

constexpr int GRAM_ROWS = 64;    // rows per FP32 Gram partial before carrying to FP64
constexpr int GRAM_THREADS = 256;

// ------------------------------------------------------------------ device kernels
// w_ij = val_ij S_j / S_i off the diagonal (0 on it); rowsum_i = sum_j w_ij.
__global__ void solve_weights_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                     const float* __restrict__ val, const double* __restrict__ S, int64_t n,
                                     float* w, float* rowsum)
{
    const int lane = threadIdx.x & 31;
    int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t step = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; i < n; i += step) {
        const double isi = 1.0 / S[i];
        float s = 0.f;
        for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
            const int32_t j = col[e];
            const float v = j == i ? 0.f : (float)((double)val[e] * (S[j] * isi));
            w[e] = v;
            s += v;
        }
        s = warp_sum_f32(s);
        if (lane == 0) rowsum[i] = s;
    }
}

__global__ void max_kernel(const float* __restrict__ v, int64_t n, float* out)
{
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, v[i]);
    m = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m)));
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned*)out, __float_as_uint(m));
}

// Counter-based initial block: splitmix64 of (seed, element) mapped to [-1, 1).
__global__ void random_block_kernel(float* Z, int64_t count, uint64_t seed)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint64_t x = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    Z[i] = (float)((double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

// Columns [r, B) of an [n][B] block refilled with counter-based random values.
__global__ void refill_kernel(float* Z, int64_t n, int B, int r, uint64_t seed)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int width = B - r;
    if (idx >= n * width) return;
    const int64_t i = idx / width;
    const int b = r + (int)(idx - i * width);
    uint64_t x = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(idx + 1);
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    Z[i * B + b] = (float)((double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

// out = a1 (L Y) + a2 Y + a3 X for an [n][B] block, B = 32 CPL; one warp per row,
// lane c handles columns c, c + 32, ...
template <int CPL>
__global__ void __launch_bounds__(256) spmm_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                                   const float* __restrict__ w, int64_t n, const float* __restrict__ Y,
                                                   const float* __restrict__ X, float* out, float a1, float a2,
                                                   float a3)
{
    constexpr int B = 32 * CPL;
    const int lane = threadIdx.x & 31;
    int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t step = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; i < n; i += step) {
        float yi[CPL], acc[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            yi[c] = Y[i * B + lane + 32 * c];
            acc[c] = 0.f;
        }
        const int64_t rb = row_ptr[i], re = row_ptr[i + 1];
        for (int64_t e0 = rb; e0 < re; e0 += 32) {
            const int64_t e = e0 + lane;
            const int32_t jl = e < re ? col[e] : 0;
            const float wl = e < re ? w[e] : 0.f;
            const int cnt = (int)(re - e0 < 32 ? re - e0 : 32);
            for (int u = 0; u < cnt; ++u) {
                const int32_t j = __shfl_sync(0xffffffffu, jl, u);
                const float wv = __shfl_sync(0xffffffffu, wl, u);
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[c] = fmaf(wv, Y[(int64_t)j * B + lane + 32 * c] - yi[c], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            float r = a1 * acc[c] + a2 * yi[c];
            if (X) r += a3 * X[i * B + lane + 32 * c];
            out[i * B + lane + 32 * c] = r;
        }
    }
}

// Partial Gram matrices: part[blk][a][b] = sum_i wgt_i A[i][a] C[i][b] over the block's rows,
// FP32 within GRAM_ROWS rows, FP64 across them.  wgt = S^2 (or 1 when wgt2 == nullptr).
__global__ void __launch_bounds__(GRAM_THREADS) gram_kernel(const float* __restrict__ A, const float* __restrict__ C,
                                                            const double* __restrict__ S, int64_t n, int B,
                                                            double* part)
{
    extern __shared__ float gsh[];
    float* As = gsh;                      // [GRAM_ROWS][B]
    float* Cs = gsh + GRAM_ROWS * B;      // [GRAM_ROWS][B]
    const int t = threadIdx.x;
    const int per = (B * B + GRAM_THREADS - 1) / GRAM_THREADS;   // <= 64 for B <= 128
    double accd[64];
    for (int q = 0; q < per; ++q) accd[q] = 0.0;
    const int64_t nchunks = (n + GRAM_ROWS - 1) / GRAM_ROWS;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t r0 = ch * GRAM_ROWS;
        for (int idx = t; idx < GRAM_ROWS * B; idx += GRAM_THREADS) {
            const int64_t r = r0 + idx / B;
            float wv = 0.f, av = 0.f, cv = 0.f;
            if (r < n) {
                const double s = S ? S[r] : 1.0;
                wv = (float)(s * s);
                av = A[r * B + idx % B];
                cv = C[r * B + idx % B];
            }
            As[idx] = av * wv;
            Cs[idx] = cv;
        }
        __syncthreads();
        for (int q = 0; q < per; ++q) {
            const int e = t + q * GRAM_THREADS;
            if (e >= B * B) break;
            const int a = e / B, b = e % B;
            float s = 0.f;
            for (int r = 0; r < GRAM_ROWS; ++r) s = fmaf(As[r * B + a], Cs[r * B + b], s);
            accd[q] += (double)s;
        }
        __syncthreads();
    }
    for (int q = 0; q < per; ++q) {
        const int e = t + q * GRAM_THREADS;
        if (e < B * B) part[(int64_t)blockIdx.x * B * B + e] = accd[q];
    }
}

__global__ void gram_reduce_kernel(const double* __restrict__ part, int nblk, int BB, double inv_n, double* G)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= BB) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * BB + e];
    G[e] = s * inv_n;
}

// out[i][b] = sum_c Y[i][c] M[c][b] (M: B x B FP32 in shared memory)
__global__ void __launch_bounds__(256) rotate_kernel(const float* __restrict__ Y, const float* __restrict__ M,
                                                     int64_t n, int B, float* out)
{
    extern __shared__ float Ms[];
    for (int e = threadIdx.x; e < B * B; e += blockDim.x) Ms[e] = M[e];
    __syncthreads();
    const int64_t total = n * B;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / B;
        const int b = (int)(idx - i * B);
        const float* yr = Y + i * B;
        float s = 0.f;
        for (int c = 0; c < B; ++c) s = fmaf(yr[c], Ms[c * B + b], s);
        out[idx] = s;
    }
}

// phi[j][i] = Z[i][j] for the first ell + 1 columns
__global__ void extract_kernel(const float* __restrict__ Z, int64_t n, int B, int cols, float* phi)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * cols) return;
    const int64_t j = idx / n, i = idx - j * n;
    phi[idx] = Z[i * B + j];
}

// f_i = sum_{j=1..ell} coef_j Z[i][j]
__global__ void combine_kernel(const float* __restrict__ Z, int64_t n, int B, const float* __restrict__ coef, int cols,
                               float* f)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int j = 1; j < cols; ++j) s = fmaf(coef[j], Z[i * B + j], s);
    f[i] = s;
}

// g~_j = sum_i S_i^2 Z[i][j] g_i / n, accumulated per block then reduced (columns < cols)
__global__ void project_kernel(const float* __restrict__ Z, const float* __restrict__ g, const double* __restrict__ S,
                               int64_t n, int B, int cols, double* part)
{
    __shared__ double sh[8][128];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double acc[4] = {0, 0, 0, 0};
    for (int64_t i = blockIdx.x * 8 + w; i < n; i += (int64_t)gridDim.x * 8) {
        const double s = S[i];
        const float wg = (float)(s * s) * g[i];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = lane + 32 * c;
            if (j < cols) acc[c] += (double)(wg * Z[i * B + j]);
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) sh[w][lane + 32 * c] = acc[c];
    __syncthreads();
    if (threadIdx.x < 128) {
        double s = 0.0;
        for (int ww = 0; ww < 8; ++ww) s += sh[ww][threadIdx.x];
        part[(int64_t)blockIdx.x * 128 + threadIdx.x] = s;
    }
}

// ------------------------------------------------------------------ host: small dense FP64 algebra
// Cyclic Jacobi eigen-decomposition of a symmetric B x B matrix (row-major):
// on return A's diagonal holds the eigenvalues and V the eigenvectors (columns).
static void jacobi_eig(std::vector<double>& A, std::vector<double>& V, int B)
{
    V.assign((size_t)B * B, 0.0);
    for (int i = 0; i < B; ++i) V[(size_t)i * B + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < B; ++p)
            for (int q = 0; q < B; ++q) {
                const double a = A[(size_t)p * B + q] * A[(size_t)p * B + q];
                tot += a;
                if (p != q) off += a;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < B - 1; ++p)
            for (int q = p + 1; q < B; ++q) {
                const double apq = A[(size_t)p * B + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * B + p], aqq = A[(size_t)q * B + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double tt = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(tt * tt + 1.0), s = tt * c;
                for (int k = 0; k < B; ++k) {   // columns p, q
                    const double akp = A[(size_t)k * B + p], akq = A[(size_t)k * B + q];
                    A[(size_t)k * B + p] = c * akp - s * akq;
                    A[(size_t)k * B + q] = s * akp + c * akq;
                }
                for (int k = 0; k < B; ++k) {   // rows p, q
                    const double apk = A[(size_t)p * B + k], aqk = A[(size_t)q * B + k];
                    A[(size_t)p * B + k] = c * apk - s * aqk;
                    A[(size_t)q * B + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < B; ++k) {
                    const double vkp = V[(size_t)k * B + p], vkq = V[(size_t)k * B + q];
                    V[(size_t)k * B + p] = c * vkp - s * vkq;
                    V[(size_t)k * B + q] = s * vkp + c * vkq;
                }
            }
    }
}

struct SolveWs {
    float* w;       // nnz weights
    float* rowsum;  // n
    float* fmax;    // 1
    float* Z;       // n B
    float* Y;       // n B
    float* X;       // n B
    float* LY;      // n B
    float* M;       // B B rotation (FP32)
    double* part;   // nblk B B
    double* G;      // B B
    double* proj;   // nblk 128
    float* coef;    // 128
};

static int solve_block(int ell, int block)
{
    int B = block > 0 ? block : std::max(2 * (ell + 1), ell + 17);
    B = ((B + 31) / 32) * 32;
    // the default stays within the 128-vector limit while it leaves 16 spare vectors
    if (block <= 0 && B > 128 && ell + 17 <= 128) B = 128;
    return B;
}
constexpr int GRAM_BLOCKS = 152;

static size_t solve_plan(Carve& c, int64_t n, int64_t cap, int B, SolveWs* o)
{
    SolveWs w;
    w.w = c.take<float>(cap);
    w.rowsum = c.take<float>(n);
    w.fmax = c.take<float>(1);
    w.Z = c.take<float>(n * B);
    w.Y = c.take<float>(n * B);
    w.X = c.take<float>(n * B);
    w.LY = c.take<float>(n * B);
    w.M = c.take<float>((size_t)B * B);
    w.part = c.take<double>((size_t)GRAM_BLOCKS * B * B);
    w.G = c.take<double>((size_t)B * B);
    w.proj = c.take<double>((size_t)GRAM_BLOCKS * 128);
    w.coef = c.take<float>(128);
    if (o) *o = w;
    return c.off;
}

size_t solve_ws_bytes(int64_t n, int64_t cap, const vb_solve_params* p)
{
    Carve c(nullptr);
    return solve_plan(c, n, cap, solve_block(p ? p->ell : 16, p ? p->block : 0), nullptr);
}

template <int CPL>
static void spmm(cudaStream_t s, const vb_graph* g, const float* w, const float* Y, const float* X, float* out,
                 float a1, float a2, float a3)
{
    spmm_kernel<CPL><<<kRowBlocks, kRowThreads, 0, s>>>(g->row_ptr, g->col, w, g->n, Y, X, out, a1, a2, a3);
}

vb_status solve_run(Ctx* ctx, const vb_graph* g, int64_t cap, const float* val, const double* S,
                    const vb_solve_params* p, double* evals, float* phi, const float* rhs, float* f, int32_t* iters,
                    void* ws, size_t ws_bytes)
{
    if (!g || !g->row_ptr || !val || !S || !p || !evals || p->ell < 1 || g->n < 2) return VB_ERR_ARG;
    const int B = solve_block(p->ell, p->block);
    const int CPL = B / 32;
    if (B > 128 || p->ell + 1 > B || (int64_t)B > g->n) return VB_ERR_ARG;
    const int nwant = p->ell + 1;
    SolveWs w;
    Carve c(ws);
    if (!ws || ws_bytes < solve_plan(c, g->n, cap, B, &w)) return VB_ERR_WORKSPACE;
    cudaStream_t s = ctx->stream;
    const int64_t n = g->n;
    const int degree = p->degree > 0 ? p->degree : 30;
    const int max_iter = p->max_iter > 0 ? p->max_iter : 60;
    const double tol = p->tol > 0 ? p->tol : 1e-7;

    solve_weights_kernel<<<kRowBlocks, kRowThreads, 0, s>>>(g->row_ptr, g->col, val, S, n, w.w, w.rowsum);
    cudaMemsetAsync(w.fmax, 0, sizeof(float), s);
    max_kernel<<<152, 256, 0, s>>>(w.rowsum, n, w.fmax);
    random_block_kernel<<<(unsigned)((n * B + 255) / 256), 256, 0, s>>>(w.Z, n * B, p->seed ^ 0x5EEDull);
    float fmax_h = 0.f;
    if (cudaMemcpyAsync(&fmax_h, w.fmax, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VB_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VB_ERR_CUDA;
    // spectrum of M = -L lies in [0, mu_max]
    const double mu_max = 2.0 * (double)fmax_h * 1.0001 + 1e-30;
    auto SPMM = [&](const float* Y, const float* X, float* out, float a1, float a2, float a3) {
        switch (CPL) {
            case 1: spmm<1>(s, g, w.w, Y, X, out, a1, a2, a3); break;
            case 2: spmm<2>(s, g, w.w, Y, X, out, a1, a2, a3); break;
            case 3: spmm<3>(s, g, w.w, Y, X, out, a1, a2, a3); break;
            default: spmm<4>(s, g, w.w, Y, X, out, a1, a2, a3); break;
        }
    };
    const size_t gsm = (size_t)2 * GRAM_ROWS * B * sizeof(float);
    static bool gattr[16] = {};
    if (!gattr[ctx->device & 15]) {
        if (cudaFuncSetAttribute(gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * GRAM_ROWS * 128 * 4) !=
            cudaSuccess)
            return VB_ERR_CUDA;
        // the rotation keeps the whole B x B matrix in shared memory: 64 KB at B = 128
        if (cudaFuncSetAttribute(rotate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 4) !=
            cudaSuccess)
            return VB_ERR_CUDA;
        gattr[ctx->device & 15] = true;
    }
    std::vector<double> Gh((size_t)B * B), Hh((size_t)B * B);
    auto gram = [&](const float* A, const float* C2, std::vector<double>& out) -> vb_status {
        gram_kernel<<<GRAM_BLOCKS, GRAM_THREADS, gsm, s>>>(A, C2, S, n, B, w.part);
        gram_reduce_kernel<<<(B * B + 255) / 256, 256, 0, s>>>(w.part, GRAM_BLOCKS, B * B, 1.0 / (double)n, w.G);
        if (cudaMemcpyAsync(out.data(), w.G, sizeof(double) * B * B, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return VB_ERR_CUDA;
        return cuda_status(cudaStreamSynchronize(s));
    };

    std::vector<double> theta(B, 0.0), prev(nwant, 0.0);
    std::vector<float> Mh((size_t)B * B);
    float* bufs[3] = {w.Z, w.Y, w.X};
    int zi = 0;   // which of bufs holds the current Ritz block
    double mu_cut = 0.5 * mu_max;
    int it = 0, stable = 0;
    bool converged = false;
    vb_status st = VB_OK;
    uint64_t reseed = p->seed;
    for (it = 0; it < max_iter; ++it) {
        // Chebyshev filter of degree `degree` damping [mu_cut, mu_max] of M = -L, Y <- p(M) Z
        // (Zhou & Saad's scaled three-term recurrence; M Y = -(L Y)).
        float* Xb = bufs[zi];
        float* Yb = bufs[(zi + 1) % 3];
        float* Tb = bufs[(zi + 2) % 3];
        if (it > 0) {
            const double e = (mu_max - mu_cut) / 2.0, cc = (mu_max + mu_cut) / 2.0;
            double sigma = e / (0.0 - cc);
            const double tau = 2.0 / sigma;
            // Y = (sigma / e) (M Z - c Z) = -(sigma/e) L Z - (sigma c / e) Z
            SPMM(Xb, nullptr, Yb, (float)(-sigma / e), (float)(-sigma * cc / e), 0.f);
            for (int k = 2; k <= degree; ++k) {
                const double sn = 1.0 / (tau - sigma);
                // T = (2 sn / e) (M Y - c Y) - sigma sn X
                SPMM(Yb, Xb, Tb, (float)(-2.0 * sn / e), (float)(-2.0 * sn * cc / e), (float)(-sigma * sn));
                float* tmp = Xb;
                Xb = Yb;
                Yb = Tb;
                Tb = tmp;
                sigma = sn;
            }
        } else {
            Yb = bufs[zi];
        }
        // Rayleigh-Ritz in the S-inner product: G = Y^T W Y, H = Y^T W (L Y)
        SPMM(Yb, nullptr, w.LY, 1.f, 0.f, 0.f);
        if ((st = gram(Yb, Yb, Gh)) != VB_OK) return st;
        if ((st = gram(Yb, w.LY, Hh)) != VB_OK) return st;
        for (int a = 0; a < B; ++a)
            for (int b = 0; b < a; ++b) {
                const double hs = 0.5 * (Hh[(size_t)a * B + b] + Hh[(size_t)b * B + a]);
                Hh[(size_t)a * B + b] = Hh[(size_t)b * B + a] = hs;
                const double gs = 0.5 * (Gh[(size_t)a * B + b] + Gh[(size_t)b * B + a]);
                Gh[(size_t)a * B + b] = Gh[(size_t)b * B + a] = gs;
            }
        // G = V diag(g) V^T; keep the r directions with g > 1e-12 max(g): C1 = V_r g_r^-1/2 (B x r)
        std::vector<double> V1, V2;
        jacobi_eig(Gh, V1, B);
        double gmax = 0.0;
        for (int a = 0; a < B; ++a) gmax = std::max(gmax, Gh[(size_t)a * B + a]);
        std::vector<int> keep;
        for (int a = 0; a < B; ++a)
            if (Gh[(size_t)a * B + a] > 1e-12 * gmax) keep.push_back(a);
        const int r = (int)keep.size();
        if (r < nwant) return VB_ERR_NOT_CONVERGED;
        std::vector<double> C1((size_t)B * r);
        for (int q = 0; q < r; ++q) {
            const double sc = 1.0 / std::sqrt(Gh[(size_t)keep[q] * B + keep[q]]);
            for (int row = 0; row < B; ++row) C1[(size_t)row * r + q] = V1[(size_t)row * B + keep[q]] * sc;
        }
        // H' = C1^T H C1 (r x r), eigen-decomposed; Ritz vectors Y C1 U, values descending
        std::vector<double> T1((size_t)B * r), Hp((size_t)r * r);
        for (int row = 0; row < B; ++row)
            for (int b = 0; b < r; ++b) {
                double sacc = 0.0;
                for (int k = 0; k < B; ++k) sacc += Hh[(size_t)row * B + k] * C1[(size_t)k * r + b];
                T1[(size_t)row * r + b] = sacc;
            }
        for (int a = 0; a < r; ++a)
            for (int b = 0; b < r; ++b) {
                double sacc = 0.0;
                for (int k = 0; k < B; ++k) sacc += C1[(size_t)k * r + a] * T1[(size_t)k * r + b];
                Hp[(size_t)a * r + b] = sacc;
            }
        jacobi_eig(Hp, V2, r);
        std::vector<int> ord(r);
        for (int a = 0; a < r; ++a) ord[a] = a;
        std::sort(ord.begin(), ord.end(), [&](int x, int y) { return Hp[(size_t)x * r + x] > Hp[(size_t)y * r + y]; });
        for (int a = 0; a < r; ++a) theta[a] = Hp[(size_t)ord[a] * r + ord[a]];
        std::fill(Mh.begin(), Mh.end(), 0.f);
        for (int row = 0; row < B; ++row)
            for (int b = 0; b < r; ++b) {
                double sacc = 0.0;
                for (int k = 0; k < r; ++k) sacc += C1[(size_t)row * r + k] * V2[(size_t)k * r + ord[b]];
                Mh[(size_t)row * B + b] = (float)sacc;
            }
        if (cudaMemcpyAsync(w.M, Mh.data(), sizeof(float) * B * B, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return VB_ERR_CUDA;
        // the rotated block goes to a buffer other than Yb
        int out = 0;
        while (bufs[out] == Yb) ++out;
        rotate_kernel<<<152 * 4, 256, (size_t)B * B * sizeof(float), s>>>(Yb, w.M, n, B, bufs[out]);
        zi = out;
        if (r < B) {   // rank lost in the filter: refill the dropped columns with fresh random vectors
            reseed = reseed * 6364136223846793005ull + 1442695040888963407ull;
            refill_kernel<<<(unsigned)((n * (B - r) + 255) / 256), 256, 0, s>>>(bufs[zi], n, B, r, reseed);
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return VB_ERR_CUDA;
        // unwanted interval starts at the block's most negative Ritz value
        mu_cut = std::max(-theta[r - 1], 1e-12 * mu_max);
        // convergence: the wanted Ritz values stop moving
        double scale = 0.0;
        for (int a = 0; a < nwant; ++a) scale = std::max(scale, std::fabs(theta[a]));
        double change = 0.0;
        for (int a = 0; a < nwant; ++a) change = std::max(change, std::fabs(theta[a] - prev[a]));
        for (int a = 0; a < nwant; ++a) prev[a] = theta[a];
        if (it > 0 && change <= tol * scale) {
            if (++stable >= 2) { converged = true; ++it; break; }
        } else {
            stable = 0;
        }
    }
    w.Z = bufs[zi];
    if (cudaMemcpyAsync(evals, theta.data(), sizeof(double) * nwant, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return VB_ERR_CUDA;
    if (phi)
        extract_kernel<<<(unsigned)((n * nwant + 255) / 256), 256, 0, s>>>(w.Z, n, B, nwant, phi);
    if (rhs && f) {
        // Eq. (LS minimiser): g~_j = <phi_j, g>_S, f~_j = g~_j / lambda_j (j = 1..ell), f = Q f~
        project_kernel<<<GRAM_BLOCKS, 256, 0, s>>>(w.Z, rhs, S, n, B, nwant, w.proj);
        std::vector<double> ph((size_t)GRAM_BLOCKS * 128);
        if (cudaMemcpyAsync(ph.data(), w.proj, sizeof(double) * ph.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return VB_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return VB_ERR_CUDA;
        std::vector<float> cf(128, 0.f);
        for (int j = 1; j < nwant; ++j) {
            double gt = 0.0;
            for (int b = 0; b < GRAM_BLOCKS; ++b) gt += ph[(size_t)b * 128 + j];
            gt /= (double)n;
            cf[j] = (float)(gt / theta[j]);
        }
        if (cudaMemcpyAsync(w.coef, cf.data(), sizeof(float) * 128, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return VB_ERR_CUDA;
        combine_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.Z, n, B, w.coef, nwant, f);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return VB_ERR_CUDA;
    if (iters) *iters = it;
    return converged ? VB_OK : VB_ERR_NOT_CONVERGED;
}

}  // namespace vb
