// Gradient representation in the eigenbasis (Sec. 3.2).
//
// With eigenpairs (lambda_l, phi_l) of L, <f, g>_S = f^T S^2 g / n and
// C_ljk = <phi_l, phi_j * phi_k>_S, the truncated Eq. (gradient of u) reads
//     du/dx_s = sum_{l,j,k} u_j v_k (C_ljk / 2) (lambda_l - lambda_j - lambda_k) phi_l,
// u_j = <u, phi_j>_S, v_k = <x_s, phi_k>_S.  Summing over j and k first,
//     sum_{j,k} u_j v_k C_ljk (lambda_l - lambda_j - lambda_k)
//       = lambda_l <phi_l, a b>_S - <phi_l, c b + a d>_S
// with a = sum_j u_j phi_j, c = sum_j lambda_j u_j phi_j, b = sum_k v_k phi_k and
// d = sum_k lambda_k v_k phi_k (an exact rearrangement of the same finite sums), so
// the ell^3 n contraction becomes a few projections and expansions over the
// eigenvectors, O(ell n) per coordinate:
//   1. coefficients of u and of every coordinate x_s (projection, one pass over phi);
//   2. per sample a, c, b_s, d_s and the products p_s = a b_s, q_s = c b_s + a d_s;
//   3. coefficients of every p_s and q_s (projection);
//   4. w_ls = (lambda_l <phi_l, p_s>_S - <phi_l, q_s>_S) / 2;
//   5. du/dx_s = sum_l w_ls phi_l (expansion).
// Projections sum 1024-sample chunks in FP32 and the chunks in FP64 in a fixed order,
// so results are reproducible run to run.
#include "vb_internal.cuh"

#include <algorithm>

namespace vb {

constexpr int GP_T = 16;       // projection tile: 16 eigenvectors x 16 vectors per block
constexpr int GP_K = 64;       // samples staged per step
constexpr int GP_CHUNK = 1024; // samples per block (FP32 partial sums)
constexpr int GE_S = 8;        // vectors expanded per pass

// y[r][i]: u (r = 0) and the coordinates x_s (r = 1 + s), each scaled by w_i = S_i^2 / n.
__global__ void grad_stage_kernel(const float* __restrict__ u, const float* __restrict__ x, const double* __restrict__ S,
                                  int64_t n, int m, float* y)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float w = (float)(S[i] * S[i] / (double)n);
    y[i] = w * u[i];
    for (int s = 0; s < m; ++s) y[(int64_t)(1 + s) * n + i] = w * x[i * m + s];
}

// The same scaling for the products p_s, q_s (2m vectors of n, in place).
__global__ void grad_scale_kernel(const double* __restrict__ S, int64_t n, int R, float* y)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float w = (float)(S[i] * S[i] / (double)n);
    for (int r = 0; r < R; ++r) y[(int64_t)r * n + i] *= w;
}

// partial[chunk][j][r] = sum over the chunk's samples of phi_j[i] y_r[i] (FP32 within the chunk).
__global__ void __launch_bounds__(GP_T * GP_T) grad_project_kernel(const float* __restrict__ phi, int64_t n, int L1,
                                                                  const float* __restrict__ y, int R, double* partial)
{
    __shared__ float ph[GP_T][GP_K + 1], ys[GP_T][GP_K + 1];
    const int tj = threadIdx.x / GP_T, tr = threadIdx.x % GP_T;
    const int j0 = blockIdx.x * GP_T, r0 = blockIdx.y * GP_T;
    const int64_t c0 = (int64_t)blockIdx.z * GP_CHUNK;
    float acc = 0.f;
    for (int64_t k0 = c0; k0 < min(n, c0 + GP_CHUNK); k0 += GP_K) {
        for (int e = threadIdx.x; e < GP_T * GP_K; e += blockDim.x) {
            const int row = e / GP_K, col = e % GP_K;
            const int64_t i = k0 + col;
            ph[row][col] = (j0 + row < L1 && i < n) ? phi[(int64_t)(j0 + row) * n + i] : 0.f;
            ys[row][col] = (r0 + row < R && i < n) ? y[(int64_t)(r0 + row) * n + i] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GP_K; ++kk) acc = fmaf(ph[tj][kk], ys[tr][kk], acc);
        __syncthreads();
    }
    if (j0 + tj < L1 && r0 + tr < R)
        partial[((int64_t)blockIdx.z * L1 + j0 + tj) * R + r0 + tr] = (double)acc;
}

// coef[j][r] = sum over chunks, in chunk order.
__global__ void grad_reduce_kernel(const double* __restrict__ partial, int nch, int L1, int R, double* coef)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L1 * R) return;
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += partial[(int64_t)c * L1 * R + e];
    coef[e] = s;
}

// Step 2: per sample a, c and, for GE_S coordinates at a time, b_s, d_s, then p_s and q_s.
// coef: [L1][1 + m] (column 0: u, column 1 + s: x_s).
__global__ void grad_products_kernel(const float* __restrict__ phi, int64_t n, int L1, const double* __restrict__ lam,
                                     const double* __restrict__ coef, int m, float* pq)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int R = 1 + m;
    float a = 0.f, c = 0.f;
    for (int j = 0; j < L1; ++j) {
        const float p = phi[(int64_t)j * n + i];
        const float uj = (float)coef[j * R];
        a = fmaf(uj, p, a);
        c = fmaf((float)lam[j] * uj, p, c);
    }
    for (int s0 = 0; s0 < m; s0 += GE_S) {
        float b[GE_S], d[GE_S];
#pragma unroll
        for (int q = 0; q < GE_S; ++q) { b[q] = 0.f; d[q] = 0.f; }
        for (int j = 0; j < L1; ++j) {
            const float p = phi[(int64_t)j * n + i];
            const float lj = (float)lam[j];
#pragma unroll
            for (int q = 0; q < GE_S; ++q) {
                if (s0 + q < m) {
                    const float vk = (float)coef[j * R + 1 + s0 + q];
                    b[q] = fmaf(vk, p, b[q]);
                    d[q] = fmaf(lj * vk, p, d[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < GE_S; ++q) {
            if (s0 + q < m) {
                pq[(int64_t)(s0 + q) * n + i] = a * b[q];
                pq[(int64_t)(m + s0 + q) * n + i] = fmaf(c, b[q], a * d[q]);
            }
        }
    }
}

// Step 4: w[l][s] = (lambda_l <phi_l, p_s>_S - <phi_l, q_s>_S) / 2; coef2: [L1][2m].
__global__ void grad_weights_kernel(const double* __restrict__ coef2, const double* __restrict__ lam, int L1, int m,
                                    float* w)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L1 * m) return;
    const int l = e / m, s = e - l * m;
    w[e] = (float)(0.5 * (lam[l] * coef2[l * 2 * m + s] - coef2[l * 2 * m + m + s]));
}

// Step 5: grad[i][s] = sum_l w[l][s] phi_l[i], row-major n x m.
__global__ void grad_expand_kernel(const float* __restrict__ phi, int64_t n, int L1, const float* __restrict__ w, int m,
                                   float* grad)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int s0 = 0; s0 < m; s0 += GE_S) {
        float g[GE_S];
#pragma unroll
        for (int q = 0; q < GE_S; ++q) g[q] = 0.f;
        for (int l = 0; l < L1; ++l) {
            const float p = phi[(int64_t)l * n + i];
#pragma unroll
            for (int q = 0; q < GE_S; ++q)
                if (s0 + q < m) g[q] = fmaf(w[l * m + s0 + q], p, g[q]);
        }
#pragma unroll
        for (int q = 0; q < GE_S; ++q)
            if (s0 + q < m) grad[i * m + s0 + q] = g[q];
    }
}

struct GradWs {
    float* y;          // (1 + m) x n, then 2m x n (the products)
    double* partial;   // chunks x L1 x max(1 + m, 2m)
    double* coef1;     // L1 x (1 + m)
    double* coef2;     // L1 x 2m
    float* w;          // L1 x m
};

static size_t grad_plan(Carve& c, int64_t n, int L1, int m, GradWs* out)
{
    const int64_t nch = (n + GP_CHUNK - 1) / GP_CHUNK;
    const int Rmax = std::max(1 + m, 2 * m);
    GradWs t;
    t.y = c.take<float>((size_t)Rmax * n);
    t.partial = c.take<double>((size_t)nch * L1 * Rmax);
    t.coef1 = c.take<double>((size_t)L1 * (1 + m));
    t.coef2 = c.take<double>((size_t)L1 * 2 * m);
    t.w = c.take<float>((size_t)L1 * m);
    if (out) *out = t;
    return c.off;
}

size_t gradient_ws_bytes(int64_t n, int32_t ell, int32_t m)
{
    Carve c(nullptr);
    return grad_plan(c, n, ell + 1, m, nullptr);
}

static void project(cudaStream_t s, const float* phi, int64_t n, int L1, const float* y, int R, double* partial,
                    double* coef)
{
    const int nch = (int)((n + GP_CHUNK - 1) / GP_CHUNK);
    dim3 grid((unsigned)((L1 + GP_T - 1) / GP_T), (unsigned)((R + GP_T - 1) / GP_T), (unsigned)nch);
    grad_project_kernel<<<grid, GP_T * GP_T, 0, s>>>(phi, n, L1, y, R, partial);
    grad_reduce_kernel<<<(unsigned)((L1 * R + 255) / 256), 256, 0, s>>>(partial, nch, L1, R, coef);
}

vb_status gradient_run(Ctx* ctx, int64_t n, int32_t ell, const double* evals, const float* phi, const double* S,
                       const float* u, const float* x, int32_t m, float* grad, void* ws, size_t ws_bytes)
{
    if (!evals || !phi || !S || !u || !x || !grad || n < 1 || ell < 0 || ell > 1023 || m < 1 || m > 128)
        return VB_ERR_ARG;
    if ((int64_t)(n + GP_CHUNK - 1) / GP_CHUNK > 65535) return VB_ERR_UNSUPPORTED;   // grid z
    const int L1 = ell + 1;
    GradWs w;
    Carve c(ws);
    const size_t need = grad_plan(c, n, L1, m, &w);
    if (!ws || ws_bytes < need) return VB_ERR_WORKSPACE;
    cudaStream_t s = ctx->stream;
    const unsigned gn = (unsigned)((n + 255) / 256);
    grad_stage_kernel<<<gn, 256, 0, s>>>(u, x, S, n, m, w.y);
    project(s, phi, n, L1, w.y, 1 + m, w.partial, w.coef1);
    grad_products_kernel<<<gn, 256, 0, s>>>(phi, n, L1, evals, w.coef1, m, w.y);
    grad_scale_kernel<<<gn, 256, 0, s>>>(S, n, 2 * m, w.y);
    project(s, phi, n, L1, w.y, 2 * m, w.partial, w.coef2);
    grad_weights_kernel<<<(unsigned)((L1 * m + 255) / 256), 256, 0, s>>>(w.coef2, evals, L1, m, w.w);
    grad_expand_kernel<<<gn, 256, 0, s>>>(phi, n, L1, w.w, m, grad);
    ctx->launches += 9;
    return last_launch();
}

}  // namespace vb
