// The sample update of the particle evolution of a time-dependent density (Sec. 6,
// "Evolution of a time-dependent density"): the samples of psi(.; t) follow
// dX = (u - grad f) dt + sigma dW, with f the solution of L_{1,psi} f = g on the
// current samples, and one explicit step is
//     x_{t+dt} = x_t + dt (u - grad f) + sqrt(dt) sigma W,  W ~ N(0, I)
// (Eq. discrete sample evolution).  The operator, the solve and grad f come from
// the build, vb_solve and vb_gradient; this file holds the two small kernels of a
// step: the centring of the source, g - mean(g) (the sample mean standing for the
// expectation under psi(.; t)), and the update itself.  The Gaussian draws W are
// inputs, so a step is a deterministic function of its arguments.
#include "vb_internal.cuh"

namespace vb {

constexpr int kCentreThreads = 1024;

// gc = g - mean(g), one block: FP64 partial sums per thread over a fixed stride, then a
// fixed tree, so the mean is the same bits run to run.
__global__ void __launch_bounds__(kCentreThreads) centre_source_kernel(const float* __restrict__ g, int64_t n,
                                                                       float* gc)
{
    __shared__ double part[kCentreThreads];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int64_t i = t; i < n; i += kCentreThreads) s += (double)g[i];
    part[t] = s;
    __syncthreads();
    for (int w = kCentreThreads / 2; w > 0; w >>= 1) {
        if (t < w) part[t] += part[t + w];
        __syncthreads();
    }
    const double mean = part[0] / (double)n;
    for (int64_t i = t; i < n; i += kCentreThreads) gc[i] = (float)((double)g[i] - mean);
}

// x_next[i][a] = x[i][a] + dt (u[i][a] - grad[i][a]) + sqrt(dt) sum_b sigma[a][b] W[i][b],
// in FP64, rounded once to FP32.  One thread per coordinate.
__global__ void evolve_update_kernel(const float* __restrict__ x, int64_t n, int m, const float* __restrict__ u,
                                     const float* __restrict__ grad, const float* __restrict__ sigma,
                                     const float* __restrict__ W, double dt, double sdt, float* x_next)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    const int64_t i = e / m;
    const int a = (int)(e - i * m);
    double noise = 0.0;
    for (int b = 0; b < m; ++b) noise += (double)sigma[a * m + b] * (double)W[i * m + b];
    const double drift = (u ? (double)u[e] : 0.0) - (double)grad[e];
    x_next[e] = (float)((double)x[e] + dt * drift + sdt * noise);
}

vb_status evolve_centre_launch(cudaStream_t s, const float* g, int64_t n, float* gc)
{
    centre_source_kernel<<<1, kCentreThreads, 0, s>>>(g, n, gc);
    return last_launch();
}

vb_status evolve_update_launch(cudaStream_t s, const float* x, int64_t n, int m, const float* u, const float* grad,
                               const float* sigma, const float* W, double dt, float* x_next)
{
    const int64_t total = n * m;
    evolve_update_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(x, n, m, u, grad, sigma, W, dt, sqrt(dt),
                                                                         x_next);
    return last_launch();
}

}  // namespace vb
