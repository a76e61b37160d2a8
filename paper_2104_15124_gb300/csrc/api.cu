// The extern "C" boundary of libvb (declared in include/vb.h): argument checks,
// device selection, workspace sizing and the ordering of the launches.
#include "vb_internal.cuh"

#include <algorithm>
#include <new>

using namespace vb;

namespace {

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

Ctx* C(vb_ctx* c) { return reinterpret_cast<Ctx*>(c); }

// A batched build keeps the cloud of every point at the front of the workspace.
size_t cloud_id_bytes(int64_t n, int B) { return B > 1 ? (((size_t)n * sizeof(int32_t) + 255) & ~(size_t)255) : 0; }

size_t build_ws(int64_t n, int32_t m, const vb_build_params* p, int B = 1)
{
    Carve c(nullptr);
    size_t knn = knn_plan(c, n, m, &p->knn, nullptr);
    size_t s = std::max({knn, graph_plan_bytes(n, p->knn.k), sweep_ws_bytes(n, B), density_ws_bytes(n, B),
                         centre_ws_bytes(n, B), kernel_csr_ws_bytes(n, B)});
    return s + cloud_id_bytes(n, B);
}

__global__ void cloud_id_kernel(const int64_t* __restrict__ ptr, int B, int64_t n, int32_t* id)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) id[i] = cloud_of(ptr, B, i);
}

// The chain a0-a13 for one cloud (cl.B == 1) or a batch of clouds.
vb_status build_run(Ctx* c, const float* x, int64_t n, int32_t m, const vb_build_params* p, const vb_build_out* o,
                    void* ws, size_t ws_bytes, Clouds cl)
{
    const int32_t k = p->knn.k;
    const int32_t k_bw = p->k_bw > 0 ? p->k_bw : k;
    if (k_bw > k) return VB_ERR_ARG;
    if (!ws || ws_bytes < build_ws(n, m, p, cl.B)) return VB_ERR_WORKSPACE;
    if (cl.B > 1) {
        int32_t* id = (int32_t*)ws;
        const size_t off = cloud_id_bytes(n, cl.B);
        cloud_id_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(cl.ptr, cl.B, n, id);
        c->launches += 1;
        cl.id = id;
        ws = (char*)ws + off;
        ws_bytes -= off;
    }
    vb_status st = knn_run(c, x, n, m, &p->knn, o->nbr, o->nbr_d2, ws, ws_bytes, cl);
    if (st) return st;
    st = graph_run(c, n, k, o->nbr, o->nbr_d2, o->row_ptr, o->col, o->ed2, o->cap, o->nnz, ws, ws_bytes);
    if (st) return st;
    st = bandwidth_run(c, n, k, k_bw, o->nbr_d2, o->b);
    if (st) return st;
    vb_graph gr{n, o->row_ptr, o->col, o->ed2};
    if (!p->pin_eps) {
        st = sweep_run(c, &gr, o->b, 1.0, nullptr, p->xi_lo, p->xi_hi, p->dxi, 1, o->eps2_den, o->chi_den, o->dim_den,
                       ws, ws_bytes, cl);
        if (st) return st;
    }
    st = density_run(c, &gr, o->b, o->eps2_den, p->op.d, p->op.beta, o->psi, o->P, ws, ws_bytes, cl);
    if (st) return st;
    st = centre_run(c, &gr, o->b, o->P, o->xi_c, ws, ws_bytes, cl);
    if (st) return st;
    if (!p->pin_eps) {
        st = sweep_run(c, &gr, o->P, 4.0, o->xi_c, p->xi_lo, p->xi_hi, p->dxi, 2, o->eps2_op, o->chi_op, o->dim_op, ws,
                       ws_bytes, cl);
        if (st) return st;
    }
    return kernel_csr_run(c, &gr, o->psi, o->P, &p->op, o->eps2_op, o->val, o->q, o->D, o->S, ws, ws_bytes, cl);
}

}  // namespace

extern "C" {

const char* vb_status_string(vb_status s)
{
    switch (s) {
        case VB_OK: return "ok";
        case VB_ERR_ARG: return "invalid argument";
        case VB_ERR_CUDA: return "CUDA error";
        case VB_ERR_WORKSPACE: return "workspace too small";
        case VB_ERR_DEGENERATE: return "degenerate input (zero bandwidth or non-finite coordinate)";
        case VB_ERR_EPS_BOUNDARY: return "epsilon at the end of its grid";
        case VB_ERR_NOT_CONVERGED: return "eigen-solver did not converge";
        case VB_ERR_TIMEOUT: return "device-side wait timed out";
        case VB_ERR_BOUNDS: return "index out of bounds";
        case VB_ERR_UNSUPPORTED: return "unsupported request";
        default: return "unknown status";
    }
}

vb_status vb_create(vb_ctx** out, int32_t device, void* stream)
{
    if (!out) return VB_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return VB_ERR_ARG;
    DeviceGuard g(device);
    if (!g.ok) return VB_ERR_CUDA;
    Ctx* c = new (std::nothrow) Ctx();
    if (!c) return VB_ERR_CUDA;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (cudaMalloc(&c->rep, sizeof(DevReport)) != cudaSuccess) { delete c; return VB_ERR_CUDA; }
    if (cudaMallocHost(&c->host_rep, sizeof(vb_report)) != cudaSuccess) {
        cudaFree(c->rep);
        delete c;
        return VB_ERR_CUDA;
    }
    if (cudaMemsetAsync(c->rep, 0, sizeof(DevReport), c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaFree(c->rep);
        cudaFreeHost(c->host_rep);
        delete c;
        return VB_ERR_CUDA;
    }
    *out = reinterpret_cast<vb_ctx*>(c);
    return VB_OK;
}

vb_status vb_destroy(vb_ctx* ctx)
{
    if (!ctx) return VB_ERR_ARG;
    Ctx* c = C(ctx);
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    cudaFree(c->rep);
    cudaFreeHost(c->host_rep);
    delete c;
    return VB_OK;
}

vb_status vb_set_stream(vb_ctx* ctx, void* stream)
{
    if (!ctx) return VB_ERR_ARG;
    C(ctx)->stream = (cudaStream_t)stream;
    return VB_OK;
}

vb_status vb_report_read(vb_ctx* ctx, vb_report* out)
{
    if (!ctx || !out) return VB_ERR_ARG;
    Ctx* c = C(ctx);
    DeviceGuard g(c->device);
    if (cudaMemcpyAsync(c->host_rep, c->rep, sizeof(vb_report), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return VB_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return VB_ERR_CUDA;
    *out = *c->host_rep;
    return VB_OK;
}

vb_status vb_report_reset(vb_ctx* ctx)
{
    if (!ctx) return VB_ERR_ARG;
    Ctx* c = C(ctx);
    DeviceGuard g(c->device);
    return cuda_status(cudaMemsetAsync(c->rep, 0, sizeof(DevReport), c->stream));
}

vb_status vb_profile_enable(vb_ctx* ctx, int32_t on)
{
    if (!ctx) return VB_ERR_ARG;
    Ctx* c = C(ctx);
    DeviceGuard g(c->device);
    if (on && !c->ev[0]) {
        for (auto& e : c->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return VB_ERR_CUDA;
    }
    c->prof = on != 0;
    c->recorded = 0;
    c->launches = 0;
    return VB_OK;
}

vb_status vb_profile_read(vb_ctx* ctx, float* ms, int64_t* launches)
{
    if (!ctx) return VB_ERR_ARG;
    Ctx* c = C(ctx);
    DeviceGuard g(c->device);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return VB_ERR_CUDA;
    if (ms) {
        for (int s = 0; s < VB_NUM_STAGES; ++s) {
            ms[s] = -1.f;
            if (c->ev[0] && (c->recorded >> s & 1u)) {
                float t = 0.f;
                if (cudaEventElapsedTime(&t, c->ev[2 * s], c->ev[2 * s + 1]) == cudaSuccess) ms[s] = t;
            }
        }
        c->recorded = 0;
    }
    if (launches) *launches = c->launches;
    return VB_OK;
}

size_t vb_knn_workspace(int64_t n, int32_t m, const vb_knn_params* p)
{
    Carve c(nullptr);
    return knn_plan(c, n, m, p, nullptr);
}

vb_status vb_knn(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const vb_knn_params* p, int32_t* nbr,
                 double* nbr_d2, void* ws, size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return knn_run(C(ctx), x, n, m, p, nbr, nbr_d2, ws, ws_bytes);
}

size_t vb_graph_workspace(int64_t n, int32_t k) { return graph_plan_bytes(n, k); }

vb_status vb_graph_build(vb_ctx* ctx, int64_t n, int32_t k, const int32_t* nbr, const double* nbr_d2,
                         int64_t* row_ptr, int32_t* col, float* ed2, int64_t cap, int64_t* nnz_dev, void* ws,
                         size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return graph_run(C(ctx), n, k, nbr, nbr_d2, row_ptr, col, ed2, cap, nnz_dev, ws, ws_bytes);
}

vb_status vb_bandwidth(vb_ctx* ctx, int64_t n, int32_t k, int32_t k_bw, const double* nbr_d2, double* b)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return bandwidth_run(C(ctx), n, k, k_bw, nbr_d2, b);
}

size_t vb_epsilon_tune_workspace(int64_t n) { return sweep_ws_bytes(n); }

vb_status vb_epsilon_tune(vb_ctx* ctx, const vb_graph* gr, const double* rho, double scale, const double* xi_c_dev,
                          double xi_lo, double xi_hi, double dxi, int32_t warn_bit, double* eps2_dev, double* chi_dev,
                          double* dim_est_dev, void* ws, size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return sweep_run(C(ctx), gr, rho, scale, xi_c_dev, xi_lo, xi_hi, dxi, warn_bit, eps2_dev, chi_dev, dim_est_dev, ws,
                     ws_bytes);
}

size_t vb_density_workspace(int64_t n) { return density_ws_bytes(n); }

vb_status vb_density(vb_ctx* ctx, const vb_graph* gr, const double* b, const double* eps2_dev, double d, double beta,
                     double* psi, double* P, void* ws, size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return density_run(C(ctx), gr, b, eps2_dev, d, beta, psi, P, ws, ws_bytes);
}

size_t vb_operator_centre_workspace(int64_t n) { return centre_ws_bytes(n); }

vb_status vb_operator_centre(vb_ctx* ctx, const vb_graph* gr, const double* b, const double* P, double* xi_c_dev,
                             void* ws, size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return centre_run(C(ctx), gr, b, P, xi_c_dev, ws, ws_bytes);
}

size_t vb_kernel_csr_workspace(int64_t n) { return kernel_csr_ws_bytes(n); }

vb_status vb_kernel_csr(vb_ctx* ctx, const vb_graph* gr, const double* psi, const double* P, const vb_op_params* op,
                        const double* eps2_op_dev, float* val, double* q, double* D, double* S, void* ws,
                        size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return kernel_csr_run(C(ctx), gr, psi, P, op, eps2_op_dev, val, q, D, S, ws, ws_bytes);
}

size_t vb_spmv_workspace(int64_t n) { return spmv_ws_bytes(n); }

vb_status vb_spmv(vb_ctx* ctx, const vb_graph* gr, const float* val, const double* S, int32_t mode, float alpha,
                  const float* x, float beta, float* y, void* ws, size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return spmv_run(C(ctx), gr, val, S, mode, alpha, x, beta, y, ws, ws_bytes);
}

size_t vb_gradient_workspace(int64_t n, int32_t ell, int32_t m) { return gradient_ws_bytes(n, ell, m); }

vb_status vb_gradient(vb_ctx* ctx, int64_t n, int32_t ell, const double* evals, const float* phi, const double* S,
                      const float* u, const float* x, int32_t m, float* grad, void* ws, size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return gradient_run(C(ctx), n, ell, evals, phi, S, u, x, m, grad, ws, ws_bytes);
}

size_t vb_solve_workspace(int64_t n, int64_t cap, const vb_solve_params* p) { return solve_ws_bytes(n, cap, p); }

vb_status vb_solve(vb_ctx* ctx, const vb_graph* gr, int64_t cap, const float* val, const double* S,
                   const vb_solve_params* p, double* evals, float* phi, const float* g_rhs, float* f, int32_t* iters,
                   void* ws, size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return solve_run(C(ctx), gr, cap, val, S, p, evals, phi, g_rhs, f, iters, ws, ws_bytes);
}

size_t vb_build_workspace(int64_t n, int32_t m, const vb_build_params* p)
{
    if (!p) return 0;
    return build_ws(n, m, p);
}

vb_status vb_build(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const vb_build_params* p,
                   const vb_build_out* o, void* ws, size_t ws_bytes)
{
    if (!ctx || !p || !o) return VB_ERR_ARG;
    Ctx* c = C(ctx);
    DeviceGuard g(c->device);
    if (!g.ok) return VB_ERR_CUDA;
    return build_run(c, x, n, m, p, o, ws, ws_bytes, Clouds());
}

size_t vb_build_batch_workspace(int64_t n, int32_t m, int32_t B, const vb_build_params* p)
{
    if (!p || B < 1) return 0;
    return build_ws(n, m, p, B);
}

vb_status vb_build_batch(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const int64_t* cloud_ptr_host,
                         const int64_t* cloud_ptr_dev, int32_t B, const vb_build_params* p, const vb_build_out* o,
                         void* ws, size_t ws_bytes)
{
    if (!ctx || !p || !o || !cloud_ptr_host || !cloud_ptr_dev || B < 1) return VB_ERR_ARG;
    if (cloud_ptr_host[0] != 0 || cloud_ptr_host[B] != n) return VB_ERR_ARG;
    for (int32_t b = 0; b < B; ++b)
        if (cloud_ptr_host[b + 1] - cloud_ptr_host[b] < (int64_t)p->knn.k + 1) return VB_ERR_ARG;
    Ctx* c = C(ctx);
    DeviceGuard g(c->device);
    if (!g.ok) return VB_ERR_CUDA;
    Clouds cl;
    cl.ptr = cloud_ptr_dev;
    cl.B = B;
    return build_run(c, x, n, m, p, o, ws, ws_bytes, cl);
}

size_t vb_radius_workspace(int64_t n, int32_t m) { return radius_ws_bytes(n, m); }

vb_status vb_radius_pattern(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const double* rho, double eps2,
                            double delta_tol, int64_t* row_ptr, int32_t* col, double* d2, int64_t cap,
                            int64_t* nnz_dev, void* ws, size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return radius_pattern_run(C(ctx), x, n, m, rho, eps2, delta_tol, row_ptr, col, d2, cap, nnz_dev, ws, ws_bytes);
}

vb_status vb_radius_sweep(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const double* rho, double scale,
                          double xi_lo, double xi_hi, double dxi, double delta_tol, double* chi_dev, double* eps2_dev,
                          double* dim_est_dev, void* ws, size_t ws_bytes)
{
    if (!ctx) return VB_ERR_ARG;
    DeviceGuard g(C(ctx)->device);
    if (!g.ok) return VB_ERR_CUDA;
    return radius_sweep_run(C(ctx), x, n, m, rho, scale, xi_lo, xi_hi, dxi, delta_tol, chi_dev, eps2_dev,
                            dim_est_dev, ws, ws_bytes);
}

size_t vb_evolve_workspace(int64_t n, int32_t m, const vb_evolve_params* p)
{
    if (!p || n < 2 || m < 1) return 0;
    const int64_t cap = n * (2 * (int64_t)p->build.knn.k + 1);
    const int32_t ell = p->solve.ell;
    Carve c(nullptr);
    c.take<float>(n);                            // centred source
    c.take<double>(ell + 1);                     // eigenvalues
    c.take<float>((size_t)(ell + 1) * n);        // eigenvectors
    const size_t stages = std::max({build_ws(n, m, &p->build), solve_ws_bytes(n, cap, &p->solve),
                                    gradient_ws_bytes(n, ell, m)});
    return c.off + stages + 256;
}

vb_status vb_evolve_step(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const vb_evolve_params* p,
                         const float* u, const float* sigma, const float* W, const float* g, const vb_build_out* o,
                         float* f, float* grad, float* x_next, void* ws, size_t ws_bytes)
{
    if (!ctx || !p || !o || !x || !sigma || !W || !g || !f || !grad || !x_next) return VB_ERR_ARG;
    if (!(p->dt > 0) || p->build.op.c != 1.0 || p->solve.ell < 1 || n < 2 || m < 1 || m > 128) return VB_ERR_ARG;
    if (x_next == x || o->cap < n * (2 * (int64_t)p->build.knn.k + 1)) return VB_ERR_ARG;
    if (!ws || ws_bytes < vb_evolve_workspace(n, m, p)) return VB_ERR_WORKSPACE;
    Ctx* c = C(ctx);
    DeviceGuard dg(c->device);
    if (!dg.ok) return VB_ERR_CUDA;
    const int32_t ell = p->solve.ell;
    Carve cv(ws);
    float* gc = cv.take<float>(n);
    double* evals = cv.take<double>(ell + 1);
    float* phi = cv.take<float>((size_t)(ell + 1) * n);
    void* rest = (char*)ws + ((cv.off + 255) & ~(size_t)255);
    const size_t rest_bytes = ws_bytes - ((cv.off + 255) & ~(size_t)255);
    // L_{1,psi} on the current samples
    vb_status st = build_run(c, x, n, m, &p->build, o, rest, rest_bytes, Clouds());
    if (st) return st;
    // f with L_{1,psi} f = g - mean(g) over ell eigenpairs (Sec. 3.1), then grad f (Sec. 3.2)
    st = evolve_centre_launch(c->stream, g, n, gc);
    if (st) return st;
    vb_graph gr{n, o->row_ptr, o->col, o->ed2};
    int32_t iters = 0;
    const vb_status solved = solve_run(c, &gr, o->cap, o->val, o->S, &p->solve, evals, phi, gc, f, &iters, rest,
                                       rest_bytes);
    if (solved != VB_OK && solved != VB_ERR_NOT_CONVERGED) return solved;
    st = gradient_run(c, n, ell, evals, phi, o->S, f, x, m, grad, rest, rest_bytes);
    if (st) return st;
    st = evolve_update_launch(c->stream, x, n, m, u, grad, sigma, W, p->dt, x_next);
    c->launches += 2;
    return st != VB_OK ? st : solved;
}

}  // extern "C"
