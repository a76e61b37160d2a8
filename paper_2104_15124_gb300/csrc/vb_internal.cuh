// Internal declarations shared by the libvb translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/vb.h"

namespace vb {

// Device report block (layout mirrors vb_report; lives in cudaMalloc'd memory of the ctx).
struct DevReport {
    int32_t error;
    int32_t warnings;
    unsigned long long knn_fallback_rows;
    unsigned long long knn_candidates;
    unsigned long long union_big_rows;
    unsigned long long knn_heap_levels;
    unsigned long long knn_tiles_staged;
    unsigned long long knn_insert_rounds;
    unsigned long long knn_retry_tiles;
    unsigned long long knn_rows_short;
    unsigned long long knn_rows_long_run;
    unsigned long long knn_rows_uncertified;
    unsigned long long knn_retry_candidates;
    unsigned long long knn_redo_tiles;
};
static_assert(sizeof(DevReport) == sizeof(vb_report), "report layout");

struct Ctx {
    int device;
    cudaStream_t stream;
    DevReport* rep;        // device
    vb_report* host_rep;   // pinned host mirror
    bool prof = false;
    cudaEvent_t ev[2 * VB_NUM_STAGES] = {};
    unsigned recorded = 0;      // stages with both events recorded since the last read
    long long launches = 0;     // kernels enqueued (host-side count)
};

inline void mark(Ctx* c, int stage, int end)
{
    if (!c->prof) return;
    cudaEventRecord(c->ev[2 * stage + end], c->stream);
    if (end) c->recorded |= 1u << stage;
}

__device__ __forceinline__ void report_error(DevReport* r, int code)
{
    atomicCAS(&r->error, 0, code);
}

// ------------------------------------------------------------------ workspace carving
// A bump allocator over the caller's workspace.  With base == nullptr it only
// measures, so the same plan code gives both the size and the layout.
struct Carve {
    char* base;
    size_t off = 0;
    explicit Carve(void* b) : base((char*)b) {}
    template <class T> T* take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// ------------------------------------------------------------------ warp helpers
__device__ __forceinline__ double warp_sum_f64(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_f32(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// 2^x with the SFU (ex2.approx, flush-to-zero): the hardware instruction, not a library routine.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// log2(x) with the SFU (lg2.approx): the hardware instruction.
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// x^y = 2^(y log2 x) for x > 0 on the SFU; relative error about |y log2 x| 2^-22.
__device__ __forceinline__ float pow_sfu(float x, float y) { return ex2_approx(y * lg2_approx(x)); }

// ------------------------------------------------------------------ point clouds of a batched build
// Cloud b holds the points [ptr[b], ptr[b + 1]) (device array of B + 1 entries);
// B == 1 with ptr == nullptr is the single cloud [0, n).
struct Clouds {
    const int64_t* ptr = nullptr;
    int32_t B = 1;
    const int32_t* id = nullptr;   // optional: the cloud of every point (filled once per batched build)
};
// The cloud that holds point i: the largest b with ptr[b] <= i.
__device__ __forceinline__ int cloud_of(const int64_t* __restrict__ ptr, int B, int64_t i)
{
    if (B <= 1) return 0;
    int lo = 0, hi = B;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ptr[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}
// The same through the per-point table when the build has one.
__device__ __forceinline__ int cloud_id(const Clouds& c, int64_t i)
{
    if (c.B <= 1) return 0;
    return c.id ? c.id[i] : cloud_of(c.ptr, c.B, i);
}
__device__ __forceinline__ int64_t cloud_lo(const Clouds& c, int b) { return c.B <= 1 ? 0 : c.ptr[b]; }
__device__ __forceinline__ int64_t cloud_hi(const Clouds& c, int b, int64_t n) { return c.B <= 1 ? n : c.ptr[b + 1]; }

constexpr float kLog2e = 1.4426950408889634f;
constexpr int kMaxGrid = 64;          // epsilon sweep grid points per launch
constexpr int kRowBlocks = 152 * 8;   // fixed grid of the row passes (deterministic reductions)
constexpr int kRowThreads = 256;

// ------------------------------------------------------------------ launch wrappers (defined per .cu)
// kNN (knn.cu)
size_t gradient_ws_bytes(int64_t n, int32_t ell, int32_t m);
vb_status gradient_run(Ctx* ctx, int64_t n, int32_t ell, const double* evals, const float* phi, const double* S,
                       const float* u, const float* x, int32_t m, float* grad, void* ws, size_t ws_bytes);
size_t knn_plan(Carve& c, int64_t n, int32_t m, const vb_knn_params* p, struct KnnWs* w);
vb_status knn_run(Ctx* ctx, const float* x, int64_t n, int32_t m, const vb_knn_params* p, int32_t* nbr,
                  double* nbr_d2, void* ws, size_t ws_bytes, Clouds cl = Clouds());
// The kNN search's spatial order, for other tile searches (knn.cu): sorted coordinates in FP64
// (exact copies, [.][mp] rows), boxes of 64-point tiles ([ntiles][mp]), perm = sorted
// position -> original index.  The pointers live in the workspace given to order_run.
struct PointOrder {
    const double* xs64;
    const float* tlo;
    const float* thi;
    const uint32_t* perm;
    int mp;
    int64_t ntiles;
};
size_t order_ws_bytes(int64_t n, int32_t m);
vb_status order_run(Ctx* ctx, const float* x, int64_t n, int32_t m, void* ws, size_t ws_bytes, PointOrder* o);
// symmetric union (graph.cu)
size_t graph_plan_bytes(int64_t n, int32_t k);
vb_status graph_run(Ctx* ctx, int64_t n, int32_t k, const int32_t* nbr, const double* nbr_d2, int64_t* row_ptr,
                    int32_t* col, float* ed2, int64_t cap, int64_t* nnz_dev, void* ws, size_t ws_bytes);
vb_status bandwidth_run(Ctx* ctx, int64_t n, int32_t k, int32_t k_bw, const double* nbr_d2, double* b);
// row passes (passes.cu)
// Per-cloud scalars (eps^2, xi_c, chi, dimension) are arrays of cl.B entries (chi: cl.B x G).
size_t sweep_ws_bytes(int64_t n, int B = 1);
vb_status sweep_run(Ctx* ctx, const vb_graph* g, const double* rho, double scale, const double* xi_c_dev,
                    double xi_lo, double xi_hi, double dxi, int warn_bit, double* eps2, double* chi, double* dim,
                    void* ws, size_t ws_bytes, Clouds cl = Clouds());
size_t density_ws_bytes(int64_t n, int B = 1);
vb_status density_run(Ctx* ctx, const vb_graph* g, const double* b, const double* eps2_dev, double d, double beta,
                      double* psi, double* P, void* ws, size_t ws_bytes, Clouds cl = Clouds(), int lpr = 8);
size_t centre_ws_bytes(int64_t n, int B = 1);
vb_status centre_run(Ctx* ctx, const vb_graph* g, const double* b, const double* P, double* xi_c_dev, void* ws,
                     size_t ws_bytes, Clouds cl = Clouds());
size_t kernel_csr_ws_bytes(int64_t n, int B = 1);
vb_status kernel_csr_run(Ctx* ctx, const vb_graph* g, const double* psi, const double* P, const vb_op_params* op,
                         const double* eps2_op_dev, float* val, double* q, double* D, double* S, void* ws,
                         size_t ws_bytes, Clouds cl = Clouds(), int lpr = 8);
size_t spmv_ws_bytes(int64_t n);
vb_status spmv_lap_launch(cudaStream_t s, const vb_graph* g, const float* val, const double* S, float alpha,
                          const float* x, float beta, float* y, double* z, float* sf);
vb_status spmv_run(Ctx* ctx, const vb_graph* g, const float* val, const double* S, int mode, float alpha,
                   const float* x, float beta, float* y, void* ws, size_t ws_bytes);

// learned radius (mlp.cu): R2[pos] = (inflate exp(net(xs[pos]) + shift + cloud_shift[cloud]))^2
// for sorted points (sorted positions keep the clouds' ranges)
vb_status mlp_radius_r2(cudaStream_t s, const vb_mlp* mlp, const float* xs, int64_t n, int m, int mp, float shift,
                        float inflate, float* r2, const float* cloud_shift, Clouds cl, DevReport* rep);

// eigen-solve (solve.cu)
size_t solve_ws_bytes(int64_t n, int64_t cap, const vb_solve_params* p);
vb_status solve_run(Ctx* ctx, const vb_graph* g, int64_t cap, const float* val, const double* S,
                    const vb_solve_params* p, double* evals, float* phi, const float* rhs, float* f, int32_t* iters,
                    void* ws, size_t ws_bytes);

// the delta_tol radius pattern and its per-grid-point sweep (radius.cu)
size_t radius_ws_bytes(int64_t n, int32_t m);
vb_status radius_pattern_run(Ctx* ctx, const float* x, int64_t n, int32_t m, const double* rho, double eps2,
                             double delta_tol, int64_t* row_ptr, int32_t* col, double* d2, int64_t cap,
                             int64_t* nnz_dev, void* ws, size_t ws_bytes);
vb_status radius_sweep_run(Ctx* ctx, const float* x, int64_t n, int32_t m, const double* rho, double scale,
                           double xi_lo, double xi_hi, double dxi, double delta_tol, double* chi, double* eps2,
                           double* dim, void* ws, size_t ws_bytes);

// particle evolution (evolve.cu): gc = g - mean(g); the explicit sample update
vb_status evolve_centre_launch(cudaStream_t s, const float* g, int64_t n, float* gc);
vb_status evolve_update_launch(cudaStream_t s, const float* x, int64_t n, int m, const float* u, const float* grad,
                               const float* sigma, const float* W, double dt, float* x_next);

// exclusive scan of n int32 counts into n + 1 int64 offsets (graph.cu)
size_t scan_ws_bytes(int64_t n);
vb_status scan_counts(cudaStream_t s, const int32_t* counts, int64_t n, int64_t* out, void* ws);

inline vb_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VB_OK : VB_ERR_CUDA; }
inline vb_status last_launch() { return cuda_status(cudaGetLastError()); }

}  // namespace vb
