// vb_spmv_laplacian_noalloc: the difference-form SpMV with its scratch in a
// static device array, for callers that cannot allocate device memory.
//
// Who needs it: code that applies L-hat from inside a CUDA stream capture (an
// eigen-solver loop recorded into a CUDA graph, where cudaMalloc is not
// allowed), host runtimes that hand this library only pre-existing buffers,
// and embeddings that run under a fixed device-memory budget.  They still
// pass their inputs and outputs; only the scratch moves into the library.
//
// The scratch (z = x / S in FP64 and S in FP32, 12 bytes per row) lives in
// the file-scope array g_lap_scratch, sized for VB_NOALLOC_MAX_N rows; every
// GPU that loads libvb holds it (about 12.6 MB) until the process exits.  Host
// code cannot use the array's name as a device address, so the first call on
// each device, with that device current, resolves it once with
// cudaGetSymbolAddress and caches the result.
#include "vb_internal.cuh"

#include <mutex>

namespace {

constexpr int64_t kMaxN = VB_NOALLOC_MAX_N;
constexpr size_t kZBytes = ((size_t)kMaxN * sizeof(double) + 255) & ~(size_t)255;
constexpr size_t kScratchBytes = kZBytes + (size_t)kMaxN * sizeof(float);

static __device__ __align__(256) unsigned char g_lap_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_lap_scratch on the current device (resolved once per device).
vb_status scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VB_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lap_scratch) != cudaSuccess || !p) return VB_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return VB_OK;
}

}  // namespace

extern "C" vb_status vb_spmv_laplacian_noalloc(void* stream, const vb_graph* g, const float* val, const double* S,
                                               float alpha, const float* x, float beta, float* y)
{
    if (!g || !g->row_ptr || !g->col || !val || !S || !x || !y || x == y || g->n < 1) return VB_ERR_ARG;
    if (g->n > kMaxN) return VB_ERR_UNSUPPORTED;   // larger graphs need vb_spmv with a workspace
    void* base = nullptr;
    vb_status st = scratch_address(&base);
    if (st != VB_OK) return st;
    double* z = (double*)base;
    float* sf = (float*)((char*)base + kZBytes);
    return vb::spmv_lap_launch((cudaStream_t)stream, g, val, S, alpha, x, beta, y, z, sf);
}
