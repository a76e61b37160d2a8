// Launch-shape autotuner of the kNN search (part of the batched build, a16): the
// heap depth k + margin and the seed window decide the shared memory of a query
// tile, hence how many tiles an SM holds, against how early the pruning bound
// tightens; the best pair depends on m, k, the precision and the size, so it is
// measured on the caller's input and cached per (m, k, precision, prune, log2 n).
// For 16-bit tiles the choice also covers the kernel (staged or pipelined).
#include "vb_internal.cuh"

#include <map>
#include <mutex>
#include <tuple>

namespace {

using Key = std::tuple<int, int, int, int, int>;
struct Shape {
    int margin, seed_tiles, tc_variant;
};
std::map<Key, Shape> g_cache;
std::mutex g_mu;

int log2_floor(int64_t n)
{
    int b = 0;
    while ((n >> (b + 1)) > 0) ++b;
    return b;
}

}  // namespace

using namespace vb;

extern "C" vb_status vb_knn_autotune(vb_ctx* ctx, const float* x, int64_t n, int32_t m,
                                     const int64_t* cloud_ptr_dev, int32_t B, const vb_knn_params* p, int32_t* nbr,
                                     double* nbr_d2, void* ws, size_t ws_bytes, vb_knn_params* best, float* best_ms)
{
    if (!ctx || !p || !best || !best_ms || B < 1 || (B > 1 && !cloud_ptr_dev)) return VB_ERR_ARG;
    Clouds cl;
    cl.ptr = B > 1 ? cloud_ptr_dev : nullptr;
    cl.B = B;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    int dev_prev = -1;
    if (cudaGetDevice(&dev_prev) != cudaSuccess) return VB_ERR_CUDA;
    if (dev_prev != c->device && cudaSetDevice(c->device) != cudaSuccess) return VB_ERR_CUDA;
    struct Restore {
        int d, cur;
        ~Restore()
        {
            if (d >= 0 && d != cur) cudaSetDevice(d);
        }
    } restore{dev_prev, c->device};

    const Key key{m, p->k, p->precision, p->prune, log2_floor(n / B)};
    *best = *p;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            best->margin = it->second.margin;
            best->seed_tiles = it->second.seed_tiles;
            best->tc_variant = it->second.tc_variant;
            *best_ms = 0.f;
            return VB_OK;
        }
    }
    const bool fp32 = p->precision == VB_PREC_FP32;
    // margin 2 only for the FP32 search (its certificate band is ~1e-6 relative; 16-bit bands need more)
    const int margins[] = {2, 4, 8, 16, 32};
    const int seeds_fp32[] = {1, 2, 3};
    const int seeds_tc[] = {0};
    // 16-bit tiles: both kernels; the FP32 search has one
    const int variants_tc[] = {VB_TC_PIPELINED, VB_TC_STAGED};
    const int nv = fp32 ? 1 : 2;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return VB_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return VB_ERR_CUDA; }
    float bms = INFINITY;
    Shape bs{p->margin, p->seed_tiles, p->tc_variant};
    vb_status st = VB_OK;
    const bool prof = c->prof;
    c->prof = false;
    for (int mg : margins) {
        if (p->k + mg > 256 || (mg < 4 && !fp32)) continue;
        const int* seeds = fp32 && p->prune != VB_PRUNE_LEARNED ? seeds_fp32 : seeds_tc;
        const int ns = fp32 && p->prune != VB_PRUNE_LEARNED ? 3 : 1;
        for (int vs = 0; vs < nv * ns; ++vs) {
            const int vi = vs / ns, si = vs % ns;
            vb_knn_params q = *p;
            q.dbg_d2 = nullptr;   // the diagnostic rows are sized for the caller's margin only
            q.dbg_idx = nullptr;
            q.margin = mg;
            q.seed_tiles = seeds[si];
            if (!fp32) q.tc_variant = variants_tc[vi];
            float t = INFINITY;
            for (int rep = 0; rep < 3 && st == VB_OK; ++rep) {   // the first run warms up
                cudaEventRecord(e0, c->stream);
                st = knn_run(c, x, n, m, &q, nbr, nbr_d2, ws, ws_bytes, cl);
                cudaEventRecord(e1, c->stream);
                if (st != VB_OK) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) { st = VB_ERR_CUDA; break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) t = fminf(t, ms);
            }
            if (st == VB_ERR_UNSUPPORTED) { st = VB_OK; continue; }   // shape too large for this kernel
            if (st != VB_OK) break;
            if (t < bms) { bms = t; bs = Shape{mg, seeds[si], q.tc_variant}; }
        }
        if (st != VB_OK) break;
    }
    c->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != VB_OK) return st;
    if (!(bms < INFINITY)) return VB_ERR_UNSUPPORTED;
    // leave the outputs holding the chosen shape's result (identical in any case: the search is exact)
    vb_knn_params q = *p;
    q.dbg_d2 = nullptr;
    q.dbg_idx = nullptr;
    q.margin = bs.margin;
    q.seed_tiles = bs.seed_tiles;
    q.tc_variant = bs.tc_variant;
    st = knn_run(c, x, n, m, &q, nbr, nbr_d2, ws, ws_bytes, cl);
    if (st != VB_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = bs;
    }
    best->margin = bs.margin;
    best->seed_tiles = bs.seed_tiles;
    best->tc_variant = bs.tc_variant;
    *best_ms = bms;
    return cuda_status(cudaStreamSynchronize(c->stream));
}
