// Symmetric sparsity pattern (step a6) and the bandwidth function (step a8).
//
// a6: E = {(i, i)} U {(i, j): j in N_k(i) or i in N_k(j)} as CSR with rows
//     sorted by column.  Algorithm 1 keeps the diagonal (its inner loop
//     starts at j = i) and sets K^ij and K^ji together, so every kNN pair
//     enters in both directions.  Construction: in-degree count (int
//     atomics) -> exclusive scan -> scatter of own and transposed entries
//     into raw rows -> per-row sort by column and de-duplication (one warp
//     per row in shared memory; one block per row for rows longer than the
//     warp limit) -> scan of the unique counts -> compaction.  The FP32
//     squared distance of every entry is the FP32 rounding of the canonical
//     FP64 value, identical for (i, j) and (j, i).
// a8: b_i^2 = sum_{r=1}^{k_bw} d2(i, I(i, r)) in rank order, FP64 (Eq.
//     bandwidth parameter).
#include "vb_internal.cuh"

#include <algorithm>

namespace vb {

constexpr int ROW_CAP = 512;        // warp path: raw entries per row held in shared memory
constexpr int BIG_CAP = 8192;       // block path: raw entries per row
constexpr int SORT_WARPS = 4;
constexpr int SCAN_T = 1024;
constexpr int SCAN_ITEMS = 8;       // counts per thread per scan block

// ------------------------------------------------------------------ exclusive scan int32 -> int64[n+1]
size_t scan_ws_bytes(int64_t n)
{
    int64_t nb = (n + SCAN_T * SCAN_ITEMS - 1) / (SCAN_T * SCAN_ITEMS);
    return (size_t)(nb + 1) * sizeof(int64_t) + 256;
}

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total)
{
    // 1024 threads: warp inclusive scans, then a scan of the 32 warp totals
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = sh[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    int64_t r = x - v + (w ? sh[w - 1] : 0);
    if (total) *total = sh[31];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_T) scan_reduce_kernel(const int32_t* __restrict__ c, int64_t n, int64_t* bsum)
{
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_T * SCAN_ITEMS;
    int64_t s = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t e = base + (int64_t)i * SCAN_T + threadIdx.x;
        if (e < n) s += c[e];
    }
    int64_t tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) scan_top_kernel(int64_t* bsum, int64_t nb)
{
    __shared__ int64_t sh[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_T) {
        int64_t i = b0 + threadIdx.x;
        int64_t v = i < nb ? bsum[i] : 0;
        int64_t tot;
        int64_t ex = block_excl_scan(v, sh, &tot);
        if (i < nb) bsum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(SCAN_T) scan_apply_kernel(const int32_t* __restrict__ c, int64_t n,
                                                           const int64_t* __restrict__ bsum, int64_t nb, int64_t* out)
{
    __shared__ int64_t sh[32];
    // each thread owns SCAN_ITEMS consecutive counts of the block's chunk
    int64_t base = (int64_t)blockIdx.x * SCAN_T * SCAN_ITEMS + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? c[base + i] : 0;
        s += v[i];
    }
    int64_t run = bsum[blockIdx.x] + block_excl_scan(s, sh, nullptr);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bsum[nb];
}

vb_status scan_counts(cudaStream_t s, const int32_t* counts, int64_t n, int64_t* out, void* ws)
{
    int64_t nb = (n + SCAN_T * SCAN_ITEMS - 1) / (SCAN_T * SCAN_ITEMS);
    int64_t* bsum = (int64_t*)ws;
    scan_reduce_kernel<<<(unsigned)nb, SCAN_T, 0, s>>>(counts, n, bsum);
    scan_top_kernel<<<1, SCAN_T, 0, s>>>(bsum, nb);
    scan_apply_kernel<<<(unsigned)nb, SCAN_T, 0, s>>>(counts, n, bsum, nb, out);
    return last_launch();
}

// ------------------------------------------------------------------ a6
struct GraphWs {
    int32_t* indeg;    // n, then reused as transposed fill counters
    int32_t* fill;     // n
    int32_t* cnt;      // n raw counts, then unique counts
    int64_t* raw_ptr;  // n + 1
    int32_t* raw_col;  // n (2k + 1)
    float* raw_d2;     // n (2k + 1)
    int32_t* big;      // n (rows for the block path)
    int32_t* nbig;     // 1
    void* scan;        // scan_ws_bytes(n)
};

static size_t graph_plan(Carve& c, int64_t n, int32_t k, GraphWs* w)
{
    GraphWs t;
    t.indeg = c.take<int32_t>(n);
    t.fill = c.take<int32_t>(n);
    t.cnt = c.take<int32_t>(n);
    t.raw_ptr = c.take<int64_t>(n + 1);
    t.raw_col = c.take<int32_t>(n * (2 * (int64_t)k + 1));
    t.raw_d2 = c.take<float>(n * (2 * (int64_t)k + 1));
    t.big = c.take<int32_t>(n);
    t.nbig = c.take<int32_t>(1);
    t.scan = c.take<char>(scan_ws_bytes(n));
    if (w) *w = t;
    return c.off;
}
size_t graph_plan_bytes(int64_t n, int32_t k)
{
    Carve c(nullptr);
    return graph_plan(c, n, k, nullptr);
}

__global__ void zero_i32_kernel(int32_t* a, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = 0;
}

__global__ void indeg_kernel(const int32_t* __restrict__ nbr, int64_t nk, int32_t* indeg)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nk) atomicAdd(&indeg[nbr[e]], 1);
}

__global__ void raw_count_kernel(const int32_t* __restrict__ indeg, int64_t n, int k, int32_t* cnt, int32_t* fill)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        cnt[i] = 1 + k + indeg[i];
        fill[i] = 0;
    }
}

__global__ void raw_scatter_kernel(const int32_t* __restrict__ nbr, const double* __restrict__ nbr_d2, int64_t n,
                                   int k, const int64_t* __restrict__ raw_ptr, int32_t* fill, int32_t* raw_col,
                                   float* raw_d2)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) {   // diagonal
        raw_col[raw_ptr[e]] = (int32_t)e;
        raw_d2[raw_ptr[e]] = 0.f;
    }
    if (e >= n * k) return;
    int64_t i = e / k;
    int r = (int)(e - i * k);
    int32_t j = nbr[e];
    float d = (float)nbr_d2[e];
    int64_t own = raw_ptr[i] + 1 + r;
    raw_col[own] = j;
    raw_d2[own] = d;
    int slot = atomicAdd(&fill[j], 1);
    int64_t tr = raw_ptr[j] + 1 + k + slot;
    raw_col[tr] = (int32_t)i;
    raw_d2[tr] = d;
}

// bitonic sort of P (power of two) 64-bit keys in shared memory by `nthr` threads
__device__ __forceinline__ void bitonic_smem(uint64_t* a, int P, int tid, int nthr, bool warp_only)
{
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < P / 2; i += nthr) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool up = (lo & size) == 0;
                uint64_t x = a[lo], y = a[hi];
                if ((x > y) == up) { a[lo] = y; a[hi] = x; }
            }
            if (warp_only) __syncwarp(); else __syncthreads();
        }
    }
}

// Sort one row's raw entries by column, drop duplicates, write back in place.
__device__ void sort_dedupe_row(uint64_t* buf, int c, int P, int64_t rb, int32_t* raw_col, float* raw_d2,
                                int32_t* cnt, int64_t i, int tid, int nthr, bool warp_only, int32_t* s_tot)
{
    for (int e = tid; e < P; e += nthr)
        buf[e] = e < c ? ((uint64_t)(uint32_t)raw_col[rb + e] << 32) | __float_as_uint(raw_d2[rb + e]) : ~0ull;
    if (warp_only) __syncwarp(); else __syncthreads();
    bitonic_smem(buf, P, tid, nthr, warp_only);
    // unique entries: first of each run of equal columns, compacted in order
    const int lane = tid & 31;
    int32_t base = 0;
    for (int e0 = 0; e0 < c; e0 += nthr) {
        int e = e0 + tid;
        bool first = e < c && (e == 0 || (buf[e] >> 32) != (buf[e - 1] >> 32));
        unsigned bal = __ballot_sync(0xffffffffu, first);
        int32_t off = __popc(bal & ((1u << lane) - 1u));
        int32_t tot;
        if (warp_only) {
            tot = __popc(bal);
        } else {
            const int w = tid >> 5, nw = nthr >> 5;
            if (lane == 0) s_tot[w] = __popc(bal);
            __syncthreads();
            tot = 0;
            for (int ww = 0; ww < nw; ++ww) {
                if (ww < w) off += s_tot[ww];
                tot += s_tot[ww];
            }
            __syncthreads();
        }
        if (first) {
            raw_col[rb + base + off] = (int32_t)(buf[e] >> 32);
            raw_d2[rb + base + off] = __uint_as_float((uint32_t)buf[e]);
        }
        base += tot;
    }
    if (tid == 0) cnt[i] = base;
}

__global__ void __launch_bounds__(SORT_WARPS * 32) row_sort_kernel(const int64_t* __restrict__ raw_ptr, int64_t n,
                                                                    int32_t* raw_col, float* raw_d2, int32_t* cnt,
                                                                    int32_t* big, int32_t* nbig, DevReport* rep)
{
    __shared__ uint64_t buf[SORT_WARPS][ROW_CAP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * SORT_WARPS + w; i < n; i += (int64_t)gridDim.x * SORT_WARPS) {
        int64_t rb = raw_ptr[i];
        int c = (int)(raw_ptr[i + 1] - rb);
        if (c > ROW_CAP) {
            if (lane == 0) {
                int s = atomicAdd(nbig, 1);
                big[s] = (int32_t)i;
                atomicAdd(&rep->union_big_rows, 1ull);
            }
            continue;
        }
        int P = 32;
        while (P < c) P <<= 1;
        sort_dedupe_row(buf[w], c, P, rb, raw_col, raw_d2, cnt, i, lane, 32, true, nullptr);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(1024) big_row_sort_kernel(const int64_t* __restrict__ raw_ptr, int32_t* raw_col,
                                                           float* raw_d2, int32_t* cnt, const int32_t* __restrict__ big,
                                                           const int32_t* __restrict__ nbig, DevReport* rep)
{
    extern __shared__ uint64_t bbuf[];
    __shared__ int32_t s_tot[32];
    const int nb = *nbig;
    for (int f = blockIdx.x; f < nb; f += gridDim.x) {
        int64_t i = big[f];
        int64_t rb = raw_ptr[i];
        int c = (int)(raw_ptr[i + 1] - rb);
        if (c > BIG_CAP) {
            if (threadIdx.x == 0) {
                report_error(rep, VB_ERR_UNSUPPORTED);
                cnt[i] = 0;
            }
            continue;
        }
        int P = 32;
        while (P < c) P <<= 1;
        sort_dedupe_row(bbuf, c, P, rb, raw_col, raw_d2, cnt, i, threadIdx.x, blockDim.x, false, s_tot);
        __syncthreads();
    }
}

__global__ void compact_kernel(const int64_t* __restrict__ raw_ptr, const int64_t* __restrict__ row_ptr, int64_t n,
                               const int32_t* __restrict__ raw_col, const float* __restrict__ raw_d2, int32_t* col,
                               float* ed2, int64_t cap, int64_t* nnz_dev, DevReport* rep)
{
    const int lane = threadIdx.x & 31;
    int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (wid == 0 && lane == 0) {
        *nnz_dev = row_ptr[n];
        if (row_ptr[n] > cap) report_error(rep, VB_ERR_BOUNDS);
    }
    for (int64_t i = wid; i < n; i += nw) {
        int64_t rb = raw_ptr[i], ob = row_ptr[i], c = row_ptr[i + 1] - ob;
        if (ob + c > cap) continue;
        for (int64_t e = lane; e < c; e += 32) {
            col[ob + e] = raw_col[rb + e];
            ed2[ob + e] = raw_d2[rb + e];
        }
    }
}

vb_status graph_run(Ctx* ctx, int64_t n, int32_t k, const int32_t* nbr, const double* nbr_d2, int64_t* row_ptr,
                    int32_t* col, float* ed2, int64_t cap, int64_t* nnz_dev, void* ws, size_t ws_bytes)
{
    if (n < 2 || k < 1 || k > n - 1 || !nbr || !nbr_d2 || !row_ptr || !col || !ed2 || !nnz_dev) return VB_ERR_ARG;
    if (cap < n * (2 * (int64_t)k + 1)) return VB_ERR_ARG;
    GraphWs w;
    Carve c(ws);
    size_t need = graph_plan(c, n, k, &w);
    if (!ws || ws_bytes < need) return VB_ERR_WORKSPACE;
    cudaStream_t s = ctx->stream;
    const int64_t nk = n * k;
    const unsigned gz = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8);
    mark(ctx, VB_STAGE_GRAPH, 0);
    zero_i32_kernel<<<gz, 256, 0, s>>>(w.indeg, n);
    zero_i32_kernel<<<1, 32, 0, s>>>(w.nbig, 1);
    indeg_kernel<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(nbr, nk, w.indeg);
    raw_count_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.indeg, n, k, w.cnt, w.fill);
    vb_status st = scan_counts(s, w.cnt, n, w.raw_ptr, w.scan);
    if (st != VB_OK) return st;
    raw_scatter_kernel<<<(unsigned)((std::max(nk, n) + 255) / 256), 256, 0, s>>>(nbr, nbr_d2, n, k, w.raw_ptr, w.fill,
                                                                             w.raw_col, w.raw_d2);
    row_sort_kernel<<<152 * 16, SORT_WARPS * 32, 0, s>>>(w.raw_ptr, n, w.raw_col, w.raw_d2, w.cnt, w.big, w.nbig,
                                                         ctx->rep);
    static bool big_attr[16] = {};
    int dev = ctx->device & 15;
    if (!big_attr[dev]) {
        if (cudaFuncSetAttribute(big_row_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 BIG_CAP * 8) != cudaSuccess)
            return VB_ERR_CUDA;
        big_attr[dev] = true;
    }
    big_row_sort_kernel<<<152, 1024, BIG_CAP * 8, s>>>(w.raw_ptr, w.raw_col, w.raw_d2, w.cnt, w.big, w.nbig, ctx->rep);
    st = scan_counts(s, w.cnt, n, row_ptr, w.scan);
    if (st != VB_OK) return st;
    compact_kernel<<<152 * 8, 256, 0, s>>>(w.raw_ptr, row_ptr, n, w.raw_col, w.raw_d2, col, ed2, cap, nnz_dev,
                                           ctx->rep);
    mark(ctx, VB_STAGE_GRAPH, 1);
    ctx->launches += 14;
    return last_launch();
}

// ------------------------------------------------------------------ a8
__global__ void bandwidth_kernel(const double* __restrict__ nbr_d2, int64_t n, int k, int k_bw, double* b,
                                 DevReport* rep)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* d = nbr_d2 + i * k;
    double s = d[0];
    for (int r = 1; r < k_bw; ++r) s = __dadd_rn(s, d[r]);
    double v = sqrt(s);
    b[i] = v;
    if (!(v > 0.0) || !isfinite(v)) report_error(rep, VB_ERR_DEGENERATE);
}

vb_status bandwidth_run(Ctx* ctx, int64_t n, int32_t k, int32_t k_bw, const double* nbr_d2, double* b)
{
    if (n < 1 || k < 1 || k_bw < 1 || k_bw > k || !nbr_d2 || !b) return VB_ERR_ARG;
    mark(ctx, VB_STAGE_BANDWIDTH, 0);
    bandwidth_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(nbr_d2, n, k, k_bw, b, ctx->rep);
    mark(ctx, VB_STAGE_BANDWIDTH, 1);
    ctx->launches += 1;
    return last_launch();
}

}  // namespace vb
