// Symmetric sparsity pattern (step a6) and the bandwidth function (step a8).
//
// a6: E = {(i, i)} U {(i, j): j in N_k(i) or i in N_k(j)} as CSR with rows
//     sorted by column.  Algorithm 1 keeps the diagonal (its inner loop
//     starts at j = i) and sets K^ij and K^ji together, so every kNN pair
//     enters in both directions.  The FP32 squared distance of every entry is
//     the FP32 rounding of the canonical FP64 value, identical for (i, j) and
//     (j, i).  Construction below (sorted own lists, filtered reverse entries,
//     merge by rank).
// a8: b_i^2 = sum_{r=1}^{k_bw} d2(i, I(i, r)) in rank order, FP64 (Eq.
//     bandwidth parameter).
#include "vb_internal.cuh"

#include <algorithm>

namespace vb {

constexpr int BIG_CAP = 8192;       // block path: reverse entries per row
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
// Row j of E is the disjoint union of {j}, its own kNN list N(j), and the reverse
// entries R(j) = {i : j in N(i), i not in N(j)}.  Construction: every kNN list is
// sorted by column (one warp per row); a reverse candidate (i -> j) is kept unless i is
// in N(j), which for exact lists ordered by (d2, index) holds exactly when
// (d2(i, j), i) <= (d2 and index of j's k-th neighbour), one 16-byte load instead of a
// search, so mutual pairs enter once; the counts
// 1 + k + |R(j)| give row_ptr directly (one scan); the kept reverse entries are
// scattered into a side buffer; finally one warp per row sorts R(j) and places
// every entry by its rank (own index + reverse entries below it + the diagonal),
// which merges the three sorted sets with no duplicates left to remove.
constexpr int RCAP = 256;           // warp path: reverse entries per row held in shared memory
constexpr int OWN_CAP = 256;        // longest kNN list (k + margin <= 256)

struct Kth {
    double d2;         // j's k-th neighbour distance and index
    int32_t idx, pad;
};

struct GraphWs {
    Kth* kth;          // n
    int32_t* own_col;  // n k: kNN lists sorted by column
    float* own_d2;     // n k
    int32_t* rcnt;     // n reverse entries per row
    int32_t* fill;     // n scatter cursors
    int32_t* cnt;      // n row lengths
    int32_t* rev_col;  // n k reverse entries, row j at row_ptr[j] - j (1 + k)
    float* rev_d2;     // n k
    int32_t* big;      // n rows for the block path
    int32_t* nbig;     // 1
    void* scan;        // scan_ws_bytes(n)
};

static size_t graph_plan(Carve& c, int64_t n, int32_t k, GraphWs* w)
{
    GraphWs t;
    t.kth = c.take<Kth>(n);
    t.own_col = c.take<int32_t>(n * (int64_t)k);
    t.own_d2 = c.take<float>(n * (int64_t)k);
    t.rcnt = c.take<int32_t>(n);
    t.fill = c.take<int32_t>(n);
    t.cnt = c.take<int32_t>(n);
    t.rev_col = c.take<int32_t>(n * (int64_t)k);
    t.rev_d2 = c.take<float>(n * (int64_t)k);
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

// Number of entries of the ascending list a[0..len) below v.
__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int len, int32_t v)
{
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int lower_bound_key(const uint64_t* a, int len, int32_t v)
{
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int32_t)(a[mid] >> 32) < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

constexpr int SORT_WARPS = 4;

// The k-th pair (distance, index) of every list, 16 bytes per point: the table the mutual
// test below reads at random stays in L2, where the lists themselves (12 k bytes per point)
// do not.
__global__ void kth_kernel(const int32_t* __restrict__ nbr, const double* __restrict__ nbr_d2, int64_t n, int k,
                           Kth* kth)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Kth q;
    q.d2 = nbr_d2[i * k + k - 1];
    q.idx = nbr[i * k + k - 1];
    q.pad = 0;
    kth[i] = q;
}

// Own kNN lists sorted by column, one warp per row; the FP32 value of each entry is the
// rounding of its canonical FP64 distance (identical for (i, j) and (j, i)).  The columns of a
// list are distinct, so an entry's place in the sorted list is the number of columns below its
// own: every column is broadcast to the warp once (a shuffle) and each lane counts for the KL
// entries it holds, then writes each entry straight to its place.  No shared memory: a
// bitonic network over 64-bit keys in shared memory was bound by its shared-memory traffic.
// The same pass counts, for every point j, the lists that name j without j naming their owner
// (the reverse entries of row j): (i -> j) is mutual exactly when (d2(i, j), i) does not exceed
// the k-th pair of j's own list (kth[j]).  A non-mutual entry carries the sign bit in own_d2
// (distances are >= 0), so the scatter pass reads the sorted lists alone.
// For k <= 64 and n <= 2^26 the list is instead sorted as 32-bit keys column << 6 | position
// (columns distinct, so the order is the columns' order) by a bitonic network across the warp,
// two keys per lane: 21 compare-exchange steps of one shuffle each instead of k broadcasts with
// k compares, and each sorted key names the entry it came from.
template <int KL>
__device__ __forceinline__ void warp_bitonic(uint32_t (&key)[KL], int lane)
{
    constexpr int N = 32 * KL;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride == 32) {   // N = 64: the partner is this lane's other key
                const uint32_t a = key[0], b = key[KL - 1];
                key[0] = min(a, b);
                key[KL - 1] = max(a, b);
            } else {
#pragma unroll
                for (int s = 0; s < KL; ++s) {
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, key[s], stride);
                    const bool lower = (lane & stride) == 0, up = ((lane + 32 * s) & size) == 0;
                    key[s] = lower == up ? min(key[s], o) : max(key[s], o);
                }
            }
        }
    }
}

template <int KL>
__global__ void __launch_bounds__(SORT_WARPS * 32) own_sort_kernel(const int32_t* __restrict__ nbr,
                                                                    const double* __restrict__ nbr_d2, int64_t n,
                                                                    int k, int32_t* own_col, float* own_d2,
                                                                    const Kth* __restrict__ kth, int32_t* rcnt)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (KL <= 2) {
        if (n <= ((int64_t)1 << 26)) {
            for (int64_t i = (int64_t)blockIdx.x * SORT_WARPS + w; i < n; i += (int64_t)gridDim.x * SORT_WARPS) {
                const int32_t* row = nbr + i * k;
                uint32_t key[KL];
#pragma unroll
                for (int s = 0; s < KL; ++s) {
                    const int e = lane + 32 * s;
                    key[s] = e < k ? ((uint32_t)row[e] << 6) | (uint32_t)e : 0xffffffffu;
                }
                warp_bitonic<KL>(key, lane);
#pragma unroll
                for (int s = 0; s < KL; ++s) {
                    const int pos = lane + 32 * s;   // the key's place in the sorted list
                    if (pos < k) {
                        const int32_t j = (int32_t)(key[s] >> 6);
                        const int e = (int)(key[s] & 63u);
                        const double d = nbr_d2[i * k + e];
                        const Kth q = kth[j];
                        const bool rev = !(d < q.d2 || (d == q.d2 && (int32_t)i <= q.idx));
                        own_col[i * k + pos] = j;
                        own_d2[i * k + pos] = rev ? -(float)d : (float)d;
                        if (rev) atomicAdd(&rcnt[j], 1);
                    }
                }
            }
            return;
        }
    }
    for (int64_t i = (int64_t)blockIdx.x * SORT_WARPS + w; i < n; i += (int64_t)gridDim.x * SORT_WARPS) {
        const int32_t* row = nbr + i * k;
        int32_t c[KL];
        int rank[KL];
#pragma unroll
        for (int s = 0; s < KL; ++s) {
            const int e = lane + 32 * s;
            c[s] = e < k ? row[e] : INT32_MAX;
            rank[s] = 0;
        }
#pragma unroll
        for (int s2 = 0; s2 < KL; ++s2) {
            const int32_t v = c[s2];
            const int lim = min(32, k - 32 * s2);
            for (int l = 0; l < lim; ++l) {
                const int32_t cb = __shfl_sync(0xffffffffu, v, l);
#pragma unroll
                for (int s = 0; s < KL; ++s) rank[s] += cb < c[s] ? 1 : 0;
            }
        }
#pragma unroll
        for (int s = 0; s < KL; ++s) {
            const int e = lane + 32 * s;
            if (e < k) {
                const double d = nbr_d2[i * k + e];
                const int32_t j = c[s];
                const Kth q = kth[j];
                const bool rev = !(d < q.d2 || (d == q.d2 && (int32_t)i <= q.idx));
                own_col[i * k + rank[s]] = j;
                own_d2[i * k + rank[s]] = rev ? -(float)d : (float)d;
                if (rev) atomicAdd(&rcnt[j], 1);
            }
        }
    }
}

// The non-mutual entries (i -> j) of the sorted lists (sign bit set in own_d2), scattered
// into row j's reverse slots.
__global__ void reverse_kernel(const int32_t* __restrict__ own_col, const float* __restrict__ own_d2, int64_t n, int k,
                               const int64_t* __restrict__ row_ptr, int32_t* fill, int32_t* rev_col, float* rev_d2)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * k) return;
    const float d = own_d2[e];
    if (!signbit(d)) return;   // mutual: already in row j's own list
    const int64_t i = e / k;
    const int32_t j = own_col[e];
    const int slot = atomicAdd(&fill[j], 1);
    const int64_t off = row_ptr[j] - (int64_t)j * (1 + k) + slot;
    rev_col[off] = (int32_t)i;
    rev_d2[off] = -d;
}

__global__ void row_len_kernel(const int32_t* __restrict__ rcnt, int64_t n, int k, int32_t* cnt, int32_t* fill)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        cnt[i] = 1 + k + rcnt[i];
        fill[i] = 0;
    }
}

// Row j: sort R(j) in shared memory, then write every entry at its rank.
// oc_s: shared-memory room for the row's own columns (k ints), or nullptr to search them in
// global memory (the block path).
__device__ void merge_row(int64_t j, int k, int r, uint64_t* rb, const int64_t* __restrict__ row_ptr,
                          const int32_t* __restrict__ own_col, const float* __restrict__ own_d2,
                          const int32_t* __restrict__ rev_col, const float* __restrict__ rev_d2, int32_t* col,
                          float* ed2, int tid, int nthr, bool warp_only, int32_t* oc_s = nullptr)
{
    int P = 32;
    while (P < r) P <<= 1;
    const int64_t roff = row_ptr[j] - j * (1 + k);
    for (int e = tid; e < P; e += nthr)
        rb[e] = e < r ? ((uint64_t)(uint32_t)rev_col[roff + e] << 32) | __float_as_uint(rev_d2[roff + e]) : ~0ull;
    const int32_t* oc = own_col + j * k;
    if (oc_s) {   // the own columns, searched once per reverse entry, from shared memory
        for (int e = tid; e < k; e += nthr) oc_s[e] = oc[e];
        oc = oc_s;
    }
    if (warp_only) __syncwarp(); else __syncthreads();
    if (r > 1) bitonic_smem(rb, P, tid, nthr, warp_only);
    const int64_t ob = row_ptr[j];
    const float* od = own_d2 + j * k;
    for (int a = tid; a < k; a += nthr) {
        const int32_t c = oc[a];   // (own_col + j k)[a]
        const int rank = a + lower_bound_key(rb, r, c) + ((int32_t)j < c ? 1 : 0);
        col[ob + rank] = c;
        ed2[ob + rank] = fabsf(od[a]);   // without the non-mutual mark
    }
    for (int b = tid; b < r; b += nthr) {
        const int32_t c = (int32_t)(rb[b] >> 32);
        const int rank = b + lower_bound_i32(oc, k, c) + ((int32_t)j < c ? 1 : 0);
        col[ob + rank] = c;
        ed2[ob + rank] = __uint_as_float((uint32_t)rb[b]);
    }
    if (tid == 0) {
        const int rank = lower_bound_i32(oc, k, (int32_t)j) + lower_bound_key(rb, r, (int32_t)j);
        col[ob + rank] = (int32_t)j;
        ed2[ob + rank] = 0.f;
    }
}

// The same for a row with at most 32 reverse entries (nearly every row), one per lane, without
// sorting them: every reverse column is broadcast to the warp once, and each lane counts the
// reverse columns below its own reverse entry (its rank among them; the columns of R(j) are
// distinct) and below each of its own-list entries; a reverse entry's place among the own
// entries is a binary search of the sorted own columns in shared memory.
template <int OWN_PER_LANE>   // own-list entries per lane: k <= 32 OWN_PER_LANE
__device__ void merge_row_small(int64_t j, int k, int r, const int64_t* __restrict__ row_ptr,
                                const int32_t* __restrict__ own_col, const float* __restrict__ own_d2,
                                const int32_t* __restrict__ rev_col, const float* __restrict__ rev_d2, int32_t* col,
                                float* ed2, int lane, int32_t* oc_s)
{
    const int64_t roff = row_ptr[j] - j * (1 + k);
    int32_t rc = INT32_MAX;
    float rd = 0.f;
    if (lane < r) {
        rc = rev_col[roff + lane];
        rd = rev_d2[roff + lane];
    }
    const int32_t* oc = own_col + j * k;
    int32_t c[OWN_PER_LANE];
    int below[OWN_PER_LANE];
#pragma unroll
    for (int s = 0; s < OWN_PER_LANE; ++s) {
        const int a = lane + 32 * s;
        c[s] = a < k ? oc[a] : INT32_MAX;
        below[s] = 0;
        if (a < k) oc_s[a] = c[s];
    }
    int rrank = 0;
    for (int b = 0; b < r; ++b) {
        const int32_t cb = __shfl_sync(0xffffffffu, rc, b);
        rrank += cb < rc ? 1 : 0;
#pragma unroll
        for (int s = 0; s < OWN_PER_LANE; ++s) below[s] += cb < c[s] ? 1 : 0;
    }
    const int rev_below_j = __popc(__ballot_sync(0xffffffffu, lane < r && rc < (int32_t)j));
    __syncwarp();   // the own columns in shared memory, for the searches below
    const int64_t ob = row_ptr[j];
    const float* od = own_d2 + j * k;
#pragma unroll
    for (int s = 0; s < OWN_PER_LANE; ++s) {
        const int a = lane + 32 * s;
        if (a < k) {
            const int rank = a + below[s] + ((int32_t)j < c[s] ? 1 : 0);
            col[ob + rank] = c[s];
            ed2[ob + rank] = fabsf(od[a]);   // without the non-mutual mark
        }
    }
    if (lane < r) {
        const int rank = rrank + lower_bound_i32(oc_s, k, rc) + ((int32_t)j < rc ? 1 : 0);
        col[ob + rank] = rc;
        ed2[ob + rank] = rd;
    }
    if (lane == 0) {
        const int rank = lower_bound_i32(oc_s, k, (int32_t)j) + rev_below_j;
        col[ob + rank] = (int32_t)j;
        ed2[ob + rank] = 0.f;
    }
}

template <int KL>   // own-list entries per lane, k <= 32 KL
__global__ void __launch_bounds__(SORT_WARPS * 32) merge_kernel(const int64_t* __restrict__ row_ptr, int64_t n, int k,
                                                                 const int32_t* __restrict__ own_col,
                                                                 const float* __restrict__ own_d2,
                                                                 const int32_t* __restrict__ rev_col,
                                                                 const float* __restrict__ rev_d2, int32_t* col,
                                                                 float* ed2, int64_t cap, int32_t* big, int32_t* nbig,
                                                                 int64_t* nnz_dev, DevReport* rep)
{
    __shared__ uint64_t buf[SORT_WARPS][RCAP];
    __shared__ int32_t ocs[SORT_WARPS][OWN_CAP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *nnz_dev = row_ptr[n];
        if (row_ptr[n] > cap) report_error(rep, VB_ERR_BOUNDS);
    }
    if (row_ptr[n] > cap) return;
    for (int64_t j = (int64_t)blockIdx.x * SORT_WARPS + w; j < n; j += (int64_t)gridDim.x * SORT_WARPS) {
        const int r = (int)(row_ptr[j + 1] - row_ptr[j]) - 1 - k;
        if (r > RCAP) {
            if (lane == 0) {
                big[atomicAdd(nbig, 1)] = (int32_t)j;
                atomicAdd(&rep->union_big_rows, 1ull);
            }
            continue;
        }
        if (r <= 32)
            merge_row_small<KL>(j, k, r, row_ptr, own_col, own_d2, rev_col, rev_d2, col, ed2, lane, ocs[w]);
        else
            merge_row(j, k, r, buf[w], row_ptr, own_col, own_d2, rev_col, rev_d2, col, ed2, lane, 32, true, ocs[w]);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(1024) big_merge_kernel(const int64_t* __restrict__ row_ptr, int64_t n, int k,
                                                        const int32_t* __restrict__ own_col,
                                                        const float* __restrict__ own_d2,
                                                        const int32_t* __restrict__ rev_col,
                                                        const float* __restrict__ rev_d2, int32_t* col, float* ed2,
                                                        int64_t cap, const int32_t* __restrict__ big,
                                                        const int32_t* __restrict__ nbig, DevReport* rep)
{
    extern __shared__ uint64_t bbuf[];
    if (row_ptr[n] > cap) return;
    const int nb = *nbig;
    for (int f = blockIdx.x; f < nb; f += gridDim.x) {
        const int64_t j = big[f];
        const int r = (int)(row_ptr[j + 1] - row_ptr[j]) - 1 - k;
        if (r > BIG_CAP) {   // a hub point in more than BIG_CAP other lists
            if (threadIdx.x == 0) report_error(rep, VB_ERR_UNSUPPORTED);
            continue;
        }
        merge_row(j, k, r, bbuf, row_ptr, own_col, own_d2, rev_col, rev_d2, col, ed2, threadIdx.x, blockDim.x, false);
        __syncthreads();
    }
}

vb_status graph_run(Ctx* ctx, int64_t n, int32_t k, const int32_t* nbr, const double* nbr_d2, int64_t* row_ptr,
                    int32_t* col, float* ed2, int64_t cap, int64_t* nnz_dev, void* ws, size_t ws_bytes)
{
    if (n < 2 || k < 1 || k > n - 1 || k > OWN_CAP || !nbr || !nbr_d2 || !row_ptr || !col || !ed2 || !nnz_dev)
        return VB_ERR_ARG;
    if (cap < n * (2 * (int64_t)k + 1)) return VB_ERR_ARG;
    GraphWs w;
    Carve c(ws);
    size_t need = graph_plan(c, n, k, &w);
    if (!ws || ws_bytes < need) return VB_ERR_WORKSPACE;
    cudaStream_t s = ctx->stream;
    const int64_t nk = n * k;
    const unsigned gz = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8);
    const unsigned ge = (unsigned)((nk + 255) / 256);
    mark(ctx, VB_STAGE_GRAPH, 0);
    zero_i32_kernel<<<gz, 256, 0, s>>>(w.rcnt, n);
    zero_i32_kernel<<<1, 32, 0, s>>>(w.nbig, 1);
    kth_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nbr, nbr_d2, n, k, w.kth);
    if (k <= 32)
        own_sort_kernel<1><<<152 * 16, SORT_WARPS * 32, 0, s>>>(nbr, nbr_d2, n, k, w.own_col, w.own_d2, w.kth,
                                                                   w.rcnt);
    else if (k <= 64)
        own_sort_kernel<2><<<152 * 16, SORT_WARPS * 32, 0, s>>>(nbr, nbr_d2, n, k, w.own_col, w.own_d2, w.kth,
                                                                   w.rcnt);
    else if (k <= 128)
        own_sort_kernel<4><<<152 * 16, SORT_WARPS * 32, 0, s>>>(nbr, nbr_d2, n, k, w.own_col, w.own_d2, w.kth,
                                                                   w.rcnt);
    else
        own_sort_kernel<8><<<152 * 16, SORT_WARPS * 32, 0, s>>>(nbr, nbr_d2, n, k, w.own_col, w.own_d2, w.kth,
                                                                   w.rcnt);
    row_len_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.rcnt, n, k, w.cnt, w.fill);
    vb_status st = scan_counts(s, w.cnt, n, row_ptr, w.scan);
    if (st != VB_OK) return st;
    reverse_kernel<<<ge, 256, 0, s>>>(w.own_col, w.own_d2, n, k, row_ptr, w.fill, w.rev_col, w.rev_d2);
    if (k <= 32)
        merge_kernel<1><<<152 * 16, SORT_WARPS * 32, 0, s>>>(row_ptr, n, k, w.own_col, w.own_d2, w.rev_col, w.rev_d2, col, ed2,
                                                      cap, w.big, w.nbig, nnz_dev, ctx->rep);
    else if (k <= 64)
        merge_kernel<2><<<152 * 16, SORT_WARPS * 32, 0, s>>>(row_ptr, n, k, w.own_col, w.own_d2, w.rev_col, w.rev_d2, col, ed2,
                                                      cap, w.big, w.nbig, nnz_dev, ctx->rep);
    else if (k <= 128)
        merge_kernel<4><<<152 * 16, SORT_WARPS * 32, 0, s>>>(row_ptr, n, k, w.own_col, w.own_d2, w.rev_col, w.rev_d2, col, ed2,
                                                      cap, w.big, w.nbig, nnz_dev, ctx->rep);
    else
        merge_kernel<OWN_CAP / 32><<<152 * 16, SORT_WARPS * 32, 0, s>>>(row_ptr, n, k, w.own_col, w.own_d2, w.rev_col, w.rev_d2, col, ed2,
                                                      cap, w.big, w.nbig, nnz_dev, ctx->rep);
    static bool big_attr[16] = {};
    int dev = ctx->device & 15;
    if (!big_attr[dev]) {
        if (cudaFuncSetAttribute(big_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BIG_CAP * 8) !=
            cudaSuccess)
            return VB_ERR_CUDA;
        big_attr[dev] = true;
    }
    big_merge_kernel<<<152, 1024, BIG_CAP * 8, s>>>(row_ptr, n, k, w.own_col, w.own_d2, w.rev_col, w.rev_d2, col, ed2,
                                                    cap, w.big, w.nbig, ctx->rep);
    mark(ctx, VB_STAGE_GRAPH, 1);
    ctx->launches += 12;
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
