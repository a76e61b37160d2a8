// Exact k-nearest-neighbour search on the GPU (steps a1-a5 of the build).
//
// Definition (Sec. 2.1, the index map I(x, r) of the bandwidth function): the k
// nearest other samples of every point, ordered by the canonical FP64 squared
// distance and then by index.  The search itself runs in FP32 and is made
// exact by an FP64 certificate:
//   a1  spatial order: bounding box, 32-bit Hilbert keys of the m coordinates when
//       2 <= m <= 4 (Morton keys on request, and at m = 1), else Morton keys of the
//       projections on the cloud's 5 leading principal axes (sampled covariance,
//       subspace iteration), stable LSD radix sort, gather of the coordinates into
//       64-point tiles (zero-padded to MP = 4, 8, ..., 128).
//   a2  pruning: every tile carries its bounding box; a candidate tile is
//       skipped when the box-to-box (and, per query, point-to-box) distance,
//       rounded down by a proven FP32 error factor, exceeds the running
//       (k+margin)-th smallest FP32 distance of the query tile.
//   a3  distances: FP32 difference form sum_r (q_r - c_r)^2 on the ALUs.
//   a4  selection: per query a max-heap of the k + margin smallest keys
//       (FP32 distance bits << 32 | sorted position) in shared memory.
//   a5  rescoring: FP64 canonical distances of the kept candidates, ranked by
//       (d2, index); the row is certified when the k-th FP64 distance lies
//       below the smallest FP64 distance any excluded candidate can have,
//       H (1 - 2 gamma), H = the largest kept FP32 distance and
//       gamma = (m + 2) 2^-24 the relative error bound of the FP32 sum.
//       Uncertified rows (ties, duplicates) are recomputed by an exact FP64
//       radix selection over all points.
#include "vb_internal.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

namespace vb {

constexpr int TILE = 64;            // points per query tile and per candidate tile
constexpr int RADIX_T = 256;        // threads of the radix kernels
constexpr int RADIX_ITEMS = 2048;   // keys per radix block (8 rounds of 256)
constexpr int USCAN_T = 1024, USCAN_ITEMS = 8, USCAN_CHUNK = USCAN_T * USCAN_ITEMS;   // histogram scan
constexpr int FB_THREADS = 256;

struct KnnWs {
    int* bbox;            // 16 ordered ints: min[8], max[8]
    double* pcs;          // m > 4: sampled moments (1 + m + m * m), then the principal axes
    float* pcc;           // m > 4: the covariance (m x m)
    float* proj;          // m > 4: n x 5 projections on the leading principal axes
    uint32_t* key[2];
    uint32_t* val[2];     // val[0] after the sort = perm (sorted position -> original index)
    uint32_t* hist;       // 256 * nblk
    uint32_t* hsum;       // block sums of the histogram scan
    float* xs;            // npad * MP sorted coordinates
    double* xs64;         // the same in FP64 (exact copies), read by the FP64 rescoring
    uint64_t* hdump;      // 16-bit search: npad x (k + max(margin, 32)) heap keys handed to the row finish
    float* tlo;           // ntiles * MP
    float* thi;
    float* slo;           // ceil(ntiles / 64) * MP: boxes of super-tiles (64 consecutive tiles)
    float* shi;
    int* fb_list;         // n
    int* fb_count;        // [0] fallback rows, [1] next query tile, [2] next failed tile, [3] failed tiles,
                          // [4] next tile of the second list, [5] tiles in it
    float* r2;            // n (radius search: squared radius bound per sorted point)
    int* fail_flag;       // 2 ntiles: flags of radius passes 1 and 2
    int* fail_list;       // 2 ntiles: tiles left by passes 1 and 2
    // pipelined 16-bit search only (precision != FP32)
    unsigned char* blk;   // npad / 64 tile blocks: 16-bit operand image + 64 FP32 norms
    uint32_t* lbw;        // TCP_MAX_CTAS * ntiles: box bounds of the candidate tiles (per CTA)
    uint64_t* tlist;      // TCP_MAX_CTAS * ntiles: candidate tiles ordered by bound (per CTA)
    uint4* lbs;           // TCP_MAX_CTAS * ntiles: their bounds for each group of 32 queries (per CTA)
    int* crange;          // 256 ordered ints: per-coordinate min and max of the cloud
    float* trad;          // ntiles: radius of each tile's ball about its box centre
};

constexpr int TCP_MAX_CTAS = 304;   // persistent grid of the pipelined search (2 per SM on 152 SMs)
static int pad_k16(int m) { return (m + 15) / 16 * 16; }
// bytes of one 64-point tile block of the pipelined search: operand image, then norms
__host__ __device__ inline size_t tcp_img_bytes(int kp) { return (size_t)64 * kp * 2; }
__host__ __device__ inline size_t tcp_blk_bytes(int kp) { return tcp_img_bytes(kp) + 64 * sizeof(float); }

static int pad_dim(int m)
{
    int mp = 4;
    while (mp < m) mp *= 2;
    return mp;
}
constexpr int PCA_D = 5;           // principal axes of the Morton key when m > 4
static int morton_dims(int m) { return m <= 4 ? m : PCA_D; }
static int morton_bits(int md) { return md == 1 ? 30 : md == 2 ? 15 : md == 3 ? 10 : md == 4 ? 8 : md == 5 ? 6 : 5; }

size_t knn_plan(Carve& c, int64_t n, int32_t m, const vb_knn_params* p, KnnWs* w)
{
    const int mp = pad_dim(m);
    const int64_t ntiles = (n + TILE - 1) / TILE;
    const int64_t npad = (ntiles + (ntiles & 1)) * TILE;   // even tile count: the tensor-core search pairs tiles
    const int64_t nblk = (n + RADIX_ITEMS - 1) / RADIX_ITEMS;
    KnnWs t;
    t.bbox = c.take<int>(16);
    t.pcs = nullptr;
    t.pcc = nullptr;
    t.proj = nullptr;
    if (m > 4) {
        t.pcc = c.take<float>((size_t)m * m);
        t.pcs = c.take<double>(1 + m + (size_t)m * m + (size_t)m * PCA_D);
        t.proj = c.take<float>((size_t)n * PCA_D);
    }
    t.key[0] = c.take<uint32_t>(n);
    t.key[1] = c.take<uint32_t>(n);
    t.val[0] = c.take<uint32_t>(n);
    t.val[1] = c.take<uint32_t>(n);
    t.hist = c.take<uint32_t>(256 * nblk);
    t.hsum = c.take<uint32_t>((256 * nblk + USCAN_CHUNK - 1) / USCAN_CHUNK + 1);
    t.xs = c.take<float>(npad * mp);
    t.xs64 = c.take<double>(npad * mp);
    t.hdump = nullptr;
    if (p && p->precision != VB_PREC_FP32) {   // L <= k + max(margin, 32), the autotuner's range
        const int64_t lmax = std::min(256, p->k + std::max(p->margin, 32));
        t.hdump = c.take<uint64_t>((size_t)npad * lmax);
    }
    t.tlo = c.take<float>(ntiles * mp);
    t.thi = c.take<float>(ntiles * mp);
    t.slo = c.take<float>((ntiles + TILE - 1) / TILE * mp);
    t.shi = c.take<float>((ntiles + TILE - 1) / TILE * mp);
    t.fb_list = c.take<int>(n);
    t.fb_count = c.take<int>(8);
    t.r2 = c.take<float>(npad);
    t.fail_flag = c.take<int>(2 * ntiles);
    t.fail_list = c.take<int>(2 * ntiles);
    t.blk = nullptr;
    t.lbw = nullptr;
    t.tlist = nullptr;
    t.lbs = nullptr;
    t.crange = nullptr;
    t.trad = nullptr;
    if (p && p->precision != VB_PREC_FP32) {
        t.blk = c.take<unsigned char>((size_t)(npad / TILE) * tcp_blk_bytes(pad_k16(m)));
        t.lbw = c.take<uint32_t>((size_t)TCP_MAX_CTAS * ntiles);
        t.tlist = c.take<uint64_t>((size_t)TCP_MAX_CTAS * ntiles);
        t.lbs = c.take<uint4>((size_t)TCP_MAX_CTAS * ntiles);
        t.crange = c.take<int>(256);
        t.trad = c.take<float>(ntiles);
    }
    if (w) *w = t;
    return c.off;
}

// ------------------------------------------------------------------ a1: order
__device__ __forceinline__ int f2ord(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void bbox_init_kernel(int* bbox, int* fb_count)
{
    int t = threadIdx.x;
    if (t < 8) bbox[t] = 0x7fffffff;
    else if (t < 16) bbox[t] = (int)0x80000000;
    if (t < 8) fb_count[t] = 0;
}

// Bounding box of the Morton coordinates; also rejects non-finite input.
__global__ void bbox_kernel(const float* __restrict__ x, int64_t n, int m, int md, int* bbox, DevReport* rep)
{
    int lo[8], hi[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) { lo[r] = 0x7fffffff; hi[r] = (int)0x80000000; }
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int r = 0; r < m; ++r) {
            float v = x[i * m + r];
            if (!isfinite(v)) bad = true;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q == r && r < md) {
                    int o = f2ord(v);
                    lo[q] = min(lo[q], o);
                    hi[q] = max(hi[q], o);
                }
            }
        }
    }
    if (bad) report_error(rep, VB_ERR_DEGENERATE);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        int a = __reduce_min_sync(0xffffffffu, lo[r]);
        int b = __reduce_max_sync(0xffffffffu, hi[r]);
        if ((threadIdx.x & 31) == 0 && r < md) {
            atomicMin(&bbox[r], a);
            atomicMax(&bbox[8 + r], b);
        }
    }
}

// Hilbert curve index of md coordinates of `bits` bits each, by Skilling's transpose method
// (J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707, 2004): undo the excess
// work of the coordinates from the top bit down (invert the low bits of the first coordinate,
// or exchange them with those of coordinate i), Gray-encode across the coordinates, then
// interleave the bits as a Morton key would.  Consecutive indices are unit steps in space, so
// the 64-point tiles of the order never straddle a jump of the curve, as Morton tiles can.
__device__ __forceinline__ uint32_t hilbert_key(uint32_t (&X)[8], int md, int bits)
{
    const uint32_t M = 1u << (bits - 1);
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
        for (int i = 0; i < md; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    for (int i = 1; i < md; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[md - 1] & Q) t ^= Q - 1;
    for (int i = 0; i < md; ++i) X[i] ^= t;
    uint32_t k = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int r = 0; r < md; ++r) k = (k << 1) | ((X[r] >> b) & 1u);
    return k;
}

__global__ void morton_kernel(const float* __restrict__ x, int64_t n, int m, int md, int bits,
                              const int* __restrict__ bbox, uint32_t* key, uint32_t* val, int hilbert)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float qmax = (float)((1u << bits) - 1u);
    uint32_t q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int r = 0; r < md; ++r) {
        float lo = ord2f(bbox[r]), hi = ord2f(bbox[8 + r]);
        float ext = hi - lo;
        float s = ext > 0.f ? qmax / ext : 0.f;
        float v = fminf(fmaxf((x[i * m + r] - lo) * s, 0.f), qmax);
        q[r] = min((uint32_t)v, (1u << bits) - 1u);
    }
    uint32_t k = 0;
    if (hilbert) {
        k = hilbert_key(q, md, bits);
    } else {
        for (int b = bits - 1; b >= 0; --b)
            for (int r = 0; r < md; ++r) k = (k << 1) | ((q[r] >> b) & 1u);
    }
    key[i] = k;
    val[i] = (uint32_t)i;
}

// ---- m > 4: the Morton key is built on the projections onto the cloud's PCA_D leading
// principal axes, so that 64-point tiles are compact in the directions the points spread
// along (the first coordinates of a wide input need not be those).  The axes only decide
// the order of the search; the neighbour lists are exact whatever they are.
constexpr int PCA_SAMPLE = 16384;   // rows sampled for the second moments
constexpr int PCA_ROWS = 64;        // sampled rows staged per step
constexpr int PCA_BLOCKS = 16;      // blocks of the moment pass (few, so few atomics)
constexpr int PCA_EPT = 65;         // moments per thread: (128 * 128 + 128) / 256 rounded up
constexpr int PCA_ITERS = 40;       // subspace iterations

__global__ void pca_zero_kernel(double* mom, int64_t len)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        mom[i] = 0.0;
}

// Sampled first and second moments: mom[0] = rows, mom[1 + r] = sum x_r, mom[1 + m + r m + c] = sum x_r x_c.
// Each of PCA_BLOCKS blocks sums its share of the sampled rows in FP32 registers, then adds
// them to the FP64 totals once.
__global__ void __launch_bounds__(256) pca_moments_kernel(const float* __restrict__ x, int64_t n, int m, int64_t stride,
                                                        int64_t rows, double* mom)
{
    __shared__ float xs[PCA_ROWS][128];
    const int t = threadIdx.x;
    const int ne = m * m + m;
    float acc[PCA_EPT];
#pragma unroll
    for (int j = 0; j < PCA_EPT; ++j) acc[j] = 0.f;
    int64_t taken = 0;
    for (int64_t r0 = (int64_t)blockIdx.x * PCA_ROWS; r0 < rows; r0 += (int64_t)gridDim.x * PCA_ROWS) {
        const int nr = (int)min((int64_t)PCA_ROWS, rows - r0);
        __syncthreads();
        for (int i = t; i < nr * m; i += blockDim.x) {
            const int rr = i / m, c = i - rr * m;
            xs[rr][c] = x[(r0 + rr) * stride * m + c];
        }
        __syncthreads();
        taken += nr;
#pragma unroll
        for (int j = 0; j < PCA_EPT; ++j) {
            const int e = t + j * 256;
            if (e < m * m) {
                const int a = e / m, b = e - a * m;
                for (int rr = 0; rr < nr; ++rr) acc[j] = fmaf(xs[rr][a], xs[rr][b], acc[j]);
            } else if (e < ne) {
                const int a = e - m * m;
                for (int rr = 0; rr < nr; ++rr) acc[j] += xs[rr][a];
            }
        }
    }
#pragma unroll
    for (int j = 0; j < PCA_EPT; ++j) {
        const int e = t + j * 256;
        if (e < m * m) atomicAdd(&mom[1 + m + e], (double)acc[j]);
        else if (e < ne) atomicAdd(&mom[1 + (e - m * m)], (double)acc[j]);
    }
    if (t == 0) atomicAdd(&mom[0], (double)taken);
}

// One block: covariance from the moments, then PCA_ITERS steps of subspace iteration
// V <- orth(C V) for PCA_D columns (modified Gram-Schmidt); writes V (m x PCA_D).
__global__ void __launch_bounds__(256) pca_axes_kernel(double* mom, int m, float* C)
{
    __shared__ float V[128][PCA_D], Wm[128][PCA_D];
    __shared__ float red[8];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const double N = fmax(mom[0], 1.0);
    const double* mu = mom + 1;
    const double* S = mom + 1 + m;
    for (int i = t; i < m * m; i += blockDim.x) {   // covariance, FP32 from here on
        const int r = i / m, c = i - r * m;
        C[i] = (float)(S[i] / N - (mu[r] / N) * (mu[c] / N));
    }
    for (int i = t; i < m * PCA_D; i += blockDim.x) {   // a fixed, well-spread start
        const int r = i / PCA_D, d = i - r * PCA_D;
        const uint32_t h = (uint32_t)(r * 2654435761u) ^ (uint32_t)(d * 40503u + 0x9e3779b9u);
        V[r][d] = (float)((h >> 8) & 0xffff) / 65536.f - 0.5f + (r % PCA_D == d ? 1.f : 0.f);
    }
    __syncthreads();
    for (int it = 0; it < PCA_ITERS; ++it) {
        for (int i = t; i < m * PCA_D; i += blockDim.x) {   // W = C V, C = S / N - mu mu^T
            const int r = i / PCA_D, d = i - r * PCA_D;
            float acc = 0.f;
            for (int c = 0; c < m; ++c) acc = fmaf(C[r * m + c], V[c][d], acc);
            Wm[r][d] = acc;
        }
        __syncthreads();
        for (int d = 0; d < PCA_D; ++d) {   // Gram-Schmidt on column d against the earlier ones
            for (int e = 0; e <= d; ++e) {
                float part = 0.f;
                for (int r = t; r < m; r += blockDim.x) part += (e < d ? V[r][e] : Wm[r][d]) * Wm[r][d];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                if (lane == 0) red[w] = part;
                __syncthreads();
                float dot = 0.f;
                for (int q = 0; q < 8; ++q) dot += red[q];
                __syncthreads();
                if (e < d) {
                    for (int r = t; r < m; r += blockDim.x) Wm[r][d] -= dot * V[r][e];
                } else {
                    const float inv = dot > 0.f ? rsqrtf(dot) : 0.f;
                    for (int r = t; r < m; r += blockDim.x) V[r][d] = Wm[r][d] * inv;
                }
                __syncthreads();
            }
        }
    }
    double* out = mom + 1 + m + (size_t)m * m;
    for (int i = t; i < m * PCA_D; i += blockDim.x) out[i] = (double)V[i / PCA_D][i % PCA_D];
}

// Projections of every point on the axes: proj[i][d] = sum_r x_ir V_rd.
__global__ void pca_project_kernel(const float* __restrict__ x, int64_t n, int m, const double* __restrict__ axes,
                                   float* proj)
{
    __shared__ float V[128 * PCA_D];
    for (int i = threadIdx.x; i < m * PCA_D; i += blockDim.x) V[i] = (float)axes[i];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc[PCA_D] = {};
    for (int r = 0; r < m; ++r) {
        const float v = x[i * m + r];
#pragma unroll
        for (int d = 0; d < PCA_D; ++d) acc[d] = fmaf(v, V[r * PCA_D + d], acc[d]);
    }
#pragma unroll
    for (int d = 0; d < PCA_D; ++d) proj[i * PCA_D + d] = acc[d];
}

// Key of the cloud passes: the cloud of each point, in the current (Morton) order.
__global__ void cloud_key_kernel(const uint32_t* __restrict__ val, int64_t n, Clouds cl, uint32_t* key)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) key[i] = (uint32_t)cloud_id(cl, (int64_t)val[i]);
}

__global__ void radix_hist_kernel(const uint32_t* __restrict__ key, int64_t n, int shift, uint32_t* hist, int nblk)
{
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RADIX_ITEMS;
    for (int r = 0; r < RADIX_ITEMS / RADIX_T; ++r) {
        int64_t e = base + r * RADIX_T + threadIdx.x;
        if (e < n) atomicAdd(&cnt[(key[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// In-place exclusive scan of len uint32 values: per-block sums of 8192 values, one
// block scans the block sums, then every block rescans its chunk with its offset.
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* sh, uint32_t* total)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t z = sh[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        sh[lane] = z;
    }
    __syncthreads();
    const uint32_t r = x - v + (w ? sh[w - 1] : 0u);
    if (total) *total = sh[31];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(USCAN_T) uscan_reduce_kernel(const uint32_t* __restrict__ a, int64_t len,
                                                              uint32_t* bsum)
{
    __shared__ uint32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * USCAN_CHUNK + (int64_t)threadIdx.x * USCAN_ITEMS;
    uint32_t v = 0;
#pragma unroll
    for (int i = 0; i < USCAN_ITEMS; ++i)
        if (base + i < len) v += a[base + i];
    uint32_t tot;
    block_excl_scan_u32(v, sh, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(USCAN_T) uscan_top_kernel(uint32_t* bsum, int nb)
{
    __shared__ uint32_t sh[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += USCAN_T) {
        const int i = b0 + threadIdx.x;
        const uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan_u32(v, sh, &tot);
        if (i < nb) bsum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(USCAN_T) uscan_apply_kernel(uint32_t* a, int64_t len, const uint32_t* __restrict__ bsum)
{
    __shared__ uint32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * USCAN_CHUNK + (int64_t)threadIdx.x * USCAN_ITEMS;
    uint32_t v[USCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < USCAN_ITEMS; ++i) {
        v[i] = base + i < len ? a[base + i] : 0u;
        s += v[i];
    }
    uint32_t run = (bsum ? bsum[blockIdx.x] : 0u) + block_excl_scan_u32(s, sh, nullptr);
#pragma unroll
    for (int i = 0; i < USCAN_ITEMS; ++i) {
        if (base + i < len) a[base + i] = run;
        run += v[i];
    }
}

// Returns the number of kernels launched (one when len fits a single chunk).
static int scan_u32(cudaStream_t s, uint32_t* a, int64_t len, uint32_t* bsum)
{
    const int nb = (int)((len + USCAN_CHUNK - 1) / USCAN_CHUNK);
    if (nb == 1) {
        uscan_apply_kernel<<<1, USCAN_T, 0, s>>>(a, len, nullptr);
        return 1;
    }
    uscan_reduce_kernel<<<nb, USCAN_T, 0, s>>>(a, len, bsum);
    uscan_top_kernel<<<1, USCAN_T, 0, s>>>(bsum, nb);
    uscan_apply_kernel<<<nb, USCAN_T, 0, s>>>(a, len, bsum);
    return 3;
}

// Stable scatter: inside a block, rounds of 256 consecutive keys; inside a
// round the order is (warp, lane), ranked with __match_any_sync.
__global__ void radix_scatter_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                     uint32_t* kout, uint32_t* vout, int64_t n, int shift,
                                     const uint32_t* __restrict__ hist, int nblk)
{
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[RADIX_T / 32][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    base[t] = hist[(int64_t)t * nblk + blockIdx.x];
    int64_t b0 = (int64_t)blockIdx.x * RADIX_ITEMS;
    for (int r = 0; r < RADIX_ITEMS / RADIX_T; ++r) {
        for (int i = t; i < (RADIX_T / 32) * 256; i += RADIX_T) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        int64_t e = b0 + r * RADIX_T + t;
        bool ok = e < n;
        uint32_t k = ok ? kin[e] : 0u, v = ok ? vin[e] : 0u;
        uint32_t dg = (k >> shift) & 255u;
        unsigned act = __ballot_sync(0xffffffffu, ok);
        unsigned peers = 0;
        if (ok) {
            peers = __match_any_sync(act, dg);
            int leader = __ffs(peers) - 1;
            if (lane == leader) wcnt[w][dg] = __popc(peers);
        }
        __syncthreads();
        if (ok) {
            uint32_t off = base[dg] + __popc(peers & ((1u << lane) - 1u));
            for (int ww = 0; ww < w; ++ww) off += wcnt[ww][dg];
            kout[off] = k;
            vout[off] = v;
        }
        __syncthreads();
        uint32_t add = 0;
        for (int ww = 0; ww < RADIX_T / 32; ++ww) add += wcnt[ww][t];
        base[t] += add;
        __syncthreads();
    }
}

__global__ void gather_kernel(const float* __restrict__ x, const uint32_t* __restrict__ perm, int64_t n,
                              int64_t npad, int m, int mp, float* xs, double* xs64)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad * mp) return;
    int64_t p = i / mp;
    int r = (int)(i - p * mp);
    const float v = (p < n && r < m) ? x[(int64_t)perm[p] * m + r] : 0.f;
    xs[i] = v;
    xs64[i] = (double)v;
}

// One warp per tile: radius of the ball about the tile's box centre that holds its valid
// points, rounded up past the FP32 error of the sum (relative (m + 2) 2^-24 on the square).
__global__ void tile_ball_kernel(const float* __restrict__ xs, int64_t n, int64_t ntiles, int m, int mp,
                                 const float* __restrict__ tlo, const float* __restrict__ thi, float* trad)
{
    const int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= ntiles) return;
    const int64_t p0 = tile * TILE + lane, p1 = p0 + 32;
    float s0 = 0.f, s1 = 0.f;
    for (int r = 0; r < m; ++r) {
        const float c = 0.5f * (tlo[tile * mp + r] + thi[tile * mp + r]);
        if (p0 < n) { const float d = xs[p0 * mp + r] - c; s0 = fmaf(d, d, s0); }
        if (p1 < n) { const float d = xs[p1 * mp + r] - c; s1 = fmaf(d, d, s1); }
    }
    float sm = fmaxf(s0, s1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
    if (lane == 0) trad[tile] = __fmul_ru(sqrtf(sm), 1.00002f);
}

// One warp per tile: bounding box of its valid points (padding dims stay 0).
__global__ void tile_box_kernel(const float* __restrict__ xs, int64_t n, int64_t ntiles, int m, int mp,
                                float* tlo, float* thi)
{
    int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (tile >= ntiles) return;
    int64_t p0 = tile * TILE + lane, p1 = p0 + 32;
    for (int r = 0; r < mp; ++r) {
        float lo = INFINITY, hi = -INFINITY;
        if (p0 < n) { float v = xs[p0 * mp + r]; lo = fminf(lo, v); hi = fmaxf(hi, v); }
        if (p1 < n) { float v = xs[p1 * mp + r]; lo = fminf(lo, v); hi = fmaxf(hi, v); }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            tlo[tile * mp + r] = r < m ? lo : 0.f;
            thi[tile * mp + r] = r < m ? hi : 0.f;
        }
    }
}

// Box of every super-tile of 64 consecutive tiles (the union of their boxes), one warp each:
// a query tile skips a whole super-tile whose box lies beyond its threshold.
__global__ void super_box_kernel(const float* __restrict__ tlo, const float* __restrict__ thi, int64_t ntiles, int mp,
                                 float* slo, float* shi)
{
    const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= (ntiles + TILE - 1) / TILE) return;
    const int64_t t0 = g * TILE + lane, t1 = t0 + 32;
    for (int r = 0; r < mp; ++r) {
        float lo = INFINITY, hi = -INFINITY;
        if (t0 < ntiles) { lo = tlo[t0 * mp + r]; hi = thi[t0 * mp + r]; }
        if (t1 < ntiles) { lo = fminf(lo, tlo[t1 * mp + r]); hi = fmaxf(hi, thi[t1 * mp + r]); }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            slo[g * mp + r] = lo;
            shi[g * mp + r] = hi;
        }
    }
}

// ------------------------------------------------------------------ a2-a5: the tiled search
__device__ __forceinline__ double canon_d2(const float* a, const float* b, int m)
{
    double acc = 0.0;
    for (int r = 0; r < m; ++r) {
        double dl = __dsub_rn((double)a[r], (double)b[r]);
        double s = __dmul_rn(dl, dl);
        acc = r == 0 ? s : __dadd_rn(acc, s);
    }
    return acc;
}

// canon_d2 on FP64 copies of the FP32 coordinates: the same arithmetic (the FP32 to
// FP64 conversion is exact), without the conversions, which occupy the narrow FP64 pipe.
__device__ __forceinline__ double canon_d2_64(const double* a, const double* __restrict__ b, int m)
{
    double acc = 0.0;
    for (int r = 0; r < m; ++r) {
        const double dl = __dsub_rn(a[r], b[r]);
        const double s = __dmul_rn(dl, dl);
        acc = r == 0 ? s : __dadd_rn(acc, s);
    }
    return acc;
}

// The same for a query held in registers (q[0..MP)) and a 16-byte aligned candidate row.
template <int MP>
__device__ __forceinline__ double canon_d2_q64(const double* q, const double* __restrict__ c, int m)
{
    double cv[MP];
#pragma unroll
    for (int r2 = 0; r2 < MP / 2; ++r2) {
        const double2 v = *(const double2*)(c + 2 * r2);
        cv[2 * r2] = v.x;
        cv[2 * r2 + 1] = v.y;
    }
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < MP; ++r) {
        if (r < m) {
            const double dl = __dsub_rn(q[r], cv[r]);
            const double sq = __dmul_rn(dl, dl);
            acc = r == 0 ? sq : __dadd_rn(acc, sq);
        }
    }
    return acc;
}

struct TileArgs {
    const float* xs;
    const double* xs64;   // FP64 copies of xs (exact), for the FP64 rescoring
    const float* tlo;
    const float* thi;
    const float* slo;     // boxes of super-tiles (64 consecutive tiles; FP32 search)
    const float* shi;
    const uint32_t* perm;
    int64_t n;
    int64_t ntiles;
    int m, k, L, prune, nseed;
    float lb_factor;     // 1 - 4 (m + 2) 2^-24, applied rounding down
    float band;          // 1 + 4 (m + 2) 2^-24: FP32 distances closer than this may swap in FP64
    double cert_factor;  // 1 - 2 (m + 2) 2^-24
    int32_t* nbr;
    double* nbr_d2;
    int* fb_list;
    int* fb_count;
    int* work;           // next query tile (persistent grid)
    const int* tile_list;   // optional list of query tiles to process (else all tiles)
    const int* tile_count;  // its length (device)
    const float* r2;        // radius search: per sorted point, squared radius bound
    float r2_scale;         // radius search: factor on r2 for this pass
    int count_retries;      // radius search: count the tiles this pass hands on (last pass only)
    int cap;                // radius search: candidates kept per query
    int* fail_flag;         // radius search: per query tile, set once it joins fail_list
    int* fail_list;
    int* fail_count;
    Clouds cl;              // batched build: queries only take candidates from their own cloud
    DevReport* rep;
    // pipelined 16-bit search
    const unsigned char* blk;   // tile blocks (operand image + norms), tcp_blk_bytes(kp) each
    int kp;                     // K: m padded to 16
    int stages;                 // ring slots of staged tile blocks
    uint32_t* lbw;              // per CTA scratch: ntiles box bounds
    uint64_t* tlist;            // per CTA scratch: ntiles (bound, tile) keys in bound order
    uint4* lbs;                 // per CTA scratch: ntiles bounds of the four 32-query groups
    const float* trad;          // per tile: radius of its ball about the box centre (pipelined search)
    uint64_t* hdump;            // pipelined search: heaps handed to its row finish ([L][128] per query tile)
    float* dbg_d2;              // diagnostic: kept 16-bit distances per row ([n][L], original order)
    int32_t* dbg_idx;           // their original indices
};

constexpr int IB = 8;         // candidate distances computed per batch before any insertion
constexpr int SCAP = 256;     // candidate tiles per sorted chunk
constexpr int FLAT_SUPERS = 16;   // up to this many super-tiles (64 tiles each) in range: one-level scan
constexpr int RUN = 8;        // longest run of FP32-indistinguishable neighbours ordered in registers
constexpr int FB = 8;         // keys rescored per batch in the 16-bit row finish
constexpr int FB_ROW = 4;     // the same in the FP32 row finish (fewer registers: more CTAs per SM)

// Sift key down from node i of the max-heap heap[0..size) (column t of a [.][COLS] array).
template <int COLS = TILE, class K>
__device__ __forceinline__ void sift_down(K* heap, int t, int i, int size, K key, unsigned& levels)
{
    for (;;) {
        int l = 2 * i + 1;
        if (l >= size) break;
        ++levels;
        K ck = heap[l * COLS + t];
        int ch = l;
        if (l + 1 < size) {
            K rk = heap[(l + 1) * COLS + t];
            if (rk > ck) { ck = rk; ch = l + 1; }
        }
        if (ck <= key) break;
        heap[i * COLS + t] = ck;
        i = ch;
    }
    heap[i * COLS + t] = key;
}

// The same for a D-ary max-heap (children of node i: D i + 1 .. D i + D).  The D child loads
// of a level are independent, so a level costs one shared-memory round trip, and the heap is
// log_D of its size deep: fewer dependent round trips per insertion than the binary heap's.
template <int COLS, int D, class K>
__device__ __forceinline__ void sift_down_d(K* heap, int t, int i, int size, K key, unsigned& levels)
{
    for (;;) {
        const int c = D * i + 1;
        if (c >= size) break;
        ++levels;
        K ck[D];
#pragma unroll
        for (int j = 0; j < D; ++j) ck[j] = c + j < size ? heap[(c + j) * COLS + t] : (K)0;   // 0: no child
        K best = ck[0];
        int bc = c;
#pragma unroll
        for (int j = 1; j < D; ++j)
            if (ck[j] > best) { best = ck[j]; bc = c + j; }
        if (best <= key) break;
        heap[i * COLS + t] = best;
        i = bc;
    }
    heap[i * COLS + t] = key;
}

// v[i] for a run-time i in [0, N), N a power of two, from registers: a tree of selects on the
// bits of i, log2 N deep, instead of a chain of N dependent ones.
template <int N> struct Pick {
    static __device__ __forceinline__ float get(const float* v, int i)
    {
        float h[N / 2];
        const bool b = i & 1;
#pragma unroll
        for (int j = 0; j < N / 2; ++j) h[j] = b ? v[2 * j + 1] : v[2 * j];
        return Pick<N / 2>::get(h, i >> 1);
    }
};
template <> struct Pick<1> {
    static __device__ __forceinline__ float get(const float* v, int) { return v[0]; }
};

// Floyd's bottom-up construction of a max-heap over heap[0..size).
template <int COLS = TILE, class K>
__device__ __forceinline__ void heapify(K* heap, int t, int size, unsigned& levels)
{
    for (int i = size / 2 - 1; i >= 0; --i) sift_down<COLS>(heap, t, i, size, heap[i * COLS + t], levels);
}

// Heap keys of the FP32 search.  Full: FP32 distance bits << 32 | sorted position.
// Compact (32-bit, half the shared memory, so twice the CTAs per SM): the distance bits
// truncated to 18 (sign dropped, 8 exponent and 10 mantissa bits: the key is a lower edge of
// a bucket 2^-10 wide) << 14 | slot, slot = visit number << 6 | lane of the candidate tile;
// the CTA keeps the tile of every visit number.  Both order by distance first.
template <bool K32> struct KeyOps;
template <> struct KeyOps<false> {
    using T = uint64_t;
    static constexpr T EMPTY = ~0ull;
    // FP32 bits no smaller than the distance of any key <= k
    static __device__ __forceinline__ uint32_t dist_hi(T k) { return (uint32_t)(k >> 32); }
    static __device__ __forceinline__ T make(uint32_t dbits, int, int, int64_t cp)
    {
        return ((uint64_t)dbits << 32) | (uint32_t)cp;
    }
};
constexpr int VMAX = 255;      // visits a compact-key query tile may make (slot 0x3fff stays unused)
template <> struct KeyOps<true> {
    using T = uint32_t;
    static constexpr T EMPTY = ~0u;
    static __device__ __forceinline__ uint32_t dist_hi(T k) { return k == ~0u ? ~0u : (((k >> 14) << 13) | 0x1fffu); }
    static __device__ __forceinline__ T make(uint32_t dbits, int vis, int c, int64_t)
    {
        return ((dbits >> 13) << 14) | ((uint32_t)vis << 6) | (uint32_t)c;
    }
};

template <int MP>
__device__ __forceinline__ float point_box_lb(const float* q, const float* lo, const float* hi)
{
    float acc = 0.f;
#pragma unroll
    for (int r = 0; r < MP; ++r) {
        float g = fmaxf(fmaxf(lo[r] - q[r], q[r] - hi[r]), 0.f);
        acc = fmaf(g, g, acc);
    }
    return acc;
}

// Orders the candidates of one query and writes its row (step a5).  arr[0..size)
// holds keys (FP32 distance bits << 32 | sorted position), column t of a [.][TILE]
// array; is_heap says whether it already is a max-heap.  After an in-place heap
// sort the keys are walked in ascending order: FP64 canonical distances are
// computed for the first k (plus the run straddling rank k), and keys whose FP32
// distances lie within the error band of each other ("runs") are ordered exactly
// by (d2, index) in registers.  Certificate: the largest kept FP32 distance bounds
// every excluded candidate, and the k-th FP64 distance must lie below it minus the
// relative FP32 error band.  Returns false when the row needs the exact fallback.
// Compact keys (K = uint32_t) decode through vtab, the tile of every visit number, and carry
// a distance bucket [lo, hi] instead of a value: runs and the certificate use its edges.
template <int MP, int COLS = TILE, class K = uint64_t>
__device__ bool finalize_row(const TileArgs& a, K* arr, int t, int size, bool is_heap, int64_t pq,
                             int64_t ncl, unsigned& levels, const int* vtab = nullptr, int* short_flag = nullptr)
{
    constexpr bool K32 = sizeof(K) == 4;
    constexpr K EMPTY = (K)~(K)0;
    if (!is_heap) heapify<COLS>(arr, t, size, levels);
    for (int e = size - 1; e > 0; --e) {
        const K top = arr[t];
        const K key = arr[e * COLS + t];
        arr[e * COLS + t] = top;
        sift_down<COLS>(arr, t, 0, e, key, levels);
    }
    const K Hkey = arr[(size - 1) * COLS + t];
    const uint32_t oq = a.perm[pq];
    const double* qc = a.xs64 + pq * MP;
    constexpr bool QR = MP <= 16;
    double qv[QR ? MP : 1];
    if constexpr (QR) {
#pragma unroll
        for (int r = 0; r < MP; ++r) qv[r] = qc[r];
    }
    uint64_t rd[RUN];   // FP64 distance bits
    uint32_t ro[RUN];
    int rlen = 0, out = 0;
    float run_last = 0.f;
    bool ok = true, done = false;
    double dk = 0.0;
    auto emit = [&]() {
#pragma unroll
        for (int u = 0; u < RUN; ++u) {
            if (u < rlen && out < a.k) {
                a.nbr[(int64_t)oq * a.k + out] = (int32_t)ro[u];
                a.nbr_d2[(int64_t)oq * a.k + out] = __longlong_as_double((long long)rd[u]);
                if (out == a.k - 1) dk = __longlong_as_double((long long)rd[u]);
                ++out;
            }
        }
        rlen = 0;
    };
    // keys are taken FB_ROW at a time: their index and coordinate loads are issued together
    for (int r0 = 0; r0 < size && !done; r0 += FB_ROW) {
        uint32_t cpb[FB_ROW], ojb[FB_ROW];
        uint64_t djb[FB_ROW];
        float dfb[FB_ROW], dfh[FB_ROW];
#pragma unroll
        for (int u = 0; u < FB_ROW; ++u) {
            const K key = r0 + u < size ? arr[(r0 + u) * COLS + t] : EMPTY;
            if constexpr (K32) {
                const uint32_t slot = key & 0x3fffu, q = (key >> 14) << 13;
                // slot 0x3fff: an empty slot or a radius sentinel (visit numbers stop at VMAX - 1)
                cpb[u] = slot == 0x3fffu ? 0xffffffffu : (uint32_t)vtab[slot >> 6] * TILE + (slot & 63u);
                dfb[u] = __uint_as_float(q);
                dfh[u] = __uint_as_float(q | 0x1fffu);
            } else {
                cpb[u] = (uint32_t)key;
                dfb[u] = dfh[u] = __uint_as_float((uint32_t)(key >> 32));
            }
        }
#pragma unroll
        for (int u = 0; u < FB_ROW; ++u) {
            ojb[u] = 0;
            djb[u] = 0;
            if (cpb[u] != 0xffffffffu) {
                ojb[u] = a.perm[cpb[u]];
                double d;
                if constexpr (QR) d = canon_d2_q64<MP>(qv, a.xs64 + (int64_t)cpb[u] * MP, a.m);
                else d = canon_d2_64(qc, a.xs64 + (int64_t)cpb[u] * MP, a.m);
                djb[u] = (uint64_t)__double_as_longlong(d);
            }
        }
#pragma unroll
        for (int u = 0; u < FB_ROW; ++u) {
            if (done) break;
            if (cpb[u] == 0xffffffffu) { done = true; break; }   // empty slot or radius sentinel
            const float df = dfb[u];
            // a new run starts once the distance clears the error band (tiny distances, where
            // FP32 may have underflowed, and overflowed ones all stay in one run)
            if (rlen > 0 && df > run_last * a.band && df > 1e-30f && df <= 3.402823466e38f) {
                emit();
                if (out >= a.k) { done = true; break; }
            }
            if (rlen == RUN) { ok = false; done = true; break; }
            const uint64_t dj = djb[u];
            const uint32_t oj = ojb[u];
            // insert (dj, oj) into the run, kept sorted by (d2, index); non-negative doubles
            // order like their bit patterns, so the comparisons stay on the integer pipe
#pragma unroll
            for (int v = 0; v < RUN; ++v)
                if (v == rlen) { rd[v] = dj; ro[v] = oj; }
#pragma unroll
            for (int v = RUN - 1; v > 0; --v) {
                if (v <= rlen && (rd[v] < rd[v - 1] || (rd[v] == rd[v - 1] && ro[v] < ro[v - 1]))) {
                    uint64_t td = rd[v]; rd[v] = rd[v - 1]; rd[v - 1] = td;
                    uint32_t to = ro[v]; ro[v] = ro[v - 1]; ro[v - 1] = to;
                }
            }
            ++rlen;
            run_last = dfh[u];
        }
    }
    if (ok && out < a.k) emit();
    if (!ok) { atomicAdd(&a.rep->knn_rows_long_run, 1ull); return false; }
    if (out < a.k) {
        atomicAdd(&a.rep->knn_rows_short, 1ull);
        if (short_flag) *short_flag = 1;
        return false;
    }
    // every candidate was kept (a small cloud without a radius, or an unfilled heap); a radius
    // excludes the candidates beyond it even in a small cloud, so the certificate decides there
    if ((ncl - 1 <= (int64_t)size && !a.r2) || Hkey == EMPTY) return true;
    float B;
    // the lower edge of the largest kept key's bucket; a radius sentinel's own bucket holds no
    // excluded candidate (one there has a smaller key and is kept), so the next bucket's edge
    if constexpr (K32) B = __uint_as_float(((Hkey >> 14) + ((Hkey & 0x3fffu) == 0x3fffu ? 1u : 0u)) << 13);
    else B = __uint_as_float((uint32_t)(Hkey >> 32));
    const bool cert = isfinite(B) && dk < (double)B * a.cert_factor - (double)a.m * 1.1754943508222875e-38;
    if (!cert) atomicAdd(&a.rep->knn_rows_uncertified, 1ull);
    return cert;
}

// Error model of the 16-bit distance tiles.  Operands are q' = q - c0 and x' = x - c0
// (c0 the query tile's box centre) rounded to 16 bits with unit roundoff u, plus an
// absolute term for FP16 subnormals; the approximate distance |q~|^2 + |x~|^2 - 2 q~.x~
// is formed with FP32 sums and the tensor cores' FP32 accumulation.  For a pair at
// exact distance d <= D, |x'| <= |q'| + sqrt(D), so with Z = 2 |q'| + sqrt(D):
//     |d~ - d| <= E_D(d) = 2 sqrt(d) delta + delta^2 + rho,
//     delta = u Z + delta_abs,  rho = 2 (K + 4) 2^-24 Z^2.
// Every use below takes D = the current k-th FP64 distance of the row, so the
// bound covers exactly the candidates that could still enter the row.
struct Band {
    float u, dabs, rho_k;   // unit roundoff, absolute term, 2 (K + 4) 2^-24
    // E_D(d) with sD = sqrt(D) rounded up.  Evaluated in FP32: its own rounding (a few ulps over
    // the dozen operations) is far inside the outer factor 1.02 (the bound itself needs 1.01),
    // and the absolute floor covers subnormal intermediates; an overflow gives +inf, which only
    // makes the scan longer or the certificate fail.
    __device__ __forceinline__ float E(float qn, float sD, float d) const
    {
        const float Z = 1.01f * (2.f * qn + sD);
        const float delta = u * Z * 1.01f + dabs;
        return 1.02f * (2.f * __fsqrt_ru(fmaxf(d, 0.f)) * delta + delta * delta + rho_k * Z * Z) + 1e-37f;
    }
    static __device__ __forceinline__ float root_up(double D) { return __fsqrt_ru(__double2float_ru(D)); }
};

// Rescoring for 16-bit distance tiles, whose error band is wide enough that long
// runs of candidates are indistinguishable.  The kept keys, ascending by
// approximate distance df, are rescored in FP64 one by one and inserted into the
// output row, which stays sorted by (d2, index).  A key whose exact distance could
// still be below the current k-th distance dk has df <= dk + E_dk(dk), so the scan
// stops once df - E_dk(df) passes dk.  Certificate: every excluded candidate has
// df >= B (the largest kept key, or the radius sentinel), so none can lie below
// dk when dk < (B - E_dk(B)) (1 - 2 gamma); far operands clamped to +-30000 in FP16
// lie at exact distance >= 4e8, which the certificate also requires dk to stay below.
// Keys of the 16-bit searches.  Full (64-bit): FP32 bits of the tile distance << 32 | sorted
// position; the radius sentinel carries position 0xffffffff.  Compact (32-bit, the staged
// kernel at m <= 16): the distance bits truncated to 18 << 14 | slot, slot = visit << 6 | lane,
// with the CTA's table of the tile of every visit; slot 0x3fff marks a sentinel.  A compact key
// stands for a bucket [lo, hi] of distances: lo bounds every distance of the bucket from
// below (the scan's stop test), hi from above (the filter).
template <class K> struct BandKey;
template <> struct BandKey<uint64_t> {
    static constexpr uint64_t EMPTY = ~0ull;
    static __device__ __forceinline__ bool none(uint64_t k) { return (uint32_t)k == 0xffffffffu; }
    static __device__ __forceinline__ float lo(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
    static __device__ __forceinline__ uint32_t hi_bits(uint64_t k) { return (uint32_t)(k >> 32); }
    static __device__ __forceinline__ uint32_t pos(uint64_t k, const int*) { return (uint32_t)k; }
    static __device__ __forceinline__ uint64_t make(uint32_t dbits, int, int, uint32_t cp)
    {
        return ((uint64_t)dbits << 32) | cp;
    }
    static __device__ __forceinline__ uint64_t sentinel(uint32_t r2bits) { return ((uint64_t)r2bits << 32) | 0xffffffffu; }
    static __device__ __forceinline__ float excl(uint64_t k) { return lo(k); }
};
template <> struct BandKey<uint32_t> {
    static constexpr uint32_t EMPTY = ~0u;
    static __device__ __forceinline__ bool none(uint32_t k) { return (k & 0x3fffu) == 0x3fffu; }
    static __device__ __forceinline__ float lo(uint32_t k) { return __uint_as_float((k >> 14) << 13); }
    static __device__ __forceinline__ uint32_t hi_bits(uint32_t k) { return k == ~0u ? ~0u : (((k >> 14) << 13) | 0x1fffu); }
    static __device__ __forceinline__ uint32_t pos(uint32_t k, const int* vtab)
    {
        return (uint32_t)vtab[(k >> 6) & 0xffu] * TILE + (k & 63u);
    }
    static __device__ __forceinline__ uint32_t make(uint32_t dbits, int vis, int lane, uint32_t)
    {
        return ((dbits >> 13) << 14) | ((uint32_t)vis << 6) | (uint32_t)lane;
    }
    static __device__ __forceinline__ uint32_t sentinel(uint32_t r2bits) { return ((r2bits >> 13) << 14) | 0x3fffu; }
    // a lower bound of every candidate left out of a heap whose largest key is k: a sentinel's
    // own bucket holds none (a candidate there has a smaller key and is kept)
    static __device__ __forceinline__ float excl(uint32_t k)
    {
        return __uint_as_float(((k >> 14) + (none(k) ? 1u : 0u)) << 13);
    }
};

template <int MP, int COLS, class K = uint64_t, int D = 2>
__device__ bool finalize_row_band(const TileArgs& a, K* arr, int t, int size, int64_t pq, int64_t ncl,
                                  unsigned& levels, const Band& bd, float qn, const int* vtab = nullptr,
                                  int* short_flag = nullptr)
{
    using BK = BandKey<K>;
    for (int e = size - 1; e > 0; --e) {   // heap sort (arr is a D-ary max-heap)
        const K top = arr[t];
        const K key = arr[e * COLS + t];
        arr[e * COLS + t] = top;
        sift_down_d<COLS, D>(arr, t, 0, e, key, levels);
    }
    const K Hkey = arr[(size - 1) * COLS + t];
    const uint32_t oq = a.perm[pq];
    if (a.dbg_d2) {   // diagnostic: the kept keys' 16-bit distances, ascending, before any rescoring
        for (int r = 0; r < size && r < a.L; ++r) {
            const K key = arr[r * COLS + t];
            a.dbg_idx[(int64_t)oq * a.L + r] = BK::none(key) ? -1 : (int32_t)a.perm[BK::pos(key, vtab)];
            a.dbg_d2[(int64_t)oq * a.L + r] = BK::lo(key);
        }
    }
    const double* qc = a.xs64 + pq * MP;
    int32_t* on = a.nbr + (int64_t)oq * a.k;
    double* od = a.nbr_d2 + (int64_t)oq * a.k;
    const int k = a.k;
    constexpr bool QR = MP <= 16;
    double qv[QR ? MP : 1];
    if constexpr (QR) {
#pragma unroll
        for (int r = 0; r < MP; ++r) qv[r] = qc[r];
    }
    int out = 0;
    double dk = INFINITY;
    float sD = INFINITY;        // sqrt(dk), rounded up
    double dlast = 0.0;         // the row's last entry so far, (od, on)[out - 1], kept in registers
    int32_t ilast = 0;
    bool done = false;
    // keys are taken FB at a time: their index and coordinate loads are issued together
    for (int r0 = 0; r0 < size && !done; r0 += FB) {
        uint32_t cpb[FB];
        int32_t ojb[FB];
        double djb[FB];
        float dfb[FB];
#pragma unroll
        for (int u = 0; u < FB; ++u) {
            const K key = r0 + u < size ? arr[(r0 + u) * COLS + t] : BK::EMPTY;
            const bool none = BK::none(key);
            cpb[u] = none ? 0xffffffffu : BK::pos(key, vtab);
            dfb[u] = BK::lo(key);
            ojb[u] = 0;
            djb[u] = 0.0;
            if (!none) {
                ojb[u] = (int32_t)a.perm[cpb[u]];
                if constexpr (QR) djb[u] = canon_d2_q64<MP>(qv, a.xs64 + (int64_t)cpb[u] * MP, a.m);
                else djb[u] = canon_d2_64(qc, a.xs64 + (int64_t)cpb[u] * MP, a.m);
            }
        }
#pragma unroll
        for (int u = 0; u < FB; ++u) {
            if (done) break;
            if (cpb[u] == 0xffffffffu) { done = true; break; }   // sentinel: nothing further was kept
            if (out == k && (double)__fsub_rd(dfb[u], bd.E(qn, sD, dfb[u])) * a.cert_factor > dk) {
                done = true;
                break;
            }
            const double dj = djb[u];
            const int32_t oj = ojb[u];
            // insertion into the row, sorted by (d2, index); keys arrive nearly in order, so the
            // common case appends after the last entry, which is compared from registers
            if (out < k) {
                int pos = out;
                if (out > 0 && !(dlast < dj || (dlast == dj && ilast < oj))) {
                    od[pos] = dlast;   // the last entry moves up one; it stays the last
                    on[pos] = ilast;
                    --pos;
                    while (pos > 0) {
                        const double dp = od[pos - 1];
                        const int32_t ip = on[pos - 1];
                        if (dp < dj || (dp == dj && ip < oj)) break;
                        od[pos] = dp;
                        on[pos] = ip;
                        --pos;
                    }
                } else {
                    dlast = dj;
                    ilast = oj;
                }
                od[pos] = dj;
                on[pos] = oj;
                if (++out == k) {
                    dk = dlast;
                    sD = Band::root_up(dk);
                }
            } else {
                if (!(dj < dlast || (dj == dlast && oj < ilast))) continue;
                // the last entry drops out; the new one goes in below it
                double ld = dj;
                int32_t li = oj;
                int pos = k - 1;
                while (pos > 0) {
                    const double dp = od[pos - 1];
                    const int32_t ip = on[pos - 1];
                    if (dp < dj || (dp == dj && ip < oj)) break;
                    od[pos] = dp;
                    on[pos] = ip;
                    if (pos == k - 1) { ld = dp; li = ip; }
                    --pos;
                }
                od[pos] = dj;
                on[pos] = oj;
                dlast = ld;
                ilast = li;
                dk = dlast;
                sD = Band::root_up(dk);
            }
        }
    }
    if (out < k) {
        atomicAdd(&a.rep->knn_rows_short, 1ull);
        if (short_flag) *short_flag = 1;
        return false;
    }
    // every candidate was kept (a small cloud without a radius, or an unfilled heap); with a
    // radius the candidates beyond it were never kept, so the certificate decides
    if ((ncl - 1 <= (int64_t)size && !a.r2) || Hkey == BK::EMPTY) return true;
    const float B = BK::excl(Hkey);
    const bool cert = isfinite(B) && dk < 4e8 &&
                      dk < (double)__fsub_rd(B, bd.E(qn, sD, B)) * a.cert_factor - (double)a.m * 1.1754943508222875e-38;
    if (!cert) atomicAdd(&a.rep->knn_rows_uncertified, 1ull);
    return cert;
}

// Appends key, for the threads whose keep is set, to lst at positions cnt, cnt + 1, ... in
// thread order, and advances cnt (a register, the same in every thread) by the number kept in
// the block.  One barrier.  The per-warp counts go to wc[par], and par alternates between calls:
// a warp that runs ahead to the next call writes the other half while the others still read
// this one, and cannot come back to this half before all of them pass the next barrier.  The
// count is never read from shared memory after the barrier, so no warp can see a count that
// another warp has already advanced (every warp takes the same branch on cnt).
template <int NW>
__device__ __forceinline__ void block_append(uint64_t* lst, int& cnt, bool keep, uint64_t key, int (*wc)[NW], int& par)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wc[par][warp] = __popc(bal);
    __syncthreads();
    int off = cnt, tot = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int c = wc[par][w];
        if (w < warp) off += c;
        tot += c;
    }
    if (keep) lst[off + __popc(bal & ((1u << lane) - 1u))] = key;
    cnt += tot;
    par ^= 1;
}

// Query tiles are taken from a global counter by a persistent grid of 64-thread
// CTAs, one query per thread.  Shared memory:
//   heap  [L][64]  key  max-heap per query of keys (KeyOps: 64-bit full or 32-bit compact)
//   cand  [MP][64] f32  staged candidate tile, coordinate-major (MP <= 16; [64][MP] for wider inputs)
//   qs    [MP][64] f32  query coordinates (MP > 16 only)
//   slist [SCAP]   u64  surviving candidate tiles keyed (box lower bound bits << 32 | tile)
//   vtab  [VMAX]   i32  compact keys: the candidate tile of every visit number
// MR <= MP is the number of coordinates the distance loop reads (the rest are zero padding).
// Up to 10 CTAs per SM for MP <= 8 (at most 102 registers a thread, 21.5 KB of shared memory at
// k + M = 68 with compact keys), 8 for wider inputs, whose query and candidate rows need more.
// With compact keys a query tile that needs more than VMAX visits, or has a row that fails the
// certificate, is listed for the plain search with full keys (a second pass).
template <int MP, int MR = MP, bool K32 = false>
__global__ void __launch_bounds__(TILE, MP <= 8 ? 10 : 8) knn_tile_kernel(TileArgs a)
{
    using KO = KeyOps<K32>;
    using KT = typename KO::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = a.L;
    KT* heap = (KT*)smem;
    uint64_t* slist = (uint64_t*)(heap + (size_t)L * TILE);
    float* cand = (float*)(slist + SCAP);
    float* qs = cand + TILE * MP;
    int* vtab = (int*)(qs + (MP > 16 ? TILE * MP : 0));
    __shared__ float sqlo[MP], sqhi[MP];
    __shared__ uint32_t sred[2];
    __shared__ int s_tile, s_nvis, s_short;
    __shared__ int s_wc[2][TILE / 32];   // block_append scratch
    int apar = 0;
    __shared__ int64_t s_ct[2];

    constexpr bool QREG = MP <= 16;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t nt = a.ntiles;
    unsigned long long evaluated = 0;
    unsigned levels = 0, staged = 0, rounds = 0;

    // radius-first: a tile with a row short of k points inside its radius is searched once more at
    // twice the radius before it goes to the exact search (its rows are rewritten)
    bool redo = false;
    for (;;) {
        if (t == 0) {
            if (!redo) {
                const int idx = atomicAdd(a.work, 1);
                s_tile = a.tile_list ? (idx < *a.tile_count ? a.tile_list[idx] : 0x7fffffff) : idx;
            }
            s_short = 0;
        }
        __syncthreads();
        const int64_t qt = s_tile;
        if (qt >= nt) break;
        const int64_t p = qt * TILE + t;
        const bool valid = p < a.n;
        int64_t qlo = 0, qhi = a.n;   // the query's cloud
        if (a.cl.B > 1 && valid) {
            const int b = cloud_id(a.cl, p);
            qlo = a.cl.ptr[b];
            qhi = a.cl.ptr[b + 1];
        }
        if (t == 0) {   // candidate tiles that hold points of this tile's clouds
            s_ct[0] = 0;
            s_ct[1] = nt;
            if (a.cl.B > 1) {
                const int64_t p0 = qt * TILE, pl = min(a.n, p0 + TILE) - 1;
                s_ct[0] = a.cl.ptr[cloud_of(a.cl.ptr, a.cl.B, p0)] / TILE;
                s_ct[1] = (a.cl.ptr[cloud_of(a.cl.ptr, a.cl.B, pl) + 1] + TILE - 1) / TILE;
            }
        }
        float qr[QREG ? MP : 1];
        if constexpr (QREG) {
#pragma unroll
            for (int r = 0; r < MP; ++r) qr[r] = a.xs[p * MP + r];
        } else {
            for (int r = 0; r < MP; ++r) qs[r * TILE + t] = a.xs[p * MP + r];
        }
        for (int sl = 0; sl < L; ++sl) heap[sl * TILE + t] = KO::EMPTY;
        if (t == 0) s_nvis = 0;
        bool overflow = false;   // compact keys: more visits than vtab holds
        for (int r = t; r < MP; r += TILE) {
            sqlo[r] = a.tlo[qt * MP + r];
            sqhi[r] = a.thi[qt * MP + r];
        }
        KT maxkey = KO::EMPTY;
        int fill = 0;               // keys stored so far; the heap is ordered once it holds L
        uint32_t thr_blk = 0xffffffffu;
        const bool rmode = a.r2 != nullptr;
        KT sentinel = KO::EMPTY;
        if (rmode) {
            // radius-first: every slot starts as a sentinel at the query's radius bound, so only
            // candidates inside the radius ever enter and tiles are pruned from the start (appending
            // the first L keys and ordering them once instead was slower: the one-time heapify of a
            // lane holds up its warp)
            const float R2 = valid ? __fmul_ru(a.r2[p], redo ? 4.f * a.r2_scale : a.r2_scale) : 0.f;
            if constexpr (K32) sentinel = ((__float_as_uint(R2) >> 13) << 14) | 0x3fffu;   // slot 0x3fff: no candidate
            else sentinel = ((uint64_t)__float_as_uint(R2) << 32) | 0xffffffffu;
            for (int sl = 0; sl < L; ++sl) heap[sl * TILE + t] = sentinel;
            fill = L;
            maxkey = sentinel;
            const uint32_t wmax = __reduce_max_sync(0xffffffffu, valid ? KO::dist_hi(sentinel) : 0u);
            if (lane == 0) sred[warp] = wmax;
        }
        __syncthreads();
        if (rmode) thr_blk = max(sred[0], sred[1]);
        const int64_t ct_lo = s_ct[0], ct_hi = s_ct[1];
        __syncthreads();

        // Visit candidate tile ct for every query of this tile that may still gain from it.
        auto visit = [&](int64_t ct) {
            if (K32 && overflow) return;   // the tile goes to the full-key search anyway
            const float* clo = a.tlo + ct * MP;
            const float* chi = a.thi + ct * MP;
            bool need = valid;
            if (need && a.prune) {
                float lb;
                if constexpr (QREG) {
                    lb = point_box_lb<MP>(qr, clo, chi);
                } else {
                    float acc = 0.f;
                    for (int r = 0; r < MP; ++r) {
                        float qv = qs[r * TILE + t];
                        float g = fmaxf(fmaxf(clo[r] - qv, qv - chi[r]), 0.f);
                        acc = fmaf(g, g, acc);
                    }
                    lb = acc;
                }
                need = __float_as_uint(__fmul_rd(lb, a.lb_factor)) <= KO::dist_hi(maxkey);
            }
            if (!__syncthreads_or(need)) return;
            int vis = 0;   // compact keys: this visit's number (read by all threads between barriers)
            if constexpr (K32) {
                vis = s_nvis;
                if (vis >= VMAX) {
                    overflow = true;
                    return;
                }
            }
            staged += t == 0;
            {
                if constexpr (QREG) {   // transposed: the distance loop reads one coordinate of four candidates
                    const float4* src = (const float4*)(a.xs + (ct * TILE + t) * MP);
#pragma unroll
                    for (int r4 = 0; r4 < MP / 4; ++r4) {
                        const float4 v = src[r4];
                        cand[(4 * r4 + 0) * TILE + t] = v.x;
                        cand[(4 * r4 + 1) * TILE + t] = v.y;
                        cand[(4 * r4 + 2) * TILE + t] = v.z;
                        cand[(4 * r4 + 3) * TILE + t] = v.w;
                    }
                } else {
                    const float4* src = (const float4*)(a.xs + ct * TILE * MP);
                    float4* dst = (float4*)cand;
                    for (int i = t; i < TILE * MP / 4; i += TILE) dst[i] = src[i];
                }
            }
            __syncthreads();
            if constexpr (K32) {
                if (t == 0) {   // read again only after the barriers that end this visit
                    vtab[vis] = (int)ct;
                    s_nvis = vis + 1;
                }
            }
            if (need) {
                evaluated += TILE;
                const int64_t c0 = ct * TILE;
                // the whole candidate tile lies in this query's cloud and is not its own tile
                const bool whole = ct != qt && c0 >= qlo && c0 + TILE <= qhi;
                for (int cb = 0; cb < TILE; cb += IB) {
                    // distances of one batch, all computed before any key is stored: the shared-memory
                    // loads of the batch are then free to overlap (a store to the heap could alias them)
                    const uint32_t thr_hi = KO::dist_hi(maxkey);
                    float dist[IB];
                    if constexpr (QREG) {
                        // two candidates per packed FP32 instruction: d = x - q (the same square as
                        // q - x under round-to-nearest), then d0^2 + d1^2 + ... with the rounding
                        // sequence of the scalar form, so the distances are the same bits
                        float2 acc[IB / 2];
#pragma unroll
                        for (int r = 0; r < MR; ++r) {
                            const float2 nq = make_float2(-qr[r], -qr[r]);
#pragma unroll
                            for (int h = 0; h < IB / 4; ++h) {
                                const float4 v = *(const float4*)(cand + r * TILE + cb + 4 * h);
                                const float2 d0 = __fadd2_rn(make_float2(v.x, v.y), nq);
                                const float2 d1 = __fadd2_rn(make_float2(v.z, v.w), nq);
                                acc[2 * h] = r == 0 ? __fmul2_rn(d0, d0) : __ffma2_rn(d0, d0, acc[2 * h]);
                                acc[2 * h + 1] = r == 0 ? __fmul2_rn(d1, d1) : __ffma2_rn(d1, d1, acc[2 * h + 1]);
                            }
                        }
#pragma unroll
                        for (int j = 0; j < IB / 2; ++j) {
                            dist[2 * j] = acc[j].x;
                            dist[2 * j + 1] = acc[j].y;
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < IB; ++u) {
                            const int c = cb + u;
                            float acc = 0.f;
                            for (int r = 0; r < MP; ++r) {
                                float d = qs[r * TILE + t] - cand[c * MP + r];
                                acc = fmaf(d, d, acc);
                            }
                            dist[u] = acc;
                        }
                    }
                    unsigned pass = 0;
#pragma unroll
                    for (int u = 0; u < IB; ++u) pass |= (unsigned)(__float_as_uint(dist[u]) <= thr_hi) << u;
                    // keys under the heap maximum go in one by one (rare once the heap is full); a key
                    // at or above the current maximum cannot be among the L smallest
                    while (pass) {
                        const int u = __ffs(pass) - 1;
                        pass &= pass - 1;
                        const float du = Pick<IB>::get(dist, u);
                        const int c = cb + u;
                        const int64_t cp = c0 + c;
                        const KT key = KO::make(__float_as_uint(du), vis, c, cp);
                        if (!(key < maxkey) || !(whole || (cp != p && cp >= qlo && cp < qhi))) continue;
                        ++rounds;
                        if (fill < L) {   // first L keys: append, then order them in one pass
                            heap[fill * TILE + t] = key;
                            if (++fill == L) {
                                heapify(heap, t, L, levels);
                                maxkey = heap[t];
                            }
                            continue;
                        }
                        sift_down(heap, t, 0, L, key, levels);   // replace the root
                        maxkey = heap[t];
                    }
                }
            }
            // tile threshold = largest heap maximum among the tile's valid queries
            uint32_t mine = valid ? KO::dist_hi(maxkey) : 0u;
            uint32_t wmax = __reduce_max_sync(0xffffffffu, mine);
            if (lane == 0) sred[warp] = wmax;
            __syncthreads();
            thr_blk = max(sred[0], sred[1]);
            __syncthreads();
        };

        // seed: the tile itself and its neighbours in Morton order (not needed with a radius bound)
        for (int sidx = 0; sidx < (rmode ? 0 : a.nseed); ++sidx) {
            int64_t s2 = (sidx + 1) >> 1;
            int64_t ct = (sidx & 1) ? qt + s2 : qt - s2;
            if (ct >= ct_lo && ct < ct_hi) visit(ct);
        }
        // Every other tile whose box lower bound does not exceed the threshold, nearest first.
        // Two levels: super-tiles (64 consecutive tiles) first, nearest first; a super-tile whose
        // box lies beyond the threshold is skipped whole (its box contains every tile box, and the
        // bound is monotone in the box, rounding included), otherwise its 64 tiles are bounded,
        // gathered, sorted and visited.  slist[SCAP/2 ..) holds super-tiles, slist[0 .. SCAP/2) tiles
        // (all of slist when the super-tiles are too few to be worth bounding).
        auto sort_keys = [&](uint64_t* lst, int cnt) {   // ascending bitonic sort of lst[0..cnt)
            int P = 1;
            while (P < cnt) P <<= 1;
            for (int i = cnt + t; i < P; i += TILE) lst[i] = ~0ull;
            __syncthreads();
            for (int size = 2; size <= P; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int i = t; i < P / 2; i += TILE) {
                        int lo = 2 * i - (i & (stride - 1));
                        int hi = lo + stride;
                        bool up = (lo & size) == 0;
                        uint64_t x = lst[lo], y = lst[hi];
                        if ((x > y) == up) { lst[lo] = y; lst[hi] = x; }
                    }
                    __syncthreads();
                }
            }
        };
        // appends (bound, index) of the threads that keep theirs to lst at cnt
        auto append = [&](uint64_t* lst, int& cnt, bool keep, float lb, int64_t idx) {
            block_append<TILE / 32>(lst, cnt, keep, ((uint64_t)__float_as_uint(lb) << 32) | (uint32_t)idx, s_wc, apar);
        };
        uint64_t* sup = slist + SCAP / 2;
        const int64_t g_lo = ct_lo / TILE, g_hi = (ct_hi + TILE - 1) / TILE;
        // few super-tiles (a small cloud): their tiles are scanned directly, in index order
        const bool flat = g_hi - g_lo <= FLAT_SUPERS;
        const int tcap = flat ? SCAP - TILE : SCAP / 2 - TILE;   // tiles gathered before a sort
        for (int64_t g0 = g_lo; g0 < g_hi;) {
            int ng = 0;
            if (flat) {
                ng = (int)(g_hi - g_lo);
                g0 = g_hi;
            } else {
                for (; g0 < g_hi; g0 += TILE) {
                    const int64_t g = g0 + t;
                    bool keep = g < g_hi;
                    float lb = 0.f;
                    if (keep) {
                        float acc = 0.f;
                        for (int r = 0; r < MP; ++r) {
                            float gp = fmaxf(fmaxf(a.slo[g * MP + r] - sqhi[r], sqlo[r] - a.shi[g * MP + r]), 0.f);
                            acc = fmaf(gp, gp, acc);
                        }
                        lb = __fmul_rd(acc, a.lb_factor);
                        keep = !a.prune || __float_as_uint(lb) <= thr_blk;
                    }
                    append(sup, ng, keep, lb, g);
                    if (ng > SCAP / 2 - TILE) { g0 += TILE; break; }
                }
                sort_keys(sup, ng);
            }
            // tiles of the kept super-tiles, nearest super-tile first, gathered until the list holds
            // more than tcap, then sorted and visited nearest first
            int gi = 0;
            while (gi < ng) {
                int cnt = 0;
                for (; gi < ng; ++gi) {
                    int64_t g = g_lo + gi;
                    if (!flat) {
                        const uint64_t eg = sup[gi];
                        if (a.prune && (uint32_t)(eg >> 32) > thr_blk) {   // sorted: the rest lie farther
                            gi = ng;
                            break;
                        }
                        g = (int64_t)(uint32_t)eg;
                    }
                    const int64_t ct = g * TILE + t;
                    bool keep = ct >= ct_lo && ct < ct_hi;
                    if (keep && !rmode) {
                        const int64_t dct = ct - qt;
                        keep = (dct > (a.nseed >> 1) || dct < -((a.nseed - 1) >> 1));   // not a seed tile
                    }
                    float lb = 0.f;
                    if (keep) {
                        float acc = 0.f;
                        for (int r = 0; r < MP; ++r) {
                            float gp = fmaxf(fmaxf(a.tlo[ct * MP + r] - sqhi[r], sqlo[r] - a.thi[ct * MP + r]), 0.f);
                            acc = fmaf(gp, gp, acc);
                        }
                        lb = __fmul_rd(acc, a.lb_factor);
                        keep = !a.prune || __float_as_uint(lb) <= thr_blk;
                    }
                    append(slist, cnt, keep, lb, ct);
                    if (cnt > tcap) {
                        ++gi;
                        break;
                    }
                }
                sort_keys(slist, cnt);
                for (int si = 0; si < cnt; ++si) {
                    const uint64_t e = slist[si];
                    if (a.prune && (uint32_t)(e >> 32) > thr_blk) break;
                    visit((int64_t)(uint32_t)e);
                }
                __syncthreads();
            }
        }

        // ---------------- a5: order the kept candidates, rescore in FP64, certify
        bool row_ok = true;
        if (valid && !(K32 && overflow))
            row_ok = finalize_row<MP, TILE, KT>(a, heap, t, L, fill == L, p, qhi - qlo, levels, vtab, &s_short);
        if (K32 && overflow) row_ok = false;
        bool again = false;
        if (rmode || K32) {
            // a row with fewer than k points inside its radius, or uncertified: once more at twice the
            // radius when a row came up short, else redo the tile exactly
            const bool fail = __syncthreads_or(!row_ok);
            again = rmode && !redo && fail && s_short;
            if (again && t == 0) atomicAdd(&a.rep->knn_redo_tiles, 1ull);
            if (fail && !again && t == 0 && atomicExch(&a.fail_flag[qt], 1) == 0) {
                a.fail_list[atomicAdd(a.fail_count, 1)] = (int)qt;
                atomicAdd(&a.rep->knn_retry_tiles, 1ull);
            }
        } else if (!row_ok) {
            int slot = atomicAdd(a.fb_count, 1);
            a.fb_list[slot] = (int)a.perm[p];
            atomicAdd(&a.rep->knn_fallback_rows, 1ull);
        }
        __syncthreads();   // every thread has read s_short before thread 0 resets it
        redo = again;
    }
    unsigned long long ev = evaluated;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if (lane == 0 && ev) {
        atomicAdd(&a.rep->knn_candidates, ev);
        if (a.tile_list) atomicAdd(&a.rep->knn_retry_candidates, ev);   // the pass over handed-back tiles
    }
    unsigned long long lv = levels, st = staged, rd = rounds;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lv += __shfl_xor_sync(0xffffffffu, lv, o);
        st += __shfl_xor_sync(0xffffffffu, st, o);
        rd += __shfl_xor_sync(0xffffffffu, rd, o);
    }
    if (lane == 0) {
        atomicAdd(&a.rep->knn_heap_levels, lv);
        atomicAdd(&a.rep->knn_tiles_staged, st);
        atomicAdd(&a.rep->knn_insert_rounds, rd);
    }
}

// ------------------------------------------------------------------ 16-bit distance tiles on the tensor cores (a15)
// Query tiles of 128 points (two 64-point tiles, one TMEM lane and one thread per
// query) against candidate tiles, two 64-point tiles per visit: one chain of
// tcgen05.mma (kind::f16, M = 128, N = 128, K = m padded to 16; BF16 or FP16 operands,
// FP32 accumulation in tensor memory) gives the 128 x 128 dot products, read back
// with tcgen05.ld; distances are |q~|^2 + |x~|^2 - 2 q~.x~ with both operands
// recentred on the query tile's box centre before rounding, and at m <= 4 each
// coordinate carried as a hi + lo pair (see SPLIT below).  As in the FP32 search,
// candidate tiles are sorted by box distance (super-tiles first), visited nearest first,
// and skipped once their box distance passes the largest heap bound of the query tile,
// which tightens after every visit; each query keeps a 4-ary max-heap of its k + margin
// smallest keys, started full of sentinels at its radius bound when a radius is
// given (learned pruning) and at +inf otherwise.  Rows are finished by
// finalize_row_band.  With a radius, a query tile with a row short of k points is
// searched again at twice the radius by the same CTA; a tile still failing (short,
// uncertified, or past the visit table) goes to the exact FP32 search.
constexpr int T2 = 128;
constexpr int TC_ARITY = 4;   // the per-query heaps are 4-ary
constexpr int SCAP_TC = 512;  // sorted candidate-tile list: tiles in the first half, super-tiles in the second
constexpr float kHalfClamp = 30000.f;   // FP16 operands are clamped here (finite products)

// 16-bit operand types of the tiles: BF16 (8-bit significand) or FP16 (11-bit).
template <bool F16> struct Half16;
template <> struct Half16<false> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T from(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float to(T x) { return __bfloat162float(x); }
    static __device__ __forceinline__ uint16_t bits(T x) { return __bfloat16_as_ushort(x); }
    static constexpr float unit = 0.00390625f;     // 2^-8
    static constexpr float dabs = 0.f;
    static constexpr float clampv = 3.0e38f;
};
template <> struct Half16<true> {
    using T = __half;
    static __device__ __forceinline__ T from(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float to(T x) { return __half2float(x); }
    static __device__ __forceinline__ uint16_t bits(T x) { return __half_as_ushort(x); }
    static constexpr float unit = 0.00048828125f;  // 2^-11
    static constexpr float dabs = 1.0e-6f;         // >= sqrt(128) 2^-25: subnormal spacing over 128 coordinates
    static constexpr float clampv = kHalfClamp;
};

template <int MP, bool F16, bool K32 = false>
__global__ void __launch_bounds__(T2) knn_tc_kernel(TileArgs a)
{
    using KT = typename std::conditional<K32, uint32_t, uint64_t>::type;
    using BK = BandKey<KT>;
    constexpr int KP = MP < 16 ? 16 : MP;
    // m <= 4: every coordinate as a sum of two 16-bit numbers, hi + lo, and the four products
    // hi.hi, hi.lo, lo.hi, lo.lo in the K = 16 that one MMA step runs anyway (operands
    // A = [q_hi q_hi q_lo q_lo], B = [x_hi x_lo x_hi x_lo]): the dot product of hi + lo
    // with FP32 accumulation, so the representation error falls from u to u^2
    constexpr bool SPLIT = MP <= 4;
    using HT = Half16<F16>;
    using half_t = typename HT::T;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int C = a.cap;
    half_t* sa = (half_t*)smem;                                // [T2][KP] core-matrix layout
    half_t* sb = sa + T2 * KP;                                 // [2 TILE][KP]: two candidate tiles
    float* sqb = (float*)(sb + 2 * TILE * KP);                 // [2 TILE]
    uint64_t* slist = (uint64_t*)(sqb + 2 * TILE);             // [SCAP_TC]
    KT* buf = (KT*)(slist + SCAP_TC);                          // [C][T2] max-heaps
    __shared__ float sqlo[MP], sqhi[MP], scen[MP];
    __shared__ uint32_t sred[4];
    __shared__ int s_tile, s_fail, s_abort, s_short;
    __shared__ int s_wc[2][T2 / 32];   // block_append scratch
    int apar = 0;
    __shared__ int s_need[2][T2 / 32];   // per warp: bit h set if a query needs the visit's tile h
    int npar = 0;
    __shared__ int64_t s_ct[2];
    __shared__ float s_amax[4];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int vtab[K32 ? VMAX + 1 : 1];   // compact keys: the tile of every visit number
    __shared__ int s_nvis;

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t nt = a.ntiles;
    const int64_t nst = (nt + 1) / 2;
    const bool rmode = a.r2 != nullptr;
    Band bd;
    // split operands: |q' - (hi + lo)| <= u^2 |q'|, plus the FP32 rounding of q - c (2^-24 |q'|)
    bd.u = SPLIT ? HT::unit * HT::unit + 1.2e-7f : HT::unit;
    bd.dabs = HT::dabs;
    bd.rho_k = 2.f * (float)(KP + 4) * 5.9604645e-8f;
    unsigned long long evaluated = 0;
    unsigned levels = 0, staged = 0;
    if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * TILE);
    if (t == 0) { tc::mbar_init(&bar, 1); s_abort = 0; }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    uint32_t phase = 0;
    constexpr uint32_t idesc = tc::idesc_f16(T2, TILE, F16);        // one candidate tile per visit
    constexpr uint32_t idesc2 = tc::idesc_f16(T2, 2 * TILE, F16);   // two

    // radius-first: a query tile with a row short of k points inside its radius is searched once
    // more at twice the radius before it goes to the FP32 search (its rows are rewritten)
    bool redo = false;
    for (;;) {
        if (t == 0) {
            if (!redo) s_tile = atomicAdd(a.work, 1);
            s_fail = 0;
            s_short = 0;
            s_nvis = 0;
        }
        __syncthreads();
        const int64_t qs = s_tile;
        if (qs >= nst || s_abort) break;
        const int64_t p = qs * T2 + t;
        const bool valid = p < a.n;
        int64_t qlo = 0, qhi = a.n;   // the query's cloud
        if (a.cl.B > 1 && valid) {
            const int b = cloud_id(a.cl, p);
            qlo = a.cl.ptr[b];
            qhi = a.cl.ptr[b + 1];
        }
        if (t == 0) {   // candidate tiles that hold points of this query tile's clouds
            s_ct[0] = 0;
            s_ct[1] = nt;
            if (a.cl.B > 1) {
                const int64_t p0 = qs * T2, pl = min(a.n, p0 + T2) - 1;
                s_ct[0] = a.cl.ptr[cloud_of(a.cl.ptr, a.cl.B, p0)] / TILE;
                s_ct[1] = (a.cl.ptr[cloud_of(a.cl.ptr, a.cl.B, pl) + 1] + TILE - 1) / TILE;
            }
        }
        for (int r = t; r < MP; r += T2) {   // union box of tiles 2 qs and 2 qs + 1
            float lo = a.tlo[(2 * qs) * MP + r], hi = a.thi[(2 * qs) * MP + r];
            if (2 * qs + 1 < nt) {
                lo = fminf(lo, a.tlo[(2 * qs + 1) * MP + r]);
                hi = fmaxf(hi, a.thi[(2 * qs + 1) * MP + r]);
            }
            sqlo[r] = lo;
            sqhi[r] = hi;
            scen[r] = 0.5f * (lo + hi);
        }
        __syncthreads();
        // query operand: 16-bit (q - centre), |q~|^2
        float qr[MP];
        float sqa = 0.f;
#pragma unroll
        for (int r = 0; r < MP; ++r) qr[r] = a.xs[p * MP + r];
        if constexpr (SPLIT) {
            uint16_t vh[8], vl[8];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float x = r < MP && valid ? fminf(fmaxf(qr[r < MP ? r : 0] - scen[r < MP ? r : 0], -HT::clampv),
                                                        HT::clampv)
                                                : 0.f;
                const half_t h = HT::from(x);
                const float hb = HT::to(h);
                const half_t l = HT::from(x - hb);   // x - hb is exact in FP32
                const float xv = hb + HT::to(l);    // exact in FP32
                sqa = fmaf(xv, xv, sqa);
                vh[r] = HT::bits(h);
                vh[4 + r] = HT::bits(h);
                vl[r] = HT::bits(l);
                vl[4 + r] = HT::bits(l);
            }
            *(uint4*)((char*)sa + tc::operand_offset(t, 0, KP)) = tc::pack8(vh);
            *(uint4*)((char*)sa + tc::operand_offset(t, 8, KP)) = tc::pack8(vl);
        } else {
#pragma unroll
            for (int j = 0; j < KP / 8; ++j) {
                uint16_t v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int r = 8 * j + e;
                    const float x = r < MP && valid ? fminf(fmaxf(qr[r] - scen[r], -HT::clampv), HT::clampv) : 0.f;
                    const half_t h = HT::from(x);
                    v[e] = HT::bits(h);
                    const float xb = HT::to(h);
                    sqa = fmaf(xb, xb, sqa);
                }
                *(uint4*)((char*)sa + tc::operand_offset(t, 8 * j, KP)) = tc::pack8(v);
            }
        }
        const float qn = sqrtf(sqa);
        const float R2 = rmode && valid ? __fmul_ru(a.r2[p], redo ? 4.f * a.r2_scale : a.r2_scale) : INFINITY;
        const KT sentinel = rmode ? BK::sentinel(__float_as_uint(R2)) : BK::EMPTY;
        for (int sl = 0; sl < C; ++sl) buf[sl * T2 + t] = sentinel;
        KT heapmax = sentinel;
        {
            const uint32_t wr = __reduce_max_sync(0xffffffffu, valid ? BK::hi_bits(sentinel) : 0u);
            const uint32_t wa = __reduce_max_sync(0xffffffffu, valid ? __float_as_uint(qn) : 0u);
            if (lane == 0) { sred[warp] = wr; s_amax[warp] = __uint_as_float(wa); }
        }
        tc::fence_async_smem();
        __syncthreads();
        const int64_t ct_lo = s_ct[0], ct_hi = s_ct[1];
        uint32_t thr_blk = max(max(sred[0], sred[1]), max(sred[2], sred[3]));
        const float amax = fmaxf(fmaxf(s_amax[0], s_amax[1]), fmaxf(s_amax[2], s_amax[3]));
        // FP16 range: a query tile whose own extent is not small against the clamp goes to FP32
        const bool far = F16 && amax > 0.25f * kHalfClamp;

        // Visit candidate tiles cta and ctb (ctb < 0: one tile) for every query that may still gain
        // from them: stage their 16-bit operands (one candidate per thread), one MMA chain
        // (N = 64 per tile) into tensor memory, then each query folds the distances of the tiles it
        // needs into its heap; finally the tile bound tightens.  Two tiles per visit halve the
        // barriers and MMA round trips per candidate.  Returns false once a bounded wait ran out or
        // the visit table is full.
        auto visit = [&](int64_t cta, int64_t ctb) -> bool {
            auto needs = [&](int64_t ct) {
                if (!valid || ct < 0) return false;
                float acc = 0.f;
#pragma unroll
                for (int r = 0; r < MP; ++r) {
                    const float g = fmaxf(fmaxf(a.tlo[ct * MP + r] - qr[r], qr[r] - a.thi[ct * MP + r]), 0.f);
                    acc = fmaf(g, g, acc);
                }
                return __float_as_uint(__fmul_rd(acc, a.lb_factor)) <= BK::hi_bits(heapmax);
            };
            bool need0 = needs(cta), need1 = needs(ctb);
            {   // one barrier for both tiles; two halves, as a warp can be one visit ahead
                const unsigned b0 = __ballot_sync(0xffffffffu, need0), b1 = __ballot_sync(0xffffffffu, need1);
                if (lane == 0) s_need[npar][warp] = (b0 ? 1 : 0) | (b1 ? 2 : 0);
            }
            __syncthreads();
            const int nw = s_need[npar][0] | s_need[npar][1] | s_need[npar][2] | s_need[npar][3];
            npar ^= 1;
            const bool any0 = nw & 1, any1 = nw & 2;
            if (!any0 && !any1) return true;
            // the tiles to stage, in order: slot h holds tile ct_h (needed by some query)
            const int64_t ct0 = any0 ? cta : ctb;
            const int64_t ct1 = any0 && any1 ? ctb : -1;
            if (!any0) { need0 = need1; need1 = false; }
            const int ntl = ct1 >= 0 ? 2 : 1;
            int vis = 0;   // compact keys: this visit's first number (the same in every thread)
            if constexpr (K32) {
                vis = s_nvis;
                if (vis + ntl > VMAX) {   // more visits than the table holds: the FP32 search redoes the tile
                    if (t == 0) s_fail = 1;
                    __syncthreads();   // every thread sees the flag before the loops test it
                    return false;
                }
            }
            staged += t == 0 ? ntl : 0;
            if (t < TILE * ntl) {   // candidate operand: row t = candidate t % 64 of slot t / 64
                const int64_t cp = (t < TILE ? ct0 : ct1) * TILE + (t & (TILE - 1));
                float xv[MP];
                if constexpr (MP % 4 == 0) {
#pragma unroll
                    for (int r4 = 0; r4 < MP / 4; ++r4) {
                        const float4 v4 = *(const float4*)(a.xs + cp * MP + 4 * r4);
                        xv[4 * r4] = v4.x; xv[4 * r4 + 1] = v4.y; xv[4 * r4 + 2] = v4.z; xv[4 * r4 + 3] = v4.w;
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < MP; ++r) xv[r] = a.xs[cp * MP + r];
                }
                float sq = 0.f;
                if constexpr (SPLIT) {
                    uint16_t v[8];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const float x = r < MP ? fminf(fmaxf(xv[r < MP ? r : 0] - scen[r < MP ? r : 0], -HT::clampv),
                                                       HT::clampv)
                                               : 0.f;
                        const half_t h = HT::from(x);
                        const float hb = HT::to(h);
                        const half_t l = HT::from(x - hb);
                        const float xw = hb + HT::to(l);
                        sq = fmaf(xw, xw, sq);
                        v[r] = HT::bits(h);
                        v[4 + r] = HT::bits(l);
                    }
                    const uint4 w = tc::pack8(v);
                    *(uint4*)((char*)sb + tc::operand_offset(t, 0, KP)) = w;
                    *(uint4*)((char*)sb + tc::operand_offset(t, 8, KP)) = w;
                } else {
#pragma unroll
                    for (int j = 0; j < KP / 8; ++j) {
                        uint16_t v[8];
#pragma unroll
                        for (int e2 = 0; e2 < 8; ++e2) {
                            const int r = 8 * j + e2;
                            const float x = r < MP ? fminf(fmaxf(xv[r < MP ? r : 0] - scen[r < MP ? r : 0], -HT::clampv),
                                                           HT::clampv)
                                                   : 0.f;
                            const half_t h = HT::from(x);
                            v[e2] = HT::bits(h);
                            const float xb = HT::to(h);
                            sq = fmaf(xb, xb, sq);
                        }
                        *(uint4*)((char*)sb + tc::operand_offset(t, 8 * j, KP)) = tc::pack8(v);
                    }
                }
                sqb[t] = sq;
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if constexpr (K32) {
                if (t == 0) {   // read again only after the barriers that end this visit
                    vtab[vis] = (int)ct0;
                    if (ntl == 2) vtab[vis + 1] = (int)ct1;
                    s_nvis = vis + ntl;
                }
            }
            if (t == 0) {
                constexpr uint32_t sbo = (uint32_t)(KP / 8) * 128;
                const uint32_t id = ntl == 2 ? idesc2 : idesc;
#pragma unroll
                for (int s = 0; s < KP / 16; ++s) {
                    const uint64_t ad = tc::smem_desc(tc::smem_addr(sa) + s * 256, 128, sbo);
                    const uint64_t bd2 = tc::smem_desc(tc::smem_addr(sb) + s * 256, 128, sbo);
                    tc::mma_bf16(tb, ad, bd2, id, s > 0 ? 1u : 0u);
                }
                tc::mma_commit(&bar);
            }
            // a warp reads tensor memory only if the wait ended in time for all its lanes (the load
            // is warp-wide); the end-of-visit barrier tells every thread whether one did not
            const bool done = __all_sync(0xffffffffu, tc::mbar_wait(&bar, phase));
            phase ^= 1u;
            tc::fence_after_sync();
            if (!done) need0 = need1 = false;
            evaluated += (need0 ? TILE : 0) + (need1 ? TILE : 0);
            const uint32_t hb = BK::hi_bits(heapmax);
            float hmf = hb == 0xffffffffu ? INFINITY : __uint_as_float(hb);
#pragma unroll 1
            for (int ch = 0; ch < (done ? 2 * ntl : 0); ++ch) {
                const int h = ch >> 1;
                float v[32];
                tc::tmem_ld32(tb + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32), v);
                if (!(h == 0 ? need0 : need1)) continue;
                const int64_t cth = h == 0 ? ct0 : ct1;
                // distances of the 32 columns (registers only), and the mask of those under the bound
                uint32_t msk = 0;
                const float4* sq4 = (const float4*)(sqb + ch * 32);
#pragma unroll
                for (int i4 = 0; i4 < 8; ++i4) {
                    const float4 q4 = sq4[i4];
                    v[4 * i4 + 0] = fmaf(-2.f, v[4 * i4 + 0], sqa + q4.x);
                    v[4 * i4 + 1] = fmaf(-2.f, v[4 * i4 + 1], sqa + q4.y);
                    v[4 * i4 + 2] = fmaf(-2.f, v[4 * i4 + 2], sqa + q4.z);
                    v[4 * i4 + 3] = fmaf(-2.f, v[4 * i4 + 3], sqa + q4.w);
                }
#pragma unroll
                for (int i = 0; i < 32; ++i) msk |= (v[i] <= hmf ? 1u : 0u) << i;
                while (msk) {   // the full key test and the heap update
                    const int i = __ffs(msk) - 1;
                    msk &= msk - 1u;
                    const float d = Pick<32>::get(v, i);
                    const int lt = (ch & 1) * 32 + i;   // the candidate's lane in its tile
                    const int64_t cp = cth * TILE + lt;
                    const KT key = BK::make(__float_as_uint(fmaxf(d, 0.f)), vis + h, lt, (uint32_t)cp);
                    if (key < heapmax && cp != p && cp >= qlo && cp < qhi) {
                        sift_down_d<T2, TC_ARITY>(buf, t, 0, C, key, levels);
                        heapmax = buf[t];
                    }
                }
                const uint32_t h2 = BK::hi_bits(heapmax);
                hmf = h2 == 0xffffffffu ? INFINITY : __uint_as_float(h2);
            }
            tc::fence_before_sync();
            // tile threshold = largest heap bound among the tile's valid queries
            const uint32_t wmax = __reduce_max_sync(0xffffffffu, valid ? BK::hi_bits(heapmax) : 0u);
            if (lane == 0) sred[warp] = wmax;
            if (__syncthreads_or(!done)) {   // a bounded wait ran out: record it and stop
                if (t == 0) { report_error(a.rep, VB_ERR_TIMEOUT); s_abort = 1; }
                __syncthreads();   // every thread sees the flag before the loops test it
                return false;
            }
            thr_blk = max(max(sred[0], sred[1]), max(sred[2], sred[3]));
            return true;
        };

        // seed tiles (without a radius bound): the query tile's own two tiles and their
        // neighbours in Morton order, so the heaps fill with near points before any pruning
        const int64_t sw = (a.nseed - 1) / 2;   // tiles on each side
        const int64_t s_lo = rmode || far ? 0 : max(ct_lo, 2 * qs - sw);
        const int64_t s_hi = rmode || far ? 0 : min(ct_hi, 2 * qs + 2 + sw);
        for (int64_t ct = s_lo; ct < s_hi && !s_abort && !s_fail; ct += 2)
            if (!visit(ct, ct + 1 < s_hi ? ct + 1 : -1)) break;
        // every other tile whose box lower bound does not exceed the tile bound, nearest first.
        // Two levels, as in the FP32 search: super-tiles (64 consecutive tiles) by their boxes,
        // nearest first, skipped whole beyond the threshold (a super-tile's box holds its tiles'
        // boxes); the tiles of the kept ones, two super-tiles per pass of the block, are bounded,
        // gathered, sorted and visited.  Few super-tiles (a small cloud): tiles scanned directly.
        // slist[0, SCAP_TC/2) holds tiles, slist[SCAP_TC/2, SCAP_TC) super-tiles.
        auto sort_keys = [&](uint64_t* lst, int cnt) {   // ascending bitonic sort of lst[0..cnt)
            int P = 1;
            while (P < cnt) P <<= 1;
            for (int i = cnt + t; i < P; i += T2) lst[i] = ~0ull;
            __syncthreads();
            for (int size = 2; size <= P; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int i = t; i < P / 2; i += T2) {
                        const int lo = 2 * i - (i & (stride - 1));
                        const int hi = lo + stride;
                        const bool up = (lo & size) == 0;
                        const uint64_t x = lst[lo], y = lst[hi];
                        if ((x > y) == up) { lst[lo] = y; lst[hi] = x; }
                    }
                    __syncthreads();
                }
            }
        };
        auto tile_lb = [&](int64_t ct, const float* lo, const float* hi) {
            float acc = 0.f;
            for (int r = 0; r < MP; ++r) {
                const float g = fmaxf(fmaxf(lo[ct * MP + r] - sqhi[r], sqlo[r] - hi[ct * MP + r]), 0.f);
                acc = fmaf(g, g, acc);
            }
            return __fmul_rd(acc, a.lb_factor);
        };
        // visits the sorted tiles slist[0..cnt) while their bound passes the threshold
        auto visit_sorted = [&](int cnt) {
            for (int si = 0; si < cnt;) {
                const uint64_t e = slist[si];
                if ((uint32_t)(e >> 32) > thr_blk) break;   // sorted: the rest lie farther
                // the next tile too, when its bound passes the threshold as it stands (a threshold
                // that tightens during this visit only makes the pair a little wider than needed)
                const bool pair = si + 1 < cnt && (uint32_t)(slist[si + 1] >> 32) <= thr_blk;
                if (!visit((int64_t)(uint32_t)e, pair ? (int64_t)(uint32_t)slist[si + 1] : -1)) break;
                si += pair ? 2 : 1;
            }
            __syncthreads();
        };
        uint64_t* sup = slist + SCAP_TC / 2;
        const int64_t g_lo = ct_lo / TILE, g_hi = (ct_hi + TILE - 1) / TILE;
        if (g_hi - g_lo <= FLAT_SUPERS) {
            for (int64_t c0 = ct_lo; c0 < ct_hi && !far && !s_abort && !s_fail;) {
                int cnt = 0;
                for (; c0 < ct_hi; c0 += T2) {
                    const int64_t ct = c0 + t;
                    bool keep = ct < ct_hi && (ct < s_lo || ct >= s_hi);
                    float lb = 0.f;
                    if (keep) {
                        lb = tile_lb(ct, a.tlo, a.thi);
                        keep = __float_as_uint(lb) <= thr_blk;
                    }
                    block_append<T2 / 32>(slist, cnt, keep, ((uint64_t)__float_as_uint(lb) << 32) | (uint32_t)ct, s_wc, apar);
                    if (cnt > SCAP_TC - T2) { c0 += T2; break; }
                }
                sort_keys(slist, cnt);
                visit_sorted(cnt);
            }
        } else {
            for (int64_t g0 = g_lo; g0 < g_hi && !far && !s_abort && !s_fail;) {
                int ng = 0;
                for (; g0 < g_hi; g0 += T2) {
                    const int64_t g = g0 + t;
                    bool keep = g < g_hi;
                    float lb = 0.f;
                    if (keep) {
                        lb = tile_lb(g, a.slo, a.shi);
                        keep = __float_as_uint(lb) <= thr_blk;
                    }
                    block_append<T2 / 32>(sup, ng, keep, ((uint64_t)__float_as_uint(lb) << 32) | (uint32_t)g, s_wc, apar);
                    if (ng > SCAP_TC / 2 - T2) { g0 += T2; break; }
                }
                sort_keys(sup, ng);
                for (int gi = 0; gi < ng && !s_abort && !s_fail;) {
                    int cnt = 0;
                    for (; gi < ng; gi += T2 / TILE) {
                        if ((uint32_t)(sup[gi] >> 32) > thr_blk) {   // sorted: the rest lie farther
                            gi = ng;
                            break;
                        }
                        const int sg = gi + t / TILE;   // this thread's super-tile and tile in it
                        int64_t ct = -1;
                        bool keep = false;
                        float lb = 0.f;
                        if (sg < ng && (uint32_t)(sup[sg] >> 32) <= thr_blk) {
                            ct = (int64_t)(uint32_t)sup[sg] * TILE + (t & (TILE - 1));
                            keep = ct >= ct_lo && ct < ct_hi && (ct < s_lo || ct >= s_hi);
                            if (keep) {
                                lb = tile_lb(ct, a.tlo, a.thi);
                                keep = __float_as_uint(lb) <= thr_blk;
                            }
                        }
                        block_append<T2 / 32>(slist, cnt, keep, ((uint64_t)__float_as_uint(lb) << 32) | (uint32_t)ct, s_wc,
                                              apar);
                        if (cnt > SCAP_TC / 2 - T2) { gi += T2 / TILE; break; }
                    }
                    sort_keys(slist, cnt);
                    visit_sorted(cnt);
                }
            }
        }
        if (s_abort) break;

        bool ok = !far && !s_fail;   // s_fail here: the visit table overflowed (compact keys)
        if (valid && ok)
            ok = finalize_row_band<MP, T2, KT, TC_ARITY>(a, buf, t, C, p, qhi - qlo, levels, bd, qn, vtab, &s_short);
        if (valid && !ok) s_fail = 1;
        __syncthreads();
        const bool again = rmode && !redo && s_fail && s_short;
        if (!again && t == 0 && s_fail) {
            for (int h = 0; h < 2; ++h) {
                const int64_t qt = 2 * qs + h;
                if (qt < nt && atomicExch(&a.fail_flag[qt], 1) == 0) {
                    a.fail_list[atomicAdd(a.fail_count, 1)] = (int)qt;
                    atomicAdd(&a.rep->knn_retry_tiles, 1ull);
                }
            }
        }
        if (again && t == 0) atomicAdd(&a.rep->knn_redo_tiles, 1ull);
        __syncthreads();   // every thread has read the flags before thread 0 resets them
        redo = again;
    }
    unsigned long long ev = evaluated, lv = levels, st = staged;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
        lv += __shfl_xor_sync(0xffffffffu, lv, o);
        st += __shfl_xor_sync(0xffffffffu, st, o);
    }
    if (lane == 0) {
        atomicAdd(&a.rep->knn_candidates, ev);
        atomicAdd(&a.rep->knn_heap_levels, lv);
        atomicAdd(&a.rep->knn_tiles_staged, st);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tb, 2 * TILE);
}

// ------------------------------------------------------------------ pipelined 16-bit distance tiles (a3, a15)
// The warp-specialised form of the 16-bit search, for inputs wide enough that the
// contraction is real work.  Each 64-point tile is converted once per call into a
// tile block: its 16-bit operand (coordinates minus the cloud's mid-range centre,
// K = m padded to 16, clamped like the staged kernel's) laid out exactly as the
// no-swizzle K-major core-matrix image the MMA reads, followed by the tile's FP32
// norms |x~|^2.  A query tile (128 points: two 64-point tiles, one TMEM lane each)
// then runs as a pipeline of three roles:
//   warp 4 (producer)  walks the candidate tiles in order of their box lower bound and
//                      stages each block with one bulk copy (TMA) into a ring of S slots;
//   warp 5 (MMA)       issues K/16 tcgen05.mma (M = 128, N = 64, FP32 accumulation) per
//                      tile into one of four 64-column tensor-memory buffers and copies the
//                      tile's norms beside it;
//   warps 0-3          one query per thread: read the 64 dot products, form
//                      |q~|^2 + |x~|^2 - 2 q~.x~ and fold them into the query's max-heap.
// The producer skips tiles whose bound exceeds the largest heap bound of the query tile
// (published by the epilogue warps after every tile; a stale value is only larger) and
// stops at the first counting-sort bin beyond it: the list is ordered by the top bits of
// the bound, a monotone key, so the stop is exact.  Rows finish as in the staged kernel
// (finalize_row_band); a row that is not certified sends its tiles to the FP32 search.
// Every wait is bounded in time (an expired wait records VB_ERR_TIMEOUT and stops the CTA).
constexpr int TCP_BUF = 4;         // tensor-memory accumulator buffers of 64 columns
constexpr int TCP_META = 16;       // tile ids in flight (>= slots + buffers + 1)
constexpr int TCP_THREADS = 192;   // warps 0-3 epilogue, 4 producer, 5 MMA
constexpr int TCP_BINS = 4096;     // counting-sort bins: FP32 bits of the bound >> 19 (6 % wide)
constexpr int TCP_SHIFT = 19;

__global__ void tcp_range_init_kernel(int* crange)
{
    const int r = threadIdx.x;
    if (r < 128) {
        crange[r] = 0x7fffffff;
        crange[128 + r] = (int)0x80000000;
    }
}

// Per-coordinate min and max over the sorted coordinates of the n real points.
__global__ void tcp_range_kernel(const float* __restrict__ xs, int64_t n, int m, int mp, int* crange)
{
    const int r = threadIdx.x;
    if (r >= m) return;
    int lo = 0x7fffffff, hi = (int)0x80000000;
    const int64_t p0 = (int64_t)blockIdx.x * 64, p1 = min(n, p0 + 64);
    for (int64_t p = p0; p < p1; ++p) {
        const int v = f2ord(xs[p * mp + r]);
        lo = min(lo, v);
        hi = max(hi, v);
    }
    atomicMin(&crange[r], lo);
    atomicMax(&crange[128 + r], hi);
}

// Tile blocks: 16-bit (x - c) of every padded sorted point in the core-matrix image of
// its tile, and |x~|^2 summed in FP32 from the rounded values (padding rows are zero).
template <bool F16>
__global__ void tcp_block_kernel(const float* __restrict__ xs, int64_t n, int64_t npad, int m, int mp, int kp,
                                 const int* __restrict__ crange, unsigned char* blk)
{
    using HT = Half16<F16>;
    using half_t = typename HT::T;
    __shared__ float cen[128];
    for (int r = threadIdx.x; r < 128; r += blockDim.x)
        cen[r] = r < m ? 0.5f * (ord2f(crange[r]) + ord2f(crange[128 + r])) : 0.f;
    __syncthreads();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= npad) return;
    unsigned char* tb = blk + (p / TILE) * tcp_blk_bytes(kp);
    const int row = (int)(p % TILE);
    float sq = 0.f;
    for (int j = 0; j < kp / 8; ++j) {
        uint16_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int r = 8 * j + e;
            const float x = r < m && p < n ? fminf(fmaxf(xs[p * mp + r] - cen[r], -HT::clampv), HT::clampv) : 0.f;
            const half_t h = HT::from(x);
            v[e] = HT::bits(h);
            const float xb = HT::to(h);
            sq = fmaf(xb, xb, sq);
        }
        *(uint4*)(tb + tc::operand_offset(row, 8 * j, kp)) = tc::pack8(v);
    }
    ((float*)(tb + tcp_img_bytes(kp)))[row] = sq;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier, giving up when another role has stopped the
// CTA or after about four seconds (then the CTA is stopped and VB_ERR_TIMEOUT recorded).
__device__ __noinline__ bool tcp_wait(uint64_t* bar, uint32_t parity, volatile int* stop, DevReport* rep)
{
    const uint32_t ad = tc::smem_addr(bar);
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(ad), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 31) == 0) {
            if (*stop) return false;
            const uint64_t now = global_ns();
            if (it == 0) t0 = now;
            else if (now - t0 > 4000000000ull) {
                *stop = 1;
                report_error(rep, VB_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

template <int MP, bool F16>
__global__ void __launch_bounds__(TCP_THREADS, 1) knn_tcp_kernel(TileArgs a)
{
    using HT = Half16<F16>;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int KP = a.kp, S = a.stages, L = a.cap;
    const uint32_t IMG = (uint32_t)tcp_img_bytes(KP), BLK = (uint32_t)tcp_blk_bytes(KP);
    unsigned char* sa = smem;                                // query operand: two tile images
    unsigned char* slots = smem + 2 * IMG;                   // S staged tile blocks
    uint64_t* heap = (uint64_t*)(slots + (size_t)S * BLK);   // [L][T2] max-heaps
    uint32_t* hist = (uint32_t*)heap;                        // [2][TCP_BINS] while the tile list is built
    __shared__ __align__(8) uint64_t full[4], empty[4], tfull[TCP_BUF], tempty[TCP_BUF], qbar, dbar;
    __shared__ __align__(16) float txn[TCP_BUF][TILE];
    __shared__ volatile int meta[TCP_META];
    __shared__ volatile uint32_t sred[4];
    __shared__ uint64_t pkeys[32];
    __shared__ volatile int s_stop;
    __shared__ int s_tile, s_cnt;
    __shared__ int64_t s_ct[2];
    __shared__ float sqlo[MP], sqhi[MP];
    __shared__ float s_rq;
    __shared__ float sblo[4][MP], sbhi[4][MP], sbr[4];   // the four 32-query groups: boxes, ball radii
    __shared__ uint4 psub[32];
    __shared__ uint32_t tmem_base;

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t nt = a.ntiles;
    const int64_t nst = (nt + 1) / 2;
    unsigned long long evaluated = 0;
    unsigned levels = 0, staged = 0;
    uint32_t pseq = 0, mseq = 0, eseq = 0, qcount = 0;   // role-local sequence numbers
    if (warp == 5) tc::tmem_alloc(&tmem_base, TCP_BUF * TILE);
    if (t == 0) {
        for (int i = 0; i < S; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < TCP_BUF; ++i) {
            tc::mbar_init(&tfull[i], 2);    // the MMA completion and the MMA warp's own arrival
            tc::mbar_init(&tempty[i], 4);   // one arrival per epilogue warp
        }
        tc::mbar_init(&qbar, 1);
        tc::mbar_init(&dbar, 1);
        s_stop = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    constexpr uint32_t idesc = tc::idesc_f16(T2, TILE, F16);
    uint32_t* lbw = a.lbw + (int64_t)blockIdx.x * nt;
    uint64_t* tl = a.tlist + (int64_t)blockIdx.x * nt;

    for (;;) {
        if (t == 0) s_tile = atomicAdd(a.work, 1);
        __syncthreads();
        const int64_t qs = s_tile;
        if (qs >= nst || s_stop) break;
        const bool epi = warp < 4;
        const int64_t p = qs * T2 + (epi ? t : 0);
        const bool valid = epi && p < a.n;
        int64_t qlo = 0, qhi = a.n;   // the query's cloud
        if (a.cl.B > 1 && valid) {
            const int b = cloud_id(a.cl, p);
            qlo = a.cl.ptr[b];
            qhi = a.cl.ptr[b + 1];
        }
        if (t == 0) {   // candidate tiles that hold points of this query tile's clouds
            s_ct[0] = 0;
            s_ct[1] = nt;
            if (a.cl.B > 1) {
                const int64_t p0 = qs * T2, pl = min(a.n, p0 + T2) - 1;
                s_ct[0] = a.cl.ptr[cloud_of(a.cl.ptr, a.cl.B, p0)] / TILE;
                s_ct[1] = (a.cl.ptr[cloud_of(a.cl.ptr, a.cl.B, pl) + 1] + TILE - 1) / TILE;
            }
        }
        for (int r = t; r < MP; r += TCP_THREADS) {   // union box of tiles 2 qs and 2 qs + 1
            float lo = a.tlo[(2 * qs) * MP + r], hi = a.thi[(2 * qs) * MP + r];
            if (2 * qs + 1 < nt) {
                lo = fminf(lo, a.tlo[(2 * qs + 1) * MP + r]);
                hi = fmaxf(hi, a.thi[(2 * qs + 1) * MP + r]);
            }
            sqlo[r] = lo;
            sqhi[r] = hi;
        }
        if (warp == 5) {
            // ball of the query tile about its box centre: the two tiles' balls moved to that centre
            // (triangle inequality), FP32 sums rounded up
            float rq = 0.f;
            for (int h = 0; h < 2; ++h) {
                const int64_t tq = 2 * qs + h;
                if (tq >= nt) break;
                float s2 = 0.f;
                for (int r = lane; r < a.m; r += 32) {
                    float lo = a.tlo[(2 * qs) * MP + r], hi = a.thi[(2 * qs) * MP + r];
                    if (2 * qs + 1 < nt) {
                        lo = fminf(lo, a.tlo[(2 * qs + 1) * MP + r]);
                        hi = fmaxf(hi, a.thi[(2 * qs + 1) * MP + r]);
                    }
                    const float d = 0.5f * (a.tlo[tq * MP + r] + a.thi[tq * MP + r]) - 0.5f * (lo + hi);
                    s2 = fmaf(d, d, s2);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                rq = fmaxf(rq, __fadd_ru(__fmul_ru(sqrtf(s2), 1.00002f), a.trad[tq]));
            }
            if (lane == 0) s_rq = __fmul_ru(rq, 1.00002f);
        }
        for (int i = t; i < 2 * TCP_BINS; i += TCP_THREADS) hist[i] = 0;
        // query norm (from the tile block) and the heap's starting key
        float sqa = 0.f;
        if (valid) sqa = ((const float*)(a.blk + (p / TILE) * (size_t)BLK + IMG))[p % TILE];
        const float R2 = a.r2 && valid ? __fmul_ru(a.r2[p], a.r2_scale) : INFINITY;
        const uint64_t sentinel = a.r2 ? (((uint64_t)__float_as_uint(R2) << 32) | 0xffffffffu) : ~0ull;
        if (epi) {
            const uint32_t wr = __reduce_max_sync(0xffffffffu, valid ? (uint32_t)(sentinel >> 32) : 0u);
            if (lane == 0) sred[warp] = wr;
            // this warp's 32 queries: their box, and the ball about its centre (FP32 sums rounded up)
            const bool any = __any_sync(0xffffffffu, valid);
            float s2 = 0.f;
            for (int r = 0; r < MP; ++r) {
                const float v = valid && r < a.m ? a.xs[p * MP + r] : 0.f;
                float l = valid ? v : INFINITY, h = valid ? v : -INFINITY;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    l = fminf(l, __shfl_xor_sync(0xffffffffu, l, o));
                    h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
                }
                if (!any) { l = 0.f; h = 0.f; }
                if (lane == 0) { sblo[warp][r] = l; sbhi[warp][r] = h; }
                const float d = valid ? v - 0.5f * (l + h) : 0.f;
                s2 = fmaf(d, d, s2);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s2 = fmaxf(s2, __shfl_xor_sync(0xffffffffu, s2, o));
            if (lane == 0) sbr[warp] = any ? __fmul_ru(sqrtf(s2), 1.00002f) : -1.f;   // -1: no query here
        }
        __syncthreads();
        const int64_t ct_lo = s_ct[0], ct_hi = s_ct[1];
        // candidate tiles by box lower bound: bounds, bin counts, scan, scatter
        const float rq = s_rq;
        for (int64_t ct = ct_lo + t; ct < ct_hi; ct += TCP_THREADS) {
            // two lower bounds on the distance of any candidate in tile ct to any query of this
            // tile: box to box, and ball to ball (centres apart minus both radii), which is the
            // tighter one for wide inputs on a low-dimensional set; the same two for each group of
            // 32 queries (one per selection warp), which the producer tests against that warp's
            // own largest heap bound.  One pass over the coordinates serves all five.
            float acc = 0.f, cd = 0.f, ab[4] = {0.f, 0.f, 0.f, 0.f}, cb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int r = 0; r < a.m; ++r) {
                const float lo = a.tlo[ct * MP + r], hi = a.thi[ct * MP + r];
                const float cc = 0.5f * (lo + hi);
                const float g = fmaxf(fmaxf(lo - sqhi[r], sqlo[r] - hi), 0.f);
                acc = fmaf(g, g, acc);
                const float dc = cc - 0.5f * (sqlo[r] + sqhi[r]);
                cd = fmaf(dc, dc, cd);
#pragma unroll
                for (int w4 = 0; w4 < 4; ++w4) {
                    const float bl = sblo[w4][r], bh = sbhi[w4][r];
                    const float gw = fmaxf(fmaxf(lo - bh, bl - hi), 0.f);
                    ab[w4] = fmaf(gw, gw, ab[w4]);
                    const float dw = cc - 0.5f * (bl + bh);
                    cb[w4] = fmaf(dw, dw, cb[w4]);
                }
            }
            const float rct = a.trad[ct];
            const float gap = __fsub_rd(__fmul_rd(sqrtf(cd), 0.99998f), __fadd_ru(rq, rct));
            if (gap > 0.f) acc = fmaxf(acc, __fmul_rd(__fmul_rd(gap, gap), 0.99998f));
            const uint32_t lbb = __float_as_uint(__fmul_rd(acc, a.lb_factor));
            lbw[ct - ct_lo] = lbb;
            uint32_t sub[4];
#pragma unroll
            for (int w4 = 0; w4 < 4; ++w4) {
                float abw = ab[w4];
                const float gw = __fsub_rd(__fmul_rd(sqrtf(cb[w4]), 0.99998f), __fadd_ru(sbr[w4], rct));
                if (gw > 0.f) abw = fmaxf(abw, __fmul_rd(__fmul_rd(gw, gw), 0.99998f));
                sub[w4] = sbr[w4] < 0.f ? 0x7f800000u : __float_as_uint(__fmul_rd(abw, a.lb_factor));   // empty group
            }
            a.lbs[(int64_t)blockIdx.x * nt + (ct - ct_lo)] = make_uint4(sub[0], sub[1], sub[2], sub[3]);
            atomicAdd(&hist[min(lbb >> TCP_SHIFT, (uint32_t)TCP_BINS - 1)], 1u);
        }
        __syncthreads();
        if (warp == 0) {
            constexpr int PER = TCP_BINS / 32;
            uint32_t sum = 0;
            for (int i = 0; i < PER; ++i) sum += hist[lane * PER + i];
            uint32_t inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            uint32_t run = inc - sum;
            for (int i = 0; i < PER; ++i) {
                const uint32_t c = hist[lane * PER + i];
                hist[TCP_BINS + lane * PER + i] = run;
                run += c;
            }
            if (lane == 31) s_cnt = (int)inc;
        }
        __syncthreads();
        for (int64_t ct = ct_lo + t; ct < ct_hi; ct += TCP_THREADS) {
            const uint32_t lbb = lbw[ct - ct_lo];
            const uint32_t pos = atomicAdd(&hist[TCP_BINS + min(lbb >> TCP_SHIFT, (uint32_t)TCP_BINS - 1)], 1u);
            tl[pos] = ((uint64_t)lbb << 32) | (uint32_t)ct;
        }
        __syncthreads();   // the list is complete and the bins are free for the heaps

        if (warp == 4) {
            // ---------------- producer: query operand, then the candidate tiles in bound order
            // (the list is read 32 keys at a time by the whole warp; lane 0 decides and issues)
            if (lane == 0) {
                tc::mbar_arrive_tx(&qbar, 2 * IMG);
                tc::bulk_g2s(sa, a.blk + (2 * qs) * (size_t)BLK, IMG, &qbar);
                tc::bulk_g2s(sa + IMG, a.blk + (2 * qs + 1) * (size_t)BLK, IMG, &qbar);
            }
            const int cnt = s_cnt;
            int go = 1;
            for (int base = 0; go; base += 32) {
                const uint64_t kl = base + lane < cnt ? tl[base + lane] : ~0ull;
                pkeys[lane] = kl;
                if (kl != ~0ull) psub[lane] = a.lbs[(int64_t)blockIdx.x * nt + ((int64_t)(uint32_t)kl - ct_lo)];
                __syncwarp();
                if (lane == 0) {
                    for (int j = 0; j < 32 && go; ++j) {
                        const uint64_t key = pkeys[j];
                        int ct = -1;   // -1: end of this query tile
                        if (key != ~0ull) {
                            const uint32_t lbb = (uint32_t)(key >> 32);
                            const uint32_t thr = max(max(sred[0], sred[1]), max(sred[2], sred[3]));
                            if (lbb > thr && (lbb >> TCP_SHIFT) <= (thr >> TCP_SHIFT)) continue;   // skip this tile only
                            if (lbb <= thr) {                                        // else: this bin and beyond
                                const uint4 sb = psub[j];   // skip unless some group of 32 queries may gain
                                if (sb.x > sred[0] && sb.y > sred[1] && sb.z > sred[2] && sb.w > sred[3]) continue;
                                ct = (int)(uint32_t)key;
                            }
                        }
                        const int sl = (int)(pseq % (uint32_t)S);
                        if (!tcp_wait(&empty[sl], ((pseq / (uint32_t)S) & 1u) ^ 1u, &s_stop, a.rep)) {
                            go = 0;
                            break;
                        }
                        meta[pseq % TCP_META] = ct;
                        if (ct >= 0) {
                            tc::mbar_arrive_tx(&full[sl], BLK);
                            tc::bulk_g2s(slots + (size_t)sl * BLK, a.blk + (size_t)ct * BLK, BLK, &full[sl]);
                            ++staged;
                        } else {
                            tc::mbar_arrive(&full[sl]);
                            go = 0;
                        }
                        ++pseq;
                    }
                }
                go = __shfl_sync(0xffffffffu, go, 0);
                __syncwarp();
            }
        } else if (warp == 5) {
            // ---------------- MMA issue
            if (lane == 0) {
                bool go = tcp_wait(&qbar, qcount & 1u, &s_stop, a.rep);
                while (go) {
                    const int sl = (int)(mseq % (uint32_t)S), b = (int)(mseq % TCP_BUF);
                    if (!tcp_wait(&full[sl], (mseq / (uint32_t)S) & 1u, &s_stop, a.rep)) break;
                    const int ct = meta[mseq % TCP_META];
                    if (!tcp_wait(&tempty[b], ((mseq / TCP_BUF) & 1u) ^ 1u, &s_stop, a.rep)) break;
                    if (ct >= 0) {
                        const float4* sx = (const float4*)(slots + (size_t)sl * BLK + IMG);
                        float4* dx = (float4*)txn[b];
#pragma unroll
                        for (int i = 0; i < TILE / 4; ++i) dx[i] = sx[i];
                        tc::fence_after_sync();
                        const uint32_t sbo = (uint32_t)(KP / 8) * 128;
                        const uint32_t a0 = tc::smem_addr(sa), b0 = tc::smem_addr(slots + (size_t)sl * BLK);
                        for (int ks = 0; ks < KP / 16; ++ks)
                            tc::mma_bf16(tb + (uint32_t)(b * TILE), tc::smem_desc(a0 + ks * 256, 128, sbo),
                                         tc::smem_desc(b0 + ks * 256, 128, sbo), idesc, ks > 0 ? 1u : 0u);
                        tc::mma_commit(&empty[sl]);
                        tc::mma_commit(&tfull[b]);
                    } else {
                        tc::mbar_arrive(&empty[sl]);
                        tc::mbar_arrive(&tfull[b]);
                    }
                    tc::mbar_arrive(&tfull[b]);   // orders the norms and the tile id before the epilogue
                    ++mseq;
                    if (ct < 0) break;
                }
            }
            __syncwarp();
        } else {
            // ---------------- epilogue: one query per thread
            for (int sl = 0; sl < L; ++sl) heap[sl * T2 + t] = sentinel;
            uint64_t heapmax = sentinel;
            uint32_t hb = (uint32_t)(heapmax >> 32);
            float hmf = hb == 0xffffffffu ? INFINITY : __uint_as_float(hb);
            const uint32_t lane_addr = tb + ((uint32_t)(warp * 32) << 16);
            for (;;) {
                const int b = (int)(eseq % TCP_BUF);
                int ok = 1;
                if (lane == 0) ok = tcp_wait(&tfull[b], (eseq / TCP_BUF) & 1u, &s_stop, a.rep) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
                __syncwarp();
                const int ct = meta[eseq % TCP_META];
                tc::fence_after_sync();
                float v[TILE];
                if (ct >= 0) {
                    tc::tmem_ld64(lane_addr + (uint32_t)(b * TILE), v);
                    const float4* x4 = (const float4*)txn[b];
#pragma unroll
                    for (int i4 = 0; i4 < TILE / 4; ++i4) {
                        const float4 q4 = x4[i4];
                        v[4 * i4 + 0] = fmaf(-2.f, v[4 * i4 + 0], sqa + q4.x);
                        v[4 * i4 + 1] = fmaf(-2.f, v[4 * i4 + 1], sqa + q4.y);
                        v[4 * i4 + 2] = fmaf(-2.f, v[4 * i4 + 2], sqa + q4.z);
                        v[4 * i4 + 3] = fmaf(-2.f, v[4 * i4 + 3], sqa + q4.w);
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&tempty[b]);
                ++eseq;
                if (ct < 0) break;
                if (valid) {
                    evaluated += TILE;
#pragma unroll
                    for (int ch = 0; ch < TILE / 32; ++ch) {
                        // mask of the columns under the bound: four independent 8-bit chains
                        uint32_t mq[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                        for (int i = 0; i < 32; ++i) mq[i & 3] |= (v[ch * 32 + i] <= hmf ? 1u : 0u) << i;
                        uint32_t msk = (mq[0] | mq[1]) | (mq[2] | mq[3]);
                        while (msk) {   // the full key test and the heap update
                            const int i = __ffs(msk) - 1;
                            msk &= msk - 1u;
                            float d = 0.f;
#pragma unroll
                            for (int j = 0; j < 32; ++j) d = j == i ? v[ch * 32 + j] : d;
                            const int64_t cp = (int64_t)ct * TILE + ch * 32 + i;
                            const uint64_t key = ((uint64_t)__float_as_uint(fmaxf(d, 0.f)) << 32) | (uint32_t)cp;
                            if (key < heapmax && cp != p && cp >= qlo && cp < qhi) {
                                sift_down<T2>(heap, t, 0, L, key, levels);
                                heapmax = heap[t];
                            }
                        }
                        hb = (uint32_t)(heapmax >> 32);
                        hmf = hb == 0xffffffffu ? INFINITY : __uint_as_float(hb);
                    }
                }
                const uint32_t wmax = __reduce_max_sync(0xffffffffu, valid ? (uint32_t)(heapmax >> 32) : 0u);
                if (lane == 0) sred[warp] = wmax;
            }
            // the rows are finished by tcp_finish_kernel, which keeps the FP64 rescoring off
            // this kernel's tensor pipeline: hand the heaps over in the same [L][128] layout
            uint64_t* hd = a.hdump + (size_t)qs * L * T2;
            for (int sl = 0; sl < L; ++sl) hd[(size_t)sl * T2 + t] = heap[sl * T2 + t];
        }
        ++qcount;
        __syncthreads();
        if (s_stop) break;
    }
    // every MMA of this CTA has completed, and no bulk copy is still landing, before exit
    if (warp == 5 && lane == 0) {
        tc::mma_commit(&dbar);
        tc::mbar_wait(&dbar, 0, 1u << 22);
    }
    if (warp == 4 && lane == 0 && s_stop) {
        for (uint32_t q = pseq > (uint32_t)S ? pseq - (uint32_t)S : 0u; q < pseq; ++q)
            tc::mbar_wait(&full[q % (uint32_t)S], (q / (uint32_t)S) & 1u, 1u << 22);
        tc::mbar_wait(&qbar, (qcount - 1u) & 1u, 1u << 22);
    }
    unsigned long long ev = evaluated, lv = levels, st = staged;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
        lv += __shfl_xor_sync(0xffffffffu, lv, o);
        st += __shfl_xor_sync(0xffffffffu, st, o);
    }
    if (lane == 0) {
        if (ev) atomicAdd(&a.rep->knn_candidates, ev);
        if (lv) atomicAdd(&a.rep->knn_heap_levels, lv);
        if (st) atomicAdd(&a.rep->knn_tiles_staged, st);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 5) tc::tmem_dealloc(tb, TCP_BUF * TILE);
}

// Row finish of the pipelined search, one CTA of 128 threads per query tile, on the heaps
// the search left in a.hdump ([L][128] per query tile, max-heaps): heap sort, FP64
// rescoring against the 16-bit error band and the certificate (finalize_row_band); a
// query tile with a row that is not certified goes to the FP32 search.  Run as its own
// kernel so that the narrow FP64 pipe works at full occupancy instead of stalling the
// tensor-core pipeline of one CTA per SM.
template <int MP, bool F16>
__global__ void __launch_bounds__(T2) tcp_finish_kernel(TileArgs a)
{
    using HT = Half16<F16>;
    const int64_t qs = blockIdx.x;
    const int t = threadIdx.x;
    const int L = a.cap;
    const int64_t p = qs * T2 + t;
    const bool valid = p < a.n;
    Band bd;
    bd.u = HT::unit;
    bd.dabs = HT::dabs;
    bd.rho_k = 2.f * (float)(a.kp + 4) * 5.9604645e-8f;
    unsigned levels = 0;
    bool ok = true;
    if (valid) {
        int64_t qlo = 0, qhi = a.n;
        if (a.cl.B > 1) {
            const int b = cloud_id(a.cl, p);
            qlo = a.cl.ptr[b];
            qhi = a.cl.ptr[b + 1];
        }
        const size_t BLK = tcp_blk_bytes(a.kp);
        const float sqa = ((const float*)(a.blk + (p / TILE) * BLK + tcp_img_bytes(a.kp)))[p % TILE];
        const float qn = sqrtf(sqa);
        ok = !(F16 && qn > 0.25f * kHalfClamp);
        if (ok) ok = finalize_row_band<MP, T2>(a, a.hdump + (size_t)qs * L * T2, t, L, p, qhi - qlo, levels, bd, qn);
    }
    if (__syncthreads_or(!ok) && t == 0) {
        for (int h = 0; h < 2; ++h) {
            const int64_t qt = 2 * qs + h;
            if (qt < a.ntiles && atomicExch(&a.fail_flag[qt], 1) == 0) {
                a.fail_list[atomicAdd(a.fail_count, 1)] = (int)qt;
                atomicAdd(&a.rep->knn_retry_tiles, 1ull);
            }
        }
    }
    unsigned long long lv = levels;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lv += __shfl_xor_sync(0xffffffffu, lv, o);
    if ((t & 31) == 0 && lv) atomicAdd(&a.rep->knn_heap_levels, lv);
}

// R2[pos] = (inflate * radius[perm[pos]])^2 for the sorted points (caller-provided radii).
__global__ void radius_gather_kernel(const float* __restrict__ radius, const uint32_t* __restrict__ perm, int64_t n,
                                     float inflate, float* r2)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float r = radius[perm[i]] * inflate;
    r2[i] = __fmul_ru(r, r);
}

// ------------------------------------------------------------------ exact FP64 fallback rows
// One block per listed row: radix selection of the k-th smallest canonical
// FP64 distance (8 passes over the 8 bytes of its bit pattern), then the
// strictly smaller ones plus the lowest-index ties, ranked by (d2, index).
__global__ void __launch_bounds__(FB_THREADS) knn_fallback_kernel(const float* __restrict__ x, int64_t n, int m,
                                                                   int k, const int* __restrict__ fb_list,
                                                                   const int* __restrict__ fb_count, Clouds cl,
                                                                   int32_t* nbr, double* nbr_d2)
{
    __shared__ uint32_t hist[256];
    __shared__ uint64_t skey[256];
    __shared__ uint32_t sidx[256];
    __shared__ uint64_t s_prefix, s_mask;
    __shared__ uint32_t s_need, s_less, s_wtot[FB_THREADS / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int cnt = *fb_count;
    for (int f = blockIdx.x; f < cnt; f += gridDim.x) {
        const int64_t q = fb_list[f];
        const float* xq = x + q * m;
        const int cb = cloud_id(cl, q);
        const int64_t lo = cloud_lo(cl, cb), hi = cloud_hi(cl, cb, n);   // candidates: the query's cloud
        if (t == 0) { s_prefix = 0; s_mask = 0; s_need = (uint32_t)k; s_less = 0; }
        __syncthreads();
        for (int byte = 7; byte >= 0; --byte) {
            hist[t] = 0;
            __syncthreads();
            const uint64_t prefix = s_prefix, mask = s_mask;
            for (int64_t j = lo + t; j < hi; j += FB_THREADS) {
                if (j == q) continue;
                uint64_t key = (uint64_t)__double_as_longlong(canon_d2(xq, x + j * m, m));
                if ((key & mask) == prefix) atomicAdd(&hist[(key >> (8 * byte)) & 255u], 1u);
            }
            __syncthreads();
            if (t == 0) {
                uint32_t need = s_need, cum = 0;
                int dgt = 0;
                for (; dgt < 256; ++dgt) {
                    if (cum + hist[dgt] >= need) break;
                    cum += hist[dgt];
                }
                s_prefix = prefix | ((uint64_t)dgt << (8 * byte));
                s_mask = mask | (0xffull << (8 * byte));
                s_need = need - cum;
            }
            __syncthreads();
        }
        const uint64_t T = s_prefix;
        const uint32_t need = s_need;          // how many ties at T are taken
        const uint32_t nless = (uint32_t)k - need;
        for (int64_t j = lo + t; j < hi; j += FB_THREADS) {
            if (j == q) continue;
            uint64_t key = (uint64_t)__double_as_longlong(canon_d2(xq, x + j * m, m));
            if (key < T) {
                uint32_t s = atomicAdd(&s_less, 1u);
                skey[s] = key;
                sidx[s] = (uint32_t)j;
            }
        }
        __syncthreads();
        uint32_t taken = 0;
        for (int64_t b0 = lo; b0 < hi && taken < need; b0 += FB_THREADS) {
            int64_t j = b0 + t;
            bool fl = j < hi && j != q &&
                      (uint64_t)__double_as_longlong(canon_d2(xq, x + j * m, m)) == T;
            unsigned bal = __ballot_sync(0xffffffffu, fl);
            if (lane == 0) s_wtot[w] = __popc(bal);
            __syncthreads();
            uint32_t off = __popc(bal & ((1u << lane) - 1u));
            uint32_t tot = 0;
            for (int ww = 0; ww < FB_THREADS / 32; ++ww) {
                if (ww < w) off += s_wtot[ww];
                tot += s_wtot[ww];
            }
            if (fl && taken + off < need) {
                skey[nless + taken + off] = T;
                sidx[nless + taken + off] = (uint32_t)j;
            }
            taken += tot;
            __syncthreads();
        }
        __syncthreads();
        for (int s = t; s < k; s += FB_THREADS) {
            uint64_t ks = skey[s];
            uint32_t is = sidx[s];
            int rank = 0;
            for (int u = 0; u < k; ++u) rank += (skey[u] < ks) || (skey[u] == ks && sidx[u] < is);
            nbr[q * k + rank] = (int32_t)is;
            nbr_d2[q * k + rank] = __longlong_as_double((long long)ks);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host orchestration
template <int MP, bool K32 = false>
static size_t tile_smem(int L)
{
    const size_t kb = K32 ? 4 : 8;
    return (size_t)L * TILE * kb + SCAP * 8 + TILE * MP * 4 + (MP > 16 ? TILE * MP * 4 : 0) +
           (K32 ? VMAX * sizeof(int) : 0);
}

// The staged search keeps compact 32-bit heap keys at m <= 16 (visits of a query tile stay
// far below the visit table there), full 64-bit keys for wider inputs, and at m <= 4 also
// when the caller asks for full keys (their diagnostic output is the FP32 tile distance
// itself rather than the lower edge of its bucket).
template <int MP> constexpr bool tc_compact() { return MP <= 16; }
template <int MP, bool K32 = tc_compact<MP>()>
static size_t tc_smem(int C)
{
    constexpr int KP = MP < 16 ? 16 : MP;
    return (size_t)T2 * KP * 2 + 2 * TILE * KP * 2 + 2 * TILE * 4 + SCAP_TC * 8 + (size_t)C * T2 * (K32 ? 4 : 8);
}

template <int MP, bool F16, bool K32 = tc_compact<MP>()>
static vb_status launch_tc(TileArgs a, cudaStream_t s)
{
    const size_t sm = tc_smem<MP, K32>(a.cap);
    if (sm > 220 * 1024) return VB_ERR_UNSUPPORTED;   // k + margin too large for 128 heaps with these operands
    static bool attr_set[16] = {};
    static int sms[16] = {}, smem_sm[16] = {}, static_smem[16] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr_set[dev & 15]) {
        if (cudaFuncSetAttribute(knn_tc_kernel<MP, F16, K32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(220 * 1024)) != cudaSuccess ||
            cudaFuncSetAttribute(knn_tc_kernel<MP, F16, K32>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return VB_ERR_CUDA;
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, knn_tc_kernel<MP, F16, K32>) != cudaSuccess) return VB_ERR_CUDA;
        static_smem[dev & 15] = (int)fa.sharedSizeBytes;
        if (cudaDeviceGetAttribute(&sms[dev & 15], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm[dev & 15], cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
                cudaSuccess)
            return VB_ERR_CUDA;
        attr_set[dev & 15] = true;
    }
    // CTAs per SM from shared memory (1 KB reserved per CTA), at most 4 (128 TMEM columns each, 512 per SM);
    // extra CTAs of this persistent grid would only wait for a free slot
    const int per_cta = (int)sm + static_smem[dev & 15] + 1024;
    const int per_sm = std::max(1, std::min(4, smem_sm[dev & 15] / per_cta));
    const int64_t nst = (a.ntiles + 1) / 2;
    const int64_t grid = std::min<int64_t>(nst, (int64_t)per_sm * sms[dev & 15]);
    knn_tc_kernel<MP, F16, K32><<<(unsigned)grid, T2, sm, s>>>(a);
    return last_launch();
}

// Pipelined 16-bit search: ring slots as many (2..4) as shared memory allows next to the
// query operand and the heaps; VB_ERR_UNSUPPORTED when not even two fit.
template <int MP, bool F16>
static vb_status launch_tcp(TileArgs a, cudaStream_t s)
{
    const size_t img = tcp_img_bytes(a.kp), blk = tcp_blk_bytes(a.kp);
    const size_t heap = std::max((size_t)a.cap * T2 * sizeof(uint64_t), (size_t)2 * TCP_BINS * sizeof(uint32_t));
    static bool attr_set[16] = {};
    static int sms[16] = {}, smem_sm[16] = {}, static_smem[16] = {}, optin[16] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const int dv = dev & 15;
    if (!attr_set[dv]) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, knn_tcp_kernel<MP, F16>) != cudaSuccess) return VB_ERR_CUDA;
        static_smem[dv] = (int)fa.sharedSizeBytes;
        if (cudaDeviceGetAttribute(&sms[dv], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm[dv], cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin[dv], cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return VB_ERR_CUDA;
        if (cudaFuncSetAttribute(knn_tcp_kernel<MP, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin[dv] - static_smem[dv]) != cudaSuccess ||
            cudaFuncSetAttribute(knn_tcp_kernel<MP, F16>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return VB_ERR_CUDA;
        attr_set[dv] = true;
    }
    int S = 0;
    for (int c = 4; c >= 2 && !S; --c)
        if (2 * img + c * blk + heap + (size_t)static_smem[dv] <= (size_t)optin[dv]) S = c;
    if (!S) return VB_ERR_UNSUPPORTED;
    a.stages = S;
    const size_t sm = 2 * img + S * blk + heap;
    // CTAs per SM: shared memory (1 KB reserved per CTA), at most 2 (256 TMEM columns each)
    const int per_cta = (int)sm + static_smem[dv] + 1024;
    const int per_sm = std::max(1, std::min(2, smem_sm[dv] / per_cta));
    const int64_t nst = (a.ntiles + 1) / 2;
    const int64_t grid = std::min<int64_t>({nst, (int64_t)per_sm * sms[dv], (int64_t)TCP_MAX_CTAS});
    knn_tcp_kernel<MP, F16><<<(unsigned)grid, TCP_THREADS, sm, s>>>(a);
    tcp_finish_kernel<MP, F16><<<(unsigned)nst, T2, 0, s>>>(a);
    return last_launch();
}

template <int MP, int MR = MP, bool K32 = false>
static vb_status launch_tile_m(const TileArgs& a, cudaStream_t s)
{
    size_t sm = tile_smem<MP, K32>(a.L);
    static bool attr_set[16] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr_set[dev & 15]) {
        if (cudaFuncSetAttribute(knn_tile_kernel<MP, MR, K32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem<MP, K32>(256)) != cudaSuccess ||
            cudaFuncSetAttribute(knn_tile_kernel<MP, MR, K32>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return VB_ERR_CUDA;
        attr_set[dev & 15] = true;
    }
    // one CTA per tile for a full pass; a pass over a list of handed-back tiles (usually few or
    // none) takes them from the same counter with one resident wave of CTAs, so that an empty
    // list costs one short launch rather than a CTA per tile of the cloud
    const int64_t grid = a.tile_list ? std::min<int64_t>(a.ntiles, 152 * 10) : a.ntiles;
    knn_tile_kernel<MP, MR, K32><<<(unsigned)grid, TILE, sm, s>>>(a);
    return last_launch();
}

// m <= 4: the distance loop reads only the m real coordinates of the 4-wide rows.
template <int MP, bool K32 = false>
static vb_status launch_tile(const TileArgs& a, cudaStream_t s)
{
    if constexpr (MP == 4) {
        switch (a.m) {
            case 1: return launch_tile_m<4, 1, K32>(a, s);
            case 2: return launch_tile_m<4, 2, K32>(a, s);
            case 3: return launch_tile_m<4, 3, K32>(a, s);
            default: return launch_tile_m<4, 4, K32>(a, s);
        }
    }
    return launch_tile_m<MP, MP, K32>(a, s);
}

// a1: the spatial order of the points (Morton key on the coordinates, or on the projections on
// the leading principal axes when m > 4; then the cloud id above it in a batch), the sorted
// coordinates in FP32 and FP64, and the boxes of 64-point tiles and 64-tile super-tiles.
// perm (sorted position -> original index) is w.val[*cur] afterwards.
static vb_status order_points(Ctx* ctx, const float* x, int64_t n, int32_t m, const KnnWs& w, Clouds cl,
                              const uint32_t** perm_out, int curve = VB_CURVE_AUTO)
{
    cudaStream_t s = ctx->stream;
    const int mp = pad_dim(m), md = morton_dims(m), bits = morton_bits(md);
    const int64_t ntiles = (n + TILE - 1) / TILE, npad = (ntiles + (ntiles & 1)) * TILE;
    const int nblk = (int)((n + RADIX_ITEMS - 1) / RADIX_ITEMS);
    bbox_init_kernel<<<1, 32, 0, s>>>(w.bbox, w.fb_count);
    const unsigned bbox_grid = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 4);
    if (m <= 4) {
        bbox_kernel<<<bbox_grid, 256, 0, s>>>(x, n, m, md, w.bbox, ctx->rep);
        // the Hilbert curve at 2 <= m <= 4 unless the caller asks for the Morton curve
        const int hilbert = curve == VB_CURVE_AUTO && md >= 2 ? 1 : 0;
        morton_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, m, md, bits, w.bbox, w.key[0], w.val[0],
                                                                  hilbert);
    } else {
        // finite check of the input, then the key on the leading principal axes
        bbox_kernel<<<bbox_grid, 256, 0, s>>>(x, n, m, 0, w.bbox, ctx->rep);
        const int64_t stride = std::max<int64_t>(1, n / PCA_SAMPLE), rows = (n + stride - 1) / stride;
        const int64_t mlen = 1 + m + (int64_t)m * m;
        pca_zero_kernel<<<(unsigned)((mlen + 255) / 256), 256, 0, s>>>(w.pcs, mlen);
        pca_moments_kernel<<<PCA_BLOCKS, 256, 0, s>>>(x, n, m, stride, rows, w.pcs);
        pca_axes_kernel<<<1, 256, 0, s>>>(w.pcs, m, w.pcc);
        pca_project_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, m, w.pcs + mlen, w.proj);
        bbox_kernel<<<bbox_grid, 256, 0, s>>>(w.proj, n, PCA_D, PCA_D, w.bbox, ctx->rep);
        morton_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.proj, n, PCA_D, PCA_D, bits, w.bbox, w.key[0],
                                                                  w.val[0], 0);
        ctx->launches += 5;   // moments zeroed, moments, axes, projection, box of the projections
    }
    int cur = 0;
    for (int shift = 0; shift < 32; shift += 8) {
        radix_hist_kernel<<<nblk, RADIX_T, 0, s>>>(w.key[cur], n, shift, w.hist, nblk);
        ctx->launches += 2 + scan_u32(s, w.hist, (int64_t)256 * nblk, w.hsum);
        radix_scatter_kernel<<<nblk, RADIX_T, 0, s>>>(w.key[cur], w.val[cur], w.key[cur ^ 1], w.val[cur ^ 1], n,
                                                      shift, w.hist, nblk);
        cur ^= 1;
    }
    if (cl.B > 1) {
        // stable passes on the cloud id: (cloud, Morton) order, so cloud b occupies the sorted
        // positions [ptr[b], ptr[b + 1]), the same range as its points in the input
        cloud_key_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.val[cur], n, cl, w.key[cur]);
        ctx->launches += 1;
        for (int shift = 0; (int64_t)(cl.B - 1) >> shift; shift += 8) {
            radix_hist_kernel<<<nblk, RADIX_T, 0, s>>>(w.key[cur], n, shift, w.hist, nblk);
            ctx->launches += 2 + scan_u32(s, w.hist, (int64_t)256 * nblk, w.hsum);
            radix_scatter_kernel<<<nblk, RADIX_T, 0, s>>>(w.key[cur], w.val[cur], w.key[cur ^ 1], w.val[cur ^ 1], n,
                                                          shift, w.hist, nblk);
            cur ^= 1;
        }
    }
    const uint32_t* perm = w.val[cur];
    gather_kernel<<<(unsigned)((npad * mp + 255) / 256), 256, 0, s>>>(x, perm, n, npad, m, mp, w.xs, w.xs64);
    tile_box_kernel<<<(unsigned)((ntiles * 32 + 255) / 256), 256, 0, s>>>(w.xs, n, ntiles, m, mp, w.tlo, w.thi);
    super_box_kernel<<<(unsigned)(((ntiles + TILE - 1) / TILE * 32 + 255) / 256), 256, 0, s>>>(w.tlo, w.thi, ntiles, mp,
                                                                                              w.slo, w.shi);
    *perm_out = perm;
    return last_launch();
}

size_t order_ws_bytes(int64_t n, int32_t m)
{
    vb_knn_params p = {};
    p.k = 1;
    p.precision = VB_PREC_FP32;
    p.prune = VB_PRUNE_EXACT;
    Carve c(nullptr);
    return knn_plan(c, n, m, &p, nullptr);
}

vb_status order_run(Ctx* ctx, const float* x, int64_t n, int32_t m, void* ws, size_t ws_bytes, PointOrder* o)
{
    if (!x || !o || n < 1 || n >= INT32_MAX || m < 1 || m > 128) return VB_ERR_ARG;
    vb_knn_params p = {};
    p.k = 1;
    p.precision = VB_PREC_FP32;
    p.prune = VB_PRUNE_EXACT;
    KnnWs w;
    Carve c(ws);
    if (!ws || ws_bytes < knn_plan(c, n, m, &p, &w)) return VB_ERR_WORKSPACE;
    const uint32_t* perm = nullptr;
    vb_status st = order_points(ctx, x, n, m, w, Clouds(), &perm);
    if (st != VB_OK) return st;
    o->xs64 = w.xs64;
    o->tlo = w.tlo;
    o->thi = w.thi;
    o->perm = perm;
    o->mp = pad_dim(m);
    o->ntiles = (n + TILE - 1) / TILE;
    return VB_OK;
}

vb_status knn_run(Ctx* ctx, const float* x, int64_t n, int32_t m, const vb_knn_params* p, int32_t* nbr,
                  double* nbr_d2, void* ws, size_t ws_bytes, Clouds cl)
{
    if (cl.B < 1 || (cl.B > 1 && !cl.ptr)) return VB_ERR_ARG;
    if (!x || !nbr || !nbr_d2 || !p || n < 2 || n >= INT32_MAX || m < 1 || m > 128) return VB_ERR_ARG;
    if (p->k < 1 || (int64_t)p->k > n - 1 || p->margin < 0 || p->k + p->margin > 256) return VB_ERR_ARG;
    if (p->precision < VB_PREC_FP32 || p->precision > VB_PREC_FP16) return VB_ERR_UNSUPPORTED;
    if (p->precision != VB_PREC_FP32 && p->prune == VB_PRUNE_NONE) return VB_ERR_UNSUPPORTED;
    if (p->prune == VB_PRUNE_LEARNED && !p->radius && !p->mlp) return VB_ERR_ARG;
    if (p->prune < VB_PRUNE_NONE || p->prune > VB_PRUNE_LEARNED) return VB_ERR_ARG;
    KnnWs w;
    Carve c(ws);
    size_t need = knn_plan(c, n, m, p, &w);
    if (!ws || ws_bytes < need) return VB_ERR_WORKSPACE;
    cudaStream_t s = ctx->stream;
    const int mp = pad_dim(m);
    const int64_t ntiles = (n + TILE - 1) / TILE, npad = (ntiles + (ntiles & 1)) * TILE;

    mark(ctx, VB_STAGE_KNN_ORDER, 0);
    const uint32_t* perm = nullptr;
    vb_status st = order_points(ctx, x, n, m, w, cl, &perm, p->curve);
    if (st != VB_OK) return st;
    mark(ctx, VB_STAGE_KNN_ORDER, 1);

    TileArgs a = {};
    a.xs = w.xs; a.xs64 = w.xs64; a.hdump = w.hdump; a.tlo = w.tlo; a.thi = w.thi; a.slo = w.slo; a.shi = w.shi; a.perm = perm; a.n = n; a.ntiles = ntiles;
    a.m = m; a.k = p->k; a.L = p->k + p->margin; a.prune = p->prune != VB_PRUNE_NONE;
    // enough neighbouring tiles to fill every heap, unless the caller (the autotuner) chose
    a.nseed = p->seed_tiles > 0 ? 1 + 2 * p->seed_tiles : 1 + 2 * (int)((a.L + TILE) / TILE);
    a.lb_factor = 1.0f - 4.0f * (float)(m + 2) * 5.9604645e-8f;
    a.band = 1.0f + 4.0f * (float)(m + 2) * 5.9604645e-8f;
    a.cert_factor = 1.0 - 2.0 * (double)(m + 2) * 5.9604644775390625e-8;
    a.nbr = nbr; a.nbr_d2 = nbr_d2; a.fb_list = w.fb_list; a.fb_count = w.fb_count; a.rep = ctx->rep;
    a.work = w.fb_count + 1;
    a.cl = cl;
    a.dbg_d2 = p->dbg_idx ? p->dbg_d2 : nullptr;
    a.dbg_idx = p->dbg_idx;
    const bool radius_first = p->prune == VB_PRUNE_LEARNED;
    const bool tensor = p->precision == VB_PREC_BF16 || p->precision == VB_PREC_FP16;
    // the tiles a radius-first or 16-bit first pass hands back are searched with compact keys
    // before the full-key search takes what is left
    const bool compact_retry = (radius_first || tensor) && p->heap_keys != VB_KEYS_FULL && mp <= 16;
    int launches = 0;
    if (radius_first || tensor) {
        if (radius_first) {
            mark(ctx, VB_STAGE_KNN_RADIUS, 0);
            const float inflate = p->radius_inflate > 0.f ? p->radius_inflate : 1.5f;
            if (p->mlp) {
                st = mlp_radius_r2(s, p->mlp, w.xs, n, m, mp, p->radius_log_shift, inflate, w.r2, p->cloud_log_shift,
                                   cl, ctx->rep);
            } else {
                radius_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p->radius, perm, n, inflate, w.r2);
                st = last_launch();
            }
            if (st != VB_OK) return st;
            mark(ctx, VB_STAGE_KNN_RADIUS, 1);
            launches += 1;
        }
        if (cudaMemsetAsync(w.fail_flag, 0, sizeof(int) * 2 * ntiles, s) != cudaSuccess) return VB_ERR_CUDA;
        // counters: [1] first-pass work, [2] exact-search work, [3] first-pass failures
        a.r2 = radius_first ? w.r2 : nullptr;
        mark(ctx, VB_STAGE_KNN_TILE, 0);
        const bool f16 = p->precision == VB_PREC_FP16;
        a.r2_scale = 1.f;
        a.work = w.fb_count + 1;
        a.fail_flag = w.fail_flag;
        a.fail_list = w.fail_list;
        a.fail_count = w.fb_count + 3;
        if (tensor) {
            a.cap = a.L;
            st = VB_ERR_UNSUPPORTED;
            // automatic choice: pipelined for FP16; BF16's 8-bit significand needs the staged kernel's
            // operands recentred on every query tile (its error band at the cloud's centre is too wide)
            if ((p->tc_variant == VB_TC_PIPELINED || (p->tc_variant == VB_TC_AUTO && f16)) && w.blk) {
                // tile blocks of the pipelined search: centre, 16-bit images and norms
                a.kp = pad_k16(m);
                a.blk = w.blk;
                a.lbw = w.lbw;
                a.tlist = w.tlist;
                a.lbs = w.lbs;
                a.trad = w.trad;
                tile_ball_kernel<<<(unsigned)((ntiles * 32 + 255) / 256), 256, 0, s>>>(w.xs, n, ntiles, m, mp, w.tlo,
                                                                                      w.thi, w.trad);
                tcp_range_init_kernel<<<1, 128, 0, s>>>(w.crange);
                tcp_range_kernel<<<(unsigned)((n + 63) / 64), 128, 0, s>>>(w.xs, n, m, mp, w.crange);
                if (f16)
                    tcp_block_kernel<true><<<(unsigned)((npad + 255) / 256), 256, 0, s>>>(w.xs, n, npad, m, mp, a.kp,
                                                                                         w.crange, w.blk);
                else
                    tcp_block_kernel<false><<<(unsigned)((npad + 255) / 256), 256, 0, s>>>(w.xs, n, npad, m, mp,
                                                                                          a.kp, w.crange, w.blk);
                launches += 4;   // tile balls, range init, range, tile blocks
                switch (mp) {
                    case 4: st = f16 ? launch_tcp<4, true>(a, s) : launch_tcp<4, false>(a, s); break;
                    case 8: st = f16 ? launch_tcp<8, true>(a, s) : launch_tcp<8, false>(a, s); break;
                    case 16: st = f16 ? launch_tcp<16, true>(a, s) : launch_tcp<16, false>(a, s); break;
                    case 32: st = f16 ? launch_tcp<32, true>(a, s) : launch_tcp<32, false>(a, s); break;
                    case 64: st = f16 ? launch_tcp<64, true>(a, s) : launch_tcp<64, false>(a, s); break;
                    default: st = f16 ? launch_tcp<128, true>(a, s) : launch_tcp<128, false>(a, s); break;
                }
                if (st == VB_ERR_UNSUPPORTED && p->tc_variant == VB_TC_PIPELINED) return st;
                if (st == VB_OK) launches += 2;   // search, row finish
            }
            if (st == VB_ERR_UNSUPPORTED) {
                launches += 1;   // staged search (its rows are finished inside)
                switch (mp) {
                    case 4:
                        if (p->heap_keys == VB_KEYS_FULL)
                            st = f16 ? launch_tc<4, true, false>(a, s) : launch_tc<4, false, false>(a, s);
                        else
                            st = f16 ? launch_tc<4, true>(a, s) : launch_tc<4, false>(a, s);
                        break;
                    case 8: st = f16 ? launch_tc<8, true>(a, s) : launch_tc<8, false>(a, s); break;
                    case 16: st = f16 ? launch_tc<16, true>(a, s) : launch_tc<16, false>(a, s); break;
                    case 32: st = f16 ? launch_tc<32, true>(a, s) : launch_tc<32, false>(a, s); break;
                    case 64: st = f16 ? launch_tc<64, true>(a, s) : launch_tc<64, false>(a, s); break;
                    default: st = f16 ? launch_tc<128, true>(a, s) : launch_tc<128, false>(a, s); break;
                }
            }
        } else {
            launches += 1;   // radius-first FP32 search: compact keys at m <= 16 as in the plain search
            const bool compact = p->heap_keys != VB_KEYS_FULL && mp <= 16;
            switch (mp) {
                case 4: st = compact ? launch_tile<4, true>(a, s) : launch_tile<4>(a, s); break;
                case 8: st = compact ? launch_tile<8, true>(a, s) : launch_tile<8>(a, s); break;
                case 16: st = compact ? launch_tile<16, true>(a, s) : launch_tile<16>(a, s); break;
                case 32: st = launch_tile<32>(a, s); break;
                case 64: st = launch_tile<64>(a, s); break;
                default: st = launch_tile<128>(a, s); break;
            }
        }
        if (st != VB_OK) return st;
        // tiles the first pass could not settle: the exact FP32 search (seeded, no radius) on that list only
        a.r2 = nullptr;
        a.work = w.fb_count + 2;
        a.tile_list = w.fail_list;
        a.tile_count = w.fb_count + 3;
    } else if (p->heap_keys != VB_KEYS_FULL && mp <= 16) {
        // compact 32-bit heap keys first; tiles that overflow the visit table or have a row that
        // fails the certificate are redone below with full keys (wide inputs, where the box bounds
        // prune little and a query tile visits hundreds of tiles, keep full keys)
        if (cudaMemsetAsync(w.fail_flag, 0, sizeof(int) * 2 * ntiles, s) != cudaSuccess) return VB_ERR_CUDA;
        mark(ctx, VB_STAGE_KNN_TILE, 0);
        a.fail_flag = w.fail_flag;
        a.fail_list = w.fail_list;
        a.fail_count = w.fb_count + 3;
        launches += 1;
        switch (mp) {
            case 4: st = launch_tile<4, true>(a, s); break;
            case 8: st = launch_tile<8, true>(a, s); break;
            case 16: st = launch_tile<16, true>(a, s); break;
            case 32: st = launch_tile<32, true>(a, s); break;
            case 64: st = launch_tile<64, true>(a, s); break;
            default: st = launch_tile<128, true>(a, s); break;
        }
        if (st != VB_OK) return st;
        a.work = w.fb_count + 2;
        a.tile_list = w.fail_list;
        a.tile_count = w.fb_count + 3;
    }
    // the exact FP32 search: the only pass, or the passes over the tiles the first handed back
    const bool retry = a.tile_list != nullptr;
    if (retry) {
        mark(ctx, VB_STAGE_KNN_TILE, 1);
        mark(ctx, VB_STAGE_KNN_RETRY, 0);
    } else {
        mark(ctx, VB_STAGE_KNN_TILE, 0);
    }
    if (compact_retry) {
        // compact keys first (twice the CTAs per SM); the tiles that overflow the visit table or
        // fail the certificate go on, through the second half of the lists, to full keys
        a.fail_flag = w.fail_flag + ntiles;
        a.fail_list = w.fail_list + ntiles;
        a.fail_count = w.fb_count + 5;
        launches += 1;
        switch (mp) {
            case 4: st = launch_tile<4, true>(a, s); break;
            case 8: st = launch_tile<8, true>(a, s); break;
            default: st = launch_tile<16, true>(a, s); break;
        }
        if (st != VB_OK) return st;
        a.work = w.fb_count + 4;
        a.tile_list = w.fail_list + ntiles;
        a.tile_count = w.fb_count + 5;
    }
    switch (mp) {
        case 4: st = launch_tile<4>(a, s); break;
        case 8: st = launch_tile<8>(a, s); break;
        case 16: st = launch_tile<16>(a, s); break;
        case 32: st = launch_tile<32>(a, s); break;
        case 64: st = launch_tile<64>(a, s); break;
        default: st = launch_tile<128>(a, s); break;
    }
    if (st != VB_OK) return st;
    mark(ctx, retry ? VB_STAGE_KNN_RETRY : VB_STAGE_KNN_TILE, 1);
    mark(ctx, VB_STAGE_KNN_FALLBACK, 0);
    ctx->launches += launches;
    knn_fallback_kernel<<<152, FB_THREADS, 0, s>>>(x, n, m, p->k, w.fb_list, w.fb_count, cl, nbr, nbr_d2);
    mark(ctx, VB_STAGE_KNN_FALLBACK, 1);
    ctx->launches += 8;   // order: bbox init, bbox, Morton keys, gather, boxes, super-tile boxes (radix passes counted above); search; fallback
    return last_launch();
}

}  // namespace vb
