// Row passes over the symmetric pattern (steps a9-a14 of the build).
//
// Every pass is a fixed grid of warps walking CSR rows (warp w takes rows
// w, w + W, ...; the reductions take contiguous row ranges per block, split per
// point cloud), lanes striding the row's entries.  Per-entry arithmetic is FP32
// (ex2 on the SFU); a row's lane partials are added by a fixed FP32 shuffle tree
// (GB300's FP64 pipe is narrow: an FP64 tree per row cost more than the row),
// and sums across rows and blocks are carried in FP64 in a fixed order, so every
// result is bitwise reproducible run to run.
//   a9/a11 epsilon sweep (Sec. 2.3): chi_g = sum_E exp(-ed2 / (scale 2^xi_g rho_i rho_j))
//          for all grid points in one pass; the diagonal contributes n.
//   a10    density (Sec. 2.1): psi_i = sum_j K_eps^ij / (n (pi eps^2 b_i^2)^(d/2)), P = psi^beta.
//   (R9)   operator-sweep centre from sum_E' ed2/(4 P_i P_j) and sum_E' ed2/(b_i b_j).
//   a12    K_{eps,beta}, q = psi^(-beta d) K 1, K~ = K / (q_i q_j)^alpha, D = K~ 1, S = P D^(1/2) (Sec. 2.2).
//   a13    L-hat_ij = K~^ij / (eps^2 S_i S_j), L-hat_ii = -sum_{j != i} K~^ij / (eps^2 S_i^2).
//          Each off-diagonal value is a product of pairwise products
//          (x_i * x_j), so (i, j) and (j, i) give the same bits.
//   a14    CSR SpMV, plain and difference (Laplacian) form.
#include "vb_internal.cuh"

#include <algorithm>
#include <cmath>

namespace vb {

constexpr int WARPS = kRowThreads / 32;
constexpr int FLUSH = 1024;   // entries a warp sums in FP32 before carrying to FP64

struct RowIter {
    int64_t i, step;
    int lane, w;
    __device__ RowIter()
    {
        lane = threadIdx.x & 31;
        w = threadIdx.x >> 5;
        i = (int64_t)blockIdx.x * WARPS + w;
        step = (int64_t)gridDim.x * WARPS;
    }
};

// Rows handled by groups of LPR lanes (8, 16 or 32; 8 by default: four rows per warp keep
// more gathers in flight, 0.62 -> 0.43 ms for the operator pass and 0.55 -> 0.44 ms for L-hat
// at 1M torus points against 16 lanes), 32 / LPR rows per warp at a time; the loop
// over row bases is warp-uniform so the group sums can use full-warp shuffles.  Every
// entry point uses the same LPR, so a build and its step-by-step calls agree bit for bit.
template <int LPR>
struct RowGroup {
    static constexpr int RPW = 32 / LPR;
    int64_t base, step;
    int sub, grp;
    __device__ RowGroup()
    {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        sub = lane % LPR;
        grp = lane / LPR;
        base = ((int64_t)blockIdx.x * WARPS + w) * RPW;
        step = (int64_t)gridDim.x * WARPS * RPW;
    }
    static __device__ __forceinline__ float sum(float v)
    {
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
};

// A lane's next UNR entries of a row (stride LPR): their column and squared distance
// loaded together (column -1 past the row's end), so the gathers that follow are all in
// flight at once; the lane still adds its entries in increasing order, as a plain loop would.
constexpr int UNR = 4;
template <int LPR>
__device__ __forceinline__ void load_entries(const int32_t* __restrict__ col, const float* __restrict__ ed2,
                                             int64_t e0, int64_t re, int32_t* jj, float* xx)
{
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
        const int64_t e = e0 + (int64_t)u * LPR;
        const bool in = e < re;
        jj[u] = in ? col[e] : -1;
        xx[u] = in ? ed2[e] : 0.f;
    }
}

// The lane's quad of consecutive entries b0 .. b0 + 3 (b0 a multiple of 4) of the row [rb, re):
// one 16-byte load of the columns and one of the squared distances when the quad lies inside
// the row and the arrays are 16-byte aligned, else four masked loads (column -1 outside the
// row).  A group of LPR lanes covers 4 LPR consecutive entries per step, so each load
// instruction of the group reads whole 16-byte pieces.
static_assert(UNR == 4, "a quad of entries per lane");
__device__ __forceinline__ void load_quad(const int32_t* __restrict__ col, const float* __restrict__ ed2, bool vec,
                                          int64_t b0, int64_t rb, int64_t re, int32_t* jj, float* xx)
{
    if (vec && b0 >= rb && b0 + 3 < re) {
        const int4 c4 = *(const int4*)(col + b0);
        const float4 x4 = *(const float4*)(ed2 + b0);
        jj[0] = c4.x; jj[1] = c4.y; jj[2] = c4.z; jj[3] = c4.w;
        xx[0] = x4.x; xx[1] = x4.y; xx[2] = x4.z; xx[3] = x4.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t e = b0 + u;
            const bool in = e >= rb && e < re;
            jj[u] = in ? col[e] : -1;
            xx[u] = in ? ed2[e] : 0.f;
        }
    }
}
__device__ __forceinline__ bool aligned16(const void* a, const void* b)
{
    return (((uintptr_t)a | (uintptr_t)b) & 15u) == 0;
}
__device__ __forceinline__ int64_t quad_start(int64_t rb, int sub) { return (rb & ~(int64_t)3) + 4 * (int64_t)sub; }

__global__ void recip_f32_kernel(const double* __restrict__ v, int64_t n, float scale, float* out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)(1.0 / v[i]) * scale;
}

// ------------------------------------------------------------------ a9 / a11 epsilon sweep
struct SweepConst {
    float negr[kMaxGrid];   // -2^-(xi_lo + g dxi)
};

// Segmented reductions: block bl of the fixed grid owns the rows [bl per, (bl + 1) per),
// per = ceil(n / grid); the rows of each cloud inside that range form one segment,
// whose sums go to slot bl + cloud.  Slots are disjoint, every slot holds one cloud's
// rows, and cloud b's slots are bl + b for the blocks bl that meet it, so each
// cloud's total is summed in a fixed order.
__host__ __device__ inline int64_t rows_per_block(int64_t n, int nblk) { return (n + nblk - 1) / nblk; }
inline size_t seg_slots(int B) { return (size_t)kRowBlocks + (size_t)B; }
// The sweeps run one resident wave (three 256-thread blocks per SM, their launch bound): each
// warp then owns a longer range of entries, which amortises its 57 end-of-range reductions.
constexpr int kSweepBlocks = 152 * 2;

// Column totals over cloud b's slots (slots of G values) by a block of SEG_T threads:
// thread t sums column t % 64 over the slots bl = t / 64, t / 64 + SEG_PARTS, ... (reads of
// consecutive columns are contiguous), then the SEG_PARTS partial sums of every column
// are added in a fixed order.  out[g] for g < G; every thread must call it.
constexpr int SEG_T = 1024, SEG_COLS = 64, SEG_PARTS = SEG_T / SEG_COLS;
__device__ void seg_totals(const double* __restrict__ partial, int G, const Clouds& cl, int b, int64_t n, int nblk,
                           double* sh /* [SEG_PARTS][SEG_COLS] */, double* out)
{
    const int64_t per = rows_per_block(n, nblk);
    const int64_t lo = cloud_lo(cl, b), hi = cloud_hi(cl, b, n);
    const int64_t bl0 = lo / per, bl1 = (hi - 1) / per;
    const int g = threadIdx.x % SEG_COLS, part = threadIdx.x / SEG_COLS;
    // eight independent accumulators keep eight loads in flight per thread; the order of the
    // additions is fixed, so the totals are deterministic
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (g < G) {
        int64_t bl = bl0 + part;
        for (; bl + 7 * SEG_PARTS <= bl1; bl += 8 * SEG_PARTS) {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += partial[(bl + u * SEG_PARTS + b) * G + g];
        }
#pragma unroll
        for (int u = 0; u < 7; ++u)
            if (bl + u * SEG_PARTS <= bl1) acc[u] += partial[(bl + u * SEG_PARTS + b) * G + g];
    }
    sh[part * SEG_COLS + g] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    __syncthreads();
    if (threadIdx.x < G) {
        double t = 0.0;
        for (int q = 0; q < SEG_PARTS; ++q) t += sh[q * SEG_COLS + threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kRowThreads) sweep_kernel(const int64_t* __restrict__ row_ptr,
                                                          const int32_t* __restrict__ col,
                                                          const float* __restrict__ ed2, int64_t n,
                                                          const float* __restrict__ irho,
                                                          const double* __restrict__ xi_c_dev, double scale, int G,
                                                          SweepConst sc, Clouds cl, double* partial)
{
    __shared__ double wacc[WARPS][kMaxGrid];
    __shared__ float s_c0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = rows_per_block(n, gridDim.x);
    const int64_t r0 = min(n, (int64_t)blockIdx.x * per), r1 = min(n, r0 + per);
    if (r0 >= r1) return;
    const int cf = cloud_of(cl.ptr, cl.B, r0), cla = cloud_of(cl.ptr, cl.B, r1 - 1);
    float acc[kMaxGrid];
    for (int cb = cf; cb <= cla; ++cb) {
        for (int i = threadIdx.x; i < WARPS * kMaxGrid; i += blockDim.x) (&wacc[0][0])[i] = 0.0;
        if (threadIdx.x == 0) {
            const double xc = xi_c_dev ? xi_c_dev[cb] : 0.0;
            s_c0 = (float)(1.4426950408889634 / (scale * exp2(xc)));
        }
        __syncthreads();
        const float c0 = s_c0;
        const int64_t s0 = max(r0, cloud_lo(cl, cb)), s1 = min(r1, cloud_hi(cl, cb, n));
        const int64_t pw = (s1 - s0 + WARPS - 1) / WARPS;
        const int64_t a0 = min(s1, s0 + w * pw), a1 = min(s1, a0 + pw);
#pragma unroll
        for (int g = 0; g < kMaxGrid; ++g) acc[g] = 0.f;
        int since = 0;
        auto flush = [&]() {
#pragma unroll
            for (int g = 0; g < kMaxGrid; ++g) {
                if (g < G) {
                    float v = warp_sum_f32(acc[g]);
                    if (lane == 0) wacc[w][g] += (double)v;
                }
                acc[g] = 0.f;
            }
        };
        for (int64_t i = a0; i < a1; ++i) {
            const int64_t rb = row_ptr[i], re = row_ptr[i + 1];
            const float ri = irho[i];
            for (int64_t e = rb + lane; e < re; e += 32) {
                const int32_t j = col[e];
                if (j == i) continue;
                const float u = ed2[e] * (ri * irho[j]) * c0;
#pragma unroll
                for (int g = 0; g < kMaxGrid; ++g)
                    if (g < G) acc[g] += ex2_approx(u * sc.negr[g]);
            }
            since += (int)(re - rb);
            if (since >= FLUSH) {
                flush();
                since = 0;
            }
        }
        flush();
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
            double sum = 0.0;
            for (int ww = 0; ww < WARPS; ++ww) sum += wacc[ww][g];
            partial[((int64_t)blockIdx.x + cb) * G + g] = sum;
        }
        __syncthreads();
    }
}

// The standard grid (57 points, dxi = 1/4): with r_g = 2^-(xi_lo + g/4),
// r_{g-4} = 2 r_g, so exp(-t r_{g-4}) = exp(-t r_g)^2.  Each of the four chains
// g = 56 - c, 52 - c, ... takes an ex2 at every fourth step and squares in
// between (relative error at most 8x that of ex2, about 2e-6), which moves the
// pass from the SFU to the FMA pipe.  A warp owns a contiguous range of rows and
// its lanes stride that range's entries, so every lane stays busy whatever the
// row lengths; the row of an entry is tracked by a cursor per lane.
constexpr int G57 = 57;

// Warp reduce-scatter of 64 per-lane partial sums (slots >= 57 are zero): five halving
// steps, each lane trading half its slots with the partner lane o apart and keeping the half
// that its bit o selects, leave lane l with the warp's totals of slots 2l and 2l + 1 (the kept
// halves' offsets add up to 2l).  62 shuffles instead of 57 full butterflies, and the FP64
// accumulation that follows is two full-warp additions per flush instead of 57 one-lane ones
// (the FP64 pipe is narrow on this part).
__device__ __forceinline__ void warp_reduce_scatter64(const float (&a)[G57], float& s0, float& s1)
{
    const int lane = threadIdx.x & 31;
    float b[32], c[16], d[8], e[4], f[2];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const float lo = a[i], hi = i + 32 < G57 ? a[i + 32] : 0.f;
            b[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, 16);
        }
    }
    {
        const bool up = lane & 8;
#pragma unroll
        for (int i = 0; i < 16; ++i) c[i] = (up ? b[i + 16] : b[i]) + __shfl_xor_sync(0xffffffffu, up ? b[i] : b[i + 16], 8);
    }
    {
        const bool up = lane & 4;
#pragma unroll
        for (int i = 0; i < 8; ++i) d[i] = (up ? c[i + 8] : c[i]) + __shfl_xor_sync(0xffffffffu, up ? c[i] : c[i + 8], 4);
    }
    {
        const bool up = lane & 2;
#pragma unroll
        for (int i = 0; i < 4; ++i) e[i] = (up ? d[i + 4] : d[i]) + __shfl_xor_sync(0xffffffffu, up ? d[i] : d[i + 4], 2);
    }
    {
        const bool up = lane & 1;
#pragma unroll
        for (int i = 0; i < 2; ++i) f[i] = (up ? e[i + 2] : e[i]) + __shfl_xor_sync(0xffffffffu, up ? e[i] : e[i + 2], 1);
    }
    s0 = f[0];
    s1 = f[1];
}

__global__ void __launch_bounds__(kRowThreads, 2) sweep57_kernel(const int64_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col,
                                                            const float* __restrict__ ed2, int64_t n,
                                                            const float* __restrict__ irho,
                                                            const double* __restrict__ xi_c_dev, double scale,
                                                            SweepConst sc, Clouds cl, double* partial)
{
    __shared__ double wacc[WARPS][G57];
    __shared__ float s_c0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = rows_per_block(n, gridDim.x);
    const int64_t r0 = min(n, (int64_t)blockIdx.x * per), r1 = min(n, r0 + per);
    if (r0 >= r1) return;
    const int cf = cloud_of(cl.ptr, cl.B, r0), cla = cloud_of(cl.ptr, cl.B, r1 - 1);
    float acc[G57];
    for (int cb = cf; cb <= cla; ++cb) {
        for (int i = threadIdx.x; i < WARPS * G57; i += blockDim.x) (&wacc[0][0])[i] = 0.0;
        if (threadIdx.x == 0) {
            const double xc = xi_c_dev ? xi_c_dev[cb] : 0.0;
            s_c0 = (float)(1.4426950408889634 / (scale * exp2(xc)));
        }
        __syncthreads();
        const float c0 = s_c0;
        const int64_t s0 = max(r0, cloud_lo(cl, cb)), s1 = min(r1, cloud_hi(cl, cb, n));
        const int64_t pw = (s1 - s0 + WARPS - 1) / WARPS;
        const int64_t a0 = min(s1, s0 + w * pw), a1 = min(s1, a0 + pw);
        const int64_t e0 = row_ptr[a0], e1 = row_ptr[a1];
#pragma unroll
        for (int g = 0; g < G57; ++g) acc[g] = 0.f;
        double dacc0 = 0.0, dacc1 = 0.0;   // this lane's share of the warp's totals: slots 2 lane, 2 lane + 1
        auto flush = [&]() {
            float s0, s1;
            warp_reduce_scatter64(acc, s0, s1);
            dacc0 += (double)s0;
            dacc1 += (double)s1;
#pragma unroll
            for (int g = 0; g < G57; ++g) acc[g] = 0.f;
        };
        int64_t i = a0;
        int64_t inext = row_ptr[min(a0 + 1, n)];
        float ri = a0 < n ? irho[a0] : 0.f;
        int64_t inext2 = row_ptr[min(a0 + 2, n)];   // the next row's end and bandwidth, loaded a row ahead
        float ri_next = irho[min(a0 + 1, n - 1)];
        int since = 0;
        // software pipeline: the column and squared distance of the entry three chunks ahead and
        // the bandwidth gather of the entry two chunks ahead are in flight while this chunk's 57
        // kernel values are formed (column -1: past the warp's range); the row cursor keeps the
        // next row's end and bandwidth loaded a row ahead
        int32_t j0 = -1, j1 = -1, j2 = -1;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        if (e0 + lane < e1) { j0 = col[e0 + lane]; x0 = ed2[e0 + lane]; }
        if (e0 + 32 + lane < e1) { j1 = col[e0 + 32 + lane]; x1 = ed2[e0 + 32 + lane]; }
        if (e0 + 64 + lane < e1) { j2 = col[e0 + 64 + lane]; x2 = ed2[e0 + 64 + lane]; }
        float rj0 = j0 >= 0 ? irho[j0] : 0.f;
        float rj1 = j1 >= 0 ? irho[j1] : 0.f;
        for (int64_t eb = e0; eb < e1; eb += 32) {
            const int64_t e = eb + lane;
            int32_t j3 = -1;
            float x3 = 0.f;
            if (e + 96 < e1) { j3 = col[e + 96]; x3 = ed2[e + 96]; }
            const float rj2 = j2 >= 0 ? irho[j2] : 0.f;
            float u = INFINITY;
            if (e < e1) {
                while (inext <= e) {
                    ++i;
                    inext = inext2;
                    ri = ri_next;
                    inext2 = row_ptr[min(i + 2, n)];
                    ri_next = irho[min(i + 1, n - 1)];
                }
                if (j0 != i) u = x0 * (ri * rj0) * c0;
            }
            j0 = j1; x0 = x1; rj0 = rj1;
            j1 = j2; x1 = x2; rj1 = rj2;
            j2 = j3; x2 = x3;
            float prev[4];
#pragma unroll
            for (int g = G57 - 1; g >= 0; --g) {
                const int c = (G57 - 1 - g) & 3, step = (G57 - 1 - g) >> 2;
                const float v = (step & 3) == 0 ? ex2_approx(u * sc.negr[g]) : prev[c] * prev[c];
                prev[c] = v;
                acc[g] += v;
            }
            if (++since == 32) {
                since = 0;
                flush();
            }
        }
        flush();
        if (2 * lane < G57) wacc[w][2 * lane] = dacc0;
        if (2 * lane + 1 < G57) wacc[w][2 * lane + 1] = dacc1;
        __syncthreads();
        for (int g = threadIdx.x; g < G57; g += blockDim.x) {
            double sum = 0.0;
            for (int ww = 0; ww < WARPS; ++ww) sum += wacc[ww][g];
            partial[((int64_t)blockIdx.x + cb) * G57 + g] = sum;
        }
        __syncthreads();
    }
}

// One block per cloud: the column totals over the cloud's slots (seg_totals), then
// the threads take one log each and one warp finds the first maximiser of chi'.
__global__ void __launch_bounds__(1024) sweep_finish_kernel(const double* __restrict__ partial, int nblk, int G,
                                                           int64_t n, Clouds cl, double xi_lo, double dxi,
                                                           const double* __restrict__ xi_c_dev, int warn_bit,
                                                           double* eps2, double* chi, double* dim, DevReport* rep)
{
    __shared__ double sh[kMaxGrid], lg[kMaxGrid];
    __shared__ double part[SEG_PARTS * SEG_COLS];
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double nb = (double)(cloud_hi(cl, b, n) - cloud_lo(cl, b));
    seg_totals(partial, G, cl, b, n, nblk, part, sh);
    if (threadIdx.x < G) {
        sh[threadIdx.x] += nb;   // diagonal entries: exp(0) = 1 each
        chi[(int64_t)b * G + threadIdx.x] = sh[threadIdx.x];
    }
    __syncthreads();
    if (threadIdx.x < G) lg[threadIdx.x] = log(sh[threadIdx.x]);
    __syncthreads();
    if (w == 0) {
        const double inv = 1.0 / (dxi * 0.69314718055994531);
        double bv = -INFINITY;
        int best = 0;
        for (int h = lane; h + 1 < G; h += 32) {
            double cp = (lg[h + 1] - lg[h]) * inv;
            if (cp > bv) { bv = cp; best = h; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            int ob = __shfl_xor_sync(0xffffffffu, best, o);
            if (ov > bv || (ov == bv && ob < best)) { bv = ov; best = ob; }
        }
        if (lane == 0) {
            const double xc = xi_c_dev ? xi_c_dev[b] : 0.0;
            eps2[b] = exp2(xc + xi_lo + best * dxi);
            dim[b] = 2.0 * bv;
            if (best == 0 || best == G - 2) atomicOr(&rep->warnings, warn_bit);
        }
    }
}

size_t sweep_ws_bytes(int64_t n, int B)
{
    Carve c(nullptr);
    c.take<float>(n);
    c.take<double>(seg_slots(B) * kMaxGrid);
    return c.off;
}

vb_status sweep_run(Ctx* ctx, const vb_graph* g, const double* rho, double scale, const double* xi_c_dev,
                    double xi_lo, double xi_hi, double dxi, int warn_bit, double* eps2, double* chi, double* dim,
                    void* ws, size_t ws_bytes, Clouds cl)
{
    if (!g || !g->row_ptr || !g->col || !g->ed2 || g->n < 1 || !rho || !eps2 || !chi || !dim) return VB_ERR_ARG;
    if (!(dxi > 0) || !(scale > 0) || cl.B < 1 || (cl.B > 1 && !cl.ptr)) return VB_ERR_ARG;
    const int G = (int)std::lround((xi_hi - xi_lo) / dxi) + 1;
    if (G < 3 || G > kMaxGrid) return VB_ERR_ARG;
    Carve c(ws);
    float* irho = c.take<float>(g->n);
    double* partial = c.take<double>(seg_slots(cl.B) * kMaxGrid);
    if (!ws || ws_bytes < c.off) return VB_ERR_WORKSPACE;
    SweepConst sc;
    for (int h = 0; h < kMaxGrid; ++h) sc.negr[h] = h < G ? -(float)std::exp2(-(xi_lo + h * dxi)) : 0.f;
    cudaStream_t s = ctx->stream;
    const int stage = warn_bit == 2 ? VB_STAGE_SWEEP_OPERATOR : VB_STAGE_SWEEP_DENSITY;
    recip_f32_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(rho, g->n, 1.f, irho);
    mark(ctx, stage, 0);
    if (G == G57 && dxi == 0.25)
        sweep57_kernel<<<kSweepBlocks, kRowThreads, 0, s>>>(g->row_ptr, g->col, g->ed2, g->n, irho, xi_c_dev, scale, sc,
                                                          cl, partial);
    else
        sweep_kernel<<<kSweepBlocks, kRowThreads, 0, s>>>(g->row_ptr, g->col, g->ed2, g->n, irho, xi_c_dev, scale, G, sc,
                                                        cl, partial);
    mark(ctx, stage, 1);
    sweep_finish_kernel<<<(unsigned)cl.B, 1024, 0, s>>>(partial, kSweepBlocks, G, g->n, cl, xi_lo, dxi, xi_c_dev,
                                                        warn_bit, eps2, chi, dim, ctx->rep);
    ctx->launches += 3;
    return last_launch();
}

// ------------------------------------------------------------------ a10 density
// Per-cloud FP32 constant log2(e) / eps^2 of the density kernel.
__global__ void density_const_kernel(const double* __restrict__ eps2, int B, float* c)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) c[b] = (float)(1.4426950408889634 / eps2[b]);
}

template <int LPR>
__global__ void __launch_bounds__(kRowThreads) density_kernel(const int64_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col,
                                                            const float* __restrict__ ed2, int64_t n,
                                                            const float* __restrict__ ib,
                                                            const float* __restrict__ cden, Clouds cl, double* psi)
{
    RowGroup<LPR> it;
    const bool vec = aligned16(col, ed2);
    for (int64_t b0 = it.base; b0 < n; b0 += it.step) {
        const int64_t i = b0 + it.grp;
        const bool ok = i < n;
        const float c = ok ? cden[cloud_id(cl, i)] : 0.f;
        const int64_t rb = ok ? row_ptr[i] : 0, re = ok ? row_ptr[i + 1] : 0;
        const float bi = ok ? ib[i] : 0.f;
        float s = 0.f;
        for (int64_t e0 = quad_start(rb, it.sub); e0 < re; e0 += 4 * LPR) {
            int32_t jj[UNR];
            float xx[UNR];
            load_quad(col, ed2, vec, e0, rb, re, jj, xx);
#pragma unroll
            for (int u = 0; u < UNR; ++u)
                if (jj[u] >= 0) s += ex2_approx(-(xx[u] * (bi * ib[jj[u]])) * c);
        }
        const float tot = RowGroup<LPR>::sum(s);
        if (ok && it.sub == 0) psi[i] = (double)tot;
    }
}

// w_i = n_b (pi eps_b^2 b_i^2)^(d/2) with n_b and eps_b those of the point's cloud,
// psi_i = sum_i / w_i, P_i = psi_i^beta, one thread per point.  FP64 powers: P enters
// every operator-kernel exponent, so its error is multiplied by exponents of up to
// about 60 in the smallest stored entries.
__global__ void density_finish_kernel(const double* __restrict__ b, const double* __restrict__ eps2_dev, int64_t n,
                                      Clouds cl, double d, double beta, double* psi, double* P)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cb = cloud_id(cl, i);
    const double nb = (double)(cloud_hi(cl, cb, n) - cloud_lo(cl, cb));
    const double bb = b[i];
    // the FP64 pipe is narrow: the exponents of the workloads (d / 2 = 1/2, 1, 5/2; beta = -1/4)
    // avoid the general power, x^1 = x exactly and the roots correctly rounded
    const double x = 3.14159265358979323846 * eps2_dev[cb] * bb * bb, e = 0.5 * d;
    const double w = nb * (e == 1.0 ? x : e == 0.5 ? sqrt(x) : e == 2.5 ? x * x * sqrt(x) : pow(x, e));
    const double ps = psi[i] / w;
    psi[i] = ps;
    P[i] = beta == -0.25 ? 1.0 / sqrt(sqrt(ps)) : pow(ps, beta);
}

size_t density_ws_bytes(int64_t n, int B)
{
    Carve c(nullptr);
    c.take<float>(n);
    c.take<float>(B);
    return c.off;
}

vb_status density_run(Ctx* ctx, const vb_graph* g, const double* b, const double* eps2_dev, double d, double beta,
                      double* psi, double* P, void* ws, size_t ws_bytes, Clouds cl, int lpr)
{
    if (!g || !g->row_ptr || !b || !eps2_dev || !psi || !P || !(d > 0)) return VB_ERR_ARG;
    if (cl.B < 1 || (cl.B > 1 && !cl.ptr)) return VB_ERR_ARG;
    Carve c(ws);
    float* ib = c.take<float>(g->n);
    float* cden = c.take<float>(cl.B);
    if (!ws || ws_bytes < c.off) return VB_ERR_WORKSPACE;
    cudaStream_t s = ctx->stream;
    mark(ctx, VB_STAGE_DENSITY, 0);
    recip_f32_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(b, g->n, 1.f, ib);
    density_const_kernel<<<(unsigned)((cl.B + 255) / 256), 256, 0, s>>>(eps2_dev, cl.B, cden);
    switch (lpr) {
        case 8: density_kernel<8><<<kRowBlocks, kRowThreads, 0, s>>>(g->row_ptr, g->col, g->ed2, g->n, ib, cden, cl, psi); break;
        case 16: density_kernel<16><<<kRowBlocks, kRowThreads, 0, s>>>(g->row_ptr, g->col, g->ed2, g->n, ib, cden, cl, psi); break;
        default: density_kernel<32><<<kRowBlocks, kRowThreads, 0, s>>>(g->row_ptr, g->col, g->ed2, g->n, ib, cden, cl, psi); break;
    }
    density_finish_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(b, eps2_dev, g->n, cl, d, beta, psi, P);
    mark(ctx, VB_STAGE_DENSITY, 1);
    ctx->launches += 4;
    return last_launch();
}

// ------------------------------------------------------------------ operator-sweep centre
// Segmented like the sweeps: slot bl + cloud holds the two sums of one cloud's rows.
// 1 / b and 1 / P of every point as one 8-byte record, so that each entry's gather is one load.
__global__ void recip_bp_kernel(const double* __restrict__ b, const double* __restrict__ P, int64_t n, float2* bp)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) bp[i] = make_float2((float)(1.0 / b[i]), (float)(1.0 / P[i]));
}

__global__ void __launch_bounds__(kRowThreads) centre_kernel(const int64_t* __restrict__ row_ptr,
                                                           const int32_t* __restrict__ col,
                                                           const float* __restrict__ ed2, int64_t n,
                                                           const float2* __restrict__ bp, Clouds cl, double* partial)
{
    __shared__ double sh[WARPS][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = rows_per_block(n, gridDim.x);
    const int64_t r0 = min(n, (int64_t)blockIdx.x * per), r1 = min(n, r0 + per);
    if (r0 >= r1) return;
    const int cf = cloud_of(cl.ptr, cl.B, r0), cla = cloud_of(cl.ptr, cl.B, r1 - 1);
    for (int cb = cf; cb <= cla; ++cb) {
        const int64_t s0 = max(r0, cloud_lo(cl, cb)), s1 = min(r1, cloud_hi(cl, cb, n));
        double a_op = 0.0, a_den = 0.0;
        for (int64_t i = s0 + w; i < s1; i += WARPS) {
            const int64_t rb = row_ptr[i], re = row_ptr[i + 1];
            const float2 bpi = bp[i];
            const float pi_ = bpi.y, bi = bpi.x;
            float so = 0.f, sd = 0.f;
            for (int64_t e0 = rb + lane; e0 < re; e0 += UNR * 32) {
                int32_t jj[UNR];
                float xx[UNR];
                load_entries<32>(col, ed2, e0, re, jj, xx);
                float2 bj[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u)
                    if (jj[u] >= 0) bj[u] = bp[jj[u]];
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const int32_t j = jj[u];
                    if (j < 0 || j == i) continue;
                    so += xx[u] * (pi_ * bj[u].y);
                    sd += xx[u] * (bi * bj[u].x);
                }
            }
            so = warp_sum_f32(so);   // FP32 tree over the lanes; the FP64 pipe is narrow
            sd = warp_sum_f32(sd);
            a_op += (double)so;
            a_den += (double)sd;
        }
        if (lane == 0) { sh[w][0] = a_op; sh[w][1] = a_den; }
        __syncthreads();
        if (threadIdx.x < 2) {
            double sum = 0.0;
            for (int ww = 0; ww < WARPS; ++ww) sum += sh[ww][threadIdx.x];
            partial[2 * ((int64_t)blockIdx.x + cb) + threadIdx.x] = sum;
        }
        __syncthreads();
    }
}

// One block per cloud.
__global__ void __launch_bounds__(SEG_T) centre_finish_kernel(const double* __restrict__ partial, int nblk, int64_t n,
                                                              Clouds cl, double* xi_c)
{
    __shared__ double part[SEG_PARTS * SEG_COLS];
    __shared__ double tot[2];
    const int b = blockIdx.x;
    seg_totals(partial, 2, cl, b, n, nblk, part, tot);
    // R9: the operator argument is ed2 / (4 P_i P_j); tot[0] holds sum ed2 / (P_i P_j)
    if (threadIdx.x == 0) xi_c[b] = floor(4.0 * log2(0.25 * tot[0] / tot[1]) + 0.5) / 4.0;
}

size_t centre_ws_bytes(int64_t n, int B)
{
    Carve c(nullptr);
    c.take<float2>(n);
    c.take<double>(seg_slots(B) * 2);
    return c.off;
}

vb_status centre_run(Ctx* ctx, const vb_graph* g, const double* b, const double* P, double* xi_c_dev, void* ws,
                     size_t ws_bytes, Clouds cl)
{
    if (!g || !g->row_ptr || !b || !P || !xi_c_dev) return VB_ERR_ARG;
    if (cl.B < 1 || (cl.B > 1 && !cl.ptr)) return VB_ERR_ARG;
    Carve c(ws);
    float2* bp = c.take<float2>(g->n);
    double* partial = c.take<double>(seg_slots(cl.B) * 2);
    if (!ws || ws_bytes < c.off) return VB_ERR_WORKSPACE;
    cudaStream_t s = ctx->stream;
    mark(ctx, VB_STAGE_CENTRE, 0);
    recip_bp_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(b, P, g->n, bp);
    centre_kernel<<<kRowBlocks, kRowThreads, 0, s>>>(g->row_ptr, g->col, g->ed2, g->n, bp, cl, partial);
    centre_finish_kernel<<<(unsigned)cl.B, SEG_T, 0, s>>>(partial, kRowBlocks, g->n, cl, xi_c_dev);
    mark(ctx, VB_STAGE_CENTRE, 1);
    ctx->launches += 3;
    return last_launch();
}

// ------------------------------------------------------------------ a12 / a13 operator and L-hat
// The per-point values every entry gathers from its column j, packed in one 16-byte record so
// that a gather is one sector: 1 / P as an unevaluated pair (hi, lo) of floats, q^-alpha (set
// by the q pass) and 1 / S (set by the D pass).
struct __align__(16) PointOp {
    float iPh, iPl, qa, iS;
};

__global__ void recip_pair_kernel(const double* __restrict__ v, int64_t n, PointOp* pv)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = 1.0 / v[i];
    const float h = (float)r;
    pv[i].iPh = h;
    pv[i].iPl = (float)(r - (double)h);
}

// K_{eps,beta}^ij = 2^-u, u = ed2 * (c1 * (iP_i * iP_j)), c1 = log2(e) / (4 eps^2).  The
// exponent is carried as a float pair (error-free products with fmaf), because an
// exponent error du changes K by the relative amount du ln 2 and u reaches about
// 60 in the smallest stored entries.  Every step is symmetric in (i, j), so
// K^ij and K^ji have the same bits.
__device__ __forceinline__ float k_op(float x, float ahi, float ali, float ahj, float alj, float ch, float cl)
{
    const float wh = ahi * ahj;
    const float wl = fmaf(ahi, ahj, -wh) + (ahi * alj + ali * ahj);
    const float th = ch * wh;
    const float tl = fmaf(ch, wh, -th) + (ch * wl + cl * wh);
    const float uh = x * th;
    const float ul = fmaf(x, th, -uh) + x * tl;
    return ex2_approx(-uh) * fmaf(-ul, 0.6931471805599453f, 1.0f);
}

// Per-cloud constants of the operator kernel: c1 = log2(e) / (4 eps^2) as a float
// pair (h, l), and 1 / eps^2.
struct __align__(16) C1 {
    float h, l, ie, pad;
};
__global__ void op_const_kernel(const double* __restrict__ eps2, int B, C1* out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double c = 1.4426950408889634 / (4.0 * eps2[b]);
    C1 r;
    r.h = (float)c;
    r.l = (float)(c - (double)r.h);
    r.ie = (float)(1.0 / eps2[b]);
    r.pad = 0.f;
    out[b] = r;
}

// A lane's next UNR entries with their column records gathered, all loads in flight together.
__device__ __forceinline__ void load_op_entries(const int32_t* __restrict__ col, const float* __restrict__ ed2,
                                                const PointOp* __restrict__ pv, bool vec, int64_t e0, int64_t rb,
                                                int64_t re, int32_t* jj, float* xx, PointOp* pj)
{
    load_quad(col, ed2, vec, e0, rb, re, jj, xx);
#pragma unroll
    for (int u = 0; u < UNR; ++u)
        if (jj[u] >= 0) pj[u] = pv[jj[u]];
}

// q pass: q_i = psi_i^(-beta d) sum_j K^ij; with ALPHA0 (alpha = 0, so q^-alpha = 1 and
// K~ = K) the same row sum is also D_i, and the pass writes D, S = P D^(1/2) and 1 / S
// too: the D pass would add the same values in the same order.
template <int LPR, bool ALPHA0>
__global__ void __launch_bounds__(kRowThreads) q_kernel(const int64_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col, const float* __restrict__ ed2,
                                                      int64_t n, const double* __restrict__ psi, PointOp* pv,
                                                      const C1* __restrict__ cop, Clouds cl, double beta, double d,
                                                      double alpha, double* q, const double* __restrict__ P,
                                                      double* D, double* S)
{
    const float mbd = (float)(-beta * d), malpha = (float)(-alpha);
    RowGroup<LPR> it;
    const bool vec = aligned16(col, ed2);
    for (int64_t b0 = it.base; b0 < n; b0 += it.step) {
        const int64_t i = b0 + it.grp;
        const bool ok = i < n;
        const C1 c1 = cop[ok ? cloud_id(cl, i) : 0];
        const int64_t rb = ok ? row_ptr[i] : 0, re = ok ? row_ptr[i + 1] : 0;
        const float ph = ok ? pv[i].iPh : 0.f, pl = ok ? pv[i].iPl : 0.f;
        float s = 0.f;
        for (int64_t e0 = quad_start(rb, it.sub); e0 < re; e0 += 4 * LPR) {
            int32_t jj[UNR];
            float xx[UNR];
            PointOp pj[UNR];
            load_op_entries(col, ed2, pv, vec, e0, rb, re, jj, xx, pj);
#pragma unroll
            for (int u = 0; u < UNR; ++u)
                if (jj[u] >= 0) s += k_op(xx[u], ph, pl, pj[u].iPh, pj[u].iPl, c1.h, c1.l);
        }
        const float sum = RowGroup<LPR>::sum(s);
        if (ok && it.sub == 0) {
            const float qi = pow_sfu((float)psi[i], mbd) * sum;
            q[i] = (double)qi;
            pv[i].qa = pow_sfu(qi, malpha);
            if constexpr (ALPHA0) {
                const double tot = (double)sum;
                const double si = P[i] * sqrt(tot);
                D[i] = tot;
                S[i] = si;
                pv[i].iS = (float)(1.0 / si);
            }
        }
    }
}

template <int LPR>
__global__ void __launch_bounds__(kRowThreads) d_kernel(const int64_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col, const float* __restrict__ ed2,
                                                      int64_t n, PointOp* pv, const double* __restrict__ P,
                                                      const C1* __restrict__ cop, Clouds cl, double* D, double* S)
{
    RowGroup<LPR> it;
    const bool vec = aligned16(col, ed2);
    for (int64_t b0 = it.base; b0 < n; b0 += it.step) {
        const int64_t i = b0 + it.grp;
        const bool ok = i < n;
        const C1 c1 = cop[ok ? cloud_id(cl, i) : 0];
        const int64_t rb = ok ? row_ptr[i] : 0, re = ok ? row_ptr[i + 1] : 0;
        const PointOp pi = ok ? pv[i] : PointOp{0.f, 0.f, 0.f, 0.f};
        float s = 0.f;
        for (int64_t e0 = quad_start(rb, it.sub); e0 < re; e0 += 4 * LPR) {
            int32_t jj[UNR];
            float xx[UNR];
            PointOp pj[UNR];
            load_op_entries(col, ed2, pv, vec, e0, rb, re, jj, xx, pj);
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                if (jj[u] < 0) continue;
                s += k_op(xx[u], pi.iPh, pi.iPl, pj[u].iPh, pj[u].iPl, c1.h, c1.l) * (pi.qa * pj[u].qa);
            }
        }
        const double tot = (double)RowGroup<LPR>::sum(s);
        if (ok && it.sub == 0) {
            const double si = P[i] * sqrt(tot);
            D[i] = tot;
            S[i] = si;
            pv[i].iS = (float)(1.0 / si);
        }
    }
}

template <int LPR>
__global__ void __launch_bounds__(kRowThreads, 4) lhat_kernel(const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col,
                                                         const float* __restrict__ ed2, int64_t n,
                                                         const PointOp* __restrict__ pv, const double* __restrict__ S,
                                                         const C1* __restrict__ cop,
                                                         const double* __restrict__ eps2_dev, Clouds cl, float* val)
{
    RowGroup<LPR> it;
    const bool vec = aligned16(col, ed2) && aligned16(val, val);
    for (int64_t b0 = it.base; b0 < n; b0 += it.step) {
        const int64_t i = b0 + it.grp;
        const bool ok = i < n;
        const int cb = ok ? cloud_id(cl, i) : 0;
        const C1 c1 = cop[cb];
        const float ie = c1.ie;
        const int64_t rb = ok ? row_ptr[i] : 0, re = ok ? row_ptr[i + 1] : 0;
        const PointOp pi = ok ? pv[i] : PointOp{0.f, 0.f, 0.f, 0.f};
        float off = 0.f;
        int64_t diag = -1;
        for (int64_t e0 = quad_start(rb, it.sub); e0 < re; e0 += 4 * LPR) {
            int32_t jj[UNR];
            float xx[UNR];
            PointOp pj[UNR];
            load_op_entries(col, ed2, pv, vec, e0, rb, re, jj, xx, pj);
            float vq[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                vq[u] = 0.f;
                const int32_t j = jj[u];
                if (j < 0) continue;
                if (j == i) { diag = e0 + u; continue; }
                const float kt = k_op(xx[u], pi.iPh, pi.iPl, pj[u].iPh, pj[u].iPl, c1.h, c1.l) * (pi.qa * pj[u].qa);
                off += kt;
                vq[u] = kt * (pi.iS * pj[u].iS) * ie;
            }
            if (vec && e0 >= rb && e0 + 3 < re) {   // one 16-byte store (a diagonal slot is rewritten below)
                *(float4*)(val + e0) = make_float4(vq[0], vq[1], vq[2], vq[3]);
            } else {
#pragma unroll
                for (int u = 0; u < UNR; ++u)
                    if (jj[u] >= 0 && jj[u] != i) val[e0 + u] = vq[u];
            }
        }
        const double tot = (double)RowGroup<LPR>::sum(off);
        if (diag >= 0) {
            const double sii = S[i];
            val[diag] = (float)(-tot / (eps2_dev[cb] * sii * sii));
        }
    }
}

size_t kernel_csr_ws_bytes(int64_t n, int B)
{
    Carve c(nullptr);
    c.take<PointOp>(n);
    c.take<C1>(B);
    return c.off;
}

vb_status kernel_csr_run(Ctx* ctx, const vb_graph* g, const double* psi, const double* P, const vb_op_params* op,
                         const double* eps2_op_dev, float* val, double* q, double* D, double* S, void* ws,
                         size_t ws_bytes, Clouds cl, int lpr)
{
    if (!g || !g->row_ptr || !psi || !P || !op || !eps2_op_dev || !val || !q || !D || !S) return VB_ERR_ARG;
    if (!(op->d > 0) || cl.B < 1 || (cl.B > 1 && !cl.ptr)) return VB_ERR_ARG;
    Carve c(ws);
    PointOp* pv = c.take<PointOp>(g->n);
    C1* cop = c.take<C1>(cl.B);
    if (!ws || ws_bytes < c.off) return VB_ERR_WORKSPACE;
    // Sec. 2.2: c = 2 - 2 alpha + d beta + 2 beta
    const double alpha = (2.0 - op->c + op->d * op->beta + 2.0 * op->beta) / 2.0;
    cudaStream_t s = ctx->stream;
    const int64_t n = g->n;
    mark(ctx, VB_STAGE_OPERATOR, 0);
    recip_pair_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, n, pv);
    op_const_kernel<<<(unsigned)((cl.B + 255) / 256), 256, 0, s>>>(eps2_op_dev, cl.B, cop);
#define VB_ROWS(K, ...)                                                        \
    switch (lpr) {                                                             \
        case 8: K<8><<<kRowBlocks, kRowThreads, 0, s>>>(__VA_ARGS__); break;   \
        case 16: K<16><<<kRowBlocks, kRowThreads, 0, s>>>(__VA_ARGS__); break; \
        default: K<32><<<kRowBlocks, kRowThreads, 0, s>>>(__VA_ARGS__); break; \
    }
#define VB_ROWS2(K, A0, ...)                                                       \
    switch (lpr) {                                                                 \
        case 8: K<8, A0><<<kRowBlocks, kRowThreads, 0, s>>>(__VA_ARGS__); break;   \
        case 16: K<16, A0><<<kRowBlocks, kRowThreads, 0, s>>>(__VA_ARGS__); break; \
        default: K<32, A0><<<kRowBlocks, kRowThreads, 0, s>>>(__VA_ARGS__); break; \
    }
    if (alpha == 0.0) {   // K~ = K: one pass gives q, D and S
        VB_ROWS2(q_kernel, true, g->row_ptr, g->col, g->ed2, n, psi, pv, cop, cl, op->beta, op->d, alpha, q, P, D, S)
        ctx->launches += 1;
    } else {
        VB_ROWS2(q_kernel, false, g->row_ptr, g->col, g->ed2, n, psi, pv, cop, cl, op->beta, op->d, alpha, q, P, D, S)
        VB_ROWS(d_kernel, g->row_ptr, g->col, g->ed2, n, pv, P, cop, cl, D, S)
        ctx->launches += 2;
    }
    mark(ctx, VB_STAGE_OPERATOR, 1);
    mark(ctx, VB_STAGE_LHAT, 0);
    VB_ROWS(lhat_kernel, g->row_ptr, g->col, g->ed2, n, pv, S, cop, eps2_op_dev, cl, val)
#undef VB_ROWS
#undef VB_ROWS2
    mark(ctx, VB_STAGE_LHAT, 1);
    ctx->launches += 3;
    return last_launch();
}

// ------------------------------------------------------------------ a14 SpMV
__global__ void __launch_bounds__(kRowThreads) spmv_plain_kernel(const int64_t* __restrict__ row_ptr,
                                                               const int32_t* __restrict__ col,
                                                               const float* __restrict__ val, int64_t n, float alpha,
                                                               const float* __restrict__ x, float beta, float* y)
{
    RowIter it;
    for (int64_t i = it.i; i < n; i += it.step) {
        const int64_t rb = row_ptr[i], re = row_ptr[i + 1];
        float s = 0.f;
        for (int64_t e = rb + it.lane; e < re; e += 32) s = fmaf(val[e], x[col[e]], s);
        const double tot = (double)warp_sum_f32(s);
        if (it.lane == 0) y[i] = (float)((double)alpha * tot + (beta != 0.f ? (double)beta * y[i] : 0.0));
    }
}

__global__ void lap_prep_kernel(const float* __restrict__ x, const double* __restrict__ S, int64_t n, double* z,
                                float* sf)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const double si = S[i];
        z[i] = (double)x[i] / si;
        sf[i] = (float)si;
    }
}

// y_i = alpha sum_{j != i} val_ij S_j (z_j - z_i) + beta y_i, z = x / S: the
// differences are taken in FP64 so that smooth vectors keep their accuracy.
__global__ void __launch_bounds__(kRowThreads) spmv_lap_kernel(const int64_t* __restrict__ row_ptr,
                                                             const int32_t* __restrict__ col,
                                                             const float* __restrict__ val, int64_t n, float alpha,
                                                             const double* __restrict__ z, const float* __restrict__ sf,
                                                             float beta, float* y)
{
    RowIter it;
    for (int64_t i = it.i; i < n; i += it.step) {
        const int64_t rb = row_ptr[i], re = row_ptr[i + 1];
        const double zi = z[i];
        float s = 0.f;
        for (int64_t e = rb + it.lane; e < re; e += 32) {
            const int32_t j = col[e];
            if (j == i) continue;
            s = fmaf(val[e] * sf[j], (float)(z[j] - zi), s);
        }
        const double tot = (double)warp_sum_f32(s);
        if (it.lane == 0) y[i] = (float)((double)alpha * tot + (beta != 0.f ? (double)beta * y[i] : 0.0));
    }
}

// Laplacian-form SpMV with caller-chosen scratch (z: n FP64, sf: n FP32); used by
// the entry point that owns its scratch in a static device array.
vb_status spmv_lap_launch(cudaStream_t s, const vb_graph* g, const float* val, const double* S, float alpha,
                          const float* x, float beta, float* y, double* z, float* sf)
{
    lap_prep_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(x, S, g->n, z, sf);
    spmv_lap_kernel<<<kRowBlocks, kRowThreads, 0, s>>>(g->row_ptr, g->col, val, g->n, alpha, z, sf, beta, y);
    return last_launch();
}

size_t spmv_ws_bytes(int64_t n)
{
    Carve c(nullptr);
    c.take<double>(n);
    c.take<float>(n);
    return c.off;
}

vb_status spmv_run(Ctx* ctx, const vb_graph* g, const float* val, const double* S, int mode, float alpha,
                   const float* x, float beta, float* y, void* ws, size_t ws_bytes)
{
    if (!g || !g->row_ptr || !g->col || !val || !x || !y || x == y) return VB_ERR_ARG;
    if (mode == VB_SPMV_PLAIN) {
        spmv_plain_kernel<<<kRowBlocks, kRowThreads, 0, ctx->stream>>>(g->row_ptr, g->col, val, g->n, alpha, x, beta, y);
        ctx->launches += 1;
    } else if (mode == VB_SPMV_LAPLACIAN) {
        if (!S) return VB_ERR_ARG;
        Carve c(ws);
        double* z = c.take<double>(g->n);
        float* sf = c.take<float>(g->n);
        if (!ws || ws_bytes < c.off) return VB_ERR_WORKSPACE;
        lap_prep_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, ctx->stream>>>(x, S, g->n, z, sf);
        spmv_lap_kernel<<<kRowBlocks, kRowThreads, 0, ctx->stream>>>(g->row_ptr, g->col, val, g->n, alpha, z, sf, beta, y);
        ctx->launches += 2;
    } else {
        return VB_ERR_ARG;
    }
    return last_launch();
}

}  // namespace vb
