// The paper's delta_tol sparsity pattern (Algorithm 1 and Sec. 4, "Computing the kernel
// matrix with a k-d tree"): an entry (i, j) of a kernel matrix
//     K^ij = exp(-||x_i - x_j||^2 / (eps^2 rho_i rho_j))
// is kept only where it exceeds delta_tol.  The test is taken as t_ij < tau with
// t_ij = d2_ij / (eps^2 (rho_i rho_j)) (the product rho_i rho_j first, so t_ij = t_ji bit
// for bit) and tau = -log(delta_tol) computed once in FP64: exp is decreasing, and the
// threshold form is one that two implementations can evaluate identically.  d2 is the
// canonical FP64 squared distance of the kNN search (RN differences and squares summed in
// coordinate order), and the diagonal is kept (t = 0).
//
// The search reuses the kNN search's spatial order: points in Morton order, 64-point tiles
// with boxes.  A candidate tile is skipped for a query tile when even the nearest points of
// the two boxes, with the largest rho of each tile, give t >= tau (the FP64 box gap is a
// lower bound of every canonical distance between the boxes, and every step of t is
// monotone under round-to-nearest), which is the paper's critical-radius ball with a
// per-tile bandwidth.  Pairs are tested one by one in FP64.
//
// vb_radius_sweep sums Eq. (bandwidth sensitivity) with the pattern of every grid point:
// chi_xi = sum over (i, j) with t_ij / 2^xi < tau of exp(-t_ij / 2^xi), t with scale in place
// of eps^2, 2^xi from the host's pow (the values every FP64 implementation of the grid gets).
#include "vb_internal.cuh"

#include <cmath>

namespace vb {

constexpr int RQ = 64;           // queries (threads) per query tile
constexpr int RSORT_MAX = 2048;  // longest row the in-block column sort takes
constexpr int RSORT_T = 256;

struct GridVals {
    double v[kMaxGrid];          // 2^xi_g
};

__global__ void tile_rho_kernel(const double* __restrict__ rho, const uint32_t* __restrict__ perm, int64_t n,
                                int64_t ntiles, double* trho)
{
    const int64_t ct = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ct >= ntiles) return;
    double mx = 0.0;
    for (int64_t p = ct * RQ; p < min(n, (ct + 1) * RQ); ++p) mx = fmax(mx, rho[perm[p]]);
    trho[ct] = mx;
}

// Lower bound of t over the pairs of tiles qt and ct: FP64 box gaps squared and summed in
// coordinate order, over eps2 (rho_max(qt) rho_max(ct)).
__device__ __forceinline__ double tile_t_lb(const PointOrder& o, int m, int64_t qt, int64_t ct, const double* trho,
                                            double eps2)
{
    double acc = 0.0;
    for (int r = 0; r < m; ++r) {
        const double ql = o.tlo[qt * o.mp + r], qh = o.thi[qt * o.mp + r];
        const double cl = o.tlo[ct * o.mp + r], ch = o.thi[ct * o.mp + r];
        const double g = fmax(fmax(__dsub_rn(cl, qh), __dsub_rn(ql, ch)), 0.0);
        const double s = __dmul_rn(g, g);
        acc = r == 0 ? s : __dadd_rn(acc, s);
    }
    return __ddiv_rn(acc, __dmul_rn(eps2, __dmul_rn(trho[qt], trho[ct])));
}

__device__ __forceinline__ double canon_d2_rows(const double* __restrict__ a, const double* __restrict__ b, int m)
{
    double acc = 0.0;
    for (int r = 0; r < m; ++r) {
        const double dl = __dsub_rn(a[r], b[r]);
        const double s = __dmul_rn(dl, dl);
        acc = r == 0 ? s : __dadd_rn(acc, s);
    }
    return acc;
}

enum RadiusMode { kCount = 0, kFill = 1, kSweep = 2 };

// One query tile per block iteration, one query per thread.  kCount: entries per row
// (original order).  kFill: the row's entries (original column, canonical d2) at row_ptr
// (unsorted).  kSweep: per-block sums of exp(-t / 2^xi_g) over the kept pairs of every
// grid point, into part[block][G].
template <int MODE>
__global__ void __launch_bounds__(RQ) radius_pass_kernel(PointOrder o, int64_t n, int m,
                                                         const double* __restrict__ rho,
                                                         const double* __restrict__ trho, double eps2, double tau,
                                                         int32_t* count, const int64_t* __restrict__ row_ptr,
                                                         int64_t cap, int32_t* col, double* d2out, GridVals gv, int G,
                                                         double* part, DevReport* rep)
{
    __shared__ double acc[MODE == kSweep ? kMaxGrid * RQ : 1];
    const int t = threadIdx.x;
    if constexpr (MODE == kSweep)
        for (int g = 0; g < G; ++g) acc[g * RQ + t] = 0.0;
    if constexpr (MODE == kFill) {
        if (row_ptr[n] > cap) {   // the caller's arrays cannot hold the pattern
            if (blockIdx.x == 0 && t == 0) report_error(rep, VB_ERR_WORKSPACE);
            return;
        }
    }
    // a tile pair is skipped when its lower bound fails the test (at the largest grid point for a
    // sweep: t / 2^xi only grows as xi falls); every step is monotone, so no kept pair is lost
    const double gdiv = MODE == kSweep ? gv.v[G - 1] : 1.0;
    for (int64_t qt = blockIdx.x; qt < o.ntiles; qt += gridDim.x) {
        const int64_t p = qt * RQ + t;
        const bool valid = p < n;
        const uint32_t oi = valid ? o.perm[p] : 0u;
        const double ri = valid ? rho[oi] : 0.0;
        const double* q = o.xs64 + (valid ? p : 0) * o.mp;
        int32_t cnt = 0;
        int64_t wpos = MODE == kFill && valid ? row_ptr[oi] : 0;
        for (int64_t ct = 0; ct < o.ntiles; ++ct) {
            if (!(__ddiv_rn(tile_t_lb(o, m, qt, ct, trho, eps2), gdiv) < tau)) continue;   // uniform over the block
            if (!valid) continue;
            const int64_t c1 = min(n, (ct + 1) * RQ);
            for (int64_t cp = ct * RQ; cp < c1; ++cp) {
                const uint32_t oj = o.perm[cp];
                const double d2 = canon_d2_rows(q, o.xs64 + cp * o.mp, m);
                const double tij = __ddiv_rn(d2, __dmul_rn(eps2, __dmul_rn(ri, rho[oj])));
                if constexpr (MODE == kSweep) {
                    for (int g = 0; g < G; ++g) {
                        const double u = __ddiv_rn(tij, gv.v[g]);
                        if (u < tau) acc[g * RQ + t] += exp(-u);
                    }
                } else if (tij < tau) {
                    if constexpr (MODE == kFill) {
                        col[wpos] = (int32_t)oj;
                        d2out[wpos] = d2;
                        ++wpos;
                    } else {
                        ++cnt;
                    }
                }
            }
        }
        if constexpr (MODE == kCount)
            if (valid) count[oi] = cnt;
    }
    if constexpr (MODE == kSweep) {
        __syncthreads();
        if (t < G) {   // the block's sum of grid point t, over its threads in a fixed order
            double s = 0.0;
            for (int u = 0; u < RQ; ++u) s += acc[t * RQ + u];
            part[(int64_t)blockIdx.x * G + t] = s;
        }
    }
}

__global__ void nnz_copy_kernel(const int64_t* __restrict__ row_ptr, int64_t n, int64_t* nnz)
{
    *nnz = row_ptr[n];
}

// Sorts every row's entries by column (block-wide bitonic sort in shared memory; rows
// longer than RSORT_MAX are reported as unsupported and left unsorted).
__global__ void __launch_bounds__(RSORT_T) row_sort_kernel(const int64_t* __restrict__ row_ptr, int64_t n, int64_t cap,
                                                           int32_t* col, double* d2, DevReport* rep)
{
    __shared__ int32_t kc[RSORT_MAX];
    __shared__ double kd[RSORT_MAX];
    if (row_ptr[n] > cap) return;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t rb = row_ptr[i], len = row_ptr[i + 1] - rb;
        if (len <= 1) continue;
        if (len > RSORT_MAX) {
            if (threadIdx.x == 0) report_error(rep, VB_ERR_UNSUPPORTED);
            continue;
        }
        int P = 1;
        while (P < len) P <<= 1;
        for (int e = threadIdx.x; e < P; e += RSORT_T) {
            kc[e] = e < len ? col[rb + e] : INT32_MAX;
            kd[e] = e < len ? d2[rb + e] : 0.0;
        }
        __syncthreads();
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int e = threadIdx.x; e < P / 2; e += RSORT_T) {
                    const int lo = 2 * e - (e & (stride - 1)), hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    if ((kc[lo] > kc[hi]) == up) {
                        const int32_t c = kc[lo];
                        kc[lo] = kc[hi];
                        kc[hi] = c;
                        const double d = kd[lo];
                        kd[lo] = kd[hi];
                        kd[hi] = d;
                    }
                }
                __syncthreads();
            }
        }
        for (int e = threadIdx.x; e < len; e += RSORT_T) {
            col[rb + e] = kc[e];
            d2[rb + e] = kd[e];
        }
        __syncthreads();
    }
}

// chi_g = sum of the block partials in block order; chi'_g forward differences; the first
// maximiser gives eps^2 = 2^xi (the host's value) and the dimension 2 chi'.
__global__ void radius_sweep_finish_kernel(const double* __restrict__ part, int nblk, int G, GridVals gv, double dxi,
                                           double* chi, double* eps2, double* dim)
{
    __shared__ double c[kMaxGrid];
    const int g = threadIdx.x;
    if (g < G) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * G + g];
        c[g] = s;
        chi[g] = s;
    }
    __syncthreads();
    if (g == 0) {
        int best = 0;
        double bv = -INFINITY;
        for (int h = 0; h + 1 < G; ++h) {
            const double cp = (log(c[h + 1]) - log(c[h])) / (dxi * 0.6931471805599453);
            if (cp > bv) { bv = cp; best = h; }
        }
        *eps2 = gv.v[best];
        *dim = 2.0 * bv;
    }
}

constexpr int kRadiusBlocks = 152 * 8;

static size_t radius_ws(int64_t n, int32_t m, int G)
{
    Carve c(nullptr);
    c.take<unsigned char>(order_ws_bytes(n, m));
    c.take<double>((n + RQ - 1) / RQ);           // per-tile rho max
    c.take<int32_t>(n);                          // row counts
    c.take<double>((size_t)kRadiusBlocks * G);   // sweep partials
    c.take<unsigned char>(scan_ws_bytes(n));
    return c.off;
}

size_t radius_ws_bytes(int64_t n, int32_t m) { return radius_ws(n, m, kMaxGrid); }

struct RadiusWs {
    PointOrder o;
    double* trho;
    int32_t* count;
    double* part;
    void* scan;
};

static vb_status radius_setup(Ctx* ctx, const float* x, int64_t n, int32_t m, const double* rho, void* ws,
                              size_t ws_bytes, RadiusWs* r)
{
    Carve c(ws);
    void* ows = c.take<unsigned char>(order_ws_bytes(n, m));
    r->trho = c.take<double>((n + RQ - 1) / RQ);
    r->count = c.take<int32_t>(n);
    r->part = c.take<double>((size_t)kRadiusBlocks * kMaxGrid);
    r->scan = c.take<unsigned char>(scan_ws_bytes(n));
    if (!ws || ws_bytes < c.off) return VB_ERR_WORKSPACE;
    vb_status st = order_run(ctx, x, n, m, ows, order_ws_bytes(n, m), &r->o);
    if (st != VB_OK) return st;
    tile_rho_kernel<<<(unsigned)((r->o.ntiles + 255) / 256), 256, 0, ctx->stream>>>(rho, r->o.perm, n, r->o.ntiles,
                                                                                  r->trho);
    ctx->launches += 1;
    return last_launch();
}

vb_status radius_pattern_run(Ctx* ctx, const float* x, int64_t n, int32_t m, const double* rho, double eps2,
                             double delta_tol, int64_t* row_ptr, int32_t* col, double* d2, int64_t cap,
                             int64_t* nnz_dev, void* ws, size_t ws_bytes)
{
    if (!x || !rho || !row_ptr || !col || !d2 || !nnz_dev || n < 1 || m < 1 || m > 128 || cap < n) return VB_ERR_ARG;
    if (!(eps2 > 0) || !(delta_tol > 0 && delta_tol < 1)) return VB_ERR_ARG;
    RadiusWs r;
    vb_status st = radius_setup(ctx, x, n, m, rho, ws, ws_bytes, &r);
    if (st != VB_OK) return st;
    const double tau = -std::log(delta_tol);
    cudaStream_t s = ctx->stream;
    const unsigned grid = (unsigned)std::min<int64_t>(r.o.ntiles, kRadiusBlocks);
    GridVals gv = {};
    radius_pass_kernel<kCount><<<grid, RQ, 0, s>>>(r.o, n, m, rho, r.trho, eps2, tau, r.count, nullptr, cap, nullptr,
                                                   nullptr, gv, 0, nullptr, ctx->rep);
    st = scan_counts(s, r.count, n, row_ptr, r.scan);
    if (st != VB_OK) return st;
    radius_pass_kernel<kFill><<<grid, RQ, 0, s>>>(r.o, n, m, rho, r.trho, eps2, tau, nullptr, row_ptr, cap, col, d2,
                                                  gv, 0, nullptr, ctx->rep);
    row_sort_kernel<<<kRadiusBlocks, RSORT_T, 0, s>>>(row_ptr, n, cap, col, d2, ctx->rep);
    nnz_copy_kernel<<<1, 1, 0, s>>>(row_ptr, n, nnz_dev);
    ctx->launches += 5;
    return last_launch();
}

vb_status radius_sweep_run(Ctx* ctx, const float* x, int64_t n, int32_t m, const double* rho, double scale,
                           double xi_lo, double xi_hi, double dxi, double delta_tol, double* chi, double* eps2,
                           double* dim, void* ws, size_t ws_bytes)
{
    if (!x || !rho || !chi || !eps2 || !dim || n < 2 || m < 1 || m > 128) return VB_ERR_ARG;
    if (!(scale > 0) || !(delta_tol > 0 && delta_tol < 1) || !(dxi > 0) || !(xi_hi > xi_lo)) return VB_ERR_ARG;
    const int G = (int)std::lround((xi_hi - xi_lo) / dxi) + 1;
    if (G < 2 || G > kMaxGrid) return VB_ERR_ARG;
    RadiusWs r;
    vb_status st = radius_setup(ctx, x, n, m, rho, ws, ws_bytes, &r);
    if (st != VB_OK) return st;
    GridVals gv = {};
    for (int g = 0; g < G; ++g) gv.v[g] = std::pow(2.0, xi_lo + dxi * (double)g);
    const double tau = -std::log(delta_tol);
    cudaStream_t s = ctx->stream;
    const unsigned grid = (unsigned)std::min<int64_t>(r.o.ntiles, kRadiusBlocks);
    radius_pass_kernel<kSweep><<<grid, RQ, 0, s>>>(r.o, n, m, rho, r.trho, scale, tau, nullptr, nullptr, 0, nullptr,
                                                   nullptr, gv, G, r.part, ctx->rep);
    radius_sweep_finish_kernel<<<1, kMaxGrid, 0, s>>>(r.part, (int)grid, G, gv, dxi, chi, eps2, dim);
    ctx->launches += 2;
    return last_launch();
}

}  // namespace vb
