// Learned radius (step a7): a small MLP in -> 64 -> 64 -> 1 with GELU (erf form)
// that predicts log r_k, the log distance from a point to its k-th neighbour,
// from the point's coordinates.  The kNN search uses exp(prediction) as a
// per-point radius guess; the search stays exact whatever the guess.
//
// Forward passes read BF16 weights (a round-to-nearest copy of the FP32
// master) and compute in FP32.  Training: one thread per sample for the
// forward and the per-sample backward vectors; the weight gradients, sums of
// per-sample outer products, are formed block-wide from shared-memory copies of
// those vectors, written as per-block partials and reduced in a fixed order, so
// a training run is bitwise reproducible.  Adam updates the FP32 master and
// refreshes the BF16 copy.
#include "vb_internal.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

namespace vb {

constexpr int H = VB_MLP_HIDDEN;
constexpr int MT = 128;            // samples (threads) per training block pass
constexpr int MAXP = 64 * VB_MLP_MAX_IN + 4 * H + H * H + 1;
constexpr int PER_T = (MAXP + MT - 1) / MT;

__host__ __device__ inline int param_count(int in) { return H * in + H + H * H + H + H + 1; }

struct MlpK {
    int in;
    const __nv_bfloat16* wb;
    float mean[VB_MLP_MAX_IN], scale[VB_MLP_MAX_IN];
    float out_mean, out_scale;
};

static MlpK mk(const vb_mlp* m)
{
    MlpK k;
    k.in = m->in_dim;
    k.wb = (const __nv_bfloat16*)m->weights;
    for (int r = 0; r < VB_MLP_MAX_IN; ++r) {
        k.mean[r] = r < m->in_dim ? m->in_mean[r] : 0.f;
        k.scale[r] = r < m->in_dim && m->in_scale[r] != 0.f ? m->in_scale[r] : 1.f;
    }
    k.out_mean = m->out_mean;
    k.out_scale = m->out_scale != 0.f ? m->out_scale : 1.f;
    return k;
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// parameter offsets
struct Off {
    int w1, b1, w2, b2, w3, b3;
    __host__ __device__ explicit Off(int in)
    {
        w1 = 0;
        b1 = H * in;
        w2 = b1 + H;
        b2 = w2 + H * H;
        w3 = b2 + H;
        b3 = w3 + H;
    }
};

// Loads the BF16 weights into shared memory as FP32.
__device__ __forceinline__ void load_weights(const MlpK& k, float* W)
{
    const int P = param_count(k.in);
    for (int e = threadIdx.x; e < P; e += blockDim.x) W[e] = __bfloat162float(k.wb[e]);
}

// Forward pass of one standardised input; keeps z1 (pre-activations) and h1 for the backward.
__device__ __forceinline__ float forward(const MlpK& k, const float* W, const float* xin, float* z1, float* h1, float* z2)
{
    const Off o(k.in);
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
        float s = W[o.b1 + j];
        for (int r = 0; r < k.in; ++r) s = fmaf(W[o.w1 + j * k.in + r], xin[r], s);
        z1[j] = s;
        h1[j] = gelu(s);
    }
    float out = W[o.b3];
    for (int j = 0; j < H; ++j) {
        float s = W[o.b2 + j];
#pragma unroll 8
        for (int i = 0; i < H; ++i) s = fmaf(W[o.w2 + j * H + i], h1[i], s);
        z2[j] = s;
        out = fmaf(W[o.w3 + j], gelu(s), out);
    }
    return out;
}

__device__ __forceinline__ void standardise(const MlpK& k, const float* x, int ld, int64_t row, float* xin)
{
    for (int r = 0; r < k.in; ++r) xin[r] = (x[row * ld + r] - k.mean[r]) / k.scale[r];
}

// Forward pass for inference only: the hidden layer stays in registers and the second
// layer is folded into the output as it is formed (no per-sample arrays in local memory).
// The same operations in the same order as forward(), so the same bits.
__device__ __forceinline__ float forward_infer(const MlpK& k, const float* W, const float* xin)
{
    const Off o(k.in);
    float h1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float s = W[o.b1 + j];
        for (int r = 0; r < k.in; ++r) s = fmaf(W[o.w1 + j * k.in + r], xin[r], s);
        h1[j] = gelu(s);
    }
    float out = W[o.b3];
    for (int j = 0; j < H; ++j) {
        float s = W[o.b2 + j];
#pragma unroll
        for (int i = 0; i < H; ++i) s = fmaf(W[o.w2 + j * H + i], h1[i], s);
        out = fmaf(W[o.w3 + j], gelu(s), out);
    }
    return out;
}

// ------------------------------------------------------------------ inference
__global__ void __launch_bounds__(128) mlp_predict_kernel(MlpK k, const float* __restrict__ x, int ld, int64_t n,
                                                          float* y, int mode, float shift, float inflate,
                                                          const float* __restrict__ cloud_shift, Clouds cl)
{
    extern __shared__ float W[];
    load_weights(k, W);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float xin[VB_MLP_MAX_IN];
        standardise(k, x, ld, i, xin);
        const float logr = k.out_mean + k.out_scale * forward_infer(k, W, xin);
        if (mode == 0) {
            y[i] = logr;
        } else {   // squared radius bound for the radius-first kNN search
            const float sh = cloud_shift ? shift + cloud_shift[cloud_of(cl.ptr, cl.B, i)] : shift;
            const float r = expf(logr + sh) * inflate;
            y[i] = __fmul_ru(r, r);
        }
    }
}

// ------------------------------------------------------------------ training
// Per-block partial gradient over rows [r0, r1) of (x, y): part[blockIdx][P] and loss part[..][P].
// scale_g multiplies the gradient of sum_i (net(x_i) - y_std_i)^2 (1/batch for a mean).
__global__ void __launch_bounds__(MT) mlp_grad_kernel(MlpK k, const float* __restrict__ x, int ld,
                                                      const float* __restrict__ y, int64_t r0, int64_t r1,
                                                      int64_t n, float scale_g, float* part)
{
    extern __shared__ float sm[];
    const int P = param_count(k.in);
    float* W = sm;                       // P
    float* sh1 = W + P;                  // [MT][H]
    float* sdz2 = sh1 + MT * H;          // [MT][H]
    float* sdz1 = sdz2 + MT * H;         // [MT][H]
    float* sx = sdz1 + MT * H;           // [MT][in]
    float* sdo = sx + MT * VB_MLP_MAX_IN;   // [MT] d loss / d out
    __shared__ float sloss[MT];
    const Off o(k.in);
    load_weights(k, W);
    const int t = threadIdx.x;
    float acc[PER_T];
#pragma unroll
    for (int q = 0; q < PER_T; ++q) acc[q] = 0.f;
    float lsum = 0.f;
    const int64_t span = r1 - r0;
    const int64_t npass = (span + (int64_t)gridDim.x * MT - 1) / ((int64_t)gridDim.x * MT);
    __syncthreads();
    for (int64_t pass = 0; pass < npass; ++pass) {
        const int64_t rel = (pass * gridDim.x + blockIdx.x) * MT + t;
        const bool ok = rel < span;
        int64_t row = r0 + rel;
        if (row >= n) row -= n;   // windows may wrap around the end of the data
        float xin[VB_MLP_MAX_IN], z1[H], h1[H], z2[H];
        float dout = 0.f;
        if (ok) {
            standardise(k, x, ld, row, xin);
            const float out = forward(k, W, xin, z1, h1, z2);
            const float e = out - (y[row] - k.out_mean) / k.out_scale;
            lsum += e * e;
            dout = 2.f * e * scale_g;
        } else {
            for (int r = 0; r < k.in; ++r) xin[r] = 0.f;
            for (int j = 0; j < H; ++j) { z1[j] = 0.f; h1[j] = 0.f; z2[j] = 0.f; }
        }
        // backward vectors of this sample
        float dz2[H];
        for (int j = 0; j < H; ++j) dz2[j] = ok ? dout * W[o.w3 + j] * gelu_d(z2[j]) : 0.f;
        for (int i = 0; i < H; ++i) {
            float s = 0.f;
#pragma unroll 8
            for (int j = 0; j < H; ++j) s = fmaf(W[o.w2 + j * H + i], dz2[j], s);
            sdz1[t * H + i] = ok ? s * gelu_d(z1[i]) : 0.f;
            sh1[t * H + i] = h1[i];
            sdz2[t * H + i] = dz2[i];
        }
        for (int r = 0; r < k.in; ++r) sx[t * VB_MLP_MAX_IN + r] = xin[r];
        sdo[t] = dout;
        // h2 is needed for the w3 gradient: keep it in the z2 slot of sx-free storage via recompute
        for (int j = 0; j < H; ++j) z2[j] = ok ? gelu(z2[j]) : 0.f;
        __syncthreads();
        // each thread owns parameters e = t, t + MT, ...
#pragma unroll
        for (int q = 0; q < PER_T; ++q) {
            const int e = t + q * MT;
            if (e >= P) break;
            float s = 0.f;
            if (e < o.b1) {                      // W1[j][r]
                const int j = e / k.in, r = e - j * k.in;
                for (int u = 0; u < MT; ++u) s = fmaf(sdz1[u * H + j], sx[u * VB_MLP_MAX_IN + r], s);
            } else if (e < o.w2) {               // b1[j]
                const int j = e - o.b1;
                for (int u = 0; u < MT; ++u) s += sdz1[u * H + j];
            } else if (e < o.b2) {               // W2[j][i]
                const int j = (e - o.w2) / H, i = (e - o.w2) - j * H;
                for (int u = 0; u < MT; ++u) s = fmaf(sdz2[u * H + j], sh1[u * H + i], s);
            } else if (e < o.w3) {               // b2[j]
                const int j = e - o.b2;
                for (int u = 0; u < MT; ++u) s += sdz2[u * H + j];
            } else {
                s = 0.f;                          // w3, b3: from h2 and dout below
            }
            acc[q] += s;
        }
        __syncthreads();
        // w3[j] += dout h2[j], b3 += dout: h2 rows through shared memory (reuse sh1)
        for (int j = 0; j < H; ++j) sh1[t * H + j] = z2[j];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER_T; ++q) {
            const int e = t + q * MT;
            if (e < o.w3 || e >= P) continue;
            float s = 0.f;
            if (e < o.b3) {
                const int j = e - o.w3;
                for (int u = 0; u < MT; ++u) s = fmaf(sdo[u], sh1[u * H + j], s);
            } else {
                for (int u = 0; u < MT; ++u) s += sdo[u];
            }
            acc[q] += s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PER_T; ++q) {
        const int e = t + q * MT;
        if (e < P) part[(int64_t)blockIdx.x * (P + 1) + e] = acc[q];
    }
    sloss[t] = lsum;
    __syncthreads();
    if (t == 0) {
        float s = 0.f;
        for (int u = 0; u < MT; ++u) s += sloss[u];
        part[(int64_t)blockIdx.x * (P + 1) + P] = s;
    }
}

// grad[e] = sum over blocks (fixed order); loss = sum / count
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int nblk, int P, float* grad, float* loss,
                                  float inv_count)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e > P) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += (double)part[(int64_t)b * (P + 1) + e];
    if (e < P) grad[e] = (float)s;
    else if (loss) *loss = (float)(s * inv_count);
}

__global__ void mlp_adam_kernel(float* master, __nv_bfloat16* wb, float* m1, float* m2, const float* __restrict__ g,
                                int P, float lr, float bc1, float bc2)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P) return;
    const float ge = g[e];
    const float a = 0.9f * m1[e] + 0.1f * ge;
    const float b = 0.999f * m2[e] + 0.001f * ge * ge;
    m1[e] = a;
    m2[e] = b;
    const float w = master[e] - lr * (a / bc1) / (sqrtf(b / bc2) + 1e-8f);
    master[e] = w;
    wb[e] = __float2bfloat16_rn(w);
}

__global__ void mlp_init_kernel(float* master, __nv_bfloat16* wb, float* m1, float* m2, int in, uint64_t seed)
{
    const int P = param_count(in);
    const Off o(in);
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P) return;
    float sd = 0.f;
    if (e < o.b1) sd = sqrtf(2.f / (float)in);
    else if (e >= o.w2 && e < o.b2) sd = sqrtf(2.f / (float)H);
    else if (e >= o.w3 && e < o.b3) sd = sqrtf(1.f / (float)H);
    // Box-Muller on two counter-based uniforms (splitmix64)
    auto u01 = [&](uint64_t c) {
        uint64_t x = seed + 0x9E3779B97F4A7C15ull * (c + 1);
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    const double u1 = u01(2 * (uint64_t)e), u2 = u01(2 * (uint64_t)e + 1);
    const float z = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    const float w = sd * z;
    master[e] = w;
    wb[e] = __float2bfloat16_rn(w);
    m1[e] = 0.f;
    m2[e] = 0.f;
}

// ------------------------------------------------------------------ host wrappers
static size_t grad_smem(int in) { return sizeof(float) * ((size_t)param_count(in) + 3 * MT * H + MT * VB_MLP_MAX_IN + MT); }
static size_t pred_smem(int in) { return sizeof(float) * (size_t)param_count(in); }
constexpr int GRAD_BLOCKS = 152;

static vb_status set_attrs(int dev)
{
    static bool done[16] = {};
    if (done[dev & 15]) return VB_OK;
    if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)grad_smem(VB_MLP_MAX_IN)) != cudaSuccess)
        return VB_ERR_CUDA;
    done[dev & 15] = true;
    return VB_OK;
}

size_t mlp_ws_bytes(int in, int64_t)
{
    Carve c(nullptr);
    c.take<float>((size_t)GRAD_BLOCKS * (param_count(in) + 1));
    c.take<float>(param_count(in));
    return c.off;
}

static vb_status grad_run(Ctx* ctx, const vb_mlp* m, const float* x, int ld, const float* y, int64_t n, int64_t r0,
                          int64_t r1, float scale_g, float* grad, float* loss, float inv_count, void* ws,
                          size_t ws_bytes, int nblk)
{
    Carve c(ws);
    float* part = c.take<float>((size_t)GRAD_BLOCKS * (param_count(m->in_dim) + 1));
    if (!ws || ws_bytes < c.off) return VB_ERR_WORKSPACE;
    vb_status st = set_attrs(ctx->device);
    if (st != VB_OK) return st;
    const int P = param_count(m->in_dim);
    mlp_grad_kernel<<<nblk, MT, grad_smem(m->in_dim), ctx->stream>>>(mk(m), x, ld, y, r0, r1, n, scale_g, part);
    mlp_reduce_kernel<<<(P + 1 + 255) / 256, 256, 0, ctx->stream>>>(part, nblk, P, grad, loss, inv_count);
    ctx->launches += 2;
    return last_launch();
}

// ------------------------------------------------------------------ inference on the tensor cores
// The radius guesses of the kNN search: 128 samples per step, one thread and one tensor-memory
// lane per sample.  Layer 1 is one tcgen05.mma (M = 128 samples, N = 64 hidden units, K = 16:
// the standardised inputs, zero-padded) and layer 2 four (K = 64), both BF16 x BF16 with FP32
// accumulation in tensor memory; biases, GELU and the output layer run in FP32 on the values
// read back with tcgen05.ld.  Weights (BF16) stay in shared memory as the B operands.  The
// activations are rounded to BF16 where the FP32 forward keeps them in FP32, a relative change
// of about 2^-9 that only moves a radius guess (the search stays exact for any guess).
constexpr int MI = 128;   // samples per step
constexpr uint32_t MLP_TMEM_COLS = 128;   // D1 in columns [0, 64), D2 in [64, 128)
constexpr size_t MI_A1 = MI * 16 * 2, MI_B1 = H * 16 * 2, MI_A2 = MI * H * 2, MI_B2 = H * H * 2;
constexpr size_t MI_SMEM = MI_A1 + MI_B1 + MI_A2 + MI_B2 + 3 * H * sizeof(float) + 16;

__global__ void __launch_bounds__(MI) mlp_radius_tc_kernel(MlpK k, const float* __restrict__ xs, int ld, int64_t n,
                                                           float* r2, int mode, float shift, float inflate,
                                                           const float* __restrict__ cloud_shift, Clouds cl,
                                                           DevReport* rep)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __nv_bfloat16* a1 = (__nv_bfloat16*)smem;
    __nv_bfloat16* b1w = (__nv_bfloat16*)(smem + MI_A1);
    __nv_bfloat16* a2 = (__nv_bfloat16*)(smem + MI_A1 + MI_B1);
    __nv_bfloat16* b2w = (__nv_bfloat16*)(smem + MI_A1 + MI_B1 + MI_A2);
    float* bias1 = (float*)(smem + MI_A1 + MI_B1 + MI_A2 + MI_B2);
    float* bias2 = bias1 + H;
    float* w3 = bias2 + H;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int t = threadIdx.x, warp = t >> 5;
    const Off o(k.in);
    // B operands: row j (hidden unit) holds its input weights along K
    for (int e = t; e < H * 16; e += MI) {
        const int j = e / 16, r = e % 16;
        const __nv_bfloat16 v = r < k.in ? k.wb[o.w1 + j * k.in + r] : __float2bfloat16_rn(0.f);
        *(__nv_bfloat16*)((char*)b1w + tc::operand_offset(j, r, 16)) = v;
    }
    for (int e = t; e < H * H; e += MI) {
        const int j = e / H, i = e % H;
        *(__nv_bfloat16*)((char*)b2w + tc::operand_offset(j, i, H)) = k.wb[o.w2 + j * H + i];
    }
    for (int j = t; j < H; j += MI) {
        bias1[j] = __bfloat162float(k.wb[o.b1 + j]);
        bias2[j] = __bfloat162float(k.wb[o.b2 + j]);
        w3[j] = __bfloat162float(k.wb[o.w3 + j]);
    }
    const float b3 = __bfloat162float(k.wb[o.b3]);
    if (warp == 0) tc::tmem_alloc(&tmem_base, MLP_TMEM_COLS);
    if (t == 0) { tc::mbar_init(&bar, 1); s_abort = 0; }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    const uint32_t lane_addr = tb + ((uint32_t)(warp * 32) << 16);
    constexpr uint32_t idesc = tc::idesc_bf16(MI, H);
    uint32_t phase = 0;
    for (int64_t base = (int64_t)blockIdx.x * MI; base < n; base += (int64_t)gridDim.x * MI) {
        const int64_t i = base + t;
        const bool valid = i < n;
        // layer-1 operand: the standardised inputs of this thread's sample, K padded to 16
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            uint16_t v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int r = 8 * c + e;
                const float xv = valid && r < k.in ? (xs[i * ld + r] - k.mean[r]) / k.scale[r] : 0.f;
                v[e] = __bfloat16_as_ushort(__float2bfloat16_rn(xv));
            }
            *(uint4*)((char*)a1 + tc::operand_offset(t, 8 * c, 16)) = tc::pack8(v);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
            tc::mma_bf16(tb, tc::smem_desc(tc::smem_addr(a1), 128, 256), tc::smem_desc(tc::smem_addr(b1w), 128, 256),
                         idesc, 0u);
            tc::mma_commit(&bar);
        }
        bool done = tc::mbar_wait(&bar, phase);
        phase ^= 1u;
        tc::fence_after_sync();
        if (__syncthreads_or(!done)) {
            if (t == 0) { report_error(rep, VB_ERR_TIMEOUT); s_abort = 1; }
            break;
        }
        {
            float z[H];
            tc::tmem_ld64(lane_addr, z);
#pragma unroll
            for (int c = 0; c < H / 8; ++c) {
                uint16_t v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    v[e] = __bfloat16_as_ushort(__float2bfloat16_rn(gelu(z[8 * c + e] + bias1[8 * c + e])));
                *(uint4*)((char*)a2 + tc::operand_offset(t, 8 * c, H)) = tc::pack8(v);
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
#pragma unroll
            for (int sk = 0; sk < H / 16; ++sk)
                tc::mma_bf16(tb + 64, tc::smem_desc(tc::smem_addr(a2) + sk * 256, 128, (H / 8) * 128),
                             tc::smem_desc(tc::smem_addr(b2w) + sk * 256, 128, (H / 8) * 128), idesc, sk > 0 ? 1u : 0u);
            tc::mma_commit(&bar);
        }
        done = tc::mbar_wait(&bar, phase);
        phase ^= 1u;
        tc::fence_after_sync();
        if (__syncthreads_or(!done)) {
            if (t == 0) { report_error(rep, VB_ERR_TIMEOUT); s_abort = 1; }
            break;
        }
        float z[H];
        tc::tmem_ld64(lane_addr + 64, z);
        float out = b3;
#pragma unroll
        for (int j = 0; j < H; ++j) out = fmaf(w3[j], gelu(z[j] + bias2[j]), out);
        if (valid) {
            const float logr = k.out_mean + k.out_scale * out;
            if (mode == 0) {
                r2[i] = logr;
            } else {   // squared radius bound for the radius-first kNN search
                const float sh = cloud_shift ? shift + cloud_shift[cloud_of(cl.ptr, cl.B, i)] : shift;
                const float r = expf(logr + sh) * inflate;
                r2[i] = __fmul_ru(r, r);
            }
        }
        tc::fence_before_sync();
        __syncthreads();   // the operands of the next step overwrite these only after every read
    }
    if (s_abort) {   // a bounded wait ran out: no further step was issued; the tensor memory goes back
        tc::fence_before_sync();
    }
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tb, MLP_TMEM_COLS);
}

static vb_status mlp_tc_launch(cudaStream_t s, const vb_mlp* mlp, const float* xs, int ld, int64_t n, float* out,
                               int mode, float shift, float inflate, const float* cloud_shift, Clouds cl,
                               DevReport* rep)
{
    static bool attr[16] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr[dev & 15]) {
        if (cudaFuncSetAttribute(mlp_radius_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MI_SMEM + 1024) !=
            cudaSuccess)
            return VB_ERR_CUDA;
        attr[dev & 15] = true;
    }
    // 4 CTAs per SM (128 tensor-memory columns each), persistent over the sample tiles
    const int64_t tiles = (n + MI - 1) / MI;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, 152 * 4);
    mlp_radius_tc_kernel<<<grid, MI, MI_SMEM + 1024, s>>>(mk(mlp), xs, ld, n, out, mode, shift, inflate, cloud_shift,
                                                          cl, rep);
    return last_launch();
}

vb_status mlp_radius_r2(cudaStream_t s, const vb_mlp* mlp, const float* xs, int64_t n, int m, int mp, float shift,
                        float inflate, float* r2, const float* cloud_shift, Clouds cl, DevReport* rep)
{
    if (!mlp || mlp->in_dim < 1 || mlp->in_dim > VB_MLP_MAX_IN || mlp->in_dim > m || !mlp->weights) return VB_ERR_ARG;
    return mlp_tc_launch(s, mlp, xs, mp, n, r2, 1, shift, inflate, cloud_shift, cl, rep);
}

}  // namespace vb

using namespace vb;

namespace vb {

// Column c of the inputs (c < in) or the targets (c == in): mean and sample standard deviation
// (n - 1), FP64 partials per thread over a fixed stride, then a fixed tree; one block per column.
constexpr int STD_T = 1024;
__global__ void __launch_bounds__(STD_T) mlp_moments_kernel(const float* __restrict__ x, int ld, const float* __restrict__ y,
                                                            int64_t n, int in, double* out)
{
    __shared__ double s1[STD_T], s2[STD_T];
    const int c = blockIdx.x, t = threadIdx.x;
    // shifted by the first value, so that a column far from zero keeps its variance
    const double ref = c < in ? (double)x[c] : (double)y[0];
    double a = 0.0, b = 0.0;
    for (int64_t i = t; i < n; i += STD_T) {
        const double v = (c < in ? (double)x[i * ld + c] : (double)y[i]) - ref;
        a += v;
        b += v * v;
    }
    s1[t] = a;
    s2[t] = b;
    __syncthreads();
    for (int w = STD_T / 2; w > 0; w >>= 1) {
        if (t < w) {
            s1[t] += s1[t + w];
            s2[t] += s2[t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        const double mean_s = s1[0] / (double)n;
        const double var = n > 1 ? (s2[0] - s1[0] * mean_s) / (double)(n - 1) : 0.0;
        out[2 * c] = ref + mean_s;
        out[2 * c + 1] = sqrt(fmax(var, 0.0));
    }
}

}  // namespace vb

extern "C" {

int64_t vb_mlp_param_count(int32_t in_dim) { return param_count(in_dim); }

vb_status vb_mlp_standardise(vb_ctx* ctx, vb_mlp* m, const float* x, int32_t ld, const float* y, int64_t n, void* ws,
                             size_t ws_bytes)
{
    if (!ctx || !m || !x || !y || n < 1 || ld < m->in_dim || m->in_dim < 1 || m->in_dim > VB_MLP_MAX_IN)
        return VB_ERR_ARG;
    const int in = m->in_dim;
    if (!ws || ws_bytes < sizeof(double) * 2 * (VB_MLP_MAX_IN + 1)) return VB_ERR_WORKSPACE;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    double* out = (double*)ws;
    mlp_moments_kernel<<<in + 1, STD_T, 0, c->stream>>>(x, ld, y, n, in, out);
    c->launches += 1;
    vb_status st = last_launch();
    if (st != VB_OK) return st;
    double h[2 * (VB_MLP_MAX_IN + 1)];
    if (cudaMemcpyAsync(h, out, sizeof(double) * 2 * (in + 1), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return VB_ERR_CUDA;
    for (int r = 0; r < in; ++r) {
        m->in_mean[r] = (float)h[2 * r];
        m->in_scale[r] = (float)std::max(h[2 * r + 1], 1e-12);
    }
    m->out_mean = (float)h[2 * in];
    m->out_scale = (float)std::max(h[2 * in + 1], 1e-12);
    return VB_OK;
}

size_t vb_mlp_workspace(int32_t in_dim, int64_t batch) { return mlp_ws_bytes(in_dim, batch); }

vb_status vb_mlp_init(vb_ctx* ctx, vb_mlp* m, uint64_t seed)
{
    if (!ctx || !m || m->in_dim < 1 || m->in_dim > VB_MLP_MAX_IN || !m->master || !m->weights || !m->adam_m ||
        !m->adam_v)
        return VB_ERR_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    const int P = param_count(m->in_dim);
    mlp_init_kernel<<<(P + 255) / 256, 256, 0, c->stream>>>(m->master, (__nv_bfloat16*)m->weights, m->adam_m,
                                                            m->adam_v, m->in_dim, seed);
    m->step = 0;
    c->launches += 1;
    return last_launch();
}

vb_status vb_mlp_gradient(vb_ctx* ctx, const vb_mlp* m, const float* x, int32_t ld, const float* y, int64_t n,
                          float* grad, float* loss_dev, void* ws, size_t ws_bytes)
{
    if (!ctx || !m || !x || !y || !grad || n < 1 || ld < m->in_dim || m->in_dim < 1 || m->in_dim > VB_MLP_MAX_IN)
        return VB_ERR_ARG;
    return grad_run(reinterpret_cast<Ctx*>(ctx), m, x, ld, y, n, 0, n, 1.f / (float)n, grad, loss_dev,
                    1.f / (float)n, ws, ws_bytes, GRAD_BLOCKS);
}

vb_status vb_mlp_train_epoch(vb_ctx* ctx, vb_mlp* m, const float* x, int32_t ld, const float* y, int64_t n,
                             int32_t batch, float lr, uint64_t seed, float* loss_dev, void* ws, size_t ws_bytes)
{
    if (!ctx || !m || !x || !y || n < 1 || batch < 1 || ld < m->in_dim || m->in_dim < 1 ||
        m->in_dim > VB_MLP_MAX_IN || !(lr > 0.f))
        return VB_ERR_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Carve cv(ws);
    cv.take<float>((size_t)GRAD_BLOCKS * (param_count(m->in_dim) + 1));
    float* grad = cv.take<float>(param_count(m->in_dim));
    if (!ws || ws_bytes < cv.off) return VB_ERR_WORKSPACE;
    const int P = param_count(m->in_dim);
    const int64_t nb = (n + batch - 1) / batch;
    const int64_t first = (int64_t)(seed % (uint64_t)nb);
    const int nblk = (int)std::min<int64_t>(GRAD_BLOCKS, (batch + MT - 1) / MT);
    if (loss_dev && cudaMemsetAsync(loss_dev, 0, sizeof(float), c->stream) != cudaSuccess) return VB_ERR_CUDA;
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t r0 = ((first + b) % nb) * batch;
        const int64_t r1 = std::min<int64_t>(r0 + batch, n);
        vb_status st = grad_run(c, m, x, ld, y, n, r0, r1, 1.f / (float)(r1 - r0), grad, b == nb - 1 ? loss_dev : nullptr,
                                1.f / (float)(r1 - r0), ws, ws_bytes, nblk);
        if (st != VB_OK) return st;
        m->step += 1;
        const float bc1 = 1.f - (float)std::pow(0.9, (double)m->step);
        const float bc2 = 1.f - (float)std::pow(0.999, (double)m->step);
        mlp_adam_kernel<<<(P + 255) / 256, 256, 0, c->stream>>>(m->master, (__nv_bfloat16*)m->weights, m->adam_m,
                                                                m->adam_v, grad, P, lr, bc1, bc2);
        c->launches += 1;
        if ((st = last_launch()) != VB_OK) return st;
    }
    return VB_OK;
}

vb_status vb_mlp_predict_tc(vb_ctx* ctx, const vb_mlp* m, const float* x, int32_t ld, int64_t n, float* y)
{
    if (!ctx || !m || !x || !y || n < 1 || ld < m->in_dim || m->in_dim < 1 || m->in_dim > VB_MLP_MAX_IN)
        return VB_ERR_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    c->launches += 1;
    return mlp_tc_launch(c->stream, m, x, ld, n, y, 0, 0.f, 1.f, nullptr, Clouds(), c->rep);
}

vb_status vb_mlp_predict(vb_ctx* ctx, const vb_mlp* m, const float* x, int32_t ld, int64_t n, float* y)
{
    if (!ctx || !m || !x || !y || n < 1 || ld < m->in_dim || m->in_dim < 1 || m->in_dim > VB_MLP_MAX_IN)
        return VB_ERR_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    mlp_predict_kernel<<<152 * 4, 128, pred_smem(m->in_dim), c->stream>>>(mk(m), x, ld, n, y, 0, 0.f, 1.f,
                                                                               nullptr, Clouds());
    c->launches += 1;
    return last_launch();
}

}  // extern "C"
