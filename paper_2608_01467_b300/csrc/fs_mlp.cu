// Learned pruning at the checkpoint boundary: a 16 -> 128 -> 128 -> 1 MLP
// (ReLU) that scores checkpoint-table entries (partial histories after the
// prefix of Algorithm 2) by the predicted log10 |exact subtree sum|; entries
// scoring below a threshold tau are cut, the rest are enumerated exactly.
//
// Numerics: BF16 operands on the tensor cores with FP32 accumulation;
// FP32 master weights and Adam state.  Scoring (forward, learned pruning)
// runs on tcgen05.mma with the accumulators in tensor memory; training
// (forward + backward on minibatches, off the amplitude path) uses
// mma.sync m16n8k16.  Rounded to BF16: the inputs X, W1, W2, w3, the hidden
// activation h1 (layer-2 operand) and, in the backward pass, the GEMM
// operands dh2 and dh1.  Everything else is FP32.
//
// Parameter layout (FP32, 18817 values): W1[16][128] at 0, b1[128] at 2048,
// W2[128][128] at 2176, b2[128] at 18560, w3[128] at 18688, b3 at 18816;
// W[k][n] multiplies input k into output n.
#include <cuda_bf16.h>

#include "fs_internal.h"

namespace fs {

namespace {

constexpr int H = 128;
constexpr int F = 16;
constexpr int OFF_W1 = 0, OFF_B1 = 2048, OFF_W2 = 2176, OFF_B2 = 18560, OFF_W3 = 18688, OFF_B3 = 18816;
constexpr int W1T_STRIDE = 24;    // bf16 per row of W1t[n][k] (padded: no bank conflicts)
constexpr int W2_STRIDE = 136;    // bf16 per row of W2t / W2s (padded)
constexpr int T_STRIDE = 136;     // bf16 per row of per-warp 16 x 128 tiles
constexpr int X_STRIDE = 24;      // bf16 per row of per-warp 16 x 16 input tiles
constexpr int BWD_WARPS = 4;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned long long warp_sum_cuts(unsigned long long v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack2(const __nv_bfloat16 lo, const __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Shared weights: W1t[n][k], W2t[n][k] (forward) and optionally W2s[k][n].
__device__ void stage_weights(const float* __restrict__ P, __nv_bfloat16* w1t, __nv_bfloat16* w2t,
                              __nv_bfloat16* w2s)
{
    for (int i = threadIdx.x; i < F * H; i += blockDim.x) {
        const int k = i / H, n = i % H;
        w1t[n * W1T_STRIDE + k] = __float2bfloat16_rn(P[OFF_W1 + i]);
    }
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
        const int k = i / H, n = i % H;
        const __nv_bfloat16 v = __float2bfloat16_rn(P[OFF_W2 + i]);
        w2t[n * W2_STRIDE + k] = v;
        if (w2s) w2s[k * W2_STRIDE + n] = v;
    }
}

// Forward pass of one warp's 16 rows.  xs: the warp's bf16 input tile
// [16][X_STRIDE].  Returns y for rows g and g+8 in lanes with t == 0 and
// leaves h1pre/h2pre (C-fragment layout, 16 n-tiles x 4) for the backward.
struct Fwd {
    float h1[16][4];
    float h2[16][4];
    float y0, y1;   // rows g, g + 8 (all lanes of the group hold them)
};

__device__ __forceinline__ void forward_tile(const float* __restrict__ P, const __nv_bfloat16* xs,
                                             const __nv_bfloat16* w1t, const __nv_bfloat16* w2t, Fwd& f)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t a[4];
    a[0] = ld32(xs + g * X_STRIDE + 2 * t);
    a[1] = ld32(xs + (g + 8) * X_STRIDE + 2 * t);
    a[2] = ld32(xs + g * X_STRIDE + 2 * t + 8);
    a[3] = ld32(xs + (g + 8) * X_STRIDE + 2 * t + 8);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float b0 = P[OFF_B1 + 8 * j + 2 * t], b1v = P[OFF_B1 + 8 * j + 2 * t + 1];
        f.h1[j][0] = b0; f.h1[j][1] = b1v; f.h1[j][2] = b0; f.h1[j][3] = b1v;
        const __nv_bfloat16* wb = w1t + (8 * j + g) * W1T_STRIDE + 2 * t;
        mma_bf16(f.h1[j], a, ld32(wb), ld32(wb + 8));
    }
    // layer 2: A fragments from relu(h1) rounded to bf16
    uint32_t a2[8][4];
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
        const float* c0 = f.h1[2 * kt];
        const float* c1 = f.h1[2 * kt + 1];
        a2[kt][0] = pack_bf16(fmaxf(c0[0], 0.f), fmaxf(c0[1], 0.f));
        a2[kt][1] = pack_bf16(fmaxf(c0[2], 0.f), fmaxf(c0[3], 0.f));
        a2[kt][2] = pack_bf16(fmaxf(c1[0], 0.f), fmaxf(c1[1], 0.f));
        a2[kt][3] = pack_bf16(fmaxf(c1[2], 0.f), fmaxf(c1[3], 0.f));
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float b0 = P[OFF_B2 + 8 * j + 2 * t], b1v = P[OFF_B2 + 8 * j + 2 * t + 1];
        f.h2[j][0] = b0; f.h2[j][1] = b1v; f.h2[j][2] = b0; f.h2[j][3] = b1v;
#pragma unroll
        for (int kt = 0; kt < 8; ++kt) {
            const __nv_bfloat16* wb = w2t + (8 * j + g) * W2_STRIDE + 16 * kt + 2 * t;
            mma_bf16(f.h2[j], a2[kt], ld32(wb), ld32(wb + 8));
        }
    }
    // layer 3 (FP32 dot with bf16-rounded w3)
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float w0 = bf16r(P[OFF_W3 + 8 * j + 2 * t]), w1 = bf16r(P[OFF_W3 + 8 * j + 2 * t + 1]);
        s0 += fmaxf(f.h2[j][0], 0.f) * w0 + fmaxf(f.h2[j][1], 0.f) * w1;
        s1 += fmaxf(f.h2[j][2], 0.f) * w0 + fmaxf(f.h2[j][3], 0.f) * w1;
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    f.y0 = s0 + P[OFF_B3];
    f.y1 = s1 + P[OFF_B3];
}

// Loads 16 rows of 16 FP32 features (rows >= n are zero) as bf16 into xs.
__device__ __forceinline__ void load_x(const float* __restrict__ X, long long row0, long long n, __nv_bfloat16* xs)
{
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < 16 * F; i += 32) {
        const int r = i / F, k = i % F;
        const long long row = row0 + r;
        xs[r * X_STRIDE + k] = __float2bfloat16_rn(row < n ? X[row * F + k] : 0.f);
    }
    __syncwarp();
}

// Loss and gradients (accumulated into G, 18817 FP32 + 1 loss, zeroed by the
// caller): forward, MSE loss mean((y - target)^2), backward.
__global__ void __launch_bounds__(BWD_WARPS * 32) mlp_grad_kernel(const float* __restrict__ P,
                                                                  const float* __restrict__ X,
                                                                  const float* __restrict__ T, long long n,
                                                                  float* __restrict__ G)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* w1t = (__nv_bfloat16*)smem;
    __nv_bfloat16* w2t = w1t + H * W1T_STRIDE;
    __nv_bfloat16* w2s = w2t + H * W2_STRIDE;
    __nv_bfloat16* tiles_bf = w2s + H * W2_STRIDE;                 // per warp: xs, h1, dh2, dh1
    const int per_warp = 16 * X_STRIDE + 3 * 16 * T_STRIDE;
    float* acc_w1 = (float*)(tiles_bf + BWD_WARPS * per_warp);    // 16 x 128
    float* acc_w2 = acc_w1 + F * H;                                // 128 x 128
    float* acc_b1 = acc_w2 + H * H;
    float* acc_b2 = acc_b1 + H;
    float* acc_w3 = acc_b2 + H;
    float* acc_misc = acc_w3 + H;                                  // b3, loss
    stage_weights(P, w1t, w2t, w2s);
    for (int i = threadIdx.x; i < F * H + H * H + 3 * H + 2; i += blockDim.x) acc_w1[i] = 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    __nv_bfloat16* xs = tiles_bf + warp * per_warp;
    __nv_bfloat16* h1s = xs + 16 * X_STRIDE;
    __nv_bfloat16* dh2s = h1s + 16 * T_STRIDE;
    __nv_bfloat16* dh1s = dh2s + 16 * T_STRIDE;
    const float inv_n = 1.0f / (float)n;
    const long long tiles = (n + 15) / 16;
    for (long long tile = (long long)blockIdx.x * BWD_WARPS + warp; tile < tiles; tile += (long long)gridDim.x * BWD_WARPS) {
        load_x(X, tile * 16, n, xs);
        Fwd f;
        forward_tile(P, xs, w1t, w2t, f);
        const long long r0 = tile * 16 + g, r1 = r0 + 8;
        const bool v0 = r0 < n, v1 = r1 < n;
        const float e0 = v0 ? f.y0 - T[r0] : 0.f, e1 = v1 ? f.y1 - T[r1] : 0.f;
        const float dy0 = 2.f * e0 * inv_n, dy1 = 2.f * e1 * inv_n;
        if (t == 0) {
            atomicAdd(&acc_misc[1], (e0 * e0 + e1 * e1) * inv_n);
            atomicAdd(&acc_misc[0], dy0 + dy1);
        }
        // h1 (relu, bf16) into smem for dW2
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = 8 * j + 2 * t;
            *reinterpret_cast<uint32_t*>(h1s + g * T_STRIDE + col) = pack_bf16(fmaxf(f.h1[j][0], 0.f), fmaxf(f.h1[j][1], 0.f));
            *reinterpret_cast<uint32_t*>(h1s + (g + 8) * T_STRIDE + col) = pack_bf16(fmaxf(f.h1[j][2], 0.f), fmaxf(f.h1[j][3], 0.f));
        }
        // dh2pre = dy w3 relu'(h2pre); dw3 += relu(h2) dy; db2 += dh2pre
        uint32_t ad[8][4];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = 8 * j + 2 * t;
            const float w0 = bf16r(P[OFF_W3 + col]), w1 = bf16r(P[OFF_W3 + col + 1]);
            const float d00 = f.h2[j][0] > 0.f ? dy0 * w0 : 0.f, d01 = f.h2[j][1] > 0.f ? dy0 * w1 : 0.f;
            const float d10 = f.h2[j][2] > 0.f ? dy1 * w0 : 0.f, d11 = f.h2[j][3] > 0.f ? dy1 * w1 : 0.f;
            float gw0 = fmaxf(f.h2[j][0], 0.f) * dy0 + fmaxf(f.h2[j][2], 0.f) * dy1;
            float gw1 = fmaxf(f.h2[j][1], 0.f) * dy0 + fmaxf(f.h2[j][3], 0.f) * dy1;
            float gb0 = d00 + d10, gb1 = d01 + d11;
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                gw0 += __shfl_xor_sync(0xffffffffu, gw0, off);
                gw1 += __shfl_xor_sync(0xffffffffu, gw1, off);
                gb0 += __shfl_xor_sync(0xffffffffu, gb0, off);
                gb1 += __shfl_xor_sync(0xffffffffu, gb1, off);
            }
            if (g == 0) {
                atomicAdd(&acc_w3[col], gw0);
                atomicAdd(&acc_w3[col + 1], gw1);
                atomicAdd(&acc_b2[col], gb0);
                atomicAdd(&acc_b2[col + 1], gb1);
            }
            const uint32_t p0 = pack_bf16(d00, d01), p1 = pack_bf16(d10, d11);
            *reinterpret_cast<uint32_t*>(dh2s + g * T_STRIDE + col) = p0;
            *reinterpret_cast<uint32_t*>(dh2s + (g + 8) * T_STRIDE + col) = p1;
            // A fragments of dh2 for dh1 = dh2 W2^T (k-tile j/2)
            ad[j >> 1][(j & 1) ? 2 : 0] = p0;
            ad[j >> 1][(j & 1) ? 3 : 1] = p1;
        }
        // dh1pre = (dh2 W2^T) relu'(h1pre)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 8; ++kt) {
                const __nv_bfloat16* wb = w2s + (8 * j + g) * W2_STRIDE + 16 * kt + 2 * t;
                mma_bf16(d, ad[kt], ld32(wb), ld32(wb + 8));
            }
            const int col = 8 * j + 2 * t;
            const float q00 = f.h1[j][0] > 0.f ? d[0] : 0.f, q01 = f.h1[j][1] > 0.f ? d[1] : 0.f;
            const float q10 = f.h1[j][2] > 0.f ? d[2] : 0.f, q11 = f.h1[j][3] > 0.f ? d[3] : 0.f;
            float gb0 = q00 + q10, gb1 = q01 + q11;
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                gb0 += __shfl_xor_sync(0xffffffffu, gb0, off);
                gb1 += __shfl_xor_sync(0xffffffffu, gb1, off);
            }
            if (g == 0) {
                atomicAdd(&acc_b1[col], gb0);
                atomicAdd(&acc_b1[col + 1], gb1);
            }
            *reinterpret_cast<uint32_t*>(dh1s + g * T_STRIDE + col) = pack_bf16(q00, q01);
            *reinterpret_cast<uint32_t*>(dh1s + (g + 8) * T_STRIDE + col) = pack_bf16(q10, q11);
        }
        __syncwarp();
        // dW1 += X^T dh1  (M = 16 features, N = 128, K = 16 rows)
        {
            uint32_t a[4];
            a[0] = pack2(xs[(2 * t) * X_STRIDE + g], xs[(2 * t + 1) * X_STRIDE + g]);
            a[1] = pack2(xs[(2 * t) * X_STRIDE + g + 8], xs[(2 * t + 1) * X_STRIDE + g + 8]);
            a[2] = pack2(xs[(2 * t + 8) * X_STRIDE + g], xs[(2 * t + 9) * X_STRIDE + g]);
            a[3] = pack2(xs[(2 * t + 8) * X_STRIDE + g + 8], xs[(2 * t + 9) * X_STRIDE + g + 8]);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n0 = 8 * j + g;
                const uint32_t b0 = pack2(dh1s[(2 * t) * T_STRIDE + n0], dh1s[(2 * t + 1) * T_STRIDE + n0]);
                const uint32_t b1 = pack2(dh1s[(2 * t + 8) * T_STRIDE + n0], dh1s[(2 * t + 9) * T_STRIDE + n0]);
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                mma_bf16(d, a, b0, b1);
                const int col = 8 * j + 2 * t;
                atomicAdd(&acc_w1[g * H + col], d[0]);
                atomicAdd(&acc_w1[g * H + col + 1], d[1]);
                atomicAdd(&acc_w1[(g + 8) * H + col], d[2]);
                atomicAdd(&acc_w1[(g + 8) * H + col + 1], d[3]);
            }
        }
        // dW2 += h1^T dh2  (M = 128, N = 128, K = 16 rows)
#pragma unroll 1
        for (int mt = 0; mt < 8; ++mt) {
            uint32_t a[4];
            const int m0 = 16 * mt + g;
            a[0] = pack2(h1s[(2 * t) * T_STRIDE + m0], h1s[(2 * t + 1) * T_STRIDE + m0]);
            a[1] = pack2(h1s[(2 * t) * T_STRIDE + m0 + 8], h1s[(2 * t + 1) * T_STRIDE + m0 + 8]);
            a[2] = pack2(h1s[(2 * t + 8) * T_STRIDE + m0], h1s[(2 * t + 9) * T_STRIDE + m0]);
            a[3] = pack2(h1s[(2 * t + 8) * T_STRIDE + m0 + 8], h1s[(2 * t + 9) * T_STRIDE + m0 + 8]);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n0 = 8 * j + g;
                const uint32_t b0 = pack2(dh2s[(2 * t) * T_STRIDE + n0], dh2s[(2 * t + 1) * T_STRIDE + n0]);
                const uint32_t b1 = pack2(dh2s[(2 * t + 8) * T_STRIDE + n0], dh2s[(2 * t + 9) * T_STRIDE + n0]);
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                mma_bf16(d, a, b0, b1);
                const int col = 8 * j + 2 * t;
                atomicAdd(&acc_w2[(16 * mt + g) * H + col], d[0]);
                atomicAdd(&acc_w2[(16 * mt + g) * H + col + 1], d[1]);
                atomicAdd(&acc_w2[(16 * mt + g + 8) * H + col], d[2]);
                atomicAdd(&acc_w2[(16 * mt + g + 8) * H + col + 1], d[3]);
            }
        }
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < F * H; i += blockDim.x) atomicAdd(&G[OFF_W1 + i], acc_w1[i]);
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) atomicAdd(&G[OFF_W2 + i], acc_w2[i]);
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        atomicAdd(&G[OFF_B1 + i], acc_b1[i]);
        atomicAdd(&G[OFF_B2 + i], acc_b2[i]);
        atomicAdd(&G[OFF_W3 + i], acc_w3[i]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&G[OFF_B3], acc_misc[0]);
        atomicAdd(&G[MLP_PARAMS], acc_misc[1]);
    }
}

__global__ void adam_kernel(float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                            const float* __restrict__ G, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.f - b1) * g;
        const float v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// ---------------------------------------------------------------- features

// 1 + log2 |x - y| (0 when x = y) of two 128-bit registers read as unsigned
// integers (qubit q = bit q); the fraction comes from the 32 bits below the
// leading one.
__device__ __forceinline__ float log2_distance(const uint32_t* x, const uint32_t* y)
{
    uint32_t xv[4], yv[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        xv[w] = x[w];
        yv[w] = y[w];
    }
    bool ge = true, decided = false;   // x >= y ?
#pragma unroll
    for (int w = 3; w >= 0; --w) {
        if (!decided && xv[w] != yv[w]) {
            ge = xv[w] > yv[w];
            decided = true;
        }
    }
    uint32_t d[4];
    uint32_t borrow = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t a = ge ? xv[w] : yv[w], b = ge ? yv[w] : xv[w];
        d[w] = a - b - borrow;
        borrow = (a < b || (a == b && borrow)) ? 1u : 0u;
    }
    float res = 0.f;
    bool found = false;
#pragma unroll
    for (int w = 3; w >= 0; --w) {
        if (!found && d[w]) {
            found = true;
            const int msb = 31 - __clz(d[w]);
            // 24 bits below and including the leading one
            const uint32_t lo = w ? d[w > 0 ? w - 1 : 0] : 0u;
            const uint32_t top = msb >= 23 ? (d[w] >> (msb - 23))
                                           : ((d[w] << (23 - msb)) | (lo >> (32 - (23 - msb))));
            const float mant = (float)top * (1.0f / 8388608.0f);   // in [1, 2)
            res = (float)(32 * w + msb + 1) + __log2f(mant);
        }
    }
    return res;
}

// 16 features of one live checkpoint entry (partial history after the
// prefix): |beta|, log10|beta|, Re beta/|beta|, Im beta/|beta|,
// (1 + log2 |int(sigma) - int(b_in)|)/8 (0 if equal), prefix depth c1/G, remaining
// artificial sources (A - A_p)/A, Hamming distance(sigma, b_in)/n, and
// (sigma xor b_in) on the qubits of the next 8 artificial sources.  Bottom
// entries give NaN in feature 0.
__device__ __forceinline__ void entry_features_of(const JobDev& J, const Entry& e, unsigned long long local,
                                                  const FeatureSpec& sp, float* out)
{
    const unsigned long long pair = local >> J.Ap;
    unsigned long long sidx, o;
    if (J.S == 1) {   // the 64-bit division routine would use the FP64 pipe
        o = pair;
        sidx = 0;
    } else if (pair < (1ull << 32)) {   // multiplier division (the job's s_magic, s_shift)
        const uint32_t p32 = (uint32_t)pair, t = __umulhi(J.s_magic, p32);
        const uint32_t o32 = (t + ((p32 - t) >> 1)) >> (J.s_shift - 1);
        o = o32;
        sidx = p32 - o32 * (uint32_t)J.S;
    } else {
        o = pair / (unsigned long long)J.S;
        sidx = pair - o * (unsigned long long)J.S;
    }
    (void)o;
    const uint32_t* bin = J.ins + 4 * sidx;
    if (((unsigned long long)__double_as_longlong(e.amp.x) << 1) > 0xffe0000000000000ull) {   // bottom (NaN)
        for (int k = 0; k < 16; ++k) out[k] = 0.f;
        out[0] = __int_as_float(0x7fc00000);
        return;
    }
    // FP32 is enough: the features are rounded to bfloat16 for the MLP
    const float re = (float)e.amp.x, im = (float)e.amp.y;
    const float mag = sqrtf(re * re + im * im);
    const float lg = mag > 0.f ? __log10f(mag) : -30.f;
    out[0] = mag;
    out[1] = fmaxf(lg, -30.f);
    out[2] = mag > 0.f ? __fdividef(re, mag) : 0.f;
    out[3] = mag > 0.f ? __fdividef(im, mag) : 0.f;
    out[4] = log2_distance(e.st, bin) / 8.f;
    out[5] = sp.depth;
    out[6] = sp.remaining;
    int ham = 0;
    for (int w = 0; w < 4; ++w) ham += __popc(e.st[w] ^ bin[w]);
    out[7] = (float)ham / (float)sp.n_qubits;
    for (int k = 0; k < 8; ++k) {
        const int q = sp.next_qubits[k];
        const int w = q >> 5;   // register word, selected without a local-memory index
        const uint32_t sw = w == 0 ? e.st[0] : w == 1 ? e.st[1] : w == 2 ? e.st[2] : e.st[3];
        out[8 + k] = q < 0 ? 0.f : (float)(((sw ^ bin[w & 3]) >> (q & 31)) & 1u);
    }
}

__device__ void entry_features(const JobDev& J, unsigned long long local, const FeatureSpec& sp, float* out)
{
    entry_features_of(J, J.table[local], local, sp, out);
}

// Training target of one logged subtree sum S (re, im): log10 |S| in FP64,
// floored (an exactly zero sum gives the floor), rounded to FP32.
__global__ void targets_kernel(const double2* __restrict__ sums, unsigned long long n, double floor_v,
                               float* __restrict__ t)
{
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const double2 v = sums[i];
        const double mag = hypot(v.x, v.y);
        const double lg = mag > 0.0 ? log10(mag) : floor_v;
        t[i] = (float)(lg > floor_v ? lg : floor_v);
    }
}

__global__ void features_kernel(const JobDev* __restrict__ jobs, int job, FeatureSpec sp, float* __restrict__ feat,
                                unsigned long long n)
{
    const JobDev& J = jobs[job];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        entry_features(J, i, sp, feat + 16 * i);
}

// ------------------------------------------------------- tcgen05 scoring
//
// Inference on the 5th-generation tensor cores (tcgen05.mma, accumulators in
// tensor memory).  A CTA of 256 threads runs two independent pipelines, one
// per warpgroup; each scores tiles of 128 rows, one row per thread:
//   X (128 x 16 bf16, shared)  --1 MMA (M 128, N 128, K 16)-->  D (FP32, TMEM)
//   epilogue 1: D + b1, ReLU, round to bf16 -> H1 (128 x 128 bf16, shared)
//   H1 --8 MMAs (K 16 each)--> D (the same 128 TMEM columns)
//   epilogue 2: D + b2, ReLU, dot with bf16(w3), + b3 -> y.
// The operands, roundings and FP32 accumulation are those of the training
// kernels (only the summation order inside the tensor core differs).
// Shared operands use the K-major layout without swizzle: core matrices of
// 8 rows x 16 bytes (8 bf16 of one row), LBO = byte distance between core
// matrices along K (128 here), SBO = between 8-row groups along M or N.

constexpr int TC_THREADS = 256;
// CTAs per compaction block when the scorer writes the compaction: a
// block's (at most 8) tiles of 128 live entries go one per warpgroup, so a
// block that holds most of the live entries is not scored tile after tile
// by one CTA; part 0 writes the block's compaction, every part lists the
// block's live entries in its own shared memory.
constexpr int TC_SPLIT = 4;
constexpr uint32_t TC_COLS = 256;             // TMEM columns per CTA, 128 per warpgroup
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;  // default mbarrier polls before a wait gives up
constexpr uint32_t TC_DRAIN_LIMIT = 1u << 24; // polls for the commit left pending by a give-up
constexpr int SM_W1 = 0;                      // B of layer 1: 128 n x 16 k
constexpr int SM_W2 = SM_W1 + 4096;           // B of layer 2: 128 n x 128 k
constexpr int SM_X = SM_W2 + 32768;           // per warpgroup: 128 rows x 16 k
constexpr int SM_H1 = SM_X + 2 * 4096;        // per warpgroup: 128 rows x 128 k
constexpr int SM_VEC = SM_H1 + 2 * 32768;     // b1, b2, bf16(w3) (FP32), b3
constexpr int SM_BAR = SM_VEC + (3 * H + 4) * 4;   // 2 mbarriers, TMEM address, 2 abort flags
constexpr int SM_LIST = SM_BAR + 64;          // one compaction block's live entries (from_live = 2)
constexpr int TC_SMEM = SM_LIST + 2 * COMPACT_BLOCK;
static_assert(SM_BAR % 8 == 0, "mbarrier alignment");
static_assert(2 * (TC_SMEM + 128 + 1024) <= 233472, "two CTAs per SM (dynamic, static and reserved shared memory)");

// instruction descriptor of kind::f16: FP32 D (bits 4-5 = 1), bf16 A and B
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in a K-major no-swizzle operand whose
// 8-row groups are sbo bytes apart
__device__ __forceinline__ uint32_t kmajor_off(int row, int k, uint32_t sbo)
{
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4
// (16-29), SBO >> 4 (32-45), descriptor version 1 (46-48), base offset 0,
// no swizzle (61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(a), "l"(b), "r"(TC_IDESC), "r"(accumulate)
        : "memory");
}

// arrives on the mbarrier once every MMA issued so far by this thread is done
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// named barrier of one warpgroup (ids 1 and 2; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int grp)
{
    if (grp == 0) asm volatile("bar.sync 1, 128;" ::: "memory");
    else asm volatile("bar.sync 2, 128;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// 32 consecutive FP32 columns of this thread's TMEM lane; the wait is in the
// same statement so no use of v can be scheduled before the data arrive
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

// Packed FP32 pairs (low word = even column) for the epilogues.
__device__ __forceinline__ uint64_t pack_f32x2(uint32_t lo, uint32_t hi)
{
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

__device__ __forceinline__ uint64_t add_f32x2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint64_t fma_f32x2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ uint64_t relu_f32x2(uint64_t a)
{
    const float lo = fmaxf(__uint_as_float((uint32_t)a), 0.f);
    const float hi = fmaxf(__uint_as_float((uint32_t)(a >> 32)), 0.f);
    return pack_f32x2(__float_as_uint(lo), __float_as_uint(hi));
}

// ReLU of both halves, rounded to bf16 (nearest even), low half first
__device__ __forceinline__ uint32_t relu_bf16x2(uint64_t a)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;"
        : "=r"(d)
        : "f"(__uint_as_float((uint32_t)(a >> 32))), "f"(__uint_as_float((uint32_t)a)));
    return d;
}

// Thread 0 of the warpgroup polls the MMA-completion barrier (at most
// `limit` polls); the group then learns the outcome together.  False: the
// wait gave up, the error word has DEV_ERR_TIMEOUT and the group issues no
// further MMA (the commit it stopped waiting for is drained before the
// tensor memory is released, see the end of mlp_tc_kernel).
__device__ __forceinline__ bool group_wait(uint32_t bar, uint32_t parity, volatile uint32_t* abort_flag, int r,
                                           int grp, uint32_t* err, uint32_t limit)
{
    if (r == 0) {
        bool ok = false;
        for (uint32_t i = 0; i < limit && !ok; ++i) ok = mbar_try_wait(bar, parity);
        if (!ok) {
            *abort_flag = 1u;
            if (err) atomicOr(err, DEV_ERR_TIMEOUT);
        }
    }
    group_sync(grp);
    tc_fence_after();
    return *abort_flag == 0u;
}

// PRUNE: rows are the entries of a job's checkpoint table, features computed
// here, entries scoring below tau cut (amplitude set to NaN, counted in
// stats[5]).  With from_live = 1 the rows are the job's compacted live
// entries (row i = table entry live[i], stats[6] of them: the exact bound
// has cut the others already); with from_live = 2 the TC_SPLIT CTAs of
// table block b list its live entries in shared memory (the bound counted
// them per block), the first also writes the block's compaction, and each
// scores its share of the list (one launch less; the history reads the same
// live list); otherwise every table entry,
// and the entries left live are counted per compaction block.  Without
// PRUNE rows are X [n][16] and y goes to Y.
template <bool PRUNE>
__global__ void __launch_bounds__(TC_THREADS, 2)
    mlp_tc_kernel(const float* __restrict__ P, const float* __restrict__ X, long long n_rows, float* __restrict__ Y,
                  const JobDev* __restrict__ jobs, int job, FeatureSpec sp, float tau, uint32_t* err,
                  uint32_t wait_limit, int from_live)
{
    FS_GRID_DEP();
    extern __shared__ __align__(128) unsigned char sm[];
    const int tid = threadIdx.x, grp = tid >> 7, r = tid & 127, warp = tid >> 5;
    const JobDev* J = PRUNE ? &jobs[job] : nullptr;
    uint16_t* blist = (uint16_t*)(sm + SM_LIST);   // from_live = 2: the block's live entries
    long long n, t_first, tstride;
    const unsigned blk = blockIdx.x / TC_SPLIT, part = blockIdx.x % TC_SPLIT;   // from_live = 2
    if (PRUNE && from_live == 2) {
        n = (long long)compact_block_write(*J, blk, gridDim.x / TC_SPLIT, 0, blist, part == 0, true);
        t_first = 2 * part + grp;
        tstride = 2 * TC_SPLIT;
    } else {
        n = PRUNE ? (from_live ? (long long)J->stats[6] : (long long)(J->n_pairs << J->Ap)) : n_rows;
        t_first = (long long)blockIdx.x * 2 + grp;
        tstride = (long long)gridDim.x * 2;
    }
    const long long tiles = (n + 127) / 128;
    // a CTA with no tile leaves before staging anything (the live count of a
    // from_live launch is known only on the device)
    if (t_first - grp >= tiles) return;
    float* vb1 = (float*)(sm + SM_VEC);
    float* vb2 = vb1 + H;
    float* vw3 = vb2 + H;
    uint64_t* bars = (uint64_t*)(sm + SM_BAR);
    uint32_t* tmem_slot = (uint32_t*)(sm + SM_BAR + 16);
    volatile uint32_t* abort_flag = (volatile uint32_t*)(sm + SM_BAR + 20) + grp;

    // weights as the B operands (B[n][k] = W[k][n]), biases, bf16-rounded w3.
    // A thread takes 8 k x 4 n of W (eight 16-byte loads along n, coalesced
    // over the warp) and writes each of its 4 columns' 8 k values as one
    // 16-byte row segment of a core matrix: the staging is on every CTA's
    // critical path, and element-wise 2-byte shared stores queue up in the
    // shared-memory pipe.
    if (((uintptr_t)P & 15u) == 0u) {
        const float4* P4 = reinterpret_cast<const float4*>(P);
        auto stage_w = [&](int off, int unit, int sbo, int dst) {
            const int kg = unit / (H / 4), n0 = 4 * (unit % (H / 4));
            float4 v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = __ldg(P4 + (off + (8 * kg + e) * H + n0) / 4);
            *(uint4*)(sm + dst + kmajor_off(n0, 8 * kg, sbo)) =
                make_uint4(pack_bf16(v[0].x, v[1].x), pack_bf16(v[2].x, v[3].x), pack_bf16(v[4].x, v[5].x),
                           pack_bf16(v[6].x, v[7].x));
            *(uint4*)(sm + dst + kmajor_off(n0 + 1, 8 * kg, sbo)) =
                make_uint4(pack_bf16(v[0].y, v[1].y), pack_bf16(v[2].y, v[3].y), pack_bf16(v[4].y, v[5].y),
                           pack_bf16(v[6].y, v[7].y));
            *(uint4*)(sm + dst + kmajor_off(n0 + 2, 8 * kg, sbo)) =
                make_uint4(pack_bf16(v[0].z, v[1].z), pack_bf16(v[2].z, v[3].z), pack_bf16(v[4].z, v[5].z),
                           pack_bf16(v[6].z, v[7].z));
            *(uint4*)(sm + dst + kmajor_off(n0 + 3, 8 * kg, sbo)) =
                make_uint4(pack_bf16(v[0].w, v[1].w), pack_bf16(v[2].w, v[3].w), pack_bf16(v[4].w, v[5].w),
                           pack_bf16(v[6].w, v[7].w));
        };
        for (int u = tid; u < (F / 8) * (H / 4); u += TC_THREADS) stage_w(OFF_W1, u, 256, SM_W1);
#pragma unroll 2
        for (int u = tid; u < (H / 8) * (H / 4); u += TC_THREADS) stage_w(OFF_W2, u, 2048, SM_W2);
    } else {
        for (int i = tid; i < F * H; i += TC_THREADS) {
            const int k = i / H, n = i % H;
            *(__nv_bfloat16*)(sm + SM_W1 + kmajor_off(n, k, 256)) = __float2bfloat16_rn(P[OFF_W1 + i]);
        }
#pragma unroll 8
        for (int i = tid; i < H * H; i += TC_THREADS) {
            const int k = i / H, n = i % H;
            *(__nv_bfloat16*)(sm + SM_W2 + kmajor_off(n, k, 2048)) = __float2bfloat16_rn(P[OFF_W2 + i]);
        }
    }
    for (int i = tid; i < H; i += TC_THREADS) {
        vb1[i] = P[OFF_B1 + i];
        vb2[i] = P[OFF_B2 + i];
        vw3[i] = bf16r(P[OFF_W3 + i]);
    }
    if (tid == 0) {
        vw3[H] = P[OFF_B3];
        for (int g = 0; g < 2; ++g)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[g])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 2) ((volatile uint32_t*)(sm + SM_BAR + 20))[tid] = 0u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const uint32_t tmem = *tmem_slot + (uint32_t)grp * 128u;          // this group's columns
    const uint32_t t_row = tmem + ((uint32_t)(warp & 3) * 32u << 16);  // lane quarter of this warp
    unsigned char* xs = sm + SM_X + grp * 4096;
    unsigned char* h1 = sm + SM_H1 + grp * 32768;
    const uint32_t sx = smem_u32(xs), sh = smem_u32(h1);
    const uint32_t sw1 = smem_u32(sm + SM_W1), sw2 = smem_u32(sm + SM_W2);
    const uint32_t bar = smem_u32(&bars[grp]);
    const float b3 = vw3[H];
    uint32_t phase = 0;
    unsigned long long cuts = 0;
    // table index of a row
    auto entry_of = [&](long long row_) -> unsigned long long {
        if (from_live == 2) return (unsigned long long)blk * COMPACT_BLOCK + blist[row_];
        return from_live ? J->live[row_] : (unsigned long long)row_;
    };
    // PRUNE: the entry of the next tile is loaded while this tile's MMAs run
    Entry cur;
    unsigned long long cur_e = 0;
    {
        const long long row0 = t_first * 128 + r;
        if (PRUNE && row0 < n) {
            cur_e = entry_of(row0);
            cur = J->table[cur_e];
        }
    }
    // features of one row (bf16) into this group's X operand; false: the row
    // is outside the table or a bottom entry (zero features, never cut)
    auto stage_x = [&](long long row_, const Entry& e, unsigned long long e_idx) -> bool {
        float fv[16];
        bool lv = false;
        if (row_ < n) {
            if (PRUNE) {
                entry_features_of(*J, e, e_idx, sp, fv);
                lv = !isnan(fv[0]);
            } else {
                const float4* x4 = reinterpret_cast<const float4*>(X + row_ * F);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 v = x4[q];
                    fv[4 * q] = v.x; fv[4 * q + 1] = v.y; fv[4 * q + 2] = v.z; fv[4 * q + 3] = v.w;
                }
                lv = true;
            }
        }
        if (!lv) {
#pragma unroll
            for (int k = 0; k < F; ++k) fv[k] = 0.f;
        }
        *(uint4*)(xs + kmajor_off(r, 0, 256)) = make_uint4(pack_bf16(fv[0], fv[1]), pack_bf16(fv[2], fv[3]),
                                                           pack_bf16(fv[4], fv[5]), pack_bf16(fv[6], fv[7]));
        *(uint4*)(xs + kmajor_off(r, 8, 256)) = make_uint4(pack_bf16(fv[8], fv[9]), pack_bf16(fv[10], fv[11]),
                                                           pack_bf16(fv[12], fv[13]), pack_bf16(fv[14], fv[15]));
        return lv;
    };
    // the features of tile i + 1 are computed while tile i's layer-2 MMAs run
    long long tile = t_first;
    bool live = tile < tiles ? stage_x(tile * 128 + r, cur, cur_e) : false;
    unsigned long long row_e = cur_e;   // table index of this tile's row
    for (; tile < tiles; tile += tstride) {
        const long long row = tile * 128 + r;
        const long long nrow = row + tstride * 128;
        fence_async_smem();
        group_sync(grp);
        if (r == 0) {
            tc_fence_after();
            tc_mma(tmem, sdesc(sx, 256), sdesc(sw1, 256), 0u);
            tc_commit(bar);
        }
        if (PRUNE && nrow < n) {
            cur_e = entry_of(nrow);
            cur = J->table[cur_e];
        }
        if (!group_wait(bar, phase, abort_flag, r, grp, err, wait_limit)) break;
        phase ^= 1u;
        // epilogue 1: h1 = bf16(relu(x W1 + b1)) into the layer-2 A operand
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t v[32];
            tmem_ld32(t_row + 32u * c, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int n0 = 32 * c + 8 * q + 2 * e;
                    const uint64_t x = add_f32x2(pack_f32x2(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]),
                                                 *(const uint64_t*)(vb1 + n0));
                    w[e] = relu_bf16x2(x);
                }
                *(uint4*)(h1 + kmajor_off(r, 32 * c + 8 * q, 2048)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        fence_async_smem();
        tc_fence_before();
        group_sync(grp);
        if (r == 0) {
            tc_fence_after();
#pragma unroll
            for (int kt = 0; kt < 8; ++kt)
                tc_mma(tmem, sdesc(sh + 256u * kt, 2048), sdesc(sw2 + 256u * kt, 2048), kt ? 1u : 0u);
            tc_commit(bar);
        }
        // next tile's X (the layer-1 MMA that read X has completed)
        const bool live_next = tile + tstride < tiles ? stage_x(nrow, cur, cur_e) : false;
        if (!group_wait(bar, phase, abort_flag, r, grp, err, wait_limit)) break;
        phase ^= 1u;
        // epilogue 2: y = relu(h1 W2 + b2) . bf16(w3) + b3
        uint64_t acc2 = 0;   // two FP32 partial sums (even, odd columns)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t v[32];
            tmem_ld32(t_row + 32u * c, v);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int n0 = 32 * c + 2 * e;
                const uint64_t x = add_f32x2(pack_f32x2(v[2 * e], v[2 * e + 1]), *(const uint64_t*)(vb2 + n0));
                acc2 = fma_f32x2(relu_f32x2(x), *(const uint64_t*)(vw3 + n0), acc2);
            }
        }
        tc_fence_before();   // TMEM reads complete before the next tile's MMA
        const float y = (__uint_as_float((uint32_t)acc2) + __uint_as_float((uint32_t)(acc2 >> 32))) + b3;
        if (PRUNE) {
            const bool cut = live && y < tau;
            if (cut) {
                J->table[row_e].amp.x = __longlong_as_double((long long)LEARNED_CUT_BITS);
                ++cuts;
            }
            // entries left live, counted per compaction block (the warp's 32
            // rows lie in one block); the compaction's own count pass is skipped
            if (!from_live) {
                const unsigned keep = __ballot_sync(0xffffffffu, live && !cut);
                if ((tid & 31) == 0 && keep)
                    atomicAdd(&J->blk[(unsigned long long)(tile * 128 + (r & ~31)) / COMPACT_BLOCK], (unsigned)__popc(keep));
            }
        } else if (row < n) {
            Y[row] = y;
        }
        live = live_next;
        row_e = cur_e;
    }
    if (PRUNE) {
        cuts = warp_sum_cuts(cuts);
        if ((tid & 31) == 0 && cuts) atomicAdd(&J->stats[5], cuts);
    }
    // A group that gave up left one commit pending (parity `phase`): its MMAs
    // may still read shared memory and write this group's tensor-memory
    // columns, so thread 0 of the group waits for that commit (bounded)
    // before the CTA releases the tensor memory.
    if (*abort_flag != 0u && r == 0) {
        bool done = false;
        for (uint32_t i = 0; i < TC_DRAIN_LIMIT && !done; ++i) done = mbar_try_wait(bar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tmem_slot), "r"(TC_COLS)
                     : "memory");
    }
}

// Polls of a bounded tensor-core wait before it gives up (process-wide).
uint32_t g_wait_limit = TC_WAIT_LIMIT;

template <bool PRUNE>
cudaError_t launch_tc(const float* P, const float* X, long long n_rows, float* Y, const JobDev* jobs, int job,
                      const FeatureSpec& sp, float tau, uint32_t* err, unsigned long long rows, cudaStream_t s,
                      int from_live = 0)
{
    const unsigned long long tiles = (rows + 127) / 128;
    unsigned long long blocks = (tiles + 1) / 2;
    if (blocks > 148 * 2) blocks = 148 * 2;
    if (from_live == 2) blocks = TC_SPLIT * ((rows + COMPACT_BLOCK - 1) / COMPACT_BLOCK);   // TC_SPLIT per compaction block
    return launch_pdl(mlp_tc_kernel<PRUNE>, dim3((unsigned)blocks), dim3(TC_THREADS), TC_SMEM, s, P, X, n_rows, Y,
                      jobs, job, sp, tau, err, g_wait_limit, from_live);
}


size_t grad_smem_bytes()
{
    const size_t per_warp = 16 * X_STRIDE + 3 * 16 * T_STRIDE;
    return (size_t)(H * W1T_STRIDE + 2 * H * W2_STRIDE + BWD_WARPS * per_warp) * sizeof(__nv_bfloat16) +
           (size_t)(F * H + H * H + 3 * H + 2) * sizeof(float);
}

}  // namespace

cudaError_t mlp_forward(const float* d_params, const float* d_x, long long n, float* d_y, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    return launch_tc<false>(d_params, d_x, n, d_y, nullptr, 0, FeatureSpec{}, 0.f, nullptr,
                            (unsigned long long)n, s);
}

cudaError_t mlp_grad(const float* d_params, const float* d_x, const float* d_t, long long n, float* d_grad,
                     cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_grad, 0, (MLP_PARAMS + 1) * sizeof(float), s);
    if (e != cudaSuccess || n <= 0) return e;
    const size_t smem = grad_smem_bytes();
    e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (n + 15) / 16;
    long long blocks = (tiles + BWD_WARPS - 1) / BWD_WARPS;
    if (blocks > 148) blocks = 148;
    mlp_grad_kernel<<<(unsigned)blocks, BWD_WARPS * 32, smem, s>>>(d_params, d_x, d_t, n, d_grad);
    return cudaGetLastError();
}

cudaError_t mlp_features(const JobDev* d_jobs, int job, const FeatureSpec& sp, float* d_feat,
                         unsigned long long n_entries, cudaStream_t s)
{
    if (n_entries == 0) return cudaSuccess;
    unsigned long long blocks = (n_entries + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    features_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_jobs, job, sp, d_feat, n_entries);
    return cudaGetLastError();
}

cudaError_t mlp_targets(const double* d_sums, unsigned long long n, double floor_v, float* d_t, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    unsigned long long blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    targets_kernel<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const double2*>(d_sums), n, floor_v, d_t);
    return cudaGetLastError();
}

cudaError_t mlp_learned_prune(const float* d_params, const JobDev* d_jobs, int job, const FeatureSpec& sp,
                              float tau, unsigned long long n_entries, uint32_t* d_err, cudaStream_t s, int rows)
{
    if (n_entries == 0) return cudaSuccess;
    if (rows == 2 && (n_entries + COMPACT_BLOCK - 1) / COMPACT_BLOCK > (unsigned long long)COMPACT_DIRECT_BLOCKS)
        return cudaErrorInvalidValue;   // the fused compaction adds the block counts itself
    return launch_tc<true>(d_params, nullptr, 0, nullptr, d_jobs, job, sp, tau, d_err, n_entries, s, rows);
}

void mlp_set_wait_limit(uint32_t polls) { g_wait_limit = polls; }
uint32_t mlp_default_wait_limit() { return TC_WAIT_LIMIT; }

cudaError_t mlp_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(mlp_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
}

cudaError_t mlp_adam(float* d_params, float* d_m, float* d_v, const float* d_grad, float lr, int step,
                     cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(MLP_PARAMS + 255) / 256, 256, 0, s>>>(d_params, d_m, d_v, d_grad, MLP_PARAMS, lr, b1, b2,
                                                         1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace fs
