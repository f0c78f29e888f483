// Learned pruning at the checkpoint boundary: a 16 -> 128 -> 128 -> 1 MLP
// (ReLU) that scores checkpoint-table entries (partial histories after the
// prefix of Algorithm 2) by the predicted log10 |exact subtree sum|; entries
// scoring below a threshold tau are cut, the rest are enumerated exactly.
//
// Numerics: BF16 operands on the tensor cores (mma.sync m16n8k16, FP32
// accumulate); FP32 master weights and Adam state.  Rounded to BF16: the
// inputs X, W1, W2, w3, the hidden activation h1 (layer-2 operand) and, in the
// backward pass, the GEMM operands dh2 and dh1.  Everything else is FP32.
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
constexpr int FWD_WARPS = 8;
constexpr int BWD_WARPS = 4;
constexpr int PRUNE_WARPS = 4;

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

// Inference-only forward of 16 rows: layer-2 tiles are reduced into the
// layer-3 dot as they are produced, so neither h1 nor h2 stays live
// (low register use).  Same operands, roundings and sums as forward_tile.
__device__ __forceinline__ void score_tile(const float* __restrict__ P, const __nv_bfloat16* xs,
                                           const __nv_bfloat16* w1t, const __nv_bfloat16* w2t,
                                           float& y0, float& y1)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t a[4];
    a[0] = ld32(xs + g * X_STRIDE + 2 * t);
    a[1] = ld32(xs + (g + 8) * X_STRIDE + 2 * t);
    a[2] = ld32(xs + g * X_STRIDE + 2 * t + 8);
    a[3] = ld32(xs + (g + 8) * X_STRIDE + 2 * t + 8);
    uint32_t a2[8][4];
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
        float c[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * kt + h;
            const float b0 = P[OFF_B1 + 8 * j + 2 * t], b1v = P[OFF_B1 + 8 * j + 2 * t + 1];
            c[h][0] = b0; c[h][1] = b1v; c[h][2] = b0; c[h][3] = b1v;
            const __nv_bfloat16* wb = w1t + (8 * j + g) * W1T_STRIDE + 2 * t;
            mma_bf16(c[h], a, ld32(wb), ld32(wb + 8));
        }
        a2[kt][0] = pack_bf16(fmaxf(c[0][0], 0.f), fmaxf(c[0][1], 0.f));
        a2[kt][1] = pack_bf16(fmaxf(c[0][2], 0.f), fmaxf(c[0][3], 0.f));
        a2[kt][2] = pack_bf16(fmaxf(c[1][0], 0.f), fmaxf(c[1][1], 0.f));
        a2[kt][3] = pack_bf16(fmaxf(c[1][2], 0.f), fmaxf(c[1][3], 0.f));
    }
    float s0 = 0.f, s1 = 0.f;
#pragma unroll 4
    for (int j = 0; j < 16; ++j) {
        float d[4];
        const float b0 = P[OFF_B2 + 8 * j + 2 * t], b1v = P[OFF_B2 + 8 * j + 2 * t + 1];
        d[0] = b0; d[1] = b1v; d[2] = b0; d[3] = b1v;
#pragma unroll
        for (int kt = 0; kt < 8; ++kt) {
            const __nv_bfloat16* wb = w2t + (8 * j + g) * W2_STRIDE + 16 * kt + 2 * t;
            mma_bf16(d, a2[kt], ld32(wb), ld32(wb + 8));
        }
        const float w0 = bf16r(P[OFF_W3 + 8 * j + 2 * t]), w1 = bf16r(P[OFF_W3 + 8 * j + 2 * t + 1]);
        s0 += fmaxf(d[0], 0.f) * w0 + fmaxf(d[1], 0.f) * w1;
        s1 += fmaxf(d[2], 0.f) * w0 + fmaxf(d[3], 0.f) * w1;
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    y0 = s0 + P[OFF_B3];
    y1 = s1 + P[OFF_B3];
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

__global__ void __launch_bounds__(FWD_WARPS * 32) mlp_forward_kernel(const float* __restrict__ P,
                                                                     const float* __restrict__ X, long long n,
                                                                     float* __restrict__ Y)
{
    __shared__ __align__(16) __nv_bfloat16 w1t[H * W1T_STRIDE];
    __shared__ __align__(16) __nv_bfloat16 w2t[H * W2_STRIDE];
    __shared__ __align__(16) __nv_bfloat16 xs_all[FWD_WARPS][16 * X_STRIDE];
    stage_weights(P, w1t, w2t, nullptr);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    __nv_bfloat16* xs = xs_all[warp];
    const long long tiles = (n + 15) / 16;
    for (long long tile = (long long)blockIdx.x * FWD_WARPS + warp; tile < tiles; tile += (long long)gridDim.x * FWD_WARPS) {
        load_x(X, tile * 16, n, xs);
        float y0, y1;
        score_tile(P, xs, w1t, w2t, y0, y1);
        if (t == 0) {
            const long long r0 = tile * 16 + g, r1 = r0 + 8;
            if (r0 < n) Y[r0] = y0;
            if (r1 < n) Y[r1] = y1;
        }
        __syncwarp();
    }
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
    uint32_t d[4];
    bool ge = true;   // x >= y ?
    for (int w = 3; w >= 0; --w) {
        if (x[w] != y[w]) { ge = x[w] > y[w]; break; }
    }
    const uint32_t* a = ge ? x : y;
    const uint32_t* b = ge ? y : x;
    uint32_t borrow = 0;
    for (int w = 0; w < 4; ++w) {
        const uint32_t t = a[w] - b[w] - borrow;
        borrow = (a[w] < b[w] || (a[w] == b[w] && borrow)) ? 1u : 0u;
        d[w] = t;
    }
    for (int w = 3; w >= 0; --w) {
        if (d[w]) {
            const int msb = 31 - __clz(d[w]);
            // 24 bits below and including the leading one
            const uint32_t lo = w ? d[w - 1] : 0u;
            const uint32_t top = msb >= 23 ? (d[w] >> (msb - 23))
                                           : ((d[w] << (23 - msb)) | (lo >> (32 - (23 - msb))));
            const float mant = (float)top * (1.0f / 8388608.0f);   // in [1, 2)
            return (float)(32 * w + msb + 1) + __log2f(mant);
        }
    }
    return 0.f;
}

// 16 features of one live checkpoint entry (partial history after the
// prefix): |beta|, log10|beta|, Re beta/|beta|, Im beta/|beta|,
// (1 + log2 |int(sigma) - int(b_in)|)/8 (0 if equal), prefix depth c1/G, remaining
// artificial sources (A - A_p)/A, Hamming distance(sigma, b_in)/n, and
// (sigma xor b_in) on the qubits of the next 8 artificial sources.  Bottom
// entries give NaN in feature 0.
__device__ void entry_features(const JobDev& J, unsigned long long local, const FeatureSpec& sp, float* out)
{
    const unsigned long long pair = local >> J.Ap;
    const unsigned long long o = pair / (unsigned long long)J.S;
    const unsigned long long sidx = pair - o * (unsigned long long)J.S;
    const Entry e = J.table[local];
    const uint32_t* bin = J.ins + 4 * sidx;
    if (isnan(e.amp.x)) {
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
        out[8 + k] = q < 0 ? 0.f : (float)(((e.st[q >> 5] ^ bin[q >> 5]) >> (q & 31)) & 1u);
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

// Scores every live entry of a job's checkpoint table with the MLP and cuts
// (marks bottom) those predicted below tau; counts cuts into stats[5].
__global__ void __launch_bounds__(PRUNE_WARPS * 32) learned_prune_kernel(const float* __restrict__ P,
                                                                         const JobDev* __restrict__ jobs, int job,
                                                                         FeatureSpec sp, float tau)
{
    __shared__ __align__(16) __nv_bfloat16 w1t[H * W1T_STRIDE];
    __shared__ __align__(16) __nv_bfloat16 w2t[H * W2_STRIDE];
    __shared__ __align__(16) __nv_bfloat16 xs_all[PRUNE_WARPS][32 * X_STRIDE];
    stage_weights(P, w1t, w2t, nullptr);
    __syncthreads();
    const JobDev& J = jobs[job];
    const unsigned long long n = J.n_pairs << J.Ap;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    __nv_bfloat16* xs = xs_all[warp];
    const long long tiles = (long long)((n + 31) / 32);
    unsigned long long cuts = 0;
    for (long long tile = (long long)blockIdx.x * PRUNE_WARPS + warp; tile < tiles; tile += (long long)gridDim.x * PRUNE_WARPS) {
        // every lane computes the features of one entry
        const unsigned long long row = (unsigned long long)tile * 32 + lane;
        float fv[16];
        bool ok = false;
        if (row < n) {
            entry_features(J, row, sp, fv);
            ok = !isnan(fv[0]);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) xs[lane * X_STRIDE + k] = __float2bfloat16_rn(ok ? fv[k] : 0.f);
        const unsigned live = __ballot_sync(0xffffffffu, ok);
        __syncwarp();
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            float y0, y1;
            score_tile(P, xs + 16 * half * X_STRIDE, w1t, w2t, y0, y1);
            if (t == 0) {
                const int r0 = 16 * half + g, r1 = r0 + 8;
                if (((live >> r0) & 1u) && y0 < tau) {
                    J.table[(unsigned long long)tile * 32 + r0].amp.x = __longlong_as_double(0x7ff8000000000000ll);
                    ++cuts;
                }
                if (((live >> r1) & 1u) && y1 < tau) {
                    J.table[(unsigned long long)tile * 32 + r1].amp.x = __longlong_as_double(0x7ff8000000000000ll);
                    ++cuts;
                }
            }
        }
        __syncwarp();
    }
    cuts = warp_sum_cuts(cuts);
    if (lane == 0 && cuts) atomicAdd(&J.stats[5], cuts);
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
    const long long tiles = (n + 15) / 16;
    long long blocks = (tiles + FWD_WARPS - 1) / FWD_WARPS;
    if (blocks > 148 * 4) blocks = 148 * 4;
    mlp_forward_kernel<<<(unsigned)blocks, FWD_WARPS * 32, 0, s>>>(d_params, d_x, n, d_y);
    return cudaGetLastError();
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

cudaError_t mlp_learned_prune(const float* d_params, const JobDev* d_jobs, int job, const FeatureSpec& sp,
                              float tau, unsigned long long n_entries, cudaStream_t s)
{
    if (n_entries == 0) return cudaSuccess;
    const unsigned long long tiles = (n_entries + 31) / 32;
    unsigned long long blocks = (tiles + PRUNE_WARPS - 1) / PRUNE_WARPS;
    if (blocks > 148 * 16) blocks = 148 * 16;
    learned_prune_kernel<<<(unsigned)blocks, PRUNE_WARPS * 32, 0, s>>>(d_params, d_jobs, job, sp, tau);
    return cudaGetLastError();
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
