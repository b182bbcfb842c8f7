// Kernels of the learned warm start: BF16 tensor-core implicit-GEMM 3x3
// convolutions (stride 1, padding 1, NHWC) with FP32 accumulation, their
// weight gradient, and the small element-wise / pooling / optimiser kernels.
//
// Tensor cores: mma.sync.aligned.m16n8k16 (bf16 x bf16 -> f32).  Shared
// tiles hold A as [m][k] and B as [n][k] (k contiguous, rows padded to 40
// elements so that the fragment loads hit distinct banks).  A block computes
// a 64 x 64 output tile with 4 warps (32 x 32 each = 2 x 4 mma tiles) and
// walks K in steps of 32 with double-buffered shared tiles.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace inim {
namespace cnn {

constexpr int kBM = 64, kBN = 64, kBK = 32, kPad = 40;   // tile sizes, padded k-row length
constexpr int kConvThreads = 128;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 32 x 32 warp tile from the shared A [64][kPad] / B [64][kPad] tiles
__device__ __forceinline__ void warp_mma_tile(const __nv_bfloat16* As, const __nv_bfloat16* Bs, int wm, int wn,
                                              float (&acc)[2][4][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
        unsigned a[2][4], b[4][2];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            const __nv_bfloat16* base = As + (wm * 32 + mi * 16 + g) * kPad + kk + 2 * t;
            a[mi][0] = *reinterpret_cast<const unsigned*>(base);
            a[mi][1] = *reinterpret_cast<const unsigned*>(base + 8 * kPad);
            a[mi][2] = *reinterpret_cast<const unsigned*>(base + 8);
            a[mi][3] = *reinterpret_cast<const unsigned*>(base + 8 * kPad + 8);
        }
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const __nv_bfloat16* base = Bs + (wn * 32 + ni * 8 + g) * kPad + kk + 2 * t;
            b[ni][0] = *reinterpret_cast<const unsigned*>(base);
            b[ni][1] = *reinterpret_cast<const unsigned*>(base + 8);
        }
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni]);
    }
}

// ---------------------------------------------------------------------------
// forward 3x3 conv: Y[p][co] = act(bias[co] + sum_{tap,ci} X[p+tap][ci] W[co][tap][ci])
//   X [B][H][W][Cin] bf16, W [Cout][9][Cin] bf16, Y [B][H][W][Cout] (bf16 or f32)
//   GEMM: M = B*H*W, N = Cout, K = 9*Cin
// ---------------------------------------------------------------------------
struct ConvArgs {
    const __nv_bfloat16* x;
    const __nv_bfloat16* w;
    const float* bias;        // nullable
    __nv_bfloat16* y_bf16;    // one of the two outputs
    float* y_f32;
    int B, H, W, Cin, Cout;
    int relu;
};

// one 8-wide k chunk of the im2col row of output pixel p (zero outside)
__device__ __forceinline__ uint4 im2col_chunk(const ConvArgs& a, int p, int k) {
    const int K = 9 * a.Cin;
    uint4 z = make_uint4(0, 0, 0, 0);
    if (p >= a.B * a.H * a.W || k >= K) return z;
    const int x = p % a.W, y = (p / a.W) % a.H, b = p / (a.W * a.H);
    if ((a.Cin & 7) == 0) {
        const int tap = k / a.Cin, ci = k - tap * a.Cin;
        const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
        if (yy < 0 || yy >= a.H || xx < 0 || xx >= a.W) return z;
        return *reinterpret_cast<const uint4*>(a.x + (((size_t)b * a.H + yy) * a.W + xx) * a.Cin + ci);
    }
    // generic (Cin not a multiple of 8): element by element
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int kk = k + e;
        v[e] = __float2bfloat16(0.0f);
        if (kk < K) {
            const int tap = kk / a.Cin, ci = kk - tap * a.Cin;
            const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
            if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) v[e] = a.x[(((size_t)b * a.H + yy) * a.W + xx) * a.Cin + ci];
        }
    }
    return *reinterpret_cast<const uint4*>(v);
}

__device__ __forceinline__ uint4 weight_chunk(const ConvArgs& a, int co, int k) {
    const int K = 9 * a.Cin;
    if (co >= a.Cout || k >= K) return make_uint4(0, 0, 0, 0);
    if ((K & 7) == 0) return *reinterpret_cast<const uint4*>(a.w + (size_t)co * K + k);
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (k + e < K) ? a.w[(size_t)co * K + k + e] : __float2bfloat16(0.0f);
    return *reinterpret_cast<const uint4*>(v);
}

__global__ void __launch_bounds__(kConvThreads) k_conv3x3_fwd(ConvArgs a) {
    __shared__ __align__(16) __nv_bfloat16 As[2][kBM * kPad];
    __shared__ __align__(16) __nv_bfloat16 Bs[2][kBN * kPad];
    const int M = a.B * a.H * a.W, K = 9 * a.Cin;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    const int tid = threadIdx.x, warp = tid >> 5, wm = warp >> 1, wn = warp & 1;
    float acc[2][4][4] = {};
    // each thread loads 2 chunks of A and 2 of B per k step (64 rows x 4 chunks)
    auto load = [&](int buf, int k0) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + r * kConvThreads;       // 0..255
            const int row = idx >> 2, ch = (idx & 3) * 8;
            *reinterpret_cast<uint4*>(&As[buf][row * kPad + ch]) = im2col_chunk(a, m0 + row, k0 + ch);
            *reinterpret_cast<uint4*>(&Bs[buf][row * kPad + ch]) = weight_chunk(a, n0 + row, k0 + ch);
        }
    };
    const int nk = (K + kBK - 1) / kBK;
    load(0, 0);
    __syncthreads();
    for (int s = 0; s < nk; ++s) {
        if (s + 1 < nk) load((s + 1) & 1, (s + 1) * kBK);
        warp_mma_tile(As[s & 1], Bs[s & 1], wm, wn, acc);
        __syncthreads();
    }
    // epilogue: bias, relu, store
    const int lane = tid & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int col = n0 + wn * 32 + ni * 8 + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm * 32 + mi * 16 + g + 8 * h;
                if (row >= M) continue;
                float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
                if (a.bias) {
                    if (col < a.Cout) v0 += a.bias[col];
                    if (col + 1 < a.Cout) v1 += a.bias[col + 1];
                }
                if (a.relu) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
                if (a.y_f32) {
                    if (col < a.Cout) a.y_f32[(size_t)row * a.Cout + col] = v0;
                    if (col + 1 < a.Cout) a.y_f32[(size_t)row * a.Cout + col + 1] = v1;
                } else {
                    if (col + 1 < a.Cout && ((a.Cout & 1) == 0)) {
                        *reinterpret_cast<__nv_bfloat162*>(a.y_bf16 + (size_t)row * a.Cout + col) =
                            __floats2bfloat162_rn(v0, v1);
                    } else {
                        if (col < a.Cout) a.y_bf16[(size_t)row * a.Cout + col] = __float2bfloat16(v0);
                        if (col + 1 < a.Cout) a.y_bf16[(size_t)row * a.Cout + col + 1] = __float2bfloat16(v1);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// weight gradient: dW[co][k] += sum_p dZ[p][co] * im2col(X)[p][k]
//   GEMM: M = Cout, N = 9*Cin, reduction over the pixels p (split across
//   blockIdx.z, FP32 atomics into dW).  A = dZ^T and B = im2col(X)^T are
//   transposed into the [m][k] / [n][k] shared layout while loading.
// ---------------------------------------------------------------------------
struct WgradArgs {
    const __nv_bfloat16* dz;   // [P][Cout]
    const __nv_bfloat16* x;    // [B][H][W][Cin]
    float* dw;                 // [Cout][9*Cin]
    int B, H, W, Cin, Cout;
    int p_per_split;           // multiple of kBK
};

__global__ void __launch_bounds__(kConvThreads) k_conv3x3_wgrad(WgradArgs a) {
    __shared__ __align__(16) __nv_bfloat16 As[kBM * kPad];   // [co][p]
    __shared__ __align__(16) __nv_bfloat16 Bs[kBN * kPad];   // [k][p]
    const int P = a.B * a.H * a.W, K = 9 * a.Cin;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    const int p_begin = blockIdx.z * a.p_per_split;
    const int p_end = min(P, p_begin + a.p_per_split);
    const int tid = threadIdx.x, warp = tid >> 5, wm = warp >> 1, wn = warp & 1;
    float acc[2][4][4] = {};
    ConvArgs ca{};
    ca.x = a.x; ca.B = a.B; ca.H = a.H; ca.W = a.W; ca.Cin = a.Cin; ca.Cout = a.Cout;
    for (int p0 = p_begin; p0 < p_end; p0 += kBK) {
        // 32 pixels x 64 co of dZ, 32 pixels x 64 k of im2col(X): 8-wide chunks
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + r * kConvThreads;     // 0..255
            const int pl = idx >> 3, ch = (idx & 7) * 8;  // pixel 0..31, chunk of 8 co / k
            const int p = p0 + pl;
            __align__(16) __nv_bfloat16 va[8];
            __align__(16) __nv_bfloat16 vb[8];
            const bool pin = p < p_end;
            if (pin && (a.Cout & 7) == 0 && m0 + ch + 8 <= a.Cout) {
                *reinterpret_cast<uint4*>(va) = *reinterpret_cast<const uint4*>(a.dz + (size_t)p * a.Cout + m0 + ch);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    va[e] = (pin && m0 + ch + e < a.Cout) ? a.dz[(size_t)p * a.Cout + m0 + ch + e]
                                                          : __float2bfloat16(0.0f);
            }
            *reinterpret_cast<uint4*>(vb) = pin ? im2col_chunk(ca, p, n0 + ch) : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                As[(ch + e) * kPad + pl] = va[e];
                Bs[(ch + e) * kPad + pl] = vb[e];
            }
        }
        __syncthreads();
        warp_mma_tile(As, Bs, wm, wn, acc);
        __syncthreads();
    }
    const int lane = tid & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int co = m0 + wm * 32 + mi * 16 + g + 8 * h;
                const int k = n0 + wn * 32 + ni * 8 + 2 * t;
                if (co >= a.Cout) continue;
                if (k < K) atomicAdd(&a.dw[(size_t)co * K + k], acc[mi][ni][2 * h]);
                if (k + 1 < K) atomicAdd(&a.dw[(size_t)co * K + k + 1], acc[mi][ni][2 * h + 1]);
            }
}

// ---------------------------------------------------------------------------
// element-wise, pooling and optimiser kernels
// ---------------------------------------------------------------------------
// bias gradient: db[c] += sum_p dz[p][c]
__global__ void k_bias_grad(const __nv_bfloat16* dz, float* db, int P, int C) {
    const int c = threadIdx.x % C;
    const int lanes = blockDim.x / C;
    const int sub = threadIdx.x / C;
    if (sub >= lanes) return;
    float s = 0.0f;
    for (int p = blockIdx.x * lanes + sub; p < P; p += gridDim.x * lanes) s += __bfloat162float(dz[(size_t)p * C + c]);
    atomicAdd(&db[c], s);
}

// dz = dy * (z > 0), in place on dy (bf16)
__global__ void k_relu_grad(__nv_bfloat16* dy, const __nv_bfloat16* z, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(z[i]) > 0.0f)) dy[i] = __float2bfloat16(0.0f);
}

// y = a + b
__global__ void k_add(__nv_bfloat16* y, const __nv_bfloat16* a, const __nv_bfloat16* b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

// y += a (gradient accumulation)
__global__ void k_accum(__nv_bfloat16* y, const __nv_bfloat16* a, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(__bfloat162float(y[i]) + __bfloat162float(a[i]));
}

// 2x2 average pool, NHWC: y [B][H/2][W/2][C]
__global__ void k_pool2(__nv_bfloat16* y, const __nv_bfloat16* x, int B, int H, int W, int C) {
    const size_t n = (size_t)B * (H / 2) * (W / 2) * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = i % C;
        size_t q = i / C;
        const int xo = q % (W / 2); q /= (W / 2);
        const int yo = q % (H / 2);
        const int b = (int)(q / (H / 2));
        float s = 0.0f;
#pragma unroll
        for (int d = 0; d < 4; ++d)
            s += __bfloat162float(x[(((size_t)b * H + 2 * yo + (d >> 1)) * W + 2 * xo + (d & 1)) * C + c]);
        y[i] = __float2bfloat16(0.25f * s);
    }
}

// gradient of the 2x2 average pool: dx = dy / 4 on each of the 4 pixels
__global__ void k_pool2_grad(__nv_bfloat16* dx, const __nv_bfloat16* dy, int B, int H, int W, int C) {
    const size_t n = (size_t)B * H * W * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = i % C;
        size_t q = i / C;
        const int x = q % W; q /= W;
        const int y = q % H;
        const int b = (int)(q / H);
        dx[i] = __float2bfloat16(0.25f * __bfloat162float(dy[(((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]));
    }
}

// nearest 2x upsample: y [B][2H][2W][C]
__global__ void k_up2(__nv_bfloat16* y, const __nv_bfloat16* x, int B, int H, int W, int C) {
    const size_t n = (size_t)B * 4 * H * W * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = i % C;
        size_t q = i / C;
        const int xo = q % (2 * W); q /= (2 * W);
        const int yo = q % (2 * H);
        const int b = (int)(q / (2 * H));
        y[i] = x[(((size_t)b * H + yo / 2) * W + xo / 2) * C + c];
    }
}

// gradient of the nearest 2x upsample: dx = sum of the 4 children
__global__ void k_up2_grad(__nv_bfloat16* dx, const __nv_bfloat16* dy, int B, int H, int W, int C) {
    const size_t n = (size_t)B * H * W * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = i % C;
        size_t q = i / C;
        const int x = q % W; q /= W;
        const int y = q % H;
        const int b = (int)(q / H);
        float s = 0.0f;
#pragma unroll
        for (int d = 0; d < 4; ++d)
            s += __bfloat162float(dy[(((size_t)b * 2 * H + 2 * y + (d >> 1)) * 2 * W + 2 * x + (d & 1)) * C + c]);
        dx[i] = __float2bfloat16(s);
    }
}

// f32 -> bf16
__global__ void k_to_bf16(__nv_bfloat16* y, const float* x, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// weights for the data gradient: wt[ci][tap][co] = w[co][8 - tap][ci]
__global__ void k_flip_weights(__nv_bfloat16* wt, const float* w, int Cin, int Cout) {
    const size_t n = (size_t)Cin * 9 * Cout;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int co = i % Cout;
        const int tap = (i / Cout) % 9;
        const int ci = (int)(i / ((size_t)Cout * 9));
        wt[i] = __float2bfloat16(w[((size_t)co * 9 + (8 - tap)) * Cin + ci]);
    }
}

// mean squared error of pred vs target (f32); dpred (bf16) = 2 (pred - target) / n
// running sum of the step losses (one thread)
__global__ void k_accum_loss(double* sum, const float* loss) { *sum += (double)*loss; }

__global__ void k_mse(const float* pred, const float* target, __nv_bfloat16* dpred, float* loss, size_t n) {
    float s = 0.0f;
    const float inv = 1.0f / (float)n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = pred[i] - target[i];
        s += d * d;
        dpred[i] = __float2bfloat16(2.0f * d * inv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv);
}

// Adam (bias-corrected), f32 master weights
__global__ void k_adam(float* w, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace cnn
}  // namespace inim
