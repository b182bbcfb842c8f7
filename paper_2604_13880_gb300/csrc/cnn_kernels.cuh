// Kernels of the learned warm start: BF16 tensor-core implicit-GEMM 3x3
// convolutions (stride 1, padding 1, NHWC) with FP32 accumulation, their
// weight gradient, and the small element-wise / pooling / optimiser kernels.
//
// Tensor cores: mma.sync.aligned.m16n8k16 (bf16 x bf16 -> f32).  Shared
// tiles hold A as [m][k] and B as [n][k] (k contiguous, rows padded to 40
// elements so that the fragment loads hit distinct banks).  A block computes
// a BM x BN output tile with 4 warps of 32 x 32 (2 x 4 mma tiles each): 64 x 64,
// or 128 x 32 for layers of at most 32 output channels, so that no half of
// the tile is idle; K is walked in steps of 32 with double-buffered shared
// tiles.  Feature maps have power-of-two sides and (past the first layer)
// power-of-two channel counts: pixel and tap indices are shifts and masks.
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
    const __nv_bfloat16* mask;   // nullable: outputs where mask <= 0 are 0 (a ReLU's gradient)
    int lw;                   // log2 W (W = H, a power of two)
    int lc;                   // log2 Cin, or -1 when Cin is not a power of two
};

// the output pixel p as (b, y, x) of a square map of side 2^lw
struct Pix { int b, y, x; bool in; };
__device__ __forceinline__ Pix pix_of(const ConvArgs& a, int p) {
    Pix q;
    q.in = p < (a.B << (2 * a.lw));
    q.x = p & ((1 << a.lw) - 1);
    q.y = (p >> a.lw) & ((1 << a.lw) - 1);
    q.b = p >> (2 * a.lw);
    return q;
}

// one 8-wide k chunk of the im2col row of output pixel q (zero outside)
__device__ __forceinline__ uint4 im2col_chunk_at(const ConvArgs& a, const Pix& q, int k) {
    const int K = 9 * a.Cin;
    const uint4 z = make_uint4(0, 0, 0, 0);
    if (!q.in || k >= K) return z;
    if (a.lc >= 3) {                                   // Cin a power of two >= 8: whole chunks
        const int tap = k >> a.lc, ci = k & (a.Cin - 1);
        const int dy = (tap * 11) >> 5, dx = tap - 3 * dy;   // tap / 3, tap % 3 for tap < 9
        const int yy = q.y + dy - 1, xx = q.x + dx - 1;
        if (yy < 0 || yy >= a.H || xx < 0 || xx >= a.W) return z;
        return *reinterpret_cast<const uint4*>(a.x + ((((size_t)q.b << a.lw) + yy) << a.lw) * a.Cin +
                                               (size_t)xx * a.Cin + ci);
    }
    const int x = q.x, y = q.y, b = q.b;
    // generic (Cin not a power of two of at least 8): element by element
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

__device__ __forceinline__ uint4 im2col_chunk(const ConvArgs& a, int p, int k) {
    return im2col_chunk_at(a, pix_of(a, p), k);
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

template <int BM, int BN>
__global__ void __launch_bounds__(kConvThreads) k_conv3x3_fwd(ConvArgs a) {
    static_assert((BM / 32) * (BN / 32) == kConvThreads / 32, "4 warps of 32 x 32");
    constexpr int WN = BN / 32;                           // warps along N
    constexpr int RA = BM * 4 / kConvThreads;             // A chunks a thread loads per k step
    constexpr int RB = BN * 4 / kConvThreads;             // B chunks
    __shared__ __align__(16) __nv_bfloat16 As[2][BM * kPad];
    __shared__ __align__(16) __nv_bfloat16 Bs[2][BN * kPad];
    const int M = a.B * a.H * a.W, K = 9 * a.Cin;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x, warp = tid >> 5, wm = warp / WN, wn = warp % WN;
    float acc[2][4][4] = {};
    // this thread's A rows (output pixels) do not change along K
    Pix rows[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) rows[r] = pix_of(a, m0 + ((tid + r * kConvThreads) >> 2));
    auto load = [&](int buf, int k0) {
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const int idx = tid + r * kConvThreads;
            const int row = idx >> 2, ch = (idx & 3) * 8;
            *reinterpret_cast<uint4*>(&As[buf][row * kPad + ch]) = im2col_chunk_at(a, rows[r], k0 + ch);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int idx = tid + r * kConvThreads;
            const int row = idx >> 2, ch = (idx & 3) * 8;
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
                if (a.mask) {
                    if (col < a.Cout && !(__bfloat162float(a.mask[(size_t)row * a.Cout + col]) > 0.0f)) v0 = 0.0f;
                    if (col + 1 < a.Cout && !(__bfloat162float(a.mask[(size_t)row * a.Cout + col + 1]) > 0.0f)) v1 = 0.0f;
                }
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

// The same convolution for Cin a power of two >= 8 (every layer but the
// first): the tiles arrive by 16-byte asynchronous copies (cp.async, zero
// fill outside the map) in a three-stage pipeline, and the fragments are read
// with ldmatrix.  Results identical to k_conv3x3_fwd (same products, same
// accumulation order).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const __nv_bfloat16* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(static_cast<unsigned>(__cvta_generic_to_shared(p))));
}

// 32 x 32 warp tile from A [m][kPad] / B [n][kPad] by ldmatrix
__device__ __forceinline__ void warp_mma_tile_ldsm(const __nv_bfloat16* As, const __nv_bfloat16* Bs, int wm, int wn,
                                                   float (&acc)[2][4][4]) {
    const int lane = threadIdx.x & 31;
    const int q = lane >> 3, rr = lane & 7;
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
        unsigned a[2][4], b[4][2];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            // matrices (m, k): (0, 0), (8, 0), (0, 8), (8, 8) -> a0, a1, a2, a3
            const int m = wm * 32 + mi * 16 + rr + ((q & 1) << 3), k = kk + ((q >> 1) << 3);
            ldsm_x4(a[mi], As + m * kPad + k);
        }
#pragma unroll
        for (int np = 0; np < 2; ++np) {
            // matrices (n, k): (0, 0), (0, 8), (8, 0), (8, 8) -> b[2np][0], b[2np][1], b[2np+1][0], b[2np+1][1]
            const int n = wn * 32 + np * 16 + rr + ((q >> 1) << 3), k = kk + ((q & 1) << 3);
            unsigned r[4];
            ldsm_x4(r, Bs + n * kPad + k);
            b[2 * np][0] = r[0]; b[2 * np][1] = r[1]; b[2 * np + 1][0] = r[2]; b[2 * np + 1][1] = r[3];
        }
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni]);
    }
}

constexpr int kFwdStages = 3;

template <int BM, int BN>
__global__ void __launch_bounds__(kConvThreads) k_conv3x3_fwd_async(ConvArgs a) {
    static_assert((BM / 32) * (BN / 32) == kConvThreads / 32, "4 warps of 32 x 32");
    constexpr int WN = BN / 32;
    constexpr int RA = BM * 4 / kConvThreads;
    constexpr int RB = BN * 4 / kConvThreads;
    __shared__ __align__(16) __nv_bfloat16 As[kFwdStages][BM * kPad];
    __shared__ __align__(16) __nv_bfloat16 Bs[kFwdStages][BN * kPad];
    const int M = a.B * a.H * a.W, K = 9 * a.Cin;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x, warp = tid >> 5, wm = warp / WN, wn = warp % WN;
    float acc[2][4][4] = {};
    Pix rows[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) rows[r] = pix_of(a, m0 + ((tid + r * kConvThreads) >> 2));
    auto issue = [&](int buf, int k0) {
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const int idx = tid + r * kConvThreads;
            const int row = idx >> 2, k = k0 + (idx & 3) * 8;
            const Pix& q = rows[r];
            const int tap = k >> a.lc, ci = k & (a.Cin - 1);
            const int dy = (tap * 11) >> 5, dx = tap - 3 * dy;
            const int yy = q.y + dy - 1, xx = q.x + dx - 1;
            const bool ok = q.in && k < K && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            const __nv_bfloat16* src = ok ? a.x + ((((size_t)q.b << a.lw) + yy) << a.lw) * a.Cin + (size_t)xx * a.Cin + ci
                                          : a.x;
            cp_async16(&As[buf][row * kPad + (idx & 3) * 8], src, ok);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int idx = tid + r * kConvThreads;
            const int row = idx >> 2, k = k0 + (idx & 3) * 8;
            const bool ok = n0 + row < a.Cout && k < K;
            const __nv_bfloat16* src = ok ? a.w + (size_t)(n0 + row) * K + k : a.w;
            cp_async16(&Bs[buf][row * kPad + (idx & 3) * 8], src, ok);
        }
    };
    const int nk = (K + kBK - 1) / kBK;
#pragma unroll
    for (int s = 0; s < kFwdStages - 1; ++s) {
        if (s < nk) issue(s, s * kBK);
        cp_async_commit();
    }
    for (int s = 0; s < nk; ++s) {
        cp_async_wait<kFwdStages - 2>();
        __syncthreads();
        warp_mma_tile_ldsm(As[s % kFwdStages], Bs[s % kFwdStages], wm, wn, acc);
        const int nx = s + kFwdStages - 1;
        if (nx < nk) issue(nx % kFwdStages, nx * kBK);
        cp_async_commit();
    }
    cp_async_wait<0>();
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
                if (a.mask) {
                    if (col < a.Cout && !(__bfloat162float(a.mask[(size_t)row * a.Cout + col]) > 0.0f)) v0 = 0.0f;
                    if (col + 1 < a.Cout && !(__bfloat162float(a.mask[(size_t)row * a.Cout + col + 1]) > 0.0f)) v1 = 0.0f;
                }
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
//   blockIdx.z, FP32 atomics into dW).  Both operands are staged pixel-major
//   as they lie in memory (dZ[p][co] and im2col(X)[p][k], 16-byte chunks,
//   rows padded to 72 elements), and the fragments of A = dZ^T and of the
//   column-major B are read with ldmatrix.trans.  64 pixels per stage,
//   double-buffered.
// ---------------------------------------------------------------------------
struct WgradArgs {
    const __nv_bfloat16* dz;   // [P][Cout]
    const __nv_bfloat16* x;    // [B][H][W][Cin]
    float* dw;                 // [Cout][9*Cin]
    float* db;                 // nullable: [Cout] bias gradient (sum of dZ over the pixels), by the blocks of N tile 0
    int B, H, W, Cin, Cout;
    int p_per_split;           // multiple of kWK
    int lw, lc;                // log2 W, log2 Cin (-1: not a power of two)
};

constexpr int kWK = 64;                    // pixels per stage
constexpr int kWPad = 72;                  // padded row (elements) of the pixel-major tiles

__device__ __forceinline__ void ldsm_x4_trans(unsigned (&r)[4], const __nv_bfloat16* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(static_cast<unsigned>(__cvta_generic_to_shared(p))));
}

// 32 x 32 warp tile of A = dZ^T (At [p][co]) times B (Bt [p][k]) over kWK pixels
__device__ __forceinline__ void warp_mma_tile_t(const __nv_bfloat16* At, const __nv_bfloat16* Bt, int wm, int wn,
                                                float (&acc)[2][4][4]) {
    const int lane = threadIdx.x & 31;
    const int q = lane >> 3, rr = lane & 7;          // matrix of the x4 load, row within it
#pragma unroll
    for (int kk = 0; kk < kWK; kk += 16) {
        unsigned a[2][4], b[4][2];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            // matrices (m, k): (0, 0), (8, 0), (0, 8), (8, 8) -> a0, a1, a2, a3
            const int k = kk + rr + ((q >> 1) << 3), m = wm * 32 + mi * 16 + ((q & 1) << 3);
            ldsm_x4_trans(a[mi], At + k * kWPad + m);
        }
#pragma unroll
        for (int np = 0; np < 2; ++np) {
            // matrices (k, n): (0, 0), (8, 0), (0, 8), (8, 8) -> b[2np][0], b[2np][1], b[2np+1][0], b[2np+1][1]
            const int k = kk + rr + ((q & 1) << 3), n = wn * 32 + np * 16 + ((q >> 1) << 3);
            unsigned r[4];
            ldsm_x4_trans(r, Bt + k * kWPad + n);
            b[2 * np][0] = r[0]; b[2 * np][1] = r[1]; b[2 * np + 1][0] = r[2]; b[2 * np + 1][1] = r[3];
        }
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni]);
    }
}

__global__ void __launch_bounds__(kConvThreads) k_conv3x3_wgrad(WgradArgs a) {
    __shared__ __align__(16) __nv_bfloat16 At[2][kWK * kWPad];   // [p][co]
    __shared__ __align__(16) __nv_bfloat16 Bt[2][kWK * kWPad];   // [p][k]
    const int P = a.B * a.H * a.W, K = 9 * a.Cin;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    const int p_begin = blockIdx.z * a.p_per_split;
    const int p_end = min(P, p_begin + a.p_per_split);
    const int tid = threadIdx.x, warp = tid >> 5, wm = warp >> 1, wn = warp & 1;
    float acc[2][4][4] = {};
    ConvArgs ca{};
    ca.x = a.x; ca.B = a.B; ca.H = a.H; ca.W = a.W; ca.Cin = a.Cin; ca.Cout = a.Cout;
    ca.lw = a.lw; ca.lc = a.lc;
    const bool vec_dz = (a.Cout & 7) == 0;
    const bool vec_x = a.lc >= 3;
    const bool bias_blk = a.db != nullptr && blockIdx.y == 0;     // uniform over the block
    float db_acc = 0.0f;
    // a thread stages chunks idx = tid + 128 r (r < 4): pixel idx >> 3, 8 channels / k at (idx & 7) * 8;
    // whole 16-byte chunks by asynchronous copies (zero fill outside), the
    // others (the 2-channel head, the 1-channel input) through registers
    auto load = [&](int buf, int p0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = tid + r * kConvThreads;
            const int pl = idx >> 3, ch = (idx & 7) * 8;
            const int p = p0 + pl;
            const bool pin = p < p_end;
            __nv_bfloat16* da = &At[buf][pl * kWPad + ch];
            if (vec_dz) {
                const bool ok = pin && m0 + ch + 8 <= a.Cout;
                cp_async16(da, ok ? a.dz + (size_t)p * a.Cout + m0 + ch : a.dz, ok);
            } else {
                __align__(16) __nv_bfloat16 v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    v[e] = (pin && m0 + ch + e < a.Cout) ? a.dz[(size_t)p * a.Cout + m0 + ch + e]
                                                         : __float2bfloat16(0.0f);
                *reinterpret_cast<uint4*>(da) = *reinterpret_cast<const uint4*>(v);
            }
            __nv_bfloat16* db = &Bt[buf][pl * kWPad + ch];
            const int k = n0 + ch;
            if (vec_x) {
                const Pix q = pix_of(ca, p);
                const int tap = k >> a.lc, ci = k & (a.Cin - 1);
                const int dy = (tap * 11) >> 5, dx = tap - 3 * dy;
                const int yy = q.y + dy - 1, xx = q.x + dx - 1;
                const bool ok = pin && k < K && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
                cp_async16(db, ok ? a.x + ((((size_t)q.b << a.lw) + yy) << a.lw) * a.Cin + (size_t)xx * a.Cin + ci
                                  : a.x, ok);
            } else {
                *reinterpret_cast<uint4*>(db) = pin ? im2col_chunk(ca, p, k) : make_uint4(0, 0, 0, 0);
            }
        }
    };
    const int ns = (p_end - p_begin + kWK - 1) / kWK;
    if (ns > 0) load(0, p_begin);
    cp_async_commit();
    for (int s = 0; s < ns; ++s) {
        if (s + 1 < ns) load((s + 1) & 1, p_begin + (s + 1) * kWK);     // the buffer of stage s - 1
        cp_async_commit();
        cp_async_wait<1>();                   // this stage's copies (the next stage's may be in flight)
        __syncthreads();
        warp_mma_tile_t(At[s & 1], Bt[s & 1], wm, wn, acc);
        if (bias_blk) {                       // the stage's dZ column sums: two threads a channel
            const __nv_bfloat16* col = At[s & 1] + (tid & 63);
#pragma unroll 8
            for (int p = (tid >> 6); p < kWK; p += 2) db_acc += __bfloat162float(col[p * kWPad]);
        }
        __syncthreads();
    }
    cp_async_wait<0>();
    if (bias_blk) {
        __shared__ float dbs[kConvThreads];
        dbs[tid] = db_acc;
        __syncthreads();
        const int co = m0 + tid;
        if (tid < 64 && co < a.Cout) atomicAdd(&a.db[co], dbs[tid] + dbs[tid + 64]);
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
