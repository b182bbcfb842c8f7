// The learned warm start: an encoder-decoder CNN that maps the start map's
// density texture (log(d/d0), 512^2, average-pooled to 64^2 by the density
// kernel) to the 2-channel total displacement the InIm iteration would
// produce, on a 64^2 lattice.  BF16 activations and weights on the tensor
// cores, FP32 accumulation, FP32 master weights, Adam.
//
//   64^2:  conv 1->32, conv 32->32 (e1) -> pool
//   32^2:  conv 32->64, conv 64->64 (e2) -> pool
//   16^2:  conv 64->128, conv 128->128 (e3) -> pool
//    8^2:  conv 128->256 (bottleneck) -> up
//   16^2:  conv 256->128 + e3, conv 128->128 -> up
//   32^2:  conv 128->64 + e2, conv 64->64 -> up
//   64^2:  conv 64->32 + e1, conv 32->32, conv 32->2 (linear)
// Every conv is 3x3, stride 1, padding 1, followed by ReLU except the last;
// pooling is 2x2 average, up-sampling nearest.  1,163,234 parameters.
//
// Input resolution: 64^2 by default; a network created with a 128^2 or
// 256^2 input (the density texture pooled less) runs its first convolution
// (1 -> 32) at that resolution and average-pools its output down to 64^2
// (a stem), the rest unchanged: the same parameters, more detail seen by
// the first layer.
#include <cmath>
#include <cstring>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "cnn_kernels.cuh"
#include "inim_internal.cuh"

using namespace inim;
using namespace inim::cnn;

namespace {

struct LayerSpec { int cin, cout, res, relu; };
constexpr int kLayers = 14;
constexpr LayerSpec kSpec[kLayers] = {
    {1, 32, 64, 1},    {32, 32, 64, 1},   {32, 64, 32, 1},   {64, 64, 32, 1},  {64, 128, 16, 1},
    {128, 128, 16, 1}, {128, 256, 8, 1},  {256, 128, 16, 1}, {128, 128, 16, 1}, {128, 64, 32, 1},
    {64, 64, 32, 1},   {64, 32, 64, 1},   {32, 32, 64, 1},   {32, 2, 64, 0}};
constexpr int kRes = 64;

size_t w_count(int l) { return (size_t)kSpec[l].cout * 9 * kSpec[l].cin; }

size_t total_params() {
    size_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += w_count(l) + kSpec[l].cout;
    return n;
}

thread_local std::string g_cnn_err;

int cfail(int code, const std::string& m) {
    g_cnn_err = m;
    return code;
}

#define CK(expr)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) return cfail(INIM_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

int grid_for(size_t n) {
    size_t g = (n + 255) / 256;
    return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

}  // namespace

struct inim_cnn {
    // parameters: one f32 blob [layer: W (cout*9*cin), b (cout)]*, grads, Adam moments
    float* params = nullptr;
    float* grads = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    size_t n_params = 0;
    size_t w_off[kLayers], b_off[kLayers];
    __nv_bfloat16* wb[kLayers] = {};     // bf16 weights [cout][9][cin]
    __nv_bfloat16* wf[kLayers] = {};     // bf16 flipped weights [cin][9][cout] (data gradient)
    int step = 0;
    int in_res = 64;                     // input resolution: 64, 128 or 256
    int stem = 0;                        // log2(in_res / 64): pools after the first convolution
    // stem tensors (stem > 0): [0] the input (1 channel, in_res^2), [1 + k]
    // the first convolution's output pooled k times (32 channels)
    std::vector<__nv_bfloat16*> s_act, s_grd;
    // activations / gradients for a batch of B
    int B = 0;
    std::vector<__nv_bfloat16*> act, grd;
    float* out = nullptr;                // [B][64][64][2]
    float* loss = nullptr;               // device scalar
    double* loss_sum = nullptr;          // device: sum of the step losses since the last read
    int loss_steps = 0;                  // steps in loss_sum
    float* xin = nullptr;                // training inputs copied on the caller's stream
    float* yin = nullptr;
    int in_B = 0;                        // batch the copies are sized for
    cudaEvent_t ev_in = nullptr;         // the copies are done (caller's stream)
    cudaEvent_t ev_done = nullptr;       // the last step's kernels are done (network's stream)
    cudaStream_t stream = nullptr;

    ~inim_cnn() {
        release_batch();
        for (int l = 0; l < kLayers; ++l) { dfree(wb[l]); dfree(wf[l]); }
        dfree(params); dfree(grads); dfree(m1); dfree(m2); dfree(loss); dfree(loss_sum); dfree(xin); dfree(yin);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_done) cudaEventDestroy(ev_done);
        if (stream) cudaStreamDestroy(stream);
    }
    void release_batch() {
        for (auto& p : act) dfree(p);
        for (auto& p : grd) dfree(p);
        for (auto& p : s_act) dfree(p);
        for (auto& p : s_grd) dfree(p);
        act.clear(); grd.clear(); s_act.clear(); s_grd.clear();
        dfree(out);
        B = 0;
    }
};

namespace {

// activation tensors (name = index): per tensor its resolution and channels
enum T {
    X0, A0, E1, P1, A2, E2, P2, A4, E3, P3, BT, U3, Z7, D3, D3B, U2, Z9, D2, D2B, U1, Z11, D1, D1B, NT
};
constexpr int kTRes[NT] = {64, 64, 64, 32, 32, 32, 16, 16, 16, 8, 8, 16, 16, 16, 16, 32, 32, 32, 32, 64, 64, 64, 64};
constexpr int kTCh[NT] = {1, 32, 32, 32, 64, 64, 64, 128, 128, 128, 256, 256, 128, 128, 128, 128, 64, 64, 64, 64, 32, 32, 32};

size_t tsize(int t, int B) { return (size_t)B * kTRes[t] * kTRes[t] * kTCh[t]; }

int ensure_batch(inim_cnn& c, int B) {
    if (c.B >= B) return INIM_OK;
    c.release_batch();
    c.act.assign(NT, nullptr);
    c.grd.assign(NT, nullptr);
    for (int t = 0; t < NT; ++t) {
        CK(cudaMalloc(&c.act[t], tsize(t, B) * sizeof(__nv_bfloat16)));
        CK(cudaMalloc(&c.grd[t], tsize(t, B) * sizeof(__nv_bfloat16)));
    }
    if (c.stem > 0) {
        c.s_act.assign(c.stem + 1, nullptr);
        c.s_grd.assign(c.stem + 1, nullptr);
        for (int k = 0; k <= c.stem; ++k) {
            const size_t r = (size_t)(k == 0 ? c.in_res : c.in_res >> (k - 1));
            const size_t n = (size_t)B * r * r * (k == 0 ? 1 : 32);
            CK(cudaMalloc(&c.s_act[k], n * sizeof(__nv_bfloat16)));
            CK(cudaMalloc(&c.s_grd[k], n * sizeof(__nv_bfloat16)));
        }
    }
    CK(cudaMalloc(&c.out, (size_t)B * kRes * kRes * 2 * sizeof(float)));
    c.B = B;
    return INIM_OK;
}

cudaError_t refresh_bf16(inim_cnn& c) {
    for (int l = 0; l < kLayers; ++l) {
        const size_t n = w_count(l);
        k_to_bf16<<<grid_for(n), 256, 0, c.stream>>>(c.wb[l], c.params + c.w_off[l], n);
        k_flip_weights<<<grid_for(n), 256, 0, c.stream>>>(c.wf[l], c.params + c.w_off[l], kSpec[l].cin, kSpec[l].cout);
    }
    return cudaGetLastError();
}

// log2 of a power of two, -1 otherwise
int ilog2_exact(int v) {
    if (v <= 0 || (v & (v - 1))) return -1;
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

void conv(inim_cnn& c, int B, int res, const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias, int cin,
          int cout, int relu, __nv_bfloat16* y, float* yf, const __nv_bfloat16* mask = nullptr) {
    ConvArgs a{};
    a.x = x; a.w = w; a.bias = bias; a.y_bf16 = y; a.y_f32 = yf; a.mask = mask;
    a.B = B; a.H = res; a.W = res; a.Cin = cin; a.Cout = cout; a.relu = relu;
    a.lw = ilog2_exact(res);
    a.lc = ilog2_exact(cin);
    const int M = B * res * res;
    const bool async = a.lc >= 3;      // whole 16-byte chunks: the asynchronous-copy kernel
    if (cout <= 32) {                  // 128 x 32 tiles: no idle half for the 32-channel layers
        dim3 grid((M + 127) / 128, (cout + 31) / 32);
        if (async) k_conv3x3_fwd_async<128, 32><<<grid, kConvThreads, 0, c.stream>>>(a);
        else k_conv3x3_fwd<128, 32><<<grid, kConvThreads, 0, c.stream>>>(a);
    } else {
        dim3 grid((M + kBM - 1) / kBM, (cout + kBN - 1) / kBN);
        if (async) k_conv3x3_fwd_async<kBM, kBN><<<grid, kConvThreads, 0, c.stream>>>(a);
        else k_conv3x3_fwd<kBM, kBN><<<grid, kConvThreads, 0, c.stream>>>(a);
    }
}

void layer_fwd(inim_cnn& c, int l, int B, const __nv_bfloat16* x, __nv_bfloat16* y, float* yf = nullptr,
               int res = 0) {
    const LayerSpec& s = kSpec[l];
    conv(c, B, res ? res : s.res, x, c.wb[l], c.params + c.b_off[l], s.cin, s.cout, s.relu, y, yf);
}

// weight / bias gradient of layer l from dz (already masked) and its input x;
// the data gradient into dx when dx != nullptr
// dx_mask: the ReLU output whose gradient dx is (dx is zeroed where it is
// <= 0, in the data-gradient convolution's epilogue), or nullptr
void layer_bwd(inim_cnn& c, int l, int B, const __nv_bfloat16* dz, const __nv_bfloat16* x, __nv_bfloat16* dx,
               int res_override = 0, const __nv_bfloat16* dx_mask = nullptr) {
    LayerSpec s = kSpec[l];
    if (res_override) s.res = res_override;
    const int P = B * s.res * s.res;
    WgradArgs a{};
    a.dz = dz; a.x = x; a.dw = c.grads + c.w_off[l];
    a.B = B; a.H = s.res; a.W = s.res; a.Cin = s.cin; a.Cout = s.cout;
    a.lw = ilog2_exact(s.res);
    a.lc = ilog2_exact(s.cin);
    const int splits = std::max(1, std::min(256, P / 2048));
    a.p_per_split = ((P + splits - 1) / splits + kWK - 1) / kWK * kWK;
    dim3 grid((s.cout + kBM - 1) / kBM, (9 * s.cin + kBN - 1) / kBN, (P + a.p_per_split - 1) / a.p_per_split);
    a.db = c.grads + c.b_off[l];              // the bias gradient rides along (N tile 0)
    k_conv3x3_wgrad<<<grid, kConvThreads, 0, c.stream>>>(a);
    if (dx) conv(c, B, s.res, dz, c.wf[l], nullptr, s.cout, s.cin, 0, dx, nullptr, dx_mask);
}

void relu_grad(inim_cnn& c, int t, int B) {
    const size_t n = tsize(t, B);
    k_relu_grad<<<grid_for(n), 256, 0, c.stream>>>(c.grd[t], c.act[t], n);
}

// forward of the whole network for a batch of B pooled inputs x (f32 [B][64][64])
int forward(inim_cnn& c, const float* x, int B) {
    int st = ensure_batch(c, B);
    if (st != INIM_OK) return st;
    auto& A = c.act;
    if (c.stem > 0) {
        // stem: the first convolution at the input resolution, then 2x2
        // average pools down to 64^2
        auto& S = c.s_act;
        const size_t n0 = (size_t)B * c.in_res * c.in_res;
        k_to_bf16<<<grid_for(n0), 256, 0, c.stream>>>(S[0], x, n0);
        layer_fwd(c, 0, B, S[0], S[1], nullptr, c.in_res);
        for (int k = 1; k <= c.stem; ++k) {
            const int r = c.in_res >> (k - 1);
            __nv_bfloat16* dst = k == c.stem ? A[A0] : S[k + 1];
            k_pool2<<<grid_for((size_t)B * (r / 2) * (r / 2) * 32), 256, 0, c.stream>>>(dst, S[k], B, r, r, 32);
        }
    } else {
        const size_t n0 = (size_t)B * kRes * kRes;
        k_to_bf16<<<grid_for(n0), 256, 0, c.stream>>>(A[X0], x, n0);
        layer_fwd(c, 0, B, A[X0], A[A0]);
    }
    layer_fwd(c, 1, B, A[A0], A[E1]);
    k_pool2<<<grid_for(tsize(P1, B)), 256, 0, c.stream>>>(A[P1], A[E1], B, 64, 64, 32);
    layer_fwd(c, 2, B, A[P1], A[A2]);
    layer_fwd(c, 3, B, A[A2], A[E2]);
    k_pool2<<<grid_for(tsize(P2, B)), 256, 0, c.stream>>>(A[P2], A[E2], B, 32, 32, 64);
    layer_fwd(c, 4, B, A[P2], A[A4]);
    layer_fwd(c, 5, B, A[A4], A[E3]);
    k_pool2<<<grid_for(tsize(P3, B)), 256, 0, c.stream>>>(A[P3], A[E3], B, 16, 16, 128);
    layer_fwd(c, 6, B, A[P3], A[BT]);
    k_up2<<<grid_for(tsize(U3, B)), 256, 0, c.stream>>>(A[U3], A[BT], B, 8, 8, 256);
    layer_fwd(c, 7, B, A[U3], A[Z7]);
    k_add<<<grid_for(tsize(D3, B)), 256, 0, c.stream>>>(A[D3], A[Z7], A[E3], tsize(D3, B));
    layer_fwd(c, 8, B, A[D3], A[D3B]);
    k_up2<<<grid_for(tsize(U2, B)), 256, 0, c.stream>>>(A[U2], A[D3B], B, 16, 16, 128);
    layer_fwd(c, 9, B, A[U2], A[Z9]);
    k_add<<<grid_for(tsize(D2, B)), 256, 0, c.stream>>>(A[D2], A[Z9], A[E2], tsize(D2, B));
    layer_fwd(c, 10, B, A[D2], A[D2B]);
    k_up2<<<grid_for(tsize(U1, B)), 256, 0, c.stream>>>(A[U1], A[D2B], B, 32, 32, 64);
    layer_fwd(c, 11, B, A[U1], A[Z11]);
    k_add<<<grid_for(tsize(D1, B)), 256, 0, c.stream>>>(A[D1], A[Z11], A[E1], tsize(D1, B));
    layer_fwd(c, 12, B, A[D1], A[D1B]);
    layer_fwd(c, 13, B, A[D1B], nullptr, c.out);
    CK(cudaGetLastError());
    return INIM_OK;
}

// loss and gradients (into c.grads) for targets y (f32 [B][64][64][2])
int backward(inim_cnn& c, const float* y, int B) {
    auto& A = c.act;
    auto& G = c.grd;
    CK(cudaMemsetAsync(c.grads, 0, c.n_params * sizeof(float), c.stream));
    CK(cudaMemsetAsync(c.loss, 0, sizeof(float), c.stream));
    const size_t no = (size_t)B * kRes * kRes * 2;
    // the head's output gradient reuses the X0 gradient buffer (B*64*64*2 bf16 fits in U1's)
    __nv_bfloat16* gout = G[U1];
    k_mse<<<grid_for(no), 256, 0, c.stream>>>(c.out, y, gout, c.loss, no);
    layer_bwd(c, 13, B, gout, A[D1B], G[D1B], 0, A[D1B]);
    layer_bwd(c, 12, B, G[D1B], A[D1], G[D1]);             // d1 = z11 + e1
    CK(cudaMemcpyAsync(G[Z11], G[D1], tsize(D1, B) * 2, cudaMemcpyDeviceToDevice, c.stream));
    relu_grad(c, Z11, B);
    layer_bwd(c, 11, B, G[Z11], A[U1], G[U1]);
    k_up2_grad<<<grid_for(tsize(D2B, B)), 256, 0, c.stream>>>(G[D2B], G[U1], B, 32, 32, 64);
    relu_grad(c, D2B, B);
    layer_bwd(c, 10, B, G[D2B], A[D2], G[D2]);             // d2 = z9 + e2
    CK(cudaMemcpyAsync(G[Z9], G[D2], tsize(D2, B) * 2, cudaMemcpyDeviceToDevice, c.stream));
    relu_grad(c, Z9, B);
    layer_bwd(c, 9, B, G[Z9], A[U2], G[U2]);
    k_up2_grad<<<grid_for(tsize(D3B, B)), 256, 0, c.stream>>>(G[D3B], G[U2], B, 16, 16, 128);
    relu_grad(c, D3B, B);
    layer_bwd(c, 8, B, G[D3B], A[D3], G[D3]);              // d3 = z7 + e3
    CK(cudaMemcpyAsync(G[Z7], G[D3], tsize(D3, B) * 2, cudaMemcpyDeviceToDevice, c.stream));
    relu_grad(c, Z7, B);
    layer_bwd(c, 7, B, G[Z7], A[U3], G[U3]);
    k_up2_grad<<<grid_for(tsize(BT, B)), 256, 0, c.stream>>>(G[BT], G[U3], B, 8, 8, 256);
    relu_grad(c, BT, B);
    layer_bwd(c, 6, B, G[BT], A[P3], G[P3]);
    k_pool2_grad<<<grid_for(tsize(E3, B)), 256, 0, c.stream>>>(G[E3], G[P3], B, 16, 16, 128);
    k_accum<<<grid_for(tsize(E3, B)), 256, 0, c.stream>>>(G[E3], G[D3], tsize(E3, B));   // skip into d3
    relu_grad(c, E3, B);
    layer_bwd(c, 5, B, G[E3], A[A4], G[A4], 0, A[A4]);
    layer_bwd(c, 4, B, G[A4], A[P2], G[P2]);
    k_pool2_grad<<<grid_for(tsize(E2, B)), 256, 0, c.stream>>>(G[E2], G[P2], B, 32, 32, 64);
    k_accum<<<grid_for(tsize(E2, B)), 256, 0, c.stream>>>(G[E2], G[D2], tsize(E2, B));   // skip into d2
    relu_grad(c, E2, B);
    layer_bwd(c, 3, B, G[E2], A[A2], G[A2], 0, A[A2]);
    layer_bwd(c, 2, B, G[A2], A[P1], G[P1]);
    k_pool2_grad<<<grid_for(tsize(E1, B)), 256, 0, c.stream>>>(G[E1], G[P1], B, 64, 64, 32);
    k_accum<<<grid_for(tsize(E1, B)), 256, 0, c.stream>>>(G[E1], G[D1], tsize(E1, B));   // skip into d1
    relu_grad(c, E1, B);
    layer_bwd(c, 1, B, G[E1], A[A0], G[A0], 0, c.stem > 0 ? nullptr : A[A0]);
    if (c.stem > 0) {
        // back through the stem's pools to the first convolution's output,
        // its ReLU mask, and its weights at the input resolution
        auto& S = c.s_act;
        auto& GS = c.s_grd;
        for (int k = c.stem; k >= 1; --k) {
            const int r = c.in_res >> (k - 1);
            const __nv_bfloat16* src = k == c.stem ? G[A0] : GS[k + 1];
            k_pool2_grad<<<grid_for((size_t)B * r * r * 32), 256, 0, c.stream>>>(GS[k], src, B, r, r, 32);
        }
        const size_t n1 = (size_t)B * c.in_res * c.in_res * 32;
        k_relu_grad<<<grid_for(n1), 256, 0, c.stream>>>(GS[1], S[1], n1);
        layer_bwd(c, 0, B, GS[1], S[0], nullptr, c.in_res);
    } else {
        layer_bwd(c, 0, B, G[A0], A[X0], nullptr);
    }
    CK(cudaGetLastError());
    return INIM_OK;
}

std::mutex g_ws_mu;
inim_cnn* g_warmstart = nullptr;      // network used by params.warm_start

}  // namespace

namespace inim {
// prediction for the solver's warm start: pooled inputs [B][64][64] -> fields [B][64][64][2]
int warmstart_predict(const float* x, int B, float* y, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if (!g_warmstart) return INIM_E_STATE;
    inim_cnn& c = *g_warmstart;
    cudaEvent_t in;
    cudaEventCreateWithFlags(&in, cudaEventDisableTiming);
    cudaEventRecord(in, s);                 // the inputs are produced on s
    cudaStreamWaitEvent(c.stream, in, 0);
    cudaEventDestroy(in);
    int st = forward(c, x, B);
    if (st != INIM_OK) return st;
    if (cudaMemcpyAsync(y, c.out, (size_t)B * kRes * kRes * 2 * sizeof(float), cudaMemcpyDeviceToDevice, c.stream) !=
        cudaSuccess)
        return INIM_E_CUDA;
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, c.stream);
    cudaStreamWaitEvent(s, ev, 0);
    cudaEventDestroy(ev);
    return INIM_OK;
}
bool warmstart_loaded() { return g_warmstart != nullptr; }
int warmstart_input_res() {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    return g_warmstart ? g_warmstart->in_res : kRes;
}
}  // namespace inim

extern "C" {

int inim_cnn_create_res(int32_t seed, int32_t in_res, inim_cnn** out) {
    if (!out) return cfail(INIM_E_ARG, "out is NULL");
    if (in_res != 64 && in_res != 128 && in_res != 256) return cfail(INIM_E_ARG, "input resolution must be 64, 128 or 256");
    auto c = new inim_cnn();
    c->in_res = in_res;
    c->stem = in_res == 256 ? 2 : (in_res == 128 ? 1 : 0);
    size_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        c->w_off[l] = off;
        off += w_count(l);
        c->b_off[l] = off;
        off += kSpec[l].cout;
    }
    c->n_params = off;
    std::vector<float> h(off, 0.0f);
    std::mt19937_64 rng((uint64_t)seed);
    for (int l = 0; l < kLayers; ++l) {
        // He initialisation for the ReLU layers, small for the linear head
        const double fan_in = 9.0 * kSpec[l].cin;
        const double sd = kSpec[l].relu ? std::sqrt(2.0 / fan_in) : 0.1 * std::sqrt(1.0 / fan_in);
        std::normal_distribution<double> nd(0.0, sd);
        for (size_t k = 0; k < w_count(l); ++k) h[c->w_off[l] + k] = (float)nd(rng);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->params, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->grads, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->m1, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->m2, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->loss_sum, sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(c->loss_sum, 0, sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming);
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
        e = cudaMalloc(&c->wb[l], w_count(l) * 2);
        if (e == cudaSuccess) e = cudaMalloc(&c->wf[l], w_count(l) * 2);
    }
    // everything on the network's own (non-blocking) stream, which orders it
    // before the kernels that follow
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->params, h.data(), off * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->m1, 0, off * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->m2, 0, off * 4, c->stream);
    if (e == cudaSuccess) e = refresh_bf16(*c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        delete c;
        return cfail(INIM_E_CUDA, std::string("cnn create: ") + cudaGetErrorString(e));
    }
    *out = c;
    return INIM_OK;
}

int inim_cnn_create(int32_t seed, inim_cnn** out) { return inim_cnn_create_res(seed, kRes, out); }

int inim_cnn_input_res(const inim_cnn* c) { return c ? c->in_res : 0; }

int inim_cnn_destroy(inim_cnn* c) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if (c == g_warmstart) g_warmstart = nullptr;
    delete c;
    return INIM_OK;
}

long long inim_cnn_num_params(const inim_cnn* c) { return c ? (long long)c->n_params : (long long)total_params(); }

int inim_cnn_get_params(const inim_cnn* c, float* out, long long n) {
    if (!c || !out || n != (long long)c->n_params) return cfail(INIM_E_ARG, "bad arguments");
    CK(cudaMemcpyAsync(out, c->params, c->n_params * 4, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return INIM_OK;
}

int inim_cnn_set_params(inim_cnn* c, const float* in, long long n) {
    if (!c || !in || n != (long long)c->n_params) return cfail(INIM_E_ARG, "bad arguments");
    CK(cudaMemcpyAsync(c->params, in, c->n_params * 4, cudaMemcpyDefault, c->stream));
    CK(cudaMemsetAsync(c->m1, 0, c->n_params * 4, c->stream));
    CK(cudaMemsetAsync(c->m2, 0, c->n_params * 4, c->stream));
    c->step = 0;
    CK(refresh_bf16(*c));
    CK(cudaStreamSynchronize(c->stream));
    return INIM_OK;
}

int inim_cnn_forward(inim_cnn* c, const float* x, int32_t B, float* y, void* stream) {
    if (!c || !x || !y || B < 1) return cfail(INIM_E_ARG, "bad arguments");
    CK(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    int st = forward(*c, x, B);
    if (st != INIM_OK) return st;
    CK(cudaMemcpyAsync(y, c->out, (size_t)B * kRes * kRes * 2 * 4, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return INIM_OK;
}

int inim_cnn_gradients(inim_cnn* c, const float* x, const float* y, int32_t B, float* loss, float* grads,
                       void* stream) {
    if (!c || !x || !y || B < 1) return cfail(INIM_E_ARG, "bad arguments");
    CK(cudaStreamSynchronize((cudaStream_t)stream));   // the caller's earlier work (NULL: legacy stream)
    int st = forward(*c, x, B);
    if (st == INIM_OK) st = backward(*c, y, B);
    if (st != INIM_OK) return st;
    if (loss) CK(cudaMemcpyAsync(loss, c->loss, 4, cudaMemcpyDeviceToHost, c->stream));
    if (grads) CK(cudaMemcpyAsync(grads, c->grads, c->n_params * 4, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return INIM_OK;
}

int inim_cnn_train_step(inim_cnn* c, const float* x, const float* y, int32_t B, float lr, float* loss,
                        void* stream) {
    if (!c || !x || !y || B < 1 || !(lr > 0.0f)) return cfail(INIM_E_ARG, "bad arguments");
    cudaStream_t cs = (cudaStream_t)stream;
    const size_t nx = (size_t)B * c->in_res * c->in_res, ny = (size_t)B * kRes * kRes * 2;
    if (c->in_B < B) {
        CK(cudaStreamSynchronize(c->stream));
        dfree(c->xin);
        dfree(c->yin);
        CK(cudaMalloc(&c->xin, nx * sizeof(float)));
        CK(cudaMalloc(&c->yin, ny * sizeof(float)));
        c->in_B = B;
    }
    // the inputs are copied on the caller's stream (after its producers; the
    // caller may free or reuse its buffers in that stream's order), once the
    // previous step no longer reads the copies; the step runs on the
    // network's stream after the copies, and the host does not wait for it
    CK(cudaStreamWaitEvent(cs, c->ev_done, 0));
    CK(cudaMemcpyAsync(c->xin, x, nx * sizeof(float), cudaMemcpyDefault, cs));
    CK(cudaMemcpyAsync(c->yin, y, ny * sizeof(float), cudaMemcpyDefault, cs));
    CK(cudaEventRecord(c->ev_in, cs));
    CK(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
    int st = forward(*c, c->xin, B);
    if (st == INIM_OK) st = backward(*c, c->yin, B);
    if (st != INIM_OK) return st;
    c->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)c->step), c2 = 1.0f - std::pow(b2, (float)c->step);
    k_adam<<<grid_for(c->n_params), 256, 0, c->stream>>>(c->params, c->grads, c->m1, c->m2, c->n_params, lr, b1, b2,
                                                         1e-8f, c1, c2);
    k_accum_loss<<<1, 1, 0, c->stream>>>(c->loss_sum, c->loss);
    c->loss_steps += 1;
    CK(refresh_bf16(*c));
    CK(cudaEventRecord(c->ev_done, c->stream));
    if (loss) {
        CK(cudaMemcpyAsync(loss, c->loss, 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return INIM_OK;
}

int inim_cnn_loss_mean(inim_cnn* c, double* mean) {
    if (!c || !mean) return cfail(INIM_E_ARG, "bad arguments");
    double sum = 0.0;
    CK(cudaMemcpyAsync(&sum, c->loss_sum, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemsetAsync(c->loss_sum, 0, sizeof(double), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *mean = c->loss_steps > 0 ? sum / c->loss_steps : 0.0;
    c->loss_steps = 0;
    return INIM_OK;
}

const char* inim_cnn_last_error(void) { return g_cnn_err.c_str(); }

int inim_warmstart_load_res(const void* weights, size_t bytes, int32_t in_res) {
    const size_t n = total_params();
    if (!weights || bytes != n * sizeof(float)) return cfail(INIM_E_ARG, "weights must be the f32 parameter blob");
    inim_cnn* c = nullptr;
    int st = inim_cnn_create_res(0, in_res, &c);
    if (st != INIM_OK) return st;
    st = inim_cnn_set_params(c, static_cast<const float*>(weights), (long long)n);
    if (st != INIM_OK) { inim_cnn_destroy(c); return st; }
    std::lock_guard<std::mutex> lk(g_ws_mu);
    delete g_warmstart;
    g_warmstart = c;
    return INIM_OK;
}

int inim_warmstart_load(const void* weights, size_t bytes) { return inim_warmstart_load_res(weights, bytes, kRes); }

}  // extern "C"
