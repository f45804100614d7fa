// Learned temporal interpolator (C ABI in include/neurosim_evsim.h,
// "Learned interpolator"): a 3-level convolutional U-Net that predicts the
// three log-intensity frames between two keyframes 4 frame periods apart, so
// that a renderer can run at a quarter of the event camera's frame rate.
// Every convolution, transposed convolution and their data and weight
// gradients run as BF16 tcgen05 GEMMs with FP32 accumulation in TMEM
// (umma_gemm.cuh, interp_layers.cuh); loss, bias gradients, AdamW and weight
// packing are small CUDA-core kernels.  The paper has no counterpart: it
// renders every frame (Sec. 2); the network is this project's.
//
// Network (activations BF16 NHWC; concatenations share one buffer):
//   x  = [L0, L4 - L0, 0 x 6]                                   P   x 8
//   e1 = relu(conv3(x, W1) + b1)        -> cat1[:, 32:64]        P   x 32
//   e2 = relu(conv3s2(e1, W2) + b2)     -> cat2[:, 64:128]       P/4 x 64
//   e3 = relu(conv3s2(e2, W3) + b3)                              P/16 x 128
//   e4 = relu(conv3(e3, W4) + b4)                                P/16 x 128
//   u1 = convT2(e4, W5) + b5            -> cat2[:, 0:64]         P/4 x 64
//   d1 = relu(conv3(cat2, W6) + b6)                              P/4 x 64
//   u2 = convT2(d1, W7) + b7            -> cat1[:, 0:32]         P   x 32
//   d2 = relu(conv3(cat1, W8) + b8)                              P   x 32
//   L_j = L0 + j/4 (L4 - L0) + (d2 W9 + b9)_j,  j = 1..3          FP32
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"
#include "interp_layers.cuh"
#include "umma_mn.cuh"
#include "umma_tma.cuh"

using namespace interp;

namespace {

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return nsim::report_error(code, buf);
}

#define ICUDA(expr)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(NEUROSIM_E_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                           \
    } while (0)

// ---- parameters: one flat FP32 array, weights first, then biases ---------------------
enum LayerKind { CONV, CONVT, FINAL };
struct LayerDef {
    LayerKind kind;
    int cin, cout;
};
constexpr int kLayers = 9;
constexpr LayerDef kDefs[kLayers] = {
    {CONV, 8, 32},   {CONV, 32, 64},  {CONV, 64, 128}, {CONV, 128, 128}, {CONVT, 128, 64},
    {CONV, 128, 64}, {CONVT, 64, 32}, {CONV, 64, 32},  {FINAL, 32, 16},
};

constexpr int64_t weight_count(const LayerDef& d)
{
    return d.kind == CONV ? 9ll * d.cin * d.cout : d.kind == CONVT ? 4ll * d.cin * d.cout : (int64_t)d.cin * d.cout;
}

struct ParamLayout {
    int64_t w_off[kLayers], b_off[kLayers];
    int64_t n_weights = 0, total = 0;
    ParamLayout()
    {
        int64_t o = 0;
        for (int l = 0; l < kLayers; ++l) {
            w_off[l] = o;
            o += weight_count(kDefs[l]);
        }
        n_weights = o;
        for (int l = 0; l < kLayers; ++l) {
            b_off[l] = o;
            o += kDefs[l].cout;
        }
        total = o;
    }
};

// ---- CUDA-core kernels -------------------------------------------------------------
__global__ void pack_input_kernel(const float* L0, const float* L4, int64_t plane_stride, int HW, int P, bf16* x0,
                                  float* l0c, float* l4c)
{
    // L0 / L4 of image n at L0 + n * plane_stride (keyframes inside a clip array)
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const int n = p / HW, q = p - n * HW;
        const float a = L0[(size_t)n * plane_stride + q], b = L4[(size_t)n * plane_stride + q];
        l0c[p] = a;
        l4c[p] = b;
        float v[8] = {a, b - a, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        *reinterpret_cast<uint4*>(x0 + (size_t)p * 8) = pack8(v);
    }
}

// Charbonnier loss over out [3][P] against the targets (frames 1..3 of each
// clip) and its gradient, written as BF16 [P][16] (columns 3..15 zero).
__global__ void loss_kernel(const float* out, const float* clips, int HW, int P, float inv_count, bf16* gr,
                            double* loss_sum)
{
    __shared__ double s_part[32];
    double acc = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const int n = p / HW, q = p - n * HW;
        float g[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float d = out[(size_t)j * P + p] - clips[((size_t)n * 5 + 1 + j) * HW + q];
            const float s = sqrtf(d * d + 1e-6f);
            acc += (double)s;
            g[j] = d / s * inv_count;
        }
        uint4* dst = reinterpret_cast<uint4*>(gr + (size_t)p * 16);
        dst[0] = pack8(g);
        dst[1] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
        atomicAdd(loss_sum, t);
    }
}

// db[c] += sum over rows of g[row * stride + off + c], c < C (C divides 256).
__global__ void bias_grad_kernel(const bf16* g, int rows, int stride, int off, int C, float* db)
{
    __shared__ float s[256];
    const int c = threadIdx.x % C, grp = threadIdx.x / C, G = blockDim.x / C;
    float acc = 0.0f;
    for (int r = blockIdx.x * G + grp; r < rows; r += gridDim.x * G)
        acc += __bfloat162float(g[(size_t)r * stride + off + c]);
    s[threadIdx.x] = acc;
    __syncthreads();
    if (grp == 0) {
        for (int k = 1; k < G; ++k) acc += s[k * C + c];
        atomicAdd(db + c, acc);
    }
}

// AdamW on the flat parameters; decoupled weight decay on [0, n_weights).
__global__ void adamw_kernel(float* w, const float* g, float* m, float* v, int64_t n, int64_t n_weights, float lr,
                             float wd, float b1, float b2, float eps, float bc1, float bc2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float upd = (mi / bc1) / (sqrtf(vi / bc2) + eps);
        if (i < n_weights) upd += wd * w[i];
        w[i] -= lr * upd;
    }
}

// BF16 GEMM operands of one layer from its FP32 master weights:
//   fwd [N_f][K_f]: conv [cout][tap * cin + c], convT [(ab) * cout + o][cin], final [j][cin]
//   bwd [N_b][K_b]: conv [cin][tap * cout + o], convT [cin][ab * cout + o], final [cin][j]
__global__ void pack_weights_kernel(const float* w, int kind, int cin, int cout, bf16* fwd, bf16* bwd)
{
    const int taps = kind == CONV ? 9 : kind == CONVT ? 4 : 1;
    const int n = taps * cin * cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // master index i = (tap * cin + c) * cout + o  (conv, final: tap = 0)
        //                  c * (4 cout) + ab * cout + o  (convT)
        int tap, c, o;
        if (kind == CONVT) {
            c = i / (4 * cout);
            const int r = i - c * 4 * cout;
            tap = r / cout;
            o = r - tap * cout;
        } else {
            o = i % cout;
            const int tc = i / cout;
            tap = tc / cin;
            c = tc - tap * cin;
        }
        const bf16 val = __float2bfloat16_rn(w[i]);
        if (kind == CONVT) {
            fwd[(size_t)(tap * cout + o) * cin + c] = val;
            bwd[(size_t)c * (4 * cout) + tap * cout + o] = val;
        } else {
            fwd[(size_t)o * (taps * cin) + tap * cin + c] = val;
            bwd[(size_t)c * (taps * cout) + tap * cout + o] = val;
        }
    }
}

// He-normal initial weights (fan-in), zero final layer and biases: the
// untrained network is linear interpolation.  Normal draws: Irwin-Hall(12)
// of SplitMix64 outputs, counter-based by parameter index.
__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1ull) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void init_weights_kernel(float* w, int64_t n, float scale, int64_t base, uint64_t seed, int kind, int cin,
                                    int cout, int zero_pad_in)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t acc = 0;
        for (int k = 0; k < 12; ++k) acc += (int64_t)(sm64(seed, (uint64_t)(base + i) * 12ull + k) >> 44);
        float z = (float)(acc - 6ll * (1ll << 20)) * 0x1p-20f;
        const int c = kind == CONVT ? (int)(i / (4 * cout)) : (int)((i / cout) % cin);
        if (c >= zero_pad_in) z = 0.0f;
        w[i] = z * scale;
    }
}

unsigned grid_for(int64_t n, int threads = 256)
{
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 4096));
}

}  // namespace

struct neurosim_interp {
    cudaStream_t stream = nullptr;
    int device = 0, sms = 0;
    int64_t Pmax = 0;
    ParamLayout lay;
    float* params = nullptr;   // master FP32
    float* grads = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    bf16* wf[kLayers] = {};    // forward GEMM operands
    bf16* wb[kLayers] = {};    // backward-data GEMM operands
    int64_t step = 0;
    // activations (BF16 NHWC) and their gradients
    bf16 *x0 = nullptr, *cat1 = nullptr, *cat2 = nullptr, *e3 = nullptr, *e4 = nullptr, *d1 = nullptr, *d2 = nullptr;
    bf16 *gcat1 = nullptr, *gcat2 = nullptr, *ge3 = nullptr, *ge4 = nullptr, *gd1 = nullptr, *gd2 = nullptr,
         *gr = nullptr;
    float *l0 = nullptr, *l4 = nullptr, *out = nullptr;
    double* loss = nullptr;
    unsigned int* err = nullptr;
    uint64_t launches = 0;
};

namespace {

template <class T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

void release(neurosim_interp* h)
{
    void* ptrs[] = {h->params, h->grads, h->m, h->v, h->x0, h->cat1, h->cat2, h->e3, h->e4, h->d1, h->d2,
                    h->gcat1, h->gcat2, h->ge3, h->ge4, h->gd1, h->gd2, h->gr, h->l0, h->l4, h->out, h->loss,
                    h->err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < kLayers; ++l) {
        if (h->wf[l]) cudaFree(h->wf[l]);
        if (h->wb[l]) cudaFree(h->wb[l]);
    }
}

// ---- GEMM dispatch -------------------------------------------------------------------
template <int BN, class AG, class BG, class EP>
cudaError_t gemm_bn(neurosim_interp* h, const AG& a, const BG& b, const EP& ep, int M, int N, int K, int splits,
                    int k_per_split)
{
    ugemm::GemmArgs<AG, BG, EP> g;
    g.a = a;
    g.b = b;
    g.ep = ep;
    g.M = M;
    g.N = N;
    g.K = K;
    g.k_per_split = k_per_split;
    g.err = h->err;
    g.limit_ns = 2000000000ull;
    h->launches += 1;
    return ugemm::launch_gemm<BN>(g, splits, h->stream);
}

// D[M x N] = A * B over K; `split_k` spreads K over CTAs (weight gradients).
template <class AG, class BG, class EP>
cudaError_t gemm(neurosim_interp* h, const AG& a, const BG& b, const EP& ep, int M, int N, int K, bool split_k)
{
    int splits = 1, kps = ((K + ugemm::BK - 1) / ugemm::BK) * ugemm::BK;
    if (split_k) {
        const int mt = (M + ugemm::BM - 1) / ugemm::BM;
        const int want = std::max(1, (4 * h->sms + mt - 1) / mt);
        const int kt = (K + ugemm::BK - 1) / ugemm::BK;
        const int per = std::max(1, (kt + want - 1) / want);
        kps = per * ugemm::BK;
        splits = (K + kps - 1) / kps;
    }
    if (N <= 16) return gemm_bn<16>(h, a, b, ep, M, N, K, splits, kps);
    if (N <= 32) return gemm_bn<32>(h, a, b, ep, M, N, K, splits, kps);
    if (N <= 64) return gemm_bn<64>(h, a, b, ep, M, N, K, splits, kps);
    if (N <= 128) return gemm_bn<128>(h, a, b, ep, M, N, K, splits, kps);
    return gemm_bn<256>(h, a, b, ep, M, N, K, splits, kps);
}

// ---- TMA path for 3x3 stride-1 convolutions over >= 64 channels ---------------------
// Output tile TW x TH pixels (TW * TH = 128) chosen to waste the fewest rows.
void pick_tile(int W, int H, int* TW, int* TH)
{
    int best = -1;
    for (int tw = 128; tw >= 8; tw >>= 1) {
        const int th = 128 / tw;
        const long long tiles = (long long)((W + tw - 1) / tw) * ((H + th - 1) / th);
        const long long waste = tiles * 128 - (long long)W * H;
        if (best < 0 || waste < best) {
            best = (int)waste;
            *TW = tw;
            *TH = th;
        }
    }
}

template <int BN, int SW, class EP>
cudaError_t conv_tma_bn(neurosim_interp* h, const bf16* buf, int cstride, int off, int C, int flip, int N, int H,
                        int W, const bf16* wpacked, int n_out, const EP& ep, int stride)
{
    constexpr int BKS = utma::bk_of(SW);
    if (stride != 1 && (stride != 2 || flip)) return cudaErrorInvalidValue;
    int TW = 128, TH = 1;
    pick_tile(W, H, &TW, &TH);
    utma::TmaArgs<utma::ConvTapA, EP> g;
    // the input is stride x the output size
    const int Wi = stride * W, Hi = stride * H;
    const cuuint64_t dims[4] = {(cuuint64_t)cstride, (cuuint64_t)Wi, (cuuint64_t)Hi, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)cstride * 2u, (cuuint64_t)Wi * cstride * 2u,
                                   (cuuint64_t)Hi * Wi * cstride * 2u};
    const cuuint32_t box[4] = {(cuuint32_t)BKS, (cuuint32_t)(stride * TW), (cuuint32_t)(stride * TH), 1u};
    const cuuint32_t estr[4] = {1u, (cuuint32_t)stride, (cuuint32_t)stride, 1u};
    if (!utma::encode_tiled(&g.ta, 4, buf, dims, strides, box, SW, estr) ||
        !utma::encode_kmajor(&g.tb, wpacked, n_out, 9 * C, BN, SW))
        return cudaErrorInvalidValue;
    const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH;
    g.a = utma::ConvTapA{C, off, flip, W, H, N, TW, TH, tx, ty, BKS, stride};
    g.ep = ep;
    g.N = n_out;
    g.err = h->err;
    g.limit_ns = 2000000000ull;
    h->launches += 1;
    return utma::launch_tma_gemm<BN, SW>(g, N * tx * ty, h->stream);
}

// Data gradient of a 2x2 stride-2 transposed convolution: g (Cout channels at
// `off` of rows of `cstride`, 2H x 2W per image) through the packed backward
// weights [cin][ab * Cout + o] into the low-resolution epilogue (H x W), one
// TMA GEMM over the four sub-positions (S2DTapA).  Cout: 32 (64-byte swizzle)
// or a multiple of 64.
template <int BN, int SW, class EP>
cudaError_t convt_dgrad_bn(neurosim_interp* h, const bf16* g, int cstride, int off, int Cout, int N, int H, int W,
                           const bf16* wpacked, int n_out, const EP& ep)
{
    constexpr int BKS = utma::bk_of(SW);
    if (Cout % BKS) return cudaErrorInvalidValue;
    int TW = 128, TH = 1;
    pick_tile(W, H, &TW, &TH);
    utma::TmaArgs<utma::S2DTapA, EP> a;
    const cuuint64_t dims[4] = {(cuuint64_t)cstride, (cuuint64_t)(2 * W), (cuuint64_t)(2 * H), (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)cstride * 2u, (cuuint64_t)(2 * W) * cstride * 2u,
                                   (cuuint64_t)(4 * H * W) * cstride * 2u};
    const cuuint32_t box[4] = {(cuuint32_t)BKS, (cuuint32_t)(2 * TW), (cuuint32_t)(2 * TH), 1u};
    const cuuint32_t estr[4] = {1u, 2u, 2u, 1u};
    if (!utma::encode_tiled(&a.ta, 4, g, dims, strides, box, SW, estr) ||
        !utma::encode_kmajor(&a.tb, wpacked, n_out, 4 * Cout, BN, SW))
        return cudaErrorInvalidValue;
    const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH;
    a.a = utma::S2DTapA{Cout, off, W, H, N, TW, TH, tx, ty, BKS};
    a.ep = ep;
    a.N = n_out;
    a.err = h->err;
    a.limit_ns = 2000000000ull;
    h->launches += 1;
    return utma::launch_tma_gemm<BN, SW>(a, N * tx * ty, h->stream);
}

// Data gradient of a 3x3 stride-2 convolution: g (Cout channels at `off` of
// rows of `cstride`, Ho x Wo per image) through the packed backward weights
// [cin][tap * Cout + o] into the input-size epilogue, as four tcgen05 GEMMs,
// one per parity class of the input pixels (ParityTapA): every product is
// one of the convolution's, none is a zero of the stride.
template <int BN, class EP>
cudaError_t conv_s2_dgrad_bn(neurosim_interp* h, const bf16* g, int cstride, int off, int Cout, int N, int Ho, int Wo,
                             const bf16* wpacked, int n_out, const EP& ep)
{
    constexpr int SW = 128, BKS = utma::bk_of(SW);
    if (Cout % BKS) return cudaErrorInvalidValue;
    int TW = 128, TH = 1;
    pick_tile(Wo, Ho, &TW, &TH);
    const int tx = (Wo + TW - 1) / TW, ty = (Ho + TH - 1) / TH;
    utma::TmaArgs<utma::ParityTapA, EP> a;
    const cuuint64_t dims[4] = {(cuuint64_t)cstride, (cuuint64_t)Wo, (cuuint64_t)Ho, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)cstride * 2u, (cuuint64_t)Wo * cstride * 2u,
                                   (cuuint64_t)Ho * Wo * cstride * 2u};
    const cuuint32_t box[4] = {(cuuint32_t)BKS, (cuuint32_t)TW, (cuuint32_t)TH, 1u};
    if (!utma::encode_tiled(&a.ta, 4, g, dims, strides, box, SW) ||
        !utma::encode_kmajor(&a.tb, wpacked, n_out, 9 * Cout, BN, SW))
        return cudaErrorInvalidValue;
    a.ep = ep;
    a.N = n_out;
    a.err = h->err;
    a.limit_ns = 2000000000ull;
    for (int py = 0; py < 2; ++py)
        for (int px = 0; px < 2; ++px) {
            utma::ParityTapA& L = a.a;
            L = utma::ParityTapA{};
            L.Cout = Cout;
            L.off = off;
            L.Wo = Wo;
            L.Ho = Ho;
            L.N = N;
            L.py = py;
            L.px = px;
            L.TW = TW;
            L.TH = TH;
            L.tiles_x = tx;
            L.tiles_y = ty;
            L.bk = BKS;
            // taps of the class: dy = 1 (oy 0) for py = 0; dy = 0 (oy 1), 2 (oy 0) for py = 1
            const int ndy = py ? 2 : 1, ndx = px ? 2 : 1;
            for (int i = 0; i < ndy; ++i)
                for (int j = 0; j < ndx; ++j) {
                    const int dy = py ? 2 * i : 1, dx = px ? 2 * j : 1;
                    L.tap[L.ntaps] = 3 * dy + dx;
                    L.oy[L.ntaps] = (py && dy == 0) ? 1 : 0;
                    L.ox[L.ntaps] = (px && dx == 0) ? 1 : 0;
                    ++L.ntaps;
                }
            h->launches += 1;
            const cudaError_t e = utma::launch_tma_gemm<BN, SW>(a, N * tx * ty, h->stream);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

// out = conv3x3 (stride 1) of the view [off, off + C) of `buf` from halo
// tiles of 128-pixel rows (W >= 128; C 8 (forward), 32 with a 64-byte swizzle
// of the weights, or 64 with a 128-byte swizzle).
template <int BN, int SW, int SWA, int CC, class EP>
cudaError_t conv_halo_bn(neurosim_interp* h, const bf16* buf, int cstride, int off, int C, int flip, int N, int H,
                         int W, const bf16* wpacked, int n_out, const EP& ep)
{
    utma::HaloArgs<EP> g;
    const cuuint64_t dims[4] = {(cuuint64_t)cstride, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)cstride * 2u, (cuuint64_t)W * cstride * 2u,
                                   (cuuint64_t)H * W * cstride * 2u};
    const cuuint32_t box[4] = {SWA ? (cuuint32_t)(SWA / 2) : 8u, (cuuint32_t)utma::kHaloW, 3u, 1u};
    if (!utma::encode_tiled(&g.ta, 4, buf, dims, strides, box, SWA) ||
        !utma::encode_kmajor(&g.tb, wpacked, n_out, 9 * C, BN, SW))
        return cudaErrorInvalidValue;
    g.ep = ep;
    g.C = C;
    g.off = off;
    g.flip = flip;
    g.W = W;
    g.H = H;
    g.N = N;
    g.n_tiles = N * H * ((W + 127) / 128);
    g.n_out = n_out;
    g.err = h->err;
    g.limit_ns = 2000000000ull;
    h->launches += 1;
    return utma::launch_halo_conv<BN, SW, SWA, CC>(g, h->sms, h->stream);
}

// As conv_halo_bn with the weights streamed per (tap, 64-channel) K tile, for
// inputs whose weights do not fit resident (C a multiple of 64).
template <int BN, int CC, class EP>
cudaError_t conv_halo_stream_bn(neurosim_interp* h, const bf16* buf, int cstride, int off, int flip, int N, int H,
                                int W, const bf16* wpacked, int n_out, const EP& ep)
{
    utma::HaloArgs<EP> g;
    const cuuint64_t dims[4] = {(cuuint64_t)cstride, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)cstride * 2u, (cuuint64_t)W * cstride * 2u,
                                   (cuuint64_t)H * W * cstride * 2u};
    const cuuint32_t box[4] = {64u, (cuuint32_t)utma::kHaloW, 3u, 1u};
    if (!utma::encode_tiled(&g.ta, 4, buf, dims, strides, box, 128) ||
        !utma::encode_kmajor(&g.tb, wpacked, n_out, 9 * CC, BN, 128))
        return cudaErrorInvalidValue;
    g.ep = ep;
    g.C = CC;
    g.off = off;
    g.flip = flip;
    g.W = W;
    g.H = H;
    g.N = N;
    g.n_tiles = N * H * ((W + 127) / 128);
    g.n_out = n_out;
    g.err = h->err;
    g.limit_ns = 2000000000ull;
    h->launches += 1;
    return utma::launch_halo_conv_stream<BN, CC>(g, h->sms, h->stream);
}

// out (H x W) = conv3x3 with padding 1 and the given stride of the view
// [off, off + C) of `buf` (stride H x stride W); flip = 1 for the data
// gradient (taps mirrored, stride 1).  C must be a multiple of 64 (128-byte
// swizzle) or equal 32 (64-byte swizzle).
template <class EP>
cudaError_t conv_tma(neurosim_interp* h, const bf16* buf, int cstride, int off, int C, int flip, int N, int H, int W,
                     const bf16* wpacked, int n_out, const EP& ep, int stride = 1)
{
    if (stride == 1 && W >= 128 && n_out <= 128 && ((C == 128) || (C == 64 && n_out > 64))) {
        if (C == 128)
            return n_out <= 64 ? conv_halo_stream_bn<64, 128>(h, buf, cstride, off, flip, N, H, W, wpacked, n_out, ep)
                               : conv_halo_stream_bn<128, 128>(h, buf, cstride, off, flip, N, H, W, wpacked, n_out, ep);
        return conv_halo_stream_bn<128, 64>(h, buf, cstride, off, flip, N, H, W, wpacked, n_out, ep);
    }
    if (stride == 1 && W >= 128 && n_out <= 64 && (C == 32 || C == 64 || (C == 8 && !flip && n_out <= 32))) {
        if (C == 8)
            return conv_halo_bn<32, 128, 0, 8>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep);
        if (C == 32)
            return n_out <= 32 ? conv_halo_bn<32, 64, 64, 32>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep)
                               : conv_halo_bn<64, 64, 64, 32>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep);
        return n_out <= 32 ? conv_halo_bn<32, 128, 128, 64>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep)
                           : conv_halo_bn<64, 128, 128, 64>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep);
    }
    if (C == 32) {
        if (n_out <= 32) return conv_tma_bn<32, 64>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep, stride);
        if (n_out <= 64) return conv_tma_bn<64, 64>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep, stride);
        return conv_tma_bn<128, 64>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep, stride);
    }
    if (n_out <= 32) return conv_tma_bn<32, 128>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep, stride);
    if (n_out <= 64) return conv_tma_bn<64, 128>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep, stride);
    return conv_tma_bn<128, 128>(h, buf, cstride, off, C, flip, N, H, W, wpacked, n_out, ep, stride);
}

// out[P][n_out] = view [off, off + C) of the rows of a [P][cstride] buffer
// times the packed [n_out][C] weights (1x1 layers, transposed-conv
// forward).  C: 32 (64-byte swizzle) or a multiple of 64.
template <int BN, int SW, class EP>
cudaError_t pix_tma_bn(neurosim_interp* h, const bf16* buf, int cstride, int off, int C, int P, const bf16* wpacked,
                       int n_out, const EP& ep)
{
    if constexpr (BN > 32) {
        // the transposed convolutions: epilogue-heavy scatters, faster with many
        // short-lived CTAs per SM (43.2 / 56.4 us persistent against 34.0 /
        // 46.4 us on 256^2 crops)
        utma::TmaArgs<utma::DenseA, EP> g;
        if (!utma::encode_kmajor(&g.ta, buf, P, cstride, utma::BM, SW, cstride) ||
            !utma::encode_kmajor(&g.tb, wpacked, n_out, C, BN, SW))
            return cudaErrorInvalidValue;
        g.a = utma::DenseA{P, C, off, utma::bk_of(SW)};
        g.ep = ep;
        g.N = n_out;
        g.err = h->err;
        g.limit_ns = 2000000000ull;
        h->launches += 1;
        return utma::launch_tma_gemm<BN, SW>(g, (P + utma::BM - 1) / utma::BM, h->stream);
    } else {
        // the final 1x1 layer: persistent, weights resident, A tiles through a ring,
        // two accumulators (42.7 -> 18.5 us on 256^2 crops)
        utma::PixArgs<EP> g;
        if (!utma::encode_kmajor(&g.ta, buf, P, cstride, utma::BM, SW, cstride) ||
            !utma::encode_kmajor(&g.tb, wpacked, n_out, C, BN, SW))
            return cudaErrorInvalidValue;
        g.ep = ep;
        g.M = P;
        g.K = C;
        g.off = off;
        g.n_tiles = (P + utma::BM - 1) / utma::BM;
        g.n_out = n_out;
        g.err = h->err;
        g.limit_ns = 2000000000ull;
        h->launches += 1;
        return utma::launch_pix_gemm<BN, SW>(g, h->sms, h->stream);
    }
}

struct Shape {
    int N, H, W;        // batch and full size
    int P, P2, P4;      // pixels at full, half and quarter size
};

Act act(const bf16* p, int N, int H, int W, int stride, int off) { return Act{p, N, H, W, stride, off}; }

int log2i(int c)
{
    int k = 0;
    while ((1 << k) < c) ++k;
    return k;
}
Conv3K conv3k(Act x, int C, int Ho, int Wo, int s, int M) { return Conv3K{x, C, Ho, Wo, s, M, log2i(C)}; }

const float* bias_of(const neurosim_interp* h, int l) { return h->params + h->lay.b_off[l]; }

int pack_all(neurosim_interp* h)
{
    for (int l = 0; l < kLayers; ++l) {
        const LayerDef& d = kDefs[l];
        pack_weights_kernel<<<grid_for(weight_count(d)), 256, 0, h->stream>>>(h->params + h->lay.w_off[l], d.kind,
                                                                            d.cin, d.cout, h->wf[l], h->wb[l]);
        h->launches += 1;
    }
    ICUDA(cudaGetLastError());
    return NEUROSIM_OK;
}

// Forward pass; L0 / L4 planes of image n at L0 + n * plane_stride.
int forward(neurosim_interp* h, const Shape& s, const float* L0, const float* L4, int64_t plane_stride)
{
    const int N = s.N, H = s.H, W = s.W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    pack_input_kernel<<<grid_for(s.P), 256, 0, h->stream>>>(L0, L4, plane_stride, H * W, s.P, h->x0, h->l0, h->l4);
    h->launches += 1;
    ICUDA(cudaGetLastError());
    // e1 -> cat1[:, 32:64]
    if (W >= 128)
        ICUDA(conv_tma(h, h->x0, 8, 0, 8, 0, N, H, W, h->wf[0], 32, EpiAct{h->cat1, 64, 32, bias_of(h, 0), 1}));
    else
        ICUDA(gemm(h, conv3k(act(h->x0, N, H, W, 8, 0), 8, H, W, 1, s.P), ugemm::DenseK{h->wf[0], 32, 72},
                   EpiAct{h->cat1, 64, 32, bias_of(h, 0), 1}, s.P, 32, 72, false));
    // e2 -> cat2[:, 64:128]
    ICUDA(conv_tma(h, h->cat1, 64, 32, 32, 0, N, H2, W2, h->wf[1], 64, EpiAct{h->cat2, 128, 64, bias_of(h, 1), 1}, 2));
    // e3
    ICUDA(conv_tma(h, h->cat2, 128, 64, 64, 0, N, H4, W4, h->wf[2], 128, EpiAct{h->e3, 128, 0, bias_of(h, 2), 1}, 2));
    // e4
    ICUDA(conv_tma(h, h->e3, 128, 0, 128, 0, N, H4, W4, h->wf[3], 128, EpiAct{h->e4, 128, 0, bias_of(h, 3), 1}));
    // u1 -> cat2[:, 0:64]
    ICUDA((pix_tma_bn<256, 128>(h, h->e4, 128, 0, 128, s.P4, h->wf[4], 256,
                                 EpiConvT{h->cat2, 128, 0, bias_of(h, 4), 64, H4, W4})));
    // d1
    ICUDA(conv_tma(h, h->cat2, 128, 0, 128, 0, N, H2, W2, h->wf[5], 64, EpiAct{h->d1, 64, 0, bias_of(h, 5), 1}));
    // u2 -> cat1[:, 0:32]
    ICUDA((pix_tma_bn<128, 128>(h, h->d1, 64, 0, 64, s.P2, h->wf[6], 128,
                                 EpiConvT{h->cat1, 64, 0, bias_of(h, 6), 32, H2, W2})));
    // d2
    ICUDA(conv_tma(h, h->cat1, 64, 0, 64, 0, N, H, W, h->wf[7], 32, EpiAct{h->d2, 32, 0, bias_of(h, 7), 1}));
    // frames
    ICUDA((pix_tma_bn<16, 64>(h, h->d2, 32, 0, 32, s.P, h->wf[8], 16, EpiOut{h->out, h->l0, h->l4, bias_of(h, 8), s.P})));
    return NEUROSIM_OK;
}

// ---- weight gradients over pixels with TMA-loaded MN-major operands ------------------
template <int BN>
int dw_mn_bn(neurosim_interp* h, const Act& xa, const umn::MnOp& a, const Act& xb, const umn::MnOp& b, int Ho, int Wo,
             float* dw, int M, int N, bool* done)
{
    umn::MnArgs<BN> g;
    g.a = a;
    g.b = b;
    if (!umn::encode_op(&g.ta, xa.p, xa.stride, xa.W, xa.H, xa.N, a) ||
        !umn::encode_op(&g.tb, xb.p, xb.stride, xb.W, xb.H, xb.N, b))
        return NEUROSIM_OK;                       // not done: the gather form runs instead
    const int runs = (Wo + umn::KT - 1) / umn::KT;
    g.geom = umn::MnGeom{Ho, Wo, runs, xa.N * Ho * runs};
    g.M = M;
    g.N = N;
    g.dw = dw;
    g.err = h->err;
    g.limit_ns = 2000000000ull;
    h->launches += 1;
    // one wave: two CTAs per SM fit with up to 64 gradient columns
    ICUDA(umn::launch_mn_gemm<BN>(g, (BN <= 64 ? 2 : 1) * h->sms, h->stream));
    *done = true;
    return NEUROSIM_OK;
}

// The halo form for 3x3 stride-1 convolutions over 64-channel parts with up
// to 64 gradient columns: all 9 taps of a part from one halo per pixel run.
template <int BN>
int dw_halo_bn(neurosim_interp* h, const Act& xa, int C, const Act& xb, const umn::MnOp& b, int Ho, int Wo, float* dw,
               int N, bool* done)
{
    umn::MnHaloArgs<BN> g;
    if (!umn::encode_halo(&g.ta, xa.p, xa.stride, xa.W, xa.H, xa.N) ||
        !umn::encode_op(&g.tb, xb.p, xb.stride, xb.W, xb.H, xb.N, b))
        return NEUROSIM_OK;
    const int runs = (Wo + umn::KT - 1) / umn::KT;
    g.C = C;
    g.off = xa.off;
    g.b = b;
    g.geom = umn::MnGeom{Ho, Wo, runs, xa.N * Ho * runs};
    g.N = N;
    g.dw = dw;
    g.err = h->err;
    g.limit_ns = 2000000000ull;
    h->launches += 1;
    ICUDA(umn::launch_mn_halo<BN>(g, h->sms, h->stream));
    *done = true;
    return NEUROSIM_OK;
}

// dw[M x N] += sum over the pixel grid (batch, Ho, Wo) of A(m, p) B(n, p): A
// is operand kind akind over the view xa (aC channels per tap, stride as),
// B kind bkind over xb (bC channels).  Pixel runs narrower than 64 take the
// gather GEMM `fallback` instead.
template <class Fallback>
int weight_grad(neurosim_interp* h, Act xa, int akind, int aC, int as, Act xb, int bkind, int bC, int Ho, int Wo,
                float* dw, int M, int N, Fallback&& fallback)
{
    bool done = false;
    int rc = NEUROSIM_OK;
    if (Wo >= umn::KT && N % 16 == 0 && N <= 256) {
        const umn::MnOp a{akind, aC, xa.off, as, M, umn::pick_sw(aC)};
        const umn::MnOp b{bkind, bC, xb.off, 1, N, umn::pick_sw(bC)};
        if (akind == umn::kConv3 && as == 1 && aC % 64 == 0 && bkind == umn::kPix && N <= 64)
            rc = N <= 32 ? dw_halo_bn<32>(h, xa, aC, xb, b, Ho, Wo, dw, N, &done)
                         : dw_halo_bn<64>(h, xa, aC, xb, b, Ho, Wo, dw, N, &done);
        if (rc || done) return rc;
        rc = N <= 16 ? dw_mn_bn<16>(h, xa, a, xb, b, Ho, Wo, dw, M, N, &done)
             : N <= 32 ? dw_mn_bn<32>(h, xa, a, xb, b, Ho, Wo, dw, M, N, &done)
             : N <= 64 ? dw_mn_bn<64>(h, xa, a, xb, b, Ho, Wo, dw, M, N, &done)
             : N <= 128 ? dw_mn_bn<128>(h, xa, a, xb, b, Ho, Wo, dw, M, N, &done)
                        : dw_mn_bn<256>(h, xa, a, xb, b, Ho, Wo, dw, M, N, &done);
    }
    if (rc || done) return rc;
    ICUDA(fallback());
    return NEUROSIM_OK;
}

int bias_grad(neurosim_interp* h, const bf16* g, int rows, int stride, int off, int C, int layer)
{
    const int G = 256 / C;
    const unsigned blocks = (unsigned)std::max(1, std::min(4 * h->sms, (rows + G * 64 - 1) / (G * 64)));
    bias_grad_kernel<<<blocks, 256, 0, h->stream>>>(g, rows, stride, off, C, h->grads + h->lay.b_off[layer]);
    h->launches += 1;
    ICUDA(cudaGetLastError());
    return NEUROSIM_OK;
}

// Backward pass after forward() and the loss kernel (gradient of the three
// outputs in h->gr); accumulates every parameter gradient into h->grads.
int backward(neurosim_interp* h, const Shape& s)
{
    const int N = s.N, H = s.H, W = s.W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    float* G = h->grads;
    const ParamLayout& L = h->lay;
    int rc;
    ICUDA(cudaMemsetAsync(G, 0, (size_t)L.total * sizeof(float), h->stream));
    // ---- final 1x1: W9, b9, d(d2)
    if ((rc = weight_grad(h, act(h->d2, N, H, W, 32, 0), umn::kPix, 32, 1, act(h->gr, N, H, W, 16, 0), umn::kPix, 16, H,
                          W, G + L.w_off[8], 32, 16, [&] {
                              return gemm(h, PixMN{act(h->d2, N, H, W, 32, 0), 32, s.P},
                                          PixMN{act(h->gr, N, H, W, 16, 0), 16, s.P}, EpiDW{G + L.w_off[8], 16}, 32,
                                          16, s.P, true);
                          })))
        return rc;
    if ((rc = bias_grad(h, h->gr, s.P, 16, 0, 16, 8))) return rc;
    ICUDA(gemm(h, PixK{act(h->gr, N, H, W, 16, 0), s.P}, ugemm::DenseK{h->wb[8], 32, 16},
               EpiGrad{h->gd2, 32, 0, h->d2, 32, 0, 0, 0}, s.P, 32, 16, false));
    // ---- conv8 (cat1 -> d2): W8, b8, d(cat1) (u2 linear, e1 masked)
    if ((rc = weight_grad(h, act(h->cat1, N, H, W, 64, 0), umn::kConv3, 64, 1, act(h->gd2, N, H, W, 32, 0), umn::kPix,
                          32, H, W, G + L.w_off[7], 576, 32, [&] {
                              return gemm(h, Im2colMN{act(h->cat1, N, H, W, 64, 0), 64, H, W, 1, 576, s.P},
                                          PixMN{act(h->gd2, N, H, W, 32, 0), 32, s.P}, EpiDW{G + L.w_off[7], 32}, 576,
                                          32, s.P, true);
                          })))
        return rc;
    if ((rc = bias_grad(h, h->gd2, s.P, 32, 0, 32, 7))) return rc;
    ICUDA(conv_tma(h, h->gd2, 32, 0, 32, 1, N, H, W, h->wb[7], 64, EpiGrad{h->gcat1, 64, 0, h->cat1, 64, 0, 32, 0}));
    // ---- convT2 (d1 -> u2): W7, b7, d(d1)
    if ((rc = weight_grad(h, act(h->d1, N, H2, W2, 64, 0), umn::kPix, 64, 1, act(h->gcat1, N, H, W, 64, 0), umn::kS2D,
                          32, H2, W2, G + L.w_off[6], 64, 128, [&] {
                              return gemm(h, PixMN{act(h->d1, N, H2, W2, 64, 0), 64, s.P2},
                                          S2DMN{act(h->gcat1, N, H, W, 64, 0), 32, H2, W2, 128, s.P2},
                                          EpiDW{G + L.w_off[6], 128}, 64, 128, s.P2, true);
                          })))
        return rc;
    if ((rc = bias_grad(h, h->gcat1, s.P, 64, 0, 32, 6))) return rc;
    ICUDA((convt_dgrad_bn<64, 64>(h, h->gcat1, 64, 0, 32, N, H2, W2, h->wb[6], 64,
                                  EpiGrad{h->gd1, 64, 0, h->d1, 64, 0, 0, 0})));
    // ---- conv6 (cat2 -> d1): W6, b6, d(cat2) (u1 linear, e2 masked)
    if ((rc = weight_grad(h, act(h->cat2, N, H2, W2, 128, 0), umn::kConv3, 128, 1, act(h->gd1, N, H2, W2, 64, 0),
                          umn::kPix, 64, H2, W2, G + L.w_off[5], 1152, 64, [&] {
                              return gemm(h, Im2colMN{act(h->cat2, N, H2, W2, 128, 0), 128, H2, W2, 1, 1152, s.P2},
                                          PixMN{act(h->gd1, N, H2, W2, 64, 0), 64, s.P2}, EpiDW{G + L.w_off[5], 64},
                                          1152, 64, s.P2, true);
                          })))
        return rc;
    if ((rc = bias_grad(h, h->gd1, s.P2, 64, 0, 64, 5))) return rc;
    ICUDA(conv_tma(h, h->gd1, 64, 0, 64, 1, N, H2, W2, h->wb[5], 128, EpiGrad{h->gcat2, 128, 0, h->cat2, 128, 0, 64, 0}));
    // ---- convT1 (e4 -> u1): W5, b5, d(e4)
    if ((rc = weight_grad(h, act(h->e4, N, H4, W4, 128, 0), umn::kPix, 128, 1, act(h->gcat2, N, H2, W2, 128, 0),
                          umn::kS2D, 64, H4, W4, G + L.w_off[4], 128, 256, [&] {
                              return gemm(h, PixMN{act(h->e4, N, H4, W4, 128, 0), 128, s.P4},
                                          S2DMN{act(h->gcat2, N, H2, W2, 128, 0), 64, H4, W4, 256, s.P4},
                                          EpiDW{G + L.w_off[4], 256}, 128, 256, s.P4, true);
                          })))
        return rc;
    if ((rc = bias_grad(h, h->gcat2, s.P2, 128, 0, 64, 4))) return rc;
    ICUDA((convt_dgrad_bn<128, 128>(h, h->gcat2, 128, 0, 64, N, H4, W4, h->wb[4], 128,
                                    EpiGrad{h->ge4, 128, 0, h->e4, 128, 0, 0, 0})));
    // ---- conv4 (e3 -> e4): W4, b4, d(e3)
    if ((rc = weight_grad(h, act(h->e3, N, H4, W4, 128, 0), umn::kConv3, 128, 1, act(h->ge4, N, H4, W4, 128, 0),
                          umn::kPix, 128, H4, W4, G + L.w_off[3], 1152, 128, [&] {
                              return gemm(h, Im2colMN{act(h->e3, N, H4, W4, 128, 0), 128, H4, W4, 1, 1152, s.P4},
                                          PixMN{act(h->ge4, N, H4, W4, 128, 0), 128, s.P4},
                                          EpiDW{G + L.w_off[3], 128}, 1152, 128, s.P4, true);
                          })))
        return rc;
    if ((rc = bias_grad(h, h->ge4, s.P4, 128, 0, 128, 3))) return rc;
    ICUDA(conv_tma(h, h->ge4, 128, 0, 128, 1, N, H4, W4, h->wb[3], 128, EpiGrad{h->ge3, 128, 0, h->e3, 128, 0, 0, 0}));
    // ---- conv3 (e2 -> e3, stride 2): W3, b3, d(e2) added into d(cat2)[:, 64:128]
    if ((rc = weight_grad(h, act(h->cat2, N, H2, W2, 128, 64), umn::kConv3, 64, 2, act(h->ge3, N, H4, W4, 128, 0),
                          umn::kPix, 128, H4, W4, G + L.w_off[2], 576, 128, [&] {
                              return gemm(h, Im2colMN{act(h->cat2, N, H2, W2, 128, 64), 64, H4, W4, 2, 576, s.P4},
                                          PixMN{act(h->ge3, N, H4, W4, 128, 0), 128, s.P4},
                                          EpiDW{G + L.w_off[2], 128}, 576, 128, s.P4, true);
                          })))
        return rc;
    if ((rc = bias_grad(h, h->ge3, s.P4, 128, 0, 128, 2))) return rc;
    ICUDA((conv_s2_dgrad_bn<64>(h, h->ge3, 128, 0, 128, N, H4, W4, h->wb[2], 64,
                                EpiGrad{h->gcat2, 128, 64, h->cat2, 128, 64, 0, 1})));
    // ---- conv2 (e1 -> e2, stride 2): W2, b2, d(e1) added into d(cat1)[:, 32:64]
    if ((rc = weight_grad(h, act(h->cat1, N, H, W, 64, 32), umn::kConv3, 32, 2, act(h->gcat2, N, H2, W2, 128, 64),
                          umn::kPix, 64, H2, W2, G + L.w_off[1], 288, 64, [&] {
                              return gemm(h, Im2colMN{act(h->cat1, N, H, W, 64, 32), 32, H2, W2, 2, 288, s.P2},
                                          PixMN{act(h->gcat2, N, H2, W2, 128, 64), 64, s.P2},
                                          EpiDW{G + L.w_off[1], 64}, 288, 64, s.P2, true);
                          })))
        return rc;
    if ((rc = bias_grad(h, h->gcat2, s.P2, 128, 64, 64, 1))) return rc;
    ICUDA((conv_s2_dgrad_bn<32>(h, h->gcat2, 128, 64, 64, N, H2, W2, h->wb[1], 32,
                                EpiGrad{h->gcat1, 64, 32, h->cat1, 64, 32, 0, 1})));
    // ---- conv1 (x -> e1): W1, b1
    if ((rc = weight_grad(h, act(h->x0, N, H, W, 8, 0), umn::kConv3, 8, 1, act(h->gcat1, N, H, W, 64, 32), umn::kPix, 32,
                          H, W, G + L.w_off[0], 72, 32, [&] {
                              return gemm(h, Im2colMN{act(h->x0, N, H, W, 8, 0), 8, H, W, 1, 72, s.P},
                                          PixMN{act(h->gcat1, N, H, W, 64, 32), 32, s.P}, EpiDW{G + L.w_off[0], 32},
                                          72, 32, s.P, true);
                          })))
        return rc;
    if ((rc = bias_grad(h, h->gcat1, s.P, 64, 32, 32, 0))) return rc;
    return NEUROSIM_OK;
}

int check_shape(const neurosim_interp* h, int batch, int height, int width, Shape* s)
{
    if (batch < 1 || height < 4 || width < 4 || height % 4 || width % 4)
        return fail(NEUROSIM_E_INVALID, "batch >= 1 and height, width >= 4 and divisible by 4 required");
    const int64_t P = (int64_t)batch * height * width;
    if (P > h->Pmax) return fail(NEUROSIM_E_INVALID, "batch * height * width %lld exceeds the capacity %lld", (long long)P,
                                 (long long)h->Pmax);
    s->N = batch;
    s->H = height;
    s->W = width;
    s->P = (int)P;
    s->P2 = (int)(P / 4);
    s->P4 = (int)(P / 16);
    return NEUROSIM_OK;
}

int finish(neurosim_interp* h)
{
    unsigned int e = 0;
    ICUDA(cudaMemcpyAsync(&e, h->err, sizeof e, cudaMemcpyDeviceToHost, h->stream));
    ICUDA(cudaStreamSynchronize(h->stream));
    if (e) {
        cudaMemsetAsync(h->err, 0, sizeof(unsigned int), h->stream);
        return fail(NEUROSIM_E_TIMEOUT, "a bounded tensor-core wait timed out");
    }
    return NEUROSIM_OK;
}

int loss_and_backward(neurosim_interp* h, const Shape& s, const float* clips, float* loss_out)
{
    const int HW = s.H * s.W;
    int rc = forward(h, s, clips, clips + 4 * (int64_t)HW, 5ll * HW);
    if (rc) return rc;
    ICUDA(cudaMemsetAsync(h->loss, 0, sizeof(double), h->stream));
    loss_kernel<<<grid_for(s.P), 256, 0, h->stream>>>(h->out, clips, HW, s.P, 1.0f / (3.0f * (float)s.P), h->gr, h->loss);
    h->launches += 1;
    ICUDA(cudaGetLastError());
    rc = backward(h, s);
    if (rc) return rc;
    if (loss_out) {
        double l = 0.0;
        ICUDA(cudaMemcpyAsync(&l, h->loss, sizeof l, cudaMemcpyDeviceToHost, h->stream));
        rc = finish(h);
        if (rc) return rc;
        *loss_out = (float)(l / (3.0 * (double)s.P));
    }
    return NEUROSIM_OK;
}

struct IGuard {
    int prev = -1;
    bool ok = true;
    explicit IGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~IGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

int64_t neurosim_interp_param_count(void) { return ParamLayout().total; }

int neurosim_interp_create(int32_t max_batch, int32_t max_height, int32_t max_width, uint64_t seed, void* cuda_stream,
                           neurosim_interp** out)
{
    if (!out) return fail(NEUROSIM_E_INVALID, "out is NULL");
    *out = nullptr;
    if (max_batch < 1 || max_height < 4 || max_width < 4 || max_height % 4 || max_width % 4)
        return fail(NEUROSIM_E_INVALID, "max_batch >= 1 and max_height, max_width >= 4 and divisible by 4 required");
    const int64_t P = (int64_t)max_batch * max_height * max_width;
    if (P > (1ll << 30) / 64) return fail(NEUROSIM_E_INVALID, "max_batch * max_height * max_width too large");
    neurosim_interp* h = new (std::nothrow) neurosim_interp();
    if (!h) return fail(NEUROSIM_E_NOMEM, "host allocation failed");
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->Pmax = P;
    auto bail = [&](int code) {
        release(h);
        delete h;
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return bail(fail(NEUROSIM_E_CUDA, "no CUDA device"));
    const ParamLayout& L = h->lay;
    bool ok = dalloc(&h->params, L.total) == cudaSuccess && dalloc(&h->grads, L.total) == cudaSuccess &&
              dalloc(&h->m, L.total) == cudaSuccess && dalloc(&h->v, L.total) == cudaSuccess;
    for (int l = 0; l < kLayers && ok; ++l)
        ok = dalloc(&h->wf[l], weight_count(kDefs[l])) == cudaSuccess &&
             dalloc(&h->wb[l], weight_count(kDefs[l])) == cudaSuccess;
    const size_t p = (size_t)P, p2 = p / 4, p4 = p / 16;
    ok = ok && dalloc(&h->x0, p * 8) == cudaSuccess && dalloc(&h->cat1, p * 64) == cudaSuccess &&
         dalloc(&h->cat2, p2 * 128) == cudaSuccess && dalloc(&h->e3, p4 * 128) == cudaSuccess &&
         dalloc(&h->e4, p4 * 128) == cudaSuccess && dalloc(&h->d1, p2 * 64) == cudaSuccess &&
         dalloc(&h->d2, p * 32) == cudaSuccess && dalloc(&h->gcat1, p * 64) == cudaSuccess &&
         dalloc(&h->gcat2, p2 * 128) == cudaSuccess && dalloc(&h->ge3, p4 * 128) == cudaSuccess &&
         dalloc(&h->ge4, p4 * 128) == cudaSuccess && dalloc(&h->gd1, p2 * 64) == cudaSuccess &&
         dalloc(&h->gd2, p * 32) == cudaSuccess && dalloc(&h->gr, p * 16) == cudaSuccess &&
         dalloc(&h->l0, p) == cudaSuccess && dalloc(&h->l4, p) == cudaSuccess && dalloc(&h->out, 3 * p) == cudaSuccess &&
         dalloc(&h->loss, 1) == cudaSuccess && dalloc(&h->err, 1) == cudaSuccess;
    if (!ok) return bail(fail(NEUROSIM_E_NOMEM, "device allocation of the interpolator failed"));
    if (cudaMemsetAsync(h->params, 0, (size_t)L.total * 4, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->m, 0, (size_t)L.total * 4, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->v, 0, (size_t)L.total * 4, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->err, 0, 4, h->stream) != cudaSuccess)
        return bail(fail(NEUROSIM_E_CUDA, "cudaMemsetAsync failed"));
    for (int l = 0; l < kLayers - 1; ++l) {
        const LayerDef& d = kDefs[l];
        const int fan_in = d.kind == CONV ? 9 * d.cin : d.cin;
        init_weights_kernel<<<grid_for(weight_count(d)), 256, 0, h->stream>>>(
            h->params + L.w_off[l], weight_count(d), std::sqrt(2.0f / (float)fan_in), L.w_off[l], seed, d.kind, d.cin,
            d.cout, l == 0 ? 2 : d.cin);
    }
    if (cudaGetLastError() != cudaSuccess || pack_all(h) || cudaStreamSynchronize(h->stream) != cudaSuccess)
        return bail(fail(NEUROSIM_E_CUDA, "initialising the weights failed"));
    *out = h;
    return NEUROSIM_OK;
}

int neurosim_interp_forward(neurosim_interp* h, const float* L0_dev, const float* L4_dev, int32_t batch,
                            int32_t height, int32_t width, float* out_dev)
{
    if (!h || !L0_dev || !L4_dev || !out_dev) return fail(NEUROSIM_E_INVALID, "NULL argument");
    Shape s;
    int rc = check_shape(h, batch, height, width, &s);
    if (rc) return rc;
    IGuard g(h->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the device");
    rc = forward(h, s, L0_dev, L4_dev, (int64_t)height * width);
    if (rc) return rc;
    ICUDA(cudaMemcpyAsync(out_dev, h->out, (size_t)3 * s.P * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    return NEUROSIM_OK;
}

int neurosim_interp_gradients(neurosim_interp* h, const float* clips_dev, int32_t batch, int32_t height, int32_t width,
                              float* grads_host, float* loss_out)
{
    if (!h || !clips_dev) return fail(NEUROSIM_E_INVALID, "NULL argument");
    Shape s;
    int rc = check_shape(h, batch, height, width, &s);
    if (rc) return rc;
    IGuard g(h->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the device");
    float l = 0.0f;
    rc = loss_and_backward(h, s, clips_dev, &l);
    if (rc) return rc;
    if (loss_out) *loss_out = l;
    if (grads_host) {
        ICUDA(cudaMemcpyAsync(grads_host, h->grads, (size_t)h->lay.total * 4, cudaMemcpyDeviceToHost, h->stream));
        ICUDA(cudaStreamSynchronize(h->stream));
    }
    return NEUROSIM_OK;
}

int neurosim_interp_train_step(neurosim_interp* h, const float* clips_dev, int32_t batch, int32_t height,
                               int32_t width, float lr, float weight_decay, float* loss_out)
{
    if (!h || !clips_dev) return fail(NEUROSIM_E_INVALID, "NULL argument");
    if (!(lr >= 0.0f && lr < 1.0f) || !(weight_decay >= 0.0f && weight_decay < 1.0f))
        return fail(NEUROSIM_E_INVALID, "lr and weight_decay must be in [0, 1)");
    Shape s;
    int rc = check_shape(h, batch, height, width, &s);
    if (rc) return rc;
    IGuard g(h->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the device");
    rc = loss_and_backward(h, s, clips_dev, loss_out);
    if (rc) return rc;
    h->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float bc1 = (float)(1.0 - std::pow(b1, (double)h->step)), bc2 = (float)(1.0 - std::pow(b2, (double)h->step));
    adamw_kernel<<<grid_for(h->lay.total), 256, 0, h->stream>>>(h->params, h->grads, h->m, h->v, h->lay.total,
                                                                h->lay.n_weights, lr, weight_decay, (float)b1,
                                                                (float)b2, 1e-8f, bc1, bc2);
    h->launches += 1;
    ICUDA(cudaGetLastError());
    rc = pack_all(h);
    if (rc) return rc;
    if (loss_out) return finish(h);
    return NEUROSIM_OK;
}

int neurosim_interp_get_params(neurosim_interp* h, float* host, int64_t n)
{
    if (!h || !host) return fail(NEUROSIM_E_INVALID, "NULL argument");
    if (n != h->lay.total) return fail(NEUROSIM_E_INVALID, "n must be %lld", (long long)h->lay.total);
    IGuard g(h->device);
    ICUDA(cudaMemcpyAsync(host, h->params, (size_t)n * 4, cudaMemcpyDeviceToHost, h->stream));
    ICUDA(cudaStreamSynchronize(h->stream));
    return NEUROSIM_OK;
}

int neurosim_interp_set_params(neurosim_interp* h, const float* host, int64_t n)
{
    if (!h || !host) return fail(NEUROSIM_E_INVALID, "NULL argument");
    if (n != h->lay.total) return fail(NEUROSIM_E_INVALID, "n must be %lld", (long long)h->lay.total);
    IGuard g(h->device);
    ICUDA(cudaMemcpyAsync(h->params, host, (size_t)n * 4, cudaMemcpyHostToDevice, h->stream));
    ICUDA(cudaMemsetAsync(h->m, 0, (size_t)n * 4, h->stream));
    ICUDA(cudaMemsetAsync(h->v, 0, (size_t)n * 4, h->stream));
    h->step = 0;
    int rc = pack_all(h);
    if (rc) return rc;
    ICUDA(cudaStreamSynchronize(h->stream));
    return NEUROSIM_OK;
}

// ---- checkpoints -------------------------------------------------------------------------
// File layout (little-endian, as written by the host):
//   0  char[8]  "NSIMUNT1"
//   8  uint32   format version (1)
//  12  uint32   flags: bit 0 = the AdamW moments follow the parameters
//  16  int64    n = parameter count
//  24  int64    optimiser step count
//  32  float[n] parameters, then float[n] first and float[n] second moments if flagged
//  end uint64   FNV-1a 64-bit hash of every byte before it
namespace {

constexpr char kCkptMagic[8] = {'N', 'S', 'I', 'M', 'U', 'N', 'T', '1'};
constexpr uint32_t kCkptVersion = 1;
constexpr size_t kCkptHeader = 32;

uint64_t fnv1a(const unsigned char* p, size_t n)
{
    uint64_t x = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) {
        x ^= p[i];
        x *= 0x100000001b3ull;
    }
    return x;
}

bool host_little_endian()
{
    const uint32_t one = 1u;
    unsigned char b;
    memcpy(&b, &one, 1);
    return b == 1;
}

}  // namespace

int neurosim_interp_save(neurosim_interp* h, const char* path, int32_t with_optimizer)
{
    if (!h || !path) return fail(NEUROSIM_E_INVALID, "NULL argument");
    if (!host_little_endian()) return fail(NEUROSIM_E_INVALID, "checkpoints are little-endian only");
    const int64_t n = h->lay.total;
    const int arrays = with_optimizer ? 3 : 1;
    const size_t body = (size_t)arrays * (size_t)n * 4;
    std::vector<unsigned char> buf;
    try {
        buf.resize(kCkptHeader + body + 8);
    } catch (...) {
        return fail(NEUROSIM_E_NOMEM, "no host memory for a %zu-byte checkpoint", buf.size());
    }
    unsigned char* b = buf.data();
    const uint32_t flags = with_optimizer ? 1u : 0u;
    const int64_t step = h->step;
    memcpy(b, kCkptMagic, 8);
    memcpy(b + 8, &kCkptVersion, 4);
    memcpy(b + 12, &flags, 4);
    memcpy(b + 16, &n, 8);
    memcpy(b + 24, &step, 8);
    {
        IGuard g(h->device);
        float* src[3] = {h->params, h->m, h->v};
        for (int a = 0; a < arrays; ++a)
            ICUDA(cudaMemcpyAsync(b + kCkptHeader + (size_t)a * n * 4, src[a], (size_t)n * 4, cudaMemcpyDeviceToHost,
                                  h->stream));
        ICUDA(cudaStreamSynchronize(h->stream));
    }
    const uint64_t hash = fnv1a(b, kCkptHeader + body);
    memcpy(b + kCkptHeader + body, &hash, 8);
    // write beside the target, then rename: a reader never sees half a file
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(NEUROSIM_E_IO, "cannot open %s for writing", tmp.c_str());
    const size_t put = fwrite(b, 1, buf.size(), f);
    const int closed = fclose(f);
    if (put != buf.size() || closed != 0) {
        remove(tmp.c_str());
        return fail(NEUROSIM_E_IO, "short write to %s", tmp.c_str());
    }
    if (rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return fail(NEUROSIM_E_IO, "cannot rename %s to %s", tmp.c_str(), path);
    }
    return NEUROSIM_OK;
}

int neurosim_interp_load(neurosim_interp* h, const char* path)
{
    if (!h || !path) return fail(NEUROSIM_E_INVALID, "NULL argument");
    if (!host_little_endian()) return fail(NEUROSIM_E_INVALID, "checkpoints are little-endian only");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(NEUROSIM_E_IO, "cannot open %s", path);
    std::vector<unsigned char> buf;
    unsigned char chunk[1 << 16];
    size_t got = 0;
    bool too_big = false;
    const int64_t n = h->lay.total;
    const size_t max_size = kCkptHeader + 3 * (size_t)n * 4 + 8;
    while ((got = fread(chunk, 1, sizeof chunk, f)) > 0) {
        if (buf.size() + got > max_size) {
            too_big = true;
            break;
        }
        buf.insert(buf.end(), chunk, chunk + got);
    }
    const bool read_error = ferror(f) != 0;
    fclose(f);
    if (read_error) return fail(NEUROSIM_E_IO, "read error on %s", path);
    if (too_big) return fail(NEUROSIM_E_INVALID, "%s: larger than any checkpoint of this network", path);
    if (buf.size() < kCkptHeader + 8 || memcmp(buf.data(), kCkptMagic, 8) != 0)
        return fail(NEUROSIM_E_INVALID, "%s: not an interpolator checkpoint", path);
    const unsigned char* b = buf.data();
    uint32_t version = 0, flags = 0;
    int64_t fn = 0, step = 0;
    memcpy(&version, b + 8, 4);
    memcpy(&flags, b + 12, 4);
    memcpy(&fn, b + 16, 8);
    memcpy(&step, b + 24, 8);
    if (version != kCkptVersion) return fail(NEUROSIM_E_INVALID, "%s: format version %u, expected %u", path, version,
                                             kCkptVersion);
    if (fn != n) return fail(NEUROSIM_E_INVALID, "%s: %lld parameters, the network has %lld", path, (long long)fn,
                             (long long)n);
    if ((flags & ~1u) != 0u || step < 0) return fail(NEUROSIM_E_INVALID, "%s: bad header", path);
    const int arrays = (flags & 1u) ? 3 : 1;
    const size_t body = (size_t)arrays * (size_t)n * 4;
    if (buf.size() != kCkptHeader + body + 8)
        return fail(NEUROSIM_E_INVALID, "%s: %zu bytes, expected %zu (truncated?)", path, buf.size(),
                    kCkptHeader + body + 8);
    uint64_t hash = 0;
    memcpy(&hash, b + kCkptHeader + body, 8);
    if (hash != fnv1a(b, kCkptHeader + body)) return fail(NEUROSIM_E_INVALID, "%s: checksum mismatch", path);
    IGuard g(h->device);
    float* dst[3] = {h->params, h->m, h->v};
    for (int a = 0; a < 3; ++a) {
        if (a < arrays)
            ICUDA(cudaMemcpyAsync(dst[a], b + kCkptHeader + (size_t)a * n * 4, (size_t)n * 4, cudaMemcpyHostToDevice,
                                  h->stream));
        else
            ICUDA(cudaMemsetAsync(dst[a], 0, (size_t)n * 4, h->stream));
    }
    h->step = arrays == 3 ? step : 0;
    int rc = pack_all(h);
    if (rc) return rc;
    ICUDA(cudaStreamSynchronize(h->stream));
    return NEUROSIM_OK;
}

int neurosim_interp_launches(neurosim_interp* h, uint64_t* launches)
{
    if (!h || !launches) return fail(NEUROSIM_E_INVALID, "NULL argument");
    *launches = h->launches;
    return NEUROSIM_OK;
}

void neurosim_interp_destroy(neurosim_interp* h)
{
    if (!h) return;
    {
        IGuard g(h->device);
        cudaStreamSynchronize(h->stream);
        release(h);
    }
    delete h;
}

}  // extern "C"
