// Operand gathers and epilogues that turn the U-Net layers of the learned
// interpolator into tensor-core GEMMs (umma_gemm.cuh).  Activations are BF16
// NHWC; a view selects `C` channels at offset `off` of rows of `stride`
// channels, so that a concatenation is one buffer written by two layers.
// Every gather moves 16-byte chunks of 8 channels (channel counts, offsets
// and strides are multiples of 8).
//
//   forward   conv 3x3 (stride 1 or 2):  D[pixel][cout] = im2col(x) * W
//             convT 2x2 stride 2:        D[in pixel][(a, b, cout)] = x * W
//   backward  data of the final 1x1 layer: D[pixel][cin] = dy * W^T
//             weights:       D[(tap, cin)][cout] = sum over pixels (split over
//                            the grid's y dimension, FP32 atomics), where the
//                            pixel runs are too short for the TMA form
// (the other data gradients run on TMA-fed kernels: umma_tma.cuh)
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "umma_gemm.cuh"

namespace interp {

using bf16 = __nv_bfloat16;
using ugemm::BK;
using ugemm::kmajor_chunk;
using ugemm::mnmajor_chunk;
using ugemm::st_chunk;

struct Act {            // BF16 NHWC view
    const bf16* p;
    int N, H, W;        // image size of the view
    int stride, off;    // channels per pixel row, first channel of the view
    __device__ __forceinline__ const bf16* at(int n, int y, int x, int c) const
    {
        return p + ((size_t)((size_t)n * H + y) * W + x) * stride + off + c;
    }
};

__device__ __forceinline__ uint4 ld16(const bf16* p) { return *reinterpret_cast<const uint4*>(p); }

// ---- K-major A gathers (rows = output pixels of the GEMM) ---------------------------
// Thread t always fills chunk column kc = t % 8 of rows t / 8 + 16 j: its
// rows' pixel coordinates are decoded once per tile (prep) and each K tile
// only adds the tap offset.  Channel counts are powers of two (cshift).
__host__ __device__ constexpr int kRowsPerThread(int R) { return R / 16; }

// conv 3x3, zero padding 1, stride s: row (n, yo, xo), k = tap * C + c reads
// x(n, s yo + dy - 1, s xo + dx - 1, c).
struct Conv3K {
    static constexpr bool MN = false;
    Act x;
    int C, Ho, Wo, s, M;
    int cshift;
    template <int R>
    struct Rows {
        int nH[kRowsPerThread(R)];     // n * H of the input, or -1 for rows past M
        int ys[kRowsPerThread(R)];     // s yo - 1
        int xs[kRowsPerThread(R)];     // s xo - 1
    };
    template <int R>
    __device__ __forceinline__ void prep(Rows<R>& rw, int r0, int tid) const
    {
        const int hw = Ho * Wo;
#pragma unroll
        for (int j = 0; j < kRowsPerThread(R); ++j) {
            const int m = r0 + (tid >> 3) + 16 * j;
            if (m < M) {
                const int n = m / hw, rem = m - n * hw, yo = rem / Wo, xo = rem - yo * Wo;
                rw.nH[j] = n * x.H;
                rw.ys[j] = yo * s - 1;
                rw.xs[j] = xo * s - 1;
            } else {
                rw.nH[j] = -1;
                rw.ys[j] = rw.xs[j] = 0;
            }
        }
    }
    template <int R>
    __device__ __forceinline__ void gather(unsigned char* tile, const Rows<R>& rw, int, int k0, int kn, int tid) const
    {
        const int kc = tid & 7, k = k0 + kc * 8;
        const int tap = k >> cshift, c = k & (C - 1);
        const int dy = tap / 3, dx = tap - 3 * dy;
        const bool kok = kc * 8 < kn;
#pragma unroll
        for (int j = 0; j < kRowsPerThread(R); ++j) {
            const int r = (tid >> 3) + 16 * j;
            const int yi = rw.ys[j] + dy, xi = rw.xs[j] + dx;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (kok && rw.nH[j] >= 0 && (unsigned)yi < (unsigned)x.H && (unsigned)xi < (unsigned)x.W)
                v = ld16(x.p + ((size_t)(rw.nH[j] + yi) * x.W + xi) * x.stride + x.off + c);
            st_chunk(tile, kmajor_chunk(r, kc * 8), v);
        }
    }
};

// 1x1: row = pixel, k = channel.
struct PixK {
    static constexpr bool MN = false;
    Act x;
    int M;
    UGEMM_NO_ROWS
    template <int R>
    __device__ __forceinline__ void gather(unsigned char* tile, const Rows<R>&, int r0, int k0, int kn, int tid) const
    {
        const int kc = tid & 7;
        const bool kok = kc * 8 < kn;
#pragma unroll
        for (int j = 0; j < kRowsPerThread(R); ++j) {
            const int r = (tid >> 3) + 16 * j, m = r0 + r;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (kok && m < M) v = ld16(x.p + (size_t)m * x.stride + x.off + k0 + kc * 8);
            st_chunk(tile, kmajor_chunk(r, kc * 8), v);
        }
    }
};

// ---- MN-major gathers (weight gradients: K = pixels) -------------------------------
// rows (tap, c) of a conv 3x3 stride s at output pixel p: x(n, s yo + dy - 1, s xo + dx - 1, c).
struct Im2colMN {
    static constexpr bool MN = true;
    UGEMM_NO_ROWS
    Act x;
    int C, Ho, Wo, s, rows, P;
    template <int R>
    __device__ __forceinline__ void gather(unsigned char* tile, const Rows<R>&, int r0, int k0, int kn, int tid) const
    {
        for (int i = tid; i < (R / 8) * BK; i += 128) {
            const int k = i / (R / 8), rc = i % (R / 8);
            const int row = r0 + rc * 8, p = k0 + k;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (row < rows && k < kn && p < P) {
                const int hw = Ho * Wo;
                const int n = p / hw, rem = p - n * hw, yo = rem / Wo, xo = rem - (rem / Wo) * Wo;
                const int tap = row / C, c = row - tap * C;
                const int yi = yo * s + tap / 3 - 1, xi = xo * s + tap % 3 - 1;
                if ((unsigned)yi < (unsigned)x.H && (unsigned)xi < (unsigned)x.W) v = ld16(x.at(n, yi, xi, c));
            }
            st_chunk(tile, mnmajor_chunk<R>(rc * 8, k), v);
        }
    }
};

// rows = channels at pixel p.
struct PixMN {
    static constexpr bool MN = true;
    UGEMM_NO_ROWS
    Act x;
    int rows, P;
    template <int R>
    __device__ __forceinline__ void gather(unsigned char* tile, const Rows<R>&, int r0, int k0, int kn, int tid) const
    {
        for (int i = tid; i < (R / 8) * BK; i += 128) {
            const int k = i / (R / 8), rc = i % (R / 8);
            const int row = r0 + rc * 8, p = k0 + k;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (row < rows && k < kn && p < P) v = ld16(x.p + (size_t)p * x.stride + x.off + row);
            st_chunk(tile, mnmajor_chunk<R>(rc * 8, k), v);
        }
    }
};

// rows (2a + b, c) at low-size pixel p: g(n, 2y + a, 2x + b, c).
struct S2DMN {
    static constexpr bool MN = true;
    UGEMM_NO_ROWS
    Act g;
    int C, Hl, Wl, rows, P;
    template <int R>
    __device__ __forceinline__ void gather(unsigned char* tile, const Rows<R>&, int r0, int k0, int kn, int tid) const
    {
        for (int i = tid; i < (R / 8) * BK; i += 128) {
            const int k = i / (R / 8), rc = i % (R / 8);
            const int row = r0 + rc * 8, p = k0 + k;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (row < rows && k < kn && p < P) {
                const int hw = Hl * Wl;
                const int n = p / hw, rem = p - n * hw, y = rem / Wl, xx = rem - (rem / Wl) * Wl;
                const int ab = row / C, c = row - ab * C;
                v = ld16(g.at(n, 2 * y + (ab >> 1), 2 * xx + (ab & 1), c));
            }
            st_chunk(tile, mnmajor_chunk<R>(rc * 8, k), v);
        }
    }
};

// ---- epilogues --------------------------------------------------------------------
__device__ __forceinline__ uint4 pack8(const float (&v)[8])
{
    uint4 o;
    __nv_bfloat162 h;
    h = __floats2bfloat162_rn(v[0], v[1]);
    o.x = *reinterpret_cast<uint32_t*>(&h);
    h = __floats2bfloat162_rn(v[2], v[3]);
    o.y = *reinterpret_cast<uint32_t*>(&h);
    h = __floats2bfloat162_rn(v[4], v[5]);
    o.z = *reinterpret_cast<uint32_t*>(&h);
    h = __floats2bfloat162_rn(v[6], v[7]);
    o.w = *reinterpret_cast<uint32_t*>(&h);
    return o;
}

__device__ __forceinline__ void unpack8(uint4 u, float (&v)[8])
{
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[i]);
        const float2 f = __bfloat1622float2(h);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

// out[row][off + col] = bf16(relu?(acc + bias[col]))
struct EpiAct {
    bf16* out;
    int stride, off;
    const float* bias;
    int relu;
    static constexpr bool kStaged = true;
    __device__ __forceinline__ bf16* row_ptr(int row) const { return out + (size_t)row * stride + off; }
    // staged drain: destination of columns c0 .. c0 + 31 of row = base_ptr(row) + col_offset(c0)
    __device__ __forceinline__ bf16* base_ptr(int row) const { return row_ptr(row); }
    __device__ __forceinline__ size_t col_offset(int c0) const { return (size_t)c0; }
    // columns c0 .. c0 + 31 of one pixel as four 16-byte chunks
    __device__ __forceinline__ void pack32(int c0, const float (&v)[32], uint4 (&o)[4]) const
    {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float t[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float s = v[8 * q + i] + bias[c0 + 8 * q + i];
                t[i] = relu ? fmaxf(s, 0.0f) : s;
            }
            o[q] = pack8(t);
        }
    }
    __device__ __forceinline__ void store(int row, int c0, const float (&v)[8], int) const
    {
        float o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float t = v[i] + bias[c0 + i];
            o[i] = relu ? fmaxf(t, 0.0f) : t;
        }
        *reinterpret_cast<uint4*>(out + (size_t)row * stride + off + c0) = pack8(o);
    }
};

// convT 2x2 stride 2: column (2a + b) * Cout + o of input pixel (n, y, x)
// goes to output pixel (n, 2y + a, 2x + b), channel off + o.
struct EpiConvT {
    bf16* out;
    int stride, off;
    const float* bias;
    int Cout, Hl, Wl;
    // staged drain (Cout a multiple of 32): the 32 columns c0 .. c0 + 31 of a
    // low-resolution pixel are 64 contiguous bytes of one output pixel, so the
    // warp writes whole sectors instead of 16-byte pieces 256 bytes apart
    static constexpr bool kStaged = true;
    __device__ __forceinline__ bf16* base_ptr(int row) const
    {
        const int hw = Hl * Wl;
        const int n = row / hw, rem = row - n * hw, y = rem / Wl, x = rem - (rem / Wl) * Wl;
        return out + (((size_t)n * 2 * Hl + 2 * y) * (2 * Wl) + 2 * x) * stride + off;
    }
    __device__ __forceinline__ size_t col_offset(int c0) const
    {
        const int ab = c0 / Cout, o = c0 - ab * Cout;
        return ((size_t)(ab >> 1) * (2 * Wl) + (ab & 1)) * stride + o;
    }
    __device__ __forceinline__ void pack32(int c0, const float (&v)[32], uint4 (&o)[4]) const
    {
        const int oc = c0 % Cout;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float t[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) t[i] = v[8 * q + i] + bias[oc + 8 * q + i];
            o[q] = pack8(t);
        }
    }
    __device__ __forceinline__ void store(int row, int c0, const float (&v)[8], int) const
    {
        const int hw = Hl * Wl;
        const int n = row / hw, rem = row - n * hw, y = rem / Wl, x = rem - (rem / Wl) * Wl;
        const int ab = c0 / Cout, o = c0 - ab * Cout;
        const size_t pix = ((size_t)n * 2 * Hl + 2 * y + (ab >> 1)) * (2 * Wl) + 2 * x + (ab & 1);
        float t[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = v[i] + bias[o + i];
        *reinterpret_cast<uint4*>(out + pix * stride + off + o) = pack8(t);
    }
};

// Gradient of a layer input: out[row][off + col] = bf16((acc ? out : 0) + v *
// mask), mask = act[row][aoff + col] > 0 for col >= mask_from (ReLU inputs),
// else 1 (linear inputs).
struct EpiGrad {
    bf16* out;
    int stride, off;
    const bf16* act;
    int astride, aoff, mask_from, accumulate;
    __device__ __forceinline__ void store(int row, int c0, const float (&v)[8], int) const
    {
        bf16* dst = out + (size_t)row * stride + off + c0;
        float o[8], a[8], old[8];
        unpack8(ld16(act + (size_t)row * astride + aoff + c0), a);
        if (accumulate) unpack8(ld16(dst), old);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float m = (c0 + i < mask_from || a[i] > 0.0f) ? 1.0f : 0.0f;
            o[i] = v[i] * m + (accumulate ? old[i] : 0.0f);
        }
        *reinterpret_cast<uint4*>(dst) = pack8(o);
    }
};

// Final 1x1 layer: L_j = L0 + (j / 4)(L4 - L0) + r_{j - 1} + b, j = 1..3 (FP32).
struct EpiOut {
    float* out;            // [3][P]
    const float* L0;
    const float* L4;
    const float* bias;
    int P;
    __device__ __forceinline__ void store(int row, int c0, const float (&v)[8], int) const
    {
        if (c0 != 0) return;
        const float a = L0[row], d = L4[row] - a;
#pragma unroll
        for (int j = 0; j < 3; ++j) out[(size_t)j * P + row] = a + 0.25f * (float)(j + 1) * d + (v[j] + bias[j]);
    }
};

// Weight gradient: dw[row][col] += acc (FP32 atomics over the K splits).
struct EpiDW {
    float* dw;
    int ld;
    __device__ __forceinline__ void store(int row, int c0, const float (&v)[8], int) const
    {
        float* d = dw + (size_t)row * ld + c0;
#pragma unroll
        for (int i = 0; i < 8; ++i) atomicAdd(d + i, v[i]);
    }
};

}  // namespace interp
