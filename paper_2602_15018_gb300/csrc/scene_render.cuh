// Procedural texture scene rendered on the device: the frame source of the
// render-fused event step and of the stand-alone renderer (render_fused.cu).
//
// The paper renders its scenes with a graphics engine and argues that event
// data should be produced on the fly, without storing the rendered images
// (Sec. 1); its scenes are not available here, so the library renders a
// seeded procedural scene with the same role: 4-octave value noise under a
// smooth affine camera path, with moving occluding rectangles drawn
// last-on-top (the scene of the benchmark's HD workload).  Rendering inside
// the emission kernel removes the frame read, 4 bytes per pixel-frame.
//
// Both users call the same device function texture_pixel, whose every
// floating-point operation is an explicitly rounded intrinsic: the fused step
// sees bit for bit the intensities the stand-alone renderer writes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"

namespace nsim {

constexpr int kMaxRects = NEUROSIM_MAX_RECTS;

// Per-frame camera and occluder placement, computed on the device in double
// from the scene and the frame time, stored in FP32 (one table row per frame).
struct SceneFrame {
    float A, B, Cx;        // texture x = A x + B y + Cx (pixel x, y)
    float D, E, Cy;        // texture y = D x + E y + Cy
    float pad[2];
    float4 rect[kMaxRects];   // centre x, centre y, half width, half height
    float rval[kMaxRects];    // intensity inside the rectangle
};

// 32-bit integer hash of a lattice point (multiply-xorshift mixing), as a
// value in [0, 1).
__device__ __forceinline__ float lattice_value(int32_t ix, int32_t iy, uint32_t salt)
{
    uint32_t h = ((uint32_t)ix * 0x8DA6B343u) ^ ((uint32_t)iy * 0xD8163841u) ^ salt;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return __fmul_rn(__uint2float_rn(h), 2.3283064365386963e-10f);   // 2^-32
}

// Value noise of the texture at (x, y): octaves of smoothstep-interpolated
// lattice values, each octave at half the period and `gain` times the
// amplitude of the one before, mapped to [lo, lo + span].
__device__ __forceinline__ float texture_noise(const SceneConst& sc, const SceneFrame& fr, float x, float y)
{
    const float wx = __fmaf_rn(fr.A, x, __fmaf_rn(fr.B, y, fr.Cx));
    const float wy = __fmaf_rn(fr.D, x, __fmaf_rn(fr.E, y, fr.Cy));
    float acc = 0.0f, norm = 0.0f, amp = 1.0f, inv = sc.inv_period;
    uint32_t salt = sc.salt;
    for (int o = 0; o < sc.octaves; ++o) {
        salt += 0x9E3779B9u;
        const float u = __fmul_rn(wx, inv), v = __fmul_rn(wy, inv);
        const float iu = floorf(u), iv = floorf(v);
        const float fu = __fsub_rn(u, iu), fv = __fsub_rn(v, iv);
        const float su = __fmul_rn(__fmul_rn(fu, fu), __fmaf_rn(-2.0f, fu, 3.0f));
        const float sv = __fmul_rn(__fmul_rn(fv, fv), __fmaf_rn(-2.0f, fv, 3.0f));
        const int32_t i0 = (int32_t)iu, j0 = (int32_t)iv;
        const float h00 = lattice_value(i0, j0, salt);
        const float h10 = lattice_value(i0 + 1, j0, salt);
        const float h01 = lattice_value(i0, j0 + 1, salt);
        const float h11 = lattice_value(i0 + 1, j0 + 1, salt);
        const float top = __fmaf_rn(__fsub_rn(h10, h00), su, h00);
        const float bot = __fmaf_rn(__fsub_rn(h11, h01), su, h01);
        acc = __fmaf_rn(amp, __fmaf_rn(__fsub_rn(bot, top), sv, top), acc);
        norm = __fadd_rn(norm, amp);
        amp = __fmul_rn(amp, sc.gain);
        inv = __fmul_rn(inv, 2.0f);
    }
    return __fmaf_rn(sc.span, __fdiv_rn(acc, norm), sc.lo);
}

// texture_noise of four pixels at once: the same operations for each pixel
// in the same order (so the same bits), the octave loop outside, so that the
// four pixels' independent hash and interpolation chains interleave.
__device__ __forceinline__ void texture_noise4(const SceneConst& sc, const SceneFrame& fr, const float (&x)[4],
                                               const float (&y)[4], float (&out)[4])
{
    float wx[4], wy[4], acc[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        wx[m] = __fmaf_rn(fr.A, x[m], __fmaf_rn(fr.B, y[m], fr.Cx));
        wy[m] = __fmaf_rn(fr.D, x[m], __fmaf_rn(fr.E, y[m], fr.Cy));
        acc[m] = 0.0f;
    }
    float norm = 0.0f, amp = 1.0f, inv = sc.inv_period;
    uint32_t salt = sc.salt;
    for (int o = 0; o < sc.octaves; ++o) {
        salt += 0x9E3779B9u;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float u = __fmul_rn(wx[m], inv), v = __fmul_rn(wy[m], inv);
            const float iu = floorf(u), iv = floorf(v);
            const float fu = __fsub_rn(u, iu), fv = __fsub_rn(v, iv);
            const float su = __fmul_rn(__fmul_rn(fu, fu), __fmaf_rn(-2.0f, fu, 3.0f));
            const float sv = __fmul_rn(__fmul_rn(fv, fv), __fmaf_rn(-2.0f, fv, 3.0f));
            const int32_t i0 = (int32_t)iu, j0 = (int32_t)iv;
            const float h00 = lattice_value(i0, j0, salt);
            const float h10 = lattice_value(i0 + 1, j0, salt);
            const float h01 = lattice_value(i0, j0 + 1, salt);
            const float h11 = lattice_value(i0 + 1, j0 + 1, salt);
            const float top = __fmaf_rn(__fsub_rn(h10, h00), su, h00);
            const float bot = __fmaf_rn(__fsub_rn(h11, h01), su, h01);
            acc[m] = __fmaf_rn(amp, __fmaf_rn(__fsub_rn(bot, top), sv, top), acc[m]);
        }
        norm = __fadd_rn(norm, amp);
        amp = __fmul_rn(amp, sc.gain);
        inv = __fmul_rn(inv, 2.0f);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) out[m] = __fmaf_rn(sc.span, __fdiv_rn(acc[m], norm), sc.lo);
}

// Whether rectangle r = (centre x, centre y, half width, half height) covers
// pixel (x, y).
__device__ __forceinline__ bool rect_covers(float4 r, float x, float y)
{
    return fabsf(__fsub_rn(x, r.x)) < r.z && fabsf(__fsub_rn(y, r.y)) < r.w;
}

// Intensity of pixel (x, y): the noise, overdrawn by every rectangle that
// covers the pixel, in rectangle order (the last one is on top).
__device__ __forceinline__ float texture_pixel(const SceneConst& sc, const SceneFrame& fr, float x, float y)
{
    float v = texture_noise(sc, fr, x, y);
    for (int k = 0; k < sc.n_rects; ++k)
        if (rect_covers(fr.rect[k], x, y)) v = fr.rval[k];
    return v;
}

}  // namespace nsim
