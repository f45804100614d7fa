// Sensor bandwidth limit (declared in include/neurosim_evsim.h as
// neurosim_lowpass_log).  Sec. 2 of the paper lists bandwidth limitations
// among the sensor non-idealities Neurosim simulates (and lets the user turn
// off) without giving a model.  This library's reading: a first-order
// low-pass filter on each pixel's log intensity, one update per frame,
//   s_k = s_{k-1} + alpha (L_k - s_{k-1}),   alpha = 1 - exp(-2 pi f_c dt),
// evaluated in FP32 as d = L - s (rounded), s = fma(alpha, d, s) (one
// rounding), so that the CPU oracle reaches the same bits.  The filtered log
// frames feed the unchanged event emission with input_is_log = 1.
//
// Memory-bound: 4 B read and 4 B written per pixel-frame.  One thread owns
// four adjacent pixels (128-bit loads and stores) for all frames of the call
// and keeps their filter state in registers; loads of the next frames do not
// depend on the recurrence, so four frames are loaded before they are used.
// out may equal L (in place): every element is read by the thread that
// writes it, before it writes it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"

namespace {

__device__ __forceinline__ float lp_update(float s, float L, float alpha)
{
    return __fmaf_rn(alpha, __fsub_rn(L, s), s);
}

// n4 groups of 4 pixels; frames [T][n_pix] with n_pix = 4 n4.
__global__ void lowpass4_kernel(const float4* L, float4* out, int T, int64_t n4,
                                float alpha, float4* state, int init)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    float4 s = init ? L[i] : state[i];
    int f = 0;
    for (; f + 4 <= T; f += 4) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldcs(L + (int64_t)(f + u) * n4 + i);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            s.x = lp_update(s.x, v[u].x, alpha);
            s.y = lp_update(s.y, v[u].y, alpha);
            s.z = lp_update(s.z, v[u].z, alpha);
            s.w = lp_update(s.w, v[u].w, alpha);
            __stcs(out + (int64_t)(f + u) * n4 + i, s);
        }
    }
    for (; f < T; ++f) {
        const float4 v = __ldcs(L + (int64_t)f * n4 + i);
        s.x = lp_update(s.x, v.x, alpha);
        s.y = lp_update(s.y, v.y, alpha);
        s.z = lp_update(s.z, v.z, alpha);
        s.w = lp_update(s.w, v.w, alpha);
        __stcs(out + (int64_t)f * n4 + i, s);
    }
    state[i] = s;
}

__global__ void lowpass1_kernel(const float* L, float* out, int T, int64_t n, float alpha,
                                float* state, int init)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = init ? L[i] : state[i];
    for (int f = 0; f < T; ++f) {
        s = lp_update(s, L[(int64_t)f * n + i], alpha);
        out[(int64_t)f * n + i] = s;
    }
    state[i] = s;
}

// Sensor leak: the log input rises by C+_u * r * (t - origin), FP32 as
// fl(L + fl(fl(C+_u * r_us) * (float)(t - origin))) with r_us = (float)(r 1e-6).
// One thread per pixel for all frames (4 B read + 4 B written per pixel-frame).
__global__ void leak_kernel(const float* L, float* out, int T, int64_t n, int64_t t0, int dt, int64_t origin,
                            float rate_us, const float* cpos, float cpos_u)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float k = __fmul_rn(cpos ? cpos[i] : cpos_u, rate_us);
    for (int f = 0; f < T; ++f) {
        const float s = __ll2float_rn(t0 + (int64_t)f * dt - origin);
        out[(int64_t)f * n + i] = __fadd_rn(L[(int64_t)f * n + i], __fmul_rn(k, s));
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// Gain of the filter for a cutoff: a first-order low-pass with cutoff f_c has
// the time constant 1 / (2 pi f_c); sampled every dt it keeps exp(-2 pi f_c dt)
// of its old level per frame, so alpha = 1 - exp(-2 pi f_c dt), evaluated on
// the host in double and rounded once to FP32.
extern "C" int neurosim_lowpass_alpha(double cutoff_hz, int32_t dt_us, float* alpha_out)
{
    if (!alpha_out) return nsim::report_error(NEUROSIM_E_INVALID, "alpha_out is NULL");
    if (!(cutoff_hz > 0.0) || !std::isfinite(cutoff_hz))
        return nsim::report_error(NEUROSIM_E_INVALID, "cutoff_hz must be positive and finite");
    if (dt_us < 1) return nsim::report_error(NEUROSIM_E_INVALID, "dt_us must be >= 1");
    const double omega_dt = 2.0 * 3.14159265358979323846 * cutoff_hz * ((double)dt_us * 1e-6);
    const float a = (float)(1.0 - std::exp(-omega_dt));
    if (!(a > 0.0f)) return nsim::report_error(NEUROSIM_E_INVALID, "cutoff_hz * dt too small: the gain rounds to 0");
    *alpha_out = a;
    return NEUROSIM_OK;
}

extern "C" int neurosim_lowpass_log(const float* L_dev, float* out_dev, int32_t n_frames, int64_t n_pix, float alpha,
                                    float* state_dev, int32_t init, void* cuda_stream)
{
    if (n_frames < 0 || n_pix < 0) return nsim::report_error(NEUROSIM_E_INVALID, "n_frames and n_pix must be >= 0");
    if (!(alpha > 0.0f && alpha <= 1.0f)) return nsim::report_error(NEUROSIM_E_INVALID, "alpha must be in (0, 1]");
    if (n_pix == 0 || (n_frames == 0 && !init)) return NEUROSIM_OK;
    if (!state_dev || (n_frames > 0 && (!L_dev || !out_dev)))
        return nsim::report_error(NEUROSIM_E_INVALID, "NULL buffer");
    if (init && n_frames == 0) return nsim::report_error(NEUROSIM_E_INVALID, "init needs at least one frame");
    if (L_dev != out_dev && (const void*)L_dev < (const void*)(out_dev + (size_t)n_frames * n_pix) &&
        (const void*)out_dev < (const void*)(L_dev + (size_t)n_frames * n_pix))
        return nsim::report_error(NEUROSIM_E_INVALID, "L_dev and out_dev overlap without being equal");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    constexpr int threads = 256;
    if ((n_pix + threads - 1) / threads > 0x7FFFFFFFll)
        return nsim::report_error(NEUROSIM_E_INVALID, "n_pix too large for one launch");
    if (n_pix % 4 == 0 && aligned16(L_dev) && aligned16(out_dev) && aligned16(state_dev)) {
        const int64_t n4 = n_pix / 4;
        lowpass4_kernel<<<(unsigned)((n4 + threads - 1) / threads), threads, 0, st>>>(
            reinterpret_cast<const float4*>(L_dev), reinterpret_cast<float4*>(out_dev), n_frames, n4, alpha,
            reinterpret_cast<float4*>(state_dev), init);
    } else {
        lowpass1_kernel<<<(unsigned)((n_pix + threads - 1) / threads), threads, 0, st>>>(L_dev, out_dev, n_frames,
                                                                                           n_pix, alpha, state_dev,
                                                                                           init);
    }
    if (cudaGetLastError() != cudaSuccess) return nsim::report_error(NEUROSIM_E_CUDA, "low-pass launch failed");
    return NEUROSIM_OK;
}

extern "C" int neurosim_leak_log(const float* L_dev, float* out_dev, int32_t n_frames, int64_t n_pix, int64_t t0_us,
                                 int32_t dt_us, int64_t origin_us, double rate_hz, const float* c_pos_dev, float c_pos,
                                 void* cuda_stream)
{
    if (n_frames < 0 || n_pix < 0) return nsim::report_error(NEUROSIM_E_INVALID, "n_frames and n_pix must be >= 0");
    if (!(rate_hz >= 0.0) || !std::isfinite(rate_hz)) return nsim::report_error(NEUROSIM_E_INVALID, "rate_hz must be >= 0");
    if (dt_us < 1 || t0_us < origin_us)
        return nsim::report_error(NEUROSIM_E_TIME, "need dt_us >= 1 and t0_us >= origin_us");
    if (!c_pos_dev && !(c_pos > 0.0f)) return nsim::report_error(NEUROSIM_E_INVALID, "c_pos must be > 0");
    if (n_pix == 0 || n_frames == 0) return NEUROSIM_OK;
    if (!L_dev || !out_dev) return nsim::report_error(NEUROSIM_E_INVALID, "NULL buffer");
    if (L_dev != out_dev && (const void*)L_dev < (const void*)(out_dev + (size_t)n_frames * n_pix) &&
        (const void*)out_dev < (const void*)(L_dev + (size_t)n_frames * n_pix))
        return nsim::report_error(NEUROSIM_E_INVALID, "L_dev and out_dev overlap without being equal");
    constexpr int threads = 256;
    if ((n_pix + threads - 1) / threads > 0x7FFFFFFFll)
        return nsim::report_error(NEUROSIM_E_INVALID, "n_pix too large for one launch");
    const float rate_us = (float)(rate_hz * 1e-6);
    leak_kernel<<<(unsigned)((n_pix + threads - 1) / threads), threads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        L_dev, out_dev, n_frames, n_pix, t0_us, dt_us, origin_us, rate_us, c_pos_dev, c_pos);
    if (cudaGetLastError() != cudaSuccess) return nsim::report_error(NEUROSIM_E_CUDA, "leak launch failed");
    return NEUROSIM_OK;
}
