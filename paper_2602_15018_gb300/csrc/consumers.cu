// Event-stream consumers on the device (declared in include/neurosim_evsim.h):
// the time surface of the paper's RL appendix (Observation Space paragraph),
//   S(x, y, p) <- S(x, y, p) * exp(-dt / tau) + 1 at every event,
// and per-window polarity event frames (the 20 ms frames of Fig. 1).
//
// Time surface: the library keeps S evaluated at one reference time t_ref
// for every cell.  Moving it to a later query time t_q and adding the events
// of (t_ref, t_q] is, by exp(a) exp(b) = exp(a + b),
//   S(t_q) = S(t_ref) exp(-(t_q - t_ref) / tau) + sum_i exp(-(t_q - t_i) / tau),
// which equals the per-event recursion evaluated at t_q up to rounding, and
// is order-independent: one decay pass over the cells and one atomic add per
// event, with no sort.  Event frames are integer atomics and exact.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"

namespace {

__global__ void decay_kernel(float* S, int64_t cells, float factor)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x)
        S[i] *= factor;
}

// rec: [63:32] t | [31:17] y | [16:1] x | [0] p
__global__ void surface_add_kernel(float* S, int W, int H, const uint64_t* ev, int64_t n, int64_t t_q, float inv_tau,
                                   unsigned int* bad)
{
    const int64_t plane = (int64_t)W * H;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e = ev[i];
        const int64_t t = (int64_t)(e >> 32);
        const int y = (int)((e >> 17) & 0x7FFFu), x = (int)((e >> 1) & 0xFFFFu), p = (int)(e & 1u);
        if (x >= W || y >= H || t > t_q) {
            atomicOr(bad, 1u);
            continue;
        }
        atomicAdd(S + p * plane + (int64_t)y * W + x, expf(-(float)(t_q - t) * inv_tau));
    }
}

__global__ void frames_kernel(int32_t* out, int W, int H, const uint64_t* ev, int64_t n, int64_t t_start, int64_t win,
                              int n_win, unsigned int* bad)
{
    const int64_t plane = (int64_t)W * H;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e = ev[i];
        const int64_t t = (int64_t)(e >> 32);
        const int y = (int)((e >> 17) & 0x7FFFu), x = (int)((e >> 1) & 0xFFFFu), p = (int)(e & 1u);
        if (x >= W || y >= H) {
            atomicOr(bad, 1u);
            continue;
        }
        if (t < t_start) continue;
        const int64_t w = (t - t_start) / win;
        if (w >= n_win) continue;
        atomicAdd(out + (w * 2 + p) * plane + (int64_t)y * W + x, 1);
    }
}

unsigned grid_of(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 8192) b = 8192;
    return (unsigned)(b < 1 ? 1 : b);
}

int check_flag(unsigned int* bad, cudaStream_t st, const char* what)
{
    unsigned int h = 0;
    if (cudaMemcpyAsync(&h, bad, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaFreeAsync(bad, st);
        return nsim::report_error(NEUROSIM_E_CUDA, "consumer kernel failed");
    }
    cudaFreeAsync(bad, st);
    if (h) return nsim::report_error(NEUROSIM_E_INVALID, what);
    return NEUROSIM_OK;
}

}  // namespace

extern "C" int neurosim_time_surface(float* S_dev, int32_t width, int32_t height, int64_t* t_ref_us,
                                     const uint64_t* events_dev, int64_t n, int64_t t_query_us, float tau_us,
                                     void* cuda_stream)
{
    if (!S_dev || !t_ref_us || (n > 0 && !events_dev) || n < 0 || width < 1 || height < 1)
        return nsim::report_error(NEUROSIM_E_INVALID, "bad arguments to neurosim_time_surface");
    if (!(tau_us > 0.0f)) return nsim::report_error(NEUROSIM_E_INVALID, "tau_us must be > 0");
    if (t_query_us < *t_ref_us) return nsim::report_error(NEUROSIM_E_TIME, "t_query_us is before the surface's time");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t cells = 2ll * width * height;
    unsigned int* bad = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&bad), sizeof(unsigned int), st) != cudaSuccess ||
        cudaMemsetAsync(bad, 0, sizeof(unsigned int), st) != cudaSuccess)
        return nsim::report_error(NEUROSIM_E_CUDA, "cannot allocate the error word");
    const float factor = expf(-(float)(t_query_us - *t_ref_us) / tau_us);
    if (factor != 1.0f) decay_kernel<<<grid_of(cells), 256, 0, st>>>(S_dev, cells, factor);
    if (n > 0)
        surface_add_kernel<<<grid_of(n), 256, 0, st>>>(S_dev, width, height, events_dev, n, t_query_us,
                                                       1.0f / tau_us, bad);
    if (cudaGetLastError() != cudaSuccess) {
        cudaFreeAsync(bad, st);
        return nsim::report_error(NEUROSIM_E_CUDA, "time-surface launch failed");
    }
    const int rc = check_flag(bad, st, "an event lies outside the sensor or after t_query_us");
    if (rc == NEUROSIM_OK) *t_ref_us = t_query_us;
    return rc;
}

extern "C" int neurosim_event_frames(int32_t* counts_dev, int32_t width, int32_t height, const uint64_t* events_dev,
                                     int64_t n, int64_t t_start_us, int64_t window_us, int32_t n_windows,
                                     void* cuda_stream)
{
    if (!counts_dev || (n > 0 && !events_dev) || n < 0 || width < 1 || height < 1 || window_us < 1 || n_windows < 1)
        return nsim::report_error(NEUROSIM_E_INVALID, "bad arguments to neurosim_event_frames");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned int* bad = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&bad), sizeof(unsigned int), st) != cudaSuccess ||
        cudaMemsetAsync(bad, 0, sizeof(unsigned int), st) != cudaSuccess)
        return nsim::report_error(NEUROSIM_E_CUDA, "cannot allocate the error word");
    if (n > 0)
        frames_kernel<<<grid_of(n), 256, 0, st>>>(counts_dev, width, height, events_dev, n, t_start_us, window_us,
                                                  n_windows, bad);
    if (cudaGetLastError() != cudaSuccess) {
        cudaFreeAsync(bad, st);
        return nsim::report_error(NEUROSIM_E_CUDA, "event-frame launch failed");
    }
    return check_flag(bad, st, "an event lies outside the sensor");
}
