// Sensor shot noise and the merging of event streams (declared in
// include/neurosim_evsim.h as neurosim_shot_noise and neurosim_merge_events).
//
// Sec. 2 of the paper lists noise among the non-idealities Neurosim models,
// with no model.  This library's reading of shot noise: spurious events,
// independent of the signal and of the pixel state.  For every tile of 64
// consecutive pixels (row-major; the last one may be shorter, `len` pixels)
// and every interval (start ta, length D us) the count is Poisson with mean
// lambda = rate * len * D * 1e-6, drawn by inversion of the 53-bit uniform
// U of SplitMix64 output (ta * n_tiles + tile) * 32 of the noise seed: the
// least n with U < floor(F(n) 2^53), F the Poisson CDF, at most 15 (the mean
// is kept at most 4).  Event i takes outputs base + 1 + 2i (pixel
// tile * 64 + floor(hi32 * len / 2^32), time ta + floor(lo32 * D / 2^32))
// and base + 2 + 2i (polarity: the top bit).  SplitMix64 is the published
// generator (Steele, Lea and Flood, OOPSLA 2014) used as a counter-based one.
// The thresholds floor(F(n) 2^53) are computed on the host in double.
//
// Kernels: one thread per (interval, tile) for the counts; one CTA per
// interval scans its tiles' counts, writes their events into shared memory,
// sorts them (bitonic network on packed records) and writes the interval's
// records in the order of the event stream; a merge kernel places every
// record of two sorted streams by a binary search in the other one.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"

namespace nsim {
namespace {

constexpr int kShotTile = 64;
constexpr int kShotMax = 15;
constexpr int kShotSortCap = 8192;   // records of one interval sorted in shared memory
constexpr int kShotThreads = 512;

struct ShotTables {
    // thresholds of the four means: [first interval?][ragged last tile?][n]
    unsigned long long thr[2][2][kShotMax];
};

__device__ __forceinline__ uint64_t splitmix_at(uint64_t seed, uint64_t index)
{
    uint64_t z = seed + (index + 1ull) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

struct ShotGeom {
    uint64_t seed;
    int64_t npix, n_tiles;
    int32_t W;
    int64_t ta0;
    int32_t D0, dt;
    int32_t n_intervals;
    int32_t last_len;     // pixels of the last tile
};

__device__ __forceinline__ void interval_at(const ShotGeom& g, int j, int64_t& ta, int32_t& D)
{
    ta = j == 0 ? g.ta0 : g.ta0 + g.D0 + (int64_t)(j - 1) * g.dt;
    D = j == 0 ? g.D0 : g.dt;
}

__device__ __forceinline__ int shot_count(const ShotGeom& g, const ShotTables& tb, int j, int64_t tile, int64_t ta)
{
    const bool last = tile == g.n_tiles - 1 && g.last_len != kShotTile;
    const unsigned long long* thr = tb.thr[j == 0 ? 1 : 0][last ? 1 : 0];
    const uint64_t base = ((uint64_t)ta * (uint64_t)g.n_tiles + (uint64_t)tile) * 32ull;
    const uint64_t U = splitmix_at(g.seed, base) >> 11;
    int n = kShotMax;
    for (int k = kShotMax - 1; k >= 0; --k)
        if (U < thr[k]) n = k;
    return n;
}

// counts[j * n_tiles + tile], and the per-interval totals (atomics).
__global__ void shot_count_kernel(ShotGeom g, ShotTables tb, uint8_t* counts, unsigned long long* totals)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)g.n_intervals * g.n_tiles) return;
    const int j = (int)(i / g.n_tiles);
    const int64_t tile = i - (int64_t)j * g.n_tiles;
    int64_t ta;
    int32_t D;
    interval_at(g, j, ta, D);
    const int n = shot_count(g, tb, j, tile, ta);
    counts[i] = (uint8_t)n;
    if (n) atomicAdd(&totals[j], (unsigned long long)n);
}

// One CTA per interval: events of every tile into shared memory at the
// tile's prefix position, bitonic sort, write out.
__global__ void __launch_bounds__(kShotThreads) shot_emit_kernel(ShotGeom g, const uint8_t* counts,
                                                                 const int64_t* seg, uint64_t* out,
                                                                 unsigned int* err)
{
    extern __shared__ unsigned long long rec[];
    __shared__ unsigned int s_warp[kShotThreads / 32];
    __shared__ unsigned int s_carry;
    const int j = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n_j = seg[j + 1] - seg[j];
    if (n_j > kShotSortCap) {
        if (tid == 0) atomicOr(err, 1u);
        return;
    }
    int64_t ta;
    int32_t D;
    interval_at(g, j, ta, D);
    if (tid == 0) s_carry = 0u;
    __syncthreads();
    for (int64_t t0 = 0; t0 < g.n_tiles; t0 += kShotThreads) {
        const int64_t tile = t0 + tid;
        const unsigned int c = tile < g.n_tiles ? counts[(int64_t)j * g.n_tiles + tile] : 0u;
        unsigned int incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned int nb = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += nb;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const unsigned int w = lane < kShotThreads / 32 ? s_warp[lane] : 0u;
            unsigned int wi = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned int nb = __shfl_up_sync(0xffffffffu, wi, d);
                if (lane >= d) wi += nb;
            }
            if (lane < kShotThreads / 32) s_warp[lane] = wi - w;
        }
        __syncthreads();
        const unsigned int pos = s_carry + s_warp[warp] + incl - c;
        if (c) {
            const int64_t len = (tile == g.n_tiles - 1) ? g.last_len : kShotTile;
            const uint64_t base = ((uint64_t)ta * (uint64_t)g.n_tiles + (uint64_t)tile) * 32ull;
            for (unsigned int i = 0; i < c; ++i) {
                const uint64_t d1 = splitmix_at(g.seed, base + 1ull + 2ull * i);
                const uint64_t d2 = splitmix_at(g.seed, base + 2ull + 2ull * i);
                const int64_t pix = tile * kShotTile + (int64_t)(((d1 >> 32) * (uint64_t)len) >> 32);
                const uint64_t t = (uint64_t)ta + (((d1 & 0xFFFFFFFFull) * (uint64_t)D) >> 32);
                const uint32_t y = (uint32_t)(pix / g.W), x = (uint32_t)(pix - (int64_t)y * g.W);
                rec[pos + i] = (t << 32) | ((uint64_t)y << 17) | ((uint64_t)x << 1) | (d2 >> 63);
            }
        }
        __syncthreads();
        if (tid == kShotThreads - 1) s_carry = pos + c;
        __syncthreads();
    }
    const int n = (int)n_j;
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = n + tid; i < P; i += kShotThreads) rec[i] = ~0ull;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int s = k >> 1; s > 0; s >>= 1) {
            for (int i = tid; i < P; i += kShotThreads) {
                const int l = i ^ s;
                if (l > i) {
                    const unsigned long long a = rec[i], b = rec[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        rec[i] = b;
                        rec[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    uint64_t* dst = out + seg[j];
    for (int i = tid; i < n; i += kShotThreads) dst[i] = rec[i];
}

// Every record of two interval-structured sorted streams to its place in the
// merged stream: its index in its own interval plus its rank in the other
// stream's interval (records of a before equal records of b).
__global__ void merge_kernel(const uint64_t* a, const int64_t* seg_a, const uint64_t* b, const int64_t* seg_b,
                             int n_int, int64_t na, int64_t nb, uint64_t* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na + nb) return;
    const bool in_a = i < na;
    const int64_t k = in_a ? i : i - na;
    const int64_t* sx = in_a ? seg_a : seg_b;
    const int64_t* so = in_a ? seg_b : seg_a;
    const uint64_t* other = in_a ? b : a;
    int lo = 0, hi = n_int - 1;          // interval: last j with sx[j] <= k
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sx[mid] <= k) lo = mid; else hi = mid - 1;
    }
    const int j = lo;
    const uint64_t v = (in_a ? a : b)[k];
    int64_t l = so[j], h = so[j + 1];   // a: count of b < v; b: count of a <= v
    while (l < h) {
        const int64_t m = (l + h) >> 1;
        const bool before = in_a ? (other[m] < v) : (other[m] <= v);
        if (before) l = m + 1; else h = m;
    }
    out[seg_a[j] + seg_b[j] + (k - sx[j]) + (l - so[j])] = v;
}

void poisson_thresholds(double lam, unsigned long long* thr)
{
    double p = std::exp(-lam), F = p;
    for (int k = 0; k < kShotMax; ++k) {
        const double v = F * 9007199254740992.0;   // 2^53
        thr[k] = v >= 9007199254740992.0 ? (1ull << 53) : (unsigned long long)v;
        p = p * lam / (double)(k + 1);
        F += p;
    }
}

}  // namespace
}  // namespace nsim

using namespace nsim;

extern "C" int neurosim_shot_noise(int32_t width, int32_t height, double rate_hz, uint64_t seed, int64_t ta0_us,
                                   int32_t D0_us, int32_t dt_us, int32_t n_intervals, uint64_t* events_dev,
                                   uint64_t capacity, int64_t* seg_offsets, uint64_t* n_events, void* cuda_stream)
{
    if (width < 1 || height < 1 || width > 65535 || height > 32767)
        return report_error(NEUROSIM_E_INVALID, "width/height out of range");
    if (n_intervals < 0) return report_error(NEUROSIM_E_INVALID, "n_intervals < 0");
    if (!(rate_hz >= 0.0) || !std::isfinite(rate_hz)) return report_error(NEUROSIM_E_INVALID, "rate_hz must be >= 0");
    if (D0_us < 1 || dt_us < 1 || D0_us >= (1 << 24) || dt_us >= (1 << 24) || ta0_us < 0)
        return report_error(NEUROSIM_E_TIME, "need ta0_us >= 0 and interval lengths in [1, 2^24)");
    if (rate_hz * kShotTile * (double)std::max(D0_us, dt_us) * 1e-6 > 4.0)
        return report_error(NEUROSIM_E_INVALID, "rate too high: the mean count of a 64-pixel tile must be <= 4");
    if (!seg_offsets || !n_events) return report_error(NEUROSIM_E_INVALID, "NULL output");
    const int64_t last_t = ta0_us + (n_intervals > 0 ? D0_us + (int64_t)(n_intervals - 1) * dt_us : 0);
    if (last_t > 0xFFFFFFFFll) return report_error(NEUROSIM_E_TIME, "times exceed 2^32 us");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    ShotGeom g;
    g.seed = seed;
    g.npix = (int64_t)width * height;
    g.n_tiles = (g.npix + kShotTile - 1) / kShotTile;
    g.W = width;
    g.ta0 = ta0_us;
    g.D0 = D0_us;
    g.dt = dt_us;
    g.n_intervals = n_intervals;
    g.last_len = (int32_t)(g.npix - (g.n_tiles - 1) * kShotTile);
    seg_offsets[0] = 0;
    *n_events = 0;
    if (n_intervals == 0) return NEUROSIM_OK;
    ShotTables tb;
    for (int first = 0; first < 2; ++first)
        for (int last = 0; last < 2; ++last) {
            const double len = last ? g.last_len : kShotTile;
            const double D = first ? D0_us : dt_us;
            poisson_thresholds(rate_hz * len * D * 1e-6, tb.thr[first][last]);
        }
    const int64_t n_items = (int64_t)n_intervals * g.n_tiles;
    uint8_t* counts = nullptr;
    unsigned long long* totals = nullptr;
    int64_t* seg_dev = nullptr;
    unsigned int* err = nullptr;
    int rc = NEUROSIM_OK;
    std::vector<unsigned long long> tot((size_t)n_intervals);
    unsigned int herr = 0;
    if (cudaMallocAsync(reinterpret_cast<void**>(&counts), (size_t)n_items, st) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&totals), (size_t)n_intervals * 8, st) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&seg_dev), (size_t)(n_intervals + 1) * 8, st) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&err), 4, st) != cudaSuccess) {
        rc = report_error(NEUROSIM_E_NOMEM, "cannot allocate the shot-noise scratch");
        goto done;
    }
    if (cudaMemsetAsync(totals, 0, (size_t)n_intervals * 8, st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, 4, st) != cudaSuccess) {
        rc = report_error(NEUROSIM_E_CUDA, "memset failed");
        goto done;
    }
    shot_count_kernel<<<(unsigned)((n_items + 255) / 256), 256, 0, st>>>(g, tb, counts, totals);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(tot.data(), totals, (size_t)n_intervals * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        rc = report_error(NEUROSIM_E_CUDA, "shot-noise count failed");
        goto done;
    }
    for (int j = 0; j < n_intervals; ++j) {
        if (tot[j] > (unsigned long long)kShotSortCap) {
            rc = report_error(NEUROSIM_E_OVERFLOW, "more than 8192 shot-noise events in one interval");
            goto done;
        }
        seg_offsets[j + 1] = seg_offsets[j] + (int64_t)tot[j];
    }
    *n_events = (uint64_t)seg_offsets[n_intervals];
    if (*n_events > capacity) {
        rc = report_error(NEUROSIM_E_OVERFLOW, "capacity below the shot-noise event count (see *n_events)");
        goto done;
    }
    if (*n_events > 0 && !events_dev) {
        rc = report_error(NEUROSIM_E_INVALID, "events_dev is NULL");
        goto done;
    }
    if (cudaMemcpyAsync(seg_dev, seg_offsets, (size_t)(n_intervals + 1) * 8, cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
        rc = report_error(NEUROSIM_E_CUDA, "offset copy failed");
        goto done;
    }
    {
        const int smem = kShotSortCap * 8;
        if (cudaFuncSetAttribute(shot_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
            rc = report_error(NEUROSIM_E_CUDA, "cannot configure the shot-noise kernel");
            goto done;
        }
        shot_emit_kernel<<<(unsigned)n_intervals, kShotThreads, smem, st>>>(g, counts, seg_dev, events_dev, err);
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        rc = report_error(NEUROSIM_E_CUDA, "shot-noise emission failed");
        goto done;
    }
    if (herr) rc = report_error(NEUROSIM_E_OVERFLOW, "more than 8192 shot-noise events in one interval");
done:
    if (counts) cudaFreeAsync(counts, st);
    if (totals) cudaFreeAsync(totals, st);
    if (seg_dev) cudaFreeAsync(seg_dev, st);
    if (err) cudaFreeAsync(err, st);
    cudaStreamSynchronize(st);
    return rc;
}

extern "C" int neurosim_merge_events(const uint64_t* a_dev, const int64_t* seg_a, const uint64_t* b_dev,
                                     const int64_t* seg_b, int32_t n_intervals, uint64_t* out_dev,
                                     int64_t* seg_out, void* cuda_stream)
{
    if (n_intervals < 0 || !seg_a || !seg_b) return report_error(NEUROSIM_E_INVALID, "bad interval offsets");
    for (int j = 0; j < n_intervals; ++j)
        if (seg_a[j + 1] < seg_a[j] || seg_b[j + 1] < seg_b[j])
            return report_error(NEUROSIM_E_INVALID, "offsets must not decrease");
    if (seg_a[0] != 0 || seg_b[0] != 0) return report_error(NEUROSIM_E_INVALID, "offsets must start at 0");
    const int64_t na = seg_a[n_intervals], nb = seg_b[n_intervals];
    if (seg_out)
        for (int j = 0; j <= n_intervals; ++j) seg_out[j] = seg_a[j] + seg_b[j];
    if (na + nb == 0 || n_intervals == 0) return NEUROSIM_OK;
    if (!out_dev || (na && !a_dev) || (nb && !b_dev)) return report_error(NEUROSIM_E_INVALID, "NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int64_t* segs = nullptr;
    const size_t bytes = (size_t)(n_intervals + 1) * 8;
    if (cudaMallocAsync(reinterpret_cast<void**>(&segs), 2 * bytes, st) != cudaSuccess)
        return report_error(NEUROSIM_E_NOMEM, "cannot allocate the offsets");
    int rc = NEUROSIM_OK;
    if (cudaMemcpyAsync(segs, seg_a, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(segs + n_intervals + 1, seg_b, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = report_error(NEUROSIM_E_CUDA, "offset copy failed");
    } else {
        merge_kernel<<<(unsigned)((na + nb + 255) / 256), 256, 0, st>>>(a_dev, segs, b_dev, segs + n_intervals + 1,
                                                                        n_intervals, na, nb, out_dev);
        if (cudaGetLastError() != cudaSuccess) rc = report_error(NEUROSIM_E_CUDA, "merge launch failed");
    }
    cudaFreeAsync(segs, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == NEUROSIM_OK)
        rc = report_error(NEUROSIM_E_CUDA, "merge failed");
    return rc;
}
