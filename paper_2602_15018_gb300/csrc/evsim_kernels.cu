// Event-generation kernels for sm_103a (GB300).
//
// Model: arXiv 2602.15018, Sec. 2 ("Neurosim simulates event cameras at
// multi-kilohertz rates"): per-pixel state holding the level of the last
// triggered event, contrast-threshold crossings, a variable number of events
// per frame gathered with few global atomics.  Sec. 1 fixes the event tuple
// (integer microsecond timestamp, pixel, polarity).
//
// Readings of the silent points (shared with the header's model statement):
// L = log(clamp(I, 0, 1e6) + eps) with this file's FP32 log (or clamp(I, -32,
// 32) for log input); linear interpolation of L between frames; one crossing
// at a time with sequential FP32 adds (ref moves to the crossed level);
// t = ta + floor(frac * D) with frac = (lvl - a) / (b - a) in FP32;
// refractory suppression that still moves ref; output interval-major and
// ascending by (t, y, x, p) inside an interval.
//
// Every floating-point operation of the model is an explicitly rounded
// intrinsic (__fadd_rn, __fmul_rn, __fdiv_rn, __fmaf_rn) so that no compiler
// contraction or approximation can change a result.
//
// Kernels of one step:
//   emit_kernel     (evsim_emit.cuh) one warp per tile of 32*PPT contiguous
//                   pixels for all T frames, no block-level barriers; a cheap
//                   per-pixel filter on the raw input, the exact model on a
//                   warp-converged slow path; the events of a warp tile in
//                   one interval form one contiguous chunk (pixel order) of
//                   a paged key buffer (one global atomic per page, not per
//                   frame); chunk (offset, count) goes to a table indexed by
//                   (interval, tile).
//   seg_count       sums the chunk counts of each interval.
//   seg_scan        exclusive scan of the interval sizes -> output offsets.
//   sort_kernel     one CTA per interval: gathers the interval's chunks in
//                   tile order (so pixel order), then a stable LSD radix sort
//                   on the in-interval time offset in shared memory, writing
//                   the packed 64-bit records in (t, y, x, p) order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "evsim_internal.h"
#include "scene_render.cuh"

namespace nsim {
namespace {

// --------------------------------------------------------------------------
// FP32 natural log used by the model (textbook atanh-series method):
// x = m 2^e with m in [sqrt(1/2), sqrt(2)); s = (m - 1)/(m + 1);
// log m = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9); log x = log m + e ln2, with
// ln2 split into a 16-bit head (exact product with e) and a tail.
// --------------------------------------------------------------------------
__device__ __forceinline__ float model_log(float x)
{
    if (!(x > 0.0f)) return (x == 0.0f) ? __int_as_float(0xff800000) : __int_as_float(0x7fc00000);
    if (x == __int_as_float(0x7f800000)) return x;
    int e = 0;
    uint32_t bits = __float_as_uint(x);
    if (bits < 0x00800000u) {                 // subnormal: scale by 2^24
        x = __fmul_rn(x, 16777216.0f);
        bits = __float_as_uint(x);
        e = -24;
    }
    e += (int)(bits >> 23) - 127;
    float m = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) {                 // sqrt(2) rounded to FP32
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float z = __fmul_rn(s, s);
    float q = __fmaf_rn(z, 0x1.c71c72p-4f, 0x1.24924ap-3f);   // 1/9, 1/7
    q = __fmaf_rn(z, q, 0x1.99999ap-3f);                       // 1/5
    q = __fmaf_rn(z, q, 0x1.555556p-2f);                       // 1/3
    const float s2 = __fadd_rn(s, s);
    const float lm = __fmaf_rn(s2, __fmul_rn(z, q), s2);
    const float fe = (float)e;
    const float tail = __fmaf_rn(fe, 0x1.7f7d1cp-20f, lm);     // ln2 tail
    return __fmaf_rn(fe, 0x1.62e4p-1f, tail);                   // ln2 head (16 bits)
}

// Descriptor set of this launch: the host's s0, or the device array (with a
// device clock, the set whose *_in buffers hold the current state).
__device__ __forceinline__ const StreamDesc* stream_set(const StepLaunch& L)
{
    return L.clock ? L.streams_dev + (size_t)(L.clock->parity & 1u) * L.n_streams : L.streams_dev;
}

__device__ __forceinline__ const StreamDesc* stream_of_item(const StepLaunch& L, int item)
{
    if (L.streams_dev == nullptr) return &L.s0;
    const StreamDesc* sd = stream_set(L);
    int lo = 0, hi = L.n_streams - 1;            // last stream with item_base <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sd[mid].item_base <= item) lo = mid; else hi = mid - 1;
    }
    return &sd[lo];
}

__device__ __forceinline__ const StreamDesc* stream_of_seg(const StepLaunch& L, int seg)
{
    if (L.streams_dev == nullptr) return &L.s0;
    const StreamDesc* sd = stream_set(L);
    int lo = 0, hi = L.n_streams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sd[mid].seg_base <= seg) lo = mid; else hi = mid - 1;
    }
    return &sd[lo];
}

// Start time of the step's first interval: the host's value, or the device
// clock (time of the last frame consumed).
__device__ __forceinline__ int64_t step_ta0(const StepLaunch& L, const StreamDesc& sd)
{
    return L.clock ? (int64_t)L.clock->tau : sd.ta0;
}

// Device clock: a failed earlier step stops every later one.
__device__ __forceinline__ bool step_stopped(const StepLaunch& L)
{
    return L.clock != nullptr && L.clock->sticky != 0u;
}

__device__ __forceinline__ int64_t interval_start(int64_t ta0, const StreamDesc& sd, int j, int dt)
{
    return ta0 + (j == 0 ? 0 : (int64_t)sd.D0 + (int64_t)(j - 1) * dt);
}

#include "evsim_emit.cuh"

// --------------------------------------------------------------------------
// Segment sizes and offsets
// --------------------------------------------------------------------------
__global__ void seg_count_kernel(const __grid_constant__ StepLaunch L)
{
    const int warps = blockDim.x >> 5;
    const int seg = blockIdx.x * warps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (seg >= L.n_segs || step_stopped(L)) return;
    const StreamDesc* sdp = stream_of_seg(L, seg);
    const int j = seg - sdp->seg_base;
    const uint2* row = L.chunks + sdp->chunk_base + (int64_t)j * sdp->n_tiles;
    uint32_t s = 0;
    for (int i = lane; i < sdp->n_tiles; i += 32) s += row[i].y;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) L.seg_count[seg] = s;
}

// Single CTA: exclusive scan of segment sizes; appends the step's records
// after the ones pending from earlier steps.
__global__ void __launch_bounds__(1024) seg_scan_kernel(const __grid_constant__ StepLaunch L)
{
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (step_stopped(L)) return;
    const unsigned long long base = L.ctl->run_total;
    // device clock: the step's offsets follow the pending ones, if they fit
    const int64_t pend0 = L.clock ? (int64_t)L.clock->pending_segs : 0;
    const bool pend_ok = !L.clock || pend0 + L.n_segs <= L.max_pending;
    if (tid == 0) s_carry = 0ull;
    __syncthreads();
    for (int c0 = 0; c0 < L.n_segs; c0 += 1024) {
        const int seg = c0 + tid;
        const unsigned long long v = (seg < L.n_segs) ? L.seg_count[seg] : 0ull;
        unsigned long long incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long nb = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += nb;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = s_w[lane], wi = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long nb = __shfl_up_sync(0xffffffffu, wi, d);
                if (lane >= d) wi += nb;
            }
            s_w[lane] = wi - w;
        }
        __syncthreads();
        const unsigned long long rel = s_carry + s_w[warp] + incl - v;
        if (seg < L.n_segs) {
            L.seg_rel[seg] = (int64_t)rel;
            L.seg_abs[seg] = (int64_t)(base + rel);
            if (L.clock) {
                if (pend_ok) L.seg_off_out[pend0 + seg] = (int64_t)(base + rel);
            } else {
                const StreamDesc* sdp = stream_of_seg(L, seg);
                L.seg_off_out[sdp->out_seg_index + (seg - sdp->seg_base)] = (int64_t)(base + rel);
            }
        }
        __syncthreads();
        if (tid == 1023) s_carry = rel + v;
        __syncthreads();
    }
    if (tid == 0) {
        Ctl* c = L.ctl;
        const unsigned long long total = base + s_carry;
        c->run_total = total;
        if (total > c->out_demand_max) c->out_demand_max = total;
        if (total > L.out_cap) c->err |= kErrOutOverflow;
        if (!pend_ok) c->err |= kErrPendingOverflow;
        if (c->page_ctr > c->page_demand_max) c->page_demand_max = c->page_ctr;
        c->page_ctr = 0u;                      // pages are free again for the next step
    }
}

// --------------------------------------------------------------------------
// Per-interval stable LSD radix sort on the time offset
// --------------------------------------------------------------------------
template <typename KeyT>
struct ChunkSrc {          // logical key i of the interval, gathered from its chunks
    const KeyT* keys;
    const uint32_t* cpre;  // shared: exclusive prefix of chunk counts, nt + 1 entries
    const uint32_t* coff;  // shared: page offset of each chunk
    int nt;
    __device__ __forceinline__ KeyT operator()(uint32_t i) const
    {
        int lo = 0, hi = nt - 1;                 // last chunk with cpre <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cpre[mid] <= i) lo = mid; else hi = mid - 1;
        }
        return keys[(size_t)coff[lo] + (i - cpre[lo])];
    }
};

template <typename KeyT>
struct ArraySrc {
    const KeyT* p;
    __device__ __forceinline__ KeyT operator()(uint32_t i) const { return p[i]; }
};

struct RecordSink {        // final pass: packed 64-bit records
    uint64_t* out;
    uint32_t ta;
    int W;
    int tshift;
    uint32_t pixmask;
    float invW;            // fl(1 / W)
    template <typename KeyT>
    __device__ __forceinline__ void put(uint32_t pos, KeyT key) const
    {
        const uint32_t toff = (uint32_t)(key >> tshift);
        const uint32_t pix = (uint32_t)(key >> 1) & pixmask;
        // y = pix / W: pix < 2^23 converts exactly and the product errs by
        // less than 1, so one correction step makes the quotient exact
        int y = (int)((float)pix * invW);
        int x = (int)pix - y * W;
        if (x < 0) {
            --y;
            x += W;
        } else if (x >= W) {
            ++y;
            x -= W;
        }
        out[pos] = ((uint64_t)(ta + toff) << 32) | ((uint64_t)y << 17) | ((uint64_t)x << 1) |
                   (uint64_t)(key & (KeyT)1);
    }
};

template <typename KeyT>
struct KeySink {
    KeyT* p;
    __device__ __forceinline__ void put(uint32_t pos, KeyT key) const { p[pos] = key; }
};

// Lanes of the warp (among `m`) whose digit d (of `bits` bits) equals this
// lane's: one ballot per digit bit, every lane of the warp taking part.
__device__ __forceinline__ unsigned digit_peers(uint32_t d, int bits, unsigned m)
{
    unsigned peers = m;
    for (int k = 0; k < bits; ++k) {
        const bool bit = (d >> k) & 1u;
        const unsigned b = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? b : ~b;
    }
    return peers;
}

// One stable counting pass of the CTA over [0, N): digit = (key >> shift) & (NB-1).
// Warp w owns the contiguous range [w N / NW, (w+1) N / NW); inside a warp,
// groups of 32 consecutive keys are ranked by their digit peers (lanes below
// with the same digit), so the pass keeps the input order of equal digits.
template <int THREADS, typename KeyT, typename Src, typename Sink>
__device__ __forceinline__ void radix_pass(const Src& src, const Sink& sink, uint32_t N, int shift,
                                           int NB, uint32_t* hist /*[NW][64]*/, uint32_t* binbase)
{
    constexpr int NW = THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lo = (uint32_t)(((uint64_t)N * warp) / NW);
    const uint32_t hi = (uint32_t)(((uint64_t)N * (warp + 1)) / NW);
    uint32_t* h = hist + warp * 64;
    for (int d = lane; d < 64; d += 32) h[d] = 0u;
    __syncwarp();
    const uint32_t lt = (1u << lane) - 1u;
    const int bits = 31 - __clz(NB);
    // counts of the warp's range (order does not matter here)
    for (uint32_t i = lo + lane; i < hi; i += 32)
        atomicAdd(&h[(uint32_t)(src(i) >> shift) & (uint32_t)(NB - 1)], 1u);
    __syncthreads();
    if (tid < NB) {
        uint32_t run = 0;
        for (int w = 0; w < NW; ++w) {
            const uint32_t c = hist[w * 64 + tid];
            hist[w * 64 + tid] = run;
            run += c;
        }
        binbase[tid] = run;
    }
    __syncthreads();
    if (warp == 0) {
        const uint32_t a = (lane < NB) ? binbase[lane] : 0u;
        const uint32_t b = (lane + 32 < NB) ? binbase[lane + 32] : 0u;
        uint32_t ia = a;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t nb = __shfl_up_sync(0xffffffffu, ia, d);
            if (lane >= d) ia += nb;
        }
        const uint32_t tot_a = __shfl_sync(0xffffffffu, ia, 31);
        uint32_t ib = b;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t nb = __shfl_up_sync(0xffffffffu, ib, d);
            if (lane >= d) ib += nb;
        }
        __syncwarp();
        if (lane < NB) binbase[lane] = ia - a;
        if (lane + 32 < NB) binbase[lane + 32] = tot_a + ib - b;
    }
    __syncthreads();
    for (uint32_t g = lo; g < hi; g += 32) {
        const uint32_t i = g + lane;
        const bool act = i < hi;
        const unsigned m = __ballot_sync(0xffffffffu, act);
        KeyT key = 0;
        uint32_t d = 0;
        if (act) {
            key = src(i);
            d = (uint32_t)(key >> shift) & (uint32_t)(NB - 1);
        }
        const unsigned peers = digit_peers(d, bits, m);
        if (act) {
            const uint32_t pos = binbase[d] + h[d] + (uint32_t)__popc(peers & lt);
            sink.put(pos, key);
        }
        __syncwarp();
        if (act && (peers & lt) == 0u) h[d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
}

template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads) sort_kernel(const __grid_constant__ StepLaunch L)
{
    constexpr int THREADS = kSortThreads;
    constexpr int NW = THREADS / 32;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int maxnt = L.max_tiles;
    const int cpre_len = (maxnt + 1 + 3) & ~3;                       // keep 16-byte alignment
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem_raw);         // NW * 64
    uint32_t* binbase = hist + NW * 64;                               // 64
    uint32_t* cpre = binbase + 64;                                    // maxnt + 1
    uint32_t* coff = cpre + cpre_len;                                 // maxnt
    KeyT* sbuf = reinterpret_cast<KeyT*>(coff + cpre_len);
    const size_t fixed = (size_t)(NW * 64 + 64 + 2 * cpre_len) * sizeof(uint32_t);
    const uint32_t cap = (L.sort_smem > (int)fixed)
                             ? (uint32_t)(((size_t)L.sort_smem - fixed) / sizeof(KeyT)) : 0u;

    const int tid = threadIdx.x;
    const int tb = L.t_bits;
    const int npass = (tb + kMaxDigitBits - 1) / kMaxDigitBits;
    const int bits = (tb + npass - 1) / npass;
    const int NB = 1 << bits;
    if (step_stopped(L)) return;

    for (int seg = blockIdx.x; seg < L.n_segs; seg += gridDim.x) {
        const uint32_t N = L.seg_count[seg];
        const int64_t abs0 = L.seg_abs[seg];
        if (N == 0u || (uint64_t)abs0 + N > L.out_cap) continue;    // overflow flagged by scan
        const StreamDesc* sdp = stream_of_seg(L, seg);
        const int j = seg - sdp->seg_base;
        const int nt = sdp->n_tiles;
        const uint2* row = L.chunks + sdp->chunk_base + (int64_t)j * nt;

        // exclusive prefix of the chunk counts (tile order = pixel order)
        __shared__ uint32_t s_carry;
        __shared__ uint32_t s_w[NW];
        if (tid == 0) s_carry = 0u;
        __syncthreads();
        for (int c0 = 0; c0 < nt; c0 += THREADS) {
            const int c = c0 + tid;
            uint2 e = make_uint2(0u, 0u);
            if (c < nt) e = row[c];
            uint32_t incl = e.y;
            const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t nb = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += nb;
            }
            if (lane == 31) s_w[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                const uint32_t w = (lane < NW) ? s_w[lane] : 0u;
                uint32_t wi = w;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t nb = __shfl_up_sync(0xffffffffu, wi, d);
                    if (lane >= d) wi += nb;
                }
                if (lane < NW) s_w[lane] = wi - w;
            }
            __syncthreads();
            const uint32_t ex = s_carry + s_w[warp] + incl - e.y;
            if (c < nt) { cpre[c] = ex; coff[c] = e.x; }
            __syncthreads();
            if (tid == THREADS - 1) s_carry = ex + e.y;
            __syncthreads();
        }
        if (tid == 0) cpre[nt] = s_carry;
        __syncthreads();

        const int tshift = sdp->pix_bits + 1;
        const uint32_t ta = (uint32_t)interval_start(step_ta0(L, *sdp), *sdp, j, L.dt);
        const RecordSink rsink{L.out + abs0, ta, sdp->W, tshift, (1u << sdp->pix_bits) - 1u, 1.0f / (float)sdp->W};
        if (2u * N <= cap) {
            // the interval fits twice in shared memory: copy its chunks (tile
            // order) into one array, then sort between two shared arrays
            KeyT* X = sbuf;
            KeyT* Y = sbuf + N;
            const ChunkSrc<KeyT> csrc{reinterpret_cast<const KeyT*>(L.keys), cpre, coff, nt};
            // consecutive threads take consecutive keys; four independent
            // chunk searches and loads in flight per thread
            for (uint32_t i0 = tid; i0 < N; i0 += 4 * THREADS) {
                KeyT v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t i = i0 + u * THREADS;
                    v[u] = (i < N) ? csrc(i) : (KeyT)0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t i = i0 + u * THREADS;
                    if (i < N) X[i] = v[u];
                }
            }
            __syncthreads();
            KeyT* cur = X;
            KeyT* nxt = Y;
            for (int p = 0; p < npass - 1; ++p) {
                radix_pass<THREADS, KeyT>(ArraySrc<KeyT>{cur}, KeySink<KeyT>{nxt}, N, tshift + p * bits, NB, hist,
                                          binbase);
                KeyT* t = cur;
                cur = nxt;
                nxt = t;
            }
            radix_pass<THREADS, KeyT>(ArraySrc<KeyT>{cur}, rsink, N, tshift + (npass - 1) * bits, NB, hist, binbase);
            continue;
        }
        const bool fit = (npass <= 2) ? (N <= cap) : (2u * N <= cap);
        KeyT* X = fit ? sbuf : reinterpret_cast<KeyT*>(L.temp) + L.seg_rel[seg];
        KeyT* Y = fit ? sbuf + N : reinterpret_cast<KeyT*>(L.out + abs0);
        const ChunkSrc<KeyT> csrc{reinterpret_cast<const KeyT*>(L.keys), cpre, coff, nt};

        if (npass == 1) {
            radix_pass<THREADS, KeyT>(csrc, rsink, N, tshift, NB, hist, binbase);
        } else {
            // pass p writes to X when (npass - 2 - p) is even, else to Y; last pass -> records
            KeyT* dst0 = ((npass - 2) % 2 == 0) ? X : Y;
            radix_pass<THREADS, KeyT>(csrc, KeySink<KeyT>{dst0}, N, tshift, NB, hist, binbase);
            KeyT* cur = dst0;
            for (int p = 1; p < npass - 1; ++p) {
                KeyT* dst = ((npass - 2 - p) % 2 == 0) ? X : Y;
                radix_pass<THREADS, KeyT>(ArraySrc<KeyT>{cur}, KeySink<KeyT>{dst}, N,
                                          tshift + p * bits, NB, hist, binbase);
                cur = dst;
            }
            radix_pass<THREADS, KeyT>(ArraySrc<KeyT>{cur}, rsink, N, tshift + (npass - 1) * bits,
                                      NB, hist, binbase);
        }
    }
}

// --------------------------------------------------------------------------
// Create-time thresholds and the log check kernel
// --------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1ull) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Irwin-Hall(12) normal: twelve 20-bit uniforms summed, minus 6 * 2^20, times 2^-20.
__device__ __forceinline__ float normal_ih12(uint64_t seed, uint64_t slot)
{
    int64_t acc = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc += (int64_t)(splitmix64_at(seed, slot * 12ull + (uint64_t)k) >> 44);
    return __fmul_rn((float)(acc - 6ll * (1ll << 20)), 0x1p-20f);
}

__global__ void threshold_kernel(float* cpos, float* cneg, int64_t npix, float c_pos, float c_neg,
                                 float sigma, float c_min, uint64_t seed)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < npix;
         u += (int64_t)gridDim.x * blockDim.x) {
        float vp = c_pos, vn = c_neg;
        if (sigma != 0.0f) {
            vp = __fadd_rn(c_pos, __fmul_rn(sigma, normal_ih12(seed, (uint64_t)u * 2ull)));
            vn = __fadd_rn(c_neg, __fmul_rn(sigma, normal_ih12(seed, (uint64_t)u * 2ull + 1ull)));
        }
        cpos[u] = fmaxf(c_min, vp);
        cneg[u] = fmaxf(c_min, vn);
    }
}

// The event model's log intensity of raw frames: L = log(clamp(I, 0, 1e6) + eps)
// with the library's log (the same function the emission kernel applies).
__global__ void log_intensity_kernel(const float* I, float* L, int64_t n, float eps)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        L[i] = model_L(I[i], eps, 0);
}

__global__ void debug_log_kernel(const float* x, float* y, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = model_log(x[i]);
}

// Closing offset of the interval list: the record count after the step.
__global__ void write_total_kernel(const Ctl* ctl, int64_t* dst)
{
    *dst = (int64_t)ctl->run_total;
}

// Device clock: commits a step that raised no error (state parity, time,
// pending offsets, committed records), or discards it and stops later steps.
// `add_tau` advances the clock by the step's span; an init launch (add_tau
// < 0) sets it to tau_init.
__global__ void advance_kernel(DevClock* clk, Ctl* ctl, int n_segs, long long add_tau, long long tau_init)
{
    if (clk->sticky != 0u) return;
    unsigned int err = ctl->err;
    const long long tau = add_tau < 0 ? tau_init : clk->tau + add_tau;
    if (tau > 0xFFFFFFFEll) err |= kErrTime;
    if (err != 0u) {
        clk->sticky = err;
        ctl->run_total = clk->committed_total;   // the step's records are dropped
        return;
    }
    clk->parity ^= 1u;
    clk->tau = tau;
    clk->pending_segs += n_segs;
    clk->committed_total = ctl->run_total;
    clk->steps += 1ull;
}

// A rendered step (scene_tab set) takes the frames from the texture renderer.
template <int PPT, int PF>
cudaError_t launch_emit_t(const StepLaunch& L, size_t smem)
{
    constexpr int WARPS = 64 / PPT;
    // (the dynamic shared-memory attribute was set by emit_occupancy at create
    // time, so that launches stay capturable)
    const bool tex = L.n_streams == 1 && L.streams_dev == nullptr && L.s0.scene_tab != nullptr;
    if (tex) {
        if (L.key64)
            emit_kernel<PPT, WARPS, PF, uint64_t, 1><<<L.grid_emit, WARPS * 32, smem, L.stream>>>(L);
        else
            emit_kernel<PPT, WARPS, PF, uint32_t, 1><<<L.grid_emit, WARPS * 32, smem, L.stream>>>(L);
    } else if (L.key64) {
        emit_kernel<PPT, WARPS, PF, uint64_t, 0><<<L.grid_emit, WARPS * 32, smem, L.stream>>>(L);
    } else {
        emit_kernel<PPT, WARPS, PF, uint32_t, 0><<<L.grid_emit, WARPS * 32, smem, L.stream>>>(L);
    }
    return cudaGetLastError();
}

const void* emit_fn(int ppt, int pf, int key64, int src)
{
#define NSIM_PICK(P, F)                                                                                 \
    if (ppt == P && pf == F) {                                                                          \
        if (src) return key64 ? (const void*)emit_kernel<P, 64 / P, F, uint64_t, 1>                    \
                              : (const void*)emit_kernel<P, 64 / P, F, uint32_t, 1>;                   \
        return key64 ? (const void*)emit_kernel<P, 64 / P, F, uint64_t, 0>                             \
                     : (const void*)emit_kernel<P, 64 / P, F, uint32_t, 0>;                            \
    }
    NSIM_PICK(8, 2) NSIM_PICK(8, 3) NSIM_PICK(16, 2) NSIM_PICK(16, 3)
#undef NSIM_PICK
    return nullptr;
}

}  // namespace

int emit_warps_per_cta(int ppt) { return 64 / ppt; }

size_t emit_smem_bytes(int ppt)
{
    const size_t per_warp = (ppt == 8) ? WarpSlice<8>::FLOATS : WarpSlice<16>::FLOATS;
    return (size_t)emit_warps_per_cta(ppt) * per_warp * sizeof(float);
}

cudaError_t emit_occupancy(int ppt, int pf, int key64, int* blocks_per_sm, int src)
{
    const void* fn = emit_fn(ppt, pf, key64, src);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = emit_smem_bytes(ppt);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, emit_warps_per_cta(ppt) * 32, smem);
}

cudaError_t sort_configure(int* smem_bytes)
{
    // two sort CTAs per SM: 110 KB of shared memory each (with the 1 KB the
    // runtime reserves per CTA, two fit in the 228 KB of an SM)
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    int want = 110 * 1024;
    if (want > optin) want = optin;
    e = cudaFuncSetAttribute(sort_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sort_kernel<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
    if (e != cudaSuccess) return e;
    *smem_bytes = want;
    return cudaSuccess;
}

cudaError_t launch_step(const StepLaunch& L, uint64_t* launches)
{
    cudaError_t e = cudaSuccess;
    if (L.ev_begin && (e = cudaEventRecord(L.ev_begin, L.stream)) != cudaSuccess) return e;
    const size_t smem = emit_smem_bytes(L.ppt);
    if (L.ppt == 8 && L.pf == 2) e = launch_emit_t<8, 2>(L, smem);
    else if (L.ppt == 8 && L.pf == 3) e = launch_emit_t<8, 3>(L, smem);
    else if (L.ppt == 16 && L.pf == 2) e = launch_emit_t<16, 2>(L, smem);
    else if (L.ppt == 16 && L.pf == 3) e = launch_emit_t<16, 3>(L, smem);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    *launches += 1;
    if (L.ev_emitted && (e = cudaEventRecord(L.ev_emitted, L.stream)) != cudaSuccess) return e;
    if (L.n_segs > 0) {
        const int wpb = 8;
        seg_count_kernel<<<(L.n_segs + wpb - 1) / wpb, wpb * 32, 0, L.stream>>>(L);
        seg_scan_kernel<<<1, 1024, 0, L.stream>>>(L);
        if (L.key64)
            sort_kernel<uint64_t><<<L.grid_sort, kSortThreads, L.sort_smem, L.stream>>>(L);
        else
            sort_kernel<uint32_t><<<L.grid_sort, kSortThreads, L.sort_smem, L.stream>>>(L);
        *launches += 3;
    }
    if (L.clock) {
        const bool init = L.n_segs == 0;   // an init launch consumes one frame: no intervals
        advance_kernel<<<1, 1, 0, L.stream>>>(L.clock, L.ctl, L.n_segs,
                                              init ? -1ll : (long long)L.T * L.dt, (long long)L.tau_init);
        *launches += 1;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (L.ev_sorted && (e = cudaEventRecord(L.ev_sorted, L.stream)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_threshold_maps(float* cpos, float* cneg, int64_t npix, float c_pos, float c_neg,
                                  float sigma, float c_min, uint64_t seed, cudaStream_t stream)
{
    const int threads = 256;
    int64_t blocks = (npix + threads - 1) / threads;
    if (blocks > 65535) blocks = 65535;
    threshold_kernel<<<(unsigned)blocks, threads, 0, stream>>>(cpos, cneg, npix, c_pos, c_neg, sigma,
                                                                c_min, seed);
    return cudaGetLastError();
}

cudaError_t launch_log_intensity(const float* I, float* L, int64_t n, float eps, cudaStream_t stream)
{
    const int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    log_intensity_kernel<<<(unsigned)blocks, threads, 0, stream>>>(I, L, n, eps);
    return cudaGetLastError();
}

cudaError_t launch_debug_log(const float* x, float* y, int64_t n, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    debug_log_kernel<<<(unsigned)blocks, threads, 0, stream>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_write_total(const Ctl* ctl, int64_t* dst, cudaStream_t stream)
{
    write_total_kernel<<<1, 1, 0, stream>>>(ctl, dst);
    return cudaGetLastError();
}

}  // namespace nsim
