// C-ABI host code of the batched simulator (declarations and semantics in
// include/neurosim_evsim.h, "Batched sensors").  Many independent sensor
// streams of mixed resolutions share one launch per kernel and step; the
// step's changing quantities live in a device clock so that the launches can
// be captured once into a CUDA graph and replayed (arXiv 2602.15018, Sec. 4
// and the RL appendix: several simulation instances run concurrently on one
// GPU).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"

using namespace nsim;

namespace nsim {
int validate_stream_params(const neurosim_evsim_params* p);   // evsim_api.cu
}

namespace {

constexpr uint32_t kBatchPageKeys = 2048;   // smaller pages: many warps hold a partial page
constexpr uint64_t kBatchWaitLimitNs = 2000000000ull;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return report_error(code, buf);
}

#define BCUDA(expr)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(NEUROSIM_E_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                           \
    } while (0)

int bits_of(uint64_t v)
{
    int b = 1;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

struct BatchStream {
    int W = 0, H = 0, npix = 0, pix_bits = 1, n_tiles = 0;
    float* ref[2] = {nullptr, nullptr};
    float* lprev[2] = {nullptr, nullptr};
    uint32_t* tlast[2] = {nullptr, nullptr};
    float* cpos = nullptr;   // null: uniform thresholds
    float* cneg = nullptr;
    float cpos_u = 0.2f, cneg_u = 0.2f;
    neurosim_evsim_params p{};
};

}  // namespace

struct neurosim_evsim_batch {
    neurosim_evsim_batch_params bp{};
    cudaStream_t stream = nullptr;
    int device = 0, sms = 0;
    int n = 0, T = 0, dt = 0;
    int ppt = 16, pf = 2;
    int key64 = 0, t_bits = 1;
    int n_items = 0, max_tiles = 0, grid_emit = 0, sort_smem = 0;
    int64_t n_segs = 0;           // intervals per step (n_streams * T)
    int64_t max_pending = 0;      // pending interval capacity
    std::vector<BatchStream> s;

    int slots = 2;
    StreamDesc* d_step = nullptr;   // [slots][2][n] step descriptors (by slot and state parity)
    StreamDesc* d_init = nullptr;   // [2][n] init descriptors
    void* keys = nullptr;
    void* temp = nullptr;
    size_t key_bytes = 0;
    uint32_t n_pages = 0;
    uint2* chunks = nullptr;
    uint32_t* seg_count = nullptr;
    int64_t* seg_rel = nullptr;
    int64_t* seg_abs = nullptr;
    int64_t* seg_off = nullptr;   // [max_pending]
    uint64_t* out = nullptr;
    uint64_t out_cap = 0;
    Ctl* ctl = nullptr;
    DevClock* clock = nullptr;

    std::vector<bool> slot_set;
    bool initialised = false;
    uint64_t launches = 0;
};

namespace {

void release(neurosim_evsim_batch* b)
{
    for (auto& st : b->s) {
        for (int i = 0; i < 2; ++i) {
            if (st.ref[i]) cudaFree(st.ref[i]);
            if (st.lprev[i]) cudaFree(st.lprev[i]);
            if (st.tlast[i]) cudaFree(st.tlast[i]);
        }
        if (st.cpos) cudaFree(st.cpos);
        if (st.cneg) cudaFree(st.cneg);
    }
    void* ptrs[] = {b->d_step, b->d_init, b->keys, b->temp, b->chunks, b->seg_count, b->seg_rel,
                    b->seg_abs, b->seg_off, b->out, b->ctl, b->clock};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// Descriptor of stream i for a launch whose state is read from buffer `par`.
StreamDesc make_desc(const neurosim_evsim_batch* b, int i, int par, bool init, const float* frames,
                     int64_t frame_stride, int item_base, int seg_base, int64_t chunk_base)
{
    const BatchStream& st = b->s[i];
    StreamDesc d;
    memset(&d, 0, sizeof d);
    d.frames = frames;
    d.ref_in = st.ref[par];
    d.lprev_in = st.lprev[par];
    d.tlast_in = st.tlast[par];
    d.ref_out = st.ref[1 - par];
    d.lprev_out = st.lprev[1 - par];
    d.tlast_out = st.tlast[1 - par];
    d.cpos = st.cpos;
    d.cneg = st.cneg;
    d.cpos_u = st.cpos_u;
    d.cneg_u = st.cneg_u;
    d.log_eps = st.p.log_eps;
    d.input_is_log = st.p.input_is_log;
    d.refractory = st.p.refractory_us;
    d.W = st.W;
    d.npix = st.npix;
    d.n_tiles = st.n_tiles;
    d.item_base = item_base;
    d.seg_base = seg_base;
    d.n_segs = init ? 0 : b->T;
    d.init = init ? 1 : 0;
    d.vec = (st.npix % 4 == 0 && frame_stride % 4 == 0 && (reinterpret_cast<uintptr_t>(frames) & 15u) == 0) ? 1 : 0;
    d.frame_stride = frame_stride;
    d.pix_bits = st.pix_bits;
    d.D0 = b->dt;
    d.ta0 = 0;                   // taken from the device clock
    d.chunk_base = chunk_base;
    d.out_seg_index = 0;         // taken from the device clock
    return d;
}

// Uploads both parity sets of descriptors for the given frame pointers
// (frame_strides: floats between frames per stream, nullable = W * H).
int upload_descs(neurosim_evsim_batch* b, StreamDesc* dst, bool init, const float* const* frames,
                 const int64_t* frame_strides)
{
    std::vector<StreamDesc> h((size_t)2 * b->n);
    for (int par = 0; par < 2; ++par) {
        int item = 0, seg = 0;
        int64_t chunk = 0;
        for (int i = 0; i < b->n; ++i) {
            const int64_t fs = frame_strides ? frame_strides[i] : 0;
            h[(size_t)par * b->n + i] =
                make_desc(b, i, par, init, frames[i], fs ? fs : (int64_t)b->s[i].npix, item, seg, chunk);
            item += b->s[i].n_tiles;
            seg += init ? 0 : b->T;
            chunk += (int64_t)b->T * b->s[i].n_tiles;
        }
    }
    BCUDA(cudaMemcpyAsync(dst, h.data(), h.size() * sizeof(StreamDesc), cudaMemcpyHostToDevice, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    return NEUROSIM_OK;
}

StepLaunch make_launch(const neurosim_evsim_batch* b, bool init, int slot)
{
    StepLaunch L;
    memset(&L, 0, sizeof L);
    L.streams_dev = init ? b->d_init : b->d_step + (size_t)slot * 2 * b->n;
    L.n_streams = b->n;
    L.n_items = b->n_items;
    L.n_segs = init ? 0 : (int32_t)b->n_segs;
    L.T = init ? 1 : b->T;
    L.dt = b->dt;
    L.key64 = b->key64;
    L.t_bits = b->t_bits;
    L.ppt = b->ppt;
    L.pf = b->pf;
    L.grid_emit = b->grid_emit;
    L.grid_sort = std::max(1, (int)std::min<int64_t>(b->n_segs, (int64_t)b->sms * 2));
    L.sort_smem = b->sort_smem;
    L.max_tiles = b->max_tiles;
    L.keys = b->keys;
    L.n_pages = b->n_pages;
    L.page_keys = kBatchPageKeys;
    L.temp = b->temp;
    L.chunks = b->chunks;
    L.seg_count = b->seg_count;
    L.seg_rel = b->seg_rel;
    L.seg_abs = b->seg_abs;
    L.seg_off_out = b->seg_off;
    L.out = b->out;
    L.out_cap = b->out_cap;
    L.ctl = b->ctl;
    L.stream = b->stream;
    L.wait_limit_ns = kBatchWaitLimitNs;
    L.clock = b->clock;
    L.max_pending = b->max_pending;
    L.tau_init = b->bp.t0_us;
    return L;
}

struct BatchGuard {
    int prev = -1;
    bool ok = true;
    explicit BatchGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~BatchGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int read_device_counters(neurosim_evsim_batch* b, Ctl* c, DevClock* k)
{
    BCUDA(cudaStreamSynchronize(b->stream));
    BCUDA(cudaMemcpy(c, b->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    BCUDA(cudaMemcpy(k, b->clock, sizeof(DevClock), cudaMemcpyDeviceToHost));
    return NEUROSIM_OK;
}

}  // namespace

extern "C" {

void neurosim_evsim_batch_default_params(neurosim_evsim_batch_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->n_streams = 1;
    p->frames_per_step = 16;
    p->dt_us = 1000;
}

int neurosim_evsim_batch_create(const neurosim_evsim_params* streams, const neurosim_evsim_batch_params* bp,
                                void* cuda_stream, neurosim_evsim_batch** out)
{
    if (!out) return fail(NEUROSIM_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!streams || !bp) return fail(NEUROSIM_E_INVALID, "streams and batch params must not be NULL");
    if (bp->n_streams < 1 || bp->n_streams > (1 << 20)) return fail(NEUROSIM_E_INVALID, "n_streams must be in [1, 2^20]");
    if (bp->frames_per_step < 1 || bp->frames_per_step > 4096)
        return fail(NEUROSIM_E_INVALID, "frames_per_step must be in [1, 4096]");
    if (bp->dt_us < 1 || bp->dt_us >= (1 << 24)) return fail(NEUROSIM_E_TIME, "dt_us must be in [1, 2^24)");
    if (bp->t0_us < 0 || bp->t0_us > 0xFFFFFFFEll) return fail(NEUROSIM_E_TIME, "t0_us must be in [0, 2^32 - 2]");
    if (bp->max_pending_steps < 0) return fail(NEUROSIM_E_INVALID, "max_pending_steps < 0");
    if (bp->pixels_per_thread != 0 && bp->pixels_per_thread != 8 && bp->pixels_per_thread != 16)
        return fail(NEUROSIM_E_INVALID, "pixels_per_thread must be 0, 8 or 16");
    if (bp->prefetch_frames != 0 && bp->prefetch_frames != 2 && bp->prefetch_frames != 3)
        return fail(NEUROSIM_E_INVALID, "prefetch_frames must be 0, 2 or 3");
    if (bp->frame_slots < 0 || bp->frame_slots > 16) return fail(NEUROSIM_E_INVALID, "frame_slots must be in [0, 16]");
    if (bp->ctas_per_sm < 0 || bp->ctas_per_sm > 64) return fail(NEUROSIM_E_INVALID, "ctas_per_sm must be in [0, 64]");
    for (int i = 0; i < 4; ++i)
        if (bp->reserved[i] != 0) return fail(NEUROSIM_E_INVALID, "reserved fields must be zero");
    for (int i = 0; i < bp->n_streams; ++i) {
        const int rc = validate_stream_params(&streams[i]);
        if (rc) return rc;
    }

    neurosim_evsim_batch* b = new (std::nothrow) neurosim_evsim_batch();
    if (!b) return fail(NEUROSIM_E_NOMEM, "host allocation failed");
    b->bp = *bp;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->n = bp->n_streams;
    b->T = bp->frames_per_step;
    b->dt = bp->dt_us;
    b->ppt = bp->pixels_per_thread ? bp->pixels_per_thread : 16;
    b->pf = bp->prefetch_frames ? bp->prefetch_frames : 2;
    b->slots = bp->frame_slots ? bp->frame_slots : 2;
    b->slot_set.assign(b->slots, false);
    const int pend_steps = bp->max_pending_steps ? bp->max_pending_steps : 4;
    auto bail = [&](int code) {
        release(b);
        delete b;
        return code;
    };
    if (cudaGetDevice(&b->device) != cudaSuccess) return bail(fail(NEUROSIM_E_CUDA, "no CUDA device"));
    if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
        return bail(fail(NEUROSIM_E_CUDA, "cannot query the SM count"));

    b->s.resize(b->n);
    int max_pix_bits = 1;
    uint64_t total_px = 0;
    for (int i = 0; i < b->n; ++i) {
        BatchStream& st = b->s[i];
        st.p = streams[i];
        st.p.c_pos_map = st.p.c_neg_map = nullptr;
        st.W = streams[i].width;
        st.H = streams[i].height;
        st.npix = st.W * st.H;
        st.pix_bits = bits_of((uint64_t)(st.npix - 1));
        st.n_tiles = (st.npix + 32 * b->ppt - 1) / (32 * b->ppt);
        if (st.n_tiles > kMaxTilesPerStream)
            return bail(fail(NEUROSIM_E_INVALID, "stream %d: too many pixels for pixels_per_thread %d", i, b->ppt));
        max_pix_bits = std::max(max_pix_bits, st.pix_bits);
        if ((int64_t)b->n_items + st.n_tiles > (int64_t)INT32_MAX / 2)
            return bail(fail(NEUROSIM_E_INVALID, "too many pixels in the batch"));
        b->n_items += st.n_tiles;
        b->max_tiles = std::max(b->max_tiles, st.n_tiles);
        total_px += (uint64_t)st.npix;
        const size_t n = (size_t)st.npix;
        for (int k = 0; k < 2; ++k)
            if (dalloc(&st.ref[k], n) || dalloc(&st.lprev[k], n) || dalloc(&st.tlast[k], n))
                return bail(fail(NEUROSIM_E_NOMEM, "device allocation of stream %d's state failed", i));
        if (streams[i].c_pos_map) {
            for (size_t u = 0; u < n; ++u)
                if (!(std::isfinite(streams[i].c_pos_map[u]) && streams[i].c_pos_map[u] >= 1e-3f &&
                      std::isfinite(streams[i].c_neg_map[u]) && streams[i].c_neg_map[u] >= 1e-3f))
                    return bail(fail(NEUROSIM_E_INVALID, "stream %d: threshold maps must be finite and >= 1e-3", i));
            if (dalloc(&st.cpos, n) || dalloc(&st.cneg, n))
                return bail(fail(NEUROSIM_E_NOMEM, "device allocation of stream %d's thresholds failed", i));
            if (cudaMemcpy(st.cpos, streams[i].c_pos_map, n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(st.cneg, streams[i].c_neg_map, n * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(NEUROSIM_E_CUDA, "threshold map upload failed"));
        } else if (streams[i].sigma_c > 0.0f) {
            if (dalloc(&st.cpos, n) || dalloc(&st.cneg, n))
                return bail(fail(NEUROSIM_E_NOMEM, "device allocation of stream %d's thresholds failed", i));
            if (launch_threshold_maps(st.cpos, st.cneg, st.npix, streams[i].c_pos, streams[i].c_neg,
                                      streams[i].sigma_c, streams[i].c_min, streams[i].seed, b->stream) != cudaSuccess)
                return bail(fail(NEUROSIM_E_CUDA, "threshold kernel launch failed"));
        }
        st.cpos_u = std::max(streams[i].c_min, streams[i].c_pos);
        st.cneg_u = std::max(streams[i].c_min, streams[i].c_neg);
    }
    b->t_bits = bits_of((uint64_t)b->dt);
    b->key64 = (b->t_bits + max_pix_bits + 1 > 32) ? 1 : 0;
    b->n_segs = (int64_t)b->n * b->T;
    if (b->n_segs > INT32_MAX / 2) return bail(fail(NEUROSIM_E_INVALID, "n_streams * frames_per_step too large"));
    b->max_pending = b->n_segs * pend_steps;

    int bps = 0;
    if (emit_occupancy(b->ppt, b->pf, 0, &bps) != cudaSuccess || bps < 1)
        return bail(fail(NEUROSIM_E_CUDA, "emission kernel does not fit (ppt %d, prefetch %d)", b->ppt, b->pf));
    int bps64 = 0;
    if (emit_occupancy(b->ppt, b->pf, 1, &bps64) != cudaSuccess || bps64 < 1)
        return bail(fail(NEUROSIM_E_CUDA, "emission kernel does not fit (ppt %d, prefetch %d)", b->ppt, b->pf));
    const int wpc = emit_warps_per_cta(b->ppt);
    int per_sm = b->key64 ? bps64 : bps;
    if (bp->ctas_per_sm > 0) per_sm = std::min(per_sm, bp->ctas_per_sm);
    b->grid_emit = std::min((b->n_items + wpc - 1) / wpc, b->sms * per_sm);
    if (sort_configure(&b->sort_smem) != cudaSuccess)
        return bail(fail(NEUROSIM_E_CUDA, "cannot configure the sort kernel"));

    uint64_t cap = bp->event_capacity;
    if (cap == 0) cap = std::max<uint64_t>(1u << 20, total_px * (uint64_t)b->T * pend_steps / 16);
    b->out_cap = cap;
    // keys of one step: up to the record capacity, plus one partial page per warp
    const uint64_t warps = (uint64_t)b->grid_emit * wpc;
    const uint64_t key_count = cap + warps * kBatchPageKeys;
    if (key_count / kBatchPageKeys > 0xFFFFFFFFull / kBatchPageKeys - 1)
        return bail(fail(NEUROSIM_E_INVALID, "event_capacity too large"));
    b->key_bytes = (size_t)key_count * (b->key64 ? 8 : 4);
    b->n_pages = (uint32_t)(key_count / kBatchPageKeys);
    int64_t chunk_entries = 0;
    for (const auto& st : b->s) chunk_entries += (int64_t)b->T * st.n_tiles;
    if (dalloc(&b->d_step, (size_t)b->slots * 2 * b->n) || dalloc(&b->d_init, (size_t)2 * b->n) ||
        cudaMalloc(&b->keys, b->key_bytes) != cudaSuccess || cudaMalloc(&b->temp, b->key_bytes) != cudaSuccess ||
        dalloc(&b->chunks, (size_t)chunk_entries) || dalloc(&b->seg_count, (size_t)b->n_segs) ||
        dalloc(&b->seg_rel, (size_t)b->n_segs) || dalloc(&b->seg_abs, (size_t)b->n_segs) ||
        dalloc(&b->seg_off, (size_t)b->max_pending) || dalloc(&b->out, (size_t)cap) ||
        dalloc(&b->ctl, 1) || dalloc(&b->clock, 1))
        return bail(fail(NEUROSIM_E_NOMEM, "device allocation of the batch buffers failed"));
    if (cudaMemsetAsync(b->ctl, 0, sizeof(Ctl), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->clock, 0, sizeof(DevClock), b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bail(fail(NEUROSIM_E_CUDA, "initialising the batch counters failed"));
    *out = b;
    return NEUROSIM_OK;
}

int neurosim_evsim_batch_set_frames_strided(neurosim_evsim_batch* b, int32_t slot, const float* const* frames_dev,
                                            const int64_t* frame_strides)
{
    if (!b || !frames_dev) return fail(NEUROSIM_E_INVALID, "batch and frames_dev must not be NULL");
    if (frame_strides)
        for (int i = 0; i < b->n; ++i)
            if (frame_strides[i] != 0 && frame_strides[i] < (int64_t)b->s[i].npix)
                return fail(NEUROSIM_E_INVALID, "frame_strides[%d] is smaller than W * H", i);
    if (slot < 0 || slot >= b->slots) return fail(NEUROSIM_E_INVALID, "slot %d not in [0, %d)", slot, b->slots);
    for (int i = 0; i < b->n; ++i)
        if (!frames_dev[i]) return fail(NEUROSIM_E_INVALID, "frames_dev[%d] is NULL", i);
    BatchGuard g(b->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the batch's device");
    const int rc = upload_descs(b, b->d_step + (size_t)slot * 2 * b->n, false, frames_dev, frame_strides);
    if (rc) return rc;
    b->slot_set[slot] = true;
    return NEUROSIM_OK;
}

int neurosim_evsim_batch_set_frames(neurosim_evsim_batch* b, int32_t slot, const float* const* frames_dev)
{
    return neurosim_evsim_batch_set_frames_strided(b, slot, frames_dev, nullptr);
}

int neurosim_evsim_batch_init(neurosim_evsim_batch* b, const float* const* first_frames_dev)
{
    if (!b || !first_frames_dev) return fail(NEUROSIM_E_INVALID, "batch and first_frames_dev must not be NULL");
    if (b->initialised) return fail(NEUROSIM_E_STATE, "the batch is initialised already");
    for (int i = 0; i < b->n; ++i)
        if (!first_frames_dev[i]) return fail(NEUROSIM_E_INVALID, "first_frames_dev[%d] is NULL", i);
    BatchGuard g(b->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the batch's device");
    int rc = upload_descs(b, b->d_init, true, first_frames_dev, nullptr);
    if (rc) return rc;
    const StepLaunch L = make_launch(b, true, 0);
    BCUDA(launch_step(L, &b->launches));
    b->initialised = true;
    return NEUROSIM_OK;
}

int neurosim_evsim_batch_step(neurosim_evsim_batch* b, int32_t slot)
{
    if (!b) return fail(NEUROSIM_E_INVALID, "batch is NULL");
    if (slot < 0 || slot >= b->slots) return fail(NEUROSIM_E_INVALID, "slot %d not in [0, %d)", slot, b->slots);
    if (!b->initialised || !b->slot_set[slot])
        return fail(NEUROSIM_E_STATE, "call neurosim_evsim_batch_init and register slot %d before stepping", slot);
    BatchGuard g(b->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the batch's device");
    const StepLaunch L = make_launch(b, false, slot);
    BCUDA(launch_step(L, &b->launches));
    return NEUROSIM_OK;
}

int neurosim_evsim_batch_pending(neurosim_evsim_batch* b, uint64_t* n_events, int64_t* n_segments)
{
    if (!b) return fail(NEUROSIM_E_INVALID, "batch is NULL");
    BatchGuard g(b->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the batch's device");
    Ctl c;
    DevClock k;
    const int rc = read_device_counters(b, &c, &k);
    if (rc) return rc;
    if (n_events) *n_events = k.committed_total;
    if (n_segments) *n_segments = k.pending_segs;
    return NEUROSIM_OK;
}

int neurosim_evsim_batch_drain(neurosim_evsim_batch* b, void* out, uint64_t capacity, int32_t out_is_device,
                               uint64_t* n_out, int64_t* seg_offsets, int64_t seg_capacity, int64_t* n_segments)
{
    if (!b) return fail(NEUROSIM_E_INVALID, "batch is NULL");
    if (n_out) *n_out = 0;
    if (n_segments) *n_segments = 0;
    BatchGuard g(b->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the batch's device");
    Ctl c;
    DevClock k;
    int rc = read_device_counters(b, &c, &k);
    if (rc) return rc;
    const uint64_t n = k.committed_total;
    const int64_t ns = k.pending_segs;
    if (n_segments) *n_segments = ns;
    if (n > capacity || (n > 0 && !out)) {
        if (n_out) *n_out = n;
        return fail(NEUROSIM_E_OVERFLOW, "capacity %llu < %llu pending events", (unsigned long long)capacity,
                    (unsigned long long)n);
    }
    if (seg_offsets && seg_capacity < ns + 1)
        return fail(NEUROSIM_E_OVERFLOW, "seg_capacity %lld < %lld", (long long)seg_capacity, (long long)(ns + 1));
    if (n > 0)
        BCUDA(cudaMemcpyAsync(out, b->out, n * sizeof(uint64_t),
                              out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    if (seg_offsets) {
        if (ns > 0)
            BCUDA(cudaMemcpyAsync(seg_offsets, b->seg_off, (size_t)ns * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                  b->stream));
        BCUDA(cudaStreamSynchronize(b->stream));
        seg_offsets[ns] = (int64_t)n;
    }
    // clear the pending records and any stop condition
    const uint32_t sticky = k.sticky;
    k.committed_total = 0;
    k.pending_segs = 0;
    k.sticky = 0u;
    c.run_total = 0;
    c.err = 0u;
    c.page_ctr = 0u;
    BCUDA(cudaMemcpyAsync(b->clock, &k, sizeof(DevClock), cudaMemcpyHostToDevice, b->stream));
    BCUDA(cudaMemcpyAsync(b->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    if (n_out) *n_out = n;
    if (sticky & kErrTimeout) return fail(NEUROSIM_E_TIMEOUT, "a bounded device wait timed out; steps were dropped");
    if (sticky & kErrTime) return fail(NEUROSIM_E_TIME, "the device clock left the 32-bit timestamp range; steps were dropped");
    if (sticky & (kErrOutOverflow | kErrPageOverflow | kErrPendingOverflow))
        return fail(NEUROSIM_E_OVERFLOW,
                    "a step overflowed the batch's %s (record demand %llu of %llu, key pages %u of %u); it and "
                    "the later steps were dropped",
                    (sticky & kErrPendingOverflow) ? "pending intervals (drain more often)"
                                                   : "event capacity (create a larger batch)",
                    (unsigned long long)c.out_demand_max, (unsigned long long)b->out_cap, c.page_demand_max,
                    b->n_pages);
    return NEUROSIM_OK;
}

int neurosim_evsim_batch_get_state(neurosim_evsim_batch* b, int32_t stream, float* ref, float* lprev,
                                   uint32_t* tlast, int64_t* tau_us)
{
    if (!b) return fail(NEUROSIM_E_INVALID, "batch is NULL");
    if (stream < 0 || stream >= b->n) return fail(NEUROSIM_E_INVALID, "stream index out of range");
    BatchGuard g(b->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the batch's device");
    Ctl c;
    DevClock k;
    const int rc = read_device_counters(b, &c, &k);
    if (rc) return rc;
    const BatchStream& st = b->s[stream];
    const int par = (int)(k.parity & 1u);
    const size_t n = (size_t)st.npix;
    if (ref) BCUDA(cudaMemcpy(ref, st.ref[par], n * 4, cudaMemcpyDeviceToHost));
    if (lprev) BCUDA(cudaMemcpy(lprev, st.lprev[par], n * 4, cudaMemcpyDeviceToHost));
    if (tlast) BCUDA(cudaMemcpy(tlast, st.tlast[par], n * 4, cudaMemcpyDeviceToHost));
    if (tau_us) *tau_us = k.tau;
    return NEUROSIM_OK;
}

int neurosim_evsim_batch_get_thresholds(neurosim_evsim_batch* b, int32_t stream, float* c_pos, float* c_neg)
{
    if (!b || !c_pos || !c_neg) return fail(NEUROSIM_E_INVALID, "NULL argument");
    if (stream < 0 || stream >= b->n) return fail(NEUROSIM_E_INVALID, "stream index out of range");
    BatchGuard g(b->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the batch's device");
    BCUDA(cudaStreamSynchronize(b->stream));
    const BatchStream& st = b->s[stream];
    const size_t n = (size_t)st.npix;
    if (st.cpos) {
        BCUDA(cudaMemcpy(c_pos, st.cpos, n * 4, cudaMemcpyDeviceToHost));
        BCUDA(cudaMemcpy(c_neg, st.cneg, n * 4, cudaMemcpyDeviceToHost));
    } else {
        for (size_t u = 0; u < n; ++u) {
            c_pos[u] = st.cpos_u;
            c_neg[u] = st.cneg_u;
        }
    }
    return NEUROSIM_OK;
}

int neurosim_evsim_batch_counters(neurosim_evsim_batch* b, uint64_t* launches, uint64_t* steps)
{
    if (!b) return fail(NEUROSIM_E_INVALID, "batch is NULL");
    if (launches) *launches = b->launches;
    if (steps) {
        BatchGuard g(b->device);
        if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the batch's device");
        Ctl c;
        DevClock k;
        const int rc = read_device_counters(b, &c, &k);
        if (rc) return rc;
        *steps = k.steps;
    }
    return NEUROSIM_OK;
}

void neurosim_evsim_batch_destroy(neurosim_evsim_batch* b)
{
    if (!b) return;
    {
        BatchGuard g(b->device);
        cudaStreamSynchronize(b->stream);
        release(b);
    }
    delete b;
}

}  // extern "C"
