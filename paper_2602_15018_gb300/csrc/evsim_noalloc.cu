// One event-generation step that allocates nothing (declared in
// include/neurosim_evsim.h as neurosim_evsim_step_noalloc).
//
// Some callers cannot call cudaMalloc: real-time control loops that must
// never enter the device allocator (it can block on a device-wide
// synchronisation), and host programs that only borrow device buffers from
// another runtime or framework and have no allocator of their own to call.
// For them this entry point runs one step of the event model from buffers
// the caller owns (frames, thresholds, per-pixel state in and out, event
// records and interval offsets out) and keeps every intermediate — the paged
// event keys, the (interval, tile) chunk table, the per-interval counts and
// offsets, the control block — in one file-scope device array of fixed size.
//
// The array is shared by every call on a device and keeps the last call's
// contents; the control block is cleared at the start of each call.  Two
// calls whose work overlaps on the GPU (different streams, no ordering
// between them) race on the array.  The call synchronises the caller's
// stream before it returns (it reads the event count back to the host).  The
// first call on a device looks up the array's device address and configures
// the kernels; it should happen before any stream capture.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"

namespace {

// 32 MiB of scratch per device, held until the process exits.
constexpr size_t kScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
constexpr uint32_t kPageKeysNoalloc = 512;   // small pages: the key area is small
constexpr int kPpt = 16, kPf = 2;

struct DeviceSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;   // device address of g_noalloc_scratch
    int sms = 0, grid32 = 0, grid64 = 0, sort_smem = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return nsim::report_error(code, buf);
}

int bits_of(uint64_t v)
{
    int b = 1;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Per-device set-up, with that device current: the array's device address
// (the host-side symbol is only a stand-in) and the kernels' launch shapes.
int setup_device(int dev, DeviceSetup** out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(NEUROSIM_E_INVALID, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& d = g_setup[dev];
    if (!d.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(NEUROSIM_E_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return fail(NEUROSIM_E_CUDA, "cannot query the SM count: %s", cudaGetErrorString(e));
        int b32 = 0, b64 = 0;
        if ((e = nsim::emit_occupancy(kPpt, kPf, 0, &b32)) != cudaSuccess ||
            (e = nsim::emit_occupancy(kPpt, kPf, 1, &b64)) != cudaSuccess || b32 < 1 || b64 < 1)
            return fail(NEUROSIM_E_CUDA, "emission kernel does not fit: %s", cudaGetErrorString(e));
        if ((e = nsim::sort_configure(&d.sort_smem)) != cudaSuccess)
            return fail(NEUROSIM_E_CUDA, "cannot configure the sort kernel: %s", cudaGetErrorString(e));
        d.scratch = static_cast<unsigned char*>(p);
        d.grid32 = d.sms * b32;
        d.grid64 = d.sms * b64;
        d.ready = true;
    }
    *out = &d;
    return NEUROSIM_OK;
}

bool finite_min(float v, float lo) { return v == v && v >= lo && v < 3.0e38f; }

}  // namespace

extern "C" int neurosim_evsim_step_noalloc(
    const float* frames_dev, int32_t n_frames, int32_t width, int32_t height, int64_t t0_us,
    int32_t dt_us, const float* c_pos_dev, const float* c_neg_dev, float c_pos, float c_neg,
    uint32_t refractory_us, float log_eps, int32_t input_is_log, const float* ref_in,
    const float* lprev_in, const uint32_t* tlast_in, float* ref_out, float* lprev_out,
    uint32_t* tlast_out, int32_t has_prev, int64_t tau_prev, uint64_t* events_dev,
    uint64_t events_capacity, int64_t* seg_offsets_dev, uint64_t* n_events, void* cuda_stream)
{
    using namespace nsim;
    // ---- arguments --------------------------------------------------------
    if (!n_events) return fail(NEUROSIM_E_INVALID, "n_events is NULL");
    *n_events = 0;
    if (width < 1 || width > 65535 || height < 1 || height > 32767)
        return fail(NEUROSIM_E_INVALID, "width must be in [1, 65535] and height in [1, 32767]");
    const int64_t npix = (int64_t)width * height;
    if (n_frames < 1) return fail(NEUROSIM_E_INVALID, "n_frames must be >= 1");
    if (!frames_dev || !ref_out || !lprev_out || !tlast_out || !seg_offsets_dev)
        return fail(NEUROSIM_E_INVALID, "frames, state outputs and seg_offsets must not be NULL");
    if (has_prev != 0 && has_prev != 1) return fail(NEUROSIM_E_INVALID, "has_prev must be 0 or 1");
    if (has_prev && (!ref_in || !lprev_in || !tlast_in))
        return fail(NEUROSIM_E_INVALID, "state inputs are required when has_prev is 1");
    if (has_prev && (ref_in == ref_out || lprev_in == lprev_out || tlast_in == tlast_out))
        return fail(NEUROSIM_E_INVALID, "state outputs must not be the state inputs");
    if ((c_pos_dev == nullptr) != (c_neg_dev == nullptr))
        return fail(NEUROSIM_E_INVALID, "c_pos_dev and c_neg_dev must be given together");
    if (!c_pos_dev && (!finite_min(c_pos, 1e-3f) || !finite_min(c_neg, 1e-3f)))
        return fail(NEUROSIM_E_INVALID, "c_pos and c_neg must be finite and >= 1e-3");
    if (!(log_eps >= 1e-8f && log_eps <= 1.0f)) return fail(NEUROSIM_E_INVALID, "log_eps must be in [1e-8, 1]");
    if (input_is_log != 0 && input_is_log != 1) return fail(NEUROSIM_E_INVALID, "input_is_log must be 0 or 1");
    if (events_capacity > 0 && !events_dev) return fail(NEUROSIM_E_INVALID, "events_dev is NULL");
    {
        const uintptr_t a16 = reinterpret_cast<uintptr_t>(ref_out) | reinterpret_cast<uintptr_t>(lprev_out) |
                              reinterpret_cast<uintptr_t>(tlast_out) | reinterpret_cast<uintptr_t>(ref_in) |
                              reinterpret_cast<uintptr_t>(lprev_in) | reinterpret_cast<uintptr_t>(tlast_in) |
                              reinterpret_cast<uintptr_t>(c_pos_dev) | reinterpret_cast<uintptr_t>(c_neg_dev);
        const uintptr_t a8 = reinterpret_cast<uintptr_t>(events_dev) | reinterpret_cast<uintptr_t>(seg_offsets_dev);
        if ((a16 & 15u) || (a8 & 7u))
            return fail(NEUROSIM_E_INVALID, "state and threshold arrays must be 16-byte aligned, "
                                            "events and offsets 8-byte aligned");
    }
    if (dt_us < 1 || dt_us >= (1 << 24)) return fail(NEUROSIM_E_TIME, "dt_us must be in [1, 2^24)");
    if (t0_us < 0) return fail(NEUROSIM_E_TIME, "t0_us must be >= 0");
    if (t0_us + (int64_t)(n_frames - 1) * dt_us > 0xFFFFFFFEll)
        return fail(NEUROSIM_E_TIME, "last frame time exceeds 2^32 - 2 us");
    if (has_prev && (t0_us <= tau_prev || t0_us - tau_prev >= (1 << 24) || tau_prev < 0))
        return fail(NEUROSIM_E_TIME, "t0_us must follow tau_prev by 1 .. 2^24 - 1 us");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(NEUROSIM_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    DeviceSetup* d = nullptr;
    int rc = setup_device(dev, &d);
    if (rc) return rc;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    // ---- step geometry (as neurosim_evsim_step) -----------------------------
    const bool init = !has_prev;
    const int32_t D0 = init ? dt_us : (int32_t)(t0_us - tau_prev);
    const int64_t ta0 = init ? t0_us : tau_prev;
    const int32_t n_segs = init ? n_frames - 1 : n_frames;
    const int pix_bits = bits_of((uint64_t)(npix - 1));
    const int t_bits = bits_of((uint64_t)std::max(D0, dt_us));
    const int key64 = (t_bits + pix_bits + 1 > 32) ? 1 : 0;
    const int n_tiles = (int)((npix + 32 * kPpt - 1) / (32 * kPpt));
    if (n_tiles > kMaxTilesPerStream)
        return fail(NEUROSIM_E_INVALID, "width*height must be <= %d", kMaxTilesPerStream * 32 * kPpt);

    // ---- carve the fixed scratch ----------------------------------------------
    size_t off = 0;
    Ctl* ctl = reinterpret_cast<Ctl*>(d->scratch + off);
    off = align_up(off + sizeof(Ctl), 256);
    uint32_t* seg_count = reinterpret_cast<uint32_t*>(d->scratch + off);
    off = align_up(off + sizeof(uint32_t) * (size_t)std::max(n_segs, 1), 256);
    int64_t* seg_rel = reinterpret_cast<int64_t*>(d->scratch + off);
    off = align_up(off + sizeof(int64_t) * (size_t)std::max(n_segs, 1), 256);
    int64_t* seg_abs = reinterpret_cast<int64_t*>(d->scratch + off);
    off = align_up(off + sizeof(int64_t) * (size_t)std::max(n_segs, 1), 256);
    uint2* chunks = reinterpret_cast<uint2*>(d->scratch + off);
    off = align_up(off + sizeof(uint2) * (size_t)std::max(n_segs, 1) * n_tiles, 256);
    if (off > kScratchBytes / 2)
        return fail(NEUROSIM_E_INVALID,
                    "n_frames x tiles too large for the %zu-byte scratch (%d intervals x %d tiles); "
                    "split the frames into smaller calls", kScratchBytes, n_segs, n_tiles);
    const size_t key_bytes = (kScratchBytes - off) / 2 / 256 * 256;
    void* keys = d->scratch + off;
    void* temp = d->scratch + off + key_bytes;

    StepLaunch L;
    memset(&L, 0, sizeof L);
    StreamDesc& s = L.s0;
    s.frames = frames_dev;
    s.ref_in = init ? ref_out : ref_in;
    s.lprev_in = init ? lprev_out : lprev_in;
    s.tlast_in = init ? tlast_out : tlast_in;
    s.ref_out = ref_out;
    s.lprev_out = lprev_out;
    s.tlast_out = tlast_out;
    s.cpos = c_pos_dev;
    s.cneg = c_neg_dev;
    s.cpos_u = c_pos;
    s.cneg_u = c_neg;
    s.log_eps = log_eps;
    s.input_is_log = input_is_log;
    s.refractory = refractory_us;
    s.W = width;
    s.npix = (int32_t)npix;
    s.n_tiles = n_tiles;
    s.n_segs = n_segs;
    s.init = init ? 1 : 0;
    s.vec = (npix % 4 == 0 && (reinterpret_cast<uintptr_t>(frames_dev) & 15u) == 0) ? 1 : 0;
    s.pix_bits = pix_bits;
    s.D0 = D0;
    s.ta0 = ta0;
    L.n_streams = 1;
    L.n_items = n_tiles;
    L.n_segs = n_segs;
    L.T = n_frames;
    L.dt = dt_us;
    L.key64 = key64;
    L.t_bits = t_bits;
    L.ppt = kPpt;
    L.pf = kPf;
    const int wpc = emit_warps_per_cta(kPpt);
    L.grid_emit = std::min((n_tiles + wpc - 1) / wpc, key64 ? d->grid64 : d->grid32);
    L.grid_sort = std::max(1, std::min(n_segs, d->sms * 2));
    L.sort_smem = d->sort_smem;
    L.max_tiles = n_tiles;
    L.keys = keys;
    L.page_keys = kPageKeysNoalloc;
    L.n_pages = (uint32_t)(key_bytes / ((size_t)kPageKeysNoalloc * (key64 ? 8 : 4)));
    L.temp = temp;
    L.chunks = chunks;
    L.seg_count = seg_count;
    L.seg_rel = seg_rel;
    L.seg_abs = seg_abs;
    L.seg_off_out = seg_offsets_dev;
    L.out = events_dev;
    L.out_cap = events_capacity;
    L.ctl = ctl;
    L.stream = stream;
    L.wait_limit_ns = 2000000000ull;

    // ---- run -----------------------------------------------------------------
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), stream)) != cudaSuccess)
        return fail(NEUROSIM_E_CUDA, "clearing the control block: %s", cudaGetErrorString(e));
    uint64_t launches = 0;
    if ((e = launch_step(L, &launches)) != cudaSuccess)
        return fail(NEUROSIM_E_CUDA, "step launch: %s", cudaGetErrorString(e));
    if ((e = launch_write_total(ctl, seg_offsets_dev + n_segs, stream)) != cudaSuccess)
        return fail(NEUROSIM_E_CUDA, "offset launch: %s", cudaGetErrorString(e));
    Ctl c;
    if ((e = cudaMemcpyAsync(&c, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
        return fail(NEUROSIM_E_CUDA, "step: %s", cudaGetErrorString(e));
    *n_events = c.run_total;
    if (c.err & kErrTimeout) return fail(NEUROSIM_E_TIMEOUT, "a bounded device wait timed out");
    if (c.err & kErrPageOverflow)
        return fail(NEUROSIM_E_OVERFLOW,
                    "the step's events exceed the fixed scratch (%zu bytes of keys); split the frames "
                    "into smaller calls", key_bytes);
    if (c.err & kErrOutOverflow)
        return fail(NEUROSIM_E_OVERFLOW, "events_capacity %llu < %llu events",
                    (unsigned long long)events_capacity, (unsigned long long)c.run_total);
    return NEUROSIM_OK;
}
