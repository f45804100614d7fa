// C-ABI host code of libneurosim_evsim.so (declarations and semantics in
// include/neurosim_evsim.h).  Owns the device buffers of a simulator,
// validates arguments, fills the launch descriptors and resolves event-buffer
// overflow by growing the buffers and replaying the pending steps from the
// state committed at the last drain (arXiv 2602.15018, Sec. 2: each frame
// yields a variable number of events, so capacity cannot be known upfront).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <memory>
#include <new>
#include <vector>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"

using namespace nsim;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(NEUROSIM_E_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                           \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// DLPack exchange format (v0.8 ABI, the layout every DLPack consumer reads):
// a 1-D 64-bit integer tensor on a CUDA device, owned by its producer.  The
// struct layouts follow the DLPack specification; the library fills them and
// the consumer calls `deleter` when it is done with the view.
struct DLDevice {
    int32_t device_type;   // 2: CUDA device memory
    int32_t device_id;
};
struct DLDataType {
    uint8_t code;          // 0: signed integer
    uint8_t bits;
    uint16_t lanes;
};
struct DLTensor {
    void* data;
    DLDevice device;
    int32_t ndim;
    DLDataType dtype;
    int64_t* shape;
    int64_t* strides;      // NULL: compact row-major
    uint64_t byte_offset;
};
struct DLManagedTensor {
    DLTensor dl_tensor;
    void* manager_ctx;
    void (*deleter)(DLManagedTensor* self);
};
struct DLPackBox {         // one allocation: the descriptor and its shape
    DLManagedTensor t;
    int64_t shape[1];
};

void dlpack_delete(DLManagedTensor* self) { delete reinterpret_cast<DLPackBox*>(self); }

// A view of n records at `data` (device `dev`) as int64 (the record bits,
// as drains to device memory hand them out); the records stay the
// library's (the deleter frees the descriptor only).
void* make_dlpack_i64(const uint64_t* data, int64_t n, int dev)
{
    DLPackBox* b = new (std::nothrow) DLPackBox;
    if (!b) return nullptr;
    b->shape[0] = n;
    b->t.dl_tensor.data = const_cast<uint64_t*>(data);
    b->t.dl_tensor.device = DLDevice{2, dev};
    b->t.dl_tensor.ndim = 1;
    b->t.dl_tensor.dtype = DLDataType{0, 64, 1};
    b->t.dl_tensor.shape = b->shape;
    b->t.dl_tensor.strides = nullptr;
    b->t.dl_tensor.byte_offset = 0;
    b->t.manager_ctx = b;
    b->t.deleter = dlpack_delete;
    return &b->t;
}

int bits_of(uint64_t v)  // bits needed to hold v (>= 1)
{
    int b = 1;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

constexpr uint32_t kPageKeys = 8192;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s bound on every device-side wait

struct StepRec {
    const float* frames;  // device pointer, or host pointer when host == true
    bool host;
    int32_t T;
    int64_t t0;
    int32_t dt;
    std::shared_ptr<neurosim_texture_scene> scene;   // rendered step: the scene (frames unused)
};

template <typename T>
cudaError_t dmalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

template <typename T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

}  // namespace

struct neurosim_evsim {
    neurosim_evsim_params p{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sms = 0;
    int W = 0, H = 0, npix = 0, pix_bits = 1;
    int ppt = 16, pf = 2, n_tiles = 0;
    int grid_emit32 = 0, grid_emit64 = 0, sort_smem = 0;
    int grid_tex32 = 0, grid_tex64 = 0;   // render-fused steps
    int Tmax = 1024;
    int64_t max_pending = 65536;

    // per-pixel state, double buffered: [cidx] committed at the last drain
    float* ref[2] = {nullptr, nullptr};
    float* lprev[2] = {nullptr, nullptr};
    uint32_t* tlast[2] = {nullptr, nullptr};
    int cidx = 0;
    int64_t tau_c = 0, tau_w = 0;
    bool has_c = false, has_w = false;

    float* cpos = nullptr;  // null: uniform thresholds cpos_u / cneg_u
    float* cneg = nullptr;
    float cpos_u = 0.2f, cneg_u = 0.2f;

    void* keys = nullptr;
    void* temp = nullptr;
    size_t key_bytes = 0;
    uint2* chunks = nullptr;
    uint32_t* seg_count = nullptr;
    int64_t* seg_rel = nullptr;
    int64_t* seg_abs = nullptr;
    int64_t* seg_off = nullptr;  // pending interval offsets [max_pending]
    uint64_t* out = nullptr;
    uint64_t out_cap = 0;
    Ctl* ctl = nullptr;

    float* staging = nullptr;  // device copy of host frames (step_host)
    void* scene_tab = nullptr; // per-frame scene table of a render-fused step (Tmax rows)

    std::vector<StepRec> pending;
    int64_t n_pending_segs = 0;
    bool broken = false;  // a device wait timed out: state is not trustworthy

    // counters and optional per-step timing
    neurosim_evsim_stats stats{};
    bool profiling = false;
    std::vector<cudaEvent_t> ev_free;             // recycled events
    std::vector<std::array<cudaEvent_t, 3>> ev_open;  // timed steps not yet summed
};

namespace {

cudaError_t take_event(neurosim_evsim* h, cudaEvent_t* ev)
{
    if (!h->ev_free.empty()) {
        *ev = h->ev_free.back();
        h->ev_free.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(ev);
}

// Sums the elapsed times of finished timed steps (stream already synchronised).
void collect_timings(neurosim_evsim* h)
{
    for (auto& e : h->ev_open) {
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, e[0], e[1]) == cudaSuccess) h->stats.emit_ms += a;
        if (cudaEventElapsedTime(&b, e[1], e[2]) == cudaSuccess) h->stats.sort_ms += b;
        h->stats.timed_steps += 1;
        for (int i = 0; i < 3; ++i) h->ev_free.push_back(e[i]);
    }
    h->ev_open.clear();
}

void release(neurosim_evsim* h)
{
    for (auto& e : h->ev_open)
        for (int i = 0; i < 3; ++i) h->ev_free.push_back(e[i]);
    h->ev_open.clear();
    for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
    h->ev_free.clear();
    for (int i = 0; i < 2; ++i) {
        dfree(h->ref[i]);
        dfree(h->lprev[i]);
        dfree(h->tlast[i]);
    }
    dfree(h->cpos);
    dfree(h->cneg);
    if (h->keys) cudaFree(h->keys);
    if (h->temp) cudaFree(h->temp);
    h->keys = h->temp = nullptr;
    dfree(h->chunks);
    dfree(h->seg_count);
    dfree(h->seg_rel);
    dfree(h->seg_abs);
    dfree(h->seg_off);
    dfree(h->out);
    dfree(h->ctl);
    dfree(h->staging);
    if (h->scene_tab) cudaFree(h->scene_tab);
    h->scene_tab = nullptr;
}

int alloc_event_buffers(neurosim_evsim* h, uint64_t out_cap, size_t key_bytes)
{
    if (h->out) cudaFree(h->out);
    if (h->keys) cudaFree(h->keys);
    if (h->temp) cudaFree(h->temp);
    h->out = nullptr;
    h->keys = h->temp = nullptr;
    key_bytes = (key_bytes + 65535) & ~(size_t)65535;
    CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&h->out), out_cap * sizeof(uint64_t)));
    CUDA_TRY(cudaMalloc(&h->keys, key_bytes));
    CUDA_TRY(cudaMalloc(&h->temp, key_bytes));
    h->out_cap = out_cap;
    h->key_bytes = key_bytes;
    return NEUROSIM_OK;
}

bool finite_pos(float v, float lo) { return std::isfinite(v) && v >= lo; }

int validate(const neurosim_evsim_params* p)
{
    if (!p) return fail(NEUROSIM_E_INVALID, "params is NULL");
    if (p->width < 1 || p->width > 65535 || p->height < 1 || p->height > 32767)
        return fail(NEUROSIM_E_INVALID, "width must be in [1, 65535] and height in [1, 32767]");
    if ((int64_t)p->width * p->height > (int64_t)kMaxTilesPerStream * 32 * 16)
        return fail(NEUROSIM_E_INVALID, "width*height must be <= %d", kMaxTilesPerStream * 32 * 16);
    const bool maps = p->c_pos_map != nullptr || p->c_neg_map != nullptr;
    if (maps && (p->c_pos_map == nullptr || p->c_neg_map == nullptr))
        return fail(NEUROSIM_E_INVALID, "c_pos_map and c_neg_map must be given together");
    if (!maps && (!finite_pos(p->c_pos, 1e-3f) || !finite_pos(p->c_neg, 1e-3f)))
        return fail(NEUROSIM_E_INVALID, "c_pos and c_neg must be finite and >= 1e-3");
    if (!finite_pos(p->c_min, 1e-3f)) return fail(NEUROSIM_E_INVALID, "c_min must be >= 1e-3");
    if (!(std::isfinite(p->sigma_c) && p->sigma_c >= 0.0f))
        return fail(NEUROSIM_E_INVALID, "sigma_c must be finite and >= 0");
    if (!(p->log_eps >= 1e-8f && p->log_eps <= 1.0f))
        return fail(NEUROSIM_E_INVALID, "log_eps must be in [1e-8, 1]");
    if (p->input_is_log != 0 && p->input_is_log != 1)
        return fail(NEUROSIM_E_INVALID, "input_is_log must be 0 or 1");
    if (p->max_frames_per_step < 0 || p->max_frames_per_step > (1 << 20))
        return fail(NEUROSIM_E_INVALID, "max_frames_per_step must be in [0, 2^20]");
    if (p->max_pending_intervals < 0) return fail(NEUROSIM_E_INVALID, "max_pending_intervals < 0");
    if (p->pixels_per_thread != 0 && p->pixels_per_thread != 8 && p->pixels_per_thread != 16)
        return fail(NEUROSIM_E_INVALID, "pixels_per_thread must be 0, 8 or 16");
    if (p->prefetch_frames != 0 && p->prefetch_frames != 2 && p->prefetch_frames != 3)
        return fail(NEUROSIM_E_INVALID, "prefetch_frames must be 0, 2 or 3");
    if (p->ctas_per_sm < 0 || p->ctas_per_sm > 64) return fail(NEUROSIM_E_INVALID, "ctas_per_sm must be in [0, 64]");
    for (int i = 0; i < 5; ++i)
        if (p->reserved[i] != 0) return fail(NEUROSIM_E_INVALID, "reserved fields must be zero");
    return NEUROSIM_OK;
}

int check_handle(neurosim_evsim* h)
{
    if (!h) return fail(NEUROSIM_E_INVALID, "handle is NULL");
    if (h->broken)
        return fail(NEUROSIM_E_TIMEOUT, "a device wait timed out earlier; destroy this handle");
    return NEUROSIM_OK;
}

// Fills the launch descriptor of one step and enqueues it.
int enqueue_step(neurosim_evsim* h, const float* frames_dev, int32_t T, int64_t t0, int32_t dt,
                 const neurosim_texture_scene* scene = nullptr)
{
    const bool init = !h->has_w;
    const int32_t D0 = init ? dt : (int32_t)(t0 - h->tau_w);
    const int64_t ta0 = init ? t0 : h->tau_w;
    const int32_t n_segs = init ? T - 1 : T;
    const int t_bits = bits_of((uint64_t)std::max(D0, dt));
    const int key64 = (t_bits + h->pix_bits + 1 > 32) ? 1 : 0;
    const int in = h->pending.empty() ? h->cidx : 1 - h->cidx;
    const int wk = 1 - h->cidx;

    StepLaunch L;
    memset(&L, 0, sizeof L);
    StreamDesc& s = L.s0;
    s.frames = frames_dev;
    s.ref_in = h->ref[in];
    s.lprev_in = h->lprev[in];
    s.tlast_in = h->tlast[in];
    s.ref_out = h->ref[wk];
    s.lprev_out = h->lprev[wk];
    s.tlast_out = h->tlast[wk];
    s.cpos = h->cpos;
    s.cneg = h->cneg;
    s.cpos_u = h->cpos_u;
    s.cneg_u = h->cneg_u;
    s.log_eps = h->p.log_eps;
    s.input_is_log = h->p.input_is_log;
    s.refractory = h->p.refractory_us;
    s.W = h->W;
    s.npix = h->npix;
    s.n_tiles = h->n_tiles;
    s.item_base = 0;
    s.seg_base = 0;
    s.n_segs = n_segs;
    s.init = init ? 1 : 0;
    s.vec = (h->npix % 4 == 0 && (reinterpret_cast<uintptr_t>(frames_dev) & 15u) == 0) ? 1 : 0;
    s.pix_bits = h->pix_bits;
    s.D0 = D0;
    s.ta0 = ta0;
    s.chunk_base = 0;
    s.out_seg_index = h->n_pending_segs;
    if (scene) {
        // render-fused: the per-frame camera and rectangles, then the frames
        // come from the renderer inside the emission kernel
        if (!h->scene_tab) CUDA_TRY(cudaMalloc(&h->scene_tab, (size_t)h->Tmax * scene_frame_bytes()));
        CUDA_TRY(launch_scene_frames(*scene, t0, dt, T, h->scene_tab, h->stream));
        h->stats.kernel_launches += 1;
        s.frames = nullptr;
        s.vec = 0;
        s.scene_tab = h->scene_tab;
        s.scene = make_scene_const(*scene);
    }

    L.streams_dev = nullptr;
    L.n_streams = 1;
    L.n_items = h->n_tiles;
    L.n_segs = n_segs;
    L.T = T;
    L.dt = dt;
    L.key64 = key64;
    L.t_bits = t_bits;
    L.ppt = h->ppt;
    L.pf = h->pf;
    L.grid_emit = scene ? (key64 ? h->grid_tex64 : h->grid_tex32) : (key64 ? h->grid_emit64 : h->grid_emit32);
    L.grid_sort = std::max(1, std::min(n_segs, h->sms * 2));
    L.sort_smem = h->sort_smem;
    L.max_tiles = h->n_tiles;
    L.keys = h->keys;
    L.page_keys = kPageKeys;
    // key offsets are 32-bit: keep n_pages * page_keys below 2^32
    L.n_pages = (uint32_t)std::min<size_t>(0xFFFFFFFFu / kPageKeys - 1,
                                           h->key_bytes / ((size_t)kPageKeys * (key64 ? 8 : 4)));
    L.temp = h->temp;
    L.chunks = h->chunks;
    L.seg_count = h->seg_count;
    L.seg_rel = h->seg_rel;
    L.seg_abs = h->seg_abs;
    L.seg_off_out = h->seg_off;
    L.out = h->out;
    L.out_cap = h->out_cap;
    L.ctl = h->ctl;
    L.stream = h->stream;
    L.wait_limit_ns = kWaitLimitNs;
    std::array<cudaEvent_t, 3> evs{nullptr, nullptr, nullptr};
    if (h->profiling) {
        for (int i = 0; i < 3; ++i) CUDA_TRY(take_event(h, &evs[i]));
        L.ev_begin = evs[0];
        L.ev_emitted = evs[1];
        L.ev_sorted = evs[2];
    }
    CUDA_TRY(launch_step(L, &h->stats.kernel_launches));
    if (h->profiling) h->ev_open.push_back(evs);
    h->stats.steps += 1;
    h->stats.px_frames += (uint64_t)T * (uint64_t)h->npix;

    h->tau_w = t0 + (int64_t)(T - 1) * dt;
    h->has_w = true;
    h->n_pending_segs += n_segs;
    return NEUROSIM_OK;
}

int check_times(neurosim_evsim* h, int32_t T, int64_t t0, int32_t dt)
{
    if (T < 0) return fail(NEUROSIM_E_INVALID, "n_frames < 0");
    if (T > h->Tmax) return fail(NEUROSIM_E_INVALID, "n_frames %d > max_frames_per_step %d", T, h->Tmax);
    if (dt < 1 || dt >= (1 << 24)) return fail(NEUROSIM_E_TIME, "dt_us must be in [1, 2^24)");
    if (t0 < 0) return fail(NEUROSIM_E_TIME, "t0_us must be >= 0");
    if (T == 0) return NEUROSIM_OK;
    if (t0 + (int64_t)(T - 1) * dt > 0xFFFFFFFEll)
        return fail(NEUROSIM_E_TIME, "last frame time exceeds 2^32 - 2 us");
    if (h->has_w) {
        if (t0 <= h->tau_w)
            return fail(NEUROSIM_E_TIME, "t0_us %lld is not after the previous frame time %lld",
                        (long long)t0, (long long)h->tau_w);
        if (t0 - h->tau_w >= (1 << 24))
            return fail(NEUROSIM_E_TIME, "gap to the previous frame must be < 2^24 us");
    }
    const int64_t segs = h->has_w ? T : T - 1;
    if (h->n_pending_segs + segs > h->max_pending)
        return fail(NEUROSIM_E_OVERFLOW, "more than %lld intervals pending: drain first",
                    (long long)h->max_pending);
    return NEUROSIM_OK;
}

int upload_host_frames(neurosim_evsim* h, const float* frames_host, int32_t T)
{
    if (!h->staging) CUDA_TRY(dmalloc(&h->staging, (size_t)h->Tmax * h->npix));
    CUDA_TRY(cudaMemcpyAsync(h->staging, frames_host, (size_t)T * h->npix * sizeof(float),
                             cudaMemcpyHostToDevice, h->stream));
    return NEUROSIM_OK;
}

// Device address from which the step reads host frames.  Page-locked host
// memory mapped into the device's address space is read in place by the
// emission kernel (each frame crosses the host link once, while the kernel
// runs); any other host memory is first copied to the staging buffer.
int host_frames_for_step(neurosim_evsim* h, const float* frames_host, int32_t T, const float** out)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, frames_host) == cudaSuccess && a.type == cudaMemoryTypeHost &&
        a.devicePointer != nullptr) {
        *out = static_cast<const float*>(a.devicePointer);
        return NEUROSIM_OK;
    }
    (void)cudaGetLastError();
    const int rc = upload_host_frames(h, frames_host, T);
    if (rc) return rc;
    *out = h->staging;
    return NEUROSIM_OK;
}

int read_ctl(neurosim_evsim* h, Ctl* c)
{
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    CUDA_TRY(cudaMemcpy(c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    return NEUROSIM_OK;
}

// Synchronises and, on overflow, grows the buffers and replays the pending
// steps from the committed state.  On success c holds the final counters.
int resolve(neurosim_evsim* h, Ctl* c)
{
    memset(c, 0, sizeof *c);
    if (h->pending.empty()) return NEUROSIM_OK;
    int rc = read_ctl(h, c);
    if (rc) return rc;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if (c->err & kErrTimeout) {
            h->broken = true;
            return fail(NEUROSIM_E_TIMEOUT, "a bounded device wait timed out during a step");
        }
        if (!(c->err & (kErrPageOverflow | kErrOutOverflow))) return NEUROSIM_OK;
        // grow: output to the demand seen, keys to the page demand (as 64-bit keys)
        const uint64_t need_out = std::max<uint64_t>(h->out_cap, c->out_demand_max + c->out_demand_max / 4 + 4096);
        const size_t need_keys = std::max<size_t>(
            h->key_bytes, (size_t)c->page_demand_max * kPageKeys * 8 * 5 / 4 + (size_t)kPageKeys * 8 * h->sms * 8);
        rc = alloc_event_buffers(h, need_out, need_keys);
        if (rc) return rc;
        CUDA_TRY(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->stream));
        h->n_pending_segs = 0;
        h->has_w = h->has_c;
        h->tau_w = h->tau_c;
        std::vector<StepRec> steps;
        steps.swap(h->pending);
        for (const StepRec& s : steps) {
            const float* fr = s.frames;
            if (s.host) {
                rc = host_frames_for_step(h, s.frames, s.T, &fr);
                if (rc) return rc;
            }
            rc = enqueue_step(h, fr, s.T, s.t0, s.dt, s.scene.get());
            if (rc) return rc;
            h->pending.push_back(s);
        }
        rc = read_ctl(h, c);
        if (rc) return rc;
    }
    return fail(NEUROSIM_E_OVERFLOW, "event buffers still overflow after regrowth");
}

}  // namespace

namespace nsim {
// Sets the calling thread's last-error message (used by the other C-ABI units).
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }
// Checks one sensor's parameters as neurosim_evsim_create does (batches).
int validate_stream_params(const neurosim_evsim_params* p) { return validate(p); }
}  // namespace nsim

extern "C" {

void neurosim_evsim_default_params(neurosim_evsim_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->c_pos = 0.2f;
    p->c_neg = 0.2f;
    p->sigma_c = 0.0f;
    p->c_min = 0.01f;
    p->refractory_us = 0;
    p->log_eps = 1e-3f;
    p->input_is_log = 0;
}

int neurosim_evsim_create(const neurosim_evsim_params* p, void* cuda_stream, neurosim_evsim** out)
{
    if (!out) return fail(NEUROSIM_E_INVALID, "out is NULL");
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    neurosim_evsim* h = new (std::nothrow) neurosim_evsim();
    if (!h) return fail(NEUROSIM_E_NOMEM, "host allocation failed");
    h->p = *p;
    h->p.c_pos_map = h->p.c_neg_map = nullptr;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    auto bail = [&](int code) {
        release(h);
        delete h;
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(fail(NEUROSIM_E_CUDA, "no CUDA device"));
    if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return bail(fail(NEUROSIM_E_CUDA, "cannot query the SM count"));
    h->W = p->width;
    h->H = p->height;
    h->npix = p->width * p->height;
    h->pix_bits = bits_of((uint64_t)(h->npix - 1));
    h->Tmax = p->max_frames_per_step ? p->max_frames_per_step : 1024;
    h->max_pending = p->max_pending_intervals ? p->max_pending_intervals : 65536;
    if (h->max_pending < h->Tmax) h->max_pending = h->Tmax;

    h->ppt = p->pixels_per_thread ? p->pixels_per_thread : 16;
    if ((h->npix + 32 * h->ppt - 1) / (32 * h->ppt) > kMaxTilesPerStream) h->ppt = 16;
    h->n_tiles = (h->npix + 32 * h->ppt - 1) / (32 * h->ppt);
    if (h->n_tiles > kMaxTilesPerStream)
        return bail(fail(NEUROSIM_E_INVALID, "too many pixels for pixels_per_thread %d", h->ppt));
    h->pf = p->prefetch_frames ? p->prefetch_frames : 2;
    int bps32 = 0, bps64 = 0;
    if (emit_occupancy(h->ppt, h->pf, 0, &bps32) != cudaSuccess ||
        emit_occupancy(h->ppt, h->pf, 1, &bps64) != cudaSuccess || bps32 < 1 || bps64 < 1)
        return bail(fail(NEUROSIM_E_CUDA, "emission kernel does not fit (ppt %d, prefetch %d)",
                         h->ppt, h->pf));
    const int wpc = emit_warps_per_cta(h->ppt);
    if (p->ctas_per_sm > 0) {          // the caller's (or the autotuner's) launch shape
        bps32 = std::min(bps32, p->ctas_per_sm);
        bps64 = std::min(bps64, p->ctas_per_sm);
    }
    h->grid_emit32 = std::min((h->n_tiles + wpc - 1) / wpc, h->sms * bps32);
    h->grid_emit64 = std::min((h->n_tiles + wpc - 1) / wpc, h->sms * bps64);
    int tps32 = 0, tps64 = 0;
    if (emit_occupancy(h->ppt, h->pf, 0, &tps32, 1) != cudaSuccess ||
        emit_occupancy(h->ppt, h->pf, 1, &tps64, 1) != cudaSuccess || tps32 < 1 || tps64 < 1)
        return bail(fail(NEUROSIM_E_CUDA, "render-fused emission kernel does not fit (ppt %d)", h->ppt));
    h->grid_tex32 = std::min((h->n_tiles + wpc - 1) / wpc, h->sms * tps32);
    h->grid_tex64 = std::min((h->n_tiles + wpc - 1) / wpc, h->sms * tps64);
    if (sort_configure(&h->sort_smem) != cudaSuccess)
        return bail(fail(NEUROSIM_E_CUDA, "cannot configure the sort kernel"));

    const size_t n = (size_t)h->npix;
    for (int i = 0; i < 2; ++i) {
        if (dmalloc(&h->ref[i], n) || dmalloc(&h->lprev[i], n) || dmalloc(&h->tlast[i], n))
            return bail(fail(NEUROSIM_E_NOMEM, "device allocation of the pixel state failed"));
    }
    if (dmalloc(&h->chunks, (size_t)h->Tmax * h->n_tiles) || dmalloc(&h->seg_count, (size_t)h->Tmax) ||
        dmalloc(&h->seg_rel, (size_t)h->Tmax) || dmalloc(&h->seg_abs, (size_t)h->Tmax) ||
        dmalloc(&h->seg_off, (size_t)h->max_pending) || dmalloc(&h->ctl, 1))
        return bail(fail(NEUROSIM_E_NOMEM, "device allocation of the step tables failed"));
    if (cudaMemset(h->ctl, 0, sizeof(Ctl)) != cudaSuccess)
        return bail(fail(NEUROSIM_E_CUDA, "cudaMemset failed"));

    uint64_t cap = p->event_capacity;
    if (cap == 0) cap = std::max<uint64_t>(1u << 20, (uint64_t)h->npix * h->Tmax / 16);
    rc = alloc_event_buffers(h, cap, (size_t)cap * 8 + (size_t)kPageKeys * 8 * h->sms * 8);
    if (rc) return bail(rc);

    // thresholds
    if (p->c_pos_map) {
        for (size_t i = 0; i < n; ++i)
            if (!finite_pos(p->c_pos_map[i], 1e-3f) || !finite_pos(p->c_neg_map[i], 1e-3f))
                return bail(fail(NEUROSIM_E_INVALID, "threshold maps must be finite and >= 1e-3"));
        if (dmalloc(&h->cpos, n) || dmalloc(&h->cneg, n))
            return bail(fail(NEUROSIM_E_NOMEM, "device allocation of the threshold maps failed"));
        if (cudaMemcpy(h->cpos, p->c_pos_map, n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->cneg, p->c_neg_map, n * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(NEUROSIM_E_CUDA, "threshold map upload failed"));
    } else if (p->sigma_c > 0.0f) {
        if (dmalloc(&h->cpos, n) || dmalloc(&h->cneg, n))
            return bail(fail(NEUROSIM_E_NOMEM, "device allocation of the threshold maps failed"));
        if (launch_threshold_maps(h->cpos, h->cneg, h->npix, p->c_pos, p->c_neg, p->sigma_c, p->c_min,
                                  p->seed, h->stream) != cudaSuccess)
            return bail(fail(NEUROSIM_E_CUDA, "threshold kernel launch failed"));
    }
    h->cpos_u = std::max(p->c_min, p->c_pos);
    h->cneg_u = std::max(p->c_min, p->c_neg);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
        return bail(fail(NEUROSIM_E_CUDA, "stream synchronisation failed at create"));
    *out = h;
    return NEUROSIM_OK;
}

int neurosim_evsim_step(neurosim_evsim* h, const float* frames_dev, int32_t n_frames, int64_t t0_us,
                        int32_t dt_us)
{
    int rc = check_handle(h);
    if (rc) return rc;
    rc = check_times(h, n_frames, t0_us, dt_us);
    if (rc || n_frames == 0) return rc;
    if (!frames_dev) return fail(NEUROSIM_E_INVALID, "frames_dev is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the handle's device");
    rc = enqueue_step(h, frames_dev, n_frames, t0_us, dt_us);
    if (rc) return rc;
    h->pending.push_back(StepRec{frames_dev, false, n_frames, t0_us, dt_us, nullptr});
    return NEUROSIM_OK;
}

int neurosim_evsim_step_host(neurosim_evsim* h, const float* frames_host, int32_t n_frames,
                             int64_t t0_us, int32_t dt_us)
{
    int rc = check_handle(h);
    if (rc) return rc;
    rc = check_times(h, n_frames, t0_us, dt_us);
    if (rc || n_frames == 0) return rc;
    if (!frames_host) return fail(NEUROSIM_E_INVALID, "frames_host is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the handle's device");
    const float* fr = nullptr;
    rc = host_frames_for_step(h, frames_host, n_frames, &fr);
    if (rc) return rc;
    rc = enqueue_step(h, fr, n_frames, t0_us, dt_us);
    if (rc) return rc;
    h->pending.push_back(StepRec{frames_host, true, n_frames, t0_us, dt_us, nullptr});
    return NEUROSIM_OK;
}

int neurosim_evsim_step_texture(neurosim_evsim* h, const neurosim_texture_scene* scene, int32_t n_frames,
                                int64_t t0_us, int32_t dt_us)
{
    int rc = check_handle(h);
    if (rc) return rc;
    rc = check_scene(scene);
    if (rc) return rc;
    if (scene->width != h->W || scene->height != h->H)
        return fail(NEUROSIM_E_INVALID, "scene is %dx%d, the sensor %dx%d", scene->width, scene->height, h->W, h->H);
    rc = check_times(h, n_frames, t0_us, dt_us);
    if (rc || n_frames == 0) return rc;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(NEUROSIM_E_CUDA, "cannot select the handle's device");
    auto copy = std::make_shared<neurosim_texture_scene>(*scene);
    rc = enqueue_step(h, nullptr, n_frames, t0_us, dt_us, copy.get());
    if (rc) return rc;
    h->pending.push_back(StepRec{nullptr, false, n_frames, t0_us, dt_us, copy});
    return NEUROSIM_OK;
}

int neurosim_evsim_pending(neurosim_evsim* h, uint64_t* n_events, int64_t* n_intervals)
{
    int rc = check_handle(h);
    if (rc) return rc;
    DeviceGuard g(h->device);
    Ctl c;
    rc = resolve(h, &c);
    if (rc) return rc;
    if (n_events) *n_events = c.run_total;
    if (n_intervals) *n_intervals = h->n_pending_segs;
    return NEUROSIM_OK;
}

int neurosim_evsim_drain_events(neurosim_evsim* h, uint64_t* out, uint64_t out_capacity,
                                int32_t out_is_device, uint64_t* n_out, int64_t* seg_offsets,
                                int64_t seg_capacity, int64_t* n_segs)
{
    int rc = check_handle(h);
    if (rc) return rc;
    DeviceGuard g(h->device);
    Ctl c;
    rc = resolve(h, &c);
    if (rc) return rc;
    const uint64_t n = c.run_total;
    if (n_out) *n_out = n;
    if (n_segs) *n_segs = h->n_pending_segs;
    if (n > out_capacity) return fail(NEUROSIM_E_OVERFLOW, "out_capacity %llu < %llu pending events",
                                      (unsigned long long)out_capacity, (unsigned long long)n);
    if (seg_offsets && seg_capacity < h->n_pending_segs + 1)
        return fail(NEUROSIM_E_OVERFLOW, "seg_capacity %lld < %lld", (long long)seg_capacity,
                    (long long)(h->n_pending_segs + 1));
    if (n > 0 && !out) return fail(NEUROSIM_E_INVALID, "out is NULL");
    if (n > 0)
        CUDA_TRY(cudaMemcpyAsync(out, h->out, n * sizeof(uint64_t),
                                 out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 h->stream));
    if (seg_offsets) {
        if (h->n_pending_segs > 0)
            CUDA_TRY(cudaMemcpyAsync(seg_offsets, h->seg_off, (size_t)h->n_pending_segs * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, h->stream));
    }
    CUDA_TRY(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->stats.events_drained += n;
    if (seg_offsets) seg_offsets[h->n_pending_segs] = (int64_t)n;
    if (!h->pending.empty()) {
        h->cidx = 1 - h->cidx;
        h->tau_c = h->tau_w;
        h->has_c = h->has_w;
    }
    h->pending.clear();
    h->n_pending_segs = 0;
    return NEUROSIM_OK;
}

int neurosim_evsim_peek_events(neurosim_evsim* h, const uint64_t** events_dev, uint64_t* n_out,
                               int64_t* seg_offsets, int64_t seg_capacity, int64_t* n_segs)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!events_dev) return fail(NEUROSIM_E_INVALID, "events_dev is NULL");
    DeviceGuard g(h->device);
    Ctl c;
    rc = resolve(h, &c);
    if (rc) return rc;
    if (seg_offsets && seg_capacity < h->n_pending_segs + 1)
        return fail(NEUROSIM_E_OVERFLOW, "seg_capacity %lld < %lld", (long long)seg_capacity,
                    (long long)(h->n_pending_segs + 1));
    if (seg_offsets) {
        if (h->n_pending_segs > 0)
            CUDA_TRY(cudaMemcpyAsync(seg_offsets, h->seg_off, (size_t)h->n_pending_segs * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        seg_offsets[h->n_pending_segs] = (int64_t)c.run_total;
    }
    *events_dev = h->out;
    if (n_out) *n_out = c.run_total;
    if (n_segs) *n_segs = h->n_pending_segs;
    return NEUROSIM_OK;
}

int neurosim_evsim_release_events(neurosim_evsim* h)
{
    int rc = check_handle(h);
    if (rc) return rc;
    DeviceGuard g(h->device);
    Ctl c;
    rc = resolve(h, &c);
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->stats.events_drained += c.run_total;
    if (!h->pending.empty()) {
        h->cidx = 1 - h->cidx;
        h->tau_c = h->tau_w;
        h->has_c = h->has_w;
    }
    h->pending.clear();
    h->n_pending_segs = 0;
    return NEUROSIM_OK;
}

int neurosim_evsim_events_dlpack(neurosim_evsim* h, void** managed_tensor)
{
    if (!managed_tensor) return fail(NEUROSIM_E_INVALID, "managed_tensor is NULL");
    const uint64_t* ev = nullptr;
    uint64_t n = 0;
    int rc = neurosim_evsim_peek_events(h, &ev, &n, nullptr, 0, nullptr);
    if (rc) return rc;
    *managed_tensor = make_dlpack_i64(ev, (int64_t)n, h->device);
    if (!*managed_tensor) return fail(NEUROSIM_E_NOMEM, "cannot allocate the DLPack descriptor");
    return NEUROSIM_OK;
}

int neurosim_evsim_get_state(neurosim_evsim* h, float* ref, float* lprev, uint32_t* tlast,
                             int64_t* tau_prev, int32_t* has_prev)
{
    int rc = check_handle(h);
    if (rc) return rc;
    DeviceGuard g(h->device);
    Ctl c;
    rc = resolve(h, &c);
    if (rc) return rc;
    const int idx = h->pending.empty() ? h->cidx : 1 - h->cidx;
    const size_t n = (size_t)h->npix;
    if (ref) CUDA_TRY(cudaMemcpy(ref, h->ref[idx], n * 4, cudaMemcpyDeviceToHost));
    if (lprev) CUDA_TRY(cudaMemcpy(lprev, h->lprev[idx], n * 4, cudaMemcpyDeviceToHost));
    if (tlast) CUDA_TRY(cudaMemcpy(tlast, h->tlast[idx], n * 4, cudaMemcpyDeviceToHost));
    if (tau_prev) *tau_prev = h->tau_w;
    if (has_prev) *has_prev = h->has_w ? 1 : 0;
    return NEUROSIM_OK;
}

int neurosim_evsim_set_state(neurosim_evsim* h, const float* ref, const float* lprev,
                             const uint32_t* tlast, int64_t tau_prev, int32_t has_prev)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->pending.empty() || h->n_pending_segs)
        return fail(NEUROSIM_E_STATE, "set_state needs no pending steps: drain first");
    if (has_prev != 0 && has_prev != 1) return fail(NEUROSIM_E_INVALID, "has_prev must be 0 or 1");
    if (has_prev && (!ref || !lprev || !tlast))
        return fail(NEUROSIM_E_INVALID, "ref, lprev and tlast are required when has_prev is 1");
    if (has_prev && (tau_prev < 0 || tau_prev > 0xFFFFFFFEll))
        return fail(NEUROSIM_E_TIME, "tau_prev out of range");
    DeviceGuard g(h->device);
    const size_t n = (size_t)h->npix;
    if (has_prev) {
        CUDA_TRY(cudaMemcpy(h->ref[h->cidx], ref, n * 4, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h->lprev[h->cidx], lprev, n * 4, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(h->tlast[h->cidx], tlast, n * 4, cudaMemcpyHostToDevice));
    }
    h->has_c = h->has_w = has_prev != 0;
    h->tau_c = h->tau_w = has_prev ? tau_prev : 0;
    return NEUROSIM_OK;
}

int neurosim_evsim_get_thresholds(neurosim_evsim* h, float* c_pos, float* c_neg)
{
    if (!h) return fail(NEUROSIM_E_INVALID, "handle is NULL");
    if (!c_pos || !c_neg) return fail(NEUROSIM_E_INVALID, "output pointers are NULL");
    DeviceGuard g(h->device);
    const size_t n = (size_t)h->npix;
    if (h->cpos) {
        CUDA_TRY(cudaMemcpy(c_pos, h->cpos, n * 4, cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(c_neg, h->cneg, n * 4, cudaMemcpyDeviceToHost));
    } else {
        std::fill(c_pos, c_pos + n, h->cpos_u);
        std::fill(c_neg, c_neg + n, h->cneg_u);
    }
    return NEUROSIM_OK;
}

void neurosim_evsim_destroy(neurosim_evsim* h)
{
    if (!h) return;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
}

int neurosim_evsim_set_profiling(neurosim_evsim* h, int32_t enable)
{
    if (!h) return fail(NEUROSIM_E_INVALID, "handle is NULL");
    h->profiling = enable != 0;
    return NEUROSIM_OK;
}

int neurosim_evsim_get_stats(neurosim_evsim* h, neurosim_evsim_stats* out)
{
    if (!h || !out) return fail(NEUROSIM_E_INVALID, "NULL argument");
    DeviceGuard g(h->device);
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    collect_timings(h);
    *out = h->stats;
    return NEUROSIM_OK;
}

const char* neurosim_last_error(void) { return g_err.c_str(); }

int32_t neurosim_abi_version(void) { return NEUROSIM_EVSIM_ABI_VERSION; }

int neurosim_log_intensity(const float* I_dev, float* L_dev, int64_t n, float log_eps, void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!I_dev || !L_dev))) return fail(NEUROSIM_E_INVALID, "bad arguments");
    if (!(log_eps >= 1e-8f && log_eps <= 1.0f)) return fail(NEUROSIM_E_INVALID, "log_eps must be in [1e-8, 1]");
    if (n == 0) return NEUROSIM_OK;
    CUDA_TRY(launch_log_intensity(I_dev, L_dev, n, log_eps, static_cast<cudaStream_t>(cuda_stream)));
    return NEUROSIM_OK;
}

int neurosim_debug_log(const float* x_dev, float* y_dev, int64_t n, void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!x_dev || !y_dev))) return fail(NEUROSIM_E_INVALID, "bad arguments");
    CUDA_TRY(launch_debug_log(x_dev, y_dev, n, static_cast<cudaStream_t>(cuda_stream)));
    return NEUROSIM_OK;
}

}  // extern "C"
