/*
 * neurosim_evsim.h — C ABI of the GB300 event-generation library
 * (libneurosim_evsim.so).
 *
 * The library turns streams of high-frame-rate intensity frames into DVS
 * event streams under the contrast-threshold model of
 * "Neurosim: A Fast Simulator for Neuromorphic Robot Perception"
 * (arXiv 2602.15018):
 *   - Sec. 1 defines an event as a tuple (t, u, p): integer timestamp in
 *     microseconds, integer pixel u, polarity p in {-1, +1}.
 *   - Sec. 2, paragraph "Neurosim simulates event cameras at multi-kilohertz
 *     rates": every pixel keeps the intensity of its last triggered event and
 *     fires when the change passes a contrast threshold; noise is a
 *     non-ideality the user may disable; each rendered frame produces a
 *     variable number of events, gathered with few global atomics.
 *
 * Model as implemented (the paper gives it in prose; the readings taken are):
 *   L = log(clamp(I, 0, 1e6) + log_eps) with the library's own FP32 log
 *   (input_is_log: L = clamp(I, -32, 32)); log intensity is linear in time
 *   between consecutive frames; ON crossings while fl(ref + C+) <= L_b, OFF
 *   while fl(ref - C-) >= L_b, one threshold at a time, ref moving to each
 *   crossed level; crossing time t = ta + floor(frac * (tb - ta)),
 *   frac = (lvl - L_a) / (L_b - L_a) in FP32; a crossing within
 *   refractory_us of the pixel's last emitted event is suppressed (ref still
 *   moves); per-pixel thresholds C+-_u = max(c_min, C+- + sigma_c * z),
 *   z an Irwin-Hall(12) normal drawn from SplitMix64 at create time.
 *   The first frame a sensor sees initialises ref and emits nothing.
 *
 * Event record (uint64_t): [63:32] t (us, unsigned) | [31:17] y | [16:1] x |
 * [0] p (1 = ON, 0 = OFF).  Output order: interval-major (one interval =
 * the time between two consecutive frames); inside an interval ascending by
 * the record value, i.e. by (t, y, x, p).
 *
 * Threading: a handle is used from one host thread at a time.  All device
 * work of a handle runs on the CUDA stream given at create time.
 * Errors: every call returns a NEUROSIM_* status; the message of the last
 * failure on the calling thread is returned by neurosim_last_error().
 */
#ifndef NEUROSIM_EVSIM_H
#define NEUROSIM_EVSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NEUROSIM_EVSIM_ABI_VERSION 1

enum neurosim_status {
    NEUROSIM_OK = 0,
    NEUROSIM_E_INVALID = 1,   /* bad argument (null, size, range)             */
    NEUROSIM_E_CUDA = 2,      /* a CUDA runtime call failed                   */
    NEUROSIM_E_TIME = 3,      /* timestamps not increasing / out of range     */
    NEUROSIM_E_OVERFLOW = 4,  /* event or interval capacity exceeded          */
    NEUROSIM_E_TIMEOUT = 5,   /* a bounded device wait gave up                */
    NEUROSIM_E_NOMEM = 6,     /* device or host allocation failed             */
    NEUROSIM_E_STATE = 7      /* call not allowed in the handle's state       */
};

/* Opaque simulator handle for one sensor; owned by the library. */
typedef struct neurosim_evsim neurosim_evsim;

typedef struct neurosim_evsim_params {
    int32_t width;               /* 1..65535 pixels                            */
    int32_t height;              /* 1..32767 pixels; width*height <= 2^22      */
    float c_pos;                 /* mean ON threshold in log units (> 0)       */
    float c_neg;                 /* mean OFF threshold in log units (> 0)      */
    float sigma_c;               /* per-pixel threshold std; 0 disables noise  */
    float c_min;                 /* lower clamp of noisy thresholds (>= 1e-3)  */
    uint32_t refractory_us;      /* 0 disables the refractory period           */
    float log_eps;               /* offset inside the log, in [1e-8, 1]        */
    int32_t input_is_log;        /* 1: frames already hold log intensity       */
    uint64_t seed;               /* threshold-noise seed                       */
    const float *c_pos_map;      /* optional HOST [height*width] ON thresholds,
                                    copied at create; overrides c_pos/sigma_c  */
    const float *c_neg_map;      /* optional HOST OFF thresholds (both or none)*/
    uint64_t event_capacity;     /* initial record capacity; 0 = automatic.
                                    Grows on overflow (see drain).            */
    int32_t max_frames_per_step; /* frames per step call; 0 = 1024             */
    int32_t max_pending_intervals; /* intervals between drains; 0 = 65536      */
    int32_t pixels_per_thread;   /* emission pixels per CUDA thread: 8 or 16
                                    (a warp owns 32x that many pixels); 0 = auto */
    int32_t prefetch_frames;     /* frames each thread keeps in flight: 2 or 3;
                                    0 = auto                                    */
    int32_t reserved[6];         /* must be zero                               */
} neurosim_evsim_params;

/* Fills *p with defaults: C+ = C- = 0.2, sigma 0, c_min 0.01, no refractory,
 * log_eps 1e-3, intensity input.  width/height are left 0 and must be set. */
void neurosim_evsim_default_params(neurosim_evsim_params *p);

/* Creates a simulator.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream) on the current device; all device work of the handle is enqueued
 * there.  Allocates the per-pixel state, threshold maps and event buffers on
 * the current device.  Returns NEUROSIM_E_INVALID for bad params. */
int neurosim_evsim_create(const neurosim_evsim_params *p, void *cuda_stream,
                          neurosim_evsim **out);

/* Enqueues one step over n_frames DEVICE frames, FP32 [n_frames][height][width]
 * row-major, frame f at time t0_us + f * dt_us (us).  Asynchronous: returns
 * after enqueueing, without a host synchronisation, and may be captured into a
 * CUDA graph.  The first frame ever initialises the sensor; every later frame
 * closes one interval.  Requires t0_us > the previous frame time (else
 * NEUROSIM_E_TIME), t0_us - previous < 2^24, 1 <= dt_us < 2^24 and the last
 * frame time <= 2^32 - 2.  The caller keeps `frames_dev` valid and unchanged
 * until the next successful drain: a drain that finds an overflow grows the
 * buffers and replays the pending steps from these frames. */
int neurosim_evsim_step(neurosim_evsim *h, const float *frames_dev, int32_t n_frames,
                        int64_t t0_us, int32_t dt_us);

/* As neurosim_evsim_step, but `frames_host` is HOST memory (pinned for best
 * speed): the frames are copied to a library-owned device buffer on the
 * handle's stream before the step.  The host frames must stay valid until
 * the next successful drain (replay on overflow). */
int neurosim_evsim_step_host(neurosim_evsim *h, const float *frames_host, int32_t n_frames,
                             int64_t t0_us, int32_t dt_us);

/* Synchronises the handle's stream and reports the events and intervals
 * pending since the last drain.  Resolves a capacity overflow by growing the
 * buffers and replaying the pending steps (results stay exact).  Either
 * output pointer may be NULL. */
int neurosim_evsim_pending(neurosim_evsim *h, uint64_t *n_events, int64_t *n_intervals);

/* Copies the pending events, in output order, into `out` (DEVICE memory if
 * out_is_device, else HOST memory) and clears them.  out_capacity is in
 * records; if it is smaller than the pending count the call returns
 * NEUROSIM_E_OVERFLOW, sets *n_out to the count needed and keeps the events.
 * If seg_offsets is not NULL it receives n_intervals + 1 HOST int64 offsets
 * (interval k holds records [seg_offsets[k], seg_offsets[k+1])), provided
 * seg_capacity >= n_intervals + 1 (else NEUROSIM_E_OVERFLOW).  n_segs (may be
 * NULL) receives n_intervals.  Synchronises the stream. */
int neurosim_evsim_drain_events(neurosim_evsim *h, uint64_t *out, uint64_t out_capacity,
                                int32_t out_is_device, uint64_t *n_out, int64_t *seg_offsets,
                                int64_t seg_capacity, int64_t *n_segs);

/* Copies the per-pixel state after the last enqueued step into HOST arrays
 * of height*width entries: ref (reference log level), lprev (log intensity of
 * the last frame), tlast (time of the last emitted event, 0xFFFFFFFF = none).
 * *tau_prev gets the last frame time, *has_prev whether a frame was seen.
 * Any pointer may be NULL.  Synchronises (and resolves overflow like
 * neurosim_evsim_pending). */
int neurosim_evsim_get_state(neurosim_evsim *h, float *ref, float *lprev, uint32_t *tlast,
                             int64_t *tau_prev, int32_t *has_prev);

/* Replaces the per-pixel state (HOST arrays as in get_state; all three
 * required when has_prev is 1).  Allowed only with no pending events or
 * intervals (else NEUROSIM_E_STATE).  A resumed run reproduces the events of
 * an uninterrupted one bit for bit. */
int neurosim_evsim_set_state(neurosim_evsim *h, const float *ref, const float *lprev,
                             const uint32_t *tlast, int64_t tau_prev, int32_t has_prev);

/* Copies the per-pixel ON/OFF thresholds (HOST, height*width each). */
int neurosim_evsim_get_thresholds(neurosim_evsim *h, float *c_pos, float *c_neg);

/* Frees all device and host resources of the handle (synchronises first). */
void neurosim_evsim_destroy(neurosim_evsim *h);

/* Counters of a handle (all since create; replays after overflow included). */
typedef struct neurosim_evsim_stats {
    uint64_t steps;            /* step launches enqueued                        */
    uint64_t kernel_launches;  /* CUDA kernels launched by the library           */
    uint64_t px_frames;        /* pixel-frames processed by those steps          */
    uint64_t events_drained;   /* records handed out by drains                   */
    uint64_t timed_steps;      /* steps enqueued while profiling was on          */
    double emit_ms;            /* summed emission-kernel time of timed steps     */
    double sort_ms;            /* summed interval count + scan + sort time       */
} neurosim_evsim_stats;

/* Turns per-step timing on (1) or off (0).  When on, every step records CUDA
 * events on the handle's stream around the emission kernel and around the
 * interval sort; neurosim_evsim_get_stats sums them.  Leave off while
 * capturing a CUDA graph. */
int neurosim_evsim_set_profiling(neurosim_evsim *h, int32_t enable);

/* Synchronises the handle's stream and fills *out. */
int neurosim_evsim_get_stats(neurosim_evsim *h, neurosim_evsim_stats *out);

/* Message of the last failed call on this host thread ("" if none). */
const char *neurosim_last_error(void);

/* Library ABI version (NEUROSIM_EVSIM_ABI_VERSION of the build). */
int32_t neurosim_abi_version(void);

/* Evaluates the library's FP32 log (the one the event model uses) on n DEVICE
 * floats x_dev into y_dev on cuda_stream; for verification of the log. */
int neurosim_debug_log(const float *x_dev, float *y_dev, int64_t n, void *cuda_stream);

/* One step of the event model that allocates nothing.  The paper has no
 * counterpart: this is a library convenience for callers that cannot call
 * cudaMalloc (code inside a CUDA graph being captured, real-time loops that
 * must never enter the allocator, hosts that only borrow device buffers).
 * The caller owns every buffer; the library keeps its intermediates (event
 * keys, chunk table, per-interval counts, control block) in one fixed 32 MiB
 * device array compiled into the library (held by every GPU that loads it,
 * until exit).
 *
 * Inputs (DEVICE memory unless noted): frames_dev FP32 [n_frames][height]
 * [width] at times t0_us + f * dt_us; thresholds c_pos_dev / c_neg_dev
 * (height*width each, 16-byte aligned) or both NULL for the uniform c_pos /
 * c_neg (>= 1e-3); refractory_us, log_eps, input_is_log as in the params.
 * State: with has_prev = 1, ref_in / lprev_in / tlast_in hold the state after
 * the frame at tau_prev (as returned by a previous call); with has_prev = 0
 * the first frame initialises the state and emits nothing.  The new state is
 * written to ref_out / lprev_out / tlast_out (all 16-byte aligned; they must
 * not overlap the input arrays, so that a failed call can be repeated from
 * the same inputs).  Outputs: events_dev receives the step's records in
 * output order (capacity events_capacity), seg_offsets_dev the n_intervals + 1
 * DEVICE int64 offsets (n_intervals = n_frames - 1 + has_prev), *n_events
 * (HOST) the record count.
 * Errors: NEUROSIM_E_INVALID for bad sizes, NULL or misaligned pointers and
 * for steps whose chunk table (n_intervals x ceil(width*height / 512) entries)
 * does not fit half of the fixed array; NEUROSIM_E_OVERFLOW when the events
 * exceed events_capacity (*n_events = the count needed) or the array's key
 * area — then the outputs are not usable and the call can be repeated with a
 * larger buffer or fewer frames.  Synchronises cuda_stream before returning.
 * Every call shares the one array and it keeps the last call's contents (the
 * control block is cleared at the start of each call): calls whose GPU work
 * overlaps — on different streams with no order between them — race.  The
 * first call on a device looks up the array's device address and sets up the
 * kernels; make it before any stream capture. */
int neurosim_evsim_step_noalloc(const float *frames_dev, int32_t n_frames, int32_t width,
                                int32_t height, int64_t t0_us, int32_t dt_us,
                                const float *c_pos_dev, const float *c_neg_dev, float c_pos,
                                float c_neg, uint32_t refractory_us, float log_eps,
                                int32_t input_is_log, const float *ref_in, const float *lprev_in,
                                const uint32_t *tlast_in, float *ref_out, float *lprev_out,
                                uint32_t *tlast_out, int32_t has_prev, int64_t tau_prev,
                                uint64_t *events_dev, uint64_t events_capacity,
                                int64_t *seg_offsets_dev, uint64_t *n_events, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* NEUROSIM_EVSIM_H */
