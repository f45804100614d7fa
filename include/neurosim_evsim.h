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

#define NEUROSIM_EVSIM_ABI_VERSION 2

enum neurosim_status {
    NEUROSIM_OK = 0,
    NEUROSIM_E_INVALID = 1,   /* bad argument (null, size, range)             */
    NEUROSIM_E_CUDA = 2,      /* a CUDA runtime call failed                   */
    NEUROSIM_E_TIME = 3,      /* timestamps not increasing / out of range     */
    NEUROSIM_E_OVERFLOW = 4,  /* event or interval capacity exceeded          */
    NEUROSIM_E_TIMEOUT = 5,   /* a bounded device wait gave up                */
    NEUROSIM_E_NOMEM = 6,     /* device or host allocation failed             */
    NEUROSIM_E_STATE = 7,     /* call not allowed in the handle's state       */
    NEUROSIM_E_IO = 8         /* a file could not be opened, read or written  */
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
                                    0 = auto.  The emission kernel models the
                                    frames in pairs and keeps one pair in
                                    flight: 2 and 3 behave the same          */
    int32_t ctas_per_sm;         /* emission CTAs resident per SM (each CTA
                                    holds 64 / pixels_per_thread warps, one
                                    tile each at a time); 0 = as many as fit */
    int32_t reserved[5];         /* must be zero                               */
} neurosim_evsim_params;

/* Fills *p with defaults: C+ = C- = 0.2, sigma 0, c_min 0.01, no refractory,
 * log_eps 1e-3, intensity input.  width/height are left 0 and must be set. */
void neurosim_evsim_default_params(neurosim_evsim_params *p);

/* Creates a simulator: one event camera of width x height pixels.  Paper:
 * Sec. 2, paragraph "Neurosim simulates event cameras at multi-kilohertz
 * rates" (each pixel keeps the level of its last triggered event, compared
 * against contrast thresholds; noise is a user-disableable non-ideality, here
 * the per-pixel threshold maps drawn at create).  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream) on the current device; all device work of the handle is enqueued
 * there.  Allocates the per-pixel state, threshold maps and event buffers on
 * the current device.  Returns NEUROSIM_E_INVALID for bad params. */
int neurosim_evsim_create(const neurosim_evsim_params *p, void *cuda_stream,
                          neurosim_evsim **out);

/* Enqueues one step over n_frames DEVICE frames, FP32 [n_frames][height][width]
 * row-major, frame f at time t0_us + f * dt_us (us).  Paper: Sec. 2, same
 * paragraph (every rendered intensity frame updates each pixel's state against
 * its last event level and yields a variable number of events, gathered with
 * few global atomics); Sec. 1 for the event tuple (t in us, pixel, polarity).  Asynchronous: returns
 * after enqueueing, without a host synchronisation, and may be captured into a
 * CUDA graph.  The first frame ever initialises the sensor; every later frame
 * closes one interval.  Requires t0_us > the previous frame time (else
 * NEUROSIM_E_TIME), t0_us - previous < 2^24, 1 <= dt_us < 2^24 and the last
 * frame time <= 2^32 - 2.  The caller keeps `frames_dev` valid and unchanged
 * until the next successful drain: a drain that finds an overflow grows the
 * buffers and replays the pending steps from these frames. */
int neurosim_evsim_step(neurosim_evsim *h, const float *frames_dev, int32_t n_frames,
                        int64_t t0_us, int32_t dt_us);

/* As neurosim_evsim_step, but `frames_host` is HOST memory holding n_frames
 * frames.  Page-locked memory that is mapped into the device's address space
 * (cudaHostAlloc / cudaHostRegister memory on a system with unified
 * addressing) is read in place by the emission kernel: each frame crosses the
 * host link once, while the step runs.  Other host memory is first copied to
 * a library-owned device buffer on the handle's stream.  The host frames must
 * stay valid and unchanged until the next successful drain (replay on
 * overflow). */
int neurosim_evsim_step_host(neurosim_evsim *h, const float *frames_host, int32_t n_frames,
                             int64_t t0_us, int32_t dt_us);

/* Synchronises the handle's stream and reports the events and intervals
 * pending since the last drain.  Resolves a capacity overflow by growing the
 * buffers and replaying the pending steps (results stay exact).  Either
 * output pointer may be NULL. */
int neurosim_evsim_pending(neurosim_evsim *h, uint64_t *n_events, int64_t *n_intervals);

/* Copies the pending events, in output order, into `out` (DEVICE memory if
 * out_is_device, else HOST memory) and clears them.  Paper: Sec. 1 defines
 * the event as (t, u, p) with integer microsecond timestamps; Sec. 2 (same
 * paragraph) makes the number of events per frame variable, so the caller
 * learns the count here.  Records are packed as described at the top.  out_capacity is in
 * records; if it is smaller than the pending count the call returns
 * NEUROSIM_E_OVERFLOW, sets *n_out to the count needed and keeps the events.
 * If seg_offsets is not NULL it receives n_intervals + 1 HOST int64 offsets
 * (interval k holds records [seg_offsets[k], seg_offsets[k+1])), provided
 * seg_capacity >= n_intervals + 1 (else NEUROSIM_E_OVERFLOW).  n_segs (may be
 * NULL) receives n_intervals.  Synchronises the stream. */
int neurosim_evsim_drain_events(neurosim_evsim *h, uint64_t *out, uint64_t out_capacity,
                                int32_t out_is_device, uint64_t *n_out, int64_t *seg_offsets,
                                int64_t seg_capacity, int64_t *n_segs);

/* Zero-copy access to the pending events (Sec. 3 of the paper hands sensor
 * data to NumPy / PyTorch consumers without copies; this is the in-process
 * counterpart).  peek resolves a capacity overflow like
 * neurosim_evsim_pending (synchronises), then sets *events_dev to the
 * library's DEVICE buffer holding the n_out pending records in output order,
 * and fills seg_offsets (HOST, nullable, capacity seg_capacity) as drain
 * does.  The records stay the library's: the pointer is valid until the next
 * step, drain, release, set_state or destroy of the handle, and the events
 * stay pending.  release then clears them (and commits the state, as a drain
 * does) without copying anything. */
int neurosim_evsim_peek_events(neurosim_evsim *h, const uint64_t **events_dev, uint64_t *n_out,
                               int64_t *seg_offsets, int64_t seg_capacity, int64_t *n_segs);
int neurosim_evsim_release_events(neurosim_evsim *h);

/* As peek, returning the records as a DLPack tensor (a DLManagedTensor of the
 * DLPack v0.8 ABI: 1-D, 64-bit integer holding the record bits, CUDA device
 * memory of the handle's device, compact), for any DLPack consumer (torch.from_dlpack, CuPy, JAX).
 * The view aliases the library's buffer with the same validity as peek; the
 * consumer's call of the tensor's deleter frees the descriptor only.  Wrap
 * *managed_tensor in a capsule named "dltensor" to hand it over. */
int neurosim_evsim_events_dlpack(neurosim_evsim *h, void **managed_tensor);

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

/* Frees all device and host resources of the handle (synchronises first):
 * the per-pixel state of Sec. 2's event model, the threshold maps and the
 * event buffers.  NULL is ignored. */
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

/* ------------------------------------------------------------------------
 * Batched sensors: many independent streams in one launch per step.
 *
 * Sec. 4 (event-based RL paragraph) and the RL appendix run several
 * independent simulation instances concurrently on one GPU; a batch steps
 * all of their event cameras together: one emission launch over a flattened
 * (stream, tile) work list, one interval sort over every (stream, interval),
 * streams of different resolutions and parameters side by side.  Each
 * stream's events are exactly those of a single-stream simulator fed the
 * same frames.
 *
 * Every step consumes frames_per_step frames per stream from one of the
 * frame-buffer sets ("slots") registered with neurosim_evsim_batch_set_frames.
 * Everything that changes from step to step (times, state buffer, pending
 * intervals, record count) lives in device memory, so
 * neurosim_evsim_batch_step allocates nothing, never synchronises, and may
 * be captured into a CUDA graph on the batch's stream (one graph per slot)
 * and replayed; the caller refills a slot's buffers between the replays
 * that read it.  Frame j of step k (k = 0, 1, ...) is at
 * t0_us + (1 + k * frames_per_step + j) * dt_us; frame t0_us is the one
 * given to neurosim_evsim_batch_init.
 * ---------------------------------------------------------------------- */
typedef struct neurosim_evsim_batch neurosim_evsim_batch;

typedef struct {
    int32_t n_streams;           /* >= 1                                          */
    int32_t frames_per_step;     /* T >= 1, frames per stream per step            */
    int32_t dt_us;               /* frame spacing, 1 <= dt_us < 2^24              */
    int32_t max_pending_steps;   /* steps that may run between drains (0 = 4)     */
    int64_t t0_us;               /* time of the initialising frame, >= 0          */
    uint64_t event_capacity;     /* records kept between drains (0 = auto:
                                    sum(W*H) * T * max_pending_steps / 16)        */
    int32_t pixels_per_thread;   /* emission tile: 0 (16), 8 or 16                */
    int32_t prefetch_frames;     /* frames in flight per lane: 0 (2), 2 or 3
                                    (one pair of frames either way)              */
    int32_t frame_slots;         /* frame-buffer sets that can be registered
                                    (0 = 2, at most 16): a renderer fills one
                                    while the steps read another               */
    int32_t ctas_per_sm;         /* emission CTAs per SM: 0 = as many as fit      */
    int32_t reserved[4];         /* must be zero                                  */
} neurosim_evsim_batch_params;

/* Fills *p with defaults (n_streams 1, T 16, dt 1000 us). */
void neurosim_evsim_batch_default_params(neurosim_evsim_batch_params *p);

/* Creates a batch of bp->n_streams sensors; streams[i] describes sensor i
 * exactly as for neurosim_evsim_create (its event_capacity,
 * max_frames_per_step, max_pending_intervals, pixels_per_thread and
 * prefetch_frames are ignored; threshold maps are copied).  Device work runs
 * on cuda_stream (NULL = legacy default stream).  Errors: NEUROSIM_E_INVALID
 * (params), NEUROSIM_E_NOMEM, NEUROSIM_E_CUDA. */
int neurosim_evsim_batch_create(const neurosim_evsim_params *streams,
                                const neurosim_evsim_batch_params *bp, void *cuda_stream,
                                neurosim_evsim_batch **out);

/* Registers the frame buffers of slot `slot` (0 <= slot < frame_slots):
 * frames_dev is a HOST array of n_streams DEVICE pointers, stream i's buffer
 * holding frames_per_step FP32 frames [T][H_i][W_i].  The buffers stay owned
 * by the caller and must stay valid while steps that read them may run.
 * Synchronises the batch's stream; not capturable.  NEUROSIM_E_INVALID for
 * a NULL pointer or a bad slot. */
int neurosim_evsim_batch_set_frames(neurosim_evsim_batch *b, int32_t slot,
                                    const float *const *frames_dev);

/* As neurosim_evsim_batch_set_frames, with stream i's frame f at
 * frames_dev[i] + f * frame_strides[i] floats (HOST array; 0 or NULL = W*H,
 * else >= W*H): frames of many sensors can sit interleaved in one array,
 * e.g. the [3][batch][H][W] output of the learned interpolator. */
int neurosim_evsim_batch_set_frames_strided(neurosim_evsim_batch *b, int32_t slot,
                                            const float *const *frames_dev, const int64_t *frame_strides);

/* Initialises every stream from one frame at t0_us (HOST array of n_streams
 * DEVICE pointers to one [H_i][W_i] FP32 frame each): ref = L_prev = L, no
 * events.  Enqueued on the batch's stream.  NEUROSIM_E_STATE if the batch
 * was initialised already. */
int neurosim_evsim_batch_init(neurosim_evsim_batch *b, const float *const *first_frames_dev);

/* Enqueues one step over the buffers registered in `slot` (emission,
 * interval count, scan, sort and the device clock's advance: 5 kernels).
 * Capturable.  If a step overflows a capacity, it and every later step are
 * dropped on the device (state, clock and pending intervals stay as after
 * the last good step) and the next drain reports it.  NEUROSIM_E_STATE
 * before init or before the slot was registered. */
int neurosim_evsim_batch_step(neurosim_evsim_batch *b, int32_t slot);

/* Synchronises; *n_events = records of the committed steps since the last
 * drain, *n_segments = their intervals (steps * n_streams * T). */
int neurosim_evsim_batch_pending(neurosim_evsim_batch *b, uint64_t *n_events, int64_t *n_segments);

/* Synchronises and hands out the committed records: out (capacity records;
 * DEVICE memory if out_is_device, else HOST) receives them in order step,
 * stream, interval, then (t, y, x, p); seg_offsets (HOST, nullable,
 * seg_capacity >= n_segments + 1) receives the n_segments + 1 offsets of
 * the (step, stream, interval) segments in that order.  Clears the pending
 * records.  If a step was dropped, delivers the committed records, clears
 * the condition and returns NEUROSIM_E_OVERFLOW (records, keys or pending
 * intervals; the message names which and the demand) or NEUROSIM_E_TIME;
 * the caller re-runs the dropped steps' frames, on a larger batch if the
 * capacity was the cause.  NEUROSIM_E_OVERFLOW with nothing copied if
 * capacity < n_events or seg_capacity is too small. */
int neurosim_evsim_batch_drain(neurosim_evsim_batch *b, void *out, uint64_t capacity,
                               int32_t out_is_device, uint64_t *n_out, int64_t *seg_offsets,
                               int64_t seg_capacity, int64_t *n_segments);

/* Copies stream i's state after the last committed step to HOST arrays of
 * W_i*H_i entries (ref, L_prev, t_last with 0xFFFFFFFF = none) and *tau_us
 * (time of the last frame consumed).  Synchronises. */
int neurosim_evsim_batch_get_state(neurosim_evsim_batch *b, int32_t stream, float *ref,
                                   float *lprev, uint32_t *tlast, int64_t *tau_us);

/* Copies stream i's per-pixel thresholds to HOST arrays of W_i*H_i floats. */
int neurosim_evsim_batch_get_thresholds(neurosim_evsim_batch *b, int32_t stream, float *c_pos,
                                        float *c_neg);

/* Kernel launches enqueued by the batch so far (*launches) and committed
 * steps (*steps, synchronises). */
int neurosim_evsim_batch_counters(neurosim_evsim_batch *b, uint64_t *launches, uint64_t *steps);

/* Frees the batch (synchronises its stream first). */
void neurosim_evsim_batch_destroy(neurosim_evsim_batch *b);

/* ------------------------------------------------------------------------
 * Autotuner: picks the emission launch shape for a workload by timing every
 * variant on the caller's frames: the warp tile (pixels_per_thread 8 or 16:
 * 256 or 512 pixels per warp) times the number of emission CTAs resident per
 * SM (1 up to what fits).  The paper has no autotuner (it fixes one thread
 * per pixel).
 *
 * Times `repeats` (>= 1) steps of n_frames frames (DEVICE [T][H][W] FP32 at
 * spacing dt_us) with each variant on a fresh simulator of params p (the
 * params' launch fields are ignored) and keeps the one with the smallest
 * median emission + sort time; all variants produce the same events.  If
 * cache_path is not NULL, a result cached there for this GPU model, width,
 * height and n_frames is returned without timing, and a new result is
 * appended to it (one JSON object per line: {"gpu": ..., "width": W,
 * "height": H, "frames": T, "pixels_per_thread": P, "ctas_per_sm": C,
 * "ms": M, "timings": [[P, C, ms], ...]}, every variant timed).  *ms_out
 * (nullable) gets the winner's median time.  Returns NEUROSIM_E_INVALID /
 * NEUROSIM_E_CUDA / NEUROSIM_E_NOMEM. */
int neurosim_evsim_autotune(const neurosim_evsim_params *p, const float *frames_dev,
                            int32_t n_frames, int32_t dt_us, int32_t repeats,
                            const char *cache_path, int32_t *pixels_per_thread,
                            int32_t *ctas_per_sm, double *ms_out);

/* ------------------------------------------------------------------------
 * Learned interpolator.  The paper has no counterpart (it renders every frame,
 * Sec. 2); this is the project's way to run the renderer at a quarter of the
 * event camera's rate: a 3-level convolutional U-Net predicts the three log
 * frames between two log keyframes L0 (time tau) and L4 (tau + 4 dt):
 *   L_j = L0 + (j / 4)(L4 - L0) + r_j(L0, L4),  j = 1, 2, 3,
 * with BF16 weights and activations, FP32 accumulation on the tensor cores,
 * and r = 0 for the untrained network (linear interpolation).  Layers:
 * conv3x3 8->32, conv3x3/2 32->64, conv3x3/2 64->128, conv3x3 128->128,
 * convT2x2/2 128->64 | skip, conv3x3 128->64, convT2x2/2 64->32 | skip,
 * conv3x3 64->32, conv1x1 32->3; ReLU after every 3x3 convolution.
 *
 * Parameters (FP32, neurosim_interp_param_count() values): weights, then
 * biases, layer by layer; 3x3 layers as [3][3][Cin][Cout], transposed layers
 * as [Cin][2][2][Cout], the 1x1 layer as [32][16] (outputs 3..15 unused and
 * zero), biases [Cout] (the last one 16 with 3..15 zero).
 * ---------------------------------------------------------------------- */
typedef struct neurosim_interp neurosim_interp;

/* Number of FP32 parameters in the flat layout above. */
int64_t neurosim_interp_param_count(void);

/* Creates a network for up to max_batch images of max_height x max_width
 * (both divisible by 4), with seeded He-normal weights; device work runs on
 * cuda_stream. */
int neurosim_interp_create(int32_t max_batch, int32_t max_height, int32_t max_width, uint64_t seed,
                           void *cuda_stream, neurosim_interp **out);

/* Predicts frames 1..3 between DEVICE log keyframes L0_dev and L4_dev
 * ([batch][height][width] FP32) into out_dev ([3][batch][height][width]
 * FP32).  Asynchronous on the network's stream. */
int neurosim_interp_forward(neurosim_interp *h, const float *L0_dev, const float *L4_dev, int32_t batch,
                            int32_t height, int32_t width, float *out_dev);

/* One AdamW step (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay on the
 * weights) on DEVICE training clips [batch][5][height][width] of log frames
 * at 1000 FPS: frames 0 and 4 are the keyframes, 1..3 the targets; loss =
 * mean Charbonnier (eps 1e-3) over the three frames.  *loss_out (HOST,
 * nullable; synchronises when given) receives the loss before the step. */
int neurosim_interp_train_step(neurosim_interp *h, const float *clips_dev, int32_t batch, int32_t height,
                               int32_t width, float lr, float weight_decay, float *loss_out);

/* Loss and parameter gradients (HOST array of param_count floats, nullable)
 * for clips as in train_step, without updating.  Synchronises. */
int neurosim_interp_gradients(neurosim_interp *h, const float *clips_dev, int32_t batch, int32_t height,
                              int32_t width, float *grads_host, float *loss_out);

/* Copies the FP32 parameters to / from HOST memory (n = param_count);
 * set_params also resets the optimiser state.  Synchronise. */
int neurosim_interp_get_params(neurosim_interp *h, float *host, int64_t n);
int neurosim_interp_set_params(neurosim_interp *h, const float *host, int64_t n);

/* Checkpoints of the network.  save writes the FP32 parameters and, when
 * with_optimizer != 0, the AdamW moments and step count to the HOST file
 * `path` (written to path + ".tmp", then renamed over path).  load reads
 * such a file into a network of any max sizes: the parameters, and the
 * optimiser state if the file holds it (else the state is reset, as by
 * set_params).  Layout (little-endian): "NSIMUNT1", uint32 version 1,
 * uint32 flags (bit 0: moments present), int64 parameter count, int64 step,
 * the FP32 arrays, then the FNV-1a 64-bit hash of all preceding bytes.
 * Errors: NEUROSIM_E_IO (open, read, write, rename), NEUROSIM_E_INVALID (not
 * a checkpoint, other version, other parameter count, truncated, hash
 * mismatch; the network is then unchanged), NEUROSIM_E_CUDA.  Synchronise. */
int neurosim_interp_save(neurosim_interp *h, const char *path, int32_t with_optimizer);
int neurosim_interp_load(neurosim_interp *h, const char *path);

/* Kernels launched by the network so far. */
int neurosim_interp_launches(neurosim_interp *h, uint64_t *launches);

/* Frees the network (synchronises its stream first). */
void neurosim_interp_destroy(neurosim_interp *h);

/* Time surface (RL appendix of the paper, Observation Space paragraph:
 * S(x, y, p) <- S(x, y, p) exp(-dt / tau) + 1 at every event of that cell).
 * S_dev: DEVICE FP32 [2][height][width] (p = 0 OFF, 1 ON) holding the surface
 * evaluated at *t_ref_us (HOST in/out; start with S = 0).  Moves S to
 * t_query_us >= *t_ref_us and adds the DEVICE records events_dev[0..n), all
 * with t <= t_query_us:  S <- S exp(-(t_q - t_ref)/tau) + sum exp(-(t_q - t_i)/tau)
 * (the per-event recursion evaluated at t_q, up to FP32 rounding), then
 * sets *t_ref_us = t_query_us.  Synchronises cuda_stream.  NEUROSIM_E_INVALID
 * for an event outside the sensor or after t_query_us, NEUROSIM_E_TIME for
 * t_query_us < *t_ref_us. */
int neurosim_time_surface(float *S_dev, int32_t width, int32_t height, int64_t *t_ref_us,
                          const uint64_t *events_dev, int64_t n, int64_t t_query_us, float tau_us,
                          void *cuda_stream);

/* Polarity event frames: counts_dev (DEVICE int32 [n_windows][2][height][width],
 * accumulated into) gets one count per event of window
 * (t - t_start_us) / window_us in [0, n_windows).  Synchronises cuda_stream. */
int neurosim_event_frames(int32_t *counts_dev, int32_t width, int32_t height, const uint64_t *events_dev,
                          int64_t n, int64_t t_start_us, int64_t window_us, int32_t n_windows,
                          void *cuda_stream);

/* Scores HOST event records `pred` against `ref` (any order): events match
 * one to one inside the same pixel and polarity, greedily in time order,
 * when their times differ by at most tol_us.  counts = {matched, n_pred,
 * n_ref, sum over (pixel, polarity) of |n_pred - n_ref|}; scores =
 * {precision, recall, F1, count error = counts[3] / n_ref}.  The paper defines
 * no score; this is the one the learned interpolator is scored by. */
int neurosim_event_f1(const uint64_t *pred, int64_t n_pred, const uint64_t *ref, int64_t n_ref,
                      int64_t tol_us, int64_t *counts, double *scores);

/* ------------------------------------------------------------------------
 * Render-fused event simulation.  Sec. 1 of the paper argues that event data
 * should be produced on the fly, without storing the rendered images.  The
 * library carries a seeded procedural scene (the scenes of the paper are
 * rendered by a graphics engine, not available here) that the emission
 * kernel can render itself, pixel by pixel, in place of reading frames: a
 * fused step moves no frame bytes through memory.  The same scene can be
 * rendered to memory by neurosim_render_texture, bit for bit the
 * intensities the fused step sees.
 *
 * Scene: value noise of `octaves` octaves (hashed integer lattice with
 * smoothstep interpolation, base period `base_period` px, each octave at
 * half the period and `gain` times the amplitude of the one before; octave
 * o (from 0) hashes with salt + 0x9E3779B9 (o + 1)), mapped to
 * [intensity_lo, intensity_hi]; seen through a camera that rotates by
 * theta(t) = rot_amp / k (cos(rot_phase) - cos(k t + rot_phase)),
 * k = 2 pi / rot_period (the integral of a rotation rate rot_amp
 * sin(k t + rot_phase), rad/s), zooms by z(t) = 1 + zoom_amp
 * sin(2 pi t / zoom_period + zoom_phase) about the image centre and
 * translates by (vx, vy) t + (offset_x, offset_y): pixel (x, y) sees texture
 * point R(theta) ((x, y) - centre) / z + centre + (vx, vy) t + offset.
 * Then n_rects rectangles, drawn in order (the last on top): rectangle i
 * of size rect_w x rect_h has constant intensity rect_value and its centre
 * at ((rect_x + rect_vx t) mod (W + rect_w) - rect_w / 2, (rect_y + rect_vy t)
 * mod (H + rect_h) - rect_h / 2); it covers the pixels strictly within half
 * its size of the centre.  Times in seconds.  The per-frame camera and
 * rectangles are evaluated in double, the pixels in FP32.
 * ---------------------------------------------------------------------- */
#define NEUROSIM_MAX_RECTS 16

typedef struct neurosim_texture_scene {
    int32_t width, height;       /* pixels, as a sensor's params               */
    uint32_t salt;               /* value-noise hash salt                      */
    int32_t octaves;             /* 1..8                                       */
    float base_period;           /* px, in [1, 65536]                          */
    float gain;                  /* amplitude ratio of successive octaves, (0, 1] */
    float intensity_lo, intensity_hi;  /* noise range, 0 <= lo <= hi <= 1e6   */
    double vx, vy;               /* camera translation, px/s                   */
    double offset_x, offset_y;   /* texture offset, px                         */
    double rot_amp_rad_s, rot_period_s, rot_phase;
    double zoom_amp, zoom_period_s, zoom_phase;   /* |zoom_amp| < 0.5          */
    int32_t n_rects;             /* 0..NEUROSIM_MAX_RECTS                      */
    int32_t reserved;            /* must be zero                               */
    double rect_x[NEUROSIM_MAX_RECTS], rect_y[NEUROSIM_MAX_RECTS];
    double rect_w[NEUROSIM_MAX_RECTS], rect_h[NEUROSIM_MAX_RECTS];
    double rect_vx[NEUROSIM_MAX_RECTS], rect_vy[NEUROSIM_MAX_RECTS];
    double rect_value[NEUROSIM_MAX_RECTS];
} neurosim_texture_scene;

/* Renders frames t0_us + f * dt_us, f < n_frames (<= 65535), of the scene
 * into frames_dev (DEVICE FP32 [n_frames][height][width], caller-owned).
 * Asynchronous on cuda_stream (allocates its per-frame table there).
 * NEUROSIM_E_INVALID for a bad scene or a NULL buffer, NEUROSIM_E_TIME for
 * t0_us < 0 or dt_us < 1. */
int neurosim_render_texture(const neurosim_texture_scene *scene, float *frames_dev, int32_t n_frames,
                            int64_t t0_us, int32_t dt_us, void *cuda_stream);

/* As neurosim_evsim_step over the frames neurosim_render_texture would
 * render for (scene, n_frames, t0_us, dt_us), with the rendering fused into
 * the emission kernel (Sec. 2 per-frame update on frames produced on the
 * fly, Sec. 1).  The scene must have the sensor's width and height; it is
 * copied, so the caller may change it after the call.  Same timing rules,
 * asynchrony and errors as neurosim_evsim_step; events are identical to
 * those of neurosim_evsim_step on the rendered frames. */
int neurosim_evsim_step_texture(neurosim_evsim *h, const neurosim_texture_scene *scene, int32_t n_frames,
                                int64_t t0_us, int32_t dt_us);

/* Message of the last failed call on this host thread ("" if none). */
const char *neurosim_last_error(void);

/* Library ABI version (NEUROSIM_EVSIM_ABI_VERSION of the build). */
int32_t neurosim_abi_version(void);

/* Verification of the library's tensor-core GEMM core (used by the learned
 * interpolator): C[M][N] (FP32, DEVICE, row-major) = sum_k A(m, k) B(n, k)
 * with BF16 DEVICE operands; modes 0-3 gather the operands with CUDA cores:
 * bit 0: A stored [K][M] (else [M][K]), bit 1: B stored [K][N] (else
 * [N][K]); modes 4 and 5 load A [M][K] and B [N][K] with TMA into 128- or
 * 64-byte-swizzled tiles (16-byte-aligned operands); mode 6 loads A [K][M]
 * and B [K][N] with TMA as MN-major tiles (the weight-gradient GEMM over
 * pixels, K split over CTAs and summed with atomics).  16 <= N <= 256,
 * N % 16 == 0, K % 8 == 0, M % 8 == 0 when A is stored [K][M].
 * Synchronises cuda_stream. */
int neurosim_debug_umma_gemm(int32_t mode, int32_t M, int32_t N, int32_t K, const void *A,
                             const void *B, float *C, void *cuda_stream);

/* Verification of the bounded device waits (no counterpart in the paper):
 * every wait of the library's kernels on an mbarrier gives up after a time
 * limit, records NEUROSIM_E_TIMEOUT and lets the kernel return, so that a
 * lost arrival cannot hang the GPU.  This launches one warp that waits, with
 * that same bounded wait and a limit of limit_ns (1 us .. 100 ms), on an
 * mbarrier that it arrives on itself when arrive != 0 and that nothing
 * arrives on otherwise.  Returns NEUROSIM_OK when the wait completed and
 * NEUROSIM_E_TIMEOUT when it gave up (the GPU context stays usable).
 * Synchronises cuda_stream.  NEUROSIM_E_INVALID for a limit out of range. */
int neurosim_debug_expiring_wait(int32_t arrive, uint64_t limit_ns, void *cuda_stream);

/* The event model's log intensity of n DEVICE floats (Sec. 2 contrast model,
 * reading: L = log(clamp(I, 0, 1e6) + log_eps) with the library's FP32 log):
 * L_dev[i] = the L the emission kernel computes for I_dev[i].  Feeding these
 * frames with input_is_log = 1 gives the same events as the raw frames with
 * input_is_log = 0.  Asynchronous on cuda_stream. */
int neurosim_log_intensity(const float *I_dev, float *L_dev, int64_t n, float log_eps, void *cuda_stream);

/* Sensor bandwidth limit (Sec. 2 of the paper: "bandwidth limitations" are
 * among the non-idealities the simulator models and the user may turn off;
 * the paper gives no model).  This library's reading: a first-order low-pass
 * filter on each pixel's log intensity, one update per frame,
 *   s_k = s_{k-1} + alpha (L_k - s_{k-1}),  alpha = 1 - exp(-2 pi f_c dt),
 * in FP32 as d = L - s, s = fma(alpha, d, s).  L_dev: DEVICE log frames
 * [n_frames][n_pix] FP32; out_dev: DEVICE [n_frames][n_pix], equal to L_dev
 * (in place) or not overlapping it; state_dev: DEVICE [n_pix] filter levels,
 * read unless init != 0 (then set from frame 0, which passes unchanged) and
 * always written back, so that consecutive calls continue one stream.
 * alpha in (0, 1]; alpha = 1 follows the frames (within the rounding of
 * L - s).  Feed the output to
 * the event model with input_is_log = 1.  Asynchronous on cuda_stream.
 * Errors: NEUROSIM_E_INVALID (sizes, alpha, NULL or partly overlapping
 * buffers, init with no frame), NEUROSIM_E_CUDA. */
int neurosim_lowpass_log(const float *L_dev, float *out_dev, int32_t n_frames, int64_t n_pix, float alpha,
                         float *state_dev, int32_t init, void *cuda_stream);

/* Gain of the bandwidth filter above for a cutoff frequency (same reading of
 * Sec. 2's "bandwidth limitations"): a first-order filter with cutoff f_c
 * (time constant 1 / (2 pi f_c)) sampled every dt keeps exp(-2 pi f_c dt) of
 * its level per frame, so *alpha_out = 1 - exp(-2 pi f_c dt), computed on the
 * host in double and rounded once to FP32.  cutoff_hz > 0 and finite,
 * dt_us >= 1 (microseconds).  NEUROSIM_E_INVALID for other arguments, a NULL
 * alpha_out, or a gain that rounds to 0.  Host only; no device work. */
int neurosim_lowpass_alpha(double cutoff_hz, int32_t dt_us, float *alpha_out);

/* Sensor leak (Sec. 2 of the paper lists noise among the non-idealities the
 * simulator models and the user may turn off; it gives no model).  This
 * library's reading: junction leakage makes each pixel's reference level
 * drift down at C+_u * rate_hz per second, so that a still pixel fires ON
 * events rate_hz times a second; for the crossing test this equals the log
 * intensity rising by C+_u * rate_hz * (t - origin_us).  Applied to DEVICE
 * log frames L_dev [n_frames][n_pix] at t0_us + f * dt_us (t0_us >=
 * origin_us) into out_dev (= L_dev for in place, or not overlapping it), in
 * FP32 as fl(L + fl(fl(C+_u * (float)(rate_hz * 1e-6)) * (float)(t -
 * origin))); c_pos_dev: the sensor's per-pixel ON thresholds [n_pix]
 * (neurosim_evsim_get_thresholds) or NULL for the uniform c_pos.  Feed the
 * output to the event model with input_is_log = 1.  Long runs saturate at the
 * model's clamp of 32 after (32 - L) / (C+ rate) seconds.  Asynchronous.
 * NEUROSIM_E_INVALID / NEUROSIM_E_TIME for bad arguments. */
int neurosim_leak_log(const float *L_dev, float *out_dev, int32_t n_frames, int64_t n_pix, int64_t t0_us,
                      int32_t dt_us, int64_t origin_us, double rate_hz, const float *c_pos_dev, float c_pos,
                      void *cuda_stream);

/* Shot noise (same passage; this library's reading): spurious events,
 * independent of the signal and of the pixel state.  For each tile of 64
 * consecutive pixels (row-major; the last one may be shorter, len pixels)
 * and each interval (start ta, length D us), the count is Poisson of mean
 * rate_hz * len * D * 1e-6 (at most 4: NEUROSIM_E_INVALID above), drawn by
 * inversion of the 53-bit uniform of SplitMix64 output
 * (ta * n_tiles + tile) * 32 of `seed`, capped at 15; event i takes outputs
 * base + 1 + 2i (pixel tile * 64 + floor(hi32 * len / 2^32), time
 * ta + floor(lo32 * D / 2^32)) and base + 2 + 2i (polarity: its top bit).
 * Intervals: the first from ta0_us, D0_us long, then n_intervals - 1 of
 * dt_us (a step's intervals).  Writes the records (format of the event
 * stream, interval-major, ascending per interval) to events_dev (DEVICE,
 * capacity records) and n_intervals + 1 HOST offsets to seg_offsets;
 * *n_events gets the count (also when it exceeds capacity:
 * NEUROSIM_E_OVERFLOW).  At most 8192 events per interval.  Synchronises. */
int neurosim_shot_noise(int32_t width, int32_t height, double rate_hz, uint64_t seed, int64_t ta0_us,
                        int32_t D0_us, int32_t dt_us, int32_t n_intervals, uint64_t *events_dev,
                        uint64_t capacity, int64_t *seg_offsets, uint64_t *n_events, void *cuda_stream);

/* Merges two event streams with the same intervals (DEVICE records, HOST
 * offsets seg_a / seg_b of n_intervals + 1 entries from 0), each ascending
 * per interval, into out_dev (DEVICE, seg_a[n] + seg_b[n] records) in the
 * stream's order, interval by interval; seg_out (HOST, nullable) gets the
 * merged offsets.  E.g. a drained signal stream and its shot noise.
 * Synchronises. */
int neurosim_merge_events(const uint64_t *a_dev, const int64_t *seg_a, const uint64_t *b_dev, const int64_t *seg_b,
                          int32_t n_intervals, uint64_t *out_dev, int64_t *seg_out, void *cuda_stream);

/* Evaluates the library's FP32 log (the one the event model uses) on n DEVICE
 * floats x_dev into y_dev on cuda_stream; for verification of the log. */
int neurosim_debug_log(const float *x_dev, float *y_dev, int64_t n, void *cuda_stream);

/* One step of the event model that allocates nothing.  The paper has no
 * counterpart: this is a library convenience for callers that cannot call
 * cudaMalloc: real-time control loops that must never enter the device
 * allocator (an allocation can wait on a device-wide synchronisation), and
 * host programs that only borrow device buffers from another runtime and
 * have no allocator of their own.  The caller owns every buffer; the library keeps its intermediates (event
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
