// Internal declarations shared by the kernels (evsim_kernels.cu) and the C-ABI
// host code (evsim_api.cu) of libneurosim_evsim.so.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/neurosim_evsim.h"

namespace nsim {

constexpr uint32_t kTlastNone = 0xFFFFFFFFu;   // "no event yet" marker of t_last
constexpr uint32_t kNoChunk = 0xFFFFFFFFu;     // chunk not stored (page overflow)

// Bits of Ctl::err.
constexpr uint32_t kErrPageOverflow = 1u;   // intermediate key pages exhausted
constexpr uint32_t kErrOutOverflow = 2u;    // output record buffer exhausted
constexpr uint32_t kErrTimeout = 4u;        // a bounded mbarrier wait gave up

constexpr int kMaxTilesPerStream = 8192; // chunk prefix of one segment fits in shared memory
constexpr int kSortThreads = 512;
constexpr int kMaxDigitBits = 6;         // radix digit width of the segment sort

// Device control block of one simulator (or one batch).
struct Ctl {
    unsigned long long run_total;       // records written since the last drain (demand)
    unsigned long long out_demand_max;  // largest run_total seen (for regrowth)
    unsigned int page_ctr;              // key pages handed out in the current step
    unsigned int page_demand_max;       // largest page_ctr over the steps since reset
    unsigned int err;                   // kErr* bits
    unsigned int pad;
};

constexpr uint32_t kErrPendingOverflow = 8u;  // pending interval offsets exhausted (device clock)
constexpr uint32_t kErrTime = 16u;            // device clock left the 32-bit timestamp range

// Device-side clock of a batch whose steps run from captured CUDA graphs:
// everything that changes from one step to the next lives here, so that the
// same launches can be replayed.  Advanced by advance_kernel after a step
// that raised no error; a failed step sets `sticky`, and every later step
// does nothing until the host drains and clears it.
struct DevClock {
    long long tau;                        // time of the last frame consumed (us)
    long long pending_segs;               // interval offsets written since the last drain
    unsigned long long committed_total;   // records of committed steps since the last drain
    unsigned long long steps;             // committed steps
    unsigned int parity;                  // state buffer holding the current state
    unsigned int sticky;                  // kErr* bits of the failed step, 0 if none
};

// Constants of a procedural texture scene that every rendered pixel needs
// (scene_render.cuh).
struct SceneConst {
    uint32_t salt;
    int32_t octaves;
    float inv_period;      // 1 / base period (px)
    float gain;            // amplitude ratio of successive octaves
    float lo, span;        // intensity = lo + span * noise / sum of amplitudes
    int32_t n_rects;
    int32_t W;
};

// One sensor stream inside a step launch.
struct StreamDesc {
    const float* frames;          // [T][npix] FP32 (device)
    const float* ref_in;          // per-pixel state read at the start of the step
    const float* lprev_in;
    const uint32_t* tlast_in;
    float* ref_out;               // per-pixel state written at the end of the step
    float* lprev_out;
    uint32_t* tlast_out;
    const float* cpos;            // per-pixel thresholds, or nullptr for uniform
    const float* cneg;
    float cpos_u, cneg_u;         // uniform thresholds (used when maps are null)
    float log_eps;
    int32_t input_is_log;
    uint32_t refractory;          // us; 0 = off
    int32_t W, npix;
    int32_t n_tiles;              // work items (warp tiles of 32*ppt pixels) of this stream
    int32_t item_base;            // index of its first work item in the launch
    int32_t seg_base;             // index of its first segment in the launch
    int32_t n_segs;               // intervals this stream closes in the step
    int32_t init;                 // 1: frame 0 initialises the state
    int32_t vec;                  // 1: frames 16-byte aligned rows -> bulk copies
    int32_t pix_bits;             // bits of npix - 1 (>= 1)
    int32_t D0;                   // length of the first interval (us)
    int64_t ta0;                  // start time of the first interval (us)
    int64_t chunk_base;           // chunk-table offset of (segment 0, tile 0)
    int64_t out_seg_index;        // slot of segment 0 in the pending offset array
    int64_t frame_stride;         // floats from one frame to the next (0: npix)
    const void* scene_tab;        // per-frame SceneFrame table of a rendered step, or
                                  // nullptr: frames are read from `frames`
    SceneConst scene;             // constants of the rendered scene
};

// Everything one step launch needs (passed by value as a __grid_constant__).
struct StepLaunch {
    const StreamDesc* streams_dev;  // device array when n_streams > 1
    StreamDesc s0;                  // the stream when n_streams == 1
    int32_t n_streams;
    int32_t n_items;                // sum of n_tiles
    int32_t n_segs;                 // sum of n_segs
    int32_t T;                      // frames per stream in this step
    int32_t dt;                     // us
    int32_t key64;                  // 1: 64-bit intermediate keys
    int32_t t_bits;                 // bits of the largest in-interval offset
    int32_t ppt;                    // emission pixels per lane (8 or 16; warp tile 32*ppt)
    int32_t pf;                     // frames each lane keeps in flight (2 or 3)
    int32_t grid_emit;
    int32_t grid_sort;
    int32_t sort_smem;              // dynamic shared memory of the sort CTA
    int32_t max_tiles;              // largest n_tiles over the streams
    void* keys;                     // paged intermediate key buffer
    uint32_t n_pages, page_keys;
    void* temp;                     // sort scratch (same size as keys)
    uint2* chunks;                  // [segments][tiles] (offset, count)
    uint32_t* seg_count;            // [n_segs]
    int64_t* seg_rel;               // [n_segs] start relative to this step's first record
    int64_t* seg_abs;               // [n_segs] start in the output buffer
    int64_t* seg_off_out;           // pending per-interval offsets (for the drain)
    uint64_t* out;                  // output records
    uint64_t out_cap;
    Ctl* ctl;
    cudaStream_t stream;
    uint64_t wait_limit_ns;         // bound of every device-side wait
    DevClock* clock;                // device clock (batches), or nullptr: times,
                                    // parity and pending offsets come from the host
    int64_t max_pending;            // capacity of seg_off_out in intervals (device clock)
    int64_t tau_init;               // device clock: an init launch sets tau to this
    cudaEvent_t ev_begin;           // optional timing events (nullptr: none):
    cudaEvent_t ev_emitted;         //   before emission, after emission,
    cudaEvent_t ev_sorted;          //   after the interval sort
};

// Per-frame camera and occluder table of a texture scene (scene_render.cuh)
// for frames t0 + f dt, f < n_frames, into `tab` (device, n_frames rows of
// scene_frame_bytes()); and the renderer writing FP32 frames [n][H][W].
size_t scene_frame_bytes();
cudaError_t launch_scene_frames(const neurosim_texture_scene& sc, int64_t t0_us, int32_t dt_us, int n_frames,
                                void* tab, cudaStream_t stream);
SceneConst make_scene_const(const neurosim_texture_scene& sc);
int check_scene(const neurosim_texture_scene* s);   // NEUROSIM_OK or reports the bad field

// Enqueues emission, segment count, segment scan and segment sort (and, with
// a device clock, the clock advance); adds the number of kernels launched to
// *launches.  With a device clock, streams_dev holds two descriptor sets of
// n_streams entries: set `parity` reads the state from its *_in buffers.
cudaError_t launch_step(const StepLaunch& L, uint64_t* launches);

// Emission launch geometry helpers (CTA = 64/ppt warps).
int emit_warps_per_cta(int ppt);
size_t emit_smem_bytes(int ppt);
// src 0: frames read from memory; 1: frames rendered from a texture scene
cudaError_t emit_occupancy(int ppt, int pf, int key64, int* blocks_per_sm, int src = 0);
cudaError_t sort_configure(int* smem_bytes);

// Create-time per-pixel thresholds: C+-_u = max(c_min, C+- + sigma * z+-_u).
cudaError_t launch_threshold_maps(float* cpos, float* cneg, int64_t npix, float c_pos,
                                  float c_neg, float sigma, float c_min, uint64_t seed,
                                  cudaStream_t stream);

// L = log(clamp(I, 0, 1e6) + eps) with the library's log (the event model's L).
cudaError_t launch_log_intensity(const float* I, float* L, int64_t n, float eps, cudaStream_t stream);

// Debug/verification: y = library log(x).
cudaError_t launch_debug_log(const float* x, float* y, int64_t n, cudaStream_t stream);

// *dst = ctl->run_total (closing offset of the interval list), on `stream`.
cudaError_t launch_write_total(const Ctl* ctl, int64_t* dst, cudaStream_t stream);

// Sets the calling thread's neurosim_last_error() message; returns `code`.
int report_error(int code, const char* msg);

}  // namespace nsim
