// Procedural texture scene: per-frame camera/occluder tables and the
// stand-alone renderer (declared in include/neurosim_evsim.h as
// neurosim_render_texture).  The render-fused event step uses the same
// per-pixel function (scene_render.cuh) inside the emission kernel.
//
// The renderer is ALU-bound (four octaves of hashed value noise per pixel)
// and memory-light: it writes 4 B per pixel-frame and reads one 384-byte
// table row per frame.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"
#include "scene_render.cuh"

namespace nsim {
namespace {

// One thread per frame: camera and rectangles at t = t0 + f dt (seconds),
// evaluated in double, stored in FP32.
__global__ void scene_frames_kernel(const neurosim_texture_scene sc, int64_t t0_us, int32_t dt_us, int n_frames,
                                    SceneFrame* out)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_frames) return;
    const double t = (double)(t0_us + (int64_t)f * dt_us) * 1e-6;
    const double two_pi = 6.283185307179586476925286766559;
    // rotation angle: integral of the rate rot_amp sin(2 pi t / P + phase)
    const double k = two_pi / sc.rot_period_s;
    const double theta = sc.rot_amp_rad_s / k * (cos(sc.rot_phase) - cos(k * t + sc.rot_phase));
    const double z = 1.0 + sc.zoom_amp * sin(two_pi * t / sc.zoom_period_s + sc.zoom_phase);
    const double c = cos(theta), s = sin(theta);
    const double cx = 0.5 * sc.width, cy = 0.5 * sc.height;
    // texture point of pixel (x, y): R(theta) ((x, y) - centre) / z + centre + v t + offset
    const double A = c / z, B = -s / z, D = s / z, E = c / z;
    SceneFrame r;
    r.A = (float)A;
    r.B = (float)B;
    r.Cx = (float)(cx - A * cx - B * cy + sc.vx * t + sc.offset_x);
    r.D = (float)D;
    r.E = (float)E;
    r.Cy = (float)(cy - D * cx - E * cy + sc.vy * t + sc.offset_y);
    r.pad[0] = r.pad[1] = 0.0f;
    for (int i = 0; i < kMaxRects; ++i) {
        if (i < sc.n_rects) {
            // the rectangle wraps around a field one rectangle larger than the image
            const double mw = sc.width + sc.rect_w[i], mh = sc.height + sc.rect_h[i];
            double ax = sc.rect_x[i] + sc.rect_vx[i] * t, ay = sc.rect_y[i] + sc.rect_vy[i] * t;
            ax -= mw * floor(ax / mw);
            ay -= mh * floor(ay / mh);
            r.rect[i] = make_float4((float)(ax - 0.5 * sc.rect_w[i]), (float)(ay - 0.5 * sc.rect_h[i]),
                                    (float)(0.5 * sc.rect_w[i]), (float)(0.5 * sc.rect_h[i]));
            r.rval[i] = (float)sc.rect_value[i];
        } else {
            r.rect[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // covers nothing
            r.rval[i] = 0.0f;
        }
    }
    out[f] = r;
}

// Frames [n][H][W]: grid (pixel blocks, frames); each thread writes 4
// consecutive pixels of one frame (one 16-byte store when they are aligned).
__global__ void render_kernel(const SceneFrame* __restrict__ tab, SceneConst sc, int H, float* __restrict__ out,
                              int64_t npix, int vec)
{
    const int f = blockIdx.y;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (i >= npix) return;
    const SceneFrame& fr = tab[f];
    float xs[4], ys[4], v[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int64_t g = i + m;
        const int y = (int)(g / sc.W), x = (int)(g - (int64_t)y * sc.W);
        xs[m] = (float)x;
        ys[m] = (float)y;
    }
    texture_noise4(sc, fr, xs, ys, v);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        for (int k = 0; k < sc.n_rects; ++k)
            if (rect_covers(fr.rect[k], xs[m], ys[m])) v[m] = fr.rval[k];
        if (i + m >= npix) v[m] = 0.0f;
    }
    float* dst = out + (int64_t)f * npix + i;
    if (vec && i + 4 <= npix) {
        __stcs(reinterpret_cast<float4*>(dst), make_float4(v[0], v[1], v[2], v[3]));
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (i + m < npix) dst[m] = v[m];
    }
    (void)H;
}

}  // namespace

size_t scene_frame_bytes() { return sizeof(SceneFrame); }

SceneConst make_scene_const(const neurosim_texture_scene& sc)
{
    SceneConst k;
    k.salt = sc.salt;
    k.octaves = sc.octaves;
    k.inv_period = (float)(1.0 / sc.base_period);
    k.gain = sc.gain;
    k.lo = sc.intensity_lo;
    k.span = sc.intensity_hi - sc.intensity_lo;
    k.n_rects = sc.n_rects;
    k.W = sc.width;
    return k;
}

cudaError_t launch_scene_frames(const neurosim_texture_scene& sc, int64_t t0_us, int32_t dt_us, int n_frames,
                                void* tab, cudaStream_t stream)
{
    if (n_frames <= 0) return cudaSuccess;
    scene_frames_kernel<<<(n_frames + 127) / 128, 128, 0, stream>>>(sc, t0_us, dt_us, n_frames,
                                                                     static_cast<SceneFrame*>(tab));
    return cudaGetLastError();
}

// Checks a scene's fields; returns NEUROSIM_OK or reports the first bad one.
int check_scene(const neurosim_texture_scene* s)
{
    if (!s) return report_error(NEUROSIM_E_INVALID, "scene is NULL");
    if (s->width < 1 || s->height < 1 || s->width > 65535 || s->height > 32767 ||
        (int64_t)s->width * s->height > (1 << 22))
        return report_error(NEUROSIM_E_INVALID, "scene size out of range");
    if (s->octaves < 1 || s->octaves > 8) return report_error(NEUROSIM_E_INVALID, "octaves must be in [1, 8]");
    if (!(s->base_period >= 1.0f && s->base_period <= 65536.0f))
        return report_error(NEUROSIM_E_INVALID, "base_period must be in [1, 65536]");
    if (!(s->gain > 0.0f && s->gain <= 1.0f)) return report_error(NEUROSIM_E_INVALID, "gain must be in (0, 1]");
    if (!(s->intensity_lo >= 0.0f) || !(s->intensity_hi >= s->intensity_lo) || !(s->intensity_hi <= 1e6f))
        return report_error(NEUROSIM_E_INVALID, "need 0 <= intensity_lo <= intensity_hi <= 1e6");
    if (s->n_rects < 0 || s->n_rects > NEUROSIM_MAX_RECTS)
        return report_error(NEUROSIM_E_INVALID, "n_rects must be in [0, 16]");
    if (!(s->rot_period_s > 0.0) || !(s->zoom_period_s > 0.0) || !(std::fabs(s->zoom_amp) < 0.5))
        return report_error(NEUROSIM_E_INVALID, "periods must be > 0 and |zoom_amp| < 0.5");
    const double big = 1e7;
    const double vals[] = {s->vx, s->vy, s->offset_x, s->offset_y, s->rot_amp_rad_s, s->rot_phase, s->zoom_phase};
    for (double v : vals)
        if (!(std::fabs(v) < big)) return report_error(NEUROSIM_E_INVALID, "scene motion parameters out of range");
    for (int i = 0; i < s->n_rects; ++i) {
        if (!(s->rect_w[i] > 0.0 && s->rect_h[i] > 0.0 && s->rect_w[i] < big && s->rect_h[i] < big) ||
            !(std::fabs(s->rect_x[i]) < big && std::fabs(s->rect_y[i]) < big && std::fabs(s->rect_vx[i]) < big &&
              std::fabs(s->rect_vy[i]) < big) ||
            !(s->rect_value[i] >= 0.0 && s->rect_value[i] <= 1e6))
            return report_error(NEUROSIM_E_INVALID, "rectangle out of range");
    }
    return NEUROSIM_OK;
}

}  // namespace nsim

extern "C" int neurosim_render_texture(const neurosim_texture_scene* scene, float* frames_dev, int32_t n_frames,
                                       int64_t t0_us, int32_t dt_us, void* cuda_stream)
{
    using namespace nsim;
    int rc = check_scene(scene);
    if (rc) return rc;
    if (n_frames < 0 || n_frames > 65535) return report_error(NEUROSIM_E_INVALID, "n_frames must be in [0, 65535]");
    if (n_frames == 0) return NEUROSIM_OK;
    if (!frames_dev) return report_error(NEUROSIM_E_INVALID, "frames_dev is NULL");
    if (t0_us < 0 || dt_us < 1) return report_error(NEUROSIM_E_TIME, "need t0_us >= 0 and dt_us >= 1");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    void* tab = nullptr;
    if (cudaMallocAsync(&tab, (size_t)n_frames * sizeof(SceneFrame), st) != cudaSuccess)
        return report_error(NEUROSIM_E_NOMEM, "cannot allocate the scene table");
    cudaError_t e = launch_scene_frames(*scene, t0_us, dt_us, n_frames, tab, st);
    const int64_t npix = (int64_t)scene->width * scene->height;
    const int vec = (npix % 4 == 0 && (reinterpret_cast<uintptr_t>(frames_dev) & 15u) == 0) ? 1 : 0;
    if (e == cudaSuccess) {
        const int threads = 256;
        const int64_t bx = (npix + 4 * threads - 1) / (4 * threads);
        render_kernel<<<dim3((unsigned)bx, (unsigned)n_frames), threads, 0, st>>>(
            static_cast<const SceneFrame*>(tab), make_scene_const(*scene), scene->height, frames_dev, npix, vec);
        e = cudaGetLastError();
    }
    cudaFreeAsync(tab, st);
    if (e != cudaSuccess) return report_error(NEUROSIM_E_CUDA, "render launch failed");
    return NEUROSIM_OK;
}
