// Autotuner of the emission launch shape (declared in include/neurosim_evsim.h
// as neurosim_evsim_autotune).  Every variant computes the same events; the
// tuner only times them on the caller's frames and keeps the fastest, with a
// per-GPU JSON-lines cache so that the sweep runs once per workload shape.
// The paper has no counterpart: its kernel fixes one thread per pixel.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"

namespace {

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return nsim::report_error(code, buf);
}

struct Variant {
    int ppt, ctas;     // pixels per lane (warp tile 32 * ppt) and emission CTAs per SM
};

// The launch shapes to time: both warp tiles, each with 1 up to as many
// CTAs per SM as fit (the occupancy of the kernel with 32-bit keys).
int variants(std::vector<Variant>* out)
{
    out->clear();
    for (int ppt : {8, 16}) {
        int bps = 0;
        if (nsim::emit_occupancy(ppt, 2, 0, &bps) != cudaSuccess || bps < 1) return NEUROSIM_E_CUDA;
        for (int c = 1; c <= bps; ++c) out->push_back(Variant{ppt, c});
    }
    return NEUROSIM_OK;
}

// Value of "key": in one JSON line (number or string); false if absent.
bool json_field(const std::string& line, const char* key, std::string* out)
{
    const std::string pat = std::string("\"") + key + "\":";
    size_t i = line.find(pat);
    if (i == std::string::npos) return false;
    i += pat.size();
    while (i < line.size() && line[i] == ' ') ++i;
    if (i < line.size() && line[i] == '"') {
        const size_t j = line.find('"', i + 1);
        if (j == std::string::npos) return false;
        *out = line.substr(i + 1, j - i - 1);
        return true;
    }
    size_t j = i;
    while (j < line.size() && line[j] != ',' && line[j] != '}') ++j;
    *out = line.substr(i, j - i);
    return true;
}

bool cache_lookup(const char* path, const std::string& gpu, int W, int H, int T, int* ppt, int* ctas, double* ms)
{
    FILE* f = fopen(path, "r");
    if (!f) return false;
    bool found = false;
    std::vector<char> buf(1 << 16);
    while (fgets(buf.data(), (int)buf.size(), f)) {
        const std::string line(buf.data());
        std::string g, w, h, t, p, c, m;
        if (!json_field(line, "gpu", &g) || !json_field(line, "width", &w) || !json_field(line, "height", &h) ||
            !json_field(line, "frames", &t) || !json_field(line, "pixels_per_thread", &p) ||
            !json_field(line, "ctas_per_sm", &c))
            continue;
        if (g != gpu || atoi(w.c_str()) != W || atoi(h.c_str()) != H || atoi(t.c_str()) != T) continue;
        const int pv = atoi(p.c_str()), cv = atoi(c.c_str());
        if ((pv != 8 && pv != 16) || cv < 1 || cv > 64) continue;
        *ppt = pv;
        *ctas = cv;
        *ms = json_field(line, "ms", &m) ? atof(m.c_str()) : 0.0;
        found = true;   // the last matching line wins
    }
    fclose(f);
    return found;
}

// Median emission + sort time of `repeats` steps of one variant.
int time_variant(const neurosim_evsim_params* p, const float* frames, int T, int dt, int repeats, cudaStream_t st,
                 uint64_t** buf, uint64_t* buf_cap, double* median_ms)
{
    neurosim_evsim* h = nullptr;
    int rc = neurosim_evsim_create(p, st, &h);
    if (rc) return rc;
    std::vector<double> ms;
    const int64_t span = (int64_t)T * dt;
    for (int k = 0; k <= repeats && rc == 0; ++k) {
        if (k == 1) rc = neurosim_evsim_set_profiling(h, 1);
        neurosim_evsim_stats s0{}, s1{};
        if (!rc && k > 0) rc = neurosim_evsim_get_stats(h, &s0);
        if (!rc) rc = neurosim_evsim_step(h, frames, T, (int64_t)k * span, dt);
        uint64_t n_ev = 0;
        int64_t n_seg = 0;
        if (!rc) rc = neurosim_evsim_pending(h, &n_ev, &n_seg);
        if (!rc && std::max<uint64_t>(n_ev, 1) > *buf_cap) {
            if (*buf) cudaFree(*buf);
            *buf = nullptr;
            *buf_cap = 0;
            n_ev = std::max<uint64_t>(n_ev, 1);
            if (cudaMalloc(reinterpret_cast<void**>(buf), n_ev * sizeof(uint64_t)) != cudaSuccess) {
                rc = fail(NEUROSIM_E_NOMEM, "autotune: no device memory for %llu events", (unsigned long long)n_ev);
                break;
            }
            *buf_cap = n_ev;
        }
        uint64_t n_out = 0;
        if (!rc) rc = neurosim_evsim_drain_events(h, *buf, *buf_cap, 1, &n_out, nullptr, 0, nullptr);
        if (!rc && k > 0) {
            rc = neurosim_evsim_get_stats(h, &s1);
            if (!rc) ms.push_back((s1.emit_ms - s0.emit_ms) + (s1.sort_ms - s0.sort_ms));
        }
    }
    neurosim_evsim_destroy(h);
    if (rc) return rc;
    std::sort(ms.begin(), ms.end());
    *median_ms = ms[ms.size() / 2];
    return NEUROSIM_OK;
}

}  // namespace

extern "C" int neurosim_evsim_autotune(const neurosim_evsim_params* p, const float* frames_dev, int32_t n_frames,
                                       int32_t dt_us, int32_t repeats, const char* cache_path,
                                       int32_t* pixels_per_thread, int32_t* ctas_per_sm, double* ms_out)
{
    if (!p || !frames_dev || !pixels_per_thread || !ctas_per_sm)
        return fail(NEUROSIM_E_INVALID, "params, frames_dev and the outputs must not be NULL");
    if (n_frames < 2) return fail(NEUROSIM_E_INVALID, "n_frames must be >= 2");
    if (repeats < 1 || repeats > 100) return fail(NEUROSIM_E_INVALID, "repeats must be in [1, 100]");
    if (dt_us < 1 || dt_us >= (1 << 24)) return fail(NEUROSIM_E_TIME, "dt_us must be in [1, 2^24)");
    if ((int64_t)(repeats + 1) * n_frames * dt_us > 0xFFFFFFFEll)
        return fail(NEUROSIM_E_TIME, "repeats * n_frames * dt_us exceeds the 32-bit timestamp range");
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return fail(NEUROSIM_E_CUDA, "no CUDA device");
    const std::string gpu(prop.name);
    double best_ms = 0.0;
    int best_ppt = 0, best_ctas = 0;
    if (cache_path && cache_lookup(cache_path, gpu, p->width, p->height, n_frames, &best_ppt, &best_ctas, &best_ms)) {
        *pixels_per_thread = best_ppt;
        *ctas_per_sm = best_ctas;
        if (ms_out) *ms_out = best_ms;
        return NEUROSIM_OK;
    }
    std::vector<Variant> vs;
    if (variants(&vs) != NEUROSIM_OK) return fail(NEUROSIM_E_CUDA, "cannot query the emission kernel's occupancy");
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return fail(NEUROSIM_E_CUDA, "cannot create a stream");
    uint64_t* buf = nullptr;
    uint64_t cap = 0;
    int rc = NEUROSIM_OK;
    std::string timings;
    for (const Variant& v : vs) {
        neurosim_evsim_params q = *p;
        q.pixels_per_thread = v.ppt;
        q.prefetch_frames = 0;
        q.ctas_per_sm = v.ctas;
        q.max_frames_per_step = std::max(q.max_frames_per_step, n_frames);
        double ms = 0.0;
        rc = time_variant(&q, frames_dev, n_frames, dt_us, repeats, st, &buf, &cap, &ms);
        if (rc) break;
        char item[64];
        snprintf(item, sizeof item, "%s[%d, %d, %.4f]", timings.empty() ? "" : ", ", v.ppt, v.ctas, ms);
        timings += item;
        if (best_ppt == 0 || ms < best_ms) {
            best_ms = ms;
            best_ppt = v.ppt;
            best_ctas = v.ctas;
        }
    }
    if (buf) cudaFree(buf);
    cudaStreamDestroy(st);
    if (rc) return rc;
    *pixels_per_thread = best_ppt;
    *ctas_per_sm = best_ctas;
    if (ms_out) *ms_out = best_ms;
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (f) {
            fprintf(f,
                    "{\"gpu\": \"%s\", \"width\": %d, \"height\": %d, \"frames\": %d, \"pixels_per_thread\": %d, "
                    "\"ctas_per_sm\": %d, \"ms\": %.4f, \"timings\": [%s]}\n",
                    gpu.c_str(), p->width, p->height, n_frames, best_ppt, best_ctas, best_ms, timings.c_str());
            fclose(f);
        }
    }
    return NEUROSIM_OK;
}
