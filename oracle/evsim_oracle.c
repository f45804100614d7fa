/*
 * Oracle for the Neurosim event-generation path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded CPU
 * restatement of the event model, written to check the CUDA library against.
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant
 * generator with the CUDA path, and the CUDA path never calls it.
 *
 * Paper: "Neurosim: A Fast Simulator for Neuromorphic Robot Perception",
 * arXiv 2602.15018.
 *   - Sec. 1: an event is a tuple (t, u, p) with an integer timestamp in
 *     microseconds, an integer pixel u and a polarity p in {-1, +1}.
 *   - Sec. 2, paragraph "Neurosim simulates event cameras at multi-kilohertz
 *     rates": each pixel keeps the intensity level of its last triggered
 *     event; an event fires when the change from that level passes a
 *     contrast threshold (the contrast-threshold model of the cited ESIM);
 *     noise is among the non-idealities the user may switch off; each
 *     rendering step yields a variable number of events.
 * The paper gives the model in prose only.  Every reading of a silent point
 * taken here is listed in the "Readings" block below and is the same reading
 * the CUDA path implements.
 *
 * Readings (the paper is silent on all of these; R9-R12 concern the step
 * interface, consumers, batches and the learned interpolator, which this
 * file does not hold):
 *   R1  L = log(clamp(I, 0, 1e6) + eps) in FP32 with the project's own log
 *       (oracle_mylog below); with input_is_log the frame already holds L and
 *       is clamped to [-32, 32].  NaN intensities clamp to 0 (or to -32 in the
 *       log domain).
 *   R2  Log intensity is linear in time between consecutive frames (ESIM).
 *   R3  Crossings are taken one threshold at a time with sequential FP32
 *       adds: ON while fl(ref + C+) <= b, OFF while fl(ref - C-) >= b, and on
 *       each crossing ref moves to the crossed level (not to b).
 *   R4  Crossing time t = ta + floor(frac * D) with frac = (lvl - a)/(b - a)
 *       in FP32 and D = tb - ta in integer microseconds, so t lies in
 *       [ta, tb].  A negative t - ta (only reachable from an imported state
 *       that breaks the reference-band invariant) is clamped to 0.
 *   R5  Refractory period R: a crossing with t - t_last < R is suppressed;
 *       ref still moves, t_last keeps the last emitted time.
 *   R6  Per-pixel thresholds C+-_u = max(c_min, C+- + sigma * z+-_u), drawn
 *       once.  z is an Irwin-Hall(12) normal (sum of twelve 20-bit uniforms
 *       minus 6) from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as
 *       a counter-based generator: draw k of pixel u and polarity q is output
 *       number ((2u + q) * 12 + k) of the SplitMix64 stream seeded with seed.
 *   R7  The first frame a sensor ever sees sets ref = L_prev = L and emits
 *       nothing.
 *   R8  Output order: interval-major; inside one interval ascending by the
 *       packed record (t, y, x, p), OFF (p = 0) before ON (p = 1).
 *   R13 Sensor bandwidth (Sec. 2 names "bandwidth limitations" among the
 *       non-idealities, with no model): a first-order low-pass filter on
 *       each pixel's log intensity, one update per frame, applied before the
 *       event model: s_k = s_{k-1} + alpha (L_k - s_{k-1}) with
 *       alpha = 1 - exp(-2 pi f_c dt) for a cutoff f_c (in double, rounded
 *       once to FP32: oracle_lowpass_alpha); the filter starts at the first
 *       frame's value.  FP32: d = L - s rounded, then s = fma(alpha, d, s)
 *       with one rounding (oracle_lowpass_log below).
 *   R14 Sensor leak (Sec. 2 lists noise among the modelled non-idealities,
 *       with no model; junction leakage makes a pixel's reference level
 *       drift): the reference drifts down at C+_u * r per second, which for
 *       the crossing test L - ref is the same as the log intensity rising by
 *       delta(t) = C+_u * r * (t - origin).  Applied to log frames before the
 *       event model: L' = L + delta(t_k), FP32 as
 *       fl(L + fl(fl(C+_u * fl(r * 1e-6)) * (float)(t_k - origin))), with
 *       t in microseconds (oracle_leak_log below).  A still pixel then fires
 *       ON events r times a second.
 *   R15 Shot noise (same paragraph): spurious events independent of the
 *       signal and of the pixel state.  For every tile of 64 consecutive
 *       pixels (row-major; the last may be shorter, `len` pixels) and every
 *       interval (start ta, length D us), the count is Poisson with mean
 *       lambda = r * len * D * 1e-6, drawn by inversion: with the 53-bit
 *       uniform U of SplitMix64 output ((ta * n_tiles + tile) * 32) of the
 *       noise seed, the count is the least n with U < floor(F(n) * 2^53),
 *       F the Poisson CDF accumulated in double from exp(-lambda), at most
 *       15 (the mean is kept at most 4, where more than 15 has probability
 *       below 1e-6).  Event i uses outputs base + 1 + 2i (pixel tile * 64 +
 *       floor(hi32 * len / 2^32), time ta + floor(lo32 * D / 2^32)) and
 *       base + 2 + 2i (polarity: its top bit).  Merged into a stream
 *       interval by interval in the order of R8 (oracle_shot_noise,
 *       oracle_merge_events).
 *
 * Packed record (64 bits): [63:32] t (us) | [31:17] y | [16:1] x | [0] p.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared.
 * Contraction must stay off: the FP32 variant mirrors the operation order of
 * the model exactly so that its events are reproducible bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_E_INVALID 1
#define ORACLE_E_NOMEM 2
#define ORACLE_E_TIME 3

#define LOG_DOMAIN_MAX 32.0f
#define INTENSITY_MAX 1.0e6f
#define TLAST_NONE (-1)

static uint32_t f2u(float x) { uint32_t u; memcpy(&u, &x, 4); return u; }
static float u2f(uint32_t u) { float x; memcpy(&x, &u, 4); return x; }

/* ------------------------------------------------------------------------ */
/* The project's own single-precision natural log (reading R1).             */
/*                                                                          */
/* Textbook method: x = m * 2^e with m in [sqrt(1/2), sqrt(2)); with        */
/* s = (m - 1)/(m + 1), log m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + s^7/7    */
/* + s^9/9 + ...), truncated after s^9 (|s| < 0.1716 so the next term is    */
/* below 1e-9 relative); log x = log m + e ln2 with ln2 split into a 16-bit */
/* head (so that e * head is exact) and a tail.  Every operation is one     */
/* IEEE-rounded FP32 operation in the order written.                        */
/* ------------------------------------------------------------------------ */
static const float C_INV3 = 0x1.555556p-2f;   /* 1/3 rounded to FP32 */
static const float C_INV5 = 0x1.99999ap-3f;   /* 1/5 */
static const float C_INV7 = 0x1.24924ap-3f;   /* 1/7 */
static const float C_INV9 = 0x1.c71c72p-4f;   /* 1/9 */
static const float C_LN2_HI = 0x1.62e4p-1f;   /* round(ln2 * 2^16) / 2^16 */
static const float C_LN2_LO = 0x1.7f7d1cp-20f; /* ln2 - C_LN2_HI, rounded */
static const float C_SQRT2 = 0x1.6a09e6p+0f;  /* sqrt(2) rounded */

float oracle_mylog(float x)
{
    if (x != x) return x;                 /* NaN */
    if (x < 0.0f) return NAN;
    if (x == 0.0f) return -INFINITY;
    if (x == INFINITY) return INFINITY;
    int e = 0;
    uint32_t bits = f2u(x);
    if (bits < 0x00800000u) {             /* subnormal: scale by 2^24 (exact) */
        x = x * 0x1p24f;
        bits = f2u(x);
        e = -24;
    }
    e += (int)(bits >> 23) - 127;
    float m = u2f((bits & 0x007fffffu) | 0x3f800000u);   /* [1, 2) */
    if (m > C_SQRT2) {
        m = m * 0.5f;
        e += 1;
    }
    float num = m - 1.0f;
    float den = m + 1.0f;
    float s = num / den;
    float z = s * s;
    float q = fmaf(z, C_INV9, C_INV7);
    q = fmaf(z, q, C_INV5);
    q = fmaf(z, q, C_INV3);
    float s2 = s + s;
    float zq = z * q;
    float lm = fmaf(s2, zq, s2);
    float fe = (float)e;
    float tail = fmaf(fe, C_LN2_LO, lm);
    return fmaf(fe, C_LN2_HI, tail);
}

void oracle_mylog_batch(const float *x, float *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = oracle_mylog(x[i]);
}

/* Distance in units in the last place between a float and a double
 * reference, measured on the FP32 grid around the reference. */
static double ulp_err(float got, double ref)
{
    if (isinf(ref) || isnan(ref)) return (got == (float)ref) ? 0.0 : INFINITY;
    double a = fabs(ref);
    int ex;
    frexp(a, &ex);                 /* a = f * 2^ex, f in [0.5, 1) */
    double ulp = ldexp(1.0, ex - 24);
    if (ulp < 0x1p-149) ulp = 0x1p-149;
    return fabs((double)got - ref) / ulp;
}

/* Scans every FP32 value with bit pattern in [lo_bits, hi_bits] (positive
 * floats only) and reports the largest error of oracle_mylog against the
 * double-precision libm log, in FP32 ulps. */
double oracle_mylog_max_ulp(uint32_t lo_bits, uint32_t hi_bits, uint32_t stride,
                            uint32_t *worst_bits)
{
    double worst = 0.0;
    uint32_t wb = lo_bits;
    if (stride == 0) stride = 1;
    for (uint64_t b = lo_bits; b <= hi_bits; b += stride) {
        float x = u2f((uint32_t)b);
        double e = ulp_err(oracle_mylog(x), log((double)x));
        if (e > worst) { worst = e; wb = (uint32_t)b; }
    }
    if (worst_bits) *worst_bits = wb;
    return worst;
}

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood 2014): state += 0x9e3779b97f4a7c15, then  */
/* the output is the state passed through the variant-13 mixer.  Output     */
/* number i (0-based) of the stream seeded with s therefore only depends on */
/* s + (i + 1) * gamma, which makes it usable as a counter-based generator. */
/* ------------------------------------------------------------------------ */
uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t index)
{
    uint64_t z = seed + (index + 1u) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* Irwin-Hall(12) standard normal draw number `slot` (reading R6): the sum of
 * twelve uniforms on {0..2^20-1}, minus 6 * 2^20, scaled by 2^-20.  The sum is
 * below 2^24 so the FP32 result is exact. */
float oracle_normal_ih12(uint64_t seed, uint64_t slot)
{
    int64_t acc = 0;
    for (int k = 0; k < 12; ++k)
        acc += (int64_t)(oracle_splitmix64_at(seed, slot * 12u + (uint64_t)k) >> 44);
    int64_t centred = acc - 6 * (int64_t)(1 << 20);
    return (float)centred * 0x1p-20f;
}

/* Per-pixel thresholds (reading R6): C+-_u = max(c_min, C+- + sigma * z+-_u)
 * with one FP32 multiply and one FP32 add. */
void oracle_threshold_maps(int32_t width, int32_t height, float c_pos, float c_neg,
                           float sigma, float c_min, uint64_t seed,
                           float *cpos_out, float *cneg_out)
{
    int64_t n = (int64_t)width * height;
    for (int64_t u = 0; u < n; ++u) {
        float vp = c_pos, vn = c_neg;
        if (sigma != 0.0f) {
            float zp = oracle_normal_ih12(seed, (uint64_t)u * 2u + 0u);
            float zn = oracle_normal_ih12(seed, (uint64_t)u * 2u + 1u);
            float dp = sigma * zp;
            float dn = sigma * zn;
            vp = c_pos + dp;
            vn = c_neg + dn;
        }
        cpos_out[u] = fmaxf(c_min, vp);
        cneg_out[u] = fmaxf(c_min, vn);
    }
}

/* ------------------------------------------------------------------------ */
/* Event buffer                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t *ev;
    int64_t n, cap;
    int64_t *seg;       /* interval offsets, n_seg + 1 entries */
    int32_t n_seg, seg_cap;
    int failed;
} evbuf;

static void eb_push(evbuf *b, uint64_t rec)
{
    if (b->failed) return;
    if (b->n == b->cap) {
        int64_t nc = b->cap ? b->cap * 2 : 4096;
        uint64_t *p = (uint64_t *)realloc(b->ev, (size_t)nc * sizeof(uint64_t));
        if (!p) { b->failed = 1; return; }
        b->ev = p;
        b->cap = nc;
    }
    b->ev[b->n++] = rec;
}

static void eb_close_segment(evbuf *b)
{
    if (b->failed) return;
    if (b->n_seg + 2 > b->seg_cap) {
        int32_t nc = b->seg_cap ? b->seg_cap * 2 : 256;
        int64_t *p = (int64_t *)realloc(b->seg, (size_t)nc * sizeof(int64_t));
        if (!p) { b->failed = 1; return; }
        b->seg = p;
        b->seg_cap = nc;
    }
    if (b->n_seg == 0) b->seg[0] = 0;
    b->seg[++b->n_seg] = b->n;
}

static int cmp_u64(const void *pa, const void *pb)
{
    uint64_t a = *(const uint64_t *)pa, b = *(const uint64_t *)pb;
    return (a > b) - (a < b);
}

static uint64_t pack(int64_t t, int32_t x, int32_t y, int on)
{
    return ((uint64_t)(uint32_t)t << 32) | ((uint64_t)(uint32_t)y << 17) |
           ((uint64_t)(uint32_t)x << 1) | (uint64_t)(on ? 1u : 0u);
}

static int check_args(int32_t W, int32_t H, int32_t T, int64_t t0, int32_t dt,
                      int has_prev, int64_t tau_prev)
{
    if (W <= 0 || H <= 0 || W > 65535 || H > 32767 || T < 0) return ORACLE_E_INVALID;
    if (dt <= 0 || dt >= (1 << 24) || t0 < 0) return ORACLE_E_TIME;
    if (T == 0) return ORACLE_OK;
    int64_t last = t0 + (int64_t)(T - 1) * dt;
    if (last > 0xFFFFFFFEll) return ORACLE_E_TIME;
    if (has_prev && (t0 <= tau_prev || t0 - tau_prev >= (1 << 24))) return ORACLE_E_TIME;
    return ORACLE_OK;
}

static void finish(evbuf *b, uint64_t **events_out, int64_t *n_events_out,
                   int64_t **seg_out, int32_t *n_seg_out)
{
    if (b->n_seg == 0) {                 /* always hand back seg[0] = 0 */
        b->seg = (int64_t *)malloc(sizeof(int64_t));
        if (b->seg) b->seg[0] = 0;
    }
    *events_out = b->ev;
    *n_events_out = b->n;
    *seg_out = b->seg;
    *n_seg_out = b->n_seg;
}

/* ------------------------------------------------------------------------ */
/* One step of the event model, FP32 mirrored (readings R1-R8).             */
/*                                                                          */
/* frames: T frames of H x W row-major FP32 intensities (or log intensities */
/* when input_is_log).  Frame f is at time t0 + f * dt.  State arrays are   */
/* read and updated in place.  tlast holds -1 for "no event yet".           */
/* On return *events_out holds the step's records in output order and       */
/* *seg_out the n_seg + 1 interval offsets; release both with oracle_free.  */
/* ------------------------------------------------------------------------ */
int oracle_evsim_step_f32(int32_t W, int32_t H, const float *frames, int32_t T,
                          int64_t t0, int32_t dt, const float *cpos, const float *cneg,
                          uint32_t refractory_us, float log_eps, int32_t input_is_log,
                          float *ref, float *lprev, int64_t *tlast, int32_t *has_prev,
                          int64_t *tau_prev, uint64_t **events_out, int64_t *n_events_out,
                          int64_t **seg_out, int32_t *n_seg_out)
{
    int rc = check_args(W, H, T, t0, dt, *has_prev, *tau_prev);
    if (rc != ORACLE_OK) return rc;
    const int64_t npix = (int64_t)W * H;
    evbuf b;
    memset(&b, 0, sizeof b);

    for (int32_t f = 0; f < T; ++f) {
        const float *fr = frames + (int64_t)f * npix;
        const int64_t tb = t0 + (int64_t)f * dt;
        if (!*has_prev) {                                   /* R7 */
            for (int64_t u = 0; u < npix; ++u) {
                float L;
                if (input_is_log) L = fminf(fmaxf(fr[u], -LOG_DOMAIN_MAX), LOG_DOMAIN_MAX);
                else L = oracle_mylog(fminf(fmaxf(fr[u], 0.0f), INTENSITY_MAX) + log_eps);
                ref[u] = L;
                lprev[u] = L;
                tlast[u] = TLAST_NONE;
            }
            *has_prev = 1;
            *tau_prev = tb;
            continue;
        }
        const int64_t ta = *tau_prev;
        const int64_t D = tb - ta;
        const float Df = (float)D;
        const int64_t seg_start = b.n;
        for (int64_t u = 0; u < npix; ++u) {
            const int32_t y = (int32_t)(u / W), x = (int32_t)(u % W);
            float L;
            if (input_is_log) L = fminf(fmaxf(fr[u], -LOG_DOMAIN_MAX), LOG_DOMAIN_MAX);
            else L = oracle_mylog(fminf(fmaxf(fr[u], 0.0f), INTENSITY_MAX) + log_eps);
            const float a = lprev[u];
            const float bb = L;
            float r = ref[u];
            int64_t tl = tlast[u];
            if (bb > a) {
                const float den = bb - a;
                for (;;) {                                   /* R3 (ON) */
                    const float lvl = r + cpos[u];
                    if (!(lvl <= bb)) break;
                    const float num = lvl - a;
                    const float frac = num / den;
                    float tf = floorf(frac * Df);            /* R4 */
                    if (tf < 0.0f) tf = 0.0f;
                    const int64_t t = ta + (int64_t)tf;
                    r = lvl;
                    if (refractory_us != 0 && tl != TLAST_NONE && t - tl < (int64_t)refractory_us)
                        continue;                            /* R5 */
                    eb_push(&b, pack(t, x, y, 1));
                    tl = t;
                }
            } else if (bb < a) {
                const float den = bb - a;
                for (;;) {                                   /* R3 (OFF) */
                    const float lvl = r - cneg[u];
                    if (!(lvl >= bb)) break;
                    const float num = lvl - a;
                    const float frac = num / den;
                    float tf = floorf(frac * Df);
                    if (tf < 0.0f) tf = 0.0f;
                    const int64_t t = ta + (int64_t)tf;
                    r = lvl;
                    if (refractory_us != 0 && tl != TLAST_NONE && t - tl < (int64_t)refractory_us)
                        continue;
                    eb_push(&b, pack(t, x, y, 0));
                    tl = t;
                }
            }
            ref[u] = r;
            tlast[u] = tl;
            lprev[u] = bb;
        }
        if (!b.failed && b.n > seg_start)                   /* R8 */
            qsort(b.ev + seg_start, (size_t)(b.n - seg_start), sizeof(uint64_t), cmp_u64);
        eb_close_segment(&b);
        *tau_prev = tb;
    }
    if (b.failed) {
        free(b.ev);
        free(b.seg);
        return ORACLE_E_NOMEM;
    }
    finish(&b, events_out, n_events_out, seg_out, n_seg_out);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* The same model in FP64 with the libm log: the precision reference that    */
/* the FP32 path is compared against (at most 1e-4 of events differ, times  */
/* within 1 us).  Thresholds come in as the same FP32 maps.                 */
/* ------------------------------------------------------------------------ */
int oracle_evsim_step_f64(int32_t W, int32_t H, const float *frames, int32_t T,
                          int64_t t0, int32_t dt, const float *cpos, const float *cneg,
                          uint32_t refractory_us, double log_eps, int32_t input_is_log,
                          double *ref, double *lprev, int64_t *tlast, int32_t *has_prev,
                          int64_t *tau_prev, uint64_t **events_out, int64_t *n_events_out,
                          int64_t **seg_out, int32_t *n_seg_out)
{
    int rc = check_args(W, H, T, t0, dt, *has_prev, *tau_prev);
    if (rc != ORACLE_OK) return rc;
    const int64_t npix = (int64_t)W * H;
    evbuf b;
    memset(&b, 0, sizeof b);

    for (int32_t f = 0; f < T; ++f) {
        const float *fr = frames + (int64_t)f * npix;
        const int64_t tb = t0 + (int64_t)f * dt;
        if (!*has_prev) {
            for (int64_t u = 0; u < npix; ++u) {
                double L;
                if (input_is_log) L = fmin(fmax((double)fr[u], -32.0), 32.0);
                else L = log(fmin(fmax((double)fr[u], 0.0), 1.0e6) + log_eps);
                ref[u] = L;
                lprev[u] = L;
                tlast[u] = TLAST_NONE;
            }
            *has_prev = 1;
            *tau_prev = tb;
            continue;
        }
        const int64_t ta = *tau_prev;
        const double D = (double)(tb - ta);
        const int64_t seg_start = b.n;
        for (int64_t u = 0; u < npix; ++u) {
            const int32_t y = (int32_t)(u / W), x = (int32_t)(u % W);
            double L;
            if (input_is_log) L = fmin(fmax((double)fr[u], -32.0), 32.0);
            else L = log(fmin(fmax((double)fr[u], 0.0), 1.0e6) + log_eps);
            const double a = lprev[u], bb = L;
            double r = ref[u];
            int64_t tl = tlast[u];
            const int on = bb > a;
            if (bb != a) {
                const double c = on ? (double)cpos[u] : -(double)cneg[u];
                for (;;) {
                    const double lvl = r + c;
                    if (on ? !(lvl <= bb) : !(lvl >= bb)) break;
                    double tf = floor((lvl - a) / (bb - a) * D);
                    if (tf < 0.0) tf = 0.0;
                    const int64_t t = ta + (int64_t)tf;
                    r = lvl;
                    if (refractory_us != 0 && tl != TLAST_NONE && t - tl < (int64_t)refractory_us)
                        continue;
                    eb_push(&b, pack(t, x, y, on));
                    tl = t;
                }
            }
            ref[u] = r;
            tlast[u] = tl;
            lprev[u] = bb;
        }
        if (!b.failed && b.n > seg_start)
            qsort(b.ev + seg_start, (size_t)(b.n - seg_start), sizeof(uint64_t), cmp_u64);
        eb_close_segment(&b);
        *tau_prev = tb;
    }
    if (b.failed) {
        free(b.ev);
        free(b.seg);
        return ORACLE_E_NOMEM;
    }
    finish(&b, events_out, n_events_out, seg_out, n_seg_out);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Sensor bandwidth filter (reading R13).  L, out: [T][n] FP32 (out may be L); */
/* state: [n], read unless init (then set to frame 0) and written back.       */
/* ------------------------------------------------------------------------ */
int oracle_lowpass_log(const float *L, float *out, int32_t T, int64_t n, float alpha, float *state, int32_t init)
{
    if (T < 0 || n < 0 || !(alpha > 0.0f && alpha <= 1.0f) || (init && T == 0)) return ORACLE_E_INVALID;
    for (int64_t i = 0; i < n; ++i) {
        float s = init ? L[i] : state[i];
        for (int32_t k = 0; k < T; ++k) {
            const float d = L[(int64_t)k * n + i] - s;
            s = fmaf(alpha, d, s);
            out[(int64_t)k * n + i] = s;
        }
        state[i] = s;
    }
    return ORACLE_OK;
}

/* Per-frame gain of the bandwidth filter (reading R13): the first-order     */
/* filter with cutoff f_c, time constant 1 / (2 pi f_c), sampled every dt,   */
/* keeps exp(-2 pi f_c dt) of the old level: alpha = 1 - exp(-2 pi f_c dt),   */
/* evaluated in double and rounded once to FP32.  dt_us in microseconds.     */
/* Returns 0 for arguments outside f_c > 0, dt_us >= 1 or a gain that rounds */
/* to zero.                                                                  */
float oracle_lowpass_alpha(double cutoff_hz, int32_t dt_us)
{
    const double two_pi = 6.283185307179586476925286766559;
    if (!(cutoff_hz > 0.0) || !isfinite(cutoff_hz) || dt_us < 1) return 0.0f;
    const double keep = exp(-two_pi * cutoff_hz * ((double)dt_us * 1e-6));
    return (float)(1.0 - keep);
}

/* ------------------------------------------------------------------------ */
/* Sensor leak (reading R14).  L, out: [T][n] FP32 log frames at t0 + k dt  */
/* (out may be L); cpos: per-pixel ON thresholds [n] or NULL for cpos_u.    */
/* ------------------------------------------------------------------------ */
int oracle_leak_log(const float *L, float *out, int32_t T, int64_t n, int64_t t0_us, int32_t dt_us,
                    int64_t origin_us, double rate_hz, const float *cpos, float cpos_u)
{
    if (T < 0 || n < 0 || dt_us < 1 || !(rate_hz >= 0.0) || t0_us < origin_us) return ORACLE_E_INVALID;
    const float rate_us = (float)(rate_hz * 1e-6);
    for (int64_t i = 0; i < n; ++i) {
        const float k = (cpos ? cpos[i] : cpos_u) * rate_us;
        for (int32_t f = 0; f < T; ++f) {
            const float s = (float)(t0_us + (int64_t)f * dt_us - origin_us);
            const float delta = k * s;
            out[(int64_t)f * n + i] = L[(int64_t)f * n + i] + delta;
        }
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Shot noise (reading R15).                                                */
/* ------------------------------------------------------------------------ */
#define SHOT_TILE 64
#define SHOT_MAX 15

/* thr[n] = floor(F(n) 2^53) for the Poisson CDF F of mean lam, n < SHOT_MAX */
static void poisson_thresholds(double lam, uint64_t thr[SHOT_MAX])
{
    double p = exp(-lam), F = p;
    for (int k = 0; k < SHOT_MAX; ++k) {
        double v = F * 9007199254740992.0;   /* 2^53 */
        thr[k] = v >= 9007199254740992.0 ? (uint64_t)1 << 53 : (uint64_t)v;
        p = p * lam / (double)(k + 1);
        F += p;
    }
}

int oracle_shot_noise(int32_t W, int32_t H, double rate_hz, uint64_t seed, int64_t ta0_us, int32_t D0_us,
                      int32_t dt_us, int32_t n_intervals, uint64_t **events_out, int64_t *n_events,
                      int64_t **seg_out)
{
    if (W <= 0 || H <= 0 || W > 65535 || H > 32767 || n_intervals < 0 || !(rate_hz >= 0.0) || D0_us < 1 ||
        dt_us < 1 || ta0_us < 0)
        return ORACLE_E_INVALID;
    if (rate_hz * SHOT_TILE * (double)(D0_us > dt_us ? D0_us : dt_us) * 1e-6 > 4.0) return ORACLE_E_INVALID;
    const int64_t npix = (int64_t)W * H;
    const int64_t n_tiles = (npix + SHOT_TILE - 1) / SHOT_TILE;
    int64_t cap = 1024, n = 0;
    uint64_t *ev = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
    int64_t *seg = (int64_t *)malloc((size_t)(n_intervals + 1) * sizeof(int64_t));
    if (!ev || !seg) {
        free(ev);
        free(seg);
        return ORACLE_E_NOMEM;
    }
    seg[0] = 0;
    for (int32_t j = 0; j < n_intervals; ++j) {
        const int64_t ta = j == 0 ? ta0_us : ta0_us + D0_us + (int64_t)(j - 1) * dt_us;
        const int32_t D = j == 0 ? D0_us : dt_us;
        if (ta + D > 0xFFFFFFFFll) {
            free(ev);
            free(seg);
            return ORACLE_E_TIME;
        }
        const int64_t start = n;
        for (int64_t tile = 0; tile < n_tiles; ++tile) {
            const int64_t len = (tile + 1) * SHOT_TILE <= npix ? SHOT_TILE : npix - tile * SHOT_TILE;
            uint64_t thr[SHOT_MAX];
            poisson_thresholds(rate_hz * (double)len * (double)D * 1e-6, thr);
            const uint64_t base = ((uint64_t)ta * (uint64_t)n_tiles + (uint64_t)tile) * 32u;
            const uint64_t U = oracle_splitmix64_at(seed, base) >> 11;
            int count = SHOT_MAX;
            for (int k = 0; k < SHOT_MAX; ++k)
                if (U < thr[k]) {
                    count = k;
                    break;
                }
            for (int i = 0; i < count; ++i) {
                const uint64_t d1 = oracle_splitmix64_at(seed, base + 1u + 2u * (uint64_t)i);
                const uint64_t d2 = oracle_splitmix64_at(seed, base + 2u + 2u * (uint64_t)i);
                const int64_t pix = tile * SHOT_TILE + (int64_t)(((d1 >> 32) * (uint64_t)len) >> 32);
                const int64_t t = ta + (int64_t)(((d1 & 0xFFFFFFFFull) * (uint64_t)D) >> 32);
                if (n == cap) {
                    cap *= 2;
                    uint64_t *q = (uint64_t *)realloc(ev, (size_t)cap * sizeof(uint64_t));
                    if (!q) {
                        free(ev);
                        free(seg);
                        return ORACLE_E_NOMEM;
                    }
                    ev = q;
                }
                ev[n++] = pack(t, (int32_t)(pix % W), (int32_t)(pix / W), (int)(d2 >> 63));
            }
        }
        qsort(ev + start, (size_t)(n - start), sizeof(uint64_t), cmp_u64);
        seg[j + 1] = n;
    }
    *events_out = ev;
    *n_events = n;
    *seg_out = seg;
    return ORACLE_OK;
}

/* Two interval-structured streams (seg_a, seg_b: n_intervals + 1 offsets)  */
/* merged interval by interval in record order (R8); out holds both.        */
int oracle_merge_events(const uint64_t *a, const int64_t *seg_a, const uint64_t *b, const int64_t *seg_b,
                        int32_t n_intervals, uint64_t *out, int64_t *seg_out)
{
    if (n_intervals < 0) return ORACLE_E_INVALID;
    int64_t o = 0;
    seg_out[0] = 0;
    for (int32_t j = 0; j < n_intervals; ++j) {
        const int64_t start = o;
        for (int64_t i = seg_a[j]; i < seg_a[j + 1]; ++i) out[o++] = a[i];
        for (int64_t i = seg_b[j]; i < seg_b[j + 1]; ++i) out[o++] = b[i];
        qsort(out + start, (size_t)(o - start), sizeof(uint64_t), cmp_u64);
        seg_out[j + 1] = o;
    }
    return ORACLE_OK;
}

void oracle_free(void *p) { free(p); }
