/*
 * Oracle for the event-stream consumers and the scoring of an event stream.
 *
 * TEST INFRASTRUCTURE ONLY (same rules as evsim_oracle.c: loaded by the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark only; no
 * code is shared with the CUDA path).
 *
 * Packed record (64 bits): [63:32] t (us) | [31:17] y | [16:1] x | [0] p.
 *
 *  - oracle_time_surface: the time surface of the supplementary RL section of
 *    arXiv 2602.15018: for each event at time t, pixel (x, y), polarity p,
 *    S(x, y, p) <- S(x, y, p) * exp(-dt / tau) + 1, dt being the time since
 *    the previous update of that same cell; S starts at zero.  FP64.
 *  - oracle_event_frames: events accumulated per pixel and polarity over
 *    fixed windows (the 20 ms polarity event frames of Sec. 2, Fig. 2B and
 *    Sec. 4).
 *  - oracle_match_f1: event-stream F1 and count error.  Reading (the paper
 *    defines no score): predicted and reference events are matched one to
 *    one within the same pixel and polarity, greedily in time order, when
 *    their timestamps differ by at most tol_us.  P = matched / predicted,
 *    R = matched / reference, F1 = 2PR / (P + R); count error =
 *    sum over (pixel, polarity) of |n_pred - n_ref| / n_ref_total.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static void unpack(uint64_t e, int64_t *t, int32_t *x, int32_t *y, int32_t *p)
{
    *t = (int64_t)(e >> 32);
    *y = (int32_t)((e >> 17) & 0x7FFFu);
    *x = (int32_t)((e >> 1) & 0xFFFFu);
    *p = (int32_t)(e & 1u);
}

/* S and last are [2][H][W]; last = -1 marks a cell never updated. */
int oracle_time_surface(int32_t W, int32_t H, const uint64_t *ev, int64_t n, double *S,
                        int64_t *last, double tau_us)
{
    if (W <= 0 || H <= 0 || !(tau_us > 0.0)) return 1;
    const int64_t plane = (int64_t)W * H;
    for (int64_t i = 0; i < n; ++i) {
        int64_t t;
        int32_t x, y, p;
        unpack(ev[i], &t, &x, &y, &p);
        if (x >= W || y >= H) return 1;
        const int64_t c = (int64_t)p * plane + (int64_t)y * W + x;
        double decay = 1.0;
        if (last[c] >= 0) decay = exp(-(double)(t - last[c]) / tau_us);
        S[c] = S[c] * decay + 1.0;
        last[c] = t;
    }
    return 0;
}

/* out is [n_win][2][H][W] counts; event i goes to window (t - t_start) / win
 * when 0 <= that < n_win. */
int oracle_event_frames(int32_t W, int32_t H, const uint64_t *ev, int64_t n, int64_t t_start,
                        int64_t win_us, int32_t n_win, int32_t *out)
{
    if (W <= 0 || H <= 0 || win_us <= 0 || n_win < 0) return 1;
    const int64_t plane = (int64_t)W * H;
    for (int64_t i = 0; i < n; ++i) {
        int64_t t;
        int32_t x, y, p;
        unpack(ev[i], &t, &x, &y, &p);
        if (x >= W || y >= H) return 1;
        if (t < t_start) continue;
        const int64_t w = (t - t_start) / win_us;
        if (w >= n_win) continue;
        out[(w * 2 + p) * plane + (int64_t)y * W + x] += 1;
    }
    return 0;
}

static int cmp_u64(const void *pa, const void *pb)
{
    uint64_t a = *(const uint64_t *)pa, b = *(const uint64_t *)pb;
    return (a > b) - (a < b);
}

/* (pixel, polarity, time) ordering key. */
static uint64_t cell_key(uint64_t e)
{
    const uint64_t t = e >> 32, y = (e >> 17) & 0x7FFFu, x = (e >> 1) & 0xFFFFu, p = e & 1u;
    return (y << 49) | (x << 33) | (p << 32) | t;
}

/* counts[4] = matched, n_pred, n_ref, sum |n_pred - n_ref| over cells;
 * scores[4] = precision, recall, F1, count error. */
int oracle_match_f1(int32_t W, int32_t H, const uint64_t *pred, int64_t n_pred,
                    const uint64_t *refv, int64_t n_ref, int64_t tol_us, int64_t *counts,
                    double *scores)
{
    (void)W;
    (void)H;
    uint64_t *a = (uint64_t *)malloc((size_t)(n_pred > 0 ? n_pred : 1) * 8);
    uint64_t *b = (uint64_t *)malloc((size_t)(n_ref > 0 ? n_ref : 1) * 8);
    if (!a || !b) { free(a); free(b); return 2; }
    for (int64_t i = 0; i < n_pred; ++i) a[i] = cell_key(pred[i]);
    for (int64_t i = 0; i < n_ref; ++i) b[i] = cell_key(refv[i]);
    qsort(a, (size_t)n_pred, 8, cmp_u64);
    qsort(b, (size_t)n_ref, 8, cmp_u64);
    int64_t i = 0, j = 0, matched = 0, cnt_err = 0;
    while (i < n_pred || j < n_ref) {
        /* next cell: the smaller cell id of the two heads */
        uint64_t ca = i < n_pred ? (a[i] >> 32) : UINT64_MAX;
        uint64_t cb = j < n_ref ? (b[j] >> 32) : UINT64_MAX;
        uint64_t cell = ca < cb ? ca : cb;
        int64_t i1 = i, j1 = j;
        while (i1 < n_pred && (a[i1] >> 32) == cell) ++i1;
        while (j1 < n_ref && (b[j1] >> 32) == cell) ++j1;
        cnt_err += llabs((i1 - i) - (j1 - j));
        /* greedy two-pointer matching within the cell, in time order */
        int64_t ii = i, jj = j;
        while (ii < i1 && jj < j1) {
            const int64_t ta = (int64_t)(a[ii] & 0xFFFFFFFFu), tb = (int64_t)(b[jj] & 0xFFFFFFFFu);
            if (llabs(ta - tb) <= tol_us) { ++matched; ++ii; ++jj; }
            else if (ta < tb) ++ii;
            else ++jj;
        }
        i = i1;
        j = j1;
    }
    free(a);
    free(b);
    counts[0] = matched;
    counts[1] = n_pred;
    counts[2] = n_ref;
    counts[3] = cnt_err;
    const double P = n_pred ? (double)matched / (double)n_pred : (n_ref ? 0.0 : 1.0);
    const double R = n_ref ? (double)matched / (double)n_ref : (n_pred ? 0.0 : 1.0);
    scores[0] = P;
    scores[1] = R;
    scores[2] = (P + R) > 0 ? 2.0 * P * R / (P + R) : 0.0;
    scores[3] = n_ref ? (double)cnt_err / (double)n_ref : (n_pred ? INFINITY : 0.0);
    return 0;
}
