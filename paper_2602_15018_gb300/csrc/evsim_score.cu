// Scoring of an event stream against a reference stream (declared in
// include/neurosim_evsim.h as neurosim_event_f1): host code, not on any hot
// path.  Used to score the learned interpolator's events against the plain
// high-rate path.  The paper defines no score; the definition taken is:
// predicted and reference events match one to one inside the same pixel and
// polarity, greedily in time order, when their times differ by at most
// tol_us; P = matched / predicted, R = matched / reference,
// F1 = 2 P R / (P + R); count error = sum over (pixel, polarity) of
// |n_pred - n_ref| / (reference events).
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"

namespace {

// (y, x, p) cell in the high 32 bits, time in the low 32 bits
inline uint64_t by_cell(uint64_t rec)
{
    const uint64_t t = rec >> 32, y = (rec >> 17) & 0x7FFFu, x = (rec >> 1) & 0xFFFFu, p = rec & 1u;
    return (((y << 17) | (x << 1) | p) << 32) | t;
}

}  // namespace

extern "C" int neurosim_event_f1(const uint64_t* pred, int64_t n_pred, const uint64_t* ref, int64_t n_ref,
                                 int64_t tol_us, int64_t* counts, double* scores)
{
    if (n_pred < 0 || n_ref < 0 || (n_pred > 0 && !pred) || (n_ref > 0 && !ref) || !counts || !scores || tol_us < 0)
        return nsim::report_error(NEUROSIM_E_INVALID, "bad arguments to neurosim_event_f1");
    std::vector<uint64_t> a((size_t)n_pred), b((size_t)n_ref);
    for (int64_t i = 0; i < n_pred; ++i) a[(size_t)i] = by_cell(pred[i]);
    for (int64_t i = 0; i < n_ref; ++i) b[(size_t)i] = by_cell(ref[i]);
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    int64_t matched = 0, abs_err = 0;
    size_t i = 0, j = 0;
    while (i < a.size() || j < b.size()) {
        const uint64_t ca = i < a.size() ? a[i] >> 32 : UINT64_MAX;
        const uint64_t cb = j < b.size() ? b[j] >> 32 : UINT64_MAX;
        const uint64_t cell = std::min(ca, cb);
        size_t ie = i, je = j;
        while (ie < a.size() && (a[ie] >> 32) == cell) ++ie;
        while (je < b.size() && (b[je] >> 32) == cell) ++je;
        abs_err += std::llabs((long long)(ie - i) - (long long)(je - j));
        size_t u = i, v = j;
        while (u < ie && v < je) {
            const int64_t tu = (int64_t)(a[u] & 0xFFFFFFFFu), tv = (int64_t)(b[v] & 0xFFFFFFFFu);
            if (std::llabs(tu - tv) <= tol_us) {
                ++matched;
                ++u;
                ++v;
            } else if (tu < tv) {
                ++u;
            } else {
                ++v;
            }
        }
        i = ie;
        j = je;
    }
    counts[0] = matched;
    counts[1] = n_pred;
    counts[2] = n_ref;
    counts[3] = abs_err;
    const double P = n_pred ? (double)matched / (double)n_pred : (n_ref ? 0.0 : 1.0);
    const double R = n_ref ? (double)matched / (double)n_ref : (n_pred ? 0.0 : 1.0);
    scores[0] = P;
    scores[1] = R;
    scores[2] = P + R > 0.0 ? 2.0 * P * R / (P + R) : 0.0;
    scores[3] = n_ref ? (double)abs_err / (double)n_ref : (n_pred ? INFINITY : 0.0);
    return NEUROSIM_OK;
}
