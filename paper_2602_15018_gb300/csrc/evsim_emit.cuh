// Emission kernel of the event path (included by evsim_kernels.cu, inside the
// anonymous namespace; uses model_log, stream_of_item and the StepLaunch of
// evsim_internal.h).
//
// Model: arXiv 2602.15018, Sec. 2 — per-pixel state with the level of the last
// triggered event, contrast-threshold crossings, timestamps between frames,
// a variable number of events per frame gathered with few global atomics.
//
// Work split: one warp owns a tile of 32 * PPT contiguous pixels of one stream
// for all T frames of the step; warps never wait on each other.  Tile-local
// pixel p = q*128 + lane*4 + c (q < PPT/4, c < 4) is loaded by lane `lane`
// as part of its q-th float4, so every load instruction of the warp reads 512
// contiguous bytes.  The exact per-pixel state (ref, t_last, last computed
// log intensity), the raw inputs of the frame before the current pair and of
// the pair, and the pixel's filter bounds live in the warp's slice of shared
// memory, indexed by p; per-pixel thresholds are read from global memory when
// needed.
//
// Fast path (every pixel, every frame): the raw input v is compared with
// bounds vd < v < vu chosen so that inside them the model's log intensity of
// v lies strictly between ref - C- and ref + C+: no crossing is possible and
// only L_prev moves.  In the log domain the bounds are the exact FP32 levels
// ref + C+ and ref - C- (the clamp to [-32, 32] keeps the implication).  For
// intensities, x = fl(clamp(v, 0, 1e6) + eps) is monotone in v, and
//   xu = 2^((ref + C+) log2 e) (1 - 1e-4),  vu = fl(xu - eps),
//   xd = 2^((ref - C-) log2 e) (1 + 1e-4),  vd = fl(xd - eps),
// with the 1e-4 margin about 30 times the combined error of ex2.approx, the
// FP32 roundings and the 2-ulp bound of the model's log on [1e-8, 1e6 + 1];
// the filter may send a pixel to the slow path for nothing, never the other
// way.  A NaN input fails both comparisons and is always tested exactly.
//
// Slow path, once per pair of frames (f, f + 1): both frames are filtered
// with the bounds from before the pair.  A pixel out of its band at f is
// modelled exactly over both frames (its filter result at f + 1 is stale); a
// pixel in its band at f but out at f + 1 only over f + 1.  These pixels are
// compacted into a list in pixel order and handed out one per lane, so that
// the list build, the threshold loads, the log of the previous input and the
// bounds update are paid once per pair, not once per frame.  Each lane runs
// the exact FP32 model for its pixel, commits the state and keeps the first
// two keys of each frame in registers; per frame a warp prefix of the counts
// (list order = pixel order) places the tile's keys of that interval as one
// contiguous chunk of the paged key buffer, both frames' chunks in one run
// (one global atomic per page, not per frame).  More than 32 listed pixels
// fall back to the general path frame by frame; more than two events of a
// pixel in a frame regenerate its keys from the saved state.

constexpr float kBoundMargin = 1.0e-4f;
constexpr float kMaxIntensity = 1.0e6f;

// L2 eviction policies: frames are read once and should leave L2 first; the
// per-pixel thresholds are re-read on every slow path and should stay.
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ float4 ld_stream4(const float* p, uint64_t pol)
{
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ float ld_stream(const float* p, uint64_t pol)
{
    float v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ float ld_keep(const float* p, uint64_t pol)
{
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ float ex2_approx(float v)
{
    float r;
    asm("ex2.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float transform_in(float v, float eps, int is_log)
{
    if (is_log) return fminf(fmaxf(v, -32.0f), 32.0f);
    return __fadd_rn(fminf(fmaxf(v, 0.0f), kMaxIntensity), eps);
}

__device__ __forceinline__ float model_L(float v, float eps, int is_log)
{
    const float x = transform_in(v, eps, is_log);
    return is_log ? x : model_log(x);
}

// Raw-input bound below which no ON crossing of level `up` is possible.
__device__ __forceinline__ float raw_bound_up(float up, float eps, int is_log)
{
    if (is_log) return up;
    const float xu = __fmul_rn(ex2_approx(__fmul_rn(up, 1.44269504f)), 1.0f - kBoundMargin);
    if (!(xu > eps)) return __int_as_float(0xff800000);                        // test every input
    if (xu > __fadd_rn(kMaxIntensity, eps)) return __int_as_float(0x7f800000);  // unreachable
    return __fsub_rn(xu, eps);
}

// Raw-input bound above which no OFF crossing of level `dn` is possible.
__device__ __forceinline__ float raw_bound_dn(float dn, float eps, int is_log)
{
    if (is_log) return dn;
    const float xd = __fmul_rn(ex2_approx(__fmul_rn(dn, 1.44269504f)), 1.0f + kBoundMargin);
    if (xd < eps) return __int_as_float(0xff800000);                              // every input is above
    if (!(xd < __fadd_rn(kMaxIntensity, eps))) return __int_as_float(0x7f800000);  // test every input
    return __fsub_rn(xd, eps);
}

// Crossings of one pixel over one interval (L_a at ta, L_b at ta + D), both
// polarities in one loop: ON uses +C+, OFF uses -C- (fl(r - c) == fl(r + -c)).
// Advances ref and t_last.  MODE 0: count only; MODE 1: also keep keys 0 and
// 1 in k0 / k1; MODE 2: write every key to out[].  Returns the count.
template <int MODE, typename KeyT>
__device__ __forceinline__ int pixel_events(float& r, uint32_t& tl, float a, float b, float cp,
                                            float cn, uint32_t ta, float Df, uint32_t R,
                                            KeyT pixkey, int tshift, KeyT& k0, KeyT& k1,
                                            KeyT* out)
{
    if (!(b != a)) return 0;
    const bool on = b > a;
    const float c = on ? cp : -cn;
    const float den = __fsub_rn(b, a);
    const KeyT pol = on ? (KeyT)1 : (KeyT)0;
    int n = 0;
    for (;;) {
        const float lvl = __fadd_rn(r, c);
        if (on ? !(lvl <= b) : !(lvl >= b)) break;
        const float frac = __fdiv_rn(__fsub_rn(lvl, a), den);
        const float tf = fmaxf(floorf(__fmul_rn(frac, Df)), 0.0f);
        const uint32_t toff = (uint32_t)tf;
        const uint32_t t = ta + toff;
        r = lvl;
        if (R != 0u && tl != kTlastNone && (int64_t)t - (int64_t)tl < (int64_t)R) continue;
        if (MODE != 0) {
            const KeyT key = ((KeyT)toff << tshift) | pixkey | pol;
            if (MODE == 2) out[n] = key;
            else if (n == 0) k0 = key;
            else if (n == 1) k1 = key;
        }
        ++n;
        tl = t;
    }
    return n;
}

// Per-warp shared-memory slice (arrays of WPX = 32*PPT entries indexed by the
// tile-local pixel, plus the trigger list and the lanes' "L cached" masks).
// The raw inputs of frame f live in input slot f % 3: the previous frame and
// the two frames of the current pair.
template <int PPT>
struct WarpSlice {
    static constexpr int WPX = 32 * PPT;
    static constexpr int FLOATS = 8 * WPX + WPX + 32;   // 8 arrays, list (u32), masks
    float* base;
    __device__ __forceinline__ float* vs(int slot) const { return base + slot * WPX; }
    __device__ __forceinline__ float* vu() const { return base + 3 * WPX; }
    __device__ __forceinline__ float* vd() const { return base + 4 * WPX; }
    __device__ __forceinline__ float* ref() const { return base + 5 * WPX; }
    __device__ __forceinline__ uint32_t* tl() const { return reinterpret_cast<uint32_t*>(base + 6 * WPX); }
    __device__ __forceinline__ float* lb() const { return base + 7 * WPX; }
    __device__ __forceinline__ uint32_t* list() const { return reinterpret_cast<uint32_t*>(base + 8 * WPX); }
    __device__ __forceinline__ uint32_t* lvm() const { return reinterpret_cast<uint32_t*>(base + 9 * WPX); }
};

// Everything the slow path needs about the current tile and frame.
struct TileCtx {
    const float* cpos;   // per-pixel thresholds of the stream (global), or null
    const float* cneg;
    float cpos_u, cneg_u;
    uint32_t ta;         // start and length of the frame's interval
    float Df;
    uint32_t R;
    float eps;
    int is_log;
    int tshift;
    int g0;              // global index of the tile's pixel 0
    const float* vcur;   // raw inputs of the frame and of the one before it
    float* vprev;
    uint64_t keep;       // L2 evict_last policy for the thresholds
};

__device__ __forceinline__ void thresholds_of(const TileCtx& c, int p, float& cp, float& cn)
{
    if (c.cpos) {
        cp = ld_keep(c.cpos + c.g0 + p, c.keep);
        cn = ld_keep(c.cneg + c.g0 + p, c.keep);
    } else {
        cp = c.cpos_u;
        cn = c.cneg_u;
    }
}

// L_a of pixel p: cached L of the previous frame if its owner lane's mask says
// so, else the model's log of the previous input.
template <int PPT>
__device__ __forceinline__ float L_prev(const WarpSlice<PPT>& s, const TileCtx& c, const float* vprev, int p)
{
    const int owner = (p & 127) >> 2;
    const int bit = ((p >> 7) << 2) | (p & 3);
    if ((s.lvm()[owner] >> bit) & 1u) return s.lb()[p];
    return model_L(vprev[p], c.eps, c.is_log);
}

// `total` consecutive keys from the warp's page (a new page run when they do
// not fit); kNoChunk and the overflow bit when the key buffer is exhausted.
__device__ __forceinline__ uint32_t take_keys(uint32_t& pg_cur, uint32_t& pg_end, uint32_t total, int lane,
                                              uint32_t page_keys, uint32_t n_pages, unsigned int* page_ctr,
                                              unsigned int* err)
{
    if (total == 0u) return kNoChunk;
    if (pg_end - pg_cur >= total) {
        const uint32_t b = pg_cur;
        pg_cur += total;
        return b;
    }
    const uint32_t np_ = (total + page_keys - 1u) / page_keys;
    uint32_t first = 0u;
    if (lane == 0) first = atomicAdd(page_ctr, np_);
    first = __shfl_sync(0xffffffffu, first, 0);
    if ((uint64_t)first + np_ <= (uint64_t)n_pages) {
        const uint32_t b = first * page_keys;
        pg_cur = b + total;
        pg_end = (first + np_) * page_keys;
        return b;
    }
    if (lane == 0) atomicOr(err, kErrPageOverflow);
    pg_cur = pg_end = 0u;
    return kNoChunk;
}

// Writes the tile-local pixels whose bit is set in the lanes' masks m (bit
// q*4 + c = pixel q*128 + lane*4 + c) to list[] in pixel order (group q, then
// lane, then component), each entry p | (bit of `flag` for p) << 10.
// Returns the count (warp-uniform).
template <int PPT>
__device__ __forceinline__ int build_list(uint32_t m, uint32_t flag, int lane, uint32_t* list)
{
    constexpr int NQ = PPT / 4;
    uint32_t packed = 0u;   // 8-bit count per group (at most 128)
#pragma unroll
    for (int q = 0; q < NQ; ++q) packed |= (uint32_t)__popc((m >> (q * 4)) & 15u) << (q * 8);
    uint32_t incl = packed;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t nb = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += nb;
    }
    const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t ex = incl - packed;
    int n = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        int pos = n + (int)((ex >> (q * 8)) & 255u);
        uint32_t mm = (m >> (q * 4)) & 15u;
        while (mm) {
            const int cbit = __ffs(mm) - 1;
            mm &= mm - 1u;
            list[pos++] = (uint32_t)(q * 128 + lane * 4 + cbit) | (((flag >> (q * 4 + cbit)) & 1u) << 10);
        }
        n += (int)((tot >> (q * 8)) & 255u);
    }
    return n;
}

// Exclusive prefix and total of the lanes' counts n >= 0.
__device__ __forceinline__ void count_prefix(int n, int lane, int& excl, uint32_t& total)
{
    if (__any_sync(0xffffffffu, n > 3)) {
        int in = n;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int nb = __shfl_up_sync(0xffffffffu, in, d);
            if (lane >= d) in += nb;
        }
        excl = in - n;
        total = (uint32_t)__shfl_sync(0xffffffffu, in, 31);
    } else {
        const uint32_t lt = (1u << lane) - 1u;
        const uint32_t b0 = __ballot_sync(0xffffffffu, (n & 1) != 0);
        const uint32_t b1 = __ballot_sync(0xffffffffu, (n & 2) != 0);
        excl = __popc(b0 & lt) + 2 * __popc(b1 & lt);
        total = (uint32_t)(__popc(b0) + 2 * __popc(b1));
    }
}

// General path for one warp-frame: any number of list entries (n_list, in
// pixel order) and events.  Pass 1 commits every entry and saves (L_a, ref,
// t_last) before the step in the vu / vd / previous-input slots and its count
// in the list entry; then the keys are regenerated into out[] in list order;
// then fresh bounds.
template <int PPT, typename KeyT>
__device__ __noinline__ void slow_general(const WarpSlice<PPT> s, const TileCtx c, int lane,
                                          int n_list, KeyT* keys, uint32_t page_keys, uint32_t n_pages,
                                          unsigned int* page_ctr, unsigned int* err,
                                          uint32_t& pg_cur, uint32_t& pg_end, uint32_t* chunk_off,
                                          uint32_t* chunk_cnt)
{
    uint32_t* vprev_bits = reinterpret_cast<uint32_t*>(c.vprev);
    uint32_t total = 0;
    for (int r0 = 0; r0 < n_list; r0 += 32) {
        const int e = r0 + lane;
        int n = 0;
        if (e < n_list) {
            const int p = (int)(s.list()[e] & 1023u);
            float cp, cn;
            thresholds_of(c, p, cp, cn);
            const float b = model_L(c.vcur[p], c.eps, c.is_log);
            const float a = L_prev(s, c, c.vprev, p);
            float r = s.ref()[p];
            uint32_t tl = s.tl()[p];
            s.vu()[p] = a;
            s.vd()[p] = r;
            vprev_bits[p] = tl;
            s.lb()[p] = b;
            KeyT d0 = 0, d1 = 0;
            n = pixel_events<0, KeyT>(r, tl, a, b, cp, cn, c.ta, c.Df, c.R, (KeyT)0, 0, d0, d1, nullptr);
            s.ref()[p] = r;
            s.tl()[p] = tl;
            s.list()[e] = (uint32_t)p | ((uint32_t)n << 10);
        }
        total += __reduce_add_sync(0xffffffffu, (uint32_t)n);
    }
    __syncwarp();
    // one contiguous chunk for the whole warp-frame
    const uint32_t base = take_keys(pg_cur, pg_end, total, lane, page_keys, n_pages, page_ctr, err);
    *chunk_off = base == kNoChunk ? 0u : base;
    *chunk_cnt = base == kNoChunk ? 0u : total;
    uint32_t carry = 0;
    for (int r0 = 0; r0 < n_list; r0 += 32) {
        const int e = r0 + lane;
        const uint32_t ent = (e < n_list) ? s.list()[e] : 0u;
        const int p = (int)(ent & 1023u);
        const int n = (int)(ent >> 10);
        int incl = n;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int nb = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += nb;
        }
        if (e < n_list) {
            float cp, cn;
            thresholds_of(c, p, cp, cn);
            if (base != kNoChunk && n > 0) {
                float r = s.vd()[p];
                uint32_t tl = vprev_bits[p];
                KeyT d0 = 0, d1 = 0;
                pixel_events<2, KeyT>(r, tl, s.vu()[p], s.lb()[p], cp, cn, c.ta, c.Df, c.R,
                                      (KeyT)(c.g0 + p) << 1, c.tshift, d0, d1,
                                      keys + (size_t)base + carry + (uint32_t)(incl - n));
            }
            const float rr = s.ref()[p];
            s.vu()[p] = raw_bound_up(__fadd_rn(rr, cp), c.eps, c.is_log);
            s.vd()[p] = raw_bound_dn(__fsub_rn(rr, cn), c.eps, c.is_log);
        }
        carry += (uint32_t)__shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
}

template <int PPT>
__device__ __forceinline__ void load_frame(float4 (&b)[PPT / 4], const float* p, int nvq, int vec,
                                           int lane_left, uint64_t pol)
{
    // p points at the lane's first float of group 0; group q is 128 floats further.
#pragma unroll
    for (int q = 0; q < PPT / 4; ++q) {
        if (vec) {
            b[q] = (q < nvq) ? ld_stream4(p + q * 128, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            float e[4];
            const int left = lane_left - q * 128;
#pragma unroll
            for (int m = 0; m < 4; ++m) e[m] = (m < left) ? ld_stream(p + q * 128 + m, pol) : 0.0f;
            b[q] = make_float4(e[0], e[1], e[2], e[3]);
        }
    }
}

__device__ __forceinline__ uint32_t outside4(const float4 v, const float4 u, const float4 d)
{
    return ((v.x < u.x && v.x > d.x) ? 0u : 1u) | ((v.y < u.y && v.y > d.y) ? 0u : 2u) |
           ((v.z < u.z && v.z > d.z) ? 0u : 4u) | ((v.w < u.w && v.w > d.w) ? 0u : 8u);
}

// Start and length of interval j of the step.
__device__ __forceinline__ void interval_of(int64_t ta0, int D0, int dt, int j, uint32_t& ta, float& Df)
{
    ta = (uint32_t)(ta0 + (j == 0 ? 0 : (int64_t)D0 + (int64_t)(j - 1) * dt));
    Df = (float)(j == 0 ? D0 : dt);
}

// Frame sources of the emission kernel: frames read from memory, or rendered
// from a texture scene (scene_render.cuh) in place of the read.
template <int PPT>
struct MemSource {
    const float* fp;       // the lane's first pixel in frame 0
    int64_t fstride;
    int nvq, vec, lane_left;
    uint64_t pol;
    __device__ __forceinline__ void load(float4 (&b)[PPT / 4], int f) const
    {
        load_frame<PPT>(b, fp + (int64_t)f * fstride, nvq, vec, lane_left, pol);
    }
};

template <int PPT>
struct TexSource {
    const SceneFrame* tab;   // row f: camera and rectangles of the step's frame f
    SceneConst sc;
    int lane;
    float y_lo, y_hi;        // rows the warp's tile spans
    int x0[PPT / 4], y0[PPT / 4];   // pixel of (q, component 0)
    // Renders the lane's pixels of frame f.  Warp-collective: the rectangles
    // that can reach the tile's rows are found with one ballot and applied in
    // rectangle order, as texture_pixel does.
    __device__ __forceinline__ void load(float4 (&b)[PPT / 4], int f) const
    {
        const SceneFrame& fr = tab[f];
        float4 rk = make_float4(0.f, 0.f, 0.f, 0.f);
        float vk = 0.0f;
        bool rel = false;
        if (lane < sc.n_rects) {
            rk = fr.rect[lane];
            vk = fr.rval[lane];
            // a pixel row y can be covered only if |y - cy| < hh (one row of margin
            // for the rounding of y - cy)
            rel = __fadd_rn(__fadd_rn(rk.y, rk.w), 1.0f) > y_lo && __fsub_rn(__fsub_rn(rk.y, rk.w), 1.0f) < y_hi;
        }
        uint32_t rmask = __ballot_sync(0xffffffffu, rel);
#pragma unroll
        for (int q = 0; q < PPT / 4; ++q) {
            float xs[4], ys[4], v[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                int x = x0[q] + m, y = y0[q];
                if (x >= sc.W) { x -= sc.W; y += 1; }
                xs[m] = (float)x;
                ys[m] = (float)y;
            }
            texture_noise4(sc, fr, xs, ys, v);
            b[q] = make_float4(v[0], v[1], v[2], v[3]);
        }
        while (rmask) {
            const int k = __ffs(rmask) - 1;
            rmask &= rmask - 1u;
            const float4 r = make_float4(__shfl_sync(0xffffffffu, rk.x, k), __shfl_sync(0xffffffffu, rk.y, k),
                                         __shfl_sync(0xffffffffu, rk.z, k), __shfl_sync(0xffffffffu, rk.w, k));
            const float val = __shfl_sync(0xffffffffu, vk, k);
#pragma unroll
            for (int q = 0; q < PPT / 4; ++q) {
                float* c = reinterpret_cast<float*>(&b[q]);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    int x = x0[q] + m, y = y0[q];
                    if (x >= sc.W) { x -= sc.W; y += 1; }
                    if (rect_covers(r, (float)x, (float)y)) c[m] = val;
                }
            }
        }
    }
};

// The render-fused variant asks for three resident CTAs per SM (two with the
// 8-warp CTAs of 256-pixel tiles): rendering wants the warps more than the
// registers (measured 28.0 ms per HD step against 37.4 ms at its
// unconstrained 213 registers and two CTAs per SM).
template <int PPT, int WARPS, int PF, typename KeyT, int SRC>
__global__ void __launch_bounds__(WARPS * 32, SRC == 1 ? (PPT == 16 ? 3 : 2) : 1)
    emit_kernel(const __grid_constant__ StepLaunch L)
{
    (void)PF;   // one pair of frames in flight whatever the prefetch setting
    constexpr int NQ = PPT / 4;
    constexpr int WPX = 32 * PPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const WarpSlice<PPT> s{reinterpret_cast<float*>(smem_raw) + (size_t)wib * WarpSlice<PPT>::FLOATS};
    KeyT* const keys = reinterpret_cast<KeyT*>(L.keys);
    uint32_t pg_cur = 0u, pg_end = 0u;      // warp-uniform free range of the warp's key page
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const int gw = blockIdx.x * WARPS + wib;
    const int nw = gridDim.x * WARPS;
    if (step_stopped(L)) return;

    for (int item = gw; item < L.n_items; item += nw) {
        const StreamDesc* sdp = stream_of_item(L, item);
        const int npix = sdp->npix;
        const int tile = item - sdp->item_base;
        const int init = sdp->init;
        const int vec = sdp->vec;
        const int T = L.T;
        const int dt = L.dt;
        const int D0 = sdp->D0;
        const int64_t ta0 = step_ta0(L, *sdp);
        uint2* const chunk_col = L.chunks + sdp->chunk_base + tile;
        const int n_tiles = sdp->n_tiles;
        TileCtx c;
        c.cpos = sdp->cpos;
        c.cneg = sdp->cneg;
        c.cpos_u = sdp->cpos_u;
        c.cneg_u = sdp->cneg_u;
        c.R = sdp->refractory;
        c.eps = sdp->log_eps;
        c.is_log = sdp->input_is_log;
        c.tshift = sdp->pix_bits + 1;
        c.g0 = tile * WPX;
        c.keep = pol_keep;
        const int lane_g = c.g0 + lane * 4;                  // global pixel of (q=0, c=0)
        const int lane_left = npix - lane_g;                 // valid pixels from there on
        const int64_t fstride = sdp->frame_stride ? sdp->frame_stride : (int64_t)npix;
        int nvq = 0;                                         // complete float4 groups (vec)
#pragma unroll
        for (int q = 0; q < NQ; ++q) nvq += (lane_left - q * 128 >= 4) ? 1 : 0;
        uint32_t valid = 0u;                                 // bit q*4+m: pixel exists
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) valid |= (lane_left - q * 128 > m ? 1u : 0u) << (q * 4 + m);

        // state -> shared memory
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int p = q * 128 + lane * 4;
            const int g = c.g0 + p;
            float r[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
            uint32_t t[4] = {kTlastNone, kTlastNone, kTlastNone, kTlastNone};
            if (!init) {
                if (((valid >> (q * 4)) & 15u) == 15u) {
                    const float4 r4 = *reinterpret_cast<const float4*>(sdp->ref_in + g);
                    const float4 l4 = *reinterpret_cast<const float4*>(sdp->lprev_in + g);
                    const uint4 t4 = *reinterpret_cast<const uint4*>(sdp->tlast_in + g);
                    r[0] = r4.x; r[1] = r4.y; r[2] = r4.z; r[3] = r4.w;
                    l[0] = l4.x; l[1] = l4.y; l[2] = l4.z; l[3] = l4.w;
                    t[0] = t4.x; t[1] = t4.y; t[2] = t4.z; t[3] = t4.w;
                } else {
                    for (int m = 0; m < 4; ++m)
                        if ((valid >> (q * 4 + m)) & 1u) {
                            r[m] = sdp->ref_in[g + m];
                            l[m] = sdp->lprev_in[g + m];
                            t[m] = sdp->tlast_in[g + m];
                        }
                }
            }
            float u[4], d[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                float cp, cn;
                if ((valid >> (q * 4 + m)) & 1u) thresholds_of(c, p + m, cp, cn);
                else cp = cn = 1.0f;
                const bool ok = !init && ((valid >> (q * 4 + m)) & 1u);
                u[m] = ok ? raw_bound_up(__fadd_rn(r[m], cp), c.eps, c.is_log) : __int_as_float(0x7f800000);
                d[m] = ok ? raw_bound_dn(__fsub_rn(r[m], cn), c.eps, c.is_log) : __int_as_float(0xff800000);
            }
            *reinterpret_cast<float4*>(s.ref() + p) = make_float4(r[0], r[1], r[2], r[3]);
            *reinterpret_cast<float4*>(s.lb() + p) = make_float4(l[0], l[1], l[2], l[3]);
            *reinterpret_cast<uint4*>(s.tl() + p) = make_uint4(t[0], t[1], t[2], t[3]);
            *reinterpret_cast<float4*>(s.vu() + p) = make_float4(u[0], u[1], u[2], u[3]);
            *reinterpret_cast<float4*>(s.vd() + p) = make_float4(d[0], d[1], d[2], d[3]);
        }
        uint32_t lvalid = init ? 0u : valid;   // lb holds L of the frame before the next one

        // frame pipeline: one pair of frames in flight per lane
        typename std::conditional<SRC == 0, MemSource<PPT>, TexSource<PPT>>::type src;
        if constexpr (SRC == 0) {
            src.fp = sdp->frames + lane_g;
            src.fstride = fstride;
            src.nvq = nvq;
            src.vec = vec;
            src.lane_left = lane_left;
            src.pol = pol_stream;
        } else {
            src.tab = static_cast<const SceneFrame*>(sdp->scene_tab);
            src.sc = sdp->scene;
            src.lane = lane;
            const int W = sdp->scene.W;
            src.y_lo = (float)(c.g0 / W);
            src.y_hi = (float)((min(c.g0 + WPX, npix) - 1) / W);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int g = lane_g + q * 128;
                src.y0[q] = g / W;
                src.x0[q] = g - src.y0[q] * W;
            }
        }
        float4 buf[2][NQ];
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (u < T) src.load(buf[u], u);
        int fs = 0;
        if (init && T > 0) {
            // frame 0 initialises the state; the pairs start at frame 1
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                *reinterpret_cast<float4*>(s.vs(0) + q * 128 + lane * 4) = buf[0][q];
            for (int k = 0; k < PPT; ++k) {
                if (!((valid >> k) & 1u)) continue;
                const int p = (k >> 2) * 128 + lane * 4 + (k & 3);
                float cp, cn;
                thresholds_of(c, p, cp, cn);
                const float Lv = model_L(s.vs(0)[p], c.eps, c.is_log);
                s.ref()[p] = Lv;
                s.lb()[p] = Lv;
                s.vu()[p] = raw_bound_up(__fadd_rn(Lv, cp), c.eps, c.is_log);
                s.vd()[p] = raw_bound_dn(__fsub_rn(Lv, cn), c.eps, c.is_log);
            }
            lvalid = valid;
            fs = 1;
#pragma unroll
            for (int q = 0; q < NQ; ++q) buf[0][q] = buf[1][q];
            if (2 < T) src.load(buf[1], 2);
        }
        __syncwarp();

        for (int f0 = fs; f0 < T; f0 += 2) {
            const int nf = (T - f0 >= 2) ? 2 : 1;
            float* v0 = s.vs(f0 % 3);
            float* v1 = s.vs((f0 + 1) % 3);
            float* vp = s.vs((f0 + 2) % 3);               // frame f0 - 1
            uint32_t trig0 = 0u, trig1 = 0u;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int p = q * 128 + lane * 4;
                const float4 u4 = *reinterpret_cast<const float4*>(s.vu() + p);
                const float4 d4 = *reinterpret_cast<const float4*>(s.vd() + p);
                *reinterpret_cast<float4*>(v0 + p) = buf[0][q];
                trig0 |= outside4(buf[0][q], u4, d4) << (q * 4);
                if (nf == 2) {
                    *reinterpret_cast<float4*>(v1 + p) = buf[1][q];
                    trig1 |= outside4(buf[1][q], u4, d4) << (q * 4);
                }
            }
            trig0 &= valid;
            trig1 &= valid;
            if (f0 + 2 < T) src.load(buf[0], f0 + 2);
            if (f0 + 3 < T) src.load(buf[1], f0 + 3);
            const int j0 = f0 - init;                     // intervals of the pair's frames
            const uint32_t mall = trig0 | trig1;
            if (!__any_sync(0xffffffffu, mall != 0u)) {
                if (lane == 0) {
                    chunk_col[(int64_t)j0 * n_tiles] = make_uint2(0u, 0u);
                    if (nf == 2) chunk_col[(int64_t)(j0 + 1) * n_tiles] = make_uint2(0u, 0u);
                }
                lvalid = 0u;
                continue;
            }
            s.lvm()[lane] = lvalid;
            const int n_list = build_list<PPT>(mall, trig0, lane, s.list());
            __syncwarp();

            if (n_list <= 32) {
                // one round: lane e handles list entry e over the pair's frames
                uint32_t ta0i, ta1i;
                float Df0, Df1;
                interval_of(ta0, D0, dt, j0, ta0i, Df0);
                interval_of(ta0, D0, dt, j0 + 1, ta1i, Df1);
                int n0 = 0, n1 = 0, p = 0;
                KeyT k00 = 0, k01 = 0, k10 = 0, k11 = 0, pixkey = 0;
                float cp = 0.f, cn = 0.f, a = 0.f, b = 0.f, cL = 0.f, rs0 = 0.f, rs1 = 0.f;
                uint32_t ts0 = 0u, ts1 = 0u;
                if (lane < n_list) {
                    const uint32_t ent = s.list()[lane];
                    p = (int)(ent & 1023u);
                    const bool both = (ent >> 10) & 1u;
                    pixkey = (KeyT)(c.g0 + p) << 1;
                    thresholds_of(c, p, cp, cn);
                    float r = s.ref()[p];
                    uint32_t tl = s.tl()[p];
                    b = model_L(v0[p], c.eps, c.is_log);
                    if (both) {
                        a = L_prev(s, c, vp, p);
                        rs0 = r;
                        ts0 = tl;
                        n0 = pixel_events<1, KeyT>(r, tl, a, b, cp, cn, ta0i, Df0, c.R, pixkey, c.tshift, k00, k01,
                                                   nullptr);
                    }
                    cL = b;
                    if (nf == 2) {
                        cL = model_L(v1[p], c.eps, c.is_log);
                        rs1 = r;
                        ts1 = tl;
                        n1 = pixel_events<1, KeyT>(r, tl, b, cL, cp, cn, ta1i, Df1, c.R, pixkey, c.tshift, k10, k11,
                                                   nullptr);
                    }
                    s.ref()[p] = r;
                    s.tl()[p] = tl;
                    s.lb()[p] = cL;
                    s.vu()[p] = raw_bound_up(__fadd_rn(r, cp), c.eps, c.is_log);
                    s.vd()[p] = raw_bound_dn(__fsub_rn(r, cn), c.eps, c.is_log);
                }
                int ex0, ex1;
                uint32_t tot0, tot1;
                count_prefix(n0, lane, ex0, tot0);
                count_prefix(n1, lane, ex1, tot1);
                const uint32_t base = take_keys(pg_cur, pg_end, tot0 + tot1, lane, L.page_keys, L.n_pages,
                                                &L.ctl->page_ctr, &L.ctl->err);
                if (lane == 0) {
                    chunk_col[(int64_t)j0 * n_tiles] =
                        make_uint2(base == kNoChunk ? 0u : base, base == kNoChunk ? 0u : tot0);
                    if (nf == 2)
                        chunk_col[(int64_t)(j0 + 1) * n_tiles] =
                            make_uint2(base == kNoChunk ? 0u : base + tot0, base == kNoChunk ? 0u : tot1);
                }
                if (base != kNoChunk) {
                    if (n0 > 0) {
                        KeyT* out = keys + (size_t)base + (size_t)ex0;
                        if (n0 <= 2) {
                            out[0] = k00;
                            if (n0 == 2) out[1] = k01;
                        } else {
                            float rr = rs0;
                            uint32_t tt = ts0;
                            pixel_events<2, KeyT>(rr, tt, a, b, cp, cn, ta0i, Df0, c.R, pixkey, c.tshift, k00, k01,
                                                  out);
                        }
                    }
                    if (n1 > 0) {
                        KeyT* out = keys + (size_t)base + tot0 + (size_t)ex1;
                        if (n1 <= 2) {
                            out[0] = k10;
                            if (n1 == 2) out[1] = k11;
                        } else {
                            float rr = rs1;
                            uint32_t tt = ts1;
                            pixel_events<2, KeyT>(rr, tt, b, cL, cp, cn, ta1i, Df1, c.R, pixkey, c.tshift, k10, k11,
                                                  out);
                        }
                    }
                }
                lvalid = mall;
            } else {
                // many pixels at once: the general path, frame by frame
                uint32_t off = 0u, cntv = 0u;
                int n0l = 0;
                if (__any_sync(0xffffffffu, trig0 != 0u)) {
                    __syncwarp();
                    n0l = build_list<PPT>(trig0, 0u, lane, s.list());
                    __syncwarp();
                }
                if (n0l > 0) {
                    interval_of(ta0, D0, dt, j0, c.ta, c.Df);
                    c.vcur = v0;
                    c.vprev = vp;
                    slow_general<PPT, KeyT>(s, c, lane, n0l, keys, L.page_keys, L.n_pages, &L.ctl->page_ctr,
                                            &L.ctl->err, pg_cur, pg_end, &off, &cntv);
                    lvalid = trig0;
                } else {
                    lvalid = 0u;
                }
                if (lane == 0) chunk_col[(int64_t)j0 * n_tiles] = make_uint2(off, cntv);
                if (nf == 2) {
                    __syncwarp();
                    // the second frame against the bounds after the first
                    uint32_t t1 = 0u;
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const int pq = q * 128 + lane * 4;
                        t1 |= outside4(*reinterpret_cast<const float4*>(v1 + pq),
                                       *reinterpret_cast<const float4*>(s.vu() + pq),
                                       *reinterpret_cast<const float4*>(s.vd() + pq))
                              << (q * 4);
                    }
                    t1 &= valid;
                    off = 0u;
                    cntv = 0u;
                    if (__any_sync(0xffffffffu, t1 != 0u)) {
                        s.lvm()[lane] = lvalid;
                        const int n1l = build_list<PPT>(t1, 0u, lane, s.list());
                        __syncwarp();
                        interval_of(ta0, D0, dt, j0 + 1, c.ta, c.Df);
                        c.vcur = v1;
                        c.vprev = v0;
                        slow_general<PPT, KeyT>(s, c, lane, n1l, keys, L.page_keys, L.n_pages, &L.ctl->page_ctr,
                                                &L.ctl->err, pg_cur, pg_end, &off, &cntv);
                        lvalid = t1;
                    } else {
                        lvalid = 0u;
                    }
                    if (lane == 0) chunk_col[(int64_t)(j0 + 1) * n_tiles] = make_uint2(off, cntv);
                }
            }
            __syncwarp();
        }

        // shared memory -> state
        const float* vl = s.vs((T - 1) % 3);
        for (int k = 0; k < PPT; ++k) {
            if (!((valid >> k) & 1u)) continue;
            const int p = (k >> 2) * 128 + lane * 4 + (k & 3);
            const int g = c.g0 + p;
            sdp->ref_out[g] = s.ref()[p];
            sdp->tlast_out[g] = s.tl()[p];
            sdp->lprev_out[g] = ((lvalid >> k) & 1u) ? s.lb()[p] : model_L(vl[p], c.eps, c.is_log);
        }
        __syncwarp();
    }
}
