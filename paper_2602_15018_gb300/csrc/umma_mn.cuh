// Tensor-core GEMM over pixels with MN-major operands loaded by TMA, for the
// weight gradients of the learned interpolator's layers:
//   D[M x N] += sum over pixels p of A(m, p) B(n, p)
// where A and B are BF16 NHWC activations (or shifted / strided views of
// them) whose rows are channels.  K = pixels, enumerated in K tiles of 64
// consecutive pixels of one image row (one "pixel run"); the last run of a
// row may reach past the image, where the TMA zero fill makes its products 0.
//
// Each K tile of an operand is assembled from "parts": one TMA box of cb
// channels x 64 pixels each, cb = 64, 32 or 8 channels for a 128-byte,
// 64-byte or no swizzle.  In shared memory a part is 64 pixel rows of
// 2 * cb bytes, channel-contiguous: an MN-major operand whose MN atom (cb
// channels) is one part.  The tensor core reads it through an MN-major
// descriptor: for the swizzled forms the leading byte offset is the step
// between parts (MN atoms) and the stride byte offset the step between
// 8-pixel groups (8 rows of 2 * cb bytes); without swizzle the two swap
// roles (leading = next 8-pixel group, stride = next 8-channel atom).
//
// Operand kinds (rows of the operand = the GEMM's M or N dimension):
//   kPix   rows c of the channel view [off, off + C) at pixel (n, y, x)
//   kConv3 rows (tap, c) of a 3x3 convolution with padding 1 and stride s:
//          input pixel (n, s y + dy - 1, s x + dx - 1), tap = 3 dy + dx
//          (the im2col view of the convolution's input over its output
//          pixels; out-of-image coordinates read the zero fill)
//   kS2D   rows (2a + b, c) of a 2x2 stride-2 transposed convolution's
//          output gradient at low-resolution pixel (n, y, x): high-resolution
//          pixel (n, 2y + a, 2x + b)
// A part never straddles two taps or sub-positions (cb divides C).
//
// One CTA of 128 threads computes a 128 x BN tile of D over one slice of
// the K tiles (the grid's y dimension; the partial tiles are added into an
// FP32 result with atomics).  Thread 0 issues the TMA loads into a 4-stage
// ring, thread 32 the MMAs, and all four warps drain TMEM.  Every wait is
// bounded: on timeout the CTA records an error bit and returns after its
// MMAs (bounded) and its TMEM release.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "umma.cuh"
#include "umma_tma.cuh"

namespace umn {

constexpr int BM = 128;
constexpr int KT = 64;          // pixels per K tile
constexpr int STAGES = 4;
constexpr int kMaxParts = 32;
constexpr uint32_t kErrTimeout = 1u;

enum { kPix = 0, kConv3 = 1, kS2D = 2 };

// One operand: its kind, channel view and swizzle.
struct MnOp {
    int kind;
    int C;       // channels per tap / sub-position (rows = taps * C)
    int off;     // first channel of the view in the buffer
    int s;       // convolution stride (kConv3)
    int rows;    // operand rows that exist (M or N)
    int sw;      // 128, 64 or 0 (bytes of a swizzle row; 0: none)
    __host__ __device__ int cb() const { return sw == 128 ? 64 : sw == 64 ? 32 : 8; }
    __host__ __device__ uint32_t part_bytes() const { return (uint32_t)KT * (uint32_t)cb() * 2u; }
};

// K tiles: runs of 64 pixels of the GEMM's pixel grid (n, y, x), Ho x Wo per
// image; run kt is (n, y, xb) with xb fastest.
struct MnGeom {
    int Ho, Wo, xblocks, n_kt;
};

// Descriptor of K step st (16 pixels) of an operand tile at saddr.
__device__ __forceinline__ uint64_t desc_mn(uint32_t saddr, int sw, int st)
{
    if (sw == 0) {
        // 8-pixel groups of 8 x 16 B = 128 B, 8-channel atoms 1 KB apart
        return umma::smem_desc(saddr + (uint32_t)st * 256u, 128u, 1024u);
    }
    const uint32_t row = (uint32_t)sw;                  // bytes per pixel row of a part
    uint64_t d = umma::smem_desc(saddr + (uint32_t)st * 16u * row, (uint32_t)KT * row, 8u * row);
    d |= (uint64_t)(sw == 128 ? 2u : 4u) << 61;
    return d;
}

// The parts of operand tile rows [r0, r0 + nrows) as box offsets: part j
// of K tile (n, y, x0) is the box at (channel off + c0, step x0 + ox,
// step y + oy, n), step = 2 for strided views (kConv3 with s = 2, kS2D).
// Parts whose first row is at or past op.rows are left out.  Returns the
// part count; the offsets do not depend on the K tile, so the producer
// computes them once.
__device__ __forceinline__ int part_table(const MnOp& op, int r0, int nrows, int4* tab)
{
    const int cb = op.cb();
    int np = 0;
    for (int j = 0; j * cb < nrows && j < kMaxParts; ++j) {
        const int r = r0 + j * cb;
        if (r >= op.rows) break;
        const int grp = r / op.C, c0 = r - grp * op.C;
        int ox = 0, oy = 0;
        if (op.kind == kConv3) {
            ox = grp % 3 - 1;
            oy = grp / 3 - 1;
        } else if (op.kind == kS2D) {
            ox = grp & 1;
            oy = grp >> 1;
        }
        tab[np++] = make_int4(op.off + c0, ox, oy, 0);
    }
    return np;
}

__device__ __forceinline__ int op_step(const MnOp& op)
{
    return (op.kind == kS2D || (op.kind == kConv3 && op.s == 2)) ? 2 : 1;
}

template <int BN>
struct MnArgs {
    CUtensorMap ta, tb;
    MnOp a, b;
    MnGeom geom;
    int M, N;              // D is M x N (row-major, ld N), N <= BN, N % 8 == 0
    int kt_per_split;
    float* dw;
    unsigned int* err;
    uint64_t limit_ns;
};

template <int BN>
__host__ __device__ constexpr size_t mn_stage_bytes()
{
    return (size_t)BM * KT * 2 + (size_t)BN * KT * 2;
}

// Dynamic shared memory of a launch with `ns` stages: alignment, the ring,
// the barriers, and 8 KB of slack after them, so that a descriptor read
// never leaves the CTA's allocation.
template <int BN>
__host__ __device__ constexpr size_t mn_smem_bytes(int ns = STAGES)
{
    return 1024 + (size_t)ns * mn_stage_bytes<BN>() + 256 + 8192;
}

template <int BN>
__global__ void __launch_bounds__(128) mn_gemm_kernel(const __grid_constant__ MnArgs<BN> g)
{
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 N for M = 128");
    constexpr uint32_t TCOLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    constexpr uint32_t A_BYTES = BM * KT * 2, STAGE = (uint32_t)mn_stage_bytes<BN>();
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (umma::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * BM;
    const int kb = blockIdx.y * g.kt_per_split;
    const int ke = min(g.geom.n_kt, kb + g.kt_per_split);
    const int n_kt = ke > kb ? ke - kb : 0;
    if (n_kt == 0) return;                       // nothing to add (block-uniform)
    const int ns = n_kt < STAGES ? n_kt : STAGES;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)ns * STAGE);
    uint64_t* empty = full + ns;
    uint64_t* done = empty + ns;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ unsigned int s_fail;

    if (tid == 0) {
        for (int s = 0; s < ns; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        umma::mbar_init(done, 1);
        s_fail = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) umma::tmem_alloc(tslot, TCOLS);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, BN, true, true);

    if (tid == 0) {
        // producer: all parts of A and B of a K tile complete one stage; the
        // K tile's pixel run (n, y, xb) advances without divisions
        int4 ta[kMaxParts], tb[kMaxParts];
        const int npa = part_table(g.a, m0, BM, ta), npb = part_table(g.b, 0, BN, tb);
        const int sa = op_step(g.a), sb = op_step(g.b);
        const uint32_t pa = g.a.part_bytes(), pb = g.b.part_bytes();
        const uint32_t bytes = (uint32_t)npa * pa + (uint32_t)npb * pb;
        int xb = kb % g.geom.xblocks, y = (kb / g.geom.xblocks) % g.geom.Ho, n = kb / g.geom.xblocks / g.geom.Ho;
        for (int i = 0; i < n_kt; ++i) {
            const int s = i % ns;
            if (i >= ns && !umma::mbar_wait(&empty[s], (uint32_t)((i / ns - 1) & 1), g.limit_ns)) {
                atomicOr(&s_fail, 1u);
                break;
            }
            unsigned char* st = smem + (size_t)s * STAGE;
            utma::mbar_expect_tx(&full[s], bytes);
            const int x0 = xb * KT;
            for (int j = 0; j < npa; ++j)
                utma::tma_load_4d(st + (size_t)j * pa, &g.ta, ta[j].x, sa * x0 + ta[j].y, sa * y + ta[j].z, n,
                                  &full[s]);
            for (int j = 0; j < npb; ++j)
                utma::tma_load_4d(st + A_BYTES + (size_t)j * pb, &g.tb, tb[j].x, sb * x0 + tb[j].y,
                                  sb * y + tb[j].z, n, &full[s]);
            if (++xb == g.geom.xblocks) {
                xb = 0;
                if (++y == g.geom.Ho) {
                    y = 0;
                    ++n;
                }
            }
        }
    } else if (tid == 32) {
        // MMA issuer: the descriptors of stage 0, once; a stage adds its
        // offset to the start-address field (no carry: shared addresses are
        // below 256 KB)
        const uint32_t base = umma::smem_u32(smem);
        uint64_t da[KT / 16], db[KT / 16];
#pragma unroll
        for (int k = 0; k < KT / 16; ++k) {
            da[k] = desc_mn(base, g.a.sw, k);
            db[k] = desc_mn(base + A_BYTES, g.b.sw, k);
        }
        for (int i = 0; i < n_kt; ++i) {
            const int s = i % ns;
            if (!umma::mbar_wait(&full[s], (uint32_t)((i / ns) & 1), g.limit_ns)) {
                atomicOr(&s_fail, 1u);
                break;
            }
            umma::fence_after_sync();
            const uint64_t off = (uint64_t)(((uint32_t)s * STAGE) >> 4);
#pragma unroll
            for (int k = 0; k < KT / 16; ++k)
                umma::mma_bf16(tmem, da[k] + off, db[k] + off, idesc, (i > 0 || k > 0) ? 1u : 0u);
            umma::mma_commit(&empty[s]);
        }
        umma::mma_commit(done);
    }
    bool ok = umma::mbar_wait(done, 0u, g.limit_ns);
    umma::fence_after_sync();
    ok = __syncthreads_and(ok && s_fail == 0u);
    if (ok) {
        const int row = m0 + warp * 32 + (tid & 31);
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        float* d = g.dw + (size_t)row * g.N;
#pragma unroll 1
        for (int c = 0; c < g.N; c += 8) {
            float v[8];
            umma::tmem_ld8(lane_addr + (uint32_t)c, v);
            if (row < g.M) {
#pragma unroll
                for (int i = 0; i < 8; ++i) atomicAdd(d + c + i, v[i]);
            }
        }
    } else if (tid == 0) {
        atomicOr(g.err, kErrTimeout);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, TCOLS);
}

// ---- host ------------------------------------------------------------------------------
// Swizzle of an operand view of C channels per tap (C a multiple of 8).
inline int pick_sw(int C) { return C % 64 == 0 ? 128 : C % 32 == 0 ? 64 : 0; }

// 4-D map of a BF16 NHWC buffer (stride channels per pixel, W x H x N) for the
// parts of `op`: box cb channels x 64 * step pixels x 1 x 1, traversal step
// 2 along W for strided views (kConv3 with s = 2, kS2D).
inline bool encode_op(CUtensorMap* map, const void* base, int stride, int W, int H, int N, const MnOp& op)
{
    const int step = (op.kind == kS2D || (op.kind == kConv3 && op.s == 2)) ? 2 : 1;
    const cuuint64_t dims[4] = {(cuuint64_t)stride, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)stride * 2u, (cuuint64_t)stride * 2u * W,
                                   (cuuint64_t)stride * 2u * W * H};
    const cuuint32_t box[4] = {(cuuint32_t)op.cb(), (cuuint32_t)(KT * step), 1u, 1u};
    const cuuint32_t es[4] = {1u, (cuuint32_t)step, 1u, 1u};
    return utma::encode_tiled(map, 4, base, dims, strides, box, op.sw, es);
}

// Adds the K-tile slices' partial tiles into dw (M x N, FP32, row-major).
// `ctas` is the grid size to aim for (K tiles are split to reach it).
template <int BN>
cudaError_t launch_mn_gemm(MnArgs<BN>& g, int ctas, cudaStream_t stream)
{
    const int mt = (g.M + BM - 1) / BM;
    const int want = ctas > mt ? (ctas + mt - 1) / mt : 1;
    g.kt_per_split = (g.geom.n_kt + want - 1) / want;
    if (g.kt_per_split < 1) g.kt_per_split = 1;
    const int splits = (g.geom.n_kt + g.kt_per_split - 1) / g.kt_per_split;
    const int ns = g.kt_per_split < STAGES ? g.kt_per_split : STAGES;
    cudaError_t e = cudaFuncSetAttribute(mn_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mn_smem_bytes<BN>());
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)mt, (unsigned)(splits > 0 ? splits : 1));
    mn_gemm_kernel<BN><<<grid, 128, mn_smem_bytes<BN>(ns), stream>>>(g);
    return cudaGetLastError();
}

}  // namespace umn

namespace umn {

// ---- weight gradient of a 3x3 stride-1 convolution from a halo -----------------------
// D rows (tap, c) for one 64-channel part cp of the input view, all 9 taps,
// against B = the output gradient (BN <= 64 channels, pixel boxes).  Per K
// tile (64 output pixels of row y) one TMA box brings the input rows
// y - 1 .. y + 1, pixels x0 - 1 .. x0 + 70, 64 channels: 3 x 72 rows of
// 128 bytes, 128-byte swizzle.  The operand of tap (dy, dx) is that halo
// from row dy * 72 + dx on: an MN-major operand whose 8-pixel groups are
// 1024 B apart, starting inside a swizzle atom (the tensor core swizzles by
// address, as the TMA wrote it).  Taps are paired into M = 128 MMAs: the
// second tap is the second MN atom, at a leading byte offset equal to the
// distance between the two taps' first rows.  Tap 8 pairs with the halo
// shifted one more pixel, whose rows the epilogue drops.  Five FP32
// accumulators of BN columns stay in TMEM for the CTA's whole K slice.
constexpr int kHaloRows = 72;                       // pixels x0 - 1 .. x0 + 70 of a halo row
constexpr uint32_t kHaloBytes = 3u * kHaloRows * 128u;

template <int BN>
struct MnHaloArgs {
    CUtensorMap ta, tb;
    int C, off;            // input view: C channels (multiple of 64) at `off`
    MnOp b;                // output gradient (kPix), rows = BN
    MnGeom geom;
    int N;                 // gradient columns (<= BN)
    int kt_per_split;
    float* dw;             // [(tap, c)][N]
    unsigned int* err;
    uint64_t limit_ns;
};

template <int BN>
__host__ __device__ constexpr size_t mn_halo_stage_bytes()
{
    return (size_t)kHaloBytes + (size_t)BN * KT * 2;
}

template <int BN>
__host__ __device__ constexpr size_t mn_halo_smem_bytes(int ns = STAGES)
{
    return 1024 + (size_t)ns * mn_halo_stage_bytes<BN>() + 256 + 8192;
}

__device__ __forceinline__ uint32_t tap_row(int t) { return (uint32_t)((t / 3) * kHaloRows + t % 3); }

template <int BN>
__global__ void __launch_bounds__(128) mn_halo_kernel(const __grid_constant__ MnHaloArgs<BN> g)
{
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 64, "five accumulators of BN columns in 512 TMEM columns");
    constexpr uint32_t TCOLS = 5 * BN <= 256 ? 256 : 512;
    constexpr uint32_t STAGE = (uint32_t)mn_halo_stage_bytes<BN>();
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (umma::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int cp = blockIdx.x;                   // 64-channel part of the input view
    const int kb = blockIdx.y * g.kt_per_split;
    const int ke = min(g.geom.n_kt, kb + g.kt_per_split);
    const int n_kt = ke > kb ? ke - kb : 0;
    if (n_kt == 0) return;
    const int ns = n_kt < STAGES ? n_kt : STAGES;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)ns * STAGE);
    uint64_t* empty = full + ns;
    uint64_t* done = empty + ns;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ unsigned int s_fail;

    if (tid == 0) {
        for (int s = 0; s < ns; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        umma::mbar_init(done, 1);
        s_fail = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) umma::tmem_alloc(tslot, TCOLS);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, BN, true, true);

    if (tid == 0) {
        const int nbp = (BN + g.b.cb() - 1) / g.b.cb();
        const uint32_t pb = g.b.part_bytes();
        const int nb = (g.b.rows + g.b.cb() - 1) / g.b.cb() < nbp ? (g.b.rows + g.b.cb() - 1) / g.b.cb() : nbp;
        const uint32_t bytes = kHaloBytes + (uint32_t)nb * pb;
        int xb = kb % g.geom.xblocks, y = (kb / g.geom.xblocks) % g.geom.Ho, n = kb / g.geom.xblocks / g.geom.Ho;
        for (int i = 0; i < n_kt; ++i) {
            const int s = i % ns;
            if (i >= ns && !umma::mbar_wait(&empty[s], (uint32_t)((i / ns - 1) & 1), g.limit_ns)) {
                atomicOr(&s_fail, 1u);
                break;
            }
            unsigned char* st = smem + (size_t)s * STAGE;
            utma::mbar_expect_tx(&full[s], bytes);
            const int x0 = xb * KT;
            utma::tma_load_4d(st, &g.ta, g.off + cp * 64, x0 - 1, y - 1, n, &full[s]);
            for (int j = 0; j < nb; ++j)
                utma::tma_load_4d(st + kHaloBytes + (size_t)j * pb, &g.tb, g.b.off + j * g.b.cb(), x0, y, n, &full[s]);
            if (++xb == g.geom.xblocks) {
                xb = 0;
                if (++y == g.geom.Ho) {
                    y = 0;
                    ++n;
                }
            }
        }
    } else if (tid == 32) {
        // MMA issuer: every descriptor is a stage-0 descriptor plus constants
        // (start address >> 4 in bits 0-13, leading byte offset >> 4 in bits
        // 16-29), so that issuing an MMA costs a 64-bit add
        const uint32_t base = umma::smem_u32(smem);
        const uint64_t dh = umma::smem_desc(base, 0u, 1024u) | ((uint64_t)2u << 61);
        uint64_t db[KT / 16];
#pragma unroll
        for (int k = 0; k < KT / 16; ++k) db[k] = desc_mn(base + kHaloBytes, g.b.sw, k);
        for (int i = 0; i < n_kt; ++i) {
            const int s = i % ns;
            if (!umma::mbar_wait(&full[s], (uint32_t)((i / ns) & 1), g.limit_ns)) {
                atomicOr(&s_fail, 1u);
                break;
            }
            umma::fence_after_sync();
            const uint64_t off = (uint64_t)(((uint32_t)s * STAGE) >> 4);
#pragma unroll
            for (int p = 0; p < 5; ++p) {
                const uint32_t ra = tap_row(2 * p), rb = p < 4 ? tap_row(2 * p + 1) : ra + 1u;
#pragma unroll
                for (int k = 0; k < KT / 16; ++k) {
                    const uint64_t add = (uint64_t)((ra * 128u + (uint32_t)k * 2048u) >> 4) |
                                         ((uint64_t)(((rb - ra) * 128u) >> 4) << 16);
                    umma::mma_bf16(tmem + (uint32_t)(p * BN), dh + add + off, db[k] + off, idesc,
                                   (i > 0 || k > 0) ? 1u : 0u);
                }
            }
            umma::mma_commit(&empty[s]);
        }
        umma::mma_commit(done);
    }
    bool ok = umma::mbar_wait(done, 0u, g.limit_ns);
    umma::fence_after_sync();
    ok = __syncthreads_and(ok && s_fail == 0u);
    if (ok) {
        const int r = warp * 32 + (tid & 31);
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int p = 0; p < 5; ++p) {
            const int tap = 2 * p + (r >= 64 ? 1 : 0);
            const int row = tap * g.C + cp * 64 + (r & 63);
            float* d = g.dw + (size_t)row * g.N;
#pragma unroll 1
            for (int c = 0; c < g.N; c += 8) {
                float v[8];
                umma::tmem_ld8(lane_addr + (uint32_t)(p * BN + c), v);
                if (tap < 9) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) atomicAdd(d + c + q, v[q]);
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(g.err, kErrTimeout);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, TCOLS);
}

// Halo map of the input view: box 64 channels x 72 pixels x 3 rows x 1.
inline bool encode_halo(CUtensorMap* map, const void* base, int stride, int W, int H, int N)
{
    const cuuint64_t dims[4] = {(cuuint64_t)stride, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)stride * 2u, (cuuint64_t)stride * 2u * W,
                                   (cuuint64_t)stride * 2u * W * H};
    const cuuint32_t box[4] = {64u, (cuuint32_t)kHaloRows, 3u, 1u};
    return utma::encode_tiled(map, 4, base, dims, strides, box, 128);
}

template <int BN>
cudaError_t launch_mn_halo(MnHaloArgs<BN>& g, int ctas, cudaStream_t stream)
{
    const int parts = g.C / 64;
    const int want = ctas > parts ? (ctas + parts - 1) / parts : 1;
    g.kt_per_split = (g.geom.n_kt + want - 1) / want;
    if (g.kt_per_split < 1) g.kt_per_split = 1;
    const int splits = (g.geom.n_kt + g.kt_per_split - 1) / g.kt_per_split;
    const int ns = g.kt_per_split < STAGES ? g.kt_per_split : STAGES;
    cudaError_t e = cudaFuncSetAttribute(mn_halo_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mn_halo_smem_bytes<BN>());
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)parts, (unsigned)(splits > 0 ? splits : 1));
    mn_halo_kernel<BN><<<grid, 128, mn_halo_smem_bytes<BN>(ns), stream>>>(g);
    return cudaGetLastError();
}

}  // namespace umn
