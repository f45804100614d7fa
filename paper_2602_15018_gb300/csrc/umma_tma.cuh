// Tensor-core GEMM with TMA-loaded operands: D[M x N] = A[M x K] * B[K x N]
// where every K tile of A and B is one tensor-map box copied by the Tensor
// Memory Accelerator into 128-byte-swizzled shared memory, in a 4-stage
// pipeline with warp roles: one thread issues the TMA loads, one thread the
// tcgen05 MMAs, and all four warps drain TMEM in the epilogue.
//
// A comes from an "A loader" that maps (tile, K tile) to box coordinates and
// TMEM lane to output row: a dense row-major matrix, or the tap boxes of a
// 3 x 3 stride-1 convolution over BF16 NHWC activations (one box of 64
// channels x TW x TH pixels per tap and channel chunk; zero fill outside the
// image is the convolution's padding).  B is a packed K-major weight matrix.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "umma.cuh"

namespace utma {

constexpr int BM = 128;
constexpr int BK = 64;           // K of one 128-byte swizzle row of BF16
constexpr int STAGES = 4;
// K of one stage for a swizzle width SW (bytes): one swizzle row of BF16
__host__ __device__ constexpr int bk_of(int SW) { return SW / 2; }
constexpr uint32_t kErrTimeout = 1u;

// ---- host: tensor maps (driver entry point looked up through the runtime) -------------
// BF16 tiled map with a 128- or 64-byte swizzle and zero fill outside the
// tensor; strides_bytes has rank - 1 entries (dimension 0 is contiguous).
// elem_strides (optional, rank entries): traversal stride per dimension; a
// box then holds box[i] / elem_strides[i] elements along dimension i.
inline bool encode_tiled(CUtensorMap* map, int rank, const void* base, const cuuint64_t* dims,
                         const cuuint64_t* strides_bytes, const cuuint32_t* box, int swizzle = 128,
                         const cuuint32_t* elem_strides = nullptr)
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return false;
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    const cuuint32_t ones[5] = {1u, 1u, 1u, 1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), dims, strides_bytes,
              box, elem_strides ? elem_strides : ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
              swizzle == 0 ? CU_TENSOR_MAP_SWIZZLE_NONE
                           : swizzle == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// K-major BF16 matrix [rows][ld] (K = the first `K` columns) as a 2-D map,
// box (SW / 2, box_rows).
inline bool encode_kmajor(CUtensorMap* map, const void* base, int rows, int K, int box_rows, int swizzle = 128,
                          int ld = 0)
{
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld ? ld : K) * 2u};
    const cuuint32_t box[2] = {(cuuint32_t)bk_of(swizzle), (cuuint32_t)box_rows};
    return encode_tiled(map, 2, base, dims, strides, box, swizzle);
}

// ---- device helpers --------------------------------------------------------------------
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(umma::smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :: "r"(umma::smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1),
           "r"(umma::smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        :: "r"(umma::smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
           "r"(umma::smem_u32(mbar)) : "memory");
}

// K-major operand in the swizzled layout written by TMA: rows of SW bytes
// (SW / 2 BF16 of K), 8-row atoms of 8 SW bytes; k-step s (K = 16) starts
// 32 B further inside the row.  Layout type 2 = SWIZZLE_128B, 4 = SWIZZLE_64B.
template <int SW>
__device__ __forceinline__ uint64_t desc_sw(uint32_t saddr, int s)
{
    static_assert(SW == 128 || SW == 64, "128- or 64-byte swizzle");
    uint64_t d = umma::smem_desc(saddr + (uint32_t)s * 32u, 16u, 8u * SW);
    d |= (uint64_t)(SW == 128 ? 2u : 4u) << 61;
    return d;
}

// ---- A loaders ---------------------------------------------------------------------------
// Row-major A: row m is K values starting at column `off` of a [M][ld]
// matrix (a dense matrix, or the pixels x channels view of an NHWC buffer);
// 2-D map (ld, M), box (bk, 128).
struct DenseA {
    int M, K, off, bk;
    __host__ __device__ __forceinline__ int n_kt() const { return (K + bk - 1) / bk; }
    __device__ __forceinline__ void load(void* dst, const CUtensorMap* map, int tile, int kt, uint64_t* mbar) const
    {
        tma_load_2d(dst, map, off + kt * bk, tile * BM, mbar);
    }
    __device__ __forceinline__ int row_of(int tile, int r) const
    {
        const int m = tile * BM + r;
        return m < M ? m : -1;
    }
    // rows 32 w .. 32 w + 31 of a tile are pixels row0 .. row0 + 31 (n_valid exist)
    __device__ __forceinline__ bool warp_rows(int tile, int w, int& row0, int& n_valid) const
    {
        row0 = tile * BM + 32 * w;
        n_valid = M - row0;
        return true;
    }
};

// 3 x 3 convolution with padding 1 over NHWC activations (4-D map: channels
// of the buffer, W, H, N of the input; box bk x s TW x s TH x 1 with traversal
// stride s in W and H, so that one box holds TW x TH pixels).  Output tile =
// TW x TH pixels of one image; K tile = (tap, bk-channel chunk) of the view
// [off, off + C).
// flip = 0: out(y, x) reads in(s y + dy - 1, s x + dx - 1)      (forward)
// flip = 1: out(y, x) reads g(y + 1 - dy, x + 1 - dx), s = 1    (data gradient)
struct ConvTapA {
    int C, off, flip;
    int W, H, N;          // output size
    int TW, TH, tiles_x, tiles_y;
    int bk;               // channels per K tile (the swizzle row)
    int stride;           // 1 or 2
    __host__ __device__ __forceinline__ int n_kt() const { return 9 * (C / bk); }
    __device__ __forceinline__ void origin(int tile, int& n, int& x0, int& y0) const
    {
        const int per = tiles_x * tiles_y;
        n = tile / per;
        const int rem = tile - n * per;
        const int ty = rem / tiles_x;
        y0 = ty * TH;
        x0 = (rem - ty * tiles_x) * TW;
    }
    __device__ __forceinline__ void load(void* dst, const CUtensorMap* map, int tile, int kt, uint64_t* mbar) const
    {
        int n, x0, y0;
        origin(tile, n, x0, y0);
        const int cc = C / bk;
        const int tap = kt / cc, c = off + (kt - tap * cc) * bk;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        tma_load_4d(dst, map, c, flip ? x0 - dx : stride * x0 + dx, flip ? y0 - dy : stride * y0 + dy, n, mbar);
    }
    __device__ __forceinline__ int row_of(int tile, int r) const
    {
        int n, x0, y0;
        origin(tile, n, x0, y0);
        const int ty = r / TW, x = x0 + (r - ty * TW), y = y0 + ty;
        return (x < W && y < H) ? (n * H + y) * W + x : -1;
    }
    // as DenseA::warp_rows; consecutive only when a warp's 32 rows lie in one tile row
    __device__ __forceinline__ bool warp_rows(int tile, int w, int& row0, int& n_valid) const
    {
        if (TW % 32 != 0) return false;
        int n, x0, y0;
        origin(tile, n, x0, y0);
        const int r = 32 * w, ty = r / TW, x = x0 + (r - ty * TW), y = y0 + ty;
        row0 = (n * H + y) * W + x;
        n_valid = y < H ? W - x : 0;
        return true;
    }
};

// Data gradient of a 2 x 2 stride-2 transposed convolution: low-resolution
// pixel (y, x) takes sub-position (a, b) of the output gradient at
// (2y + a, 2x + b).  Output tile = TW x TH low-resolution pixels of one image;
// K tile = (sub-position ab = 2a + b, bk-channel chunk) of the gradient view
// [off, off + Cout).  4-D map of the gradient (channels of the buffer, 2 W,
// 2 H, N), box bk x 2 TW x 2 TH x 1 with traversal stride 2 in W and H, so
// that one box holds TW x TH pixels.  B is the packed [cin][ab * Cout + o].
struct S2DTapA {
    int Cout, off;
    int W, H, N;          // low-resolution size (the data gradient's)
    int TW, TH, tiles_x, tiles_y;
    int bk;
    __host__ __device__ __forceinline__ int n_kt() const { return 4 * (Cout / bk); }
    __device__ __forceinline__ void origin(int tile, int& n, int& x0, int& y0) const
    {
        const int per = tiles_x * tiles_y;
        n = tile / per;
        const int rem = tile - n * per;
        const int ty = rem / tiles_x;
        y0 = ty * TH;
        x0 = (rem - ty * tiles_x) * TW;
    }
    __device__ __forceinline__ void load(void* dst, const CUtensorMap* map, int tile, int kt, uint64_t* mbar) const
    {
        int n, x0, y0;
        origin(tile, n, x0, y0);
        const int cc = Cout / bk;
        const int ab = kt / cc, c = off + (kt - ab * cc) * bk;
        tma_load_4d(dst, map, c, 2 * x0 + (ab & 1), 2 * y0 + (ab >> 1), n, mbar);
    }
    __device__ __forceinline__ int row_of(int tile, int r) const
    {
        int n, x0, y0;
        origin(tile, n, x0, y0);
        const int ty = r / TW, x = x0 + (r - ty * TW), y = y0 + ty;
        return (x < W && y < H) ? (n * H + y) * W + x : -1;
    }
    __device__ __forceinline__ bool warp_rows(int tile, int w, int& row0, int& n_valid) const
    {
        if (TW % 32 != 0) return false;
        int n, x0, y0;
        origin(tile, n, x0, y0);
        const int r = 32 * w, ty = r / TW, x = x0 + (r - ty * TW), y = y0 + ty;
        row0 = (n * H + y) * W + x;
        n_valid = y < H ? W - x : 0;
        return true;
    }
};

// Data gradient of a 3 x 3 stride-2 convolution with padding 1, for the
// input pixels of one parity class (py, px).  Input pixel (2a + py, 2b + px)
// receives tap (dy, dx) of the output gradient at (a + oy, b + ox): for py = 0
// only dy = 1 (oy = 0), for py = 1 dy = 0 (oy = 1) and dy = 2 (oy = 0); the
// same along x.  So the classes hold 1, 2, 2 and 4 of the 9 taps and no
// product is a structural zero.  Output tile = TW x TH pixels (a, b) of the
// gradient's grid; K tile = (class tap t, bk-channel chunk).  4-D map of the
// gradient (channels of the buffer, Wo, Ho, N), box bk x TW x TH x 1; B (the
// packed [cin][tap * Cout + o] weights) is read at column tap * Cout + chunk.
struct ParityTapA {
    int Cout, off;        // gradient channels and their offset in the buffer
    int Wo, Ho, N;        // gradient grid (the convolution's output)
    int py, px;           // parity class of the input pixels written
    int TW, TH, tiles_x, tiles_y;
    int bk;
    int ntaps;
    int tap[4], ox[4], oy[4];
    __host__ __device__ __forceinline__ int n_kt() const { return ntaps * (Cout / bk); }
    __device__ __forceinline__ void origin(int tile, int& n, int& x0, int& y0) const
    {
        const int per = tiles_x * tiles_y;
        n = tile / per;
        const int rem = tile - n * per;
        const int ty = rem / tiles_x;
        y0 = ty * TH;
        x0 = (rem - ty * tiles_x) * TW;
    }
    __device__ __forceinline__ void load(void* dst, const CUtensorMap* map, int tile, int kt, uint64_t* mbar) const
    {
        int n, x0, y0;
        origin(tile, n, x0, y0);
        const int cc = Cout / bk;
        const int t = kt / cc, c = kt - t * cc;
        tma_load_4d(dst, map, off + c * bk, x0 + ox[t], y0 + oy[t], n, mbar);
    }
    __device__ __forceinline__ int b_col(int kt) const
    {
        const int cc = Cout / bk;
        const int t = kt / cc, c = kt - t * cc;
        return tap[t] * Cout + c * bk;
    }
    __device__ __forceinline__ int row_of(int tile, int r) const
    {
        int n, x0, y0;
        origin(tile, n, x0, y0);
        const int ty = r / TW, b = x0 + (r - ty * TW), a = y0 + ty;
        return (a < Ho && b < Wo) ? (n * 2 * Ho + 2 * a + py) * (2 * Wo) + 2 * b + px : -1;
    }
    __device__ __forceinline__ bool warp_rows(int, int, int&, int&) const { return false; }
};

// B column of K tile kt: the loader's b_col where it has one, else kt x the
// stage's K.
template <class AL, class = void>
struct al_bcol : std::false_type {};
template <class AL>
struct al_bcol<AL, std::void_t<decltype(std::declval<const AL&>().b_col(0))>> : std::true_type {};

// Epilogue of one accumulator row: 32 columns per TMEM load (one wait), then
// the epilogue functor on 8 columns at a time, unrolled so that the global
// loads some functors make (masks, accumulation) are in flight together.
template <int BN, class EP>
__device__ __forceinline__ void drain_row(uint32_t lane_addr, int row, int n_cols, const EP& ep)
{
    static_assert(BN % 16 == 0, "columns");
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        if (c0 + 32 <= BN) {
            umma::tmem_ld32(lane_addr + (uint32_t)c0, v);
        } else {
            float w[8];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                umma::tmem_ld8(lane_addr + (uint32_t)(c0 + 8 * q), w);
#pragma unroll
                for (int i = 0; i < 8; ++i) v[8 * q + i] = w[i];
            }
        }
        if (row < 0) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = c0 + 8 * q;
            if (c < BN && c < n_cols) {
                float u[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) u[i] = v[8 * q + i];
                ep.store(row, c, u, 0);
            }
        }
    }
}

// Epilogues that can also hand over 32 finished columns of one pixel as four
// 16-byte chunks (EP::kStaged, EP::pack32, EP::row_ptr) are drained through
// a per-warp shared-memory transpose: a plain drain stores 16 B of each of
// 32 pixels per instruction, half of a 32-byte sector each, while the staged
// drain stores 8 pixels x 64 contiguous bytes, whole sectors, and halves the
// L2 write requests.  The 32 rows of a warp must be consecutive pixels.
template <class EP, class = void>
struct ep_staged : std::false_type {};
template <class EP>
struct ep_staged<EP, std::void_t<decltype(EP::kStaged)>> : std::bool_constant<EP::kStaged> {};

constexpr int kStageU4 = 4 * 32 * 4;   // 4 epilogue warps x 32 pixels x 4 chunks of 16 B

// Drains TMEM columns [0, BN) of the warp's 32 lanes (= pixels row0 .. row0 +
// 31, of which the first n_valid exist) through stage (128 uint4 of this
// warp).  n_cols must be a multiple of 32.
template <int BN, class EP>
__device__ __forceinline__ void drain_row_staged(uint32_t lane_addr, int row0, int n_valid, int n_cols, const EP& ep,
                                                 uint4* stage, int lane)
{
    static_assert(BN % 32 == 0, "columns");
    // destination rows of this lane's four stores, once per tile
    decltype(ep.base_ptr(0)) base[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int px = 8 * i + (lane >> 2);
        base[i] = px < n_valid ? ep.base_ptr(row0 + px) : ep.base_ptr(row0);
    }
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        umma::tmem_ld32(lane_addr + (uint32_t)c0, v);
        if (c0 >= n_cols) continue;                                   // warp-uniform
        uint4 o[4];
        ep.pack32(c0, v, o);
        // chunk q of pixel l at l * 4 + (q ^ ((l >> 1) & 3)): conflict-free both ways
#pragma unroll
        for (int q = 0; q < 4; ++q) stage[lane * 4 + (q ^ ((lane >> 1) & 3))] = o[q];
        __syncwarp();
        const size_t co = ep.col_offset(c0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int px = 8 * i + (lane >> 2), q = lane & 3;
            const uint4 val = stage[px * 4 + (q ^ ((px >> 1) & 3))];
            if (px < n_valid) *reinterpret_cast<uint4*>(base[i] + co + 8 * q) = val;
        }
        __syncwarp();
    }
}

template <class AL, class EP>
struct TmaArgs {
    CUtensorMap ta;       // A map
    CUtensorMap tb;       // B map: packed weights (K, N), box (64, BN)
    AL a;
    EP ep;
    int N;                // real columns (<= BN)
    unsigned int* err;
    uint64_t limit_ns;
};

// Dynamic shared memory of a launch with `ns` pipeline stages.
template <int BN, int SW = 128>
__host__ __device__ constexpr size_t tma_smem_bytes(int ns = STAGES)
{
    return 1024 + (size_t)ns * (BM * SW + BN * SW) + 256;
}

template <int BN, int SW, class AL, class EP>
__global__ void __launch_bounds__(128) tma_gemm_kernel(const __grid_constant__ TmaArgs<AL, EP> g)
{
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 N for M = 128");
    constexpr uint32_t TCOLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    constexpr int SBK = bk_of(SW);
    constexpr uint32_t A_BYTES = BM * SW, B_BYTES = BN * SW;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment of the swizzled tiles
    unsigned char* smem = smem_raw + ((1024u - (umma::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tile = blockIdx.x;
    const int n_kt = g.a.n_kt();
    // stages in use: no more than the K tiles (the launch sized the shared memory so)
    const int ns = n_kt < STAGES ? (n_kt > 0 ? n_kt : 1) : STAGES;
    unsigned char* sA = smem;
    unsigned char* sB = smem + ns * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + ns * B_BYTES);
    uint64_t* empty = full + ns;
    uint64_t* done = empty + ns;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);

    if (tid == 0) {
        for (int s = 0; s < ns; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        umma::mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) umma::tmem_alloc(tslot, TCOLS);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, BN, false, false);

    __shared__ unsigned int s_fail;
    __shared__ uint4 s_stage[ep_staged<EP>::value ? kStageU4 : 1];
    if (tid == 0) s_fail = 0u;
    __syncthreads();
    if (tid == 0) {
        // producer: TMA loads of A and B, one stage ahead of the tensor core
        for (int kt = 0; kt < n_kt; ++kt) {
            const int s = kt % ns;
            if (kt >= ns &&
                !umma::mbar_wait(&empty[s], (uint32_t)((kt / ns - 1) & 1), g.limit_ns)) {
                atomicOr(&s_fail, 1u);
                break;
            }
            mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
            g.a.load(sA + s * A_BYTES, &g.ta, tile, kt, &full[s]);
            if constexpr (al_bcol<AL>::value)
                tma_load_2d(sB + s * B_BYTES, &g.tb, g.a.b_col(kt), 0, &full[s]);
            else
                tma_load_2d(sB + s * B_BYTES, &g.tb, kt * SBK, 0, &full[s]);
        }
    } else if (tid == 32) {
        // MMA issuer: stage-0 descriptors once, a stage adds its offset to the
        // start-address field
        const uint64_t da0 = desc_sw<SW>(umma::smem_u32(sA), 0), db0 = desc_sw<SW>(umma::smem_u32(sB), 0);
        for (int kt = 0; kt < n_kt; ++kt) {
            const int s = kt % ns;
            if (!umma::mbar_wait(&full[s], (uint32_t)((kt / ns) & 1), g.limit_ns)) {
                atomicOr(&s_fail, 1u);
                break;
            }
            umma::fence_after_sync();
            const uint64_t oa = (uint64_t)(((uint32_t)s * A_BYTES) >> 4), ob = (uint64_t)(((uint32_t)s * B_BYTES) >> 4);
#pragma unroll
            for (int k = 0; k < SBK / 16; ++k)
                umma::mma_bf16(tmem, da0 + oa + (uint64_t)(k * 2), db0 + ob + (uint64_t)(k * 2), idesc,
                               (kt > 0 || k > 0) ? 1u : 0u);
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
        int row0 = 0, n_valid = 0;
        if constexpr (ep_staged<EP>::value) {
            if (g.N % 32 == 0 && g.a.warp_rows(tile, warp, row0, n_valid))
                drain_row_staged<BN>(lane_addr, row0, n_valid, g.N, g.ep, s_stage + warp * 128, tid & 31);
            else
                drain_row<BN>(lane_addr, g.a.row_of(tile, r), g.N, g.ep);
        } else {
            drain_row<BN>(lane_addr, g.a.row_of(tile, r), g.N, g.ep);
        }
    } else if (tid == 0) {
        atomicOr(g.err, kErrTimeout);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, TCOLS);
}

template <int BN, int SW, class AL, class EP>
cudaError_t launch_tma_gemm(const TmaArgs<AL, EP>& g, int tiles, cudaStream_t stream)
{
    const int n_kt = g.a.n_kt();
    const int ns = n_kt < STAGES ? (n_kt > 0 ? n_kt : 1) : STAGES;
    cudaError_t e = cudaFuncSetAttribute(tma_gemm_kernel<BN, SW, AL, EP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes<BN, SW>());
    if (e != cudaSuccess) return e;
    tma_gemm_kernel<BN, SW, AL, EP><<<tiles, 128, tma_smem_bytes<BN, SW>(ns), stream>>>(g);
    return cudaGetLastError();
}


// ---- 3 x 3 stride-1 convolution from a halo tile ----------------------------------------
// Output tile: 128 consecutive pixels x0 .. x0 + 127 of row y0 of image n
// (W >= 128; the last tile of a row may reach past W: its halo reads the zero
// fill and its rows past W are not stored).  The A operands of all 9 taps come from one halo
// tile: the channel view [off, off + C) of rows y0 - 1 .. y0 + 1 and pixels
// x0 - 1 .. x0 + 128, brought in by TMA as C / 8 planes of 3 x 130 pixels x 8
// channels (16 bytes per pixel, no swizzle; zero fill outside the image is
// the padding), planes padded to 128-byte multiples.  Inside a plane the
// pixels of the three rows follow each other 16 bytes apart, so the
// 128 x 16 operand of tap (dy, dx) and channel group g is a canonical
// no-swizzle K-major matrix that starts (row * 130 + col) * 16 bytes into
// plane 2g: core matrices of 8 pixels x 16 bytes, SBO = 128 bytes (next 8
// pixels), LBO = one plane (next 8 channels).  Each input pixel is read from
// L2 once per tile instead of once per tap.
// With a 128- or 64-byte swizzle (SWA = 128 or 64, C a multiple of SWA / 2)
// the halo instead comes as C / (SWA / 2) boxes of 3 x 130 pixels x SWA / 2
// channels (rows of SWA bytes, far fewer TMA rows).  The operand of tap
// (dy, dx) then starts on a pixel row that is not 8-row aligned; the tensor
// core applies the swizzle by shared-memory address bits, as the TMA wrote
// it, so such a start needs no base offset (measured on GB300: base offset
// (start >> 7) & 7 gave wrong results, 0 gives exact ones).
// With 8 channels (one plane) a K = 16 step takes two taps: the second core
// matrix along K is the same plane shifted to the next tap, so LBO is the
// distance between the two taps' start rows; the 9th tap pairs with the
// zero-filled weight columns 72..79 (and the plane's zeroed padding rows).
// flip = 0: out(y, x) reads in(y + dy - 1, x + dx - 1)          (forward)
// flip = 1: out(y, x) reads g(y + 1 - dy, x + 1 - dx)           (data gradient)
//
// Persistent, warp-specialised CTA of 6 warps: warp 4 loads (the packed
// weights of all taps once, then one halo per tile into two alternating
// buffers), warp 5 issues the MMAs of a tile into one of two TMEM
// accumulators, warps 0-3 drain the other accumulator through the epilogue.
// So the next tile's halo load and MMAs overlap this tile's epilogue.
constexpr int kHaloW = 130;                         // 128 + 2 pixels
constexpr uint32_t kHaloPlane = 3 * kHaloW * 16;    // 6240 bytes written per plane
constexpr uint32_t kHaloPlaneStride = (kHaloPlane + 127u) / 128u * 128u;
constexpr int kHaloThreads = 192;
// one halo box of the swizzled forms: 390 rows of SWA bytes, padded to 1024
__host__ __device__ constexpr uint32_t halo_box_bytes(int SWA) { return 3u * kHaloW * (uint32_t)SWA; }
__host__ __device__ constexpr uint32_t halo_box_stride(int SWA) { return (halo_box_bytes(SWA) + 1023u) / 1024u * 1024u; }

__host__ __device__ constexpr uint32_t halo_bytes_of(int C, int SWA)
{
    return SWA ? (uint32_t)(C / (SWA / 2)) * halo_box_stride(SWA) : (uint32_t)(C / 8) * kHaloPlaneStride;
}

template <class EP>
struct HaloArgs {
    CUtensorMap ta;       // NHWC activations: (cstride, W, H, N), box (8, 130, 3, 1), no swizzle
    CUtensorMap tb;       // packed weights (9C, n_out), box (bk, BN)
    EP ep;
    int C, off, flip;
    int W, H, N;          // image size (input = output)
    int n_tiles;
    int n_out;            // real columns (<= BN)
    unsigned int* err;
    uint64_t limit_ns;
};

template <int BN, int SW, int SWA>
__host__ __device__ constexpr size_t halo_smem_bytes(int C)
{
    return 1024 + (size_t)((9 * C + bk_of(SW) - 1) / bk_of(SW)) * BN * SW + 2 * (size_t)halo_bytes_of(C, SWA) + 256;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(mbar)) : "memory");
}

template <int BN, int SW, int SWA, int CC, class EP>
__global__ void __launch_bounds__(kHaloThreads) halo_conv_kernel(const __grid_constant__ HaloArgs<EP> g)
{
    static_assert(SWA == 0 || SWA == 64 || SWA == 128, "halo layouts");
    static_assert((CC == 8 && SWA == 0) || (CC % 16 == 0 && CC % (SWA ? SWA / 2 : 1) == 0 && CC % bk_of(SW) == 0),
                  "channels");
    constexpr int HC = SWA ? SWA / 2 : 8;           // channels per halo box
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "tcgen05 N for M = 128, two accumulators");
    constexpr uint32_t TC = BN <= 32 ? 32 : BN <= 64 ? 64 : 128;    // columns of one accumulator
    constexpr int SBK = bk_of(SW);
    constexpr uint32_t B_BYTES = BN * SW;           // one K tile of the weights
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (umma::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int planes = CC / 8;
    constexpr int n_kt = (9 * CC + SBK - 1) / SBK;             // K tiles of the weights (zero-filled tail)
    constexpr uint32_t halo_bytes = halo_bytes_of(CC, SWA);
    unsigned char* sB = smem;                                   // 1024-aligned swizzled tiles
    unsigned char* sA = smem + (size_t)n_kt * B_BYTES;          // two halo buffers
    uint64_t* bar = reinterpret_cast<uint64_t*>(sA + 2 * (size_t)halo_bytes);
    uint64_t* bfull = bar;          // weights landed
    uint64_t* afull = bar + 1;      // [2] halo landed
    uint64_t* aempty = bar + 3;     // [2] halo consumed by the MMAs
    uint64_t* tfull = bar + 5;      // [2] accumulator complete
    uint64_t* tempty = bar + 7;     // [2] accumulator drained by the epilogue
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 9);
    __shared__ unsigned int s_fail;
    __shared__ uint4 s_stage[ep_staged<EP>::value ? kStageU4 : 1];
    const int tiles_x = (g.W + 127) / 128;
    const int per = g.H * tiles_x;

    if (tid == 0) {
        s_fail = 0u;
        umma::mbar_init(bfull, 1);
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(&afull[b], 1);
            umma::mbar_init(&aempty[b], 1);
            umma::mbar_init(&tfull[b], 1);
            umma::mbar_init(&tempty[b], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (CC == 8 && tid < 2 * (int)((kHaloPlaneStride - kHaloPlane) / 16)) {
        // the rows past the plane's 390 (read, times zero weights, by the 9th tap)
        constexpr int per_buf = (int)((kHaloPlaneStride - kHaloPlane) / 16);
        *reinterpret_cast<uint4*>(sA + (size_t)(tid / per_buf) * halo_bytes + kHaloPlane + (tid % per_buf) * 16) =
            make_uint4(0u, 0u, 0u, 0u);
        umma::fence_async_smem();
    }
    if (warp == 0) umma::tmem_alloc(tslot, 2 * TC);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, BN, false, false);

    if (warp == 4) {
        if (lane == 0) {
            // producer: the weights once, then one halo per tile
            uint32_t issued = 0;
            mbar_expect_tx(bfull, (uint32_t)n_kt * B_BYTES);
            for (int kt = 0; kt < n_kt; ++kt) tma_load_2d(sB + (size_t)kt * B_BYTES, &g.tb, kt * SBK, 0, bfull);
            uint32_t i = 0;
            for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
                const uint32_t b = i & 1u, use = i >> 1;
                if (i >= 2 && !umma::mbar_wait(&aempty[b], (use - 1u) & 1u, g.limit_ns)) {
                    atomicOr(&s_fail, 1u);
                    break;
                }
                if (*(volatile unsigned int*)&s_fail) break;
                issued = i + 1;
                const int n = tile / per;
                const int rem = tile - n * per;
                const int y0 = rem / tiles_x;
                const int x0 = (rem - y0 * tiles_x) * 128;
                unsigned char* dst = sA + (size_t)b * halo_bytes;
                if (SWA) {
                    mbar_expect_tx(&afull[b], (uint32_t)(CC / HC) * halo_box_bytes(SWA));
                    for (int p = 0; p < CC / HC; ++p)
                        tma_load_4d(dst + (size_t)p * halo_box_stride(SWA), &g.ta, g.off + HC * p, x0 - 1, y0 - 1,
                                    n, &afull[b]);
                } else {
                    mbar_expect_tx(&afull[b], (uint32_t)planes * kHaloPlane);
                    for (int p = 0; p < planes; ++p)
                        tma_load_4d(dst + (size_t)p * kHaloPlaneStride, &g.ta, g.off + 8 * p, x0 - 1, y0 - 1, n,
                                    &afull[b]);
                }
            }
            if (*(volatile unsigned int*)&s_fail) {
                // let the copies in flight land before the CTA leaves (bounded)
                umma::mbar_wait(bfull, 0u, g.limit_ns);
                for (uint32_t j = issued >= 2 ? issued - 2 : 0; j < issued; ++j)
                    umma::mbar_wait(&afull[j & 1u], (j >> 1) & 1u, g.limit_ns);
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer: 9 taps x C / 16 channel groups per tile
            bool ok = umma::mbar_wait(bfull, 0u, g.limit_ns);
            uint32_t i = 0;
            for (int tile = blockIdx.x; ok && tile < g.n_tiles; tile += gridDim.x, ++i) {
                const uint32_t b = i & 1u, use = i >> 1;
                ok = umma::mbar_wait(&afull[b], use & 1u, g.limit_ns) &&
                     (i < 2 || umma::mbar_wait(&tempty[b], (use - 1u) & 1u, g.limit_ns));
                if (!ok || *(volatile unsigned int*)&s_fail) break;
                umma::fence_after_sync();
                // descriptors differ from the tile's first ones only in the
                // start-address field: add (byte offset >> 4)
                const uint32_t a0 = umma::smem_u32(sA + (size_t)b * halo_bytes), b0 = umma::smem_u32(sB);
                const uint64_t ad0 = SWA == 128  ? (umma::smem_desc(a0, 16u, 1024u) | ((uint64_t)2u << 61))
                                     : SWA == 64 ? (umma::smem_desc(a0, 16u, 512u) | ((uint64_t)4u << 61))
                                                 : umma::smem_desc(a0, kHaloPlaneStride, 128u);
                const uint64_t bd0 = desc_sw<SW>(b0, 0);
                const uint32_t d = tmem + b * TC;
                if (CC == 8) {
                    // tap pairs (2j, 2j + 1) per K = 16 step; tap 9 is the zero weight tail
#pragma unroll
                    for (int j = 0; j < 5; ++j) {
                        const int t0 = 2 * j, t1 = 2 * j + 1;
                        const int s0 = g.flip ? (2 - t0 / 3) * kHaloW + (2 - t0 % 3) : (t0 / 3) * kHaloW + t0 % 3;
                        const int s1 = t1 < 9 ? (g.flip ? (2 - t1 / 3) * kHaloW + (2 - t1 % 3)
                                                        : (t1 / 3) * kHaloW + t1 % 3)
                                              : s0 + 1;
                        const uint64_t adesc =
                            umma::smem_desc(a0 + (uint32_t)s0 * 16u, (uint32_t)(s1 - s0) * 16u, 128u);
                        const uint32_t boff = (uint32_t)((16 * j) / SBK) * B_BYTES + (uint32_t)((16 * j % SBK) / 16) * 32u;
                        umma::mma_bf16(d, adesc, bd0 + (boff >> 4), idesc, j > 0 ? 1u : 0u);
                    }
                }
#pragma unroll
                for (int tap = 0; tap < (CC == 8 ? 0 : 9); ++tap) {
                    const int dy = tap / 3, dx = tap % 3;
                    const uint32_t shift = (uint32_t)(g.flip ? (2 - dy) * kHaloW + (2 - dx) : dy * kHaloW + dx);
#pragma unroll
                    for (int c16 = 0; c16 < CC / 16; ++c16) {
                        constexpr int KS = HC / 16;           // K steps of 16 per swizzled row
                        const uint32_t aoff = SWA ? (uint32_t)(c16 / KS) * halo_box_stride(SWA) + shift * (uint32_t)SWA +
                                                        (uint32_t)(c16 % KS) * 32u
                                                  : (uint32_t)(2 * c16) * kHaloPlaneStride + shift * 16u;
                        const int kt = tap * (CC / SBK) + (c16 * 16) / SBK;
                        const uint32_t boff = (uint32_t)kt * B_BYTES + (uint32_t)((c16 * 16 % SBK) / 16) * 32u;
                        umma::mma_bf16(d, ad0 + (aoff >> 4), bd0 + (boff >> 4), idesc,
                                       (tap > 0 || c16 > 0) ? 1u : 0u);
                    }
                }
                umma::mma_commit(&aempty[b]);
                umma::mma_commit(&tfull[b]);
            }
            if (!ok) atomicOr(&s_fail, 1u);
        }
    } else {
        // epilogue warps 0-3: TMEM lanes 32 w .. 32 w + 31 = tile rows
        uint32_t i = 0;
        for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
            const uint32_t b = i & 1u, use = i >> 1;
            bool ok = umma::mbar_wait(&tfull[b], use & 1u, g.limit_ns);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) atomicOr(&s_fail, 1u);
                break;
            }
            umma::fence_after_sync();
            const int n = tile / per;
            const int rem = tile - n * per;
            const int y0 = rem / tiles_x;
            const int x0 = (rem - y0 * tiles_x) * 128;
            const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16) + b * TC;
            if constexpr (ep_staged<EP>::value) {
                const int xw = x0 + warp * 32;
                drain_row_staged<BN>(lane_addr, (n * g.H + y0) * g.W + xw, g.W - xw, g.n_out, g.ep,
                                     s_stage + warp * 128, lane);
            } else {
                const int x = x0 + warp * 32 + lane;
                const int row = x < g.W ? (n * g.H + y0) * g.W + x : -1;
                drain_row<BN>(lane_addr, row, g.n_out, g.ep);
            }
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (tid == 0 && s_fail) atomicOr(g.err, kErrTimeout);
    if (warp == 0) umma::tmem_dealloc(tmem, 2 * TC);
}

// CTAs of a persistent kernel that fit on one SM at once: registers (per-warp
// allocation in units of 256), shared memory (with the per-block reserve),
// threads, and the SM's 512 TMEM columns.  Computed from the kernel's
// attributes: the runtime's occupancy query returned 1 for these kernels on
// GB300 where the SM holds up to 6 of them (the profiler's own limits).
inline cudaError_t resident_per_sm(const void* fn, int threads, size_t dyn_smem, int tmem_cols, int* per_sm)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, reserved = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess)
        return e;
    const int warps = (threads + 31) / 32;
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    int n = warp_regs > 0 ? regs_sm / warp_regs / warps : 32;
    n = std::min(n, (int)((size_t)smem_sm / (dyn_smem + fa.sharedSizeBytes + (size_t)reserved)));
    n = std::min(n, thr_sm / threads);
    n = std::min(n, 512 / tmem_cols);
    n = std::min(n, 32);
    *per_sm = n;
    return n >= 1 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <int BN, int SW, int SWA, int CC, class EP>
cudaError_t launch_halo_conv(const HaloArgs<EP>& g, int num_sms, cudaStream_t stream)
{
    if (g.C != CC || (ep_staged<EP>::value && g.n_out % 32 != 0)) return cudaErrorInvalidValue;
    const size_t smem = halo_smem_bytes<BN, SW, SWA>(CC);
    cudaError_t e = cudaFuncSetAttribute(halo_conv_kernel<BN, SW, SWA, CC, EP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // resident CTAs must also fit in the SM's 512 TMEM columns (2 accumulators each)
    constexpr int tc = BN <= 32 ? 32 : BN <= 64 ? 64 : 128;
    int per_sm = 0;
    e = resident_per_sm(reinterpret_cast<const void*>(halo_conv_kernel<BN, SW, SWA, CC, EP>), kHaloThreads, smem,
                        2 * tc, &per_sm);
    if (e != cudaSuccess) return e;
    const int grid = std::min(g.n_tiles, num_sms * per_sm);
    halo_conv_kernel<BN, SW, SWA, CC, EP><<<grid, kHaloThreads, smem, stream>>>(g);
    return cudaGetLastError();
}

// ---- 3 x 3 stride-1 convolution from halo tiles, weights streamed ---------------------------
// For inputs whose weights of all taps do not fit in shared memory beside two
// halos (C a multiple of 64 with 128 output channels, or C = 128): the halo of
// a tile comes one 64-channel box (3 x 130 pixels, 128-byte swizzle) at a time
// through a ring of two box slots, and the weights one (tap, 64-channel) K
// tile at a time through a ring of halo_stream_stages<BN>() stages.  The K
// loop of a tile runs box by box, tap by tap; tile t + 1's first box loads
// while tile t's second box is multiplied.  Taps are shifted descriptors into
// the box as in halo_conv_kernel; warps as there (4 = loads, 5 = MMAs, 0-3 =
// epilogue, two TMEM accumulators).
//
// Every tile re-reads its weights from L2.  The ring holds 4 K tiles: 12
// stages (64 output channels) measured no faster on GB300, and 7 (128 output
// channels) 12 % slower.
constexpr size_t kHaloSmemMax = 227u * 1024u;   // dynamic shared memory per CTA
constexpr size_t kHaloStreamTail = 512;         // barriers (4 + 2 S + 4) and the TMEM slot
constexpr int kHaloStreamMaxStages = 4;

template <int BN>
__host__ __device__ constexpr int halo_stream_stages()
{
    constexpr size_t room = kHaloSmemMax - 1024 - 2 * (size_t)halo_box_stride(128) - kHaloStreamTail;
    return room / ((size_t)BN * 128) < (size_t)kHaloStreamMaxStages ? (int)(room / ((size_t)BN * 128))
                                                                     : kHaloStreamMaxStages;
}

template <int BN>
__host__ __device__ constexpr size_t halo_stream_smem_bytes()
{
    return 1024 + 2 * (size_t)halo_box_stride(128) + (size_t)halo_stream_stages<BN>() * BN * 128 + kHaloStreamTail;
}

template <int BN, int CC, class EP>
__global__ void __launch_bounds__(kHaloThreads) halo_conv_stream_kernel(const __grid_constant__ HaloArgs<EP> g)
{
    static_assert(CC % 64 == 0 && BN % 16 == 0 && BN >= 16 && BN <= 128, "shape");
    constexpr uint32_t TC = BN <= 32 ? 32 : BN <= 64 ? 64 : 128;
    constexpr int NBOX = CC / 64;
    constexpr int S = halo_stream_stages<BN>();
    static_assert(S >= 2 && (4 + 2 * S + 4) * 8 + 4 <= (int)kHaloStreamTail, "weight ring");
    static_assert(halo_stream_smem_bytes<BN>() <= kHaloSmemMax, "shared memory");
    constexpr uint32_t B_BYTES = BN * 128;           // one (tap, 64-channel) K tile of the weights
    constexpr uint32_t BOX = halo_box_stride(128);
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (umma::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* sA = smem;                        // two box slots
    unsigned char* sB = smem + 2 * (size_t)BOX;      // weight stages
    uint64_t* bar = reinterpret_cast<uint64_t*>(sB + (size_t)S * B_BYTES);
    uint64_t* afull = bar;                           // [2] box landed
    uint64_t* aempty = bar + 2;                      // [2] box consumed
    uint64_t* bfull = bar + 4;                       // [S] weight tile landed
    uint64_t* bempty = bfull + S;                    // [S] weight tile consumed
    uint64_t* tfull = bempty + S;                    // [2] accumulator complete
    uint64_t* tempty = tfull + 2;                    // [2] accumulator drained
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
    __shared__ unsigned int s_fail;
    __shared__ uint4 s_stage[ep_staged<EP>::value ? kStageU4 : 1];
    const int tiles_x = (g.W + 127) / 128;
    const int per = g.H * tiles_x;

    if (tid == 0) {
        s_fail = 0u;
        for (int k = 0; k < 2; ++k) {
            umma::mbar_init(&afull[k], 1);
            umma::mbar_init(&aempty[k], 1);
            umma::mbar_init(&tfull[k], 1);
            umma::mbar_init(&tempty[k], 4);
        }
        for (int k = 0; k < S; ++k) {
            umma::mbar_init(&bfull[k], 1);
            umma::mbar_init(&bempty[k], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) umma::tmem_alloc(tslot, 2 * TC);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, BN, false, false);

    if (warp == 4) {
        if (lane == 0) {
            // producer: per tile, per box: the box, then its 9 weight tiles
            uint32_t ia = 0, ib = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < g.n_tiles; tile += gridDim.x) {
                const int n = tile / per;
                const int rem = tile - n * per;
                const int y0 = rem / tiles_x;
                const int x0 = (rem - y0 * tiles_x) * 128;
                for (int box = 0; ok && box < NBOX; ++box) {
                    const uint32_t sa = ia & 1u, ua = ia >> 1;
                    if (ia >= 2 && !umma::mbar_wait(&aempty[sa], (ua - 1u) & 1u, g.limit_ns)) {
                        ok = false;
                        break;
                    }
                    if (*(volatile unsigned int*)&s_fail) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&afull[sa], halo_box_bytes(128));
                    tma_load_4d(sA + (size_t)sa * BOX, &g.ta, g.off + 64 * box, x0 - 1, y0 - 1, n, &afull[sa]);
                    ++ia;
                    for (int tap = 0; tap < 9; ++tap) {
                        const uint32_t sb = ib % S, ub = ib / S;
                        if (ib >= S && !umma::mbar_wait(&bempty[sb], (ub - 1u) & 1u, g.limit_ns)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&bfull[sb], B_BYTES);
                        tma_load_2d(sB + (size_t)sb * B_BYTES, &g.tb, tap * CC + 64 * box, 0, &bfull[sb]);
                        ++ib;
                    }
                }
            }
            if (!ok) {
                atomicOr(&s_fail, 1u);
                // let the copies in flight land before the CTA leaves (bounded)
                for (uint32_t j = ia >= 2 ? ia - 2 : 0; j < ia; ++j)
                    umma::mbar_wait(&afull[j & 1u], (j >> 1) & 1u, g.limit_ns);
                for (uint32_t j = ib >= (uint32_t)S ? ib - S : 0; j < ib; ++j)
                    umma::mbar_wait(&bfull[j % S], (j / S) & 1u, g.limit_ns);
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer: per tile, per box, per tap, 4 K = 16 steps inside the box's 128-byte rows
            uint32_t ia = 0, ib = 0, it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < g.n_tiles; tile += gridDim.x, ++it) {
                const uint32_t b = it & 1u, use = it >> 1;
                if (it >= 2 && !umma::mbar_wait(&tempty[b], (use - 1u) & 1u, g.limit_ns)) {
                    ok = false;
                    break;
                }
                const uint32_t d = tmem + b * TC;
                int k = 0;
                for (int box = 0; ok && box < NBOX; ++box) {
                    const uint32_t sa = ia & 1u, ua = ia >> 1;
                    if (!umma::mbar_wait(&afull[sa], ua & 1u, g.limit_ns) || *(volatile unsigned int*)&s_fail) {
                        ok = false;
                        break;
                    }
                    ++ia;
                    const uint32_t a0 = umma::smem_u32(sA + (size_t)sa * BOX);
                    const uint64_t ad0 = umma::smem_desc(a0, 16u, 1024u) | ((uint64_t)2u << 61);
                    for (int tap = 0; tap < 9; ++tap) {
                        const uint32_t sb = ib % S, ub = ib / S;
                        if (!umma::mbar_wait(&bfull[sb], ub & 1u, g.limit_ns)) {
                            ok = false;
                            break;
                        }
                        ++ib;
                        umma::fence_after_sync();
                        const uint64_t bd0 = desc_sw<128>(umma::smem_u32(sB + (size_t)sb * B_BYTES), 0);
                        const int dy = tap / 3, dx = tap % 3;
                        const uint32_t shift = (uint32_t)(g.flip ? (2 - dy) * kHaloW + (2 - dx) : dy * kHaloW + dx);
#pragma unroll
                        for (int c16 = 0; c16 < 4; ++c16, ++k) {
                            const uint32_t aoff = shift * 128u + (uint32_t)c16 * 32u;
                            umma::mma_bf16(d, ad0 + (aoff >> 4), bd0 + (((uint32_t)c16 * 32u) >> 4), idesc,
                                           k > 0 ? 1u : 0u);
                        }
                        umma::mma_commit(&bempty[sb]);
                    }
                    if (ok) umma::mma_commit(&aempty[sa]);
                }
                if (ok) umma::mma_commit(&tfull[b]);
            }
            if (!ok) atomicOr(&s_fail, 1u);
        }
    } else {
        // epilogue warps 0-3: TMEM lanes 32 w .. 32 w + 31 = tile rows
        uint32_t it = 0;
        for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++it) {
            const uint32_t b = it & 1u, use = it >> 1;
            bool ok = umma::mbar_wait(&tfull[b], use & 1u, g.limit_ns);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) atomicOr(&s_fail, 1u);
                break;
            }
            umma::fence_after_sync();
            const int n = tile / per;
            const int rem = tile - n * per;
            const int y0 = rem / tiles_x;
            const int x0 = (rem - y0 * tiles_x) * 128;
            const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16) + b * TC;
            if constexpr (ep_staged<EP>::value) {
                const int xw = x0 + warp * 32;
                drain_row_staged<BN>(lane_addr, (n * g.H + y0) * g.W + xw, g.W - xw, g.n_out, g.ep,
                                     s_stage + warp * 128, lane);
            } else {
                const int x = x0 + warp * 32 + lane;
                const int row = x < g.W ? (n * g.H + y0) * g.W + x : -1;
                drain_row<BN>(lane_addr, row, g.n_out, g.ep);
            }
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (tid == 0 && s_fail) atomicOr(g.err, kErrTimeout);
    if (warp == 0) umma::tmem_dealloc(tmem, 2 * TC);
}

template <int BN, int CC, class EP>
cudaError_t launch_halo_conv_stream(const HaloArgs<EP>& g, int num_sms, cudaStream_t stream)
{
    if (g.C != CC || (ep_staged<EP>::value && g.n_out % 32 != 0)) return cudaErrorInvalidValue;
    constexpr size_t smem = halo_stream_smem_bytes<BN>();
    cudaError_t e = cudaFuncSetAttribute(halo_conv_stream_kernel<BN, CC, EP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    constexpr int tc = BN <= 32 ? 32 : BN <= 64 ? 64 : 128;
    int per_sm = 0;
    e = resident_per_sm(reinterpret_cast<const void*>(halo_conv_stream_kernel<BN, CC, EP>), kHaloThreads, smem,
                        2 * tc, &per_sm);
    if (e != cudaSuccess) return e;
    const int grid = std::min(g.n_tiles, num_sms * per_sm);
    halo_conv_stream_kernel<BN, CC, EP><<<grid, kHaloThreads, smem, stream>>>(g);
    return cudaGetLastError();
}


// ---- persistent GEMM over pixel rows (1x1 and transposed convolutions) -------------------
// D[128 x BN] per tile of 128 consecutive rows of A ([M][lda] BF16, columns
// off .. off + K, 2-D map (lda, M), box (bk, 128)); B = the packed weights
// [BN][K] (box (bk, BN)), loaded once and kept in shared memory.  As the halo
// kernels: warp 4 loads A tiles into a ring of kPixStages stages, warp 5
// issues the MMAs into one of two TMEM accumulators, warps 0-3 drain the other
// one, so a CTA's loads, MMAs and epilogue overlap across tiles.
constexpr int kPixStages = 3;

template <class EP>
struct PixArgs {
    CUtensorMap ta, tb;
    EP ep;
    int M, K, off;
    int n_tiles, n_out;
    unsigned int* err;
    uint64_t limit_ns;
};

template <int BN, int SW>
__host__ __device__ constexpr size_t pix_smem_bytes(int K)
{
    return 1024 + (size_t)((K + bk_of(SW) - 1) / bk_of(SW)) * (BN + kPixStages * BM) * SW + 256;
}

template <int BN, int SW, class EP>
__global__ void __launch_bounds__(kHaloThreads) pix_gemm_kernel(const __grid_constant__ PixArgs<EP> g)
{
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 N for M = 128");
    constexpr uint32_t TC = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    constexpr int SBK = bk_of(SW);
    constexpr uint32_t A_BYTES = BM * SW, B_BYTES = BN * SW;
    constexpr int S = kPixStages;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (umma::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_kt = (g.K + SBK - 1) / SBK;
    unsigned char* sB = smem;                                    // n_kt weight tiles
    unsigned char* sA = smem + (size_t)n_kt * B_BYTES;           // S stages of n_kt tiles
    uint64_t* bar = reinterpret_cast<uint64_t*>(sA + (size_t)S * n_kt * A_BYTES);
    uint64_t* bfull = bar;              // weights landed
    uint64_t* afull = bar + 1;          // [S] A stage landed
    uint64_t* aempty = afull + S;       // [S] A stage consumed
    uint64_t* tfull = aempty + S;       // [2] accumulator complete
    uint64_t* tempty = tfull + 2;       // [2] accumulator drained
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
    __shared__ unsigned int s_fail;

    if (tid == 0) {
        s_fail = 0u;
        umma::mbar_init(bfull, 1);
        for (int s = 0; s < S; ++s) {
            umma::mbar_init(&afull[s], 1);
            umma::mbar_init(&aempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(&tfull[b], 1);
            umma::mbar_init(&tempty[b], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) umma::tmem_alloc(tslot, 2 * TC);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, BN, false, false);

    if (warp == 4) {
        if (lane == 0) {
            // producer: the weights once, then the A tiles of this CTA's row tiles
            uint32_t issued = 0;
            mbar_expect_tx(bfull, (uint32_t)n_kt * B_BYTES);
            for (int kt = 0; kt < n_kt; ++kt) tma_load_2d(sB + (size_t)kt * B_BYTES, &g.tb, kt * SBK, 0, bfull);
            uint32_t i = 0;
            for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
                const uint32_t s = i % S, use = i / S;
                if (i >= (uint32_t)S && !umma::mbar_wait(&aempty[s], (use - 1u) & 1u, g.limit_ns)) {
                    atomicOr(&s_fail, 1u);
                    break;
                }
                if (*(volatile unsigned int*)&s_fail) break;
                issued = i + 1;
                mbar_expect_tx(&afull[s], (uint32_t)n_kt * A_BYTES);
                for (int kt = 0; kt < n_kt; ++kt)
                    tma_load_2d(sA + ((size_t)s * n_kt + kt) * A_BYTES, &g.ta, g.off + kt * SBK, tile * BM,
                                &afull[s]);
            }
            if (*(volatile unsigned int*)&s_fail) {
                // let the copies in flight land before the CTA leaves (bounded)
                umma::mbar_wait(bfull, 0u, g.limit_ns);
                for (uint32_t j = issued >= (uint32_t)S ? issued - S : 0; j < issued; ++j)
                    umma::mbar_wait(&afull[j % S], (j / S) & 1u, g.limit_ns);
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            bool ok = umma::mbar_wait(bfull, 0u, g.limit_ns);
            uint32_t i = 0;
            for (int tile = blockIdx.x; ok && tile < g.n_tiles; tile += gridDim.x, ++i) {
                const uint32_t s = i % S, b = i & 1u;
                ok = umma::mbar_wait(&afull[s], (i / S) & 1u, g.limit_ns) &&
                     (i < 2 || umma::mbar_wait(&tempty[b], ((i >> 1) - 1u) & 1u, g.limit_ns));
                if (!ok || *(volatile unsigned int*)&s_fail) break;
                umma::fence_after_sync();
                const uint32_t a0 = umma::smem_u32(sA + (size_t)s * n_kt * A_BYTES), b0 = umma::smem_u32(sB);
                const uint32_t d = tmem + b * TC;
                for (int kt = 0; kt < n_kt; ++kt) {
#pragma unroll
                    for (int k = 0; k < SBK / 16; ++k)
                        umma::mma_bf16(d, desc_sw<SW>(a0 + (uint32_t)kt * A_BYTES, k),
                                       desc_sw<SW>(b0 + (uint32_t)kt * B_BYTES, k), idesc, (kt > 0 || k > 0) ? 1u : 0u);
                }
                umma::mma_commit(&aempty[s]);
                umma::mma_commit(&tfull[b]);
            }
            if (!ok) atomicOr(&s_fail, 1u);
        }
    } else {
        // epilogue warps 0-3: TMEM lanes 32 w .. 32 w + 31 = tile rows
        uint32_t i = 0;
        for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, ++i) {
            const uint32_t b = i & 1u;
            bool ok = umma::mbar_wait(&tfull[b], (i >> 1) & 1u, g.limit_ns);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) atomicOr(&s_fail, 1u);
                break;
            }
            umma::fence_after_sync();
            const int row = tile * BM + warp * 32 + lane;
            const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16) + b * TC;
            drain_row<BN>(lane_addr, row < g.M ? row : -1, g.n_out, g.ep);
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (tid == 0 && s_fail) atomicOr(g.err, kErrTimeout);
    if (warp == 0) umma::tmem_dealloc(tmem, 2 * TC);
}

template <int BN, int SW, class EP>
cudaError_t launch_pix_gemm(const PixArgs<EP>& g, int num_sms, cudaStream_t stream)
{
    const size_t smem = pix_smem_bytes<BN, SW>(g.K);
    if (g.K < 1 || smem > 227u * 1024u) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(pix_gemm_kernel<BN, SW, EP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    constexpr int tc = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    int per_sm = 0;
    e = resident_per_sm(reinterpret_cast<const void*>(pix_gemm_kernel<BN, SW, EP>), kHaloThreads, smem, 2 * tc,
                        &per_sm);
    if (e != cudaSuccess) return e;
    const int grid = std::min(g.n_tiles, num_sms * per_sm);
    if (grid < 1) return cudaSuccess;
    pix_gemm_kernel<BN, SW, EP><<<grid, kHaloThreads, smem, stream>>>(g);
    return cudaGetLastError();
}

}  // namespace utma
