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
              swizzle == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
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
};

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
            tma_load_2d(sB + s * B_BYTES, &g.tb, kt * SBK, 0, &full[s]);
        }
    } else if (tid == 32) {
        // MMA issuer
        for (int kt = 0; kt < n_kt; ++kt) {
            const int s = kt % ns;
            if (!umma::mbar_wait(&full[s], (uint32_t)((kt / ns) & 1), g.limit_ns)) {
                atomicOr(&s_fail, 1u);
                break;
            }
            umma::fence_after_sync();
            const uint32_t a0 = umma::smem_u32(sA + s * A_BYTES), b0 = umma::smem_u32(sB + s * B_BYTES);
#pragma unroll
            for (int k = 0; k < SBK / 16; ++k)
                umma::mma_bf16(tmem, desc_sw<SW>(a0, k), desc_sw<SW>(b0, k), idesc, (kt > 0 || k > 0) ? 1u : 0u);
            umma::mma_commit(&empty[s]);
        }
        umma::mma_commit(done);
    }
    bool ok = umma::mbar_wait(done, 0u, g.limit_ns);
    umma::fence_after_sync();
    ok = __syncthreads_and(ok && s_fail == 0u);
    if (ok) {
        const int r = warp * 32 + (tid & 31);
        const int row = g.a.row_of(tile, r);
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < BN; c += 8) {
            float v[8];
            umma::tmem_ld8(lane_addr + (uint32_t)c, v);
            if (row >= 0 && c < g.N) g.ep.store(row, c, v, 0);
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

}  // namespace utma
