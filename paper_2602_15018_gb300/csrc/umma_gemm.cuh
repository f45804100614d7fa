// Tensor-core GEMM core with gathered operands: D[M x N] = A[M x K] * B[K x N]
// with A and B produced tile by tile into shared memory by "gather" functors
// (dense matrices, or implicit im2col views of NHWC activations), FP32
// accumulation in TMEM, and an epilogue functor that consumes the FP32 tile.
//
// One CTA of 128 threads computes a 128 x BN tile of D over a K range (the
// grid's y dimension splits K for reductions over pixels).  The K loop is
// double buffered: the threads gather K-tile k+1 while the tensor core works
// on K-tile k; one thread issues the MMAs and commits them to the stage's
// mbarrier, which gates the reuse of that stage.  Every wait is bounded: on
// timeout the CTA records an error bit, waits (bounded) for its MMAs, frees
// its TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "umma.cuh"

namespace ugemm {

constexpr int BM = 128;   // rows of D per CTA (TMEM lanes)
constexpr int BK = 64;    // K per pipeline stage (4 MMAs of K = 16)
constexpr uint32_t kErrTimeout = 1u;

// ---- operand tiles in shared memory (no swizzle, see umma.cuh) -------------------
// Byte offset of the 16-byte chunk holding elements (r, k..k+7) of a K-major
// tile, or (r..r+7, k) of an MN-major tile with R rows.
__device__ __forceinline__ uint32_t kmajor_chunk(int r, int k)
{
    return (uint32_t)((r >> 3) * (BK / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16);
}

template <int R>
__device__ __forceinline__ uint32_t mnmajor_chunk(int r, int k)
{
    return (uint32_t)((r >> 3) * 128 + (k >> 3) * (R / 8) * 128 + (k & 7) * 16);
}

// Descriptor of the k-step s (K = 16) of a tile at saddr (G::MN: layout of
// the gather G).  In both layouts the leading byte offset is the step
// between core matrices that are adjacent along K and the stride byte
// offset the step between core matrices adjacent along M (or N).
template <class G, int R>
__device__ __forceinline__ uint64_t tile_desc(uint32_t saddr, int s)
{
    if (!G::MN) {
        // K-major: K-adjacent core matrices 128 B apart, 8-row groups BK / 8 * 128 B
        return umma::smem_desc(saddr + (uint32_t)s * 256u, 128u, (uint32_t)(BK / 8) * 128u);
    } else {
        // MN-major: 8-deep K groups R / 8 * 128 B apart, MN-adjacent core matrices 128 B
        const uint32_t kstep = (uint32_t)(R / 8) * 128u;
        return umma::smem_desc(saddr + (uint32_t)s * 2u * kstep, kstep, 128u);
    }
}

__device__ __forceinline__ void st_chunk(unsigned char* tile, uint32_t off, uint4 v)
{
    *reinterpret_cast<uint4*>(tile + off) = v;
}

// ---- the kernel ---------------------------------------------------------------------
template <class AG, class BG, class EP>
struct GemmArgs {
    AG a;               // gathers A tiles: rows = M, in its own major
    BG b;               // gathers B tiles: rows = N
    EP ep;              // consumes D rows
    int M, N, K;        // logical sizes (N <= BN; K multiple of 8)
    int k_per_split;    // K range of one grid.y slice (multiple of BK)
    unsigned int* err;  // error bits (kErrTimeout)
    uint64_t limit_ns;  // bound of every wait
};

template <int BN>
__host__ __device__ constexpr size_t gemm_smem_bytes()
{
    return (size_t)2 * BM * BK * 2 + (size_t)2 * BN * BK * 2 + 64;
}

template <int BN, class AG, class BG, class EP>
__global__ void __launch_bounds__(128) gemm_kernel(const __grid_constant__ GemmArgs<AG, BG, EP> g)
{
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 N for M = 128");
    constexpr uint32_t TCOLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                       // [2][A_BYTES]
    unsigned char* sB = smem + 2 * A_BYTES;         // [2][B_BYTES]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + 2 * B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * BM;
    const int kb = blockIdx.y * g.k_per_split;
    const int ke = min(g.K, kb + g.k_per_split);
    const int n_kt = ke > kb ? (ke - kb + BK - 1) / BK : 0;

    if (tid == 0) {
        umma::mbar_init(&mbar[0], 1);
        umma::mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) umma::tmem_alloc(tslot, TCOLS);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, BN, AG::MN, BG::MN);

    // per-thread row coordinates of this tile, computed once
    typename AG::template Rows<BM> ra;
    typename BG::template Rows<BN> rb;
    g.a.template prep<BM>(ra, m0, tid);
    g.b.template prep<BN>(rb, 0, tid);

    bool ok = true;
    for (int kt = 0; kt < n_kt; ++kt) {
        const int st = kt & 1;
        if (kt >= 2) {
            // the MMAs of K-tile kt - 2 used this stage
            if (!umma::mbar_wait(&mbar[st], (uint32_t)(((kt - 2) >> 1) & 1), g.limit_ns)) ok = false;
        }
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        g.a.template gather<BM>(sA + st * A_BYTES, ra, m0, kb + kt * BK, min(BK, ke - kb - kt * BK), tid);
        g.b.template gather<BN>(sB + st * B_BYTES, rb, 0, kb + kt * BK, min(BK, ke - kb - kt * BK), tid);
        umma::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            const uint32_t a0 = umma::smem_u32(sA + st * A_BYTES), b0 = umma::smem_u32(sB + st * B_BYTES);
#pragma unroll
            for (int s = 0; s < BK / 16; ++s)
                umma::mma_bf16(tmem, tile_desc<AG, BM>(a0, s), tile_desc<BG, BN>(b0, s), idesc,
                               (kt > 0 || s > 0) ? 1u : 0u);
            umma::mma_commit(&mbar[st]);
        }
    }
    // wait for the last MMAs (stage of tile n_kt - 1; also n_kt - 2 if the loop broke early)
    if (n_kt > 0) {
        const int last = n_kt - 1;
        if (!umma::mbar_wait(&mbar[last & 1], (uint32_t)((last >> 1) & 1), g.limit_ns)) ok = false;
        if (n_kt > 1 && !umma::mbar_wait(&mbar[(last - 1) & 1], (uint32_t)(((last - 1) >> 1) & 1), g.limit_ns))
            ok = false;
    }
    umma::fence_after_sync();
    ok = __syncthreads_and(ok);
    if (ok) {
        const int row = m0 + warp * 32 + (tid & 31);
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < BN; c += 8) {
            float v[8];
            if (n_kt > 0) {
                umma::tmem_ld8(lane_addr + (uint32_t)c, v);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = 0.0f;
            }
            if (row < g.M && c < g.N) g.ep.store(row, c, v, blockIdx.y);
        }
    } else if (tid == 0) {
        atomicOr(g.err, kErrTimeout);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, TCOLS);
}

// ---- dense operands (row-major, leading dimension ld) ------------------------------
// Gathers without per-row state declare an empty row cache.
#define UGEMM_NO_ROWS                                                      \
    template <int R>                                                       \
    struct Rows {};                                                        \
    template <int R>                                                       \
    __device__ __forceinline__ void prep(Rows<R>&, int, int) const {}

// K-major: row r of the operand is src[r * ld + k].
struct DenseK {
    static constexpr bool MN = false;
    UGEMM_NO_ROWS
    const __nv_bfloat16* src;
    int rows, ld;
    template <int R>
    __device__ __forceinline__ void gather(unsigned char* tile, const Rows<R>&, int r0, int k0, int kn, int tid) const
    {
        // R rows x BK: chunks (r, kc)
        for (int i = tid; i < R * (BK / 8); i += 128) {
            const int r = i / (BK / 8), kc = i % (BK / 8);
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (r0 + r < rows && kc * 8 < kn)
                v = *reinterpret_cast<const uint4*>(src + (size_t)(r0 + r) * ld + k0 + kc * 8);
            st_chunk(tile, kmajor_chunk(r, kc * 8), v);
        }
    }
};

// MN-major: element (r, k) of the operand is src[k * ld + r].
struct DenseMN {
    static constexpr bool MN = true;
    UGEMM_NO_ROWS
    const __nv_bfloat16* src;
    int rows, ld;
    template <int R>
    __device__ __forceinline__ void gather(unsigned char* tile, const Rows<R>&, int r0, int k0, int kn, int tid) const
    {
        // R rows x BK: chunks (rc, k) of 8 rows
        for (int i = tid; i < (R / 8) * BK; i += 128) {
            const int k = i / (R / 8), rc = i % (R / 8);
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (r0 + rc * 8 < rows && k < kn)
                v = *reinterpret_cast<const uint4*>(src + (size_t)(k0 + k) * ld + r0 + rc * 8);
            st_chunk(tile, mnmajor_chunk<R>(rc * 8, k), v);
        }
    }
};

// Row-major FP32 output D[r * ld + c].
struct StoreF32 {
    float* dst;
    int ld;
    __device__ __forceinline__ void store(int r, int c, const float (&v)[8], int) const
    {
        float4* p = reinterpret_cast<float4*>(dst + (size_t)r * ld + c);
        p[0] = make_float4(v[0], v[1], v[2], v[3]);
        p[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
};

// Launches the kernel for a 128 x BN tile grid with `splits` K slices.
// `extra_smem` adds unused shared memory after the tiles (layout checks).
template <int BN, class AG, class BG, class EP>
cudaError_t launch_gemm(const GemmArgs<AG, BG, EP>& g, int splits, cudaStream_t stream, size_t extra_smem = 0)
{
    const size_t smem = gemm_smem_bytes<BN>() + extra_smem;
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel<BN, AG, BG, EP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)splits);
    gemm_kernel<BN, AG, BG, EP><<<grid, 128, smem, stream>>>(g);
    return cudaGetLastError();
}

}  // namespace ugemm
