// Verification entry point of the tensor-core GEMM core (declared in
// include/neurosim_evsim.h as neurosim_debug_umma_gemm): plain dense GEMMs
// with every operand layout, compared against a host GEMM by the tests.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/neurosim_evsim.h"
#include "evsim_internal.h"
#include "umma_gemm.cuh"
#include "umma_tma.cuh"
#include "umma_mn.cuh"

namespace {

using namespace ugemm;

template <int BN, class AG, class BG>
int run(const AG& a, const BG& b, int M, int N, int K, float* C, unsigned int* err, cudaStream_t st)
{
    GemmArgs<AG, BG, StoreF32> g;
    g.a = a;
    g.b = b;
    g.ep = StoreF32{C, N};
    g.M = M;
    g.N = N;
    g.K = K;
    g.k_per_split = ((K + BK - 1) / BK) * BK;
    g.err = err;
    g.limit_ns = 2000000000ull;
    // 64 KB of slack after the tiles: a descriptor that strides further than
    // the layout intends still reads shared memory the CTA owns
    if (launch_gemm<BN>(g, 1, st, 64 * 1024) != cudaSuccess) return NEUROSIM_E_CUDA;
    return NEUROSIM_OK;
}

template <int BN>
int dispatch(int mode, int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C,
             unsigned int* err, cudaStream_t st)
{
    const bool amn = mode & 1, bmn = mode & 2;
    const DenseK ak{A, M, K}, bk{B, N, K};
    const DenseMN am{A, M, M}, bm{B, N, N};
    if (!amn && !bmn) return run<BN>(ak, bk, M, N, K, C, err, st);
    if (amn && !bmn) return run<BN>(am, bk, M, N, K, C, err, st);
    if (!amn && bmn) return run<BN>(ak, bm, M, N, K, C, err, st);
    return run<BN>(am, bm, M, N, K, C, err, st);
}

// Row-major FP32 output for the TMA kernel.
struct StoreRow {
    float* dst;
    int ld;
    __device__ __forceinline__ void store(int r, int c, const float (&v)[8], int) const
    {
        float4* p = reinterpret_cast<float4*>(dst + (size_t)r * ld + c);
        p[0] = make_float4(v[0], v[1], v[2], v[3]);
        p[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
};

template <int BN, int SW>
int run_tma(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, unsigned int* err,
            cudaStream_t st)
{
    utma::TmaArgs<utma::DenseA, StoreRow> g;
    if (!utma::encode_kmajor(&g.ta, A, M, K, utma::BM, SW) || !utma::encode_kmajor(&g.tb, B, N, K, BN, SW))
        return NEUROSIM_E_CUDA;
    g.a = utma::DenseA{M, K, 0, utma::bk_of(SW)};
    g.ep = StoreRow{C, N};
    g.N = N;
    g.err = err;
    g.limit_ns = 2000000000ull;
    if (utma::launch_tma_gemm<BN, SW>(g, (M + utma::BM - 1) / utma::BM, st) != cudaSuccess) return NEUROSIM_E_CUDA;
    return NEUROSIM_OK;
}

// MN-major TMA GEMM over "pixels": A stored [K][M] and B stored [K][N] are
// viewed as one image row of K pixels with M (N) channels; C is zeroed and
// the K-slice partial tiles are added into it.
template <int BN>
int run_mn(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, unsigned int* err,
           cudaStream_t st)
{
    umn::MnArgs<BN> g;
    g.a = umn::MnOp{umn::kPix, M, 0, 1, M, umn::pick_sw(M)};
    g.b = umn::MnOp{umn::kPix, N, 0, 1, N, umn::pick_sw(N)};
    if (!umn::encode_op(&g.ta, A, M, K, 1, 1, g.a) || !umn::encode_op(&g.tb, B, N, K, 1, 1, g.b))
        return NEUROSIM_E_CUDA;
    const int xb = (K + umn::KT - 1) / umn::KT;
    g.geom = umn::MnGeom{1, K, xb, xb};
    g.M = M;
    g.N = N;
    g.dw = C;
    g.err = err;
    g.limit_ns = 2000000000ull;
    if (cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(float), st) != cudaSuccess) return NEUROSIM_E_CUDA;
    // a few K slices, so that the partial tiles are really added
    if (umn::launch_mn_gemm<BN>(g, 3 * ((M + umn::BM - 1) / umn::BM), st) != cudaSuccess) return NEUROSIM_E_CUDA;
    return NEUROSIM_OK;
}

// One CTA of 32 threads: thread 0 sets up an mbarrier expecting one arrival
// and, if `arrive`, arrives on it; then the whole warp waits for the phase
// with the same bounded wait as the tensor-core kernels (umma::mbar_wait).
// Nothing else ever arrives, so without `arrive` every wait gives up after
// limit_ns and the kernel records kErrTimeout and returns.
__global__ void expiring_wait_kernel(int arrive, uint64_t limit_ns, unsigned int* err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        umma::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (threadIdx.x == 0 && arrive)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(&bar)) : "memory");
    __syncwarp();
    const bool ok = umma::mbar_wait(&bar, 0, limit_ns);
    if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicOr(err, nsim::kErrTimeout);
}

}  // namespace

extern "C" int neurosim_debug_expiring_wait(int32_t arrive, uint64_t limit_ns, void* cuda_stream)
{
    if (limit_ns < 1000ull || limit_ns > 100000000ull)
        return nsim::report_error(NEUROSIM_E_INVALID, "limit_ns must be in [1 us, 100 ms]");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned int* err = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&err), sizeof(unsigned int), st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(unsigned int), st) != cudaSuccess)
        return nsim::report_error(NEUROSIM_E_CUDA, "cannot allocate the error word");
    expiring_wait_kernel<<<1, 32, 0, st>>>(arrive != 0, limit_ns, err);
    int rc = cudaGetLastError() == cudaSuccess ? NEUROSIM_OK : NEUROSIM_E_CUDA;
    unsigned int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        rc = rc ? rc : NEUROSIM_E_CUDA;
    cudaFreeAsync(err, st);
    if (rc) return nsim::report_error(rc, "wait kernel launch failed");
    if (h & nsim::kErrTimeout) return nsim::report_error(NEUROSIM_E_TIMEOUT, "the bounded mbarrier wait gave up");
    return NEUROSIM_OK;
}

extern "C" int neurosim_debug_umma_gemm(int32_t mode, int32_t M, int32_t N, int32_t K, const void* A,
                                        const void* B, float* C, void* cuda_stream)
{
    if (!A || !B || !C) return nsim::report_error(NEUROSIM_E_INVALID, "NULL operand");
    if (mode < 0 || mode > 6) return nsim::report_error(NEUROSIM_E_INVALID, "mode must be in [0, 6]");
    if (mode >= 4 && (reinterpret_cast<uintptr_t>(A) & 15u || reinterpret_cast<uintptr_t>(B) & 15u))
        return nsim::report_error(NEUROSIM_E_INVALID, "TMA operands must be 16-byte aligned");
    const bool amn = (mode < 4 && (mode & 1)) || mode == 6, bmn = (mode < 4 && (mode & 2)) || mode == 6;
    if (M < 1 || N < 16 || N > 256 || N % 16 || K < 8 || K % 8 || (amn && M % 8) || (bmn && N % 8))
        return nsim::report_error(NEUROSIM_E_INVALID,
                                  "need M >= 1, 16 <= N <= 256 with N % 16 == 0, K % 8 == 0, MN-major rows % 8 == 0");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned int* err = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&err), sizeof(unsigned int), st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(unsigned int), st) != cudaSuccess)
        return nsim::report_error(NEUROSIM_E_CUDA, "cannot allocate the error word");
    const auto* a = static_cast<const __nv_bfloat16*>(A);
    const auto* b = static_cast<const __nv_bfloat16*>(B);
    int rc = mode == 6 ? (N <= 16 ? run_mn<16>(M, N, K, a, b, C, err, st)
                          : N <= 32 ? run_mn<32>(M, N, K, a, b, C, err, st)
                          : N <= 64 ? run_mn<64>(M, N, K, a, b, C, err, st)
                          : N <= 128 ? run_mn<128>(M, N, K, a, b, C, err, st) : run_mn<256>(M, N, K, a, b, C, err, st))
             : mode == 4 ? (N <= 64 ? run_tma<64, 128>(M, N, K, a, b, C, err, st) : run_tma<256, 128>(M, N, K, a, b, C, err, st))
             : mode == 5 ? (N <= 64 ? run_tma<64, 64>(M, N, K, a, b, C, err, st) : run_tma<256, 64>(M, N, K, a, b, C, err, st))
             : N <= 64 ? dispatch<64>(mode, M, N, K, a, b, C, err, st)
                       : dispatch<256>(mode, M, N, K, a, b, C, err, st);
    unsigned int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        rc = rc ? rc : NEUROSIM_E_CUDA;
    cudaFreeAsync(err, st);
    if (rc) return nsim::report_error(rc, "GEMM launch failed");
    if (h) return nsim::report_error(NEUROSIM_E_TIMEOUT, "a bounded MMA wait timed out");
    return NEUROSIM_OK;
}
