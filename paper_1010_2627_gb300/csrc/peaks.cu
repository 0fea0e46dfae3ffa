// peaks.cu -- the library's own peak-rate microbenchmarks, the denominators
// of the roofline fractions the benchmark reports (no paper counterpart):
//
//   KNIT_PEAK_MMA_BF16  tcgen05.mma.cta_group::1.kind::f16, bf16 operands,
//                       f32 accumulation, M = 128, N = 256, K = 16 per
//                       instruction (2 M N K flop), operands in shared memory
//   KNIT_PEAK_MMA_TF32  the same with kind::tf32 (K = 8 per instruction)
//   KNIT_PEAK_MMA_N64 / _N16   the bf16 loop with N = 64 / N = 16
//   KNIT_PEAK_MMA_RESIDUAL     the wide sweep's residual MMA pattern per K-chunk
//                              (six MMAs into staggered accumulators; _TF32 the
//                              same with kind::tf32), which sustains a higher
//                              rate than the single-tile loop
//   KNIT_PEAK_DFMA      FP64 fused multiply-add on the CUDA cores
//   KNIT_PEAK_FFMA      FP32 fused multiply-add on the CUDA cores
//
// Each launch runs a fixed amount of work on every SM (one CTA per SM for
// the tensor-core loops, eight 256-thread CTAs per SM for the FMA loops);
// the caller times it.  The MMA loops issue back-to-back instructions from
// one thread into two accumulators in turn, and wait once at the end
// (bounded wait); their operands are small non-zero constants.

#include <cuda_runtime.h>

#include "../../include/knit.h"
#include "tc_common.cuh"

using namespace tc;

namespace {

constexpr int PEAK_THREADS_MMA = 128;
constexpr int PEAK_THREADS_FMA = 256;
constexpr int PEAK_FMA_CTAS_PER_SM = 8;

struct PeakSmem {
    alignas(1024) unsigned char a[3][128 * 32];   // 128 rows x 32 bytes of K (16 bf16 / 8 tf32)
    alignas(1024) unsigned char b[2][448 * 32];   // up to 448 rows x 32 bytes of K
    unsigned long long mbar;
    uint32_t tmem;
};

__device__ int g_peak_status;      // set when a bounded wait ran out
__device__ double g_peak_sink;     // keeps the FMA loops' results alive

// shape: 0 the dense peak (N = 256, one operand pair); 1 N = 64; 2 N = 16;
// 3 the residual's pattern per K-chunk of the wide tensor-core sweep: three A
// digit tiles, each against B digits side by side (N = 256 then 192 / 128 /
// 64) into staggered accumulators, two alternating B buffers
__global__ void __launch_bounds__(PEAK_THREADS_MMA, 1)
peak_mma_kernel(long long iters, int tf32, int shape, int *status)
{
    __shared__ PeakSmem sm;
    const int tid = threadIdx.x, warp = tid >> 5;
    // small non-zero operands (2^-12 as two bf16, or as one tf32 value), so
    // that the tensor cores see data rather than zeros
    const uint32_t word = tf32 ? 0x39800000u : 0x39803980u;
    for (int i = tid; i < (int)sizeof(sm.a) / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(sm.a)[i] = word;
    for (int i = tid; i < (int)sizeof(sm.b) / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(sm.b)[i] = word;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&sm.tmem)), "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    async_proxy_fence();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem;
    if (tid == 0) {
        // D f32; A and B bf16 (format 1) or tf32 (format 2), both K-major
        const uint32_t fmt = tf32 ? 2u : 1u;
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((256u >> 3) << 17) |
                               ((128u >> 4) << 24);
        const uint64_t ad = smem_desc(smem_u32(sm.a[0])), bd = smem_desc(smem_u32(sm.b[0]));
        if (shape == 0) {
            // two accumulators in turn (columns 0 and 256), so that consecutive
            // instructions do not wait on each other's accumulation
            for (long long it = 0; it < iters; ++it) {
                const uint32_t d = tmem + 256u * (uint32_t)(it & 1);
                if (tf32)
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                                 ::"r"(d), "l"(ad), "l"(bd), "r"(idesc), "r"(it > 1 ? 1u : 0u));
                else
                    mma_bf16(d, ad, bd, idesc, it > 1 ? 1u : 0u);
            }
        } else if (shape == 1 || shape == 2) {
            const uint32_t n = shape == 1 ? 64u : 16u;
            const uint32_t id = (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
            for (long long it = 0; it < iters; ++it) mma_bf16(tmem, ad, bd, id, it > 0 ? 1u : 0u);
        } else {
            const uint32_t fmt = tf32 ? 2u : 1u;
            for (long long it = 0; it < iters; ++it) {
                const uint64_t b0 = smem_desc(smem_u32(sm.b[it & 1]));
                const uint64_t b4 = smem_desc(smem_u32(sm.b[it & 1] + 4 * 64 * 32));
                for (int q = 0; q < 3; ++q) {
                    const uint64_t aq = smem_desc(smem_u32(sm.a[q]));
                    const uint32_t acc = it > 0 || q > 0 ? 1u : 0u;
                    const uint32_t i0 = (1u << 4) | (fmt << 7) | (fmt << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
                    const uint32_t i1 = (1u << 4) | (fmt << 7) | (fmt << 10) |
                                        (((uint32_t)(64 * (3 - q)) >> 3) << 17) | ((128u >> 4) << 24);
                    if (tf32) {
                        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                                     ::"r"(tmem + 64 * q), "l"(aq), "l"(b0), "r"(i0), "r"(acc));
                        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                                     ::"r"(tmem + 64 * (q + 4)), "l"(aq), "l"(b4), "r"(i1), "r"(acc));
                    } else {
                        mma_bf16(tmem + 64 * q, aq, b0, i0, acc);
                        mma_bf16(tmem + 64 * (q + 4), aq, b4, i1, acc);
                    }
                }
            }
        }
        mma_commit(&sm.mbar);
        if (!mbar_wait(&sm.mbar, 0)) {
            atomicExch(status, 1);
            mbar_wait(&sm.mbar, 0);   // a second bounded wait before the release
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
}

// eight independent FMA chains per thread; the result is stored only when
// it equals a value it cannot take, so that the loop is not removed
template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS_FMA)
peak_fma_kernel(long long iters)
{
    T a[8];
    const T b = (T)0.999999, c = (T)1e-7;
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x + k);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == (T)-1.2345) g_peak_sink = (double)s;
}

}  // namespace

extern "C" knit_status knit_peak_probe(int32_t kind, int64_t iters, int32_t nsm, double *flop,
                                       int32_t *timed_out, void *stream)
{
    if (iters < 1 || nsm < 1 || !flop) return KNIT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int *status = nullptr;
    if (timed_out) {
        const int zero = 0;
        if (cudaMemcpyToSymbolAsync(g_peak_status, &zero, sizeof(int), 0,
                                    cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&status, g_peak_status) != cudaSuccess)
            return KNIT_ERR_CUDA;
    }
    switch (kind) {
    case KNIT_PEAK_MMA_BF16:
    case KNIT_PEAK_MMA_TF32: {
        if (!status && cudaGetSymbolAddress((void **)&status, g_peak_status) != cudaSuccess)
            return KNIT_ERR_CUDA;
        const int tf32 = kind == KNIT_PEAK_MMA_TF32;
        const double k = tf32 ? 8.0 : 16.0;
        *flop = 2.0 * 128.0 * 256.0 * k * (double)iters * nsm;
        peak_mma_kernel<<<nsm, PEAK_THREADS_MMA, 0, st>>>(iters, tf32, 0, status);
        break;
    }
    case KNIT_PEAK_MMA_N64:
    case KNIT_PEAK_MMA_N16:
    case KNIT_PEAK_MMA_RESIDUAL:
    case KNIT_PEAK_MMA_RESIDUAL_TF32: {
        if (!status && cudaGetSymbolAddress((void **)&status, g_peak_status) != cudaSuccess)
            return KNIT_ERR_CUDA;
        const int shape = kind == KNIT_PEAK_MMA_N64 ? 1 : kind == KNIT_PEAK_MMA_N16 ? 2 : 3;
        const int tf32 = kind == KNIT_PEAK_MMA_RESIDUAL_TF32;
        const double n = shape == 1 ? 64.0 : shape == 2 ? 16.0 : 1152.0;
        *flop = 2.0 * 128.0 * n * (tf32 ? 8.0 : 16.0) * (double)iters * nsm;
        peak_mma_kernel<<<nsm, PEAK_THREADS_MMA, 0, st>>>(iters, tf32, shape, status);
        break;
    }
    case KNIT_PEAK_DFMA:
        *flop = 2.0 * 8 * 16 * (double)iters * PEAK_THREADS_FMA * PEAK_FMA_CTAS_PER_SM * nsm;
        peak_fma_kernel<double><<<nsm * PEAK_FMA_CTAS_PER_SM, PEAK_THREADS_FMA, 0, st>>>(iters);
        break;
    case KNIT_PEAK_FFMA:
        *flop = 2.0 * 8 * 16 * (double)iters * PEAK_THREADS_FMA * PEAK_FMA_CTAS_PER_SM * nsm;
        peak_fma_kernel<float><<<nsm * PEAK_FMA_CTAS_PER_SM, PEAK_THREADS_FMA, 0, st>>>(iters);
        break;
    default:
        return KNIT_ERR_INVALID;
    }
    if (cudaGetLastError() != cudaSuccess) return KNIT_ERR_CUDA;
    if (timed_out) {
        if (cudaMemcpyFromSymbolAsync(timed_out, g_peak_status, sizeof(int), 0,
                                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return KNIT_ERR_CUDA;
    }
    return KNIT_OK;
}
