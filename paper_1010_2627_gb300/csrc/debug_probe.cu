// debug_probe.cu -- a test hook for the bounded tensor-core waits (no paper
// counterpart).  Every tcgen05 kernel of the library waits for its MMAs
// through tc::mbar_wait, a poll with an iteration bound after which the
// kernel records KNIT_ERR_TIMEOUT, waits (again bounded) for the commit it
// still has in flight, releases its tensor memory and returns.  This probe
// runs that path on purpose: it issues one MMA and commits it to barrier A,
// then waits on barrier B, which nothing completes, with a host-set bound;
// the wait runs out, the cleanup waits for A and frees the tensor memory,
// and the status word tells the host.  Nothing hangs or faults: both waits
// are bounded and every access is in bounds.

#include <cuda_runtime.h>

#include "../../include/knit.h"
#include "tc_common.cuh"

using namespace tc;

namespace {

struct ProbeSmem {
    alignas(1024) unsigned char a[128 * 32];
    alignas(1024) unsigned char b[64 * 32];
    unsigned long long bar_a, bar_b;
    uint32_t tmem;
};

__device__ int g_probe_status[2];   // [0]: status of the wait; [1]: 1 if the cleanup wait completed

__global__ void __launch_bounds__(128, 1) wait_probe_kernel(long polls)
{
    __shared__ ProbeSmem sm;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (int)sizeof(sm.a) / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(sm.a)[i] = 0u;
    for (int i = tid; i < (int)sizeof(sm.b) / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(sm.b)[i] = 0u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&sm.tmem)), "r"(64u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.bar_a)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.bar_b)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    async_proxy_fence();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem;
    if (tid == 0) {
        mma_bf16(tmem, smem_desc(smem_u32(sm.a)), smem_desc(smem_u32(sm.b)), idesc_bf16_m128(64), 0u);
        mma_commit(&sm.bar_a);
        // barrier B: nothing arrives, so this wait runs out after `polls` polls
        const int ok = mbar_wait(&sm.bar_b, 0, polls);
        g_probe_status[0] = ok ? KNIT_OK : KNIT_ERR_TIMEOUT;
        // the sweeps' cleanup: a bounded wait for the commit still in flight
        g_probe_status[1] = mbar_wait(&sm.bar_a, 0);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64u));
}

}  // namespace

extern "C" knit_status knit_debug_wait_probe(int64_t polls, int32_t *wait_status,
                                             int32_t *cleanup_done)
{
    if (polls < 1 || polls > (1LL << 24) || !wait_status || !cleanup_done) return KNIT_ERR_INVALID;
    int h[2] = {-1, -1};
    if (cudaMemcpyToSymbol(g_probe_status, h, sizeof(h)) != cudaSuccess) return KNIT_ERR_CUDA;
    wait_probe_kernel<<<1, 128>>>((long)polls);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return KNIT_ERR_CUDA;
    if (cudaMemcpyFromSymbol(h, g_probe_status, sizeof(h)) != cudaSuccess) return KNIT_ERR_CUDA;
    *wait_status = h[0];
    *cleanup_done = h[1];
    return KNIT_OK;
}
