// tc_common.cuh -- tcgen05 building blocks shared by the tensor-core kernels:
// shared-memory matrix descriptors for the no-swizzle K-major layout, bf16
// MMA issue and commit, bounded mbarrier waits, tensor-memory loads/stores.
//
// Operand tiles use the no-swizzle K-major layout: 8-row x 16-byte core
// matrices, K-adjacent core matrices 128 B apart (descriptor leading byte
// offset), 8-row groups 256 B apart (stride byte offset).  A tile of R rows
// and 16 bf16 along K therefore takes R x 32 bytes.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

#include "knit_common.cuh"

namespace tc {

constexpr long WAIT_LIMIT = 1L << 24;   // bounded mbarrier polling
constexpr int A_TILE = 128 * 16 * 2;    // bytes of one 128 x 16 bf16 tile
constexpr int B_TILE = 64 * 16 * 2;     // bytes of one 64 x 16 bf16 tile

// instruction descriptor: D f32, A and B bf16, both K-major, M = 128, N = n
KNIT_DEV uint32_t idesc_bf16_m128(uint32_t n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

KNIT_DEV uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row r, k c) in a K-major tile with 16 values along K
KNIT_DEV int tile_off(int r, int c) { return (r >> 3) * 256 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2; }

KNIT_DEV uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;     // K-adjacent core matrices
    d |= (uint64_t)(256 >> 4) << 32;     // 8-row groups
    d |= (uint64_t)1 << 46;              // descriptor version
    return d;
}

// two K-adjacent values (c even) in one 32-bit store
KNIT_DEV void put_bf16x2(unsigned char *tile, int r, int c, float v0, float v1)
{
    *reinterpret_cast<__nv_bfloat162 *>(tile + tile_off(r, c)) = __floats2bfloat162_rn(v0, v1);
}

KNIT_DEV void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem_d), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

KNIT_DEV void mma_commit(unsigned long long *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(mbar)) : "memory");
}

// bounded wait for the mbarrier phase `parity` (at most `limit` polls);
// returns 0 on timeout
KNIT_DEV int mbar_wait(unsigned long long *mbar, uint32_t parity, long limit = WAIT_LIMIT)
{
    uint32_t done = 0;
    for (long it = 0; it < limit; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
        if (done) return 1;
    }
    return 0;
}

KNIT_DEV void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

KNIT_DEV void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                   "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr));
}

// zero 8 consecutive accumulator columns of the warp's 32 TMEM lanes
KNIT_DEV void tmem_zero8(uint32_t taddr)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};"
                 ::"r"(taddr), "r"(0u) : "memory");
}

KNIT_DEV void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
KNIT_DEV void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
KNIT_DEV void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
KNIT_DEV void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace tc
