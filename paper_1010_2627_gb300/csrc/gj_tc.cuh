// gj_tc.cuh -- complex64 Gauss-Jordan inverse of a 64 x 64 shared-memory
// matrix (order M <= 64, identity in the padding) whose rank-8 panel updates
// run on the tensor cores.
//
// Same elimination as gj_lookahead in mixed_common.cuh (implicit partial
// pivoting on |Re| + |Im|, in-place inverse with u = column - e_p, panels of
// 8 columns, result permuted as store_inverse expects), scheduled for a
// block whose CUDA cores would otherwise be shared by the pivot chain and
// the updates.  Per panel of 8 columns:
//
//  * warp 0 alone takes the 8 pivot steps on the panel columns (registers),
//    and inside each step forms that step's row v_k of V for all 64 columns,
//    v_k = (X[p_k, :] + e_k - sum_{c<k} u_c[p_k] v_c) / pivot_k, from the
//    matrix at the start of the panel -- the forward substitution of
//    gj_lookahead, spread over the latency of the pivot chain;
//  * all threads cut U (64 x 8) and V (8 x 64) into three bf16 terms each,
//    x = h + m + l exactly for every fp32 x (bit masks, no conversions),
//    into the operand tiles of
//    D = V^T U^T in real form: A (128 x 16) row 2n + r holds row n of V^T as
//    [Re V^T, -Im V^T] (r = 0) or [Im V^T, Re V^T] (r = 1), B^T (64 x 16)
//    row i holds [Re U, Im U] of row i, so D row 2n + r, column i is
//    Re / Im of (U V)[i][n];
//  * one thread issues all nine products of terms (p, q) as three
//    tcgen05.mma (M = 128, K = 16, f32 accumulate in tensor memory): term p
//    of A against the three terms of B side by side (N = 192) at accumulator
//    base 64 p, so that accumulator d = p + q (d = 0 .. 4, 320 columns)
//    collects the products of one order of magnitude and small terms are
//    not rounded away against large ones;
//  * every warp reads its quarter of the tensor-memory lanes (X columns n,
//    real and imaginary parts in adjacent lanes) for 16 rows i, sums the five
//    accumulators smallest first and applies X -= U V; adjacent lanes touch
//    adjacent words of X, so the update is free of bank conflicts.
//
// Waits on the tensor cores are bounded (ST_TIMEOUT); the caller owns the
// tensor-memory columns (320, at tmem_d) and the mbarrier and its phase.
#pragma once

#include "mixed_common.cuh"
#include "tc_common.cuh"

namespace mixed {

// shared-memory work area of gj_tc
struct GjTcWork {
    float2 U[64 * gj_ust(8)];                          // u vectors of the panel, row i
    float2 V[8 * 64];                                  // v vectors of the panel
    alignas(128) unsigned char adg[3 * tc::A_TILE];    // terms of V^T in real form
    alignas(128) unsigned char bdg[3 * tc::B_TILE];    // terms of U
};

// 1 / a, no scaling: the pivots of gj_tc come from rows scaled to O(1); an
// overflowing or vanishing |a|^2 yields a non-finite or useless inverse that
// the refinement rejects
KNIT_DEV float2 crcp_direct(float2 a)
{
    const float d = __fdividef(1.0f, fmaf(a.x, a.x, a.y * a.y));
    return make_float2(a.x * d, -a.y * d);
}

// the exact split x = h + m + l into bf16 values by truncation: h keeps the
// upper 16 bits of x, m those of x - h, and l = x - h - m has at most 8
// significant bits, so every term's lower 16 bits are zero and its upper
// half is the bf16 value (bit patterns returned)
KNIT_DEV void bf16_split3(float x, uint32_t &h, uint32_t &m, uint32_t &l)
{
    h = __float_as_uint(x) & 0xffff0000u;
    const float r = x - __uint_as_float(h);
    m = __float_as_uint(r) & 0xffff0000u;
    l = __float_as_uint(r - __uint_as_float(m));
}

// two terms (upper halves) into one word, a at the lower address
KNIT_DEV uint32_t pack_hi16(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x7632); }

template <int NTH>
__device__ __forceinline__ int gj_tc(float2 *X, int M, GjTcWork &w, GJShared<64> &g,
                                     uint32_t tmem_d, unsigned long long *mbar, uint32_t &phase)
{
    constexpr int MP = 64, NB = 8, R2 = 2, IB = 6, UST = gj_ust(NB);
    static_assert(NTH == 512, "read-back: 16 warps, one per lane quarter and 16 rows");
    constexpr unsigned IMASK = (1u << IB) - 1u, FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    bool open[R2];   // warp 0: row lane + 32t may still become a pivot row
#pragma unroll
    for (int t = 0; t < R2; ++t) open[t] = lane + 32 * t < M;
    const int NP = (M + NB - 1) / NB;
    for (int P = 0; P < NP; ++P) {
        const int K = P * NB, nk = min(NB, M - K);
        if (warp == 0) {
            float2 pc[R2][NB];   // panel columns, rows lane + 32t
#pragma unroll
            for (int t = 0; t < R2; ++t)
#pragma unroll
                for (int c = 0; c < NB; ++c) pc[t][c] = X[(lane + 32 * t) * MP + K + c];
            float2 v[NB][R2];    // v_k for columns lane + 32t
            bool bad = false;
            auto steps = [&](auto fullc) {
                constexpr bool FULLP = decltype(fullc)::value;
                // the search of step kk > 0 runs on column kk times the
                // previous pivot (zs), formed before that pivot's reciprocal
                // is known; |Re| + |Im| of a rotated value stays within a
                // factor sqrt(2), so the choice is still a partial pivot
                float2 zs[R2];
#pragma unroll
                for (int kk = 0; kk < NB; ++kk) {
                    if (!FULLP && kk >= nk) break;
                    unsigned key = 0u;
#pragma unroll
                    for (int t = 0; t < R2; ++t) {
                        const float2 sv = kk > 0 ? zs[t] : pc[t][kk];
                        const unsigned kt = (__float_as_uint(cabs1f(sv)) & ~IMASK) |
                                            (IMASK - (unsigned)(lane + 32 * t));
                        key = max(key, open[t] ? kt : 0u);
                    }
                    key = __reduce_max_sync(FULL, key);
                    bad |= (key & ~IMASK) == 0u;
                    const int p = (int)(IMASK - (key & IMASK)), pl = p & 31, pt = p >> 5;
                    // the pivot row's panel entries, from lane p % 32
                    float2 prow[NB];
                    auto fetch = [&](int c) {
                        float2 own = pc[0][c];
#pragma unroll
                        for (int t = 1; t < R2; ++t) own = t == pt ? pc[t][c] : own;
                        prow[c] = make_float2(__shfl_sync(FULL, own.x, pl), __shfl_sync(FULL, own.y, pl));
                    };
                    fetch(kk);
                    if (kk + 1 < NB) fetch(kk + 1);
                    float2 u[R2];
#pragma unroll
                    for (int t = 0; t < R2; ++t) {
                        u[t] = pc[t][kk];
                        u[t].x -= lane + 32 * t == p ? 1.f : 0.f;
                    }
                    if (kk + 1 < NB)
#pragma unroll
                        for (int t = 0; t < R2; ++t)
                            zs[t] = cfmsf(u[t], prow[kk + 1], cmulf(prow[kk], pc[t][kk + 1]));
                    const float2 rinv = crcp_direct(prow[kk]);
                    if (kk + 1 < NB)
#pragma unroll
                        for (int t = 0; t < R2; ++t) pc[t][kk + 1] = cmulf(zs[t], rinv);
#pragma unroll
                    for (int c = kk + 2; c < NB; ++c) fetch(c);
#pragma unroll
                    for (int c = kk + 2; c < NB; ++c) {
                        const float2 vk = cmulf(prow[c], rinv);
#pragma unroll
                        for (int t = 0; t < R2; ++t) pc[t][c] = cfmsf(u[t], vk, pc[t][c]);
                    }
#pragma unroll
                    for (int t = 0; t < R2; ++t) {
                        const int i = lane + 32 * t;
                        w.U[i * UST + kk] = u[t];
                        open[t] = open[t] && i != p;
                    }
                    // v_kk from row p of the matrix at the start of the panel
                    __syncwarp();
                    float2 xr[R2];
#pragma unroll
                    for (int t = 0; t < R2; ++t) {
                        xr[t] = X[p * MP + lane + 32 * t];
                        if (lane + 32 * t == K + kk) xr[t].x += 1.f;
                    }
#pragma unroll
                    for (int c = 0; c < kk; ++c) {
                        const float2 uc = w.U[p * UST + c];
#pragma unroll
                        for (int t = 0; t < R2; ++t) xr[t] = cfmsf(uc, v[c][t], xr[t]);
                    }
#pragma unroll
                    for (int t = 0; t < R2; ++t) v[kk][t] = cmulf(xr[t], rinv);
                    if (lane == 0) g.perm[K + kk] = p;
                }
            };
            if (nk == NB) steps(BoolC<true>{});
            else steps(BoolC<false>{});
            // steps a partial panel does not take contribute nothing
#pragma unroll
            for (int kk = 0; kk < NB; ++kk)
                if (kk >= nk)
#pragma unroll
                    for (int t = 0; t < R2; ++t) {
                        v[kk][t] = make_float2(0.f, 0.f);
                        w.U[(lane + 32 * t) * UST + kk] = make_float2(0.f, 0.f);
                    }
#pragma unroll
            for (int kk = 0; kk < NB; ++kk)
#pragma unroll
                for (int t = 0; t < R2; ++t) w.V[kk * MP + lane + 32 * t] = v[kk][t];
            if (lane == 0) g.flag = bad ? 1 : 0;
        }
        __syncthreads();
        if (g.flag) return ST_SINGULAR;

        // bf16 terms of the operands: thread (n, r, s) splits eight values
        // once and writes their three terms, 16 bytes each: s = 0, 1 the
        // K halves of A row 2n + r, s = 2 the K half r of B^T row n
        if (tid < 6 * MP) {
            const int n = tid & (MP - 1), r = (tid >> 6) & 1, s = tid >> 7;
            float x[NB];
            if (s < 2) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const float2 vv = w.V[c * MP + n];
                    x[c] = s == 0 ? (r ? vv.y : vv.x) : (r ? vv.x : -vv.y);
                }
            } else {
#pragma unroll
                for (int c = 0; c < NB; c += 2) {
                    const float4 uu = *reinterpret_cast<const float4 *>(w.U + n * UST + c);
                    x[c] = r ? uu.y : uu.x;
                    x[c + 1] = r ? uu.w : uu.z;
                }
            }
            uint32_t t0[4], t1[4], t2[4];
#pragma unroll
            for (int c = 0; c < NB; c += 2) {
                uint32_t h0, m0, l0, h1, m1, l1;
                bf16_split3(x[c], h0, m0, l0);
                bf16_split3(x[c + 1], h1, m1, l1);
                t0[c / 2] = pack_hi16(h0, h1);
                t1[c / 2] = pack_hi16(m0, m1);
                t2[c / 2] = pack_hi16(l0, l1);
            }
            unsigned char *const base = s < 2 ? w.adg + tc::tile_off(2 * n + r, 8 * s)
                                              : w.bdg + tc::tile_off(n, 8 * r);
            const int stride = s < 2 ? tc::A_TILE : tc::B_TILE;
            *reinterpret_cast<uint4 *>(base) = make_uint4(t0[0], t0[1], t0[2], t0[3]);
            *reinterpret_cast<uint4 *>(base + stride) = make_uint4(t1[0], t1[1], t1[2], t1[3]);
            *reinterpret_cast<uint4 *>(base + 2 * stride) = make_uint4(t2[0], t2[1], t2[2], t2[3]);
        }
        {
            const uint32_t tz = tmem_d + ((uint32_t)(32 * (warp & 3)) << 16) + 192 + 32 * (warp >> 2);
#pragma unroll
            for (int c = 0; c < 32; c += 8) tc::tmem_zero8(tz + c);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        tc::async_proxy_fence();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            // term p of A against the three terms of B side by side (N = 192)
            // at accumulator base 64 p: product (p, q) lands in accumulator p + q
#pragma unroll
            for (int p = 0; p < 3; ++p)
                tc::mma_bf16(tmem_d + 64 * p, tc::smem_desc(tc::smem_u32(w.adg + p * tc::A_TILE)),
                             tc::smem_desc(tc::smem_u32(w.bdg)), tc::idesc_bf16_m128(192),
                             p ? 1u : 0u);
            tc::mma_commit(mbar);
        }
        const int ok = tid == 0 ? tc::mbar_wait(mbar, phase) : 1;
        phase ^= 1u;
        if (__syncthreads_or(!ok)) return ST_TIMEOUT;
        tc::fence_after();
        {
            // lane 32q + l of warp w: X column n = 16q + l/2, part l % 2, rows 16(w/4) ..
            const int q = warp & 3, i0 = 16 * (warp >> 2);
            const int n = 16 * q + (lane >> 1), part = lane & 1;
            const uint32_t ta = tmem_d + ((uint32_t)(32 * q) << 16) + i0;
            float sum[16];
            {
                uint32_t a4[16], a3[16], a2[16];
                tc::tmem_ld16(ta + 256, a4);
                tc::tmem_ld16(ta + 192, a3);
                tc::tmem_ld16(ta + 128, a2);
                tc::wait_ld();
#pragma unroll
                for (int r = 0; r < 16; ++r)
                    sum[r] = (__uint_as_float(a4[r]) + __uint_as_float(a3[r])) + __uint_as_float(a2[r]);
            }
            {
                uint32_t a1[16], a0[16];
                tc::tmem_ld16(ta + 64, a1);
                tc::tmem_ld16(ta, a0);
                tc::wait_ld();
#pragma unroll
                for (int r = 0; r < 16; ++r) sum[r] = (sum[r] + __uint_as_float(a1[r])) + __uint_as_float(a0[r]);
            }
            float *const Xf = reinterpret_cast<float *>(X);
#pragma unroll
            for (int r = 0; r < 16; ++r) Xf[2 * ((i0 + r) * MP + n) + part] -= sum[r];
        }
        tc::fence_before();
        __syncthreads();
    }
    return ST_OK;
}

}  // namespace mixed
