// sweep_mixed_tc.cu -- mixed-precision slice sweep with the refinement
// residual on the tcgen05 tensor cores (padded width MP = 64, i.e. M in 33..64).
//
// Same recursion as sweep_mixed.cu (KNIT user guide Sec. 5.3 D, Eq. 2 by
// block elimination; complex64 inversion + refinement, state g carried as
// hi + lo, T from G_LL by the unitarity identity).  Per slice n:
//
//  * Gv' = V g V^dagger (+ Sigma terms) + H0 - D_n in double-float, so that
//    A_n = -Gv' and the residual of an approximate inverse X' is
//    R = I - A_n X' = I + Gv' X';
//  * X = complex64 inverse of fl32(A_n) by blocked Gauss-Jordan with
//    implicit partial pivoting, the rank-8 panel updates on the tensor cores
//    (gj_tc.cuh: bf16 terms, five exact-order accumulators in the same
//    tensor memory, 320 of the 512 columns);
//  * X is rounded at a per-column power-of-two scale tau_n to 24 bits,
//    X' = tau_n 2^-8 (d0 + d1 2^-8 + d2 2^-16), |d| <= 256 integers (three
//    bf16 "digits", exact, and X' itself exact in fp32); the refinement uses
//    X' consistently, so X' only needs to be a good approximate inverse;
//  * Gv' is cut at a per-row scale sigma_i into seven digits (56 bits),
//    Gv' ~= sigma_i 2^-8 sum_p e_p 2^-8p;
//  * the complex product is the real product of [[Gr, -Gi], [Gi, Gr]]
//    (128 x 128) with [Xr; Xi] (128 x 64): the 18 digit products
//    (p + q <= 6, q <= 2) of a K-chunk of 16 run as 7 tcgen05.mma kind::f16
//    (bf16 in, f32 accumulate in tensor memory), one per A digit p against
//    the chunk's B digits q = 0 .. min(2, 6 - p) stored side by side
//    (N = 64 per digit), so product (p, q) lands in accumulator p + q.
//    Digits are stored pre-scaled by 2^-8p / 2^-8q, so every product of one
//    anti-diagonal d = p + q is an integer multiple of 2^-8d below 2^24 in
//    magnitude: each of the seven accumulators d = 0 .. 6 sums exactly;
//  * the seven accumulators are summed -- 3 .. 6 (below 2^-24 of the
//    leading one) in fp32, then with 0 .. 2 in double-float -- scaled by
//    sigma_i tau_n 2^-16, the identity added, and R rounded once to fp32;
//  * g = X' (I + R + R^2 + ...) with as many terms as max|R_ij| asks for
//    (mixed_common.cuh: neumann_terms), the product X' S on the tensor cores
//    as six bf16-term MMAs per K-chunk (refine_tc), or accumulated
//    error-free on the CUDA cores where max|R_ij| is large (refine_exact).
// The digit products are the Ozaki splitting (Ozaki, Ogita, Oishi & Rump
// 2012) with bf16 slices, specialised to the residual of an approximate
// inverse.
//
// Shared-memory operand tiles use the no-swizzle K-major layout of
// tc_common.cuh: 8-row x 16-byte core matrices, K-adjacent core matrices
// 128 B apart (descriptor leading byte offset), 8-row groups 256 B apart
// (stride byte offset).

#include <cuda_bf16.h>

#include "gj_tc.cuh"
#include "mixed_common.cuh"
#include "tc_common.cuh"

using namespace mixed;
using namespace tc;

namespace {

constexpr int MPT = 64;               // padded width handled here
constexpr int NTT = 512, TYT = 16, TXT = 32;   // 16 x 32 thread grid
constexpr int RA = MPT / TYT, RB = MPT / TXT;
constexpr int NDA = 7;                // digits of Gv
constexpr int NDB = 3;                // digits of X
constexpr int NACC = 7;               // accumulators d = p + q = 0 .. 6, each exact
constexpr int RS = MPT + 1;           // padded row stride of R
constexpr int MAX_NNZ = 256;          // sparse H0 rows cached in shared memory up to this
constexpr uint32_t TMEM_COLS = 512;   // 7 accumulators x 64 columns, rounded up


struct TcSmem {
    float2 X[MPT * MPT];                         // inverse, then X' (rounded)
    union {
        unsigned char adig[2 * NDA * A_TILE];    // A digits of two K-chunks
        float2 R[MPT * RS];                      // residual (after the products)
        GjTcWork gw;                             // Gauss-Jordan panel and its operand terms
    } u;
    union {
        struct {
            unsigned char bdig[NDB * 8 * B_TILE];  // B digits of all 8 K-chunks
            float2 Gh[MPT * MPT];                  // g (hi) / Gv (hi)
            float2 Gl[MPT * MPT];                  // g (lo) / Gv (lo)
        } s;
    } w;
    static_assert(MPT * RS * sizeof(float2) <= sizeof(w.s.bdig), "series buffer");
    static_assert(sizeof(X) + sizeof(u) >= MPT * MPT * sizeof(double2), "FP64 fallback matrix");
    GJShared<MPT> gj;
    double eps[MPT];
    float2 vh[2][MPT];
    float2 vl[2][MPT];
    int vuni[2];
    float vch[2], vcl[2];
    int rexp[MPT];
    int cexp[MPT];
    float cmax[NTT / MPT][MPT];
    int h0rp[MPT + 1];
    int h0c[MAX_NNZ];
    float2 h0h[MAX_NNZ];
    float2 h0l[MAX_NNZ];
    double red[NTT / 32];
    unsigned redu[NTT / 32];
    unsigned long long mbar;
    uint32_t tmem;
    int inst;
    int cur_sys;
    int h0_cached;
};

// 2^e as a float for |e| <= 126 (exact power of two)
KNIT_DEV float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// exponent e with |v| < 2^e for the largest |v| (0 for an all-zero set)
KNIT_DEV int scale_exp(float mx)
{
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    return e;
}

// x = h + m + l exactly, three bf16 values (bit patterns in the upper
// halves), each cut at round to nearest: h takes the leading 8 significant
// bits of the 24, r = x - h and l = r - m are exact (Sterbenz), and
// |m| <= 2^-8 |x|, |l| <= 2^-16 |x| up to the half-ulp of each cut
KNIT_DEV void bf16_split3_rn(float x, uint32_t &h, uint32_t &m, uint32_t &l)
{
    h = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x)) << 16;
    const float r = x - __uint_as_float(h);
    m = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(r)) << 16;
    l = __float_as_uint(r - __uint_as_float(m));
}

// two terms (upper halves) into one word, a at the lower address
KNIT_DEV uint32_t pack_hi(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x7632); }

// g = X' + X' S on the tensor cores, X' in sm.X, S (row stride RS, zero
// outside M x M) in sm.u.R, result as double-float in (Gh, Gl).  X' S is
// formed as its transpose S^T X'^T in a split real form: A row 2n + r holds
// column n of S, real (r = 0) or imaginary (r = 1) parts, along K = k (64:
// four K-chunks); B row j holds row j of X' (real parts) and B row 64 + j
// its imaginary parts (N = 128).  Accumulator lane 2n + r, column j then
// holds (X'_re S_r)[j][n] and column 64 + j (X'_im S_r)[j][n]; with
// Re (X'S) = X'_re S_re - X'_im S_im and Im (X'S) = X'_re S_im + X'_im S_re
// one exchange between the lanes 2n and 2n + 1 completes the entry.  Every
// value is cut into three bf16 terms (bf16_split3_rn, exact); the six term
// products with p + q <= 2 run (those left out are ~2^-24 of the product
// and below), the leading one into accumulator 0 (columns 0 .. 127), the
// other five into accumulator 1 (128 .. 255), summed smallest first.
// A terms: 12 tiles of 128 x 16 in the B-digit buffer; B terms: 12 tiles
// over Gh / Gl, which hold nothing until the result is written there.
// Returns 0 when the wait on the tensor cores runs out (phase flipped as
// for a completed wait).
KNIT_DEV int refine_tc(TcSmem &sm, uint32_t tmem, uint32_t &phase)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char *const at = sm.w.s.bdig;
    unsigned char *const bt = reinterpret_cast<unsigned char *>(sm.w.s.Gh);
    static_assert(sizeof(sm.w.s.bdig) >= 12 * A_TILE, "A terms of S");
    static_assert(sizeof(sm.w.s.Gh) + sizeof(sm.w.s.Gl) >= 12 * A_TILE, "B terms of X'");
    const float2 *const S = sm.u.R;
    // item e: chunk c = e / 512, row n (A) or j (B) = (e / 8) % 64, K pair
    // 2 (e % 8) of the chunk; eight lanes share a row (conflict-free loads)
    for (int e = tid; e < 4 * MPT * 8; e += NTT) {
        const int kp = e & 7, rI = (e >> 3) & 63, c = e >> 9, k = 16 * c + 2 * kp;
        uint32_t t[2][2][3];   // [re / im][k / k+1][term]
        {
            const float2 s0 = S[k * RS + rI], s1 = S[(k + 1) * RS + rI];
            bf16_split3_rn(s0.x, t[0][0][0], t[0][0][1], t[0][0][2]);
            bf16_split3_rn(s1.x, t[0][1][0], t[0][1][1], t[0][1][2]);
            bf16_split3_rn(s0.y, t[1][0][0], t[1][0][1], t[1][0][2]);
            bf16_split3_rn(s1.y, t[1][1][0], t[1][1][1], t[1][1][2]);
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    *reinterpret_cast<uint32_t *>(at + (c * 3 + q) * A_TILE + tile_off(2 * rI + r, 2 * kp)) =
                        pack_hi(t[r][0][q], t[r][1][q]);
        }
        {
            const float4 x = *reinterpret_cast<const float4 *>(sm.X + rI * MPT + k);
            bf16_split3_rn(x.x, t[0][0][0], t[0][0][1], t[0][0][2]);
            bf16_split3_rn(x.z, t[0][1][0], t[0][1][1], t[0][1][2]);
            bf16_split3_rn(x.y, t[1][0][0], t[1][0][1], t[1][0][2]);
            bf16_split3_rn(x.w, t[1][1][0], t[1][1][1], t[1][1][2]);
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    *reinterpret_cast<uint32_t *>(bt + (c * 3 + q) * A_TILE + tile_off(64 * r + rI, 2 * kp)) =
                        pack_hi(t[r][0][q], t[r][1][q]);
        }
    }
    async_proxy_fence();
    fence_before();
    __syncthreads();
    if (tid == 0) {
        fence_after();
        const uint32_t idesc = idesc_bf16_m128(128);
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3 - p; ++q) {
                    const bool lead = p + q == 0;
                    const uint32_t acc = lead ? (c > 0) : !(c == 0 && p == 0 && q == 1);
                    mma_bf16(tmem + (lead ? 0u : 128u), smem_desc(smem_u32(at + (c * 3 + p) * A_TILE)),
                             smem_desc(smem_u32(bt + (c * 3 + q) * A_TILE)), idesc, acc);
                }
        mma_commit(&sm.mbar);
    }
    const int ok = tid == 0 ? mbar_wait(&sm.mbar, phase) : 1;
    phase ^= 1u;
    if (__syncthreads_or(!ok)) return 0;
    fence_after();
    {
        // warp w: lanes 32 (w % 4) .. (columns n = 16 (w % 4) + lane / 2,
        // part r = lane % 2), rows j = 16 (w / 4) ..
        const int qd = warp & 3, j0 = 16 * (warp >> 2);
        const int n = 16 * qd + (lane >> 1), r = lane & 1;
        const uint32_t ta = tmem + ((uint32_t)(32 * qd) << 16) + j0;
        uint32_t a0[16], b0[16], a1[16], b1[16];
        tmem_ld16(ta, a0);
        tmem_ld16(ta + 64, b0);
        tmem_ld16(ta + 128, a1);
        tmem_ld16(ta + 192, b1);
        wait_ld();
        float *const Xf = reinterpret_cast<float *>(sm.X);
        float *const Ghf = reinterpret_cast<float *>(sm.w.s.Gh);
        float *const Glf = reinterpret_cast<float *>(sm.w.s.Gl);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            const float d1 = __uint_as_float(a1[jj]) + __uint_as_float(a0[jj]);
            const float d2 = __uint_as_float(b1[jj]) + __uint_as_float(b0[jj]);
            const float o = __shfl_xor_sync(0xffffffffu, d2, 1);
            const float v = r ? d1 + o : d1 - o;
            const int e = 2 * ((j0 + jj) * MPT + n) + r;
            float h, l;
            two_sum(Xf[e], v, h, l);
            Ghf[e] = h;
            Glf[e] = l;
        }
    }
    fence_before();
    return 1;
}

__global__ void fill_status(int *st, int n, int v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) st[i] = v;
}

}  // namespace

__global__ void __launch_bounds__(NTT, 1)
knit_sweep_mixed_tc_kernel(InstDev in)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smem_raw);
    float2 *const Gh = sm.w.s.Gh;
    float2 *const Gl = sm.w.s.Gl;
    const int tid = threadIdx.x, ty = tid / TXT, tx = tid % TXT;
    const int warp = tid >> 5, lane = tid & 31;
    // D f32, A and B bf16, both K-major, N = 64, M = 128
    const uint32_t idesc_n64 = (1u << 4) | (1u << 7) | (1u << 10) |
                           ((128u >> 4) << 24);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&sm.tmem)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        sm.cur_sys = -1;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem;
    uint32_t phase = 0;
    bool timed_out = false;

    for (;;) {
        if (tid == 0) {
            const int q = atomicAdd(in.queue, 1);
            sm.inst = q < in.n ? take_position(in, q) : -1;
        }
        __syncthreads();
        const int inst = sm.inst;
        const int si = inst >= 0 && in.sys_of ? in.sys_of[inst] : 0;
        const bool reload = inst >= 0 && si != sm.cur_sys;
        __syncthreads();
        if (inst < 0) break;
        const SysDev s = in.sys[si];
        const int M = s.M, L = s.L;
        const size_t MM = (size_t)M * M;
        if (reload) {
            // per-system constants: diagonal of V as double-float, sparse H0 rows
            for (int q = 0; q < 2; ++q)
                for (int i = tid; i < MPT; i += NTT) {
                    double2 v = make_double2(0.0, 0.0);
                    if (i < M) v = s.V[(size_t)(q % s.Vperiod) * MM + (size_t)i * M + i];
                    float hx, lx, hy, ly;
                    to_df(v.x, hx, lx);
                    to_df(v.y, hy, ly);
                    sm.vh[q][i] = make_float2(hx, hy);
                    sm.vl[q][i] = make_float2(lx, ly);
                }
            if (tid < 2)
                classify_vdiag(s.V + (size_t)(tid % s.Vperiod) * MM, M + 1, M, sm.vuni[tid],
                               sm.vch[tid], sm.vcl[tid]);
            const int nnz = s.h0_rowptr[M];
            for (int i = tid; i <= MPT; i += NTT) sm.h0rp[i] = s.h0_rowptr[min(i, M)];
            if (nnz <= MAX_NNZ)
                for (int c = tid; c < nnz; c += NTT) {
                    const double2 h = s.h0_val[c];
                    float a, b, cc, d;
                    to_df(h.x, a, b);
                    to_df(h.y, cc, d);
                    sm.h0c[c] = s.h0_col[c];
                    sm.h0h[c] = make_float2(a, cc);
                    sm.h0l[c] = make_float2(b, d);
                }
            if (tid == 0) {
                sm.cur_sys = si;
                sm.h0_cached = nnz <= MAX_NNZ;
            }
            __syncthreads();
        }
        const bool h0_cached = sm.h0_cached;
        const InstParams ip = inst_params(in, inst, M);
        const double E = ip.E;
        const uint64_t ms = ip.ms;
        const double W = ip.W;
        const double2 *SL = ip.SL;
        const double2 *SR = ip.SR;
        int st = ip.st;

        for (int n = 0; n < L && st == ST_OK; ++n) {
            slice_diag<MPT, NTT>(sm.eps, s, ms, W, E, n);
            form_gv<MPT, NTT>(Gh, Gl, sm.vh, sm.vl, M, n, L, SL, SR, sm.vuni, sm.vch, sm.vcl);
            __syncthreads();
            // Gv' = Gv + H0 - D in double-float, one row per thread, so that
            // A_n = -Gv' and the residual is R = I + Gv' X'
            for (int i = tid; i < M; i += NTT) {
                float dh, dl;
                to_df(sm.eps[i], dh, dl);
                cdf_add(Gh[i * MPT + i], Gl[i * MPT + i], make_float2(-dh, 0.f),
                        make_float2(-dl, 0.f));
                for (int c = sm.h0rp[i]; c < sm.h0rp[i + 1]; ++c) {
                    int col;
                    float2 hh, hl;
                    if (h0_cached) {
                        col = sm.h0c[c];
                        hh = sm.h0h[c];
                        hl = sm.h0l[c];
                    } else {
                        col = s.h0_col[c];
                        const double2 hd = s.h0_val[c];
                        to_df(hd.x, hh.x, hl.x);
                        to_df(hd.y, hh.y, hl.y);
                    }
                    cdf_add(Gh[i * MPT + col], Gl[i * MPT + col], hh, hl);
                }
            }
            __syncthreads();

            // row scales of Gv and X = fl32(A_n) = -Gv'_hi (identity in the
            // padding) in one pass: warp w takes rows 4w..4w+3, lanes run
            // along the row, the four maxima reduce side by side
            {
                constexpr int RPW = MPT / (NTT / 32);
                float mx[RPW];
#pragma unroll
                for (int r = 0; r < RPW; ++r) {
                    const int i = RPW * warp + r;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = lane + 32 * h;
                        const float2 g = Gh[i * MPT + j];
                        const float m = fmaxf(fabsf(g.x), fabsf(g.y));
                        mx[r] = h ? fmaxf(mx[r], m) : m;
                        sm.X[i * MPT + j] = (i < M && j < M) ? make_float2(-g.x, -g.y)
                                                             : make_float2(i == j ? 1.f : 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int r = 0; r < RPW; ++r) mx[r] = fmaxf(mx[r], __shfl_xor_sync(0xffffffffu, mx[r], o));
                if (lane < RPW) {
                    float m = mx[0];
#pragma unroll
                    for (int r = 1; r < RPW; ++r) m = lane == r ? mx[r] : m;
                    sm.rexp[RPW * warp + lane] = scale_exp(m);
                }
            }
            __syncthreads();
            st = gj_tc<NTT>(sm.X, M, sm.u.gw, sm.gj, tmem, &sm.mbar, phase);
            if (st != ST_OK) {
                timed_out = st == ST_TIMEOUT;
                break;
            }
            {
                float2 x[RA][RB];
#pragma unroll
                for (int a = 0; a < RA; ++a)
#pragma unroll
                    for (int b = 0; b < RB; ++b) x[a][b] = sm.X[(ty + TYT * a) * MPT + tx + TXT * b];
                store_inverse<MPT, TYT, TXT>(x, M, sm.gj, sm.X);
            }

            // column scales of X: thread t scans rows 8 (t / 64) .. of column t % 64
            {
                const int nn = tid & 63, part = tid >> 6;
                float mx = 0.f;
#pragma unroll 4
                for (int k = part * 8; k < part * 8 + 8; ++k) {
                    const float2 v = sm.X[k * MPT + nn];
                    mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
                }
                sm.cmax[part][nn] = mx;
            }
            __syncthreads();
            if (tid < MPT) {
                float mx = 0.f;
                for (int part = 0; part < NTT / MPT; ++part) mx = fmaxf(mx, sm.cmax[part][tid]);
                sm.cexp[tid] = scale_exp(mx);
            }
            __syncthreads();

            // B digits (three per value) and X' = X rounded to them; work item
            // e takes X[k][nn] and X[k+1][nn] (k even), lanes along nn, so each
            // digit pair is one 32-bit store into B^T[nn][k..k+1]
            for (int e = tid; e < MPT * MPT / 2; e += NTT) {
                const int k = (e >> 6) * 2, nn = e & 63;
                const int ce = sm.cexp[nn];
                const float dn = pow2f(-ce), up = pow2f(ce - 8);
                float d[2][2][NDB];   // [row k / k+1][re / im][digit]
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float2 xv = sm.X[(k + r) * MPT + nn];
                    float re, im;
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        float a = (part ? xv.y : xv.x) * dn;
#pragma unroll
                        for (int q = 0; q < NDB; ++q) {
                            a *= 256.f;
                            d[r][part][q] = rintf(a);
                            a -= d[r][part][q];
                        }
                        const float xr = (d[r][part][0] + d[r][part][1] * 0.00390625f +
                                          d[r][part][2] * 1.52587890625e-05f) * up;
                        if (part) im = xr; else re = xr;
                    }
                    sm.X[(k + r) * MPT + nn] = make_float2(re, im);
                }
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    const int K = k + 64 * part;
                    unsigned char *t = sm.w.s.bdig + (K >> 4) * NDB * B_TILE;
                    float sc = 1.f;
#pragma unroll
                    for (int q = 0; q < NDB; ++q) {
                        put_bf16x2(t + q * B_TILE, nn, K & 15, d[0][part][q] * sc,
                                   d[1][part][q] * sc);
                        sc *= 0.00390625f;
                    }
                }
            }

            // products: four groups, each two K-chunks sharing Gv columns 16g..16g+15
            // accumulators to zero (each warp the columns its epilogue reads), so
            // that every product accumulates
            {
                fence_after();
                const uint32_t tz = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 16 * (warp >> 2);
#pragma unroll
                for (int dacc = 0; dacc < NACC; ++dacc) {
                    tmem_zero8(tz + 64 * dacc);
                    tmem_zero8(tz + 64 * dacc + 8);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            for (int g = 0; g < 4 && !timed_out; ++g) {
                if (g > 0) {
                    const int ok = tid == 0 ? mbar_wait(&sm.mbar, phase) : 1;
                    phase ^= 1u;
                    if (__syncthreads_or(!ok)) { timed_out = true; break; }
                }
                // A digits of Gv columns 16g..16g+15: chunk slot 0 holds K-chunk g
                // (rows < 64: Gr, rows >= 64: Gi), slot 1 K-chunk g+4 (-Gi, Gr);
                // work item e takes row i, columns kk and kk+1 (one 32-bit store)
                for (int e = tid; e < MPT * 8; e += NTT) {
                    const int i = e >> 3, kk = (e & 7) * 2, k = 16 * g + kk;
                    const float dn = pow2f(-sm.rexp[i]);
                    const float2 gh0 = Gh[i * MPT + k], gl0 = Gl[i * MPT + k];
                    const float2 gh1 = Gh[i * MPT + k + 1], gl1 = Gl[i * MPT + k + 1];
                    // [column][re / im] running double-float remainders
                    float ah[2][2] = {{gh0.x * dn, gh0.y * dn}, {gh1.x * dn, gh1.y * dn}};
                    float al[2][2] = {{gl0.x * dn, gl0.y * dn}, {gl1.x * dn, gl1.y * dn}};
                    unsigned char *t0 = sm.u.adig;
                    unsigned char *t1 = sm.u.adig + NDA * A_TILE;
                    float scale = 1.f;
#pragma unroll
                    for (int p = 0; p < NDA; ++p) {
                        float dg[2][2];
#pragma unroll
                        for (int c = 0; c < 2; ++c)
#pragma unroll
                            for (int part = 0; part < 2; ++part) {
                                float h = ah[c][part] * 256.f, l = al[c][part] * 256.f;
                                const float d = rintf(h);
                                h -= d;
                                two_sum(h, l, ah[c][part], al[c][part]);
                                dg[c][part] = d * scale;
                            }
                        scale *= 0.00390625f;
                        put_bf16x2(t0 + p * A_TILE, i, kk, dg[0][0], dg[1][0]);        // Gr
                        put_bf16x2(t1 + p * A_TILE, i + 64, kk, dg[0][0], dg[1][0]);   // Gr
                        put_bf16x2(t0 + p * A_TILE, i + 64, kk, dg[0][1], dg[1][1]);   // Gi
                        put_bf16x2(t1 + p * A_TILE, i, kk, -dg[0][1], -dg[1][1]);      // -Gi
                    }
                }
                async_proxy_fence();
                fence_before();
                __syncthreads();
                if (tid == 0) {
                    fence_after();
                    // one MMA per A digit p against the B digits q = 0 .. min(2, 6 - p)
                    // of the chunk, stored contiguously (N = 64 per digit): products
                    // (p, q) land in accumulators p + q, i.e. columns 64 p ..
                    for (int slot = 0; slot < 2; ++slot) {
                        const int chunk = g + 4 * slot;
                        const uint64_t bd = smem_desc(smem_u32(sm.w.s.bdig + chunk * NDB * B_TILE));
#pragma unroll
                        for (int p = 0; p < NDA; ++p) {
                            const uint32_t nq = (uint32_t)min(NDB, NDA - p);
                            const uint64_t ad =
                                smem_desc(smem_u32(sm.u.adig + (slot * NDA + p) * A_TILE));
                            mma_bf16(tmem + 64 * p, ad, bd, idesc_n64 | (((64u * nq) >> 3) << 17), 1u);
                        }
                    }
                    mma_commit(&sm.mbar);
                }
            }
            if (!timed_out) {
                const int ok = tid == 0 ? mbar_wait(&sm.mbar, phase) : 1;
                phase ^= 1u;
                if (__syncthreads_or(!ok)) timed_out = true;
            }
            if (timed_out) {
                st = ST_TIMEOUT;
                break;
            }
            fence_after();

            // R = I + Gv' X' = I + sigma_i tau_n 2^-16 (D0 + ... + D6):
            // lane m of warp w holds row 32 (w % 4) + lane of [Re; Im],
            // columns 16 (w / 4) ..; the seven accumulators are summed (the
            // leading three as double-float) before the single rounding to
            // the stored R
            float rloc = 0.f;
            {
                const int m = 32 * (warp & 3) + lane, c0 = 16 * (warp >> 2);
                const int i = m & 63, part = m >> 6;
                const int re = sm.rexp[i];
                float *const Rf = reinterpret_cast<float *>(sm.u.R);
                const uint32_t tb = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + c0;
                for (int j8 = 0; j8 < 16; j8 += 8) {
                    uint32_t v0[8], v1[8], v2[8], v3[8];
                    float small[8];
                    // accumulators 3 .. 6 are below 2^-24 of the leading one:
                    // their fp32 sum is as accurate as the double-float result
                    tmem_ld8(tb + 192 + j8, v0);
                    tmem_ld8(tb + 256 + j8, v1);
                    tmem_ld8(tb + 320 + j8, v2);
                    tmem_ld8(tb + 384 + j8, v3);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int jx = 0; jx < 8; ++jx)
                        small[jx] = ((__uint_as_float(v3[jx]) + __uint_as_float(v2[jx])) +
                                     __uint_as_float(v1[jx])) + __uint_as_float(v0[jx]);
                    tmem_ld8(tb + j8, v0);
                    tmem_ld8(tb + 64 + j8, v1);
                    tmem_ld8(tb + 128 + j8, v2);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int jx = 0; jx < 8; ++jx) {
                        const int nn = c0 + j8 + jx;
                        float hs, ls, t, te;
                        two_sum(__uint_as_float(v0[jx]), __uint_as_float(v1[jx]), hs, ls);
                        two_sum(hs, __uint_as_float(v2[jx]), t, te);
                        ls += te;
                        two_sum(t, small[jx], hs, te);
                        ls += te;
                        t = hs;
                        const float sc = pow2f(re + sm.cexp[nn] - 16);
                        hs = t * sc;
                        ls *= sc;
                        if (part == 0 && i == nn) {
                            two_sum(hs, 1.0f, t, te);
                            hs = t;
                            ls += te;
                        }
                        const float r = (i < M && nn < M) ? hs + ls : 0.f;
                        Rf[2 * (i * RS + nn) + part] = r;
                        rloc = fmaxf(rloc, fabsf(r));
                    }
                }
            }
            fence_before();

            // further Neumann terms where A_n is ill-conditioned, in the B-digit
            // buffer (free once the products are read back)
            const float rmax = block_max_nonneg<NTT>(rloc, sm.redu);
            if (refinement_fails(rmax, M)) {
                // near-singular A_n: this slice in FP64, in the X and
                // residual buffers (contiguous), scratch in the B digits
                double2 *const A64 = reinterpret_cast<double2 *>(sm.X);
                fallback_form_a(A64, Gh, Gl, MPT, M, nullptr, s);
                st = gj_invert64(A64, M, fallback_scratch(sm.w.s.bdig, M));
                if (st != ST_OK) break;
                fallback_store_g(A64, Gh, Gl, MPT, MPT, M);
                continue;
            }
            const int nx = neumann_terms(rmax, M);
            float2 *const S = nx ? reinterpret_cast<float2 *>(sm.w.s.bdig) : sm.u.R;
            neumann_inplace<MPT, RS, TYT, TXT>(sm.u.R, S, M, nx);
            if (rmax > EXACT_RMAX) {
                refine_exact<MPT, RS, TYT, TXT>(sm.X, S, Gh, Gl, M);
            } else {
                if (nx) {
                    // the series into the residual's place: the B-digit
                    // buffer takes the operand terms
                    for (int e = tid; e < MPT * RS; e += NTT) sm.u.R[e] = S[e];
                    __syncthreads();
                }
                if (!refine_tc(sm, tmem, phase)) {
                    st = ST_TIMEOUT;
                    timed_out = true;
                    break;
                }
            }
            __syncthreads();
        }

        double T = 0.0;
        if (st == ST_OK) {
            T = ward_T_df<MPT, NTT>(Gh, Gl, reinterpret_cast<float4 *>(sm.X), SR, M, sm.red);
            if (in.GLL) store_gll_df<MPT, NTT>(Gh, Gl, M, in.GLL + (size_t)ip.out * M * M);
            if (!isfinite(T)) st = ST_NONFINITE;
        }
        if (tid == 0) {
            in.T[ip.out] = T;
            if (in.status) in.status[ip.out] = st;
        }
        __syncthreads();
        if (timed_out) break;
    }
    if (timed_out) {
        // the wait that ran out flipped the phase; the tensor cores may still
        // write the accumulators of that commit: give it a second bounded wait
        // before the tensor memory is released
        if (tid == 0) mbar_wait(&sm.mbar, phase ^ 1u);
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// Host launch helper.  Instances that a timed-out CTA never reaches keep the
// ST_TIMEOUT status written here first.
extern "C" cudaError_t knit_launch_mixed_tc(const InstDev *in, int grid, cudaStream_t stream)
{
    static_assert(sizeof(TcSmem) <= 227 * 1024, "shared memory budget");
    // outputs of instances a timed-out CTA never reaches keep ST_TIMEOUT
    if (in->status && !in->out_index)
        fill_status<<<(in->n + 255) / 256, 256, 0, stream>>>(in->status, in->n, ST_TIMEOUT);
    size_t smb = sizeof(TcSmem);
    cudaError_t e = cudaFuncSetAttribute(knit_sweep_mixed_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    if (e != cudaSuccess) return e;
    knit_sweep_mixed_tc_kernel<<<grid, NTT, smb, stream>>>(*in);
    return cudaGetLastError();
}

extern "C" size_t knit_mixed_tc_smem_bytes(void) { return sizeof(TcSmem); }
