// sweep_mixed_tc128.cu -- the mixed-precision slice sweep for widths 65..128
// (padded MP = 128) with all three matrix products on the tcgen05 tensor
// cores: the Gauss-Jordan panel updates, the exact residual and the
// refinement product.
//
// Same recursion and arithmetic as the other mixed sweeps (KNIT user guide
// Sec. 5.3 D knitting in slice form, Eq. 2 by block elimination; complex64
// inverse refined against a residual exact to ~2^-48, state g carried as
// hi + lo, T from G_LL by the unitarity identity, sweep_mixed.cu).  Per
// slice n, one CTA of 512 threads per instance:
//
//  A. Gv' = V g V^dagger (or Sigma_L at n = 0) (+ Sigma_R at n = L - 1)
//     + H0 - diag(E - onsite) in double-float, in place over the state in a
//     per-CTA workspace (L2); A_n = -Gv'.  X = fl32(A_n) goes straight into
//     tensor memory: lane i = row i, columns 2c, 2c + 1 = Re, Im of X[i][c]
//     (256 of the 512 columns).
//  B. Gauss-Jordan with implicit partial pivoting (the elimination of
//     gj_lookahead, panels of 8 columns) on X in tensor memory.  Per panel:
//     the four lane-quarter warps copy the panel columns out of tensor
//     memory, warp 0 runs the 8 pivot steps on them (4 rows per lane), the
//     pivot rows of X at the start of the panel are read back, one thread
//     per column forms the panel's v vectors by forward substitution, and
//     X -= U V is issued as tcgen05.mma with D = X itself: A = -[Re U | Im U]
//     (128 x 16), B^T row 2j + r = the real form of column j of V, each
//     operand cut exactly into three bf16 terms, the six products of term
//     order <= 2 accumulated in f32 -- an fp32-quality update with no read
//     back.  The next panel's 16 columns go first in an N = 16 MMA of their
//     own, so its pivot chain starts while the rest of the update runs.
//  C. The permuted inverse is copied from tensor memory into shared memory
//     in its true order (A^-1[pos[i]][perm[c]] = X[i][c]) and rounded per
//     column j to X' = 2^(t_j - 8) (d0 + d1 2^-8 + d2 2^-16), |d| <= 128,
//     t_j one more than the exponent of the column's largest entry.
//  D. R = I + Gv' X' exact: transposed, R^T = I + X'^T Gv'^T, so that the
//     tensor-memory lanes are the columns j of R: A = the three X' digits
//     (128 x 256 in real form, the contraction over X''s rows in their
//     stored order, Gv''s columns gathered to match), B = the seven digits
//     of 32 rows of Gv' per pass (cut at the row scale s_i + 1), products (p, q) of one
//     anti-diagonal d = p + q in accumulator d (seven exact f32
//     accumulators of 64 columns, 448 columns), four passes over the rows
//     of Gv'.  With every digit at most 128 in magnitude each accumulator
//     sums at most 3 x 2^14 x 256 < 2^24 per K of 256: exact by
//     construction.  The accumulators are summed (3..6 in fp32, then with
//     0..2 in double-float), scaled, the identity added and R rounded once.
//  E. Neumann terms where max|R_ij| asks for them, an error-free product
//     where max|R_ij| > 1e-4, and an FP64 inversion of the slice where the
//     series cannot converge (CUDA cores, rare; mixed_common.cuh).
//  F. g = X' + X' S: A = X' digits (rows i), B = the three bf16 terms of
//     S scaled by 2^(t_k - 8) (exact powers of two), the six products of
//     term order <= 2 into one f32 accumulator (256 columns), read back as
//     g = X' + D with two_sum into the hi + lo state.
//
// Operand tiles use the no-swizzle K-major layout of tc_common.cuh.  Every
// wait on the tensor cores is bounded (ST_TIMEOUT), and the tensor memory is
// released after a second bounded wait for the last commit.

#include <cuda_bf16.h>

#include "gj_tc.cuh"
#include "mixed_common.cuh"
#include "tc_common.cuh"

using namespace mixed;
using namespace tc;

namespace {

constexpr int MP = 128;                // padded width
constexpr int NTH = 512;               // 16 warps
constexpr int PST = 9;                 // row stride (float2) of the panel and U buffers
constexpr int NB = 8;                  // Gauss-Jordan panel width
constexpr int NDG = 7;                 // digits of Gv'
constexpr int NDX = 3;                 // digits of X'
constexpr int BT_RES = 64 * 32;        // bytes of one 64-row x 16 bf16 tile
constexpr int BT_256 = 256 * 32;       // bytes of one 256-row x 16 bf16 tile
constexpr uint32_t TMEM_COLS = 512;

// the six bf16 term products (p, q) with p + q <= 2, smallest first
__constant__ int kProdP[6] = {2, 1, 0, 1, 0, 0};
__constant__ int kProdQ[6] = {0, 1, 2, 0, 1, 0};

struct Tc128Smem {
    union {
        struct {                                       // Gauss-Jordan
            struct {
                unsigned key;                          // the warp's best pivot key
                unsigned pad;
                float2 row[NB];                        // that row's panel entries
            } cand[2][4];                              // per step parity, per lane-quarter warp
            float2 U[MP * PST];                        // u vectors of the panel
            float2 prow[NB * MP];                      // pivot rows at the start of the panel
            alignas(128) unsigned char adg[3 * A_TILE];    // -[Re U | Im U] terms, 128 x 16
            alignas(128) unsigned char bdg[3 * BT_256];    // V terms in real form, 256 x 16
        } gj;
        struct {                                       // residual
            alignas(128) unsigned char lres[16][NDX * A_TILE];   // X'^T digits of every K-chunk
            alignas(128) unsigned char b[2][NDG * BT_RES];       // Gv' digits of a K-chunk
        } res;
        struct {                                       // products X' S and R S
            alignas(128) unsigned char a[2][NDX * A_TILE];
            alignas(128) unsigned char b[2][3 * BT_256];
        } ref;
        struct {                                       // slice set-up: V's 4 x 4 block rows
            float2 vh[MP * 4], vl[MP * 4];             // row r: V[r][4 (r / 4) + b], b = 0 .. 3
        } va;
        struct {                                       // double-float inversion of a slice
            float2 hi[MP * MP];                        // hi parts of X, row-major
            float4 U[MP * 8];                          // u vectors of the panel, row i at 8 i
            float4 V[8 * MP];                          // v vectors of the panel, step c at c MP
            float4 prow[8];                            // the pivot row's panel entries
            float4 rinv[8];                            // 1 / pivot of each step
            float key[4];                              // per warp: best pivot key and its row
            int idx[4];
            int pinv[MP];                              // row of the inverse that column j is
        } fb;
    } u;
    double eps[MP];
    int vkind[4];                  // per coupling V[q]: 0 diagonal, 1 4 x 4 blocks, 2 tridiagonal
    int vuni[4];
    float vch[4], vcl[4];
    int rexp[MP];                  // Gv' row exponents (one bit of headroom included)
    int cexp[MP];                  // X' column exponents, by true column
    unsigned rmaxu[MP];            // row maxima of |Gv'| (float bits)
    unsigned cmaxu[MP];            // column maxima of |X|, by stored column (float bits)
    int perm[MP];
    int pos[MP];
    float2 rinv[NB];
    int flag;
    double red[NTH / 32];
    unsigned redu[NTH / 32];
    unsigned long long bar[4];     // 0: next-panel MMAs, 1: rest of the panel update, 2-3: chunk slots
    uint32_t tmem;
    int inst;
    int cur_sys;
};

// per-CTA device workspace
static_assert((2 * MP + 1) * 16 + (MP + 2) * 4 <= (2 * MP + 48) * 16, "fallback scratch");
static_assert(2 * (MP / 4) * (MP / 4) <= 4 * NTH, "gv_blocks4 keeps at most 4 items per thread");

struct Tc128Work {
    float4 Gh[(MP / 2) * MP];      // state g / Gv' (hi): column pair jp, row i at jp * MP + i
    float4 Gl[(MP / 2) * MP];      // (lo)
    float4 Xt[(MP / 2) * MP];      // X' in true order, same layout
    float2 R[MP * MP];             // residual, row-pair layout (sidx)
    float2 S1[MP * MP];            // Neumann terms (two buffers in turn)
    float2 S2[MP * MP];
    double2 A64[MP * MP];          // FP64 fallback matrix; G_LL for the trace
    double2 scr[2 * MP + 48];      // gj_invert64 scratch: (2M + 1) complex128 + (M + 2) ints
};

// float2 index of element (k, j) in the row-pair layout of R and S: rows k
// and k + 1 (k even) of column j are adjacent
KNIT_DEV int sidx(int k, int j) { return (((k >> 1) * MP + j) << 1) | (k & 1); }

KNIT_DEV float pow2f(int e) { return __int_as_float((127 + e) << 23); }

KNIT_DEV int scale_exp(float mx)
{
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    return e;
}

KNIT_DEV void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                   "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                   "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                   "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
}

KNIT_DEV void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
                 "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
                   "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]),
                   "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
                 : "memory");
}

// three exact bf16 terms of 8 values, packed two per word (value 2c in the
// low half), each term as two 16-byte halves of a 16-value tile row
KNIT_DEV void split8(const float (&x)[8], uint4 &t0, uint4 &t1, uint4 &t2)
{
    uint32_t h[8], m[8], l[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) bf16_split3(x[c], h[c], m[c], l[c]);
    t0 = make_uint4(pack_hi16(h[0], h[1]), pack_hi16(h[2], h[3]), pack_hi16(h[4], h[5]), pack_hi16(h[6], h[7]));
    t1 = make_uint4(pack_hi16(m[0], m[1]), pack_hi16(m[2], m[3]), pack_hi16(m[4], m[5]), pack_hi16(m[6], m[7]));
    t2 = make_uint4(pack_hi16(l[0], l[1]), pack_hi16(l[2], l[3]), pack_hi16(l[4], l[5]), pack_hi16(l[6], l[7]));
}

// write the three terms of 16 K-values of tile row r (row stride of the
// term tiles: `stride` bytes)
KNIT_DEV void put_terms16(unsigned char *tile, int stride, int r, const float (&lo)[8],
                          const float (&hi)[8])
{
    uint4 a0, a1, a2, b0, b1, b2;
    split8(lo, a0, a1, a2);
    split8(hi, b0, b1, b2);
    unsigned char *p = tile + tile_off(r, 0);
    *reinterpret_cast<uint4 *>(p) = a0;
    *reinterpret_cast<uint4 *>(p + 128) = b0;
    *reinterpret_cast<uint4 *>(p + stride) = a1;
    *reinterpret_cast<uint4 *>(p + stride + 128) = b1;
    *reinterpret_cast<uint4 *>(p + 2 * stride) = a2;
    *reinterpret_cast<uint4 *>(p + 2 * stride + 128) = b2;
}

// 2^-e x cut into 7 digits (double-float input), digit p pre-scaled by 2^-8p
KNIT_DEV void digits7(float h, float l, float dn, float (&dg)[NDG])
{
    float ah = h * dn, al = l * dn;
    float scale = 1.f;
#pragma unroll
    for (int p = 0; p < NDG; ++p) {
        float th = ah * 256.f, tl = al * 256.f;
        const float d = rintf(th);
        th -= d;
        two_sum(th, tl, ah, al);
        dg[p] = d * scale;
        scale *= 0.00390625f;
    }
}

// X' digits (exact: X' is a 24-bit value at the column scale)
KNIT_DEV void digits3(float x, float dn, float (&dg)[NDX])
{
    float a = x * dn;
    float scale = 1.f;
#pragma unroll
    for (int q = 0; q < NDX; ++q) {
        a *= 256.f;
        const float d = rintf(a);
        a -= d;
        dg[q] = d * scale;
        scale *= 0.00390625f;
    }
}

// Commits in flight and the phase each barrier waits for next, kept
// identically by every thread (all control flow around them is uniform).
struct Bars {
    uint32_t ph[4];
    uint32_t pend[4];
};

// thread 0 waits (bounded) for barrier b; every thread learns the outcome.
// On success the phase flips; after a time-out it stays, so that the
// cleanup can wait once more for the commit still in flight.
__device__ __forceinline__ bool bar_wait(Tc128Smem &sm, Bars &br, int b)
{
    const int ok = threadIdx.x == 0 ? mbar_wait(&sm.bar[b], br.ph[b]) : 1;
    if (__syncthreads_or(!ok)) return false;
    br.ph[b] ^= 1u;
    br.pend[b] = 0u;
    return true;
}

__global__ void fill_status128(int *st, int n, int v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) st[i] = v;
}

// ---------------------------------------------------------------------------
// A. Gv' in place over the state, X = -Gv'_hi into tensor memory

// V g V^dagger for 4 x 4 block-diagonal V (coupling of parity q) into the
// workspace buffers S1 / S2 (hi / lo, same layout as the state): V's block
// rows are staged in shared memory first; work item (block B, C; column
// half hc) forms columns 4C + 2hc, 4C + 2hc + 1 of block (B, C)
__device__ void gv_blocks4(Tc128Work &wk, Tc128Smem &sm, const SysDev &s, int M, int q)
{
    const size_t MM = (size_t)M * M;
    const double2 *Vq = s.V + (size_t)(q % s.Vperiod) * MM;
    for (int e = threadIdx.x; e < MP * 4; e += NTH) {
        const int r = e >> 2, c = 4 * (r >> 2) + (e & 3);
        const double2 v = (r < M && c < M) ? Vq[(size_t)r * M + c] : make_double2(0.0, 0.0);
        float2 h, l;
        to_df(v.x, h.x, l.x);
        to_df(v.y, h.y, l.y);
        sm.u.va.vh[e] = h;
        sm.u.va.vl[e] = l;
    }
    __syncthreads();
    float4 *const oh = reinterpret_cast<float4 *>(wk.S1);
    float4 *const ol = reinterpret_cast<float4 *>(wk.S2);
    const int nb = (M + 3) / 4;
    for (int e = threadIdx.x; e < 2 * nb * nb; e += NTH) {
        const int hc = e & 1, B = (e >> 1) % nb, C = (e >> 1) / nb;
        // u[a][s] = sum_b g[4B+a][4C+b] conj(V[4C+2hc+s][4C+b])
        float2 uh[4][2], ul[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float2 gh[4], gl[4];
#pragma unroll
            for (int cp = 0; cp < 2; ++cp) {
                const int idx = (2 * C + cp) * MP + 4 * B + a;
                const float4 h = wk.Gh[idx], l = wk.Gl[idx];
                gh[2 * cp] = make_float2(h.x, h.y);
                gh[2 * cp + 1] = make_float2(h.z, h.w);
                gl[2 * cp] = make_float2(l.x, l.y);
                gl[2 * cp + 1] = make_float2(l.z, l.w);
            }
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const int vr = 4 * C + 2 * hc + s2;
                float2 sh = make_float2(0.f, 0.f), sl = make_float2(0.f, 0.f);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    float2 vh = sm.u.va.vh[vr * 4 + b], vl = sm.u.va.vl[vr * 4 + b];
                    if (vh.x == 0.f && vh.y == 0.f) continue;
                    vh.y = -vh.y;
                    vl.y = -vl.y;
                    float2 ph, pl;
                    cdf_mul(gh[b], gl[b], vh, vl, ph, pl);
                    cdf_add(sh, sl, ph, pl);
                }
                uh[a][s2] = sh;
                ul[a][s2] = sl;
            }
        }
        // Gv[a][s] = sum_b V[4B+a][4B+b] u[b][s]
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float2 gvh[2], gvl[2];
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                float2 sh = make_float2(0.f, 0.f), sl = make_float2(0.f, 0.f);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float2 vh = sm.u.va.vh[(4 * B + a) * 4 + b], vl = sm.u.va.vl[(4 * B + a) * 4 + b];
                    if (vh.x == 0.f && vh.y == 0.f) continue;
                    float2 ph, pl;
                    cdf_mul(vh, vl, uh[b][s2], ul[b][s2], ph, pl);
                    cdf_add(sh, sl, ph, pl);
                }
                gvh[s2] = sh;
                gvl[s2] = sl;
            }
            const int idx = (2 * C + hc) * MP + 4 * B + a;
            oh[idx] = make_float4(gvh[0].x, gvh[0].y, gvh[1].x, gvh[1].y);
            ol[idx] = make_float4(gvl[0].x, gvl[0].y, gvl[1].x, gvl[1].y);
        }
    }
}

// V g V^dagger for a tridiagonal V (coupling q) in two passes through the
// workspace: U = g V^dagger into S1 / S2, then V U back into the state
// buffers (g is no longer needed); V's three diagonals staged in shared
// memory (row r: V[r][r - 1], V[r][r], V[r][r + 1] at r, 128 + r, 256 + r)
__device__ void gv_tridiag(Tc128Work &wk, Tc128Smem &sm, const SysDev &s, int M, int q)
{
    const size_t MM = (size_t)M * M;
    const double2 *Vq = s.V + (size_t)(q % s.Vperiod) * MM;
    for (int e = threadIdx.x; e < 3 * MP; e += NTH) {
        const int k = e / MP - 1, r = e % MP, c = r + k;
        const double2 v = (r < M && c >= 0 && c < M) ? Vq[(size_t)r * M + c] : make_double2(0.0, 0.0);
        float2 h, l;
        to_df(v.x, h.x, l.x);
        to_df(v.y, h.y, l.y);
        sm.u.va.vh[e] = h;
        sm.u.va.vl[e] = l;
    }
    __syncthreads();
    float4 *const uh = reinterpret_cast<float4 *>(wk.S1);
    float4 *const ul = reinterpret_cast<float4 *>(wk.S2);
    // U[a][j] = sum_{b = j-1 .. j+1} g[a][b] conj(V[j][b])
    for (int e = threadIdx.x; e < (MP / 2) * MP; e += NTH) {
        const int a = e % MP, jp = e / MP;
        float2 gh[4], gl[4];   // g[a][2jp - 1 .. 2jp + 2]
        {
            const float4 h0 = jp > 0 ? wk.Gh[(jp - 1) * MP + a] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 l0 = jp > 0 ? wk.Gl[(jp - 1) * MP + a] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 h1 = wk.Gh[jp * MP + a], l1 = wk.Gl[jp * MP + a];
            const float4 h2 = jp + 1 < MP / 2 ? wk.Gh[(jp + 1) * MP + a] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 l2 = jp + 1 < MP / 2 ? wk.Gl[(jp + 1) * MP + a] : make_float4(0.f, 0.f, 0.f, 0.f);
            gh[0] = make_float2(h0.z, h0.w); gl[0] = make_float2(l0.z, l0.w);
            gh[1] = make_float2(h1.x, h1.y); gl[1] = make_float2(l1.x, l1.y);
            gh[2] = make_float2(h1.z, h1.w); gl[2] = make_float2(l1.z, l1.w);
            gh[3] = make_float2(h2.x, h2.y); gl[3] = make_float2(l2.x, l2.y);
        }
        float2 oh[2], ol[2];
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            const int j = 2 * jp + s2;
            float2 sh = make_float2(0.f, 0.f), sl = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = -1; k <= 1; ++k) {
                float2 vh = sm.u.va.vh[(k + 1) * MP + j], vl = sm.u.va.vl[(k + 1) * MP + j];
                if (vh.x == 0.f && vh.y == 0.f) continue;
                vh.y = -vh.y;
                vl.y = -vl.y;
                float2 ph, pl;
                cdf_mul(gh[s2 + k + 1], gl[s2 + k + 1], vh, vl, ph, pl);
                cdf_add(sh, sl, ph, pl);
            }
            oh[s2] = sh;
            ol[s2] = sl;
        }
        uh[e] = make_float4(oh[0].x, oh[0].y, oh[1].x, oh[1].y);
        ul[e] = make_float4(ol[0].x, ol[0].y, ol[1].x, ol[1].y);
    }
    __syncthreads();
    // Gv[i][j] = sum_{a = i-1 .. i+1} V[i][a] U[a][j]
    for (int e = threadIdx.x; e < (MP / 2) * MP; e += NTH) {
        const int i = e % MP, jp = e / MP;
        float2 oh[2] = {}, ol[2] = {};
#pragma unroll
        for (int k = -1; k <= 1; ++k) {
            const int a = i + k;
            const float2 vh = sm.u.va.vh[(k + 1) * MP + i], vl = sm.u.va.vl[(k + 1) * MP + i];
            if (a < 0 || a >= MP || (vh.x == 0.f && vh.y == 0.f)) continue;
            const float4 h = uh[jp * MP + a], l = ul[jp * MP + a];
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                float2 ph, pl;
                cdf_mul(vh, vl, s2 ? make_float2(h.z, h.w) : make_float2(h.x, h.y),
                        s2 ? make_float2(l.z, l.w) : make_float2(l.x, l.y), ph, pl);
                cdf_add(oh[s2], ol[s2], ph, pl);
            }
        }
        wk.Gh[e] = make_float4(oh[0].x, oh[0].y, oh[1].x, oh[1].y);
        wk.Gl[e] = make_float4(ol[0].x, ol[0].y, ol[1].x, ol[1].y);
    }
}

// Gv' = (V g V^dagger or Sigma_L) + Sigma_R + H0 - diag(E - onsite) in
// double-float, elementwise into the state buffers; zero in the padding.
// vmode: 0 general diagonal V, 1 V g V^dagger already formed (4 x 4 block
// couplings: read from S1 / S2) or |v|^2 = 1, 2 scalar |v|^2 (vch + vcl)
__device__ void gv_elementwise(Tc128Work &wk, Tc128Smem &sm, const SysDev &s, int M, int n, int L,
                               int vmode, bool from_s, const double2 *SL, const double2 *SR)
{
    const int q = n % s.Vperiod;
    const double2 *Vd = s.V + (size_t)(q % s.Vperiod) * M * M;   // diagonal at stride M + 1
    const float4 *srch = from_s ? reinterpret_cast<const float4 *>(wk.S1) : wk.Gh;
    const float4 *srcl = from_s ? reinterpret_cast<const float4 *>(wk.S2) : wk.Gl;
    for (int e = threadIdx.x; e < (MP / 2) * MP; e += NTH) {
        const int i = e % MP, jp = e / MP;
        const float4 h4 = srch[e], l4 = srcl[e];
        const float4 hh4 = s.h0_dfh[e], hl4 = s.h0_dfl[e];
        float2 oh[2], ol[2];
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            const int j = 2 * jp + s2;
            float2 gh = s2 ? make_float2(h4.z, h4.w) : make_float2(h4.x, h4.y);
            float2 gl = s2 ? make_float2(l4.z, l4.w) : make_float2(l4.x, l4.y);
            if (i < M && j < M) {
                if (n == 0) {
                    const double2 v = SL[(size_t)i * M + j];
                    float a, b, c, d;
                    to_df(v.x, a, b);
                    to_df(v.y, c, d);
                    gh = make_float2(a, c);
                    gl = make_float2(b, d);
                } else if (vmode == 2) {
                    cdf_mul(gh, gl, make_float2(sm.vch[q], 0.f), make_float2(sm.vcl[q], 0.f), gh, gl);
                } else if (vmode == 0) {
                    const double2 vi = Vd[(size_t)i * (M + 1)], vj = Vd[(size_t)j * (M + 1)];
                    float2 vih, vil, vjh, vjl, th, tl;
                    to_df(vi.x, vih.x, vil.x);
                    to_df(vi.y, vih.y, vil.y);
                    to_df(vj.x, vjh.x, vjl.x);
                    to_df(-vj.y, vjh.y, vjl.y);
                    cdf_mul(gh, gl, vjh, vjl, th, tl);
                    cdf_mul(vih, vil, th, tl, gh, gl);
                }
                if (n == L - 1) {
                    const double2 v = SR[(size_t)i * M + j];
                    float a, b, c, d;
                    to_df(v.x, a, b);
                    to_df(v.y, c, d);
                    cdf_add(gh, gl, make_float2(a, c), make_float2(b, d));
                }
                cdf_add(gh, gl, s2 ? make_float2(hh4.z, hh4.w) : make_float2(hh4.x, hh4.y),
                        s2 ? make_float2(hl4.z, hl4.w) : make_float2(hl4.x, hl4.y));
                if (i == j) {
                    float dh, dl;
                    to_df(sm.eps[i], dh, dl);
                    cdf_add(gh, gl, make_float2(-dh, 0.f), make_float2(-dl, 0.f));
                }
            } else {
                gh = gl = make_float2(0.f, 0.f);
            }
            oh[s2] = gh;
            ol[s2] = gl;
        }
        wk.Gh[e] = make_float4(oh[0].x, oh[0].y, oh[1].x, oh[1].y);
        wk.Gl[e] = make_float4(ol[0].x, ol[0].y, ol[1].x, ol[1].y);
    }
}

// X = -Gv'_hi (identity in the padding) into tensor memory and the partial
// row maxima of |Gv'|: warp w takes rows 32 (w & 3) + lane and complex
// columns 32 (w >> 2) .. + 31
__device__ void x_to_tmem(const Tc128Work &wk, Tc128Smem &sm, uint32_t tmem, int M)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qd = warp & 3, cg = warp >> 2, i = 32 * qd + lane;
    float mx = 0.f;
#pragma unroll 1
    for (int gi = 0; gi < 4; ++gi) {
        uint32_t v[16];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int jp = 16 * cg + 4 * gi + u;
            const float4 h = wk.Gh[jp * MP + i];
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(h.x), fabsf(h.y)), fmaxf(fabsf(h.z), fabsf(h.w))));
            const int j0 = 2 * jp;
            float2 x0 = make_float2(-h.x, -h.y), x1 = make_float2(-h.z, -h.w);
            if (i >= M || j0 >= M) x0 = make_float2(i == j0 ? 1.f : 0.f, 0.f);
            if (i >= M || j0 + 1 >= M) x1 = make_float2(i == j0 + 1 ? 1.f : 0.f, 0.f);
            v[4 * u] = __float_as_uint(x0.x);
            v[4 * u + 1] = __float_as_uint(x0.y);
            v[4 * u + 2] = __float_as_uint(x1.x);
            v[4 * u + 3] = __float_as_uint(x1.y);
        }
        tmem_st16(tmem + ((uint32_t)(32 * qd) << 16) + 64 * cg + 16 * gi, v);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    atomicMax(&sm.rmaxu[i], __float_as_uint(mx));
}

// ---------------------------------------------------------------------------
// B. Gauss-Jordan on X in tensor memory

__device__ int gj_tmem(Tc128Smem &sm, uint32_t tmem, int M, Bars &br)
{
    constexpr int IB = 7;
    constexpr unsigned IMASK = (1u << IB) - 1u, FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Mp = (M + NB - 1) / NB * NB;   // columns that the updates touch
    const int NP = Mp / NB;
    // warps 0 .. 3 own the rows of their tensor-memory lane quarter
    const int myrow = 32 * (warp & 3) + lane;
    bool open = warp < 4 && myrow < M;   // the row may still become a pivot row
    int st = ST_OK;
    for (int P = 0; P < NP; ++P) {
        const int K = P * NB, nk = min(NB, M - K);
        bool to0 = false;   // the wait for the previous panel's first MMAs ran out
        // 1-2. the pivot steps, spread over the four lane-quarter warps: each
        //      lane holds its own row's panel entries (out of tensor memory,
        //      after the previous panel's first MMAs); per step every warp
        //      posts its best candidate (key and row) and one 128-thread
        //      barrier lets all four agree on the pivot
        if (warp < 4) {
            if (P > 0) to0 = !mbar_wait(&sm.bar[0], br.ph[0]);
            fence_after();
            float2 pc[NB];
            {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 2 * K, v);
                wait_ld();
#pragma unroll
                for (int c = 0; c < NB; ++c) pc[c] = make_float2(__uint_as_float(v[2 * c]), __uint_as_float(v[2 * c + 1]));
            }
            bool bad = to0;
#pragma unroll
            for (int kk = 0; kk < NB; ++kk) {
                if (kk < nk) {
                    const unsigned kt = open ? ((__float_as_uint(cabs1f(pc[kk])) & ~IMASK) |
                                                (IMASK - (unsigned)myrow))
                                             : 0u;
                    const unsigned wmax = __reduce_max_sync(FULL, kt);
                    auto &slot = sm.u.gj.cand[kk & 1][warp];
                    if (lane == 0) slot.key = wmax;
                    if (wmax != 0u && kt == wmax)
#pragma unroll
                        for (int c = kk; c < NB; ++c) slot.row[c] = pc[c];
                    asm volatile("bar.sync 2, 128;" ::: "memory");
                    unsigned best = sm.u.gj.cand[kk & 1][0].key;
#pragma unroll
                    for (int w2 = 1; w2 < 4; ++w2) best = max(best, sm.u.gj.cand[kk & 1][w2].key);
                    bad |= (best & ~IMASK) == 0u;
                    const int p = (int)(IMASK - (best & IMASK));
                    const auto &win = sm.u.gj.cand[kk & 1][(p >> 5) & 3];
                    float2 prow[NB];
#pragma unroll
                    for (int c = kk; c < NB; ++c) prow[c] = win.row[c];
                    const float2 rinv = crcp_fastf(prow[kk]);
                    float2 u = pc[kk];
                    u.x -= myrow == p ? 1.f : 0.f;
#pragma unroll
                    for (int c = kk + 1; c < NB; ++c) pc[c] = cfmsf(u, cmulf(prow[c], rinv), pc[c]);
                    sm.u.gj.U[myrow * PST + kk] = u;
                    open = open && myrow != p;
                    if (warp == 0 && lane == 0) {
                        sm.perm[K + kk] = p;
                        sm.rinv[kk] = rinv;
                    }
                }
            }
            // steps a partial panel does not take contribute nothing
            for (int kk = nk; kk < NB; ++kk) sm.u.gj.U[myrow * PST + kk] = make_float2(0.f, 0.f);
            if (warp == 0 && lane == 0) sm.flag = bad ? 1 : 0;
        }
        // 3. X at the start of the panel (the whole previous update done):
        //    the pivot rows into shared memory
        {
            const int ok = (P > 0 && tid == 0) ? mbar_wait(&sm.bar[1], br.ph[1]) : 1;
            if (__syncthreads_or(!ok || to0)) {
                st = ST_TIMEOUT;
                break;
            }
            if (P > 0) {
                br.ph[0] ^= 1u;
                br.ph[1] ^= 1u;
                br.pend[0] = br.pend[1] = 0u;
            }
        }
        if (sm.flag) {
            st = ST_SINGULAR;
            break;
        }
        fence_after();
        {
            const int qd = warp & 3, cg = warp >> 2, i = 32 * qd + lane;
            int kpiv = -1;
            for (int kk = 0; kk < nk; ++kk) kpiv = sm.perm[K + kk] == i ? kk : kpiv;
            if (__any_sync(FULL, kpiv >= 0)) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + 64 * cg + 32 * h, v);
                    wait_ld();
                    if (kpiv >= 0)
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            sm.u.gj.prow[kpiv * MP + 32 * cg + 16 * h + c] =
                                make_float2(__uint_as_float(v[2 * c]), __uint_as_float(v[2 * c + 1]));
                }
            }
        }
        fence_before();
        __syncthreads();
        // 4. v vectors (one thread per column j) and the operand terms:
        //    B^T rows 2j = [Re v_k[j] | -Im v_k[j]], 2j + 1 = [Im v_k[j] | Re v_k[j]];
        //    A rows i = -[Re u_k[i] | Im u_k[i]]
        if (tid < MP) {
            const int j = tid;
            float2 vj[NB];
#pragma unroll
            for (int kk = 0; kk < NB; ++kk) {
                vj[kk] = make_float2(0.f, 0.f);
                if (kk < nk) {
                    const int p = sm.perm[K + kk];
                    float2 r = sm.u.gj.prow[kk * MP + j];
                    if (j == K + kk) r.x += 1.f;
#pragma unroll
                    for (int c = 0; c < kk; ++c) r = cfmsf(sm.u.gj.U[p * PST + c], vj[c], r);
                    vj[kk] = cmulf(r, sm.rinv[kk]);
                }
            }
            float re[NB], im[NB], nim[NB];
#pragma unroll
            for (int kk = 0; kk < NB; ++kk) {
                re[kk] = vj[kk].x;
                im[kk] = vj[kk].y;
                nim[kk] = -vj[kk].y;
            }
            put_terms16(sm.u.gj.bdg, BT_256, 2 * j, re, nim);
            put_terms16(sm.u.gj.bdg, BT_256, 2 * j + 1, im, re);
        } else if (tid < 2 * MP) {
            const int i = tid - MP;
            float re[NB], im[NB];
#pragma unroll
            for (int kk = 0; kk < NB; ++kk) {
                const float2 uv = sm.u.gj.U[i * PST + kk];
                re[kk] = -uv.x;
                im[kk] = -uv.y;
            }
            put_terms16(sm.u.gj.adg, A_TILE, i, re, im);
        }
        async_proxy_fence();
        fence_before();
        __syncthreads();
        // 5. the update X -= U V: the next panel's 16 columns first (bar 0),
        //    then the rest of the touched columns (bar 1); issued from warp 4,
        //    so that the pivot warp is not held while the MMA queue drains
        if (tid == 128) {
            fence_after();
            const int K2 = K + NB;
            auto issue = [&](int c0, int ncol) {   // tensor-memory columns c0 .. c0 + ncol - 1
                if (ncol <= 0) return;
                const uint32_t idesc = idesc_bf16_m128((uint32_t)ncol);
#pragma unroll
                for (int pr = 0; pr < 6; ++pr) {
                    const uint64_t ad = smem_desc(smem_u32(sm.u.gj.adg + kProdP[pr] * A_TILE));
                    const uint64_t bd = smem_desc(smem_u32(sm.u.gj.bdg + kProdQ[pr] * BT_256 + (c0 / 8) * 256));
                    mma_bf16(tmem + (uint32_t)c0, ad, bd, idesc, 1u);
                }
            };
            if (K2 < Mp) {
                issue(2 * K2, 16);
                mma_commit(&sm.bar[0]);
                issue(0, 2 * K2);
                issue(2 * K2 + 16, 2 * Mp - 2 * K2 - 16);
            } else {
                issue(0, 2 * Mp);
            }
            mma_commit(&sm.bar[1]);
        }
        if (K + NB < Mp) br.pend[0] = 1u;
        br.pend[1] = 1u;
    }
    if (st == ST_OK) {
        // the last update complete before anyone reads X
        if (!bar_wait(sm, br, 1)) st = ST_TIMEOUT;   // polled by thread 0, shared by the block
        fence_after();
    }
    return st;
}

// ---------------------------------------------------------------------------
// C. X' from the permuted X in tensor memory (A^-1[pos[i]][perm[c]] =
//    X[i][c]): column exponents, then per element the three digits at the
//    column scale, written straight into the residual's A tiles (row j =
//    true column, K = true row; chunk = part * 8 + row / 16) and X' itself
//    in true order into the workspace

__device__ void x_prime_from_tmem(Tc128Smem &sm, Tc128Work &wk, uint32_t tmem, int M)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int k = tid; k < MP; k += NTH) {
        if (k >= M) sm.perm[k] = k;
        sm.cmaxu[k] = 0u;
    }
    __syncthreads();
    for (int k = tid; k < MP; k += NTH) sm.pos[sm.perm[k]] = k;
    const int qd = warp & 3, cg = warp >> 2, i = 32 * qd + lane;
    // column maxima over the stored rows (warp reductions, then across quarters)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + 64 * cg + 32 * h, v);
        wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float m = fmaxf(fabsf(__uint_as_float(v[2 * c])), fabsf(__uint_as_float(v[2 * c + 1])));
            const unsigned mu = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
            if (lane == c) atomicMax(&sm.cmaxu[32 * cg + 16 * h + c], mu);
        }
    }
    __syncthreads();
    if (tid < MP) {
        sm.cexp[sm.perm[tid]] = scale_exp(__uint_as_float(sm.cmaxu[tid])) + 1;   // |digits| <= 128
        sm.rexp[tid] = scale_exp(__uint_as_float(sm.rmaxu[tid])) + 1;
    }
    __syncthreads();
    float2 *const xt = reinterpret_cast<float2 *>(wk.Xt);
    const int ti = sm.pos[i];
    // the residual contracts over X''s rows in their stored order (K
    // position i, the Gv' columns gathered through pos), so that a warp's
    // lanes write 32 consecutive K positions of one tile row: even lanes
    // store their value and their neighbour's as one word
    unsigned char *const tre = sm.u.res.lres[i >> 4];        // real part: chunk i / 16
    unsigned char *const tim = sm.u.res.lres[8 + (i >> 4)];  // imaginary part
    const int kk = i & 14;
    const bool even = (lane & 1) == 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + 64 * cg + 32 * h, v);
        wait_ld();
#pragma unroll 4
        for (int c = 0; c < 16; ++c) {
            const int j = sm.perm[32 * cg + 16 * h + c];
            const int ce = sm.cexp[j];
            const float dn = pow2f(-ce), up = pow2f(ce - 8);
            float dr[NDX], di[NDX];
            digits3(__uint_as_float(v[2 * c]), dn, dr);
            digits3(__uint_as_float(v[2 * c + 1]), dn, di);
            const int off = tile_off(j, kk);
#pragma unroll
            for (int q = 0; q < NDX; ++q) {
                const float nr = __shfl_down_sync(0xffffffffu, dr[q], 1);
                const float ni = __shfl_down_sync(0xffffffffu, di[q], 1);
                if (even) {
                    *reinterpret_cast<__nv_bfloat162 *>(tre + q * A_TILE + off) = __floats2bfloat162_rn(dr[q], nr);
                    *reinterpret_cast<__nv_bfloat162 *>(tim + q * A_TILE + off) = __floats2bfloat162_rn(di[q], ni);
                }
            }
            xt[((j >> 1) * MP + ti) * 2 + (j & 1)] =
                make_float2((dr[0] + dr[1] + dr[2]) * up, (di[0] + di[1] + di[2]) * up);
        }
    }
    fence_before();
    __syncthreads();
}

// ---------------------------------------------------------------------------
// D. the residual R = I + Gv' X' (transposed on the tensor cores)

// B tiles of chunk c (rows 2i' = Gr, 2i' + 1 = Gi of Gv' rows i = 32 pass + i',
// K = k - 16 c) from the double-float Gv' in the workspace, seven digits
// side by side (digit p at p * BT_RES).  Work item = thread: warp w takes
// tile rows 8 (w % 8) .. + 7 and K pairs 4 (w / 8) .. + 3, lane l row
// l / 4 and K pair l % 4 of those, so that a warp's 32 four-byte stores fill
// 128 contiguous bytes (no bank conflicts); tile row r = 2 i' + part.  The
// loads (one float4 of hi and one of lo: (i, k) and (i, k + 1)) are issued
// a chunk ahead.
struct GvPre {
    float4 h, l;
};

KNIT_DEV void res_b_item(int &ip, int &kk, int &part)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int r = 8 * (w & 7) + (l >> 2);
    ip = r >> 1;
    part = r & 1;
    kk = 2 * ((l & 3) + 4 * (w >> 3));
}

// K positions are X''s stored rows: Gv' columns pos[16 (c % 8) + kk] and the next
KNIT_DEV GvPre res_b_load(const Tc128Work &wk, const Tc128Smem &sm, int pass, int c)
{
    int ip, kk, part;
    res_b_item(ip, kk, part);
    const int i = 32 * pass + ip, ks = 16 * (c & 7) + kk;
    const int k0 = sm.pos[ks], k1 = sm.pos[ks + 1];
    const float2 *gh = reinterpret_cast<const float2 *>(wk.Gh);
    const float2 *gl = reinterpret_cast<const float2 *>(wk.Gl);
    const int f0 = ((k0 >> 1) * MP + i) * 2 + (k0 & 1), f1 = ((k1 >> 1) * MP + i) * 2 + (k1 & 1);
    const float2 h0 = gh[f0], h1 = gh[f1], l0 = gl[f0], l1 = gl[f1];
    GvPre g;
    g.h = make_float4(h0.x, h0.y, h1.x, h1.y);
    g.l = make_float4(l0.x, l0.y, l1.x, l1.y);
    return g;
}

__device__ void res_b_build(const GvPre &g, const Tc128Smem &sm, unsigned char *b, int pass)
{
    int ip, kk, part;
    res_b_item(ip, kk, part);
    const float dn = pow2f(-sm.rexp[32 * pass + ip]);
    float dg0[NDG], dg1[NDG];
    digits7(part ? g.h.y : g.h.x, part ? g.l.y : g.l.x, dn, dg0);
    digits7(part ? g.h.w : g.h.z, part ? g.l.w : g.l.z, dn, dg1);
#pragma unroll
    for (int p = 0; p < NDG; ++p) put_bf16x2(b + p * BT_RES, 2 * ip + part, kk, dg0[p], dg1[p]);
}

// the B tiles of chunk c + 8 from those of chunk c: rows 2i' = -Gi, 2i' + 1 = Gr
__device__ void res_b_swap(const unsigned char *src, unsigned char *dst)
{
    // one 16-byte piece per work item: digit p, row r, K half h
    for (int e = threadIdx.x; e < NDG * 64 * 2; e += NTH) {
        const int h = e & 1, r = (e >> 1) & 63, p = e >> 7;
        const int rs = r ^ 1;
        const uint4 v = *reinterpret_cast<const uint4 *>(src + p * BT_RES + tile_off(rs, 8 * h));
        uint4 w = v;
        if ((r & 1) == 0) {   // -Gi: flip the sign bits of the eight bf16 values
            w.x ^= 0x80008000u;
            w.y ^= 0x80008000u;
            w.z ^= 0x80008000u;
            w.w ^= 0x80008000u;
        }
        *reinterpret_cast<uint4 *>(dst + p * BT_RES + tile_off(r, 8 * h)) = w;
    }
}

// read back one pass: lane j of quarter qd, columns 16 cg .. + 15 (rows
// i = 32 pass + 8 cg + c / 2, part c % 2) of every accumulator; returns the
// largest |R_ij| written
__device__ float res_readback(Tc128Work &wk, const Tc128Smem &sm, uint32_t tmem, int pass, int M)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qd = warp & 3, cg = warp >> 2, j = 32 * qd + lane;
    const uint32_t tb = tmem + ((uint32_t)(32 * qd) << 16) + 16 * cg;
    const int ce = sm.cexp[j];
    float rloc = 0.f;
    float out[16];
#pragma unroll
    for (int j8 = 0; j8 < 16; j8 += 8) {
        uint32_t v0[8], v1[8], v2[8], v3[8];
        float small[8];
        tmem_ld8(tb + 192 + j8, v0);
        tmem_ld8(tb + 256 + j8, v1);
        tmem_ld8(tb + 320 + j8, v2);
        tmem_ld8(tb + 384 + j8, v3);
        wait_ld();
#pragma unroll
        for (int x = 0; x < 8; ++x)
            small[x] = ((__uint_as_float(v3[x]) + __uint_as_float(v2[x])) + __uint_as_float(v1[x])) +
                       __uint_as_float(v0[x]);
        tmem_ld8(tb + j8, v0);
        tmem_ld8(tb + 64 + j8, v1);
        tmem_ld8(tb + 128 + j8, v2);
        wait_ld();
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int col = 16 * cg + j8 + x;        // accumulator column: row i' = col / 2, part col % 2
            const int i = 32 * pass + (col >> 1), part = col & 1;
            float hs, ls, t, te;
            two_sum(__uint_as_float(v0[x]), __uint_as_float(v1[x]), hs, ls);
            two_sum(hs, __uint_as_float(v2[x]), t, te);
            ls += te;
            two_sum(t, small[x], hs, te);
            ls += te;
            const float sc = pow2f(sm.rexp[i] + ce - 16);
            hs *= sc;
            ls *= sc;
            if (part == 0 && i == j) {
                two_sum(hs, 1.0f, t, te);
                hs = t;
                ls += te;
            }
            const float r = (i < M && j < M) ? hs + ls : 0.f;
            out[j8 + x] = r;
            rloc = fmaxf(rloc, fabsf(r));
        }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int i = 32 * pass + 8 * cg + c;
        wk.R[sidx(i, j)] = make_float2(out[2 * c], out[2 * c + 1]);
    }
    return rloc;
}

// ---------------------------------------------------------------------------
// F. the products D = X' S (refinement) and D = R S (further Neumann terms)
//    on the tensor cores: A rows i, K = 16 (c % 8) + kk in the real form
//    [Re | Im] (c < 8 | c >= 8), B^T rows 2j = [Re S | -Im S], 2j + 1 =
//    [Im S | Re S], three exact bf16 terms each, the six products of term
//    order <= 2 into one f32 accumulator (tensor-memory columns 0 .. 255).
//    The chunks of one K range (c and c + 8) use the same loaded values.

// values of S (and of R for a Neumann term) one work item per thread half:
// items e = tid, tid + NTH
struct ProdPre {
    float4 s[4];      // (k, j), (k + 1, j) of S for the thread's four B items
    float4 a[2];      // (i, k), (i, k + 1) of X' or R for the thread's two A items
};

// B item h of a thread (4 per thread, 2048 per chunk): tile row 2j + sub and
// K pair kp; a warp's 32 four-byte stores cover 8 consecutive tile rows
// (four columns j, both parities) x 4 K pairs = 128 contiguous bytes
KNIT_DEV void prod_b_item(int h, int &j, int &sub, int &kp)
{
    const int e = threadIdx.x + h * NTH, l = e & 31, w = e >> 5;   // w = 0 .. 63
    j = 4 * (w & 31) + (l >> 3);
    sub = (l >> 2) & 1;
    kp = (l & 3) + 4 * (w >> 5);
}

// A item h (2 per thread): tile row i, K pair kp; a warp covers 8 rows x 4
// K pairs (conflict-free), the two items the two K halves
KNIT_DEV void prod_a_item(int h, int &i, int &kp)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    i = 8 * w + (l >> 2);
    kp = (l & 3) + 4 * h;
}

KNIT_DEV ProdPre prod_load(const float2 *S, const float2 *R, const float4 *Xt, int c)
{
    const int k0 = 16 * (c & 7);
    ProdPre q;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        int j, sub, kp;
        prod_b_item(h, j, sub, kp);
        q.s[h] = *reinterpret_cast<const float4 *>(S + sidx(k0 + 2 * kp, j));
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int i, kp;
        prod_a_item(h, i, kp);
        const int k = k0 + 2 * kp;
        if (R) {
            const float2 r0 = R[sidx(i, k)], r1 = R[sidx(i, k + 1)];
            q.a[h] = make_float4(r0.x, r0.y, r1.x, r1.y);
        } else {
            q.a[h] = Xt[(k >> 1) * MP + i];
        }
    }
    return q;
}

// A tile from X' (digits, at the column scale of X'; the scale goes into B)
KNIT_DEV void prod_a_x(const ProdPre &q, const Tc128Smem &sm, unsigned char *a, int c)
{
    const int part = c >> 3, k0 = 16 * (c & 7);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int i, kp;
        prod_a_item(h, i, kp);
        const int kk = 2 * kp;
        float d0[NDX], d1[NDX];
        digits3(part ? q.a[h].y : q.a[h].x, pow2f(-sm.cexp[k0 + kk]), d0);
        digits3(part ? q.a[h].w : q.a[h].z, pow2f(-sm.cexp[k0 + kk + 1]), d1);
#pragma unroll
        for (int qq = 0; qq < NDX; ++qq) put_bf16x2(a + qq * A_TILE, i, kk, d0[qq], d1[qq]);
    }
}

// A tile from R (three exact bf16 terms of each fp32 value)
KNIT_DEV void prod_a_r(const ProdPre &q, unsigned char *a, int c)
{
    const int part = c >> 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int i, kp;
        prod_a_item(h, i, kp);
        const int kk = 2 * kp;
        const float v0 = part ? q.a[h].y : q.a[h].x;
        const float v1 = part ? q.a[h].w : q.a[h].z;
        uint32_t h0, m0, l0, h1, m1, l1;
        bf16_split3(v0, h0, m0, l0);
        bf16_split3(v1, h1, m1, l1);
        unsigned char *p = a + tile_off(i, kk);
        *reinterpret_cast<uint32_t *>(p) = pack_hi16(h0, h1);
        *reinterpret_cast<uint32_t *>(p + A_TILE) = pack_hi16(m0, m1);
        *reinterpret_cast<uint32_t *>(p + 2 * A_TILE) = pack_hi16(l0, l1);
    }
}

// B tile from S, scaled by 2^(t_k - 8) when A holds the X' digits:
// row 2j = [Re | -Im], row 2j + 1 = [Im | Re] of column j of S
KNIT_DEV void prod_b(const ProdPre &q, const Tc128Smem &sm, unsigned char *b, int c, bool scaled)
{
    const int part = c >> 3, k0 = 16 * (c & 7);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        int j, sub, kp;
        prod_b_item(h, j, sub, kp);
        const int kk = 2 * kp, k = k0 + kk;
        const float4 sv = q.s[h];
        const float u0 = scaled ? pow2f(sm.cexp[k] - 8) : 1.f;
        const float u1 = scaled ? pow2f(sm.cexp[k + 1] - 8) : 1.f;
        // (part, sub): (0, 0) Re, (0, 1) Im, (1, 0) -Im, (1, 1) Re
        const bool re = (part ^ sub) == 0;
        const float sg = (part == 1 && sub == 0) ? -1.f : 1.f;
        const float v0 = sg * (re ? sv.x : sv.y) * u0;
        const float v1 = sg * (re ? sv.z : sv.w) * u1;
        uint32_t h0, m0, l0, h1, m1, l1;
        bf16_split3(v0, h0, m0, l0);
        bf16_split3(v1, h1, m1, l1);
        unsigned char *p = b + tile_off(2 * j + sub, kk);
        *reinterpret_cast<uint32_t *>(p) = pack_hi16(h0, h1);
        *reinterpret_cast<uint32_t *>(p + BT_256) = pack_hi16(m0, m1);
        *reinterpret_cast<uint32_t *>(p + 2 * BT_256) = pack_hi16(l0, l1);
    }
}

// g = X' + D into the state: lane i of quarter qd, complex columns 32 cg ..
__device__ void ref_readback(Tc128Work &wk, uint32_t tmem, int M)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qd = warp & 3, cg = warp >> 2, i = 32 * qd + lane;
    const float2 *X = reinterpret_cast<const float2 *>(wk.Xt);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + 64 * cg + 32 * h, v);
        wait_ld();
#pragma unroll
        for (int cp = 0; cp < 8; ++cp) {
            float2 oh[2], ol[2];
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const int c = 2 * cp + s2, j = 32 * cg + 16 * h + c;
                const float2 x = X[((j >> 1) * MP + i) * 2 + (j & 1)];
                if (i < M && j < M) {
                    two_sum(x.x, __uint_as_float(v[2 * c]), oh[s2].x, ol[s2].x);
                    two_sum(x.y, __uint_as_float(v[2 * c + 1]), oh[s2].y, ol[s2].y);
                } else {
                    oh[s2] = make_float2(i == j ? 1.f : 0.f, 0.f);
                    ol[s2] = make_float2(0.f, 0.f);
                }
            }
            const int jp = 16 * cg + 8 * h + cp;
            wk.Gh[jp * MP + i] = make_float4(oh[0].x, oh[0].y, oh[1].x, oh[1].y);
            wk.Gl[jp * MP + i] = make_float4(ol[0].x, ol[0].y, ol[1].x, ol[1].y);
        }
    }
}

// a further Neumann term: So = R + D (zero outside M x M)
__device__ void neumann_readback(const float2 *R, float2 *So, uint32_t tmem, int M)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qd = warp & 3, cg = warp >> 2, i = 32 * qd + lane;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + 64 * cg + 32 * h, v);
        wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int j = 32 * cg + 16 * h + c;
            float2 o = make_float2(0.f, 0.f);
            if (i < M && j < M) {
                const float2 r = R[sidx(i, j)];
                o = make_float2(r.x + __uint_as_float(v[2 * c]), r.y + __uint_as_float(v[2 * c + 1]));
            }
            So[sidx(i, j)] = o;
        }
    }
}

// D = A S on the tensor cores with A = X' (R null) or A = R; double-buffered
// over the two chunk slots; every thread polls the slot's barrier before it
// rewrites the slot, and the next K range's loads are issued a chunk ahead.
// Returns false when a wait ran out (the commits in flight stay recorded).
__device__ __noinline__ bool product_tc(Tc128Smem &sm, Bars &br, uint32_t tmem, const float2 *S,
                           const float2 *R, const float4 *Xt, int nchunk)
{
    const int nseq = 2 * nchunk;
    ProdPre cur = prod_load(S, R, Xt, 0), nxt = cur;
    for (int sq = 0; sq < nseq; ++sq) {
        const int slot = sq & 1, c = (sq >> 1) + 8 * (sq & 1);
        const int ok = sq >= 2 ? mbar_wait(&sm.bar[2 + slot], br.ph[2 + slot]) : 1;
        if ((sq & 1) == 0 && sq + 2 < nseq) nxt = prod_load(S, R, Xt, (sq >> 1) + 1);
        unsigned char *const a = sm.u.ref.a[slot];
        unsigned char *const b = sm.u.ref.b[slot];
        if (R) prod_a_r(cur, a, c);
        else prod_a_x(cur, sm, a, c);
        prod_b(cur, sm, b, c, R == nullptr);
        async_proxy_fence();
        fence_before();
        if (__syncthreads_or(!ok)) return false;
        if (sq >= 2) {
            br.ph[2 + slot] ^= 1u;
            br.pend[2 + slot] = 0u;
        }
        if (threadIdx.x == 0) {
            fence_after();
#pragma unroll
            for (int pr = 0; pr < 6; ++pr) {
                const uint64_t ad = smem_desc(smem_u32(a + kProdP[pr] * A_TILE));
                const uint64_t bd = smem_desc(smem_u32(b + kProdQ[pr] * BT_256));
                mma_bf16(tmem, ad, bd, idesc_bf16_m128(256), (sq == 0 && pr == 0) ? 0u : 1u);
            }
            mma_commit(&sm.bar[2 + slot]);
        }
        br.pend[2 + slot] = 1u;
        if (sq & 1) cur = nxt;
    }
    return bar_wait(sm, br, 2) && bar_wait(sm, br, 3);
}

// ---------------------------------------------------------------------------
// E. the rare paths on the CUDA cores (workspace operands)

// g = X' + X' S with X' S accumulated error-free (TwoProduct + TwoSum)
__device__ void refine_exact128(Tc128Work &wk, const float2 *S, int M)
{
    const float2 *X = reinterpret_cast<const float2 *>(wk.Xt);
    float2 *const gh = reinterpret_cast<float2 *>(wk.Gh);
    float2 *const gl = reinterpret_cast<float2 *>(wk.Gl);
    for (int e = threadIdx.x; e < MP * MP; e += NTH) {
        const int i = e & (MP - 1), j = e >> 7;
        const int f = ((j >> 1) * MP + i) * 2 + (j & 1);
        if (i >= M || j >= M) {
            gh[f] = make_float2(i == j ? 1.f : 0.f, 0.f);
            gl[f] = make_float2(0.f, 0.f);
            continue;
        }
        float2 sh = make_float2(0.f, 0.f), se = make_float2(0.f, 0.f);
        for (int k = 0; k < M; ++k) {
            const float2 xa = X[((k >> 1) * MP + i) * 2 + (k & 1)], sb = S[sidx(k, j)];
            dot2_acc1(xa.x, sb.x, sh.x, se.x);
            dot2_acc1(-xa.y, sb.y, sh.x, se.x);
            dot2_acc1(xa.x, sb.y, sh.y, se.y);
            dot2_acc1(xa.y, sb.x, sh.y, se.y);
        }
        const float2 xv = X[((j >> 1) * MP + i) * 2 + (j & 1)];
        float hx, lx, hy, ly;
        two_sum(xv.x, sh.x, hx, lx);
        lx += se.x;
        two_sum(hx, lx, hx, lx);
        two_sum(xv.y, sh.y, hy, ly);
        ly += se.y;
        two_sum(hy, ly, hy, ly);
        gh[f] = make_float2(hx, hy);
        gl[f] = make_float2(lx, ly);
    }
}

// near-singular A_n: this slice in FP64 from Gv' (still in the state)
__device__ int fallback64(Tc128Work &wk, int M)
{
    const float2 *gh = reinterpret_cast<const float2 *>(wk.Gh);
    const float2 *gl = reinterpret_cast<const float2 *>(wk.Gl);
    for (int e = threadIdx.x; e < M * M; e += NTH) {
        const int i = e / M, j = e - i * M;
        const int f = ((j >> 1) * MP + i) * 2 + (j & 1);
        wk.A64[e] = make_double2(-((double)gh[f].x + (double)gl[f].x), -((double)gh[f].y + (double)gl[f].y));
    }
    __syncthreads();
    const int st = gj_invert64(wk.A64, M, fallback_scratch(wk.scr, M));
    if (st != ST_OK) return st;
    float2 *const oh = reinterpret_cast<float2 *>(wk.Gh);
    float2 *const ol = reinterpret_cast<float2 *>(wk.Gl);
    for (int e = threadIdx.x; e < MP * MP; e += NTH) {
        const int i = e & (MP - 1), j = e >> 7;
        const int f = ((j >> 1) * MP + i) * 2 + (j & 1);
        float2 h, l;
        if (i < M && j < M) {
            const double2 v = wk.A64[i * M + j];
            to_df(v.x, h.x, l.x);
            to_df(v.y, h.y, l.y);
        } else {
            h = make_float2(i == j ? 1.f : 0.f, 0.f);
            l = make_float2(0.f, 0.f);
        }
        oh[f] = h;
        ol[f] = l;
    }
    __syncthreads();
    return ST_OK;
}

// near-singular A_n: this slice inverted in double-float on the CUDA cores
// (entries as (hi, lo) float pairs, ~2^-46 relative per operation), from
// Gv' in the state.  The in-place Gauss-Jordan elimination with implicit
// partial pivoting and deferred panel updates of the width-64 kernel
// (gj_blocked in mixed_common.cuh), in double-float: per panel of 8 columns
// four warps (one row per thread) take the pivot steps on the panel columns
// in registers and keep u = column - e_p; one thread per column forms the v
// vectors by forward substitution from the pivot rows at the start of the
// panel; then every thread applies X -= U V to its elements.  With p_k the
// pivot row of step k, the inverse is g[r][c] = X[p_r][q_c] for q the
// inverse permutation.  X's hi parts live in shared memory, the lo parts in
// the workspace.
__device__ __noinline__ int fallback_df(Tc128Work &wk, Tc128Smem &sm, int M)
{
    constexpr int NBK = 8;
    float2 *const ah = sm.u.fb.hi;                               // row-major MP x MP
    float2 *const al = reinterpret_cast<float2 *>(wk.A64);       // same layout
    const float2 *gh = reinterpret_cast<const float2 *>(wk.Gh);
    const float2 *gl = reinterpret_cast<const float2 *>(wk.Gl);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < MP * MP; e += NTH) {
        const int i = e >> 7, j = e & (MP - 1);
        float2 h = make_float2(0.f, 0.f), l = h;
        if (i < M && j < M) {
            const int f = ((j >> 1) * MP + i) * 2 + (j & 1);
            h = make_float2(-gh[f].x, -gh[f].y);
            l = make_float2(-gl[f].x, -gl[f].y);
        }
        ah[e] = h;
        al[e] = l;
    }
    if (tid == 0) sm.flag = 0;
    __syncthreads();
    bool open = tid < M;   // threads 0 .. 127: row tid may still become a pivot row
    for (int K = 0; K < M; K += NBK) {
        const int nk = min(NBK, M - K);
        // ---- the pivot steps on the panel columns, one row per thread
        if (tid < MP) {
            float4 pc[NBK];
#pragma unroll
            for (int c = 0; c < NBK; ++c) {
                const int e = tid * MP + K + c;
                pc[c] = K + c < M ? make_float4(ah[e].x, ah[e].y, al[e].x, al[e].y)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int kk = 0; kk < NBK; ++kk) {
                if (kk < nk) {
                    float v = open ? fabsf(pc[kk].x) + fabsf(pc[kk].y) : -1.f;
                    int bi = tid;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
                        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                        if (ov > v || (ov == v && oi < bi)) {
                            v = ov;
                            bi = oi;
                        }
                    }
                    if (lane == 0) {
                        sm.u.fb.key[warp] = v;
                        sm.u.fb.idx[warp] = bi;
                    }
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    float bv = sm.u.fb.key[0];
                    int p = sm.u.fb.idx[0];
#pragma unroll
                    for (int w = 1; w < 4; ++w)
                        if (sm.u.fb.key[w] > bv) {
                            bv = sm.u.fb.key[w];
                            p = sm.u.fb.idx[w];
                        }
                    const bool ok = bv > 0.f && isfinite(bv);
                    if (!ok) p = 0;
                    if (tid == p) {
                        if (!ok) sm.flag = 1;
                        sm.perm[K + kk] = p;
#pragma unroll
                        for (int c = 0; c < NBK; ++c) sm.u.fb.prow[c] = pc[c];
                        const double pr = (double)pc[kk].x + (double)pc[kk].z;
                        const double pi = (double)pc[kk].y + (double)pc[kk].w;
                        const double d = 1.0 / (pr * pr + pi * pi);
                        float4 ri;
                        to_df(pr * d, ri.x, ri.z);
                        to_df(-pi * d, ri.y, ri.w);
                        sm.u.fb.rinv[kk] = ri;
                    }
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    const float4 ri = sm.u.fb.rinv[kk];
                    const float4 u = tid == p ? df4_add_real(pc[kk], -1.f) : pc[kk];
                    sm.u.fb.U[tid * NBK + kk] = u;
#pragma unroll
                    for (int c = kk + 1; c < NBK; ++c)
                        pc[c] = df4_fms(pc[c], u, df4_mul(sm.u.fb.prow[c], ri));
                    open = open && tid != p;
                } else {
                    sm.u.fb.U[tid * NBK + kk] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
        __syncthreads();
        if (sm.flag) return ST_SINGULAR;
        // ---- v vectors: one thread per column j, forward substitution from the
        // pivot rows of X at the start of the panel
        if (tid < MP) {
            const int j = tid;
            float4 v[NBK];
#pragma unroll
            for (int kk = 0; kk < NBK; ++kk) {
                v[kk] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (kk < nk && j < M) {
                    const int p = sm.perm[K + kk];
                    float4 r = make_float4(ah[p * MP + j].x, ah[p * MP + j].y, al[p * MP + j].x,
                                           al[p * MP + j].y);
                    if (j == K + kk) r = df4_add_real(r, 1.f);
#pragma unroll
                    for (int c = 0; c < kk; ++c) r = df4_fms(r, sm.u.fb.U[p * NBK + c], v[c]);
                    v[kk] = df4_mul(r, sm.u.fb.rinv[kk]);
                }
            }
#pragma unroll
            for (int kk = 0; kk < NBK; ++kk) sm.u.fb.V[kk * MP + j] = v[kk];
        }
        __syncthreads();
        // ---- X -= U V over the whole matrix (lo parts loaded eight at a time)
        constexpr int FB = 8;
#pragma unroll 1
        for (int e0 = tid; e0 < MP * MP; e0 += FB * NTH) {
            float2 lb[FB];
#pragma unroll
            for (int b = 0; b < FB; ++b) lb[b] = al[e0 + b * NTH];
#pragma unroll
            for (int b = 0; b < FB; ++b) {
                const int e = e0 + b * NTH, i = e >> 7, j = e & (MP - 1);
                float4 x = make_float4(ah[e].x, ah[e].y, lb[b].x, lb[b].y);
#pragma unroll
                for (int c = 0; c < NBK; ++c)
                    if (c < nk) x = df4_fms(x, sm.u.fb.U[i * NBK + c], sm.u.fb.V[c * MP + j]);
                if (i < M && j < M) {
                    ah[e] = make_float2(x.x, x.y);
                    al[e] = make_float2(x.z, x.w);
                }
            }
        }
        __syncthreads();
    }
    // g[r][c] = X[p_r][q_c], q the inverse of the pivot permutation
    for (int j = tid; j < M; j += NTH) sm.u.fb.pinv[sm.perm[j]] = j;
    __syncthreads();
    float2 *const oh = reinterpret_cast<float2 *>(wk.Gh);
    float2 *const ol = reinterpret_cast<float2 *>(wk.Gl);
    for (int e = tid; e < MP * MP; e += NTH) {
        const int r = e & (MP - 1), c = e >> 7;
        const int f = ((c >> 1) * MP + r) * 2 + (c & 1);
        if (r < M && c < M) {
            const int src = sm.perm[r] * MP + sm.u.fb.pinv[c];
            oh[f] = ah[src];
            ol[f] = al[src];
        } else {
            oh[f] = make_float2(r == c ? 1.f : 0.f, 0.f);
            ol[f] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    return ST_OK;
}

// T from G_LL = Gh + Gl by the unitarity identity (as ward_T of
// mixed_common.cuh), in double-float on the CUDA cores (GB300's FP64 rate
// is 1/72 of its FP32 rate; an FP64 trace would cost as much as ~20 slices):
//   T = Re Tr[Gamma_R i(G - G^dagger)] - Re sum_ij (Gamma_R G)_ij conj((G Gamma_R)_ij)
// with (G Gamma G^dagger)'s trace written through the Hermitian Gamma_R =
// i(Sigma_R - Sigma_R^dagger), formed here in double-float (row-major hi / lo
// in the workspace buffers R and S1).  Per-thread partial sums in FP64.
__device__ double ward_T128(Tc128Work &wk, const double2 *SR, int M, double *red)
{
    float2 *const gmh = wk.R, *const gml = wk.S1;   // Gamma_R, row-major MP x MP
    const float2 *gh = reinterpret_cast<const float2 *>(wk.Gh);
    const float2 *gl = reinterpret_cast<const float2 *>(wk.Gl);
    for (int e = threadIdx.x; e < MP * MP; e += NTH) {
        const int i = e >> 7, k = e & (MP - 1);
        float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
        if (i < M && k < M) {
            const double2 a = SR[(size_t)i * M + k], b = SR[(size_t)k * M + i];
            // i (a - conj(b))
            to_df(-(a.y + b.y), h.x, l.x);
            to_df(a.x - b.x, h.y, l.y);
        }
        gmh[e] = h;
        gml[e] = l;
    }
    __syncthreads();
    double t = 0.0;
    // Re Tr[Gamma i(G - G^dagger)] = Re sum_ij Gamma_ij i (G_ji - conj(G_ij))
    for (int e = threadIdx.x; e < M * M; e += NTH) {
        const int i = e / M, j = e - i * M;
        const int fji = ((i >> 1) * MP + j) * 2 + (i & 1), fij = ((j >> 1) * MP + i) * 2 + (j & 1);
        const double gjr = (double)gh[fji].x + gl[fji].x, gji = (double)gh[fji].y + gl[fji].y;
        const double gir = (double)gh[fij].x + gl[fij].x, gii = (double)gh[fij].y + gl[fij].y;
        // a = i (G_ji - conj(G_ij)) = i ((gjr - gir) + i (gji + gii))
        const double ar = -(gji + gii), ai = gjr - gir;
        const double cr = (double)gmh[i * MP + j].x + gml[i * MP + j].x;
        const double ci = (double)gmh[i * MP + j].y + gml[i * MP + j].y;
        t += cr * ar - ci * ai;
    }
    // sum_ij (Gamma G)_ij conj((G Gamma)_ij): item (row i, column pair jp),
    // lanes along jp (coalesced rows of G and Gamma, broadcast row i)
    for (int e = threadIdx.x; e < MP * (MP / 2); e += NTH) {
        const int i = e >> 6, jp = e & 63;
        if (i >= M || 2 * jp >= M) continue;
        float2 yh[2] = {}, yl[2] = {}, zh[2] = {}, zl[2] = {};
        for (int k = 0; k < M; ++k) {
            const float2 gik_h = gh[((k >> 1) * MP + i) * 2 + (k & 1)];
            const float2 gik_l = gl[((k >> 1) * MP + i) * 2 + (k & 1)];
            const float2 cik_h = gmh[i * MP + k], cik_l = gml[i * MP + k];
            const float4 gkh = wk.Gh[jp * MP + k], gkl = wk.Gl[jp * MP + k];            // G[k][2jp], G[k][2jp + 1]
            const float4 ckh = *reinterpret_cast<const float4 *>(gmh + k * MP + 2 * jp);  // Gamma[k][2jp ..]
            const float4 ckl = *reinterpret_cast<const float4 *>(gml + k * MP + 2 * jp);
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const float2 gkj_h = s2 ? make_float2(gkh.z, gkh.w) : make_float2(gkh.x, gkh.y);
                const float2 gkj_l = s2 ? make_float2(gkl.z, gkl.w) : make_float2(gkl.x, gkl.y);
                const float2 ckj_h = s2 ? make_float2(ckh.z, ckh.w) : make_float2(ckh.x, ckh.y);
                const float2 ckj_l = s2 ? make_float2(ckl.z, ckl.w) : make_float2(ckl.x, ckl.y);
                float2 ph, pl;
                cdf_mul(cik_h, cik_l, gkj_h, gkj_l, ph, pl);   // Gamma_ik G_kj
                cdf_add(yh[s2], yl[s2], ph, pl);
                cdf_mul(gik_h, gik_l, ckj_h, ckj_l, ph, pl);   // G_ik Gamma_kj
                cdf_add(zh[s2], zl[s2], ph, pl);
            }
        }
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            if (2 * jp + s2 >= M) continue;
            const double yr = (double)yh[s2].x + yl[s2].x, yi = (double)yh[s2].y + yl[s2].y;
            const double zr = (double)zh[s2].x + zl[s2].x, zi = (double)zh[s2].y + zl[s2].y;
            t -= yr * zr + yi * zi;
        }
    }
    return block_sum(t, red);
}

}  // namespace

__global__ void __launch_bounds__(NTH, 1)
knit_sweep_mixed_tc128_kernel(InstDev in, Tc128Work *work)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Tc128Smem &sm = *reinterpret_cast<Tc128Smem *>(smem_raw);
    Tc128Work &wk = work[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&sm.tmem)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        sm.cur_sys = -1;
        for (int b = 0; b < 4; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.bar[b])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sm.tmem;
    Bars br = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
    bool timed_out = false;

    for (;;) {
        if (tid == 0) {
            const int qn = atomicAdd(in.queue, 1);
            sm.inst = qn < in.n ? take_position(in, qn) : -1;
        }
        __syncthreads();
        const int inst = sm.inst;
        const int si = inst >= 0 && in.sys_of ? in.sys_of[inst] : 0;
        const bool reload = inst >= 0 && si != sm.cur_sys;
        __syncthreads();
        if (inst < 0) break;
        const SysDev s = in.sys[si];
        const int M = s.M, L = s.L, vb = s.vb;
        const size_t MM = (size_t)M * M;
        if (reload) {
            // the kind of each coupling: diagonal (scalar when uniform), 4 x 4
            // blocks, or tridiagonal (the host admits nothing else); every
            // thread that sees an off-diagonal entry writes the same kind
            if (tid < 4) sm.vkind[tid] = 0;
            __syncthreads();
            if (vb != 1)
                for (int q = 0; q < s.Vperiod; ++q)
                    for (int e = tid; e < M * M; e += NTH) {
                        const double2 v = s.V[(size_t)q * MM + e];
                        if (e / M != e % M && (v.x != 0.0 || v.y != 0.0)) sm.vkind[q] = vb == 4 ? 1 : 2;
                    }
            __syncthreads();
            if (tid < s.Vperiod) {
                sm.vuni[tid] = 1;
                if (sm.vkind[tid] == 0)
                    classify_vdiag(s.V + (size_t)tid * MM, M + 1, M, sm.vuni[tid], sm.vch[tid], sm.vcl[tid]);
            }
            if (tid == 0) sm.cur_sys = si;
            __syncthreads();
        }
        const InstParams ip = inst_params(in, inst, M);
        int st = ip.st;
        int dfrun = 0;   // consecutive slices that needed the double-float inversion

        for (int n = 0; n < L && st == ST_OK; ++n) {
            // ---- A
            slice_diag<MP, NTH>(sm.eps, s, ip.ms, ip.W, ip.E, n);
            for (int i = tid; i < MP; i += NTH) sm.rmaxu[i] = 0u;
            const int q = n % s.Vperiod, vk = sm.vkind[q];
            if (vk == 1 && n > 0) gv_blocks4(wk, sm, s, M, q);
            if (vk == 2 && n > 0) gv_tridiag(wk, sm, s, M, q);
            __syncthreads();   // eps (and the block passes' output) complete
            const int vmode = vk != 0 ? 1 : (sm.vuni[q] == 1 ? 1 : (sm.vuni[q] == 2 ? 2 : 0));
            gv_elementwise(wk, sm, s, M, n, L, vmode, vk == 1 && n > 0, ip.SL, ip.SR);
            __syncthreads();
            if (dfrun > 0 && (dfrun & 7) != 0) {
                // the slice before needed the double-float inversion; this one,
                // next to the same resonance, goes there directly (every eighth
                // slice of such a run tries the complex64 path again)
                st = fallback_df(wk, sm, M);
                if (st != ST_OK) st = fallback64(wk, M);
                ++dfrun;
                __syncthreads();
                continue;
            }
            fence_after();
            x_to_tmem(wk, sm, tmem, M);
            fence_before();
            __syncthreads();
            fence_after();
            // ---- B
            st = gj_tmem(sm, tmem, M, br);
            if (st != ST_OK) {
                timed_out = st == ST_TIMEOUT;
                break;
            }
            // ---- C
            x_prime_from_tmem(sm, wk, tmem, M);
            // ---- D
            float rloc = 0.f;
            const int nchunk = (M + 15) / 16;          // K-chunks per part
            const int npass = (M + 31) / 32;
            for (int pass = 0; pass < npass && !timed_out; ++pass) {
                const int nseq = 2 * nchunk;
                GvPre cur = res_b_load(wk, sm, pass, 0), nxt = cur;
                for (int sq = 0; sq < nseq; ++sq) {
                    const int slot = sq & 1;
                    const int c = (sq >> 1) + 8 * (sq & 1);
                    // every thread waits for the MMAs that last read this slot
                    const int ok = sq >= 2 ? mbar_wait(&sm.bar[2 + slot], br.ph[2 + slot]) : 1;
                    if ((sq & 1) == 0 && sq + 2 < nseq) nxt = res_b_load(wk, sm, pass, (sq >> 1) + 1);
                    const unsigned char *const a = sm.u.res.lres[c];
                    unsigned char *const b = sm.u.res.b[slot];
                    if ((sq & 1) == 0) res_b_build(cur, sm, b, pass);
                    else res_b_swap(sm.u.res.b[slot ^ 1], b);
                    async_proxy_fence();
                    fence_before();
                    if (__syncthreads_or(!ok)) { timed_out = true; break; }
                    if (sq >= 2) {
                        br.ph[2 + slot] ^= 1u;
                        br.pend[2 + slot] = 0u;
                    }
                    if (tid == 0) {
                        fence_after();
                        const uint64_t bd0 = smem_desc(smem_u32(b));
                        const uint64_t bd4 = smem_desc(smem_u32(b + 4 * BT_RES));
#pragma unroll
                        for (int qd = 0; qd < NDX; ++qd) {
                            const uint64_t ad = smem_desc(smem_u32(a + qd * A_TILE));
                            const uint32_t first = (sq == 0 && qd == 0) ? 0u : 1u;
                            // B digits p = 0 .. 3 side by side (N = 256) at accumulator qd,
                            // then p = 4 .. 6 - qd (N = 64 (3 - qd)) at accumulator qd + 4
                            mma_bf16(tmem + 64 * qd, ad, bd0, idesc_bf16_m128(256), first);
                            mma_bf16(tmem + 64 * (qd + 4), ad, bd4,
                                     idesc_bf16_m128((uint32_t)(64 * (3 - qd))), first);
                        }
                        mma_commit(&sm.bar[2 + slot]);
                    }
                    br.pend[2 + slot] = 1u;
                    if (sq & 1) cur = nxt;
                }
                if (timed_out) break;
                // both slots' last commits
                if (!bar_wait(sm, br, 2) || !bar_wait(sm, br, 3)) { timed_out = true; break; }
                fence_after();
                rloc = fmaxf(rloc, res_readback(wk, sm, tmem, pass, M));
                fence_before();
                __syncthreads();
            }
            if (timed_out) {
                st = ST_TIMEOUT;
                break;
            }
            // zero R in the rows no pass wrote (M < 128)
            for (int e = tid; e < MP * MP; e += NTH) {
                const int i = e >> 7, j = e & (MP - 1);
                if (i >= 32 * npass) wk.R[sidx(i, j)] = make_float2(0.f, 0.f);
            }
            // ---- E
            const float rmax = block_max_nonneg<NTH>(rloc, sm.redu);
            if (refinement_fails(rmax, M)) {
                // double-float Gauss-Jordan; FP64 if it meets an exact zero pivot
                st = fallback_df(wk, sm, M);
                if (st != ST_OK) st = fallback64(wk, M);
                ++dfrun;
                __syncthreads();
                continue;
            }
            dfrun = 0;
            const int nx = neumann_terms(rmax, M);
            const float2 *S = wk.R;
            for (int t = 0; t < nx && !timed_out; ++t) {
                // S <- R + R S on the tensor cores
                float2 *const So = (t & 1) ? wk.S2 : wk.S1;
                if (!product_tc(sm, br, tmem, S, wk.R, wk.Xt, nchunk)) { timed_out = true; break; }
                fence_after();
                neumann_readback(wk.R, So, tmem, M);
                fence_before();
                __syncthreads();
                S = So;
            }
            if (timed_out) {
                st = ST_TIMEOUT;
                break;
            }
            if (rmax > EXACT_RMAX) {
                refine_exact128(wk, S, M);
                __syncthreads();
                continue;
            }
            // ---- F
            if (!product_tc(sm, br, tmem, S, nullptr, wk.Xt, nchunk)) {
                timed_out = true;
                st = ST_TIMEOUT;
                break;
            }
            fence_after();
            ref_readback(wk, tmem, M);
            fence_before();
            __syncthreads();
        }

        double T = 0.0;
        if (st == ST_OK) {
            T = ward_T128(wk, ip.SR, M, sm.red);
            if (in.GLL) {
                // G_LL in FP64 for the eigenvalue stage
                const float2 *gh = reinterpret_cast<const float2 *>(wk.Gh);
                const float2 *gl = reinterpret_cast<const float2 *>(wk.Gl);
                double2 *const dst = in.GLL + (size_t)ip.out * M * M;
                for (int e = tid; e < M * M; e += NTH) {
                    const int i = e / M, j = e - i * M;
                    const int f = ((j >> 1) * MP + i) * 2 + (j & 1);
                    dst[e] = make_double2((double)gh[f].x + gl[f].x, (double)gh[f].y + gl[f].y);
                }
            }
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
        // a wait ran out: every barrier with a commit still in flight gets a
        // second bounded wait before the tensor memory is released
        if (tid == 0)
            for (int b = 0; b < 4; ++b)
                if (br.pend[b]) mbar_wait(&sm.bar[b], br.ph[b]);
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

extern "C" size_t knit_mixed_tc128_work_bytes(void) { return sizeof(Tc128Work); }
extern "C" size_t knit_mixed_tc128_smem_bytes(void) { return sizeof(Tc128Smem); }

// Host launch helper.  Instances that a timed-out CTA never reaches keep the
// ST_TIMEOUT status written here first.
extern "C" cudaError_t knit_launch_mixed_tc128(const InstDev *in, int grid, void *work,
                                               cudaStream_t stream)
{
    static_assert(sizeof(Tc128Smem) <= 227 * 1024, "shared memory budget");
    if (in->status && !in->out_index)
        fill_status128<<<(in->n + 255) / 256, 256, 0, stream>>>(in->status, in->n, ST_TIMEOUT);
    const size_t smb = sizeof(Tc128Smem);
    cudaError_t e = cudaFuncSetAttribute(knit_sweep_mixed_tc128_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    if (e != cudaSuccess) return e;
    knit_sweep_mixed_tc128_kernel<<<grid, NTH, smb, stream>>>(*in, (Tc128Work *)work);
    return cudaGetLastError();
}
