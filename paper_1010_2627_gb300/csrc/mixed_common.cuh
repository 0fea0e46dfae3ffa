// mixed_common.cuh -- pieces shared by the two mixed-precision sweep kernels
// (sweep_mixed.cu: double-float residual on CUDA cores; sweep_mixed_tc.cu:
// residual on the tcgen05 tensor cores).  One CTA of 256 threads works on a
// padded MP x MP complex matrix; thread (ty, tx) = (tid / 16, tid % 16) owns
// rows ty + 16a and columns tx + 16b (a, b < MP / 16).
#pragma once

#include "knit_common.cuh"

namespace mixed {

constexpr int NT = 256;

KNIT_DEV void to_df(double d, float &h, float &l)
{
    h = __double2float_rn(d);
    l = __double2float_rn(d - (double)h);
}

// (ah + al) * (bh + bl) for real double-floats -> (p, e) unnormalised
KNIT_DEV void df_mul(float ah, float al, float bh, float bl, float &p, float &e)
{
    p = ah * bh;
    e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
}

// complex double-float product
KNIT_DEV void cdf_mul(float2 ah, float2 al, float2 bh, float2 bl, float2 &rh, float2 &rl)
{
    float p1, e1, p2, e2, s, t;
    df_mul(ah.x, al.x, bh.x, bl.x, p1, e1);
    df_mul(ah.y, al.y, bh.y, bl.y, p2, e2);
    two_sum(p1, -p2, s, t);
    t += e1 - e2;
    two_sum(s, t, rh.x, rl.x);
    df_mul(ah.x, al.x, bh.y, bl.y, p1, e1);
    df_mul(ah.y, al.y, bh.x, bl.x, p2, e2);
    two_sum(p1, p2, s, t);
    t += e1 + e2;
    two_sum(s, t, rh.y, rl.y);
}

KNIT_DEV void cdf_add(float2 &h, float2 &l, float2 bh, float2 bl)
{
    float s, t;
    two_sum(h.x, bh.x, s, t);
    t += l.x + bl.x;
    two_sum(s, t, h.x, l.x);
    two_sum(h.y, bh.y, s, t);
    t += l.y + bl.y;
    two_sum(s, t, h.y, l.y);
}

template <int MP>
struct GJShared {
    float2 col[2][MP];
    float2 rowp[2][MP];
    float val[2][MP];
    int used[MP];
    int perm[MP];
    int pos[MP];
    int flag;
};

// E - onsite of slice n for orbitals 0..MP-1 (0 in the padding)
template <int MP, int NTH = NT>
__device__ void slice_diag(double *eps, const SysDev &s, uint64_t ms, double W, double E, int n)
{
    for (int i = threadIdx.x; i < MP; i += NTH) {
        double d = 0.0;
        if (i < s.M) {
            double o = 0.0;
            if (s.onsite) o = s.onsite[(size_t)n * s.M + i];
            else if (W != 0.0) o = s.sign[i % s.block] * knit_disorder(ms, n, i / s.block, W);
            d = E - o;
        }
        eps[i] = d;
    }
}

// Gv = V_n g V_n^dagger (+ Sigma_L at n = 0, + Sigma_R at n = L - 1) in
// double-float, in place over (Gh, Gl); vh/vl: diagonal of V per parity.
template <int MP, int NTH = NT>
__device__ void form_gv(float2 *Gh, float2 *Gl, const float2 (*vh)[MP], const float2 (*vl)[MP],
                        int M, int n, int L, const double2 *SL, const double2 *SR)
{
    const int q = n & 1;
    for (int e = threadIdx.x; e < MP * MP; e += NTH) {
        const int i = e / MP, j = e - i * MP;
        float2 gh = make_float2(0.f, 0.f), gl = make_float2(0.f, 0.f);
        if (i < M && j < M) {
            if (n > 0) {
                float2 th, tl;
                float2 vjh = vh[q][j], vjl = vl[q][j];
                vjh.y = -vjh.y;
                vjl.y = -vjl.y;
                cdf_mul(Gh[e], Gl[e], vjh, vjl, th, tl);
                cdf_mul(vh[q][i], vl[q][i], th, tl, gh, gl);
            } else {
                double2 v = SL[(size_t)i * M + j];
                float a, b, c, d;
                to_df(v.x, a, b);
                to_df(v.y, c, d);
                gh = make_float2(a, c);
                gl = make_float2(b, d);
            }
            if (n == L - 1) {
                double2 v = SR[(size_t)i * M + j];
                float a, b, c, d;
                to_df(v.x, a, b);
                to_df(v.y, c, d);
                cdf_add(gh, gl, make_float2(a, c), make_float2(b, d));
            }
        }
        Gh[e] = gh;
        Gl[e] = gl;
    }
}

// Gauss-Jordan inversion of the register tile x (M x M inside MP x MP) with
// implicit partial pivoting: no rows are moved; the pivot of column k is the
// largest |Re|+|Im| among rows not yet used (lowest row on ties).  Column k
// and the pivot row are zeroed in registers after staging, so every element
// then takes the same update x -= c_i r_j (c_p = -1, r_k = 1/pivot).  On
// return A^{-1}[k][P[k']] = x[P[k]][k'], P[k] = g.perm[k].  Returns ST_OK or
// ST_SINGULAR (uniform over the block).
template <int MP, int TY = 16, int TX = 16>
__device__ __forceinline__ int gj_regs(float2 (&x)[MP / TY][MP / TX], int M, GJShared<MP> &g)
{
    constexpr int RA = MP / TY, RB = MP / TX, NTH = TY * TX;
    const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX, lane = tid & 31;
    int st = ST_OK;
    for (int i = tid; i < MP; i += NTH) g.used[i] = 0;
    __syncthreads();
    for (int k = 0; k < M; ++k) {
        const int q = k & 1, kt = k % TX, kb = k / TX;
        if (tx == kt) {
#pragma unroll
            for (int a = 0; a < RA; ++a) {
                float2 v = x[a][0];
#pragma unroll
                for (int b = 1; b < RB; ++b)
                    if (b == kb) v = x[a][b];
#pragma unroll
                for (int b = 0; b < RB; ++b)
                    if (b == kb) x[a][b] = make_float2(0.f, 0.f);
                const int i = ty + TY * a;
                g.col[q][i] = v;
                g.val[q][i] = (i < M && !g.used[i]) ? cabs1f(v) : -1.f;
            }
        }
        __syncthreads();
        float best = -1.f;
        int p = MP;
        for (int i = lane; i < MP; i += 32) {
            float v = g.val[q][i];
            if (v > best) { best = v; p = i; }
        }
        warp_argmaxf(best, p);
        if (best <= 0.f) {
            st = ST_SINGULAR;
            break;
        }
        if (ty == p % TY) {
            const int pa = p / TY;
#pragma unroll
            for (int a = 0; a < RA; ++a) {
                if (a != pa) continue;
#pragma unroll
                for (int b = 0; b < RB; ++b) {
                    g.rowp[q][tx + TX * b] = x[a][b];
                    x[a][b] = make_float2(0.f, 0.f);
                }
            }
        }
        if (tid == 0) {
            g.perm[k] = p;
            g.used[p] = 1;
        }
        __syncthreads();
        const float2 pinv = crcpf(g.col[q][p]);
        float2 rs[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int j = tx + TX * b;
            rs[b] = (j == k) ? pinv : cmulf(g.rowp[q][j], pinv);
        }
#pragma unroll
        for (int a = 0; a < RA; ++a) {
            const int i = ty + TY * a;
            const float2 ci = (i == p) ? make_float2(-1.f, 0.f) : g.col[q][i];
#pragma unroll
            for (int b = 0; b < RB; ++b) x[a][b] = cfmsf(ci, rs[b], x[a][b]);
        }
    }
    if (__syncthreads_or(st != ST_OK)) return ST_SINGULAR;
    return ST_OK;
}

// 1 / a for the pivots of gj_blocked: a is scaled by the power of two 2^-e
// (e the exponent of max(|Re|, |Im|), exact) into [1, 2), so one IEEE
// reciprocal of |a|^2 in [1, 8] suffices and nothing overflows or flushes
KNIT_DEV float2 crcp_pow2f(float2 a)
{
    const float m = fmaxf(fabsf(a.x), fabsf(a.y));
    const int e = min(max(((__float_as_int(m) >> 23) & 0xff) - 127, -126), 126);
    const float s = __int_as_float((127 - e) << 23);
    const float ax = a.x * s, ay = a.y * s;
    const float d = __frcp_rn(fmaf(ax, ax, ay * ay)) * s;
    return make_float2(ax * d, -ay * d);
}

// Blocked Gauss-Jordan inversion of X (M x M inside MP x MP, row-major,
// shared memory, in place) with the same implicit partial pivoting and the
// same result layout as gj_regs.  One elimination step with pivot row p and
// column k is the exact rank-1 update x -= u v^T with u = x[:, k] - e_p and
// v = (x[p, :] + e_k) / x[p][k]: it zeroes the pivot column and row and
// writes their new values in one stroke.  Steps are grouped in panels of NB
// columns.  Warp 0 runs a panel's steps alone, keeping the panel columns
// current in registers and forming each pivot row from X minus the panel's
// pending updates; U (NB x MP) and V (NB x MP) collect u and v.  Then the
// whole block applies X -= U^T V.  So the block meets at two barriers per
// panel instead of two per column, and the pivot search is one warp
// reduction of (|Re|+|Im| with its low mantissa bits cleared | inverted row)
// keys: the largest magnitude to 2^-17, lowest row on near-ties.
template <int MP, int TY, int TX, int NB = 8>
__device__ __forceinline__ int gj_blocked(float2 *X, int M, float2 *U, float2 *V, GJShared<MP> &g)
{
    static_assert(MP % 32 == 0 && MP % NB == 0 && 32 % NB == 0 && MP <= 128, "panel layout");
    constexpr int RA = MP / TY, RB = MP / TX, R2 = MP / 32, IB = MP <= 64 ? 6 : 7;
    constexpr unsigned IMASK = (1u << IB) - 1u, FULL = 0xffffffffu;
    const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX, lane = tid & 31;
    bool open[R2];   // warp 0: row lane + 32t may still become a pivot row
#pragma unroll
    for (int t = 0; t < R2; ++t) open[t] = lane + 32 * t < M;
    for (int K = 0; K < M; K += NB) {
        if (tid < 32) {
            const int tK = K >> 5, lK = K & 31;   // panel columns: lanes lK.., slot tK
            float2 pc[R2][NB];   // panel columns, rows lane + 32t
            float2 vh[R2][NB];   // this lane's entries of the panel's v vectors
#pragma unroll
            for (int t = 0; t < R2; ++t)
#pragma unroll
                for (int c = 0; c < NB; ++c) pc[t][c] = X[(lane + 32 * t) * MP + K + c];
            int bad = 0;
#pragma unroll
            for (int kk = 0; kk < NB; ++kk) {
                const int k = K + kk;
                if (k >= M) break;
                unsigned key = 0u;
#pragma unroll
                for (int t = 0; t < R2; ++t)
                    if (open[t])
                        key = max(key, (__float_as_uint(cabs1f(pc[t][kk])) & ~IMASK) |
                                           (IMASK - (unsigned)(lane + 32 * t)));
                key = __reduce_max_sync(FULL, key);
                if ((key & ~IMASK) == 0u) { bad = 1; break; }
                const int p = (int)(IMASK - (key & IMASK)), pl = p & 31, pt = p >> 5;
                float2 own = pc[0][kk];
#pragma unroll
                for (int t = 1; t < R2; ++t)
                    if (t == pt) own = pc[t][kk];
                const float2 piv = make_float2(__shfl_sync(FULL, own.x, pl),
                                               __shfl_sync(FULL, own.y, pl));
                float2 up[NB];   // u vectors of the earlier steps at row p
#pragma unroll
                for (int c = 0; c < kk; ++c) up[c] = U[c * MP + p];
                float2 rv[R2];
#pragma unroll
                for (int t = 0; t < R2; ++t) {
                    float2 r = X[p * MP + lane + 32 * t];
#pragma unroll
                    for (int c = 0; c < kk; ++c) r = cfmsf(up[c], vh[t][c], r);
                    rv[t] = r;
                }
                const float2 rinv = crcp_pow2f(piv);
                float2 uu[R2];
#pragma unroll
                for (int t = 0; t < R2; ++t) {
                    const int j = lane + 32 * t;
                    float2 v = cmulf(rv[t], rinv);
                    if (j == k) { v.x += rinv.x; v.y += rinv.y; }
                    vh[t][kk] = v;
                    V[kk * MP + j] = v;
                    float2 u = pc[t][kk];
                    if (j == p) { u.x -= 1.f; open[t] = false; }
                    U[kk * MP + j] = u;
                    uu[t] = u;
                }
                if (lane == 0) g.perm[k] = p;
                float2 vs = vh[0][kk];
#pragma unroll
                for (int t = 1; t < R2; ++t)
                    if (t == tK) vs = vh[t][kk];
#pragma unroll
                for (int c = kk + 1; c < NB; ++c) {
                    const float2 vk = make_float2(__shfl_sync(FULL, vs.x, lK + c),
                                                  __shfl_sync(FULL, vs.y, lK + c));
#pragma unroll
                    for (int t = 0; t < R2; ++t) pc[t][c] = cfmsf(uu[t], vk, pc[t][c]);
                }
                __syncwarp();
            }
            if (lane == 0) g.flag = bad;
        }
        __syncthreads();
        if (g.flag) return ST_SINGULAR;
        // X -= U^T V over the whole matrix, a register tile per thread
        const int nk = min(NB, M - K);
        float2 acc[RA][RB];
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int b = 0; b < RB; ++b) acc[a][b] = X[(ty + TY * a) * MP + tx + TX * b];
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            if (c < nk) {
                float2 ua[RA], vb[RB];
#pragma unroll
                for (int a = 0; a < RA; ++a) ua[a] = U[c * MP + ty + TY * a];
#pragma unroll
                for (int b = 0; b < RB; ++b) vb[b] = V[c * MP + tx + TX * b];
#pragma unroll
                for (int a = 0; a < RA; ++a)
#pragma unroll
                    for (int b = 0; b < RB; ++b) acc[a][b] = cfmsf(ua[a], vb[b], acc[a][b]);
            }
        }
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int b = 0; b < RB; ++b) X[(ty + TY * a) * MP + tx + TX * b] = acc[a][b];
        __syncthreads();
    }
    return ST_OK;
}

// store the inverse held in x (see gj_regs) into X (MP x MP, row-major)
template <int MP, int TY = 16, int TX = 16>
__device__ __forceinline__ void store_inverse(const float2 (&x)[MP / TY][MP / TX], int M,
                                              GJShared<MP> &g, float2 *X)
{
    constexpr int RA = MP / TY, RB = MP / TX, NTH = TY * TX;
    const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX;
    for (int k = tid; k < M; k += NTH) g.pos[g.perm[k]] = k;
    __syncthreads();
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int i = ty + TY * a, c = tx + TX * b;
            if (i < M && c < M) X[g.pos[i] * MP + g.perm[c]] = x[a][b];
            else X[i * MP + c] = x[a][b];
        }
    __syncthreads();
}

// one refinement step g = X + X R, kept as hi + lo in (Gh, Gl); R has row
// stride RS (padded rows avoid shared-memory bank conflicts where R is
// written one row per lane)
template <int MP, int RS = MP, int TY = 16, int TX = 16, int RA0 = 0, int NRA = MP / TY>
__device__ __forceinline__ void refine(const float2 *X, const float2 *R, float2 *Gh, float2 *Gl,
                                       int M)
{
    constexpr int RB = MP / TX;
    const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX;
    float2 acc[NRA][RB];
#pragma unroll
    for (int a = 0; a < NRA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int k = 0; k < M; ++k) {
        float2 xa[NRA], rb[RB];
#pragma unroll
        for (int a = 0; a < NRA; ++a) xa[a] = X[(ty + TY * (RA0 + a)) * MP + k];
#pragma unroll
        for (int b = 0; b < RB; ++b) rb[b] = R[k * RS + tx + TX * b];
#pragma unroll
        for (int a = 0; a < NRA; ++a)
#pragma unroll
            for (int b = 0; b < RB; ++b) acc[a][b] = cfmaf(xa[a], rb[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < NRA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int e = (ty + TY * (RA0 + a)) * MP + tx + TX * b;
            const float2 xv = X[e];
            float hx, lx, hy, ly;
            two_sum(xv.x, acc[a][b].x, hx, lx);
            two_sum(xv.y, acc[a][b].y, hy, ly);
            Gh[e] = make_float2(hx, hy);
            Gl[e] = make_float2(lx, ly);
        }
}

// Largest value of a non-negative float over the block (NTH threads);
// buf holds NTH / 32 words.  Non-negative floats order like their bit
// patterns, so each warp reduces the bits in one instruction.
template <int NTH>
__device__ __forceinline__ float block_max_nonneg(float v, unsigned *buf)
{
    const unsigned k = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
    if ((threadIdx.x & 31) == 0) buf[threadIdx.x >> 5] = k;
    __syncthreads();
    unsigned m = 0u;
#pragma unroll
    for (int w = 0; w < NTH / 32; ++w) m = max(m, buf[w]);
    return __uint_as_float(m);
}

// With R = I - A X' exact, A^{-1} = X' (I - R)^{-1} = X' (I + R + R^2 + ...):
// one refinement step keeps I + R and leaves an error of order |R|^2, each
// further term multiplies it by |R|.  neumann_terms picks how many further
// terms bring (sqrt(M) max|R_ij|)^(2 + n) below NEUMANN_TOL (at most
// NEUMANN_MAX); well-conditioned slices need none.
constexpr int NEUMANN_MAX = 8;
constexpr float NEUMANN_TOL = 1e-8f;
KNIT_DEV int neumann_terms(float rmax, int M)
{
    const float p = sqrtf((float)M) * rmax;
    float t = p * p;
    int n = 0;
    while (t > NEUMANN_TOL && n < NEUMANN_MAX) {
        t *= p;
        ++n;
    }
    return n;
}

// One Horner step of the series on the thread's tile rows RA0 .. RA0+NRA-1:
// acc = R + R S (R, S with row stride RS; zero outside M x M)
template <int MP, int RS, int TY, int TX, int RA0 = 0, int NRA = MP / TY>
__device__ __forceinline__ void neumann_tile(const float2 *R, const float2 *S,
                                             float2 (&acc)[NRA][MP / TX], int M)
{
    constexpr int RB = MP / TX;
    const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX;
#pragma unroll
    for (int a = 0; a < NRA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[a][b] = R[(ty + TY * (RA0 + a)) * RS + tx + TX * b];
    for (int k = 0; k < M; ++k) {
        float2 ra[NRA], sb[RB];
#pragma unroll
        for (int a = 0; a < NRA; ++a) ra[a] = R[(ty + TY * (RA0 + a)) * RS + k];
#pragma unroll
        for (int b = 0; b < RB; ++b) sb[b] = S[k * RS + tx + TX * b];
#pragma unroll
        for (int a = 0; a < NRA; ++a)
#pragma unroll
            for (int b = 0; b < RB; ++b) acc[a][b] = cfmaf(ra[a], sb[b], acc[a][b]);
    }
}

// The further terms in place: S (row stride RS) receives R + R S_prev n
// times, starting from S_prev = R.  Every thread holds its whole tile, so
// one barrier between the reads and the writes of a step suffices.
template <int MP, int RS, int TY, int TX>
__device__ __forceinline__ void neumann_inplace(const float2 *R, float2 *S, int M, int n)
{
    constexpr int RA = MP / TY, RB = MP / TX;
    const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX;
    for (int t = 0; t < n; ++t) {
        float2 acc[RA][RB];
        neumann_tile<MP, RS, TY, TX>(R, t == 0 ? R : S, acc, M);
        __syncthreads();
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int b = 0; b < RB; ++b) S[(ty + TY * a) * RS + tx + TX * b] = acc[a][b];
        __syncthreads();
    }
}

// Above this largest |R_ij| the refinement product X S is accumulated
// error-free (refine_exact): the rounding of an fp32 product, about
// 2^-24 sqrt(M) max|R_ij| relative, would otherwise enter every later slice.
constexpr float EXACT_RMAX = 1e-4f;

// s + e += a * b with the product's rounding error kept (TwoProduct by FMA,
// running sum by two_sum)
KNIT_DEV void dot2_acc1(float a, float b, float &s, float &e)
{
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    float t, te;
    two_sum(s, p, t, te);
    s = t;
    e += te + pe;
}

// refine with X S accumulated as double-float: g = X + (X S)_hi + (X S)_lo
template <int MP, int RS = MP, int TY = 16, int TX = 16, int RA0 = 0, int NRA = MP / TY>
__device__ __forceinline__ void refine_exact(const float2 *X, const float2 *S, float2 *Gh,
                                             float2 *Gl, int M)
{
    constexpr int RB = MP / TX;
    const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX;
    float2 sh[NRA][RB], se[NRA][RB];
#pragma unroll
    for (int a = 0; a < NRA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            sh[a][b] = make_float2(0.f, 0.f);
            se[a][b] = make_float2(0.f, 0.f);
        }
    for (int k = 0; k < M; ++k) {
        float2 xa[NRA], sb[RB];
#pragma unroll
        for (int a = 0; a < NRA; ++a) xa[a] = X[(ty + TY * (RA0 + a)) * MP + k];
#pragma unroll
        for (int b = 0; b < RB; ++b) sb[b] = S[k * RS + tx + TX * b];
#pragma unroll
        for (int a = 0; a < NRA; ++a)
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                dot2_acc1(xa[a].x, sb[b].x, sh[a][b].x, se[a][b].x);
                dot2_acc1(-xa[a].y, sb[b].y, sh[a][b].x, se[a][b].x);
                dot2_acc1(xa[a].x, sb[b].y, sh[a][b].y, se[a][b].y);
                dot2_acc1(xa[a].y, sb[b].x, sh[a][b].y, se[a][b].y);
            }
    }
#pragma unroll
    for (int a = 0; a < NRA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int e = (ty + TY * (RA0 + a)) * MP + tx + TX * b;
            const float2 xv = X[e];
            float hx, lx, hy, ly;
            two_sum(xv.x, sh[a][b].x, hx, lx);
            lx += se[a][b].x;
            two_sum(hx, lx, hx, lx);
            two_sum(xv.y, sh[a][b].y, hy, ly);
            ly += se[a][b].y;
            two_sum(hy, ly, hy, ly);
            Gh[e] = make_float2(hx, hy);
            Gl[e] = make_float2(lx, ly);
        }
}

// Transmission from G_LL = Gh + Gl by the unitarity identity, in FP64:
// T = Re Tr[Gamma_R i(G - G^dagger)] - Re Tr[Gamma_R G Gamma_R G^dagger].
// G: MP*MP complex128 scratch.
template <int MP, int NTH = NT>
__device__ double ward_T(const float2 *Gh, const float2 *Gl, double2 *G, const double2 *SR, int M,
                         double *red)
{
    const int tid = threadIdx.x;
    for (int e = tid; e < MP * MP; e += NTH) {
        float2 h = Gh[e], l = Gl[e];
        G[e] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
    }
    __syncthreads();
    double t = 0.0;
    for (int e = tid; e < M * M; e += NTH) {
        const int i = e / M, j = e - i * M;
        double2 d = csub(SR[(size_t)i * M + j], cconj(SR[(size_t)j * M + i]));
        double2 gij = make_double2(-d.y, d.x);
        double2 u = csub(G[j * MP + i], cconj(G[i * MP + j]));
        double2 a = make_double2(-u.y, u.x);
        t += gij.x * a.x - gij.y * a.y;
        double2 y = make_double2(0.0, 0.0), z = make_double2(0.0, 0.0);
        for (int k = 0; k < M; ++k) {
            double2 d1 = csub(SR[(size_t)i * M + k], cconj(SR[(size_t)k * M + i]));
            double2 d2 = csub(SR[(size_t)k * M + j], cconj(SR[(size_t)j * M + k]));
            y = cfma(make_double2(-d1.y, d1.x), G[k * MP + j], y);
            z = cfma(G[i * MP + k], make_double2(-d2.y, d2.x), z);
        }
        t -= y.x * z.x + y.y * z.y;
    }
    return block_sum(t, red);
}

}  // namespace mixed
