// mixed_common.cuh -- pieces shared by the two mixed-precision sweep kernels
// (sweep_mixed.cu: double-float residual on CUDA cores; sweep_mixed_tc.cu:
// residual on the tcgen05 tensor cores).  One CTA of 256 threads works on a
// padded MP x MP complex matrix; thread (ty, tx) = (tid / 16, tid % 16) owns
// rows ty + 16a and columns tx + 16b (a, b < MP / 16).
#pragma once

#include "knit_common.cuh"
#include "dense_fp64.cuh"

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

// double-float complex values as float4 (hi.re, hi.im, lo.re, lo.im)
KNIT_DEV float4 df4_mul(float4 a, float4 b)
{
    float2 h, l;
    cdf_mul(make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y), make_float2(b.z, b.w), h,
            l);
    return make_float4(h.x, h.y, l.x, l.y);
}

// x - c r in one compensated pass: the products of the hi parts exact
// (TwoProduct), the hi-lo cross terms in fp32, the sums compensated (TwoSum),
// normalised once per part (~2^-46 relative to |x| + |c| |r|)
KNIT_DEV float4 df4_fms(float4 x, float4 c, float4 r)
{
    float p, pe, s1, t, er, ei;
    p = c.x * r.x;
    pe = fmaf(c.x, r.x, -p);
    two_sum(x.x, -p, s1, t);
    er = (x.z + t) - pe;
    p = c.y * r.y;
    pe = fmaf(c.y, r.y, -p);
    two_sum(s1, p, s1, t);
    er += t + pe;
    er -= fmaf(c.x, r.z, fmaf(c.z, r.x, -fmaf(c.y, r.w, c.w * r.y)));
    float4 o;
    two_sum(s1, er, o.x, o.z);
    p = c.x * r.y;
    pe = fmaf(c.x, r.y, -p);
    two_sum(x.y, -p, s1, t);
    ei = (x.w + t) - pe;
    p = c.y * r.x;
    pe = fmaf(c.y, r.x, -p);
    two_sum(s1, -p, s1, t);
    ei += t - pe;
    ei -= fmaf(c.x, r.w, fmaf(c.z, r.y, fmaf(c.y, r.z, c.w * r.x)));
    two_sum(s1, ei, o.y, o.w);
    return o;
}

// x + d for a real float d
KNIT_DEV float4 df4_add_real(float4 x, float d)
{
    float s1, t;
    two_sum(x.x, d, s1, t);
    t += x.z;
    two_sum(s1, t, x.x, x.z);
    return x;
}

template <int MP>
struct GJShared {
    float2 col[2][MP];
    float2 rowp[2][MP];
    float val[2][MP];
    int used[MP];
    int perm[MP];
    int pos[MP];
    float2 rinv[16];   // gj_blocked: 1 / pivot of the current panel's steps
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
            else if (W != 0.0 && s.xmap)
                o = s.sign[0] * knit_disorder(ms, n >> 1, s.xmap[((((n >> 1) & 1) << 1) | (n & 1)) * s.M + i], W);
            else if (W != 0.0) o = s.sign[i % s.block] * knit_disorder(ms, n, i / s.block, W);
            d = E - o;
        }
        eps[i] = d;
    }
}

// A diagonal V with one value v on every orbital multiplies g by the real
// number |v|^2 in V g V^dagger.  vuni (per parity): 0 general, 1 |v|^2 = 1
// (V g V^dagger = g), 2 the factor (vch + vcl) as double-float.  Called by
// thread 0 on the double diagonal of V (M values, stride `stride`).
KNIT_DEV void classify_vdiag(const double2 *Vd, int stride, int M, int &vuni, float &vch, float &vcl)
{
    const double2 v0 = Vd[0];
    bool same = true;
    for (int i = 1; i < M; ++i) {
        const double2 v = Vd[(size_t)i * stride];
        same = same && v.x == v0.x && v.y == v0.y;
    }
    const double c = v0.x * v0.x + v0.y * v0.y;
    vuni = !same || c == 0.0 ? 0 : (c == 1.0 ? 1 : 2);
    to_df(c, vch, vcl);
}

// Gv = V_n g V_n^dagger (+ Sigma_L at n = 0, + Sigma_R at n = L - 1) in
// double-float, in place over (Gh, Gl); vh/vl: diagonal of V per parity;
// vuni/vch/vcl (per parity, classify_vdiag) select the scalar form on the
// slices without a lead term.
template <int MP, int NTH = NT>
__device__ void form_gv(float2 *Gh, float2 *Gl, const float2 (*vh)[MP], const float2 (*vl)[MP],
                        int M, int n, int L, const double2 *SL, const double2 *SR,
                        const int *vuni, const float *vch, const float *vcl)
{
    const int q = n & 1;
    if (n > 0 && n < L - 1 && vuni[q]) {
        const bool unit = vuni[q] == 1;
        const float ch = vch[q], cl = vcl[q];
        for (int e = threadIdx.x; e < MP * MP; e += NTH) {
            const int i = e / MP, j = e - i * MP;
            if (i >= M || j >= M) {
                Gh[e] = make_float2(0.f, 0.f);
                Gl[e] = make_float2(0.f, 0.f);
            } else if (!unit) {
                float2 gh = Gh[e], gl = Gl[e];
                cdf_mul(gh, gl, make_float2(ch, 0.f), make_float2(cl, 0.f), gh, gl);
                Gh[e] = gh;
                Gl[e] = gl;
            }
        }
        return;
    }
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
// columns.  Warp 0 runs a panel's steps alone on the panel columns, kept
// current in registers: the pivot search, 1 / pivot and the update of the
// panel need nothing outside them.  Then the same warp forms the panel's v
// vectors for every column by forward substitution,
// v_k = (X[p_k, :] - sum_{c<k} u_c[p_k] v_c + e_k) / x[p_k][k], and the
// whole block applies X -= U V (U: MP x gj_ust(NB), row i holds u_c[i];
// V: NB x MP).  So the block meets at two barriers per panel, and a step's
// latency is one warp reduction of (|Re|+|Im| with its low mantissa bits
// cleared | inverted row) keys -- the largest magnitude to 2^-17, lowest
// row on near-ties -- plus broadcasts of the pivot row's panel entries.
//
// row stride of gj_blocked's U: rows of NB complex values padded to a
// multiple of 16 bytes plus 16, so that two steps load as one 16-byte vector
// and the panel warp's column stores spread over the banks
__host__ __device__ constexpr int gj_ust(int nb) { return nb + 2; }

template <int MP, int TY, int TX, int NB = 8>
__device__ __forceinline__ int gj_blocked(float2 *X, int M, float2 *U, float2 *V, GJShared<MP> &g)
{
    static_assert(MP % 32 == 0 && MP % NB == 0 && 32 % NB == 0 && MP <= 128, "panel layout");
    static_assert(NB % 2 == 0, "steps are loaded in pairs");
    constexpr int RA = MP / TY, RB = MP / TX, R2 = MP / 32, IB = MP <= 64 ? 6 : 7;
    constexpr int UST = gj_ust(NB);
    constexpr unsigned IMASK = (1u << IB) - 1u, FULL = 0xffffffffu;
    const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX, lane = tid & 31;
    bool open[R2];   // warp 0: row lane + 32t may still become a pivot row
#pragma unroll
    for (int t = 0; t < R2; ++t) open[t] = lane + 32 * t < M;
    for (int K = 0; K < M; K += NB) {
        const int nk = min(NB, M - K);
        if (tid < 32) {
            float2 pc[R2][NB];   // panel columns, rows lane + 32t
#pragma unroll
            for (int t = 0; t < R2; ++t)
#pragma unroll
                for (int c = 0; c < NB; ++c) pc[t][c] = X[(lane + 32 * t) * MP + K + c];
            int bad = 0;
#pragma unroll
            for (int kk = 0; kk < NB; ++kk) {
                if (kk >= nk) break;
                unsigned key = 0u;
#pragma unroll
                for (int t = 0; t < R2; ++t)
                    if (open[t])
                        key = max(key, (__float_as_uint(cabs1f(pc[t][kk])) & ~IMASK) |
                                           (IMASK - (unsigned)(lane + 32 * t)));
                key = __reduce_max_sync(FULL, key);
                if ((key & ~IMASK) == 0u) { bad = 1; break; }
                const int p = (int)(IMASK - (key & IMASK)), pl = p & 31, pt = p >> 5;
                // the pivot row's current panel entries, from lane p % 32
                float2 prow[NB];
#pragma unroll
                for (int c = kk; c < NB; ++c) {
                    float2 own = pc[0][c];
#pragma unroll
                    for (int t = 1; t < R2; ++t)
                        if (t == pt) own = pc[t][c];
                    prow[c] = make_float2(__shfl_sync(FULL, own.x, pl), __shfl_sync(FULL, own.y, pl));
                }
                const float2 rinv = crcp_pow2f(prow[kk]);
                float2 uu[R2];
#pragma unroll
                for (int t = 0; t < R2; ++t) {
                    const int i = lane + 32 * t;
                    float2 u = pc[t][kk];
                    if (i == p) { u.x -= 1.f; open[t] = false; }
                    U[i * UST + kk] = u;
                    uu[t] = u;
                }
                if (lane == 0) {
                    g.perm[K + kk] = p;
                    g.rinv[kk] = rinv;
                }
#pragma unroll
                for (int c = kk + 1; c < NB; ++c) {
                    const float2 vk = cmulf(prow[c], rinv);
#pragma unroll
                    for (int t = 0; t < R2; ++t) pc[t][c] = cfmsf(uu[t], vk, pc[t][c]);
                }
            }
            __syncwarp();
            if (!bad) {
                // v vectors of the panel for columns j = lane + 32t, one t at a
                // time in registers; V is stored after each, so that no store
                // sits between the loads of X and U of one substitution
#pragma unroll
                for (int t = 0; t < R2; ++t) {
                    const int j = lane + 32 * t;
                    float2 vj[NB];
#pragma unroll
                    for (int kk = 0; kk < NB; ++kk) {
                        if (kk < nk) {
                            const int p = g.perm[K + kk];
                            float2 r = X[p * MP + j];
#pragma unroll
                            for (int c = 0; c < kk; ++c) r = cfmsf(U[p * UST + c], vj[c], r);
                            if (j == K + kk) r.x += 1.f;
                            vj[kk] = cmulf(r, g.rinv[kk]);
                        }
                    }
#pragma unroll
                    for (int kk = 0; kk < NB; ++kk)
                        if (kk < nk) V[kk * MP + j] = vj[kk];
                }
            }
            if (lane == 0) g.flag = bad;
        }
        __syncthreads();
        if (g.flag) return ST_SINGULAR;
        // X -= U V over the whole matrix, a register tile per thread; U rows
        // are read two steps per 16-byte load
        float2 acc[RA][RB];
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int b = 0; b < RB; ++b) acc[a][b] = X[(ty + TY * a) * MP + tx + TX * b];
#pragma unroll
        for (int c = 0; c < NB; c += 2) {
            if (c < nk) {
                float4 ua[RA];
                float2 vb0[RB], vb1[RB];
#pragma unroll
                for (int a = 0; a < RA; ++a)
                    ua[a] = *reinterpret_cast<const float4 *>(U + (ty + TY * a) * UST + c);
#pragma unroll
                for (int b = 0; b < RB; ++b) {
                    vb0[b] = V[c * MP + tx + TX * b];
                    vb1[b] = V[(c + 1) * MP + tx + TX * b];
                }
                const bool two = c + 1 < nk;
#pragma unroll
                for (int a = 0; a < RA; ++a)
#pragma unroll
                    for (int b = 0; b < RB; ++b) {
                        acc[a][b] = cfmsf(make_float2(ua[a].x, ua[a].y), vb0[b], acc[a][b]);
                        if (two) acc[a][b] = cfmsf(make_float2(ua[a].z, ua[a].w), vb1[b], acc[a][b]);
                    }
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

template <bool B> struct BoolC { static constexpr bool value = B; };

// 1 / a for the pivots of gj_lookahead, without a branch: a is scaled by
// the power of two 2^-e (e the exponent of max(|Re|, |Im|), exact) into
// [1, 2), and |a|^2 in [1, 8] takes one approximate reciprocal.  The result
// only seeds an inverse that the refinement corrects.
KNIT_DEV float2 crcp_fastf(float2 a)
{
    const float m = fmaxf(fabsf(a.x), fabsf(a.y));
    const int e = min(max(((__float_as_int(m) >> 23) & 0xff) - 127, -126), 126);
    const float s = __int_as_float((127 - e) << 23);
    const float ax = a.x * s, ay = a.y * s;
    const float d = __fdividef(1.0f, fmaf(ax, ax, ay * ay)) * s;
    return make_float2(ax * d, -ay * d);
}

// Gauss-Jordan with look-ahead: the algorithm of gj_blocked (same implicit
// pivoting, same result layout), rescheduled so that a panel's elimination
// overlaps the previous panel's rank update.  For panel P (columns
// K .. K+NB-1) one step reads only the panel columns, so
//   * the warps on the other three schedulers (warp 0 keeps its scheduler
//     to itself) apply X -= U V of panel P-1 to the panel-P columns, signal
//     warp 0 through named barrier 1, and go on with all other columns,
//     register-tiled over their rows, while
//   * warp 0 runs the NB steps on the panel-P columns;
// then, after one barrier, one thread per column forms panel P's v vectors
// by forward substitution from the pivot rows of the matrix at the start of
// the panel (an explicit inverse of the substitution's triangular matrix
// would not be bounded by the pivoting, and loses accuracy on
// ill-conditioned A).  Ub / Vb hold two panels' U (MP x gj_ust(NB)) and
// V (NB x MP) in turn.
template <int MP, int NTH, int TY, int TX, int NB = 8, int NWA = NTH / 32 - NTH / 128>
__device__ __forceinline__ int gj_lookahead(float2 *X, int M, float2 *Ub, float2 *Vb,
                                            GJShared<MP> &g)
{
    static_assert(MP % 32 == 0 && MP % NB == 0 && 32 % NB == 0 && MP <= 128, "panel layout");
    static_assert(NB % 2 == 0 && MP <= NTH && TY * TX == NTH, "thread layout");
    constexpr int RA = MP / TY, RB = MP / TX, R2 = MP / 32, IB = MP <= 64 ? 6 : 7;
    constexpr int UST = gj_ust(NB), NW = NTH / 32;
    static_assert(NWA >= 1 && NWA <= NW - NW / 4, "workers: warps off warp 0's scheduler");
    constexpr unsigned IMASK = (1u << IB) - 1u, FULL = 0xffffffffu;
    const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX, lane = tid & 31, warp = tid >> 5;
    bool open[R2];   // warp 0: row lane + 32t may still become a pivot row
#pragma unroll
    for (int t = 0; t < R2; ++t) open[t] = lane + 32 * t < M;
    const int NP = (M + NB - 1) / NB;
    for (int P = 0;; ++P) {
        const int K = P * NB;
        const float2 *Up = Ub + ((P + 1) & 1) * MP * UST;   // panel P-1
        const float2 *Vp = Vb + ((P + 1) & 1) * NB * MP;
        const int nkp = P > 0 ? min(NB, M - (P - 1) * NB) : 0;
        if (P == NP) {
            // the last panel's update, over the whole matrix
            float2 acc[RA][RB];
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[a][b] = X[(ty + TY * a) * MP + tx + TX * b];
#pragma unroll
            for (int c = 0; c < NB; c += 2) {
                if (c < nkp) {
                    float4 ua[RA];
                    float2 vb0[RB], vb1[RB];
#pragma unroll
                    for (int a = 0; a < RA; ++a)
                        ua[a] = *reinterpret_cast<const float4 *>(Up + (ty + TY * a) * UST + c);
#pragma unroll
                    for (int b = 0; b < RB; ++b) {
                        vb0[b] = Vp[c * MP + tx + TX * b];
                        vb1[b] = Vp[(c + 1) * MP + tx + TX * b];
                    }
                    const bool two = c + 1 < nkp;
#pragma unroll
                    for (int a = 0; a < RA; ++a)
#pragma unroll
                        for (int b = 0; b < RB; ++b) {
                            acc[a][b] = cfmsf(make_float2(ua[a].x, ua[a].y), vb0[b], acc[a][b]);
                            if (two) acc[a][b] = cfmsf(make_float2(ua[a].z, ua[a].w), vb1[b], acc[a][b]);
                        }
                }
            }
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < RB; ++b) X[(ty + TY * a) * MP + tx + TX * b] = acc[a][b];
            __syncthreads();
            return ST_OK;
        }
        const int nk = min(NB, M - K);
        float2 *const U = Ub + (P & 1) * MP * UST;
        float2 *const V = Vb + (P & 1) * NB * MP;
        if (warp == 0) {
            // wait until the workers have brought the panel columns up to date
            if (P > 0) asm volatile("bar.sync 1, %0;" ::"r"(32 * (NWA + 1)) : "memory");
            float2 pc[R2][NB];   // panel columns, rows lane + 32t
#pragma unroll
            for (int t = 0; t < R2; ++t)
#pragma unroll
                for (int c = 0; c < NB; ++c) pc[t][c] = X[(lane + 32 * t) * MP + K + c];
            int pk[NB];        // pivot rows of the panel's steps
            float2 rk[NB];     // and 1 / pivot
            bool bad = false;
            // the NB steps; a full panel runs them without bound checks, and
            // no step branches (a vanishing pivot only raises bad)
            auto steps = [&](auto fullc) {
                constexpr bool FULLP = decltype(fullc)::value;
#pragma unroll
                for (int kk = 0; kk < NB; ++kk) {
                    if (!FULLP && kk >= nk) break;
                    unsigned key = 0u;
#pragma unroll
                    for (int t = 0; t < R2; ++t) {
                        const unsigned kt = (__float_as_uint(cabs1f(pc[t][kk])) & ~IMASK) |
                                            (IMASK - (unsigned)(lane + 32 * t));
                        key = max(key, open[t] ? kt : 0u);
                    }
                    key = __reduce_max_sync(FULL, key);
                    bad |= (key & ~IMASK) == 0u;
                    const int p = (int)(IMASK - (key & IMASK)), pl = p & 31, pt = p >> 5;
                    pk[kk] = p;
                    // the pivot row's current panel entries, from lane p % 32:
                    // the pivot and the next column first (they lead to the
                    // next step's pivot search), the rest after
                    float2 prow[NB];
                    auto fetch = [&](int c) {
                        float2 own = pc[0][c];
#pragma unroll
                        for (int t = 1; t < R2; ++t) own = t == pt ? pc[t][c] : own;
                        prow[c] = make_float2(__shfl_sync(FULL, own.x, pl), __shfl_sync(FULL, own.y, pl));
                    };
                    fetch(kk);
                    if (kk + 1 < NB) fetch(kk + 1);
                    const float2 rinv = crcp_fastf(prow[kk]);
                    if (kk + 1 < NB) {
                        const float2 vk = cmulf(prow[kk + 1], rinv);
#pragma unroll
                        for (int t = 0; t < R2; ++t) {
                            float2 u = pc[t][kk];
                            u.x -= lane + 32 * t == p ? 1.f : 0.f;
                            pc[t][kk + 1] = cfmsf(u, vk, pc[t][kk + 1]);
                        }
                    }
#pragma unroll
                    for (int c = kk + 2; c < NB; ++c) fetch(c);
#pragma unroll
                    for (int c = kk + 2; c < NB; ++c) {
                        const float2 vk = cmulf(prow[c], rinv);
#pragma unroll
                        for (int t = 0; t < R2; ++t) {
                            const int i = lane + 32 * t;
                            float2 u = pc[t][kk];
                            u.x -= i == p ? 1.f : 0.f;
                            pc[t][c] = cfmsf(u, vk, pc[t][c]);
                        }
                    }
#pragma unroll
                    for (int t = 0; t < R2; ++t) {
                        const int i = lane + 32 * t;
                        float2 u = pc[t][kk];
                        u.x -= i == p ? 1.f : 0.f;
                        U[i * UST + kk] = u;
                        open[t] = open[t] && i != p;
                    }
                    rk[kk] = rinv;
                }
            };
            if (nk == NB) steps(BoolC<true>{});
            else steps(BoolC<false>{});
            if (lane == 0)
#pragma unroll
                for (int kk = 0; kk < NB; ++kk)
                    if (kk < nk) {
                        g.perm[K + kk] = pk[kk];
                        g.rinv[kk] = rk[kk];
                    }
            if (lane == 0) g.flag = bad ? 1 : 0;
        } else if ((warp & 3) != 0 && warp - 1 - (warp >> 2) < NWA && P > 0) {
            // workers (the warps off warp 0's scheduler) apply X -= U V of
            // panel P-1: first to the panel-P columns, which warp 0 waits
            // for, then to all other columns
            const int wa = warp - 1 - (warp >> 2);   // 0 .. NWA-1
            for (int e = wa * 32 + lane; e < MP * NB; e += 32 * NWA) {
                const int i = e / NB, c = e % NB;
                float2 acc = X[i * MP + K + c];
#pragma unroll
                for (int cp = 0; cp < NB; ++cp)
                    if (cp < nkp) acc = cfmsf(Up[i * UST + cp], Vp[cp * MP + K + c], acc);
                X[i * MP + K + c] = acc;
            }
            asm volatile("bar.arrive 1, %0;" ::"r"(32 * (NWA + 1)) : "memory");
            // rows wa, wa + NWA, ... (at most RW), lanes along the row, in
            // chunks of RWC rows (at most 12 accumulators per lane)
            constexpr int RW = (MP + NWA - 1) / NWA;
            constexpr int RWC = RW < 12 / R2 ? RW : (12 / R2 > 0 ? 12 / R2 : 1);
#pragma unroll 1
            for (int r0 = 0; r0 < RW; r0 += RWC) {
                float2 acc[RWC][R2];
#pragma unroll
                for (int r = 0; r < RWC; ++r) {
                    const int i = wa + NWA * (r0 + r);
#pragma unroll
                    for (int t = 0; t < R2; ++t)
                        acc[r][t] = i < MP ? X[i * MP + lane + 32 * t] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int c = 0; c < NB; c += 2) {
                    if (c < nkp) {
                        float2 v0[R2], v1[R2];
#pragma unroll
                        for (int t = 0; t < R2; ++t) {
                            v0[t] = Vp[c * MP + lane + 32 * t];
                            v1[t] = Vp[(c + 1) * MP + lane + 32 * t];
                        }
                        const bool two = c + 1 < nkp;
#pragma unroll
                        for (int r = 0; r < RWC; ++r) {
                            const int i = wa + NWA * (r0 + r);
                            if (i < MP) {
                                const float4 q = *reinterpret_cast<const float4 *>(Up + i * UST + c);
#pragma unroll
                                for (int t = 0; t < R2; ++t) {
                                    acc[r][t] = cfmsf(make_float2(q.x, q.y), v0[t], acc[r][t]);
                                    if (two) acc[r][t] = cfmsf(make_float2(q.z, q.w), v1[t], acc[r][t]);
                                }
                            }
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < RWC; ++r) {
                    const int i = wa + NWA * (r0 + r);
                    if (i < MP)
#pragma unroll
                        for (int t = 0; t < R2; ++t) {
                            const int j = lane + 32 * t;
                            if (j < K || j >= K + NB) X[i * MP + j] = acc[r][t];
                        }
                }
            }
        }
        __syncthreads();
        if (g.flag) return ST_SINGULAR;
        if (tid < MP) {
            // the panel's v vectors by forward substitution, one column per
            // thread: v_k = (X[p_k, j] + [j = K+k] - sum_{c<k} u_c[p_k] v_c) / pivot_k
            const int j = tid;
            float2 vj[NB];
#pragma unroll
            for (int kk = 0; kk < NB; ++kk) {
                if (kk < nk) {
                    const int p = g.perm[K + kk];
                    float2 r = X[p * MP + j];
                    if (j == K + kk) r.x += 1.f;
#pragma unroll
                    for (int c = 0; c < kk; ++c) r = cfmsf(U[p * UST + c], vj[c], r);
                    vj[kk] = cmulf(r, g.rinv[kk]);
                }
            }
#pragma unroll
            for (int kk = 0; kk < NB; ++kk)
                if (kk < nk) V[kk * MP + j] = vj[kk];
        }
        __syncthreads();
    }
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

// The series cannot reach NEUMANN_TOL within NEUMANN_MAX terms (or max|R_ij|
// is not a number): the complex64 inverse is no approximate inverse, A_n
// being nearly singular -- near a resonance of the part of the system left
// of slice n, which long disordered samples meet.  The slice is then
// inverted in FP64 (fallback_*).
KNIT_DEV bool refinement_fails(float rmax, int M)
{
    const float p = sqrtf((float)M) * rmax;
    float t = p * p;
#pragma unroll
    for (int n = 0; n < NEUMANN_MAX; ++n) t *= p;
    return !(t <= NEUMANN_TOL);
}

// scratch of gj_invert64 carved from raw memory: (2M + 1) complex128 and
// M + 2 ints, 16-byte aligned base
KNIT_DEV GJScratch64 fallback_scratch(void *base, int M)
{
    GJScratch64 sc;
    sc.row = reinterpret_cast<double2 *>(base);
    sc.col = sc.row + M;
    sc.pval = sc.col + M;
    sc.perm = reinterpret_cast<int *>(sc.pval + 1);
    sc.flag = sc.perm + M;
    sc.piv = sc.flag + 1;
    return sc;
}

// A_n in FP64 (row-major, leading dimension M) from the double-float Gv
// (Gh + Gl, row stride ldg): A = -Gv, plus diag(eps) - H0 when eps is given
// (kernels whose Gv does not already carry them).  Ends with __syncthreads.
KNIT_DEV void fallback_form_a(double2 *A, const float2 *Gh, const float2 *Gl, int ldg, int M,
                              const double *eps, const SysDev &s)
{
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        const int i = e / M, j = e - i * M;
        const float2 h = Gh[i * ldg + j], l = Gl[i * ldg + j];
        A[e] = make_double2(-((double)h.x + (double)l.x), -((double)h.y + (double)l.y));
    }
    __syncthreads();
    if (eps) {
        for (int i = threadIdx.x; i < M; i += blockDim.x) {
            A[i * M + i].x += eps[i];
            for (int c = s.h0_rowptr[i]; c < s.h0_rowptr[i + 1]; ++c) {
                const double2 h = s.h0_val[c];
                double2 &a = A[i * M + s.h0_col[c]];
                a.x -= h.x;
                a.y -= h.y;
            }
        }
        __syncthreads();
    }
}

// the FP64 inverse back into the double-float state (identity in the
// padding, as the refinement leaves it).  Ends with __syncthreads.
KNIT_DEV void fallback_store_g(const double2 *A, float2 *Gh, float2 *Gl, int ldg, int MPad, int M)
{
    for (int e = threadIdx.x; e < MPad * MPad; e += blockDim.x) {
        const int i = e / MPad, j = e - i * MPad;
        float2 h, l;
        if (i < M && j < M) {
            const double2 v = A[i * M + j];
            to_df(v.x, h.x, l.x);
            to_df(v.y, h.y, l.y);
        } else {
            h = make_float2(i == j ? 1.f : 0.f, 0.f);
            l = make_float2(0.f, 0.f);
        }
        Gh[i * ldg + j] = h;
        Gl[i * ldg + j] = l;
    }
    __syncthreads();
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

// ward_T in double-float on the CUDA cores: its two M^3 complex products in
// FP64 take ~M^3 FP64 FMAs per instance on a part whose FP64 rate is 1/64 of
// FP32.  Gamma_R = i(Sigma_R - Sigma_R^dagger) is staged in double-float in
// Gam (MPT x MPT float4, a buffer the caller no longer needs); (Gamma G) and
// (G Gamma) are accumulated in double-float, the traces in FP64.  Gh, Gl:
// G_LL row-major with leading dimension MPT.
template <int MPT, int NTT>
__device__ __noinline__ double ward_T_df(const float2 *Gh, const float2 *Gl, float4 *Gam,
                                         const double2 *SR, int M, double *red)
{
    const int tid = threadIdx.x;
    for (int e = tid; e < MPT * MPT; e += NTT) {
        const int i = e / MPT, j = e - i * MPT;
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < M && j < M) {
            const double2 d = csub(SR[(size_t)i * M + j], cconj(SR[(size_t)j * M + i]));
            to_df(-d.y, g.x, g.z);
            to_df(d.x, g.y, g.w);
        }
        Gam[e] = g;
    }
    __syncthreads();
    double t = 0.0;
    for (int e = tid; e < M * M; e += NTT) {
        const int i = e / M, j = e - i * M;
        const float4 gij = Gam[i * MPT + j];
        const double gr = (double)gij.x + (double)gij.z, gi = (double)gij.y + (double)gij.w;
        const double2 gji = make_double2((double)Gh[j * MPT + i].x + (double)Gl[j * MPT + i].x,
                                         (double)Gh[j * MPT + i].y + (double)Gl[j * MPT + i].y);
        const double2 gijc = make_double2((double)Gh[i * MPT + j].x + (double)Gl[i * MPT + j].x,
                                          (double)Gh[i * MPT + j].y + (double)Gl[i * MPT + j].y);
        // a = i (G_ji - conj(G_ij)); t += Re(Gamma_ij a)
        const double ux = gji.x - gijc.x, uy = gji.y + gijc.y;
        t += gr * (-uy) - gi * ux;
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f), z = y;
        for (int k = 0; k < M; ++k) {
            const float4 gik = Gam[i * MPT + k], gkj = Gam[k * MPT + j];
            const float2 ah = Gh[k * MPT + j], al = Gl[k * MPT + j], bh = Gh[i * MPT + k], bl = Gl[i * MPT + k];
            y = df4_fms(y, make_float4(-gik.x, -gik.y, -gik.z, -gik.w), make_float4(ah.x, ah.y, al.x, al.y));
            z = df4_fms(z, make_float4(-bh.x, -bh.y, -bl.x, -bl.y), gkj);
        }
        // t -= Re(y conj(z))
        const double yr = (double)y.x + (double)y.z, yi = (double)y.y + (double)y.w;
        const double zr = (double)z.x + (double)z.z, zi = (double)z.y + (double)z.w;
        t -= yr * zr + yi * zi;
    }
    return block_sum(t, red);
}

// G_LL = Gh + Gl (row-major, leading dimension MP) into dst (M x M, complex128)
template <int MP, int NTH = NT>
__device__ void store_gll_df(const float2 *Gh, const float2 *Gl, int M, double2 *dst)
{
    for (int e = threadIdx.x; e < M * M; e += NTH) {
        const int i = e / M, j = e - i * M;
        dst[e] = make_double2((double)Gh[i * MP + j].x + (double)Gl[i * MP + j].x,
                              (double)Gh[i * MP + j].y + (double)Gl[i * MP + j].y);
    }
}

// G_LL from ward_T's scratch G (MP x MP, row-major) into dst (M x M)
template <int MP, int NTH = NT>
__device__ void store_gll(const double2 *G, int M, double2 *dst)
{
    for (int e = threadIdx.x; e < M * M; e += NTH) {
        const int i = e / M, j = e - i * M;
        dst[e] = G[i * MP + j];
    }
}

}  // namespace mixed
