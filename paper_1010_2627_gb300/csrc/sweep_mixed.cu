// sweep_mixed.cu -- the slice sweep in mixed precision with the residual on
// CUDA cores (complex64 inversion, double-float refinement), padded widths
// MP in {16, 32, 64}, and the local density of states built on it.
//
// Per slice n (mixed_step), with the state g_{n-1} carried as hi + lo
// complex64 pairs (KNIT user guide Sec. 5.3 D knitting in slice form; Eq. 2
// by block elimination):
//   1. Gv = V_n g_{n-1} V_n^dagger (+ Sigma_L at n = 0, + Sigma_R at n = L-1)
//      formed in double-float, so that A_n = D_n - Gv with D_n = E - H_n;
//   2. X = fl32(D_n - Gv_hi) inverted by Gauss-Jordan with implicit partial
//      pivoting (look-ahead blocked form for MP >= 32, in registers at 16);
//   3. residual R = I - A_n X accumulated with error-free products and sums
//      (TwoProduct / TwoSum, "Dot2" of Ogita, Rump & Oishi 2005), using the
//      exact D_n and both words of Gv, then rounded to complex64;
//   4. g_n = X (I + R + R^2 + ...) kept as hi + lo, with as many terms as
//      max|R_ij| asks for, the product X S error-free when max|R_ij| is large,
//      and the slice inverted in FP64 when the series cannot converge
//      (mixed_common.cuh).
// The last g (slice L-1, which includes Sigma_R) is the exact G_{L-1,L-1} of
// the whole system, and the transmission follows from it by the unitarity
// (Ward) identity i(G - G^dagger) = G (Gamma_L + Gamma_R) G^dagger:
//   T = Re Tr[Gamma_R i(G_LL - G_LL^dagger)] - Re Tr[Gamma_R G_LL Gamma_R G_LL^dagger],
// evaluated in FP64.  This equals the Sec. 2.3 formula
// Tr[Gamma_L G_{0,L-1} Gamma_R G_{0,L-1}^dagger] (two-terminal reciprocity)
// without carrying the off-diagonal chain G_{0,n}.
//
// Supported structure: inter-slice couplings V diagonal (square lattices,
// brick-wall masks).  One CTA per instance at a time, instances taken from an
// atomic counter.  sweep_mixed_tc.cu moves step 3 to the tensor cores for
// MP = 64.

#include "mixed_common.cuh"

using namespace mixed;

namespace {

template <int MP>
struct MixedSmem {
    float2 X[MP * MP];     // inverse of the complex64 A_n (columns in final order)
    float2 R[MP * MP];     // residual (X and R together hold G_LL as complex128 at the end,
                           // and A_n as complex128 on a slice inverted in FP64)
    float2 Gh[MP * MP];    // g (hi) / Gv (hi)
    float2 Gl[MP * MP];    // g (lo) / Gv (lo)
    float2 H0f[MP * MP];   // complex64 copy of H0 for forming X
    float2 S[MP * MP];     // further Neumann terms of the refinement
    GJShared<MP> gj;
    double eps[MP];        // E - onsite for the current slice
    int vuni[2];           // V's diagonal uniform (classify_vdiag), per parity
    float vch[2], vcl[2];
    float2 vh[2][MP];      // diagonal of V (per parity), hi
    float2 vl[2][MP];      // lo
    double red[NT / 32];
    unsigned redu[NT / 32];
    int inst;
    int cur_sys;
};

}  // namespace

// per-system constants: H0 as complex64, diagonal of V (per parity) as
// double-float
template <int MP>
__device__ __forceinline__ void mixed_load_system(MixedSmem<MP> &sm, const SysDev &s)
{
    const int tid = threadIdx.x, M = s.M;
    const size_t MM = (size_t)M * M;
    // per-system constants: H0 as complex64, diagonal of V as double-float
    for (int e = tid; e < MP * MP; e += NT) {
        int i = e / MP, j = e - i * MP;
        double2 h = (i < M && j < M) ? s.H0[(size_t)i * M + j] : make_double2(0.0, 0.0);
        sm.H0f[e] = make_float2((float)h.x, (float)h.y);
    }
    for (int q = 0; q < 2; ++q)
        for (int i = tid; i < MP; i += NT) {
            double2 v = make_double2(0.0, 0.0);
            if (i < M) v = s.V[(size_t)(q % s.Vperiod) * MM + (size_t)i * M + i];
            float hx, lx, hy, ly;
            to_df(v.x, hx, lx);
            to_df(v.y, hy, ly);
            sm.vh[q][i] = make_float2(hx, hy);
            sm.vl[q][i] = make_float2(lx, ly);
        }
    if (tid < 2)
        classify_vdiag(s.V + (size_t)(tid % s.Vperiod) * MM, M + 1, M, sm.vuni[tid], sm.vch[tid],
                       sm.vcl[tid]);
    __syncthreads();
}

// One slice of the sweep: the state g_{n-1} in (Gh, Gl) becomes g_n.
// Returns ST_OK or ST_SINGULAR.  Called by all NT threads.
template <int MP>
__device__ __forceinline__ int mixed_step(MixedSmem<MP> &sm, const SysDev &s, const InstParams &ip,
                                          int M, int n, int L)
{
    constexpr int RT = MP / 16;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const double E = ip.E;
    const uint64_t ms = ip.ms;
    const double W = ip.W;
    const double2 *SL = ip.SL;
    const double2 *SR = ip.SR;
    int st = ST_OK;
        slice_diag<MP>(sm.eps, s, ms, W, E, n);
        form_gv<MP>(sm.Gh, sm.Gl, sm.vh, sm.vl, M, n, L, SL, SR, sm.vuni, sm.vch, sm.vcl);
        __syncthreads();

        // ---- X = fl32(D - Gv_hi), Gauss-Jordan in registers
        float2 x[RT][RT];
#pragma unroll
        for (int a = 0; a < RT; ++a)
#pragma unroll
            for (int b = 0; b < RT; ++b) {
                int i = ty + 16 * a, j = tx + 16 * b;
                float2 v;
                if (i < M && j < M) {
                    float2 g = sm.Gh[i * MP + j], h = sm.H0f[i * MP + j];
                    v = make_float2(-g.x - h.x, -g.y - h.y);
                    if (i == j) v.x += (float)sm.eps[i];
                } else {
                    v = make_float2(i == j ? 1.f : 0.f, 0.f);
                }
                x[a][b] = v;
            }
        if constexpr (MP >= 32) {
            // look-ahead Gauss-Jordan in shared memory (U, V panels in the
            // residual and series buffers, free until the residual)
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < RT; ++b) sm.X[(ty + 16 * a) * MP + tx + 16 * b] = x[a][b];
            __syncthreads();
            st = gj_lookahead<MP, NT, 16, 16>(sm.X, M, sm.R, sm.S, sm.gj);
            if (st != ST_OK) return st;
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < RT; ++b) x[a][b] = sm.X[(ty + 16 * a) * MP + tx + 16 * b];
        } else {
            st = gj_regs<MP>(x, M, sm.gj);
            if (st != ST_OK) return st;
        }
        store_inverse<MP>(x, M, sm.gj, sm.X);

        // ---- residual R = I - D X + Gv X in double-float
        float rloc = 0.f;
        {
            float2 ah[RT][RT], al[RT][RT];
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < RT; ++b) {
                    ah[a][b] = make_float2(0.f, 0.f);
                    al[a][b] = make_float2(0.f, 0.f);
                }
            for (int k = 0; k < M; ++k) {
                float2 gh[RT], gl[RT], xv[RT];
#pragma unroll
                for (int a = 0; a < RT; ++a) {
                    gh[a] = sm.Gh[(ty + 16 * a) * MP + k];
                    gl[a] = sm.Gl[(ty + 16 * a) * MP + k];
                }
#pragma unroll
                for (int b = 0; b < RT; ++b) xv[b] = sm.X[k * MP + tx + 16 * b];
#pragma unroll
                for (int a = 0; a < RT; ++a)
#pragma unroll
                    for (int b = 0; b < RT; ++b) {
                        dot2_acc(gh[a].x, gl[a].x, xv[b].x, ah[a][b].x, al[a][b].x);
                        dot2_acc(-gh[a].y, -gl[a].y, xv[b].y, ah[a][b].x, al[a][b].x);
                        dot2_acc(gh[a].x, gl[a].x, xv[b].y, ah[a][b].y, al[a][b].y);
                        dot2_acc(gh[a].y, gl[a].y, xv[b].x, ah[a][b].y, al[a][b].y);
                    }
            }
            // - D X = -(E - onsite_i) X_ij + sum_c H0_ic X_cj, and + I
#pragma unroll
            for (int a = 0; a < RT; ++a) {
                const int i = ty + 16 * a;
                if (i >= M) continue;
                float dh, dl;
                to_df(sm.eps[i], dh, dl);
#pragma unroll
                for (int b = 0; b < RT; ++b) {
                    const int j = tx + 16 * b;
                    float2 xij = sm.X[i * MP + j];
                    dot2_acc(-dh, -dl, xij.x, ah[a][b].x, al[a][b].x);
                    dot2_acc(-dh, -dl, xij.y, ah[a][b].y, al[a][b].y);
                }
                for (int c = s.h0_rowptr[i]; c < s.h0_rowptr[i + 1]; ++c) {
                    const int col = s.h0_col[c];
                    double2 h = s.h0_val[c];
                    float hxh, hxl, hyh, hyl;
                    to_df(h.x, hxh, hxl);
                    to_df(h.y, hyh, hyl);
#pragma unroll
                    for (int b = 0; b < RT; ++b) {
                        float2 xv = sm.X[col * MP + tx + 16 * b];
                        dot2_acc(hxh, hxl, xv.x, ah[a][b].x, al[a][b].x);
                        dot2_acc(-hyh, -hyl, xv.y, ah[a][b].x, al[a][b].x);
                        dot2_acc(hxh, hxl, xv.y, ah[a][b].y, al[a][b].y);
                        dot2_acc(hyh, hyl, xv.x, ah[a][b].y, al[a][b].y);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < RT; ++b) {
                    const int i = ty + 16 * a, j = tx + 16 * b;
                    float2 r = make_float2(0.f, 0.f);
                    if (i < M && j < M) {
                        float sx = ah[a][b].x, ex = al[a][b].x;
                        if (i == j) {
                            float t, te;
                            two_sum(sx, 1.0f, t, te);
                            sx = t;
                            ex += te;
                        }
                        r = make_float2(sx + ex, ah[a][b].y + al[a][b].y);
                    }
                    sm.R[i * MP + j] = r;
                    rloc = fmaxf(rloc, fmaxf(fabsf(r.x), fabsf(r.y)));
                }
        }
        const float rmax = block_max_nonneg<NT>(rloc, sm.redu);
        if (refinement_fails(rmax, M)) {
            // near-singular A_n: this slice in FP64, in the X and R
            // buffers (contiguous), scratch in the series buffer
            double2 *const A64 = reinterpret_cast<double2 *>(sm.X);
            fallback_form_a(A64, sm.Gh, sm.Gl, MP, M, sm.eps, s);
            st = gj_invert64(A64, M, fallback_scratch(sm.S, M));
            if (st != ST_OK) return st;
            fallback_store_g(A64, sm.Gh, sm.Gl, MP, MP, M);
            return ST_OK;
        }
        const int nx = neumann_terms(rmax, M);
        float2 *const S = nx ? sm.S : sm.R;
        neumann_inplace<MP, MP, 16, 16>(sm.R, S, M, nx);
        if (rmax > EXACT_RMAX)
            refine_exact<MP>(sm.X, S, sm.Gh, sm.Gl, M);
        else
            refine<MP>(sm.X, S, sm.Gh, sm.Gl, M);
        __syncthreads();
    return ST_OK;
}

template <int MP>
__global__ void __launch_bounds__(NT, 1)
knit_sweep_mixed_kernel(InstDev in)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MixedSmem<MP> &sm = *reinterpret_cast<MixedSmem<MP> *>(smem_raw);
    const int tid = threadIdx.x;
    if (tid == 0) sm.cur_sys = -1;

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
        if (reload) {
            mixed_load_system<MP>(sm, s);
            if (tid == 0) sm.cur_sys = si;
        }
        const InstParams ip = inst_params(in, inst, M);
        int st = ip.st;
        for (int n = 0; n < L && st == ST_OK; ++n) st = mixed_step<MP>(sm, s, ip, M, n, L);

        double T = 0.0;
        if (st == ST_OK) {
            T = ward_T_df<MP, NT>(sm.Gh, sm.Gl, reinterpret_cast<float4 *>(sm.X), ip.SR, M, sm.red);
            if (in.GLL) store_gll_df<MP>(sm.Gh, sm.Gl, M, in.GLL + (size_t)ip.out * M * M);
            if (!isfinite(T)) st = ST_NONFINITE;
        }
        if (tid == 0) {
            in.T[ip.out] = T;
            if (in.status) in.status[ip.out] = st;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Local density of states in mixed precision (Sec. 5.3 D knitting and sewing).
// The forward pass is the sweep above with g_n checkpointed as double-float
// every `save` slices; the backward (sewing) pass
//   G_nn = g_n + g_n V_{n+1}^dagger G_{n+1,n+1} V_{n+1} g_n,  LDOS = -Im G_nn[x][x] / pi,
// recomputes each segment's g_n from its checkpoint with the same mixed step
// and forms both products in double-float arithmetic (error-free products and
// sums on CUDA cores): complex64 products there would leave relative LDOS
// errors of 1e-4 .. 1e-3 on a 64 x 256 disordered bar.

// s + e += (xh + xl)(yh + yl) for real double-floats: the product's rounding
// error by FMA plus the cross terms, the running sum by two_sum
KNIT_DEV void df2_acc(float xh, float xl, float yh, float yl, float &s, float &e)
{
    const float p = xh * yh;
    float pe = fmaf(xh, yh, -p);
    pe = fmaf(xh, yl, pe);
    pe = fmaf(xl, yh, pe);
    float t, te;
    two_sum(s, p, t, te);
    s = t;
    e += te + pe;
}

// the thread's RT x RT tile of C = A B for double-float complex A, B (row
// stride MP, inner dimension M), as (hi, lo) per real part
template <int MP>
__device__ __forceinline__ void gemm_df_tile(const float2 *Ah, const float2 *Al, const float2 *Bh,
                                             const float2 *Bl, int M, float2 (&ch)[MP / 16][MP / 16],
                                             float2 (&cl)[MP / 16][MP / 16])
{
    constexpr int RT = MP / 16;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
        for (int b = 0; b < RT; ++b) {
            ch[a][b] = make_float2(0.f, 0.f);
            cl[a][b] = make_float2(0.f, 0.f);
        }
    for (int k = 0; k < M; ++k) {
        float2 ah[RT], al[RT], bh[RT], bl[RT];
#pragma unroll
        for (int a = 0; a < RT; ++a) {
            ah[a] = Ah[(ty + 16 * a) * MP + k];
            al[a] = Al[(ty + 16 * a) * MP + k];
        }
#pragma unroll
        for (int b = 0; b < RT; ++b) {
            bh[b] = Bh[k * MP + tx + 16 * b];
            bl[b] = Bl[k * MP + tx + 16 * b];
        }
#pragma unroll
        for (int a = 0; a < RT; ++a)
#pragma unroll
            for (int b = 0; b < RT; ++b) {
                df2_acc(ah[a].x, al[a].x, bh[b].x, bl[b].x, ch[a][b].x, cl[a][b].x);
                df2_acc(-ah[a].y, -al[a].y, bh[b].y, bl[b].y, ch[a][b].x, cl[a][b].x);
                df2_acc(ah[a].x, al[a].x, bh[b].y, bl[b].y, ch[a][b].y, cl[a][b].y);
                df2_acc(ah[a].y, al[a].y, bh[b].x, bl[b].x, ch[a][b].y, cl[a][b].y);
            }
    }
}

// double-float matrix (hi, lo, MP x MP each) between shared and global memory
template <int MP>
__device__ __forceinline__ void df_store(float2 *dst, const float2 *h, const float2 *l)
{
    for (int e = threadIdx.x; e < MP * MP; e += NT) {
        dst[e] = h[e];
        dst[MP * MP + e] = l[e];
    }
}
template <int MP>
__device__ __forceinline__ void df_load(float2 *h, float2 *l, const float2 *src)
{
    for (int e = threadIdx.x; e < MP * MP; e += NT) {
        h[e] = src[e];
        l[e] = src[MP * MP + e];
    }
    __syncthreads();
}

template <int MP>
__global__ void __launch_bounds__(NT, 1)
knit_ldos_mixed_kernel(InstDev in, int Lmax, int save, float2 *work, double *ldos,
                       long long ldos_stride)
{
    constexpr int RT = MP / 16;
    constexpr size_t DF = 2 * (size_t)MP * MP;   // float2 per double-float matrix
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MixedSmem<MP> &sm = *reinterpret_cast<MixedSmem<MP> *>(smem_raw);
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int nckmax = (Lmax + save - 1) / save;
    float2 *const cks = work + (size_t)blockIdx.x * (nckmax + save + 1) * DF;   // g_0, g_save, ...
    float2 *const seg = cks + (size_t)nckmax * DF;   // slot m - c: g_m of the current segment
    float2 *const Gs = seg + (size_t)save * DF;      // G_{n+1,n+1}
    if (tid == 0) sm.cur_sys = -1;

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
        if (reload) {
            mixed_load_system<MP>(sm, s);
            if (tid == 0) sm.cur_sys = si;
        }
        const InstParams ip = inst_params(in, inst, M);
        double *const out = ldos + (size_t)ip.out * ldos_stride;
        int st = ip.st;
        for (int n = 0; n < L && st == ST_OK; ++n) {
            st = mixed_step<MP>(sm, s, ip, M, n, L);
            if (st == ST_OK && n % save == 0 && n < L - 1) {
                df_store<MP>(cks + (size_t)(n / save) * DF, sm.Gh, sm.Gl);
                __syncthreads();
            }
        }
        double T = 0.0;
        if (st == ST_OK) {
            df_store<MP>(Gs, sm.Gh, sm.Gl);   // G_{L-1,L-1} = g_{L-1}
            for (int x = tid; x < M; x += NT)
                out[(size_t)(L - 1) * M + x] =
                    -((double)sm.Gh[x * MP + x].y + (double)sm.Gl[x * MP + x].y) / 3.141592653589793;
            T = ward_T_df<MP, NT>(sm.Gh, sm.Gl, reinterpret_cast<float4 *>(sm.X), ip.SR, M, sm.red);
            if (!isfinite(T)) st = ST_NONFINITE;
        }
        int seg_lo = -1;   // checkpoint slice whose segment the slots hold
        for (int n = L - 2; n >= 0 && st == ST_OK; --n) {
            const float2 *gn;
            if (n % save == 0) {
                gn = cks + (size_t)(n / save) * DF;
            } else {
                const int c = (n / save) * save;
                if (seg_lo != c) {
                    // recompute g_{c+1} .. g_n from the checkpoint g_c
                    df_load<MP>(sm.Gh, sm.Gl, cks + (size_t)(c / save) * DF);
                    for (int m = c + 1; m <= n && st == ST_OK; ++m) {
                        st = mixed_step<MP>(sm, s, ip, M, m, L);
                        if (st == ST_OK) df_store<MP>(seg + (size_t)(m - c) * DF, sm.Gh, sm.Gl);
                        __syncthreads();
                    }
                    seg_lo = c;
                    __syncthreads();
                    if (st != ST_OK) break;
                }
                gn = seg + (size_t)(n - c) * DF;
            }
            // g_n into (Gh, Gl); F = V^dagger G V (V of slice n + 1, diagonal)
            // into (X, R) as (hi, lo)
            const int q = (n + 1) & 1;
            for (int e = tid; e < MP * MP; e += NT) {
                const int i = e / MP, j = e - i * MP;
                sm.Gh[e] = gn[e];
                sm.Gl[e] = gn[MP * MP + e];
                float2 fh = make_float2(0.f, 0.f), fl = make_float2(0.f, 0.f);
                if (i < M && j < M) {
                    float2 th, tl, vih = sm.vh[q][i], vil = sm.vl[q][i];
                    vih.y = -vih.y;
                    vil.y = -vil.y;
                    cdf_mul(vih, vil, Gs[e], Gs[MP * MP + e], th, tl);
                    cdf_mul(th, tl, sm.vh[q][j], sm.vl[q][j], fh, fl);
                }
                sm.X[e] = fh;
                sm.R[e] = fl;
            }
            __syncthreads();
            float2 yh[RT][RT], yl[RT][RT];
            gemm_df_tile<MP>(sm.Gh, sm.Gl, sm.X, sm.R, M, yh, yl);   // g_n F
            __syncthreads();
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < RT; ++b) {
                    const int e = (ty + 16 * a) * MP + tx + 16 * b;
                    float2 h = yh[a][b], l = yl[a][b];
                    two_sum(h.x, l.x, h.x, l.x);
                    two_sum(h.y, l.y, h.y, l.y);
                    sm.X[e] = h;
                    sm.R[e] = l;
                }
            __syncthreads();
            gemm_df_tile<MP>(sm.X, sm.R, sm.Gh, sm.Gl, M, yh, yl);   // (g_n F) g_n
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < RT; ++b) {
                    const int i = ty + 16 * a, j = tx + 16 * b, e = i * MP + j;
                    float2 h = sm.Gh[e], l = sm.Gl[e];
                    float2 zh = yh[a][b], zl = yl[a][b];
                    two_sum(zh.x, zl.x, zh.x, zl.x);
                    two_sum(zh.y, zl.y, zh.y, zl.y);
                    cdf_add(h, l, zh, zl);
                    Gs[e] = h;
                    Gs[MP * MP + e] = l;
                    if (i == j && i < M)
                        out[(size_t)n * M + i] = -((double)h.y + (double)l.y) / 3.141592653589793;
                }
            __syncthreads();
        }
        if (tid == 0) {
            if (in.T) in.T[ip.out] = T;
            if (in.status) in.status[ip.out] = st;
        }
        __syncthreads();
    }
}

template __global__ void knit_sweep_mixed_kernel<16>(InstDev);
template __global__ void knit_sweep_mixed_kernel<32>(InstDev);
template __global__ void knit_sweep_mixed_kernel<64>(InstDev);
template __global__ void knit_ldos_mixed_kernel<16>(InstDev, int, int, float2 *, double *, long long);
template __global__ void knit_ldos_mixed_kernel<32>(InstDev, int, int, float2 *, double *, long long);
template __global__ void knit_ldos_mixed_kernel<64>(InstDev, int, int, float2 *, double *, long long);

// device workspace of the mixed LDOS kernel per CTA: ceil(Lmax / save)
// checkpoints, `save` segment slots and the backward state, each a
// double-float MP x MP matrix
extern "C" size_t knit_ldos_mixed_work_bytes(int Mmax, int Lmax, int save)
{
    const size_t MP = Mmax <= 16 ? 16 : Mmax <= 32 ? 32 : 64;
    return sizeof(float2) * 2 * MP * MP * ((size_t)(Lmax + save - 1) / save + save + 1);
}

template <int MP>
static cudaError_t launch_ldos_mixed(const InstDev *in, int Lmax, int grid, int save, void *work,
                                     double *ldos, long long stride, cudaStream_t stream)
{
    const size_t sm = sizeof(MixedSmem<MP>);
    cudaError_t e = cudaFuncSetAttribute(knit_ldos_mixed_kernel<MP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    knit_ldos_mixed_kernel<MP><<<grid, NT, sm, stream>>>(*in, Lmax, save,
                                                         static_cast<float2 *>(work), ldos, stride);
    return cudaGetLastError();
}

// widths up to 64 with diagonal inter-slice couplings
extern "C" cudaError_t knit_launch_ldos_mixed(const InstDev *in, int Mmax, int Lmax, int grid,
                                              int save, void *work, double *ldos, long long stride,
                                              cudaStream_t stream)
{
    if (Mmax <= 16) return launch_ldos_mixed<16>(in, Lmax, grid, save, work, ldos, stride, stream);
    if (Mmax <= 32) return launch_ldos_mixed<32>(in, Lmax, grid, save, work, ldos, stride, stream);
    if (Mmax <= 64) return launch_ldos_mixed<64>(in, Lmax, grid, save, work, ldos, stride, stream);
    return cudaErrorInvalidValue;
}

extern "C" cudaError_t knit_launch_mixed_tc(const InstDev *in, int grid, cudaStream_t stream);

// Host-side launch helper (the host API lives in knit_api.cu).  Mmax is the
// largest width among the launch's systems; widths 33..64 take the
// tensor-core residual when use_tc is set.
extern "C" cudaError_t knit_launch_mixed_impl(const InstDev *in, int Mmax, int grid, int use_tc,
                                              cudaStream_t stream)
{
    const int M = Mmax;
    if (M <= 16) {
        size_t sm = sizeof(MixedSmem<16>);
        cudaFuncSetAttribute(knit_sweep_mixed_kernel<16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        knit_sweep_mixed_kernel<16><<<grid, NT, sm, stream>>>(*in);
    } else if (M <= 32) {
        size_t sm = sizeof(MixedSmem<32>);
        cudaFuncSetAttribute(knit_sweep_mixed_kernel<32>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        knit_sweep_mixed_kernel<32><<<grid, NT, sm, stream>>>(*in);
    } else if (M <= 64) {
        if (use_tc) return knit_launch_mixed_tc(in, grid, stream);
        size_t sm = sizeof(MixedSmem<64>);
        cudaFuncSetAttribute(knit_sweep_mixed_kernel<64>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        knit_sweep_mixed_kernel<64><<<grid, NT, sm, stream>>>(*in);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

extern "C" int knit_mixed_max_M(void) { return 64; }

// CTAs of the CUDA-core mixed sweep for widths up to Mmax that fit on one SM
// at once (1 for the tensor-core variant, which takes all tensor memory)
extern "C" int knit_mixed_ctas_per_sm(int Mmax, int use_tc)
{
    int n = 1;
    if (Mmax <= 16) {
        const size_t sm = sizeof(MixedSmem<16>);
        cudaFuncSetAttribute(knit_sweep_mixed_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, knit_sweep_mixed_kernel<16>, NT, sm);
    } else if (Mmax <= 32) {
        const size_t sm = sizeof(MixedSmem<32>);
        cudaFuncSetAttribute(knit_sweep_mixed_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, knit_sweep_mixed_kernel<32>, NT, sm);
    } else if (Mmax <= 64 && !use_tc) {
        const size_t sm = sizeof(MixedSmem<64>);
        cudaFuncSetAttribute(knit_sweep_mixed_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, knit_sweep_mixed_kernel<64>, NT, sm);
    }
    return n < 1 ? 1 : n;
}
