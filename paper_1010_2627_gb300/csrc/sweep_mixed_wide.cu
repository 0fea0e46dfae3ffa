// sweep_mixed_wide.cu -- mixed-precision slice sweep for widths 65..128
// (padded MP in {96, 128}), inter-slice couplings diagonal or block-diagonal
// with 4 x 4 blocks (spin x Nambu sites).
//
// Same recursion and arithmetic as sweep_mixed.cu (KNIT user guide Sec. 5.3 D;
// complex64 look-ahead Gauss-Jordan with implicit partial pivoting,
// refinement against a double-float residual with as many Neumann terms as
// max|R_ij| asks for and an FP64 inversion of slices where it cannot
// converge, state g kept as hi + lo, T from G_LL by the unitarity identity),
// laid out for the larger matrices:
//  * one CTA of 512 threads per instance; thread (ty, tx) = (tid / 32, tid % 32)
//    owns rows ty + 16a (a < MP/16) and columns tx + 32b (b < MP/32) of the
//    register tile, so a warp shares one row set and its lanes run along rows
//    (broadcast loads of the state rows, conflict-free shared columns);
//  * the inverse X and the Gauss-Jordan panels (4 columns) live in shared
//    memory; the state (hi, lo), the residual, the series buffers and the
//    FP64 scratch live in a per-CTA workspace in device memory (L2-resident);
//  * the residual and the refinement product are computed in two passes over
//    half the tile rows each to bound registers.

#include "mixed_common.cuh"

using namespace mixed;

namespace {

constexpr int NTW = 512, TYW = 16, TXW = 32;
constexpr int VBMAX = 4;

constexpr int GJW_NB = 4;   // Gauss-Jordan panel width (four rows per lane at MP = 128)

template <int MP>
struct WideSmem {
    float2 X[MP * MP];
    float2 gjU[2 * MP * gj_ust(GJW_NB)];   // Gauss-Jordan panels (two in turn)
    float2 gjV[2 * GJW_NB * MP];
    GJShared<MP> gj;
    double eps[MP];
    float2 vbh[2][MP * VBMAX];   // diagonal blocks of V per parity: [i][kk] = V[i][bi + kk]
    float2 vbl[2][MP * VBMAX];
    double red[NTW / 32];
    unsigned redu[NTW / 32];
    int inst;
    int cur_sys;
};

template <int MP>
struct WideWork {   // per-CTA device workspace
    float2 Gh[MP * MP];   // state g_{n-1} (hi, lo)
    float2 Gl[MP * MP];
    float2 R[MP * MP];    // residual
    float2 S[2][MP * MP]; // further Neumann terms (two buffers in turn); A_n as complex128
                          // on a slice inverted in FP64
    union {
        struct {
            float2 Vh[MP * MP];   // Gv (hi, lo) during the sweep
            float2 Vl[MP * MP];
        } v;
        double2 G[MP * MP];       // G_LL in FP64 for the final trace
    } u;
};

// Gv = V g V^dagger (+ Sigma terms) in double-float from the state (Gh, Gl)
// into (Oh, Ol), for diagonal V (vb = 1) or block-diagonal V with 4 x 4
// blocks (vb = 4)
template <int MP>
__device__ void form_gv_block(const float2 *Gh, const float2 *Gl, float2 *Oh, float2 *Ol,
                              const float2 *vbh, const float2 *vbl, int vb, int M, int n, int L,
                              const double2 *SL, const double2 *SR)
{
    if (vb == 1) {
        for (int e = threadIdx.x; e < MP * MP; e += NTW) {
            const int i = e / MP, j = e - i * MP;
            float2 gh = make_float2(0.f, 0.f), gl = make_float2(0.f, 0.f);
            if (i < M && j < M) {
                if (n > 0) {
                    float2 th, tl;
                    float2 vjh = vbh[j * VBMAX], vjl = vbl[j * VBMAX];
                    vjh.y = -vjh.y;
                    vjl.y = -vjl.y;
                    cdf_mul(Gh[e], Gl[e], vjh, vjl, th, tl);
                    cdf_mul(vbh[i * VBMAX], vbl[i * VBMAX], th, tl, gh, gl);
                } else {
                    const double2 v = SL[(size_t)i * M + j];
                    float a, b, c, d;
                    to_df(v.x, a, b);
                    to_df(v.y, c, d);
                    gh = make_float2(a, c);
                    gl = make_float2(b, d);
                }
                if (n == L - 1) {
                    const double2 v = SR[(size_t)i * M + j];
                    float a, b, c, d;
                    to_df(v.x, a, b);
                    to_df(v.y, c, d);
                    cdf_add(gh, gl, make_float2(a, c), make_float2(b, d));
                }
            }
            Oh[e] = gh;
            Ol[e] = gl;
        }
        return;
    }
    constexpr int VB = VBMAX;   // vb == 4: out of place, one element per thread
    for (int e = threadIdx.x; e < MP * MP; e += NTW) {
        const int i = e / MP, j = e - i * MP;
        float2 gh = make_float2(0.f, 0.f), gl = make_float2(0.f, 0.f);
        if (i < M && j < M) {
            const int bi = (i / VB) * VB, bj = (j / VB) * VB;
            if (n > 0) {
                // u_l = sum_k V[i][bi+k] g[bi+k][bj+l];  Gv_ij = sum_l u_l conj(V[j][bj+l])
#pragma unroll
                for (int ll = 0; ll < VB; ++ll) {
                    float2 uh = make_float2(0.f, 0.f), ul = make_float2(0.f, 0.f);
#pragma unroll
                    for (int kk = 0; kk < VB; ++kk) {
                        const int g_e = (bi + kk) * MP + bj + ll;
                        float2 ph, pl;
                        cdf_mul(vbh[i * VBMAX + kk], vbl[i * VBMAX + kk], Gh[g_e], Gl[g_e], ph, pl);
                        cdf_add(uh, ul, ph, pl);
                    }
                    float2 vh = vbh[j * VBMAX + ll], vl = vbl[j * VBMAX + ll];
                    vh.y = -vh.y;
                    vl.y = -vl.y;
                    float2 ph, pl;
                    cdf_mul(uh, ul, vh, vl, ph, pl);
                    cdf_add(gh, gl, ph, pl);
                }
            } else {
                const double2 v = SL[(size_t)i * M + j];
                float a, b, c, d;
                to_df(v.x, a, b);
                to_df(v.y, c, d);
                gh = make_float2(a, c);
                gl = make_float2(b, d);
            }
            if (n == L - 1) {
                const double2 v = SR[(size_t)i * M + j];
                float a, b, c, d;
                to_df(v.x, a, b);
                to_df(v.y, c, d);
                cdf_add(gh, gl, make_float2(a, c), make_float2(b, d));
            }
        }
        Oh[e] = gh;
        Ol[e] = gl;
    }
}

// residual rows ty + 16 (A0 + a), a < NA, in double-float; written to R
template <int MP, int A0, int NA>
__device__ __forceinline__ float residual_pass(const SysDev &s, const float2 *X, const float2 *Gh,
                                               const float2 *Gl, const double *eps, float2 *R)
{
    float rloc = 0.f;   // largest |Re|, |Im| written, returned
    constexpr int RB = MP / TXW;
    const int tid = threadIdx.x, ty = tid / TXW, tx = tid % TXW;
    const int M = s.M;
    float2 ah[NA][RB], al[NA][RB];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            ah[a][b] = make_float2(0.f, 0.f);
            al[a][b] = make_float2(0.f, 0.f);
        }
    for (int k = 0; k < M; ++k) {
        float2 gh[NA], gl[NA], xv[RB];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int i = ty + TYW * (A0 + a);
            gh[a] = Gh[i * MP + k];
            gl[a] = Gl[i * MP + k];
        }
#pragma unroll
        for (int b = 0; b < RB; ++b) xv[b] = X[k * MP + tx + TXW * b];
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                dot2_acc(gh[a].x, gl[a].x, xv[b].x, ah[a][b].x, al[a][b].x);
                dot2_acc(-gh[a].y, -gl[a].y, xv[b].y, ah[a][b].x, al[a][b].x);
                dot2_acc(gh[a].x, gl[a].x, xv[b].y, ah[a][b].y, al[a][b].y);
                dot2_acc(gh[a].y, gl[a].y, xv[b].x, ah[a][b].y, al[a][b].y);
            }
    }
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int i = ty + TYW * (A0 + a);
        if (i < M) {
            float dh, dl;
            to_df(eps[i], dh, dl);
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                const float2 xij = X[i * MP + tx + TXW * b];
                dot2_acc(-dh, -dl, xij.x, ah[a][b].x, al[a][b].x);
                dot2_acc(-dh, -dl, xij.y, ah[a][b].y, al[a][b].y);
            }
            for (int c = s.h0_rowptr[i]; c < s.h0_rowptr[i + 1]; ++c) {
                const int col = s.h0_col[c];
                const double2 h = s.h0_val[c];
                float hxh, hxl, hyh, hyl;
                to_df(h.x, hxh, hxl);
                to_df(h.y, hyh, hyl);
#pragma unroll
                for (int b = 0; b < RB; ++b) {
                    const float2 xc = X[col * MP + tx + TXW * b];
                    dot2_acc(hxh, hxl, xc.x, ah[a][b].x, al[a][b].x);
                    dot2_acc(-hyh, -hyl, xc.y, ah[a][b].x, al[a][b].x);
                    dot2_acc(hxh, hxl, xc.y, ah[a][b].y, al[a][b].y);
                    dot2_acc(hyh, hyl, xc.x, ah[a][b].y, al[a][b].y);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int j = tx + TXW * b;
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
            R[i * MP + j] = r;
            rloc = fmaxf(rloc, fmaxf(fabsf(r.x), fabsf(r.y)));
        }
    }
    return rloc;
}

// rows RA0 .. RA0+NRA-1 of the thread's tile of acc into S (row stride MP)
template <int MP, int RA0, int NRA>
__device__ __forceinline__ void store_tile(const float2 (&acc)[NRA][MP / TXW], float2 *S)
{
    const int tid = threadIdx.x, ty = tid / TXW, tx = tid % TXW;
#pragma unroll
    for (int a = 0; a < NRA; ++a)
#pragma unroll
        for (int b = 0; b < MP / TXW; ++b) S[(ty + TYW * (RA0 + a)) * MP + tx + TXW * b] = acc[a][b];
}

}  // namespace

template <int MP>
__global__ void __launch_bounds__(NTW, 1)
knit_sweep_mixed_wide_kernel(InstDev in, WideWork<MP> *work)
{
    constexpr int RA = MP / TYW, RB = MP / TXW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WideSmem<MP> &sm = *reinterpret_cast<WideSmem<MP> *>(smem_raw);
    WideWork<MP> &wk = work[blockIdx.x];
    const int tid = threadIdx.x, ty = tid / TXW, tx = tid % TXW;
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
        const int M = s.M, L = s.L, vb = s.vb;
        const size_t MM = (size_t)M * M;
        if (reload) {
            for (int q = 0; q < 2; ++q)
                for (int e = tid; e < MP * VBMAX; e += NTW) {
                    const int i = e / VBMAX, kk = e - i * VBMAX;
                    double2 v = make_double2(0.0, 0.0);
                    if (i < M && kk < vb) {
                        const int col = (i / vb) * vb + kk;
                        v = s.V[(size_t)(q % s.Vperiod) * MM + (size_t)i * M + col];
                    }
                    float hx, lx, hy, ly;
                    to_df(v.x, hx, lx);
                    to_df(v.y, hy, ly);
                    sm.vbh[q][e] = make_float2(hx, hy);
                    sm.vbl[q][e] = make_float2(lx, ly);
                }
            if (tid == 0) sm.cur_sys = si;
            __syncthreads();
        }
        const InstParams ip = inst_params(in, inst, M);
        int st = ip.st;

        for (int n = 0; n < L && st == ST_OK; ++n) {
            slice_diag<MP, NTW>(sm.eps, s, ip.ms, ip.W, ip.E, n);
            form_gv_block<MP>(wk.Gh, wk.Gl, wk.u.v.Vh, wk.u.v.Vl, sm.vbh[n & 1], sm.vbl[n & 1], vb,
                              M, n, L, ip.SL, ip.SR);
            __syncthreads();
            // X = fl32(D - Gv_hi): diagonal part, then sparse H0 rows
            for (int e = tid; e < MP * MP; e += NTW) {
                const int i = e / MP, j = e - i * MP;
                float2 v;
                if (i < M && j < M) {
                    const float2 g = wk.u.v.Vh[e];
                    v = make_float2(-g.x, -g.y);
                    if (i == j) v.x += (float)sm.eps[i];
                } else {
                    v = make_float2(i == j ? 1.f : 0.f, 0.f);
                }
                sm.X[e] = v;
            }
            __syncthreads();
            for (int i = tid; i < M; i += NTW)
                for (int c = s.h0_rowptr[i]; c < s.h0_rowptr[i + 1]; ++c) {
                    const double2 h = s.h0_val[c];
                    float2 &v = sm.X[i * MP + s.h0_col[c]];
                    v.x -= (float)h.x;
                    v.y -= (float)h.y;
                }
            __syncthreads();
            st = gj_lookahead<MP, NTW, TYW, TXW, GJW_NB>(sm.X, M, sm.gjU, sm.gjV, sm.gj);
            if (st != ST_OK) break;
            {
                float2 x[RA][RB];
#pragma unroll
                for (int a = 0; a < RA; ++a)
#pragma unroll
                    for (int b = 0; b < RB; ++b) x[a][b] = sm.X[(ty + TYW * a) * MP + tx + TXW * b];
                store_inverse<MP, TYW, TXW>(x, M, sm.gj, sm.X);
            }
            float rloc = residual_pass<MP, 0, 4>(s, sm.X, wk.u.v.Vh, wk.u.v.Vl, sm.eps, wk.R);
            rloc = fmaxf(rloc, residual_pass<MP, 4, RA - 4>(s, sm.X, wk.u.v.Vh, wk.u.v.Vl, sm.eps,
                                                            wk.R));
            // further Neumann terms where A_n is ill-conditioned (two buffers in turn)
            const float rmax = block_max_nonneg<NTW>(rloc, sm.redu);
            if (refinement_fails(rmax, M)) {
                // near-singular A_n: this slice in FP64, in the two series
                // buffers (contiguous), scratch in the residual buffer
                double2 *const A64 = reinterpret_cast<double2 *>(wk.S[0]);
                fallback_form_a(A64, wk.u.v.Vh, wk.u.v.Vl, MP, M, sm.eps, s);
                st = gj_invert64(A64, M, fallback_scratch(wk.R, M));
                if (st != ST_OK) break;
                fallback_store_g(A64, wk.Gh, wk.Gl, MP, MP, M);
                continue;
            }
            const int nx = neumann_terms(rmax, M);
            const float2 *S = wk.R;
            for (int t = 0; t < nx; ++t) {
                float2 *const So = wk.S[t & 1];
                {
                    float2 acc[4][RB];
                    neumann_tile<MP, MP, TYW, TXW, 0, 4>(wk.R, S, acc, M);
                    store_tile<MP, 0, 4>(acc, So);
                }
                {
                    float2 acc[RA - 4][RB];
                    neumann_tile<MP, MP, TYW, TXW, 4, RA - 4>(wk.R, S, acc, M);
                    store_tile<MP, 4, RA - 4>(acc, So);
                }
                __syncthreads();
                S = So;
            }
            if (rmax > EXACT_RMAX) {
                refine_exact<MP, MP, TYW, TXW, 0, 4>(sm.X, S, wk.Gh, wk.Gl, M);
                refine_exact<MP, MP, TYW, TXW, 4, RA - 4>(sm.X, S, wk.Gh, wk.Gl, M);
            } else {
                refine<MP, MP, TYW, TXW, 0, 4>(sm.X, S, wk.Gh, wk.Gl, M);
                refine<MP, MP, TYW, TXW, 4, RA - 4>(sm.X, S, wk.Gh, wk.Gl, M);
            }
            __syncthreads();
        }

        double T = 0.0;
        if (st == ST_OK) {
            T = ward_T<MP, NTW>(wk.Gh, wk.Gl, wk.u.G, ip.SR, M, sm.red);
            if (in.GLL) store_gll<MP, NTW>(wk.u.G, M, in.GLL + (size_t)ip.out * M * M);
            if (!isfinite(T)) st = ST_NONFINITE;
        }
        if (tid == 0) {
            in.T[ip.out] = T;
            if (in.status) in.status[ip.out] = st;
        }
        __syncthreads();
    }
}

template __global__ void knit_sweep_mixed_wide_kernel<96>(InstDev, WideWork<96> *);
template __global__ void knit_sweep_mixed_wide_kernel<128>(InstDev, WideWork<128> *);

// bytes of device workspace per CTA for width Mmax
extern "C" size_t knit_mixed_wide_work_bytes(int Mmax)
{
    return Mmax <= 96 ? sizeof(WideWork<96>) : sizeof(WideWork<128>);
}

extern "C" cudaError_t knit_launch_mixed_wide(const InstDev *in, int Mmax, int grid, void *work,
                                              cudaStream_t stream)
{
    if (Mmax <= 96) {
        const size_t sm = sizeof(WideSmem<96>);
        cudaError_t e = cudaFuncSetAttribute(knit_sweep_mixed_wide_kernel<96>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        knit_sweep_mixed_wide_kernel<96><<<grid, NTW, sm, stream>>>(*in,
                                                                     (WideWork<96> *)work);
    } else if (Mmax <= 128) {
        const size_t sm = sizeof(WideSmem<128>);
        cudaError_t e = cudaFuncSetAttribute(knit_sweep_mixed_wide_kernel<128>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        knit_sweep_mixed_wide_kernel<128><<<grid, NTW, sm, stream>>>(*in,
                                                                       (WideWork<128> *)work);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
