// sweep_mixed.cu -- the slice sweep in mixed precision with the residual on
// CUDA cores (complex64 inversion, double-float refinement), padded widths
// MP in {16, 32, 64}.
//
// Per slice n, with the state g_{n-1} carried as hi + lo complex64 pairs
// (KNIT user guide Sec. 5.3 D knitting in slice form; Eq. 2 by block
// elimination):
//   1. Gv = V_n g_{n-1} V_n^dagger (+ Sigma_L at n = 0, + Sigma_R at n = L-1)
//      formed in double-float, so that A_n = D_n - Gv with D_n = E - H_n;
//   2. X = fl32(D_n - Gv_hi) inverted by Gauss-Jordan with implicit partial
//      pivoting in registers;
//   3. residual R = I - A_n X accumulated with error-free products and sums
//      (TwoProduct / TwoSum, "Dot2" of Ogita, Rump & Oishi 2005), using the
//      exact D_n and both words of Gv, then rounded to complex64;
//   4. one refinement step g_n = X + X R, kept as hi + lo (TwoSum).
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
    float2 vh[2][MP];      // diagonal of V (per parity), hi
    float2 vl[2][MP];      // lo
    double red[NT / 32];
    unsigned redu[NT / 32];
    int inst;
    int cur_sys;
};

}  // namespace

template <int MP>
__global__ void __launch_bounds__(NT, 1)
knit_sweep_mixed_kernel(InstDev in)
{
    constexpr int RT = MP / 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MixedSmem<MP> &sm = *reinterpret_cast<MixedSmem<MP> *>(smem_raw);
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
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
        const size_t MM = (size_t)M * M;
        if (reload) {
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
            if (tid == 0) sm.cur_sys = si;
            __syncthreads();
        }
        const InstParams ip = inst_params(in, inst, M);
        const double E = ip.E;
        const uint64_t ms = ip.ms;
        const double W = ip.W;
        const double2 *SL = ip.SL;
        const double2 *SR = ip.SR;
        int st = ip.st;

        for (int n = 0; n < L && st == ST_OK; ++n) {
            slice_diag<MP>(sm.eps, s, ms, W, E, n);
            form_gv<MP>(sm.Gh, sm.Gl, sm.vh, sm.vl, M, n, L, SL, SR);
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
                if (st != ST_OK) break;
#pragma unroll
                for (int a = 0; a < RT; ++a)
#pragma unroll
                    for (int b = 0; b < RT; ++b) x[a][b] = sm.X[(ty + 16 * a) * MP + tx + 16 * b];
            } else {
                st = gj_regs<MP>(x, M, sm.gj);
                if (st != ST_OK) break;
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
                if (st != ST_OK) break;
                fallback_store_g(A64, sm.Gh, sm.Gl, MP, MP, M);
                continue;
            }
            const int nx = neumann_terms(rmax, M);
            float2 *const S = nx ? sm.S : sm.R;
            neumann_inplace<MP, MP, 16, 16>(sm.R, S, M, nx);
            if (rmax > EXACT_RMAX)
                refine_exact<MP>(sm.X, S, sm.Gh, sm.Gl, M);
            else
                refine<MP>(sm.X, S, sm.Gh, sm.Gl, M);
            __syncthreads();
        }

        double T = 0.0;
        if (st == ST_OK) {
            T = ward_T<MP>(sm.Gh, sm.Gl, reinterpret_cast<double2 *>(sm.X), SR, M, sm.red);
            if (!isfinite(T)) st = ST_NONFINITE;
        }
        if (tid == 0) {
            in.T[ip.out] = T;
            if (in.status) in.status[ip.out] = st;
        }
        __syncthreads();
    }
}

template __global__ void knit_sweep_mixed_kernel<16>(InstDev);
template __global__ void knit_sweep_mixed_kernel<32>(InstDev);
template __global__ void knit_sweep_mixed_kernel<64>(InstDev);

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
