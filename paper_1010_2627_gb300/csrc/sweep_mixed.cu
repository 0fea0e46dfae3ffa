// sweep_mixed.cu -- the slice sweep in mixed precision (complex64 inversion,
// double-float refinement), for padded widths MP in {16, 32, 64}.
//
// Per slice n, with the state g_{n-1} carried as hi + lo complex64 pairs
// (KNIT user guide Sec. 5.3 D knitting in slice form; Eq. 2 by block
// elimination):
//   1. Gv = V_n g_{n-1} V_n^dagger (+ Sigma_L at n = 0, + Sigma_R at n = L-1)
//      formed in double-float, so that A_n = D_n - Gv with D_n = E - H_n;
//   2. X = fl32(D_n - Gv_hi) inverted by Gauss-Jordan with partial pivoting
//      (largest |Re|+|Im|, lowest row on ties) in registers, 256 threads each
//      holding a (MP/16) x (MP/16) tile;
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
// atomic counter.

#include "knit_common.cuh"

namespace {

constexpr int NT = 256;   // 16 x 16 thread tile grid

template <int MP>
struct MixedSmem {
    float2 X[MP * MP];     // inverse of the complex64 A_n (columns in final order)
    float2 R[MP * MP];     // residual (X and R together hold G_LL as complex128 at the end)
    float2 Gh[MP * MP];    // g (hi) / Gv (hi)
    float2 Gl[MP * MP];    // g (lo) / Gv (lo)
    float2 H0f[MP * MP];   // complex64 copy of H0 for forming X
    float2 col[2][MP];
    float2 rowk[2][MP];
    float2 rowp[2][MP];
    float val[2][MP];
    double eps[MP];        // E - onsite for the current slice
    float2 vh[2][MP];      // diagonal of V (per parity), hi
    float2 vl[2][MP];      // lo
    int perm[MP];
    int pos[MP];
    int used[MP];
    double red[NT / 32];
    int flag;
    int inst;
};

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

// complex double-float product (a) * (b); a = (arh + arl, aih + ail)
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

}  // namespace

template <int MP>
__global__ void __launch_bounds__(NT, 1)
knit_sweep_mixed_kernel(SysDev s, InstDev in)
{
    constexpr int RT = MP / 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MixedSmem<MP> &sm = *reinterpret_cast<MixedSmem<MP> *>(smem_raw);
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int lane = tid & 31;
    const int M = s.M, L = s.L;
    const size_t MM = (size_t)M * M;

    // per-launch constants: H0 as complex64, diagonal of V as double-float
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
    __syncthreads();

    for (;;) {
        if (tid == 0) sm.inst = atomicAdd(in.queue, 1);
        __syncthreads();
        const int inst = sm.inst;
        __syncthreads();
        if (inst >= in.n) break;
        const int ie = inst / in.nS;
        const double E = in.E[ie];
        const uint64_t ms = knit_mix64(in.seeds ? in.seeds[inst - ie * in.nS] : 0ull);
        const double W = in.W;
        const double2 *SL = in.sigL + (size_t)ie * MM;
        const double2 *SR = in.sigR + (size_t)ie * MM;
        int st = in.lstatus ? in.lstatus[ie] : ST_OK;

        for (int n = 0; n < L && st == ST_OK; ++n) {
            // ---- slice diagonal E - onsite (double)
            for (int i = tid; i < MP; i += NT) {
                double d = 0.0;
                if (i < M) {
                    double o = 0.0;
                    if (s.onsite) o = s.onsite[(size_t)n * M + i];
                    else if (W != 0.0) o = s.sign[i % s.block] * knit_disorder(ms, n, i / s.block, W);
                    d = E - o;
                }
                sm.eps[i] = d;
            }
            // ---- 1. Gv in place over (Gh, Gl)
            {
                const int q = n & 1;
                for (int e = tid; e < MP * MP; e += NT) {
                    int i = e / MP, j = e - i * MP;
                    float2 gh = make_float2(0.f, 0.f), gl = make_float2(0.f, 0.f);
                    if (i < M && j < M) {
                        if (n > 0) {
                            // v_i g_ij conj(v_j)
                            float2 th, tl;
                            float2 vjh = sm.vh[q][j], vjl = sm.vl[q][j];
                            vjh.y = -vjh.y;
                            vjl.y = -vjl.y;
                            cdf_mul(sm.Gh[e], sm.Gl[e], vjh, vjl, th, tl);
                            cdf_mul(sm.vh[q][i], sm.vl[q][i], th, tl, gh, gl);
                        }
                        if (n == 0) {
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
                    sm.Gh[e] = gh;
                    sm.Gl[e] = gl;
                }
            }
            __syncthreads();

            // ---- 2. X = fl32(D - Gv_hi), Gauss-Jordan in registers
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
            // Gauss-Jordan with implicit partial pivoting: no rows are moved; the
            // pivot of column k is the largest |Re|+|Im| among rows not yet used
            // (lowest row on ties).  Column k and the pivot row are zeroed in
            // registers after staging, so every element then takes the same
            // update x -= c_i r_j (c_p = -1, r_k = 1/pivot).  At the end
            // A^{-1}[k][P[k']] = x[P[k]][k'] with P[k] the pivot row of step k.
            for (int i = tid; i < MP; i += NT) sm.used[i] = 0;
            __syncthreads();
            for (int k = 0; k < M; ++k) {
                const int q = k & 1, kt = k & 15, kb = k >> 4;
                // S1: stage column k and the pivot candidates, zero column k
                if (tx == kt) {
#pragma unroll
                    for (int a = 0; a < RT; ++a) {
                        float2 v = x[a][0];
#pragma unroll
                        for (int b = 1; b < RT; ++b)
                            if (b == kb) v = x[a][b];
#pragma unroll
                        for (int b = 0; b < RT; ++b)
                            if (b == kb) x[a][b] = make_float2(0.f, 0.f);
                        const int i = ty + 16 * a;
                        sm.col[q][i] = v;
                        sm.val[q][i] = (i < M && !sm.used[i]) ? cabs1f(v) : -1.f;
                    }
                }
                __syncthreads();
                // S2: every warp finds the pivot row p; its owners stage and zero it
                float best = -1.f;
                int p = MP;
                for (int i = lane; i < MP; i += 32) {
                    float v = sm.val[q][i];
                    if (v > best) { best = v; p = i; }
                }
                warp_argmaxf(best, p);
                if (best <= 0.f) {   // exact zero pivot (or no candidate)
                    st = ST_SINGULAR;
                    break;
                }
                if (ty == (p & 15)) {
                    const int pa = p >> 4;
#pragma unroll
                    for (int a = 0; a < RT; ++a) {
                        if (a != pa) continue;
#pragma unroll
                        for (int b = 0; b < RT; ++b) {
                            sm.rowp[q][tx + 16 * b] = x[a][b];
                            x[a][b] = make_float2(0.f, 0.f);
                        }
                    }
                }
                if (tid == 0) {
                    sm.perm[k] = p;
                    sm.used[p] = 1;
                }
                __syncthreads();
                // S3: uniform rank-1 update
                const float2 pinv = crcpf(sm.col[q][p]);
                float2 rs[RT];
#pragma unroll
                for (int b = 0; b < RT; ++b) {
                    const int j = tx + 16 * b;
                    rs[b] = (j == k) ? pinv : cmulf(sm.rowp[q][j], pinv);
                }
#pragma unroll
                for (int a = 0; a < RT; ++a) {
                    const int i = ty + 16 * a;
                    const float2 ci = (i == p) ? make_float2(-1.f, 0.f) : sm.col[q][i];
#pragma unroll
                    for (int b = 0; b < RT; ++b) x[a][b] = cfmsf(ci, rs[b], x[a][b]);
                }
            }
            if (__syncthreads_or(st != ST_OK)) { st = ST_SINGULAR; break; }
            // row r of x is row Pinv[r] of the inverse, column c is column P[c]
            for (int k = tid; k < M; k += NT) sm.pos[sm.perm[k]] = k;
            __syncthreads();
#pragma unroll
            for (int a = 0; a < RT; ++a)
#pragma unroll
                for (int b = 0; b < RT; ++b) {
                    const int i = ty + 16 * a, c = tx + 16 * b;
                    if (i < M && c < M) sm.X[sm.pos[i] * MP + sm.perm[c]] = x[a][b];
                    else sm.X[i * MP + c] = x[a][b];
                }
            __syncthreads();

            // ---- 3. residual R = I - D X + Gv X in double-float
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
                    }
            }
            __syncthreads();

            // ---- 4. g = X + X R, kept as hi + lo
            {
                float2 acc[RT][RT];
#pragma unroll
                for (int a = 0; a < RT; ++a)
#pragma unroll
                    for (int b = 0; b < RT; ++b) acc[a][b] = make_float2(0.f, 0.f);
                for (int k = 0; k < M; ++k) {
                    float2 xa[RT], rb[RT];
#pragma unroll
                    for (int a = 0; a < RT; ++a) xa[a] = sm.X[(ty + 16 * a) * MP + k];
#pragma unroll
                    for (int b = 0; b < RT; ++b) rb[b] = sm.R[k * MP + tx + 16 * b];
#pragma unroll
                    for (int a = 0; a < RT; ++a)
#pragma unroll
                        for (int b = 0; b < RT; ++b) acc[a][b] = cfmaf(xa[a], rb[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < RT; ++a)
#pragma unroll
                    for (int b = 0; b < RT; ++b) {
                        const int e = (ty + 16 * a) * MP + tx + 16 * b;
                        float2 xv = sm.X[e];
                        float hx, lx, hy, ly;
                        two_sum(xv.x, acc[a][b].x, hx, lx);
                        two_sum(xv.y, acc[a][b].y, hy, ly);
                        sm.Gh[e] = make_float2(hx, hy);
                        sm.Gl[e] = make_float2(lx, ly);
                    }
            }
            __syncthreads();
        }

        // ---- transmission from G_LL by the unitarity identity, in FP64
        double T = 0.0;
        if (st == ST_OK) {
            double2 *G = reinterpret_cast<double2 *>(sm.X);   // X and R: MP*MP double2
            for (int e = tid; e < MP * MP; e += NT) {
                float2 h = sm.Gh[e], l = sm.Gl[e];
                G[e] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
            }
            __syncthreads();
            double t = 0.0;
            for (int e = tid; e < M * M; e += NT) {
                const int i = e / M, j = e - i * M;
                // Gamma_R[i][j]
                double2 d = csub(SR[(size_t)i * M + j], cconj(SR[(size_t)j * M + i]));
                double2 gij = make_double2(-d.y, d.x);
                // i (G - G^dagger)[j][i]
                double2 u = csub(G[j * MP + i], cconj(G[i * MP + j]));
                double2 a = make_double2(-u.y, u.x);
                t += gij.x * a.x - gij.y * a.y;
                // Y_ij = (Gamma_R G)_ij, Z_ij = (G Gamma_R)_ij, accumulate Re(Y conj(Z))
                double2 y = make_double2(0.0, 0.0), z = make_double2(0.0, 0.0);
                for (int k = 0; k < M; ++k) {
                    double2 d1 = csub(SR[(size_t)i * M + k], cconj(SR[(size_t)k * M + i]));
                    double2 d2 = csub(SR[(size_t)k * M + j], cconj(SR[(size_t)j * M + k]));
                    y = cfma(make_double2(-d1.y, d1.x), G[k * MP + j], y);
                    z = cfma(G[i * MP + k], make_double2(-d2.y, d2.x), z);
                }
                t -= y.x * z.x + y.y * z.y;
            }
            T = block_sum(t, sm.red);
            if (!isfinite(T)) st = ST_NONFINITE;
        }
        if (tid == 0) {
            in.T[inst] = T;
            if (in.status) in.status[inst] = st;
        }
        __syncthreads();
    }
}

template __global__ void knit_sweep_mixed_kernel<16>(SysDev, InstDev);
template __global__ void knit_sweep_mixed_kernel<32>(SysDev, InstDev);
template __global__ void knit_sweep_mixed_kernel<64>(SysDev, InstDev);

// Host-side launch helper (the host API lives in knit_api.cu).
extern "C" cudaError_t knit_launch_mixed(const SysDev *s, const InstDev *in, int grid,
                                         cudaStream_t stream)
{
    const int M = s->M;
    if (M <= 16) {
        size_t sm = sizeof(MixedSmem<16>);
        cudaFuncSetAttribute(knit_sweep_mixed_kernel<16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        knit_sweep_mixed_kernel<16><<<grid, NT, sm, stream>>>(*s, *in);
    } else if (M <= 32) {
        size_t sm = sizeof(MixedSmem<32>);
        cudaFuncSetAttribute(knit_sweep_mixed_kernel<32>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        knit_sweep_mixed_kernel<32><<<grid, NT, sm, stream>>>(*s, *in);
    } else if (M <= 64) {
        size_t sm = sizeof(MixedSmem<64>);
        cudaFuncSetAttribute(knit_sweep_mixed_kernel<64>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        knit_sweep_mixed_kernel<64><<<grid, NT, sm, stream>>>(*s, *in);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

extern "C" int knit_mixed_max_M(void) { return 64; }
