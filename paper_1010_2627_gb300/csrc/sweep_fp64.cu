// sweep_fp64.cu -- the slice sweep in complex128 (the plain FP64 path).
//
// One CTA walks one instance (energy, disorder seed, system) at a time and
// takes the next one from an atomic counter over a cost-ordered queue.  Per
// slice n (KNIT user guide Sec. 5.3 D, knitting in slice form; Eq. 2 by block
// elimination):
//     A_0 = E - H_0 - Sigma_L,   A_n = E - H_n - V_n g_{n-1} V_n^dagger (n >= 1),
//     A_{L-1} additionally - Sigma_R,
//     g_n = A_n^{-1}                                   (Gauss-Jordan, FP64)
//     G_{0,0} = g_0,  G_{0,n} = G_{0,n-1} V_n^dagger g_n
// and at the end the Sec. 2.3 transmission
//     T = Re Tr[Gamma_L G_{0,L-1} Gamma_R G_{0,L-1}^dagger],  Gamma = i(Sigma - Sigma^dagger).
// The LDOS kernel adds the sewing pass (Sec. 5.3 D):
//     G_{L-1,L-1} = g_{L-1},  G_{n,n} = g_n + g_n V_{n+1}^dagger G_{n+1,n+1} V_{n+1} g_n,
//     LDOS[n][x] = -Im G_{n,n}[x][x] / pi,
// with the forward g_n kept every `save` slices (KNIT's saving_level) and
// the slices in between recomputed segment by segment.
//
// Matrices live in shared memory when three (four for LDOS) Mmax x Mmax
// complex128 buffers fit, else in a per-CTA global workspace; Mmax is the
// largest width among the launch's systems.

#include "dense_fp64.cuh"

namespace {

struct Bufs {
    double2 *P, *Q, *F, *X;
    GJScratch64 gj;
    double *red;
};

__device__ Bufs carve(int Mmax, double2 *work, int use_smem, int nbuf)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const size_t MM = (size_t)Mmax * Mmax;
    Bufs b;
    unsigned char *p = smem_raw;
    double2 *mat;
    if (use_smem) {
        mat = reinterpret_cast<double2 *>(p);
        p += sizeof(double2) * MM * nbuf;
    } else {
        mat = work + (size_t)blockIdx.x * MM * nbuf;
    }
    b.P = mat;
    b.Q = mat + MM;
    b.F = mat + 2 * MM;
    b.X = nbuf > 3 ? mat + 3 * MM : nullptr;
    b.gj.row = reinterpret_cast<double2 *>(p);
    p += sizeof(double2) * Mmax;
    b.gj.col = reinterpret_cast<double2 *>(p);
    p += sizeof(double2) * Mmax;
    b.gj.pval = reinterpret_cast<double2 *>(p);
    p += sizeof(double2);
    b.red = reinterpret_cast<double *>(p);
    p += sizeof(double) * 32;
    b.gj.perm = reinterpret_cast<int *>(p);
    p += sizeof(int) * Mmax;
    b.gj.flag = reinterpret_cast<int *>(p);
    p += sizeof(int);
    b.gj.piv = reinterpret_cast<int *>(p);
    return b;
}

// on-site energy of orbital x in slice n
KNIT_DEV double onsite_at(const SysDev &s, uint64_t ms, double W, int n, int x)
{
    if (s.onsite) return s.onsite[(size_t)n * s.M + x];
    if (W == 0.0) return 0.0;
    return s.sign[x % s.block] * knit_disorder(ms, n, x / s.block, W);
}

// A = E - H_n - [Sigma_L | V_n gprev V_n^dagger] - [Sigma_R]
__device__ void form_A(const SysDev &s, int n, double E, uint64_t ms, double W,
                       const double2 *gprev, const double2 *SL, const double2 *SR, double2 *A)
{
    const int M = s.M, L = s.L;
    const double2 *Vn = s.V + (size_t)(n % s.Vperiod) * M * M;
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        int i = e / M, j = e - i * M;
        double2 h = s.H0[e];
        double2 a = make_double2(-h.x, -h.y);
        if (i == j) a.x += E - onsite_at(s, ms, W, n, i);
        if (n == 0) a = csub(a, SL[e]);
        else a = csub(a, vxvd64(Vn, gprev, M, s.vb, i, j));
        if (n == L - 1) a = csub(a, SR[e]);
        A[e] = a;
    }
    __syncthreads();
}

__device__ void copy_mat(const double2 *src, double2 *dst, int M)
{
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) dst[e] = src[e];
    __syncthreads();
}

// C = (A V^dagger) B; for a diagonal V the columns of A are scaled in place
// first (A is the previous G_{0,n-1}, dead after this product)
__device__ void g1_update(double2 *A, const double2 *V, int vb, int band, const double2 *B, double2 *C,
                          int M)
{
    if (vb == 1) {
        for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
            int k = e % M;
            A[e] = cmul(A[e], cconj(V[(size_t)k * M + k]));
        }
        __syncthreads();
        gemm64(A, B, C, M);
    } else {
        gemm64_avd_b(A, V, vb, band, B, C, M);
    }
}

// next instance from the queue (all threads), or -1 when the queue is empty
__device__ int take_instance(const InstDev &in, int *sh)
{
    if (threadIdx.x == 0) {
        int q = atomicAdd(in.queue, 1);
        *sh = q < in.n ? take_position(in, q) : -1;
    }
    __syncthreads();
    int v = *sh;
    __syncthreads();
    return v;
}

// forward sweep: on return P = g_{L-1}, Q = G_{0,L-1}, F free
__device__ int forward(const SysDev &s, const InstParams &ip, Bufs &b, double2 *&P, double2 *&Q,
                       double2 *&F, double2 *ckpt, int save)
{
    const int M = s.M, L = s.L;
    const size_t MM = (size_t)M * M;
    int st = ip.st;
    for (int n = 0; n < L && st == ST_OK; ++n) {
        form_A(s, n, ip.E, ip.ms, ip.W, P, ip.SL, ip.SR, F);
        st = gj_invert64(F, M, b.gj);
        if (st != ST_OK) break;
        if (ckpt && n % save == 0) copy_mat(F, ckpt + (size_t)(n / save) * MM, M);
        if (n == 0) {
            copy_mat(F, Q, M);
        } else {
            const double2 *Vn = s.V + (size_t)(n % s.Vperiod) * MM;
            g1_update(Q, Vn, s.vb, s.vband, F, P, M);   // G_{0,n} = G_{0,n-1} V_n^dagger g_n
            double2 *t = Q;
            Q = P;
            P = t;
        }
        double2 *t = P;   // g_n becomes the previous slice's function
        P = F;
        F = t;
    }
    return st;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" __global__ void __launch_bounds__(256)
knit_sweep_fp64_kernel(InstDev in, int Mmax, double2 *work, int use_smem)
{
    __shared__ int sh_inst;
    Bufs b = carve(Mmax, work, use_smem, 3);
    for (;;) {
        const int inst = take_instance(in, &sh_inst);
        if (inst < 0) break;
        const SysDev s = inst_system(in, inst);
        const InstParams ip = inst_params(in, inst, s.M);
        double2 *P = b.P, *Q = b.Q, *F = b.F;   // P = g_{n-1}, Q = G_{0,n-1}, F free
        int st = forward(s, ip, b, P, Q, F, nullptr, 1);
        double T = 0.0;
        if (st == ST_OK) {
            if (in.GLL) copy_mat(P, in.GLL + (size_t)ip.out * s.M * s.M, s.M);   // G_LL = g_{L-1}
            gemm64_gamma(Q, ip.SR, F, s.M);     // G Gamma_R
            gemm64_nc(F, Q, P, s.M);            // G Gamma_R G^dagger
            T = trace_gamma64(ip.SL, P, s.M, b.red);
            if (!isfinite(T)) st = ST_NONFINITE;
        }
        if (threadIdx.x == 0) {
            in.T[ip.out] = T;
            if (in.status) in.status[ip.out] = st;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Forward sweep with checkpoints + sewing.  ckpt: per CTA ((Lmax + save - 1)/save)
// saved g's followed by `save` segment slots, Mmax*Mmax complex each.  ldos
// receives L*M values per instance at out * ldos_stride.
extern "C" __global__ void __launch_bounds__(256)
knit_ldos_fp64_kernel(InstDev in, int Mmax, int Lmax, double2 *work, int use_smem, double2 *ckpt,
                      int save, double *ldos, long long ldos_stride)
{
    __shared__ int sh_inst;
    Bufs b = carve(Mmax, work, use_smem, 4);
    const int nckmax = (Lmax + save - 1) / save;
    for (;;) {
        const int inst = take_instance(in, &sh_inst);
        if (inst < 0) break;
        const SysDev s = inst_system(in, inst);
        const InstParams ip = inst_params(in, inst, s.M);
        const int M = s.M, L = s.L;
        const size_t MM = (size_t)M * M;
        double2 *cks = ckpt + (size_t)blockIdx.x * (nckmax + save) * Mmax * Mmax;
        double2 *seg = cks + (size_t)((L + save - 1) / save) * MM;
        double *out = ldos + (size_t)ip.out * ldos_stride;
        double2 *P = b.P, *Q = b.Q, *F = b.F;
        int st = forward(s, ip, b, P, Q, F, cks, save);
        double T = 0.0;
        if (st == ST_OK) {
            gemm64_gamma(Q, ip.SR, F, M);
            gemm64_nc(F, Q, b.X, M);
            T = trace_gamma64(ip.SL, b.X, M, b.red);
            if (!isfinite(T)) st = ST_NONFINITE;
        }
        // sewing: G_nn in Q, walking n = L-1 .. 0
        if (st == ST_OK) {
            copy_mat(P, Q, M);   // P holds g_{L-1} = G_{L-1,L-1}
            for (int x = threadIdx.x; x < M; x += blockDim.x)
                out[(size_t)(L - 1) * M + x] = -Q[(size_t)x * M + x].y / 3.141592653589793;
            int seg_lo = -1;   // first slice held in the segment slots
            for (int n = L - 2; n >= 0 && st == ST_OK; --n) {
                const double2 *gn;
                if (n % save == 0) {
                    gn = cks + (size_t)(n / save) * MM;
                } else {
                    const int c = (n / save) * save;
                    if (seg_lo != c) {
                        // recompute g_{c+1} .. g_n from checkpoint g_c
                        copy_mat(cks + (size_t)(c / save) * MM, P, M);
                        const int hi = min(c + save, L);
                        for (int m = c + 1; m < hi && m <= n; ++m) {
                            form_A(s, m, ip.E, ip.ms, ip.W, P, ip.SL, ip.SR, F);
                            st = gj_invert64(F, M, b.gj);
                            if (st != ST_OK) break;
                            copy_mat(F, seg + (size_t)(m - c) * MM, M);
                            double2 *t = P;
                            P = F;
                            F = t;
                        }
                        seg_lo = c;
                        if (st != ST_OK) break;
                    }
                    gn = seg + (size_t)(n - c) * MM;
                }
                const double2 *Vn1 = s.V + (size_t)((n + 1) % s.Vperiod) * MM;
                // F = V^dagger G_{n+1,n+1} V
                for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
                    int i = e / M, j = e - i * M;
                    F[e] = vdxv64(Vn1, Q, M, s.vb, i, j);
                }
                __syncthreads();
                gemm64(gn, F, b.X, M);   // g_n V^dagger G V
                gemm64(b.X, gn, Q, M);   // ... g_n
                for (int e = threadIdx.x; e < M * M; e += blockDim.x) Q[e] = cadd(Q[e], gn[e]);
                __syncthreads();
                for (int x = threadIdx.x; x < M; x += blockDim.x)
                    out[(size_t)n * M + x] = -Q[(size_t)x * M + x].y / 3.141592653589793;
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) {
            if (in.T) in.T[ip.out] = T;
            if (in.status) in.status[ip.out] = st;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Lead-resolved lesser function (Sec. 2.3: G^< = sum_l f_l i G Gamma_l G^+,
// A^l = G Gamma_l G^+) along the sewing pass.  Walking n = L-1 .. 0 with
// Q = G_{n+1,n+1}, R = G_{n+1,L-1} (the column towards the right lead) and
// PR = R Gamma_R:
//     X = V_{n+1} g_n,  Y = G_{n+1,n} = Q X,  Z = G_{n,n+1} = g_n V_{n+1}^dagger Q,
//     G_{n,n} = g_n + Z X,  R' = G_{n,L-1} = g_n V_{n+1}^dagger R,  PR' = R' Gamma_R.
// A = i (G - G^dagger) = A^L + A^R gives the left-injected part from the
// right-injected one, A^R = R Gamma_R R'^dagger (blocks (n+1, n) and (n, n)):
//     rhoR[n][x] = A^R_nn[x][x] / 2pi,   rhoL[n][x] = -Im G_nn[x][x] / pi - rhoR[n][x],
//     jx[n][x]   = sum_{y in block(x)} -2 Im[(V_{n+1}^dagger)_xy A^L_{n+1,n}[y][x]],
//     jt[n][e]   = -2 Im[H0_xy A^L_nn[y][x]] for the e-th edge x < y of H0
// (bond currents carried by states injected from the left lead, positive
// from x to y; Sec. 2.3 local currents).  Work: 8 Mmax^2 per CTA in global
// memory; checkpoints as for the LDOS kernel.
__device__ double2 dot_conj(const double2 *a, const double2 *b, int M)
{
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < M; ++k) acc = cfma(a[k], cconj(b[k]), acc);
    return acc;
}

__device__ void lesser_slice_out(const SysDev &s, int n, const double2 *Gnn, const double2 *Rn,
                                 const double2 *PRn, const int2 *edges, int nedge, double *rhoL,
                                 double *rhoR, double *jt)
{
    const int M = s.M;
    if (rhoL || rhoR)
        for (int x = threadIdx.x; x < M; x += blockDim.x) {
            const double ar = dot_conj(PRn + (size_t)x * M, Rn + (size_t)x * M, M).x;
            const double rr = ar / (2.0 * 3.141592653589793);
            if (rhoR) rhoR[(size_t)n * M + x] = rr;
            if (rhoL) rhoL[(size_t)n * M + x] = -Gnn[(size_t)x * M + x].y / 3.141592653589793 - rr;
        }
    if (jt)
        for (int e = threadIdx.x; e < nedge; e += blockDim.x) {
            const int x = edges[e].x, y = edges[e].y;
            const double2 gyx = Gnn[(size_t)y * M + x], gxy = Gnn[(size_t)x * M + y];
            // A_yx = i (G_yx - conj(G_xy)), A^R_yx = (PR R^dagger)_yx
            const double2 a = make_double2(-(gyx.y + gxy.y), gyx.x - gxy.x);
            const double2 ar = dot_conj(PRn + (size_t)y * M, Rn + (size_t)x * M, M);
            const double2 al = csub(a, ar);
            const double2 h = s.H0[(size_t)x * M + y];
            jt[(size_t)n * nedge + e] = -2.0 * (h.x * al.y + h.y * al.x);
        }
}

extern "C" __global__ void __launch_bounds__(256)
knit_lesser_fp64_kernel(InstDev in, int Mmax, int Lmax, double2 *work, double2 *ckpt, int save,
                        const int2 *edges, int nedge, double *rhoL, double *rhoR, double *jx,
                        double *jt)
{
    __shared__ int sh_inst;
    Bufs b = carve(Mmax, work, 0, 8);
    const size_t MMax = (size_t)Mmax * Mmax;
    double2 *const R0 = b.P + 4 * MMax, *const PR = b.P + 5 * MMax, *const Y = b.P + 6 * MMax,
                   *const Z = b.P + 7 * MMax;
    const int nckmax = (Lmax + save - 1) / save;
    for (;;) {
        const int inst = take_instance(in, &sh_inst);
        if (inst < 0) break;
        const SysDev s = inst_system(in, inst);
        const InstParams ip = inst_params(in, inst, s.M);
        const int M = s.M, L = s.L, vb = s.vb;
        const size_t MM = (size_t)M * M;
        double2 *cks = ckpt + (size_t)blockIdx.x * (nckmax + save) * MMax;
        double2 *seg = cks + (size_t)((L + save - 1) / save) * MM;
        double *oL = rhoL ? rhoL + (size_t)ip.out * L * M : nullptr;
        double *oR = rhoR ? rhoR + (size_t)ip.out * L * M : nullptr;
        double *ox = jx ? jx + (size_t)ip.out * (L - 1) * M : nullptr;
        double *ot = jt ? jt + (size_t)ip.out * L * nedge : nullptr;
        double2 *P = b.P, *Q = b.Q, *F = b.F, *R = R0;
        int st = forward(s, ip, b, P, Q, F, cks, save);
        double T = 0.0;
        if (st == ST_OK) {
            gemm64_gamma(Q, ip.SR, F, M);
            gemm64_nc(F, Q, b.X, M);
            T = trace_gamma64(ip.SL, b.X, M, b.red);
            if (!isfinite(T)) st = ST_NONFINITE;
        }
        if (st == ST_OK) {
            copy_mat(P, Q, M);   // G_{L-1,L-1}
            copy_mat(P, R, M);   // and the right column block G_{L-1,L-1}
            gemm64_gamma(R, ip.SR, PR, M);
            lesser_slice_out(s, L - 1, Q, R, PR, edges, nedge, oL, oR, ot);
            __syncthreads();
            int seg_lo = -1;
            for (int n = L - 2; n >= 0 && st == ST_OK; --n) {
                const double2 *gn;
                if (n % save == 0) {
                    gn = cks + (size_t)(n / save) * MM;
                } else {
                    const int c = (n / save) * save;
                    if (seg_lo != c) {
                        copy_mat(cks + (size_t)(c / save) * MM, P, M);
                        const int hi = min(c + save, L);
                        for (int m = c + 1; m < hi && m <= n; ++m) {
                            form_A(s, m, ip.E, ip.ms, ip.W, P, ip.SL, ip.SR, F);
                            st = gj_invert64(F, M, b.gj);
                            if (st != ST_OK) break;
                            copy_mat(F, seg + (size_t)(m - c) * MM, M);
                            double2 *t = P;
                            P = F;
                            F = t;
                        }
                        seg_lo = c;
                        if (st != ST_OK) break;
                    }
                    gn = seg + (size_t)(n - c) * MM;
                }
                const double2 *V = s.V + (size_t)((n + 1) % s.Vperiod) * MM;
                // X = V g_n and F = V^dagger Q (block-diagonal V, blocks of vb)
                for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
                    const int i = e / M, j = e - i * M, i0 = i - i % vb;
                    double2 x = make_double2(0.0, 0.0), f = make_double2(0.0, 0.0);
                    for (int k = i0; k < i0 + vb; ++k) {
                        x = cfma(V[(size_t)i * M + k], gn[(size_t)k * M + j], x);
                        f = cfma(cconj(V[(size_t)k * M + i]), Q[(size_t)k * M + j], f);
                    }
                    b.X[e] = x;
                    F[e] = f;
                }
                __syncthreads();
                gemm64(Q, b.X, Y, M);    // G_{n+1,n}
                gemm64(gn, F, Z, M);     // G_{n,n+1}
                // F = V^dagger R, then R' = g_n F into P
                for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
                    const int i = e / M, j = e - i * M, i0 = i - i % vb;
                    double2 f = make_double2(0.0, 0.0);
                    for (int k = i0; k < i0 + vb; ++k) f = cfma(cconj(V[(size_t)k * M + i]), R[(size_t)k * M + j], f);
                    F[e] = f;
                }
                __syncthreads();
                gemm64(gn, F, P, M);     // R' = G_{n,L-1}
                if (ox)
                    for (int e = threadIdx.x; e < M * vb; e += blockDim.x) {
                        const int x = e / vb, y = x - x % vb + e % vb;
                        // A^L_{n+1,n}[y][x] = i (Y_yx - conj(Z_xy)) - (PR R'^dagger)_yx
                        const double2 yv = Y[(size_t)y * M + x], zv = Z[(size_t)x * M + y];
                        const double2 a = make_double2(-(yv.y + zv.y), yv.x - zv.x);
                        const double2 al = csub(a, dot_conj(PR + (size_t)y * M, P + (size_t)x * M, M));
                        const double2 vd = cconj(V[(size_t)y * M + x]);   // (V^dagger)_xy
                        const double c = -2.0 * (vd.x * al.y + vd.y * al.x);
                        // one thread per x sums its block (e % vb == 0 collects)
                        Y[(size_t)y * M + x] = make_double2(c, 0.0);
                    }
                __syncthreads();
                if (ox)
                    for (int x = threadIdx.x; x < M; x += blockDim.x) {
                        double sum = 0.0;
                        for (int y = x - x % vb; y < x - x % vb + vb; ++y) sum += Y[(size_t)y * M + x].x;
                        ox[(size_t)n * M + x] = sum;
                    }
                // G_{n,n} = g_n + Z X into Q; PR' = R' Gamma_R
                gemm64(Z, b.X, Q, M);
                for (int e = threadIdx.x; e < M * M; e += blockDim.x) Q[e] = cadd(Q[e], gn[e]);
                __syncthreads();
                gemm64_gamma(P, ip.SR, PR, M);
                double2 *t = R;
                R = P;
                P = t;
                lesser_slice_out(s, n, Q, R, PR, edges, nedge, oL, oR, ot);
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) {
            if (in.T) in.T[ip.out] = T;
            if (in.status) in.status[ip.out] = st;
        }
        __syncthreads();
    }
}

// shared-memory bytes for the kernels above (matrices in shared memory or not)
extern "C" size_t knit_fp64_smem_bytes(int M, int use_smem, int nbuf)
{
    size_t b = (size_t)M * sizeof(double2) * 2 + sizeof(double2) + sizeof(double) * 32 +
               sizeof(int) * (M + 2) + 64;
    if (use_smem) b += (size_t)nbuf * M * M * sizeof(double2);
    return b;
}

// host launch helpers used by the C-ABI implementation
extern "C" cudaError_t knit_launch_sweep_fp64(const InstDev *in, int Mmax, int grid, double2 *work,
                                              int use_smem, cudaStream_t stream)
{
    size_t sm = knit_fp64_smem_bytes(Mmax, use_smem, 3);
    cudaError_t e = cudaFuncSetAttribute(knit_sweep_fp64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    knit_sweep_fp64_kernel<<<grid, 256, sm, stream>>>(*in, Mmax, work, use_smem);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_launch_lesser_fp64(const InstDev *in, int Mmax, int Lmax, int grid,
                                               double2 *work, double2 *ckpt, int save,
                                               const int2 *edges, int nedge, double *rhoL,
                                               double *rhoR, double *jx, double *jt,
                                               cudaStream_t stream)
{
    size_t sm = knit_fp64_smem_bytes(Mmax, 0, 8);
    cudaError_t e = cudaFuncSetAttribute(knit_lesser_fp64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    knit_lesser_fp64_kernel<<<grid, 256, sm, stream>>>(*in, Mmax, Lmax, work, ckpt, save, edges,
                                                       nedge, rhoL, rhoR, jx, jt);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_launch_ldos_fp64(const InstDev *in, int Mmax, int Lmax, int grid,
                                             double2 *work, int use_smem, double2 *ckpt, int save,
                                             double *ldos, long long ldos_stride,
                                             cudaStream_t stream)
{
    size_t sm = knit_fp64_smem_bytes(Mmax, use_smem, 4);
    cudaError_t e = cudaFuncSetAttribute(knit_ldos_fp64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    knit_ldos_fp64_kernel<<<grid, 256, sm, stream>>>(*in, Mmax, Lmax, work, use_smem, ckpt, save,
                                                     ldos, ldos_stride);
    return cudaGetLastError();
}
