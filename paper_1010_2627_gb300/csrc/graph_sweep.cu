// graph_sweep.cu -- the knitting sweep for an arbitrary geometry with P >= 2
// leads (KNIT user guide Sec. 5.3: knitting adds the system site by site
// through an interface whose width M_int varies along the way; Sec. 2.2
// worked example, Fig. 3; Sec. 7.3 conductance_matrix).  The host
// (knit_graph_create*) orders the sites into slices of varying width --
// breadth-first layers from lead 0's sites, the layers from the first one
// that holds a site of another lead onwards merged into the last slice -- so
// that H is block tridiagonal with rectangular couplings V_k = H_{k,k-1}
// (M_k x M_{k-1}) and every lead but lead 0 sits in the last slice.  Per
// energy, in FP64:
//     A_0 = E - H_0 - Sigma_0,  A_k = E - H_k - V_k g_{k-1} V_k^dagger,
//     A_{K-1} additionally - Sigma_p on lead p's positions (p >= 1),
//     g_k = A_k^{-1} (Gauss-Jordan),
//     G_{0,k} = G_{0,k-1} V_k^dagger g_k,   G_{k,0} = g_k V_k G_{k-1,0},
// so that G_{0,K-1}, G_{K-1,0} and G_{K-1,K-1} = g_{K-1} hold the Green
// function between every pair of leads, and
//     T_kl = Re Tr[Gamma_k G_kl Gamma_l G_kl^dagger]   (k != l)
// (Sec. 2.3, G^+_lk = G_kl^dagger, Gamma = i (Sigma - Sigma^dagger)).  One CTA
// per energy; matrices in a per-CTA global workspace (L2-resident),
// Gauss-Jordan scratch in shared memory.

#include "dense_fp64.cuh"

namespace {

// C (m x n) = A (m x k) B (k x n), all row-major compact
__device__ void gemm_r(const double2 *A, const double2 *B, double2 *C, int m, int k, int n)
{
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        double2 acc = make_double2(0.0, 0.0);
        for (int l = 0; l < k; ++l) acc = cfma(A[(size_t)i * k + l], B[(size_t)l * n + j], acc);
        C[e] = acc;
    }
    __syncthreads();
}

// C (m x n) = A (m x k) B^dagger with B (n x k)
__device__ void gemm_r_nc(const double2 *A, const double2 *B, double2 *C, int m, int k, int n)
{
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        double2 acc = make_double2(0.0, 0.0);
        for (int l = 0; l < k; ++l) acc = cfma(A[(size_t)i * k + l], cconj(B[(size_t)j * k + l]), acc);
        C[e] = acc;
    }
    __syncthreads();
}

KNIT_DEV double2 gamma_at(const double2 *S, int w, int i, int j)
{
    const double2 a = S[(size_t)i * w + j], b = S[(size_t)j * w + i];
    return make_double2(-(a.y + b.y), a.x - b.x);   // i (a - conj(b))
}

}  // namespace

extern "C" __global__ void __launch_bounds__(256)
knit_graph_fp64_kernel(GraphDev gd, const double *E, int nE, double2 *work, double *Tm, int *status)
{
    extern __shared__ __align__(16) unsigned char gsm[];
    __shared__ double red[8];
    const int Mmax = gd.Mmax, K = gd.K, P = gd.P, M0 = gd.lw[0];
    const size_t MM = (size_t)Mmax * Mmax;
    GJScratch64 sc;
    {
        unsigned char *p = gsm;
        sc.row = reinterpret_cast<double2 *>(p);
        p += sizeof(double2) * Mmax;
        sc.col = reinterpret_cast<double2 *>(p);
        p += sizeof(double2) * Mmax;
        sc.pval = reinterpret_cast<double2 *>(p);
        p += sizeof(double2);
        sc.perm = reinterpret_cast<int *>(p);
        p += sizeof(int) * Mmax;
        sc.flag = reinterpret_cast<int *>(p);
        p += sizeof(int);
        sc.piv = reinterpret_cast<int *>(p);
    }
    double2 *const base = work + (size_t)blockIdx.x * 6 * MM;
    double2 *gp = base, *A = base + MM, *G0 = base + 2 * MM, *Gc = base + 3 * MM,
            *t1 = base + 4 * MM, *t2 = base + 5 * MM;
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        const double Ee = E[e];
        int st = ST_OK, Mprev = 0;
        for (int k = 0; k < K && st == ST_OK; ++k) {
            const int Mk = gd.width[k];
            const double2 *Hk = gd.blocks + gd.hoff[k];
            const double2 *Vk = k > 0 ? gd.blocks + gd.voff[k] : nullptr;
            if (k > 0) {
                gemm_r_nc(gp, Vk, t1, Mprev, Mprev, Mk);   // g_{k-1} V_k^dagger
                gemm_r(Vk, t1, A, Mk, Mprev, Mk);          // V_k g_{k-1} V_k^dagger
            }
            const double2 *S0 = gd.sig[0] + (size_t)e * M0 * M0;
            for (int q = threadIdx.x; q < Mk * Mk; q += blockDim.x) {
                const int i = q / Mk, j = q - i * Mk;
                const double2 h = Hk[q];
                double2 a = make_double2(-h.x, -h.y);
                if (i == j) a.x += Ee;
                if (k == 0) a = csub(a, S0[q]);
                else a = csub(a, A[q]);
                A[q] = a;
            }
            __syncthreads();
            if (k == K - 1)
                for (int p = 1; p < P; ++p) {
                    const int w = gd.lw[p];
                    const int *pos = gd.lpos + gd.loff[p];
                    const double2 *Sp = gd.sig[p] + (size_t)e * w * w;
                    for (int q = threadIdx.x; q < w * w; q += blockDim.x) {
                        const size_t at = (size_t)pos[q / w] * Mk + pos[q % w];
                        A[at] = csub(A[at], Sp[q]);
                    }
                    __syncthreads();
                }
            st = gj_invert64(A, Mk, sc);
            if (st != ST_OK) break;
            if (k == 0) {
                for (int q = threadIdx.x; q < Mk * Mk; q += blockDim.x) G0[q] = Gc[q] = A[q];
                __syncthreads();
            } else {
                gemm_r_nc(G0, Vk, t2, M0, Mprev, Mk);      // G_{0,k-1} V_k^dagger
                gemm_r(t2, A, G0, M0, Mk, Mk);             // ... g_k
                gemm_r(Vk, Gc, t2, Mk, Mprev, M0);         // V_k G_{k-1,0}
                gemm_r(A, t2, Gc, Mk, Mk, M0);             // g_k ...
            }
            double2 *t = gp;   // g_k becomes the previous slice's function
            gp = A;
            A = t;
            Mprev = Mk;
        }
        // T_kl for every ordered pair of leads
        const int ML = gd.width[K - 1];
        for (int kl = 0; kl < P * P; ++kl) {
            const int k = kl / P, l = kl % P;
            double Tv = 0.0;
            if (k != l && st == ST_OK) {
                const int wk = gd.lw[k], wl = gd.lw[l];
                const int *pk = gd.lpos + gd.loff[k], *pl = gd.lpos + gd.loff[l];
                const double2 *Sk = gd.sig[k] + (size_t)e * wk * wk, *Sl = gd.sig[l] + (size_t)e * wl * wl;
                // G_kl[a][b] from G_{0,K-1} (k = 0), G_{K-1,0} (l = 0) or g_{K-1}
                auto Gkl = [&](int a, int b) -> double2 {
                    if (k == 0) return G0[(size_t)a * ML + pl[b]];
                    if (l == 0) return Gc[(size_t)pk[a] * M0 + b];
                    return gp[(size_t)pk[a] * ML + pl[b]];
                };
                // C1 = G_kl Gamma_l (wk x wl) into t1
                for (int q = threadIdx.x; q < wk * wl; q += blockDim.x) {
                    const int a = q / wl, b = q - a * wl;
                    double2 acc = make_double2(0.0, 0.0);
                    for (int c = 0; c < wl; ++c) acc = cfma(Gkl(a, c), gamma_at(Sl, wl, c, b), acc);
                    t1[q] = acc;
                }
                __syncthreads();
                double part = 0.0;
                for (int q = threadIdx.x; q < wk * wk; q += blockDim.x) {
                    const int i = q / wk, j = q - i * wk;
                    double2 cb = make_double2(0.0, 0.0);   // (C1 G_kl^dagger)_ji
                    for (int b = 0; b < wl; ++b) cb = cfma(t1[(size_t)j * wl + b], cconj(Gkl(i, b)), cb);
                    const double2 g = gamma_at(Sk, wk, i, j);
                    part += g.x * cb.x - g.y * cb.y;
                }
                Tv = block_sum(part, red);
                if (!isfinite(Tv)) st = ST_NONFINITE;
            }
            if (threadIdx.x == 0) Tm[(size_t)e * P * P + kl] = Tv;
            __syncthreads();
        }
        if (threadIdx.x == 0 && status) status[e] = st;
        __syncthreads();
    }
}

// T[e] = Tm[e][k][l]
extern "C" __global__ void knit_graph_pick_kernel(const double *Tm, int nE, int P, int k, int l,
                                                  double *T)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nE) T[e] = Tm[(size_t)e * P * P + k * P + l];
}

extern "C" size_t knit_graph_smem_bytes(int Mmax)
{
    return sizeof(double2) * (2 * (size_t)Mmax + 1) + sizeof(int) * ((size_t)Mmax + 2) + 64;
}

extern "C" cudaError_t knit_launch_graph_fp64(const GraphDev *gd, const double *E, int nE,
                                              double2 *work, int grid, double *Tm, int *status,
                                              cudaStream_t stream)
{
    const size_t sm = knit_graph_smem_bytes(gd->Mmax);
    cudaError_t e = cudaFuncSetAttribute(knit_graph_fp64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    knit_graph_fp64_kernel<<<grid, 256, sm, stream>>>(*gd, E, nE, work, Tm, status);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_launch_graph_pick(const double *Tm, int nE, int P, int k, int l,
                                              double *T, cudaStream_t stream)
{
    knit_graph_pick_kernel<<<(nE + 255) / 256, 256, 0, stream>>>(Tm, nE, P, k, l, T);
    return cudaGetLastError();
}
