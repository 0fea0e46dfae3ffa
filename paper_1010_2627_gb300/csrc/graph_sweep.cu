// graph_sweep.cu -- the knitting sweep for an arbitrary two-lead geometry
// (KNIT user guide Sec. 5.3: knitting adds the system site by site through
// an interface whose width M_int varies along the way; Sec. 2.2 worked
// example, Fig. 3).  The host (knit_graph_create) orders the sites into
// slices of varying width -- breadth-first layers from lead 0's sites, the
// layers from the first one that holds a lead-1 site onwards merged into the
// last slice -- so that H is block tridiagonal with rectangular couplings
// V_k = H_{k,k-1} (M_k x M_{k-1}).  Per energy, in FP64:
//     A_0 = E - H_0 - Sigma_0,  A_k = E - H_k - V_k g_{k-1} V_k^dagger,
//     A_{K-1} additionally - Sigma_1 on lead 1's positions in the last slice,
//     g_k = A_k^{-1} (Gauss-Jordan),  G_{0,0} = g_0,  G_{0,k} = G_{0,k-1} V_k^dagger g_k,
//     T_01 = Re Tr[Gamma_0 G_{0,1} Gamma_1 G_{0,1}^dagger]
// (Sec. 2.3, k = 0, l = 1; G_{0,1} the columns of G_{0,K-1} at lead 1's
// sites, Gamma = i (Sigma - Sigma^dagger)).  One CTA per energy; matrices in a
// per-CTA global workspace (L2-resident), Gauss-Jordan scratch in shared memory.

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
knit_graph_fp64_kernel(GraphDev gd, const double *E, int nE, const double2 *sig0,
                       const double2 *sig1, double2 *work, double *T, int *status)
{
    extern __shared__ __align__(16) unsigned char gsm[];
    __shared__ double red[8];
    const int Mmax = gd.Mmax, M0 = gd.w0, w1 = gd.w1, K = gd.K;
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
    double2 *const base = work + (size_t)blockIdx.x * 5 * MM;
    double2 *gp = base, *A = base + MM, *G0 = base + 2 * MM, *t1 = base + 3 * MM, *t2 = base + 4 * MM;
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        const double Ee = E[e];
        const double2 *S0 = sig0 + (size_t)e * M0 * M0, *S1 = sig1 + (size_t)e * w1 * w1;
        int st = ST_OK, Mprev = 0;
        for (int k = 0; k < K && st == ST_OK; ++k) {
            const int Mk = gd.width[k];
            const double2 *Hk = gd.blocks + gd.hoff[k];
            if (k > 0) {
                const double2 *Vk = gd.blocks + gd.voff[k];
                gemm_r_nc(gp, Vk, t1, Mprev, Mprev, Mk);   // g_{k-1} V_k^dagger
                gemm_r(Vk, t1, A, Mk, Mprev, Mk);          // V_k g_{k-1} V_k^dagger
            }
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
                for (int q = threadIdx.x; q < w1 * w1; q += blockDim.x) {
                    const int a = q / w1, b = q - a * w1;
                    const size_t pos = (size_t)gd.p1[a] * Mk + gd.p1[b];
                    A[pos] = csub(A[pos], S1[q]);
                }
            __syncthreads();
            st = gj_invert64(A, Mk, sc);
            if (st != ST_OK) break;
            if (k == 0) {
                for (int q = threadIdx.x; q < Mk * Mk; q += blockDim.x) G0[q] = A[q];
                __syncthreads();
            } else {
                const double2 *Vk = gd.blocks + gd.voff[k];
                gemm_r_nc(G0, Vk, t2, M0, Mprev, Mk);      // G_{0,k-1} V_k^dagger
                gemm_r(t2, A, G0, M0, Mk, Mk);             // ... g_k
            }
            double2 *t = gp;   // g_k becomes the previous slice's function
            gp = A;
            A = t;
            Mprev = Mk;
        }
        double Tv = 0.0;
        if (st == ST_OK) {
            // B = G_{0,K-1}[:, p1] (M0 x w1), C1 = B Gamma_1 into t1, then
            // T = Re sum_ij Gamma0_ij (C1 B^dagger)_ji
            const int ML = gd.width[K - 1];
            for (int q = threadIdx.x; q < M0 * w1; q += blockDim.x) {
                const int i = q / w1, a = q - i * w1;
                double2 acc = make_double2(0.0, 0.0);
                for (int b = 0; b < w1; ++b)
                    acc = cfma(G0[(size_t)i * ML + gd.p1[b]], gamma_at(S1, w1, b, a), acc);
                t1[q] = acc;
            }
            __syncthreads();
            double part = 0.0;
            for (int q = threadIdx.x; q < M0 * M0; q += blockDim.x) {
                const int i = q / M0, j = q - i * M0;
                double2 cb = make_double2(0.0, 0.0);   // (C1 B^dagger)_ji
                for (int a = 0; a < w1; ++a)
                    cb = cfma(t1[(size_t)j * w1 + a], cconj(G0[(size_t)i * ML + gd.p1[a]]), cb);
                const double2 g = gamma_at(S0, M0, i, j);
                part += g.x * cb.x - g.y * cb.y;
            }
            Tv = block_sum(part, red);
            if (!isfinite(Tv)) st = ST_NONFINITE;
        }
        if (threadIdx.x == 0) {
            T[e] = Tv;
            if (status) status[e] = st;
        }
        __syncthreads();
    }
}

extern "C" size_t knit_graph_smem_bytes(int Mmax)
{
    return sizeof(double2) * (2 * (size_t)Mmax + 1) + sizeof(int) * ((size_t)Mmax + 2) + 64;
}

extern "C" cudaError_t knit_launch_graph_fp64(const GraphDev *gd, const double *E, int nE,
                                              const double2 *sig0, const double2 *sig1,
                                              double2 *work, int grid, double *T, int *status,
                                              cudaStream_t stream)
{
    const size_t sm = knit_graph_smem_bytes(gd->Mmax);
    cudaError_t e = cudaFuncSetAttribute(knit_graph_fp64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    knit_graph_fp64_kernel<<<grid, 256, sm, stream>>>(*gd, E, nE, sig0, sig1, work, T, status);
    return cudaGetLastError();
}
