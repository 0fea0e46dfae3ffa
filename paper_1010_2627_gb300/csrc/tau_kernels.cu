// tau_kernels.cu -- transmission eigenvalues and shot noise of the two-terminal
// system (KNIT user guide Sec. 8 lists "conductance, shot noise, transmission
// eigenvalues" among the transport properties; Sec. 2.3 writes T_kl as the
// trace of G_kl Gamma_l G_kl^+ Gamma_k, whose eigenvalues are the
// transmission eigenvalues tau_n; the zero-temperature shot noise is
// proportional to sum_n tau_n (1 - tau_n)).
//
// The eigenvalues are taken at the right end of the sweep, where every sweep
// kernel holds G = G_LL.  With S = Gamma_R^{1/2}, the unitarity identity of
// the retarded function, G - G^dagger = -i G (Gamma_L + Gamma_R) G^dagger,
// gives for its (L, L) block
//     S G_L1 Gamma_L G_L1^dagger S = i (C - C^dagger) - C C^dagger,   C = S G S,
// a Hermitian matrix Q whose trace is the T of the sweep kernels and whose
// eigenvalues are the tau_n (the paper's product has the same nonzero
// spectrum; a lossless two-terminal scattering matrix makes the left and right
// transmission spectra equal).  Steps, all FP64:
//  * knit_tau_gamma_kernel: Gamma_R(E_e) = i (Sigma_R - Sigma_R^dagger);
//  * knit_jacobi_kernel (lead_kernels.cu, batched, with eigenvectors):
//    Gamma_R = U diag(w) U^dagger;
//  * knit_tau_sqrt_kernel: S = U diag(sqrt(max(w, 0))) U^dagger;
//  * knit_tau_form_kernel: Q = i (C - C^dagger) - C C^dagger per instance;
//  * knit_jacobi_kernel (batched, eigenvalues only) on every Q;
//  * knit_tau_sort_kernel: tau in decreasing order and sum tau (1 - tau).

#include "dense_fp64.cuh"

extern "C" cudaError_t knit_launch_jacobi_batch(double2 *A, double2 *U, int M, int count,
                                                cudaStream_t stream);

namespace {

// Gamma(E_e) = i (Sigma - Sigma^dagger) for nE blocks of M x M
__global__ void knit_tau_gamma_kernel(const double2 *sig, int M, int nE, double2 *gam)
{
    const size_t MM = (size_t)M * M, tot = MM * nE;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < tot;
         q += (size_t)gridDim.x * blockDim.x) {
        const size_t e = q / MM, r = q - e * MM;
        const int i = (int)(r / M), j = (int)(r - (size_t)i * M);
        const double2 a = sig[e * MM + (size_t)i * M + j], b = sig[e * MM + (size_t)j * M + i];
        gam[q] = make_double2(-(a.y + b.y), a.x - b.x);   // i (a - conj(b))
    }
}

// S = U diag(sqrt(max(w_k, 0))) U^dagger with w_k on the diagonal of D
__global__ void __launch_bounds__(256)
knit_tau_sqrt_kernel(const double2 *U, const double2 *D, int M, int nE, double2 *S)
{
    const size_t MM = (size_t)M * M;
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        const double2 *u = U + e * MM, *d = D + e * MM;
        for (int q = threadIdx.x; q < M * M; q += blockDim.x) {
            const int i = q / M, j = q - i * M;
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < M; ++k) {
                const double w = sqrt(fmax(d[(size_t)k * M + k].x, 0.0));
                const double2 uik = u[(size_t)i * M + k];
                acc = cfma(make_double2(uik.x * w, uik.y * w), cconj(u[(size_t)j * M + k]), acc);
            }
            S[e * MM + q] = acc;
        }
    }
}

// Q_i = i (C - C^dagger) - C C^dagger, C = S G S, for instances i (grid-stride,
// one CTA each): G_LL of instance i at GLL + i M^2, S of its energy i / nS.
// work: 2 M^2 per CTA.
__global__ void __launch_bounds__(256)
knit_tau_form_kernel(const double2 *GLL, const double2 *S, int M, int n, int nS, double2 *work,
                     double2 *Q)
{
    const size_t MM = (size_t)M * M;
    double2 *T1 = work + (size_t)blockIdx.x * 2 * MM, *C = T1 + MM;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const double2 *g = GLL + (size_t)i * MM, *s = S + (size_t)(i / nS) * MM;
        gemm64(s, g, T1, M);      // S G
        gemm64(T1, s, C, M);      // C = S G S
        gemm64_nc(C, C, T1, M);   // C C^dagger
        double2 *q = Q + (size_t)i * MM;
        for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
            const int a = e / M, b = e - a * M;
            const double2 c = C[e], ct = cconj(C[(size_t)b * M + a]);
            q[e] = make_double2(-(c.y - ct.y) - T1[e].x, (c.x - ct.x) - T1[e].y);
        }
        __syncthreads();
    }
}

// tau_i (decreasing) from the diagonal of the diagonalised Q_i, and
// noise_i = sum tau (1 - tau); an instance with a non-zero status gets NaN.
// Dynamic shared memory: M doubles.
__global__ void __launch_bounds__(256)
knit_tau_sort_kernel(const double2 *Q, int M, int n, const int *status, double *tau,
                     double *noise)
{
    extern __shared__ double w[];
    __shared__ double red[8];
    const size_t MM = (size_t)M * M;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const bool bad = status && status[i] != 0;
        for (int k = threadIdx.x; k < M; k += blockDim.x) w[k] = Q[(size_t)i * MM + (size_t)k * M + k].x;
        __syncthreads();
        double ns = 0.0;
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            const double v = w[k];
            int pos = 0;
            for (int m = 0; m < M; ++m) pos += (w[m] > v) || (w[m] == v && m < k);
            if (bad) tau[(size_t)i * M + k] = nan;
            else tau[(size_t)i * M + pos] = v;
            ns += v * (1.0 - v);
        }
        ns = block_sum(ns, red);
        if (threadIdx.x == 0 && noise) noise[i] = bad ? nan : ns;
        __syncthreads();
    }
}

}  // namespace

// Gamma_R^{1/2} for nE energies from Sigma_R (nE x M x M): work 2 nE M^2
// (the eigen-decomposition), result S (nE x M x M).
extern "C" cudaError_t knit_launch_gamma_sqrt(const double2 *sigR, int M, int nE, double2 *work,
                                              double2 *S, cudaStream_t stream)
{
    const size_t MM = (size_t)M * M;
    double2 *D = work, *U = work + MM * nE;
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((MM * nE + threads - 1) / threads, 65535);
    knit_tau_gamma_kernel<<<blocks, threads, 0, stream>>>(sigR, M, nE, D);
    cudaError_t e = knit_launch_jacobi_batch(D, U, M, nE, stream);
    if (e != cudaSuccess) return e;
    knit_tau_sqrt_kernel<<<nE, 256, 0, stream>>>(U, D, M, nE, S);
    return cudaGetLastError();
}

// tau (n x M, decreasing) and noise (n, optional) from G_LL (n x M x M) and
// S = Gamma_R^{1/2} (one per energy, instance i at energy i / nS).  Q: n M^2
// scratch; work: 2 M^2 per CTA of `grid`.
extern "C" cudaError_t knit_launch_tau(const double2 *GLL, const double2 *S, int M, int n, int nS,
                                       const int *status, double2 *Q, double2 *work, int grid,
                                       double *tau, double *noise, cudaStream_t stream)
{
    knit_tau_form_kernel<<<grid, 256, 0, stream>>>(GLL, S, M, n, nS, work, Q);
    cudaError_t e = knit_launch_jacobi_batch(Q, nullptr, M, n, stream);
    if (e != cudaSuccess) return e;
    knit_tau_sort_kernel<<<std::min(n, 65535), 256, sizeof(double) * M, stream>>>(Q, M, n, status,
                                                                                 tau, noise);
    return cudaGetLastError();
}
