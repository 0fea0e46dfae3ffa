// tau_kernels.cu -- transmission eigenvalues and shot noise of the two-terminal
// system (KNIT user guide Sec. 8 lists "conductance, shot noise, transmission
// eigenvalues" among the transport properties; Sec. 2.3 writes T_kl as the
// trace of G_kl Gamma_l G_kl^+ Gamma_k, whose eigenvalues are the
// transmission eigenvalues tau_n; the zero-temperature shot noise is
// proportional to sum_n tau_n (1 - tau_n)).
//
// The eigenvalues are taken at the right end of the sweep, where every sweep
// kernel holds G = G_LL.  The unitarity identity of the retarded function,
// G - G^dagger = -i G (Gamma_L + Gamma_R) G^dagger, gives for its (L, L) block
//     G_L1 Gamma_L G_L1^dagger = K = i (G - G^dagger) - G Gamma_R G^dagger,
// and the tau_n are the nonzero eigenvalues of K Gamma_R (the paper's product
// seen from the right lead; a lossless two-terminal scattering matrix has the
// same transmission spectrum from both sides).  With any factor Gamma_R =
// W W^dagger (W: M x r) they are the eigenvalues of the r x r Hermitian matrix
//     Q = W^dagger K W = i (C - C^dagger) - C C^dagger,   C = W^dagger G W,
// whose trace is the T of the sweep kernels.  All steps in FP64:
//  * knit_tau_chol_kernel, per energy: Gamma_R = i (Sigma_R - Sigma_R^dagger)
//    by Cholesky with diagonal pivoting, stopped when the largest remaining
//    diagonal element falls below CHOL_TOL times Gamma_R's largest -- r is
//    then the number of open channels of the right lead;
//  * knit_tau_eig_kernel, per instance: C and Q (shared memory for M <= 64),
//    Householder reduction of Q to a real symmetric tridiagonal matrix (the
//    complex off-diagonal phases drop out of the spectrum), eigenvalues by
//    bisection on Sturm counts, the M - r closed channels as zeros, all in
//    decreasing order, and sum tau (1 - tau).

#include <algorithm>

#include "dense_fp64.cuh"

namespace {

constexpr double CHOL_TOL = 1e-14;

// largest value over the block and the lowest index attaining it
__device__ void block_argmax(double &v, int &idx, double *rv, int *ri)
{
    warp_argmax(v, idx);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        rv[w] = v;
        ri[w] = idx;
    }
    __syncthreads();
    v = rv[0];
    idx = ri[0];
    for (int k = 1; k < nw; ++k)
        if (rv[k] > v || (rv[k] == v && ri[k] < idx)) {
            v = rv[k];
            idx = ri[k];
        }
}

// Gamma_R(E_e) = W W^dagger (+ remainder below CHOL_TOL), W column j at
// W[x * M + j] for orbital x; rank[e] = r.  A: M^2 scratch per energy.
__global__ void __launch_bounds__(256)
knit_tau_chol_kernel(const double2 *sig, int M, int nE, double2 *A, double2 *Wout, int *rank)
{
    __shared__ int perm[256];
    __shared__ double rv[8];
    __shared__ int ri[8];
    const size_t MM = (size_t)M * M;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        const double2 *s = sig + e * MM;
        double2 *a = A + e * MM, *w = Wout + e * MM;
        for (int q = tid; q < M * M; q += nt) {
            const int i = q / M, j = q - i * M;
            const double2 x = s[(size_t)i * M + j], y = s[(size_t)j * M + i];
            a[q] = make_double2(-(x.y + y.y), x.x - y.x);   // i (x - conj(y))
            w[q] = make_double2(0.0, 0.0);
        }
        for (int i = tid; i < M; i += nt) perm[i] = i;
        __syncthreads();
        double d0 = 0.0;
        int dummy = 0;
        {
            double v = 0.0;
            for (int i = tid; i < M; i += nt) v = fmax(v, a[(size_t)i * M + i].x);
            d0 = v;
            block_argmax(d0, dummy, rv, ri);
        }
        int r = 0;
        for (int j = 0; j < M; ++j) {
            double v = -1.0;
            int p = M;
            for (int i = j + tid; i < M; i += nt) {
                const double d = a[(size_t)perm[i] * M + perm[i]].x;
                if (d > v) {
                    v = d;
                    p = i;
                }
            }
            block_argmax(v, p, rv, ri);
            if (!(d0 > 0.0) || !(v > CHOL_TOL * d0)) break;   // also stops on NaN
            __syncthreads();
            if (tid == 0) {
                const int t = perm[j];
                perm[j] = perm[p];
                perm[p] = t;
            }
            __syncthreads();
            const int pj = perm[j];
            const double ljj = sqrt(v), inv = 1.0 / ljj;
            for (int i = j + 1 + tid; i < M; i += nt) {
                const int x = perm[i];
                const double2 c = a[(size_t)x * M + pj];
                w[(size_t)x * M + j] = make_double2(c.x * inv, c.y * inv);
            }
            if (tid == 0) w[(size_t)pj * M + j] = make_double2(ljj, 0.0);
            __syncthreads();
            const int m = M - j - 1;
            for (int q = tid; q < m * m; q += nt) {
                const int x = perm[j + 1 + q / m], y = perm[j + 1 + q % m];
                a[(size_t)x * M + y] = cfma(make_double2(-w[(size_t)x * M + j].x, -w[(size_t)x * M + j].y),
                                            cconj(w[(size_t)y * M + j]), a[(size_t)x * M + y]);
            }
            __syncthreads();
            r = j + 1;
        }
        if (tid == 0) rank[e] = r;
        __syncthreads();
    }
}

// eigenvalues of the real symmetric tridiagonal matrix (d, b^2 off-diagonal
// squares, order r) below x: the number of negative pivots of T - x I
__device__ int sturm_count(const double *d, const double *b2, int r, double x)
{
    const double pivmin = 1e-290;
    double q = d[0] - x;
    int c = q < 0.0;
    for (int i = 1; i < r; ++i) {
        if (fabs(q) < pivmin) q = -pivmin;
        q = d[i] - x - b2[i - 1] / q;
        c += q < 0.0;
    }
    return c;
}

// tau of instances i (grid-stride, one CTA each) from G_LL (GLL + i M^2) and
// the factor W of its energy i / nS.  Work area (3 M^2 complex128): dynamic
// shared memory when use_smem, else `work` + 3 M^2 per CTA.
__global__ void __launch_bounds__(256)
knit_tau_eig_kernel(const double2 *GLL, const double2 *W, const int *rank, int M, int n, int nS,
                    const int *status, double2 *work, int use_smem, double *tau, double *noise)
{
    extern __shared__ double2 dsm[];
    __shared__ double dd[256], b2[256], lam[256];
    __shared__ double2 vv[256], pp[256];
    __shared__ double red[8];
    const size_t MM = (size_t)M * M;
    const int tid = threadIdx.x, nt = blockDim.x;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    double2 *Ws = use_smem ? dsm : work + (size_t)blockIdx.x * 3 * MM;
    double2 *T1 = Ws + MM, *C = T1 + MM;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int e = i / nS, r = rank[e];
        const bool bad = status && status[i] != 0;
        if (bad) {
            for (int k = tid; k < M; k += nt) tau[(size_t)i * M + k] = nan;
            if (tid == 0 && noise) noise[i] = nan;
            continue;
        }
        const double2 *g = GLL + (size_t)i * MM, *we = W + (size_t)e * MM;
        // W (M x r, stride r); T1 = G W (M x r); C = W^dagger T1 (r x r)
        for (int q = tid; q < M * r; q += nt) Ws[q] = we[(size_t)(q / r) * M + q % r];
        __syncthreads();
        for (int q = tid; q < M * r; q += nt) {
            const int x = q / r, c = q - x * r;
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < M; ++k) acc = cfma(g[(size_t)x * M + k], Ws[k * r + c], acc);
            T1[q] = acc;
        }
        __syncthreads();
        for (int q = tid; q < r * r; q += nt) {
            const int a = q / r, c = q - a * r;
            double2 acc = make_double2(0.0, 0.0);
            for (int x = 0; x < M; ++x) acc = cfma(cconj(Ws[x * r + a]), T1[x * r + c], acc);
            C[q] = acc;
        }
        __syncthreads();
        // Q = i (C - C^dagger) - C C^dagger into T1 (r x r)
        double2 *Q = T1;
        for (int q = tid; q < r * r; q += nt) {
            const int a = q / r, c = q - a * r;
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < r; ++k) acc = cfma(C[a * r + k], cconj(C[c * r + k]), acc);
            const double2 x = C[q], y = cconj(C[c * r + a]);
            Q[q] = make_double2(-(x.y - y.y) - acc.x, (x.x - y.x) - acc.y);
        }
        __syncthreads();
        // Householder: Q -> tridiagonal, d on the diagonal, b2 = |off-diagonal|^2
        for (int k = 0; k + 2 < r; ++k) {
            double s2 = 0.0;
            for (int x = k + 1 + tid; x < r; x += nt) {
                const double2 z = Q[x * r + k];
                s2 += z.x * z.x + z.y * z.y;
            }
            s2 = block_sum(s2, red);
            const double2 x0 = Q[(k + 1) * r + k];
            const double ax0 = hypot(x0.x, x0.y), nrm = sqrt(s2);
            if (tid == 0) {
                dd[k] = Q[k * r + k].x;
                b2[k] = s2;
            }
            if (s2 - ax0 * ax0 <= 0.0) {   // column already reduced
                __syncthreads();
                continue;
            }
            // alpha = -e^{i arg x0} |x|, v = (x - alpha e_1) / |x - alpha e_1|
            const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
            const double2 alpha = make_double2(-ph.x * nrm, -ph.y * nrm);
            const double vn = sqrt(2.0 * s2 + 2.0 * ax0 * nrm);   // |x - alpha e_1|
            for (int x = k + 1 + tid; x < r; x += nt) {
                double2 z = Q[x * r + k];
                if (x == k + 1) z = make_double2(z.x - alpha.x, z.y - alpha.y);
                vv[x] = make_double2(z.x / vn, z.y / vn);
            }
            __syncthreads();
            // p = Q v on the trailing block, beta = v^dagger p
            double bl = 0.0;
            for (int x = k + 1 + tid; x < r; x += nt) {
                double2 acc = make_double2(0.0, 0.0);
                for (int c = k + 1; c < r; ++c) acc = cfma(Q[x * r + c], vv[c], acc);
                pp[x] = acc;
                bl += vv[x].x * acc.x + vv[x].y * acc.y;
            }
            const double beta = block_sum(bl, red);
            // w = 2 p - 2 beta v; Q -= v w^dagger + w v^dagger
            for (int x = k + 1 + tid; x < r; x += nt)
                pp[x] = make_double2(2.0 * (pp[x].x - beta * vv[x].x), 2.0 * (pp[x].y - beta * vv[x].y));
            __syncthreads();
            const int m = r - k - 1;
            for (int q = tid; q < m * m; q += nt) {
                const int x = k + 1 + q / m, c = k + 1 + q % m;
                double2 z = Q[x * r + c];
                z = cfma(make_double2(-vv[x].x, -vv[x].y), cconj(pp[c]), z);
                z = cfma(make_double2(-pp[x].x, -pp[x].y), cconj(vv[c]), z);
                Q[x * r + c] = z;
            }
            __syncthreads();
        }
        if (tid == 0 && r > 0) {
            if (r >= 2) {
                dd[r - 2] = Q[(r - 2) * r + r - 2].x;
                const double2 z = Q[(r - 1) * r + r - 2];
                b2[r - 2] = z.x * z.x + z.y * z.y;
            }
            dd[r - 1] = Q[(r - 1) * r + r - 1].x;
        }
        __syncthreads();
        // bisection: thread j finds the j-th largest eigenvalue
        double lo = 0.0, hi = 0.0;
        for (int x = 0; x < r; ++x) {
            const double bl = x > 0 ? sqrt(b2[x - 1]) : 0.0, br = x + 1 < r ? sqrt(b2[x]) : 0.0;
            lo = x ? fmin(lo, dd[x] - bl - br) : dd[x] - bl - br;
            hi = x ? fmax(hi, dd[x] + bl + br) : dd[x] + bl + br;
        }
        const double pad = 1e-12 * fmax(1.0, fmax(fabs(lo), fabs(hi)));
        lo -= pad;
        hi += pad;
        for (int j = tid; j < r; j += nt) {
            const int ks = r - 1 - j;   // index from the bottom
            double a = lo, b = hi;
            for (int it = 0; it < 80; ++it) {
                const double mid = 0.5 * (a + b);
                if (mid <= a || mid >= b) break;
                if (sturm_count(dd, b2, r, mid) > ks) b = mid;
                else a = mid;
            }
            lam[j] = 0.5 * (a + b);
        }
        __syncthreads();
        // decreasing order with the M - r closed channels as zeros
        double ns = 0.0;
        int npos = 0;
        for (int j = 0; j < r; ++j) npos += lam[j] >= 0.0;
        for (int j = tid; j < r; j += nt) {
            const double v = lam[j];
            tau[(size_t)i * M + (v >= 0.0 ? j : j + (M - r))] = v;
            ns += v * (1.0 - v);
        }
        for (int k = tid; k < M - r; k += nt) tau[(size_t)i * M + npos + k] = 0.0;
        ns = block_sum(ns, red);
        if (tid == 0 && noise) noise[i] = ns;
        __syncthreads();
    }
}

}  // namespace

// the factor W (nE x M x M, first rank[e] columns) of Gamma_R for nE
// energies from Sigma_R (nE x M x M); work: nE M^2
extern "C" cudaError_t knit_launch_gamma_factor(const double2 *sigR, int M, int nE, double2 *work,
                                                double2 *W, int *rank, cudaStream_t stream)
{
    knit_tau_chol_kernel<<<std::min(nE, 65535), 256, 0, stream>>>(sigR, M, nE, work, W, rank);
    return cudaGetLastError();
}

// bytes of global work area per CTA of knit_launch_tau (0 when shared memory serves)
extern "C" size_t knit_tau_work_bytes(int M)
{
    return M <= 64 ? 0 : sizeof(double2) * 3 * (size_t)M * M;
}

// tau (n x M, decreasing) and noise (n, optional) from G_LL (n x M x M) and
// the factors W / rank of knit_launch_gamma_factor (instance i at energy
// i / nS); work: knit_tau_work_bytes(M) per CTA of `grid`
extern "C" cudaError_t knit_launch_tau(const double2 *GLL, const double2 *W, const int *rank,
                                       int M, int n, int nS, const int *status, void *work,
                                       int grid, double *tau, double *noise, cudaStream_t stream)
{
    const int use_smem = M <= 64;
    const size_t smb = use_smem ? sizeof(double2) * 3 * (size_t)M * M : 0;
    cudaError_t e = cudaFuncSetAttribute(knit_tau_eig_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    if (e != cudaSuccess) return e;
    knit_tau_eig_kernel<<<grid, 256, smb, stream>>>(GLL, W, rank, M, n, nS, status,
                                                    static_cast<double2 *>(work), use_smem, tau,
                                                    noise);
    return cudaGetLastError();
}
