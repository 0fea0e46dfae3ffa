// lead_modes_p2.cu -- period-2 leads solved sector by sector in the basis of
// the lead cell's transverse modes.
//
// A lead whose slices repeat with two alternating couplings (A between the
// two slices of a cell, B between cells) is a semi-infinite chain of
// two-slice supercells (Sec. 5.3 B applied to the supercell; Sec. 6.3 for the
// armchair ribbon).  In the eigenbasis U of the slice Hamiltonian H0 the
// supercell often falls apart into small decoupled blocks: for the armchair
// ribbon the couplings are masks (-1)^x-alternating diagonals that pair the
// transverse mode k with its partner M + 1 - k only, so the 2M x 2M supercell
// becomes M / 2 blocks of 4 x 4.  The host finds those blocks (connected
// components of U^dagger A U and U^dagger B U); here
//   * knit_small_decimation_kernel runs the Sancho-Rubio decimation of every
//     (block, energy) pair in one thread, with the same iteration, retries,
//     fixed-point and retarded-branch checks as the one-CTA decimation of
//     lead_kernels.cu, and writes each block's supercell surface function;
//   * knit_p2_sector_sigma_kernel puts the system's end-slice self-energy
//     back together: with g11 the surface slice's block of the supercell
//     surface function, Sigma = C g11 C^dagger (left lead) or
//     C^dagger g11 C (right lead), and g11 = U ghat11 U^dagger with ghat11
//     block-diagonal, so Sigma = Chat ghat11 Chat^dagger with
//     Chat = (C or C^dagger) U, restricted to the rows where Chat is nonzero;
//   * knit_p2_sector_cell_kernel forms the whole supercell surface function in
//     the orbital basis (for the lead residual check only).

#include "dense_fp64.cuh"

namespace {

// in-place inverse of the N x N matrix A (row-major, one thread) by
// Gauss-Jordan elimination with partial pivoting; X: N x N scratch
template <int N>
__device__ bool small_inverse(double2 *A, double2 *X)
{
#pragma unroll
    for (int q = 0; q < N * N; ++q) X[q] = make_double2(q / N == q % N ? 1.0 : 0.0, 0.0);
    for (int k = 0; k < N; ++k) {
        int p = k;
        double best = cabs1(A[k * N + k]);
        for (int i = k + 1; i < N; ++i) {
            const double v = cabs1(A[i * N + k]);
            if (v > best) {
                best = v;
                p = i;
            }
        }
        if (!(best > 0.0) || !isfinite(best)) return false;
        if (p != k) {
            for (int j = 0; j < N; ++j) {
                double2 t = A[k * N + j];
                A[k * N + j] = A[p * N + j];
                A[p * N + j] = t;
                t = X[k * N + j];
                X[k * N + j] = X[p * N + j];
                X[p * N + j] = t;
            }
        }
        const double2 inv = crcp(A[k * N + k]);
        for (int j = 0; j < N; ++j) {
            A[k * N + j] = cmul(A[k * N + j], inv);
            X[k * N + j] = cmul(X[k * N + j], inv);
        }
        for (int i = 0; i < N; ++i) {
            if (i == k) continue;
            const double2 f = A[i * N + k];
            if (f.x == 0.0 && f.y == 0.0) continue;
            for (int j = 0; j < N; ++j) {
                A[i * N + j] = cfms(f, A[k * N + j], A[i * N + j]);
                X[i * N + j] = cfms(f, X[k * N + j], X[i * N + j]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < N * N; ++q) A[q] = X[q];
    return true;
}

// C = A B (N x N, one thread)
template <int N>
__device__ void small_gemm(const double2 *A, const double2 *B, double2 *C)
{
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < N; ++k) acc = cfma(A[i * N + k], B[k * N + j], acc);
            C[i * N + j] = acc;
        }
}

// positive semidefinite up to -1e-9 * max_k A_kk (semidefinite Cholesky, the
// criterion of the block-cooperative check in lead_kernels.cu); A overwritten
template <int N>
__device__ bool small_psd(double2 *A)
{
    double m = 0.0;
    for (int k = 0; k < N; ++k) m = fmax(m, A[k * N + k].x);
    const double tol = 1e-9 * m;
    for (int k = 0; k < N; ++k) {
        const double piv = A[k * N + k].x;
        if (!(piv >= -tol)) return false;
        const double inv = piv > tol ? 1.0 / sqrt(piv) : 0.0;
        for (int i = k + 1; i < N; ++i) A[i * N + k] = cscale(A[i * N + k], inv);
        for (int i = k + 1; i < N; ++i)
            for (int j = k + 1; j < N; ++j)
                A[i * N + j] = cfms(A[i * N + k], cconj(A[j * N + k]), A[i * N + j]);
    }
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// Sancho-Rubio decimation of nsec independent N x N cells, one thread per
// (cell c, energy e), t = c * nE + e.  side 0: alpha = V (surface -> next
// cell outward), beta = V^dagger; side 1: the reverse.  Output: the surface
// function g[t] (N x N, NaN unless converged), iters[t], status[t].
template <int N>
__global__ void __launch_bounds__(128)
knit_small_decimation_kernel(const double2 *H0s, const double2 *Vs, int nsec, int side,
                             const double *E, int nE, double eta, double tol, int maxit,
                             double2 *gout, int *iters, int *status, int only_failed)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nsec * nE) return;
    if (only_failed && status[t] == ST_OK) return;
    const int c = (int)(t / nE), e = (int)(t - (long)c * nE);
    const double2 *H = H0s + (size_t)c * N * N, *V = Vs + (size_t)c * N * N;
    double2 eps[N * N], eps_s[N * N], al[N * N], be[N * N], gb[N * N], t1[N * N], t2[N * N],
        t3[N * N];
    double2 *G = gout + (size_t)t * N * N;
    int it = 0, st = ST_NOCONVERGE;
    double eta_k = eta;
    for (int attempt = 0; attempt < DEC_ATTEMPTS; ++attempt, eta_k *= 100.0) {
        const double2 z = make_double2(E[e], eta_k);
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                const double2 v = V[i * N + j], vd = cconj(V[j * N + i]);
                eps[i * N + j] = eps_s[i * N + j] = H[i * N + j];
                al[i * N + j] = side == 0 ? v : vd;
                be[i * N + j] = side == 0 ? vd : v;
            }
        st = ST_NOCONVERGE;
        for (it = 0; it < maxit; ++it) {
            double na = 0.0, nb = 0.0;
            for (int q = 0; q < N * N; ++q) {
                na = fmax(na, hypot(al[q].x, al[q].y));
                nb = fmax(nb, hypot(be[q].x, be[q].y));
            }
            if (na + nb < tol) {
                st = ST_OK;
                break;
            }
            if (!isfinite(na + nb)) break;
            for (int q = 0; q < N * N; ++q) {
                gb[q] = make_double2(-eps[q].x, -eps[q].y);
                if (q / N == q % N) gb[q] = cadd(gb[q], z);
            }
            if (!small_inverse<N>(gb, t3)) {
                st = ST_SINGULAR;
                break;
            }
            small_gemm<N>(gb, be, t1);   // gb beta
            small_gemm<N>(gb, al, t2);   // gb alpha
            small_gemm<N>(al, t1, t3);   // alpha gb beta
            for (int q = 0; q < N * N; ++q) {
                eps_s[q] = cadd(eps_s[q], t3[q]);
                eps[q] = cadd(eps[q], t3[q]);
            }
            small_gemm<N>(be, t2, t3);   // beta gb alpha
            for (int q = 0; q < N * N; ++q) eps[q] = cadd(eps[q], t3[q]);
            small_gemm<N>(al, t2, t3);   // alpha gb alpha: the next alpha
            small_gemm<N>(be, t1, gb);   // beta gb beta: the next beta
            for (int q = 0; q < N * N; ++q) {
                al[q] = t3[q];
                be[q] = gb[q];
            }
        }
        if (st == ST_OK) {
            for (int q = 0; q < N * N; ++q) {
                gb[q] = make_double2(-eps_s[q].x, -eps_s[q].y);
                if (q / N == q % N) gb[q] = cadd(gb[q], z);
            }
            if (!small_inverse<N>(gb, t3)) st = ST_SINGULAR;
        }
        if (st == ST_OK) {
            // the fixed point at z: t1 = (z - H0 - V g V^dagger)^{-1} (left;
            // right with V^dagger, V) against g, relative max-norm
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    double2 acc = make_double2(0.0, 0.0);
                    for (int k = 0; k < N; ++k)
                        acc = side == 0 ? cfma(gb[i * N + k], cconj(V[j * N + k]), acc)
                                        : cfma(gb[i * N + k], V[k * N + j], acc);
                    t2[i * N + j] = acc;   // g V^dagger (left), g V (right)
                }
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    double2 acc = make_double2(0.0, 0.0);
                    for (int k = 0; k < N; ++k)
                        acc = side == 0 ? cfma(V[i * N + k], t2[k * N + j], acc)
                                        : cfma(cconj(V[k * N + i]), t2[k * N + j], acc);
                    double2 v = make_double2(-H[i * N + j].x - acc.x, -H[i * N + j].y - acc.y);
                    if (i == j) v = cadd(v, z);
                    t1[i * N + j] = v;
                }
            if (!small_inverse<N>(t1, t3)) {
                st = ST_SINGULAR;
            } else {
                double dm = 0.0, gm = 0.0;
                for (int q = 0; q < N * N; ++q) {
                    dm = fmax(dm, cabs1(csub(t1[q], gb[q])));
                    gm = fmax(gm, cabs1(gb[q]));
                }
                for (int k = 0; k < N; ++k)
                    if (gb[k * N + k].y > 0.0) dm = INFINITY;
                if (!(dm <= DEC_SELF_TOL * gm)) st = ST_NOCONVERGE;
            }
        }
        if (st == ST_OK) {
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    const double2 a = gb[i * N + j], b = cconj(gb[j * N + i]);
                    t2[i * N + j] = make_double2(-(a.y - b.y), a.x - b.x);   // i (a - b)
                }
            if (!small_psd<N>(t2)) st = ST_NOCONVERGE;
        }
        if (st == ST_OK) break;
    }
    for (int q = 0; q < N * N; ++q) G[q] = st == ST_OK ? gb[q] : make_double2(nan(""), nan(""));
    if (iters) iters[t] = it;
    if (status) status[t] = st;
}

extern "C" cudaError_t knit_launch_small_decimation(const double2 *H0s, const double2 *Vs, int nsec,
                                                    int N, int side, const double *E, int nE,
                                                    double eta, double tol, int maxit,
                                                    double2 *gout, int *iters, int *status,
                                                    int only_failed, cudaStream_t stream)
{
    const long n = (long)nsec * nE;
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 127) / 128);
    switch (N) {
    case 2:
        knit_small_decimation_kernel<2><<<grid, 128, 0, stream>>>(H0s, Vs, nsec, side, E, nE, eta,
                                                                  tol, maxit, gout, iters, status,
                                                                  only_failed);
        break;
    case 4:
        knit_small_decimation_kernel<4><<<grid, 128, 0, stream>>>(H0s, Vs, nsec, side, E, nE, eta,
                                                                  tol, maxit, gout, iters, status,
                                                                  only_failed);
        break;
    case 6:
        knit_small_decimation_kernel<6><<<grid, 128, 0, stream>>>(H0s, Vs, nsec, side, E, nE, eta,
                                                                  tol, maxit, gout, iters, status,
                                                                  only_failed);
        break;
    case 8:
        knit_small_decimation_kernel<8><<<grid, 128, 0, stream>>>(H0s, Vs, nsec, side, E, nE, eta,
                                                                  tol, maxit, gout, iters, status,
                                                                  only_failed);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Newton's method on the fixed point of each N x N cell from a guess, one
// thread per (cell c, energy e), t = c * nE + e (the learned warm start of
// KNIT_LEAD_LEARNED for a lead solved in blocks).  At the real energy E:
//   F(g) = A g - I,  A = E - H0 - Vl g Vr,  (Vl, Vr) = (V, V^dagger) on the
//   left, (V^dagger, V) on the right; the step D solves A D - Vl D (Vr g) = -F,
// a dense N^2 x N^2 system (vec of D row by row) by Gaussian elimination with
// partial pivoting.  Accepted when max |F_ij| < tol, the result is retarded
// (i(g - g^dagger) positive semidefinite, the test of the decimation) and it
// lies within a tenth of the guess's size of the guess: the fixed-point
// equation has other solutions (at a real energy in a gap they are real
// too), and only a root near a good guess is taken to be the physical one;
// otherwise status ST_NOCONVERGE (the caller then decimates).  guess: float (re, im) pairs of cell c at guess + e * gstride
// + 2 N^2 c.
template <int N>
__global__ void __launch_bounds__(128)
knit_small_newton_kernel(const double2 *H0s, const double2 *Vs, int nsec, int side,
                         const double *E, int nE, const float *guess, long gstride, double tol,
                         int maxit, double2 *gout, int *iters, int *status)
{
    constexpr int NN = N * N;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)nsec * nE) return;
    const int c = (int)(t / nE), e = (int)(t - (long)c * nE);
    const double2 *H = H0s + (size_t)c * NN, *V = Vs + (size_t)c * NN;
    double2 g[NN], A[NN], B[NN], F[NN], J[NN * NN];
    const float *gs = guess + (size_t)e * gstride + 2 * NN * c;
    double gsz = 0.0;
    for (int q = 0; q < NN; ++q) {
        g[q] = make_double2((double)gs[2 * q], (double)gs[2 * q + 1]);
        gsz = fmax(gsz, cabs1(g[q]));
    }
    auto vl = [&](int i, int k) { return side == 0 ? V[i * N + k] : cconj(V[k * N + i]); };
    auto vr = [&](int i, int k) { return side == 0 ? cconj(V[k * N + i]) : V[i * N + k]; };
    const double En = E[e];
    int it = 0, st = ST_NOCONVERGE;
    for (it = 0; it <= maxit; ++it) {
        // A = E - H0 - Vl g Vr, B = Vr g
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                double2 s = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
                for (int k = 0; k < N; ++k) {
                    double2 u = make_double2(0.0, 0.0);
                    for (int l = 0; l < N; ++l) u = cfma(g[k * N + l], vr(l, j), u);
                    s = cfma(vl(i, k), u, s);
                    b = cfma(vr(i, k), g[k * N + j], b);
                }
                double2 a = make_double2(-H[i * N + j].x - s.x, -H[i * N + j].y - s.y);
                if (i == j) a.x += En;
                A[i * N + j] = a;
                B[i * N + j] = b;
            }
        double fm = 0.0;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                double2 s = make_double2(i == j ? -1.0 : 0.0, 0.0);
                for (int k = 0; k < N; ++k) s = cfma(A[i * N + k], g[k * N + j], s);
                F[i * N + j] = s;
                fm = fmax(fm, fabs(s.x) + fabs(s.y));
            }
        if (!isfinite(fm)) break;
        if (fm < tol) {
            st = ST_OK;
            break;
        }
        if (it == maxit) break;
        // J[(i,j),(k,l)] = A[i][k] delta(l,j) - Vl[i][k] B[l][j]; right-hand side -F
        for (int p = 0; p < NN; ++p) {
            const int i = p / N, j = p - i * N;
            for (int r = 0; r < NN; ++r) {
                const int k = r / N, l = r - k * N;
                double2 v = cmul(vl(i, k), B[l * N + j]);
                v = make_double2(-v.x, -v.y);
                if (l == j) v = cadd(v, A[i * N + k]);
                J[p * NN + r] = v;
            }
            F[p] = make_double2(-F[p].x, -F[p].y);
        }
        bool ok = true;
        for (int k = 0; k < NN && ok; ++k) {
            int pv = k;
            double best = cabs1(J[k * NN + k]);
            for (int i = k + 1; i < NN; ++i)
                if (cabs1(J[i * NN + k]) > best) {
                    best = cabs1(J[i * NN + k]);
                    pv = i;
                }
            if (!(best > 0.0)) {
                ok = false;
                break;
            }
            if (pv != k) {
                for (int j = k; j < NN; ++j) {
                    const double2 tt = J[k * NN + j];
                    J[k * NN + j] = J[pv * NN + j];
                    J[pv * NN + j] = tt;
                }
                const double2 tt = F[k];
                F[k] = F[pv];
                F[pv] = tt;
            }
            const double2 inv = crcp(J[k * NN + k]);
            for (int i = k + 1; i < NN; ++i) {
                const double2 f = cmul(J[i * NN + k], inv);
                if (f.x == 0.0 && f.y == 0.0) continue;
                for (int j = k + 1; j < NN; ++j) J[i * NN + j] = cfms(f, J[k * NN + j], J[i * NN + j]);
                F[i] = cfms(f, F[k], F[i]);
            }
        }
        if (!ok) break;
        for (int k = NN - 1; k >= 0; --k) {
            double2 s = F[k];
            for (int j = k + 1; j < NN; ++j) s = cfms(J[k * NN + j], F[j], s);
            F[k] = cmul(s, crcp(J[k * NN + k]));   // the step D, in place
        }
        for (int q = 0; q < NN; ++q) g[q] = cadd(g[q], F[q]);
    }
    if (st == ST_OK) {
        double moved = 0.0;
        for (int q = 0; q < NN; ++q)
            moved = fmax(moved, cabs1(csub(g[q], make_double2((double)gs[2 * q], (double)gs[2 * q + 1]))));
        if (!(moved <= 0.1 * gsz)) st = ST_NOCONVERGE;
    }
    if (st == ST_OK) {
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                const double2 a = g[i * N + j], b = cconj(g[j * N + i]);
                A[i * N + j] = make_double2(-(a.y - b.y), a.x - b.x);   // i (g - g^dagger)
            }
        if (!small_psd<N>(A)) st = ST_NOCONVERGE;
    }
    double2 *G = gout + (size_t)t * NN;
    for (int q = 0; q < NN; ++q) G[q] = st == ST_OK ? g[q] : make_double2(nan(""), nan(""));
    if (iters) iters[t] = it;
    if (status) status[t] = st;
}

extern "C" cudaError_t knit_launch_small_newton(const double2 *H0s, const double2 *Vs, int nsec, int N,
                                                int side, const double *E, int nE, const float *guess,
                                                long gstride, double tol, int maxit, double2 *gout,
                                                int *iters, int *status, cudaStream_t stream)
{
    const long n = (long)nsec * nE;
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 127) / 128);
    switch (N) {
    case 2:
        knit_small_newton_kernel<2><<<grid, 128, 0, stream>>>(H0s, Vs, nsec, side, E, nE, guess, gstride,
                                                              tol, maxit, gout, iters, status);
        break;
    case 4:
        knit_small_newton_kernel<4><<<grid, 128, 0, stream>>>(H0s, Vs, nsec, side, E, nE, guess, gstride,
                                                              tol, maxit, gout, iters, status);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sigma (M x M per energy) = Chat ghat11 Chat^dagger on the nnz rows nzr[]
// (zero elsewhere).  Cq: the nonzero rows of Chat with the modes in sector
// order, stored transposed (Cq[q * nnz + r] = Chat[nzr[r]][mode at sector
// position q]); ghat11: the first ms x ms block of each sector's supercell
// surface function (gsec[(c * nE + e)] is 2ms x 2ms, surface slice first).
// One CTA per energy (grid-stride); Y: nnz x M per CTA.
extern "C" __global__ void __launch_bounds__(256)
knit_p2_sector_sigma_kernel(const double2 *Cq, const int *nzr, int nnz, int nsec, int ms,
                            const double2 *gsec, int M, int nE, double2 *ywork, double2 *sigma)
{
    extern __shared__ int isnz[];   // M flags
    const int nm = nsec * ms, N = 2 * ms;
    double2 *Y = ywork + (size_t)blockIdx.x * nnz * nm;
    for (int i = threadIdx.x; i < M; i += blockDim.x) isnz[i] = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < nnz; r += blockDim.x) isnz[nzr[r]] = 1;
    __syncthreads();
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        double2 *S = sigma + (size_t)e * M * M;
        for (int q = threadIdx.x; q < M * M; q += blockDim.x)
            if (!isnz[q / M] || !isnz[q % M]) S[q] = make_double2(0.0, 0.0);
        // Y[r][c ms + a] = sum_b Chat[r][c ms + b] ghat_c[b][a]
        for (int x = threadIdx.x; x < nnz * nm; x += blockDim.x) {
            const int r = x % nnz, q = x / nnz, c = q / ms, a = q - c * ms;
            const double2 *g = gsec + ((size_t)c * nE + e) * N * N;
            double2 acc = make_double2(0.0, 0.0);
            for (int b = 0; b < ms; ++b) acc = cfma(Cq[(size_t)(c * ms + b) * nnz + r], g[b * N + a], acc);
            Y[(size_t)r * nm + q] = acc;
        }
        __syncthreads();
        // Sigma[nzr[r]][nzr[s]] = sum_q Y[r][q] conj(Chat[s][q])
        for (int x = threadIdx.x; x < nnz * nnz; x += blockDim.x) {
            const int r = x / nnz, s = x - r * nnz;
            double2 acc = make_double2(0.0, 0.0);
            for (int q = 0; q < nm; ++q) acc = cfma(Y[(size_t)r * nm + q], cconj(Cq[(size_t)q * nnz + s]), acc);
            S[(size_t)nzr[r] * M + nzr[s]] = acc;
        }
        __syncthreads();
    }
}

extern "C" cudaError_t knit_launch_p2_sector_sigma(const double2 *Cq, const int *nzr, int nnz,
                                                   int nsec, int ms, const double2 *gsec, int M,
                                                   int nE, double2 *ywork, double2 *sigma, int grid,
                                                   cudaStream_t stream)
{
    knit_p2_sector_sigma_kernel<<<grid, 256, sizeof(int) * M, stream>>>(Cq, nzr, nnz, nsec, ms, gsec,
                                                                         M, nE, ywork, sigma);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The supercell surface function in the orbital basis (2M x 2M per energy,
// slice h at rows h M .. h M + M - 1): gcell[(h1, i)][(h2, j)] =
// sum_c sum_{a, b} U[i][k_a] ghat_c[(h1, a)][(h2, b)] conj(U[j][k_b]), the
// modes k of sector c at sidx[c ms ..].  One thread per element.
extern "C" __global__ void __launch_bounds__(256)
knit_p2_sector_cell_kernel(const double2 *U, const int *sidx, int nsec, int ms, const double2 *gsec,
                           int M, int nE, double2 *gcell)
{
    const int Mp = 2 * M, N = 2 * ms;
    const long n = (long)nE * Mp * Mp;
    for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long)gridDim.x * blockDim.x) {
        const int e = (int)(x / ((long)Mp * Mp));
        const int I = (int)(x / Mp % Mp), J = (int)(x % Mp);
        const int h1 = I / M, i = I - h1 * M, h2 = J / M, j = J - h2 * M;
        double2 acc = make_double2(0.0, 0.0);
        for (int c = 0; c < nsec; ++c) {
            const double2 *g = gsec + ((size_t)c * nE + e) * N * N;
            for (int a = 0; a < ms; ++a) {
                const double2 ua = U[(size_t)i * M + sidx[c * ms + a]];
                double2 r = make_double2(0.0, 0.0);
                for (int b = 0; b < ms; ++b)
                    r = cfma(g[(h1 * ms + a) * N + h2 * ms + b], cconj(U[(size_t)j * M + sidx[c * ms + b]]), r);
                acc = cfma(ua, r, acc);
            }
        }
        gcell[x] = acc;
    }
}

extern "C" cudaError_t knit_launch_p2_sector_cell(const double2 *U, const int *sidx, int nsec, int ms,
                                                  const double2 *gsec, int M, int nE, double2 *gcell,
                                                  int grid, cudaStream_t stream)
{
    knit_p2_sector_cell_kernel<<<grid, 256, 0, stream>>>(U, sidx, nsec, ms, gsec, M, nE, gcell);
    return cudaGetLastError();
}
