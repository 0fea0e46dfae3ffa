// dense_fp64.cuh -- block-cooperative FP64 dense kernels on M x M complex
// matrices held in shared or global memory (generic pointers, row-major,
// leading dimension M): Gauss-Jordan inversion with partial pivoting and the
// small products the slice sweep and the lead solvers need.  Every routine is
// called by all threads of the block and ends with __syncthreads().
#pragma once

#include "knit_common.cuh"

struct GJScratch64 {
    double2 *row;   // M
    double2 *col;   // M
    int *perm;      // M
    int *flag;      // 1
    int *piv;       // 1
    double2 *pval;  // 1
};

// In-place inversion of a (M x M) by Gauss-Jordan elimination with partial
// pivoting: at step k the pivot is the row i >= k with the largest
// |Re| + |Im| in column k (lowest row on ties); rows are exchanged, the pivot
// row scaled, every other row eliminated, and the columns of the result
// permuted back at the end.  Returns 0, or ST_SINGULAR (matrix left
// unspecified) if a pivot is exactly zero.
static __device__ int gj_invert64(double2 *a, int M, GJScratch64 sc)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    for (int k = 0; k < M; ++k) {
        if (warp == 0) {
            double best = -1.0;
            int bi = M;
            for (int i = k + lane; i < M; i += 32) {
                double v = cabs1(a[(size_t)i * M + k]);
                if (v > best) { best = v; bi = i; }
            }
            warp_argmax(best, bi);
            if (lane == 0) {
                *sc.piv = bi;
                sc.perm[k] = bi;
                *sc.flag = (best == 0.0);
                *sc.pval = a[(size_t)bi * M + k];
            }
        }
        __syncthreads();
        if (*sc.flag) { __syncthreads(); return ST_SINGULAR; }
        const int p = *sc.piv;
        const double2 pinv = crcp(*sc.pval);
        // phase A: exchange rows k and p, stage the scaled pivot row and column k
        for (int j = tid; j < M; j += nt) {
            double2 rk = a[(size_t)k * M + j];
            double2 rp = a[(size_t)p * M + j];
            if (p != k) a[(size_t)p * M + j] = rk;
            sc.row[j] = (j == k) ? pinv : cmul(rp, pinv);
        }
        for (int i = tid; i < M; i += nt) {
            if (i == k) continue;
            sc.col[i] = (i == p) ? a[(size_t)k * M + k] : a[(size_t)i * M + k];
        }
        __syncthreads();
        // phase B: eliminate
        for (int e = tid; e < M * M; e += nt) {
            int i = e / M, j = e - i * M;
            if (i == k) {
                a[e] = sc.row[j];
            } else if (j == k) {
                a[e] = cmul(make_double2(-sc.col[i].x, -sc.col[i].y), pinv);
            } else {
                a[e] = cfms(sc.col[i], sc.row[j], a[e]);
            }
        }
        __syncthreads();
    }
    // undo the row exchanges as column exchanges, last first
    for (int k = M - 1; k >= 0; --k) {
        int p = sc.perm[k];
        if (p != k) {
            for (int i = tid; i < M; i += nt) {
                double2 t = a[(size_t)i * M + k];
                a[(size_t)i * M + k] = a[(size_t)i * M + p];
                a[(size_t)i * M + p] = t;
            }
        }
        __syncthreads();
    }
    return ST_OK;
}

// C = A * B
static __device__ void gemm64(const double2 *A, const double2 *B, double2 *C, int M)
{
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        int i = e / M, j = e - i * M;
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < M; ++k) acc = cfma(A[(size_t)i * M + k], B[(size_t)k * M + j], acc);
        C[e] = acc;
    }
    __syncthreads();
}

// C = A * B^dagger
static __device__ void gemm64_nc(const double2 *A, const double2 *B, double2 *C, int M)
{
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        int i = e / M, j = e - i * M;
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < M; ++k) acc = cfma(A[(size_t)i * M + k], cconj(B[(size_t)j * M + k]), acc);
        C[e] = acc;
    }
    __syncthreads();
}

// C = A * Gamma with Gamma = i (S - S^dagger) formed on the fly
static __device__ void gemm64_gamma(const double2 *A, const double2 *S, double2 *C, int M)
{
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        int i = e / M, j = e - i * M;
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < M; ++k) {
            double2 d = csub(S[(size_t)k * M + j], cconj(S[(size_t)j * M + k]));
            acc = cfma(A[(size_t)i * M + k], make_double2(-d.y, d.x), acc);
        }
        C[e] = acc;
    }
    __syncthreads();
}

// Re Tr[Gamma(S) X] = sum_ij Re(Gamma_ij X_ji); result in every thread
static __device__ double trace_gamma64(const double2 *S, const double2 *X, int M, double *red)
{
    double t = 0.0;
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        int i = e / M, j = e - i * M;
        double2 d = csub(S[e], cconj(S[(size_t)j * M + i]));
        double2 g = make_double2(-d.y, d.x);
        double2 x = X[(size_t)j * M + i];
        t += g.x * x.x - g.y * x.y;
    }
    return block_sum(t, red);
}

// (V X V^dagger)_ij for a block-diagonal V with vb x vb blocks
KNIT_DEV double2 vxvd64(const double2 *V, const double2 *X, int M, int vb, int i, int j)
{
    if (vb == 1)
        return cmul(cmul(V[(size_t)i * M + i], X[(size_t)i * M + j]), cconj(V[(size_t)j * M + j]));
    int bi = (i / vb) * vb, bj = (j / vb) * vb;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = bi; k < bi + vb; ++k) {
        double2 vik = V[(size_t)i * M + k];
        if (vik.x == 0.0 && vik.y == 0.0) continue;
        double2 r = make_double2(0.0, 0.0);
        for (int l = bj; l < bj + vb; ++l)
            r = cfma(X[(size_t)k * M + l], cconj(V[(size_t)j * M + l]), r);
        acc = cfma(vik, r, acc);
    }
    return acc;
}

// decimation retries: eta, 100 eta, 1e4 eta, 1e6 eta; a surface g counts as
// converged when it satisfies its fixed point at its own eta to this relative
// max-norm and lies on the retarded branch (i(g - g^dagger) positive
// semidefinite): at eta ~ 1e-12 the doubling can lose enough precision on wide
// leads to land on another solution of the fixed-point equation
constexpr int DEC_ATTEMPTS = 4;
constexpr double DEC_SELF_TOL = 1e-5;

// (V^dagger X V)_ij for a block-diagonal V
KNIT_DEV double2 vdxv64(const double2 *V, const double2 *X, int M, int vb, int i, int j)
{
    if (vb == 1)
        return cmul(cmul(cconj(V[(size_t)i * M + i]), X[(size_t)i * M + j]), V[(size_t)j * M + j]);
    int bi = (i / vb) * vb, bj = (j / vb) * vb;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = bi; k < bi + vb; ++k) {
        double2 vki = cconj(V[(size_t)k * M + i]);
        if (vki.x == 0.0 && vki.y == 0.0) continue;
        double2 r = make_double2(0.0, 0.0);
        for (int l = bj; l < bj + vb; ++l) r = cfma(X[(size_t)k * M + l], V[(size_t)l * M + j], r);
        acc = cfma(vki, r, acc);
    }
    return acc;
}

// C = (A V^dagger) B for a block-diagonal V, i.e. sum_k (A V^dagger)_ik B_kj;
// V's nonzeros lie within `band` of the diagonal (band >= vb: anywhere in the
// block; a tridiagonal V is one block of M with band 1)
static __device__ void gemm64_avd_b(const double2 *A, const double2 *V, int vb, int band,
                                    const double2 *B, double2 *C, int M)
{
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        int i = e / M, j = e - i * M;
        double2 acc = make_double2(0.0, 0.0);
        for (int kb = 0; kb < M; kb += vb) {
            for (int k = kb; k < kb + vb; ++k) {
                // (A V^dagger)_ik = sum_{l in block, |l - k| <= band} A_il conj(V_kl)
                double2 avd = make_double2(0.0, 0.0);
                const int l0 = max(kb, k - band), l1 = min(kb + vb, k + band + 1);
                for (int l = l0; l < l1; ++l)
                    avd = cfma(A[(size_t)i * M + l], cconj(V[(size_t)k * M + l]), avd);
                acc = cfma(avd, B[(size_t)k * M + j], acc);
            }
        }
        C[e] = acc;
    }
    __syncthreads();
}
