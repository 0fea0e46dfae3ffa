// lead_mlp.cu -- learned warm start for the lead fixed point.
//
// A small multilayer perceptron maps the energy to the surface Green function
// of one lead cell: input u = (E - E_mid) / E_half, three hidden layers of 128
// tanh units, linear output of the 2 M^2 real and imaginary parts of g.  It is
// trained on the GPU by the kernels below (forward, backward, Adam) on pairs
// (E, g) that the library's own Sancho-Rubio decimation produces.  Its output
// starts Newton's method on the fixed point of KNIT user guide Sec. 5.3 B,
//     F(g) = A(g) g - I = 0,   A(g) = E - H0 - V g V^dagger (left lead),
// whose Newton step solves A D - V D (V^dagger g) = -F (right lead: V and
// V^dagger exchanged); with D stacked row-wise this is one dense M^2 x M^2
// complex system, solved in FP64 by Gauss-Jordan in shared memory (M <= 8).
// Decimation stays the fallback whenever Newton does not reach the tolerance.
//
// Parameter layout (float): for layer l = 0..3, W_l (out x in, row-major)
// followed by b_l (out).

#include "dense_fp64.cuh"

namespace {

constexpr int TILE = 16;

// Y = act(X W^T + b); X: B x din, W: dout x din, Y: B x dout; act 1 = tanh
__global__ void mlp_linear_fwd(const float *X, int B, int din, const float *W, const float *b,
                               int dout, float *Y, int act)
{
    __shared__ float xs[TILE][TILE + 1], ws[TILE][TILE + 1];
    const int r = blockIdx.y * TILE + threadIdx.y, o = blockIdx.x * TILE + threadIdx.x;
    float acc = 0.f;
    for (int k0 = 0; k0 < din; k0 += TILE) {
        const int kx = k0 + threadIdx.x, ky = k0 + threadIdx.y;
        xs[threadIdx.y][threadIdx.x] = (r < B && kx < din) ? X[(size_t)r * din + kx] : 0.f;
        const int ow = blockIdx.x * TILE + threadIdx.y;
        ws[threadIdx.y][threadIdx.x] = (ow < dout && kx < din) ? W[(size_t)ow * din + kx] : 0.f;
        (void)ky;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TILE; ++k) acc = fmaf(xs[threadIdx.y][k], ws[threadIdx.x][k], acc);
        __syncthreads();
    }
    if (r < B && o < dout) {
        float v = acc + b[o];
        Y[(size_t)r * dout + o] = act ? tanhf(v) : v;
    }
}

// dX = (dY W) * (1 - A^2) where A = tanh output of the previous layer (or no
// factor when prev_act == 0); dY: B x dout, W: dout x din
__global__ void mlp_linear_bwd_in(const float *dY, int B, int dout, const float *W, int din,
                                  const float *A, int prev_act, float *dX)
{
    __shared__ float ds[TILE][TILE + 1], ws[TILE][TILE + 1];
    const int r = blockIdx.y * TILE + threadIdx.y, i = blockIdx.x * TILE + threadIdx.x;
    float acc = 0.f;
    for (int o0 = 0; o0 < dout; o0 += TILE) {
        const int ox = o0 + threadIdx.x, oy = o0 + threadIdx.y;
        ds[threadIdx.y][threadIdx.x] = (r < B && ox < dout) ? dY[(size_t)r * dout + ox] : 0.f;
        ws[threadIdx.y][threadIdx.x] = (oy < dout && i < din) ? W[(size_t)oy * din + i] : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TILE; ++k) acc = fmaf(ds[threadIdx.y][k], ws[k][threadIdx.x], acc);
        __syncthreads();
    }
    if (r < B && i < din) {
        float f = 1.f;
        if (prev_act) {
            const float a = A[(size_t)r * din + i];
            f = 1.f - a * a;
        }
        dX[(size_t)r * din + i] = acc * f;
    }
}

// dW = dY^T X (dout x din), db = column sums of dY; X: B x din
__global__ void mlp_linear_bwd_w(const float *dY, const float *X, int B, int dout, int din,
                                 float *dW, float *db)
{
    __shared__ float ds[TILE][TILE + 1], xs[TILE][TILE + 1];
    const int o = blockIdx.y * TILE + threadIdx.y, i = blockIdx.x * TILE + threadIdx.x;
    float acc = 0.f, accb = 0.f;
    for (int r0 = 0; r0 < B; r0 += TILE) {
        const int rx = r0 + threadIdx.x, ry = r0 + threadIdx.y;
        const int oo = blockIdx.y * TILE + threadIdx.x;
        // ds[k][t] = dY[r0 + k][o-tile t]
        ds[threadIdx.y][threadIdx.x] = (ry < B && oo < dout) ? dY[(size_t)ry * dout + oo] : 0.f;
        xs[threadIdx.y][threadIdx.x] = (ry < B && i < din) ? X[(size_t)ry * din + i] : 0.f;
        (void)rx;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TILE; ++k) {
            const float d = ds[k][threadIdx.y];
            acc = fmaf(d, xs[k][threadIdx.x], acc);
            accb += d;
        }
        __syncthreads();
    }
    if (o < dout && i < din) dW[(size_t)o * din + i] = acc;
    if (o < dout && blockIdx.x == 0 && threadIdx.x == 0) db[o] = accb;
}

// dY = 2 (Y - T) / n, loss += sum (Y - T)^2 / n
__global__ void mlp_mse(const float *Y, const float *T, int n, float *dY, float *loss)
{
    __shared__ float red[8];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < n) {
        const float d = Y[i] - T[i];
        dY[i] = 2.f * d / n;
        l = d * d / n;
    }
    l = warp_sum(l);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s);
    }
}

__global__ void mlp_adam(float *p, const float *g, float *m, float *v, int n, float lr, float b1,
                         float b2, float eps, float c1, float c2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// inputs u = (E - mid) / half (FP64 energies to FP32 features)
__global__ void mlp_inputs(const double *E, const int *idx, int n, double mid, double half, float *U)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) U[i] = (float)((E[idx ? idx[i] : i] - mid) / half);
}

// training targets: the 2 M^2 real parts of g, in float
__global__ void mlp_targets(const double2 *g, const int *idx, int n, int MM, float *Tt)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * MM) return;
    const int r = q / MM, e = q - r * MM;
    const double2 v = g[(size_t)(idx ? idx[r] : r) * MM + e];
    Tt[(size_t)r * 2 * MM + 2 * e] = (float)v.x;
    Tt[(size_t)r * 2 * MM + 2 * e + 1] = (float)v.y;
}

// ---------------------------------------------------------------------------
// Newton refinement of the lead fixed point from the network's guess, one CTA
// per energy, M <= 8 (Jacobian n = M^2 <= 64 in shared memory).  side 0:
// A = E - H0 - V g V^dagger, B = V^dagger g, J D = A D - V D B;
// side 1: A = E - H0 - V^dagger g V, B = V g, J D = A D - V^dagger D B.
// Outputs Sigma, g, iterations and status (ST_NOCONVERGE if the tolerance is
// not met or the result is not retarded: -Im g_kk < 0 for some k).
constexpr int NMAX = 64;

__global__ void __launch_bounds__(256)
lead_newton_kernel(const double2 *H0, const double2 *V, int M, int side, const double *E, int nE,
                   const float *guess, double tol, int maxit, double2 *sigma, double2 *gout,
                   int *iters, int *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *J = reinterpret_cast<double2 *>(smem_raw);   // n x n, dynamic
    __shared__ double2 g[NMAX], A[NMAX], Bm[NMAX], F[NMAX], Vl[NMAX], Vr[NMAX], Dv[NMAX];
    __shared__ double2 row[NMAX], col[NMAX], pval;
    __shared__ int perm[NMAX], flag, piv;
    __shared__ double red[8];
    GJScratch64 sc{row, col, perm, &flag, &piv, &pval};
    const int n = M * M, tid = threadIdx.x;
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        const double En = E[e];
        // Vl = operator on the left of D, Vr^dagger ... : side 0 uses V, side 1 uses V^dagger
        for (int q = tid; q < n; q += blockDim.x) {
            const int i = q / M, j = q - i * M;
            const double2 v = V[q], vd = cconj(V[(size_t)j * M + i]);
            Vl[q] = side == 0 ? v : vd;    // coupling applied on the left
            Vr[q] = side == 0 ? vd : v;    // and its adjoint on the right
            g[q] = make_double2((double)guess[(size_t)e * 2 * n + 2 * q],
                                (double)guess[(size_t)e * 2 * n + 2 * q + 1]);
        }
        __syncthreads();
        int it = 0, st = ST_NOCONVERGE;
        for (it = 0; it <= maxit; ++it) {
            // A = E - H0 - Vl g Vr, B = Vr g
            for (int q = tid; q < n; q += blockDim.x) {
                const int i = q / M, j = q - i * M;
                double2 s = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
                for (int k = 0; k < M; ++k) {
                    double2 t = make_double2(0.0, 0.0);
                    for (int l = 0; l < M; ++l) t = cfma(g[k * M + l], Vr[l * M + j], t);
                    s = cfma(Vl[i * M + k], t, s);
                    b = cfma(Vr[i * M + k], g[k * M + j], b);
                }
                double2 a = make_double2(-H0[q].x - s.x, -H0[q].y - s.y);
                if (i == j) a.x += En;
                A[q] = a;
                Bm[q] = b;
            }
            __syncthreads();
            // F = A g - I and its max norm
            double fm = 0.0;
            for (int q = tid; q < n; q += blockDim.x) {
                const int i = q / M, j = q - i * M;
                double2 s = make_double2(i == j ? -1.0 : 0.0, 0.0);
                for (int k = 0; k < M; ++k) s = cfma(A[i * M + k], g[k * M + j], s);
                F[q] = s;
                fm = fmax(fm, fabs(s.x) + fabs(s.y));
            }
            for (int o = 16; o > 0; o >>= 1) fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, o));
            if ((tid & 31) == 0) red[tid >> 5] = fm;
            __syncthreads();
            double fmax_all = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) fmax_all = fmax(fmax_all, red[w]);
            __syncthreads();
            if (!isfinite(fmax_all)) break;
            if (fmax_all < tol) { st = ST_OK; break; }
            if (it == maxit) break;
            // J[(i,j),(k,l)] = A[i][k] delta(l,j) - Vl[i][k] B[l][j]
            for (int q = tid; q < n * n; q += blockDim.x) {
                const int p = q / n, r = q - p * n;
                const int i = p / M, j = p - i * M, k = r / M, l = r - k * M;
                double2 v = cmul(Vl[i * M + k], Bm[l * M + j]);
                v = make_double2(-v.x, -v.y);
                if (l == j) v = cadd(v, A[i * M + k]);
                J[q] = v;
            }
            __syncthreads();
            if (gj_invert64(J, n, sc) != ST_OK) break;
            // D = -J^{-1} vec(F); g += D
            for (int p = tid; p < n; p += blockDim.x) {
                double2 s = make_double2(0.0, 0.0);
                for (int r = 0; r < n; ++r) s = cfma(J[p * n + r], F[r], s);
                Dv[p] = make_double2(-s.x, -s.y);
            }
            __syncthreads();
            for (int q = tid; q < n; q += blockDim.x) g[q] = cadd(g[q], Dv[q]);
            __syncthreads();
        }
        // retarded branch: the local density -Im g_kk must not be negative
        if (st == ST_OK) {
            int bad = 0;
            for (int k = tid; k < M; k += blockDim.x) bad |= g[k * M + k].y > 1e-12;
            if (__syncthreads_or(bad)) st = ST_NOCONVERGE;
        } else {
            __syncthreads();
        }
        double2 *S = sigma + (size_t)e * n;
        for (int q = tid; q < n; q += blockDim.x) {
            const int i = q / M, j = q - i * M;
            double2 s = make_double2(0.0, 0.0);
            for (int k = 0; k < M; ++k) {
                double2 t = make_double2(0.0, 0.0);
                for (int l = 0; l < M; ++l) t = cfma(g[k * M + l], Vr[l * M + j], t);
                s = cfma(Vl[i * M + k], t, s);
            }
            S[q] = st == ST_OK ? s : make_double2(nan(""), nan(""));
            if (gout) gout[(size_t)e * n + q] = g[q];
        }
        if (tid == 0) {
            if (iters) iters[e] = it;
            if (status) status[e] = st;
        }
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launch helpers (the API lives in knit_api.cu)

extern "C" cudaError_t knit_mlp_linear_fwd(const float *X, int B, int din, const float *W,
                                           const float *b, int dout, float *Y, int act,
                                           cudaStream_t st)
{
    dim3 blk(TILE, TILE), grd((dout + TILE - 1) / TILE, (B + TILE - 1) / TILE);
    mlp_linear_fwd<<<grd, blk, 0, st>>>(X, B, din, W, b, dout, Y, act);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_mlp_linear_bwd(const float *dY, const float *Xin, int B, int din,
                                           const float *W, int dout, float *dW, float *db,
                                           float *dX, int prev_act, cudaStream_t st)
{
    dim3 blk(TILE, TILE);
    dim3 gw((din + TILE - 1) / TILE, (dout + TILE - 1) / TILE);
    mlp_linear_bwd_w<<<gw, blk, 0, st>>>(dY, Xin, B, dout, din, dW, db);
    if (dX) {
        dim3 gx((din + TILE - 1) / TILE, (B + TILE - 1) / TILE);
        mlp_linear_bwd_in<<<gx, blk, 0, st>>>(dY, B, dout, W, din, Xin, prev_act, dX);
    }
    return cudaGetLastError();
}

extern "C" cudaError_t knit_mlp_mse(const float *Y, const float *T, int n, float *dY, float *loss,
                                    cudaStream_t st)
{
    mlp_mse<<<(n + 255) / 256, 256, 0, st>>>(Y, T, n, dY, loss);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_mlp_adam(float *p, const float *g, float *m, float *v, int n, float lr,
                                     int t, cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    mlp_adam<<<(n + 255) / 256, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_mlp_inputs(const double *E, const int *idx, int n, double mid,
                                       double half, float *U, cudaStream_t st)
{
    mlp_inputs<<<(n + 255) / 256, 256, 0, st>>>(E, idx, n, mid, half, U);
    return cudaGetLastError();
}

// targets of a lead solved in blocks: sample r (energy idx[r]) gets every
// block's surface function, block c at 2 nn c; g holds block c of energy e
// at (c nE + e) nn
__global__ void mlp_targets_blocks(const double2 *g, const int *idx, int n, int nsec, int nn, int nE,
                                   float *Tt)
{
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)n * nsec * nn) return;
    const int r = (int)(q / ((long)nsec * nn)), rem = (int)(q - (long)r * nsec * nn);
    const int c = rem / nn, k = rem - c * nn;
    const double2 v = g[((size_t)c * nE + (idx ? idx[r] : r)) * nn + k];
    Tt[(size_t)r * 2 * nsec * nn + 2 * rem] = (float)v.x;
    Tt[(size_t)r * 2 * nsec * nn + 2 * rem + 1] = (float)v.y;
}

// largest |g_ij| over every block of each energy (the training set leaves out
// energies next to a band edge, where g diverges)
__global__ void mlp_block_gmax(const double2 *g, int nsec, int nn, int nE, float *gmax)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    float m = 0.f;
    for (int c = 0; c < nsec; ++c)
        for (int k = 0; k < nn; ++k) {
            const double2 v = g[((size_t)c * nE + e) * nn + k];
            m = fmaxf(m, (float)(fabs(v.x) + fabs(v.y)));
        }
    gmax[e] = m;
}

extern "C" cudaError_t knit_mlp_block_gmax(const double2 *g, int nsec, int nn, int nE, float *gmax,
                                           cudaStream_t st)
{
    mlp_block_gmax<<<(nE + 127) / 128, 128, 0, st>>>(g, nsec, nn, nE, gmax);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_mlp_targets_blocks(const double2 *g, const int *idx, int n, int nsec, int nn,
                                               int nE, float *T, cudaStream_t st)
{
    const long tot = (long)n * nsec * nn;
    mlp_targets_blocks<<<(int)((tot + 255) / 256), 256, 0, st>>>(g, idx, n, nsec, nn, nE, T);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_mlp_targets(const double2 *g, const int *idx, int n, int MM, float *T,
                                        cudaStream_t st)
{
    mlp_targets<<<(n * MM + 255) / 256, 256, 0, st>>>(g, idx, n, MM, T);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_launch_lead_newton(const double2 *H0, const double2 *V, int M, int side,
                                               const double *E, int nE, const float *guess,
                                               double tol, int maxit, double2 *sigma,
                                               double2 *gout, int *iters, int *status, int grid,
                                               cudaStream_t st)
{
    if (M * M > NMAX) return cudaErrorInvalidValue;
    const size_t smb = sizeof(double2) * (size_t)M * M * M * M;
    cudaError_t e = cudaFuncSetAttribute(lead_newton_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    if (e != cudaSuccess) return e;
    lead_newton_kernel<<<grid, 256, smb, st>>>(H0, V, M, side, E, nE, guess, tol, maxit, sigma,
                                               gout, iters, status);
    return cudaGetLastError();
}
