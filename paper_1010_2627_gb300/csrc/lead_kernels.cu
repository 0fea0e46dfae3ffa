// lead_kernels.cu -- lead surface Green functions and self-energies in FP64
// (KNIT user guide Sec. 5.3 B: a lead is the semi-infinite repetition of its
// interface cell H0 with inter-cell hopping V; the hopping to the system is
// the same V).  Left lead: g = (E - H0 - V g V^dagger)^{-1}, Sigma = V g V^dagger;
// right lead: g = (E - H0 - V^dagger g V)^{-1}, Sigma = V^dagger g V.
//
//  * knit_jacobi_kernel: eigen-decomposition H0 = U diag(w) U^dagger of a
//    Hermitian cell by parallel cyclic Jacobi rotations (one CTA, once per
//    lead).  For V = t I every transverse mode k is a 1D chain with the
//    retarded surface function g_k = (x - i sqrt(4|t|^2 - x^2)) / (2|t|^2),
//    x = E - w_k, inside the band and (x - sgn(x) sqrt(x^2 - 4|t|^2)) / (2|t|^2)
//    outside; knit_modes_sigma_kernel assembles Sigma = |t|^2 U diag(g_k) U^dagger.
//  * knit_decimation_kernel: Sancho-Rubio decimation (Lopez Sancho, Lopez
//    Sancho & Rubio 1985) at E + i eta for general cells, one CTA per energy.
//  * knit_lead_residual_kernel: max-norm of g - (E - H0 - V g V^dagger)^{-1}
//    at eta = 0, the fixed-point check of either solver (work: 3 M*M per CTA).

#include <algorithm>
#include "dense_fp64.cuh"

// W = V G V^dagger (side 0) or V^dagger G V (side 1): elementwise for
// block-diagonal V (blocks up to 4), as two products for a dense V (a
// period-2 lead's supercell coupling).  tmp: M*M scratch.  Ends with a barrier.
static __device__ void vgv64(const double2 *V, const double2 *G, int M, int vb, int side,
                             double2 *tmp, double2 *W)
{
    if (vb <= 4) {
        for (int q = threadIdx.x; q < M * M; q += blockDim.x) {
            const int i = q / M, j = q - i * M;
            W[q] = side == 0 ? vxvd64(V, G, M, vb, i, j) : vdxv64(V, G, M, vb, i, j);
        }
        __syncthreads();
        return;
    }
    if (side == 0) {
        gemm64(V, G, tmp, M);       // V G
        gemm64_nc(tmp, V, W, M);    // (V G) V^dagger
        return;
    }
    gemm64(G, V, tmp, M);           // G V
    for (int q = threadIdx.x; q < M * M; q += blockDim.x) {
        const int i = q / M, j = q - i * M;
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < M; ++k) acc = cfma(cconj(V[(size_t)k * M + i]), tmp[(size_t)k * M + j], acc);
        W[q] = acc;
    }
    __syncthreads();
}

// Is the Hermitian matrix A (M x M, row-major, overwritten) positive
// semidefinite up to -tol * max_k A_kk?  Semidefinite Cholesky: a pivot below
// that bound fails; pivots within it end their column (set to zero).  All
// threads of the block call it; red holds 32 doubles.
static __device__ int psd_check64(double2 *A, int M, double *red)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    double dmax = 0.0;
    for (int k = tid; k < M; k += nt) dmax = fmax(dmax, A[(size_t)k * M + k].x);
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = dmax;
    __syncthreads();
    double m = 0.0;
    for (int w = 0; w < nt / 32; ++w) m = fmax(m, red[w]);
    __syncthreads();
    const double tol = 1e-9 * m;
    for (int k = 0; k < M; ++k) {
        const double piv = A[(size_t)k * M + k].x;   // uniform: read after a barrier
        if (!(piv >= -tol)) return 0;
        const double inv = piv > tol ? 1.0 / sqrt(piv) : 0.0;
        for (int i = k + 1 + tid; i < M; i += nt) A[(size_t)i * M + k] = cscale(A[(size_t)i * M + k], inv);
        __syncthreads();
        const int n = M - k - 1;
        for (int e = tid; e < n * n; e += nt) {
            const int i = k + 1 + e / n, j = k + 1 + e % n;
            A[(size_t)i * M + j] = cfms(A[(size_t)i * M + k], cconj(A[(size_t)j * M + k]),
                                        A[(size_t)i * M + j]);
        }
        __syncthreads();
    }
    return 1;
}


// ---------------------------------------------------------------------------
// A (M x M, Hermitian) -> diag in A, eigenvectors in U (global memory).
extern "C" __global__ void __launch_bounds__(256)
knit_jacobi_kernel(double2 *A, double2 *U, int M, int max_sweeps, double tol, int *sweeps_out)
{
    __shared__ double rc[128], rs[128];
    __shared__ double2 rph[128];
    __shared__ int rp[128], rq[128];
    __shared__ double red[8];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Me = M + (M & 1);   // even count with a dummy index M for odd M
    const int npair = Me / 2;
    for (int e = tid; e < M * M; e += nt) {
        int i = e / M, j = e - i * M;
        U[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int e = tid; e < M * M; e += nt) {
            int i = e / M, j = e - i * M;
            double v = fabs(A[e].x) + fabs(A[e].y);
            if (i != j) off = fmax(off, v);
            else dia = fmax(dia, v);
        }
        // block max via shared memory
        for (int o = 16; o > 0; o >>= 1) {
            off = fmax(off, __shfl_xor_sync(0xffffffffu, off, o));
            dia = fmax(dia, __shfl_xor_sync(0xffffffffu, dia, o));
        }
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = off;
        __syncthreads();
        double offm = 0.0;
        for (int w = 0; w < nt / 32; ++w) offm = fmax(offm, red[w]);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = dia;
        __syncthreads();
        double diam = 0.0;
        for (int w = 0; w < nt / 32; ++w) diam = fmax(diam, red[w]);
        __syncthreads();
        if (offm <= tol * fmax(diam, 1e-300) || offm == 0.0) break;
        for (int r = 0; r < Me - 1; ++r) {
            // round-robin pairing: slot 0 fixed, slots 1..Me-1 rotate by r
            for (int t = tid; t < npair; t += nt) {
                int a = t == 0 ? 0 : 1 + (t - 1 + r) % (Me - 1);
                int bslot = Me - 1 - t;
                int b = 1 + (bslot - 1 + r) % (Me - 1);
                int p = min(a, b), q = max(a, b);
                double c = 1.0, sn = 0.0;
                double2 ph = make_double2(1.0, 0.0);
                if (q < M) {
                    double2 apq = A[(size_t)p * M + q];
                    double rr = hypot(apq.x, apq.y);
                    if (rr > 0.0) {
                        ph = make_double2(apq.x / rr, apq.y / rr);
                        double tau = (A[(size_t)q * M + q].x - A[(size_t)p * M + p].x) / (2.0 * rr);
                        double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        sn = tt * c;
                    }
                }
                rp[t] = p;
                rq[t] = q;
                rc[t] = c;
                rs[t] = sn;
                rph[t] = ph;
            }
            __syncthreads();
            // columns: A <- A W, U <- U W with W = [[c, s], [-s e^{-i phi}, c e^{-i phi}]]
            for (int e = tid; e < npair * M; e += nt) {
                int t = e / M, i = e - t * M;
                int p = rp[t], q = rq[t];
                if (q >= M) continue;
                double c = rc[t], sn = rs[t];
                double2 phc = cconj(rph[t]);
                for (int w = 0; w < 2; ++w) {
                    double2 *X = w == 0 ? A : U;
                    double2 xp = X[(size_t)i * M + p], xq = X[(size_t)i * M + q];
                    double2 xqp = cmul(phc, xq);
                    X[(size_t)i * M + p] = make_double2(c * xp.x - sn * xqp.x, c * xp.y - sn * xqp.y);
                    X[(size_t)i * M + q] = make_double2(sn * xp.x + c * xqp.x, sn * xp.y + c * xqp.y);
                }
            }
            __syncthreads();
            // rows: A <- W^dagger A
            for (int e = tid; e < npair * M; e += nt) {
                int t = e / M, j = e - t * M;
                int p = rp[t], q = rq[t];
                if (q >= M) continue;
                double c = rc[t], sn = rs[t];
                double2 ph = rph[t];
                double2 ap = A[(size_t)p * M + j], aq = A[(size_t)q * M + j];
                double2 aqp = cmul(ph, aq);
                A[(size_t)p * M + j] = make_double2(c * ap.x - sn * aqp.x, c * ap.y - sn * aqp.y);
                A[(size_t)q * M + j] = make_double2(sn * ap.x + c * aqp.x, sn * ap.y + c * aqp.y);
            }
            __syncthreads();
        }
    }
    if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// ---------------------------------------------------------------------------
// Sigma(E_e) = |t|^2 U diag(g_k(E_e - w_k)) U^dagger, one CTA per energy (grid-stride)
extern "C" __global__ void __launch_bounds__(256)
knit_modes_sigma_kernel(const double2 *U, const double2 *Adiag, int M, double t2, const double *E,
                        int nE, double2 *sigma, double2 *gout)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *gk = reinterpret_cast<double2 *>(smem_raw);
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        const double En = E[e];
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            double x = En - Adiag[(size_t)k * M + k].x;
            double b = 4.0 * t2;
            double2 g;
            if (x * x < b) g = make_double2(x / (2.0 * t2), -sqrt(b - x * x) / (2.0 * t2));
            else g = make_double2((x - copysign(sqrt(x * x - b), x)) / (2.0 * t2), 0.0);
            gk[k] = g;
        }
        __syncthreads();
        double2 *S = sigma + (size_t)e * M * M;
        double2 *G = gout ? gout + (size_t)e * M * M : nullptr;
        for (int q = threadIdx.x; q < M * M; q += blockDim.x) {
            int i = q / M, j = q - i * M;
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < M; ++k)
                acc = cfma(cmul(U[(size_t)i * M + k], gk[k]), cconj(U[(size_t)j * M + k]), acc);
            S[q] = cscale(acc, t2);
            if (G) G[q] = acc;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Sancho-Rubio decimation, one CTA per energy (grid-stride).  side 0: alpha = V
// (surface -> next cell outward), beta = V^dagger; side 1: the reverse.
// work: per CTA 8 M*M complex.  Outputs Sigma, g, iterations, status.
extern "C" __global__ void __launch_bounds__(256)
knit_decimation_kernel(const double2 *H0, const double2 *V, int M, int vb, int side, const double *E,
                       int nE, double eta, double tol, int maxit, double2 *work, double2 *sigma,
                       double2 *gout, int *iters, int *status, int only_failed)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GJScratch64 sc;
    unsigned char *p = smem_raw;
    sc.row = reinterpret_cast<double2 *>(p);
    p += sizeof(double2) * M;
    sc.col = reinterpret_cast<double2 *>(p);
    p += sizeof(double2) * M;
    sc.pval = reinterpret_cast<double2 *>(p);
    p += sizeof(double2);
    double *red = reinterpret_cast<double *>(p);
    p += sizeof(double) * 32;
    sc.perm = reinterpret_cast<int *>(p);
    p += sizeof(int) * M;
    sc.flag = reinterpret_cast<int *>(p);
    p += sizeof(int);
    sc.piv = reinterpret_cast<int *>(p);

    const size_t MM = (size_t)M * M;
    double2 *w = work + (size_t)blockIdx.x * 8 * MM;
    double2 *eps = w, *eps_s = w + MM, *al = w + 2 * MM, *be = w + 3 * MM;
    double2 *gb = w + 4 * MM, *t1 = w + 5 * MM, *t2 = w + 6 * MM, *t3 = w + 7 * MM;
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        if (only_failed && status[e] == ST_OK) continue;   // uniform over the block
        double2 *S = sigma + (size_t)e * MM;
        double2 *G = gout + (size_t)e * MM;
        int it = 0, st = ST_NOCONVERGE;
        // decimation at E + i eta; if the surface g does not satisfy its own
        // fixed point at that eta (the doubling lost precision, which wide
        // leads with many slow modes meet at eta ~ 1e-13), again at 100x eta
        double eta_k = eta;
        for (int attempt = 0; attempt < DEC_ATTEMPTS; ++attempt, eta_k *= 100.0) {
        const double2 z = make_double2(E[e], eta_k);
        for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
            int i = q / M, j = q - i * M;
            double2 v = V[q], vd = cconj(V[(size_t)j * M + i]);
            eps[q] = H0[q];
            eps_s[q] = H0[q];
            al[q] = side == 0 ? v : vd;
            be[q] = side == 0 ? vd : v;
        }
        __syncthreads();
        st = ST_NOCONVERGE;
        for (it = 0; it < maxit; ++it) {
            double na = 0.0, nb = 0.0;
            for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
                na = fmax(na, hypot(al[q].x, al[q].y));
                nb = fmax(nb, hypot(be[q].x, be[q].y));
            }
            for (int o = 16; o > 0; o >>= 1) {
                na = fmax(na, __shfl_xor_sync(0xffffffffu, na, o));
                nb = fmax(nb, __shfl_xor_sync(0xffffffffu, nb, o));
            }
            __syncthreads();
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = na + 0.0 * nb;
            if ((threadIdx.x & 31) == 0) red[16 + (threadIdx.x >> 5)] = nb;
            __syncthreads();
            double mna = 0.0, mnb = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                mna = fmax(mna, red[q]);
                mnb = fmax(mnb, red[16 + q]);
            }
            __syncthreads();
            if (mna + mnb < tol) { st = ST_OK; break; }
            if (!isfinite(mna + mnb)) break;
            // gb = (z - eps)^{-1}
            for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
                int i = q / M, j = q - i * M;
                double2 v = make_double2(-eps[q].x, -eps[q].y);
                if (i == j) v = cadd(v, z);
                gb[q] = v;
            }
            __syncthreads();
            if (gj_invert64(gb, M, sc) != ST_OK) { st = ST_SINGULAR; break; }
            gemm64(gb, be, t1, M);    // gb beta
            gemm64(gb, al, t2, M);    // gb alpha
            gemm64(al, t1, t3, M);    // alpha gb beta
            for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
                eps_s[q] = cadd(eps_s[q], t3[q]);
                eps[q] = cadd(eps[q], t3[q]);
            }
            __syncthreads();
            gemm64(be, t2, t3, M);    // beta gb alpha
            for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) eps[q] = cadd(eps[q], t3[q]);
            __syncthreads();
            gemm64(al, t2, t3, M);    // alpha gb alpha -> new alpha (after beta update)
            gemm64(be, t1, t2, M);    // beta gb beta
            for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
                al[q] = t3[q];
                be[q] = t2[q];
            }
            __syncthreads();
        }
        if (st == ST_OK) {
            for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
                int i = q / M, j = q - i * M;
                double2 v = make_double2(-eps_s[q].x, -eps_s[q].y);
                if (i == j) v = cadd(v, z);
                G[q] = v;
            }
            __syncthreads();
            if (gj_invert64(G, M, sc) != ST_OK) st = ST_SINGULAR;
        }
        if (st == ST_OK) {
            // self-consistency at z: t1 = (z - H0 - V g V^dagger)^{-1} (left;
            // right with V^dagger, V) against g, relative max-norm
            vgv64(V, G, M, vb, side, t2, t3);
            for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
                int i = q / M, j = q - i * M;
                double2 v = make_double2(-H0[q].x - t3[q].x, -H0[q].y - t3[q].y);
                if (i == j) v = cadd(v, z);
                t1[q] = v;
            }
            __syncthreads();
            if (gj_invert64(t1, M, sc) != ST_OK) {
                st = ST_SINGULAR;
            } else {
                // dm: fixed-point mismatch; gm: size of g; plus the retarded
                // branch, whose diagonal of i(g - g^dagger) = -2 Im g_kk is >= 0
                // (the doubling can also land on a non-retarded fixed point)
                double dm = 0.0, gm = 0.0;
                for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
                    dm = fmax(dm, cabs1(csub(t1[q], G[q])));
                    gm = fmax(gm, cabs1(G[q]));
                }
                for (int k = threadIdx.x; k < M; k += blockDim.x)
                    if (G[(size_t)k * M + k].y > 0.0) dm = INFINITY;
                for (int o = 16; o > 0; o >>= 1) {
                    dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
                    gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
                }
                __syncthreads();
                if ((threadIdx.x & 31) == 0) {
                    red[threadIdx.x >> 5] = dm;
                    red[16 + (threadIdx.x >> 5)] = gm;
                }
                __syncthreads();
                double mdm = 0.0, mgm = 0.0;
                for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                    mdm = fmax(mdm, red[q]);
                    mgm = fmax(mgm, red[16 + q]);
                }
                __syncthreads();
                if (!(mdm <= DEC_SELF_TOL * mgm)) st = ST_NOCONVERGE;   // also NaN
            }
        }
        if (st == ST_OK) {
            // the whole retarded condition: i(g - g^dagger) positive semidefinite
            for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
                const int i = q / M, j = q - i * M;
                const double2 a = G[q], b = cconj(G[(size_t)j * M + i]);
                t2[q] = make_double2(-(a.y - b.y), a.x - b.x);   // i (a - b)
            }
            __syncthreads();
            if (!psd_check64(t2, M, red)) st = ST_NOCONVERGE;
        }
        if (st == ST_OK) break;
        }
        if (st == ST_OK) {
            // Sigma = alpha0 g beta0: left V g V^dagger, right V^dagger g V
            vgv64(V, G, M, vb, side, t1, S);
        } else {
            for (int q = threadIdx.x; q < (int)MM; q += blockDim.x)
                S[q] = make_double2(nan(""), nan(""));
        }
        if (threadIdx.x == 0) {
            if (iters) iters[e] = it;
            if (status) status[e] = st;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// residual[e] = max |g - (E - H0 - V g V^dagger)^{-1}| (side 0) or with
// V^dagger g V (side 1), at eta = 0.  work: per CTA 1 M*M complex.
extern "C" __global__ void __launch_bounds__(256)
knit_lead_residual_kernel(const double2 *H0, const double2 *V, int M, int vb, int side, const double *E,
                          int nE, const double2 *g, double2 *work, double *residual)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GJScratch64 sc;
    unsigned char *p = smem_raw;
    sc.row = reinterpret_cast<double2 *>(p);
    p += sizeof(double2) * M;
    sc.col = reinterpret_cast<double2 *>(p);
    p += sizeof(double2) * M;
    sc.pval = reinterpret_cast<double2 *>(p);
    p += sizeof(double2);
    double *red = reinterpret_cast<double *>(p);
    p += sizeof(double) * 32;
    sc.perm = reinterpret_cast<int *>(p);
    p += sizeof(int) * M;
    sc.flag = reinterpret_cast<int *>(p);
    p += sizeof(int);
    sc.piv = reinterpret_cast<int *>(p);
    const size_t MM = (size_t)M * M;
    double2 *A = work + (size_t)blockIdx.x * 3 * MM, *tmp = A + MM, *Wv = A + 2 * MM;
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        const double2 *ge = g + (size_t)e * MM;
        vgv64(V, ge, M, vb, side, tmp, Wv);
        for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
            int i = q / M, j = q - i * M;
            double2 v = csub(make_double2(-H0[q].x, -H0[q].y), Wv[q]);
            if (i == j) v.x += E[e];
            A[q] = v;
        }
        __syncthreads();
        double r = 0.0;
        if (gj_invert64(A, M, sc) != ST_OK) {
            r = INFINITY;
        } else {
            for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
                double2 d = csub(A[q], ge[q]);
                r = fmax(r, hypot(d.x, d.y));
            }
        }
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, red[q]);
            residual[e] = m;
        }
        __syncthreads();
    }
}

extern "C" size_t knit_gj_smem_bytes(int M)
{
    return (size_t)M * sizeof(double2) * 2 + sizeof(double2) + sizeof(double) * 32 +
           sizeof(int) * (M + 2) + 64;
}

// host launch helpers used by the C-ABI implementation
extern "C" cudaError_t knit_launch_jacobi(double2 *A, double2 *U, int M, int *sweeps,
                                          cudaStream_t stream)
{
    knit_jacobi_kernel<<<1, 256, 0, stream>>>(A, U, M, 60, 1e-15, sweeps);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_launch_modes_sigma(const double2 *U, const double2 *A, int M, double t2,
                                               const double *E, int nE, double2 *sigma,
                                               double2 *g, int grid, cudaStream_t stream)
{
    knit_modes_sigma_kernel<<<grid, 256, sizeof(double2) * M, stream>>>(U, A, M, t2, E, nE,
                                                                         sigma, g);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_launch_decimation(const double2 *H0, const double2 *V, int M, int vb,
                                              int side, const double *E, int nE, double eta,
                                              double tol, int maxit, double2 *work,
                                              double2 *sigma, double2 *g, int *iters,
                                              int *status, int grid, cudaStream_t stream)
{
    knit_decimation_kernel<<<grid, 256, knit_gj_smem_bytes(M), stream>>>(
        H0, V, M, vb, side, E, nE, eta, tol, maxit, work, sigma, g, iters, status, 0);
    return cudaGetLastError();
}

// decimation of only the energies whose status is not ST_OK (fallback after
// the learned start); their iteration counts are overwritten
extern "C" cudaError_t knit_launch_decimation_failed(const double2 *H0, const double2 *V, int M,
                                                     int vb, int side, const double *E, int nE,
                                                     double eta, double tol, int maxit,
                                                     double2 *work, double2 *sigma, double2 *g,
                                                     int *iters, int *status, int grid,
                                                     cudaStream_t stream)
{
    knit_decimation_kernel<<<grid, 256, knit_gj_smem_bytes(M), stream>>>(
        H0, V, M, vb, side, E, nE, eta, tol, maxit, work, sigma, g, iters, status, 1);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_launch_lead_residual(const double2 *H0, const double2 *V, int M, int vb,
                                                 int side, const double *E, int nE,
                                                 const double2 *g, double2 *work,
                                                 double *residual, int grid, cudaStream_t stream)
{
    knit_lead_residual_kernel<<<grid, 256, knit_gj_smem_bytes(M), stream>>>(H0, V, M, vb, side, E,
                                                                            nE, g, work, residual);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Self-energy on the system's end slice from a two-slice supercell lead:
// g11 = the surface slice's block of the supercell surface function gcell
// (Mp x Mp, Mp = 2M, per energy); left Sigma = C g11 C^dagger, right
// Sigma = C^dagger g11 C.  One CTA per energy (grid-stride), tmp: M*M per CTA.
extern "C" __global__ void __launch_bounds__(256)
knit_sigma_block_kernel(const double2 *C, const double2 *gcell, int M, int Mp, int side, int nE,
                        double2 *tmp, double2 *sigma)
{
    const size_t MM = (size_t)M * M, MMp = (size_t)Mp * Mp;
    double2 *T = tmp + (size_t)blockIdx.x * MM;
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        const double2 *g = gcell + (size_t)e * MMp;
        // T = C g11 (left) or C^dagger g11 (right)
        for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
            const int i = q / M, j = q - i * M;
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < M; ++k) {
                const double2 c = side == 0 ? C[(size_t)i * M + k] : cconj(C[(size_t)k * M + i]);
                acc = cfma(c, g[(size_t)k * Mp + j], acc);
            }
            T[q] = acc;
        }
        __syncthreads();
        // Sigma = T C^dagger (left) or T C (right)
        double2 *S = sigma + (size_t)e * MM;
        for (int q = threadIdx.x; q < (int)MM; q += blockDim.x) {
            const int i = q / M, j = q - i * M;
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < M; ++k) {
                const double2 c = side == 0 ? cconj(C[(size_t)j * M + k]) : C[(size_t)k * M + j];
                acc = cfma(T[(size_t)i * M + k], c, acc);
            }
            S[q] = acc;
        }
        __syncthreads();
    }
}

extern "C" cudaError_t knit_launch_sigma_block(const double2 *C, const double2 *gcell, int M, int Mp,
                                               int side, int nE, double2 *tmp, double2 *sigma,
                                               int grid, cudaStream_t stream)
{
    knit_sigma_block_kernel<<<grid, 256, 0, stream>>>(C, gcell, M, Mp, side, nE, tmp, sigma);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Leads whose cell splits into sectors: when the orbitals of a lead cell fall
// into groups that neither H0 nor V connects (the electron and hole halves of
// a normal Nambu lead), the surface g of Sec. 5.3 B is block-diagonal in that
// grouping and each block solves the fixed point of its own sector.  The host
// decimates every sector alone (an (M / k)^3 problem each) and these kernels
// put the blocks back: out[e][idx[s ms + a]][idx[s ms + b]] = blk[s][e][a][b],
// zero between sectors.

__global__ void sector_zero_kernel(size_t n, double2 *out)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        out[q] = make_double2(0.0, 0.0);
}

__global__ void sector_place_kernel(const double2 *blk, const int *idx, int nsec, int ms, int M,
                                    int nE, double2 *out)
{
    const size_t MM = (size_t)M * M, mm = (size_t)ms * ms;
    const size_t total = (size_t)nsec * nE * mm;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(q / ((size_t)nE * mm));
        const size_t rem = q - (size_t)s * nE * mm;
        const int e = (int)(rem / mm);
        const int ab = (int)(rem - (size_t)e * mm);
        const int a = ab / ms, b = ab - a * ms;
        out[(size_t)e * MM + (size_t)idx[s * ms + a] * M + idx[s * ms + b]] = blk[q];
    }
}

// per energy: the largest status and iteration count over the sectors
__global__ void sector_status_kernel(const int *st, const int *it, int nsec, int nE, int *st_out,
                                     int *it_out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    int s0 = 0, i0 = 0;
    for (int s = 0; s < nsec; ++s) {
        s0 = max(s0, st[(size_t)s * nE + e]);
        i0 = max(i0, it[(size_t)s * nE + e]);
    }
    if (st_out) st_out[e] = s0;
    if (it_out) it_out[e] = i0;
}

// a sector's Sigma or g from its mode blocks: out[e] = U diag(blk_0[e], ..,
// blk_{nb-1}[e]) U^dagger, ms = nb mu, block r of energy e at blk + (r nE +
// e) mu^2, U (ms x ms) with the modes of block r in columns r mu .. r mu +
// mu - 1; one CTA per energy (grid-stride), T = U diag(.) in a per-CTA
// scratch of ms^2
__global__ void __launch_bounds__(256)
sector_unmode_kernel(const double2 *blk, const double2 *U, int nb, int mu, int nE, double2 *scratch,
                     double2 *out)
{
    const int ms = nb * mu;
    const size_t mm = (size_t)ms * ms, uu = (size_t)mu * mu;
    double2 *T = scratch + (size_t)blockIdx.x * mm;
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        for (int q = threadIdx.x; q < (int)mm; q += blockDim.x) {
            const int i = q / ms, c = q - i * ms, r = c / mu, b = c - r * mu;
            const double2 *B = blk + ((size_t)r * nE + e) * uu;
            const double2 *Ui = U + (size_t)i * ms + r * mu;
            double2 acc = make_double2(0.0, 0.0);
            for (int a = 0; a < mu; ++a) acc = cfma(Ui[a], B[(size_t)a * mu + b], acc);
            T[q] = acc;
        }
        __syncthreads();
        double2 *O = out + (size_t)e * mm;
        for (int q = threadIdx.x; q < (int)mm; q += blockDim.x) {
            const int i = q / ms, j = q - i * ms;
            double2 acc = make_double2(0.0, 0.0);
            for (int c = 0; c < ms; ++c)
                acc = cfma(T[(size_t)i * ms + c], cconj(U[(size_t)j * ms + c]), acc);
            O[q] = acc;
        }
        __syncthreads();
    }
}

// a particle-hole pair of sectors from the first sector alone: src holds the
// first sector at nE + nX energies (the caller's nE first, then the extra
// energies -E that the list lacks), map[e] the index of -E_e there; out gets
// both sectors at the caller's energies, block 0 = src[e], block 1 =
// -S conj(src[map[e]]) S^dagger, S = 1 (x) i sigma_y on orbital pairs:
// X1[a][b] = -(-1)^(a + b) conj(X0[a ^ 1][b ^ 1])
__global__ void sector_ph_kernel(const double2 *src, const int *map, int ms, int nE, double2 *out)
{
    const size_t mm = (size_t)ms * ms, total = (size_t)nE * mm;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(q / mm), ab = (int)(q - (size_t)e * mm), a = ab / ms, b = ab - a * ms;
        out[q] = src[q];
        const double2 x = src[(size_t)map[e] * mm + (size_t)(a ^ 1) * ms + (b ^ 1)];
        const double sg = ((a + b) & 1) ? 1.0 : -1.0;
        out[total + q] = make_double2(sg * x.x, -sg * x.y);
    }
}

__global__ void sector_ph_status_kernel(const int *st, const int *it, const int *map, int nE, int *st_out,
                                        int *it_out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    st_out[e] = st[e];
    it_out[e] = it[e];
    st_out[nE + e] = st[map[e]];
    it_out[nE + e] = it[map[e]];
}

extern "C" cudaError_t knit_launch_sector_ph(const double2 *src, const int *map, int ms, int nE,
                                             double2 *out, cudaStream_t stream)
{
    const size_t total = (size_t)nE * ms * ms;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 65535);
    sector_ph_kernel<<<grid, 256, 0, stream>>>(src, map, ms, nE, out);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_launch_sector_ph_status(const int *st, const int *it, const int *map, int nE,
                                                    int *st_out, int *it_out, cudaStream_t stream)
{
    sector_ph_status_kernel<<<(nE + 255) / 256, 256, 0, stream>>>(st, it, map, nE, st_out, it_out);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_launch_sector_assemble(const double2 *blk, const int *idx, int nsec,
                                                   int ms, int M, int nE, double2 *out,
                                                   cudaStream_t stream)
{
    const int threads = 256;
    const size_t n0 = (size_t)nE * M * M, n1 = (size_t)nsec * nE * ms * ms;
    const int g0 = (int)std::min<size_t>((n0 + threads - 1) / threads, 65535);
    const int g1 = (int)std::min<size_t>((n1 + threads - 1) / threads, 65535);
    sector_zero_kernel<<<g0, threads, 0, stream>>>(n0, out);
    sector_place_kernel<<<g1, threads, 0, stream>>>(blk, idx, nsec, ms, M, nE, out);
    return cudaGetLastError();
}

extern "C" cudaError_t knit_launch_sector_status(const int *st, const int *it, int nsec, int nE,
                                                 int *st_out, int *it_out, cudaStream_t stream)
{
    sector_status_kernel<<<(nE + 255) / 256, 256, 0, stream>>>(st, it, nsec, nE, st_out, it_out);
    return cudaGetLastError();
}

// scratch: ms^2 complex per CTA, for min(grid, nE) CTAs
extern "C" cudaError_t knit_launch_sector_unmode(const double2 *blk, const double2 *U, int nb, int mu,
                                                 int nE, double2 *scratch, double2 *out, int grid,
                                                 cudaStream_t stream)
{
    if (nE <= 0) return cudaSuccess;
    sector_unmode_kernel<<<std::min(grid, nE), 256, 0, stream>>>(blk, U, nb, mu, nE, scratch, out);
    return cudaGetLastError();
}
