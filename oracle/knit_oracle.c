/*
 * knit_oracle.c -- plain, slow, FP64 CPU oracle for the two-terminal KNIT problem.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  It shares no
 * code, header, table or helper with the CUDA library under
 * paper_1010_2627_gb300/ and must never be called from the product path.
 *
 * What it computes (KNIT user guide, Sec. 2.3):
 *   - Eq. (1): a tight-binding Hamiltonian H with m x m blocks per site, here
 *     organised in L slices of M orbitals: diagonal blocks H_n, inter-slice
 *     blocks H_{n,n-1} = V_n and H_{n-1,n} = V_n^dagger.
 *   - Eq. (2): the retarded Green function of the system with its leads,
 *     G = (E - H - Sigma_L - Sigma_R)^{-1}.  The garbled "+ i Sigma" sign of
 *     Eq. (2) is read as the textbook retarded form with Im Sigma <= 0.
 *   - Sec. 2.3 transmission: T_kl = Tr[G_kl Gamma_l G_kl^dagger Gamma_k], with
 *     Gamma = i (Sigma - Sigma^dagger) (the text's "Gamma = Im Sigma" loses the
 *     factor -2 and the Hermitian form; with it a clean chain would give T = 1/4).
 *   - Local density of states -Im G_ii / pi ("single particle density",
 *     Sec. 2.1 b).
 *   - Sec. 5.3 B: a lead is the semi-infinite repetition of its interface slice;
 *     the system-to-lead hopping equals the lead's own inter-slice hopping.
 *     Left lead:  g_L = (E - H0 - V g_L V^dagger)^{-1},  Sigma_L = V g_L V^dagger.
 *     Right lead: g_R = (E - H0 - V^dagger g_R V)^{-1}, Sigma_R = V^dagger g_R V.
 *
 * Functions:
 *   orc_lu_factor / orc_lu_solve   complex LU with partial pivoting (pivot =
 *                                  largest |Re|+|Im|, lowest row on ties)
 *   orc_onsite                     counter-based Anderson disorder (SplitMix64)
 *   orc_sigma_square               closed-form self-energy of a clean square-
 *                                  lattice lead via its transverse modes
 *   orc_lead_decimation            Sancho-Rubio decimation of a general lead
 *   orc_dense                      the plain definition: assemble the dense
 *                                  (E - H - Sigma) of the whole system, LU-solve
 *   orc_rgf                        the method itself in slice form (Sec. 5.3 D,
 *                                  knitting; sewing for the diagonal), plain loops
 *   orc_rgf_batch                  orc_rgf over many instances (OpenMP), the
 *                                  timed CPU baseline
 *
 * Layout conventions: complex numbers are (re, im) pairs of doubles, matrices
 * are row-major, slice index n runs 0..L-1, orbital index x runs 0..M-1.
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_OK 0
#define ORC_ERR_SINGULAR 4
#define ORC_ERR_NOCONVERGE 5
#define ORC_ERR_INVALID 1
#define ORC_ERR_OOM 2

static double cabs1(cplx z) { return fabs(creal(z)) + fabs(cimag(z)); }

/* ------------------------------------------------------------------------ */
/* Complex LU with partial pivoting.  A (N x N, row-major) is overwritten by
 * L (unit lower, below the diagonal) and U; perm[k] is the row swapped into
 * position k at step k.  Returns 0, or k+1 if the pivot at step k is zero. */
int orc_lu_factor(int N, cplx *A, int *perm)
{
    for (int k = 0; k < N; ++k) {
        int p = k;
        double best = cabs1(A[(size_t)k * N + k]);
        for (int i = k + 1; i < N; ++i) {
            double v = cabs1(A[(size_t)i * N + k]);
            if (v > best) { best = v; p = i; }
        }
        perm[k] = p;
        if (best == 0.0) return k + 1;
        if (p != k) {
            for (int j = 0; j < N; ++j) {
                cplx t = A[(size_t)k * N + j];
                A[(size_t)k * N + j] = A[(size_t)p * N + j];
                A[(size_t)p * N + j] = t;
            }
        }
        cplx piv = A[(size_t)k * N + k];
        for (int i = k + 1; i < N; ++i) {
            cplx l = A[(size_t)i * N + k] / piv;
            A[(size_t)i * N + k] = l;
            if (l == 0.0) continue;
            for (int j = k + 1; j < N; ++j)
                A[(size_t)i * N + j] -= l * A[(size_t)k * N + j];
        }
    }
    return 0;
}

/* Solve A X = B in place for B (N x nrhs, row-major) with the factors above. */
void orc_lu_solve(int N, const cplx *LU, const int *perm, cplx *B, int nrhs)
{
    for (int k = 0; k < N; ++k) {
        int p = perm[k];
        if (p != k)
            for (int j = 0; j < nrhs; ++j) {
                cplx t = B[(size_t)k * nrhs + j];
                B[(size_t)k * nrhs + j] = B[(size_t)p * nrhs + j];
                B[(size_t)p * nrhs + j] = t;
            }
    }
    for (int i = 0; i < N; ++i)            /* forward: unit lower */
        for (int k = 0; k < i; ++k) {
            cplx l = LU[(size_t)i * N + k];
            if (l == 0.0) continue;
            for (int j = 0; j < nrhs; ++j) B[(size_t)i * nrhs + j] -= l * B[(size_t)k * nrhs + j];
        }
    for (int i = N - 1; i >= 0; --i) {     /* backward: upper */
        for (int k = i + 1; k < N; ++k) {
            cplx u = LU[(size_t)i * N + k];
            if (u == 0.0) continue;
            for (int j = 0; j < nrhs; ++j) B[(size_t)i * nrhs + j] -= u * B[(size_t)k * nrhs + j];
        }
        cplx d = LU[(size_t)i * N + i];
        for (int j = 0; j < nrhs; ++j) B[(size_t)i * nrhs + j] /= d;
    }
}

/* Inverse of an M x M matrix (A is destroyed).  Returns 0 or ORC_ERR_SINGULAR. */
static int inverse(int M, cplx *A, cplx *Ainv, int *perm)
{
    if (orc_lu_factor(M, A, perm)) return ORC_ERR_SINGULAR;
    memset(Ainv, 0, sizeof(cplx) * (size_t)M * M);
    for (int i = 0; i < M; ++i) Ainv[(size_t)i * M + i] = 1.0;
    orc_lu_solve(M, A, perm, Ainv, M);
    return ORC_OK;
}

/* C = op(A) op(B) with op = identity or conjugate transpose ('N' / 'C'). */
static void matmul(int M, const cplx *A, char ta, const cplx *B, char tb, cplx *C)
{
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            cplx s = 0.0;
            for (int k = 0; k < M; ++k) {
                cplx a = (ta == 'N') ? A[(size_t)i * M + k] : conj(A[(size_t)k * M + i]);
                cplx b = (tb == 'N') ? B[(size_t)k * M + j] : conj(B[(size_t)j * M + k]);
                s += a * b;
            }
            C[(size_t)i * M + j] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* Anderson disorder (Sec. 6.1, "Introducing disorder": on-site energy
 * W (r - 1/2) with r uniform in [0,1)).  The paper draws r from Python's
 * Mersenne Twister in site order; here r comes from a counter keyed by
 * (seed, slice n, site x) so that any implementation reproduces it:
 * SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) applied twice,
 *   r = (mix(mix(seed) xor (n * 2^32 + x)) >> 11) * 2^-53. */
uint64_t orc_splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double orc_onsite(uint64_t seed, int n, int x, double W)
{
    uint64_t key = ((uint64_t)(uint32_t)n << 32) | (uint64_t)(uint32_t)x;
    uint64_t r = orc_splitmix64(orc_splitmix64(seed) ^ key);
    double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    return W * (u - 0.5);
}

/* Fill eps[n*M + x] for a slice system of L slices and M orbitals with
 * `block` orbitals per site: the site draws one value and component c of the
 * site receives sign[c] times it (for spin x Nambu blocks the hole
 * components carry -eps). */
void orc_onsite_fill(uint64_t seed, int L, int M, int block, const double *sign,
                     double W, double *eps)
{
    for (int n = 0; n < L; ++n)
        for (int x = 0; x < M; ++x) {
            int site = x / block, c = x % block;
            eps[(size_t)n * M + x] = sign[c] * orc_onsite(seed, n, site, W);
        }
}

/* ------------------------------------------------------------------------ */
/* Closed-form self-energy of a clean square-lattice lead of width M, hopping
 * t (Sec. 5.3 B lead = repeated interface slice; textbook transverse modes).
 * Transverse modes phi_k(y) = sqrt(2/(M+1)) sin(k pi y/(M+1)), energies
 * e_k = 2 t cos(k pi/(M+1)).  Each mode is a 1D chain whose retarded surface
 * function is g(x) = (x - i sqrt(4t^2 - x^2))/(2t^2) inside the band and
 * (x - sgn(x) sqrt(x^2 - 4t^2))/(2t^2) outside, with x = E - e_k.
 * Sigma = t^2 sum_k phi_k phi_k^T g(E - e_k).  Same for both leads. */
void orc_sigma_square(int M, double t, double E, cplx *Sigma)
{
    double *phi = (double *)malloc(sizeof(double) * (size_t)M * M);
    cplx *gk = (cplx *)malloc(sizeof(cplx) * (size_t)M);
    double nrm = sqrt(2.0 / (M + 1));
    for (int y = 0; y < M; ++y)
        for (int k = 0; k < M; ++k)
            phi[(size_t)y * M + k] = nrm * sin((double)(y + 1) * (k + 1) * M_PI / (M + 1));
    for (int k = 0; k < M; ++k) {
        double ek = 2.0 * t * cos((k + 1) * M_PI / (M + 1));
        double x = E - ek, b = 4.0 * t * t;
        if (x * x < b) gk[k] = (x - I * sqrt(b - x * x)) / (2.0 * t * t);
        else gk[k] = (x - copysign(sqrt(x * x - b), x)) / (2.0 * t * t);
    }
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            cplx s = 0.0;
            for (int k = 0; k < M; ++k) s += phi[(size_t)i * M + k] * phi[(size_t)j * M + k] * gk[k];
            Sigma[(size_t)i * M + j] = t * t * s;
        }
    free(phi);
    free(gk);
}

/* ------------------------------------------------------------------------ */
/* Sancho-Rubio decimation (Lopez Sancho, Lopez Sancho & Rubio, J. Phys. F 15,
 * 851 (1985)) for the surface Green function of a lead made of cells H0
 * coupled by V (Sec. 5.3 B).  side 0 = left lead (surface couples to the next
 * cell outward through alpha = V, back through beta = V^dagger); side 1 =
 * right lead (alpha = V^dagger, beta = V).  At energy z = E + i eta:
 *   gb = (z - eps)^{-1}
 *   eps_s += alpha gb beta;  eps += alpha gb beta + beta gb alpha;
 *   alpha = alpha gb alpha;  beta = beta gb beta
 * until max|alpha| + max|beta| < tol; then g = (z - eps_s)^{-1} and
 * Sigma = alpha0 g beta0 with the original couplings.
 * Returns ORC_OK, ORC_ERR_SINGULAR or ORC_ERR_NOCONVERGE. */
int orc_lead_decimation(int M, const cplx *H0, const cplx *V, double E, double eta,
                        int side, double tol, int maxit, cplx *g_out, cplx *Sigma_out,
                        int *iters_out)
{
    size_t MM = (size_t)M * M;
    cplx *buf = (cplx *)malloc(sizeof(cplx) * MM * 10);
    int *perm = (int *)malloc(sizeof(int) * (size_t)M);
    if (!buf || !perm) { free(buf); free(perm); return ORC_ERR_OOM; }
    cplx *eps = buf, *eps_s = buf + MM, *al = buf + 2 * MM, *be = buf + 3 * MM;
    cplx *gb = buf + 4 * MM, *tmp = buf + 5 * MM, *t1 = buf + 6 * MM, *t2 = buf + 7 * MM;
    cplx *a0 = buf + 8 * MM, *b0 = buf + 9 * MM;
    cplx z = E + I * eta;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            cplx v = V[(size_t)i * M + j], vd = conj(V[(size_t)j * M + i]);
            a0[(size_t)i * M + j] = side == 0 ? v : vd;
            b0[(size_t)i * M + j] = side == 0 ? vd : v;
        }
    memcpy(eps, H0, sizeof(cplx) * MM);
    memcpy(eps_s, H0, sizeof(cplx) * MM);
    memcpy(al, a0, sizeof(cplx) * MM);
    memcpy(be, b0, sizeof(cplx) * MM);
    int it = 0, rc = ORC_ERR_NOCONVERGE;
    for (it = 0; it < maxit; ++it) {
        double na = 0.0, nb = 0.0;
        for (size_t q = 0; q < MM; ++q) {
            if (cabs(al[q]) > na) na = cabs(al[q]);
            if (cabs(be[q]) > nb) nb = cabs(be[q]);
        }
        if (na + nb < tol) { rc = ORC_OK; break; }
        for (size_t q = 0; q < MM; ++q) tmp[q] = -eps[q];
        for (int i = 0; i < M; ++i) tmp[(size_t)i * M + i] += z;
        if (inverse(M, tmp, gb, perm)) { rc = ORC_ERR_SINGULAR; goto done; }
        matmul(M, gb, 'N', be, 'N', t1);     /* gb beta */
        matmul(M, al, 'N', t1, 'N', t2);     /* alpha gb beta */
        for (size_t q = 0; q < MM; ++q) { eps_s[q] += t2[q]; eps[q] += t2[q]; }
        matmul(M, gb, 'N', al, 'N', t1);     /* gb alpha */
        matmul(M, be, 'N', t1, 'N', t2);     /* beta gb alpha */
        for (size_t q = 0; q < MM; ++q) eps[q] += t2[q];
        matmul(M, al, 'N', t1, 'N', t2);     /* alpha gb alpha */
        memcpy(tmp, t2, sizeof(cplx) * MM);
        matmul(M, gb, 'N', be, 'N', t1);
        matmul(M, be, 'N', t1, 'N', t2);     /* beta gb beta */
        memcpy(al, tmp, sizeof(cplx) * MM);
        memcpy(be, t2, sizeof(cplx) * MM);
    }
    if (rc == ORC_OK) {
        for (size_t q = 0; q < MM; ++q) tmp[q] = -eps_s[q];
        for (int i = 0; i < M; ++i) tmp[(size_t)i * M + i] += z;
        if (inverse(M, tmp, g_out, perm)) { rc = ORC_ERR_SINGULAR; goto done; }
        matmul(M, g_out, 'N', b0, 'N', t1);
        matmul(M, a0, 'N', t1, 'N', Sigma_out);
    }
done:
    if (iters_out) *iters_out = it;
    free(buf);
    free(perm);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* A slice system (Eq. 1 grouped by slices).  Slice n has H_n = H0 +
 * diag(eps_n); slice n couples to slice n-1 by H_{n,n-1} = V[n % Vperiod]
 * (n = 1..L-1) and back by its conjugate transpose. */
typedef struct {
    int M, L;
    const cplx *H0;     /* M*M */
    const double *eps;  /* L*M diagonal shifts, or NULL for a clean system */
    const cplx *V;      /* Vperiod * M*M */
    int Vperiod;
} orc_system;

static const cplx *Vn(const orc_system *s, int n)
{
    return s->V + (size_t)(n % s->Vperiod) * s->M * s->M;
}

/* Gamma = i (Sigma - Sigma^dagger). */
static void gamma_of(int M, const cplx *S, cplx *G)
{
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j)
            G[(size_t)i * M + j] = I * (S[(size_t)i * M + j] - conj(S[(size_t)j * M + i]));
}

/* Re Tr[Ga X Gb X^dagger] for M x M blocks. */
static double trace_gxgx(int M, const cplx *Ga, const cplx *X, const cplx *Gb)
{
    size_t MM = (size_t)M * M;
    cplx *t1 = (cplx *)malloc(sizeof(cplx) * MM), *t2 = (cplx *)malloc(sizeof(cplx) * MM);
    matmul(M, X, 'N', Gb, 'N', t1);   /* X Gb */
    matmul(M, t1, 'N', X, 'C', t2);   /* X Gb X^dagger */
    double tr = 0.0;
    for (int i = 0; i < M; ++i)
        for (int k = 0; k < M; ++k) tr += creal(Ga[(size_t)i * M + k] * t2[(size_t)k * M + i]);
    free(t1);
    free(t2);
    return tr;
}

/* The plain definition (Eq. 2 and the transmission formula of Sec. 2.3):
 * assemble the dense N x N matrix A = E - H - Sigma_L (+) 0 ... (+) Sigma_R,
 * N = M L, factor it once and solve for the first and last block columns of
 * G = A^{-1}.  Outputs (any may be NULL):
 *   T[0] = T_LR = Re Tr[Gamma_L G_{1L} Gamma_R G_{1L}^dagger]
 *   T[1] = T_RL = Re Tr[Gamma_R G_{L1} Gamma_L G_{L1}^dagger]
 *   G11, G1L, GL1 (M x M each), ldos (L x M, needs all N columns: O(N^3)).
 * Returns ORC_OK or ORC_ERR_SINGULAR / ORC_ERR_OOM. */
int orc_dense(const orc_system *s, double E, const cplx *SigL, const cplx *SigR,
              double *T, cplx *G11, cplx *G1L, cplx *GL1, double *ldos)
{
    int M = s->M, L = s->L;
    size_t N = (size_t)M * L, MM = (size_t)M * M;
    cplx *A = (cplx *)calloc(N * N, sizeof(cplx));
    int *perm = (int *)malloc(sizeof(int) * N);
    cplx *X = (cplx *)malloc(sizeof(cplx) * N * M);
    cplx *Y = (cplx *)malloc(sizeof(cplx) * N * M);
    cplx *GaL = (cplx *)malloc(sizeof(cplx) * MM), *GaR = (cplx *)malloc(sizeof(cplx) * MM);
    cplx *blk = (cplx *)malloc(sizeof(cplx) * MM);
    int rc = ORC_OK;
    if (!A || !perm || !X || !Y || !GaL || !GaR || !blk) { rc = ORC_ERR_OOM; goto out; }
    for (int n = 0; n < L; ++n) {
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) {
                size_t r = (size_t)n * M + i, c = (size_t)n * M + j;
                cplx h = s->H0[(size_t)i * M + j];
                if (i == j) h += s->eps ? s->eps[(size_t)n * M + i] : 0.0;
                A[r * N + c] = (i == j ? E : 0.0) - h;
            }
        if (n > 0) {
            const cplx *V = Vn(s, n);
            for (int i = 0; i < M; ++i)
                for (int j = 0; j < M; ++j) {
                    size_t rn = (size_t)n * M + i, cp = (size_t)(n - 1) * M + j;
                    A[rn * N + cp] = -V[(size_t)i * M + j];           /* H_{n,n-1} = V_n */
                    A[cp * N + rn] = -conj(V[(size_t)i * M + j]);     /* H_{n-1,n} = V_n^dagger */
                }
        }
    }
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            A[(size_t)i * N + j] -= SigL[(size_t)i * M + j];
            size_t r = (size_t)(L - 1) * M + i, c = (size_t)(L - 1) * M + j;
            A[r * N + c] -= SigR[(size_t)i * M + j];
        }
    if (orc_lu_factor((int)N, A, perm)) { rc = ORC_ERR_SINGULAR; goto out; }
    /* first block column: X = A^{-1} [I; 0; ...] */
    memset(X, 0, sizeof(cplx) * N * M);
    for (int i = 0; i < M; ++i) X[(size_t)i * M + i] = 1.0;
    orc_lu_solve((int)N, A, perm, X, M);
    /* last block column */
    memset(Y, 0, sizeof(cplx) * N * M);
    for (int i = 0; i < M; ++i) Y[((size_t)(L - 1) * M + i) * M + i] = 1.0;
    orc_lu_solve((int)N, A, perm, Y, M);
    gamma_of(M, SigL, GaL);
    gamma_of(M, SigR, GaR);
    if (G11) memcpy(G11, X, sizeof(cplx) * MM);
    if (GL1) memcpy(GL1, X + (size_t)(L - 1) * M * M, sizeof(cplx) * MM);
    if (G1L) memcpy(G1L, Y, sizeof(cplx) * MM);
    if (T) {
        memcpy(blk, Y, sizeof(cplx) * MM);                         /* G_{1L} */
        T[0] = trace_gxgx(M, GaL, blk, GaR);
        memcpy(blk, X + (size_t)(L - 1) * M * M, sizeof(cplx) * MM); /* G_{L1} */
        T[1] = trace_gxgx(M, GaR, blk, GaL);
    }
    if (ldos) {
        /* diagonal of A^{-1}, one unit column at a time */
        cplx *e = (cplx *)malloc(sizeof(cplx) * N);
        if (!e) { rc = ORC_ERR_OOM; goto out; }
        for (size_t c = 0; c < N; ++c) {
            memset(e, 0, sizeof(cplx) * N);
            e[c] = 1.0;
            orc_lu_solve((int)N, A, perm, e, 1);
            ldos[c] = -cimag(e[c]) / M_PI;
        }
        free(e);
    }
out:
    free(A); free(perm); free(X); free(Y); free(GaL); free(GaR); free(blk);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* The method in slice form (Sec. 5.3 D: knitting adds the system to the
 * thread one slice at a time; sewing walks back from the other lead).
 * Forward:  A_0 = E - H_0 - Sigma_L,
 *           A_n = E - H_n - V_n g_{n-1} V_n^dagger      (n >= 1),
 *           A_{L-1} additionally - Sigma_R,
 *           g_n = A_n^{-1},  G_{0,0} = g_0,  G_{0,n} = G_{0,n-1} V_n^dagger g_n.
 * T_LR = Re Tr[Gamma_L G_{0,L-1} Gamma_R G_{0,L-1}^dagger].
 * Backward (only if ldos != NULL): G_{L-1,L-1} = g_{L-1},
 *           G_{n,n} = g_n + g_n V_{n+1}^dagger G_{n+1,n+1} V_{n+1} g_n,
 *           ldos[n*M + x] = -Im G_{n,n}[x][x] / pi.
 * G11_out (M x M) receives G_{0,0} of the full system when ldos is computed;
 * G1L_out (M x M, optional) receives G_{0,L-1}.
 * Returns ORC_OK, ORC_ERR_SINGULAR or ORC_ERR_OOM. */
int orc_rgf(const orc_system *s, double E, const cplx *SigL, const cplx *SigR,
            double *T, double *ldos, cplx *G11_out, cplx *G1L_out)
{
    int M = s->M, L = s->L;
    size_t MM = (size_t)M * M;
    int keep = ldos != NULL;
    cplx *gs = (cplx *)malloc(sizeof(cplx) * MM * (keep ? (size_t)L : 1));
    cplx *A = (cplx *)malloc(sizeof(cplx) * MM), *t1 = (cplx *)malloc(sizeof(cplx) * MM);
    cplx *t2 = (cplx *)malloc(sizeof(cplx) * MM), *G1n = (cplx *)malloc(sizeof(cplx) * MM);
    cplx *gprev = (cplx *)malloc(sizeof(cplx) * MM), *Ga = (cplx *)malloc(sizeof(cplx) * MM);
    cplx *Gb = (cplx *)malloc(sizeof(cplx) * MM);
    int *perm = (int *)malloc(sizeof(int) * (size_t)M);
    int rc = ORC_OK;
    if (!gs || !A || !t1 || !t2 || !G1n || !gprev || !Ga || !Gb || !perm) { rc = ORC_ERR_OOM; goto out; }
    for (int n = 0; n < L; ++n) {
        cplx *g = gs + (keep ? (size_t)n * MM : 0);
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) {
                cplx h = s->H0[(size_t)i * M + j];
                if (i == j) h += s->eps ? s->eps[(size_t)n * M + i] : 0.0;
                A[(size_t)i * M + j] = (i == j ? E : 0.0) - h;
            }
        if (n == 0) {
            for (size_t q = 0; q < MM; ++q) A[q] -= SigL[q];
        } else {
            const cplx *V = Vn(s, n);
            matmul(M, gprev, 'N', V, 'C', t1);  /* g_{n-1} V^dagger */
            matmul(M, V, 'N', t1, 'N', t2);     /* V g_{n-1} V^dagger */
            for (size_t q = 0; q < MM; ++q) A[q] -= t2[q];
        }
        if (n == L - 1)
            for (size_t q = 0; q < MM; ++q) A[q] -= SigR[q];
        if (inverse(M, A, g, perm)) { rc = ORC_ERR_SINGULAR; goto out; }
        if (n == 0) {
            memcpy(G1n, g, sizeof(cplx) * MM);
        } else {
            matmul(M, G1n, 'N', Vn(s, n), 'C', t1);  /* G_{0,n-1} V_n^dagger */
            matmul(M, t1, 'N', g, 'N', G1n);
        }
        memcpy(gprev, g, sizeof(cplx) * MM);
    }
    gamma_of(M, SigL, Ga);
    gamma_of(M, SigR, Gb);
    if (T) *T = trace_gxgx(M, Ga, G1n, Gb);
    if (G1L_out) memcpy(G1L_out, G1n, sizeof(cplx) * MM);
    if (keep) {
        /* sewing: G_{n,n} from G_{n+1,n+1}; Gnn held in gprev */
        memcpy(gprev, gs + (size_t)(L - 1) * MM, sizeof(cplx) * MM);
        for (int x = 0; x < M; ++x) ldos[(size_t)(L - 1) * M + x] = -cimag(gprev[(size_t)x * M + x]) / M_PI;
        for (int n = L - 2; n >= 0; --n) {
            const cplx *g = gs + (size_t)n * MM, *V = Vn(s, n + 1);
            matmul(M, V, 'N', g, 'N', t1);        /* V_{n+1} g_n */
            matmul(M, gprev, 'N', t1, 'N', t2);   /* G_{n+1,n+1} V g_n */
            matmul(M, V, 'C', t2, 'N', t1);       /* V^dagger G V g_n */
            matmul(M, g, 'N', t1, 'N', t2);       /* g_n V^dagger G V g_n */
            for (size_t q = 0; q < MM; ++q) gprev[q] = g[q] + t2[q];
            for (int x = 0; x < M; ++x) ldos[(size_t)n * M + x] = -cimag(gprev[(size_t)x * M + x]) / M_PI;
        }
        if (G11_out) memcpy(G11_out, gprev, sizeof(cplx) * MM);
    }
out:
    free(gs); free(A); free(t1); free(t2); free(G1n); free(gprev); free(Ga); free(Gb); free(perm);
    return rc;
}

/* orc_rgf over nInst independent instances that share H0, V and block
 * structure; instance i has energy E[i], self-energies SigL/SigR at
 * sig_index[i] * M*M and disorder drawn from (seed[i], W[i]).  One OpenMP
 * thread per instance at a time; nthreads <= 0 uses the runtime default.
 * This is the CPU baseline: nothing here is tuned beyond running
 * independent instances on separate cores. */
int orc_rgf_batch(int M, int L, const cplx *H0, const cplx *V, int Vperiod, int block,
                  const double *sign, int nInst, const double *E, const uint64_t *seed,
                  const double *W, const cplx *SigL, const cplx *SigR, const int *sig_index,
                  int nthreads, double *T, int *status)
{
    int rc_all = ORC_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < nInst; ++i) {
        double *eps = (double *)malloc(sizeof(double) * (size_t)L * M);
        if (!eps) { status[i] = ORC_ERR_OOM; continue; }
        orc_onsite_fill(seed[i], L, M, block, sign, W[i], eps);
        orc_system s = {M, L, H0, eps, V, Vperiod};
        size_t off = (size_t)sig_index[i] * M * M;
        status[i] = orc_rgf(&s, E[i], SigL + off, SigR + off, &T[i], NULL, NULL, NULL);
        free(eps);
    }
    for (int i = 0; i < nInst; ++i)
        if (status[i] != ORC_OK) rc_all = status[i];
    return rc_all;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Flat-argument entry points for foreign-function callers. */
int orc_dense_flat(int M, int L, const cplx *H0, const double *eps, const cplx *V, int Vperiod,
                   double E, const cplx *SigL, const cplx *SigR, double *T, cplx *G11,
                   cplx *G1L, cplx *GL1, double *ldos)
{
    orc_system s = {M, L, H0, eps, V, Vperiod};
    return orc_dense(&s, E, SigL, SigR, T, G11, G1L, GL1, ldos);
}

int orc_rgf_flat(int M, int L, const cplx *H0, const double *eps, const cplx *V, int Vperiod,
                 double E, const cplx *SigL, const cplx *SigR, double *T, double *ldos,
                 cplx *G11, cplx *G1L)
{
    orc_system s = {M, L, H0, eps, V, Vperiod};
    return orc_rgf(&s, E, SigL, SigR, T, ldos, G11, G1L);
}

/* The plain definition for an arbitrary geometry with two leads (Sec. 2.2
 * worked example, Sec. 2.3 formulas): A = E - H - Sigma_0 on the n0 interface
 * sites idx0 - Sigma_1 on the n1 sites idx1 (N x N dense, H Hermitian),
 * G = A^{-1}; T[0] = T_{1<-0} = Re Tr[Gamma_1 G_{10} Gamma_0 G_{10}^dagger],
 * T[1] = T_{0<-1}.  Returns ORC_OK, ORC_ERR_SINGULAR or ORC_ERR_OOM. */
int orc_dense_general(int N, const cplx *H, double E, int n0, const int *idx0,
                      const cplx *Sig0, int n1, const int *idx1, const cplx *Sig1, double *T)
{
    cplx *A = (cplx *)malloc(sizeof(cplx) * (size_t)N * N);
    int *perm = (int *)malloc(sizeof(int) * (size_t)N);
    int nm = n0 > n1 ? n0 : n1;
    cplx *X = (cplx *)malloc(sizeof(cplx) * (size_t)N * nm);
    cplx *G10 = (cplx *)malloc(sizeof(cplx) * (size_t)n1 * n0);
    cplx *G01 = (cplx *)malloc(sizeof(cplx) * (size_t)n0 * n1);
    cplx *Ga0 = (cplx *)malloc(sizeof(cplx) * (size_t)n0 * n0);
    cplx *Ga1 = (cplx *)malloc(sizeof(cplx) * (size_t)n1 * n1);
    int rc = ORC_OK;
    if (!A || !perm || !X || !G10 || !G01 || !Ga0 || !Ga1) { rc = ORC_ERR_OOM; goto out; }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            A[(size_t)i * N + j] = (i == j ? E : 0.0) - H[(size_t)i * N + j];
    for (int a = 0; a < n0; ++a)
        for (int b = 0; b < n0; ++b) A[(size_t)idx0[a] * N + idx0[b]] -= Sig0[(size_t)a * n0 + b];
    for (int a = 0; a < n1; ++a)
        for (int b = 0; b < n1; ++b) A[(size_t)idx1[a] * N + idx1[b]] -= Sig1[(size_t)a * n1 + b];
    if (orc_lu_factor(N, A, perm)) { rc = ORC_ERR_SINGULAR; goto out; }
    gamma_of(n0, Sig0, Ga0);
    gamma_of(n1, Sig1, Ga1);
    /* columns of lead 0 -> G_{10} */
    memset(X, 0, sizeof(cplx) * (size_t)N * n0);
    for (int b = 0; b < n0; ++b) X[(size_t)idx0[b] * n0 + b] = 1.0;
    orc_lu_solve(N, A, perm, X, n0);
    for (int a = 0; a < n1; ++a)
        for (int b = 0; b < n0; ++b) G10[(size_t)a * n0 + b] = X[(size_t)idx1[a] * n0 + b];
    /* columns of lead 1 -> G_{01} */
    memset(X, 0, sizeof(cplx) * (size_t)N * n1);
    for (int b = 0; b < n1; ++b) X[(size_t)idx1[b] * n1 + b] = 1.0;
    orc_lu_solve(N, A, perm, X, n1);
    for (int a = 0; a < n0; ++a)
        for (int b = 0; b < n1; ++b) G01[(size_t)a * n1 + b] = X[(size_t)idx0[a] * n1 + b];
    /* T_{1<-0} = sum Gamma1[a,a'] G10[a',b] Gamma0[b,b'] conj(G10[a,b']) */
    for (int w = 0; w < 2; ++w) {
        int na = w == 0 ? n1 : n0, nb = w == 0 ? n0 : n1;
        const cplx *Ga = w == 0 ? Ga1 : Ga0, *Gb = w == 0 ? Ga0 : Ga1, *G = w == 0 ? G10 : G01;
        double tr = 0.0;
        for (int a = 0; a < na; ++a)
            for (int a2 = 0; a2 < na; ++a2)
                for (int b = 0; b < nb; ++b)
                    for (int b2 = 0; b2 < nb; ++b2)
                        tr += creal(Ga[(size_t)a * na + a2] * G[(size_t)a2 * nb + b] *
                                    Gb[(size_t)b * nb + b2] * conj(G[(size_t)a * nb + b2]));
        T[w] = tr;
    }
out:
    free(A); free(perm); free(X); free(G10); free(G01); free(Ga0); free(Ga1);
    return rc;
}
