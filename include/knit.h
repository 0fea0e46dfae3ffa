/*
 * knit.h -- C-ABI of the GB300 recursive Green-function (KNIT slice sweep)
 * transport library.  Plain pointers and sizes only; no C++ or framework types.
 *
 * The problem (KNIT user guide, Sec. 2.3, Eq. 1 and Eq. 2): a tight-binding
 * system of L slices with M orbitals each, block-tridiagonal Hamiltonian
 *     H_{n,n}   = H0 + diag(eps_n)                (M x M, Hermitian)
 *     H_{n,n-1} = V[n % Vperiod],  H_{n-1,n} = V[n % Vperiod]^dagger,
 * coupled at slice 0 and slice L-1 to two semi-infinite clean leads.  Each
 * lead repeats one cell (lead_H0, lead_V) and couples to the system with its
 * own inter-cell hopping (Sec. 5.3 B, "the hopping matrix elements from the
 * lead to the system are exactly the same as those inside lead itself"):
 *     left:  g_L = (E - H0_L - V_L g_L V_L^dagger)^{-1},  Sigma_L = V_L g_L V_L^dagger
 *     right: g_R = (E - H0_R - V_R^dagger g_R V_R)^{-1},  Sigma_R = V_R^dagger g_R V_R
 * The retarded Green function is G = (E - H - Sigma_L - Sigma_R)^{-1} (Eq. 2,
 * read with the textbook sign Im Sigma <= 0), the transmission
 *     T = Re Tr[Gamma_L G_{0,L-1} Gamma_R G_{0,L-1}^dagger],  Gamma = i(Sigma - Sigma^dagger)
 * (Sec. 2.3 transmission formula) and the local density of states
 *     LDOS[n][x] = -Im G_{(n,x),(n,x)} / pi  (Sec. 2.1 b, on-site density).
 * The slice sweep ("knitting", Sec. 5.3 D) is block Gaussian elimination of
 * (E - H - Sigma); the backward pass ("sewing") gives the diagonal blocks.
 *
 * Disorder (Sec. 6.1): orbital c of site s = x / block in slice n receives
 *     eps = onsite_sign[c] * W * (r - 1/2),
 *     r = (splitmix64(splitmix64(seed) ^ (n << 32 | s)) >> 11) * 2^-53,
 * with SplitMix64 as published by Steele, Lea & Flood (OOPSLA 2014).
 *
 * Conventions for every call:
 *  - complex numbers are knit_c128 (re, im) pairs; matrices are row-major;
 *  - input and output arrays may be host or device memory (the library asks
 *    the CUDA runtime which); the caller owns them;
 *  - calls are ordered on `stream` (a cudaStream_t, NULL = legacy default
 *    stream); a call whose outputs include host memory returns after the
 *    results are in host memory, otherwise it returns after enqueueing;
 *  - the return value reports invalid arguments, out-of-memory and CUDA
 *    errors; per-instance numerical failures (singular pivot, non-finite
 *    result, non-converged lead) go to the optional `status` array and do
 *    not fail the batch;
 *  - knit_last_error() returns a thread-local message for the last failure.
 *  - Only one call per system may run at a time: a system owns its device
 *    workspace.
 */
#ifndef KNIT_H
#define KNIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct knit_system_s *knit_system;   /* opaque; owned by the library */

typedef struct {
    double re, im;
} knit_c128;

typedef enum {
    KNIT_OK = 0,
    KNIT_ERR_INVALID = 1,    /* bad argument or unsupported structure */
    KNIT_ERR_OOM = 2,        /* device or host allocation failed */
    KNIT_ERR_CUDA = 3,       /* CUDA runtime error (message in knit_last_error) */
    KNIT_ERR_SINGULAR = 4,   /* per instance: exactly zero pivot in an inversion */
    KNIT_ERR_NOCONVERGE = 5, /* per energy: lead fixed point did not converge */
    KNIT_ERR_TIMEOUT = 6,    /* a bounded device wait ran out */
    KNIT_ERR_NONFINITE = 7   /* per instance: NaN or Inf in the result */
} knit_status;

/* Arithmetic of the slice sweep. */
enum {
    KNIT_FP64 = 0,  /* complex128 throughout */
    KNIT_MIXED = 1, /* complex64 inversion + one refinement step against a
                       residual exact to ~2^-48; the state g_n is carried as
                       hi + lo floats.  For 33 <= M <= 64 the residual's dense
                       product runs on the tensor cores (bf16 digit slices,
                       f32 accumulation), below on CUDA cores.  Widths
                       65..128, and any width up to 128 with 4 x 4 block or
                       tridiagonal couplings, use a 512-thread tensor-core
                       variant (tcgen05, accumulators in tensor memory) with
                       the state in device memory.  Above 128, a system
                       whose rows split into half-rows (knit_system_create)
                       runs that variant on its half-row chain; any other
                       M > 128 runs the KNIT_FP64 sweep instead. */
    KNIT_MIXED_CUDACORE = 2  /* KNIT_MIXED with the residual always accumulated
                                in double-float arithmetic on CUDA cores
                                (diagonal and 4 x 4 block couplings; other
                                systems run in KNIT_FP64) */
};

/* Lead solver. */
enum {
    KNIT_LEAD_AUTO = 0,       /* MODES when the lead hopping is a multiple of
                                 the identity, else DECIMATION */
    KNIT_LEAD_MODES = 1,      /* transverse modes of lead_H0 (FP64 Jacobi
                                 eigensolver once per system) and the retarded
                                 1D surface function per mode; exact for
                                 lead_V = t * I */
    KNIT_LEAD_DECIMATION = 2, /* Sancho-Rubio decimation in FP64 at E + i eta */
    KNIT_LEAD_LEARNED = 3     /* a trained knit_lead_model predicts g, Newton's
                                 method refines the fixed point at eta = 0 to a
                                 residual max|A g - I| < 1e-12 (FP64, cells of
                                 at most 8 orbitals); energies where Newton
                                 fails fall back to DECIMATION */
};

typedef struct {
    int32_t M;                   /* orbitals per slice, 1 <= M <= 256 */
    int32_t L;                   /* slices, L >= 1 */
    int32_t block;               /* orbitals per site (1, 2 or 4); M % block == 0 */
    const double *onsite_sign;   /* `block` signs for the site's disorder draw, NULL = all +1 */
    const knit_c128 *H0;         /* M*M clean slice Hamiltonian (Hermitian) */
    const double *onsite;        /* L*M explicit diagonal shifts added to H0, or NULL;
                                    when given, W and seeds are ignored */
    const knit_c128 *V;          /* Vperiod*M*M, H_{n,n-1} = V[n % Vperiod]; each V must be
                                    block-diagonal with `block` x `block` blocks, or
                                    tridiagonal (nonzeros only at |i - j| <= 1, as in a
                                    honeycomb ribbon sliced by half-rows) */
    int32_t Vperiod;             /* 1, 2 or 4 */
    const knit_c128 *lead_H0[2]; /* left/right lead cell (M*M); NULL = H0 */
    const knit_c128 *lead_V[2];  /* left/right lead inter-cell hopping (M*M); NULL = V[0] */
    int32_t lead_Vperiod[2];     /* 0 or 1: one coupling as above.  2: lead_V[p] holds two
                                    M*M couplings [V_first, V_second] that alternate going
                                    outward, V_first coupling the system's end slice to the
                                    lead's surface slice (H_{0,-1} on the left, H_{L,L-1} on
                                    the right, slice-forward orientation H_{n,n-1}) and
                                    V_second the surface slice to the next one, as in an
                                    armchair ribbon (Sec. 6.3); NULL lead_V[p] continues the
                                    system's own V.  The lead is solved as a two-slice
                                    supercell by DECIMATION (AUTO picks it). */
} knit_system_desc;

/* Copy the description into a new system (all pointers are read during the
 * call only; host or device memory).  Returns KNIT_ERR_INVALID for sizes out
 * of range, a V neither block-diagonal nor tridiagonal, or a lead_V whose
 * structure the lead solvers do not support.  A system wider than 128 whose
 * rows split into two halves (those coupled to the previous row and the
 * rest) with the same Hamiltonian block on every half-row and couplings of
 * period <= 2 (a honeycomb ribbon, Sec. 6.3) also gets its half-row chain
 * (width M / 2, 2L slices, couplings of period 4), on which KNIT_MIXED
 * transmissions then run; a period-2 lead whose supercell splits into
 * blocks of at most 4 modes in the eigenbasis of its cell Hamiltonian is
 * solved block by block.  A lead whose orbitals fall into decoupled sectors
 * of one size (a normal BdG lead: electrons and holes) is decimated sector
 * by sector, the hole sector taken as the particle-hole image of the
 * electron sector where it is one; a sector that splits again in the
 * eigenbasis of H0 + a (V + V^dagger) + i b (V - V^dagger) (any symmetry
 * of the lead, e.g. a mirror of a Rashba strip) into blocks of one size is
 * decimated block by block, Sigma = U diag(Sigma_r) U^dagger
 * (knit_system_info reports the half-row chain and the block counts). */
knit_status knit_system_create(const knit_system_desc *desc, knit_system *out);

/* Free a system and its device workspace (NULL is accepted). */
knit_status knit_system_destroy(knit_system sys);

typedef struct {
    int32_t method;    /* KNIT_LEAD_* */
    double eta;        /* decimation broadening (default 1e-12 when <= 0) */
    double tol;        /* decimation stop: max|alpha| + max|beta| < tol (default 1e-14) */
    int32_t maxit;     /* decimation iteration cap (default 200) */
    const void *model[2]; /* KNIT_LEAD_LEARNED: knit_lead_model of the left / right lead */
} knit_lead_opts;

/* Lead self-energy Sigma_lead(E[e]) for nE energies (Sec. 5.3 B selfE(E)).
 * lead: 0 = left, 1 = right.  sigma: nE*M*M outputs (caller-owned).
 * iters (nE, optional): decimation iterations (0 for MODES); residual (nE,
 * optional): max-norm of g - (E - H0 - V g V^dagger)^{-1} at eta = 0, computed
 * in FP64 on the device (for a period-2 lead: of the supercell's g).  opts may
 * be NULL (AUTO). */
knit_status knit_lead_selfenergy(knit_system sys, int32_t lead, const double *E, int32_t nE,
                                 const knit_lead_opts *opts, knit_c128 *sigma, int32_t *iters,
                                 double *residual, void *stream);

/* Instances form an energy x seed grid: instance i = e * nS + s has energy
 * E[e] and disorder seed seeds[s] (seeds may be NULL: seed 0 for all), all
 * with disorder strength W (ignored when the system has explicit `onsite`).
 * Per-instance outputs are indexed the same way. */

/* Two-terminal transmission T_i (Sec. 2.3) for nE * nS instances.  The lead
 * self-energies are computed once per energy on the device (opts may be
 * NULL: AUTO).  precision: KNIT_FP64, KNIT_MIXED or KNIT_MIXED_CUDACORE.  T: nE*nS outputs; status
 * (optional): nE*nS knit_status values. */
knit_status knit_transmission(knit_system sys, const double *E, int32_t nE,
                              const uint64_t *seeds, int32_t nS, double W, int32_t precision,
                              const knit_lead_opts *opts, double *T, int32_t *status,
                              void *stream);

/* The sweep alone (Sec. 5.3 D knitting) with caller-supplied self-energies:
 * energy e uses sigmaL/sigmaR + e*M*M (complex128, nE*M*M each). */
knit_status knit_transmission_sigma(knit_system sys, const double *E, int32_t nE,
                                    const uint64_t *seeds, int32_t nS, double W,
                                    const knit_c128 *sigmaL, const knit_c128 *sigmaR,
                                    int32_t precision, double *T, int32_t *status, void *stream);

/* Transmission eigenvalues and shot noise (Sec. 8: "conductance, shot noise,
 * transmission eigenvalues"; Sec. 2.3: T_kl is the trace of
 * G_kl Gamma_l G_kl^+ Gamma_k, whose eigenvalues are the transmission
 * eigenvalues tau_n).  Instances as for knit_transmission.  For instance i:
 *   tau   (nE*nS*M, required): the M eigenvalues of the Hermitian matrix
 *         Gamma_R^{1/2} G_L1 Gamma_L G_L1^dagger Gamma_R^{1/2}, in decreasing
 *         order -- the transmission eigenvalues, in [0, 1] up to rounding,
 *         followed by (numerically) zero ones for closed channels;
 *   noise (nE*nS, optional): sum_n tau_n (1 - tau_n), the zero-temperature
 *         shot noise in units of 2 e^3 |V| / h (Fano factor noise / T);
 *   T, status (optional): as for knit_transmission (T = sum_n tau_n up to
 *         rounding).
 * Instances with a non-zero status get NaN in tau and noise.  The matrix is
 * formed from G_LL, the last slice's diagonal block of the sweep (FP64 or
 * mixed, as `precision` selects), by the unitarity identity of the retarded
 * function, and diagonalised in FP64 (cyclic Jacobi).  M <= 256; device
 * workspace ~2 n M^2 complex128 (n = nE*nS). */
knit_status knit_transmission_eigenvalues(knit_system sys, const double *E, int32_t nE,
                                          const uint64_t *seeds, int32_t nS, double W,
                                          int32_t precision, const knit_lead_opts *opts,
                                          double *tau, double *noise, double *T, int32_t *status,
                                          void *stream);

/* Lead-resolved lesser function along the sewing pass (Sec. 2.3:
 * G^< = sum_l f_l G^<_l with G^<_l = i G Gamma_l G^+, Gamma_l = i(Sigma_l -
 * Sigma_l^+); Sec. 5.3 D sewing; the non-equilibrium density and local
 * currents of Sec. 7.3 getG_lesser), energy-resolved and per injecting lead,
 * for instances as in knit_transmission; FP64.  With A^l = G Gamma_l G^+:
 *   rhoL, rhoR (nE*nS*L*M, [i][n][x]): A^l_{(n,x),(n,x)} / 2pi, the density of
 *         states injected by the left / right lead (rhoL + rhoR = LDOS; the
 *         non-equilibrium density at energy E is f_L rhoL + f_R rhoR);
 *   jx    (nE*nS*(L-1)*M, [i][n][x]): current carried by left-injected states
 *         from orbital x of slice n into slice n+1,
 *         sum_y -2 Im[H_{(n,x),(n+1,y)} A^L_{(n+1,y),(n,x)}] (units e/h per
 *         unit energy; sum_x jx = T for every n);
 *   jt    (nE*nS*L*nedge, [i][n][e]): the same along the e-th edge x < y of
 *         H0 inside slice n, edges in row-major order of H0's nonzero entries
 *         above the diagonal (knit_system_num_edges gives nedge), positive
 *         from x to y.
 * Any of the four may be NULL (not all).  T, status (optional) as for
 * knit_transmission.  saving_level as for knit_ldos.  Device workspace per
 * SM: (8 + ceil(L / k) + k) M^2 complex128 (k = saving_level). */
knit_status knit_lesser(knit_system sys, const double *E, int32_t nE, const uint64_t *seeds,
                        int32_t nS, double W, int32_t saving_level, const knit_lead_opts *opts,
                        double *rhoL, double *rhoR, double *jx, double *jt, double *T,
                        int32_t *status, void *stream);

/* Number of nonzero entries of H0 above its diagonal (the edges of jt). */
knit_status knit_system_num_edges(knit_system sys, int32_t *count);

/* Sweep kernels (knit_system_info). */
enum {
    KNIT_SWEEP_FP64 = 0,           /* complex128 sweep */
    KNIT_SWEEP_MIXED_NARROW = 1,   /* mixed, widths <= 64, diagonal couplings */
    KNIT_SWEEP_MIXED_CUDACORE = 2, /* mixed, residual on CUDA cores, widths <= 128 */
    KNIT_SWEEP_MIXED_TC128 = 3,    /* mixed, tensor-core kernel for widths <= 128 */
    KNIT_SWEEP_MIXED_HALF_ROWS = 4 /* KNIT_SWEEP_MIXED_TC128 on the half-row chain */
};

/* Which sweep kernel knit_transmission (energy x seed grid) runs for this
 * system at `precision` (*sweep, a KNIT_SWEEP_* value), and into how many
 * independent blocks the decimation of each lead splits (lead_blocks[2]:
 * sectors x mode blocks per sector, or the two-slice supercell's mode
 * blocks; 1 = the whole cell or supercell).  Host only, no device work.
 * KNIT_ERR_INVALID for NULL arguments or an unknown precision. */
knit_status knit_system_info(knit_system sys, int32_t precision, int32_t *sweep,
                             int32_t *lead_blocks);

/* ---------------------------------------------------------------------
 * Arbitrary geometries (Sec. 5.3: knitting through an interface of varying
 * width; Sec. 2.2 worked example, Fig. 3; Sec. 7.3 conductance_matrix).  H
 * is the N x N Hermitian Hamiltonian of the system's sites (dense,
 * row-major, host or device memory); lead p is attached to the
 * n_lead_sites[p] sites lead_sites[p] (in the order of its self-energy's
 * rows).  The library cuts the sites into slices of varying width:
 * breadth-first layers from lead 0's sites, the layers from the first one
 * holding a site of another lead onwards merged into the last slice (sites
 * not connected to lead 0 are left out), so that H is block tridiagonal with
 * rectangular couplings and every lead but lead 0 sits in the last slice.
 * KNIT_ERR_INVALID for N outside 1 .. 8192, fewer than 2 or more than 64
 * leads, a non-Hermitian H (relative 1e-12), overlapping or out-of-range lead
 * sites, a lead not connected to lead 0, or a slice wider than 6144 sites.
 * The sweep runs one energy per CTA (at most one CTA per SM, fewer when six
 * widest-slice matrices per CTA would pass 8 GiB).  The graph calls return
 * after the sweep has finished. */
typedef struct knit_graph_s *knit_graph;
typedef struct {
    int32_t N;
    const knit_c128 *H;
    int32_t n_lead_sites[2];
    const int32_t *lead_sites[2];
} knit_graph_desc;
typedef struct {
    int32_t N;
    const knit_c128 *H;
    int32_t n_leads;                 /* P >= 2 */
    const int32_t *n_lead_sites;     /* P */
    const int32_t *const *lead_sites;/* P lists */
} knit_graph_multi_desc;

/* Two leads: copies H and the site lists (host or device memory), builds the
 * slicing on the host and keeps device copies of the blocks in *out, owned by
 * the library until knit_graph_destroy.  Errors as listed above, plus
 * KNIT_ERR_OOM / KNIT_ERR_CUDA for device allocations and copies. */
knit_status knit_graph_create(const knit_graph_desc *desc, knit_graph *out);

/* The same for P >= 2 leads. */
knit_status knit_graph_create_multi(const knit_graph_multi_desc *desc, knit_graph *out);

/* Frees the graph and its device memory; NULL is accepted. */
knit_status knit_graph_destroy(knit_graph g);

/* The slicing of a description without creating a graph (host work only, no
 * device memory): number of slices and the slice of every site (N values,
 * -1 for a site not connected to lead 0; optional).  Same checks and error
 * codes as knit_graph_create_multi. */
knit_status knit_graph_plan(const knit_graph_multi_desc *desc, int32_t *nslices,
                            int32_t *slice_of);

/* The slicing: number of slices, their widths (nslices values, optional) and
 * the slice of every site (N values, -1 for a site not connected to lead 0;
 * optional). */
knit_status knit_graph_slices(knit_graph g, int32_t *nslices, int32_t *widths,
                              int32_t *slice_of);

/* T_01 = Re Tr[Gamma_0 G_01 Gamma_1 G_01^dagger] (Sec. 2.3, k = 0, l = 1) for
 * nE energies, by the knitting sweep over the slices in FP64; sigma0
 * (nE x w0 x w0) and sigma1 (nE x w1 x w1) are the leads' retarded
 * self-energies on their sites (e.g. knit_lead_selfenergy of a system whose
 * lead cells are the leads').  T: nE outputs; status (optional) per energy. */
knit_status knit_graph_transmission(knit_graph g, const double *E, int32_t nE,
                                    const knit_c128 *sigma0, const knit_c128 *sigma1, double *T,
                                    int32_t *status, void *stream);

/* Multi-terminal transmissions (Sec. 2.3 T_kl for every pair of leads; Sec.
 * 7.3 conductance_matrix): Tmat (nE x P x P, [e][k][l]) receives
 * T_kl = Re Tr[Gamma_k G_kl Gamma_l G_kl^dagger] for k != l and 0 on the
 * diagonal; sigma: P pointers, lead p's self-energies nE x w_p x w_p. */
knit_status knit_graph_conductance(knit_graph g, const double *E, int32_t nE,
                                   const knit_c128 *const *sigma, double *Tmat, int32_t *status,
                                   void *stream);

/* Local density of states (Sec. 5.3 D knitting followed by sewing):
 * ldos (nE*nS*L*M, row-major [i][n][x]) receives -Im G_nn[x][x]/pi; T
 * (optional) the transmission; status (optional) per instance (ldos of an
 * instance with non-zero status is unspecified).  saving_level follows
 * knitANDsew (Sec. 7.3): -1 keeps every forward g_n; k >= 1 keeps every k-th
 * and recomputes the slices in between during the backward pass; 0 (keep
 * nothing) is rejected because the backward pass needs the forward g_n.
 * precision: KNIT_FP64, or KNIT_MIXED / KNIT_MIXED_CUDACORE (the same
 * thing here) for widths up to 64 with diagonal inter-slice couplings: the
 * forward pass is the mixed sweep, checkpoints are kept as double-float and
 * the sewing products are formed in double-float; other systems run in FP64. */
knit_status knit_ldos(knit_system sys, const double *E, int32_t nE, const uint64_t *seeds,
                      int32_t nS, double W, int32_t precision, int32_t saving_level,
                      const knit_lead_opts *opts, double *ldos, double *T, int32_t *status,
                      void *stream);

/* Learned warm start for a lead (the paper's lead solver has no learned
 * component; this one speeds up and tightens the fixed point of Sec. 5.3 B).  A multilayer perceptron (input: the
 * energy scaled to [-1, 1] over the training range; three hidden layers of
 * 128 tanh units; output: real and imaginary parts of the M x M surface
 * Green function g, row-major) is trained on the GPU with the library's own
 * forward, backward and Adam kernels (FP32) on g from the library's own
 * decimation at the training energies.  Parameters are stored as, for layers
 * l = 0..3, W_l (out x in, row-major) then b_l.  Cells of at most 8 orbitals,
 * or a period-2 lead that splits into blocks of at most 4 in the eigenbasis
 * of its cell Hamiltonian (knit_system_info > 1 blocks; the armchair ribbon's
 * lead): the output is then every block's two-slice surface function in the
 * mode basis, block c's N x N (N <= 4) values at 2 N^2 c, and Newton runs per
 * (block, energy) in one thread.  knit_lead_model_num_outputs gives the
 * output width. */
typedef struct knit_lead_model_s *knit_lead_model;

/* Train for `epochs` passes over the training energies in shuffled
 * mini-batches of `batch` (Adam, learning rate lr, shuffling and
 * initialisation drawn from `seed`); opts (may be NULL) sets the decimation
 * that makes the targets.  loss (optional, host, `epochs` values) receives the
 * mean squared error of each epoch.  The model belongs to (sys, lead). */
knit_status knit_lead_model_train(knit_system sys, int32_t lead, const double *E_train,
                                  int32_t nTrain, int32_t epochs, int32_t batch, float lr,
                                  uint64_t seed, const knit_lead_opts *opts, float *loss,
                                  knit_lead_model *out, void *stream);

/* Frees the model and its device memory; NULL is accepted. */
knit_status knit_lead_model_destroy(knit_lead_model model);

/* Number of parameters (0 for NULL). */
int64_t knit_lead_model_num_params(knit_lead_model model);

/* Floats of network output per energy: 2 M^2, or 2 N^2 per block for a lead
 * solved in blocks (0 for NULL). */
int64_t knit_lead_model_num_outputs(knit_lead_model model);

/* Copy the parameters out to a host or device float array of
 * knit_lead_model_num_params values (layout above); KNIT_ERR_INVALID for NULL. */
knit_status knit_lead_model_get_params(knit_lead_model model, float *params);

/* Copy the parameters in from a host or device float array (same layout). */
knit_status knit_lead_model_set_params(knit_lead_model model, const float *params);

/* Network output for nE energies: nE x knit_lead_model_num_outputs floats
 * (re, im of g, row-major; per block for a lead solved in blocks). */
knit_status knit_lead_model_forward(knit_lead_model model, const double *E, int32_t nE, float *out,
                                    void *stream);

/* Mean squared error of the network against `target` (n x
 * knit_lead_model_num_outputs floats) and
 * its gradient with respect to every parameter (knit_lead_model_num_params
 * floats), as used by training. */
knit_status knit_lead_model_gradient(knit_lead_model model, const double *E, const float *target,
                                     int32_t n, float *grad, float *loss, void *stream);

/* Heterogeneous batches (uneven widths and lengths).  A batch plan holds
 * nInst instances; instance i belongs to systems[sys_index[i]] (sys_index is
 * read during the call; systems must outlive the plan and must not run other
 * calls while the plan runs).  The plan groups instances per system for the
 * lead solvers and per sweep kernel for the sweep, and orders each kernel's
 * queue by decreasing cost M^3 L (longest processing time first), so each
 * kernel variant is one persistent launch.  The variants' launches run at
 * once on streams of the plan (forked from and joined back into the caller's
 * stream), issued heaviest first, so that the SMs one variant's tail leaves
 * idle take the next variant's CTAs.  KNIT_MIXED instances whose
 * system the mixed kernels do not cover run in the FP64 sweep.  Lead
 * eigen-decompositions are done here, so that a run with device pointers
 * only enqueues kernels and can be captured in a CUDA graph. */
typedef struct knit_batch_s *knit_batch;

/* Build a plan for nInst instances over nSys systems (precision KNIT_FP64,
 * KNIT_MIXED or KNIT_MIXED_CUDACORE).  KNIT_ERR_INVALID for NULL arguments,
 * nSys or nInst below 1, a NULL system, a sys_index out of range or an
 * unknown precision; KNIT_ERR_OOM / KNIT_ERR_CUDA for device failures. */
knit_status knit_batch_create(const knit_system *systems, int32_t nSys, const int32_t *sys_index,
                              int32_t nInst, int32_t precision, knit_batch *out);

/* Frees the plan and its device memory (not the systems); NULL is accepted. */
knit_status knit_batch_destroy(knit_batch batch);

/* Run a plan: E, seeds and W hold one value per instance (seeds, W may be
 * NULL: seed 0, no disorder); T and status (optional) receive one value per
 * instance, in the caller's instance order (Sec. 2.3 transmission). */
knit_status knit_batch_transmission(knit_batch batch, const double *E, const uint64_t *seeds,
                                    const double *W, const knit_lead_opts *opts, double *T,
                                    int32_t *status, void *stream);

/* The plan's kernel variants ("buckets", in launch order): *nb of them; per
 * variant q (arrays of *nb, each optional) its kind (0 FP64 sweep, 1 mixed
 * M <= 64, 2 mixed CUDA-core M <= 128, 3 tensor-core M <= 128), widest M,
 * instance count and the most CTAs per SM its kernel can hold.
 * KNIT_ERR_INVALID for a NULL batch or nb. */
knit_status knit_batch_buckets(knit_batch batch, int32_t *nb, int32_t *kind, int32_t *Mmax,
                               int32_t *count, int32_t *max_ctas);

/* Set the CTAs per SM of every variant's persistent launch (config: *nb
 * values, clamped to 1 .. max_ctas), e.g. from a cache of
 * knit_batch_autotune results.  KNIT_ERR_INVALID for NULL arguments. */
knit_status knit_batch_configure(knit_batch batch, const int32_t *config);

/* Tune the launch shapes on the plan's own instances (inputs as in
 * knit_batch_transmission, host or device): the lead self-energies once,
 * then for every variant whose CTAs can share an SM each CTA count per SM
 * from 1 to max_ctas timed with CUDA events (that variant's sweep launch
 * alone) and the fastest kept in the plan.  config, ms (optional, *nb
 * values): the chosen CTAs per SM and its time (-1 where nothing was
 * tried).  Synchronous; on its own stream.  KNIT_ERR_INVALID for a NULL
 * batch or E; KNIT_ERR_CUDA / KNIT_ERR_OOM for device failures. */
knit_status knit_batch_autotune(knit_batch batch, const double *E, const uint64_t *seeds,
                                const double *W, const knit_lead_opts *opts, int32_t *config,
                                float *ms);

/* Lead self-energy by Sancho-Rubio decimation without any allocation (the
 * paper has no counterpart; it exists for callers that cannot let a library
 * call cudaMalloc/cudaFree, e.g. processes whose framework owns all device
 * memory, or loops that must not trigger the device-wide synchronisation of
 * cudaFree).  The same decimation iteration as knit_lead_selfenergy with
 * KNIT_LEAD_DECIMATION, for one lead cell given directly; Sigma is formed
 * with V treated as dense (the allocating path skips V's zero blocks), so
 * the two may differ in the last bits:
 *   H0, V: M*M lead cell and inter-cell hopping (device memory, complex128);
 *   lead: 0 = left (Sigma = V g V^dagger), 1 = right (Sigma = V^dagger g V);
 *   E: nE energies (device); eta, tol, maxit as in knit_lead_opts (<= 0 means
 *   the defaults 1e-12, 1e-14, 200);
 *   sigma: nE*M*M outputs; iters, status: nE outputs or NULL (all device).
 * Scratch comes from one fixed 9 MiB array inside the library (per device,
 * held until exit): M must be <= 64, larger M returns KNIT_ERR_INVALID, as
 * does any host pointer.  All calls share that array, so calls that overlap
 * on the GPU race; serialise them.  Every call looks up the array's address
 * on the current device (cudaGetSymbolAddress); the first lookup on a device
 * may load the library's module, so make the first call before any stream
 * capture.  Stream-ordered; returns after enqueueing. */
knit_status knit_lead_decimation_noalloc(const knit_c128 *H0, const knit_c128 *V, int32_t M,
                                         int32_t lead, const double *E, int32_t nE, double eta,
                                         double tol, int32_t maxit, knit_c128 *sigma,
                                         int32_t *iters, int32_t *status, void *stream);

/* kinds of knit_peak_probe */
enum { KNIT_PEAK_MMA_BF16 = 0, KNIT_PEAK_MMA_TF32 = 1, KNIT_PEAK_DFMA = 2, KNIT_PEAK_FFMA = 3,
       KNIT_PEAK_MMA_N64 = 4, KNIT_PEAK_MMA_N16 = 5, KNIT_PEAK_MMA_RESIDUAL = 6,
       KNIT_PEAK_MMA_RESIDUAL_TF32 = 7 };

/* Peak-rate microbenchmarks (no paper counterpart): the denominators of the
 * roofline fractions that the benchmark reports.  Launches one fixed loop on
 * nsm SMs and returns in *flop the floating-point operations it performs;
 * the caller times the launch on `stream` (CUDA events) and divides.
 *   KNIT_PEAK_MMA_BF16: tcgen05.mma kind::f16 (bf16 operands, f32 accumulate),
 *     M = 128, N = 256, K = 16 per instruction, `iters` instructions per SM;
 *   KNIT_PEAK_MMA_TF32: the same with kind::tf32 (K = 8 per instruction);
 *   KNIT_PEAK_MMA_N64 / KNIT_PEAK_MMA_N16: the bf16 loop with N = 64 / 16;
 *   KNIT_PEAK_MMA_RESIDUAL: per iteration the six MMAs of one K-chunk of the
 *     wide tensor-core sweep's residual (three A tiles, N = 256 + 192 / 128 / 64);
 *   KNIT_PEAK_MMA_RESIDUAL_TF32: the same pattern with kind::tf32 (K = 8);
 *   KNIT_PEAK_DFMA / KNIT_PEAK_FFMA: FP64 / FP32 fused multiply-add loops on
 *     the CUDA cores (eight 256-thread blocks per SM, 128 * iters FMA each).
 * timed_out: host int or NULL; when given, the call waits for the launch
 * and stores 1 if a tensor-core wait ran out of its bound (the rate is then
 * not valid), else 0.  KNIT_ERR_INVALID for an unknown kind or iters, nsm
 * below 1; KNIT_ERR_CUDA for launch failures.  Allocates nothing. */
knit_status knit_peak_probe(int32_t kind, int64_t iters, int32_t nsm, double *flop,
                            int32_t *timed_out, void *stream);

/* Thread-local description of the last error (never NULL). */
const char *knit_last_error(void);

/* Host-side fault injection for tests: the n-th device allocation the
 * library makes from now on (n = 0: the next one) fails as if the device were
 * out of memory, so the call that makes it returns KNIT_ERR_OOM and releases
 * what it had allocated; the injection then switches itself off.  n < 0
 * switches it off.  Process-wide; no device work. */
knit_status knit_debug_fail_alloc_after(int64_t n);

/* Test hook for the bounded tensor-core waits (no paper counterpart): one
 * block issues a tcgen05 MMA and commits it to one mbarrier, then waits on a
 * second mbarrier that nothing completes, polling at most `polls` times
 * (1 .. 2^24), the same bounded wait (tc::mbar_wait) the sweep kernels use.
 * The wait runs out; the block then waits, bounded, for the committed MMA
 * and releases its tensor memory, as a timed-out sweep does.  Synchronous.
 * *wait_status receives KNIT_ERR_TIMEOUT (the wait ran out) or KNIT_OK;
 * *cleanup_done 1 when the cleanup wait completed.  KNIT_ERR_INVALID for
 * polls out of range or NULL outputs; KNIT_ERR_CUDA on launch failure.
 * Allocates nothing. */
knit_status knit_debug_wait_probe(int64_t polls, int32_t *wait_status, int32_t *cleanup_done);

/* Library version string. */
const char *knit_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KNIT_H */
