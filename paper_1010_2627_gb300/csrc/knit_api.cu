// knit_api.cu -- implementation of the C-ABI declared in include/knit.h:
// argument validation, host/device staging, workspace management and kernel
// launches.  No arithmetic of the method runs here; every step of the path
// is a kernel in sweep_fp64.cu, sweep_mixed.cu or lead_kernels.cu.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/knit.h"
#include "knit_common.cuh"

extern "C" cudaError_t knit_launch_sweep_fp64(const InstDev *, int, int, double2 *, int,
                                              cudaStream_t);
extern "C" cudaError_t knit_launch_ldos_fp64(const InstDev *, int, int, int, double2 *, int,
                                             double2 *, int, double *, long long, cudaStream_t);
extern "C" size_t knit_fp64_smem_bytes(int, int, int);
extern "C" cudaError_t knit_launch_graph_fp64(const GraphDev *, const double *, int, double2 *, int,
                                              double *, int *, cudaStream_t);
extern "C" cudaError_t knit_launch_graph_pick(const double *, int, int, int, int, double *,
                                              cudaStream_t);
extern "C" cudaError_t knit_launch_lesser_fp64(const InstDev *, int, int, int, double2 *, double2 *,
                                               int, const int2 *, int, double *, double *, double *,
                                               double *, cudaStream_t);
extern "C" cudaError_t knit_launch_mixed_impl(const InstDev *, int, int, int, cudaStream_t);
extern "C" int knit_mixed_ctas_per_sm(int, int);
extern "C" int knit_mixed_max_M(void);
extern "C" size_t knit_ldos_mixed_work_bytes(int, int, int);
extern "C" cudaError_t knit_launch_ldos_mixed(const InstDev *, int, int, int, int, void *, double *,
                                              long long, cudaStream_t);
extern "C" size_t knit_mixed_wide_work_bytes(int);
extern "C" cudaError_t knit_launch_mixed_wide(const InstDev *, int, int, void *, cudaStream_t);
extern "C" size_t knit_mixed_tc128_work_bytes(void);
extern "C" cudaError_t knit_launch_mixed_tc128(const InstDev *, int, void *, cudaStream_t);
extern "C" cudaError_t knit_launch_sector_assemble(const double2 *, const int *, int, int, int, int,
                                                   double2 *, cudaStream_t);
extern "C" cudaError_t knit_launch_sector_status(const int *, const int *, int, int, int *, int *,
                                                 cudaStream_t);
extern "C" cudaError_t knit_launch_jacobi(double2 *, double2 *, int, int *, cudaStream_t);
extern "C" cudaError_t knit_launch_sector_unmode(const double2 *, const double2 *, int, int, int, double2 *,
                                                 double2 *, int, cudaStream_t);
extern "C" cudaError_t knit_launch_small_decimation(const double2 *, const double2 *, int, int, int,
                                                    const double *, int, double, double, int,
                                                    double2 *, int *, int *, int, cudaStream_t);
extern "C" cudaError_t knit_launch_sector_ph(const double2 *, const int *, int, int, double2 *, cudaStream_t);
extern "C" cudaError_t knit_launch_sector_ph_status(const int *, const int *, const int *, int, int *, int *,
                                                    cudaStream_t);
extern "C" cudaError_t knit_launch_small_newton(const double2 *, const double2 *, int, int, int,
                                                const double *, int, const float *, long, double, int,
                                                double2 *, int *, int *, cudaStream_t);
extern "C" cudaError_t knit_mlp_block_gmax(const double2 *, int, int, int, float *, cudaStream_t);
extern "C" cudaError_t knit_mlp_targets_blocks(const double2 *, const int *, int, int, int, int, float *,
                                               cudaStream_t);
extern "C" cudaError_t knit_launch_p2_sector_sigma(const double2 *, const int *, int, int, int,
                                                   const double2 *, int, int, double2 *, double2 *,
                                                   int, cudaStream_t);
extern "C" cudaError_t knit_launch_p2_sector_cell(const double2 *, const int *, int, int,
                                                  const double2 *, int, int, double2 *, int,
                                                  cudaStream_t);
extern "C" cudaError_t knit_launch_gamma_factor(const double2 *, int, int, double2 *, double2 *,
                                                int *, cudaStream_t);
extern "C" size_t knit_tau_work_bytes(int);
extern "C" cudaError_t knit_launch_tau(const double2 *, const double2 *, const int *, int, int, int,
                                       const int *, void *, int, double *, double *, cudaStream_t);
extern "C" cudaError_t knit_launch_modes_sigma(const double2 *, const double2 *, int, double,
                                               const double *, int, double2 *, double2 *, int,
                                               cudaStream_t);
extern "C" cudaError_t knit_launch_decimation(const double2 *, const double2 *, int, int, int,
                                              const double *, int, double, double, int, double2 *,
                                              double2 *, double2 *, int *, int *, int,
                                              cudaStream_t);
extern "C" cudaError_t knit_launch_sigma_block(const double2 *, const double2 *, int, int, int, int,
                                               double2 *, double2 *, int, cudaStream_t);
extern "C" cudaError_t knit_launch_decimation_failed(const double2 *, const double2 *, int, int,
                                                     int, const double *, int, double, double, int,
                                                     double2 *, double2 *, double2 *, int *, int *,
                                                     int, cudaStream_t);
extern "C" cudaError_t knit_mlp_linear_fwd(const float *, int, int, const float *, const float *,
                                           int, float *, int, cudaStream_t);
extern "C" cudaError_t knit_mlp_linear_bwd(const float *, const float *, int, int, const float *,
                                           int, float *, float *, float *, int, cudaStream_t);
extern "C" cudaError_t knit_mlp_mse(const float *, const float *, int, float *, float *,
                                    cudaStream_t);
extern "C" cudaError_t knit_mlp_adam(float *, const float *, float *, float *, int, float, int,
                                     cudaStream_t);
extern "C" cudaError_t knit_mlp_inputs(const double *, const int *, int, double, double, float *,
                                       cudaStream_t);
extern "C" cudaError_t knit_mlp_targets(const double2 *, const int *, int, int, float *,
                                        cudaStream_t);
extern "C" cudaError_t knit_launch_lead_newton(const double2 *, const double2 *, int, int,
                                               const double *, int, const float *, double, int,
                                               double2 *, double2 *, int *, int *, int,
                                               cudaStream_t);
extern "C" cudaError_t knit_launch_lead_residual(const double2 *, const double2 *, int, int, int,
                                                 const double *, int, const double2 *, double2 *,
                                                 double *, int, cudaStream_t);

namespace {

thread_local std::string g_err = "no error";

knit_status fail(knit_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

knit_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(KNIT_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(KNIT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Every device allocation of the library goes through dev_alloc, so that a
// test can make the n-th one from now on fail as if the device were out of
// memory (host-side fault injection, armed by knit_debug_fail_alloc_after;
// one-shot; off by default).
std::atomic<long long> g_fail_alloc_after{-1};

cudaError_t dev_alloc(void **p, size_t bytes)
{
    long long k = g_fail_alloc_after.load();
    while (k > 0 && !g_fail_alloc_after.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0 && g_fail_alloc_after.compare_exchange_strong(k, -1)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) *p = nullptr;
    return e;
}

struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t ensure(size_t bytes)
    {
        if (bytes <= n) return cudaSuccess;
        release();
        cudaError_t e = dev_alloc(&p, std::max<size_t>(bytes, 256));
        if (e == cudaSuccess) n = std::max<size_t>(bytes, 256);
        return e;
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

struct Lead {
    double2 *H0 = nullptr, *V = nullptr;   // device copies (Mp x Mp)
    int Mp = 0;         // cell size: M, or 2M for a period-2 lead solved as a supercell
    double2 *C = nullptr;                  // period-2 lead: system-to-surface coupling (M x M)
    int vb = 1;
    int scalar = 0;     // V = t * identity
    double t2 = 0.0;    // |t|^2
    double2 *U = nullptr, *A = nullptr;    // modes: eigenvectors and diagonalised cell
    int modes_ready = 0;
    std::vector<double2> hH0, hV;          // host copies (structure checks)
    // sectors: orbital groups that neither H0 nor V connects (equal sizes ms);
    // sector s holds orbitals sidx[s ms .. s ms + ms - 1] in increasing order
    int nsec = 1, ms = 0;
    double2 *sH0 = nullptr, *sV = nullptr;   // nsec blocks of ms x ms
    int *sidx = nullptr;
    // period-2 lead split in the cell's eigenbasis U (held in U): nsec
    // supercell blocks of 2 ms x 2 ms in sH0 / sV, the modes of block c at
    // sidx[c ms ..]; Cq: the nnz nonzero rows nzr[] of (C or C^dagger) U,
    // modes in block order, transposed (nm x nnz)
    double2 *Cq = nullptr;
    int *nzr = nullptr;
    int nnz = 0;
    // two sectors, the second the particle-hole image of the first:
    // X1 = -S conj(X0) S^dagger for H0 and V, S = 1 (x) i sigma_y on
    // consecutive orbital pairs, so that g1(E) = -S conj(g0(-E)) S^dagger
    int ph = 0;
    // orbital sectors that split further in a mode basis: sector q is
    // Uq diag(block q nsub + r) Uq^dagger with nsub blocks of mu modes each
    // (uU: nsec unitaries of ms x ms, columns grouped by block; uH0 / uV:
    // nsec nsub blocks of mu x mu)
    int nsub = 1, mu = 0;
    double2 *uU = nullptr, *uH0 = nullptr, *uV = nullptr;
};

// U^dagger X U for M x M row-major matrices (host, FP64)
std::vector<double2> unitary_sandwich(const std::vector<double2> &U, const double2 *X, int M)
{
    auto cm = [](double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
    const size_t MM = (size_t)M * M;
    std::vector<double2> T(MM), R(MM);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < M; ++k) {
                const double2 t = cm(X[(size_t)i * M + k], U[(size_t)k * M + j]);
                acc.x += t.x;
                acc.y += t.y;
            }
            T[(size_t)i * M + j] = acc;
        }
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < M; ++k) {
                const double2 u = U[(size_t)k * M + i];
                const double2 t = cm(make_double2(u.x, -u.y), T[(size_t)k * M + j]);
                acc.x += t.x;
                acc.y += t.y;
            }
            R[(size_t)i * M + j] = acc;
        }
    return R;
}

// connected components of the graph on 0 .. n-1 with an edge (i, j) where
// linked(i, j); components in order of their smallest member, members
// increasing
template <typename F>
std::vector<std::vector<int>> graph_components(int n, F linked)
{
    std::vector<int> par(n);
    for (int i = 0; i < n; ++i) par[i] = i;
    auto find = [&](int x) {
        while (par[x] != x) x = par[x] = par[par[x]];
        return x;
    };
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (linked(i, j)) {
                const int a = find(i), b = find(j);
                if (a != b) par[a] = b;
            }
    std::vector<std::vector<int>> comp;
    std::vector<int> slot(n, -1);
    for (int i = 0; i < n; ++i) {
        const int r = find(i);
        if (slot[r] < 0) {
            slot[r] = (int)comp.size();
            comp.emplace_back();
        }
        comp[slot[r]].push_back(i);
    }
    return comp;
}

// Split a lead cell into the connected components of the orbital graph with
// an edge wherever H0 or V (either direction) is non-zero.  Sets ld.nsec and
// fills the sector blocks (host side) when there are at least two components
// of one common size; otherwise leaves the cell whole.
void lead_sectors(Lead &ld, int M, std::vector<double2> &bH0, std::vector<double2> &bV,
                  std::vector<int> &idx)
{
    std::vector<int> par(M);
    for (int i = 0; i < M; ++i) par[i] = i;
    auto find = [&](int x) {
        while (par[x] != x) x = par[x] = par[par[x]];
        return x;
    };
    auto nz = [](double2 v) { return v.x != 0.0 || v.y != 0.0; };
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j)
            if (nz(ld.hH0[(size_t)i * M + j]) || nz(ld.hV[(size_t)i * M + j])) {
                const int a = find(i), b = find(j);
                if (a != b) par[a] = b;
            }
    std::vector<std::vector<int>> comp;
    std::vector<int> slot(M, -1);
    for (int i = 0; i < M; ++i) {
        const int r = find(i);
        if (slot[r] < 0) {
            slot[r] = (int)comp.size();
            comp.emplace_back();
        }
        comp[slot[r]].push_back(i);
    }
    ld.nsec = 1;
    if (comp.size() < 2) return;
    const size_t ms = comp[0].size();
    for (auto &c : comp)
        if (c.size() != ms) return;
    ld.nsec = (int)comp.size();
    ld.ms = (int)ms;
    bH0.assign(comp.size() * ms * ms, make_double2(0.0, 0.0));
    bV = bH0;
    idx.clear();
    for (size_t c = 0; c < comp.size(); ++c) {
        for (size_t a = 0; a < ms; ++a) {
            idx.push_back(comp[c][a]);
            for (size_t b = 0; b < ms; ++b) {
                bH0[(c * ms + a) * ms + b] = ld.hH0[(size_t)comp[c][a] * M + comp[c][b]];
                bV[(c * ms + a) * ms + b] = ld.hV[(size_t)comp[c][a] * M + comp[c][b]];
            }
        }
    }
    // the Nambu structure of a normal BdG lead (Sec. 6.2; basis c_up, c_dn,
    // c_dn^+, -c_up^+): the hole sector is the particle-hole image of the
    // electron sector, X1[a][b] = -(-1)^(a + b) conj(X0[a ^ 1][b ^ 1])
    ld.ph = 0;
    if (comp.size() == 2 && ms % 2 == 0) {
        double scale = 0.0;
        for (size_t q = 0; q < ms * ms; ++q)
            scale = std::max({scale, std::fabs(bH0[q].x) + std::fabs(bH0[q].y), std::fabs(bV[q].x) + std::fabs(bV[q].y)});
        bool ok = true;
        for (size_t a = 0; a < ms && ok; ++a)
            for (size_t b = 0; b < ms && ok; ++b) {
                const double sg = ((a + b) & 1) ? 1.0 : -1.0;
                for (int w = 0; w < 2 && ok; ++w) {
                    const std::vector<double2> &X = w ? bV : bH0;
                    const double2 x0 = X[(a ^ 1) * ms + (b ^ 1)], x1 = X[(ms + a) * ms + b];
                    ok = std::fabs(x1.x - sg * x0.x) + std::fabs(x1.y + sg * x0.y) <= 1e-13 * std::max(scale, 1e-300);
                }
            }
        ld.ph = ok ? 1 : 0;
    }
}

}  // namespace

struct knit_system_s {
    int M = 0, L = 0, block = 1, Vperiod = 1, vb = 1;
    int vtri = 0;   // some V is tridiagonal, not block-diagonal (vb = M then)
    int device = 0, nsm = 1;
    // the same system sliced by half-rows (width M / 2, 2L slices), which runs
    // its KNIT_MIXED sweeps when M > 128; hsup: the half-rows the left and the
    // right self-energy act on (2 x M / 2 sites of the end rows)
    knit_system_s *half = nullptr;
    int *hsup = nullptr;
    int *xmap = nullptr;   // set on a half-row system: its orbitals' row sites
    double2 *H0 = nullptr, *V = nullptr, *h0_val = nullptr;
    double *sign = nullptr, *onsite = nullptr;
    SysDev *d_sys = nullptr;   // device copy of dev() for the kernels' system table
    int *h0_rowptr = nullptr, *h0_col = nullptr;
    int2 *h0_edges = nullptr;  // nonzeros of H0 above the diagonal, row-major (x < y)
    float4 *h0_dfh = nullptr, *h0_dfl = nullptr;   // H0 as double-float, width-128 layout
    int n_edges = 0;
    Lead lead[2];
    int leads_same = 0;
    // grow-only workspaces
    DevBuf E, seeds, T, status, queue, sigL, sigR, gL, gR, lst, lit, lres, work, ckpt, decw, ldos;
    DevBuf p2g, p2s, p2t;   // period-2 leads: supercell g and Sigma, block-product scratch
    DevBuf secs, secg, secst, secit;   // sector leads: per-sector Sigma, g, status, iterations
    DevBuf phE, phmap, phs, phg, phst, phit;   // particle-hole sector pairs: energies, map, first sector
    DevBuf subs, subg, subst, subit, subt;     // mode blocks of a sector: Sigma, g, status, iterations, scratch
    DevBuf gll, tw, ts, tg, trk, tau, noise;   // transmission eigenvalues: G_LL, scratch, W, rank, out
    DevBuf lrl, lrr, ljx, ljt;                 // lesser function outputs staged for host pointers

    SysDev dev() const
    {
        SysDev s;
        s.M = M;
        s.L = L;
        s.block = block;
        s.Vperiod = Vperiod;
        s.vdiag = vb == 1;
        s.vb = vb;
        s.vband = vtri ? 1 : vb;
        s.H0 = H0;
        s.V = V;
        s.sign = sign;
        s.onsite = onsite;
        s.h0_rowptr = h0_rowptr;
        s.h0_col = h0_col;
        s.h0_val = h0_val;
        s.h0_dfh = h0_dfh;
        s.h0_dfl = h0_dfl;
        s.xmap = xmap;
        return s;
    }
};

// an arbitrary geometry with P leads cut into slices of varying width (graph_sweep.cu)
struct knit_graph_s {
    int N = 0, K = 0, Mmax = 0, P = 0, device = 0, nsm = 1;
    std::vector<int> hwidth, hslice_of, hlw;   // slice widths; slice of every site; lead widths
    double2 *blocks = nullptr;
    int *width = nullptr, *lw = nullptr, *lpos = nullptr, *loff = nullptr;
    long long *hoff = nullptr, *voff = nullptr;
    DevBuf work, E, Tm, T, status, sigp, sigs;
};

// learned warm start of a lead's surface Green function (lead_mlp.cu)
struct knit_lead_model_s {
    static constexpr int NL = 4, HID = 128;
    knit_system sys = nullptr;
    int lead = 0, M = 0, device = 0;
    int nsec = 0, nb = 0;   // a lead solved in blocks: nsec blocks of nb x nb (else 0)
    int dims[NL + 1] = {1, HID, HID, HID, 0};
    size_t woff[NL] = {}, boff[NL] = {}, nparam = 0;
    double mid = 0.0, half = 1.0;
    DevBuf params, grads, m, v, act, dact, U, Tt, loss, idx, tmpE;
    int step = 0;
    int maxB = 0;
    knit_lead_model_s(int M_, int nout) : M(M_)
    {
        dims[NL] = nout;
        size_t o = 0;
        for (int l = 0; l < NL; ++l) {
            woff[l] = o;
            o += (size_t)dims[l + 1] * dims[l];
            boff[l] = o;
            o += dims[l + 1];
        }
        nparam = o;
    }
    size_t act_off(int l) const   // activation l (0 = input) for a batch of maxB
    {
        size_t o = 0;
        for (int k = 0; k < l; ++k) o += (size_t)maxB * dims[k];
        return o;
    }
    size_t act_total() const { return act_off(NL + 1); }
};

namespace {

template <typename T>
knit_status to_host(std::vector<T> &dst, const void *src, size_t count, const char *what)
{
    dst.resize(count);
    if (count == 0) return KNIT_OK;
    if (!src) return fail(KNIT_ERR_INVALID, "%s is NULL", what);
    if (is_device_ptr(src))
        CK(cudaMemcpy(dst.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost), what);
    else
        std::memcpy(dst.data(), src, sizeof(T) * count);   // host input: no driver needed
    return KNIT_OK;
}

template <typename T>
knit_status to_device(T **dst, const T *src, size_t count, const char *what)
{
    CK(dev_alloc((void **)dst, sizeof(T) * std::max<size_t>(count, 1)), what);
    if (count) CK(cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice), what);
    return KNIT_OK;
}

// block size of a block-diagonal M x M matrix whose blocks are at most `block`
// wide: 1 if diagonal, `block` if block-diagonal, 0 otherwise
int block_structure(const double2 *A, int M, int block)
{
    bool diag = true, bdiag = true;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            double2 v = A[(size_t)i * M + j];
            if (v.x == 0.0 && v.y == 0.0) continue;
            if (i != j) diag = false;
            if (i / block != j / block) bdiag = false;
        }
    return diag ? 1 : (bdiag ? block : 0);
}

// nonzeros only on the main diagonal and the two next to it
bool tridiagonal(const double2 *A, int M)
{
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            const double2 v = A[(size_t)i * M + j];
            if ((v.x != 0.0 || v.y != 0.0) && std::abs(i - j) > 1) return false;
        }
    return true;
}

bool hermitian(const double2 *A, int M)
{
    double mx = 0.0;
    for (int q = 0; q < M * M; ++q) mx = std::max(mx, std::fabs(A[q].x) + std::fabs(A[q].y));
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            double2 a = A[(size_t)i * M + j], b = A[(size_t)j * M + i];
            if (std::fabs(a.x - b.x) + std::fabs(a.y + b.y) > 1e-12 * std::max(mx, 1.0)) return false;
        }
    return true;
}

bool scalar_identity(const double2 *A, int M, double *t2)
{
    double2 d = A[0];
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            double2 v = A[(size_t)i * M + j];
            if (i == j) {
                if (v.x != d.x || v.y != d.y) return false;
            } else if (v.x != 0.0 || v.y != 0.0) {
                return false;
            }
        }
    *t2 = d.x * d.x + d.y * d.y;
    return *t2 > 0.0;
}

// stage an input array on the device (no copy if it already is device memory)
template <typename T>
knit_status stage_in(DevBuf &buf, const T *src, size_t count, cudaStream_t st, const T **out,
                     const char *what)
{
    if (!src) {
        *out = nullptr;
        return KNIT_OK;
    }
    if (is_device_ptr(src)) {
        *out = src;
        return KNIT_OK;
    }
    CK(buf.ensure(sizeof(T) * count), what);
    CK(cudaMemcpyAsync(buf.p, src, sizeof(T) * count, cudaMemcpyHostToDevice, st), what);
    *out = buf.as<T>();
    return KNIT_OK;
}

template <typename T>
knit_status stage_out(DevBuf &buf, T *dst, size_t count, T **out, bool *host, const char *what)
{
    *host = false;
    if (!dst) {
        *out = nullptr;
        return KNIT_OK;
    }
    if (is_device_ptr(dst)) {
        *out = dst;
        return KNIT_OK;
    }
    *host = true;
    CK(buf.ensure(sizeof(T) * count), what);
    *out = buf.as<T>();
    return KNIT_OK;
}

// Hermitian eigenbasis of an M x M matrix on the device (Jacobi); false when
// the rotations leave an off-diagonal entry above tol (U, D then unset)
knit_status device_eigenbasis(const std::vector<double2> &K, int M, double tol,
                              std::vector<double2> &U, std::vector<double2> &D, bool *ok)
{
    const size_t MM = (size_t)M * M;
    U.assign(MM, make_double2(0.0, 0.0));
    D = U;
    double2 *dA = nullptr, *dU = nullptr;
    CK(dev_alloc((void **)&dA, sizeof(double2) * MM), "lead eigenbasis");
    cudaError_t e = dev_alloc((void **)&dU, sizeof(double2) * MM);
    if (e == cudaSuccess) e = cudaMemcpy(dA, K.data(), sizeof(double2) * MM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = knit_launch_jacobi(dA, dU, M, nullptr, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e == cudaSuccess) e = cudaMemcpy(U.data(), dU, sizeof(double2) * MM, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(D.data(), dA, sizeof(double2) * MM, cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dU);
    CK(e, "lead eigenbasis");
    double off = 0.0;
    for (size_t q = 0; q < MM; ++q)
        if (q / M != q % M) off = std::max(off, std::fabs(D[q].x) + std::fabs(D[q].y));
    *ok = off <= tol;
    return KNIT_OK;
}

// Orbital sectors that split further in a mode basis.  Every unitary
// symmetry of a sector's lead (for the Rashba bar: the transverse mirror
// combined with a spin rotation) commutes with its cell H0 and coupling V,
// hence with K = H0 + a (V + V^dagger) + i b (V - V^dagger), a Hermitian
// element of the algebra they generate.  With b != 0, K is odd under time
// reversal, which lifts the Kramers pairs of a time-reversal invariant lead,
// so its eigenvectors are generically non-degenerate and each carries one
// symmetry label; in that eigenbasis U, U^dagger H0 U and U^dagger V U are
// block-diagonal and every block is a lead of its own: g = U diag(g_r)
// U^dagger, Sigma = U diag(Sigma_r) U^dagger (the fixed point of Sec. 5.3 B
// is covariant under a unitary change of basis).  Entries below 1e-11 of the
// largest |H0|, |V| count as zero (the eigenbasis is exact to ~1e-14).
// Leaves ld.nsub = 1 unless every sector splits into blocks of one common
// size.  bH0 / bV: the nsec sector blocks of ms x ms.
knit_status mode_subsectors(Lead &ld, const std::vector<double2> &bH0, const std::vector<double2> &bV)
{
    ld.nsub = 1;
    const int ns = ld.nsec, ms = ld.ms;
    if (ns < 2 || ms < 2) return KNIT_OK;
    const size_t mm = (size_t)ms * ms;
    constexpr double KA = 0.3711, KB = 0.6180;   // any values with KB != 0 will do
    auto cab = [](double2 v) { return std::fabs(v.x) + std::fabs(v.y); };
    std::vector<double2> uU((size_t)ns * mm), uH, uV;
    int nsub = 0, mu = 0;
    for (int q = 0; q < ns; ++q) {
        const double2 *H = bH0.data() + q * mm, *V = bV.data() + q * mm;
        std::vector<double2> K(mm);
        double scale = 0.0;
        for (int i = 0; i < ms; ++i)
            for (int j = 0; j < ms; ++j) {
                const double2 h = H[(size_t)i * ms + j], v = V[(size_t)i * ms + j];
                const double2 vt = make_double2(V[(size_t)j * ms + i].x, -V[(size_t)j * ms + i].y);   // (V^dagger)_ij
                // a (V + V^dagger) + i b (V - V^dagger)
                K[(size_t)i * ms + j] = make_double2(h.x + KA * (v.x + vt.x) - KB * (v.y - vt.y),
                                                     h.y + KA * (v.y + vt.y) + KB * (v.x - vt.x));
                scale = std::max({scale, cab(h), cab(v)});
            }
        const double tol = 1e-11 * std::max(scale, 1e-300);
        std::vector<double2> U, D;
        bool ok = false;
        knit_status r = device_eigenbasis(K, ms, tol, U, D, &ok);
        if (r != KNIT_OK) return r;
        if (!ok) return KNIT_OK;
        const std::vector<double2> Hh = unitary_sandwich(U, H, ms), Vh = unitary_sandwich(U, V, ms);
        const auto comp = graph_components(ms, [&](int i, int j) {
            return cab(Hh[(size_t)i * ms + j]) > tol || cab(Vh[(size_t)i * ms + j]) > tol;
        });
        const int n = (int)comp.size(), m = (int)comp[0].size();
        if (n < 2) return KNIT_OK;
        for (auto &c : comp)
            if ((int)c.size() != m) return KNIT_OK;
        if (q == 0) {
            nsub = n;
            mu = m;
            uH.assign((size_t)ns * n * m * m, make_double2(0.0, 0.0));
            uV = uH;
        } else if (n != nsub || m != mu) {
            return KNIT_OK;
        }
        // columns of Uq grouped by block; the blocks of H^, V^ (entries
        // between blocks are below tol and dropped)
        for (int c = 0; c < n; ++c)
            for (int a = 0; a < m; ++a) {
                for (int i = 0; i < ms; ++i) uU[q * mm + (size_t)i * ms + c * m + a] = U[(size_t)i * ms + comp[c][a]];
                for (int b = 0; b < m; ++b) {
                    const size_t src = (size_t)comp[c][a] * ms + comp[c][b];
                    const size_t dst = (((size_t)q * n + c) * m + a) * m + b;
                    uH[dst] = Hh[src];
                    uV[dst] = Vh[src];
                }
            }
    }
    knit_status r;
    if ((r = to_device(&ld.uU, uU.data(), uU.size(), "lead mode blocks")) != KNIT_OK ||
        (r = to_device(&ld.uH0, uH.data(), uH.size(), "lead mode blocks")) != KNIT_OK ||
        (r = to_device(&ld.uV, uV.data(), uV.size(), "lead mode blocks")) != KNIT_OK)
        return r;
    ld.nsub = nsub;
    ld.mu = mu;
    return KNIT_OK;
}

// A period-2 lead (cell H0, couplings A inside the two-slice supercell and B
// between supercells, C = B to the system) in the eigenbasis U of H0: the
// supercell blocks that U^dagger A U and U^dagger B U leave decoupled (entries
// below 1e-11 of the largest |H0|, |A|, |B| count as zero), each solved by
// itself (lead_modes_p2.cu).  Leaves ld.nsec = 1 (the whole supercell) when
// the eigenbasis does not split it into blocks of equal size up to 4 modes.
knit_status p2_mode_sectors(Lead &ld, int M, int side, const std::vector<double2> &H0,
                            const double2 *A, const double2 *B)
{
    const size_t MM = (size_t)M * M;
    std::vector<double2> U(MM), D(MM);
    {
        double2 *dA = nullptr;
        CK(dev_alloc((void **)&dA, sizeof(double2) * MM), "lead eigenbasis");
        if (!ld.U) {
            cudaError_t e = dev_alloc((void **)&ld.U, sizeof(double2) * MM);
            if (e != cudaSuccess) {
                cudaFree(dA);
                CK(e, "lead eigenbasis");
            }
        }
        cudaError_t e = cudaMemcpy(dA, H0.data(), sizeof(double2) * MM, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = knit_launch_jacobi(dA, ld.U, M, nullptr, 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(0);
        if (e == cudaSuccess) e = cudaMemcpy(U.data(), ld.U, sizeof(double2) * MM, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(D.data(), dA, sizeof(double2) * MM, cudaMemcpyDeviceToHost);
        cudaFree(dA);
        CK(e, "lead eigenbasis");
    }
    auto cab = [](double2 v) { return std::fabs(v.x) + std::fabs(v.y); };
    auto cm = [](double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
    double scale = 0.0, off = 0.0;
    for (size_t q = 0; q < MM; ++q) {
        scale = std::max({scale, cab(H0[q]), cab(A[q]), cab(B[q])});
        if (q / M != q % M) off = std::max(off, cab(D[q]));
    }
    const double tol = 1e-11 * std::max(scale, 1e-300);
    if (!(off <= tol)) return KNIT_OK;   // the eigensolver did not settle: keep the supercell
    const std::vector<double2> Ah = unitary_sandwich(U, A, M), Bh = unitary_sandwich(U, B, M);
    const auto comp = graph_components(M, [&](int i, int j) {
        return cab(Ah[(size_t)i * M + j]) > tol || cab(Bh[(size_t)i * M + j]) > tol;
    });
    const int ms = (int)comp[0].size(), ns = (int)comp.size();
    if (ns < 2 || ms > 4) return KNIT_OK;
    for (auto &c : comp)
        if ((int)c.size() != ms) return KNIT_OK;
    // per block: the supercell in the mode basis, (slice h, mode a) at h ms + a;
    // left  [[lam, A^], [A^+, lam]] with coupling B^ from slice 1 to slice 0
    // outward, right [[lam, A^+], [A^, lam]] with B^ from slice 0 to slice 1
    const int N = 2 * ms;
    std::vector<double2> sH((size_t)ns * N * N, make_double2(0.0, 0.0)), sV = sH;
    std::vector<int> idx;
    for (int c = 0; c < ns; ++c) {
        double2 *h = sH.data() + (size_t)c * N * N, *v = sV.data() + (size_t)c * N * N;
        for (int a = 0; a < ms; ++a) {
            idx.push_back(comp[c][a]);
            for (int b = 0; b < ms; ++b) {
                const size_t ab = (size_t)comp[c][a] * M + comp[c][b], ba = (size_t)comp[c][b] * M + comp[c][a];
                const double2 ah = Ah[ab], ahd = make_double2(Ah[ba].x, -Ah[ba].y);
                if (a == b) h[a * N + b] = h[(ms + a) * N + ms + b] = D[ab];
                if (side == 0) {
                    h[a * N + ms + b] = ah;
                    h[(ms + a) * N + b] = ahd;
                    v[(ms + a) * N + b] = Bh[ab];
                } else {
                    h[(ms + a) * N + b] = ah;
                    h[a * N + ms + b] = ahd;
                    v[a * N + ms + b] = Bh[ab];
                }
            }
        }
    }
    // Chat = C U (left) or C^dagger U (right), C = B; its nonzero rows
    std::vector<int> nz;
    std::vector<double2> Ch(MM);
    for (int i = 0; i < M; ++i) {
        bool any = false;
        for (int j = 0; j < M; ++j) {
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < M; ++k) {
                const double2 c = side == 0 ? B[(size_t)i * M + k]
                                            : make_double2(B[(size_t)k * M + i].x, -B[(size_t)k * M + i].y);
                const double2 t = cm(c, U[(size_t)k * M + j]);
                acc.x += t.x;
                acc.y += t.y;
            }
            Ch[(size_t)i * M + j] = acc;
            any = any || acc.x != 0.0 || acc.y != 0.0;
        }
        if (any) nz.push_back(i);
    }
    if (nz.empty()) return KNIT_OK;
    const int nnz = (int)nz.size(), nm = ns * ms;
    std::vector<double2> Cq((size_t)nm * nnz);
    for (int q = 0; q < nm; ++q)
        for (int r = 0; r < nnz; ++r) Cq[(size_t)q * nnz + r] = Ch[(size_t)nz[r] * M + idx[q]];
    knit_status r;
    if ((r = to_device(&ld.sH0, sH.data(), sH.size(), "lead blocks")) != KNIT_OK ||
        (r = to_device(&ld.sV, sV.data(), sV.size(), "lead blocks")) != KNIT_OK ||
        (r = to_device(&ld.sidx, idx.data(), idx.size(), "lead blocks")) != KNIT_OK ||
        (r = to_device(&ld.Cq, Cq.data(), Cq.size(), "lead blocks")) != KNIT_OK ||
        (r = to_device(&ld.nzr, nz.data(), nz.size(), "lead blocks")) != KNIT_OK)
        return r;
    ld.nsec = ns;
    ld.ms = ms;
    ld.nnz = nnz;
    return KNIT_OK;
}

// Half-row slicing.  A system whose rows split into halves a_n (the sites
// coupled to row n - 1) and b_n (the rest) such that the coupling to row n + 1
// leaves from b_n only, every half-row carries the same Hamiltonian block, and
// the split repeats with period 2 -- the honeycomb ribbon of Sec. 6.3 cut
// between its two zigzag sublattice rows -- is the chain a_0, b_0, a_1, b_1,
// ... of half the width: H_{b_n, a_n} = H0[b_n, a_n], H_{a_n, b_{n-1}} =
// V_n[a_n, b_{n-1}] (couplings of period 4).  The same Green function, so the
// same transmission, at a quarter of the dense work per row.
struct HalfRows {
    std::vector<int> a[2], b[2];   // by row parity, sites in increasing order
};

bool half_rows(const std::vector<double2> &H0, const std::vector<double2> &V, int M, int P, int B,
               HalfRows &h)
{
    if (B != 1 || (P != 1 && P != 2) || M % 2 || M / 2 > 128) return false;
    auto nz = [](double2 v) { return v.x != 0.0 || v.y != 0.0; };
    const size_t MM = (size_t)M * M;
    for (int pi = 0; pi < 2; ++pi) {
        const double2 *Vn = V.data() + (size_t)(pi % P) * MM, *Vx = V.data() + (size_t)((pi + 1) % P) * MM;
        std::vector<char> ina(M, 0);
        for (int x = 0; x < M; ++x)
            for (int y = 0; y < M; ++y)
                if (nz(Vn[(size_t)x * M + y])) ina[x] = 1;
        h.a[pi].clear();
        h.b[pi].clear();
        for (int x = 0; x < M; ++x) (ina[x] ? h.a[pi] : h.b[pi]).push_back(x);
        if ((int)h.a[pi].size() != M / 2) return false;
        for (int x = 0; x < M; ++x)
            for (int y = 0; y < M; ++y)
                if (nz(Vx[(size_t)x * M + y]) && ina[y]) return false;
    }
    const int Mh = M / 2;
    const std::vector<int> *blk[4] = {&h.a[0], &h.b[0], &h.a[1], &h.b[1]};
    for (int k = 1; k < 4; ++k)
        for (int i = 0; i < Mh; ++i)
            for (int j = 0; j < Mh; ++j) {
                const double2 u = H0[(size_t)(*blk[0])[i] * M + (*blk[0])[j]];
                const double2 v = H0[(size_t)(*blk[k])[i] * M + (*blk[k])[j]];
                if (u.x != v.x || u.y != v.y) return false;
            }
    return true;
}

// the half-row system of `s` (M > 128), or nullptr when s does not split or
// its leads act outside the end half-rows
knit_system make_half_rows(knit_system s, const std::vector<double2> &H0, const std::vector<double2> &V,
                           const std::vector<double> &sign, const std::vector<double> &onsite,
                           const std::vector<double2> *C)
{
    const int M = s->M, L = s->L, Mh = M / 2;
    HalfRows hr;
    if (M <= 128 || !half_rows(H0, V, M, s->Vperiod, s->block, hr)) return nullptr;
    auto nz = [](double2 v) { return v.x != 0.0 || v.y != 0.0; };
    // left Sigma on the rows of its coupling, right Sigma on the columns
    const std::vector<int> &aL = hr.a[0], &bR = hr.b[(L - 1) & 1];
    std::vector<char> inL(M, 0), inR(M, 0);
    for (int x : aL) inL[x] = 1;
    for (int x : bR) inR[x] = 1;
    for (int x = 0; x < M; ++x)
        for (int y = 0; y < M; ++y) {
            if (nz(C[0][(size_t)x * M + y]) && !inL[x]) return nullptr;
            if (nz(C[1][(size_t)x * M + y]) && !inR[y]) return nullptr;
        }
    const size_t mm = (size_t)Mh * Mh, MM = (size_t)M * M;
    std::vector<double2> Hh(mm), Vh(4 * mm);
    const int P = s->Vperiod;
    for (int i = 0; i < Mh; ++i)
        for (int j = 0; j < Mh; ++j) {
            Hh[(size_t)i * Mh + j] = H0[(size_t)hr.a[0][i] * M + hr.a[0][j]];
            // slice m = 2n + h: m % 4 = 0 (n even) a_n <- b_{n-1}, 1 b_n <- a_n,
            // 2 (n odd) a_n <- b_{n-1}, 3 b_n <- a_n
            Vh[0 * mm + (size_t)i * Mh + j] = V[(size_t)(0 % P) * MM + (size_t)hr.a[0][i] * M + hr.b[1][j]];
            Vh[1 * mm + (size_t)i * Mh + j] = H0[(size_t)hr.b[0][i] * M + hr.a[0][j]];
            Vh[2 * mm + (size_t)i * Mh + j] = V[(size_t)(1 % P) * MM + (size_t)hr.a[1][i] * M + hr.b[0][j]];
            Vh[3 * mm + (size_t)i * Mh + j] = H0[(size_t)hr.b[1][i] * M + hr.a[1][j]];
        }
    std::vector<double> on;
    if (!onsite.empty()) {
        on.resize((size_t)2 * L * Mh);
        for (int n = 0; n < L; ++n)
            for (int i = 0; i < Mh; ++i) {
                on[(size_t)(2 * n) * Mh + i] = onsite[(size_t)n * M + hr.a[n & 1][i]];
                on[(size_t)(2 * n + 1) * Mh + i] = onsite[(size_t)n * M + hr.b[n & 1][i]];
            }
    }
    knit_system_desc d{};
    d.M = Mh;
    d.L = 2 * L;
    d.block = 1;
    d.onsite_sign = sign.data();
    d.H0 = (const knit_c128 *)Hh.data();
    d.onsite = on.empty() ? nullptr : on.data();
    d.V = (const knit_c128 *)Vh.data();
    d.Vperiod = 4;
    knit_system h = nullptr;
    if (knit_system_create(&d, &h) != KNIT_OK) return nullptr;
    std::vector<int> xm(4 * Mh), sup(2 * Mh);
    for (int i = 0; i < Mh; ++i) {
        xm[0 * Mh + i] = hr.a[0][i];
        xm[1 * Mh + i] = hr.b[0][i];
        xm[2 * Mh + i] = hr.a[1][i];
        xm[3 * Mh + i] = hr.b[1][i];
        sup[i] = aL[i];
        sup[Mh + i] = bR[i];
    }
    if (to_device(&h->xmap, xm.data(), xm.size(), "half-row map") != KNIT_OK ||
        to_device(&s->hsup, sup.data(), sup.size(), "half-row support") != KNIT_OK) {
        knit_system_destroy(h);
        return nullptr;
    }
    const SysDev sd = h->dev();
    if (cudaMemcpy(h->d_sys, &sd, sizeof(SysDev), cudaMemcpyHostToDevice) != cudaSuccess) {
        knit_system_destroy(h);
        return nullptr;
    }
    return h;
}

knit_status ensure_modes(knit_system s, int p)
{
    Lead &ld = s->lead[p];
    if (ld.modes_ready) return KNIT_OK;
    const size_t MM = (size_t)s->M * s->M;
    if (!ld.U) CK(dev_alloc((void **)&ld.U, sizeof(double2) * MM), "modes U");
    if (!ld.A) CK(dev_alloc((void **)&ld.A, sizeof(double2) * MM), "modes A");
    CK(cudaMemcpy(ld.A, ld.H0, sizeof(double2) * MM, cudaMemcpyDeviceToDevice), "modes copy");
    CK(knit_launch_jacobi(ld.A, ld.U, s->M, nullptr, 0), "jacobi launch");
    CK(cudaStreamSynchronize(0), "jacobi");
    ld.modes_ready = 1;
    return KNIT_OK;
}

int resolve_method(const knit_system s, int p, const knit_lead_opts *o)
{
    int m = o ? o->method : KNIT_LEAD_AUTO;
    if (m == KNIT_LEAD_AUTO) m = s->lead[p].scalar ? KNIT_LEAD_MODES : KNIT_LEAD_DECIMATION;
    return m;
}

// ---- learned lead model helpers
knit_status model_reserve(knit_lead_model md, int B)
{
    if (B <= md->maxB) return KNIT_OK;
    md->maxB = B;
    CK(md->act.ensure(sizeof(float) * md->act_total()), "model activations");
    CK(md->dact.ensure(sizeof(float) * md->act_total()), "model gradients");
    CK(md->Tt.ensure(sizeof(float) * (size_t)B * md->dims[knit_lead_model_s::NL]), "model targets");
    return KNIT_OK;
}

knit_status model_forward(knit_lead_model md, int B, cudaStream_t st)
{
    const int NL = knit_lead_model_s::NL;
    const float *P = md->params.as<float>();
    float *A = md->act.as<float>();
    for (int l = 0; l < NL; ++l)
        CK(knit_mlp_linear_fwd(A + md->act_off(l), B, md->dims[l], P + md->woff[l], P + md->boff[l],
                               md->dims[l + 1], A + md->act_off(l + 1), l < NL - 1 ? 1 : 0, st),
           "model forward");
    return KNIT_OK;
}

// mean squared error against md->Tt, gradients into md->grads, loss added to md->loss
knit_status model_backward(knit_lead_model md, int B, cudaStream_t st)
{
    const int NL = knit_lead_model_s::NL;
    const float *P = md->params.as<float>();
    float *A = md->act.as<float>(), *D = md->dact.as<float>(), *G = md->grads.as<float>();
    const int dout = md->dims[NL];
    CK(knit_mlp_mse(A + md->act_off(NL), md->Tt.as<float>(), B * dout, D + md->act_off(NL),
                    md->loss.as<float>(), st),
       "model loss");
    for (int l = NL - 1; l >= 0; --l)
        CK(knit_mlp_linear_bwd(D + md->act_off(l + 1), A + md->act_off(l), B, md->dims[l],
                               P + md->woff[l], md->dims[l + 1], G + md->woff[l], G + md->boff[l],
                               l > 0 ? D + md->act_off(l) : nullptr, l > 0 ? 1 : 0, st),
           "model backward");
    return KNIT_OK;
}

// Sigma_p at nE device energies into sig (and g into gout), per-energy status into lst
knit_status compute_sigma(knit_system s, int p, const double *dE, int nE,
                          const knit_lead_opts *o, double2 *sig, double2 *gout, int *lst,
                          int *lit, cudaStream_t st)
{
    const int M = s->M;
    const int method = resolve_method(s, p, o);
    const int grid = std::min(nE, s->nsm * 4);
    if (s->lead[p].Mp != M) {
        // period-2 lead: decimation of the two-slice supercell, then the end
        // slice's Sigma from the surface block
        const bool blocks_learned = method == KNIT_LEAD_LEARNED && s->lead[p].nsec > 1 &&
                                    2 * s->lead[p].ms <= 4;
        if (method != KNIT_LEAD_DECIMATION && !blocks_learned)
            return fail(KNIT_ERR_INVALID,
                        "lead %d has period 2: only DECIMATION applies (LEARNED where it splits into blocks "
                        "of at most 4)", p);
        const int Mp = s->lead[p].Mp;
        const size_t MMp = (size_t)Mp * Mp;
        const double eta = (o && o->eta > 0) ? o->eta : 1e-12;
        const double tol = (o && o->tol > 0) ? o->tol : 1e-14;
        const int maxit = (o && o->maxit > 0) ? o->maxit : 200;
        const Lead &ld = s->lead[p];
        if (ld.nsec > 1) {
            // block by block in the cell's eigenbasis (lead_modes_p2.cu), one
            // thread per (block, energy), then Sigma from the surface blocks
            const int ns = ld.nsec, N = 2 * ld.ms;
            const size_t nn = (size_t)N * N;
            CK(s->secg.ensure(sizeof(double2) * nn * nE * ns), "block g");
            CK(s->secst.ensure(sizeof(int) * (size_t)nE * ns), "block status");
            CK(s->secit.ensure(sizeof(int) * (size_t)nE * ns), "block iterations");
            CK(s->p2t.ensure(sizeof(double2) * (size_t)ld.nnz * ns * ld.ms * grid), "block scratch");
            if (method == KNIT_LEAD_LEARNED) {
                // the network's guess for every block, Newton per (block, energy),
                // decimation where Newton did not settle
                knit_lead_model md = o ? (knit_lead_model)o->model[p] : nullptr;
                if (!md || md->sys != s || md->lead != p || md->nsec != ns || md->nb != N)
                    return fail(KNIT_ERR_INVALID, "KNIT_LEAD_LEARNED needs a model trained for this lead");
                knit_status r = model_reserve(md, nE);
                if (r != KNIT_OK) return r;
                CK(knit_mlp_inputs(dE, nullptr, nE, md->mid, md->half, md->act.as<float>(), st),
                   "model inputs");
                if ((r = model_forward(md, nE, st)) != KNIT_OK) return r;
                CK(knit_launch_small_newton(ld.sH0, ld.sV, ns, N, p, dE, nE,
                                            md->act.as<float>() + md->act_off(knit_lead_model_s::NL),
                                            md->dims[knit_lead_model_s::NL], 1e-12, 8,
                                            s->secg.as<double2>(), s->secit.as<int>(), s->secst.as<int>(),
                                            st),
                   "block newton");
                CK(knit_launch_small_decimation(ld.sH0, ld.sV, ns, N, p, dE, nE, eta, tol, maxit,
                                                s->secg.as<double2>(), s->secit.as<int>(),
                                                s->secst.as<int>(), 1, st),
                   "block decimation fallback");
            } else {
                CK(knit_launch_small_decimation(ld.sH0, ld.sV, ns, N, p, dE, nE, eta, tol, maxit,
                                                s->secg.as<double2>(), s->secit.as<int>(),
                                                s->secst.as<int>(), 0, st),
                   "block decimation");
            }
            CK(knit_launch_p2_sector_sigma(ld.Cq, ld.nzr, ld.nnz, ns, ld.ms, s->secg.as<double2>(), M,
                                           nE, s->p2t.as<double2>(), sig, grid, st),
               "block self-energy");
            CK(knit_launch_sector_status(s->secst.as<int>(), s->secit.as<int>(), ns, nE, lst, lit, st),
               "block status");
            (void)gout;
            return KNIT_OK;
        }
        CK(s->decw.ensure(sizeof(double2) * 8 * MMp * grid), "decimation workspace");
        CK(s->p2g.ensure(sizeof(double2) * MMp * nE), "supercell g");
        CK(s->p2s.ensure(sizeof(double2) * MMp * nE), "supercell sigma");
        CK(s->p2t.ensure(sizeof(double2) * (size_t)M * M * grid), "block scratch");
        CK(knit_launch_decimation(s->lead[p].H0, s->lead[p].V, Mp, Mp, p, dE, nE, eta, tol, maxit,
                                  s->decw.as<double2>(), s->p2s.as<double2>(),
                                  s->p2g.as<double2>(), lit, lst, grid, st),
           "supercell decimation");
        CK(knit_launch_sigma_block(s->lead[p].C, s->p2g.as<double2>(), M, Mp, p, nE,
                                   s->p2t.as<double2>(), sig, grid, st),
           "supercell self-energy");
        (void)gout;
        return KNIT_OK;
    }
    if (method == KNIT_LEAD_MODES) {
        if (!s->lead[p].scalar)
            return fail(KNIT_ERR_INVALID, "lead %d: MODES needs lead_V = t * identity", p);
        knit_status r = ensure_modes(s, p);
        if (r != KNIT_OK) return r;
        CK(knit_launch_modes_sigma(s->lead[p].U, s->lead[p].A, M, s->lead[p].t2, dE, nE, sig,
                                   gout, grid, st),
           "modes sigma");
        if (lst) CK(cudaMemsetAsync(lst, 0, sizeof(int) * nE, st), "lead status");
        if (lit) CK(cudaMemsetAsync(lit, 0, sizeof(int) * nE, st), "lead iters");
        return KNIT_OK;
    }
    double eta = (o && o->eta > 0) ? o->eta : 1e-12;
    double tol = (o && o->tol > 0) ? o->tol : 1e-14;
    int maxit = (o && o->maxit > 0) ? o->maxit : 200;
    const size_t MM = (size_t)M * M;
    if (method == KNIT_LEAD_LEARNED) {
        knit_lead_model md = o ? (knit_lead_model)o->model[p] : nullptr;
        if (!md || md->M != M || md->sys != s || md->lead != p)
            return fail(KNIT_ERR_INVALID, "KNIT_LEAD_LEARNED needs a model trained for this lead");
        if (!lit || !lst)
            return fail(KNIT_ERR_INVALID, "KNIT_LEAD_LEARNED needs status and iteration buffers");
        knit_status r = model_reserve(md, nE);
        if (r != KNIT_OK) return r;
        CK(knit_mlp_inputs(dE, nullptr, nE, md->mid, md->half, md->act.as<float>(), st),
           "model inputs");
        if ((r = model_forward(md, nE, st)) != KNIT_OK) return r;
        CK(knit_launch_lead_newton(s->lead[p].H0, s->lead[p].V, M, p, dE, nE,
                                   md->act.as<float>() + md->act_off(knit_lead_model_s::NL), 1e-12,
                                   8, sig, gout, lit, lst, grid, st),
           "lead newton");
        // decimation for the energies Newton did not settle (the fallback, and the
        // arbiter of the warm start's error)
        CK(s->decw.ensure(sizeof(double2) * 8 * MM * grid), "decimation workspace");
        CK(knit_launch_decimation_failed(s->lead[p].H0, s->lead[p].V, M, s->lead[p].vb, p, dE, nE,
                                         eta, tol, maxit, s->decw.as<double2>(), sig, gout, lit,
                                         lst, grid, st),
           "decimation fallback");
        return KNIT_OK;
    }
    if (method != KNIT_LEAD_DECIMATION) return fail(KNIT_ERR_INVALID, "unknown lead method %d", method);
    const Lead &ld = s->lead[p];
    if (ld.nsec > 1) {
        // one decimation per sector (Sec. 5.3 B on each decoupled block), then
        // the blocks put back in the orbital order
        const int ns = ld.nsec, ms = ld.ms;
        const size_t mm = (size_t)ms * ms;
        CK(s->decw.ensure(sizeof(double2) * 8 * mm * grid), "decimation workspace");
        CK(s->secs.ensure(sizeof(double2) * mm * nE * ns), "sector sigma");
        CK(s->secg.ensure(sizeof(double2) * mm * nE * ns), "sector g");
        CK(s->secst.ensure(sizeof(int) * (size_t)nE * ns), "sector status");
        CK(s->secit.ensure(sizeof(int) * (size_t)nE * ns), "sector iterations");
        // sector q at n energies into Sigma / g blocks (ms x ms per energy),
        // status and iterations per energy: the block as a whole, or its mode
        // blocks one by one put back as Uq diag(.) Uq^dagger
        auto sector_decimation = [&](int q, const double *Eq, int n, int gq, double2 *so, double2 *go,
                                     int *ito, int *sto) -> knit_status {
            if (ld.nsub == 1) {
                CK(knit_launch_decimation(ld.sH0 + q * mm, ld.sV + q * mm, ms, ms, p, Eq, n, eta, tol,
                                          maxit, s->decw.as<double2>(), so, go, ito, sto, gq, st),
                   "sector decimation");
                return KNIT_OK;
            }
            const int nb = ld.nsub, mu = ld.mu;
            const size_t uu = (size_t)mu * mu;
            CK(s->subs.ensure(sizeof(double2) * uu * n * nb), "mode blocks");
            CK(s->subg.ensure(sizeof(double2) * uu * n * nb), "mode blocks");
            CK(s->subst.ensure(sizeof(int) * (size_t)n * nb), "mode blocks");
            CK(s->subit.ensure(sizeof(int) * (size_t)n * nb), "mode blocks");
            CK(s->subt.ensure(sizeof(double2) * mm * gq), "mode blocks");
            for (int r = 0; r < nb; ++r) {
                const size_t b = (size_t)q * nb + r;
                CK(knit_launch_decimation(ld.uH0 + b * uu, ld.uV + b * uu, mu, mu, p, Eq, n, eta, tol,
                                          maxit, s->decw.as<double2>(), s->subs.as<double2>() + r * uu * n,
                                          s->subg.as<double2>() + r * uu * n, s->subit.as<int>() + (size_t)r * n,
                                          s->subst.as<int>() + (size_t)r * n, gq, st),
                   "mode block decimation");
            }
            CK(knit_launch_sector_unmode(s->subs.as<double2>(), ld.uU + q * mm, nb, mu, n,
                                         s->subt.as<double2>(), so, gq, st),
               "mode blocks");
            CK(knit_launch_sector_unmode(s->subg.as<double2>(), ld.uU + q * mm, nb, mu, n,
                                         s->subt.as<double2>(), go, gq, st),
               "mode blocks");
            CK(knit_launch_sector_status(s->subst.as<int>(), s->subit.as<int>(), nb, n, sto, ito, st),
               "mode blocks");
            // near a subband edge the doubling can end off its fixed point in
            // one basis and not in the other (the acceptance sits at a 1e-5
            // mismatch there): the energies a block failed, once more on the
            // whole sector
            CK(knit_launch_decimation_failed(ld.sH0 + q * mm, ld.sV + q * mm, ms, ms, p, Eq, n, eta, tol,
                                             maxit, s->decw.as<double2>(), so, go, ito, sto, gq, st),
               "sector decimation of failed energies");
            return KNIT_OK;
        };
        knit_status rs;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(st, &cap), "capture status");
        if (ld.ph && cap == cudaStreamCaptureStatusNone) {
            // particle-hole pair: the electron sector at E and at -E (energies
            // of the list reused where -E is in it, to 1e-12), the hole sector
            // from it; halves the work on a grid symmetric about zero
            std::vector<double> hE(nE);
            CK(cudaMemcpyAsync(hE.data(), dE, sizeof(double) * nE, cudaMemcpyDeviceToHost, st), "energies");
            CK(cudaStreamSynchronize(st), "energies");
            std::vector<int> order(nE), map(nE);
            for (int e = 0; e < nE; ++e) order[e] = e;
            std::sort(order.begin(), order.end(), [&](int a, int b) { return hE[a] < hE[b]; });
            std::vector<double> ext(hE);
            for (int e = 0; e < nE; ++e) {
                const double t = -hE[e], tol = 1e-12 * std::max(1.0, std::fabs(t));
                auto it = std::lower_bound(order.begin(), order.end(), t - tol,
                                           [&](int a, double v) { return hE[a] < v; });
                if (it != order.end() && std::fabs(hE[*it] - t) <= tol) {
                    map[e] = *it;
                } else {
                    map[e] = (int)ext.size();
                    ext.push_back(t);
                }
            }
            const int nX = (int)ext.size();
            CK(s->phE.ensure(sizeof(double) * nX), "particle-hole energies");
            CK(s->phmap.ensure(sizeof(int) * nE), "particle-hole map");
            CK(s->phs.ensure(sizeof(double2) * mm * nX), "particle-hole sector");
            CK(s->phg.ensure(sizeof(double2) * mm * nX), "particle-hole sector");
            CK(s->phst.ensure(sizeof(int) * nX), "particle-hole sector");
            CK(s->phit.ensure(sizeof(int) * nX), "particle-hole sector");
            CK(cudaMemcpy(s->phE.p, ext.data(), sizeof(double) * nX, cudaMemcpyHostToDevice), "energies");
            CK(cudaMemcpy(s->phmap.p, map.data(), sizeof(int) * nE, cudaMemcpyHostToDevice), "map");
            const int gx = std::min(nX, s->nsm * 4);
            CK(s->decw.ensure(sizeof(double2) * 8 * mm * gx), "decimation workspace");
            if ((rs = sector_decimation(0, s->phE.as<double>(), nX, gx, s->phs.as<double2>(),
                                        s->phg.as<double2>(), s->phit.as<int>(), s->phst.as<int>())) != KNIT_OK)
                return rs;
            CK(knit_launch_sector_ph(s->phs.as<double2>(), s->phmap.as<int>(), ms, nE, s->secs.as<double2>(), st),
               "particle-hole sector");
            CK(knit_launch_sector_ph(s->phg.as<double2>(), s->phmap.as<int>(), ms, nE, s->secg.as<double2>(), st),
               "particle-hole sector");
            CK(knit_launch_sector_ph_status(s->phst.as<int>(), s->phit.as<int>(), s->phmap.as<int>(), nE,
                                            s->secst.as<int>(), s->secit.as<int>(), st),
               "particle-hole sector");
        } else {
            for (int q = 0; q < ns; ++q)
                if ((rs = sector_decimation(q, dE, nE, grid, s->secs.as<double2>() + q * mm * nE,
                                            s->secg.as<double2>() + q * mm * nE,
                                            s->secit.as<int>() + (size_t)q * nE,
                                            s->secst.as<int>() + (size_t)q * nE)) != KNIT_OK)
                    return rs;
        }
        CK(knit_launch_sector_assemble(s->secs.as<double2>(), ld.sidx, ns, ms, M, nE, sig, st),
           "sector sigma assembly");
        if (gout)
            CK(knit_launch_sector_assemble(s->secg.as<double2>(), ld.sidx, ns, ms, M, nE, gout, st),
               "sector g assembly");
        CK(knit_launch_sector_status(s->secst.as<int>(), s->secit.as<int>(), ns, nE, lst, lit, st),
           "sector status");
        return KNIT_OK;
    }
    CK(s->decw.ensure(sizeof(double2) * 8 * MM * grid), "decimation workspace");
    CK(knit_launch_decimation(s->lead[p].H0, s->lead[p].V, M, s->lead[p].vb, p, dE, nE, eta, tol,
                              maxit, s->decw.as<double2>(), sig, gout, lit, lst, grid, st),
       "decimation");
    return KNIT_OK;
}

knit_status check_system(knit_system s)
{
    if (!s) return fail(KNIT_ERR_INVALID, "NULL system");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    return KNIT_OK;
}

// Sigma_L / Sigma_R for the energies in dE; combined per-energy status in s->lst
knit_status both_sigmas(knit_system s, const double *dE, int nE, const knit_lead_opts *o,
                        cudaStream_t st, const double2 **sL, const double2 **sR, const int **lst)
{
    const size_t MM = (size_t)s->M * s->M;
    CK(s->sigL.ensure(sizeof(double2) * MM * nE), "sigma workspace");
    CK(s->gL.ensure(sizeof(double2) * MM * nE), "g workspace");
    CK(s->lst.ensure(sizeof(int) * 2 * nE), "lead status");
    int *st0 = s->lst.as<int>(), *st1 = st0 + nE;
    CK(s->lit.ensure(sizeof(int) * nE * 2), "iterations");
    knit_status r = compute_sigma(s, 0, dE, nE, o, s->sigL.as<double2>(), s->gL.as<double2>(),
                                  st0, s->lit.as<int>(), st);
    if (r != KNIT_OK) return r;
    *sL = s->sigL.as<double2>();
    if (s->leads_same && s->lead[0].scalar && resolve_method(s, 1, o) == KNIT_LEAD_MODES) {
        *sR = *sL;    // V = t I and identical cells: Sigma_R = Sigma_L
        CK(cudaMemsetAsync(st1, 0, sizeof(int) * nE, st), "lead status");
    } else {
        CK(s->sigR.ensure(sizeof(double2) * MM * nE), "sigma workspace");
        CK(s->gR.ensure(sizeof(double2) * MM * nE), "g workspace");
        r = compute_sigma(s, 1, dE, nE, o, s->sigR.as<double2>(), s->gR.as<double2>(), st1,
                          s->lit.as<int>() + nE, st);
        if (r != KNIT_OK) return r;
        *sR = s->sigR.as<double2>();
    }
    *lst = st0;   // the sweep reads st0[e] | st1[e] through the combined array below
    return KNIT_OK;
}

// Sigma_L / Sigma_R (M x M per energy) restricted to the end half-rows
// sup[0 .. Mh - 1] / sup[Mh .. 2 Mh - 1]; an energy whose self-energy has an
// entry outside them (which the half-row chain cannot carry) gets status
// KNIT_ERR_INVALID in lst (per energy, copied from lin or zero first).  One
// CTA per energy (grid-stride).
__global__ void __launch_bounds__(256)
half_sigma_kernel(const double2 *SL, const double2 *SR, int M, const int *sup, int Mh, int nE,
                  double2 *hL, double2 *hR, const int *lin, int *lst)
{
    __shared__ unsigned char inL[256], inR[256];
    __shared__ int bad;
    for (int x = threadIdx.x; x < M; x += blockDim.x) inL[x] = inR[x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < Mh; i += blockDim.x) {
        inL[sup[i]] = 1;
        inR[sup[Mh + i]] = 1;
    }
    __syncthreads();
    const size_t MM = (size_t)M * M, mm = (size_t)Mh * Mh;
    for (int e = blockIdx.x; e < nE; e += gridDim.x) {
        if (threadIdx.x == 0) bad = 0;
        __syncthreads();
        int b = 0;
        for (size_t q = threadIdx.x; q < MM; q += blockDim.x) {
            const int x = (int)(q / M), y = (int)(q % M);
            const double2 l = SL[e * MM + q], r = SR[e * MM + q];
            if ((l.x != 0.0 || l.y != 0.0) && !(inL[x] && inL[y])) b = 1;
            if ((r.x != 0.0 || r.y != 0.0) && !(inR[x] && inR[y])) b = 1;
        }
        if (b) bad = 1;
        for (size_t q = threadIdx.x; q < mm; q += blockDim.x) {
            const int i = (int)(q / Mh), j = (int)(q % Mh);
            hL[e * mm + q] = SL[e * MM + (size_t)sup[i] * M + sup[j]];
            hR[e * mm + q] = SR[e * MM + (size_t)sup[Mh + i] * M + sup[Mh + j]];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int s0 = lin ? lin[e] : 0;
            lst[e] = s0 != 0 ? s0 : (bad ? (int)KNIT_ERR_INVALID : 0);
        }
        __syncthreads();
    }
}

__global__ void combine_status(int *a, const int *b, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && a[i] == 0) a[i] = b[i];
}

// which sweep kernel serves a system at a given precision
enum SweepKind { SWEEP_FP64 = 0, SWEEP_MIXED = 1, SWEEP_WIDE = 2, SWEEP_TC128 = 3, SWEEP_HALF = 4 };

// KNIT_MIXED: widths <= 64 with diagonal couplings on sweep_mixed(_tc).cu,
// everything else up to 128 (diagonal, 4 x 4 block or tridiagonal couplings)
// on the tensor-core kernel of sweep_mixed_tc128.cu; KNIT_MIXED_CUDACORE
// keeps the CUDA-core residual kernels (sweep_mixed.cu, sweep_mixed_wide.cu),
// which take diagonal and 4 x 4 block couplings
// SWEEP_HALF (only where half_ok: an energy x seed grid without G_LL):
// KNIT_MIXED on a system wider than 128 that splits into half-rows runs the
// tensor-core kernel on the half-row chain
int sweep_kind(const knit_system_s *s, int precision, bool half_ok = false)
{
    if (precision == KNIT_FP64) return SWEEP_FP64;
    if (half_ok && precision == KNIT_MIXED && s->half) return SWEEP_HALF;
    if (s->vb == 1 && s->M <= knit_mixed_max_M()) return SWEEP_MIXED;
    if (s->M > 128) return SWEEP_FP64;
    if (precision == KNIT_MIXED && (s->vb == 1 || s->vb == 4 || s->vtri)) return SWEEP_TC128;
    if (precision == KNIT_MIXED_CUDACORE && (s->vb == 1 || s->vb == 4)) return SWEEP_WIDE;
    return SWEEP_FP64;
}

knit_status run_sweep(knit_system s, InstDev in, int precision, cudaStream_t st)
{
    in.sys = s->d_sys;
    CK(s->queue.ensure(sizeof(int)), "queue");
    in.queue = s->queue.as<int>();
    CK(cudaMemsetAsync(in.queue, 0, sizeof(int), st), "queue reset");
    const int grid = std::max(1, std::min(in.n, s->nsm));
    const int kind = sweep_kind(s, precision, !in.per_instance && !in.GLL);
    if (kind == SWEEP_HALF) {
        knit_system h = s->half;
        const int nE = in.n / in.nS, Mh = h->M;
        const size_t mm = (size_t)Mh * Mh;
        CK(h->sigL.ensure(sizeof(double2) * mm * nE), "half-row sigma");
        CK(h->sigR.ensure(sizeof(double2) * mm * nE), "half-row sigma");
        CK(h->lst.ensure(sizeof(int) * nE), "half-row lead status");
        CK(h->queue.ensure(sizeof(int)), "queue");
        half_sigma_kernel<<<std::max(1, std::min(nE, 4 * s->nsm)), 256, 0, st>>>(
            in.sigL, in.sigR, s->M, s->hsup, Mh, nE, h->sigL.as<double2>(), h->sigR.as<double2>(),
            in.lstatus, h->lst.as<int>());
        CK(cudaGetLastError(), "half-row sigma");
        InstDev hi = in;
        hi.sys = h->d_sys;
        hi.sigL = h->sigL.as<double2>();
        hi.sigR = h->sigR.as<double2>();
        hi.lstatus = h->lst.as<int>();
        hi.queue = h->queue.as<int>();
        CK(cudaMemsetAsync(hi.queue, 0, sizeof(int), st), "queue reset");
        CK(h->work.ensure(knit_mixed_tc128_work_bytes() * grid), "tensor-core sweep workspace");
        CK(knit_launch_mixed_tc128(&hi, grid, h->work.p, st), "half-row sweep launch");
        return KNIT_OK;
    }
    if (kind == SWEEP_MIXED) {
        CK(knit_launch_mixed_impl(&in, s->M, grid, precision == KNIT_MIXED, st), "mixed sweep launch");
        return KNIT_OK;
    }
    if (kind == SWEEP_WIDE) {
        CK(s->work.ensure(knit_mixed_wide_work_bytes(s->M) * grid), "wide sweep workspace");
        CK(knit_launch_mixed_wide(&in, s->M, grid, s->work.p, st), "wide mixed sweep launch");
        return KNIT_OK;
    }
    if (kind == SWEEP_TC128) {
        CK(s->work.ensure(knit_mixed_tc128_work_bytes() * grid), "tensor-core sweep workspace");
        CK(knit_launch_mixed_tc128(&in, grid, s->work.p, st), "tensor-core wide sweep launch");
        return KNIT_OK;
    }
    const size_t MM = (size_t)s->M * s->M;
    int use_smem = knit_fp64_smem_bytes(s->M, 1, 3) <= 220 * 1024;
    if (!use_smem) CK(s->work.ensure(sizeof(double2) * 3 * MM * grid), "sweep workspace");
    CK(knit_launch_sweep_fp64(&in, s->M, grid, s->work.as<double2>(), use_smem, st),
       "fp64 sweep launch");
    return KNIT_OK;
}

knit_status check_batch(knit_system s, const double *E, int nE, int nS, int precision, double W)
{
    if (!E) return fail(KNIT_ERR_INVALID, "E is NULL");
    if (nE <= 0 || nS <= 0) return fail(KNIT_ERR_INVALID, "nE and nS must be positive");
    if ((long long)nE * nS > 0x7fffffffLL) return fail(KNIT_ERR_INVALID, "nE * nS too large");
    if (!std::isfinite(W)) return fail(KNIT_ERR_INVALID, "W is not finite");
    if (precision != KNIT_FP64 && precision != KNIT_MIXED && precision != KNIT_MIXED_CUDACORE)
        return fail(KNIT_ERR_INVALID, "unknown precision %d", precision);
    return KNIT_OK;
}

knit_status finish(cudaStream_t st, bool sync, const char *what)
{
    CK(cudaGetLastError(), what);
    if (sync) CK(cudaStreamSynchronize(st), what);
    return KNIT_OK;
}

}  // namespace

// ===========================================================================
// Heterogeneous batches: instances of several systems, grouped per system for
// the lead solvers and per kernel variant ("bucket") for the sweep, each
// bucket's queue in decreasing cost M^3 L (longest-processing-time order).

namespace {

__global__ void gather_instances(const double *E, const uint64_t *seeds, const double *W,
                                 const int *perm, int n, double *Ep, uint64_t *Sp, double *Wp)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = perm[p];
    Ep[p] = E[i];
    Sp[p] = seeds ? seeds[i] : 0ull;
    Wp[p] = W ? W[i] : 0.0;
}

__global__ void fill_int(int *a, int n, int v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

}  // namespace

struct knit_batch_s {
    struct Bucket {
        int kind = 0;          // 0 FP64 sweep, 1 mixed M <= 64, 2 mixed wide, 3 tensor-core M <= 128
        int use_tc = 0;
        int Mmax = 0, Lmax = 0;
        int ctas = 1, max_ctas = 1;   // CTAs per SM of its persistent launch
        double cost0 = 0.0;           // M^3 L of its heaviest instance
        size_t work_off = 0;          // its part of the workspace (bytes)
        std::vector<int> order;   // plan positions in cost order
        DevBuf d_order;
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
    };
    cudaEvent_t ready = nullptr;
    int nInst = 0, precision = 0, device = 0, nsm = 1;
    std::vector<knit_system> sys;            // distinct systems (not owned)
    std::vector<int> perm;                   // plan position -> caller's instance
    std::vector<int> start, count;           // per system: first plan position, count
    std::vector<long long> sig_off;          // per plan position (elements)
    long long sig_total = 0, g_max = 0;
    std::vector<Bucket> buckets;
    DevBuf d_systab, d_sys_of, d_perm, d_sig_off, E, seeds, W, Ep, Sp, Wp, sigL, sigR, gbuf,
        lst, T, status, queue, work;
};

namespace {

knit_status batch_release(knit_batch b)
{
    DevBuf *bufs[] = {&b->d_systab, &b->d_sys_of, &b->d_perm, &b->d_sig_off, &b->E, &b->seeds,
                      &b->W, &b->Ep, &b->Sp, &b->Wp, &b->sigL, &b->sigR, &b->gbuf, &b->lst,
                      &b->T, &b->status, &b->queue, &b->work};
    for (DevBuf *x : bufs) x->release();
    for (auto &bk : b->buckets) {
        bk.d_order.release();
        if (bk.stream) cudaStreamDestroy(bk.stream);
        if (bk.done) cudaEventDestroy(bk.done);
        bk.stream = nullptr;
        bk.done = nullptr;
    }
    if (b->ready) cudaEventDestroy(b->ready);
    b->ready = nullptr;
    return KNIT_OK;
}

}  // namespace

extern "C" {

const char *knit_last_error(void) { return g_err.c_str(); }

// lets other translation units of the library report an error message
void knit_set_last_error(const char *msg) { g_err = msg ? msg : "unknown error"; }

const char *knit_version(void) { return "knit-gb300 0.1 (sm_103a)"; }

knit_status knit_debug_fail_alloc_after(int64_t n)
{
    g_fail_alloc_after.store(n < 0 ? -1 : (long long)n);
    return KNIT_OK;
}

knit_status knit_system_create(const knit_system_desc *d, knit_system *out)
{
    if (!d || !out) return fail(KNIT_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const int M = d->M, L = d->L, B = d->block, P = d->Vperiod;
    if (M < 1 || M > 256) return fail(KNIT_ERR_INVALID, "M = %d out of range [1, 256]", M);
    if (L < 1) return fail(KNIT_ERR_INVALID, "L = %d must be >= 1", L);
    if (B != 1 && B != 2 && B != 4) return fail(KNIT_ERR_INVALID, "block must be 1, 2 or 4");
    if (M % B) return fail(KNIT_ERR_INVALID, "M must be a multiple of block");
    if (P != 1 && P != 2 && P != 4) return fail(KNIT_ERR_INVALID, "Vperiod must be 1, 2 or 4");
    if (!d->H0 || !d->V) return fail(KNIT_ERR_INVALID, "H0 and V are required");
    const size_t MM = (size_t)M * M;
    std::vector<double2> H0, V, sign, onsite_dummy;
    std::vector<double> hs, hon;
    knit_status r;
    if ((r = to_host(H0, d->H0, MM, "H0")) != KNIT_OK) return r;
    if ((r = to_host(V, d->V, MM * P, "V")) != KNIT_OK) return r;
    if (!hermitian(H0.data(), M)) return fail(KNIT_ERR_INVALID, "H0 is not Hermitian");
    int vb = 1, vtri = 0;
    for (int q = 0; q < P; ++q) {
        int b = block_structure(V.data() + q * MM, M, B);
        if (b == 0 && tridiagonal(V.data() + q * MM, M)) {
            vtri = 1;
            b = M;   // the FP64 paths treat it as a dense coupling
        }
        if (b == 0)
            return fail(KNIT_ERR_INVALID, "V[%d] is neither block-diagonal with %dx%d blocks nor tridiagonal",
                        q, B, B);
        vb = std::max(vb, b);
    }
    hs.assign(B, 1.0);
    if (d->onsite_sign && (r = to_host(hs, d->onsite_sign, B, "onsite_sign")) != KNIT_OK) return r;
    if (d->onsite && (r = to_host(hon, d->onsite, (size_t)L * M, "onsite")) != KNIT_OK) return r;
    for (double v : hon)
        if (!std::isfinite(v)) return fail(KNIT_ERR_INVALID, "onsite has non-finite values");

    knit_system s = new (std::nothrow) knit_system_s;
    if (!s) return fail(KNIT_ERR_OOM, "host allocation");
    s->M = M;
    s->L = L;
    s->block = B;
    s->Vperiod = P;
    s->vb = vb;
    s->vtri = vtri;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device);
    // sparse rows of H0 for the mixed residual
    std::vector<int> rp(M + 1, 0), cols;
    std::vector<double2> vals;
    for (int i = 0; i < M; ++i) {
        for (int j = 0; j < M; ++j) {
            double2 v = H0[(size_t)i * M + j];
            if (v.x != 0.0 || v.y != 0.0) {
                cols.push_back(j);
                vals.push_back(v);
            }
        }
        rp[i + 1] = (int)cols.size();
    }
    std::vector<double2> hC[2], cellH[2], cellA[2];   // period-2 leads: C = V_first, H0, V_second
    for (int p = 0; p < 2; ++p) {
        Lead &ld = s->lead[p];
        const int per = d->lead_Vperiod[p] <= 1 ? 1 : d->lead_Vperiod[p];
        if (per != 1 && per != 2) {
            knit_system_destroy(s);
            return fail(KNIT_ERR_INVALID, "lead_Vperiod[%d] must be 0, 1 or 2", p);
        }
        const void *hsrc = d->lead_H0[p] ? (const void *)d->lead_H0[p] : (const void *)d->H0;
        if ((r = to_host(ld.hH0, hsrc, MM, "lead_H0")) != KNIT_OK) {
            knit_system_destroy(s);
            return r;
        }
        if (!hermitian(ld.hH0.data(), M)) {
            knit_system_destroy(s);
            return fail(KNIT_ERR_INVALID, "lead_H0[%d] is not Hermitian", p);
        }
        if (per == 1) {
            const void *vsrc = d->lead_V[p] ? (const void *)d->lead_V[p] : (const void *)d->V;
            if ((r = to_host(ld.hV, vsrc, MM, "lead_V")) != KNIT_OK) {
                knit_system_destroy(s);
                return r;
            }
            ld.Mp = M;
            int b = block_structure(ld.hV.data(), M, B);
            ld.vb = b == 0 ? M : b;   // dense coupling allowed for the decimation solver
            ld.scalar = scalar_identity(ld.hV.data(), M, &ld.t2);
            continue;
        }
        // period 2: [V_first, V_second], given or continuing the system's V
        std::vector<double2> vv;
        if (d->lead_V[p]) {
            if ((r = to_host(vv, d->lead_V[p], 2 * MM, "lead_V")) != KNIT_OK) {
                knit_system_destroy(s);
                return r;
            }
        } else {
            const int n0 = p == 0 ? 0 : L % P, n1 = p == 0 ? 1 % P : (L + 1) % P;
            vv.assign(V.begin() + (size_t)n0 * MM, V.begin() + (size_t)(n0 + 1) * MM);
            vv.insert(vv.end(), V.begin() + (size_t)n1 * MM, V.begin() + (size_t)(n1 + 1) * MM);
        }
        const double2 *Vf = vv.data(), *Vs = vv.data() + MM;
        cellH[p] = ld.hH0;
        cellA[p].assign(Vs, Vs + MM);
        // supercell (surface slice first): left  H0c = [[H0, A], [A^+, H0]], coupling to the
        // next cell outward [[0, 0], [B, 0]]; right H0c = [[H0, A^+], [A, H0]], coupling
        // [[0, B], [0, 0]] (slice-forward orientation); A = V_second, B = V_first
        const int Mp = 2 * M;
        ld.Mp = Mp;
        std::vector<double2> Hc((size_t)Mp * Mp, make_double2(0.0, 0.0)), Vc = Hc;
        auto at = [&](std::vector<double2> &X, int i, int j) -> double2 & { return X[(size_t)i * Mp + j]; };
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) {
                const double2 h = ld.hH0[(size_t)i * M + j];
                const double2 a = Vs[(size_t)i * M + j], b = Vf[(size_t)i * M + j];
                const double2 ad = make_double2(Vs[(size_t)j * M + i].x, -Vs[(size_t)j * M + i].y);
                at(Hc, i, j) = h;
                at(Hc, M + i, M + j) = h;
                if (p == 0) {
                    at(Hc, i, M + j) = a;
                    at(Hc, M + i, j) = ad;
                    at(Vc, M + i, j) = b;
                } else {
                    at(Hc, M + i, j) = a;
                    at(Hc, i, M + j) = ad;
                    at(Vc, i, M + j) = b;
                }
            }
        ld.hH0 = Hc;
        ld.hV = Vc;
        hC[p].assign(Vf, Vf + MM);
        ld.vb = Mp;
        ld.scalar = 0;
    }
    s->leads_same = s->lead[0].Mp == M && s->lead[1].Mp == M && std::equal(s->lead[0].hH0.begin(), s->lead[0].hH0.end(), s->lead[1].hH0.begin(),
                               [](double2 a, double2 b) { return a.x == b.x && a.y == b.y; }) &&
                    std::equal(s->lead[0].hV.begin(), s->lead[0].hV.end(), s->lead[1].hV.begin(),
                               [](double2 a, double2 b) { return a.x == b.x && a.y == b.y; });
    std::vector<int2> edges;
    for (int x = 0; x < M; ++x)
        for (int y = x + 1; y < M; ++y) {
            const double2 h = H0[(size_t)x * M + y];
            if (h.x != 0.0 || h.y != 0.0) edges.push_back(make_int2(x, y));
        }
    s->n_edges = (int)edges.size();
    if (!edges.empty() && (r = to_device(&s->h0_edges, edges.data(), edges.size(), "H0 edges")) != KNIT_OK) {
        knit_system_destroy(s);
        return r;
    }
    if ((r = to_device(&s->H0, H0.data(), MM, "H0")) != KNIT_OK ||
        (r = to_device(&s->V, V.data(), MM * P, "V")) != KNIT_OK ||
        (r = to_device(&s->sign, hs.data(), (size_t)B, "sign")) != KNIT_OK ||
        (r = to_device(&s->h0_rowptr, rp.data(), rp.size(), "H0 rows")) != KNIT_OK ||
        (r = to_device(&s->h0_col, cols.data(), cols.size(), "H0 cols")) != KNIT_OK ||
        (r = to_device(&s->h0_val, vals.data(), vals.size(), "H0 vals")) != KNIT_OK) {
        knit_system_destroy(s);
        return r;
    }
    if (M <= 128) {
        // H0 in double-float, columns in pairs (jp, row i) as the width-128 sweep reads it
        std::vector<float4> fh(64 * 128, make_float4(0.f, 0.f, 0.f, 0.f)), fl = fh;
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) {
                const double2 v = H0[(size_t)i * M + j];
                const float hx = (float)v.x, hy = (float)v.y;
                const float lx = (float)(v.x - (double)hx), ly = (float)(v.y - (double)hy);
                float4 &a = fh[(j >> 1) * 128 + i], &b = fl[(j >> 1) * 128 + i];
                if (j & 1) { a.z = hx; a.w = hy; b.z = lx; b.w = ly; }
                else { a.x = hx; a.y = hy; b.x = lx; b.y = ly; }
            }
        if ((r = to_device(&s->h0_dfh, fh.data(), fh.size(), "H0 double-float")) != KNIT_OK ||
            (r = to_device(&s->h0_dfl, fl.data(), fl.size(), "H0 double-float")) != KNIT_OK) {
            knit_system_destroy(s);
            return r;
        }
    }
    if (d->onsite && (r = to_device(&s->onsite, hon.data(), hon.size(), "onsite")) != KNIT_OK) {
        knit_system_destroy(s);
        return r;
    }
    for (int p = 0; p < 2; ++p) {
        Lead &ld = s->lead[p];
        const size_t MMp = (size_t)ld.Mp * ld.Mp;
        if ((r = to_device(&ld.H0, ld.hH0.data(), MMp, "lead_H0")) != KNIT_OK ||
            (r = to_device(&ld.V, ld.hV.data(), MMp, "lead_V")) != KNIT_OK ||
            (ld.Mp != M && (r = to_device(&ld.C, hC[p].data(), MM, "lead coupling")) != KNIT_OK)) {
            knit_system_destroy(s);
            return r;
        }
        if (ld.Mp != M) {
            if ((r = p2_mode_sectors(ld, M, p, cellH[p], cellA[p].data(), hC[p].data())) != KNIT_OK) {
                knit_system_destroy(s);
                return r;
            }
        } else if (!ld.scalar) {
            std::vector<double2> bH0, bV;
            std::vector<int> idx;
            lead_sectors(ld, M, bH0, bV, idx);
            if (ld.nsec > 1 &&
                ((r = to_device(&ld.sH0, bH0.data(), bH0.size(), "lead sectors")) != KNIT_OK ||
                 (r = to_device(&ld.sV, bV.data(), bV.size(), "lead sectors")) != KNIT_OK ||
                 (r = to_device(&ld.sidx, idx.data(), idx.size(), "lead sectors")) != KNIT_OK ||
                 (r = mode_subsectors(ld, bH0, bV)) != KNIT_OK)) {
                knit_system_destroy(s);
                return r;
            }
        }
    }
    {
        SysDev sd = s->dev();
        if ((r = to_device(&s->d_sys, &sd, 1, "system table")) != KNIT_OK) {
            knit_system_destroy(s);
            return r;
        }
    }
    if (M > 128) {
        const std::vector<double2> C[2] = {s->lead[0].Mp == M ? s->lead[0].hV : hC[0],
                                           s->lead[1].Mp == M ? s->lead[1].hV : hC[1]};
        const std::string keep = g_err;   // a system that does not split is no error
        s->half = make_half_rows(s, H0, V, hs, hon, C);
        g_err = keep;
    }
    *out = s;
    return KNIT_OK;
}

knit_status knit_system_destroy(knit_system s)
{
    if (!s) return KNIT_OK;
    cudaSetDevice(s->device);
    knit_system_destroy(s->half);
    cudaFree(s->hsup);
    cudaFree(s->xmap);
    cudaFree(s->H0);
    cudaFree(s->V);
    cudaFree(s->sign);
    cudaFree(s->onsite);
    cudaFree(s->h0_rowptr);
    cudaFree(s->h0_col);
    cudaFree(s->h0_val);
    cudaFree(s->h0_edges);
    cudaFree(s->h0_dfh);
    cudaFree(s->h0_dfl);
    cudaFree(s->d_sys);
    for (int p = 0; p < 2; ++p) {
        cudaFree(s->lead[p].H0);
        cudaFree(s->lead[p].V);
        cudaFree(s->lead[p].C);
        cudaFree(s->lead[p].U);
        cudaFree(s->lead[p].A);
        cudaFree(s->lead[p].sH0);
        cudaFree(s->lead[p].sV);
        cudaFree(s->lead[p].sidx);
        cudaFree(s->lead[p].Cq);
        cudaFree(s->lead[p].nzr);
        cudaFree(s->lead[p].uU);
        cudaFree(s->lead[p].uH0);
        cudaFree(s->lead[p].uV);
    }
    DevBuf *bufs[] = {&s->E, &s->seeds, &s->T, &s->status, &s->queue, &s->sigL, &s->sigR, &s->gL,
                      &s->gR, &s->lst, &s->lit, &s->lres, &s->work, &s->ckpt, &s->decw, &s->ldos,
                      &s->p2g, &s->p2s, &s->p2t, &s->gll, &s->tw, &s->ts, &s->tg, &s->trk,
                      &s->tau, &s->noise, &s->lrl, &s->lrr, &s->ljx, &s->ljt, &s->secs,
                      &s->secg, &s->secst, &s->secit, &s->phE, &s->phmap, &s->phs, &s->phg,
                      &s->phst, &s->phit, &s->subs, &s->subg, &s->subst, &s->subit, &s->subt};
    for (DevBuf *b : bufs) b->release();
    delete s;
    return KNIT_OK;
}

knit_status knit_lead_selfenergy(knit_system s, int32_t lead, const double *E, int32_t nE,
                                 const knit_lead_opts *opts, knit_c128 *sigma, int32_t *iters,
                                 double *residual, void *stream)
{
    knit_status r = check_system(s);
    if (r != KNIT_OK) return r;
    if (lead != 0 && lead != 1) return fail(KNIT_ERR_INVALID, "lead must be 0 or 1");
    if (!E || nE <= 0 || !sigma) return fail(KNIT_ERR_INVALID, "E, nE and sigma are required");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t MM = (size_t)s->M * s->M;
    const double *dE;
    if ((r = stage_in(s->E, E, (size_t)nE, st, &dE, "E")) != KNIT_OK) return r;
    double2 *dS = nullptr;
    bool hS;
    if ((r = stage_out(s->sigL, (double2 *)sigma, MM * nE, &dS, &hS, "sigma")) != KNIT_OK) return r;
    CK(s->gL.ensure(sizeof(double2) * MM * nE), "g workspace");
    CK(s->lit.ensure(sizeof(int) * nE * 2), "iterations");
    int *dIt = s->lit.as<int>(), *dSt = dIt + nE;
    if ((r = compute_sigma(s, lead, dE, nE, opts, dS, s->gL.as<double2>(), dSt, dIt, st)) != KNIT_OK)
        return r;
    bool sync = hS;
    if (hS) CK(cudaMemcpyAsync(sigma, dS, sizeof(double2) * MM * nE, cudaMemcpyDeviceToHost, st), "sigma out");
    if (iters) {
        if (is_device_ptr(iters)) {
            CK(cudaMemcpyAsync(iters, dIt, sizeof(int) * nE, cudaMemcpyDeviceToDevice, st), "iters");
        } else {
            CK(cudaMemcpyAsync(iters, dIt, sizeof(int) * nE, cudaMemcpyDeviceToHost, st), "iters");
            sync = true;
        }
    }
    if (residual) {
        const int grid = std::min(nE, s->nsm * 4);
        const Lead &ld = s->lead[lead];
        const bool cell2 = ld.Mp != s->M;   // residual of the supercell's g
        if (cell2 && ld.nsec > 1) {
            CK(s->p2g.ensure(sizeof(double2) * (size_t)ld.Mp * ld.Mp * nE), "supercell g");
            CK(knit_launch_p2_sector_cell(ld.U, ld.sidx, ld.nsec, ld.ms, s->secg.as<double2>(), s->M, nE,
                                          s->p2g.as<double2>(), s->nsm * 8, st),
               "supercell g from blocks");
        }
        CK(s->decw.ensure(sizeof(double2) * 3 * (size_t)ld.Mp * ld.Mp * grid), "residual workspace");
        CK(s->lres.ensure(sizeof(double) * nE), "residual");
        CK(knit_launch_lead_residual(ld.H0, ld.V, ld.Mp, ld.vb, lead, dE, nE,
                                     cell2 ? s->p2g.as<double2>() : s->gL.as<double2>(),
                                     s->decw.as<double2>(), s->lres.as<double>(), grid, st),
           "lead residual");
        bool hr = !is_device_ptr(residual);
        CK(cudaMemcpyAsync(residual, s->lres.p, sizeof(double) * nE,
                           hr ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st),
           "residual out");
        sync = sync || hr;
    }
    return finish(st, sync, "knit_lead_selfenergy");
}

static knit_status transmission_impl(knit_system s, const double *E, int32_t nE,
                                     const uint64_t *seeds, int32_t nS, double W,
                                     const knit_c128 *sigmaL, const knit_c128 *sigmaR,
                                     int32_t precision, const knit_lead_opts *opts, double *T,
                                     int32_t *status, void *stream)
{
    knit_status r = check_system(s);
    if (r != KNIT_OK) return r;
    if ((r = check_batch(s, E, nE, nS, precision, W)) != KNIT_OK) return r;
    if (!T) return fail(KNIT_ERR_INVALID, "T is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t MM = (size_t)s->M * s->M;
    const int n = nE * nS;
    InstDev in{};
    in.n = n;
    in.nS = nS;
    in.W = W;
    if ((r = stage_in(s->E, E, (size_t)nE, st, &in.E, "E")) != KNIT_OK) return r;
    if ((r = stage_in(s->seeds, seeds, (size_t)nS, st, &in.seeds, "seeds")) != KNIT_OK) return r;
    if (sigmaL) {
        const double2 *a = nullptr, *b = nullptr;
        if ((r = stage_in(s->sigL, (const double2 *)sigmaL, MM * nE, st, &a, "sigmaL")) != KNIT_OK ||
            (r = stage_in(s->sigR, (const double2 *)sigmaR, MM * nE, st, &b, "sigmaR")) != KNIT_OK)
            return r;
        in.sigL = a;
        in.sigR = b;
        in.lstatus = nullptr;
    } else {
        const int *lst;
        if ((r = both_sigmas(s, in.E, nE, opts, st, &in.sigL, &in.sigR, &lst)) != KNIT_OK) return r;
        int *l0 = s->lst.as<int>();
        combine_status<<<(nE + 255) / 256, 256, 0, st>>>(l0, l0 + nE, nE);
        CK(cudaGetLastError(), "status combine");
        in.lstatus = l0;
    }
    bool hT, hSt = false;
    if ((r = stage_out(s->T, T, (size_t)n, &in.T, &hT, "T")) != KNIT_OK) return r;
    if ((r = stage_out(s->status, (int *)status, (size_t)n, &in.status, &hSt, "status")) != KNIT_OK)
        return r;
    if ((r = run_sweep(s, in, precision, st)) != KNIT_OK) return r;
    if (hT) CK(cudaMemcpyAsync(T, in.T, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "T out");
    if (hSt)
        CK(cudaMemcpyAsync(status, in.status, sizeof(int) * n, cudaMemcpyDeviceToHost, st), "status out");
    return finish(st, hT || hSt, "knit_transmission");
}

knit_status knit_transmission(knit_system s, const double *E, int32_t nE, const uint64_t *seeds,
                              int32_t nS, double W, int32_t precision,
                              const knit_lead_opts *opts, double *T, int32_t *status, void *stream)
{
    return transmission_impl(s, E, nE, seeds, nS, W, nullptr, nullptr, precision, opts, T, status,
                             stream);
}

knit_status knit_transmission_sigma(knit_system s, const double *E, int32_t nE,
                                    const uint64_t *seeds, int32_t nS, double W,
                                    const knit_c128 *sigmaL, const knit_c128 *sigmaR,
                                    int32_t precision, double *T, int32_t *status, void *stream)
{
    if (!sigmaL || !sigmaR) return fail(KNIT_ERR_INVALID, "sigmaL and sigmaR are required");
    return transmission_impl(s, E, nE, seeds, nS, W, sigmaL, sigmaR, precision, nullptr, T, status,
                             stream);
}

knit_status knit_transmission_eigenvalues(knit_system s, const double *E, int32_t nE,
                                          const uint64_t *seeds, int32_t nS, double W,
                                          int32_t precision, const knit_lead_opts *opts,
                                          double *tau, double *noise, double *T, int32_t *status,
                                          void *stream)
{
    knit_status r = check_system(s);
    if (r != KNIT_OK) return r;
    if ((r = check_batch(s, E, nE, nS, precision, W)) != KNIT_OK) return r;
    if (!tau) return fail(KNIT_ERR_INVALID, "tau is NULL");
    if (s->M > 256) return fail(KNIT_ERR_INVALID, "transmission eigenvalues need M <= 256 (M = %d)", s->M);
    cudaStream_t st = (cudaStream_t)stream;
    const int M = s->M;
    const size_t MM = (size_t)M * M;
    const int n = nE * nS;
    InstDev in{};
    in.n = n;
    in.nS = nS;
    in.W = W;
    if ((r = stage_in(s->E, E, (size_t)nE, st, &in.E, "E")) != KNIT_OK) return r;
    if ((r = stage_in(s->seeds, seeds, (size_t)nS, st, &in.seeds, "seeds")) != KNIT_OK) return r;
    const int *lst;
    if ((r = both_sigmas(s, in.E, nE, opts, st, &in.sigL, &in.sigR, &lst)) != KNIT_OK) return r;
    int *l0 = s->lst.as<int>();
    combine_status<<<(nE + 255) / 256, 256, 0, st>>>(l0, l0 + nE, nE);
    CK(cudaGetLastError(), "status combine");
    in.lstatus = l0;
    // the status array is always needed on the device: it marks the
    // instances whose eigenvalues are undefined
    bool hT = false, hSt = false, hTau = false, hNoise = false;
    if ((r = stage_out(s->T, T, (size_t)n, &in.T, &hT, "T")) != KNIT_OK) return r;
    if (!in.T) {
        CK(s->T.ensure(sizeof(double) * n), "T");
        in.T = s->T.as<double>();
    }
    if ((r = stage_out(s->status, (int *)status, (size_t)n, &in.status, &hSt, "status")) != KNIT_OK)
        return r;
    if (!in.status) {
        CK(s->status.ensure(sizeof(int) * n), "status");
        in.status = s->status.as<int>();
    }
    double *dtau, *dnoise;
    if ((r = stage_out(s->tau, tau, (size_t)n * M, &dtau, &hTau, "tau")) != KNIT_OK) return r;
    if ((r = stage_out(s->noise, noise, (size_t)n, &dnoise, &hNoise, "noise")) != KNIT_OK) return r;
    CK(s->gll.ensure(sizeof(double2) * MM * n), "G_LL workspace");
    in.GLL = s->gll.as<double2>();
    if ((r = run_sweep(s, in, precision, st)) != KNIT_OK) return r;
    // Gamma_R = W W^dagger per energy, then Q = W^dagger K W per instance and its eigenvalues
    CK(s->tg.ensure(sizeof(double2) * MM * nE), "Gamma workspace");
    CK(s->ts.ensure(sizeof(double2) * MM * nE), "Gamma factor");
    CK(s->trk.ensure(sizeof(int) * nE), "Gamma rank");
    CK(knit_launch_gamma_factor(in.sigR, M, nE, s->tg.as<double2>(), s->ts.as<double2>(),
                                s->trk.as<int>(), st),
       "Gamma factor launch");
    const int grid = std::max(1, std::min(n, s->nsm));
    CK(s->tw.ensure(std::max<size_t>(knit_tau_work_bytes(M) * grid, 256)), "eigenvalue scratch");
    CK(knit_launch_tau(in.GLL, s->ts.as<double2>(), s->trk.as<int>(), M, n, nS, in.status, s->tw.p,
                       grid, dtau, dnoise, st),
       "eigenvalue launch");
    if (hTau) CK(cudaMemcpyAsync(tau, dtau, sizeof(double) * n * M, cudaMemcpyDeviceToHost, st), "tau out");
    if (hNoise)
        CK(cudaMemcpyAsync(noise, dnoise, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "noise out");
    if (hT) CK(cudaMemcpyAsync(T, in.T, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "T out");
    if (hSt)
        CK(cudaMemcpyAsync(status, in.status, sizeof(int) * n, cudaMemcpyDeviceToHost, st), "status out");
    return finish(st, hTau || hNoise || hT || hSt, "knit_transmission_eigenvalues");
}

knit_status knit_graph_destroy(knit_graph g)
{
    if (!g) return KNIT_OK;
    cudaSetDevice(g->device);
    cudaFree(g->blocks);
    cudaFree(g->width);
    cudaFree(g->lw);
    cudaFree(g->lpos);
    cudaFree(g->loff);
    cudaFree(g->hoff);
    cudaFree(g->voff);
    DevBuf *bufs[] = {&g->work, &g->E, &g->Tm, &g->T, &g->status, &g->sigp, &g->sigs};
    for (DevBuf *b : bufs) b->release();
    delete g;
    return KNIT_OK;
}

namespace {

// widest slice the graph sweep takes: its Gauss-Jordan scratch (two rows of
// complex128 plus indices) must fit in one CTA's shared memory
constexpr int KNIT_GRAPH_MAX_WIDTH = 6144;

// the slicing of a geometry (host only): slices sl (site lists), every
// site's slice (-1: not connected to lead 0) and position within it
struct GraphPlan {
    std::vector<std::vector<int>> sl, ls;
    std::vector<int> slice_of, pos;
    std::vector<double2> H;
};

knit_status graph_plan(int N, const knit_c128 *Hin, int P, const int32_t *nsites,
                       const int32_t *const *sites, GraphPlan &gp)
{
    if (N <= 0 || N > 8192) return fail(KNIT_ERR_INVALID, "N = %d out of range (1 .. 8192)", N);
    if (P < 2 || P > 64) return fail(KNIT_ERR_INVALID, "%d leads: 2 .. 64 supported", P);
    if (!Hin || !nsites || !sites) return fail(KNIT_ERR_INVALID, "H and the lead site lists are required");
    std::vector<double2> H;
    knit_status r;
    if ((r = to_host(H, Hin, (size_t)N * N, "H")) != KNIT_OK) return r;
    std::vector<std::vector<int>> ls(P);
    std::vector<int> which(N, -1);
    for (int p = 0; p < P; ++p) {
        if (nsites[p] <= 0 || !sites[p]) return fail(KNIT_ERR_INVALID, "lead %d has no sites", p);
        if ((r = to_host(ls[p], sites[p], (size_t)nsites[p], "lead sites")) != KNIT_OK) return r;
        for (int v : ls[p]) {
            if (v < 0 || v >= N) return fail(KNIT_ERR_INVALID, "lead site %d out of range", v);
            if (which[v] != -1) return fail(KNIT_ERR_INVALID, "site %d listed twice among the leads", v);
            which[v] = p;
        }
    }
    double hmax = 0.0;
    for (double2 h : H) hmax = std::max(hmax, std::hypot(h.x, h.y));
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < i; ++j) {
            const double2 a = H[(size_t)i * N + j], b = H[(size_t)j * N + i];
            if (std::fabs(a.x - b.x) > 1e-12 * hmax || std::fabs(a.y + b.y) > 1e-12 * hmax)
                return fail(KNIT_ERR_INVALID, "H is not Hermitian at (%d, %d)", i, j);
        }
    // breadth-first layers from lead 0's sites
    std::vector<int> depth(N, -1), queue(ls[0]);
    for (int v : ls[0]) depth[v] = 0;
    for (size_t q = 0; q < queue.size(); ++q) {
        const int u = queue[q];
        for (int v = 0; v < N; ++v) {
            const double2 h = H[(size_t)u * N + v];
            if (v != u && depth[v] < 0 && (h.x != 0.0 || h.y != 0.0)) {
                depth[v] = depth[u] + 1;
                queue.push_back(v);
            }
        }
    }
    int d1 = 1 << 30;
    for (int p = 1; p < P; ++p)
        for (int v : ls[p]) {
            if (depth[v] < 0)
                return fail(KNIT_ERR_INVALID, "site %d of lead %d is not connected to lead 0", v, p);
            d1 = std::min(d1, depth[v]);
        }
    // Slices are the level sets of an integer function l with l = 0 exactly
    // on lead 0's sites, l = K - 1 = d1 on every other lead's sites, and
    // |l(u) - l(v)| <= 1 along every edge (so H is block tridiagonal).  The
    // family l_s(v) = max(1, min(depth(v), d1, d1 - dist(v) + s)), dist the
    // distance to the other leads' sites, has these properties for every
    // s >= 0: s = 0 folds the sites behind a lead back into earlier slices,
    // s = max dist gives the breadth-first layers with everything from depth
    // d1 on merged into the last slice.  The plan takes the s with the least
    // sweep work (sum of w_k^3 + w_k^2 w_{k-1}), the layers on ties.
    std::vector<int> dist(N, -1), q2;
    for (int p = 1; p < P; ++p)
        for (int v : ls[p]) {
            dist[v] = 0;
            q2.push_back(v);
        }
    for (size_t q = 0; q < q2.size(); ++q) {
        const int u = q2[q];
        for (int v = 0; v < N; ++v) {
            const double2 h = H[(size_t)u * N + v];
            if (v != u && dist[v] < 0 && (h.x != 0.0 || h.y != 0.0)) {
                dist[v] = dist[u] + 1;
                q2.push_back(v);
            }
        }
    }
    int smax = 0;
    for (int v = 0; v < N; ++v)
        if (depth[v] >= 0) smax = std::max(smax, dist[v]);
    auto level = [&](int v, int s) {
        return depth[v] == 0 ? 0 : std::max(1, std::min(std::min(depth[v], d1), d1 - dist[v] + s));
    };
    const int K = d1 + 1;
    int best_s = smax;
    double best = -1.0;
    std::vector<double> w(K);
    for (int sv = smax; sv >= 0; --sv) {
        std::fill(w.begin(), w.end(), 0.0);
        for (int v = 0; v < N; ++v)
            if (depth[v] >= 0) w[level(v, sv)] += 1.0;
        double cost = 0.0;
        for (int k = 0; k < K; ++k) cost += w[k] * w[k] * (w[k] + (k > 0 ? w[k - 1] : 0.0));
        if (best < 0.0 || cost < best) {
            best = cost;
            best_s = sv;
        }
    }
    std::vector<std::vector<int>> sl(K);
    sl[0] = ls[0];
    for (int v = 0; v < N; ++v)
        if (depth[v] > 0) sl[level(v, best_s)].push_back(v);
    for (const auto &v : sl)
        if ((int)v.size() > KNIT_GRAPH_MAX_WIDTH)
            return fail(KNIT_ERR_INVALID, "a slice of %d sites: at most %d supported", (int)v.size(),
                        KNIT_GRAPH_MAX_WIDTH);
    gp.slice_of.assign(N, -1);
    gp.pos.assign(N, -1);
    for (int k = 0; k < K; ++k)
        for (size_t a = 0; a < sl[k].size(); ++a) {
            gp.slice_of[sl[k][a]] = k;
            gp.pos[sl[k][a]] = (int)a;
        }
    gp.sl = std::move(sl);
    gp.ls = std::move(ls);
    gp.H = std::move(H);
    return KNIT_OK;
}

knit_status graph_build(int N, const knit_c128 *Hin, int P, const int32_t *nsites,
                        const int32_t *const *sites, knit_graph *out)
{
    *out = nullptr;
    GraphPlan gp;
    knit_status r = graph_plan(N, Hin, P, nsites, sites, gp);
    if (r != KNIT_OK) return r;
    const std::vector<std::vector<int>> &sl = gp.sl, &ls = gp.ls;
    const std::vector<double2> &H = gp.H;
    const int K = (int)sl.size();
    auto g = new knit_graph_s;
    g->N = N;
    g->K = K;
    g->P = P;
    g->hslice_of = gp.slice_of;
    const std::vector<int> &pos = gp.pos;
    for (int k = 0; k < K; ++k) {
        g->hwidth.push_back((int)sl[k].size());
        g->Mmax = std::max(g->Mmax, (int)sl[k].size());
    }
    std::vector<int> lpos, loff;
    for (int p = 0; p < P; ++p) {
        g->hlw.push_back((int)ls[p].size());
        loff.push_back((int)lpos.size());
        for (int v : ls[p]) lpos.push_back(pos[v]);
    }
    // blocks: H_k, then V_k = H_{k,k-1}
    std::vector<double2> blk;
    std::vector<long long> hoff(K), voff(K, 0);
    for (int k = 0; k < K; ++k) {
        hoff[k] = (long long)blk.size();
        for (int a : sl[k])
            for (int b : sl[k]) blk.push_back(H[(size_t)a * N + b]);
        if (k > 0) {
            voff[k] = (long long)blk.size();
            for (int a : sl[k])
                for (int b : sl[k - 1]) blk.push_back(H[(size_t)a * N + b]);
        }
    }
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, g->device);
    if ((r = to_device(&g->blocks, blk.data(), blk.size(), "graph blocks")) != KNIT_OK ||
        (r = to_device(&g->width, g->hwidth.data(), (size_t)K, "slice widths")) != KNIT_OK ||
        (r = to_device(&g->lw, g->hlw.data(), (size_t)P, "lead widths")) != KNIT_OK ||
        (r = to_device(&g->lpos, lpos.data(), lpos.size(), "lead positions")) != KNIT_OK ||
        (r = to_device(&g->loff, loff.data(), loff.size(), "lead offsets")) != KNIT_OK ||
        (r = to_device(&g->hoff, hoff.data(), (size_t)K, "block offsets")) != KNIT_OK ||
        (r = to_device(&g->voff, voff.data(), (size_t)K, "block offsets")) != KNIT_OK) {
        knit_graph_destroy(g);
        return r;
    }
    *out = g;
    return KNIT_OK;
}

// the sweep for nE energies: Tm (device, nE x P x P) and status (device)
knit_status graph_run(knit_graph g, const double *E, int nE, const knit_c128 *const *sigma,
                      double *Tm, int *status, cudaStream_t st)
{
    knit_status r;
    const double *dE;
    if ((r = stage_in(g->E, E, (size_t)nE, st, &dE, "E")) != KNIT_OK) return r;
    // self-energies: device copies of host arrays in one buffer, then the pointer table
    std::vector<const double2 *> ptr(g->P);
    size_t host_elems = 0;
    for (int p = 0; p < g->P; ++p) {
        if (!sigma[p]) return fail(KNIT_ERR_INVALID, "self-energy of lead %d is NULL", p);
        if (!is_device_ptr(sigma[p])) host_elems += (size_t)nE * g->hlw[p] * g->hlw[p];
    }
    CK(g->sigs.ensure(sizeof(double2) * std::max<size_t>(host_elems, 1)), "self-energy staging");
    size_t off = 0;
    for (int p = 0; p < g->P; ++p) {
        const size_t n = (size_t)nE * g->hlw[p] * g->hlw[p];
        if (is_device_ptr(sigma[p])) {
            ptr[p] = (const double2 *)sigma[p];
        } else {
            ptr[p] = g->sigs.as<double2>() + off;
            CK(cudaMemcpyAsync((void *)ptr[p], sigma[p], sizeof(double2) * n, cudaMemcpyHostToDevice, st),
               "self-energy in");
            off += n;
        }
    }
    CK(g->sigp.ensure(sizeof(double2 *) * g->P), "self-energy table");
    CK(cudaMemcpyAsync(g->sigp.p, ptr.data(), sizeof(double2 *) * g->P, cudaMemcpyHostToDevice, st),
       "self-energy table");
    // one CTA per energy up to one per SM, fewer when the per-CTA workspace
    // (six Mmax x Mmax complex matrices) would pass 8 GiB in total
    const size_t per_cta = sizeof(double2) * 6 * (size_t)g->Mmax * g->Mmax;
    const int fit = (int)std::max<size_t>(1, (size_t(8) << 30) / per_cta);
    const int grid = std::max(1, std::min(std::min(nE, g->nsm), fit));
    CK(g->work.ensure(per_cta * grid), "graph workspace");
    GraphDev gd{g->K, g->Mmax, g->P, g->width, g->hoff, g->voff, g->blocks, g->lw, g->lpos, g->loff,
                g->sigp.as<const double2 *>()};
    CK(knit_launch_graph_fp64(&gd, dE, nE, g->work.as<double2>(), grid, Tm, status, st),
       "graph sweep launch");
    // the pointer table and host staging must outlive the launch
    CK(cudaStreamSynchronize(st), "graph sweep");
    return KNIT_OK;
}

}  // namespace

knit_status knit_graph_plan(const knit_graph_multi_desc *d, int32_t *nslices, int32_t *slice_of)
{
    if (!d || !nslices) return fail(KNIT_ERR_INVALID, "knit_graph_plan: NULL argument");
    GraphPlan gp;
    knit_status r = graph_plan(d->N, d->H, d->n_leads, d->n_lead_sites, d->lead_sites, gp);
    if (r != KNIT_OK) return r;
    *nslices = (int32_t)gp.sl.size();
    if (slice_of) std::copy(gp.slice_of.begin(), gp.slice_of.end(), slice_of);
    return KNIT_OK;
}

knit_status knit_graph_create(const knit_graph_desc *d, knit_graph *out)
{
    if (!d || !out) return fail(KNIT_ERR_INVALID, "knit_graph_create: NULL argument");
    return graph_build(d->N, d->H, 2, d->n_lead_sites, d->lead_sites, out);
}

knit_status knit_graph_create_multi(const knit_graph_multi_desc *d, knit_graph *out)
{
    if (!d || !out) return fail(KNIT_ERR_INVALID, "knit_graph_create_multi: NULL argument");
    return graph_build(d->N, d->H, d->n_leads, d->n_lead_sites, d->lead_sites, out);
}

knit_status knit_graph_slices(knit_graph g, int32_t *nslices, int32_t *widths, int32_t *slice_of)
{
    if (!g || !nslices) return fail(KNIT_ERR_INVALID, "knit_graph_slices: NULL argument");
    *nslices = g->K;
    if (widths) std::copy(g->hwidth.begin(), g->hwidth.end(), widths);
    if (slice_of) std::copy(g->hslice_of.begin(), g->hslice_of.end(), slice_of);
    return KNIT_OK;
}

knit_status knit_graph_conductance(knit_graph g, const double *E, int32_t nE,
                                   const knit_c128 *const *sigma, double *Tmat, int32_t *status,
                                   void *stream)
{
    if (!g) return fail(KNIT_ERR_INVALID, "graph is NULL");
    if (!E || !sigma || !Tmat) return fail(KNIT_ERR_INVALID, "E, sigma and Tmat are required");
    if (nE <= 0) return fail(KNIT_ERR_INVALID, "nE must be positive");
    cudaSetDevice(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    knit_status r;
    bool hT, hSt = false;
    double *dT;
    int *dSt;
    const size_t nT = (size_t)nE * g->P * g->P;
    if ((r = stage_out(g->Tm, Tmat, nT, &dT, &hT, "Tmat")) != KNIT_OK ||
        (r = stage_out(g->status, (int *)status, (size_t)nE, &dSt, &hSt, "status")) != KNIT_OK)
        return r;
    if ((r = graph_run(g, E, nE, sigma, dT, dSt, st)) != KNIT_OK) return r;
    if (hT) CK(cudaMemcpyAsync(Tmat, dT, sizeof(double) * nT, cudaMemcpyDeviceToHost, st), "Tmat out");
    if (hSt) CK(cudaMemcpyAsync(status, dSt, sizeof(int) * nE, cudaMemcpyDeviceToHost, st), "status out");
    return finish(st, hT || hSt, "knit_graph_conductance");
}

knit_status knit_graph_transmission(knit_graph g, const double *E, int32_t nE,
                                    const knit_c128 *sigma0, const knit_c128 *sigma1, double *T,
                                    int32_t *status, void *stream)
{
    if (!g) return fail(KNIT_ERR_INVALID, "graph is NULL");
    if (g->P != 2) return fail(KNIT_ERR_INVALID, "knit_graph_transmission needs a two-lead graph");
    if (!E || !sigma0 || !sigma1 || !T) return fail(KNIT_ERR_INVALID, "E, sigma0, sigma1 and T are required");
    if (nE <= 0) return fail(KNIT_ERR_INVALID, "nE must be positive");
    cudaSetDevice(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    knit_status r;
    bool hT, hSt = false;
    double *dT;
    int *dSt;
    if ((r = stage_out(g->T, T, (size_t)nE, &dT, &hT, "T")) != KNIT_OK ||
        (r = stage_out(g->status, (int *)status, (size_t)nE, &dSt, &hSt, "status")) != KNIT_OK)
        return r;
    CK(g->Tm.ensure(sizeof(double) * 4 * (size_t)nE), "transmission matrix");
    const knit_c128 *sig[2] = {sigma0, sigma1};
    if ((r = graph_run(g, E, nE, sig, g->Tm.as<double>(), dSt, st)) != KNIT_OK) return r;
    CK(knit_launch_graph_pick(g->Tm.as<double>(), nE, 2, 0, 1, dT, st), "transmission pick");
    if (hT) CK(cudaMemcpyAsync(T, dT, sizeof(double) * nE, cudaMemcpyDeviceToHost, st), "T out");
    if (hSt) CK(cudaMemcpyAsync(status, dSt, sizeof(int) * nE, cudaMemcpyDeviceToHost, st), "status out");
    return finish(st, hT || hSt, "knit_graph_transmission");
}

knit_status knit_system_info(knit_system s, int32_t precision, int32_t *sweep, int32_t *lead_blocks)
{
    knit_status r = check_system(s);
    if (r != KNIT_OK) return r;
    if (!sweep || !lead_blocks) return fail(KNIT_ERR_INVALID, "sweep and lead_blocks are required");
    if (precision != KNIT_FP64 && precision != KNIT_MIXED && precision != KNIT_MIXED_CUDACORE)
        return fail(KNIT_ERR_INVALID, "unknown precision %d", precision);
    static_assert((int)SWEEP_FP64 == (int)KNIT_SWEEP_FP64 && (int)SWEEP_MIXED == (int)KNIT_SWEEP_MIXED_NARROW &&
                      (int)SWEEP_WIDE == (int)KNIT_SWEEP_MIXED_CUDACORE &&
                      (int)SWEEP_TC128 == (int)KNIT_SWEEP_MIXED_TC128 &&
                      (int)SWEEP_HALF == (int)KNIT_SWEEP_MIXED_HALF_ROWS,
                  "sweep kinds");
    *sweep = sweep_kind(s, precision, true);
    for (int p = 0; p < 2; ++p) lead_blocks[p] = s->lead[p].nsec * s->lead[p].nsub;
    return KNIT_OK;
}

knit_status knit_system_num_edges(knit_system s, int32_t *count)
{
    knit_status r = check_system(s);
    if (r != KNIT_OK) return r;
    if (!count) return fail(KNIT_ERR_INVALID, "count is NULL");
    *count = s->n_edges;
    return KNIT_OK;
}

knit_status knit_lesser(knit_system s, const double *E, int32_t nE, const uint64_t *seeds,
                        int32_t nS, double W, int32_t saving_level, const knit_lead_opts *opts,
                        double *rhoL, double *rhoR, double *jx, double *jt, double *T,
                        int32_t *status, void *stream)
{
    knit_status r = check_system(s);
    if (r != KNIT_OK) return r;
    if ((r = check_batch(s, E, nE, nS, KNIT_FP64, W)) != KNIT_OK) return r;
    if (!rhoL && !rhoR && !jx && !jt) return fail(KNIT_ERR_INVALID, "no output requested");
    if (saving_level == 0)
        return fail(KNIT_ERR_INVALID, "saving_level 0 keeps nothing: no local observables");
    if (saving_level < -1) return fail(KNIT_ERR_INVALID, "saving_level must be -1 or >= 1");
    const int save = saving_level == -1 ? 1 : std::min(saving_level, s->L);
    cudaStream_t st = (cudaStream_t)stream;
    const int M = s->M, L = s->L;
    const size_t MM = (size_t)M * M;
    const int n = nE * nS;
    InstDev in{};
    in.n = n;
    in.nS = nS;
    in.W = W;
    if ((r = stage_in(s->E, E, (size_t)nE, st, &in.E, "E")) != KNIT_OK) return r;
    if ((r = stage_in(s->seeds, seeds, (size_t)nS, st, &in.seeds, "seeds")) != KNIT_OK) return r;
    const int *lst;
    if ((r = both_sigmas(s, in.E, nE, opts, st, &in.sigL, &in.sigR, &lst)) != KNIT_OK) return r;
    int *l0 = s->lst.as<int>();
    combine_status<<<(nE + 255) / 256, 256, 0, st>>>(l0, l0 + nE, nE);
    CK(cudaGetLastError(), "status combine");
    in.lstatus = l0;
    bool hl = false, hr = false, hx = false, ht = false, hT = false, hSt = false;
    double *dl, *dr, *dx, *dt;
    const size_t nlm = (size_t)n * L * M, nx = (size_t)n * (L - 1) * M, ne = (size_t)n * L * s->n_edges;
    if ((r = stage_out(s->lrl, rhoL, nlm, &dl, &hl, "rhoL")) != KNIT_OK ||
        (r = stage_out(s->lrr, rhoR, nlm, &dr, &hr, "rhoR")) != KNIT_OK ||
        (r = stage_out(s->ljx, jx, std::max<size_t>(nx, 1), &dx, &hx, "jx")) != KNIT_OK ||
        (r = stage_out(s->ljt, jt, std::max<size_t>(ne, 1), &dt, &ht, "jt")) != KNIT_OK ||
        (r = stage_out(s->T, T, (size_t)n, &in.T, &hT, "T")) != KNIT_OK ||
        (r = stage_out(s->status, (int *)status, (size_t)n, &in.status, &hSt, "status")) != KNIT_OK)
        return r;
    in.sys = s->d_sys;
    CK(s->queue.ensure(sizeof(int)), "queue");
    in.queue = s->queue.as<int>();
    CK(cudaMemsetAsync(in.queue, 0, sizeof(int), st), "queue reset");
    const int grid = std::max(1, std::min(n, s->nsm));
    CK(s->work.ensure(sizeof(double2) * 8 * MM * grid), "lesser workspace");
    const int nck = (L + save - 1) / save;
    CK(s->ckpt.ensure(sizeof(double2) * MM * (size_t)(nck + save) * grid), "checkpoint workspace");
    CK(knit_launch_lesser_fp64(&in, M, L, grid, s->work.as<double2>(), s->ckpt.as<double2>(), save,
                               s->h0_edges, s->n_edges, dl, dr, dx, s->n_edges ? dt : nullptr, st),
       "lesser launch");
    if (hl) CK(cudaMemcpyAsync(rhoL, dl, sizeof(double) * nlm, cudaMemcpyDeviceToHost, st), "rhoL out");
    if (hr) CK(cudaMemcpyAsync(rhoR, dr, sizeof(double) * nlm, cudaMemcpyDeviceToHost, st), "rhoR out");
    if (hx && nx) CK(cudaMemcpyAsync(jx, dx, sizeof(double) * nx, cudaMemcpyDeviceToHost, st), "jx out");
    if (ht && ne) CK(cudaMemcpyAsync(jt, dt, sizeof(double) * ne, cudaMemcpyDeviceToHost, st), "jt out");
    if (hT) CK(cudaMemcpyAsync(T, in.T, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "T out");
    if (hSt)
        CK(cudaMemcpyAsync(status, in.status, sizeof(int) * n, cudaMemcpyDeviceToHost, st), "status out");
    return finish(st, hl || hr || hx || ht || hT || hSt, "knit_lesser");
}

knit_status knit_ldos(knit_system s, const double *E, int32_t nE, const uint64_t *seeds,
                      int32_t nS, double W, int32_t precision, int32_t saving_level,
                      const knit_lead_opts *opts, double *ldos, double *T, int32_t *status,
                      void *stream)
{
    knit_status r = check_system(s);
    if (r != KNIT_OK) return r;
    if ((r = check_batch(s, E, nE, nS, precision, W)) != KNIT_OK) return r;
    if (!ldos) return fail(KNIT_ERR_INVALID, "ldos is NULL");
    if (saving_level == 0)
        return fail(KNIT_ERR_INVALID, "saving_level 0 keeps nothing: no local observables");
    if (saving_level < -1) return fail(KNIT_ERR_INVALID, "saving_level must be -1 or >= 1");
    const int save = saving_level == -1 ? 1 : std::min(saving_level, s->L);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t MM = (size_t)s->M * s->M;
    const int n = nE * nS;
    InstDev in{};
    in.n = n;
    in.nS = nS;
    in.W = W;
    if ((r = stage_in(s->E, E, (size_t)nE, st, &in.E, "E")) != KNIT_OK) return r;
    if ((r = stage_in(s->seeds, seeds, (size_t)nS, st, &in.seeds, "seeds")) != KNIT_OK) return r;
    const int *lst;
    if ((r = both_sigmas(s, in.E, nE, opts, st, &in.sigL, &in.sigR, &lst)) != KNIT_OK) return r;
    int *l0 = s->lst.as<int>();
    combine_status<<<(nE + 255) / 256, 256, 0, st>>>(l0, l0 + nE, nE);
    in.lstatus = l0;
    bool hL, hT = false, hSt = false;
    double *dL;
    if ((r = stage_out(s->ldos, ldos, (size_t)n * s->L * s->M, &dL, &hL, "ldos")) != KNIT_OK) return r;
    if ((r = stage_out(s->T, T, (size_t)n, &in.T, &hT, "T")) != KNIT_OK) return r;
    if ((r = stage_out(s->status, (int *)status, (size_t)n, &in.status, &hSt, "status")) != KNIT_OK)
        return r;
    in.sys = s->d_sys;
    CK(s->queue.ensure(sizeof(int)), "queue");
    in.queue = s->queue.as<int>();
    CK(cudaMemsetAsync(in.queue, 0, sizeof(int), st), "queue reset");
    const int grid = std::max(1, std::min(n, s->nsm));
    if (sweep_kind(s, precision) == SWEEP_MIXED) {
        CK(s->ckpt.ensure(knit_ldos_mixed_work_bytes(s->M, s->L, save) * grid),
           "checkpoint workspace");
        CK(knit_launch_ldos_mixed(&in, s->M, s->L, grid, save, s->ckpt.p, dL,
                                  (long long)s->L * s->M, st),
           "mixed ldos launch");
    } else {
        int use_smem = knit_fp64_smem_bytes(s->M, 1, 4) <= 220 * 1024;
        if (!use_smem) CK(s->work.ensure(sizeof(double2) * 4 * MM * grid), "ldos workspace");
        const int nck = (s->L + save - 1) / save;
        CK(s->ckpt.ensure(sizeof(double2) * MM * (size_t)(nck + save) * grid),
           "checkpoint workspace");
        CK(knit_launch_ldos_fp64(&in, s->M, s->L, grid, s->work.as<double2>(), use_smem,
                                 s->ckpt.as<double2>(), save, dL, (long long)s->L * s->M, st),
           "ldos launch");
    }
    if (hL) CK(cudaMemcpyAsync(ldos, dL, sizeof(double) * n * s->L * s->M, cudaMemcpyDeviceToHost, st), "ldos out");
    if (hT) CK(cudaMemcpyAsync(T, in.T, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "T out");
    if (hSt)
        CK(cudaMemcpyAsync(status, in.status, sizeof(int) * n, cudaMemcpyDeviceToHost, st), "status out");
    return finish(st, hL || hT || hSt, "knit_ldos");
}


knit_status knit_batch_create(const knit_system *systems, int32_t nSys, const int32_t *sys_index,
                              int32_t nInst, int32_t precision, knit_batch *out)
{
    if (!systems || !sys_index || !out || nSys <= 0 || nInst <= 0)
        return fail(KNIT_ERR_INVALID, "knit_batch_create: bad arguments");
    if (precision != KNIT_FP64 && precision != KNIT_MIXED && precision != KNIT_MIXED_CUDACORE)
        return fail(KNIT_ERR_INVALID, "unknown precision %d", precision);
    *out = nullptr;
    std::vector<int> idx;
    knit_status r = to_host(idx, sys_index, (size_t)nInst, "sys_index");
    if (r != KNIT_OK) return r;
    for (int i = 0; i < nSys; ++i)
        if (!systems[i]) return fail(KNIT_ERR_INVALID, "systems[%d] is NULL", i);
    for (int v : idx)
        if (v < 0 || v >= nSys) return fail(KNIT_ERR_INVALID, "sys_index out of range");
    knit_batch b = new (std::nothrow) knit_batch_s;
    if (!b) return fail(KNIT_ERR_OOM, "host allocation");
    b->nInst = nInst;
    b->precision = precision;
    b->sys.assign(systems, systems + nSys);
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    // plan order: instances grouped by system
    b->start.assign(nSys, 0);
    b->count.assign(nSys, 0);
    for (int v : idx) b->count[v]++;
    for (int k = 1; k < nSys; ++k) b->start[k] = b->start[k - 1] + b->count[k - 1];
    b->perm.assign(nInst, 0);
    std::vector<int> fill(b->start), sys_of(nInst);
    for (int i = 0; i < nInst; ++i) {
        const int p = fill[idx[i]]++;
        b->perm[p] = i;
        sys_of[p] = idx[i];
    }
    b->sig_off.assign(nInst, 0);
    long long off = 0;
    for (int k = 0; k < nSys; ++k) {
        const long long MM = (long long)b->sys[k]->M * b->sys[k]->M;
        for (int j = 0; j < b->count[k]; ++j) b->sig_off[b->start[k] + j] = off + j * MM;
        off += MM * b->count[k];
        b->g_max = std::max(b->g_max, MM * b->count[k]);
    }
    b->sig_total = off;
    // buckets by kernel variant
    auto kind_of = [&](knit_system s, int *use_tc, int *cls) {
        const int k = sweep_kind(s, precision);
        *use_tc = 0;
        if (k == SWEEP_FP64) { *cls = 0; return 0; }
        if (k == SWEEP_WIDE) { *cls = 5; return 2; }
        if (k == SWEEP_TC128) { *cls = 6; return 3; }
        *use_tc = precision == KNIT_MIXED && s->M > 32;
        *cls = s->M <= 16 ? 1 : s->M <= 32 ? 2 : (*use_tc ? 3 : 4);
        return 1;
    };
    std::vector<int> cls_bucket(7, -1);
    for (int p = 0; p < nInst; ++p) {
        knit_system s = b->sys[sys_of[p]];
        int use_tc, cls;
        int kind = kind_of(s, &use_tc, &cls);
        if (cls_bucket[cls] < 0) {
            cls_bucket[cls] = (int)b->buckets.size();
            b->buckets.emplace_back();
            b->buckets.back().kind = kind;
            b->buckets.back().use_tc = use_tc;
        }
        auto &bk = b->buckets[cls_bucket[cls]];
        bk.order.push_back(p);
        bk.Mmax = std::max(bk.Mmax, s->M);
        bk.Lmax = std::max(bk.Lmax, s->L);
    }
    auto cost = [&](int p) {
        knit_system sp = b->sys[sys_of[p]];
        return (double)sp->M * sp->M * sp->M * sp->L;
    };
    for (auto &bk : b->buckets) {
        std::stable_sort(bk.order.begin(), bk.order.end(), [&](int a, int c) { return cost(a) > cost(c); });
        bk.cost0 = cost(bk.order[0]);
        if (bk.kind == 1 && !bk.use_tc) bk.max_ctas = knit_mixed_ctas_per_sm(bk.Mmax, 0);
    }
    // all variants run at once on their own streams, launched heaviest first:
    // the SMs a variant's tail leaves idle take the next variant's CTAs
    std::stable_sort(b->buckets.begin(), b->buckets.end(),
                     [](const knit_batch_s::Bucket &x, const knit_batch_s::Bucket &y) { return x.cost0 > y.cost0; });
    // device tables
    std::vector<SysDev> tab(nSys);
    for (int k = 0; k < nSys; ++k) tab[k] = b->sys[k]->dev();
    cudaError_t e;
    if ((e = b->d_systab.ensure(sizeof(SysDev) * nSys)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_systab.p, tab.data(), sizeof(SysDev) * nSys, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = b->d_sys_of.ensure(sizeof(int) * nInst)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_sys_of.p, sys_of.data(), sizeof(int) * nInst, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = b->d_perm.ensure(sizeof(int) * nInst)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_perm.p, b->perm.data(), sizeof(int) * nInst, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = b->d_sig_off.ensure(sizeof(long long) * nInst)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_sig_off.p, b->sig_off.data(), sizeof(long long) * nInst, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = b->Ep.ensure(sizeof(double) * nInst)) != cudaSuccess ||
        (e = b->Sp.ensure(sizeof(uint64_t) * nInst)) != cudaSuccess ||
        (e = b->Wp.ensure(sizeof(double) * nInst)) != cudaSuccess ||
        (e = b->sigL.ensure(sizeof(double2) * b->sig_total)) != cudaSuccess ||
        (e = b->sigR.ensure(sizeof(double2) * b->sig_total)) != cudaSuccess ||
        (e = b->gbuf.ensure(sizeof(double2) * b->g_max)) != cudaSuccess ||
        (e = b->lst.ensure(sizeof(int) * 2 * nInst)) != cudaSuccess ||
        (e = b->queue.ensure(sizeof(int) * b->buckets.size())) != cudaSuccess) {
        batch_release(b);
        delete b;
        return cuda_fail(e, "knit_batch_create");
    }
    size_t work = 0;
    if ((e = cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming)) != cudaSuccess) {
        batch_release(b);
        delete b;
        return cuda_fail(e, "knit_batch_create");
    }
    for (auto &bk : b->buckets) {
        if ((e = bk.d_order.ensure(sizeof(int) * bk.order.size())) != cudaSuccess ||
            (e = cudaMemcpy(bk.d_order.p, bk.order.data(), sizeof(int) * bk.order.size(),
                            cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&bk.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&bk.done, cudaEventDisableTiming)) != cudaSuccess) {
            batch_release(b);
            delete b;
            return cuda_fail(e, "knit_batch_create");
        }
        // each variant its own workspace, since they run concurrently
        work = (work + 255) & ~(size_t)255;
        bk.work_off = work;
        if (bk.kind == 0 && knit_fp64_smem_bytes(bk.Mmax, 1, 3) > 220 * 1024)
            work += sizeof(double2) * 3 * (size_t)bk.Mmax * bk.Mmax * b->nsm;
        if (bk.kind == 2) work += knit_mixed_wide_work_bytes(bk.Mmax) * b->nsm;
        if (bk.kind == 3) work += knit_mixed_tc128_work_bytes() * b->nsm;
    }
    if (work && (e = b->work.ensure(work)) != cudaSuccess) {
        batch_release(b);
        delete b;
        return cuda_fail(e, "knit_batch_create");
    }
    // lead eigen-decompositions now, so that runs only enqueue kernels
    for (int k = 0; k < nSys; ++k)
        for (int p = 0; p < 2; ++p)
            if (b->sys[k]->lead[p].scalar && (r = ensure_modes(b->sys[k], p)) != KNIT_OK) {
                batch_release(b);
                delete b;
                return r;
            }
    *out = b;
    return KNIT_OK;
}

knit_status knit_batch_destroy(knit_batch b)
{
    if (!b) return KNIT_OK;
    cudaSetDevice(b->device);
    batch_release(b);
    delete b;
    return KNIT_OK;
}

}  // extern "C"

namespace {

// instance parameters gathered into plan order, both leads' self-energies per
// system, lead status combined (all on st)
knit_status batch_prepare(knit_batch b, const double *E, const uint64_t *seeds, const double *W,
                          const knit_lead_opts *opts, cudaStream_t st)
{
    const int n = b->nInst;
    knit_status r;
    const double *dE, *dW;
    const uint64_t *dS;
    if ((r = stage_in(b->E, E, (size_t)n, st, &dE, "E")) != KNIT_OK ||
        (r = stage_in(b->seeds, seeds, (size_t)n, st, &dS, "seeds")) != KNIT_OK ||
        (r = stage_in(b->W, W, (size_t)n, st, &dW, "W")) != KNIT_OK)
        return r;
    double *Ep = b->Ep.as<double>(), *Wp = b->Wp.as<double>();
    uint64_t *Sp = b->Sp.as<uint64_t>();
    gather_instances<<<(n + 255) / 256, 256, 0, st>>>(dE, dS, dW, b->d_perm.as<int>(), n, Ep, Sp, Wp);
    CK(cudaGetLastError(), "gather");
    int *lst = b->lst.as<int>();
    for (size_t k = 0; k < b->sys.size(); ++k) {
        if (!b->count[k]) continue;
        knit_system s = b->sys[k];
        const int p0 = b->start[k];
        const long long off = b->sig_off[p0];
        if ((r = compute_sigma(s, 0, Ep + p0, b->count[k], opts, b->sigL.as<double2>() + off,
                               b->gbuf.as<double2>(), lst + p0, nullptr, st)) != KNIT_OK ||
            (r = compute_sigma(s, 1, Ep + p0, b->count[k], opts, b->sigR.as<double2>() + off,
                               b->gbuf.as<double2>(), lst + n + p0, nullptr, st)) != KNIT_OK)
            return r;
    }
    combine_status<<<(n + 255) / 256, 256, 0, st>>>(lst, lst + n, n);
    CK(cudaGetLastError(), "status combine");
    return KNIT_OK;
}

// the persistent sweep launch of variant q on stream st (its queue counter
// already zeroed), with `ctas` CTAs per SM
knit_status batch_launch(knit_batch b, size_t q, int ctas, double *dT, int *dSt, cudaStream_t st)
{
    auto &bk = b->buckets[q];
    InstDev in{};
    in.n = (int)bk.order.size();
    in.nS = 1;
    in.per_instance = 1;
    in.sys = b->d_systab.as<SysDev>();
    in.sys_of = b->d_sys_of.as<int>();
    in.order = bk.d_order.as<int>();
    in.E = b->Ep.as<double>();
    in.seeds = b->Sp.as<uint64_t>();
    in.Wi = b->Wp.as<double>();
    in.sigL = b->sigL.as<double2>();
    in.sigR = b->sigR.as<double2>();
    in.sig_off = b->d_sig_off.as<long long>();
    in.T = dT;
    in.status = dSt;
    in.out_index = b->d_perm.as<int>();
    in.lstatus = b->lst.as<int>();
    in.queue = b->queue.as<int>() + q;
    const int grid = std::max(1, std::min(in.n, b->nsm * std::max(1, ctas)));
    void *work = static_cast<char *>(b->work.p) + bk.work_off;
    if (bk.kind == 1) {
        CK(knit_launch_mixed_impl(&in, bk.Mmax, grid, bk.use_tc, st), "mixed sweep launch");
    } else if (bk.kind == 2) {
        CK(knit_launch_mixed_wide(&in, bk.Mmax, grid, work, st), "wide mixed sweep launch");
    } else if (bk.kind == 3) {
        CK(knit_launch_mixed_tc128(&in, grid, work, st), "tensor-core wide sweep launch");
    } else {
        const int use_smem = knit_fp64_smem_bytes(bk.Mmax, 1, 3) <= 220 * 1024;
        CK(knit_launch_sweep_fp64(&in, bk.Mmax, grid, static_cast<double2 *>(work), use_smem, st),
           "fp64 sweep launch");
    }
    return KNIT_OK;
}

}  // namespace

extern "C" {

knit_status knit_batch_transmission(knit_batch b, const double *E, const uint64_t *seeds,
                                    const double *W, const knit_lead_opts *opts, double *T,
                                    int32_t *status, void *stream)
{
    if (!b || !E || !T) return fail(KNIT_ERR_INVALID, "knit_batch_transmission: bad arguments");
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = b->nInst;
    knit_status r;
    if ((r = batch_prepare(b, E, seeds, W, opts, st)) != KNIT_OK) return r;
    bool hT, hSt = false;
    double *dT;
    int *dSt;
    if ((r = stage_out(b->T, T, (size_t)n, &dT, &hT, "T")) != KNIT_OK ||
        (r = stage_out(b->status, (int *)status, (size_t)n, &dSt, &hSt, "status")) != KNIT_OK)
        return r;
    if (dSt) fill_int<<<(n + 255) / 256, 256, 0, st>>>(dSt, n, ST_TIMEOUT);
    CK(cudaMemsetAsync(b->queue.p, 0, sizeof(int) * b->buckets.size(), st), "queue reset");
    // fork: every variant on its own stream after the work above, heaviest
    // first; join back into st
    CK(cudaEventRecord(b->ready, st), "fork");
    for (size_t q = 0; q < b->buckets.size(); ++q) {
        auto &bk = b->buckets[q];
        CK(cudaStreamWaitEvent(bk.stream, b->ready, 0), "fork");
        if ((r = batch_launch(b, q, bk.ctas, dT, dSt, bk.stream)) != KNIT_OK) return r;
        CK(cudaEventRecord(bk.done, bk.stream), "join");
        CK(cudaStreamWaitEvent(st, bk.done, 0), "join");
    }
    if (hT) CK(cudaMemcpyAsync(T, dT, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "T out");
    if (hSt) CK(cudaMemcpyAsync(status, dSt, sizeof(int) * n, cudaMemcpyDeviceToHost, st), "status out");
    return finish(st, hT || hSt, "knit_batch_transmission");
}

knit_status knit_batch_buckets(knit_batch b, int32_t *nb, int32_t *kind, int32_t *Mmax, int32_t *count,
                               int32_t *max_ctas)
{
    if (!b || !nb) return fail(KNIT_ERR_INVALID, "knit_batch_buckets: bad arguments");
    *nb = (int32_t)b->buckets.size();
    for (size_t q = 0; q < b->buckets.size(); ++q) {
        const auto &bk = b->buckets[q];
        if (kind) kind[q] = bk.kind;
        if (Mmax) Mmax[q] = bk.Mmax;
        if (count) count[q] = (int32_t)bk.order.size();
        if (max_ctas) max_ctas[q] = bk.max_ctas;
    }
    return KNIT_OK;
}

knit_status knit_batch_configure(knit_batch b, const int32_t *config)
{
    if (!b || !config) return fail(KNIT_ERR_INVALID, "knit_batch_configure: bad arguments");
    for (size_t q = 0; q < b->buckets.size(); ++q) {
        auto &bk = b->buckets[q];
        bk.ctas = std::max(1, std::min((int)config[q], bk.max_ctas));
    }
    return KNIT_OK;
}

knit_status knit_batch_autotune(knit_batch b, const double *E, const uint64_t *seeds, const double *W,
                                const knit_lead_opts *opts, int32_t *config, float *ms)
{
    if (!b || !E) return fail(KNIT_ERR_INVALID, "knit_batch_autotune: bad arguments");
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    cudaStream_t st = nullptr;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "autotune stream");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    };
    knit_status r = KNIT_OK;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cleanup();
        return cuda_fail(ce, "autotune events");
    }
    const int n = b->nInst;
    if ((r = batch_prepare(b, E, seeds, W, opts, st)) != KNIT_OK ||
        (ce = b->T.ensure(sizeof(double) * n)) != cudaSuccess ||
        (ce = b->status.ensure(sizeof(int) * n)) != cudaSuccess) {
        cleanup();
        return r != KNIT_OK ? r : cuda_fail(ce, "autotune buffers");
    }
    for (size_t q = 0; q < b->buckets.size() && r == KNIT_OK; ++q) {
        auto &bk = b->buckets[q];
        float best = -1.0f;
        int best_k = bk.ctas;
        for (int k = 1; k <= bk.max_ctas && bk.max_ctas > 1; ++k) {
            float t = 0.0f;
            if ((ce = cudaMemsetAsync(b->queue.as<int>() + q, 0, sizeof(int), st)) != cudaSuccess ||
                (ce = cudaEventRecord(e0, st)) != cudaSuccess) break;
            if ((r = batch_launch(b, q, k, b->T.as<double>(), b->status.as<int>(), st)) != KNIT_OK) break;
            if ((ce = cudaEventRecord(e1, st)) != cudaSuccess || (ce = cudaEventSynchronize(e1)) != cudaSuccess ||
                (ce = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess)
                break;
            if (best < 0.0f || t < best) {
                best = t;
                best_k = k;
            }
        }
        if (r == KNIT_OK && ce != cudaSuccess) r = cuda_fail(ce, "autotune launch");
        bk.ctas = best_k;
        if (config) config[q] = best_k;
        if (ms) ms[q] = best;
    }
    cleanup();
    return r;
}


// ---------------------------------------------------------------------------
// learned lead model

knit_status knit_lead_model_train(knit_system s, int32_t lead, const double *E_train, int32_t nTrain,
                                  int32_t epochs, int32_t batch, float lr, uint64_t seed,
                                  const knit_lead_opts *opts, float *loss_out,
                                  knit_lead_model *out, void *stream)
{
    knit_status r = check_system(s);
    if (r != KNIT_OK) return r;
    if (!out || !E_train || nTrain < 2 || epochs < 1 || batch < 1 || !(lr > 0.f))
        return fail(KNIT_ERR_INVALID, "knit_lead_model_train: bad arguments");
    if (lead != 0 && lead != 1) return fail(KNIT_ERR_INVALID, "lead must be 0 or 1");
    const Lead &ld = s->lead[lead];
    // a period-2 lead split into blocks of at most 4: the network predicts
    // every block's supercell surface function; otherwise the whole cell's g
    const bool blocks = ld.Mp != s->M && ld.nsec > 1 && 2 * ld.ms <= 4;
    if (!blocks && s->M > 8)
        return fail(KNIT_ERR_INVALID, "learned leads support cells of at most 8 orbitals, or period-2 "
                                      "leads that split into blocks of at most 4");
    if (!blocks && ld.Mp != s->M)
        return fail(KNIT_ERR_INVALID, "this period-2 lead does not split into blocks of at most 4");
    const int bsz = blocks ? 2 * ld.ms : 0, nsec = blocks ? ld.nsec : 0;
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> hE;
    if ((r = to_host(hE, E_train, (size_t)nTrain, "E_train")) != KNIT_OK) return r;
    knit_lead_model md = new (std::nothrow)
        knit_lead_model_s(s->M, blocks ? 2 * nsec * bsz * bsz : 2 * s->M * s->M);
    if (!md) return fail(KNIT_ERR_OOM, "host allocation");
    md->nsec = nsec;
    md->nb = bsz;
    md->sys = s;
    md->lead = lead;
    md->device = s->device;
    const double lo = *std::min_element(hE.begin(), hE.end());
    const double hi = *std::max_element(hE.begin(), hE.end());
    md->mid = 0.5 * (lo + hi);
    md->half = std::max(0.5 * (hi - lo), 1e-6);
    auto cleanup = [&](knit_status code) {
        DevBuf *bufs[] = {&md->params, &md->grads, &md->m, &md->v, &md->act, &md->dact, &md->U,
                          &md->Tt, &md->loss, &md->idx, &md->tmpE};
        for (DevBuf *b : bufs) b->release();
        delete md;
        return code;
    };
    // initial weights: uniform in +-sqrt(6 / (fan_in + fan_out)) from a SplitMix64 stream
    std::vector<float> P(md->nparam, 0.f);
    uint64_t z = seed;
    auto urand = [&]() {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        return (double)(x >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < knit_lead_model_s::NL; ++l) {
        const double a = std::sqrt(6.0 / (md->dims[l] + md->dims[l + 1]));
        for (size_t q = 0; q < (size_t)md->dims[l + 1] * md->dims[l]; ++q)
            P[md->woff[l] + q] = (float)(a * (2.0 * urand() - 1.0));
    }
    cudaError_t e;
    if ((e = md->params.ensure(sizeof(float) * md->nparam)) != cudaSuccess ||
        (e = md->grads.ensure(sizeof(float) * md->nparam)) != cudaSuccess ||
        (e = md->m.ensure(sizeof(float) * md->nparam)) != cudaSuccess ||
        (e = md->v.ensure(sizeof(float) * md->nparam)) != cudaSuccess ||
        (e = md->loss.ensure(sizeof(float))) != cudaSuccess ||
        (e = md->tmpE.ensure(sizeof(double) * nTrain)) != cudaSuccess ||
        (e = md->idx.ensure(sizeof(int) * nTrain)) != cudaSuccess ||
        (e = cudaMemcpy(md->params.p, P.data(), sizeof(float) * md->nparam, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(md->m.p, 0, sizeof(float) * md->nparam)) != cudaSuccess ||
        (e = cudaMemset(md->v.p, 0, sizeof(float) * md->nparam)) != cudaSuccess ||
        (e = cudaMemcpy(md->tmpE.p, hE.data(), sizeof(double) * nTrain, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cleanup(cuda_fail(e, "model allocation"));
    // targets: the library's own decimation at every training energy (for a
    // lead in blocks, the blocks' surface functions stay in the system's
    // block buffer, energy-major per block)
    const size_t MM = (size_t)s->M * s->M;
    DevBuf gtr, sgtr, sttr;
    if ((e = gtr.ensure(sizeof(double2) * (blocks ? 1 : MM * nTrain))) != cudaSuccess ||
        (e = sgtr.ensure(sizeof(double2) * MM * nTrain)) != cudaSuccess ||
        (e = sttr.ensure(sizeof(int) * nTrain)) != cudaSuccess)
        return cleanup(cuda_fail(e, "training targets"));
    knit_lead_opts dec{};
    dec.method = KNIT_LEAD_DECIMATION;
    if (opts) {
        dec.eta = opts->eta;
        dec.tol = opts->tol;
        dec.maxit = opts->maxit;
    }
    if ((r = compute_sigma(s, lead, md->tmpE.as<double>(), nTrain, &dec, sgtr.as<double2>(),
                           gtr.as<double2>(), sttr.as<int>(), nullptr, st)) != KNIT_OK)
        return cleanup(r);
    std::vector<int> hst(nTrain);
    if ((e = cudaMemcpyAsync(hst.data(), sttr.p, sizeof(int) * nTrain, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cleanup(cuda_fail(e, "training targets"));
    std::vector<int> valid;
    for (int i = 0; i < nTrain; ++i)
        if (hst[i] == ST_OK) valid.push_back(i);
    if (blocks && valid.size() > 16) {
        // a lead in blocks: leave out the energies next to a band edge of some
        // block (largest |g| above 8x the median), where g diverges like
        // 1/sqrt(E - E_edge) and would dominate the squared error; Newton falls
        // back to decimation there anyway
        DevBuf gm;
        std::vector<float> hg(nTrain);
        if ((e = gm.ensure(sizeof(float) * nTrain)) != cudaSuccess ||
            (e = knit_mlp_block_gmax(s->secg.as<double2>(), nsec, bsz * bsz, nTrain, gm.as<float>(), st)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(hg.data(), gm.p, sizeof(float) * nTrain, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cleanup(cuda_fail(e, "training targets"));
        std::vector<float> v;
        for (int i : valid) v.push_back(hg[i]);
        std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
        const float cap = 8.f * v[v.size() / 2];
        std::vector<int> kept;
        for (int i : valid)
            if (hg[i] <= cap) kept.push_back(i);
        valid.swap(kept);
    }
    if (valid.size() < 2) return cleanup(fail(KNIT_ERR_NOCONVERGE, "decimation failed on the training set"));
    const int nv = (int)valid.size();
    const int B = std::min(batch, nv);
    if ((r = model_reserve(md, B)) != KNIT_OK) return cleanup(r);
    const int dout = md->dims[knit_lead_model_s::NL];
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = nv - 1; i > 0; --i) {   // Fisher-Yates shuffle of the valid set
            const int j = (int)(urand() * (i + 1));
            std::swap(valid[i], valid[std::min(j, i)]);
        }
        if ((e = cudaMemcpyAsync(md->idx.p, valid.data(), sizeof(int) * nv, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(md->loss.p, 0, sizeof(float), st)) != cudaSuccess)
            return cleanup(cuda_fail(e, "training"));
        int nb = 0;
        for (int b0 = 0; b0 + B <= nv; b0 += B, ++nb) {
            const int *ib = md->idx.as<int>() + b0;
            if ((e = knit_mlp_inputs(md->tmpE.as<double>(), ib, B, md->mid, md->half,
                                     md->act.as<float>(), st)) != cudaSuccess ||
                (e = blocks ? knit_mlp_targets_blocks(s->secg.as<double2>(), ib, B, nsec, bsz * bsz, nTrain,
                                                      md->Tt.as<float>(), st)
                            : knit_mlp_targets(gtr.as<double2>(), ib, B, (int)MM, md->Tt.as<float>(), st)) !=
                    cudaSuccess)
                return cleanup(cuda_fail(e, "training batch"));
            if ((r = model_forward(md, B, st)) != KNIT_OK || (r = model_backward(md, B, st)) != KNIT_OK)
                return cleanup(r);
            if ((e = knit_mlp_adam(md->params.as<float>(), md->grads.as<float>(), md->m.as<float>(),
                                   md->v.as<float>(), (int)md->nparam, lr, ++md->step, st)) != cudaSuccess)
                return cleanup(cuda_fail(e, "adam"));
        }
        if (loss_out) {
            float l = 0.f;
            if ((e = cudaMemcpyAsync(&l, md->loss.p, sizeof(float), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return cleanup(cuda_fail(e, "training loss"));
            loss_out[ep] = nb ? l / nb : 0.f;
        }
    }
    (void)dout;
    CK(cudaStreamSynchronize(st), "training");
    *out = md;
    return KNIT_OK;
}

knit_status knit_lead_model_destroy(knit_lead_model md)
{
    if (!md) return KNIT_OK;
    cudaSetDevice(md->device);
    DevBuf *bufs[] = {&md->params, &md->grads, &md->m, &md->v, &md->act, &md->dact, &md->U,
                      &md->Tt, &md->loss, &md->idx, &md->tmpE};
    for (DevBuf *b : bufs) b->release();
    delete md;
    return KNIT_OK;
}

int64_t knit_lead_model_num_params(knit_lead_model md) { return md ? (int64_t)md->nparam : 0; }

int64_t knit_lead_model_num_outputs(knit_lead_model md)
{
    return md ? (int64_t)md->dims[knit_lead_model_s::NL] : 0;
}

knit_status knit_lead_model_get_params(knit_lead_model md, float *params)
{
    if (!md || !params) return fail(KNIT_ERR_INVALID, "NULL argument");
    CK(cudaMemcpy(params, md->params.p, sizeof(float) * md->nparam, cudaMemcpyDefault), "get params");
    return KNIT_OK;
}

knit_status knit_lead_model_set_params(knit_lead_model md, const float *params)
{
    if (!md || !params) return fail(KNIT_ERR_INVALID, "NULL argument");
    CK(cudaMemcpy(md->params.p, params, sizeof(float) * md->nparam, cudaMemcpyDefault), "set params");
    return KNIT_OK;
}

knit_status knit_lead_model_forward(knit_lead_model md, const double *E, int32_t nE, float *out,
                                    void *stream)
{
    if (!md || !E || !out || nE < 1) return fail(KNIT_ERR_INVALID, "bad arguments");
    CK(cudaSetDevice(md->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    knit_status r;
    const double *dE;
    if ((r = stage_in(md->tmpE, E, (size_t)nE, st, &dE, "E")) != KNIT_OK) return r;
    if ((r = model_reserve(md, nE)) != KNIT_OK) return r;
    CK(knit_mlp_inputs(dE, nullptr, nE, md->mid, md->half, md->act.as<float>(), st), "inputs");
    if ((r = model_forward(md, nE, st)) != KNIT_OK) return r;
    const size_t n = (size_t)nE * md->dims[knit_lead_model_s::NL];
    CK(cudaMemcpyAsync(out, md->act.as<float>() + md->act_off(knit_lead_model_s::NL),
                       sizeof(float) * n, cudaMemcpyDefault, st), "forward out");
    return finish(st, true, "knit_lead_model_forward");
}

knit_status knit_lead_model_gradient(knit_lead_model md, const double *E, const float *target,
                                     int32_t n, float *grad, float *loss, void *stream)
{
    if (!md || !E || !target || !grad || n < 1) return fail(KNIT_ERR_INVALID, "bad arguments");
    CK(cudaSetDevice(md->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    knit_status r;
    const double *dE;
    if ((r = stage_in(md->tmpE, E, (size_t)n, st, &dE, "E")) != KNIT_OK) return r;
    if ((r = model_reserve(md, n)) != KNIT_OK) return r;
    const int dout = md->dims[knit_lead_model_s::NL];
    CK(cudaMemcpyAsync(md->Tt.p, target, sizeof(float) * (size_t)n * dout, cudaMemcpyDefault, st),
       "targets");
    CK(knit_mlp_inputs(dE, nullptr, n, md->mid, md->half, md->act.as<float>(), st), "inputs");
    CK(md->loss.ensure(sizeof(float)), "loss");
    CK(cudaMemsetAsync(md->loss.p, 0, sizeof(float), st), "loss");
    if ((r = model_forward(md, n, st)) != KNIT_OK || (r = model_backward(md, n, st)) != KNIT_OK)
        return r;
    CK(cudaMemcpyAsync(grad, md->grads.p, sizeof(float) * md->nparam, cudaMemcpyDefault, st), "grad");
    if (loss) CK(cudaMemcpyAsync(loss, md->loss.p, sizeof(float), cudaMemcpyDefault, st), "loss");
    return finish(st, true, "knit_lead_model_gradient");
}

}  // extern "C"
