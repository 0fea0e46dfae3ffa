// lead_noalloc.cu -- a lead self-energy entry point that allocates nothing.
//
// knit_lead_selfenergy keeps its decimation workspace in device memory that
// the library allocates (and grows) with cudaMalloc.  Some callers cannot let
// a library do that: a serving process whose framework owns every byte of
// device memory through its own pool and budgets it, a latency-critical loop
// that must not hit cudaFree (which synchronises the whole device), or code
// embedded in another runtime that forbids allocation.  For them,
// knit_lead_decimation_noalloc runs the same Sancho-Rubio decimation kernel
// with its scratch taken from one fixed array compiled into the library:
//
//   * every GPU that loads the library holds the array (9 MiB) until the
//     process exits, whether or not the entry point is ever called;
//   * the array bounds what one call can do: lead cells up to
//     KNIT_NOALLOC_MAX_M = 64 orbitals, energies processed 16 at a time;
//   * all calls share the array and it keeps the last call's contents, so
//     calls that overlap on the GPU (two streams, or two host threads) race
//     and must be serialised by the caller;
//   * every call looks up the array's device address on the current device
//     with cudaGetSymbolAddress (cheap next to the launch, and never stale
//     after a cudaDeviceReset reloads the module); the first lookup on a
//     device may load the library's module, so make the first call before
//     any stream capture.
//
// Sigma is formed with V treated as a dense M x M matrix (the allocating
// entry point knows the lead's block structure and skips V's zero blocks),
// so the two entry points run the same decimation iteration but may round
// Sigma differently in the last bits.
// The kernel initialises every workspace matrix it reads for each energy from
// the inputs, so nothing in the array needs to start at zero.

#include <cuda_runtime.h>

#include "../../include/knit.h"
#include "knit_common.cuh"

extern "C" cudaError_t knit_launch_decimation(const double2 *, const double2 *, int, int, int,
                                              const double *, int, double, double, int, double2 *,
                                              double2 *, double2 *, int *, int *, int,
                                              cudaStream_t);
extern "C" void knit_set_last_error(const char *msg);

#define KNIT_NOALLOC_MAX_M 64
#define KNIT_NOALLOC_CTAS 16
#define KNIT_NOALLOC_MATS 9   // 8 decimation work matrices + the surface g, per CTA

static __device__ __align__(256) double2
    knit_noalloc_scratch[(size_t)KNIT_NOALLOC_CTAS * KNIT_NOALLOC_MATS * KNIT_NOALLOC_MAX_M *
                         KNIT_NOALLOC_MAX_M];

namespace {

bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

knit_status noalloc_fail(knit_status st, const char *msg)
{
    knit_set_last_error(msg);
    return st;
}

}  // namespace

extern "C" knit_status knit_lead_decimation_noalloc(const knit_c128 *H0, const knit_c128 *V,
                                                    int32_t M, int32_t lead, const double *E,
                                                    int32_t nE, double eta, double tol,
                                                    int32_t maxit, knit_c128 *sigma,
                                                    int32_t *iters, int32_t *status, void *stream)
{
    if (M < 1 || M > KNIT_NOALLOC_MAX_M)
        return noalloc_fail(KNIT_ERR_INVALID,
                            "knit_lead_decimation_noalloc: M must be in [1, 64] (fixed scratch)");
    if (lead != 0 && lead != 1)
        return noalloc_fail(KNIT_ERR_INVALID, "knit_lead_decimation_noalloc: lead must be 0 or 1");
    if (nE < 1) return noalloc_fail(KNIT_ERR_INVALID, "knit_lead_decimation_noalloc: nE < 1");
    if (!on_device(H0) || !on_device(V) || !on_device(E) || !on_device(sigma) ||
        (iters && !on_device(iters)) || (status && !on_device(status)))
        return noalloc_fail(KNIT_ERR_INVALID,
                            "knit_lead_decimation_noalloc: every array must be device memory");
    if (!(eta > 0.0)) eta = 1e-12;
    if (!(tol > 0.0)) tol = 1e-14;
    if (maxit <= 0) maxit = 200;

    // the array's address on the current device, looked up on every call
    void *p = nullptr;
    const cudaError_t ge = cudaGetSymbolAddress(&p, knit_noalloc_scratch);
    if (ge != cudaSuccess || !p) {
        cudaGetLastError();
        return noalloc_fail(KNIT_ERR_CUDA,
                            "knit_lead_decimation_noalloc: cudaGetSymbolAddress failed");
    }
    double2 *const scratch = static_cast<double2 *>(p);
    const size_t MM = (size_t)M * M;
    double2 *work = scratch;                                   // 8 M*M per CTA
    double2 *gslots = scratch + (size_t)KNIT_NOALLOC_CTAS * 8 * MM;   // one M*M per energy in flight
    cudaStream_t st = (cudaStream_t)stream;
    for (int e0 = 0; e0 < nE; e0 += KNIT_NOALLOC_CTAS) {
        const int n = nE - e0 < KNIT_NOALLOC_CTAS ? nE - e0 : KNIT_NOALLOC_CTAS;
        // V block size M: V is treated as a dense M x M matrix when Sigma is
        // formed (two full M^3 products for M > 4)
        cudaError_t e = knit_launch_decimation(
            reinterpret_cast<const double2 *>(H0), reinterpret_cast<const double2 *>(V), M, M,
            lead, E + e0, n, eta, tol, maxit, work, reinterpret_cast<double2 *>(sigma) + e0 * MM,
            gslots, iters ? iters + e0 : nullptr, status ? status + e0 : nullptr, n, st);
        if (e != cudaSuccess)
            return noalloc_fail(KNIT_ERR_CUDA, cudaGetErrorString(e));
    }
    return KNIT_OK;
}
