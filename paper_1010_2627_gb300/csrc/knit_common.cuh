// knit_common.cuh -- device helpers shared by the library's kernels:
// complex arithmetic on double2/float2, double-float (hi + lo) error-free
// transformations, the disorder counter, block reductions, and the kernel
// parameter blocks.  Included by every .cu file of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define KNIT_DEV __device__ __forceinline__

// ---------------------------------------------------------------------------
// complex double (double2) and complex float (float2)

KNIT_DEV double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
KNIT_DEV double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
KNIT_DEV double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
KNIT_DEV double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
KNIT_DEV double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// acc + a * b
KNIT_DEV double2 cfma(double2 a, double2 b, double2 acc)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
// acc - a * b
KNIT_DEV double2 cfms(double2 a, double2 b, double2 acc)
{
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
KNIT_DEV double2 crcp(double2 a)
{
    double d = 1.0 / fma(a.x, a.x, a.y * a.y);
    return make_double2(a.x * d, -a.y * d);
}
KNIT_DEV double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }

KNIT_DEV float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
KNIT_DEV float2 cmulf(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
KNIT_DEV float2 cfmaf(float2 a, float2 b, float2 acc)
{
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
KNIT_DEV float2 cfmsf(float2 a, float2 b, float2 acc)
{
    acc.x = fmaf(-a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(-a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
    return acc;
}
KNIT_DEV float2 crcpf(float2 a)
{
    // reciprocal through a scaled denominator so that |a| near the float
    // range limits neither overflows nor flushes
    float m = fmaxf(fabsf(a.x), fabsf(a.y));
    float s = 1.0f / m;
    float ax = a.x * s, ay = a.y * s;
    float d = 1.0f / fmaf(ax, ax, ay * ay);
    return make_float2(ax * d * s, -ay * d * s);
}
KNIT_DEV float cabs1f(float2 a) { return fabsf(a.x) + fabsf(a.y); }

// ---------------------------------------------------------------------------
// Error-free transformations (Knuth TwoSum; TwoProduct with FMA, Ogita, Rump
// & Oishi 2005).  A double-float value is hi + lo with |lo| <= ulp(hi)/2.

KNIT_DEV void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// accumulate the exact product a*b plus the low-order term c*b into (s, e):
// s + e ~= s + e + (a + c) * b with the rounding error of the running sum kept
KNIT_DEV void dot2_acc(float a, float c, float b, float &s, float &e)
{
    float p = a * b;
    float pe = fmaf(a, b, -p);
    pe = fmaf(c, b, pe);
    float t, te;
    two_sum(s, p, t, te);
    s = t;
    e += te + pe;
}

// ---------------------------------------------------------------------------
// Disorder counter: SplitMix64 output function (Steele, Lea & Flood 2014),
// r = (mix(mix(seed) ^ (n << 32 | site)) >> 11) * 2^-53, eps = W (r - 1/2).

KNIT_DEV uint64_t knit_mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

KNIT_DEV double knit_disorder(uint64_t mixed_seed, int n, int site, double W)
{
    uint64_t key = ((uint64_t)(uint32_t)n << 32) | (uint64_t)(uint32_t)site;
    uint64_t r = knit_mix64(mixed_seed ^ key);
    double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    return W * (u - 0.5);
}

// ---------------------------------------------------------------------------
// Block reductions

template <typename T>
KNIT_DEV T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block; `red` has blockDim.x/32 entries; result valid in all threads
template <typename T>
__device__ T block_sum(T v, T *red)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    for (int i = 0; i < nw; ++i) s += red[i];
    return s;
}

// argmax over a warp with ties broken towards the lower index
KNIT_DEV void warp_argmax(double &v, int &i)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
    }
}
KNIT_DEV void warp_argmaxf(float &v, int &i)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
    }
}

// ---------------------------------------------------------------------------
// Status codes written per instance (same values as knit_status)
enum {
    ST_OK = 0,
    ST_SINGULAR = 4,
    ST_NOCONVERGE = 5,
    ST_TIMEOUT = 6,
    ST_NONFINITE = 7
};

// ---------------------------------------------------------------------------
// Parameter blocks (plain structs passed by value to the kernels)

struct SysDev {
    int M, L, block, Vperiod;
    int vdiag;                 // 1: every V is diagonal (block-diagonal with 1 x 1 blocks)
    int vb;                    // block size of the block-diagonal V (M for a tridiagonal V)
    int vband;                 // nonzeros of V within this distance of the diagonal (>= vb: any)
    const double2 *H0;         // M*M
    const double2 *V;          // Vperiod*M*M
    const double *sign;        // block
    const double *onsite;      // L*M or nullptr
    // sparse copy of H0 (rows with their non-zeros), used by the mixed residual
    const int *h0_rowptr;      // M+1
    const int *h0_col;         // nnz
    const double2 *h0_val;     // nnz
    // H0 as double-float (hi, lo) in the width-128 layout: column pair jp,
    // row i at float4 jp * 128 + i; zero outside M x M (M <= 128, else null)
    const float4 *h0_dfh, *h0_dfl;
    // a honeycomb-type system run by half-rows: orbital i of slice m is the
    // site xmap[((((m >> 1) & 1) << 1) | (m & 1)) * M + i] of row m >> 1, whose
    // disorder it draws (block 1); nullptr for every other system
    const int *xmap;
};

struct InstDev {
    int n;                     // instances in this launch
    int nS;                    // energy x seed grid: seeds per energy
    int per_instance;          // 1: E, seed, W and self-energies given per instance
    const SysDev *sys;         // system table (device memory)
    const int *sys_of;         // system of each instance, or nullptr (system 0)
    const int *order;          // queue position -> instance (cost order), or nullptr
    const double *E;           // grid: nE values; per instance: one per instance
    const uint64_t *seeds;     // grid: nS values; per instance: one per instance; nullptr = 0
    double W;                  // disorder strength (grid mode, or when Wi is nullptr)
    const double *Wi;          // per-instance disorder strength or nullptr
    const double2 *sigL;       // grid: nE*M*M; per instance: concatenated blocks
    const double2 *sigR;
    const long long *sig_off;  // per instance: element offset of its blocks
    double *T;                 // results, at out_index[inst] (or inst)
    int *status;               // or nullptr
    const int *out_index;      // output position of each instance, or nullptr
    const int *lstatus;        // lead-solver status (grid: per energy; else per instance)
    int *queue;                // one int, zeroed before launch: next queue position
    double2 *GLL;              // optional: G_LL (M x M, complex128) at out position * M * M
};

// an arbitrary geometry with P leads cut into K slices (graph_sweep.cu):
// lead 0's sites are slice 0 (in order), every other lead's sites lie in the
// last slice at positions lpos[loff[p] + a]
struct GraphDev {
    int K, Mmax, P;
    const int *width;          // K slice widths
    const long long *hoff;     // offset of H_k (M_k x M_k) in blocks
    const long long *voff;     // offset of V_k = H_{k,k-1} (M_k x M_{k-1}) in blocks, k >= 1
    const double2 *blocks;
    const int *lw;             // P lead widths
    const int *lpos;           // lead sites' positions (slice 0 for lead 0, else the last slice)
    const int *loff;           // P offsets into lpos
    const double2 *const *sig; // P self-energy arrays, lead p at energy e: sig[p] + e * lw[p]^2
};

// parameters of one instance
struct InstParams {
    int out;                   // output position
    double E;
    uint64_t ms;               // mixed seed of the disorder counter
    double W;
    const double2 *SL, *SR;
    int st;                    // initial status (lead failures)
};

KNIT_DEV int take_position(const InstDev &in, int q) { return in.order ? in.order[q] : q; }

KNIT_DEV const SysDev &inst_system(const InstDev &in, int inst)
{
    return in.sys[in.sys_of ? in.sys_of[inst] : 0];
}

KNIT_DEV InstParams inst_params(const InstDev &in, int inst, int M)
{
    InstParams p;
    const size_t MM = (size_t)M * M;
    if (in.per_instance) {
        p.E = in.E[inst];
        p.ms = knit_mix64(in.seeds ? in.seeds[inst] : 0ull);
        p.W = in.Wi ? in.Wi[inst] : in.W;
        const size_t off = in.sig_off ? (size_t)in.sig_off[inst] : (size_t)inst * MM;
        p.SL = in.sigL + off;
        p.SR = in.sigR + off;
        p.st = in.lstatus ? in.lstatus[inst] : ST_OK;
    } else {
        const int ie = inst / in.nS;
        p.E = in.E[ie];
        p.ms = knit_mix64(in.seeds ? in.seeds[inst - ie * in.nS] : 0ull);
        p.W = in.W;
        p.SL = in.sigL + (size_t)ie * MM;
        p.SR = in.sigR + (size_t)ie * MM;
        p.st = in.lstatus ? in.lstatus[ie] : ST_OK;
    }
    p.out = in.out_index ? in.out_index[inst] : inst;
    return p;
}
