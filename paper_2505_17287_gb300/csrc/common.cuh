// Internal declarations shared by the translation units of libibm.so.
// Not part of the public ABI (include/ibm.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/ibm.h"

namespace ibm {

constexpr uint8_t FLUID = IBM_FLUID, GHOST = IBM_GHOST, DEAD = IBM_DEAD;

// Deterministic reductions: every reduction kernel runs on a fixed grid of
// RED_BLOCKS blocks of RED_THREADS threads, writes one partial per block,
// and a single block then adds the partials in a fixed order.
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 152 * 8;   // 8 blocks of 256 threads per SM on a 152-SM GB300
// Reduction grids grow with the cell count up to RED_BLOCKS blocks (about
// eight cells per thread); the FP32 operator product, whose threads
// otherwise walk tens of cells on dependent loads, takes up to RED_BLOCKS_MAX.
// The partial-sum buffer is sized for that maximum.
constexpr int RED_BLOCKS_MAX = 152 * 32;

// host-side status carrier: message + code
struct Err {
    ibm_status code = IBM_OK;
    std::string msg;
};

// Failure helpers used by every host function of the library.
#define IBM_CUDA(ctx, call)                                                          \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            return (ctx)->fail(IBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                            \
    } while (0)
#define IBM_LAUNCHED(ctx) IBM_CUDA(ctx, cudaGetLastError())
#define IBM_TRY(expr)                          \
    do {                                       \
        ibm_status s_ = (expr);                \
        if (s_ != IBM_OK) return s_;           \
    } while (0)

// Division by a fixed 32-bit divisor with a multiply-high and a shift
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): q = (hi(n*m) + n) >> s, with the addition done
// without overflow as ((n - t) >> 1) + t.
struct FastDiv {
    uint32_t d = 1, m = 0, s = 0;
    FastDiv() = default;
    explicit FastDiv(uint32_t div) : d(div) {
        uint32_t l = 0;
        while ((1ull << l) < div) ++l;          // l = ceil(log2 d)
        m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1);
        s = l;
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        if (d == 1) return n;
        const uint32_t t = __umulhi(n, m);
        return (t + ((n - t) >> 1)) >> (s - 1);
    }
};

// device view of a grid level (coordinates and extents)
// j and k of grid row `row` (= j + ny k) by the multiply-shift divider:
// a 64-bit (or even 32-bit) integer division costs tens of instructions per
// thread, a measurable share of the issue slots of a streaming stencil pass
__device__ __forceinline__ void row_jk(uint32_t row, const FastDiv &fny, int ny, int &j, int &k) {
    const uint32_t kk = fny.div(row);
    k = (int)kk;
    j = (int)(row - kk * (uint32_t)ny);
}

struct GridDev {
    int nx, ny, nz, ndim;
    int64_t n;            // nx*ny*nz
    const double *xf, *yf, *zf;   // faces
    const double *xc, *yc, *zc;   // centres
    const double *dx, *dy, *dz;   // widths
    const double *hx, *hy, *hz;   // centre spacing; h?[i] = c[i]-c[i-1] for i>=1, [0] unused
    // full pressure operator per axis, divided by the cell volume:
    // cXm[i] = 1/(h[i] d[i]) (0 at the low wall), cXp[i] = 1/(h[i+1] d[i]) (0 at
    // the high wall), cXs = cXm + cXp
    const double *cxm, *cxp, *cxs, *cym, *cyp, *cys, *czm, *czp, *czs;
    FastDiv fnx, fny;     // division by nx and ny (cell index < 2^32)
    const double *rdx, *rdy, *rdz;  // 1 / cell widths
    const double *rhx, *rhy, *rhz;  // 1 / centre spacing h (index 0 unused, 0)
};

// cell (i, j, k) of a linear index below 2^32
__device__ __forceinline__ void split3(const GridDev &g, uint32_t c, int &i, int &j, int &k) {
    const uint32_t t = g.fnx.div(c);
    i = (int)(c - t * (uint32_t)g.nx);
    const uint32_t kk = g.fny.div(t);
    j = (int)(t - kk * (uint32_t)g.ny);
    k = (int)kk;
}

// per-ghost tables (device, structure of arrays)
struct GhostDev {
    int64_t ng;
    const int64_t *gidx;      // ascending
    const int64_t *sidx;      // 8 per ghost
    const double *wv, *wp;    // 8 per ghost
    const double *bv, *bp;    // 1 per ghost
};

// one multigrid level of the staircase operator K = sum_open T (x_c - x_nb)
// (T the open face area over the centre spacing). A "fine" level holds no
// coefficient arrays: it derives them from the cell types and 1D metrics.
template <typename T>
struct MGLevel {
    int nx, ny, nz;
    int64_t n;
    FastDiv fnx, fny;
    T *tx, *ty, *tz;   // coefficient of the face on the low side of each cell
    T *d, *dinv;       // diagonal (sum of the six faces) and its inverse (0 if isolated)
    T *x, *f;          // correction and right-hand side of coarse levels
    // fine-level description
    const uint8_t *type;
    const uint8_t *omask;       // bit f: face f (-x,+x,-y,+y,-z,+z) open; bit 7: cell FLUID
    const T *wx, *wy, *wz;      // cell widths
    const T *rhx, *rhy, *rhz;   // 1 / centre spacing (index i: face between i-1 and i)
};

struct Ctx;

// allocation through the user hook or cudaMalloc; tracked for release
void *dev_alloc(Ctx *c, size_t bytes);
void dev_free(Ctx *c, void *p);

// reduction helper: block partials to one value (device function kernels in solver.cu)
ibm_status reduce_sum(Ctx *c, const double *partials, int nparts, double *out_dev);

}  // namespace ibm

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
namespace ibm {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block sum in a fixed order; result valid in thread 0
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < NT / 32 ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// block sum of FP32 per-thread partials: summed in FP32 within each warp,
// then in FP64 across the warps (fixed order; valid in thread 0). On GB300 a
// warp-wide FP64 instruction takes the FP64 pipe for many cycles, and the
// FP64 shuffle tree cost the FP32 streaming kernels a third of their time
template <int NT>
__device__ __forceinline__ double block_sum(float v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = (double)v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < NT / 32; ++q) t += sh[q];
    __syncthreads();
    return t;
}

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace ibm
