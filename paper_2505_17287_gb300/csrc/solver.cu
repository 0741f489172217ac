// Pressure Poisson solver (Section 2.1, pressure equation; Section 2.2,
// Neumann ghost-cell rows) on one GPU.
//
//   outer:  FP64 Krylov iteration on P A phi = P b, where A is the full
//           ghost-cell operator (FLUID rows: variable-coefficient 7-point
//           (2D: 5-point) div-grad including ghost neighbours; GHOST rows:
//           phi_G - sum wp phi_m; DEAD rows: identity) and P removes the
//           volume-weighted FLUID mean (compatibility). BiCGStab (the
//           paper's Poisson solver, Section 2.1) or restarted FGMRES;
//   preconditioner: multigrid-preconditioned CG on the staircase operator
//           K = sum over open faces T_f (x_c - x_nb) (a face is open when
//           both sides are FLUID; symmetric positive semi-definite), in FP64
//           or FP32 (storage and arithmetic; dot products accumulate in
//           FP64); then the ghost rows; then damped Jacobi sweeps of the full
//           operator on the cells within two faces of a ghost cell;
//   multigrid: V(nu1,nu2) cycle, red-black Gauss-Seidel smoothing,
//           restriction by summing children, piecewise-constant prolongation,
//           coarse operators rediscretised from the open child-face areas,
//           coarsest level solved by red-black sweeps in one thread block.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so the FP64 kernels here are
// written to minimise FP64 instructions: per-axis 1D operator coefficients,
// reciprocal diagonals, no division in the inner loops.
#include "ctx.cuh"

#include <utility>

#include <math.h>
#include <stdio.h>
#include <stdlib.h>

namespace ibm {

// device scalar slots
enum {
    S_RZ = 0, S_PQ = 1, S_AL = 2, S_RZN = 3, S_BE = 4, S_MEAN = 5, S_TMP = 8, S_MD = 16,
    B_RHO = 34, B_ALPHA = 35, B_OMEGA = 36, B_BETA = 37, B_RHO1 = 38, B_DEN = 39, B_TS = 58, B_TT = 59,
    B_FLAG = 60
};

#define KL(kid, kern, grid, block, ...)                      \
    do {                                                     \
        kt_begin(c, kid);                                    \
        ++c->nlaunch;                                        \
        kern<<<(grid), (block), 0, c->s>>>(__VA_ARGS__);     \
        kt_end(c, kid);                                      \
    } while (0)

static inline unsigned nblk(int64_t n, int t = 256) {
    int64_t b = (n + t - 1) / t;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

static inline dim3 rows_grid(int nx, int ny, int nz, int per_thread, int bx) {
    const int64_t rows = (int64_t)ny * nz;
    const int xs = (nx + per_thread - 1) / per_thread;
    return dim3((unsigned)rows, (unsigned)((xs + bx - 1) / bx), 1);
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------

// out[col] = scale * sum_i part[col*nparts + i], in a fixed order; one block
// per column
__global__ void k_finalize(const double *__restrict__ part, int nparts, double scale, double *__restrict__ out) {
    __shared__ double sh[32];
    const int col = blockIdx.x;
    double v = 0.0;
#pragma unroll 4
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[(size_t)col * nparts + i];
    v = block_sum<RED_THREADS>(v, sh);
    if (threadIdx.x == 0) out[col] = v * scale;
}

ibm_status finalize(Ctx *c, const double *part, int nparts, int ncols, double scale, double *out_dev) {
    KL(-1, k_finalize, (unsigned)ncols, RED_THREADS, part, nparts, scale, out_dev);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

ibm_status reduce_sum(Ctx *c, const double *partials, int nparts, double *out_dev) {
    return finalize(c, partials, nparts, 1, 1.0, out_dev);
}

ibm_status sync_scalars(Ctx *c, int n) {
    IBM_CUDA(c, cudaMemcpyAsync(c->hscal, c->scal, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    return IBM_OK;
}

#define GRID_STRIDE(c, n) \
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < (n); c += (int64_t)gridDim.x * blockDim.x)

// sum over FLUID cells of vol * x (x null: the FLUID volume)
__global__ void k_fluid_volsum(GridDev g, const uint8_t *__restrict__ type, const double *__restrict__ x,
                               double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    GRID_STRIDE(c, g.n) {
        if (type[c] != FLUID) continue;
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        acc += (g.dx[i] * g.dy[j] * g.dz[k]) * (x ? x[c] : 1.0);
    }
    acc = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// x -= mean on FLUID (and GHOST if ghosts) cells; DEAD cells set to 0
__global__ void k_sub_mean(int64_t n, const uint8_t *__restrict__ type, double *__restrict__ x,
                           const double *__restrict__ mean, int ghosts) {
    const double m = *mean;
    GRID_STRIDE(c, n) {
        const uint8_t t = type[c];
        if (t == FLUID || (ghosts && t == GHOST)) x[c] -= m;
        else if (t == DEAD) x[c] = 0.0;
    }
}

ibm_status fluid_mean(Ctx *c, const double *x, bool ghosts_too, double *mean_host) {
    (void)ghosts_too;
    KL(-1, k_fluid_volsum, c->nred, RED_THREADS, c->g, c->type, x, c->part);
    IBM_LAUNCHED(c);
    IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN));
    if (mean_host) {
        IBM_TRY(sync_scalars(c, S_MEAN + 1));
        *mean_host = c->hscal[S_MEAN];
    }
    return IBM_OK;
}

// ---------------------------------------------------------------------------
// full ghost-cell pressure operator (FP64)
// ---------------------------------------------------------------------------

// Accumulator type of per-thread partial sums: FP64 for FP64 vectors; FP32
// for FP32 vectors, whose cross-thread reductions are FP64 (per-element FP64
// arithmetic would make the FP32 streaming kernels FP64-bound on GB300)
// Dot products and volume sums accumulate in FP64 in both precisions (the
// FP32 inner Krylov cycle included). FP32 vectors form leaves of four
// products in FP32 (the lanes of one 16-byte load, or four consecutive
// cells) and add each leaf to an FP64 per-thread partial: one FP64 add per
// four cells, so the FP32 streaming kernels stay off the FP64 pipe's limit.
template <typename T> struct Acc { typedef double type; };

// per-axis operator coefficients in precision T (the FP64 ones are the
// GridDev arrays; FP32 copies serve the FP32 Krylov cycle of mixed mode)
template <typename T>
struct OpT {
    const T *cxm, *cxp, *cxs, *cym, *cyp, *cys, *czm, *czp, *czs;
    const T *dx, *dy, *dz;
    const T *wp;     // ghost weights, 8 per ghost
    const T *vol, *dg;   // FP64 only: per-cell volume and diagonal
};

// (A x)_c of a FLUID cell with the per-axis coefficients; boundary faces
// have coefficient 0, so a wall reads the cell itself
template <typename T>
__device__ __forceinline__ T A_row(const GridDev &g, const OpT<T> &o, const T *__restrict__ x, int64_t c, int i,
                                   int j, int k) {
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const T xc = x[c];
    const T xm = i > 0 ? x[c - 1] : xc, xp = i < g.nx - 1 ? x[c + 1] : xc;
    const T ym = j > 0 ? x[c - sy] : xc, yp = j < g.ny - 1 ? x[c + sy] : xc;
    if (sizeof(T) == 4) {
        // FP32: difference form, so constants are annihilated exactly
        T s = o.cxm[i] * (xm - xc) + o.cxp[i] * (xp - xc) + o.cym[j] * (ym - xc) + o.cyp[j] * (yp - xc);
        if (g.ndim == 3) {
            const T zm = k > 0 ? x[c - sz] : xc, zp = k < g.nz - 1 ? x[c + sz] : xc;
            s += o.czm[k] * (zm - xc) + o.czp[k] * (zp - xc);
        }
        return s;
    }
    // FP64: fewest FP64 instructions (one FMA per neighbour, stored diagonal)
    T s = o.cxm[i] * xm + o.cxp[i] * xp + o.cym[j] * ym + o.cyp[j] * yp;
    if (g.ndim == 3) {
        const T zm = k > 0 ? x[c - sz] : xc, zp = k < g.nz - 1 ? x[c + sz] : xc;
        s += o.czm[k] * zm + o.czp[k] * zp;
    }
    return s - o.dg[c] * xc;
}

// y = sgn * (A x) + b  on FLUID and DEAD rows (b may be null = 0); GHOST rows
// are written by k_ghost_rows. Partials (FP64): sum over FLUID of vol * y.
// (PLAIN: b null and sgn = 1, the product of every Krylov step; two FP64
// operations per cell fewer)
template <typename T, bool PLAIN = false>
__global__ void k_apply_A(GridDev g, OpT<T> o, const uint8_t *__restrict__ type, const T *__restrict__ x,
                          const T *__restrict__ b, T sgn, T *__restrict__ y, double *__restrict__ part) {
    __shared__ double sh[32];
    typename Acc<T>::type acc = 0;
    GRID_STRIDE(c, g.n) {
        const uint8_t t = type[c];
        if (t == GHOST) continue;
        if (t == DEAD) { y[c] = T(0); continue; }
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        const T v = PLAIN ? A_row<T>(g, o, x, c, i, j, k) : sgn * A_row<T>(g, o, x, c, i, j, k) + (b ? b[c] : T(0));
        y[c] = v;
        if constexpr (sizeof(T) == 8) acc += o.vol[c] * v;
        else acc += (double)((o.dx[i] * o.dy[j] * o.dz[k]) * v);
    }
    const double tot = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// FP32 operator product four cells at a time, for grids whose rows hold a
// multiple of four cells (16-byte aligned vectors): one 16-byte load per
// neighbour direction and the four cell types in one word, so each thread
// keeps several loads in flight where the one-cell loop stalls on load
// latency. Each cell gets the same expression as A_row<float>; GHOST cells
// are computed but not stored. The partial sums add a quad's cells in x order.
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float f4get(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
__device__ __forceinline__ uint8_t u4get(const uchar4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

__global__ void __launch_bounds__(RED_THREADS)
    k_apply_A4(GridDev g, OpT<float> o, const uint8_t *__restrict__ type, const float *__restrict__ x,
               const float *__restrict__ b, float sgn, float *__restrict__ y, double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    GRID_STRIDE(q, g.n / 4) {
        const int64_t c = 4 * q;
        const uchar4 t4 = reinterpret_cast<const uchar4 *>(type)[q];
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        const float4 xc = ld4(x + c);
        const float xl = i > 0 ? x[c - 1] : xc.x;
        const float xr = i + 4 < g.nx ? x[c + 4] : xc.w;
        const float4 ym = j > 0 ? ld4(x + c - sy) : xc;
        const float4 yp = j < g.ny - 1 ? ld4(x + c + sy) : xc;
        float4 zm = xc, zp = xc;
        if (g.ndim == 3) {
            if (k > 0) zm = ld4(x + c - sz);
            if (k < g.nz - 1) zp = ld4(x + c + sz);
        }
        const float4 bb = b ? ld4(b + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 cm = ld4(o.cxm + i), cp = ld4(o.cxp + i), dxv = ld4(o.dx + i);
        const float cym = o.cym[j], cyp = o.cyp[j], dyj = o.dy[j], dzk = o.dz[k];
        const float czm = g.ndim == 3 ? o.czm[k] : 0.f, czp = g.ndim == 3 ? o.czp[k] : 0.f;
        float out[4];
        bool ghost = false;
        float leaf = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float xe = f4get(xc, e);
            const float xm = e == 0 ? xl : f4get(xc, e - 1);
            const float xp = e == 3 ? xr : f4get(xc, e + 1);
            float s = f4get(cm, e) * (xm - xe) + f4get(cp, e) * (xp - xe) + cym * (f4get(ym, e) - xe) +
                      cyp * (f4get(yp, e) - xe);
            if (g.ndim == 3) s += czm * (f4get(zm, e) - xe) + czp * (f4get(zp, e) - xe);
            const float v = sgn * s + f4get(bb, e);
            const uint8_t t = u4get(t4, e);
            ghost |= t == GHOST;
            out[e] = t == DEAD ? 0.f : v;
            if (t == FLUID) leaf += (f4get(dxv, e) * dyj * dzk) * v;
        }
        acc += (double)leaf;
        if (!ghost) {
            *reinterpret_cast<float4 *>(y + c) = make_float4(out[0], out[1], out[2], out[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (u4get(t4, e) != GHOST) y[c + e] = out[e];
        }
    }
    const double tot = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

static inline bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// GHOST rows: y_g = sgn * (x_g - sum_m wp_m x_m) + b_g (b may be null = 0;
// the pressure equation has b_g = 0, a defect-correction right-hand side not)
template <typename T>
__global__ void k_ghost_rows(GhostDev gh, OpT<T> o, const T *__restrict__ x, const T *__restrict__ b, T sgn,
                             T *__restrict__ y) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= gh.ng) return;
    const int64_t gi = gh.gidx[q];
    T s = x[gi];
    for (int m = 0; m < 8; ++m) s -= o.wp[8 * q + m] * x[gh.sidx[8 * q + m]];
    y[gi] = sgn * s + (b ? b[gi] : T(0));
}

__global__ void k_zero_at(int64_t m, const int64_t *__restrict__ idx, double *__restrict__ x) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < m) x[idx[q]] = 0.0;
}

// x -= mean on FLUID cells (precision T); DEAD cells set to 0
// (FP32: four cells per 16-byte access, the tail one by one)
template <typename T>
__global__ void k_sub_meanT(int64_t n, const uint8_t *__restrict__ type, T *__restrict__ x,
                            const double *__restrict__ mean) {
    const T m = (T)*mean;
    int64_t n0 = 0;
    if constexpr (sizeof(T) == 4) {
        n0 = n / 4 * 4;
        GRID_STRIDE(q, n / 4) {
            const uchar4 t4 = reinterpret_cast<const uchar4 *>(type)[q];
            float4 a = reinterpret_cast<const float4 *>(x)[q];
            a.x = t4.x == FLUID ? a.x - m : (t4.x == DEAD ? 0.f : a.x);
            a.y = t4.y == FLUID ? a.y - m : (t4.y == DEAD ? 0.f : a.y);
            a.z = t4.z == FLUID ? a.z - m : (t4.z == DEAD ? 0.f : a.z);
            a.w = t4.w == FLUID ? a.w - m : (t4.w == DEAD ? 0.f : a.w);
            reinterpret_cast<float4 *>(x)[q] = a;
        }
    }
    for (int64_t c = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t t = type[c];
        if (t == FLUID) x[c] -= m;
        else if (t == DEAD) x[c] = T(0);
    }
}

template <typename T>
static OpT<T> op_of(Ctx *c);
template <>
OpT<double> op_of<double>(Ctx *c) {
    return OpT<double>{c->g.cxm, c->g.cxp, c->g.cxs, c->g.cym, c->g.cyp, c->g.cys, c->g.czm, c->g.czp, c->g.czs,
                       c->g.dx, c->g.dy, c->g.dz, c->wp, c->vol_c, c->dg_c};
}
template <>
OpT<float> op_of<float>(Ctx *c) {
    const float *const *a = (const float *const *)c->op32;
    return OpT<float>{a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7], a[8], a[9], a[10], a[11], c->wp32,
                      nullptr, nullptr};
}

// y = P(sgn * A x + b)
template <typename T>
static ibm_status apply_PA(Ctx *c, const T *x, const T *b, T sgn, T *y) {
    const OpT<T> o = op_of<T>(c);
    const int nb = sizeof(T) == 4 ? c->nred_wide : c->nred;
    if constexpr (sizeof(T) == 4) {
        if (c->g.nx % 4 == 0 && al16(x) && al16(y) && (!b || al16(b)))
            KL(K_APPLY_A, k_apply_A4, nb, RED_THREADS, c->g, o, c->type, x, b, sgn, y, c->part);
        else
            KL(K_APPLY_A, k_apply_A<T>, nb, RED_THREADS, c->g, o, c->type, x, b, sgn, y, c->part);
    } else if (!b && sgn == T(1)) {
        KL(K_APPLY_A, (k_apply_A<T, true>), nb, RED_THREADS, c->g, o, c->type, x, b, sgn, y, c->part);
    } else {
        KL(K_APPLY_A, k_apply_A<T>, nb, RED_THREADS, c->g, o, c->type, x, b, sgn, y, c->part);
    }
    IBM_LAUNCHED(c);
    if (c->ng > 0) {
        KL(-1, k_ghost_rows<T>, (unsigned)((c->ng + 255) / 256), 256, c->gh, o, x, b, sgn, y);
        IBM_LAUNCHED(c);
    }
    IBM_TRY(finalize(c, c->part, nb, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN));
    KL(-1, k_sub_meanT<T>, c->nred_wide, RED_THREADS, c->N, c->type, y, c->scal + S_MEAN);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

// ---------------------------------------------------------------------------
// FP64 vector kernels: FGMRES
// ---------------------------------------------------------------------------

struct Coef {
    double v[17];
};


// 16-byte vector of T
template <typename T> struct Vec16;
template <> struct Vec16<float> { typedef float4 type; enum { W = 4 }; };
template <> struct Vec16<double> { typedef double2 type; enum { W = 2 }; };
template <typename V> __device__ __forceinline__ auto vget(const V &v, int e);
__device__ __forceinline__ float vget(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
__device__ __forceinline__ double vget(const double2 &v, int e) { return e == 0 ? v.x : v.y; }
__device__ __forceinline__ void vset(float4 &v, int e, float a) { if (e == 0) v.x = a; else if (e == 1) v.y = a; else if (e == 2) v.z = a; else v.w = a; }
__device__ __forceinline__ void vset(double2 &v, int e, double a) { if (e == 0) v.x = a; else v.y = a; }

// Krylov basis vectors handed to a kernel by value (kernel parameter space),
// so the loop loads no pointers from global memory
template <typename T>
struct VPtrs {
    const T *p[17];
};

// partial dots: col q < NC: (w, V_q). The column count is a template
// parameter so every loop is unrolled without predicates; 16-byte loads (the
// vectors come from cudaMalloc or PyTorch's allocator, 256-byte aligned)
template <typename T, int NC>
__global__ void __launch_bounds__(RED_THREADS) k_mdot(int64_t n, const T *__restrict__ w, VPtrs<T> V,
                                                      double *__restrict__ part) {
    typedef typename Acc<T>::type A;
    typedef typename Vec16<T>::type VT;
    constexpr int W = Vec16<T>::W;
    __shared__ double sh[32];
    A acc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = A(0);
    const int64_t nv = n / W;
    GRID_STRIDE(v, nv) {
        const VT a = reinterpret_cast<const VT *>(w)[v];
        VT b[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) b[q] = reinterpret_cast<const VT *>(V.p[q])[v];
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            if constexpr (sizeof(T) == 4) {
                T leaf = T(0);
#pragma unroll
                for (int e = 0; e < W; ++e) leaf += vget(a, e) * vget(b[q], e);
                acc[q] += (A)leaf;
            } else {
#pragma unroll
                for (int e = 0; e < W; ++e) acc[q] += (A)vget(a, e) * (A)vget(b[q], e);
            }
        }
    }
    for (int64_t c = nv * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < NC; ++q) acc[q] += (A)(w[c] * V.p[q][c]);
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const double t = block_sum<RED_THREADS>(acc[q], sh);
        if (threadIdx.x == 0) part[(size_t)q * gridDim.x + blockIdx.x] = t;
    }
}

// w -= sum_q h_q V_q ; partial (w, w)
template <typename T, int NC>
__global__ void __launch_bounds__(RED_THREADS) k_orth(int64_t n, T *__restrict__ w, VPtrs<T> V, Coef h,
                                                      double *__restrict__ part) {
    typedef typename Acc<T>::type A;
    typedef typename Vec16<T>::type VT;
    constexpr int W = Vec16<T>::W;
    __shared__ double sh[32];
    A ww = A(0);
    const int64_t nv = n / W;
    GRID_STRIDE(v, nv) {
        VT a = reinterpret_cast<const VT *>(w)[v];
        VT b[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) b[q] = reinterpret_cast<const VT *>(V.p[q])[v];
#pragma unroll
        for (int q = 0; q < NC; ++q)
#pragma unroll
            for (int e = 0; e < W; ++e) vset(a, e, vget(a, e) - (T)h.v[q] * vget(b[q], e));
        reinterpret_cast<VT *>(w)[v] = a;
        if constexpr (sizeof(T) == 4) {
            T leaf = T(0);
#pragma unroll
            for (int e = 0; e < W; ++e) leaf += vget(a, e) * vget(a, e);
            ww += (A)leaf;
        } else {
#pragma unroll
            for (int e = 0; e < W; ++e) ww += (A)vget(a, e) * (A)vget(a, e);
        }
    }
    for (int64_t c = nv * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        T a = w[c];
#pragma unroll
        for (int q = 0; q < NC; ++q) a -= (T)h.v[q] * V.p[q][c];
        w[c] = a;
        ww += (A)(a * a);
    }
    const double t = block_sum<RED_THREADS>(ww, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// kernel tables indexed by the column count - 1
template <typename T>
using MdotFn = void (*)(int64_t, const T *, VPtrs<T>, double *);
template <typename T>
using OrthFn = void (*)(int64_t, T *, VPtrs<T>, Coef, double *);
template <typename T, int... I>
static const MdotFn<T> *mdot_table(std::integer_sequence<int, I...>) {
    static const MdotFn<T> t[] = {&k_mdot<T, I + 1>...};
    return t;
}
template <typename T, int... I>
static const OrthFn<T> *orth_table(std::integer_sequence<int, I...>) {
    static const OrthFn<T> t[] = {&k_orth<T, I + 1>...};
    return t;
}

// dst = a src. FP32 to FP32 in FP32 arithmetic, four elements per 16-byte
// access (per-element FP64 arithmetic makes an FP32 stream FP64-bound)
__device__ __forceinline__ void scale_f32(int64_t n, float *__restrict__ dst, const float *__restrict__ src,
                                          float a) {
    GRID_STRIDE(q, n / 4) {
        float4 v = reinterpret_cast<const float4 *>(src)[q];
        v.x *= a;
        v.y *= a;
        v.z *= a;
        v.w *= a;
        reinterpret_cast<float4 *>(dst)[q] = v;
    }
    for (int64_t c = n / 4 * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
        dst[c] = a * src[c];
}

// grid of the multi-dot: each block ends with one FP64 tree sum per column,
// which on GB300's FP64 pipe costs about as much as a few hundred elements, so
// the FP64 kernel takes half the usual blocks (each thread streams twice the
// elements)
template <typename T>
static unsigned mdot_blocks(const Ctx *c) { return sizeof(T) == 8 ? (unsigned)((c->nred + 1) / 2) : (unsigned)c->nred; }

template <typename T, typename S>
__global__ void k_scale(int64_t n, T *__restrict__ dst, const S *__restrict__ src, double a) {
    if constexpr (sizeof(T) == 4 && sizeof(S) == 4) scale_f32(n, dst, src, (float)a);
    else GRID_STRIDE(c, n) dst[c] = (T)(a * (double)src[c]);
}

// x += sum_i y_i Z_i
template <typename T>
__global__ void k_xupd(int64_t n, T *__restrict__ x, const T *const *__restrict__ Z, int ncols, Coef y) {
    T yv[17];
#pragma unroll
    for (int q = 0; q < 17; ++q) yv[q] = (T)y.v[q];
    GRID_STRIDE(c, n) {
        T a = x[c];
#pragma unroll
        for (int q = 0; q < 17; ++q)
            if (q < ncols) a += yv[q] * Z[q][c];
        x[c] = a;
    }
}

// phi += a * ((double) d - mean) on FLUID and GHOST cells (FP64 update of the
// outer iterate; the constant part of the correction is discarded)
__global__ void k_add_scaled(int64_t n, const uint8_t *__restrict__ type, double *__restrict__ phi,
                             const float *__restrict__ d, double a, const double *__restrict__ mean) {
    const double m = *mean;
    GRID_STRIDE(c, n) if (type[c] != DEAD) phi[c] += a * ((double)d[c] - m);
}

// FLUID volume-weighted sum of an FP32 vector: FP32 volumes and products,
// leaves of four consecutive cells in FP32, FP64 across leaves, warps and
// blocks
__global__ void k_fluid_volsum32(GridDev g, OpT<float> o, const uint8_t *__restrict__ type,
                                 const float *__restrict__ x, double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    GRID_STRIDE(q, (g.n + 3) / 4) {
        float leaf = 0.f;
        for (int64_t c = 4 * q; c < 4 * q + 4 && c < g.n; ++c) {
            if (type[c] != FLUID) continue;
            int i, j, k;
            split3(g, (uint32_t)c, i, j, k);
            leaf += (o.dx[i] * o.dy[j] * o.dz[k]) * x[c];
        }
        acc += (double)leaf;
    }
    const double t = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// (FP32 vectors: leaves of four consecutive products in FP32, FP64
// per-thread partials, FP64 across warps and blocks)
template <typename T>
__global__ void k_dotT(int64_t n, const T *__restrict__ a, const T *__restrict__ b, double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    if constexpr (sizeof(T) == 4) {
        GRID_STRIDE(q, (n + 3) / 4) {
            T leaf = T(0);
            for (int64_t c = 4 * q; c < 4 * q + 4 && c < n; ++c) leaf += a[c] * b[c];
            acc += (double)leaf;
        }
    } else {
        GRID_STRIDE(c, n) acc += a[c] * b[c];
    }
    const double t = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// ---------------------------------------------------------------------------
// FP64 vector kernels: BiCGStab (scalars live on the device)
// ---------------------------------------------------------------------------

__global__ void k_dot64(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                        double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    GRID_STRIDE(c, n) acc += a[c] * b[c];
    acc = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// beta = (rho1 / rho) (alpha / omega), rho = rho1; flag 1 on breakdown
__global__ void k_bicg_beta(double *s) {
    const double rho1 = s[B_RHO1], rho = s[B_RHO], om = s[B_OMEGA];
    if (!(rho != 0.0) || !(om != 0.0) || !isfinite(rho1)) { s[B_FLAG] = 1.0; s[B_BETA] = 0.0; }
    else s[B_BETA] = (rho1 / rho) * (s[B_ALPHA] / om);
    s[B_RHO] = rho1;
}
__global__ void k_bicg_alpha(double *s) {
    const double den = s[B_DEN];
    if (!(den != 0.0) || !isfinite(den)) { s[B_FLAG] = 1.0; s[B_ALPHA] = 0.0; }
    else s[B_ALPHA] = s[B_RHO] / den;
}
__global__ void k_bicg_omega(double *s) {
    const double tt = s[B_TT];
    s[B_OMEGA] = (tt > 0.0 && isfinite(tt)) ? s[B_TS] / tt : 0.0;
    if (!(s[B_OMEGA] != 0.0)) s[B_FLAG] = 1.0;
}
__global__ void k_bicg_init(double *s) {
    s[B_RHO] = 1.0;
    s[B_ALPHA] = 1.0;
    s[B_OMEGA] = 1.0;
    s[B_FLAG] = 0.0;
}

// p = r + beta (p - omega v)
__global__ void k_bicg_p(int64_t n, const double *__restrict__ r, double *__restrict__ p,
                         const double *__restrict__ v, const double *__restrict__ s) {
    const double be = s[B_BETA], om = s[B_OMEGA];
    GRID_STRIDE(c, n) p[c] = r[c] + be * (p[c] - om * v[c]);
}
// sv = r - alpha v
__global__ void k_bicg_s(int64_t n, const double *__restrict__ r, const double *__restrict__ v,
                         double *__restrict__ sv, const double *__restrict__ s) {
    const double al = s[B_ALPHA];
    GRID_STRIDE(c, n) sv[c] = r[c] - al * v[c];
}
// partial (t, s) and (t, t)
__global__ void k_bicg_tdots(int64_t n, const double *__restrict__ t, const double *__restrict__ sv,
                             double *__restrict__ part) {
    __shared__ double sh[32];
    double ts = 0.0, tt = 0.0;
    GRID_STRIDE(c, n) {
        const double a = t[c];
        ts += a * sv[c];
        tt += a * a;
    }
    ts = block_sum<RED_THREADS>(ts, sh);
    tt = block_sum<RED_THREADS>(tt, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ts;
        part[gridDim.x + blockIdx.x] = tt;
    }
}
// x += alpha ph + omega sh ; r = sv - omega t ; partial (r, r)
__global__ void k_bicg_xr(int64_t n, double *__restrict__ x, const double *__restrict__ ph,
                          const double *__restrict__ sh_, double *__restrict__ r, const double *__restrict__ sv,
                          const double *__restrict__ t, const double *__restrict__ s, double *__restrict__ part) {
    __shared__ double sh[32];
    const double al = s[B_ALPHA], om = s[B_OMEGA];
    double rr = 0.0;
    GRID_STRIDE(c, n) {
        x[c] += al * ph[c] + om * sh_[c];
        const double v = sv[c] - om * t[c];
        r[c] = v;
        rr += v * v;
    }
    rr = block_sum<RED_THREADS>(rr, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = rr;
}

// ---------------------------------------------------------------------------
// multigrid on the staircase operator, precision T
// ---------------------------------------------------------------------------

// quotient for the FP32 finest-level smoother (CUDA's approximate division
// intrinsic; the operands are positive sums of face coefficients, far from
// its 2^126 limit); FP64 keeps the correctly rounded division
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }

// over-relaxed update o + w (q - o), rounded in a fixed way (no contraction
// left to the compiler, so every kernel that relaxes a cell gives its bits)
__device__ __forceinline__ float relax(float o, float q, float w) { return __fmaf_rn(w, __fsub_rn(q, o), o); }
__device__ __forceinline__ double relax(double o, double q, double w) { return __fma_rn(w, __dsub_rn(q, o), o); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }

// v > 0 for the non-negative tables pn and dinv: an integer test of the bit
// pattern for FP64 (an FP64 compare occupies GB300's slow FP64 pipe; -0 and
// +0 both read as not positive)
__device__ __forceinline__ bool pos(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool pos(float v) { return v > 0.f; }

// sum over the open faces of T_f x_nb, and the diagonal sum T_f, at cell c
// of a level (FINE: derived from the cell types and 1D metrics)
template <typename T, bool FINE>
__device__ __forceinline__ T k_offdiag(const MGLevel<T> &L, const T *__restrict__ x, int64_t c, int i, int j, int k,
                                       T &d, T s0 = T(0)) {
    const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
    T s = s0;
    if (FINE) {
        d = T(0);
        const unsigned msk = L.omask[c];
        const T ayz = L.wy[j] * L.wz[k], axz = L.wx[i] * L.wz[k], axy = L.wx[i] * L.wy[j];
        T t;
        if (msk & 1u) { t = ayz * L.rhx[i]; d += t; s += t * x[c - 1]; }
        if (msk & 2u) { t = ayz * L.rhx[i + 1]; d += t; s += t * x[c + 1]; }
        if (msk & 4u) { t = axz * L.rhy[j]; d += t; s += t * x[c - sy]; }
        if (msk & 8u) { t = axz * L.rhy[j + 1]; d += t; s += t * x[c + sy]; }
        if (msk & 16u) { t = axy * L.rhz[k]; d += t; s += t * x[c - sz]; }
        if (msk & 32u) { t = axy * L.rhz[k + 1]; d += t; s += t * x[c + sz]; }
    } else {
        if (i > 0) s += L.tx[c] * x[c - 1];
        if (i < L.nx - 1) s += L.tx[c + 1] * x[c + 1];
        if (j > 0) s += L.ty[c] * x[c - sy];
        if (j < L.ny - 1) s += L.ty[c + sy] * x[c + sy];
        if (k > 0) s += L.tz[c] * x[c - sz];
        if (k < L.nz - 1) s += L.tz[c + sz] * x[c + sz];
        d = L.d[c];
    }
    return s;
}

template <typename T, bool FINE>
__device__ __forceinline__ bool active(const MGLevel<T> &L, int64_t c) {
    if (FINE) return (L.omask[c] & 0x80u) != 0;
    return pos(L.dinv[c]);
}

// open-face mask of the finest level
__global__ void k_open_mask(GridDev g, const uint8_t *__restrict__ type, uint8_t *__restrict__ m) {
    GRID_STRIDE(c, g.n) {
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
        unsigned v = 0;
        if (type[c] == FLUID) {
            v = 0x80u;
            if (i > 0 && type[c - 1] == FLUID) v |= 1u;
            if (i < g.nx - 1 && type[c + 1] == FLUID) v |= 2u;
            if (j > 0 && type[c - sy] == FLUID) v |= 4u;
            if (j < g.ny - 1 && type[c + sy] == FLUID) v |= 8u;
            if (g.ndim == 3 && k > 0 && type[c - sz] == FLUID) v |= 16u;
            if (g.ndim == 3 && k < g.nz - 1 && type[c + sz] == FLUID) v |= 32u;
        }
        m[c] = (uint8_t)v;
    }
}

// red-black Gauss-Seidel, one colour: x_c = (f_c + sum T x_nb) / D_c on the
// cells of colour col ((i + j + k) even = 0) with D_c > 0; with OMEGA the
// over-relaxed update x_c += w ((f_c + sum T x_nb) / D_c - x_c)
// (at most 32 registers, so that 2048 threads fit an SM, which the
// latency-bound FP32 pass needs; no spills. The bound admits every block
// size tile_x allows, up to 512 threads.)
template <typename T, bool FINE, bool OMEGA = false>
__global__ void __launch_bounds__(512, 4)
    k_rbgs(MGLevel<T> L, const T *__restrict__ f, T *__restrict__ x, int col, T w = T(1)) {
    const int64_t row = blockIdx.x;
    int j, k;
    row_jk((uint32_t)blockIdx.x, L.fny, L.ny, j, k);
    const int i = 2 * (blockIdx.y * blockDim.x + threadIdx.x) + ((j + k + col) & 1);
    if (i >= L.nx) return;
    const int64_t c = row * L.nx + i;
    if (!active<T, FINE>(L, c)) return;
    T d;
    // the stored-coefficient levels accumulate onto f (one FP64 add fewer)
    const T s = FINE ? f[c] + k_offdiag<T, FINE>(L, x, c, i, j, k, d) : k_offdiag<T, FINE>(L, x, c, i, j, k, d, f[c]);
    if (FINE) {
        // (FP32 only: the approximate quotient, two instructions instead of
        // the correctly rounded division's sequence, in an issue-bound pass)
        if (d > T(0)) {
            const T q = fast_div(s, d);
            x[c] = OMEGA ? relax(x[c], q, w) : q;
        }
    } else {
        x[c] = OMEGA ? relax(x[c], s * L.dinv[c], w) : s * L.dinv[c];
    }
}

// diagonal sum of the open faces at a cell of the finest level (the d of
// k_offdiag<T, true>, summed in the same order)
template <typename T>
__device__ __forceinline__ T fine_diag(const MGLevel<T> &L, unsigned msk, int i, int j, int k) {
    const T ayz = L.wy[j] * L.wz[k], axz = L.wx[i] * L.wz[k], axy = L.wx[i] * L.wy[j];
    T d = T(0);
    if (msk & 1u) d += ayz * L.rhx[i];
    if (msk & 2u) d += ayz * L.rhx[i + 1];
    if (msk & 4u) d += axz * L.rhy[j];
    if (msk & 8u) d += axz * L.rhy[j + 1];
    if (msk & 16u) d += axy * L.rhz[k];
    if (msk & 32u) d += axy * L.rhz[k + 1];
    return d;
}

// The first colour pass of a level, from x = 0: the neighbour sum vanishes,
// so x_c = f_c / D_c (times w) on the active cells of colour col, the same
// value k_rbgs gives, without reading x or the face coefficients. Each
// thread owns the pair of cells (2t, 2t + 1) of its row; with zero_rest it
// writes 0 to the pair's other cell and to inactive cells, in place of
// clearing x beforehand.
template <typename T, bool FINE, bool OMEGA = false>
__global__ void __launch_bounds__(512, 4)
    k_rbgs_first(MGLevel<T> L, const T *__restrict__ f, T *__restrict__ x, int col, T w, int zero_rest) {
    const int64_t row = blockIdx.x;
    int j, k;
    row_jk((uint32_t)blockIdx.x, L.fny, L.ny, j, k);
    const int i0 = 2 * (blockIdx.y * blockDim.x + threadIdx.x);
    if (i0 >= L.nx) return;
    const int par = (j + k + col) & 1;
    const int ic = i0 + par, io = i0 + 1 - par;   // the cell of colour col, the other
    if (zero_rest && io < L.nx) x[row * L.nx + io] = T(0);
    if (ic >= L.nx) return;
    const int64_t c = row * L.nx + ic;
    T v = T(0);
    bool wr = zero_rest != 0;
    if (FINE) {
        const unsigned msk = L.omask[c];
        if (msk & 0x80u) {
            const T d = fine_diag<T>(L, msk, ic, j, k);
            if (d > T(0)) {
                v = OMEGA ? rmul(w, fast_div(f[c], d)) : fast_div(f[c], d);
                wr = true;
            }
        }
    } else if (active<T, false>(L, c)) {
        v = OMEGA ? w * (f[c] * L.dinv[c]) : f[c] * L.dinv[c];
        wr = true;
    }
    if (wr) x[c] = v;
}

// ---------------------------------------------------------------------------
// Level 0 in colour-split storage (FP32 fine variant)
// ---------------------------------------------------------------------------
//
// The cells of colour q of row (j, k) sit at packed index h = i >> 1 of row
// j + ny k in array q (H = nx / 2 packed cells per row; nx a multiple of 8,
// so a packed row is a whole number of 16-byte quads). The cell at packed h
// has i = 2h + pc, pc = (q + j + k) & 1, and all six neighbours have the
// other colour: x - 1 at packed h - 1 + pc and x + 1 at h + pc of the same
// row, the y and z neighbours at h of the neighbouring rows. A colour pass
// then reads the other colour's x once (s/2 per cell), its own f (s/2) and
// mask byte (1/2) and writes its own x (s/2): the method's minimum, where
// the cell-ordered pass moves whole 32-byte sectors of both colours.
//
// A thread updates one quad (four consecutive packed cells of one colour)
// with 16-byte accesses: the other colour's quad of the same row and one
// edge value give both x neighbours, one quad per y and z neighbour row.
// Each cell evaluates the expression of k_offdiag<float, true> in its
// order, so results equal the cell-ordered kernels bit for bit.

template <typename T>
struct SplitLv {
    int nx, ny, nz, H;   // H = nx / 2
    FastDiv fq, fny;     // division by the quads per packed row (H / 4) and by ny
    int64_t nq;          // quads per colour
    const T *wy, *wz, *rhy, *rhz;
    const T *swx0, *swx1, *srm0, *srm1, *srp0, *srp1;   // per row offset pc (see MGHier)
};

template <typename T>
static SplitLv<T> split_of(const MGHier<T> &H) {
    const MGLevel<T> &L = H.lv[0];
    SplitLv<T> s;
    s.nx = L.nx;
    s.ny = L.ny;
    s.nz = L.nz;
    s.H = L.nx / 2;
    s.fq = FastDiv((uint32_t)(L.nx / 8));
    s.fny = FastDiv((uint32_t)L.ny);
    s.nq = L.n / 8;
    s.wy = H.wy;
    s.wz = H.wz;
    s.rhy = H.rhy;
    s.rhz = H.rhz;
    s.swx0 = H.swx[0]; s.swx1 = H.swx[1];
    s.srm0 = H.srm[0]; s.srm1 = H.srm[1];
    s.srp0 = H.srp[0]; s.srp1 = H.srp[1];
    return s;
}

__device__ __forceinline__ float f4at(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

// quad q of a colour: packed row, first packed index, (j, k)
__device__ __forceinline__ void split_quad_pos(const SplitLv<float> &L, int64_t q, int64_t &base, int &h0, int &j,
                                               int &k) {
    const uint32_t row = L.fq.div((uint32_t)q);
    h0 = 4 * (int)((uint32_t)q - row * (uint32_t)(L.H / 4));
    row_jk(row, L.fny, L.ny, j, k);
    base = (int64_t)row * L.H + h0;
}

// the other colour's values a quad needs: its own row's quad O and the edge
// value xe (x - 1 of cell 0 for pc = 0, x + 1 of cell 3 for pc = 1), and the
// quads of the y and z neighbour rows (O where there is no row: unused, the
// mask has no open face there). All loads are issued together.
struct QuadNb {
    float4 O, ym, yp, zm, zp;
    float xe;
};

__device__ __forceinline__ QuadNb split_loads(const SplitLv<float> &L, const float *__restrict__ xo, int64_t base,
                                              int h0, int j, int k, int pc) {
    const int64_t sy = L.H, sz = (int64_t)L.H * L.ny;
    QuadNb q;
    q.O = ld4(xo + base);
    const int64_t ie = pc == 0 ? base - 1 : base + 4;
    const bool he = pc == 0 ? h0 > 0 : h0 + 4 < L.H;
    q.xe = he ? xo[ie] : 0.f;
    q.ym = ld4(xo + (j > 0 ? base - sy : base));
    q.yp = ld4(xo + (j < L.ny - 1 ? base + sy : base));
    q.zm = ld4(xo + (L.nz > 1 && k > 0 ? base - sz : base));
    q.zp = ld4(xo + (L.nz > 1 && k < L.nz - 1 ? base + sz : base));
    return q;
}

// sum over the open faces of T_f x_nb and the face sum d for the four cells
// of a quad (the order and operations of k_offdiag<float, true>)
__device__ __forceinline__ void split_offdiag(const SplitLv<float> &L, const QuadNb &N, int h0, int j, int k,
                                              int pc, uchar4 m4, float s[4], float d[4]) {
    // the 1D metrics are small arrays (L1 hits), read per cell as needed so
    // they hold no registers across the loop
    const float *swx = (pc ? L.swx1 : L.swx0) + h0, *srm = (pc ? L.srm1 : L.srm0) + h0;
    const float *srp = (pc ? L.srp1 : L.srp0) + h0;
    const float wyj = L.wy[j], wzk = L.wz[k], ry0 = L.rhy[j], ry1 = L.rhy[j + 1], rz0 = L.rhz[k], rz1 = L.rhz[k + 1];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const unsigned msk = e == 0 ? m4.x : e == 1 ? m4.y : e == 2 ? m4.z : m4.w;
        const float xm = pc ? f4at(N.O, e) : (e == 0 ? N.xe : f4at(N.O, e - 1));
        const float xp = pc ? (e == 3 ? N.xe : f4at(N.O, e + 1)) : f4at(N.O, e);
        const float wxe = swx[e];
        const float ayz = wyj * wzk, axz = wxe * wzk, axy = wxe * wyj;
        float dd = 0.f, ss = 0.f, t;
        if (msk & 1u) { t = ayz * srm[e]; dd += t; ss += t * xm; }
        if (msk & 2u) { t = ayz * srp[e]; dd += t; ss += t * xp; }
        if (msk & 4u) { t = axz * ry0; dd += t; ss += t * f4at(N.ym, e); }
        if (msk & 8u) { t = axz * ry1; dd += t; ss += t * f4at(N.yp, e); }
        if (msk & 16u) { t = axy * rz0; dd += t; ss += t * f4at(N.zm, e); }
        if (msk & 32u) { t = axy * rz1; dd += t; ss += t * f4at(N.zp, e); }
        s[e] = ss;
        d[e] = dd;
    }
}

// One colour pass (colour col, other colour's x in xo) on level 0 in split
// storage; cells that are not updated keep their value. With NAT the pass is
// the last of the V-cycle: instead of xq it writes the cell-ordered output
// xn (both colours: this colour's new values, the other colour's from xo).
// Every load of a quad is issued before the first use, so a thread waits
// for memory once.
template <bool OMEGA, bool NAT>
__global__ void __launch_bounds__(256, 5)
    k_rbgs_split(SplitLv<float> L, const float *__restrict__ fq, const uint8_t *__restrict__ mq,
                 const float *__restrict__ xo, float *__restrict__ xq, int col, float w, float *__restrict__ xn) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= L.nq) return;
    int64_t base;
    int h0, j, k;
    split_quad_pos(L, q, base, h0, j, k);
    const int pc = (col + j + k) & 1;
    const uchar4 m4 = *reinterpret_cast<const uchar4 *>(mq + base);
    const float4 f4 = ld4(fq + base);
    const QuadNb N = split_loads(L, xo, base, h0, j, k, pc);
    float4 old = make_float4(0.f, 0.f, 0.f, 0.f);
    if (OMEGA) old = ld4(xq + base);
    const unsigned any = (m4.x | m4.y | m4.z | m4.w) & 0x80u;
    if (!NAT && !any) return;   // no active cell: nothing changes
    float sv[4], dv[4];
    split_offdiag(L, N, h0, j, k, pc, m4, sv, dv);
    float v[4];
    bool up[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const unsigned msk = e == 0 ? m4.x : e == 1 ? m4.y : e == 2 ? m4.z : m4.w;
        const float s = f4at(f4, e) + sv[e];
        up[e] = (msk & 0x80u) && dv[e] > 0.f;
        v[e] = up[e] ? fast_div(s, dv[e]) : 0.f;
    }
    const bool all = up[0] && up[1] && up[2] && up[3];
    if (OMEGA || !all) {
        // the old values: the relaxation needs them, and cells not updated keep them
        if (!OMEGA) old = ld4(xq + base);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float o = f4at(old, e);
            v[e] = up[e] ? (OMEGA ? relax(o, v[e], w) : v[e]) : o;
        }
    }
    if (NAT) {
        // cell i = 2 h + pc of this colour, 2 h + 1 - pc of the other
        float a[8];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            a[2 * e + pc] = v[e];
            a[2 * e + 1 - pc] = f4at(N.O, e);
        }
        float *dst = xn + base * 2;   // cell 2 h0 of the row (2 H = nx)
        *reinterpret_cast<float4 *>(dst) = make_float4(a[0], a[1], a[2], a[3]);
        *reinterpret_cast<float4 *>(dst + 4) = make_float4(a[4], a[5], a[6], a[7]);
    } else {
        *reinterpret_cast<float4 *>(xq + base) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// The first pass of a V-cycle on level 0 in split storage, from x = 0:
// splits the cell-ordered right-hand side f0 into fs (both colours), writes
// colour 0 as x = f / D (times w) on active cells with open faces and 0
// elsewhere, and colour 1 as 0 (the values and zeros k_rbgs_first writes).
template <bool OMEGA>
__global__ void __launch_bounds__(256)
    k_rbgs_first_split(SplitLv<float> L, const float *__restrict__ f0, const uint8_t *__restrict__ m0,
                       float *__restrict__ fs0, float *__restrict__ fs1, float *__restrict__ xs0,
                       float *__restrict__ xs1, float w) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= L.nq) return;
    int64_t base;
    int h0, j, k;
    split_quad_pos(L, q, base, h0, j, k);
    const int pc = (j + k) & 1;   // colour 0's offset in this row
    const float *src = f0 + base * 2;   // cells 2 h0 .. 2 h0 + 7 of the row (2 base = row nx + 2 h0)
    const float4 a = ld4(src), b = ld4(src + 4);
    const float n8[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    float c0[4], c1[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        c0[e] = n8[2 * e + pc];
        c1[e] = n8[2 * e + 1 - pc];
    }
    *reinterpret_cast<float4 *>(fs0 + base) = make_float4(c0[0], c0[1], c0[2], c0[3]);
    *reinterpret_cast<float4 *>(fs1 + base) = make_float4(c1[0], c1[1], c1[2], c1[3]);
    const uchar4 m4 = *reinterpret_cast<const uchar4 *>(m0 + base);
    const float4 wx4 = ld4((pc ? L.swx1 : L.swx0) + h0);
    const float4 rm4 = ld4((pc ? L.srm1 : L.srm0) + h0);
    const float4 rp4 = ld4((pc ? L.srp1 : L.srp0) + h0);
    const float wyj = L.wy[j], wzk = L.wz[k], ry0 = L.rhy[j], ry1 = L.rhy[j + 1], rz0 = L.rhz[k], rz1 = L.rhz[k + 1];
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const unsigned msk = e == 0 ? m4.x : e == 1 ? m4.y : e == 2 ? m4.z : m4.w;
        v[e] = 0.f;
        if (msk & 0x80u) {
            // fine_diag's sum, in its order
            const float wxe = f4at(wx4, e);
            const float ayz = wyj * wzk, axz = wxe * wzk, axy = wxe * wyj;
            float d = 0.f;
            if (msk & 1u) d += ayz * f4at(rm4, e);
            if (msk & 2u) d += ayz * f4at(rp4, e);
            if (msk & 4u) d += axz * ry0;
            if (msk & 8u) d += axz * ry1;
            if (msk & 16u) d += axy * rz0;
            if (msk & 32u) d += axy * rz1;
            if (d > 0.f) v[e] = OMEGA ? rmul(w, fast_div(c0[e], d)) : fast_div(c0[e], d);
        }
    }
    *reinterpret_cast<float4 *>(xs0 + base) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4 *>(xs1 + base) = make_float4(0.f, 0.f, 0.f, 0.f);
}

// cell-ordered x from the two split colours (a V-cycle without post-smoothing)
__global__ void k_split_merge(SplitLv<float> L, const float *__restrict__ xs0, const float *__restrict__ xs1,
                              float *__restrict__ xn) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= L.nq) return;
    int64_t base;
    int h0, j, k;
    split_quad_pos(L, q, base, h0, j, k);
    const int pc = (j + k) & 1;
    const float4 a = ld4(xs0 + base), b = ld4(xs1 + base);
    float o[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        o[2 * e + pc] = f4at(a, e);
        o[2 * e + 1 - pc] = f4at(b, e);
    }
    float *dst = xn + base * 2;
    *reinterpret_cast<float4 *>(dst) = make_float4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<float4 *>(dst + 4) = make_float4(o[4], o[5], o[6], o[7]);
}

// per-colour copies of the level-0 open-face mask
__global__ void k_split_mask(SplitLv<float> L, const uint8_t *__restrict__ m, uint8_t *__restrict__ m0,
                             uint8_t *__restrict__ m1) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= L.nq) return;
    int64_t base;
    int h0, j, k;
    split_quad_pos(L, q, base, h0, j, k);
    const int pc = (j + k) & 1;
    const uint8_t *src = m + base * 2;
    uint8_t a[4], b[4];
    for (int e = 0; e < 4; ++e) {
        a[e] = src[2 * e + pc];
        b[e] = src[2 * e + 1 - pc];
    }
    *reinterpret_cast<uchar4 *>(m0 + base) = make_uchar4(a[0], a[1], a[2], a[3]);
    *reinterpret_cast<uchar4 *>(m1 + base) = make_uchar4(b[0], b[1], b[2], b[3]);
}

// coarse f_C = sum over children of (f - K x); coarse x_C = 0
template <typename T, bool FINE>
__global__ void k_resid_restrict(MGLevel<T> L, const T *__restrict__ f, const T *__restrict__ x, MGLevel<T> C,
                                 int fx, int fy, int fz) {
    const int64_t row = blockIdx.x;
    int J, K;
    row_jk((uint32_t)blockIdx.x, C.fny, C.ny, J, K);
    const int I = blockIdx.y * blockDim.x + threadIdx.x;
    if (I >= C.nx) return;
    T acc = T(0);
    for (int dk = 0; dk < fz; ++dk) {
        const int k = fz * K + dk;
        if (k >= L.nz) break;
        for (int dj = 0; dj < fy; ++dj) {
            const int j = fy * J + dj;
            if (j >= L.ny) break;
            for (int di = 0; di < fx; ++di) {
                const int i = fx * I + di;
                if (i >= L.nx) break;
                const int64_t c = ((int64_t)k * L.ny + j) * L.nx + i;
                if (!active<T, FINE>(L, c)) continue;
                T d;
                const T off = k_offdiag<T, FINE>(L, x, c, i, j, k, d);
                acc += f[c] - (d * x[c] - off);
            }
        }
    }
    const int64_t cc = row * C.nx + I;
    C.f[cc] = acc;
    C.x[cc] = T(0);
}

// x_c += x_parent(c) on active cells
template <typename T, bool FINE>
__global__ void k_prolong(MGLevel<T> L, T *__restrict__ x, MGLevel<T> C, int fx, int fy, int fz) {
    const int64_t row = blockIdx.x;
    int j, k;
    row_jk((uint32_t)blockIdx.x, L.fny, L.ny, j, k);
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= L.nx) return;
    const int64_t c = row * L.nx + i;
    if (!active<T, FINE>(L, c)) return;
    const int64_t p = ((int64_t)(k / fz) * C.ny + (j / fy)) * C.nx + (i / fx);
    x[c] += C.x[p];
}

// trilinear transfer ----------------------------------------------------------
//
// Prolongation P interpolates each fine cell from the (up to) 2x2x2 coarse
// cells around it with separable linear weights, renormalised over the
// active coarse cells (pn); restriction is its transpose. Both are applied
// one axis at a time, which needs a few multiply-adds per fine cell instead
// of one per (fine cell, coarse cell) pair.

template <typename T>
struct Xfer {
    const int *Ix, *Jx, *Iy, *Jy, *Iz, *Jz;   // scatter: fine index -> coarse
    const T *wx, *wy, *wz;                    // weight of coarse I
    const int *Gx, *Gy, *Gz;                  // gather: coarse index -> 4 fine
    const T *gwx, *gwy, *gwz;
    const T *vx, *vy, *vz;                    // weight of coarse J (1 - w)
};

// the up-to-two coarse indices and weights of fine index i along one axis
template <typename T>
__device__ __forceinline__ int xfer_axis(const int *I, const int *J, const T *w, const T *v, int i, int *idx,
                                         T *wt) {
    idx[0] = I[i];
    wt[0] = w[i];
    if (J[i] >= 0) {
        idx[1] = J[i];
        wt[1] = v[i];
        return 2;
    }
    return 1;
}

// pn_c = 1 / (sum of the weights of the active coarse cells of c), 0 if c inactive
template <typename T, bool FINE>
__global__ void k_pnorm(MGLevel<T> L, MGLevel<T> C, Xfer<T> X, T *__restrict__ pn) {
    const int64_t row = blockIdx.x;
    int j, k;
    row_jk((uint32_t)blockIdx.x, L.fny, L.ny, j, k);
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= L.nx) return;
    const int64_t c = row * L.nx + i;
    if (!active<T, FINE>(L, c)) { pn[c] = T(0); return; }
    int ia[2], ib[2], ic[2];
    T wa[2], wb[2], wc[2];
    const int na = xfer_axis(X.Ix, X.Jx, X.wx, X.vx, i, ia, wa);
    const int nb = xfer_axis(X.Iy, X.Jy, X.wy, X.vy, j, ib, wb);
    const int nc = xfer_axis(X.Iz, X.Jz, X.wz, X.vz, k, ic, wc);
    T sum = T(0);
    for (int q3 = 0; q3 < nc; ++q3)
        for (int q2 = 0; q2 < nb; ++q2)
            for (int q1 = 0; q1 < na; ++q1) {
                const int64_t cc = ((int64_t)ic[q3] * C.ny + ib[q2]) * C.nx + ia[q1];
                if (C.dinv[cc] > T(0)) sum += (wa[q1] * wb[q2]) * wc[q3];
            }
    pn[c] = sum > T(0) ? T(1) / sum : T(0);
}

// Restriction, first axis, fused with the fine residual: for one fine row
// (j, k) and RX_THREADS coarse x-indices I,
//   tA[I + cnx (j + ny k)] = sum_s gwx[4I+s] * (pn r)(gIx[4I+s], j, k),
// r = f - K x. The block computes pn r for the fine cells its coarse cells
// gather from (two more than twice their number when x is coarsened) into
// shared memory, then each thread sums its four. zcol >= 0 names the colour
// the smoother relaxed last: the residual of every cell it updated is zero
// (up to rounding) and is taken as zero without evaluating the stencil.
constexpr int RX_THREADS = 128;
template <typename T, bool FINE>
__global__ void __launch_bounds__(RX_THREADS)
    k_resid_rx(MGLevel<T> L, const T *__restrict__ f, const T *__restrict__ x, const T *__restrict__ pn, Xfer<T> X,
               int cnx, int fx, int zcol, T *__restrict__ tA) {
    __shared__ T sg[2 * RX_THREADS + 2];
    const int64_t row = blockIdx.x;
    int j, k;
    row_jk((uint32_t)blockIdx.x, L.fny, L.ny, j, k);
    const int I0 = blockIdx.y * RX_THREADS;
    const int lo = fx == 2 ? 2 * I0 - 1 : I0;
    const int cnt = fx == 2 ? 2 * RX_THREADS + 2 : RX_THREADS;
    // pn r at fine cell lo + t (0 outside the row)
    auto pr = [&](int t) -> T {
        const int i = lo + t;
        if (i < 0 || i >= L.nx) return T(0);
        const int64_t c = row * L.nx + i;
        const T p = pn[c];
        if (!pos(p)) return T(0);
        T d;
        // r = (f + sum T x_nb) - D x, accumulated onto f
        const T s = k_offdiag<T, FINE>(L, x, c, i, j, k, d, f[c]);
        return p * (s - d * x[c]);
    };
    if (!FINE && zcol >= 0) {
        // The lanes of a warp take cells of one colour, so that the skipped
        // colour leaves no idle lanes in the warps that evaluate the other
        // (with alternating colours per lane every warp paid the full
        // stencil: on GB300's FP64 pipe that doubled the cost).
        const int r0 = ((lo + j + k) & 1) == zcol ? 0 : 1;   // first relaxed slot
        for (int u = threadIdx.x; 2 * u + (1 - r0) < cnt; u += RX_THREADS) {
            const int t = 2 * u + (1 - r0);
            sg[t] = pr(t);
        }
        for (int u = threadIdx.x; 2 * u + r0 < cnt; u += RX_THREADS) sg[2 * u + r0] = T(0);
    } else {
        // the finest FP32 level (latency-bound, not pipe-bound) keeps one
        // slot per lane: the colour split cost it registers and warps. A
        // relaxed cell is skipped only if it has an open face (it was updated).
        for (int t = threadIdx.x; t < cnt; t += RX_THREADS) {
            const int i = lo + t;
            const bool relaxed = FINE && ((i + j + k) & 1) == zcol && i >= 0 && i < L.nx &&
                                 (L.omask[row * L.nx + i] & 0x3fu) != 0;
            sg[t] = relaxed ? T(0) : pr(t);
        }
    }
    __syncthreads();
    const int I = I0 + threadIdx.x;
    if (I < cnx) {
        T acc = T(0);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int i = X.Gx[4 * I + s];
            if (i >= 0 && (unsigned)(i - lo) < (unsigned)cnt) acc += X.gwx[4 * I + s] * sg[i - lo];
        }
        tA[row * cnx + I] = acc;
    }
}

// Restriction, second and third axes: f_C = sum_z gwz sum_y gwy tA (tA has
// the coarse x extent and the fine y, z extents); x_C = 0, and f_C = 0 on
// inactive coarse cells.
template <typename T>
__global__ void k_restrict_yz(MGLevel<T> C, const T *__restrict__ tA, int fny, Xfer<T> X) {
    const int64_t row = blockIdx.x;
    int Jc, Kc;
    row_jk((uint32_t)blockIdx.x, C.fny, C.ny, Jc, Kc);
    const int Ic = blockIdx.y * blockDim.x + threadIdx.x;
    if (Ic >= C.nx) return;
    const int64_t cc = row * C.nx + Ic;
    C.x[cc] = T(0);
    if (!pos(C.dinv[cc])) { C.f[cc] = T(0); return; }
    T acc = T(0);
#pragma unroll
    for (int s3 = 0; s3 < 4; ++s3) {
        const int k = X.Gz[4 * Kc + s3];
        if (k < 0) continue;
        T a2 = T(0);
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2) {
            const int j = X.Gy[4 * Jc + s2];
            if (j >= 0) a2 += X.gwy[4 * Jc + s2] * tA[((int64_t)k * fny + j) * C.nx + Ic];
        }
        acc += X.gwz[4 * Kc + s3] * a2;
    }
    C.f[cc] = acc;
}

// Prolongation, first axis: tB[i + fnx (J + cny K)] = the x-interpolation of
// coarse row (J, K) at fine index i. Coarse x is zero on inactive coarse
// cells (restriction clears it, smoothing and the coarse solve write only
// active cells), so no mask is needed here.
template <typename T>
__global__ void k_prolong_x(int fnx, MGLevel<T> C, Xfer<T> X, T *__restrict__ tB) {
    const int64_t row = blockIdx.x;
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= fnx) return;
    const T *xr = C.x + row * C.nx;
    const int J2 = X.Jx[i];
    T v = X.wx[i] * xr[X.Ix[i]];
    if (J2 >= 0) v += X.vx[i] * xr[J2];
    tB[row * fnx + i] = v;
}

// Prolongation, second and third axes, and the correction:
// x_c += pn_c * sum_z wz sum_y wy tB on fine cells with pn_c > 0
template <typename T>
__global__ void k_prolong_yz(MGLevel<T> L, T *__restrict__ x, const T *__restrict__ tB, int cny, Xfer<T> X,
                             const T *__restrict__ pn) {
    const int64_t row = blockIdx.x;
    int j, k;
    row_jk((uint32_t)blockIdx.x, L.fny, L.ny, j, k);
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= L.nx) return;
    const int64_t c = row * L.nx + i;
    // pn, x and the (up to four) tB values are loaded together; the
    // interpolation indices depend on the row only
    int ib[2], ic[2];
    T wb[2], wc[2];
    const int nb = xfer_axis(X.Iy, X.Jy, X.wy, X.vy, j, ib, wb);
    const int nc = xfer_axis(X.Iz, X.Jz, X.wz, X.vz, k, ic, wc);
    T tv[2][2];
#pragma unroll
    for (int q3 = 0; q3 < 2; ++q3)
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
            tv[q3][q2] = tB[((int64_t)ic[q3 < nc ? q3 : 0] * cny + ib[q2 < nb ? q2 : 0]) * L.nx + i];
    const T p = pn[c];
    const T xc = x[c];
    if (!pos(p)) return;
    T acc = T(0);
    for (int q3 = 0; q3 < nc; ++q3) {
        T a2 = T(0);
        for (int q2 = 0; q2 < nb; ++q2) a2 += wb[q2] * tv[q3][q2];
        acc += wc[q3] * a2;
    }
    x[c] = xc + acc * p;
}

// k_resid_rx on level 0 in colour-split storage (x and f split; the mask and
// pn cell-ordered): the same cells, values and order of evaluation
__global__ void __launch_bounds__(RX_THREADS)
    k_resid_rx_split(MGLevel<float> L, const float *__restrict__ fs0, const float *__restrict__ fs1,
                     const float *__restrict__ xs0, const float *__restrict__ xs1, const float *__restrict__ pn,
                     Xfer<float> X, int cnx, int fx, int zcol, float *__restrict__ tA) {
    __shared__ float sg[2 * RX_THREADS + 2];
    const int64_t row = blockIdx.x;
    int j, k;
    row_jk((uint32_t)blockIdx.x, L.fny, L.ny, j, k);
    const int H = L.nx / 2;
    const int64_t prow = row * H, sy = H, sz = (int64_t)H * L.ny;
    const int I0 = blockIdx.y * RX_THREADS;
    const int lo = fx == 2 ? 2 * I0 - 1 : I0;
    const int cnt = fx == 2 ? 2 * RX_THREADS + 2 : RX_THREADS;
    for (int t = threadIdx.x; t < cnt; t += RX_THREADS) {
        const int i = lo + t;
        float r = 0.f;
        if (i >= 0 && i < L.nx) {
            const int64_t c = row * L.nx + i;
            const unsigned msk = L.omask[c];
            const int col = (i + j + k) & 1;
            const bool relaxed = col == zcol && (msk & 0x3fu) != 0;
            const float p = pn[c];
            if (!relaxed && p > 0.f) {
                const float *xo = col ? xs0 : xs1;
                const int64_t pb = prow + (i >> 1);
                const float ayz = L.wy[j] * L.wz[k], axz = L.wx[i] * L.wz[k], axy = L.wx[i] * L.wy[j];
                float d = 0.f, s = (col ? fs1 : fs0)[pb], tt;
                if (msk & 1u) { tt = ayz * L.rhx[i]; d += tt; s += tt * xo[prow + ((i - 1) >> 1)]; }
                if (msk & 2u) { tt = ayz * L.rhx[i + 1]; d += tt; s += tt * xo[prow + ((i + 1) >> 1)]; }
                if (msk & 4u) { tt = axz * L.rhy[j]; d += tt; s += tt * xo[pb - sy]; }
                if (msk & 8u) { tt = axz * L.rhy[j + 1]; d += tt; s += tt * xo[pb + sy]; }
                if (msk & 16u) { tt = axy * L.rhz[k]; d += tt; s += tt * xo[pb - sz]; }
                if (msk & 32u) { tt = axy * L.rhz[k + 1]; d += tt; s += tt * xo[pb + sz]; }
                r = p * (s - d * (col ? xs1 : xs0)[pb]);
            }
        }
        sg[t] = r;
    }
    __syncthreads();
    const int I = I0 + threadIdx.x;
    if (I < cnx) {
        float acc = 0.f;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int i = X.Gx[4 * I + s];
            if (i >= 0 && (unsigned)(i - lo) < (unsigned)cnt) acc += X.gwx[4 * I + s] * sg[i - lo];
        }
        tA[row * cnx + I] = acc;
    }
}

// k_resid_rx on level 0 in colour-split storage when x is coarsened by two
// (nx a multiple of 8): one thread per four coarse x-cells I0 .. I0 + 3 of a
// row. Coarse I gathers fine cells 2I - 1 .. 2I + 2, so the thread evaluates
// pn r on the ten fine cells 2 I0 - 1 .. 2 I0 + 8 (the two outer ones also by
// its neighbours) with 16-byte loads: the colour relaxed last (1) has zero
// residual where it has an open face and p f where it has none; colour 0
// takes the full stencil, in the order and operations of k_resid_rx. The
// restriction then sums in the gather table's order, so the result equals
// k_resid_rx bit for bit.
__global__ void __launch_bounds__(256)
    k_resid_rx_split4(MGLevel<float> L, SplitLv<float> S, const float *__restrict__ fs0, const float *__restrict__ fs1,
                      const float *__restrict__ xs0, const float *__restrict__ xs1, const float *__restrict__ pn,
                      Xfer<float> X, float *__restrict__ tA) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= S.nq) return;
    const int H = S.H, nx = L.nx;
    const uint32_t rw = S.fq.div((uint32_t)q);
    const int I0 = 4 * (int)((uint32_t)q - rw * (uint32_t)(H / 4));   // packed quad h0 = I0 (H = coarse nx)
    int j, k;
    row_jk(rw, S.fny, S.ny, j, k);
    const int64_t row = rw, base = row * H + I0, crow = row * nx;
    const int pc0 = (j + k) & 1;             // colour 0 sits at i = 2 h + pc0
    const int64_t sy = H, sz = (int64_t)H * L.ny;
    const int i0 = 2 * I0 - 1;               // first fine cell of the window
    // colour 0 of the window: packed I0 - pc0 .. I0 + 4 - pc0 = the quad at
    // I0 and one edge cell he
    const float4 x0q = ld4(xs0 + base), f0q = ld4(fs0 + base);
    const int he = pc0 ? I0 - 1 : I0 + 4;
    const bool heok = he >= 0 && he < H;
    const int64_t be = row * H + (heok ? he : I0);
    const float x0e = heok ? xs0[be] : 0.f, f0e = heok ? fs0[be] : 0.f;
    // colour 1: packed I0 - 1 .. I0 + 4 of the row (x neighbours), and the
    // y / z rows at the colour-0 cells' packed indices
    const float4 c1q = ld4(xs1 + base);
    const float c1m = I0 > 0 ? xs1[base - 1] : 0.f, c1p = I0 + 4 < H ? xs1[base + 4] : 0.f;
    const float4 ymq = ld4(xs1 + (j > 0 ? base - sy : base)), ypq = ld4(xs1 + (j < L.ny - 1 ? base + sy : base));
    const float yme = (j > 0 && heok) ? xs1[be - sy] : 0.f, ype = (j < L.ny - 1 && heok) ? xs1[be + sy] : 0.f;
    float4 zmq = c1q, zpq = c1q;
    float zme = 0.f, zpe = 0.f;
    if (L.nz > 1) {
        if (k > 0) {
            zmq = ld4(xs1 + base - sz);
            if (heok) zme = xs1[be - sz];
        }
        if (k < L.nz - 1) {
            zpq = ld4(xs1 + base + sz);
            if (heok) zpe = xs1[be + sz];
        }
    }
    // cell-ordered pn and open-face mask of the window
    const float4 pA = ld4(pn + crow + 2 * I0), pB = ld4(pn + crow + 2 * I0 + 4);
    const float pm = I0 > 0 ? pn[crow + i0] : 0.f, pp = 2 * I0 + 8 < nx ? pn[crow + 2 * I0 + 8] : 0.f;
    const uint2 mm = *reinterpret_cast<const uint2 *>(L.omask + crow + 2 * I0);
    const unsigned mlo = I0 > 0 ? L.omask[crow + i0] : 0u, mhi = 2 * I0 + 8 < nx ? L.omask[crow + 2 * I0 + 8] : 0u;
    const float wyj = L.wy[j], wzk = L.wz[k], ry0 = L.rhy[j], ry1 = L.rhy[j + 1], rz0 = L.rhz[k], rz1 = L.rhz[k + 1];
    float r[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) {
        const int i = i0 + t;
        const float p = t == 0 ? pm : (t == 9 ? pp : (t < 5 ? f4at(pA, t - 1) : f4at(pB, t - 5)));
        const unsigned msk = t == 0 ? mlo : (t == 9 ? mhi : (((t < 5 ? mm.x : mm.y) >> (8 * ((t - 1) & 3))) & 0xffu));
        float v = 0.f;
        if (i >= 0 && i < nx && p > 0.f) {
            if (((t + pc0 + 1) & 1) == 0) {
                // colour 0, the e-th of the window's five (t = 2 e - pc0 + 1)
                const int e = (t + pc0 - 1) >> 1;
                const bool edge = pc0 ? e == 0 : e == 4;
                const int qq = pc0 ? e - 1 : e;
                const float xc = edge ? x0e : f4at(x0q, qq & 3), fc = edge ? f0e : f4at(f0q, qq & 3);
                // x neighbours (colour 1) at packed I0 - 1 + e and I0 + e
                const float xm = e == 0 ? c1m : f4at(c1q, (e - 1) & 3);
                const float xp = e == 4 ? c1p : f4at(c1q, e & 3);
                const float ym = edge ? yme : f4at(ymq, qq & 3), yp = edge ? ype : f4at(ypq, qq & 3);
                const float zm = edge ? zme : f4at(zmq, qq & 3), zp = edge ? zpe : f4at(zpq, qq & 3);
                const float ayz = wyj * wzk, axz = L.wx[i] * wzk, axy = L.wx[i] * wyj;
                float d = 0.f, s = fc, tt;
                if (msk & 1u) { tt = ayz * L.rhx[i]; d += tt; s += tt * xm; }
                if (msk & 2u) { tt = ayz * L.rhx[i + 1]; d += tt; s += tt * xp; }
                if (msk & 4u) { tt = axz * ry0; d += tt; s += tt * ym; }
                if (msk & 8u) { tt = axz * ry1; d += tt; s += tt * yp; }
                if (msk & 16u) { tt = axy * rz0; d += tt; s += tt * zm; }
                if (msk & 32u) { tt = axy * rz1; d += tt; s += tt * zp; }
                v = p * (s - d * xc);
            } else if ((msk & 0x3fu) == 0) {
                // colour 1 (relaxed last) without an open face: not updated by
                // the smoother, r = p (f - 0 x)
                const int64_t pb = row * H + (i >> 1);
                const float d = 0.f;
                v = p * (fs1[pb] - d * xs1[pb]);
            }
        }
        r[t] = v;
    }
    // coarse I = I0 + u gathers the consecutive fine cells 2I - 1 .. 2I + 2
    // (2I .. 2I + 2 at the row start): window positions 2u + s + sh
    // (each coarse cell's four table entries in one 16-byte load apiece)
    float out[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int I = I0 + u;
        const int4 gi = *reinterpret_cast<const int4 *>(X.Gx + 4 * I);
        const float4 gw = ld4(X.gwx + 4 * I);
        const bool sh = gi.x != 2 * I - 1;
        const int g4[4] = {gi.x, gi.y, gi.z, gi.w};
        float acc = 0.f;
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2) {
            if (g4[s2] < 0) continue;
            const float rv = sh ? (2 * u + s2 + 1 <= 9 ? r[(2 * u + s2 + 1) > 9 ? 9 : (2 * u + s2 + 1)] : 0.f) : r[2 * u + s2];
            acc += f4at(gw, s2) * rv;
        }
        out[u] = acc;
    }
    *reinterpret_cast<float4 *>(tA + base) = make_float4(out[0], out[1], out[2], out[3]);
}

// k_prolong_yz on level 0 in colour-split storage, eight consecutive fine
// cells (one quad of each colour) per thread: tB, pn and both colours' x in
// 16-byte accesses; each cell gets the expression of k_prolong_yz (cells
// with pn = 0 keep their value)
__global__ void __launch_bounds__(256)
    k_prolong_yz_split8(MGLevel<float> L, SplitLv<float> S, float *__restrict__ xs0, float *__restrict__ xs1,
                        const float *__restrict__ tB, int cny, Xfer<float> X, const float *__restrict__ pn) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= S.nq) return;
    int64_t base;
    int h0, j, k;
    split_quad_pos(S, q, base, h0, j, k);
    const int pc0 = (j + k) & 1;
    const int64_t nat = base * 2;   // cell 2 h0 of the row
    int ib[2], ic[2];
    float wb[2], wc[2];
    const int nb = xfer_axis(X.Iy, X.Jy, X.wy, X.vy, j, ib, wb);
    const int nc = xfer_axis(X.Iz, X.Jz, X.wz, X.vz, k, ic, wc);
    const int64_t off = 2 * (int64_t)h0;
    float4 tv[2][2][2];
#pragma unroll
    for (int q3 = 0; q3 < 2; ++q3)
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
            const float *r = tB + ((int64_t)ic[q3 < nc ? q3 : 0] * cny + ib[q2 < nb ? q2 : 0]) * L.nx + off;
            tv[q3][q2][0] = ld4(r);
            tv[q3][q2][1] = ld4(r + 4);
        }
    const float4 pA = ld4(pn + nat), pB = ld4(pn + nat + 4);
    const float4 a0 = ld4(xs0 + base), a1 = ld4(xs1 + base);
    float o0[4] = {a0.x, a0.y, a0.z, a0.w}, o1[4] = {a1.x, a1.y, a1.z, a1.w};
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const float p = m < 4 ? f4at(pA, m) : f4at(pB, m - 4);
        if (!pos(p)) continue;
        float acc = 0.f;
        for (int q3 = 0; q3 < nc; ++q3) {
            float a2 = 0.f;
            for (int q2 = 0; q2 < nb; ++q2) a2 += wb[q2] * f4at(tv[q3][q2][m >> 2], m & 3);
            acc += wc[q3] * a2;
        }
        const bool c0 = ((m + pc0) & 1) == 0;
        const int e = m >> 1;   // packed position of cell 2 h0 + m in its colour
        if (c0) o0[e] = o0[e] + acc * p;
        else o1[e] = o1[e] + acc * p;
    }
    *reinterpret_cast<float4 *>(xs0 + base) = make_float4(o0[0], o0[1], o0[2], o0[3]);
    *reinterpret_cast<float4 *>(xs1 + base) = make_float4(o1[0], o1[1], o1[2], o1[3]);
}

// coarsest level: red-black sweeps in one block, all data in shared memory.
// The level operator is singular (constants); the right-hand side is made
// compatible by removing its mean over the active cells, and the solution is
// returned with zero mean there, so no constant mode builds up in the
// preconditioner (which would swamp FP32 corrections).
constexpr int COARSE_MAX = 512;

template <typename T>
__device__ __forceinline__ T block_mean_active(T v, bool act, T *red, int *cnt) {
    // plain shared-memory tree sum over COARSE_MAX slots (threads beyond
    // COARSE_MAX only take part in the barriers)
    const int c = threadIdx.x;
    if (c < COARSE_MAX) {
        red[c] = act ? v : T(0);
        cnt[c] = act ? 1 : 0;
    }
    __syncthreads();
    for (int o = COARSE_MAX / 2; o > 0; o >>= 1) {
        if (c < o) {
            red[c] += red[c + o];
            cnt[c] += cnt[c + o];
        }
        __syncthreads();
    }
    const T m = cnt[0] > 0 ? red[0] / T(cnt[0]) : T(0);
    __syncthreads();
    return m;
}

template <typename T>
struct CoarseSmem {
    T sx[COARSE_MAX], sf[COARSE_MAX], stx[COARSE_MAX], sty[COARSE_MAX], stz[COARSE_MAX], sdi[COARSE_MAX],
        red[COARSE_MAX];
    int cnt[COARSE_MAX];
};

// the coarsest-level solve by the threads of one block (at least COARSE_MAX)
template <typename T>
__device__ void coarse_solve_dev(const MGLevel<T> &L, const T *__restrict__ f, T *__restrict__ x, int sweeps,
                                 CoarseSmem<T> &S) {
    const int n = (int)L.n;
    const int c = threadIdx.x;
    int i = 0, j = 0, k = 0;
    bool act = false;
    if (c < n) {
        i = c % L.nx;
        j = (c / L.nx) % L.ny;
        k = c / (L.nx * L.ny);
        S.sx[c] = T(0);
        S.sf[c] = f[c];
        S.stx[c] = L.tx[c];
        S.sty[c] = L.ty[c];
        S.stz[c] = L.tz[c];
        S.sdi[c] = L.dinv[c];
        act = S.sdi[c] > T(0);
    }
    __syncthreads();
    const T fm = block_mean_active<T>(c < n ? S.sf[c] : T(0), act, S.red, S.cnt);
    if (act) S.sf[c] -= fm;
    __syncthreads();
    const int sy = L.nx, sz = L.nx * L.ny;
    const int par = (i + j + k) & 1;
    for (int pass = 0; pass < 4 * sweeps; ++pass) {
        // sweeps x (red, black) then sweeps x (black, red): a palindrome
        const int colour = pass < 2 * sweeps ? (pass & 1) : 1 - (pass & 1);
        if (c < n && par == colour && act) {
            T s = S.sf[c];
            if (i > 0) s += S.stx[c] * S.sx[c - 1];
            if (i < L.nx - 1) s += S.stx[c + 1] * S.sx[c + 1];
            if (j > 0) s += S.sty[c] * S.sx[c - sy];
            if (j < L.ny - 1) s += S.sty[c + sy] * S.sx[c + sy];
            if (k > 0) s += S.stz[c] * S.sx[c - sz];
            if (k < L.nz - 1) s += S.stz[c + sz] * S.sx[c + sz];
            S.sx[c] = s * S.sdi[c];
        }
        __syncthreads();
    }
    const T xm = block_mean_active<T>(c < n ? S.sx[c] : T(0), act, S.red, S.cnt);
    if (c < n) x[c] = act ? S.sx[c] - xm : T(0);
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(COARSE_MAX) k_coarse_solve(MGLevel<T> L, const T *__restrict__ f,
                                                             T *__restrict__ x, int sweeps) {
    __shared__ CoarseSmem<T> S;
    coarse_solve_dev<T>(L, f, x, sweeps, S);
}

// ---------------------------------------------------------------------------
// Persistent V-cycle tail: the coarse levels in one launch
// ---------------------------------------------------------------------------
//
// Below a few ten thousand cells the kernels of a level cannot fill the GPU,
// and each still costs a launch (about twelve per level and V-cycle). The
// tail runs the V-cycle from level l0 down to the coarsest level and back up
// in one launch of a single thread-block cluster. Each phase of the cycle (a
// colour pass, the residual-restriction along x, the restriction along y and
// z, the coarsest solve, the two prolongation passes) is a list of
// independent items (one cell, or one entry of a transfer row) that the
// cluster's threads take in turn; consecutive phases are separated by the
// cluster's hardware barrier (a block barrier for a one-block cluster), with
// release/acquire ordering of the global-memory writes. Nothing spins. Every
// item evaluates the expression of the per-level kernel it stands for, so
// the cycle's values are those of the launched kernels.

constexpr int TAIL_THREADS = 1024, TAIL_MAX_CTAS = 8;

// the arrays of level l that the tail reads and writes (fixed for the life
// of the hierarchy; the coarsest level uses L alone)
template <typename T>
struct TailLv {
    MGLevel<T> L;
    const T *pn;   // 1 / (active coarse weight sum) of the cells of l
    T *tmp;        // transfer scratch between l and l + 1
    Xfer<T> X;     // transfer tables between l and l + 1
};

__device__ __forceinline__ void tail_sync(int ncta) {
    if (ncta == 1) {
        __syncthreads();
    } else {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
}

// one colour pass (first: the first pass from x = 0, as k_rbgs_first with
// the zeros already in place; else k_rbgs) of a coarse level
template <typename T, bool OMEGA>
__device__ __forceinline__ void tail_colour(const MGLevel<T> &L, int col, T w, bool first, int gt, int nt) {
    const int np = (L.nx + 1) >> 1;
    const int items = L.ny * L.nz * np;
    for (int t = gt; t < items; t += nt) {
        const int row = t / np;
        int j, k;
        row_jk((uint32_t)row, L.fny, L.ny, j, k);
        const int i = 2 * (t - row * np) + ((j + k + col) & 1);
        if (i >= L.nx) continue;
        const int64_t c = (int64_t)row * L.nx + i;
        if (!active<T, false>(L, c)) continue;
        if (first) {
            L.x[c] = OMEGA ? w * (L.f[c] * L.dinv[c]) : L.f[c] * L.dinv[c];
        } else {
            T d;
            const T sm = k_offdiag<T, false>(L, L.x, c, i, j, k, d, L.f[c]);
            L.x[c] = OMEGA ? relax(L.x[c], sm * L.dinv[c], w) : sm * L.dinv[c];
        }
    }
}

// the residual-restriction along x (k_resid_rx<T, false>): one item per
// (fine row, coarse x index)
template <typename T>
__device__ __forceinline__ void tail_resid_rx(const TailLv<T> &A, int cnx, int zcol, int gt, int nt) {
    const MGLevel<T> &L = A.L;
    const int items = L.ny * L.nz * cnx;
    for (int t = gt; t < items; t += nt) {
        const int row = t / cnx, I = t - row * cnx;
        int j, k;
        row_jk((uint32_t)row, L.fny, L.ny, j, k);
        T acc = T(0);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int i = A.X.Gx[4 * I + s];
            if (i < 0) continue;
            T v = T(0);
            if (i < L.nx && !(zcol >= 0 && ((i + j + k) & 1) == zcol)) {
                const int64_t c = (int64_t)row * L.nx + i;
                const T p = A.pn[c];
                if (pos(p)) {
                    T d;
                    const T sm = k_offdiag<T, false>(L, L.x, c, i, j, k, d, L.f[c]);
                    v = p * (sm - d * L.x[c]);
                }
            }
            acc += A.X.gwx[4 * I + s] * v;
        }
        A.tmp[(int64_t)row * cnx + I] = acc;
    }
}

// the restriction along y and z into level C (k_restrict_yz)
template <typename T>
__device__ __forceinline__ void tail_restrict_yz(const MGLevel<T> &C, const T *tA, int fny, const Xfer<T> &X, int gt,
                                                 int nt) {
    const int items = C.ny * C.nz * C.nx;
    for (int t = gt; t < items; t += nt) {
        const int row = t / C.nx, Ic = t - row * C.nx;
        int Jc, Kc;
        row_jk((uint32_t)row, C.fny, C.ny, Jc, Kc);
        const int64_t cc = (int64_t)row * C.nx + Ic;
        C.x[cc] = T(0);
        if (!pos(C.dinv[cc])) {
            C.f[cc] = T(0);
            continue;
        }
        T acc = T(0);
#pragma unroll
        for (int s3 = 0; s3 < 4; ++s3) {
            const int k = X.Gz[4 * Kc + s3];
            if (k < 0) continue;
            T a2 = T(0);
#pragma unroll
            for (int s2 = 0; s2 < 4; ++s2) {
                const int j = X.Gy[4 * Jc + s2];
                if (j >= 0) a2 += X.gwy[4 * Jc + s2] * tA[((int64_t)k * fny + j) * C.nx + Ic];
            }
            acc += X.gwz[4 * Kc + s3] * a2;
        }
        C.f[cc] = acc;
    }
}

// the prolongation along x from level C (k_prolong_x)
template <typename T>
__device__ __forceinline__ void tail_prolong_x(int fnx, const MGLevel<T> &C, const Xfer<T> &X, T *tB, int gt, int nt) {
    const int items = C.ny * C.nz * fnx;
    for (int t = gt; t < items; t += nt) {
        const int row = t / fnx, i = t - row * fnx;
        const T *xr = C.x + (int64_t)row * C.nx;
        const int J2 = X.Jx[i];
        T v = X.wx[i] * xr[X.Ix[i]];
        if (J2 >= 0) v += X.vx[i] * xr[J2];
        tB[(int64_t)row * fnx + i] = v;
    }
}

// the prolongation along y and z and the correction of level l (k_prolong_yz)
template <typename T>
__device__ __forceinline__ void tail_prolong_yz(const TailLv<T> &A, int cny, int gt, int nt) {
    const MGLevel<T> &L = A.L;
    const Xfer<T> &X = A.X;
    const int items = L.ny * L.nz * L.nx;
    for (int t = gt; t < items; t += nt) {
        const int row = t / L.nx, i = t - row * L.nx;
        int j, k;
        row_jk((uint32_t)row, L.fny, L.ny, j, k);
        const int64_t c = (int64_t)row * L.nx + i;
        int ib[2], ic[2];
        T wb[2], wc[2];
        const int nb = xfer_axis(X.Iy, X.Jy, X.wy, X.vy, j, ib, wb);
        const int nc = xfer_axis(X.Iz, X.Jz, X.wz, X.vz, k, ic, wc);
        const T p = A.pn[c];
        if (!pos(p)) continue;
        T acc = T(0);
        for (int q3 = 0; q3 < nc; ++q3) {
            T a2 = T(0);
            for (int q2 = 0; q2 < nb; ++q2) a2 += wb[q2] * A.tmp[((int64_t)ic[q3] * cny + ib[q2]) * L.nx + i];
            acc += wc[q3] * a2;
        }
        L.x[c] = L.x[c] + acc * p;
    }
}

// The V-cycle from level l0 (its f and zeroed x written by the restriction
// from l0 - 1) to the coarsest level nl - 1 and back, nu1 / nu2 sweeps per
// level, cs sweep pairs on the coarsest level. One cluster of ncta blocks
// (gridDim.x == ncta).
template <typename T, bool OMEGA>
__global__ void __launch_bounds__(TAIL_THREADS)
    k_vtail(const TailLv<T> *__restrict__ A, int l0, int nl, int nu1, int nu2, int cs, T w, int ncta) {
    __shared__ CoarseSmem<T> S;
    const int gt = blockIdx.x * TAIL_THREADS + threadIdx.x, nt = ncta * TAIL_THREADS;
    const int zcol = 1;   // each pre-smoothing sweep ends with colour 1
    for (int l = l0; l < nl - 1; ++l) {
        const TailLv<T> &F = A[l];
        for (int s = 0; s < nu1; ++s) {
            tail_colour<T, OMEGA>(F.L, 0, w, s == 0, gt, nt);
            tail_sync(ncta);
            tail_colour<T, OMEGA>(F.L, 1, w, false, gt, nt);
            tail_sync(ncta);
        }
        const MGLevel<T> &C = A[l + 1].L;
        tail_resid_rx<T>(F, C.nx, zcol, gt, nt);
        tail_sync(ncta);
        tail_restrict_yz<T>(C, F.tmp, F.L.ny, F.X, gt, nt);
        tail_sync(ncta);
    }
    if (blockIdx.x == 0) {
        const MGLevel<T> &C = A[nl - 1].L;
        coarse_solve_dev<T>(C, C.f, C.x, cs, S);
    }
    tail_sync(ncta);
    for (int l = nl - 2; l >= l0; --l) {
        const TailLv<T> &F = A[l];
        const MGLevel<T> &C = A[l + 1].L;
        tail_prolong_x<T>(F.L.nx, C, F.X, F.tmp, gt, nt);
        tail_sync(ncta);
        tail_prolong_yz<T>(F, C.ny, gt, nt);
        tail_sync(ncta);
        for (int s = 0; s < nu2; ++s) {
            tail_colour<T, OMEGA>(F.L, 1, w, false, gt, nt);
            tail_sync(ncta);
            tail_colour<T, OMEGA>(F.L, 0, w, false, gt, nt);
            tail_sync(ncta);
        }
    }
}

// q = K p ; partial (p, q) in FP64
template <typename T, bool FINE>
__global__ void k_spmv_dot(MGLevel<T> L, const T *__restrict__ p, T *__restrict__ q, double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    GRID_STRIDE(c, L.n) {
        T v = T(0);
        if (active<T, FINE>(L, c)) {
            const uint32_t t = L.fnx.div((uint32_t)c);
            const int i = (int)((uint32_t)c - t * (uint32_t)L.nx);
            const uint32_t kk = L.fny.div(t);
            const int j = (int)(t - kk * (uint32_t)L.ny), k = (int)kk;
            T d;
            const T off = k_offdiag<T, FINE>(L, p, c, i, j, k, d);
            v = d * p[c] - off;
        }
        q[c] = v;
        acc += (double)p[c] * (double)v;
    }
    acc = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

template <typename T>
__global__ void k_dot(int64_t n, const T *__restrict__ a, const T *__restrict__ b, double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    GRID_STRIDE(c, n) acc += (double)a[c] * (double)b[c];
    acc = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

template <typename T>
__global__ void k_axpy2(int64_t n, T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
                        const T *__restrict__ q, const double *__restrict__ scal) {
    const T a = (T)scal[S_AL];
    GRID_STRIDE(c, n) {
        x[c] += a * p[c];
        r[c] -= a * q[c];
    }
}

template <typename T>
__global__ void k_pupd(int64_t n, T *__restrict__ p, const T *__restrict__ z, const double *__restrict__ scal) {
    const T b = (T)scal[S_BE];
    GRID_STRIDE(c, n) p[c] = z[c] + b * p[c];
}

// scalar updates (one thread)
__global__ void k_alpha(double *scal) {
    const double pq = scal[S_PQ];
    scal[S_AL] = (pq > 0.0 && isfinite(pq)) ? scal[S_RZ] / pq : 0.0;
}
__global__ void k_beta(double *scal) {
    const double rz = scal[S_RZ];
    scal[S_BE] = (rz != 0.0 && isfinite(rz)) ? scal[S_RZN] / rz : 0.0;
    scal[S_RZ] = scal[S_RZN];
}

// preconditioner input / output conversion
template <typename T>
__global__ void k_pre_in(GridDev g, OpT<T> o, const uint8_t *__restrict__ type, const T *__restrict__ v,
                         T *__restrict__ f) {
    GRID_STRIDE(c, g.n) {
        if (type[c] != FLUID) { f[c] = T(0); continue; }
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        if constexpr (sizeof(T) == 8) f[c] = -o.vol[c] * v[c];
        else f[c] = -(o.dx[i] * o.dy[j] * o.dz[k]) * v[c];
    }
}
// FP32 input four cells at a time (rows of a multiple of four cells)
__global__ void k_pre_in4(GridDev g, OpT<float> o, const uint8_t *__restrict__ type, const float *__restrict__ v,
                          float *__restrict__ f) {
    GRID_STRIDE(q, g.n / 4) {
        const int64_t c = 4 * q;
        const uchar4 t4 = reinterpret_cast<const uchar4 *>(type)[q];
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        const float4 vv = ld4(v + c), dxv = ld4(o.dx + i);
        const float dyj = o.dy[j], dzk = o.dz[k];
        float out[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            out[e] = u4get(t4, e) == FLUID ? -(f4get(dxv, e) * dyj * dzk) * f4get(vv, e) : 0.f;
        *reinterpret_cast<float4 *>(f + c) = make_float4(out[0], out[1], out[2], out[3]);
    }
}
template <typename T>
__global__ void k_pre_out(int64_t n, const uint8_t *__restrict__ type, const T *__restrict__ x, T *__restrict__ z) {
    int64_t n0 = 0;
    if constexpr (sizeof(T) == 4) {
        n0 = n / 4 * 4;
        GRID_STRIDE(q, n / 4) {
            const uchar4 t4 = reinterpret_cast<const uchar4 *>(type)[q];
            const float4 a = reinterpret_cast<const float4 *>(x)[q];
            reinterpret_cast<float4 *>(z)[q] = make_float4(t4.x == FLUID ? a.x : 0.f, t4.y == FLUID ? a.y : 0.f,
                                                           t4.z == FLUID ? a.z : 0.f, t4.w == FLUID ? a.w : 0.f);
        }
    }
    for (int64_t c = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        z[c] = type[c] == FLUID ? x[c] : T(0);
}
// ghost rows of the preconditioner: z_g = v_g + sum over FLUID corners wp z_m
template <typename T>
__global__ void k_pre_ghost(GhostDev gh, const T *__restrict__ wp, const uint8_t *__restrict__ type,
                            const T *__restrict__ v, T *__restrict__ z) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= gh.ng) return;
    const int64_t gi = gh.gidx[q];
    T s = v[gi];
    for (int m = 0; m < 8; ++m) {
        const int64_t s_m = gh.sidx[8 * q + m];
        if (type[s_m] == FLUID) s += wp[8 * q + m] * z[s_m];
    }
    z[gi] = s;
}

// one damped Jacobi pass of the full operator on the band, in precision T
// (o: the operator of op_of<T>; the FP64 A_row reads its stored diagonal dg,
// the FP32 one the per-axis sums): the new value of band cell q. z is read
// through a plain pointer: the single-block form below writes it in place.
template <typename T>
__device__ __forceinline__ T band_value(const GridDev &g, const GhostDev &gh, const OpT<T> &o, const int64_t *band,
                                        const int64_t *band_g, const T *v, const T *z, T omega, int64_t q) {
    const int64_t c = band[q];
    const int64_t gq = band_g[q];
    T res, diag;
    if (gq >= 0) {
        T s = z[c];
        for (int m = 0; m < 8; ++m) s -= o.wp[8 * gq + m] * z[gh.sidx[8 * gq + m]];
        res = v[c] - s;
        diag = T(1);
    } else {
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        res = v[c] - A_row<T>(g, o, z, c, i, j, k);
        if constexpr (sizeof(T) == 8) diag = -o.dg[c];
        else diag = -(o.cxs[i] + o.cys[j] + (g.ndim == 3 ? o.czs[k] : T(0)));
    }
    return z[c] + omega * res / diag;
}
// tmp = the new band values (a pass over the whole band; k_band_scatter
// then writes them into z)
template <typename T>
__global__ void k_band_jacobi(GridDev g, GhostDev gh, OpT<T> o, int64_t nb, const int64_t *__restrict__ band,
                              const int64_t *__restrict__ band_g, const T *__restrict__ v, const T *__restrict__ z,
                              T omega, T *__restrict__ tmp) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < nb) tmp[q] = band_value<T>(g, gh, o, band, band_g, v, z, omega, q);
}
// All sweeps in one block of BAND_BLOCK threads, for bands of at most
// BAND_BLOCK * BAND_PER_THREAD cells: each sweep computes every new value
// into registers, then (after a block barrier) writes them; the values
// equal those of the two-kernel form.
constexpr int BAND_BLOCK = 1024, BAND_PER_THREAD = 8;
template <typename T>
__global__ void __launch_bounds__(BAND_BLOCK)
    k_band_block(GridDev g, GhostDev gh, OpT<T> o, int64_t nb, const int64_t *__restrict__ band,
                 const int64_t *__restrict__ band_g, const T *__restrict__ v, T *z, T omega, int sweeps) {
    T nv[BAND_PER_THREAD];
    for (int s = 0; s < sweeps; ++s) {
#pragma unroll
        for (int u = 0; u < BAND_PER_THREAD; ++u) {
            const int64_t q = threadIdx.x + (int64_t)u * BAND_BLOCK;
            if (q < nb) nv[u] = band_value<T>(g, gh, o, band, band_g, v, z, omega, q);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < BAND_PER_THREAD; ++u) {
            const int64_t q = threadIdx.x + (int64_t)u * BAND_BLOCK;
            if (q < nb) z[band[q]] = nv[u];
        }
        __syncthreads();
    }
}
template <typename T>
__global__ void k_band_scatter(int64_t nb, const int64_t *__restrict__ band, const T *__restrict__ tmp,
                               T *__restrict__ z) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < nb) z[band[q]] = tmp[q];
}

// level coefficient construction ------------------------------------------

// level 0 open face areas: face on the low side of cell c along each axis is
// open when c and its low neighbour are both FLUID
__global__ void k_open_area0(GridDev g, const uint8_t *__restrict__ type, double *__restrict__ ox,
                             double *__restrict__ oy, double *__restrict__ oz) {
    GRID_STRIDE(c, g.n) {
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        const bool fl = type[c] == FLUID;
        const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
        ox[c] = (fl && i > 0 && type[c - 1] == FLUID) ? g.dy[j] * g.dz[k] : 0.0;
        oy[c] = (fl && j > 0 && type[c - sy] == FLUID) ? g.dx[i] * g.dz[k] : 0.0;
        oz[c] = (g.ndim == 3 && fl && k > 0 && type[c - sz] == FLUID) ? g.dx[i] * g.dy[j] : 0.0;
    }
}

// coarse open areas: the coarse low face gathers the low faces of the
// children that touch it
__global__ void k_open_area_coarsen(int nx, int ny, int nz, const double *__restrict__ ox,
                                    const double *__restrict__ oy, const double *__restrict__ oz, int cnx, int cny,
                                    int cnz, int fx, int fy, int fz, double *__restrict__ cx, double *__restrict__ cy,
                                    double *__restrict__ cz) {
    const int64_t cn = (int64_t)cnx * cny * cnz;
    GRID_STRIDE(cc, cn) {
        const int64_t t = cc / cnx;
        const int I = (int)(cc - t * cnx), J = (int)(t % cny), K = (int)(t / cny);
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int dk = 0; dk < fz; ++dk) {
            const int k = fz * K + dk;
            if (k >= nz) break;
            for (int dj = 0; dj < fy; ++dj) {
                const int j = fy * J + dj;
                if (j >= ny) break;
                for (int di = 0; di < fx; ++di) {
                    const int i = fx * I + di;
                    if (i >= nx) break;
                    const int64_t c = ((int64_t)k * ny + j) * nx + i;
                    if (di == 0) ax += ox[c];
                    if (dj == 0) ay += oy[c];
                    if (dk == 0) az += oz[c];
                }
            }
        }
        cx[cc] = ax;
        cy[cc] = ay;
        cz[cc] = az;
    }
}

// T = open area / centre spacing
template <typename T>
__global__ void k_level_coef(int nx, int ny, int nz, const double *__restrict__ ox, const double *__restrict__ oy,
                             const double *__restrict__ oz, const double *__restrict__ hx,
                             const double *__restrict__ hy, const double *__restrict__ hz, T *__restrict__ tx,
                             T *__restrict__ ty, T *__restrict__ tz) {
    const int64_t n = (int64_t)nx * ny * nz;
    GRID_STRIDE(c, n) {
        const int64_t t = c / nx;
        const int i = (int)(c - t * nx), j = (int)(t % ny), k = (int)(t / ny);
        tx[c] = i > 0 ? (T)(ox[c] / hx[i]) : T(0);
        ty[c] = j > 0 ? (T)(oy[c] / hy[j]) : T(0);
        tz[c] = k > 0 ? (T)(oz[c] / hz[k]) : T(0);
    }
}
// D = sum of the six faces; dinv = 1/D (0 when D = 0)
template <typename T>
__global__ void k_level_diag(MGLevel<T> L) {
    GRID_STRIDE(c, L.n) {
        const int64_t t = c / L.nx;
        const int i = (int)(c - t * L.nx), j = (int)(t % L.ny), k = (int)(t / L.ny);
        const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
        T d = L.tx[c] + L.ty[c] + L.tz[c];
        if (i < L.nx - 1) d += L.tx[c + 1];
        if (j < L.ny - 1) d += L.ty[c + sy];
        if (k < L.nz - 1) d += L.tz[c + sz];
        L.d[c] = d;
        L.dinv[c] = d > T(0) ? T(1) / d : T(0);
    }
}

// band: FLUID cells within band_width faces of a ghost cell, plus the ghosts
__global__ void k_band_seed(int64_t n, const uint8_t *__restrict__ type, uint8_t *__restrict__ f) {
    GRID_STRIDE(c, n) f[c] = type[c] == GHOST;
}
__global__ void k_band_dilate(GridDev g, const uint8_t *__restrict__ type, const uint8_t *__restrict__ in,
                              uint8_t *__restrict__ out) {
    GRID_STRIDE(c, g.n) {
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
        bool b = in[c];
        if (!b && type[c] == FLUID) {
            b = (i > 0 && in[c - 1]) || (i < g.nx - 1 && in[c + 1]) || (j > 0 && in[c - sy]) ||
                (j < g.ny - 1 && in[c + sy]) || (k > 0 && in[c - sz]) || (k < g.nz - 1 && in[c + sz]);
        }
        out[c] = b;
    }
}
// band_g[q] = position of band[q] in the ascending ghost list, or -1
__global__ void k_band_gpos(int64_t nb, const int64_t *__restrict__ band, int64_t ng, const int64_t *__restrict__ gidx,
                            int64_t *__restrict__ band_g) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nb) return;
    const int64_t c = band[q];
    int64_t lo = 0, hi = ng;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (gidx[mid] < c) lo = mid + 1; else hi = mid;
    }
    band_g[q] = (lo < ng && gidx[lo] == c) ? lo : -1;
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------

template <typename T>
static Xfer<T> xfer_of(Ctx *c, int l);
template <>
Xfer<double> xfer_of<double>(Ctx *c, int l) {
    return Xfer<double>{c->tI[0][l],   c->tJ[0][l],   c->tI[1][l],   c->tJ[1][l],   c->tI[2][l],
                        c->tJ[2][l],   c->tw64[0][l], c->tw64[1][l], c->tw64[2][l], c->gI[0][l],
                        c->gI[1][l],   c->gI[2][l],   c->gw64[0][l], c->gw64[1][l], c->gw64[2][l],
                        c->tv64[0][l], c->tv64[1][l], c->tv64[2][l]};
}
template <>
Xfer<float> xfer_of<float>(Ctx *c, int l) {
    return Xfer<float>{c->tI[0][l],   c->tJ[0][l],   c->tI[1][l],   c->tJ[1][l],   c->tI[2][l],
                       c->tJ[2][l],   c->tw32[0][l], c->tw32[1][l], c->tw32[2][l], c->gI[0][l],
                       c->gI[1][l],   c->gI[2][l],   c->gw32[0][l], c->gw32[1][l], c->gw32[2][l],
                       c->tv32[0][l], c->tv32[1][l], c->tv32[2][l]};
}

template <typename T>
static ibm_status alloc_level_arrays(Ctx *c, MGLevel<T> &M, bool coeffs, bool vecs) {
    const size_t bytes = sizeof(T) * (size_t)M.n;
    M.tx = M.ty = M.tz = M.d = M.dinv = M.x = M.f = nullptr;
    if (coeffs) {
        M.tx = (T *)dev_alloc(c, bytes);
        M.ty = (T *)dev_alloc(c, bytes);
        M.tz = (T *)dev_alloc(c, bytes);
        M.d = (T *)dev_alloc(c, bytes);
        M.dinv = (T *)dev_alloc(c, bytes);
        if (!M.tx || !M.ty || !M.tz || !M.d || !M.dinv) return c->fail(IBM_ERR_OOM, "multigrid level allocation failed");
    }
    if (vecs) {
        M.x = (T *)dev_alloc(c, bytes);
        M.f = (T *)dev_alloc(c, bytes);
        if (!M.x || !M.f) return c->fail(IBM_ERR_OOM, "multigrid level allocation failed");
    }
    return IBM_OK;
}

template <typename T>
static T *upload_as(Ctx *c, const std::vector<double> &h, bool reciprocal) {
    std::vector<T> v(h.size());
    for (size_t i = 0; i < h.size(); ++i) v[i] = reciprocal ? (h[i] != 0.0 ? (T)(1.0 / h[i]) : T(0)) : (T)h[i];
    T *d = (T *)dev_alloc(c, sizeof(T) * (v.size() ? v.size() : 1));
    if (d && v.size()) cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return d;
}

template <typename T>
static ibm_status build_hier(Ctx *c, MGHier<T> &H, bool fine0) {
    const int L = (int)c->lg.size();
    H.lv.resize(L);
    H.fine0 = fine0;
    for (int l = 0; l < L; ++l) {
        auto &G = c->lg[l];
        MGLevel<T> &M = H.lv[l];
        M = MGLevel<T>{};
        M.nx = G.nx;
        M.ny = G.ny;
        M.nz = G.nz;
        M.n = (int64_t)G.nx * G.ny * G.nz;
        M.fnx = FastDiv((uint32_t)G.nx);
        M.fny = FastDiv((uint32_t)G.ny);
        IBM_TRY(alloc_level_arrays(c, M, !(l == 0 && fine0), l > 0));
    }
    if (fine0) {
        H.wx = upload_as<T>(c, c->hdx, false);
        H.wy = upload_as<T>(c, c->hdy, false);
        H.wz = upload_as<T>(c, c->hdz, false);
        H.rhx = upload_as<T>(c, c->hhx, true);
        H.rhy = upload_as<T>(c, c->hhy, true);
        H.rhz = upload_as<T>(c, c->hhz, true);
        if (!H.wx || !H.wy || !H.wz || !H.rhx || !H.rhy || !H.rhz) return c->fail(IBM_ERR_OOM, "metric allocation failed");
        MGLevel<T> &M = H.lv[0];
        M.type = c->type;
        M.wx = H.wx; M.wy = H.wy; M.wz = H.wz;
        M.rhx = H.rhx; M.rhy = H.rhy; M.rhz = H.rhz;
        // colour-split storage of level 0 (FP32, rows of whole 16-byte quads)
        if (sizeof(T) == 4 && c->nx % 8 == 0 && L > 1) {
            const size_t hn = (size_t)c->N / 2;
            for (int q = 0; q < 2; ++q) {
                H.xs[q] = (T *)dev_alloc(c, sizeof(T) * hn);
                H.fs[q] = (T *)dev_alloc(c, sizeof(T) * hn);
                H.ms[q] = (uint8_t *)dev_alloc(c, hn);
                if (!H.xs[q] || !H.fs[q] || !H.ms[q]) return c->fail(IBM_ERR_OOM, "split level allocation failed");
                std::vector<double> wx(c->nx / 2), rm(c->nx / 2), rp(c->nx / 2);
                for (int h = 0; h < c->nx / 2; ++h) {
                    wx[h] = c->hdx[2 * h + q];
                    rm[h] = c->hhx[2 * h + q];
                    rp[h] = c->hhx[2 * h + q + 1];
                }
                H.swx[q] = upload_as<T>(c, wx, false);
                H.srm[q] = upload_as<T>(c, rm, true);
                H.srp[q] = upload_as<T>(c, rp, true);
                if (!H.swx[q] || !H.srm[q] || !H.srp[q]) return c->fail(IBM_ERR_OOM, "split metric allocation failed");
            }
            H.split = true;
        }
    }
    H.res.assign(L, nullptr);
    H.pn.assign(L, nullptr);
    for (int l = 0; l + 1 < L; ++l) {
        const size_t bytes = sizeof(T) * (size_t)H.lv[l].n;
        H.pn[l] = (T *)dev_alloc(c, bytes);
        if (l > 0) H.res[l] = (T *)dev_alloc(c, bytes);
        if (!H.pn[l] || (l > 0 && !H.res[l])) return c->fail(IBM_ERR_OOM, "transfer buffer allocation failed");
    }
    const size_t b0 = sizeof(T) * (size_t)c->N;
    H.px = (T *)dev_alloc(c, b0);
    H.pr = (T *)dev_alloc(c, b0);
    H.pz = (T *)dev_alloc(c, b0);
    H.pp = (T *)dev_alloc(c, b0);
    H.pq = (T *)dev_alloc(c, b0);
    if (!H.px || !H.pr || !H.pz || !H.pp || !H.pq) return c->fail(IBM_ERR_OOM, "PCG vector allocation failed");
    // the persistent tail's per-level table (pointers fixed from here on)
    if (L >= 3) {
        std::vector<TailLv<T>> tl(L);
        for (int l = 0; l < L; ++l) {
            tl[l] = TailLv<T>{};
            tl[l].L = H.lv[l];
            if (l + 1 < L) {
                tl[l].pn = H.pn[l];
                tl[l].tmp = l > 0 ? H.res[l] : nullptr;
                tl[l].X = xfer_of<T>(c, l + 1);
            }
        }
        H.tail = dev_alloc(c, sizeof(TailLv<T>) * (size_t)L);
        if (!H.tail) return c->fail(IBM_ERR_OOM, "tail table allocation failed");
        IBM_CUDA(c, cudaMemcpy(H.tail, tl.data(), sizeof(TailLv<T>) * (size_t)L, cudaMemcpyHostToDevice));
    }
    H.built = true;
    return IBM_OK;
}

template <typename T>
static ibm_status fill_hier(Ctx *c, MGHier<T> &H, const std::vector<double *> &ox, const std::vector<double *> &oy,
                            const std::vector<double *> &oz) {
    const int L = (int)H.lv.size();
    for (int l = 0; l < L; ++l) {
        MGLevel<T> &M = H.lv[l];
        if (l == 0 && H.fine0) {
            M.type = c->type;
            if (!H.omask) H.omask = (uint8_t *)dev_alloc(c, c->N);
            if (!H.omask) return c->fail(IBM_ERR_OOM, "open-face mask allocation failed");
            KL(-1, k_open_mask, nblk(c->N), 256, c->g, c->type, H.omask);
            IBM_LAUNCHED(c);
            M.omask = H.omask;
            if constexpr (sizeof(T) == 4) {
                if (H.split) {
                    const SplitLv<float> S = split_of(H);
                    KL(-1, k_split_mask, (unsigned)((S.nq + 255) / 256), 256, S, H.omask, H.ms[0], H.ms[1]);
                    IBM_LAUNCHED(c);
                }
            }
            continue;
        }
        KL(-1, k_level_coef<T>, nblk(M.n), 256, M.nx, M.ny, M.nz, ox[l], oy[l], oz[l], c->lhx[l], c->lhy[l],
           c->lhz[l], M.tx, M.ty, M.tz);
        KL(-1, k_level_diag<T>, nblk(M.n), 256, M);
        IBM_LAUNCHED(c);
    }
    // trilinear transfer normalisation of every fine level
    for (int l = 0; l + 1 < L; ++l) {
        MGLevel<T> &M = H.lv[l];
        const dim3 grid = rows_grid(M.nx, M.ny, M.nz, 1, 128);
        if (l == 0 && H.fine0) KL(-1, (k_pnorm<T, true>), grid, 128, M, H.lv[l + 1], xfer_of<T>(c, l + 1), H.pn[l]);
        else KL(-1, (k_pnorm<T, false>), grid, 128, M, H.lv[l + 1], xfer_of<T>(c, l + 1), H.pn[l]);
        IBM_LAUNCHED(c);
    }
    return IBM_OK;
}

ibm_status compact_flags(Ctx *c, const uint8_t *flags, int64_t **out, int64_t *count);

// Multigrid hierarchies of the staircase operator and the near-body band for
// the current classification.
ibm_status mg_build(Ctx *c) {
    const int L = (int)c->lg.size();
    ++c->mg_gen;
    IBM_TRY(hist_reset(c));
    std::vector<double *> ox(L), oy(L), oz(L);
    for (int l = 0; l < L; ++l) {
        const int64_t n = (int64_t)c->lg[l].nx * c->lg[l].ny * c->lg[l].nz;
        ox[l] = (double *)dev_alloc(c, sizeof(double) * n);
        oy[l] = (double *)dev_alloc(c, sizeof(double) * n);
        oz[l] = (double *)dev_alloc(c, sizeof(double) * n);
        if (!ox[l] || !oy[l] || !oz[l]) return c->fail(IBM_ERR_OOM, "open-area allocation failed");
    }
    KL(-1, k_open_area0, nblk(c->N), 256, c->g, c->type, ox[0], oy[0], oz[0]);
    IBM_LAUNCHED(c);
    for (int l = 1; l < L; ++l) {
        auto &F = c->lg[l - 1];
        auto &C = c->lg[l];
        const int64_t n = (int64_t)C.nx * C.ny * C.nz;
        KL(-1, k_open_area_coarsen, nblk(n), 256, F.nx, F.ny, F.nz, ox[l - 1], oy[l - 1], oz[l - 1], C.nx, C.ny, C.nz,
           C.fx, C.fy, C.fz, ox[l], oy[l], oz[l]);
        IBM_LAUNCHED(c);
    }
    // each hierarchy is built when its precision is first used and refreshed
    // on every later classification
    const bool need64 = c->opts.precision == IBM_FP64 || c->mg64.built;
    const bool need32 = c->opts.precision == IBM_MIXED || c->mg32.built;
    if (need64) {
        if (!c->mg64.built) IBM_TRY(build_hier<double>(c, c->mg64, false));
        IBM_TRY(fill_hier<double>(c, c->mg64, ox, oy, oz));
    }
    if (need32) {
        if (!c->mg32.built) IBM_TRY(build_hier<float>(c, c->mg32, true));
        IBM_TRY(fill_hier<float>(c, c->mg32, ox, oy, oz));
    }
    // near-body band
    uint8_t *f0 = (uint8_t *)dev_alloc(c, c->N), *f1 = (uint8_t *)dev_alloc(c, c->N);
    if (!f0 || !f1) return c->fail(IBM_ERR_OOM, "band flag allocation failed");
    KL(-1, k_band_seed, nblk(c->N), 256, c->N, c->type, f0);
    for (int d = 0; d < c->opts.band_width; ++d) {
        KL(-1, k_band_dilate, nblk(c->N), 256, c->g, c->type, f0, f1);
        std::swap(f0, f1);
    }
    IBM_LAUNCHED(c);
    dev_free(c, c->band);
    dev_free(c, c->band_g);
    dev_free(c, c->btmp);
    c->band = c->band_g = nullptr;
    c->btmp = nullptr;
    IBM_TRY(compact_flags(c, f0, &c->band, &c->nband));
    c->band_g = (int64_t *)dev_alloc(c, sizeof(int64_t) * (c->nband > 0 ? c->nband : 1));
    c->btmp = (double *)dev_alloc(c, sizeof(double) * (c->nband > 0 ? c->nband : 1));
    if (!c->band_g || !c->btmp) return c->fail(IBM_ERR_OOM, "band allocation failed");
    if (c->nband > 0) {
        KL(-1, k_band_gpos, (unsigned)((c->nband + 255) / 256), 256, c->nband, c->band, c->ng, c->gidx, c->band_g);
        IBM_LAUNCHED(c);
    }
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    dev_free(c, f0);
    dev_free(c, f1);
    for (int l = 0; l < L; ++l) {
        dev_free(c, ox[l]);
        dev_free(c, oy[l]);
        dev_free(c, oz[l]);
    }
    return IBM_OK;
}

// first: 0 a colour pass; 1 the first pass of the level from x = 0; 2 the
// same, also writing the zeros of x (no clearing before)
template <typename T>
static ibm_status rbgs(Ctx *c, MGHier<T> &H, int l, const T *f, T *x, int col, int first = 0) {
    MGLevel<T> &L = H.lv[l];
    const int bx = c->opts.tile_x;
    const dim3 grid = rows_grid(L.nx, L.ny, L.nz, 2, bx);
    const double w = c->opts.smooth_omega;
    // (the first pass moves fewer bytes than a colour pass: timed apart, so
    // that the finest-level id keeps to full passes)
    const int kid = -1;
    if (first) {
        const int z = first == 2;
        const bool fine = l == 0 && H.fine0;
        if (w != 1.0) {
            if (fine) KL(kid, (k_rbgs_first<T, true, true>), grid, bx, L, f, x, col, (T)w, z);
            else KL(kid, (k_rbgs_first<T, false, true>), grid, bx, L, f, x, col, (T)w, z);
        } else {
            if (fine) KL(kid, (k_rbgs_first<T, true>), grid, bx, L, f, x, col, T(1), z);
            else KL(kid, (k_rbgs_first<T, false>), grid, bx, L, f, x, col, T(1), z);
        }
        IBM_LAUNCHED(c);
        return IBM_OK;
    }
    if (w != 1.0) {
        if (l == 0 && H.fine0) KL(K_RBGS0, (k_rbgs<T, true, true>), grid, bx, L, f, x, col, (T)w);
        else KL(l == 0 ? K_RBGS0 : K_RBGS_C, (k_rbgs<T, false, true>), grid, bx, L, f, x, col, (T)w);
    } else if (l == 0 && H.fine0) KL(K_RBGS0, (k_rbgs<T, true>), grid, bx, L, f, x, col, T(1));
    else KL(l == 0 ? K_RBGS0 : K_RBGS_C, (k_rbgs<T, false>), grid, bx, L, f, x, col, T(1));
    IBM_LAUNCHED(c);
    return IBM_OK;
}

// level 0 of the FP32 hierarchy in colour-split storage for this cycle
template <typename T>
static bool split_on(const Ctx *c, const MGHier<T> &H) {
    return sizeof(T) == 4 && H.split && c->opts.fine_split == 1 && c->opts.mg_interp == 1 && H.lv.size() > 1;
}

// split-storage passes of level 0: kind 0 a colour pass, 1 the first pass
// from x = 0 (also splitting f0), 2 the last colour-0 pass writing the
// cell-ordered output x0, 3 the merge of both colours into x0
static ibm_status split_pass(Ctx *c, MGHier<float> &H, int kind, int col, const float *f0, float *x0) {
    const SplitLv<float> S = split_of(H);
    const unsigned nb = (unsigned)((S.nq + 255) / 256);
    const double w = c->opts.smooth_omega;
    const bool om = w != 1.0;
    if (kind == 1) {
        if (om) KL(-1, k_rbgs_first_split<true>, nb, 256, S, f0, H.ms[0], H.fs[0], H.fs[1], H.xs[0], H.xs[1], (float)w);
        else KL(-1, k_rbgs_first_split<false>, nb, 256, S, f0, H.ms[0], H.fs[0], H.fs[1], H.xs[0], H.xs[1], 1.f);
    } else if (kind == 3) {
        KL(-1, k_split_merge, nb, 256, S, H.xs[0], H.xs[1], x0);
    } else {
        const float *fq = H.fs[col], *xo = H.xs[1 - col];
        const uint8_t *mq = H.ms[col];
        float *xq = H.xs[col];
        if (kind == 2) {
            if (om) KL(K_RBGS0, (k_rbgs_split<true, true>), nb, 256, S, fq, mq, xo, xq, col, (float)w, x0);
            else KL(K_RBGS0, (k_rbgs_split<false, true>), nb, 256, S, fq, mq, xo, xq, col, 1.f, x0);
        } else {
            if (om) KL(K_RBGS0, (k_rbgs_split<true, false>), nb, 256, S, fq, mq, xo, xq, col, (float)w, nullptr);
            else KL(K_RBGS0, (k_rbgs_split<false, false>), nb, 256, S, fq, mq, xo, xq, col, 1.f, nullptr);
        }
    }
    IBM_LAUNCHED(c);
    return IBM_OK;
}

// First level of the persistent tail for this hierarchy and options (the
// first level below 0 with at most tail_cells cells, if it leaves at least
// one level to smooth above the coarsest), or -1; ncta: blocks of its cluster
template <typename T>
static int tail_level(const Ctx *c, const MGHier<T> &H, int *ncta) {
    const int L = (int)H.lv.size();
    if (c->opts.tail_cells <= 0 || c->opts.mg_interp != 1 || !H.tail || L < 3) return -1;
    int l0 = 1;
    while (l0 < L && H.lv[l0].n > c->opts.tail_cells) ++l0;
    if (l0 > L - 2) return -1;
    const int64_t per = 2 * (int64_t)TAIL_THREADS;
    *ncta = (int)std::min<int64_t>(TAIL_MAX_CTAS, std::max<int64_t>(1, (H.lv[l0].n + per - 1) / per));
    return l0;
}

template <typename T>
static ibm_status launch_tail(Ctx *c, MGHier<T> &H, int l0, int ncta) {
    const int L = (int)H.lv.size();
    const TailLv<T> *A = reinterpret_cast<const TailLv<T> *>(H.tail);
    // (every tail level lies below the finest)
    const int nu1 = c->opts.nu_coarse > 0 ? c->opts.nu_coarse : c->opts.nu1;
    const int nu2 = c->opts.nu_coarse > 0 ? c->opts.nu_coarse : c->opts.nu2, cs = c->opts.coarse_sweeps;
    const double w = c->opts.smooth_omega;
    auto kern = w != 1.0 ? k_vtail<T, true> : k_vtail<T, false>;
    kt_begin(c, K_TAIL);
    ++c->nlaunch;
    if (ncta == 1) {
        kern<<<1, TAIL_THREADS, 0, c->s>>>(A, l0, L, nu1, nu2, cs, (T)w, 1);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)ncta, 1, 1);
        cfg.blockDim = dim3(TAIL_THREADS, 1, 1);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = c->s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)ncta;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        IBM_CUDA(c, cudaLaunchKernelEx(&cfg, kern, A, l0, L, nu1, nu2, cs, (T)w, ncta));
    }
    kt_end(c, K_TAIL);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

template <typename T>
static ibm_status vcycle(Ctx *c, MGHier<T> &H, const T *f0, T *x0) {
    const int L = (int)H.lv.size();
    const int nu1 = c->opts.nu1, nu2 = c->opts.nu2, cs = c->opts.coarse_sweeps;
    // sweeps on the levels below the finest
    const int nuc1 = c->opts.nu_coarse > 0 ? c->opts.nu_coarse : nu1;
    const int nuc2 = c->opts.nu_coarse > 0 ? c->opts.nu_coarse : nu2;
    const int bx = c->opts.tile_x;
    if (L == 1) {
        KL(-1, k_coarse_solve<T>, 1, COARSE_MAX, H.lv[0], f0, x0, cs);
        IBM_LAUNCHED(c);
        return IBM_OK;
    }
    // x0 starts at zero: the first colour pass writes it whole (the coarse
    // levels' x is cleared by the restriction)
    if (nu1 < 1) IBM_CUDA(c, cudaMemsetAsync(x0, 0, sizeof(T) * (size_t)c->N, c->s));
    const bool sp = split_on(c, H);
    // levels lt .. L - 1 in one persistent launch (lt = L - 1: the coarsest
    // solve alone)
    int ncta = 1;
    const int l0 = tail_level(c, H, &ncta);
    const int lt = l0 > 0 ? l0 : L - 1;
    for (int l = 0; l < lt; ++l) {
        const T *f = l == 0 ? f0 : H.lv[l].f;
        T *x = l == 0 ? x0 : H.lv[l].x;
        if constexpr (sizeof(T) == 4) {
            if (l == 0 && sp) {
                for (int s = 0; s < nu1; ++s) {
                    if (s == 0) IBM_TRY(split_pass(c, H, 1, 0, f0, x0));
                    else IBM_TRY(split_pass(c, H, 0, 0, f0, x0));
                    IBM_TRY(split_pass(c, H, 0, 1, f0, x0));
                }
            }
        }
        if (!(l == 0 && sp)) {
            const int n1 = l == 0 ? nu1 : nuc1;
            for (int s = 0; s < n1; ++s) {
                IBM_TRY(rbgs(c, H, l, f, x, 0, s == 0 ? (l == 0 ? 2 : 1) : 0));
                IBM_TRY(rbgs(c, H, l, f, x, 1));
            }
        }
        MGLevel<T> &Lf = H.lv[l];
        MGLevel<T> &Cl = H.lv[l + 1];
        auto &CG = c->lg[l + 1];
        const dim3 grid = rows_grid(Cl.nx, Cl.ny, Cl.nz, 1, bx);
        if (c->opts.mg_interp == 1) {
            // fine residual and restriction along x, then along y and z
            // (transpose of the trilinear prolongation)
            T *tA = l == 0 ? H.pq : H.res[l];
            const Xfer<T> X = xfer_of<T>(c, l + 1);
            const dim3 rgrid((unsigned)((int64_t)Lf.ny * Lf.nz), (unsigned)((Cl.nx + RX_THREADS - 1) / RX_THREADS));
            const int zcol = nu1 > 0 ? 1 : -1;   // each pre-smoothing sweep ends with colour 1
            bool done = false;
            if constexpr (sizeof(T) == 4) {
                if (l == 0 && sp) {
                    if (CG.fx == 2 && zcol == 1) {
                        const SplitLv<float> S = split_of(H);
                        KL(K_RESTRICT, k_resid_rx_split4, (unsigned)((S.nq + 255) / 256), 256, Lf, S, H.fs[0],
                           H.fs[1], H.xs[0], H.xs[1], H.pn[l], X, tA);
                    } else {
                        KL(K_RESTRICT, k_resid_rx_split, rgrid, RX_THREADS, Lf, H.fs[0], H.fs[1], H.xs[0], H.xs[1],
                           H.pn[l], X, Cl.nx, CG.fx, zcol, tA);
                    }
                    done = true;
                }
            }
            if (done) {
            } else if (l == 0 && H.fine0)
                KL(K_RESTRICT, (k_resid_rx<T, true>), rgrid, RX_THREADS, Lf, f, x, H.pn[l], X, Cl.nx, CG.fx, zcol, tA);
            else
                KL(K_RESTRICT, (k_resid_rx<T, false>), rgrid, RX_THREADS, Lf, f, x, H.pn[l], X, Cl.nx, CG.fx, zcol,
                   tA);
            KL(K_RESTRICT, k_restrict_yz<T>, grid, bx, Cl, tA, Lf.ny, X);
        } else if (l == 0 && H.fine0) {
            KL(K_RESTRICT, (k_resid_restrict<T, true>), grid, bx, Lf, f, x, Cl, CG.fx, CG.fy, CG.fz);
        } else {
            KL(K_RESTRICT, (k_resid_restrict<T, false>), grid, bx, Lf, f, x, Cl, CG.fx, CG.fy, CG.fz);
        }
        IBM_LAUNCHED(c);
    }
    if (l0 > 0) {
        IBM_TRY(launch_tail(c, H, l0, ncta));
    } else {
        KL(-1, k_coarse_solve<T>, 1, COARSE_MAX, H.lv[L - 1], H.lv[L - 1].f, H.lv[L - 1].x, cs);
        IBM_LAUNCHED(c);
    }
    for (int l = lt - 1; l >= 0; --l) {
        const T *f = l == 0 ? f0 : H.lv[l].f;
        T *x = l == 0 ? x0 : H.lv[l].x;
        MGLevel<T> &Lf = H.lv[l];
        auto &CG = c->lg[l + 1];
        const dim3 grid = rows_grid(Lf.nx, Lf.ny, Lf.nz, 1, bx);
        if (c->opts.mg_interp == 1) {
            MGLevel<T> &Cl = H.lv[l + 1];
            T *tB = l == 0 ? H.pq : H.res[l];
            const Xfer<T> X = xfer_of<T>(c, l + 1);
            KL(K_PROLONG, k_prolong_x<T>, rows_grid(Lf.nx, Cl.ny, Cl.nz, 1, bx), bx, Lf.nx, Cl, X, tB);
            bool done = false;
            if constexpr (sizeof(T) == 4) {
                if (l == 0 && sp) {
                    const SplitLv<float> S = split_of(H);
                    KL(K_PROLONG, k_prolong_yz_split8, (unsigned)((S.nq + 255) / 256), 256, Lf, S, H.xs[0], H.xs[1], tB,
                       Cl.ny, X, H.pn[l]);
                    done = true;
                }
            }
            if (!done) KL(K_PROLONG, k_prolong_yz<T>, grid, bx, Lf, x, tB, Cl.ny, X, H.pn[l]);
        } else if (l == 0 && H.fine0) {
            KL(K_PROLONG, (k_prolong<T, true>), grid, bx, Lf, x, H.lv[l + 1], CG.fx, CG.fy, CG.fz);
        } else {
            KL(K_PROLONG, (k_prolong<T, false>), grid, bx, Lf, x, H.lv[l + 1], CG.fx, CG.fy, CG.fz);
        }
        IBM_LAUNCHED(c);
        if constexpr (sizeof(T) == 4) {
            if (l == 0 && sp) {
                // the last colour-0 pass writes the cell-ordered output x0
                for (int s = 0; s < nu2; ++s) {
                    IBM_TRY(split_pass(c, H, 0, 1, f0, x0));
                    IBM_TRY(split_pass(c, H, s + 1 == nu2 ? 2 : 0, 0, f0, x0));
                }
                if (nu2 < 1) IBM_TRY(split_pass(c, H, 3, 0, f0, x0));
                continue;
            }
        }
        for (int s = 0; s < (l == 0 ? nu2 : nuc2); ++s) {
            IBM_TRY(rbgs(c, H, l, f, x, 1));
            IBM_TRY(rbgs(c, H, l, f, x, 0));
        }
    }
    return IBM_OK;
}

// The V-cycle pr -> pz as one CUDA graph: captured from the stream the
// first time (and again after a multigrid rebuild or a change of its
// settings), then replayed with a single launch. Its buffers are fixed, so
// the graph stays valid for the life of the hierarchy.
template <typename T>
static ibm_status vcycle_graph(Ctx *c, MGHier<T> &H, T *out) {
    const ibm_solver_opts &o = c->opts;
    const uint64_t key = ((((((c->mg_gen * 64 + (uint64_t)o.nu1) * 64 + (uint64_t)o.nu2) * 4096 +
                           (uint64_t)o.coarse_sweeps) * 1024 + (uint64_t)o.tile_x) * 4 + (uint64_t)o.mg_interp * 2 +
                         (uint64_t)o.fine_split) * 1000003 + (uint64_t)o.tail_cells) * 16 + (uint64_t)o.nu_coarse + 1;
    auto drop_all = [&]() -> ibm_status {
        IBM_CUDA(c, cudaStreamSynchronize(c->s));
        for (int i = 0; i < MGHier<T>::NVG; ++i) {
            if (H.vgraph[i]) cudaGraphExecDestroy(H.vgraph[i]);
            H.vgraph[i] = nullptr;
            H.vgraph_out[i] = nullptr;
        }
        return IBM_OK;
    };
    if (H.vgraph_key != key) {
        IBM_TRY(drop_all());
        H.vgraph_key = key;
    }
    int slot = -1;
    for (int i = 0; i < MGHier<T>::NVG && slot < 0; ++i)
        if (H.vgraph[i] && H.vgraph_out[i] == out) slot = i;
    if (slot < 0) {
        for (int i = 0; i < MGHier<T>::NVG && slot < 0; ++i)
            if (!H.vgraph[i]) slot = i;
        if (slot < 0) {
            IBM_TRY(drop_all());
            slot = 0;
        }
        const int64_t n0 = c->nlaunch;
        IBM_CUDA(c, cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
        const ibm_status st = vcycle(c, H, H.pr, out);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->s, &g);
        IBM_TRY(st);
        if (e != cudaSuccess) return c->fail(IBM_ERR_CUDA, std::string("V-cycle capture: ") + cudaGetErrorString(e));
        const cudaError_t e2 = cudaGraphInstantiate(&H.vgraph[slot], g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) {
            H.vgraph[slot] = nullptr;
            return c->fail(IBM_ERR_CUDA, std::string("V-cycle graph instantiation: ") + cudaGetErrorString(e2));
        }
        H.vgraph_out[slot] = out;
        H.vgraph_kernels = c->nlaunch - n0;
        c->nlaunch = n0;   // counted when the graph runs
    }
    IBM_CUDA(c, cudaGraphLaunch(H.vgraph[slot], c->s));
    c->nlaunch += H.vgraph_kernels;
    return IBM_OK;
}

// Scheduled relaxation Jacobi on the staircase operator K of level 0:
// x_new = x + w (f + sum T x_nb - D x) / D on active cells, from x = 0, with
// relaxation factors w_k = 1 / tau_k, tau_k the Chebyshev points of
// [lmin, 2] (the Jacobi-scaled spectrum of K lies in [0, 2]), taken in
// bit-reversed order so large and small factors alternate. A fixed linear
// operator: usable as the right preconditioner of BiCGStab.
template <typename T, bool FINE>
__global__ void k_srj_sweep(MGLevel<T> L, const T *__restrict__ f, const T *__restrict__ x, T *__restrict__ xn, T w) {
    GRID_STRIDE(c, L.n) {
        T v = T(0);
        if (active<T, FINE>(L, c)) {
            const uint32_t t = L.fnx.div((uint32_t)c);
            const int i = (int)((uint32_t)c - t * (uint32_t)L.nx);
            const uint32_t kk = L.fny.div(t);
            const int j = (int)(t - kk * (uint32_t)L.ny), k = (int)kk;
            T d;
            const T s = k_offdiag<T, FINE>(L, x, c, i, j, k, d);
            if (!FINE) d = L.d[c];
            const T xc = x[c];
            v = d > T(0) ? xc + w * ((f[c] + s) / d - xc) : xc;
        }
        xn[c] = v;
    }
}

std::vector<double> srj_factors(int m, double lmin) {
    if (!(lmin > 0.0)) lmin = 2.0 / ((double)m * m);
    const double lmax = 2.0, pi = 3.14159265358979323846;
    std::vector<double> w(m);
    for (int k = 0; k < m; ++k) {
        const double tau = 0.5 * (lmax + lmin) + 0.5 * (lmax - lmin) * cos(pi * (2.0 * k + 1.0) / (2.0 * m));
        w[k] = 1.0 / tau;
    }
    // bit-reversed order when m is a power of two
    if ((m & (m - 1)) == 0) {
        int bits = 0;
        while ((1 << bits) < m) ++bits;
        std::vector<double> o(m);
        for (int k = 0; k < m; ++k) {
            int r = 0;
            for (int b = 0; b < bits; ++b)
                if (k & (1 << b)) r |= 1 << (bits - 1 - b);
            o[r] = w[k];
        }
        return o;
    }
    return w;
}

template <typename T>
static ibm_status srj(Ctx *c, MGHier<T> &H, const T *f, T **out) {
    MGLevel<T> &L = H.lv[0];
    const std::vector<double> w = srj_factors(c->opts.srj_sweeps, c->opts.srj_lmin);
    T *x = H.px, *xn = H.pz;
    IBM_CUDA(c, cudaMemsetAsync(x, 0, sizeof(T) * (size_t)c->N, c->s));
    for (size_t k = 0; k < w.size(); ++k) {
        if (H.fine0) KL(K_RBGS0, (k_srj_sweep<T, true>), nblk(c->N), 256, L, f, x, xn, (T)w[k]);
        else KL(K_RBGS0, (k_srj_sweep<T, false>), nblk(c->N), 256, L, f, x, xn, (T)w[k]);
        T *t = x;
        x = xn;
        xn = t;
    }
    IBM_LAUNCHED(c);
    *out = x;
    return IBM_OK;
}

// MG-PCG with a fixed number of iterations: K x = f, with f in H.pr on
// entry (it becomes the residual); the solution is left in H.px
template <typename T>
static ibm_status pcg(Ctx *c, MGHier<T> &H, int iters) {
    const int64_t n = c->N;
    MGLevel<T> &L0 = H.lv[0];
    IBM_CUDA(c, cudaMemsetAsync(H.px, 0, sizeof(T) * (size_t)n, c->s));
    IBM_TRY(vcycle(c, H, H.pr, H.pz));
    IBM_CUDA(c, cudaMemcpyAsync(H.pp, H.pz, sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, c->s));
    KL(-1, k_dot<T>, c->nred, RED_THREADS, n, H.pr, H.pz, c->part);
    IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + S_RZ));
    for (int it = 0; it < iters; ++it) {
        if (H.fine0) KL(K_SPMV0, (k_spmv_dot<T, true>), c->nred, RED_THREADS, L0, H.pp, H.pq, c->part);
        else KL(K_SPMV0, (k_spmv_dot<T, false>), c->nred, RED_THREADS, L0, H.pp, H.pq, c->part);
        IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + S_PQ));
        KL(-1, k_alpha, 1, 1, c->scal);
        KL(-1, k_axpy2<T>, c->nred_wide, RED_THREADS, n, H.px, H.pr, H.pp, H.pq, c->scal);
        IBM_LAUNCHED(c);
        if (it + 1 < iters) {
            IBM_TRY(vcycle(c, H, H.pr, H.pz));
            KL(-1, k_dot<T>, c->nred, RED_THREADS, n, H.pr, H.pz, c->part);
            IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + S_RZN));
            KL(-1, k_beta, 1, 1, c->scal);
            KL(-1, k_pupd<T>, c->nred_wide, RED_THREADS, n, H.pp, H.pz, c->scal);
            IBM_LAUNCHED(c);
        }
    }
    return IBM_OK;
}

// z = M^{-1} v, vectors and multigrid in precision T
template <typename T>
static ibm_status precond(Ctx *c, MGHier<T> &H, const T *v, T *z) {
    const OpT<T> oin = op_of<T>(c);
    if constexpr (sizeof(T) == 4) {
        if (c->g.nx % 4 == 0 && al16(v) && al16(H.pr))
            KL(-1, k_pre_in4, c->nred_wide, RED_THREADS, c->g, oin, c->type, v, H.pr);
        else
            KL(-1, k_pre_in<T>, c->nred_wide, RED_THREADS, c->g, oin, c->type, v, H.pr);
    } else {
        KL(-1, k_pre_in<T>, c->nred_wide, RED_THREADS, c->g, oin, c->type, v, H.pr);
    }
    IBM_LAUNCHED(c);
    const T *xin = H.px;
    if (c->opts.precond == 1) {
        T *xo = nullptr;
        IBM_TRY(srj(c, H, H.pr, &xo));
        xin = xo;
    } else if (c->opts.inner_iters == 1 && c->opts.outer == IBM_OUTER_FGMRES) {
        // one CG step is alpha times one V-cycle; FGMRES is invariant to
        // that scalar, so the V-cycle output is used directly. On large
        // grids it is written straight into z: the V-cycle leaves every cell
        // outside the active (FLUID) set at zero, so the copy below would be
        // the identity (small grids keep one buffer and one graph)
        T *xo = c->N >= (int64_t)1 << 20 ? z : H.pz;
        // (the legacy default stream cannot be captured: launched directly there)
        if (c->opts.graph == 1 && !c->kt.on && !c->capturing && c->s != nullptr && c->s != cudaStreamLegacy)
            IBM_TRY(vcycle_graph(c, H, xo));
        else IBM_TRY(vcycle(c, H, H.pr, xo));
        xin = xo;
    } else {
        IBM_TRY(pcg(c, H, c->opts.inner_iters));
    }
    if (xin != z) {
        KL(-1, k_pre_out<T>, c->nred_wide, RED_THREADS, c->N, c->type, xin, z);
        IBM_LAUNCHED(c);
    }
    const OpT<T> o = op_of<T>(c);
    if (c->ng > 0) {
        KL(-1, k_pre_ghost<T>, (unsigned)((c->ng + 255) / 256), 256, c->gh, o.wp, c->type, v, z);
        IBM_LAUNCHED(c);
    }
    if (c->nband > 0 && c->opts.band_sweeps > 0 && c->nband <= (int64_t)BAND_BLOCK * BAND_PER_THREAD) {
        KL(-1, k_band_block<T>, 1, BAND_BLOCK, c->g, c->gh, o, c->nband, c->band, c->band_g, v, z,
           (T)c->opts.band_omega, c->opts.band_sweeps);
        IBM_LAUNCHED(c);
    } else if (c->nband > 0) {
        // (btmp holds nband doubles: room for either precision)
        const unsigned gb = (unsigned)((c->nband + 255) / 256);
        T *tmp = reinterpret_cast<T *>(c->btmp);
        for (int s = 0; s < c->opts.band_sweeps; ++s) {
            KL(-1, k_band_jacobi<T>, gb, 256, c->g, c->gh, o, c->nband, c->band, c->band_g, v, (const T *)z,
               (T)c->opts.band_omega, tmp);
            KL(-1, k_band_scatter<T>, gb, 256, c->nband, c->band, (const T *)tmp, z);
            IBM_LAUNCHED(c);
        }
    }
    return IBM_OK;
}

// ||x||^2 over all cells (FP64 accumulation)
template <typename T>
static ibm_status norm2(Ctx *c, const T *x, double *out) {
    KL(-1, k_dotT<T>, c->nred, RED_THREADS, c->N, x, x, c->part);
    IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + S_TMP));
    IBM_TRY(sync_scalars(c, S_TMP + 1));
    *out = c->hscal[S_TMP];
    return IBM_OK;
}

template <typename T>
struct Krylov {
    std::vector<T *> V, Z;
    T **Vdev, **Zdev;
    T *w, *r;
    MGHier<T> *H;
};
static Krylov<double> kry64(Ctx *c) { return Krylov<double>{c->V, c->Z, c->Vdev, c->Zdev, c->w, c->rr, &c->mg64}; }
static Krylov<float> kry32(Ctx *c) { return Krylov<float>{c->V32, c->Z32, c->Vdev32, c->Zdev32, c->w32, c->r32, &c->mg32}; }

// Restarted FGMRES in precision T on P A x = b, x in/out. Stops at
// ||P(b - A x)|| <= rtol * bnorm, after maxit steps, or (single_cycle)
// after one restart cycle. Dot products accumulate in FP64.
template <typename T>
static ibm_status fgmres(Ctx *c, Krylov<T> K, T *x, const T *b, double bnorm, double rtol, int maxit,
                         bool single_cycle, int *outer_out, int *inner_out, double *rel_out) {
    const int64_t n = c->N;
    const int m = c->opts.restart;
    int outer = 0, inner = 0;
    double rel = 0.0;
    ibm_status status = IBM_OK;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
    bool done = false;
    int cycles = 0;
    while (!done) {
        IBM_TRY(apply_PA<T>(c, x, b, T(-1), K.r));
        double rn2;
        IBM_TRY(norm2<T>(c, K.r, &rn2));
        const double beta = sqrt(rn2);
        rel = beta / bnorm;
        if (!isfinite(rel)) { status = c->fail(IBM_ERR_DIVERGED, "Poisson residual is not finite"); break; }
        if (rel <= rtol || (single_cycle && cycles > 0)) break;
        if (outer >= maxit) { status = IBM_ERR_NOT_CONVERGED; break; }
        ++cycles;
        KL(-1, (k_scale<T, T>), c->nred_wide, RED_THREADS, n, K.V[0], K.r, 1.0 / beta);
        IBM_LAUNCHED(c);
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int jlast = -1;
        for (int j = 0; j < m && outer < maxit; ++j) {
            IBM_TRY(precond<T>(c, *K.H, K.V[j], K.Z[j]));
            inner += c->opts.inner_iters;
            IBM_TRY(apply_PA<T>(c, K.Z[j], nullptr, T(1), K.w));
            // classical Gram-Schmidt, with a second pass when the norm drops
            // below reorth_eta (default 0.3) of its value (the test of Daniel,
            // Gragg, Kaufman and Stewart 1976, with a looser threshold)
            VPtrs<T> vp{};
            for (int i = 0; i <= j; ++i) vp.p[i] = K.V[i];
            double hcol[17] = {0};
            double wbefore2 = 0.0, wafter2 = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                KL(K_MDOT, mdot_table<T>(std::make_integer_sequence<int, 17>())[j], mdot_blocks<T>(c), RED_THREADS,
                   n, K.w, vp, c->part);
                IBM_TRY(finalize(c, c->part, mdot_blocks<T>(c), j + 1, 1.0, c->scal + S_MD));
                IBM_TRY(sync_scalars(c, S_MD + j + 1));
                Coef h{};
                double h2 = 0.0;
                for (int i = 0; i <= j; ++i) {
                    h.v[i] = c->hscal[S_MD + i];
                    h2 += h.v[i] * h.v[i];
                }
                KL(K_ORTH, orth_table<T>(std::make_integer_sequence<int, 17>())[j], c->nred, RED_THREADS, n,
                   K.w, vp, h, c->part);
                IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + S_TMP));
                IBM_TRY(sync_scalars(c, S_TMP + 1));
                wafter2 = c->hscal[S_TMP];
                // ||w||^2 before the pass, from the orthogonal decomposition
                wbefore2 = wafter2 + h2;
                for (int i = 0; i <= j; ++i) hcol[i] += h.v[i];
                const double eta = c->opts.reorth_eta;
                if (!(wafter2 <= eta * eta * wbefore2)) break;
            }
            const double hn = sqrt(wafter2);
            ++outer;
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
            H[(size_t)(j + 1) * m + j] = hn;
            if (!isfinite(hn)) { status = c->fail(IBM_ERR_DIVERGED, "FGMRES breakdown (non-finite)"); done = true; break; }
            for (int i = 0; i < j; ++i) {
                const double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
            }
            const double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
            const double rho = hypot(a, bb);
            cs[j] = rho > 0 ? a / rho : 1.0;
            sn[j] = rho > 0 ? bb / rho : 0.0;
            H[(size_t)j * m + j] = rho;
            H[(size_t)(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            jlast = j;
            const double est = fabs(gv[j + 1]) / bnorm;
            if (hn > 0.0 && j + 1 < m) {
                KL(-1, (k_scale<T, T>), c->nred_wide, RED_THREADS, n, K.V[j + 1], K.w, 1.0 / hn);
                IBM_LAUNCHED(c);
            }
            if (est <= rtol || hn == 0.0) break;
        }
        if (done) break;
        if (jlast < 0) { status = IBM_ERR_NOT_CONVERGED; break; }
        for (int i = jlast; i >= 0; --i) {
            double sacc = gv[i];
            for (int k = i + 1; k <= jlast; ++k) sacc -= H[(size_t)i * m + k] * y[k];
            y[i] = sacc / H[(size_t)i * m + i];
        }
        Coef yc{};
        for (int i = 0; i <= jlast; ++i) yc.v[i] = y[i];
        KL(-1, k_xupd<T>, c->nred_wide, RED_THREADS, n, x, (const T *const *)K.Zdev, jlast + 1, yc);
        IBM_LAUNCHED(c);
    }
    *outer_out = outer;
    *inner_out = inner;
    *rel_out = rel;
    return status;
}

static ibm_status apply_prec(Ctx *c, const double *v, double *z);

// FP32 storage of mixed mode: operator coefficients, ghost weights, Krylov
// vectors (allocated on first use)
__global__ void k_to_float(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
    GRID_STRIDE(q, n) b[q] = (float)a[q];
}
static ibm_status ensure_mixed(Ctx *c) {
    if (!c->op32[0]) {
        const double *src[12] = {c->g.cxm, c->g.cxp, c->g.cxs, c->g.cym, c->g.cyp, c->g.cys,
                                 c->g.czm, c->g.czp, c->g.czs, c->g.dx, c->g.dy, c->g.dz};
        const int64_t len[12] = {c->nx, c->nx, c->nx, c->ny, c->ny, c->ny, c->nz, c->nz, c->nz, c->nx, c->ny, c->nz};
        for (int q = 0; q < 12; ++q) {
            c->op32[q] = (float *)dev_alloc(c, sizeof(float) * len[q]);
            if (!c->op32[q]) return c->fail(IBM_ERR_OOM, "FP32 coefficient allocation failed");
            KL(-1, k_to_float, 1, 256, len[q], src[q], c->op32[q]);
        }
        IBM_LAUNCHED(c);
    }
    if (c->wp32_n != c->ng) {
        dev_free(c, c->wp32);
        c->wp32 = (float *)dev_alloc(c, sizeof(float) * 8 * (c->ng > 0 ? c->ng : 1));
        if (!c->wp32) return c->fail(IBM_ERR_OOM, "FP32 weight allocation failed");
        if (c->ng > 0) KL(-1, k_to_float, nblk(8 * c->ng), 256, 8 * c->ng, c->wp, c->wp32);
        IBM_LAUNCHED(c);
        c->wp32_n = c->ng;
    }
    const int m = c->opts.restart;
    if (m > c->m32_cap) {
        for (float *p : c->V32) dev_free(c, p);
        for (float *p : c->Z32) dev_free(c, p);
        c->V32.assign(m + 1, nullptr);
        c->Z32.assign(m, nullptr);
        for (int i = 0; i <= m; ++i)
            if (!(c->V32[i] = (float *)dev_alloc(c, sizeof(float) * c->N))) return c->fail(IBM_ERR_OOM, "FP32 Krylov allocation failed");
        for (int i = 0; i < m; ++i)
            if (!(c->Z32[i] = (float *)dev_alloc(c, sizeof(float) * c->N))) return c->fail(IBM_ERR_OOM, "FP32 Krylov allocation failed");
        if (!c->Vdev32) c->Vdev32 = (float **)dev_alloc(c, sizeof(float *) * 17);
        if (!c->Zdev32) c->Zdev32 = (float **)dev_alloc(c, sizeof(float *) * 17);
        if (!c->w32) c->w32 = (float *)dev_alloc(c, sizeof(float) * c->N);
        if (!c->r32) c->r32 = (float *)dev_alloc(c, sizeof(float) * c->N);
        if (!c->d32) c->d32 = (float *)dev_alloc(c, sizeof(float) * c->N);
        if (!c->b32) c->b32 = (float *)dev_alloc(c, sizeof(float) * c->N);
        if (!c->Vdev32 || !c->Zdev32 || !c->w32 || !c->r32 || !c->d32 || !c->b32)
            return c->fail(IBM_ERR_OOM, "FP32 Krylov allocation failed");
        IBM_CUDA(c, cudaMemcpyAsync(c->Vdev32, c->V32.data(), sizeof(float *) * (m + 1), cudaMemcpyHostToDevice, c->s));
        IBM_CUDA(c, cudaMemcpyAsync(c->Zdev32, c->Z32.data(), sizeof(float *) * m, cudaMemcpyHostToDevice, c->s));
        IBM_CUDA(c, cudaStreamSynchronize(c->s));
        c->m32_cap = m;
    }
    return IBM_OK;
}

// Mixed mode: FP64 defect correction around FP32 FGMRES cycles.
//   r = P(b - A phi) in FP64; stop at ||r|| <= rtol ||b||;
//   solve P A d = r / ||r|| approximately in FP32 (one FGMRES cycle, or
//   until a reduction of mixed_inner_rtol); phi += ||r|| d in FP64.
static ibm_status mixed_refinement(Ctx *c, double *phi, double bnorm, double rtol, int maxit, int *outer_out,
                                   int *inner_out, double *rel_out) {
    IBM_TRY(ensure_mixed(c));
    const int64_t n = c->N;
    int steps = 0, inner = 0, refinements = 0, stalls = 0;
    double rel = 0.0, last_rel = 1e300;
    ibm_status status = IBM_OK;
    while (true) {
        IBM_TRY(apply_PA<double>(c, phi, c->b, -1.0, c->rr));
        double rn2;
        IBM_TRY(norm2<double>(c, c->rr, &rn2));
        const double rn = sqrt(rn2);
        rel = rn / bnorm;
        if (!isfinite(rel)) return c->fail(IBM_ERR_DIVERGED, "Poisson residual is not finite");
        if (rel <= rtol) break;
        if (steps >= maxit || refinements >= 256) { status = IBM_ERR_NOT_CONVERGED; break; }
        ++refinements;
        KL(-1, (k_scale<float, double>), c->nred_wide, RED_THREADS, n, c->b32, c->rr, 1.0 / rn);
        IBM_CUDA(c, cudaMemsetAsync(c->d32, 0, sizeof(float) * n, c->s));
        IBM_LAUNCHED(c);
        // inner target: the FP64 goal, but no tighter than FP32 can reach
        const double target = fmax(c->opts.mixed_inner_rtol, 0.5 * rtol / rel);
        int o = 0, in = 0;
        double irel = 0.0;
        // one FP32 restart cycle per refinement: an FP32 solve cannot always
        // reach the target at this conditioning, and the FP64 residual of
        // the next pass measures what it did achieve
        ibm_status s = fgmres<float>(c, kry32(c), c->d32, c->b32, 1.0, target, maxit - steps, true, &o, &in, &irel);
        if (s != IBM_OK && s != IBM_ERR_NOT_CONVERGED) return s;
        if (getenv("IBM_TRACE"))
            fprintf(stderr, "[ibm] refinement %d: rel %.3e target %.3e fgmres32 steps %d rel32 %.3e status %d\n",
                    refinements, rel, target, o, irel, (int)s);
        steps += o;
        inner += in;
        KL(-1, k_fluid_volsum32, c->nred, RED_THREADS, c->g, op_of<float>(c), c->type, c->d32, c->part);
        IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN));
        KL(-1, k_add_scaled, c->nred_wide, RED_THREADS, n, c->type, phi, c->d32, rn, c->scal + S_MEAN);
        IBM_LAUNCHED(c);
        if (o == 0) { status = IBM_ERR_NOT_CONVERGED; break; }
        if (refinements > 1 && !(rel < 0.999 * last_rel)) stalls++;
        else stalls = 0;
        if (stalls >= 3) { status = c->fail(IBM_ERR_NOT_CONVERGED, "mixed-precision refinement stalled"); break; }
        last_rel = rel;
    }
    *outer_out = steps;
    *inner_out = inner;
    *rel_out = rel;
    return status;
}

static ibm_status apply_prec(Ctx *c, const double *v, double *z) {
    if (c->opts.precision == IBM_MIXED) {
        // FP64 vectors through the FP32 multigrid: convert in and out
        IBM_TRY(ensure_mixed(c));
        KL(-1, (k_scale<float, double>), c->nred_wide, RED_THREADS, c->N, c->b32, v, 1.0);
        IBM_TRY(precond<float>(c, c->mg32, c->b32, c->d32));
        KL(-1, (k_scale<double, float>), c->nred_wide, RED_THREADS, c->N, z, c->d32, 1.0);
        IBM_LAUNCHED(c);
        return IBM_OK;
    }
    return precond<double>(c, c->mg64, v, z);
}

// BiCGStab (van der Vorst 1992) with right preconditioning; scalars stay on
// the device; one host synchronisation per iteration for the stopping test.
// A breakdown (rho, (rh, v) or omega zero) restarts from the true residual.
static ibm_status bicgstab(Ctx *c, double *phi, double bnorm, double rtol, int maxit, int *outer_out,
                           int *inner_out, double *rel_out) {
    const int64_t n = c->N;
    double *r = c->V[0], *rh = c->V[1], *p = c->V[2], *v = c->V[3], *sv = c->V[4], *t = c->V[5];
    double *ph = c->Z[0], *shv = c->Z[1];
    int it = 0, inner = 0;
    double rel = 1.0;
    ibm_status status = IBM_OK;
    bool fresh = true;
    while (true) {
        if (fresh) {
            // true residual
            IBM_TRY(apply_PA<double>(c, phi, c->b, -1.0, r));
            double rn2;
            IBM_TRY(norm2<double>(c, r, &rn2));
            rel = sqrt(rn2) / bnorm;
            if (!isfinite(rel)) return c->fail(IBM_ERR_DIVERGED, "Poisson residual is not finite");
            if (rel <= rtol) break;
            if (it >= maxit) { status = IBM_ERR_NOT_CONVERGED; break; }
            IBM_CUDA(c, cudaMemcpyAsync(rh, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
            IBM_CUDA(c, cudaMemsetAsync(p, 0, sizeof(double) * n, c->s));
            IBM_CUDA(c, cudaMemsetAsync(v, 0, sizeof(double) * n, c->s));
            KL(-1, k_bicg_init, 1, 1, c->scal);
            IBM_LAUNCHED(c);
            fresh = false;
        }
        // rho1 = (rh, r); beta; p = r + beta (p - omega v)
        KL(-1, k_dot64, c->nred, RED_THREADS, n, rh, r, c->part);
        IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + B_RHO1));
        KL(-1, k_bicg_beta, 1, 1, c->scal);
        KL(-1, k_bicg_p, c->nred_wide, RED_THREADS, n, r, p, v, c->scal);
        IBM_LAUNCHED(c);
        IBM_TRY(apply_prec(c, p, ph));
        IBM_TRY(apply_PA<double>(c, ph, nullptr, 1.0, v));
        KL(-1, k_dot64, c->nred, RED_THREADS, n, rh, v, c->part);
        IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + B_DEN));
        KL(-1, k_bicg_alpha, 1, 1, c->scal);
        KL(-1, k_bicg_s, c->nred_wide, RED_THREADS, n, r, v, sv, c->scal);
        IBM_LAUNCHED(c);
        IBM_TRY(apply_prec(c, sv, shv));
        IBM_TRY(apply_PA<double>(c, shv, nullptr, 1.0, t));
        KL(-1, k_bicg_tdots, c->nred, RED_THREADS, n, t, sv, c->part);
        IBM_TRY(finalize(c, c->part, c->nred, 2, 1.0, c->scal + B_TS));
        KL(-1, k_bicg_omega, 1, 1, c->scal);
        KL(-1, k_bicg_xr, c->nred, RED_THREADS, n, phi, ph, shv, r, sv, t, c->scal, c->part);
        IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + S_TMP));
        IBM_LAUNCHED(c);
        inner += 2 * c->opts.inner_iters;
        ++it;
        IBM_TRY(sync_scalars(c, B_FLAG + 1));
        const double rr = sqrt(c->hscal[S_TMP]) / bnorm;
        if (!isfinite(rr)) return c->fail(IBM_ERR_DIVERGED, "Poisson residual is not finite");
        // converged by the recurrence, breakdown or limit: check the true residual
        if (rr <= rtol || c->hscal[B_FLAG] != 0.0 || it >= maxit) fresh = true;
    }
    *outer_out = it;
    *inner_out = inner;
    *rel_out = rel;
    return status;
}

// Solve P A phi = P rhs. rhs: FLUID rows read; phi: guess in, solution out.
// ---------------------------------------------------------------------------
// Device-controlled Poisson solve (captured into the step graph)
//
// The same FGMRES(m) and mixed-precision refinement as above, with every
// decision taken on the device: the Hessenberg column, Givens rotations,
// residual estimate, restart and stopping tests run in one-thread kernels
// on a control block in device memory, and the loops are conditional graph
// nodes (a WHILE node per restart loop, an IF node per Arnoldi step and per
// re-orthogonalisation pass) whose conditions those kernels set.
// ---------------------------------------------------------------------------

struct DevFG {
    double H[17 * 16], cs[16], sn[16], g[17], y[16], hcol[17];
    double beta, bnorm, rtol, rel, scale, wb, wa;
    int outer, maxit, jlast, active, reorth, go, cycles, single, status, ncols, zero;
    // mixed-precision refinement (outer block only)
    double rn, last_rel, inner_rtol;
    int refinements, stalls, steps, stop;
};

// statistics accumulated by the step graphs over one ibm_step call
struct DevStats {
    int steps, outer, helm_sweeps, status;
    double rel;
};

static DevFG *dfg(Ctx *c, int i) { return reinterpret_cast<DevFG *>(c->dctl) + i; }

ibm_status cond_handle(Ctx *c, cudaGraphConditionalHandle *h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    IBM_CUDA(c, cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive || !g) return c->fail(IBM_ERR_CUDA, "conditional handle outside capture");
    IBM_CUDA(c, cudaGraphConditionalHandleCreate(h, g, 0, cudaGraphCondAssignDefault));
    return IBM_OK;
}

// add an IF/WHILE node with handle h at the capture point of c->s and
// capture its body on a side stream until cond_close
ibm_status cond_open(Ctx *c, cudaGraphConditionalNodeType type, cudaGraphConditionalHandle h, CondScope *sc) {
    if (c->side_depth >= 8 || !c->side[c->side_depth]) return c->fail(IBM_ERR_ARG, "conditional nesting too deep");
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    IBM_CUDA(c, cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &g, &deps, &ed, &nd));
    if (cs != cudaStreamCaptureStatusActive || !g) return c->fail(IBM_ERR_CUDA, "conditional node outside capture");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    IBM_CUDA(c, cudaGraphAddNode(&node, g, deps, ed, nd, &p));
    IBM_CUDA(c, cudaStreamUpdateCaptureDependencies(c->s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t side = c->side[c->side_depth];
    IBM_CUDA(c, cudaStreamBeginCaptureToGraph(side, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
    ++c->side_depth;
    sc->outer = c->s;
    c->s = side;
    return IBM_OK;
}

ibm_status cond_close(Ctx *c, CondScope *sc) {
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->s, &g);
    c->s = sc->outer;
    --c->side_depth;
    if (e != cudaSuccess) return c->fail(IBM_ERR_CUDA, std::string("conditional body capture: ") + cudaGetErrorString(e));
    return IBM_OK;
}

__global__ void k_set_cond(cudaGraphConditionalHandle h, const int *flag) { cudaGraphSetConditional(h, *flag ? 1u : 0u); }

template <typename T, typename S>
__global__ void k_scale_dev(int64_t n, T *__restrict__ dst, const S *__restrict__ src, const double *__restrict__ a) {
    const double f = *a;
    if constexpr (sizeof(T) == 4 && sizeof(S) == 4) scale_f32(n, dst, src, (float)f);
    else GRID_STRIDE(c, n) dst[c] = (T)(f * (double)src[c]);
}

// w -= sum_q h_q V_q with h in device memory; partial (w, w)
template <typename T, int NC>
__global__ void __launch_bounds__(RED_THREADS) k_orth_dev(int64_t n, T *__restrict__ w, VPtrs<T> V,
                                                          const double *__restrict__ h, double *__restrict__ part) {
    typedef typename Acc<T>::type A;
    typedef typename Vec16<T>::type VT;
    constexpr int W = Vec16<T>::W;
    __shared__ double sh[32];
    T hv[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) hv[q] = (T)h[q];
    A ww = A(0);
    const int64_t nv = n / W;
    GRID_STRIDE(v, nv) {
        VT a = reinterpret_cast<const VT *>(w)[v];
        VT b[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) b[q] = reinterpret_cast<const VT *>(V.p[q])[v];
#pragma unroll
        for (int q = 0; q < NC; ++q)
#pragma unroll
            for (int e = 0; e < W; ++e) vset(a, e, vget(a, e) - hv[q] * vget(b[q], e));
        reinterpret_cast<VT *>(w)[v] = a;
        if constexpr (sizeof(T) == 4) {
            T leaf = T(0);
#pragma unroll
            for (int e = 0; e < W; ++e) leaf += vget(a, e) * vget(a, e);
            ww += (A)leaf;
        } else {
#pragma unroll
            for (int e = 0; e < W; ++e) ww += (A)vget(a, e) * (A)vget(a, e);
        }
    }
    for (int64_t c = nv * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        T a = w[c];
#pragma unroll
        for (int q = 0; q < NC; ++q) a -= hv[q] * V.p[q][c];
        w[c] = a;
        ww += (A)(a * a);
    }
    const double t = block_sum<RED_THREADS>(ww, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <typename T>
using OrthDevFn = void (*)(int64_t, T *, VPtrs<T>, const double *, double *);
template <typename T, int... I>
static const OrthDevFn<T> *orth_dev_table(std::integer_sequence<int, I...>) {
    static const OrthDevFn<T> t[] = {&k_orth_dev<T, I + 1>...};
    return t;
}

// x += sum_{q < ncols} y_q Z_q with y and ncols from the control block
template <typename T>
__global__ void k_xupd_dev(int64_t n, T *__restrict__ x, VPtrs<T> Z, const DevFG *__restrict__ F) {
    const int nc = F->ncols;
    if (nc <= 0) return;
    T yv[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) yv[q] = q < nc ? (T)F->y[q] : T(0);
    GRID_STRIDE(c, n) {
        T a = x[c];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (q < nc) a += yv[q] * Z.p[q][c];
        x[c] = a;
    }
}

__global__ void k_zero_if(int64_t n, double *__restrict__ x, const int *__restrict__ flag) {
    if (!*flag) return;
    GRID_STRIDE(c, n) x[c] = 0.0;
}

// phi += rn * ((double) d - mean) on FLUID and GHOST cells, rn from the control block
__global__ void k_add_scaled_dev(int64_t n, const uint8_t *__restrict__ type, double *__restrict__ phi,
                                 const float *__restrict__ d, const DevFG *__restrict__ R,
                                 const double *__restrict__ mean) {
    const double a = R->rn, m = *mean;
    GRID_STRIDE(c, n) if (type[c] != DEAD) phi[c] += a * ((double)d[c] - m);
}

__global__ void k_fg_setup(DevFG *F, const double *bn2, double rtol, int maxit) {
    const double bnorm = sqrt(*bn2);
    F->bnorm = bnorm;
    // a non-finite right-hand side is reported, not solved (phi is zeroed)
    const bool bad = !isfinite(bnorm);
    F->zero = bad || !(bnorm > 1e-300);
    F->rtol = rtol;
    F->maxit = maxit;
    F->outer = 0;
    F->cycles = 0;
    F->single = 0;
    F->status = bad ? IBM_ERR_DIVERGED : 0;
    F->rel = 0.0;
    F->refinements = 0;
    F->stalls = 0;
    F->steps = 0;
    F->stop = 0;
    F->last_rel = 1e300;
    F->ncols = 0;
}

__global__ void k_copy_inner_rtol(DevFG *R, double v) { R->inner_rtol = v; }

// restart test at the top of a cycle: beta = ||r||, rel = beta / bnorm
__global__ void k_fg_cycle(DevFG *F, const double *rn2, cudaGraphConditionalHandle h) {
    const double beta = sqrt(*rn2);
    F->rel = F->zero ? 0.0 : beta / F->bnorm;
    if (!isfinite(F->rel)) F->status = IBM_ERR_DIVERGED;
    int go = !F->zero && F->status == 0 && F->rel > F->rtol && !(F->single && F->cycles > 0);
    if (go && F->outer >= F->maxit) {
        go = 0;
        F->status = IBM_ERR_NOT_CONVERGED;
    }
    F->go = go;
    if (go) {
        F->cycles += 1;
        for (int i = 0; i < 17; ++i) F->g[i] = 0.0;
        F->g[0] = beta;
        F->scale = 1.0 / beta;
        F->jlast = -1;
        F->active = 1;
        F->ncols = 0;
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// after the first Gram-Schmidt pass of step j: h in md[0..j], ||w||^2 after
// in *wa2; a second pass when ||w||^2 dropped to eta2 of its value before the
// pass (||w_after||^2 + sum h^2) or below
__global__ void k_fg_post1(DevFG *F, const double *md, const double *wa2, int j, double eta2) {
    double h2 = 0.0;
    for (int i = 0; i <= j; ++i) {
        F->hcol[i] = md[i];
        h2 += md[i] * md[i];
    }
    F->wa = *wa2;
    F->wb = F->wa + h2;   // ||w||^2 before the pass, from the orthogonal decomposition
    F->reorth = F->wa <= eta2 * F->wb;
}

__global__ void k_fg_post2(DevFG *F, const double *md, const double *wa2, int j) {
    for (int i = 0; i <= j; ++i) F->hcol[i] += md[i];
    F->wa = *wa2;
}

// Hessenberg column j, Givens rotations, residual estimate and the decision
// to take step j + 1
__global__ void k_fg_givens(DevFG *F, int j, int m) {
    const double hn = sqrt(F->wa);
    F->outer += 1;
    double *H = F->H;
    for (int i = 0; i <= j; ++i) H[i * m + j] = F->hcol[i];
    H[(j + 1) * m + j] = hn;
    if (!isfinite(hn)) {
        F->status = IBM_ERR_DIVERGED;
        F->active = 0;
        return;
    }
    for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], b = H[(i + 1) * m + j];
        H[i * m + j] = F->cs[i] * a + F->sn[i] * b;
        H[(i + 1) * m + j] = -F->sn[i] * a + F->cs[i] * b;
    }
    const double a = H[j * m + j], b = H[(j + 1) * m + j];
    const double rho = hypot(a, b);
    F->cs[j] = rho > 0 ? a / rho : 1.0;
    F->sn[j] = rho > 0 ? b / rho : 0.0;
    H[j * m + j] = rho;
    H[(j + 1) * m + j] = 0.0;
    F->g[j + 1] = -F->sn[j] * F->g[j];
    F->g[j] = F->cs[j] * F->g[j];
    F->jlast = j;
    const double est = fabs(F->g[j + 1]) / F->bnorm;
    F->scale = hn > 0.0 ? 1.0 / hn : 0.0;
    F->active = !(est <= F->rtol || hn == 0.0) && F->outer < F->maxit && j + 1 < m;
}

// back substitution H y = g over the steps taken
__global__ void k_fg_ysolve(DevFG *F, int m) {
    const int jl = F->jlast;
    if (F->status != 0 || jl < 0) {
        if (F->status == 0) F->status = IBM_ERR_NOT_CONVERGED;
        F->ncols = 0;
        return;
    }
    for (int i = jl; i >= 0; --i) {
        double s = F->g[i];
        for (int k = i + 1; k <= jl; ++k) s -= F->H[i * m + k] * F->y[k];
        F->y[i] = s / F->H[i * m + i];
    }
    F->ncols = jl + 1;
}

// refinement test: rel = ||P(b - A phi)|| / ||b||; sets up the FP32 cycle
__global__ void k_ref_start(DevFG *R, DevFG *F, const double *rn2, cudaGraphConditionalHandle h) {
    const double rn = sqrt(*rn2);
    R->rn = rn;
    R->rel = R->zero ? 0.0 : rn / R->bnorm;
    if (!isfinite(R->rel)) R->status = IBM_ERR_DIVERGED;
    int go = !R->zero && R->status == 0 && !R->stop && R->rel > R->rtol;
    if (go && (R->steps >= R->maxit || R->refinements >= 256)) {
        go = 0;
        R->status = IBM_ERR_NOT_CONVERGED;
    }
    if (go) {
        R->refinements += 1;
        R->scale = 1.0 / rn;
        F->bnorm = 1.0;
        F->zero = 0;
        F->rtol = fmax(R->inner_rtol, 0.5 * R->rtol / R->rel);
        F->maxit = R->maxit - R->steps;
        F->outer = 0;
        F->cycles = 0;
        F->single = 1;
        F->status = 0;
        F->ncols = 0;
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_ref_after(DevFG *R, const DevFG *F) {
    R->steps += F->outer;
    if (F->outer == 0) {
        R->status = IBM_ERR_NOT_CONVERGED;
        R->stop = 1;
        return;
    }
    if (R->refinements > 1 && !(R->rel < 0.999 * R->last_rel)) R->stalls += 1;
    else R->stalls = 0;
    if (R->stalls >= 3) {
        R->status = IBM_ERR_NOT_CONVERGED;
        R->stop = 1;
    }
    R->last_rel = R->rel;
}

// ||x||^2 into scal[slot] without a host read
template <typename T>
static ibm_status norm2_dev(Ctx *c, const T *x, int slot) {
    KL(-1, k_dotT<T>, c->nred, RED_THREADS, c->N, x, x, c->part);
    IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + slot));
    return IBM_OK;
}

// one restart cycle of device-controlled FGMRES on control block F (the
// cycle's residual r must be in K.r and F->scale = 1 / ||r||), then x update
template <typename T>
static ibm_status fgmres_dev_cycle(Ctx *c, Krylov<T> K, T *x, DevFG *F) {
    const int64_t n = c->N;
    const int m = c->opts.restart;
    VPtrs<T> vp{}, zp{};
    for (int i = 0; i <= m && i < 17; ++i) vp.p[i] = K.V[i];
    for (int i = 0; i < m; ++i) zp.p[i] = K.Z[i];
    for (int j = 0; j < m; ++j) {
        cudaGraphConditionalHandle hj, hr;
        IBM_TRY(cond_handle(c, &hj));
        KL(-1, k_set_cond, 1, 1, hj, &F->active);
        CondScope sj;
        IBM_TRY(cond_open(c, cudaGraphCondTypeIf, hj, &sj));
        {
            // V_j = (j == 0 ? r : w) / norm
            KL(-1, (k_scale_dev<T, T>), c->nred_wide, RED_THREADS, n, K.V[j], j == 0 ? K.r : K.w, &F->scale);
            IBM_TRY(precond<T>(c, *K.H, K.V[j], K.Z[j]));
            IBM_TRY(apply_PA<T>(c, K.Z[j], nullptr, T(1), K.w));
            KL(K_MDOT, mdot_table<T>(std::make_integer_sequence<int, 17>())[j], mdot_blocks<T>(c), RED_THREADS, n,
               K.w, vp, c->part);
            IBM_TRY(finalize(c, c->part, mdot_blocks<T>(c), j + 1, 1.0, c->scal + S_MD));
            KL(K_ORTH, orth_dev_table<T>(std::make_integer_sequence<int, 17>())[j], c->nred, RED_THREADS, n, K.w,
               vp, c->scal + S_MD, c->part);
            IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + S_TMP));
            KL(-1, k_fg_post1, 1, 1, F, c->scal + S_MD, c->scal + S_TMP, j,
               c->opts.reorth_eta * c->opts.reorth_eta);
            IBM_TRY(cond_handle(c, &hr));
            KL(-1, k_set_cond, 1, 1, hr, &F->reorth);
            CondScope sr;
            IBM_TRY(cond_open(c, cudaGraphCondTypeIf, hr, &sr));
            {
                KL(K_MDOT, mdot_table<T>(std::make_integer_sequence<int, 17>())[j], mdot_blocks<T>(c), RED_THREADS,
                   n, K.w, vp, c->part);
                IBM_TRY(finalize(c, c->part, mdot_blocks<T>(c), j + 1, 1.0, c->scal + S_MD));
                KL(K_ORTH, orth_dev_table<T>(std::make_integer_sequence<int, 17>())[j], c->nred, RED_THREADS, n,
                   K.w, vp, c->scal + S_MD, c->part);
                IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0, c->scal + S_TMP));
                KL(-1, k_fg_post2, 1, 1, F, c->scal + S_MD, c->scal + S_TMP, j);
            }
            IBM_TRY(cond_close(c, &sr));
            KL(-1, k_fg_givens, 1, 1, F, j, m);
        }
        IBM_TRY(cond_close(c, &sj));
    }
    KL(-1, k_fg_ysolve, 1, 1, F, m);
    KL(-1, k_xupd_dev<T>, c->nred_wide, RED_THREADS, n, x, zp, F);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

// FP64 FGMRES(m) with restarts, all on the device (control block 0)
static ibm_status fgmres64_dev(Ctx *c, double *x, DevFG *F) {
    Krylov<double> K = kry64(c);
    cudaGraphConditionalHandle hw;
    IBM_TRY(cond_handle(c, &hw));
    IBM_TRY(apply_PA<double>(c, x, c->b, -1.0, K.r));
    IBM_TRY(norm2_dev<double>(c, K.r, S_TMP));
    KL(-1, k_fg_cycle, 1, 1, F, c->scal + S_TMP, hw);
    CondScope sw;
    IBM_TRY(cond_open(c, cudaGraphCondTypeWhile, hw, &sw));
    {
        IBM_TRY(fgmres_dev_cycle<double>(c, K, x, F));
        IBM_TRY(apply_PA<double>(c, x, c->b, -1.0, K.r));
        IBM_TRY(norm2_dev<double>(c, K.r, S_TMP));
        KL(-1, k_fg_cycle, 1, 1, F, c->scal + S_TMP, hw);
    }
    IBM_TRY(cond_close(c, &sw));
    return IBM_OK;
}

// FP64 defect correction around one FP32 FGMRES cycle per pass (control
// blocks 0: refinement, 1: FP32 cycle)
static ibm_status mixed_dev(Ctx *c, double *phi, DevFG *R, DevFG *F) {
    const int64_t n = c->N;
    Krylov<float> K = kry32(c);
    cudaGraphConditionalHandle hr;
    IBM_TRY(cond_handle(c, &hr));
    IBM_TRY(apply_PA<double>(c, phi, c->b, -1.0, c->rr));
    IBM_TRY(norm2_dev<double>(c, c->rr, S_TMP));
    KL(-1, k_ref_start, 1, 1, R, F, c->scal + S_TMP, hr);
    CondScope sr;
    IBM_TRY(cond_open(c, cudaGraphCondTypeWhile, hr, &sr));
    {
        KL(-1, (k_scale_dev<float, double>), c->nred_wide, RED_THREADS, n, c->b32, c->rr, &R->scale);
        IBM_CUDA(c, cudaMemsetAsync(c->d32, 0, sizeof(float) * n, c->s));
        // the FP32 cycle: r32 = P(b32 - A d32), then one restart cycle if needed
        cudaGraphConditionalHandle hi;
        IBM_TRY(cond_handle(c, &hi));
        IBM_TRY(apply_PA<float>(c, c->d32, c->b32, -1.0f, K.r));
        IBM_TRY(norm2_dev<float>(c, K.r, S_TMP));
        KL(-1, k_fg_cycle, 1, 1, F, c->scal + S_TMP, hi);
        CondScope si;
        IBM_TRY(cond_open(c, cudaGraphCondTypeIf, hi, &si));
        IBM_TRY(fgmres_dev_cycle<float>(c, K, c->d32, F));
        IBM_TRY(cond_close(c, &si));
        KL(-1, k_fluid_volsum32, c->nred, RED_THREADS, c->g, op_of<float>(c), c->type, c->d32, c->part);
        IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN));
        KL(-1, k_add_scaled_dev, c->nred_wide, RED_THREADS, n, c->type, phi, c->d32, R, c->scal + S_MEAN);
        KL(-1, k_ref_after, 1, 1, R, F);
        IBM_TRY(apply_PA<double>(c, phi, c->b, -1.0, c->rr));
        IBM_TRY(norm2_dev<double>(c, c->rr, S_TMP));
        KL(-1, k_ref_start, 1, 1, R, F, c->scal + S_TMP, hr);
    }
    IBM_TRY(cond_close(c, &sr));
    IBM_LAUNCHED(c);
    return IBM_OK;
}

// buffers and control blocks the captured solve needs (outside capture)
ibm_status poisson_dev_prepare(Ctx *c) {
    if ((c->opts.precision == IBM_FP64 && !c->mg64.built) || (c->opts.precision == IBM_MIXED && !c->mg32.built))
        IBM_TRY(mg_build(c));
    if (c->opts.precision == IBM_MIXED) IBM_TRY(ensure_mixed(c));
    else IBM_TRY(alloc_krylov(c, c->opts.restart));
    if (!c->dctl) {
        c->dctl = dev_alloc(c, sizeof(DevFG) * 2);
        c->dstats = dev_alloc(c, sizeof(DevStats));
        if (!c->dctl || !c->dstats) return c->fail(IBM_ERR_OOM, "control block allocation failed");
        IBM_CUDA(c, cudaMemsetAsync(c->dctl, 0, sizeof(DevFG) * 2, c->s));
        IBM_CUDA(c, cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->s));
    }
    return IBM_OK;
}

// the Poisson solve of poisson_solve with device-side control; capturable
ibm_status poisson_solve_dev(Ctx *c, const double *rhs, double *phi, double rtol, int maxit) {
    const int64_t n = c->N;
    DevFG *R = dfg(c, 0), *F = dfg(c, 1);
    KL(-1, k_fluid_volsum, c->nred, RED_THREADS, c->g, c->type, rhs, c->part);
    IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN));
    IBM_CUDA(c, cudaMemcpyAsync(c->b, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
    KL(-1, k_sub_mean, c->nred_wide, RED_THREADS, n, c->type, c->b, c->scal + S_MEAN, 0);
    if (c->ng > 0) KL(-1, k_zero_at, (unsigned)((c->ng + 255) / 256), 256, c->ng, c->gidx, c->b);
    IBM_TRY(norm2_dev<double>(c, c->b, S_TMP));
    KL(-1, k_fg_setup, 1, 1, R, c->scal + S_TMP, rtol, maxit);
    IBM_LAUNCHED(c);
    if (c->opts.precision == IBM_MIXED) {
        KL(-1, k_copy_inner_rtol, 1, 1, R, c->opts.mixed_inner_rtol);
        IBM_TRY(mixed_dev(c, phi, R, F));
    } else {
        IBM_TRY(fgmres64_dev(c, phi, R));
    }
    KL(-1, k_zero_if, c->nred_wide, RED_THREADS, n, phi, &R->zero);
    KL(-1, k_fluid_volsum, c->nred, RED_THREADS, c->g, c->type, phi, c->part);
    IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN));
    KL(-1, k_sub_mean, c->nred_wide, RED_THREADS, n, c->type, phi, c->scal + S_MEAN, 1);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

// per-step statistics of the captured step: Poisson iterations and status,
// Helmholtz sweeps (hsw[0..2], status in hsw[3]), ghost refresh status
__global__ void k_step_stats(DevStats *S, const DevFG *R, const int *hsw) {
    S->steps += 1;
    S->outer += R->refinements > 0 ? R->steps : R->outer;
    S->helm_sweeps += hsw[0] + hsw[1] + hsw[2];
    S->rel = R->rel;
    int st = R->status;
    if (hsw[3] != 0 && (st == 0 || hsw[3] == IBM_ERR_DIVERGED)) st = hsw[3];
    if (st == IBM_ERR_DIVERGED || S->status == 0) S->status = st ? st : S->status;
}

ibm_status step_stats_dev(Ctx *c, const int *hsw) {
    KL(-1, k_step_stats, 1, 1, (DevStats *)c->dstats, dfg(c, 0), hsw);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

ibm_status step_stats_read(Ctx *c, ibm_step_stats *st) {
    DevStats h{};
    IBM_CUDA(c, cudaMemcpyAsync(&h, c->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, c->s));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    IBM_CUDA(c, cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->s));
    if (st) {
        st->steps += h.steps;
        st->poisson_outer += h.outer;
        st->poisson_inner += h.outer;
        st->helm_sweeps += h.helm_sweeps;
        if (h.steps > 0) st->rel_residual = h.rel;
    }
    if (h.status == IBM_ERR_DIVERGED) return c->fail(IBM_ERR_DIVERGED, "a solve in the step produced a non-finite value");
    if (h.status == IBM_ERR_NOT_CONVERGED) {
        c->fail(IBM_ERR_NOT_CONVERGED, "a solve in the step reached its iteration limit");
        return IBM_ERR_NOT_CONVERGED;
    }
    return IBM_OK;
}

// ---------------------------------------------------------------------------
// Poisson initial guess from earlier solves (least-squares projection)
// ---------------------------------------------------------------------------
//
// The pressure operator of a body at rest is the same at every step, so the
// solutions x_i of the last L steps and their projected right-hand sides
// b_i = P rhs_i are pairs with A x_i = b_i (to the solve tolerance). For a
// new right-hand side b the guess x0 = sum c_i x_i with c minimising
// || P b - sum c_i b_i ||_2 leaves that least-squares residual (Fischer's
// projection onto earlier solutions, 1998); it contains the polynomial
// extrapolation of the last pressures. The pairs sit in a ring of L slots;
// the Gram matrix G_ij = (b_i, b_j) is updated as a pair enters (its dots
// are the ones the guess of that step computed), and the normal equations
// (G + eps I) c = (b_i, P b) are solved by Cholesky in one thread. All of it
// runs on the device, so the captured step graph holds it as well.

template <typename T>
static inline const MdotFn<T> *mdot_fns() {
    return mdot_table<T>(std::make_integer_sequence<int, 17>());
}

// rhs - mean on FLUID cells, 0 elsewhere (the solver's P rhs)
__global__ void k_hist_bp(int64_t n, const uint8_t *__restrict__ type, const double *__restrict__ rhs,
                          const HistCtl *__restrict__ H, double *__restrict__ bp) {
    const double m = H->mean;
    GRID_STRIDE(c, n) bp[c] = type[c] == FLUID ? rhs[c] - m : 0.0;
}

// c over the m active slots (0 elsewhere, and everywhere if the factorisation
// meets a non-positive pivot)
__global__ void k_hist_solve(HistCtl *H) {
    const int m = H->count;
    for (int i = 0; i < HIST_MAX; ++i) H->c[i] = 0.0;
    if (m == 0) return;
    double a[HIST_MAX * HIST_MAX], y[HIST_MAX];
    double dmax = 0.0;
    for (int i = 0; i < m; ++i) dmax = fmax(dmax, H->G[i * HIST_MAX + i]);
    if (!(dmax > 0.0)) return;
    const double eps = 1e-12 * dmax;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) a[i * HIST_MAX + j] = H->G[i * HIST_MAX + j] + (i == j ? eps : 0.0);
    // Cholesky a = R^T R (upper R in place)
    for (int k = 0; k < m; ++k) {
        double piv = a[k * HIST_MAX + k];
        for (int q = 0; q < k; ++q) piv -= a[q * HIST_MAX + k] * a[q * HIST_MAX + k];
        if (!(piv > 0.0)) return;
        const double r = sqrt(piv);
        a[k * HIST_MAX + k] = r;
        for (int j = k + 1; j < m; ++j) {
            double v = a[k * HIST_MAX + j];
            for (int q = 0; q < k; ++q) v -= a[q * HIST_MAX + k] * a[q * HIST_MAX + j];
            a[k * HIST_MAX + j] = v / r;
        }
    }
    for (int i = 0; i < m; ++i) {   // R^T y = d
        double v = H->d[i];
        for (int q = 0; q < i; ++q) v -= a[q * HIST_MAX + i] * y[q];
        y[i] = v / a[i * HIST_MAX + i];
    }
    for (int i = m - 1; i >= 0; --i) {   // R c = y
        double v = y[i];
        for (int q = i + 1; q < m; ++q) v -= a[i * HIST_MAX + q] * H->c[q];
        H->c[i] = v / a[i * HIST_MAX + i];
    }
}

// phi = sum over the active slots of c_i X_i (phi untouched with no pairs);
// slot i starts at X + i ld
__global__ void k_hist_guess(int64_t n, int64_t ld, const HistCtl *__restrict__ H, const double *__restrict__ X,
                             double *__restrict__ phi) {
    const int m = H->count;
    if (m == 0) return;
    GRID_STRIDE(c, n) {
        double v = 0.0;
        for (int i = 0; i < m; ++i) v += H->c[i] * X[(int64_t)i * ld + c];
        phi[c] = v;
    }
}

// the pair of this step into the current slot
__global__ void k_hist_insert(int64_t n, int64_t ld, const HistCtl *__restrict__ H, const double *__restrict__ phi,
                              const double *__restrict__ bp, double *__restrict__ X, double *__restrict__ B) {
    const int64_t off = (int64_t)H->slot * ld;
    GRID_STRIDE(c, n) {
        X[off + c] = phi[c];
        B[off + c] = bp[c];
    }
}

// Gram row and column of the new pair; advance the ring
__global__ void k_hist_advance(HistCtl *H, int L) {
    const int k = H->slot;
    for (int i = 0; i < L; ++i) {
        if (i == k) continue;
        H->G[k * HIST_MAX + i] = H->d[i];
        H->G[i * HIST_MAX + k] = H->d[i];
    }
    H->G[k * HIST_MAX + k] = H->d[L];
    H->slot = (k + 1) % L;
    H->count = H->count < L ? H->count + 1 : L;
}

// ring storage for opts.poisson_hist pairs (allocated outside any capture;
// a new size starts an empty history)
ibm_status hist_prepare(Ctx *c) {
    const int L = c->opts.poisson_hist;
    if (L <= c->hist_cap) {
        // a history kept for another pair count starts over
        if (L != c->hist_len) {
            IBM_TRY(hist_reset(c));
            c->hist_len = L;
        }
        return IBM_OK;
    }
    dev_free(c, c->hist_x);
    dev_free(c, c->hist_b);
    c->hist_x = c->hist_b = nullptr;
    c->hist_cap = 0;
    // each slot starts on a 256-byte boundary: the multi-dot reads its
    // columns with 16-byte loads
    c->hist_ld = (c->N + 31) / 32 * 32;
    const size_t nb = sizeof(double) * (size_t)c->hist_ld * (size_t)L;
    c->hist_x = (double *)dev_alloc(c, nb);
    c->hist_b = (double *)dev_alloc(c, nb);
    if (!c->hist_bp) c->hist_bp = (double *)dev_alloc(c, sizeof(double) * (size_t)c->N);
    if (!c->hist_ctl) c->hist_ctl = dev_alloc(c, sizeof(HistCtl));
    if (!c->hist_x || !c->hist_b || !c->hist_bp || !c->hist_ctl) return c->fail(IBM_ERR_OOM, "Poisson history allocation failed");
    // zero vectors: the dots of unused slots are 0
    IBM_CUDA(c, cudaMemsetAsync(c->hist_b, 0, nb, c->s));
    IBM_CUDA(c, cudaMemsetAsync(c->hist_x, 0, nb, c->s));
    IBM_CUDA(c, cudaMemsetAsync(c->hist_ctl, 0, sizeof(HistCtl), c->s));
    c->hist_cap = L;
    c->hist_len = L;
    return IBM_OK;
}

// forget the pairs (the operator changed)
ibm_status hist_reset(Ctx *c) {
    if (c->hist_ctl) IBM_CUDA(c, cudaMemsetAsync(c->hist_ctl, 0, sizeof(HistCtl), c->s));
    return IBM_OK;
}

// phi = the projection guess for rhs, if the history holds a pair
ibm_status hist_guess(Ctx *c, const double *rhs, double *phi) {
    const int L = c->opts.poisson_hist;
    if (L <= 0) return IBM_OK;
    if (L > c->hist_cap || L != c->hist_len) return c->fail(IBM_ERR_STATE, "Poisson history not prepared");
    HistCtl *H = reinterpret_cast<HistCtl *>(c->hist_ctl);
    KL(-1, k_fluid_volsum, c->nred, RED_THREADS, c->g, c->type, rhs, c->part);
    IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0 / c->fluid_vol, &H->mean));
    KL(-1, k_hist_bp, c->nelem, 256, c->N, c->type, rhs, H, c->hist_bp);
    VPtrs<double> vp{};
    for (int i = 0; i < L; ++i) vp.p[i] = c->hist_b + (size_t)i * c->hist_ld;
    vp.p[L] = c->hist_bp;
    for (int i = 0; i <= L; ++i)
        if (!al16(vp.p[i])) return c->fail(IBM_ERR_STATE, "Poisson history column not 16-byte aligned");
    KL(-1, mdot_fns<double>()[L], mdot_blocks<double>(c), RED_THREADS, c->N, c->hist_bp, vp, c->part);
    IBM_TRY(finalize(c, c->part, mdot_blocks<double>(c), L + 1, 1.0, H->d));
    KL(-1, k_hist_solve, 1, 1, H);
    KL(-1, k_hist_guess, c->nelem, 256, c->N, c->hist_ld, H, c->hist_x, phi);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

// this step's pair (phi the solution of hist_guess's right-hand side)
ibm_status hist_store(Ctx *c, const double *phi) {
    const int L = c->opts.poisson_hist;
    if (L <= 0) return IBM_OK;
    HistCtl *H = reinterpret_cast<HistCtl *>(c->hist_ctl);
    KL(-1, k_hist_insert, c->nelem, 256, c->N, c->hist_ld, H, phi, c->hist_bp, c->hist_x, c->hist_b);
    KL(-1, k_hist_advance, 1, 1, H, L);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

ibm_status poisson_solve(Ctx *c, const double *rhs, double *phi, double rtol, int maxit, ibm_solve_stats *st) {
    if ((c->opts.precision == IBM_FP64 && !c->mg64.built) || (c->opts.precision == IBM_MIXED && !c->mg32.built))
        IBM_TRY(mg_build(c));
    const int64_t n = c->N;
    IBM_CUDA(c, cudaEventRecord(c->ev4, c->s));
    // b = P rhs on FLUID rows, 0 elsewhere
    KL(-1, k_fluid_volsum, c->nred, RED_THREADS, c->g, c->type, rhs, c->part);
    IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN));
    IBM_CUDA(c, cudaMemcpyAsync(c->b, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
    KL(-1, k_sub_mean, c->nred_wide, RED_THREADS, n, c->type, c->b, c->scal + S_MEAN, 0);
    IBM_LAUNCHED(c);
    // GHOST rows of b are 0 (homogeneous Neumann on the body)
    if (c->ng > 0) {
        KL(-1, k_zero_at, (unsigned)((c->ng + 255) / 256), 256, c->ng, c->gidx, c->b);
        IBM_LAUNCHED(c);
    }
    double bn2;
    IBM_TRY(norm2<double>(c, c->b, &bn2));
    const double bnorm = sqrt(bn2);
    if (!isfinite(bnorm)) return c->fail(IBM_ERR_DIVERGED, "Poisson right-hand side is not finite");
    int outer = 0, inner = 0;
    double rel = 0.0;
    ibm_status status = IBM_OK;
    if (!(bnorm > 1e-300)) {
        IBM_CUDA(c, cudaMemsetAsync(phi, 0, sizeof(double) * n, c->s));
    } else {
        if (c->opts.outer == IBM_OUTER_BICGSTAB || c->opts.precision != IBM_MIXED)
            IBM_TRY(alloc_krylov(c, c->opts.restart));
        if (c->opts.outer == IBM_OUTER_BICGSTAB) status = bicgstab(c, phi, bnorm, rtol, maxit, &outer, &inner, &rel);
        else if (c->opts.precision == IBM_MIXED) status = mixed_refinement(c, phi, bnorm, rtol, maxit, &outer, &inner, &rel);
        else status = fgmres<double>(c, kry64(c), phi, c->b, bnorm, rtol, maxit, false, &outer, &inner, &rel);
        if (status != IBM_OK && status != IBM_ERR_NOT_CONVERGED) return status;
        // normalise: zero volume-weighted FLUID mean, shift ghosts too
        KL(-1, k_fluid_volsum, c->nred, RED_THREADS, c->g, c->type, phi, c->part);
        IBM_TRY(finalize(c, c->part, c->nred, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN));
        KL(-1, k_sub_mean, c->nred_wide, RED_THREADS, n, c->type, phi, c->scal + S_MEAN, 1);
        IBM_LAUNCHED(c);
    }
    IBM_TRY(kt_flush(c));
    IBM_CUDA(c, cudaEventRecord(c->ev5, c->s));
    IBM_CUDA(c, cudaEventSynchronize(c->ev5));
    float ms = 0.f;
    IBM_CUDA(c, cudaEventElapsedTime(&ms, c->ev4, c->ev5));
    if (st) {
        st->outer_iters = outer;
        st->inner_iters = inner;
        st->rel_residual = rel;
        st->ms = ms;
    }
    if (status == IBM_ERR_NOT_CONVERGED) c->fail(IBM_ERR_NOT_CONVERGED, "Poisson solve reached its iteration limit");
    return status;
}

}  // namespace ibm
