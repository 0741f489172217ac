// Pressure Poisson solver (Section 2.1, pressure equation; Section 2.2,
// Neumann ghost-cell rows) on one GPU.
//
//   outer: restarted FGMRES in FP64 on P A phi = P b, where A is the full
//          ghost-cell operator (FLUID rows: variable-coefficient 7-point
//          (2D: 5-point) div-grad with ghost neighbours; GHOST rows:
//          phi_G - sum wp phi_m; DEAD rows: identity) and P removes the
//          volume-weighted FLUID mean (compatibility);
//   preconditioner: multigrid-preconditioned CG on the staircase operator
//          K = sum over open faces T_f (x_c - x_nb) (a face is open when
//          both sides are FLUID), symmetric positive semi-definite, in FP64
//          or FP32 (storage and arithmetic; dot products accumulate in
//          FP64), followed by one pass over the ghost rows;
//   multigrid: V(nu1,nu2) cycle, red-black Gauss-Seidel smoothing, restriction
//          by summing children, piecewise-constant prolongation, coarse
//          operators rediscretised from the open child-face areas.
#include "ctx.cuh"

#include <math.h>

namespace ibm {

// device scalar slots
enum { S_RZ = 0, S_PQ = 1, S_AL = 2, S_RZN = 3, S_BE = 4, S_MEAN = 5, S_TMP = 8, S_MD = 16 };

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------

// out[col] = scale * sum_i part[col*nparts + i], in a fixed order
__global__ void k_finalize(const double *__restrict__ part, int nparts, int ncols, double scale,
                           double *__restrict__ out) {
    __shared__ double sh[32];
    for (int col = 0; col < ncols; ++col) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[(size_t)col * nparts + i];
        v = block_sum<RED_THREADS>(v, sh);
        if (threadIdx.x == 0) out[col] = v * scale;
    }
}

ibm_status finalize(Ctx *c, const double *part, int nparts, int ncols, double scale, double *out_dev) {
    ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(part, nparts, ncols, scale, out_dev);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

ibm_status reduce_sum(Ctx *c, const double *partials, int nparts, double *out_dev) {
    ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(partials, nparts, 1, 1.0, out_dev);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

ibm_status sync_scalars(Ctx *c, int n) {
    IBM_CUDA(c, cudaMemcpyAsync(c->hscal, c->scal, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    return IBM_OK;
}

__device__ __forceinline__ void cell_ijk(int64_t cidx, int nx, int ny, int &i, int &j, int &k) {
    int64_t t = cidx / nx;
    i = (int)(cidx - t * nx);
    j = (int)(t % ny);
    k = (int)(t / ny);
}

// sum over FLUID cells of vol * x (x null: the FLUID volume)
__global__ void k_fluid_volsum(GridDev g, const uint8_t *__restrict__ type, const double *__restrict__ x,
                               double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (type[c] != FLUID) continue;
        int i, j, k;
        cell_ijk(c, g.nx, g.ny, i, j, k);
        acc += (g.dx[i] * g.dy[j] * g.dz[k]) * (x ? x[c] : 1.0);
    }
    acc = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// x -= mean on FLUID (and GHOST if ghosts) cells; DEAD cells set to 0
__global__ void k_sub_mean(int64_t n, const uint8_t *__restrict__ type, double *__restrict__ x,
                           const double *__restrict__ mean, int ghosts) {
    const double m = *mean;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        uint8_t t = type[c];
        if (t == FLUID || (ghosts && t == GHOST)) x[c] -= m;
        else if (t == DEAD) x[c] = 0.0;
    }
}

ibm_status fluid_mean(Ctx *c, const double *x, bool ghosts_too, double *mean_host) {
    (void)ghosts_too;
    ++c->nlaunch, k_fluid_volsum<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(c->g, c->type, x, c->part);
    IBM_LAUNCHED(c);
    ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(c->part, RED_BLOCKS, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN);
    IBM_LAUNCHED(c);
    if (mean_host) {
        IBM_TRY(sync_scalars(c, S_MEAN + 1));
        *mean_host = c->hscal[S_MEAN];
    }
    return IBM_OK;
}

// ---------------------------------------------------------------------------
// full ghost-cell pressure operator (FP64)
// ---------------------------------------------------------------------------

// y = sgn * (A x) + b  on FLUID and DEAD rows (b may be null = 0); GHOST rows
// are written by k_ghost_rows. Partials: sum over FLUID of vol * y.
__global__ void k_apply_A(GridDev g, const uint8_t *__restrict__ type, const double *__restrict__ x,
                          const double *__restrict__ b, double sgn, double *__restrict__ y,
                          double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    const int64_t sx = 1, sy = g.nx, sz = (int64_t)g.nx * g.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t t = type[c];
        if (t == GHOST) continue;
        if (t == DEAD) { y[c] = 0.0; continue; }
        int i, j, k;
        cell_ijk(c, g.nx, g.ny, i, j, k);
        const double xc = x[c];
        const double ax = g.dy[j] * g.dz[k], ay = g.dx[i] * g.dz[k], az = g.dx[i] * g.dy[j];
        double s = 0.0;
        if (i > 0) s += ax / g.hx[i] * (x[c - sx] - xc);
        if (i < g.nx - 1) s += ax / g.hx[i + 1] * (x[c + sx] - xc);
        if (j > 0) s += ay / g.hy[j] * (x[c - sy] - xc);
        if (j < g.ny - 1) s += ay / g.hy[j + 1] * (x[c + sy] - xc);
        if (g.ndim == 3) {
            if (k > 0) s += az / g.hz[k] * (x[c - sz] - xc);
            if (k < g.nz - 1) s += az / g.hz[k + 1] * (x[c + sz] - xc);
        }
        const double vol = g.dx[i] * g.dy[j] * g.dz[k];
        double v = sgn * (s / vol) + (b ? b[c] : 0.0);
        y[c] = v;
        acc += vol * v;
    }
    acc = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// GHOST rows: y_g = sgn * (x_g - sum_m wp_m x_m)   (b_g = 0)
__global__ void k_ghost_rows(GhostDev gh, const double *__restrict__ x, double sgn, double *__restrict__ y) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= gh.ng) return;
    const int64_t gi = gh.gidx[q];
    double s = x[gi];
    for (int m = 0; m < 8; ++m) s -= gh.wp[8 * q + m] * x[gh.sidx[8 * q + m]];
    y[gi] = sgn * s;
}

// y = P(sgn * A x + b)
static ibm_status apply_PA(Ctx *c, const double *x, const double *b, double sgn, double *y) {
    kt_begin(c, K_APPLY_A);
    ++c->nlaunch, k_apply_A<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(c->g, c->type, x, b, sgn, y, c->part);
    kt_end(c, K_APPLY_A);
    IBM_LAUNCHED(c);
    if (c->ng > 0) {
        ++c->nlaunch, k_ghost_rows<<<(unsigned)((c->ng + 255) / 256), 256, 0, c->s>>>(c->gh, x, sgn, y);
        IBM_LAUNCHED(c);
    }
    ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(c->part, RED_BLOCKS, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN);
    IBM_LAUNCHED(c);
    ++c->nlaunch, k_sub_mean<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(c->N, c->type, y, c->scal + S_MEAN, 0);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

// ---------------------------------------------------------------------------
// FP64 vector kernels for FGMRES
// ---------------------------------------------------------------------------

struct Coef {
    double v[17];
};

// partial dots: col i < ncols: (w, V_i); col ncols: (w, w)
__global__ void k_mdot(int64_t n, const double *__restrict__ w, const double *const *__restrict__ V, int ncols,
                       double *__restrict__ part) {
    __shared__ double sh[32];
    double acc[17];
#pragma unroll
    for (int q = 0; q < 17; ++q) acc[q] = 0.0;
    double ww = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const double a = w[c];
        ww += a * a;
#pragma unroll
        for (int q = 0; q < 17; ++q)
            if (q < ncols) acc[q] += a * V[q][c];
    }
    for (int q = 0; q < ncols; ++q) {
        double t = block_sum<RED_THREADS>(acc[q], sh);
        if (threadIdx.x == 0) part[(size_t)q * gridDim.x + blockIdx.x] = t;
    }
    double t = block_sum<RED_THREADS>(ww, sh);
    if (threadIdx.x == 0) part[(size_t)ncols * gridDim.x + blockIdx.x] = t;
}

// w -= sum_i h_i V_i ; partial (w, w)
__global__ void k_orth(int64_t n, double *__restrict__ w, const double *const *__restrict__ V, int ncols, Coef h,
                       double *__restrict__ part) {
    __shared__ double sh[32];
    double ww = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        double a = w[c];
#pragma unroll
        for (int q = 0; q < 17; ++q)
            if (q < ncols) a -= h.v[q] * V[q][c];
        w[c] = a;
        ww += a * a;
    }
    double t = block_sum<RED_THREADS>(ww, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_scale(int64_t n, double *__restrict__ dst, const double *__restrict__ src, double a) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        dst[c] = a * src[c];
}

// x += sum_i y_i Z_i
__global__ void k_xupd(int64_t n, double *__restrict__ x, const double *const *__restrict__ Z, int ncols, Coef y) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        double a = x[c];
#pragma unroll
        for (int q = 0; q < 17; ++q)
            if (q < ncols) a += y.v[q] * Z[q][c];
        x[c] = a;
    }
}

// ---------------------------------------------------------------------------
// multigrid on the staircase operator, precision T
// ---------------------------------------------------------------------------

// red-black Gauss-Seidel, one colour: x_c = (f_c + sum T x_nb) / D_c for the
// cells of colour col ((i + j + k) even = 0) with D_c > 0
template <typename T>
__global__ void k_rbgs(MGLevel<T> L, const T *__restrict__ D, const T *__restrict__ f, T *__restrict__ x, int col) {
    const int64_t row = blockIdx.x;             // j + ny * k
    const int j = (int)(row % L.ny), k = (int)(row / L.ny);
    const int par = (j + k + col) & 1;
    const int i = 2 * (blockIdx.y * blockDim.x + threadIdx.x) + par;
    if (i >= L.nx) return;
    const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
    const int64_t c = row * L.nx + i;
    const T d = D[c];
    if (d <= T(0)) return;
    T s = f[c];
    if (i > 0) s += L.tx[c] * x[c - 1];
    if (i < L.nx - 1) s += L.tx[c + 1] * x[c + 1];
    if (j > 0) s += L.ty[c] * x[c - sy];
    if (j < L.ny - 1) s += L.ty[c + sy] * x[c + sy];
    if (k > 0) s += L.tz[c] * x[c - sz];
    if (k < L.nz - 1) s += L.tz[c + sz] * x[c + sz];
    x[c] = s / d;
}

template <typename T>
__device__ __forceinline__ T k_row(const MGLevel<T> &L, const T *__restrict__ D, const T *__restrict__ x, int64_t c,
                                   int i, int j, int k) {
    const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
    T s = D[c] * x[c];
    if (i > 0) s -= L.tx[c] * x[c - 1];
    if (i < L.nx - 1) s -= L.tx[c + 1] * x[c + 1];
    if (j > 0) s -= L.ty[c] * x[c - sy];
    if (j < L.ny - 1) s -= L.ty[c + sy] * x[c + sy];
    if (k > 0) s -= L.tz[c] * x[c - sz];
    if (k < L.nz - 1) s -= L.tz[c + sz] * x[c + sz];
    return s;
}

// coarse f_C = sum over children of (f - K x); coarse x_C = 0
template <typename T>
__global__ void k_resid_restrict(MGLevel<T> L, const T *__restrict__ D, const T *__restrict__ f,
                                 const T *__restrict__ x, MGLevel<T> C, int fx, int fy, int fz) {
    const int64_t row = blockIdx.x;
    const int J = (int)(row % C.ny), K = (int)(row / C.ny);
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
                if (D[c] > T(0)) acc += f[c] - k_row(L, D, x, c, i, j, k);
            }
        }
    }
    const int64_t cc = row * C.nx + I;
    C.f[cc] = acc;
    C.x[cc] = T(0);
}

// x_c += x_parent(c) on cells with D > 0
template <typename T>
__global__ void k_prolong(MGLevel<T> L, const T *__restrict__ D, T *__restrict__ x, MGLevel<T> C, int fx, int fy,
                          int fz) {
    const int64_t row = blockIdx.x;
    const int j = (int)(row % L.ny), k = (int)(row / L.ny);
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= L.nx) return;
    const int64_t c = row * L.nx + i;
    if (D[c] <= T(0)) return;
    const int64_t p = ((int64_t)(k / fz) * C.ny + (j / fy)) * C.nx + (i / fx);
    x[c] += C.x[p];
}

// q = K p ; partial (p, q) in FP64
template <typename T>
__global__ void k_spmv_dot(MGLevel<T> L, const T *__restrict__ D, const T *__restrict__ p, T *__restrict__ q,
                           double *__restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < L.n; c += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(c, L.nx, L.ny, i, j, k);
        T v = D[c] > T(0) ? k_row(L, D, p, c, i, j, k) : T(0);
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
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        acc += (double)a[c] * (double)b[c];
    acc = block_sum<RED_THREADS>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

template <typename T>
__global__ void k_axpy2(int64_t n, T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
                        const T *__restrict__ q, const double *__restrict__ scal) {
    const T a = (T)scal[S_AL];
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        x[c] += a * p[c];
        r[c] -= a * q[c];
    }
}

template <typename T>
__global__ void k_pupd(int64_t n, T *__restrict__ p, const T *__restrict__ z, const double *__restrict__ scal) {
    const T b = (T)scal[S_BE];
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        p[c] = z[c] + b * p[c];
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

__global__ void k_zero_at(int64_t m, const int64_t *__restrict__ idx, double *__restrict__ x) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < m) x[idx[q]] = 0.0;
}

// preconditioner input / output conversion
template <typename T>
__global__ void k_pre_in(GridDev g, const uint8_t *__restrict__ type, const double *__restrict__ v, T *__restrict__ f) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (type[c] != FLUID) { f[c] = T(0); continue; }
        int i, j, k;
        cell_ijk(c, g.nx, g.ny, i, j, k);
        f[c] = (T)(-(g.dx[i] * g.dy[j] * g.dz[k]) * v[c]);
    }
}
template <typename T>
__global__ void k_pre_out(int64_t n, const uint8_t *__restrict__ type, const T *__restrict__ x, double *__restrict__ z) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        z[c] = type[c] == FLUID ? (double)x[c] : 0.0;
}
// ghost rows of the preconditioner: z_g = v_g + sum over FLUID corners wp z_m
__global__ void k_pre_ghost(GhostDev gh, const uint8_t *__restrict__ type, const double *__restrict__ v,
                            double *__restrict__ z) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= gh.ng) return;
    const int64_t gi = gh.gidx[q];
    double s = v[gi];
    for (int m = 0; m < 8; ++m) {
        const int64_t s_m = gh.sidx[8 * q + m];
        if (type[s_m] == FLUID) s += gh.wp[8 * q + m] * z[s_m];
    }
    z[gi] = s;
}

// level coefficient construction ------------------------------------------

// level 0 open face areas: face on the low side of cell c along each axis is
// open when c and its low neighbour are both FLUID
__global__ void k_open_area0(GridDev g, const uint8_t *__restrict__ type, double *__restrict__ ox,
                             double *__restrict__ oy, double *__restrict__ oz) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(c, g.nx, g.ny, i, j, k);
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
    for (int64_t cc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cc < cn; cc += (int64_t)gridDim.x * blockDim.x) {
        int I, J, K;
        cell_ijk(cc, cnx, cny, I, J, K);
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

// T = open area / centre spacing, then D = sum of the six faces
template <typename T>
__global__ void k_level_coef(int nx, int ny, int nz, const double *__restrict__ ox, const double *__restrict__ oy,
                             const double *__restrict__ oz, const double *__restrict__ hx,
                             const double *__restrict__ hy, const double *__restrict__ hz, T *__restrict__ tx,
                             T *__restrict__ ty, T *__restrict__ tz) {
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(c, nx, ny, i, j, k);
        tx[c] = i > 0 ? (T)(ox[c] / hx[i]) : T(0);
        ty[c] = j > 0 ? (T)(oy[c] / hy[j]) : T(0);
        tz[c] = k > 0 ? (T)(oz[c] / hz[k]) : T(0);
    }
}
template <typename T>
__global__ void k_level_diag(MGLevel<T> L, T *__restrict__ D) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < L.n; c += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(c, L.nx, L.ny, i, j, k);
        const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
        T d = L.tx[c] + L.ty[c] + L.tz[c];
        if (i < L.nx - 1) d += L.tx[c + 1];
        if (j < L.ny - 1) d += L.ty[c + sy];
        if (k < L.nz - 1) d += L.tz[c + sz];
        D[c] = d;
    }
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------

static inline unsigned nblk(int64_t n, int t = 256) {
    int64_t b = (n + t - 1) / t;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

static inline dim3 rows_grid(int nx, int ny, int nz, int per_thread, int bx) {
    int64_t rows = (int64_t)ny * nz;
    int xs = (nx + per_thread - 1) / per_thread;
    return dim3((unsigned)rows, (unsigned)((xs + bx - 1) / bx), 1);
}

template <typename T>
static ibm_status build_hier(Ctx *c, MGHier<T> &H, const std::vector<double *> &oax,
                             const std::vector<double *> &oay, const std::vector<double *> &oaz) {
    const int L = (int)c->lg.size();
    H.lv.resize(L);
    H.dg.resize(L);
    for (int l = 0; l < L; ++l) {
        auto &G = c->lg[l];
        MGLevel<T> &M = H.lv[l];
        M.nx = G.nx;
        M.ny = G.ny;
        M.nz = G.nz;
        M.n = (int64_t)G.nx * G.ny * G.nz;
        const size_t bytes = sizeof(T) * (size_t)M.n;
        M.tx = (T *)dev_alloc(c, bytes);
        M.ty = (T *)dev_alloc(c, bytes);
        M.tz = (T *)dev_alloc(c, bytes);
        H.dg[l] = (T *)dev_alloc(c, bytes);
        M.x = l == 0 ? nullptr : (T *)dev_alloc(c, bytes);
        M.f = l == 0 ? nullptr : (T *)dev_alloc(c, bytes);
        M.r = nullptr;
        if (!M.tx || !M.ty || !M.tz || !H.dg[l] || (l > 0 && (!M.x || !M.f)))
            return c->fail(IBM_ERR_OOM, "multigrid level allocation failed");
        ++c->nlaunch, k_level_coef<T><<<nblk(M.n), 256, 0, c->s>>>(M.nx, M.ny, M.nz, oax[l], oay[l], oaz[l], c->lhx[l], c->lhy[l],
                                                     c->lhz[l], M.tx, M.ty, M.tz);
        IBM_LAUNCHED(c);
        ++c->nlaunch, k_level_diag<T><<<nblk(M.n), 256, 0, c->s>>>(M, H.dg[l]);
        IBM_LAUNCHED(c);
    }
    const size_t b0 = sizeof(T) * (size_t)c->N;
    H.px = (T *)dev_alloc(c, b0);
    H.pr = (T *)dev_alloc(c, b0);
    H.pz = (T *)dev_alloc(c, b0);
    H.pp = (T *)dev_alloc(c, b0);
    H.pq = (T *)dev_alloc(c, b0);
    if (!H.px || !H.pr || !H.pz || !H.pp || !H.pq) return c->fail(IBM_ERR_OOM, "PCG vector allocation failed");
    H.built = true;
    return IBM_OK;
}

// Multigrid hierarchy of the staircase operator for the current
// classification. Level geometry (c->lg, c->lh*) is built at grid creation.
ibm_status mg_build(Ctx *c) {
    const int L = (int)c->lg.size();
    std::vector<double *> ox(L), oy(L), oz(L);
    for (int l = 0; l < L; ++l) {
        const int64_t n = (int64_t)c->lg[l].nx * c->lg[l].ny * c->lg[l].nz;
        ox[l] = (double *)dev_alloc(c, sizeof(double) * n);
        oy[l] = (double *)dev_alloc(c, sizeof(double) * n);
        oz[l] = (double *)dev_alloc(c, sizeof(double) * n);
        if (!ox[l] || !oy[l] || !oz[l]) return c->fail(IBM_ERR_OOM, "open-area allocation failed");
    }
    ++c->nlaunch, k_open_area0<<<nblk(c->N), 256, 0, c->s>>>(c->g, c->type, ox[0], oy[0], oz[0]);
    IBM_LAUNCHED(c);
    for (int l = 1; l < L; ++l) {
        auto &F = c->lg[l - 1];
        auto &C = c->lg[l];
        const int64_t n = (int64_t)C.nx * C.ny * C.nz;
        ++c->nlaunch, k_open_area_coarsen<<<nblk(n), 256, 0, c->s>>>(F.nx, F.ny, F.nz, ox[l - 1], oy[l - 1], oz[l - 1], C.nx, C.ny,
                                                        C.nz, C.fx, C.fy, C.fz, ox[l], oy[l], oz[l]);
        IBM_LAUNCHED(c);
    }
    if (!c->mg64.built) IBM_TRY(build_hier<double>(c, c->mg64, ox, oy, oz));
    else {
        for (int l = 0; l < L; ++l) {
            auto &M = c->mg64.lv[l];
            ++c->nlaunch, k_level_coef<double><<<nblk(M.n), 256, 0, c->s>>>(M.nx, M.ny, M.nz, ox[l], oy[l], oz[l], c->lhx[l],
                                                              c->lhy[l], c->lhz[l], M.tx, M.ty, M.tz);
            ++c->nlaunch, k_level_diag<double><<<nblk(M.n), 256, 0, c->s>>>(M, c->mg64.dg[l]);
        }
        IBM_LAUNCHED(c);
    }
    if (c->opts.precision == IBM_MIXED) {
        if (!c->mg32.built) IBM_TRY(build_hier<float>(c, c->mg32, ox, oy, oz));
        else {
            for (int l = 0; l < L; ++l) {
                auto &M = c->mg32.lv[l];
                ++c->nlaunch, k_level_coef<float><<<nblk(M.n), 256, 0, c->s>>>(M.nx, M.ny, M.nz, ox[l], oy[l], oz[l], c->lhx[l],
                                                                 c->lhy[l], c->lhz[l], M.tx, M.ty, M.tz);
                ++c->nlaunch, k_level_diag<float><<<nblk(M.n), 256, 0, c->s>>>(M, c->mg32.dg[l]);
            }
            IBM_LAUNCHED(c);
        }
    }
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    for (int l = 0; l < L; ++l) {
        dev_free(c, ox[l]);
        dev_free(c, oy[l]);
        dev_free(c, oz[l]);
    }
    return IBM_OK;
}

template <typename T>
static ibm_status rbgs(Ctx *c, MGHier<T> &H, int l, const T *f, T *x, int col) {
    MGLevel<T> &L = H.lv[l];
    const int bx = 128;
    kt_begin(c, l == 0 ? K_RBGS0 : K_RBGS_C);
    ++c->nlaunch, k_rbgs<T><<<rows_grid(L.nx, L.ny, L.nz, 2, bx), bx, 0, c->s>>>(L, H.dg[l], f, x, col);
    kt_end(c, l == 0 ? K_RBGS0 : K_RBGS_C);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

template <typename T>
static ibm_status vcycle(Ctx *c, MGHier<T> &H, const T *f0, T *x0) {
    const int L = (int)H.lv.size();
    const int nu1 = c->opts.nu1, nu2 = c->opts.nu2, cs = c->opts.coarse_sweeps;
    IBM_CUDA(c, cudaMemsetAsync(x0, 0, sizeof(T) * (size_t)c->N, c->s));
    const int bx = 128;
    for (int l = 0; l < L - 1; ++l) {
        const T *f = l == 0 ? f0 : H.lv[l].f;
        T *x = l == 0 ? x0 : H.lv[l].x;
        for (int s = 0; s < nu1; ++s) {
            IBM_TRY(rbgs(c, H, l, f, x, 0));
            IBM_TRY(rbgs(c, H, l, f, x, 1));
        }
        MGLevel<T> Lf = H.lv[l];
        MGLevel<T> &Cl = H.lv[l + 1];
        auto &CG = c->lg[l + 1];
        kt_begin(c, K_RESTRICT);
        ++c->nlaunch, k_resid_restrict<T><<<rows_grid(Cl.nx, Cl.ny, Cl.nz, 1, bx), bx, 0, c->s>>>(Lf, H.dg[l], f, x, Cl, CG.fx,
                                                                                     CG.fy, CG.fz);
        kt_end(c, K_RESTRICT);
        IBM_LAUNCHED(c);
    }
    {
        const int l = L - 1;
        const T *f = l == 0 ? f0 : H.lv[l].f;
        T *x = l == 0 ? x0 : H.lv[l].x;
        for (int s = 0; s < cs; ++s) {
            IBM_TRY(rbgs(c, H, l, f, x, 0));
            IBM_TRY(rbgs(c, H, l, f, x, 1));
        }
        for (int s = 0; s < cs; ++s) {
            IBM_TRY(rbgs(c, H, l, f, x, 1));
            IBM_TRY(rbgs(c, H, l, f, x, 0));
        }
    }
    for (int l = L - 2; l >= 0; --l) {
        const T *f = l == 0 ? f0 : H.lv[l].f;
        T *x = l == 0 ? x0 : H.lv[l].x;
        MGLevel<T> &Lf = H.lv[l];
        auto &CG = c->lg[l + 1];
        kt_begin(c, K_PROLONG);
        ++c->nlaunch, k_prolong<T><<<rows_grid(Lf.nx, Lf.ny, Lf.nz, 1, bx), bx, 0, c->s>>>(Lf, H.dg[l], x, H.lv[l + 1], CG.fx, CG.fy,
                                                                              CG.fz);
        kt_end(c, K_PROLONG);
        IBM_LAUNCHED(c);
        for (int s = 0; s < nu2; ++s) {
            IBM_TRY(rbgs(c, H, l, f, x, 1));
            IBM_TRY(rbgs(c, H, l, f, x, 0));
        }
    }
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
    ++c->nlaunch, k_dot<T><<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, H.pr, H.pz, c->part);
    ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(c->part, RED_BLOCKS, 1, 1.0, c->scal + S_RZ);
    IBM_LAUNCHED(c);
    for (int it = 0; it < iters; ++it) {
        kt_begin(c, K_SPMV0);
        ++c->nlaunch, k_spmv_dot<T><<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(L0, H.dg[0], H.pp, H.pq, c->part);
        kt_end(c, K_SPMV0);
        ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(c->part, RED_BLOCKS, 1, 1.0, c->scal + S_PQ);
        ++c->nlaunch, k_alpha<<<1, 1, 0, c->s>>>(c->scal);
        ++c->nlaunch, k_axpy2<T><<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, H.px, H.pr, H.pp, H.pq, c->scal);
        IBM_LAUNCHED(c);
        if (it + 1 < iters) {
            IBM_TRY(vcycle(c, H, H.pr, H.pz));
            ++c->nlaunch, k_dot<T><<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, H.pr, H.pz, c->part);
            ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(c->part, RED_BLOCKS, 1, 1.0, c->scal + S_RZN);
            ++c->nlaunch, k_beta<<<1, 1, 0, c->s>>>(c->scal);
            ++c->nlaunch, k_pupd<T><<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, H.pp, H.pz, c->scal);
            IBM_LAUNCHED(c);
        }
    }
    return IBM_OK;
}

// z = M^{-1} v : FP64 in, FP64 out
template <typename T>
static ibm_status precond(Ctx *c, MGHier<T> &H, const double *v, double *z) {
    ++c->nlaunch, k_pre_in<T><<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(c->g, c->type, v, H.pr);
    IBM_LAUNCHED(c);
    IBM_TRY(pcg(c, H, c->opts.inner_iters));
    ++c->nlaunch, k_pre_out<T><<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(c->N, c->type, H.px, z);
    IBM_LAUNCHED(c);
    if (c->ng > 0) {
        ++c->nlaunch, k_pre_ghost<<<(unsigned)((c->ng + 255) / 256), 256, 0, c->s>>>(c->gh, c->type, v, z);
        IBM_LAUNCHED(c);
    }
    return IBM_OK;
}

static ibm_status apply_prec(Ctx *c, const double *v, double *z) {
    if (c->opts.precision == IBM_MIXED) return precond<float>(c, c->mg32, v, z);
    return precond<double>(c, c->mg64, v, z);
}

// ||x||^2 over all cells
static ibm_status norm2(Ctx *c, const double *x, double *out) {
    ++c->nlaunch, k_dot<double><<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(c->N, x, x, c->part);
    ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(c->part, RED_BLOCKS, 1, 1.0, c->scal + S_TMP);
    IBM_LAUNCHED(c);
    IBM_TRY(sync_scalars(c, S_TMP + 1));
    *out = c->hscal[S_TMP];
    return IBM_OK;
}

// Solve P A phi = P rhs. rhs: FLUID rows read; phi: guess in, solution out.
ibm_status poisson_solve(Ctx *c, const double *rhs, double *phi, double rtol, int maxit, ibm_solve_stats *st) {
    if (!c->mg64.built || (c->opts.precision == IBM_MIXED && !c->mg32.built)) IBM_TRY(mg_build(c));
    const int64_t n = c->N;
    const int m = c->opts.restart;
    IBM_CUDA(c, cudaEventRecord(c->ev0, c->s));
    // b = P rhs on FLUID rows, 0 elsewhere
    ++c->nlaunch, k_fluid_volsum<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(c->g, c->type, rhs, c->part);
    ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(c->part, RED_BLOCKS, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN);
    IBM_LAUNCHED(c);
    IBM_CUDA(c, cudaMemcpyAsync(c->b, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
    ++c->nlaunch, k_sub_mean<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, c->type, c->b, c->scal + S_MEAN, 0);
    IBM_LAUNCHED(c);
    // GHOST rows of b are 0 (homogeneous Neumann on the body)
    if (c->ng > 0) {
        ++c->nlaunch, k_zero_at<<<(unsigned)((c->ng + 255) / 256), 256, 0, c->s>>>(c->ng, c->gidx, c->b);
        IBM_LAUNCHED(c);
    }
    double bn2;
    IBM_TRY(norm2(c, c->b, &bn2));
    const double bnorm = sqrt(bn2);
    int outer = 0, inner = 0;
    double rel = 0.0;
    ibm_status status = IBM_OK;
    if (!(bnorm > 1e-300)) {
        IBM_CUDA(c, cudaMemsetAsync(phi, 0, sizeof(double) * n, c->s));
        rel = 0.0;
    } else {
        std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
        bool done = false;
        while (!done) {
            // r = P(b - A phi)
            IBM_TRY(apply_PA(c, phi, c->b, -1.0, c->rr));
            double rn2;
            IBM_TRY(norm2(c, c->rr, &rn2));
            const double beta = sqrt(rn2);
            rel = beta / bnorm;
            if (!isfinite(rel)) { status = c->fail(IBM_ERR_DIVERGED, "Poisson residual is not finite"); break; }
            if (rel <= rtol) break;
            if (outer >= maxit) { status = IBM_ERR_NOT_CONVERGED; break; }
            ++c->nlaunch, k_scale<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, c->V[0], c->rr, 1.0 / beta);
            IBM_LAUNCHED(c);
            std::fill(gv.begin(), gv.end(), 0.0);
            gv[0] = beta;
            int jlast = -1;
            for (int j = 0; j < m && outer < maxit; ++j) {
                IBM_TRY(apply_prec(c, c->V[j], c->Z[j]));
                inner += c->opts.inner_iters;
                IBM_TRY(apply_PA(c, c->Z[j], nullptr, 1.0, c->w));
                // classical Gram-Schmidt, once, with a second pass when the
                // norm drops by more than 0.7 (Daniel-Gragg-Kaufman-Stewart)
                double hcol[17] = {0};
                double wbefore2 = 0.0, wafter2 = 0.0;
                for (int pass = 0; pass < 2; ++pass) {
                    kt_begin(c, K_MDOT);
                    ++c->nlaunch, k_mdot<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, c->w, (const double *const *)c->Vdev, j + 1,
                                                                  c->part);
                    kt_end(c, K_MDOT);
                    ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(c->part, RED_BLOCKS, j + 2, 1.0, c->scal + S_MD);
                    IBM_LAUNCHED(c);
                    IBM_TRY(sync_scalars(c, S_MD + j + 2));
                    Coef h{};
                    for (int i = 0; i <= j; ++i) h.v[i] = c->hscal[S_MD + i];
                    wbefore2 = c->hscal[S_MD + j + 1];
                    kt_begin(c, K_ORTH);
                    ++c->nlaunch, k_orth<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, c->w, (const double *const *)c->Vdev, j + 1, h,
                                                                  c->part);
                    kt_end(c, K_ORTH);
                    ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(c->part, RED_BLOCKS, 1, 1.0, c->scal + S_TMP);
                    IBM_LAUNCHED(c);
                    IBM_TRY(sync_scalars(c, S_TMP + 1));
                    wafter2 = c->hscal[S_TMP];
                    for (int i = 0; i <= j; ++i) hcol[i] += h.v[i];
                    if (wafter2 > 0.49 * wbefore2) break;
                }
                const double hn = sqrt(wafter2);
                ++outer;
                for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
                H[(size_t)(j + 1) * m + j] = hn;
                if (!isfinite(hn)) { status = c->fail(IBM_ERR_DIVERGED, "FGMRES breakdown (non-finite)"); done = true; break; }
                // apply previous rotations to column j
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
                    ++c->nlaunch, k_scale<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, c->V[j + 1], c->w, 1.0 / hn);
                    IBM_LAUNCHED(c);
                }
                if (est <= rtol || hn == 0.0) break;
            }
            if (done) break;
            if (jlast < 0) { status = IBM_ERR_NOT_CONVERGED; break; }
            // back substitution H y = g
            for (int i = jlast; i >= 0; --i) {
                double s = gv[i];
                for (int k = i + 1; k <= jlast; ++k) s -= H[(size_t)i * m + k] * y[k];
                y[i] = s / H[(size_t)i * m + i];
            }
            Coef yc{};
            for (int i = 0; i <= jlast; ++i) yc.v[i] = y[i];
            ++c->nlaunch, k_xupd<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, phi, (const double *const *)c->Zdev, jlast + 1, yc);
            IBM_LAUNCHED(c);
        }
        // normalise: zero volume-weighted FLUID mean, shift ghosts too
        ++c->nlaunch, k_fluid_volsum<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(c->g, c->type, phi, c->part);
        ++c->nlaunch, k_finalize<<<1, RED_THREADS, 0, c->s>>>(c->part, RED_BLOCKS, 1, 1.0 / c->fluid_vol, c->scal + S_MEAN);
        ++c->nlaunch, k_sub_mean<<<RED_BLOCKS, RED_THREADS, 0, c->s>>>(n, c->type, phi, c->scal + S_MEAN, 1);
        IBM_LAUNCHED(c);
    }
    IBM_CUDA(c, cudaEventRecord(c->ev1, c->s));
    IBM_CUDA(c, cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    IBM_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    if (st) {
        st->outer_iters = outer;
        st->inner_iters = inner;
        st->rel_residual = rel;
        st->lambda_est = 0.0;
        st->ms = ms;
    }
    if (status == IBM_ERR_NOT_CONVERGED)
        c->fail(IBM_ERR_NOT_CONVERGED, "Poisson solve reached its iteration limit");
    return status;
}

}  // namespace ibm
