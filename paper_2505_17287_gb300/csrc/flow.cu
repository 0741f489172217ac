// Fractional step around the Poisson solve (Section 2.1 of the paper):
// conservative central convection (Eq. 1) with Adams-Bashforth-2, Crank-
// Nicolson diffusion solved by red-black Gauss-Seidel with the Dirichlet
// ghost-cell rows of Section 2.2, face velocities and their divergence, and
// the projection that makes the face velocities divergence-free. All FP64.
#include "ctx.cuh"

#include <math.h>

namespace ibm {

enum { F_NET = 0, F_AREA = 1 };

// per component, per outer face: Dirichlet flag and value
struct BCInfo {
    int dir[3][6];
    double val[3][6];
    int code[6];
    double uinf[3];
};

static BCInfo make_bc(const Ctx *c) {
    BCInfo b{};
    for (int f = 0; f < 6; ++f) b.code[f] = c->desc.bc[f];
    for (int a = 0; a < 3; ++a) b.uinf[a] = c->desc.u_inf[a];
    for (int comp = 0; comp < 3; ++comp)
        for (int f = 0; f < 6; ++f) {
            const int axis = f / 2, code = c->desc.bc[f];
            if (code == IBM_BC_INFLOW) { b.dir[comp][f] = 1; b.val[comp][f] = c->desc.u_inf[comp]; }
            else if (code == IBM_BC_SLIP && comp == axis) { b.dir[comp][f] = 1; b.val[comp][f] = 0.0; }
            else { b.dir[comp][f] = 0; b.val[comp][f] = 0.0; }
        }
    return b;
}

__device__ __forceinline__ void ijk(int64_t c, int nx, int ny, int &i, int &j, int &k) {
    const int64_t t = c / nx;
    i = (int)(c - t * nx);
    j = (int)(t % ny);
    k = (int)(t / ny);
}

// face indices of the low face of cell (i,j,k) along each axis
__device__ __forceinline__ int64_t fx_lo(const GridDev &g, int i, int j, int k) {
    return (int64_t)i + (int64_t)(g.nx + 1) * (j + (int64_t)g.ny * k);
}
__device__ __forceinline__ int64_t fy_lo(const GridDev &g, int i, int j, int k) {
    return (int64_t)i + (int64_t)g.nx * (j + (int64_t)(g.ny + 1) * k);
}
__device__ __forceinline__ int64_t fz_lo(const GridDev &g, int i, int j, int k) {
    return (int64_t)i + (int64_t)g.nx * (j + (int64_t)g.ny * k);
}

struct Fields3 {
    double *p[3];
};
struct CFields3 {
    const double *p[3];
};

// one of three values by a runtime index, by selection
template <typename P>
__device__ __forceinline__ P pick3(int q, P a, P b, P c) { return q == 0 ? a : (q == 1 ? b : c); }

// Convective term N^n, explicit viscous term and the AB2 + CN right-hand side
// on FLUID cells; other cells get rhs = 0 and N = 0. Per axis the face area
// over the volume is 1/width, and the viscous face coefficients are the
// pressure operator's per-axis coefficients; a Dirichlet wall contributes
// 2 (value - u_c) / width^2.
__global__ void k_conv_rhs(GridDev g, const uint8_t *__restrict__ type, const double *__restrict__ dg, CFields3 u,
                           CFields3 F, CFields3 Nold, int first, const uint8_t *__restrict__ fresh, Fields3 Nnew,
                           Fields3 rhs, BCInfo bc, double dt, double alpha, int ncomp) {
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (type[c] != FLUID) {
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (q < ncomp) { Nnew.p[q][c] = 0.0; rhs.p[q][c] = 0.0; }
            continue;
        }
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        const int idx[3] = {i, j, k};
        const int nn[3] = {g.nx, g.ny, g.nz};
        const int64_t st[3] = {1, sy, sz};
        const double rw[3] = {g.rdx[i], g.rdy[j], g.rdz[k]};
        const double hrw[3] = {0.5 * rw[0], 0.5 * rw[1], 0.5 * rw[2]};
        const double cm[3] = {g.cxm[i], g.cym[j], g.czm[k]}, cp[3] = {g.cxp[i], g.cyp[j], g.czp[k]};
        double Flo[3], Fhi[3];
        Flo[0] = F.p[0][fx_lo(g, i, j, k)];
        Fhi[0] = F.p[0][fx_lo(g, i, j, k) + 1];
        Flo[1] = F.p[1][fy_lo(g, i, j, k)];
        Fhi[1] = F.p[1][fy_lo(g, i, j, k) + g.nx];
        if (g.ndim == 3) {
            Flo[2] = F.p[2][fz_lo(g, i, j, k)];
            Fhi[2] = F.p[2][fz_lo(g, i, j, k) + sz];
        } else {
            Flo[2] = Fhi[2] = 0.0;
        }
        const double dint = dg[c];   // sum of the interior face coefficients
        // N = sum over axes of (F_hi (u_c + u_hi) - F_lo (u_c + u_lo)) / (2 w)
        //   = u_c sum_a (fh_a - fl_a) + sum_a (fh_a u_hi - fl_a u_lo),
        // fh = F_hi / (2 w), fl = F_lo / (2 w) shared by the components (the
        // factored form takes a third of the FP64 operations per component);
        // at a wall u_lo (u_hi) is 2 v - u_c for a Dirichlet value v and u_c
        // otherwise (zero gradient)
        // (the axis loops are unrolled to their bound of 3, so that these
        // small arrays stay in registers: indexed by a loop counter they went
        // to local memory; the component loop stays rolled, which keeps the
        // registers of one component live at a time)
        double fl[3], fh[3], dF = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a >= g.ndim) break;
            fl[a] = hrw[a] * Flo[a];
            fh[a] = hrw[a] * Fhi[a];
            dF += fh[a] - fl[a];
        }
        const double c15 = 1.5 * dt, c05 = 0.5 * dt;
#pragma unroll 1
        for (int q = 0; q < ncomp; ++q) {
            // per-component pointers and wall data by selection (indexing the
            // parameter arrays with q would copy them to local memory)
            const double *uq = pick3(q, u.p[0], u.p[1], u.p[2]);
            const double *noq = pick3(q, Nold.p[0], Nold.p[1], Nold.p[2]);
            double *nnq = pick3(q, Nnew.p[0], Nnew.p[1], Nnew.p[2]);
            double *rq = pick3(q, rhs.p[0], rhs.p[1], rhs.p[2]);
            const double uc = uq[c];
            // lap = off - D uc with off the neighbour (and Dirichlet wall)
            // terms and D the diagonal; src is the wall values' share of the
            // implicit half of Crank-Nicolson
            double N = dF * uc, off = 0.0, D = dint, src = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a >= g.ndim) break;
                double ulo, uhi;
                if (idx[a] > 0) {
                    ulo = uq[c - st[a]];
                    off += cm[a] * ulo;
                } else if (pick3(q, bc.dir[0][2 * a], bc.dir[1][2 * a], bc.dir[2][2 * a])) {
                    const double v = pick3(q, bc.val[0][2 * a], bc.val[1][2 * a], bc.val[2][2 * a]), w2 = 2.0 * rw[a] * rw[a];
                    ulo = 2.0 * v - uc;
                    off += w2 * v;
                    D += w2;
                    src += w2 * v;
                } else {
                    ulo = uc;
                }
                if (idx[a] < nn[a] - 1) {
                    uhi = uq[c + st[a]];
                    off += cp[a] * uhi;
                } else if (pick3(q, bc.dir[0][2 * a + 1], bc.dir[1][2 * a + 1], bc.dir[2][2 * a + 1])) {
                    const double v = pick3(q, bc.val[0][2 * a + 1], bc.val[1][2 * a + 1], bc.val[2][2 * a + 1]), w2 = 2.0 * rw[a] * rw[a];
                    uhi = 2.0 * v - uc;
                    off += w2 * v;
                    D += w2;
                    src += w2 * v;
                } else {
                    uhi = uc;
                }
                N += fh[a] * uhi - fl[a] * ulo;
            }
            // Euler start on the first step, and at fresh cells (no history)
            const double No = (first || (fresh && fresh[c])) ? N : noq[c];
            nnq[c] = N;
            rq[c] = (uc - c15 * N + c05 * No) + alpha * ((off - D * uc) + src);
        }
    }
}

// diagonal of (I - alpha L0) for component q at FLUID cell (i, j, k)
__device__ __forceinline__ double helm_D(const GridDev &g, const BCInfo &bc, int q, double alpha, int i, int j,
                                         int k) {
    double d = g.cxs[i] + g.cys[j] + (g.ndim == 3 ? g.czs[k] : 0.0);
    const bool edge = i == 0 || i == g.nx - 1 || j == 0 || j == g.ny - 1 ||
                      (g.ndim == 3 && (k == 0 || k == g.nz - 1));
    if (edge) {
        const double rx2 = 2.0 * g.rdx[i] * g.rdx[i], ry2 = 2.0 * g.rdy[j] * g.rdy[j];
        const double rz2 = 2.0 * g.rdz[k] * g.rdz[k];
        if (i == 0 && bc.dir[q][0]) d += rx2;
        if (i == g.nx - 1 && bc.dir[q][1]) d += rx2;
        if (j == 0 && bc.dir[q][2]) d += ry2;
        if (j == g.ny - 1 && bc.dir[q][3]) d += ry2;
        if (g.ndim == 3) {
            if (k == 0 && bc.dir[q][4]) d += rz2;
            if (k == g.nz - 1 && bc.dir[q][5]) d += rz2;
        }
    }
    return 1.0 + alpha * d;
}

// inverse diagonal of (I - alpha L0) for component q on FLUID cells
__global__ void k_helm_diag(GridDev g, const uint8_t *__restrict__ type, BCInfo bc, int q, double alpha,
                            double *__restrict__ hinv) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (type[c] != FLUID) { hinv[c] = 0.0; continue; }
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        hinv[c] = 1.0 / helm_D(g, bc, q, alpha, i, j, k);
    }
}

// the viscous face coefficients times alpha (per axis, low and high face)
struct HelmCoef {
    const double *xm, *xp, *ym, *yp, *zm, *zp;
};

// s0 + alpha sum_f c_f u_nb over the interior faces, accumulated onto s0
// (one FP64 FMA per face: the scaling by alpha is folded into the stored
// coefficients)
__device__ __forceinline__ double visc_sum(const GridDev &g, const HelmCoef &h, const double *__restrict__ u,
                                           int64_t c, int i, int j, int k, double s0) {
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    double s = s0;
    if (i > 0) s += h.xm[i] * u[c - 1];
    if (i < g.nx - 1) s += h.xp[i] * u[c + 1];
    if (j > 0) s += h.ym[j] * u[c - sy];
    if (j < g.ny - 1) s += h.yp[j] * u[c + sy];
    if (g.ndim == 3) {
        if (k > 0) s += h.zm[k] * u[c - sz];
        if (k < g.nz - 1) s += h.zp[k] * u[c + sz];
    }
    return s;
}

__global__ void k_scaled_copy(int n, const double *__restrict__ src, double a, double *__restrict__ dst) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = a * src[t];
}

// Poisson initial guess by polynomial extrapolation of the last pressures:
// order 0 phi^n, 1 2 phi^n - phi^(n-1), 2 3 phi^n - 3 phi^(n-1) + phi^(n-2)
// (phi changes smoothly between steps: on the 9.4M-cell wing the linear
// guess saves ~10% of the iterations of phi^n, the quadratic one ~6% more);
// the history shifts by one
__global__ void k_phi_guess(int64_t n, double *__restrict__ p, double *__restrict__ pp, double *__restrict__ pp2,
                            int order) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const double t = p[c], t1 = pp[c];
        if (order == 1) p[c] = 2.0 * t - t1;
        else if (order == 2) p[c] = 3.0 * (t - t1) + pp2[c];
        pp2[c] = t1;
        pp[c] = t;
    }
}

// order of the Poisson guess of the step about to run. Neither phi^0 (the
// zero start) nor phi^1 (the impulsive first step, far from the pressures
// that follow: extrapolating from it cost the third step of a 208M-cell case
// ~30% more iterations) is extrapolated from: linear on the fourth step,
// quadratic from the fifth
static int phi_order(const Ctx *c) { return c->nstep >= 4 ? 2 : (c->nstep == 3 ? 1 : 0); }

// Helmholtz (I - alpha L0) u = rhs: one red-black colour on FLUID cells;
// SOR: u += w (Gauss-Seidel value - u)
template <bool SOR>
__global__ void k_helm_rb(GridDev g, HelmCoef h, const uint8_t *__restrict__ type, const double *__restrict__ rhs,
                          const double *__restrict__ hinv, double *__restrict__ u, int col, double w) {
    const int64_t row = blockIdx.x;
    int j, k;
    row_jk((uint32_t)blockIdx.x, g.fny, g.ny, j, k);
    const int i = 2 * (blockIdx.y * blockDim.x + threadIdx.x) + ((j + k + col) & 1);
    if (i >= g.nx) return;
    const int64_t c = row * g.nx + i;
    if (type[c] != FLUID) return;
    const double gs = visc_sum(g, h, u, c, i, j, k, rhs[c]) * hinv[c];
    if (SOR) {
        const double uc = u[c];
        u[c] = uc + w * (gs - uc);
    } else {
        u[c] = gs;
    }
}

// one damped-Jacobi sweep of the Helmholtz system: out = u + w (D^{-1}(rhs +
// alpha L_off u) - u) on FLUID cells, u elsewhere (ghost rows are refreshed after)
__global__ void k_helm_jacobi(GridDev g, HelmCoef h, const uint8_t *__restrict__ type, const double *__restrict__ rhs,
                              const double *__restrict__ hinv, const double *__restrict__ u, double *__restrict__ out,
                              double w) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        const double uc = u[c];
        if (type[c] != FLUID) { out[c] = uc; continue; }
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        out[c] = uc + w * (visc_sum(g, h, u, c, i, j, k, rhs[c]) * hinv[c] - uc);
    }
}

// residual of the Helmholtz system on FLUID rows; partial columns |r|^2, |rhs|^2
// (the diagonal is formed again rather than divided out of hinv: an FP64
// division costs several times the few adds)
__global__ void k_helm_resid(GridDev g, HelmCoef h, const uint8_t *__restrict__ type, const double *__restrict__ rhs,
                             BCInfo bc, int q, const double *__restrict__ u, double alpha,
                             double *__restrict__ part) {
    __shared__ double sh[32];
    double rr = 0.0, bb = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (type[c] != FLUID) continue;
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        const double r = visc_sum(g, h, u, c, i, j, k, rhs[c]) - u[c] * helm_D(g, bc, q, alpha, i, j, k);
        rr += r * r;
        bb += rhs[c] * rhs[c];
    }
    rr = block_sum<RED_THREADS>(rr, sh);
    bb = block_sum<RED_THREADS>(bb, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = rr;
        part[gridDim.x + blockIdx.x] = bb;
    }
}

// Dirichlet ghost rows for up to three components at once:
// tmp[q*ng + g] = (2 - bv) u_BI - sum_m wv_m u_m, with u_BI the body velocity
// at the intercept (ubi, 3 per ghost; null: body at rest, u_BI = 0); the
// fields u.p[0..ncomp) are velocity components comp0, comp0 + 1, ...
__global__ void k_vghost_compute(GhostDev gh, Fields3 u, int ncomp, const double *__restrict__ ubi, int comp0,
                                 double *__restrict__ tmp, double *__restrict__ res, int want_res) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    __shared__ double sh[32];
    double r2 = 0.0;
    if (q < gh.ng) {
        for (int cq = 0; cq < ncomp; ++cq) {
            const double *uu = u.p[cq];
            // (u.p[cq] is velocity component comp0 + cq)
            double s = ubi ? (2.0 - gh.bv[q]) * ubi[3 * q + comp0 + cq] : 0.0;
            for (int m = 0; m < 8; ++m) s -= gh.wv[8 * q + m] * uu[gh.sidx[8 * q + m]];
            tmp[cq * gh.ng + q] = s;
            const double d = s - uu[gh.gidx[q]];
            r2 = fmax(r2, fabs(d));
        }
    }
    if (want_res) {
        r2 = warp_max(r2);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = r2;
        __syncthreads();
        if (threadIdx.x < 32) {
            double t = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
            t = warp_max(t);
            if (threadIdx.x == 0) res[blockIdx.x] = t;
        }
    }
}
__global__ void k_vghost_scatter(GhostDev gh, Fields3 u, int ncomp, const double *__restrict__ tmp) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= gh.ng) return;
    for (int cq = 0; cq < ncomp; ++cq) u.p[cq][gh.gidx[q]] = tmp[cq * gh.ng + q];
}
__global__ void k_max_final(const double *__restrict__ part, int n, double *__restrict__ out) {
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, part[i]);
    m = warp_max(m);
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_max(t);
        if (threadIdx.x == 0) *out = t;
    }
}

// face velocities of axis a from cell values (interior and outer faces)
__global__ void k_faces(GridDev g, const uint8_t *__restrict__ type, const double *__restrict__ ua, int a,
                        BCInfo bc, double *__restrict__ Fa, FastDiv fdx, FastDiv fdy) {
    const int nfx = g.nx + (a == 0), nfy = g.ny + (a == 1), nfz = g.nz + (a == 2);
    const int64_t nf = (int64_t)nfx * nfy * nfz;
    const int64_t st = a == 0 ? 1 : (a == 1 ? (int64_t)g.nx : (int64_t)g.nx * g.ny);
    const int nax = a == 0 ? g.nx : (a == 1 ? g.ny : g.nz);
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = fdx.div((uint32_t)f), fkk = fdy.div(t);
        const int fi = (int)((uint32_t)f - t * (uint32_t)nfx), fj = (int)(t - fkk * (uint32_t)nfy), fk = (int)fkk;
        const int fa = a == 0 ? fi : (a == 1 ? fj : fk);
        // cell on the high side (index fa along a) and on the low side (fa-1)
        const int ci = fi, cj = fj, ck = fk;
        double v;
        if (fa == 0 || fa == nax) {
            const int side = fa == 0 ? 0 : 1;
            const int code = bc.code[2 * a + side];
            if (code == IBM_BC_INFLOW) v = bc.uinf[a];
            else if (code == IBM_BC_SLIP) v = 0.0;
            else {
                const int64_t cc = side == 0 ? (int64_t)ci + (int64_t)g.nx * (cj + (int64_t)g.ny * ck)
                                             : (int64_t)(a == 0 ? ci - 1 : ci) +
                                                   (int64_t)g.nx * ((a == 1 ? cj - 1 : cj) + (int64_t)g.ny * (a == 2 ? ck - 1 : ck));
                v = type[cc] == FLUID ? ua[cc] : 0.0;
            }
        } else {
            const int64_t cR = (int64_t)ci + (int64_t)g.nx * (cj + (int64_t)g.ny * ck);
            const int64_t cL = cR - st;
            const uint8_t tL = type[cL], tR = type[cR];
            const bool ok = tL != DEAD && tR != DEAD && (tL == FLUID || tR == FLUID);
            v = ok ? 0.5 * (ua[cL] + ua[cR]) : 0.0;
        }
        Fa[f] = v;
    }
}

// net inflow through the outer faces and the FLUID outflow area
__global__ void k_bnd_flux(GridDev g, const uint8_t *__restrict__ type, CFields3 F, BCInfo bc, double *__restrict__ part) {
    __shared__ double sh[32];
    double net = 0.0, area = 0.0;
    const int64_t nyz = (int64_t)g.ny * g.nz, nxz = (int64_t)g.nx * g.nz, nxy = (int64_t)g.nx * g.ny;
    const int64_t tot = 2 * nyz + 2 * nxz + (g.ndim == 3 ? 2 * nxy : 0);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int a, side;
        int64_t r = e;
        if (r < 2 * nyz) { a = 0; side = (int)(r / nyz); r %= nyz; }
        else if ((r -= 2 * nyz) < 2 * nxz) { a = 1; side = (int)(r / nxz); r %= nxz; }
        else { r -= 2 * nxz; a = 2; side = (int)(r / nxy); r %= nxy; }
        int i, j, k;
        int64_t fidx, cidx;
        double A;
        if (a == 0) {
            j = (int)(r % g.ny); k = (int)(r / g.ny); i = side ? g.nx - 1 : 0;
            fidx = (int64_t)(side ? g.nx : 0) + (int64_t)(g.nx + 1) * (j + (int64_t)g.ny * k);
            A = g.dy[j] * g.dz[k];
        } else if (a == 1) {
            i = (int)(r % g.nx); k = (int)(r / g.nx); j = side ? g.ny - 1 : 0;
            fidx = (int64_t)i + (int64_t)g.nx * ((side ? g.ny : 0) + (int64_t)(g.ny + 1) * k);
            A = g.dx[i] * g.dz[k];
        } else {
            i = (int)(r % g.nx); j = (int)(r / g.nx); k = side ? g.nz - 1 : 0;
            fidx = (int64_t)i + (int64_t)g.nx * (j + (int64_t)g.ny * (side ? g.nz : 0));
            A = g.dx[i] * g.dy[j];
        }
        cidx = (int64_t)i + (int64_t)g.nx * (j + (int64_t)g.ny * k);
        const double v = F.p[a][fidx];
        net += (side == 0 ? 1.0 : -1.0) * (A * v);
        if (bc.code[2 * a + side] == IBM_BC_OUTFLOW && type[cidx] == FLUID) area += A;
    }
    net = block_sum<RED_THREADS>(net, sh);
    area = block_sum<RED_THREADS>(area, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = net;
        part[gridDim.x + blockIdx.x] = area;
    }
}

// uniform correction of OUTFLOW faces over FLUID cells: corr = net / area
__global__ void k_outflow_corr(GridDev g, const uint8_t *__restrict__ type, Fields3 F, BCInfo bc,
                               const double *__restrict__ sums) {
    const double area = sums[F_AREA];
    if (!(area > 0.0)) return;
    const double corr = sums[F_NET] / area;
    const int64_t nyz = (int64_t)g.ny * g.nz, nxz = (int64_t)g.nx * g.nz, nxy = (int64_t)g.nx * g.ny;
    const int64_t tot = 2 * nyz + 2 * nxz + (g.ndim == 3 ? 2 * nxy : 0);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int a, side;
        int64_t r = e;
        if (r < 2 * nyz) { a = 0; side = (int)(r / nyz); r %= nyz; }
        else if ((r -= 2 * nyz) < 2 * nxz) { a = 1; side = (int)(r / nxz); r %= nxz; }
        else { r -= 2 * nxz; a = 2; side = (int)(r / nxy); r %= nxy; }
        if (bc.code[2 * a + side] != IBM_BC_OUTFLOW) continue;
        int i, j, k;
        int64_t fidx;
        if (a == 0) {
            j = (int)(r % g.ny); k = (int)(r / g.ny); i = side ? g.nx - 1 : 0;
            fidx = (int64_t)(side ? g.nx : 0) + (int64_t)(g.nx + 1) * (j + (int64_t)g.ny * k);
        } else if (a == 1) {
            i = (int)(r % g.nx); k = (int)(r / g.nx); j = side ? g.ny - 1 : 0;
            fidx = (int64_t)i + (int64_t)g.nx * ((side ? g.ny : 0) + (int64_t)(g.ny + 1) * k);
        } else {
            i = (int)(r % g.nx); j = (int)(r / g.nx); k = side ? g.nz - 1 : 0;
            fidx = (int64_t)i + (int64_t)g.nx * (j + (int64_t)g.ny * (side ? g.nz : 0));
        }
        const int64_t cidx = (int64_t)i + (int64_t)g.nx * (j + (int64_t)g.ny * k);
        if (type[cidx] == FLUID) F.p[a][fidx] += (side == 0 ? -corr : corr);
    }
}

// b_raw = div(F) / dt on FLUID cells, 0 elsewhere
__global__ void k_divergence(GridDev g, const uint8_t *__restrict__ type, CFields3 F, double inv_dt,
                             double *__restrict__ out) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (type[c] != FLUID) { out[c] = 0.0; continue; }
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        // (face area x flux difference) / volume = flux difference / width, per
        // axis: stored reciprocal widths, no FP64 division
        double d = (F.p[0][fx_lo(g, i, j, k) + 1] - F.p[0][fx_lo(g, i, j, k)]) * g.rdx[i];
        d += (F.p[1][fy_lo(g, i, j, k) + g.nx] - F.p[1][fy_lo(g, i, j, k)]) * g.rdy[j];
        if (g.ndim == 3)
            d += (F.p[2][fz_lo(g, i, j, k) + (int64_t)g.nx * g.ny] - F.p[2][fz_lo(g, i, j, k)]) * g.rdz[k];
        out[c] = d * inv_dt;
    }
}

// projection of the interior faces of axis a that have a FLUID side
// (fdx, fdy: multiply-shift dividers by the face counts along x and y; the
// gradient multiplies by the stored reciprocal centre spacing)
__global__ void k_project_faces(GridDev g, const uint8_t *__restrict__ type, const double *__restrict__ phi, int a,
                                double dt, double *__restrict__ Fa, FastDiv fdx, FastDiv fdy) {
    const int nfx = g.nx + (a == 0), nfy = g.ny + (a == 1), nfz = g.nz + (a == 2);
    const int64_t nf = (int64_t)nfx * nfy * nfz;
    const int64_t st = a == 0 ? 1 : (a == 1 ? (int64_t)g.nx : (int64_t)g.nx * g.ny);
    const int nax = a == 0 ? g.nx : (a == 1 ? g.ny : g.nz);
    const double *rh = a == 0 ? g.rhx : (a == 1 ? g.rhy : g.rhz);
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = fdx.div((uint32_t)f), fk = fdy.div(t);
        const int fi = (int)((uint32_t)f - t * (uint32_t)nfx), fj = (int)(t - fk * (uint32_t)nfy);
        const int fa = a == 0 ? fi : (a == 1 ? fj : (int)fk);
        if (fa == 0 || fa == nax) continue;
        const int64_t cR = (int64_t)fi + (int64_t)g.nx * (fj + (int64_t)g.ny * fk);
        const int64_t cL = cR - st;
        if (type[cL] != FLUID && type[cR] != FLUID) continue;
        Fa[f] -= dt * (phi[cR] - phi[cL]) * rh[fa];
    }
}

// cell velocities on FLUID cells: u_a -= dt * mean of the two face gradients
__global__ void k_project_cells(GridDev g, const uint8_t *__restrict__ type, const double *__restrict__ phi,
                                CFields3 us, Fields3 u, double dt) {
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t t = type[c];
        if (t != FLUID) {
            u.p[0][c] = us.p[0][c];
            u.p[1][c] = us.p[1][c];
            if (g.ndim == 3) u.p[2][c] = us.p[2][c];
            continue;
        }
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        const double pc = phi[c];
        double glo, ghi;
        glo = i > 0 ? (pc - phi[c - 1]) * g.rhx[i] : 0.0;
        ghi = i < g.nx - 1 ? (phi[c + 1] - pc) * g.rhx[i + 1] : 0.0;
        u.p[0][c] = us.p[0][c] - dt * (0.5 * (glo + ghi));
        glo = j > 0 ? (pc - phi[c - sy]) * g.rhy[j] : 0.0;
        ghi = j < g.ny - 1 ? (phi[c + sy] - pc) * g.rhy[j + 1] : 0.0;
        u.p[1][c] = us.p[1][c] - dt * (0.5 * (glo + ghi));
        if (g.ndim == 3) {
            glo = k > 0 ? (pc - phi[c - sz]) * g.rhz[k] : 0.0;
            ghi = k < g.nz - 1 ? (phi[c + sz] - pc) * g.rhz[k + 1] : 0.0;
            u.p[2][c] = us.p[2][c] - dt * (0.5 * (glo + ghi));
        }
    }
}

__global__ void k_init_cells(int64_t n, const uint8_t *__restrict__ type, Fields3 u, double u0, double u1, double u2,
                             int ncomp, double *__restrict__ p) {
    const double v[3] = {u0, u1, u2};
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const bool fl = type[c] == FLUID;
        for (int q = 0; q < ncomp; ++q) u.p[q][c] = fl ? v[q] : 0.0;
        p[c] = 0.0;
    }
}

// max |div F - mean| over FLUID cells, in two passes
__global__ void k_div_stats(GridDev g, const uint8_t *__restrict__ type, const double *__restrict__ div,
                            const double *__restrict__ mean, double *__restrict__ part) {
    const double m = mean ? *mean : 0.0;
    double mx = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x)
        if (type[c] == FLUID) mx = fmax(mx, fabs(div[c] - m));
    __shared__ double sh[32];
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_max(t);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------

static inline dim3 rb_grid(const Ctx *c) {
    const int64_t rows = (int64_t)c->ny * c->nz;
    const int xs = (c->nx + 1) / 2;
    return dim3((unsigned)rows, (unsigned)((xs + 127) / 128), 1);
}

// body velocity at the ghosts' intercepts (null while the body is at rest)
static const double *ghost_ubi(const Ctx *c) { return c->moving ? c->ubi : nullptr; }

static ibm_status faces_from(Ctx *c, double *const *ucell) {
    const BCInfo bc = make_bc(c);
    for (int a = 0; a < c->ndim; ++a) {
        const int64_t nf = a == 0 ? c->NFx : (a == 1 ? c->NFy : c->NFz);
        const unsigned nb = (unsigned)((nf + 255) / 256 > 152 * 32 ? 152 * 32 : (nf + 255) / 256);
        ++c->nlaunch, k_faces<<<nb, 256, 0, c->s>>>(c->g, c->type, ucell[a], a, bc, c->F[a], FastDiv((uint32_t)(c->nx + (a == 0))),
                                                  FastDiv((uint32_t)(c->ny + (a == 1))));
        IBM_LAUNCHED(c);
    }
    CFields3 F{{c->F[0], c->F[1], c->F[2]}};
    ++c->nlaunch, k_bnd_flux<<<c->nred, RED_THREADS, 0, c->s>>>(c->g, c->type, F, bc, c->part);
    IBM_LAUNCHED(c);
    IBM_TRY(finalize(c, c->part, c->nred, 2, 1.0, c->scal + 56));
    Fields3 Fw{{c->F[0], c->F[1], c->F[2]}};
    ++c->nlaunch, k_outflow_corr<<<c->nred, RED_THREADS, 0, c->s>>>(c->g, c->type, Fw, bc, c->scal + 56);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

// velocity ghost refresh by Jacobi passes over the ghost rows (all
// components at once) until the largest change is below ghost_tol (relative
// to max(1, |u_inf|)) or ghost_maxit passes
static ibm_status ghost_refresh_all(Ctx *c, double *const *ucell, int *passes) {
    *passes = 0;
    if (c->ng == 0) return IBM_OK;
    const int nc = c->ndim;
    Fields3 U{{ucell[0], ucell[1], nc == 3 ? ucell[2] : ucell[1]}};
    const unsigned gb = (unsigned)((c->ng + 255) / 256);
    double scale = 1.0;
    for (int a = 0; a < 3; ++a) scale = fmax(scale, fabs(c->desc.u_inf[a]));
    const int check_every = 4;
    for (int it = 0; it < c->opts.ghost_maxit; ++it) {
        const int want = ((it + 1) % check_every == 0) || it + 1 == c->opts.ghost_maxit;
        ++c->nlaunch, k_vghost_compute<<<gb, 256, 0, c->s>>>(c->gh, U, nc, ghost_ubi(c), 0, c->gtmp, c->part, want);
        ++c->nlaunch, k_vghost_scatter<<<gb, 256, 0, c->s>>>(c->gh, U, nc, c->gtmp);
        IBM_LAUNCHED(c);
        ++*passes;
        if (want) {
            ++c->nlaunch, k_max_final<<<1, 256, 0, c->s>>>(c->part, (int)gb, c->scal + 40);
            IBM_LAUNCHED(c);
            IBM_TRY(sync_scalars(c, 41));
            const double d = c->hscal[40];
            if (!isfinite(d)) return c->fail(IBM_ERR_DIVERGED, "velocity ghost refresh produced a non-finite value");
            if (d <= c->opts.ghost_tol * scale) return IBM_OK;
        }
    }
    return IBM_OK;
}

ibm_status ghost_refresh_velocity(Ctx *c, int comp, int *iters) {
    (void)comp;
    return ghost_refresh_all(c, c->u, iters);
}

ibm_status flow_init(Ctx *c) {
    Fields3 U{{c->u[0], c->u[1], c->u[2]}};
    const unsigned nb = 152 * 16;
    ++c->nlaunch, k_init_cells<<<nb, 256, 0, c->s>>>(c->N, c->type, U, c->desc.u_inf[0], c->desc.u_inf[1], c->desc.u_inf[2],
                                      c->ndim, c->p);
    IBM_LAUNCHED(c);
    int passes = 0;
    IBM_TRY(ghost_refresh_all(c, c->u, &passes));
    IBM_TRY(faces_from(c, c->u));
    c->nstep = 0;
    c->have_nold = false;
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    return IBM_OK;
}

// sweep count of the residual test after one at s sweeps (the first test
// comes after opts.helm_check_first sweeps): gaps grow with s, so a solve
// that needs n sweeps takes O(log n) tests and overshoots by at most n / 4
__host__ __device__ __forceinline__ int helm_next_check(int s) { return s + (s / 4 > 2 ? s / 4 : 2); }

static HelmCoef helm_coef(const Ctx *c) {
    const int nx = c->desc.nx, ny = c->desc.ny, nz = c->desc.ndim == 3 ? c->desc.nz : 1;
    const double *h = c->hac;
    return HelmCoef{h, h + nx, h + 2 * nx, h + 2 * nx + ny, h + 2 * nx + 2 * ny, h + 2 * nx + 2 * ny + nz};
}

// Helmholtz solve for component q, u = ustar (initial guess u^n)
static ibm_status helm_prepare(Ctx *c) {
    const BCInfo bc = make_bc(c);
    const double alpha = c->desc.dt / (2.0 * c->desc.Re);
    if (!c->hinv_ok) {
        const int nx = c->desc.nx, ny = c->desc.ny, nz = c->desc.ndim == 3 ? c->desc.nz : 1;
        if (!c->hac) c->hac = (double *)dev_alloc(c, sizeof(double) * 2 * (size_t)(nx + ny + nz));
        if (!c->hac) return c->fail(IBM_ERR_OOM, "Helmholtz coefficient allocation failed");
        const double *src[6] = {c->g.cxm, c->g.cxp, c->g.cym, c->g.cyp, c->g.czm, c->g.czp};
        const int len[6] = {nx, nx, ny, ny, nz, nz};
        size_t off = 0;
        for (int a = 0; a < 6; ++a) {
            ++c->nlaunch, k_scaled_copy<<<(len[a] + 255) / 256, 256, 0, c->s>>>(len[a], src[a], alpha, c->hac + off);
            off += (size_t)len[a];
        }
        for (int cq = 0; cq < c->ndim; ++cq) {
            if (!c->hinv[cq]) c->hinv[cq] = (double *)dev_alloc(c, sizeof(double) * c->N);
            if (!c->hinv[cq]) return c->fail(IBM_ERR_OOM, "Helmholtz diagonal allocation failed");
            ++c->nlaunch, k_helm_diag<<<c->nelem, 256, 0, c->s>>>(c->g, c->type, bc, cq, alpha, c->hinv[cq]);
        }
        IBM_LAUNCHED(c);
        c->hinv_ok = true;
    }
    return IBM_OK;
}

// bound on the spectral radius of the Jacobi iteration of H = I - alpha L:
// alpha S / (1 + alpha S), S the largest diagonal of L, bounded per axis from
// the 1D coefficients (a Dirichlet wall counting 2 / w^2)
static double helm_rho(const Ctx *c) {
    const double alpha = c->desc.dt / (2.0 * c->desc.Re);
    auto axis_max = [](const std::vector<double> &w, const std::vector<double> &h) {
        double m = 0.0;
        const size_t n = w.size();
        for (size_t i = 0; i < n; ++i) {
            const double cm = i > 0 ? 1.0 / (h[i] * w[i]) : 2.0 / (w[i] * w[i]);
            const double cp = i + 1 < n ? 1.0 / (h[i + 1] * w[i]) : 2.0 / (w[i] * w[i]);
            m = fmax(m, cm + cp);
        }
        return m;
    };
    double S = axis_max(c->hdx, c->hhx) + axis_max(c->hdy, c->hhy);
    if (c->ndim == 3) S += axis_max(c->hdz, c->hhz);
    return alpha * S / (1.0 + alpha * S);
}

// relaxation factor of the red-black Helmholtz sweeps (opts.helm_omega; 0:
// Young's optimum 2 / (1 + sqrt(1 - rho^2)) for the bound rho, which for a
// red-black (consistently ordered) operator takes the error reduction per
// sweep from rho^2 to about omega - 1)
static double helm_omega(const Ctx *c) {
    const double w = c->opts.helm_omega;
    if (w != 0.0) return w;
    const double r = helm_rho(c);
    return 2.0 / (1.0 + sqrt(1.0 - r * r));
}

// Helmholtz by scheduled relaxation Jacobi: cycles of 8 sweeps with factors
// 1/tau_k, tau_k the Chebyshev points of [1 - rho, 1 + rho] (the spectrum of
// D^{-1} H for H = I - alpha L, rho = alpha S / (1 + alpha S) with S the
// largest diagonal of L, bounded per axis from the 1D coefficients), the
// ghost rows refreshed after every sweep; the residual test after each
// cycle is the one of the Gauss-Seidel path
static ibm_status helmholtz_srj(Ctx *c, int q, int *sweeps) {
    const double alpha = c->desc.dt / (2.0 * c->desc.Re);
    if (!c->htmp) {
        c->htmp = (double *)dev_alloc(c, sizeof(double) * c->N);
        if (!c->htmp) return c->fail(IBM_ERR_OOM, "Helmholtz buffer allocation failed");
    }
    const double rho = helm_rho(c), pi = 3.14159265358979323846;
    const int M = 8;
    double w[M];
    const int order[M] = {0, 4, 2, 6, 1, 5, 3, 7};   // bit-reversed
    for (int k = 0; k < M; ++k) w[order[k]] = 1.0 / (1.0 + rho * cos(pi * (2.0 * k + 1.0) / (2.0 * M)));
    const double *hinv = c->hinv[q];
    double *u = c->ustar[q], *t = c->htmp;
    const double *rhs = c->rhs[q];
    const unsigned gb = (unsigned)((c->ng + 255) / 256);
    *sweeps = 0;
    double rhs2 = -1.0;
    for (int it = 0; it < c->opts.helm_maxit; it += M) {
        for (int k = 0; k < M; ++k) {
            kt_begin(c, K_HELM);
            ++c->nlaunch, k_helm_jacobi<<<c->nelem, 256, 0, c->s>>>(c->g, helm_coef(c), c->type, rhs, hinv, u, t, w[k]);
            kt_end(c, K_HELM);
            if (c->ng > 0) {
                Fields3 T3{{t, t, t}};
                ++c->nlaunch, k_vghost_compute<<<gb, 256, 0, c->s>>>(c->gh, T3, 1, ghost_ubi(c), q, c->gtmp, c->part, 0);
                ++c->nlaunch, k_vghost_scatter<<<gb, 256, 0, c->s>>>(c->gh, T3, 1, c->gtmp);
            }
            IBM_LAUNCHED(c);
            double *x = u;
            u = t;
            t = x;
            ++*sweeps;
        }
        // M is even: the iterate is back in ustar[q]
        Fields3 U{{u, u, u}};
        ++c->nlaunch, k_helm_resid<<<c->nred, RED_THREADS, 0, c->s>>>(c->g, helm_coef(c), c->type, rhs, make_bc(c), q, u, alpha, c->part);
        IBM_LAUNCHED(c);
        IBM_TRY(finalize(c, c->part, c->nred, 2, 1.0, c->scal + 48));
        double gmax = 0.0;
        if (c->ng > 0) {
            ++c->nlaunch, k_vghost_compute<<<gb, 256, 0, c->s>>>(c->gh, U, 1, ghost_ubi(c), q, c->gtmp, c->part + 2 * RED_BLOCKS_MAX, 1);
            ++c->nlaunch, k_max_final<<<1, 256, 0, c->s>>>(c->part + 2 * RED_BLOCKS_MAX, (int)gb, c->scal + 50);
            IBM_LAUNCHED(c);
        }
        IBM_TRY(sync_scalars(c, 51));
        const double r2 = c->hscal[48];
        if (rhs2 < 0) rhs2 = c->hscal[49];
        if (c->ng > 0) gmax = c->hscal[50];
        if (!isfinite(r2)) return c->fail(IBM_ERR_DIVERGED, "Helmholtz residual is not finite");
        const double bn = sqrt(rhs2) > 0 ? sqrt(rhs2) : 1.0;
        double scale = 1.0;
        for (int a = 0; a < 3; ++a) scale = fmax(scale, fabs(c->desc.u_inf[a]));
        if (sqrt(r2) <= c->opts.helm_rtol * bn && gmax <= c->opts.helm_rtol * scale) return IBM_OK;
    }
    return IBM_ERR_NOT_CONVERGED;
}

// one red-black colour pass of the Helmholtz sweeps (kernel launch)
static void helm_rb(Ctx *c, const double *rhs, const double *hinv, double *u, int col) {
    const double w = helm_omega(c);
    if (w != 1.0) k_helm_rb<true><<<rb_grid(c), 128, 0, c->s>>>(c->g, helm_coef(c), c->type, rhs, hinv, u, col, w);
    else k_helm_rb<false><<<rb_grid(c), 128, 0, c->s>>>(c->g, helm_coef(c), c->type, rhs, hinv, u, col, 1.0);
}

// one Jacobi pass of the ghost rows of component q: u_G = (2 - bv) u_BI -
// sum wv u_m from the current neighbour values. The Helmholtz sweeps take
// one after each colour pass: the fluid cells next to a ghost see its value,
// which depends on fluid values near its image point, and refreshing it
// between the colours, not once per sweep, takes the 25.2M-cell wing from 6
// to 4 sweeps per component at a 1e-12 residual (the 201M-cell wing, whose
// finer cells converge more slowly, still needs 6).
static void helm_ghost_pass(Ctx *c, int q, Fields3 U, unsigned gb) {
    if (c->ng == 0) return;
    ++c->nlaunch, k_vghost_compute<<<gb, 256, 0, c->s>>>(c->gh, U, 1, ghost_ubi(c), q, c->gtmp, c->part, 0);
    ++c->nlaunch, k_vghost_scatter<<<gb, 256, 0, c->s>>>(c->gh, U, 1, c->gtmp);
}

static ibm_status helmholtz(Ctx *c, int q, int *sweeps) {
    const double alpha = c->desc.dt / (2.0 * c->desc.Re);
    IBM_TRY(helm_prepare(c));
    if (c->opts.helm_solver == 1) return helmholtz_srj(c, q, sweeps);
    const double *hinv = c->hinv[q];
    double *u = c->ustar[q];
    const double *rhs = c->rhs[q];
    int next_check = c->opts.helm_check_first;
    *sweeps = 0;
    double rhs2 = -1.0;
    const unsigned gb = (unsigned)((c->ng + 255) / 256);
    Fields3 U{{u, u, u}};
    for (int it = 0; it < c->opts.helm_maxit; ++it) {
        // each colour pass is followed by a Jacobi pass of the ghost rows
        for (int col = 0; col < 2; ++col) {
            kt_begin(c, K_HELM);
            ++c->nlaunch, helm_rb(c, rhs, hinv, u, col);
            kt_end(c, K_HELM);
            IBM_LAUNCHED(c);
            helm_ghost_pass(c, q, U, gb);
        }
        ++*sweeps;
        if (*sweeps == next_check || it + 1 == c->opts.helm_maxit) {
            next_check = helm_next_check(next_check);
            ++c->nlaunch, k_helm_resid<<<c->nred, RED_THREADS, 0, c->s>>>(c->g, helm_coef(c), c->type, rhs, make_bc(c), q, u, alpha, c->part);
            IBM_LAUNCHED(c);
            IBM_TRY(finalize(c, c->part, c->nred, 2, 1.0, c->scal + 48));
            double gmax = 0.0;
            if (c->ng > 0) {
                // ghost-row residual: largest change a further Jacobi pass would make
                ++c->nlaunch, k_vghost_compute<<<gb, 256, 0, c->s>>>(c->gh, U, 1, ghost_ubi(c), q, c->gtmp, c->part + 2 * RED_BLOCKS_MAX, 1);
                ++c->nlaunch, k_max_final<<<1, 256, 0, c->s>>>(c->part + 2 * RED_BLOCKS_MAX, (int)gb, c->scal + 50);
                IBM_LAUNCHED(c);
            }
            IBM_TRY(sync_scalars(c, 51));
            const double r2 = c->hscal[48];
            if (rhs2 < 0) rhs2 = c->hscal[49];
            if (c->ng > 0) gmax = c->hscal[50];
            if (!isfinite(r2)) return c->fail(IBM_ERR_DIVERGED, "Helmholtz residual is not finite");
            const double bn = sqrt(rhs2) > 0 ? sqrt(rhs2) : 1.0;
            double scale = 1.0;
            for (int a = 0; a < 3; ++a) scale = fmax(scale, fabs(c->desc.u_inf[a]));
            if (sqrt(r2) <= c->opts.helm_rtol * bn && gmax <= c->opts.helm_rtol * scale) return IBM_OK;
        }
    }
    return IBM_ERR_NOT_CONVERGED;
}

ibm_status flow_step(Ctx *c, ibm_step_stats *st) {
    const int nc = c->ndim;
    const double dt = c->desc.dt, alpha = dt / (2.0 * c->desc.Re);
    IBM_TRY(hist_prepare(c));
    IBM_CUDA(c, cudaEventRecord(c->ev0, c->s));
    CFields3 u{{c->u[0], c->u[1], nc == 3 ? c->u[2] : c->u[1]}};
    CFields3 F{{c->F[0], c->F[1], nc == 3 ? c->F[2] : c->F[1]}};
    CFields3 No{{c->Nold[0], c->Nold[1], nc == 3 ? c->Nold[2] : c->Nold[1]}};
    Fields3 Nn{{c->Nnew[0], c->Nnew[1], nc == 3 ? c->Nnew[2] : c->Nnew[1]}};
    Fields3 R{{c->rhs[0], c->rhs[1], nc == 3 ? c->rhs[2] : c->rhs[1]}};
    kt_begin(c, K_CONV);
    ++c->nlaunch, k_conv_rhs<<<c->nelem, 256, 0, c->s>>>(c->g, c->type, c->dg_c, u, F, No, c->have_nold ? 0 : 1, c->fresh_pending ? c->fresh : nullptr, Nn, R, make_bc(c), dt,
                                           alpha, nc);
    kt_end(c, K_CONV);
    IBM_LAUNCHED(c);
    ibm_status status = IBM_OK;
    int sweeps_total = 0;
    for (int q = 0; q < nc; ++q) {
        IBM_CUDA(c, cudaMemcpyAsync(c->ustar[q], c->u[q], sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->s));
        int sw = 0;
        ibm_status s = helmholtz(c, q, &sw);
        sweeps_total += sw;
        if (s == IBM_ERR_NOT_CONVERGED) status = s;
        else if (s != IBM_OK) return s;
    }
    IBM_TRY(faces_from(c, c->ustar));
    CFields3 Fs{{c->F[0], c->F[1], nc == 3 ? c->F[2] : c->F[1]}};
    double *braw = c->rhs[0];
    ++c->nlaunch, k_divergence<<<c->nelem, 256, 0, c->s>>>(c->g, c->type, Fs, 1.0 / dt, braw);
    IBM_LAUNCHED(c);
    ++c->nlaunch, k_phi_guess<<<c->nelem, 256, 0, c->s>>>(c->N, c->p, c->p_prev, c->p_prev2, phi_order(c));
    IBM_LAUNCHED(c);
    IBM_TRY(hist_guess(c, braw, c->p));
    IBM_CUDA(c, cudaEventRecord(c->ev2, c->s));
    ibm_solve_stats ps{};
    ibm_status s = poisson_solve(c, braw, c->p, c->opts.rtol, c->opts.max_outer, &ps);
    if (s == IBM_ERR_NOT_CONVERGED) status = s;
    else if (s != IBM_OK) return s;
    IBM_TRY(hist_store(c, c->p));
    IBM_CUDA(c, cudaEventRecord(c->ev3, c->s));
    for (int a = 0; a < nc; ++a) {
        const int64_t nf = a == 0 ? c->NFx : (a == 1 ? c->NFy : c->NFz);
        const unsigned nb = (unsigned)((nf + 255) / 256 > 152 * 32 ? 152 * 32 : (nf + 255) / 256);
        ++c->nlaunch, k_project_faces<<<nb, 256, 0, c->s>>>(c->g, c->type, c->p, a, dt, c->F[a],
                                                          FastDiv((uint32_t)(c->nx + (a == 0))),
                                                          FastDiv((uint32_t)(c->ny + (a == 1))));
    }
    IBM_LAUNCHED(c);
    CFields3 us{{c->ustar[0], c->ustar[1], nc == 3 ? c->ustar[2] : c->ustar[1]}};
    Fields3 un{{c->u[0], c->u[1], nc == 3 ? c->u[2] : c->u[1]}};
    ++c->nlaunch, k_project_cells<<<c->nelem, 256, 0, c->s>>>(c->g, c->type, c->p, us, un, dt);
    IBM_LAUNCHED(c);
    int passes = 0;
    IBM_TRY(ghost_refresh_all(c, c->u, &passes));
    for (int q = 0; q < 3; ++q) {
        double *t = c->Nold[q];
        c->Nold[q] = c->Nnew[q];
        c->Nnew[q] = t;
    }
    c->have_nold = true;
    c->nstep += 1;
    if (c->fresh_pending) {
        // the fresh cells of the last move took their Euler start
        IBM_CUDA(c, cudaMemsetAsync(c->fresh, 0, (size_t)c->N, c->s));
        c->fresh_pending = false;
    }
    IBM_CUDA(c, cudaEventRecord(c->ev1, c->s));
    IBM_CUDA(c, cudaEventSynchronize(c->ev1));
    if (st) {
        float a = 0, b = 0, t = 0;
        cudaEventElapsedTime(&t, c->ev0, c->ev1);
        cudaEventElapsedTime(&a, c->ev0, c->ev2);
        cudaEventElapsedTime(&b, c->ev3, c->ev1);
        st->steps += 1;
        st->poisson_outer += ps.outer_iters;
        st->poisson_inner += ps.inner_iters;
        st->helm_sweeps += sweeps_total;
        st->rel_residual = ps.rel_residual;
        st->ms_total += t;
        st->ms_predictor += a;
        st->ms_poisson += ps.ms;
        st->ms_projection += b;
    }
    if (status == IBM_ERR_NOT_CONVERGED) c->fail(status, "a solve in the step reached its iteration limit");
    return status;
}

// ---------------------------------------------------------------------------
// moving body: the fields after a move (Section 2.2)
// ---------------------------------------------------------------------------

__global__ void k_fresh_flags(int64_t n, const uint8_t *__restrict__ type, const uint8_t *__restrict__ old,
                              uint8_t *__restrict__ fresh) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        fresh[c] = (type[c] == FLUID && old[c] != FLUID) ? 1 : 0;
}

// fresh values, one Jacobi pass over the fresh rows (all components):
// tmp = sum_m w_m u_m + wb u_BI; res: largest change
__global__ void k_fresh_compute(int64_t nf, const int64_t *__restrict__ fidx, const int64_t *__restrict__ sidx,
                                const double *__restrict__ w, const double *__restrict__ wb,
                                const double *__restrict__ ub, Fields3 u, int ncomp, double *__restrict__ tmp,
                                double *__restrict__ res) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    __shared__ double sh[32];
    double r = 0.0;
    if (f < nf) {
        for (int cq = 0; cq < ncomp; ++cq) {
            const double *uu = u.p[cq];
            double s = wb[f] * ub[3 * f + cq];
            for (int m = 0; m < 8; ++m) s += w[8 * f + m] * uu[sidx[8 * f + m]];
            tmp[cq * nf + f] = s;
            r = fmax(r, fabs(s - uu[fidx[f]]));
        }
    }
    r = warp_max(r);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_max(t);
        if (threadIdx.x == 0) res[blockIdx.x] = t;
    }
}
__global__ void k_fresh_scatter(int64_t nf, const int64_t *__restrict__ fidx, Fields3 u, int ncomp,
                                const double *__restrict__ tmp) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    for (int cq = 0; cq < ncomp; ++cq) u.p[cq][fidx[f]] = tmp[cq * nf + f];
}
// start value of the fresh cells: the body velocity at their intercept
__global__ void k_fresh_start(int64_t nf, const int64_t *__restrict__ fidx, const double *__restrict__ ub, Fields3 u,
                              int ncomp) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    for (int cq = 0; cq < ncomp; ++cq) u.p[cq][fidx[f]] = ub[3 * f + cq];
}

__global__ void k_dead_zero(int64_t n, const uint8_t *__restrict__ type, Fields3 u, int ncomp) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        if (type[c] == DEAD)
            for (int q = 0; q < ncomp; ++q) u.p[q][c] = 0.0;
}

// interior faces of axis a next to a cell whose type changed: the face rule
// (mean of the two cells on faces with a FLUID side and no DEAD side, else 0)
__global__ void k_faces_changed(GridDev g, const uint8_t *__restrict__ type, const uint8_t *__restrict__ old,
                                const double *__restrict__ ua, int a, double *__restrict__ Fa) {
    const int nfx = g.nx + (a == 0), nfy = g.ny + (a == 1);
    const int64_t nf = (int64_t)nfx * nfy * (g.nz + (a == 2));
    const int64_t st = a == 0 ? 1 : (a == 1 ? g.nx : (int64_t)g.nx * g.ny);
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = f / nfx;
        const int i = (int)(f - t * nfx), j = (int)(t % nfy), k = (int)(t / nfy);
        const int ia = a == 0 ? i : (a == 1 ? j : k);
        const int na = a == 0 ? g.nx : (a == 1 ? g.ny : g.nz);
        if (ia == 0 || ia == na) continue;   // outer faces keep their values
        const int64_t cR = (int64_t)i + (int64_t)g.nx * (j + (int64_t)g.ny * k), cL = cR - st;
        if (type[cL] == old[cL] && type[cR] == old[cR]) continue;
        const uint8_t L = type[cL], R = type[cR];
        const bool ok = L != DEAD && R != DEAD && (L == FLUID || R == FLUID);
        Fa[f] = ok ? 0.5 * (ua[cL] + ua[cR]) : 0.0;
    }
}

ibm_status flow_move(Ctx *c) {
    const int nc = c->ndim;
    Fields3 U{{c->u[0], c->u[1], nc == 3 ? c->u[2] : c->u[1]}};
    // body velocity at the ghosts' intercepts
    if (c->ng > c->ubi_cap || !c->ubi) {
        dev_free(c, c->ubi);
        c->ubi_cap = c->ng > 0 ? c->ng : 1;
        c->ubi = (double *)dev_alloc(c, sizeof(double) * 3 * c->ubi_cap);
        if (!c->ubi) return c->fail(IBM_ERR_OOM, "body velocity allocation failed");
    }
    IBM_TRY(geom_body_velocity(c, c->ng, c->bi, c->ubi));
    // fresh cells: FLUID now, not FLUID before the move
    ++c->nlaunch, k_fresh_flags<<<c->nelem, 256, 0, c->s>>>(c->N, c->type, c->type_old, c->fresh);
    IBM_LAUNCHED(c);
    int64_t *fidx = nullptr, nf = 0;
    IBM_TRY(compact_flags(c, c->fresh, &fidx, &nf));
    c->n_fresh = nf;
    if (nf > 0) {
        double *fbi = (double *)dev_alloc(c, sizeof(double) * 3 * nf);
        double *fub = (double *)dev_alloc(c, sizeof(double) * 3 * nf);
        double *fw = (double *)dev_alloc(c, sizeof(double) * 8 * nf);
        double *fwb = (double *)dev_alloc(c, sizeof(double) * nf);
        double *ftmp = (double *)dev_alloc(c, sizeof(double) * 3 * nf);
        int64_t *fs = (int64_t *)dev_alloc(c, sizeof(int64_t) * 8 * nf);
        uint8_t *fk = (uint8_t *)dev_alloc(c, nf);
        if (!fbi || !fub || !fw || !fwb || !ftmp || !fs || !fk) return c->fail(IBM_ERR_OOM, "fresh-cell allocation failed");
        IBM_TRY(geom_fresh_tables(c, nf, fidx, fbi, fk, fs, fw, fwb));
        IBM_TRY(geom_body_velocity(c, nf, fbi, fub));
        const unsigned fb = (unsigned)((nf + 255) / 256);
        ++c->nlaunch, k_fresh_start<<<fb, 256, 0, c->s>>>(nf, fidx, fub, U, nc);
        IBM_LAUNCHED(c);
        // fresh corners are implicit unknowns: Jacobi passes to ghost_tol
        double scale = 1.0;
        for (int a = 0; a < 3; ++a) scale = fmax(scale, fmax(fabs(c->desc.u_inf[a]), fabs(c->motion[a])));
        bool done = false;
        for (int it = 0; it < 4 * c->opts.ghost_maxit && !done; ++it) {
            ++c->nlaunch, k_fresh_compute<<<fb, 256, 0, c->s>>>(nf, fidx, fs, fw, fwb, fub, U, nc, ftmp, c->part);
            ++c->nlaunch, k_fresh_scatter<<<fb, 256, 0, c->s>>>(nf, fidx, U, nc, ftmp);
            IBM_LAUNCHED(c);
            if ((it + 1) % 4 == 0) {
                ++c->nlaunch, k_max_final<<<1, 256, 0, c->s>>>(c->part, (int)fb, c->scal + 40);
                IBM_LAUNCHED(c);
                IBM_TRY(sync_scalars(c, 41));
                const double d = c->hscal[40];
                if (!isfinite(d)) return c->fail(IBM_ERR_DIVERGED, "fresh-cell values are not finite");
                done = d <= c->opts.ghost_tol * scale;
            }
        }
        IBM_CUDA(c, cudaStreamSynchronize(c->s));
        dev_free(c, fbi);
        dev_free(c, fub);
        dev_free(c, fw);
        dev_free(c, fwb);
        dev_free(c, ftmp);
        dev_free(c, fs);
        dev_free(c, fk);
    }
    dev_free(c, fidx);
    ++c->nlaunch, k_dead_zero<<<c->nelem, 256, 0, c->s>>>(c->N, c->type, U, nc);
    IBM_LAUNCHED(c);
    int passes = 0;
    IBM_TRY(ghost_refresh_all(c, c->u, &passes));
    for (int a = 0; a < nc; ++a)
        ++c->nlaunch, k_faces_changed<<<c->nelem, 256, 0, c->s>>>(c->g, c->type, c->type_old, c->u[a], a, c->F[a]);
    IBM_LAUNCHED(c);
    c->fresh_pending = nf > 0;
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    return IBM_OK;
}

// max |div U - mean| over FLUID cells of the current face field
ibm_status div_stat(Ctx *c, double *out) {
    CFields3 F{{c->F[0], c->F[1], c->ndim == 3 ? c->F[2] : c->F[1]}};
    double *d = c->rhs[1];
    ++c->nlaunch, k_divergence<<<c->nelem, 256, 0, c->s>>>(c->g, c->type, F, 1.0, d);
    IBM_LAUNCHED(c);
    IBM_TRY(fluid_mean(c, d, false, nullptr));
    ++c->nlaunch, k_div_stats<<<c->nred, RED_THREADS, 0, c->s>>>(c->g, c->type, d, c->scal + 5, c->part);
    ++c->nlaunch, k_max_final<<<1, 256, 0, c->s>>>(c->part, c->nred, c->scal + 52);
    IBM_LAUNCHED(c);
    IBM_TRY(sync_scalars(c, 53));
    *out = c->hscal[52];
    return IBM_OK;
}

// ---------------------------------------------------------------------------
// Device-controlled step (opts.graph == 2)
//
// The fractional step above, captured into one CUDA graph: the Helmholtz
// sweeps and the velocity ghost refresh become WHILE nodes with the same
// four-sweep trips and the same stopping tests, evaluated by one-thread
// kernels; the Poisson solve is poisson_solve_dev. The host launches the
// graph and reads the accumulated statistics once per ibm_step call.
// ---------------------------------------------------------------------------

struct HelmCtl {
    int sweeps[3];
    int status;   // IBM_ERR_DIVERGED / IBM_ERR_NOT_CONVERGED of the Helmholtz or ghost loops
    double rhs2;
    int passes;
    int next_check;   // sweep count of the next Helmholtz residual test
    int due;          // a test runs after the current sweep
};

__global__ void k_hc_reset(HelmCtl *H, int q, int first_check, cudaGraphConditionalHandle h) {
    if (q == 0) H->status = 0;
    if (q >= 0) {
        H->sweeps[q] = 0;
        H->rhs2 = -1.0;
        H->next_check = first_check;
    } else {
        H->passes = 0;
    }
    cudaGraphSetConditional(h, 1u);
}

// after each sweep: count it and open the residual test when it is due
__global__ void k_helm_tick(HelmCtl *H, int q, int maxit, cudaGraphConditionalHandle hif) {
    const int s = ++H->sweeps[q];
    const bool due = s == H->next_check || s >= maxit;
    if (due) H->next_check = helm_next_check(H->next_check);
    H->due = due;
    cudaGraphSetConditional(hif, due ? 1u : 0u);
}

__global__ void k_helm_decide(HelmCtl *H, int q, const double *__restrict__ scal, int has_ghost, double tol,
                              double scale, int maxit, cudaGraphConditionalHandle h) {
    if (!H->due) {
        cudaGraphSetConditional(h, 1u);
        return;
    }
    const double r2 = scal[48];
    if (H->rhs2 < 0.0) H->rhs2 = scal[49];
    const double gmax = has_ghost ? scal[50] : 0.0;
    if (!isfinite(r2)) {
        H->status = IBM_ERR_DIVERGED;
        cudaGraphSetConditional(h, 0u);
        return;
    }
    const double bn = sqrt(H->rhs2) > 0.0 ? sqrt(H->rhs2) : 1.0;
    const bool conv = sqrt(r2) <= tol * bn && gmax <= tol * scale;
    const bool go = !conv && H->sweeps[q] < maxit;
    if (!conv && !go && H->status == 0) H->status = IBM_ERR_NOT_CONVERGED;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_ghost_decide(HelmCtl *H, const double *__restrict__ d, double tol, int maxit, int trip,
                               cudaGraphConditionalHandle h) {
    H->passes += trip;
    const double v = *d;
    if (!isfinite(v)) {
        H->status = IBM_ERR_DIVERGED;
        cudaGraphSetConditional(h, 0u);
        return;
    }
    cudaGraphSetConditional(h, (v > tol && H->passes < maxit) ? 1u : 0u);
}

static double u_scale(Ctx *c) {
    double scale = 1.0;
    for (int a = 0; a < 3; ++a) scale = fmax(scale, fabs(c->desc.u_inf[a]));
    return scale;
}

static ibm_status helmholtz_dev(Ctx *c, int q) {
    const double alpha = c->desc.dt / (2.0 * c->desc.Re);
    HelmCtl *H = (HelmCtl *)c->hctl;
    const double *hinv = c->hinv[q];
    double *u = c->ustar[q];
    const double *rhs = c->rhs[q];
    const unsigned gb = (unsigned)((c->ng + 255) / 256);
    Fields3 U{{u, u, u}};
    cudaGraphConditionalHandle h, hif;
    IBM_TRY(cond_handle(c, &h));
    IBM_TRY(cond_handle(c, &hif));
    ++c->nlaunch, k_hc_reset<<<1, 1, 0, c->s>>>(H, q, c->opts.helm_check_first, h);
    CondScope sc;
    IBM_TRY(cond_open(c, cudaGraphCondTypeWhile, h, &sc));
    {
        // one sweep per trip; the residual test (an IF node) on the same
        // sweep counts as the host-driven solve
        for (int col = 0; col < 2; ++col) {
            ++c->nlaunch, helm_rb(c, rhs, hinv, u, col);
            helm_ghost_pass(c, q, U, gb);
        }
        ++c->nlaunch, k_helm_tick<<<1, 1, 0, c->s>>>(H, q, c->opts.helm_maxit, hif);
        IBM_LAUNCHED(c);
        CondScope si;
        IBM_TRY(cond_open(c, cudaGraphCondTypeIf, hif, &si));
        ++c->nlaunch, k_helm_resid<<<c->nred, RED_THREADS, 0, c->s>>>(c->g, helm_coef(c), c->type, rhs, make_bc(c), q, u, alpha,
                                                                     c->part);
        IBM_LAUNCHED(c);
        IBM_TRY(finalize(c, c->part, c->nred, 2, 1.0, c->scal + 48));
        if (c->ng > 0) {
            ++c->nlaunch, k_vghost_compute<<<gb, 256, 0, c->s>>>(c->gh, U, 1, ghost_ubi(c), q, c->gtmp, c->part + 2 * RED_BLOCKS_MAX, 1);
            ++c->nlaunch, k_max_final<<<1, 256, 0, c->s>>>(c->part + 2 * RED_BLOCKS_MAX, (int)gb, c->scal + 50);
            IBM_LAUNCHED(c);
        }
        IBM_TRY(cond_close(c, &si));
        ++c->nlaunch, k_helm_decide<<<1, 1, 0, c->s>>>(H, q, c->scal, c->ng > 0, c->opts.helm_rtol, u_scale(c),
                                                     c->opts.helm_maxit, h);
        IBM_LAUNCHED(c);
    }
    IBM_TRY(cond_close(c, &sc));
    return IBM_OK;
}

static ibm_status ghost_refresh_dev(Ctx *c) {
    if (c->ng == 0) return IBM_OK;
    HelmCtl *H = (HelmCtl *)c->hctl;
    const int nc = c->ndim;
    Fields3 U{{c->u[0], c->u[1], nc == 3 ? c->u[2] : c->u[1]}};
    const unsigned gb = (unsigned)((c->ng + 255) / 256);
    const int trip = 4;
    cudaGraphConditionalHandle h;
    IBM_TRY(cond_handle(c, &h));
    ++c->nlaunch, k_hc_reset<<<1, 1, 0, c->s>>>(H, -1, 0, h);
    CondScope sc;
    IBM_TRY(cond_open(c, cudaGraphCondTypeWhile, h, &sc));
    for (int t = 0; t < trip; ++t) {
        ++c->nlaunch, k_vghost_compute<<<gb, 256, 0, c->s>>>(c->gh, U, nc, ghost_ubi(c), 0, c->gtmp, c->part, t == trip - 1);
        ++c->nlaunch, k_vghost_scatter<<<gb, 256, 0, c->s>>>(c->gh, U, nc, c->gtmp);
    }
    ++c->nlaunch, k_max_final<<<1, 256, 0, c->s>>>(c->part, (int)gb, c->scal + 40);
    ++c->nlaunch, k_ghost_decide<<<1, 1, 0, c->s>>>(H, c->scal + 40, c->opts.ghost_tol * u_scale(c),
                                                  c->opts.ghost_maxit, trip, h);
    IBM_LAUNCHED(c);
    IBM_TRY(cond_close(c, &sc));
    return IBM_OK;
}

// the captured body of one step (the first step after a classification
// takes the Euler start, as in flow_step)
static ibm_status flow_step_capture(Ctx *c) {
    const int nc = c->ndim;
    const double dt = c->desc.dt, alpha = dt / (2.0 * c->desc.Re);
    CFields3 u{{c->u[0], c->u[1], nc == 3 ? c->u[2] : c->u[1]}};
    CFields3 F{{c->F[0], c->F[1], nc == 3 ? c->F[2] : c->F[1]}};
    CFields3 No{{c->Nold[0], c->Nold[1], nc == 3 ? c->Nold[2] : c->Nold[1]}};
    Fields3 Nn{{c->Nnew[0], c->Nnew[1], nc == 3 ? c->Nnew[2] : c->Nnew[1]}};
    Fields3 R{{c->rhs[0], c->rhs[1], nc == 3 ? c->rhs[2] : c->rhs[1]}};
    ++c->nlaunch, k_conv_rhs<<<c->nelem, 256, 0, c->s>>>(c->g, c->type, c->dg_c, u, F, No, c->have_nold ? 0 : 1, c->fresh_pending ? c->fresh : nullptr, Nn, R,
                                                       make_bc(c), dt, alpha, nc);
    IBM_LAUNCHED(c);
    for (int q = 0; q < nc; ++q) {
        IBM_CUDA(c, cudaMemcpyAsync(c->ustar[q], c->u[q], sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->s));
        IBM_TRY(helmholtz_dev(c, q));
    }
    IBM_TRY(faces_from(c, c->ustar));
    CFields3 Fs{{c->F[0], c->F[1], nc == 3 ? c->F[2] : c->F[1]}};
    double *braw = c->rhs[0];
    ++c->nlaunch, k_divergence<<<c->nelem, 256, 0, c->s>>>(c->g, c->type, Fs, 1.0 / dt, braw);
    IBM_LAUNCHED(c);
    ++c->nlaunch, k_phi_guess<<<c->nelem, 256, 0, c->s>>>(c->N, c->p, c->p_prev, c->p_prev2, phi_order(c));
    IBM_LAUNCHED(c);
    IBM_TRY(hist_guess(c, braw, c->p));
    IBM_TRY(poisson_solve_dev(c, braw, c->p, c->opts.rtol, c->opts.max_outer));
    IBM_TRY(hist_store(c, c->p));
    for (int a = 0; a < nc; ++a) {
        const int64_t nf = a == 0 ? c->NFx : (a == 1 ? c->NFy : c->NFz);
        const unsigned nb = (unsigned)((nf + 255) / 256 > 152 * 32 ? 152 * 32 : (nf + 255) / 256);
        ++c->nlaunch, k_project_faces<<<nb, 256, 0, c->s>>>(c->g, c->type, c->p, a, dt, c->F[a],
                                                          FastDiv((uint32_t)(c->nx + (a == 0))),
                                                          FastDiv((uint32_t)(c->ny + (a == 1))));
    }
    CFields3 us{{c->ustar[0], c->ustar[1], nc == 3 ? c->ustar[2] : c->ustar[1]}};
    Fields3 un{{c->u[0], c->u[1], nc == 3 ? c->u[2] : c->u[1]}};
    ++c->nlaunch, k_project_cells<<<c->nelem, 256, 0, c->s>>>(c->g, c->type, c->p, us, un, dt);
    IBM_LAUNCHED(c);
    IBM_TRY(ghost_refresh_dev(c));
    IBM_TRY(step_stats_dev(c, ((HelmCtl *)c->hctl)->sweeps));
    return IBM_OK;
}

// whether this step can run as a captured graph
ibm_status step_graph_eligible(Ctx *c) {
    const ibm_solver_opts &o = c->opts;
    if (o.graph != 2 || c->kt.on || c->s == nullptr || c->s == cudaStreamLegacy) return IBM_ERR_STATE;
    if (o.outer != IBM_OUTER_FGMRES || o.inner_iters != 1 || o.helm_solver != 0) return IBM_ERR_STATE;
    // a moving body changes the tables every step: host-driven steps
    if (c->moving) return IBM_ERR_STATE;
    return IBM_OK;
}

static uint64_t graph_key(Ctx *c) {
    // FNV-1a over the options and the multigrid generation
    uint64_t h = 1469598103934665603ull;
    const unsigned char *b = (const unsigned char *)&c->opts;
    for (size_t i = 0; i < sizeof(c->opts); ++i) h = (h ^ b[i]) * 1099511628211ull;
    const unsigned char *g = (const unsigned char *)&c->mg_gen;
    for (size_t i = 0; i < sizeof(c->mg_gen); ++i) h = (h ^ g[i]) * 1099511628211ull;
    h = (h ^ (c->have_nold ? 1u : 2u)) * 1099511628211ull;
    h = (h ^ (uint64_t)(3 + phi_order(c))) * 1099511628211ull;   // order of the Poisson guess
    return h | 1ull;
}

static ibm_status capture_step(Ctx *c, cudaGraphExec_t *out) {
    IBM_TRY(helm_prepare(c));
    IBM_TRY(poisson_dev_prepare(c));
    IBM_TRY(hist_prepare(c));
    if (!c->hctl) {
        c->hctl = dev_alloc(c, sizeof(HelmCtl));
        if (!c->hctl) return c->fail(IBM_ERR_OOM, "control block allocation failed");
        IBM_CUDA(c, cudaMemsetAsync(c->hctl, 0, sizeof(HelmCtl), c->s));
    }
    for (int i = 0; i < 8; ++i)
        if (!c->side[i]) IBM_CUDA(c, cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking));
    cudaStream_t s0 = c->s;
    c->capturing = true;
    c->side_depth = 0;
    IBM_CUDA(c, cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
    ibm_status st = flow_step_capture(c);
    // unwind any body capture left open by an error
    while (c->side_depth > 0) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(c->side[--c->side_depth], &g);
    }
    c->s = s0;
    c->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s0, &g);
    if (st != IBM_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    }
    if (e != cudaSuccess || !g) return c->fail(IBM_ERR_CUDA, std::string("step capture: ") + cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        *out = nullptr;
        return c->fail(IBM_ERR_CUDA, std::string("step graph instantiation: ") + cudaGetErrorString(e2));
    }
    return IBM_OK;
}

// the graph slot for the current settings, start (Euler or AB2) and buffer
// parity; captured if missing
static ibm_status graph_for_state(Ctx *c, int *slot_out) {
    const uint64_t key = graph_key(c);
    int slot = -1;
    for (int i = 0; i < Ctx::NSGRAPH; ++i)
        if (c->sgraph[i] && c->sgraph_key[i] == key && c->sgraph_nold[i] == c->Nold[0]) slot = i;
    if (slot < 0) {
        for (int i = 0; i < Ctx::NSGRAPH && slot < 0; ++i)
            if (!c->sgraph[i]) slot = i;
        if (slot < 0) {
            // all slots hold graphs of other settings: release them
            IBM_CUDA(c, cudaStreamSynchronize(c->s));
            for (int i = 0; i < Ctx::NSGRAPH; ++i) {
                cudaGraphExecDestroy(c->sgraph[i]);
                c->sgraph[i] = nullptr;
            }
            slot = 0;
        }
        IBM_TRY(capture_step(c, &c->sgraph[slot]));
        c->sgraph_key[slot] = key;
        c->sgraph_nold[slot] = c->Nold[0];
    }
    *slot_out = slot;
    return IBM_OK;
}

static void swap_nold(Ctx *c) {
    for (int q = 0; q < 3; ++q) {
        double *t = c->Nold[q];
        c->Nold[q] = c->Nnew[q];
        c->Nnew[q] = t;
    }
}

// one step through the captured graph of the current state
ibm_status flow_step_graph(Ctx *c) {
    int slot = 0;
    IBM_TRY(graph_for_state(c, &slot));
    IBM_CUDA(c, cudaGraphLaunch(c->sgraph[slot], c->s));
    swap_nold(c);
    c->have_nold = true;
    c->nstep += 1;
    return IBM_OK;
}

// capture the graphs of the next step and of both buffer parities of the
// steps after it, without running anything
ibm_status flow_graph_prepare(Ctx *c) {
    // the next six steps' states (start, buffer parity, order of the
    // Poisson guess) cover every state of the steps after them
    const bool h0 = c->have_nold;
    const int64_t n0 = c->nstep;
    int slot = 0;
    ibm_status st = IBM_OK;
    int swaps = 0;
    for (int k = 0; k < 6 && st == IBM_OK; ++k) {
        st = graph_for_state(c, &slot);
        swap_nold(c);
        ++swaps;
        c->have_nold = true;
        c->nstep += 1;
    }
    if (swaps % 2) swap_nold(c);
    c->have_nold = h0;
    c->nstep = n0;
    return st;
}

}  // namespace ibm
