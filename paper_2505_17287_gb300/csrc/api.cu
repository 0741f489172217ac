// C ABI of libibm.so (declared in include/ibm.h): context lifetime, argument
// validation, host<->device copies and the call order of the solver phases.
#include "ctx.cuh"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <utility>
#include <vector>

using namespace ibm;

struct ibm_ctx : public Ctx {};

static thread_local std::string g_create_error;

namespace ibm {

void *dev_alloc(Ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (c->desc.alloc) {
        p = c->desc.alloc(bytes, c->desc.alloc_ctx);
        if (p && ((uintptr_t)p & 15u)) {
            // the vector kernels load and store 16 bytes at a time
            if (c->desc.free) c->desc.free(p, c->desc.alloc_ctx);
            p = nullptr;
        }
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocs.push_back(p);
    return p;
}

void dev_free(Ctx *c, void *p) {
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it == c->allocs.end()) return;
    c->allocs.erase(it);
    if (c->desc.free) c->desc.free(p, c->desc.alloc_ctx);
    else cudaFree(p);
}

void kt_begin(Ctx *c, int id) {
    if (!c->kt.on) return;
    if (id < 0) id = K_OTHER;
    if (c->kt.used + 2 > (int)c->kt.pool.size()) kt_flush(c);
    cudaEventRecord(c->kt.pool[c->kt.used], c->s);
    c->kt.ids[c->kt.used / 2] = id;
}

void kt_end(Ctx *c, int id) {
    (void)id;
    if (!c->kt.on) return;
    cudaEventRecord(c->kt.pool[c->kt.used + 1], c->s);
    c->kt.used += 2;
}

ibm_status kt_flush(Ctx *c) {
    if (c->kt.used == 0) return IBM_OK;
    IBM_CUDA(c, cudaEventSynchronize(c->kt.pool[c->kt.used - 1]));
    for (int q = 0; q < c->kt.used; q += 2) {
        float ms = 0.f;
        IBM_CUDA(c, cudaEventElapsedTime(&ms, c->kt.pool[q], c->kt.pool[q + 1]));
        const int id = c->kt.ids[q / 2];
        c->kt.ms[id] += ms;
        c->kt.n[id] += 1;
    }
    c->kt.used = 0;
    return IBM_OK;
}

}  // namespace ibm

static void release_all(Ctx *c) {
    if (c->s) cudaStreamSynchronize(c->s);
    for (int i = 0; i < MGHier<double>::NVG; ++i) {
        if (c->mg64.vgraph[i]) cudaGraphExecDestroy(c->mg64.vgraph[i]);
        if (c->mg32.vgraph[i]) cudaGraphExecDestroy(c->mg32.vgraph[i]);
    }
    for (int i = 0; i < Ctx::NSGRAPH; ++i)
        if (c->sgraph[i]) cudaGraphExecDestroy(c->sgraph[i]);
    for (int i = 0; i < 8; ++i)
        if (c->side[i]) cudaStreamDestroy(c->side[i]);
    std::vector<void *> a = c->allocs;
    for (void *p : a) dev_free(c, p);
    if (c->hscal) cudaFreeHost(c->hscal);
    cudaEvent_t ev[6] = {c->ev0, c->ev1, c->ev2, c->ev3, c->ev4, c->ev5};
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    for (auto e : c->kt.pool) cudaEventDestroy(e);
}

extern "C" ibm_status ibm_default_opts(ibm_solver_opts *o) {
    if (!o) return IBM_ERR_ARG;
    o->rtol = 1e-10;
    o->max_outer = 400;
    o->restart = 16;
    o->inner_iters = 1;
    o->nu1 = 2;
    o->nu2 = 1;
    o->coarse_sweeps = 32;
    o->helm_rtol = 1e-12;
    o->helm_maxit = 500;
    o->ghost_tol = 1e-15;
    o->ghost_maxit = 100;
    o->precision = IBM_FP64;
    o->outer = IBM_OUTER_FGMRES;
    o->band_sweeps = 8;
    o->band_omega = 0.85;
    o->mixed_inner_rtol = 1e-4;
    o->mg_interp = 1;
    o->tile_x = 128;
    o->graph = 1;
    o->precond = 0;
    o->srj_sweeps = 16;
    o->srj_lmin = 0.0;
    o->helm_solver = 0;
    o->smooth_omega = 1.0;
    o->reorth_eta = 0.3;
    o->helm_check_first = 6;
    o->helm_omega = 1.0;
    o->fine_split = 1;
    o->band_width = 3;
    o->poisson_hist = 8;
    o->tail_cells = 0;
    o->nu_coarse = 3;
    return IBM_OK;
}

static bool opts_ok(const ibm_solver_opts *o, std::string &why) {
    if (!(o->rtol > 0.0 && o->rtol < 1.0)) { why = "rtol must be in (0, 1)"; return false; }
    if (o->max_outer < 1) { why = "max_outer must be >= 1"; return false; }
    if (o->restart < 1 || o->restart > 16) { why = "restart must be in [1, 16]"; return false; }
    if (o->inner_iters < 1 || o->inner_iters > 64) { why = "inner_iters must be in [1, 64]"; return false; }
    if (o->nu1 < 1 || o->nu2 < 1 || o->nu1 > 8 || o->nu2 > 8) { why = "nu1, nu2 must be in [1, 8]"; return false; }
    // the inner MG-PCG (inner_iters > 1) needs a symmetric V-cycle; FGMRES and
    // BiCGStab accept any preconditioner
    if (o->inner_iters > 1 && o->nu1 != o->nu2) { why = "nu1 = nu2 is required when inner_iters > 1 (CG needs a symmetric V-cycle)"; return false; }
    if (o->coarse_sweeps < 1) { why = "coarse_sweeps must be >= 1"; return false; }
    if (!(o->helm_rtol > 0.0) || o->helm_maxit < 1) { why = "bad Helmholtz tolerance or limit"; return false; }
    if (!(o->ghost_tol > 0.0) || o->ghost_maxit < 1) { why = "bad ghost refresh tolerance or limit"; return false; }
    if (o->precision != IBM_FP64 && o->precision != IBM_MIXED) { why = "precision must be IBM_FP64 or IBM_MIXED"; return false; }
    if (o->outer != IBM_OUTER_BICGSTAB && o->outer != IBM_OUTER_FGMRES) { why = "unknown outer method"; return false; }
    if (o->band_sweeps < 0 || o->band_sweeps > 64) { why = "band_sweeps must be in [0, 64]"; return false; }
    if (!(o->band_omega > 0.0 && o->band_omega <= 1.0)) { why = "band_omega must be in (0, 1]"; return false; }
    if (!(o->mixed_inner_rtol > 0.0 && o->mixed_inner_rtol < 1.0)) { why = "mixed_inner_rtol must be in (0, 1)"; return false; }
    if (o->mg_interp != 0 && o->mg_interp != 1) { why = "mg_interp must be 0 or 1"; return false; }
    if (o->tile_x != 32 && o->tile_x != 64 && o->tile_x != 128 && o->tile_x != 256 && o->tile_x != 512) {
        why = "tile_x must be 32, 64, 128, 256 or 512";
        return false;
    }
    if (o->graph < 0 || o->graph > 2) { why = "graph must be 0, 1 or 2"; return false; }
    if (o->precond != 0 && o->precond != 1) { why = "precond must be 0 (multigrid) or 1 (SRJ)"; return false; }
    if (o->srj_sweeps < 1 || o->srj_sweeps > 64) { why = "srj_sweeps must be in [1, 64]"; return false; }
    if (!(o->srj_lmin >= 0.0 && o->srj_lmin < 2.0)) { why = "srj_lmin must be in [0, 2)"; return false; }
    if (o->helm_solver != 0 && o->helm_solver != 1) { why = "helm_solver must be 0 or 1"; return false; }
    if (!(o->reorth_eta >= 0.0 && o->reorth_eta <= 1.0)) { why = "reorth_eta must be in [0, 1]"; return false; }
    if (o->helm_check_first < 1) { why = "helm_check_first must be >= 1"; return false; }
    if (!(o->helm_omega == 0.0 || (o->helm_omega > 0.0 && o->helm_omega < 2.0))) {
        why = "helm_omega must be 0 (automatic) or in (0, 2)";
        return false;
    }
    if (!(o->smooth_omega > 0.0 && o->smooth_omega < 2.0)) { why = "smooth_omega must be in (0, 2)"; return false; }
    if (o->fine_split != 0 && o->fine_split != 1) { why = "fine_split must be 0 or 1"; return false; }
    if (o->band_width < 1 || o->band_width > 4) { why = "band_width must be in [1, 4]"; return false; }
    if (o->tail_cells < 0) { why = "tail_cells must be >= 0"; return false; }
    if (o->poisson_hist < 0 || o->poisson_hist > 16) { why = "poisson_hist must be in [0, 16]"; return false; }
    if (o->nu_coarse < 0 || o->nu_coarse > 8) { why = "nu_coarse must be in [0, 8]"; return false; }
    if (o->inner_iters > 1 && o->smooth_omega != 1.0) { why = "smooth_omega must be 1 when inner_iters > 1"; return false; }
    return true;
}

namespace ibm {
// FP64 Krylov storage, allocated on first use by an FP64 outer iteration:
// FGMRES(m) needs m+1 basis and m preconditioned vectors; BiCGStab uses six
// of the first and two of the second. Mixed precision never allocates it.
ibm_status alloc_krylov(Ctx *c, int m) {
    if (m <= c->m_cap) return IBM_OK;
    for (double *p : c->V) dev_free(c, p);
    for (double *p : c->Z) dev_free(c, p);
    const int nv = m + 1 > 6 ? m + 1 : 6, nz = m > 2 ? m : 2;
    c->V.assign(nv, nullptr);
    c->Z.assign(nz, nullptr);
    for (int i = 0; i < nv; ++i)
        if (!(c->V[i] = (double *)dev_alloc(c, sizeof(double) * c->N))) return c->fail(IBM_ERR_OOM, "Krylov vector allocation failed");
    for (int i = 0; i < nz; ++i)
        if (!(c->Z[i] = (double *)dev_alloc(c, sizeof(double) * c->N))) return c->fail(IBM_ERR_OOM, "Krylov vector allocation failed");
    if (!c->Vdev) c->Vdev = (double **)dev_alloc(c, sizeof(double *) * 17);
    if (!c->Zdev) c->Zdev = (double **)dev_alloc(c, sizeof(double *) * 17);
    if (!c->Vdev || !c->Zdev) return c->fail(IBM_ERR_OOM, "pointer table allocation failed");
    IBM_CUDA(c, cudaMemcpyAsync(c->Vdev, c->V.data(), sizeof(double *) * (m + 1), cudaMemcpyHostToDevice, c->s));
    IBM_CUDA(c, cudaMemcpyAsync(c->Zdev, c->Z.data(), sizeof(double *) * nz, cudaMemcpyHostToDevice, c->s));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    c->m_cap = m;
    return IBM_OK;
}
}  // namespace ibm

static double *upload(Ctx *c, const std::vector<double> &h) {
    double *d = (double *)dev_alloc(c, sizeof(double) * (h.size() ? h.size() : 1));
    if (d && h.size()) cudaMemcpyAsync(d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, c->s);
    return d;
}

static void axis_arrays(const std::vector<double> &f, std::vector<double> &cc, std::vector<double> &w,
                        std::vector<double> &h) {
    const size_t n = f.size() - 1;
    cc.resize(n);
    w.resize(n);
    h.assign(n + 1, 0.0);
    for (size_t i = 0; i < n; ++i) {
        cc[i] = 0.5 * (f[i] + f[i + 1]);
        w[i] = f[i + 1] - f[i];
    }
    for (size_t i = 1; i < n; ++i) h[i] = cc[i] - cc[i - 1];
}

static ibm_status build_levels(Ctx *c) {
    c->lg.clear();
    LevelGeom L0{c->nx, c->ny, c->nz, 1, 1, 1, c->hxf, c->hyf, c->hzf};
    c->lg.push_back(L0);
    while ((int)c->lg.size() < 24) {
        const LevelGeom &L = c->lg.back();
        const int64_t n = (int64_t)L.nx * L.ny * L.nz;
        if (n <= 512 || (L.nx <= 2 && L.ny <= 2 && L.nz <= 2)) break;
        LevelGeom C;
        C.fx = L.nx > 2 ? 2 : 1;
        C.fy = L.ny > 2 ? 2 : 1;
        C.fz = L.nz > 2 ? 2 : 1;
        C.nx = (L.nx + C.fx - 1) / C.fx;
        C.ny = (L.ny + C.fy - 1) / C.fy;
        C.nz = (L.nz + C.fz - 1) / C.fz;
        auto coarsen = [](const std::vector<double> &f, int nfine, int fac, int ncoarse) {
            if (fac == 1) return f;
            std::vector<double> o(ncoarse + 1);
            for (int k = 0; k < ncoarse; ++k) o[k] = f[2 * k];
            o[ncoarse] = f[nfine];
            return o;
        };
        C.xf = coarsen(L.xf, L.nx, C.fx, C.nx);
        C.yf = coarsen(L.yf, L.ny, C.fy, C.ny);
        C.zf = coarsen(L.zf, L.nz, C.fz, C.nz);
        c->lg.push_back(C);
    }
    {
        const LevelGeom &L = c->lg.back();
        if ((int64_t)L.nx * L.ny * L.nz > 512) return c->fail(IBM_ERR_ARG, "grid too anisotropic to coarsen to 512 cells");
    }
    for (auto &L : c->lg) {
        std::vector<double> cc, w, h;
        axis_arrays(L.xf, cc, w, h);
        c->lhx.push_back(upload(c, h));
        axis_arrays(L.yf, cc, w, h);
        c->lhy.push_back(upload(c, h));
        axis_arrays(L.zf, cc, w, h);
        c->lhz.push_back(upload(c, h));
        if (!c->lhx.back() || !c->lhy.back() || !c->lhz.back()) return c->fail(IBM_ERR_OOM, "level geometry allocation failed");
    }
    // trilinear transfer tables: linear interpolation between the two coarse
    // centres around each fine centre (the nearer-side neighbour of its
    // parent), the parent alone at the ends and along uncoarsened axes
    for (int a = 0; a < 3; ++a) {
        c->tI[a].assign(c->lg.size(), nullptr);
        c->tJ[a].assign(c->lg.size(), nullptr);
        c->tw64[a].assign(c->lg.size(), nullptr);
        c->tw32[a].assign(c->lg.size(), nullptr);
        c->tv64[a].assign(c->lg.size(), nullptr);
        c->tv32[a].assign(c->lg.size(), nullptr);
        c->gI[a].assign(c->lg.size(), nullptr);
        c->gw64[a].assign(c->lg.size(), nullptr);
        c->gw32[a].assign(c->lg.size(), nullptr);
    }
    for (size_t l = 1; l < c->lg.size(); ++l) {
        const LevelGeom &F = c->lg[l - 1], &C = c->lg[l];
        const std::vector<double> *ff[3] = {&F.xf, &F.yf, &F.zf}, *cf[3] = {&C.xf, &C.yf, &C.zf};
        const int fac[3] = {C.fx, C.fy, C.fz};
        for (int a = 0; a < 3; ++a) {
            const std::vector<double> &fa = *ff[a], &ca = *cf[a];
            const int nf = (int)fa.size() - 1, nc = (int)ca.size() - 1;
            std::vector<int> I(nf), J(nf);
            std::vector<double> w(nf), w32d(nf);
            std::vector<float> w32(nf);
            for (int i = 0; i < nf; ++i) {
                const double xi = 0.5 * (fa[i] + fa[i + 1]);
                if (fac[a] == 1) { I[i] = i; J[i] = -1; w[i] = 1.0; }
                else {
                    int pI = i / 2 < nc - 1 ? i / 2 : nc - 1;
                    const double XI = 0.5 * (ca[pI] + ca[pI + 1]);
                    int pJ = xi < XI ? pI - 1 : pI + 1;
                    if (xi == XI || pJ < 0 || pJ >= nc) { I[i] = pI; J[i] = -1; w[i] = 1.0; }
                    else {
                        const double XJ = 0.5 * (ca[pJ] + ca[pJ + 1]);
                        I[i] = pI; J[i] = pJ; w[i] = (xi - XJ) / (XI - XJ);
                    }
                }
                w32[i] = (float)w[i];
            }
            int *dI = (int *)dev_alloc(c, sizeof(int) * nf), *dJ = (int *)dev_alloc(c, sizeof(int) * nf);
            double *dw = (double *)dev_alloc(c, sizeof(double) * nf);
            float *dw32 = (float *)dev_alloc(c, sizeof(float) * nf);
            if (!dI || !dJ || !dw || !dw32) return c->fail(IBM_ERR_OOM, "transfer table allocation failed");
            IBM_CUDA(c, cudaMemcpy(dI, I.data(), sizeof(int) * nf, cudaMemcpyHostToDevice));
            IBM_CUDA(c, cudaMemcpy(dJ, J.data(), sizeof(int) * nf, cudaMemcpyHostToDevice));
            IBM_CUDA(c, cudaMemcpy(dw, w.data(), sizeof(double) * nf, cudaMemcpyHostToDevice));
            IBM_CUDA(c, cudaMemcpy(dw32, w32.data(), sizeof(float) * nf, cudaMemcpyHostToDevice));
            c->tI[a][l] = dI;
            c->tJ[a][l] = dJ;
            c->tw64[a][l] = dw;
            c->tw32[a][l] = dw32;
            {
                std::vector<double> v(nf);
                std::vector<float> v32(nf);
                for (int i = 0; i < nf; ++i) {
                    v[i] = 1.0 - w[i];
                    v32[i] = 1.0f - w32[i];
                }
                double *dv = (double *)dev_alloc(c, sizeof(double) * nf);
                float *dv32 = (float *)dev_alloc(c, sizeof(float) * nf);
                if (!dv || !dv32) return c->fail(IBM_ERR_OOM, "transfer table allocation failed");
                IBM_CUDA(c, cudaMemcpy(dv, v.data(), sizeof(double) * nf, cudaMemcpyHostToDevice));
                IBM_CUDA(c, cudaMemcpy(dv32, v32.data(), sizeof(float) * nf, cudaMemcpyHostToDevice));
                c->tv64[a][l] = dv;
                c->tv32[a][l] = dv32;
            }
            // transpose: the weight of fine i in coarse I[i] is w, in J[i] it
            // is 1 - w, rounded in each precision as the prolongation rounds it
            std::vector<int> gi((size_t)4 * nc, -1);
            std::vector<double> gw((size_t)4 * nc, 0.0);
            std::vector<float> gw32((size_t)4 * nc, 0.0f);
            std::vector<int> fill(nc, 0);
            for (int i = 0; i < nf; ++i) {
                const int targets[2] = {I[i], J[i]};
                for (int t = 0; t < 2; ++t) {
                    const int C2 = targets[t];
                    if (C2 < 0) continue;
                    if (fill[C2] >= 4) return c->fail(IBM_ERR_ARG, "transfer table: more than four fine cells per coarse cell");
                    const size_t q = (size_t)4 * C2 + fill[C2]++;
                    gi[q] = i;
                    gw[q] = t == 0 ? w[i] : 1.0 - w[i];
                    gw32[q] = t == 0 ? w32[i] : 1.0f - w32[i];
                }
            }
            int *dgi = (int *)dev_alloc(c, sizeof(int) * 4 * nc);
            double *dgw = (double *)dev_alloc(c, sizeof(double) * 4 * nc);
            float *dgw32 = (float *)dev_alloc(c, sizeof(float) * 4 * nc);
            if (!dgi || !dgw || !dgw32) return c->fail(IBM_ERR_OOM, "transfer table allocation failed");
            IBM_CUDA(c, cudaMemcpy(dgi, gi.data(), sizeof(int) * 4 * nc, cudaMemcpyHostToDevice));
            IBM_CUDA(c, cudaMemcpy(dgw, gw.data(), sizeof(double) * 4 * nc, cudaMemcpyHostToDevice));
            IBM_CUDA(c, cudaMemcpy(dgw32, gw32.data(), sizeof(float) * 4 * nc, cudaMemcpyHostToDevice));
            c->gI[a][l] = dgi;
            c->gw64[a][l] = dgw;
            c->gw32[a][l] = dgw32;
        }
    }
    return IBM_OK;
}

// per-cell volume and FP64 operator diagonal, in the operation order the
// operator used when it computed them per call: (dx dy) dz, (cxs + cys) + czs
__global__ void k_cell_metrics(GridDev g, double *__restrict__ vol, double *__restrict__ dg) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.n; c += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        split3(g, (uint32_t)c, i, j, k);
        vol[c] = g.dx[i] * g.dy[j] * g.dz[k];
        double s = g.cxs[i] + g.cys[j];
        if (g.ndim == 3) s += g.czs[k];
        dg[c] = s;
    }
}

static ibm_status create_impl(Ctx *c, const ibm_grid_desc *d) {
    c->desc = *d;
    c->desc.xf = c->desc.yf = c->desc.zf = nullptr;
    c->s = (cudaStream_t)d->stream;
    ibm_default_opts(&c->opts);
    c->opts.precision = d->precision;
    c->ndim = d->ndim;
    c->nx = d->nx;
    c->ny = d->ny;
    c->nz = d->ndim == 2 ? 1 : d->nz;
    c->N = (int64_t)c->nx * c->ny * c->nz;
    c->NFx = (int64_t)(c->nx + 1) * c->ny * c->nz;
    c->NFy = (int64_t)c->nx * (c->ny + 1) * c->nz;
    c->NFz = (int64_t)c->nx * c->ny * (c->nz + 1);
    {
        const int64_t r = (c->N + 8 * RED_THREADS - 1) / (8 * RED_THREADS);
        c->nred = (int)(r < 1 ? 1 : (r > RED_BLOCKS ? RED_BLOCKS : r));
        const int64_t w = (c->N + 2 * RED_THREADS - 1) / (2 * RED_THREADS);
        c->nred_wide = (int)(w < 1 ? 1 : (w > RED_BLOCKS_MAX ? RED_BLOCKS_MAX : w));
        const int64_t e = (c->N + 255) / 256;
        c->nelem = (unsigned)(e < 1 ? 1 : (e > 152 * 16 ? 152 * 16 : e));
    }
    c->hxf.assign(d->xf, d->xf + c->nx + 1);
    c->hyf.assign(d->yf, d->yf + c->ny + 1);
    if (c->ndim == 3) c->hzf.assign(d->zf, d->zf + c->nz + 1);
    else c->hzf = {0.0, 1.0};
    axis_arrays(c->hxf, c->hxc, c->hdx, c->hhx);
    axis_arrays(c->hyf, c->hyc, c->hdy, c->hhy);
    axis_arrays(c->hzf, c->hzc, c->hdz, c->hhz);
    IBM_CUDA(c, cudaEventCreate(&c->ev0));
    IBM_CUDA(c, cudaEventCreate(&c->ev1));
    IBM_CUDA(c, cudaEventCreate(&c->ev2));
    IBM_CUDA(c, cudaEventCreate(&c->ev3));
    IBM_CUDA(c, cudaEventCreate(&c->ev4));
    IBM_CUDA(c, cudaEventCreate(&c->ev5));
    IBM_CUDA(c, cudaMallocHost((void **)&c->hscal, sizeof(double) * 64));
    c->xf = upload(c, c->hxf); c->yf = upload(c, c->hyf); c->zf = upload(c, c->hzf);
    c->xc = upload(c, c->hxc); c->yc = upload(c, c->hyc); c->zc = upload(c, c->hzc);
    c->dx = upload(c, c->hdx); c->dy = upload(c, c->hdy); c->dz = upload(c, c->hdz);
    c->hx = upload(c, c->hhx); c->hy = upload(c, c->hhy); c->hz = upload(c, c->hhz);
    if (!c->xf || !c->yf || !c->zf || !c->xc || !c->yc || !c->zc || !c->dx || !c->dy || !c->dz || !c->hx || !c->hy || !c->hz)
        return c->fail(IBM_ERR_OOM, "grid allocation failed");
    // per-axis coefficients of the full pressure operator divided by the volume
    auto coef = [&](const std::vector<double> &h, const std::vector<double> &w, double **m, double **p, double **sm) {
        const size_t n = w.size();
        std::vector<double> a(n, 0.0), b(n, 0.0), s(n, 0.0);
        for (size_t i = 0; i < n; ++i) {
            if (i > 0) a[i] = 1.0 / (h[i] * w[i]);
            if (i + 1 < n) b[i] = 1.0 / (h[i + 1] * w[i]);
            s[i] = a[i] + b[i];
        }
        *m = upload(c, a);
        *p = upload(c, b);
        *sm = upload(c, s);
    };
    double *cxm, *cxp, *cxs, *cym, *cyp, *cys, *czm, *czp, *czs;
    coef(c->hhx, c->hdx, &cxm, &cxp, &cxs);
    coef(c->hhy, c->hdy, &cym, &cyp, &cys);
    coef(c->hhz, c->hdz, &czm, &czp, &czs);
    if (!cxm || !cxp || !cxs || !cym || !cyp || !cys || !czm || !czp || !czs)
        return c->fail(IBM_ERR_OOM, "grid allocation failed");
    auto recip = [](const std::vector<double> &w) {
        std::vector<double> r(w.size());
        for (size_t i = 0; i < w.size(); ++i) r[i] = 1.0 / w[i];
        return r;
    };
    double *rdx = upload(c, recip(c->hdx)), *rdy = upload(c, recip(c->hdy)), *rdz = upload(c, recip(c->hdz));
    if (!rdx || !rdy || !rdz) return c->fail(IBM_ERR_OOM, "grid allocation failed");
    // 1 / centre spacing; entry 0 (no spacing below the first centre) is 0
    auto recip_h = [](const std::vector<double> &h) {
        std::vector<double> r(h.size(), 0.0);
        for (size_t i = 1; i < h.size(); ++i) r[i] = 1.0 / h[i];
        return r;
    };
    double *rhx = upload(c, recip_h(c->hhx)), *rhy = upload(c, recip_h(c->hhy)), *rhz = upload(c, recip_h(c->hhz));
    if (!rhx || !rhy || !rhz) return c->fail(IBM_ERR_OOM, "grid allocation failed");
    c->g = GridDev{c->nx, c->ny, c->nz, c->ndim, c->N, c->xf, c->yf, c->zf, c->xc, c->yc, c->zc,
                   c->dx, c->dy, c->dz, c->hx, c->hy, c->hz, cxm, cxp, cxs, cym, cyp, cys, czm, czp, czs,
                   FastDiv((uint32_t)c->nx), FastDiv((uint32_t)c->ny), rdx, rdy, rdz, rhx, rhy, rhz};
    const size_t nb = sizeof(double) * c->N;
    c->vol_c = (double *)dev_alloc(c, nb);
    c->dg_c = (double *)dev_alloc(c, nb);
    if (!c->vol_c || !c->dg_c) return c->fail(IBM_ERR_OOM, "cell metric allocation failed");
    ++c->nlaunch;
    k_cell_metrics<<<c->nelem, 256, 0, c->s>>>(c->g, c->vol_c, c->dg_c);
    IBM_LAUNCHED(c);
    c->type = (uint8_t *)dev_alloc(c, c->N);
    c->inside = (uint8_t *)dev_alloc(c, c->N);
    if (!c->type || !c->inside) return c->fail(IBM_ERR_OOM, "cell arrays allocation failed");
    const int64_t nf[3] = {c->NFx, c->NFy, c->NFz};
    for (int q = 0; q < 3; ++q) {
        const bool used = q < c->ndim;
        const size_t cb = used ? nb : 8;
        c->u[q] = (double *)dev_alloc(c, cb);
        c->Nold[q] = (double *)dev_alloc(c, cb);
        c->Nnew[q] = (double *)dev_alloc(c, cb);
        c->ustar[q] = (double *)dev_alloc(c, cb);
        c->rhs[q] = (double *)dev_alloc(c, q < 2 ? nb : cb);
        c->F[q] = (double *)dev_alloc(c, used ? sizeof(double) * nf[q] : 8);
        if (!c->u[q] || !c->Nold[q] || !c->Nnew[q] || !c->ustar[q] || !c->rhs[q] || !c->F[q])
            return c->fail(IBM_ERR_OOM, "flow field allocation failed");
    }
    c->p = (double *)dev_alloc(c, nb);
    c->p_prev = (double *)dev_alloc(c, nb);
    c->p_prev2 = (double *)dev_alloc(c, nb);
    c->b = (double *)dev_alloc(c, nb);
    c->w = (double *)dev_alloc(c, nb);
    c->rr = (double *)dev_alloc(c, nb);
    c->part = (double *)dev_alloc(c, sizeof(double) * RED_BLOCKS_MAX * 40);
    c->scal = (double *)dev_alloc(c, sizeof(double) * 64);
    if (!c->p || !c->p_prev || !c->p_prev2 || !c->b || !c->w || !c->rr || !c->part || !c->scal)
        return c->fail(IBM_ERR_OOM, "solver vector allocation failed");
    IBM_CUDA(c, cudaMemsetAsync(c->p, 0, nb, c->s));
    IBM_CUDA(c, cudaMemsetAsync(c->p_prev, 0, nb, c->s));
    IBM_CUDA(c, cudaMemsetAsync(c->p_prev2, 0, nb, c->s));
    IBM_CUDA(c, cudaMemsetAsync(c->scal, 0, sizeof(double) * 64, c->s));
    IBM_TRY(build_levels(c));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    return IBM_OK;
}

static bool increasing(const double *f, int n) {
    for (int i = 0; i < n; ++i)
        if (!(f[i + 1] > f[i]) || !isfinite(f[i]) || !isfinite(f[i + 1])) return false;
    return true;
}

extern "C" ibm_status ibm_create_grid(const ibm_grid_desc *d, ibm_ctx **out) {
    if (!out) { g_create_error = "out is NULL"; return IBM_ERR_ARG; }
    *out = nullptr;
    if (!d) { g_create_error = "descriptor is NULL"; return IBM_ERR_ARG; }
    if (d->ndim != 2 && d->ndim != 3) { g_create_error = "ndim must be 2 or 3"; return IBM_ERR_ARG; }
    if (d->nx < 2 || d->ny < 2 || (d->ndim == 3 && d->nz < 2) || (d->ndim == 2 && d->nz != 1)) {
        g_create_error = "cell counts must be >= 2 (nz = 1 in 2D)";
        return IBM_ERR_ARG;
    }
    if (!d->xf || !d->yf || (d->ndim == 3 && !d->zf)) { g_create_error = "face coordinates are NULL"; return IBM_ERR_ARG; }
    if (!increasing(d->xf, d->nx) || !increasing(d->yf, d->ny) || (d->ndim == 3 && !increasing(d->zf, d->nz))) {
        g_create_error = "face coordinates must be finite and strictly increasing";
        return IBM_ERR_ARG;
    }
    if (!(d->Re > 0.0) || !(d->dt > 0.0)) { g_create_error = "Re and dt must be positive"; return IBM_ERR_ARG; }
    for (int f = 0; f < 6; ++f)
        if (d->bc[f] < IBM_BC_INFLOW || d->bc[f] > IBM_BC_SLIP) { g_create_error = "unknown boundary code"; return IBM_ERR_ARG; }
    if (d->precision != IBM_FP64 && d->precision != IBM_MIXED) { g_create_error = "bad precision"; return IBM_ERR_ARG; }
    if ((d->alloc == nullptr) != (d->free == nullptr)) { g_create_error = "alloc and free hooks must be given together"; return IBM_ERR_ARG; }
    const double ncell = (double)d->nx * d->ny * (d->ndim == 3 ? d->nz : 1);
    if (ncell >= 4294967296.0) { g_create_error = "grid too large (at most 2^32 - 1 cells)"; return IBM_ERR_ARG; }
    {
        // face arrays are indexed with 32-bit multiply-shift division too
        const double nz = d->ndim == 3 ? d->nz : 1;
        double nf = fmax((d->nx + 1.0) * d->ny * nz, d->nx * (d->ny + 1.0) * nz);
        if (d->ndim == 3) nf = fmax(nf, (double)d->nx * d->ny * (nz + 1.0));
        if (nf >= 4294967296.0) { g_create_error = "grid too large (at most 2^32 - 1 faces per axis)"; return IBM_ERR_ARG; }
    }
    ibm_ctx *c = new (std::nothrow) ibm_ctx();
    if (!c) { g_create_error = "host allocation failed"; return IBM_ERR_OOM; }
    ibm_status s = create_impl(c, d);
    if (s != IBM_OK) {
        g_create_error = c->err.msg;
        release_all(c);
        delete c;
        return s;
    }
    *out = c;
    return IBM_OK;
}

extern "C" ibm_status ibm_set_opts(ibm_ctx *c, const ibm_solver_opts *o) {
    if (!c || !o) return IBM_ERR_ARG;
    std::string why;
    if (!opts_ok(o, why)) return c->fail(IBM_ERR_ARG, why);
    c->opts = *o;

    return IBM_OK;
}

// closed, consistently oriented surface: every directed edge (3D) appears
// once and its reverse once; in 2D every vertex starts one and ends one segment
static bool mesh_closed(int ndim, const double *v, int64_t nv, const int32_t *e, int64_t ne, std::string &why) {
    for (int64_t q = 0; q < nv * 3; ++q)
        if (!isfinite(v[q])) { why = "non-finite vertex coordinate"; return false; }
    const int k = ndim == 3 ? 3 : 2;
    for (int64_t q = 0; q < ne * k; ++q)
        if (e[q] < 0 || e[q] >= nv) { why = "element index out of range"; return false; }
    if (ndim == 2) {
        std::vector<int> outd(nv, 0), ind(nv, 0);
        for (int64_t q = 0; q < ne; ++q) {
            if (e[2 * q] == e[2 * q + 1]) { why = "degenerate segment"; return false; }
            outd[e[2 * q]]++;
            ind[e[2 * q + 1]]++;
        }
        for (int64_t q = 0; q < nv; ++q)
            if (outd[q] != ind[q] || outd[q] > 1) { why = "polyline is not closed and simple"; return false; }
        return true;
    }
    std::vector<std::pair<int64_t, int64_t>> ed;
    ed.reserve((size_t)ne * 3);
    for (int64_t q = 0; q < ne; ++q)
        for (int r = 0; r < 3; ++r) {
            const int64_t a = e[3 * q + r], b = e[3 * q + (r + 1) % 3];
            if (a == b) { why = "degenerate triangle"; return false; }
            ed.emplace_back(a, b);
        }
    std::sort(ed.begin(), ed.end());
    for (size_t q = 1; q < ed.size(); ++q)
        if (ed[q] == ed[q - 1]) { why = "an edge is used twice in the same direction"; return false; }
    for (auto &x : ed)
        if (!std::binary_search(ed.begin(), ed.end(), std::make_pair(x.second, x.first))) {
            why = "surface is not closed (an edge has no opposite edge)";
            return false;
        }
    return true;
}

extern "C" ibm_status ibm_set_body(ibm_ctx *c, const double *verts, int64_t nv, const int32_t *elems, int64_t ne) {
    if (!c) return IBM_ERR_ARG;
    if (!verts || !elems || nv < 3 || ne < (c->ndim == 3 ? 4 : 3)) return c->fail(IBM_ERR_ARG, "empty or NULL mesh");
    std::string why;
    if (!mesh_closed(c->ndim, verts, nv, elems, ne, why)) return c->fail(IBM_ERR_MESH, why);
    const int k = c->ndim == 3 ? 3 : 2;
    const int64_t base = c->nv;
    if (base + nv > INT32_MAX) return c->fail(IBM_ERR_ARG, "too many vertices");
    c->verts.insert(c->verts.end(), verts, verts + nv * 3);
    for (int64_t q = 0; q < ne * k; ++q) c->elems.push_back((int32_t)(elems[q] + base));
    c->nv += nv;
    c->ne += ne;
    dev_free(c, c->d_verts);
    dev_free(c, c->d_elems);
    c->d_verts = (double *)dev_alloc(c, sizeof(double) * c->verts.size());
    c->d_elems = (int32_t *)dev_alloc(c, sizeof(int32_t) * c->elems.size());
    if (!c->d_verts || !c->d_elems) return c->fail(IBM_ERR_OOM, "mesh allocation failed");
    IBM_CUDA(c, cudaMemcpyAsync(c->d_verts, c->verts.data(), sizeof(double) * c->verts.size(), cudaMemcpyHostToDevice, c->s));
    IBM_CUDA(c, cudaMemcpyAsync(c->d_elems, c->elems.data(), sizeof(int32_t) * c->elems.size(), cudaMemcpyHostToDevice, c->s));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    c->classified = false;
    return IBM_OK;
}

// classification, ghost tables, FLUID volume and multigrid operators of the
// current body position
static ibm_status geometry_update(ibm_ctx *c) {
    IBM_TRY(geom_classify(c));
    c->wp32_n = -1;  // FP32 copies of the ghost weights are stale
    c->hinv_ok = false;
    if (c->n_fluid == 0) return c->fail(IBM_ERR_ARG, "no fluid cells");
    // FLUID volume
    double vol = 0.0;
    {
        const double saved = c->fluid_vol;
        c->fluid_vol = 1.0;
        ibm_status s = fluid_mean(c, nullptr, false, &vol);
        c->fluid_vol = saved;
        IBM_TRY(s);
    }
    c->fluid_vol = vol;
    return mg_build(c);
}

extern "C" ibm_status ibm_classify_cells(ibm_ctx *c, ibm_table_info *out) {
    if (!c) return IBM_ERR_ARG;
    if (c->ne == 0) return c->fail(IBM_ERR_STATE, "ibm_set_body must be called before ibm_classify_cells");
    c->moving = false;
    c->fresh_pending = false;
    IBM_TRY(geometry_update(c));
    IBM_TRY(flow_init(c));
    c->classified = true;
    if (out) {
        out->n_fluid = c->n_fluid;
        out->n_ghost = c->ng;
        out->n_dead = c->n_dead;
        for (int q = 0; q < 3; ++q) out->n_kind[q] = c->n_kind[q];
    }
    return IBM_OK;
}

extern "C" ibm_status ibm_move_body(ibm_ctx *c, const double *verts, int64_t nv, const double *motion,
                                    ibm_table_info *out) {
    if (!c) return IBM_ERR_ARG;
    if (!verts || !motion) return c->fail(IBM_ERR_ARG, "verts and motion must not be NULL");
    if (!c->classified) return c->fail(IBM_ERR_STATE, "ibm_classify_cells must be called before ibm_move_body");
    if (nv != c->nv) return c->fail(IBM_ERR_ARG, "ibm_move_body needs the vertex count of the bodies set");
    for (int64_t q = 0; q < 3 * nv; ++q)
        if (!isfinite(verts[q])) return c->fail(IBM_ERR_ARG, "vertex coordinates must be finite");
    for (int q = 0; q < 9; ++q)
        if (!isfinite(motion[q])) return c->fail(IBM_ERR_ARG, "motion must be finite");
    if (c->ndim == 2) {
        for (int64_t q = 0; q < nv; ++q)
            if (verts[3 * q + 2] != 0.0) return c->fail(IBM_ERR_ARG, "2D vertices must have z = 0");
        if (motion[2] != 0.0 || motion[3] != 0.0 || motion[4] != 0.0)
            return c->fail(IBM_ERR_ARG, "2D motion: U_z, Omega_x and Omega_y must be 0");
    }
    if (!c->type_old) c->type_old = (uint8_t *)dev_alloc(c, (size_t)c->N);
    if (!c->fresh) {
        c->fresh = (uint8_t *)dev_alloc(c, (size_t)c->N);
        if (c->fresh) IBM_CUDA(c, cudaMemsetAsync(c->fresh, 0, (size_t)c->N, c->s));
    }
    if (!c->type_old || !c->fresh) return c->fail(IBM_ERR_OOM, "moving-body allocation failed");
    if (c->fresh_pending) {
        // flags of a move with no step after it: those cells are FLUID
        // already, so they are not fresh at this move
        IBM_CUDA(c, cudaMemsetAsync(c->fresh, 0, (size_t)c->N, c->s));
        c->fresh_pending = false;
    }
    std::copy(verts, verts + 3 * nv, c->verts.begin());
    IBM_CUDA(c, cudaMemcpyAsync(c->d_verts, c->verts.data(), sizeof(double) * c->verts.size(), cudaMemcpyHostToDevice,
                                c->s));
    IBM_CUDA(c, cudaMemcpyAsync(c->type_old, c->type, (size_t)c->N, cudaMemcpyDeviceToDevice, c->s));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    IBM_TRY(geometry_update(c));
    for (int q = 0; q < 9; ++q) c->motion[q] = motion[q];
    c->moving = true;
    IBM_TRY(flow_move(c));
    if (out) {
        out->n_fluid = c->n_fluid;
        out->n_ghost = c->ng;
        out->n_dead = c->n_dead;
        for (int q = 0; q < 3; ++q) out->n_kind[q] = c->n_kind[q];
    }
    return IBM_OK;
}

// enqueue nsteps steps; host-driven steps complete here, captured ones are
// only launched (their statistics are collected by step_collect)
static ibm_status step_enqueue(ibm_ctx *c, int nsteps) {
    for (int q = 0; q < nsteps; ++q) {
        if (step_graph_eligible(c) == IBM_OK) {
            if (c->pend_graph == 0) IBM_CUDA(c, cudaEventRecord(c->ev2, c->s));
            IBM_TRY(flow_step_graph(c));
            ++c->pend_graph;
            continue;
        }
        ibm_status s = flow_step(c, &c->pend);
        if (s == IBM_ERR_NOT_CONVERGED) c->pend_status = s;
        else if (s != IBM_OK) return s;
    }
    return IBM_OK;
}

static ibm_status step_collect(ibm_ctx *c, ibm_step_stats *out) {
    ibm_status status = c->pend_status;
    ibm_status hard = IBM_OK;
    if (c->pend_graph > 0) {
        IBM_CUDA(c, cudaEventRecord(c->ev3, c->s));
        const ibm_status s = step_stats_read(c, &c->pend);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev2, c->ev3);
        c->pend.ms_total += ms;
        c->pend_graph = 0;
        if (s == IBM_ERR_NOT_CONVERGED) status = s;
        else if (s != IBM_OK) hard = s;
    }
    if (hard == IBM_OK && c->pend.steps > 0) hard = div_stat(c, &c->pend.max_div);
    if (out) *out = c->pend;
    c->pend = ibm_step_stats{};
    c->pend_status = IBM_OK;
    return hard != IBM_OK ? hard : status;
}

extern "C" ibm_status ibm_step(ibm_ctx *c, int nsteps, ibm_step_stats *out) {
    if (!c) return IBM_ERR_ARG;
    if (nsteps < 0) return c->fail(IBM_ERR_ARG, "nsteps must be >= 0");
    if (!c->classified) return c->fail(IBM_ERR_STATE, "ibm_classify_cells must be called before ibm_step");
    const ibm_status s = step_enqueue(c, nsteps);
    const ibm_status r = step_collect(c, out);
    return s != IBM_OK ? s : r;
}

extern "C" ibm_status ibm_step_async(ibm_ctx *c, int nsteps) {
    if (!c) return IBM_ERR_ARG;
    if (nsteps < 0) return c->fail(IBM_ERR_ARG, "nsteps must be >= 0");
    if (!c->classified) return c->fail(IBM_ERR_STATE, "ibm_classify_cells must be called before ibm_step_async");
    return step_enqueue(c, nsteps);
}

extern "C" ibm_status ibm_step_prepare(ibm_ctx *c) {
    if (!c) return IBM_ERR_ARG;
    if (!c->classified) return c->fail(IBM_ERR_STATE, "ibm_classify_cells must be called before ibm_step_prepare");
    if (step_graph_eligible(c) != IBM_OK) return IBM_OK;
    return flow_graph_prepare(c);
}

extern "C" ibm_status ibm_step_wait(ibm_ctx *c, ibm_step_stats *out) {
    if (!c) return IBM_ERR_ARG;
    return step_collect(c, out);
}

extern "C" ibm_status ibm_poisson_solve(ibm_ctx *c, const double *rhs, double *phi, double rtol, int maxit,
                                        ibm_solve_stats *st) {
    if (!c) return IBM_ERR_ARG;
    if (!rhs || !phi) return c->fail(IBM_ERR_ARG, "rhs and phi must be device pointers");
    if (!c->classified) return c->fail(IBM_ERR_STATE, "ibm_classify_cells must be called before ibm_poisson_solve");
    const char *a0 = (const char *)rhs, *b0 = (const char *)phi;
    const size_t nb = sizeof(double) * c->N;
    if (a0 < b0 + nb && b0 < a0 + nb) return c->fail(IBM_ERR_ARG, "rhs and phi overlap");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, rhs) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
        cudaPointerGetAttributes(&at, phi) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return c->fail(IBM_ERR_ARG, "rhs and phi must be device memory");
    }
    return poisson_solve(c, rhs, phi, rtol > 0 ? rtol : c->opts.rtol, maxit > 0 ? maxit : c->opts.max_outer, st);
}

extern "C" ibm_status ibm_get_tables(ibm_ctx *c, const ibm_tables_host *t) {
    if (!c || !t) return IBM_ERR_ARG;
    if (!c->classified) return c->fail(IBM_ERR_STATE, "no tables before ibm_classify_cells");
    const int64_t g = c->ng;
    auto cp = [&](void *dst, const void *src, size_t bytes) -> ibm_status {
        if (!dst || bytes == 0) return IBM_OK;
        IBM_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->s));
        return IBM_OK;
    };
    IBM_TRY(cp(t->type, c->type, c->N));
    IBM_TRY(cp(t->gidx, c->gidx, 8 * g));
    IBM_TRY(cp(t->bi, c->bi, 24 * g));
    IBM_TRY(cp(t->nrm, c->nrm, 24 * g));
    IBM_TRY(cp(t->ip, c->ipt, 24 * g));
    IBM_TRY(cp(t->dist, c->dist, 8 * g));
    IBM_TRY(cp(t->base, c->base, 8 * g));
    IBM_TRY(cp(t->kind, c->kind, g));
    IBM_TRY(cp(t->cmask, c->cmask, g));
    IBM_TRY(cp(t->sidx, c->sidx, 64 * g));
    IBM_TRY(cp(t->wv, c->wv, 64 * g));
    IBM_TRY(cp(t->wp, c->wp, 64 * g));
    IBM_TRY(cp(t->bv, c->bv, 8 * g));
    IBM_TRY(cp(t->bp, c->bp, 8 * g));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    return IBM_OK;
}

static ibm_status field_ptr(Ctx *c, int field, void **p, size_t *bytes) {
    const size_t nb = sizeof(double) * c->N;
    const int nd = c->ndim;
    switch (field) {
    case IBM_FIELD_U: case IBM_FIELD_V: case IBM_FIELD_W:
        if (field - IBM_FIELD_U >= nd) return c->fail(IBM_ERR_ARG, "no w component in 2D");
        *p = c->u[field - IBM_FIELD_U]; *bytes = nb; return IBM_OK;
    case IBM_FIELD_P: *p = c->p; *bytes = nb; return IBM_OK;
    case IBM_FIELD_FACE_U: *p = c->F[0]; *bytes = sizeof(double) * c->NFx; return IBM_OK;
    case IBM_FIELD_FACE_V: *p = c->F[1]; *bytes = sizeof(double) * c->NFy; return IBM_OK;
    case IBM_FIELD_FACE_W:
        if (nd < 3) return c->fail(IBM_ERR_ARG, "no z faces in 2D");
        *p = c->F[2]; *bytes = sizeof(double) * c->NFz; return IBM_OK;
    case IBM_FIELD_NOLD_U: case IBM_FIELD_NOLD_V: case IBM_FIELD_NOLD_W:
        if (field - IBM_FIELD_NOLD_U >= nd) return c->fail(IBM_ERR_ARG, "no w component in 2D");
        *p = c->Nold[field - IBM_FIELD_NOLD_U]; *bytes = nb; return IBM_OK;
    case IBM_FIELD_TYPE: *p = c->type; *bytes = c->N; return IBM_OK;
    case IBM_FIELD_USTAR_U: case IBM_FIELD_USTAR_V: case IBM_FIELD_USTAR_W:
        if (field - IBM_FIELD_USTAR_U >= nd) return c->fail(IBM_ERR_ARG, "no w component in 2D");
        *p = c->ustar[field - IBM_FIELD_USTAR_U]; *bytes = nb; return IBM_OK;
    case IBM_FIELD_RHS: *p = c->b; *bytes = nb; return IBM_OK;
    case IBM_FIELD_P_PREV: *p = c->p_prev; *bytes = nb; return IBM_OK;
    case IBM_FIELD_P_PREV2: *p = c->p_prev2; *bytes = nb; return IBM_OK;
    default: return c->fail(IBM_ERR_ARG, "unknown field id");
    }
}

// Host <-> device copy of a field. A pinned host buffer is visible to the GPU
// (GB300 reaches host memory over NVLink-C2C), so a kernel on every SM pulls
// or pushes it, faster than one copy engine; pageable memory goes through
// cudaMemcpyAsync. Both are ordered on the context stream.
__global__ void k_copy_bytes(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst, size_t nb) {
    const size_t n16 = (((uintptr_t)src | (uintptr_t)dst) & 15) == 0 ? nb / 16 : 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    size_t q = t0;
    for (; q + 3 * stride < n16; q += 4 * stride) {
        const uint4 a = s4[q], b = s4[q + stride], c = s4[q + 2 * stride], d = s4[q + 3 * stride];
        d4[q] = a;
        d4[q + stride] = b;
        d4[q + 2 * stride] = c;
        d4[q + 3 * stride] = d;
    }
    for (; q < n16; q += stride) d4[q] = s4[q];
    for (size_t b = n16 * 16 + t0; b < nb; b += stride) dst[b] = src[b];
}

static ibm_status host_copy(Ctx *c, void *dst, const void *src, size_t nb, bool to_device) {
    const void *host = to_device ? src : dst;
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, host);
    if (e == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer) {
        const uint8_t *s8 = (const uint8_t *)(to_device ? a.devicePointer : src);
        uint8_t *d8 = (uint8_t *)(to_device ? dst : a.devicePointer);
        ++c->nlaunch;
        k_copy_bytes<<<152 * 8, 256, 0, c->s>>>(s8, d8, nb);
        IBM_LAUNCHED(c);
    } else {
        cudaGetLastError();
        IBM_CUDA(c, cudaMemcpyAsync(dst, src, nb, to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, c->s));
    }
    return IBM_OK;
}

// the guess history's stored vectors, slot-major without the slots'
// padding (each slot is N doubles in the caller's buffer)
static ibm_status hist_vec_io(Ctx *c, int field, void *buf, int is_device, size_t bytes, bool to_ctx) {
    const int L = c->opts.poisson_hist;
    if (L <= 0) return c->fail(IBM_ERR_ARG, "the Poisson guess history is off (poisson_hist 0)");
    const size_t nb = sizeof(double) * (size_t)c->N;
    if (bytes != nb * (size_t)L) return c->fail(IBM_ERR_ARG, "byte count does not match the field size");
    IBM_TRY(hist_prepare(c));
    double *base = field == IBM_FIELD_P_HIST_X ? c->hist_x : c->hist_b;
    for (int i = 0; i < L; ++i) {
        double *slot = base + (size_t)i * (size_t)c->hist_ld;
        uint8_t *user = (uint8_t *)buf + (size_t)i * nb;
        if (is_device) {
            IBM_CUDA(c, cudaMemcpyAsync(to_ctx ? (void *)slot : (void *)user, to_ctx ? (const void *)user : (const void *)slot,
                                        nb, cudaMemcpyDeviceToDevice, c->s));
        } else if (to_ctx) {
            IBM_TRY(host_copy(c, slot, user, nb, true));
        } else {
            IBM_TRY(host_copy(c, user, slot, nb, false));
        }
    }
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    return IBM_OK;
}

// the guess history's control values as doubles: pairs held, next slot,
// the Gram matrix (poisson_hist^2, row-major)
static ibm_status hist_ctl_io(Ctx *c, void *buf, int is_device, size_t bytes, bool to_ctx) {
    const int L = c->opts.poisson_hist;
    if (L <= 0) return c->fail(IBM_ERR_ARG, "the Poisson guess history is off (poisson_hist 0)");
    if (bytes != sizeof(double) * (size_t)(2 + L * L)) return c->fail(IBM_ERR_ARG, "byte count does not match the field size");
    IBM_TRY(hist_prepare(c));
    HistCtl h{};
    IBM_CUDA(c, cudaMemcpyAsync(&h, c->hist_ctl, sizeof(HistCtl), cudaMemcpyDeviceToHost, c->s));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    std::vector<double> v((size_t)(2 + L * L));
    if (to_ctx) {
        if (is_device) IBM_CUDA(c, cudaMemcpy(v.data(), buf, bytes, cudaMemcpyDeviceToHost));
        else memcpy(v.data(), buf, bytes);
        if (!(v[0] >= 0 && v[0] <= L && v[1] >= 0 && v[1] < L && v[0] == (int)v[0] && v[1] == (int)v[1]))
            return c->fail(IBM_ERR_ARG, "history control values out of range");
        h.count = (int)v[0];
        h.slot = (int)v[1];
        for (int i = 0; i < L; ++i)
            for (int j = 0; j < L; ++j) h.G[i * HIST_MAX + j] = v[2 + (size_t)i * L + j];
        IBM_CUDA(c, cudaMemcpyAsync(c->hist_ctl, &h, sizeof(HistCtl), cudaMemcpyHostToDevice, c->s));
        IBM_CUDA(c, cudaStreamSynchronize(c->s));
    } else {
        v[0] = h.count;
        v[1] = h.slot;
        for (int i = 0; i < L; ++i)
            for (int j = 0; j < L; ++j) v[2 + (size_t)i * L + j] = h.G[i * HIST_MAX + j];
        if (is_device) IBM_CUDA(c, cudaMemcpy(buf, v.data(), bytes, cudaMemcpyHostToDevice));
        else memcpy(buf, v.data(), bytes);
    }
    return IBM_OK;
}

extern "C" ibm_status ibm_get_field(ibm_ctx *c, int field, void *dst, int is_device, size_t bytes) {
    if (!c || !dst) return IBM_ERR_ARG;
    if (field == IBM_FIELD_P_HIST_CTL) return hist_ctl_io(c, dst, is_device, bytes, false);
    if (field == IBM_FIELD_P_HIST_X || field == IBM_FIELD_P_HIST_B) return hist_vec_io(c, field, dst, is_device, bytes, false);
    if (field == IBM_FIELD_STEP) {
        if (bytes != sizeof(int64_t)) return c->fail(IBM_ERR_ARG, "step counter is one int64");
        int64_t v = c->nstep + (c->have_nold ? 0 : 0);
        if (is_device) IBM_CUDA(c, cudaMemcpy(dst, &v, 8, cudaMemcpyHostToDevice));
        else memcpy(dst, &v, 8);
        return IBM_OK;
    }
    void *p = nullptr;
    size_t nb = 0;
    IBM_TRY(field_ptr(c, field, &p, &nb));
    if (bytes != nb) return c->fail(IBM_ERR_ARG, "byte count does not match the field size");
    if (is_device) IBM_CUDA(c, cudaMemcpyAsync(dst, p, nb, cudaMemcpyDeviceToDevice, c->s));
    else IBM_TRY(host_copy(c, dst, p, nb, false));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    return IBM_OK;
}

extern "C" ibm_status ibm_set_field(ibm_ctx *c, int field, const void *src, int is_device, size_t bytes) {
    if (!c || !src) return IBM_ERR_ARG;
    if (field == IBM_FIELD_P_HIST_CTL) return hist_ctl_io(c, const_cast<void *>(src), is_device, bytes, true);
    if (field == IBM_FIELD_P_HIST_X || field == IBM_FIELD_P_HIST_B)
        return hist_vec_io(c, field, const_cast<void *>(src), is_device, bytes, true);
    if (field == IBM_FIELD_STEP) {
        if (bytes != sizeof(int64_t)) return c->fail(IBM_ERR_ARG, "step counter is one int64");
        int64_t v = 0;
        if (is_device) IBM_CUDA(c, cudaMemcpy(&v, src, 8, cudaMemcpyDeviceToHost));
        else memcpy(&v, src, 8);
        if (v < 0) return c->fail(IBM_ERR_ARG, "negative step counter");
        c->nstep = v;
        c->have_nold = v > 0;
        return IBM_OK;
    }
    if (field == IBM_FIELD_TYPE) return c->fail(IBM_ERR_ARG, "cell types are set by ibm_classify_cells");
    void *p = nullptr;
    size_t nb = 0;
    IBM_TRY(field_ptr(c, field, &p, &nb));
    if (bytes != nb) return c->fail(IBM_ERR_ARG, "byte count does not match the field size");
    if (is_device) IBM_CUDA(c, cudaMemcpyAsync(p, src, nb, cudaMemcpyDeviceToDevice, c->s));
    else IBM_TRY(host_copy(c, p, src, nb, true));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    return IBM_OK;
}

extern "C" ibm_status ibm_sizes(ibm_ctx *c, int64_t *n_cells, int64_t *n_ghost) {
    if (!c) return IBM_ERR_ARG;
    if (n_cells) *n_cells = c->N;
    if (n_ghost) *n_ghost = c->ng;
    return IBM_OK;
}

extern "C" ibm_status ibm_kernel_timer(ibm_ctx *c, int enable) {
    if (!c) return IBM_ERR_ARG;
    IBM_TRY(kt_flush(c));
    if (enable && c->kt.pool.empty()) {
        c->kt.pool.resize(4096);
        c->kt.ids.resize(2048);
        for (auto &e : c->kt.pool) IBM_CUDA(c, cudaEventCreate(&e));
    }
    c->kt.on = enable != 0;
    for (int q = 0; q < K_NKERNELS; ++q) { c->kt.ms[q] = 0.0; c->kt.n[q] = 0; }
    return IBM_OK;
}

extern "C" ibm_status ibm_kernel_time(ibm_ctx *c, int kernel, double *ms_total, int64_t *launches) {
    if (!c || !ms_total || !launches || kernel < 0 || kernel >= K_NKERNELS) return IBM_ERR_ARG;
    IBM_TRY(kt_flush(c));
    *ms_total = c->kt.ms[kernel];
    *launches = c->kt.n[kernel];
    return IBM_OK;
}

extern "C" ibm_status ibm_launch_count(ibm_ctx *c, int64_t *count) {
    if (!c || !count) return IBM_ERR_ARG;
    *count = c->nlaunch;
    return IBM_OK;
}

extern "C" ibm_status ibm_destroy(ibm_ctx *c) {
    if (!c) return IBM_OK;
    release_all(c);
    delete c;
    return IBM_OK;
}

extern "C" const char *ibm_last_error(ibm_ctx *c) {
    if (!c) return g_create_error.c_str();
    return c->err.msg.c_str();
}
