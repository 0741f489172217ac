// Context of one grid: every device allocation of the library hangs here.
#pragma once

#include "common.cuh"

namespace ibm {

// device control block of the Poisson guess history (solver.cu): pairs in
// the ring, next slot, Gram matrix of the stored right-hand sides, this
// step's dots and coefficients, and the FLUID mean of its right-hand side
constexpr int HIST_MAX = 16;
struct HistCtl {
    int count, slot;
    double G[HIST_MAX * HIST_MAX];
    double d[HIST_MAX + 1];
    double c[HIST_MAX];
    double mean;
};

template <typename T>
struct MGHier {
    std::vector<MGLevel<T>> lv;
    bool fine0 = false;     // level 0 derives its coefficients (no arrays)
    uint8_t *omask = nullptr;  // open-face mask of level 0 (fine variant)
    // 1D metrics of level 0 in precision T (fine variant)
    T *wx = nullptr, *wy = nullptr, *wz = nullptr, *rhx = nullptr, *rhy = nullptr, *rhz = nullptr;
    // PCG vectors on level 0
    T *px = nullptr, *pr = nullptr, *pz = nullptr, *pp = nullptr, *pq = nullptr;
    // level 0 in colour-split storage (fine variant, nx a multiple of 8):
    // the cells of colour q ((i + j + k) & 1 == q) of each row packed in i
    // order at h = i >> 1, row stride nx / 2; xs and fs are the V-cycle's
    // level-0 x and f during a cycle, ms the open-face mask. The per-row
    // metrics of the packed cells: swx[pc][h] = wx[2h + pc], srm[pc][h] =
    // rhx[2h + pc], srp[pc][h] = rhx[2h + pc + 1] (pc the row's offset of the
    // colour, (q + j + k) & 1)
    bool split = false;
    T *xs[2] = {nullptr, nullptr}, *fs[2] = {nullptr, nullptr};
    uint8_t *ms[2] = {nullptr, nullptr};
    T *swx[2] = {nullptr, nullptr}, *srm[2] = {nullptr, nullptr}, *srp[2] = {nullptr, nullptr};
    // per fine level: residual scratch (level >= 1) and 1 / sum of the active
    // coarse interpolation weights of each cell (trilinear transfer)
    std::vector<T *> res, pn;
    // per-level table of the persistent V-cycle tail (TailLv<T>[levels],
    // device memory), null below three levels
    void *tail = nullptr;
    bool built = false;
    // the V-cycle z = M^{-1} r (pr -> an output buffer) captured as CUDA
    // graphs, one per output buffer (pz, or a Krylov vector written in
    // place), with the settings they were captured for and the kernel count
    static constexpr int NVG = 18;
    cudaGraphExec_t vgraph[NVG] = {};
    const void *vgraph_out[NVG] = {};
    uint64_t vgraph_key = 0;
    int64_t vgraph_kernels = 0;
};

// 1D coordinates of one multigrid level (host) and the axis coarsening flags
struct LevelGeom {
    int nx, ny, nz;
    int fx, fy, fz;   // coarsening factor from the level above (1 or 2)
    std::vector<double> xf, yf, zf;
};

// kernel ids of the diagnostic event timer
enum KernelId {
    K_RBGS0 = 0,      // red-black Gauss-Seidel colour pass, finest level
    K_SPMV0 = 1,      // staircase operator product + dot, finest level
    K_APPLY_A = 2,    // full ghost-cell pressure operator
    K_MDOT = 3,       // FGMRES multi-dot
    K_ORTH = 4,       // FGMRES orthogonalisation update
    K_HELM = 5,       // Crank-Nicolson Helmholtz colour pass
    K_CONV = 6,       // convective term + AB2/CN right-hand side
    K_RBGS_C = 7,     // red-black colour pass, coarse levels
    K_RESTRICT = 8,   // residual + restriction
    K_PROLONG = 9,    // prolongation + correction
    K_OTHER = 10,     // every other kernel of the Poisson solver
    K_TAIL = 11,      // persistent V-cycle tail (the coarse levels in one launch)
    K_NKERNELS = 12
};

// Records a CUDA event pair around every launch of the timed kernels on the
// context stream; the pairs are read back at the next flush.
struct KTimer {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<int> ids;
    int used = 0;
    double ms[K_NKERNELS] = {0};
    int64_t n[K_NKERNELS] = {0};
};

struct Ctx {
    Err err;
    KTimer kt;
    ibm_grid_desc desc{};
    ibm_solver_opts opts{};
    cudaStream_t s = nullptr;
    std::vector<void *> allocs;

    // grid
    int ndim = 0, nx = 0, ny = 0, nz = 0;
    int64_t N = 0, NFx = 0, NFy = 0, NFz = 0;  // cells and faces per axis
    std::vector<double> hxf, hyf, hzf, hxc, hyc, hzc, hdx, hdy, hdz, hhx, hhy, hhz;
    double *xf = nullptr, *yf = nullptr, *zf = nullptr, *xc = nullptr, *yc = nullptr, *zc = nullptr;
    double *dx = nullptr, *dy = nullptr, *dz = nullptr, *hx = nullptr, *hy = nullptr, *hz = nullptr;
    GridDev g{};

    // immersed bodies (host accumulation of all set_body calls)
    std::vector<double> verts;
    std::vector<int32_t> elems;
    int64_t nv = 0, ne = 0;
    bool classified = false;
    double *d_verts = nullptr;
    int32_t *d_elems = nullptr;
    int64_t *d_vq = nullptr;

    // cells and ghost tables
    uint8_t *type = nullptr, *inside = nullptr;
    double fluid_vol = 0.0;
    int64_t n_fluid = 0, n_dead = 0, ng = 0, n_kind[3] = {0, 0, 0};
    int64_t *gidx = nullptr, *base = nullptr, *sidx = nullptr;
    double *bi = nullptr, *nrm = nullptr, *ipt = nullptr, *dist = nullptr;
    double *wv = nullptr, *wp = nullptr, *bv = nullptr, *bp = nullptr;
    uint8_t *kind = nullptr, *cmask = nullptr;
    int64_t ng_cap = 0;
    GhostDev gh{};

    // flow state
    double *u[3] = {nullptr, nullptr, nullptr}, *F[3] = {nullptr, nullptr, nullptr};
    double *p_prev = nullptr, *p_prev2 = nullptr;   // pressures of the two steps before (Poisson guess)
    double *p = nullptr, *Nold[3] = {nullptr, nullptr, nullptr}, *Nnew[3] = {nullptr, nullptr, nullptr};
    double *ustar[3] = {nullptr, nullptr, nullptr}, *rhs[3] = {nullptr, nullptr, nullptr};
    double *b = nullptr, *gtmp = nullptr;
    double *hinv[3] = {nullptr, nullptr, nullptr};   // Helmholtz inverse diagonals per component
    bool hinv_ok = false;
    double *hac = nullptr;   // alpha-scaled viscous face coefficients: x-, x+ (nx each), y-, y+, z-, z+
    // per-cell FP64 volume (dx dy dz) and operator diagonal (cxs + cys + czs),
    // stored so the FP64 operator spends no FP64 instructions rebuilding them
    double *vol_c = nullptr, *dg_c = nullptr;
    double *htmp = nullptr;   // second buffer of the Jacobi (SRJ) Helmholtz sweeps
    int64_t nstep = 0;
    bool have_nold = false;
    // moving body (ibm_move_body): rigid motion (U, Omega, centre), the body
    // velocity at every ghost's intercept (3 per ghost), the cell types
    // before the last move and the per-cell flags of the fresh cells it
    // made, which the next step's convective term reads (Euler start there)
    bool moving = false;
    double motion[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double *ubi = nullptr;
    int64_t ubi_cap = 0;
    uint8_t *type_old = nullptr, *fresh = nullptr;
    bool fresh_pending = false;
    int64_t n_fresh = 0;

    // reductions and scalars
    double *part = nullptr;      // partials: RED_BLOCKS * 32
    double *scal = nullptr;      // device scalars (64)
    double *hscal = nullptr;     // pinned host mirror (64)

    // Poisson (FP64 FGMRES)
    int m_cap = 0;
    std::vector<double *> V, Z;
    double **Vdev = nullptr, **Zdev = nullptr;   // device arrays of the V / Z pointers
    double *w = nullptr, *rr = nullptr;
    // FP32 storage of mixed mode
    float *op32[12] = {nullptr};         // cxm..czs, dx, dy, dz in FP32
    float *wp32 = nullptr;
    int64_t wp32_n = -1;
    std::vector<float *> V32, Z32;
    float **Vdev32 = nullptr, **Zdev32 = nullptr;
    float *w32 = nullptr, *r32 = nullptr, *d32 = nullptr, *b32 = nullptr;
    int m32_cap = 0;
    // Poisson guess history: hist_cap pairs of N doubles (solutions, projected
    // right-hand sides), this step's projected right-hand side, HistCtl
    int hist_cap = 0, hist_len = 0;   // allocated pairs; pair count of the history held
    int64_t hist_ld = 0;              // slot stride (N rounded up to 32 doubles)
    double *hist_x = nullptr, *hist_b = nullptr, *hist_bp = nullptr;
    void *hist_ctl = nullptr;
    // near-body band for the preconditioner's local relaxation
    int64_t nband = 0;
    int64_t *band = nullptr;      // cell index
    int64_t *band_g = nullptr;    // position in gidx, -1 for FLUID cells
    double *btmp = nullptr;
    std::vector<LevelGeom> lg;
    std::vector<double *> lhx, lhy, lhz;   // per level centre spacing (device)
    // trilinear transfer from level l-1 to level l, per axis (entry 0 unused):
    // fine index i interpolates coarse tI[i] with weight tw[i] and coarse
    // tJ[i] (-1: none) with 1 - tw[i]
    std::vector<int *> tI[3], tJ[3];
    std::vector<double *> tw64[3], tv64[3];   // tv = 1 - tw, rounded as the kernels did
    std::vector<float *> tw32[3], tv32[3];
    // the transpose, for restriction: coarse index I gathers from up to four
    // fine indices gI[4I+s] (-1: none) with weights gw[4I+s]
    std::vector<int *> gI[3];
    std::vector<double *> gw64[3];
    std::vector<float *> gw32[3];
    MGHier<double> mg64;
    MGHier<float> mg32;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
    cudaEvent_t ev4 = nullptr, ev5 = nullptr;   // Poisson solve timing

    // device-controlled step (opts.graph == 2): the whole fractional step is
    // captured once per buffer parity into a CUDA graph whose loops are
    // conditional nodes; dctl holds the solver control blocks, dstats the
    // statistics accumulated by the graphs
    bool capturing = false;
    cudaStream_t side[8] = {nullptr};
    int side_depth = 0;
    void *dctl = nullptr;
    void *dstats = nullptr;
    void *hctl = nullptr;   // Helmholtz / ghost refresh control of the captured step
    // steps enqueued by ibm_step_async and not yet collected by ibm_step_wait
    ibm_step_stats pend{};
    int pend_graph = 0;
    ibm_status pend_status = IBM_OK;
    static constexpr int NSGRAPH = 6;   // first four steps, then two buffer parities
    cudaGraphExec_t sgraph[NSGRAPH] = {nullptr};
    uint64_t sgraph_key[NSGRAPH] = {0};
    const double *sgraph_nold[NSGRAPH] = {nullptr};
    int64_t nlaunch = 0;   // kernels launched by this context so far
    // launch sizes that follow the grid: reduction kernels run nred blocks of
    // RED_THREADS (about 8 cells per thread, at most RED_BLOCKS; a function
    // of N only, so reductions stay deterministic); the FP32 operator product
    // and the Krylov/preconditioner vector kernels nred_wide (about 2 cells
    // per thread, at most RED_BLOCKS_MAX: a thread walking tens of cells is
    // latency-bound); the flow kernels nelem blocks of 256
    int nred = RED_BLOCKS;
    int nred_wide = RED_BLOCKS;
    unsigned nelem = 152 * 16;
    uint64_t mg_gen = 0;   // multigrid rebuild counter (invalidates captured V-cycles)

    ibm_status fail(ibm_status code, const std::string &m) {
        err.code = code;
        err.msg = m;
        return code;
    }
};

// FP64 Krylov storage on first use (api.cu)
ibm_status alloc_krylov(Ctx *c, int m);

// event timer (api.cu)
void kt_begin(Ctx *c, int id);
void kt_end(Ctx *c, int id);
ibm_status kt_flush(Ctx *c);

// solver.cu
ibm_status mg_build(Ctx *c);
// Poisson guess history (solver.cu): storage, reset, the projection guess
// for a right-hand side (after the extrapolated guess is in phi), and the
// pair of a finished solve
ibm_status hist_prepare(Ctx *c);
ibm_status hist_reset(Ctx *c);
ibm_status hist_guess(Ctx *c, const double *rhs, double *phi);
ibm_status hist_store(Ctx *c, const double *phi);
ibm_status poisson_solve(Ctx *c, const double *rhs, double *phi, double rtol, int maxit,
                         ibm_solve_stats *st);
ibm_status fluid_mean(Ctx *c, const double *x, bool ghosts_too, double *mean_host);
ibm_status sync_scalars(Ctx *c, int n);
ibm_status finalize(Ctx *c, const double *part, int nparts, int ncols, double scale, double *out_dev);

// geom.cu
ibm_status geom_classify(Ctx *c);
// body velocity of the rigid motion c->motion at n points (3 per point)
ibm_status geom_body_velocity(Ctx *c, int64_t n, const double *pts, double *out);
// fresh-cell tables of the cells in fidx: body intercept, kind, stencil,
// weights (u = sum w u_m + wb u_BI)
ibm_status geom_fresh_tables(Ctx *c, int64_t nf, const int64_t *fidx, double *bi, uint8_t *kind, int64_t *sidx,
                             double *w, double *wb);
ibm_status compact_flags(Ctx *c, const uint8_t *flags, int64_t **out, int64_t *count);

// flow.cu
ibm_status flow_init(Ctx *c);
ibm_status flow_step(Ctx *c, ibm_step_stats *st);
ibm_status step_graph_eligible(Ctx *c);
ibm_status flow_step_graph(Ctx *c);
ibm_status flow_graph_prepare(Ctx *c);
ibm_status step_graph_begin(Ctx *c);
ibm_status step_graph_end(Ctx *c, ibm_step_stats *st, int steps);
ibm_status poisson_solve_dev(Ctx *c, const double *rhs, double *phi, double rtol, int maxit);
ibm_status poisson_dev_prepare(Ctx *c);
ibm_status step_stats_dev(Ctx *c, const int *hsw);
ibm_status step_stats_read(Ctx *c, ibm_step_stats *st);
// conditional graph nodes during stream capture
struct CondScope {
    cudaStream_t outer = nullptr;
};
ibm_status cond_handle(Ctx *c, cudaGraphConditionalHandle *h);
ibm_status cond_open(Ctx *c, cudaGraphConditionalNodeType type, cudaGraphConditionalHandle h, CondScope *sc);
ibm_status cond_close(Ctx *c, CondScope *sc);
ibm_status ghost_refresh_velocity(Ctx *c, int comp, int *iters);
// the fields after a body move (fresh cells, dead cells, ghost rows, faces)
ibm_status flow_move(Ctx *c);
ibm_status div_stat(Ctx *c, double *out);

}  // namespace ibm
