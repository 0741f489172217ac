/*
 * ibm.h -- C ABI of the GB300 ghost-cell immersed-boundary solver library
 * (libibm.so). Plain C types only: host or device pointers and sizes.
 *
 * The library advances the incompressible Navier-Stokes equations in
 * conservative form (Eq. 1 of the paper) on a non-uniform Cartesian grid
 * with a sharp-interface ghost-cell immersed body (Section 2.2), by the
 * fractional-step method (Section 2.1): an Adams-Bashforth-2 convection /
 * Crank-Nicolson diffusion predictor, a pressure Poisson solve with
 * ghost-cell-modified boundary rows, and a projection.
 *
 * Conventions used by every call below:
 *   - cells are stored structure-of-arrays with x the unit-stride axis:
 *     linear index c = i + nx*(j + ny*k); 2D grids have nz = 1;
 *   - x-face arrays hold (nx+1)*ny*nz values, index i + (nx+1)*(j + ny*k);
 *     y-face arrays nx*(ny+1)*nz values, index i + nx*(j + (ny+1)*k);
 *     z-face arrays nx*ny*(nz+1) values, index i + nx*(j + ny*k);
 *   - cell types are bytes: IBM_FLUID, IBM_GHOST, IBM_DEAD;
 *   - every call returns an ibm_status; none aborts, traps or exits. A
 *     per-context message is kept for ibm_last_error();
 *   - every call enqueues its GPU work on the stream given at creation and
 *     returns after synchronising that stream, so a device-side error is
 *     reported by the call that caused it;
 *   - host arrays passed in are copied before the call returns; device
 *     pointers passed in are borrowed for the duration of the call only.
 *   - a context may be used by one host thread at a time.
 */
#ifndef IBM_H
#define IBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibm_ctx ibm_ctx;

typedef enum {
    IBM_OK = 0,
    IBM_ERR_ARG = 1,           /* invalid argument (null pointer, size, range) */
    IBM_ERR_OOM = 2,           /* device or host allocation failed */
    IBM_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
    IBM_ERR_MESH = 4,          /* body mesh not closed/manifold, or degenerate */
    IBM_ERR_STATE = 5,         /* call order violated (e.g. step before classify) */
    IBM_ERR_NOT_CONVERGED = 6, /* iteration limit reached before the tolerance */
    IBM_ERR_DIVERGED = 7,      /* NaN or Inf met in a residual */
    IBM_ERR_TIMEOUT = 8        /* a bounded device-side wait gave up */
} ibm_status;

enum { IBM_FLUID = 0, IBM_GHOST = 1, IBM_DEAD = 2 };

/* outer boundary conditions, per face in the order x-, x+, y-, y+, z-, z+ */
enum {
    IBM_BC_INFLOW = 0,  /* Dirichlet u = u_inf on every component */
    IBM_BC_OUTFLOW = 1, /* zero normal gradient; outflow face velocities get one
                           uniform correction so the net boundary flux is zero */
    IBM_BC_SLIP = 2     /* normal component 0, tangential zero gradient */
};

/* arithmetic of the Poisson solver's inner multigrid-preconditioned CG */
enum { IBM_FP64 = 0, IBM_MIXED = 1 };

/* outer Krylov method of the Poisson solver */
enum { IBM_OUTER_BICGSTAB = 0, IBM_OUTER_FGMRES = 1 };

typedef struct {
    int ndim;              /* 2 or 3 */
    int nx, ny, nz;        /* cells per axis, each >= 2 (nz = 1 when ndim == 2) */
    const double *xf;      /* host, nx+1 increasing face coordinates (copied) */
    const double *yf;      /* host, ny+1 increasing face coordinates (copied) */
    const double *zf;      /* host, nz+1 increasing face coordinates; ignored in 2D */
    double Re;             /* Reynolds number (> 0) */
    double dt;             /* time step (> 0) */
    double u_inf[3];       /* inflow velocity */
    int bc[6];             /* IBM_BC_* per outer face */
    int precision;         /* IBM_FP64 or IBM_MIXED */
    void *stream;          /* cudaStream_t to run on (borrowed); NULL = default stream */
    /* optional device allocator; both NULL = cudaMalloc/cudaFree. The
       context frees everything it allocated through the same hook. Blocks
       must be 16-byte aligned (the streaming kernels use 16-byte accesses);
       a misaligned block is freed and reported as IBM_ERR_OOM. */
    void *(*alloc)(size_t bytes, void *alloc_ctx);
    void (*free)(void *ptr, void *alloc_ctx);
    void *alloc_ctx;
} ibm_grid_desc;

typedef struct {
    double rtol;        /* Poisson: relative residual ||P(b-A phi)||/||P b|| target */
    int max_outer;      /* Poisson: outer iteration limit (BiCGStab iterations or
                           FGMRES steps over all restarts) */
    int restart;        /* Poisson: FGMRES restart length (1..16) */
    int inner_iters;    /* Poisson: MG-PCG iterations per preconditioner call */
    int nu1, nu2;       /* multigrid pre/post red-black Gauss-Seidel sweeps, 1..8; equal
                           when inner_iters > 1 (CG needs a symmetric V-cycle) */
    int coarse_sweeps;  /* red-black sweep pairs on the coarsest level */
    double helm_rtol;   /* Crank-Nicolson Helmholtz: relative residual target */
    int helm_maxit;     /* Helmholtz: sweep limit */
    double ghost_tol;   /* velocity ghost refresh: max relative change */
    int ghost_maxit;    /* velocity ghost refresh: Jacobi pass limit */
    int precision;      /* IBM_FP64 or IBM_MIXED */
    int outer;          /* IBM_OUTER_BICGSTAB or IBM_OUTER_FGMRES */
    int band_sweeps;    /* damped Jacobi sweeps of the full ghost-cell operator on the
                           near-body band (band_width), after the multigrid cycle of
                           each preconditioner call, in its precision (0 = none).
                           The cycle works on the staircase operator, whose faces
                           between FLUID and GHOST cells are closed; these sweeps
                           correct the preconditioned vector where the two
                           operators differ */
    double band_omega;  /* their damping factor, in (0, 1] */
    double mixed_inner_rtol; /* IBM_MIXED with FGMRES: residual reduction asked of each
                           FP32 Krylov solve inside the FP64 defect correction */
    int mg_interp;      /* multigrid transfer: 1 trilinear prolongation with its transpose
                           as restriction, 0 piecewise constant with summation */
    int tile_x;         /* threads per block along x of the multigrid smoother and
                           transfer kernels (one block per grid row segment):
                           32, 64, 128, 256 or 512 */
    int graph;          /* 1: the multigrid V-cycle is captured once into a CUDA graph
                           and replayed at every preconditioner call (one launch
                           instead of ~10 per level; not on the legacy default
                           stream, which cannot be captured, nor while the kernel
                           timer runs); 2: the whole fractional step is one captured
                           graph with device-side loop control (ibm_step_async);
                           0: launched kernel by kernel */
    int precond;        /* Poisson preconditioner: 0 multigrid V-cycle; 1 scheduled
                           relaxation Jacobi (SRJ): srj_sweeps damped-Jacobi sweeps of
                           the same staircase operator from a zero guess, relaxation
                           factors 1/tau_k with tau_k the Chebyshev points of
                           [srj_lmin, 2] (Section 2.1 names SRJ as the preconditioner
                           of its BiCGStab) */
    int srj_sweeps;     /* SRJ sweeps per preconditioner call, 1..64 */
    double srj_lmin;    /* lower end of the damped interval of the Jacobi-scaled
                           spectrum, in [0, 2); 0 = 2 / srj_sweeps^2 */
    int helm_solver;    /* Crank-Nicolson Helmholtz: 0 red-black Gauss-Seidel; 1 scheduled
                           relaxation Jacobi (Section 2.1's solver for the
                           advection-diffusion step): cycles of 8 damped-Jacobi sweeps
                           with Chebyshev factors over the Jacobi-scaled spectrum
                           [1 - rho, 1 + rho], rho bounded from the grid; host-driven */
    double smooth_omega; /* relaxation factor of the multigrid red-black smoother, in
                           (0, 2): 1 = Gauss-Seidel, > 1 over-relaxed */
    double reorth_eta;  /* FGMRES classical Gram-Schmidt: a second orthogonalisation pass
                           when ||w|| drops below reorth_eta times its value before the
                           first pass, in [0, 1] (0 = never, 1 = always). Default 0.3:
                           the usual 1/sqrt(2) fires in most steps here, where the
                           multigrid-preconditioned vectors lie close to the basis, and
                           buys no iteration */
    int helm_check_first; /* Helmholtz red-black solve: sweeps before the first residual
                           test, >= 1; later tests follow at s + max(2, s / 4) sweeps
                           (s the sweep count of the previous test), so that a solve
                           needing n sweeps takes O(log n) tests. Each test costs
                           about two sweeps in FP64; default 6, the count the 3D
                           wing's components need at helm_rtol 1e-12 on its
                           201M-cell grid (4 on the 25.2M-cell grid, where 4
                           saves 4% of the step) */
    double helm_omega;  /* Helmholtz red-black relaxation factor: 0 = automatic,
                           2 / (1 + sqrt(1 - rho^2)) with rho the grid's bound on the
                           Jacobi spectral radius (Young's optimum for a red-black
                           ordered 7-point operator); 1 = Gauss-Seidel; otherwise the
                           factor itself, in (0, 2) */
    int fine_split;     /* 1: the finest FP32 multigrid level (mixed precision, nx a
                           multiple of 8) keeps x, f and the open-face mask with the
                           two red-black colours stored apart (each row's cells of one
                           colour packed in x order), so a colour pass streams only the
                           other colour's x and its own f; same arithmetic and results
                           bit for bit as 0, the cell-ordered layout */
    int band_width;     /* the near-body band of band_sweeps: the ghost cells and the
                           FLUID cells within band_width faces of one, 1..4; read
                           when the cells are classified (ibm_classify_cells,
                           ibm_move_body) */
    int poisson_hist;   /* pairs (solution, projected right-hand side) of earlier
                           pressure solves kept on the device, 0..16: each step
                           starts its Poisson solve from the combination of the
                           stored solutions whose right-hand sides best fit the
                           new one in the least-squares sense (a projection onto
                           earlier solutions, which contains the polynomial
                           extrapolation of the last pressures); 0 = the
                           extrapolation alone. Cleared by ibm_classify_cells and
                           ibm_move_body (the operator changes), kept by
                           ibm_set_field (the pairs stay solutions of the same
                           operator); a checkpoint that must restart bit for bit
                           saves IBM_FIELD_P_HIST_*. Costs 16 bytes per cell and
                           pair */
    int tail_cells;     /* multigrid levels below the finest with at most tail_cells
                           cells run as one persistent launch per V-cycle (a
                           cluster of up to 8 blocks walks their passes with
                           hardware cluster barriers between them; same values as
                           the per-level kernels, bit for bit); 0 = every level
                           launched on its own, the default: on GB300 the
                           per-level kernels replayed from CUDA graphs measured
                           faster (2D 256x128 cylinder step 2.28 ms without the
                           tail, 2.42-2.58 ms with it). Needs mg_interp 1 and
                           three levels or more */
    int nu_coarse;      /* red-black sweeps before and after the coarse-grid correction on
                           the multigrid levels below the finest, 1..8; 0 = nu1 and nu2
                           there too */
} ibm_solver_opts;

typedef struct {
    int64_t n_fluid, n_ghost, n_dead;
    int64_t n_kind[3];  /* ghosts per stencil kind: 0 eight fluid/ghost corners,
                           1 the ghost itself is a corner (boundary row), 2 fallback */
} ibm_table_info;

typedef struct {
    int outer_iters;         /* FGMRES iterations */
    int inner_iters;         /* MG-PCG iterations summed over preconditioner calls */
    double rel_residual;     /* final ||P(b - A phi)|| / ||P b||, in FP64 */
    double ms;               /* device time of the solve */
} ibm_solve_stats;

typedef struct {
    int steps;               /* steps taken by this call */
    int poisson_outer;       /* FGMRES iterations, summed over steps */
    int poisson_inner;       /* MG-PCG iterations, summed */
    int helm_sweeps;         /* Helmholtz red-black sweeps, summed over components */
    double rel_residual;     /* Poisson relative residual of the last step */
    double max_div;          /* max |div U| over FLUID cells after the last projection,
                                minus its volume-weighted FLUID mean */
    double ms_total, ms_predictor, ms_poisson, ms_projection;
} ibm_step_stats;

/* Per-ghost tables, host destinations; any pointer may be NULL (skipped).
   Sizes: type N; gidx, dist, base, kind, cmask, bv, bp n_ghost;
   bi, nrm, ip 3*n_ghost; sidx, wv, wp 8*n_ghost (row per ghost). */
typedef struct {
    uint8_t *type;
    int64_t *gidx;
    double *bi, *nrm, *ip, *dist;
    int64_t *base;
    uint8_t *kind, *cmask;
    int64_t *sidx;
    double *wv, *wp, *bv, *bp;
} ibm_tables_host;

/* fields for ibm_get_field / ibm_set_field (element type and count) */
enum {
    IBM_FIELD_U = 0, IBM_FIELD_V = 1, IBM_FIELD_W = 2,   /* cell velocity, double, N */
    IBM_FIELD_P = 3,                                      /* pressure, double, N */
    IBM_FIELD_FACE_U = 4, IBM_FIELD_FACE_V = 5, IBM_FIELD_FACE_W = 6, /* face velocity, double */
    IBM_FIELD_NOLD_U = 7, IBM_FIELD_NOLD_V = 8, IBM_FIELD_NOLD_W = 9, /* previous convective term */
    IBM_FIELD_TYPE = 10,                                  /* uint8, N */
    IBM_FIELD_USTAR_U = 11, IBM_FIELD_USTAR_V = 12, IBM_FIELD_USTAR_W = 13, /* last predictor */
    IBM_FIELD_RHS = 14,                                   /* last Poisson right-hand side, N */
    IBM_FIELD_STEP = 15,                                  /* int64 step counter, 1 value */
    IBM_FIELD_P_PREV = 16,                                /* pressure of the step before, N */
    IBM_FIELD_P_PREV2 = 17,                               /* pressure two steps before, N. The Poisson
                                                             initial guess is P on the first three
                                                             steps, 2 P - P_PREV on the fourth, then
                                                             3 P - 3 P_PREV + P_PREV2 (both are part
                                                             of a checkpoint), unless the guess
                                                             history (poisson_hist) holds a pair */
    IBM_FIELD_P_HIST_X = 18,   /* Poisson guess history (poisson_hist > 0): the stored
                                  solutions, poisson_hist x N doubles (slot-major) */
    IBM_FIELD_P_HIST_B = 19,   /* their projected right-hand sides, poisson_hist x N */
    IBM_FIELD_P_HIST_CTL = 20  /* pairs held, next slot and the Gram matrix of the
                                  stored right-hand sides: 2 + poisson_hist^2 doubles */
};

/* Defaults: rtol 1e-10, max_outer 400, inner_iters 1, nu1 2, nu2 1 (nu_coarse 3 on the
   levels below the finest),
   coarse_sweeps 32, helm_rtol 1e-12, helm_maxit 500, ghost_tol 1e-15,
   ghost_maxit 100, precision IBM_FP64, outer IBM_OUTER_FGMRES, restart 16,
   band_sweeps 8, band_omega 0.85, mixed_inner_rtol 1e-4, mg_interp 1,
   tile_x 128, graph 1, precond 0, srj_sweeps 16, srj_lmin 0, helm_solver 0, smooth_omega 1, reorth_eta 0.3,
   helm_check_first 6, helm_omega 1, fine_split 1, band_width 3, poisson_hist 8, tail_cells 0, nu_coarse 3. */
ibm_status ibm_default_opts(ibm_solver_opts *opts);

/* Create a context for one grid (Section 2.1: non-uniform Cartesian grid).
   Validates the descriptor (IBM_ERR_ARG), copies the face coordinates to
   the device, allocates every field and solver buffer (IBM_ERR_OOM) and
   builds the multigrid hierarchy of the grid. *out is NULL on failure. */
ibm_status ibm_create_grid(const ibm_grid_desc *desc, ibm_ctx **out);

/* Replace solver options (validated: IBM_ERR_ARG). May be called at any time
   after creation; switching to IBM_MIXED allocates the FP32 buffers. */
ibm_status ibm_set_opts(ibm_ctx *ctx, const ibm_solver_opts *opts);

/* Add one closed immersed body (Section 2.2: the unstructured surface mesh
   immersed in the Cartesian grid). verts: host, nv*3 doubles (z ignored in
   2D). elems: host int32, 3D triangles ne*3 counter-clockwise seen from
   outside, 2D segments ne*2 counter-clockwise around the body. Both are
   copied. Several calls add several bodies (their union; they must not
   overlap). IBM_ERR_MESH if an edge (3D) or vertex (2D) is not shared by
   exactly two elements in opposite directions, or an index is out of range.
   Invalidates earlier classification (IBM_ERR_STATE until re-classified). */
ibm_status ibm_set_body(ibm_ctx *ctx, const double *verts, int64_t nv,
                        const int32_t *elems, int64_t ne);

/* Classify cells and build the ghost-cell tables (Section 2.2: ray tracing
   to blank dead cells, ghost = dead cell with a fluid face neighbour, body
   intercept, image point, the 8 surrounding cells and the weights of Eq. 2
   from the Vandermonde system of Eq. 3). All on the GPU. Then resets the
   flow to an impulsive start: u = u_inf on FLUID cells, Dirichlet ghost
   values, 0 in DEAD cells, face velocities from those, p = 0, step 0.
   out may be NULL. IBM_ERR_STATE if no body was set. */
ibm_status ibm_classify_cells(ibm_ctx *ctx, ibm_table_info *out);

/* Move the bodies (Section 2.2, moving bodies: the body moves at the start
   of a step; dead cells that become fluid, "fresh cells", take an
   interpolation that uses the body velocity at their body intercept).
   verts: host, nv x 3 doubles, the new positions of every vertex added by
   ibm_set_body, in the same order (the elements are kept; copied). motion:
   host, 9 doubles: the rigid velocity U (3), angular velocity Omega (3) and
   rotation centre (3); the body velocity at a surface point x is
   U + Omega x (x - centre). In 2D the vertices keep z = 0 and U_z, Omega_x,
   Omega_y are 0. The call reclassifies the cells and rebuilds the ghost
   tables and multigrid operators of the new position, keeps the flow state,
   and then:
     - fresh cells (FLUID now, not before): u = sum w_m u_m + wb u_BI from the
       trilinear fit on the lattice cell of centres that has the fresh cell as
       a corner and extends away from the body, the fresh cell's row replaced
       by the Dirichlet row at its intercept; other fresh corners are solved
       with it (Jacobi passes to ghost_tol); a ghost or dead corner gives
       u = u_BI; the next step takes the Euler start of the convective term
       at these cells;
     - DEAD cells get u = 0; ghost rows use u_BI = the body velocity at their
       intercept, in this call and in the steps after it (until the next
       ibm_classify_cells, which puts the body at rest);
     - interior face velocities next to a cell whose type changed take the
       face rule (mean of the two cells with a FLUID side and no DEAD side,
       else 0); the other faces keep theirs.
   The pressure closure stays dp/dn = 0. Steps after a move are host-driven
   (opts graph 2 falls back). out may be NULL. IBM_ERR_STATE before
   ibm_classify_cells; IBM_ERR_ARG for another vertex count, non-finite
   input, or 2D input off the plane. */
ibm_status ibm_move_body(ibm_ctx *ctx, const double *verts, int64_t nv, const double *motion,
                         ibm_table_info *out);

/* Advance nsteps fractional steps (Section 2.1): convective term, AB2 + CN
   right-hand side, CN Helmholtz solve with Dirichlet ghost rows, face
   velocities and divergence, pressure Poisson solve (BiCGStab or FGMRES in
   FP64 around multigrid-preconditioned CG on the staircase operator), projection,
   velocity ghost refresh. out may be NULL. Returns IBM_ERR_NOT_CONVERGED
   when a solve hit its iteration limit (the step is still completed),
   IBM_ERR_DIVERGED on NaN/Inf (state then undefined). */
ibm_status ibm_step(ibm_ctx *ctx, int nsteps, ibm_step_stats *out);

/* Device-controlled steps (no counterpart in the paper). With opts.graph ==
   2 every step after the first of a classification runs as one captured
   CUDA graph whose Helmholtz, ghost-refresh, FGMRES and refinement loops are
   conditional nodes decided on the device (same kernels and stopping tests
   as ibm_step; Givens rotations evaluated on the device), so a step needs
   no host round trip; not available on the legacy default stream or with
   BiCGStab or inner_iters > 1 (those steps run host-driven). The graphs are
   captured on first use and again after a re-classification or an option
   change. ibm_step_async enqueues nsteps such steps on the context stream
   and returns without waiting (steps that cannot be captured still run to
   completion inside the call); ibm_step_wait waits for them and returns
   their statistics and status as ibm_step would (per-phase times are not
   split: ms_total only). ibm_step is ibm_step_async + ibm_step_wait. */
ibm_status ibm_step_async(ibm_ctx *ctx, int nsteps);
/* Capture now the graphs the next steps will use (the next step and both
   alternations of the step buffers after it), so that later ibm_step /
   ibm_step_async calls launch without capturing; a no-op when the steps
   would not be captured. */
ibm_status ibm_step_prepare(ibm_ctx *ctx);
ibm_status ibm_step_wait(ibm_ctx *ctx, ibm_step_stats *out);

/* Solve the ghost-cell pressure Poisson system A phi = P b (Section 2.1
   pressure equation; Section 2.2 Neumann ghost rows) on the classified
   grid. rhs_dev: device, N doubles; only FLUID rows are read, and their
   volume-weighted mean is removed (compatibility). phi_dev: device, N
   doubles; in: initial guess, out: solution with zero volume-weighted mean
   over FLUID cells (DEAD cells 0). rhs_dev and phi_dev must not overlap.
   rtol <= 0 or maxit <= 0 take the context options. stats may be NULL. */
ibm_status ibm_poisson_solve(ibm_ctx *ctx, const double *rhs_dev, double *phi_dev,
                             double rtol, int maxit, ibm_solve_stats *stats);

/* Copy the classification and ghost tables to host arrays (tests, tools). */
ibm_status ibm_get_tables(ibm_ctx *ctx, const ibm_tables_host *dst);

/* Copy a field out of / into the context (checkpoint and restart, tests).
   dst/src: host pointer when is_device == 0, device pointer otherwise;
   bytes must equal the field's size exactly (IBM_ERR_ARG otherwise). */
ibm_status ibm_get_field(ibm_ctx *ctx, int field, void *dst, int is_device, size_t bytes);
ibm_status ibm_set_field(ibm_ctx *ctx, int field, const void *src, int is_device, size_t bytes);

/* Number of N-sized cells and of ghost cells (after classification). */
ibm_status ibm_sizes(ibm_ctx *ctx, int64_t *n_cells, int64_t *n_ghost);

/* Number of CUDA kernels this context has launched since creation
   (diagnostics: lets a caller count the device work behind a call). */
ibm_status ibm_launch_count(ibm_ctx *ctx, int64_t *count);

/* Diagnostic event timer. ibm_kernel_timer(ctx, 1) starts recording a CUDA
   event pair on the context stream around every launch of the kernels
   listed below (and clears the totals); 0 stops. ibm_kernel_time returns the
   summed device time (ms) and the launch count of one kernel since the
   timer was started. Kernel ids: 0 red-black Gauss-Seidel colour pass on
   the finest multigrid level; 1 staircase-operator product on the finest
   level; 2 full ghost-cell pressure operator; 3 FGMRES multi-dot; 4 FGMRES
   orthogonalisation; 5 Helmholtz colour pass; 6 convective term and
   AB2/CN right-hand side; 7 red-black pass on coarse levels; 8 residual +
   restriction; 9 prolongation; 10 every other kernel of the Poisson solver;
   11 the persistent V-cycle tail (tail_cells).
   Recording adds host overhead per launch. */
ibm_status ibm_kernel_timer(ibm_ctx *ctx, int enable);
ibm_status ibm_kernel_time(ibm_ctx *ctx, int kernel, double *ms_total, int64_t *launches);

/* Allocation-free residual check (no counterpart in the paper): returns in
   *rel_out (host or device pointer) the relative residual
   ||P(b - A phi)||_2 / ||P b||_2 of a pressure solution phi_dev for the
   right-hand side rhs_dev (both device memory, N doubles, else IBM_ERR_ARG;
   b = rhs with its volume-weighted FLUID mean removed), the quantity
   ibm_poisson_solve reports as rel_residual. For callers that cannot
   allocate device memory: an application whose memory manager owns the whole
   device and forbids libraries to allocate during its step, or a caller
   running with the device already full. It calls no cudaMalloc/cudaFree and
   keeps its partial sums in a 96 KiB file-scope device array, held by every
   GPU that loads the library until exit. Grids above 268,435,456 cells are
   rejected (IBM_ERR_ARG). The first call on each device looks up that
   array's device address with that device current, so make it before
   starting any stream capture. Calls share the array: calls that overlap on
   the GPU (other streams or host threads) race. The call synchronises the
   context's stream before it returns. IBM_ERR_STATE before
   ibm_classify_cells. */
ibm_status ibm_poisson_residual_noalloc(ibm_ctx *ctx, const double *rhs_dev, const double *phi_dev,
                                        double *rel_out);

/* Release every allocation of the context. NULL is accepted. */
ibm_status ibm_destroy(ibm_ctx *ctx);

/* Message of the last failed call on ctx ("" if none); ctx NULL gives the
   message of the last failed ibm_create_grid on this thread. */
const char *ibm_last_error(ibm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* IBM_H */
