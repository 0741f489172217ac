/*
 * ibm_serve.h -- request loop over many independent immersed-boundary cases
 * on one GPU (part of libibm.so). Plain C types only.
 *
 * The paper runs one case at a time (its Section 3). This interface has no
 * counterpart there: it serves a stream of independent cases of mixed grid
 * sizes, each one a grid plus bodies plus either some fractional steps
 * (Section 2.1) or one pressure Poisson solve, through the calls of ibm.h.
 *
 * Model:
 *   - The server owns `max_slots` slots. Each slot has its own host worker
 *     thread and its own non-blocking CUDA stream, so the kernels of cases in
 *     different slots overlap on the device.
 *   - Requests wait in one first-in first-out queue. The head request is
 *     admitted when a slot is free and its device footprint (ibm_case_bytes)
 *     fits both under the server's byte budget, counted over the cases
 *     already admitted, and under the device's free memory (cudaMemGetInfo
 *     plus what the server's pool holds unused) minus `hbm_reserve`. A
 *     request that arrives while others run is thus admitted as soon as a
 *     slot and memory free up, and runs beside them.
 *   - An admitted case keeps all its fields resident on the device from
 *     classification to its last step; only its results are copied back.
 *   - Device memory comes from a stream-ordered pool owned by the server, so
 *     creating and releasing cases never synchronises the whole device.
 *   - Every kernel of the library uses a fixed launch shape and fixed-order
 *     reductions, so a case gives the same bits alone and in a mix.
 *
 * Thread safety: ibm_server_submit, _wait and _get_stats may be called from
 * any host thread, concurrently; ibm_server_destroy must not overlap any
 * other call on the same server.
 */
#ifndef IBM_SERVE_H
#define IBM_SERVE_H

#include "ibm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibm_server ibm_server;

typedef struct {
    int max_slots;       /* cases resident and advancing at once, 1..64 */
    int device;          /* CUDA device ordinal */
    size_t hbm_reserve;  /* bytes of device memory the server leaves free */
    size_t hbm_budget;   /* bound on the summed footprint of admitted cases;
                            0 = free device memory at creation minus hbm_reserve */
} ibm_server_opts;

enum { IBM_REQ_STEP = 0, IBM_REQ_POISSON = 1 };

typedef struct {
    int kind;                    /* IBM_REQ_STEP or IBM_REQ_POISSON */
    ibm_grid_desc grid;          /* as for ibm_create_grid; stream and the
                                    allocator fields are ignored (the server's) */
    const ibm_solver_opts *opts; /* NULL = ibm_default_opts with grid.precision */
    int nbodies;                 /* bodies, each as for ibm_set_body */
    const double *const *verts;  /* [nbodies] host, nverts[b] * 3 doubles (z ignored in 2D) */
    const int64_t *nverts;       /* [nbodies] */
    const int32_t *const *elems; /* [nbodies] host, nelems[b] * ndim ints */
    const int64_t *nelems;       /* [nbodies] */
    int nsteps;                  /* IBM_REQ_STEP: fractional steps to take (>= 1) */
    const double *rhs;           /* IBM_REQ_POISSON: host right-hand side, N doubles */
    double rtol;                 /* IBM_REQ_POISSON: relative residual target */
    int maxit;                   /* IBM_REQ_POISSON: outer iteration limit */
    /* optional host outputs, N doubles each (NULL = not wanted), written
       before the request completes (out_w is ignored in 2D); for
       IBM_REQ_POISSON out_p receives phi.
       They must stay valid until ibm_server_wait returns for the request. */
    double *out_u, *out_v, *out_w, *out_p;
} ibm_request;

typedef struct {
    ibm_status status;     /* the request's own outcome */
    int64_t cells;         /* N of its grid */
    int steps;             /* fractional steps taken */
    double t_submit;       /* seconds since the server was created */
    double t_admit;
    double t_done;
    size_t bytes_estimate; /* footprint used for admission */
    size_t bytes_peak;     /* device bytes the case actually held at most */
    ibm_step_stats step;   /* IBM_REQ_STEP */
    ibm_solve_stats solve; /* IBM_REQ_POISSON */
    int slot;              /* slot that ran it */
    char error[160];       /* message when status != IBM_OK */
} ibm_result;

typedef struct {
    int64_t submitted, completed, failed, queued, running;
    int peak_running;      /* most cases resident at once */
    size_t budget;         /* byte budget in force */
    size_t admitted_bytes; /* summed footprint of the running cases */
    size_t peak_admitted_bytes;
} ibm_server_stats;

/* Device footprint estimate of one case (bytes), an upper bound on what the
   library allocates for that grid, precision and total body element count
   with the default options (a Poisson guess history of 8 pairs; the server
   adds the difference for a request whose options keep more). */
size_t ibm_case_bytes(int ndim, int nx, int ny, int nz, int precision, int64_t nelems_total);

/* Start the slots' worker threads on opts->device. IBM_ERR_ARG for a bad
   option, IBM_ERR_CUDA if the device, streams or pool cannot be set up. */
ibm_status ibm_server_create(const ibm_server_opts *opts, ibm_server **out);

/* Queue a request: every host input is copied before the call returns (the
   output pointers are kept). *id identifies it for ibm_server_wait.
   IBM_ERR_ARG for an invalid request, IBM_ERR_OOM when its footprint
   exceeds the budget even with nothing else admitted, IBM_ERR_STATE once
   the server is shutting down. */
ibm_status ibm_server_submit(ibm_server *srv, const ibm_request *req, int64_t *id);

/* Wait up to timeout_s seconds (< 0: forever) for request id. IBM_OK: done,
   *out filled, and the id is released. IBM_ERR_TIMEOUT: still queued or
   running. IBM_ERR_ARG: unknown id. */
ibm_status ibm_server_wait(ibm_server *srv, int64_t id, double timeout_s, ibm_result *out);

ibm_status ibm_server_get_stats(ibm_server *srv, ibm_server_stats *out);

/* Finish the running requests, fail the queued ones with IBM_ERR_STATE,
   join the workers and release every device resource. */
ibm_status ibm_server_destroy(ibm_server *srv);

/* Autotuner (no counterpart in the paper): builds the case (desc, bodies,
   on desc's stream and allocator), then for each of the ncand option sets
   restores the same impulsive-start state with an empty Poisson guess
   history, takes one untimed step (which also captures any CUDA graph the
   options ask for), restores the state again and times `steps` fractional
   steps with CUDA events on the stream.
   ms_per_step[i] (host, ncand values) receives candidate i's device time
   per step, or a negative value if it failed (IBM_ERR_ARG options,
   non-convergence); *best the index of the fastest. IBM_ERR_ARG for bad
   arguments, IBM_ERR_NOT_CONVERGED if no candidate succeeded; errors in
   building the case are returned as they come. */
ibm_status ibm_tune(const ibm_grid_desc *desc, int nbodies, const double *const *verts, const int64_t *nverts,
                    const int32_t *const *elems, const int64_t *nelems, const ibm_solver_opts *cand, int ncand,
                    int steps, int *best, double *ms_per_step);

#ifdef __cplusplus
}
#endif

#endif /* IBM_SERVE_H */
