// Allocation-free Poisson residual, for callers that cannot allocate device
// memory: a host application whose memory manager owns the whole device (a
// framework's caching pool, or a fixed arena sized at start-up) and forbids
// libraries to allocate while it runs a step, or a caller running with the
// device already full, which must not fail for want of a few kilobytes of
// partial sums. It evaluates the quantity that ibm_poisson_solve reports as
// rel_residual, ||P(b - A phi)||_2 / ||P b||_2, and needs no buffer from the
// caller besides its inputs and output: the per-block partial sums live in a
// file-scope device array. It has no counterpart in the paper.
//
// The array g_noalloc_partials is 3 * NOALLOC_MAX_BLOCKS doubles (96 KiB).
// Every GPU that loads the library holds it until the process exits. One
// block handles NOALLOC_CELLS_PER_BLOCK cells, so grids of at most
// NOALLOC_MAX_BLOCKS * NOALLOC_CELLS_PER_BLOCK = 268,435,456 cells are
// accepted; larger ones are rejected with IBM_ERR_ARG.
//
// All calls share the one array and each call overwrites every entry it
// reads before reading it, so nothing needs clearing between calls; two
// calls that overlap on the GPU (different streams, or different host
// threads) race on it. In host code the array's name is only a host-side
// stand-in for the device symbol, so the device address is fetched with
// cudaGetSymbolAddress once per device, the first time the entry point runs
// with that device current; that first call should therefore come before
// any stream capture begins. The call ends by copying the ratio to rel_out
// and waiting for the stream.
#include "ctx.cuh"

#include <math.h>

#include <mutex>

namespace ibm {

constexpr int NOALLOC_MAX_BLOCKS = 4096;
constexpr int64_t NOALLOC_CELLS_PER_BLOCK = 65536;
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_partials[3 * NOALLOC_MAX_BLOCKS];

static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

// residual of the full ghost-cell pressure operator at cell c:
// FLUID rows b - A phi, GHOST rows -(phi_G - sum wp phi_m), DEAD rows 0
__device__ __forceinline__ double fluid_residual(const GridDev &g, const uint8_t *type, const double *b,
                                                 const double *x, int64_t c, int i, int j, int k) {
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const double xc = x[c];
    const double ax = g.dy[j] * g.dz[k], ay = g.dx[i] * g.dz[k], az = g.dx[i] * g.dy[j];
    double s = 0.0;
    if (i > 0) s += ax / g.hx[i] * (x[c - 1] - xc);
    if (i < g.nx - 1) s += ax / g.hx[i + 1] * (x[c + 1] - xc);
    if (j > 0) s += ay / g.hy[j] * (x[c - sy] - xc);
    if (j < g.ny - 1) s += ay / g.hy[j + 1] * (x[c + sy] - xc);
    if (g.ndim == 3) {
        if (k > 0) s += az / g.hz[k] * (x[c - sz] - xc);
        if (k < g.nz - 1) s += az / g.hz[k + 1] * (x[c + sz] - xc);
    }
    return b[c] - s / (g.dx[i] * g.dy[j] * g.dz[k]);
}

// pass 1 (mode 0): columns sum vol*rhs, sum vol*(rhs - A phi) over FLUID
// pass 2 (mode 1): columns sum (rhs - mu_b)^2, sum (r - mu_r)^2 over FLUID
__global__ void k_noalloc_fluid(GridDev g, const uint8_t *__restrict__ type, const double *__restrict__ rhs,
                                const double *__restrict__ phi, int mode, double *__restrict__ part) {
    __shared__ double sh[32];
    const double mub = mode ? part[3 * NOALLOC_MAX_BLOCKS - 2] : 0.0;
    const double mur = mode ? part[3 * NOALLOC_MAX_BLOCKS - 1] : 0.0;
    double a0 = 0.0, a1 = 0.0;
    const int64_t c0 = (int64_t)blockIdx.x * NOALLOC_CELLS_PER_BLOCK;
    const int64_t c1 = c0 + NOALLOC_CELLS_PER_BLOCK < g.n ? c0 + NOALLOC_CELLS_PER_BLOCK : g.n;
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        if (type[c] != FLUID) continue;
        const int64_t t = c / g.nx;
        const int i = (int)(c - t * g.nx), j = (int)(t % g.ny), k = (int)(t / g.ny);
        const double r = fluid_residual(g, type, rhs, phi, c, i, j, k);
        if (mode == 0) {
            const double vol = g.dx[i] * g.dy[j] * g.dz[k];
            a0 += vol * rhs[c];
            a1 += vol * r;
        } else {
            // P b = rhs - mu_b and P(b - A phi) = (rhs - A phi) - mu_r on FLUID rows
            const double db = rhs[c] - mub, dr = r - mur;
            a0 += db * db;
            a1 += dr * dr;
        }
    }
    a0 = block_sum<NOALLOC_THREADS>(a0, sh);
    a1 = block_sum<NOALLOC_THREADS>(a1, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a0;
        part[NOALLOC_MAX_BLOCKS + blockIdx.x] = a1;
    }
}

// ghost rows: sum of squares into column 2 (one block, fixed order)
__global__ void k_noalloc_ghost(GhostDev gh, const double *__restrict__ phi, double *__restrict__ part) {
    __shared__ double sh[32];
    double a = 0.0;
    for (int64_t q = threadIdx.x; q < gh.ng; q += blockDim.x) {
        const int64_t gi = gh.gidx[q];
        double s = phi[gi];
        for (int m = 0; m < 8; ++m) s -= gh.wp[8 * q + m] * phi[gh.sidx[8 * q + m]];
        a += s * s;
    }
    a = block_sum<NOALLOC_THREADS>(a, sh);
    if (threadIdx.x == 0) part[2 * NOALLOC_MAX_BLOCKS] = a;
}

// fixed-order sums of the two block columns; mode 0 stores the volume-
// weighted FLUID means of rhs (mu_b) and of rhs - A phi (mu_r), mode 1 the
// final ratio
__global__ void k_noalloc_final(int nblocks, int mode, double inv_vol, double *__restrict__ part) {
    __shared__ double sh[32];
    double a0 = 0.0, a1 = 0.0;
    for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
        a0 += part[q];
        a1 += part[NOALLOC_MAX_BLOCKS + q];
    }
    a0 = block_sum<NOALLOC_THREADS>(a0, sh);
    a1 = block_sum<NOALLOC_THREADS>(a1, sh);
    if (threadIdx.x == 0) {
        if (mode == 0) {
            part[3 * NOALLOC_MAX_BLOCKS - 2] = a0 * inv_vol;
            part[3 * NOALLOC_MAX_BLOCKS - 1] = a1 * inv_vol;
        } else {
            const double bn = sqrt(a0), rn = sqrt(a1 + part[2 * NOALLOC_MAX_BLOCKS]);
            part[3 * NOALLOC_MAX_BLOCKS - 3] = bn > 0.0 ? rn / bn : 0.0;
        }
    }
}

// device address of the scratch array for the current device, fetched once
static ibm_status noalloc_scratch(Ctx *c, double **out) {
    int dev = -1;
    IBM_CUDA(c, cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return c->fail(IBM_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p)
            return c->fail(IBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = (double *)p;
    }
    *out = g_noalloc_ptr[dev];
    return IBM_OK;
}

}  // namespace ibm

using namespace ibm;

struct ibm_ctx : public Ctx {};

extern "C" ibm_status ibm_poisson_residual_noalloc(ibm_ctx *c, const double *rhs_dev, const double *phi_dev,
                                                    double *rel_out) {
    if (!c) return IBM_ERR_ARG;
    if (!rhs_dev || !phi_dev || !rel_out) return c->fail(IBM_ERR_ARG, "rhs, phi and rel_out must not be NULL");
    if (!c->classified) return c->fail(IBM_ERR_STATE, "ibm_classify_cells must be called first");
    // a host or stale pointer must not reach the kernels
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, rhs_dev) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
        cudaPointerGetAttributes(&at, phi_dev) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return c->fail(IBM_ERR_ARG, "rhs and phi must be device memory");
    }
    const int64_t nblocks = (c->N + NOALLOC_CELLS_PER_BLOCK - 1) / NOALLOC_CELLS_PER_BLOCK;
    if (nblocks > NOALLOC_MAX_BLOCKS)
        return c->fail(IBM_ERR_ARG, "grid has more than 268,435,456 cells, the scratch limit of "
                                    "ibm_poisson_residual_noalloc");
    double *part = nullptr;
    IBM_TRY(noalloc_scratch(c, &part));
    const double inv_vol = 1.0 / c->fluid_vol;
    k_noalloc_fluid<<<(unsigned)nblocks, NOALLOC_THREADS, 0, c->s>>>(c->g, c->type, rhs_dev, phi_dev, 0, part);
    k_noalloc_final<<<1, NOALLOC_THREADS, 0, c->s>>>((int)nblocks, 0, inv_vol, part);
    k_noalloc_fluid<<<(unsigned)nblocks, NOALLOC_THREADS, 0, c->s>>>(c->g, c->type, rhs_dev, phi_dev, 1, part);
    k_noalloc_ghost<<<1, NOALLOC_THREADS, 0, c->s>>>(c->gh, phi_dev, part);
    k_noalloc_final<<<1, NOALLOC_THREADS, 0, c->s>>>((int)nblocks, 1, inv_vol, part);
    IBM_LAUNCHED(c);
    IBM_CUDA(c, cudaMemcpyAsync(rel_out, part + 3 * NOALLOC_MAX_BLOCKS - 3, sizeof(double), cudaMemcpyDefault, c->s));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    return IBM_OK;
}
