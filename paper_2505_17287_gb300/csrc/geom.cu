// Immersed-body geometry on the GPU (Section 2.2 of the paper): dead-cell
// blanking by ray parity ("ray tracing"), fluid/ghost/dead classification,
// body intercept (closest surface point), image point, and the weights of
// Eq. 2 from the Vandermonde system of Eq. 3 (batched 8x8, FP64, one thread
// per ghost cell; 4x4 in 2D).
//
// Exactness: inside/outside runs on quantised integer coordinates with
// 128-bit products, so it is exact; the centre is perturbed symbolically to
// (X+e^2, Y+e^4, Z-e) (2D: (X+e^2, Y-e)). All floating-point work uses one
// correctly rounded IEEE operation per written operation, in the written
// order; this file is compiled with --fmad=false so no multiply-add is fused.
#include "ctx.cuh"

#include <math.h>

namespace ibm {

typedef __int128 i128;

__global__ void k_quantize(const double *__restrict__ x, int64_t n, double lo, double s, int64_t *__restrict__ q) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) q[t] = __double2ll_rn((x[t] - lo) * s);
}

__global__ void k_quantize_verts(const double *__restrict__ v, int64_t nv, int nd, double lo0, double lo1,
                                 double lo2, double s, int64_t *__restrict__ q) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nv) return;
    q[nd * t + 0] = __double2ll_rn((v[3 * t + 0] - lo0) * s);
    q[nd * t + 1] = __double2ll_rn((v[3 * t + 1] - lo1) * s);
    if (nd == 3) q[nd * t + 2] = __double2ll_rn((v[3 * t + 2] - lo2) * s);
}

__device__ __forceinline__ int sgn128(i128 v) { return (v > 0) - (v < 0); }

// sign of orient(p->q, P) with P perturbed to (X+e, Y+e^2)
__device__ __forceinline__ int orient_pert(int64_t px, int64_t py, int64_t qx, int64_t qy, int64_t X, int64_t Y,
                                           i128 &w) {
    w = (i128)(qx - px) * (i128)(Y - py) - (i128)(qy - py) * (i128)(X - px);
    if (w != 0) return sgn128(w);
    if (qy != py) return (qy - py) > 0 ? -1 : 1;
    if (qx != px) return (qx - px) > 0 ? 1 : -1;
    return 0;
}

constexpr int MAX_CROSS = 64;
constexpr int TRI_TILE = 128;

// 3D: one thread per column (i, j); ray along +z. Vq: quantised vertices
// (nv*3), tris (nt*3). inside[c] in {0,1}.
__global__ void __launch_bounds__(128) k_inside3d(int nx, int ny, int nz, const int64_t *__restrict__ Xq,
                                                  const int64_t *__restrict__ Yq, const int64_t *__restrict__ Zq,
                                                  const int64_t *__restrict__ Vq, int64_t nt,
                                                  const int32_t *__restrict__ tris, uint8_t *__restrict__ inside,
                                                  int *__restrict__ err) {
    __shared__ int64_t tv[TRI_TILE][9];
    const int j = blockIdx.x;
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    const bool active = i < nx;
    const int64_t X = active ? Xq[i] : 0, Y = Yq[j];
    i128 S[MAX_CROSS], Dn[MAX_CROSS];
    int nc = 0;
    bool overflow = false;
    for (int64_t t0 = 0; t0 < nt; t0 += TRI_TILE) {
        __syncthreads();
        for (int q = threadIdx.x; q < TRI_TILE * 3; q += blockDim.x) {
            const int64_t t = t0 + q / 3;
            const int corner = q % 3;
            if (t < nt) {
                const int64_t v = tris[3 * t + corner];
                tv[q / 3][3 * corner + 0] = Vq[3 * v + 0];
                tv[q / 3][3 * corner + 1] = Vq[3 * v + 1];
                tv[q / 3][3 * corner + 2] = Vq[3 * v + 2];
            }
        }
        __syncthreads();
        if (!active) continue;
        const int cnt = (int)min((int64_t)TRI_TILE, nt - t0);
        for (int q = 0; q < cnt; ++q) {
            const int64_t *a = tv[q], *b = tv[q] + 3, *cc = tv[q] + 6;
            int64_t mnx = min(a[0], min(b[0], cc[0])), mxx = max(a[0], max(b[0], cc[0]));
            int64_t mny = min(a[1], min(b[1], cc[1])), mxy = max(a[1], max(b[1], cc[1]));
            if (X < mnx || X >= mxx || Y < mny || Y >= mxy) continue;
            const i128 den = (i128)(b[0] - a[0]) * (i128)(cc[1] - a[1]) - (i128)(b[1] - a[1]) * (i128)(cc[0] - a[0]);
            if (den == 0) continue;
            i128 wa, wb, wc;
            const int sa = orient_pert(b[0], b[1], cc[0], cc[1], X, Y, wa);
            const int sb = orient_pert(cc[0], cc[1], a[0], a[1], X, Y, wb);
            const int sc = orient_pert(a[0], a[1], b[0], b[1], X, Y, wc);
            if (!(sa == sb && sb == sc && sa != 0)) continue;
            if (nc >= MAX_CROSS) { overflow = true; continue; }
            S[nc] = wa * (i128)a[2] + wb * (i128)b[2] + wc * (i128)cc[2];
            Dn[nc] = den;
            ++nc;
        }
    }
    if (!active) return;
    if (overflow) atomicExch(err, 1);
    const int64_t plane = (int64_t)nx * ny;
    for (int k = 0; k < nz; ++k) {
        const i128 Z = (i128)Zq[k];
        int par = 0;
        for (int q = 0; q < nc; ++q) par ^= (sgn128(S[q] - Z * Dn[q]) * sgn128(Dn[q]) >= 0) ? 1 : 0;
        inside[(int64_t)i + (int64_t)nx * j + plane * k] = (uint8_t)par;
    }
}

// 2D: one thread per cell; ray along +y over all segments (Vq: nv*2)
__global__ void k_inside2d(int nx, int ny, const int64_t *__restrict__ Xq, const int64_t *__restrict__ Yq,
                           const int64_t *__restrict__ Vq, int64_t ne, const int32_t *__restrict__ segs,
                           uint8_t *__restrict__ inside) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= (int64_t)nx * ny) return;
    const int i = (int)(c % nx), j = (int)(c / nx);
    const int64_t X = Xq[i], Y = Yq[j];
    int par = 0;
    for (int64_t e = 0; e < ne; ++e) {
        const int64_t *a = Vq + 2 * (int64_t)segs[2 * e];
        const int64_t *b = Vq + 2 * (int64_t)segs[2 * e + 1];
        const bool cross = (a[0] <= X && X < b[0]) || (b[0] <= X && X < a[0]);
        if (!cross) continue;
        const i128 dxs = (i128)(b[0] - a[0]);
        const int sd = dxs > 0 ? 1 : -1;
        const i128 num = (i128)(a[1] - Y) * dxs + (i128)(b[1] - a[1]) * (i128)(X - a[0]);
        if (sgn128(num) * sd >= 0) par ^= 1;
    }
    inside[c] = (uint8_t)par;
}

__global__ void k_classify(int nx, int ny, int nz, const uint8_t *__restrict__ ins, uint8_t *__restrict__ type) {
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        if (!ins[c]) { type[c] = FLUID; continue; }
        const int64_t t = c / nx;
        const int i = (int)(c - t * nx), j = (int)(t % ny), k = (int)(t / ny);
        const int64_t sy = nx, sz = (int64_t)nx * ny;
        bool fl = (i > 0 && !ins[c - 1]) || (i < nx - 1 && !ins[c + 1]) || (j > 0 && !ins[c - sy]) ||
                  (j < ny - 1 && !ins[c + sy]) || (k > 0 && !ins[c - sz]) || (k < nz - 1 && !ins[c + sz]);
        type[c] = fl ? GHOST : DEAD;
    }
}

// ordered stream compaction of ghost indices: counts per chunk, one-block
// exclusive scan, ordered write
constexpr int CHUNK = 1024;

__global__ void k_count_types(int64_t n, const uint8_t *__restrict__ type, int64_t *__restrict__ cnt) {
    // cnt[3*b + t] = number of cells of type t in chunk b
    __shared__ int sh[3];
    if (threadIdx.x < 3) sh[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * CHUNK;
    int loc[3] = {0, 0, 0};
    for (int q = threadIdx.x; q < CHUNK; q += blockDim.x) {
        const int64_t c = base + q;
        if (c < n) loc[type[c]]++;
    }
    for (int t = 0; t < 3; ++t) {
        int v = loc[t];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sh[t], v);
    }
    __syncthreads();
    if (threadIdx.x < 3) cnt[3 * (int64_t)blockIdx.x + threadIdx.x] = sh[threadIdx.x];
}

// exclusive scan of the ghost counts (column 1) in one block; totals[0..2]
__global__ void k_scan_counts(int64_t nb, const int64_t *__restrict__ cnt, int64_t *__restrict__ off,
                              int64_t *__restrict__ totals) {
    __shared__ int64_t sh[1024];
    __shared__ int64_t carry;
    __shared__ int64_t tot[3];
    if (threadIdx.x == 0) { carry = 0; tot[0] = tot[1] = tot[2] = 0; }
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t v = b < nb ? cnt[3 * b + 1] : 0;
        if (b < nb) {
            atomicAdd((unsigned long long *)&tot[0], (unsigned long long)cnt[3 * b + 0]);
            atomicAdd((unsigned long long *)&tot[2], (unsigned long long)cnt[3 * b + 2]);
        }
        sh[threadIdx.x] = v;
        __syncthreads();
        // Hillis-Steele inclusive scan
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            int64_t t = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (b < nb) off[b] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += sh[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        totals[0] = tot[0];
        totals[1] = carry;
        totals[2] = tot[2];
    }
}

__global__ void k_write_ghosts(int64_t n, const uint8_t *__restrict__ type, const int64_t *__restrict__ off,
                               int64_t *__restrict__ gidx) {
    // one block of 1024 threads per chunk: ballot-ordered write
    __shared__ int wsum[32];
    const int64_t c = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
    const bool g = c < n && type[c] == GHOST;
    const unsigned bal = __ballot_sync(0xffffffffu, g);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int q = 0; q < w; ++q) before += wsum[q];
    if (g) gidx[off[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u))] = c;
}

// counts of set flags per chunk, in column 1 of the 3-column layout
__global__ void k_count_flags(int64_t n, const uint8_t *__restrict__ f, int64_t *__restrict__ cnt) {
    __shared__ int sh;
    if (threadIdx.x == 0) sh = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * CHUNK;
    int loc = 0;
    for (int q = threadIdx.x; q < CHUNK; q += blockDim.x) {
        const int64_t c = base + q;
        if (c < n && f[c]) ++loc;
    }
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sh, loc);
    __syncthreads();
    if (threadIdx.x == 0) {
        cnt[3 * (int64_t)blockIdx.x + 0] = 0;
        cnt[3 * (int64_t)blockIdx.x + 1] = sh;
        cnt[3 * (int64_t)blockIdx.x + 2] = 0;
    }
}

__global__ void k_write_flags(int64_t n, const uint8_t *__restrict__ f, const int64_t *__restrict__ off,
                              int64_t *__restrict__ out) {
    __shared__ int wsum[32];
    const int64_t c = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
    const bool g = c < n && f[c];
    const unsigned bal = __ballot_sync(0xffffffffu, g);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int q = 0; q < w; ++q) before += wsum[q];
    if (g) out[off[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u))] = c;
}

// ascending list of the cells whose flag is set (allocated here)
ibm_status compact_flags(Ctx *c, const uint8_t *flags, int64_t **out, int64_t *count) {
    const int64_t nb = (c->N + CHUNK - 1) / CHUNK;
    int64_t *cnt = (int64_t *)dev_alloc(c, sizeof(int64_t) * 3 * nb);
    int64_t *off = (int64_t *)dev_alloc(c, sizeof(int64_t) * nb);
    int64_t *tot = (int64_t *)dev_alloc(c, sizeof(int64_t) * 4);
    if (!cnt || !off || !tot) return c->fail(IBM_ERR_OOM, "compaction scratch allocation failed");
    ++c->nlaunch, k_count_flags<<<(unsigned)nb, 256, 0, c->s>>>(c->N, flags, cnt);
    ++c->nlaunch, k_scan_counts<<<1, 1024, 0, c->s>>>(nb, cnt, off, tot);
    IBM_LAUNCHED(c);
    int64_t htot[3] = {0, 0, 0};
    IBM_CUDA(c, cudaMemcpyAsync(htot, tot, sizeof(int64_t) * 3, cudaMemcpyDeviceToHost, c->s));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    *count = htot[1];
    *out = (int64_t *)dev_alloc(c, sizeof(int64_t) * (htot[1] > 0 ? htot[1] : 1));
    if (!*out) return c->fail(IBM_ERR_OOM, "compaction output allocation failed");
    if (htot[1] > 0) {
        ++c->nlaunch, k_write_flags<<<(unsigned)nb, CHUNK, 0, c->s>>>(c->N, flags, off, *out);
        IBM_LAUNCHED(c);
    }
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    dev_free(c, cnt);
    dev_free(c, off);
    dev_free(c, tot);
    return IBM_OK;
}

// ---------------------------------------------------------------------------
// closest points and weights (must match the oracle operation for operation)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double dot3(const double *u, const double *v) { return (u[0] * v[0] + u[1] * v[1]) + u[2] * v[2]; }

// closest point on triangle abc to p by the Voronoi-region method
// (Ericson, Real-Time Collision Detection, 2005, Sec. 5.1.5)
__device__ void closest_on_tri(const double *p, const double *a, const double *b, const double *c, double *q) {
    double ab[3], ac[3], ap[3], bp[3], cp[3];
    for (int d = 0; d < 3; ++d) { ab[d] = b[d] - a[d]; ac[d] = c[d] - a[d]; ap[d] = p[d] - a[d]; }
    const double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) { for (int d = 0; d < 3; ++d) q[d] = a[d]; return; }
    for (int d = 0; d < 3; ++d) bp[d] = p[d] - b[d];
    const double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) { for (int d = 0; d < 3; ++d) q[d] = b[d]; return; }
    const double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        const double v = d1 / (d1 - d3);
        for (int d = 0; d < 3; ++d) q[d] = a[d] + v * ab[d];
        return;
    }
    for (int d = 0; d < 3; ++d) cp[d] = p[d] - c[d];
    const double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) { for (int d = 0; d < 3; ++d) q[d] = c[d]; return; }
    const double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        const double w = d2 / (d2 - d6);
        for (int d = 0; d < 3; ++d) q[d] = a[d] + w * ac[d];
        return;
    }
    const double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
        const double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int d = 0; d < 3; ++d) q[d] = b[d] + w * (c[d] - b[d]);
        return;
    }
    const double den = 1.0 / ((va + vb) + vc);
    const double v = vb * den, w = vc * den;
    for (int d = 0; d < 3; ++d) q[d] = (a[d] + ab[d] * v) + ac[d] * w;
}

__device__ void closest_on_seg(const double *p, const double *a, const double *b, double *q) {
    const double ab0 = b[0] - a[0], ab1 = b[1] - a[1];
    const double ap0 = p[0] - a[0], ap1 = p[1] - a[1];
    double t = (ap0 * ab0 + ap1 * ab1) / (ab0 * ab0 + ab1 * ab1);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    q[0] = a[0] + t * ab0;
    q[1] = a[1] + t * ab1;
    q[2] = 0.0;
}

// per element: a point on it (the centroid) and its bounding box, 9 doubles
// (centroid, low corner, high corner)
__global__ void k_elem_boxes(int ndim, int64_t ne, const double *__restrict__ verts, const int32_t *__restrict__ elems,
                             double *__restrict__ box) {
    const int nvpe = ndim == 2 ? 2 : 3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, s[3] = {0, 0, 0};
        for (int k = 0; k < nvpe; ++k) {
            const int64_t v = elems[nvpe * e + k];
            for (int d = 0; d < 3; ++d) {
                const double x = verts[3 * v + d];
                lo[d] = fmin(lo[d], x);
                hi[d] = fmax(hi[d], x);
                s[d] += x;
            }
        }
        for (int d = 0; d < 3; ++d) {
            box[9 * e + d] = s[d] / nvpe;
            box[9 * e + 3 + d] = lo[d];
            box[9 * e + 6 + d] = hi[d];
        }
    }
}

// body intercept: one warp per ghost (four per block), elements staged
// through shared memory and shared out over the lanes. The closest point is
// the one of the first element (in element order) with the smallest squared
// distance, as in a search over every element: each lane keeps the first
// minimum of its elements (visited in element order) and the warp takes the
// smallest distance, the lowest element on ties. Elements that cannot hold
// the minimum are skipped: with U the smallest squared distance to an
// element's centroid (a point of the element, so an upper bound of the
// minimum) and b the lane's best so far, an element whose bounding box lies
// farther than min(U, b) (1 + 1e-6) is farther than the minimum beyond any
// rounding of the evaluated distances, and one the full search would not take.
constexpr int ELEM_TILE = 128;
constexpr int BI_WARPS = 4;

__global__ void __launch_bounds__(128) k_body_intercept(int ndim, int nx, int ny, const double *__restrict__ xc,
                                                        const double *__restrict__ yc, const double *__restrict__ zc,
                                                        int64_t ng, const int64_t *__restrict__ gidx,
                                                        const double *__restrict__ verts, int64_t ne,
                                                        const int32_t *__restrict__ elems,
                                                        const double *__restrict__ box, double *__restrict__ bi) {
    __shared__ double ev[ELEM_TILE][9];
    __shared__ double eb[ELEM_TILE][9];
    const int lane = threadIdx.x & 31;
    const int64_t g = blockIdx.x * (int64_t)BI_WARPS + (threadIdx.x >> 5);
    const bool active = g < ng;
    double p[3] = {0, 0, 0};
    if (active) {
        const int64_t c = gidx[g];
        const int64_t t = c / nx;
        const int i = (int)(c - t * nx), j = (int)(t % ny), k = (int)(t / ny);
        p[0] = xc[i];
        p[1] = yc[j];
        p[2] = ndim == 2 ? 0.0 : zc[k];
    }
    const int nvpe = ndim == 2 ? 2 : 3;
    // upper bound from the centroids
    double U = INFINITY;
    for (int64_t e0 = 0; e0 < ne; e0 += ELEM_TILE) {
        __syncthreads();
        for (int r = threadIdx.x; r < ELEM_TILE * 3; r += blockDim.x) {
            const int64_t e = e0 + r / 3;
            if (e < ne) eb[r / 3][r % 3] = box[9 * e + r % 3];
        }
        __syncthreads();
        if (!active) continue;
        const int cnt = (int)min((int64_t)ELEM_TILE, ne - e0);
        for (int r = lane; r < cnt; r += 32) {
            const double d0 = eb[r][0] - p[0], d1 = eb[r][1] - p[1], d2 = eb[r][2] - p[2];
            U = fmin(U, d0 * d0 + d1 * d1 + d2 * d2);
        }
    }
    for (int o = 16; o > 0; o >>= 1) U = fmin(U, __shfl_xor_sync(0xffffffffu, U, o));
    double best = INFINITY, q[3] = {0, 0, 0};
    int64_t bidx = ne;
    for (int64_t e0 = 0; e0 < ne; e0 += ELEM_TILE) {
        __syncthreads();
        for (int r = threadIdx.x; r < ELEM_TILE * nvpe; r += blockDim.x) {
            const int64_t e = e0 + r / nvpe;
            const int corner = r % nvpe;
            if (e < ne) {
                const int64_t v = elems[nvpe * e + corner];
                ev[r / nvpe][3 * corner + 0] = verts[3 * v + 0];
                ev[r / nvpe][3 * corner + 1] = verts[3 * v + 1];
                ev[r / nvpe][3 * corner + 2] = verts[3 * v + 2];
            }
        }
        for (int r = threadIdx.x; r < ELEM_TILE * 6; r += blockDim.x) {
            const int64_t e = e0 + r / 6;
            if (e < ne) eb[r / 6][3 + r % 6] = box[9 * e + 3 + r % 6];
        }
        __syncthreads();
        if (!active) continue;
        const int cnt = (int)min((int64_t)ELEM_TILE, ne - e0);
        for (int r = lane; r < cnt; r += 32) {
            double ad = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double o = fmax(fmax(eb[r][3 + d] - p[d], p[d] - eb[r][6 + d]), 0.0);
                ad += o * o;
            }
            if (ad > fmin(U, best) * (1.0 + 1e-6)) continue;
            double qq[3];
            if (ndim == 2) closest_on_seg(p, ev[r], ev[r] + 3, qq);
            else closest_on_tri(p, ev[r], ev[r] + 3, ev[r] + 6, qq);
            double dv[3] = {qq[0] - p[0], qq[1] - p[1], qq[2] - p[2]};
            const double dd = dot3(dv, dv);
            if (dd < best) {
                best = dd;
                bidx = e0 + r;
                q[0] = qq[0]; q[1] = qq[1]; q[2] = qq[2];
            }
        }
    }
    // the warp's first minimum
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, (long long)bidx, o);
        const double o0 = __shfl_xor_sync(0xffffffffu, q[0], o);
        const double o1 = __shfl_xor_sync(0xffffffffu, q[1], o);
        const double o2 = __shfl_xor_sync(0xffffffffu, q[2], o);
        if (ob < best || (ob == best && oi < bidx)) {
            best = ob;
            bidx = oi;
            q[0] = o0; q[1] = o1; q[2] = o2;
        }
    }
    if (active && lane == 0) {
        bi[3 * g + 0] = q[0];
        bi[3 * g + 1] = q[1];
        bi[3 * g + 2] = q[2];
    }
}

// element boxes of the current vertex positions (scratch owned by the caller)
static ibm_status elem_boxes(Ctx *c, double **box) {
    *box = (double *)dev_alloc(c, sizeof(double) * 9 * (size_t)(c->ne > 0 ? c->ne : 1));
    if (!*box) return c->fail(IBM_ERR_OOM, "element box allocation failed");
    ++c->nlaunch, k_elem_boxes<<<(unsigned)((c->ne + 255) / 256), 256, 0, c->s>>>(c->ndim, c->ne, c->d_verts, c->d_elems, *box);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

// LU with partial pivoting; 1 when a pivot is below 1e-12 max|M|
__device__ int lu_solve(int n, double *M, double *r, double *x) {
    double scale = 0.0;
    for (int i = 0; i < n * n; ++i) { const double v = fabs(M[i]); if (v > scale) scale = v; }
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(M[k * n + k]);
        for (int i = k + 1; i < n; ++i) { const double v = fabs(M[i * n + k]); if (v > best) { best = v; p = i; } }
        if (best < 1e-12 * scale) return 1;
        if (p != k) {
            for (int j = 0; j < n; ++j) { const double t = M[k * n + j]; M[k * n + j] = M[p * n + j]; M[p * n + j] = t; }
            const double t = r[k]; r[k] = r[p]; r[p] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            const double l = M[i * n + k] / M[k * n + k];
            for (int j = k + 1; j < n; ++j) M[i * n + j] = M[i * n + j] - l * M[k * n + j];
            r[i] = r[i] - l * r[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = r[i];
        for (int j = i + 1; j < n; ++j) s = s - M[i * n + j] * x[j];
        x[i] = s / M[i * n + i];
    }
    return 0;
}

__device__ void basis(int ndim, double x, double y, double z, double *b) {
    if (ndim == 2) { b[0] = 1.0; b[1] = x; b[2] = y; b[3] = x * y; return; }
    b[0] = 1.0; b[1] = x; b[2] = y; b[3] = z;
    b[4] = x * y; b[5] = y * z; b[6] = z * x; b[7] = (x * y) * z;
}

__device__ void basis_dn(int ndim, double x, double y, double z, const double *nrm, double hx, double hy, double hz,
                         double *g) {
    const double ax = nrm[0] / hx, ay = nrm[1] / hy;
    if (ndim == 2) { g[0] = 0.0; g[1] = ax; g[2] = ay; g[3] = ax * y + ay * x; return; }
    const double az = nrm[2] / hz;
    g[0] = 0.0; g[1] = ax; g[2] = ay; g[3] = az;
    g[4] = ax * y + ay * x;
    g[5] = ay * z + az * y;
    g[6] = ax * z + az * x;
    g[7] = (ax * (y * z) + ay * (x * z)) + az * (x * y);
}

__device__ int count_le(const double *c, int n, double v) {
    int lo = 0, hi = n;
    while (lo < hi) { const int mid = (lo + hi) / 2; if (c[mid] <= v) lo = mid + 1; else hi = mid; }
    return lo;
}

struct TabOut {
    double *bi, *nrm, *ip, *dist, *wv, *wp, *bv, *bp;
    int64_t *base, *sidx;
    uint8_t *kind, *cmask;
};

// normal, image point, base cell, corners, kind and weights; one thread per ghost
__global__ void __launch_bounds__(64) k_ghost_tables(int ndim, int nx, int ny, int nz, const double *__restrict__ xc,
                                                     const double *__restrict__ yc, const double *__restrict__ zc,
                                                     const double *__restrict__ dx, const double *__restrict__ dy,
                                                     const double *__restrict__ dz, const uint8_t *__restrict__ type,
                                                     int64_t ng, const int64_t *__restrict__ gidx, TabOut o) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int nc = ndim == 2 ? 4 : 8;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    const int64_t c = gidx[g];
    const int64_t tq = c / nx;
    const int i = (int)(c - tq * nx), j = (int)(tq % ny), k = (int)(tq / ny);
    const double p[3] = {xc[i], yc[j], ndim == 2 ? 0.0 : zc[k]};
    const double q[3] = {o.bi[3 * g], o.bi[3 * g + 1], o.bi[3 * g + 2]};
    const double dv[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
    const double d = sqrt(dot3(dv, dv));
    double hloc = dx[i] < dy[j] ? dx[i] : dy[j];
    if (ndim == 3 && dz[k] < hloc) hloc = dz[k];
    const bool degenerate = !(d >= 1e-9 * hloc);
    double n[3] = {0, 0, 0}, x[3];
    if (!degenerate) {
        n[0] = dv[0] / d; n[1] = dv[1] / d; n[2] = dv[2] / d;
        x[0] = 2.0 * q[0] - p[0]; x[1] = 2.0 * q[1] - p[1]; x[2] = 2.0 * q[2] - p[2];
    } else {
        x[0] = p[0]; x[1] = p[1]; x[2] = p[2];
    }
    if (ndim == 2) x[2] = 0.0;
    for (int a = 0; a < 3; ++a) { o.nrm[3 * g + a] = n[a]; o.ip[3 * g + a] = x[a]; }
    o.dist[g] = d;
    int i0 = count_le(xc, nx, x[0]) - 1, j0 = count_le(yc, ny, x[1]) - 1, k0 = 0;
    i0 = i0 < 0 ? 0 : (i0 > nx - 2 ? nx - 2 : i0);
    j0 = j0 < 0 ? 0 : (j0 > ny - 2 ? ny - 2 : j0);
    if (ndim == 3) {
        k0 = count_le(zc, nz, x[2]) - 1;
        k0 = k0 < 0 ? 0 : (k0 > nz - 2 ? nz - 2 : k0);
    }
    o.base[g] = (int64_t)i0 + sy * j0 + sz * k0;
    const double hx = xc[i0 + 1] - xc[i0], hy = yc[j0 + 1] - yc[j0];
    const double hz = ndim == 3 ? zc[k0 + 1] - zc[k0] : 1.0;
    int64_t cidx[8];
    int self = -1;
    bool dead = false;
    uint8_t msk = 0;
    for (int m = 0; m < nc; ++m) {
        const int di = m & 1, dj = (m >> 1) & 1, dk = (m >> 2) & 1;
        cidx[m] = (int64_t)(i0 + di) * sx + (int64_t)(j0 + dj) * sy + (int64_t)(k0 + dk) * sz;
        const uint8_t t = type[cidx[m]];
        if (t != FLUID) msk |= (uint8_t)(1u << m);
        if (cidx[m] == c) self = m;
        else if (t == DEAD) dead = true;
    }
    o.cmask[g] = msk;
    int kd = degenerate ? 2 : (dead ? 2 : (self >= 0 ? 1 : 0));
    double xv[8], xp[8];
    if (kd != 2) {
        double bIP[8], bBI[8], gBI[8], Mv[64], Mp[64], rv[8], rp[8];
        const double xi = (x[0] - xc[i0]) / hx, et = (x[1] - yc[j0]) / hy;
        const double ze = ndim == 3 ? (x[2] - zc[k0]) / hz : 0.0;
        basis(ndim, xi, et, ze, bIP);
        if (kd == 1) {
            const double bxi = (q[0] - xc[i0]) / hx, bet = (q[1] - yc[j0]) / hy;
            const double bze = ndim == 3 ? (q[2] - zc[k0]) / hz : 0.0;
            basis(ndim, bxi, bet, bze, bBI);
            basis_dn(ndim, bxi, bet, bze, n, hx, hy, hz, gBI);
        }
        for (int m = 0; m < nc; ++m) {
            double row[8];
            if (m == self) {
                for (int r = 0; r < nc; ++r) row[r] = bBI[r];
            } else {
                basis(ndim, (double)(m & 1), (double)((m >> 1) & 1), (double)((m >> 2) & 1), row);
            }
            for (int r = 0; r < nc; ++r) Mv[r * nc + m] = row[r];
            if (m == self)
                for (int r = 0; r < nc; ++r) row[r] = gBI[r];
            for (int r = 0; r < nc; ++r) Mp[r * nc + m] = row[r];
        }
        for (int r = 0; r < nc; ++r) { rv[r] = bIP[r]; rp[r] = bIP[r]; }
        const int s1 = lu_solve(nc, Mv, rv, xv);
        const int s2 = lu_solve(nc, Mp, rp, xp);
        if (s1 || s2) kd = 2;
    }
    o.kind[g] = (uint8_t)kd;
    double *WV = o.wv + 8 * g, *WP = o.wp + 8 * g;
    int64_t *SI = o.sidx + 8 * g;
    o.bv[g] = 0.0;
    o.bp[g] = 0.0;
    if (kd != 2) {
        for (int m = 0; m < 8; ++m) {
            if (m < nc && m != self) { SI[m] = cidx[m]; WV[m] = xv[m]; WP[m] = xp[m]; }
            else { SI[m] = c; WV[m] = 0.0; WP[m] = 0.0; }
        }
        if (self >= 0) { o.bv[g] = xv[self]; o.bp[g] = xp[self]; }
    } else {
        int64_t pick = -1;
        double bd = INFINITY;
        for (int m = 0; m < nc; ++m) {
            if (type[cidx[m]] != FLUID) continue;
            const int ci = i0 + (m & 1), cj = j0 + ((m >> 1) & 1), ck = k0 + ((m >> 2) & 1);
            const double e0 = xc[ci] - x[0], e1 = yc[cj] - x[1], e2 = ndim == 3 ? zc[ck] - x[2] : 0.0;
            const double dd = (e0 * e0 + e1 * e1) + e2 * e2;
            if (dd < bd) { bd = dd; pick = cidx[m]; }
        }
        if (pick < 0) {
            int64_t nb[6] = {-1, -1, -1, -1, -1, -1};
            if (i > 0) nb[0] = c - sx;
            if (i < nx - 1) nb[1] = c + sx;
            if (j > 0) nb[2] = c - sy;
            if (j < ny - 1) nb[3] = c + sy;
            if (ndim == 3 && k > 0) nb[4] = c - sz;
            if (ndim == 3 && k < nz - 1) nb[5] = c + sz;
            for (int t = 0; t < 6 && pick < 0; ++t)
                if (nb[t] >= 0 && type[nb[t]] == FLUID) pick = nb[t];
        }
        for (int m = 0; m < 8; ++m) { SI[m] = pick; WV[m] = 0.0; WP[m] = 0.0; }
        WV[0] = 1.0;
        WP[0] = 1.0;
    }
}

// ---------------------------------------------------------------------------
// moving bodies (Section 2.2): body velocity and fresh cells
// ---------------------------------------------------------------------------

struct Motion {
    double U[3], w[3], c[3];
};

// U + Omega x (p - centre), the operations of the oracle's body_velocity
__global__ void k_body_velocity(int64_t n, const double *__restrict__ pts, Motion m, double *__restrict__ out) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n) return;
    const double r0 = pts[3 * g] - m.c[0], r1 = pts[3 * g + 1] - m.c[1], r2 = pts[3 * g + 2] - m.c[2];
    out[3 * g + 0] = m.U[0] + (m.w[1] * r2 - m.w[2] * r1);
    out[3 * g + 1] = m.U[1] + (m.w[2] * r0 - m.w[0] * r2);
    out[3 * g + 2] = m.U[2] + (m.w[0] * r1 - m.w[1] * r0);
}

// Fresh cell (a FLUID cell that was not FLUID before the move): the
// trilinear fit on the lattice cell of centres with the fresh cell FC as a
// corner, extending towards n = (FC - BI) / |FC - BI| along each axis
// (clamped into the grid), with FC's row replaced by the Dirichlet row at
// the body intercept, evaluated at FC: u_FC = sum_{m != FC} w_m u_m + wb u_BI.
// Other corners must be FLUID (fresh ones are implicit unknowns); a GHOST or
// DEAD corner, a singular system or FC on the surface gives kind 2,
// u_FC = u_BI. One thread per fresh cell; the operations of the oracle's
// orc_fresh_tables in its order.
__global__ void __launch_bounds__(64) k_fresh_tables(int ndim, int nx, int ny, int nz, const double *__restrict__ xc,
                                                     const double *__restrict__ yc, const double *__restrict__ zc,
                                                     const double *__restrict__ dx, const double *__restrict__ dy,
                                                     const double *__restrict__ dz, const uint8_t *__restrict__ type,
                                                     int64_t nf, const int64_t *__restrict__ fidx,
                                                     const double *__restrict__ bi, uint8_t *__restrict__ kind,
                                                     int64_t *__restrict__ sidx, double *__restrict__ w,
                                                     double *__restrict__ wb) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int nc = ndim == 2 ? 4 : 8;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    const int64_t c = fidx[f];
    const int64_t tq = c / nx;
    const int i = (int)(c - tq * nx), j = (int)(tq % ny), k = (int)(tq / ny);
    const double p[3] = {xc[i], yc[j], ndim == 2 ? 0.0 : zc[k]};
    const double q[3] = {bi[3 * f], bi[3 * f + 1], bi[3 * f + 2]};
    const double dv[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    const double d = sqrt(dot3(dv, dv));
    double hloc = dx[i] < dy[j] ? dx[i] : dy[j];
    if (ndim == 3 && dz[k] < hloc) hloc = dz[k];
    int kd = !(d >= 1e-9 * hloc) ? 2 : 1;
    double n[3] = {0, 0, 0};
    if (kd == 1) { n[0] = dv[0] / d; n[1] = dv[1] / d; n[2] = dv[2] / d; }
    int i0 = n[0] >= 0.0 ? i : i - 1, j0 = n[1] >= 0.0 ? j : j - 1, k0 = 0;
    i0 = i0 < 0 ? 0 : (i0 > nx - 2 ? nx - 2 : i0);
    j0 = j0 < 0 ? 0 : (j0 > ny - 2 ? ny - 2 : j0);
    if (ndim == 3) {
        k0 = n[2] >= 0.0 ? k : k - 1;
        k0 = k0 < 0 ? 0 : (k0 > nz - 2 ? nz - 2 : k0);
    }
    int64_t cidx[8];
    int self = -1;
    for (int m = 0; m < nc; ++m) {
        const int di = m & 1, dj = (m >> 1) & 1, dk = (m >> 2) & 1;
        cidx[m] = (int64_t)(i0 + di) * sx + (int64_t)(j0 + dj) * sy + (int64_t)(k0 + dk) * sz;
        if (cidx[m] == c) self = m;
        else if (type[cidx[m]] != FLUID) kd = 2;
    }
    double xw[8];
    if (kd == 1) {
        const double hx = xc[i0 + 1] - xc[i0], hy = yc[j0 + 1] - yc[j0];
        const double hz = ndim == 3 ? zc[k0 + 1] - zc[k0] : 1.0;
        const double bxi = (q[0] - xc[i0]) / hx, bet = (q[1] - yc[j0]) / hy;
        const double bze = ndim == 3 ? (q[2] - zc[k0]) / hz : 0.0;
        double bBI[8], bFC[8], M[64], r[8];
        basis(ndim, bxi, bet, bze, bBI);
        basis(ndim, (double)(self & 1), (double)((self >> 1) & 1), (double)((self >> 2) & 1), bFC);
        for (int m = 0; m < nc; ++m) {
            double row[8];
            if (m == self) {
                for (int t = 0; t < nc; ++t) row[t] = bBI[t];
            } else {
                basis(ndim, (double)(m & 1), (double)((m >> 1) & 1), (double)((m >> 2) & 1), row);
            }
            for (int t = 0; t < nc; ++t) M[t * nc + m] = row[t];
        }
        for (int t = 0; t < nc; ++t) r[t] = bFC[t];
        if (lu_solve(nc, M, r, xw)) kd = 2;
    }
    kind[f] = (uint8_t)kd;
    int64_t *SI = sidx + 8 * f;
    double *W = w + 8 * f;
    if (kd == 1) {
        for (int m = 0; m < 8; ++m) {
            if (m < nc && m != self) { SI[m] = cidx[m]; W[m] = xw[m]; }
            else { SI[m] = c; W[m] = 0.0; }
        }
        wb[f] = xw[self];
    } else {
        for (int m = 0; m < 8; ++m) { SI[m] = c; W[m] = 0.0; }
        wb[f] = 1.0;
    }
}

__global__ void k_kind_counts(int64_t ng, const uint8_t *__restrict__ kind, unsigned long long *__restrict__ cnt) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < ng) atomicAdd(&cnt[kind[g]], 1ull);
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------

static ibm_status ensure_ghost_capacity(Ctx *c, int64_t ng) {
    if (ng <= c->ng_cap && c->gidx) return IBM_OK;
    const int64_t cap = ng < 1 ? 1 : ng;
    auto A = [&](size_t bytes) { return dev_alloc(c, bytes); };
    void *old[] = {c->gidx, c->base, c->sidx, c->bi, c->nrm, c->ipt, c->dist, c->wv, c->wp, c->bv, c->bp, c->kind, c->cmask, c->gtmp};
    for (void *p : old)
        if (p) dev_free(c, p);
    c->gidx = (int64_t *)A(sizeof(int64_t) * cap);
    c->base = (int64_t *)A(sizeof(int64_t) * cap);
    c->sidx = (int64_t *)A(sizeof(int64_t) * 8 * cap);
    c->bi = (double *)A(sizeof(double) * 3 * cap);
    c->nrm = (double *)A(sizeof(double) * 3 * cap);
    c->ipt = (double *)A(sizeof(double) * 3 * cap);
    c->dist = (double *)A(sizeof(double) * cap);
    c->wv = (double *)A(sizeof(double) * 8 * cap);
    c->wp = (double *)A(sizeof(double) * 8 * cap);
    c->bv = (double *)A(sizeof(double) * cap);
    c->bp = (double *)A(sizeof(double) * cap);
    c->kind = (uint8_t *)A(cap);
    c->cmask = (uint8_t *)A(cap);
    c->gtmp = (double *)A(sizeof(double) * 3 * cap);
    if (!c->gidx || !c->base || !c->sidx || !c->bi || !c->nrm || !c->ipt || !c->dist || !c->wv || !c->wp || !c->bv ||
        !c->bp || !c->kind || !c->cmask || !c->gtmp)
        return c->fail(IBM_ERR_OOM, "ghost table allocation failed");
    c->ng_cap = cap;
    return IBM_OK;
}

ibm_status geom_body_velocity(Ctx *c, int64_t n, const double *pts, double *out) {
    if (n <= 0) return IBM_OK;
    Motion m;
    for (int a = 0; a < 3; ++a) {
        m.U[a] = c->motion[a];
        m.w[a] = c->motion[3 + a];
        m.c[a] = c->motion[6 + a];
    }
    ++c->nlaunch, k_body_velocity<<<(unsigned)((n + 255) / 256), 256, 0, c->s>>>(n, pts, m, out);
    IBM_LAUNCHED(c);
    return IBM_OK;
}

ibm_status geom_fresh_tables(Ctx *c, int64_t nf, const int64_t *fidx, double *bi, uint8_t *kind, int64_t *sidx,
                             double *w, double *wb) {
    if (nf <= 0) return IBM_OK;
    double *box = nullptr;
    IBM_TRY(elem_boxes(c, &box));
    ++c->nlaunch, k_body_intercept<<<(unsigned)((nf + BI_WARPS - 1) / BI_WARPS), 128, 0, c->s>>>(c->ndim, c->nx, c->ny, c->xc, c->yc, c->zc, nf,
                                                                                  fidx, c->d_verts, c->ne, c->d_elems, box, bi);
    IBM_LAUNCHED(c);
    ++c->nlaunch, k_fresh_tables<<<(unsigned)((nf + 63) / 64), 64, 0, c->s>>>(c->ndim, c->nx, c->ny, c->nz, c->xc, c->yc, c->zc,
                                                                             c->dx, c->dy, c->dz, c->type, nf, fidx, bi,
                                                                             kind, sidx, w, wb);
    IBM_LAUNCHED(c);
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    dev_free(c, box);
    return IBM_OK;
}

ibm_status geom_classify(Ctx *c) {
    const int nd = c->ndim;
    // quantisation: lo per axis, s = 2^(30 - e) from the largest extent
    double lo[3], hi[3];
    const std::vector<double> *F[3] = {&c->hxf, &c->hyf, &c->hzf};
    for (int a = 0; a < nd; ++a) {
        lo[a] = (*F[a]).front();
        hi[a] = (*F[a]).back();
        for (int64_t v = 0; v < c->nv; ++v) {
            const double x = c->verts[3 * v + a];
            if (x < lo[a]) lo[a] = x;
            if (x > hi[a]) hi[a] = x;
        }
    }
    double E = 0.0;
    for (int a = 0; a < nd; ++a) E = (hi[a] - lo[a]) > E ? (hi[a] - lo[a]) : E;
    int e2 = 0;
    frexp(E, &e2);
    const double s = ldexp(1.0, 30 - e2);
    const int64_t nmax = c->nx > c->ny ? (c->nx > c->nz ? c->nx : c->nz) : (c->ny > c->nz ? c->ny : c->nz);
    int64_t *Cq = (int64_t *)dev_alloc(c, sizeof(int64_t) * 3 * nmax);
    int *derr = (int *)dev_alloc(c, sizeof(int) * 4);
    int64_t *vq = (int64_t *)dev_alloc(c, sizeof(int64_t) * 3 * (c->nv > 0 ? c->nv : 1));
    if (!Cq || !derr || !vq) return c->fail(IBM_ERR_OOM, "classification scratch allocation failed");
    IBM_CUDA(c, cudaMemsetAsync(derr, 0, sizeof(int) * 4, c->s));
    const double *cen[3] = {c->xc, c->yc, c->zc};
    const int nn[3] = {c->nx, c->ny, c->nz};
    for (int a = 0; a < nd; ++a) {
        ++c->nlaunch, k_quantize<<<(nn[a] + 255) / 256, 256, 0, c->s>>>(cen[a], nn[a], lo[a], s, Cq + a * nmax);
        IBM_LAUNCHED(c);
    }
    // vertices: q[v*nd + a] = rint((x - lo[a]) * s)
    ++c->nlaunch, k_quantize_verts<<<(unsigned)((c->nv + 255) / 256), 256, 0, c->s>>>(c->d_verts, c->nv, nd, lo[0], lo[1],
                                                                        nd == 3 ? lo[2] : 0.0, s, vq);
    IBM_LAUNCHED(c);
    if (nd == 3) {
        dim3 grid((unsigned)c->ny, (unsigned)((c->nx + 127) / 128));
        ++c->nlaunch, k_inside3d<<<grid, 128, 0, c->s>>>(c->nx, c->ny, c->nz, Cq, Cq + nmax, Cq + 2 * nmax, vq, c->ne, c->d_elems,
                                           c->inside, derr);
    } else {
        const int64_t n = (int64_t)c->nx * c->ny;
        ++c->nlaunch, k_inside2d<<<(unsigned)((n + 255) / 256), 256, 0, c->s>>>(c->nx, c->ny, Cq, Cq + nmax, vq, c->ne, c->d_elems,
                                                                  c->inside);
    }
    IBM_LAUNCHED(c);
    ++c->nlaunch, k_classify<<<(unsigned)((c->N + 255) / 256 > 152 * 64 ? 152 * 64 : (c->N + 255) / 256), 256, 0, c->s>>>(
        c->nx, c->ny, c->nz, c->inside, c->type);
    IBM_LAUNCHED(c);
    // compaction
    const int64_t nb = (c->N + CHUNK - 1) / CHUNK;
    int64_t *cnt = (int64_t *)dev_alloc(c, sizeof(int64_t) * 3 * nb);
    int64_t *off = (int64_t *)dev_alloc(c, sizeof(int64_t) * nb);
    int64_t *tot = (int64_t *)dev_alloc(c, sizeof(int64_t) * 4);
    if (!cnt || !off || !tot) return c->fail(IBM_ERR_OOM, "compaction scratch allocation failed");
    ++c->nlaunch, k_count_types<<<(unsigned)nb, 256, 0, c->s>>>(c->N, c->type, cnt);
    ++c->nlaunch, k_scan_counts<<<1, 1024, 0, c->s>>>(nb, cnt, off, tot);
    IBM_LAUNCHED(c);
    int64_t htot[4] = {0, 0, 0, 0};
    int herr[4] = {0, 0, 0, 0};
    IBM_CUDA(c, cudaMemcpyAsync(htot, tot, sizeof(int64_t) * 3, cudaMemcpyDeviceToHost, c->s));
    IBM_CUDA(c, cudaMemcpyAsync(herr, derr, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->s));
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    if (herr[0]) return c->fail(IBM_ERR_MESH, "a grid column crosses the surface more than 64 times");
    c->n_fluid = htot[0];
    c->ng = htot[1];
    c->n_dead = htot[2];
    IBM_TRY(ensure_ghost_capacity(c, c->ng));
    if (c->ng > 0) {
        ++c->nlaunch, k_write_ghosts<<<(unsigned)nb, CHUNK, 0, c->s>>>(c->N, c->type, off, c->gidx);
        IBM_LAUNCHED(c);
        const unsigned gb = (unsigned)((c->ng + BI_WARPS - 1) / BI_WARPS);
        double *box = nullptr;
        IBM_TRY(elem_boxes(c, &box));
        ++c->nlaunch, k_body_intercept<<<gb, 128, 0, c->s>>>(nd, c->nx, c->ny, c->xc, c->yc, c->zc, c->ng, c->gidx, c->d_verts,
                                               c->ne, c->d_elems, box, c->bi);
        IBM_LAUNCHED(c);
        IBM_CUDA(c, cudaStreamSynchronize(c->s));
        dev_free(c, box);
        TabOut o{c->bi, c->nrm, c->ipt, c->dist, c->wv, c->wp, c->bv, c->bp, c->base, c->sidx, c->kind, c->cmask};
        ++c->nlaunch, k_ghost_tables<<<(unsigned)((c->ng + 63) / 64), 64, 0, c->s>>>(nd, c->nx, c->ny, c->nz, c->xc, c->yc, c->zc,
                                                                       c->dx, c->dy, c->dz, c->type, c->ng, c->gidx, o);
        IBM_LAUNCHED(c);
        unsigned long long *kc = (unsigned long long *)tot;
        IBM_CUDA(c, cudaMemsetAsync(kc, 0, sizeof(unsigned long long) * 3, c->s));
        ++c->nlaunch, k_kind_counts<<<(unsigned)((c->ng + 255) / 256), 256, 0, c->s>>>(c->ng, c->kind, kc);
        IBM_LAUNCHED(c);
        unsigned long long hk[3] = {0, 0, 0};
        IBM_CUDA(c, cudaMemcpyAsync(hk, kc, sizeof(hk), cudaMemcpyDeviceToHost, c->s));
        IBM_CUDA(c, cudaStreamSynchronize(c->s));
        for (int q = 0; q < 3; ++q) c->n_kind[q] = (int64_t)hk[q];
    } else {
        c->n_kind[0] = c->n_kind[1] = c->n_kind[2] = 0;
    }
    c->gh = GhostDev{c->ng, c->gidx, c->sidx, c->wv, c->wp, c->bv, c->bp};
    IBM_CUDA(c, cudaStreamSynchronize(c->s));
    dev_free(c, Cq);
    dev_free(c, derr);
    dev_free(c, vq);
    dev_free(c, cnt);
    dev_free(c, off);
    dev_free(c, tot);
    return IBM_OK;
}

}  // namespace ibm
