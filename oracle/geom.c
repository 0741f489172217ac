/*
 * Oracle geometry: plain, slow, single-threaded C for the immersed-body
 * tables of the ghost-cell method. TEST INFRASTRUCTURE ONLY: the product
 * path never links or calls this file; only tests/, the smoke check and the
 * CPU-baseline leg of the benchmark load it.
 *
 * What it computes (Section 2.2 of the paper):
 *   - which cell centres lie inside the closed body surface ("ray tracing",
 *     Section 2.2 and its cell-blanking figure), by the parity of surface
 *     crossings along the ray from the centre in the +y (2D) or +z (3D)
 *     direction, with every predicate exact on quantised integer
 *     coordinates;
 *   - the fluid / ghost / dead classification (Section 2.2: ghost cells are
 *     dead cells with a fluid neighbour);
 *   - per ghost cell: the body intercept (closest surface point), the image
 *     point (the normal from the ghost cell through the intercept, extended
 *     into the fluid), the 8 (2D: 4) surrounding cells and the interpolation
 *     weights beta of Eq. (2), obtained from the Vandermonde system of
 *     Eq. (3) by LU with partial pivoting.
 *
 * Readings of the paper fixed here (the paper is silent on them):
 *   - a centre is perturbed symbolically to (X+e^2, Y+e^4, Z-e) (2D:
 *     (X+e^2, Y-e)), so every tie resolves the same way on any machine;
 *   - the image point is the mirror of the ghost centre, IP = 2 BI - GC;
 *   - the ghost cell, when it is one of the 8 corners, takes the boundary
 *     row: Dirichlet b(x_BI), Neumann n . grad b(x_BI);
 *   - a dead corner, a near-singular system (|pivot| < 1e-12 max|V|) or a
 *     ghost centre on the surface (|BI-GC| < 1e-9 h) selects the fallback
 *     (kind 2): the image value is the value of the nearest fluid corner.
 *
 * Floating point: every operation is a single correctly rounded IEEE
 * double operation in the order written; build with -ffp-contract=off so the
 * compiler never fuses a multiply and an add.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

enum { FLUID = 0, GHOST = 1, DEAD = 2 };

/* round-to-nearest-even quantisation q = rint((x - lo) * s), s a power of 2 */
void orc_quantize(const double *x, int64_t n, double lo, double s, int64_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = llrint((x[i] - lo) * s);
}

static int sgn128(i128 v) { return (v > 0) - (v < 0); }

/* sign of orient((p->q), P) with P perturbed to (X+e, Y+e^2), e -> 0+ */
static int orient_perturbed(int64_t px, int64_t py, int64_t qx, int64_t qy,
                            int64_t X, int64_t Y, i128 *w)
{
    i128 v = (i128)(qx - px) * (i128)(Y - py) - (i128)(qy - py) * (i128)(X - px);
    *w = v;
    if (v != 0) return sgn128(v);
    if (qy != py) return (qy - py) > 0 ? -1 : 1;  /* e term: -(qy-py) */
    if (qx != px) return (qx - px) > 0 ? 1 : -1;  /* e^2 term: (qx-px) */
    return 0;
}

/*
 * 3D inside flags. Xq[nx], Yq[ny], Zq[nz]: quantised centre coordinates.
 * Vq[nv*3] quantised vertices, tris[nt*3]. inside[N] (N = nx*ny*nz) gets 0/1.
 */
void orc_inside_3d(int nx, int ny, int nz, const int64_t *Xq, const int64_t *Yq,
                   const int64_t *Zq, const int64_t *Vq, int64_t nt, const int32_t *tris,
                   uint8_t *inside)
{
    int64_t *cnt = (int64_t *)calloc((size_t)nz + 1, sizeof(int64_t));
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            memset(cnt, 0, sizeof(int64_t) * ((size_t)nz + 1));
            const int64_t X = Xq[i], Y = Yq[j];
            for (int64_t t = 0; t < nt; ++t) {
                const int64_t *a = Vq + 3 * (int64_t)tris[3 * t];
                const int64_t *b = Vq + 3 * (int64_t)tris[3 * t + 1];
                const int64_t *c = Vq + 3 * (int64_t)tris[3 * t + 2];
                /* exact prefilter: the perturbed column must be inside the
                   projected bounding box (X+e in [min,max), same for Y) */
                int64_t mnx = a[0] < b[0] ? a[0] : b[0]; mnx = c[0] < mnx ? c[0] : mnx;
                int64_t mxx = a[0] > b[0] ? a[0] : b[0]; mxx = c[0] > mxx ? c[0] : mxx;
                int64_t mny = a[1] < b[1] ? a[1] : b[1]; mny = c[1] < mny ? c[1] : mny;
                int64_t mxy = a[1] > b[1] ? a[1] : b[1]; mxy = c[1] > mxy ? c[1] : mxy;
                if (X < mnx || X >= mxx || Y < mny || Y >= mxy) continue;
                i128 den = (i128)(b[0] - a[0]) * (i128)(c[1] - a[1]) -
                           (i128)(b[1] - a[1]) * (i128)(c[0] - a[0]);
                if (den == 0) continue;
                i128 wa, wb, wc;
                int sa = orient_perturbed(b[0], b[1], c[0], c[1], X, Y, &wa);
                int sb = orient_perturbed(c[0], c[1], a[0], a[1], X, Y, &wb);
                int sc = orient_perturbed(a[0], a[1], b[0], b[1], X, Y, &wc);
                if (!(sa == sb && sb == sc && sa != 0)) continue;
                /* plane height at (X,Y): z0 = (wa za + wb zb + wc zc) / den.
                   Cell k counts this crossing iff z0 >= Z_k (centre perturbed
                   downwards), i.e. (S - Z_k den) * sign(den) >= 0. */
                i128 S = wa * (i128)a[2] + wb * (i128)b[2] + wc * (i128)c[2];
                int sd = sgn128(den);
                /* number of centres with Z_k <= z0: centres are increasing */
                int m = 0;
                while (m < nz && sgn128(S - (i128)Zq[m] * den) * sd >= 0) ++m;
                cnt[m] += 1;
            }
            /* cell k is crossed by every crossing with m > k */
            int64_t acc = 0;
            for (int k = nz - 1; k >= 0; --k) {
                acc += cnt[k + 1];
                inside[(int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k)] = (uint8_t)(acc & 1);
            }
        }
    free(cnt);
}

/* 2D inside flags: ray along +y from each centre; Vq[nv*2] quantised xy. */
void orc_inside_2d(int nx, int ny, const int64_t *Xq, const int64_t *Yq, const int64_t *Vq,
                   int64_t ne, const int32_t *segs, uint8_t *inside)
{
    int64_t *cnt = (int64_t *)calloc((size_t)ny + 1, sizeof(int64_t));
    for (int i = 0; i < nx; ++i) {
        memset(cnt, 0, sizeof(int64_t) * ((size_t)ny + 1));
        const int64_t X = Xq[i];
        for (int64_t e = 0; e < ne; ++e) {
            const int64_t *a = Vq + 2 * (int64_t)segs[2 * e];
            const int64_t *b = Vq + 2 * (int64_t)segs[2 * e + 1];
            /* column x = X+e crosses the segment iff one end is <= X and the
               other is > X */
            int cross = (a[0] <= X && X < b[0]) || (b[0] <= X && X < a[0]);
            if (!cross) continue;
            i128 dx = (i128)(b[0] - a[0]);
            /* y0 - Y = ((ay - Y) dx + (by - ay)(X - ax)) / dx */
            int sd = dx > 0 ? 1 : -1;
            int m = 0;
            while (m < ny) {
                i128 num = (i128)(a[1] - Yq[m]) * dx + (i128)(b[1] - a[1]) * (i128)(X - a[0]);
                if (sgn128(num) * sd >= 0) ++m; else break;
            }
            cnt[m] += 1;
        }
        int64_t acc = 0;
        for (int j = ny - 1; j >= 0; --j) {
            acc += cnt[j + 1];
            inside[(int64_t)i + (int64_t)nx * j] = (uint8_t)(acc & 1);
        }
    }
    free(cnt);
}

/* type[] from inside[]: DEAD if inside, GHOST if inside with a face
   neighbour (inside the domain) that is outside. Returns n_ghost and writes
   ascending linear indices of ghosts to gidx (may be NULL to count). */
int64_t orc_classify(int nx, int ny, int nz, const uint8_t *inside, uint8_t *type, int64_t *gidx)
{
    int64_t ng = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t c = (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
                if (!inside[c]) { type[c] = FLUID; continue; }
                int fl = 0;
                if (i > 0 && !inside[c - 1]) fl = 1;
                if (i < nx - 1 && !inside[c + 1]) fl = 1;
                if (j > 0 && !inside[c - nx]) fl = 1;
                if (j < ny - 1 && !inside[c + nx]) fl = 1;
                if (k > 0 && !inside[c - (int64_t)nx * ny]) fl = 1;
                if (k < nz - 1 && !inside[c + (int64_t)nx * ny]) fl = 1;
                type[c] = fl ? GHOST : DEAD;
                if (fl) { if (gidx) gidx[ng] = c; ++ng; }
            }
    return ng;
}

/* ---------------------------------------------------------------------- */
/* closest points (fixed operation order)                                  */
/* ---------------------------------------------------------------------- */

static double dot3(const double *u, const double *v) { return (u[0] * v[0] + u[1] * v[1]) + u[2] * v[2]; }

/* closest point on triangle abc to p, by the Voronoi-region method
   (Ericson, Real-Time Collision Detection, 2005, Sec. 5.1.5). */
static void closest_on_tri(const double *p, const double *a, const double *b, const double *c, double *q)
{
    double ab[3], ac[3], ap[3], bp[3], cp[3];
    for (int d = 0; d < 3; ++d) { ab[d] = b[d] - a[d]; ac[d] = c[d] - a[d]; ap[d] = p[d] - a[d]; }
    double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) { for (int d = 0; d < 3; ++d) q[d] = a[d]; return; }
    for (int d = 0; d < 3; ++d) bp[d] = p[d] - b[d];
    double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) { for (int d = 0; d < 3; ++d) q[d] = b[d]; return; }
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        double v = d1 / (d1 - d3);
        for (int d = 0; d < 3; ++d) q[d] = a[d] + v * ab[d];
        return;
    }
    for (int d = 0; d < 3; ++d) cp[d] = p[d] - c[d];
    double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) { for (int d = 0; d < 3; ++d) q[d] = c[d]; return; }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        double w = d2 / (d2 - d6);
        for (int d = 0; d < 3; ++d) q[d] = a[d] + w * ac[d];
        return;
    }
    double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
        double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int d = 0; d < 3; ++d) q[d] = b[d] + w * (c[d] - b[d]);
        return;
    }
    double den = 1.0 / ((va + vb) + vc);
    double v = vb * den, w = vc * den;
    for (int d = 0; d < 3; ++d) q[d] = (a[d] + ab[d] * v) + ac[d] * w;
}

/* closest point on segment ab (z ignored: all z are 0 in 2D) */
static void closest_on_seg(const double *p, const double *a, const double *b, double *q)
{
    double ab0 = b[0] - a[0], ab1 = b[1] - a[1];
    double ap0 = p[0] - a[0], ap1 = p[1] - a[1];
    double t = (ap0 * ab0 + ap1 * ab1) / (ab0 * ab0 + ab1 * ab1);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    q[0] = a[0] + t * ab0;
    q[1] = a[1] + t * ab1;
    q[2] = 0.0;
}

/* ---------------------------------------------------------------------- */
/* small dense solve                                                      */
/* ---------------------------------------------------------------------- */

/* Solve M x = r (n x n, row-major) by LU with partial pivoting.
   Returns 0 on success, 1 when a pivot is below 1e-12 * max|M|. */
static int lu_solve(int n, double *M, double *r, double *x)
{
    double scale = 0.0;
    for (int i = 0; i < n * n; ++i) { double v = fabs(M[i]); if (v > scale) scale = v; }
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(M[k * n + k]);
        for (int i = k + 1; i < n; ++i) { double v = fabs(M[i * n + k]); if (v > best) { best = v; p = i; } }
        if (best < 1e-12 * scale) return 1;
        if (p != k) {
            for (int j = 0; j < n; ++j) { double t = M[k * n + j]; M[k * n + j] = M[p * n + j]; M[p * n + j] = t; }
            double t = r[k]; r[k] = r[p]; r[p] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double l = M[i * n + k] / M[k * n + k];
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

/* trilinear basis [1,x,y,z,xy,yz,zx,xyz]; bilinear [1,x,y,xy] in 2D */
static void basis(int ndim, double x, double y, double z, double *b)
{
    if (ndim == 2) { b[0] = 1.0; b[1] = x; b[2] = y; b[3] = x * y; return; }
    b[0] = 1.0; b[1] = x; b[2] = y; b[3] = z;
    b[4] = x * y; b[5] = y * z; b[6] = z * x; b[7] = (x * y) * z;
}

/* n . grad b in physical units; (hx,hy,hz) the base-cell centre spacing */
static void basis_dn(int ndim, double x, double y, double z, const double *nrm,
                     double hx, double hy, double hz, double *g)
{
    double ax = nrm[0] / hx, ay = nrm[1] / hy;
    if (ndim == 2) {
        g[0] = 0.0; g[1] = ax; g[2] = ay; g[3] = ax * y + ay * x;
        return;
    }
    double az = nrm[2] / hz;
    g[0] = 0.0; g[1] = ax; g[2] = ay; g[3] = az;
    g[4] = ax * y + ay * x;
    g[5] = ay * z + az * y;
    g[6] = ax * z + az * x;
    g[7] = (ax * (y * z) + ay * (x * z)) + az * (x * y);
}

/* number of entries of c[0..n) that are <= v (c increasing) */
static int count_le(const double *c, int n, double v)
{
    int lo = 0, hi = n;
    while (lo < hi) { int mid = (lo + hi) / 2; if (c[mid] <= v) lo = mid + 1; else hi = mid; }
    return lo;
}

/*
 * Ghost-cell tables for ng ghosts (gidx ascending). Inputs: centre
 * coordinates xc[nx], yc[ny], zc[nz], cell sizes dx, dy, dz, type[N],
 * mesh verts[nv*3] and elems (2D segments ne*2, 3D triangles ne*3).
 * Outputs per ghost g:
 *   bi[3g..], nrm[3g..], ip[3g..], dist[g], base[g], kind[g], cmask[g],
 *   sidx[8g..] (cell indices of the 8 slots), wv[8g..], wp[8g..]
 *   (velocity = Dirichlet, pressure = Neumann weights of the slots),
 *   bv[g], bp[g] (weights of the boundary row, kind 1 only).
 */
void orc_ghost_tables(int ndim, int nx, int ny, int nz,
                      const double *xc, const double *yc, const double *zc,
                      const double *dx, const double *dy, const double *dz,
                      const uint8_t *type, int64_t ng, const int64_t *gidx,
                      const double *verts, int64_t ne, const int32_t *elems,
                      double *bi, double *nrm, double *ip, double *dist,
                      int64_t *base, uint8_t *kind, uint8_t *cmask,
                      int64_t *sidx, double *wv, double *wp, double *bv, double *bp)
{
    const int nc = ndim == 2 ? 4 : 8;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    for (int64_t g = 0; g < ng; ++g) {
        const int64_t c = gidx[g];
        const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / sz);
        double p[3] = {xc[i], yc[j], ndim == 2 ? 0.0 : zc[k]};
        /* body intercept: lowest (squared distance, element index) */
        double best = INFINITY, q[3] = {0, 0, 0};
        int64_t bel = -1;
        for (int64_t e = 0; e < ne; ++e) {
            double qq[3];
            if (ndim == 2)
                closest_on_seg(p, verts + 3 * (int64_t)elems[2 * e], verts + 3 * (int64_t)elems[2 * e + 1], qq);
            else
                closest_on_tri(p, verts + 3 * (int64_t)elems[3 * e], verts + 3 * (int64_t)elems[3 * e + 1],
                               verts + 3 * (int64_t)elems[3 * e + 2], qq);
            double dv[3] = {qq[0] - p[0], qq[1] - p[1], qq[2] - p[2]};
            double dd = dot3(dv, dv);
            if (dd < best) { best = dd; bel = e; q[0] = qq[0]; q[1] = qq[1]; q[2] = qq[2]; }
        }
        (void)bel;
        double dv[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
        double d = sqrt(dot3(dv, dv));
        double hloc = dx[i] < dy[j] ? dx[i] : dy[j];
        if (ndim == 3 && dz[k] < hloc) hloc = dz[k];
        int degenerate = !(d >= 1e-9 * hloc);
        double n[3] = {0, 0, 0}, x[3];
        if (!degenerate) {
            n[0] = dv[0] / d; n[1] = dv[1] / d; n[2] = dv[2] / d;
            x[0] = 2.0 * q[0] - p[0]; x[1] = 2.0 * q[1] - p[1]; x[2] = 2.0 * q[2] - p[2];
        } else {
            x[0] = p[0]; x[1] = p[1]; x[2] = p[2];
        }
        if (ndim == 2) x[2] = 0.0;
        for (int a = 0; a < 3; ++a) { bi[3 * g + a] = q[a]; nrm[3 * g + a] = n[a]; ip[3 * g + a] = x[a]; }
        dist[g] = d;
        /* base cell: lower corner of the centre-lattice cell holding IP */
        int i0 = count_le(xc, nx, x[0]) - 1, j0 = count_le(yc, ny, x[1]) - 1, k0 = 0;
        if (i0 < 0) i0 = 0;
        if (i0 > nx - 2) i0 = nx - 2;
        if (j0 < 0) j0 = 0;
        if (j0 > ny - 2) j0 = ny - 2;
        if (ndim == 3) {
            k0 = count_le(zc, nz, x[2]) - 1;
            if (k0 < 0) k0 = 0;
            if (k0 > nz - 2) k0 = nz - 2;
        }
        base[g] = (int64_t)i0 + sy * j0 + sz * k0;
        double hx = xc[i0 + 1] - xc[i0], hy = yc[j0 + 1] - yc[j0];
        double hz = ndim == 3 ? zc[k0 + 1] - zc[k0] : 1.0;
        int64_t cidx[8];
        int self = -1, dead = 0;
        uint8_t msk = 0;
        for (int m = 0; m < nc; ++m) {
            int di = m & 1, dj = (m >> 1) & 1, dk = (m >> 2) & 1;
            cidx[m] = (int64_t)(i0 + di) * sx + (int64_t)(j0 + dj) * sy + (int64_t)(k0 + dk) * sz;
            uint8_t t = type[cidx[m]];
            if (t != FLUID) msk |= (uint8_t)(1u << m);
            if (cidx[m] == c) self = m;
            else if (t == DEAD) dead = 1;
        }
        cmask[g] = msk;
        int kd = degenerate ? 2 : (dead ? 2 : (self >= 0 ? 1 : 0));
        double bIP[8], bBI[8], gBI[8], Mv[64], Mp[64], rv[8], rp[8], xv[8], xp[8];
        if (kd != 2) {
            double xi = (x[0] - xc[i0]) / hx, et = (x[1] - yc[j0]) / hy;
            double ze = ndim == 3 ? (x[2] - zc[k0]) / hz : 0.0;
            basis(ndim, xi, et, ze, bIP);
            if (kd == 1) {
                double bxi = (q[0] - xc[i0]) / hx, bet = (q[1] - yc[j0]) / hy;
                double bze = ndim == 3 ? (q[2] - zc[k0]) / hz : 0.0;
                basis(ndim, bxi, bet, bze, bBI);
                basis_dn(ndim, bxi, bet, bze, n, hx, hy, hz, gBI);
            }
            /* rows of V are the basis at each corner; M = V^T */
            for (int m = 0; m < nc; ++m) {
                double row[8];
                if (m == self) {
                    for (int r = 0; r < nc; ++r) row[r] = bBI[r];
                } else {
                    basis(ndim, (double)(m & 1), (double)((m >> 1) & 1), (double)((m >> 2) & 1), row);
                }
                for (int r = 0; r < nc; ++r) Mv[r * nc + m] = row[r];
                if (m == self) for (int r = 0; r < nc; ++r) row[r] = gBI[r];
                for (int r = 0; r < nc; ++r) Mp[r * nc + m] = row[r];
            }
            for (int r = 0; r < nc; ++r) { rv[r] = bIP[r]; rp[r] = bIP[r]; }
            int s1 = lu_solve(nc, Mv, rv, xv);
            int s2 = lu_solve(nc, Mp, rp, xp);
            if (s1 || s2) kd = 2;
        }
        kind[g] = (uint8_t)kd;
        double *WV = wv + 8 * g, *WP = wp + 8 * g;
        int64_t *SI = sidx + 8 * g;
        bv[g] = 0.0;
        bp[g] = 0.0;
        if (kd != 2) {
            for (int m = 0; m < 8; ++m) {
                if (m < nc && m != self) { SI[m] = cidx[m]; WV[m] = xv[m]; WP[m] = xp[m]; }
                else { SI[m] = c; WV[m] = 0.0; WP[m] = 0.0; }
            }
            if (self >= 0) { bv[g] = xv[self]; bp[g] = xp[self]; }
        } else {
            /* nearest FLUID corner to IP (first on ties); else the first
               FLUID face neighbour in the order -x,+x,-y,+y,-z,+z */
            int64_t pick = -1;
            double bd = INFINITY;
            for (int m = 0; m < nc; ++m) {
                if (type[cidx[m]] != FLUID) continue;
                int ci = i0 + (m & 1), cj = j0 + ((m >> 1) & 1), ck = k0 + ((m >> 2) & 1);
                double e0 = xc[ci] - x[0], e1 = yc[cj] - x[1], e2 = ndim == 3 ? zc[ck] - x[2] : 0.0;
                double dd = (e0 * e0 + e1 * e1) + e2 * e2;
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
}

/*
 * Fresh cells (Section 2.2: cells that were inside a moving body and are
 * fluid now; their value comes from an interpolation that uses the body
 * velocity at the body intercept). Reading fixed here: for a fresh cell FC
 * with body intercept BI (closest surface point) and normal n = (FC - BI) /
 * |FC - BI| (into the fluid), the trilinear basis is fitted on the lattice
 * cell of centres that has FC as a corner and extends towards n along each
 * axis (clamped into the grid); the row of the corner FC itself is the
 * Dirichlet row b(x_BI), and the fit is evaluated at FC:
 *     u_FC = sum_{m != FC} w_m u_m + wb u_BI.
 * Other corners must be FLUID (fresh corners included, as implicit
 * unknowns); a GHOST or DEAD corner, a near-singular system or an FC on the
 * surface (|FC - BI| < 1e-9 h) gives kind 2: u_FC = u_BI (w = 0, wb = 1).
 * Output per fresh cell: bi[3], kind, sidx[8] (the FC itself with weight 0
 * in unused slots), w[8], wb.
 */
void orc_fresh_tables(int ndim, int nx, int ny, int nz,
                      const double *xc, const double *yc, const double *zc,
                      const double *dx, const double *dy, const double *dz,
                      const uint8_t *type, int64_t nf, const int64_t *fidx,
                      const double *verts, int64_t ne, const int32_t *elems,
                      double *bi, uint8_t *kind, int64_t *sidx, double *w, double *wb)
{
    const int nc = ndim == 2 ? 4 : 8;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    for (int64_t f = 0; f < nf; ++f) {
        const int64_t c = fidx[f];
        const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / sz);
        double p[3] = {xc[i], yc[j], ndim == 2 ? 0.0 : zc[k]};
        double best = INFINITY, q[3] = {0, 0, 0};
        for (int64_t e = 0; e < ne; ++e) {
            double qq[3];
            if (ndim == 2)
                closest_on_seg(p, verts + 3 * (int64_t)elems[2 * e], verts + 3 * (int64_t)elems[2 * e + 1], qq);
            else
                closest_on_tri(p, verts + 3 * (int64_t)elems[3 * e], verts + 3 * (int64_t)elems[3 * e + 1],
                               verts + 3 * (int64_t)elems[3 * e + 2], qq);
            double dv[3] = {qq[0] - p[0], qq[1] - p[1], qq[2] - p[2]};
            double dd = dot3(dv, dv);
            if (dd < best) { best = dd; q[0] = qq[0]; q[1] = qq[1]; q[2] = qq[2]; }
        }
        for (int a = 0; a < 3; ++a) bi[3 * f + a] = q[a];
        double dv[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
        double d = sqrt(dot3(dv, dv));
        double hloc = dx[i] < dy[j] ? dx[i] : dy[j];
        if (ndim == 3 && dz[k] < hloc) hloc = dz[k];
        int kd = !(d >= 1e-9 * hloc) ? 2 : 1;
        double n[3] = {0, 0, 0};
        if (kd == 1) { n[0] = dv[0] / d; n[1] = dv[1] / d; n[2] = dv[2] / d; }
        int i0 = n[0] >= 0.0 ? i : i - 1, j0 = n[1] >= 0.0 ? j : j - 1, k0 = 0;
        if (i0 < 0) i0 = 0;
        if (i0 > nx - 2) i0 = nx - 2;
        if (j0 < 0) j0 = 0;
        if (j0 > ny - 2) j0 = ny - 2;
        if (ndim == 3) {
            k0 = n[2] >= 0.0 ? k : k - 1;
            if (k0 < 0) k0 = 0;
            if (k0 > nz - 2) k0 = nz - 2;
        }
        int64_t cidx[8];
        int self = -1;
        for (int m = 0; m < nc; ++m) {
            int di = m & 1, dj = (m >> 1) & 1, dk = (m >> 2) & 1;
            cidx[m] = (int64_t)(i0 + di) * sx + (int64_t)(j0 + dj) * sy + (int64_t)(k0 + dk) * sz;
            if (cidx[m] == c) self = m;
            else if (type[cidx[m]] != FLUID) kd = 2;
        }
        double xw[8];
        if (kd == 1) {
            double hx = xc[i0 + 1] - xc[i0], hy = yc[j0 + 1] - yc[j0];
            double hz = ndim == 3 ? zc[k0 + 1] - zc[k0] : 1.0;
            double bxi = (q[0] - xc[i0]) / hx, bet = (q[1] - yc[j0]) / hy;
            double bze = ndim == 3 ? (q[2] - zc[k0]) / hz : 0.0;
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
}
