/*
 * dwg_oracle.c -- plain FP64 CPU oracle for Diffusing Winding Gradients.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Every function is a direct, slow, sequential-per-output transcription of
 * the paper's definitions:
 *   - the discrete generalized winding number (Sec. 3, Eq. 2 with the Poisson
 *     kernel of Eq. 3) and its screened variant (Sec. 4.2, Eq. 5), with the
 *     "small constant added to the denominator" of Sec. 3 read as Plummer
 *     softening rho^2 = |p - q|^2 + eps^2, and terms with p == q skipped;
 *   - the gradient of either sum with respect to the query point, normals
 *     held fixed (Sec. 4.1); the paper prints no formula, the closed form
 *     used here is the exact derivative of the softened term;
 *   - the iteration of Algorithm 1 / Sec. 4.3: octree of depth d around the
 *     cloud (Sec. 5.1), w at the octree's leaf corners, iso-value w_bar as the
 *     mean of w over the input points (Eq. 6 read per the abstract), level
 *     set extraction (Marching Cubes, realised as the six-tetrahedron split
 *     of each leaf cube), per-face gradient from the cross product, scatter
 *     of each face gradient onto its k nearest input points and
 *     normalisation (Eq. 7);
 *   - the convergence rule of Sec. 5.1: mean of the largest 1% of the
 *     per-point normal changes, in degrees, compared with eps (0.1 deg);
 *   - the modified Poisson kernel of Sec. 5.2 ("Poisson Kernels"): with a
 *     per-source radius delta_j the denominator becomes delta_j^3 when
 *     |p_j - q| < delta_j (no softening then).  Whether a pair is inside is
 *     an integer decision taken from floating point, so it is taken in the
 *     CUDA kernel's precision: |p_j - q|^2 in float32 (offsets rounded to
 *     float, squares summed with fused multiply-adds) against delta_j^2
 *     rounded to float32.  Everything else stays FP64.
 *
 * All arithmetic is double precision.  Build with -ffp-contract=off so that
 * a*b+c is never fused: the cell-quantisation step below must round exactly
 * like the CUDA side's explicit __dmul_rn/__dsub_rn sequence.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* threads of the parallel loops (n <= 0: the OpenMP default); returns the
 * count in effect, 1 without OpenMP */
int dwgo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

#define DWGO_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Eq. 2/3 and Eq. 5: w(q) and grad_q w(q)                                  */
/* ------------------------------------------------------------------------ */

/* Is source p within the clamp radius delta of q?  Decided like the CUDA
 * kernel: float32 offsets, squares summed by fused multiply-adds in the
 * order x, y, z, compared with delta^2 rounded to float32. */
static int clamp_inside(const double *p, const double *q, double delta)
{
    float dx = (float)p[0] - (float)q[0];
    float dy = (float)p[1] - (float)q[1];
    float dz = (float)p[2] - (float)q[2];
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    return r2 < (float)(delta * delta);
}

/*
 * One source term and its gradient with respect to q.
 *   d = p - q, rho^2 = |d|^2 + eps^2, m = a n / (4 pi), phi = <m, d> / rho^3.
 *   plain:    t = phi,                grad t = -m / rho^3 + 3 phi d / rho^2
 *   screened: F = exp(-s rho)(1 + s rho), s = sqrt(lambda)
 *             t = F phi,              grad t = F grad(phi) + phi s^2 exp(-s rho) d
 * (grad_q rho = -d / rho and dF/drho = -s^2 rho exp(-s rho)).
 * Modified kernel (delta > 0, eps unused): rho = |d| outside the radius; inside
 * it rho = delta is constant, so t = F(delta) <m, d> / delta^3 and
 * grad t = -F(delta) m / delta^3.
 */
static void term(const double *p, const double *nrm, double a, const double *q,
                 int screened, double eps, double delta, double s, double *t, double g[3])
{
    double d[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    double m[3] = {a * nrm[0] / (4.0 * DWGO_PI), a * nrm[1] / (4.0 * DWGO_PI),
                   a * nrm[2] / (4.0 * DWGO_PI)};
    int inside = delta > 0.0 && clamp_inside(p, q, delta);
    double rho2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (delta > 0.0) {
        if (inside) rho2 = delta * delta;
    } else {
        rho2 += eps * eps;
    }
    double rho = sqrt(rho2);
    double rho3 = rho2 * rho;
    double phi = (m[0] * d[0] + m[1] * d[1] + m[2] * d[2]) / rho3;
    double F = 1.0, E = 0.0;
    if (screened) {
        E = exp(-s * rho);
        F = E * (1.0 + s * rho);
    }
    *t = F * phi;
    for (int k = 0; k < 3; ++k) {
        double gphi = -m[k] / rho3 + (inside ? 0.0 : 3.0 * phi * d[k] / rho2);
        g[k] = F * gphi + (inside ? 0.0 : phi * s * s * E * d[k]);
    }
}

/*
 * w and grad w at m queries from n oriented, weighted points.
 *   p, nrm: n x 3 row-major; a: n weights (Sec. 3: Voronoi areas, or 1);
 *   q: m x 3; kernel 0 = plain (Eq. 2/3), 1 = screened (Eq. 5);
 *   delta: n clamp radii of the modified kernel (Sec. 5.2), or NULL for the
 *   softened kernel with eps;
 *   w: m outputs; g: m x 3 outputs or NULL.
 * Terms with p_j == q exactly (all three coordinates) are skipped.
 */
void dwgo_gwn(int64_t n, const double *p, const double *nrm, const double *a,
              int64_t m, const double *q, int kernel, double eps, double lambda,
              const double *delta, double *w, double *g)
{
    double s = sqrt(lambda > 0 ? lambda : 0.0);
    int screened = (kernel == 1);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        const double *qi = q + 3 * i;
        double wi = 0.0, gi[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            const double *pj = p + 3 * j;
            if (pj[0] == qi[0] && pj[1] == qi[1] && pj[2] == qi[2])
                continue;
            double t, gt[3];
            term(pj, nrm + 3 * j, a[j], qi, screened, eps, delta ? delta[j] : 0.0, s, &t, gt);
            wi += t;
            gi[0] += gt[0];
            gi[1] += gt[1];
            gi[2] += gt[2];
        }
        w[i] = wi;
        if (g) {
            g[3 * i + 0] = gi[0];
            g[3 * i + 1] = gi[1];
            g[3 * i + 2] = gi[2];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 5.1: the octree around the cloud                                    */
/* ------------------------------------------------------------------------ */

/*
 * The root cube: centred on the bounding box of the (float32) input
 * coordinates, edge L = 1.125 * (largest bounding-box extent), or 1 when all
 * points coincide.  Cells at depth d have edge h = L / 2^d; a point's cell
 * index along each axis is floor((x - lo) * (2^d / L)) clamped to
 * [0, 2^d - 1].  out = {lo_x, lo_y, lo_z, L, h, inv_h}.
 */
void dwgo_cube(int64_t n, const double *p, int d, double *out)
{
    double mn[3] = {p[0], p[1], p[2]}, mx[3] = {p[0], p[1], p[2]};
    for (int64_t i = 1; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            if (p[3 * i + k] < mn[k]) mn[k] = p[3 * i + k];
            if (p[3 * i + k] > mx[k]) mx[k] = p[3 * i + k];
        }
    double ext = 0.0;
    for (int k = 0; k < 3; ++k)
        if (mx[k] - mn[k] > ext) ext = mx[k] - mn[k];
    double L = ext > 0.0 ? ext * 1.125 : 1.0;
    for (int k = 0; k < 3; ++k) {
        double c = (mn[k] + mx[k]) * 0.5;
        out[k] = c - L * 0.5;
    }
    out[3] = L;
    out[4] = L / ldexp(1.0, d);
    out[5] = ldexp(1.0, d) / L;
}

static int64_t cell_of(double x, double lo, double inv_h, int d)
{
    double t = (x - lo) * inv_h;
    int64_t c = (int64_t)floor(t);
    int64_t hi = ((int64_t)1 << d) - 1;
    if (c < 0) c = 0;
    if (c > hi) c = hi;
    return c;
}

/* Cell coordinates (depth d) of every point: n x 3 int64. */
void dwgo_cells(int64_t n, const double *p, int d, int64_t *cells)
{
    double cube[6];
    dwgo_cube(n, p, d, cube);
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k)
            cells[3 * i + k] = cell_of(p[3 * i + k], cube[k], cube[5], d);
}

typedef struct {
    int d;
    const int64_t *cells; /* n x 3 */
    int64_t *leaves;      /* nleaves x 5: level, ix, iy, iz, nonempty */
    int64_t nleaves, cap;
} octree_ctx;

static void push_leaf(octree_ctx *c, int64_t level, int64_t ix, int64_t iy, int64_t iz,
                      int64_t nonempty)
{
    if (c->leaves && c->nleaves < c->cap) {
        int64_t *L = c->leaves + 5 * c->nleaves;
        L[0] = level; L[1] = ix; L[2] = iy; L[3] = iz; L[4] = nonempty;
    }
    c->nleaves++;
}

/* Subdivide a non-empty node holding the points idx[0..cnt). */
static void subdivide(octree_ctx *c, int level, int64_t ix, int64_t iy, int64_t iz,
                      int64_t *idx, int64_t cnt)
{
    if (level == c->d) {
        push_leaf(c, level, ix, iy, iz, 1);
        return;
    }
    int shift = c->d - level - 1;
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt > 0 ? cnt : 1));
    for (int ch = 0; ch < 8; ++ch) {
        int64_t cx = 2 * ix + (ch & 1), cy = 2 * iy + ((ch >> 1) & 1), cz = 2 * iz + (ch >> 2);
        int64_t k = 0;
        for (int64_t t = 0; t < cnt; ++t) {
            const int64_t *cl = c->cells + 3 * idx[t];
            if ((cl[0] >> shift) == cx && (cl[1] >> shift) == cy && (cl[2] >> shift) == cz)
                tmp[k++] = idx[t];
        }
        if (k == 0) {
            push_leaf(c, level + 1, cx, cy, cz, 0);
        } else {
            int64_t *sub = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
            memcpy(sub, tmp, sizeof(int64_t) * (size_t)k);
            subdivide(c, level + 1, cx, cy, cz, sub, k);
            free(sub);
        }
    }
    free(tmp);
}

/*
 * Leaves of the octree of depth d: a node containing input points is split
 * into its 8 children until depth d; empty children are leaves of their own
 * level.  Returns the number of leaves; if leaves != NULL, writes up to cap
 * records (level, ix, iy, iz, nonempty) with (ix, iy, iz) in units of the
 * leaf's own level, in depth-first order, children in order x fastest.
 */
int64_t dwgo_octree(int64_t n, const double *p, int d, int64_t *leaves, int64_t cap)
{
    int64_t *cells = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)n);
    dwgo_cells(n, p, d, cells);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    octree_ctx c = {d, cells, leaves, 0, cap};
    subdivide(&c, 0, 0, 0, 0, idx, n);
    free(idx);
    free(cells);
    return c.nleaves;
}

/* Corner of leaf record L, number v (bit 0 = +x, bit 1 = +y, bit 2 = +z), in
 * depth-d lattice units. */
static void leaf_corner(const int64_t *L, int d, int v, int64_t X[3])
{
    int64_t s = (int64_t)1 << (d - (int)L[0]);
    X[0] = (L[1] + (v & 1)) * s;
    X[1] = (L[2] + ((v >> 1) & 1)) * s;
    X[2] = (L[3] + ((v >> 2) & 1)) * s;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* key of a lattice corner: X * (S+1)^2 + Y * (S+1) + Z, S = 2^d */
static int64_t corner_key(const int64_t X[3], int d)
{
    int64_t S1 = ((int64_t)1 << d) + 1;
    return (X[0] * S1 + X[1]) * S1 + X[2];
}

/*
 * Distinct corners of all leaves, as sorted keys X*(S+1)^2 + Y*(S+1) + Z.
 * Returns the count; writes up to cap keys if keys != NULL.
 */
int64_t dwgo_corners(int64_t nleaves, const int64_t *leaves, int d, int64_t *keys, int64_t cap)
{
    int64_t *all = (int64_t *)malloc(sizeof(int64_t) * 8 * (size_t)(nleaves > 0 ? nleaves : 1));
    for (int64_t l = 0; l < nleaves; ++l)
        for (int v = 0; v < 8; ++v) {
            int64_t X[3];
            leaf_corner(leaves + 5 * l, d, v, X);
            all[8 * l + v] = corner_key(X, d);
        }
    qsort(all, (size_t)(8 * nleaves), sizeof(int64_t), cmp_i64);
    int64_t u = 0;
    for (int64_t i = 0; i < 8 * nleaves; ++i)
        if (i == 0 || all[i] != all[i - 1]) {
            if (keys && u < cap) keys[u] = all[i];
            ++u;
        }
    free(all);
    return u;
}

/* Positions of corner keys: lo + X * h per axis in double, then rounded to
 * float32 (the query positions the library evaluates at). */
void dwgo_corner_positions(int64_t nc, const int64_t *keys, int d, const double *cube,
                           double *pos)
{
    int64_t S1 = ((int64_t)1 << d) + 1;
    for (int64_t i = 0; i < nc; ++i) {
        int64_t Z = keys[i] % S1, Y = (keys[i] / S1) % S1, X = keys[i] / (S1 * S1);
        pos[3 * i + 0] = (double)(float)(cube[0] + (double)X * cube[4]);
        pos[3 * i + 1] = (double)(float)(cube[1] + (double)Y * cube[4]);
        pos[3 * i + 2] = (double)(float)(cube[2] + (double)Z * cube[4]);
    }
}

static int64_t find_key(const int64_t *keys, int64_t nc, int64_t key)
{
    int64_t lo = 0, hi = nc - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (keys[mid] == key) return mid;
        if (keys[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Level set extraction (Sec. 4.3, Alg. 1): faces and their gradients       */
/* ------------------------------------------------------------------------ */

/* The six tetrahedra of a cube around its 0-7 diagonal. */
static const int TETS[6][4] = {{0, 1, 3, 7}, {0, 3, 2, 7}, {0, 2, 6, 7},
                               {0, 6, 4, 7}, {0, 4, 5, 7}, {0, 5, 1, 7}};

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* crossing point on edge (a,b) of the linear interpolant's zero */
static void edge_point(const double *xa, double fa, const double *xb, double fb, double out[3])
{
    double t = fa / (fa - fb);
    for (int k = 0; k < 3; ++k) out[k] = xa[k] + t * (xb[k] - xa[k]);
}

/*
 * The level-set polygon of one tetrahedron (x: 4 x 3 positions, f: values
 * minus the iso-value).  A vertex is "above" when f > 0.  With one or three
 * vertices above the polygon is a triangle, with two a quadrilateral.
 * area: the polygon's vector area (half the cross product of its diagonals;
 * for a triangle, half the cross product of two edges), oriented toward the
 * above side, i.e. along the gradient of w.  centroid: mean of the polygon's
 * vertices.  Returns 0 when the tetrahedron holds no level set.
 */
static int tet_face(const double x[4][3], const double f[4], double area[3], double centroid[3])
{
    int above[4], na = 0;
    for (int i = 0; i < 4; ++i) {
        above[i] = f[i] > 0.0;
        na += above[i];
    }
    if (na == 0 || na == 4) return 0;
    double P[4][3];
    int np;
    if (na == 1 || na == 3) {
        int lone = -1;
        for (int i = 0; i < 4; ++i)
            if (above[i] == (na == 1)) lone = i;
        np = 0;
        for (int i = 0; i < 4; ++i)
            if (i != lone) edge_point(x[lone], f[lone], x[i], f[i], P[np++]);
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = P[1][k] - P[0][k];
            e2[k] = P[2][k] - P[0][k];
        }
        cross3(e1, e2, area);
    } else {
        int a0 = -1, a1 = -1, b0 = -1, b1 = -1;
        for (int i = 0; i < 4; ++i) {
            if (above[i]) { if (a0 < 0) a0 = i; else a1 = i; }
            else { if (b0 < 0) b0 = i; else b1 = i; }
        }
        /* cyclic order (a0,b0) (a0,b1) (a1,b1) (a1,b0) */
        edge_point(x[a0], f[a0], x[b0], f[b0], P[0]);
        edge_point(x[a0], f[a0], x[b1], f[b1], P[1]);
        edge_point(x[a1], f[a1], x[b1], f[b1], P[2]);
        edge_point(x[a1], f[a1], x[b0], f[b0], P[3]);
        np = 4;
        double d1[3], d2[3];
        for (int k = 0; k < 3; ++k) {
            d1[k] = P[2][k] - P[0][k];
            d2[k] = P[3][k] - P[1][k];
        }
        cross3(d1, d2, area);
    }
    for (int k = 0; k < 3; ++k) area[k] *= 0.5;
    /* orient toward the above side: the interpolant grows from the mean of
     * the below vertices to the mean of the above vertices */
    double ca[3] = {0, 0, 0}, cb[3] = {0, 0, 0};
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) {
            if (above[i]) ca[k] += x[i][k] / na;
            else cb[k] += x[i][k] / (4 - na);
        }
    double dir = 0.0;
    for (int k = 0; k < 3; ++k) dir += area[k] * (ca[k] - cb[k]);
    if (dir < 0.0)
        for (int k = 0; k < 3; ++k) area[k] = -area[k];
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += P[i][k];
        centroid[k] = s / np;
    }
    return 1;
}

/*
 * Faces of the iso-level set over all leaves.  wc: w at the sorted corner
 * keys; iso: the iso-value.  Writes up to cap faces as 6 doubles each
 * (area vector, centroid).  Returns the face count.
 */
int64_t dwgo_faces(int64_t nleaves, const int64_t *leaves, int d, const double *cube,
                   int64_t nc, const int64_t *keys, const double *wc, double iso,
                   double *faces, int64_t cap)
{
    int64_t nf = 0;
    for (int64_t l = 0; l < nleaves; ++l) {
        double xv[8][3], fv[8];
        for (int v = 0; v < 8; ++v) {
            int64_t X[3];
            leaf_corner(leaves + 5 * l, d, v, X);
            int64_t c = find_key(keys, nc, corner_key(X, d));
            for (int k = 0; k < 3; ++k)
                xv[v][k] = (double)(float)(cube[k] + (double)X[k] * cube[4]);
            fv[v] = wc[c] - iso;
        }
        for (int t = 0; t < 6; ++t) {
            double xt[4][3], ft[4], A[3], C[3];
            for (int i = 0; i < 4; ++i) {
                memcpy(xt[i], xv[TETS[t][i]], sizeof(xt[i]));
                ft[i] = fv[TETS[t][i]];
            }
            if (tet_face(xt, ft, A, C)) {
                if (faces && nf < cap) {
                    double *F = faces + 6 * nf;
                    F[0] = A[0]; F[1] = A[1]; F[2] = A[2];
                    F[3] = C[0]; F[4] = C[1]; F[5] = C[2];
                }
                ++nf;
            }
        }
    }
    return nf;
}

/* ------------------------------------------------------------------------ */
/* k nearest input points (brute force, ties by smaller index)              */
/* ------------------------------------------------------------------------ */

void dwgo_knn(int64_t n, const double *p, int64_t m, const double *q, int k, int64_t *idx)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        double bd[64];
        int64_t bi[64];
        int cnt = 0;
        const double *qi = q + 3 * i;
        for (int64_t j = 0; j < n; ++j) {
            double dx = p[3 * j] - qi[0], dy = p[3 * j + 1] - qi[1], dz = p[3 * j + 2] - qi[2];
            double dd = dx * dx + dy * dy + dz * dz;
            /* keep the k smallest (dd, j) pairs in ascending order; j only
             * grows, so an equal distance never displaces an earlier index */
            if (cnt == k && !(dd < bd[k - 1])) continue;
            int pos = cnt < k ? cnt++ : k - 1;
            while (pos > 0 && bd[pos - 1] > dd) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = dd;
            bi[pos] = j;
        }
        for (int t = 0; t < k; ++t) idx[(int64_t)k * i + t] = t < cnt ? bi[t] : -1;
    }
}

/* ------------------------------------------------------------------------ */
/* Convergence measure (Sec. 5.1)                                            */
/* ------------------------------------------------------------------------ */

/* angle between unit vectors in degrees, atan2 form */
static double angle_deg(const double a[3], const double b[3])
{
    double c[3];
    cross3(a, b, c);
    double s = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    double d = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    return atan2(s, d) * (180.0 / DWGO_PI);
}

static int cmp_desc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

/* Mean of the ceil(n / 100) largest values. */
double dwgo_top1_mean(int64_t n, const double *v)
{
    if (n <= 0) return 0.0;
    double *s = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(s, v, sizeof(double) * (size_t)n);
    qsort(s, (size_t)n, sizeof(double), cmp_desc);
    int64_t k = (n + 99) / 100;
    double acc = 0.0;
    for (int64_t i = 0; i < k; ++i) acc += s[i];
    free(s);
    return acc / (double)k;
}

/* ------------------------------------------------------------------------ */
/* One iteration and the full loop                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int kernel;      /* 0 plain, 1 screened */
    double eps;      /* softening length */
    double lambda;   /* screening constant */
    int depth;       /* octree depth d */
    int knn;         /* k of Eq. 7's face-to-point assignment */
    int mode;        /* 0 level-set update (Eq. 7), 1 point-gradient update */
    int max_iters;
    double tol;      /* degrees */
    int rule;        /* 0: top-1 % mean change (Sec. 5.1); 1: mean |n_new - n_old| (Fig. 6) */
    const double *delta; /* n clamp radii of the modified kernel (Sec. 5.2), or NULL */
} dwgo_params;

/*
 * New normals from a face list (Eq. 7): each face adds its gradient to its
 * k nearest points; the outward normal is minus the normalised sum (w is
 * 1 inside, 0 outside, so its gradient points inward).  A point that no face
 * selected keeps its normal.
 */
void dwgo_scatter_normals(int64_t n, const double *p, int64_t nf, const double *faces, int k,
                          const double *n_old, double *n_new)
{
    double *acc = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *cent = (double *)malloc(sizeof(double) * 3 * (size_t)(nf > 0 ? nf : 1));
    int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * (size_t)k * (size_t)(nf > 0 ? nf : 1));
    for (int64_t f = 0; f < nf; ++f)
        for (int c = 0; c < 3; ++c) cent[3 * f + c] = faces[6 * f + 3 + c];
    dwgo_knn(n, p, nf, cent, k, nb);
    for (int64_t f = 0; f < nf; ++f)
        for (int t = 0; t < k; ++t) {
            int64_t j = nb[(int64_t)k * f + t];
            if (j < 0) continue;
            for (int c = 0; c < 3; ++c) acc[3 * j + c] += faces[6 * f + c];
        }
    for (int64_t j = 0; j < n; ++j) {
        double *a = acc + 3 * j;
        double len = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int c = 0; c < 3; ++c)
            n_new[3 * j + c] = len > 0.0 ? -a[c] / len : n_old[3 * j + c];
    }
    free(nb);
    free(cent);
    free(acc);
}

/*
 * One iteration from normals n_old.  Outputs: n_new, per-point change dtheta
 * (degrees), w at the points (wp), grad w at the points (gp, may be NULL),
 * and the iso-value.  Returns the number of level-set faces (mode 0) or 0.
 */
int64_t dwgo_iterate(int64_t n, const double *p, const double *a, const double *n_old,
                     const dwgo_params *prm, double *n_new, double *dtheta, double *wp,
                     double *gp, double *iso_out)
{
    double *g = gp ? gp : (double *)malloc(sizeof(double) * 3 * (size_t)n);
    dwgo_gwn(n, p, n_old, a, n, p, prm->kernel, prm->eps, prm->lambda, prm->delta, wp, g);
    double iso = 0.0;
    for (int64_t i = 0; i < n; ++i) iso += wp[i];
    iso /= (double)n;
    *iso_out = iso;
    int64_t nf = 0;
    if (prm->mode == 0) {
        int d = prm->depth;
        int64_t nl = dwgo_octree(n, p, d, NULL, 0);
        int64_t *leaves = (int64_t *)malloc(sizeof(int64_t) * 5 * (size_t)nl);
        dwgo_octree(n, p, d, leaves, nl);
        int64_t nc = dwgo_corners(nl, leaves, d, NULL, 0);
        int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
        dwgo_corners(nl, leaves, d, keys, nc);
        double cube[6];
        dwgo_cube(n, p, d, cube);
        double *cpos = (double *)malloc(sizeof(double) * 3 * (size_t)nc);
        dwgo_corner_positions(nc, keys, d, cube, cpos);
        double *wc = (double *)malloc(sizeof(double) * (size_t)nc);
        dwgo_gwn(n, p, n_old, a, nc, cpos, prm->kernel, prm->eps, prm->lambda, prm->delta, wc,
                 NULL);
        nf = dwgo_faces(nl, leaves, d, cube, nc, keys, wc, iso, NULL, 0);
        double *faces = (double *)malloc(sizeof(double) * 6 * (size_t)(nf > 0 ? nf : 1));
        dwgo_faces(nl, leaves, d, cube, nc, keys, wc, iso, faces, nf);
        dwgo_scatter_normals(n, p, nf, faces, prm->knn, n_old, n_new);
        free(faces);
        free(wc);
        free(cpos);
        free(keys);
        free(leaves);
    } else {
        for (int64_t i = 0; i < n; ++i) {
            const double *gi = g + 3 * i;
            double len = sqrt(gi[0] * gi[0] + gi[1] * gi[1] + gi[2] * gi[2]);
            for (int c = 0; c < 3; ++c)
                n_new[3 * i + c] = (len > 0.0 && isfinite(len)) ? -gi[c] / len : n_old[3 * i + c];
        }
    }
    for (int64_t i = 0; i < n; ++i) dtheta[i] = angle_deg(n_old + 3 * i, n_new + 3 * i);
    if (!gp) free(g);
    return nf;
}

/*
 * Algorithm 1: iterate from n0 until the mean of the largest 1% of the
 * normal changes is <= tol degrees (rule 0, Sec. 5.1) -- or, with rule 1,
 * until the mean over all points of |n_new - n_old| (the quantity plotted in
 * Fig. 6) is <= 2 sin(tol / 2), the chord of tol degrees -- or max_iters
 * iterations.  Writes the
 * final normals, the number of iterations performed, and per-iteration
 * traces of the iso-value and of the convergence statistic (max_iters
 * entries each, may be NULL).  Returns 1 if converged, 0 otherwise.
 */
int dwgo_orient(int64_t n, const double *p, const double *a, const double *n0,
                const dwgo_params *prm, double *n_out, int *iters, double *trace_iso,
                double *trace_stat)
{
    double *cur = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *nxt = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *dth = (double *)malloc(sizeof(double) * (size_t)n);
    double *wp = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(cur, n0, sizeof(double) * 3 * (size_t)n);
    int conv = 0, t = 0;
    while (t < prm->max_iters) {
        double iso;
        dwgo_iterate(n, p, a, cur, prm, nxt, dth, wp, NULL, &iso);
        double stat = dwgo_top1_mean(n, dth);
        double mean_dn = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double dx = nxt[3 * i] - cur[3 * i], dy = nxt[3 * i + 1] - cur[3 * i + 1],
                   dz = nxt[3 * i + 2] - cur[3 * i + 2];
            mean_dn += sqrt(dx * dx + dy * dy + dz * dz);
        }
        mean_dn /= (double)n;
        if (trace_iso) trace_iso[t] = iso;
        if (trace_stat) trace_stat[t] = stat;
        double *sw = cur; cur = nxt; nxt = sw;
        ++t;
        int met = prm->rule == 1 ? mean_dn <= 2.0 * sin(prm->tol * DWGO_PI / 360.0)
                                 : stat <= prm->tol;
        if (met) { conv = 1; break; }
    }
    memcpy(n_out, cur, sizeof(double) * 3 * (size_t)n);
    *iters = t;
    free(wp); free(dth); free(nxt); free(cur);
    return conv;
}

/* ------------------------------------------------------------------------ */
/* Barnes-Hut far field (Sec. 5.2 "Octree Traversal")                        */
/* ------------------------------------------------------------------------ */

/*
 * The hierarchy: the input points sorted along the Morton curve of the root
 * cube (21 bits per axis, stable, ties in input order), cut into buckets of
 * `bucket` consecutive points; a complete binary tree over the buckets (heap
 * order: node 1 is the root, node k has children 2k and 2k+1, the 2^L leaves
 * are the buckets, the last ones possibly empty).  Each node is a contiguous
 * Morton range, like an octree node refined at bucket granularity.
 *
 * Node data, all sums in double, leaves summed sequentially in sorted order
 * and internal nodes as (left + right):
 *   A = sum a_i,  c = sum a_i p_i / A  ("mass center", area weighted),
 *   r = max |p_i - c| over a leaf's points, and for an internal node
 *       max over its non-empty children of |c_child - c| + r_child (an upper
 *       bound of the largest distance, so the opening test is conservative),
 *   M = sum a_i n_i  (the node's area-weighted normal, Sec. 5.2).
 * A query q uses node as one dipole at c with moment M when it is far:
 *   |q - c|^2 > (beta r)^2, evaluated in float32 as
 *   dx = q - c_f (each axis), d2 = fma(dz, dz, fma(dy, dy, dx * dx)),
 *   far iff d2 > br2_f, with c_f = (float)c and br2_f = (float)((beta r)^2);
 * otherwise it descends, and a leaf's points are summed exactly.  beta is the
 * inverse opening angle (Sec. 5.2 uses 2.3).
 */
typedef struct {
    int L;               /* leaves = 2^L */
    int64_t nleaf, n;
    int bucket;
    int64_t *order;      /* sorted index -> input index */
    double *A, *c, *r;   /* per node */
    double *M;           /* per node, 3 */
    float *cf, *br2;     /* per node */
} bh_tree;

typedef struct { uint64_t key; int64_t idx; } key_idx;

static int cmp_key_idx(const void *a, const void *b)
{
    const key_idx *x = (const key_idx *)a, *y = (const key_idx *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static uint64_t spread21(uint64_t v)
{
    uint64_t out = 0;
    for (int b = 0; b < 21; ++b) out |= ((v >> b) & 1ull) << (3 * b);
    return out;
}

/* Morton order of the points in the root cube (21 bits per axis) */
void dwgo_morton_order(int64_t n, const double *p, int64_t *order)
{
    double cube[6];
    dwgo_cube(n, p, 21, cube);
    key_idx *ki = (key_idx *)malloc(sizeof(key_idx) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t cx = (uint64_t)cell_of(p[3 * i + 0], cube[0], cube[5], 21);
        uint64_t cy = (uint64_t)cell_of(p[3 * i + 1], cube[1], cube[5], 21);
        uint64_t cz = (uint64_t)cell_of(p[3 * i + 2], cube[2], cube[5], 21);
        ki[i].key = spread21(cx) | (spread21(cy) << 1) | (spread21(cz) << 2);
        ki[i].idx = i;
    }
    qsort(ki, (size_t)n, sizeof(key_idx), cmp_key_idx);
    for (int64_t i = 0; i < n; ++i) order[i] = ki[i].idx;
    free(ki);
}

/* delta (n, input order, or NULL): clamp radii of the modified kernel.  A
 * node then opens unless the query is farther than both beta r and
 * r + delta_max from its centre, delta_max the largest radius of its points
 * (as sqrt of the float32-rounded delta^2 the kernel stores), so a far
 * node never holds a point whose radius reaches the query. */
static void bh_build(bh_tree *T, int64_t n, const double *p, const double *nrm, const double *a,
                     int bucket, double beta, const double *delta)
{
    T->n = n;
    T->bucket = bucket;
    int64_t nb = (n + bucket - 1) / bucket;
    int L = 0;
    while (((int64_t)1 << L) < nb) ++L;
    T->L = L;
    T->nleaf = (int64_t)1 << L;
    int64_t nn = 2 * T->nleaf;
    T->order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    dwgo_morton_order(n, p, T->order);
    T->A = (double *)calloc((size_t)nn, sizeof(double));
    T->c = (double *)calloc(3 * (size_t)nn, sizeof(double));
    T->r = (double *)calloc((size_t)nn, sizeof(double));
    T->M = (double *)calloc(3 * (size_t)nn, sizeof(double));
    T->cf = (float *)calloc(3 * (size_t)nn, sizeof(float));
    T->br2 = (float *)calloc((size_t)nn, sizeof(float));
    double *Sp = (double *)calloc(3 * (size_t)nn, sizeof(double));
    /* leaves */
    for (int64_t b = 0; b < T->nleaf; ++b) {
        int64_t node = T->nleaf + b, j0 = b * bucket, j1 = j0 + bucket < n ? j0 + bucket : n;
        double sa = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
        for (int64_t j = j0; j < j1; ++j) {
            int64_t i = T->order[j];
            sa = sa + a[i];
            sx = sx + a[i] * p[3 * i]; sy = sy + a[i] * p[3 * i + 1]; sz = sz + a[i] * p[3 * i + 2];
            mx = mx + a[i] * nrm[3 * i]; my = my + a[i] * nrm[3 * i + 1]; mz = mz + a[i] * nrm[3 * i + 2];
        }
        T->A[node] = sa;
        Sp[3 * node] = sx; Sp[3 * node + 1] = sy; Sp[3 * node + 2] = sz;
        T->M[3 * node] = mx; T->M[3 * node + 1] = my; T->M[3 * node + 2] = mz;
    }
    for (int64_t node = T->nleaf - 1; node >= 1; --node) {
        int64_t l = 2 * node, rr = 2 * node + 1;
        T->A[node] = T->A[l] + T->A[rr];
        for (int k = 0; k < 3; ++k) {
            Sp[3 * node + k] = Sp[3 * l + k] + Sp[3 * rr + k];
            T->M[3 * node + k] = T->M[3 * l + k] + T->M[3 * rr + k];
        }
    }
    for (int64_t node = 1; node < nn; ++node)
        if (T->A[node] > 0.0)
            for (int k = 0; k < 3; ++k) T->c[3 * node + k] = Sp[3 * node + k] / T->A[node];
    /* radii: leaves exact, internal nodes bounded through the children */
    for (int64_t b = 0; b < T->nleaf; ++b) {
        int64_t node = T->nleaf + b, j0 = b * bucket, j1 = j0 + bucket < n ? j0 + bucket : n;
        double rm = 0.0;
        for (int64_t j = j0; j < j1; ++j) {
            int64_t i = T->order[j];
            double dx = p[3 * i] - T->c[3 * node], dy = p[3 * i + 1] - T->c[3 * node + 1],
                   dz = p[3 * i + 2] - T->c[3 * node + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (d > rm) rm = d;
        }
        T->r[node] = rm;
    }
    for (int64_t node = T->nleaf - 1; node >= 1; --node) {
        double rm = 0.0;
        for (int64_t ch = 2 * node; ch <= 2 * node + 1; ++ch) {
            if (!(T->A[ch] > 0.0)) continue;
            double dx = T->c[3 * ch] - T->c[3 * node], dy = T->c[3 * ch + 1] - T->c[3 * node + 1],
                   dz = T->c[3 * ch + 2] - T->c[3 * node + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz) + T->r[ch];
            if (d > rm) rm = d;
        }
        T->r[node] = rm;
    }
    double *dmax = NULL;
    if (delta) {
        dmax = (double *)calloc((size_t)nn, sizeof(double));
        for (int64_t b = 0; b < T->nleaf; ++b) {
            int64_t node = T->nleaf + b, j0 = b * bucket, j1 = j0 + bucket < n ? j0 + bucket : n;
            for (int64_t j = j0; j < j1; ++j) {
                double d = sqrt((double)(float)(delta[T->order[j]] * delta[T->order[j]]));
                if (d > dmax[node]) dmax[node] = d;
            }
        }
        for (int64_t node = T->nleaf - 1; node >= 1; --node)
            dmax[node] = dmax[2 * node] > dmax[2 * node + 1] ? dmax[2 * node] : dmax[2 * node + 1];
    }
    for (int64_t node = 1; node < nn; ++node) {
        for (int k = 0; k < 3; ++k) T->cf[3 * node + k] = (float)T->c[3 * node + k];
        double br = beta * T->r[node];
        if (dmax && T->r[node] + dmax[node] > br) br = T->r[node] + dmax[node];
        T->br2[node] = (float)(br * br);
    }
    free(dmax);
    free(Sp);
}

static void bh_free(bh_tree *T)
{
    free(T->order); free(T->A); free(T->c); free(T->r); free(T->M); free(T->cf); free(T->br2);
}

/* far-field term of a node: a dipole of moment M at c_f (float-rounded
 * position and moment M / (4 pi) rounded to float, as the library stores
 * them), kernel evaluated in double */
static void dipole_term(const float *cf, const double *M, const double *q, int screened, double eps,
                        double s, double *t, double g[3])
{
    double pc[3] = {(double)cf[0], (double)cf[1], (double)cf[2]};
    double m[3], one[3];
    for (int k = 0; k < 3; ++k) m[k] = (double)(float)(M[k] / (4.0 * DWGO_PI));
    /* term() builds m = a n / (4 pi); pass a = 4 pi and n = m so that it
     * rebuilds exactly m up to one rounding of (4 pi m) / (4 pi) */
    double nrm_len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    if (nrm_len == 0.0) { *t = 0.0; g[0] = g[1] = g[2] = 0.0; return; }
    for (int k = 0; k < 3; ++k) one[k] = m[k] / nrm_len;
    term(pc, one, nrm_len * 4.0 * DWGO_PI, q, screened, eps, 0.0, s, t, g);
}

static int far_test(const bh_tree *T, int64_t node, const double *q)
{
    float qx = (float)q[0], qy = (float)q[1], qz = (float)q[2];
    float dx = qx - T->cf[3 * node], dy = qy - T->cf[3 * node + 1], dz = qz - T->cf[3 * node + 2];
    float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    return d2 > T->br2[node];
}

static void bh_query(const bh_tree *T, int64_t node, const double *p, const double *nrm,
                     const double *a, const double *delta, const double *q, int screened,
                     double eps, double s, double *w, double g[3], double *count, double *bound)
{
    if (!(T->A[node] > 0.0)) return; /* empty */
    if (far_test(T, node, q)) {
        double t, gt[3];
        dipole_term(T->cf + 3 * node, T->M + 3 * node, q, screened, eps, s, &t, gt);
        *w += t;
        g[0] += gt[0]; g[1] += gt[1]; g[2] += gt[2];
        *count += 1.0;
        if (bound) {
            double dx = q[0] - T->c[3 * node], dy = q[1] - T->c[3 * node + 1],
                   dz = q[2] - T->c[3 * node + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz) - T->r[node];
            *bound += T->A[node] * T->r[node] / (2.0 * DWGO_PI * d * d * d);
        }
        return;
    }
    if (node >= T->nleaf) {
        int64_t b = node - T->nleaf, j0 = b * T->bucket;
        int64_t j1 = j0 + T->bucket < T->n ? j0 + T->bucket : T->n;
        for (int64_t j = j0; j < j1; ++j) {
            int64_t i = T->order[j];
            const double *pi = p + 3 * i;
            if (pi[0] == q[0] && pi[1] == q[1] && pi[2] == q[2]) continue;
            double t, gt[3];
            term(pi, nrm + 3 * i, a[i], q, screened, eps, delta ? delta[i] : 0.0, s, &t, gt);
            *w += t;
            g[0] += gt[0]; g[1] += gt[1]; g[2] += gt[2];
            *count += 1.0;
        }
        return;
    }
    bh_query(T, 2 * node, p, nrm, a, delta, q, screened, eps, s, w, g, count, bound);
    bh_query(T, 2 * node + 1, p, nrm, a, delta, q, screened, eps, s, w, g, count, bound);
}

/*
 * Barnes-Hut w and grad w at m queries (Sec. 5.2) with buckets of `bucket`
 * points and opening factor beta = 1 / theta.  count (m, may be NULL):
 * kernel evaluations per query (points plus far nodes).  bound (m, may be
 * NULL): sum over far nodes of A r / (2 pi (|q - c| - r)^3), a bound of the
 * plain kernel's first-order far-field error for eps -> 0.
 */
void dwgo_tree_gwn(int64_t n, const double *p, const double *nrm, const double *a, int64_t m,
                   const double *q, int kernel, double eps, double lambda, double beta,
                   int bucket, const double *delta, double *w, double *g, double *count,
                   double *bound)
{
    bh_tree T;
    bh_build(&T, n, p, nrm, a, bucket, beta, delta);
    double s = sqrt(lambda > 0 ? lambda : 0.0);
    int screened = (kernel == 1);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        double wi = 0.0, gi[3] = {0, 0, 0}, ci = 0.0, bi = 0.0;
        bh_query(&T, 1, p, nrm, a, delta, q + 3 * i, screened, eps, s, &wi, gi, &ci,
                 bound ? &bi : NULL);
        w[i] = wi;
        if (g) { g[3 * i] = gi[0]; g[3 * i + 1] = gi[1]; g[3 * i + 2] = gi[2]; }
        if (count) count[i] = ci;
        if (bound) bound[i] = bi;
    }
    bh_free(&T);
}

/*
 * The same far field with the opening test applied to groups of queries (a
 * conservative form of the test of Sec. 5.2).  The queries are cut into
 * groups of `group` consecutive queries in the given order.  A node is far
 * for a whole group when the squared distance from its float centre c_f to
 * the group's bounding box (of the float32 query coordinates) exceeds
 * br2_f, in float32:
 *   e_x = max(max(lo_x - c_x, c_x - hi_x), 0) for each axis,
 *   d2 = fma(e_z, e_z, fma(e_y, e_y, e_x * e_x)),  far iff d2 > br2_f.
 * Far for the box implies far for every query in it, so every far node a
 * query uses is one the per-query test would accept, or a descendant of one;
 * since a node's first-order bound A r / (2 pi (d - r)^3) is at least the sum
 * of its children's, each query's error bound is at most its per-query bound.
 * Every query of a group sums the same far nodes and the same leaves; a leaf
 * point equal to the query is skipped as in the exact sum.
 */
typedef struct {
    int64_t *far, *near;
    int64_t nfar, nnear, cap_far, cap_near;
} group_lists;

static void push_id(int64_t **v, int64_t *cnt, int64_t *cap, int64_t id)
{
    if (*cnt == *cap) {
        *cap = *cap ? 2 * *cap : 256;
        *v = (int64_t *)realloc(*v, sizeof(int64_t) * (size_t)*cap);
    }
    (*v)[(*cnt)++] = id;
}

static void bh_group_lists(const bh_tree *T, int64_t node, const float lo[3], const float hi[3],
                           group_lists *L)
{
    if (!(T->A[node] > 0.0)) return; /* empty */
    const float *c = T->cf + 3 * node;
    float ex = fmaxf(fmaxf(lo[0] - c[0], c[0] - hi[0]), 0.0f);
    float ey = fmaxf(fmaxf(lo[1] - c[1], c[1] - hi[1]), 0.0f);
    float ez = fmaxf(fmaxf(lo[2] - c[2], c[2] - hi[2]), 0.0f);
    float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
    if (d2 > T->br2[node]) {
        push_id(&L->far, &L->nfar, &L->cap_far, node);
        return;
    }
    if (node >= T->nleaf) {
        push_id(&L->near, &L->nnear, &L->cap_near, node);
        return;
    }
    bh_group_lists(T, 2 * node, lo, hi, L);
    bh_group_lists(T, 2 * node + 1, lo, hi, L);
}

void dwgo_tree_gwn_group(int64_t n, const double *p, const double *nrm, const double *a,
                         int64_t m, const double *q, int kernel, double eps, double lambda,
                         double beta, int bucket, int group, const double *delta, double *w,
                         double *g, double *count)
{
    bh_tree T;
    bh_build(&T, n, p, nrm, a, bucket, beta, delta);
    double s = sqrt(lambda > 0 ? lambda : 0.0);
    int screened = (kernel == 1);
    int64_t ngroups = (m + group - 1) / group;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t gi = 0; gi < ngroups; ++gi) {
        int64_t i0 = gi * group, i1 = i0 + group < m ? i0 + group : m;
        float lo[3], hi[3];
        for (int k = 0; k < 3; ++k) lo[k] = hi[k] = (float)q[3 * i0 + k];
        for (int64_t i = i0; i < i1; ++i)
            for (int k = 0; k < 3; ++k) {
                float v = (float)q[3 * i + k];
                if (v < lo[k]) lo[k] = v;
                if (v > hi[k]) hi[k] = v;
            }
        group_lists L = {NULL, NULL, 0, 0, 0, 0};
        bh_group_lists(&T, 1, lo, hi, &L);
        for (int64_t i = i0; i < i1; ++i) {
            const double *qi = q + 3 * i;
            double wi = 0.0, gq[3] = {0, 0, 0}, ci = 0.0, t, gt[3];
            for (int64_t f = 0; f < L.nfar; ++f) {
                int64_t node = L.far[f];
                dipole_term(T.cf + 3 * node, T.M + 3 * node, qi, screened, eps, s, &t, gt);
                wi += t;
                gq[0] += gt[0]; gq[1] += gt[1]; gq[2] += gt[2];
                ci += 1.0;
            }
            for (int64_t e = 0; e < L.nnear; ++e) {
                int64_t b = L.near[e] - T.nleaf, j0 = b * T.bucket;
                int64_t j1 = j0 + T.bucket < T.n ? j0 + T.bucket : T.n;
                for (int64_t j = j0; j < j1; ++j) {
                    int64_t k = T.order[j];
                    const double *pk = p + 3 * k;
                    if (pk[0] == qi[0] && pk[1] == qi[1] && pk[2] == qi[2]) continue;
                    term(pk, nrm + 3 * k, a[k], qi, screened, eps, delta ? delta[k] : 0.0, s,
                         &t, gt);
                    wi += t;
                    gq[0] += gt[0]; gq[1] += gt[1]; gq[2] += gt[2];
                    ci += 1.0;
                }
            }
            w[i] = wi;
            if (g) { g[3 * i] = gq[0]; g[3 * i + 1] = gq[1]; g[3 * i + 2] = gq[2]; }
            if (count) count[i] = ci;
        }
        free(L.far);
        free(L.near);
    }
    bh_free(&T);
}
