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
 *     per-point normal changes, in degrees, compared with eps (0.1 deg).
 *
 * All arithmetic is double precision.  Build with -ffp-contract=off so that
 * a*b+c is never fused: the cell-quantisation step below must round exactly
 * like the CUDA side's explicit __dmul_rn/__dsub_rn sequence.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DWGO_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Eq. 2/3 and Eq. 5: w(q) and grad_q w(q)                                  */
/* ------------------------------------------------------------------------ */

/*
 * One source term and its gradient with respect to q.
 *   d = p - q, rho^2 = |d|^2 + eps^2, m = a n / (4 pi), phi = <m, d> / rho^3.
 *   plain:    t = phi,                grad t = -m / rho^3 + 3 phi d / rho^2
 *   screened: F = exp(-s rho)(1 + s rho), s = sqrt(lambda)
 *             t = F phi,              grad t = F grad(phi) + phi s^2 exp(-s rho) d
 * (grad_q rho = -d / rho and dF/drho = -s^2 rho exp(-s rho)).
 */
static void term(const double *p, const double *nrm, double a, const double *q,
                 int screened, double eps, double s, double *t, double g[3])
{
    double d[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    double m[3] = {a * nrm[0] / (4.0 * DWGO_PI), a * nrm[1] / (4.0 * DWGO_PI),
                   a * nrm[2] / (4.0 * DWGO_PI)};
    double rho2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps * eps;
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
        double gphi = -m[k] / rho3 + 3.0 * phi * d[k] / rho2;
        g[k] = F * gphi + phi * s * s * E * d[k];
    }
}

/*
 * w and grad w at m queries from n oriented, weighted points.
 *   p, nrm: n x 3 row-major; a: n weights (Sec. 3: Voronoi areas, or 1);
 *   q: m x 3; kernel 0 = plain (Eq. 2/3), 1 = screened (Eq. 5);
 *   w: m outputs; g: m x 3 outputs or NULL.
 * Terms with p_j == q exactly (all three coordinates) are skipped.
 */
void dwgo_gwn(int64_t n, const double *p, const double *nrm, const double *a,
              int64_t m, const double *q, int kernel, double eps, double lambda,
              double *w, double *g)
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
            term(pj, nrm + 3 * j, a[j], qi, screened, eps, s, &t, gt);
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
    dwgo_gwn(n, p, n_old, a, n, p, prm->kernel, prm->eps, prm->lambda, wp, g);
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
        dwgo_gwn(n, p, n_old, a, nc, cpos, prm->kernel, prm->eps, prm->lambda, wc, NULL);
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
 * normal changes is <= tol degrees, or max_iters iterations.  Writes the
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
        if (trace_iso) trace_iso[t] = iso;
        if (trace_stat) trace_stat[t] = stat;
        double *sw = cur; cur = nxt; nxt = sw;
        ++t;
        if (stat <= prm->tol) { conv = 1; break; }
    }
    memcpy(n_out, cur, sizeof(double) * 3 * (size_t)n);
    *iters = t;
    free(wp); free(dth); free(nxt); free(cur);
    return conv;
}
