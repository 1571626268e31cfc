/*
 * oracle.c -- plain, slow FP64 CPU oracle for synchronized tracing of
 * blobtree implicit surfaces (Zanni 2023, "Synchronized-tracing of implicit
 * surfaces").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code with the CUDA path: it reads the scene description arrays itself and
 * restates every formula from the paper in the most direct form.
 *
 * What it computes (each function cites the passage it follows):
 *   - primitive distance fields (Sec. 4 / Sec. 10 primitives, exact SDFs)
 *   - sharp CSG (Eq. 1-3), smooth polynomial operators (Eq. 4-7) and the
 *     compact smooth operators G_op (Sec. 5, Eq. "smooth_comp" and
 *     "compact_smooth_union", transition function b_r)
 *   - ranges of interest propagated from the root (Sec. 5)
 *   - post-order linearisation, isLeft, ignoreMod (Sec. 4, Sec. 9) and fast
 *     ancestor pointers by their recursive definition (Sec. 7.2, cut at
 *     intersections and right-child -> difference edges, Sec. 9)
 *   - the pruned field f_A of an active set A (Sec. 3 local equivalence,
 *     Sec. 5/9: an absent operand may be taken as +inf) and the pruned
 *     tree view by its plain definition (the tree induced by A, with the
 *     usage rewrite of Sec. 9)
 *   - primitive volumes of interest (Sec. 6.1) and brute-force per-tile
 *     culling (Sec. 6.2) in FP64, and in FP32 with the fixed operation order
 *     that the GPU culling kernel documents (the integer hit decisions are
 *     taken in the same precision on both sides)
 *   - naive dense sphere tracing (Sec. 2.2, Sec. 10) with Newton polish and
 *     central-difference normals, and the over-relaxed variant with sphere
 *     reuse, minimum step and iso-crossing detection that Sec. 10 states
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define K_SPHERE 0
#define K_RBOX 1
#define K_CAPSULE 2
#define K_TORUS 12
#define K_SCONE 13
#define K_ELLIPSOID 14
#define K_RTRI 15
#define K_QUADRIC 11
#define K_UNION 16
#define K_INTER 17
#define K_DIFF 18
#define K_SUNION 19
#define K_SINTER 20
#define K_SDIFF 21

#define NREC 16

typedef struct {
    int n, root;
    const int32_t *kind, *left, *right;
    const float *params;
    int *parent;   /* desc-indexed, -1 for the root */
    int *isleft;   /* desc-indexed, 1 if the node is a left child */
} Tree;

static int is_prim(int k) { return k < 16; }

static void tree_init(Tree *t, int n, int root, const int32_t *kind, const int32_t *left,
                      const int32_t *right, const float *params) {
    t->n = n; t->root = root; t->kind = kind; t->left = left; t->right = right;
    t->params = params;
    t->parent = (int *)malloc(sizeof(int) * (size_t)n);
    t->isleft = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) { t->parent[i] = -1; t->isleft[i] = 0; }
    for (int i = 0; i < n; ++i) {
        if (!is_prim(kind[i])) {
            t->parent[left[i]] = i; t->isleft[left[i]] = 1;
            t->parent[right[i]] = i; t->isleft[right[i]] = 0;
        }
    }
}

static void tree_free(Tree *t) { free(t->parent); free(t->isleft); }

/* ------------------------------------------------------------------------ */
/* Primitive distance fields (exact SDFs, Lipschitz 1).                      */

static double sdf_sphere(const float *q, const double p[3]) {
    double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    return sqrt(dx * dx + dy * dy + dz * dz) - (double)q[3];
}

/* Rounded box: q = |M (p - c)| - b ; |max(q, 0)| + min(max_i q_i, 0) - r. */
static double sdf_rbox(const float *q, const double p[3]) {
    double w[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    double a[3], out = 0.0, mx = -DBL_MAX;
    for (int i = 0; i < 3; ++i) {
        double l = q[3 + 3 * i] * w[0] + q[4 + 3 * i] * w[1] + q[5 + 3 * i] * w[2];
        a[i] = fabs(l) - (double)q[12 + i];
        if (a[i] > 0) out += a[i] * a[i];
        if (a[i] > mx) mx = a[i];
    }
    return sqrt(out) + (mx < 0 ? mx : 0.0) - (double)q[15];
}

/* Capsule: distance to segment [a, b] minus radius. */
static double sdf_capsule(const float *q, const double p[3]) {
    double pa[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    double ba[3] = {(double)q[3] - q[0], (double)q[4] - q[1], (double)q[5] - q[2]};
    double bb = ba[0] * ba[0] + ba[1] * ba[1] + ba[2] * ba[2];
    double h = bb > 0 ? (pa[0] * ba[0] + pa[1] * ba[1] + pa[2] * ba[2]) / bb : 0.0;
    if (h < 0) h = 0;
    if (h > 1) h = 1;
    double dx = pa[0] - h * ba[0], dy = pa[1] - h * ba[1], dz = pa[2] - h * ba[2];
    return sqrt(dx * dx + dy * dy + dz * dz) - (double)q[6];
}

/* Unit vector of a record's axis (FP64). */
static void unit3(const float *a, double u[3]) {
    double n = sqrt((double)a[0] * a[0] + (double)a[1] * a[1] + (double)a[2] * a[2]);
    for (int k = 0; k < 3; ++k) u[k] = a[k] / n;
}

/* Torus: points within r of the circle of radius R around the axis through
 * c; distance to that circle minus r.  The circle's nearest point lies in the
 * direction of p's component perpendicular to the axis. */
static double sdf_torus(const float *q, const double p[3]) {
    double ax[3], v[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    unit3(q + 3, ax);
    double h = v[0] * ax[0] + v[1] * ax[1] + v[2] * ax[2];
    double w[3] = {v[0] - h * ax[0], v[1] - h * ax[1], v[2] - h * ax[2]};
    double rho = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double dr = rho - (double)q[6];
    return sqrt(dr * dr + h * h) - (double)q[7];
}

/* Sphere-cone: the convex hull of the balls (a, r_a) and (b, r_b).  In the
 * plane through the axis, with y along the axis from a, x >= 0 the distance to
 * it and h = |b - a|, the hull's side is tangent to both circles: outward
 * normal n = (cos, sin) with sin = (r_a - r_b) / h, tangent points at
 * parameter 0 and cos h along the side.  Nearest feature: ball a behind the
 * first tangent point, ball b beyond the second, the side in between. */
static double sdf_scone(const float *q, const double p[3]) {
    double ba[3] = {(double)q[3] - q[0], (double)q[4] - q[1], (double)q[5] - q[2]};
    double h = sqrt(ba[0] * ba[0] + ba[1] * ba[1] + ba[2] * ba[2]);
    double ra = q[6], rb = q[7];
    double sn = (ra - rb) / h, cs = sqrt(1.0 - sn * sn);
    double v[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    double y = (v[0] * ba[0] + v[1] * ba[1] + v[2] * ba[2]) / h;
    double w[3] = {v[0] - y * ba[0] / h, v[1] - y * ba[1] / h, v[2] - y * ba[2] / h};
    double x = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double lam = cs * y - sn * x;   /* position along the side */
    if (lam < 0.0) return sqrt(x * x + y * y) - ra;
    if (lam > cs * h) return sqrt(x * x + (y - h) * (y - h)) - rb;
    return cs * x + sn * y - ra;
}

/* Ellipsoid (c, M world -> local, radii r): the Lipschitz-1 bound
 * min(r) (|M (p - c) / r| - 1); zero exactly on the ellipsoid, negative
 * inside, and never above the distance to it. */
static double sdf_ellipsoid(const float *q, const double p[3]) {
    double w[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    double s = 0.0, rmin = q[12];
    for (int i = 0; i < 3; ++i) {
        double l = q[3 + 3 * i] * w[0] + q[4 + 3 * i] * w[1] + q[5 + 3 * i] * w[2];
        double z = l / (double)q[12 + i];
        s += z * z;
        if (q[12 + i] < rmin) rmin = q[12 + i];
    }
    return rmin * (sqrt(s) - 1.0);
}

/* Rounded triangle (vertices a, b, c, rounding r): Euclidean distance to the
 * triangle minus r.  The nearest point of the triangle is the orthogonal
 * projection onto its plane when that projection falls inside (p on the
 * inner side of all three edges, tested with the normal N = (b-a) x (c-a)),
 * otherwise the nearest point of the nearest edge segment. */
static double seg_dist(const double p[3], const double a[3], const double b[3]) {
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    double t = (ap[0] * ab[0] + ap[1] * ab[1] + ap[2] * ab[2]) / (ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    double x = ap[0] - t * ab[0], y = ap[1] - t * ab[1], z = ap[2] - t * ab[2];
    return sqrt(x * x + y * y + z * z);
}
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double sdf_rtri(const float *q, const double p[3]) {
    double v[3][3];
    for (int i = 0; i < 3; ++i) for (int k = 0; k < 3; ++k) v[i][k] = q[3 * i + k];
    double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
    double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
    double N[3];
    cross3(e1, e2, N);
    int inside = 1;
    for (int i = 0; i < 3; ++i) {
        const double *s = v[i], *t = v[(i + 1) % 3];
        double ed[3] = {t[0] - s[0], t[1] - s[1], t[2] - s[2]}, sp[3] = {p[0] - s[0], p[1] - s[1], p[2] - s[2]};
        double c[3];
        cross3(ed, sp, c);   /* along +N when p is on the inner side of edge s -> t */
        if (c[0] * N[0] + c[1] * N[1] + c[2] * N[2] < 0) inside = 0;
    }
    double dist;
    if (inside) {
        double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        dist = fabs((p[0] - v[0][0]) * N[0] + (p[1] - v[0][1]) * N[1] + (p[2] - v[0][2]) * N[2]) / nn;
    } else {
        dist = seg_dist(p, v[0], v[1]);
        double d1 = seg_dist(p, v[1], v[2]), d2 = seg_dist(p, v[2], v[0]);
        if (d1 < dist) dist = d1;
        if (d2 < dist) dist = d2;
    }
    return dist - (double)q[9];
}

/* Bounded quadric: the solid {q(u) <= 0} of q(u) = alpha u0^2 + beta u1^2 +
 * gamma u2^2 + delta u2 + kappa, clipped by the box |u_i| <= e_i, in the local
 * frame u = R^T (p - c) of the unit quaternion's rotation R.  Its field:
 * max(q(clamp(u)) / G, box distance), G = |(2|alpha| e0, 2|beta| e1,
 * 2|gamma| e2 + |delta|)| bounding |grad q| on the box, so that q / G is
 * 1-Lipschitz there and its clamped extension is 1-Lipschitz everywhere; the
 * zero set is exactly the boundary of {q <= 0} inside the box. */
static void quat_rot(const float *qq, double R[3][3]) {
    double w = qq[0], x = qq[1], y = qq[2], z = qq[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - z * w);     R[0][2] = 2 * (x * z + y * w);
    R[1][0] = 2 * (x * y + z * w);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - x * w);
    R[2][0] = 2 * (x * z - y * w);     R[2][1] = 2 * (y * z + x * w);     R[2][2] = 1 - 2 * (x * x + y * y);
}
static double quadric_g(const float *q) {
    double g0 = 2.0 * fabs((double)q[10]) * q[7], g1 = 2.0 * fabs((double)q[11]) * q[8];
    double g2 = 2.0 * fabs((double)q[12]) * q[9] + fabs((double)q[13]);
    return sqrt(g0 * g0 + g1 * g1 + g2 * g2);
}
static double sdf_quadric(const float *q, const double p[3]) {
    double R[3][3];
    quat_rot(q + 3, R);
    double w[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]}, u[3], uc[3];
    double out = 0.0, mx = -DBL_MAX;
    for (int i = 0; i < 3; ++i) {
        u[i] = R[0][i] * w[0] + R[1][i] * w[1] + R[2][i] * w[2];   /* (R^T w)_i */
        double e = q[7 + i];
        uc[i] = u[i] < -e ? -e : (u[i] > e ? e : u[i]);
        double a = fabs(u[i]) - e;
        if (a > 0) out += a * a;
        if (a > mx) mx = a;
    }
    double box = sqrt(out) + (mx < 0 ? mx : 0.0);
    double qv = q[10] * uc[0] * uc[0] + q[11] * uc[1] * uc[1] + q[12] * uc[2] * uc[2] + q[13] * uc[2] + q[14];
    double f = qv / quadric_g(q);
    return f > box ? f : box;
}

static double sdf_prim(int kind, const float *q, const double p[3]) {
    switch (kind) {
    case K_SPHERE: return sdf_sphere(q, p);
    case K_RBOX: return sdf_rbox(q, p);
    case K_CAPSULE: return sdf_capsule(q, p);
    case K_TORUS: return sdf_torus(q, p);
    case K_SCONE: return sdf_scone(q, p);
    case K_ELLIPSOID: return sdf_ellipsoid(q, p);
    case K_RTRI: return sdf_rtri(q, p);
    case K_QUADRIC: return sdf_quadric(q, p);
    }
    return INFINITY;
}

/* ------------------------------------------------------------------------ */
/* Operators.                                                                */

/* Eq. 5: d(f0, f1, k) = k/6 max(1 - |f0 - f1|/k, 0)^3.  A blend range that
 * is not positive (including the not-a-number case named in Sec. 5) gives
 * no displacement. */
static double disp(double f0, double f1, double k) {
    if (!(k > 0)) return 0.0;
    double x = 1.0 - fabs(f0 - f1) / k;
    if (!(x > 0)) return 0.0;
    return k / 6.0 * x * x * x;
}

/* Eq. 1-3 (sharp CSG). */
static double csg(int op, double f0, double f1) {
    switch (op) {
    case K_UNION: case K_SUNION: return f0 < f1 ? f0 : f1;
    case K_INTER: case K_SINTER: return f0 > f1 ? f0 : f1;
    default: return f0 > -f1 ? f0 : -f1;
    }
}

/* Eq. 4, 6, 7 (smooth polynomial operators with blend range k). */
static double gsmooth(int op, double f0, double f1, double k) {
    switch (op) {
    case K_UNION: return csg(op, f0, f1) - disp(f0, f1, k);
    case K_INTER: return csg(op, f0, f1) + disp(f0, f1, k);
    default: return csg(op, f0, f1) + disp(f0, -f1, k);
    }
}

/* Sec. 5: b_r(x, k, d) = k max(1 - 6x / (6d - k), 0). */
static double b_r(double x, double k, double d) {
    double t = 1.0 - 6.0 * x / (6.0 * d - k);
    if (!(t > 0)) return 0.0;
    return k * t;
}

/* Sec. 5, Eq. "smooth_comp": G_op = gbar_op on (-inf, d_o]^2, csg_op outside;
 * gbar_op(f0, f1) = g_op(f0, f1, b_r(g_op(f0, f1, k), k, d_o)), with the blend
 * range bounded by k for intersection and difference and taken in absolute
 * value for the difference. */
double or_op(int op, double k, double d_o, double f0, double f1) {
    if (op == K_SUNION || op == K_SINTER || op == K_SDIFF) return csg(op, f0, f1);
    if (!(f0 <= d_o && f1 <= d_o)) return csg(op, f0, f1);
    double kr = b_r(gsmooth(op, f0, f1, k), k, d_o);
    if (op == K_DIFF) kr = fabs(kr);
    if (op != K_UNION && kr > k) kr = k;
    if (isnan(kr)) kr = 0.0;
    return gsmooth(op, f0, f1, kr);
}

/* Plain smooth operator of Eq. 4-7 with fixed k (no compaction). */
double or_smooth(int op, double k, double f0, double f1) { return gsmooth(op, f0, f1, k); }

double or_b_r(double x, double k, double d) { return b_r(x, k, d); }

/* ------------------------------------------------------------------------ */
/* Field evaluation.                                                         */

/* Dense field of the whole blobtree (post-order recursion on the tree).  With
 * ``active`` non-NULL, every primitive with active[node] == 0 contributes
 * +inf: this is the pruned field f_A of Sec. 3 (an operand outside its range
 * of interest may be replaced by an infinite value, Sec. 5 and Sec. 9). */
static double field_rec(const Tree *t, int node, const double p[3], const uint8_t *active) {
    int k = t->kind[node];
    const float *q = t->params + (size_t)node * NREC;
    if (is_prim(k)) {
        if (active && !active[node]) return INFINITY;
        return sdf_prim(k, q, p);
    }
    double f0 = field_rec(t, t->left[node], p, active);
    double f1 = field_rec(t, t->right[node], p, active);
    return or_op(k, q[0], q[1], f0, f1);
}

void or_field(int n, int root, const int32_t *kind, const int32_t *left, const int32_t *right,
              const float *params, const uint8_t *active, int npts, const double *pts,
              double *out) {
    Tree t;
    tree_init(&t, n, root, kind, left, right, params);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < npts; ++i) out[i] = field_rec(&t, root, pts + 3 * (size_t)i, active);
    tree_free(&t);
}

/* ------------------------------------------------------------------------ */
/* Tree structure: post-order, ranges of interest, fast ancestor pointers.   */

static void postorder_rec(const Tree *t, int node, int *counter, int *po) {
    if (!is_prim(t->kind[node])) {
        postorder_rec(t, t->left[node], counter, po);
        postorder_rec(t, t->right[node], counter, po);
    }
    po[node] = (*counter)++;
}

/* Sec. 5: the root's range of interest is (-inf, 0]; an operator passes
 * R_o U R_p to its children (R_o = (-inf, d_o] for compact smooth operators,
 * empty for sharp CSG). */
static void roi_rec(const Tree *t, int node, double d_node, double *roi) {
    roi[node] = d_node;
    int k = t->kind[node];
    if (is_prim(k)) return;
    double dc = d_node;
    if (k == K_UNION || k == K_INTER || k == K_DIFF) {
        double d_o = t->params[(size_t)node * NREC + 1];
        if (d_o > dc) dc = d_o;
    }
    roi_rec(t, t->left[node], dc, roi);
    roi_rec(t, t->right[node], dc, roi);
}

/* Sec. 9 ignoreMod: 00 union-like, 10 difference-like (ignore if the left
 * operand is absent), 11 intersection-like. */
static int ignore_mod(int kind) {
    switch (kind) {
    case K_INTER: case K_SINTER: return 3;
    case K_DIFF: case K_SDIFF: return 2;
    default: return 0;
    }
}

/* Whether operator node a passes a lone operand coming from side `from_left`
 * through unchanged (so that an ancestor pointer may jump over it). */
static int passes_through(int kind, int from_left) {
    int m = ignore_mod(kind);
    return !(m & (from_left ? 1 : 2));
}

/* Sec. 7.2 fast ancestor pointers, recursive definition: from node P with
 * parent A, keep climbing while the jump direction (left/right) does not
 * change, never jumping over an intersection nor over a difference reached
 * from its right operand (Sec. 9).  The root has no ancestor (-1). */
static int fast_ancestor(const Tree *t, int p) {
    int a = t->parent[p];
    if (a < 0) return -1;
    if (t->parent[a] < 0) return a;
    if (t->isleft[p] != t->isleft[a]) return a;
    if (!passes_through(t->kind[a], t->isleft[p])) return a;
    return fast_ancestor(t, a);
}

/* Post-order stack depth of Alg. 3 evaluation (max live entries). */
static int stack_rec(const Tree *t, int node) {
    if (is_prim(t->kind[node])) return 1;
    int a = stack_rec(t, t->left[node]);
    int b = stack_rec(t, t->right[node]) + 1;
    return a > b ? a : b;
}

/* Outputs are indexed by post-order address:
 *   po_of[desc]      post-order address of each description node
 *   parent[po]       parent address, -1 for the root
 *   isleft[po]       1 if left child (root: 0)
 *   igm[po]          ignoreMod
 *   fast[po]         fast ancestor address, -1 for the root
 *   roi[po]          upper bound d_n of the node's range of interest
 * Returns the post-order stack depth of the full tree. */
int or_structure(int n, int root, const int32_t *kind, const int32_t *left, const int32_t *right,
                 const float *params, int32_t *po_of, int32_t *parent, int32_t *isleft,
                 int32_t *igm, int32_t *fast, double *roi) {
    Tree t;
    tree_init(&t, n, root, kind, left, right, params);
    int counter = 0;
    int *po = (int *)malloc(sizeof(int) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    postorder_rec(&t, root, &counter, po);
    roi_rec(&t, root, 0.0, r);
    for (int i = 0; i < n; ++i) {
        int a = po[i];
        po_of[i] = a;
        parent[a] = t.parent[i] < 0 ? -1 : po[t.parent[i]];
        isleft[a] = t.isleft[i];
        igm[a] = is_prim(kind[i]) ? 0 : ignore_mod(kind[i]);
        int f = fast_ancestor(&t, i);
        fast[a] = f < 0 ? -1 : po[f];
        roi[a] = r[i];
    }
    int depth = stack_rec(&t, root);
    free(po); free(r);
    tree_free(&t);
    return depth;
}

/* ------------------------------------------------------------------------ */
/* Pruned tree view by definition (Sec. 8 "local pruned tree view", Sec. 9). */

typedef struct { int32_t *addr, *op; int n; } ViewOut;

/* Returns 1 if the subtree holds an active primitive; *usage receives the
 * usage bit.  Nodes with two present operands are appended in post-order
 * with their operator type rewritten from the operands' usage bits. */
static int view_rec(const Tree *t, int node, const uint8_t *active, const int *po,
                    ViewOut *v, int *usage) {
    int k = t->kind[node];
    if (is_prim(k)) {
        if (!active[node]) { *usage = 0; return 0; }
        v->addr[v->n] = po[node]; v->op[v->n] = 3; v->n++;
        *usage = 1;
        return 1;
    }
    int ul = 0, ur = 0;
    int hl = view_rec(t, t->left[node], active, po, v, &ul);
    int hr = view_rec(t, t->right[node], active, po, v, &ur);
    if (!hl && !hr) { *usage = 0; return 0; }
    int b, m = ignore_mod(k);
    if (hl && hr) b = (ul << 1) | ur;
    else if (hl) b = ul << 1;
    else b = ur;
    int ok = ((~b) & m & 3) == 0;
    if (hl && hr) { v->addr[v->n] = po[node]; v->op[v->n] = ok ? b : 0; v->n++; }
    *usage = ok && b != 0;
    return 1;
}

/* active[desc] flags; out arrays sized >= 2 * n_active - 1.  op = 3 keeps the
 * node's own operator, 0 = +inf, 1 = right operand, 2 = left operand.
 * Returns the view length; *root_usage gets the root usage bit. */
int or_pruned_view(int n, int root, const int32_t *kind, const int32_t *left,
                   const int32_t *right, const uint8_t *active, int32_t *out_addr,
                   int32_t *out_op, int32_t *root_usage) {
    Tree t;
    tree_init(&t, n, root, kind, left, right, NULL);
    int counter = 0;
    int *po = (int *)malloc(sizeof(int) * (size_t)n);
    postorder_rec(&t, root, &counter, po);
    ViewOut v = {out_addr, out_op, 0};
    int u = 0;
    view_rec(&t, root, active, po, &v, &u);
    *root_usage = u;
    free(po);
    tree_free(&t);
    return v.n;
}

/* ------------------------------------------------------------------------ */
/* Volumes of interest and scene bounds.                                     */

/* Sec. 6.1: primitive bounding volume offset by the primitive's range of
 * interest bound d.  Sphere -> sphere (c, r + d); rounded box -> oriented box
 * (c, M, b + r_round + d); capsule -> capsule (a, b, r + d).  The VOI family
 * of the further primitives contains their offset volume {f <= d}: torus ->
 * capped cylinder around its axis (radius R + r + d, half-height r + d, kept
 * as a capsule-shaped record whose ends are the cap centres, tested without
 * the spherical caps); sphere-cone -> capsule (a, b, max(r_a, r_b) + d);
 * ellipsoid -> oriented box (c, M, r (1 + d / min r)), the box around the
 * ellipsoid that {f <= d} is.  Output record: the family's layout (sphere:
 * c, r; box: c, M, e at [12:15]; capsule / cylinder: a, b, r at [6]). */
static void voi_rec(int kind, const float *q, double d, double *v) {
    for (int i = 0; i < NREC; ++i) v[i] = q[i];
    switch (kind) {
    case K_SPHERE: v[3] = (double)q[3] + d; break;
    case K_RBOX:
        for (int i = 0; i < 3; ++i) v[12 + i] = (double)q[12 + i] + (double)q[15] + d;
        break;
    case K_CAPSULE: v[6] = (double)q[6] + d; break;
    case K_TORUS: {
        double ax[3];
        unit3(q + 3, ax);
        double hh = (double)q[7] + d;
        for (int k = 0; k < 3; ++k) { v[k] = q[k] - hh * ax[k]; v[3 + k] = q[k] + hh * ax[k]; }
        v[6] = (double)q[6] + q[7] + d;
        break;
    }
    case K_SCONE: v[6] = (q[6] > q[7] ? (double)q[6] : (double)q[7]) + d; break;
    case K_ELLIPSOID: {
        double rmin = q[12];
        for (int i = 1; i < 3; ++i) if (q[12 + i] < rmin) rmin = q[12 + i];
        for (int i = 0; i < 3; ++i) v[12 + i] = (double)q[12 + i] * (1.0 + d / rmin);
        break;
    }
    case K_RTRI: v[9] = (double)q[9] + d; break;   /* vertices, radius r + d */
    case K_QUADRIC: {   /* oriented box: centre, M = R^T rows, e + d */
        double R[3][3];
        quat_rot(q + 3, R);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) v[3 + 3 * i + j] = R[j][i];
        for (int i = 0; i < 3; ++i) v[12 + i] = (double)q[7 + i] + d;
        break;
    }
    }
}

/* Axis-aligned bounds of a primitive's zero iso-volume. */
static void prim_aabb(int kind, const float *q, double lo[3], double hi[3]) {
    if (kind == K_RTRI) {   /* the vertices' box grown by the rounding */
        for (int j = 0; j < 3; ++j) {
            double a = q[j], b = q[3 + j], c = q[6 + j];
            double mn = a < b ? a : b, mx = a > b ? a : b;
            if (c < mn) mn = c;
            if (c > mx) mx = c;
            lo[j] = mn - q[9]; hi[j] = mx + q[9];
        }
        return;
    }
    if (kind == K_QUADRIC) {   /* inside its clipping box */
        double R[3][3];
        quat_rot(q + 3, R);
        for (int j = 0; j < 3; ++j) {
            double e = 0;
            for (int i = 0; i < 3; ++i) e += fabs(R[j][i]) * q[7 + i];
            lo[j] = q[j] - e; hi[j] = q[j] + e;
        }
        return;
    }
    if (kind == K_SPHERE) {
        for (int j = 0; j < 3; ++j) { lo[j] = q[j] - (double)q[3]; hi[j] = q[j] + (double)q[3]; }
    } else if (kind == K_RBOX) {
        for (int j = 0; j < 3; ++j) {
            double e = 0;
            for (int i = 0; i < 3; ++i) e += fabs((double)q[3 + 3 * i + j]) * ((double)q[12 + i] + q[15]);
            lo[j] = q[j] - e; hi[j] = q[j] + e;
        }
    } else if (kind == K_CAPSULE) {
        for (int j = 0; j < 3; ++j) {
            double a = q[j], b = q[3 + j];
            lo[j] = (a < b ? a : b) - q[6]; hi[j] = (a > b ? a : b) + q[6];
        }
    } else if (kind == K_TORUS) {
        double ax[3];
        unit3(q + 3, ax);
        for (int j = 0; j < 3; ++j) {
            double e = (double)q[6] * sqrt(fmax(0.0, 1.0 - ax[j] * ax[j])) + q[7];
            lo[j] = q[j] - e; hi[j] = q[j] + e;
        }
    } else if (kind == K_SCONE) {
        for (int j = 0; j < 3; ++j) {
            double la = q[j] - (double)q[6], lb = q[3 + j] - (double)q[7];
            double ha = q[j] + (double)q[6], hb = q[3 + j] + (double)q[7];
            lo[j] = la < lb ? la : lb; hi[j] = ha > hb ? ha : hb;
        }
    } else {   /* ellipsoid: inside its oriented box of half extents r */
        for (int j = 0; j < 3; ++j) {
            double e = 0;
            for (int i = 0; i < 3; ++i) e += fabs((double)q[3 + 3 * i + j]) * (double)q[12 + i];
            lo[j] = q[j] - e; hi[j] = q[j] + e;
        }
    }
}

/* Scene bounding box of all primitive bounds; returns its diagonal. */
double or_scene_bounds(int n, const int32_t *kind, const float *params, double *lo, double *hi) {
    for (int j = 0; j < 3; ++j) { lo[j] = DBL_MAX; hi[j] = -DBL_MAX; }
    for (int i = 0; i < n; ++i) {
        if (!is_prim(kind[i])) continue;
        double a[3], b[3];
        prim_aabb(kind[i], params + (size_t)i * NREC, a, b);
        for (int j = 0; j < 3; ++j) {
            if (a[j] < lo[j]) lo[j] = a[j];
            if (b[j] > hi[j]) hi[j] = b[j];
        }
    }
    double s = 0;
    for (int j = 0; j < 3; ++j) s += (hi[j] - lo[j]) * (hi[j] - lo[j]);
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Camera.                                                                   */

typedef struct {
    double o[3], F[3], R[3], U[3];   /* FP64 basis (R, U pre-scaled) */
    float of[3], Ff[3], Rf[3], Uf[3]; /* its FP32 rounding */
    int W, H;
} Cam;

/* Pinhole camera: F = normalize(target - eye), R = normalize(F x up),
 * U = R x F; R is scaled by tan(fov/2) * W/H and U by tan(fov/2).  Pixel
 * (i, j) centre: d = F + u R + v U with u = (2i+1)/W - 1, v = 1 - (2j+1)/H.
 * Points on the ray are o + t d; since d.F = 1, t is the planar view depth. */
static void cam_init(Cam *c, const float *cam) {
    double e[3] = {cam[0], cam[1], cam[2]}, tg[3] = {cam[3], cam[4], cam[5]};
    double up[3] = {cam[6], cam[7], cam[8]};
    double vfov = cam[9];
    c->W = (int)cam[10]; c->H = (int)cam[11];
    double F[3] = {tg[0] - e[0], tg[1] - e[1], tg[2] - e[2]};
    double nf = sqrt((F[0] * F[0] + F[1] * F[1]) + F[2] * F[2]);
    for (int j = 0; j < 3; ++j) F[j] = F[j] / nf;
    double R[3] = {F[1] * up[2] - F[2] * up[1], F[2] * up[0] - F[0] * up[2], F[0] * up[1] - F[1] * up[0]};
    double nr = sqrt((R[0] * R[0] + R[1] * R[1]) + R[2] * R[2]);
    for (int j = 0; j < 3; ++j) R[j] = R[j] / nr;
    double U[3] = {R[1] * F[2] - R[2] * F[1], R[2] * F[0] - R[0] * F[2], R[0] * F[1] - R[1] * F[0]};
    double th = tan(vfov * M_PI / 360.0);
    double aspect = (double)c->W / (double)c->H;
    for (int j = 0; j < 3; ++j) {
        c->o[j] = e[j];
        c->F[j] = F[j];
        c->R[j] = R[j] * th * aspect;
        c->U[j] = U[j] * th;
        c->of[j] = (float)c->o[j];
        c->Ff[j] = (float)c->F[j];
        c->Rf[j] = (float)c->R[j];
        c->Uf[j] = (float)c->U[j];
    }
}

static void cam_ray64(const Cam *c, int i, int j, double d[3]) {
    double u = (2.0 * i + 1.0) / c->W - 1.0, v = 1.0 - (2.0 * j + 1.0) / c->H;
    for (int k = 0; k < 3; ++k) d[k] = c->F[k] + u * c->R[k] + v * c->U[k];
}

/* FP32 ray, fixed order: u = (float)(2i+1) / (float)W - 1,
 * v = 1 - (float)(2j+1) / (float)H, d_k = (F_k + u R_k) + v U_k. */
static void cam_ray32(const Cam *c, int i, int j, float d[3]) {
    float u = (float)(2 * i + 1) / (float)c->W - 1.0f;
    float v = 1.0f - (float)(2 * j + 1) / (float)c->H;
    for (int k = 0; k < 3; ++k) {
        float a = u * c->Rf[k];
        float b = v * c->Uf[k];
        d[k] = (c->Ff[k] + a) + b;
    }
}

void or_camera_rays(const float *cam, int npx, const int32_t *pi, const int32_t *pj,
                    double *d64, float *d32) {
    Cam c;
    cam_init(&c, cam);
    for (int n = 0; n < npx; ++n) {
        if (d64) cam_ray64(&c, pi[n], pj[n], d64 + 3 * (size_t)n);
        if (d32) cam_ray32(&c, pi[n], pj[n], d32 + 3 * (size_t)n);
    }
}

/* ------------------------------------------------------------------------ */
/* Ray / volume-of-interest intervals, FP64 (exact geometry).                */

/* Ray o + t d against sphere (c, r): roots of |o + t d - c|^2 = r^2. */
static int ray_sphere64(const double o[3], const double d[3], const double c[3], double r,
                        double *t0, double *t1) {
    double w[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
    double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double tc = (w[0] * d[0] + w[1] * d[1] + w[2] * d[2]) / dd;
    double h2 = 0;
    for (int k = 0; k < 3; ++k) { double q = w[k] - tc * d[k]; h2 += q * q; }
    if (h2 > r * r) return 0;
    double s = sqrt((r * r - h2) / dd);
    *t0 = tc - s; *t1 = tc + s;
    return 1;
}

/* Ray against oriented box (c, M world->local, half extents e): slabs. */
static int ray_obox64(const double o[3], const double d[3], const double *v, double *t0,
                      double *t1) {
    double lo = -INFINITY, hi = INFINITY;
    double w[3] = {o[0] - v[0], o[1] - v[1], o[2] - v[2]};
    for (int i = 0; i < 3; ++i) {
        const double *m = v + 3 + 3 * i;
        double lo_i = m[0] * w[0] + m[1] * w[1] + m[2] * w[2];
        double ld_i = m[0] * d[0] + m[1] * d[1] + m[2] * d[2];
        double e = v[12 + i];
        if (ld_i == 0.0) {
            if (lo_i < -e || lo_i > e) return 0;
            continue;
        }
        double ta = (-e - lo_i) / ld_i, tb = (e - lo_i) / ld_i;
        double a = ta < tb ? ta : tb, b = ta < tb ? tb : ta;
        if (a > lo) lo = a;
        if (b < hi) hi = b;
    }
    if (lo > hi) return 0;
    *t0 = lo; *t1 = hi;
    return 1;
}

/* Ray against the cylinder of radius r around segment [a, b], capped by the
 * planes through a and b. */
static int ray_cylinder64(const double o[3], const double d[3], const double *v, double *t0,
                          double *t1) {
    double a[3] = {v[0], v[1], v[2]}, b[3] = {v[3], v[4], v[5]}, r = v[6];
    double ba[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double w[3] = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
    double bb = ba[0] * ba[0] + ba[1] * ba[1] + ba[2] * ba[2];
    if (!(bb > 0)) return 0;
    double wb = w[0] * ba[0] + w[1] * ba[1] + w[2] * ba[2];
    double db = d[0] * ba[0] + d[1] * ba[1] + d[2] * ba[2];
    double wp[3], dp[3];
    for (int k = 0; k < 3; ++k) { wp[k] = w[k] - wb / bb * ba[k]; dp[k] = d[k] - db / bb * ba[k]; }
    double A = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
    double c0 = -INFINITY, c1 = INFINITY;
    if (A > 0) {
        double tc = -(wp[0] * dp[0] + wp[1] * dp[1] + wp[2] * dp[2]) / A;
        double h2 = 0;
        for (int k = 0; k < 3; ++k) { double q = wp[k] + tc * dp[k]; h2 += q * q; }
        if (h2 > r * r) return 0;
        double s = sqrt((r * r - h2) / A);
        c0 = tc - s; c1 = tc + s;
    } else if (wp[0] * wp[0] + wp[1] * wp[1] + wp[2] * wp[2] > r * r) {
        return 0;
    }
    if (db == 0) {
        if (wb < 0 || wb > bb) return 0;
    } else {
        double ta = -wb / db, tb = (bb - wb) / db;
        double sa = ta < tb ? ta : tb, sb = ta < tb ? tb : ta;
        if (sa > c0) c0 = sa;
        if (sb < c1) c1 = sb;
        if (c0 > c1) return 0;
    }
    *t0 = c0; *t1 = c1;
    return 1;
}

/* Ray against capsule (a, b, r) = cylinder between the end planes U two
 * spheres; the capsule is convex so its interval is the hull of the parts. */
static int ray_capsule64(const double o[3], const double d[3], const double *v, double *t0,
                         double *t1) {
    double lo = INFINITY, hi = -INFINITY, s0, s1;
    double a[3] = {v[0], v[1], v[2]}, b[3] = {v[3], v[4], v[5]}, r = v[6];
    if (ray_sphere64(o, d, a, r, &s0, &s1)) { lo = fmin(lo, s0); hi = fmax(hi, s1); }
    if (ray_sphere64(o, d, b, r, &s0, &s1)) { lo = fmin(lo, s0); hi = fmax(hi, s1); }
    if (ray_cylinder64(o, d, v, &s0, &s1)) { lo = fmin(lo, s0); hi = fmax(hi, s1); }
    if (lo > hi) return 0;
    *t0 = lo; *t1 = hi;
    return 1;
}

/* Ray against the sphere-triangle (points within r of the triangle a, b, c;
 * v = a, b, c at [0:9], r at [9]): it is convex, the union of the prism
 * {|n.(x - a)| <= r, x on the inner side of the three edge planes} and the
 * three edge capsules, so its interval is the hull of the parts'. */
static int ray_stri64(const double o[3], const double d[3], const double *v, double *t0, double *t1) {
    const double *P[3] = {v, v + 3, v + 6};
    double r = v[9];
    double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
    double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
    double N[3];
    cross3(e1, e2, N);
    double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    for (int k = 0; k < 3; ++k) N[k] /= nn;
    double lo = INFINITY, hi = -INFINITY;
    /* prism */
    double a_lo = -INFINITY, a_hi = INFINITY;
    int ok = 1;
    double so = (o[0] - P[0][0]) * N[0] + (o[1] - P[0][1]) * N[1] + (o[2] - P[0][2]) * N[2];
    double sd = d[0] * N[0] + d[1] * N[1] + d[2] * N[2];
    if (sd == 0) { if (fabs(so) > r) ok = 0; }
    else {
        double ta = (-r - so) / sd, tb = (r - so) / sd;
        a_lo = ta < tb ? ta : tb; a_hi = ta < tb ? tb : ta;
    }
    for (int i = 0; i < 3 && ok; ++i) {
        const double *s = P[i], *t = P[(i + 1) % 3];
        double ed[3] = {t[0] - s[0], t[1] - s[1], t[2] - s[2]}, m[3];
        cross3(ed, N, m);   /* outward in-plane normal of edge s -> t */
        double g = (o[0] - s[0]) * m[0] + (o[1] - s[1]) * m[1] + (o[2] - s[2]) * m[2];
        double gd = d[0] * m[0] + d[1] * m[1] + d[2] * m[2];
        if (gd == 0) { if (g > 0) ok = 0; }
        else if (gd > 0) { double tl = -g / gd; if (tl < a_hi) a_hi = tl; }
        else { double tl = -g / gd; if (tl > a_lo) a_lo = tl; }
    }
    if (ok && a_lo <= a_hi) { lo = a_lo; hi = a_hi; }
    /* edges */
    for (int i = 0; i < 3; ++i) {
        double cap[7], s0, s1;
        for (int k = 0; k < 3; ++k) { cap[k] = P[i][k]; cap[3 + k] = P[(i + 1) % 3][k]; }
        cap[6] = r;
        if (ray_capsule64(o, d, cap, &s0, &s1)) { lo = fmin(lo, s0); hi = fmax(hi, s1); }
    }
    if (lo > hi) return 0;
    *t0 = lo; *t1 = hi;
    return 1;
}

static int ray_voi64(int kind, const double *v, const double o[3], const double d[3],
                     double *t0, double *t1) {
    switch (kind) {
    case K_RTRI: return ray_stri64(o, d, v, t0, t1);
    case K_QUADRIC: return ray_obox64(o, d, v, t0, t1);
    case K_SPHERE: { double c[3] = {v[0], v[1], v[2]}; return ray_sphere64(o, d, c, v[3], t0, t1); }
    case K_RBOX: return ray_obox64(o, d, v, t0, t1);
    case K_CAPSULE: case K_SCONE: return ray_capsule64(o, d, v, t0, t1);
    case K_TORUS: return ray_cylinder64(o, d, v, t0, t1);
    case K_ELLIPSOID: return ray_obox64(o, d, v, t0, t1);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Ray / volume-of-interest intervals, FP32 in the documented fixed order.   */
/* Every line below is one IEEE single operation (compiled without FMA       */
/* contraction); the VOI radius / extents carry the absolute pad `pad`.      */

static int ray_sphere32(const float o[3], const float d[3], const float c[3], float r,
                        float *t0, float *t1) {
    float wx = c[0] - o[0], wy = c[1] - o[1], wz = c[2] - o[2];
    float dd = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    float wd = (wx * d[0] + wy * d[1]) + wz * d[2];
    float tc = wd / dd;
    float qx = wx - tc * d[0], qy = wy - tc * d[1], qz = wz - tc * d[2];
    float h2 = (qx * qx + qy * qy) + qz * qz;
    float r2 = r * r;
    if (h2 > r2) return 0;
    float s = sqrtf((r2 - h2) / dd);
    *t0 = tc - s; *t1 = tc + s;
    return 1;
}

static int ray_obox32(const float o[3], const float d[3], const float *q, const float e[3],
                      float *t0, float *t1) {
    float lo = -INFINITY, hi = INFINITY;
    float wx = o[0] - q[0], wy = o[1] - q[1], wz = o[2] - q[2];
    for (int i = 0; i < 3; ++i) {
        const float *m = q + 3 + 3 * i;
        float lo_i = (m[0] * wx + m[1] * wy) + m[2] * wz;
        float ld_i = (m[0] * d[0] + m[1] * d[1]) + m[2] * d[2];
        if (ld_i == 0.0f) {
            if (lo_i < -e[i] || lo_i > e[i]) return 0;
            continue;
        }
        float ta = (-e[i] - lo_i) / ld_i, tb = (e[i] - lo_i) / ld_i;
        float a = ta < tb ? ta : tb, b = ta < tb ? tb : ta;
        if (a > lo) lo = a;
        if (b < hi) hi = b;
    }
    if (lo > hi) return 0;
    *t0 = lo; *t1 = hi;
    return 1;
}

/* The cylinder part of the capsule test (radius r around [a, b], capped by
 * the end planes), also the torus's volume of interest. */
static int ray_cylinder32(const float o[3], const float d[3], const float *a, const float *b, float r,
                          float *t0, float *t1) {
    float bx = b[0] - a[0], by = b[1] - a[1], bz = b[2] - a[2];
    float wx = o[0] - a[0], wy = o[1] - a[1], wz = o[2] - a[2];
    float bb = (bx * bx + by * by) + bz * bz;
    if (!(bb > 0.0f)) return 0;
    float wb = (wx * bx + wy * by) + wz * bz;
    float db = (d[0] * bx + d[1] * by) + d[2] * bz;
    float fw = wb / bb, fd = db / bb;
    float px = wx - fw * bx, py = wy - fw * by, pz = wz - fw * bz;
    float ux = d[0] - fd * bx, uy = d[1] - fd * by, uz = d[2] - fd * bz;
    float A = (ux * ux + uy * uy) + uz * uz;
    float r2 = r * r;
    float c0 = -INFINITY, c1 = INFINITY;
    if (A > 0.0f) {
        float pu = (px * ux + py * uy) + pz * uz;
        float tc = -(pu / A);
        float hx = px + tc * ux, hy = py + tc * uy, hz = pz + tc * uz;
        float h2 = (hx * hx + hy * hy) + hz * hz;
        if (h2 > r2) return 0;
        float sq = sqrtf((r2 - h2) / A);
        c0 = tc - sq; c1 = tc + sq;
    } else {
        float p2 = (px * px + py * py) + pz * pz;
        if (p2 > r2) return 0;
    }
    if (db == 0.0f) {
        if (wb < 0.0f || wb > bb) return 0;
    } else {
        float ta = -(wb / db), tb = (bb - wb) / db;
        float sa = ta < tb ? ta : tb, sb = ta < tb ? tb : ta;
        if (sa > c0) c0 = sa;
        if (sb < c1) c1 = sb;
        if (c0 > c1) return 0;
    }
    *t0 = c0; *t1 = c1;
    return 1;
}

static int ray_capsule32(const float o[3], const float d[3], const float *q, float r,
                         float *t0, float *t1) {
    float lo = INFINITY, hi = -INFINITY, s0, s1;
    const float *a = q, *b = q + 3;
    if (ray_sphere32(o, d, a, r, &s0, &s1)) { if (s0 < lo) lo = s0; if (s1 > hi) hi = s1; }
    if (ray_sphere32(o, d, b, r, &s0, &s1)) { if (s0 < lo) lo = s0; if (s1 > hi) hi = s1; }
    if (ray_cylinder32(o, d, a, b, r, &s0, &s1)) { if (s0 < lo) lo = s0; if (s1 > hi) hi = s1; }
    if (lo > hi) return 0;
    *t0 = lo; *t1 = hi;
    return 1;
}

/* Sphere-triangle in FP32 (the same operations as the GPU culling kernel):
 * the prism over the triangle, then the three edge capsules; the interval is
 * the hull of the parts' (the volume is convex).  a, b, c: vertices as the
 * kernel reconstructs them from the record words; n, m[0..2]: unit normal
 * and in-plane edge normals of edges a-b, b-c, c-a; r: the radius. */
static int ray_stri32(const float o[3], const float d[3], const float a[3], const float b[3], const float c[3],
                      const float n[3], const float m[3][3], float r, float *t0, float *t1) {
    float lo = INFINITY, hi = -INFINITY, s0, s1;
    float oa[3] = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
    float ob[3] = {o[0] - b[0], o[1] - b[1], o[2] - b[2]};
    float oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
    float so = (n[0] * oa[0] + n[1] * oa[1]) + n[2] * oa[2];
    float g[3];
    g[0] = (m[0][0] * oa[0] + m[0][1] * oa[1]) + m[0][2] * oa[2];
    g[1] = (m[1][0] * ob[0] + m[1][1] * ob[1]) + m[1][2] * ob[2];
    g[2] = (m[2][0] * oc[0] + m[2][1] * oc[1]) + m[2][2] * oc[2];
    float a_lo = -INFINITY, a_hi = INFINITY;
    int ok = 1;
    float sd = (n[0] * d[0] + n[1] * d[1]) + n[2] * d[2];
    if (sd == 0.0f) {
        if (so < -r || so > r) ok = 0;
    } else {
        float ta = (-r - so) / sd, tb = (r - so) / sd;
        a_lo = ta < tb ? ta : tb;
        a_hi = ta < tb ? tb : ta;
    }
    for (int i = 0; i < 3; ++i) {
        float gd = (m[i][0] * d[0] + m[i][1] * d[1]) + m[i][2] * d[2];
        if (gd == 0.0f) {
            if (g[i] > 0.0f) ok = 0;
        } else {
            float tl = (-g[i]) / gd;
            if (gd > 0.0f) { if (tl < a_hi) a_hi = tl; }
            else { if (tl > a_lo) a_lo = tl; }
        }
    }
    if (ok && a_lo <= a_hi) { lo = a_lo; hi = a_hi; }
    const float *P[3] = {a, b, c};
    for (int i = 0; i < 3; ++i) {
        float cap[6];
        for (int k = 0; k < 3; ++k) { cap[k] = P[i][k]; cap[3 + k] = P[(i + 1) % 3][k]; }
        if (ray_capsule32(o, d, cap, r, &s0, &s1)) { if (s0 < lo) lo = s0; if (s1 > hi) hi = s1; }
    }
    if (lo > hi) return 0;
    *t0 = lo; *t1 = hi;
    return 1;
}

/* Record words of a rounded triangle as the library's host preparation
 * derives them in FP64 and rounds once to FP32 (edges e0 = b - a,
 * e2 = a - c, unit normal n = e0 x (c - a) / |.|, edge normals m_i = e_i x n),
 * and the vertices b = a + e0, c = a - e2 that the culling kernel rebuilds
 * from them in FP32. */
static void tri_words32(const float *q, float a[3], float b[3], float c[3], float n[3], float m[3][3]) {
    double e[3][3];
    for (int k = 0; k < 3; ++k) {
        e[0][k] = (double)q[3 + k] - q[k];
        e[1][k] = (double)q[6 + k] - q[3 + k];
        e[2][k] = (double)q[k] - q[6 + k];
    }
    double ca[3] = {-e[2][0], -e[2][1], -e[2][2]};
    double cr[3] = {e[0][1] * ca[2] - e[0][2] * ca[1], e[0][2] * ca[0] - e[0][0] * ca[2],
                    e[0][0] * ca[1] - e[0][1] * ca[0]};
    double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    double nd[3];
    for (int k = 0; k < 3; ++k) nd[k] = len > 0.0 ? cr[k] / len : 0.0;
    for (int i = 0; i < 3; ++i) {
        m[i][0] = (float)(e[i][1] * nd[2] - e[i][2] * nd[1]);
        m[i][1] = (float)(e[i][2] * nd[0] - e[i][0] * nd[2]);
        m[i][2] = (float)(e[i][0] * nd[1] - e[i][1] * nd[0]);
    }
    for (int k = 0; k < 3; ++k) {
        n[k] = (float)nd[k];
        a[k] = q[k];
        b[k] = a[k] + (float)e[0][k];
        c[k] = a[k] - (float)e[2][k];
    }
}

/* Rotation rows of a bounded quadric as the library's host preparation
 * derives them (M = R^T of the normalised quaternion, FP64, rounded once);
 * out: centre at [0:3], M at [3:12] (the oriented-box record layout). */
static void quadric_box32(const float *q, float *box) {
    double w = q[3], x = q[4], y = q[5], z = q[6];
    double nq = sqrt(w * w + x * x + y * y + z * z);
    if (nq > 0.0) { w /= nq; x /= nq; y /= nq; z /= nq; }
    double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)},
                      {2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)},
                      {2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)}};
    for (int k = 0; k < 3; ++k) box[k] = q[k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) box[3 + 3 * i + j] = (float)R[j][i];
}

/* Record words that the library's host preparation derives in FP64 and
 * rounds once to FP32 (the unit axis of a torus). */
static void unit3_f32(const float *a, float u[3]) {
    double n = sqrt((double)a[0] * a[0] + (double)a[1] * a[1] + (double)a[2] * a[2]);
    for (int k = 0; k < 3; ++k) u[k] = (float)(a[k] / n);
}

/* ------------------------------------------------------------------------ */
/* Brute-force per-tile culling (Sec. 6.2): for every tile and primitive,
 * test every pixel-centre ray of the tile against the primitive's volume of
 * interest; entry = min over hitting rays of the (front-clipped) entry depth,
 * exit = max of the exit depth; a primitive is listed iff at least one ray
 * hits.  Lists are sorted by (entry depth, post-order address).
 *
 * mode 0: FP64 exact geometry, no pad.  mode 1: FP32 fixed-order arithmetic
 * with the VOI extents enlarged by `pad` (the GPU's documented formulas).
 * Only the tiles in `tiles[0..ntiles)` are computed.  Output: counts[ntiles];
 * entries (z_in, z_out, addr) written at tile-major slots of capacity `cap`
 * per tile.  Returns 0, or -1 if a tile exceeds `cap`. */
typedef struct { double zi, zo; int32_t a; float zi32, zo32; } Entry;

static int entry_cmp(const void *x, const void *y) {
    const Entry *a = (const Entry *)x, *b = (const Entry *)y;
    if (a->zi < b->zi) return -1;
    if (a->zi > b->zi) return 1;
    return (a->a > b->a) - (a->a < b->a);
}

int or_cull(int n, int root, const int32_t *kind, const int32_t *left, const int32_t *right,
            const float *params, const float *cam, int tile, int mode, float pad, int ntiles,
            const int32_t *tiles, int cap, int32_t *counts, double *z_in, double *z_out,
            int32_t *addr) {
    Tree t;
    tree_init(&t, n, root, kind, left, right, params);
    Cam c;
    cam_init(&c, cam);
    int counter = 0;
    int *po = (int *)malloc(sizeof(int) * (size_t)n);
    double *roi = (double *)malloc(sizeof(double) * (size_t)n);
    postorder_rec(&t, root, &counter, po);
    roi_rec(&t, root, 0.0, roi);
    int tiles_x = (c.W + tile - 1) / tile;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int ti = 0; ti < ntiles; ++ti) {
        int tx = tiles[ti] % tiles_x, ty = tiles[ti] / tiles_x;
        Entry *buf = (Entry *)malloc(sizeof(Entry) * (size_t)(n > 0 ? n : 1));
        int cnt = 0;
        for (int i = 0; i < n; ++i) {
            int k = kind[i];
            if (!is_prim(k)) continue;
            const float *q = params + (size_t)i * NREC;
            double v64[NREC];
            voi_rec(k, q, roi[i], v64);
            /* FP32 VOI: extents ((size + d) + pad) in single precision. */
            float dp = (float)roi[i];
            float rr32 = 0, e32[3] = {0, 0, 0}, ca32[3] = {0, 0, 0}, cb32[3] = {0, 0, 0};
            float ta32[3], tb32[3], tc32[3], tn32[3], tm32[3][3], qbox32[12];
            if (k == K_SPHERE) rr32 = (q[3] + dp) + pad;
            else if (k == K_RTRI) {
                tri_words32(q, ta32, tb32, tc32, tn32, tm32);
                rr32 = (q[9] + dp) + pad;
            } else if (k == K_QUADRIC) {
                quadric_box32(q, qbox32);
                for (int a = 0; a < 3; ++a) e32[a] = (q[7 + a] + dp) + pad;
            }
            else if (k == K_CAPSULE) rr32 = (q[6] + dp) + pad;
            else if (k == K_SCONE) rr32 = ((q[6] > q[7] ? q[6] : q[7]) + dp) + pad;
            else if (k == K_TORUS) {
                /* cylinder: radius ((R + r) + d) + pad, half-height (r + d) + pad */
                float ax[3];
                unit3_f32(q + 3, ax);
                rr32 = ((q[6] + q[7]) + dp) + pad;
                float hh = (q[7] + dp) + pad;
                for (int a = 0; a < 3; ++a) { ca32[a] = q[a] - hh * ax[a]; cb32[a] = q[a] + hh * ax[a]; }
            } else if (k == K_ELLIPSOID) {
                float rmin = q[12];
                if (q[13] < rmin) rmin = q[13];
                if (q[14] < rmin) rmin = q[14];
                float grow = 1.0f + dp / rmin;
                for (int a = 0; a < 3; ++a) e32[a] = q[12 + a] * grow + pad;
            } else for (int a = 0; a < 3; ++a) e32[a] = ((q[12 + a] + q[15]) + dp) + pad;
            int hit = 0;
            double zi = INFINITY, zo = -INFINITY;
            float zi32 = INFINITY, zo32 = -INFINITY;
            for (int py = ty * tile; py < (ty + 1) * tile && py < c.H; ++py) {
                for (int px = tx * tile; px < (tx + 1) * tile && px < c.W; ++px) {
                    if (mode == 0) {
                        double d[3], t0, t1;
                        cam_ray64(&c, px, py, d);
                        if (!ray_voi64(k, v64, c.o, d, &t0, &t1)) continue;
                        if (t0 < 0) t0 = 0;
                        if (t1 < t0) continue;
                        hit = 1;
                        if (t0 < zi) zi = t0;
                        if (t1 > zo) zo = t1;
                    } else {
                        float d[3], t0, t1;
                        int h;
                        cam_ray32(&c, px, py, d);
                        if (k == K_SPHERE) h = ray_sphere32(c.of, d, q, rr32, &t0, &t1);
                        else if (k == K_RBOX || k == K_ELLIPSOID) h = ray_obox32(c.of, d, q, e32, &t0, &t1);
                        else if (k == K_QUADRIC) h = ray_obox32(c.of, d, qbox32, e32, &t0, &t1);
                        else if (k == K_RTRI)
                            h = ray_stri32(c.of, d, ta32, tb32, tc32, tn32, tm32, rr32, &t0, &t1);
                        else if (k == K_TORUS) h = ray_cylinder32(c.of, d, ca32, cb32, rr32, &t0, &t1);
                        else h = ray_capsule32(c.of, d, q, rr32, &t0, &t1);
                        if (!h) continue;
                        t0 = t0 > 0.0f ? t0 : 0.0f;
                        if (!(t1 >= t0)) continue;
                        hit = 1;
                        if (t0 < zi32) zi32 = t0;
                        if (t1 > zo32) zo32 = t1;
                    }
                }
            }
            if (!hit) continue;
            Entry e;
            e.a = po[i];
            if (mode == 0) { e.zi = zi; e.zo = zo; }
            else { e.zi = zi32; e.zo = zo32; }
            buf[cnt++] = e;
        }
        qsort(buf, (size_t)cnt, sizeof(Entry), entry_cmp);
        counts[ti] = cnt;
        if (cnt > cap) {
#pragma omp atomic write
            err = -1;
        } else {
            for (int j = 0; j < cnt; ++j) {
                size_t s = (size_t)ti * cap + j;
                z_in[s] = buf[j].zi; z_out[s] = buf[j].zo; addr[s] = buf[j].a;
            }
        }
        free(buf);
    }
    free(po); free(roi);
    tree_free(&t);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Naive sphere tracing of the dense field (Sec. 2.2 "Ray processing          */
/* routines", Sec. 10 "Ray processing": step f / L with L = 1.45).           */

static double field_at(const Tree *t, const double o[3], const double d[3], double z) {
    double p[3] = {o[0] + z * d[0], o[1] + z * d[1], o[2] + z * d[2]};
    return field_rec(t, t->root, p, NULL);
}

static void grad_at(const Tree *t, const double p[3], double h, double g[3]) {
    for (int k = 0; k < 3; ++k) {
        double a[3] = {p[0], p[1], p[2]}, b[3] = {p[0], p[1], p[2]};
        a[k] += h; b[k] -= h;
        g[k] = (field_rec(t, t->root, a, NULL) - field_rec(t, t->root, b, NULL)) / (2 * h);
    }
}

/* Depth, normal and residual of one traced ray.  A hit at z is refined by
 * up to `newton` Newton steps along the ray (step clamped to +-newton_clamp in
 * distance); depth = z |d| (Euclidean distance to the eye); the normal is the
 * normalised central-difference gradient (h = 1e-6); resid is the field value
 * at the refined point.  A miss gets depth = resid = +inf and a zero normal. */
static void finish_ray(const Tree *t, const Cam *c, const double d[3], double dn, double z, int hit,
                       int newton, double newton_clamp, double *depth, double *normal, double *resid) {
    if (!hit) {
        *depth = INFINITY;
        *resid = INFINITY;
        for (int k = 0; k < 3; ++k) normal[k] = 0.0;
        return;
    }
    for (int it = 0; it < newton; ++it) {
        double p[3] = {c->o[0] + z * d[0], c->o[1] + z * d[1], c->o[2] + z * d[2]}, g[3];
        double fz = field_rec(t, t->root, p, NULL);
        grad_at(t, p, 1e-6, g);
        double gd = g[0] * d[0] + g[1] * d[1] + g[2] * d[2];
        if (gd == 0.0) break;
        double dz = -fz / gd;
        double lim = newton_clamp / dn;
        if (dz > lim) dz = lim;
        if (dz < -lim) dz = -lim;
        z += dz;
    }
    double p[3] = {c->o[0] + z * d[0], c->o[1] + z * d[1], c->o[2] + z * d[2]}, g[3];
    grad_at(t, p, 1e-6, g);
    double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    *resid = field_rec(t, t->root, p, NULL);
    *depth = z * dn;
    for (int k = 0; k < 3; ++k) normal[k] = gn > 0 ? g[k] / gn : 0.0;
}

/* Rays start at planar depth Z_NEAR (the near plane).  A ray whose first
 * sample there is inside the solid (f < -eps: the eye is inside the shape) is
 * a hit clipped at the near plane, with no refinement. */
#define Z_NEAR 0.01

/* Per pixel (i, j):  z starts at z_near and advances by f / (L |d|) until
 * f <= eps (hit), z > z_far (miss: exit of the bounding sphere of the
 * primitives' bounds) or max_steps.  A hit is refined by up to `newton`
 * Newton steps along the ray (step clamped to +-newton_clamp in distance),
 * then depth = z |d| (Euclidean distance to the eye) and the normal is the
 * normalised central-difference gradient (h = 1e-6).  min_f receives the
 * smallest field value met along the ray and resid the field value at the
 * refined hit (both for the silhouette-band test: a hit whose refined point
 * is not a root is a near miss, the ray grazes within eps of the surface).
 * flags: bit0 hit, bit1 step cap reached. */
void or_trace(int n, int root, const int32_t *kind, const int32_t *left, const int32_t *right,
              const float *params, const float *cam, double eps, double lipschitz,
              int max_steps, int newton, double newton_clamp, int npx, const int32_t *pi,
              const int32_t *pj, double *depth, double *normal, int32_t *steps,
              uint8_t *flags, double *min_f, double *resid) {
    Tree t;
    tree_init(&t, n, root, kind, left, right, params);
    Cam c;
    cam_init(&c, cam);
    double lo[3], hi[3];
    double diag = or_scene_bounds(n, kind, params, lo, hi);
    double bc[3] = {0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2])};
    double br = 0.5 * diag;
#pragma omp parallel for schedule(dynamic, 16)
    for (int px = 0; px < npx; ++px) {
        double d[3];
        cam_ray64(&c, pi[px], pj[px], d);
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double t0, t1, mf = INFINITY;
        int st = 0;
        uint8_t fl = 0;
        double z = Z_NEAR, f = INFINITY;
        int clip = 0;
        if (ray_sphere64(c.o, d, bc, br, &t0, &t1) && t1 > z) {
            if (t0 > z) z = t0;
            double zfar = t1;
            for (;;) {
                f = field_at(&t, c.o, d, z);
                if (f < mf) mf = f;
                if (f <= eps) { fl |= 1; clip = st == 0 && z == Z_NEAR && f < -eps; break; }
                if (st >= max_steps) { fl |= 2; break; }
                ++st;
                z += f / (lipschitz * dn);
                if (z > zfar) break;
            }
        }
        finish_ray(&t, &c, d, dn, z, fl & 1, clip ? 0 : newton, newton_clamp, depth + px,
                   normal + 3 * (size_t)px, resid + px);
        steps[px] = st;
        flags[px] = fl;
        min_f[px] = mf;
    }
    tree_free(&t);
}

/* The ray processing stated in Sec. 10 ("Ray processing"), over the dense
 * field: over-relaxed sphere tracing with factor omega, where a step whose
 * end sphere does not overlap the sphere it started from is undone; the end
 * sphere is kept and over-relaxation stays off until plain steps reach it,
 * whereupon the ray jumps across it (the sphere is free of surface).  No
 * step cap; instead every step is at least min_step long (distance units),
 * and a hit is the first sample with f <= 0 (iso-crossing detection), then
 * refined and shaded as in or_trace (a first sample inside the solid at the
 * near plane with f < -eps is a clipped hit there, as in or_trace).
 * Readings where Sec. 10 is silent: a plain or minimum-length step is never
 * undone (only relaxed steps are tested); an undone step whose end point lies
 * inside the solid (f <= 0) stores no sphere to jump across (a crossing lies
 * before it, which plain steps will bracket).  max_steps only guards against
 * a broken field (flag bit1); steps counts field evaluations. */
void or_trace_relaxed(int n, int root, const int32_t *kind, const int32_t *left, const int32_t *right,
                      const float *params, const float *cam, double eps, double lipschitz, double omega,
                      double min_step, int max_steps, int newton, double newton_clamp, int npx,
                      const int32_t *pi, const int32_t *pj, double *depth, double *normal,
                      int32_t *steps, uint8_t *flags, double *min_f, double *resid) {
    Tree t;
    tree_init(&t, n, root, kind, left, right, params);
    Cam c;
    cam_init(&c, cam);
    double lo[3], hi[3];
    double diag = or_scene_bounds(n, kind, params, lo, hi);
    double bc[3] = {0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2])};
    double br = 0.5 * diag;
#pragma omp parallel for schedule(dynamic, 16)
    for (int px = 0; px < npx; ++px) {
        double d[3];
        cam_ray64(&c, pi[px], pj[px], d);
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double h = min_step / dn;            /* shortest step in ray parameter */
        double t0, t1, mf = INFINITY;
        int st = 0;
        uint8_t fl = 0;
        int clip = 0;
        double z = Z_NEAR;
        if (ray_sphere64(c.o, d, bc, br, &t0, &t1) && t1 > z) {
            if (t0 > z) z = t0;
            double zfar = t1;
            double rp = 0.0;                 /* surface-free radius at the previous sample */
            double dzp = 0.0;                /* last relaxed step (0: none to verify) */
            double zf = z;                   /* where the plain step from the previous sample lands */
            double zs = 0.0, rs = -1.0;      /* stored sphere (rs < 0: none) */
            int relax = 1;
            for (;;) {
                if (st >= max_steps) { fl |= 2; break; }
                double f = field_at(&t, c.o, d, z);
                ++st;
                if (f < mf) mf = f;
                double r = fabs(f) / (lipschitz * dn);
                if (dzp > 0.0 && r + rp < dzp) {
                    /* undo the relaxed step */
                    if (f > 0.0) { zs = z; rs = r; } else { zs = INFINITY; rs = 0.0; }
                    relax = 0;
                    z = zf;
                    dzp = 0.0;
                    if (rs >= 0.0 && z >= zs - rs) { z = zs + rs; rs = -1.0; relax = 1; }
                    if (z > zfar) break;
                    continue;
                }
                if (f <= 0.0) { fl |= 1; clip = st == 1 && z == Z_NEAR && f < -eps; break; }
                double om = relax ? omega : 1.0;
                double dz = om * r;
                if (dz <= h) { dz = h; om = 1.0; }
                zf = z + (r > h ? r : h);
                rp = r;
                dzp = om > 1.0 ? dz : 0.0;
                z += dz;
                if (!relax && rs >= 0.0 && z >= zs - rs) {
                    if (z < zs + rs) z = zs + rs;
                    rs = -1.0;
                    relax = 1;
                    dzp = 0.0;
                }
                if (z > zfar) break;
            }
        }
        finish_ray(&t, &c, d, dn, z, fl & 1, clip ? 0 : newton, newton_clamp, depth + px,
                   normal + 3 * (size_t)px, resid + px);
        steps[px] = st;
        flags[px] = fl;
        min_f[px] = mf;
    }
    tree_free(&t);
}

/* Fine FP64 ray marching (step `h` in t) from z_near to z_stop, reporting the
 * first sign change of f (or the first f <= 0); used to check that no surface
 * lies before a reported first hit.  Returns the first crossing depth in t,
 * or +inf when none. */
void or_march(int n, int root, const int32_t *kind, const int32_t *left, const int32_t *right,
              const float *params, const float *cam, double h, int npx, const int32_t *pi,
              const int32_t *pj, const double *z_stop, double *z_first) {
    Tree t;
    tree_init(&t, n, root, kind, left, right, params);
    Cam c;
    cam_init(&c, cam);
#pragma omp parallel for schedule(dynamic, 1)
    for (int px = 0; px < npx; ++px) {
        double d[3];
        cam_ray64(&c, pi[px], pj[px], d);
        double z = 0.01, res = INFINITY;
        while (z <= z_stop[px]) {
            if (field_at(&t, c.o, d, z) <= 0.0) { res = z; break; }
            z += h;
        }
        z_first[px] = res;
    }
    tree_free(&t);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
