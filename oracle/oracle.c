/*
 * oracle.c -- plain, slow, FP64 CPU reference of the parallel direct cut.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker the CUDA
 * library is compared against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it; the library never does, and the two
 * share no source, header, table or helper.
 *
 * What it computes (one element E of the background grid, one closed cut
 * surface S), following Sec. "Parallel Direct Cut Algorithm" of the paper:
 *
 *   1. Linearised geometry (Sec. 4.2 and Fig. quadsplit): each of the 6 faces
 *      of an order-p hex is a (p+1)^2 node grid, split into p^2 linear quads and
 *      each quad into 2 triangles (12 p^2 triangles per element); each order-q
 *      cut face likewise gives 2 q^2 triangles.
 *   2. d(E) = min over element-boundary triangles Te and surface triangles Ts
 *      of the Euclidean distance between the closed triangles (the quantity the
 *      modified Moller triangle-triangle test of Sec. 4.2 returns).
 *   3. FRINGE ("intersecting", Sec. 4.2 first paragraph) iff d(E) <= tol
 *      (tol = 1e-7, Alg. cp1 / cp2).
 *   4. Otherwise E lies wholly on one side of S: HOLE iff corner node 0 of E is
 *      inside S, decided by the generalised winding number (sum of oriented
 *      solid angles, Van Oosterom & Strackee 1983), else FIELD.
 *   5. dist = +d (FIELD), -d (HOLE), d (FRINGE).
 *
 * It also evaluates the paper's own side rule (Sec. 4.1/4.2: dot product of
 * the minimal vector with the outward normal; equidistant faces: average the
 * normals when the dots disagree in sign, otherwise keep the largest |dot|) on
 * the tie set, so the tests can count elements where the two rules disagree.
 *
 * Two search modes give the same d(E):
 *   brute  -- every face of S is tested against every element;
 *   pruned -- faces are visited in increasing axis-aligned box distance
 *             (Alg. bboxdix) and the search stops once that lower bound exceeds
 *             the best distance found (branch and bound; nothing is truncated).
 *
 * Compile with -ffp-contract=off so a*b+c is never fused: the pose transform
 * below must round exactly like the element-wise form it is written in.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_HOLE 0
#define ORC_FIELD 1
#define ORC_FRINGE (-1)

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
typedef struct { double x, y, z; } vec;

static vec mk(const double *p) { vec r = {p[0], p[1], p[2]}; return r; }
static vec vsub(vec a, vec b) { vec r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static vec vadd(vec a, vec b) { vec r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static vec vscale(vec a, double s) { vec r = {a.x * s, a.y * s, a.z * s}; return r; }
static double vdot(vec a, vec b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec vcross(vec a, vec b) {
    vec r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
    return r;
}
static double vnorm(vec a) { return sqrt(vdot(a, a)); }
static void store(double *out, vec a) { if (out) { out[0] = a.x; out[1] = a.y; out[2] = a.z; } }

/* signed volume (times 6) of tetrahedron (a, b, c, d) */
static double orient(vec a, vec b, vec c, vec d) {
    return vdot(vcross(vsub(b, a), vsub(c, a)), vsub(d, a));
}

/* ------------------------------------------------------------------------ */
/* distance primitives (closed forms, textbook geometry)                     */
/* ------------------------------------------------------------------------ */

/* closest point of segment [a,b] to p */
static double pt_seg(vec p, vec a, vec b, vec *cl) {
    vec ab = vsub(b, a);
    double L2 = vdot(ab, ab);
    double t = 0.0;
    if (L2 > 0.0) {
        t = vdot(vsub(p, a), ab) / L2;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    vec c = vadd(a, vscale(ab, t));
    if (cl) *cl = c;
    return vnorm(vsub(p, c));
}

/* closest point of triangle (a,b,c) to p: the orthogonal projection when it
 * falls inside the triangle, otherwise the nearest point of the three edges */
static double pt_tri(vec p, vec a, vec b, vec c, vec *cl) {
    vec n = vcross(vsub(b, a), vsub(c, a));
    double n2 = vdot(n, n);
    if (n2 > 0.0) {
        vec pp = vsub(p, vscale(n, vdot(n, vsub(p, a)) / n2));
        double s0 = vdot(n, vcross(vsub(b, a), vsub(pp, a)));
        double s1 = vdot(n, vcross(vsub(c, b), vsub(pp, b)));
        double s2 = vdot(n, vcross(vsub(a, c), vsub(pp, c)));
        if (s0 >= 0.0 && s1 >= 0.0 && s2 >= 0.0) {
            if (cl) *cl = pp;
            return vnorm(vsub(p, pp));
        }
    }
    vec c0, c1, c2;
    double d0 = pt_seg(p, a, b, &c0);
    double d1 = pt_seg(p, b, c, &c1);
    double d2 = pt_seg(p, c, a, &c2);
    double d = d0; vec cc = c0;
    if (d1 < d) { d = d1; cc = c1; }
    if (d2 < d) { d = d2; cc = c2; }
    if (cl) *cl = cc;
    return d;
}

/* distance between segments [p0,p1] and [q0,q1]: the minimum of a convex
 * quadratic over the unit square is either at its interior stationary point
 * or on one of the square's four sides (four point-segment distances). */
static double seg_seg(vec p0, vec p1, vec q0, vec q1, vec *cp, vec *cq) {
    vec t1, t2;
    double best, d;
    vec bp, bq;
    best = pt_seg(p0, q0, q1, &t2); bp = p0; bq = t2;
    d = pt_seg(p1, q0, q1, &t2); if (d < best) { best = d; bp = p1; bq = t2; }
    d = pt_seg(q0, p0, p1, &t1); if (d < best) { best = d; bp = t1; bq = q0; }
    d = pt_seg(q1, p0, p1, &t1); if (d < best) { best = d; bp = t1; bq = q1; }
    vec d1 = vsub(p1, p0), d2 = vsub(q1, q0), r = vsub(p0, q0);
    double a = vdot(d1, d1), e = vdot(d2, d2), b = vdot(d1, d2);
    double c = vdot(d1, r), f = vdot(d2, r);
    double den = a * e - b * b;
    if (den > 0.0) {
        double s = (b * f - c * e) / den;
        double t = (a * f - b * c) / den;
        if (s > 0.0 && s < 1.0 && t > 0.0 && t < 1.0) {
            vec xp = vadd(p0, vscale(d1, s)), xq = vadd(q0, vscale(d2, t));
            d = vnorm(vsub(xp, xq));
            if (d < best) { best = d; bp = xp; bq = xq; }
        }
    }
    if (cp) *cp = bp;
    if (cq) *cq = bq;
    return best;
}

/* does segment [p,q] meet triangle (a,b,c)?  Signed-volume test: the segment
 * must reach both closed sides of the plane and the line pq must pass inside
 * the three edges.  The coplanar case is left to the distance features. */
static int seg_tri_hit(vec p, vec q, vec a, vec b, vec c, vec *x) {
    double o1 = orient(a, b, c, p), o2 = orient(a, b, c, q);
    if ((o1 > 0.0 && o2 > 0.0) || (o1 < 0.0 && o2 < 0.0)) return 0;
    if (o1 == 0.0 && o2 == 0.0) return 0;
    double s1 = orient(p, q, a, b), s2 = orient(p, q, b, c), s3 = orient(p, q, c, a);
    int pos = (s1 >= 0.0 && s2 >= 0.0 && s3 >= 0.0);
    int neg = (s1 <= 0.0 && s2 <= 0.0 && s3 <= 0.0);
    if (!(pos || neg)) return 0;
    if (x) *x = vadd(p, vscale(vsub(q, p), o1 / (o1 - o2)));
    return 1;
}

/* Distance between closed triangles A and B (9 doubles each).  Zero when an
 * edge of one meets the other; otherwise the minimum over the 6 vertex-triangle
 * and 9 edge-edge distances, which is where the closest pair of two disjoint
 * convex polygons lies.  cA, cB receive the closest points. */
double orc_tritri(const double *A, const double *B, double *cA, double *cB) {
    vec a[3] = {mk(A), mk(A + 3), mk(A + 6)};
    vec b[3] = {mk(B), mk(B + 3), mk(B + 6)};
    vec x;
    for (int i = 0; i < 3; ++i) {
        if (seg_tri_hit(a[i], a[(i + 1) % 3], b[0], b[1], b[2], &x)) { store(cA, x); store(cB, x); return 0.0; }
        if (seg_tri_hit(b[i], b[(i + 1) % 3], a[0], a[1], a[2], &x)) { store(cA, x); store(cB, x); return 0.0; }
    }
    double best = INFINITY, d;
    vec ba = a[0], bb = b[0], t1, t2;
    for (int i = 0; i < 3; ++i) {
        d = pt_tri(a[i], b[0], b[1], b[2], &t2);
        if (d < best) { best = d; ba = a[i]; bb = t2; }
        d = pt_tri(b[i], a[0], a[1], a[2], &t1);
        if (d < best) { best = d; ba = t1; bb = b[i]; }
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            d = seg_seg(a[i], a[(i + 1) % 3], b[j], b[(j + 1) % 3], &t1, &t2);
            if (d < best) { best = d; ba = t1; bb = t2; }
        }
    store(cA, ba);
    store(cB, bb);
    return best;
}

double orc_pt_tri(const double *P, const double *T, double *cl) {
    vec c;
    double d = pt_tri(mk(P), mk(T), mk(T + 3), mk(T + 6), &c);
    store(cl, c);
    return d;
}

double orc_seg_seg(const double *P0, const double *P1, const double *Q0, const double *Q1, double *cp, double *cq) {
    vec a, b;
    double d = seg_seg(mk(P0), mk(P1), mk(Q0), mk(Q1), &a, &b);
    store(cp, a);
    store(cq, b);
    return d;
}

/* ------------------------------------------------------------------------ */
/* linearisation (Sec. 4.2, Fig. quadsplit)                                  */
/* ------------------------------------------------------------------------ */
int orc_elem_ntri(int p) { return 12 * p * p; }
int orc_face_ntri(int q) { return 2 * q * q; }

static int node_index(int p, int i, int j, int k) { return i + (p + 1) * (j + (p + 1) * k); }

/* Element faces: 0 xi=-1, 1 xi=+1, 2 eta=-1, 3 eta=+1, 4 zeta=-1, 5 zeta=+1.
 * On each face the node grid (a,b) runs over the two free directions in
 * (xi,eta,zeta) order; quad (a,b) gives triangles (00,10,11) and (00,11,01).
 * Triangle t of face f is number f*2p^2 + 2*(b*p + a) + half. */
static int face_node(int p, int f, int a, int b) {
    int fix = (f & 1) ? p : 0;
    switch (f >> 1) {
    case 0: return node_index(p, fix, a, b);
    case 1: return node_index(p, a, fix, b);
    default: return node_index(p, a, b, fix);
    }
}

void orc_elem_tris(int p, const double *nodes, double *tris) {
    int t = 0;
    for (int f = 0; f < 6; ++f)
        for (int b = 0; b < p; ++b)
            for (int a = 0; a < p; ++a) {
                int n00 = face_node(p, f, a, b), n10 = face_node(p, f, a + 1, b);
                int n11 = face_node(p, f, a + 1, b + 1), n01 = face_node(p, f, a, b + 1);
                int tri[2][3] = {{n00, n10, n11}, {n00, n11, n01}};
                for (int h = 0; h < 2; ++h, ++t)
                    for (int v = 0; v < 3; ++v)
                        memcpy(tris + 9 * t + 3 * v, nodes + 3 * tri[h][v], 3 * sizeof(double));
            }
}

/* Cut face nodes (i,j) at i + (q+1) j; quad (a,b) -> (00,10,11), (00,11,01);
 * both keep the orientation d/dxi x d/deta of the face. */
void orc_face_tris(int q, const double *fnodes, double *tris) {
    int t = 0;
    for (int b = 0; b < q; ++b)
        for (int a = 0; a < q; ++a) {
            int n00 = a + (q + 1) * b, n10 = a + 1 + (q + 1) * b;
            int n11 = a + 1 + (q + 1) * (b + 1), n01 = a + (q + 1) * (b + 1);
            int tri[2][3] = {{n00, n10, n11}, {n00, n11, n01}};
            for (int h = 0; h < 2; ++h, ++t)
                for (int v = 0; v < 3; ++v)
                    memcpy(tris + 9 * t + 3 * v, fnodes + 3 * tri[h][v], 3 * sizeof(double));
        }
}

/* ------------------------------------------------------------------------ */
/* inside / outside                                                          */
/* ------------------------------------------------------------------------ */

/* Generalised winding number of a closed oriented triangle set about P:
 * (1/4pi) sum of signed solid angles, tan(Omega/2) = det[a b c] /
 * (|a||b||c| + (a.b)|c| + (a.c)|b| + (b.c)|a|) with a,b,c = vertices - P. */
double orc_winding(const double *P, int64_t ntri, const double *tris) {
    vec p = mk(P);
    double sum = 0.0;
    for (int64_t t = 0; t < ntri; ++t) {
        vec a = vsub(mk(tris + 9 * t), p), b = vsub(mk(tris + 9 * t + 3), p), c = vsub(mk(tris + 9 * t + 6), p);
        double la = vnorm(a), lb = vnorm(b), lc = vnorm(c);
        double det = vdot(a, vcross(b, c));
        double den = la * lb * lc + vdot(a, b) * lc + vdot(a, c) * lb + vdot(b, c) * la;
        sum += 2.0 * atan2(det, den);
    }
    return sum / (4.0 * M_PI);
}

/* Signed enclosed volume (divergence theorem); > 0 when the normals point out
 * of the enclosed region. */
double orc_signed_volume(int64_t ntri, const double *tris) {
    double v = 0.0;
    for (int64_t t = 0; t < ntri; ++t)
        v += vdot(mk(tris + 9 * t), vcross(mk(tris + 9 * t + 3), mk(tris + 9 * t + 6)));
    return v / 6.0;
}

/* x' = R x + t, rounded exactly as ((R0 x + R1 y) + R2 z) + t (no fusion). */
void orc_apply_pose(int64_t npts, const double *in, const double *pose, double *out) {
    for (int64_t i = 0; i < npts; ++i) {
        double x = in[3 * i], y = in[3 * i + 1], z = in[3 * i + 2];
        for (int a = 0; a < 3; ++a) {
            const double *R = pose + 4 * a;
            out[3 * i + a] = ((R[0] * x + R[1] * y) + R[2] * z) + R[3];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* the paper's side rule on the tie set                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double d;
    vec ce, cs;      /* closest points on the element and on the surface */
    int64_t ts;      /* global surface triangle index */
} tie_t;

/* weight of surface triangle T at point x lying on it: the interior angle when
 * x is one of its vertices, pi on an edge, 2 pi inside (angle-weighted
 * pseudonormal, Baerentzen & Aanaes 2005) */
static double corner_weight(const double *T, vec x, double eps) {
    vec v[3] = {mk(T), mk(T + 3), mk(T + 6)};
    for (int i = 0; i < 3; ++i)
        if (vnorm(vsub(x, v[i])) <= eps) {
            vec e1 = vsub(v[(i + 1) % 3], v[i]), e2 = vsub(v[(i + 2) % 3], v[i]);
            double c = vdot(e1, e2) / (vnorm(e1) * vnorm(e2));
            if (c > 1.0) c = 1.0;
            if (c < -1.0) c = -1.0;
            return acos(c);
        }
    for (int i = 0; i < 3; ++i) {
        vec cl;
        if (pt_seg(x, v[i], v[(i + 1) % 3], &cl) <= eps) return M_PI;
    }
    return 2.0 * M_PI;
}

/* Returns +1 (FIELD side), -1 (HOLE side); *dotmag = the deciding |cos|.
 * Ties whose surface closest points coincide form a group whose normal is the
 * angle-weighted average of its triangles' normals (the "average the normals"
 * case); between groups the largest |dot| decides (the "same-sign" case). */
static int paper_side(const tie_t *ties, int nt, const double *stris, double eps, double *dotmag) {
    int *grp = (int *)malloc(sizeof(int) * (size_t)(nt > 0 ? nt : 1));
    int ng = 0;
    for (int i = 0; i < nt; ++i) grp[i] = -1;
    int best_sign = 1;
    double best_mag = -1.0;
    for (int i = 0; i < nt; ++i) {
        if (grp[i] >= 0) continue;
        grp[i] = ng;
        for (int j = i + 1; j < nt; ++j)
            if (grp[j] < 0 && vnorm(vsub(ties[j].cs, ties[i].cs)) <= eps) grp[j] = ng;
        /* group members: distinct surface triangles */
        vec nsum = {0, 0, 0};
        int lead = i;
        for (int j = i; j < nt; ++j) {
            if (grp[j] != ng) continue;
            if (ties[j].d < ties[lead].d) lead = j;
            int dup = 0;
            for (int k = i; k < j; ++k)
                if (grp[k] == ng && ties[k].ts == ties[j].ts) { dup = 1; break; }
            if (dup) continue;
            const double *T = stris + 9 * ties[j].ts;
            vec n = vcross(vsub(mk(T + 3), mk(T)), vsub(mk(T + 6), mk(T)));
            double ln = vnorm(n);
            if (ln > 0.0) nsum = vadd(nsum, vscale(n, corner_weight(T, ties[i].cs, eps) / ln));
        }
        vec vv = vsub(ties[lead].ce, ties[lead].cs);
        double den = vnorm(vv) * vnorm(nsum);
        double c = den > 0.0 ? vdot(vv, nsum) / den : 0.0;
        if (fabs(c) > best_mag) { best_mag = fabs(c); best_sign = c > 0.0 ? 1 : -1; }
        ++ng;
    }
    free(grp);
    *dotmag = best_mag;
    return best_sign;
}

/* ------------------------------------------------------------------------ */
/* the cut                                                                   */
/* ------------------------------------------------------------------------ */
static void aabb_of(const double *pts, int n, double *bb) {
    for (int a = 0; a < 3; ++a) { bb[a] = INFINITY; bb[3 + a] = -INFINITY; }
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double x = pts[3 * i + a];
            if (x < bb[a]) bb[a] = x;
            if (x > bb[3 + a]) bb[3 + a] = x;
        }
}

/* Alg. bboxdix: Euclidean distance between two axis-aligned boxes
 * B = [min x, min y, min z, max x, max y, max z] (loop over the 3 axes). */
double orc_box_dist(const double *B1, const double *B2) {
    double D = 0.0;
    for (int i = 0; i < 3; ++i)
        if (B1[i + 3] < B2[i] || B2[i + 3] < B1[i]) {
            double d = fmax(B2[i] - B1[i + 3], B1[i] - B2[i + 3]);
            D += d * d;
        }
    return sqrt(D);
}

typedef struct { double lb; int64_t f; } lbf_t;
static int cmp_lbf(const void *x, const void *y) {
    const lbf_t *a = (const lbf_t *)x, *b = (const lbf_t *)y;
    if (a->lb < b->lb) return -1;
    if (a->lb > b->lb) return 1;
    return (a->f < b->f) ? -1 : (a->f > b->f);
}

static double tie_limit(double best) { return best * (1.0 + 1e-9) + 1e-14; }

/*
 * orc_cut: classify elements.
 *   p, n_elem, nodes           background, [n_elem][(p+1)^3][3]
 *   q, n_faces, faces, pose    cut surface [n_faces][(q+1)^2][3]; pose = 12
 *                              doubles [R|t] row-major or NULL
 *   tol                        fringe tolerance (absolute)
 *   brute                      1: all faces for every element; 0: pruned
 *   ids, n_ids                 elements to evaluate (NULL: all, n_ids ignored)
 *   flags, dist, paper_flags   outputs per evaluated element (any may be NULL)
 *   stats[8]                   [0] tri-tri tests, [1] S* element-face pairs
 *                              (box distance <= d(E)), [2] triangle pairs of S*
 *                              with triangle box distance <= d(E), [3] number
 *                              of undecidable elements, [4] paper-rule vs
 *                              winding disagreements, [5] fringe count,
 *                              [6] hole count, [7] field count
 * Returns 0, or -1 on bad arguments.
 */
int orc_cut(int p, int64_t n_elem, const double *nodes, int q, int64_t n_faces, const double *faces,
            const double *pose, double tol, int brute, const int64_t *ids, int64_t n_ids, int8_t *flags,
            double *dist, int8_t *paper_flags, int64_t *stats, int nthreads) {
    if (p < 1 || q < 1 || n_elem < 0 || n_faces < 1 || !nodes || !faces) return -1;
    const int npe = (p + 1) * (p + 1) * (p + 1), npf = (q + 1) * (q + 1);
    const int nte = 12 * p * p, ntf = 2 * q * q;
    const int64_t nts = n_faces * ntf;
    int64_t nev = ids ? n_ids : n_elem;

    double *fx = (double *)malloc(sizeof(double) * 3 * npf * n_faces);
    if (pose) orc_apply_pose(npf * n_faces, faces, pose, fx);
    else memcpy(fx, faces, sizeof(double) * 3 * npf * n_faces);
    double *stris = (double *)malloc(sizeof(double) * 9 * nts);
    double *fbox = (double *)malloc(sizeof(double) * 6 * n_faces);
    double *tbox = (double *)malloc(sizeof(double) * 6 * nts);
    for (int64_t f = 0; f < n_faces; ++f) {
        orc_face_tris(q, fx + 3 * npf * f, stris + 9 * ntf * f);
        aabb_of(fx + 3 * npf * f, npf, fbox + 6 * f);
    }
    for (int64_t t = 0; t < nts; ++t) aabb_of(stris + 9 * t, 3, tbox + 6 * t);

    int64_t st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        int64_t lst[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        double *etris = (double *)malloc(sizeof(double) * 9 * nte);
        double *ebox_t = (double *)malloc(sizeof(double) * 6 * nte);
        lbf_t *order = (lbf_t *)malloc(sizeof(lbf_t) * n_faces);
        int tcap = 256, nt = 0;
        tie_t *ties = (tie_t *)malloc(sizeof(tie_t) * tcap);
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < nev; ++k) {
            int64_t e = ids ? ids[k] : k;
            const double *en = nodes + 3 * npe * e;
            double ebox[6];
            aabb_of(en, npe, ebox);
            orc_elem_tris(p, en, etris);
            for (int t = 0; t < nte; ++t) aabb_of(etris + 9 * t, 3, ebox_t + 6 * t);
            for (int64_t f = 0; f < n_faces; ++f) {
                order[f].lb = orc_box_dist(ebox, fbox + 6 * f);
                order[f].f = f;
            }
            if (!brute) qsort(order, (size_t)n_faces, sizeof(lbf_t), cmp_lbf);
            double best = INFINITY;
            nt = 0;
            for (int64_t oi = 0; oi < n_faces; ++oi) {
                if (!brute && order[oi].lb > tie_limit(best)) break;
                int64_t f = order[oi].f;
                for (int ts = 0; ts < ntf; ++ts) {
                    const double *Ts = stris + 9 * (f * ntf + ts);
                    for (int te = 0; te < nte; ++te) {
                        double ca[3], cb[3];
                        double d = orc_tritri(etris + 9 * te, Ts, ca, cb);
                        lst[0]++;
                        if (d <= tie_limit(best)) {
                            if (nt == tcap) { tcap *= 2; ties = (tie_t *)realloc(ties, sizeof(tie_t) * tcap); }
                            ties[nt].d = d; ties[nt].ce = mk(ca); ties[nt].cs = mk(cb);
                            ties[nt].ts = f * ntf + ts;
                            ++nt;
                            if (d < best) {
                                best = d;
                                int w = 0;   /* drop ties that no longer qualify */
                                for (int i = 0; i < nt; ++i)
                                    if (ties[i].d <= tie_limit(best)) ties[w++] = ties[i];
                                nt = w;
                            }
                        }
                    }
                }
            }
            /* necessary-work counts for this element */
            for (int64_t f = 0; f < n_faces; ++f) {
                double lb = orc_box_dist(ebox, fbox + 6 * f);
                if (lb > best) continue;
                lst[1]++;
                for (int ts = 0; ts < ntf; ++ts)
                    for (int te = 0; te < nte; ++te)
                        if (orc_box_dist(ebox_t + 6 * te, tbox + 6 * (f * ntf + ts)) <= best) lst[2]++;
            }
            int8_t fl, pf;
            int undecidable = fabs(best - tol) < 1e-12;
            if (best <= tol) {
                fl = ORC_FRINGE;
                pf = ORC_FRINGE;
            } else {
                double w = orc_winding(en, nts, stris);
                fl = (w > 0.5) ? ORC_HOLE : ORC_FIELD;
                double scale = fmax(ebox[3] - ebox[0], fmax(ebox[4] - ebox[1], ebox[5] - ebox[2]));
                double mag;
                int s = paper_side(ties, nt, stris, 1e-9 * scale, &mag);
                pf = (s > 0) ? ORC_FIELD : ORC_HOLE;
                if (mag < 1e-12) undecidable = 1;
                if (fabs(w - 0.5) < 0.25) undecidable = 1;
            }
            if (undecidable) lst[3]++;
            if (pf != fl) lst[4]++;
            if (fl == ORC_FRINGE) lst[5]++;
            else if (fl == ORC_HOLE) lst[6]++;
            else lst[7]++;
            if (flags) flags[k] = fl;
            if (paper_flags) paper_flags[k] = pf;
            if (dist) dist[k] = (fl == ORC_HOLE) ? -best : best;
        }
#pragma omp critical
        for (int i = 0; i < 8; ++i) st[i] += lst[i];
        free(etris);
        free(ebox_t);
        free(order);
        free(ties);
    }
    if (stats) memcpy(stats, st, sizeof(st));
    free(fx);
    free(stris);
    free(fbox);
    free(tbox);
    return 0;
}

/* distance from P to the linearised surface and its winding number */
double orc_point_surface(const double *P, int64_t ntri, const double *tris, double *winding) {
    vec p = mk(P);
    double best = INFINITY;
    for (int64_t t = 0; t < ntri; ++t) {
        double d = pt_tri(p, mk(tris + 9 * t), mk(tris + 9 * t + 3), mk(tris + 9 * t + 6), NULL);
        if (d < best) best = d;
    }
    if (winding) *winding = orc_winding(P, ntri, tris);
    return best;
}
