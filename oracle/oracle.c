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
 * The paper's truncating variant (orc_heuristic, end of file) is here too:
 * OBB keys, the 16 nearest faces, pass 1 on corner triangles, the 4 nearest,
 * pass 2 on the three element faces at the nearest corner.  Its steps are
 * pinned one by one; the effect of the truncations on the result is parity
 * unpinned (the paper gives no reference output for it), and is what the tests
 * measure against the exact result above.
 *
 * The donor search of the point-connectivity step (orc_locate, end of file)
 * is the plain definition: every element whose box holds the point, in index
 * order, then the paper's clamped Newton inversion of the isoparametric map.
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

/* Distance of element-face pairs (Sec. 4.2, the curved element-face test of
 * Alg. cp2, here over all triangles, with no truncation): d(E, F) = the
 * minimum over E's 12 p^2 boundary triangles and F's 2 q^2 triangles of the
 * closed-triangle distance.  For each of the n pairs (elem[k], face[k]) of the
 * given (already posed) faces; OpenMP over the pairs.  The element-surface
 * distance d(E) is the minimum of d(E, F) over all faces F.
 * Returns 0, or -1 on bad arguments. */
int orc_pair_dist(int p, int64_t n_elem, const double *nodes, int q, int64_t n_faces, const double *faces,
                  int64_t n, const int64_t *elem, const int64_t *face, double *out, int nthreads) {
    if (p < 1 || q < 1 || n_elem < 1 || n_faces < 1 || n < 0 || !nodes || !faces || !elem || !face || !out)
        return -1;
    for (int64_t k = 0; k < n; ++k)
        if (elem[k] < 0 || elem[k] >= n_elem || face[k] < 0 || face[k] >= n_faces) return -1;
    const int npe = (p + 1) * (p + 1) * (p + 1), npf = (q + 1) * (q + 1);
    const int nte = 12 * p * p, ntf = 2 * q * q;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        double *etris = (double *)malloc(sizeof(double) * 9 * nte);
        double *ftris = (double *)malloc(sizeof(double) * 9 * ntf);
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < n; ++k) {
            orc_elem_tris(p, nodes + 3 * npe * elem[k], etris);
            orc_face_tris(q, faces + 3 * npf * face[k], ftris);
            double best = INFINITY;
            for (int i = 0; i < nte; ++i)
                for (int j = 0; j < ntf; ++j) {
                    double d = orc_tritri(etris + 9 * i, ftris + 9 * j, NULL, NULL);
                    if (d < best) best = d;
                }
            out[k] = best;
        }
        free(etris);
        free(ftris);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* the paper's truncating variant (Sec. 4.2 and Alg. cp0, bboxdix, cp1, cp2)  */
/* ------------------------------------------------------------------------ */
/*
 * The fast variant the paper runs on every filtered element E, with the
 * truncations it describes.  Parity unpinned: whether its answer matches the
 * exact one depends on the truncation (the paper says so for skewed elements);
 * the steps themselves are pinned separately (OBB, keys, pass 1, pass 2).
 *
 *   0. OBB of E from its 8 corner nodes: centroid e_cg, axes = eigenvectors of
 *      the corners' covariance (cyclic Jacobi), extents B_e = box of the
 *      rotated corners.
 *   1. Alg. cp0: for every face F, rotate its 4 corner nodes into the OBB axes,
 *      B_f = their box, key = 0.01 |f_cg - e_cg| + boxDist(B_f, B_e), f_cg
 *      the mean of F's corners.  Keep the nf1 (16) smallest keys (ties: lower
 *      face id).
 *   2. Alg. cp1: for each kept face, corner c of E nearest to f_cg (lowest
 *      index on ties); the 3 faces of E at c, each its corner quad split into 2
 *      triangles; F's corner quad split into 2 triangles; D1 = the smallest of
 *      the 12 triangle distances, 0 when below tol.  Keep the nf2 (4) smallest
 *      D1 (ties: the key order of step 1).
 *   3. Alg. cp2: for each face kept there, the order-p triangles of the 3
 *      faces of E at its corner c against F's 2q^2 triangles; a distance below
 *      tol makes the element intersecting.
 *   4. Smallest distance below tol: FRINGE.  Otherwise the side from the
 *      minimal vector and the outward normal, over the triangle pairs at the
 *      smallest distance (the same tie rule as the exact oracle: coincident
 *      surface points average their normals, otherwise the largest |dot|).
 *
 * margins[6] per element, how far each decision was from going the other way:
 *   [0] key gap between the nf1-th and (nf1+1)-th face (INF when all kept),
 *   [1] smallest gap between the nearest and second-nearest corner over the
 *       kept faces, [2] D1 gap at the nf2 boundary (INF when both are 0),
 *   [3] key gap of the two boundary faces when both D1 are 0 (else INF),
 *   [4] |D2min - tol|, [5] the deciding |cos| of the side rule (INF when
 *   FRINGE).
 * flagset per element: bit (flag + 1) for each flag reached by the selection
 * in the paper's order and by every other selection an exact D1 tie at the
 * nf2 boundary allows (faces sharing the nearest edge tie exactly, and which
 * of them a computation keeps is then a matter of rounding).
 */
static void jacobi3(double A[3][3], double V[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
        double scale = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
        if (off <= 1e-15 * scale || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {       /* A <- A J (columns p, q) */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {       /* A <- J^T A (rows p, q) */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {       /* V <- V J */
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
}

/* OBB of n points: axes R (rows, unit) and box of the rotated points */
void orc_obb(const double *pts, int n, double *R, double *box, double *cg) {
    vec c = {0, 0, 0};
    for (int i = 0; i < n; ++i) c = vadd(c, mk(pts + 3 * i));
    c = vscale(c, 1.0 / n);
    double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, V[3][3];
    for (int i = 0; i < n; ++i) {
        vec d = vsub(mk(pts + 3 * i), c);
        double v[3] = {d.x, d.y, d.z};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) A[a][b] += v[a] * v[b] / n;
    }
    jacobi3(A, V);
    for (int r = 0; r < 3; ++r)
        for (int a = 0; a < 3; ++a) R[3 * r + a] = V[a][r];   /* row r = eigenvector r */
    for (int a = 0; a < 3; ++a) { box[a] = INFINITY; box[3 + a] = -INFINITY; }
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < 3; ++r) {
            double x = R[3 * r] * pts[3 * i] + R[3 * r + 1] * pts[3 * i + 1] + R[3 * r + 2] * pts[3 * i + 2];
            if (x < box[r]) box[r] = x;
            if (x > box[3 + r]) box[3 + r] = x;
        }
    if (cg) store(cg, c);
}

/* Alg. cp0: approximate distance of face corners Xf[4] to an element OBB */
double orc_approx_dist(const double *R, const double *Be, const double *ecg, const double *Xf) {
    double Bf[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    vec fcg = {0, 0, 0};
    for (int i = 0; i < 4; ++i) {
        fcg = vadd(fcg, mk(Xf + 3 * i));
        for (int r = 0; r < 3; ++r) {
            double x = R[3 * r] * Xf[3 * i] + R[3 * r + 1] * Xf[3 * i + 1] + R[3 * r + 2] * Xf[3 * i + 2];
            if (x < Bf[r]) Bf[r] = x;
            if (x > Bf[3 + r]) Bf[3 + r] = x;
        }
    }
    fcg = vscale(fcg, 0.25);
    return 0.01 * vnorm(vsub(fcg, mk(ecg))) + orc_box_dist(Bf, Be);
}

/* corner c (i + 2j + 4k) of an order-p element: node (i p, j p, k p) */
static int corner_node(int p, int c) { return node_index(p, (c & 1) * p, ((c >> 1) & 1) * p, ((c >> 2) & 1) * p); }

/* Alg. cp1: nearest corner to the face centroid, and the distance between the
 * corner triangles of the 3 element faces at that corner and the face's 2
 * corner triangles (0 below tol).  Returns D1; *corner, *gap (second-nearest
 * corner distance minus nearest). */
double orc_pass1(int p, const double *en, int q, const double *fn, double tol, int *corner, double *gap) {
    const int npf = (q + 1) * (q + 1);
    int fc[4] = {0, q, npf - 1, q * (q + 1)};             /* (0,0) (q,0) (q,q) (0,q) */
    vec fcg = {0, 0, 0};
    for (int i = 0; i < 4; ++i) fcg = vadd(fcg, mk(fn + 3 * fc[i]));
    fcg = vscale(fcg, 0.25);
    double best = INFINITY, second = INFINITY;
    int c = 0;
    for (int i = 0; i < 8; ++i) {
        double d = vnorm(vsub(mk(en + 3 * corner_node(p, i)), fcg));
        if (d < best) { second = best; best = d; c = i; }
        else if (d < second) second = d;
    }
    *corner = c;
    *gap = second - best;
    double TF[2][9];
    int tf[2][3] = {{0, 1, 2}, {0, 2, 3}};                 /* (00,10,11), (00,11,01) */
    for (int h = 0; h < 2; ++h)
        for (int v = 0; v < 3; ++v) memcpy(TF[h] + 3 * v, fn + 3 * fc[tf[h][v]], 3 * sizeof(double));
    int fsel[3] = {c & 1, 2 + ((c >> 1) & 1), 4 + ((c >> 2) & 1)};
    double D = INFINITY;
    for (int k = 0; k < 3; ++k) {
        int f = fsel[k];
        int n00 = face_node(p, f, 0, 0), n10 = face_node(p, f, p, 0), n11 = face_node(p, f, p, p), n01 = face_node(p, f, 0, p);
        int tri[2][3] = {{n00, n10, n11}, {n00, n11, n01}};
        for (int h = 0; h < 2; ++h) {
            double TC[9];
            for (int v = 0; v < 3; ++v) memcpy(TC + 3 * v, en + 3 * tri[h][v], 3 * sizeof(double));
            for (int j = 0; j < 2; ++j) {
                double d = orc_tritri(TC, TF[j], NULL, NULL);
                if (d < D) D = d;
            }
        }
    }
    return D < tol ? 0.0 : D;
}

typedef struct { double key, d1; int64_t f; int rank, corner; } hface_t;
static int cmp_key(const void *x, const void *y) {
    const hface_t *a = (const hface_t *)x, *b = (const hface_t *)y;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->f < b->f) ? -1 : (a->f > b->f);
}
static int cmp_d1(const void *x, const void *y) {
    const hface_t *a = (const hface_t *)x, *b = (const hface_t *)y;
    if (a->d1 < b->d1) return -1;
    if (a->d1 > b->d1) return 1;
    return a->rank - b->rank;
}

/* pass 2 (Alg. cp2) of one kept face, computed once per element and face:
 * the smallest triangle distance, whether one fell below tol, and the pairs
 * within the tie limit of that smallest distance */
typedef struct { int done, hit, nt, cap; double best; tie_t *ties; } pass2_t;

static void heur_pass2(int p, int q, const double *etris, const double *stris, const hface_t *h, double tol,
                       pass2_t *r) {
    const int ntf = 2 * q * q, tpf = 2 * p * p;
    const int c = h->corner;
    const int fsel[3] = {c & 1, 2 + ((c >> 1) & 1), 4 + ((c >> 2) & 1)};
    r->best = INFINITY;
    r->hit = 0;
    r->nt = 0;
    for (int s = 0; s < 3 && !r->hit; ++s)
        for (int t = 0; t < tpf && !r->hit; ++t) {
            const double *Te = etris + 9 * (fsel[s] * tpf + t);
            for (int ts = 0; ts < ntf; ++ts) {
                double ca[3], cb[3];
                double d = orc_tritri(Te, stris + 9 * (h->f * ntf + ts), ca, cb);
                if (d < tol) { r->best = d; r->hit = 1; break; }   /* the "return 0" of Alg. cp2 */
                if (d <= tie_limit(r->best)) {
                    if (r->nt == r->cap) { r->cap *= 2; r->ties = (tie_t *)realloc(r->ties, sizeof(tie_t) * r->cap); }
                    r->ties[r->nt].d = d; r->ties[r->nt].ce = mk(ca); r->ties[r->nt].cs = mk(cb);
                    r->ties[r->nt].ts = h->f * ntf + ts;
                    ++r->nt;
                    if (d < r->best) {
                        r->best = d;
                        int w = 0;
                        for (int j = 0; j < r->nt; ++j)
                            if (r->ties[j].d <= tie_limit(r->best)) r->ties[w++] = r->ties[j];
                        r->nt = w;
                    }
                }
            }
        }
    r->done = 1;
}

/* steps 3-4 for the kept faces sel[0..nsel): FRINGE when a distance falls
 * below tol, else the side rule over the pairs at the smallest distance */
static int8_t heur_decide(int p, int q, const double *en, const double *etris, const double *stris,
                          const hface_t *hf, const int *sel, int nsel, pass2_t *p2, double tol, double scale,
                          double *best_out, tie_t **ties, int *tcap, double *cosmag) {
    (void)en;
    double best = INFINITY;
    int hit = 0;
    for (int i = 0; i < nsel; ++i) {
        pass2_t *r = &p2[sel[i]];
        if (!r->done) heur_pass2(p, q, etris, stris, &hf[sel[i]], tol, r);
        if (r->hit) hit = 1;
        if (r->best < best) best = r->best;
    }
    *best_out = best;
    *cosmag = INFINITY;
    if (hit || best < tol) return ORC_FRINGE;
    int nt = 0;
    for (int i = 0; i < nsel; ++i) {
        const pass2_t *r = &p2[sel[i]];
        for (int j = 0; j < r->nt; ++j)
            if (r->ties[j].d <= tie_limit(best)) {
                if (nt == *tcap) { *tcap *= 2; *ties = (tie_t *)realloc(*ties, sizeof(tie_t) * (*tcap)); }
                (*ties)[nt++] = r->ties[j];
            }
    }
    double mag;
    int s = paper_side(*ties, nt, stris, 1e-9 * scale, &mag);
    *cosmag = mag;
    return s > 0 ? ORC_FIELD : ORC_HOLE;
}

int orc_heuristic(int p, int64_t n_elem, const double *nodes, int q, int64_t n_faces, const double *faces,
                  const double *pose, double tol, int nf1, int nf2, const int64_t *ids, int64_t n_ids, int8_t *flags,
                  uint8_t *flagset, double *dist, double *margins, int nthreads) {
    if (p < 1 || q < 1 || n_elem < 0 || n_faces < 1 || !nodes || !faces || nf1 < 1 || nf2 < 1 || nf2 > nf1 || nf1 > 64)
        return -1;
    const int npe = (p + 1) * (p + 1) * (p + 1), npf = (q + 1) * (q + 1);
    const int nte = 12 * p * p, ntf = 2 * q * q;
    const int64_t nts = n_faces * ntf;
    const int64_t nev = ids ? n_ids : n_elem;
    double *fx = (double *)malloc(sizeof(double) * 3 * npf * n_faces);
    if (pose) orc_apply_pose(npf * n_faces, faces, pose, fx);
    else memcpy(fx, faces, sizeof(double) * 3 * npf * n_faces);
    double *stris = (double *)malloc(sizeof(double) * 9 * nts);
    double *fcorn = (double *)malloc(sizeof(double) * 12 * n_faces);
    const int fc[4] = {0, q, npf - 1, q * (q + 1)};
    for (int64_t f = 0; f < n_faces; ++f) {
        orc_face_tris(q, fx + 3 * npf * f, stris + 9 * ntf * f);
        for (int i = 0; i < 4; ++i) memcpy(fcorn + 12 * f + 3 * i, fx + 3 * (npf * f + fc[i]), 3 * sizeof(double));
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        hface_t *hf = (hface_t *)malloc(sizeof(hface_t) * (size_t)n_faces);
        double *etris = (double *)malloc(sizeof(double) * 9 * nte);
        int tcap = 256;
        tie_t *ties = (tie_t *)malloc(sizeof(tie_t) * tcap);
        pass2_t p2[64];
        for (int i = 0; i < 64; ++i) { p2[i].cap = 32; p2[i].ties = (tie_t *)malloc(sizeof(tie_t) * 32); }
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < nev; ++k) {
            int64_t e = ids ? ids[k] : k;
            const double *en = nodes + 3 * npe * e;
            double cpts[24], R[9], Be[6], ecg[3];
            for (int c = 0; c < 8; ++c) memcpy(cpts + 3 * c, en + 3 * corner_node(p, c), 3 * sizeof(double));
            orc_obb(cpts, 8, R, Be, ecg);
            /* step 1 */
            for (int64_t f = 0; f < n_faces; ++f) {
                hf[f].key = orc_approx_dist(R, Be, ecg, fcorn + 12 * f);
                hf[f].f = f;
            }
            qsort(hf, (size_t)n_faces, sizeof(hface_t), cmp_key);
            const int n1 = n_faces < nf1 ? (int)n_faces : nf1;
            double m[6] = {INFINITY, INFINITY, INFINITY, INFINITY, INFINITY, INFINITY};
            if (n_faces > nf1) m[0] = hf[nf1].key - hf[nf1 - 1].key;
            /* step 2 */
            for (int i = 0; i < n1; ++i) {
                double gap;
                hf[i].rank = i;
                hf[i].d1 = orc_pass1(p, en, q, fx + 3 * npf * hf[i].f, tol, &hf[i].corner, &gap);
                if (gap < m[1]) m[1] = gap;
            }
            qsort(hf, (size_t)n1, sizeof(hface_t), cmp_d1);
            const int n2 = n1 < nf2 ? n1 : nf2;
            if (n1 > nf2) {
                const hface_t *a = &hf[nf2 - 1], *b = &hf[nf2];
                if (a->d1 == 0.0 && b->d1 == 0.0) {
                    /* both zero: the key order of step 1 decided */
                    m[3] = fabs(hf[nf2].key - hf[nf2 - 1].key);
                    for (int i = 0; i < nf2; ++i)
                        if (hf[i].d1 == 0.0) {
                            for (int j = nf2; j < n1; ++j)
                                if (hf[j].d1 == 0.0 && fabs(hf[j].key - hf[i].key) < m[3]) m[3] = fabs(hf[j].key - hf[i].key);
                        }
                } else {
                    m[2] = b->d1 - a->d1;
                }
            }
            /* steps 3-4 for the selection the paper's order gives, and for every
             * other selection that an exact D1 tie at the nf2 boundary allows */
            orc_elem_tris(p, en, etris);
            double scale = 0.0;
            for (int a = 0; a < 3; ++a) if (Be[3 + a] - Be[a] > scale) scale = Be[3 + a] - Be[a];
            for (int i = 0; i < n1; ++i) p2[i].done = 0;
            int sel[64], nsel = 0;
            for (int i = 0; i < n2; ++i) sel[nsel++] = i;
            double best;
            int8_t fl = heur_decide(p, q, en, etris, stris, hf, sel, nsel, p2, tol, scale, &best, &ties, &tcap, &m[5]);
            m[4] = fabs(best - tol);
            unsigned fs = 1u << (fl + 1);
            if (n1 > nf2 && hf[nf2 - 1].d1 > 0.0) {
                const double v = hf[nf2 - 1].d1, lim = v * (1.0 + 1e-12) + 1e-15;
                int lo = 0, hiT = 0;       /* faces below the tie band, faces in it */
                int tied[16];
                for (int i = 0; i < n1; ++i) {
                    if (hf[i].d1 < v - (lim - v)) ++lo;
                    else if (hf[i].d1 <= lim && hiT < 16) tied[hiT++] = i;
                }
                const int need = nf2 - lo;
                if (hiT > need && need > 0 && hiT <= 12) {
                    for (unsigned mask = 0; mask < (1u << hiT); ++mask) {
                        if (__builtin_popcount(mask) != need) continue;
                        nsel = 0;
                        for (int i = 0; i < lo; ++i) sel[nsel++] = i;
                        for (int t = 0; t < hiT; ++t) if (mask >> t & 1u) sel[nsel++] = tied[t];
                        double b2, c2;
                        int8_t f2 = heur_decide(p, q, en, etris, stris, hf, sel, nsel, p2, tol, scale, &b2, &ties, &tcap, &c2);
                        fs |= 1u << (f2 + 1);
                    }
                } else if (hiT > need && need > 0) {
                    fs = 7u;   /* too many tied faces to enumerate: any flag */
                }
            }
            if (flags) flags[k] = fl;
            if (flagset) flagset[k] = (uint8_t)fs;
            if (dist) dist[k] = fl == ORC_HOLE ? -best : best;
            if (margins) memcpy(margins + 6 * k, m, sizeof(m));
        }
        free(hf);
        free(etris);
        free(ties);
        for (int i = 0; i < 64; ++i) free(p2[i].ties);
    }
    free(fx);
    free(stris);
    free(fcorn);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* donor search for receptor points (Sec. "Donor/Receptor Point             */
/* Connectivity on GPUs", Eqs. reftophys, ref-update, Jac)                   */
/* ------------------------------------------------------------------------ */
/*
 * For each point x_p (world frame) and a donor grid of order-p hexes moved
 * rigidly by pose [R|t] (initial frame -> world; NULL: identity):
 *   1. the point in the grid's initial frame: x = R^T (x_p - t);
 *   2. every element whose node box contains x (brute force over all
 *      elements, in index order; the ADT of the paper only finds these
 *      faster);
 *   3. Newton on the isoparametric map x(xi) = sum_ijk x_ijk l_i(xi) l_j(eta)
 *      l_k(zeta) (Lagrange basis on the p+1 equispaced nodes of [-1,1]):
 *      xi^0 = 0, xi^{n+1} = xi^n + J^{-1}(xi^n) (x - x(xi^n)), each component
 *      clamped to [-1 - 1e-4, 1 + 1e-4], at most 10 iterations, stopping when
 *      |x - x(xi)| <= 1e-10 h (h: the element box's largest side);
 *   4. the donor is the first element (lowest index) where the iteration
 *      stopped that way with max |xi_a| <= 1 + 1e-8; its xi is returned.
 *      No such element: donor -1.
 * margins[2] per point: residual gap (1e-10 h - |x - x(xi)|) and reference
 * gap (1 + 1e-8 - max |xi_a|) of the returned donor (of the last element
 * tried when none is found), how close its acceptance was to flipping.
 */
#define ORC_NEWTON_ITERS 10
#define ORC_NEWTON_CLAMP 1e-4
#define ORC_INSIDE_TOL 1e-8
#define ORC_RESID_REL 1e-10

/* Lagrange basis on equispaced nodes of [-1,1] and its derivative */
void orc_lagrange(int p, double x, double *l, double *dl) {
    double nd[8];
    for (int i = 0; i <= p; ++i) nd[i] = -1.0 + 2.0 * i / p;
    for (int i = 0; i <= p; ++i) {
        double v = 1.0, dv = 0.0;
        for (int j = 0; j <= p; ++j) {
            if (j == i) continue;
            const double inv = 1.0 / (nd[i] - nd[j]);
            dv = dv * (x - nd[j]) * inv + v * inv;   /* product rule, left to right */
            v *= (x - nd[j]) * inv;
        }
        l[i] = v;
        if (dl) dl[i] = dv;
    }
}

/* x(xi) and the Jacobian d x / d xi (row a: component a) of one element */
void orc_map(int p, const double *en, const double *xi, double *x, double *J) {
    double lx[8], ly[8], lz[8], dx[8], dy[8], dz[8];
    orc_lagrange(p, xi[0], lx, dx);
    orc_lagrange(p, xi[1], ly, dy);
    orc_lagrange(p, xi[2], lz, dz);
    for (int a = 0; a < 3; ++a) { x[a] = 0.0; if (J) J[3 * a] = J[3 * a + 1] = J[3 * a + 2] = 0.0; }
    for (int k = 0; k <= p; ++k)
        for (int j = 0; j <= p; ++j)
            for (int i = 0; i <= p; ++i) {
                const double *X = en + 3 * node_index(p, i, j, k);
                const double N = lx[i] * ly[j] * lz[k];
                const double Nx = dx[i] * ly[j] * lz[k], Ny = lx[i] * dy[j] * lz[k], Nz = lx[i] * ly[j] * dz[k];
                for (int a = 0; a < 3; ++a) {
                    x[a] += X[a] * N;
                    if (J) { J[3 * a] += X[a] * Nx; J[3 * a + 1] += X[a] * Ny; J[3 * a + 2] += X[a] * Nz; }
                }
            }
}

/* solve J d = r (3x3, Cramer's rule); 0 when J is singular */
static int solve3(const double *J, const double *r, double *d) {
    const double c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
    const double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    if (!(fabs(det) > 0.0)) return 0;
    const double inv = 1.0 / det;
    d[0] = (r[0] * c00 + r[1] * (J[2] * J[7] - J[1] * J[8]) + r[2] * (J[1] * J[5] - J[2] * J[4])) * inv;
    d[1] = (r[0] * c01 + r[1] * (J[0] * J[8] - J[2] * J[6]) + r[2] * (J[2] * J[3] - J[0] * J[5])) * inv;
    d[2] = (r[0] * c02 + r[1] * (J[1] * J[6] - J[0] * J[7]) + r[2] * (J[0] * J[4] - J[1] * J[3])) * inv;
    return 1;
}

/* Eq. ref-update from xi = 0: returns 1 when the residual fell within
 * 1e-10 h; xi, the last residual norm and the iteration count out */
int orc_newton(int p, const double *en, const double *x, double h, double *xi, double *resid, int *iters) {
    xi[0] = xi[1] = xi[2] = 0.0;
    const double lim = 1.0 + ORC_NEWTON_CLAMP, tolx = ORC_RESID_REL * h;
    double X[3], J[9], r[3], d[3];
    int n = 0;
    for (;;) {
        orc_map(p, en, xi, X, J);
        for (int a = 0; a < 3; ++a) r[a] = x[a] - X[a];
        const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        *resid = rn;
        *iters = n;
        if (rn <= tolx) return 1;
        if (n == ORC_NEWTON_ITERS || !solve3(J, r, d)) return 0;
        for (int a = 0; a < 3; ++a) {
            double v = xi[a] + d[a];
            xi[a] = v < -lim ? -lim : (v > lim ? lim : v);
        }
        ++n;
    }
}

int orc_locate(int p, int64_t n_elem, const double *nodes, int64_t n_pts, const double *pts, const double *pose,
               int64_t *donor, double *ref, double *margins, int nthreads) {
    if (p < 1 || p > 7 || n_elem < 1 || n_pts < 0 || !nodes || !pts) return -1;
    const int npe = (p + 1) * (p + 1) * (p + 1);
    double *box = (double *)malloc(sizeof(double) * 6 * n_elem);
    for (int64_t e = 0; e < n_elem; ++e) aabb_of(nodes + 3 * npe * e, npe, box + 6 * e);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n_pts; ++k) {
        const double *P = pts + 3 * k;
        double x[3];
        if (pose) {
            const double q[3] = {P[0] - pose[3], P[1] - pose[7], P[2] - pose[11]};
            for (int a = 0; a < 3; ++a) x[a] = (pose[a] * q[0] + pose[4 + a] * q[1]) + pose[8 + a] * q[2];
        } else {
            x[0] = P[0]; x[1] = P[1]; x[2] = P[2];
        }
        int64_t found = -1;
        double xi[3] = {0, 0, 0}, m[2] = {-INFINITY, -INFINITY};
        for (int64_t e = 0; e < n_elem && found < 0; ++e) {
            const double *b = box + 6 * e;
            if (x[0] < b[0] || x[0] > b[3] || x[1] < b[1] || x[1] > b[4] || x[2] < b[2] || x[2] > b[5]) continue;
            const double h = fmax(b[3] - b[0], fmax(b[4] - b[1], b[5] - b[2]));
            double t[3], rn;
            int it;
            const int conv = orc_newton(p, nodes + 3 * npe * e, x, h, t, &rn, &it);
            const double mx = fmax(fabs(t[0]), fmax(fabs(t[1]), fabs(t[2])));
            m[0] = ORC_RESID_REL * h - rn;
            m[1] = 1.0 + ORC_INSIDE_TOL - mx;
            if (conv && mx <= 1.0 + ORC_INSIDE_TOL) {
                found = e;
                xi[0] = t[0]; xi[1] = t[1]; xi[2] = t[2];
            }
        }
        donor[k] = found;
        if (ref) { ref[3 * k] = xi[0]; ref[3 * k + 1] = xi[1]; ref[3 * k + 2] = xi[2]; }
        if (margins) { margins[2 * k] = m[0]; margins[2 * k + 1] = m[1]; }
    }
    free(box);
    return 0;
}
