/*
 * ccs_oracle.c -- plain, slow, FP64 CPU oracle for closest-hit ray intersection with bicubic Bezier
 * and Gregory patches by recursive (u,v) subdivision with sub-domain bounding boxes
 * (Binder & Keller, "Massively Parallel Stackless Ray Tracing of Catmull-Clark Subdivision Surfaces",
 * arXiv 1811.03510).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker of the CUDA library, not part of it: only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or constant with the CUDA path and includes nothing from it.
 *
 * What it computes.  The method does not solve the ray/surface equation; it returns the entry
 * distance of the closest hit leaf bounding box of the hierarchy of (u,v) sub-domains (Sec. 3,
 * Sec. 3.3: testing bounding boxes alone suffices).  This oracle computes exactly that
 * answer in FP64, with an explicit stack in place of the paper's bit trails:
 *   - domains split alternately along u and v, starting with u (Sec. 3.3; Algorithm 3), leaf depth L
 *     splits per axis, i.e. 2L tree levels;
 *   - Bezier node control points are the de Casteljau halves of the parent's (Sec. 3.1);
 *   - Gregory nodes recompute (q, d) = calcPointsAndD(p_org, D) on their own domain D (Algorithm 2,
 *     with Algorithm 1 for the crop), and their children are the de Casteljau halves of q with the
 *     upper corner raised by d (Sec. 3.3: the displacement bound comes from the coarser level);
 *   - the ray interval of a node is its box's slab interval intersected with its parent's interval,
 *     which makes the boxes nested, so the answer does not depend on traversal order;
 *   - both children are tested, the nearer one is descended first, ties go to the lower half
 *     (Sec. 3.3; Algorithm 3); nodes whose entry exceeds the best distance are pruned;
 *   - leaves are compared by the key (t_entry, patch id, cell index), smaller wins.
 *
 * Readings of the paper this file takes (the paper is silent or inconsistent there):
 *   A1 Gregory weights: p_ij(u,v) = p^v + h_ij (p^u - p^v) with h_11 = u/(u+v), h_21 = (1-u)/((1-u)+v),
 *      h_12 = u/(u+(1-v)), h_22 = (1-u)/((1-u)+(1-v)), the convention of Algorithm 2 (the weight table
 *      of Sec. 3.2 prints the swapped one).
 *   A2 Bernstein bounds: w_{.,1} is clamped toward 1/3 with 3w(1-w)^2, w_{.,2} toward 2/3 with 3w^2(1-w),
 *      as in Algorithm 2 (the text's example formula belongs to B_2).
 *   A4 0/0 in h at a domain corner: h = 1/2 (its Bernstein weight is zero there).
 *   A6 backtracking: replaced by the explicit stack, which visits the same nodes in the same order.
 *   A9 reported (u, v): centre of the leaf cell; reported t: the leaf's entry distance.
 *
 * Parity is pinned in tests/test_oracle_*.py against closed forms (planar and bilinear patches),
 * invariants (convex hull, Gregory inner-point and displacement bounds, Gregory == Bezier when
 * p^u == p^v), brute force over all leaves, and dense tessellation.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_SCALE_BITS 52   /* domain positions are integers in [0, 2^52] */
#define ORC_MAX_L 26

typedef struct { double x, y, z; } v3;

static v3 v3make(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return v3make(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return v3make(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return v3make(a.x * s, a.y * s, a.z * s); }
static v3 vmin(v3 a, v3 b) { return v3make(fmin(a.x, b.x), fmin(a.y, b.y), fmin(a.z, b.z)); }
static v3 vmax(v3 a, v3 b) { return v3make(fmax(a.x, b.x), fmax(a.y, b.y), fmax(a.z, b.z)); }
static v3 vabs(v3 a) { return v3make(fabs(a.x), fabs(a.y), fabs(a.z)); }
static double comp(v3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

/* ------------------------------------------------------------------------------------------------
 * Bicubic Bezier patch: f(u,v) = sum_{i,j} B_i^3(u) B_j^3(v) p_ij, p_ij stored at index 4*j + i
 * (i along u, j along v).  Sec. 3.1.
 * ---------------------------------------------------------------------------------------------- */

static void bernstein(double t, double B[4])
{
    double s = 1.0 - t;
    B[0] = s * s * s;
    B[1] = 3.0 * t * s * s;
    B[2] = 3.0 * t * t * s;
    B[3] = t * t * t;
}

static void bernstein_d(double t, double D[4])
{
    double s = 1.0 - t;
    D[0] = -3.0 * s * s;
    D[1] = 3.0 * s * s - 6.0 * t * s;
    D[2] = 6.0 * t * s - 3.0 * t * t;
    D[3] = 3.0 * t * t;
}

/* derivative order (du, dv) in {0,1} of the tensor product surface */
static v3 eval_bezier_d(const v3 p[16], double u, double v, int du, int dv)
{
    double Bu[4], Bv[4];
    if (du) bernstein_d(u, Bu); else bernstein(u, Bu);
    if (dv) bernstein_d(v, Bv); else bernstein(v, Bv);
    v3 r = v3make(0, 0, 0);
    for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i)
            r = add(r, scl(p[4 * j + i], Bu[i] * Bv[j]));
    return r;
}

static v3 evalBezier(const v3 p[16], double u, double v) { return eval_bezier_d(p, u, v, 0, 0); }
static v3 evalBezierDu(const v3 p[16], double u, double v) { return eval_bezier_d(p, u, v, 1, 0); }
static v3 evalBezierDv(const v3 p[16], double u, double v) { return eval_bezier_d(p, u, v, 0, 1); }
static v3 evalBezierDuDv(const v3 p[16], double u, double v) { return eval_bezier_d(p, u, v, 1, 1); }

/* Algorithm 1 (cropBezierPatch): control points q of the patch restricted to [u0,u1] x [v0,v1],
 * from corner values, corner first derivatives and corner twists.  q is indexed q[4*j + i] = q_{i,j}. */
static void cropBezierPatch(const v3 p[16], double u0, double u1, double v0, double v1, v3 q[16])
{
    double Du = (u1 - u0) / 3.0;
    double Dv = (v1 - v0) / 3.0;
#define Q(i, j) q[4 * (j) + (i)]
    /* corners */
    Q(0, 0) = evalBezier(p, u0, v0);
    Q(3, 0) = evalBezier(p, u1, v0);
    Q(0, 3) = evalBezier(p, u0, v1);
    Q(3, 3) = evalBezier(p, u1, v1);
    /* points on the boundary */
    Q(1, 0) = add(Q(0, 0), scl(evalBezierDu(p, u0, v0), Du));
    Q(2, 0) = sub(Q(3, 0), scl(evalBezierDu(p, u1, v0), Du));
    Q(0, 1) = add(Q(0, 0), scl(evalBezierDv(p, u0, v0), Dv));
    Q(3, 1) = add(Q(3, 0), scl(evalBezierDv(p, u1, v0), Dv));
    Q(0, 2) = sub(Q(0, 3), scl(evalBezierDv(p, u0, v1), Dv));
    Q(3, 2) = sub(Q(3, 3), scl(evalBezierDv(p, u1, v1), Dv));
    Q(1, 3) = add(Q(0, 3), scl(evalBezierDu(p, u0, v1), Du));
    Q(2, 3) = sub(Q(3, 3), scl(evalBezierDu(p, u1, v1), Du));
    /* inner control points */
    Q(1, 1) = add(add(Q(1, 0), scl(evalBezierDv(p, u0, v0), Dv)), scl(evalBezierDuDv(p, u0, v0), Du * Dv));
    Q(2, 1) = sub(sub(Q(3, 1), scl(evalBezierDu(p, u1, v0), Du)), scl(evalBezierDuDv(p, u1, v0), Du * Dv));
    Q(1, 2) = sub(sub(Q(1, 3), scl(evalBezierDv(p, u0, v1), Dv)), scl(evalBezierDuDv(p, u0, v1), Du * Dv));
    Q(2, 2) = add(sub(Q(2, 3), scl(evalBezierDv(p, u1, v1), Dv)), scl(evalBezierDuDv(p, u1, v1), Du * Dv));
#undef Q
}

/* de Casteljau subdivision at 1/2 along axis (0 = u, 1 = v), Sec. 3.1 / Sec. 3.4. */
static void subdivideDeCasteljau(const v3 p[16], int axis, v3 L[16], v3 R[16])
{
    for (int r = 0; r < 4; ++r) {
        int idx[4];
        for (int k = 0; k < 4; ++k) idx[k] = axis == 0 ? 4 * r + k : 4 * k + r;
        v3 b0 = p[idx[0]], b1 = p[idx[1]], b2 = p[idx[2]], b3 = p[idx[3]];
        v3 m01 = scl(add(b0, b1), 0.5), m12 = scl(add(b1, b2), 0.5), m23 = scl(add(b2, b3), 0.5);
        v3 m012 = scl(add(m01, m12), 0.5), m123 = scl(add(m12, m23), 0.5);
        v3 m = scl(add(m012, m123), 0.5);
        L[idx[0]] = b0; L[idx[1]] = m01; L[idx[2]] = m012; L[idx[3]] = m;
        R[idx[0]] = m; R[idx[1]] = m123; R[idx[2]] = m23; R[idx[3]] = b3;
    }
}

/* ------------------------------------------------------------------------------------------------
 * Gregory patch, Sec. 3.2.  20 points: slots 0..15 the 4x4 grid with p^u in the inner slots
 * (1,1),(2,1),(1,2),(2,2); slots 16..19 p^v of the same inner points, in that order.
 * ---------------------------------------------------------------------------------------------- */

static const int INNER_SLOT[4] = {5, 6, 9, 10};   /* (1,1), (2,1), (1,2), (2,2) */

static double ratio_or_half(double a, double b)   /* a / (a + b); reading A4: 1/2 when 0/0 */
{
    double s = a + b;
    return s == 0.0 ? 0.5 : a / s;
}

/* h_ij(u, v), the weight of p^u (reading A1) */
static double gregory_h(int k, double u, double v)
{
    switch (k) {
    case 0: return ratio_or_half(u, v);                       /* (1,1) */
    case 1: return ratio_or_half(1.0 - u, v);                 /* (2,1) */
    case 2: return ratio_or_half(u, 1.0 - v);                 /* (1,2) */
    default: return ratio_or_half(1.0 - u, 1.0 - v);          /* (2,2) */
    }
}

/* the Bezier patch a Gregory patch reduces to at (u, v) */
static void gregory_reduce(const v3 g[20], double u, double v, v3 p[16])
{
    memcpy(p, g, 16 * sizeof(v3));
    for (int k = 0; k < 4; ++k) {
        v3 pu = g[INNER_SLOT[k]], pv = g[16 + k];
        p[INNER_SLOT[k]] = add(pv, scl(sub(pu, pv), gregory_h(k, u, v)));
    }
}

static v3 eval_gregory(const v3 g[20], double u, double v)
{
    v3 p[16];
    gregory_reduce(g, u, v, p);
    return evalBezier(p, u, v);
}

/* Algorithm 2 (calcPointsAndD): lower bounding Bezier patch q restricted to D and the displacement
 * d of the upper bound.  For a Bezier patch the lower patch is the patch itself and d = 0.
 * pmin/pmax (optional) receive the bounds of the four inner points over D. */
static void calcPointsAndD(const v3 g[20], int isGregoryPatch, double u0, double u1, double v0, double v1,
                           v3 q[16], v3 *d, v3 pmin[4], v3 pmax[4])
{
    v3 p[16];
    memcpy(p, g, 16 * sizeof(v3));
    *d = v3make(0, 0, 0);
    if (isGregoryPatch) {
        /* the two extreme weights of each h over D sit at opposite corners of D */
        double hA[4], hB[4];
        hA[0] = gregory_h(0, u0, v1); hB[0] = gregory_h(0, u1, v0);  /* h_11 increasing in u, decreasing in v */
        hA[1] = gregory_h(1, u0, v0); hB[1] = gregory_h(1, u1, v1);  /* h_21 decreasing in u and in v */
        hA[2] = gregory_h(2, u1, v1); hB[2] = gregory_h(2, u0, v0);  /* h_12 increasing in u and in v */
        hA[3] = gregory_h(3, u1, v0); hB[3] = gregory_h(3, u0, v1);  /* h_22 decreasing in u, increasing in v */
        v3 lo[4], hi[4];
        for (int k = 0; k < 4; ++k) {
            v3 pu = g[INNER_SLOT[k]], pv = g[16 + k];
            v3 a = add(pv, scl(sub(pu, pv), hA[k]));
            v3 b = add(pv, scl(sub(pu, pv), hB[k]));
            lo[k] = vmin(a, b);
            hi[k] = vmax(a, b);
            if (pmin) pmin[k] = lo[k];
            if (pmax) pmax[k] = hi[k];
        }
        /* maxima of B_1^3 and B_2^3 over [t0, t1] (reading A2) */
        double w[2][2];   /* [axis][1 or 2] */
        const double t0s[2] = {u0, v0}, t1s[2] = {u1, v1};
        for (int a = 0; a < 2; ++a) {
            double t0 = t0s[a], t1 = t1s[a];
            double w1 = (t0 <= 1.0 / 3.0 && t1 >= 1.0 / 3.0) ? 1.0 / 3.0 : (t1 <= 1.0 / 3.0 ? t1 : t0);
            double w2 = (t0 <= 2.0 / 3.0 && t1 >= 2.0 / 3.0) ? 2.0 / 3.0 : (t1 < 2.0 / 3.0 ? t1 : t0);
            w[a][0] = 3.0 * w1 * (1.0 - w1) * (1.0 - w1);
            w[a][1] = 3.0 * w2 * w2 * (1.0 - w2);
        }
        for (int k = 0; k < 4; ++k) p[INNER_SLOT[k]] = lo[k];
        /* inner point k = (i, j) with i = 1 + (k & 1), j = 1 + (k >> 1) */
        v3 dd = v3make(0, 0, 0);
        for (int k = 0; k < 4; ++k) {
            double wk = w[0][k & 1] * w[1][k >> 1];
            dd = add(dd, scl(vabs(sub(hi[k], lo[k])), wk));
        }
        *d = dd;
    }
    cropBezierPatch(p, u0, u1, v0, v1, q);
}

/* ------------------------------------------------------------------------------------------------
 * Ray / box slab test (Sec. 3.4 asks for a careful test; in FP64 the plain one is exact enough).
 * Returns 1 and the interval [t0, t1] of the ray inside the box, intersected with [a, b].
 * ---------------------------------------------------------------------------------------------- */
typedef struct { v3 o, d; double tmin, tmax; } ray_t;

static int slab(const ray_t *r, v3 lo, v3 hi, double a, double b, double *t0, double *t1)
{
    for (int k = 0; k < 3; ++k) {
        double o = comp(r->o, k), d = comp(r->d, k), l = comp(lo, k), h = comp(hi, k);
        if (d == 0.0) {
            if (o < l || o > h) return 0;
            continue;
        }
        double ta = (l - o) / d, tb = (h - o) / d;
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > a) a = ta;
        if (tb < b) b = tb;
    }
    *t0 = a;
    *t1 = b;
    return a <= b;
}

/* ------------------------------------------------------------------------------------------------
 * Per (ray, patch) traversal of the sub-domain tree.
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
    v3 g[20];         /* patch control points (Gregory: 20, Bezier: first 16) */
    int greg;
    uint32_t id;
    v3 lo, hi;        /* root box: AABB of the 16 (Bezier) or 20 (Gregory) points */
    int local;        /* boxes below the root are taken in the patch's own frame (Sec. 3.4) */
    v3 R[3];          /* rows of that frame */
    v3 gl[20];        /* the control points in it: R p */
} patch_t;

static double dot3(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross3(v3 a, v3 b) { return v3make(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }

/* Local frame of a patch (Sec. 3.4 intersects patches in local frames to shrink the boxes' overlap):
 * z along the normal of the corner quad (the cross product of its diagonals p33 - p00 and p03 - p30),
 * x along its u edge p30 - p00 made orthogonal to z, y = z x x.  The world frame where that is
 * degenerate.  Rows of R; a point p has local coordinates R p. */
static void local_frame(const v3 g[20], v3 R[3])
{
    R[0] = v3make(1, 0, 0);
    R[1] = v3make(0, 1, 0);
    R[2] = v3make(0, 0, 1);
    v3 z = cross3(sub(g[15], g[0]), sub(g[12], g[3]));
    const double nz = sqrt(dot3(z, z));
    if (!(nz > 0.0)) return;
    z = scl(z, 1.0 / nz);
    const v3 e = sub(g[3], g[0]);
    v3 x = sub(e, scl(z, dot3(e, z)));
    const double nx = sqrt(dot3(x, x));
    if (!(nx > 0.0)) return;
    x = scl(x, 1.0 / nx);
    R[0] = x;
    R[1] = cross3(z, x);
    R[2] = z;
}

static v3 rotate(const v3 R[3], v3 p) { return v3make(dot3(R[0], p), dot3(R[1], p), dot3(R[2], p)); }

static void patch_set_frame(patch_t *P, int local)
{
    P->local = local;
    if (local) local_frame(P->g, P->R);
    else { P->R[0] = v3make(1, 0, 0); P->R[1] = v3make(0, 1, 0); P->R[2] = v3make(0, 0, 1); }
    for (int k = 0; k < 20; ++k) P->gl[k] = local ? rotate(P->R, P->g[k]) : P->g[k];
}

/* the ray in the frame of the patch's boxes below the root */
static ray_t local_ray(const patch_t *P, const ray_t *r)
{
    ray_t l = *r;
    if (P->local) { l.o = rotate(P->R, r->o); l.d = rotate(P->R, r->d); }
    return l;
}

/* Box extension of Sec. 3.4 (closing the gaps that the transform into a local frame may open): below the
 * root, a box thinner than tau along an axis of the patch frame is widened symmetrically to tau.  tau
 * exceeds twice the FP32 error of the ray's transform: 2^-19 (1 + L1 distance of the origin from the
 * patch's box centre).  0 without local frames. */
static double box_tau(const patch_t *P, const ray_t *r)
{
    if (!P->local) return 0.0;
    const v3 c = scl(add(P->lo, P->hi), 0.5);
    const v3 oc = vabs(sub(r->o, c));
    return ldexp(1.0, -19) * (1.0 + oc.x + oc.y + oc.z);
}

static void extend_box(v3 *lo, v3 *hi, double tau)
{
    double l[3] = {lo->x, lo->y, lo->z}, h[3] = {hi->x, hi->y, hi->z};
    for (int k = 0; k < 3; ++k) {
        const double w = h[k] - l[k];
        if (w < tau) { const double e = 0.5 * (tau - w); l[k] -= e; h[k] += e; }
    }
    *lo = v3make(l[0], l[1], l[2]);
    *hi = v3make(h[0], h[1], h[2]);
}

typedef struct {
    double t;
    uint32_t pid;
    uint64_t cell;
    int hit;
    int level;        /* tree level of the recorded leaf (2L unless a screen-space leaf) */
} best_t;

typedef struct {
    uint64_t bvh_nodes, expand_bez, expand_greg, leaves, pops;
} stats_t;

typedef struct {
    v3 q[16];         /* Bezier: node control points */
    int level;
    uint64_t pu, pv;  /* lower domain corner, scale 2^52 */
    double t0, t1;    /* effective ray interval */
    double diag;      /* L1 length of the node box's diagonal */
} node_t;

/* Screen-space termination (Sec. 3.3): partitioning stops at a node whose box diagonal, seen from the ray
 * at the node's entry distance, spans less than half a pixel.  A ray of a pinhole camera covers `spread`
 * radians per pixel, so the test is L1(diagonal) < spread / 2 * t_entry.  Only nodes made by a split are
 * tested (the patch root never is); spread = 0 keeps the fixed depth 2L. */
static int screen_leaf(double spread, int level, double diag, double t_entry)
{
    return spread > 0.0 && level > 0 && diag < 0.5 * spread * t_entry;
}

static double box_diag_l1(v3 lo, v3 hi) { return (hi.x - lo.x) + (hi.y - lo.y) + (hi.z - lo.z); }

static int key_less(double t, uint32_t pid, uint64_t cell, const best_t *b)
{
    if (t != b->t) return t < b->t;
    if (pid != b->pid) return pid < b->pid;
    return cell < b->cell;
}

static void node_domain(int level, uint64_t pu, uint64_t pv, double *u0, double *u1, double *v0, double *v1)
{
    int su = (level + 1) / 2, sv = level / 2;
    uint64_t szu = 1ull << (ORC_SCALE_BITS - su), szv = 1ull << (ORC_SCALE_BITS - sv);
    const double S = ldexp(1.0, ORC_SCALE_BITS);
    *u0 = (double)pu / S;
    *u1 = (double)(pu + szu) / S;
    *v0 = (double)pv / S;
    *v1 = (double)(pv + szv) / S;
}

static uint64_t leaf_cell(uint64_t pu, uint64_t pv, int L)
{
    uint64_t cu = pu >> (ORC_SCALE_BITS - L), cv = pv >> (ORC_SCALE_BITS - L);
    return (cv << L) | cu;
}

/* mode 0: closest hit (best updated as leaves are found).
 * mode 1: enumerate, with loose and strict intervals (see enumerate_patch), every leaf that is alive
 *         under the loose boxes and enters before a fixed bound, calling back for each. */
typedef void (*leaf_cb)(void *ctx, uint32_t pid, uint64_t cell, double t_loose, int strict, double t_strict);

static void enumerate_patch(const patch_t *P, const ray_t *r, int L, double spread, double bound, double eps,
                            leaf_cb cb, void *ctx);

static void intersect_patch(const patch_t *P, const ray_t *r, int L, double spread, best_t *best, stats_t *st,
                            int mode, double bound, leaf_cb cb, void *ctx, double eps)
{
    if (mode == 1) {
        enumerate_patch(P, r, L, spread, bound, eps, cb, ctx);
        return;
    }
    node_t stack[2 * ORC_MAX_L + 4];
    int sp = 0;
    double lim = mode == 0 ? best->t : bound;
    double t0, t1;
    if (!slab(r, P->lo, P->hi, r->tmin, r->tmax, &t0, &t1)) return;   /* the root box is the world one */
    if (t0 > lim) return;
    const ray_t rl = local_ray(P, r);
    const double tau = box_tau(P, r);
    node_t *root = &stack[sp++];
    memcpy(root->q, P->gl, sizeof(root->q));
    root->level = 0;
    root->pu = root->pv = 0;
    root->t0 = t0;
    root->t1 = t1;
    root->diag = box_diag_l1(P->lo, P->hi);
    while (sp > 0) {
        node_t N = stack[--sp];
        if (st) st->pops++;
        lim = mode == 0 ? best->t : bound;
        if (N.t0 > lim) continue;
        if (N.level == 2 * L || screen_leaf(spread, N.level, N.diag, N.t0)) {
            uint64_t cell = leaf_cell(N.pu, N.pv, L);   /* lowest leaf cell of the node */
            if (st) st->leaves++;
            if (mode == 0) {
                if (key_less(N.t0, P->id, cell, best)) {
                    best->t = N.t0;
                    best->pid = P->id;
                    best->cell = cell;
                    best->hit = 1;
                    best->level = N.level;
                }
            }
            continue;
        }
        int axis = N.level & 1;
        v3 q[16], d;
        if (P->greg) {
            double u0, u1, v0, v1;
            node_domain(N.level, N.pu, N.pv, &u0, &u1, &v0, &v1);
            calcPointsAndD(P->gl, 1, u0, u1, v0, v1, q, &d, NULL, NULL);
            if (st) st->expand_greg++;
        } else {
            memcpy(q, N.q, sizeof(q));
            d = v3make(0, 0, 0);
            if (st) st->expand_bez++;
        }
        v3 H[2][16];
        subdivideDeCasteljau(q, axis, H[0], H[1]);
        double c0[2], c1[2], diag[2];
        int hit[2];
        for (int s = 0; s < 2; ++s) {
            v3 lo = H[s][0], hi = H[s][0];
            for (int k = 1; k < 16; ++k) { lo = vmin(lo, H[s][k]); hi = vmax(hi, H[s][k]); }
            hi = add(hi, d);
            extend_box(&lo, &hi, tau);
            diag[s] = box_diag_l1(lo, hi);
            hit[s] = slab(&rl, lo, hi, N.t0, N.t1, &c0[s], &c1[s]) && c0[s] <= lim;
        }
        int su = (N.level + 1) / 2, sv = N.level / 2;   /* splits already taken along u, v */
        uint64_t half = axis == 0 ? (1ull << (ORC_SCALE_BITS - su - 1)) : (1ull << (ORC_SCALE_BITS - sv - 1));
        int first = (hit[0] && hit[1]) ? (c0[1] < c0[0] ? 1 : 0) : (hit[0] ? 0 : 1);
        for (int pass = 0; pass < 2; ++pass) {
            int s = pass == 0 ? 1 - first : first;     /* push the farther child first */
            if (!hit[s]) continue;
            node_t *C = &stack[sp++];
            memcpy(C->q, H[s], sizeof(C->q));
            C->level = N.level + 1;
            C->pu = N.pu + (axis == 0 && s == 1 ? half : 0);
            C->pv = N.pv + (axis == 1 && s == 1 ? half : 0);
            C->t0 = c0[s];
            C->t1 = c1[s];
            C->diag = diag[s];
        }
    }
}


/* ------------------------------------------------------------------------------------------------
 * FP32 error model for the parity flags.  The CUDA path computes the same boxes in FP32; its boxes
 * lie within `eps` (absolute, coordinates) of these and its far distances are scaled up by at most
 * 1 + 1e-6.  A leaf is "loose-alive" if the ray meets every box of its chain inflated by eps (with
 * far distances scaled up), and "strict-alive" if it meets every box deflated by eps (a box thinner
 * than 2 eps along an axis collapses to its mid-plane there).  Every strict-alive leaf is alive for
 * the FP32 path and every leaf alive for the FP32 path is loose-alive, so the FP32 answer is one of
 * the loose-alive leaves entering no later than the nearest strict-alive one.
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
    v3 q[16];
    int level;
    uint64_t pu, pv;
    double l0, l1;    /* loose interval */
    double s0, s1;    /* strict interval (valid if strict) */
    int strict;
    double diag;      /* L1 diagonal of the exact box */
} enode_t;

/* relative slack of the screen-space test under FP32 (the product and the comparison round; the
 * entry distance and the box extents carry the box error model's eps and far scale) */
static const double ORC_SS_MARGIN = 1e-5;

static void grow_box(v3 *lo, v3 *hi, double eps, int deflate)
{
    if (!deflate) {
        *lo = sub(*lo, v3make(eps, eps, eps));
        *hi = add(*hi, v3make(eps, eps, eps));
        return;
    }
    double l[3] = {lo->x, lo->y, lo->z}, h[3] = {hi->x, hi->y, hi->z};
    for (int k = 0; k < 3; ++k) {
        if (h[k] - l[k] > 2.0 * eps) { l[k] += eps; h[k] -= eps; }
        else { double m = 0.5 * (l[k] + h[k]); l[k] = h[k] = m; }
    }
    *lo = v3make(l[0], l[1], l[2]);
    *hi = v3make(h[0], h[1], h[2]);
}

static const double ORC_FAR_SCALE = 1.0 + 1e-6;

static void enumerate_patch(const patch_t *P, const ray_t *r, int L, double spread, double bound, double eps,
                            leaf_cb cb, void *ctx)
{
    enode_t stack[2 * ORC_MAX_L + 4];
    int sp = 0;
    v3 lo = P->lo, hi = P->hi;
    double a, b;
    grow_box(&lo, &hi, eps, 0);
    if (!slab(r, lo, hi, r->tmin, r->tmax, &a, &b)) return;
    b *= ORC_FAR_SCALE;
    if (a > bound || a > b) return;
    /* below the root the FP32 path compares the boxes with the ray anchored at its entry into the patch box
     * (its origin formed without losing the cancellation, as accurately as in FP64, rotated into the patch
     * frame with local frames and rounded once; the direction in FP32) and measures distances from there: the error of that ray grows with the size of
     * the anchored origin and of the patch, not with the distance from the ray's own origin; 3e-7 per unit
     * of |entry point - box centre| + the box's diagonal bounds it */
    const ray_t rl = local_ray(P, r);
    const v3 cen = scl(add(P->lo, P->hi), 0.5);
    const v3 ec = sub(add(r->o, scl(r->d, a)), cen);
    const v3 dg = sub(P->hi, P->lo);
    const double eps_in = eps + 3e-7 * (sqrt(dot3(ec, ec)) + sqrt(dot3(dg, dg)));
    const double tau = box_tau(P, r);
    enode_t *root = &stack[sp++];
    memcpy(root->q, P->gl, sizeof(root->q));
    root->level = 0;
    root->pu = root->pv = 0;
    root->l0 = a;
    root->l1 = b;
    lo = P->lo;
    hi = P->hi;
    grow_box(&lo, &hi, eps, 1);
    root->strict = slab(r, lo, hi, r->tmin, r->tmax, &root->s0, &root->s1);
    root->diag = box_diag_l1(P->lo, P->hi);
    while (sp > 0) {
        enode_t N = stack[--sp];
        if (N.level == 2 * L) {
            cb(ctx, P->id, leaf_cell(N.pu, N.pv, L), N.l0, N.strict, N.s0);
            continue;
        }
        if (spread > 0.0 && N.level > 0) {
            /* screen-space test under the error model: certainly a leaf, certainly split, or either (then
             * the node is a possible, not a certain, leaf and its subtree stays possible too) */
            const double ta = N.strict ? fmin(N.l0, N.s0) : N.l0, tb = N.strict ? fmax(N.l0, N.s0) : N.l0;
            const double thr_lo = 0.5 * spread * ta * (1.0 - ORC_SS_MARGIN);
            const double thr_hi = 0.5 * spread * tb * (1.0 + ORC_SS_MARGIN);
            const double dlo = fmax(0.0, N.diag - 6.0 * eps_in), dhi = N.diag + 6.0 * eps_in;
            if (dhi < thr_lo) {
                cb(ctx, P->id, leaf_cell(N.pu, N.pv, L), N.l0, N.strict, N.s0);
                continue;
            }
            if (!(dlo >= thr_hi)) cb(ctx, P->id, leaf_cell(N.pu, N.pv, L), N.l0, 0, N.s0);
        }
        int axis = N.level & 1;
        v3 q[16], d;
        if (P->greg) {
            double u0, u1, v0, v1;
            node_domain(N.level, N.pu, N.pv, &u0, &u1, &v0, &v1);
            calcPointsAndD(P->gl, 1, u0, u1, v0, v1, q, &d, NULL, NULL);
        } else {
            memcpy(q, N.q, sizeof(q));
            d = v3make(0, 0, 0);
        }
        v3 H[2][16];
        subdivideDeCasteljau(q, axis, H[0], H[1]);
        int su = (N.level + 1) / 2, sv = N.level / 2;
        uint64_t half = axis == 0 ? (1ull << (ORC_SCALE_BITS - su - 1)) : (1ull << (ORC_SCALE_BITS - sv - 1));
        for (int s = 0; s < 2; ++s) {
            v3 blo = H[s][0], bhi = H[s][0];
            for (int k = 1; k < 16; ++k) { blo = vmin(blo, H[s][k]); bhi = vmax(bhi, H[s][k]); }
            bhi = add(bhi, d);
            extend_box(&blo, &bhi, tau);
            v3 llo = blo, lhi = bhi;
            grow_box(&llo, &lhi, eps_in, 0);
            double c0, c1;
            if (!slab(&rl, llo, lhi, -INFINITY, INFINITY, &c0, &c1)) continue;
            c1 *= ORC_FAR_SCALE;
            c0 = fmax(c0, N.l0);
            c1 = fmin(c1, N.l1);
            if (c0 > c1 || c0 > bound) continue;
            enode_t *C = &stack[sp++];
            memcpy(C->q, H[s], sizeof(C->q));
            C->level = N.level + 1;
            C->pu = N.pu + (axis == 0 && s == 1 ? half : 0);
            C->pv = N.pv + (axis == 1 && s == 1 ? half : 0);
            C->l0 = c0;
            C->l1 = c1;
            C->diag = box_diag_l1(blo, bhi);
            C->strict = 0;
            if (N.strict) {
                v3 slo = blo, shi = bhi;
                grow_box(&slo, &shi, eps_in, 1);
                C->strict = slab(&rl, slo, shi, N.s0, N.s1, &C->s0, &C->s1);
            }
        }
    }
}

/* ------------------------------------------------------------------------------------------------
 * Brute force definition for tiny inputs: every leaf whose whole ancestor chain has a non-empty
 * interval is a candidate; the answer is the smallest key.  No pruning, no ordering.
 * ---------------------------------------------------------------------------------------------- */
static void brute_rec(const patch_t *P, const ray_t *r, int L, double spread, const v3 q_in[16], int level,
                      uint64_t pu, uint64_t pv, double t0, double t1, double diag, best_t *best)
{
    if (level == 2 * L || screen_leaf(spread, level, diag, t0)) {
        uint64_t cell = leaf_cell(pu, pv, L);
        if (t0 <= r->tmax && key_less(t0, P->id, cell, best)) {
            best->t = t0; best->pid = P->id; best->cell = cell; best->hit = 1; best->level = level;
        }
        return;
    }
    int axis = level & 1;
    v3 q[16], d;
    const ray_t rl = local_ray(P, r);
    const double tau = box_tau(P, r);
    if (P->greg) {
        double u0, u1, v0, v1;
        node_domain(level, pu, pv, &u0, &u1, &v0, &v1);
        calcPointsAndD(P->gl, 1, u0, u1, v0, v1, q, &d, NULL, NULL);
    } else {
        memcpy(q, q_in, sizeof(q));
        d = v3make(0, 0, 0);
    }
    v3 H[2][16];
    subdivideDeCasteljau(q, axis, H[0], H[1]);
    int su = (level + 1) / 2, sv = level / 2;
    uint64_t half = axis == 0 ? (1ull << (ORC_SCALE_BITS - su - 1)) : (1ull << (ORC_SCALE_BITS - sv - 1));
    for (int s = 0; s < 2; ++s) {
        v3 lo = H[s][0], hi = H[s][0];
        for (int k = 1; k < 16; ++k) { lo = vmin(lo, H[s][k]); hi = vmax(hi, H[s][k]); }
        hi = add(hi, d);
        extend_box(&lo, &hi, tau);
        double a, b;
        if (!slab(&rl, lo, hi, t0, t1, &a, &b)) continue;
        brute_rec(P, r, L, spread, H[s], level + 1, pu + (axis == 0 && s ? half : 0),
                  pv + (axis == 1 && s ? half : 0), a, b, box_diag_l1(lo, hi), best);
    }
}

/* ------------------------------------------------------------------------------------------------
 * Scene: patches + a simple median-split BVH of its own (Sec. 4 uses a binned-SAH BVH; any
 * conservative hierarchy gives the same answer because patch boxes are nested in node boxes).
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
    v3 lo, hi;
    int left, right;     /* children, or -1 */
    int first, count;    /* leaf range into order[] */
} bnode_t;

typedef struct {
    patch_t *P;
    uint32_t n;
    bnode_t *nodes;
    int nnodes;
    uint32_t *order;
} scene_t;

static int g_sort_axis;
static const patch_t *g_sort_P;
static int cmp_centroid(const void *a, const void *b)
{
    const patch_t *pa = &g_sort_P[*(const uint32_t *)a], *pb = &g_sort_P[*(const uint32_t *)b];
    double ca = comp(pa->lo, g_sort_axis) + comp(pa->hi, g_sort_axis);
    double cb = comp(pb->lo, g_sort_axis) + comp(pb->hi, g_sort_axis);
    return ca < cb ? -1 : (ca > cb ? 1 : 0);
}

static int bvh_build_rec(scene_t *S, int first, int count)
{
    int idx = S->nnodes++;
    bnode_t *nd = &S->nodes[idx];
    v3 lo = S->P[S->order[first]].lo, hi = S->P[S->order[first]].hi;
    for (int i = 1; i < count; ++i) {
        lo = vmin(lo, S->P[S->order[first + i]].lo);
        hi = vmax(hi, S->P[S->order[first + i]].hi);
    }
    nd->lo = lo; nd->hi = hi; nd->first = first; nd->count = count; nd->left = nd->right = -1;
    if (count <= 2) return idx;
    v3 ext = sub(hi, lo);
    g_sort_axis = ext.x >= ext.y && ext.x >= ext.z ? 0 : (ext.y >= ext.z ? 1 : 2);
    g_sort_P = S->P;
    qsort(S->order + first, count, sizeof(uint32_t), cmp_centroid);
    int h = count / 2;
    int l = bvh_build_rec(S, first, h);
    int r = bvh_build_rec(S, first + h, count - h);
    S->nodes[idx].left = l;
    S->nodes[idx].right = r;
    return idx;
}

static void scene_init(scene_t *S, const float *x, const float *y, const float *z, const uint8_t *types, uint32_t n,
                       int local)
{
    S->n = n;
    S->P = (patch_t *)malloc(sizeof(patch_t) * (n ? n : 1));
    for (uint32_t i = 0; i < n; ++i) {
        patch_t *P = &S->P[i];
        P->greg = types[i] != 0;
        P->id = i;
        for (int k = 0; k < 20; ++k)
            P->g[k] = v3make((double)x[20 * i + k], (double)y[20 * i + k], (double)z[20 * i + k]);
        int np = P->greg ? 20 : 16;
        P->lo = P->hi = P->g[0];
        for (int k = 1; k < np; ++k) { P->lo = vmin(P->lo, P->g[k]); P->hi = vmax(P->hi, P->g[k]); }
        patch_set_frame(P, local);
    }
    S->nodes = (bnode_t *)malloc(sizeof(bnode_t) * (2 * (size_t)n + 2));
    S->order = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint32_t i = 0; i < n; ++i) S->order[i] = i;
    S->nnodes = 0;
    if (n) bvh_build_rec(S, 0, (int)n);
}

static void scene_free(scene_t *S)
{
    free(S->P);
    free(S->nodes);
    free(S->order);
}

/* closest hit over the scene (mode 0), or leaf enumeration below a fixed bound (mode 1) */
static void trace(const scene_t *S, const ray_t *r, int L, double spread, best_t *best, stats_t *st, int mode,
                  double bound, leaf_cb cb, void *ctx, double eps)
{
    if (S->nnodes == 0) return;
    int stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const bnode_t *nd = &S->nodes[stack[--sp]];
        double lim = mode == 0 ? best->t : bound;
        double t0, t1;
        if (st) st->bvh_nodes++;
        v3 lo = nd->lo, hi = nd->hi;
        if (mode == 1) grow_box(&lo, &hi, eps, 0);
        if (!slab(r, lo, hi, r->tmin, r->tmax, &t0, &t1) || t0 > lim) continue;
        if (nd->left < 0) {
            for (int i = 0; i < nd->count; ++i)
                intersect_patch(&S->P[S->order[nd->first + i]], r, L, spread, best, st, mode, bound, cb, ctx, eps);
            continue;
        }
        stack[sp++] = nd->right;
        stack[sp++] = nd->left;
    }
}

static void make_ray(ray_t *r, const float *const planes[8], uint32_t i)
{
    r->o = v3make(planes[0][i], planes[1][i], planes[2][i]);
    r->d = v3make(planes[3][i], planes[4][i], planes[5][i]);
    r->tmin = planes[6][i];
    r->tmax = planes[7][i];
}

/* ------------------------------------------------------------------------------------------------
 * Flags that exclude rays whose answer FP32 cannot be expected to reproduce (FP32 error model of
 * enumerate_patch; t* is the oracle's entry distance, R the nearest strict-alive entry):
 *   bit 0 another patch has a loose-alive leaf entering no later than min(R, t* (1 + rel_t));
 *   bit 1 the hit patch has such a leaf more than one cell away from the hit cell;
 *   bit 2 hit/miss may differ: a miss with a loose-alive leaf, or a hit without any strict-alive leaf;
 *   bit 3 t may leave the tolerance: such a leaf enters before t* (1 - rel_t), or R > t* (1 + rel_t);
 *   bit 4 (flags_mode 2) hit/miss changes when the origin moves by +-perturb along two axes normal to d.
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
    uint32_t pid;
    uint64_t cell;
    double tl, ts;
    int strict;
} leaf_rec;

typedef struct {
    leaf_rec *v;
    size_t n, cap;
} leaf_list;

static void list_cb(void *vctx, uint32_t pid, uint64_t cell, double tl, int strict, double ts)
{
    leaf_list *l = (leaf_list *)vctx;
    if (l->n == l->cap) {
        size_t cap = l->cap ? 2 * l->cap : 64;
        leaf_rec *nv = (leaf_rec *)realloc(l->v, cap * sizeof(leaf_rec));
        if (!nv) return;
        l->v = nv;
        l->cap = cap;
    }
    leaf_rec *e = &l->v[l->n++];
    e->pid = pid; e->cell = cell; e->tl = tl; e->strict = strict; e->ts = ts;
}

static int far_cell(uint64_t a, uint64_t b, int L)
{
    int64_t mask = (1ll << L) - 1;
    int64_t du = (int64_t)(a & mask) - (int64_t)(b & mask);
    int64_t dv = (int64_t)(a >> L) - (int64_t)(b >> L);
    return du < -1 || du > 1 || dv < -1 || dv > 1;
}

static double min_strict(const leaf_list *l)
{
    double R = INFINITY;
    for (size_t i = 0; i < l->n; ++i)
        if (l->v[i].strict && l->v[i].ts < R) R = l->v[i].ts;
    return R;
}

static uint8_t fp32_flags(const scene_t *S, const ray_t *r, int L, double spread, const best_t *b, double rel_t,
                          double eps, double *t2)
{
    leaf_list l = {NULL, 0, 0};
    best_t dummy = {0, 0, 0, 0};
    uint8_t flags = 0;
    *t2 = INFINITY;
    if (!b->hit) {
        trace(S, r, L, spread, &dummy, NULL, 1, r->tmax, list_cb, &l, eps);
        if (l.n) flags |= 4;
        free(l.v);
        return flags;
    }
    const double B = b->t + fabs(b->t) * rel_t;
    trace(S, r, L, spread, &dummy, NULL, 1, B, list_cb, &l, eps);
    double R = min_strict(&l);
    if (R > B) {
        leaf_list all = {NULL, 0, 0};
        trace(S, r, L, spread, &dummy, NULL, 1, r->tmax, list_cb, &all, eps);
        double Ra = min_strict(&all);
        flags |= isinf(Ra) ? 4 : 8;
        free(all.v);
    }
    const double lim = R < B ? R : B;
    for (size_t i = 0; i < l.n; ++i) {
        const leaf_rec *e = &l.v[i];
        if (e->tl > lim) continue;
        if (e->pid != b->pid) {
            flags |= 1;
            if (e->tl < *t2) *t2 = e->tl;
        } else if (far_cell(e->cell, b->cell, L)) {
            flags |= 2;
        }
        if (e->tl < b->t - fabs(b->t) * rel_t) flags |= 8;
    }
    free(l.v);
    return flags;
}

static void ortho_basis(v3 d, v3 *e1, v3 *e2)
{
    v3 a = fabs(d.x) < 0.6 ? v3make(1, 0, 0) : (fabs(d.y) < 0.6 ? v3make(0, 1, 0) : v3make(0, 0, 1));
    /* e1 = normalize(a - (a.d) d), e2 = d x e1 */
    double dd = d.x * d.x + d.y * d.y + d.z * d.z;
    double ad = a.x * d.x + a.y * d.y + a.z * d.z;
    v3 u = sub(a, scl(d, ad / dd));
    double nu = sqrt(u.x * u.x + u.y * u.y + u.z * u.z);
    *e1 = scl(u, 1.0 / nu);
    v3 w = v3make(d.y * e1->z - d.z * e1->y, d.z * e1->x - d.x * e1->z, d.x * e1->y - d.y * e1->x);
    double nw = sqrt(w.x * w.x + w.y * w.y + w.z * w.z);
    *e2 = scl(w, 1.0 / nw);
}

/* ------------------------------------------------------------------------------------------------
 * Threaded driver.
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
    const scene_t *S;
    const float *planes[8];
    uint32_t n_rays;
    int L;
    int flags_mode;
    double rel_t, eps, perturb;
    double *t_out;
    float *u_out, *v_out;
    uint32_t *pid_out;
    uint64_t *cell_out;
    uint8_t *flag_out;
    double *t2_out;
    uint64_t *stats_out;   /* per ray: bvh_nodes, expand_bez, expand_greg, leaves, pops */
    double spread;         /* screen-space termination (0: fixed depth) */
    uint8_t *level_out;    /* per ray: tree level of the recorded leaf */
    uint32_t next;
    pthread_mutex_t mu;
} job_t;

static void run_one(job_t *J, uint32_t i)
{
    ray_t r;
    make_ray(&r, J->planes, i);
    best_t b = {r.tmax, 0xFFFFFFFFu, ~0ull, 0};
    stats_t st = {0, 0, 0, 0, 0};
    int valid = !(isnan(r.o.x) || isnan(r.o.y) || isnan(r.o.z) || isnan(r.d.x) || isnan(r.d.y) || isnan(r.d.z) ||
                  isnan(r.tmin) || isnan(r.tmax) || r.tmin > r.tmax);
    if (valid) trace(J->S, &r, J->L, J->spread, &b, &st, 0, 0.0, NULL, NULL, 0.0);
    double cells = ldexp(1.0, J->L);
    if (b.hit) {
        /* u, v: centre of the leaf's domain (a cell at level 2L, a larger block for a screen-space leaf) */
        const int su = (b.level + 1) / 2, sv = b.level / 2;
        J->t_out[i] = b.t;
        J->u_out[i] = (float)((double)(b.cell & ((1ull << J->L) - 1)) / cells + ldexp(0.5, -su));
        J->v_out[i] = (float)((double)(b.cell >> J->L) / cells + ldexp(0.5, -sv));
        J->pid_out[i] = b.pid;
        J->cell_out[i] = b.cell;
    } else {
        J->t_out[i] = INFINITY;
        J->u_out[i] = 0.0f;
        J->v_out[i] = 0.0f;
        J->pid_out[i] = 0xFFFFFFFFu;
        J->cell_out[i] = ~0ull;
    }
    if (J->level_out) J->level_out[i] = (uint8_t)(b.hit ? b.level : 0);
    if (J->stats_out) {
        uint64_t *s = J->stats_out + 5 * (size_t)i;
        s[0] = st.bvh_nodes; s[1] = st.expand_bez; s[2] = st.expand_greg; s[3] = st.leaves; s[4] = st.pops;
    }
    if (!J->flags_mode || !valid) {
        if (J->flag_out) J->flag_out[i] = 0;
        if (J->t2_out) J->t2_out[i] = INFINITY;
        return;
    }
    double t2 = INFINITY;
    uint8_t flags = fp32_flags(J->S, &r, J->L, J->spread, &b, J->rel_t, J->eps, &t2);
    if (J->flags_mode == 2) {
        v3 e1, e2;
        ortho_basis(r.d, &e1, &e2);
        for (int k = 0; k < 4 && !(flags & 16); ++k) {
            ray_t rp = r;
            v3 off = scl(k < 2 ? e1 : e2, (k & 1) ? -J->perturb : J->perturb);
            rp.o = add(r.o, off);
            best_t bp = {rp.tmax, 0xFFFFFFFFu, ~0ull, 0};
            trace(J->S, &rp, J->L, J->spread, &bp, NULL, 0, 0.0, NULL, NULL, 0.0);
            if (bp.hit != b.hit) flags |= 16;
        }
    }
    J->flag_out[i] = flags;
    if (J->t2_out) J->t2_out[i] = t2;
}

static void *worker(void *arg)
{
    job_t *J = (job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        uint32_t s = J->next;
        J->next = s + 64 > J->n_rays ? J->n_rays : s + 64;
        uint32_t e = J->next;
        pthread_mutex_unlock(&J->mu);
        if (s >= e) break;
        for (uint32_t i = s; i < e; ++i) run_one(J, i);
    }
    return NULL;
}

/* ------------------------------------------------------------------------------------------------
 * Exported entry points (called through ctypes from oracle/__init__.py).
 * ---------------------------------------------------------------------------------------------- */

int orc_num_cores(void) { long n = sysconf(_SC_NPROCESSORS_ONLN); return n > 0 ? (int)n : 1; }

/* Closest hit of every ray.  Inputs: patch planes x,y,z [n*20] (layout of the module header), types
 * [n] (0 Bezier, 1 Gregory), ray planes ox..tmax [n_rays].  Outputs per ray: t (INF on miss), u, v
 * (cell centre), patch id (0xFFFFFFFF on miss), cell index v_cell * 2^L + u_cell; optionally flags
 * (flags_mode 1: FP32 error model with box error eps and t tolerance rel_t; 2: also the origin
 * perturbation test), t2 and 5 traversal counters.  Returns the number of threads used. */
int orc_intersect(const float *x, const float *y, const float *z, const uint8_t *types, uint32_t n_patches,
                  const float *ox, const float *oy, const float *oz, const float *dx, const float *dy,
                  const float *dz, const float *tmin, const float *tmax, uint32_t n_rays, int L, int n_threads,
                  int flags_mode, double rel_t, double eps, double perturb, double *t_out, float *u_out, float *v_out,
                  uint32_t *pid_out, uint64_t *cell_out, uint8_t *flag_out, double *t2_out, uint64_t *stats_out,
                  double spread, uint8_t *level_out, int local)
{
    if (L < 1 || L > ORC_MAX_L) return -1;
    scene_t S;
    scene_init(&S, x, y, z, types, n_patches, local);
    job_t J;
    memset(&J, 0, sizeof(J));
    J.S = &S;
    J.planes[0] = ox; J.planes[1] = oy; J.planes[2] = oz; J.planes[3] = dx; J.planes[4] = dy; J.planes[5] = dz;
    J.planes[6] = tmin; J.planes[7] = tmax;
    J.n_rays = n_rays; J.L = L; J.flags_mode = flags_mode; J.rel_t = rel_t; J.eps = eps; J.perturb = perturb;
    J.t_out = t_out; J.u_out = u_out; J.v_out = v_out; J.pid_out = pid_out; J.cell_out = cell_out;
    J.flag_out = flag_out; J.t2_out = t2_out; J.stats_out = stats_out;
    J.spread = spread; J.level_out = level_out;
    pthread_mutex_init(&J.mu, NULL);
    if (n_threads <= 0) n_threads = orc_num_cores();
    if (n_threads > 256) n_threads = 256;
    if ((uint32_t)n_threads > (n_rays + 63) / 64) n_threads = (int)((n_rays + 63) / 64);
    if (n_threads < 1) n_threads = 1;
    pthread_t th[256];
    for (int i = 1; i < n_threads; ++i) pthread_create(&th[i], NULL, worker, &J);
    worker(&J);
    for (int i = 1; i < n_threads; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&J.mu);
    scene_free(&S);
    return n_threads;
}

static void load_patch(patch_t *P, const double *g60, int greg, int local)
{
    P->greg = greg;
    P->id = 0;
    for (int k = 0; k < 20; ++k) P->g[k] = v3make(g60[3 * k], g60[3 * k + 1], g60[3 * k + 2]);
    int np = greg ? 20 : 16;
    P->lo = P->hi = P->g[0];
    for (int k = 1; k < np; ++k) { P->lo = vmin(P->lo, P->g[k]); P->hi = vmax(P->hi, P->g[k]); }
    patch_set_frame(P, local);
}

static void load_ray(ray_t *r, const double *r8)
{
    r->o = v3make(r8[0], r8[1], r8[2]);
    r->d = v3make(r8[3], r8[4], r8[5]);
    r->tmin = r8[6];
    r->tmax = r8[7];
}

/* Single (ray, patch) query.  g60: 20 points xyz-interleaved; r8: ox oy oz dx dy dz tmin tmax.
 * brute != 0 uses the all-leaves definition.  Returns 1 on hit with *t and *cell. */
int orc_intersect_patch(const double *g60, int greg, const double *r8, int L, int brute, double *t, uint64_t *cell,
                        uint64_t *stats5, double spread, int *level, int local)
{
    if (L < 1 || L > ORC_MAX_L) return -1;
    patch_t P;
    load_patch(&P, g60, greg, local);
    ray_t r;
    load_ray(&r, r8);
    best_t b = {r.tmax, 0xFFFFFFFFu, ~0ull, 0};
    stats_t st = {0, 0, 0, 0, 0};
    if (brute) {
        double t0, t1;
        if (slab(&r, P.lo, P.hi, r.tmin, r.tmax, &t0, &t1))
            brute_rec(&P, &r, L, spread, P.gl, 0, 0, 0, t0, t1, box_diag_l1(P.lo, P.hi), &b);
    } else {
        intersect_patch(&P, &r, L, spread, &b, &st, 0, 0.0, NULL, NULL, 0.0);
    }
    if (level) *level = b.hit ? b.level : -1;
    if (stats5) { stats5[0] = st.bvh_nodes; stats5[1] = st.expand_bez; stats5[2] = st.expand_greg; stats5[3] = st.leaves; stats5[4] = st.pops; }
    *t = b.hit ? b.t : INFINITY;
    *cell = b.hit ? b.cell : ~0ull;
    return b.hit;
}

static void load16(v3 p[16], const double *p48) { for (int k = 0; k < 16; ++k) p[k] = v3make(p48[3 * k], p48[3 * k + 1], p48[3 * k + 2]); }
static void store16(double *p48, const v3 p[16]) { for (int k = 0; k < 16; ++k) { p48[3 * k] = p[k].x; p48[3 * k + 1] = p[k].y; p48[3 * k + 2] = p[k].z; } }

/* f, f_u, f_v, f_uv of a Bezier patch (16 points xyz-interleaved) at (u, v): out12 */
void orc_bezier_eval(const double *p48, double u, double v, double *out12)
{
    v3 p[16];
    load16(p, p48);
    v3 r[4] = {evalBezier(p, u, v), evalBezierDu(p, u, v), evalBezierDv(p, u, v), evalBezierDuDv(p, u, v)};
    for (int k = 0; k < 4; ++k) { out12[3 * k] = r[k].x; out12[3 * k + 1] = r[k].y; out12[3 * k + 2] = r[k].z; }
}

void orc_crop(const double *p48, double u0, double u1, double v0, double v1, double *q48)
{
    v3 p[16], q[16];
    load16(p, p48);
    cropBezierPatch(p, u0, u1, v0, v1, q);
    store16(q48, q);
}

void orc_split(const double *p48, int axis, double *l48, double *r48)
{
    v3 p[16], L[16], R[16];
    load16(p, p48);
    subdivideDeCasteljau(p, axis, L, R);
    store16(l48, L);
    store16(r48, R);
}

/* Gregory surface point and the reduced inner points p_ij(u,v) (4 x xyz) */
void orc_gregory_eval(const double *g60, double u, double v, double *out3, double *inner12)
{
    v3 g[20], p[16];
    for (int k = 0; k < 20; ++k) g[k] = v3make(g60[3 * k], g60[3 * k + 1], g60[3 * k + 2]);
    gregory_reduce(g, u, v, p);
    v3 f = evalBezier(p, u, v);
    out3[0] = f.x; out3[1] = f.y; out3[2] = f.z;
    if (inner12)
        for (int k = 0; k < 4; ++k) { v3 a = p[INNER_SLOT[k]]; inner12[3 * k] = a.x; inner12[3 * k + 1] = a.y; inner12[3 * k + 2] = a.z; }
}

/* Surface point and partial derivatives of the (Gregory-reduced) patch at (u, v): out9 = f, f_u, f_v.
 * For a Gregory patch the derivatives are those of the Bezier patch it reduces to at (u, v). */
void orc_patch_frame(const double *g60, int greg, double u, double v, double *out9)
{
    v3 g[20], p[16];
    for (int k = 0; k < 20; ++k) g[k] = v3make(g60[3 * k], g60[3 * k + 1], g60[3 * k + 2]);
    if (greg) gregory_reduce(g, u, v, p); else memcpy(p, g, sizeof(p));
    v3 f = evalBezier(p, u, v), fu = evalBezierDu(p, u, v), fv = evalBezierDv(p, u, v);
    out9[0] = f.x; out9[1] = f.y; out9[2] = f.z;
    out9[3] = fu.x; out9[4] = fu.y; out9[5] = fu.z;
    out9[6] = fv.x; out9[7] = fv.y; out9[8] = fv.z;
}

/* Algorithm 2: q48 (lower patch cropped to D), d3, and the inner-point bounds pmin12 / pmax12 */
void orc_calc_points_and_d(const double *g60, int greg, double u0, double u1, double v0, double v1, double *q48,
                           double *d3, double *pmin12, double *pmax12)
{
    v3 g[20], q[16], d, lo[4], hi[4];
    for (int k = 0; k < 20; ++k) g[k] = v3make(g60[3 * k], g60[3 * k + 1], g60[3 * k + 2]);
    calcPointsAndD(g, greg, u0, u1, v0, v1, q, &d, lo, hi);
    store16(q48, q);
    d3[0] = d.x; d3[1] = d.y; d3[2] = d.z;
    if (greg) {
        for (int k = 0; k < 4; ++k) {
            pmin12[3 * k] = lo[k].x; pmin12[3 * k + 1] = lo[k].y; pmin12[3 * k + 2] = lo[k].z;
            pmax12[3 * k] = hi[k].x; pmax12[3 * k + 1] = hi[k].y; pmax12[3 * k + 2] = hi[k].z;
        }
    }
}

/* Child boxes of the node (level, pu, pv) as the traversal computes them: lo/hi of both halves
 * (xyz), the Bezier node points being the de Casteljau descent from the root.  box12 = loL hiL loR hiR. */
void orc_child_boxes(const double *g60, int greg, int level, uint64_t pu, uint64_t pv, double *box12)
{
    v3 g[20], q[16], d;
    for (int k = 0; k < 20; ++k) g[k] = v3make(g60[3 * k], g60[3 * k + 1], g60[3 * k + 2]);
    if (greg) {
        double u0, u1, v0, v1;
        node_domain(level, pu, pv, &u0, &u1, &v0, &v1);
        calcPointsAndD(g, 1, u0, u1, v0, v1, q, &d, NULL, NULL);
    } else {
        memcpy(q, g, sizeof(q));
        d = v3make(0, 0, 0);
        for (int l = 0; l < level; ++l) {
            int su = (l + 1) / 2, sv = l / 2, axis = l & 1;
            uint64_t bit = axis == 0 ? (1ull << (ORC_SCALE_BITS - su - 1)) : (1ull << (ORC_SCALE_BITS - sv - 1));
            int right = axis == 0 ? (pu & bit) != 0 : (pv & bit) != 0;
            v3 Lh[16], Rh[16];
            subdivideDeCasteljau(q, axis, Lh, Rh);
            memcpy(q, right ? Rh : Lh, sizeof(q));
        }
    }
    v3 H[2][16];
    subdivideDeCasteljau(q, level & 1, H[0], H[1]);
    for (int s = 0; s < 2; ++s) {
        v3 lo = H[s][0], hi = H[s][0];
        for (int k = 1; k < 16; ++k) { lo = vmin(lo, H[s][k]); hi = vmax(hi, H[s][k]); }
        hi = add(hi, d);
        box12[6 * s + 0] = lo.x; box12[6 * s + 1] = lo.y; box12[6 * s + 2] = lo.z;
        box12[6 * s + 3] = hi.x; box12[6 * s + 4] = hi.y; box12[6 * s + 5] = hi.z;
    }
}

/* Rows of the local frame of a patch (Sec. 3.4), for tests. */
void orc_local_frame(const double *g60, double *out9)
{
    v3 g[20], R[3];
    for (int k = 0; k < 20; ++k) g[k] = v3make(g60[3 * k], g60[3 * k + 1], g60[3 * k + 2]);
    local_frame(g, R);
    for (int i = 0; i < 3; ++i) { out9[3 * i] = R[i].x; out9[3 * i + 1] = R[i].y; out9[3 * i + 2] = R[i].z; }
}
