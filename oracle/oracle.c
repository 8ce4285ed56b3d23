/*
 * FP64 CPU oracle of the batched rigid-body step -- TEST INFRASTRUCTURE ONLY.
 * See oracle.h for the interface and the published methods each stage follows.
 *
 * Everything here is plain, sequential FP64: one env at a time, stages in the
 * order broadphase -> narrowphase -> colouring once per step, then for every
 * substep gravity -> prep -> warm start -> position iterations -> integration
 * -> relax (velocity) iterations.  Rows of one colour touch disjoint dynamic
 * bodies, so solving them in constraint-list order equals solving them in
 * parallel; that is what lets a parallel GPU solver agree with this file.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* small vector algebra                                                       */
/* ------------------------------------------------------------------------- */
typedef struct { double x, y, z; } v3;
typedef struct { double x, y, z, w; } qt;          /* Hamilton, (x,y,z,w) */
typedef struct { double m[3][3]; } m3;

static v3 V(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return V(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return V(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return V(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
    return V(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double norm(v3 a) { return sqrt(dot(a, a)); }
static v3 neg(v3 a) { return V(-a.x, -a.y, -a.z); }
static double comp(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
static v3 unit_axis(int i) { return V(i == 0, i == 1, i == 2); }
static v3 with_comp(v3 a, int i, double s) {
    if (i == 0) a.x = s; else if (i == 1) a.y = s; else a.z = s;
    return a;
}
static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
/* float32 rounding, for the storage probe (oracle_set_round32) */
static double r32(double x) { return (double)(float)x; }
static v3 r32v(v3 a) { return V(r32(a.x), r32(a.y), r32(a.z)); }

static qt Q(double x, double y, double z, double w) { qt r = {x, y, z, w}; return r; }
static qt qmul(qt a, qt b) {
    /* (a_v, a_w)(b_v, b_w) = (a_w b_v + b_w a_v + a_v x b_v, a_w b_w - a_v.b_v) */
    v3 av = V(a.x, a.y, a.z), bv = V(b.x, b.y, b.z);
    v3 r = add(add(scl(bv, a.w), scl(av, b.w)), cross(av, bv));
    return Q(r.x, r.y, r.z, a.w * b.w - dot(av, bv));
}
static qt qconj(qt a) { return Q(-a.x, -a.y, -a.z, a.w); }
static qt qnormalize(qt a) {
    double n = sqrt(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w);
    return Q(a.x / n, a.y / n, a.z / n, a.w / n);
}
static m3 qmat(qt q) {
    m3 R;
    double x = q.x, y = q.y, z = q.z, w = q.w;
    R.m[0][0] = 1 - 2 * (y * y + z * z); R.m[0][1] = 2 * (x * y - z * w); R.m[0][2] = 2 * (x * z + y * w);
    R.m[1][0] = 2 * (x * y + z * w); R.m[1][1] = 1 - 2 * (x * x + z * z); R.m[1][2] = 2 * (y * z - x * w);
    R.m[2][0] = 2 * (x * z - y * w); R.m[2][1] = 2 * (y * z + x * w); R.m[2][2] = 1 - 2 * (x * x + y * y);
    return R;
}
static v3 mv(const m3* R, v3 a) {
    return V(R->m[0][0] * a.x + R->m[0][1] * a.y + R->m[0][2] * a.z,
             R->m[1][0] * a.x + R->m[1][1] * a.y + R->m[1][2] * a.z,
             R->m[2][0] * a.x + R->m[2][1] * a.y + R->m[2][2] * a.z);
}
static v3 mtv(const m3* R, v3 a) { /* R^T a */
    return V(R->m[0][0] * a.x + R->m[1][0] * a.y + R->m[2][0] * a.z,
             R->m[0][1] * a.x + R->m[1][1] * a.y + R->m[2][1] * a.z,
             R->m[0][2] * a.x + R->m[1][2] * a.y + R->m[2][2] * a.z);
}
static v3 mcol(const m3* R, int j) { return V(R->m[0][j], R->m[1][j], R->m[2][j]); }
static v3 qrot(qt q, v3 a) { m3 R = qmat(q); return mv(&R, a); }

/* Axis used to build a basis orthogonal to a unit vector n: the first index
 * i (0, 1, 2) whose |n_i| is within 0.1 of the smallest |n_j|.  Near an axis
 * direction this never flips between nearly equal tiny components, and for a
 * normal in a coordinate plane it picks the axis normal to that plane. */
static int basis_axis(v3 a) {
    double c[3] = {fabs(a.x), fabs(a.y), fabs(a.z)};
    double mn = fmin(c[0], fmin(c[1], c[2]));
    for (int i = 0; i < 3; i++) if (c[i] <= mn + 0.1) return i;
    return 2;
}

/* ------------------------------------------------------------------------- */
/* world data                                                                 */
/* ------------------------------------------------------------------------- */
/* convex hull asset (body frame = its principal frame): vertices, outward
 * counter-clockwise triangles, and what the narrowphase derives from them */
enum { H_MAXV = 16, H_MAXT = 2 * H_MAXV - 4, H_MAXE = 3 * H_MAXV - 6 };
typedef struct {
    int nv, nt, ne;
    v3 v[H_MAXV];
    int t[H_MAXT][3];
    int e[H_MAXE][2], ef[H_MAXE][2];  /* edge vertices, its two triangles */
    double rad;                       /* bounding radius about the origin */
    double vol; v3 c2;                /* volume; diagonal second moments of unit density */
} Hull;

typedef struct {
    int type; double p[3]; double mass; int dyn;
    const Hull* hull;                 /* hull bodies */
    double inv_mass; double inv_I[3]; double mu, rest; unsigned group, mask;
    v3 x; qt q; v3 v; v3 w;
    qt q0;                            /* orientation at the start of the step */
    m3 invIw;                         /* world inverse inertia, per substep */
} Body;

typedef struct {
    int type, parent, child;
    v3 fpP; qt fqP; v3 fpC; qt fqC;
    double lower, upper, kp, kd, target;
} Joint;

typedef struct {
    v3 cA, cB, n; double d; v3 aA, aB;
    double vn0;                       /* normal relative velocity at step start (restitution) */
    double lmax;                      /* largest normal impulse at the end of a substep */
} CPoint;

/* a contact point of the previous step, for warm starting across steps:
 * its normal impulse and its friction impulse as a world vector */
typedef struct { int a, b; v3 aA; double ln; v3 ft; } PrevPoint;
typedef struct { int a, b, np; CPoint p[4]; } Manifold;

enum { RK_NORMAL = 0, RK_FRICTION = 1, RK_EQ = 2, RK_LIMIT = 3, RK_DRIVE = 4 };

/* Soft constraint of a row in the position iterations (Box2D v3's "soft
 * step"): a spring-damper of natural frequency hz and damping ratio zeta
 * relative to the row's own effective mass, integrated implicitly over a
 * substep h.  With omega = 2 pi hz, a1 = 2 zeta + h omega, a2 = h omega a1:
 *   bias = (omega / a1) C,  mass scale = a2 / (1 + a2),  impulse scale = 1 / (1 + a2),
 *   dlambda = -(mass scale) (Jv + bias) / k - (impulse scale) lambda.
 * It is the implicit-Euler update (1 + 2 zeta omega h + h^2 omega^2) v' =
 * v - h omega^2 C of an isolated row.  on = 0: rigid. */
typedef struct { int on; double bias_rate, mass_scale, impulse_scale; } Soft;

typedef struct {
    int kind, a, b;                   /* a, b: env-local bodies, -1 = world */
    v3 lin, angA, angB;
    double k;                         /* J M^-1 J^T */
    double bias, relax_bias;
    double lambda, gamma, mu;
    int partner;                      /* friction: index of its normal row */
    int pt;                           /* contact point / limit side, for relax bias */
    int soft;                         /* soft in the position iterations (contact normal, joint equality) */
} Row;

typedef struct { int kind, idx, a, b, color, row0, nrows; } Constraint;

typedef struct {
    int nb, nj;
    Body* bodies; Joint* joints;
    int npairs; int (*pairs)[2];
    int nman; Manifold* man;
    int ntie; int (*tiepairs)[2];
    int ncons; Constraint* cons; int* order; int ncolors;
    int nrows; Row* rows;
    int nprev; PrevPoint* prev;       /* contact points of the previous step (warm start) */
    double* qR;                       /* pick task: joint coordinates at the last reset */
    unsigned status; long long ties;
    int round32;                      /* probe: velocities and poses stored as float32 */
    long long cnt[OC_NUM];
} Env;

struct oracle_world {
    int E; Env* envs;
    double dt; int substeps, pos_iters, vel_iters; v3 g; double margin, vmax;
    int contact_cap, pair_cap;
    double lin_damp, ang_damp, bounce; int warm;
    Soft csoft, jsoft;                /* soft contact normals, soft joint equality rows */
    /* pick task (off unless set): gripper joint, fingers, object, table */
    int task_on, t_grip, t_fa, t_fb, t_cube, t_table, t_A;
    double t_grasp_tol, t_touch_tol;
    double* t_half;                   /* [t_A] (h - l) / 2 of the delta controller */
    int nh; Hull* hulls;              /* hull library */
    int nb_total, nj_total;
    long long* body_off; long long* joint_off;
};

static const double TIE_EPS = 1e-5;    /* lengths (m) */
static const double TIE_DIR = 1e-6;    /* unit-vector components */
/* a decision is tie-adjacent when its deciding quantity is within 1e-5 of
 * the threshold but not structurally equal to it (exactly equal values, such
 * as the zero components of an axis-aligned normal, break the same way in
 * any precision) */
static void tie_w(Env* e, double a, double b, double w) { if (a != b && fabs(a - b) < w) e->ties++; }
static void tie(Env* e, double a, double b) { tie_w(e, a, b, TIE_EPS); }
/* tie check of the basis_axis choice */
static void tie_basis(Env* e, v3 a) {
    double c[3] = {fabs(a.x), fabs(a.y), fabs(a.z)};
    double mn = fmin(c[0], fmin(c[1], c[2]));
    for (int i = 0; i < 3; i++) tie_w(e, c[i], mn + 0.1, TIE_DIR);
}

/* ------------------------------------------------------------------------- */
/* shapes and mass                                                            */
/* ------------------------------------------------------------------------- */
void oracle_inertia(const double* d, double* out) {
    int type = (int)d[0];
    double m = d[4];
    if (type == OR_SPHERE) {
        double r = d[1];
        out[0] = out[1] = out[2] = 0.4 * m * r * r;
    } else if (type == OR_BOX) {
        double hx = d[1], hy = d[2], hz = d[3];
        out[0] = m / 3.0 * (hy * hy + hz * hz);
        out[1] = m / 3.0 * (hx * hx + hz * hz);
        out[2] = m / 3.0 * (hx * hx + hy * hy);
    } else if (type == OR_CAPSULE) {
        /* uniform solid: cylinder of length 2l plus two hemispheres whose
         * centroids sit 3r/8 beyond the segment ends (parallel-axis theorem) */
        double r = d[1], l = d[2];
        double vc = M_PI * r * r * 2.0 * l, vs = 4.0 / 3.0 * M_PI * r * r * r;
        double mc = m * vc / (vc + vs), ms = m * vs / (vc + vs);
        double izz = mc * r * r / 2.0 + ms * 0.4 * r * r;
        double ixx = mc * (r * r / 4.0 + l * l / 3.0) + ms * (0.4 * r * r + l * l + 0.75 * l * r);
        out[0] = out[1] = ixx; out[2] = izz;
    } else {
        out[0] = out[1] = out[2] = 0.0;
    }
}

static void body_from_desc(Body* b, const double* d) {
    memset(b, 0, sizeof(*b));
    b->type = (int)d[0];
    b->p[0] = d[1]; b->p[1] = d[2]; b->p[2] = d[3];
    b->mass = d[4];
    b->dyn = (b->type != OR_PLANE) && d[4] > 0.0;
    b->x = V(d[5], d[6], d[7]);
    b->q = qnormalize(Q(d[8], d[9], d[10], d[11]));
    b->q0 = b->q;
    b->mu = d[18];
    b->rest = d[19];
    b->group = (unsigned)d[20]; b->mask = (unsigned)d[21];
    if (b->dyn) {
        double I[3];
        oracle_inertia(d, I);
        b->inv_mass = 1.0 / b->mass;
        for (int i = 0; i < 3; i++) b->inv_I[i] = 1.0 / I[i];
        b->v = V(d[12], d[13], d[14]);
        b->w = V(d[15], d[16], d[17]);
    } else {
        b->inv_mass = 0.0;
        b->v = V(0, 0, 0); b->w = V(0, 0, 0);
    }
}

/* ------------------------------------------------------------------------- */
/* broadphase: brute force over i < j                                         */
/* ------------------------------------------------------------------------- */
static void aabb(const Body* b, double half_margin, v3* lo, v3* hi) {
    m3 R = qmat(b->q);
    v3 e;
    if (b->type == OR_SPHERE) {
        e = V(b->p[0], b->p[0], b->p[0]);
    } else if (b->type == OR_HULL) {
        /* a hull: the bounding sphere of its vertices about the body origin */
        e = V(b->hull->rad, b->hull->rad, b->hull->rad);
    } else if (b->type == OR_BOX) {
        /* half-widths of a rotated box: |R| h */
        e = V(fabs(R.m[0][0]) * b->p[0] + fabs(R.m[0][1]) * b->p[1] + fabs(R.m[0][2]) * b->p[2],
              fabs(R.m[1][0]) * b->p[0] + fabs(R.m[1][1]) * b->p[1] + fabs(R.m[1][2]) * b->p[2],
              fabs(R.m[2][0]) * b->p[0] + fabs(R.m[2][1]) * b->p[1] + fabs(R.m[2][2]) * b->p[2]);
    } else { /* capsule: segment +- l z_local, then +- r */
        v3 ax = mcol(&R, 2);
        double l = b->p[1], r = b->p[0];
        e = V(fabs(ax.x) * l + r, fabs(ax.y) * l + r, fabs(ax.z) * l + r);
    }
    e = add(e, V(half_margin, half_margin, half_margin));
    *lo = sub(b->x, e); *hi = add(b->x, e);
}

static int joint_connected(const Env* e, int i, int j) {
    for (int k = 0; k < e->nj; k++) {
        int p = e->joints[k].parent, c = e->joints[k].child;
        if ((p == i && c == j) || (p == j && c == i)) return 1;
    }
    return 0;
}

static void broadphase(const oracle_world* w, Env* e) {
    e->npairs = 0;
    for (int i = 0; i < e->nb; i++) {
        for (int j = i + 1; j < e->nb; j++) {
            const Body* A = &e->bodies[i]; const Body* B = &e->bodies[j];
            e->cnt[OC_PAIRS_TESTED]++;
            if (!A->dyn && !B->dyn) continue;
            if (!((A->group & B->mask) && (B->group & A->mask))) continue;
            if (joint_connected(e, i, j)) continue;
            int overlap = 1;
            if (A->type != OR_PLANE && B->type != OR_PLANE) {
                v3 la, ha, lb, hb;
                aabb(A, 0.5 * w->margin, &la, &ha);
                aabb(B, 0.5 * w->margin, &lb, &hb);
                overlap = la.x <= hb.x && lb.x <= ha.x && la.y <= hb.y && lb.y <= ha.y &&
                          la.z <= hb.z && lb.z <= ha.z;
            }
            if (!overlap) continue;
            if (e->npairs >= w->pair_cap) { e->status |= OR_ST_PAIR_OVERFLOW; continue; }
            e->pairs[e->npairs][0] = i; e->pairs[e->npairs][1] = j;
            e->npairs++;
        }
    }
    e->cnt[OC_PAIRS_CANDIDATE] += e->npairs;
}

/* ------------------------------------------------------------------------- */
/* narrowphase                                                                */
/* Convention: A is the lower shape rank (sphere < capsule < box < plane),    */
/* the lower index on equal ranks; n points from B toward A;                  */
/* d = n.(cA - cB) (< 0: penetration); a point is kept iff d < margin.       */
/* ------------------------------------------------------------------------- */
typedef struct { v3 cA, cB, n; double d; } Cand;
typedef struct { int n; Cand c[16]; } CandSet;

typedef struct { v3 x; m3 R; qt q; int type; double p[3]; const Hull* hull; } Shape;

static Shape shape_of(const Body* b) {
    Shape s; s.x = b->x; s.q = b->q; s.R = qmat(b->q); s.type = b->type;
    s.p[0] = b->p[0]; s.p[1] = b->p[1]; s.p[2] = b->p[2];
    s.hull = b->hull;
    return s;
}

/* pair order of the narrowphase: sphere < capsule < box < hull < plane */
static int shape_rank(int type) {
    switch (type) {
    case OR_SPHERE: return 0;
    case OR_CAPSULE: return 1;
    case OR_BOX: return 2;
    case OR_HULL: return 3;
    default: return 4;
    }
}

static void push(CandSet* cs, v3 cA, v3 cB, v3 n, double d) {
    if (cs->n < 16) { Cand* c = &cs->c[cs->n++]; c->cA = cA; c->cB = cB; c->n = n; c->d = d; }
}

/* two spheres (centres a, b; radii ra, rb); n = +z when centres coincide */
static void sphere_pair(CandSet* cs, v3 a, double ra, v3 b, double rb) {
    v3 dl = sub(a, b);
    double dist = norm(dl);
    v3 n = dist < 1e-9 ? V(0, 0, 1) : scl(dl, 1.0 / dist);
    push(cs, sub(a, scl(n, ra)), add(b, scl(n, rb)), n, dist - ra - rb);
}

/* closest point to p on segment [s0, s1] (clamped projection) */
static v3 closest_on_segment(v3 p, v3 s0, v3 s1) {
    v3 d = sub(s1, s0);
    double dd = dot(d, d);
    double t = dd > 0 ? clampd(dot(sub(p, s0), d) / dd, 0.0, 1.0) : 0.0;
    return add(s0, scl(d, t));
}

/* closest points of segments p0+s d1 and q0+t d2 (Ericson 2005, 5.1.9), with
 * the denominator |d1|^2|d2|^2 - (d1.d2)^2 written as |d1 x d2|^2 */
static void closest_segments(v3 p0, v3 p1, v3 q0, v3 q1, v3* cp, v3* cq) {
    v3 d1 = sub(p1, p0), d2 = sub(q1, q0), r = sub(p0, q0);
    double a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
    double s, t;
    if (a <= 1e-18 && e <= 1e-18) { s = t = 0.0; }
    else if (a <= 1e-18) { s = 0.0; t = clampd(f / e, 0.0, 1.0); }
    else {
        double c = dot(d1, r);
        if (e <= 1e-18) { t = 0.0; s = clampd(-c / a, 0.0, 1.0); }
        else {
            double b = dot(d1, d2);
            v3 cr = cross(d1, d2);
            double denom = dot(cr, cr);
            s = denom > 0.0 ? clampd((b * f - c * e) / denom, 0.0, 1.0) : 0.0;
            t = (b * s + f) / e;
            if (t < 0.0) { t = 0.0; s = clampd(-c / a, 0.0, 1.0); }
            else if (t > 1.0) { t = 1.0; s = clampd((b - c) / a, 0.0, 1.0); }
        }
    }
    *cp = add(p0, scl(d1, s));
    *cq = add(q0, scl(d2, t));
}

static void capsule_ends(const Shape* s, v3* e0, v3* e1) {
    v3 ax = mcol(&s->R, 2);
    *e0 = sub(s->x, scl(ax, s->p[1]));
    *e1 = add(s->x, scl(ax, s->p[1]));
}

/* sphere - sphere */
static void np_ss(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    (void)e; (void)m;
    sphere_pair(cs, A->x, A->p[0], B->x, B->p[0]);
}

/* sphere - plane */
static void np_sp(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    (void)e; (void)m;
    v3 N = mcol(&B->R, 2);
    double dist = dot(N, sub(A->x, B->x));
    push(cs, sub(A->x, scl(N, A->p[0])), sub(A->x, scl(N, dist)), N, dist - A->p[0]);
}

/* sphere - capsule */
static void np_sc(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    (void)e; (void)m;
    v3 b0, b1;
    capsule_ends(B, &b0, &b1);
    v3 q = closest_on_segment(A->x, b0, b1);
    sphere_pair(cs, A->x, A->p[0], q, B->p[0]);
}

/* sphere - box: clamp the centre into the box; if inside, leave through the
 * face of least penetration (lowest axis, + before - on ties) */
static void np_sb(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    (void)m;
    double r = A->p[0];
    v3 c = mtv(&B->R, sub(A->x, B->x));
    double h[3] = {B->p[0], B->p[1], B->p[2]};
    double cc[3] = {c.x, c.y, c.z};
    int inside = fabs(cc[0]) <= h[0] && fabs(cc[1]) <= h[1] && fabs(cc[2]) <= h[2];
    for (int i = 0; i < 3; i++) tie(e, fabs(cc[i]), h[i]);
    if (!inside) {
        double q[3];
        for (int i = 0; i < 3; i++) q[i] = clampd(cc[i], -h[i], h[i]);
        v3 ql = V(q[0], q[1], q[2]);
        v3 dl = sub(c, ql);
        double dist = norm(dl);
        v3 nl = dist > 0 ? scl(dl, 1.0 / dist) : V(0, 0, 1);
        v3 n = mv(&B->R, nl);
        v3 cB = add(B->x, mv(&B->R, ql));
        push(cs, sub(A->x, scl(n, r)), cB, n, dist - r);
    } else {
        int bi = 0; double bs = 1.0; double best = 1e300;
        for (int i = 0; i < 3; i++) {
            for (int sgn = 1; sgn >= -1; sgn -= 2) {
                double depth = h[i] - sgn * cc[i];
                if (depth < best) { best = depth; bi = i; bs = sgn; }
            }
        }
        v3 nl = scl(unit_axis(bi), bs);
        v3 ql = with_comp(c, bi, bs * h[bi]);
        v3 n = mv(&B->R, nl);
        push(cs, sub(A->x, scl(n, r)), add(B->x, mv(&B->R, ql)), n, -best - r);
    }
}

/* capsule - plane: both segment ends */
static void np_cp(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    (void)e; (void)m;
    v3 N = mcol(&B->R, 2);
    v3 ends[2];
    capsule_ends(A, &ends[0], &ends[1]);
    for (int k = 0; k < 2; k++) {
        double dist = dot(N, sub(ends[k], B->x));
        push(cs, sub(ends[k], scl(N, A->p[0])), sub(ends[k], scl(N, dist)), N, dist - A->p[0]);
    }
}

/* capsule - capsule: near-parallel overlapping axes give two points at the
 * ends of the overlap interval, otherwise the closest points of the segments */
static void np_cc(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    (void)m;
    v3 a0, a1, b0, b1;
    capsule_ends(A, &a0, &a1);
    capsule_ends(B, &b0, &b1);
    v3 dA = sub(a1, a0), dB = sub(b1, b0);
    double la = norm(dA), lb = norm(dB);
    double cr = norm(cross(dA, dB));
    tie_w(e, cr, 1e-3 * la * lb, TIE_DIR * la * lb);
    if (la > 0 && lb > 0 && cr < 1e-3 * la * lb) {
        v3 u = scl(dA, 1.0 / la);
        double t0 = dot(sub(b0, a0), u), t1 = dot(sub(b1, a0), u);
        double lo = fmax(0.0, fmin(t0, t1)), hi = fmin(la, fmax(t0, t1));
        if (lo <= hi) {
            tie_w(e, hi - lo, 1e-6, 1e-7);
            int cnt = (hi - lo) < 1e-6 ? 1 : 2;
            double xs[2] = {lo, hi};
            for (int k = 0; k < cnt; k++) {
                v3 pa = add(a0, scl(u, xs[k]));
                v3 pb = closest_on_segment(pa, b0, b1);
                sphere_pair(cs, pa, A->p[0], pb, B->p[0]);
            }
            return;
        }
    }
    v3 pa, pb;
    closest_segments(a0, a1, b0, b1, &pa, &pb);
    sphere_pair(cs, pa, A->p[0], pb, B->p[0]);
}

/* segment - box exact closest points in the box frame: the squared distance
 * along the segment is convex and piecewise quadratic between the parameters
 * where a coordinate crosses a slab face; minimise on each piece. */
static double segment_box_closest(v3 s0, v3 u, const double h[3], double* tbest) {
    double ts[8]; int nt = 0;
    ts[nt++] = 0.0; ts[nt++] = 1.0;
    double s0c[3] = {s0.x, s0.y, s0.z}, uc[3] = {u.x, u.y, u.z};
    for (int j = 0; j < 3; j++) {
        if (uc[j] == 0.0) continue;
        for (int sg = -1; sg <= 1; sg += 2) {
            double t = (sg * h[j] - s0c[j]) / uc[j];
            if (t > 0.0 && t < 1.0) ts[nt++] = t;
        }
    }
    for (int i = 1; i < nt; i++) { /* insertion sort */
        double x = ts[i]; int k = i - 1;
        while (k >= 0 && ts[k] > x) { ts[k + 1] = ts[k]; k--; }
        ts[k + 1] = x;
    }
    double best = 1e300; double bt = 0.0;
    for (int i = 0; i + 1 < nt; i++) {
        double ta = ts[i], tb = ts[i + 1];
        double tm = 0.5 * (ta + tb);
        double num = 0.0, den = 0.0;
        for (int j = 0; j < 3; j++) {
            double x = s0c[j] + tm * uc[j];
            double cj = x > h[j] ? h[j] : (x < -h[j] ? -h[j] : x);
            if (cj != x) { num += (s0c[j] - cj) * uc[j]; den += uc[j] * uc[j]; }
        }
        double cand[3] = {ta, tb, den > 0.0 ? clampd(-num / den, ta, tb) : ta};
        for (int k = 0; k < 3; k++) {
            double t = cand[k], f = 0.0;
            for (int j = 0; j < 3; j++) {
                double x = s0c[j] + t * uc[j];
                double cj = x > h[j] ? h[j] : (x < -h[j] ? -h[j] : x);
                f += (x - cj) * (x - cj);
            }
            if (f < best) { best = f; bt = t; }
        }
    }
    *tbest = bt;
    return sqrt(best);
}

/* capsule - box: SAT over the 3 box faces and the 3 crosses of box edges with
 * the segment, in the box frame.  Face case clips the segment to the face's
 * side slabs (<= 2 points); edge case gives one point. */
static void np_cb(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    double r = A->p[0];
    v3 a0, a1;
    capsule_ends(A, &a0, &a1);
    v3 s0 = mtv(&B->R, sub(a0, B->x)), s1 = mtv(&B->R, sub(a1, B->x));
    v3 u = sub(s1, s0);
    v3 mid = scl(add(s0, s1), 0.5);
    double h[3] = {B->p[0], B->p[1], B->p[2]};
    double ul = norm(u);
    v3 uh = ul > 0 ? scl(u, 1.0 / ul) : V(0, 0, 0);
    /* near[i]: an edge axis whose |cross| lies within TIE_DIR of the skip
     * threshold; psep[i] its separation had it been kept */
    double sep[6], psep[6]; v3 ax[6]; int valid[6], near[6] = {0};
    for (int i = 0; i < 6; i++) {
        v3 L;
        valid[i] = 1;
        if (i < 3) L = unit_axis(i);
        else {
            v3 c = cross(unit_axis(i - 3), uh);
            double cn = norm(c);
            near[i] = cn > 0.0 && cn != 1e-5 && fabs(cn - 1e-5) < TIE_DIR;
            valid[i] = cn >= 1e-5;
            if (!valid[i] && !near[i]) { sep[i] = -1e300; continue; }
            L = scl(c, 1.0 / cn);
        }
        if (dot(mid, L) < 0) L = neg(L);
        double hb = h[0] * fabs(L.x) + h[1] * fabs(L.y) + h[2] * fabs(L.z);
        double p0 = dot(s0, L), p1 = dot(s1, L);
        psep[i] = sep[i] = fmin(p0, p1) - hb - r;
        if (!valid[i]) sep[i] = -1e300;
        ax[i] = L;
    }
    double maxsep = -1e300;
    for (int i = 0; i < 6; i++) if (valid[i] && sep[i] > maxsep) maxsep = sep[i];
    int bf = 0;
    for (int i = 1; i < 3; i++) if (sep[i] > sep[bf]) bf = i;
    /* keeping or skipping a near-threshold axis matters only where it could
     * end the test (margin) or win over the faces: a tie only there */
    for (int i = 3; i < 6; i++)
        if (near[i] && psep[i] >= fmin(m, sep[bf] + 1e-4) - TIE_EPS) e->ties++;
    tie(e, maxsep, m);
    if (maxsep >= m) return;
    int be = -1;
    for (int i = 3; i < 6; i++) if (valid[i] && (be < 0 || sep[i] > sep[be])) be = i;
    if (be >= 0) tie(e, sep[be], sep[bf] + 1e-4);
    if (be >= 0 && sep[be] > sep[bf] + 1e-4) {
        /* edge case: the box edge parallel to e_i at the support toward L */
        v3 L = ax[be];
        int i = be - 3;
        double c[3];
        for (int k = 0; k < 3; k++) c[k] = (comp(L, k) >= 0 ? 1.0 : -1.0) * h[k];
        v3 q0 = V(c[0], c[1], c[2]), q1 = q0;
        q0 = with_comp(q0, i, -h[i]); q1 = with_comp(q1, i, h[i]);
        v3 ps, pe;
        closest_segments(s0, s1, q0, q1, &ps, &pe);
        v3 n = mv(&B->R, L);
        v3 cA = add(B->x, mv(&B->R, sub(ps, scl(L, r))));
        v3 cB = add(B->x, mv(&B->R, pe));
        push(cs, cA, cB, n, dot(L, sub(ps, pe)) - r);
        return;
    }
    /* face case on axis bf, oriented sigma */
    int k = bf;
    double sigma = comp(ax[k], k) >= 0 ? 1.0 : -1.0;
    double tlo = 0.0, thi = 1.0; int empty = 0;
    for (int j = 0; j < 3; j++) {
        if (j == k) continue;
        double sj = comp(s0, j), uj = comp(u, j);
        if (uj == 0.0) { if (fabs(sj) > h[j]) empty = 1; continue; }
        double ta = (-h[j] - sj) / uj, tb = (h[j] - sj) / uj;
        tlo = fmax(tlo, fmin(ta, tb)); thi = fmin(thi, fmax(ta, tb));
    }
    if (tlo > thi) empty = 1;
    v3 nl = scl(unit_axis(k), sigma);
    v3 n = mv(&B->R, nl);
    if (!empty) {
        double ts[2] = {tlo, thi};
        int cnt = tlo == thi ? 1 : 2;
        for (int a = 0; a < cnt; a++) {
            v3 q = add(s0, scl(u, ts[a]));
            double dist = sigma * comp(q, k) - h[k];
            v3 qb = with_comp(q, k, sigma * h[k]);
            v3 qa = sub(q, scl(nl, r));
            push(cs, add(B->x, mv(&B->R, qa)), add(B->x, mv(&B->R, qb)), n, dist - r);
        }
        return;
    }
    /* the segment misses the face's slab: one point from the exact closest
     * points of segment and box */
    double t;
    double dist = segment_box_closest(s0, u, h, &t);
    v3 q = add(s0, scl(u, t));
    v3 qb = V(clampd(q.x, -h[0], h[0]), clampd(q.y, -h[1], h[1]), clampd(q.z, -h[2], h[2]));
    v3 dl = sub(q, qb);
    v3 nn = dist > 1e-12 ? scl(dl, 1.0 / dist) : nl;
    v3 nw = mv(&B->R, nn);
    push(cs, add(B->x, mv(&B->R, sub(q, scl(nn, r)))), add(B->x, mv(&B->R, qb)), nw, dist - r);
}

/* box - plane: the 8 vertices, bit0/1/2 of the index choose +-hx/hy/hz */
static void np_bp(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    (void)e; (void)m;
    v3 N = mcol(&B->R, 2);
    for (int i = 0; i < 8; i++) {
        v3 lv = V((i & 1) ? A->p[0] : -A->p[0], (i & 2) ? A->p[1] : -A->p[1],
                  (i & 4) ? A->p[2] : -A->p[2]);
        v3 v = add(A->x, mv(&A->R, lv));
        double dist = dot(N, sub(v, B->x));
        push(cs, v, sub(v, scl(N, dist)), N, dist);
    }
}

/* Sutherland-Hodgman against dir.(x - c) <= hh */
static int clip_plane(const v3* in, int nin, v3* out, v3 dir, v3 c, double hh, Env* e) {
    int nout = 0;
    if (nin == 0) return 0;
    v3 prev = in[nin - 1];
    double fp = dot(dir, sub(prev, c)) - hh;
    for (int i = 0; i < nin; i++) {
        v3 cur = in[i];
        double fc = dot(dir, sub(cur, c)) - hh;
        tie(e, fc, 0.0);
        /* at most 8 vertices, whatever rounding does to convexity */
        if (fc <= 0.0) {
            if (fp > 0.0 && nout < 8) out[nout++] = add(prev, scl(sub(cur, prev), fp / (fp - fc)));
            if (nout < 8) out[nout++] = cur;
        } else if (fp <= 0.0 && nout < 8) {
            out[nout++] = add(prev, scl(sub(cur, prev), fp / (fp - fc)));
        }
        prev = cur; fp = fc;
    }
    return nout;
}

/* box - box: SAT over 15 axes (A faces, B faces, A_i x B_j row-major),
 * face case with incident-face clipping, or one edge-edge point */
static void np_bb(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    v3 a[3], b[3];
    for (int i = 0; i < 3; i++) { a[i] = mcol(&A->R, i); b[i] = mcol(&B->R, i); }
    const double* hA = A->p; const double* hB = B->p;
    v3 dl = sub(A->x, B->x);
    /* near[k]: an edge axis whose |cross| lies within TIE_DIR of the skip
     * threshold; psep[k] its separation had it been kept */
    double sep[15], psep[15]; v3 ax[15]; int valid[15], near[15] = {0};
    for (int k = 0; k < 15; k++) {
        v3 L;
        valid[k] = 1;
        if (k < 3) L = a[k];
        else if (k < 6) L = b[k - 3];
        else {
            v3 c = cross(a[(k - 6) / 3], b[(k - 6) % 3]);
            double cn = norm(c);
            near[k] = cn > 0.0 && cn != 1e-5 && fabs(cn - 1e-5) < TIE_DIR;
            valid[k] = cn >= 1e-5;
            if (!valid[k] && !near[k]) { sep[k] = -1e300; continue; }
            L = scl(c, 1.0 / cn);
        }
        if (dot(dl, L) < 0) L = neg(L);
        double ra = hA[0] * fabs(dot(a[0], L)) + hA[1] * fabs(dot(a[1], L)) + hA[2] * fabs(dot(a[2], L));
        double rb = hB[0] * fabs(dot(b[0], L)) + hB[1] * fabs(dot(b[1], L)) + hB[2] * fabs(dot(b[2], L));
        psep[k] = sep[k] = dot(dl, L) - ra - rb;
        if (!valid[k]) sep[k] = -1e300;
        ax[k] = L;
    }
    double maxsep = -1e300;
    for (int k = 0; k < 15; k++) if (valid[k] && sep[k] > maxsep) maxsep = sep[k];
    int fa = 0, fb = 3, be = -1;
    for (int k = 1; k < 3; k++) if (sep[k] > sep[fa]) fa = k;
    for (int k = 4; k < 6; k++) if (sep[k] > sep[fb]) fb = k;
    for (int k = 6; k < 15; k++) if (valid[k] && (be < 0 || sep[k] > sep[be])) be = k;
    double sf = fmax(sep[fa], sep[fb]);
    /* a near-threshold axis is a tie only where it could end the test or
     * win over the faces */
    for (int k = 6; k < 15; k++)
        if (near[k] && psep[k] >= fmin(m, sf + 1e-4) - TIE_EPS) e->ties++;
    tie(e, maxsep, m);
    if (maxsep >= m) return;
    if (be >= 0) tie(e, sep[be], sf + 1e-4);
    if (be >= 0 && sep[be] > sf + 1e-4) {
        v3 L = ax[be];
        int i = (be - 6) / 3, j = (be - 6) % 3;
        /* A's edge parallel to a_i at A's support toward -L; B's toward +L */
        v3 ca = A->x, cb = B->x;
        for (int k = 0; k < 3; k++) {
            if (k != i) ca = add(ca, scl(a[k], (dot(a[k], L) > 0 ? -1.0 : 1.0) * hA[k]));
            if (k != j) cb = add(cb, scl(b[k], (dot(b[k], L) >= 0 ? 1.0 : -1.0) * hB[k]));
        }
        v3 pa, pb;
        closest_segments(sub(ca, scl(a[i], hA[i])), add(ca, scl(a[i], hA[i])),
                         sub(cb, scl(b[j], hB[j])), add(cb, scl(b[j], hB[j])), &pa, &pb);
        push(cs, pa, pb, L, dot(L, sub(pa, pb)));
        return;
    }
    tie(e, sep[fb], sep[fa] + 1e-4);
    int refB = sep[fb] > sep[fa] + 1e-4;
    const Shape* Rf = refB ? B : A;   /* reference box */
    const Shape* In = refB ? A : B;   /* incident box */
    int k = refB ? fb - 3 : fa;
    v3 n = ax[refB ? fb : fa];                    /* B -> A */
    v3 nref = refB ? n : neg(n);                  /* outward normal of the reference face */
    v3 r[3], ic[3];
    for (int t = 0; t < 3; t++) { r[t] = mcol(&Rf->R, t); ic[t] = mcol(&In->R, t); }
    v3 cref = add(Rf->x, scl(nref, Rf->p[k]));
    int ju = (k + 1) % 3, jv = (k + 2) % 3;
    v3 uu = r[ju], vv = r[jv];
    double hu = Rf->p[ju], hv = Rf->p[jv];
    /* incident face: minimal dot(face normal, nref); order +x,-x,+y,-y,+z,-z */
    int fi = 0; double fs = 1.0, best = 1e300, second = 1e300;
    for (int t = 0; t < 3; t++) {
        for (int sg = 1; sg >= -1; sg -= 2) {
            double dd = sg * dot(ic[t], nref);
            if (dd < best) { second = best; best = dd; fi = t; fs = sg; }
            else if (dd < second) second = dd;
        }
    }
    tie(e, best, second);
    int i1 = (fi + 1) % 3, i2 = (fi + 2) % 3;
    v3 fc = add(In->x, scl(ic[fi], fs * In->p[fi]));
    v3 e1 = scl(ic[i1], In->p[i1]), e2 = scl(ic[i2], In->p[i2]);
    v3 poly[8], tmp[8];
    poly[0] = add(add(fc, e1), e2);
    poly[1] = add(sub(fc, e1), e2);
    poly[2] = sub(sub(fc, e1), e2);
    poly[3] = sub(add(fc, e1), e2);
    int np = 4;
    np = clip_plane(poly, np, tmp, uu, cref, hu, e);
    np = clip_plane(tmp, np, poly, neg(uu), cref, hu, e);
    np = clip_plane(poly, np, tmp, vv, cref, hv, e);
    np = clip_plane(tmp, np, poly, neg(vv), cref, hv, e);
    for (int t = 0; t < np; t++) {
        v3 x = poly[t];
        double dist = dot(nref, sub(x, cref));
        v3 xp = sub(x, scl(nref, dist));
        if (refB) push(cs, x, xp, n, dist);
        else push(cs, xp, x, n, dist);
    }
}


/* ------------------------------------------------------------------ hulls */
/* A convex polytope in world coordinates: a hull (triangular faces), or a
 * box (8 corners, 6 quadrilateral faces).  Faces are counter-clockwise
 * seen from outside; each edge lists its two faces. */
enum { P_MAXV = 16, P_MAXF = 28, P_MAXE = 42 };
typedef struct {
    int nv, nf, ne;
    v3 v[P_MAXV];
    v3 fn[P_MAXF]; double fd[P_MAXF];  /* outward unit normal, offset fn.x = fd on the face */
    int fv[P_MAXF][4], fnv[P_MAXF];
    int e[P_MAXE][2], ef[P_MAXE][2];
    v3 c;                              /* body origin (interior) */
} Poly;

static void poly_faces(Poly* P) {
    for (int f = 0; f < P->nf; f++) {
        v3 a = P->v[P->fv[f][0]], b = P->v[P->fv[f][1]], c = P->v[P->fv[f][2]];
        v3 n = cross(sub(b, a), sub(c, a));
        n = scl(n, 1.0 / norm(n));
        P->fn[f] = n; P->fd[f] = dot(n, a);
    }
}

static void poly_of(const Shape* S, Poly* P) {
    P->c = S->x;
    if (S->type == OR_BOX) {
        static const int F[6][4] = {{1, 3, 7, 5}, {2, 0, 4, 6}, {3, 2, 6, 7}, {0, 1, 5, 4}, {4, 5, 7, 6}, {2, 3, 1, 0}};
        P->nv = 8; P->nf = 6; P->ne = 0;
        for (int k = 0; k < 8; k++)
            P->v[k] = add(S->x, mv(&S->R, V((k & 1) ? S->p[0] : -S->p[0], (k & 2) ? S->p[1] : -S->p[1],
                                              (k & 4) ? S->p[2] : -S->p[2])));
        for (int f = 0; f < 6; f++) { P->fnv[f] = 4; for (int k = 0; k < 4; k++) P->fv[f][k] = F[f][k]; }
        /* each edge once, from the face listing it a -> b with a < b; its
         * other face lists b -> a */
        for (int f = 0; f < 6; f++)
            for (int k = 0; k < 4; k++) {
                int a = F[f][k], b = F[f][(k + 1) % 4];
                if (a > b) continue;
                int g = -1;
                for (int h = 0; h < 6 && g < 0; h++)
                    for (int q = 0; q < 4; q++)
                        if (F[h][q] == b && F[h][(q + 1) % 4] == a) { g = h; break; }
                P->e[P->ne][0] = a; P->e[P->ne][1] = b; P->ef[P->ne][0] = f; P->ef[P->ne][1] = g; P->ne++;
            }
    } else {
        const Hull* H = S->hull;
        P->nv = H->nv; P->nf = H->nt; P->ne = H->ne;
        for (int k = 0; k < H->nv; k++) P->v[k] = add(S->x, mv(&S->R, H->v[k]));
        for (int f = 0; f < H->nt; f++) { P->fnv[f] = 3; for (int k = 0; k < 3; k++) P->fv[f][k] = H->t[f][k]; }
        for (int k = 0; k < H->ne; k++) {
            P->e[k][0] = H->e[k][0]; P->e[k][1] = H->e[k][1];
            P->ef[k][0] = H->ef[k][0]; P->ef[k][1] = H->ef[k][1];
        }
    }
    poly_faces(P);
}

/* hull - plane: every vertex within the margin (as box - plane) */
static void np_hp(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    (void)e;
    v3 N = mcol(&B->R, 2);
    const Hull* H = A->hull;
    for (int k = 0; k < H->nv; k++) {
        v3 v = add(A->x, mv(&A->R, H->v[k]));
        double dist = dot(N, sub(v, B->x));
        if (dist < m + 1e-4) push(cs, v, sub(v, scl(N, dist)), N, dist);   /* 1e-4: margin ties stay visible */
    }
}

/* closest point of triangle (a, b, c) to p (Ericson 2005, 5.1.5) */
static v3 closest_on_triangle(v3 p, v3 a, v3 b, v3 c) {
    v3 ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
    double d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) return a;
    v3 bp = sub(p, b);
    double d3 = dot(ab, bp), d4 = dot(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) return b;
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) return add(a, scl(ab, d1 / (d1 - d3)));
    v3 cp = sub(p, c);
    double d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) return c;
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) return add(a, scl(ac, d2 / (d2 - d6)));
    double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0)
        return add(b, scl(sub(c, b), (d4 - d3) / ((d4 - d3) + (d5 - d6))));
    double den = 1.0 / (va + vb + vc);
    return add(a, add(scl(ab, vb * den), scl(ac, vc * den)));
}

/* sphere - hull: centre inside (no face plane separates it): push out along
 * the face of least penetration; outside: the closest point of the surface */
static void np_sh(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    (void)m;
    Poly P;
    poly_of(B, &P);
    v3 c = A->x;
    double r = A->p[0];
    double smax = -INFINITY, s2 = -INFINITY;
    int fb = 0;
    for (int f = 0; f < P.nf; f++) {
        double sf = dot(P.fn[f], c) - P.fd[f];
        if (sf > smax) { s2 = smax; smax = sf; fb = f; } else if (sf > s2) s2 = sf;
    }
    tie(e, smax, 0.0);
    if (smax <= 0.0) {
        tie(e, smax, s2);
        v3 n = P.fn[fb];
        push(cs, sub(c, scl(n, r)), sub(c, scl(n, smax)), n, smax - r);
        return;
    }
    double best = INFINITY;
    v3 q = c;
    for (int f = 0; f < P.nf; f++) {
        v3 t = closest_on_triangle(c, P.v[P.fv[f][0]], P.v[P.fv[f][1]], P.v[P.fv[f][2]]);
        double d2 = dot(sub(c, t), sub(c, t));
        if (d2 < best) { best = d2; q = t; }
    }
    double dist = sqrt(best);
    v3 n = scl(sub(c, q), 1.0 / dist);
    push(cs, sub(c, scl(n, r)), q, n, dist - r);
}

/* box or hull (A) - hull (B): separating axes over the face normals of A,
 * then of B, then the cross products of edge pairs that bound a face of
 * the Minkowski difference (their arcs on the Gauss map cross); a B face
 * is the reference only if it beats the best A face by 1e-4 m, an edge
 * pair only if it beats the best face by 1e-4 m.  Face case: the most
 * anti-parallel face of the other polytope is clipped against the side
 * planes of the reference face; edge case: one point, the closest points
 * of the two edges. */
static void np_poly(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    Poly PA, PB;
    poly_of(A, &PA);
    poly_of(B, &PB);
    double sa = -INFINITY; int fa = 0;
    e->cnt[OC_SAT_FACE_VERT] += PA.nf * PB.nv + PB.nf * PA.nv;
    for (int f = 0; f < PA.nf; f++) {
        double sf = INFINITY;
        for (int k = 0; k < PB.nv; k++) sf = fmin(sf, dot(PA.fn[f], PB.v[k]) - PA.fd[f]);
        if (sf > sa) { sa = sf; fa = f; }
    }
    double sb = -INFINITY; int fb = 0;
    for (int f = 0; f < PB.nf; f++) {
        double sf = INFINITY;
        for (int k = 0; k < PA.nv; k++) sf = fmin(sf, dot(PB.fn[f], PA.v[k]) - PB.fd[f]);
        if (sf > sb) { sb = sf; fb = f; }
    }
    double se = -INFINITY; int ea = -1, eb = -1; v3 axe = V(0, 0, 0);
    if (fmax(sa, sb) < m) e->cnt[OC_SAT_EDGE_PAIR] += PA.ne * PB.ne;   /* the work that remains after the face axes */
    for (int i = 0; i < PA.ne; i++) {
        v3 a = PA.fn[PA.ef[i][0]], b = PA.fn[PA.ef[i][1]];
        v3 bxa = cross(b, a);
        v3 ua = sub(PA.v[PA.e[i][1]], PA.v[PA.e[i][0]]);
        for (int j = 0; j < PB.ne; j++) {
            v3 c = neg(PB.fn[PB.ef[j][0]]), d = neg(PB.fn[PB.ef[j][1]]);
            v3 dxc = cross(d, c);
            double cba = dot(c, bxa), dba = dot(d, bxa), adc = dot(a, dxc), bdc = dot(b, dxc);
            /* a pair on the verge of this test has its axis next to a face
             * normal and that face's separation, so the 1e-4 m face
             * preference below decides the outcome either way: no tie */
            if (!(cba * dba < 0.0 && adc * bdc < 0.0 && cba * bdc > 0.0)) continue;
            v3 ub = sub(PB.v[PB.e[j][1]], PB.v[PB.e[j][0]]);
            v3 ax = cross(ua, ub);
            double l = norm(ax), lim = 1e-5 * norm(ua) * norm(ub);
            tie_w(e, l, lim, TIE_DIR * norm(ua) * norm(ub));
            if (l < lim) continue;
            ax = scl(ax, 1.0 / l);
            if (dot(ax, sub(PA.v[PA.e[i][0]], PA.c)) < 0.0) ax = neg(ax);
            double sij = dot(ax, sub(PB.v[PB.e[j][0]], PA.v[PA.e[i][0]]));
            if (sij > se) { se = sij; ea = i; eb = j; axe = ax; }
        }
    }
    double maxsep = fmax(fmax(sa, sb), se);
    tie(e, maxsep, m);
    if (maxsep >= m) return;
    double sf = fmax(sa, sb);
    if (ea >= 0) tie(e, se, sf + 1e-4);
    if (ea >= 0 && se > sf + 1e-4) {
        v3 pa, pb;
        closest_segments(PA.v[PA.e[ea][0]], PA.v[PA.e[ea][1]], PB.v[PB.e[eb][0]], PB.v[PB.e[eb][1]], &pa, &pb);
        v3 n = neg(axe);
        push(cs, pa, pb, n, dot(n, sub(pa, pb)));
        return;
    }
    tie(e, sb, sa + 1e-4);
    int refB = sb > sa + 1e-4;
    const Poly* R = refB ? &PB : &PA;
    const Poly* I = refB ? &PA : &PB;
    int rf = refB ? fb : fa;
    v3 nref = R->fn[rf];
    int inc = 0; double best = INFINITY, second = INFINITY;
    for (int g = 0; g < I->nf; g++) {
        double dd = dot(I->fn[g], nref);
        if (dd < best) { second = best; best = dd; inc = g; } else if (dd < second) second = dd;
    }
    tie_w(e, best, second, TIE_DIR);
    v3 bufa[8], bufb[8];
    v3* src = bufa; v3* dst = bufb;
    int np = I->fnv[inc];
    for (int k = 0; k < np; k++) src[k] = I->v[I->fv[inc][k]];
    int nr = R->fnv[rf];
    for (int k = 0; k < nr; k++) {
        v3 p0 = R->v[R->fv[rf][k]], p1 = R->v[R->fv[rf][(k + 1) % nr]];
        v3 side = cross(sub(p1, p0), nref);
        side = scl(side, 1.0 / norm(side));
        np = clip_plane(src, np, dst, side, p0, 0.0, e);
        v3* t = src; src = dst; dst = t;
    }
    v3 pref = R->v[R->fv[rf][0]];
    for (int k = 0; k < np; k++) {
        v3 x = src[k];
        double dist = dot(nref, sub(x, pref));
        if (!refB) push(cs, sub(x, scl(nref, dist)), x, neg(nref), dist);
        else push(cs, x, sub(x, scl(nref, dist)), nref, dist);
    }
}

/* closest points of segment [s0, s1] and the surface of polytope P (its
 * triangles): for each triangle, the segment's ends against the triangle
 * and the segment against the triangle's edges; the overall least distance */
static double segment_poly_closest(const Poly* P, v3 s0, v3 s1, v3* ps, v3* pq) {
    double best = INFINITY;
    for (int f = 0; f < P->nf; f++) {
        v3 t[3] = {P->v[P->fv[f][0]], P->v[P->fv[f][1]], P->v[P->fv[f][2]]};
        v3 q = closest_on_triangle(s0, t[0], t[1], t[2]);
        double d2 = dot(sub(s0, q), sub(s0, q));
        if (d2 < best) { best = d2; *ps = s0; *pq = q; }
        q = closest_on_triangle(s1, t[0], t[1], t[2]);
        d2 = dot(sub(s1, q), sub(s1, q));
        if (d2 < best) { best = d2; *ps = s1; *pq = q; }
        for (int k = 0; k < 3; k++) {
            v3 a, b;
            closest_segments(s0, s1, t[k], t[(k + 1) % 3], &a, &b);
            d2 = dot(sub(a, b), sub(a, b));
            if (d2 < best) { best = d2; *ps = a; *pq = b; }
        }
    }
    return sqrt(best);
}

/* capsule - hull: separating axes over the hull's face normals and the
 * cross products of the segment with the hull's edges (each edge axis in
 * the orientation that separates more); an edge axis only if it beats the
 * best face by 1e-4 m.  Face case: the segment clipped to the face's side
 * planes, up to two points, or, when nothing of it lies over the face, the
 * exact closest points of segment and hull surface; edge case: those exact
 * closest points (the edge that gives the axis need not support the hull
 * along it). */
static void np_ch(Env* e, const Shape* A, const Shape* B, double m, CandSet* cs) {
    double r = A->p[0];
    v3 s0, s1;
    capsule_ends(A, &s0, &s1);
    v3 u = sub(s1, s0);
    double ul = norm(u);
    Poly P;
    poly_of(B, &P);
    double sf = -INFINITY; int bf = 0;
    for (int f = 0; f < P.nf; f++) {
        double sg = fmin(dot(P.fn[f], s0), dot(P.fn[f], s1)) - P.fd[f] - r;
        if (sg > sf) { sf = sg; bf = f; }
    }
    double se = -INFINITY; int be = -1; v3 le = V(0, 0, 0);
    for (int k = 0; k < P.ne; k++) {
        v3 ev = sub(P.v[P.e[k][1]], P.v[P.e[k][0]]);
        v3 c = cross(ev, u);
        double cn = norm(c), lim = 1e-5 * norm(ev) * ul;
        tie_w(e, cn, lim, TIE_DIR * norm(ev) * ul);
        if (!(cn > lim)) continue;
        v3 L = scl(c, 1.0 / cn);
        double hmax = -INFINITY, hmin = INFINITY;
        for (int q = 0; q < P.nv; q++) { double t = dot(L, P.v[q]); hmax = fmax(hmax, t); hmin = fmin(hmin, t); }
        double sp = fmin(dot(L, s0), dot(L, s1)) - hmax - r;    /* capsule on the +L side */
        double sn = hmin - fmax(dot(L, s0), dot(L, s1)) - r;    /* capsule on the -L side */
        tie(e, sp, sn);
        if (sn > sp) { sp = sn; L = neg(L); }
        if (sp > se) { se = sp; be = k; le = L; }
    }
    double maxsep = fmax(sf, se);
    tie(e, maxsep, m);
    if (maxsep >= m) return;
    if (be >= 0) tie(e, se, sf + 1e-4);
    v3 n = P.fn[bf];
    int empty = 0;
    double tlo = 0.0, thi = 1.0;
    if (be >= 0 && se > sf + 1e-4) {
        /* the edge that gave the axis need not be the hull's support along
         * it: the exact closest points of segment and surface */
        empty = 1;
        n = le;
    }
    for (int k = 0; k < P.fnv[bf] && !empty; k++) {
        v3 p0 = P.v[P.fv[bf][k]], p1 = P.v[P.fv[bf][(k + 1) % P.fnv[bf]]];
        v3 sd = cross(sub(p1, p0), n);
        sd = scl(sd, 1.0 / norm(sd));
        double g0 = dot(sd, sub(s0, p0)), gu = dot(sd, u);
        if (gu == 0.0) { if (g0 > 0.0) empty = 1; continue; }
        double t = -g0 / gu;
        if (gu > 0.0) thi = fmin(thi, t); else tlo = fmax(tlo, t);
    }
    tie(e, tlo, thi);
    if (tlo > thi) empty = 1;
    if (!empty) {
        double ts[2] = {tlo, thi};
        int cnt = tlo == thi ? 1 : 2;
        for (int a = 0; a < cnt; a++) {
            v3 q = add(s0, scl(u, ts[a]));
            double dist = dot(n, q) - P.fd[bf];
            push(cs, sub(q, scl(n, r)), sub(q, scl(n, dist)), n, dist - r);
        }
        return;
    }
    v3 ps = s0, pq = P.v[0];
    double dist = segment_poly_closest(&P, s0, s1, &ps, &pq);
    v3 nn = dist > 1e-12 ? scl(sub(ps, pq), 1.0 / dist) : n;
    push(cs, sub(ps, scl(nn, r)), pq, nn, dist - r);
}

static int first_unused(const int* used, int n) {
    for (int k = 0; k < n; k++) if (!used[k]) return k;
    return 0;
}

/* reduce > 4 candidates to 4, selection order p1..p4 (positions: cB) */
static int reduce4(Env* e, const Cand* c, int n, int* sel) {
    int used[16] = {0};
    int i1 = 0;
    for (int k = 1; k < n; k++) if (c[k].d < c[i1].d) i1 = k;
    for (int k = 0; k < n; k++) if (k != i1) tie(e, c[k].d, c[i1].d);
    used[i1] = 1;
    double best, second; int i2 = first_unused(used, n);
    best = -1.0; second = -1.0;
    for (int k = 0; k < n; k++) {
        if (used[k]) continue;
        double s = dot(sub(c[k].cB, c[i1].cB), sub(c[k].cB, c[i1].cB));
        if (s > best) { second = best; best = s; i2 = k; } else if (s > second) second = s;
    }
    tie(e, best, second);
    used[i2] = 1;
    v3 e12 = sub(c[i2].cB, c[i1].cB);
    int i3 = first_unused(used, n); best = -1.0; second = -1.0;
    for (int k = 0; k < n; k++) {
        if (used[k]) continue;
        double s = norm(cross(e12, sub(c[k].cB, c[i1].cB)));
        if (s > best) { second = best; best = s; i3 = k; } else if (s > second) second = s;
    }
    tie(e, best, second);
    used[i3] = 1;
    int i4 = first_unused(used, n); best = -1.0; second = -1.0;
    v3 P1 = c[i1].cB, P2 = c[i2].cB, P3 = c[i3].cB;
    for (int k = 0; k < n; k++) {
        if (used[k]) continue;
        v3 P = c[k].cB;
        double s = norm(cross(sub(P2, P1), sub(P, P1))) + norm(cross(sub(P3, P2), sub(P, P2))) +
                   norm(cross(sub(P1, P3), sub(P, P3)));
        if (s > best) { second = best; best = s; i4 = k; } else if (s > second) second = s;
    }
    tie(e, best, second);
    sel[0] = i1; sel[1] = i2; sel[2] = i3; sel[3] = i4;
    return 4;
}

/* Narrowphase of the ordered pair (A, B); returns kept points in `out`.
 * *margin_tie is set when a candidate's d lies within 1e-5 of the margin. */
static void candidates(Env* e, const Shape* A, const Shape* B, double m, CandSet* out) {
    CandSet cs; cs.n = 0;
    int ta = A->type, tb = B->type;
    int slot = -1;
    if (ta == OR_SPHERE && tb == OR_SPHERE) { np_ss(e, A, B, m, &cs); slot = OC_NP_SS; }
    else if (ta == OR_SPHERE && tb == OR_CAPSULE) { np_sc(e, A, B, m, &cs); slot = OC_NP_SC; }
    else if (ta == OR_SPHERE && tb == OR_BOX) { np_sb(e, A, B, m, &cs); slot = OC_NP_SB; }
    else if (ta == OR_SPHERE && tb == OR_PLANE) { np_sp(e, A, B, m, &cs); slot = OC_NP_SP; }
    else if (ta == OR_CAPSULE && tb == OR_CAPSULE) { np_cc(e, A, B, m, &cs); slot = OC_NP_CC; }
    else if (ta == OR_CAPSULE && tb == OR_BOX) { np_cb(e, A, B, m, &cs); slot = OC_NP_CB; }
    else if (ta == OR_CAPSULE && tb == OR_PLANE) { np_cp(e, A, B, m, &cs); slot = OC_NP_CP; }
    else if (ta == OR_BOX && tb == OR_BOX) { np_bb(e, A, B, m, &cs); slot = OC_NP_BB; }
    else if (ta == OR_BOX && tb == OR_PLANE) { np_bp(e, A, B, m, &cs); slot = OC_NP_BP; }
    else if (ta == OR_SPHERE && tb == OR_HULL) { np_sh(e, A, B, m, &cs); slot = OC_NP_SH; }
    else if ((ta == OR_BOX || ta == OR_HULL) && tb == OR_HULL) { np_poly(e, A, B, m, &cs); slot = OC_NP_XH; }
    else if (ta == OR_HULL && tb == OR_PLANE) { np_hp(e, A, B, m, &cs); slot = OC_NP_HP; }
    else if (ta == OR_CAPSULE && tb == OR_HULL) { np_ch(e, A, B, m, &cs); slot = OC_NP_CH; }
    if (slot >= 0) e->cnt[slot]++;
    *out = cs;
}

static int collide(Env* e, const Shape* A, const Shape* B, double m, Cand* out, int* margin_tie) {
    CandSet cs;
    candidates(e, A, B, m, &cs);
    Cand kept[16]; int nk = 0;
    *margin_tie = 0;
    for (int i = 0; i < cs.n; i++) {
        if (fabs(cs.c[i].d - m) < TIE_EPS) { *margin_tie = 1; e->ties++; }
        if (cs.c[i].d < m) kept[nk++] = cs.c[i];
    }
    if (nk <= 4) {
        for (int i = 0; i < nk; i++) out[i] = kept[i];
        return nk;
    }
    int sel[4];
    reduce4(e, kept, nk, sel);
    for (int i = 0; i < 4; i++) out[i] = kept[sel[i]];
    return 4;
}

static void narrowphase(const oracle_world* w, Env* e) {
    e->nman = 0; e->ntie = 0;
    int total = 0, stop = 0;
    for (int p = 0; p < e->npairs; p++) {
        int i = e->pairs[p][0], j = e->pairs[p][1];
        const Body* Bi = &e->bodies[i]; const Body* Bj = &e->bodies[j];
        /* order by shape rank, then index */
        int a = i, b = j;
        if (shape_rank(Bj->type) < shape_rank(Bi->type)) { a = j; b = i; }
        Shape A = shape_of(&e->bodies[a]), B = shape_of(&e->bodies[b]);
        Cand pts[4]; int mt;
        int np = collide(e, &A, &B, w->margin, pts, &mt);
        if (mt) { e->tiepairs[e->ntie][0] = i; e->tiepairs[e->ntie][1] = j; e->ntie++; }
        if (np == 0) continue;
        /* keep the longest prefix of manifolds (pair order) within capacity */
        if (stop || total + np > w->contact_cap) { stop = 1; e->status |= OR_ST_CONTACT_OVERFLOW; continue; }
        Manifold* M = &e->man[e->nman++];
        M->a = a; M->b = b; M->np = np;
        const Body* BA = &e->bodies[a]; const Body* BB = &e->bodies[b];
        m3 RA = qmat(BA->q), RB = qmat(BB->q);
        for (int k = 0; k < np; k++) {
            CPoint* c = &M->p[k];
            c->cA = pts[k].cA; c->cB = pts[k].cB; c->n = pts[k].n; c->d = pts[k].d;
            c->aA = mtv(&RA, sub(c->cA, BA->x));   /* body-local anchors */
            c->aB = mtv(&RB, sub(c->cB, BB->x));
            if (e->round32) { c->n = r32v(c->n); c->aA = r32v(c->aA); c->aB = r32v(c->aB); }
            /* approach speed along n at the step-start velocities */
            v3 uA = add(BA->v, cross(BA->w, sub(c->cA, BA->x)));
            v3 uB = add(BB->v, cross(BB->w, sub(c->cB, BB->x)));
            c->vn0 = dot(c->n, sub(uA, uB));
            c->lmax = 0.0;
        }
        total += np;
    }
    e->cnt[OC_CONTACT_POINTS] += total;
}

/* ------------------------------------------------------------------------- */
/* colouring                                                                  */
/* ------------------------------------------------------------------------- */
int oracle_color(int n, const int* a, const int* b, const int* dyn, int* colors) {
    /* used[body] bitmask of colours already taken by constraints on it */
    int maxb = 0;
    for (int i = 0; i < n; i++) { if (a[i] + 1 > maxb) maxb = a[i] + 1; if (b[i] + 1 > maxb) maxb = b[i] + 1; }
    uint64_t* used = (uint64_t*)calloc((size_t)(maxb > 0 ? maxb : 1), sizeof(uint64_t));
    int ncol = 0, overflow = 0;
    for (int i = 0; i < n; i++) {
        uint64_t mask = 0;
        int da = a[i] >= 0 && dyn[a[i]], db = b[i] >= 0 && dyn[b[i]];
        if (da) mask |= used[a[i]];
        if (db) mask |= used[b[i]];
        int c = 0;
        while (c < 64 && (mask >> c) & 1ull) c++;
        if (c == 64) { colors[i] = -1; overflow = 1; continue; }
        colors[i] = c;
        if (da) used[a[i]] |= 1ull << c;
        if (db) used[b[i]] |= 1ull << c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(used);
    return overflow ? -1 : ncol;
}

static void build_constraints(Env* e) {
    int n = e->nj + e->nman;
    e->ncons = n;
    int* a = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    int* b = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    int* dyn = (int*)malloc(sizeof(int) * (e->nb > 0 ? e->nb : 1));
    int* col = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < e->nb; i++) dyn[i] = e->bodies[i].dyn;
    int row = 0;
    for (int i = 0; i < e->nj; i++) {
        Constraint* c = &e->cons[i];
        c->kind = 0; c->idx = i; c->a = e->joints[i].parent; c->b = e->joints[i].child;
        c->row0 = row; c->nrows = 8; row += 8;
        a[i] = c->a; b[i] = c->b;
    }
    for (int m = 0; m < e->nman; m++) {
        Constraint* c = &e->cons[e->nj + m];
        c->kind = 1; c->idx = m; c->a = e->man[m].a; c->b = e->man[m].b;
        c->row0 = row; c->nrows = 3 * e->man[m].np; row += c->nrows;
        a[e->nj + m] = c->a; b[e->nj + m] = c->b;
    }
    e->nrows = row;
    int nc = oracle_color(n, a, b, dyn, col);
    if (nc < 0) {
        e->status |= OR_ST_COLOR_OVERFLOW;
        nc = 64;
    }
    e->ncolors = nc;
    for (int i = 0; i < n; i++) e->cons[i].color = col[i];
    /* solve order: by colour, constraint-list order inside a colour;
     * constraints left without a colour are not solved */
    int k = 0;
    for (int c = 0; c < nc; c++)
        for (int i = 0; i < n; i++)
            if (e->cons[i].color == c) e->order[k++] = i;
    for (int i = k; i < n; i++) e->order[i] = -1;
    e->cnt[OC_CONSTRAINTS] += n;
    e->cnt[OC_COLORS] += nc;
    free(a); free(b); free(dyn); free(col);
}

/* ------------------------------------------------------------------------- */
/* constraint rows (per substep)                                              */
/* ------------------------------------------------------------------------- */
typedef struct { v3 x; qt q; m3 R; v3 v, w; double im; m3 iI; int dyn; qt q0; } BodyView;

static BodyView view(const Env* e, int i) {
    BodyView bv;
    if (i < 0) {
        bv.x = V(0, 0, 0); bv.q = Q(0, 0, 0, 1); bv.R = qmat(bv.q);
        bv.v = V(0, 0, 0); bv.w = V(0, 0, 0); bv.im = 0.0; bv.dyn = 0; bv.q0 = bv.q;
        memset(&bv.iI, 0, sizeof(bv.iI));
        return bv;
    }
    const Body* b = &e->bodies[i];
    bv.x = b->x; bv.q = b->q; bv.R = qmat(b->q); bv.v = b->v; bv.w = b->w;
    bv.im = b->inv_mass; bv.iI = b->invIw; bv.dyn = b->dyn; bv.q0 = b->q0;
    return bv;
}

static void world_inertia(Body* b) {
    memset(&b->invIw, 0, sizeof(b->invIw));
    if (!b->dyn) return;
    m3 R = qmat(b->q);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += R.m[i][k] * b->inv_I[k] * R.m[j][k];
            b->invIw.m[i][j] = s;
        }
}

static double row_k(const BodyView* A, const BodyView* B, const Row* r) {
    return (A->im + B->im) * dot(r->lin, r->lin) + dot(r->angA, mv(&A->iI, r->angA)) +
           dot(r->angB, mv(&B->iI, r->angB));
}

static void set_point_row(Row* r, v3 e, v3 rA, v3 rB) {
    r->lin = e; r->angA = cross(rA, e); r->angB = cross(e, rB);
}
static void set_ang_row(Row* r, v3 jA, v3 jB) {
    r->lin = V(0, 0, 0); r->angA = jA; r->angB = jB;
}

/* tangent basis: t1 = normalize(n x e_k), k = basis_axis(n), t2 = n x t1 */
static void tangents(v3 n, v3* t1, v3* t2) {
    int k = basis_axis(n);
    v3 c = cross(n, unit_axis(k));
    *t1 = scl(c, 1.0 / norm(c));
    *t2 = cross(n, *t1);
}

/* joint kinematics shared by prep and relax: anchors, axis and coordinate */
typedef struct { v3 wP, wC, rP, rC, a, c; double phi; qt qPw, qCw; } JointGeo;

static double wrap_pi(double x) {
    while (x > M_PI) x -= 2.0 * M_PI;
    while (x <= -M_PI) x += 2.0 * M_PI;
    return x;
}

static JointGeo joint_geo(const Joint* j, const BodyView* P, const BodyView* C) {
    JointGeo g;
    g.rP = mv(&P->R, j->fpP); g.rC = mv(&C->R, j->fpC);
    g.wP = add(P->x, g.rP); g.wC = add(C->x, g.rC);
    g.qPw = qmul(P->q, j->fqP); g.qCw = qmul(C->q, j->fqC);
    g.a = qrot(g.qPw, V(1, 0, 0));
    g.c = qrot(g.qCw, V(1, 0, 0));
    if (j->type == OR_REVOLUTE) {
        qt qrel = qmul(qconj(g.qPw), g.qCw);
        g.phi = wrap_pi(2.0 * atan2(qrel.x, qrel.w));
    } else {
        g.phi = dot(g.a, sub(g.wC, g.wP));
    }
    return g;
}

/* Contact point geometry inside a step.  The anchors keep the orientation of
 * the step start (r = R0 a) and the separation follows the bodies' motion to
 * first order in their rotation since then, theta = 2 sgn(w) vec(q q0^-1):
 *     d = n . ((x_A + r_A + theta_A x r_A) - (x_B + r_B + theta_B x r_B)),
 * the temporal-Gauss-Seidel scheme of the engine the paper builds on.  The
 * exact re-evaluation with rotating anchors lets a rolling body sink by
 * r (1 - cos theta) and be pushed back up each step, a gain of energy. */
static v3 rot_since(qt q, qt q0) {
    qt d = qmul(q, qconj(q0));
    double s = d.w >= 0.0 ? 2.0 : -2.0;
    return V(s * d.x, s * d.y, s * d.z);
}

static double contact_sep(const CPoint* p, const BodyView* A, const BodyView* B, v3* rA, v3* rB) {
    m3 RA0 = qmat(A->q0), RB0 = qmat(B->q0);
    *rA = mv(&RA0, p->aA);
    *rB = mv(&RB0, p->aB);
    v3 pa = add(add(A->x, *rA), cross(rot_since(A->q, A->q0), *rA));
    v3 pb = add(add(B->x, *rB), cross(rot_since(B->q, B->q0), *rB));
    return dot(p->n, sub(pa, pb));
}

static Soft make_soft(double hz, double zeta, double h) {
    Soft S = {0, 0.0, 1.0, 0.0};
    if (!(hz > 0.0)) return S;
    double om = 2.0 * M_PI * hz, a1 = 2.0 * zeta + h * om, a2 = h * om * a1;
    S.on = 1;
    S.bias_rate = om / a1;
    S.mass_scale = a2 / (1.0 + a2);
    S.impulse_scale = 1.0 / (1.0 + a2);
    return S;
}

/* bias of a joint equality row with error C: C / h rigid, (omega / a1) C soft */
static double eq_bias(const oracle_world* w, double C, double h) {
    return w->jsoft.on ? w->jsoft.bias_rate * C : C / h;
}

static double contact_bias(double d, double h, double vmax) {
    return d >= 0.0 ? d / h : fmax(d / h, -vmax);
}

static void prep(const oracle_world* w, Env* e, double h) {
    for (int i = 0; i < e->nb; i++) { world_inertia(&e->bodies[i]); if (e->bodies[i].dyn) e->cnt[OC_BODY_INERTIA]++; }
    for (int ci = 0; ci < e->ncons; ci++) {
        Constraint* c = &e->cons[ci];
        BodyView A = view(e, c->a), B = view(e, c->b);
        Row* R = &e->rows[c->row0];
        if (c->kind == 1) {
            Manifold* M = &e->man[c->idx];
            double mu = 0.5 * (e->bodies[M->a].mu + e->bodies[M->b].mu);
            for (int k = 0; k < M->np; k++) {
                CPoint* p = &M->p[k];
                v3 rA, rB;
                double d = contact_sep(p, &A, &B, &rA, &rB);
                v3 t1, t2;
                tangents(p->n, &t1, &t2);
                tie_basis(e, p->n);
                Row* rn = &R[k];
                rn->kind = RK_NORMAL; set_point_row(rn, p->n, rA, rB);
                rn->bias = contact_bias(d, h, w->vmax); rn->pt = k;
                /* soft normal rows: a separated point keeps its speculative
                 * bias d / h, a penetrating one takes (w / a1) d (the bias is
                 * continuous at d = 0, so softness makes no discrete decision) */
                rn->soft = w->csoft.on;
                if (rn->soft && d < 0.0) rn->bias = fmax(w->csoft.bias_rate * d, -w->vmax);
                Row* rt1 = &R[M->np + 2 * k];
                Row* rt2 = &R[M->np + 2 * k + 1];
                rt1->kind = rt2->kind = RK_FRICTION;
                set_point_row(rt1, t1, rA, rB); set_point_row(rt2, t2, rA, rB);
                rt1->bias = rt2->bias = 0.0;
                rt1->soft = rt2->soft = 0;
                rt1->partner = rt2->partner = c->row0 + k;
                rt1->mu = rt2->mu = mu;
            }
            for (int r = 0; r < c->nrows; r++) {
                R[r].a = c->a; R[r].b = c->b;
                R[r].k = row_k(&A, &B, &R[r]);
                if (R[r].kind == RK_NORMAL) R[r].mu = mu;
            }
        } else {
            Joint* j = &e->joints[c->idx];
            JointGeo g = joint_geo(j, &A, &B);
            int r = 0;
            if (j->type == OR_REVOLUTE) {
                for (int t = 0; t < 3; t++) {
                    v3 ee = unit_axis(t);
                    R[r].kind = RK_EQ; set_point_row(&R[r], ee, g.rP, g.rC);
                    R[r].bias = eq_bias(w, dot(ee, sub(g.wP, g.wC)), h); r++;
                }
                int k = basis_axis(g.a);
                tie_basis(e, g.a);
                v3 b1 = cross(g.a, unit_axis(k)); b1 = scl(b1, 1.0 / norm(b1));
                v3 b2 = cross(g.a, b1);
                v3 axc = cross(g.a, g.c);
                R[r].kind = RK_EQ; set_ang_row(&R[r], neg(b1), b1); R[r].bias = eq_bias(w, dot(b1, axc), h); r++;
                R[r].kind = RK_EQ; set_ang_row(&R[r], neg(b2), b2); R[r].bias = eq_bias(w, dot(b2, axc), h); r++;
                R[r].kind = RK_LIMIT; set_ang_row(&R[r], neg(g.a), g.a); R[r].pt = 0;
                R[r].bias = contact_bias(g.phi - j->lower, h, w->vmax); r++;
                R[r].kind = RK_LIMIT; set_ang_row(&R[r], g.a, neg(g.a)); R[r].pt = 1;
                R[r].bias = contact_bias(j->upper - g.phi, h, w->vmax); r++;
                R[r].kind = RK_DRIVE; set_ang_row(&R[r], neg(g.a), g.a);
            } else {
                int k = basis_axis(g.a);
                tie_basis(e, g.a);
                v3 b1 = cross(g.a, unit_axis(k)); b1 = scl(b1, 1.0 / norm(b1));
                v3 b2 = cross(g.a, b1);
                R[r].kind = RK_EQ; set_point_row(&R[r], b1, g.rP, g.rC);
                R[r].bias = eq_bias(w, dot(b1, sub(g.wP, g.wC)), h); r++;
                R[r].kind = RK_EQ; set_point_row(&R[r], b2, g.rP, g.rC);
                R[r].bias = eq_bias(w, dot(b2, sub(g.wP, g.wC)), h); r++;
                qt qe = qmul(g.qPw, qconj(g.qCw));
                double sg = qe.w >= 0.0 ? 1.0 : -1.0;
                v3 th = V(2.0 * sg * qe.x, 2.0 * sg * qe.y, 2.0 * sg * qe.z);
                for (int t = 0; t < 3; t++) {
                    v3 ee = unit_axis(t);
                    R[r].kind = RK_EQ; set_ang_row(&R[r], ee, neg(ee)); R[r].bias = eq_bias(w, comp(th, t), h); r++;
                }
                R[r].kind = RK_LIMIT; set_point_row(&R[r], neg(g.a), g.rP, g.rC); R[r].pt = 0;
                R[r].bias = contact_bias(g.phi - j->lower, h, w->vmax); r++;
                R[r].kind = RK_LIMIT; set_point_row(&R[r], g.a, g.rP, g.rC); R[r].pt = 1;
                R[r].bias = contact_bias(j->upper - g.phi, h, w->vmax); r++;
                R[r].kind = RK_DRIVE; set_point_row(&R[r], neg(g.a), g.rP, g.rC);
            }
            /* PD drive as an implicit spring-damper (soft constraint):
             * gamma = 1/(h (h kp + kd)), b = kp C / (h kp + kd) */
            Row* dr = &R[7];
            double den = h * j->kp + j->kd;
            double C = g.phi - j->target;
            if (den > 0.0) { dr->gamma = 1.0 / (h * den); dr->bias = j->kp * C / den; }
            else { dr->gamma = 0.0; dr->bias = 0.0; }
            for (int t = 0; t < 8; t++) {
                R[t].a = c->a; R[t].b = c->b;
                R[t].k = row_k(&A, &B, &R[t]);
                R[t].soft = R[t].kind == RK_EQ && w->jsoft.on;
            }
            if (den <= 0.0) dr->k = 0.0;  /* no drive */
        }
        e->cnt[OC_ROWS_PREP] += c->nrows;
        if (e->round32)
            for (int r = 0; r < c->nrows; r++) {
                Row* q = &R[r];
                q->lin = r32v(q->lin); q->angA = r32v(q->angA); q->angB = r32v(q->angB);
                q->k = r32(q->k); q->bias = r32(q->bias); q->gamma = r32(q->gamma); q->mu = r32(q->mu);
            }
    }
}

/* relax bias: contact normals and limits from the integrated poses */
static void relax_bias(Env* e, double h) {
    for (int ci = 0; ci < e->ncons; ci++) {
        Constraint* c = &e->cons[ci];
        BodyView A = view(e, c->a), B = view(e, c->b);
        Row* R = &e->rows[c->row0];
        if (c->kind == 1) {
            Manifold* M = &e->man[c->idx];
            for (int k = 0; k < M->np; k++) {
                v3 rA, rB;
                double d = contact_sep(&M->p[k], &A, &B, &rA, &rB);
                R[k].relax_bias = fmax(d, 0.0) / h;
            }
            for (int r = M->np; r < c->nrows; r++) R[r].relax_bias = 0.0;
        } else {
            Joint* j = &e->joints[c->idx];
            JointGeo g = joint_geo(j, &A, &B);
            for (int r = 0; r < 8; r++) R[r].relax_bias = 0.0;
            R[5].relax_bias = fmax(g.phi - j->lower, 0.0) / h;
            R[6].relax_bias = fmax(j->upper - g.phi, 0.0) / h;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* solver                                                                     */
/* ------------------------------------------------------------------------- */

static void apply_impulse(Env* e, const Row* r, double dl) {
    if (r->a >= 0 && e->bodies[r->a].dyn) {
        Body* A = &e->bodies[r->a];
        A->v = add(A->v, scl(r->lin, A->inv_mass * dl));
        A->w = add(A->w, scl(mv(&A->invIw, r->angA), dl));
    }
    if (r->b >= 0 && e->bodies[r->b].dyn) {
        Body* B = &e->bodies[r->b];
        B->v = sub(B->v, scl(r->lin, B->inv_mass * dl));
        B->w = add(B->w, scl(mv(&B->invIw, r->angB), dl));
    }
    if (e->round32) {
        if (r->a >= 0) { e->bodies[r->a].v = r32v(e->bodies[r->a].v); e->bodies[r->a].w = r32v(e->bodies[r->a].w); }
        if (r->b >= 0) { e->bodies[r->b].v = r32v(e->bodies[r->b].v); e->bodies[r->b].w = r32v(e->bodies[r->b].w); }
    }
}

static double row_jv(const Env* e, const Row* r) {
    v3 va = V(0, 0, 0), wa = V(0, 0, 0), vb = V(0, 0, 0), wb = V(0, 0, 0);
    if (r->a >= 0) { va = e->bodies[r->a].v; wa = e->bodies[r->a].w; }
    if (r->b >= 0) { vb = e->bodies[r->b].v; wb = e->bodies[r->b].w; }
    return dot(r->lin, sub(va, vb)) + dot(r->angA, wa) + dot(r->angB, wb);
}

static void solve_row(const oracle_world* w, Env* e, Row* r, int relax) {
    if (r->k <= 0.0) return;               /* inert row (no dynamic body) */
    if (relax && r->kind == RK_DRIVE) return;
    double jv = row_jv(e, r);
    double old = r->lambda, nl;
    int ndyn = (r->a >= 0 && e->bodies[r->a].dyn) + (r->b >= 0 && e->bodies[r->b].dyn);
    e->cnt[ndyn == 2 ? OC_ROW_SOLVE_2DYN : OC_ROW_SOLVE_1DYN]++;
    double bias = relax ? r->relax_bias : r->bias;
    /* soft rows in the position iterations; every row is rigid in relax */
    const Soft* S = (!relax && r->soft) ? (r->kind == RK_NORMAL ? &w->csoft : &w->jsoft) : NULL;
    switch (r->kind) {
    case RK_NORMAL:
    case RK_LIMIT:
        if (S) nl = fmax(old - S->mass_scale * (jv + bias) / r->k - S->impulse_scale * old, 0.0);
        else nl = fmax(old - (jv + bias) / r->k, 0.0);
        break;
    case RK_FRICTION: {
        double lim = r->mu * e->rows[r->partner].lambda;
        nl = clampd(old - jv / r->k, -lim, lim);
        break;
    }
    case RK_EQ:
        if (S) nl = old - S->mass_scale * (jv + bias) / r->k - S->impulse_scale * old;
        else nl = old - (jv + (relax ? 0.0 : r->bias)) / r->k;
        break;
    default: /* RK_DRIVE: dl = -(Jv + b + gamma lambda) / (1/m + gamma) */
        nl = old - (jv + r->bias + r->gamma * old) / (r->k + r->gamma);
        break;
    }
    r->lambda = e->round32 ? r32(nl) : nl;
    apply_impulse(e, r, r->lambda - old);
}

static void sweep(const oracle_world* w, Env* e, int relax) {
    for (int o = 0; o < e->ncons; o++) {
        int ci = e->order[o];
        if (ci < 0) break;
        Constraint* c = &e->cons[ci];
        for (int r = 0; r < c->nrows; r++) solve_row(w, e, &e->rows[c->row0 + r], relax);
    }
}

static void warm_start(Env* e) {
    for (int o = 0; o < e->ncons; o++) {
        int ci = e->order[o];
        if (ci < 0) break;
        Constraint* c = &e->cons[ci];
        for (int r = 0; r < c->nrows; r++) {
            Row* row = &e->rows[c->row0 + r];
            if (row->k <= 0.0) continue;
            apply_impulse(e, row, row->lambda);
            e->cnt[OC_WARM_APPLY]++;
        }
    }
}

/* symplectic Euler: x += h v; q <- normalize(q + h/2 [w,0] q) */
static void integrate(Env* e, double h) {
    for (int i = 0; i < e->nb; i++) {
        Body* b = &e->bodies[i];
        if (!b->dyn) continue;
        b->x = add(b->x, scl(b->v, h));
        qt wq = qmul(Q(b->w.x, b->w.y, b->w.z, 0.0), b->q);
        b->q = qnormalize(Q(b->q.x + 0.5 * h * wq.x, b->q.y + 0.5 * h * wq.y,
                            b->q.z + 0.5 * h * wq.z, b->q.w + 0.5 * h * wq.w));
        if (e->round32) { b->x = r32v(b->x); b->q = Q(r32(b->q.x), r32(b->q.y), r32(b->q.z), r32(b->q.w)); }
        e->cnt[OC_BODY_INTEGRATE]++;
    }
}

/* Warm start across steps (optional): joint rows keep their impulses; the
 * k-th point of a manifold takes the impulses of the k-th point of the
 * previous step's manifold of the same body pair (the manifold's point order
 * is that of the reduction; no distance test, so no new discrete decision),
 * the friction impulse kept as a world vector and projected onto the new
 * point's tangents. */
static void warm_from_cache(Env* e) {
    for (int m = 0; m < e->nman; m++) {
        Manifold* M = &e->man[m];
        Constraint* c = &e->cons[e->nj + m];
        Row* R = &e->rows[c->row0];
        /* the previous step's points of this pair, in order */
        int k = 0;
        for (int q = 0; q < e->nprev && k < M->np; q++) {
            const PrevPoint* P = &e->prev[q];
            if (P->a != M->a || P->b != M->b) continue;
            v3 t1, t2;
            tangents(M->p[k].n, &t1, &t2);
            R[k].lambda = P->ln;
            R[M->np + 2 * k].lambda = dot(P->ft, t1);
            R[M->np + 2 * k + 1].lambda = dot(P->ft, t2);
            k++;
        }
    }
}

static void store_cache(Env* e) {
    int n = 0;
    for (int m = 0; m < e->nman; m++) {
        const Manifold* M = &e->man[m];
        const Row* R = &e->rows[e->cons[e->nj + m].row0];
        for (int k = 0; k < M->np; k++) {
            PrevPoint* P = &e->prev[n++];
            const Row* f1 = &R[M->np + 2 * k];
            const Row* f2 = &R[M->np + 2 * k + 1];
            P->a = M->a; P->b = M->b; P->aA = M->p[k].aA;
            P->ln = R[k].lambda;
            P->ft = add(scl(f1->lin, f1->lambda), scl(f2->lin, f2->lambda));
        }
    }
    e->nprev = n;
}

/* Restitution (after the last substep; the rule of Box2D v3's solver): a
 * contact point whose step-start approach speed exceeds the bounce threshold
 * and that carried a normal impulse gets the normal impulse that makes its
 * normal relative velocity -e times that approach speed, accumulated impulse
 * kept >= 0.  e = average of the two bodies' restitution. */
static void restitution(const oracle_world* w, Env* e) {
    for (int o = 0; o < e->ncons; o++) {
        int ci = e->order[o];
        if (ci < 0) break;
        Constraint* c = &e->cons[ci];
        if (c->kind != 1) continue;
        Manifold* M = &e->man[c->idx];
        double ra = M->a >= 0 ? e->bodies[M->a].rest : 0.0, rb = M->b >= 0 ? e->bodies[M->b].rest : 0.0;
        double er = 0.5 * (ra + rb);
        for (int k = 0; k < M->np; k++) {
            CPoint* p = &M->p[k];
            Row* r = &e->rows[c->row0 + k];
            if (er <= 0.0 || p->vn0 > -w->bounce || p->lmax <= 0.0 || r->k <= 0.0) continue;
            double vn = row_jv(e, r);
            double old = r->lambda;
            double nl = fmax(old - (vn + er * p->vn0) / r->k, 0.0);
            r->lambda = nl;
            apply_impulse(e, r, nl - old);
        }
    }
}

static void env_step(const oracle_world* w, Env* e, const double* act, int A) {
    /* drive targets: NaN keeps the previous target */
    if (act)
        for (int j = 0; j < e->nj && j < A; j++) {
            if (isnan(act[j])) continue;
            if (w->task_on) {
                /* delta joint-position controller: clip the normalised action
                 * to [-1, 1], unnormalise by (h - l) / 2, add to the target */
                double a = fmin(fmax(act[j], -1.0), 1.0);
                e->joints[j].target += a * (j < w->t_A ? w->t_half[j] : 0.0);
            } else {
                e->joints[j].target = act[j];
            }
        }
    for (int i = 0; i < e->nb; i++) e->bodies[i].q0 = e->bodies[i].q;
    broadphase(w, e);
    narrowphase(w, e);
    build_constraints(e);
    /* impulses start at zero, or (warm start) from the previous step */
    int nj8 = 8 * e->nj;
    double jl[nj8 > 0 ? nj8 : 1];
    if (w->warm) for (int r = 0; r < nj8; r++) jl[r] = e->rows[r].lambda;
    for (int r = 0; r < e->nrows; r++) memset(&e->rows[r], 0, sizeof(Row));
    if (w->warm) {
        for (int r = 0; r < nj8; r++) e->rows[r].lambda = jl[r];
        warm_from_cache(e);
    }
    double h = w->dt / w->substeps;
    double al = 1.0 / (1.0 + h * w->lin_damp), aw = 1.0 / (1.0 + h * w->ang_damp);
    for (int s = 0; s < w->substeps; s++) {
        /* velocity damping (implicit, Box2D v3) and gravity */
        for (int i = 0; i < e->nb; i++)
            if (e->bodies[i].dyn) {
                e->bodies[i].v = add(scl(e->bodies[i].v, al), scl(w->g, h));
                e->bodies[i].w = scl(e->bodies[i].w, aw);
                if (e->round32) { e->bodies[i].v = r32v(e->bodies[i].v); e->bodies[i].w = r32v(e->bodies[i].w); }
            }
        prep(w, e, h);
        warm_start(e);
        for (int it = 0; it < w->pos_iters; it++) sweep(w, e, 0);
        integrate(e, h);
        relax_bias(e, h);
        for (int it = 0; it < w->vel_iters; it++) sweep(w, e, 1);
        for (int m = 0; m < e->nman; m++) {
            Manifold* M = &e->man[m];
            const Row* R = &e->rows[e->cons[e->nj + m].row0];
            for (int k = 0; k < M->np; k++) M->p[k].lmax = fmax(M->p[k].lmax, R[k].lambda);
        }
    }
    restitution(w, e);
    if (w->warm) store_cache(e);
    e->cnt[OC_STEPS]++;
}


/* ------------------------------------------------------------------------- */
/* pick task (Appendix "Vision-Based Sim2Real": Controller / Action Space,    */
/* Observation Space, Reward)                                                 */
/* ------------------------------------------------------------------------- */
/* joint coordinate: revolute angle or prismatic displacement (as the limits) */
static double joint_coord(const Env* e, int j) {
    const Joint* jt = &e->joints[j];
    BodyView P = view(e, jt->parent), C = view(e, jt->child);
    return joint_geo(jt, &P, &C).phi;
}

/* signed distance from body i to the table plane (its local +z through its
 * origin): the lowest point of the body along the plane normal */
static double plane_gap(const Env* e, int i, int table) {
    const Body* T = &e->bodies[table];
    const Body* B = &e->bodies[i];
    v3 n = qrot(T->q, V(0, 0, 1));
    double off = dot(n, sub(B->x, T->x));
    if (B->type == OR_SPHERE) return off - B->p[0];
    if (B->type == OR_CAPSULE) return off - fabs(dot(n, qrot(B->q, V(0, 0, 1)))) * B->p[1] - B->p[0];
    if (B->type == OR_BOX) {
        double s = 0.0;
        s += fabs(dot(n, qrot(B->q, V(1, 0, 0)))) * B->p[0];
        s += fabs(dot(n, qrot(B->q, V(0, 1, 0)))) * B->p[1];
        s += fabs(dot(n, qrot(B->q, V(0, 0, 1)))) * B->p[2];
        return off - s;
    }
    return off;
}

/* the reward's distance term: r_dist = 1 - tanh(z * distance) */
static double r_dist(double dist, double z) { return 1.0 - tanh(z * dist); }

/* One record of D = 10 + 2A values for the env's current state:
 *   reward, grasped, tcp_close, touch_table, x_tcp[3], x_cube[3],
 *   q[A] (joint coordinates; 0 past the env's joints), target[A].
 * tcp = midpoint of the two fingers' centres, g = finger b - finger a,
 * c = the cube's side (2 x its first half-extent), up = +z:
 *   r = r_dist(|tcp - x_cube|, 15) + (1 - up . g/|g|)
 *       + 2 [|tcp - x_cube| <= c/2] r_dist(| |g| - c |, 40)
 *       + [grasped] (1 + 3 r_dist(|q - q_reset|, 4/pi)) - 2 [touch_table]
 * grasped: the gripper joint is more than grasp_tol from its target (the
 * object blocks it); touch_table: a finger within touch_tol of the table.
 * Returns a mask of decisions within 1e-5 of their threshold (1 grasped,
 * 2 tcp_close, 4 touch_table). */
static unsigned task_record(const oracle_world* w, const Env* e, double* out) {
    int A = w->t_A;
    unsigned ties = 0;
    const Body* fa = &e->bodies[w->t_fa];
    const Body* fb = &e->bodies[w->t_fb];
    const Body* cu = &e->bodies[w->t_cube];
    v3 tcp = scl(add(fa->x, fb->x), 0.5);
    v3 g = sub(fb->x, fa->x);
    double gl = norm(g);
    double c = 2.0 * cu->p[0];
    double dtc = norm(sub(tcp, cu->x));
    double r = r_dist(dtc, 15.0);
    r += gl > 0.0 ? 1.0 - g.z / gl : 1.0;
    int close = dtc <= 0.5 * c;
    if (fabs(dtc - 0.5 * c) < TIE_EPS) ties |= 2u;
    if (close) r += 2.0 * r_dist(fabs(gl - c), 40.0);
    double qd2 = 0.0;
    for (int j = 0; j < A; j++) {
        double q = j < e->nj ? joint_coord(e, j) : 0.0;
        out[10 + j] = q;
        out[10 + A + j] = j < e->nj ? e->joints[j].target : 0.0;
        if (j < e->nj) qd2 += (q - e->qR[j]) * (q - e->qR[j]);
    }
    int grasped = 0;
    if (w->t_grip >= 0 && w->t_grip < e->nj) {
        double dq = fabs(out[10 + w->t_grip] - e->joints[w->t_grip].target);
        grasped = dq > w->t_grasp_tol;
        if (fabs(dq - w->t_grasp_tol) < TIE_EPS) ties |= 1u;
    }
    if (grasped) r += 1.0 + 3.0 * r_dist(sqrt(qd2), 4.0 / M_PI);
    double ga = plane_gap(e, w->t_fa, w->t_table), gb = plane_gap(e, w->t_fb, w->t_table);
    int touch = ga <= w->t_touch_tol || gb <= w->t_touch_tol;
    if (fabs(ga - w->t_touch_tol) < TIE_EPS || fabs(gb - w->t_touch_tol) < TIE_EPS) ties |= 4u;
    if (touch) r -= 2.0;
    out[0] = r; out[1] = grasped; out[2] = close; out[3] = touch;
    out[4] = tcp.x; out[5] = tcp.y; out[6] = tcp.z;
    out[7] = cu->x.x; out[8] = cu->x.y; out[9] = cu->x.z;
    return ties;
}

/* reset of the controller (after an env reset): target = q = q_reset */
static void task_reset_env(Env* e) {
    for (int j = 0; j < e->nj; j++) {
        double q = joint_coord(e, j);
        e->joints[j].target = q;
        e->qR[j] = q;
    }
}


/* ------------------------------------------------------------------------- */
/* camera rendering: RGB, depth and segmentation of every env's camera (the  */
/* paper's parallel rendering, Sec. "GPU Parallelized Simulation and          */
/* Rendering"), restated as a plain triangle rasteriser                       */
/* ------------------------------------------------------------------------- */
/* Mesh of each primitive (body frame), triangles counter-clockwise seen from
 * outside:
 *   box      6 faces x 2 triangles (corners (+-hx, +-hy, +-hz))
 *   sphere   UV sphere: rings at polar angles k pi/6 (k = 1..5), 12 points
 *            per ring at azimuths 2 pi j/12, two poles: 120 triangles
 *   capsule  the same rings, k = 1..3 shifted by +l along z and k = 3..5 by
 *            -l (the equator ring twice, bounding the cylinder): 144
 *   plane    the square [-2, 2]^2 at z = 0, normal +z: 2 triangles */
enum { R_NLON = 12, R_NLAT = 6, R_MAXTRI = 144 };
typedef struct { v3 p[3]; } Tri;

static int box_mesh(const Body* b, Tri* t) {
    static const int F[6][4][3] = {
        {{1, -1, -1}, {1, 1, -1}, {1, 1, 1}, {1, -1, 1}},
        {{-1, 1, -1}, {-1, -1, -1}, {-1, -1, 1}, {-1, 1, 1}},
        {{1, 1, -1}, {-1, 1, -1}, {-1, 1, 1}, {1, 1, 1}},
        {{-1, -1, -1}, {1, -1, -1}, {1, -1, 1}, {-1, -1, 1}},
        {{-1, -1, 1}, {1, -1, 1}, {1, 1, 1}, {-1, 1, 1}},
        {{-1, 1, -1}, {1, 1, -1}, {1, -1, -1}, {-1, -1, -1}}};
    int n = 0;
    for (int f = 0; f < 6; f++) {
        v3 c[4];
        for (int k = 0; k < 4; k++) c[k] = V(F[f][k][0] * b->p[0], F[f][k][1] * b->p[1], F[f][k][2] * b->p[2]);
        t[n].p[0] = c[0]; t[n].p[1] = c[1]; t[n].p[2] = c[2]; n++;
        t[n].p[0] = c[0]; t[n].p[1] = c[2]; t[n].p[2] = c[3]; n++;
    }
    return n;
}

/* sphere (l = 0, rings 1..5) or capsule (rings 1, 2, 3 at +l, 3, 4, 5 at -l) */
static int round_mesh(double r, double l, int capsule, Tri* t) {
    int ring_k[6], nr = 0;
    double shift[6];
    if (capsule) {
        for (int k = 1; k <= 3; k++) { ring_k[nr] = k; shift[nr] = l; nr++; }
        for (int k = 3; k <= 5; k++) { ring_k[nr] = k; shift[nr] = -l; nr++; }
    } else {
        for (int k = 1; k <= 5; k++) { ring_k[nr] = k; shift[nr] = 0.0; nr++; }
    }
    v3 ring[6][R_NLON];
    for (int a = 0; a < nr; a++) {
        double th = M_PI * ring_k[a] / R_NLAT;
        for (int j = 0; j < R_NLON; j++) {
            double ph = 2.0 * M_PI * j / R_NLON;
            ring[a][j] = V(r * sin(th) * cos(ph), r * sin(th) * sin(ph), r * cos(th) + shift[a]);
        }
    }
    v3 N = V(0, 0, r + shift[0]), S = V(0, 0, -r + shift[nr - 1]);
    int n = 0;
    for (int j = 0; j < R_NLON; j++) {
        int j1 = (j + 1) % R_NLON;
        t[n].p[0] = N; t[n].p[1] = ring[0][j]; t[n].p[2] = ring[0][j1]; n++;
    }
    for (int a = 0; a + 1 < nr; a++)
        for (int j = 0; j < R_NLON; j++) {
            int j1 = (j + 1) % R_NLON;
            t[n].p[0] = ring[a][j]; t[n].p[1] = ring[a + 1][j]; t[n].p[2] = ring[a + 1][j1]; n++;
            t[n].p[0] = ring[a][j]; t[n].p[1] = ring[a + 1][j1]; t[n].p[2] = ring[a][j1]; n++;
        }
    for (int j = 0; j < R_NLON; j++) {
        int j1 = (j + 1) % R_NLON;
        t[n].p[0] = S; t[n].p[1] = ring[nr - 1][j1]; t[n].p[2] = ring[nr - 1][j]; n++;
    }
    return n;
}

static int body_mesh(const Body* b, Tri* t) {
    if (b->type == OR_HULL) {
        const Hull* H = b->hull;
        for (int f = 0; f < H->nt; f++)
            for (int k = 0; k < 3; k++) t[f].p[k] = H->v[H->t[f][k]];
        return H->nt;
    }
    if (b->type == OR_BOX) return box_mesh(b, t);
    if (b->type == OR_SPHERE) return round_mesh(b->p[0], 0.0, 0, t);
    if (b->type == OR_CAPSULE) return round_mesh(b->p[0], b->p[1], 1, t);
    v3 c[4] = {V(-2, -2, 0), V(2, -2, 0), V(2, 2, 0), V(-2, 2, 0)};
    t[0].p[0] = c[0]; t[0].p[1] = c[1]; t[0].p[2] = c[2];
    t[1].p[0] = c[0]; t[1].p[1] = c[2]; t[1].p[2] = c[3];
    return 2;
}

typedef struct {
    v3 eye, rt, up, fw;               /* view basis: right, up, forward */
    double F, near;                   /* focal length (pixels), near plane */
    int W, H;
} Camera;

static const double R_TIE_PX = 1e-3;  /* coverage decisions within 1e-3 pixel of an edge */
static const double R_TIE_Z = 1e-5;   /* depth decisions within 1e-5 (relative) */

/* one env's image; per pixel the covering triangle of least (depth, index) */
static void render_env(const Env* e, const Camera* C, const double* rgb_body, unsigned char* rgb, double* depth,
                       int* seg, unsigned char* ties) {
    int W = C->W, H = C->H, P = W * H;
    double* zb = (double*)malloc(sizeof(double) * P);
    double* z2 = (double*)malloc(sizeof(double) * P);        /* second-nearest covering depth */
    int* win = (int*)malloc(sizeof(int) * P);
    for (int i = 0; i < P; i++) { zb[i] = INFINITY; z2[i] = INFINITY; win[i] = -1; seg[i] = 0; depth[i] = 0.0;
                                  rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0; ties[i] = 0; }
    v3 L = V(0.3, 0.2, 1.0);
    L = scl(L, 1.0 / norm(L));
    Tri mesh[R_MAXTRI];
    int tri_index = 0;
    /* shade and body of each winning triangle, by triangle index */
    int cap = 64;
    double* shade = (double*)malloc(sizeof(double) * cap);
    int* tbody = (int*)malloc(sizeof(int) * cap);
    for (int bi = 0; bi < e->nb; bi++) {
        const Body* b = &e->bodies[bi];
        int nt = body_mesh(b, mesh);
        m3 R = qmat(b->q);
        for (int ti = 0; ti < nt; ti++, tri_index++) {
            if (tri_index >= cap) {
                cap *= 2;
                shade = (double*)realloc(shade, sizeof(double) * cap);
                tbody = (int*)realloc(tbody, sizeof(int) * cap);
            }
            tbody[tri_index] = bi;
            v3 w[3], vv[3];
            for (int k = 0; k < 3; k++) {
                w[k] = add(b->x, mv(&R, mesh[ti].p[k]));
                v3 d = sub(w[k], C->eye);
                vv[k] = V(dot(C->rt, d), dot(C->up, d), dot(C->fw, d));
            }
            v3 n = cross(sub(w[1], w[0]), sub(w[2], w[0]));
            double nl = norm(n);
            shade[tri_index] = nl > 0.0 ? 0.3 + 0.7 * fmax(0.0, dot(n, L) / nl) : 0.3;
            /* back faces (facing away from the eye, or edge-on) are not drawn */
            if (dot(n, sub(w[0], C->eye)) >= 0.0) continue;
            /* clip against the near plane z >= near (view space) */
            v3 poly[4];
            int np = 0;
            for (int k = 0; k < 3; k++) {
                v3 a = vv[k], c = vv[(k + 1) % 3];
                double da = a.z - C->near, dc = c.z - C->near;
                if (da >= 0.0) poly[np++] = a;
                if ((da >= 0.0) != (dc >= 0.0)) {
                    double s = da / (da - dc);
                    poly[np++] = add(a, scl(sub(c, a), s));
                }
            }
            for (int f = 0; f + 2 < np; f++) {
                v3 q[3] = {poly[0], poly[f + 1], poly[f + 2]};
                double sx[3], sy[3], iz[3];
                for (int k = 0; k < 3; k++) {
                    sx[k] = 0.5 * W + C->F * q[k].x / q[k].z;
                    sy[k] = 0.5 * H - C->F * q[k].y / q[k].z;
                    iz[k] = 1.0 / q[k].z;
                }
                double A = (sx[1] - sx[0]) * (sy[2] - sy[0]) - (sy[1] - sy[0]) * (sx[2] - sx[0]);
                if (A == 0.0) continue;
                double sg = A > 0.0 ? 1.0 : -1.0;
                for (int py = 0; py < H; py++)
                    for (int px = 0; px < W; px++) {
                        double x = px + 0.5, y = py + 0.5;
                        double wk[3], dist_min = INFINITY;
                        for (int k = 0; k < 3; k++) {
                            int a = (k + 1) % 3, c = (k + 2) % 3;   /* edge a -> c, opposite vertex k */
                            double ex = sx[c] - sx[a], ey = sy[c] - sy[a];
                            wk[k] = sg * (ex * (y - sy[a]) - ey * (x - sx[a]));
                            double el = sqrt(ex * ex + ey * ey);
                            double dd = el > 0.0 ? wk[k] / el : wk[k];
                            if (dd < dist_min) dist_min = dd;
                        }
                        int pix = py * W + px;
                        if (fabs(dist_min) < R_TIE_PX) ties[pix] = 1;
                        if (wk[0] < 0.0 || wk[1] < 0.0 || wk[2] < 0.0) continue;
                        double sa = fabs(A);
                        double izp = (wk[0] * iz[0] + wk[1] * iz[1] + wk[2] * iz[2]) / sa;
                        double z = 1.0 / izp;
                        if (z < zb[pix] || (z == zb[pix] && tri_index < win[pix])) {
                            if (win[pix] != tri_index) z2[pix] = zb[pix];
                            zb[pix] = z; win[pix] = tri_index;
                        } else if (win[pix] != tri_index && z < z2[pix]) {
                            z2[pix] = z;
                        }
                    }
            }
        }
    }
    for (int i = 0; i < P; i++) {
        if (win[i] < 0) continue;
        if (isfinite(z2[i]) && z2[i] - zb[i] <= R_TIE_Z * zb[i]) ties[i] = 1;
        int bi = tbody[win[i]];
        seg[i] = bi + 1;
        depth[i] = zb[i];
        for (int c = 0; c < 3; c++) {
            double v = rgb_body[3 * bi + c] * shade[win[i]];
            int q = (int)floor(v * 255.0 + 0.5);
            rgb[3 * i + c] = (unsigned char)(q < 0 ? 0 : (q > 255 ? 255 : q));
        }
    }
    free(zb); free(z2); free(win); free(shade); free(tbody);
}

typedef struct {
    const oracle_world* w; const Camera* C; const double* rgb_body;
    unsigned char* rgb; double* depth; int* seg; unsigned char* ties; int e0, e1;
} RenderJob;

static void* run_render(void* p) {
    RenderJob* j = (RenderJob*)p;
    size_t P = (size_t)j->C->W * j->C->H;
    for (int ei = j->e0; ei < j->e1; ei++)
        render_env(&j->w->envs[ei], j->C, j->rgb_body + 3 * j->w->body_off[ei], j->rgb + 3 * P * ei,
                   j->depth + P * ei, j->seg + P * ei, j->ties + P * ei);
    return NULL;
}

int oracle_render(const oracle_world* w, const double* cam, const double* rgb_body, unsigned char* rgb, double* depth,
                  int* seg, unsigned char* ties, int n_threads) {
    Camera C;
    C.eye = V(cam[0], cam[1], cam[2]);
    v3 f = sub(V(cam[3], cam[4], cam[5]), C.eye);
    if (norm(f) == 0.0) return -1;
    C.fw = scl(f, 1.0 / norm(f));
    v3 r = cross(C.fw, V(0, 0, 1));
    if (norm(r) < 1e-9) return -1;
    C.rt = scl(r, 1.0 / norm(r));
    C.up = cross(C.rt, C.fw);
    C.W = (int)cam[8]; C.H = (int)cam[9];
    C.F = 0.5 * C.H / tan(0.5 * cam[6]);
    C.near = cam[7];
    if (C.W < 1 || C.H < 1 || !(C.near > 0.0) || !(cam[6] > 0.0 && cam[6] < M_PI)) return -1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > w->E) n_threads = w->E > 0 ? w->E : 1;
    RenderJob* jobs = (RenderJob*)calloc((size_t)n_threads, sizeof(RenderJob));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; t++) {
        RenderJob jb = {w, &C, rgb_body, rgb, depth, seg, ties,
                        (int)((long long)w->E * t / n_threads), (int)((long long)w->E * (t + 1) / n_threads)};
        jobs[t] = jb;
    }
    if (n_threads == 1) run_render(&jobs[0]);
    else {
        for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, run_render, &jobs[t]);
        for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    }
    free(jobs); free(th);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* world API                                                                  */
/* ------------------------------------------------------------------------- */
/* A hull asset: edges from its triangles (each once, with its two
 * triangles), bounding radius, volume and diagonal second moments of unit
 * density over the tetrahedra (origin, triangle): a tetrahedron with a
 * vertex at the origin has second moments (V/20)(a a^T + b b^T + c c^T +
 * s s^T), s = a + b + c.  Returns 0, or -1 for a mesh that is not closed. */
static int build_hull(Hull* H, const double* v, int nv, const int* t, int nt) {
    if (nv < 4 || nv > H_MAXV || nt < 4 || nt > H_MAXT) return -1;
    H->nv = nv; H->nt = nt;
    H->rad = 0.0;
    for (int k = 0; k < nv; k++) {
        H->v[k] = V(v[3 * k], v[3 * k + 1], v[3 * k + 2]);
        H->rad = fmax(H->rad, norm(H->v[k]));
    }
    for (int f = 0; f < nt; f++)
        for (int k = 0; k < 3; k++) {
            H->t[f][k] = t[3 * f + k];
            if (H->t[f][k] < 0 || H->t[f][k] >= nv) return -1;
        }
    H->ne = 0;
    for (int f = 0; f < nt; f++)
        for (int k = 0; k < 3; k++) {
            int a = H->t[f][k], b = H->t[f][(k + 1) % 3];
            if (a > b) continue;
            int g = -1;
            for (int h = 0; h < nt && g < 0; h++)
                for (int q = 0; q < 3; q++)
                    if (H->t[h][q] == b && H->t[h][(q + 1) % 3] == a) { g = h; break; }
            if (g < 0 || H->ne >= H_MAXE) return -1;
            H->e[H->ne][0] = a; H->e[H->ne][1] = b; H->ef[H->ne][0] = f; H->ef[H->ne][1] = g; H->ne++;
        }
    if (2 * H->ne != 3 * nt) return -1;
    H->vol = 0.0; H->c2 = V(0, 0, 0);
    for (int f = 0; f < nt; f++) {
        v3 a = H->v[H->t[f][0]], b = H->v[H->t[f][1]], c = H->v[H->t[f][2]];
        double v6 = dot(a, cross(b, c));
        H->vol += v6 / 6.0;
        v3 sm = add(add(a, b), c);
        double w = v6 / 120.0;
        H->c2.x += w * (a.x * a.x + b.x * b.x + c.x * c.x + sm.x * sm.x);
        H->c2.y += w * (a.y * a.y + b.y * b.y + c.y * c.y + sm.y * sm.y);
        H->c2.z += w * (a.z * a.z + b.z * b.z + c.z * c.z + sm.z * sm.z);
    }
    return H->vol > 0.0 ? 0 : -1;
}

/* inertia of a hull of the given mass about its (principal) body axes */
static void hull_inertia(const Hull* H, double mass, double* I) {
    double rho = mass / H->vol;
    I[0] = rho * (H->c2.y + H->c2.z);
    I[1] = rho * (H->c2.x + H->c2.z);
    I[2] = rho * (H->c2.x + H->c2.y);
}

int oracle_hull_inertia(const double* verts, int nv, const int* tris, int nt, double mass, double* out3) {
    Hull H;
    if (build_hull(&H, verts, nv, tris, nt) != 0) return -1;
    hull_inertia(&H, mass, out3);
    return 0;
}

oracle_world* oracle_create(int n_envs, const long long* body_off, const double* bodies,
                            const long long* joint_off, const double* joints, const double* params) {
    return oracle_create_hulls(n_envs, body_off, bodies, joint_off, joints, params, 0, NULL, NULL, NULL, NULL);
}

oracle_world* oracle_create_hulls(int n_envs, const long long* body_off, const double* bodies,
                                  const long long* joint_off, const double* joints, const double* params,
                                  int n_hulls, const int* vert_off, const double* verts, const int* tri_off,
                                  const int* tris) {
    oracle_world* w = (oracle_world*)calloc(1, sizeof(oracle_world));
    w->nh = n_hulls;
    w->hulls = (Hull*)calloc((size_t)(n_hulls > 0 ? n_hulls : 1), sizeof(Hull));
    for (int h = 0; h < n_hulls; h++)
        if (build_hull(&w->hulls[h], verts + 3 * vert_off[h], vert_off[h + 1] - vert_off[h], tris + 3 * tri_off[h],
                       tri_off[h + 1] - tri_off[h]) != 0) {
            free(w->hulls); free(w);
            return NULL;
        }
    w->E = n_envs;
    w->dt = params[0]; w->substeps = (int)params[1]; w->pos_iters = (int)params[2];
    w->vel_iters = (int)params[3]; w->g = V(params[4], params[5], params[6]);
    w->margin = params[7]; w->vmax = params[8];
    w->contact_cap = (int)params[9]; w->pair_cap = (int)params[10];
    w->lin_damp = params[11]; w->ang_damp = params[12]; w->bounce = params[13]; w->warm = (int)params[14];
    {
        /* contact softness at most a quarter of the substep rate (Box2D v3) */
        double h = w->dt / w->substeps;
        double chz = params[15] < 0.25 / h ? params[15] : 0.25 / h;
        w->csoft = make_soft(chz, params[16], h);
        w->jsoft = make_soft(params[17], params[18], h);
    }
    w->nb_total = (int)body_off[n_envs]; w->nj_total = (int)joint_off[n_envs];
    w->body_off = (long long*)malloc(sizeof(long long) * (n_envs + 1));
    w->joint_off = (long long*)malloc(sizeof(long long) * (n_envs + 1));
    memcpy(w->body_off, body_off, sizeof(long long) * (n_envs + 1));
    memcpy(w->joint_off, joint_off, sizeof(long long) * (n_envs + 1));
    w->envs = (Env*)calloc((size_t)(n_envs > 0 ? n_envs : 1), sizeof(Env));
    for (int ei = 0; ei < n_envs; ei++) {
        Env* e = &w->envs[ei];
        e->nb = (int)(body_off[ei + 1] - body_off[ei]);
        e->nj = (int)(joint_off[ei + 1] - joint_off[ei]);
        e->bodies = (Body*)calloc((size_t)(e->nb > 0 ? e->nb : 1), sizeof(Body));
        e->joints = (Joint*)calloc((size_t)(e->nj > 0 ? e->nj : 1), sizeof(Joint));
        for (int i = 0; i < e->nb; i++) {
            Body* b = &e->bodies[i];
            body_from_desc(b, bodies + 22 * (body_off[ei] + i));
            if (b->type == OR_HULL) {
                int id = (int)b->p[0];
                if (id < 0 || id >= n_hulls) id = 0;             /* the caller checks the ids */
                b->hull = &w->hulls[id];
                if (b->dyn) {
                    double I[3];
                    hull_inertia(b->hull, b->mass, I);
                    for (int k = 0; k < 3; k++) b->inv_I[k] = 1.0 / I[k];
                }
            }
        }
        for (int i = 0; i < e->nj; i++) {
            const double* d = joints + 22 * (joint_off[ei] + i);
            Joint* j = &e->joints[i];
            j->type = (int)d[0]; j->parent = (int)d[1]; j->child = (int)d[2];
            j->fpP = V(d[3], d[4], d[5]); j->fqP = qnormalize(Q(d[6], d[7], d[8], d[9]));
            j->fpC = V(d[10], d[11], d[12]); j->fqC = qnormalize(Q(d[13], d[14], d[15], d[16]));
            j->lower = d[17]; j->upper = d[18]; j->kp = d[19]; j->kd = d[20]; j->target = d[21];
        }
        int maxp = e->nb * (e->nb - 1) / 2;
        int pc = w->pair_cap < maxp ? w->pair_cap : maxp;
        e->pairs = malloc(sizeof(int[2]) * (size_t)(pc > 0 ? pc : 1));
        e->tiepairs = malloc(sizeof(int[2]) * (size_t)(maxp > 0 ? maxp : 1));
        e->man = (Manifold*)malloc(sizeof(Manifold) * (size_t)(pc > 0 ? pc : 1));
        int nc = e->nj + pc;
        e->cons = (Constraint*)malloc(sizeof(Constraint) * (size_t)(nc > 0 ? nc : 1));
        e->order = (int*)malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
        int nr = 8 * e->nj + 3 * w->contact_cap;
        e->rows = (Row*)calloc((size_t)(nr > 0 ? nr : 1), sizeof(Row));
        e->prev = (PrevPoint*)calloc((size_t)(w->contact_cap > 0 ? w->contact_cap : 1), sizeof(PrevPoint));
    }
    return w;
}

void oracle_set_round32(oracle_world* w, int on) {
    for (int e = 0; e < w->E; e++) w->envs[e].round32 = on;
}

void oracle_destroy(oracle_world* w) {
    if (!w) return;
    for (int i = 0; i < w->E; i++) {
        Env* e = &w->envs[i];
        free(e->bodies); free(e->joints); free(e->pairs); free(e->tiepairs); free(e->man);
        free(e->cons); free(e->order); free(e->rows); free(e->prev); free(e->qR);
    }
    free(w->envs); free(w->body_off); free(w->joint_off); free(w->t_half); free(w->hulls); free(w);
}

typedef struct {
    oracle_world* w; const double* act; int A, n_steps, e0, e1;
    double* out; unsigned char* ties;   /* task records [n_steps][E][D] and tie masks, or NULL */
} Job;

static void* run_job(void* p) {
    Job* j = (Job*)p;
    oracle_world* w = j->w;
    int D = 10 + 2 * w->t_A;
    for (int k = 0; k < j->n_steps; k++)
        for (int ei = j->e0; ei < j->e1; ei++) {
            env_step(w, &w->envs[ei], j->act ? j->act + ((size_t)k * w->E + ei) * j->A : NULL, j->A);
            if (j->out) {
                unsigned t = task_record(w, &w->envs[ei], j->out + ((size_t)k * w->E + ei) * D);
                if (j->ties) j->ties[(size_t)k * w->E + ei] = (unsigned char)t;
            }
        }
    return NULL;
}

static int step_jobs(oracle_world* w, const double* actions, int A, int n_steps, int n_threads, double* out,
                     unsigned char* ties) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > w->E) n_threads = w->E > 0 ? w->E : 1;
    Job* jobs = (Job*)calloc((size_t)n_threads, sizeof(Job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; t++) {
        jobs[t].w = w; jobs[t].act = actions; jobs[t].A = A; jobs[t].n_steps = n_steps;
        jobs[t].out = out; jobs[t].ties = ties;
        jobs[t].e0 = (int)((long long)w->E * t / n_threads);
        jobs[t].e1 = (int)((long long)w->E * (t + 1) / n_threads);
    }
    if (n_threads == 1) run_job(&jobs[0]);
    else {
        for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, run_job, &jobs[t]);
        for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    }
    free(jobs); free(th);
    return 0;
}

int oracle_step(oracle_world* w, const double* actions, int A, int n_steps, int n_threads) {
    return step_jobs(w, actions, A, n_steps, n_threads, NULL, NULL);
}

int oracle_step_task(oracle_world* w, const double* actions, int A, int n_steps, int n_threads, double* out,
                     unsigned char* ties) {
    if (!w->task_on) return -1;
    return step_jobs(w, actions, A, n_steps, n_threads, out, ties);
}

int oracle_set_task(oracle_world* w, const int* idx, const double* tol, int A, const double* lo, const double* hi) {
    for (int ei = 0; ei < w->E; ei++) {
        const Env* e = &w->envs[ei];
        int bodies[4] = {idx[1], idx[2], idx[3], idx[4]};
        for (int k = 0; k < 4; k++) if (bodies[k] < 0 || bodies[k] >= e->nb) return -1;
        if (idx[0] >= e->nj) return -1;
        if (e->bodies[idx[3]].type != OR_BOX || e->bodies[idx[4]].type != OR_PLANE) return -1;
    }
    w->task_on = 1;
    w->t_grip = idx[0]; w->t_fa = idx[1]; w->t_fb = idx[2]; w->t_cube = idx[3]; w->t_table = idx[4];
    w->t_grasp_tol = tol[0]; w->t_touch_tol = tol[1];
    w->t_A = A;
    free(w->t_half);
    w->t_half = (double*)calloc((size_t)(A > 0 ? A : 1), sizeof(double));
    for (int j = 0; j < A; j++) w->t_half[j] = 0.5 * (hi[j] - lo[j]);
    for (int ei = 0; ei < w->E; ei++) {
        Env* e = &w->envs[ei];
        free(e->qR);
        e->qR = (double*)calloc((size_t)(e->nj > 0 ? e->nj : 1), sizeof(double));
        task_reset_env(e);
    }
    return 0;
}

void oracle_task_reset(oracle_world* w, const unsigned char* mask) {
    if (!w->task_on) return;
    for (int ei = 0; ei < w->E; ei++)
        if (!mask || mask[ei]) task_reset_env(&w->envs[ei]);
}

int oracle_task_observe(const oracle_world* w, double* out, unsigned char* ties) {
    if (!w->task_on) return -1;
    int D = 10 + 2 * w->t_A;
    for (int ei = 0; ei < w->E; ei++) {
        unsigned t = task_record(w, &w->envs[ei], out + (size_t)ei * D);
        if (ties) ties[ei] = (unsigned char)t;
    }
    return 0;
}

void oracle_get_state(const oracle_world* w, double* out) {
    for (int ei = 0; ei < w->E; ei++) {
        const Env* e = &w->envs[ei];
        for (int i = 0; i < e->nb; i++) {
            const Body* b = &e->bodies[i];
            double* o = out + 13 * (w->body_off[ei] + i);
            o[0] = b->x.x; o[1] = b->x.y; o[2] = b->x.z;
            o[3] = b->q.x; o[4] = b->q.y; o[5] = b->q.z; o[6] = b->q.w;
            o[7] = b->v.x; o[8] = b->v.y; o[9] = b->v.z;
            o[10] = b->w.x; o[11] = b->w.y; o[12] = b->w.z;
        }
    }
}

/* Contact forces of the last step (the touch-sensor readout of the
 * dextrous-manipulation tasks): for every manifold, F = sum over its rows
 * (normal, then both friction rows of each point) of lin lambda, and
 * f_n = the sum of its normal impulses, both divided by h; body a gets +F,
 * body b -F, each gets f_n. */
void oracle_contact_forces(const oracle_world* w, double* out) {
    double h = w->dt / w->substeps;
    memset(out, 0, sizeof(double) * 4 * (size_t)w->body_off[w->E]);
    for (int ei = 0; ei < w->E; ei++) {
        const Env* e = &w->envs[ei];
        double* o = out + 4 * w->body_off[ei];
        for (int m = 0; m < e->nman; m++) {
            const Manifold* M = &e->man[m];
            const Constraint* c = &e->cons[e->nj + m];
            const Row* R = &e->rows[c->row0];
            v3 F = V(0, 0, 0);
            double fn = 0.0;
            for (int r = 0; r < c->nrows; r++) {
                F = add(F, scl(R[r].lin, R[r].lambda));
                if (R[r].kind == RK_NORMAL) fn += R[r].lambda;
            }
            F = scl(F, 1.0 / h);
            fn /= h;
            double* a = o + 4 * M->a;
            double* b = o + 4 * M->b;
            a[0] += F.x; a[1] += F.y; a[2] += F.z; a[3] += fn;
            b[0] -= F.x; b[1] -= F.y; b[2] -= F.z; b[3] += fn;
        }
    }
}

void oracle_set_state(oracle_world* w, const double* in) {
    for (int ei = 0; ei < w->E; ei++) {
        Env* e = &w->envs[ei];
        for (int i = 0; i < e->nb; i++) {
            Body* b = &e->bodies[i];
            const double* o = in + 13 * (w->body_off[ei] + i);
            b->x = V(o[0], o[1], o[2]);
            b->q = Q(o[3], o[4], o[5], o[6]);
            b->q0 = b->q;
            if (b->dyn) { b->v = V(o[7], o[8], o[9]); b->w = V(o[10], o[11], o[12]); }
        }
        /* a set state starts without warm-start memory */
        e->nprev = 0;
        for (int r = 0; r < 8 * e->nj; r++) e->rows[r].lambda = 0.0;
    }
}

void oracle_get_targets(const oracle_world* w, double* out) {
    for (int ei = 0; ei < w->E; ei++) {
        const Env* e = &w->envs[ei];
        for (int j = 0; j < e->nj; j++) out[w->joint_off[ei] + j] = e->joints[j].target;
    }
}

void oracle_set_targets(oracle_world* w, const double* in) {
    for (int ei = 0; ei < w->E; ei++) {
        Env* e = &w->envs[ei];
        for (int j = 0; j < e->nj; j++) e->joints[j].target = in[w->joint_off[ei] + j];
    }
}

unsigned oracle_env_status(const oracle_world* w, int env) { return w->envs[env].status; }
long long oracle_env_ties(const oracle_world* w, int env) { return w->envs[env].ties; }

void oracle_counters(const oracle_world* w, long long* out) {
    for (int k = 0; k < OC_NUM; k++) out[k] = 0;
    for (int ei = 0; ei < w->E; ei++)
        for (int k = 0; k < OC_NUM; k++) out[k] += w->envs[ei].cnt[k];
}

int oracle_get_manifolds(const oracle_world* w, int env, int cap, int* pairs, int* npts, double* pts) {
    const Env* e = &w->envs[env];
    for (int m = 0; m < e->nman && m < cap; m++) {
        const Manifold* M = &e->man[m];
        pairs[2 * m] = M->a; pairs[2 * m + 1] = M->b; npts[m] = M->np;
        for (int k = 0; k < 4; k++) {
            double* o = pts + (size_t)40 * m + 10 * k;
            if (k >= M->np) { memset(o, 0, sizeof(double) * 10); continue; }
            const CPoint* c = &M->p[k];
            o[0] = c->cA.x; o[1] = c->cA.y; o[2] = c->cA.z;
            o[3] = c->cB.x; o[4] = c->cB.y; o[5] = c->cB.z;
            o[6] = c->n.x; o[7] = c->n.y; o[8] = c->n.z; o[9] = c->d;
        }
    }
    return e->nman;
}

int oracle_get_margin_ties(const oracle_world* w, int env, int cap, int* pairs) {
    const Env* e = &w->envs[env];
    for (int i = 0; i < e->ntie && i < cap; i++) { pairs[2 * i] = e->tiepairs[i][0]; pairs[2 * i + 1] = e->tiepairs[i][1]; }
    return e->ntie;
}

int oracle_get_colors(const oracle_world* w, int env, int cap, int* colors) {
    const Env* e = &w->envs[env];
    for (int i = 0; i < e->ncons && i < cap; i++) colors[i] = e->cons[i].color;
    return e->ncons;
}

int oracle_get_rows(const oracle_world* w, int env, int cap, double* out) {
    const Env* e = &w->envs[env];
    for (int r = 0; r < e->nrows && r < cap; r++) {
        const Row* R = &e->rows[r];
        double* o = out + 16 * r;
        o[0] = R->a; o[1] = R->b; o[2] = R->kind;
        o[3] = R->lin.x; o[4] = R->lin.y; o[5] = R->lin.z;
        o[6] = R->angA.x; o[7] = R->angA.y; o[8] = R->angA.z;
        o[9] = R->angB.x; o[10] = R->angB.y; o[11] = R->angB.z;
        o[12] = R->k; o[13] = R->bias; o[14] = R->lambda; o[15] = R->mu;
    }
    return e->nrows;
}

static void put_cand(double* o, const Cand* c) {
    o[0] = c->cA.x; o[1] = c->cA.y; o[2] = c->cA.z;
    o[3] = c->cB.x; o[4] = c->cB.y; o[5] = c->cB.z;
    o[6] = c->n.x; o[7] = c->n.y; o[8] = c->n.z; o[9] = c->d;
}

int oracle_candidates(const double* da, const double* db, double margin, double* out) {
    Env e; memset(&e, 0, sizeof(e));
    Body A, B;
    body_from_desc(&A, da); body_from_desc(&B, db);
    Shape SA = shape_of(&A), SB = shape_of(&B);
    CandSet cs;
    candidates(&e, &SA, &SB, margin, &cs);
    for (int k = 0; k < cs.n; k++) put_cand(out + 10 * k, &cs.c[k]);
    return cs.n;
}

int oracle_reduce4(int n, const double* pts, int* sel) {
    if (n < 5 || n > 16) return -1;
    Env e; memset(&e, 0, sizeof(e));
    Cand c[16];
    for (int k = 0; k < n; k++) {
        const double* p = pts + 10 * k;
        c[k].cA = V(p[0], p[1], p[2]); c[k].cB = V(p[3], p[4], p[5]);
        c[k].n = V(p[6], p[7], p[8]); c[k].d = p[9];
    }
    return reduce4(&e, c, n, sel);
}

void oracle_tangents(const double* n, double* t1, double* t2) {
    v3 a, b;
    tangents(V(n[0], n[1], n[2]), &a, &b);
    t1[0] = a.x; t1[1] = a.y; t1[2] = a.z;
    t2[0] = b.x; t2[1] = b.y; t2[2] = b.z;
}

int oracle_collide(const double* da, const double* db, double margin, double* out) {
    Env e; memset(&e, 0, sizeof(e));
    Body A, B;
    body_from_desc(&A, da); body_from_desc(&B, db);
    Shape SA = shape_of(&A), SB = shape_of(&B);
    Cand pts[4]; int mt;
    int n = collide(&e, &SA, &SB, margin, pts, &mt);
    for (int k = 0; k < n; k++) {
        double* o = out + 10 * k;
        o[0] = pts[k].cA.x; o[1] = pts[k].cA.y; o[2] = pts[k].cA.z;
        o[3] = pts[k].cB.x; o[4] = pts[k].cB.y; o[5] = pts[k].cB.z;
        o[6] = pts[k].n.x; o[7] = pts[k].n.y; o[8] = pts[k].n.z; o[9] = pts[k].d;
    }
    return n;
}
