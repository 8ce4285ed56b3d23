// Stages of the batched rigid-body step, written once over an "env view"
// (pointers to one env's bodies, joints and workspace) and a lane group of
// G lanes (G = 1..32) that owns the env.  A warp runs 32 / G envs in
// lockstep: every loop bound below is the maximum over the warp, so all
// lanes execute the same instruction stream and the warp-wide intrinsics
// (__syncwarp, ballot, shuffles) always see the full warp.  Inactive or
// frozen envs take part with zero counts.
//
// The plain path calls each stage from its own kernel (G = 32, one env per
// warp, workspace in global memory); the batched path calls all of them from
// one persistent kernel (bodies, joints, colour lists and impulses in
// shared memory).  Both run this code, so they agree bit for bit.
//
// Per step: drive targets <- actions; broadphase; narrowphase; colouring
// (once per step, at the step-start poses).  Per substep: gravity + the
// square root of each body's world inverse inertia + rows; warm start;
// pos_iters sweeps; integration + relax bias; vel_iters relax sweeps;
// angular velocities back to world space.  The solver is substepped sequential impulses
// (Catto 2005) in the small-steps arrangement of Macklin et al. 2019, with
// PD drives as soft constraints (Catto 2011), a per-row Coulomb pyramid and
// a relax pass without penetration push.
#pragma once
#include "ms_internal.h"
#include "ms_narrow.cuh"

namespace ms {

using Params = DevParams;

enum { RK_NORMAL = 0, RK_FRICTION = 1, RK_EQ = 2, RK_LIMIT = 3, RK_DRIVE = 4 };
enum { ST_PAIR = 1u, ST_CONTACT = 2u, ST_COLOR = 4u, ST_NAN = 8u };
enum { C_NPAIRS = 0, C_NMAN = 1, C_NPTS = 2, C_NCONS = 3, C_NCOLORS = 4, C_NUM = 8 };
enum { MAX_COLORS = 64 };
#define FULL_MASK 0xffffffffu

// Between the prep of a substep and its end, a dynamic body's angular
// velocity is kept as w^ = S^-1 w, S = (world inverse inertia)^(1/2) =
// R diag(1/I)^(1/2) R^T, and every angular Jacobian a of a row as S a.  Then
// a . w = (S a) . w^, the impulse response I^-1 a dl becomes S (S a) dl =
// S . (change of w^) with w^ += (S a) dl, and a . I^-1 a = |S a|^2: a row
// solve needs no matrix product.  Static bodies keep S = identity and w^ = w:
// their velocity enters Jv, and no impulse is applied to them.
//
// One constraint row, 48 B, read-only during the sweeps:
//   a = lin, 1/k (1/(k + gamma) for a drive; 0 = inert row)
//   b = S_A angA, bias (friction rows: mu; their bias is 0)
//   c = S_B angB, relax bias (drive row: gamma; other joint rows: 0)
// A row's kind follows from its place in its constraint: joint rows 0-4 are
// equalities, 5 and 6 the lower and upper limit, 7 the drive; a manifold of
// np points has np normal rows, then a pair of friction rows per point.
// The accumulated impulse lambda of each row lives in a separate array.
struct Row {
    float4 a, b, c;
};

// Constraint record (cons, scons): a, b, first row, place | np << 2 | idx << 8
// with place: joint rows, or a manifold's rows in the shared or global part.
// A joint's rows are interleaved with the other joints' (stride njs: the
// lanes solving different joints of a colour read different banks); its
// "first row" is the joint index.  A manifold's rows are contiguous.
enum { CP_JOINT = 0, CP_MAN_S = 1, CP_MAN_G = 2 };

struct EnvView {
    int nb, nj;                       // counts the stages see (0: inactive or frozen)
    float4 *x, *q, *v, *w;            // state; v.w = inverse mass (0 = static); w holds w^ during a substep
    const float4* shape;              // p0, p1, p2, mu
    const float4* inv;                // sqrt(1/Ixx), sqrt(1/Iyy), sqrt(1/Izz), 1/m (0 = static)
    const int2* meta;                 // x: type | dyn << 8; y: group | mask << 16
    const unsigned long long* adj;    // joint adjacency bit mask per body
    const float4* jf;                 // 4 per joint: parent pos, parent quat, child pos, child quat
    const float4* jp;                 // lower, upper, kp, kd
    const int4* jm;                   // type, parent, child, -
    float* jt;                        // drive targets
    float* qR;                        // pick task: joint coordinates at the controller reset (nullable)
    const HullLib* hulls;             // hull library of the batch (nullable)
    const float* rest;                // restitution per body
    float4* wc;                       // warm-start memory of the env (null: off): 2 per contact point
    int* wc_n;                        //   its count
    float* wjl;                       //   8 impulses per joint
    float4* sq;                       // per body, 3 float4: S = (xx, xy, xz, yy), (yz, zz, -, -); q at the step start
    float4* aabb;                     // 2 per body
    int* pairs;                       // i | j << 16
    int4* man;                        // a, b, npts, first point
    float4* pts;                      // 3 per point: (aA, d), (aB, step-start approach speed), (n, max normal impulse)
    int4* cons;                       // constraint records in list order
    int* colr;                        // colour per constraint
    int4* scons;                      // the same records sorted by colour (solve order)
    int* color_off;                   // MAX_COLORS + 1
    unsigned long long* used;         // colour masks per body
    Row* rows_j;                      // 8 per joint, row r of joint j at r * njs + j
    int njs;                          // joint row stride; joint impulses are laid out the same way
    Row* rows_cs;                     // 3 per contact point < pts_s
    Row* rows_cg;                     // 3 per contact point (points >= pts_s)
    int pts_s;
    float* lam;                       // accumulated impulse per row: joints, then contact points
    int* cnt;                         // C_NUM counters
    unsigned* status;                 // env status word
    int4* rec_man;                    // recorded manifolds (nullable)
    float* rec_pts;                   // recorded points [contact_cap][10]
    int* rec_cnt;
    int* rec_col;                     // recorded colour per constraint (nullable)
    float4* force;                    // contact force per body (nullable)
};

// Workspace pointers of one env from its layout (s: shared part, gl: global part).
template <typename T>
MSD T* at(char* base, int off) { return reinterpret_cast<T*>(base + off); }

MSD void view_workspace(EnvView& e, char* s, char* gl, const Layout& L) {
    e.sq = at<float4>(s, L.sq);
    char* lb = L.lists_shared ? s : gl;
    e.scons = at<int4>(lb, L.scons);
    e.lam = at<float>(lb, L.lam);
    e.color_off = at<int>(s, L.color_off);
    e.cnt = at<int>(s, L.cnt);
    e.rows_j = at<Row>(L.rows_j_shared ? s : gl, L.rows_j);
    e.njs = L.njs;
    e.pts_s = L.pts_s;
    e.rows_cs = L.rows_cs >= 0 ? at<Row>(s, L.rows_cs) : nullptr;
    e.rows_cg = L.rows_cg >= 0 ? at<Row>(gl, L.rows_cg) : nullptr;
    e.aabb = at<float4>(gl, L.aabb);
    e.pairs = at<int>(gl, L.pairs);
    e.man = at<int4>(gl, L.man);
    e.pts = at<float4>(gl, L.pts);
    char* cb = L.color_shared ? s : gl;
    e.cons = at<int4>(cb, L.cons);
    e.colr = at<int>(cb, L.colr);
    e.used = at<unsigned long long>(cb, L.used);
}

// G lanes of a warp owning one env; all intrinsics use the full warp.
struct Grp {
    int lane, size, base;
    MSD void sync() const { __syncwarp(); }
    MSD unsigned ballot(bool p) const {
        unsigned b = __ballot_sync(FULL_MASK, p);
        return size == 32 ? b : (b >> base) & ((1u << size) - 1u);
    }
    MSD unsigned lt() const { return (1u << lane) - 1u; }
    MSD int shfl(int v, int src) const { return __shfl_sync(FULL_MASK, v, src, size); }
    MSD int wmax(int v) const { return __reduce_max_sync(FULL_MASK, v); }
    MSD int incl_scan(int v) const {
        for (int d = 1; d < size; d <<= 1) {
            int t = __shfl_up_sync(FULL_MASK, v, d, size);
            if (lane >= d) v += t;
        }
        return v;
    }
    MSD int max_all(int v) const {
        for (int d = size >> 1; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(FULL_MASK, v, d, size));
        return v;
    }
    MSD bool any(bool p) const { return ballot(p) != 0u; }
};

MSD bool is_dyn(const EnvView& e, int i) { return i >= 0 && ((e.meta[i].x >> 8) & 1); }
MSD int shape_type(const EnvView& e, int i) { return e.meta[i].x & 0xff; }

// ---------------------------------------------------------------- actions
// An action is the joint's new drive target, or, with the pick task's delta
// controller (half != null), a normalised delta: the target moves by
// clip(a, -1, 1) (h - l) / 2.  NaN leaves the target unchanged.
MSD void stage_actions(EnvView& e, const Grp& g, const float* act, int A, const float* half) {
    int n = act ? min(e.nj, A) : 0;
    int nmax = g.wmax(n);
    for (int j0 = 0; j0 < nmax; j0 += g.size) {
        int j = j0 + g.lane;
        if (j < n) {
            float t = act[j];
            if (!isnan(t)) e.jt[j] = half ? fmaf(fminf(fmaxf(t, -1.f), 1.f), half[j], e.jt[j]) : t;
        }
    }
    g.sync();
}

// ------------------------------------------------------------- broadphase
MSD void aabb_of(const EnvView& e, int i, float hm, float4& lo, float4& hi) {
    float4 s = e.shape[i];
    int t = shape_type(e, i);
    float3 c = xyz(e.x[i]);
    float3 ext;
    if (t == SH_SPHERE) {
        ext = f3(s.x, s.x, s.x);
    } else {
        M3 R = qmat(e.q[i]);
        if (t == SH_BOX) {
            ext = f3(fmaf(fabsf(R.m[2]), s.z, fmaf(fabsf(R.m[1]), s.y, fabsf(R.m[0]) * s.x)),
                     fmaf(fabsf(R.m[5]), s.z, fmaf(fabsf(R.m[4]), s.y, fabsf(R.m[3]) * s.x)),
                     fmaf(fabsf(R.m[8]), s.z, fmaf(fabsf(R.m[7]), s.y, fabsf(R.m[6]) * s.x)));
        } else if (t == SH_HULL) {
            // the bounding sphere of the hull's vertices about the body origin
            float r = e.hulls ? e.hulls->rad[(int)s.x] : 0.f;
            ext = f3(r, r, r);
        } else {
            float3 ax = mcol(R, 2);
            ext = f3(fmaf(fabsf(ax.x), s.y, s.x), fmaf(fabsf(ax.y), s.y, s.x), fmaf(fabsf(ax.z), s.y, s.x));
        }
    }
    ext = ext + f3(hm, hm, hm);
    lo = f4(c - ext, 0.f);
    hi = f4(c + ext, 0.f);
}

// p-th pair (i < j) in lexicographic order of n items
MSD void pair_from_index(int p, int n, int& i, int& j) {
    float b = 2.f * n - 1.f;
    int ii = (int)floorf((b - sqrtf(fmaxf(b * b - 8.f * p, 0.f))) * 0.5f);
    if (ii < 0) ii = 0;
    if (ii > n - 2) ii = n - 2;
    while (ii > 0 && ii * (2 * n - ii - 1) / 2 > p) ii--;
    while (ii < n - 2 && (ii + 1) * (2 * n - ii - 2) / 2 <= p) ii++;
    i = ii;
    j = p - ii * (2 * n - ii - 1) / 2 + ii + 1;
}

MSD void stage_broadphase(EnvView& e, const Grp& g, const Params& P) {
    int nb = e.nb;
    int nbmax = g.wmax(nb);
    for (int i0 = 0; i0 < nbmax; i0 += g.size) {
        int i = i0 + g.lane;
        if (i < nb && shape_type(e, i) != SH_PLANE) {
            float4 lo, hi;
            aabb_of(e, i, 0.5f * P.margin, lo, hi);
            e.aabb[2 * i] = lo;
            e.aabb[2 * i + 1] = hi;
        }
    }
    g.sync();
    int total = nb * (nb - 1) / 2;
    int tmax = g.wmax(total);
    int count = 0;
    for (int c = 0; c < tmax; c += g.size) {
        int p = c + g.lane;
        bool pred = false;
        int i = 0, j = 0;
        if (p < total) {
            pair_from_index(p, nb, i, j);
            int2 mi = e.meta[i], mj = e.meta[j];
            bool di = (mi.x >> 8) & 1, dj = (mj.x >> 8) & 1;
            unsigned gi = mi.y & 0xffff, ki = (unsigned)mi.y >> 16;
            unsigned gj = mj.y & 0xffff, kj = (unsigned)mj.y >> 16;
            pred = (di || dj) && (gi & kj) && (gj & ki) && !((e.adj[i] >> j) & 1ull);
            if (pred && (mi.x & 0xff) != SH_PLANE && (mj.x & 0xff) != SH_PLANE) {
                float4 la = e.aabb[2 * i], ha = e.aabb[2 * i + 1];
                float4 lb = e.aabb[2 * j], hb = e.aabb[2 * j + 1];
                pred = la.x <= hb.x && lb.x <= ha.x && la.y <= hb.y && lb.y <= ha.y &&
                       la.z <= hb.z && lb.z <= ha.z;
            }
        }
        unsigned bits = g.ballot(pred);
        if (pred) {
            int pos = count + __popc(bits & g.lt());
            if (pos < P.pair_cap) e.pairs[pos] = i | (j << 16);
        }
        count += __popc(bits);
    }
    if (g.lane == 0 && e.nb > 0) {
        e.cnt[C_NPAIRS] = min(count, P.pair_cap);
        if (count > P.pair_cap) *e.status |= ST_PAIR;
    }
    g.sync();
}

// ------------------------------------------------------------ narrowphase
template <bool HULLS = true>
MSD Shape shape_at(const EnvView& e, int i) {
    Shape s;
    s.x = xyz(e.x[i]);
    s.R = qmat(e.q[i]);
    s.type = shape_type(e, i);
    float4 p = e.shape[i];
    s.p0 = p.x; s.p1 = p.y; s.p2 = p.z;
    s.hull = HullRef{nullptr, nullptr, nullptr, nullptr, 0, 0, 0};
    if (HULLS && s.type == SH_HULL && e.hulls) {
        const HullLib& L = *e.hulls;
        int h = (int)p.x;
        int v0 = L.vo[h], t0 = L.to[h], e0 = L.eo[h];
        s.hull = HullRef{L.v + v0, L.t + t0, L.n + t0, L.e + e0, L.vo[h + 1] - v0, L.to[h + 1] - t0, L.eo[h + 1] - e0};
    }
    return s;
}

#ifdef MS_DEBUG_BOUNDS
// Debug builds (-DMS_DEBUG_BOUNDS): the invariants that every later stage
// indexes by, checked after the narrowphase (pair, manifold and point counts
// within their capacities; manifold bodies and point ranges in range) and
// after the colouring (colour and constraint counts; each colour-ordered
// record's bodies, joint or manifold index and row range).  An env that
// breaks one gets MS_ENV_BOUNDS and its counts are cleared, so no later stage
// reads past a buffer; nothing traps.  Every lane of the warp runs it.
MSD void stage_check_bounds(EnvView& e, const Grp& g, const Params& P, bool after_color) {
    bool live = e.nb > 0;
    int nb = e.nb, nj = e.nj;
    int npairs = live ? e.cnt[C_NPAIRS] : 0, nman = live ? e.cnt[C_NMAN] : 0, npts = live ? e.cnt[C_NPTS] : 0;
    bool bad = live && (npairs < 0 || npairs > P.pair_cap || nman < 0 || nman > P.pair_cap || npts < 0 ||
                        npts > P.contact_cap);
    int nm = bad ? 0 : nman;
    int mmax = g.wmax(nm);
    for (int m0 = 0; m0 < mmax; m0 += g.size) {
        int m = m0 + g.lane;
        if (m >= nm) continue;
        int4 M = e.man[m];
        bad |= M.x < 0 || M.x >= nb || M.y < 0 || M.y >= nb || M.z < 1 || M.z > 4 || M.w < 0 ||
               M.w + M.z > npts;
    }
    if (after_color && live) {
        int ncol = e.cnt[C_NCOLORS], ncons = e.cnt[C_NCONS];
        bad |= ncol < 0 || ncol > MAX_COLORS || ncons < 0 || ncons > nj + nman;
        bad |= ncol >= 0 && ncol <= MAX_COLORS && (e.color_off[0] != 0 || e.color_off[ncol] != ncons);
    }
    int nc = (after_color && live && !bad) ? e.cnt[C_NCONS] : 0;
    int cmax = g.wmax(nc);
    for (int k0 = 0; k0 < cmax; k0 += g.size) {
        int k = k0 + g.lane;
        if (k >= nc) continue;
        int4 c = e.scons[k];
        int place = c.w & 3, idx = c.w >> 8, np = (c.w >> 2) & 7;
        bad |= c.x < -1 || c.x >= nb || c.y < -1 || c.y >= nb;
        if (place == CP_JOINT) {
            bad |= idx < 0 || idx >= nj || c.z != idx;
        } else {
            bad |= place == 3 || idx < 0 || idx >= nman || np < 1 || np > 4 || c.z < 0 || c.z % 3 != 0 ||
                   c.z / 3 + np > npts || (place == CP_MAN_S && c.z / 3 + np > e.pts_s);
        }
    }
    bool any = g.any(bad);
    if (g.lane == 0 && any) {
        *e.status |= (unsigned)MS_ENV_BOUNDS;
        e.cnt[C_NPAIRS] = 0; e.cnt[C_NMAN] = 0; e.cnt[C_NPTS] = 0;
        e.cnt[C_NCONS] = 0; e.cnt[C_NCOLORS] = 0;
        e.color_off[0] = 0;
    }
    g.sync();
}
#define MS_CHECK_BOUNDS(e, g, P, after_color) stage_check_bounds(e, g, P, after_color)
#else
#define MS_CHECK_BOUNDS(e, g, P, after_color) ((void)0)
#endif

// HULLS = false: a batch without hulls (the hull routines compiled out)
template <bool HULLS = true>
MSD void stage_narrowphase(EnvView& e, const Grp& g, const Params& P) {
    int npairs = e.nb > 0 ? e.cnt[C_NPAIRS] : 0;
    int pmax = g.wmax(npairs);
    int total = 0, nman = 0, kept_end = 0;
    bool overflow = false;
    for (int c = 0; c < pmax; c += g.size) {
        int p = c + g.lane;
        Cand pts[4];
        int n = 0, a = 0, b = 0;
        Shape SA, SB;
        if (p < npairs) {
            int pr = e.pairs[p];
            int i = pr & 0xffff, j = pr >> 16;
            a = i; b = j;
            if (shape_rank(shape_type(e, j)) < shape_rank(shape_type(e, i))) { a = j; b = i; }
            SA = shape_at<HULLS>(e, a);
            SB = shape_at<HULLS>(e, b);
            n = collide<HULLS>(SA, SB, P.margin, pts);
        }
        int incl = g.incl_scan(n);
        int chunk_total = g.shfl(incl, g.size - 1);
        int start = total + incl - n;
        bool keep = n > 0 && start + n <= P.contact_cap;
        overflow |= (n > 0 && !keep);
        unsigned bits = g.ballot(keep);
        if (keep) {
            int midx = nman + __popc(bits & g.lt());
            e.man[midx] = make_int4(a, b, n, start);
            float3 vA = xyz(e.v[a]), wA = xyz(e.w[a]), vB = xyz(e.v[b]), wB = xyz(e.w[b]);
            for (int k = 0; k < n; k++) {
                float3 aA = mtv(SA.R, pts[k].cA - SA.x);
                float3 aB = mtv(SB.R, pts[k].cB - SB.x);
                // approach speed along n at the step-start velocities (restitution)
                float3 uA = vA + cross(wA, pts[k].cA - SA.x), uB = vB + cross(wB, pts[k].cB - SB.x);
                float4* o = e.pts + 3 * (start + k);
                o[0] = f4(aA, pts[k].d);
                o[1] = f4(aB, dot(pts[k].n, uA - uB));
                o[2] = f4(pts[k].n, 0.f);
                if (e.rec_pts) {
                    float* rp = e.rec_pts + 10 * (start + k);
                    rp[0] = pts[k].cA.x; rp[1] = pts[k].cA.y; rp[2] = pts[k].cA.z;
                    rp[3] = pts[k].cB.x; rp[4] = pts[k].cB.y; rp[5] = pts[k].cB.z;
                    rp[6] = pts[k].n.x; rp[7] = pts[k].n.y; rp[8] = pts[k].n.z; rp[9] = pts[k].d;
                }
            }
            if (e.rec_man) e.rec_man[midx] = make_int4(a, b, n, start);
        }
        kept_end = max(kept_end, g.max_all(keep ? start + n : 0));
        nman += __popc(bits);
        total += chunk_total;
    }
    bool ov = g.any(overflow);
    if (g.lane == 0 && e.nb > 0) {
        e.cnt[C_NMAN] = nman;
        e.cnt[C_NPTS] = kept_end;
        if (ov) *e.status |= ST_CONTACT;
        if (e.rec_cnt) *e.rec_cnt = nman;
    }
    g.sync();
    MS_CHECK_BOUNDS(e, g, P, false);
}

// ------------------------------------------------- dynamic row placement
// The batched kernel's placement when slots sized for the capacities do not
// fit on chip.  The envs of a warp share one shared-memory arena, handed out
// after each step's narrowphase by what the envs hold in that step: first
// the colour-ordered list and the impulses of every env (in env order), then
// the joint rows, then the contact rows, levelled so that every env keeps
// the rows of the same number of points on chip, or all of its own.  What
// does not fit stays in the env's global slot, laid out for the capacities.
// The colouring scratch goes over an env's on-chip rows when they are large
// enough (the rows are written after the colouring).  Every lane computes
// the same placement from the counts of all envs of the warp, so the loops
// and shuffles are warp-uniform.
MSD int pad16(int b) { return (b + 15) & ~15; }

MSD void place_dynamic(EnvView& e, const Grp& g, char* arena, int abytes, char* gl, const Layout& L) {
    e.scons = at<int4>(gl, L.scons);
    e.lam = at<float>(gl, L.lam);
    e.rows_j = at<Row>(gl, L.rows_j);
    e.rows_cs = nullptr;
    e.pts_s = 0;
    e.cons = at<int4>(gl, L.cons);
    e.colr = at<int>(gl, L.colr);
    e.used = at<unsigned long long>(gl, L.used);
    bool live = e.nb > 0;
    int ncons = live ? e.nj + e.cnt[C_NMAN] : 0;
    int npts = live ? e.cnt[C_NPTS] : 0;
    int blist = pad16(16 * ncons), blam = pad16(4 * (8 * e.njs + 3 * npts));
    int bl = live ? blist + blam : 0;
    int bj = live && e.nj > 0 ? (int)sizeof(Row) * 8 * e.njs : 0;
    const int BP = 3 * (int)sizeof(Row);                // the rows of one contact point
    const int K = 32 / g.size;
    int A = abytes;
    unsigned inl = 0u, inj = 0u;
    for (int k = 0; k < K; k++) {
        int b = __shfl_sync(FULL_MASK, bl, k * g.size);
        if (b > 0 && b <= A) { A -= b; inl |= 1u << k; }
    }
    for (int k = 0; k < K; k++) {
        int b = __shfl_sync(FULL_MASK, bj, k * g.size);
        if (b > 0 && b <= A) { A -= b; inj |= 1u << k; }
    }
    // the level: the most points per env whose rows, summed over the envs
    // (each env at most its own count), fit in what is left
    int lo = 0, hi = g.wmax(npts);
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int n = 0;
        for (int k = 0; k < K; k++) n += min(__shfl_sync(FULL_MASK, npts, k * g.size), mid);
        if (n <= A / BP) lo = mid;
        else hi = mid - 1;
    }
    // this env's region starts after those of the envs before it
    int gi = g.base / g.size, start = 0;
    for (int k = 0; k < K; k++) {
        int src = k * g.size;
        int b0 = __shfl_sync(FULL_MASK, bl, src), b1 = __shfl_sync(FULL_MASK, bj, src);
        int p = __shfl_sync(FULL_MASK, npts, src);
        int sz = (((inl >> k) & 1u) ? b0 : 0) + (((inj >> k) & 1u) ? b1 : 0) + BP * min(p, lo);
        if (k < gi) start += sz;
    }
    char* p = arena + start;
    if ((inl >> gi) & 1u) {
        e.scons = reinterpret_cast<int4*>(p);
        e.lam = reinterpret_cast<float*>(p + blist);
        p += bl;
    }
    char* r0 = p;
    if ((inj >> gi) & 1u) {
        e.rows_j = reinterpret_cast<Row*>(p);
        p += bj;
    }
    int ps = min(npts, lo);
    if (ps > 0) {
        e.rows_cs = reinterpret_cast<Row*>(p);
        e.pts_s = ps;
        p += BP * ps;
    }
    int bcol = pad16(4 * ncons);
    if (live && (int)(p - r0) >= blist + bcol + 8 * e.nb) {
        e.cons = reinterpret_cast<int4*>(r0);
        e.colr = reinterpret_cast<int*>(r0 + blist);
        e.used = reinterpret_cast<unsigned long long*>(r0 + blist + bcol);
    }
}

// -------------------------------------------------------------- colouring
// Constraint list = joints (index order) then manifolds (pair order).  Each
// takes the lowest colour free on both of its dynamic bodies (static bodies
// impose nothing); the solve order lists constraints colour by colour, in
// list order within a colour.  The greedy pass is sequential (one lane per
// env, shared-memory scratch); the colour-ordered copy is a parallel stable
// scatter.
MSD void stage_color(EnvView& e, const Grp& g) {
    bool live = e.nb > 0;
    int nj = e.nj, nman = live ? e.cnt[C_NMAN] : 0;
    int ncons = live ? nj + nman : 0;
    int cmax = g.wmax(ncons);
    for (int i0 = 0; i0 < cmax; i0 += g.size) {
        int i = i0 + g.lane;
        if (i < nj) {
            int4 jm = e.jm[i];
            e.cons[i] = make_int4(jm.y, jm.z, i, CP_JOINT | (i << 8));
        } else if (i < ncons) {
            int m = i - nj;
            int4 M = e.man[m];
            int place = M.w + M.z <= e.pts_s ? CP_MAN_S : CP_MAN_G;
            e.cons[i] = make_int4(M.x, M.y, 3 * M.w, place | (M.z << 2) | (m << 8));
        }
    }
    // colour masks cleared; the orientations at the start of the step, which
    // the contact rows keep
    int nbmax = g.wmax(e.nb);
    for (int b0 = 0; b0 < nbmax; b0 += g.size)
        if (b0 + g.lane < e.nb) {
            e.used[b0 + g.lane] = 0ull;
            e.sq[3 * (b0 + g.lane) + 2] = e.q[b0 + g.lane];
        }
    g.sync();
    if (g.lane == 0 && live) {
        // greedy colours; color_off counts the members of each colour
        int ncol = 0;
        bool overflow = false;
        for (int i = 0; i < ncons; i++) {
            int4 c = e.cons[i];
            bool da = c.x >= 0 && e.v[c.x].w > 0.f, db = c.y >= 0 && e.v[c.y].w > 0.f;
            unsigned long long m = (da ? e.used[c.x] : 0ull) | (db ? e.used[c.y] : 0ull);
            if (m == ~0ull) { e.colr[i] = -1; overflow = true; continue; }
            int col = __ffsll((long long)~m) - 1;        // at most ncol: a new colour is the next one
            e.colr[i] = col;
            if (da) e.used[c.x] |= 1ull << col;
            if (db) e.used[c.y] |= 1ull << col;
            if (col == ncol) { e.color_off[col] = 0; ncol++; }
            e.color_off[col]++;
        }
        int acc = 0;
        for (int c = 0; c < ncol; c++) { int n = e.color_off[c]; e.color_off[c] = acc; acc += n; }
        e.color_off[ncol] = acc;
        e.cnt[C_NCONS] = acc;                          // constraints with a colour
        e.cnt[C_NCOLORS] = ncol;
        if (overflow) *e.status |= ST_COLOR;
        if (e.rec_col)
            for (int i = 0; i < ncons; i++) e.rec_col[i] = e.colr[i];
    }
    g.sync();
    // x.w marks the bodies that carry a constraint this step (a colour bit);
    // the others keep their angular velocity in world space (S = identity)
    for (int b0 = 0; b0 < nbmax; b0 += g.size)
        if (b0 + g.lane < e.nb) e.x[b0 + g.lane].w = e.used[b0 + g.lane] != 0ull ? 1.f : 0.f;
    g.sync();
    // stable scatter into colour order: color_off[c] runs from the start to
    // the end of colour c, then is shifted back into start offsets
    int wl = g.base + g.lane;                              // lane in the warp
    for (int i0 = 0; i0 < cmax; i0 += g.size) {
        int i = i0 + g.lane;
        int col = i < ncons ? e.colr[i] : -1;
        unsigned key = col >= 0 ? (unsigned)col | ((unsigned)g.base << 8) : 0x80000000u | (unsigned)wl;
        unsigned peers = __match_any_sync(FULL_MASK, key);
        int pos = 0;
        if (col >= 0) {
            pos = e.color_off[col] + __popc(peers & ((1u << wl) - 1u));
            e.scons[pos] = e.cons[i];
        }
        g.sync();
        if (col >= 0 && (peers >> wl) == 1u) e.color_off[col] = pos + 1;   // the highest peer
        g.sync();
    }
    if (g.lane == 0 && live) {
        int ncol = e.cnt[C_NCOLORS];
        for (int c = ncol; c > 0; c--) e.color_off[c] = e.color_off[c - 1];
        e.color_off[0] = 0;
    }
    g.sync();
    int nrows = live ? 8 * e.njs + 3 * e.cnt[C_NPTS] : 0;
    int rmax = g.wmax(nrows);
    for (int r0 = 0; r0 < rmax; r0 += g.size)
        if (r0 + g.lane < nrows) e.lam[r0 + g.lane] = 0.f;
    g.sync();
}

// ------------------------------------------------------------------- prep
struct BodyPose {
    float3 x;
    float4 q;
    M3 R;
    S3 S;          // (world inverse inertia)^(1/2); identity for static bodies, 0 for the world
    float im;
    bool dyn;
};

MSD S3 load_sq(const EnvView& e, int i) {
    float4 a = e.sq[3 * i], b = e.sq[3 * i + 1];
    return S3{a.x, a.y, a.z, a.w, b.x, b.y};
}

// world angular velocity of a dynamic body from its w^ (e.w during a
// substep): S w^ minus the round-trip error r recorded at the prep
MSD float3 world_w(const EnvView& e, int i) {
    float4 b = e.sq[3 * i + 1], w = e.w[i];
    return smv(load_sq(e, i), xyz(w)) - f3(b.z, b.w, w.w);
}

MSD BodyPose pose_of(const EnvView& e, int i) {
    BodyPose b;
    if (i < 0) {
        b.x = f3(0.f, 0.f, 0.f);
        b.q = make_float4(0.f, 0.f, 0.f, 1.f);
        b.R = qmat(b.q);
        b.S = S3{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        b.im = 0.f;
        b.dyn = false;
        return b;
    }
    b.x = xyz(e.x[i]);
    b.q = e.q[i];
    b.R = qmat(b.q);
    b.S = load_sq(e, i);
    b.im = e.v[i].w;
    b.dyn = b.im > 0.f;
    return b;
}

MSD float contact_bias(float d, float h, float vmax) { return d >= 0.f ? d / h : fmaxf(d / h, -vmax); }

// bias of a joint equality row with error C: C / h rigid, rate x C soft
MSD float eq_bias(const Params& P, float C) { return P.j_is > 0.f ? P.j_rate * C : C / P.h; }

// Writes the row and returns its effective mass k (static bodies add no
// angular term).
MSD float write_row(Row& r, float3 lin, float3 angA, float3 angB, const BodyPose& A, const BodyPose& B, float b,
                    float c) {
    float3 sa = smv(A.S, angA), sb = smv(B.S, angB);
    float ka = A.dyn ? dot(sa, sa) : 0.f, kb = B.dyn ? dot(sb, sb) : 0.f;
    float k = fmaf(A.im + B.im, dot(lin, lin), ka + kb);
    r.a = f4(lin, k > 0.f ? 1.f / k : 0.f);
    r.b = f4(sa, b);
    r.c = f4(sb, c);
    return k;
}

MSD float point_row(Row& r, float3 e_, float3 rA, float3 rB, const BodyPose& A, const BodyPose& B, float b, float c) {
    return write_row(r, e_, cross(rA, e_), cross(e_, rB), A, B, b, c);
}

MSD float ang_row(Row& r, float3 jA, float3 jB, const BodyPose& A, const BodyPose& B, float b, float c) {
    return write_row(r, f3(0.f, 0.f, 0.f), jA, jB, A, B, b, c);
}

struct JointGeo {
    float3 wP, wC, rP, rC, a, c;
    float phi;
    float4 qPw, qCw;
};

MSD JointGeo joint_geo(const EnvView& e, int j, int type, const BodyPose& P, const BodyPose& C) {
    JointGeo g;
    float4 f0 = e.jf[4 * j], f1 = e.jf[4 * j + 1], f2 = e.jf[4 * j + 2], f3_ = e.jf[4 * j + 3];
    g.rP = mv(P.R, xyz(f0));
    g.rC = mv(C.R, xyz(f2));
    g.wP = P.x + g.rP;
    g.wC = C.x + g.rC;
    g.qPw = qmul(P.q, f1);
    g.qCw = qmul(C.q, f3_);
    g.a = qrot(g.qPw, f3(1.f, 0.f, 0.f));
    g.c = qrot(g.qCw, f3(1.f, 0.f, 0.f));
    if (type == 0) {
        float4 qr = qmul(qconj(g.qPw), g.qCw);
        g.phi = wrap_pi(2.f * atan2f(qr.x, qr.w));
    } else {
        g.phi = dot(g.a, g.wC - g.wP);
    }
    return g;
}

// contact tangent basis: t1 = normalize(n x e_k), k = basis_axis(n), t2 = n x t1
MSD void tangents(float3 n, float3& t1, float3& t2) {
    int ax = basis_axis(n);
    t1 = cross(n, axis3(ax));
    t1 = t1 * (1.f / len(t1));
    t2 = cross(n, t1);
}

// Contact point geometry inside a step: the anchors keep the orientation of
// the step start (r = R0 a) and the separation follows each body's motion to
// first order in its rotation since then, theta = 2 sgn(w) vec(q q0^-1),
//     d = n . ((x_A + r_A + theta_A x r_A) - (x_B + r_B + theta_B x r_B)),
// the temporal-Gauss-Seidel scheme of the engine the paper builds on.  (With
// anchors turned with the body, a rolling body sinks by r (1 - cos theta)
// inside a step and is pushed back up: it gains energy.)
struct StepFrame {
    M3 R0;          // rotation at the step start
    float3 th;      // rotation since then, to first order
};

MSD StepFrame step_frame(const EnvView& e, int i, float4 q) {
    StepFrame f;
    float4 q0 = i >= 0 ? e.sq[3 * i + 2] : make_float4(0.f, 0.f, 0.f, 1.f);
    f.R0 = qmat(q0);
    float4 d = qmul(q, qconj(q0));
    float s = d.w >= 0.f ? 2.f : -2.f;
    f.th = f3(s * d.x, s * d.y, s * d.z);
    return f;
}

MSD float contact_sep(const float4* pt, const BodyPose& A, const BodyPose& B, const StepFrame& FA,
                      const StepFrame& FB, float3& rA, float3& rB) {
    rA = mv(FA.R0, xyz(pt[0]));
    rB = mv(FB.R0, xyz(pt[1]));
    float3 pa = (A.x + rA) + cross(FA.th, rA);
    float3 pb = (B.x + rB) + cross(FB.th, rB);
    return dot(xyz(pt[2]), pa - pb);
}

MSD Row* cons_rows(const EnvView& e, int4 c) {
    int place = c.w & 3;
    return (place == CP_JOINT ? e.rows_j : (place == CP_MAN_S ? e.rows_cs : e.rows_cg)) + c.z;
}

template <bool JOINTS = true>
MSD void prep_constraint(EnvView& e, int4 c, const Params& P) {
    bool joint = (c.w & 3) == CP_JOINT;
    int idx = c.w >> 8;
    BodyPose A = pose_of(e, c.x), B = pose_of(e, c.y);
    Row* R = cons_rows(e, c);
    float h = P.h;
    if (!joint) {
        // the colour-ordered record carries the manifold: bodies c.x, c.y,
        // first row c.z = 3 x first point, point count in c.w (no load of
        // the manifold header)
        int4 M = make_int4(c.x, c.y, (c.w >> 2) & 7, c.z / 3);
        int np = M.z;
        float mu = 0.5f * (e.shape[M.x].w + e.shape[M.y].w);
        StepFrame FA = step_frame(e, c.x, A.q), FB = step_frame(e, c.y, B.q);
        for (int k = 0; k < np; k++) {
            const float4* pt = e.pts + 3 * (M.w + k);
            float3 n = xyz(pt[2]), rA, rB;
            float d = contact_sep(pt, A, B, FA, FB, rA, rB);
            float3 t1, t2;
            tangents(n, t1, t2);
            // soft normal rows keep mass scale / k; a separated point keeps
            // its speculative bias d / h, a penetrating one takes rate x d
            // (continuous at d = 0)
            bool soft = P.c_is > 0.f;
            point_row(R[k], n, rA, rB, A, B, (soft && d < 0.f) ? fmaxf(P.c_rate * d, -P.vmax) : contact_bias(d, h, P.vmax),
                      0.f);
            if (soft) R[k].a.w *= P.c_ms;
            point_row(R[np + 2 * k], t1, rA, rB, A, B, mu, 0.f);
            point_row(R[np + 2 * k + 1], t2, rA, rB, A, B, mu, 0.f);
        }
        return;
    }
    if constexpr (!JOINTS) return;              // a batch without joints
    const int J = e.njs;                        // joint row stride
    int4 jm = e.jm[idx];
    float4 jp = e.jp[idx];
    JointGeo gj = joint_geo(e, idx, jm.x, A, B);
    float kd7;
    if (jm.x == 0) {
        for (int t = 0; t < 3; t++) {
            float3 ee = axis3(t);
            point_row(R[t * J], ee, gj.rP, gj.rC, A, B, eq_bias(P, dot(ee, gj.wP - gj.wC)), 0.f);
        }
        int k = basis_axis(gj.a);
        float3 b1 = cross(gj.a, axis3(k));
        b1 = b1 * (1.f / len(b1));
        float3 b2 = cross(gj.a, b1);
        float3 axc = cross(gj.a, gj.c);
        ang_row(R[3 * J], -b1, b1, A, B, eq_bias(P, dot(b1, axc)), 0.f);
        ang_row(R[4 * J], -b2, b2, A, B, eq_bias(P, dot(b2, axc)), 0.f);
        ang_row(R[5 * J], -gj.a, gj.a, A, B, contact_bias(gj.phi - jp.x, h, P.vmax), 0.f);
        ang_row(R[6 * J], gj.a, -gj.a, A, B, contact_bias(jp.y - gj.phi, h, P.vmax), 0.f);
        kd7 = ang_row(R[7 * J], -gj.a, gj.a, A, B, 0.f, 0.f);
    } else {
        int k = basis_axis(gj.a);
        float3 b1 = cross(gj.a, axis3(k));
        b1 = b1 * (1.f / len(b1));
        float3 b2 = cross(gj.a, b1);
        point_row(R[0 * J], b1, gj.rP, gj.rC, A, B, eq_bias(P, dot(b1, gj.wP - gj.wC)), 0.f);
        point_row(R[1 * J], b2, gj.rP, gj.rC, A, B, eq_bias(P, dot(b2, gj.wP - gj.wC)), 0.f);
        float4 qe = qmul(gj.qPw, qconj(gj.qCw));
        float sg = qe.w >= 0.f ? 1.f : -1.f;
        float3 th = f3(2.f * sg * qe.x, 2.f * sg * qe.y, 2.f * sg * qe.z);
        for (int t = 0; t < 3; t++) {
            float3 ee = axis3(t);
            ang_row(R[(2 + t) * J], ee, -ee, A, B, eq_bias(P, comp(th, t)), 0.f);
        }
        point_row(R[5 * J], -gj.a, gj.rP, gj.rC, A, B, contact_bias(gj.phi - jp.x, h, P.vmax), 0.f);
        point_row(R[6 * J], gj.a, gj.rP, gj.rC, A, B, contact_bias(jp.y - gj.phi, h, P.vmax), 0.f);
        kd7 = point_row(R[7 * J], -gj.a, gj.rP, gj.rC, A, B, 0.f, 0.f);
    }
    // soft equality rows keep mass scale / k
    if (P.j_is > 0.f)
        for (int t = 0; t < 5; t++) R[t * J].a.w *= P.j_ms;
    // PD drive as an implicit spring-damper: gamma = 1/(h (h kp + kd)),
    // b = kp C / (h kp + kd), C = phi - target; the row keeps
    // 1/(k + gamma) so that each iteration is one multiply
    float kp = jp.z, kd = jp.w;
    float den = fmaf(h, kp, kd);
    Row& dr = R[7 * J];
    if (den > 0.f && kd7 > 0.f) {
        float gam = 1.f / (h * den);
        dr.c.w = gam;
        dr.b.w = kp * (gj.phi - e.jt[idx]) / den;
        dr.a.w = 1.f / (kd7 + gam);
    } else {
        dr.a.w = 0.f;
    }
}

template <bool JOINTS = true>
MSD void stage_prep(EnvView& e, const Grp& g, const Params& P) {
    float h = P.h;
    int nb = e.nb;
    int nbmax = g.wmax(nb);
    for (int i0 = 0; i0 < nbmax; i0 += g.size) {
        int i = i0 + g.lane;
        if (i >= nb) continue;
        // a dynamic body without a constraint this step (x.w = 0) keeps S =
        // identity: its angular velocity is carried exactly, not through S^-1
        // and back
        if (is_dyn(e, i)) {
            // implicit damping (factor 1 / (1 + h c); exactly 1 without) and gravity
            float4 v = e.v[i];
            v.x = fmaf(h, P.gx, v.x * P.adl); v.y = fmaf(h, P.gy, v.y * P.adl); v.z = fmaf(h, P.gz, v.z * P.adl);
            e.v[i] = v;
        }
        if (is_dyn(e, i) && e.x[i].w != 0.f) {
            float4 iv = e.inv[i];
            float3 sd = xyz(iv);                        // (principal inverse inertia)^(1/2), stored
            M3 R = qmat(e.q[i]);
            S3 S = rdrt(R, sd);
            S3 Si = rdrt(R, f3(1.f / sd.x, 1.f / sd.y, 1.f / sd.z));
            // w^ = S^-1 w, and the round trip's error r = S w^ - w, which
            // every later S w^ subtracts: only the substep's change of w^
            // goes through S (w.w and sq[3i+1].zw hold r)
            float3 w0 = xyz(e.w[i]) * P.adw;
            float3 wh = smv(Si, w0);
            float3 r = smv(S, wh) - w0;
            e.sq[3 * i] = make_float4(S.xx, S.xy, S.xz, S.yy);
            e.sq[3 * i + 1] = make_float4(S.yz, S.zz, r.x, r.y);
            e.w[i] = f4(wh, r.z);
        } else {
            if (is_dyn(e, i)) e.w[i] = f4(xyz(e.w[i]) * P.adw, 0.f);
            e.sq[3 * i] = make_float4(1.f, 0.f, 0.f, 1.f);
            e.sq[3 * i + 1] = make_float4(0.f, 1.f, 0.f, 0.f);
        }
    }
    g.sync();
    int ncons = nb > 0 ? e.cnt[C_NCONS] : 0;
    int cmax = g.wmax(ncons);
    for (int c0 = 0; c0 < cmax; c0 += g.size) {
        int ci = c0 + g.lane;
        if (ci < ncons) prep_constraint<JOINTS>(e, e.scons[ci], P);
    }
    g.sync();
}

// ------------------------------------------------------------------ solve
// Rows of one constraint, in order, with both bodies' velocities and
// inverse masses in registers.  MODE 0: warm start (apply lambda); 1:
// position iteration; 2: relax iteration (drives skipped, relax bias; joint
// equality rows carry a zero relax bias).  Every row kind goes through one
// formula,
//     lambda' = clamp(lambda - (Jv + b + gamma lambda) / (k + gamma), lo, hi)
// with gamma = 0 except for drives and (lo, hi) = (0, inf) for normals and
// limits, +-mu lambda_n for friction, unbounded otherwise; an inert row has
// 1/k = 0 and leaves lambda unchanged.  The next row is loaded while the
// current one is solved, and every term that does not depend on Jv is
// formed before it, so the chain from one row's impulse to the next row's
// is short.
// The pointers the sweeps touch, small enough to live in registers.
struct SolveCtx {
    float4* v;
    float4* w;
    const Row* rj;
    const Row* rcs;
    const Row* rcg;
    float* lam;
    int njs;
    float c_is, c_ims, j_is, j_ims;      // soft rows: impulse scale, 1 / mass scale
};

MSD SolveCtx solve_ctx(const EnvView& e, const Params& P) {
    return SolveCtx{e.v, e.w, e.rows_j, e.rows_cs, e.rows_cg, e.lam, e.njs, P.c_is, P.c_ims, P.j_is, P.j_ims};
}

// Every lane of the warp runs the same number of row iterations (nrmax, the
// warp's largest row count) through straight-line code: rows past a lane's
// own count, and lanes without a constraint (has = false), change nothing.
// Lanes that diverged on a trip count or a row kind would run their paths
// one after the other.
template <int MODE, bool JOINTS = true>
MSD void solve_constraint(const SolveCtx& x, int4 c, bool has, int nrmax) {
    int place = c.w & 3, np = (c.w >> 2) & 7;
    bool joint = JOINTS && place == CP_JOINT;
    int nrows = has ? (joint ? 8 : 3 * np) : 0;
    // addressing by the record's place (an idle lane's null record is a
    // joint record, valid in every batch), row kinds by `joint`
    bool jplace = place == CP_JOINT;
    const Row* R = (jplace ? x.rj : (place == CP_MAN_S ? x.rcs : x.rcg)) + c.z;
    float* L = x.lam + (jplace ? c.z : 8 * x.njs + c.z);
    int st = jplace ? x.njs : 1;                        // row stride
    int last = max(nrows - 1, 0);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 va = c.x >= 0 ? x.v[c.x] : z4, wa4 = c.x >= 0 ? x.w[c.x] : z4;
    float4 vb = c.y >= 0 ? x.v[c.y] : z4, wb4 = c.y >= 0 ? x.w[c.y] : z4;
    float imA = va.w, imB = vb.w, imS = imA + imB;
    // a static body's velocity enters Jv but no impulse changes it
    bool dynA = imA > 0.f, dynB = imB > 0.f;
    // the loop keeps v_A and the relative velocity dv = v_A - v_B, which is
    // all that the linear part of Jv needs: J v = lin . dv + sa . w_A + sb . w_B
    float3 vA = xyz(va), wA = xyz(wa4), wB = xyz(wb4);
    float3 dv = vA - xyz(vb);
    float4 n0 = R[0].a, n1 = R[0].b, n2 = R[0].c;
    for (int r = 0; r < nrmax; r++) {
        float4 ra = n0, rb = n1, rc = n2;
        int rn = min(r + 1, last) * st;                  // prefetch the next row (clamped, always valid)
        n0 = R[rn].a; n1 = R[rn].b; n2 = R[rn].c;
        bool live = r < nrows;
        int ri = min(r, last) * st;
        float3 lin = xyz(ra), sa = xyz(rb), sb = xyz(rc);
        // off the dependency chain: everything in lambda' except Jv
        float old = L[ri];
        float dl;
        if (MODE == 0) {
            dl = (live && ra.w > 0.f) ? old : 0.f;
        } else {
            bool fric = !joint && r >= np;
            bool drive = joint && r == 7;
            bool eq = joint && r < 5;
            // soft rows (contact normals, joint equality rows): in position
            // sweeps dl = -ms (Jv + bias) / k - is lambda with ms / k stored;
            // relax sweeps solve them rigid, 1 / k
            bool softc = !joint && !fric && x.c_is > 0.f;
            bool softj = eq && x.j_is > 0.f;
            float ik = (MODE == 2 && drive) ? 0.f
                     : (MODE == 2 ? ra.w * (softc ? x.c_ims : (softj ? x.j_ims : 1.f)) : ra.w);
            float isv = MODE == 2 ? 0.f : (softc ? x.c_is : (softj ? x.j_is : 0.f));
            float bias = fric ? 0.f : (MODE == 2 ? (drive ? 0.f : rc.w) : rb.w);
            float gam = drive ? rc.w : 0.f;
            // old (1 - is) - (bias + gamma old) / (k + gamma)
            float c1 = fmaf(-fmaf(gam, old, bias), ik, fmaf(-isv, old, old));
            // friction bound from the point's normal impulse (a valid index for every row)
            float ln = L[(fric && live) ? (r - np) >> 1 : ri];
            float lim = rb.w * ln;
            float lo = fric ? -lim : ((eq || drive) ? -INFINITY : 0.f);
            float hi = fric ? lim : INFINITY;
            // Jv as three independent products
            float jv = (dot(lin, dv) + dot(sa, wA)) + dot(sb, wB);
            float nl = fmaf(-jv, ik, c1);
            nl = fminf(fmaxf(nl, lo), hi);
            if (live) L[ri] = nl;
            dl = live ? nl - old : 0.f;
        }
        vA = madd(vA, lin, dl * imA);
        dv = madd(dv, lin, dl * imS);
        wA = madd(wA, sa, dynA ? dl : 0.f);
        wB = madd(wB, sb, dynB ? dl : 0.f);
    }
    if (has && dynA) { x.v[c.x] = f4(vA, imA); x.w[c.x] = f4(wA, wa4.w); }
    if (has && dynB) { x.v[c.y] = f4(vA - dv, imB); x.w[c.y] = f4(wB, wb4.w); }
}

template <int MODE, bool JOINTS = true>
MSD void sweep_mode(EnvView& e, const Grp& g, const Params& P) {
    SolveCtx x = solve_ctx(e, P);
    const int4* sc = e.scons;
    const int* off = e.color_off;
    int ncol = e.nb > 0 ? e.cnt[C_NCOLORS] : 0;
    int colmax = g.wmax(ncol);
    int k0 = 0;
    const int4 none = make_int4(-1, -1, 0, CP_JOINT);    // the null constraint of an idle lane
    for (int col = 0; col < colmax; col++) {
        int k1 = col < ncol ? off[col + 1] : k0;
        int wmaxn = g.wmax(k1 - k0);
        for (int m = 0; m < wmaxn; m += g.size) {
            int k = k0 + m + g.lane;
            bool has = k < k1;
            int4 c = has ? sc[k] : none;
            int nr = has ? ((c.w & 3) == CP_JOINT ? 8 : 3 * ((c.w >> 2) & 7)) : 0;
            solve_constraint<MODE, JOINTS>(x, c, has, g.wmax(nr));
        }
        g.sync();
        k0 = k1;
    }
}

template <bool JOINTS = true>
MSD void stage_sweep(EnvView& e, const Grp& g, int mode, const Params& P) {
    if (mode == 0) sweep_mode<0, JOINTS>(e, g, P);
    else if (mode == 1) sweep_mode<1, JOINTS>(e, g, P);
    else sweep_mode<2, JOINTS>(e, g, P);
}

// -------------------------------------------------------------- integrate
template <bool JOINTS = true>
MSD void relax_constraint(EnvView& e, int4 c, const Params& P) {
    bool joint = (c.w & 3) == CP_JOINT;
    int idx = c.w >> 8;
    Row* R = cons_rows(e, c);
    float h = P.h;
    BodyPose A = pose_of(e, c.x), B = pose_of(e, c.y);
    if (!joint) {
        int4 M = make_int4(c.x, c.y, (c.w >> 2) & 7, c.z / 3);   // as in prep_constraint
        StepFrame FA = step_frame(e, c.x, A.q), FB = step_frame(e, c.y, B.q);
        for (int k = 0; k < M.z; k++) {
            float3 rA, rB;
            float d = contact_sep(e.pts + 3 * (M.w + k), A, B, FA, FB, rA, rB);
            R[k].c.w = fmaxf(d, 0.f) / h;
        }
    } else if constexpr (JOINTS) {
        int4 jm = e.jm[idx];
        float4 jp = e.jp[idx];
        JointGeo gj = joint_geo(e, idx, jm.x, A, B);
        R[5 * e.njs].c.w = fmaxf(gj.phi - jp.x, 0.f) / h;
        R[6 * e.njs].c.w = fmaxf(jp.y - gj.phi, 0.f) / h;
    }
}

// symplectic Euler with w = S w^; e.w keeps w^ for the relax sweeps
template <bool JOINTS = true>
MSD void stage_integrate(EnvView& e, const Grp& g, const Params& P) {
    float h = P.h;
    int nb = e.nb;
    int nbmax = g.wmax(nb);
    for (int i0 = 0; i0 < nbmax; i0 += g.size) {
        int i = i0 + g.lane;
        if (i >= nb || !is_dyn(e, i)) continue;
        float4 x = e.x[i], q = e.q[i];
        float3 v = xyz(e.v[i]);
        float3 w = world_w(e, i);
        x.x = fmaf(h, v.x, x.x); x.y = fmaf(h, v.y, x.y); x.z = fmaf(h, v.z, x.z);
        float4 wq = qmul(make_float4(w.x, w.y, w.z, 0.f), q);
        float hh = 0.5f * h;
        q = qnormalize(make_float4(fmaf(hh, wq.x, q.x), fmaf(hh, wq.y, q.y), fmaf(hh, wq.z, q.z),
                                   fmaf(hh, wq.w, q.w)));
        e.x[i] = x;
        e.q[i] = q;
    }
    g.sync();
    int ncons = nb > 0 ? e.cnt[C_NCONS] : 0;
    int cmax = g.wmax(ncons);
    for (int c0 = 0; c0 < cmax; c0 += g.size) {
        int ci = c0 + g.lane;
        if (ci < ncons) relax_constraint<JOINTS>(e, e.scons[ci], P);
    }
    g.sync();
}

// end of a substep: angular velocities back to world space, w = S w^
MSD void stage_unscale(EnvView& e, const Grp& g) {
    int nb = e.nb;
    int nbmax = g.wmax(nb);
    for (int i0 = 0; i0 < nbmax; i0 += g.size) {
        int i = i0 + g.lane;
        if (i < nb && is_dyn(e, i)) e.w[i] = f4(world_w(e, i), 0.f);
    }
    g.sync();
}

// end-of-step check: a non-finite state freezes the env
MSD void stage_check(EnvView& e, const Grp& g) {
    bool bad = false;
    int nbmax = g.wmax(e.nb);
    for (int i0 = 0; i0 < nbmax; i0 += g.size) {
        int i = i0 + g.lane;
        if (i >= e.nb) continue;
        float4 x = e.x[i], q = e.q[i], v = e.v[i], w = e.w[i];
        float s = x.x + x.y + x.z + q.x + q.y + q.z + q.w + v.x + v.y + v.z + w.x + w.y + w.z;
        bad |= !isfinite(s);
    }
    bool any = g.any(bad);
    if (g.lane == 0 && any) *e.status |= ST_NAN;
    g.sync();
}

// ------------------------------------------------- optional solver variants
// Warm start across steps (P.warm): joint rows keep their impulses; the k-th
// point of a manifold takes the normal impulse and the friction impulse (a
// world vector, projected onto its tangents) of the k-th point of the
// previous step's manifold of the same body pair.
MSD Row* man_rows(const EnvView& e, int4 M) {
    return (M.w + M.z <= e.pts_s ? e.rows_cs : e.rows_cg) + 3 * M.w;
}

// Contact forces of a step (touch sensors): per body, the impulses of the
// contact rows of every manifold that involves it over the last substep,
// divided by h: sum of +-lin lambda (+ on body a, - on body b) and the sum of
// the normal impulses.  One lane per body, manifolds in list order, rows in
// order.  Every lane of the warp runs it (an idle lane group with nb = 0).
MSD void stage_contact_forces(EnvView& e, const Grp& g, const Params& P) {
    int nb = e.nb, nman = nb > 0 ? e.cnt[C_NMAN] : 0;
    float ih = 1.f / P.h;
    const float* L0 = e.lam + 8 * e.njs;
    int nbmax = g.wmax(nb);
    for (int i0 = 0; i0 < nbmax; i0 += g.size) {
        int i = i0 + g.lane;
        if (i >= nb) continue;
        float3 F = f3(0.f, 0.f, 0.f);
        float fn = 0.f;
        for (int m = 0; m < nman; m++) {
            int4 M = e.man[m];
            if (M.x != i && M.y != i) continue;
            float sg = M.x == i ? 1.f : -1.f;
            const Row* R = man_rows(e, M);
            const float* L = L0 + 3 * M.w;
            for (int r = 0; r < 3 * M.z; r++) {
                F = madd(F, xyz(R[r].a), sg * L[r]);
                if (r < M.z) fn += L[r];
            }
        }
        if (e.force) e.force[i] = make_float4(F.x * ih, F.y * ih, F.z * ih, fn * ih);
    }
    g.sync();
}

// Every lane of the warp runs these stages (their loops end in warp-wide
// operations); a lane group without warm-start memory (an idle slot) takes
// part with zero counts.
MSD void stage_warm_init(EnvView& e, const Grp& g) {
    bool on = e.wc != nullptr && e.nb > 0;
    int nj = on ? e.nj : 0, nman = on ? e.cnt[C_NMAN] : 0;
    int n8 = 8 * nj, m8 = g.wmax(n8);
    for (int i0 = 0; i0 < m8; i0 += g.size) {
        int i = i0 + g.lane;
        if (i < n8) e.lam[(i & 7) * e.njs + (i >> 3)] = e.wjl[i];
    }
    int nold = on ? *e.wc_n : 0;
    float* Lc = e.lam + 8 * e.njs;
    int mmax = g.wmax(nman);
    for (int m0 = 0; m0 < mmax; m0 += g.size) {
        int m = m0 + g.lane;
        if (m >= nman) continue;
        int4 M = e.man[m];
        int key = M.x | (M.y << 16);
        int k = 0;
        for (int q = 0; q < nold && k < M.z; q++) {
            float4 c0 = e.wc[2 * q];
            if (__float_as_int(c0.w) != key) continue;
            float4 c1 = e.wc[2 * q + 1];
            float3 t1, t2;
            tangents(xyz(e.pts[3 * (M.w + k) + 2]), t1, t2);
            float3 ft = f3(c1.y, c1.z, c1.w);
            Lc[3 * M.w + k] = c1.x;
            Lc[3 * M.w + M.z + 2 * k] = dot(ft, t1);
            Lc[3 * M.w + M.z + 2 * k + 1] = dot(ft, t2);
            k++;
        }
    }
    g.sync();
}

MSD void stage_store_warm(EnvView& e, const Grp& g) {
    bool on = e.wc != nullptr && e.nb > 0;
    int nj = on ? e.nj : 0, nman = on ? e.cnt[C_NMAN] : 0;
    int n8 = 8 * nj, m8 = g.wmax(n8);
    for (int i0 = 0; i0 < m8; i0 += g.size) {
        int i = i0 + g.lane;
        if (i < n8) e.wjl[i] = e.lam[(i & 7) * e.njs + (i >> 3)];
    }
    const float* Lc = e.lam + 8 * e.njs;
    int mmax = g.wmax(nman);
    for (int m0 = 0; m0 < mmax; m0 += g.size) {
        int m = m0 + g.lane;
        if (m >= nman) continue;
        int4 M = e.man[m];
        const Row* R = man_rows(e, M);
        int key = M.x | (M.y << 16);
        for (int k = 0; k < M.z; k++) {
            int pnt = M.w + k;
            float3 t1 = xyz(R[M.z + 2 * k].a), t2 = xyz(R[M.z + 2 * k + 1].a);
            float3 ft = t1 * Lc[3 * M.w + M.z + 2 * k] + t2 * Lc[3 * M.w + M.z + 2 * k + 1];
            e.wc[2 * pnt] = make_float4(e.pts[3 * pnt].x, e.pts[3 * pnt].y, e.pts[3 * pnt].z, __int_as_float(key));
            e.wc[2 * pnt + 1] = make_float4(Lc[3 * M.w + k], ft.x, ft.y, ft.z);
        }
    }
    if (g.lane == 0 && on) *e.wc_n = e.cnt[C_NPTS];   // idle and frozen envs keep theirs
    g.sync();
}

// the largest normal impulse of each contact point at a substep's end
MSD void stage_track_impulse(EnvView& e, const Grp& g) {
    int nman = e.nb > 0 ? e.cnt[C_NMAN] : 0;
    const float* Lc = e.lam + 8 * e.njs;
    int mmax = g.wmax(nman);
    for (int m0 = 0; m0 < mmax; m0 += g.size) {
        int m = m0 + g.lane;
        if (m >= nman) continue;
        int4 M = e.man[m];
        for (int k = 0; k < M.z; k++) {
            float4& o = e.pts[3 * (M.w + k) + 2];
            o.w = fmaxf(o.w, Lc[3 * M.w + k]);
        }
    }
    g.sync();
}

// Restitution, after the last substep (in w^ space): in colour order, a
// contact point whose step-start approach speed exceeds P.bounce and that
// carried a normal impulse gets the normal impulse that makes its normal
// velocity -e times that speed, the accumulated impulse kept >= 0.
MSD void stage_restitution(EnvView& e, const Grp& g, const Params& P) {
    const int4* sc = e.scons;
    const int* off = e.color_off;
    int ncol = e.nb > 0 ? e.cnt[C_NCOLORS] : 0;
    int colmax = g.wmax(ncol);
    const float* Lc0 = e.lam + 8 * e.njs;
    int k0 = 0;
    for (int col = 0; col < colmax; col++) {
        int k1 = col < ncol ? off[col + 1] : k0;
        int wmaxn = g.wmax(k1 - k0);
        for (int mm = 0; mm < wmaxn; mm += g.size) {
            int ci = k0 + mm + g.lane;
            if (ci >= k1) continue;
            int4 c = sc[ci];
            if ((c.w & 3) == CP_JOINT) continue;
            int np = (c.w >> 2) & 7;
            int4 M = e.man[c.w >> 8];
            float er = 0.5f * ((M.x >= 0 ? e.rest[M.x] : 0.f) + (M.y >= 0 ? e.rest[M.y] : 0.f));
            if (!(er > 0.f)) continue;
            const Row* R = cons_rows(e, c);
            float* L = const_cast<float*>(Lc0) + c.z;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 va = c.x >= 0 ? e.v[c.x] : z4, wa4 = c.x >= 0 ? e.w[c.x] : z4;
            float4 vb = c.y >= 0 ? e.v[c.y] : z4, wb4 = c.y >= 0 ? e.w[c.y] : z4;
            float imA = va.w, imB = vb.w;
            bool dynA = imA > 0.f, dynB = imB > 0.f;
            float3 vA = xyz(va), wA = xyz(wa4), vB = xyz(vb), wB = xyz(wb4);
            for (int k = 0; k < np; k++) {
                float4 pe = e.pts[3 * (M.w + k) + 1], pm = e.pts[3 * (M.w + k) + 2];
                float vn0 = pe.w, lmax = pm.w;
                float4 ra = R[k].a, rb = R[k].b, rc = R[k].c;
                if (vn0 > -P.bounce || !(lmax > 0.f) || !(ra.w > 0.f)) continue;
                float3 lin = xyz(ra), sa = xyz(rb), sb = xyz(rc);
                float vn = (dot(lin, vA) + dot(sa, wA)) - (dot(lin, vB) - dot(sb, wB));
                float old = L[k];
                float ik = P.c_is > 0.f ? ra.w * P.c_ims : ra.w;   // rigid 1 / k
                float nl = fmaxf(fmaf(-fmaf(er, vn0, vn), ik, old), 0.f);
                L[k] = nl;
                float dl = nl - old;
                vA = madd(vA, lin * imA, dl);
                wA = madd(wA, sa, dynA ? dl : 0.f);
                vB = madd(vB, lin * (-imB), dl);
                wB = madd(wB, sb, dynB ? dl : 0.f);
            }
            if (dynA) { e.v[c.x] = f4(vA, imA); e.w[c.x] = f4(wA, wa4.w); }
            if (dynB) { e.v[c.y] = f4(vB, imB); e.w[c.y] = f4(wB, wb4.w); }
        }
        g.sync();
        k0 = k1;
    }
}

// One substep: prep, warm start, position sweeps, integration, relax
// sweeps, the contact impulse record and (last substep) restitution, unscale.
// RESTIT = false compiles restitution out (a batch without it); JOINTS =
// false the joint rows (a batch without joints).
// The first substep's warm start applies impulses that the colouring has
// just zeroed unless they are carried across steps (warm_start): it is
// skipped (first = true), which changes no value.
template <bool RESTIT = true, bool JOINTS = true>
MSD void run_substep(EnvView& e, const Grp& g, const Params& P, bool first, bool last) {
    stage_prep<JOINTS>(e, g, P);
    if (!first || P.warm) stage_sweep<JOINTS>(e, g, 0, P);
    for (int it = 0; it < P.pos_iters; it++) stage_sweep<JOINTS>(e, g, 1, P);
    stage_integrate<JOINTS>(e, g, P);
    for (int it = 0; it < P.vel_iters; it++) stage_sweep<JOINTS>(e, g, 2, P);
    if constexpr (RESTIT) {
        if (P.restit) {
            stage_track_impulse(e, g);
            if (last) stage_restitution(e, g, P);
        }
    }
    stage_unscale(e, g);
}

// Colouring of one step, then the warm-start impulses.  P is the same for
// every lane of a warp, so the branches are warp-uniform.
MSD void begin_step_solve(EnvView& e, const Grp& g, const Params& P) {
    stage_color(e, g);
    MS_CHECK_BOUNDS(e, g, P, true);
    if (P.warm) stage_warm_init(e, g);
}

// The end of a step: the warm-start memory.
MSD void end_step_solve(EnvView& e, const Grp& g, const Params& P) {
    if (P.warm) stage_store_warm(e, g);
}

// ------------------------------------------------------------- pick task
// The pick task of the paper's sim2real appendix (Observation Space,
// Reward): joint coordinates, the is-grasped flag and the dense reward,
// from the env's state after a step.

// pose without the inertia factor (world body for i < 0)
MSD BodyPose pose_kin(const EnvView& e, int i) {
    BodyPose b;
    b.x = i < 0 ? f3(0.f, 0.f, 0.f) : xyz(e.x[i]);
    b.q = i < 0 ? make_float4(0.f, 0.f, 0.f, 1.f) : e.q[i];
    b.R = qmat(b.q);
    b.S = S3{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    b.im = 0.f;
    b.dyn = false;
    return b;
}

// revolute angle or prismatic displacement, as the joint limits see it
MSD float joint_coord(const EnvView& e, int j) {
    int4 jm = e.jm[j];
    return joint_geo(e, j, jm.x, pose_kin(e, jm.y), pose_kin(e, jm.z)).phi;
}

// signed distance from body i to the table plane (the table's local +z
// through its origin): the body's lowest point along the normal
MSD float plane_gap(const EnvView& e, int i, int table) {
    float3 n = qrot(e.q[table], f3(0.f, 0.f, 1.f));
    float off = dot(n, xyz(e.x[i]) - xyz(e.x[table]));
    float4 s = e.shape[i];
    int t = shape_type(e, i);
    if (t == SH_SPHERE) return off - s.x;
    float4 q = e.q[i];
    if (t == SH_CAPSULE) return off - fabsf(dot(n, qrot(q, f3(0.f, 0.f, 1.f)))) * s.y - s.x;
    if (t == SH_BOX)
        return off - (fabsf(dot(n, qrot(q, f3(1.f, 0.f, 0.f)))) * s.x + fabsf(dot(n, qrot(q, f3(0.f, 1.f, 0.f)))) * s.y +
                      fabsf(dot(n, qrot(q, f3(0.f, 0.f, 1.f)))) * s.z);
    return off;
}

MSD float r_dist(float d, float z) { return 1.f - tanhf(z * d); }

// The record of one env: reward, grasped, tcp_close, touch_table, x_tcp[3],
// x_cube[3], q[A], target[A] (zero past the env's joints), with
//   tcp = midpoint of the fingers, g = finger b - finger a, c = cube side,
//   r = r_dist(|tcp - x_cube|, 15) + (1 - g.z/|g|)
//       + 2 [|tcp - x_cube| <= c/2] r_dist(| |g| - c |, 40)
//       + [grasped] (1 + 3 r_dist(|q - q_reset|, 4/pi)) - 2 [touch_table],
// grasped = the gripper joint more than grasp_tol from its target, touch =
// a finger within touch_tol of the table.  A frozen env writes NaN.  Every
// lane of the warp calls this (group-wide reductions); rec = null writes
// nothing.
MSD void stage_task_record(const EnvView& e, const Grp& g, const DevTask& T, int A, float* rec, bool frozen) {
    int nj = (rec && !frozen) ? e.nj : 0;
    int amax = g.wmax(rec ? A : 0);
    float part = 0.f;
    bool gr = false;
    for (int j0 = 0; j0 < amax; j0 += g.size) {
        int j = j0 + g.lane;
        if (j >= A || !rec) continue;
        float q = 0.f, t = 0.f;
        if (j < nj) {
            q = joint_coord(e, j);
            t = e.jt[j];
            float d = q - e.qR[j];
            part = fmaf(d, d, part);
            if (j == T.grip) gr = fabsf(q - t) > T.grasp_tol;
        }
        rec[10 + j] = frozen ? __int_as_float(0x7fffffff) : q;
        rec[10 + A + j] = frozen ? __int_as_float(0x7fffffff) : t;
    }
    for (int d = g.size >> 1; d > 0; d >>= 1) part += __shfl_xor_sync(FULL_MASK, part, d, g.size);
    bool grasped = g.any(gr);
    if (g.lane == 0 && rec) {
        if (frozen) {
            for (int k = 0; k < 10; k++) rec[k] = __int_as_float(0x7fffffff);
        } else {
            float3 xa = xyz(e.x[T.fa]), xb = xyz(e.x[T.fb]), xc = xyz(e.x[T.cube]);
            float3 tcp = (xa + xb) * 0.5f;
            float3 gv = xb - xa;
            float gl = len(gv);
            float c = 2.f * e.shape[T.cube].x;
            float dtc = len(tcp - xc);
            float r = r_dist(dtc, 15.f);
            r += gl > 0.f ? 1.f - gv.z / gl : 1.f;
            bool close = dtc <= 0.5f * c;
            if (close) r += 2.f * r_dist(fabsf(gl - c), 40.f);
            if (grasped) r += 1.f + 3.f * r_dist(sqrtf(part), 4.f / 3.14159265358979f);
            bool touch = plane_gap(e, T.fa, T.table) <= T.touch_tol || plane_gap(e, T.fb, T.table) <= T.touch_tol;
            if (touch) r -= 2.f;
            rec[0] = r; rec[1] = grasped ? 1.f : 0.f; rec[2] = close ? 1.f : 0.f; rec[3] = touch ? 1.f : 0.f;
            rec[4] = tcp.x; rec[5] = tcp.y; rec[6] = tcp.z;
            rec[7] = xc.x; rec[8] = xc.y; rec[9] = xc.z;
        }
    }
    g.sync();
}

// ------------------------------------------------- env views of a batch
// the env's parameters and warm-start memory, read in place from the
// resident arrays (an idle lane group has no warm-start memory)
MSD void view_params(EnvView& e, const DevBatch& D, int b0, int j0, int env, bool active) {
    e.shape = D.shape + b0; e.inv = D.inv + b0; e.meta = D.meta + b0; e.adj = D.adj + b0;
    e.jf = D.jf + 4 * (size_t)j0; e.jp = D.jp + j0; e.jm = D.jm + j0; e.jt = D.jt + j0;
    e.rest = D.rest + b0;
    e.qR = D.T.qR ? D.T.qR + j0 : nullptr;
    e.hulls = D.hulls;
    bool w = active && D.wc;
    e.wc = w ? D.wc + 2 * (size_t)env * (size_t)D.P.contact_cap : nullptr;
    e.wc_n = w ? D.wc_n + env : nullptr;
    e.wjl = w ? D.wjl + 8 * (size_t)j0 : nullptr;
    e.force = (D.force && active) ? D.force + b0 : nullptr;
}

MSD void view_record(EnvView& e, const DevBatch& D, int env, bool active) {
    if (D.rec_man && active) {
        e.rec_man = D.rec_man + (size_t)env * D.P.pair_cap;
        e.rec_pts = D.rec_pts + (size_t)env * D.P.contact_cap * 10;
        e.rec_cnt = D.rec_cnt + env;
        e.rec_col = D.rec_col + (size_t)env * D.rec_col_stride;
    } else {
        e.rec_man = nullptr; e.rec_pts = nullptr; e.rec_cnt = nullptr; e.rec_col = nullptr;
    }
}

}  // namespace ms
