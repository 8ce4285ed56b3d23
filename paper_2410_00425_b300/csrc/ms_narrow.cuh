// Primitive narrowphase, one pair per lane.
//
// Pair convention: A is the lower shape rank (sphere < capsule < box < hull
// < plane), the lower env-local index on equal ranks; the normal n points from
// B toward A; d = n.(cA - cB) is negative when penetrating; a point is kept
// iff d < margin (speculative contacts inside the margin).  Methods: closest
// points of primitives and the separating-axis test with Sutherland-Hodgman
// clipping of the incident face (Ericson 2005, Real-Time Collision
// Detection, 4.4 and 5.1.9); more than 4 points are reduced to the deepest
// point plus three that spread the contact area.
#pragma once
#include "ms_math.cuh"

namespace ms {

enum { SH_SPHERE = 0, SH_CAPSULE = 1, SH_BOX = 2, SH_PLANE = 3, SH_HULL = 4 };

// pair order of the narrowphase: sphere < capsule < box < hull < plane
MSD int shape_rank(int t) { return t == SH_HULL ? 3 : (t == SH_PLANE ? 4 : t); }

// A convex hull of the batch's library (body frame = its principal frame):
// vertices, outward counter-clockwise triangles with their local planes
// (n, n.v = d), and edges (a, b, triangle listing a -> b, triangle listing
// b -> a), each edge once.
struct HullRef {
    const float4* v;
    const int4* t;
    const float4* n;
    const int4* e;
    int nv, nt, ne;
};

struct Shape {
    float3 x;
    M3 R;
    int type;
    float p0, p1, p2;
    HullRef hull;                 // hull bodies
};

struct Cand {
    float3 cA, cB, n;
    float d;
};

struct CandSet {
    int n;
    Cand c[16];
    MSD void push(float3 cA, float3 cB, float3 nn, float d) {
        if (n < 16) { c[n].cA = cA; c[n].cB = cB; c[n].n = nn; c[n].d = d; n++; }
    }
};

MSD void sphere_pair(CandSet& cs, float3 a, float ra, float3 b, float rb) {
    float3 dl = a - b;
    float dist = len(dl);
    float3 n = dist < 1e-9f ? f3(0.f, 0.f, 1.f) : dl * (1.f / dist);
    cs.push(a - n * ra, b + n * rb, n, dist - ra - rb);
}

MSD float3 closest_on_segment(float3 p, float3 s0, float3 s1) {
    float3 d = s1 - s0;
    float dd = dot(d, d);
    float t = dd > 0.f ? clampf(dot(p - s0, d) / dd, 0.f, 1.f) : 0.f;
    return s0 + d * t;
}

// Closest points of segments p0 + s d1 and q0 + t d2 (Ericson 5.1.9); the
// denominator |d1|^2 |d2|^2 - (d1.d2)^2 is evaluated as |d1 x d2|^2, which
// keeps its accuracy for nearly parallel segments.
MSD void closest_segments(float3 p0, float3 p1, float3 q0, float3 q1, float3& cp, float3& cq) {
    float3 d1 = p1 - p0, d2 = q1 - q0, r = p0 - q0;
    float a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
    float s, t;
    if (a <= 1e-18f && e <= 1e-18f) { s = 0.f; t = 0.f; }
    else if (a <= 1e-18f) { s = 0.f; t = clampf(f / e, 0.f, 1.f); }
    else {
        float c = dot(d1, r);
        if (e <= 1e-18f) { t = 0.f; s = clampf(-c / a, 0.f, 1.f); }
        else {
            float b = dot(d1, d2);
            float3 cr = cross(d1, d2);
            float denom = dot(cr, cr);
            s = denom > 0.f ? clampf((b * f - c * e) / denom, 0.f, 1.f) : 0.f;
            t = (b * s + f) / e;
            if (t < 0.f) { t = 0.f; s = clampf(-c / a, 0.f, 1.f); }
            else if (t > 1.f) { t = 1.f; s = clampf((b - c) / a, 0.f, 1.f); }
        }
    }
    cp = p0 + d1 * s;
    cq = q0 + d2 * t;
}

MSD void capsule_ends(const Shape& s, float3& e0, float3& e1) {
    float3 ax = mcol(s.R, 2);
    e0 = s.x - ax * s.p1;
    e1 = s.x + ax * s.p1;
}

MSD void np_ss(const Shape& A, const Shape& B, CandSet& cs) { sphere_pair(cs, A.x, A.p0, B.x, B.p0); }

MSD void np_sp(const Shape& A, const Shape& B, CandSet& cs) {
    float3 N = mcol(B.R, 2);
    float dist = dot(N, A.x - B.x);
    cs.push(A.x - N * A.p0, A.x - N * dist, N, dist - A.p0);
}

MSD void np_sc(const Shape& A, const Shape& B, CandSet& cs) {
    float3 b0, b1;
    capsule_ends(B, b0, b1);
    float3 q = closest_on_segment(A.x, b0, b1);
    sphere_pair(cs, A.x, A.p0, q, B.p0);
}

// sphere in box frame: clamp the centre; when inside, leave through the face
// of least penetration (lowest axis, + side before - side on ties)
MSD void np_sb(const Shape& A, const Shape& B, CandSet& cs) {
    float r = A.p0;
    float3 c = mtv(B.R, A.x - B.x);
    float h[3] = {B.p0, B.p1, B.p2};
    float cc[3] = {c.x, c.y, c.z};
    bool inside = fabsf(cc[0]) <= h[0] && fabsf(cc[1]) <= h[1] && fabsf(cc[2]) <= h[2];
    if (!inside) {
        float3 ql = f3(clampf(cc[0], -h[0], h[0]), clampf(cc[1], -h[1], h[1]), clampf(cc[2], -h[2], h[2]));
        float3 dl = c - ql;
        float dist = len(dl);
        float3 nl = dist > 0.f ? dl * (1.f / dist) : f3(0.f, 0.f, 1.f);
        float3 n = mv(B.R, nl);
        cs.push(A.x - n * r, B.x + mv(B.R, ql), n, dist - r);
    } else {
        int bi = 0;
        float bs = 1.f, best = 3.0e38f;
#pragma unroll
        for (int i = 0; i < 3; i++) {
#pragma unroll
            for (int k = 0; k < 2; k++) {
                float sgn = k == 0 ? 1.f : -1.f;
                float depth = h[i] - sgn * cc[i];
                if (depth < best) { best = depth; bi = i; bs = sgn; }
            }
        }
        float3 nl = axis3(bi) * bs;
        float3 ql = with_comp(c, bi, bs * h[bi]);
        float3 n = mv(B.R, nl);
        cs.push(A.x - n * r, B.x + mv(B.R, ql), n, -best - r);
    }
}

MSD void np_cp(const Shape& A, const Shape& B, CandSet& cs) {
    float3 N = mcol(B.R, 2);
    float3 e[2];
    capsule_ends(A, e[0], e[1]);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        float dist = dot(N, e[k] - B.x);
        cs.push(e[k] - N * A.p0, e[k] - N * dist, N, dist - A.p0);
    }
}

// capsule-capsule: nearly parallel overlapping axes -> two points at the ends
// of the overlap interval; otherwise the closest points of the two segments
MSD void np_cc(const Shape& A, const Shape& B, CandSet& cs) {
    float3 a0, a1, b0, b1;
    capsule_ends(A, a0, a1);
    capsule_ends(B, b0, b1);
    float3 dA = a1 - a0, dB = b1 - b0;
    float la = len(dA), lb = len(dB);
    float cr = len(cross(dA, dB));
    if (la > 0.f && lb > 0.f && cr < 1e-3f * la * lb) {
        float3 u = dA * (1.f / la);
        float t0 = dot(b0 - a0, u), t1 = dot(b1 - a0, u);
        float lo = fmaxf(0.f, fminf(t0, t1)), hi = fminf(la, fmaxf(t0, t1));
        if (lo <= hi) {
            int cnt = (hi - lo) < 1e-6f ? 1 : 2;
            for (int k = 0; k < cnt; k++) {
                float3 pa = a0 + u * (k == 0 ? lo : hi);
                float3 pb = closest_on_segment(pa, b0, b1);
                sphere_pair(cs, pa, A.p0, pb, B.p0);
            }
            return;
        }
    }
    float3 pa, pb;
    closest_segments(a0, a1, b0, b1, pa, pb);
    sphere_pair(cs, pa, A.p0, pb, B.p0);
}

// exact closest points of a segment s0 + t u (t in [0,1]) and a box of
// half-extents h centred at the origin: the squared distance is convex and
// piecewise quadratic between slab-crossing parameters; minimise per piece
MSD float segment_box_closest(float3 s0, float3 u, const float h[3], float& tbest) {
    float ts[8];
    int nt = 0;
    ts[nt++] = 0.f; ts[nt++] = 1.f;
    float s0c[3] = {s0.x, s0.y, s0.z}, uc[3] = {u.x, u.y, u.z};
    for (int j = 0; j < 3; j++) {
        if (uc[j] == 0.f) continue;
        for (int k = 0; k < 2; k++) {
            float sg = k == 0 ? -1.f : 1.f;
            float t = (sg * h[j] - s0c[j]) / uc[j];
            if (t > 0.f && t < 1.f) ts[nt++] = t;
        }
    }
    for (int i = 1; i < nt; i++) {
        float x = ts[i];
        int k = i - 1;
        while (k >= 0 && ts[k] > x) { ts[k + 1] = ts[k]; k--; }
        ts[k + 1] = x;
    }
    float best = 3.0e38f, bt = 0.f;
    for (int i = 0; i + 1 < nt; i++) {
        float ta = ts[i], tb = ts[i + 1];
        float tm = 0.5f * (ta + tb);
        float num = 0.f, den = 0.f;
        for (int j = 0; j < 3; j++) {
            float x = s0c[j] + tm * uc[j];
            float cj = x > h[j] ? h[j] : (x < -h[j] ? -h[j] : x);
            if (cj != x) { num += (s0c[j] - cj) * uc[j]; den += uc[j] * uc[j]; }
        }
        float cand[3] = {ta, tb, den > 0.f ? clampf(-num / den, ta, tb) : ta};
        for (int k = 0; k < 3; k++) {
            float t = cand[k], f = 0.f;
            for (int j = 0; j < 3; j++) {
                float x = s0c[j] + t * uc[j];
                float cj = x > h[j] ? h[j] : (x < -h[j] ? -h[j] : x);
                f += (x - cj) * (x - cj);
            }
            if (f < best) { best = f; bt = t; }
        }
    }
    tbest = bt;
    return sqrtf(best);
}

// capsule-box in the box frame: SAT over 3 box faces and 3 (box edge x
// segment) axes; face case clips the segment to the face's side slabs
// (<= 2 points), edge case gives 1 point from edge-segment closest points
MSD void np_cb(const Shape& A, const Shape& B, float m, CandSet& cs) {
    float r = A.p0;
    float3 a0, a1;
    capsule_ends(A, a0, a1);
    float3 s0 = mtv(B.R, a0 - B.x), s1 = mtv(B.R, a1 - B.x);
    float3 u = s1 - s0;
    float3 mid = (s0 + s1) * 0.5f;
    float h[3] = {B.p0, B.p1, B.p2};
    float ul = len(u);
    float3 uh = ul > 0.f ? u * (1.f / ul) : f3(0.f, 0.f, 0.f);
    float sep[6];
    float3 ax[6];
    bool valid[6];
#pragma unroll 1
    for (int i = 0; i < 6; i++) {
        float3 L;
        valid[i] = true;
        if (i < 3) L = axis3(i);
        else {
            float3 c = cross(axis3(i - 3), uh);
            float cn = len(c);
            if (cn < 1e-5f) { valid[i] = false; sep[i] = -3.0e38f; ax[i] = f3(0.f, 0.f, 0.f); continue; }
            L = c * (1.f / cn);
        }
        if (dot(mid, L) < 0.f) L = -L;
        float hb = h[0] * fabsf(L.x) + h[1] * fabsf(L.y) + h[2] * fabsf(L.z);
        float p0 = dot(s0, L), p1 = dot(s1, L);
        sep[i] = fminf(p0, p1) - hb - r;
        ax[i] = L;
    }
    float maxsep = -3.0e38f;
    for (int i = 0; i < 6; i++) if (valid[i] && sep[i] > maxsep) maxsep = sep[i];
    if (maxsep >= m) return;
    int bf = 0;
    for (int i = 1; i < 3; i++) if (sep[i] > sep[bf]) bf = i;
    int be = -1;
    for (int i = 3; i < 6; i++) if (valid[i] && (be < 0 || sep[i] > sep[be])) be = i;
    if (be >= 0 && sep[be] > sep[bf] + 1e-4f) {
        float3 L = ax[be];
        int i = be - 3;
        float3 q0 = f3((L.x >= 0.f ? 1.f : -1.f) * h[0], (L.y >= 0.f ? 1.f : -1.f) * h[1],
                       (L.z >= 0.f ? 1.f : -1.f) * h[2]);
        float3 q1 = with_comp(q0, i, h[i]);
        q0 = with_comp(q0, i, -h[i]);
        float3 ps, pe;
        closest_segments(s0, s1, q0, q1, ps, pe);
        float3 n = mv(B.R, L);
        cs.push(B.x + mv(B.R, ps - L * r), B.x + mv(B.R, pe), n, dot(L, ps - pe) - r);
        return;
    }
    int k = bf;
    float sigma = comp(ax[k], k) >= 0.f ? 1.f : -1.f;
    float tlo = 0.f, thi = 1.f;
    bool empty = false;
    for (int j = 0; j < 3; j++) {
        if (j == k) continue;
        float sj = comp(s0, j), uj = comp(u, j);
        if (uj == 0.f) { if (fabsf(sj) > h[j]) empty = true; continue; }
        float ta = (-h[j] - sj) / uj, tb = (h[j] - sj) / uj;
        tlo = fmaxf(tlo, fminf(ta, tb));
        thi = fminf(thi, fmaxf(ta, tb));
    }
    if (tlo > thi) empty = true;
    float3 nl = axis3(k) * sigma;
    float3 n = mv(B.R, nl);
    if (!empty) {
        int cnt = tlo == thi ? 1 : 2;
        for (int a = 0; a < cnt; a++) {
            float3 q = s0 + u * (a == 0 ? tlo : thi);
            float dist = sigma * comp(q, k) - h[k];
            float3 qb = with_comp(q, k, sigma * h[k]);
            float3 qa = q - nl * r;
            cs.push(B.x + mv(B.R, qa), B.x + mv(B.R, qb), n, dist - r);
        }
        return;
    }
    float t;
    float dist = segment_box_closest(s0, u, h, t);
    float3 q = s0 + u * t;
    float3 qb = f3(clampf(q.x, -h[0], h[0]), clampf(q.y, -h[1], h[1]), clampf(q.z, -h[2], h[2]));
    float3 dl = q - qb;
    float3 nn = dist > 1e-12f ? dl * (1.f / dist) : nl;
    cs.push(B.x + mv(B.R, q - nn * r), B.x + mv(B.R, qb), mv(B.R, nn), dist - r);
}

// box-plane: 8 vertices; index bits 0/1/2 select +-hx/hy/hz
MSD void np_bp(const Shape& A, const Shape& B, CandSet& cs) {
    float3 N = mcol(B.R, 2);
#pragma unroll
    for (int i = 0; i < 8; i++) {
        float3 lv = f3((i & 1) ? A.p0 : -A.p0, (i & 2) ? A.p1 : -A.p1, (i & 4) ? A.p2 : -A.p2);
        float3 v = A.x + mv(A.R, lv);
        float dist = dot(N, v - B.x);
        cs.push(v, v - N * dist, N, dist);
    }
}

// Sutherland-Hodgman against dir.(x - c) <= hh
MSD int clip_plane(const float3* in, int nin, float3* out, float3 dir, float3 c, float hh) {
    int nout = 0;
    if (nin == 0) return 0;
    float3 prev = in[nin - 1];
    float fp = dot(dir, prev - c) - hh;
    for (int i = 0; i < nin; i++) {
        float3 cur = in[i];
        float fc = dot(dir, cur - c) - hh;
        // a convex polygon gains at most one vertex per plane; the bound
        // also holds when rounding makes the input slightly non-convex
        if (fc <= 0.f) {
            if (fp > 0.f && nout < 8) out[nout++] = prev + (cur - prev) * (fp / (fp - fc));
            if (nout < 8) out[nout++] = cur;
        } else if (fp <= 0.f && nout < 8) {
            out[nout++] = prev + (cur - prev) * (fp / (fp - fc));
        }
        prev = cur;
        fp = fc;
    }
    return nout;
}

// box-box: SAT over 15 axes (A faces, B faces, A_i x B_j row major); a B
// face is the reference only if it beats the best A face by 1e-4 m, an edge
// pair only if it beats both by 1e-4 m
MSD void np_bb(const Shape& A, const Shape& B, float m, CandSet& cs) {
    float3 a[3], b[3];
#pragma unroll
    for (int i = 0; i < 3; i++) { a[i] = mcol(A.R, i); b[i] = mcol(B.R, i); }
    float hA[3] = {A.p0, A.p1, A.p2}, hB[3] = {B.p0, B.p1, B.p2};
    float3 dl = A.x - B.x;
    float sep[15];
    float3 ax[15];
    bool valid[15];
#pragma unroll 1
    for (int k = 0; k < 15; k++) {
        float3 L;
        valid[k] = true;
        if (k < 3) L = a[k];
        else if (k < 6) L = b[k - 3];
        else {
            float3 c = cross(a[(k - 6) / 3], b[(k - 6) % 3]);
            float cn = len(c);
            if (cn < 1e-5f) { valid[k] = false; sep[k] = -3.0e38f; ax[k] = f3(0.f, 0.f, 0.f); continue; }
            L = c * (1.f / cn);
        }
        if (dot(dl, L) < 0.f) L = -L;
        float ra = hA[0] * fabsf(dot(a[0], L)) + hA[1] * fabsf(dot(a[1], L)) + hA[2] * fabsf(dot(a[2], L));
        float rb = hB[0] * fabsf(dot(b[0], L)) + hB[1] * fabsf(dot(b[1], L)) + hB[2] * fabsf(dot(b[2], L));
        sep[k] = dot(dl, L) - ra - rb;
        ax[k] = L;
    }
    float maxsep = -3.0e38f;
    for (int k = 0; k < 15; k++) if (valid[k] && sep[k] > maxsep) maxsep = sep[k];
    if (maxsep >= m) return;
    int fa = 0, fb = 3, be = -1;
    for (int k = 1; k < 3; k++) if (sep[k] > sep[fa]) fa = k;
    for (int k = 4; k < 6; k++) if (sep[k] > sep[fb]) fb = k;
    for (int k = 6; k < 15; k++) if (valid[k] && (be < 0 || sep[k] > sep[be])) be = k;
    float sf = fmaxf(sep[fa], sep[fb]);
    if (be >= 0 && sep[be] > sf + 1e-4f) {
        float3 L = ax[be];
        int i = (be - 6) / 3, j = (be - 6) % 3;
        float3 ca = A.x, cb = B.x;
        for (int k = 0; k < 3; k++) {
            if (k != i) ca = ca + a[k] * ((dot(a[k], L) > 0.f ? -1.f : 1.f) * hA[k]);
            if (k != j) cb = cb + b[k] * ((dot(b[k], L) >= 0.f ? 1.f : -1.f) * hB[k]);
        }
        float3 pa, pb;
        closest_segments(ca - a[i] * hA[i], ca + a[i] * hA[i], cb - b[j] * hB[j], cb + b[j] * hB[j], pa, pb);
        cs.push(pa, pb, L, dot(L, pa - pb));
        return;
    }
    bool refB = sep[fb] > sep[fa] + 1e-4f;
    const Shape& Rf = refB ? B : A;
    const Shape& In = refB ? A : B;
    int k = refB ? fb - 3 : fa;
    float3 n = ax[refB ? fb : fa];
    float3 nref = refB ? n : -n;
    float hR[3] = {Rf.p0, Rf.p1, Rf.p2}, hI[3] = {In.p0, In.p1, In.p2};
    float3 cref = Rf.x + nref * hR[k];
    int ju = (k + 1) % 3, jv = (k + 2) % 3;
    float3 uu = mcol(Rf.R, ju), vv = mcol(Rf.R, jv);
    float hu = hR[ju], hv = hR[jv];
    int fi = 0;
    float fs = 1.f, best = 3.0e38f;
    for (int t = 0; t < 3; t++) {
        float3 ic = mcol(In.R, t);
        for (int s = 0; s < 2; s++) {
            float sg = s == 0 ? 1.f : -1.f;
            float dd = sg * dot(ic, nref);
            if (dd < best) { best = dd; fi = t; fs = sg; }
        }
    }
    int i1 = (fi + 1) % 3, i2 = (fi + 2) % 3;
    float3 fc = In.x + mcol(In.R, fi) * (fs * hI[fi]);
    float3 e1 = mcol(In.R, i1) * hI[i1], e2 = mcol(In.R, i2) * hI[i2];
    float3 poly[8], tmp[8];
    poly[0] = fc + e1 + e2;
    poly[1] = fc - e1 + e2;
    poly[2] = fc - e1 - e2;
    poly[3] = fc + e1 - e2;
    int np = 4;
    // the four side slabs +u, -u, +v, -v through one copy of the clipper
    // (even passes read poly and write tmp, odd passes the reverse)
    for (int c = 0; c < 4; c++) {
        float3 dir = c < 2 ? uu : vv;
        if (c & 1) dir = -dir;
        float hh = c < 2 ? hu : hv;
        np = clip_plane((c & 1) ? tmp : poly, np, (c & 1) ? poly : tmp, dir, cref, hh);
    }
    for (int t = 0; t < np; t++) {
        float3 x = poly[t];
        float dist = dot(nref, x - cref);
        float3 xp = x - nref * dist;
        if (refB) cs.push(x, xp, n, dist);
        else cs.push(xp, x, n, dist);
    }
}

// keep the deepest point, the one farthest from it, the one spanning the
// largest triangle with those two, and the one adding most area; ties go to
// the lowest candidate index; output in selection order
MSD int first_unused(unsigned used, int n) {
    for (int k = 0; k < n; k++)
        if (!(used >> k & 1u)) return k;
    return 0;
}

MSD void reduce4(const Cand* c, int n, int* sel) {
    unsigned used = 0;
    int i1 = 0;
    for (int k = 1; k < n; k++) if (c[k].d < c[i1].d) i1 = k;
    used |= 1u << i1;
    float best = -1.f;
    int i2 = first_unused(used, n);
    for (int k = 0; k < n; k++) {
        if (used >> k & 1u) continue;
        float3 dd = c[k].cB - c[i1].cB;
        float s = dot(dd, dd);
        if (s > best) { best = s; i2 = k; }
    }
    used |= 1u << i2;
    float3 e12 = c[i2].cB - c[i1].cB;
    int i3 = first_unused(used, n);
    best = -1.f;
    for (int k = 0; k < n; k++) {
        if (used >> k & 1u) continue;
        float s = len(cross(e12, c[k].cB - c[i1].cB));
        if (s > best) { best = s; i3 = k; }
    }
    used |= 1u << i3;
    float3 P1 = c[i1].cB, P2 = c[i2].cB, P3 = c[i3].cB;
    int i4 = first_unused(used, n);
    best = -1.f;
    for (int k = 0; k < n; k++) {
        if (used >> k & 1u) continue;
        float3 P = c[k].cB;
        float s = len(cross(P2 - P1, P - P1)) + len(cross(P3 - P2, P - P2)) + len(cross(P1 - P3, P - P3));
        if (s > best) { best = s; i4 = k; }
    }
    sel[0] = i1; sel[1] = i2; sel[2] = i3; sel[3] = i4;
}


// ------------------------------------------------------------------- hulls
// A convex polytope in world coordinates for the separating-axis test: a
// box (8 corners, 6 quadrilateral faces) or a hull (triangles).  World
// vertices and face planes are formed once; face vertex lists and edges
// are read from the hull library or the box tables.
constexpr int PV_MAXV = 16, PV_MAXF = 28, PV_MAXE = 42;

// box faces +x, -x, +y, -y, +z, -z, counter-clockwise from outside; corner
// k has signs (bit 0: x, bit 1: y, bit 2: z)
__device__ __constant__ int c_box_face[6][4] = {{1, 3, 7, 5}, {2, 0, 4, 6}, {3, 2, 6, 7},
                                               {0, 1, 5, 4}, {4, 5, 7, 6}, {2, 3, 1, 0}};
// box edges (a, b, face listing a -> b, face listing b -> a): each edge once,
// from the first face (in face order) that lists it with a < b
__device__ __constant__ int c_box_edge[12][4] = {{1, 3, 0, 5}, {3, 7, 0, 2}, {0, 4, 1, 3}, {4, 6, 1, 4},
                                                {2, 6, 2, 1}, {6, 7, 2, 4}, {0, 1, 3, 5}, {1, 5, 3, 0},
                                                {4, 5, 4, 3}, {5, 7, 4, 0}, {2, 3, 5, 2}, {0, 2, 5, 1}};

struct Poly {
    bool box;
    int nv, nf, ne;
    float3 c;                        // body origin (interior)
    float4 v[PV_MAXV];               // world vertices (w unused: 16-byte loads)
    float4 f[PV_MAXF];               // world face plane (n, n.x on the face)
    const int4* tri;
    const int4* edge;
};

MSD void poly_of(const Shape& S, Poly& P) {
    P.c = S.x;
    if (S.type == SH_BOX) {
        P.box = true; P.nv = 8; P.nf = 6; P.ne = 12;
        for (int k = 0; k < 8; k++)
            P.v[k] = f4(S.x + mv(S.R, f3((k & 1) ? S.p0 : -S.p0, (k & 2) ? S.p1 : -S.p1, (k & 4) ? S.p2 : -S.p2)), 0.f);
        const float h[3] = {S.p0, S.p1, S.p2};
        for (int f = 0; f < 6; f++) {
            float3 n = mcol(S.R, f >> 1) * ((f & 1) ? -1.f : 1.f);
            P.f[f] = f4(n, dot(n, S.x) + h[f >> 1]);
        }
        P.tri = nullptr; P.edge = nullptr;
    } else {
        const HullRef& H = S.hull;
        P.box = false; P.nv = H.nv; P.nf = H.nt; P.ne = H.ne;
        for (int k = 0; k < H.nv; k++) P.v[k] = f4(S.x + mv(S.R, xyz(H.v[k])), 0.f);
        for (int f = 0; f < H.nt; f++) {
            float4 ln = H.n[f];
            float3 n = mv(S.R, xyz(ln));
            P.f[f] = f4(n, dot(n, S.x) + ln.w);
        }
        P.tri = H.t; P.edge = H.e;
    }
}

MSD int poly_face(const Poly& P, int f, int* idx) {
    if (P.box) {
        for (int k = 0; k < 4; k++) idx[k] = c_box_face[f][k];
        return 4;
    }
    int4 t = P.tri[f];
    idx[0] = t.x; idx[1] = t.y; idx[2] = t.z;
    return 3;
}

MSD int4 poly_edge(const Poly& P, int k) {
    if (P.box) return make_int4(c_box_edge[k][0], c_box_edge[k][1], c_box_edge[k][2], c_box_edge[k][3]);
    return P.edge[k];
}

// hull - plane: every vertex within the margin (as box - plane)
MSD void np_hp(const Shape& A, const Shape& B, float m, CandSet& cs) {
    float3 N = mcol(B.R, 2);
    for (int k = 0; k < A.hull.nv; k++) {
        float3 v = A.x + mv(A.R, xyz(A.hull.v[k]));
        float dist = dot(N, v - B.x);
        if (dist < m + 1e-4f) cs.push(v, v - N * dist, N, dist);
    }
}

// closest point of triangle (a, b, c) to p (Ericson 2005, 5.1.5)
MSD float3 closest_on_triangle(float3 p, float3 a, float3 b, float3 c) {
    float3 ab = b - a, ac = c - a, ap = p - a;
    float d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= 0.f && d2 <= 0.f) return a;
    float3 bp = p - b;
    float d3 = dot(ab, bp), d4 = dot(ac, bp);
    if (d3 >= 0.f && d4 <= d3) return b;
    float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) return a + ab * (d1 / (d1 - d3));
    float3 cp = p - c;
    float d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= 0.f && d5 <= d6) return c;
    float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) return a + ac * (d2 / (d2 - d6));
    float va = d3 * d6 - d5 * d4;
    if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) return b + (c - b) * ((d4 - d3) / ((d4 - d3) + (d5 - d6)));
    float den = 1.f / (va + vb + vc);
    return a + ab * (vb * den) + ac * (vc * den);
}

// sphere - hull: centre inside every face plane: out along the face of
// least penetration; outside: the closest point of the surface
MSD void np_sh(const Shape& A, const Shape& B, CandSet& cs) {
    Poly P;
    poly_of(B, P);
    float3 c = A.x;
    float r = A.p0;
    float smax = -3e38f;
    int fb = 0;
    for (int f = 0; f < P.nf; f++) {
        float sf = dot(xyz(P.f[f]), c) - P.f[f].w;
        if (sf > smax) { smax = sf; fb = f; }
    }
    if (smax <= 0.f) {
        float3 n = xyz(P.f[fb]);
        cs.push(c - n * r, c - n * smax, n, smax - r);
        return;
    }
    float best = 3e38f;
    float3 q = c;
    for (int f = 0; f < P.nf; f++) {
        int idx[4];
        poly_face(P, f, idx);
        float3 t = closest_on_triangle(c, xyz(P.v[idx[0]]), xyz(P.v[idx[1]]), xyz(P.v[idx[2]]));
        float d2 = dot(c - t, c - t);
        if (d2 < best) { best = d2; q = t; }
    }
    float dist = sqrtf(best);
    float3 n = (c - q) * (1.f / dist);
    cs.push(c - n * r, q, n, dist - r);
}

// box or hull (A) - hull (B): separating axes over the face normals of A,
// then of B, then the cross products of edge pairs whose arcs on the Gauss
// map cross (the faces of the Minkowski difference); a B face is the
// reference only if it beats the best A face by 1e-4 m, an edge pair only
// if it beats the best face by 1e-4 m.  Face case: the most anti-parallel
// face of the other polytope clipped against the side planes of the
// reference face; edge case: the closest points of the two edges.
// The face axes of P against Q: the largest over P's faces of the least
// signed distance of Q's vertices to the face plane, and that face (the
// first maximum in face order).  Four planes at a time in registers, so a
// vertex of Q is loaded once per four faces.
MSD void face_axes(const Poly& P, const Poly& Q, float& smax, int& fmax_) {
    float s = -3e38f;
    int fi = 0;
    for (int f0 = 0; f0 < P.nf; f0 += 4) {
        float4 pl[4];
        float mn[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            pl[t] = P.f[min(f0 + t, P.nf - 1)];             // clamped; faces past nf are skipped
            mn[t] = 3e38f;
        }
        for (int k = 0; k < Q.nv; k++) {
            float3 v = xyz(Q.v[k]);
#pragma unroll
            for (int t = 0; t < 4; t++) mn[t] = fminf(mn[t], dot(xyz(pl[t]), v) - pl[t].w);
        }
#pragma unroll
        for (int t = 0; t < 4; t++)
            if (f0 + t < P.nf && mn[t] > s) { s = mn[t]; fi = f0 + t; }
    }
    smax = s;
    fmax_ = fi;
}

MSD void np_poly(const Shape& A, const Shape& B, float m, CandSet& cs) {
    Poly PA, PB;
    poly_of(A, PA);
    poly_of(B, PB);
    float sa, sb;
    int fa, fb;
    face_axes(PA, PB, sa, fa);
    face_axes(PB, PA, sb, fb);
    // the face axes already separate by the margin: no contact whatever the
    // edge pairs give (the largest separation is >= m); the bounding-sphere
    // broadphase passes many such pairs
    if (fmaxf(sa, sb) >= m) return;
    // B's edges as arcs on the Gauss map of -B: the negated normals of
    // their two faces and the arcs' plane normal, formed once per pair
    float4 bc[PV_MAXE], bd[PV_MAXE], bdxc[PV_MAXE];   // float4: one 16-byte load each
    for (int j = 0; j < PB.ne; j++) {
        int4 EB = poly_edge(PB, j);
        float3 c = -xyz(PB.f[EB.z]), d = -xyz(PB.f[EB.w]);
        bc[j] = f4(c, 0.f);
        bd[j] = f4(d, 0.f);
        bdxc[j] = f4(cross(d, c), 0.f);
    }
    float se = -3e38f; int ea = -1, eb = -1; float3 axe = f3(0.f, 0.f, 0.f);
    // B's arcs eight at a time in registers against every edge of A: an arc
    // is loaded once per eight (i, j) tests instead of once per test.  The
    // pairs are visited tile by tile, so the tie rule (equal separations:
    // the lowest i, then the lowest j) keeps the first maximum in i-major
    // order, as a plain double loop would find it.
    for (int j0 = 0; j0 < PB.ne; j0 += 8) {
        float3 cc[8], dd[8], xx[8];
#pragma unroll
        for (int t = 0; t < 8; t++) {
            int j = min(j0 + t, PB.ne - 1);               // clamped; tests past ne are skipped
            cc[t] = xyz(bc[j]); dd[t] = xyz(bd[j]); xx[t] = xyz(bdxc[j]);
        }
        for (int i = 0; i < PA.ne; i++) {
            int4 EA = poly_edge(PA, i);
            float3 a = xyz(PA.f[EA.z]), b = xyz(PA.f[EA.w]);
            float3 bxa = cross(b, a);
            // the eight Gauss-map tests unrolled; the rare pairs that pass
            // them go through one copy of the axis code, in order of j
            unsigned pass = 0u;
#pragma unroll
            for (int t = 0; t < 8; t++) {
                float cba = dot(cc[t], bxa), dba = dot(dd[t], bxa), adc = dot(a, xx[t]), bdc = dot(b, xx[t]);
                if (j0 + t < PB.ne && cba * dba < 0.f && adc * bdc < 0.f && cba * bdc > 0.f) pass |= 1u << t;
            }
            while (pass) {
                int j = j0 + __ffs(pass) - 1;
                pass &= pass - 1u;
                int4 EB = poly_edge(PB, j);
                float3 ua = xyz(PA.v[EA.y]) - xyz(PA.v[EA.x]);
                float3 ub = xyz(PB.v[EB.y]) - xyz(PB.v[EB.x]);
                float3 ax = cross(ua, ub);
                float l = len(ax);
                if (l < 1e-5f * len(ua) * len(ub)) continue;
                ax = ax * (1.f / l);
                if (dot(ax, xyz(PA.v[EA.x]) - PA.c) < 0.f) ax = -ax;
                float sij = dot(ax, xyz(PB.v[EB.x]) - xyz(PA.v[EA.x]));
                if (sij > se || (sij == se && (i < ea || (i == ea && j < eb)))) { se = sij; ea = i; eb = j; axe = ax; }
            }
        }
    }
    float maxsep = fmaxf(fmaxf(sa, sb), se);
    if (maxsep >= m) return;
    float sf = fmaxf(sa, sb);
    if (ea >= 0 && se > sf + 1e-4f) {
        int4 EA = poly_edge(PA, ea), EB = poly_edge(PB, eb);
        float3 pa, pb;
        closest_segments(xyz(PA.v[EA.x]), xyz(PA.v[EA.y]), xyz(PB.v[EB.x]), xyz(PB.v[EB.y]), pa, pb);
        float3 n = -axe;
        cs.push(pa, pb, n, dot(n, pa - pb));
        return;
    }
    bool refB = sb > sa + 1e-4f;
    const Poly& R = refB ? PB : PA;
    const Poly& I = refB ? PA : PB;
    int rf = refB ? fb : fa;
    float3 nref = xyz(R.f[rf]);
    int inc = 0;
    float best = 3e38f;
    for (int g = 0; g < I.nf; g++) {
        float dd = dot(xyz(I.f[g]), nref);
        if (dd < best) { best = dd; inc = g; }
    }
    float3 bufa[8], bufb[8];
    int ii[4], ri[4];
    int np = poly_face(I, inc, ii);
    for (int k = 0; k < np; k++) bufa[k] = xyz(I.v[ii[k]]);
    int nr = poly_face(R, rf, ri);
    for (int k = 0; k < nr; k++) {
        float3 p0 = xyz(R.v[ri[k]]), p1 = xyz(R.v[ri[k + 1 == nr ? 0 : k + 1]]);
        float3 side = cross(p1 - p0, nref);
        side = side * (1.f / len(side));
        // alternate the buffers: even k reads bufa, odd k reads bufb
        if ((k & 1) == 0) np = clip_plane(bufa, np, bufb, side, p0, 0.f);
        else np = clip_plane(bufb, np, bufa, side, p0, 0.f);
    }
    const float3* res = (nr & 1) ? bufb : bufa;
    float3 pref = xyz(R.v[ri[0]]);
    for (int k = 0; k < np; k++) {
        float3 x = res[k];
        float dist = dot(nref, x - pref);
        if (!refB) cs.push(x - nref * dist, x, -nref, dist);
        else cs.push(x, x - nref * dist, nref, dist);
    }
}


// closest points of segment [s0, s1] and the surface of polytope P (its
// triangles): per triangle, the segment's ends against the triangle and the
// segment against its edges; the least distance
MSD float segment_poly_closest(const Poly& P, float3 s0, float3 s1, float3& ps, float3& pq) {
    float best = 3e38f;
    for (int f = 0; f < P.nf; f++) {
        int idx[4];
        poly_face(P, f, idx);
        float3 tv[3] = {xyz(P.v[idx[0]]), xyz(P.v[idx[1]]), xyz(P.v[idx[2]])};
        float3 q = closest_on_triangle(s0, tv[0], tv[1], tv[2]);
        float d2 = dot(s0 - q, s0 - q);
        if (d2 < best) { best = d2; ps = s0; pq = q; }
        q = closest_on_triangle(s1, tv[0], tv[1], tv[2]);
        d2 = dot(s1 - q, s1 - q);
        if (d2 < best) { best = d2; ps = s1; pq = q; }
        for (int k = 0; k < 3; k++) {
            float3 a, b;
            closest_segments(s0, s1, tv[k], tv[k == 2 ? 0 : k + 1], a, b);
            d2 = dot(a - b, a - b);
            if (d2 < best) { best = d2; ps = a; pq = b; }
        }
    }
    return sqrtf(best);
}

// capsule - hull: separating axes over the hull's face normals and the
// segment x hull-edge axes (each in the orientation that separates more);
// an edge axis only if it beats the best face by 1e-4 m.  Face case: the
// segment clipped to the face's side planes (up to two points), or, when
// nothing of it lies over the face, the exact segment - surface closest
// points; edge case: those exact closest points (the edge that gives the
// axis need not support the hull along it).
MSD void np_ch(const Shape& A, const Shape& B, float m, CandSet& cs) {
    float r = A.p0;
    float3 s0, s1;
    capsule_ends(A, s0, s1);
    float3 u = s1 - s0;
    float ul = len(u);
    Poly P;
    poly_of(B, P);
    float sf = -3e38f; int bf = 0;
    for (int f = 0; f < P.nf; f++) {
        float3 n = xyz(P.f[f]);
        float sg = fminf(dot(n, s0), dot(n, s1)) - P.f[f].w - r;
        if (sg > sf) { sf = sg; bf = f; }
    }
    float se = -3e38f; int be = -1; float3 le = f3(0.f, 0.f, 0.f);
    for (int k = 0; k < P.ne; k++) {
        int4 E = poly_edge(P, k);
        float3 ev = xyz(P.v[E.y]) - xyz(P.v[E.x]);
        float3 c = cross(ev, u);
        float cn = len(c), lim = 1e-5f * len(ev) * ul;
        if (!(cn > lim)) continue;
        float3 L = c * (1.f / cn);
        float hmax = -3e38f, hmin = 3e38f;
        for (int q = 0; q < P.nv; q++) { float t = dot(L, xyz(P.v[q])); hmax = fmaxf(hmax, t); hmin = fminf(hmin, t); }
        float sp = fminf(dot(L, s0), dot(L, s1)) - hmax - r;
        float sn = hmin - fmaxf(dot(L, s0), dot(L, s1)) - r;
        if (sn > sp) { sp = sn; L = -L; }
        if (sp > se) { se = sp; be = k; le = L; }
    }
    float maxsep = fmaxf(sf, se);
    if (maxsep >= m) return;
    float3 n = xyz(P.f[bf]);
    float tlo = 0.f, thi = 1.f;
    bool empty = false;
    if (be >= 0 && se > sf + 1e-4f) {
        // the edge that gave the axis need not be the hull's support along
        // it: the exact closest points of segment and surface
        empty = true;
        n = le;
    }
    int idx[4];
    int nfv = poly_face(P, bf, idx);
    for (int k = 0; k < nfv && !empty; k++) {
        float3 p0 = xyz(P.v[idx[k]]), p1 = xyz(P.v[idx[k + 1 == nfv ? 0 : k + 1]]);
        float3 sd = cross(p1 - p0, n);
        sd = sd * (1.f / len(sd));
        float g0 = dot(sd, s0 - p0), gu = dot(sd, u);
        if (gu == 0.f) { if (g0 > 0.f) empty = true; continue; }
        float t = -g0 / gu;
        if (gu > 0.f) thi = fminf(thi, t); else tlo = fmaxf(tlo, t);
    }
    if (tlo > thi) empty = true;
    if (!empty) {
        int cnt = tlo == thi ? 1 : 2;
        for (int a = 0; a < cnt; a++) {
            float3 q = s0 + u * (a == 0 ? tlo : thi);
            float dist = dot(n, q) - P.f[bf].w;
            cs.push(q - n * r, q - n * dist, n, dist - r);
        }
        return;
    }
    float3 ps = s0, pq = xyz(P.v[0]);
    float dist = segment_poly_closest(P, s0, s1, ps, pq);
    float3 nn = dist > 1e-12f ? (ps - pq) * (1.f / dist) : n;
    cs.push(ps - nn * r, pq, nn, dist - r);
}

// Narrowphase of the ordered pair (A, B): up to 4 kept points in out.
// HULLS = false compiles the hull routines out (a batch without hulls).
template <bool HULLS = true>
MSD int collide(const Shape& A, const Shape& B, float m, Cand* out) {
    CandSet cs;
    cs.n = 0;
    int ta = A.type, tb = B.type;
    // box or hull against hull: one call site below, so the SAT is compiled once
    bool poly = false;
    if (ta == SH_SPHERE) {
        if (tb == SH_SPHERE) np_ss(A, B, cs);
        else if (tb == SH_CAPSULE) np_sc(A, B, cs);
        else if (tb == SH_BOX) np_sb(A, B, cs);
        else if (tb == SH_HULL) { if constexpr (HULLS) { if (B.hull.v) np_sh(A, B, cs); } }
        else np_sp(A, B, cs);
    } else if (ta == SH_CAPSULE) {
        if (tb == SH_CAPSULE) np_cc(A, B, cs);
        else if (tb == SH_BOX) np_cb(A, B, m, cs);
        else if (tb == SH_PLANE) np_cp(A, B, cs);
        else if (tb == SH_HULL) { if constexpr (HULLS) { if (B.hull.v) np_ch(A, B, m, cs); } }
    } else if (ta == SH_BOX) {
        if (tb == SH_BOX) np_bb(A, B, m, cs);
        else if (tb == SH_HULL) poly = HULLS && B.hull.v != nullptr;
        else np_bp(A, B, cs);
    } else if (HULLS && ta == SH_HULL && A.hull.v) {
        if (tb == SH_HULL) poly = B.hull.v != nullptr;
        else if (tb == SH_PLANE) np_hp(A, B, m, cs);
    }
    if constexpr (HULLS) {
        if (poly) np_poly(A, B, m, cs);
    }
    Cand kept[16];
    int nk = 0;
    for (int i = 0; i < cs.n; i++)
        if (cs.c[i].d < m) kept[nk++] = cs.c[i];
    if (nk <= 4) {
        for (int i = 0; i < nk; i++) out[i] = kept[i];
        return nk;
    }
    int sel[4];
    reduce4(kept, nk, sel);
    for (int i = 0; i < 4; i++) out[i] = kept[sel[i]];
    return 4;
}

}  // namespace ms
