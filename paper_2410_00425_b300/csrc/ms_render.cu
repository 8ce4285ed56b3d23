// Batched camera rendering: RGB, depth and segmentation of one camera per
// env from the resident body poses (the paper's parallel rendering of every
// env's camera, Sec. "GPU Parallelized Simulation and Rendering"; its 128 x
// 128 RGB observation, Appendix "Observation Space"), as a CUDA triangle
// rasteriser -- no graphics API.
//
// One CTA per env.  The env's z-buffer lives in shared memory as 64-bit keys
// (view depth bits << 32 | triangle index); every covering fragment does an
// atomicMin, so the surviving triangle -- least depth, then least index --
// does not depend on the order of the atomics.  Each lane sets up one
// triangle (pose, shade, back-face test, near clip, projection); the warp
// then rasterises its 32 triangles one at a time, lanes striding over the
// triangle's pixel bounding box.  A resolve pass writes RGBA8, depth and
// segmentation with coalesced stores.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/ms.h"
#include "ms_internal.h"
#include "ms_math.cuh"

namespace ms {

constexpr unsigned R_FULL = 0xffffffffu;

// Primitive meshes (body frame), counter-clockwise seen from outside: a vertex
// is (a, b, c, s) and maps to
//   box      (a hx, b hy, c hz)                      a, b, c in {-1, 1}
//   sphere   r (a, b, c)                             unit direction
//   capsule  r (a, b, c) + (0, 0, s l)               s in {-1, 0, 1}
//   plane    (a, b, c)                               the square [-2, 2]^2
// UV rings at polar angles k pi/6 (k = 1..5), 12 points each at azimuths
// 2 pi j / 12; the capsule's rings k = 1..3 sit at +l and k = 3..5 at -l.
struct MeshTables {
    std::vector<float4> vert;            // all types, concatenated
    std::vector<int> tri;                // a | b << 8 | c << 16, vertex indices local to the type
    int v0[4], t0[4], nt[4];             // per shape type: first vertex, first triangle, triangle count
};

static void round_mesh(MeshTables& M, int type, bool capsule) {
    const int NLON = 12, NLAT = 6;
    int base = (int)M.vert.size();
    M.v0[type] = base;
    M.t0[type] = (int)M.tri.size();
    std::vector<std::pair<int, float>> rings;   // (k, shift sign)
    if (capsule) {
        for (int k = 1; k <= 3; k++) rings.push_back({k, 1.f});
        for (int k = 3; k <= 5; k++) rings.push_back({k, -1.f});
    } else {
        for (int k = 1; k <= 5; k++) rings.push_back({k, 0.f});
    }
    int nr = (int)rings.size();
    for (int a = 0; a < nr; a++) {
        double th = M_PI * rings[a].first / NLAT;
        for (int j = 0; j < NLON; j++) {
            double ph = 2.0 * M_PI * j / NLON;
            M.vert.push_back(make_float4((float)(std::sin(th) * std::cos(ph)), (float)(std::sin(th) * std::sin(ph)),
                                         (float)std::cos(th), rings[a].second));
        }
    }
    int N = nr * NLON, S = N + 1;
    M.vert.push_back(make_float4(0.f, 0.f, 1.f, rings[0].second));
    M.vert.push_back(make_float4(0.f, 0.f, -1.f, rings[nr - 1].second));
    auto T = [&](int a, int b, int c) { M.tri.push_back(a | b << 8 | c << 16); };
    auto R = [&](int a, int j) { return a * NLON + (j % NLON); };
    for (int j = 0; j < NLON; j++) T(N, R(0, j), R(0, j + 1));
    for (int a = 0; a + 1 < nr; a++)
        for (int j = 0; j < NLON; j++) {
            T(R(a, j), R(a + 1, j), R(a + 1, j + 1));
            T(R(a, j), R(a + 1, j + 1), R(a, j + 1));
        }
    for (int j = 0; j < NLON; j++) T(S, R(nr - 1, j + 1), R(nr - 1, j));
    M.nt[type] = (int)M.tri.size() - M.t0[type];
}

static MeshTables build_meshes() {
    MeshTables M;
    // box: 8 corners, faces +x, -x, +y, -y, +z, -z as quads (a, b, c, d) -> (a, b, c), (a, c, d)
    M.v0[MS_BOX] = 0;
    M.t0[MS_BOX] = 0;
    for (int k = 0; k < 8; k++)
        M.vert.push_back(make_float4(k & 1 ? 1.f : -1.f, k & 2 ? 1.f : -1.f, k & 4 ? 1.f : -1.f, 0.f));
    auto C = [](int x, int y, int z) { return (x > 0 ? 1 : 0) | (y > 0 ? 2 : 0) | (z > 0 ? 4 : 0); };
    const int F[6][4][3] = {{{1, -1, -1}, {1, 1, -1}, {1, 1, 1}, {1, -1, 1}},
                            {{-1, 1, -1}, {-1, -1, -1}, {-1, -1, 1}, {-1, 1, 1}},
                            {{1, 1, -1}, {-1, 1, -1}, {-1, 1, 1}, {1, 1, 1}},
                            {{-1, -1, -1}, {1, -1, -1}, {1, -1, 1}, {-1, -1, 1}},
                            {{-1, -1, 1}, {1, -1, 1}, {1, 1, 1}, {-1, 1, 1}},
                            {{-1, 1, -1}, {1, 1, -1}, {1, -1, -1}, {-1, -1, -1}}};
    for (int f = 0; f < 6; f++) {
        int q[4];
        for (int k = 0; k < 4; k++) q[k] = C(F[f][k][0], F[f][k][1], F[f][k][2]);
        M.tri.push_back(q[0] | q[1] << 8 | q[2] << 16);
        M.tri.push_back(q[0] | q[2] << 8 | q[3] << 16);
    }
    M.nt[MS_BOX] = 12;
    round_mesh(M, MS_SPHERE, false);
    round_mesh(M, MS_CAPSULE, true);
    int pb = (int)M.vert.size();
    M.v0[MS_PLANE] = pb;
    M.t0[MS_PLANE] = (int)M.tri.size();
    M.vert.push_back(make_float4(-2.f, -2.f, 0.f, 0.f));
    M.vert.push_back(make_float4(2.f, -2.f, 0.f, 0.f));
    M.vert.push_back(make_float4(2.f, 2.f, 0.f, 0.f));
    M.vert.push_back(make_float4(-2.f, 2.f, 0.f, 0.f));
    M.tri.push_back(0 | 1 << 8 | 2 << 16);
    M.tri.push_back(0 | 2 << 8 | 3 << 16);
    M.nt[MS_PLANE] = 2;
    return M;
}

constexpr int R_NV = 8 + 62 + 74 + 4;      // template vertices
constexpr int R_NT = 12 + 120 + 144 + 2;   // template triangles
constexpr int R_THREADS = 256;

struct RenderCfg {
    float3 eye, rt, up, fw;
    float F, near;
    int W, H;
    int bands, band_rows;                  // image rows split over `bands` CTAs per env
    int max_tri;                           // largest triangle count of an env
    int max_nb;
    int v0[4], t0[4], nt[4];
    const float4* vert;                    // [R_NV]
    const int* tri;                        // [R_NT]
    const float* rgb;                      // [NB][3]
    uint32_t* out_rgba;                    // [E][H][W] or null
    float* out_depth;                      // [E][H][W] or null
    uint16_t* out_seg;                     // [E][H][W] or null
};

struct ScreenTri {
    float sx[3], sy[3], iz[3];
    float A;                               // signed screen area (x2)
    int x0, x1, y0, y1;                    // pixel bounding box (inclusive), empty if x1 < x0
};

__device__ __forceinline__ float3 local_vertex(float4 t, int type, float4 s) {
    if (type == MS_BOX) return f3(t.x * s.x, t.y * s.y, t.z * s.z);
    if (type == MS_SPHERE) return f3(t.x * s.x, t.y * s.x, t.z * s.x);
    if (type == MS_CAPSULE) return f3(t.x * s.x, t.y * s.x, fmaf(t.z, s.x, t.w * s.y));
    return f3(t.x, t.y, t.z);
}

// screen triangle of view-space a, b, c; its pixel bounding box is cut to rows [r0, r1)
__device__ __forceinline__ void screen_tri(const RenderCfg& R, float3 a, float3 b, float3 c, int r0, int r1,
                                           ScreenTri& s) {
    float3 q[3] = {a, b, c};
    float mnx = 3e38f, mxx = -3e38f, mny = 3e38f, mxy = -3e38f;
    for (int k = 0; k < 3; k++) {
        s.sx[k] = 0.5f * R.W + R.F * q[k].x / q[k].z;
        s.sy[k] = 0.5f * R.H - R.F * q[k].y / q[k].z;
        s.iz[k] = 1.f / q[k].z;
        mnx = fminf(mnx, s.sx[k]); mxx = fmaxf(mxx, s.sx[k]);
        mny = fminf(mny, s.sy[k]); mxy = fmaxf(mxy, s.sy[k]);
    }
    s.A = (s.sx[1] - s.sx[0]) * (s.sy[2] - s.sy[0]) - (s.sy[1] - s.sy[0]) * (s.sx[2] - s.sx[0]);
    // pixel centres (p + 0.5) inside [mn, mx]; clamped before conversion
    mnx = fminf(fmaxf(mnx - 0.5f, -1.f), (float)R.W);
    mxx = fminf(fmaxf(mxx - 0.5f, -1.f), (float)R.W);
    mny = fminf(fmaxf(mny - 0.5f, -1.f), (float)R.H);
    mxy = fminf(fmaxf(mxy - 0.5f, -1.f), (float)R.H);
    s.x0 = max((int)ceilf(mnx), 0); s.x1 = min((int)floorf(mxx), R.W - 1);
    s.y0 = max((int)ceilf(mny), r0); s.y1 = min((int)floorf(mxy), r1 - 1);
    if (s.A == 0.f || !(s.A == s.A)) s.x1 = s.x0 - 1;          // degenerate or non-finite: nothing
}

// Screen triangle records in shared memory: 13 words each -- sx[3], sy[3],
// iz[3], A, x0 | x1 << 16, y0 | y1 << 16, triangle index.
constexpr int R_REC = 13;
constexpr int R_WARPS = R_THREADS / 32;

__device__ __forceinline__ void put_rec(float* rec, const ScreenTri& s, unsigned id) {
    for (int k = 0; k < 3; k++) { rec[k] = s.sx[k]; rec[3 + k] = s.sy[k]; rec[6 + k] = s.iz[k]; }
    rec[9] = s.A;
    rec[10] = __int_as_float(s.x0 | s.x1 << 16);
    rec[11] = __int_as_float(s.y0 | s.y1 << 16);
    rec[12] = __uint_as_float(id);
}

// pixels [p0, p0 + n) (row-major in the record's bounding box), lanes of the
// warp together; the surviving key per pixel is the least (depth, index)
__device__ __forceinline__ void raster_span(const RenderCfg& R, const float* rec, int p0, int n,
                                            unsigned long long* zb, int r0, int lane) {
    float sx[3], sy[3], iz[3];
    for (int k = 0; k < 3; k++) { sx[k] = rec[k]; sy[k] = rec[3 + k]; iz[k] = rec[6 + k]; }
    float A = rec[9];
    int bx = __float_as_int(rec[10]), by = __float_as_int(rec[11]);
    unsigned id = __float_as_uint(rec[12]);
    int x0 = bx & 0xffff, x1 = bx >> 16, y0 = by & 0xffff;
    int bw = x1 - x0 + 1;
    float sg = A > 0.f ? 1.f : -1.f, sa = fabsf(A);
    for (int q = lane; q < n; q += 32) {
        int p = p0 + q;
        int py = y0 + p / bw, px = x0 + p % bw;
        float x = px + 0.5f, y = py + 0.5f;
        float w[3];
        for (int k = 0; k < 3; k++) {
            int a = k == 2 ? 0 : k + 1, c = k == 0 ? 2 : (k == 1 ? 0 : 1);
            w[k] = sg * ((sx[c] - sx[a]) * (y - sy[a]) - (sy[c] - sy[a]) * (x - sx[a]));
        }
        if (w[0] < 0.f || w[1] < 0.f || w[2] < 0.f) continue;
        float izp = (w[0] * iz[0] + w[1] * iz[1] + w[2] * iz[2]) / sa;
        float z = 1.f / izp;
        if (!(z > 0.f)) continue;
        unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | id;
        atomicMin(zb + (py - r0) * R.W + px, key);
    }
}

// shared-memory sections of k_render, each 16-byte aligned
struct RenderSmem {
    size_t vert, tri, rgb, base, list, pre, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline RenderSmem render_smem(int W, int band_rows, int max_tri, int max_nb) {
    RenderSmem m;
    m.vert = align16((size_t)W * band_rows * 8);
    m.tri = m.vert + sizeof(float4) * R_NV;
    m.rgb = align16(m.tri + sizeof(int) * R_NT);
    m.base = align16(m.rgb + sizeof(uint32_t) * max_tri);
    m.list = align16(m.base + sizeof(int) * (max_nb + 2));                 // + the list count
    m.pre = align16(m.list + sizeof(float) * R_REC * 2 * R_THREADS);       // two records per triangle of a chunk
    m.total = align16(m.pre + sizeof(int) * (2 * R_THREADS + 1));
    return m;
}

// One CTA per env.  Triangles are taken R_THREADS at a time: each thread
// sets up one (its packed colour, and up to two clipped screen triangles
// appended to a shared list); then the list's pixel bounding boxes are laid
// end to end and every warp rasterises an equal share of that pixel range,
// so one large triangle (the ground) is spread over all warps.
__global__ void __launch_bounds__(R_THREADS) k_render(DevBatch D, RenderCfg R) {
    extern __shared__ __align__(16) char smem[];
    int env = blockIdx.x / R.bands, band = blockIdx.x % R.bands;
    const int r0 = band * R.band_rows, r1 = min(R.H, r0 + R.band_rows);
    const int P = R.W * (r1 - r0);                                     // this band's pixels
    RenderSmem m = render_smem(R.W, R.band_rows, R.max_tri, R.max_nb);
    unsigned long long* zb = reinterpret_cast<unsigned long long*>(smem);
    float4* vert = reinterpret_cast<float4*>(smem + m.vert);
    int* tri = reinterpret_cast<int*>(smem + m.tri);
    uint32_t* trgb = reinterpret_cast<uint32_t*>(smem + m.rgb);         // packed colour per triangle
    int* tbase = reinterpret_cast<int*>(smem + m.base);                 // first triangle of each body, + total
    float* list = reinterpret_cast<float*>(smem + m.list);
    int* pre = reinterpret_cast<int*>(smem + m.pre);                    // exclusive prefix of the bbox areas
    int b0 = D.body_off[env], nb = D.body_off[env + 1] - b0;
    int* cnt = tbase + nb + 1;
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long EMPTY = ~0ull;
    for (int i = tid; i < P; i += R_THREADS) zb[i] = EMPTY;
    for (int i = tid; i < R_NV; i += R_THREADS) vert[i] = R.vert[i];
    for (int i = tid; i < R_NT; i += R_THREADS) tri[i] = R.tri[i];
    if (warp == 0) {                                                   // triangle offsets of the bodies
        int run = 0;
        for (int i0 = 0; i0 < nb; i0 += 32) {
            int i = i0 + lane;
            int n = 0;
            if (i < nb) {
                int ty = D.meta[b0 + i].x & 0xff;
                if (ty == MS_HULL) {
                    int h = (int)D.shape[b0 + i].x;
                    n = D.hulls ? D.hulls->to[h + 1] - D.hulls->to[h] : 0;
                } else {
                    n = R.nt[ty];
                }
            }
            int incl = n;
            for (int d = 1; d < 32; d <<= 1) {
                int t = __shfl_up_sync(R_FULL, incl, d);
                if (lane >= d) incl += t;
            }
            if (i < nb) tbase[i] = run + incl - n;
            run += __shfl_sync(R_FULL, incl, 31);
        }
        if (lane == 0) tbase[nb] = run;
    }
    __syncthreads();
    int ntri = tbase[nb];
    float3 L = f3(0.3f, 0.2f, 1.f);                                    // light direction
    L = L * (1.f / len(L));
    for (int c0 = 0; c0 < ntri; c0 += R_THREADS) {
        if (tid == 0) *cnt = 0;
        __syncthreads();
        int t = c0 + tid;
        if (t < ntri) {
            int bi = 0;                                                // body of triangle t
            while (bi + 1 < nb && tbase[bi + 1] <= t) bi++;
            int type = D.meta[b0 + bi].x & 0xff;
            float4 shp = D.shape[b0 + bi];
            float3 x = xyz(D.x[b0 + bi]);
            M3 Rb = qmat(D.q[b0 + bi]);
            float3 w[3], v[3];
            int tv = 0;
            const float4* hv = nullptr;
            if (type == MS_HULL) {                                     // a hull: its library mesh
                int h = (int)shp.x;
                int4 ht = D.hulls->t[D.hulls->to[h] + t - tbase[bi]];
                tv = ht.x | ht.y << 8 | ht.z << 16;
                hv = D.hulls->v + D.hulls->vo[h];
            } else {
                tv = tri[R.t0[type] + t - tbase[bi]];
            }
            for (int k = 0; k < 3; k++) {
                int vi = (tv >> (8 * k)) & 0xff;
                float3 p = hv ? xyz(hv[vi]) : local_vertex(vert[R.v0[type] + vi], type, shp);
                w[k] = x + mv(Rb, p);
                float3 d = w[k] - R.eye;
                v[k] = f3(dot(R.rt, d), dot(R.up, d), dot(R.fw, d));
            }
            float3 n = cross(w[1] - w[0], w[2] - w[0]);
            float nl = len(n);
            float shade = nl > 0.f ? 0.3f + 0.7f * fmaxf(0.f, dot(n, L) / nl) : 0.3f;
            const float* base = R.rgb + 3 * (size_t)(b0 + bi);
            uint32_t rgba = 0xff000000u;
            for (int ch = 0; ch < 3; ch++) {
                float val = floorf(base[ch] * shade * 255.f + 0.5f);
                rgba |= (uint32_t)fminf(fmaxf(val, 0.f), 255.f) << (8 * ch);
            }
            trgb[t] = rgba;
            if (dot(n, w[0] - R.eye) < 0.f) {                          // front-facing
                float3 poly[4];
                int np = 0;
                for (int k = 0; k < 3; k++) {
                    float3 a = v[k], c = v[k == 2 ? 0 : k + 1];
                    float da = a.z - R.near, dc = c.z - R.near;
                    if (da >= 0.f) poly[np++] = a;
                    if ((da >= 0.f) != (dc >= 0.f)) {
                        float sgm = da / (da - dc);
                        poly[np++] = a + (c - a) * sgm;
                    }
                }
                for (int f = 0; f + 2 < np; f++) {
                    ScreenTri s;
                    screen_tri(R, poly[0], poly[f + 1], poly[f + 2], r0, r1, s);
                    if (s.x1 >= s.x0 && s.y1 >= s.y0) {
                        int slot = atomicAdd(cnt, 1);                  // list order is free: keys decide
                        put_rec(list + (size_t)R_REC * slot, s, (unsigned)t);
                    }
                }
            }
        }
        __syncthreads();
        int nl = *cnt;
        if (warp == 0) {                                               // prefix of the bbox areas
            int per = (nl + 31) / 32, lo = min(lane * per, nl), hi = min(lo + per, nl);
            int sum = 0;
            for (int i = lo; i < hi; i++) {
                const float* r = list + (size_t)R_REC * i;
                int bx = __float_as_int(r[10]), by = __float_as_int(r[11]);
                sum += ((bx >> 16) - (bx & 0xffff) + 1) * ((by >> 16) - (by & 0xffff) + 1);
            }
            int incl = sum;
            for (int d = 1; d < 32; d <<= 1) {
                int u = __shfl_up_sync(R_FULL, incl, d);
                if (lane >= d) incl += u;
            }
            int run = incl - sum;
            for (int i = lo; i < hi; i++) {
                pre[i] = run;
                const float* r = list + (size_t)R_REC * i;
                int bx = __float_as_int(r[10]), by = __float_as_int(r[11]);
                run += ((bx >> 16) - (bx & 0xffff) + 1) * ((by >> 16) - (by & 0xffff) + 1);
            }
            if (lane == 31) pre[nl] = incl;
        }
        __syncthreads();
        int total = pre[nl];
        int pos = (int)((long long)total * warp / R_WARPS), end = (int)((long long)total * (warp + 1) / R_WARPS);
        if (pos < end) {
            int lo = 0, hi = nl - 1;                                   // last entry with pre <= pos
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (pre[mid] <= pos) lo = mid; else hi = mid - 1;
            }
            for (int e = lo; pos < end && e < nl; e++) {
                int stop = min(end, pre[e + 1]);
                if (stop > pos) raster_span(R, list + (size_t)R_REC * e, pos - pre[e], stop - pos, zb, r0, lane);
                pos = max(pos, stop);
            }
        }
        __syncthreads();
    }
    size_t o = (size_t)env * R.W * R.H + (size_t)r0 * R.W;
    for (int i = tid; i < P; i += R_THREADS) {
        unsigned long long key = zb[i];
        uint32_t rgba = 0u;
        float z = 0.f;
        uint16_t sg = 0;
        if (key != EMPTY) {
            unsigned t = (unsigned)(key & 0xffffffffu);
            z = __uint_as_float((unsigned)(key >> 32));
            rgba = trgb[t];
            int bi = 0;
            while (bi + 1 < nb && tbase[bi + 1] <= (int)t) bi++;
            sg = (uint16_t)(bi + 1);
        }
        if (R.out_rgba) R.out_rgba[o + i] = rgba;
        if (R.out_depth) R.out_depth[o + i] = z;
        if (R.out_seg) R.out_seg[o + i] = sg;
    }
}

size_t render_smem_bytes(int W, int band_rows, int max_tri, int max_nb) {
    return render_smem(W, band_rows, max_tri, max_nb).total;
}

// ----------------------------------------------------------------- host side
struct RenderState {
    RenderCfg cfg{};
    float4* d_vert = nullptr;
    int* d_tri = nullptr;
    float* d_rgb = nullptr;
    size_t smem = 0;
    bool ready = false;
};

RenderState* render_create() { return new RenderState(); }

void render_destroy(RenderState* r) {
    if (!r) return;
    cudaFree(r->d_vert);
    cudaFree(r->d_tri);
    cudaFree(r->d_rgb);
    delete r;
}

// validates the camera and uploads the meshes and colours; returns an
// error message or null
const char* render_configure(RenderState* r, const DevBatch& D, const ms_camera_desc* c,
                             const std::vector<uint8_t>& types, const std::vector<int>& hull_nt,
                             const std::vector<int>& body_off, int max_nb, int smem_optin) {
    if (!(c->width >= 1 && c->height >= 1 && (long long)c->width * c->height <= 16384))
        return "width x height must be in [1, 16384]";
    if (!(c->fov_y > 0.f && c->fov_y < 3.14159f) || !(c->near > 0.f) || !std::isfinite(c->near))
        return "fov_y must be in (0, pi) and near > 0";
    double e[3] = {c->eye[0], c->eye[1], c->eye[2]};
    double f[3] = {c->target[0] - e[0], c->target[1] - e[1], c->target[2] - e[2]};
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fl > 0.0) || !std::isfinite(fl)) return "eye and target must differ";
    for (double& v : f) v /= fl;
    double rt[3] = {f[1], -f[0], 0.0};                       // f x (0, 0, 1)
    double rl = std::sqrt(rt[0] * rt[0] + rt[1] * rt[1]);
    if (rl < 1e-9) return "the view direction must not be vertical";
    for (double& v : rt) v /= rl;
    double up[3] = {rt[1] * f[2] - rt[2] * f[1], rt[2] * f[0] - rt[0] * f[2], rt[0] * f[1] - rt[1] * f[0]};
    int E = (int)body_off.size() - 1, NB = body_off.back();
    for (int i = 0; i < 3 * NB; i++)
        if (!(c->body_rgb[i] >= 0.f && c->body_rgb[i] <= 1.f)) return "body_rgb must be in [0, 1]";
    MeshTables M = build_meshes();
    if ((int)M.vert.size() != R_NV || (int)M.tri.size() != R_NT) return "internal mesh table size";
    int max_tri = 0;
    for (int env = 0; env < E; env++) {
        int n = 0;
        for (int i = body_off[env]; i < body_off[env + 1]; i++) n += types[i] == MS_HULL ? hull_nt[i] : M.nt[types[i]];
        max_tri = std::max(max_tri, n);
    }
    // rows per CTA: the fewest bands whose CTAs fit two to an SM (about 113
    // KB of shared memory each), so that one CTA's barrier waits overlap the
    // other's work; the whole image in one CTA if nothing smaller fits better
    int bands = 1;
    size_t smem = render_smem_bytes(c->width, c->height, std::max(max_tri, 1), max_nb);
    for (int nbands = 1; nbands <= 8; nbands *= 2) {
        int rows = (c->height + nbands - 1) / nbands;
        size_t sm = render_smem_bytes(c->width, rows, std::max(max_tri, 1), max_nb);
        bands = nbands; smem = sm;
        if (sm <= 110 * 1024) break;
    }
    if (smem > (size_t)smem_optin) return "image too large for the shared-memory z-buffer";
    cudaFree(r->d_vert); cudaFree(r->d_tri); cudaFree(r->d_rgb);
    r->d_vert = nullptr; r->d_tri = nullptr; r->d_rgb = nullptr;
    if (cudaMalloc(&r->d_vert, sizeof(float4) * R_NV) != cudaSuccess ||
        cudaMalloc(&r->d_tri, sizeof(int) * R_NT) != cudaSuccess ||
        cudaMalloc(&r->d_rgb, sizeof(float) * 3 * std::max(NB, 1)) != cudaSuccess)
        return "out of device memory";
    cudaMemcpy(r->d_vert, M.vert.data(), sizeof(float4) * R_NV, cudaMemcpyHostToDevice);
    cudaMemcpy(r->d_tri, M.tri.data(), sizeof(int) * R_NT, cudaMemcpyHostToDevice);
    cudaMemcpy(r->d_rgb, c->body_rgb, sizeof(float) * 3 * NB, cudaMemcpyHostToDevice);
    RenderCfg& R = r->cfg;
    R.eye = make_float3((float)e[0], (float)e[1], (float)e[2]);
    R.fw = make_float3((float)f[0], (float)f[1], (float)f[2]);
    R.rt = make_float3((float)rt[0], (float)rt[1], (float)rt[2]);
    R.up = make_float3((float)up[0], (float)up[1], (float)up[2]);
    R.F = (float)(0.5 * c->height / std::tan(0.5 * (double)c->fov_y));
    R.near = c->near;
    R.W = c->width; R.H = c->height;
    R.bands = bands;
    R.band_rows = (c->height + bands - 1) / bands;
    R.max_tri = std::max(max_tri, 1);
    R.max_nb = max_nb;
    for (int k = 0; k < 4; k++) { R.v0[k] = M.v0[k]; R.t0[k] = M.t0[k]; R.nt[k] = M.nt[k]; }
    R.vert = r->d_vert; R.tri = r->d_tri; R.rgb = r->d_rgb;
    r->smem = smem;
    cudaFuncSetAttribute((const void*)k_render, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    r->ready = true;
    (void)D;
    return nullptr;
}

bool render_ready(const RenderState* r) { return r && r->ready; }

cudaError_t render_launch(RenderState* r, const DevBatch& D, uint8_t* rgba, float* depth, uint16_t* seg,
                          cudaStream_t s) {
    RenderCfg R = r->cfg;
    R.out_rgba = reinterpret_cast<uint32_t*>(rgba);
    R.out_depth = depth;
    R.out_seg = seg;
    if (D.E > 0) k_render<<<D.E * R.bands, R_THREADS, r->smem, s>>>(D, R);
    return cudaGetLastError();
}

}  // namespace ms
