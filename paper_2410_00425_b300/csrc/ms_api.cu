// Host side of the C ABI declared in include/ms.h.
//
// A batch keeps every env's state resident on the device as a structure of
// arrays with CSR offsets per env (the paper's data-oriented layout of
// objects and articulations, Sec. "Heterogeneous GPU Simulation").  ms_step
// replays a captured CUDA graph of the batched persistent kernel;
// ms_step_plain launches the per-stage kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <numeric>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/ms.h"
#include "ms_internal.h"

using namespace ms;

static thread_local std::string g_err;

static ms_status fail(ms_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                    \
    } while (0)

namespace {

struct GraphEntry {
    cudaGraph_t graph = nullptr;      // kept alive: the exec's node handles refer to it
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t kernel = nullptr;
    cudaKernelNodeParams kp{};
};

struct Tuning {
    int G = 32, warps = 4, rows_smem = 1;
};

}  // namespace

struct ms_batch {
    int device = 0;
    int E = 0, NB = 0, NJ = 0, A = 0, max_nb = 0, max_nj = 0;
    ms_sim_params params{};
    DevBatch D{};
    // device allocations
    std::vector<void*> allocs;
    int* d_body_env = nullptr;
    float* d_staging = nullptr;
    uint8_t* d_mask = nullptr;
    int* d_queue = nullptr;
    int* d_order = nullptr;
    char* d_gscratch = nullptr;
    size_t gscratch_bytes = 0;
    float* d_hact = nullptr;          // ms_step_host: device copy of the host actions
    size_t hact_cap = 0;              //   its capacity in floats
    float* d_hrec = nullptr;          // ms_step_host: device task records before the copy out
    size_t hrec_cap = 0;
    size_t bytes = 0;
    bool record = false;
    void* rec_keep[4] = {nullptr, nullptr, nullptr, nullptr};   // record buffers, kept while recording is off
    int rec_stride = 0;                                       // colours per env in the record
    // batched path
    Tuning tune;
    Layout fused_layout{};
    int fused_threads = 0, fused_grid = 0, fused_ctas_per_sm = 0;
    size_t fused_smem = 0;
    bool fused_ready = false;
    unsigned fused_var = 0;           // the configured kernel variant (FV_* bits)
    std::map<long long, GraphEntry> graphs;
    // recorded after the batch's last enqueued work, on whatever stream it
    // went to: waiting on it never touches a stream the caller may have
    // destroyed since
    cudaEvent_t done = nullptr;
    cudaStream_t setup = nullptr;     // non-blocking stream for allocation and uploads
    ms_alloc_fn alloc_fn = nullptr;   // the device-memory hook the batch was created under (null: own pool)
    ms_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    int sm_count = 0;
    size_t smem_optin = 0;
    std::vector<int> h_body_off, h_joint_off;
    std::vector<uint8_t> h_type;      // shape type per body
    std::vector<int> h_hull_nt;       // triangles of each hull body's mesh (0 otherwise)
    // pick task
    float* d_task_half = nullptr;     // [A]
    float* d_task_qR = nullptr;       // [NJ]
    std::vector<float> h_task_half;
    RenderState* render = nullptr;
    float4* d_force = nullptr;        // contact forces per body (allocated on first use)
};

// The device-memory hook of batches created from now on (ms_set_allocator).
static std::mutex g_alloc_mu;
static ms_alloc_fn g_alloc_fn = nullptr;
static ms_free_fn g_free_fn = nullptr;
static void* g_alloc_user = nullptr;

extern "C" ms_status ms_set_allocator(ms_alloc_fn alloc, ms_free_fn free_, void* user) {
    if ((alloc == nullptr) != (free_ == nullptr)) return fail(MS_ERR_INVALID_ARG, "set both functions or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc_fn = alloc;
    g_free_fn = free_;
    g_alloc_user = user;
    return MS_OK;
}

// Device memory comes from the device's stream-ordered pool on the batch's
// own non-blocking stream: creating a batch (or a server session) neither
// waits for nor stalls work running on other streams.
static ms_status dmalloc(ms_batch* b, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b->alloc_fn) {
        *p = b->alloc_fn(bytes, b->device, (void*)b->setup, b->alloc_user);
        if (!*p) return fail(MS_ERR_OOM, "the device-memory hook returned NULL for %zu bytes", bytes);
        b->allocs.push_back(*p);
        b->bytes += bytes;
        return MS_OK;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, b->setup);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->setup);
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA,
                                      "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    b->allocs.push_back(*p);
    b->bytes += bytes;
    return MS_OK;
}

template <typename T>
static ms_status upload(ms_batch* b, T** dst, const std::vector<T>& src) {
    ms_status s = dmalloc(b, (void**)dst, sizeof(T) * std::max<size_t>(src.size(), 1));
    if (s) return s;
    if (!src.empty()) CK(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, b->setup));
    return MS_OK;
}

static void drop_graphs(ms_batch* b) {
    for (auto& kv : b->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    b->graphs.clear();
}

// The batch's use of a task, contact forces or a contact record changed:
// the batched kernel (lean or not) is chosen again at the next step.
static void kernel_choice_changed(ms_batch* b) {
    b->fused_ready = false;
    drop_graphs(b);
}

static void free_all(ms_batch* b) {
    drop_graphs(b);
    render_destroy(b->render);
    b->render = nullptr;
    if (b->free_fn) {
        if (b->setup) cudaStreamSynchronize(b->setup);
        for (void* p : b->allocs) b->free_fn(p, b->device, (void*)b->setup, b->alloc_user);
    } else {
        for (void* p : b->allocs) cudaFreeAsync(p, b->setup);
    }
    b->allocs.clear();
    if (b->setup) {
        cudaStreamSynchronize(b->setup);
        cudaStreamDestroy(b->setup);
        b->setup = nullptr;
    }
    if (b->done) {
        cudaEventDestroy(b->done);
        b->done = nullptr;
    }
}

static bool finite3(const float* v, int n) {
    for (int i = 0; i < n; i++)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Body-frame principal inertia of a uniform solid of the given mass.
static void body_inertia(const ms_body_desc& d, float out[3]) {
    double I[3];
    primitive_inertia(d.type, d.mass, d.p[0], d.p[1], d.p[2], I);
    for (int k = 0; k < 3; k++) out[k] = (float)I[k];
}

// ------------------------------------------------------------------- hulls
// The library's derived data: edges (each once, from the triangle listing it
// a -> b with a < b, with the triangle listing b -> a), local face planes,
// bounding radius; volume and diagonal second moments of unit density from
// the tetrahedra (origin, triangle), each (V/20)(a a + b b + c c + s s),
// s = a + b + c, per axis.
struct HostHulls {
    int n = 0;
    std::vector<float4> v, n4;
    std::vector<int4> t, e;
    std::vector<int> vo{0}, to{0}, eo{0};
    std::vector<float> rad;
    std::vector<double> vol, c2;          // c2: 3 per hull
};

static ms_status build_hulls(const ms_hull_lib* L, HostHulls& H) {
    if (!L) return MS_OK;
    if (L->n_hulls < 0 || (L->n_hulls > 0 && (!L->vert_off || !L->verts || !L->tri_off || !L->tris)))
        return fail(MS_ERR_INVALID_ARG, "hull library: NULL table");
    H.n = L->n_hulls;
    for (int h = 0; h < H.n; h++) {
        int v0 = L->vert_off[h], nv = L->vert_off[h + 1] - v0, t0 = L->tri_off[h], nt = L->tri_off[h + 1] - t0;
        if (nv < 4 || nv > 16 || nt < 4 || nt > 2 * 16 - 4) return fail(MS_ERR_INVALID_ARG, "hull %d: %d vertices / %d triangles", h, nv, nt);
        std::vector<double> pv(3 * nv);
        double rad = 0.0;
        for (int k = 0; k < nv; k++) {
            const float* q = L->verts + 3 * (size_t)(v0 + k);
            if (!finite3(q, 3)) return fail(MS_ERR_INVALID_ARG, "hull %d: non-finite vertex", h);
            for (int c = 0; c < 3; c++) pv[3 * k + c] = q[c];
            rad = std::max(rad, std::sqrt(pv[3 * k] * pv[3 * k] + pv[3 * k + 1] * pv[3 * k + 1] + pv[3 * k + 2] * pv[3 * k + 2]));
            H.v.push_back(make_float4(q[0], q[1], q[2], 0.f));
        }
        const int32_t* tt = L->tris + 3 * (size_t)t0;
        for (int f = 0; f < 3 * nt; f++)
            if (tt[f] < 0 || tt[f] >= nv) return fail(MS_ERR_INVALID_ARG, "hull %d: vertex index out of range", h);
        double vol = 0.0, c2[3] = {0.0, 0.0, 0.0};
        for (int f = 0; f < nt; f++) {
            const double* a = &pv[3 * tt[3 * f]];
            const double* b = &pv[3 * tt[3 * f + 1]];
            const double* c = &pv[3 * tt[3 * f + 2]];
            double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, ac[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
            double n[3] = {ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2], ab[0] * ac[1] - ab[1] * ac[0]};
            double nl = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            if (!(nl > 0.0)) return fail(MS_ERR_INVALID_ARG, "hull %d: degenerate triangle %d", h, f);
            for (double& x : n) x /= nl;
            H.n4.push_back(make_float4((float)n[0], (float)n[1], (float)n[2], (float)(n[0] * a[0] + n[1] * a[1] + n[2] * a[2])));
            H.t.push_back(make_int4(tt[3 * f], tt[3 * f + 1], tt[3 * f + 2], 0));
            double v6 = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
            vol += v6 / 6.0;
            for (int k = 0; k < 3; k++) {
                double sm = a[k] + b[k] + c[k];
                c2[k] += v6 / 120.0 * (a[k] * a[k] + b[k] * b[k] + c[k] * c[k] + sm * sm);
            }
        }
        int ne = 0;
        for (int f = 0; f < nt; f++)
            for (int k = 0; k < 3; k++) {
                int a = tt[3 * f + k], bb = tt[3 * f + (k + 1) % 3];
                if (a > bb) continue;
                int g = -1;
                for (int o = 0; o < nt && g < 0; o++)
                    for (int q = 0; q < 3; q++)
                        if (tt[3 * o + q] == bb && tt[3 * o + (q + 1) % 3] == a) { g = o; break; }
                if (g < 0) return fail(MS_ERR_INVALID_ARG, "hull %d: mesh not closed", h);
                H.e.push_back(make_int4(a, bb, f, g));
                ne++;
            }
        if (2 * ne != 3 * nt) return fail(MS_ERR_INVALID_ARG, "hull %d: mesh not closed", h);
        if (!(vol > 0.0)) return fail(MS_ERR_INVALID_ARG, "hull %d: no volume (inward triangles?)", h);
        H.vo.push_back((int)H.v.size()); H.to.push_back((int)H.t.size()); H.eo.push_back((int)H.e.size());
        H.rad.push_back((float)rad);
        H.vol.push_back(vol);
        for (int k = 0; k < 3; k++) H.c2.push_back(c2[k]);
    }
    return MS_OK;
}

static ms_status validate_params(const ms_sim_params* p) {
    if (!p) return fail(MS_ERR_INVALID_ARG, "params is NULL");
    if (!(p->dt > 0.f) || !std::isfinite(p->dt)) return fail(MS_ERR_INVALID_ARG, "dt must be > 0");
    if (p->substeps < 1 || p->substeps > 1024) return fail(MS_ERR_INVALID_ARG, "substeps must be in [1, 1024]");
    if (p->pos_iters < 0 || p->vel_iters < 0 || p->pos_iters > 100000 || p->vel_iters > 100000)
        return fail(MS_ERR_INVALID_ARG, "iteration counts must be >= 0");
    if (!finite3(p->gravity, 3)) return fail(MS_ERR_INVALID_ARG, "gravity must be finite");
    if (!(p->margin >= 0.f) || !std::isfinite(p->margin)) return fail(MS_ERR_INVALID_ARG, "margin must be >= 0");
    if (!(p->max_depen_vel > 0.f)) return fail(MS_ERR_INVALID_ARG, "max_depen_vel must be > 0");
    if (p->contact_capacity < 1 || p->contact_capacity > 16384)
        return fail(MS_ERR_INVALID_ARG, "contact_capacity must be in [1, 16384]");
    if (p->pair_capacity < 1 || p->pair_capacity > 65535)
        return fail(MS_ERR_INVALID_ARG, "pair_capacity must be in [1, 65535]");
    if (!(p->linear_damping >= 0.f) || !std::isfinite(p->linear_damping) || !(p->angular_damping >= 0.f) ||
        !std::isfinite(p->angular_damping))
        return fail(MS_ERR_INVALID_ARG, "damping must be finite and >= 0");
    if (!(p->bounce_threshold >= 0.f) || !std::isfinite(p->bounce_threshold))
        return fail(MS_ERR_INVALID_ARG, "bounce_threshold must be finite and >= 0");
    if (p->warm_start != 0 && p->warm_start != 1) return fail(MS_ERR_INVALID_ARG, "warm_start must be 0 or 1");
    if (!soft_params_ok(p)) return fail(MS_ERR_INVALID_ARG, "soft-row frequencies and damping ratios must be finite and >= 0");
    return MS_OK;
}

static ms_status validate_env(int e, const ms_body_desc* bd, int nb, const ms_joint_desc* jd, int nj, int n_hulls) {
    if (nb < 1 || nb > 64) return fail(MS_ERR_INVALID_ARG, "env %d: n_bodies %d not in [1, 64]", e, nb);
    if (nj < 0 || nj > 512) return fail(MS_ERR_INVALID_ARG, "env %d: n_joints %d not in [0, 512]", e, nj);
    if (!bd) return fail(MS_ERR_INVALID_ARG, "env %d: bodies is NULL", e);
    if (nj > 0 && !jd) return fail(MS_ERR_INVALID_ARG, "env %d: joints is NULL", e);
    static const char* body_rule[] = {"", "bad type", "hull index not in the library", "non-finite field",
                                      "zero quaternion", "negative mass", "negative mu", "restitution not in [0, 1]",
                                      "shape size must be > 0"};
    static const char* joint_rule[] = {"", "bad type", "bad parent/child", "non-finite field", "lower > upper",
                                       "negative gain", "zero frame quaternion"};
    for (int i = 0; i < nb; i++) {
        int r = body_desc_check(bd[i], n_hulls, true);
        if (r) return fail(MS_ERR_INVALID_ARG, "env %d body %d: %s", e, i, body_rule[r]);
    }
    for (int j = 0; j < nj; j++) {
        int r = joint_desc_check(jd[j], nb);
        if (r) return fail(MS_ERR_INVALID_ARG, "env %d joint %d: %s", e, j, joint_rule[r]);
    }
    return MS_OK;
}

static void normq(const float* q, float* o) {
    double n = std::sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
    for (int k = 0; k < 4; k++) o[k] = (float)(q[k] / n);
}

static ms_status create_impl(const ms_body_desc* const* bodies_of, const int* nb_of, const ms_joint_desc* const* joints_of,
                             const int* nj_of, int E, const ms_sim_params* p, ms_batch** out,
                             const ms_hull_lib* hull_lib = nullptr) {
    if (!out) return fail(MS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (E < 1) return fail(MS_ERR_INVALID_ARG, "n_envs must be >= 1");
    ms_status st = validate_params(p);
    if (st) return st;
    HostHulls hh;
    if ((st = build_hulls(hull_lib, hh)) != MS_OK) return st;
    for (int e = 0; e < E; e++) {
        st = validate_env(e, bodies_of[e], nb_of[e], joints_of[e], nj_of[e], hh.n);
        if (st) return st;
    }
    ms_batch* b = new ms_batch();
    b->params = *p;
    cudaGetDevice(&b->device);
    {
        {
            std::lock_guard<std::mutex> lk(g_alloc_mu);
            b->alloc_fn = g_alloc_fn;
            b->free_fn = g_free_fn;
            b->alloc_user = g_alloc_user;
        }
        cudaError_t e = cudaStreamCreateWithFlags(&b->setup, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete b; return fail(MS_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)); }
        e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaStreamDestroy(b->setup);
            delete b;
            return fail(MS_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
        }
    }
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    b->smem_optin = (size_t)optin;
    b->E = E;
    b->h_body_off.assign(E + 1, 0);
    b->h_joint_off.assign(E + 1, 0);
    for (int e = 0; e < E; e++) {
        b->h_body_off[e + 1] = b->h_body_off[e] + nb_of[e];
        b->h_joint_off[e + 1] = b->h_joint_off[e] + nj_of[e];
        b->max_nb = std::max(b->max_nb, nb_of[e]);
        b->max_nj = std::max(b->max_nj, nj_of[e]);
    }
    b->NB = b->h_body_off[E];
    b->NJ = b->h_joint_off[E];
    b->A = b->max_nj;
    std::vector<float4> x(b->NB), q(b->NB), v(b->NB), w(b->NB), shape(b->NB), inv(b->NB);
    std::vector<float> rest(b->NB);
    std::vector<int2> meta(b->NB);
    std::vector<unsigned long long> adj(b->NB, 0ull);
    std::vector<int> body_env(b->NB);
    std::vector<float4> jf(4 * (size_t)b->NJ), jp(b->NJ);
    std::vector<int4> jm(b->NJ);
    std::vector<float> jt(b->NJ);
    b->h_type.assign(b->NB, 0);
    b->h_hull_nt.assign(b->NB, 0);
    for (int e = 0; e < E; e++) {
        int b0 = b->h_body_off[e], j0 = b->h_joint_off[e];
        for (int i = 0; i < nb_of[e]; i++) {
            const ms_body_desc& d = bodies_of[e][i];
            int k = b0 + i;
            bool dyn = d.type != MS_PLANE && d.mass > 0.f;
            float qq[4];
            normq(d.quat, qq);
            x[k] = make_float4(d.pos[0], d.pos[1], d.pos[2], 0.f);
            q[k] = make_float4(qq[0], qq[1], qq[2], qq[3]);
            // v.w carries the inverse mass (0 for static bodies)
            v[k] = dyn ? make_float4(d.linvel[0], d.linvel[1], d.linvel[2], (float)(1.0 / (double)d.mass))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
            w[k] = dyn ? make_float4(d.angvel[0], d.angvel[1], d.angvel[2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
            shape[k] = make_float4(d.p[0], d.p[1], d.p[2], d.mu);
            rest[k] = d.restitution;
            if (dyn && d.type == MS_HULL) {
                int h = (int)d.p[0];
                double rho = (double)d.mass / hh.vol[h];
                const double* c2 = &hh.c2[3 * h];
                inv[k] = make_float4(sqrtf((float)(1.0 / (rho * (c2[1] + c2[2])))),
                                     sqrtf((float)(1.0 / (rho * (c2[0] + c2[2])))),
                                     sqrtf((float)(1.0 / (rho * (c2[0] + c2[1])))), (float)(1.0 / (double)d.mass));
            } else if (dyn) {
                float I[3];
                body_inertia(d, I);
                inv[k] = make_float4(sqrtf(1.f / I[0]), sqrtf(1.f / I[1]), sqrtf(1.f / I[2]), (float)(1.0 / (double)d.mass));
            } else {
                inv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            meta[k] = make_int2(d.type | (dyn ? 1 << 8 : 0), (int)((unsigned)d.group | ((unsigned)d.mask << 16)));
            body_env[k] = e;
            b->h_type[k] = (uint8_t)d.type;
            if (d.type == MS_HULL) b->h_hull_nt[k] = hh.to[(int)d.p[0] + 1] - hh.to[(int)d.p[0]];
        }
        for (int j = 0; j < nj_of[e]; j++) {
            const ms_joint_desc& d = joints_of[e][j];
            int k = j0 + j;
            float qa[4], qb[4];
            normq(d.parent_frame + 3, qa);
            normq(d.child_frame + 3, qb);
            jf[4 * k] = make_float4(d.parent_frame[0], d.parent_frame[1], d.parent_frame[2], 0.f);
            jf[4 * k + 1] = make_float4(qa[0], qa[1], qa[2], qa[3]);
            jf[4 * k + 2] = make_float4(d.child_frame[0], d.child_frame[1], d.child_frame[2], 0.f);
            jf[4 * k + 3] = make_float4(qb[0], qb[1], qb[2], qb[3]);
            jp[k] = make_float4(d.lower, d.upper, d.kp, d.kd);
            jm[k] = make_int4(d.type, d.parent, d.child, 0);
            jt[k] = d.target0;
            if (d.parent >= 0) {
                adj[b0 + d.parent] |= 1ull << d.child;
                adj[b0 + d.child] |= 1ull << d.parent;
            }
        }
    }
    DevBatch& D = b->D;
    D.E = E; D.NB = b->NB; D.NJ = b->NJ; D.A = b->A;
    D.P.dt = p->dt; D.P.h = p->dt / (float)p->substeps;
    D.P.substeps = p->substeps; D.P.pos_iters = p->pos_iters; D.P.vel_iters = p->vel_iters;
    D.P.gx = p->gravity[0]; D.P.gy = p->gravity[1]; D.P.gz = p->gravity[2];
    D.P.margin = p->margin; D.P.vmax = p->max_depen_vel;
    D.P.pair_cap = p->pair_capacity; D.P.contact_cap = p->contact_capacity;
    D.P.adl = (float)(1.0 / (1.0 + (double)D.P.h * p->linear_damping));
    D.P.adw = (float)(1.0 / (1.0 + (double)D.P.h * p->angular_damping));
    D.P.bounce = p->bounce_threshold;
    D.P.warm = p->warm_start;
    set_soft_params(D.P, p);
    D.P.restit = 0;
    for (float r : rest) D.P.restit |= r > 0.f;
    ms_status s = MS_OK;
    int* bo = nullptr; int* jo = nullptr;
#define UP(dst, src) do { if ((s = upload(b, dst, src)) != MS_OK) { free_all(b); delete b; return s; } } while (0)
    UP(&bo, b->h_body_off);
    UP(&jo, b->h_joint_off);
    D.body_off = bo; D.joint_off = jo;
    UP(&D.x, x); UP(&D.q, q); UP(&D.v, v); UP(&D.w, w);
    float4* d_shape; float4* d_inv; int2* d_meta; unsigned long long* d_adj;
    UP(&d_shape, shape); UP(&d_inv, inv); UP(&d_meta, meta); UP(&d_adj, adj);
    D.shape = d_shape; D.inv = d_inv; D.meta = d_meta; D.adj = d_adj;
    float4* d_jf; float4* d_jp; int4* d_jm;
    UP(&d_jf, jf); UP(&d_jp, jp); UP(&d_jm, jm); UP(&D.jt, jt);
    D.jf = d_jf; D.jp = d_jp; D.jm = d_jm;
    float* d_rest;
    UP(&d_rest, rest);
    D.rest = d_rest;
    D.hulls = nullptr;
    if (hh.n > 0) {
        // the library on the device, and a HullLib of device pointers to it
        float4 *hv, *hn; int4 *ht, *he; int *hvo, *hto, *heo; float* hrad;
        UP(&hv, hh.v); UP(&hn, hh.n4); UP(&ht, hh.t); UP(&he, hh.e);
        UP(&hvo, hh.vo); UP(&hto, hh.to); UP(&heo, hh.eo); UP(&hrad, hh.rad);
        std::vector<HullLib> lib(1);
        lib[0] = HullLib{hv, ht, hn, he, hvo, hto, heo, hrad};
        HullLib* dl;
        UP(&dl, lib);
        D.hulls = dl;
    }
    D.wc = nullptr; D.wc_n = nullptr; D.wjl = nullptr;
    if (p->warm_start) {
        // warm-start memory: 2 float4 per (env, contact point), a count per
        // env, 8 impulses per joint; empty at creation
        std::vector<float4> wc(2 * (size_t)E * (size_t)p->contact_capacity, make_float4(0.f, 0.f, 0.f, 0.f));
        std::vector<int> wn(E, 0);
        std::vector<float> wj(8 * (size_t)std::max(b->NJ, 1), 0.f);
        UP(&D.wc, wc); UP(&D.wc_n, wn); UP(&D.wjl, wj);
    }
    UP(&b->d_body_env, body_env);
    std::vector<unsigned> zeros(E, 0u);
    UP(&D.status, zeros);
    // longest-first order for the batched work queue: the estimated cost is
    // dominated by rows x sweeps (8 per joint) and the pair tests
    std::vector<int> order(E);
    std::iota(order.begin(), order.end(), 0);
    std::vector<long long> cost(E);
    for (int e = 0; e < E; e++) cost[e] = 8LL * nj_of[e] * 4 + (long long)nb_of[e] * nb_of[e] + 12LL * nb_of[e];
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    UP(&b->d_order, order);
#undef UP
    if ((s = dmalloc(b, (void**)&b->d_queue, 16)) != MS_OK) { free_all(b); delete b; return s; }
    if ((s = dmalloc(b, (void**)&b->d_staging, sizeof(float) * 13 * (size_t)b->NB)) != MS_OK) { free_all(b); delete b; return s; }
    if ((s = dmalloc(b, (void**)&b->d_mask, (size_t)E)) != MS_OK) { free_all(b); delete b; return s; }
    D.plain_ws = nullptr;
    D.rec_man = nullptr; D.rec_pts = nullptr; D.rec_cnt = nullptr; D.rec_col = nullptr; D.rec_col_stride = 0;
    D.force = nullptr;
    cudaError_t ce = cudaStreamSynchronize(b->setup);
    if (ce != cudaSuccess) { free_all(b); delete b; return fail(MS_ERR_CUDA, "%s", cudaGetErrorString(ce)); }
    *out = b;
    g_err.clear();
    return MS_OK;
}

extern "C" ms_status ms_create_batch(const ms_scene_desc* descs, int n_envs, const ms_sim_params* p, ms_batch** out) {
    if (!descs) return fail(MS_ERR_INVALID_ARG, "descs is NULL");
    if (n_envs < 1) return fail(MS_ERR_INVALID_ARG, "n_envs must be >= 1");
    std::vector<const ms_body_desc*> bo(n_envs);
    std::vector<const ms_joint_desc*> jo(n_envs);
    std::vector<int> nb(n_envs), nj(n_envs);
    for (int e = 0; e < n_envs; e++) {
        bo[e] = descs[e].bodies; jo[e] = descs[e].joints;
        nb[e] = descs[e].n_bodies; nj[e] = descs[e].n_joints;
    }
    return create_impl(bo.data(), nb.data(), jo.data(), nj.data(), n_envs, p, out);
}

extern "C" ms_status ms_create_batch_flat(const ms_body_desc* bodies, const int32_t* body_off, const ms_joint_desc* joints,
                                          const int32_t* joint_off, int n_envs, const ms_sim_params* p, ms_batch** out) {
    return ms_create_batch_hulls(bodies, body_off, joints, joint_off, n_envs, p, nullptr, out);
}

extern "C" ms_status ms_create_batch_hulls(const ms_body_desc* bodies, const int32_t* body_off,
                                           const ms_joint_desc* joints, const int32_t* joint_off, int n_envs,
                                           const ms_sim_params* p, const ms_hull_lib* hulls, ms_batch** out) {
    if (!bodies || !body_off || !joint_off) return fail(MS_ERR_INVALID_ARG, "NULL table");
    if (n_envs < 1) return fail(MS_ERR_INVALID_ARG, "n_envs must be >= 1");
    std::vector<const ms_body_desc*> bo(n_envs);
    std::vector<const ms_joint_desc*> jo(n_envs);
    std::vector<int> nb(n_envs), nj(n_envs);
    if (body_off[0] != 0 || joint_off[0] != 0) return fail(MS_ERR_INVALID_ARG, "offsets must start at 0");
    for (int e = 0; e < n_envs; e++) {
        if (body_off[e + 1] < body_off[e] || joint_off[e + 1] < joint_off[e])
            return fail(MS_ERR_INVALID_ARG, "offsets must be non-decreasing (env %d)", e);
        bo[e] = bodies + body_off[e];
        jo[e] = joints ? joints + joint_off[e] : nullptr;
        nb[e] = body_off[e + 1] - body_off[e];
        nj[e] = joint_off[e + 1] - joint_off[e];
    }
    return create_impl(bo.data(), nb.data(), jo.data(), nj.data(), n_envs, p, out, hulls);
}

// --------------------------------------------------------------- plain path
static ms_status ensure_plain(ms_batch* b) {
    if (b->D.plain_ws) return MS_OK;
    const ms_sim_params& p = b->params;
    b->D.plain_layout = make_layout(b->max_nb, b->max_nj, p.pair_capacity, p.contact_capacity, false, true,
                                    p.contact_capacity, true, false);
    void* ws = nullptr;
    const Layout& L = b->D.plain_layout;
    ms_status s = dmalloc(b, &ws, (size_t)b->E * (size_t)(L.s_bytes + L.g_bytes));
    if (s) return s;
    b->D.plain_ws = (char*)ws;
    return MS_OK;
}

static ms_status check_step_args(ms_batch* b, int n_steps) {
    if (!b) return fail(MS_ERR_INVALID_ARG, "batch is NULL");
    if (n_steps < 0 || n_steps > 1000000) return fail(MS_ERR_INVALID_ARG, "n_steps must be in [0, 1e6]");
    return MS_OK;
}

extern "C" ms_status ms_step_plain(ms_batch* b, const float* actions, int n_steps, void* stream) {
    return ms_step_ex(b, actions, n_steps, nullptr, MS_STEP_PLAIN, stream);
}

// ------------------------------------------------------------- batched path
static ms_status configure_fused(ms_batch* b) {
    if (b->fused_ready) return MS_OK;
    // the variant without the code this batch does not use (FV_DYN added below)
    unsigned var = FV_JOINTS | FV_HULLS;
    if (fused_lean(b->D)) {
        var = FV_LEAN;
        if (b->NJ > 0) var |= FV_JOINTS;
        if (b->D.hulls) var |= FV_HULLS;
    }
    const ms_sim_params& p = b->params;
    Tuning& t = b->tune;
    int K = 32 / t.G;                               // envs per warp
    int envs_per_cta = t.warps * K;
    int threads = 32 * t.warps;
    int cc = p.contact_capacity;
    auto lay = [&](bool rows_j, int pts_s, bool lists) {
        return make_layout(b->max_nb, b->max_nj, p.pair_capacity, cc, true, rows_j, pts_s, lists, false);
    };
    // resident CTAs per SM of a layout (0: does not fit)
    auto occ = [&](const Layout& Lc) {
        size_t sm = (size_t)Lc.s_bytes * envs_per_cta;
        if (sm > b->smem_optin) return 0;
        int n = 0;
        if (fused_occupancy(t.G, var, threads, sm, &n) != cudaSuccess) return 0;
        return n;
    };
    // Placement.  rows_smem 1: every row on chip if one CTA fits.  0: slots
    // sized for the capacities -- lists, impulses, joint rows and the rows of
    // as many contact points as keep enough CTAs resident for every env to
    // be in flight at once -- when that holds every contact point; else the
    // dynamic placement: slots hold only the envs' bodies, and each warp's
    // envs share an arena, as large as those resident CTAs allow, that holds
    // what the envs use in each step.  2: the dynamic placement with one CTA
    // per SM (its warps share all of the SM's shared memory).
    bool all_rows = false;
    Layout L;
    int need = (b->E + envs_per_cta - 1) / envs_per_cta;
    int want_sm = (need + b->sm_count - 1) / b->sm_count;    // CTAs per SM for one wave
    bool fixed = false;
    if (t.rows_smem == 1 && occ(L = lay(true, cc, true)) >= 1) {
        all_rows = true;
        fixed = true;
    } else if (t.rows_smem == 2) {
        want_sm = 1;
    } else if (int o0 = occ(L = lay(true, 0, true))) {
        int want = std::min(o0, want_sm);
        int lo = 0, hi = cc;
        while (lo < hi) {
            int mid = (lo + hi + 1) / 2;
            if (occ(lay(true, mid, true)) >= want) lo = mid;
            else hi = mid - 1;
        }
        L = lay(true, lo, true);
        fixed = lo == cc;
    }
    size_t smem = (size_t)L.s_bytes * envs_per_cta;
    if (!fixed) {
        L = lay(false, 0, false);
        size_t base = (size_t)L.s_bytes * envs_per_cta;
        // resident CTAs of the dynamic-placement kernel with an arena of a16 * 16 bytes per warp
        auto occ_a = [&](size_t a16) {
            int n = 0;
            size_t sm = base + a16 * 16 * t.warps;
            if (sm > b->smem_optin) return 0;
            if (fused_occupancy(t.G, var | FV_DYN, threads, sm, &n) != cudaSuccess) return 0;
            return n;
        };
        int o1 = occ_a(0);
        if (o1 < 1)
            return fail(MS_ERR_INVALID_ARG, "tuning needs %zu B of shared memory per CTA (max %zu)", base,
                        b->smem_optin);
        int n_cta = std::max(1, std::min(o1, want_sm));
        // the largest arena per warp (16-byte multiple) that keeps n_cta CTAs resident
        size_t lo = 0, hi = (b->smem_optin - base) / (size_t)t.warps / 16;
        while (lo < hi) {
            size_t mid = (lo + hi + 1) / 2;
            if (occ_a(mid) >= n_cta) lo = mid;
            else hi = mid - 1;
        }
        L.arena_bytes = (int)(lo * 16);
        smem = base + (size_t)L.arena_bytes * t.warps;
    }
    int per_sm = 0;
    bool dyn = L.arena_bytes > 0;
    CK(fused_occupancy(t.G, var | (dyn ? FV_DYN : 0u), threads, smem, &per_sm));
    if (per_sm < 1) return fail(MS_ERR_INVALID_ARG, "tuning does not fit on an SM");
    int grid = per_sm * b->sm_count;
    if (grid > need) grid = need;
    size_t gbytes = (size_t)grid * envs_per_cta * L.g_bytes;
    if (gbytes > b->gscratch_bytes) {
        void* p2 = nullptr;
        ms_status s = dmalloc(b, &p2, gbytes);
        if (s) return s;
        b->d_gscratch = (char*)p2;
        b->gscratch_bytes = gbytes;
    }
    if (t.rows_smem == 1 && !all_rows) t.rows_smem = 0;
    b->fused_layout = L;
    b->fused_var = var | (dyn ? FV_DYN : 0u);
    b->fused_threads = threads;
    b->fused_grid = grid;
    b->fused_smem = smem;
    b->fused_ctas_per_sm = per_sm;
    b->fused_ready = true;
    return MS_OK;
}

static FusedCfg fused_cfg(ms_batch* b) {
    FusedCfg C;
    C.layout = b->fused_layout;
    C.queue = b->d_queue;
    C.order = b->d_order;
    C.gscratch = b->d_gscratch;
    return C;
}

// the batch's device view with this call's record buffer
static DevBatch call_view(const ms_batch* b, float* out) {
    DevBatch D = b->D;
    D.T.out = out;
    return D;
}

static ms_status enqueue_fused(ms_batch* b, const float* actions, int n_steps, float* out, cudaStream_t st) {
    CK(cudaMemsetAsync(b->d_queue, 0, sizeof(int), st));
    CK(launch_fused(call_view(b, out), actions, n_steps, fused_cfg(b), b->tune.G, b->fused_var, b->fused_grid,
                    b->fused_threads, b->fused_smem, st));
    return MS_OK;
}

static ms_status step_enqueue(ms_batch* b, const float* actions, int n_steps, float* out, cudaStream_t st) {
    if (st == nullptr) return enqueue_fused(b, actions, n_steps, out, st);   // the legacy stream cannot be captured
    long long key = (long long)n_steps;
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        ms_status es = enqueue_fused(b, actions, n_steps, out, st);
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (es) return es;
        if (ce != cudaSuccess) return fail(MS_ERR_CUDA, "stream capture: %s", cudaGetErrorString(ce));
        GraphEntry ge;
        CK(cudaGraphInstantiate(&ge.exec, graph, 0));
        size_t n = 0;
        CK(cudaGraphGetNodes(graph, nullptr, &n));
        std::vector<cudaGraphNode_t> nodes(n);
        CK(cudaGraphGetNodes(graph, nodes.data(), &n));
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            CK(cudaGraphNodeGetType(nd, &ty));
            if (ty == cudaGraphNodeTypeKernel) { ge.kernel = nd; CK(cudaGraphKernelNodeGetParams(nd, &ge.kp)); }
        }
        ge.graph = graph;
        it = b->graphs.emplace(key, ge).first;
        CK(cudaGraphLaunch(it->second.exec, st));
        return MS_OK;
    }
    // the actions and record pointers are the arguments that change between calls
    GraphEntry& ge = it->second;
    DevBatch Dv = call_view(b, out);
    const float* act = actions;
    int ns = n_steps;
    FusedCfg C = fused_cfg(b);
    void* args[] = {(void*)&Dv, (void*)&act, (void*)&ns, (void*)&C};
    cudaKernelNodeParams kp = ge.kp;
    kp.kernelParams = args;
    kp.extra = nullptr;
    CK(cudaGraphExecKernelNodeSetParams(ge.exec, ge.kernel, &kp));
    CK(cudaGraphLaunch(ge.exec, st));
    return MS_OK;
}

extern "C" ms_status ms_step_ex(ms_batch* b, const float* actions, int n_steps, float* out, int flags,
                                void* stream) {
    ms_status s = check_step_args(b, n_steps);
    if (s) return s;
    if (flags & ~MS_STEP_PLAIN) return fail(MS_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
    if (out && !b->D.T.on) return fail(MS_ERR_INVALID_ARG, "task records requested but no task is set");
    cudaStream_t st = (cudaStream_t)stream;
    if (flags & MS_STEP_PLAIN) {
        if ((s = ensure_plain(b)) != MS_OK) return s;
        launch_plain(call_view(b, out), actions, n_steps, st);
        CK(cudaGetLastError());
        CK(cudaEventRecord(b->done, st));
        return MS_OK;
    }
    if (n_steps == 0) return MS_OK;
    if ((s = configure_fused(b)) != MS_OK) return s;
    if ((s = step_enqueue(b, actions, n_steps, out, st)) != MS_OK) return s;
    CK(cudaEventRecord(b->done, st));
    return MS_OK;
}

// grows a batch-owned device buffer to at least n floats (the old one stays
// allocated until the batch is destroyed: calls already enqueued may use it)
static ms_status grow_floats(ms_batch* b, float** p, size_t* cap, size_t n) {
    if (n <= *cap) return MS_OK;
    void* q = nullptr;
    ms_status s = dmalloc(b, &q, sizeof(float) * n);
    if (s) return s;
    *p = (float*)q;
    *cap = n;
    return MS_OK;
}

extern "C" ms_status ms_step_host(ms_batch* b, const float* actions, int n_steps, float* out, int out_kind,
                                  void* stream) {
    ms_status s = check_step_args(b, n_steps);
    if (s) return s;
    if (!out) return fail(MS_ERR_INVALID_ARG, "out is NULL");
    if (out_kind != 0 && out_kind != 1) return fail(MS_ERR_INVALID_ARG, "out_kind must be 0 (state) or 1 (records)");
    if (out_kind == 1 && !b->D.T.on) return fail(MS_ERR_INVALID_ARG, "task records requested but no task is set");
    cudaStream_t st = (cudaStream_t)stream;
    const float* dact = nullptr;
    size_t na = actions ? (size_t)n_steps * b->E * b->A : 0;
    if (na > 0) {
        if ((s = grow_floats(b, &b->d_hact, &b->hact_cap, na)) != MS_OK) return s;
        CK(cudaMemcpyAsync(b->d_hact, actions, sizeof(float) * na, cudaMemcpyHostToDevice, st));
        dact = b->d_hact;
    }
    float* drec = nullptr;
    size_t nr = out_kind == 1 ? (size_t)n_steps * b->E * b->D.T.D : 0;
    if (nr > 0) {
        if ((s = grow_floats(b, &b->d_hrec, &b->hrec_cap, nr)) != MS_OK) return s;
        drec = b->d_hrec;
    }
    if ((s = ms_step_ex(b, dact, n_steps, drec, 0, stream)) != MS_OK) return s;
    if (out_kind == 1) {
        if (nr > 0) CK(cudaMemcpyAsync(out, drec, sizeof(float) * nr, cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(b->done, st));
        return MS_OK;
    }
    return ms_copy_state(b, out, 0, stream);
}

ms_status ms::batch_step_eager(ms_batch* b, const float* actions, int n_steps, cudaStream_t st) {
    ms_status s = check_step_args(b, n_steps);
    if (s) return s;
    if (n_steps == 0) return MS_OK;
    if ((s = configure_fused(b)) != MS_OK) return s;
    if ((s = enqueue_fused(b, actions, n_steps, nullptr, st)) != MS_OK) return s;
    CK(cudaEventRecord(b->done, st));
    return MS_OK;
}

extern "C" ms_status ms_step(ms_batch* b, const float* actions, int n_steps, void* stream) {
    return ms_step_ex(b, actions, n_steps, nullptr, 0, stream);
}

// ------------------------------------------------------------------ render
extern "C" ms_status ms_set_camera(ms_batch* b, const ms_camera_desc* c) {
    if (!b || !c || !c->body_rgb) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (!b->render) b->render = render_create();
    CK(cudaEventSynchronize(b->done));
    const char* err = render_configure(b->render, b->D, c, b->h_type, b->h_hull_nt, b->h_body_off, b->max_nb,
                                       (int)b->smem_optin);
    if (err) return fail(MS_ERR_INVALID_ARG, "camera: %s", err);
    CK(cudaGetLastError());
    return MS_OK;
}

extern "C" ms_status ms_render(ms_batch* b, uint8_t* rgba, float* depth, uint16_t* seg, void* stream) {
    if (!b) return fail(MS_ERR_INVALID_ARG, "batch is NULL");
    if (!render_ready(b->render)) return fail(MS_ERR_INVALID_ARG, "no camera is set");
    cudaStream_t st = (cudaStream_t)stream;
    CK(render_launch(b->render, b->D, rgba, depth, seg, st));
    CK(cudaEventRecord(b->done, st));
    return MS_OK;
}

// ---------------------------------------------------------------- pick task
extern "C" ms_status ms_set_task(ms_batch* b, const ms_task_desc* t, void* stream) {
    if (!b) return fail(MS_ERR_INVALID_ARG, "batch is NULL");
    if (!t) {
        b->D.T = DevTask{};
        kernel_choice_changed(b);
        return MS_OK;
    }
    if (t->n_joints != b->A) return fail(MS_ERR_INVALID_ARG, "task n_joints %d != the batch's A %d", t->n_joints, b->A);
    if (b->A > 0 && (!t->delta_lo || !t->delta_hi)) return fail(MS_ERR_INVALID_ARG, "delta_lo / delta_hi NULL");
    if (!(std::isfinite(t->grasp_tol) && t->grasp_tol >= 0.f && std::isfinite(t->touch_tol) && t->touch_tol >= 0.f))
        return fail(MS_ERR_INVALID_ARG, "grasp_tol / touch_tol must be finite and >= 0");
    for (int j = 0; j < b->A; j++)
        if (!(std::isfinite(t->delta_lo[j]) && std::isfinite(t->delta_hi[j])))
            return fail(MS_ERR_INVALID_ARG, "delta bound %d not finite", j);
    for (int e = 0; e < b->E; e++) {
        int nb = b->h_body_off[e + 1] - b->h_body_off[e], nj = b->h_joint_off[e + 1] - b->h_joint_off[e];
        const int bodies[4] = {t->finger_a, t->finger_b, t->cube, t->table};
        for (int k = 0; k < 4; k++)
            if (bodies[k] < 0 || bodies[k] >= nb)
                return fail(MS_ERR_INVALID_ARG, "env %d: task body index %d out of range [0, %d)", e, bodies[k], nb);
        if (t->grip_joint < -1 || t->grip_joint >= nj)
            return fail(MS_ERR_INVALID_ARG, "env %d: grip_joint %d out of range", e, t->grip_joint);
        if (b->h_type[b->h_body_off[e] + t->cube] != MS_BOX) return fail(MS_ERR_INVALID_ARG, "env %d: cube is not a box", e);
        if (b->h_type[b->h_body_off[e] + t->table] != MS_PLANE)
            return fail(MS_ERR_INVALID_ARG, "env %d: table is not a plane", e);
    }
    ms_status s;
    if (!b->d_task_half) {
        if ((s = dmalloc(b, (void**)&b->d_task_half, sizeof(float) * std::max(b->A, 1))) != MS_OK) return s;
        if ((s = dmalloc(b, (void**)&b->d_task_qR, sizeof(float) * std::max(b->NJ, 1))) != MS_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    b->h_task_half.assign(std::max(b->A, 1), 0.f);
    for (int j = 0; j < b->A; j++) b->h_task_half[j] = 0.5f * (t->delta_hi[j] - t->delta_lo[j]);
    CK(cudaMemcpyAsync(b->d_task_half, b->h_task_half.data(), sizeof(float) * b->h_task_half.size(),
                       cudaMemcpyHostToDevice, st));
    DevTask T{};
    T.on = 1;
    T.grip = t->grip_joint; T.fa = t->finger_a; T.fb = t->finger_b; T.cube = t->cube; T.table = t->table;
    T.grasp_tol = t->grasp_tol; T.touch_tol = t->touch_tol;
    T.half = b->d_task_half;
    T.qR = b->d_task_qR;
    T.out = nullptr;
    T.D = 10 + 2 * b->A;
    b->D.T = T;
    kernel_choice_changed(b);
    launch_task_reset(b->D, nullptr, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));           // the host copy of the bounds is reused by the next call
    CK(cudaEventRecord(b->done, st));
    return MS_OK;
}

extern "C" ms_status ms_task_reset(ms_batch* b, const uint8_t* env_mask, void* stream) {
    if (!b) return fail(MS_ERR_INVALID_ARG, "batch is NULL");
    if (!b->D.T.on) return fail(MS_ERR_INVALID_ARG, "no task is set");
    cudaStream_t st = (cudaStream_t)stream;
    const uint8_t* dmask = nullptr;
    if (env_mask) {
        CK(cudaMemcpyAsync(b->d_mask, env_mask, (size_t)b->E, cudaMemcpyHostToDevice, st));
        dmask = b->d_mask;
    }
    launch_task_reset(b->D, dmask, st);
    CK(cudaGetLastError());
    CK(cudaEventRecord(b->done, st));
    return MS_OK;
}

extern "C" int ms_task_record_len(const ms_batch* b) { return b && b->D.T.on ? b->D.T.D : 0; }

extern "C" ms_status ms_task_observe(ms_batch* b, float* out, void* stream) {
    if (!b || !out) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (!b->D.T.on) return fail(MS_ERR_INVALID_ARG, "no task is set");
    cudaStream_t st = (cudaStream_t)stream;
    launch_task_observe(b->D, out, st);
    CK(cudaGetLastError());
    CK(cudaEventRecord(b->done, st));
    return MS_OK;
}

// -------------------------------------------------------------------- state
extern "C" ms_status ms_get_state(ms_batch* b, ms_state_view* out) {
    if (!b || !out) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    out->n_envs = b->E; out->n_bodies = b->NB; out->n_joints = b->NJ; out->max_act = b->A;
    out->x = b->D.x; out->q = b->D.q; out->v = b->D.v; out->w = b->D.w;
    out->body_off = b->D.body_off; out->joint_off = b->D.joint_off;
    out->targets = b->D.jt; out->status = b->D.status;
    return MS_OK;
}

extern "C" ms_status ms_copy_state(ms_batch* b, float* dst, int dst_kind, void* stream) {
    if (!b || !dst) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (dst_kind != 0 && dst_kind != 1) return fail(MS_ERR_INVALID_ARG, "dst_kind must be 0 (host) or 1 (device)");
    cudaStream_t st = (cudaStream_t)stream;
    if (dst_kind == 1) {
        launch_pack_state(b->D, dst, st);
    } else {
        launch_pack_state(b->D, b->d_staging, st);
        CK(cudaMemcpyAsync(dst, b->d_staging, sizeof(float) * 13 * (size_t)b->NB, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(b->done, st));
    return MS_OK;
}

extern "C" ms_status ms_set_state(ms_batch* b, const float* src, int src_kind, const uint8_t* env_mask, void* stream) {
    if (!b || !src) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (src_kind != 0 && src_kind != 1) return fail(MS_ERR_INVALID_ARG, "src_kind must be 0 (host) or 1 (device)");
    cudaStream_t st = (cudaStream_t)stream;
    const float* dsrc = src;
    if (src_kind == 0) {
        CK(cudaMemcpyAsync(b->d_staging, src, sizeof(float) * 13 * (size_t)b->NB, cudaMemcpyHostToDevice, st));
        dsrc = b->d_staging;
    }
    const uint8_t* dmask = nullptr;
    if (env_mask) {
        CK(cudaMemcpyAsync(b->d_mask, env_mask, (size_t)b->E, cudaMemcpyHostToDevice, st));
        dmask = b->d_mask;
    }
    launch_unpack_state(b->D, dsrc, dmask, b->d_body_env, st);
    CK(cudaGetLastError());
    // the host buffers may be reused as soon as this returns
    CK(cudaEventRecord(b->done, st));
    CK(cudaStreamSynchronize(st));
    return MS_OK;
}

extern "C" ms_status ms_sync(ms_batch* b, uint32_t* env_status) {
    if (!b) return fail(MS_ERR_INVALID_ARG, "batch is NULL");
    CK(cudaEventSynchronize(b->done));
    CK(cudaGetLastError());
    std::vector<uint32_t> st(b->E);
    CK(cudaMemcpy(st.data(), b->D.status, sizeof(uint32_t) * b->E, cudaMemcpyDeviceToHost));
    uint32_t any = 0;
    for (uint32_t s : st) any |= s;
    if (env_status) memcpy(env_status, st.data(), sizeof(uint32_t) * b->E);
    if (any & MS_ENV_PAIR_OVERFLOW) return fail(MS_ERR_PAIR_OVERFLOW, "an env exceeded pair_capacity");
    if (any & MS_ENV_CONTACT_OVERFLOW) return fail(MS_ERR_CONTACT_OVERFLOW, "an env exceeded contact_capacity");
    if (any & MS_ENV_COLOR_OVERFLOW) return fail(MS_ERR_COLOR_OVERFLOW, "an env needed more than 64 colours");
    if (any & MS_ENV_NAN) return fail(MS_ERR_NAN, "an env reached a non-finite state and was frozen");
    return MS_OK;
}

extern "C" ms_status ms_destroy(ms_batch* b) {
    if (!b) return MS_OK;
    cudaEventSynchronize(b->done);
    free_all(b);
    delete b;
    return MS_OK;
}

extern "C" const char* ms_last_error(void) { return g_err.c_str(); }

void ms::set_last_error(const char* msg) { g_err = msg; }

const DevBatch& ms::batch_dev(const ::ms_batch* b) { return b->D; }

void ms::batch_dims(const ::ms_batch* b, int* E, int* A, int* max_nb, int* max_nj) {
    *E = b->E; *A = b->A; *max_nb = b->max_nb; *max_nj = b->max_nj;
}

bool ms::batch_has_graph(const ::ms_batch* b, int n_steps) {
    return b->fused_ready && b->graphs.count((long long)n_steps) != 0;
}

// ------------------------------------------------------------ introspection
extern "C" ms_status ms_set_record_contacts(ms_batch* b, int record) {
    if (!b) return fail(MS_ERR_INVALID_ARG, "batch is NULL");
    if (record && !b->rec_keep[0]) {
        void *m = nullptr, *p = nullptr, *c = nullptr, *k = nullptr;
        ms_status s;
        int stride = b->max_nj + b->params.pair_capacity;
        if ((s = dmalloc(b, &m, sizeof(int4) * (size_t)b->E * b->params.pair_capacity)) != MS_OK) return s;
        if ((s = dmalloc(b, &p, sizeof(float) * 10 * (size_t)b->E * b->params.contact_capacity)) != MS_OK) return s;
        if ((s = dmalloc(b, &c, sizeof(int) * (size_t)b->E)) != MS_OK) return s;
        if ((s = dmalloc(b, &k, sizeof(int) * (size_t)b->E * stride)) != MS_OK) return s;
        CK(cudaMemsetAsync(c, 0, sizeof(int) * (size_t)b->E, b->setup));
        CK(cudaStreamSynchronize(b->setup));
        b->rec_keep[0] = m; b->rec_keep[1] = p; b->rec_keep[2] = c; b->rec_keep[3] = k;
        b->rec_stride = stride;
    }
    b->record = record != 0;
    if (b->record) {
        b->D.rec_man = (int4*)b->rec_keep[0]; b->D.rec_pts = (float*)b->rec_keep[1];
        b->D.rec_cnt = (int*)b->rec_keep[2]; b->D.rec_col = (int*)b->rec_keep[3]; b->D.rec_col_stride = b->rec_stride;
    } else {
        b->D.rec_man = nullptr; b->D.rec_pts = nullptr; b->D.rec_cnt = nullptr; b->D.rec_col = nullptr;
    }
    kernel_choice_changed(b);
    return MS_OK;
}

extern "C" ms_status ms_enable_contact_forces(ms_batch* b, int on) {
    if (!b) return fail(MS_ERR_INVALID_ARG, "batch is NULL");
    if (on && !b->d_force) {
        void* f = nullptr;
        ms_status s = dmalloc(b, &f, sizeof(float4) * (size_t)b->NB);
        if (s != MS_OK) return s;
        CK(cudaMemsetAsync(f, 0, sizeof(float4) * (size_t)b->NB, b->setup));
        CK(cudaStreamSynchronize(b->setup));
        b->d_force = (float4*)f;
    }
    b->D.force = on ? b->d_force : nullptr;
    kernel_choice_changed(b);
    return MS_OK;
}

extern "C" ms_status ms_contact_forces(ms_batch* b, float* out, void* stream) {
    if (!b || !out) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (!b->D.force) return fail(MS_ERR_INVALID_ARG, "contact forces are off");
    CK(cudaMemcpyAsync(out, b->D.force, sizeof(float4) * (size_t)b->NB, cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
    return MS_OK;
}

extern "C" ms_status ms_get_contacts(ms_batch* b, int env, int cap, int32_t* pairs, int32_t* npts, float* pts, int* count) {
    if (!b || !count) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (!b->D.rec_man) return fail(MS_ERR_INVALID_ARG, "contact recording is off");
    if (env < 0 || env >= b->E) return fail(MS_ERR_INVALID_ARG, "env %d out of range", env);
    CK(cudaEventSynchronize(b->done));
    int n = 0;
    CK(cudaMemcpy(&n, b->D.rec_cnt + env, sizeof(int), cudaMemcpyDeviceToHost));
    *count = n;
    int m = std::min(n, cap);
    if (m <= 0) return MS_OK;
    std::vector<int4> man(m);
    CK(cudaMemcpy(man.data(), b->D.rec_man + (size_t)env * b->params.pair_capacity, sizeof(int4) * m, cudaMemcpyDeviceToHost));
    std::vector<float> P(10 * (size_t)b->params.contact_capacity);
    CK(cudaMemcpy(P.data(), b->D.rec_pts + (size_t)env * b->params.contact_capacity * 10, sizeof(float) * P.size(),
                  cudaMemcpyDeviceToHost));
    for (int i = 0; i < m; i++) {
        if (pairs) { pairs[2 * i] = man[i].x; pairs[2 * i + 1] = man[i].y; }
        if (npts) npts[i] = man[i].z;
        if (pts) {
            for (int k = 0; k < 4; k++)
                for (int f = 0; f < 10; f++)
                    pts[(size_t)40 * i + 10 * k + f] = k < man[i].z ? P[10 * (size_t)(man[i].w + k) + f] : 0.f;
        }
    }
    return MS_OK;
}

extern "C" ms_status ms_get_colors(ms_batch* b, int env, int cap, int32_t* colors, int* count) {
    if (!b || !count) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (!b->D.rec_col) return fail(MS_ERR_INVALID_ARG, "contact recording is off");
    if (env < 0 || env >= b->E) return fail(MS_ERR_INVALID_ARG, "env %d out of range", env);
    CK(cudaEventSynchronize(b->done));
    int nman = 0;
    CK(cudaMemcpy(&nman, b->D.rec_cnt + env, sizeof(int), cudaMemcpyDeviceToHost));
    int nj = b->h_joint_off[env + 1] - b->h_joint_off[env];
    int n = nj + nman;
    *count = n;
    int m = std::min(n, cap);
    if (m <= 0 || !colors) return MS_OK;
    CK(cudaMemcpy(colors, b->D.rec_col + (size_t)env * b->rec_stride, sizeof(int) * m, cudaMemcpyDeviceToHost));
    return MS_OK;
}

extern "C" ms_status ms_set_tuning(ms_batch* b, const ms_tuning* t) {
    if (!b || !t) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    if (!fused_supported(t->lanes_per_env))
        return fail(MS_ERR_INVALID_ARG, "lanes_per_env must be 1, 2, 4, 8, 16 or 32");
    if (t->warps_per_cta < 1 || t->warps_per_cta > 8) return fail(MS_ERR_INVALID_ARG, "warps_per_cta must be in [1, 8]");
    Tuning old = b->tune;
    b->tune.G = t->lanes_per_env;
    b->tune.warps = t->warps_per_cta;
    if (t->rows_in_smem < 0 || t->rows_in_smem > 2) return fail(MS_ERR_INVALID_ARG, "rows_in_smem must be 0, 1 or 2");
    b->tune.rows_smem = t->rows_in_smem;
    b->fused_ready = false;
    drop_graphs(b);
    ms_status s = configure_fused(b);
    if (s) { b->tune = old; b->fused_ready = false; configure_fused(b); return s; }
    return MS_OK;
}

extern "C" ms_status ms_get_tuning(ms_batch* b, ms_tuning* t) {
    if (!b || !t) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    ms_status s = configure_fused(b);
    if (s) return s;
    t->lanes_per_env = b->tune.G;
    t->warps_per_cta = b->tune.warps;
    t->rows_in_smem = b->tune.rows_smem;
    t->ctas_per_sm = b->fused_ctas_per_sm;
    return MS_OK;
}

static std::string signature(ms_batch* b) {
    std::ostringstream os;
    const ms_sim_params& p = b->params;
    os << "E" << b->E << "_NB" << b->NB << "_NJ" << b->NJ << "_mb" << b->max_nb << "_mj" << b->max_nj << "_pc"
       << p.pair_capacity << "_cc" << p.contact_capacity << "_s" << p.substeps << "_i" << p.pos_iters << "_" << p.vel_iters;
    return os.str();
}

static bool cache_lookup(const char* path, const std::string& key, ms_tuning* t) {
    if (!path) return false;
    std::ifstream f(path);
    if (!f) return false;
    std::stringstream ss;
    ss << f.rdbuf();
    std::string s = ss.str();
    std::string needle = "\"" + key + "\"";
    size_t p = s.find(needle);
    if (p == std::string::npos) return false;
    int G, W, R;
    if (sscanf(s.c_str() + p + needle.size(), " : [%d, %d, %d]", &G, &W, &R) != 3) return false;
    t->lanes_per_env = G; t->warps_per_cta = W; t->rows_in_smem = R;
    return true;
}

static void cache_store(const char* path, const std::string& key, const ms_tuning& t) {
    if (!path) return;
    std::map<std::string, std::string> entries;
    {
        std::ifstream f(path);
        std::string line;
        while (f && std::getline(f, line)) {
            size_t a = line.find('"'), c = line.find('"', a + 1);
            size_t lb = line.find('['), rb = line.find(']');
            if (a == std::string::npos || c == std::string::npos || lb == std::string::npos || rb == std::string::npos) continue;
            entries[line.substr(a + 1, c - a - 1)] = line.substr(lb, rb - lb + 1);
        }
    }
    char buf[64];
    snprintf(buf, sizeof(buf), "[%d, %d, %d]", t.lanes_per_env, t.warps_per_cta, t.rows_in_smem);
    entries[key] = buf;
    std::ofstream o(path);
    o << "{\n";
    size_t i = 0;
    for (auto& kv : entries) {
        o << "  \"" << kv.first << "\": " << kv.second << (++i < entries.size() ? ",\n" : "\n");
    }
    o << "}\n";
}

extern "C" ms_status ms_autotune(ms_batch* b, int n_steps, const char* cache_path, ms_tuning* best, void* stream) {
    if (!b) return fail(MS_ERR_INVALID_ARG, "batch is NULL");
    if (n_steps < 1) return fail(MS_ERR_INVALID_ARG, "n_steps must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    std::string key = signature(b);
    ms_tuning t{};
    if (cache_lookup(cache_path, key, &t) && ms_set_tuning(b, &t) == MS_OK) {
        if (best) ms_get_tuning(b, best);
        return MS_OK;
    }
    // save the state so the trials leave the batch unchanged
    float* save = nullptr;
    float* tsave = nullptr;
    unsigned* ssave = nullptr;
    CK(cudaMalloc(&save, sizeof(float) * 13 * (size_t)b->NB));
    CK(cudaMalloc(&tsave, sizeof(float) * std::max(b->NJ, 1)));
    CK(cudaMalloc(&ssave, sizeof(unsigned) * b->E));
    launch_pack_state(b->D, save, st);
    CK(cudaMemcpyAsync(tsave, b->D.jt, sizeof(float) * b->NJ, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ssave, b->D.status, sizeof(unsigned) * b->E, cudaMemcpyDeviceToDevice, st));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    ms_tuning bt = {b->tune.G, b->tune.warps, b->tune.rows_smem, 0};
    const int Gs[] = {32, 16, 8, 4, 2, 1};
    const int Ws[] = {1, 2, 4, 8};
    for (int G : Gs)
        for (int W : Ws)
            for (int R : {1, 0, 2}) {
                ms_tuning c = {G, W, R, 0};
                if (ms_set_tuning(b, &c) != MS_OK) continue;
                if (R == 1 && b->tune.rows_smem == 0) continue;   // rows did not fit: same as R = 0
                // two calls to warm up (the first captures the graph), then
                // the best of three timings of enough calls for ~5 ms
                ms_step(b, nullptr, n_steps, st);
                cudaEventRecord(e0, st);
                ms_step(b, nullptr, n_steps, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) continue;
                float one = 0.f;
                cudaEventElapsedTime(&one, e0, e1);
                int reps = std::max(2, std::min(50, (int)(5.f / std::max(one, 1e-3f))));
                float ms_ = 1e30f;
                bool ok = true;
                for (int trial = 0; trial < 3 && ok; trial++) {
                    cudaEventRecord(e0, st);
                    for (int r = 0; r < reps; r++) ms_step(b, nullptr, n_steps, st);
                    cudaEventRecord(e1, st);
                    ok = cudaEventSynchronize(e1) == cudaSuccess;
                    float t_ = 0.f;
                    cudaEventElapsedTime(&t_, e0, e1);
                    ms_ = std::min(ms_, t_ / reps);
                }
                if (!ok) continue;
                if (ms_ < best_ms) { best_ms = ms_; bt = c; }
                // restore before the next candidate
                launch_unpack_state(b->D, save, nullptr, b->d_body_env, st);
                cudaMemcpyAsync(b->D.jt, tsave, sizeof(float) * b->NJ, cudaMemcpyDeviceToDevice, st);
            }
    ms_set_tuning(b, &bt);
    launch_unpack_state(b->D, save, nullptr, b->d_body_env, st);
    cudaMemcpyAsync(b->D.jt, tsave, sizeof(float) * b->NJ, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(b->D.status, ssave, sizeof(unsigned) * b->E, cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
    cudaFree(save); cudaFree(tsave); cudaFree(ssave);
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    CK(cudaGetLastError());
    cache_store(cache_path, key, bt);
    if (best) ms_get_tuning(b, best);
    return MS_OK;
}

extern "C" ms_status ms_memory_bytes(ms_batch* b, size_t* bytes) {
    if (!b || !bytes) return fail(MS_ERR_INVALID_ARG, "NULL argument");
    *bytes = b->bytes;
    return MS_OK;
}

extern "C" ms_status ms_estimate_bytes(const int32_t* body_off, const int32_t* joint_off, int n_envs, const ms_sim_params* p,
                                       size_t* bytes) {
    if (!body_off || !joint_off || !p || !bytes || n_envs < 1) return fail(MS_ERR_INVALID_ARG, "bad argument");
    size_t NB = (size_t)body_off[n_envs], NJ = (size_t)joint_off[n_envs];
    int max_nb = 0, max_nj = 0;
    for (int e = 0; e < n_envs; e++) {
        max_nb = std::max(max_nb, body_off[e + 1] - body_off[e]);
        max_nj = std::max(max_nj, joint_off[e + 1] - joint_off[e]);
    }
    // resident state and parameters, the staging buffer and the per-env
    // workspace of the plain path (the batched path's is per resident slot)
    size_t state = NB * (16 * 6 + 8 + 8 + 4 + 52 + 4) + NJ * (64 + 16 + 16 + 4) + (size_t)n_envs * 16 + 64;
    if (p->warm_start) state += (size_t)n_envs * (32 * (size_t)p->contact_capacity + 4) + 32 * NJ;
    Layout L = make_layout(max_nb, max_nj, p->pair_capacity, p->contact_capacity, false, true, p->contact_capacity, true,
                           false);
    *bytes = state + (size_t)n_envs * (size_t)(L.s_bytes + L.g_bytes);
    return MS_OK;
}

extern "C" void ms_abi_sizes(int32_t* out5) {
    if (!out5) return;
    out5[0] = (int32_t)sizeof(ms_body_desc);
    out5[1] = (int32_t)sizeof(ms_joint_desc);
    out5[2] = (int32_t)sizeof(ms_sim_params);
    out5[3] = (int32_t)sizeof(ms_state_view);
    out5[4] = (int32_t)sizeof(ms_tuning);
}
