// ms_step_noalloc: the batched step for callers that must not allocate
// device memory.
//
// Some callers cannot call cudaMalloc: a host process whose device memory is
// owned entirely by another allocator (a framework's caching allocator or a
// fixed arena that hands out every byte), or a control loop that cannot
// afford the implicit device synchronisation and unbounded latency of an
// allocation.  ms_create_batch allocates the resident state and workspaces,
// so such callers use this entry point instead: they own every input and
// output buffer, and the kernel's workspace comes from a fixed array
// compiled into the library.
//
// The workspace is NOALLOC_SCRATCH_BYTES of file-scope device memory, held by
// every GPU that loads the library until the process exits.  Every call
// shares it and it keeps the last call's contents; the work-queue counter at
// its start is cleared by each call, and everything else is written before it
// is read.  Calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on the array and must be serialised by the
// caller.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/ms.h"
#include "ms_internal.h"
#include "ms_stages.cuh"

namespace ms {

static constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;   // 32 MiB
static constexpr size_t NOALLOC_HEADER_BYTES = 256;                  // work-queue counter
static constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

template <typename T>
__device__ __forceinline__ T* nat(char* base, int off) { return reinterpret_cast<T*>(base + off); }

struct NoallocArgs {
    int E, A;
    int max_nb, max_nj;
    DevParams P;
    const int* body_off;
    const int* joint_off;
    const ms_body_desc* bodies;
    const ms_joint_desc* joints;
    float4 *x, *q, *v, *w;
    float* targets;
    unsigned* status;
};

// unit quaternion of a descriptor, normalised in double like ms_create_batch
__device__ __forceinline__ float4 desc_quat(const float* q) {
    double n = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
    return make_float4((float)(q[0] / n), (float)(q[1] / n), (float)(q[2] / n), (float)(q[3] / n));
}

// sqrt(1/I) (body frame) and 1/m of a descriptor: the inertia formula of
// ms_create_batch (primitive_inertia), in double, its float reciprocals
// rounded to nearest as the host rounds them (the kernels are built with
// approximate float division; __frcp_rn is the IEEE-rounded reciprocal), and
// their IEEE square roots, as stored by ms_create_batch
__device__ __forceinline__ float4 desc_inverse_mass(const ms_body_desc& d, bool dyn) {
    if (!dyn) return make_float4(0.f, 0.f, 0.f, 0.f);
    double I[3];
    primitive_inertia(d.type, d.mass, d.p[0], d.p[1], d.p[2], I);
    float I0 = (float)I[0], I1 = (float)I[1], I2 = (float)I[2];
    return make_float4(sqrtf(__frcp_rn(I0)), sqrtf(__frcp_rn(I1)), sqrtf(__frcp_rn(I2)), (float)(1.0 / (double)d.mass));
}

// Same stages and lockstep env loop as the batched kernel; the env's
// parameters are derived from the caller's descriptors while loading it.
template <int G>
__global__ void __launch_bounds__(256) k_noalloc(NoallocArgs D, const float* actions, int n_steps, Layout L,
                                                 int* queue, char* gscratch) {
    extern __shared__ __align__(16) char smem[];
    constexpr int K = 32 / G;
    int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
    int gi = wl / G;
    Grp g;
    g.lane = wl % G; g.size = G; g.base = gi * G;
    int slot_id = warp * K + gi;
    char* s = smem + (size_t)slot_id * L.s_bytes;
    size_t gslot = ((size_t)blockIdx.x * (blockDim.x >> 5) + warp) * K + gi;
    char* gl = gscratch + gslot * (size_t)L.g_bytes;

    EnvView e;
    e.x = nat<float4>(s, L.x); e.q = nat<float4>(s, L.q); e.v = nat<float4>(s, L.v); e.w = nat<float4>(s, L.w);
    // the parameters derived from the descriptors live in the global part
    float4* shp = nat<float4>(gl, L.shape);
    float4* inv = nat<float4>(gl, L.inv);
    int2* meta = nat<int2>(gl, L.meta);
    unsigned long long* adj = nat<unsigned long long>(gl, L.adj);
    float4* jf = nat<float4>(gl, L.jf);
    float4* jp = nat<float4>(gl, L.jp);
    int4* jm = nat<int4>(gl, L.jm);
    e.shape = shp; e.inv = inv; e.meta = meta; e.adj = adj; e.jf = jf; e.jp = jp; e.jm = jm;
    e.jt = nat<float>(gl, L.jt);
    float* rst = nat<float>(gl, L.rest);
    e.rest = rst;
    e.hulls = nullptr;                 // no hull library on this path
    e.force = nullptr;
    e.wc = nullptr; e.wc_n = nullptr; e.wjl = nullptr;       // no warm-start memory on this path
    view_workspace(e, s, gl, L);
    e.status = nat<unsigned>(s, L.status);
    e.rec_man = nullptr; e.rec_pts = nullptr; e.rec_cnt = nullptr; e.rec_col = nullptr;

    for (;;) {
        int t0 = 0;
        if (wl == 0) t0 = atomicAdd(queue, K);
        t0 = __shfl_sync(FULL_MASK, t0, 0);
        if (t0 >= D.E) break;
        int env = t0 + gi;
        bool active = env < D.E;
        int b0 = 0, j0 = 0, nb = 0, nj = 0;
        bool invalid = false;
        if (active) {
            b0 = D.body_off[env]; j0 = D.joint_off[env];
            nb = D.body_off[env + 1] - b0; nj = D.joint_off[env + 1] - j0;
            // the descriptors were never seen by the host: an env whose
            // counts exceed the declared maxima would overrun its slot
            if (nb < 1 || nb > D.max_nb || nj < 0 || nj > D.max_nj) { invalid = true; nb = 0; nj = 0; }
        }
        // every field the step reads, checked by the rules ms_create_batch
        // applies (no hull library here: a hull body is invalid), before
        // anything of the env is loaded; an invalid env is skipped whole
        bool bad = false;
        int nbm = g.wmax(nb), njm = g.wmax(nj);
        for (int i0 = 0; i0 < nbm; i0 += G) {
            int i = i0 + g.lane;
            if (i < nb) bad |= body_desc_check(D.bodies[b0 + i], 0, false) != 0;
        }
        for (int k0 = 0; k0 < njm; k0 += G) {
            int j = k0 + g.lane;
            if (j < nj) bad |= joint_desc_check(D.joints[j0 + j], nb) != 0;
        }
        if (g.any(bad)) { invalid = true; nb = 0; nj = 0; }
        int nbmax = g.wmax(nb), njmax = g.wmax(nj);
        for (int i0 = 0; i0 < nbmax; i0 += G) {
            int i = i0 + g.lane;
            if (i < nb) {
                const ms_body_desc& d = D.bodies[b0 + i];
                bool dyn = d.type != MS_PLANE && d.mass > 0.f;
                float4 iv = desc_inverse_mass(d, dyn);
                float4 vv = D.v[b0 + i];
                e.x[i] = D.x[b0 + i]; e.q[i] = D.q[b0 + i];
                e.v[i] = make_float4(vv.x, vv.y, vv.z, iv.w);
                e.w[i] = D.w[b0 + i];
                shp[i] = make_float4(d.p[0], d.p[1], d.p[2], d.mu);
                rst[i] = d.restitution;
                inv[i] = iv;
                meta[i] = make_int2(d.type | (dyn ? 1 << 8 : 0), (int)((unsigned)d.group | ((unsigned)d.mask << 16)));
                unsigned long long m = 0ull;
                for (int j = 0; j < nj; j++) {
                    int pa = D.joints[j0 + j].parent, ch = D.joints[j0 + j].child;
                    if (pa == i && ch >= 0 && ch < nb) m |= 1ull << ch;
                    if (ch == i && pa >= 0 && pa < nb) m |= 1ull << pa;
                }
                adj[i] = m;
            }
        }
        for (int k0 = 0; k0 < njmax; k0 += G) {
            int j = k0 + g.lane;
            if (j < nj) {
                const ms_joint_desc& d = D.joints[j0 + j];
                jf[4 * j] = make_float4(d.parent_frame[0], d.parent_frame[1], d.parent_frame[2], 0.f);
                jf[4 * j + 1] = desc_quat(d.parent_frame + 3);
                jf[4 * j + 2] = make_float4(d.child_frame[0], d.child_frame[1], d.child_frame[2], 0.f);
                jf[4 * j + 3] = desc_quat(d.child_frame + 3);
                jp[j] = make_float4(d.lower, d.upper, d.kp, d.kd);
                jm[j] = make_int4(d.type, d.parent, d.child, 0);
                e.jt[j] = D.targets[j0 + j];
            }
        }
        // MS_ENV_INVALID is or-ed into the caller's status word and stays
        // set (the env is skipped) until the caller clears it
        bool inv = g.any(invalid);
        if (g.lane == 0) *e.status = active ? (D.status[env] | (inv ? (unsigned)MS_ENV_INVALID : 0u)) : 0u;
        g.sync();
        bool frozen = (*e.status & (ST_NAN | MS_ENV_INVALID)) != 0;
        e.nb = frozen ? 0 : nb;
        e.nj = frozen ? 0 : nj;
        for (int k = 0; k < n_steps; k++) {
            const float* act = (actions && active) ? actions + ((size_t)k * D.E + env) * D.A : nullptr;
            stage_actions(e, g, act, D.A, nullptr);
            stage_broadphase(e, g, D.P);
            stage_narrowphase(e, g, D.P);
            stage_color(e, g);
            MS_CHECK_BOUNDS(e, g, D.P, true);
            for (int sub = 0; sub < D.P.substeps; sub++) run_substep(e, g, D.P, sub == 0, sub == D.P.substeps - 1);
            stage_check(e, g);
            if (*e.status & ST_NAN) { e.nb = 0; e.nj = 0; }
        }
        for (int i0 = 0; i0 < nbmax; i0 += G) {
            int i = i0 + g.lane;
            if (i < nb) { D.x[b0 + i] = e.x[i]; D.q[b0 + i] = e.q[i]; D.v[b0 + i] = e.v[i]; D.w[b0 + i] = e.w[i]; }
        }
        for (int k0 = 0; k0 < njmax; k0 += G) {
            int j = k0 + g.lane;
            if (j < nj) D.targets[j0 + j] = e.jt[j];
        }
        if (g.lane == 0 && active) D.status[env] = *e.status;
        g.sync();
    }
}

static std::mutex g_setup_mu;
static char* g_scratch_ptr[NOALLOC_MAX_DEVICES];
static bool g_setup_done[NOALLOC_MAX_DEVICES];

static ms_status nfail(ms_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);          // reported by ms_last_error()
    return code;
}

// Once per device, with that device current: the device address of the
// scratch array (host code cannot use the symbol itself) and the kernels'
// shared-memory limit.  Neither allocates.
static ms_status setup_device(int dev, char** scratch) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return nfail(MS_ERR_INVALID_ARG, "device %d unsupported", dev);
    if (!g_setup_done[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return nfail(MS_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return nfail(MS_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
        const void* fns[] = {(const void*)k_noalloc<16>, (const void*)k_noalloc<32>};
        for (const void* f : fns) {
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
            if (e != cudaSuccess) return nfail(MS_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        }
        g_scratch_ptr[dev] = (char*)p;
        g_setup_done[dev] = true;
    }
    *scratch = g_scratch_ptr[dev];
    return MS_OK;
}

}  // namespace ms

using namespace ms;

extern "C" ms_status ms_step_noalloc(const ms_noalloc_batch* nb, const ms_sim_params* p, const float* actions,
                                     int n_steps, void* stream) {
    if (!nb || !p) return nfail(MS_ERR_INVALID_ARG, "NULL argument");
    if (nb->n_envs < 1) return nfail(MS_ERR_INVALID_ARG, "n_envs must be >= 1");
    if (nb->max_bodies_per_env < 1 || nb->max_bodies_per_env > 64)
        return nfail(MS_ERR_INVALID_ARG, "max_bodies_per_env must be in [1, 64]");
    if (nb->max_joints_per_env < 0 || nb->max_joints_per_env > 512)
        return nfail(MS_ERR_INVALID_ARG, "max_joints_per_env must be in [0, 512]");
    if (!nb->body_off || !nb->joint_off || !nb->bodies || (nb->max_joints_per_env > 0 && !nb->joints) || !nb->x ||
        !nb->q || !nb->v || !nb->w || (nb->max_joints_per_env > 0 && !nb->targets) || !nb->status)
        return nfail(MS_ERR_INVALID_ARG, "NULL device array");
    if (n_steps < 0 || n_steps > 1000000) return nfail(MS_ERR_INVALID_ARG, "n_steps must be in [0, 1e6]");
    if (!(p->dt > 0.f) || p->substeps < 1 || p->substeps > 1024 || p->pos_iters < 0 || p->vel_iters < 0 ||
        !(p->margin >= 0.f) || !(p->max_depen_vel > 0.f) || p->contact_capacity < 1 || p->contact_capacity > 16384 ||
        p->pair_capacity < 1 || p->pair_capacity > 65535 || !(p->linear_damping >= 0.f) ||
        !(p->angular_damping >= 0.f) || !(p->bounce_threshold >= 0.f))
        return nfail(MS_ERR_INVALID_ARG, "invalid ms_sim_params");
    if (p->warm_start) return nfail(MS_ERR_INVALID_ARG, "warm_start needs the memory of a batch (ms_create_batch)");
    if (!soft_params_ok(p))
        return nfail(MS_ERR_INVALID_ARG, "soft-row frequencies and damping ratios must be finite and >= 0");
    if (n_steps == 0) return MS_OK;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return nfail(MS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
    char* scratch = nullptr;
    ms_status st = setup_device(dev, &scratch);
    if (st) return st;

    // launch shape: one env per warp for large envs, two otherwise
    int G = nb->max_bodies_per_env > 16 ? 32 : 16, K = 32 / G, warps = 1;
    int optin = 0, sms = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int mb = nb->max_bodies_per_env, mj = nb->max_joints_per_env;
    // every row on chip if it fits; else the contact rows, then the joint
    // rows, then the lists and impulses move to the global part
    int pc = p->pair_capacity, cc = p->contact_capacity;
    Layout L = make_layout(mb, mj, pc, cc, true, true, cc, true, true);
    size_t smem = (size_t)L.s_bytes * K * warps;
    if (smem > (size_t)optin) {
        L = make_layout(mb, mj, pc, cc, true, true, 0, true, true);
        smem = (size_t)L.s_bytes * K * warps;
    }
    if (smem > (size_t)optin) {
        L = make_layout(mb, mj, pc, cc, true, false, 0, true, true);
        smem = (size_t)L.s_bytes * K * warps;
    }
    if (smem > (size_t)optin) {
        L = make_layout(mb, mj, pc, cc, true, false, 0, false, true);
        smem = (size_t)L.s_bytes * K * warps;
    }
    if (smem > (size_t)optin)
        return nfail(MS_ERR_INVALID_ARG, "an env needs %zu B of shared memory (max %d)", smem, optin);
    size_t per_cta = (size_t)L.g_bytes * K * warps;
    size_t avail = NOALLOC_SCRATCH_BYTES - NOALLOC_HEADER_BYTES;
    if (per_cta > avail)
        return nfail(MS_ERR_INVALID_ARG, "one CTA needs %zu B of scratch; the fixed scratch holds %zu B", per_cta, avail);
    const void* fn = G == 32 ? (const void*)k_noalloc<32> : (const void*)k_noalloc<16>;
    int per_sm = 0;
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * warps, smem);
    if (ce != cudaSuccess || per_sm < 1) return nfail(MS_ERR_CUDA, "occupancy query failed");
    long long grid = (long long)per_sm * sms;
    long long need = (nb->n_envs + K * warps - 1) / (K * warps);
    long long fit = (long long)(avail / per_cta);
    if (grid > need) grid = need;
    if (grid > fit) grid = fit;

    NoallocArgs D;
    D.E = nb->n_envs;
    D.A = mj;
    D.max_nb = mb; D.max_nj = mj;
    D.P.dt = p->dt; D.P.h = p->dt / (float)p->substeps;
    D.P.substeps = p->substeps; D.P.pos_iters = p->pos_iters; D.P.vel_iters = p->vel_iters;
    D.P.gx = p->gravity[0]; D.P.gy = p->gravity[1]; D.P.gz = p->gravity[2];
    D.P.margin = p->margin; D.P.vmax = p->max_depen_vel;
    D.P.pair_cap = p->pair_capacity; D.P.contact_cap = p->contact_capacity;
    D.P.adl = (float)(1.0 / (1.0 + (double)D.P.h * p->linear_damping));
    D.P.adw = (float)(1.0 / (1.0 + (double)D.P.h * p->angular_damping));
    D.P.bounce = p->bounce_threshold;
    D.P.warm = 0;
    set_soft_params(D.P, p);
    D.P.restit = 1;                          // the descriptors live on the device: always check
    D.body_off = nb->body_off; D.joint_off = nb->joint_off;
    D.bodies = nb->bodies; D.joints = nb->joints;
    D.x = (float4*)nb->x; D.q = (float4*)nb->q; D.v = (float4*)nb->v; D.w = (float4*)nb->w;
    D.targets = nb->targets; D.status = nb->status;
    int* queue = reinterpret_cast<int*>(scratch);
    char* gscratch = scratch + NOALLOC_HEADER_BYTES;
    cudaStream_t s = (cudaStream_t)stream;
    ce = cudaMemsetAsync(queue, 0, sizeof(int), s);                 // the queue starts at zero every call
    if (ce != cudaSuccess) return nfail(MS_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(ce));
    void* args[] = {(void*)&D, (void*)&actions, (void*)&n_steps, (void*)&L, (void*)&queue, (void*)&gscratch};
    ce = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(32 * warps), args, smem, s);
    if (ce != cudaSuccess) return nfail(MS_ERR_CUDA, "launch: %s", cudaGetErrorString(ce));
    return MS_OK;
}
