// Kernels of the batched rigid-body step and their launchers.
//
// Plain path: one 32-thread block per env, one launch per stage and per
// solver sweep; the env's bodies are read from the resident global SoA and
// its workspace lives in a global slot per env.
//
// Batched path: a persistent kernel.  Each warp pops 32 / G env tickets at
// once from a queue ordered longest-first, copies those envs' bodies and
// joints into shared-memory slots, runs all n_steps for all of them in
// lockstep (G lanes per env) and writes the state back once.  No wait in
// either kernel spins on another thread.
#include <nvtx3/nvToolsExt.h>

#include "ms_internal.h"
#include "ms_stages.cuh"

namespace ms {

// ------------------------------------------------------------ slot layout
static int align_up(int x, int a) { return (x + a - 1) / a * a; }

Layout make_layout(int max_nb, int max_nj, int pair_cap, int contact_cap, bool with_state, bool rows_j_shared,
                   int pts_s, bool lists_shared, bool with_params) {
    Layout L;
    int nb = max_nb > 0 ? max_nb : 1, nj = max_nj > 0 ? max_nj : 1;
    int pc = pair_cap > 0 ? pair_cap : 1, cc = contact_cap > 0 ? contact_cap : 1;
    if (pts_s < 0) pts_s = 0;
    if (pts_s > cc) pts_s = cc;
    int ncons = max_nj + (pc < cc ? pc : cc);      // every manifold has at least one point
    int nrows = 8 * nj + 3 * cc;
    L.njs = nj;
    const int RB = (int)sizeof(Row);
    int o = 0;
    auto take = [&](int bytes, int al) { o = align_up(o, al); int r = o; o += bytes; return r; };
    // shared part
    if (with_state) {
        L.x = take(16 * nb, 16); L.q = take(16 * nb, 16); L.v = take(16 * nb, 16); L.w = take(16 * nb, 16);
    } else {
        L.x = L.q = L.v = L.w = -1;
    }
    L.sq = take(48 * nb, 16);
    L.color_off = take(4 * (MAX_COLORS + 1), 4);
    L.cnt = take(4 * C_NUM, 16);
    L.status = take(4, 4);
    L.lists_shared = lists_shared;
    if (lists_shared) {
        L.scons = take(16 * ncons, 16);
        L.lam = take(4 * nrows, 16);
    }
    L.rows_j_shared = rows_j_shared;
    if (rows_j_shared) L.rows_j = take(RB * 8 * nj, 16);
    L.pts_s = pts_s;
    L.rows_cs = pts_s > 0 ? take(RB * 3 * pts_s, 16) : -1;
    // slots of the envs of a warp start 16 B apart modulo 128 B, so equal
    // offsets in different slots fall in different shared-memory banks
    L.s_bytes = align_up(o, 128) + 16;
    // global part
    o = 0;
    if (!lists_shared) {
        L.scons = take(16 * ncons, 16);
        L.lam = take(4 * nrows, 16);
    }
    if (!rows_j_shared) L.rows_j = take(RB * 8 * nj, 16);
    L.rows_cg = pts_s < cc ? take(RB * 3 * cc, 16) : -1;
    L.aabb = take(32 * nb, 16);
    L.pairs = take(4 * pc, 4);
    L.man = take(16 * pc, 16);
    L.pts = take(48 * cc, 16);
    int scratch = 16 * ncons + 4 * ncons + 8 * nb;
    int rows_s_bytes = rows_j_shared ? RB * 8 * nj + (pts_s > 0 ? RB * 3 * pts_s : 0) : 0;
    L.color_shared = rows_j_shared && scratch <= rows_s_bytes;
    if (L.color_shared) {
        L.cons = L.rows_j;
        L.colr = L.cons + 16 * ncons;
        L.used = align_up(L.colr + 4 * ncons, 8);
    } else {
        L.cons = take(16 * ncons, 16);
        L.colr = take(4 * ncons, 4);
        L.used = take(8 * nb, 8);
    }
    if (with_params) {
        L.shape = take(16 * nb, 16); L.inv = take(16 * nb, 16); L.meta = take(8 * nb, 8);
        L.adj = take(8 * nb, 8);
        L.jf = take(64 * nj, 16); L.jp = take(16 * nj, 16); L.jm = take(16 * nj, 16); L.jt = take(4 * nj, 4);
        L.rest = take(4 * nb, 4);
    } else {
        L.shape = L.inv = L.meta = L.adj = L.jf = L.jp = L.jm = L.jt = L.rest = -1;
    }
    L.g_bytes = align_up(o, 16);
    L.arena_bytes = 0;
    return L;
}

// ------------------------------------------------------------- plain path
__device__ __forceinline__ EnvView plain_view(const DevBatch& D, int env) {
    EnvView e;
    int b0 = D.body_off[env], j0 = D.joint_off[env];
    e.nb = D.body_off[env + 1] - b0;
    e.nj = D.joint_off[env + 1] - j0;
    e.x = D.x + b0; e.q = D.q + b0; e.v = D.v + b0; e.w = D.w + b0;
    view_params(e, D, b0, j0, env, true);
    const Layout& L = D.plain_layout;
    char* s = D.plain_ws + (size_t)env * (L.s_bytes + L.g_bytes);
    view_workspace(e, s, s + L.s_bytes, L);
    e.status = D.status + env;
    view_record(e, D, env, true);
    if (*e.status & ST_NAN) { e.nb = 0; e.nj = 0; }   // frozen
    return e;
}

__device__ __forceinline__ Grp warp_grp() {
    Grp g;
    g.lane = threadIdx.x & 31; g.size = 32; g.base = 0;
    return g;
}

__global__ void k_begin_step(DevBatch D, const float* actions, int step) {
    int env = blockIdx.x;
    EnvView e = plain_view(D, env);
    Grp g = warp_grp();
    stage_actions(e, g, actions ? actions + ((size_t)step * D.E + env) * D.A : nullptr, D.A, D.T.on ? D.T.half : nullptr);
    stage_broadphase(e, g, D.P);
}
__global__ void k_narrow(DevBatch D) {
    EnvView e = plain_view(D, blockIdx.x);
    stage_narrowphase(e, warp_grp(), D.P);
}
__global__ void k_color(DevBatch D) {
    EnvView e = plain_view(D, blockIdx.x);
    begin_step_solve(e, warp_grp(), D.P);
}
__global__ void k_prep(DevBatch D) {
    EnvView e = plain_view(D, blockIdx.x);
    stage_prep(e, warp_grp(), D.P);
}
__global__ void k_sweep(DevBatch D, int mode) {
    EnvView e = plain_view(D, blockIdx.x);
    stage_sweep(e, warp_grp(), mode, D.P);
}
__global__ void k_integrate(DevBatch D) {
    EnvView e = plain_view(D, blockIdx.x);
    stage_integrate(e, warp_grp(), D.P);
}
// the end of a substep: the contact impulse record, restitution after the
// last substep, angular velocities back to world space
__global__ void k_end_substep(DevBatch D, int last) {
    EnvView e = plain_view(D, blockIdx.x);
    Grp g = warp_grp();
    if (D.P.restit) {
        stage_track_impulse(e, g);
        if (last) stage_restitution(e, g, D.P);
    }
    stage_unscale(e, g);
}
__global__ void k_check(DevBatch D, int step) {
    int env = blockIdx.x;
    EnvView e = plain_view(D, env);
    Grp g = warp_grp();
    end_step_solve(e, g, D.P);
    if (D.force) stage_contact_forces(e, g, D.P);
    stage_check(e, g);
    if (D.T.out)
        stage_task_record(e, g, D.T, D.A, D.T.out + ((size_t)step * D.E + env) * D.T.D, (*e.status & ST_NAN) != 0);
}

// NVTX ranges name the launches of each stage (host-side enqueue ranges; a
// profiler can select kernels by them, e.g. ncu --nvtx --nvtx-include).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

int launch_plain(const DevBatch& D, const float* actions, int n_steps, cudaStream_t s) {
    int launches = 0;
    dim3 grid(D.E), block(32);
    NvtxRange all("ms_step_plain");
    for (int k = 0; k < n_steps; k++) {
        {
            NvtxRange r("broadphase+narrowphase+colour");
            k_begin_step<<<grid, block, 0, s>>>(D, actions, k);
            k_narrow<<<grid, block, 0, s>>>(D);
            k_color<<<grid, block, 0, s>>>(D);
            launches += 3;
        }
        for (int sub = 0; sub < D.P.substeps; sub++) {
            {
                NvtxRange r("prep+warm");
                k_prep<<<grid, block, 0, s>>>(D);
                launches++;
                if (sub > 0 || D.P.warm) {      // the first substep's warm start has nothing to apply without warm_start
                    k_sweep<<<grid, block, 0, s>>>(D, 0);
                    launches++;
                }
            }
            {
                NvtxRange r("position sweeps");
                for (int it = 0; it < D.P.pos_iters; it++) { k_sweep<<<grid, block, 0, s>>>(D, 1); launches++; }
            }
            {
                NvtxRange r("integrate+relax sweeps");
                k_integrate<<<grid, block, 0, s>>>(D);
                launches++;
                for (int it = 0; it < D.P.vel_iters; it++) { k_sweep<<<grid, block, 0, s>>>(D, 2); launches++; }
                k_end_substep<<<grid, block, 0, s>>>(D, sub == D.P.substeps - 1);
                launches++;
            }
        }
        NvtxRange r("check");
        k_check<<<grid, block, 0, s>>>(D, k);
        launches++;
    }
    return launches;
}

// ----------------------------------------------------------- batched path
// k_fused<G> lives in ms_fused.cu, one translation unit per G.
static const void* fused_fn(int G, unsigned v) {
    switch (G) {
    case 1: return fused_kernel_1(v);
    case 2: return fused_kernel_2(v);
    case 4: return fused_kernel_4(v);
    case 8: return fused_kernel_8(v);
    case 16: return fused_kernel_16(v);
    case 32: return fused_kernel_32(v);
    default: return nullptr;
    }
}

bool fused_supported(int G) { return fused_fn(G, FV_JOINTS | FV_HULLS) != nullptr; }

// Loads every variant of the batched kernel now (a kernel's first use
// otherwise loads it then, which a long-running caller such as the step
// server would see as one slow launch).
void fused_preload() {
    cudaFuncAttributes a;
    for (int G : {1, 2, 4, 8, 16, 32})
        for (unsigned v = 0; v < 16u; v++)
            if (const void* fn = fused_fn(G, v)) cudaFuncGetAttributes(&a, fn);
    cudaGetLastError();
}

bool fused_lean(const DevBatch& D) {
    return !D.T.on && !D.force && !D.P.restit && !D.P.warm && !D.rec_man;
}

cudaError_t fused_occupancy(int G, unsigned variant, int threads, size_t smem, int* blocks_per_sm) {
    const void* fn = fused_fn(G, variant);
    if (!fn) return cudaErrorInvalidValue;
    // The limit is a property of the kernel function shared by every batch
    // (and every captured graph), so it is raised once to the device maximum
    // rather than set to one batch's size; each launch still asks only for
    // what its layout uses.
    int dev = 0, optin = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err == cudaSuccess) err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, smem);
}

cudaError_t launch_fused(const DevBatch& D, const float* actions, int n_steps, const FusedCfg& C, int G, unsigned variant,
                         int grid, int threads, size_t smem, cudaStream_t s) {
    const void* fn = fused_fn(G, variant);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {(void*)&D, (void*)&actions, (void*)&n_steps, (void*)&C};
    NvtxRange r("ms_step (fused)");
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
}

// -------------------------------------------------------- state transfer
__global__ void k_pack_state(DevBatch D, float* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.NB) return;
    float4 x = D.x[i], q = D.q[i], v = D.v[i], w = D.w[i];
    float* o = out + 13 * (size_t)i;
    o[0] = x.x; o[1] = x.y; o[2] = x.z;
    o[3] = q.x; o[4] = q.y; o[5] = q.z; o[6] = q.w;
    o[7] = v.x; o[8] = v.y; o[9] = v.z;
    o[10] = w.x; o[11] = w.y; o[12] = w.z;
}

// restores dynamic bodies verbatim (a checkpoint round-trips bit for bit);
// static bodies keep their pose
__global__ void k_unpack_state(DevBatch D, const float* in, const uint8_t* env_mask, const int* body_env) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.NB) return;
    int env = body_env[i];
    if (env_mask && !env_mask[env]) return;
    if (!((D.meta[i].x >> 8) & 1)) return;
    const float* s = in + 13 * (size_t)i;
    D.x[i] = make_float4(s[0], s[1], s[2], 0.f);
    D.q[i] = make_float4(s[3], s[4], s[5], s[6]);
    D.v[i] = make_float4(s[7], s[8], s[9], D.v[i].w);     // .w keeps the inverse mass
    D.w[i] = make_float4(s[10], s[11], s[12], 0.f);
}

// a set state starts with a clear status and no warm-start memory
__global__ void k_clear_status(DevBatch D, const uint8_t* env_mask) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= D.E) return;
    if (env_mask && !env_mask[e]) return;
    D.status[e] = 0u;
    if (D.wc_n) {
        D.wc_n[e] = 0;
        for (int k = 8 * D.joint_off[e]; k < 8 * D.joint_off[e + 1]; k++) D.wjl[k] = 0.f;
    }
}

void launch_pack_state(const DevBatch& D, float* out, cudaStream_t s) {
    int t = 256, b = (D.NB + t - 1) / t;
    if (b > 0) k_pack_state<<<b, t, 0, s>>>(D, out);
}

void launch_unpack_state(const DevBatch& D, const float* in, const uint8_t* mask, const int* body_env,
                         cudaStream_t s) {
    int t = 256, b = (D.NB + t - 1) / t;
    if (b > 0) k_unpack_state<<<b, t, 0, s>>>(D, in, mask, body_env);
    int be = (D.E + t - 1) / t;
    if (be > 0) k_clear_status<<<be, t, 0, s>>>(D, mask);
}

// ---------------------------------------------------------------- pick task
// an env's resident state and parameters (no workspace), one warp per env
__device__ __forceinline__ EnvView kin_view(const DevBatch& D, int env) {
    EnvView e;
    int b0 = D.body_off[env], j0 = D.joint_off[env];
    e.nb = D.body_off[env + 1] - b0;
    e.nj = D.joint_off[env + 1] - j0;
    e.x = D.x + b0; e.q = D.q + b0; e.v = D.v + b0; e.w = D.w + b0;
    view_params(e, D, b0, j0, env, true);
    e.status = D.status + env;
    return e;
}

// controller reset after an env reset: target = q = q_reset
__global__ void k_task_reset(DevBatch D, const uint8_t* env_mask) {
    int env = blockIdx.x;
    if (env_mask && !env_mask[env]) return;              // the whole warp
    EnvView e = kin_view(D, env);
    for (int j = threadIdx.x; j < e.nj; j += 32) {
        float q = joint_coord(e, j);
        e.jt[j] = q;
        e.qR[j] = q;
    }
}

__global__ void k_task_observe(DevBatch D, float* out) {
    int env = blockIdx.x;
    EnvView e = kin_view(D, env);
    stage_task_record(e, warp_grp(), D.T, D.A, out + (size_t)env * D.T.D, (*e.status & ST_NAN) != 0);
}

void launch_task_reset(const DevBatch& D, const uint8_t* mask, cudaStream_t s) {
    if (D.E > 0) k_task_reset<<<D.E, 32, 0, s>>>(D, mask);
}

void launch_task_observe(const DevBatch& D, float* out, cudaStream_t s) {
    if (D.E > 0) k_task_observe<<<D.E, 32, 0, s>>>(D, out);
}

}  // namespace ms
