// The batched path's persistent kernel, k_fused<G, LEAN, DYN, JOINTS, HULLS>,
// for one lane-group size G (lanes per env) per translation unit: the build
// compiles this file once per G with -DMS_FUSED_G=G, so the instantiations
// compile in parallel.  Code a batch does not use is compiled out of its
// kernel (a smaller kernel: fewer registers and instruction-cache misses),
// results identical: LEAN = true has no pick-task, contact-force,
// restitution, warm-start or contact-record code; JOINTS = false no joint
// rows; HULLS = false no hull routines (both only in lean kernels).
//
// Each warp pops 32 / G env tickets at once from a queue ordered
// longest-first, copies those envs' bodies into shared-memory slots, runs
// all n_steps for all of them in lockstep (G lanes per env) and writes the
// state back once.  No wait spins on another thread.  DYN = true is the
// kernel of the dynamic placement (arena_bytes > 0): the warp's envs share
// an arena for their lists, impulses and rows, placed anew after each
// step's narrowphase; that code is compiled out of the DYN = false kernel,
// which runs the capacity-sized slots.
#include "ms_internal.h"
#include "ms_stages.cuh"

#ifndef MS_FUSED_G
#error "compile with -DMS_FUSED_G=<lanes per env: 1, 2, 4, 8, 16 or 32>"
#endif

namespace ms {

template <int G, bool LEAN, bool DYN, bool JOINTS, bool HULLS>
__global__ void __launch_bounds__(256, 1) k_fused(DevBatch D, const float* actions, int n_steps, FusedCfg C) {
    extern __shared__ __align__(16) char smem[];
    const Layout& L = C.layout;
    constexpr int K = 32 / G;                  // envs per warp
    int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
    int gi = wl / G;
    Grp g;
    g.lane = wl % G; g.size = G; g.base = gi * G;
    int slot_id = warp * K + gi;
    char* s = smem + (size_t)slot_id * L.s_bytes;
    size_t gslot = ((size_t)blockIdx.x * (blockDim.x >> 5) + warp) * K + gi;
    char* gl = C.gscratch + gslot * (size_t)L.g_bytes;

    // dynamic placement: the warp's share of the arena after the CTA's slots
    char* arena = DYN
                      ? smem + (size_t)(blockDim.x >> 5) * K * L.s_bytes + (size_t)warp * L.arena_bytes
                      : nullptr;

    EnvView e;
    e.x = at<float4>(s, L.x); e.q = at<float4>(s, L.q); e.v = at<float4>(s, L.v); e.w = at<float4>(s, L.w);
    view_workspace(e, s, gl, L);
    e.status = at<unsigned>(s, L.status);

    for (;;) {
        int t0 = 0;
        if (wl == 0) t0 = atomicAdd(C.queue, K);
        t0 = __shfl_sync(FULL_MASK, t0, 0);
        if (t0 >= D.E) break;                            // warp-uniform
        int t = t0 + gi;
        bool active = t < D.E;
        int env = active ? C.order[t] : 0;
        int b0 = 0, j0 = 0, nb = 0, nj = 0;
        if (active) {
            b0 = D.body_off[env]; j0 = D.joint_off[env];
            nb = D.body_off[env + 1] - b0; nj = D.joint_off[env + 1] - j0;
        }
        view_params(e, D, b0, j0, env, active && !LEAN);
        if constexpr (!HULLS) e.hulls = nullptr;
        int nbmax = g.wmax(nb);
        for (int i0 = 0; i0 < nbmax; i0 += G) {
            int i = i0 + g.lane;
            if (i < nb) { e.x[i] = D.x[b0 + i]; e.q[i] = D.q[b0 + i]; e.v[i] = D.v[b0 + i]; e.w[i] = D.w[b0 + i]; }
        }
        if (g.lane == 0) *e.status = active ? D.status[env] : 0u;
        view_record(e, D, env, active && !LEAN);
        g.sync();
        bool frozen = (*e.status & ST_NAN) != 0;
        e.nb = frozen ? 0 : nb;
        e.nj = frozen ? 0 : nj;
        for (int k = 0; k < n_steps; k++) {
            const float* act = (actions && active) ? actions + ((size_t)k * D.E + env) * D.A : nullptr;
            stage_actions(e, g, act, D.A, (!LEAN && D.T.on) ? D.T.half : nullptr);
            stage_broadphase(e, g, D.P);
            stage_narrowphase<HULLS>(e, g, D.P);
            if constexpr (DYN) place_dynamic(e, g, arena, L.arena_bytes, gl, L);
            if constexpr (LEAN) {
                stage_color(e, g);
                MS_CHECK_BOUNDS(e, g, D.P, true);
            } else {
                begin_step_solve(e, g, D.P);
            }
            for (int sub = 0; sub < D.P.substeps; sub++) run_substep<!LEAN, JOINTS>(e, g, D.P, sub == 0, sub == D.P.substeps - 1);
            if constexpr (!LEAN) {
                end_step_solve(e, g, D.P);
                if (D.force) stage_contact_forces(e, g, D.P);
            }
            stage_check(e, g);
            if constexpr (!LEAN) {
                if (D.T.out)
                    stage_task_record(e, g, D.T, D.A, active ? D.T.out + ((size_t)k * D.E + env) * D.T.D : nullptr,
                                      (*e.status & ST_NAN) != 0);
            }
            if (*e.status & ST_NAN) { e.nb = 0; e.nj = 0; }
        }
        for (int i0 = 0; i0 < nbmax; i0 += G) {
            int i = i0 + g.lane;
            if (i < nb) { D.x[b0 + i] = e.x[i]; D.q[b0 + i] = e.q[i]; D.v[b0 + i] = e.v[i]; D.w[b0 + i] = e.w[i]; }
        }
        if (g.lane == 0 && active) D.status[env] = *e.status;
        g.sync();
    }
}

#define MS_CAT_(a, b) a##b
#define MS_CAT(a, b) MS_CAT_(a, b)
template <bool L, bool D, bool J, bool H>
static const void* kf() { return (const void*)k_fused<MS_FUSED_G, L, D, J, H>; }

// the kernel of a variant (FV_* bits); a variant without FV_LEAN has joints and hulls
const void* MS_CAT(fused_kernel_, MS_FUSED_G)(unsigned v) {
    bool dyn = v & FV_DYN, joints = v & FV_JOINTS, hulls = v & FV_HULLS;
    if (!(v & FV_LEAN)) return dyn ? kf<false, true, true, true>() : kf<false, false, true, true>();
    if (joints && hulls) return dyn ? kf<true, true, true, true>() : kf<true, false, true, true>();
    if (joints) return dyn ? kf<true, true, true, false>() : kf<true, false, true, false>();
    if (hulls) return dyn ? kf<true, true, false, true>() : kf<true, false, false, true>();
    return dyn ? kf<true, true, false, false>() : kf<true, false, false, false>();
}

}  // namespace ms
