// Internal declarations shared by the host API and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/ms.h"
#include "ms_math.cuh"

struct ms_batch;   // include/ms.h

namespace ms {

// Byte offsets of one env's arrays inside its workspace (-1: absent).  The
// workspace has a shared part -- the data every solver sweep touches: body
// velocities and poses, the square root of each body's world inverse
// inertia, the colour-ordered constraint list, impulses, joint rows and the
// rows of the first pts_s contact points -- in shared memory on the batched
// path, and a global part: AABBs, pairs, manifolds, contact anchors, the
// colouring scratch and the rows of the remaining contact points, written
// once per step or substep and read through L1/L2.  The plain path keeps
// both parts in one global slot per env.
struct Layout {
    int s_bytes;
    int x, q, v, w;                          // body state copies (batched path only)
    int sq;                                  // S = (world inverse inertia)^(1/2), 2 float4, and the step-start q, per body
    int scons, color_off, lam, cnt, status;  // shared part unless lists_shared is false
    bool lists_shared;                       // scons and lam in the shared part
    bool rows_j_shared;                      // joint rows in the shared part
    int rows_j;                              // 8 rows per joint, interleaved: row r of joint j at r * njs + j
    int njs;                                 // joint row stride (max joints per env, >= 1)
    int pts_s;                               // contact points whose rows are in the shared part
    int rows_cs;                             // their rows (3 per point), or -1
    // colouring scratch (records, colours, colour masks per body): laid over
    // the joint and contact rows of the shared part when they are there and
    // large enough (the rows are written after colouring), else global
    bool color_shared;
    int cons, colr, used;
    int g_bytes;
    int aabb, pairs, man, pts;
    int rows_cg;                             // rows of every contact point (those >= pts_s are used), or -1
    int shape, inv, meta, adj, jf, jp, jm, jt, rest;   // parameter copies (no-allocation path only), or -1
    // batched path, dynamic placement: bytes of shared memory per warp, after
    // the CTA's slots, that the warp's envs share each step for their lists,
    // impulses and rows (0: the placement above, fixed by the capacities)
    int arena_bytes;
};

// with_state: x, q, v, w copied into the shared part; with_params: body and
// joint parameters copied into the global part.  pts_s is clamped to
// [0, contact_cap].
Layout make_layout(int max_nb, int max_nj, int pair_cap, int contact_cap, bool with_state, bool rows_j_shared,
                   int pts_s, bool lists_shared, bool with_params);

// Kernel-side view of a batch (plain pointers, passed by value).
struct DevParams {
    float dt, h;
    int substeps, pos_iters, vel_iters;
    float gx, gy, gz;
    float margin, vmax;
    int pair_cap, contact_cap;
    float adl, adw;            // velocity damping factors per substep, 1 / (1 + h c)
    float bounce;              // restitution threshold (approach speed, m/s)
    int warm;                  // impulses carried across steps
    int restit;                // some body of the batch has restitution > 0
    // soft rows in the position sweeps (rate = bias per unit error, ms =
    // mass scale, is = impulse scale, ims = 1 / ms; is = 0: rigid)
    float c_rate, c_ms, c_is, c_ims;     // contact normals of penetrating points
    float j_rate, j_ms, j_is, j_ims;     // joint equality rows
};

// Principal inertia (body frame) of a uniform solid primitive of mass m:
// sphere radius p0; box half-extents p0, p1, p2; capsule radius p0 and
// half-length p1 along z -- a cylinder of length 2 p1 and two hemispherical
// caps whose centroids sit 3 p0 / 8 past the segment ends (parallel-axis
// theorem).  The one formula of ms_create_batch and ms_step_noalloc.
__host__ __device__ inline void primitive_inertia(int type, double m, double p0, double p1, double p2, double I[3]) {
    if (type == MS_SPHERE) {
        I[0] = I[1] = I[2] = 0.4 * m * p0 * p0;
    } else if (type == MS_BOX) {
        I[0] = m * (p1 * p1 + p2 * p2) / 3.0;
        I[1] = m * (p0 * p0 + p2 * p2) / 3.0;
        I[2] = m * (p0 * p0 + p1 * p1) / 3.0;
    } else {
        const double pi = 3.14159265358979323846;
        double r = p0, l = p1;
        double vcyl = 2.0 * pi * r * r * l, vsph = 4.0 * pi * r * r * r / 3.0;
        double mcyl = m * vcyl / (vcyl + vsph), msph = m - mcyl;
        // about the capsule centre each cap contributes m_cap (2r^2/5 + l^2 + 3lr/4)
        I[0] = I[1] = mcyl * (3.0 * r * r + 4.0 * l * l) / 12.0 + msph * (0.4 * r * r + l * l + 0.75 * l * r);
        I[2] = 0.5 * mcyl * r * r + 0.4 * msph * r * r;
    }
}

__host__ __device__ inline bool finite_f(float x) { return x == x && x - x == 0.f; }

// Per-field checks of a body descriptor, the rules ms_create_batch and
// ms_step_noalloc share (0: valid; otherwise which rule failed, BD_*).
// state: also the pose and velocity fields (read by ms_create_batch only);
// n_hulls: hulls in the batch's library (0: a hull body is invalid).
enum { BD_TYPE = 1, BD_HULL, BD_NONFINITE, BD_QUAT, BD_MASS, BD_MU, BD_RESTITUTION, BD_SIZE };
__host__ __device__ inline int body_desc_check(const ms_body_desc& d, int n_hulls, bool state) {
    if (d.type < MS_SPHERE || d.type > MS_HULL) return BD_TYPE;
    if (d.type == MS_HULL && !(d.p[0] >= 0.f && d.p[0] < (float)n_hulls && d.p[0] == (float)(int)d.p[0]))
        return BD_HULL;
    if (!finite_f(d.mass) || !finite_f(d.mu)) return BD_NONFINITE;
    if (state) {
        for (int k = 0; k < 3; k++)
            if (!finite_f(d.pos[k]) || !finite_f(d.linvel[k]) || !finite_f(d.angvel[k])) return BD_NONFINITE;
        for (int k = 0; k < 4; k++)
            if (!finite_f(d.quat[k])) return BD_NONFINITE;
        double qn = (double)d.quat[0] * d.quat[0] + (double)d.quat[1] * d.quat[1] + (double)d.quat[2] * d.quat[2] +
                    (double)d.quat[3] * d.quat[3];
        if (qn < 1e-12) return BD_QUAT;
    }
    if (d.mass < 0.f) return BD_MASS;
    if (d.mu < 0.f) return BD_MU;
    if (!(d.restitution >= 0.f && d.restitution <= 1.f)) return BD_RESTITUTION;
    int need = d.type == MS_SPHERE ? 1 : (d.type == MS_CAPSULE ? 2 : (d.type == MS_BOX ? 3 : 0));
    for (int k = 0; k < need; k++)
        if (!(d.p[k] > 0.f) || !finite_f(d.p[k])) return BD_SIZE;
    return 0;
}

// The same for a joint of an env of nb bodies (JD_*).
enum { JD_TYPE = 1, JD_BODIES, JD_NONFINITE, JD_LIMITS, JD_GAINS, JD_QUAT };
__host__ __device__ inline int joint_desc_check(const ms_joint_desc& d, int nb) {
    if (d.type != MS_REVOLUTE && d.type != MS_PRISMATIC) return JD_TYPE;
    if (d.parent < -1 || d.parent >= nb || d.child < 0 || d.child >= nb || d.parent == d.child) return JD_BODIES;
    for (int k = 0; k < 7; k++)
        if (!finite_f(d.parent_frame[k]) || !finite_f(d.child_frame[k])) return JD_NONFINITE;
    if (!finite_f(d.lower) || !finite_f(d.upper) || !finite_f(d.kp) || !finite_f(d.kd) || !finite_f(d.target0))
        return JD_NONFINITE;
    if (d.lower > d.upper) return JD_LIMITS;
    if (d.kp < 0.f || d.kd < 0.f) return JD_GAINS;
    const float* qa = d.parent_frame + 3;
    const float* qb = d.child_frame + 3;
    if (qa[0] * qa[0] + qa[1] * qa[1] + qa[2] * qa[2] + qa[3] * qa[3] < 1e-12f ||
        qb[0] * qb[0] + qb[1] * qb[1] + qb[2] * qb[2] + qb[3] * qb[3] < 1e-12f)
        return JD_QUAT;
    return 0;
}

// Soft-row parameters are finite and >= 0 (host).
inline bool soft_params_ok(const ms_sim_params* p) {
    const float v[4] = {p->contact_hertz, p->contact_damping_ratio, p->joint_hertz, p->joint_damping_ratio};
    for (float x : v)
        if (!(x >= 0.f) || !(x < 3.0e38f)) return false;
    return true;
}

// The soft-row constants of DevParams from the ABI parameters (host; h set).
inline void set_soft_params(DevParams& P, const ms_sim_params* p) {
    auto soft = [&](double hz, double zeta, float& rate, float& ms, float& is, float& ims) {
        rate = 0.f; ms = 1.f; is = 0.f; ims = 1.f;
        if (!(hz > 0.0)) return;
        double h = P.h, om = 2.0 * 3.14159265358979323846 * hz, a1 = 2.0 * zeta + h * om, a2 = h * om * a1;
        rate = (float)(om / a1);
        ms = (float)(a2 / (1.0 + a2));
        is = (float)(1.0 / (1.0 + a2));
        ims = (float)((1.0 + a2) / a2);
    };
    double chz = p->contact_hertz < 0.25 / P.h ? (double)p->contact_hertz : 0.25 / P.h;
    soft(chz, p->contact_damping_ratio, P.c_rate, P.c_ms, P.c_is, P.c_ims);
    soft(p->joint_hertz, p->joint_damping_ratio, P.j_rate, P.j_ms, P.j_is, P.j_ims);
}

// Hull library of a batch on the device (see HullRef): hull h's vertices
// v[vo[h] .. vo[h + 1]), triangles t[to[h] ..) with local planes n[..],
// edges e[eo[h] ..), bounding radius rad[h].
struct HullLib {
    const float4* v;
    const int4* t;
    const float4* n;
    const int4* e;
    const int* vo;
    const int* to;
    const int* eo;
    const float* rad;
};

// Pick task: delta joint-position controller and per-step records
// (reward, indicators, tcp / cube positions, joint coordinates, targets).
struct DevTask {
    int on;                            // actions are normalised deltas; records may be written
    int grip, fa, fb, cube, table;     // env-local gripper joint (-1: none), fingers, cube, table
    float grasp_tol, touch_tol;
    const float* half;                 // [A] (h - l) / 2 per joint slot
    float* qR;                         // [NJ] joint coordinates at the last controller reset
    float* out;                        // [n_steps][E][D] records of this call, or null
    int D;                             // record length, 10 + 2 A
};

struct DevBatch {
    int E, NB, NJ, A;
    DevParams P;
    DevTask T;
    const int* body_off;
    const int* joint_off;
    float4 *x, *q, *v, *w;
    const float4* shape;
    const float4* inv;                 // sqrt(1/Ixx), sqrt(1/Iyy), sqrt(1/Izz), 1/m (0 = static)
    const int2* meta;
    const unsigned long long* adj;
    const float4* jf;
    const float4* jp;
    const int4* jm;
    float* jt;
    const float* rest;                 // restitution per body
    const HullLib* hulls;              // device copy of the hull library, or null
    float4* wc;                        // warm start: 2 per (env, contact point): (a | b << 16, aA), (ln, friction)
    int* wc_n;                         //   contact points cached per env
    float* wjl;                        //   8 impulses per joint
    unsigned* status;
    char* plain_ws;
    Layout plain_layout;
    int4* rec_man;
    float* rec_pts;
    int* rec_cnt;
    int* rec_col;                      // colour per constraint (joints, then manifolds), [E][rec_col_stride]
    int rec_col_stride;
    float4* force;                     // contact force per body of the last step (null: off)
};

struct FusedCfg {
    Layout layout;
    int* queue;
    const int* order;
    char* gscratch;        // global part of every lane group's workspace
};

int launch_plain(const DevBatch& D, const float* actions, int n_steps, cudaStream_t s);
// k_fused<G, lean> of each lane-group size (ms_fused.cu, one translation unit per G)
const void* fused_kernel_1(unsigned variant);
const void* fused_kernel_2(unsigned variant);
const void* fused_kernel_4(unsigned variant);
const void* fused_kernel_8(unsigned variant);
const void* fused_kernel_16(unsigned variant);
const void* fused_kernel_32(unsigned variant);
// kernel variant bits of k_fused: FV_LEAN (no task, contact force,
// restitution, warm start or record code), FV_DYN (dynamic placement),
// FV_JOINTS (joint rows), FV_HULLS (hull routines); a variant without
// FV_LEAN always has FV_JOINTS and FV_HULLS.
enum : unsigned { FV_LEAN = 1u, FV_DYN = 2u, FV_JOINTS = 4u, FV_HULLS = 8u };
cudaError_t fused_occupancy(int G, unsigned variant, int threads, size_t smem, int* blocks_per_sm);
bool fused_supported(int G);
void fused_preload();
bool fused_lean(const DevBatch& D);   // whether a batch can run an FV_LEAN variant
cudaError_t launch_fused(const DevBatch& D, const float* actions, int n_steps, const FusedCfg& C, int G, unsigned variant,
                         int grid, int threads, size_t smem, cudaStream_t s);
void launch_pack_state(const DevBatch& D, float* out, cudaStream_t s);
// pick task: controller reset of the masked envs (all if mask is null) and
// the records of every env at the current state
void launch_task_reset(const DevBatch& D, const uint8_t* mask, cudaStream_t s);
void launch_task_observe(const DevBatch& D, float* out, cudaStream_t s);
void set_last_error(const char* msg);   // the message ms_last_error() returns on this thread

// batched camera rendering (ms_render.cu)
struct RenderState;
RenderState* render_create();
void render_destroy(RenderState* r);
const char* render_configure(RenderState* r, const DevBatch& D, const ms_camera_desc* c,
                             const std::vector<uint8_t>& types, const std::vector<int>& hull_nt,
                             const std::vector<int>& body_off, int max_nb, int smem_optin);
bool render_ready(const RenderState* r);
cudaError_t render_launch(RenderState* r, const DevBatch& D, uint8_t* rgba, float* depth, uint16_t* seg,
                          cudaStream_t s);

// read access to a batch's device view and sizes (for the step server)
const DevBatch& batch_dev(const ::ms_batch* b);
void batch_dims(const ::ms_batch* b, int* E, int* A, int* max_nb, int* max_nj);
// true when ms_step(b, ., n_steps, stream) will replay a graph (no capture)
bool batch_has_graph(const ::ms_batch* b, int n_steps);
// ms_step without a CUDA graph (queue reset + launch enqueued directly): for
// short-lived batches, where capturing a graph per batch costs more than it saves
ms_status batch_step_eager(::ms_batch* b, const float* actions, int n_steps, cudaStream_t stream);
void launch_unpack_state(const DevBatch& D, const float* in, const uint8_t* mask, const int* body_env,
                         cudaStream_t s);

}  // namespace ms
