// Internal declarations shared by the host API and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ms_math.cuh"

struct ms_batch;   // include/ms.h

namespace ms {

// Byte offsets of one env's arrays inside its workspace (-1: absent).  The
// workspace has a shared part (bodies, joints, colour lists, impulses: the
// data every sweep touches; in shared memory on the batched path) and a
// global part (AABBs, pairs, manifolds, contact anchors: written once per
// step; rows unless they fit the shared part).  The plain path keeps both
// parts in one global slot per env.
struct Layout {
    int s_bytes;
    int x, q, v, w, shape, inv, meta, adj;  // body copies (batched path only)
    int jf, jp, jm, jt;                     // joint copies (batched path only)
    int iw, cons, colr, scons, color_off, used, lam, cnt, status;
    bool lists_shared;                      // cons, colr, scons, lam in the shared part
    int rows_s;                             // rows in the shared part, or -1
    int g_bytes;
    int aabb, pairs, man, pts;
    int rows_g;                             // rows in the global part, or -1
    int rows_bytes;
};

Layout make_layout(int max_nb, int max_nj, int pair_cap, int contact_cap, bool with_bodies, bool rows_shared,
                   bool lists_shared);

// Kernel-side view of a batch (plain pointers, passed by value).
struct DevParams {
    float dt, h;
    int substeps, pos_iters, vel_iters;
    float gx, gy, gz;
    float margin, vmax;
    int pair_cap, contact_cap;
};

struct DevBatch {
    int E, NB, NJ, A;
    DevParams P;
    const int* body_off;
    const int* joint_off;
    float4 *x, *q, *v, *w;
    const float4* shape;
    const float4* inv;
    const int2* meta;
    const unsigned long long* adj;
    const float4* jf;
    const float4* jp;
    const int4* jm;
    float* jt;
    unsigned* status;
    char* plain_ws;
    Layout plain_layout;
    int4* rec_man;
    float* rec_pts;
    int* rec_cnt;
};

struct FusedCfg {
    Layout layout;
    int* queue;
    const int* order;
    char* gscratch;        // global part of every lane group's workspace
};

int launch_plain(const DevBatch& D, const float* actions, int n_steps, cudaStream_t s);
cudaError_t fused_occupancy(int G, int threads, size_t smem, int* blocks_per_sm);
bool fused_supported(int G);
cudaError_t launch_fused(const DevBatch& D, const float* actions, int n_steps, const FusedCfg& C, int G,
                         int grid, int threads, size_t smem, cudaStream_t s);
void launch_pack_state(const DevBatch& D, float* out, cudaStream_t s);
void set_last_error(const char* msg);   // the message ms_last_error() returns on this thread

// read access to a batch's device view and sizes (for the step server)
const DevBatch& batch_dev(const ::ms_batch* b);
void batch_dims(const ::ms_batch* b, int* E, int* A, int* max_nb, int* max_nj);
// true when ms_step(b, ., n_steps, stream) will replay a graph (no capture)
bool batch_has_graph(const ::ms_batch* b, int n_steps);
void launch_unpack_state(const DevBatch& D, const float* in, const uint8_t* mask, const int* body_env,
                         cudaStream_t s);

}  // namespace ms
