/*
 * ms.h -- C ABI of the B300 batched rigid-body step (libmsim.so).
 *
 * The library advances thousands of independent manipulation environments
 * ("envs") per call on one GPU: the GPU-parallel physics step the paper's
 * simulator runs for every parallel env (Sec. "GPU Parallelized Simulation
 * and Rendering"; heterogeneous envs with different object counts and DOF,
 * Sec. "Heterogeneous GPU Simulation"), with the drive targets of its PD
 * joint-position controller (Appendix "Controller / Action Space") and the
 * simulation-frequency / solver-iteration knobs of its benchmark setup
 * (Appendix "Simulation and Rendering Benchmarking", Setup).  Each call runs,
 * per env and step: broadphase, primitive narrowphase into <= 4-point
 * manifolds, greedy constraint colouring, then per substep constraint prep,
 * a fixed-iteration Gauss-Seidel / TGS solve with a Coulomb friction pyramid
 * and soft PD drives, and symplectic integration.
 *
 * Conventions: z-up world, SI units, quaternions (x, y, z, w), capsule axis
 * and plane normal along local +z, joint axis along the joint frame's +x.
 *
 * Errors: every function returns ms_status.  Argument errors are detected
 * synchronously and nothing is enqueued.  Conditions found on the device
 * (capacity overflow, non-finite state) set per-env status bits that
 * ms_sync() returns; device code never traps or asserts.  ms_last_error()
 * returns a thread-local description of the last failure.
 *
 * Threading: a batch may be used from one host thread at a time.
 */
#ifndef MS_H
#define MS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ms_status;
enum {
    MS_OK = 0,
    MS_ERR_INVALID_ARG = 1,
    MS_ERR_OOM = 2,
    MS_ERR_CUDA = 3,
    MS_ERR_CONTACT_OVERFLOW = 4,
    MS_ERR_COLOR_OVERFLOW = 5,
    MS_ERR_NAN = 6,
    MS_ERR_TIMEOUT = 7,
    MS_ERR_NOT_ADMITTED = 8,
    MS_ERR_BUSY = 9,
    MS_ERR_PAIR_OVERFLOW = 10,
    MS_ERR_NOT_FOUND = 11
};

/* per-env device status bits (ms_sync env_status) */
enum {
    MS_ENV_PAIR_OVERFLOW = 1u,      /* more broadphase pairs than pair_capacity   */
    MS_ENV_CONTACT_OVERFLOW = 2u,   /* more contact points than contact_capacity  */
    MS_ENV_COLOR_OVERFLOW = 4u,     /* a constraint found none of 64 colours free */
    MS_ENV_NAN = 8u,                /* non-finite state; the env is frozen        */
    MS_ENV_INVALID = 16u,           /* ms_step_noalloc: descriptors out of range; the env is skipped */
    MS_ENV_BOUNDS = 32u             /* debug library only: an index past its buffer was caught; the
                                       env's contacts and constraints were dropped for that step */
};

enum { MS_SPHERE = 0, MS_CAPSULE = 1, MS_BOX = 2, MS_PLANE = 3, MS_HULL = 4 };
enum { MS_REVOLUTE = 0, MS_PRISMATIC = 1 };

/* Body descriptor (84 bytes, no padding).
 *   p: sphere {r}, capsule {r, half_length}, box {hx, hy, hz}, plane unused,
 *   hull {index into the batch's hull library (an integer), unused, unused}.
 *   mass 0 (and every plane) = static: never moves; its velocities are ignored.
 *   Two bodies may touch iff (group_a & mask_b) && (group_b & mask_a). */
typedef struct {
    int32_t type;
    float p[3];
    float mass;
    float pos[3];
    float quat[4];
    float linvel[3];
    float angvel[3];
    float mu;
    float restitution;           /* [0, 1]; a contact uses the mean of its two bodies' */
    uint16_t group, mask;
} ms_body_desc;

/* Joint descriptor (88 bytes).  parent = -1 attaches to the world.  Frames
 * are (pos[3], quat[4]) in the body's local frame; the joint axis is the
 * frame's +x.  Limits are [lower, upper] (rad or m).  The drive pulls the
 * joint coordinate toward its target with stiffness kp and damping kd
 * (kp = kd = 0: no drive).  target0 is the initial target. */
typedef struct {
    int32_t type;
    int32_t parent, child;
    float parent_frame[7];
    float child_frame[7];
    float lower, upper, kp, kd, target0;
} ms_joint_desc;

/* One env: its bodies and joints (indices are env-local). */
typedef struct {
    int32_t n_bodies, n_joints;
    const ms_body_desc* bodies;
    const ms_joint_desc* joints;
} ms_scene_desc;

/* Solver parameters shared by every env of a batch.
 *   dt: step length; substeps: h = dt / substeps; pos_iters / vel_iters:
 *   solver sweeps per substep; margin: contact margin (speculative contacts
 *   are kept while d < margin); max_depen_vel: cap on the penetration
 *   recovery speed; pair_capacity / contact_capacity: per-env limits, beyond
 *   which pairs / manifolds are dropped in order and a status bit is set.
 * Optional solver variants (0 = off; all off gives the base method):
 *   linear_damping, angular_damping (1/s): implicit velocity damping each
 *   substep, v <- v / (1 + h c) (+ h g), w <- w / (1 + h c) (Box2D v3);
 *   bounce_threshold (m/s): after the last substep, a contact point whose
 *   step-start approach speed exceeds it and that carried a normal impulse
 *   leaves with normal velocity -e x that speed (e = mean restitution);
 *   warm_start: 1 carries impulses across steps -- joint rows keep theirs,
 *   the k-th point of a manifold takes the normal and (world-vector)
 *   friction impulses of the k-th point of the previous step's manifold of
 *   the same body pair.  ms_set_state clears this memory for the envs it
 *   sets.
 * Soft rows (the "soft step" of Box2D v3; 0 Hz = rigid): in the position
 *   sweeps a soft row is a spring-damper of natural frequency f (Hz) and
 *   damping ratio zeta on the row's own effective mass, integrated
 *   implicitly over the substep: with w = 2 pi f, a1 = 2 zeta + h w,
 *   a2 = h w a1, its bias is (w / a1) C and its update
 *   dlambda = -a2/(1 + a2) (Jv + bias)/k - lambda/(1 + a2).  Relax sweeps
 *   treat every row as rigid.
 *   contact_hertz, contact_damping_ratio: every contact normal row; a
 *   penetrating point (d < 0) takes the bias (w / a1) d (at most
 *   max_depen_vel), a separated one keeps its speculative bias d / h.  The
 *   frequency is capped at a quarter of the substep rate, 0.25 / h.
 *   joint_hertz, joint_damping_ratio: the equality rows of every joint (point
 *   and angular rows; not limits or drives). */
typedef struct {
    float dt;
    int32_t substeps, pos_iters, vel_iters;
    float gravity[3];
    float margin;
    float max_depen_vel;
    int32_t contact_capacity;
    int32_t pair_capacity;
    float linear_damping, angular_damping;
    float bounce_threshold;
    int32_t warm_start;
    float contact_hertz, contact_damping_ratio;
    float joint_hertz, joint_damping_ratio;
} ms_sim_params;

typedef struct ms_batch ms_batch;

/* Borrowed device views of a batch's resident state (structure of arrays).
 * Valid until the next ms_step / ms_step_plain / ms_set_state / ms_destroy.
 * x, q, v, w: float4 per body (pos | quat xyzw | linvel | angvel; .w of x,
 * v, w unused).  body_off / joint_off: int32 [n_envs + 1] CSR offsets.
 * targets: float per joint.  status: uint32 per env. */
typedef struct {
    int32_t n_envs, n_bodies, n_joints, max_act;
    void* x;
    void* q;
    void* v;
    void* w;
    const int32_t* body_off;
    const int32_t* joint_off;
    float* targets;
    uint32_t* status;
} ms_state_view;

/* Create a batch of n_envs envs (each up to 64 bodies).  The descriptors are
 * validated and copied; the caller keeps ownership of descs.  The batch owns
 * all device memory it allocates on the current device.
 * Errors: MS_ERR_INVALID_ARG (bad descriptor or parameter; ms_last_error
 * names the env and field), MS_ERR_OOM, MS_ERR_CUDA. */
ms_status ms_create_batch(const ms_scene_desc* descs, int n_envs, const ms_sim_params* p,
                          ms_batch** out);

/* Same, from flat tables: bodies[body_off[E]], joints[joint_off[E]] with
 * body_off / joint_off int32 [n_envs + 1]. */
ms_status ms_create_batch_flat(const ms_body_desc* bodies, const int32_t* body_off,
                               const ms_joint_desc* joints, const int32_t* joint_off,
                               int n_envs, const ms_sim_params* p, ms_batch** out);

/* Convex hull library (the convex pieces of decomposed meshes), host arrays,
 * copied at creation.  Hull h has vertices verts[vert_off[h] .. vert_off[h + 1])
 * (x, y, z; 4..16 vertices) and outward counter-clockwise triangles
 * tris[tri_off[h] .. tri_off[h + 1]) (3 vertex indices local to the hull),
 * forming a closed mesh.  The body frame of a hull body is the hull's
 * principal frame: its centroid at the origin and its principal axes of
 * inertia along x, y, z (the library's vertices are given in that frame).
 * Contacts: hull - plane (vertices within the margin), sphere - hull (face
 * of least penetration when the centre is inside, else the closest surface
 * point), box or hull - hull (separating axes over face normals and the edge
 * pairs bounding the Minkowski difference; face clipping or one edge-edge
 * point), capsule - hull (separating axes over the hull's face normals and
 * the segment x edge directions; the segment clipped to the best face, up
 * to two points, else the exact closest points of segment and surface).
 * The inertia is that of
 * the uniform solid; the broadphase bounds a hull by its vertices' bounding
 * sphere about the body origin. */
typedef struct {
    int32_t n_hulls;
    const int32_t* vert_off;
    const float* verts;
    const int32_t* tri_off;
    const int32_t* tris;
} ms_hull_lib;

/* ms_create_batch_flat with a hull library (NULL: none); MS_HULL bodies
 * need one.  MS_ERR_INVALID_ARG names a malformed hull (not closed, a
 * vertex count out of range, no volume) or a body's hull index out of
 * range. */
ms_status ms_create_batch_hulls(const ms_body_desc* bodies, const int32_t* body_off,
                                const ms_joint_desc* joints, const int32_t* joint_off, int n_envs,
                                const ms_sim_params* p, const ms_hull_lib* hulls, ms_batch** out);

/* Advance every env n_steps steps on `stream` (cudaStream_t; NULL = legacy
 * default stream) with the batched path: one persistent launch pops envs
 * from a work queue (longest first) and keeps each env's bodies, contacts
 * and rows on chip for all n_steps; the launch sequence is captured once per
 * (n_steps, tuning) in a CUDA graph and replayed.
 * actions: device float [n_steps][n_envs][A] drive targets (A = the
 * batch's max joints per env), NaN = keep the previous target; NULL = no
 * change (with a task set, normalised deltas: see ms_set_task).  Must stay
 * valid until the stream reaches the step.  Asynchronous: returns after
 * enqueueing. */
ms_status ms_step(ms_batch* b, const float* actions, int n_steps, void* stream);

/* Same step through the plain comparison path: one block per env and one
 * kernel launch per stage (and per solver sweep), state in global memory.
 * Results are bit-identical to ms_step. */
ms_status ms_step_plain(ms_batch* b, const float* actions, int n_steps, void* stream);

/* Borrowed device pointers to the resident state (see ms_state_view). */
ms_status ms_get_state(ms_batch* b, ms_state_view* out);

/* Copy the state as float [n_bodies][13] = pos[3], quat[4], linvel[3],
 * angvel[3] to dst (dst_kind 0 = host, 1 = device), ordered on `stream`.
 * A host dst should be pinned for the copy to overlap. */
ms_status ms_copy_state(ms_batch* b, float* dst, int dst_kind, void* stream);

/* Overwrite the state of the envs whose env_mask byte is non-zero
 * (env_mask NULL = all envs; host array of n_envs bytes) from src float
 * [n_bodies][13] (src_kind 0 = host, 1 = device), verbatim: quaternions must
 * be unit, and a state saved with ms_copy_state restores bit for bit.
 * Static bodies keep their pose.  Clears those envs' status bits.  Used for
 * partial resets and checkpoint restore.  Returns after the copy is done. */
ms_status ms_set_state(ms_batch* b, const float* src, int src_kind, const uint8_t* env_mask,
                       void* stream);

/* Wait for the batch's last stream, then OR the per-env status bits.
 * env_status (nullable) receives uint32 [n_envs].  Returns MS_OK, or the
 * error of the first set bit in order pair, contact, colour, NaN. */
ms_status ms_sync(ms_batch* b, uint32_t* env_status);

/* Free the batch (synchronises its stream).  NULL is accepted. */
ms_status ms_destroy(ms_batch* b);

/* Thread-local description of the last error, "" if none. */
const char* ms_last_error(void);

/* ----------------------------------------------------------------------- */
/* Pick task: controller, observations, reward                              */
/* ----------------------------------------------------------------------- */

/* The pick task of the paper's sim2real appendix (Controller / Action Space,
 * Observation Space, Reward), run inside the step's kernels.  Indices are
 * env-local and must be valid in every env of the batch:
 *   grip_joint: the gripper joint (-1: none, never grasped); finger_a,
 *   finger_b: the two finger bodies (tcp = midpoint of their centres, g =
 *   finger_b - finger_a); cube: a box body (side c = 2 x its first
 *   half-extent); table: a plane body.
 *   grasp_tol: grasped = the gripper joint is more than grasp_tol (rad or m)
 *   from its target, i.e. something blocks it.  touch_tol (m): a finger
 *   whose lowest point is within touch_tol of the table touches it.
 *   n_joints must equal the batch's A (max joints per env); delta_lo,
 *   delta_hi: host float [A], the delta controller's bounds per joint slot.
 * With a task set, an action is a normalised delta: the joint's target
 * moves by clip(a, -1, 1) (h - l) / 2 each step (NaN: no change). */
typedef struct {
    int32_t grip_joint;
    int32_t finger_a, finger_b;
    int32_t cube;
    int32_t table;
    float grasp_tol;
    float touch_tol;
    int32_t n_joints;
    const float* delta_lo;
    const float* delta_hi;
} ms_task_desc;

/* Set (t != NULL) or remove (t == NULL) the batch's task.  Setting it resets
 * the controller of every env (ms_task_reset) on `stream`.  The descriptor
 * is copied.  Errors (synchronous, nothing changed): MS_ERR_INVALID_ARG for
 * an index out of range in some env, a cube that is not a box, a table that
 * is not a plane, n_joints != A, a negative or non-finite tolerance or
 * bound. */
ms_status ms_set_task(ms_batch* b, const ms_task_desc* t, void* stream);

/* Controller reset of the envs whose env_mask byte is non-zero (NULL = all;
 * host array of n_envs bytes): each joint's target and its reset coordinate
 * q_reset (used by the reward) become its current coordinate.  A partial
 * reset is ms_set_state(mask) followed by ms_task_reset(mask).
 * MS_ERR_INVALID_ARG without a task.  Returns after the mask is copied. */
ms_status ms_task_reset(ms_batch* b, const uint8_t* env_mask, void* stream);

/* Length of one task record: 10 + 2 A floats =
 *   reward, grasped (0/1), tcp_close (0/1), touch_table (0/1), x_tcp[3],
 *   x_cube[3], q[A] (joint coordinates, 0 past the env's joints),
 *   target[A].  reward = r_dist(|tcp - x_cube|, 15) + (1 - g.z / |g|)
 *   + 2 tcp_close r_dist(| |g| - c |, 40) + grasped (1 + 3 r_dist(
 *   |q - q_reset|, 4 / pi)) - 2 touch_table, r_dist(d, z) = 1 - tanh(z d),
 *   tcp_close = |tcp - x_cube| <= c / 2.  An env frozen by a non-finite
 *   state writes NaN. */
int ms_task_record_len(const ms_batch* b);

/* The record of every env at the current state into out (device float
 * [n_envs][ms_task_record_len]), on `stream`.  MS_ERR_INVALID_ARG without a
 * task. */
ms_status ms_task_observe(ms_batch* b, float* out, void* stream);

/* ms_step (flags 0) or ms_step_plain (flags MS_STEP_PLAIN) that also writes
 * one task record per step and env into out (device float
 * [n_steps][n_envs][ms_task_record_len], nullable; non-NULL needs a task).
 * out must stay valid until the stream reaches the step. */
enum { MS_STEP_PLAIN = 1 };
ms_status ms_step_ex(ms_batch* b, const float* actions, int n_steps, float* out, int flags, void* stream);

/* ms_step with host buffers on both sides, for callers whose actions and
 * results live in host memory: copies actions (host float
 * [n_steps][n_envs][n_act], nullable = keep every target) into a device
 * buffer the batch owns, steps n_steps, and copies into out (host) either
 * the state afterwards (out_kind 0: float [n_bodies][13], as ms_copy_state)
 * or the task records of every step (out_kind 1: float
 * [n_steps][n_envs][ms_task_record_len]; needs a task).  All copies and the
 * step are ordered on `stream`; pinned host buffers let the call return
 * before they finish, and both must stay valid until the stream reaches the
 * copies.  The batch's device buffers are shared by its calls: calls on
 * different streams must be ordered by the caller.  MS_ERR_INVALID_ARG for
 * a NULL out or an unknown out_kind; MS_ERR_OOM if a buffer cannot grow. */
ms_status ms_step_host(ms_batch* b, const float* actions, int n_steps, float* out, int out_kind, void* stream);

/* ----------------------------------------------------------------------- */
/* Batched camera rendering                                                 */
/* ----------------------------------------------------------------------- */

/* One pinhole camera per env, the same in every env's own frame (the
 * paper's batched rendering of every env's camera; its observation is a 128 x
 * 128 RGB image), rendered from the resident body poses by a CUDA triangle
 * rasteriser: each primitive is a fixed mesh (box 12 triangles; sphere a UV
 * mesh of 5 rings x 12 points and two poles, 120; capsule the same rings with
 * the upper hemisphere at +l and the lower at -l, 144; plane the square
 * [-2, 2]^2 of its local xy, 2).  eye looks at target with world up +z
 * (the view must not be vertical); focal length (height / 2) / tan(fov_y / 2)
 * pixels; pixel (i, j) is centred at (i + 0.5, j + 0.5), row 0 at the top.
 * Back faces are skipped, triangles are clipped to view depth >= near, a
 * pixel centre on or inside all three edges is covered, and the covering
 * triangle of least (perspective-correct view depth, triangle index) wins.
 * width x height <= 16384.  body_rgb: host float [n_bodies][3] in [0, 1],
 * copied. */
typedef struct {
    float eye[3];
    float target[3];
    float fov_y;
    float near;
    int32_t width, height;
    const float* body_rgb;
} ms_camera_desc;

/* Set the batch's camera (synchronous).  MS_ERR_INVALID_ARG for a degenerate
 * or vertical view, a size out of range, colours outside [0, 1]. */
ms_status ms_set_camera(ms_batch* b, const ms_camera_desc* c);

/* Render every env at its current state on `stream` into device buffers
 * (each nullable): rgba uint8 [n_envs][height][width][4] = round(255 base
 * (0.3 + 0.7 max(0, n.l))) per channel, alpha 255, l = normalize(0.3, 0.2, 1),
 * n the triangle's world normal, background 0; depth float [n_envs][height]
 * [width] = view depth, background 0; seg uint16 [n_envs][height][width] =
 * env-local body index + 1, background 0.  MS_ERR_INVALID_ARG without a
 * camera. */
ms_status ms_render(ms_batch* b, uint8_t* rgba, float* depth, uint16_t* seg, void* stream);

/* ----------------------------------------------------------------------- */
/* Introspection and tuning                                                */
/* ----------------------------------------------------------------------- */

/* Record the contact manifolds and the constraint colours of every env's
 * last step (off by default; costs one extra global write per contact and
 * per constraint).  record = 0 / 1. */
ms_status ms_set_record_contacts(ms_batch* b, int record);

/* Contact manifolds recorded at env `env`'s last step, in pair order:
 * pairs int32 [cap][2] (env-local bodies a, b; a is the lower shape rank or
 * index), npts int32 [cap], pts float [cap][4][10] = cA[3], cB[3], n[3], d
 * (n points from b toward a, d = n.(cA - cB)).  Host buffers; synchronises.
 * *count receives the number of manifolds (at most cap are written).
 * MS_ERR_INVALID_ARG if recording is off. */
/* Colours recorded at env `env`'s last step: colors int32 [cap], one per
 * constraint of the greedy colouring's list -- the env's joints in index
 * order, then its manifolds in pair order (those ms_get_contacts returns);
 * -1 for a constraint that found none of the 64 colours free.  Host buffer;
 * synchronises.  *count receives the constraint count.  MS_ERR_INVALID_ARG if
 * recording is off. */
ms_status ms_get_colors(ms_batch* b, int env, int cap, int32_t* colors, int* count);

ms_status ms_get_contacts(ms_batch* b, int env, int cap, int32_t* pairs, int32_t* npts,
                          float* pts, int* count);

/* Contact forces per body: the readout behind the touch sensors of the
 * paper's dextrous-manipulation tasks (appendix "Environments and Robots
 * List", "Dextrous Manipulation"), a force per link from the solver's
 * contact impulses.  ms_enable_contact_forces(b, 1) makes every later step
 * of ms_step / ms_step_plain write, for each body, the impulses of the
 * contact rows of every manifold that involves it over the step's last
 * substep, divided by the substep h: (F[3], f_n) with F = the sum of
 * +-dir lambda (+ for the manifold's body a, - for body b; the normal and
 * both friction rows) and f_n = the sum of its normal impulses.  A body at
 * rest on a support reads F = -m g.  0 turns it off (the buffer is kept).
 * The step server and the no-allocation path do not write it.
 * ms_contact_forces copies the last step's values into out (device float
 * [n_bodies][4], ordered on stream); MS_ERR_INVALID_ARG when off. */
ms_status ms_enable_contact_forces(ms_batch* b, int on);
ms_status ms_contact_forces(ms_batch* b, float* out, void* stream);

/* Batched-path launch shape.  lanes_per_env in {1, 2, 4, 8, 16, 32}: a warp
 * steps 32 / lanes_per_env envs in lockstep; warps_per_cta in [1, 8];
 * rows_in_smem (placement of the constraint lists, impulses and rows):
 *   1  every row in shared memory when one CTA fits (else as 0);
 *   0  per-env slots sized for the capacities (lists, impulses, joint rows
 *      and the rows of as many contact points as leave enough CTAs resident
 *      for all envs to be in flight at once) when that holds every contact
 *      point; otherwise the dynamic placement at that residency: each warp's
 *      envs share a shared-memory arena, handed out after every step's
 *      narrowphase by the counts of that step (lists and impulses first,
 *      then joint rows, then contact rows levelled across the envs);
 *   2  the dynamic placement with one CTA per SM.
 * Whatever is not in shared memory stays in an L2-resident global slot per
 * lane group.  Any choice gives bit-identical results; other values of
 * rows_in_smem are MS_ERR_INVALID_ARG. */
typedef struct {
    int32_t lanes_per_env;
    int32_t warps_per_cta;
    int32_t rows_in_smem;
    int32_t ctas_per_sm;     /* output of ms_get_tuning: resident CTAs per SM */
} ms_tuning;

ms_status ms_set_tuning(ms_batch* b, const ms_tuning* t);
ms_status ms_get_tuning(ms_batch* b, ms_tuning* t);

/* Time each candidate tuning on `n_steps`-step calls (state is saved and
 * restored around the trials), keep the fastest.  cache_path (nullable): a
 * JSON file mapping a scene signature to its best tuning; read first, and
 * updated after tuning.  best (nullable) receives the choice. */
ms_status ms_autotune(ms_batch* b, int n_steps, const char* cache_path, ms_tuning* best, void* stream);

/* Device-memory hook, for callers whose device memory belongs to another
 * allocator (a framework's caching allocator).  Every device allocation of a
 * batch created after the call -- its state, parameters, workspaces, record,
 * task and staging buffers -- comes from alloc(bytes, device, stream, user),
 * stream being the batch's own setup stream, and goes back through
 * free(ptr, device, stream, user) when the batch is destroyed, after the
 * batch's work has finished.  alloc returns NULL on failure (the creating
 * call then fails with MS_ERR_OOM).  A batch keeps the hook it was created
 * under, so the functions and user must outlive it; ms_set_allocator(NULL,
 * NULL, NULL) restores the library's own stream-ordered pool for later
 * batches.  Setting only one function is MS_ERR_INVALID_ARG.  The tuner's
 * temporary state copies still use the library's pool. */
typedef void* (*ms_alloc_fn)(size_t bytes, int device, void* stream, void* user);
typedef void (*ms_free_fn)(void* ptr, int device, void* stream, void* user);
ms_status ms_set_allocator(ms_alloc_fn alloc, ms_free_fn free_fn, void* user);

/* Device bytes held by the batch (state, parameters, workspaces). */
ms_status ms_memory_bytes(ms_batch* b, size_t* bytes);

/* Estimated device bytes of a batch before creating it (for admission). */
ms_status ms_estimate_bytes(const int32_t* body_off, const int32_t* joint_off, int n_envs,
                            const ms_sim_params* p, size_t* bytes);

/* sizeof(ms_body_desc), sizeof(ms_joint_desc), sizeof(ms_sim_params),
 * sizeof(ms_state_view), sizeof(ms_tuning): lets bindings check layouts. */
void ms_abi_sizes(int32_t* out5);

/* ----------------------------------------------------------------------- */
/* Measurement                                                             */
/* ----------------------------------------------------------------------- */

/* The FP32 fused-multiply-add rate of the current device, measured: a
 * full-occupancy grid whose threads each run 8 independent chains of
 * dependent FMAs, timed with CUDA events over about `seconds` (in (0, 10])
 * on the legacy default stream, synchronously.  *flops_per_s receives the
 * rate (2 flop per FMA); sm_count and measured_s (nullable) receive the SM
 * count and the timed duration.  This is the peak the batched step's ALU
 * roofline divides by (the step is not a dense contraction, so tensor-core
 * rates do not apply).  It allocates and frees a small device buffer. */
ms_status ms_measure_fp32_peak(double seconds, double* flops_per_s, int* sm_count, double* measured_s);

/* ----------------------------------------------------------------------- */
/* Stepping without any device allocation                                  */
/* ----------------------------------------------------------------------- */

/* Caller-owned device arrays of a batch (all pointers are device pointers;
 * the library never allocates or frees them).
 *   body_off, joint_off: int32 [n_envs + 1] CSR offsets.
 *   bodies, joints: descriptors (the pose / velocity fields of bodies are
 *     not read; shapes, masses, friction and filters are).
 *   x, q, v, w: float4 [n_bodies] state, read and written in place (.w of x
 *     and w unused; v.w receives the inverse mass).  q must hold unit
 *     quaternions.
 *   targets: float [n_joints] drive targets, read and written in place.
 *   status: uint32 [n_envs] status bits (MS_ENV_*), read and written.  An
 *     env whose counts exceed the maxima below, or whose descriptors break a
 *     rule ms_create_batch enforces (a body type other than sphere, capsule,
 *     box or plane; a shape size not > 0; a negative or non-finite mass or
 *     mu; restitution outside [0, 1]; a joint of unknown type, naming bodies
 *     out of range or itself, with non-finite frames or limits or gains,
 *     lower > upper, a negative gain or a zero frame quaternion) gets
 *     MS_ENV_INVALID and is skipped whole: its x, q, v, w, targets are left
 *     untouched.  The bit is or-ed into the word and stays set -- the env
 *     stays skipped -- until the caller clears status[env]; so does
 *     MS_ENV_NAN.  The offsets must lie inside the caller's arrays.
 *   max_bodies_per_env in [1, 64] and max_joints_per_env in [0, 512] bound
 *   every env; actions rows are max_joints_per_env wide. */
typedef struct {
    int32_t n_envs, max_bodies_per_env, max_joints_per_env;
    const int32_t* body_off;
    const int32_t* joint_off;
    const ms_body_desc* bodies;
    const ms_joint_desc* joints;
    float* x;
    float* q;
    float* v;
    float* w;
    float* targets;
    uint32_t* status;
} ms_noalloc_batch;

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory -- a process whose device memory is
 * owned entirely by another allocator (a framework's caching allocator or a
 * fixed arena), or a control loop that cannot afford an allocation's
 * implicit synchronisation and latency.  It advances every env n_steps
 * steps with the same stages and results as ms_step, on `stream`, calling no
 * cudaMalloc, cudaFree or allocating library routine.  It covers primitive
 * shapes only: no hull library, no warm start across steps (no memory
 * between calls; warm_start = 1 is rejected), no pick task and no contact
 * forces or contact record.  The inertia of each body is derived from its
 * descriptor by ms_create_batch's formula.
 *
 * The kernel's workspace is a fixed 32 MiB array inside the library, held by
 * every GPU that loads the library until the process exits.  A call whose
 * per-CTA workspace would not fit it returns MS_ERR_INVALID_ARG (with a
 * message from ms_last_error) and enqueues nothing.  All calls share the
 * array: calls that overlap on the GPU (different streams or host threads)
 * race and must be serialised by the caller.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) and sets the
 * kernels' shared-memory limit; make that first call before any stream
 * capture.  actions as in ms_step.  Asynchronous; argument errors are
 * synchronous. */
ms_status ms_step_noalloc(const ms_noalloc_batch* b, const ms_sim_params* p, const float* actions,
                          int n_steps, void* stream);

#ifdef __cplusplus
}
#endif
#endif
