/*
 * FP64 CPU oracle of the batched rigid-body step -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code, header or constant table
 * with the CUDA path; it consumes the same seeded scene descriptors.
 *
 * The step is the one described in the paper's GPU-parallel simulation
 * (Sec. "GPU Parallelized Simulation and Rendering", Appendix "Simulation and
 * Rendering Benchmarking", Setup: simulation frequency and solver position /
 * velocity iteration counts) with the PD joint-target drive of Appendix
 * "Controller / Action Space".  The paper delegates the physics to an engine
 * and states no algorithm, so each stage follows a named published method:
 *   broadphase       brute-force AABB overlap with a contact margin
 *   narrowphase      closest points and SAT (Ericson 2005, Real-Time Collision
 *                    Detection, 4.4, 5.1.9) with Sutherland-Hodgman clipping
 *   colouring        greedy graph colouring over the constraint list
 *   solver           substepped sequential impulses with soft drives
 *                    (Catto 2005; Catto 2011 soft constraints; Macklin et al.
 *                    2019 "Small Steps"), Coulomb friction pyramid; contact
 *                    anchors keep their step-start orientation and the
 *                    separation advances to first order in each body's
 *                    rotation since the step start (temporal Gauss-Seidel)
 *   integration      symplectic Euler with quaternion renormalisation
 *   contact forces   per body, the last substep's contact impulses / h
 *
 * Descriptor rows are doubles (converted losslessly from the float32 scene):
 *   body  [22]: type, p0, p1, p2, mass, pos[3], quat[4] (x,y,z,w), linvel[3],
 *               angvel[3], mu, restitution, group, mask
 *   joint [22]: type, parent, child, parent_frame[7] (pos, quat), child_frame[7],
 *               lower, upper, kp, kd, target0
 *   params[19]: dt, substeps, pos_iters, vel_iters, gx, gy, gz, margin,
 *               max_depen_vel, contact_capacity, pair_capacity,
 *               linear_damping, angular_damping, bounce_threshold, warm_start,
 *               contact_hertz, contact_damping_ratio, joint_hertz,
 *               joint_damping_ratio
 *
 * Soft rows (Box2D v3's "soft step"; a frequency of 0 makes them rigid): in
 * the position iterations, every contact normal row (contact_hertz, capped
 * at a quarter of the substep rate) and every joint equality row
 * (joint_hertz) is a spring-damper on the row's own effective mass,
 * integrated implicitly over the substep: with w = 2 pi hz,
 * a1 = 2 zeta + h w, a2 = h w a1,
 *     dlambda = -a2/(1 + a2) (Jv + bias)/k - lambda/(1 + a2),
 * bias = (w / a1) C for a joint error C, (w / a1) d for a penetrating
 * contact (d < 0, floored at -max_depen_vel) and d / h (speculative) for a
 * separated one; relax iterations solve every row rigid.
 *
 * Optional solver variants (all off in the default parameters):
 *   damping          per substep v <- v / (1 + h c_lin) + h g,
 *                    w <- w / (1 + h c_ang) (implicit damping, Box2D v3)
 *   restitution      after the last substep, per contact point whose
 *                    step-start approach speed exceeds bounce_threshold and
 *                    that carried a normal impulse: the normal impulse that
 *                    makes the normal velocity -e times the approach speed
 *                    (Box2D v3 solver), e = mean of the two restitutions
 *   warm start       impulses carried across steps: joint rows keep theirs;
 *                    the k-th point of a manifold takes those of the k-th
 *                    point of the previous step's manifold of the same body
 *                    pair (friction as a world vector, projected)
 */
#ifndef MS_ORACLE_H
#define MS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_world oracle_world;

enum { OR_SPHERE = 0, OR_CAPSULE = 1, OR_BOX = 2, OR_PLANE = 3, OR_HULL = 4 };
enum { OR_REVOLUTE = 0, OR_PRISMATIC = 1 };
enum { OR_ST_PAIR_OVERFLOW = 1, OR_ST_CONTACT_OVERFLOW = 2, OR_ST_COLOR_OVERFLOW = 4 };

/* Counter slots returned by oracle_counters (sums over envs and steps). */
enum {
    OC_STEPS = 0, OC_PAIRS_TESTED, OC_PAIRS_CANDIDATE,
    OC_NP_SS, OC_NP_SC, OC_NP_SB, OC_NP_SP, OC_NP_CC, OC_NP_CB, OC_NP_CP, OC_NP_BB, OC_NP_BP,
    OC_CONTACT_POINTS, OC_CONSTRAINTS, OC_ROWS_PREP, OC_ROW_SOLVE_2DYN, OC_ROW_SOLVE_1DYN,
    OC_WARM_APPLY, OC_BODY_INTEGRATE, OC_BODY_INERTIA, OC_COLORS, OC_NP_SH, OC_NP_XH, OC_NP_HP,
    OC_SAT_FACE_VERT, OC_SAT_EDGE_PAIR, OC_NP_CH, OC_NUM
};

oracle_world* oracle_create(int n_envs, const long long* body_off, const double* bodies,
                            const long long* joint_off, const double* joints,
                            const double* params);
/* The same with a hull library: hull h has vertices verts[vert_off[h] ..
 * vert_off[h + 1]) (x, y, z, body frame = its principal frame) and outward
 * counter-clockwise triangles tris[tri_off[h] .. tri_off[h + 1]) (3 vertex
 * indices local to the hull); a HULL body has p0 = its hull index.  Hulls:
 * 4..16 vertices, a closed mesh.  Returns NULL for a malformed hull.
 * Contacts: hull - plane (vertices within the margin), sphere - hull (face
 * of least penetration inside, closest surface point outside), box or
 * hull - hull (SAT over face normals and Gauss-map edge pairs, face
 * clipping or one edge-edge point), capsule - hull (SAT over face normals
 * and segment x edge axes; the segment clipped to the face, else the exact
 * segment - surface closest points). */
oracle_world* oracle_create_hulls(int n_envs, const long long* body_off, const double* bodies,
                                  const long long* joint_off, const double* joints, const double* params,
                                  int n_hulls, const int* vert_off, const double* verts, const int* tri_off,
                                  const int* tris);
/* Diagonal inertia of a hull of the given mass about its body axes (uniform
 * density); -1 for a malformed hull. */
int oracle_hull_inertia(const double* verts, int nv, const int* tris, int nt, double mass, double* out3);
void oracle_destroy(oracle_world* w);
/* Test probe (off by default): on != 0 stores, rounded to float32, what a
 * float32 implementation stores: every body's velocities and pose after each
 * update (impulse, gravity, integration), each constraint row (Jacobian,
 * effective mass, bias, softness, friction coefficient) when it is prepared,
 * each accumulated impulse after its update, and each contact point's normal
 * and body-local anchors; the arithmetic stays FP64.  Used to select envs
 * whose rollout is insensitive to that rounding. */
void oracle_set_round32(oracle_world* w, int on);

/* Advance every env n_steps steps.  actions: [n_steps][n_envs][A] drive
 * targets (NaN keeps the previous target) or NULL.  n_threads >= 1 splits the
 * envs statically over pthreads.  Returns 0. */
int oracle_step(oracle_world* w, const double* actions, int A, int n_steps, int n_threads);

/* State of all bodies, [n_bodies][13] = pos[3], quat[4], linvel[3], angvel[3]. */
void oracle_get_state(const oracle_world* w, double* out);
/* Contact forces of the last step, [n_bodies][4] = F[3], f_n: per body, the
 * impulses of the contact rows of every manifold that involves it over the
 * last substep, divided by h (+ on the manifold's body a, - on body b), and
 * the sum of its normal impulses / h. */
void oracle_contact_forces(const oracle_world* w, double* out);
/* Overwrite the state of all bodies (same layout); used for restart tests. */
void oracle_set_state(oracle_world* w, const double* in);
/* Current drive targets [n_joints]. */
void oracle_get_targets(const oracle_world* w, double* out);
/* Overwrite the drive targets [n_joints]. */
void oracle_set_targets(oracle_world* w, const double* in);

unsigned oracle_env_status(const oracle_world* w, int env);
/* Number of discrete decisions of the env (since create) whose deciding
 * quantity was within 1e-5 of its threshold. */
long long oracle_env_ties(const oracle_world* w, int env);
void oracle_counters(const oracle_world* w, long long* out /* [OC_NUM] */);

/* Contact manifolds of the env's last narrowphase, in pair order.
 * pairs [cap][2] (env-local body indices a, b), npts [cap],
 * pts [cap][4][10] = cA[3], cB[3], n[3], d.  Returns the manifold count
 * (at most cap are written). */
int oracle_get_manifolds(const oracle_world* w, int env, int cap, int* pairs, int* npts, double* pts);
/* Pairs whose any candidate point had |d - margin| < 1e-5 in the last
 * narrowphase (excluded from exact pair-set comparison).  Returns count. */
int oracle_get_margin_ties(const oracle_world* w, int env, int cap, int* pairs);
/* Colour of each constraint (joints, then manifolds) of the last step. */
int oracle_get_colors(const oracle_world* w, int env, int cap, int* colors);
/* Rows of the env's last substep in constraint-list order:
 * [cap][16] = a, b, kind, lin[3], angA[3], angB[3], k, bias, lambda, mu. */
int oracle_get_rows(const oracle_world* w, int env, int cap, double* rows);

/* Narrowphase of one pair in isolation.  bodyA, bodyB are descriptor rows
 * (A must be the lower shape rank, or the lower index for equal ranks).
 * out [8][10] as in oracle_get_manifolds.  Returns the point count after
 * the margin filter and the reduction to 4. */
int oracle_collide(const double* bodyA, const double* bodyB, double margin, double* out);

/* The candidate points of one pair before the margin filter and the
 * reduction to 4 (clip output order for box - box faces), same layout as
 * oracle_collide, out [16][10].  Returns the candidate count. */
int oracle_candidates(const double* bodyA, const double* bodyB, double margin, double* out);
/* The manifold reduction of n (5..16) candidates [n][10] (cB at 3..5, d at
 * 9): sel [4] receives the indices p1..p4.  Returns 4, or -1 for n out of
 * range. */
int oracle_reduce4(int n, const double* pts, int* sel);
/* The contact tangent basis of a unit normal n[3]: t1, t2 [3]. */
void oracle_tangents(const double* n, double* t1, double* t2);

/* Greedy colouring of a constraint list given as body pairs (-1 = static);
 * dyn[i] != 0 marks body i dynamic.  Returns the colour count or -1 on
 * overflow of 64 colours. */
int oracle_color(int n_cons, const int* a, const int* b, const int* dyn, int* colors);

/* Body-frame diagonal inertia of a descriptor row (mass > 0). */
void oracle_inertia(const double* body, double* out3);

/* Pick task of the paper's sim2real appendix (Controller / Action Space,
 * Observation Space, Reward).  idx = {gripper joint (-1 = none), finger a,
 * finger b, cube (a box), table (a plane)}, env-local and the same in every
 * env; tol = {grasp_tol, touch_tol}; lo, hi [A] the delta controller's bounds
 * per joint slot.  Once set, an action a is a normalised delta: the target
 * moves by clip(a, -1, 1) (h - l) / 2 (NaN: no change).  Setting the task
 * resets the controller of every env (target = q = q_reset).  Returns -1
 * (nothing changed) when an index is out of range or of the wrong type. */
int oracle_set_task(oracle_world* w, const int* idx, const double* tol, int A, const double* lo,
                    const double* hi);
/* Controller reset of the envs with mask[e] != 0 (all if mask is NULL):
 * target = q = q_reset from the current state. */
void oracle_task_reset(oracle_world* w, const unsigned char* mask);
/* oracle_step plus one task record per step and env: out [n_steps][E][D],
 * D = 10 + 2A = reward, grasped, tcp_close, touch_table, x_tcp[3],
 * x_cube[3], q[A], target[A]; ties [n_steps][E] (nullable) = decisions
 * within 1e-5 of their threshold (1 grasped, 2 tcp_close, 4 touch_table).
 * Returns -1 when no task is set. */
int oracle_step_task(oracle_world* w, const double* actions, int A, int n_steps, int n_threads, double* out,
                     unsigned char* ties);
/* The record of every env at the current state: out [E][D], ties [E]. */
int oracle_task_observe(const oracle_world* w, double* out, unsigned char* ties);

/* Camera images of every env at the current state (the paper's batched
 * rendering, restated as a plain triangle rasteriser).  cam[10] = eye[3],
 * target[3] (world up +z), fov_y (rad), near, W, H: a pinhole looking from
 * eye to target, focal length (H/2)/tan(fov_y/2) pixels, pixel (i, j) centred
 * at (i + 0.5, j + 0.5), row 0 at the top.  Each primitive is a fixed mesh
 * (see oracle.c); back faces are skipped, triangles are clipped to view depth
 * >= near, a pixel is covered when its centre is on the inner side of (or on)
 * all three edges, and takes the covering triangle of least (view depth,
 * triangle index), depth interpolated perspective-correctly.
 * rgb_body [n_bodies][3] in [0, 1]; outputs per env and pixel: rgb [E][H][W][3]
 * = round(255 base (0.3 + 0.7 max(0, n.l))), l = normalize(0.3, 0.2, 1);
 * depth [E][H][W] (view depth, 0 = background); seg [E][H][W] (body + 1, 0 =
 * background); ties [E][H][W] = 1 where a coverage decision was within 1e-3
 * pixel of an edge or the two nearest depths within 1e-5 (relative).
 * Returns -1 for a degenerate camera. */
int oracle_render(const oracle_world* w, const double* cam, const double* rgb_body, unsigned char* rgb,
                  double* depth, int* seg, unsigned char* ties, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
