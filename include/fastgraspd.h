/*
 * fastgraspd.h -- C ABI of the GB300 grasp-search hot path (Fast-Grasp'D,
 * arXiv 2306.08132).
 *
 * The paper's problem (Sec. III): given an object and a hand (a point set
 * carried by an articulation chain), find base poses and joint angles of stable
 * grasps by gradient descent over a simulation-based stability metric, from
 * many initialisations at once.  This library runs that search for batches of
 * candidates on one GPU.  Each step of a candidate is
 *
 *   forward kinematics  p = FK(q_h)                          (Sec. III-C)
 *   voxel-SDF lookup, trilinear, dilated by r                (Sec. III-A, III-B)
 *   7 one-step PBD simulations with contact + Coulomb        (Eq. 1, Sec. IV-A)
 *   L = L_stable + w_r L_range + w_l L_limit (+ w_pen L_pen) (Eqs. 2-4)
 *   dL/dq with the leaky contact gradient                    (Sec. III-C)
 *   q <- q - lr dL/dq                                        (Sec. IV-A)
 *
 * Conventions (every entry point):
 *  - Returns fg_status; FG_OK on success.  On failure nothing was enqueued and
 *    fg_last_error() describes the cause (thread-local).  No C++ exception
 *    crosses this boundary.
 *  - Arithmetic is float32 throughout.
 *  - Plain pointers named host_* are host memory read during the call.  Every
 *    other float / int / uint32 pointer is DEVICE memory owned by the caller,
 *    valid until the enqueued work completes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Compute calls are asynchronous: they validate arguments, enqueue kernels on
 *    `stream` and return.  A CUDA launch error is reported as FG_ERR_CUDA.
 *  - Handles (fg_hand, fg_sdf, fg_scene) own device copies of their data and are
 *    immutable after creation; they may be shared by concurrent streams.  Destroy
 *    a handle only after the work that uses it has completed.
 *  - The persistent kernels take candidates from a counter that each launch
 *    draws from a pool and leaves at zero when it ends.  Eager calls cycle
 *    through 1,024 counters per kind of call, so calls may run on concurrent
 *    streams (fewer than 1,024 launches of one kind in flight at once).  A call
 *    captured in a CUDA graph keeps the counter it drew at capture; captured
 *    calls draw from a separate range of 16,384 counters that eager calls never
 *    use, so a graph may replay while any number of eager calls run.  One graph
 *    must not be replayed on two streams at once (capture one per stream), and
 *    graphs captured 16,384 or more captures of one kind apart may share a counter
 *    (do not run those at once).  Run each kind of call once before capturing it:
 *    its first launch on a device sets kernel attributes and looks up the pool.
 *  - Configuration vector layout, per candidate (row-major [B][D]):
 *      q = (t_x, t_y, t_z, w_x, w_y, w_z, theta_0 .. theta_{J-1}),  D = 6 + J,
 *    t the palm origin (metres), w the palm rotation vector (R_b = Exp(w)),
 *    theta_j the angle of the revolute joint that drives link j+1.
 *  - Test velocities (Sec. IV-A), index m = 0..6: 0, +x, -x, +y, -y, +z, -z
 *    (times fg_params.v_test).
 */
#ifndef FASTGRASPD_H
#define FASTGRASPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FG_OK = 0,
  FG_ERR_INVALID = 1,   /* bad argument or descriptor                          */
  FG_ERR_OOM = 2,       /* device or host allocation failed                    */
  FG_ERR_BUDGET = 3,    /* request does not fit the queue's HBM budget         */
  FG_ERR_TIMEOUT = 4,   /* a bounded wait ran out                              */
  FG_ERR_CUDA = 5,      /* a CUDA runtime call or kernel launch failed         */
  FG_ERR_BUSY = 6,      /* resource in use (e.g. queue full, result not ready) */
  FG_ERR_NOT_FOUND = 7  /* unknown request id                                  */
} fg_status;

#define FG_NUM_SIMS 7     /* M = 7 test velocities (Sec. IV-A)                 */
#define FG_MAX_LINKS 32   /* links per hand (root included)                    */
#define FG_MAX_POINTS (1 << 20)

typedef struct fg_hand fg_hand;
typedef struct fg_sdf fg_sdf;
typedef struct fg_scene fg_scene;
typedef struct fg_queue fg_queue;

/* Hand description (host memory, copied by fg_hand_create).
 * Links are in topological order: parent[0] = -1 (the palm, moved by the base
 * pose), 0 <= parent[l] < l for l >= 1.  Link l >= 1 carries one revolute joint,
 * joint j = l - 1, so J = n_links - 1.  T_fix[l] is the 3x4 row-major [R | t]
 * from the parent's frame to link l's frame at zero joint angle (T_fix[0] is
 * ignored); axis[l] is the unit joint axis in link l's frame.  The link frame is
 * T_l = T_parent * T_fix_l * Rot(axis_l, theta_{l-1}) (Sec. III-C, p = FK(q_h)).
 * pts_local[P][3] are surface points in their link's frame, sorted by link
 * (link_of_point nondecreasing).  q_low/q_up[J] are the joint limits of
 * L_range and L_limit (Eqs. 3-4). */
typedef struct {
  int n_links;
  int n_points;
  const int* parent;          /* [n_links]                                */
  const float* T_fix;         /* [n_links][12]                            */
  const float* axis;          /* [n_links][3]                             */
  const float* q_low;         /* [n_links - 1]                            */
  const float* q_up;          /* [n_links - 1]                            */
  const float* pts_local;     /* [n_points][3]                            */
  const int* link_of_point;   /* [n_points]                               */
} fg_hand_desc;

/* Method parameters.  alpha_leak, dt and lr are the paper's (0.1, 1e-3, 1e-3;
 * Sec. III-C, IV-A).  v_test (test-velocity magnitude, m/s), mu (Coulomb
 * coefficient), the loss weights and the dilation start r0 (metres) are not
 * fixed by the paper.  schedule: 0 = constant dilation r0, 1 = r decreases
 * linearly from r0 at step 0 to 0 at step total_steps - 1 (Sec. III-B).
 * sim_steps: the number T of simulated steps in the grasp metric (Sec. IV-A:
 * the object's velocity after T steps; the paper's experiments use T = 1).
 *   0: one step, each simulation's constraint on the plane through the single
 *      SDF query of the point (the default path of every entry point);
 *   1..FG_MAX_SIM_STEPS: T steps, every point re-queried in the SDF (grid or
 *      mesh) at each simulation's predicted object pose of every step (Sec. III-C);
 *      accepted by fg_loss_and_grad and fg_optimize_step only (FG_ERR_INVALID
 *      elsewhere). */
#define FG_MAX_SIM_STEPS 8
/* gauss_seidel (with sim_steps = 0): 0 = the corrections of all contacts are
 * taken at the predicted pose and averaged over the active contacts (Jacobi);
 * 1 = they are projected one after another in point order, each seeing the
 * object displaced by the corrections before it (Sec. III-C: "a Gauss-Seidel
 * step" over the constraints of Eq. 1), and applied in full.  Gauss-Seidel is
 * accepted by fg_contact_wrench, fg_loss_and_grad and fg_optimize_step on grid
 * and mesh objects, for hands of at most 8,192 points (FG_ERR_INVALID elsewhere). */
typedef struct {
  float alpha_leak;
  float dt;
  float v_test;
  float mu;
  float lr;
  float r0;
  float w_range;
  float w_limit;
  float w_pen;
  int schedule;
  int sim_steps;
  int gauss_seidel;
} fg_params;

/* ------------------------------------------------------------------ misc */

/* Library version.  Never fails. */
fg_status fg_version(int* major, int* minor);

/* Static description of a status code.  Never NULL. */
const char* fg_status_string(fg_status s);

/* Copies the calling thread's last error message (NUL-terminated, truncated to
 * n bytes) into buf.  FG_ERR_INVALID if buf is NULL or n == 0. */
fg_status fg_last_error(char* buf, size_t n);

/* ------------------------------------------------------------------ handles */

/* Creates a hand handle from a host description (validated: topology, counts,
 * unit axes, sorted points).  Allocates and copies to the current device
 * (synchronous).  Errors: FG_ERR_INVALID, FG_ERR_OOM, FG_ERR_CUDA. */
fg_status fg_hand_create(const fg_hand_desc* host_desc, fg_hand** out);
fg_status fg_hand_destroy(fg_hand* hand);
/* Sizes of a hand: links L, joints J = L - 1, parameters D = 6 + J, points P. */
fg_status fg_hand_info(const fg_hand* hand, int* n_links, int* n_joints, int* n_dof, int* n_points);

/* Creates an object handle: a voxel SDF grid (Sec. III-A; negative inside),
 * float32 [nz][ny][nx] with x fastest, node (i,j,k) at origin + pitch*(i,j,k);
 * `grid` may be host or device memory (copied, synchronous).  mass > 0 and the
 * isotropic moment of inertia > 0 about the object's centre of mass, which is
 * the world origin at the canonical pose.  nx, ny, nz >= 2.
 * Errors: FG_ERR_INVALID, FG_ERR_OOM, FG_ERR_CUDA. */
fg_status fg_sdf_create(const float* grid, int nx, int ny, int nz, const float* host_origin3,
                        float pitch, float mass, float inertia, fg_sdf** out);
fg_status fg_sdf_destroy(fg_sdf* sdf);

/* Creates an object handle from a watertight triangle mesh, queried directly
 * (Sec. III-B, "Signed distance function" and "Phong SDF"): phi(r) = s |r - r*|
 * with r* the closest point on the mesh (found through a bounding volume
 * hierarchy) and s = -1 inside the mesh volume (from the angle-weighted
 * pseudonormal of the closest face, edge or vertex; on a watertight mesh this
 * is the sign the paper's ray test gives); contacts use the Phong SDF
 * rho(r) = s |r - r*_rho|, r*_rho = (1 - a) r* + a sum_x b_x psi_x(r*), where b are the
 * barycentric coordinates of r* on its face, psi_x(q) = q - ((q - v_x) . n_x) n_x
 * projects onto the tangent plane at vertex x (angle-weighted vertex normal n_x)
 * and a = phong_alpha in [0, 1] (0: the flat mesh), with the paper's gradient
 * grad rho = s (r - r*_rho)/|r - r*_rho|.
 *   vertices  host [n_vertices][3] float32, in the object frame (centre of mass at
 *             the origin at the canonical pose);
 *   faces     host [n_faces][3] vertex indices, counter-clockwise about the
 *             outward normal; every edge shared by exactly two faces (watertight,
 *             consistently oriented), no zero-area face.
 * The handle is an fg_sdf: fg_sdf_query, scenes, fg_contact_wrench, fg_loss_and_grad,
 * fg_optimize_step (both projection orders and the T-step metric) and the request
 * queue take it; the per-stage form takes grid objects only (FG_ERR_INVALID).
 * Built on the host, copied to the current device (synchronous): validation,
 * normals and pseudonormals, the BVH, and for the certified local search that
 * answers most queries before the BVH walk, the faces on the convex hull, the
 * vertex rings in fan order and a table of start faces (the closest face at the
 * nodes of a 32-node grid over the mesh's box grown by its largest side).  Device
 * memory: about 280 bytes per face plus up to 128 KB.
 * Errors: FG_ERR_INVALID (with the reason), FG_ERR_OOM, FG_ERR_CUDA. */
fg_status fg_sdf_create_mesh(const float* host_vertices, int n_vertices, const int* host_faces, int n_faces,
                             float phong_alpha, float mass, float inertia, fg_sdf** out);

/* Host only, no GPU needed: runs fg_sdf_create_mesh's validation and host build on
 * the same arguments and reports how much of the mesh the certified local search
 * can answer.  out6 (host, 6 ints): faces, faces on the convex hull (no vertex
 * more than 1e-9 of the mesh's extent outside the face's plane), vertices whose
 * faces form one fan, BVH nodes, BVH depth, nodes of the start-face table.  A query
 * whose closest feature has a face off the hull, or a vertex not in one fan, takes
 * the BVH walk.
 * Errors: FG_ERR_INVALID (with the reason, as fg_sdf_create_mesh). */
fg_status fg_mesh_describe(const float* host_vertices, int n_vertices, const int* host_faces, int n_faces,
                           int* host_out6);

/* A scene is an ordered table of objects; candidates select theirs by index
 * (obj_of_cand).  The scene keeps pointers to the objects' grids: destroy the
 * scene before its objects.  Errors: FG_ERR_INVALID, FG_ERR_OOM, FG_ERR_CUDA. */
fg_status fg_scene_create(const fg_sdf* const* host_sdfs, int n_objects, fg_scene** out);
fg_status fg_scene_destroy(fg_scene* scene);

/* ------------------------------------------------------------------ hot path */

/* Forward kinematics (Sec. III-C): world positions of every hand point for B
 * candidates.  q: [B][D].  pts: SoA [3][B*P] (x block, y block, z block; the
 * point of candidate b, index i sits at b*P + i).  B >= 0 (0 is a no-op). */
fg_status fg_fk(const fg_hand* hand, const float* q, int B, float* pts, void* stream);

/* Dilated SDF lookup (Sec. III-A, III-B): for n points (SoA [3][n]),
 * phi[n] = trilinear(grid) + outside-excess - r_dil and grad[3][n] (SoA,
 * nullable) = gradient of the undilated interpolant.  Points outside the grid
 * are clamped to it and the Euclidean excess distance is added. */
fg_status fg_sdf_query(const fg_sdf* sdf, const float* pts, int n, float r_dil, float* phi,
                       float* grad, void* stream);

/* Contact forces and object wrench of the 7 one-step simulations (Eq. 1,
 * Sec. III-C, IV-A) at dilation r_dil.  obj_of_cand: device [B] indices into
 * the scene (NULL: object 0 for all).  Outputs per candidate b and simulation m:
 * wrench[B][7][6] = sum over contacts of (f, d x f), the summed position
 * corrections times mass (before averaging); ncontact[B][7] = number of points
 * with phi_m < 0; contact_bits (nullable) [B][7][ceil(P/32)], bit (i % 32) of
 * word i / 32 set when point i is in contact.  With params.gauss_seidel = 1: the
 * sums of the corrections the sweep applied (m dx, I dth), the points it
 * projected and their bits. */
fg_status fg_contact_wrench(const fg_hand* hand, const fg_scene* scene, const int* obj_of_cand,
                            const float* q, int B, const fg_params* host_params, float r_dil,
                            float* wrench, int* ncontact, uint32_t* contact_bits, void* stream);

/* Loss and gradient (Eqs. 2-4, Sec. III-C leaky rule) at dilation r_dil,
 * forward and adjoint fused in one kernel (the adjoint recomputes the forward
 * per point; nothing per point is stored).  loss: [B]; grad: [B][D] nullable
 * (NULL: the loss alone, without the adjoint sweep).  params.sim_steps >= 1
 * selects the T-step form and params.gauss_seidel = 1 the Gauss-Seidel form
 * (each its own kernel, same arguments); grid and mesh objects. */
fg_status fg_loss_and_grad(const fg_hand* hand, const fg_scene* scene, const int* obj_of_cand,
                           const float* q, int B, const fg_params* host_params, float r_dil,
                           float* loss, float* grad, void* stream);

/* nsteps >= 1 gradient-descent steps (Sec. IV-A) in one persistent fused
 * forward + adjoint + update kernel.  q: [B][D] in/out.  The dilation of global
 * step k = step + s is r0 (schedule 0) or r0 * max(0, 1 - k / (total_steps - 1))
 * (schedule 1).  loss (nullable, [B]): loss at the last step, evaluated before
 * its update.  The T-step and Gauss-Seidel forms as for fg_loss_and_grad. */
fg_status fg_optimize_step(const fg_hand* hand, const fg_scene* scene, const int* obj_of_cand,
                           float* q, int B, const fg_params* host_params, int step, int total_steps,
                           int nsteps, float* loss, void* stream);

/* fg_optimize_step from and to host memory (Sec. IV-A, as fg_optimize_step): on
 * `stream`, copies host_q_in [B][D] to the device buffer q [B][D] (caller-owned
 * scratch, overwritten), runs the nsteps, then copies q to host_q_out [B][D] and,
 * when host_loss is non-NULL, the device loss [B] (then required) to host_loss.
 * Asynchronous like every compute call: the host buffers must stay valid, and be
 * read only after the stream reaches this point; pinned host memory makes the
 * copies asynchronous, pageable memory makes them synchronous.  host_q_in and
 * host_q_out may be the same buffer.  Errors as fg_optimize_step, plus
 * FG_ERR_INVALID for a NULL buffer. */
fg_status fg_optimize_step_host(const fg_hand* hand, const fg_scene* scene, const int* obj_of_cand,
                                const float* host_q_in, float* q, int B, const fg_params* host_params, int step,
                                int total_steps, int nsteps, float* loss, float* host_q_out, float* host_loss,
                                void* stream);

/* The same step as fg_optimize_step, run as the plain one-kernel-per-stage
 * form: FK links -> point transform -> SDF query -> contact forward -> loss ->
 * contact adjoint -> link reduction -> FK adjoint + update, with the per-point
 * intermediates in `workspace` (device memory, >= fg_plain_workspace_size
 * bytes, 256-byte aligned).  Comparison baseline for the fused kernel: the
 * one-step Jacobi form on grid objects (FG_ERR_INVALID for the other forms and
 * for mesh objects). */
fg_status fg_plain_workspace_size(const fg_hand* hand, int B, size_t* bytes);
fg_status fg_optimize_step_plain(const fg_hand* hand, const fg_scene* scene, const int* obj_of_cand,
                                 float* q, int B, const fg_params* host_params, int step,
                                 int total_steps, int nsteps, float* loss, void* workspace,
                                 size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------ request queue */

/* A request queue runs many grasp searches at once with continuous batching
 * (the paper's problem of Sec. III for a stream of objects, hands and candidate
 * counts).  It owns a scheduler thread and a CUDA stream on the device current
 * at creation.  A submitted request waits until a slot is free and its device
 * footprint fits the HBM budget: q and loss (B (D + 1) 4 bytes) plus the
 * object's grid and min-pyramid, counted once per object while any admitted
 * request uses it.  Each round launches one fused kernel over the candidates of
 * all admitted requests, up to steps_per_launch optimisation steps each;
 * finished requests are copied to host memory and free their slot and bytes,
 * and waiting requests join at the next round.  A request's result is the same
 * alone and in any mix (candidates are independent).  The hand and object
 * handles of a request must stay alive until its result is collected. */

#define FG_QUEUE_MAX_SLOTS 64

typedef struct {
  int max_slots;          /* requests on the GPU at once, <= FG_QUEUE_MAX_SLOTS (0: 32)       */
  int max_requests;       /* submitted and not yet collected (0: 4096)                         */
  int steps_per_launch;   /* optimisation steps per request per round (0: 10)                  */
  int timeout_ms;         /* bound on the wait for one round (0: 60000); past it the round's
                             requests fail with FG_ERR_TIMEOUT and the queue takes no more work */
} fg_queue_opts;

typedef struct {
  const fg_hand* hand;
  const fg_sdf* sdf;
  int B;                  /* candidates, >= 1                                   */
  int steps;              /* gradient-descent steps, >= 1 (schedule over steps) */
  const float* host_q0;   /* [B][D] initial candidates, copied at submit        */
  fg_params params;
} fg_request;

typedef struct {
  int pending, active, finished, failed;
  size_t bytes_in_use, budget;
  uint64_t rounds, candidate_steps;
} fg_queue_stat;

/* Errors: FG_ERR_INVALID, FG_ERR_OOM, FG_ERR_CUDA. */
fg_status fg_queue_create(size_t hbm_budget_bytes, const fg_queue_opts* opts, fg_queue** out);
/* Non-blocking.  FG_ERR_BUDGET if the request alone exceeds the budget (it could
 * never be admitted); FG_ERR_BUSY if max_requests are outstanding; FG_ERR_INVALID
 * for a malformed request; FG_ERR_OOM if its host copy cannot be allocated (a
 * request whose device state cannot be allocated at admission fails with
 * FG_ERR_OOM, reported by fg_queue_result); FG_ERR_CUDA once the queue has failed
 * (a round exceeded timeout_ms or a CUDA call failed) or is being destroyed. */
fg_status fg_queue_submit(fg_queue* queue, const fg_request* host_req, uint64_t* id);
/* Non-blocking: *done = 1 once the request finished (or failed). */
fg_status fg_queue_poll(fg_queue* queue, uint64_t id, int* done);
/* Blocks up to timeout_ms; FG_ERR_TIMEOUT if the request has not finished. */
fg_status fg_queue_wait(fg_queue* queue, uint64_t id, int timeout_ms);
/* Copies the final q [B][D] and the loss of the last step [B] (either nullable)
 * and the latency from submit to completion, then forgets the request.
 * FG_ERR_BUSY if not finished; the request's error if it failed. */
fg_status fg_queue_result(fg_queue* queue, uint64_t id, float* host_q, float* host_loss, double* latency_s);
fg_status fg_queue_stats(fg_queue* queue, fg_queue_stat* out);
/* Waiting requests are dropped, the round in flight completes, then the
 * queue's resources are freed.  After a round that exceeded timeout_ms the
 * kernel may still be running: destroy waits for the queue's stream at most
 * timeout_ms more and, if it has not drained, returns FG_ERR_TIMEOUT and leaves
 * the handle valid (call fg_queue_destroy again later; nothing else may be
 * called on it).  It never blocks without a bound. */
fg_status fg_queue_destroy(fg_queue* queue);

/* ------------------------------------------------------------ no allocation */

/* Bytes of the scratch array built into the library for
 * fg_optimize_step_plain_noalloc (held on every GPU that loads the library). */
#define FG_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory while running (a real-time planning loop that
 * must not block or fail on an allocation mid-cycle, or a host whose device
 * memory belongs to another runtime's allocator).  It runs the same step as
 * fg_optimize_step_plain with the per-stage scratch in a fixed array of
 * FG_NOALLOC_SCRATCH_BYTES inside the library, and calls no allocator.
 * Arguments as fg_optimize_step_plain, without the workspace.
 *  - FG_ERR_INVALID (with a message) when the step needs more scratch than the
 *    array holds (fg_plain_workspace_size(hand, B) > FG_NOALLOC_SCRATCH_BYTES;
 *    about 490,000 candidate points).
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any stream
 *    capture.
 *  - All calls share the one array and its contents persist between calls
 *    (each call writes all the scratch it reads).  Calls whose work overlaps on
 *    the GPU, e.g. on two unordered streams, race on it: order them. */
fg_status fg_optimize_step_plain_noalloc(const fg_hand* hand, const fg_scene* scene, const int* obj_of_cand,
                                         float* q, int B, const fg_params* host_params, int step,
                                         int total_steps, int nsteps, float* loss, void* stream);

/* ------------------------------------------------------------ grasp quality */

/* Grasp-quality metrics of the evaluation (Sec. V, "Metrics": contact area,
 * intersection volume and epsilon depend on the distance threshold tau used to
 * generate contacts; 5 mm for the paper's Table II).  A contact is a hand point
 * p with phi(p) < tau, phi the undilated SDF of the candidate's object at its
 * canonical pose (grid or mesh).  Both calls are asynchronous on `stream` and
 * write NaN (and -1 contacts) for a candidate whose obj_of_cand index is outside
 * the scene. */

/* Weighted contact measure: out[b] = sum of weights[i] over the hand points i
 * with phi(p_i(q_b)) < tau.  With the surface samples, the area each stands for
 * and tau the contact threshold this is the contact area CA; with a hand whose
 * points sample the links' interiors, their volumes and tau = 0 it is the
 * intersection volume IV.  weights: device [P] in the hand's point order;
 * out: device [B].  Errors: FG_ERR_INVALID (NULL buffer, B < 0, non-finite tau). */
fg_status fg_contact_measure(const fg_hand* hand, const fg_scene* scene, const int* obj_of_cand,
                             const float* q, int B, const float* weights, float tau, float* out,
                             void* stream);

/* Epsilon quality over a set of wrench-space directions.  Each contact, with
 * outward normal n = grad phi / |grad phi|, contributes the cone_edges edges of
 * its Coulomb cone f_e = -n + mu (cos(2 pi e / k) t1 + sin(2 pi e / k) t2),
 * (t1, t2) the tangent basis of n by Duff et al. (2017), as the wrenches
 * w = (f_e, torque_scale * (p - c) x f_e), c the object's origin (its centre of
 * mass).  eps[b] = min over the K unit directions u of max over all wrenches of
 * u . w: an upper bound of the Ferrari-Canny epsilon (the distance from the
 * origin to the boundary of the wrenches' convex hull), equal to it when the
 * set holds the normal of the hull facet nearest the origin; -infinity without
 * contacts.  n_contacts (nullable): device [B] contacts found.  dirs: device
 * [K][6], 1 <= K <= FG_MAX_DIRS; 1 <= cone_edges <= 32; mu >= 0;
 * torque_scale >= 0 (1 / the object's radius).  Errors: FG_ERR_INVALID. */
#define FG_MAX_DIRS 8192
fg_status fg_grasp_epsilon(const fg_hand* hand, const fg_scene* scene, const int* obj_of_cand,
                           const float* q, int B, float tau, float mu, int cone_edges, float torque_scale,
                           const float* dirs, int K, float* eps, int* n_contacts, void* stream);

/* ------------------------------------------------------------------ tuning */

/* The fused kernels are compiled in several configurations: warps per
 * candidate (points per warp = P / warps), the minimum number of resident CTAs
 * per SM the register allocation is held to, and the points each thread carries
 * per iteration of the adjoint sweep (independent dependency chains).  The selection is
 * per device (the current one) and applies to fg_loss_and_grad and
 * fg_optimize_step; it changes no result beyond float32 summation order. */
fg_status fg_fused_config_count(int* n);
fg_status fg_fused_config_info(int index, int* warps_per_candidate, int* min_ctas_per_sm,
                               int* points_per_thread);
/* index in [0, count) selects a configuration; -1 restores the default. */
fg_status fg_fused_config_select(int index);
fg_status fg_fused_config_current(int* index);

/* Autotuner: times every configuration of fg_optimize_step on this workload
 * (q is copied to a scratch buffer, not modified), reps timed launches each
 * after one warm-up, selects the fastest for the current device and returns its
 * index in *best (nullable) and the mean times in host_times_ms[count]
 * (nullable).  Synchronises `stream`; allocates its scratch with
 * cudaMallocAsync on `stream`.  Errors: FG_ERR_INVALID, FG_ERR_CUDA, FG_ERR_OOM. */
fg_status fg_autotune(const fg_hand* hand, const fg_scene* scene, const int* obj_of_cand, const float* q, int B,
                      const fg_params* host_params, int step, int total_steps, int nsteps, int reps,
                      float* host_times_ms, int* best, void* stream);

/* ---------------------------------------------------------------------- testing
 * The paper has no counterpart: a hook that lets tests exercise the library's
 * out-of-memory paths without exhausting the device.
 *
 * fg_test_fail_allocation(after): after `after` more allocation points pass,
 * the next one fails as if the allocation had returned out-of-memory, once;
 * -1 disarms.  Allocation points: the device buffers of fg_hand_create, the grid
 * of fg_sdf_create, the host copy of a request in fg_queue_submit and a request's
 * device state at admission.  Process-wide; not for use while other threads
 * create handles or submit requests.  Errors: FG_ERR_INVALID (after < -1). */
fg_status fg_test_fail_allocation(int after);

/* ------------------------------------------------------------------ measurement
 * The paper has no counterpart: this is the measured denominator of the ALU
 * roofline that the library's kernels are reported against.
 *
 * fg_fp32_peak_launch enqueues one kernel of `blocks` CTAs of 256 threads, each
 * thread running 8 independent chains of `iters` fused multiply-adds, as scalar
 * FFMA (packed = 0: 2 flops each) or packed f32x2 FMA (packed != 0: 4 flops
 * each), and stores one float per thread in out (device, blocks * 256 floats,
 * caller-owned; the values are of no use).  *host_flops (nullable) receives the
 * floating-point operations of the launch; the caller times it on `stream` (CUDA
 * events) and divides.  Size it to several hundred milliseconds and a multiple
 * of the SM count for a steady figure.  Errors: FG_ERR_INVALID (blocks < 1,
 * iters < 1, out NULL), FG_ERR_CUDA. */
fg_status fg_fp32_peak_launch(int packed, int blocks, int iters, float* out, double* host_flops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FASTGRASPD_H */
