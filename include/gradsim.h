/*
 * gradsim.h -- C ABI of the GB300 library for the differentiable explicit
 * multiphysics step of gradSim (Murthy et al., ICLR 2021) and its discrete
 * adjoint through whole rollouts.
 *
 * The method (paper sections in brackets):
 *   state s = [q, u] (node positions and velocities), lumped mass M  [Sec. 2.1]
 *   per-element forces from the stable neo-Hookean energy
 *     Psi = mu/2 (I_C - 3) + lambda/2 (J - alpha)^2 - mu/2 log(I_C + 1)
 *     on linear tetrahedra, and on triangles in the plane for cloth, plus
 *     dihedral bending f_b = k_b sin(phi/2 + alpha) d          [App. A.1, C.1]
 *   penalty contact f_n = n (k_e C + k_d dC/dt) with relaxed Coulomb
 *     friction against a ground plane and a sphere             [App. A.1, C.2]
 *   semi-implicit Euler u+ = u- + dt M^-1 f(s-), q+ = q- + dt u+  [App. B]
 *   reverse mode through the whole rollout by the discrete adjoint of
 *     that step, whose triangular Jacobians make every adjoint explicit [App. B]
 *   a loss on final node positions stands in for the paper's image loss.
 *
 * Conventions
 *   - Every call returns gs_status: 0 = GS_OK, < 0 error, > 0 warning.  On an
 *     error nothing was enqueued and gs_last_error() (thread-local) says why.
 *     No C++ exception crosses this boundary: a failed host allocation
 *     returns GS_ENOMEM, any other host-side exception GS_EINTERNAL.
 *   - Streams are passed as `void*` holding a cudaStream_t (0 = legacy
 *     default stream).  Work is enqueued asynchronously on that stream; device
 *     buffers handed in must stay valid until the stream reaches the work.
 *   - Node arrays are [n_nodes][3] row-major float in the caller's node order;
 *     element arrays are in the caller's element order.  The library keeps
 *     its own (Morton-ordered) internal layout and translates at the boundary.
 *   - `mem_space` says where a caller buffer lives: GS_MEM_DEVICE (device
 *     pointer on the context's GPU) or GS_MEM_HOST (host pointer; the call
 *     copies it, synchronising the stream for device->host results).
 *   - FP32 state and element math; FP64 for the loss and for the gradient
 *     sums over elements and time steps.  Results are deterministic: node
 *     forces are gathered in a fixed order (no floating-point atomics), and
 *     the per-element FP64 gradient sums over time take one term per element
 *     per launch, in launch order, so the same inputs give bitwise the same
 *     outputs, alone or in a batch.
 *   - One gs_ctx per GPU; a context and everything made from it must be used
 *     from one host thread at a time (the server runs its own thread).
 */
#ifndef GRADSIM_H
#define GRADSIM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define GS_VERSION 10000 /* 1.0.0 */

typedef int gs_status;
enum {
    GS_OK = 0,
    GS_EINVAL = -1,      /* bad argument, malformed mesh, non-finite input    */
    GS_ENOMEM = -2,      /* allocation failed or over the context budget      */
    GS_ECUDA = -3,       /* a CUDA runtime call failed (message has the text) */
    GS_ESTATE = -4,      /* call out of order (e.g. adjoint before rollout)   */
    GS_ENONFINITE = -5,  /* the simulation produced a NaN/Inf                 */
    GS_ETIMEOUT = -6,    /* poll timed out                                    */
    GS_ECANCELLED = -7,  /* query cancelled                                   */
    GS_ENOTFOUND = -8,   /* unknown ticket                                    */
    GS_EUNSUPPORTED = -9,
    GS_EINDEX = -10,     /* checked build: a table index was out of range     */
    GS_EINTERNAL = -11,  /* unexpected host-side failure (message has the text) */
    GS_PENDING = 1,      /* query not finished yet                            */
    GS_WUNSTABLE = 2     /* dt above the explicit stability estimate (ran)    */
};

enum { GS_TET = 0, GS_CLOTH = 1 };
enum { GS_MEM_DEVICE = 0, GS_MEM_HOST = 1 };

typedef struct gs_ctx gs_ctx;
typedef struct gs_mesh gs_mesh;
typedef struct gs_batch gs_batch;
typedef struct gs_server gs_server;

/* Device-memory provider.  alloc returns NULL on failure, else memory
 * aligned to 256 bytes (as cudaMalloc's; an unaligned block is handed back
 * to free and the call fails with GS_EINVAL); free receives the pointer and
 * size given by alloc.  Both are called on the thread making the library
 * call, with the stream the memory will first be used on. */
typedef struct gs_allocator {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void (*free)(void* ptr, size_t bytes, void* stream, void* user);
    void* user;
} gs_allocator;

/* Compliant contact, App. A.1 "Contact" and App. C.2: penetration depth C
 * along the outward normal n, f_n = n (k_e C + k_d dC/dt) with dC/dt = -v.n
 * while C > 0; relaxed Coulomb friction on v_s = v - (v.n) n:
 * f_f = -k_f v_s while k_f |v_s| <= mu_f |f_n|, else -mu_f |f_n| v_s/|v_s|.
 * Plane: {y : plane_n . y = plane_h}, plane_n unit length.  Sphere: centre,
 * radius.  Both may be active. */
typedef struct gs_contact {
    float ke, kd, kf, mu_f;
    int plane_on;
    float plane_n[3];
    float plane_h;
    int sphere_on;
    float sphere_c[3];
    float sphere_r;
} gs_contact;

/* Mesh description; every pointer is a HOST pointer and is copied.
 *   GS_TET:   elems [n_elems][4] node ids of positively oriented tets
 *             (det[X1-X0, X2-X0, X3-X0] > 0); density in kg/m^3.
 *   GS_CLOTH: elems [n_elems][3] triangles; hinges [n_hinges][4] =
 *             (x1, x2 wing tips; x3 -> x4 shared edge) with triangles
 *             (x1, x3, x4) and (x2, x4, x3) consistently oriented; density
 *             is areal (kg/m^2); kb is the per-hinge bending stiffness.
 *   X: rest positions (double, also the initial positions); v0 nullable (0).
 *   mu, lambda: Lame parameters per element (App. C.1, heterogeneous).
 *   act, hinge_act: per-element / per-hinge actuation, nullable (0).
 *   pinned: nullable; 1 marks a kinematic node (inverse mass 0, no gravity).
 *   patch_elems, block_threads: work decomposition (0 = defaults, or the
 *   tuned values); block_threads_adj: consumer threads of the adjoint patch
 *   kernels (0 = block_threads).  They change performance only, never
 *   results of a given decomposition (results may differ in the last bits
 *   between different patch sizes because the FP32 force sums are grouped
 *   differently; the thread counts do not change any sum). */
typedef struct gs_mesh_desc {
    int kind;
    int n_nodes;
    int n_elems;
    const int32_t* elems;
    int n_hinges;
    const int32_t* hinges;
    const double* X;
    const double* v0;
    const double* mu;
    const double* lambda;
    const double* density;
    const double* kb;
    const double* act;
    const double* hinge_act;
    const uint8_t* pinned;
    gs_contact contact;
    float gravity[3];
    int patch_elems;
    int block_threads;
    int block_threads_adj;
} gs_mesh_desc;

typedef struct gs_mesh_info {
    int kind, n_nodes, n_elems, n_hinges;
    int n_patches;          /* element patches (one CTA each)                 */
    int n_boundary_nodes;   /* nodes shared between patches                   */
    int patch_elems, block_threads;
    int block_threads_adj;  /* consumer threads of the adjoint patch kernels  */
    double dt_stable;       /* explicit stability estimate (seconds)          */
    size_t device_bytes;    /* bytes the mesh holds on the device             */
} gs_mesh_info;

/* Gradients of the loss; caller-owned DEVICE pointers in caller order, each
 * nullable (not computed).  Parameter gradients are FP64 sums over all time
 * steps.  For GS_TET, d_mu/d_lambda/d_density/d_act are per tet; for
 * GS_CLOTH they are per triangle and d_kb/d_hinge_act per hinge.  d_mass is
 * dL/dm_i per node (the chain to density goes through the lumped mass). */
typedef struct gs_grads {
    double* d_mu;
    double* d_lambda;
    double* d_density;
    double* d_act;
    double* d_kb;
    double* d_hinge_act;
    double* d_mass;
    float* d_x0;
    float* d_v0;
    /* [S][n_elems] / [S][n_hinges], caller order, FP32: dL/d(the actuation
     * an element / hinge has during step n) of the time-varying actuation
     * (gs_mesh_set_act_seq), for every step of the rollout (S = its length) */
    float* d_act_seq;
    float* d_hinge_act_seq;
} gs_grads;

/* ---- library ------------------------------------------------------------ */
GS_API int gs_version(void);
/* Build options of the loaded library (no paper counterpart): the bit
 * GS_BUILD_CHECKED is set in the checked build (libgradsim_check.so), whose
 * step kernels test every mesh-table index on the device before using it;
 * an out-of-range index sets the mesh's status and gs_mesh_check then
 * returns GS_EINDEX (no trap: the kernel skips the access). */
#define GS_BUILD_CHECKED 1
GS_API int gs_build_flags(void);
/* Message of the last failed call on this thread ("" if none). */
GS_API const char* gs_last_error(void);

/* ---- context ------------------------------------------------------------ */
/* One context per GPU.  hbm_budget_bytes caps what the library allocates
 * through this context (0 = no cap); alloc nullable = cudaMallocAsync. */
GS_API gs_status gs_create(gs_ctx** out, int device, size_t hbm_budget_bytes, const gs_allocator* alloc);
GS_API void gs_destroy(gs_ctx* ctx);
/* Bytes currently allocated through the context. */
GS_API size_t gs_ctx_bytes(const gs_ctx* ctx);
/* 1: capture rollout chunks in CUDA graphs (default); 0: one launch per
 * kernel per step (the plain loop).  Results are identical. */
GS_API gs_status gs_set_graphs(gs_ctx* ctx, int enable);

/* Per-launch timing of the step kernels with CUDA events on the launching
 * stream (measurement support; the paper has no counterpart).  While on,
 * every patch and boundary kernel has an event pair around it: with CUDA
 * graphs on (gs_set_graphs), each run of steps is captured as a graph of
 * its own with the events as external event nodes (which ends the
 * programmatic overlap of neighbouring kernels); with graphs off, steps run
 * as one launch per kernel.  gs_profile_read synchronises the pending
 * events and returns, per kernel, the launch count and summed milliseconds,
 * then clears them; n_out receives the number of kernels with launches. */
typedef struct gs_kernel_time {
    char name[32];
    uint64_t launches;
    double total_ms;
} gs_kernel_time;
GS_API gs_status gs_profile(gs_ctx* ctx, int enable);
GS_API gs_status gs_profile_read(gs_ctx* ctx, gs_kernel_time* out, int max, int* n_out);

/* ---- mesh (Sec. 2.1 state, App. C.1 elements, a1 set-up) ------------------ */
/* Validates indices (range, repeated corners), rest elements (inverted or
 * degenerate: GS_EINVAL), finiteness and positivity of parameters; builds the
 * internal layout; computes Dm^-1, rest volume/area and lumped masses on the
 * GPU.  Synchronous (returns when the mesh is ready). */
GS_API gs_status gs_mesh_create(gs_ctx* ctx, const gs_mesh_desc* desc, gs_mesh** out);
GS_API void gs_mesh_destroy(gs_mesh* mesh);
GS_API gs_status gs_mesh_info_get(const gs_mesh* mesh, gs_mesh_info* out);
/* Replace per-element parameters (nullable = unchanged), caller order, float.
 * A new density re-runs the lumped-mass set-up.  Enqueued on `stream`. */
GS_API gs_status gs_mesh_set_params(gs_mesh* mesh, const float* mu, const float* lambda,
                             const float* density, const float* act, const float* kb,
                             int mem_space, void* stream);
/* Time-varying actuation, the control input of the paper's visuomotor
 * control experiments (Sec. 3; the controller of App. D drives per-element
 * activations): during step n < n_steps, row n of act_seq [n_steps][n_elems]
 * (caller order) is added to each element's actuation a_e in the energy
 * (alpha = 1 + 3 mu/(4 lambda) + a_e, App. A) and row n of hinge_act_seq
 * [n_steps][n_hinges] to each hinge's rest-angle actuation; later steps add
 * nothing.  Rollouts count steps from 0; gs_step applies rows 0..n-1 on each
 * call.  Both arrays nullable; n_steps = 0 (or both NULL) clears.  Copied
 * (DEVICE or HOST per mem_space).  GS_EINVAL for n_steps < 0 or (HOST)
 * non-finite values.  The adjoint's per-step gradients come out in
 * gs_grads.d_act_seq / d_hinge_act_seq. */
GS_API gs_status gs_mesh_set_act_seq(gs_mesh* mesh, const float* act_seq, const float* hinge_act_seq, int n_steps,
                                     int mem_space, void* stream);
/* Air on the cloth surface (App. A.1 "Deformable Thin-Shells" adds lift and
 * drag from the surrounding air but prints no formula).  Flat-plate
 * reading, per triangle with deformed vector area N (|N| = A), mean corner
 * velocity minus the wind v_r, s = N . v_r:
 *   drag F_D = -k_drag |s| v_r,
 *   lift F_L = -k_lift s/(A |v_r|) (|v_r|^2 N - s v_r)  (perpendicular to v_r),
 * a third of F_D + F_L on each corner; coefficients in kg/m^3 (1/2 rho_air C
 * of a flat plate), wind in m/s.  Both enter the forward step and the
 * adjoint (dL/dx, dL/dv through the air).  GS_CLOTH meshes only (GS_EINVAL
 * otherwise); coefficients finite and >= 0, wind finite (GS_EINVAL).  NULL
 * turns the air off.  Takes effect at the next launch. */
typedef struct gs_air {
    float k_drag, k_lift;
    float wind[3];
} gs_air;
GS_API gs_status gs_mesh_set_air(gs_mesh* mesh, const gs_air* air, void* stream);
/* ---- rigid bodies (App. A.1 "Rigid Bodies") ---------------------------
 * State of a body, 13 floats: x (centre of mass), r = (w, x, y, z) unit
 * quaternion (world from body), v, omega (world frame).  Newton-Euler with
 * the compliant contact model (the particles' law, gs_contact) acting at
 * the body's contact points, and semi-implicit Euler (App. B):
 *   v+ = v + dt (g + F/m),  omega+ = omega + dt R I_b^-1 R^T (tau - omega x R I_b R^T omega),
 *   x+ = x + dt v+,  r+ = normalise(r + dt/2 (0, omega+) (x) r).
 * Design parameters per body: mass, body-frame inertia about the centre of
 * mass (Ixx, Iyy, Izz, Ixy, Ixz, Iyz), contact (ke, kd, kf, mu).  Bodies do
 * not interact; one launch runs a whole rollout of every body. */
typedef struct gs_rigid_desc {
    int n_bodies;
    const int* point_begin; /* HOST [n_bodies + 1]: body b's points are [point_begin[b], point_begin[b+1]) */
    const float* points;    /* HOST [n_points][3] body frame, about the centre of mass */
    const float* mass;      /* HOST [n_bodies], > 0 */
    const float* inertia;   /* HOST [n_bodies][6], positive definite */
    const float* contact;   /* HOST [n_bodies][4] ke, kd, kf, mu (>= 0) */
    gs_contact scene;       /* plane / sphere of the scene (its ke, kd, kf, mu_f unused) */
    float gravity[3];
} gs_rigid_desc;
typedef struct gs_rigid gs_rigid;
/* Caller-owned DEVICE outputs, each nullable. */
typedef struct gs_rigid_grads {
    float* d_state0;   /* [n_bodies][13] */
    double* d_mass;    /* [n_bodies] */
    double* d_inertia; /* [n_bodies][6] */
    double* d_contact; /* [n_bodies][4] */
} gs_rigid_grads;
/* Copies everything.  GS_EINVAL for bad offsets, non-finite points,
 * non-positive mass, an inertia that is not positive definite, negative
 * contact parameters or a non-unit plane normal. */
GS_API gs_status gs_rigid_create(gs_ctx* ctx, const gs_rigid_desc* desc, gs_rigid** out);
GS_API void gs_rigid_destroy(gs_rigid* r);
/* New per-body parameters (HOST arrays as in the description; nullable = unchanged). Synchronous. */
GS_API gs_status gs_rigid_set_params(gs_rigid* r, const float* mass, const float* inertia, const float* contact,
                                     void* stream);
/* S steps from DEVICE state0 [n_bodies][13]; stores every state for the
 * adjoint; the final state into DEVICE stateS (nullable).  A non-finite
 * state sets the sticky flag gs_rigid_check reports. */
GS_API gs_status gs_rigid_rollout(gs_rigid* r, float dt, int S, const float* state0, float* stateS, void* stream);
/* Reverse of the last rollout (GS_ESTATE without one) for the seed
 * dL/dstate(S) (DEVICE [n_bodies][13], nullable = 0).  Parameter
 * gradients are FP64 sums over the steps. */
GS_API gs_status gs_rigid_adjoint(gs_rigid* r, const float* dL_dstateS, gs_rigid_grads* grads, void* stream);
/* World positions x + R p of every point at DEVICE state [n_bodies][13] into DEVICE points [n_points][3]. */
GS_API gs_status gs_rigid_points(gs_rigid* r, const float* state, float* points, void* stream);
/* dL/dstate [n_bodies][13] (DEVICE, written; velocity entries 0) from dL/dpoints [n_points][3]. */
GS_API gs_status gs_rigid_points_backward(gs_rigid* r, const float* state, const float* dL_dpoints, float* dL_dstate,
                                          void* stream);
/* GS_OK, or GS_ENONFINITE if a rollout produced a non-finite state (reset clears). */
GS_API gs_status gs_rigid_check(gs_rigid* r, int reset, void* stream);

/* ---- differentiable soft rasteriser ------------------------------------
 * The rendering stage of Sec. 2 ("Differentiable rendering engine"): the
 * simulated surface becomes an image through SoftRas-style sigmoid edges and
 * DIB-R-style barycentric interpolation, so that a loss on pixels reaches the
 * vertex positions.  The paper prints no formulas; reading, per pixel p with
 * centre (i + 0.5, j + 0.5) and triangle t with projected corners a, b, c:
 *   projection: x_cam = R x + t, u = fx x_cam/z_cam + cx, v = fy y_cam/z_cam + cy,
 *     depth z_cam; a triangle with a corner at z_cam <= z_near or zero
 *     projected area is skipped;
 *   coverage D = sigmoid(+-d^2/sigma) with d the distance from p to the
 *     triangle's boundary (+ inside); 1 - D is kept >= 1e-6; outside pixels
 *     with D < 1e-5 are not covered;
 *   silhouette A = 1 - prod_t (1 - D_t);
 *   colour: clamped barycentrics interpolate the vertex colours and,
 *     perspective-correct, 1/z; zh = (z_far - z)/(z_far - z_near);
 *     I = (sum_t D_t e^{zh_t/gamma} C_t + e^{eps/gamma} bg) / (sum_t D_t e^{zh_t/gamma} + e^{eps/gamma}).
 * Output image [height][width][4] = (I, A), FP32, row-major. */
typedef struct gs_camera {
    float R[9];          /* world -> camera rotation, row-major */
    float t[3];
    float fx, fy, cx, cy; /* pixels */
    int width, height;   /* 1..16384 */
    float z_near, z_far; /* 0 < z_near < z_far */
} gs_camera;
typedef struct gs_raster_desc {
    int n_vertices;
    int n_faces;
    const int* faces;    /* HOST [n_faces][3] vertex indices (copied) */
    gs_camera camera;
    float sigma;         /* edge softness, pixel^2 (> 0) */
    float gamma;         /* depth softmax temperature (> 0) */
    float eps;           /* normalised depth of the background */
    float bg[3];         /* background colour */
} gs_raster_desc;
typedef struct gs_raster gs_raster;
/* GS_EINVAL for a face index outside [0, n_vertices), a bad camera or
 * non-positive sigma / gamma. */
GS_API gs_status gs_raster_create(gs_ctx* ctx, const gs_raster_desc* desc, gs_raster** out);
GS_API void gs_raster_destroy(gs_raster* r);
/* New pose / intrinsics, same image size (GS_EINVAL otherwise). */
GS_API gs_status gs_raster_set_camera(gs_raster* r, const gs_camera* camera);
/* image [H][W][4] from DEVICE x [n_vertices][3] and colours [n_vertices][3];
 * keeps copies of x, colours and the per-pixel values the backward needs.
 * Deterministic (no atomics).  Enqueued on `stream`. */
GS_API gs_status gs_raster_forward(gs_raster* r, const float* x, const float* colours, float* image, void* stream);
/* dL/dx and dL/dcolours (DEVICE [n_vertices][3], each nullable) of a loss
 * with DEVICE dL/dimage [H][W][4], at the last forward's inputs
 * (GS_ESTATE without one).  Deterministic.  Enqueued on `stream`. */
GS_API gs_status gs_raster_backward(gs_raster* r, const float* dL_dimage, float* dL_dx, float* dL_dcolours,
                                    void* stream);
/* Current state (x, v) [n_nodes][3] in caller order; nullable = unchanged. */
GS_API gs_status gs_mesh_set_state(gs_mesh* mesh, const float* x, const float* v, int mem_space, void* stream);
/* Back to the description's initial state: x = X exactly (the state is
 * held as the displacement from X), v = v0.  Enqueued on `stream`. */
GS_API gs_status gs_mesh_reset(gs_mesh* mesh, void* stream);
/* Current state (x, v) [n_nodes][3] in caller order into caller buffers
 * (nullable = not read).  DEVICE: enqueued on `stream`; HOST: copied through a
 * device scratch, and the call synchronises `stream`. */
GS_API gs_status gs_mesh_get_state(gs_mesh* mesh, float* x, float* v, int mem_space, void* stream);
/* Sticky per-mesh status from the device since the last reset: GS_OK,
 * GS_ETIMEOUT (a bounded wait inside a step kernel ran out: the kernel gave
 * up on its shared-memory copies and returned; the results are invalid) or
 * GS_ENONFINITE (a NaN/Inf appeared in the state).  Synchronises the stream. */
GS_API gs_status gs_mesh_check(gs_mesh* mesh, int reset, void* stream);

/* ---- forward (App. B semi-implicit Euler) --------------------------------- */
/* Advance the current state n_steps steps of size dt in place.  Returns
 * GS_WUNSTABLE (work still enqueued) when dt exceeds the stability estimate. */
GS_API gs_status gs_step(gs_mesh* mesh, float dt, int n_steps, void* stream);

/* Differentiable rollout: n_steps steps from the current state, keeping a
 * checkpoint of (x, v) every K steps (K = 0: ceil(sqrt(n_steps)); K = 1
 * keeps every state and the element force at each, 48 B per node and step,
 * and the adjoint then recomputes nothing).  With target (N x 3, caller order,
 * nullable) the FP64 loss L = sum_i |x_i(S) - x*_i|^2 is written to *loss_out
 * (DEVICE or HOST per mem_space; nullable).  The current state advances to
 * step S.  Enables one later gs_adjoint. */
GS_API gs_status gs_rollout(gs_mesh* mesh, float dt, int n_steps, int K, const float* target,
                     double* loss_out, int mem_space, void* stream);

/* Reverse pass of the last gs_rollout (App. B discrete adjoint): seeds
 * dL/dx(S) = 2 (x(S) - x*) from the rollout's target (if any) plus dL_dxT,
 * dL/dv(S) = dL_dvT (both nullable, N x 3, caller order, `mem_space`),
 * recomputes each checkpoint segment and runs the reverse steps.  Gradient
 * pointers in `grads` are DEVICE pointers unless mem_space is GS_MEM_HOST.
 * GS_ESTATE without a preceding rollout.  keep != 0 keeps the checkpoints
 * for another adjoint with different seeds. */
GS_API gs_status gs_adjoint(gs_mesh* mesh, const float* dL_dxT, const float* dL_dvT, const gs_grads* grads,
                     int mem_space, int keep, void* stream);

/* ---- batching: many meshes, one launch per kernel per step ----------------- */
/* The batch references the meshes (they must outlive it); each mesh keeps its
 * own state.  Results per mesh are bitwise those of the mesh run alone. */
GS_API gs_status gs_batch_create(gs_ctx* ctx, gs_mesh* const* meshes, int n, gs_batch** out);
GS_API void gs_batch_destroy(gs_batch* batch);
/* Every mesh advances n_steps steps of its own dt[i] (host array [n]), one
 * launch per kernel per step (App. B); GS_WUNSTABLE as gs_step. */
GS_API gs_status gs_batch_step(gs_batch* batch, const float* dt, int n_steps, void* stream);
/* dt[n]; targets[n] (nullable entries) device pointers; loss_out device [n]. */
GS_API gs_status gs_batch_rollout(gs_batch* batch, const float* dt, int n_steps, int K,
                           const float* const* targets, double* loss_out, void* stream);
/* grads[n] (device pointers inside). */
GS_API gs_status gs_batch_adjoint(gs_batch* batch, const gs_grads* grads, void* stream);

/* ---- loss without device allocation ----------------------------------------- */
/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory while they run: a real-time control loop
 * (for instance a model-predictive controller evaluating the loss every
 * tick) cannot afford cudaMalloc, which may synchronise the device and take
 * unbounded time, and a host that owns a fixed memory pool may forbid
 * libraries from allocating at all.
 *
 * Computes L = sum_i |x_i - target_i|^2 in FP64 into *loss_out and, when
 * dL_dx is non-NULL, dL/dx = 2 (x - target).  x, target, dL_dx: DEVICE
 * [n_nodes][3] float; loss_out: one DEVICE double; all caller-owned.  The
 * call allocates nothing: its reduction scratch is a fixed array of
 * GS_NOALLOC_MAX_NODES / 256 doubles (128 KiB) inside the library that every
 * GPU loading the library holds until exit.  n_nodes above
 * GS_NOALLOC_MAX_NODES is rejected with GS_EINVAL before any work.  The first
 * call on a device looks up the array's device address (once per device);
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: after cudaDeviceReset (which destroys the device's
 * primary context and with it the array) this entry point must not be
 * called again on that device.  All calls share the array: calls whose work
 * overlaps on the GPU race and must be serialised by the caller.  Enqueued
 * on `stream`. */
#define GS_NOALLOC_MAX_NODES 4194304
GS_API gs_status gs_loss_noalloc(const float* x, const float* target, int n_nodes, double* loss_out,
                                 float* dL_dx, void* stream);

/* ---- serving: continuous batching of gradient queries ---------------------- */
typedef struct gs_server_opts {
    size_t hbm_budget_bytes;  /* admission budget for query state + checkpoints */
    int max_active;           /* 0 = unlimited slots                            */
    int K;                    /* checkpoint interval (0 = per query, ~sqrt(S))  */
    int use_graphs;           /* reserved                                       */
    int build_threads;        /* host threads that build query meshes (0 = 4)   */
} gs_server_opts;

/* A query: one system-identification gradient request (mesh, materials,
 * dt, horizon, target).  All pointers are HOST pointers copied at submit. */
typedef struct gs_query {
    gs_mesh_desc mesh;
    float dt;
    int n_steps;
    const float* target;      /* [n_nodes][3] */
} gs_query;

typedef struct gs_result {
    gs_status status;
    double loss;
    int n_elems, n_hinges, n_nodes;
    double* d_mu;             /* host arrays owned by the result */
    double* d_lambda;
    double* d_density;
    double* d_kb;
    float* d_x0;
    float* d_v0;
    double t_submit, t_admit, t_done;  /* seconds on the server clock */
} gs_result;

typedef struct gs_server_stats {
    uint64_t submitted, completed, rejected, active, queued;
    double p50_latency_s, p99_latency_s;
    double elem_steps_per_s;   /* fwd+adjoint element-steps over busy time */
    size_t admitted_bytes;
    /* where the time went (seconds): wall time with work in the server;
     * builder-thread time building meshes (summed over threads); worker time
     * starting queries, rebuilding launch lists, uploading device records,
     * and blocked on the GPU (bounding the ticks in flight) */
    double busy_s, build_s, start_s, rebuild_s, rt_sync_s, gpu_wait_s;
    uint64_t ticks, rebuilds, rt_syncs;
} gs_server_stats;

/* Starts the worker thread and opts->build_threads mesh builders (0: 4);
 * opts nullable = defaults.  GS_ENOMEM if the threads cannot be started. */
GS_API gs_status gs_server_create(gs_ctx* ctx, const gs_server_opts* opts, gs_server** out);
/* Stops the server thread; pending queries end as GS_ECANCELLED. */
GS_API void gs_server_destroy(gs_server* server);
/* The query is deep-copied (its buffers may be freed on return).  GS_ENOMEM
 * at once if the query alone exceeds the whole budget; GS_EINTERNAL once the
 * worker has stopped on a host-side failure. */
GS_API gs_status gs_query_submit(gs_server* server, const gs_query* q, uint64_t* ticket);
/* GS_OK (result filled; free it with gs_result_free), GS_PENDING /
 * GS_ETIMEOUT (not done within timeout_ms; 0 = do not wait), GS_ECANCELLED,
 * GS_ENONFINITE, GS_ENOTFOUND, GS_EINTERNAL (the worker stopped on a
 * host-side failure).  A finished ticket is collected by this call and is
 * unknown afterwards. */
GS_API gs_status gs_query_poll(gs_server* server, uint64_t ticket, gs_result* out, int timeout_ms);
/* Marks the query cancelled: a query still queued is dropped, a running one
 * stops at the worker's next tick (steps already enqueued still run); either
 * ends as GS_ECANCELLED.  GS_ENOTFOUND for an unknown ticket. */
GS_API gs_status gs_query_cancel(gs_server* server, uint64_t ticket);
/* Counts, latency percentiles and the time breakdown since creation. */
GS_API gs_status gs_server_stats_get(gs_server* server, gs_server_stats* out);
/* Frees a polled result's host arrays and clears their pointers (NULL-safe). */
GS_API void gs_result_free(gs_result* r);

/* ---- self-test of the kernels' failure path (no paper counterpart) --------
 * Every wait inside the step kernels (for shared-memory copies, or for a
 * stage to be released) is bounded; when it runs out the kernel sets status
 * bit 2, waits once more (bounded) and returns, so that the context stays
 * usable.  This launches one CTA whose thread waits on a shared-memory
 * barrier that nothing arrives at, with `iterations` polls (1..1e6), and
 * writes the status word to *status_out (HOST): 2 when the wait ran out as
 * designed.  Synchronises the stream.  GS_EINVAL on bad arguments. */
GS_API gs_status gs_selftest_bounded_wait(int iterations, int* status_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
