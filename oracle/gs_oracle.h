/*
 * FP64 CPU oracle for the differentiable explicit step of
 * "gradSim: Differentiable simulation for system identification and
 * visuomotor control" (ICLR 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct
 * restatement of the paper's equations in double precision, used by the test
 * suite, by the package's smoke check and by the benchmark's CPU-baseline leg
 * to check the CUDA library.  Nothing in the product path may link, load or
 * call it, and it shares no code with the CUDA library.
 *
 * What it computes (paper section / equation in brackets):
 *   - stable neo-Hookean tetrahedra, Psi = mu/2 (I_C - 3) + lambda/2 (J - a)^2
 *     - mu/2 log(I_C + 1), U = sum V_e Psi_e, f = -grad U   [App. A.1, App. C.1]
 *   - constant-strain triangles with the same energy in the plane
 *     (I_C - 2 offset), and Bridson's dihedral bending force
 *     f_b = k_b sin(phi/2 + alpha) d                         [App. A.1]
 *   - a lift/drag air model on the cloth surface (flat-plate reading)
 *                                                          [App. A.1]
 *   - compliant contact f_n = n (k_e C + k_d dC/dt) with relaxed Coulomb
 *     friction against a ground plane and a sphere          [App. A.1, App. C.2]
 *   - semi-implicit Euler u+ = u- + dt M^-1 f(s-), q+ = q- + dt u+  [App. B]
 *   - the discrete adjoint of that step through the whole rollout, taken in
 *     the order of App. B: solve (dg/ds+)^T c = -(dl/ds+)^T, then
 *     dl/ds- = c^T dg/ds-, dl/dtheta += c^T dg/dtheta        [App. B]
 *   - a loss on final node positions L = sum ||x_i(S) - x*_i||^2.
 *
 * Readings of the paper that the text leaves open are listed with the
 * functions that take them (rest-stable alpha, contact sign, friction form,
 * gravity mask, bending scale).
 *
 * Derivatives: every force routine is a template over the scalar type, and
 * the per-element Jacobians used by the adjoint are exact forward-mode
 * derivatives obtained by evaluating the same routine on dual numbers.
 * Nothing is hand-differentiated here.
 */
#ifndef GS_ORACLE_H
#define GS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_model {
    int n_nodes;
    const double* X;          /* [3N] rest positions */
    int n_tets;
    const int* tets;          /* [4 n_tets] */
    const double* tet_mu;     /* [n_tets] Lame mu */
    const double* tet_lam;    /* [n_tets] Lame lambda */
    const double* tet_rho;    /* [n_tets] density */
    const double* tet_act;    /* [n_tets] actuation, nullable (0) */
    int n_tris;
    const int* tris;          /* [3 n_tris] */
    const double* tri_mu;
    const double* tri_lam;
    const double* tri_rho;    /* areal density */
    const double* tri_act;    /* nullable */
    int n_hinges;
    const int* hinges;        /* [4 n_hinges]: wing tips x1, x2; edge x3 -> x4 */
    const double* hinge_kb;
    const double* hinge_act;  /* nullable */
    const unsigned char* pinned; /* [N] nullable: 1 = kinematic (w = 0) */
    double gravity[3];
    double ke, kd, kf, mu_f;
    int plane_on;
    double plane_n[3];
    double plane_h;
    int sphere_on;
    double sphere_c[3];
    double sphere_r;
    /* time-varying actuation (the control input of Sec. 3 "visuomotor
     * control"): row n of each [n_act_steps][n] array is added to the
     * element's actuation during step n < n_act_steps; nullable */
    int n_act_steps;
    const double* tet_act_seq;
    const double* tri_act_seq;
    const double* hinge_act_seq;
    /* air on the cloth surface (App. A.1 "Deformable Thin-Shells": lift and
     * drag from the air around the cloth; the paper gives no formula, the
     * reading is stated at air_forces_t): per triangle, drag and lift
     * coefficients k_drag, k_lift (kg/m^3) against a uniform wind (m/s) */
    int air_on;
    double k_drag, k_lift;
    double wind[3];
} orc_model;

/* Gradient outputs; every pointer nullable. */
typedef struct orc_grads {
    double* x0;        /* [3N] */
    double* v0;        /* [3N] */
    double* tet_mu;    /* [n_tets] */
    double* tet_lam;
    double* tet_rho;
    double* tet_act;
    double* tri_mu;    /* [n_tris] */
    double* tri_lam;
    double* tri_rho;
    double* tri_act;
    double* hinge_kb;  /* [n_hinges] */
    double* hinge_act;
    double* contact;   /* [4]: ke, kd, kf, mu_f */
    double* node_mass; /* [N]: dL/dm_i */
    /* [S][n]: dL/d(actuation of the element during step n), every step */
    double* tet_act_seq;
    double* tri_act_seq;
    double* hinge_act_seq;
} orc_grads;

/* Directions for the forward-mode (dual number) rollout; every pointer nullable (= 0). */
typedef struct orc_dirs {
    const double* x0;
    const double* v0;
    const double* tet_mu;
    const double* tet_lam;
    const double* tet_rho;
    const double* tet_act;
    const double* tri_mu;
    const double* tri_lam;
    const double* tri_rho;
    const double* tri_act;
    const double* hinge_kb;
    const double* hinge_act;
    const double* contact; /* [4] */
    const double* tet_act_seq;   /* [n_act_steps][n] */
    const double* tri_act_seq;
    const double* hinge_act_seq;
} orc_dirs;

/* ---- rigid bodies (App. A.1 "Rigid Bodies") ----------------------------
 * State of a body: x (centre of mass), r = (w, x, y, z) unit quaternion
 * (world from body), v, omega (world frame): 13 doubles in that order.
 * Design parameters: mass m, body-frame inertia about the centre of mass
 * (Ixx, Iyy, Izz, Ixy, Ixz, Iyz) and the contact parameters (ke, kd, kf, mu)
 * of the compliant contact model, applied at every body-frame contact point
 * with the particles' contact law against the scene's plane / sphere. */
typedef struct orc_rigid {
    int n_points;
    const double* points;   /* [n_points][3] body frame, about the centre of mass */
    double mass;
    double inertia[6];      /* Ixx, Iyy, Izz, Ixy, Ixz, Iyz */
    double contact[4];      /* ke, kd, kf, mu */
    const orc_model* scene; /* plane / sphere and gravity (mesh fields unused) */
} orc_rigid;
/* rollout of S steps: state0 [13] -> stateS [13]; traj [(S+1)][13] nullable */
int orc_rigid_rollout(const orc_rigid* b, const double* state0, double dt, int S, double* stateS, double* traj);
/* L = sum_k |X_k(S) - target_k|^2 over the world positions of the points at
 * step S, plus dot(seed, state(S)) for a nullable seed [13]; gradients:
 * d_state0 [13], d_mass [1], d_inertia [6], d_contact [4] (each nullable) */
int orc_rigid_loss_grad(const orc_rigid* b, const double* state0, double dt, int S, const double* target,
                        const double* seed, double* loss, double* d_state0, double* d_mass, double* d_inertia,
                        double* d_contact);
/* the same loss and its derivative along (d_state0 [13], d_mass, d_inertia [6], d_contact [4]) by forward mode */
int orc_rigid_loss_dir(const orc_rigid* b, const double* state0, double dt, int S, const double* target,
                       const double* seed, const double* dir_state0, double dir_mass, const double* dir_inertia,
                       const double* dir_contact, double* loss, double* dloss);

/* ---- rest-state set-up ------------------------------------------------- */
void orc_tet_rest(const double X[12], double Dminv[9], double* V);
void orc_tri_rest(const double X[9], double Dminv[4], double* A);
/* air force on one triangle's corners (x, v: 3 corners x 3) */
void orc_air_forces(const double x[9], const double v[9], double k_drag, double k_lift, const double wind[3],
                    double f[9]);
/* lumped node masses m_i (pinned nodes included) */
int orc_node_masses(const orc_model* m, double* mass);

/* ---- single-element physics ------------------------------------------- */
void orc_tet_forces(const double x[12], const double Dminv[9], double V,
                    double mu, double lam, double act, double f[12]);
double orc_tet_energy(const double x[12], const double Dminv[9], double V,
                      double mu, double lam, double act);
void orc_tri_forces(const double x[9], const double Dminv[4], double A,
                    double mu, double lam, double act, double f[9]);
double orc_tri_energy(const double x[9], const double Dminv[4], double A,
                      double mu, double lam, double act);
void orc_hinge_forces(const double x[12], double kb, double act, double f[12]);
double orc_hinge_angle(const double x[12]);
/* exact d(phi)/dx by forward-mode differentiation of the atan2 angle */
void orc_hinge_angle_grad(const double x[12], double g[12]);
void orc_contact_force(const orc_model* m, const double x[3], const double v[3], double f[3]);

/* ---- whole-mesh -------------------------------------------------------- */
/* total force f(s) on every node (elastic + bending + contact, no gravity) */
int orc_forces(const orc_model* m, const double* x, const double* v, double* f);
/* S steps of semi-implicit Euler from (x0, v0); traj (nullable) receives
 * all S+1 positions [S+1][3N] */
int orc_rollout(const orc_model* m, const double* x0, const double* v0, double dt, int S,
                double* xS, double* vS, double* traj);
/* L = sum ||x(S) - target||^2 and its gradients by the discrete adjoint.
 * xbar_extra/vbar_extra (nullable) add dL/dx(S), dL/dv(S) of a further loss
 * term; target nullable (then L = 0 and only the extra seeds are used). */
int orc_loss_grad(const orc_model* m, const double* x0, const double* v0, double dt, int S,
                  const double* target, const double* xbar_extra, const double* vbar_extra,
                  double* loss, orc_grads* g);
/* forward-mode: L and dL along the given directions (dual numbers) */
int orc_loss_dir(const orc_model* m, const double* x0, const double* v0, double dt, int S,
                 const double* target, const orc_dirs* d, double* loss, double* dloss);

/* Threads for the independent per-element and per-node loops (OpenMP; the
 * node sums stay serial in element order, so results are bitwise the same
 * for any count).  n <= 0 restores the default (all cores).  Returns the
 * count now in effect; 1 when the oracle was built without OpenMP. */
int orc_set_threads(int n);
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
