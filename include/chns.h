/*
 * chns.h - C ABI of the GB300 (sm_103a) library for the matrix-free hot path of a
 * projection-based, semi-implicit Cahn-Hilliard Navier-Stokes (CHNS) scheme on adaptive
 * octrees (arXiv:2107.05123).
 *
 * What is computed follows the paper:
 *   - mesh: leaves of a 2:1-balanced octree in Morton order, nodes and hanging nodes
 *     (Sec. 5.2 "Octree construction and 2:1 balancing", Sec. 5.3 "Identification of
 *     unique, independent nodes"; hanging values interpolated from the parent, Fig. "traversal");
 *   - operators (Sec. 4.1): pressure Poisson (Def. weak_VMS_disc_pp_vel), velocity update
 *     (Def. weak_VMS_disc_vel_update), Cahn-Hilliard Newton Jacobian (Def. weak_VMS_disc_CH),
 *     RBVMS velocity prediction (Def. weak_VMS_disc, tau_m and R_m definitions);
 *   - the two-block time step of the flowchart (Fig. "flowchart_block").
 * Discretisation: Q1 hexahedra on axis-aligned box leaves, 2x2x2 Gauss quadrature.
 *
 * Conventions shared by every entry point
 *   - Units: anchors are integer coordinates in units of 2^-CHNS_MAXD of the unit cube; the
 *     physical domain is [0,Lx]x[0,Ly]x[0,Lz] (per-axis scaling of the unit octree).
 *   - Nodes: independent (non-hanging) nodes, numbered in Morton order of their integer
 *     coordinates. A nodal vector of n components is n contiguous arrays of n_nodes values
 *     (component-major), e.g. the CH pair is [phi(0..N-1), mu(0..N-1)].
 *   - Memory: every vector/field pointer is a DEVICE pointer owned by the caller, contiguous,
 *     of the element type selected by the precision argument (double for CHNS_FP64, float for
 *     the FP32 modes; coefficient fields are uint16 bfloat16 for CHNS_FP32_BF16COEF, where the
 *     phase field is stored shifted as bfloat16(1 + phi~) so that the relative error of
 *     rho(phi) stays below 2^-8 even for large density ratios). The
 *     library owns the mesh tables and a device workspace allocated by chns_mesh_create;
 *     nothing is allocated on later calls.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream). Applies are
 *     asynchronous. Solves and steps synchronise the stream when they read convergence scalars.
 *   - Errors: no exception crosses the ABI. Every call returns a chns_status; on failure
 *     chns_last_error() gives a message (thread-local). Invalid arguments are rejected before
 *     any launch. Non-convergence returns CHNS_ENOTCONV with the last iterate in x.
 *   - Calls on one mesh share its workspace: do not run two solves/steps on the same mesh
 *     concurrently.
 */
#ifndef CHNS_H
#define CHNS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHNS_MAXD 20          /* finest representable level is CHNS_MAXD-1 */
#define CHNS_GMRES_MAX_RESTART 40

typedef enum {
  CHNS_OK = 0,
  CHNS_EINVAL = 1,        /* bad argument, unsorted / overlapping / non-covering leaves */
  CHNS_EUNBALANCED = 2,   /* leaves violate the 2:1 condition (faces, edges, corners) */
  CHNS_ENOMEM = 3,        /* device or host allocation failed */
  CHNS_ECUDA = 4,         /* a CUDA runtime call failed */
  CHNS_ENOTCONV = 5,      /* iteration limit reached before the tolerance */
  CHNS_EBREAKDOWN = 6,    /* Krylov breakdown (zero or negative curvature, zero norm) */
  CHNS_ENAN = 7           /* NaN/Inf detected in a residual norm */
} chns_status;

typedef enum {
  CHNS_FP64 = 0,          /* double vectors, double coefficients */
  CHNS_FP32 = 1,          /* float vectors, float coefficients */
  CHNS_FP32_BF16COEF = 2  /* float vectors, bfloat16 coefficient fields */
} chns_precision;

typedef enum {
  CHNS_OP_POISSON = 0,    /* (grad q, (1/rho~) grad p), 1 component, natural BC */
  CHNS_OP_MASS = 1,       /* (w, rho~ u), 3 components, Dirichlet rows = identity */
  CHNS_OP_CH = 2,         /* CH Newton Jacobian, 2 components [dphi; dmu] */
  CHNS_OP_MOMENTUM = 3    /* velocity-prediction operator, 3 components, Dirichlet identity */
} chns_operator;

typedef enum { CHNS_KSP_CG = 0, CHNS_KSP_GMRES = 1 } chns_ksp;
/* JACOBI: inverse of the exact diagonal; for CHNS_OP_CH the inverse of the exact 2x2 nodal
 * (phi, mu) blocks. */
typedef enum { CHNS_PC_NONE = 0, CHNS_PC_JACOBI = 1 } chns_pc;

typedef struct chns_mesh chns_mesh;   /* opaque; owns device tables and workspace */

typedef struct {
  int64_t n_elem;
  int64_t n_nodes;        /* independent nodes (degrees of freedom per component) */
  int64_t n_hanging;
  int64_t n_boundary;     /* independent nodes on the domain boundary */
  int32_t min_level, max_level;
  double extent[3];
} chns_mesh_info;

/* Physical parameters (Sec. 3): Re, We, Cn, Pe, Fr; rho_ratio = rho_+/rho_-,
 * eta_ratio = eta_+/eta_- with phase phi = +1 the reference fluid; time step dt; C_I of tau_m. */
typedef struct {
  double Re, We, Cn, Pe, Fr, rho_ratio, eta_ratio, dt, C_I;
} chns_params;

/* Coefficient fields of an operator (device pointers, n_nodes values each, type by precision):
 *   phi_tilde: phi~ (all operators; density/viscosity use clamp(phi~, -1, 1) at quad. points)
 *   u_adv[3]:  advecting velocity (u_hat for MOMENTUM, u~ for CH), unused by POISSON/MASS
 *   mu_tilde:  mu~ (MOMENTUM: J_hat = -(alpha/Cn) grad mu~), unused otherwise */
typedef struct {
  const void* phi_tilde;
  const void* u_adv[3];
  const void* mu_tilde;
} chns_coef;

/* ---------------------------------------------------------------- mesh (Sec. 5.2, 5.3) */

/* Build the mesh from host arrays: anchors[3*n] (x,y,z per leaf, units 2^-CHNS_MAXD, aligned to
 * the leaf size), levels[n] (0..CHNS_MAXD-1), in strictly increasing Morton order, disjoint and
 * covering the unit cube, 2:1 balanced across faces, edges and corners. extent = (Lx,Ly,Lz) > 0.
 * Enumerates nodes, hanging nodes (edge midpoints: 2 parents, weight 1/2; face centres:
 * 4 parents, weight 1/4) and uploads the tables. Returns EINVAL / EUNBALANCED on bad input. */
chns_status chns_mesh_create(const uint32_t* anchors, const uint8_t* levels, int64_t n_leaves,
                             const double extent[3], void* stream, chns_mesh** out);
chns_status chns_mesh_get_info(const chns_mesh* mesh, chns_mesh_info* info);
/* Integer node coordinates (host buffer of 3*n_nodes uint32, units 2^-CHNS_MAXD). */
chns_status chns_mesh_node_coords(const chns_mesh* mesh, uint32_t* coords);
/* Boundary flag per node (host buffer of n_nodes bytes, 1 on the domain boundary). */
chns_status chns_mesh_boundary(const chns_mesh* mesh, uint8_t* flags);
void chns_mesh_destroy(chns_mesh* mesh);

/* ---------------------------------------------------------------- operator applies (Sec. 4.1)
 * y = A x, matrix-free: gather (with hanging interpolation) -> element quadrature -> scatter-add
 * (transpose incl. hanging). x and y must not alias. */
chns_status chns_apply_poisson(const chns_mesh* mesh, const chns_params* prm, const chns_coef* coef,
                               const void* x, void* y, chns_precision prec, void* stream);
chns_status chns_apply_mass(const chns_mesh* mesh, const chns_params* prm, const chns_coef* coef,
                            const void* x3, void* y3, chns_precision prec, void* stream);
chns_status chns_apply_ch(const chns_mesh* mesh, const chns_params* prm, const chns_coef* coef,
                          const void* x2, void* y2, chns_precision prec, void* stream);
chns_status chns_apply_momentum(const chns_mesh* mesh, const chns_params* prm,
                                const chns_coef* coef, const void* x3, void* y3,
                                chns_precision prec, void* stream);
/* Diagonal of an operator's assembled matrix (exact, incl. hanging-node couplings; identity on
 * Dirichlet rows). d has the operator's number of components. */
chns_status chns_operator_diagonal(const chns_mesh* mesh, chns_operator op, const chns_params* prm,
                                   const chns_coef* coef, void* d, chns_precision prec,
                                   void* stream);

/* ---------------------------------------------------------------- right-hand sides (FP64)
 * CH residual at the new-time iterate (phi, mu) (Def. weak_VMS_disc_CH): f2 = [F_phi; F_mu].
 * u_t[3] = u~. All device double arrays of n_nodes. */
chns_status chns_residual_ch(const chns_mesh* mesh, const chns_params* prm, const double* phi,
                             const double* mu, const double* phi_k, const double* mu_k,
                             const double* const u_t[3], double* f2, void* stream);
/* Velocity-prediction right-hand side b3 (Def. weak_VMS_disc; Dirichlet rows set to 0).
 * coef: phi~, u_hat, mu~ (double). u_k[3], p_k: previous velocity and pressure (p/We). */
chns_status chns_rhs_momentum(const chns_mesh* mesh, const chns_params* prm, const chns_coef* coef,
                              const double* const u_k[3], const double* p_k, double* b3,
                              void* stream);
/* Pressure-Poisson right-hand side (Def. weak_VMS_disc_pp_vel, incl. the boxed RBVMS term),
 * not mean-projected. v[3] = v^{k+1}. */
chns_status chns_rhs_poisson(const chns_mesh* mesh, const chns_params* prm, const chns_coef* coef,
                             const double* const v[3], const double* const u_k[3],
                             const double* p_k, double* b, void* stream);
/* Velocity-update right-hand side (Def. weak_VMS_disc_vel_update; Dirichlet rows = 0). */
chns_status chns_rhs_velocity_update(const chns_mesh* mesh, const chns_params* prm,
                                     const chns_coef* coef, const double* const v[3],
                                     const double* const u_k[3], const double* p_k,
                                     const double* p_new, double* b3, void* stream);
/* Integral of phi (1^T M phi) by the same quadrature, FP64 (Prop. mass_conservation). */
chns_status chns_phi_mass(const chns_mesh* mesh, const double* phi, double* out_host, void* stream);

/* The same phi integral for callers that cannot allocate memory while they run: code inside a
 * CUDA stream capture (where allocation calls are not allowed), or an application whose memory
 * is all reserved up front by its own pool so that a library may not take any more. The paper
 * has no counterpart; this is a property of the library only.
 * Nothing is allocated during the call: the block partial sums and the finishing ticket live in
 * a fixed scratch array inside the library (65,536 partial sums, ~0.5 MB, which every GPU that
 * loads the library keeps until the process exits), and the result is written to `out`, a
 * device double owned by the caller. The call is asynchronous on `stream`.
 * Limits and rules: meshes of more than 8,388,608 elements are rejected with CHNS_EINVAL. The
 * first call on a device looks up the scratch array's device address on the current device;
 * make that first call before any stream capture. Every call shares the one scratch array, so
 * calls that overlap on the GPU (other streams, other threads) race and give wrong results:
 * serialise them. */
chns_status chns_phi_mass_noalloc(const chns_mesh* mesh, const double* phi, double* out,
                                  void* stream);

/* ---------------------------------------------------------------- Krylov solves
 * Solve A x = b for an operator, b and x FP64 device arrays of the operator's component count;
 * x holds the initial guess on entry. Stops at ||b - A x||_2 <= rtol ||b||_2 (FP64 residual).
 * POISSON: b is projected to mean zero and x is returned with mean zero (pure Neumann).
 * inner_precision = CHNS_FP64 runs the whole Krylov iteration in FP64. The FP32 modes run the
 * Krylov iterations with FP32 vectors and applies, FP64 dot products, inside an FP64 iterative
 * refinement loop (r = b - A_64 x in FP64, correction solved to inner_rtol). A refinement cycle
 * that fails to reduce the FP64 residual by 4x raises the inner precision (BF16 coefficients -> FP32
 * -> FP64 Krylov for the rest of the solve); stats report how often.
 * coef arrays are FP64; reduced-precision copies are made in the mesh workspace. In
 * CHNS_FP32_BF16COEF mode the bfloat16 copies are used by the memory-bound POISSON and MASS
 * applies; CH and MOMENTUM inner applies use FP32 coefficients. The Jacobi preconditioner is
 * computed in the precision of the Krylov iteration that uses it. */
typedef struct {
  int32_t ksp;              /* chns_ksp */
  int32_t pc;               /* chns_pc */
  double rtol;
  int32_t max_it;           /* total Krylov iterations over all refinement cycles */
  int32_t restart;          /* GMRES restart length, 1..CHNS_GMRES_MAX_RESTART */
  int32_t inner_precision;  /* chns_precision */
  double inner_rtol;        /* FP32 modes: relative tolerance of each correction solve */
  int32_t max_refine;       /* FP32 modes: maximum refinement cycles */
  int32_t check_every;      /* CG: iterations between host convergence checks (>= 1) */
} chns_solver_params;

typedef struct {
  int32_t iterations;
  int32_t refinements;
  double rel_residual;      /* final ||b - A x|| / ||b|| in FP64 */
  double b_norm;
  int32_t status;           /* chns_status of the solve */
  float ms;                 /* device time of the solve (CUDA events) */
  int32_t escalations;      /* refinement cycles that raised the inner precision */
  int32_t final_precision;  /* chns_precision of the last inner iterations */
} chns_solve_stats;

chns_status chns_krylov_solve(const chns_mesh* mesh, chns_operator op, const chns_params* prm,
                              const chns_coef* coef, const double* b, double* x,
                              const chns_solver_params* sp, chns_solve_stats* stats,
                              void* stream);

/* ---------------------------------------------------------------- time step (Fig. flowchart_block)
 * Advance (phi, mu, u, u_old, p) by one step of two blocks: CH (Newton), velocity prediction,
 * pressure Poisson, velocity update. All fields FP64 device arrays of n_nodes, updated in
 * place: phi, mu, u[3] <- u^{k+1}, u_old[3] <- u^k, p <- p^{k+1} (p is pressure/We). */
typedef struct {
  double* phi;
  double* mu;
  double* u[3];
  double* u_old[3];
  double* p;
} chns_state;

typedef struct {
  chns_solver_params ch, vp, pp, vu;
  double newton_rtol;       /* ||F|| <= newton_rtol ||F_0|| (or newton_atol) ends Newton */
  double newton_atol;
  int32_t newton_max_it;
  int32_t blocks;           /* block iterations per step (2 in the paper) */
} chns_step_params;

typedef struct {
  int32_t newton_its[2];
  chns_solve_stats ch[2], vp[2], pp[2], vu[2];
  double phi_mass_before, phi_mass_after;
  float ms_ch, ms_vp, ms_pp, ms_vu, ms_total;
} chns_step_stats;

chns_status chns_step(const chns_mesh* mesh, chns_state* state, const chns_params* prm,
                      const chns_step_params* sp, chns_step_stats* stats, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* chns_last_error(void);
/* Library version string. */
const char* chns_version(void);
/* Number of kernels this library has launched since it was loaded (a diagnostic counter,
 * process-wide, all devices). */
uint64_t chns_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* CHNS_H */
