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
 *     library owns the mesh tables and a device workspace allocated by chns_mesh_create.
 *     A few buffers are added to the mesh on first use and kept until chns_mesh_destroy: the
 *     momentum quadrature data (a momentum solve), the inverse diagonals of the Schur
 *     preconditioner (a CH solve with CHNS_PC_SCHUR) and the velocity-update terms of chns_step
 *     (24 doubles per leaf). chns_transfer and chns_mesh_remesh allocate temporaries; the
 *     multigrid and learned objects own their memory.
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
  CHNS_FP32_BF16COEF = 2, /* float vectors, bfloat16 coefficient fields */
  CHNS_FP64_DF = 3        /* double vectors and coefficients; the Poisson and mass applies
                           * compute in double-float (pairs of FP32 numbers, rounding ~1e-14 per
                           * operation), the CH and momentum applies in FP64, which is faster
                           * for them (operator applies and fp64_apply only) */
} chns_precision;

typedef enum {
  CHNS_OP_POISSON = 0,    /* (grad q, (1/rho~) grad p), 1 component, natural BC */
  CHNS_OP_MASS = 1,       /* (w, rho~ u), 3 components, Dirichlet rows = identity */
  CHNS_OP_CH = 2,         /* CH Newton Jacobian, 2 components [dphi; dmu] */
  CHNS_OP_MOMENTUM = 3    /* velocity-prediction operator, 3 components, Dirichlet identity */
} chns_operator;

/* FCG: flexible CG (Polak-Ribiere beta = z_new.(r_new - r_old) / r_old.z_old), for a
 * preconditioner that changes from one application to the next; POISSON only. */
typedef enum { CHNS_KSP_CG = 0, CHNS_KSP_GMRES = 1, CHNS_KSP_FCG = 2 } chns_ksp;
/* JACOBI: inverse of the exact diagonal; for CHNS_OP_CH the inverse of the exact 2x2 nodal
 * (phi, mu) blocks. LEARNED (with CHNS_KSP_FCG on POISSON): the coarse correction c(r) of a
 * trained network (see chns_learned below) followed by one damped Jacobi step on what it
 * leaves, z = c + omega D^-1 (r - A c) with omega = 2/3. */
/* CHEBYSHEV (POISSON, with CG or FCG): z = p(D^-1 A) D^-1 r, `restart` (1..16) steps of the
 * Chebyshev iteration on [lmax/30, lmax] with lmax = 1.1 x the largest eigenvalue of D^-1 A
 * from 15 power iterations at the start of the solve (in the precision of the iteration);
 * restart - 1 extra applies per iteration. A fixed SPD preconditioner (as long as lmax bounds
 * the spectrum), run through the flexible-CG driver. */
/* SCHUR (CH with GMRES): block upper-triangular preconditioner of the Newton Jacobian
 * [A B; C D] (rows phi, mu; B = k K, D = -M/2, k = 1/(2 Pe Cn)) built on the Schur complement of
 * D, S = A - B D^-1 C, approximated by H M^-1 H with H = M/sqrt(dt) + Cn sqrt(k) K (which keeps
 * the M/dt and Cn^2 k K M^-1 K terms of S and drops advection and psi''):
 *   z_mu = -2 M^-1 r_mu,  z_phi = H^-1 M H^-1 (r_phi - k K z_mu).
 * The inner solves are fixed numbers of Jacobi-CG iterations (inner_its with H, a quarter of
 * them, at least 4, with M) from zero, so the preconditioner varies with r and GMRES runs in
 * its flexible form (the preconditioned vectors are kept: restart <= 30). For meshes and
 * parameters where the biharmonic term dominates (small Cn h^-1), where the 2x2 nodal
 * block-Jacobi preconditioner stalls. */
/* MULTIGRID (POISSON, with CG or FCG): one V-cycle of the geometric multigrid hierarchy
 * solver_params.mg (chns_mg_create below) per iteration, run through the flexible-CG driver. The
 * hierarchy's level operators are set up for the solve's coefficient phi~ at the start of the
 * solve (chns_mg_setup) in the precision of the Krylov iteration.
 * With SCHUR, a hierarchy in solver_params.mg (optional) replaces each inner CG solve with H by
 * one V-cycle of H (chns_mg_setup_shifted with sa = 1/sqrt(dt), sb = Cn sqrt(k)), kept set up
 * from one solve to the next while dt, Pe and Cn do not change. */
typedef enum {
  CHNS_PC_NONE = 0,
  CHNS_PC_JACOBI = 1,
  CHNS_PC_LEARNED = 2,
  CHNS_PC_CHEBYSHEV = 3,
  CHNS_PC_SCHUR = 4,
  CHNS_PC_MULTIGRID = 5
} chns_pc;

typedef struct chns_mesh chns_mesh;   /* opaque; owns device tables and workspace */
typedef struct chns_learned chns_learned;  /* opaque; learned coarse correction (below) */
typedef struct chns_mg chns_mg;       /* opaque; geometric multigrid hierarchy (below) */

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

/* Launch configuration of the operator applies on this mesh (performance only: results agree
 * to rounding, since the order of floating-point additions into shared nodes differs).
 *   CHNS_APPLY_PATCH:  one CTA per patch (a run of <= 256 Morton-consecutive elements whose
 *                      nodes are gathered once into shared memory).
 *   CHNS_APPLY_STREAM: persistent CTAs, each walking the patches blockIdx, blockIdx + grid, ...
 *                      and gathering the next patch's node values into shared memory (cp.async)
 *                      while the current patch is computed. Used by the FP32 Poisson and mass
 *                      applies (including the apply fused into CG); the other operators and
 *                      precisions keep CHNS_APPLY_PATCH.
 *   CHNS_APPLY_AUTO:   CHNS_APPLY_STREAM when the mesh has at least 16 patches per SM.
 * max_ctas bounds the persistent grid (0: as many CTAs as the device holds at once). Errors:
 * EINVAL for a null mesh, an unknown kernel or max_ctas < 0. Not thread-safe against applies
 * running on the same mesh from other host threads. */
typedef enum { CHNS_APPLY_AUTO = 0, CHNS_APPLY_PATCH = 1, CHNS_APPLY_STREAM = 2 } chns_apply_kernel;
chns_status chns_mesh_set_apply_config(chns_mesh* mesh, chns_apply_kernel kernel, int64_t max_ctas);

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
 * Limits and rules: meshes of more than 8,388,608 elements are rejected with CHNS_EINVAL, and so
 * is a call made while another device is current than the one the mesh was created on. The
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
  int32_t restart;          /* GMRES restart length, 1..CHNS_GMRES_MAX_RESTART; Chebyshev degree */
  int32_t inner_precision;  /* chns_precision */
  double inner_rtol;        /* FP32 modes: relative tolerance of each correction solve */
  int32_t max_refine;       /* FP32 modes: maximum refinement cycles */
  int32_t check_every;      /* CG/FCG: iterations between host convergence checks (>= 1) */
  chns_learned* learned;    /* CHNS_PC_LEARNED: the network (not owned); else ignored */
  int32_t inner_its;        /* CHNS_PC_SCHUR: CG iterations of each inner solve with H (0: 20) */
  chns_mg* mg;              /* CHNS_PC_MULTIGRID: the hierarchy of this mesh (not owned) */
  int32_t mass_its;         /* CHNS_PC_SCHUR: Jacobi-CG iterations of each M^-1 (0: the larger of
                             * 4 and inner_its / 4) */
  int32_t fp64_apply;       /* precision of this solve's FP64-vector operator applies (the
                             * refinement residuals; every iteration when inner_precision is
                             * CHNS_FP64): CHNS_FP64 (0) or CHNS_FP64_DF */
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
  int32_t fallbacks;        /* CHNS_PC_LEARNED: 1 if the learned correction stalled (the residual
                               norm did not halve in 100 iterations) and the solve continued with
                               the Jacobi preconditioner alone, else 0 */
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
  /* Training-pair collection (learned preconditioner): when `collect` is set, the right-hand
   * side of every pressure-Poisson solve of the step is also solved as chns_learned_collect
   * does (FP64 from zero to relative residual 1e-10), and the errors x* - x_k of the iterates
   * k = collect_every, 2 collect_every, ... (at most collect_max per solve) are added to its
   * replay buffer. The step's own solution is not affected. */
  chns_learned* collect;
  int32_t collect_every;
  int32_t collect_max;
  int32_t collect_with_net;  /* iterates of FCG with the network instead of Jacobi-PCG */
  /* Velocity Dirichlet data: three FP64 device arrays of n_nodes (only the entries of boundary
   * nodes are read) imposed on v^{k+1} and u^{k+1} in place of no-slip; NULL (all three) is
   * no-slip. The data is lifted into the right-hand sides of the velocity prediction and update
   * (b - A g on the other rows, g on the boundary rows), which keeps the solved systems those of
   * zero data. The paper's weak forms assume u.n = 0 on the walls (Sec. 4): data with a normal
   * component leaves the Cahn-Hilliard boundary flux out, as the paper's forms do. */
  const double* u_bc[3];
} chns_step_params;

typedef struct {
  int32_t newton_its[2];
  chns_solve_stats ch[2], vp[2], pp[2], vu[2];
  double phi_mass_before, phi_mass_after;
  float ms_ch, ms_vp, ms_pp, ms_vu, ms_total;
} chns_step_stats;

chns_status chns_step(const chns_mesh* mesh, chns_state* state, const chns_params* prm,
                      const chns_step_params* sp, chns_step_stats* stats, void* stream);

/* ---------------------------------------------------------------- geometric multigrid
 * Not in the paper's solver stack, which preconditions the pressure Poisson system with PETSc's
 * algebraic multigrid (App. A); the paper names a geometric multigrid on the octree as the
 * remedy for the AMG setup cost that dominates its solver timings (Sec. 7, Conclusions).
 * Hierarchy: level 0 is the mesh; level l+1 replaces every leaf of level l's finest octant level
 *   by its parent (the one-level coarsening of the intergrid transfer, Sec. 5.4), until the
 *   finest octant level is at most coarsest_level; the coarsest level must have <= 1024 nodes.
 * Transfers: P_l (level l+1 -> l) evaluates the coarse finite-element function, hanging
 *   constraints included, at the level-l nodes (child interpolation, Sec. 5.4); R_l = P_l^T.
 * Level operators: the Poisson operator of each level with phi~ injected from the finer level.
 * V-cycle: `degree` Chebyshev steps on D^-1 A over [lmax / smooth_range, lmax], lmax =
 *   lmax_factor x the estimate of the largest eigenvalue of D^-1 A from `power_its` power
 *   iterations started at v_i = dinv_i (h(i) / 2^32 - 1/2), h(i) = i * 2654435761 mod 2^32;
 *   restriction of the residual; the cycle on the next level; prolongation; `degree`
 *   Chebyshev steps from the corrected iterate. Coarsest level: z = (A + 1 1^T / n)^-1 r.
 * The object owns its level meshes, transfer tables and vectors; it stays tied to the mesh it
 * was built from (which must outlive it). Defaults (params NULL): coarsest_level 2, degree 3,
 * power_its 12, smooth_range 15, lmax_factor 1.1. */
typedef struct {
  int32_t coarsest_level;   /* 0..CHNS_MAXD-1 */
  int32_t degree;           /* Chebyshev steps before and after the coarse correction, 1..8 */
  int32_t power_its;        /* 1..100 */
  double smooth_range;      /* > 1 */
  double lmax_factor;       /* >= 1 */
} chns_mg_params;

chns_status chns_mg_create(const chns_mesh* mesh, const chns_mg_params* params, void* stream,
                           chns_mg** out);
void chns_mg_destroy(chns_mg* mg);
/* number of levels; n_nodes / n_elem (optional, host arrays of n_levels) per level, fine first */
chns_status chns_mg_levels(const chns_mg* mg, int32_t* n_levels, int64_t* n_nodes,
                           int64_t* n_elem);
/* Level operators for the Poisson coefficient phi~ of level 0 (device array of n_nodes in the
 * precision prec, CHNS_FP64 or CHNS_FP32; it is read by later V-cycles and must stay valid):
 * injected coefficients, exact diagonals, Chebyshev intervals and the coarsest dense inverse.
 * Synchronises the stream. */
chns_status chns_mg_setup(chns_mg* mg, const chns_params* prm, const void* phi_tilde,
                          chns_precision prec, void* stream);
/* The same for the constant-coefficient operator sa (q, p) + sb (grad q, grad p), sa > 0, sb >= 0
 * (the inner operator H of the CH Schur-complement preconditioner): no coefficient, the coarsest
 * inverse without the 1 1^T term. A setup with the sa, sb and precision of the last one returns
 * at once. The Poisson and the shifted setups are kept side by side. */
chns_status chns_mg_setup_shifted(chns_mg* mg, const chns_params* prm, double sa, double sb,
                                  chns_precision prec, void* stream);
typedef enum { CHNS_MG_POISSON = 0, CHNS_MG_SHIFTED = 1 } chns_mg_operator;
/* lmax[n_levels] of the last setup of operator op in precision prec (the coarsest level's entry
 * is 0) */
chns_status chns_mg_lambda(const chns_mg* mg, int32_t op, chns_precision prec, double* lmax);
/* z = B r, one V-cycle of operator op (chns_mg_operator; device arrays of n_nodes of level 0 in
 * precision prec; r and z must not alias). Asynchronous; no allocation and no host
 * synchronisation. */
chns_status chns_mg_vcycle(chns_mg* mg, int32_t op, const void* r, void* z, chns_precision prec,
                           void* stream);
/* x_fine = P_level x_coarse and x_coarse = R_level x_fine between levels `level` and level + 1
 * (FP64 device arrays) */
chns_status chns_mg_prolong(const chns_mg* mg, int32_t level, const double* x_coarse,
                            double* x_fine, void* stream);
chns_status chns_mg_restrict(const chns_mg* mg, int32_t level, const double* x_fine,
                             double* x_coarse, void* stream);
/* phi~ of a level after an FP64 setup (FP64 device array of that level's n_nodes) */
chns_status chns_mg_coefficient(const chns_mg* mg, int32_t level, double* phi, void* stream);

/* ---------------------------------------------------------------- learned preconditioner
 * Not in the paper: a coarse correction for the pressure-Poisson solve, computed by a small
 * 3D convolutional network on a uniform D^3 grid of cells over the domain and applied inside
 * flexible CG, followed by one damped Jacobi step (CHNS_KSP_FCG + CHNS_PC_LEARNED):
 *     c(r) = s(r) out_scale P_g net(x(r)),   z = c + omega D^-1 (r - A c).
 * Grid transfer: P_g (n_nodes x D^3) interpolates cell-centred values trilinearly at the
 *   nodes; cell (i, j, k) has its centre at ((i + 1/2)/D, (j + 1/2)/D, (k + 1/2)/D) of the box,
 *   values beyond the outermost centres are extrapolated as constants. R = P_g^T restricts.
 * Input x(r), 2 channels: R r / s(r) with s(r) = sqrt(r.r / D^3); and the cell mean
 *   (P_g^T f) / (P_g^T 1) of f = log(1/rho(clamp(phi~, -1, 1))) (0 in cells no node reaches).
 * Network (16 channels, 4 levels): enc0 = relu(conv3(x)) at D; enc_l = relu(conv3(pool(
 *   enc_{l-1}))) at D/2^l for l = 1..3; dec_l = relu(conv3(up(dec_{l+1}) + enc_l)) for
 *   l = 2, 1, 0 with dec_3 = enc_3; out = conv1(dec_0), one channel, linear. conv3: 3x3x3 taps,
 *   zero padding, bias; pool: mean of 2x2x2 cells; up: copy to the 8 children. Activations and
 *   conv weights are bfloat16 with FP32 accumulation (tensor cores); master weights, gradients
 *   and the Adam state are FP32.
 * Parameters: one FP32 vector, for each layer enc0, enc1, enc2, enc3, dec2, dec1, dec0 the
 *   weights W[27][16][cin] (tap t = 9 (dz+1) + 3 (dy+1) + (dx+1), the tap reads the input at
 *   offset (dx, dy, dz); output channel; input channel; cin = 2 for enc0, else 16) then its
 *   bias[16]; then out.W[16] and out.b[1].
 * Training: on pairs (x(r), e) of mean-free error samples e with r = A e, the relative energy
 *   norm of the error the correction leaves, loss = (e - c(r))^T A (e - c(r)) / (e^T A e), with
 *   A applied in FP32 with bfloat16 coefficients; where a pair's loss exceeds 1 its gradient is
 *   divided by the loss (the gradient of log(loss)); Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Grid arrays are FP32 device arrays indexed (channel, z, y, x), x fastest. The object owns its
 * device memory (activations, gradients, replay buffer of `capacity` pairs) and may be used
 * with any mesh. Calls are asynchronous on `stream` except those returning host values. */
/* D: power of two, 8..256. Initial parameters: He-normal conv weights drawn from `seed`, zero
 * biases, zero output layer (the untrained correction is c = 0). */
chns_status chns_learned_create(int32_t D, int32_t capacity, uint64_t seed, void* stream,
                                chns_learned** out);
void chns_learned_destroy(chns_learned* net);
int64_t chns_learned_num_params(const chns_learned* net);
/* host FP32 vectors of chns_learned_num_params values; set also clears the Adam state */
chns_status chns_learned_get_params(const chns_learned* net, float* params);
chns_status chns_learned_set_params(chns_learned* net, const float* params);
chns_status chns_learned_set_output_scale(chns_learned* net, double out_scale);  /* > 0 */
double chns_learned_output_scale(const chns_learned* net);
/* out (D^3, device) = net(x) for x (2 D^3, device); keeps the activations for backward */
chns_status chns_learned_forward(chns_learned* net, const float* x, float* out, void* stream);
/* grad (num_params, device FP32) of a loss whose derivative with respect to the output of the
 * last forward is gout (D^3, device) */
chns_status chns_learned_backward(chns_learned* net, const float* gout, float* grad,
                                  void* stream);
/* one Adam step with the gradient grad (device) and learning rate lr */
chns_status chns_learned_adam(chns_learned* net, const float* grad, double lr, void* stream);
/* x (2 D^3, device) = x(r) for a nodal residual r (FP64 device); s_host = s(r) */
chns_status chns_learned_inputs(chns_learned* net, const chns_mesh* mesh, const chns_params* prm,
                                const chns_coef* coef, const double* r, float* x,
                                double* s_host, void* stream);
/* y (n_nodes, FP64 device) = P_g grid for grid (D^3, device) */
chns_status chns_learned_prolong(chns_learned* net, const chns_mesh* mesh, const float* grid,
                                 double* y, void* stream);
/* Add the training pair of the error sample e (FP64 device, n_nodes) of the Poisson operator
 * with coefficients coef: e is first projected to nodal mean zero (constants are the operator's
 * null space), then r = A e; the pair keeps x(r), e (FP32), 1 + phi~ (bfloat16), s(r), e^T A e
 * and the grid target cell_mean(e) / s(r) (its RMS sets the default output scale). The replay
 * buffer is a ring: beyond `capacity` pairs the oldest is replaced. Its nodal part is sized by
 * the first mesh; pairs of another mesh are rejected (CHNS_EINVAL). A sample with r = 0 adds
 * nothing. */
chns_status chns_learned_add_sample(chns_learned* net, const chns_mesh* mesh,
                                    const chns_params* prm, const chns_coef* coef,
                                    const double* e, void* stream);
/* Solve A x = b in FP64 from zero to relative residual 1e-10 and add the pairs of the iterate
 * errors x* - x_k, k = every, 2 every, ... (at most max_samples); *added = count. The iterates
 * are those of Jacobi-PCG, or with with_net != 0 those of FCG with the network's own correction
 * (the residuals the trained preconditioner meets; if it stalls, Jacobi-PCG finishes x*). */
chns_status chns_learned_collect(chns_learned* net, const chns_mesh* mesh, const chns_params* prm,
                                 const chns_coef* coef, const double* b, int32_t every,
                                 int32_t max_samples, int32_t with_net, int32_t* added,
                                 void* stream);
int32_t chns_learned_num_samples(const chns_learned* net);
/* `iterations` Adam steps on pairs drawn from the replay buffer (sample k of step i chosen by a
 * hash of (seed, i)); mesh and prm are those of the pairs (the Poisson operator of the loss);
 * loss_host (optional, `iterations` floats) receives each step's loss. If the output scale was
 * never set, it is first set to the RMS of the stored grid targets. */
chns_status chns_learned_train(chns_learned* net, const chns_mesh* mesh, const chns_params* prm,
                               int32_t iterations, double lr, uint64_t seed, float* loss_host,
                               void* stream);

/* ------------------------------------------------------------------ adaptive remeshing
 * One remesh changes every leaf by one level at most and moves the fields from the current mesh
 * to the new one (Sec. 5.4, "Traversal-based Intergrid Transfers"); the interface band is
 * |phi| <= threshold (0.95 in the scaling runs, Sec. 7). */

/* Band flags of the leaves (int8, device, n_elem, Morton order): the smallest |phi_h| over the
 * leaf's 8 corners (hanging corners interpolated) and its centre (the mean of the corners) is
 * <= threshold: +1 (refine) if the leaf's level is below lmax, else 0; otherwise -1 (coarsening
 * candidate) if the level is above lmin, else 0. phi: FP64 device, n_nodes.
 * CHNS_EINVAL for null pointers, 0 <= lmin <= lmax < CHNS_MAXD violated or a non-finite
 * threshold. */
chns_status chns_remesh_flags(const chns_mesh* mesh, const double* phi, double threshold,
                              int32_t lmin, int32_t lmax, int8_t* flags, void* stream);
/* The leaves of a mesh (host buffers of 3 n_elem anchors and n_elem levels, Morton order). */
chns_status chns_mesh_leaves(const chns_mesh* mesh, uint32_t* anchors, uint8_t* levels);
/* A new mesh from the band flags of phi (chns_remesh_flags): +1 leaves are split into their 8
 * children, the 8 children of one parent that are all leaves and all -1 are merged into it, and
 * the list is completed to the coarsest 2:1-balanced octree that refines it (balancing only
 * splits). *out is a new mesh on the same device and extent, owned by the caller
 * (chns_mesh_destroy); the source mesh is unchanged. Errors as chns_remesh_flags and
 * chns_mesh_create. */
chns_status chns_mesh_remesh(const chns_mesh* mesh, const double* phi, double threshold,
                             int32_t lmin, int32_t lmax, void* stream, chns_mesh** out);
/* Intergrid transfer: dst[f][j] = the finite-element function src[f] of `from` (hanging
 * corners through their constraints) evaluated at node j of `to`, for f < n_fields (1..16).
 * src[f]: FP64 device, from's n_nodes; dst[f]: FP64 device, to's n_nodes, written. On leaves
 * both meshes share this copies the values, on leaves refined in `to` it interpolates the
 * parent's shape functions at the child nodes, on leaves coarsened in `to` it injects the
 * values at the parent's corners. The meshes must cover the same cube on the same device.
 * A temporary of 8 bytes per leaf of `from` is allocated and freed on the stream. */
chns_status chns_transfer(const chns_mesh* from, const chns_mesh* to, int32_t n_fields,
                          const double* const* src, double* const* dst, void* stream);

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
