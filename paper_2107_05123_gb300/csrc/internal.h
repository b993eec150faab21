// Internal declarations of the CHNS library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/chns.h"

namespace chns {

// Element corner indices carry the Dirichlet flag in bit 30; bit 31 is never set.
constexpr int32_t kDirBit = 1 << 30;
constexpr int32_t kIdxMask = kDirBit - 1;
// Patch slot entries: node id (< 2^29) | kOwnBit (only this patch touches the node) | kDirBit.
constexpr int32_t kOwnBit = 1 << 29;
constexpr int32_t kNodeMask = kOwnBit - 1;
// A patch is a run of Morton-consecutive elements processed by one CTA (one thread per element)
// whose distinct nodes (regular nodes and hanging corners) fit in kPatchSlots shared slots.
constexpr int kPatchElems = 256;
constexpr int kPatchSlots = 640;
// Per element of a patch, eloc holds its 8 corner slots as uint16; slots are < kPatchSlots, so the
// first entry also carries the element's level in bits 10-14.
constexpr uint32_t kElocSlotMask = 0x3ff;
constexpr int kElocLevelShift = 10;
constexpr uint32_t kElocLevelMask = 0x1f;
// The persistent, pipelined apply is chosen automatically once the mesh has at least this many
// patches per SM.
constexpr int kStreamMinPatchesPerSm = 16;

// Element geometry of one octant level on the box [0,L]^3 scaled per axis: h_d = L_d 2^-level,
// 1/h_d and det J = h_x h_y h_z / 8, in FP64 and FP32 (looked up, never recomputed per element).
struct LevelGeo {
  double h[3], ih[3], detJ;
  float hf[3], ihf[3], detJf;
};

// Device view of the mesh tables (passed by value to kernels).
struct MeshDev {
  int64_t n_elem;
  int64_t n_nodes;
  int64_t n_hang;
  const int4* enode;     // [n_elem][2] int4 = 8 corner indices: < n_nodes node, else hanging
  const uint8_t* level;  // [n_elem]
  const int4* hang;      // [n_hang] parents (with Dirichlet bit); .z=.w=-1 for edge midpoints
  const uint32_t* anchor;  // [n_elem*3] (only for diagnostics needing positions)
  double ext[3];         // physical extent
  // patch tables
  int64_t n_patch;
  const int32_t* patch_elem;  // [n_patch+1] first element of each patch
  const int32_t* patch_slot;  // [n_patch+1] first slot of each patch (regular slots, then hanging)
  const int32_t* patch_nreg;  // [n_patch] regular slots of each patch
  const int32_t* slot_node;   // [slots] regular slot: node id | kOwnBit | kDirBit
  const ushort4* slot_par;    // [slots] hanging slot: local parent slots (0xffff = none)
  const uint4* eloc;          // [n_elem] 8 local slot indices (uint16) per element + level
  const LevelGeo* geo;        // [CHNS_MAXD] per-level geometry
};

struct Workspace {
  // FP64 vectors (sized for 3 components) and FP32 mirrors
  std::vector<double*> v64;
  std::vector<float*> v32;
  double* gm_V = nullptr;      // GMRES basis (restart+1) x (3N) doubles
  float* gm_V32 = nullptr;     // FP32 GMRES basis
  double* red = nullptr;       // reduction partials + scalars
  unsigned int* counter = nullptr;
  double* h_pinned = nullptr;  // pinned host scalars
  void* coef32 = nullptr;      // reduced-precision coefficient copies (5 fields, float)
  void* coef16 = nullptr;      // bf16 copies (5 fields)
  double* coef64 = nullptr;    // FP64 step coefficients (phi~, u_hat x3, mu~ + scratch)
  double* part_big = nullptr;  // per-block partials of element-level reductions (n_elem/64+64)
  double* md_part = nullptr;   // GMRES multi-dot partials: [restart + 2][kMdMaxBlocks]
};

}  // namespace chns

struct chns_mesh {
  chns::MeshDev d;
  int min_level = 0, max_level = 0;
  int64_t n_boundary = 0;
  std::vector<uint32_t> node_coords;  // host copy, 3*n_nodes
  std::vector<uint8_t> node_bnd;      // host copy
  // host copies of the element corner and hanging tables (kept for multigrid level meshes)
  std::vector<int32_t> h_enode;
  std::vector<int4> h_hang;
  // device allocations
  int4* d_enode = nullptr;
  uint8_t* d_level = nullptr;
  int4* d_hang = nullptr;
  uint32_t* d_anchor = nullptr;
  int32_t* d_bnd = nullptr;          // boundary node indices (n_boundary)
  int32_t* d_patch_elem = nullptr;
  int32_t* d_patch_slot = nullptr;
  int32_t* d_patch_nreg = nullptr;
  int32_t* d_slot_node = nullptr;
  ushort4* d_slot_par = nullptr;
  uint4* d_eloc = nullptr;
  chns::LevelGeo* d_geo = nullptr;
  uint32_t* d_node_int = nullptr;    // node coordinates (3*n_nodes, units 2^-CHNS_MAXD)
  int64_t n_slots = 0;
  chns::Workspace ws;
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture CUDA graphs
  // quadrature data of the momentum operator during a momentum solve (see momentum_qdata_on)
  struct MomQState {
    void* qd64 = nullptr;
    void* qd32 = nullptr;
    bool on = false, has32 = false;
  };
  mutable MomQState mq;
  // inverse diagonals of the Schur preconditioner's M and H (constant coefficients: they depend
  // on the mesh and on sa, sb only), kept between solves; key = (sa_M, sb_M, sa_H, sb_H)
  struct SchurDiag {
    void* d[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [FP64, FP32][M, H]
    double key[2][4] = {};
    bool valid[2] = {false, false};
  };
  mutable SchurDiag sd;
  mutable double* qvu = nullptr;  // per-point velocity-update terms shared by the step's PP/VU
  int red_blocks = 0;
  int sm_count = 0;
  int device = 0;  // CUDA device current at chns_mesh_create (holds every device table)
  // launch configuration of the operator applies (chns_mesh_set_apply_config)
  chns_apply_kernel apply_kernel = CHNS_APPLY_AUTO;
  int64_t apply_max_ctas = 0;
};

namespace chns {

void set_error(const std::string& msg);
// Mesh construction (mesh.cu). light: no solver workspace (level meshes of a multigrid
// hierarchy, which are only applied); keep_host: keep host copies of the element and hanging
// tables. free_mesh releases a mesh built by build_mesh (also after a failed build).
chns_status build_mesh(const uint32_t* anchors, const uint8_t* levels, int64_t n,
                       const double extent[3], cudaStream_t stream, chns_mesh* m, bool light,
                       bool keep_host);
void free_mesh(chns_mesh* m);
// count of kernel launches issued by the library (diagnostic); graph launches add the number of
// kernels they contain, and launches recorded during a stream capture are taken back out
void note_launch();
void note_launches(unsigned long long k);
void note_launches_undo(unsigned long long k);
unsigned long long chns_launches_now();
chns_status cuda_fail(cudaError_t e, const char* what);

#define CHNS_CUDA(call)                                          \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return ::chns::cuda_fail(_e, #call);  \
  } while (0)

#define CHNS_CHECK(cond, code, msg)      \
  do {                                   \
    if (!(cond)) {                       \
      ::chns::set_error(msg);            \
      return code;                       \
    }                                    \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Number of FP64 workspace vectors of 3*n_nodes
constexpr int kNumVec64 = 16;
constexpr int kNumVec32 = 10;
constexpr int kRedSlots = 4096;   // partial sums per reduction
constexpr int kMdMaxBlocks = 1024; // blocks of the GMRES multi-dot
constexpr int kScalarBase = 3 * 4096;  // scalars stored after three partial arrays

// ---- apply dispatch (apply.cu)
chns_status apply_op(const chns_mesh* m, chns_operator op, const chns_params* prm,
                     const chns_coef* coef, const void* x, void* y, chns_precision prec,
                     cudaStream_t s);
// Slots of the CG scalars (offsets from the scalar area of ws.red). Iteration k (parity
// par = k & 1) reads r.z of its iterate from kCgRz0 + par and that of the previous one from
// kCgRzPrev, accumulates p.Ap into kCgPq0 + par, and accumulates the next r.z and r.r into
// kCgRz0 + (par ^ 1) and kCgRr0 + (par ^ 1). Block partials are added with FP64 atomics into
// slots that the previous kernel of the iteration cleared (a kernel boundary orders them), so no
// kernel waits for the last block of its grid.
constexpr int kCgRz0 = 32, kCgRzPrev = 34, kCgPq0 = 35, kCgRr0 = 37;
// flexible CG: iteration k reads r.z of its iterate from kFcgRz0 + par, alpha from kFcgAlpha;
// it accumulates z_new.q into kFcgZq0 + par and r_new.z_new into kFcgRz0 + (par ^ 1), and the
// next apply forms beta = -alpha z_new.q / r.z (Polak-Ribiere).
constexpr int kFcgAlpha = 5, kFcgZq0 = 40, kFcgRz0 = 42;
// One fused CG step of the Poisson operator (iteration parity par): p_new = z + beta p_old with
// beta = S[kCgRz0 + par] / S[kCgRzPrev] (fcg: -S[kFcgAlpha] S[kFcgZq0 + (par ^ 1)] /
// S[kFcgRz0 + (par ^ 1)]) during the gather, y = A p_new (y zero on entry), and
// S[kCgPq0 + par] += p_new.A p_new (cleared by the caller); clears S[kCgRz0 + (par ^ 1)] and
// S[kCgRr0 + (par ^ 1)] for the update kernel that follows.
chns_status apply_poisson_cg(const chns_mesh* m, const chns_params* prm, const chns_coef* coef,
                             const void* z, const void* p_old, void* p_new, void* y,
                             chns_precision prec, double* S_cg, int par, cudaStream_t s,
                             bool fcg = false);
// Precompute the momentum operator's quadrature data for coefficients that stay fixed over the
// applies that follow (a Krylov solve); momentum_qdata_off returns to on-the-fly evaluation.
chns_status momentum_qdata_on(const chns_mesh* m, const chns_params* prm, const chns_coef* coef64,
                              const chns_coef* coef32, cudaStream_t s);
void momentum_qdata_off(const chns_mesh* m);
// y = sa M x + sb K x (shifted Laplacian, constant sa, sb) and its exact diagonal; phi is any
// coefficient array of the precision (FP64 or FP32), read but unused.
chns_status apply_shift(const chns_mesh* m, const chns_params* prm, const void* phi, double sa,
                        double sb, const void* x, void* y, chns_precision prec, cudaStream_t s);
chns_status diag_shift(const chns_mesh* m, const chns_params* prm, const void* phi, double sa,
                       double sb, void* d, chns_precision prec, cudaStream_t s);
chns_status diag_op(const chns_mesh* m, chns_operator op, const chns_params* prm,
                    const chns_coef* coef, void* d, chns_precision prec, cudaStream_t s);
// 2x2 nodal blocks of the CH Jacobian, d4 = [d_pp, d_pm, d_mp, d_mm] x n_nodes (FP64 or FP32)
chns_status block_diag_ch(const chns_mesh* m, const chns_params* prm, const chns_coef* coef,
                          void* d4, chns_precision prec, cudaStream_t s);
// y = A x for MASS or MOMENTUM in FP64 without the Dirichlet treatment (boundary rows and columns
// kept), for lifting Dirichlet data into right-hand sides; y is overwritten.
chns_status apply_op_full(const chns_mesh* m, chns_operator op, const chns_params* prm,
                          const chns_coef* coef, const double* x, double* y, cudaStream_t s);
// y[c N + j] = x[c N + j] for every boundary node j and component c < nc (FP64)
chns_status dirichlet_set(const chns_mesh* m, int nc, const double* x, double* y, cudaStream_t s);
int op_ncomp(chns_operator op);
bool op_dirichlet(chns_operator op);
// internal operator code of the Krylov context: y = sa M x + sb K x (apply_shift)
constexpr chns_operator kOpShift = static_cast<chns_operator>(100);

// ---- vector kernels (krylov.cu)
void vec_convert_f64_f32(const double* a, float* b, int64_t n, cudaStream_t s);
// b = bfloat16(a + offset)
void vec_convert_f64_bf16(const double* a, __nv_bfloat16* b, int64_t n, double offset,
                          cudaStream_t s);
void vec_axpby(double a, const double* x, double b, const double* y, double* out, int64_t n,
               cudaStream_t s);
void vec_copy(const double* x, double* y, int64_t n, cudaStream_t s);
void vec_zero(double* x, int64_t n, cudaStream_t s);
// FP64 dot on device; result written to dst (device) as double
void dot_dev(const chns_mesh* m, const double* a, const double* b, int64_t n, double* dst,
             cudaStream_t s);
chns_status dot_host(const chns_mesh* m, const double* a, const double* b, int64_t n, double* out,
                     cudaStream_t s);
chns_status sum_host(const chns_mesh* m, const double* a, int64_t n, double* out, cudaStream_t s);
void vec_add_scalar(double* x, const double* dev_scalar, double factor, int64_t n, cudaStream_t s);

// ---- right-hand sides (rhs.cu)
chns_status phi_mass(const chns_mesh* m, const double* phi, double* out, cudaStream_t s);
chns_status residual_ch(const chns_mesh* m, const chns_params* prm, const double* phi,
                        const double* mu, const double* phik, const double* muk,
                        const double* const u[3], double* f, cudaStream_t s);
chns_status rhs_momentum(const chns_mesh* m, const chns_params* prm, const chns_coef* c,
                         const double* const uk[3], const double* pk, double* b, cudaStream_t s);
// qvu (optional, 24 n_elem doubles): also store the velocity update's per-point terms
chns_status rhs_poisson(const chns_mesh* m, const chns_params* prm, const chns_coef* c,
                        const double* const v[3], const double* const uk[3], const double* pk,
                        double* b, cudaStream_t s, double* qvu = nullptr);
// the velocity-update right-hand side from the terms rhs_poisson stored in qvu
chns_status rhs_vu_from(const chns_mesh* m, const chns_params* prm, const double* qvu,
                        const double* pk, const double* pn, double* b, cudaStream_t s);
chns_status rhs_vu(const chns_mesh* m, const chns_params* prm, const chns_coef* c,
                   const double* const v[3], const double* const uk[3], const double* pk,
                   const double* pn, double* b, cudaStream_t s);

// ---- Krylov (krylov.cu)
chns_status krylov_solve(const chns_mesh* m, chns_operator op, const chns_params* prm,
                         const chns_coef* coef, const double* b, double* x,
                         const chns_solver_params* sp, chns_solve_stats* stats, cudaStream_t s);

// ---- learned preconditioner (learned.cu)
// density channel of the input for the coefficients of this solve
chns_status learned_begin_solve(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                                const chns_coef* coef64, cudaStream_t s);
// z = (dinv ? dinv r : 0) + s(r) out_scale P_g net(x(r)), with r.r read from rr_dev (device);
// asynchronous, no allocation or host synchronisation (capturable in a CUDA graph)
template <class T>
chns_status learned_precondition(chns_learned* L, const chns_mesh* m, const T* r, const T* dinv,
                                 const double* rr_dev, T* z, cudaStream_t s);
chns_status learned_add_sample(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                               const chns_coef* coef, const double* e, cudaStream_t s);
chns_status learned_collect(chns_learned* L, const chns_mesh* m, const chns_params* prm,
                            const chns_coef* coef, const double* b, int every, int max_samples,
                            bool with_net, int* added, cudaStream_t s);
// FP64 Jacobi-PCG of the Poisson operator from x = 0 to ||r|| <= rtol ||b|| (b mean-projected),
// copying the iterates k = every, 2 every, ... (at most max_snaps) to snaps [max_snaps][n_nodes]
// (krylov.cu); x is returned mean-free. With L the iterates are those of FCG with the network's
// correction (Jacobi-PCG finishes the solve if it stalls).
chns_status pcg_snapshots(const chns_mesh* m, const chns_params* prm, const chns_coef* coef,
                          const double* b, double rtol, int every, int max_snaps, double* snaps,
                          int* n_snaps, double* x, cudaStream_t s, chns_learned* L = nullptr);

}  // namespace chns
