// Internal declarations of the geometric multigrid hierarchy (multigrid.cu).
#pragma once

#include <vector>

#include "internal.h"

namespace chns {

constexpr int kMgVecs = 4;        // per level: right-hand side, correction, apply output, direction
constexpr int kMgMaxLevels = 32;
// level operators a hierarchy can be set up for (each keeps its own diagonals, intervals and
// coarsest inverse, so that both can be live at once)
constexpr int kMgPoisson = 0;     // (grad q, (1/rho(phi~*)) grad p), pure Neumann
constexpr int kMgShifted = 1;     // sa (q, p) + sb (grad q, grad p), constant sa > 0, sb >= 0
constexpr int kMgOps = 2;

// per level and operator: coefficients (Poisson), inverse diagonal and Chebyshev interval, per
// precision (index 0 FP64, 1 FP32)
struct MgOpLevel {
  double* phi64 = nullptr;
  float* phi32 = nullptr;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  double lmax[2] = {0.0, 0.0}, lmin[2] = {0.0, 0.0};
};

struct MgLevel {
  chns_mesh* mesh = nullptr;  // level 0: the caller's mesh (not owned)
  int64_t n = 0;              // nodes
  // transfer between this level and the next coarser one (absent on the coarsest level):
  // P (rows by node of this level), R = P^T (rows by node of the coarser level), injection
  // (coarser node -> node of this level at the same point)
  int32_t* p_ptr = nullptr;
  int32_t* p_col = nullptr;
  float* p_w = nullptr;
  int32_t* r_ptr = nullptr;
  int32_t* r_col = nullptr;
  float* r_w = nullptr;
  int32_t* inj = nullptr;
  int64_t p_nnz = 0;
  // work vectors [kMgVecs] per precision (level 0 holds only vectors 2 and 3)
  double* v64[kMgVecs] = {};
  float* v32[kMgVecs] = {};
  MgOpLevel op[kMgOps];
};

// state of one level operator over the hierarchy
struct MgOpState {
  const void* phi0_64 = nullptr;  // Poisson: fine-level coefficients of the last setup
  const void* phi0_32 = nullptr;
  double sa = 0.0, sb = 0.0;      // shifted operator
  double* cinv64 = nullptr;       // dense inverse of the coarsest operator
  float* cinv32 = nullptr;
  bool ready[2] = {false, false};  // set up in FP64 / FP32
};

}  // namespace chns

struct chns_mg {
  std::vector<chns::MgLevel> lv;
  chns_mg_params prm;
  chns_params phys{};
  chns::MgOpState ops[chns::kMgOps];
  double* cwork64 = nullptr;  // FP64 work matrix of the FP32 setups
  double* slots = nullptr;    // power-iteration norms [kMgMaxLevels]
  double* h_slots = nullptr;  // pinned host copy
};

namespace chns {

chns_status mg_create(const chns_mesh* fine, const chns_mg_params* prm, cudaStream_t s,
                      chns_mg** out);
void mg_free(chns_mg* g);
// Level operators for the coefficient phi~ of the fine mesh (FP64 or FP32 device array, which
// must stay valid while V-cycles of this precision run): injection, diagonals, Chebyshev
// intervals, coarsest inverse. Synchronises the stream once.
chns_status mg_setup(chns_mg* g, const chns_params* prm, const void* phi0, chns_precision prec,
                     cudaStream_t s);
// Level operators sa M + sb K (constant coefficients, sa > 0); a repeated setup with the same
// sa, sb and precision returns at once.
chns_status mg_setup_shifted(chns_mg* g, const chns_params* prm, double sa, double sb,
                             chns_precision prec, cudaStream_t s);
// z = B r, one V-cycle of operator op (kernels only: no allocation, no host synchronisation)
template <class T>
chns_status mg_vcycle(chns_mg* g, int op, const T* r, T* z, cudaStream_t s);

}  // namespace chns
