// chns_phi_mass_noalloc: the phi mass integral computed without any allocation by the library
// during the call. Its per-block partial sums and the finishing ticket live in file-scope
// __device__ arrays of a fixed size instead of the mesh workspace, and the result is written to
// a device double the caller provides. See include/chns.h for the contract.
#include <mutex>

#include "elem.cuh"
#include "reduce.cuh"

namespace chns {
namespace {

constexpr int kNaThreads = 128;
constexpr int64_t kNaMaxBlocks = 65536;  // at most kNaMaxBlocks * kNaThreads elements
constexpr int kNaMaxDevices = 64;

// Scratch of every call on a device (held by every device that loads the library until exit).
static __device__ __align__(256) double g_na_partials[kNaMaxBlocks];
static __device__ __align__(256) unsigned int g_na_ticket[1];

// Device addresses of the arrays above, looked up once per device (host code may not use the
// symbols themselves as device pointers).
struct NaDev {
  double* partials = nullptr;
  unsigned int* ticket = nullptr;
  bool ready = false;
};
NaDev g_na_dev[kNaMaxDevices];
std::mutex g_na_mutex;

chns_status na_setup(int dev, NaDev** out) {
  CHNS_CHECK(dev >= 0 && dev < kNaMaxDevices, CHNS_EINVAL, "chns_phi_mass_noalloc: device index");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  NaDev& d = g_na_dev[dev];
  if (!d.ready) {
    CHNS_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&d.partials), g_na_partials));
    CHNS_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&d.ticket), g_na_ticket));
    d.ready = true;
  }
  *out = &d;
  return CHNS_OK;
}

// Same quadrature as the phi mass of rhs.cu: sum_e detJ sum_a phi_a, then a fixed-order sum of
// the block partials by the last block.
__global__ void __launch_bounds__(kNaThreads)
k_phi_mass_na(MeshDev m, const double* __restrict__ phi, double* __restrict__ partials,
              unsigned int* __restrict__ ticket, double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (e < m.n_elem) {
    int idx[8];
    load_corners(m, e, idx);
    const Geo<double> g = geometry<double>(m, e);
    double pe[8];
    gather<double, false>(m, idx, phi, pe);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) s += pe[a];
    v[0] = g.detJ * s;
  }
  block_reduce_finalize<1, kNaThreads>(v, partials, 0, ticket, out);
}

}  // namespace
}  // namespace chns

extern "C" chns_status chns_phi_mass_noalloc(const chns_mesh* m, const double* phi,
                                             double* out, void* stream) {
  using namespace chns;
  CHNS_CHECK(m && phi && out, CHNS_EINVAL, "chns_phi_mass_noalloc: null argument");
  const int64_t nb = (m->d.n_elem + kNaThreads - 1) / kNaThreads;
  CHNS_CHECK(nb <= kNaMaxBlocks, CHNS_EINVAL,
             "chns_phi_mass_noalloc: mesh larger than the fixed scratch allows "
             "(at most 8388608 elements)");
  int dev = 0;
  CHNS_CUDA(cudaGetDevice(&dev));
  // the mesh tables live on the device that was current at chns_mesh_create; the scratch array
  // is looked up on the current one, so both must be the same GPU
  CHNS_CHECK(dev == m->device, CHNS_EINVAL,
             "chns_phi_mass_noalloc: the current device is not the mesh's device");
  NaDev* d = nullptr;
  chns_status st = na_setup(dev, &d);
  if (st != CHNS_OK) return st;
  cudaStream_t s = as_stream(stream);
  // the ticket must start at zero (a call that never finished could have left it set)
  CHNS_CUDA(cudaMemsetAsync(d->ticket, 0, sizeof(unsigned int), s));
  note_launch();
  k_phi_mass_na<<<(unsigned)nb, kNaThreads, 0, s>>>(m->d, phi, d->partials, d->ticket, out);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}
