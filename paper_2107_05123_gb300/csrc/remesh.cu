// Adaptive remeshing and intergrid transfer (Sec. 5.4, "Traversal-based Intergrid Transfers";
// the interface band |phi| <= 0.95 of the scaling runs, Sec. 7).
//
//  * band flags, on the GPU: a leaf is in the band when the smallest |phi_h| over its 8 corners
//    (hanging corners through their constraints) and its centre (the mean of the corners) is at
//    most the threshold; it is flagged +1 (refine) in the band below lmax, -1 (coarsening
//    candidate) outside it above lmin, else 0;
//  * new leaves, on the host: +1 leaves split into their 8 children, 8 sibling leaves that are
//    all -1 merge into their parent (one level of change per remesh), then the coarsest 2:1
//    balanced refinement of that list is formed level by level, from the finest split octants to
//    the root: every octant that has children needs its 26 same-size neighbours to exist, i.e.
//    their parents to have children too;
//  * transfer, on the GPU: every node of the new mesh takes the finite-element value of the old
//    mesh at its position. The old leaf holding the point is found by binary search over the
//    Morton keys of the old leaves (a complete octree covers consecutive key ranges), and its
//    trilinear interpolant is evaluated there with the hanging corners interpolated. This is
//    the copy, child interpolation and parent injection of the three cases of Sec. 5.4.
#include <algorithm>
#include <cmath>
#include <new>

#include "elem.cuh"
#include "hostutil.h"

namespace chns {
namespace {

constexpr int kRemeshThreads = 256;
constexpr int kMaxTransferFields = 16;

__global__ void k_remesh_flags(MeshDev m, const double* __restrict__ phi, double thr, int lmin,
                               int lmax, int8_t* __restrict__ fl) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  int idx[8];
  load_corners(m, e, idx);
  double v[8];
  gather<double, false>(m, idx, phi, v);
  double mn = fabs(v[0]);
#pragma unroll
  for (int a = 1; a < 8; ++a) mn = fmin(mn, fabs(v[a]));
  const double c = (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) * 0.125;
  mn = fmin(mn, fabs(c));
  const int lev = m.level[e];
  int8_t f = 0;
  if (mn <= thr) {
    if (lev < lmax) f = 1;
  } else if (lev > lmin) {
    f = -1;
  }
  fl[e] = f;
}

__device__ __forceinline__ uint64_t d_spread3(uint64_t v) {
  v &= 0x1FFFFFull;
  v = (v | (v << 32)) & 0x1F00000000FFFFull;
  v = (v | (v << 16)) & 0x1F0000FF0000FFull;
  v = (v | (v << 8)) & 0x100F00F00F00F00Full;
  v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}
__device__ __forceinline__ uint64_t d_morton(uint32_t x, uint32_t y, uint32_t z) {
  return d_spread3(x) | (d_spread3(y) << 1) | (d_spread3(z) << 2);
}

__global__ void k_leaf_keys(MeshDev m, uint64_t* __restrict__ key) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  key[e] = d_morton(m.anchor[3 * e], m.anchor[3 * e + 1], m.anchor[3 * e + 2]);
}

struct TransferPtrs {
  const double* src[kMaxTransferFields];
  double* dst[kMaxTransferFields];
};

__global__ void k_transfer(MeshDev a, const uint64_t* __restrict__ akey,
                           const uint32_t* __restrict__ node_b, int64_t nb, int nf,
                           TransferPtrs ptr) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const uint32_t full = 1u << CHNS_MAXD;
  uint32_t p[3], q[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    p[d] = node_b[3 * j + d];
    q[d] = p[d] < full ? p[d] : full - 1;  // a point on the upper faces: the leaf below it
  }
  const uint64_t k = d_morton(q[0], q[1], q[2]);
  // last leaf whose key is <= k
  int64_t lo = 0, hi = a.n_elem;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(akey + mid) <= k)
      lo = mid;
    else
      hi = mid;
  }
  const int64_t e = lo;
  const int lev = a.level[e];
  const double inv_s = ldexp(1.0, lev - CHNS_MAXD);  // 1 / side, exact
  double xi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    xi[d] = (double)((int64_t)p[d] - (int64_t)a.anchor[3 * e + d]) * inv_s;
  double w[8];
#pragma unroll
  for (int c = 0; c < 8; ++c)
    w[c] = ((c & 1) ? xi[0] : 1.0 - xi[0]) * (((c >> 1) & 1) ? xi[1] : 1.0 - xi[1]) *
           (((c >> 2) & 1) ? xi[2] : 1.0 - xi[2]);
  int idx[8];
  load_corners(a, e, idx);
  for (int f = 0; f < nf; ++f) {
    double v[8];
    gather<double, false>(a, idx, ptr.src[f], v);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += w[c] * v[c];
    ptr.dst[f][j] = s;
  }
}

// ---- host: new leaf list
inline uint64_t okey(const uint32_t* a, int level) {  // Morton key of an octant at its level
  const int sh = CHNS_MAXD - level;
  return host::morton(a[0] >> sh, a[1] >> sh, a[2] >> sh);
}

void sort_unique(std::vector<uint64_t>& v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
}

// split[l]: octants of level l that have children. Requirements ripple from fine to coarse:
// an octant with children needs its 26 same-level neighbours (and itself) to exist, i.e. the
// parents of all of them to have children.
void balance_and_emit(std::vector<std::vector<uint64_t>>& split, int lmax,
                      std::vector<uint32_t>& A, std::vector<uint8_t>& L) {
  for (int l = lmax - 1; l >= 1; --l) {
    sort_unique(split[l]);
    const std::vector<uint64_t>& S = split[l];
    const int64_t n = (int64_t)S.size();
    const int64_t dim = int64_t(1) << l;
    // at most 2 parents per axis: the parents of c - 1, c, c + 1
    std::vector<uint64_t> req((size_t)n * 8, UINT64_MAX);
    host::parallel_for(n, [&](int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i) {
        const int64_t c[3] = {(int64_t)host::compact3(S[i]), (int64_t)host::compact3(S[i] >> 1),
                              (int64_t)host::compact3(S[i] >> 2)};
        int64_t lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
          lo[d] = std::max<int64_t>(c[d] - 1, 0) >> 1;
          hi[d] = std::min<int64_t>(c[d] + 1, dim - 1) >> 1;
        }
        int k = 0;
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
          for (int64_t y = lo[1]; y <= hi[1]; ++y)
            for (int64_t x = lo[0]; x <= hi[0]; ++x) req[8 * i + k++] = host::morton(x, y, z);
      }
    });
    sort_unique(req);
    if (!req.empty() && req.back() == UINT64_MAX) req.pop_back();
    split[l - 1].insert(split[l - 1].end(), req.begin(), req.end());
  }
  if (lmax >= 1) sort_unique(split[0]);
  std::vector<std::pair<uint64_t, uint8_t>> leaves;
  if (split.empty() || split[0].empty()) {
    A.assign(3, 0u);
    L.assign(1, 0);
    return;
  }
  for (int l = 0; l < lmax; ++l) {
    const std::vector<uint64_t>& S = split[l];
    const std::vector<uint64_t>* nxt = l + 1 < lmax ? &split[l + 1] : nullptr;
    for (uint64_t s : S) {
      const uint64_t cx = host::compact3(s), cy = host::compact3(s >> 1), cz = host::compact3(s >> 2);
      for (int ch = 0; ch < 8; ++ch) {
        const uint64_t kx = 2 * cx + (ch & 1), ky = 2 * cy + ((ch >> 1) & 1),
                       kz = 2 * cz + ((ch >> 2) & 1);
        const uint64_t kk = host::morton(kx, ky, kz);
        if (nxt && std::binary_search(nxt->begin(), nxt->end(), kk)) continue;
        const int sh = CHNS_MAXD - (l + 1);
        leaves.emplace_back(host::morton(kx << sh, ky << sh, kz << sh), (uint8_t)(l + 1));
      }
    }
  }
  std::sort(leaves.begin(), leaves.end());
  A.resize(3 * leaves.size());
  L.resize(leaves.size());
  for (size_t i = 0; i < leaves.size(); ++i) {
    const uint64_t k = leaves[i].first;
    A[3 * i] = (uint32_t)host::compact3(k);
    A[3 * i + 1] = (uint32_t)host::compact3(k >> 1);
    A[3 * i + 2] = (uint32_t)host::compact3(k >> 2);
    L[i] = leaves[i].second;
  }
}

chns_status new_leaves(const chns_mesh* m, const int8_t* fl, std::vector<uint32_t>& A,
                       std::vector<uint8_t>& L, cudaStream_t s) {
  const int64_t n = m->d.n_elem;
  std::vector<uint32_t> an((size_t)n * 3);
  std::vector<uint8_t> lv((size_t)n);
  CHNS_CUDA(cudaMemcpyAsync(an.data(), m->d_anchor, an.size() * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, s));
  CHNS_CUDA(cudaMemcpyAsync(lv.data(), m->d_level, lv.size(), cudaMemcpyDeviceToHost, s));
  CHNS_CUDA(cudaStreamSynchronize(s));
  // split / merge, recorded as octants with children per level (a leaf of level l is a child
  // of a split octant of level l - 1)
  std::vector<std::vector<uint64_t>> split(CHNS_MAXD);
  int lmax = 0;
  auto add_leaf = [&](const uint32_t* a, int l) {
    if (l >= 1) split[l - 1].push_back(okey(a, l - 1));
    lmax = std::max(lmax, l);
  };
  for (int64_t i = 0; i < n;) {
    const int l = lv[i];
    const uint32_t* a = &an[3 * i];
    bool merge = false;
    if (l > 0 && fl[i] == -1 && i + 7 < n) {
      const uint32_t s2 = 2u << (CHNS_MAXD - l), s = s2 >> 1;
      if (a[0] % s2 == 0 && a[1] % s2 == 0 && a[2] % s2 == 0) {
        merge = true;
        for (int c = 1; c < 8 && merge; ++c) {
          const uint32_t* b = &an[3 * (i + c)];
          merge = lv[i + c] == l && fl[i + c] == -1 && b[0] == a[0] + s * (c & 1) &&
                  b[1] == a[1] + s * ((c >> 1) & 1) && b[2] == a[2] + s * ((c >> 2) & 1);
        }
      }
    }
    if (merge) {
      add_leaf(a, l - 1);
      i += 8;
      continue;
    }
    if (fl[i] == 1) {
      CHNS_CHECK(l + 1 < CHNS_MAXD, CHNS_EINVAL, "remesh: refinement beyond CHNS_MAXD - 1");
      split[l].push_back(okey(a, l));
      lmax = std::max(lmax, l + 1);
    } else {
      add_leaf(a, l);
    }
    ++i;
  }
  balance_and_emit(split, lmax, A, L);
  return CHNS_OK;
}

}  // namespace
}  // namespace chns

using namespace chns;

extern "C" chns_status chns_remesh_flags(const chns_mesh* m, const double* phi, double threshold,
                                         int32_t lmin, int32_t lmax, int8_t* flags, void* stream) {
  CHNS_CHECK(m && phi && flags, CHNS_EINVAL, "chns_remesh_flags: null argument");
  CHNS_CHECK(0 <= lmin && lmin <= lmax && lmax < CHNS_MAXD, CHNS_EINVAL,
             "chns_remesh_flags: need 0 <= lmin <= lmax < CHNS_MAXD");
  CHNS_CHECK(std::isfinite(threshold), CHNS_EINVAL, "chns_remesh_flags: threshold not finite");
  const int64_t n = m->d.n_elem;
  k_remesh_flags<<<(unsigned)((n + kRemeshThreads - 1) / kRemeshThreads), kRemeshThreads, 0,
                   as_stream(stream)>>>(m->d, phi, threshold, lmin, lmax, flags);
  note_launch();
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

extern "C" chns_status chns_mesh_leaves(const chns_mesh* m, uint32_t* anchors, uint8_t* levels) {
  CHNS_CHECK(m && anchors && levels, CHNS_EINVAL, "chns_mesh_leaves: null argument");
  const int64_t n = m->d.n_elem;
  CHNS_CUDA(cudaMemcpy(anchors, m->d_anchor, (size_t)n * 3 * sizeof(uint32_t),
                       cudaMemcpyDeviceToHost));
  CHNS_CUDA(cudaMemcpy(levels, m->d_level, (size_t)n, cudaMemcpyDeviceToHost));
  return CHNS_OK;
}

extern "C" chns_status chns_mesh_remesh(const chns_mesh* m, const double* phi, double threshold,
                                        int32_t lmin, int32_t lmax, void* stream,
                                        chns_mesh** out) {
  CHNS_CHECK(out, CHNS_EINVAL, "chns_mesh_remesh: null argument");
  *out = nullptr;
  cudaStream_t s = as_stream(stream);
  int cur = 0;
  CHNS_CHECK(m, CHNS_EINVAL, "chns_mesh_remesh: null mesh");
  CHNS_CUDA(cudaGetDevice(&cur));
  CHNS_CHECK(cur == m->device, CHNS_EINVAL, "chns_mesh_remesh: mesh built on another device");
  const int64_t n = m->d.n_elem;
  int8_t* d_fl = nullptr;
  CHNS_CUDA(cudaMalloc(&d_fl, (size_t)n));
  chns_status st = chns_remesh_flags(m, phi, threshold, lmin, lmax, d_fl, stream);
  std::vector<int8_t> fl;
  if (st == CHNS_OK) {
    fl.resize((size_t)n);
    if (cudaMemcpyAsync(fl.data(), d_fl, (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("chns_mesh_remesh: flag copy failed");
      st = CHNS_ECUDA;
    }
  }
  cudaFree(d_fl);
  if (st != CHNS_OK) return st;
  std::vector<uint32_t> A;
  std::vector<uint8_t> L;
  try {
    st = new_leaves(m, fl.data(), A, L, s);
  } catch (const std::bad_alloc&) {
    set_error("chns_mesh_remesh: out of host memory");
    return CHNS_ENOMEM;
  }
  if (st != CHNS_OK) return st;
  return chns_mesh_create(A.data(), L.data(), (int64_t)L.size(), m->d.ext, stream, out);
}

extern "C" chns_status chns_transfer(const chns_mesh* from, const chns_mesh* to, int32_t n_fields,
                                     const double* const* src, double* const* dst, void* stream) {
  CHNS_CHECK(from && to && src && dst, CHNS_EINVAL, "chns_transfer: null argument");
  CHNS_CHECK(n_fields >= 1 && n_fields <= kMaxTransferFields, CHNS_EINVAL,
             "chns_transfer: n_fields must be in [1, 16]");
  CHNS_CHECK(from->device == to->device, CHNS_EINVAL, "chns_transfer: meshes on different devices");
  TransferPtrs p{};
  for (int f = 0; f < n_fields; ++f) {
    CHNS_CHECK(src[f] && dst[f], CHNS_EINVAL, "chns_transfer: null field");
    p.src[f] = src[f];
    p.dst[f] = dst[f];
  }
  cudaStream_t s = as_stream(stream);
  const int64_t ne = from->d.n_elem, nb = to->d.n_nodes;
  uint64_t* key = nullptr;
  CHNS_CUDA(cudaMallocAsync(&key, (size_t)ne * sizeof(uint64_t), s));
  k_leaf_keys<<<(unsigned)((ne + kRemeshThreads - 1) / kRemeshThreads), kRemeshThreads, 0, s>>>(
      from->d, key);
  note_launch();
  if (nb > 0) {
    k_transfer<<<(unsigned)((nb + kRemeshThreads - 1) / kRemeshThreads), kRemeshThreads, 0, s>>>(
        from->d, key, to->d_node_int, nb, n_fields, p);
    note_launch();
  }
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaFreeAsync(key, s);
  CHNS_CUDA(e1);
  CHNS_CUDA(e2);
  return CHNS_OK;
}
