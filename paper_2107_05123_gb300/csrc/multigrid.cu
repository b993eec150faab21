// Geometric multigrid V-cycle for the pressure-Poisson operator on the octree.
//
// The paper solves the pressure Poisson system with PETSc's algebraic multigrid (App. A) and
// names a geometric multigrid on the octree as the remedy for the AMG setup cost that dominates
// its solver timings (Sec. 7, component breakdown; Conclusions). This is that method, built from
// the paper's octree operations:
//   - hierarchy: level 0 is the caller's mesh; level l+1 replaces every leaf at level l's finest
//     octant level by its parent, the one-level coarsening of the intergrid transfer (Sec. 5.4,
//     "Traversal-based Intergrid Transfers"), until the finest octant level is at most
//     `coarsest_level`. A leaf at the finest level always has its seven siblings as leaves, so
//     every level is again a complete, 2:1-balanced octree;
//   - transfers: P_l (level l+1 -> l) evaluates the coarse finite-element function, with its
//     hanging constraints, at the fine nodes (child interpolation of Sec. 5.4); R_l = P_l^T.
//     Both are CSR tables built once on the host, P by fine row and R by coarse row, so that
//     neither transfer needs atomics. Every fine node lies on the half-size lattice of the
//     coarse leaf that holds it, so the weights are dyadic and exact in FP32;
//   - level operators: the Poisson operator (grad q, (1/rho(phi~*)) grad p) of each level mesh,
//     with phi~ injected (a coarse node is always a fine node), through the same patch kernels
//     as the fine operator;
//   - smoother: `degree` Chebyshev steps on D^-1 A over [lmax / range, lmax], lmax = factor x the
//     power estimate of the largest eigenvalue of D^-1 A (`power_its` iterations from a fixed
//     integer-hash start vector), before and after the coarse correction (a symmetric cycle);
//   - coarsest level: z = (A + 1 1^T / n)^-1 r, the mean-zero solution of the pure-Neumann
//     problem, with the dense inverse formed by Gauss-Jordan elimination in FP64 on the GPU at
//     every setup.
// Setup (chns_mg_setup) runs once per coefficient field; the V-cycle launches kernels only (no
// host synchronisation, no allocation), so it can sit inside the captured CUDA graphs of the
// flexible-CG iteration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hostutil.h"
#include "internal.h"
#include "multigrid.h"
#include "ops.cuh"
#include "reduce.cuh"

namespace chns {
namespace {

constexpr int kMgThreads = 256;
constexpr int kMgMaxCoarse = 1024;  // nodes of the coarsest level (dense inverse)

unsigned grid_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kMgThreads - 1) / kMgThreads, 8192));
}

#define MG_LOOP(i, n)                                                       \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- kernels
template <class T>
__global__ void k_inject(const int32_t* __restrict__ inj, const T* __restrict__ src,
                         T* __restrict__ dst, int64_t n) {
  MG_LOOP(i, n) dst[i] = src[inj[i]];
}

// y[i] (+)= sum_k w[k] x[col[k]] over row i of a CSR table; with SUB the gathered values are
// (x - x2)[col] (restriction of a residual r - A z formed on the fly)
template <class T, bool ADD, bool SUB>
__global__ void k_csr_gather(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                             const float* __restrict__ w, const T* __restrict__ x,
                             const T* __restrict__ x2, T* __restrict__ y, int64_t n) {
  MG_LOOP(i, n) {
    T acc = T(0);
    const int b = ptr[i], e = ptr[i + 1];
    for (int k = b; k < e; ++k) {
      const int c = col[k];
      const T v = SUB ? x[c] - x2[c] : x[c];
      acc += (T)w[k] * v;
    }
    y[i] = ADD ? y[i] + acc : acc;
  }
}

// first Chebyshev step: d = f dinv (r - w) (w = A z of the current iterate, or absent for a
// zero initial guess); z = d (zero guess) or z += d
template <class T, bool GUESS>
__global__ void k_cheb_first(const T* __restrict__ dinv, const T* __restrict__ r,
                             const T* __restrict__ w, T* __restrict__ z, T* __restrict__ d, T f,
                             int64_t n) {
  MG_LOOP(i, n) {
    const T ri = GUESS ? r[i] - w[i] : r[i];
    const T di = f * dinv[i] * ri;
    d[i] = di;
    z[i] = GUESS ? z[i] + di : di;
  }
}

// later Chebyshev steps: d = a d + b dinv (r - w); z += d
template <class T>
__global__ void k_cheb_next(const T* __restrict__ dinv, const T* __restrict__ r,
                            const T* __restrict__ w, T* __restrict__ z, T* __restrict__ d, T a, T b,
                            int64_t n) {
  MG_LOOP(i, n) {
    const T di = a * d[i] + b * dinv[i] * (r[i] - w[i]);
    d[i] = di;
    z[i] += di;
  }
}

// power-iteration start: v_i = dinv_i (h(i) / 2^32 - 1/2), h(i) = i * 2654435761 mod 2^32
template <class T>
__global__ void k_power_start(const T* __restrict__ dinv, T* __restrict__ v, int64_t n) {
  MG_LOOP(i, n) {
    const uint32_t h = (uint32_t)((uint64_t)i * 2654435761ull);
    v[i] = dinv[i] * (T)((double)h / 4294967296.0 - 0.5);
  }
}

template <class T>
__global__ void k_mul(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out,
                      int64_t n) {
  MG_LOOP(i, n) out[i] = a[i] * b[i];
}

// *slot += v.v (block sums by FP64 atomics; slot cleared before)
template <class T>
__global__ void __launch_bounds__(kMgThreads)
k_norm2(const T* __restrict__ v, int64_t n, double* __restrict__ slot) {
  typename Acc<T>::type t = Acc<T>::zero();
  MG_LOOP(i, n) Acc<T>::fma(t, v[i], v[i]);
  typename Acc<T>::type a[1] = {t};
  double tot[1];
  block_sum<1, kMgThreads>(a, tot);
  if (threadIdx.x == 0) atomicAdd(slot, tot[0]);
}

// v /= sqrt(*slot)
template <class T>
__global__ void k_normalise(T* __restrict__ v, const double* __restrict__ slot, int64_t n) {
  const T s = (T)(1.0 / sqrt(slot[0]));
  MG_LOOP(i, n) v[i] *= s;
}

template <class TI, class TO>
__global__ void k_invert_diag(const TI* __restrict__ d, TO* __restrict__ dinv, int64_t n) {
  MG_LOOP(i, n) {
    const double v = (double)d[i];
    dinv[i] = (TO)(v != 0.0 ? 1.0 / v : 1.0);
  }
}

template <class TI, class TO>
__global__ void k_convert(const TI* __restrict__ a, TO* __restrict__ b, int64_t n) {
  MG_LOOP(i, n) b[i] = (TO)a[i];
}

// Dense matrix of the coarsest level's operator K (Poisson or shifted), A[i * n + j] +=
// (P^T A_e P)_ij, one thread per element: the element matrix column by column (the element
// operator applied to unit vectors), distributed through the hanging constraints.
template <class K>
__global__ void k_dense_assemble(MeshDev m, DevParams p, CoefArgs<double> cf,
                                 double* __restrict__ A, int n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  int idx[8];
  load_corners(m, e, idx);
  const Geo<double> g = geometry<double>(m, e);
  K k;
  k.load(m, p, cf, idx, g);
  // corner references: up to 4 (node, weight) pairs per corner
  int ref[8][4];
  double wt[8][4];
  for (int a = 0; a < 8; ++a) {
    const int j = idx[a] & kIdxMask;
    for (int s = 0; s < 4; ++s) {
      ref[a][s] = -1;
      wt[a][s] = 0.0;
    }
    if (j < m.n_nodes) {
      ref[a][0] = j;
      wt[a][0] = 1.0;
    } else {
      const int4 h = m.hang[j - m.n_nodes];
      const bool four = h.z >= 0;
      const double w = four ? 0.25 : 0.5;
      ref[a][0] = h.x & kIdxMask;
      ref[a][1] = h.y & kIdxMask;
      wt[a][0] = wt[a][1] = w;
      if (four) {
        ref[a][2] = h.z & kIdxMask;
        ref[a][3] = h.w & kIdxMask;
        wt[a][2] = wt[a][3] = w;
      }
    }
  }
  for (int b = 0; b < 8; ++b) {
    double xin[1][8], r[1][8];
    for (int c = 0; c < 8; ++c) xin[0][c] = c == b ? 1.0 : 0.0;
    k.apply(g, p, xin, r);  // column b of the element matrix
    for (int a = 0; a < 8; ++a)
      for (int s = 0; s < 4; ++s) {
        if (ref[a][s] < 0) continue;
        for (int t = 0; t < 4; ++t) {
          if (ref[b][t] < 0) continue;
          atomicAdd(A + (int64_t)ref[a][s] * n + ref[b][t], wt[a][s] * wt[b][t] * r[0][a]);
        }
      }
  }
}

// In-place Gauss-Jordan inverse of the SPD matrix A + c 1 1^T (no pivoting: the pivots of an SPD
// matrix stay positive), one CTA.
__global__ void __launch_bounds__(1024) k_gauss_jordan(double* __restrict__ A, int n, double c) {
  __shared__ double colk[kMgMaxCoarse];
  __shared__ double piv_inv;
  for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += blockDim.x) A[q] += c;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) piv_inv = 1.0 / A[(int64_t)k * n + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double* rk = A + (int64_t)k * n;
      rk[j] = j == k ? piv_inv : rk[j] * piv_inv;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = A[(int64_t)i * n + k];
    __syncthreads();
    const double* rk = A + (int64_t)k * n;
    for (int64_t q = threadIdx.x; q < (int64_t)n * n; q += blockDim.x) {
      const int i = (int)(q / n), j = (int)(q % n);
      if (i == k) continue;
      if (j == k)
        A[q] = -colk[i] * piv_inv;
      else
        A[q] -= colk[i] * rk[j];
    }
    __syncthreads();
  }
}

// z = C r for a dense n x n matrix, one warp per row
template <class T>
__global__ void k_dense_mv(const T* __restrict__ C, const T* __restrict__ r, T* __restrict__ z,
                           int n) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= n) return;
  T acc = T(0);
  for (int j = lane; j < n; j += 32) acc += C[(int64_t)row * n + j] * r[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) z[row] = acc;
}

// ---------------------------------------------------------------- host construction
template <class P>
void dfree(P*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <class V>
chns_status upload(const std::vector<V>& h, V** d) {
  CHNS_CUDA(cudaMalloc(d, std::max<size_t>(h.size(), 1) * sizeof(V)));
  if (!h.empty())
    CHNS_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
  return CHNS_OK;
}

// One-level coarsening of the finest octant level (leaves in Morton order, in place of the first
// of each run of eight siblings).
chns_status coarsen(const std::vector<uint32_t>& a, const std::vector<uint8_t>& l,
                    std::vector<uint32_t>& ca, std::vector<uint8_t>& cl) {
  const int64_t n = (int64_t)l.size();
  int L = 0;
  for (uint8_t v : l) L = std::max(L, (int)v);
  CHNS_CHECK(L > 0, CHNS_EINVAL, "multigrid: cannot coarsen a single root leaf");
  const uint32_t sp = (uint32_t)(host::kFull >> (L - 1));
  ca.clear();
  cl.clear();
  for (int64_t i = 0; i < n;) {
    if (l[i] != L) {
      ca.insert(ca.end(), {a[3 * i], a[3 * i + 1], a[3 * i + 2]});
      cl.push_back(l[i]);
      ++i;
      continue;
    }
    const uint32_t p[3] = {a[3 * i] / sp * sp, a[3 * i + 1] / sp * sp, a[3 * i + 2] / sp * sp};
    CHNS_CHECK(i + 8 <= n && p[0] == a[3 * i] && p[1] == a[3 * i + 1] && p[2] == a[3 * i + 2],
               CHNS_EINVAL, "multigrid: finest leaves do not come in Morton-ordered sibling runs");
    for (int k = 1; k < 8; ++k)
      CHNS_CHECK(l[i + k] == L && a[3 * (i + k)] / sp * sp == p[0] &&
                     a[3 * (i + k) + 1] / sp * sp == p[1] && a[3 * (i + k) + 2] / sp * sp == p[2],
                 CHNS_EINVAL, "multigrid: finest leaves do not come in sibling runs");
    ca.insert(ca.end(), {p[0], p[1], p[2]});
    cl.push_back((uint8_t)(L - 1));
    i += 8;
  }
  return CHNS_OK;
}

// Morton keys of a mesh's nodes (ascending: nodes are numbered in Morton order)
std::vector<uint64_t> node_keys(const chns_mesh* m) {
  const int64_t N = m->d.n_nodes;
  std::vector<uint64_t> k((size_t)N);
  host::parallel_for(N, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i)
      k[i] = host::morton(m->node_coords[3 * i], m->node_coords[3 * i + 1],
                          m->node_coords[3 * i + 2]);
  });
  return k;
}

int64_t find_key(const std::vector<uint64_t>& keys, uint64_t k) {
  auto it = std::lower_bound(keys.begin(), keys.end(), k);
  if (it == keys.end() || *it != k) return -1;
  return int64_t(it - keys.begin());
}

struct Row {
  int n = 0;
  int32_t c[32];
  double w[32];
  void add(int32_t col, double v) {
    for (int k = 0; k < n; ++k)
      if (c[k] == col) {
        w[k] += v;
        return;
      }
    c[n] = col;
    w[n] = v;
    ++n;
  }
};

// Row of P for the fine node at integer point X: the coarse leaf whose half-open cell holds X
// (coordinates at the upper domain boundary moved inside by one unit, so that X lies in the
// leaf's closure), the trilinear weights of its corners at X, and the coarse hanging
// constraints. Returns false if X is not on the leaf's half-size lattice.
bool p_row(const uint32_t X[3], const std::vector<uint64_t>& lkey,
           const std::vector<uint32_t>& ca, const std::vector<uint8_t>& cl,
           const chns_mesh* cm, Row& row) {
  uint64_t q[3];
  for (int d = 0; d < 3; ++d) q[d] = std::min<uint64_t>(X[d], host::kFull - 1);
  const uint64_t k = host::morton(q[0], q[1], q[2]);
  const int64_t e = int64_t(std::upper_bound(lkey.begin(), lkey.end(), k) - lkey.begin()) - 1;
  if (e < 0) return false;
  const uint64_t s = host::kFull >> cl[e], h = s / 2;
  double xi[3];
  for (int d = 0; d < 3; ++d) {
    const uint64_t off = X[d] - ca[3 * e + d];
    if (X[d] < ca[3 * e + d] || off > s || off % h != 0) return false;
    xi[d] = (double)(off / h) * 0.5;
  }
  row.n = 0;
  const int64_t Nc = cm->d.n_nodes;
  for (int a = 0; a < 8; ++a) {
    double w = 1.0;
    for (int d = 0; d < 3; ++d) w *= ((a >> d) & 1) ? xi[d] : 1.0 - xi[d];
    if (w == 0.0) continue;
    const int32_t v = cm->h_enode[8 * e + a] & kIdxMask;
    if (v < Nc) {
      row.add(v, w);
    } else {
      const int4 hp = cm->h_hang[v - Nc];
      const bool four = hp.z >= 0;
      const double wp = four ? 0.25 : 0.5;
      row.add(hp.x & kIdxMask, w * wp);
      row.add(hp.y & kIdxMask, w * wp);
      if (four) {
        row.add(hp.z & kIdxMask, w * wp);
        row.add(hp.w & kIdxMask, w * wp);
      }
    }
  }
  return true;
}

}  // namespace

chns_status mg_build_transfer(const chns_mesh* fm, const chns_mesh* cm,
                              const std::vector<uint32_t>& ca, const std::vector<uint8_t>& cl,
                              MgLevel& L) {
  const int64_t Nf = fm->d.n_nodes, Nc = cm->d.n_nodes, Ec = (int64_t)cl.size();
  std::vector<uint64_t> lkey((size_t)Ec);
  for (int64_t e = 0; e < Ec; ++e) lkey[e] = host::morton(ca[3 * e], ca[3 * e + 1], ca[3 * e + 2]);
  // P: counts, then entries
  std::vector<int32_t> ptr((size_t)Nf + 1, 0);
  std::vector<uint8_t> bad((size_t)Nf, 0);
  host::parallel_for(Nf, [&](int64_t b, int64_t e) {
    Row row;
    for (int64_t i = b; i < e; ++i) {
      if (!p_row(&fm->node_coords[3 * i], lkey, ca, cl, cm, row)) {
        bad[i] = 1;
        continue;
      }
      int nz = 0;
      for (int k = 0; k < row.n; ++k) nz += row.w[k] != 0.0;
      ptr[i + 1] = nz;
    }
  });
  for (int64_t i = 0; i < Nf; ++i)
    CHNS_CHECK(!bad[i], CHNS_EINVAL, "multigrid: a fine node is not on a coarse half-size lattice");
  for (int64_t i = 0; i < Nf; ++i) ptr[i + 1] += ptr[i];
  std::vector<int32_t> col((size_t)ptr[Nf]);
  std::vector<float> w((size_t)ptr[Nf]);
  host::parallel_for(Nf, [&](int64_t b, int64_t e) {
    Row row;
    for (int64_t i = b; i < e; ++i) {
      p_row(&fm->node_coords[3 * i], lkey, ca, cl, cm, row);
      int o = ptr[i];
      for (int k = 0; k < row.n; ++k)
        if (row.w[k] != 0.0) {
          col[o] = row.c[k];
          w[o] = (float)row.w[k];  // dyadic: exact
          ++o;
        }
    }
  });
  // R = P^T (rows by coarse node, entries in increasing fine row)
  std::vector<int32_t> rptr((size_t)Nc + 1, 0);
  for (int32_t c : col) ++rptr[c + 1];
  for (int64_t j = 0; j < Nc; ++j) rptr[j + 1] += rptr[j];
  std::vector<int32_t> rcol(col.size()), fill(rptr.begin(), rptr.end() - 1);
  std::vector<float> rw(col.size());
  for (int64_t i = 0; i < Nf; ++i)
    for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
      const int32_t o = fill[col[k]]++;
      rcol[o] = (int32_t)i;
      rw[o] = w[k];
    }
  // injection: coarse node -> fine node at the same point
  const std::vector<uint64_t> fkey = node_keys(fm);
  std::vector<int32_t> inj((size_t)Nc);
  bool miss = false;
  for (int64_t j = 0; j < Nc; ++j) {
    const int64_t f = find_key(fkey, host::morton(cm->node_coords[3 * j], cm->node_coords[3 * j + 1],
                                                  cm->node_coords[3 * j + 2]));
    if (f < 0) miss = true;
    inj[j] = (int32_t)f;
  }
  CHNS_CHECK(!miss, CHNS_EINVAL, "multigrid: a coarse node is not a fine node");
  chns_status st;
  if ((st = upload(ptr, &L.p_ptr)) != CHNS_OK) return st;
  if ((st = upload(col, &L.p_col)) != CHNS_OK) return st;
  if ((st = upload(w, &L.p_w)) != CHNS_OK) return st;
  if ((st = upload(rptr, &L.r_ptr)) != CHNS_OK) return st;
  if ((st = upload(rcol, &L.r_col)) != CHNS_OK) return st;
  if ((st = upload(rw, &L.r_w)) != CHNS_OK) return st;
  if ((st = upload(inj, &L.inj)) != CHNS_OK) return st;
  L.p_nnz = (int64_t)col.size();
  return CHNS_OK;
}

void mg_free(chns_mg* g) {
  if (!g) return;
  for (size_t l = 0; l < g->lv.size(); ++l) {
    MgLevel& L = g->lv[l];
    if (l > 0 && L.mesh) free_mesh(L.mesh);
    dfree(L.p_ptr);
    dfree(L.p_col);
    dfree(L.p_w);
    dfree(L.r_ptr);
    dfree(L.r_col);
    dfree(L.r_w);
    dfree(L.inj);
    for (int k = 0; k < kMgVecs; ++k) {
      dfree(L.v64[k]);
      dfree(L.v32[k]);
    }
    for (int o = 0; o < kMgOps; ++o) {
      dfree(L.op[o].phi64);
      dfree(L.op[o].phi32);
      dfree(L.op[o].dinv64);
      dfree(L.op[o].dinv32);
    }
  }
  for (int o = 0; o < kMgOps; ++o) {
    dfree(g->ops[o].cinv64);
    dfree(g->ops[o].cinv32);
  }
  dfree(g->cwork64);
  dfree(g->slots);
  if (g->h_slots) cudaFreeHost(g->h_slots);
  delete g;
}

chns_status mg_create(const chns_mesh* fine, const chns_mg_params* prm, cudaStream_t s,
                      chns_mg** out) {
  CHNS_CHECK(fine && out, CHNS_EINVAL, "chns_mg_create: null argument");
  chns_mg_params p{};
  p.coarsest_level = 2;
  p.degree = 3;
  p.power_its = 12;
  p.smooth_range = 15.0;
  p.lmax_factor = 1.1;
  if (prm) p = *prm;
  CHNS_CHECK(p.coarsest_level >= 0 && p.coarsest_level < CHNS_MAXD && p.degree >= 1 &&
                 p.degree <= 8 && p.power_its >= 1 && p.power_its <= 100 &&
                 p.smooth_range > 1.0 && p.lmax_factor >= 1.0,
             CHNS_EINVAL, "chns_mg_create: parameter out of range");
  chns_mg* g = new (std::nothrow) chns_mg();
  CHNS_CHECK(g, CHNS_ENOMEM, "chns_mg_create: out of host memory");
  g->prm = p;
  chns_status st = CHNS_OK;
  // level meshes
  const int64_t E0 = fine->d.n_elem;
  std::vector<uint32_t> a((size_t)E0 * 3), ca;
  std::vector<uint8_t> l((size_t)E0), cl;
  if (cudaMemcpy(a.data(), fine->d_anchor, a.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost) !=
          cudaSuccess ||
      cudaMemcpy(l.data(), fine->d_level, l.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error("chns_mg_create: cannot read the mesh's leaves");
    mg_free(g);
    return CHNS_ECUDA;
  }
  g->lv.push_back(MgLevel{});
  g->lv[0].mesh = const_cast<chns_mesh*>(fine);
  g->lv[0].n = fine->d.n_nodes;
  int maxl = fine->max_level;
  while (maxl > p.coarsest_level && st == CHNS_OK) {
    CHNS_CHECK((int)g->lv.size() < kMgMaxLevels, CHNS_EINVAL, "chns_mg_create: too many levels");
    st = coarsen(a, l, ca, cl);
    if (st != CHNS_OK) break;
    chns_mesh* cm = new (std::nothrow) chns_mesh();
    if (!cm) {
      set_error("chns_mg_create: out of host memory");
      st = CHNS_ENOMEM;
      break;
    }
    try {
      st = build_mesh(ca.data(), cl.data(), (int64_t)cl.size(), fine->d.ext, s, cm, true, true);
    } catch (const std::bad_alloc&) {
      set_error("chns_mg_create: out of host memory");
      st = CHNS_ENOMEM;
    }
    if (st != CHNS_OK) {
      free_mesh(cm);
      break;
    }
    MgLevel L{};
    L.mesh = cm;
    L.n = cm->d.n_nodes;
    g->lv.push_back(L);
    try {
      st = mg_build_transfer(g->lv[g->lv.size() - 2].mesh, cm, ca, cl, g->lv[g->lv.size() - 2]);
    } catch (const std::bad_alloc&) {
      set_error("chns_mg_create: out of host memory");
      st = CHNS_ENOMEM;
    }
    cm->h_enode.clear();
    cm->h_enode.shrink_to_fit();
    a.swap(ca);
    l.swap(cl);
    maxl = cm->max_level;
  }
  if (st == CHNS_OK && g->lv.back().n > kMgMaxCoarse) {
    set_error("chns_mg_create: the coarsest level has more than 1024 nodes (lower coarsest_level)");
    st = CHNS_EINVAL;
  }
  // vectors: level 0 needs the apply output and the Chebyshev direction; coarser levels also
  // their right-hand side and correction; per operator the inverse diagonal (and, Poisson, the
  // injected coefficient on the coarser levels)
  auto alloc_level = [&](MgLevel& L, bool fine_level) -> chns_status {
    for (int k = fine_level ? 2 : 0; k < kMgVecs; ++k) {
      CHNS_CUDA(cudaMalloc(&L.v64[k], L.n * sizeof(double)));
      CHNS_CUDA(cudaMalloc(&L.v32[k], L.n * sizeof(float)));
    }
    for (int o = 0; o < kMgOps; ++o) {
      if (!fine_level && o == kMgPoisson) {
        CHNS_CUDA(cudaMalloc(&L.op[o].phi64, L.n * sizeof(double)));
        CHNS_CUDA(cudaMalloc(&L.op[o].phi32, L.n * sizeof(float)));
      }
      CHNS_CUDA(cudaMalloc(&L.op[o].dinv64, L.n * sizeof(double)));
      CHNS_CUDA(cudaMalloc(&L.op[o].dinv32, L.n * sizeof(float)));
    }
    return CHNS_OK;
  };
  for (size_t k = 0; k < g->lv.size() && st == CHNS_OK; ++k) st = alloc_level(g->lv[k], k == 0);
  if (st == CHNS_OK) {
    const int64_t nc = g->lv.back().n;
    bool ok = cudaMalloc(&g->cwork64, nc * nc * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&g->slots, kMgMaxLevels * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&g->h_slots, kMgMaxLevels * sizeof(double)) == cudaSuccess;
    for (int o = 0; o < kMgOps && ok; ++o)
      ok = cudaMalloc(&g->ops[o].cinv64, nc * nc * sizeof(double)) == cudaSuccess &&
           cudaMalloc(&g->ops[o].cinv32, nc * nc * sizeof(float)) == cudaSuccess;
    if (!ok) {
      set_error("chns_mg_create: device allocation failed");
      st = CHNS_ENOMEM;
    }
  }
  if (st != CHNS_OK) {
    mg_free(g);
    return st;
  }
  *out = g;
  return CHNS_OK;
}

// ---------------------------------------------------------------- setup and cycle
template <class T>
constexpr int pix() {
  return sizeof(T) == sizeof(double) ? 0 : 1;
}
template <class T>
constexpr chns_precision prec_of() {
  return sizeof(T) == sizeof(double) ? CHNS_FP64 : CHNS_FP32;
}
template <class T>
static T* pick(double* a, float* b) {
  if constexpr (sizeof(T) == sizeof(double))
    return a;
  else
    return b;
}
template <class T>
static T* lv_vec(MgLevel& L, int k) { return pick<T>(L.v64[k], L.v32[k]); }
template <class T>
static T* lv_dinv(MgLevel& L, int op) { return pick<T>(L.op[op].dinv64, L.op[op].dinv32); }

// Poisson coefficient array of level l in precision T (level 0: the caller's)
template <class T>
static const T* level_phi(chns_mg* g, int l) {
  if (l == 0)
    return static_cast<const T*>(sizeof(T) == sizeof(double) ? g->ops[kMgPoisson].phi0_64
                                                             : g->ops[kMgPoisson].phi0_32);
  return pick<T>(g->lv[l].op[kMgPoisson].phi64, g->lv[l].op[kMgPoisson].phi32);
}

template <class T>
static chns_status level_apply(chns_mg* g, int op, int l, const T* x, T* y, cudaStream_t s) {
  MgLevel& L = g->lv[l];
  if (op == kMgShifted)  // the patch kernel gathers one coefficient field, unused here
    return apply_shift(L.mesh, &g->phys, lv_dinv<T>(L, op), g->ops[op].sa, g->ops[op].sb, x, y,
                       prec_of<T>(), s);
  chns_coef c{};
  c.phi_tilde = level_phi<T>(g, l);
  return apply_op(L.mesh, CHNS_OP_POISSON, &g->phys, &c, x, y, prec_of<T>(), s);
}

template <class T>
static chns_status level_diag(chns_mg* g, int op, int l, cudaStream_t s) {
  MgLevel& L = g->lv[l];
  T* d = lv_dinv<T>(L, op);
  if (op == kMgShifted) {
    // diag_shift gathers (and ignores) a coefficient field: the apply-output vector serves
    chns_status st = diag_shift(L.mesh, &g->phys, lv_vec<T>(L, 2), g->ops[op].sa, g->ops[op].sb,
                                d, prec_of<T>(), s);
    if (st != CHNS_OK) return st;
  } else {
    chns_coef c{};
    c.phi_tilde = level_phi<T>(g, l);
    chns_status st = diag_op(L.mesh, CHNS_OP_POISSON, &g->phys, &c, d, prec_of<T>(), s);
    if (st != CHNS_OK) return st;
  }
  note_launch();
  k_invert_diag<T, T><<<grid_for(L.n), kMgThreads, 0, s>>>(d, d, L.n);
  return CHNS_OK;
}

template <class T>
chns_status mg_setup_T(chns_mg* g, int op, cudaStream_t s) {
  const int NL = (int)g->lv.size();
  MgOpState& O = g->ops[op];
  O.ready[pix<T>()] = false;
  // injected coefficients (Poisson)
  if (op == kMgPoisson)
    for (int l = 1; l < NL; ++l) {
      note_launch();
      k_inject<T><<<grid_for(g->lv[l].n), kMgThreads, 0, s>>>(
          g->lv[l - 1].inj, level_phi<T>(g, l - 1),
          pick<T>(g->lv[l].op[op].phi64, g->lv[l].op[op].phi32), g->lv[l].n);
    }
  for (int l = 0; l < NL; ++l) {
    chns_status st = level_diag<T>(g, op, l, s);
    if (st != CHNS_OK) return st;
  }
  // largest eigenvalue of D^-1 A per level (power iteration, normalised on the device)
  const int NS = NL - 1;  // the coarsest level is solved exactly
  double* slot = g->slots;
  if (NS > 0) {
    for (int l = 0; l < NS; ++l) {
      MgLevel& L = g->lv[l];
      note_launch();
      k_power_start<T><<<grid_for(L.n), kMgThreads, 0, s>>>(lv_dinv<T>(L, op), lv_vec<T>(L, 3),
                                                            L.n);
    }
    for (int it = 0; it <= g->prm.power_its; ++it) {
      CHNS_CUDA(cudaMemsetAsync(slot, 0, NS * sizeof(double), s));
      for (int l = 0; l < NS; ++l) {
        MgLevel& L = g->lv[l];
        T* v = lv_vec<T>(L, 3);
        T* w = lv_vec<T>(L, 2);
        if (it > 0) {
          chns_status st = level_apply<T>(g, op, l, v, w, s);
          if (st != CHNS_OK) return st;
          note_launch();
          k_mul<T><<<grid_for(L.n), kMgThreads, 0, s>>>(lv_dinv<T>(L, op), w, v, L.n);
        }
        note_launch();
        k_norm2<T><<<grid_for(L.n), kMgThreads, 0, s>>>(v, L.n, slot + l);
        note_launch();
        k_normalise<T><<<grid_for(L.n), kMgThreads, 0, s>>>(v, slot + l, L.n);
      }
    }
    CHNS_CUDA(cudaMemcpyAsync(g->h_slots, slot, NS * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  // coarsest: dense inverse in FP64 (Poisson: of A + 1 1^T / n, the mean-zero solution)
  {
    MgLevel& C = g->lv.back();
    const int n = (int)C.n;
    // the FP32 setup works in its own FP64 matrix, so that the FP64 inverse stays valid
    double* Aw = sizeof(T) == sizeof(double) ? O.cinv64 : g->cwork64;
    CHNS_CUDA(cudaMemsetAsync(Aw, 0, (size_t)n * n * sizeof(double), s));
    DevParams p = make_dev_params(g->phys);
    CoefArgs<double> cf{};
    cf.phi_shift = 0.0f;
    const unsigned nb = (unsigned)((C.mesh->d.n_elem + 127) / 128);
    if (op == kMgPoisson) {
      const double* phic = nullptr;
      if (sizeof(T) == sizeof(double)) {
        phic = reinterpret_cast<const double*>(level_phi<T>(g, NL - 1));
      } else {
        // FP64 copy of the FP32 coefficients in the coarsest level's FP64 apply-output vector
        double* tmp = C.v64[2];
        note_launch();
        k_convert<T, double><<<grid_for(n), kMgThreads, 0, s>>>(level_phi<T>(g, NL - 1), tmp, n);
        phic = tmp;
      }
      cf.phi = phic;
      note_launch();
      k_dense_assemble<PoissonK<double, double>><<<nb, 128, 0, s>>>(C.mesh->d, p, cf, Aw, n);
    } else {
      p.d.sa = O.sa;
      p.d.sb = O.sb;
      cf.phi = C.v64[2];  // gathered, unused
      note_launch();
      k_dense_assemble<ShiftK<double, double>><<<nb, 128, 0, s>>>(C.mesh->d, p, cf, Aw, n);
    }
    note_launch();
    k_gauss_jordan<<<1, 1024, 0, s>>>(Aw, n, op == kMgPoisson ? 1.0 / n : 0.0);
    if (sizeof(T) == sizeof(float)) {
      note_launch();
      k_convert<double, float><<<grid_for((int64_t)n * n), kMgThreads, 0, s>>>(
          Aw, O.cinv32, (int64_t)n * n);
    }
  }
  CHNS_CUDA(cudaGetLastError());
  CHNS_CUDA(cudaStreamSynchronize(s));
  for (int l = 0; l < NS; ++l) {
    const double lam = std::sqrt(g->h_slots[l]);
    CHNS_CHECK(std::isfinite(lam) && lam > 0.0, CHNS_EBREAKDOWN,
               "multigrid: power iteration failed");
    MgOpLevel& Lo = g->lv[l].op[op];
    Lo.lmax[pix<T>()] = g->prm.lmax_factor * lam;
    Lo.lmin[pix<T>()] = Lo.lmax[pix<T>()] / g->prm.smooth_range;
  }
  O.ready[pix<T>()] = true;
  return CHNS_OK;
}

// z = B r on level l (r and z of the level's size; level 0 uses the caller's vectors)
template <class T>
static chns_status vcycle(chns_mg* g, int op, int l, const T* r, T* z, cudaStream_t s) {
  const int NL = (int)g->lv.size();
  MgLevel& L = g->lv[l];
  const int64_t n = L.n;
  const unsigned vg = grid_for(n);
  if (l == NL - 1) {
    const T* C = pick<T>(g->ops[op].cinv64, g->ops[op].cinv32);
    note_launch();
    k_dense_mv<T><<<(unsigned)((n + 7) / 8), 256, 0, s>>>(C, r, z, (int)n);
    return CHNS_OK;
  }
  const MgOpLevel& Lo = L.op[op];
  const double lmax = Lo.lmax[pix<T>()], lmin = Lo.lmin[pix<T>()];
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  const T* dinv = lv_dinv<T>(L, op);
  T* w = lv_vec<T>(L, 2);
  T* d = lv_vec<T>(L, 3);
  chns_status st;
  auto smooth = [&](bool guess) -> chns_status {
    if (guess) {
      st = level_apply<T>(g, op, l, z, w, s);
      if (st != CHNS_OK) return st;
      note_launch();
      k_cheb_first<T, true><<<vg, kMgThreads, 0, s>>>(dinv, r, w, z, d, (T)(1.0 / theta), n);
    } else {
      note_launch();
      k_cheb_first<T, false><<<vg, kMgThreads, 0, s>>>(dinv, r, nullptr, z, d, (T)(1.0 / theta), n);
    }
    double rho_old = 1.0 / sigma;
    for (int i = 1; i < g->prm.degree; ++i) {
      const double rho = 1.0 / (2.0 * sigma - rho_old);
      st = level_apply<T>(g, op, l, z, w, s);
      if (st != CHNS_OK) return st;
      note_launch();
      k_cheb_next<T><<<vg, kMgThreads, 0, s>>>(dinv, r, w, z, d, (T)(rho * rho_old),
                                               (T)(2.0 * rho / delta), n);
      rho_old = rho;
    }
    return CHNS_OK;
  };
  if ((st = smooth(false)) != CHNS_OK) return st;
  // coarse correction: r_c = R (r - A z), z += P z_c
  if ((st = level_apply<T>(g, op, l, z, w, s)) != CHNS_OK) return st;
  MgLevel& Cl = g->lv[l + 1];
  T* rc = lv_vec<T>(Cl, 0);
  T* zc = lv_vec<T>(Cl, 1);
  note_launch();
  k_csr_gather<T, false, true><<<grid_for(Cl.n), kMgThreads, 0, s>>>(L.r_ptr, L.r_col, L.r_w, r, w,
                                                                      rc, Cl.n);
  if ((st = vcycle<T>(g, op, l + 1, rc, zc, s)) != CHNS_OK) return st;
  note_launch();
  k_csr_gather<T, true, false><<<vg, kMgThreads, 0, s>>>(L.p_ptr, L.p_col, L.p_w, zc, nullptr, z,
                                                         n);
  if ((st = smooth(true)) != CHNS_OK) return st;
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status mg_setup(chns_mg* g, const chns_params* prm, const void* phi0, chns_precision prec,
                     cudaStream_t s) {
  CHNS_CHECK(g && prm && phi0, CHNS_EINVAL, "multigrid setup: null argument");
  g->phys = *prm;
  MgOpState& O = g->ops[kMgPoisson];
  if (prec == CHNS_FP64) {
    O.phi0_64 = phi0;
    return mg_setup_T<double>(g, kMgPoisson, s);
  }
  if (prec == CHNS_FP32) {
    O.phi0_32 = phi0;
    return mg_setup_T<float>(g, kMgPoisson, s);
  }
  set_error("multigrid setup: precision must be CHNS_FP64 or CHNS_FP32");
  return CHNS_EINVAL;
}

chns_status mg_setup_shifted(chns_mg* g, const chns_params* prm, double sa, double sb,
                             chns_precision prec, cudaStream_t s) {
  CHNS_CHECK(g && prm && sa > 0.0 && sb >= 0.0, CHNS_EINVAL,
             "multigrid setup (shifted): null argument or sa <= 0 or sb < 0");
  CHNS_CHECK(prec == CHNS_FP64 || prec == CHNS_FP32, CHNS_EINVAL,
             "multigrid setup: precision must be CHNS_FP64 or CHNS_FP32");
  MgOpState& O = g->ops[kMgShifted];
  const int pi = prec == CHNS_FP64 ? 0 : 1;
  if (O.ready[pi] && O.sa == sa && O.sb == sb) return CHNS_OK;  // constant coefficients
  if (O.sa != sa || O.sb != sb) O.ready[0] = O.ready[1] = false;
  O.sa = sa;
  O.sb = sb;
  g->phys = *prm;
  return prec == CHNS_FP64 ? mg_setup_T<double>(g, kMgShifted, s) : mg_setup_T<float>(g, kMgShifted, s);
}

template <class T>
chns_status mg_vcycle(chns_mg* g, int op, const T* r, T* z, cudaStream_t s) {
  CHNS_CHECK(op >= 0 && op < kMgOps && g->ops[op].ready[pix<T>()], CHNS_EINVAL,
             "multigrid: V-cycle before setup of this operator in this precision");
  return vcycle<T>(g, op, 0, r, z, s);
}
template chns_status mg_vcycle<double>(chns_mg*, int, const double*, double*, cudaStream_t);
template chns_status mg_vcycle<float>(chns_mg*, int, const float*, float*, cudaStream_t);

}  // namespace chns

using namespace chns;

extern "C" chns_status chns_mg_create(const chns_mesh* fine, const chns_mg_params* prm,
                                      void* stream, chns_mg** out) {
  if (out) *out = nullptr;
  return mg_create(fine, prm, as_stream(stream), out);
}

extern "C" void chns_mg_destroy(chns_mg* g) { mg_free(g); }

extern "C" chns_status chns_mg_levels(const chns_mg* g, int32_t* n_levels, int64_t* n_nodes,
                                      int64_t* n_elem) {
  CHNS_CHECK(g && n_levels, CHNS_EINVAL, "chns_mg_levels: null argument");
  *n_levels = (int32_t)g->lv.size();
  for (size_t l = 0; l < g->lv.size(); ++l) {
    if (n_nodes) n_nodes[l] = g->lv[l].n;
    if (n_elem) n_elem[l] = g->lv[l].mesh->d.n_elem;
  }
  return CHNS_OK;
}

extern "C" chns_status chns_mg_setup(chns_mg* g, const chns_params* prm, const void* phi_tilde,
                                     chns_precision prec, void* stream) {
  return mg_setup(g, prm, phi_tilde, prec, as_stream(stream));
}

extern "C" chns_status chns_mg_setup_shifted(chns_mg* g, const chns_params* prm, double sa,
                                             double sb, chns_precision prec, void* stream) {
  return mg_setup_shifted(g, prm, sa, sb, prec, as_stream(stream));
}

extern "C" chns_status chns_mg_lambda(const chns_mg* g, int32_t op, chns_precision prec,
                                      double* lmax) {
  CHNS_CHECK(g && lmax && op >= 0 && op < kMgOps && (prec == CHNS_FP64 || prec == CHNS_FP32),
             CHNS_EINVAL, "chns_mg_lambda: bad argument");
  const int pi = prec == CHNS_FP64 ? 0 : 1;
  CHNS_CHECK(g->ops[op].ready[pi], CHNS_EINVAL, "chns_mg_lambda: no setup in this precision");
  for (size_t l = 0; l < g->lv.size(); ++l) lmax[l] = g->lv[l].op[op].lmax[pi];
  return CHNS_OK;
}

extern "C" chns_status chns_mg_vcycle(chns_mg* g, int32_t op, const void* r, void* z,
                                      chns_precision prec, void* stream) {
  CHNS_CHECK(g && r && z && r != z, CHNS_EINVAL, "chns_mg_vcycle: bad argument");
  if (prec == CHNS_FP64)
    return mg_vcycle<double>(g, op, static_cast<const double*>(r), static_cast<double*>(z),
                             as_stream(stream));
  if (prec == CHNS_FP32)
    return mg_vcycle<float>(g, op, static_cast<const float*>(r), static_cast<float*>(z),
                            as_stream(stream));
  set_error("chns_mg_vcycle: precision must be CHNS_FP64 or CHNS_FP32");
  return CHNS_EINVAL;
}

extern "C" chns_status chns_mg_prolong(const chns_mg* g, int32_t level, const double* xc,
                                       double* xf, void* stream) {
  CHNS_CHECK(g && xc && xf && level >= 0 && level + 1 < (int)g->lv.size(), CHNS_EINVAL,
             "chns_mg_prolong: bad argument");
  const MgLevel& L = g->lv[level];
  note_launch();
  k_csr_gather<double, false, false><<<grid_for(L.n), kMgThreads, 0, as_stream(stream)>>>(
      L.p_ptr, L.p_col, L.p_w, xc, nullptr, xf, L.n);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

extern "C" chns_status chns_mg_restrict(const chns_mg* g, int32_t level, const double* xf,
                                        double* xc, void* stream) {
  CHNS_CHECK(g && xc && xf && level >= 0 && level + 1 < (int)g->lv.size(), CHNS_EINVAL,
             "chns_mg_restrict: bad argument");
  const MgLevel& L = g->lv[level];
  const int64_t nc = g->lv[level + 1].n;
  note_launch();
  k_csr_gather<double, false, false><<<grid_for(nc), kMgThreads, 0, as_stream(stream)>>>(
      L.r_ptr, L.r_col, L.r_w, xf, nullptr, xc, nc);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

extern "C" chns_status chns_mg_coefficient(const chns_mg* g, int32_t level, double* phi,
                                           void* stream) {
  CHNS_CHECK(g && phi && level >= 0 && level < (int)g->lv.size() &&
                 g->ops[kMgPoisson].ready[0],
             CHNS_EINVAL, "chns_mg_coefficient: bad argument or no FP64 Poisson setup");
  const double* src = level == 0 ? static_cast<const double*>(g->ops[kMgPoisson].phi0_64)
                                 : g->lv[level].op[kMgPoisson].phi64;
  CHNS_CUDA(cudaMemcpyAsync(phi, src, g->lv[level].n * sizeof(double), cudaMemcpyDeviceToDevice,
                            as_stream(stream)));
  return CHNS_OK;
}
