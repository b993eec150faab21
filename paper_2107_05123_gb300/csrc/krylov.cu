// Krylov solvers on the matrix-free operators: Jacobi-preconditioned CG (pressure Poisson,
// velocity update) and right-preconditioned restarted GMRES (Cahn-Hilliard Newton steps,
// velocity prediction). The paper solves these systems with PETSc Krylov methods (Appendix A);
// here every vector update and every dot product is a fused device kernel, dot products and norms
// are accumulated in FP64 with a deterministic two-level reduction (per-block partial sums, then
// a fixed-order sum in the last block), and CG keeps its scalars on the device so that the host
// only reads the residual norm every `check_every` iterations.
//
// Mixed precision: with an FP32 inner precision the Krylov iteration runs on FP32 vectors and FP32
// (or BF16-coefficient) applies, with FP64 dot products, inside an FP64 iterative-refinement loop
// whose residual r = b - A_64 x uses the FP64 operator.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "multigrid.h"
#include "reduce.cuh"

namespace chns {

constexpr int kVecThreads = 256;
constexpr int kMdBlocks = 256;  // blocks per multi-dot row (partials: rows x kMdBlocks)

// device scalar slots (offsets from ws.red + kScalarBase)
enum Slot { S_RZ0 = 0, S_RZ1 = 1, S_PQ = 2, S_RR = 3, S_TMP = 8, S_AUX = 16, S_MD = 64 };

// ------------------------------------------------------------------ device kernels
// Block reduction of NV sums with the fixed-order last-block finalisation of reduce.cuh.
template <int NV, class A>
__device__ __forceinline__ void reduce_finalize(A (&v)[NV], double* __restrict__ part,
                                                unsigned* __restrict__ counter,
                                                double* __restrict__ out) {
  block_reduce_finalize<NV, kVecThreads>(v, part, kRedSlots, counter, out);
}

#define GRID_LOOP(i, n)                                                     \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

template <class A, class B>
__global__ void __launch_bounds__(kVecThreads)
k_dot(const A* __restrict__ a, const B* __restrict__ b, int64_t n, double* part, unsigned* counter,
      double* out) {
  typename Acc<A>::type t = Acc<A>::zero();  // double-float for FP32 vectors, FP64 for FP64
  GRID_LOOP(i, n) Acc<A>::fma(t, a[i], (A)b[i]);
  typename Acc<A>::type v[1] = {t};
  reduce_finalize<1>(v, part, counter, out);
}

template <class A>
__global__ void __launch_bounds__(kVecThreads)
k_sum(const A* __restrict__ a, int64_t n, double* part, unsigned* counter, double* out) {
  typename Acc<A>::type t = Acc<A>::zero();
  GRID_LOOP(i, n) Acc<A>::add(t, a[i]);
  typename Acc<A>::type v[1] = {t};
  reduce_finalize<1>(v, part, counter, out);
}

// out = a x + b y
template <class T>
__global__ void k_axpby(double a, const T* __restrict__ x, double b, const T* y, T* out,
                        int64_t n) {  // out may alias y (in-place residual updates)
  const T ta = (T)a, tb = (T)b;
  GRID_LOOP(i, n) out[i] = ta * x[i] + tb * y[i];
}

// out (TO) = scale * in (TI)
template <class TI, class TO>
__global__ void k_convert(const TI* __restrict__ a, TO* __restrict__ b, int64_t n, double scale) {
  GRID_LOOP(i, n) b[i] = (TO)((double)a[i] * scale);
}
__global__ void k_convert_bf16(const double* __restrict__ a, __nv_bfloat16* __restrict__ b,
                               int64_t n, double offset) {
  GRID_LOOP(i, n) b[i] = __float2bfloat16_rn((float)(a[i] + offset));
}

// x += factor * s[0]
template <class T>
__global__ void k_add_scalar(T* __restrict__ x, const double* __restrict__ s, double factor,
                             int64_t n) {
  const T v = (T)(s[0] * factor);
  GRID_LOOP(i, n) x[i] += v;
}

// x64 += scale * d
template <class T>
__global__ void k_accumulate(double* __restrict__ x, const T* __restrict__ d, double scale,
                             int64_t n) {
  GRID_LOOP(i, n) x[i] += scale * (double)d[i];
}

// dinv = 1/d (1 where d == 0); d may alias dinv
template <class TI, class TO>
__global__ void k_invert(const TI* d, TO* dinv, int64_t n) {
  GRID_LOOP(i, n) {
    const double v = (double)d[i];
    dinv[i] = (TO)(v != 0.0 ? 1.0 / v : 1.0);
  }
}

// z = dinv * v (dinv may be null: identity)
template <class T>
__global__ void k_mul(const T* __restrict__ dinv, const T* __restrict__ v, T* __restrict__ z,
                      int64_t n) {
  GRID_LOOP(i, n) z[i] = dinv ? dinv[i] * v[i] : v[i];
}

// Inverse of the 2x2 nodal blocks [a b; c d] (stored as 4 arrays of N), in place into `inv`.
template <class TI, class T>
__global__ void k_invert_b2(const TI* d, T* inv, int64_t N) {  // d may alias inv
  GRID_LOOP(i, N) {
    const double a = d[i], b = d[N + i], c = d[2 * N + i], e = d[3 * N + i];
    const double det = a * e - b * c;
    const double scale = fabs(a * e) + fabs(b * c);
    if (det != 0.0 && fabs(det) > 1e-14 * scale) {
      inv[i] = (T)(e / det);
      inv[N + i] = (T)(-b / det);
      inv[2 * N + i] = (T)(-c / det);
      inv[3 * N + i] = (T)(a / det);
    } else {
      inv[i] = (T)(a != 0.0 ? 1.0 / a : 1.0);
      inv[N + i] = T(0);
      inv[2 * N + i] = T(0);
      inv[3 * N + i] = (T)(e != 0.0 ? 1.0 / e : 1.0);
    }
  }
}

// z = B^-1 v with 2x2 nodal blocks (the CH pair [phi; mu], N nodes)
template <class T>
__global__ void k_mul_b2(const T* __restrict__ inv, const T* __restrict__ v, T* __restrict__ z,
                         int64_t N) {
  GRID_LOOP(i, N) {
    const T v0 = v[i], v1 = v[N + i];
    z[i] = inv[i] * v0 + inv[N + i] * v1;
    z[N + i] = inv[2 * N + i] * v0 + inv[3 * N + i] * v1;
  }
}

// ---- CG kernels. Scalars live in device memory at the parity slots of internal.h; iteration k
// has parity par = k & 1.
// alpha of the update: FP32 vectors divide in FP32 in every thread (no barrier before the loads);
// FP64 vectors let thread 0 divide once per block.
template <class T>
__device__ __forceinline__ T cg_ratio(const double* S, int num, int den, bool positive) {
  if (sizeof(T) == sizeof(float)) {
    const float nf = (float)S[num], df = (float)S[den];
    return (positive ? df > 0.f : df != 0.f) && isfinite(df) ? (T)(nf / df) : T(0);
  }
  __shared__ double s_v;
  if (threadIdx.x == 0) {
    const double nd = S[num], dd = S[den];
    s_v = (positive ? dd > 0.0 : dd != 0.0) && isfinite(dd) ? nd / dd : 0.0;
  }
  __syncthreads();
  return (T)s_v;
}

// k_cg_update: alpha = r.z / p.Ap; x += alpha p; r -= alpha q; z = dinv r (q cleared when
// zero_q); the block sums of r.z and r.r are added to the next parity's slots; block 0 keeps
// r.z as the previous value and clears the next p.Ap accumulator.
template <class T>
__global__ void __launch_bounds__(kVecThreads)
k_cg_update(T* __restrict__ x, T* __restrict__ r, T* __restrict__ z, const T* __restrict__ p,
            T* __restrict__ q, const T* __restrict__ dinv, int64_t n, double* __restrict__ S,
            bool zero_q, int par) {
  const T a = cg_ratio<T>(S, kCgRz0 + par, kCgPq0 + par, true);
  typename Acc<T>::type v0 = Acc<T>::zero(), v1 = Acc<T>::zero();
  GRID_LOOP(i, n) {
    x[i] += a * p[i];
    const T ri = r[i] - a * q[i];
    if (zero_q) q[i] = T(0);
    r[i] = ri;
    const T zi = dinv ? dinv[i] * ri : ri;
    z[i] = zi;
    Acc<T>::fma(v0, ri, zi);
    Acc<T>::fma(v1, ri, ri);
  }
  typename Acc<T>::type v[2] = {v0, v1};
  double tot[2];
  block_sum<2, kVecThreads>(v, tot);
  if (threadIdx.x == 0) {
    atomicAdd(S + kCgRz0 + (par ^ 1), tot[0]);
    atomicAdd(S + kCgRr0 + (par ^ 1), tot[1]);
    if (blockIdx.x == 0) {
      S[kCgRzPrev] = S[kCgRz0 + par];
      S[kCgPq0 + (par ^ 1)] = 0.0;
    }
  }
}

// *out += a.b (block sums added with an FP64 atomic; out cleared by an earlier kernel)
template <class T>
__global__ void __launch_bounds__(kVecThreads)
k_dot_atomic(const T* __restrict__ a, const T* __restrict__ b, int64_t n, double* __restrict__ out) {
  typename Acc<T>::type t = Acc<T>::zero();
  GRID_LOOP(i, n) Acc<T>::fma(t, a[i], b[i]);
  typename Acc<T>::type v[1] = {t};
  double tot[1];
  block_sum<1, kVecThreads>(v, tot);
  if (threadIdx.x == 0) atomicAdd(out, tot[0]);
}

// p_new = z + beta p_old with beta = r.z / r.z_prev (operators whose apply does not fuse it);
// clears the accumulators of the update that follows
template <class T>
__global__ void k_cg_pupdate(const T* __restrict__ z, const T* __restrict__ p_old,
                             T* __restrict__ p_new, int64_t n, double* __restrict__ S, int par) {
  const T b = cg_ratio<T>(S, kCgRz0 + par, kCgRzPrev, false);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S[kCgRz0 + (par ^ 1)] = 0.0;
    S[kCgRr0 + (par ^ 1)] = 0.0;
  }
  GRID_LOOP(i, n) p_new[i] = z[i] + b * p_old[i];
}

// ---- flexible CG (Polak-Ribiere beta), slots of internal.h.
// k_fcg_update: alpha = r.z / p.q; x += alpha p; r -= alpha q; r.r added to the next parity slot;
// block 0 stores alpha and clears the accumulators of the dot kernel and of the next apply
template <class T>
__global__ void __launch_bounds__(kVecThreads)
k_fcg_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
             const T* __restrict__ q, int64_t n, double* __restrict__ S, int par) {
  const T a = cg_ratio<T>(S, kFcgRz0 + par, kCgPq0 + par, true);
  typename Acc<T>::type v0 = Acc<T>::zero();
  GRID_LOOP(i, n) {
    x[i] += a * p[i];
    const T ri = r[i] - a * q[i];
    r[i] = ri;
    Acc<T>::fma(v0, ri, ri);
  }
  typename Acc<T>::type v[1] = {v0};
  double tot[1];
  block_sum<1, kVecThreads>(v, tot);
  if (threadIdx.x == 0) {
    atomicAdd(S + kCgRr0 + (par ^ 1), tot[0]);
    if (blockIdx.x == 0) {
      S[kFcgAlpha] = (double)a;
      S[kCgPq0 + (par ^ 1)] = 0.0;
      S[kFcgZq0 + par] = 0.0;
      S[kFcgRz0 + (par ^ 1)] = 0.0;
    }
  }
}

// z.q into kFcgZq0 + par and z.r into kFcgRz0 + (par ^ 1); q cleared for the next apply
template <class T>
__global__ void __launch_bounds__(kVecThreads)
k_fcg_dots(const T* __restrict__ z, T* __restrict__ q, const T* __restrict__ r, int64_t n,
           double* __restrict__ S, int par) {
  typename Acc<T>::type v0 = Acc<T>::zero(), v1 = Acc<T>::zero();
  GRID_LOOP(i, n) {
    const T zi = z[i];
    Acc<T>::fma(v0, zi, q[i]);
    q[i] = T(0);
    Acc<T>::fma(v1, zi, r[i]);
  }
  typename Acc<T>::type v[2] = {v0, v1};
  double tot[2];
  block_sum<2, kVecThreads>(v, tot);
  if (threadIdx.x == 0) {
    atomicAdd(S + kFcgZq0 + par, tot[0]);
    atomicAdd(S + kFcgRz0 + (par ^ 1), tot[1]);
  }
}

// first FCG direction: p = z (beta = -0 x 0 / 1); p.Ap accumulator cleared
__global__ void k_fcg_init(double* S) {
  S[kFcgAlpha] = 0.0;
  S[kFcgZq0 + 1] = 0.0;
  S[kFcgRz0 + 1] = 1.0;
  S[kCgPq0] = 0.0;
}

// z += omega dinv (r - w)  (w = A z)
template <class T>
__global__ void k_smooth(T* __restrict__ z, const T* __restrict__ r, const T* __restrict__ w,
                         const T* __restrict__ dinv, T omega, int64_t n) {
  GRID_LOOP(i, n) z[i] += omega * dinv[i] * (r[i] - w[i]);
}

// ---- GMRES
__global__ void __launch_bounds__(kVecThreads)
k_multidot_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double s[1] = {0.0};
  for (int b = threadIdx.x; b < nb; b += kVecThreads) s[0] += part[(int64_t)blockIdx.x * nb + b];
  double t[1];
  block_sum<1, kVecThreads>(s, t);
  if (threadIdx.x == 0) out[blockIdx.x] = t[0];
}

// x += B^-1 (sum_k y_k V_k) with 2x2 nodal blocks
template <class T>
__global__ void k_gmres_update_b2(const T* __restrict__ V, int64_t ld, int nk,
                                  const double* __restrict__ y, const T* __restrict__ inv,
                                  T* __restrict__ x, int64_t N) {
  GRID_LOOP(i, N) {
    double a0 = 0.0, a1 = 0.0;
    for (int k = 0; k < nk; ++k) {
      a0 += y[k] * (double)V[(int64_t)k * ld + i];
      a1 += y[k] * (double)V[(int64_t)k * ld + N + i];
    }
    const double z0 = (double)inv[i] * a0 + (double)inv[N + i] * a1;
    const double z1 = (double)inv[2 * N + i] * a0 + (double)inv[3 * N + i] * a1;
    x[i] = (T)((double)x[i] + z0);
    x[N + i] = (T)((double)x[N + i] + z1);
  }
}

// Multi-dot of rows V_0..V_{nk-1} with w, plus w.w as row nk. Each block stages a slice of w in
// shared memory once and sweeps all rows over it (the rows are read once, w once); per-warp sums
// accumulate in shared memory across the block's slices; partials land in part[k][blockIdx.x].
constexpr int kMd2Threads = 256;
// GMRES multi-dot: h_k = V_k . w for k < nk and h_nk = w.w. Block (c, k) of the 2D grid sums
// the products of row k (w itself for k = nk) with w over chunk c of the elements: one
// accumulator per thread (double-float for FP32 vectors), all loads coalesced and independent,
// full occupancy; w is re-read per row from L2. part[k * gridDim.x + c] -> k_multidot_final.
template <class T>
__global__ void __launch_bounds__(kMd2Threads)
k_multidot2(const T* __restrict__ V, int64_t ld, int nk, const T* __restrict__ w, int64_t n,
            double* __restrict__ part) {
  const int k = blockIdx.y;
  const T* __restrict__ a = k < nk ? V + (int64_t)k * ld : w;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * chunk;
  const int64_t i1 = i0 + chunk < n ? i0 + chunk : n;
  typename Acc<T>::type acc = Acc<T>::zero();
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kMd2Threads) Acc<T>::fma(acc, a[i], w[i]);
  typename Acc<T>::type v[1] = {acc};
  double tot[1];
  block_sum<1, kMd2Threads>(v, tot);
  if (threadIdx.x == 0) part[(int64_t)k * gridDim.x + blockIdx.x] = tot[0];
}

// w = (w - sum_k h_k V_k) * scale, with scale = 1/sqrt(h[nk] - sum_k h_k^2) when NORMALISE
// (h[nk] = w.w from the same multi-dot: Pythagoras for the classical Gram-Schmidt step). The
// update runs in the vector type (FP32 for FP32 vectors: FP64 arithmetic per element and basis
// vector would bound this kernel on GB300), the coefficients from shared memory.
template <class T, bool NORMALISE>
__global__ void k_orth_update_scale(const T* __restrict__ V, int64_t ld, int nk,
                                    const double* __restrict__ h, T* __restrict__ w, int64_t n) {
  __shared__ T hs[CHNS_GMRES_MAX_RESTART + 1];
  __shared__ T s_scale;
  if (threadIdx.x < nk) hs[threadIdx.x] = (T)h[threadIdx.x];
  if (threadIdx.x == 0) {
    double sc = 1.0;
    if (NORMALISE) {
      double hh = 0.0;
      for (int k = 0; k < nk; ++k) hh += h[k] * h[k];
      const double r = h[nk] - hh;
      sc = r > 0.0 ? rsqrt(r) : 1.0;
    }
    s_scale = (T)sc;
  }
  __syncthreads();
  const T sc = s_scale;
  GRID_LOOP(i, n) {
    T acc = w[i];
    for (int k = 0; k < nk; ++k) acc -= hs[k] * V[(int64_t)k * ld + i];
    w[i] = acc * sc;
  }
}

template <class T, bool NORMALISE>
void orth_update(const T* V, int64_t ld, int nk, const double* h, T* w, int64_t n, unsigned grid,
                 cudaStream_t s) {
  note_launch();
  k_orth_update_scale<T, NORMALISE><<<grid, kVecThreads, 0, s>>>(V, ld, nk, h, w, n);
}

template <class T>
__global__ void k_scale(T* __restrict__ a, double s, int64_t n) {
  GRID_LOOP(i, n) a[i] = (T)((double)a[i] * s);
}

// x += dinv * (sum_k y_k V_k)   (right preconditioning)
template <class T>
__global__ void k_gmres_update(const T* __restrict__ V, int64_t ld, int nk,
                               const double* __restrict__ y, const T* __restrict__ dinv,
                               T* __restrict__ x, int64_t n) {
  GRID_LOOP(i, n) {
    double acc = 0.0;
    for (int k = 0; k < nk; ++k) acc += y[k] * (double)V[(int64_t)k * ld + i];
    if (dinv) acc *= (double)dinv[i];
    x[i] = (T)((double)x[i] + acc);
  }
}

// ------------------------------------------------------------------ host helpers
static unsigned red_grid(const chns_mesh* m, int64_t n) {
  int64_t g = (n + kVecThreads - 1) / kVecThreads;
  int64_t cap = std::min<int64_t>(kRedSlots, 4 * (int64_t)m->sm_count);
  return (unsigned)std::max<int64_t>(1, std::min(g, cap));
}
static unsigned vgrid(const chns_mesh* m, int64_t n) {
  int64_t g = (n + kVecThreads - 1) / kVecThreads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 8 * (int64_t)m->sm_count));
}
static unsigned vgrid_n(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
}

void vec_axpby(double a, const double* x, double b, const double* y, double* out, int64_t n,
               cudaStream_t s) {
  note_launch();
  k_axpby<double><<<vgrid_n(n), kVecThreads, 0, s>>>(a, x, b, y, out, n);
}
void vec_copy(const double* x, double* y, int64_t n, cudaStream_t s) {
  cudaMemcpyAsync(y, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}
void vec_zero(double* x, int64_t n, cudaStream_t s) { cudaMemsetAsync(x, 0, n * sizeof(double), s); }
void vec_convert_f64_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  note_launch();
  k_convert<double, float><<<vgrid_n(n), kVecThreads, 0, s>>>(a, b, n, 1.0);
}
void vec_convert_f64_bf16(const double* a, __nv_bfloat16* b, int64_t n, double offset,
                          cudaStream_t s) {
  note_launch();
  k_convert_bf16<<<vgrid_n(n), kVecThreads, 0, s>>>(a, b, n, offset);
}
void vec_add_scalar(double* x, const double* dev_scalar, double factor, int64_t n, cudaStream_t s) {
  note_launch();
  k_add_scalar<double><<<vgrid_n(n), kVecThreads, 0, s>>>(x, dev_scalar, factor, n);
}

static double* scal(const chns_mesh* m) { return m->ws.red + kScalarBase; }

void dot_dev(const chns_mesh* m, const double* a, const double* b, int64_t n, double* dst,
             cudaStream_t s) {
  note_launch();
  k_dot<double, double><<<red_grid(m, n), kVecThreads, 0, s>>>(a, b, n, m->ws.red, m->ws.counter, dst);
}

static chns_status read_dev(const chns_mesh* m, const double* d, double* h, int count,
                            cudaStream_t s) {
  CHNS_CUDA(cudaMemcpyAsync(m->ws.h_pinned, d, count * sizeof(double), cudaMemcpyDeviceToHost, s));
  CHNS_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i) h[i] = m->ws.h_pinned[i];
  return CHNS_OK;
}

chns_status dot_host(const chns_mesh* m, const double* a, const double* b, int64_t n, double* out,
                     cudaStream_t s) {
  double* dst = scal(m) + S_AUX;
  dot_dev(m, a, b, n, dst, s);
  CHNS_CUDA(cudaGetLastError());
  return read_dev(m, dst, out, 1, s);
}

chns_status sum_host(const chns_mesh* m, const double* a, int64_t n, double* out, cudaStream_t s) {
  double* dst = scal(m) + S_AUX + 1;
  note_launch();
  k_sum<double><<<red_grid(m, n), kVecThreads, 0, s>>>(a, n, m->ws.red, m->ws.counter, dst);
  CHNS_CUDA(cudaGetLastError());
  return read_dev(m, dst, out, 1, s);
}

// ------------------------------------------------------------------ solvers
namespace {

// FCG with the learned correction stops when the residual norm has not halved in this many
// iterations; the solve then continues with the Jacobi preconditioner alone.
constexpr int kLearnedStall = 100;
// damping of the Jacobi step that follows the learned correction
constexpr double kLearnedOmega = 2.0 / 3.0;

struct Ctx {
  const chns_mesh* m;
  chns_operator op;
  const chns_params* prm;
  const chns_coef* coef64;  // FP64 coefficients
  chns_coef coefR;          // reduced-precision coefficients for the FP32 apply
  chns_precision inner;     // precision of the FP32 apply (FP32 or FP32_BF16COEF)
  cudaStream_t s;
  int64_t n;                // vector length (components * n_nodes)
  double* S;                // device scalars
  double sa = 0.0, sb = 0.0;  // op == kOpShift: y = sa M x + sb K x
  bool df = false;            // FP64 applies in double-float element arithmetic
};

template <class T>
chns_status apply_T(const Ctx& c, const T* x, T* y) {
  if (c.op == kOpShift)
    return apply_shift(c.m, c.prm, sizeof(T) == sizeof(double) ? c.coef64->phi_tilde : c.coefR.phi_tilde,
                       c.sa, c.sb, x, y, sizeof(T) == sizeof(double) ? CHNS_FP64 : CHNS_FP32, c.s);
  if (sizeof(T) == sizeof(double))
    return apply_op(c.m, c.op, c.prm, c.coef64, x, y, c.df ? CHNS_FP64_DF : CHNS_FP64, c.s);
  return apply_op(c.m, c.op, c.prm, &c.coefR, x, y, c.inner, c.s);
}

template <class T>
chns_status dot_to_host(const Ctx& c, const T* a, const T* b, double* out) {
  double* dst = c.S + S_AUX + 2;
  note_launch();
  k_dot<T, T><<<red_grid(c.m, c.n), kVecThreads, 0, c.s>>>(a, b, c.n, c.m->ws.red, c.m->ws.counter, dst);
  CHNS_CUDA(cudaGetLastError());
  return read_dev(c.m, dst, out, 1, c.s);
}

// v -= mean(v) (discrete mean over the nodes; pure-Neumann pressure)
template <class T>
chns_status project_mean(const Ctx& c, T* v) {
  double* dst = c.S + S_AUX + 3;
  note_launch();
  k_sum<T><<<red_grid(c.m, c.n), kVecThreads, 0, c.s>>>(v, c.n, c.m->ws.red, c.m->ws.counter, dst);
  note_launch();
  k_add_scalar<T><<<vgrid(c.m, c.n), kVecThreads, 0, c.s>>>(v, dst, -1.0 / (double)c.n, c.n);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

// One CG iteration (parity par) with direction buffers p_old -> p_new. Poisson: two kernels (the
// apply fuses p_new = z + beta p_old into its gather and accumulates p.Ap; the update clears q for
// the next apply). Other operators: p update, apply, dot, update.
template <class T>
chns_status cg_iteration(const Ctx& c, cudaStream_t s, T* x, T* r, T* z, const T* p_old,
                         T* p_new, T* q, const T* dinv, int par) {
  const int64_t n = c.n;
  const unsigned rg = red_grid(c.m, n), vg = vgrid(c.m, n);
  const bool fused = c.op == CHNS_OP_POISSON;
  chns_status st;
  if (fused) {
    if (sizeof(T) == sizeof(double))
      st = apply_poisson_cg(c.m, c.prm, c.coef64, z, p_old, p_new, q, CHNS_FP64, c.S, par, s);
    else
      st = apply_poisson_cg(c.m, c.prm, &c.coefR, z, p_old, p_new, q, c.inner, c.S, par, s);
    if (st != CHNS_OK) return st;
  } else {
    note_launch();
    k_cg_pupdate<T><<<vg, kVecThreads, 0, s>>>(z, p_old, p_new, n, c.S, par);
    Ctx cs = c;
    cs.s = s;
    st = apply_T<T>(cs, p_new, q);
    if (st != CHNS_OK) return st;
    note_launch();
    k_dot_atomic<T><<<rg, kVecThreads, 0, s>>>(p_new, q, n, c.S + kCgPq0 + par);
  }
  note_launch();
  k_cg_update<T><<<rg, kVecThreads, 0, s>>>(x, r, z, p_new, q, dinv, n, c.S, fused, par);
  return CHNS_OK;
}

// ---- Chebyshev polynomial preconditioner: `degree` steps of the Chebyshev iteration for
// D^-1 A z = D^-1 r from z = 0 on the interval [lmin, lmax] = [theta - delta, theta + delta]
// (three-term recurrence with rho_k = 1 / (2 sigma - rho_{k-1}), sigma = theta / delta), i.e.
// z = p(D^-1 A) D^-1 r with p the scaled Chebyshev polynomial; SPD while lmax bounds the
// spectrum of D^-1 A.
struct Cheb {
  double theta = 0.0, delta = 0.0;
  int degree = 0;
};

template <class T>
__global__ void k_cheb_init(const T* __restrict__ dinv, const T* __restrict__ r, T* __restrict__ z,
                            T* __restrict__ d, T f, int64_t n) {
  GRID_LOOP(i, n) {
    const T v = f * dinv[i] * r[i];
    z[i] = v;
    d[i] = v;
  }
}

template <class T>
__global__ void k_cheb_step(const T* __restrict__ dinv, const T* __restrict__ r,
                            const T* __restrict__ w, T* __restrict__ z, T* __restrict__ d, T a,
                            T b, int64_t n) {
  GRID_LOOP(i, n) {
    const T di = a * d[i] + b * dinv[i] * (r[i] - w[i]);
    d[i] = di;
    z[i] += di;
  }
}

template <class T>
chns_status cheb_apply(const Ctx& c, cudaStream_t s, const Cheb& ch, const T* dinv, const T* r,
                       T* z, T* w, T* d) {
  const unsigned vg = vgrid(c.m, c.n);
  const double sigma = ch.theta / ch.delta;
  double rho_old = 1.0 / sigma;
  note_launch();
  k_cheb_init<T><<<vg, kVecThreads, 0, s>>>(dinv, r, z, d, (T)(1.0 / ch.theta), c.n);
  Ctx cs = c;
  cs.s = s;
  for (int i = 1; i < ch.degree; ++i) {
    const double rho = 1.0 / (2.0 * sigma - rho_old);
    chns_status e = apply_T<T>(cs, z, w);
    if (e != CHNS_OK) return e;
    note_launch();
    k_cheb_step<T><<<vg, kVecThreads, 0, s>>>(dinv, r, w, z, d, (T)(rho * rho_old),
                                              (T)(2.0 * rho / ch.delta), c.n);
    rho_old = rho;
  }
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

// Interval of the Chebyshev preconditioner: lambda_max of D^-1 A from 15 power iterations
// started at D^-1 start, enlarged by 10 %; lmin = lmax / 30 (the polynomial damps the upper
// part of the spectrum, CG handles the rest).
template <class T>
chns_status cheb_bounds(const Ctx& c, const T* dinv, const T* start, T* v, T* w, int degree,
                        Cheb* ch) {
  const unsigned vg = vgrid(c.m, c.n);
  note_launch();
  k_mul<T><<<vg, kVecThreads, 0, c.s>>>(dinv, start, v, c.n);
  double nn = 0.0;
  chns_status st = dot_to_host<T>(c, v, v, &nn);
  if (st != CHNS_OK) return st;
  CHNS_CHECK(nn > 0.0 && std::isfinite(nn), CHNS_EBREAKDOWN, "Chebyshev: zero start vector");
  note_launch();
  k_scale<T><<<vg, kVecThreads, 0, c.s>>>(v, 1.0 / std::sqrt(nn), c.n);
  double lam = 0.0;
  for (int it = 0; it < 15; ++it) {
    st = apply_T<T>(c, v, w);
    if (st != CHNS_OK) return st;
    note_launch();
    k_mul<T><<<vg, kVecThreads, 0, c.s>>>(dinv, w, v, c.n);
    st = dot_to_host<T>(c, v, v, &nn);
    if (st != CHNS_OK) return st;
    CHNS_CHECK(nn > 0.0 && std::isfinite(nn), CHNS_EBREAKDOWN, "Chebyshev: power iteration failed");
    lam = std::sqrt(nn);
    note_launch();
    k_scale<T><<<vg, kVecThreads, 0, c.s>>>(v, 1.0 / lam, c.n);
  }
  const double lmax = 1.1 * lam, lmin = lmax / 30.0;
  ch->theta = 0.5 * (lmax + lmin);
  ch->delta = 0.5 * (lmax - lmin);
  ch->degree = degree;
  return CHNS_OK;
}

// Copies of the iterate every `every` iterations (FP64 CG only; collection of training pairs).
struct Snap {
  double* buf;  // [max][n]
  int every, max;
  int* count;
};

// Runs step(stream, it) — one iteration, which leaves r.r in S[kCgRr0 + ((it & 1) ^ 1)] — until
// sqrt(r.r) <= tol_abs or max_it iterations; rr is r.r before the first iteration. With chunk >= 2 the iterations run
// as CUDA graphs of `chunk` iterations (captured once per solve on a private stream); two graph
// instances write r.r into alternating pinned host slots so the host checks chunk k while chunk
// k+1 already runs. The solve may do up to two chunks beyond the iteration that reached the
// tolerance; they only reduce the residual. Iteration parities are preserved (chunks are even).
// With stall > 0 the iteration also stops (status CHNS_ENOTCONV) when the residual norm has not
// halved over the last `stall` iterations (checked at the host checks).
template <class T, class Step>
chns_status iterate(const Ctx& c, Step&& step, T* x, double tol_abs, int max_it, int chunk,
                    double rr, int* iters, double* rnorm, const Snap* snap, int stall = 0) {
  int it = 0;
  int ref_it = 0;
  double ref_rr = rr;
  auto stalled = [&](int now, double v) {
    if (stall <= 0) return false;
    if (v <= 0.25 * ref_rr) {
      ref_rr = v;
      ref_it = now;
      return false;
    }
    return now - ref_it >= stall;
  };
  chns_status st = CHNS_OK;
  auto bad = [&](double v) {
    if (std::isfinite(v)) return false;
    set_error("krylov: NaN/Inf in the residual norm");
    return true;
  };
  if (bad(rr)) {
    *iters = 0;
    *rnorm = rr;
    return CHNS_ENAN;
  }
  if (chunk < 2 || snap) {
    while (std::sqrt(rr) > tol_abs && it < max_it) {
      st = step(c.s, it);
      if (st != CHNS_OK) return st;
      ++it;
      if (snap && it % snap->every == 0 && *snap->count < snap->max) {
        CHNS_CUDA(cudaMemcpyAsync(snap->buf + (int64_t)(*snap->count) * c.n, x, c.n * sizeof(T),
                                  cudaMemcpyDeviceToDevice, c.s));
        ++*snap->count;
      }
      st = read_dev(c.m, c.S + kCgRr0 + (it & 1), &rr, 1, c.s);  // written by iteration it - 1
      if (st != CHNS_OK) return st;
      if (bad(rr)) {
        *iters = it;
        *rnorm = rr;
        return CHNS_ENAN;
      }
      if (stalled(it, rr)) break;
    }
  } else if (std::sqrt(rr) > tol_abs && max_it > 0) {
    chunk += chunk & 1;  // even: every chunk starts at parity 0
    cudaStream_t cs = c.m->cap_stream;
    cudaGraphExec_t ge[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    volatile double* slot = c.m->ws.h_pinned + 8;
    unsigned long long per_graph = 0;
    chns_status rc = CHNS_OK;
    for (int v = 0; v < 2 && rc == CHNS_OK; ++v) {
      cudaGraph_t g = nullptr;
      cudaError_t e0 = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e0 != cudaSuccess) {
        rc = cuda_fail(e0, "cudaStreamBeginCapture");
        break;
      }
      const unsigned long long l0 = chns_launches_now();
      for (int i = 0; i < chunk && rc == CHNS_OK; ++i) rc = step(cs, i);
      // an even chunk ends with an odd iteration, which leaves r.r in slot 0
      cudaMemcpyAsync((void*)(slot + v), c.S + kCgRr0, sizeof(double), cudaMemcpyDeviceToHost, cs);
      per_graph = chns_launches_now() - l0;
      cudaError_t e1 = cudaStreamEndCapture(cs, &g);
      if (rc != CHNS_OK) {
        if (g) cudaGraphDestroy(g);
        break;
      }
      // on a failure below, fall through to the cleanup loop so that the graph and event of
      // the other instance are released too
      if (e1 != cudaSuccess) {
        rc = cuda_fail(e1, "cudaStreamEndCapture");
        break;
      }
      cudaError_t e2 = cudaGraphInstantiate(&ge[v], g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) {
        ge[v] = nullptr;
        rc = cuda_fail(e2, "cudaGraphInstantiate");
        break;
      }
      cudaError_t e3 = cudaEventCreateWithFlags(&ev[v], cudaEventDisableTiming);
      if (e3 != cudaSuccess) {
        ev[v] = nullptr;
        rc = cuda_fail(e3, "cudaEventCreateWithFlags");
        break;
      }
    }
    note_launches_undo(2 * per_graph);  // captured, not executed
    if (rc == CHNS_OK) {
      int k = 0;
      bool done = false;
      auto ok = [&](cudaError_t e, const char* what) {
        if (e == cudaSuccess) return true;
        rc = cuda_fail(e, what);
        return false;
      };
      while (!done) {
        const int v = k & 1;
        if (!ok(cudaGraphLaunch(ge[v], c.s), "cudaGraphLaunch")) break;
        note_launches(per_graph);
        if (!ok(cudaEventRecord(ev[v], c.s), "cudaEventRecord")) break;
        it += chunk;
        // check the previous chunk while this one runs
        if (k >= 1) {
          if (!ok(cudaEventSynchronize(ev[v ^ 1]), "cudaEventSynchronize")) break;
          rr = slot[v ^ 1];
          if (bad(rr) || std::sqrt(rr) <= tol_abs || stalled(it - chunk, rr)) done = true;
        }
        if (done || it >= max_it) {
          if (!ok(cudaEventSynchronize(ev[v]), "cudaEventSynchronize")) break;
          rr = slot[v];
          done = true;
        }
        ++k;
      }
    }
    for (int v = 0; v < 2; ++v) {
      if (ge[v]) cudaGraphExecDestroy(ge[v]);
      if (ev[v]) cudaEventDestroy(ev[v]);
    }
    if (rc != CHNS_OK) return rc;
    if (!std::isfinite(rr)) {
      *iters = it;
      *rnorm = rr;
      set_error("krylov: NaN/Inf in the residual norm");
      return CHNS_ENAN;
    }
  }
  CHNS_CUDA(cudaGetLastError());
  *iters = it;
  *rnorm = std::sqrt(rr);
  return std::sqrt(rr) <= tol_abs ? CHNS_OK : CHNS_ENOTCONV;
}

// Preconditioned CG on A x = b (type T); x holds the initial guess. Runs until sqrt(r.r) <= tol_abs
// or max_it iterations (see iterate).
template <class T>
chns_status pcg(const Ctx& c, const T* b, T* x, const T* dinv, double tol_abs, int max_it,
                int chunk, T* r, T* z, T* p, T* q, T* p2, int* iters, double* rnorm,
                const Snap* snap = nullptr) {
  T* pb[2] = {p, p2};  // direction buffers: iteration k reads pb[k & 1], writes pb[(k & 1) ^ 1]
  const int64_t n = c.n;
  const unsigned rg = red_grid(c.m, n), vg = vgrid(c.m, n);
  chns_status st = apply_T<T>(c, x, q);
  if (st != CHNS_OK) return st;
  note_launch();
  k_axpby<T><<<vg, kVecThreads, 0, c.s>>>(1.0, b, -1.0, q, r, n);
  if (c.op == CHNS_OP_POISSON) project_mean<T>(c, r);
  note_launch();
  k_mul<T><<<vg, kVecThreads, 0, c.s>>>(dinv, r, z, n);
  // p_old = 0 and rz_prev = rz_cur make the first direction p = z
  CHNS_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), c.s));
  CHNS_CUDA(cudaMemsetAsync(q, 0, n * sizeof(T), c.s));
  note_launch();
  k_dot<T, T><<<rg, kVecThreads, 0, c.s>>>(r, z, n, c.m->ws.red, c.m->ws.counter, c.S + kCgRz0);
  CHNS_CUDA(cudaMemcpyAsync(c.S + kCgRzPrev, c.S + kCgRz0, sizeof(double),
                            cudaMemcpyDeviceToDevice, c.s));
  CHNS_CUDA(cudaMemsetAsync(c.S + kCgPq0, 0, sizeof(double), c.s));
  note_launch();
  k_dot<T, T><<<rg, kVecThreads, 0, c.s>>>(r, r, n, c.m->ws.red, c.m->ws.counter, c.S + kCgRr0);
  CHNS_CUDA(cudaGetLastError());
  double rr = 0.0;
  st = read_dev(c.m, c.S + kCgRr0, &rr, 1, c.s);
  if (st != CHNS_OK) return st;
  auto step = [&](cudaStream_t s, int it) {
    return cg_iteration<T>(c, s, x, r, z, pb[it & 1], pb[(it & 1) ^ 1], q, dinv, it & 1);
  };
  return iterate<T>(c, step, x, tol_abs, max_it, chunk, rr, iters, rnorm, snap);
}

// `iters` Jacobi-CG iterations on A x = b from x = 0 with no host synchronisation (the scalars
// stay in the parity slots; see cg_iteration); an inexact inner solve.
template <class T>
chns_status cg_fixed(const Ctx& c, const T* b, T* x, const T* dinv, int iters, T* r, T* z, T* p,
                     T* q, T* p2) {
  T* pb[2] = {p, p2};
  const int64_t n = c.n;
  const unsigned rg = red_grid(c.m, n), vg = vgrid(c.m, n);
  CHNS_CUDA(cudaMemsetAsync(x, 0, n * sizeof(T), c.s));
  CHNS_CUDA(cudaMemcpyAsync(r, b, n * sizeof(T), cudaMemcpyDeviceToDevice, c.s));
  note_launch();
  k_mul<T><<<vg, kVecThreads, 0, c.s>>>(dinv, r, z, n);
  CHNS_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), c.s));
  note_launch();
  k_dot<T, T><<<rg, kVecThreads, 0, c.s>>>(r, z, n, c.m->ws.red, c.m->ws.counter, c.S + kCgRz0);
  CHNS_CUDA(cudaMemcpyAsync(c.S + kCgRzPrev, c.S + kCgRz0, sizeof(double),
                            cudaMemcpyDeviceToDevice, c.s));
  CHNS_CUDA(cudaMemsetAsync(c.S + kCgPq0, 0, sizeof(double), c.s));
  for (int it = 0; it < iters; ++it) {
    chns_status st = cg_iteration<T>(c, c.s, x, r, z, pb[it & 1], pb[(it & 1) ^ 1], q, dinv, it & 1);
    if (st != CHNS_OK) return st;
  }
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

// Block upper-triangular preconditioner of the CH Newton Jacobian J = [A B; C D] (rows phi, mu;
// B = kmu K, C = (psi'' M + Cn^2 K)/2, D = -M/2): P = [S~ B; 0 D] with the Schur complement
// S = A - B D^-1 C = M/dt - adv + kmu K M^-1 M_psi'' + 2 kmu kphi K M^-1 K approximated by
// S~ = H M^-1 H, H = sqrt(1/dt) M + sqrt(2 kmu kphi) K (= M/dt + 2 kmu kphi K M^-1 K + a cross
// term 2 sqrt(2 kmu kphi / dt) K). J P^-1 is similar to a unit lower-triangular matrix when
// S~ = S. Applying P^-1 to (r_phi, r_mu):
//   z_mu = D^-1 r_mu = -2 M^-1 r_mu;  z_phi = S~^-1 (r_phi - B z_mu) = H^-1 M H^-1 (...),
// with the M and H inverses replaced by fixed numbers of Jacobi-CG iterations.
template <class T>
struct SchurPC {
  Ctx cM, cH, cK;        // N-vector contexts: M, H, kmu K
  T* dM = nullptr;       // inverse diagonals of M and H
  T* dH = nullptr;
  T* t[8] = {};          // scratch N-vectors: CG r, z, p, q, p2; t, w, u
  int itH = 20, itM = 5;
  chns_mg* mg = nullptr;  // when set, each H^-1 is one V-cycle of the shifted operator H

  // contexts and diagonals; vec: >= 10 scratch N-vectors
  chns_status setup(const Ctx& c, T* const* vec, int inner_its, chns_mg* hier = nullptr,
                    int mass_its = 0) {
    const int64_t N = c.m->d.n_nodes;
    const double dt = c.prm->dt, Pe = c.prm->Pe, Cn = c.prm->Cn;
    const double kmu = 0.5 / (Pe * Cn), kphi = 0.5 * Cn * Cn;
    itH = inner_its > 0 ? inner_its : 20;
    itM = mass_its > 0 ? mass_its : std::max(4, itH / 4);
    cM = c;
    cM.op = kOpShift;
    cM.n = N;
    cM.sa = 1.0;
    cM.sb = 0.0;
    cH = cM;
    cH.sa = std::sqrt(1.0 / dt);
    cH.sb = std::sqrt(2.0 * kmu * kphi);
    cK = cM;
    cK.sa = 0.0;
    cK.sb = kmu;
    for (int k = 0; k < 8; ++k) t[k] = vec[2 + k];
    const chns_precision pr = sizeof(T) == sizeof(double) ? CHNS_FP64 : CHNS_FP32;
    const void* phi = sizeof(T) == sizeof(double) ? c.coef64->phi_tilde : c.coefR.phi_tilde;
    mg = hier;
    if (mg) {  // H has constant coefficients: the hierarchy keeps its setup between solves
      chns_status st = mg_setup_shifted(mg, c.prm, cH.sa, cH.sb, pr, c.s);
      if (st != CHNS_OK) return st;
    }
    // the inverse diagonals of M and H, kept on the mesh between solves with the same constants
    auto& sd = c.m->sd;
    const int pi = sizeof(T) == sizeof(double) ? 0 : 1;
    const double key[4] = {cM.sa, cM.sb, cH.sa, cH.sb};
    for (int k = 0; k < 2; ++k)
      if (!sd.d[pi][k]) CHNS_CUDA(cudaMalloc(&sd.d[pi][k], N * sizeof(T)));
    dM = static_cast<T*>(sd.d[pi][0]);
    dH = static_cast<T*>(sd.d[pi][1]);
    bool same = sd.valid[pi];
    for (int k = 0; k < 4 && same; ++k) same = sd.key[pi][k] == key[k];
    if (same) return CHNS_OK;
    sd.valid[pi] = false;
    chns_status st = diag_shift(c.m, c.prm, phi, cM.sa, cM.sb, dM, pr, c.s);
    if (st != CHNS_OK) return st;
    st = diag_shift(c.m, c.prm, phi, cH.sa, cH.sb, dH, pr, c.s);
    if (st != CHNS_OK) return st;
    note_launch();
    k_invert<T, T><<<vgrid(c.m, N), kVecThreads, 0, c.s>>>(dM, dM, N);
    note_launch();
    k_invert<T, T><<<vgrid(c.m, N), kVecThreads, 0, c.s>>>(dH, dH, N);
    CHNS_CUDA(cudaGetLastError());
    for (int k = 0; k < 4; ++k) sd.key[pi][k] = key[k];
    sd.valid[pi] = true;
    return CHNS_OK;
  }

  // z = P^-1 v for the pair [phi; mu] (2N each; z must not alias v)
  chns_status apply(const T* v, T* z) {
    const int64_t N = cM.n;
    const unsigned vg = vgrid(cM.m, N);
    const T* vphi = v;
    const T* vmu = v + N;
    T* zphi = z;
    T* zmu = z + N;
    T *r = t[0], *zz = t[1], *p = t[2], *q = t[3], *p2 = t[4], *tt = t[5], *w = t[6], *u = t[7];
    chns_status st = cg_fixed<T>(cM, vmu, zmu, dM, itM, r, zz, p, q, p2);
    if (st != CHNS_OK) return st;
    note_launch();
    k_scale<T><<<vg, kVecThreads, 0, cM.s>>>(zmu, -2.0, N);
    st = apply_T<T>(cK, zmu, tt);
    if (st != CHNS_OK) return st;
    note_launch();
    k_axpby<T><<<vg, kVecThreads, 0, cM.s>>>(1.0, vphi, -1.0, tt, u, N);
    if (mg)
      st = mg_vcycle<T>(mg, kMgShifted, u, w, cM.s);
    else
      st = cg_fixed<T>(cH, u, w, dH, itH, r, zz, p, q, p2);
    if (st != CHNS_OK) return st;
    st = apply_T<T>(cM, w, tt);
    if (st != CHNS_OK) return st;
    if (mg)
      st = mg_vcycle<T>(mg, kMgShifted, tt, zphi, cM.s);
    else
      st = cg_fixed<T>(cH, tt, zphi, dH, itH, r, zz, p, q, p2);
    if (st != CHNS_OK) return st;
    CHNS_CUDA(cudaGetLastError());
    return CHNS_OK;
  }
};

// Flexible CG on the Poisson operator with the preconditioner z = M(r): with L the learned
// correction c followed by one damped Jacobi step, z = c + omega dinv (r - A c) (w: scratch
// vector); with cheb the Chebyshev polynomial (scratch w, dcheb); else Jacobi (dinv) or the
// identity.
template <class T>
chns_status fcg(const Ctx& c, const T* b, T* x, const T* dinv, chns_learned* L, double tol_abs,
                int max_it, int chunk, T* r, T* z, T* p, T* q, T* p2, T* w, int* iters,
                double* rnorm, int stall = 0, const Snap* snap = nullptr,
                const Cheb* cheb = nullptr, T* dcheb = nullptr, chns_mg* mg = nullptr) {
  T* pb[2] = {p, p2};
  const int64_t n = c.n;
  const unsigned rg = red_grid(c.m, n), vg = vgrid(c.m, n);
  // rr_slot: where r.r of the current residual is
  auto precond = [&](cudaStream_t s, int rr_slot) -> chns_status {
    if (L) {
      chns_status e = learned_precondition<T>(L, c.m, r, nullptr, c.S + rr_slot, z, s);
      if (e != CHNS_OK) return e;
      Ctx cs = c;
      cs.s = s;
      e = apply_T<T>(cs, z, w);
      if (e != CHNS_OK) return e;
      note_launch();
      k_smooth<T><<<vg, kVecThreads, 0, s>>>(z, r, w, dinv, (T)kLearnedOmega, n);
      return CHNS_OK;
    }
    if (cheb) return cheb_apply<T>(c, s, *cheb, dinv, r, z, w, dcheb);
    if (mg) return mg_vcycle<T>(mg, kMgPoisson, r, z, s);
    note_launch();
    if (dinv) k_mul<T><<<vg, kVecThreads, 0, s>>>(dinv, r, z, n);
    else k_axpby<T><<<vg, kVecThreads, 0, s>>>(1.0, r, 0.0, r, z, n);
    return CHNS_OK;
  };
  chns_status st = apply_T<T>(c, x, q);
  if (st != CHNS_OK) return st;
  note_launch();
  k_axpby<T><<<vg, kVecThreads, 0, c.s>>>(1.0, b, -1.0, q, r, n);
  project_mean<T>(c, r);
  note_launch();
  k_dot<T, T><<<rg, kVecThreads, 0, c.s>>>(r, r, n, c.m->ws.red, c.m->ws.counter, c.S + kCgRr0);
  st = precond(c.s, kCgRr0);
  if (st != CHNS_OK) return st;
  note_launch();
  k_dot<T, T><<<rg, kVecThreads, 0, c.s>>>(r, z, n, c.m->ws.red, c.m->ws.counter, c.S + kFcgRz0);
  note_launch();
  k_fcg_init<<<1, 1, 0, c.s>>>(c.S);
  CHNS_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), c.s));
  CHNS_CUDA(cudaMemsetAsync(q, 0, n * sizeof(T), c.s));
  CHNS_CUDA(cudaGetLastError());
  double rr = 0.0;
  st = read_dev(c.m, c.S + kCgRr0, &rr, 1, c.s);
  if (st != CHNS_OK) return st;
  auto step = [&](cudaStream_t s, int it) -> chns_status {
    const int par = it & 1;
    T* p_old = pb[par];
    T* p_new = pb[par ^ 1];
    chns_status e;
    if (sizeof(T) == sizeof(double))
      e = apply_poisson_cg(c.m, c.prm, c.coef64, z, p_old, p_new, q, CHNS_FP64, c.S, par, s, true);
    else
      e = apply_poisson_cg(c.m, c.prm, &c.coefR, z, p_old, p_new, q, c.inner, c.S, par, s, true);
    if (e != CHNS_OK) return e;
    note_launch();
    k_fcg_update<T><<<rg, kVecThreads, 0, s>>>(x, r, p_new, q, n, c.S, par);
    e = precond(s, kCgRr0 + (par ^ 1));
    if (e != CHNS_OK) return e;
    note_launch();
    k_fcg_dots<T><<<rg, kVecThreads, 0, s>>>(z, q, r, n, c.S, par);
    return CHNS_OK;
  };
  return iterate<T>(c, step, x, tol_abs, max_it, chunk, rr, iters, rnorm, snap, stall);
}

// multi-dot launch: (chunks, nk + 1) blocks, about four per SM in total; returns the chunk count
template <class T>
unsigned multidot(const chns_mesh* m, const T* V, int64_t ld, int nk, const T* w, int64_t n,
                  double* part, cudaStream_t s) {
  const int64_t want = 4 * (int64_t)m->sm_count / (nk + 1);
  const unsigned chunks = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>({std::max<int64_t>(want, 8), (n + kMd2Threads - 1) / kMd2Threads,
                            (int64_t)kMdMaxBlocks}));
  note_launch();
  k_multidot2<T><<<dim3(chunks, nk + 1), kMd2Threads, 0, s>>>(V, ld, nk, w, n, part);
  return chunks;
}

// Right-preconditioned restarted GMRES with classical Gram-Schmidt and one re-orthogonalisation
// pass; the second pass also returns w.w so that the new norm needs no extra reduction.
template <class T>
chns_status gmres(const Ctx& c, const T* b, T* x, const T* dinv, bool block2, double tol_abs,
                  int max_it, int restart, T* V, T* z, int* iters, double* rnorm,
                  SchurPC<T>* spc = nullptr) {
  const int64_t n = c.n, ld = n;
  // flexible form (spc): the preconditioned vectors Z_j = P^-1 V_j follow the restart + 1 basis
  // vectors in the same buffer, and the update is x += Z y
  T* Zb = V + (int64_t)(restart + 1) * ld;
  const unsigned vg = vgrid(c.m, n);
  const unsigned mdb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(kMdBlocks, (n + 255) / 256));
  double* hdev = c.S + S_MD;
  std::vector<double> H((size_t)(restart + 1) * restart, 0.0), cs(restart), sn(restart),
      g(restart + 1), y(restart), h(restart + 2);
  int it = 0;
  double beta = 0.0;
  chns_status st;
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * restart + j]; };
  for (;;) {
    // r = b - A x into V_0
    st = apply_T<T>(c, x, z);
    if (st != CHNS_OK) return st;
    note_launch();
    k_axpby<T><<<vg, kVecThreads, 0, c.s>>>(1.0, b, -1.0, z, V, n);
    st = dot_to_host<T>(c, V, V, &beta);
    if (st != CHNS_OK) return st;
    beta = std::sqrt(beta);
    if (!std::isfinite(beta)) {
      set_error("krylov: NaN/Inf in the residual norm");
      *iters = it;
      *rnorm = beta;
      return CHNS_ENAN;
    }
    if (beta <= tol_abs || it >= max_it) break;
    note_launch();
    k_scale<T><<<vg, kVecThreads, 0, c.s>>>(V, 1.0 / beta, n);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < restart; ++j) {
      T* vj = V + (int64_t)j * ld;
      T* w = V + (int64_t)(j + 1) * ld;
      T* zj = spc ? Zb + (int64_t)j * ld : z;
      if (spc) {
        st = spc->apply(vj, zj);
        if (st != CHNS_OK) return st;
      } else {
        note_launch();
        if (block2)
          k_mul_b2<T><<<vg, kVecThreads, 0, c.s>>>(dinv, vj, z, n / 2);
        else
          k_mul<T><<<vg, kVecThreads, 0, c.s>>>(dinv, vj, z, n);
      }
      st = apply_T<T>(c, zj, w);
      if (st != CHNS_OK) return st;
      // classical Gram-Schmidt: h = V^T w and w.w in one pass; a second pass only when the
      // new vector lost more than half its norm to the projection (cancellation)
      int nk = j + 1;
      const unsigned md2 = multidot(c.m, V, ld, nk, w, n, c.m->ws.md_part, c.s);
      note_launch();
      k_multidot_final<<<nk + 1, kVecThreads, 0, c.s>>>(c.m->ws.md_part, (int)md2, hdev);
      CHNS_CUDA(cudaGetLastError());
      st = read_dev(c.m, hdev, h.data(), nk + 1, c.s);
      if (st != CHNS_OK) return st;
      double hh = 0.0;
      for (int i = 0; i <= j; ++i) {
        Hij(i, j) = h[i];
        hh += h[i] * h[i];
      }
      double ww = h[nk];
      double hn2 = ww - hh;
      if (!(hn2 > 0.5 * ww)) {
        // re-orthogonalise: w -= V h, then a second multi-dot on the updated vector
        orth_update<T, false>(V, ld, nk, hdev, w, n, vg, c.s);
        multidot(c.m, V, ld, nk, w, n, c.m->ws.md_part, c.s);
        note_launch();
        k_multidot_final<<<nk + 1, kVecThreads, 0, c.s>>>(c.m->ws.md_part, (int)md2, hdev);
        CHNS_CUDA(cudaGetLastError());
        st = read_dev(c.m, hdev, h.data(), nk + 1, c.s);
        if (st != CHNS_OK) return st;
        double h2 = 0.0;
        for (int i = 0; i <= j; ++i) {
          Hij(i, j) += h[i];
          h2 += h[i] * h[i];
        }
        hn2 = h[nk] - h2;
      }
      const double hn = std::sqrt(std::max(0.0, hn2));
      Hij(j + 1, j) = hn;
      if (!std::isfinite(hn)) {
        set_error("krylov: NaN/Inf in GMRES");
        *iters = it;
        *rnorm = hn;
        return CHNS_ENAN;
      }
      if (hn > 0.0) {
        orth_update<T, true>(V, ld, nk, hdev, w, n, vg, c.s);
      }
      // Givens rotations
      for (int i = 0; i < j; ++i) {
        double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      double a = Hij(j, j), bb = Hij(j + 1, j);
      double rden = std::hypot(a, bb);
      cs[j] = rden > 0.0 ? a / rden : 1.0;
      sn[j] = rden > 0.0 ? bb / rden : 0.0;
      Hij(j, j) = rden;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      jend = j + 1;
      if (std::fabs(g[j + 1]) <= tol_abs || it >= max_it || hn == 0.0) break;
    }
    // back substitution and update x += M^-1 V y
    for (int i = jend - 1; i >= 0; --i) {
      double acc = g[i];
      for (int k = i + 1; k < jend; ++k) acc -= Hij(i, k) * y[k];
      y[i] = Hij(i, i) != 0.0 ? acc / Hij(i, i) : 0.0;
    }
    CHNS_CUDA(cudaMemcpyAsync(hdev, y.data(), jend * sizeof(double), cudaMemcpyHostToDevice, c.s));
    note_launch();
    if (spc)
      k_gmres_update<T><<<vg, kVecThreads, 0, c.s>>>(Zb, ld, jend, hdev, nullptr, x, n);
    else if (block2)
      k_gmres_update_b2<T><<<vg, kVecThreads, 0, c.s>>>(V, ld, jend, hdev, dinv, x, n / 2);
    else
      k_gmres_update<T><<<vg, kVecThreads, 0, c.s>>>(V, ld, jend, hdev, dinv, x, n);
    CHNS_CUDA(cudaGetLastError());
    CHNS_CUDA(cudaStreamSynchronize(c.s));  // y (host) is reused next cycle
  }
  *iters = it;
  *rnorm = beta;
  return beta <= tol_abs ? CHNS_OK : CHNS_ENOTCONV;
}

}  // namespace

// Convert the FP64 coefficient fields of an operator to the inner precision (workspace copies).
static chns_status make_reduced_coef(const chns_mesh* m, const chns_coef* c, chns_precision prec,
                                     chns_coef* out, cudaStream_t s) {
  const int64_t N = m->d.n_nodes;
  const void* src[5] = {c->phi_tilde, c->u_adv[0], c->u_adv[1], c->u_adv[2], c->mu_tilde};
  void* dst[5];
  for (int k = 0; k < 5; ++k) {
    dst[k] = nullptr;
    if (!src[k]) continue;
    if (prec == CHNS_FP32) {
      float* d = static_cast<float*>(m->ws.coef32) + k * N;
      vec_convert_f64_f32(static_cast<const double*>(src[k]), d, N, s);
      dst[k] = d;
    } else {
      __nv_bfloat16* d = static_cast<__nv_bfloat16*>(m->ws.coef16) + k * N;
      // phi~ is stored as 1 + phi~ (see gather_phi), the other fields as they are
      vec_convert_f64_bf16(static_cast<const double*>(src[k]), d, N, k == 0 ? 1.0 : 0.0, s);
      dst[k] = d;
    }
  }
  out->phi_tilde = dst[0];
  out->u_adv[0] = dst[1];
  out->u_adv[1] = dst[2];
  out->u_adv[2] = dst[3];
  out->mu_tilde = dst[4];
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status krylov_solve(const chns_mesh* m, chns_operator op, const chns_params* prm,
                         const chns_coef* coef, const double* b_in, double* x,
                         const chns_solver_params* sp, chns_solve_stats* stats, cudaStream_t s) {
  CHNS_CHECK(m && prm && coef && b_in && x && sp, CHNS_EINVAL, "chns_krylov_solve: null argument");
  CHNS_CHECK(op >= CHNS_OP_POISSON && op <= CHNS_OP_MOMENTUM, CHNS_EINVAL, "bad operator");
  CHNS_CHECK(sp->ksp == CHNS_KSP_CG || sp->ksp == CHNS_KSP_GMRES || sp->ksp == CHNS_KSP_FCG,
             CHNS_EINVAL, "bad ksp");
  CHNS_CHECK(sp->pc == CHNS_PC_NONE || sp->pc == CHNS_PC_JACOBI || sp->pc == CHNS_PC_LEARNED ||
                 sp->pc == CHNS_PC_CHEBYSHEV || sp->pc == CHNS_PC_SCHUR ||
                 sp->pc == CHNS_PC_MULTIGRID,
             CHNS_EINVAL, "bad preconditioner");
  CHNS_CHECK(sp->pc != CHNS_PC_MULTIGRID ||
                 (op == CHNS_OP_POISSON && sp->ksp != CHNS_KSP_GMRES && sp->mg &&
                  !sp->mg->lv.empty() && sp->mg->lv[0].mesh == m),
             CHNS_EINVAL, "multigrid: Poisson operator, CG or FCG, and a hierarchy of this mesh");
  CHNS_CHECK(sp->pc != CHNS_PC_SCHUR || !sp->mg || (!sp->mg->lv.empty() && sp->mg->lv[0].mesh == m),
             CHNS_EINVAL, "Schur preconditioner: the multigrid hierarchy is not of this mesh");
  // flexible GMRES keeps restart preconditioned vectors beside the restart + 1 basis vectors of
  // 2 n_nodes in the basis buffer of (CHNS_GMRES_MAX_RESTART + 1) x 3 n_nodes
  CHNS_CHECK(sp->pc != CHNS_PC_SCHUR ||
                 (op == CHNS_OP_CH && sp->ksp == CHNS_KSP_GMRES && sp->inner_its >= 0 &&
                  sp->mass_its >= 0 &&
                  2 * (2 * sp->restart + 1) <= 3 * (CHNS_GMRES_MAX_RESTART + 1)),
             CHNS_EINVAL,
             "Schur preconditioner: CH operator, GMRES, restart <= 30, inner_its and mass_its >= 0");
  CHNS_CHECK(sp->pc != CHNS_PC_CHEBYSHEV ||
                 (op == CHNS_OP_POISSON && sp->ksp != CHNS_KSP_GMRES && sp->restart >= 1 &&
                  sp->restart <= 16),
             CHNS_EINVAL, "Chebyshev: Poisson operator, CG or FCG, degree (restart) 1..16");
  CHNS_CHECK(sp->ksp != CHNS_KSP_FCG || op == CHNS_OP_POISSON, CHNS_EINVAL,
             "FCG is implemented for the Poisson operator only");
  CHNS_CHECK(sp->pc != CHNS_PC_LEARNED || (sp->ksp == CHNS_KSP_FCG && sp->learned), CHNS_EINVAL,
             "the learned preconditioner needs FCG and solver_params.learned");
  CHNS_CHECK(sp->rtol > 0.0 && sp->max_it >= 0, CHNS_EINVAL, "bad tolerance / max_it");
  CHNS_CHECK(sp->ksp != CHNS_KSP_GMRES ||
                 (sp->restart >= 1 && sp->restart <= CHNS_GMRES_MAX_RESTART),
             CHNS_EINVAL, "GMRES restart out of range");
  CHNS_CHECK(sp->inner_precision >= CHNS_FP64 && sp->inner_precision <= CHNS_FP32_BF16COEF,
             CHNS_EINVAL, "bad inner precision");
  CHNS_CHECK(sp->fp64_apply == CHNS_FP64 || sp->fp64_apply == CHNS_FP64_DF, CHNS_EINVAL,
             "krylov: fp64_apply must be CHNS_FP64 or CHNS_FP64_DF");
  const Workspace& ws = m->ws;
  const int nc = op_ncomp(op);
  const int64_t n = nc * m->d.n_nodes;
  // momentum quadrature data (set up below) is valid only within this solve
  struct QdGuard {
    const chns_mesh* m;
    ~QdGuard() { momentum_qdata_off(m); }
  } qd_guard{m};
  cudaEvent_t e0, e1;
  CHNS_CUDA(cudaEventCreate(&e0));
  CHNS_CUDA(cudaEventCreate(&e1));
  CHNS_CUDA(cudaEventRecord(e0, s));

  Ctx c{};
  c.m = m;
  c.op = op;
  c.prm = prm;
  c.coef64 = coef;
  c.inner = (chns_precision)sp->inner_precision;
  c.s = s;
  c.n = n;
  c.S = scal(m);
  c.df = sp->fp64_apply == CHNS_FP64_DF;

  // workspace layout (FP64): 0 b (projected), 1 r64, 2 dinv64/diag, 3..6 CG vectors,
  // 7 GMRES z; (FP32): 0 r32, 1 d32, 2 dinv32, 3..6 CG vectors, 7 GMRES z
  double* b = ws.v64[0];
  double* r64 = ws.v64[1];
  double* d64 = ws.v64[2];
  CHNS_CUDA(cudaMemcpyAsync(b, b_in, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  chns_status st = CHNS_OK;
  if (op == CHNS_OP_POISSON) {
    st = project_mean<double>(c, b);
    if (st != CHNS_OK) return st;
  }
  double bn2 = 0.0;
  st = dot_to_host<double>(c, b, b, &bn2);
  if (st != CHNS_OK) return st;
  const double bnorm = std::sqrt(bn2);
  chns_solve_stats out{};
  out.b_norm = bnorm;
  out.final_precision = sp->inner_precision;
  if (bnorm == 0.0) {
    CHNS_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  } else {
    // Jacobi preconditioner: the operator's exact diagonal (2x2 nodal blocks for the CH pair,
    // whose phi and mu unknowns are strongly coupled), computed in the precision of the Krylov
    // iteration that uses it.
    // the learned preconditioner is additive with the Jacobi smoother
    const bool jac = sp->pc == CHNS_PC_JACOBI || sp->pc == CHNS_PC_LEARNED ||
                     sp->pc == CHNS_PC_CHEBYSHEV;
    // the Chebyshev preconditioner runs through the flexible-CG driver (with a fixed SPD
    // preconditioner its iterates are those of PCG)
    const bool cheb = sp->pc == CHNS_PC_CHEBYSHEV;
    // the V-cycle preconditioner also runs through the flexible-CG driver
    chns_mg* mg = sp->pc == CHNS_PC_MULTIGRID ? sp->mg : nullptr;
    const bool use_fcg = sp->ksp == CHNS_KSP_FCG || cheb || mg;
    Cheb cheb64, cheb32;
    chns_learned* L = sp->pc == CHNS_PC_LEARNED ? sp->learned : nullptr;
    if (L) {
      st = learned_begin_solve(L, m, prm, coef, s);
      if (st != CHNS_OK) return st;
    }
    const bool block2 = (op == CHNS_OP_CH && jac);
    const int64_t Nn = m->d.n_nodes;
    // Schur-complement preconditioner of the CH pair, per precision on first use (scratch:
    // workspace vectors 3..6, twelve node vectors, free during GMRES)
    const bool schur = sp->pc == CHNS_PC_SCHUR;
    SchurPC<double> spc64;
    SchurPC<float> spc32;
    bool spc64_ok = false, spc32_ok = false;
    // the FP64 preconditioner (nullptr when not used); *err receives a setup failure
    auto schur64 = [&](chns_status* err) -> SchurPC<double>* {
      *err = CHNS_OK;
      if (!schur) return nullptr;
      if (!spc64_ok) {
        double* vec[12];
        for (int k = 0; k < 12; ++k) vec[k] = ws.v64[3 + k / 3] + (k % 3) * Nn;
        *err = spc64.setup(c, vec, sp->inner_its, sp->mg, sp->mass_its);
        if (*err != CHNS_OK) return nullptr;
        spc64_ok = true;
      }
      return &spc64;
    };
    const double* dinv64 = nullptr;
    auto make_dinv64 = [&]() -> chns_status {
      if (!jac || dinv64) return CHNS_OK;
      chns_status r;
      if (block2) {
        double* d4 = ws.coef64 + 11 * Nn;
        r = block_diag_ch(m, prm, coef, d4, CHNS_FP64, s);
        if (r != CHNS_OK) return r;
        note_launch();
        k_invert_b2<double, double><<<vgrid(m, Nn), kVecThreads, 0, s>>>(d4, d4, Nn);
        dinv64 = d4;
      } else {
        r = diag_op(m, op, prm, coef, d64, CHNS_FP64, s);
        if (r != CHNS_OK) return r;
        note_launch();
        k_invert<double, double><<<vgrid(m, n), kVecThreads, 0, s>>>(d64, d64, n);
        dinv64 = d64;
      }
      return CHNS_OK;
    };
    const double tol = sp->rtol * bnorm;
    double last_rn = -1.0;  // FP64 residual norm of the current x, when known
    if (c.inner == CHNS_FP64) {
      if (op == CHNS_OP_MOMENTUM) {
        st = momentum_qdata_on(m, prm, coef, nullptr, s);
        if (st != CHNS_OK) return st;
      }
      st = make_dinv64();
      if (st != CHNS_OK) return st;
      int its = 0;
      double rn = 0.0;
      if (cheb) {
        st = cheb_bounds<double>(c, dinv64, b, ws.v64[14], ws.v64[15], sp->restart, &cheb64);
        if (st != CHNS_OK) return st;
      }
      if (mg) {
        st = mg_setup(mg, prm, coef->phi_tilde, CHNS_FP64, s);
        if (st != CHNS_OK) return st;
      }
      if (sp->ksp == CHNS_KSP_CG && !cheb && !mg)
        st = pcg<double>(c, b, x, dinv64, tol, sp->max_it, sp->check_every, r64, ws.v64[3],
                         ws.v64[4], ws.v64[5], ws.v64[6], &its, &rn);
      else if (use_fcg) {
        st = fcg<double>(c, b, x, dinv64, L, tol, sp->max_it, sp->check_every, r64, ws.v64[3],
                         ws.v64[4], ws.v64[5], ws.v64[6], ws.v64[7], &its, &rn,
                         L ? kLearnedStall : 0, nullptr, cheb ? &cheb64 : nullptr, ws.v64[14],
                         mg);
        if (L && st == CHNS_ENOTCONV && its < sp->max_it) {
          // the learned correction stalled: Jacobi-PCG from the current iterate
          ++out.fallbacks;
          int its2 = 0;
          st = pcg<double>(c, b, x, dinv64, tol, sp->max_it - its, sp->check_every, r64,
                           ws.v64[3], ws.v64[4], ws.v64[5], ws.v64[6], &its2, &rn);
          its += its2;
        }
      }
      else {
        SchurPC<double>* pc64 = schur64(&st);
        if (st != CHNS_OK) return st;
        st = gmres<double>(c, b, x, dinv64, block2, tol, sp->max_it, sp->restart, ws.gm_V,
                           ws.v64[7], &its, &rn, pc64);
      }
      out.iterations = its;
    } else {
      // FP32 coefficient copies; the preconditioner is computed from them in FP32.
      chns_coef coef32;
      st = make_reduced_coef(m, coef, CHNS_FP32, &coef32, s);
      if (st != CHNS_OK) return st;
      if (op == CHNS_OP_MOMENTUM) {
        st = momentum_qdata_on(m, prm, coef, &coef32, s);
        if (st != CHNS_OK) return st;
      }
      float* r32 = ws.v32[0];
      float* d32 = ws.v32[1];
      float* dinv32 = nullptr;
      if (block2) {
        dinv32 = static_cast<float*>(ws.coef32) + 6 * Nn;
        st = block_diag_ch(m, prm, &coef32, dinv32, CHNS_FP32, s);
        if (st != CHNS_OK) return st;
        note_launch();
        k_invert_b2<float, float><<<vgrid(m, Nn), kVecThreads, 0, s>>>(dinv32, dinv32, Nn);
      } else if (jac) {
        dinv32 = ws.v32[2];
        st = diag_op(m, op, prm, &coef32, dinv32, CHNS_FP32, s);
        if (st != CHNS_OK) return st;
        note_launch();
        k_invert<float, float><<<vgrid(m, n), kVecThreads, 0, s>>>(dinv32, dinv32, n);
      }
      // bfloat16 coefficient storage only where the apply is memory bound (Poisson, mass); the
      // CH and momentum applies are arithmetic bound and use mu~ through its gradient.
      if (c.inner == CHNS_FP32_BF16COEF && (op == CHNS_OP_POISSON || op == CHNS_OP_MASS)) {
        st = make_reduced_coef(m, coef, CHNS_FP32_BF16COEF, &c.coefR, s);
        if (st != CHNS_OK) return st;
      } else {
        c.inner = CHNS_FP32;
        c.coefR = coef32;
      }
      int total = 0, refine = 0;
      bool learned_ok = true;
      bool mg32_ready = false;
      last_rn = -1.0;
      double prev_rn = 0.0;
      chns_precision cur = c.inner;
      (void)d32;
      for (;;) {
        // r64 = b - A_64 x (r64 = b for a zero initial guess, e.g. a Newton correction: the
        // FP64 apply is the most expensive kernel of a cycle)
        bool x_zero = false;
        if (total == 0 && refine == 0) {
          double xx = 0.0;
          st = dot_to_host<double>(c, x, x, &xx);
          if (st != CHNS_OK) return st;
          x_zero = xx == 0.0;
        }
        if (x_zero) {
          CHNS_CUDA(cudaMemcpyAsync(r64, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else {
          st = apply_op(m, op, prm, coef, x, r64, c.df ? CHNS_FP64_DF : CHNS_FP64, s);
          if (st != CHNS_OK) return st;
          note_launch();
          k_axpby<double><<<vgrid(m, n), kVecThreads, 0, s>>>(1.0, b, -1.0, r64, r64, n);
          if (op == CHNS_OP_POISSON) project_mean<double>(c, r64);
        }
        double rn2 = 0.0;
        st = dot_to_host<double>(c, r64, r64, &rn2);
        if (st != CHNS_OK) return st;
        const double rn = std::sqrt(rn2);
        last_rn = rn;
        if (!std::isfinite(rn)) {
          set_error("krylov: NaN/Inf in the refinement residual");
          st = CHNS_ENAN;
          break;
        }
        if (rn <= tol) {
          st = CHNS_OK;
          break;
        }
        if (total >= sp->max_it || refine >= sp->max_refine) {
          st = CHNS_ENOTCONV;
          break;
        }
        // A cycle that did not halve the FP64 residual means the reduced-precision operator is
        // too far from the FP64 one: raise the inner precision (BF16 coefficients -> FP32 ->
        // FP64 Krylov on the remaining correction).
        if (refine > 0 && rn > 0.25 * prev_rn) {
          ++out.escalations;
          if (cur == CHNS_FP32_BF16COEF) {
            cur = CHNS_FP32;
            c.inner = cur;
            c.coefR = coef32;
          } else {
            st = make_dinv64();
            if (st != CHNS_OK) return st;
            int its = 0;
            double frn = 0.0;
            if (cheb && cheb64.degree == 0) {
              st = cheb_bounds<double>(c, dinv64, b, ws.v64[14], ws.v64[15], sp->restart,
                                       &cheb64);
              if (st != CHNS_OK) return st;
            }
            if (mg) {
              st = mg_setup(mg, prm, coef->phi_tilde, CHNS_FP64, s);
              if (st != CHNS_OK) return st;
            }
            if (sp->ksp == CHNS_KSP_CG && !cheb && !mg)
              st = pcg<double>(c, b, x, dinv64, tol, sp->max_it - total, sp->check_every, r64,
                               ws.v64[3], ws.v64[4], ws.v64[5], ws.v64[6], &its, &frn);
            else if (use_fcg)
              st = fcg<double>(c, b, x, dinv64, nullptr, tol, sp->max_it - total,
                               sp->check_every, r64, ws.v64[3], ws.v64[4], ws.v64[5], ws.v64[6],
                               ws.v64[7], &its, &frn, 0, nullptr, cheb ? &cheb64 : nullptr,
                               ws.v64[14], mg);
            else {
              SchurPC<double>* pc64 = schur64(&st);
              if (st != CHNS_OK) return st;
              st = gmres<double>(c, b, x, dinv64, block2, tol, sp->max_it - total, sp->restart,
                                 ws.gm_V, ws.v64[7], &its, &frn, pc64);
            }
            total += its;
            cur = CHNS_FP64;
            last_rn = -1.0;
            break;
          }
        }
        prev_rn = rn;
        const double scale = 1.0 / rn;
        note_launch();
        k_convert<double, float><<<vgrid(m, n), kVecThreads, 0, s>>>(r64, r32, n, scale);
        CHNS_CUDA(cudaMemsetAsync(d32, 0, n * sizeof(float), s));
        int its = 0;
        double irn = 0.0;
        const double itol = std::max(sp->inner_rtol, 0.5 * tol / rn);
        // Each cycle gets a bounded number of iterations: an FP32 iteration that stagnates above
        // its tolerance then falls through to the FP64 residual check (and escalation) instead
        // of spending the whole budget.
        const int cap = sp->ksp == CHNS_KSP_GMRES ? 4 * sp->restart : std::max(1000, sp->max_it / 4);
        const int budget = std::min(sp->max_it - total, cap);
        chns_status ist;
        if (cheb && cheb32.degree == 0) {
          st = cheb_bounds<float>(c, dinv32, r32, ws.v32[9], ws.v32[7], sp->restart, &cheb32);
          if (st != CHNS_OK) return st;
        }
        if (mg && !mg32_ready) {
          st = mg_setup(mg, prm, coef32.phi_tilde, CHNS_FP32, s);
          if (st != CHNS_OK) return st;
          mg32_ready = true;
        }
        if (sp->ksp == CHNS_KSP_CG && !cheb && !mg)
          ist = pcg<float>(c, r32, d32, dinv32, itol, budget, sp->check_every, ws.v32[3],
                           ws.v32[4], ws.v32[5], ws.v32[6], ws.v32[8], &its, &irn);
        else if (use_fcg) {
          chns_learned* Lc = learned_ok ? L : nullptr;
          ist = fcg<float>(c, r32, d32, dinv32, Lc, itol, budget, sp->check_every, ws.v32[3],
                           ws.v32[4], ws.v32[5], ws.v32[6], ws.v32[8], ws.v32[7], &its, &irn,
                           Lc ? kLearnedStall : 0, nullptr, cheb ? &cheb32 : nullptr,
                           ws.v32[9], mg);
          if (Lc && ist == CHNS_ENOTCONV && its < budget) {
            // the learned correction stalled: Jacobi only from the next refinement cycle on
            learned_ok = false;
            ++out.fallbacks;
          }
        }
        else {
          if (schur && !spc32_ok) {
            float* vec[12];
            for (int k = 0; k < 12; ++k) vec[k] = ws.v32[3 + k / 3] + (k % 3) * Nn;
            st = spc32.setup(c, vec, sp->inner_its, sp->mg, sp->mass_its);
            if (st != CHNS_OK) return st;
            spc32_ok = true;
          }
          ist = gmres<float>(c, r32, d32, dinv32, block2, itol, budget, sp->restart, ws.gm_V32,
                             ws.v32[7], &its, &irn, schur ? &spc32 : nullptr);
        }
        if (ist != CHNS_OK && ist != CHNS_ENOTCONV) return ist;
        total += its;
        ++refine;
        note_launch();
        k_accumulate<float><<<vgrid(m, n), kVecThreads, 0, s>>>(x, d32, rn, n);
        last_rn = -1.0;
        if (its == 0) {
          st = CHNS_ENOTCONV;
          break;
        }
      }
      out.final_precision = cur;
      out.iterations = total;
      out.refinements = refine;
    }
    if (op == CHNS_OP_POISSON) project_mean<double>(c, x);
    if (last_rn >= 0.0) {
      // the refinement loop ended on an FP64 residual of this very x (removing the mean of a
      // Poisson solution does not change it): no second FP64 apply
      out.rel_residual = last_rn / bnorm;
    } else {
      // true FP64 residual
      chns_status st2 = apply_op(m, op, prm, coef, x, r64, c.df ? CHNS_FP64_DF : CHNS_FP64, s);
      if (st2 != CHNS_OK) return st2;
      note_launch();
      k_axpby<double><<<vgrid(m, n), kVecThreads, 0, s>>>(1.0, b, -1.0, r64, r64, n);
      if (op == CHNS_OP_POISSON) project_mean<double>(c, r64);
      double rr = 0.0;
      st2 = dot_to_host<double>(c, r64, r64, &rr);
      if (st2 != CHNS_OK) return st2;
      out.rel_residual = std::sqrt(rr) / bnorm;
    }
    if (st == CHNS_ENOTCONV && out.rel_residual <= sp->rtol) st = CHNS_OK;
  }
  CHNS_CUDA(cudaEventRecord(e1, s));
  CHNS_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  out.ms = ms;
  out.status = st;
  if (stats) *stats = out;
  if (st == CHNS_ENOTCONV) set_error("krylov: iteration limit reached before the tolerance");
  return st;
}

chns_status pcg_snapshots(const chns_mesh* m, const chns_params* prm, const chns_coef* coef,
                          const double* b_in, double rtol, int every, int max_snaps, double* snaps,
                          int* n_snaps, double* x, cudaStream_t s, chns_learned* L) {
  CHNS_CHECK(every >= 1 && max_snaps >= 0, CHNS_EINVAL, "pcg_snapshots: bad sampling");
  const Workspace& ws = m->ws;
  const int64_t n = m->d.n_nodes;
  Ctx c{};
  c.m = m;
  c.op = CHNS_OP_POISSON;
  c.prm = prm;
  c.coef64 = coef;
  c.inner = CHNS_FP64;
  c.s = s;
  c.n = n;
  c.S = scal(m);
  double* b = ws.v64[0];
  double* d = ws.v64[2];
  CHNS_CUDA(cudaMemcpyAsync(b, b_in, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  chns_status st = project_mean<double>(c, b);
  if (st != CHNS_OK) return st;
  double bn2 = 0.0;
  st = dot_to_host<double>(c, b, b, &bn2);
  if (st != CHNS_OK) return st;
  *n_snaps = 0;
  CHNS_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  if (bn2 == 0.0) return CHNS_OK;
  st = diag_op(m, CHNS_OP_POISSON, prm, coef, d, CHNS_FP64, s);
  if (st != CHNS_OK) return st;
  note_launch();
  k_invert<double, double><<<vgrid(m, n), kVecThreads, 0, s>>>(d, d, n);
  Snap sn{snaps, every, max_snaps, n_snaps};
  int its = 0;
  double rn = 0.0;
  const double tol = rtol * std::sqrt(bn2);
  if (L) {
    // iterates of FCG with the network's own correction; if it stalls, Jacobi-PCG finishes the
    // solve (without snapshots) so that x is the converged solution
    st = learned_begin_solve(L, m, prm, coef, s);
    if (st != CHNS_OK) return st;
    st = fcg<double>(c, b, x, d, L, tol, 100000, 1, ws.v64[1], ws.v64[3], ws.v64[4], ws.v64[5],
                     ws.v64[6], ws.v64[7], &its, &rn, kLearnedStall, &sn);
    if (st == CHNS_ENOTCONV)
      st = pcg<double>(c, b, x, d, tol, 100000, 1, ws.v64[1], ws.v64[3], ws.v64[4], ws.v64[5],
                       ws.v64[6], &its, &rn);
  } else {
    st = pcg<double>(c, b, x, d, tol, 100000, 1, ws.v64[1], ws.v64[3], ws.v64[4], ws.v64[5],
                     ws.v64[6], &its, &rn, &sn);
  }
  if (st != CHNS_OK) return st;
  return project_mean<double>(c, x);
}

}  // namespace chns

extern "C" chns_status chns_krylov_solve(const chns_mesh* m, chns_operator op,
                                         const chns_params* prm, const chns_coef* coef,
                                         const double* b, double* x, const chns_solver_params* sp,
                                         chns_solve_stats* stats, void* stream) {
  return chns::krylov_solve(m, op, prm, coef, b, x, sp, stats, chns::as_stream(stream));
}
