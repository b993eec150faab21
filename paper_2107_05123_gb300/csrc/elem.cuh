// Device building blocks of the matrix-free operators: Q1 basis on box leaves with 2x2x2 Gauss
// quadrature (Sec. 4.1, r = 1), gather with hanging-node interpolation and the transposed
// scatter-add (the top-down copy / bottom-up accumulate of Sec. 5.4 "Traversal-based Vector
// Assembly", done here with flat index tables).
//
// Element-local numbering: corner a has bits (a&1, a>>1&1, a>>2&1) for (x, y, z); quadrature
// point q uses the same bit layout with xi = -1/sqrt(3) for bit 0 and +1/sqrt(3) for bit 1.
// Along one axis the Q1 basis at the Gauss points is B = [[W0, W1], [W1, W0]] (symmetric) and the
// reference derivative is (u1 - u0)/2 at both points.
#pragma once

#include "dfloat.cuh"
#include "internal.h"

namespace chns {

constexpr double kW0 = 0.78867513459481288225;  // (1 + 1/sqrt(3)) / 2
constexpr double kW1 = 0.21132486540518711775;  // (1 - 1/sqrt(3)) / 2

// Physical parameters in device form (Sec. 3: rho(phi) = alpha phi + beta, eta = gamma phi + xi)
// with every quotient the kernels need precomputed on the host, in the kernel's own precision:
// the device code multiplies only (on GB300 an FP64 division inside an FP32 kernel costs more
// than the whole FP32 element computation around it).
template <class T>
struct PrmT {
  T alpha, beta, gamma, xi, C_I;
  T dt, idt, four_idt2, k2dt, half_dt;  // dt, 1/dt, 4/dt^2, 2/dt, dt/2
  T inv_re, h2re, inv_pe, h2pe;         // 1/Re, 1/(2Re), 1/Pe, 1/(2Pe)
  T inv_pecn, kmu, kphi, cn2;           // 1/(Pe Cn), 1/(2 Pe Cn), Cn^2/2, Cn^2
  T ka, cw, inv_fr;                     // -alpha/Cn, Cn/We, 1/Fr
  T sa, sb;  // constant-coefficient operator sa M + sb K (set per call by its apply, else 0)
};

struct DevParams {
  PrmT<double> d;
  PrmT<float> f;
  PrmT<DF> x;  // the FP64 values split into double-float
  template <class T>
  __host__ __device__ __forceinline__ const PrmT<T>& get() const;
};
template <>
__host__ __device__ __forceinline__ const PrmT<double>& DevParams::get<double>() const { return d; }
template <>
__host__ __device__ __forceinline__ const PrmT<float>& DevParams::get<float>() const { return f; }
template <>
__host__ __device__ __forceinline__ const PrmT<DF>& DevParams::get<DF>() const { return x; }

template <class T>
inline PrmT<T> make_prm(const chns_params& p) {
  const double rp = 1.0, rm = 1.0 / p.rho_ratio, ep = 1.0, em = 1.0 / p.eta_ratio;
  const double alpha = (rp - rm) / (2 * rp), beta = (rp + rm) / (2 * rp);
  const double gamma = (ep - em) / (2 * ep), xi = (ep + em) / (2 * ep);
  PrmT<T> q;
  q.alpha = (T)alpha;
  q.beta = (T)beta;
  q.gamma = (T)gamma;
  q.xi = (T)xi;
  q.C_I = (T)p.C_I;
  q.dt = (T)p.dt;
  q.idt = (T)(1.0 / p.dt);
  q.four_idt2 = (T)(4.0 / (p.dt * p.dt));
  q.k2dt = (T)(2.0 / p.dt);
  q.half_dt = (T)(0.5 * p.dt);
  q.inv_re = (T)(1.0 / p.Re);
  q.h2re = (T)(0.5 / p.Re);
  q.inv_pe = (T)(1.0 / p.Pe);
  q.h2pe = (T)(0.5 / p.Pe);
  q.inv_pecn = (T)(1.0 / (p.Pe * p.Cn));
  q.kmu = (T)(0.5 / (p.Pe * p.Cn));
  q.kphi = (T)(0.5 * p.Cn * p.Cn);
  q.cn2 = (T)(p.Cn * p.Cn);
  q.ka = (T)(-alpha / p.Cn);
  q.cw = (T)(p.Cn / p.We);
  q.inv_fr = (T)(1.0 / p.Fr);
  q.sa = q.sb = (T)0;
  return q;
}

inline DevParams make_dev_params(const chns_params& p) {
  DevParams d;
  d.d = make_prm<double>(p);
  d.f = make_prm<float>(p);
  d.x = make_prm<DF>(p);
  return d;
}

// Storage type of values computed in arithmetic type T (FP64 for double-float) and the shared
// accumulator type of the patch applies (the same).
template <class T>
using AccumT = typename std::conditional<std::is_same<T, DF>::value, double, T>::type;

template <class T>
__device__ __forceinline__ T clamp1(T v) {
  return v > T(1) ? T(1) : (v < T(-1) ? T(-1) : v);
}

// ---- loads with conversion from the storage type
template <class T>
__device__ __forceinline__ T ldv(const double* p, int64_t i) { return (T)__ldg(p + i); }
template <class T>
__device__ __forceinline__ T ldv(const float* p, int64_t i) { return (T)__ldg(p + i); }
template <class T>
__device__ __forceinline__ T ldv(const __nv_bfloat16* p, int64_t i) {
  return (T)__bfloat162float(p[i]);
}

// ---- element geometry from the octant level (never stored): h_d = L_d 2^-level
template <class T>
struct Geo {
  T h[3];
  T ih[3];
  T detJ;  // h_x h_y h_z / 8 (Gauss weights are 1)
};

template <class T>
__device__ __forceinline__ Geo<T> level_geometry(const MeshDev& m, int level) {
  const LevelGeo& L = m.geo[level];
  Geo<T> g;
  if constexpr (std::is_same<T, double>::value) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      g.h[d] = L.h[d];
      g.ih[d] = L.ih[d];
    }
    g.detJ = L.detJ;
  } else if constexpr (std::is_same<T, DF>::value) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      g.h[d] = DF(L.h[d]);
      g.ih[d] = DF(L.ih[d]);
    }
    g.detJ = DF(L.detJ);
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      g.h[d] = L.hf[d];
      g.ih[d] = L.ihf[d];
    }
    g.detJ = L.detJf;
  }
  return g;
}

template <class T>
__device__ __forceinline__ Geo<T> geometry(const MeshDev& m, int64_t e) {
  return level_geometry<T>(m, m.level[e]);
}

__device__ __forceinline__ void load_corners(const MeshDev& m, int64_t e, int idx[8]) {
  int4 a = __ldg(m.enode + 2 * e);
  int4 b = __ldg(m.enode + 2 * e + 1);
  idx[0] = a.x; idx[1] = a.y; idx[2] = a.z; idx[3] = a.w;
  idx[4] = b.x; idx[5] = b.y; idx[6] = b.z; idx[7] = b.w;
}

// Value of one node reference (with Dirichlet flag) from a nodal array; DIR zeroes flagged nodes.
template <class T, bool DIR, class S>
__device__ __forceinline__ T node_val(const S* x, int v) {
  if (DIR && (v & kDirBit)) return T(0);
  return ldv<T>(x, v & kIdxMask);
}

// Gather the 8 corner values of an element; hanging corners are interpolated from their parents
// (edge midpoint: mean of 2, face centre: mean of 4).
template <class T, bool DIR, class S>
__device__ __forceinline__ void gather(const MeshDev& m, const int idx[8], const S* x, T out[8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    int v = idx[a];
    int j = v & kIdxMask;
    if (j < m.n_nodes) {
      out[a] = node_val<T, DIR>(x, v);
    } else {
      int4 h = __ldg(m.hang + (j - m.n_nodes));
      T s = node_val<T, DIR>(x, h.x) + node_val<T, DIR>(x, h.y);
      if (h.z < 0) {
        out[a] = T(0.5) * s;
      } else {
        s += node_val<T, DIR>(x, h.z) + node_val<T, DIR>(x, h.w);
        out[a] = T(0.25) * s;
      }
    }
  }
}

template <class S>
__device__ __forceinline__ void atomic_add(S* p, S v) { atomicAdd(p, v); }

// Transposed gather: add the element vector into the nodal output, distributing hanging corners
// to their parents with the same weights. DIR skips flagged (Dirichlet) rows.
template <class T, bool DIR, class S>
__device__ __forceinline__ void scatter(const MeshDev& m, const int idx[8], const T r[8], S* y) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    int v = idx[a];
    int j = v & kIdxMask;
    if (j < m.n_nodes) {
      if (!(DIR && (v & kDirBit))) atomic_add(y + j, (S)r[a]);
    } else {
      int4 h = __ldg(m.hang + (j - m.n_nodes));
      bool four = h.z >= 0;
      S w = (S)(four ? T(0.25) * r[a] : T(0.5) * r[a]);
      if (!(DIR && (h.x & kDirBit))) atomic_add(y + (h.x & kIdxMask), w);
      if (!(DIR && (h.y & kDirBit))) atomic_add(y + (h.y & kIdxMask), w);
      if (four) {
        if (!(DIR && (h.z & kDirBit))) atomic_add(y + (h.z & kIdxMask), w);
        if (!(DIR && (h.w & kDirBit))) atomic_add(y + (h.w & kIdxMask), w);
      }
    }
  }
}

// ---- sum-factorised Q1 kernels
// o0 = W0 a + W1 b and o1 = W1 a + W0 b, written with W0 = 1 - W1 as a + W1 (b - a) and
// b - W1 (b - a): one subtraction and two fused multiply-adds.
template <class T>
__device__ __forceinline__ void interp1(T a, T b, T& o0, T& o1) {
  const T d = b - a;
  o0 = a + T(kW1) * d;
  o1 = b - T(kW1) * d;
}

// 2D interpolation of 4 values (i0 + 2 i1) to the 4 Gauss points; B symmetric => self-transpose.
template <class T>
__device__ __forceinline__ void interp2(const T in[4], T out[4]) {
  T t[4];
  interp1(in[0], in[1], t[0], t[1]);
  interp1(in[2], in[3], t[2], t[3]);
  interp1(t[0], t[2], out[0], out[2]);
  interp1(t[1], t[3], out[1], out[3]);
}

// 3D interpolation of corner values to the 8 Gauss points (self-transpose).
template <class T>
__device__ __forceinline__ void interp3(const T u[8], T v[8]) {
  T t[8], s[8];
#pragma unroll
  for (int j = 0; j < 4; ++j) interp1(u[2 * j], u[2 * j + 1], t[2 * j], t[2 * j + 1]);
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) interp1(t[x + 4 * z], t[x + 2 + 4 * z], s[x + 4 * z], s[x + 2 + 4 * z]);
#pragma unroll
  for (int i = 0; i < 4; ++i) interp1(s[i], s[i + 4], v[i], v[i + 4]);
}

// Reference-gradient data of an element: gx depends on (qy,qz) only, gy on (qx,qz), gz on (qx,qy);
// each is the bilinear interpolation of the 4 edge differences along that axis. Physical
// gradient = g / h (the factor 2/h of the Jacobian times the 1/2 of the 1D derivative).
template <class T>
__device__ __forceinline__ void grad_compact(const T u[8], T gx[4], T gy[4], T gz[4]) {
  T d[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) d[j] = u[2 * j + 1] - u[2 * j];  // j = y + 2z
  interp2(d, gx);
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) d[x + 2 * z] = u[x + 2 + 4 * z] - u[x + 4 * z];
  interp2(d, gy);
#pragma unroll
  for (int j = 0; j < 4; ++j) d[j] = u[j + 4] - u[j];  // j = x + 2y
  interp2(d, gz);
}

// Transpose of grad_compact for per-axis sums over the free Gauss coordinate:
// r_a += sign(a_d) * interp2(S_d)[other bits of a] * scale_d.
template <class T>
__device__ __forceinline__ void grad_compact_T(const T sx[4], const T sy[4], const T sz[4],
                                               const T sc[3], T r[8]) {
  T t[4];
  interp2(sx, t);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    r[2 * j + 1] += sc[0] * t[j];
    r[2 * j] -= sc[0] * t[j];
  }
  interp2(sy, t);
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      r[x + 2 + 4 * z] += sc[1] * t[x + 2 * z];
      r[x + 4 * z] -= sc[1] * t[x + 2 * z];
    }
  interp2(sz, t);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    r[j + 4] += sc[2] * t[j];
    r[j] -= sc[2] * t[j];
  }
}

// Physical gradient components at Gauss point Q from the compact data of grad_compact:
// d/dx at (qy, qz) = gx[Q >> 1] / h_x, d/dy at (qx, qz) = gy[(Q & 1) + 2 (Q >> 2)] / h_y,
// d/dz at (qx, qy) = gz[Q & 3] / h_z.
__device__ __forceinline__ constexpr int gxi(int Q) { return Q >> 1; }
__device__ __forceinline__ constexpr int gyi(int Q) { return (Q & 1) + 2 * (Q >> 2); }
__device__ __forceinline__ constexpr int gzi(int Q) { return Q & 3; }

// r_a += sum_q grad N_a(q) . V_q for per-point vectors V[d][q] (physical units, quadrature
// weights and coefficients included): the x component of grad N_a does not depend on qx, so V_x
// is first summed over qx (likewise y, z), then the compact transpose applies.
template <class T>
__device__ __forceinline__ void grad_T(const T V[3][8], const Geo<T>& g, T r[8]) {
  T sx[4], sy[4], sz[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    sx[j] = V[0][2 * j] + V[0][2 * j + 1];
    sz[j] = V[2][j] + V[2][j + 4];
  }
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) sy[x + 2 * z] = V[1][x + 4 * z] + V[1][x + 2 + 4 * z];
  const T sc[3] = {g.ih[0], g.ih[1], g.ih[2]};
  grad_compact_T(sx, sy, sz, sc, r);
}

// ---- per-quadrature-point evaluation (direct; used by the multi-field operators)
__device__ __forceinline__ constexpr double b1(int a, int q) { return a == q ? kW0 : kW1; }
__device__ __forceinline__ constexpr double sg(int a) { return a ? 1.0 : -1.0; }

// N_a(q), and the reference factor of dN_a/dx_d(q) * h_d  (= sign * product of the other two B)
__device__ __forceinline__ constexpr double Nq(int a, int q) {
  return b1(a & 1, q & 1) * b1((a >> 1) & 1, (q >> 1) & 1) * b1((a >> 2) & 1, (q >> 2) & 1);
}
__device__ __forceinline__ constexpr double dNq(int a, int q, int d) {
  return d == 0 ? sg(a & 1) * b1((a >> 1) & 1, (q >> 1) & 1) * b1((a >> 2) & 1, (q >> 2) & 1)
       : d == 1 ? sg((a >> 1) & 1) * b1(a & 1, q & 1) * b1((a >> 2) & 1, (q >> 2) & 1)
                : sg((a >> 2) & 1) * b1(a & 1, q & 1) * b1((a >> 1) & 1, (q >> 1) & 1);
}

// value and physical gradient at quadrature point Q of an element field u[8]
template <int Q, class T>
__device__ __forceinline__ void vg_at(const T u[8], const Geo<T>& g, T& v, T gr[3]) {
  v = T(0);
  gr[0] = gr[1] = gr[2] = T(0);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    v += T(Nq(a, Q)) * u[a];
    gr[0] += T(dNq(a, Q, 0)) * u[a];
    gr[1] += T(dNq(a, Q, 1)) * u[a];
    gr[2] += T(dNq(a, Q, 2)) * u[a];
  }
  gr[0] *= g.ih[0];
  gr[1] *= g.ih[1];
  gr[2] *= g.ih[2];
}

template <int Q, class T>
__device__ __forceinline__ T val_at(const T u[8]) {
  T v = T(0);
#pragma unroll
  for (int a = 0; a < 8; ++a) v += T(Nq(a, Q)) * u[a];
  return v;
}

// r_a += N_a(Q) s + grad N_a(Q) . V   (V already in physical units; scaled here by 1/h)
template <int Q, class T>
__device__ __forceinline__ void add_test(T r[8], T s, const T V[3], const Geo<T>& g) {
  T vx = V[0] * g.ih[0], vy = V[1] * g.ih[1], vz = V[2] * g.ih[2];
#pragma unroll
  for (int a = 0; a < 8; ++a)
    r[a] += T(Nq(a, Q)) * s + T(dNq(a, Q, 0)) * vx + T(dNq(a, Q, 1)) * vy + T(dNq(a, Q, 2)) * vz;
}

// Mixed second derivatives of the trilinear interpolant at Q: H_xy, H_xz, H_yz (pure ones vanish).
template <int Q, class T>
__device__ __forceinline__ void hess_at(const T u[8], const Geo<T>& g, T& hxy, T& hxz, T& hyz) {
  const int qx = Q & 1, qy = (Q >> 1) & 1, qz = (Q >> 2) & 1;
  T dxy[2], dxz[2], dyz[2];
#pragma unroll
  for (int z = 0; z < 2; ++z) dxy[z] = u[3 + 4 * z] - u[2 + 4 * z] - u[1 + 4 * z] + u[4 * z];
#pragma unroll
  for (int y = 0; y < 2; ++y) dxz[y] = u[5 + 2 * y] - u[4 + 2 * y] - u[1 + 2 * y] + u[2 * y];
#pragma unroll
  for (int x = 0; x < 2; ++x) dyz[x] = u[6 + x] - u[4 + x] - u[2 + x] + u[x];
  hxy = (T(b1(0, qz)) * dxy[0] + T(b1(1, qz)) * dxy[1]) * g.ih[0] * g.ih[1];
  hxz = (T(b1(0, qy)) * dxz[0] + T(b1(1, qy)) * dxz[1]) * g.ih[0] * g.ih[2];
  hyz = (T(b1(0, qx)) * dyz[0] + T(b1(1, qx)) * dyz[1]) * g.ih[1] * g.ih[2];
}

// Compile-time loop over the 8 quadrature points.
template <int Q = 0, class F>
__device__ __forceinline__ void for_qp(F&& f) {
  if constexpr (Q < 8) {
    f(std::integral_constant<int, Q>{});
    for_qp<Q + 1>(f);
  }
}

}  // namespace chns
