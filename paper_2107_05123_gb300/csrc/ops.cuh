// Element operators of the CHNS scheme (Sec. 4.1), each as a small struct with
//   load(...)  : gather the element's coefficient fields (hanging-interpolated) and prepare
//                per-quadrature-point data,
//   apply(...) : local y_e = A_e x_e for NC components.
// The same structs drive the matrix-free apply kernel and the exact diagonal kernel.
#pragma once

#include <type_traits>

#include "elem.cuh"

namespace chns {

template <class C>
struct CoefArgs {
  const C* phi;     // phi~ (bfloat16 storage holds 1 + phi~, see phi_shift)
  const C* u[3];    // advecting velocity (u_hat or u~)
  const C* mu;      // mu~
  float phi_shift;  // added to the stored phi values: -1 for bfloat16 storage, else 0
  const void* qd = nullptr;  // quadrature data of operators that precompute it (MomQK)
};

// Gather phi~ of an element. In bfloat16 storage the field is s = 1 + phi~, whose relative
// precision bounds the relative error of rho(phi) = alpha s + rho_- by 2^-8 even where
// rho_- << 1 (phi near -1); the shift is removed after interpolation (linear in s).
template <class T, class C>
__device__ __forceinline__ void gather_phi(const MeshDev& m, const int idx[8],
                                           const CoefArgs<C>& cf, T pe[8]) {
  gather<T, false>(m, idx, cf.phi, pe);
#pragma unroll
  for (int a = 0; a < 8; ++a) pe[a] += T(cf.phi_shift);
}

// ---------------------------------------------------------------- pressure Poisson
// (grad q, (1/rho(phi~*)) grad p) (Def. weak_VMS_disc_pp_vel, scalar test q).
template <class T>
__device__ __forceinline__ void poisson_coef(const T pe[8], const Geo<T>& g, const DevParams& p,
                                             T c[8]) {
  T pq[8];
  interp3(pe, pq);
  const PrmT<T>& k = p.get<T>();
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const T den = k.alpha * clamp1(pq[q]) + k.beta;  // rho in [rho_-, rho_+], far from 0
    if constexpr (std::is_same<T, float>::value)
      c[q] = __fdividef(g.detJ, den);  // a few ulp; the FP32 applies feed FP64-refined solves
    else
      c[q] = g.detJ / den;
  }
}

// Sum-factorised local stiffness apply with a per-quadrature-point coefficient c[q]:
// r_a = sum_q c_q grad N_a(q) . grad u(q). With E, *e = u . r = sum_q c_q |grad u(q)|^2, formed
// from the per-axis gradient data (a sum of non-negative terms for c >= 0, so it is accurate in
// the working precision; u . r itself cancels).
template <class T, bool E = false>
__device__ __forceinline__ void stiff_local(const T c[8], const Geo<T>& g, const T u[8], T r[8],
                                            T* e = nullptr) {
  T gx[4], gy[4], gz[4];
  grad_compact(u, gx, gy, gz);
  T sx[4], sy[4], sz[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) sx[j] = gx[j] * (c[2 * j] + c[2 * j + 1]);
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) sy[x + 2 * z] = gy[x + 2 * z] * (c[x + 4 * z] + c[x + 2 + 4 * z]);
#pragma unroll
  for (int k = 0; k < 4; ++k) sz[k] = gz[k] * (c[k] + c[k + 4]);
  const T sc[3] = {g.ih[0] * g.ih[0], g.ih[1] * g.ih[1], g.ih[2] * g.ih[2]};
#pragma unroll
  for (int a = 0; a < 8; ++a) r[a] = T(0);
  grad_compact_T(sx, sy, sz, sc, r);
  if constexpr (E) {
    T ex = T(0), ey = T(0), ez = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ex += gx[j] * sx[j];
      ey += gy[j] * sy[j];
      ez += gz[j] * sz[j];
    }
    *e = sc[0] * ex + sc[1] * ey + sc[2] * ez;
  }
}

template <class T, class C>
struct PoissonK {
  static constexpr bool QDATA = false;
  // CTAs of the patch apply resident per SM that the register allocation must allow (FP32: 6,
  // i.e. at most 42 registers; FP64: 3)
  static constexpr int MIN_CTAS = sizeof(T) == 4 ? 6 : 3;
  static constexpr int STREAM_CTAS = sizeof(T) == 4 ? 6 : 0;  // persistent apply (0: not used)
  static constexpr int NC = 1;
  static constexpr bool DIR = false;
  static constexpr bool DIAG_PER_COMP = false;
  static constexpr int NF = 1;  // coefficient fields: phi~
  T c[8];
  __device__ __forceinline__ void setup(const T f[NF][8], const Geo<T>& g, const DevParams& p) {
    poisson_coef(f[0], g, p, c);
  }
  __device__ __forceinline__ void load(const MeshDev& m, const DevParams& p, const CoefArgs<C>& cf,
                                       const int idx[8], const Geo<T>& g) {
    T f[NF][8];
    gather_phi(m, idx, cf, f[0]);
    setup(f, g, p);
  }
  __device__ __forceinline__ void apply(const Geo<T>& g, const DevParams&, const T x[NC][8],
                                        T r[NC][8]) const {
    stiff_local(c, g, x[0], r[0]);
  }
  // apply and the element energy x . A_e x (see stiff_local)
  static constexpr bool ENERGY = true;
  __device__ __forceinline__ T apply_energy(const Geo<T>& g, const DevParams&, const T x[NC][8],
                                            T r[NC][8]) const {
    T e;
    stiff_local<T, true>(c, g, x[0], r[0], &e);
    return e;
  }
};

// ---------------------------------------------------------------- velocity update mass
// (w, rho~ u) per component (Def. weak_VMS_disc_vel_update); Dirichlet rows are identity.
template <class T, class C>
struct MassK {
  static constexpr bool QDATA = false;
  static constexpr int MIN_CTAS = sizeof(T) == 4 ? 5 : 3;
  static constexpr int STREAM_CTAS = sizeof(T) == 4 ? 3 : 0;  // persistent apply (0: not used)
  static constexpr int NC = 3;
  static constexpr bool DIR = true;
  static constexpr bool DIAG_PER_COMP = false;
  static constexpr int NF = 1;  // phi~
  T c[8];
  __device__ __forceinline__ void setup(const T f[NF][8], const Geo<T>& g, const DevParams& p) {
    T pq[8];
    interp3(f[0], pq);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const PrmT<T>& k = p.get<T>();
      c[q] = g.detJ * (k.alpha * clamp1(pq[q]) + k.beta);
    }
  }
  __device__ __forceinline__ void load(const MeshDev& m, const DevParams& p, const CoefArgs<C>& cf,
                                       const int idx[8], const Geo<T>& g) {
    T f[NF][8];
    gather_phi(m, idx, cf, f[0]);
    setup(f, g, p);
  }
  __device__ __forceinline__ void apply(const Geo<T>&, const DevParams&, const T x[NC][8],
                                        T r[NC][8]) const {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      T v[8];
      interp3(x[k], v);
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] *= c[q];
      interp3(v, r[k]);
    }
  }
};

// ---------------------------------------------------------------- shifted Laplacian
// sa (q, u) + sb (grad q, grad u) with constant sa, sb >= 0 (DevParams sa, sb): the operator of
// the inner solves of the Cahn-Hilliard Schur-complement preconditioner. No Dirichlet rows.
template <class T, class C>
struct ShiftK {
  static constexpr bool QDATA = false;
  static constexpr int MIN_CTAS = sizeof(T) == 4 ? 6 : 3;
  static constexpr int STREAM_CTAS = sizeof(T) == 4 ? 6 : 0;  // persistent apply (FP32)
  static constexpr int NC = 1;
  static constexpr bool DIR = false;
  static constexpr bool DIAG_PER_COMP = false;
  static constexpr int NF = 1;  // (phi~ gathered but unused: the patch kernel's layout)
  static constexpr bool IGNORES_FIELDS = true;
  // Constant coefficients on a box: the 2x2x2 Gauss rule is exact, and the element matrices are
  // Kronecker products of the 1D Q1 matrices m = h/6 [[2, 1], [1, 2]] and k = 1/h [[1, -1],
  // [-1, 1]]: M_e = m x m x m, K_e = k x m x m + m x k x m + m x m x k. With P(a, b) = (2a + b,
  // a + 2b) and D(a, b) = (a - b, b - a) along one axis and V = h_x h_y h_z,
  //   y = sa M_e x + sb K_e x = Px (cm B + cy C + cz E) + cx Dx B,
  //   B = Py Pz x, C = Dy Pz x, E = Py Dz x, cm = sa V / 216, c_d = sb V / (36 h_d^2).
  T cm, cx, cy, cz;
  __device__ __forceinline__ void setup(const T[NF][8], const Geo<T>& g, const DevParams& p) {
    const PrmT<T>& k = p.get<T>();
    const T V = T(8) * g.detJ;
    cm = k.sa * V * T(1.0 / 216.0);
    const T ks = k.sb * V * T(1.0 / 36.0);
    cx = ks * g.ih[0] * g.ih[0];
    cy = ks * g.ih[1] * g.ih[1];
    cz = ks * g.ih[2] * g.ih[2];
  }
  __device__ __forceinline__ void load(const MeshDev&, const DevParams& p, const CoefArgs<C>&,
                                       const int[8], const Geo<T>& g) {
    const T f[NF][8] = {};
    setup(f, g, p);
  }
  // sb = 0 (the mass M of the Schur preconditioner) skips the stiffness part: the branch is
  // uniform over the whole launch
  __device__ __forceinline__ void apply(const Geo<T>&, const DevParams&, const T x[NC][8],
                                        T r[NC][8]) const {
    const T* X = x[0];
    T u[8], B[8], S[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // P along z: pairs (j, j + 4)
      u[j] = T(2) * X[j] + X[j + 4];
      u[j + 4] = X[j] + T(2) * X[j + 4];
    }
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
      for (int i = 0; i < 2; ++i) {  // P along y: pairs (i + 4z, i + 2 + 4z)
        const int a = i + 4 * z, b = a + 2;
        B[a] = T(2) * u[a] + u[b];
        B[b] = u[a] + T(2) * u[b];
      }
    if (cx == T(0) && cy == T(0) && cz == T(0)) {
#pragma unroll
      for (int a = 0; a < 8; ++a) S[a] = cm * B[a];
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // P along x: pairs (2j, 2j + 1)
        r[0][2 * j] = T(2) * S[2 * j] + S[2 * j + 1];
        r[0][2 * j + 1] = S[2 * j] + T(2) * S[2 * j + 1];
      }
      return;
    }
    T w[4];  // Dz x on the z = 0 layer (the z = 1 layer is its negative)
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = X[j] - X[j + 4];
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int a = i + 4 * z, b = a + 2;
        const T c = u[a] - u[b];                      // Dy Pz x
        const T e0 = T(2) * w[i] + w[i + 2];           // Py Dz x at (i, 0)
        const T e1 = w[i] + T(2) * w[i + 2];           // ... at (i, 1)
        const T sgn = z ? T(-1) : T(1);
        S[a] = cm * B[a] + cy * c + cz * (sgn * e0);
        S[b] = cm * B[b] - cy * c + cz * (sgn * e1);
      }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T dx = cx * (B[2 * j] - B[2 * j + 1]);
      r[0][2 * j] = T(2) * S[2 * j] + S[2 * j + 1] + dx;
      r[0][2 * j + 1] = S[2 * j] + T(2) * S[2 * j + 1] - dx;
    }
  }
};

// ---------------------------------------------------------------- Cahn-Hilliard Jacobian
// Newton Jacobian of Def. weak_VMS_disc_CH in (dphi, dmu), with phi~ the current iterate and
// u~ the advecting velocity (diffusion term with a plus sign, as in the strong form):
//   row phi: (q, dphi)/dt - 1/2 (grad q, u~ dphi) + 1/(2 Pe Cn) (grad q, grad dmu)
//   row mu : -1/2 (q, dmu) + 1/2 (q, psi''(phi~) dphi) + Cn^2/2 (grad q, grad dphi)
template <class T, class C>
struct ChK {
  static constexpr bool QDATA = false;
  static constexpr int MIN_CTAS = sizeof(T) == 4 ? 4 : 1;
  static constexpr int STREAM_CTAS = 0;  // persistent apply (0: not used)
  static constexpr int NC = 2;
  static constexpr bool DIR = false;
  static constexpr bool DIAG_PER_COMP = true;
  static constexpr int NF = 4;  // phi~, u~ (3)
  T pe[8];
  T ue[3][8];
  __device__ __forceinline__ void setup(const T f[NF][8], const Geo<T>&, const DevParams&) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      pe[a] = f[0][a];
      ue[0][a] = f[1][a];
      ue[1][a] = f[2][a];
      ue[2][a] = f[3][a];
    }
  }
  __device__ __forceinline__ void load(const MeshDev& m, const DevParams&, const CoefArgs<C>& cf,
                                       const int idx[8], const Geo<T>&) {
    gather_phi(m, idx, cf, pe);
#pragma unroll
    for (int d = 0; d < 3; ++d) gather<T, false>(m, idx, cf.u[d], ue[d]);
  }
  // Sum-factorised: values at the Gauss points by interp3, gradients by grad_compact, and the
  // transposes (interp3 is its own transpose, grad_T) on the per-point terms.
  __device__ __forceinline__ void apply(const Geo<T>& g, const DevParams& p, const T x[NC][8],
                                        T r[NC][8]) const {
    const PrmT<T>& pk = p.get<T>();
    const T J = g.detJ;
    T pq[8], fv[8], mv[8];
    interp3(pe, pq);
    interp3(x[0], fv);
    interp3(x[1], mv);
    T s[8], V[3][8];
    // row mu: -1/2 (q, dmu) + 1/2 (q, psi''(phi~) dphi) + Cn^2/2 (grad q, grad dphi)
#pragma unroll
    for (int q = 0; q < 8; ++q)
      s[q] = J * T(0.5) * ((T(3) * pq[q] * pq[q] - T(1)) * fv[q] - mv[q]);
    interp3(s, r[1]);
    {
      T gx[4], gy[4], gz[4];
      grad_compact(x[0], gx, gy, gz);
      const T c = J * pk.kphi;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        V[0][q] = c * gx[gxi(q)] * g.ih[0];
        V[1][q] = c * gy[gyi(q)] * g.ih[1];
        V[2][q] = c * gz[gzi(q)] * g.ih[2];
      }
      grad_T(V, g, r[1]);
    }
    // row phi: (q, dphi)/dt - 1/2 (grad q, u~ dphi) + 1/(2 Pe Cn) (grad q, grad dmu)
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = J * pk.idt * fv[q];
    interp3(s, r[0]);
    {
      T gx[4], gy[4], gz[4];
      grad_compact(x[1], gx, gy, gz);
      const T c = J * pk.kmu;
      T uq[8];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        interp3(ue[d], uq);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const T gm = d == 0 ? gx[gxi(q)] : d == 1 ? gy[gyi(q)] : gz[gzi(q)];
          V[d][q] = c * gm * g.ih[d] - J * T(0.5) * uq[q] * fv[q];
        }
      }
      grad_T(V, g, r[0]);
    }
  }
};

// ---------------------------------------------------------------- velocity prediction (RBVMS)
// Per-quadrature-point coefficients of the momentum operator (Def. weak_VMS_disc):
//   rho~, eta~ from clamp(phi~); grad eta~ = gamma grad phi~ where |phi~| < 1;
//   J_hat = -(alpha/Cn) grad mu~; G = diag(4/h^2);
//   tau_m = (4/dt^2 + u.G.u + max(u.G.J/(rho Pe), -u.G.u) + C_I (eta/(rho Re))^2 G:G)^(-1/2):
//   the printed formula with its mixed term bounded below, since unbounded the radicand goes
//   negative where J/(rho Pe) dominates u.
// The operator on one velocity component v (the same for each component):
//   s = rho/dt v + 1/2 rho u.grad v + 1/(2Pe) J.grad v                       (tested with N_a)
//   R = s - 1/(2Re) grad eta . grad v                                        (R^lin)
//   V = eta/(2Re) grad v + tau R (u/2 + J/(2 Pe rho))                       (tested with grad N_a)
template <class T>
struct VmsQ {
  T rho, eta, a0, b[3], bp[3], e, t[3], tau, uq[3], J[3], ge[3], gphi[3];
};

// The coefficients at one point from the point values of phi~ (pv, grad gp), grad mu~ (mg) and
// u_hat (uq).
template <class T>
__device__ __forceinline__ VmsQ<T> vms_point(T pv, const T gp[3], const T mg[3], const T uq[3],
                                             const Geo<T>& g, const DevParams& p) {
  VmsQ<T> o;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    o.gphi[d] = gp[d];
    o.uq[d] = uq[d];
  }
  const PrmT<T>& k = p.get<T>();
  T pc = clamp1(pv);
  o.rho = k.alpha * pc + k.beta;
  o.eta = k.gamma * pc + k.xi;
  const bool inside = pv < T(1) && pv > T(-1);
  const T ka = k.ka;
  const T ir = T(1) / o.rho;
  const T jpe = ir * k.inv_pe;
  T ugu = T(0), ugj = T(0), gg = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    o.ge[d] = inside ? k.gamma * o.gphi[d] : T(0);
    o.J[d] = ka * mg[d];
    T Gd = T(4) * g.ih[d] * g.ih[d];
    ugu += o.uq[d] * Gd * o.uq[d];
    ugj += o.uq[d] * Gd * o.J[d];
    gg += Gd * Gd;
  }
  const T er = o.eta * ir * k.inv_re;
  ugj *= jpe;
  // the printed radicand, floored at 4/dt^2 (tau_m <= dt/2) where its mixed term u.G.J/(rho Pe)
  // would take it lower or negative
  const T rad = k.four_idt2 + ugu + ugj + k.C_I * er * er * gg;
  o.tau = rsqrt(rad > k.four_idt2 ? rad : k.four_idt2);
  o.a0 = o.rho * k.idt;
  o.e = o.eta * k.h2re;
  const T h2pe = k.h2pe, h2re = k.h2re;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    o.b[d] = T(0.5) * o.rho * o.uq[d] + h2pe * o.J[d];
    o.bp[d] = o.b[d] - h2re * o.ge[d];
    o.t[d] = o.tau * (T(0.5) * o.uq[d] + h2pe * ir * o.J[d]);
  }
  return o;
}

template <int Q, class T>
__device__ __forceinline__ VmsQ<T> vms_at(const T pe[8], const T ue[3][8], const T me[8],
                                          const Geo<T>& g, const DevParams& p) {
  T pv, mv, gp[3], mg[3], uq[3];
  vg_at<Q>(pe, g, pv, gp);
  vg_at<Q>(me, g, mv, mg);
  (void)mv;
#pragma unroll
  for (int d = 0; d < 3; ++d) uq[d] = val_at<Q>(ue[d]);
  return vms_point(pv, gp, mg, uq, g, p);
}

// A field at the 8 Gauss points by sum factorisation: values (interp3) and the compact
// per-axis gradient data (grad_compact); grad(q, d) is the physical derivative d/dx_d at q.
template <class T>
struct QpField {
  T v[8], gx[4], gy[4], gz[4];
  __device__ __forceinline__ void eval(const T u[8]) {
    interp3(u, v);
    grad_compact(u, gx, gy, gz);
  }
  __device__ __forceinline__ void eval_grad(const T u[8]) { grad_compact(u, gx, gy, gz); }
  __device__ __forceinline__ T grad(int q, int d, const Geo<T>& g) const {
    return d == 0 ? gx[gxi(q)] * g.ih[0] : d == 1 ? gy[gyi(q)] * g.ih[1] : gz[gzi(q)] * g.ih[2];
  }
};

template <class T, class C>
struct MomK {
  static constexpr bool QDATA = false;
  // FP32: two CTAs per SM (at most 128 registers) instead of the one that 217 registers allow
  static constexpr int MIN_CTAS = sizeof(T) == 4 ? 2 : 1;
  static constexpr int STREAM_CTAS = 0;  // persistent apply (0: not used)
  static constexpr int NC = 3;
  static constexpr bool DIR = true;
  static constexpr bool DIAG_PER_COMP = false;
  static constexpr int NF = 5;  // phi~, u_hat (3), mu~
  T pe[8];
  T ue[3][8];
  T me[8];
  __device__ __forceinline__ void setup(const T f[NF][8], const Geo<T>&, const DevParams&) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      pe[a] = f[0][a];
      ue[0][a] = f[1][a];
      ue[1][a] = f[2][a];
      ue[2][a] = f[3][a];
      me[a] = f[4][a];
    }
  }
  __device__ __forceinline__ void load(const MeshDev& m, const DevParams&, const CoefArgs<C>& cf,
                                       const int idx[8], const Geo<T>&) {
    gather_phi(m, idx, cf, pe);
#pragma unroll
    for (int d = 0; d < 3; ++d) gather<T, false>(m, idx, cf.u[d], ue[d]);
    gather<T, false>(m, idx, cf.mu, me);
  }
  __device__ __forceinline__ void apply(const Geo<T>& g, const DevParams& p, const T x[NC][8],
                                        T r[NC][8]) const {
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
      for (int a = 0; a < 8; ++a) r[k][a] = T(0);
    const T J = g.detJ;
    for_qp([&](auto QC) {
      constexpr int Q = decltype(QC)::value;
      VmsQ<T> c = vms_at<Q>(pe, ue, me, g, p);
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        T v, vg[3];
        vg_at<Q>(x[k], g, v, vg);
        T s = c.a0 * v + c.b[0] * vg[0] + c.b[1] * vg[1] + c.b[2] * vg[2];
        T R = c.a0 * v + c.bp[0] * vg[0] + c.bp[1] * vg[1] + c.bp[2] * vg[2];
        T V[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) V[d] = J * (c.e * vg[d] + R * c.t[d]);
        add_test<Q>(r[k], J * s, V, g);
      }
    });
  }
};

// Quadrature data of the momentum operator: per element and quadrature point the 11 values
// the linear operator needs (a0, b[3], bp[3], e, t[3] of VmsQ), computed once per solve while
// the coefficients are fixed, stored value-major, qd[(q * kMomQ + v) * n_elem + e], so that a
// warp's loads are coalesced. The apply then reads 88 values per element instead of
// re-evaluating tau_m and the RBVMS vectors at every quadrature point (FP64 arithmetic is the
// bound of that evaluation on GB300).
constexpr int kMomQ = 11;

template <class T, class C>
__global__ void __launch_bounds__(128)
k_mom_qdata(MeshDev m, DevParams p, CoefArgs<C> cf, T* __restrict__ qd) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  int idx[8];
  load_corners(m, e, idx);
  const Geo<T> g = geometry<T>(m, e);
  MomK<T, C> k;
  k.load(m, p, cf, idx, g);
  const int64_t E = m.n_elem;
  // the fields at the Gauss points by sum factorisation
  QpField<T> fp, fm;
  fp.eval(k.pe);
  fm.eval_grad(k.me);
  T uq[3][8];
#pragma unroll
  for (int d = 0; d < 3; ++d) interp3(k.ue[d], uq[d]);
  for_qp([&](auto QC) {
    constexpr int Q = decltype(QC)::value;
    T gp[3], mg[3], uv[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      gp[d] = fp.grad(Q, d, g);
      mg[d] = fm.grad(Q, d, g);
      uv[d] = uq[d][Q];
    }
    const VmsQ<T> c = vms_point(fp.v[Q], gp, mg, uv, g, p);
    T* q = qd + (int64_t)Q * kMomQ * E + e;
    q[0] = c.a0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      q[(1 + d) * E] = c.b[d];
      q[(4 + d) * E] = c.bp[d];
      q[(8 + d) * E] = c.t[d];
    }
    q[7 * E] = c.e;
  });
}

// The momentum operator from quadrature data (same arithmetic as MomK::apply).
template <class T, class C>
struct MomQK {
  static constexpr bool QDATA = true;
  static constexpr int MIN_CTAS = sizeof(T) == 4 ? 2 : 1;
  static constexpr int STREAM_CTAS = 0;  // persistent apply (0: not used)
  static constexpr int NC = 3;
  static constexpr bool DIR = true;
  static constexpr bool DIAG_PER_COMP = false;
  static constexpr int NF = 1;  // (phi~ only to keep the shared-memory layout of the kernel)
  const AccumT<T>* qd = nullptr;  // FP64 data for double-float
  int64_t ne = 0, e = 0;
  __device__ __forceinline__ void setup(const T[NF][8], const Geo<T>&, const DevParams&) {}
  __device__ __forceinline__ void load(const MeshDev&, const DevParams&, const CoefArgs<C>&,
                                       const int[8], const Geo<T>&) {}
  __device__ __forceinline__ void bind(const void* q, int64_t n_elem, int64_t elem) {
    qd = static_cast<const AccumT<T>*>(q);
    ne = n_elem;
    e = elem;
  }
  __device__ __forceinline__ void apply(const Geo<T>& g, const DevParams& p, const T x[NC][8],
                                        T r[NC][8]) const {
    if constexpr (sizeof(T) == sizeof(double))
      apply_sf(g, x, r);
    else
      apply_direct(g, p, x, r);
  }
  // Sum-factorised, one component at a time (values by interp3, gradients from the compact
  // per-axis data, transposes interp3 / grad_T); the quadrature data is read per component (the
  // FP64 arithmetic, not the reads, bounds this form).
  __device__ __forceinline__ void apply_sf(const Geo<T>& g, const T x[NC][8], T r[NC][8]) const {
    const T J = g.detJ;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      T v[8], gx[4], gy[4], gz[4], s[8], V[3][8];
      interp3(x[k], v);
      grad_compact(x[k], gx, gy, gz);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const AccumT<T>* qq = qd + (int64_t)q * kMomQ * ne + e;
        const T vg[3] = {gx[gxi(q)] * g.ih[0], gy[gyi(q)] * g.ih[1], gz[gzi(q)] * g.ih[2]};
        const T a0 = T(__ldg(qq));
        T sb = a0 * v[q], R = a0 * v[q];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          sb += T(__ldg(qq + (1 + d) * ne)) * vg[d];
          R += T(__ldg(qq + (4 + d) * ne)) * vg[d];
        }
        const T ce = T(__ldg(qq + 7 * ne));
        s[q] = J * sb;
#pragma unroll
        for (int d = 0; d < 3; ++d) V[d][q] = J * (ce * vg[d] + R * T(__ldg(qq + (8 + d) * ne)));
      }
      interp3(s, r[k]);
      grad_T(V, g, r[k]);
    }
  }
  __device__ __forceinline__ void apply_direct(const Geo<T>& g, const DevParams&,
                                               const T x[NC][8], T r[NC][8]) const {
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
      for (int a = 0; a < 8; ++a) r[k][a] = T(0);
    const T J = g.detJ;
    for_qp([&](auto QC) {
      constexpr int Q = decltype(QC)::value;
      const T* q = qd + (int64_t)Q * kMomQ * ne + e;
      const T a0 = T(__ldg(q));
      T b[3], bp[3], t[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        b[d] = T(__ldg(q + (1 + d) * ne));
        bp[d] = T(__ldg(q + (4 + d) * ne));
        t[d] = T(__ldg(q + (8 + d) * ne));
      }
      const T ce = T(__ldg(q + 7 * ne));
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        T v, vg[3];
        vg_at<Q>(x[k], g, v, vg);
        T s = a0 * v + b[0] * vg[0] + b[1] * vg[1] + b[2] * vg[2];
        T R = a0 * v + bp[0] * vg[0] + bp[1] * vg[1] + bp[2] * vg[2];
        T V[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) V[d] = J * (ce * vg[d] + R * t[d]);
        add_test<Q>(r[k], J * s, V, g);
      }
    });
  }
};

// Operators that form the element energy x . A_e x alongside the apply (ENERGY = true).
template <class K, class = void>
struct HasEnergy : std::false_type {};
template <class K>
struct HasEnergy<K, std::void_t<decltype(K::ENERGY)>> : std::bool_constant<K::ENERGY> {};

// Operators whose element kernel never reads the coefficient fields it is handed (the shifted
// operator's coefficients are constants): the persistent apply gathers none for them.
template <class K, class = void>
struct IgnoresFields : std::false_type {};
template <class K>
struct IgnoresFields<K, std::void_t<decltype(K::IGNORES_FIELDS)>>
    : std::bool_constant<K::IGNORES_FIELDS> {};

}  // namespace chns
