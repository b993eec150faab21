// Right-hand sides and nonlinear residuals of the time step (FP64), and the phi mass integral.
// These are the "vector assembly" traversals of the paper (Sec. 5.4), done matrix-free with the
// same gather / element quadrature / scatter-add skeleton as the operator applies.
#include <vector>

#include "ops.cuh"

namespace chns {

constexpr int kRhsThreads = 128;
// gravity direction g_hat = (0, -1, 0) (Sec. 3): the sign of the y component
__device__ __forceinline__ int ghat(int i) { return i == 1 ? -1 : 0; }

struct Ptr3 {
  const double* c[3];
};

// The kernels below are written for an arithmetic type A and run in FP64 (A = double): in
// double-float (dfloat.cuh) they measured about 3x slower, their register pressure and spills
// outweighing the FP32 issue rate. Fields are read from and results added to FP64 arrays.

// ---- CH residual at the new-time iterate (Def. weak_VMS_disc_CH):
//   F_phi = (q, (phi - phi_k)/dt) - (grad q, u~ phi~) + 1/(Pe Cn) (grad q, grad mu~)
//   F_mu  = -(q, mu~) + (q, psi'(phi~)) + Cn^2 (grad q, grad phi~)
template <class A>
__global__ void __launch_bounds__(kRhsThreads)
k_residual_ch(MeshDev m, DevParams p, const double* __restrict__ phi, const double* __restrict__ mu,
              const double* __restrict__ phik, const double* __restrict__ muk, Ptr3 u,
              double* __restrict__ f) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  const PrmT<A>& k = p.get<A>();
  int idx[8];
  load_corners(m, e, idx);
  const Geo<A> g = geometry<A>(m, e);
  A a[8], b[8], pt[8], mt[8], dp[8], ue[3][8];
  gather<A, false>(m, idx, phi, a);
  gather<A, false>(m, idx, phik, b);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    pt[i] = A(0.5) * (a[i] + b[i]);
    dp[i] = (a[i] - b[i]) * k.idt;
  }
  gather<A, false>(m, idx, mu, a);
  gather<A, false>(m, idx, muk, b);
#pragma unroll
  for (int i = 0; i < 8; ++i) mt[i] = A(0.5) * (a[i] + b[i]);
#pragma unroll
  for (int d = 0; d < 3; ++d) gather<A, false>(m, idx, u.c[d], ue[d]);
  // sum-factorised: values at the Gauss points by interp3, gradients by grad_compact, and the
  // transposes interp3 / grad_T on the per-point terms
  A r0[8], r1[8];
  const A J = g.detJ, kmu = k.inv_pecn, c2 = k.cn2;
  A pv[8], mv[8], s[8], V[3][8];
  interp3(pt, pv);
  interp3(mt, mv);
#pragma unroll
  for (int q = 0; q < 8; ++q) s[q] = J * (pv[q] * pv[q] * pv[q] - pv[q] - mv[q]);
  interp3(s, r1);
  {
    A gx[4], gy[4], gz[4];
    grad_compact(pt, gx, gy, gz);
    const A jc = J * c2;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      V[0][q] = jc * gx[gxi(q)] * g.ih[0];
      V[1][q] = jc * gy[gyi(q)] * g.ih[1];
      V[2][q] = jc * gz[gzi(q)] * g.ih[2];
    }
    grad_T(V, g, r1);
  }
  interp3(dp, s);
#pragma unroll
  for (int q = 0; q < 8; ++q) s[q] = s[q] * J;
  interp3(s, r0);
  {
    A gx[4], gy[4], gz[4], uq[8];
    grad_compact(mt, gx, gy, gz);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      interp3(ue[d], uq);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const A gm = d == 0 ? gx[gxi(q)] : d == 1 ? gy[gyi(q)] : gz[gzi(q)];
        V[d][q] = J * (kmu * gm * g.ih[d] - uq[q] * pv[q]);
      }
    }
    grad_T(V, g, r0);
  }
  scatter<A, false>(m, idx, r0, f);
  scatter<A, false>(m, idx, r1, f + m.n_nodes);
}

// Forcing d_j(d_i phi d_j phi) of the trilinear interpolant at Q (pure second derivatives vanish
// on box elements): F_i = sum_{j != i} H_ij d_j phi.
template <int Q, class A>
__device__ __forceinline__ void forcing_at(const A pe[8], const Geo<A>& g, const A gp[3], A F[3]) {
  A hxy, hxz, hyz;
  hess_at<Q>(pe, g, hxy, hxz, hyz);
  F[0] = hxy * gp[1] + hxz * gp[2];
  F[1] = hxy * gp[0] + hyz * gp[2];
  F[2] = hxz * gp[0] + hyz * gp[1];
}

// rho g_i / Fr for the component i (g_hat = (0, -1, 0))
template <class A>
__device__ __forceinline__ A gravity(const A& rho, const PrmT<A>& k, int i) {
  return ghat(i) == 0 ? A(0) : -(rho * k.inv_fr);
}

// ---- velocity-prediction right-hand side (Def. weak_VMS_disc), per component i:
//   (w, rho u_i/dt) - 1/2 (w, rho u.grad u_i) - 1/(2Pe) (w, J.grad u_i) - 1/(2Re) (grad w, eta grad u_i)
//   + Cn/We (d_j w, d_i phi d_j phi) - (w, d_i p) + (w, rho g_i/Fr) - (grad w . t, R0_i)
// with R0_i the part of R_m that does not depend on v^{k+1}.
// Sum-factorised: every field's values and gradients at the 8 Gauss points come from interp3 /
// grad_compact, the per-point coefficients (tau_m and the advection and stabilisation vectors)
// are formed once per point, and each component's test-function sums are the transposes interp3
// and grad_T of its per-point terms.
template <class A>
struct MomPt {  // per-point data shared by the three components
  A a0, b[3], bp[3], e, t[3], rho, gphi[3], F[3], pg[3];
};

template <class A>
__global__ void __launch_bounds__(kRhsThreads)
k_rhs_momentum(MeshDev m, DevParams p, CoefArgs<double> cf, Ptr3 uk,
               const double* __restrict__ pk, double* __restrict__ b) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  const PrmT<A>& k = p.get<A>();
  int idx[8];
  load_corners(m, e, idx);
  const Geo<A> g = geometry<A>(m, e);
  const A J = g.detJ, cw = k.cw;
  MomPt<A> c[8];
  {
    A pe[8], ue[3][8], me[8], pp[8];
    gather<A, false>(m, idx, cf.phi, pe);
#pragma unroll
    for (int d = 0; d < 3; ++d) gather<A, false>(m, idx, cf.u[d], ue[d]);
    gather<A, false>(m, idx, cf.mu, me);
    gather<A, false>(m, idx, pk, pp);
    QpField<A> fp, fm, fr;
    fp.eval(pe);
    fm.eval_grad(me);
    fr.eval_grad(pp);
    A uq[3][8];
#pragma unroll
    for (int d = 0; d < 3; ++d) interp3(ue[d], uq[d]);
    for_qp([&](auto QC) {
      constexpr int Q = decltype(QC)::value;
      A gp[3], mg[3], uv[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        gp[d] = fp.grad(Q, d, g);
        mg[d] = fm.grad(Q, d, g);
        uv[d] = uq[d][Q];
      }
      const VmsQ<A> v = vms_point(fp.v[Q], gp, mg, uv, g, p);
      MomPt<A>& o = c[Q];
      o.a0 = v.a0;
      o.e = v.e;
      o.rho = v.rho;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        o.b[d] = v.b[d];
        o.bp[d] = v.bp[d];
        o.t[d] = v.t[d];
        o.gphi[d] = v.gphi[d];
        o.pg[d] = fr.grad(Q, d, g);
      }
      forcing_at<Q>(pe, g, v.gphi, o.F);
    });
  }
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
    A ui[8];
    gather<A, false>(m, idx, uk.c[i], ui);
    QpField<A> fu;
    fu.eval(ui);
    A s[8], V[3][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const MomPt<A>& o = c[q];
      const A v = fu.v[q];
      const A vg[3] = {fu.grad(q, 0, g), fu.grad(q, 1, g), fu.grad(q, 2, g)};
      const A grav = gravity(o.rho, k, i);
      const A bdot = o.b[0] * vg[0] + o.b[1] * vg[1] + o.b[2] * vg[2];
      const A bpdot = o.bp[0] * vg[0] + o.bp[1] * vg[1] + o.bp[2] * vg[2];
      const A r0 = bpdot - o.a0 * v + cw * o.F[i] + o.pg[i] - grav;
      const A fn = o.a0 * v - bdot - o.pg[i] + grav;
      s[q] = J * fn;
      const A cg = cw * o.gphi[i];
#pragma unroll
      for (int d = 0; d < 3; ++d) V[d][q] = J * (cg * o.gphi[d] - o.e * vg[d] - o.t[d] * r0);
    }
    A r[8];
    interp3(s, r);
    grad_T(V, g, r);
    scatter<A, true>(m, idx, r, b + i * m.n_nodes);
  }
}

// Full R_m,i(v) at a point (Def. of R_m) with v~ = (v + u_k)/2, from the point values vv and
// gradients vgr of v and ug of u_k (uv: u_k's values).
template <class A>
__device__ __forceinline__ void rm_point(const VmsQ<A>& c, const PrmT<A>& k, const A F[3],
                                         const A pg[3], const A vv[3], const A vgr[3][3],
                                         const A uv[3], const A ug[3][3], A R[3], A& div) {
  div = vgr[0][0] + vgr[1][1] + vgr[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    A tg[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) tg[d] = A(0.5) * (vgr[i][d] + ug[i][d]);
    const A adv = c.uq[0] * tg[0] + c.uq[1] * tg[1] + c.uq[2] * tg[2];
    const A jdv = c.J[0] * tg[0] + c.J[1] * tg[1] + c.J[2] * tg[2];
    const A edv = c.ge[0] * tg[0] + c.ge[1] * tg[1] + c.ge[2] * tg[2];
    R[i] = c.rho * (vv[i] - uv[i]) * k.idt + c.rho * adv + jdv * k.inv_pe + k.cw * F[i] + pg[i] -
           edv * k.inv_re - gravity(c.rho, k, i);
  }
}

// The fields of the pressure-Poisson and velocity-update right-hand sides at the 8 Gauss points.
template <class A>
struct ProjFields {
  QpField<A> fp, fm, fr, fv[3], fu[3];
  A uq[3][8];
  __device__ __forceinline__ void load(const MeshDev& m, const int idx[8],
                                       const CoefArgs<double>& cf, const Ptr3& v, const Ptr3& uk,
                                       const double* pk, A pe[8]) {
    A t[8];
    gather<A, false>(m, idx, cf.phi, pe);
    fp.eval(pe);
    gather<A, false>(m, idx, cf.mu, t);
    fm.eval_grad(t);
    gather<A, false>(m, idx, pk, t);
    fr.eval_grad(t);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      gather<A, false>(m, idx, cf.u[d], t);
      interp3(t, uq[d]);
      gather<A, false>(m, idx, v.c[d], t);
      fv[d].eval(t);
      gather<A, false>(m, idx, uk.c[d], t);
      fu[d].eval(t);
    }
  }
  // the coefficients, forcing, grad p_k and R_m at point Q
  template <int Q>
  __device__ __forceinline__ VmsQ<A> at(const A pe[8], const Geo<A>& g, const DevParams& p,
                                        A pg[3], A R[3], A vv[3], A& div) const {
    A gp[3], mg[3], uv0[3], vgr[3][3], ug[3][3], uv[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      gp[d] = fp.grad(Q, d, g);
      mg[d] = fm.grad(Q, d, g);
      uv0[d] = uq[d][Q];
      pg[d] = fr.grad(Q, d, g);
      vv[d] = fv[d].v[Q];
      uv[d] = fu[d].v[Q];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        vgr[d][k] = fv[d].grad(Q, k, g);
        ug[d][k] = fu[d].grad(Q, k, g);
      }
    }
    const VmsQ<A> c = vms_point(fp.v[Q], gp, mg, uv0, g, p);
    A F[3];
    forcing_at<Q>(pe, g, c.gphi, F);
    rm_point(c, p.get<A>(), F, pg, vv, vgr, uv, ug, R, div);
    return c;
  }
};

// ---- pressure-Poisson right-hand side (Def. weak_VMS_disc_pp_vel, scalar test q):
//   -(2/dt)(q, div v) - (2/dt)(grad q, tau R_m / rho~) + (grad q, grad p_k / rho~)
// With qvu, the velocity update's per-point terms J (rho~ v_i - tau R_m,i) (the same R_m) are
// stored as well, qvu[(q * 3 + i) * n_elem + e], for k_rhs_vu_q.
template <class A>
__global__ void __launch_bounds__(kRhsThreads)
k_rhs_poisson(MeshDev m, DevParams p, CoefArgs<double> cf, Ptr3 v, Ptr3 uk,
              const double* __restrict__ pk, double* __restrict__ b, double* __restrict__ qvu) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  int idx[8];
  load_corners(m, e, idx);
  const Geo<A> g = geometry<A>(m, e);
  A pe[8];
  ProjFields<A> f;
  f.load(m, idx, cf, v, uk, pk, pe);
  const A J = g.detJ, k2 = p.get<A>().k2dt;
  A s[8], V[3][8];
  for_qp([&](auto QC) {
    constexpr int Q = decltype(QC)::value;
    A pg[3], R[3], vv[3], div;
    const VmsQ<A> c = f.template at<Q>(pe, g, p, pg, R, vv, div);
    const A jr = J / c.rho, kt = k2 * c.tau;
#pragma unroll
    for (int d = 0; d < 3; ++d) V[d][Q] = jr * (pg[d] - kt * R[d]);
    s[Q] = -(J * k2 * div);
    if (qvu)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        qvu[(int64_t)(Q * 3 + i) * m.n_elem + e] = (double)(J * (c.rho * vv[i] - c.tau * R[i]));
  });
  A r[8];
  interp3(s, r);
  grad_T(V, g, r);
  scatter<A, false>(m, idx, r, b);
}

// The velocity-update right-hand side from the per-point terms stored by k_rhs_poisson (same
// v, u_k, p_k and coefficients): only the pressure-difference term is evaluated here.
__global__ void __launch_bounds__(kRhsThreads)
k_rhs_vu_q(MeshDev m, DevParams p, const double* __restrict__ qvu, const double* __restrict__ pk,
           const double* __restrict__ pn, double* __restrict__ b) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  int idx[8];
  load_corners(m, e, idx);
  const Geo<double> g = geometry<double>(m, e);
  QpField<double> fd;  // p_new - p_k
  {
    double a[8], c0[8];
    gather<double, false>(m, idx, pn, a);
    gather<double, false>(m, idx, pk, c0);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] -= c0[k];
    fd.eval_grad(a);
  }
  const double jh = g.detJ * p.d.half_dt;
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
    double s[8], r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      s[q] = __ldg(qvu + (int64_t)(q * 3 + i) * m.n_elem + e) - jh * fd.grad(q, i, g);
    interp3(s, r);
    scatter<double, true>(m, idx, r, b + i * m.n_nodes);
  }
}

// ---- velocity-update right-hand side (Def. weak_VMS_disc_vel_update), per component:
//   (w, rho~ v_i) - (w, tau R_m,i) - (dt/2)(w, d_i (p_new - p_k))
template <class A>
__global__ void __launch_bounds__(kRhsThreads)
k_rhs_vu(MeshDev m, DevParams p, CoefArgs<double> cf, Ptr3 v, Ptr3 uk,
         const double* __restrict__ pk, const double* __restrict__ pn, double* __restrict__ b) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  int idx[8];
  load_corners(m, e, idx);
  const Geo<A> g = geometry<A>(m, e);
  A pe[8];
  ProjFields<A> f;
  f.load(m, idx, cf, v, uk, pk, pe);
  QpField<A> fd;  // p_new - p_k
  {
    A a[8], c0[8];
    gather<A, false>(m, idx, pn, a);
    gather<A, false>(m, idx, pk, c0);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = a[k] - c0[k];
    fd.eval_grad(a);
  }
  const A J = g.detJ, hdt = p.get<A>().half_dt;
  A s[3][8];
  for_qp([&](auto QC) {
    constexpr int Q = decltype(QC)::value;
    A pg[3], R[3], vv[3], div;
    const VmsQ<A> c = f.template at<Q>(pe, g, p, pg, R, vv, div);
#pragma unroll
    for (int i = 0; i < 3; ++i)
      s[i][Q] = J * (c.rho * vv[i] - c.tau * R[i] - hdt * fd.grad(Q, i, g));
  });
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
    A r[8];
    interp3(s[i], r);
    scatter<A, true>(m, idx, r, b + i * m.n_nodes);
  }
}

// ---- phi mass: sum_e detJ sum_q phi(q) = sum_e detJ sum_a phi_a (2-point Gauss weights sum to 1
// per corner). Block partial sums, then a deterministic final sum on the host.
__global__ void k_phi_mass(MeshDev m, const double* __restrict__ phi, double* __restrict__ part) {
  __shared__ double sh[kRhsThreads];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v = 0.0;
  if (e < m.n_elem) {
    int idx[8];
    load_corners(m, e, idx);
    const Geo<double> g = geometry<double>(m, e);
    double pe[8];
    gather<double, false>(m, idx, phi, pe);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) s += pe[a];
    v = g.detJ * s;
  }
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = kRhsThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

static unsigned nblk(const chns_mesh* m) {
  return (unsigned)((m->d.n_elem + kRhsThreads - 1) / kRhsThreads);
}

static chns_status need(bool ok, const char* what) {
  if (!ok) {
    set_error(what);
    return CHNS_EINVAL;
  }
  return CHNS_OK;
}

chns_status phi_mass(const chns_mesh* m, const double* phi, double* out, cudaStream_t s) {
  const unsigned nb = nblk(m);
  // The block partials (n_elem/128 <= 3N values) go to the last FP64 workspace vector. The
  // Chebyshev setup (cheb_bounds) also uses that vector as scratch; sharing it is safe because
  // this call reads the partials back and synchronises the stream before it returns, and it is
  // only called between solves (before and after a step), never inside one.
  double* part = m->ws.v64[kNumVec64 - 1];
  note_launch();
  k_phi_mass<<<nb, kRhsThreads, 0, s>>>(m->d, phi, part);
  CHNS_CUDA(cudaGetLastError());
  std::vector<double> h(nb);
  CHNS_CUDA(cudaMemcpyAsync(h.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  CHNS_CUDA(cudaStreamSynchronize(s));
  double acc = 0.0;
  for (double v : h) acc += v;
  *out = acc;
  return CHNS_OK;
}

chns_status residual_ch(const chns_mesh* m, const chns_params* prm, const double* phi,
                        const double* mu, const double* phik, const double* muk,
                        const double* const u[3], double* f, cudaStream_t s) {
  const DevParams p = make_dev_params(*prm);
  Ptr3 up{{u[0], u[1], u[2]}};
  CHNS_CUDA(cudaMemsetAsync(f, 0, 2 * m->d.n_nodes * sizeof(double), s));
  note_launch();
  k_residual_ch<double><<<nblk(m), kRhsThreads, 0, s>>>(m->d, p, phi, mu, phik, muk, up, f);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

static CoefArgs<double> cargs(const chns_coef* c) {
  CoefArgs<double> a;
  a.phi = static_cast<const double*>(c->phi_tilde);
  for (int d = 0; d < 3; ++d) a.u[d] = static_cast<const double*>(c->u_adv[d]);
  a.mu = static_cast<const double*>(c->mu_tilde);
  a.phi_shift = 0.0f;
  return a;
}

chns_status rhs_momentum(const chns_mesh* m, const chns_params* prm, const chns_coef* c,
                         const double* const uk[3], const double* pk, double* b, cudaStream_t s) {
  const DevParams p = make_dev_params(*prm);
  CHNS_CUDA(cudaMemsetAsync(b, 0, 3 * m->d.n_nodes * sizeof(double), s));
  note_launch();
  const Ptr3 u3{{uk[0], uk[1], uk[2]}};
  k_rhs_momentum<double><<<nblk(m), kRhsThreads, 0, s>>>(m->d, p, cargs(c), u3, pk, b);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status rhs_poisson(const chns_mesh* m, const chns_params* prm, const chns_coef* c,
                        const double* const v[3], const double* const uk[3], const double* pk,
                        double* b, cudaStream_t s, double* qvu) {
  const DevParams p = make_dev_params(*prm);
  CHNS_CUDA(cudaMemsetAsync(b, 0, m->d.n_nodes * sizeof(double), s));
  note_launch();
  const Ptr3 v3{{v[0], v[1], v[2]}}, u3{{uk[0], uk[1], uk[2]}};
  k_rhs_poisson<double><<<nblk(m), kRhsThreads, 0, s>>>(m->d, p, cargs(c), v3, u3, pk, b, qvu);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status rhs_vu(const chns_mesh* m, const chns_params* prm, const chns_coef* c,
                   const double* const v[3], const double* const uk[3], const double* pk,
                   const double* pn, double* b, cudaStream_t s) {
  const DevParams p = make_dev_params(*prm);
  CHNS_CUDA(cudaMemsetAsync(b, 0, 3 * m->d.n_nodes * sizeof(double), s));
  note_launch();
  const Ptr3 v3{{v[0], v[1], v[2]}}, u3{{uk[0], uk[1], uk[2]}};
  k_rhs_vu<double><<<nblk(m), kRhsThreads, 0, s>>>(m->d, p, cargs(c), v3, u3, pk, pn, b);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status rhs_vu_from(const chns_mesh* m, const chns_params* prm, const double* qvu,
                        const double* pk, const double* pn, double* b, cudaStream_t s) {
  const DevParams p = make_dev_params(*prm);
  CHNS_CUDA(cudaMemsetAsync(b, 0, 3 * m->d.n_nodes * sizeof(double), s));
  note_launch();
  k_rhs_vu_q<<<nblk(m), kRhsThreads, 0, s>>>(m->d, p, qvu, pk, pn, b);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

static bool coef_ok(const chns_coef* c) {
  return c && c->phi_tilde && c->u_adv[0] && c->u_adv[1] && c->u_adv[2] && c->mu_tilde;
}

}  // namespace chns

using namespace chns;

extern "C" chns_status chns_residual_ch(const chns_mesh* m, const chns_params* prm,
                                        const double* phi, const double* mu, const double* phik,
                                        const double* muk, const double* const u[3], double* f,
                                        void* stream) {
  chns_status st = need(m && prm && phi && mu && phik && muk && u && u[0] && u[1] && u[2] && f,
                        "chns_residual_ch: null argument");
  if (st != CHNS_OK) return st;
  return residual_ch(m, prm, phi, mu, phik, muk, u, f, as_stream(stream));
}

extern "C" chns_status chns_rhs_momentum(const chns_mesh* m, const chns_params* prm,
                                         const chns_coef* c, const double* const uk[3],
                                         const double* pk, double* b, void* stream) {
  chns_status st = need(m && prm && coef_ok(c) && uk && uk[0] && uk[1] && uk[2] && pk && b,
                        "chns_rhs_momentum: null argument");
  if (st != CHNS_OK) return st;
  return rhs_momentum(m, prm, c, uk, pk, b, as_stream(stream));
}

extern "C" chns_status chns_rhs_poisson(const chns_mesh* m, const chns_params* prm,
                                        const chns_coef* c, const double* const v[3],
                                        const double* const uk[3], const double* pk, double* b,
                                        void* stream) {
  chns_status st = need(m && prm && coef_ok(c) && v && v[0] && v[1] && v[2] && uk && uk[0] &&
                            uk[1] && uk[2] && pk && b,
                        "chns_rhs_poisson: null argument");
  if (st != CHNS_OK) return st;
  return rhs_poisson(m, prm, c, v, uk, pk, b, as_stream(stream));
}

extern "C" chns_status chns_rhs_velocity_update(const chns_mesh* m, const chns_params* prm,
                                                const chns_coef* c, const double* const v[3],
                                                const double* const uk[3], const double* pk,
                                                const double* pn, double* b, void* stream) {
  chns_status st = need(m && prm && coef_ok(c) && v && v[0] && v[1] && v[2] && uk && uk[0] &&
                            uk[1] && uk[2] && pk && pn && b,
                        "chns_rhs_velocity_update: null argument");
  if (st != CHNS_OK) return st;
  return rhs_vu(m, prm, c, v, uk, pk, pn, b, as_stream(stream));
}

extern "C" chns_status chns_phi_mass(const chns_mesh* m, const double* phi, double* out,
                                     void* stream) {
  chns_status st = need(m && phi && out, "chns_phi_mass: null argument");
  if (st != CHNS_OK) return st;
  return phi_mass(m, phi, out, as_stream(stream));
}
