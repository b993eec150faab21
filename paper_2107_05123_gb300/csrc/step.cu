// One time step of the projection scheme: the two-block iteration of Fig. "flowchart_block".
// For each block: Cahn-Hilliard by Newton (GMRES on the matrix-free Jacobian), velocity
// prediction (GMRES), pressure Poisson (CG, mean zero), velocity update (CG). The host only
// orchestrates; every field operation runs in the library's kernels on the given stream.
#include <cmath>
#include <string>

#include "internal.h"

namespace chns {

// out = a*x + b*y on n entries (FP64)
static void lin(double a, const double* x, double b, const double* y, double* out, int64_t n,
                cudaStream_t s) {
  vec_axpby(a, x, b, y, out, n, s);
}

// Prefix the current error message with the phase of the step that failed.
static chns_status phase_fail(const char* phase, chns_status rc) {
  set_error(std::string("chns_step: ") + phase + ": " + chns_last_error());
  return rc;
}
#define STEP_FAIL(phase, rc)              \
  do {                                    \
    if (stats) *stats = S;                \
    return phase_fail(phase, rc);         \
  } while (0)

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  float stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

static chns_status step(const chns_mesh* m, chns_state* st, const chns_params* prm,
                        const chns_step_params* sp, chns_step_stats* stats, cudaStream_t s) {
  CHNS_CHECK(m && st && prm && sp, CHNS_EINVAL, "chns_step: null argument");
  CHNS_CHECK(st->phi && st->mu && st->p, CHNS_EINVAL, "chns_step: null field");
  for (int d = 0; d < 3; ++d)
    CHNS_CHECK(st->u[d] && st->u_old[d], CHNS_EINVAL, "chns_step: null velocity field");
  CHNS_CHECK(sp->blocks >= 1 && sp->blocks <= 2, CHNS_EINVAL, "chns_step: blocks must be 1 or 2");
  const int64_t N = m->d.n_nodes;
  const Workspace& ws = m->ws;
  double* C = ws.coef64;
  double* phit = C;                     // phi~
  double* uhat[3] = {C + N, C + 2 * N, C + 3 * N};
  double* mut = C + 4 * N;              // mu~
  double* util[3] = {C + 5 * N, C + 6 * N, C + 7 * N};
  double* phik = C + 8 * N;
  double* muk = C + 9 * N;
  double* pnew = C + 10 * N;
  double* xch = ws.v64[8];              // [phi; mu] Newton iterate
  double* f = ws.v64[9];
  double* dx = ws.v64[10];
  double* v = ws.v64[11];
  double* bv = ws.v64[12];
  double* un = ws.v64[13];
  // velocity Dirichlet data (lifted into the velocity right-hand sides): the data, the data on
  // the boundary rows only, and A applied to that (free between the Newton solves)
  const bool has_bc = sp->u_bc[0] && sp->u_bc[1] && sp->u_bc[2];
  CHNS_CHECK(has_bc || (!sp->u_bc[0] && !sp->u_bc[1] && !sp->u_bc[2]), CHNS_EINVAL,
             "chns_step: give all three velocity Dirichlet arrays or none");
  double* gfull = ws.v64[9];
  double* gb = ws.v64[10];
  double* lw = ws.v64[14];
  // b <- b - A g_b on the other rows and g on the boundary rows; x0 takes g on the boundary
  auto lift = [&](chns_operator op, const chns_coef* cf, double* b, double* x0) -> chns_status {
    for (int d = 0; d < 3; ++d)
      CHNS_CUDA(cudaMemcpyAsync(gfull + d * N, sp->u_bc[d], N * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
    CHNS_CUDA(cudaMemsetAsync(gb, 0, 3 * N * sizeof(double), s));
    chns_status r = dirichlet_set(m, 3, gfull, gb, s);
    if (r != CHNS_OK) return r;
    r = apply_op_full(m, op, prm, cf, gb, lw, s);
    if (r != CHNS_OK) return r;
    lin(1.0, b, -1.0, lw, b, 3 * N, s);
    r = dirichlet_set(m, 3, gfull, b, s);
    if (r != CHNS_OK) return r;
    return dirichlet_set(m, 3, gfull, x0, s);
  };
  chns_step_stats S{};
  Timer total(s);
  chns_status rc;

  CHNS_CUDA(cudaMemcpyAsync(phik, st->phi, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CHNS_CUDA(cudaMemcpyAsync(muk, st->mu, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CHNS_CUDA(cudaMemcpyAsync(xch, st->phi, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CHNS_CUDA(cudaMemcpyAsync(xch + N, st->mu, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  for (int d = 0; d < 3; ++d) lin(1.5, st->u[d], -0.5, st->u_old[d], uhat[d], N, s);  // [R1]
  rc = phi_mass(m, phik, &S.phi_mass_before, s);
  if (rc != CHNS_OK) return rc;

  const double* const uk[3] = {st->u[0], st->u[1], st->u[2]};
  const double* ublk[3] = {st->u[0], st->u[1], st->u[2]};
  const double* const vv[3] = {v, v + N, v + 2 * N};

  for (int l = 0; l < sp->blocks; ++l) {
    // ---- Cahn-Hilliard (Newton), advected by u~ = (u^k + u^{k+1,(l-1)})/2
    {
      Timer t(s);
      for (int d = 0; d < 3; ++d) lin(0.5, uk[d], 0.5, ublk[d], util[d], N, s);
      const double* const ut[3] = {util[0], util[1], util[2]};
      rc = residual_ch(m, prm, xch, xch + N, phik, muk, ut, f, s);
      if (rc != CHNS_OK) return rc;
      double f0 = 0.0, fn = 0.0;
      rc = dot_host(m, f, f, 2 * N, &f0, s);
      if (rc != CHNS_OK) return rc;
      f0 = std::sqrt(f0);
      fn = f0;
      int its = 0;
      chns_solve_stats ks{};
      // Inexact Newton: each linear solve only needs the accuracy the nonlinear iteration can
      // use (Eisenstat-Walker forcing eta_k = 0.9 (|F_k|/|F_k-1|)^2, eta_0 = 1e-3, at most 1e-3),
      // never tighter than what reaches the Newton target in one step (0.5 target/|F_k|), and
      // never tighter than the CH solver's rtol.
      const double target = std::max(sp->newton_rtol * f0, sp->newton_atol);
      double fprev = f0;
      while (fn > target && its < sp->newton_max_it) {
        double eta = 1e-3;
        if (its > 0) eta = std::min(1e-3, 0.9 * (fn / fprev) * (fn / fprev));
        eta = std::max(eta, 0.5 * target / fn);
        chns_solver_params chp = sp->ch;
        chp.rtol = std::max(eta, sp->ch.rtol);
        fprev = fn;
        lin(0.5, xch, 0.5, phik, phit, N, s);
        chns_coef cc{phit, {util[0], util[1], util[2]}, nullptr};
        CHNS_CUDA(cudaMemsetAsync(dx, 0, 2 * N * sizeof(double), s));
        rc = krylov_solve(m, CHNS_OP_CH, prm, &cc, f, dx, &chp, &ks, s);
        S.ch[l] = ks;
        if (rc != CHNS_OK) STEP_FAIL("Cahn-Hilliard Newton step", rc);
        lin(1.0, xch, -1.0, dx, xch, 2 * N, s);
        rc = residual_ch(m, prm, xch, xch + N, phik, muk, ut, f, s);
        if (rc != CHNS_OK) return rc;
        rc = dot_host(m, f, f, 2 * N, &fn, s);
        if (rc != CHNS_OK) return rc;
        fn = std::sqrt(fn);
        if (!std::isfinite(fn)) {
          set_error("chns_step: NaN/Inf in the CH residual");
          return CHNS_ENAN;
        }
        ++its;
      }
      if (fn > std::max(sp->newton_rtol * f0, sp->newton_atol)) {
        set_error("chns_step: Newton did not converge");
        return CHNS_ENOTCONV;
      }
      S.newton_its[l] = its;
      S.ch[l] = ks;
      S.ms_ch += t.stop();
    }
    lin(0.5, xch, 0.5, phik, phit, N, s);
    lin(0.5, xch + N, 0.5, muk, mut, N, s);
    chns_coef cv{phit, {uhat[0], uhat[1], uhat[2]}, mut};
    // ---- velocity prediction
    {
      Timer t(s);
      rc = rhs_momentum(m, prm, &cv, uk, st->p, bv, s);
      if (rc != CHNS_OK) return rc;
      for (int d = 0; d < 3; ++d)
        CHNS_CUDA(cudaMemcpyAsync(v + d * N, uk[d], N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      if (has_bc) {
        rc = lift(CHNS_OP_MOMENTUM, &cv, bv, v);
        if (rc != CHNS_OK) return rc;
      }
      rc = krylov_solve(m, CHNS_OP_MOMENTUM, prm, &cv, bv, v, &sp->vp, &S.vp[l], s);
      if (rc != CHNS_OK) STEP_FAIL("velocity prediction", rc);
      S.ms_vp += t.stop();
    }
    // ---- pressure Poisson (warm start from p^k)
    {
      Timer t(s);
      if (!m->qvu) CHNS_CUDA(cudaMalloc(&m->qvu, (size_t)24 * m->d.n_elem * sizeof(double)));
      rc = rhs_poisson(m, prm, &cv, vv, uk, st->p, bv, s, m->qvu);
      if (rc != CHNS_OK) return rc;
      CHNS_CUDA(cudaMemcpyAsync(pnew, st->p, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      rc = krylov_solve(m, CHNS_OP_POISSON, prm, &cv, bv, pnew, &sp->pp, &S.pp[l], s);
      if (rc != CHNS_OK) STEP_FAIL("pressure Poisson", rc);
      S.ms_pp += t.stop();
    }
    // ---- training pairs for the learned preconditioner (not part of the method)
    if (sp->collect) {
      int added = 0;
      rc = learned_collect(sp->collect, m, prm, &cv, bv, std::max(1, sp->collect_every),
                           std::max(0, sp->collect_max), sp->collect_with_net != 0, &added, s);
      if (rc != CHNS_OK) return rc;
    }
    // ---- velocity update
    {
      Timer t(s);
      rc = rhs_vu_from(m, prm, m->qvu, st->p, pnew, bv, s);
      if (rc != CHNS_OK) return rc;
      CHNS_CUDA(cudaMemcpyAsync(un, v, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      if (has_bc) {
        rc = lift(CHNS_OP_MASS, &cv, bv, un);
        if (rc != CHNS_OK) return rc;
      }
      rc = krylov_solve(m, CHNS_OP_MASS, prm, &cv, bv, un, &sp->vu, &S.vu[l], s);
      if (rc != CHNS_OK) STEP_FAIL("velocity update", rc);
      S.ms_vu += t.stop();
    }
    for (int d = 0; d < 3; ++d) ublk[d] = un + d * N;
  }
  // ---- roll the state
  for (int d = 0; d < 3; ++d) {
    CHNS_CUDA(cudaMemcpyAsync(st->u_old[d], st->u[d], N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CHNS_CUDA(cudaMemcpyAsync(st->u[d], un + d * N, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  CHNS_CUDA(cudaMemcpyAsync(st->p, pnew, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CHNS_CUDA(cudaMemcpyAsync(st->phi, xch, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CHNS_CUDA(cudaMemcpyAsync(st->mu, xch + N, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  rc = phi_mass(m, st->phi, &S.phi_mass_after, s);
  if (rc != CHNS_OK) return rc;
  S.ms_total = total.stop();
  if (stats) *stats = S;
  return CHNS_OK;
}

}  // namespace chns

extern "C" chns_status chns_step(const chns_mesh* m, chns_state* state, const chns_params* prm,
                                 const chns_step_params* sp, chns_step_stats* stats, void* stream) {
  return chns::step(m, state, prm, sp, stats, chns::as_stream(stream));
}
