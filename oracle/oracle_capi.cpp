/* C entry points of the CPU oracle, loaded by the tests through ctypes.
   TEST INFRASTRUCTURE ONLY: the product library never links or calls this. */
#include <cstdint>
#include <cstring>
#include <vector>
#include "tenom_oracle.hpp"
#include "exact_riemann.hpp"

namespace orc {
thread_local long long g_flops = 0;
}

using namespace orc;

static Grid norm_grid(const Grid* g) {
  Grid h = *g;
  for (int d = h.dim; d < 3; ++d) { h.n[d] = 1; h.dx[d] = 1.0; h.bc[d] = BC_PERIODIC; }
  return h;
}

static Scheme norm_scheme(const Scheme* s) {
  Scheme t = *s;
  bool any = false;
  for (int k = 0; k < 6; ++k) any |= (t.d[k] != 0.0);
  if (!any) default_weights(t.K, t.d);
  return t;
}

extern "C" {

void orc_default_weights(int K, double* d) { default_weights(K, d); }

/* n scalar reconstructions; v: [n][K] = f_{i-K/2+1}..f_{i+K/2}. */
void orc_recon(const Scheme* s, const double* v, int n, double* out, int* bits, int* ct_exp,
               double* cut_rel, double* beta_ct) {
  Scheme S = norm_scheme(s);
  const int K = S.K, h = K / 2;
  for (int q = 0; q < n; ++q) {
    const double* f = v + (long long)q * K;
    ReconDiag dg;
    out[q] = teno_m<double>(S, [&](int m) { return f[m + h - 1]; }, &dg);
    if (bits) bits[q] = dg.delta_bits;
    if (ct_exp) ct_exp[q] = dg.ct_exp;
    if (cut_rel) for (int k = 0; k < K - 2; ++k) cut_rel[q * 6 + k] = dg.cut_rel[k];
    if (beta_ct) beta_ct[q] = dg.beta_ct;
  }
}

/* Pieces of the reconstruction for the pin tests: candidates, beta_k, beta_K, tau_K,
   the MP bounds and the TVD5 / VA fluxes of one sequence f[0..K-1]. */
void orc_recon_parts(const Scheme* s, const double* f, double* cand, double* beta, double* betaK,
                     double* tau, double* mpmin, double* mpmax, double* tvd5, double* va) {
  Scheme S = norm_scheme(s);
  const int K = S.K, h = K / 2;
  auto F = [&](int m) { return f[m + h - 1]; };
  for (int k = 0; k < K - 2; ++k) {
    cand[k] = candidate<double>(k, F);
    beta[k] = beta_candidate<double>(k, F);
  }
  *betaK = beta_full<double>(K, F);
  *tau = std::fabs(*betaK - (beta[1] + beta[2] + 4.0 * beta[0]) / 6.0);
  mp_bounds<double>(S, F, mpmin, mpmax);
  *tvd5 = tvd5_flux<double>(F);
  *va = va_flux<double>(F);
}

void orc_init_state(const Grid* g, const double* prim, double* U) {
  Grid G = norm_grid(g);
  init_state<double>(G, prim, U);
}

int orc_faces(const Grid* g, const Scheme* s, const double* U, int axis, double* Fhat, uint8_t* flags,
              double* cut, double* noise, double* scale) {
  Grid G = norm_grid(g);
  Scheme S = norm_scheme(s);
  return all_faces<double>(G, S, U, axis, Fhat, flags, cut, noise, scale);
}

/* Face fluxes at a list of faces only (sampled parity at full size).
   faces: [n][3] cell multi-index with the face index on the axis component. */
int orc_faces_at(const Grid* g, const Scheme* s, const double* U, int axis, const int* faces, int n,
                 double* Fhat /* [n][nv] */, uint8_t* flags /* [n][nv][2] */, double* cut, double* noise,
                 double* scale /* [n][nv] */) {
  Grid G = norm_grid(g);
  Scheme S = norm_scheme(s);
  const int nv = G.dim + 2;
  int bad = 0;
  for (int q = 0; q < n; ++q) {
    int idx[3] = {faces[3 * q], faces[3 * q + 1], faces[3 * q + 2]};
    FaceDiag dg;
    double F[5];
    face_flux<double>(G, S, U, axis, idx, idx[axis], F, &dg);
    for (int v = 0; v < nv; ++v) {
      Fhat[q * nv + v] = F[v];
      if (scale) scale[q * nv + v] = dg.scale[v];
    }
    for (int v = 0; v < nv; ++v)
      for (int sd = 0; sd < 2; ++sd) {
        int o = (q * nv + v) * 2 + sd;
        if (flags) flags[o] = dg.flags[v][sd];
        if (cut) cut[o] = dg.cut[v][sd];
        if (noise) noise[o] = dg.noise[v][sd];
      }
    bad |= dg.nonphysical;
  }
  return bad;
}

/* Face fluxes of one axis after the positivity limiter of a forward-Euler stage of
   length dt (Section 4.4); the scheme's positivity flag is not consulted. */
int orc_faces_limited(const Grid* g, const Scheme* s, const double* U, int axis, double dt, double* Fhat) {
  Grid G = norm_grid(g);
  Scheme S = norm_scheme(s);
  int bad = all_faces<double>(G, S, U, axis, Fhat, nullptr, nullptr, nullptr);
  positivity_limit(G, U, axis, dt, Fhat);
  return bad;
}

/* The positivity limiter of a forward-Euler stage of length dt on caller-given face
   fluxes Fhat ([nv][nface]) of one axis, in place. */
void orc_positivity_limit(const Grid* g, const double* U, int axis, double dt, double* Fhat) {
  Grid G = norm_grid(g);
  positivity_limit(G, U, axis, dt, Fhat);
}

int orc_rhs(const Grid* g, const Scheme* s, const double* U, double* dUdt) {
  Grid G = norm_grid(g);
  Scheme S = norm_scheme(s);
  return rhs<double>(G, S, U, dUdt);
}

double orc_max_dt(const Grid* g, const double* U, double cfl) {
  Grid G = norm_grid(g);
  return max_dt(G, U, cfl);
}

int orc_rk3_step(const Grid* g, const Scheme* s, double* U, double dt) {
  Grid G = norm_grid(g);
  Scheme S = norm_scheme(s);
  return rk3_step<double>(G, S, U, dt);
}

/* Advance to t_end with dt = CFL/max signal speed, the last step clipped to t_end. */
int orc_advance(const Grid* g, const Scheme* s, double* U, double t_end, double cfl, int max_steps,
                double* t_out, int* steps_out) {
  Grid G = norm_grid(g);
  Scheme S = norm_scheme(s);
  double t = 0.0;
  int steps = 0, bad = 0;
  while (t < t_end && steps < max_steps) {
    double dt = max_dt(G, U, cfl);
    if (t + dt > t_end) dt = t_end - t;
    bad |= rk3_step<double>(G, S, U, dt);
    t += dt;
    ++steps;
  }
  *t_out = t;
  *steps_out = steps;
  return bad;
}

/* Forward-mode derivative of one RK3 step at fixed dt with every branch frozen at the
   forward values: U <- U^{n+1}, dU <- (d U^{n+1} / d U^n) dU. */
int orc_rk3_step_jvp(const Grid* g, const Scheme* s, double* U, double* dU, double dt) {
  Grid G = norm_grid(g);
  Scheme S = norm_scheme(s);
  long long N = (G.dim + 2) * ncell(G);
  std::vector<Dual> X(N);
  for (long long q = 0; q < N; ++q) X[q] = Dual(U[q], dU[q]);
  int bad = rk3_step<Dual>(G, S, X.data(), Dual(dt));
  for (long long q = 0; q < N; ++q) { U[q] = X[q].v; dU[q] = X[q].d; }
  return bad;
}

/* Forward-mode derivative of the operator L at U in direction dU (branches frozen). */
int orc_rhs_jvp(const Grid* g, const Scheme* s, const double* U, const double* dU, double* L, double* dL) {
  Grid G = norm_grid(g);
  Scheme S = norm_scheme(s);
  long long N = (G.dim + 2) * ncell(G);
  std::vector<Dual> X(N), Y(N);
  for (long long q = 0; q < N; ++q) X[q] = Dual(U[q], dU[q]);
  int bad = rhs<Dual>(G, S, X.data(), Y.data());
  for (long long q = 0; q < N; ++q) { L[q] = Y[q].v; dL[q] = Y[q].d; }
  return bad;
}

/* Counted FP64 operations of all faces of one axis (+,-,*,/,sqrt, compare/min/max/abs). */
long long orc_face_flops(const Grid* g, const Scheme* s, const double* U, int axis) {
  Grid G = norm_grid(g);
  Scheme S = norm_scheme(s);
  long long nf = nface(G, axis);
  long long N = (G.dim + 2) * ncell(G);
  std::vector<Counted> X(N), Fh((size_t)(G.dim + 2) * nf);
  for (long long q = 0; q < N; ++q) X[q] = Counted(U[q]);
  g_flops = 0;
  all_faces<Counted>(G, S, X.data(), axis, Fh.data(), nullptr, nullptr, nullptr);
  return g_flops;
}

/* Counted FP64 operations of the faces listed in faces[n][3] (one face per entry). */
long long orc_face_flops_at(const Grid* g, const Scheme* s, const double* U, int axis, const int* faces, int n) {
  Grid G = norm_grid(g);
  Scheme S = norm_scheme(s);
  long long N = (G.dim + 2) * ncell(G);
  std::vector<Counted> X(N);
  for (long long q = 0; q < N; ++q) X[q] = Counted(U[q]);
  g_flops = 0;
  for (int q = 0; q < n; ++q) {
    int idx[3] = {faces[3 * q], faces[3 * q + 1], faces[3 * q + 2]};
    Counted F[5];
    face_flux<Counted>(G, S, X.data(), axis, idx, idx[axis], F, nullptr);
  }
  return g_flops;
}

void orc_roe_eigen(const Grid* g, const double* UL, const double* UR, int axis, double* R, double* L) {
  Grid G = norm_grid(g);
  Point<double> PL, PR;
  point_from_U(G, UL, &PL);
  point_from_U(G, UR, &PR);
  Eigen<double> E;
  roe_eigen(G, PL, PR, axis, &E);
  const int nv = G.dim + 2;
  for (int i = 0; i < nv; ++i)
    for (int j = 0; j < nv; ++j) { R[i * nv + j] = E.R[i][j]; L[i * nv + j] = E.L[i][j]; }
}

void orc_phys_flux(const Grid* g, const double* U, int axis, double* F) {
  Grid G = norm_grid(g);
  Point<double> P;
  point_from_U(G, U, &P);
  phys_flux(G, P, axis, F);
}

void orc_scalar_rhs(const Scheme* s, int n, double dx, const double* u, double* dudt) {
  Scheme S = norm_scheme(s);
  scalar_rhs<double>(S, n, dx, u, dudt);
}

void orc_scalar_advance(const Scheme* s, int n, double dx, double* u, double dt, int nsteps) {
  Scheme S = norm_scheme(s);
  for (int q = 0; q < nsteps; ++q) scalar_rk3<double>(S, n, dx, u, dt);
}

/* Exact Riemann solution sampled at xi[0..n-1]; returns 1 on vacuum. */
int orc_exact_riemann(double rl, double ul, double pl, double rr, double ur, double pr, double gamma,
                      const double* xi, int n, double* rho, double* u, double* p, double* star) {
  RiemannState L{rl, ul, pl}, R{rr, ur, pr};
  double ps, us;
  if (star_state(L, R, gamma, &ps, &us)) return 1;
  star[0] = ps;
  star[1] = us;
  for (int q = 0; q < n; ++q) {
    RiemannState W = sample(L, R, gamma, ps, us, xi[q]);
    rho[q] = W.rho; u[q] = W.u; p[q] = W.p;
  }
  return 0;
}

}  // extern "C"
