/* Exact solution of the Riemann problem of the 1D Euler equations for an ideal gas,
   written from the wave relations of gas dynamics (shock: Rankine-Hugoniot jump
   conditions; rarefaction: isentropic fan with constant Riemann invariant; contact:
   continuous pressure and velocity).  Used to check the shock-tube runs of Section
   4.2.1 (Lax and Sod problems) and their seeded generalisation.

   TEST INFRASTRUCTURE ONLY (part of the CPU oracle). */
#pragma once
#include <cmath>

namespace orc {

struct RiemannState { double rho, u, p; };

/* Velocity change across the wave on side K as a function of the star pressure, and
   its derivative: shock branch from the Rankine-Hugoniot conditions, rarefaction
   branch from the isentropic relation p/rho^gamma = const and the Riemann invariant. */
inline void wave_fn(double p, const RiemannState& W, double g, double* f, double* df) {
  double c = std::sqrt(g * W.p / W.rho);
  if (p > W.p) {
    double A = 2.0 / ((g + 1.0) * W.rho), B = (g - 1.0) / (g + 1.0) * W.p;
    double s = std::sqrt(A / (p + B));
    *f = (p - W.p) * s;
    *df = s * (1.0 - 0.5 * (p - W.p) / (p + B));
  } else {
    double z = (g - 1.0) / (2.0 * g);
    *f = 2.0 * c / (g - 1.0) * (std::pow(p / W.p, z) - 1.0);
    *df = 1.0 / (W.rho * c) * std::pow(p / W.p, -(g + 1.0) / (2.0 * g));
  }
}

/* Star pressure and velocity: root of f_L(p) + f_R(p) + (u_R - u_L) = 0 by Newton's
   method from the two-rarefaction estimate.  Returns 0 on success, 1 on vacuum. */
inline int star_state(const RiemannState& L, const RiemannState& R, double g, double* pstar,
                      double* ustar) {
  double cL = std::sqrt(g * L.p / L.rho), cR = std::sqrt(g * R.p / R.rho);
  if (2.0 * (cL + cR) / (g - 1.0) <= R.u - L.u) return 1;  /* vacuum generated */
  double z = (g - 1.0) / (2.0 * g);
  double p = std::pow((cL + cR - 0.5 * (g - 1.0) * (R.u - L.u)) /
                          (cL / std::pow(L.p, z) + cR / std::pow(R.p, z)), 1.0 / z);
  for (int it = 0; it < 200; ++it) {
    double fL, dL, fR, dR;
    wave_fn(p, L, g, &fL, &dL);
    wave_fn(p, R, g, &fR, &dR);
    double pn = p - (fL + fR + R.u - L.u) / (dL + dR);
    if (pn <= 0) pn = 0.5 * p;
    double rel = std::fabs(pn - p) / (0.5 * (pn + p));
    p = pn;
    if (rel < 1e-15) break;
  }
  double fL, dL, fR, dR;
  wave_fn(p, L, g, &fL, &dL);
  wave_fn(p, R, g, &fR, &dR);
  *pstar = p;
  *ustar = 0.5 * (L.u + R.u) + 0.5 * (fR - fL);
  return 0;
}

/* Solution at similarity coordinate xi = (x - x0)/t. */
inline RiemannState sample(const RiemannState& L, const RiemannState& R, double g, double ps,
                           double us, double xi) {
  double g1 = (g - 1.0) / (g + 1.0), z = (g - 1.0) / (2.0 * g);
  if (xi <= us) {
    double cL = std::sqrt(g * L.p / L.rho);
    if (ps > L.p) {
      double SL = L.u - cL * std::sqrt((g + 1.0) / (2.0 * g) * ps / L.p + z);
      if (xi < SL) return L;
      return {L.rho * (ps / L.p + g1) / (g1 * ps / L.p + 1.0), us, ps};
    }
    double SH = L.u - cL, cs = cL * std::pow(ps / L.p, z), ST = us - cs;
    if (xi < SH) return L;
    if (xi > ST) return {L.rho * std::pow(ps / L.p, 1.0 / g), us, ps};
    double u = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * L.u + xi);
    double c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (L.u - xi));
    return {L.rho * std::pow(c / cL, 2.0 / (g - 1.0)), u, L.p * std::pow(c / cL, 2.0 * g / (g - 1.0))};
  }
  double cR = std::sqrt(g * R.p / R.rho);
  if (ps > R.p) {
    double SR = R.u + cR * std::sqrt((g + 1.0) / (2.0 * g) * ps / R.p + z);
    if (xi > SR) return R;
    return {R.rho * (ps / R.p + g1) / (g1 * ps / R.p + 1.0), us, ps};
  }
  double SH = R.u + cR, cs = cR * std::pow(ps / R.p, z), ST = us + cs;
  if (xi > SH) return R;
  if (xi < ST) return {R.rho * std::pow(ps / R.p, 1.0 / g), us, ps};
  double u = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * R.u + xi);
  double c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (R.u - xi));
  return {R.rho * std::pow(c / cR, 2.0 / (g - 1.0)), u, R.p * std::pow(c / cR, 2.0 * g / (g - 1.0))};
}

}  // namespace orc
