/* Frozen-branch linearisation of the face flux (adjoint of Sections 2-4 with every branch
 * taken from the forward pass; the linear form of one reconstruction is in tenom_linear.cuh).
 *
 * face_vjp_smem() is the reverse-mode derivative of face_flux_smem(): given the adjoint Fbar
 * of one face flux it returns, for each of the K stencil points, the adjoint of the point's
 * conserved state, through the back-projection, the frozen reconstructions, the LLF split
 * (alpha's argmax frozen), the characteristic projection, the Roe-averaged eigenvectors and
 * the point quantities (primitives, physical flux). */
#pragma once
#include "tenom_face.cuh"

namespace tenom {

/* Reverse of the point quantities (stage_point): adjoints of the physical flux F_AXIS (Fb),
   of the velocity (velb), sound speed (cb), enthalpy (Hb) and sqrt(rho) (sb) of one point
   -> adjoint of its conserved state, added to Ub. */
template <int NV, int AXIS>
__device__ __forceinline__ void point_vjp(const double* sm, const double* rec, int NP, int p, double gamma,
                                          const double (&Fb)[NV], double (&velb)[NV - 2], double cb, double Hb,
                                          double sb, double* Ub, int ustride) {
  using L = PointLayout<NV>;
  constexpr int D = NV - 2;
  const double rho = sm[L::cU * NP + p], E = sm[(L::cU + NV - 1) * NP + p];
  double m[D], vel[D], ke = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    m[d] = sm[(L::cU + 1 + d) * NP + p];
    vel[d] = sm[(L::cV + d) * NP + p];
    ke += m[d] * vel[d];
  }
  const double pr = (gamma - 1.0) * (E - 0.5 * ke);
  const double H = sm[L::cH * NP + p], c = sm[L::cC * NP + p];
  const double un = vel[AXIS];
  const double rinv = rec[p];                 /* 1/rho */
  double rhob = 0.0, Eb = 0.0, pb = 0.0, mb[D];
#pragma unroll
  for (int d = 0; d < D; ++d) mb[d] = 0.0;
  /* physical flux F = (rho un, m un + p e_a, (E + p) un) */
  double unb = rho * Fb[0];
  rhob += un * Fb[0];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    mb[d] += un * Fb[1 + d];
    unb += m[d] * Fb[1 + d];
  }
  pb += Fb[1 + AXIS];
  Eb += un * Fb[NV - 1];
  pb += un * Fb[NV - 1];
  unb += (E + pr) * Fb[NV - 1];
  velb[AXIS] += unb;
  /* H = (E + p)/rho */
  Eb += Hb * rinv;
  pb += Hb * rinv;
  rhob -= H * Hb * rinv;
  /* c = sqrt(gamma p / rho) */
  const double k = cb * rec[NP + p];          /* 1/(2 c rho) */
  pb += gamma * k;
  rhob -= c * c * k;
  /* sqrt(rho) */
  rhob += sb * rec[2 * NP + p];               /* 1/(2 sqrt(rho)) */
  /* p = (gamma - 1)(E - ke/2), ke = sum m_d vel_d */
  Eb += (gamma - 1.0) * pb;
  const double keb = -0.5 * (gamma - 1.0) * pb;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    mb[d] += vel[d] * keb;
    velb[d] += m[d] * keb;
  }
  /* vel_d = m_d / rho */
#pragma unroll
  for (int d = 0; d < D; ++d) {
    mb[d] += velb[d] * rinv;
    rhob -= vel[d] * velb[d] * rinv;
  }
  Ub[0] += rhob;
#pragma unroll
  for (int d = 0; d < D; ++d) Ub[(1 + d) * ustride] += mb[d];
  Ub[(NV - 1) * ustride] += Eb;
}

__device__ __forceinline__ double dsign(double x) { return ipos(x) ? 1.0 : (ineg(x) ? -1.0 : 0.0); }

/* Reverse of face_flux_smem for one face.  Fb: adjoint of the face flux.  flags: the
   forward's NV x 2 flag bytes of this face (null: decided again here).  The adjoint of
   stencil point q, component v, is ADDED to Ub[(q * NV + v) * ustride]. */
template <int NV, int K, int LIM, int AXIS, int LANES>
__device__ __forceinline__ void face_vjp_smem(const double* sm, const double* rec, int NP, int jf, int lane,
                                              double gamma, const SchemeDev& sch, const uint8_t* flags,
                                              const double (&Fb)[NV], double* Ub, int ustride, int& st) {
  using L = PointLayout<NV>;
  constexpr int D = NV - 2;
  constexpr int H = K / 2;
  auto pidx = [&](int q) { return (jf + q) * LANES + lane; };
  auto P = [&](int comp, int q) -> double { return sm[comp * NP + pidx(q)]; };
  /* ---- forward quantities of the face ---- */
  const double sL = P(L::cS, H - 1), sR = P(L::cS, H);
  const double wsum = rcp_nr(sL + sR);
  double ut[D], q2 = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    ut[d] = (sL * P(L::cV + d, H - 1) + sR * P(L::cV + d, H)) * wsum;
    q2 += ut[d] * ut[d];
  }
  const double Ht = (sL * P(L::cH, H - 1) + sR * P(L::cH, H)) * wsum;
  const double c2 = (gamma - 1.0) * (Ht - 0.5 * q2);
  const double cinv = rsqrt_nr(c2);
  const double ct = c2 * cinv;
  const double b1 = (gamma - 1.0) * (cinv * cinv);
  const double b2 = 0.5 * q2 * b1;
  const double una = ut[AXIS];
  double a_m = 0.0, a_0 = 0.0, a_p = 0.0;
  int i_m = -1, i_0 = -1, i_p = -1;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const double xm = P(L::cLm, q), x0 = iabs(P(L::cV + AXIS, q)), xp = P(L::cLp, q);
    if (dbits(a_m) < dbits(xm)) { a_m = xm; i_m = q; }
    if (dbits(a_0) < dbits(x0)) { a_0 = x0; i_0 = q; }
    if (dbits(a_p) < dbits(xp)) { a_p = xp; i_p = q; }
  }
  /* ---- adjoint accumulators ---- */
  double utb[D];
#pragma unroll
  for (int d = 0; d < D; ++d) utb[d] = 0.0;
  double Htb = 0.0, ctb = 0.0, cinvb = 0.0, b1b = 0.0, b2b = 0.0, amb = 0.0, a0b = 0.0, apb = 0.0;
  double Fq[K][NV];
#pragma unroll
  for (int q = 0; q < K; ++q)
#pragma unroll
    for (int v = 0; v < NV; ++v) Fq[q][v] = 0.0;
  /* central combination of the point fluxes, for fields smooth on both sides */
  const unsigned full = (1u << (K - 2)) - 1u;
  const bool use_fc = sch.default_d;
  double Fc[NV], accS[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    accS[v] = 0.0;
    Fc[v] = 0.0;
    if (use_fc) {
      double arr[K];
#pragma unroll
      for (int q = 0; q < K; ++q) arr[q] = P(L::cF + v, q);
      Fc[v] = central_fn<K>(arr);
    }
  }

#pragma unroll 1
  for (int s = 0; s < NV; ++s) {
    const bool acoustic = (s == 0) || (s == NV - 1);
    const double sg = (s == 0) ? 1.0 : -1.0;
    const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);
    double utt = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) utt = (d == dt) ? ut[d] : utt;
    double l[NV];
    if (acoustic) {
      l[0] = 0.5 * (b2 + sg * una * cinv);
#pragma unroll
      for (int d = 0; d < D; ++d) l[1 + d] = 0.5 * (-b1 * ut[d] - (d == AXIS ? sg * cinv : 0.0));
      l[NV - 1] = 0.5 * b1;
    } else if (s == 1) {
      l[0] = 1.0 - b2;
#pragma unroll
      for (int d = 0; d < D; ++d) l[1 + d] = b1 * ut[d];
      l[NV - 1] = -b1;
    } else {
      l[0] = -utt;
#pragma unroll
      for (int d = 0; d < D; ++d) l[1 + d] = (d == dt) ? 1.0 : 0.0;
      l[NV - 1] = 0.0;
    }
    const double ha = 0.5 * ((s == 0) ? a_m : (s == NV - 1 ? a_p : a_0));
    /* both split sides smooth with the maximal-order weights: f+ + f- = sum_q c_q (g+_q + g-_q)
       = l . sum_q c_q F_q (the central coefficients are symmetric): no alpha, no W */
    const bool smooth_lane = flags && use_fc && ((flags[2 * s] & 63u) == full) && ((flags[2 * s + 1] & 63u) == full);
    /* one path per warp: the general path is exact for smooth fields too */
    const bool smooth = __all_sync(__activemask(), smooth_lane);
    double fs = 0.0;
    bool lin_central = smooth;
    double W[K], gp[K], vm[K], op[K], omm[K];
    if (smooth) {
#pragma unroll
      for (int v = 0; v < NV; ++v) fs = fma(l[v], Fc[v], fs);
    } else {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double w, g;
      if (acoustic || s == 1) {
        w = l[0] * P(L::cU, q);
        g = l[0] * P(L::cF, q);
#pragma unroll
        for (int v = 1; v < NV; ++v) {
          w = fma(l[v], P(L::cU + v, q), w);
          g = fma(l[v], P(L::cF + v, q), g);
        }
      } else {  /* the forward's sparse shear projection */
        w = fma(-utt, P(L::cU, q), P(L::cU + 1 + dt, q));
        g = fma(-utt, P(L::cF, q), P(L::cF + 1 + dt, q));
      }
      const double hg = 0.5 * g;
      W[q] = w;
      gp[q] = fma(ha, w, hg);
      vm[K - 1 - q] = fma(-ha, w, hg);
    }
    unsigned bp, bm;
    if (flags) {
      bp = flags[2 * s] & 63u;
      bm = flags[2 * s + 1] & 63u;
    } else {
      unsigned f1, f2;
      teno_m<K, LIM>(gp, sch, f1, st);
      teno_m<K, LIM>(vm, sch, f2, st);
      bp = f1 & 63u;
      bm = f2 & 63u;
    }
    const bool cp = teno_m_weights<K, LIM>(gp, bp, sch, op);
    const bool cm = teno_m_weights<K, LIM>(vm, bm, sch, omm);
#pragma unroll
    for (int q = 0; q < K; ++q) fs += op[q] * gp[q] + omm[q] * vm[q];
    /* both reconstructions are the central scheme: the cheap reverse applies */
    lin_central = use_fc && __all_sync(__activemask(), cp && cm);
    }
    /* back-projection F = sum_s r_s fs: adjoint of fs and of r_s */
    double fsb;
    if (acoustic) {
      const double sr = -sg;
      fsb = Fb[0];
#pragma unroll
      for (int d = 0; d < D; ++d) fsb += (ut[d] + (d == AXIS ? sr * ct : 0.0)) * Fb[1 + d];
      fsb += (Ht + sr * una * ct) * Fb[NV - 1];
#pragma unroll
      for (int d = 0; d < D; ++d) utb[d] += fs * Fb[1 + d];
      ctb += sr * fs * Fb[1 + AXIS] + sr * una * fs * Fb[NV - 1];
      Htb += fs * Fb[NV - 1];
      utb[AXIS] += sr * ct * fs * Fb[NV - 1];
    } else if (s == 1) {
      fsb = Fb[0];
#pragma unroll
      for (int d = 0; d < D; ++d) fsb += ut[d] * Fb[1 + d];
      fsb += 0.5 * q2 * Fb[NV - 1];
#pragma unroll
      for (int d = 0; d < D; ++d) utb[d] += fs * (Fb[1 + d] + ut[d] * Fb[NV - 1]);
    } else {
      fsb = utt * Fb[NV - 1];
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (d == dt) fsb += Fb[1 + d];
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (d == dt) utb[d] += fs * Fb[NV - 1];
    }
    double lb[NV];
    if (lin_central) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        lb[v] = fsb * Fc[v];
        accS[v] = fma(fsb, l[v], accS[v]);
      }
    } else {
      /* frozen reconstructions and LLF split: g+ = ha W + G/2, g- = -ha W + G/2 */
      double hab = 0.0;
#pragma unroll
      for (int v = 0; v < NV; ++v) lb[v] = 0.0;
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const double gpb = op[q] * fsb, gmb = omm[K - 1 - q] * fsb;
        const double Wb = ha * (gpb - gmb), Gb = 0.5 * (gpb + gmb);
        hab += W[q] * (gpb - gmb);
        if (acoustic || s == 1) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            Ub[(q * NV + v) * ustride] += Wb * l[v];
            Fq[q][v] += Gb * l[v];
            lb[v] += Wb * P(L::cU + v, q) + Gb * P(L::cF + v, q);
          }
        } else {
          /* shear wave, l = (-u_t, e_t, 0): only l[0] depends on the Roe state */
          Ub[(q * NV) * ustride] -= Wb * utt;
          Fq[q][0] -= Gb * utt;
#pragma unroll
          for (int d = 0; d < D; ++d)
            if (d == dt) {
              Ub[(q * NV + 1 + d) * ustride] += Wb;
              Fq[q][1 + d] += Gb;
            }
          lb[0] += Wb * P(L::cU, q) + Gb * P(L::cF, q);
        }
      }
      if (s == 0) amb += 0.5 * hab;
      else if (s == NV - 1) apb += 0.5 * hab;
      else a0b += 0.5 * hab;
    }
    /* left eigenvector -> Roe state */
    if (acoustic) {
      b2b += 0.5 * lb[0];
      utb[AXIS] += 0.5 * sg * cinv * lb[0];
      cinvb += 0.5 * sg * una * lb[0];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        b1b -= 0.5 * ut[d] * lb[1 + d];
        utb[d] -= 0.5 * b1 * lb[1 + d];
      }
      cinvb -= 0.5 * sg * lb[1 + AXIS];
      b1b += 0.5 * lb[NV - 1];
    } else if (s == 1) {
      b2b -= lb[0];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        b1b += ut[d] * lb[1 + d];
        utb[d] += b1 * lb[1 + d];
      }
      b1b -= lb[NV - 1];
    } else {
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (d == dt) utb[d] -= lb[0];
    }
  }
  if (use_fc) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double e[K];
#pragma unroll
      for (int i = 0; i < K; ++i) e[i] = (i == q) ? 1.0 : 0.0;
      const double cq = central_fn<K>(e);  /* the central coefficient of point q (a constant) */
#pragma unroll
      for (int v = 0; v < NV; ++v) Fq[q][v] = fma(cq, accS[v], Fq[q][v]);
    }
  }
  /* ---- Roe average -> the two states of the face ---- */
  double q2b = 0.5 * b1 * b2b;
  b1b += 0.5 * q2 * b2b;
  cinvb += 2.0 * (gamma - 1.0) * cinv * b1b;
  double c2b = cinv * ctb;
  cinvb += c2 * ctb;
  c2b -= 0.5 * cinv * cinv * cinv * cinvb;
  Htb += (gamma - 1.0) * c2b;
  q2b -= 0.5 * (gamma - 1.0) * c2b;
  double vLb[D], vRb[D];
  double sLb = 0.0, sRb = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double u_b = utb[d] + 2.0 * ut[d] * q2b;
    vLb[d] = sL * wsum * u_b;
    vRb[d] = sR * wsum * u_b;
    sLb += (P(L::cV + d, H - 1) - ut[d]) * wsum * u_b;
    sRb += (P(L::cV + d, H) - ut[d]) * wsum * u_b;
  }
  const double HLb = sL * wsum * Htb, HRb = sR * wsum * Htb;
  sLb += (P(L::cH, H - 1) - Ht) * wsum * Htb;
  sRb += (P(L::cH, H) - Ht) * wsum * Htb;
  /* ---- points: physical flux, LLF alpha (argmax frozen), Roe inputs ---- */
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double velb[D];
#pragma unroll
    for (int d = 0; d < D; ++d) velb[d] = (q == H - 1) ? vLb[d] : ((q == H) ? vRb[d] : 0.0);
    double cb = 0.0;
    const double un = P(L::cV + AXIS, q), cq = P(L::cC, q);
    if (q == i_m) {
      const double sgm = dsign(un - cq);
      velb[AXIS] += amb * sgm;
      cb -= amb * sgm;
    }
    if (q == i_0) velb[AXIS] += a0b * dsign(un);
    if (q == i_p) {
      const double sgp = dsign(un + cq);
      velb[AXIS] += apb * sgp;
      cb += apb * sgp;
    }
    const double Hb = (q == H - 1) ? HLb : ((q == H) ? HRb : 0.0);
    const double sb = (q == H - 1) ? sLb : ((q == H) ? sRb : 0.0);
    double Fqq[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Fqq[v] = Fq[q][v];
    point_vjp<NV, AXIS>(sm, rec, NP, pidx(q), gamma, Fqq, velb, cb, Hb, sb, Ub + (q * NV) * ustride, ustride);
  }
}

}  // namespace tenom
