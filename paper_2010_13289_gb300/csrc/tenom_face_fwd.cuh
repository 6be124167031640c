/* Forward face flux with an FP32 screen of the cutoff decisions (Section 4 of arXiv
 * 2010.13289: Roe-averaged characteristic decomposition, local Lax-Friedrichs splitting,
 * TENO-M per characteristic field and split side, back-projection).
 *
 * Where every candidate of both split sides of a field is smooth (delta_k = 1, Eq.
 * cut-off) and the optimal weights are the maximal-order d_k, the field's reconstruction
 * is the K-point central formula on both sides; the mirrored f- stencil carries the same
 * symmetric coefficients c_q, so f+ + f- = sum_q c_q (g+_q + g-_q) = sum_q c_q G_q =
 * l_s . Fc with Fc = sum_q c_q F(U_q): the LLF terms cancel, and when every field of the
 * face is such a field the back-projection returns Fc itself (R L = I).  So a field needs
 * its FP64 characteristic projection only when some candidate is not certainly smooth:
 *   all fields central:  Fhat = Fc;
 *   otherwise:           Fhat = sum_s r_s fs, fs = l_s . Fc for the central fields and
 *                        f+ + f- reconstructed in FP64 for the others.
 * Whether a field is central is decided first in FP32: the characteristic sequences
 * g+-_q = (G_q +- alpha W_q)/2 are projected in FP32 from FP32 copies of the point data,
 * with a rigorous bound E on each difference, and screen_smooth certifies that every
 * candidate is smooth over that error box.  The other fields are queued per warp (their
 * l_s and alpha/2) and the CTA's threads then work through all its warps' queues together:
 * FP64 projection from the tile, certified or FP64 decisions, central formula or
 * general reconstruction, so the FP64 work runs in as few, as full warps as it can.  A queued field whose
 * two sides turn out all smooth is central too (fs = l_s . Fc), so the result does not
 * depend on which test decided.  The physical flux is not staged:
 * G = l . F(U) = u_n (l . U) + p (l_{1+a} + u_n l_E).
 */
#pragma once
#include <cstddef>
#include "tenom_recon.cuh"

namespace tenom {

/* staged point data of the forward kernels: doubles U, velocity, H, sqrt(rho), p,
   |u_a - c|, |u_a + c|; floats (for the screen) U, u_a, p and the FP64 differences to the
   next point along the axis of U, u_a, p, each truncated to FP32 */
template <int NV>
struct PointLayoutF {
  static constexpr int NC = 2 * NV + 3;
  static constexpr int cU = 0, cV = NV, cH = 2 * NV - 2, cS = 2 * NV - 1, cP = 2 * NV, cLm = 2 * NV + 1,
                       cLp = 2 * NV + 2;
  static constexpr int NF = 2 * NV + 4;
  static constexpr int fU = 0, fN = NV, fP = NV + 1, fdU = NV + 2, fdN = 2 * NV + 2, fdP = 2 * NV + 3;
};

template <int NV, int AXIS>
__device__ __forceinline__ void stage_point_fwd(const double (&u)[NV], const double (&vel)[NV - 2], double pr,
                                                double Hh, double c, double sr, double* sm, float* smf, int NP, int p) {
  using L = PointLayoutF<NV>;
  constexpr int D = NV - 2;
  const double un = vel[AXIS];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    sm[(L::cU + q) * NP + p] = u[q];
    smf[(L::fU + q) * NP + p] = f32_rz(u[q]);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) sm[(L::cV + d) * NP + p] = vel[d];
  sm[L::cH * NP + p] = Hh;
  sm[L::cS * NP + p] = sr;
  sm[L::cP * NP + p] = pr;
  sm[L::cLm * NP + p] = iabs(un - c);
  sm[L::cLp * NP + p] = iabs(un + c);
  smf[L::fN * NP + p] = f32_rz(un);
  smf[L::fP * NP + p] = f32_rz(pr);
}

/* field queue of a warp: FQCAP items, component-major: l (NV rows), alpha/2, a header
   (face row, lane, field; after processing also the two flag bytes and the all-smooth
   bits) and the result f+ + f- */
constexpr int FQCAP = 64;
template <int NV>
__host__ __device__ constexpr int fq_rows() { return NV + 3; }

/* one queued field: FP64 projection of its K points, decisions of both split sides
   (certified FP32 filter, else FP64), reconstruction; result and flags into its slot.
   REC: also the field's linearisation at tape(row, lane) + s (2K + 2) lstride.  The record
   kernels' tape, per face and characteristic field s, rows j = s (2K + 2) + ... with stride
   lstride (the number of faces): the reconstructed fs = f+ + f-, omegaW = sum_q delta_q W_q,
   sigma_q (K) and delta_q (K), where with the frozen linear weights op (f+) and om (f-, on
   the mirrored stencil) fs = sum_q sigma_q G_q + (alpha_s/2) delta_q W_q:
   sigma_q = (op_q + om_{K-1-q})/2, delta_q = op_q - om_{K-1-q}. */
template <int NV, int K, int LIM, int AXIS, int LANES, bool REC, class Tape>
__device__ __forceinline__ void field_queue_item(const double* sm, int NP, double* fq, int it, const SchemeDev& S,
                                                 int& st, const Tape& tape, long long lstride) {
  using L = PointLayoutF<NV>;
  constexpr unsigned all = (1u << (K - 2)) - 1u;
  const long long h = __double_as_longlong(fq[(NV + 1) * FQCAP + it]);
  const int jf = (int)(h & 0xffff), ln = (int)((h >> 16) & 31), s = (int)((h >> 21) & 7);
  double l[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) l[v] = fq[v * FQCAP + it];
  const double ha = fq[NV * FQCAP + it];
  const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);
  const bool shear = s >= 2 && s <= NV - 2;
  auto P = [&](int comp, int q) -> double { return sm[comp * NP + (jf + q) * LANES + ln]; };
  double wv[K], hgv[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const double un = P(L::cV + AXIS, q), pq = P(L::cP, q);
    double w, kap;
    if (shear) {
      w = fma(l[0], P(L::cU, q), P(L::cU + 1 + dt, q));
      kap = 0.0;
    } else {
      w = l[0] * P(L::cU, q);
#pragma unroll
      for (int v = 1; v < NV; ++v) w = fma(l[v], P(L::cU + v, q), w);
      kap = fma(un, l[NV - 1], l[1 + AXIS]);
    }
    wv[q] = w;
    hgv[q] = 0.5 * fma(pq, kap, un * w);  /* G/2 = (u_a W + p kappa)/2 */
  }
  /* the two split sides through one copy of the decisions and the reconstruction:
     f+ on g+_q = G_q/2 + (alpha/2) W_q, f- on g-_q = G_q/2 - (alpha/2) W_q mirrored about
     x_{i+1/2} */
  unsigned bp = 0, bm = 0;
  int ep = 7, em = 7;
  double f = 0.0;
  double op[REC ? K : 1], om[REC ? K : 1];  /* frozen linear weights of f+ and f- */
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    double v[K];
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = side ? fma(-ha, wv[K - 1 - q], hgv[K - 1 - q]) : fma(ha, wv[q], hgv[q]);
    unsigned b = 0;
    int e = 7;
    if (!teno_decide_fast<K>(v, S, b, e)) teno_decide_fp64<K>(v, S, b, e, st);
    if constexpr (REC) {
      double wt[K];
      f += teno_general<K, LIM, true>(v, S, b, wt);
#pragma unroll
      for (int q = 0; q < K; ++q) {
        if (side) om[q] = wt[q];
        else op[q] = wt[q];
      }
    } else {
      f += teno_general<K, LIM>(v, S, b);
    }
    if (side) {
      bm = b;
      em = e;
    } else {
      bp = b;
      ep = e;
    }
  }
  const unsigned flp = bp | ((unsigned)((ep - 7) & 3) << 6), flm = bm | ((unsigned)((em - 7) & 3) << 6);
  const unsigned sm2 = (bp == all ? 1u : 0u) | (bm == all ? 2u : 0u);
  fq[(NV + 2) * FQCAP + it] = f;
  fq[(NV + 1) * FQCAP + it] = __longlong_as_double((long long)(flp | (flm << 8) | (sm2 << 16)));
  if constexpr (REC) {
    /* fs = sum_q sigma_q G_q + (alpha/2) delta_q W_q with sigma_q = (op_q + om_{K-1-q})/2,
       delta_q = op_q - om_{K-1-q}; omegaW = sum_q delta_q W_q */
    double* o = tape(jf, ln) + (long long)s * (2 * K + 2) * lstride;
    double wW = 0.0;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const double dq = op[q] - om[K - 1 - q];
      o[(2 + q) * lstride] = 0.5 * (op[q] + om[K - 1 - q]);
      o[(2 + K + q) * lstride] = dq;
      wW = fma(dq, wv[q], wW);
    }
    o[0] = f;
    o[lstride] = wW;
  }
}

/* The CTA's threads work through the items of every warp's queue together (wq_n[w] items
   in warp w's queue at fq0 + w * FQCAP * fq_rows): item g goes to warp (g / 32 + rot) % W,
   so a few items fill one warp's lanes instead of a few lanes of each warp (a partially
   filled FP64 instruction occupies the FP64 pipe as long as a full one), and rot spreads
   that warp over the SM's schedulers from one CTA to the next. */
template <int NV, int K, int LIM, int AXIS, int LANES, int THREADS, bool REC = false, class Tape = std::nullptr_t>
__device__ __forceinline__ void field_queue_cta(const double* sm, int NP, double* fq0, const int* wq_n,
                                                const SchemeDev& S, int& st, int rot, const Tape& tape = nullptr,
                                                long long lstride = 0) {
  constexpr int W = THREADS / 32;
  int pre[W + 1];
  pre[0] = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) pre[w + 1] = pre[w] + wq_n[w];
  const int n = pre[W];
  const int t = ((((int)threadIdx.x >> 5) + W - rot) % W) * 32 + ((int)threadIdx.x & 31);
#pragma unroll 1
  for (int g = t; g < n; g += THREADS) {
    int w = 0;
#pragma unroll
    for (int v = 1; v < W; ++v) w += (g >= pre[v]) ? 1 : 0;
    field_queue_item<NV, K, LIM, AXIS, LANES, REC>(sm, NP, fq0 + (size_t)w * FQCAP * fq_rows<NV>(), g - pre[w], S, st,
                                                   tape, lstride);
  }
}

/* FP32 differences to the next point along the axis (point p + LANES) of U, u_a and p,
   taken in FP64 and then truncated: they keep their relative precision however small
   the change from point to point. */
template <int NV, int AXIS>
__device__ __forceinline__ void stage_differences_fwd(const double* sm, float* smf, int NP, int p, int pn) {
  using L = PointLayoutF<NV>;
#pragma unroll
  for (int v = 0; v < NV; ++v) smf[(L::fdU + v) * NP + p] = f32_rz(sm[(L::cU + v) * NP + pn] - sm[(L::cU + v) * NP + p]);
  smf[L::fdN * NP + p] = f32_rz(sm[(L::cV + AXIS) * NP + pn] - sm[(L::cV + AXIS) * NP + p]);
  smf[L::fdP * NP + p] = f32_rz(sm[L::cP * NP + pn] - sm[L::cP * NP + p]);
}

/* Flux at the face whose K stencil points are the tile points (jf + q) * LANES + lane
   (doubles sm, floats smf, NP points per component), in steps so that the CTA can work
   through the fields its warps queued together:
     begin()     Roe average, LLF speeds, the central flux Fc;
     fields()    per field the FP32 screen: central fields are done, the others are queued
                 (returns false when the warp's queue is full before the last field: the
                 caller flushes and calls it again);
     readback()  after the CTA has processed the queues: the queued fields' flags and
                 f+ + f- (or central after all);
     finish()    the face flux.
   flags (may be null): NV x 2 bytes.  fq: this warp's field queue, shared by the lanes in
   am (all make each call). */
template <int NV, int K, int LIM, int AXIS, int LANES, bool REC = false>
struct FwdFace {
  static constexpr int D = NV - 2;
  double ut[D], q2, Ht, cinv, ct, b1, b2, una, a_m, a_0, a_p;
  double Fc[NV], fsv[NV];
  unsigned cmask, qmask;
  unsigned long long qslot;
  int nq, s_next;

  __device__ __forceinline__ void begin(const double* sm, int NP, int jf, int lane, double gamma, int& st) {
    using L = PointLayoutF<NV>;
    constexpr int H = K / 2;
    auto P = [&](int comp, int q) -> double { return sm[comp * NP + (jf + q) * LANES + lane]; };
    /* Roe average of cells f-1 (point H-1) and f (point H) */
    const double sL = P(L::cS, H - 1), sR = P(L::cS, H);
    const double wsum = rcp_nr(sL + sR);
    q2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      ut[d] = (sL * P(L::cV + d, H - 1) + sR * P(L::cV + d, H)) * wsum;
      q2 += ut[d] * ut[d];
    }
    Ht = (sL * P(L::cH, H - 1) + sR * P(L::cH, H)) * wsum;
    const double c2 = (gamma - 1.0) * (Ht - 0.5 * q2);
    if (!ipos(c2)) st |= ST_ROE;
    cinv = rsqrt_nr(c2);
    ct = c2 * cinv;
    b1 = (gamma - 1.0) * (cinv * cinv);
    b2 = 0.5 * q2 * b1;
    una = ut[AXIS];
    /* LLF: alpha_s = max over the K stencil points of |lambda_s|, one per eigenvalue family */
    a_m = 0.0;
    a_0 = 0.0;
    a_p = 0.0;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      a_m = imax_nonneg(a_m, P(L::cLm, q));
      a_0 = imax_nonneg(a_0, iabs(P(L::cV + AXIS, q)));
      a_p = imax_nonneg(a_p, P(L::cLp, q));
    }
    /* Fc = sum_q c_q F(U_q), F = u_a U + p (e_{1+a} + u_a e_E) */
    double cw[K];
    central_weights<K>(cw);
    double Pc = 0.0, PUc = 0.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Fc[v] = 0.0;
      fsv[v] = 0.0;
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const double cu = cw[q] * P(L::cV + AXIS, q);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fc[v] = fma(cu, P(L::cU + v, q), Fc[v]);
      Pc = fma(cw[q], P(L::cP, q), Pc);
      PUc = fma(cu, P(L::cP, q), PUc);
    }
    Fc[1 + AXIS] += Pc;
    Fc[NV - 1] += PUc;
    cmask = 0u;
    qmask = 0u;
    qslot = 0ull;
    nq = 0;
    s_next = 0;
  }

  /* left eigenvector l_s (closed form of R^{-1}) */
  __device__ __forceinline__ void left_vector(int s, double (&l)[NV]) const {
    const double sg = (s == 0) ? 1.0 : -1.0;            /* l: +1 for u-c, -1 for u+c */
    const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);  /* shear fields: tangential axes in increasing order */
    if ((s == 0) || (s == NV - 1)) {
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
      double utt = 0.0;
#pragma unroll
      for (int d = 0; d < D; ++d) utt = (d == dt) ? ut[d] : utt;
      l[0] = -utt;
#pragma unroll
      for (int d = 0; d < D; ++d) l[1 + d] = (d == dt) ? 1.0 : 0.0;
      l[NV - 1] = 0.0;
    }
  }

  /* fields s_next.. : the FP32 screen decides which are central; the others are queued */
  __device__ __forceinline__ bool fields(const float* smf, int NP, int jf, int lane, const SchemeDev& sch,
                                         uint8_t* flags, double* fq, unsigned am, double* lin = nullptr,
                                         long long lstride = 0) {
    using L = PointLayoutF<NV>;
    constexpr unsigned all = (1u << (K - 2)) - 1u;
    auto Pf = [&](int comp, int q) -> float { return smf[comp * NP + (jf + q) * LANES + lane]; };
    const float u32 = 5.9604645e-8f;
#pragma unroll 1
    for (int s = s_next; s < NV; ++s) {
      const bool acoustic = (s == 0) || (s == NV - 1);
      const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);
      const bool shear = !acoustic && s != 1;
      double l[NV];
      left_vector(s, l);
      const double ha = 0.5 * ((s == 0) ? a_m : (s == NV - 1 ? a_p : a_0));

      /* --- FP32 screen.  With W_q = l.U_q, kappa_q = l_{1+a} + u_q l_E and G_q = u_q W_q +
         p_q kappa_q, the differences of g+-_q = G_q/2 +- (alpha/2) W_q are, exactly,
           D_t = (u_{t+1} dW_t + W_t du_t + p_{t+1} l_E du_t + kappa_t dp_t)/2 +- (alpha/2) dW_t
         with dW_t = l.dU_t and dU, du, dp the FP64 differences of the point data (truncated
         to FP32), so they are formed in FP32 to within 24 u of the magnitude of their terms,
         A_t = (|u_{t+1}| dWA_t + WA_t |du_t| + |p_{t+1}| |l_E| |du_t| + |kappa_t| |dp_t|)/2 +
         (alpha/2) dWA_t, dWA = |l|.|dU|, WA = |l|.|U| (inputs truncated to FP32, 2u each, at
         most 5 terms per product sum) --- */
      int exp_ = 7, exm_ = 7;
      bool central = false;
      if (!sch.exact_decisions && sch.default_d) {
        float lf[NV], la[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          lf[v] = f32_rz(l[v]);
          la[v] = fabsf(lf[v]);
        }
        const float haf = f32_rz(ha);
        float hdgv[K - 1], dwv[K - 1];  /* G differences / 2 and W differences */
        float Am = 0.f;
        float w0 = 0.f, wa0 = 0.f;  /* W and WA of point t */
#pragma unroll
        for (int q = 0; q < K; ++q) {
          float w, wa;
          if (shear) {
            const float u0 = Pf(L::fU, q), ut1 = Pf(L::fU + 1 + dt, q);
            w = fmaf(lf[0], u0, ut1);
            wa = fmaf(la[0], fabsf(u0), fabsf(ut1));
          } else {
            w = lf[0] * Pf(L::fU, q);
            wa = la[0] * fabsf(Pf(L::fU, q));
#pragma unroll
            for (int v = 1; v < NV; ++v) {
              const float uv = Pf(L::fU + v, q);
              w = fmaf(lf[v], uv, w);
              wa = fmaf(la[v], fabsf(uv), wa);
            }
          }
          if (q > 0) {
            const int t = q - 1;  /* difference between points t and t + 1 = q */
            float dw, dwa;
            if (shear) {
              const float d0 = Pf(L::fdU, t), d1 = Pf(L::fdU + 1 + dt, t);
              dw = fmaf(lf[0], d0, d1);
              dwa = fmaf(la[0], fabsf(d0), fabsf(d1));
            } else {
              dw = lf[0] * Pf(L::fdU, t);
              dwa = la[0] * fabsf(Pf(L::fdU, t));
#pragma unroll
              for (int v = 1; v < NV; ++v) {
                const float dv = Pf(L::fdU + v, t);
                dw = fmaf(lf[v], dv, dw);
                dwa = fmaf(la[v], fabsf(dv), dwa);
              }
            }
            const float un1 = Pf(L::fN, q), p1 = Pf(L::fP, q), du = Pf(L::fdN, t);
            float dg = fmaf(w0, du, un1 * dw);
            float ag = fmaf(wa0, fabsf(du), fabsf(un1) * dwa);
            if (!shear) {
              const float kap = fmaf(Pf(L::fN, t), lf[NV - 1], lf[1 + AXIS]);
              const float kapa = fmaf(fabsf(Pf(L::fN, t)), la[NV - 1], la[1 + AXIS]);
              const float dpp = Pf(L::fdP, t);
              dg = fmaf(p1 * lf[NV - 1], du, fmaf(kap, dpp, dg));
              ag = fmaf(fabsf(p1) * la[NV - 1], fabsf(du), fmaf(kapa, fabsf(dpp), ag));
            }
            hdgv[t] = 0.5f * dg;
            dwv[t] = dw;
            Am = fmaxf(Am, fmaf(haf, dwa, 0.5f * ag));
          }
          w0 = w;
          wa0 = wa;
        }
        const float Eb = 24.f * u32 * Am * (1.f + 4.f * u32) + 1e-30f;
        const bool nex = flags != nullptr;
        /* the two sides through one copy of the screen (a smaller loop body for the
           instruction cache): f+ on d_t = dG_t/2 + (alpha/2) dW_t, f- on the stencil mirrored
           about x_{i+1/2}, d_t = -(dG/2 - (alpha/2) dW)_{K-2-t} */
        central = true;
#pragma unroll 1
        for (int side = 0; side < 2 && central; ++side) {
          float d[K - 1], mx = 0.f;
#pragma unroll
          for (int t = 0; t < K - 1; ++t) {
            d[t] = side ? -fmaf(-haf, dwv[K - 2 - t], hdgv[K - 2 - t]) : fmaf(haf, dwv[t], hdgv[t]);
            mx = fmaxf(mx, fabsf(d[t]));
          }
          int ex_s = 7;
          central = screen_smooth<K>(d, fmaf(2.f * u32, mx, Eb) * (1.f + 2.f * u32), sch, nex, ex_s);
          if (side) exm_ = ex_s;
          else exp_ = ex_s;
        }
      }
      /* queue the field (l_s, alpha/2, header) when it is not certainly central; stop first
         when the queue cannot take the warp's fields */
      const unsigned lt = (1u << (threadIdx.x & 31u)) - 1u;
      const unsigned mq = __ballot_sync(am, !central);
      const int cnt = __popc(mq);
      if (nq + cnt > FQCAP) {
        s_next = s;  /* this field again after the flush (screened twice: rare) */
        return false;
      }
      if (central) {
        cmask |= 1u << s;
        if (flags) {
          flags[2 * s] = (uint8_t)(all | ((unsigned)(exp_ - 7) << 6));
          flags[2 * s + 1] = (uint8_t)(all | ((unsigned)(exm_ - 7) << 6));
        }
        if constexpr (REC) {  /* both sides central: op = om = the central weights c */
          double cw[K];
          central_weights<K>(cw);
          double* o = lin + (long long)s * (2 * K + 2) * lstride;
#pragma unroll
          for (int q = 0; q < K; ++q) {
            o[(2 + q) * lstride] = 0.5 * (cw[q] + cw[K - 1 - q]);
            o[(2 + K + q) * lstride] = cw[q] - cw[K - 1 - q];
          }
          double fs = l[0] * Fc[0];
#pragma unroll
          for (int v = 1; v < NV; ++v) fs = fma(l[v], Fc[v], fs);
          o[0] = fs;
          o[lstride] = 0.0;
        }
      } else {
        const int r = nq + __popc(mq & lt);
#pragma unroll
        for (int v = 0; v < NV; ++v) fq[v * FQCAP + r] = l[v];
        fq[NV * FQCAP + r] = ha;
        fq[(NV + 1) * FQCAP + r] = __longlong_as_double((long long)(jf | (lane << 16) | (s << 21)));
        qmask |= 1u << s;
        qslot |= (unsigned long long)r << (7 * s);
      }
      nq += cnt;
    }
    s_next = NV;
    return true;
  }

  /* after the CTA processed the queues: flags and f+ + f- of this face's queued fields; a
     queued field found all smooth on both sides is central after all */
  __device__ __forceinline__ void readback(const double* fq, uint8_t* flags, const SchemeDev& sch) {
#pragma unroll
    for (int s = 0; s < NV; ++s)
      if (qmask >> s & 1u) {
        const int r = (int)((qslot >> (7 * s)) & 127ull);
        const unsigned h = (unsigned)__double_as_longlong(fq[(NV + 1) * FQCAP + r]);
        if (flags) {
          flags[2 * s] = (uint8_t)(h & 0xff);
          flags[2 * s + 1] = (uint8_t)((h >> 8) & 0xff);
        }
        if (((h >> 16) & 3u) == 3u && sch.default_d) cmask |= 1u << s;
        else fsv[s] = fq[(NV + 2) * FQCAP + r];
      }
    qmask = 0u;
    qslot = 0ull;
    nq = 0;
  }

  /* Fhat = Fc when every field is central, else sum_s r_s fs (right eigenvector r_s of
     field s) with fs = l_s . Fc for the central fields.  Both sums go through the vectors
     the eigenvectors share: a = (b2, -b1 u, b1) and b = cinv (u_a, -e_a, 0) give
     l_{u-c} = (a + b)/2, l_{u+c} = (a - b)/2, l_entropy = e_0 - a, l_shear = e_{1+t} - u_t e_0,
     and with sigma = f_{u-c} + f_{u+c}, delta = (f_{u+c} - f_{u-c}) c:
       F_0 = sigma + f_1,  F_{1+d} = (sigma + f_1) u_d + (delta if d = a, else f_shear(d)),
       F_E = sigma H + delta u_a + f_1 |u|^2/2 + sum_t f_t u_t
     (the same sum as the back-projection term by term, in about a third of the FP64
     operations: this runs in the lanes of the few faces that are not all central). */
  __device__ __forceinline__ void finish(double (&Fh)[NV]) const {
    constexpr unsigned allf = (1u << NV) - 1u;
    if (cmask == allf) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Fh[v] = Fc[v];
      return;
    }
    double uF = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) uF = fma(ut[d], Fc[1 + d], uF);
    const double A = fma(b2, Fc[0], b1 * (Fc[NV - 1] - uF));
    const double B = cinv * fma(una, Fc[0], -Fc[1 + AXIS]);
    double fs[NV];
    fs[0] = (cmask & 1u) ? 0.5 * (A + B) : fsv[0];
    fs[NV - 1] = (cmask >> (NV - 1) & 1u) ? 0.5 * (A - B) : fsv[NV - 1];
    fs[1] = (cmask >> 1 & 1u) ? Fc[0] - A : fsv[1];
#pragma unroll
    for (int s = 2; s <= NV - 2; ++s) {
      const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);
      fs[s] = (cmask >> s & 1u) ? fma(-ut[dt], Fc[0], Fc[1 + dt]) : fsv[s];
    }
    const double sigma = fs[0] + fs[NV - 1];
    const double delta = (fs[NV - 1] - fs[0]) * ct;
    const double m = sigma + fs[1];
    Fh[0] = m;
    double FE = fma(sigma, Ht, fma(delta, una, 0.5 * q2 * fs[1]));
#pragma unroll
    for (int d = 0; d < D; ++d) Fh[1 + d] = m * ut[d];
    Fh[1 + AXIS] += delta;
#pragma unroll
    for (int s = 2; s <= NV - 2; ++s) {
      const int dt = (s - 2) < AXIS ? (s - 2) : (s - 1);
      Fh[1 + dt] += fs[s];
      FE = fma(ut[dt], fs[s], FE);
    }
    Fh[NV - 1] = FE;
  }
};

}  // namespace tenom
