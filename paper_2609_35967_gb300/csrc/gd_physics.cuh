// gd_physics.cuh -- the rate model of one ordered pair, templated on FP64 / FP32.
//
// Sect. 2.2 (gas disk), 2.3.1 (Epstein Stokes number), 2.5.1 (kernel and rate),
// 2.5.2 (relative speed, outcomes, grouping), 2.5.3 (moments of the size change).
// The same device functions serve the rate kernel and the sampler, so the total
// rate lambda*_i seen by the interval choice and by the first waiting time is
// the same number.
#pragma once
#include "gd_common.cuh"

namespace gd {

// Gas and Stokes-number factor at one position, FP64 (Sect. 2.2, 2.3.1):
// Sigma = Sigma_0 (R/R_0)^p, T = T_0 (R/R_0)^q, c_s = sqrt(k_B T / (mu m_H)),
// Omega = sqrt(G M / R^3), H = c_s / Omega, h = H / R,
// rho_g = Sigma / (sqrt(2 pi) H) exp(-(1 - R/r)/h^2),
// eta = -[(p + q/2 - 3/2) h^2 + q (1 - R/r)] / 2,
// St = pi rho_o s / (4 Sigma) exp((1 - R/r)/h^2)  (gst = St / s),
// Re = alpha c_s H / nu_mol, nu_mol = sqrt(8/pi) c_s lambda_mfp / 2,
// lambda_mfp = mu m_H / (rho_g sigma_H2).
struct Gas {
  double R, Z, r, Om, T, cs, H, h, Sigma, rho, eta, Re, gst;
};

__device__ __forceinline__ Gas gas_RZ(const InstDev& P, double R, double Z) {
  Gas g;
  double r = sqrt(R * R + Z * Z);
  double Om = sqrt(P.GM / (R * R * R));
  double T = P.T0 * pow(R / P.r0, P.q);
  double cs = sqrt(kKB * T / (kMu * kMH));
  double H = cs / Om;
  double h = H / R;
  double Sigma = P.sigma0 * pow(R / P.r0, P.p);
  double vert = (1.0 - R / r) / (h * h);
  double rho = Sigma / (sqrt(2.0 * kPi) * H) * exp(-vert);
  double vth = sqrt(8.0 / kPi) * cs;
  double lmfp = kMu * kMH / (rho * kSigH2);
  double numol = 0.5 * vth * lmfp;
  g.R = R; g.Z = Z; g.r = r; g.Om = Om; g.T = T; g.cs = cs; g.H = H; g.h = h;
  g.Sigma = Sigma; g.rho = rho;
  g.eta = -0.5 * ((P.p + 0.5 * P.q - 1.5) * h * h + P.q * (1.0 - R / r));
  g.Re = P.alpha * cs * H / numol;
  g.gst = kPi * P.rho_s / (4.0 * Sigma) * exp(vert);
  return g;
}

// Patch: R = R_0 + x (x radial offset); disk: cylindrical R.
__device__ __forceinline__ Gas gas_at(const InstDev& P, double x, double y, double z) {
  double R = (P.geometry == GD_GEOM_PATCH) ? P.r0 + x : sqrt(x * x + y * y);
  return gas_RZ(P, R, z);
}

// Per-particle prefactor of the pair rates, lambda_ij = pref * (pair rate in kernel units):
// physical kernel pi / (4 V_i) (Eq. rate with K_ij = pi (s_i + s_j)^2 dv / 4), in the mixed
// form pi 2^64 / (4 V_i) because its FP32 snapshot holds N_j 2^-64; the test kernels of
// Appendix A 1 / (t0 N_K) with V_i = 1.
__device__ __forceinline__ double rate_prefactor(const InstDev& P, double V, int K, bool mixed) {
  if (P.kernel_mode != GD_KERNEL_PHYSICAL) return 1.0 / (P.t0 * (double)K);
  return mixed ? kPi * 0x1p64 / (4.0 * V) : kPi / (4.0 * V);
}

__device__ __forceinline__ double grain_mass(const InstDev& P, double s) {
  return kPi * P.rho_s * s * s * s / 6.0;
}

// <J> and <J^2> of a fragmentation (Eq. frag): a = sqrt(s_min/s_i),
// <J> = 2 (1 - a + a ln a)/(1 - a), <J^2> = 4 (2 - a ln^2 a + 2 a ln a - 2 a)/(1 - a);
// Taylor series in 1 - a below 1e-3 where the closed forms cancel.
__device__ __forceinline__ void frag_moments(double s_i, double s_min, double& j1, double& j2) {
  double a = sqrt(s_min / s_i);
  if (!(a < 1.0)) { j1 = 0.0; j2 = 0.0; return; }
  double dd = 1.0 - a;
  if (dd < 1e-3) {
    j1 = dd * (1.0 + dd * (1.0 / 3.0 + dd * (1.0 / 6.0 + dd * (1.0 / 10.0 +
         dd * (1.0 / 15.0 + dd * (1.0 / 21.0))))));
    j2 = dd * dd * (4.0 / 3.0 + dd * (1.0 + dd * (11.0 / 15.0 + dd * (5.0 / 9.0 +
         dd * (137.0 / 315.0 + dd * (7.0 / 20.0))))));
    return;
  }
  double la = log(a);
  j1 = 2.0 * (1.0 - a + a * la) / (1.0 - a);
  j2 = 4.0 * (2.0 - a * la * la + 2.0 * a * la - 2.0 * a) / (1.0 - a);
}

// Query-particle quantities of one pair evaluation, in the pair precision T.
template <typename T>
struct Query {
  T s, m, inv_m;      // live diameter, grain mass, 1/m
  T St, ai, bi, hi;   // St_i, St_i/(1+St_i^2), 1/(1+St_i^2), min(St_i, 1/2)
  T g;                // St per unit diameter at i's position
  T e2, e1, zo;       // 2 eta R Omega, eta R Omega, Z Omega
  T cs, cB, Vg2, tRe; // c_s, 8 k_B T / pi, V_g^2 = 3/2 alpha c_s^2, Re^-1/2
  T vfrag, m0;
  T ferr;             // mixed form: bound on the relative error common to the particle's FP32
                      // gas constants (St factor, drift speeds, c_s, V_g^2, Re^-1/2); 0 in FP64
  int mode;
};

template <typename T>
__device__ __forceinline__ Query<T> make_query(const InstDev& P, const Gas& g, double s, double m) {
  Query<T> q;
  double St = g.gst * s;
  q.s = (T)s; q.m = (T)m; q.inv_m = (T)(1.0 / m);
  q.St = (T)St;
  q.ai = (T)(St / (1.0 + St * St));
  q.bi = (T)(1.0 / (1.0 + St * St));
  q.hi = (T)(St < 0.5 ? St : 0.5);
  q.g = (T)g.gst;
  q.e2 = (T)(2.0 * g.eta * g.R * g.Om);
  q.e1 = (T)(g.eta * g.R * g.Om);
  q.zo = (T)(g.Z * g.Om);
  q.cs = (T)g.cs;
  q.cB = (T)(8.0 * kKB * g.T / kPi);
  q.Vg2 = (T)(1.5 * P.alpha * g.cs * g.cs);
  q.tRe = (T)(1.0 / sqrt(g.Re));
  q.vfrag = (T)P.v_frag;
  q.m0 = (T)P.m0;
  q.ferr = (T)0;
  q.mode = P.kernel_mode;
  return q;
}

// Ormel & Cuzzi (2007) closed-form regimes (the paper cites them without printing):
// St1 >= St2, eps = St2/St1, t_eta = Re^-1/2, y_a = 1.6.  regime: 0 tiny (St1 < t_eta),
// 1 intermediate (St1 < 1), 2 heavy; s1, s2 receive St1, St2.
template <typename T>
__device__ __forceinline__ T turb_dv2(T sa, T sb, T vg2, T tre, int& regime, T& s1, T& s2) {
  s1 = sa > sb ? sa : sb;
  s2 = sa > sb ? sb : sa;
  const T one = (T)1;
  // mixed form: the fast FP32 quotient (about 2 ulp; every denominator here is far inside
  // its range), which costs a fraction of the IEEE division's instruction sequence
  if constexpr (sizeof(T) == 4) {
    if (s1 < tre) {
      regime = 0;
      return vg2 * __fdividef(s1 - s2, s1 + s2) * (__fdividef(s1 * s1, s1 + tre) - __fdividef(s2 * s2, s2 + tre));
    }
    if (s1 < one) {
      regime = 1;
      T e = __fdividef(s2, s1);
      const T ya = (T)1.6;
      return vg2 * s1 * ((T)2 * ya - (one + e) + __fdividef((T)2, one + e) * ((T)(1.0 / 2.6) + __fdividef(e * e * e, ya + e)));
    }
    regime = 2;
    return vg2 * (__fdividef(one, one + s1) + __fdividef(one, one + s2));
  }
  if (s1 < tre) {
    regime = 0;
    return vg2 * (s1 - s2) / (s1 + s2) * (s1 * s1 / (s1 + tre) - s2 * s2 / (s2 + tre));
  }
  if (s1 < one) {
    regime = 1;
    T e = s2 / s1;
    const T ya = (T)1.6;
    return vg2 * s1 * ((T)2 * ya - (one + e) + (T)2 / (one + e) * (one / (one + ya) + e * e * e / (ya + e)));
  }
  regime = 2;
  return vg2 * (one / (one + s1) + one / (one + s2));
}

template <typename T>
struct PairOut {
  T c0, c1;       // effective channel rates in units of the per-particle prefactor
  T ncoll, psi;
  int outcome;    // 0 sticking, 1 erosion (c0 remnant, c1 debris), 2 fragmentation
  int cert;       // mixed form: 1 when every threshold decision of the pair (outcome,
                  // grouping, turbulence regime) is certified to be the FP64 one; FP64 form: 0
                  // when a decision lies within 1e-10 of its threshold (a near tie)
  T derr;         // mixed form: bound on the relative error of c0 and c1
  T rate;         // the pair rate before the outcome split and grouping
  int group64;    // mixed form: N_coll = floor(1e-4/psi) is beyond what the FP32 values
                  // certify (1e-4/psi above 2^23 or near an integer): regroup64 forms it in FP64
};

constexpr float kU32 = 5.9604645e-8f;     // unit roundoff of FP32, 2^-24

// One ordered pair (i, j) at i's position (Sect. 2.5.2).  Rates come out in units of
// a per-particle prefactor: physical mode q = Nq_j (s_i+s_j)^2 dv with
// lambda = q pi/(4 V_i) (Nq_j = N_j, or N_j 2^-64 in FP32); test modes
// q = (m0/m_j) K_ij with lambda = q / (t0 N_K).
//
// Mixed form: every threshold the FP32 values decide is certified against an error bound.
// St_i and St_j share the query's FP32 Stokes factor, so its relative error eps (q.ferr,
// like that of the other gas constants) scales the differences St_i - St_j, a_i - a_j, ...
// rather than cancelling; the rounding of each term (a few u of its magnitude) is what
// cancels.  With dSt = |St_i - St_j| the absolute errors are bounded by
//   dv_R: |2 eta R Omega| (3 eps dSt + 4u (a_i + a_j)) + eps |dv_R|   (a = St/(1+St^2), 1-Lipschitz)
//   dv_Z: |Z Omega| (eps dSt + 2u (h_i + h_j)) + eps |dv_Z|           (h = min(St, 1/2))
//   dv_phi: |eta R Omega| (2 eps dSt + 4u (b_i + b_j)) + eps |dv_phi| (b = 1/(1+St^2))
//   dv_B: (eps + 4u) dv_B;  dv_t^2: (9 eps + 8u) |dv_t^2| + 6u V_g^2 |St1 - St2| in the tiny
//   regime, (2 eps + 30u) |dv_t^2| in the intermediate one, (2 eps + 6u) |dv_t^2| above
// and dv^2 by E2 = 2 (2 sum |dv_k| err_k + err_t + 5u dv^2) (a factor 2 of margin).  The
// decision dv < v_frag is certified when |dv^2 - v_frag^2| > E2 + 4u v_frag^2; psi = m_j/m_i
// (relative error <= 6u) against 0.1 and 1e-6 with a margin of 16u; N_coll = floor(1e-4/psi)
// when 1e-4 m_i/m_j (an IEEE quotient, within 5u) lies more than 10u of itself from an
// integer below 2^23, else the caller forms it from the FP64 masses (group64, regroup64); the
// regime of St1 against
// Re^-1/2 and 1 with a margin of 2 (eps + 2u).  The channel rates are then within
// derr = E2 / (2 dv^2) + 8u of the FP64 ones.
template <typename T>
__device__ __forceinline__ PairOut<T> pair_channels(const Query<T>& q, T s_j, T m_j, T Nq_j, T inv_m_j) {
  PairOut<T> o;
  const T one = (T)1;
  T psi;
  if constexpr (sizeof(T) == 8) psi = m_j / q.m; else psi = m_j * q.inv_m;
  T ncoll = one;
  T vg = (T)0;      // 1e-4 / psi when grouped
  if (psi <= (T)1e-6) {
    // mixed form: 1e-4 m_i / m_j with an IEEE quotient -- within 5u of the FP64 form's
    // 1e-4 / psi (the roundings of m_i, m_j, 1e-4, the product and the quotient)
    if constexpr (sizeof(T) == 4) vg = __fdiv_rn(1e-4f * q.m, m_j); else vg = (T)1e-4 / psi;
    ncoll = floor(vg);
  }
  T rate;
  int outcome;
  bool cert = true;
  T derr = (T)0;
  if (q.mode == GD_KERNEL_PHYSICAL) {
    T St_j = q.g * s_j;
    T aj, bj;
    // one quotient for both (an FP64 division is a long sequence on the narrow FP64 pipe)
    if constexpr (sizeof(T) == 8) bj = one / (one + St_j * St_j); else bj = __fdividef(one, one + St_j * St_j);
    aj = St_j * bj;
    T hj = St_j < (T)0.5 ? St_j : (T)0.5;
    T dvR = q.e2 * (q.ai - aj);
    T dvZ = q.zo * (q.hi - hj);
    T dvP = q.e1 * (q.bi - bj);
    T vb;
    // mixed form: x rsqrt(x) for the FP32 roots (x > 0 here: masses and c_s are positive)
    if constexpr (sizeof(T) == 4) { const float xb = q.cB * (q.inv_m + inv_m_j); vb = xb * rsqrtf(xb); }
    else vb = sqrt(q.cB * (q.inv_m + inv_m_j));
    T dvB = q.cs < vb ? q.cs : vb;
    int regime;
    T s1, s2;
    T t2 = turb_dv2<T>(q.St, St_j, q.Vg2, q.tRe, regime, s1, s2);
    const T dvt2 = t2;     // the squared turbulent term enters dv^2 as it is
    T dv, xd;
    if constexpr (sizeof(T) == 4) { xd = dvR * dvR + dvZ * dvZ + dvP * dvP + dvB * dvB + dvt2; dv = xd * rsqrtf(xd); }
    else { xd = dvR * dvR + dvZ * dvZ + dvP * dvP + dvB * dvB + dvt2; dv = sqrt(xd); }
    T ss = q.s + s_j;
    rate = Nq_j * (ss * ss * dv);
    outcome = (dv < q.vfrag) ? 0 : ((psi <= (T)0.1) ? 1 : 2);
    if constexpr (sizeof(T) == 4) {
      const float u = kU32, eps = q.ferr;
      const float dSt = fabsf(q.St - St_j);
      const float eR = fabsf(q.e2) * (3.f * eps * dSt + 4.f * u * (q.ai + aj)) + eps * fabsf(dvR);
      const float eZ = fabsf(q.zo) * (eps * dSt + 2.f * u * (q.hi + hj)) + eps * fabsf(dvZ);
      const float eP = fabsf(q.e1) * (2.f * eps * dSt + 4.f * u * (q.bi + bj)) + eps * fabsf(dvP);
      const float eB = (eps + 4.f * u) * dvB;
      float eT;
      if (regime == 0) eT = (9.f * eps + 8.f * u) * fabsf(t2) + 6.f * u * q.Vg2 * (s1 - s2);
      else if (regime == 1) eT = (2.f * eps + 30.f * u) * fabsf(t2);
      else eT = (2.f * eps + 6.f * u) * fabsf(t2);
      const float E2 =
          2.f * (2.f * (fabsf(dvR) * eR + fabsf(dvZ) * eZ + fabsf(dvP) * eP + dvB * eB) + eT + 5.f * u * xd);
      const float vf2 = q.vfrag * q.vfrag;
      const float mr = 2.f * (eps + 2.f * u);
      cert = fabsf(xd - vf2) > E2 + 4.f * u * vf2 && fabsf(s1 - q.tRe) > mr * (s1 + q.tRe) &&
             fabsf(s1 - one) > mr * s1;
      if (outcome != 0) cert = cert && fabsf(psi - 0.1f) > 16.f * u * 0.1f;
      derr = __fdividef(E2, 2.f * xd) + 8.f * u;
    } else {
      const double tie = 1e-10;
      cert = !(fabs(dv - q.vfrag) <= tie * q.vfrag || fabs(s1 - q.tRe) <= tie * (s1 + q.tRe) ||
               fabs(s1 - one) <= tie || (outcome != 0 && fabs(psi - 0.1) <= tie * 0.1));
    }
  } else {
    T Kk = one;
    if (q.mode == GD_KERNEL_LINEAR) Kk = (q.m + m_j) / q.m0;
    if (q.mode == GD_KERNEL_PRODUCT) Kk = q.m * m_j / (q.m0 * q.m0);
    rate = q.m0 * inv_m_j * Kk;
    outcome = 0;
    if constexpr (sizeof(T) == 4) derr = 12.f * kU32;
  }
  // grouping: psi against 1e-6 and N_coll = floor(1e-4 / psi)
  int group64 = 0;
  if constexpr (sizeof(T) == 4) {
    const float u = kU32;
    cert = cert && fabsf(psi - 1e-6f) > 16.f * u * 1e-6f;
    if (psi <= 1e-6f && !(vg < 8388608.f && vg - ncoll > 10.f * u * vg && ncoll + 1.f - vg > 10.f * u * vg))
      group64 = 1;
  } else {
    const double tie = 1e-10;
    if (fabs(psi - 1e-6) <= tie * 1e-6) cert = false;
    if (psi <= 1e-6 && (vg - ncoll <= tie * vg || ncoll + 1.0 - vg <= tie * vg)) cert = false;
  }
  o.psi = psi;
  o.ncoll = ncoll;
  o.outcome = outcome;
  o.cert = cert ? 1 : 0;
  o.derr = derr;
  o.rate = rate;
  o.group64 = group64;
  if (outcome == 0) {
    if constexpr (sizeof(T) == 4) o.c0 = (ncoll == one) ? rate : __fdividef(rate, ncoll);
    else o.c0 = (ncoll == one) ? rate : rate / ncoll;
    o.c1 = (T)0;
  } else if (outcome == 1) {
    if constexpr (sizeof(T) == 4) o.c0 = (ncoll == one) ? (one - psi) * rate : __fdividef((one - psi) * rate, ncoll);
    else o.c0 = (ncoll == one) ? (one - psi) * rate : (one - psi) * rate / ncoll;
    o.c1 = psi * rate;
  } else {
    o.c0 = rate;
    o.c1 = (T)0;
  }
  return o;
}

// Mixed form: N_coll of a grouped pair from the FP64 masses m_i and m_j, the channel rates
// recomputed with it in FP32 (N_coll rounded to FP32, half a unit more of error).  The FP64
// form forms floor(1e-4 / (m_j / m_i)); here one FP64 quotient (1e-4 m_i) / m_j, within 4
// units of the last place of that value, so the two floors differ only within 4e-16 of an
// integer.  A count within 1e-10 of an integer boundary stays uncertified, which covers that.
__device__ __forceinline__ void regroup64(PairOut<float>& o, double m_i, double m_j) {
  const double vg = (1e-4 * m_i) / m_j;
  const double n = floor(vg);
  if (vg - n <= 1e-10 * vg || n + 1.0 - vg <= 1e-10 * vg) o.cert = 0;
  const float nf = (float)n;
  o.ncoll = nf;
  if (o.outcome == 0) o.c0 = __fdividef(o.rate, nf);
  else if (o.outcome == 1) o.c0 = __fdividef((1.0f - o.psi) * o.rate, nf);
  o.derr += 3.f * kU32;
  o.group64 = 0;
}

// J = |ln(s'/s_i)| of the deterministic channels (Sect. 2.5.3): ln(1 + N psi)/3 for
// sticking, |ln(1 - N psi)|/3 and |ln psi|/3 for the erosion remnant and debris;
// fragmentation uses the precomputed <J>, <J^2> of particle i.
template <typename T>
__device__ __forceinline__ void pair_moments(const PairOut<T>& o, T fj1, T fj2, T& a, T& b) {
  if (o.outcome == 0) {
    T J;
    if constexpr (sizeof(T) == 8) J = log1p(o.ncoll * o.psi) / 3.0; else J = log1pf(o.ncoll * o.psi) * (1.0f / 3.0f);
    a = o.c0 * J;
    b = o.c0 * (J * J);
  } else if (o.outcome == 1) {
    T J0, J1;
    if constexpr (sizeof(T) == 8) {
      J0 = fabs(log1p(-o.ncoll * o.psi) / 3.0);
      J1 = fabs(log(o.psi) / 3.0);
    } else {
      J0 = fabsf(log1pf(-o.ncoll * o.psi) * (1.0f / 3.0f));
      J1 = fabsf(logf(o.psi) * (1.0f / 3.0f));
    }
    a = o.c0 * J0 + o.c1 * J1;
    b = o.c0 * (J0 * J0) + o.c1 * (J1 * J1);
  } else {
    a = o.c0 * fj1;
    b = o.c0 * fj2;
  }
}

// Drift of the mixed staggered step (Sect. 2.3.3), half a step of length h: the FP64
// position rotated by FP32 angle increments, dphi = h l_phi / R^2 about the z axis and
// dtheta = h l_theta / r^2 in the meridional plane (cos a - 1 = -2 sin^2(a/2) and sin a in
// FP32), then scaled by 1 + h v_r / r.  The first half takes phi, theta (both at the old
// radius), radius; the second half the mirrored order.
__device__ __forceinline__ void drift_f(double h, double& X, double& Y, double& Z, double VR, double LT,
                                        double LP, bool first_half) {
  auto phi = [&]() {
    const double R2 = X * X + Y * Y;
    const float dph = (float)(h * LP) / (float)R2;
    const float s2 = sinf(0.5f * dph);
    const double c1 = (double)(-2.0f * s2 * s2), s1 = (double)sinf(dph);
    const double Xr = X + (c1 * X - s1 * Y), Yr = Y + (c1 * Y + s1 * X);
    X = Xr;
    Y = Yr;
  };
  auto theta = [&]() {
    const double R = sqrt(X * X + Y * Y), r2 = R * R + Z * Z;
    const float dth = (float)(h * LT) / (float)r2;
    const float t2 = sinf(0.5f * dth);
    const double ct = (double)(-2.0f * t2 * t2), st = (double)sinf(dth);
    // theta from +z: R' = R cos + Z sin, Z' = Z cos - R sin
    const double dR = ct * R + st * Z, dZ = ct * Z - st * R;
    const double f = 1.0 + dR / R;
    X *= f;
    Y *= f;
    Z += dZ;
  };
  auto radius = [&]() {
    const double r = sqrt(X * X + Y * Y + Z * Z);
    const double f = 1.0 + h * VR / r;
    X *= f;
    Y *= f;
    Z *= f;
  };
  // first half: phi, theta (both at the old radius), radius; second half mirrored
  if (first_half) { phi(); theta(); radius(); }
  else { radius(); theta(); phi(); }
}

}  // namespace gd
