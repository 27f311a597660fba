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
  q.mode = P.kernel_mode;
  return q;
}

// Ormel & Cuzzi (2007) closed-form regimes (the paper cites them without printing):
// St1 >= St2, eps = St2/St1, t_eta = Re^-1/2, y_a = 1.6.
template <typename T>
__device__ __forceinline__ T turb_dv2(T sa, T sb, T vg2, T tre) {
  T s1 = sa > sb ? sa : sb;
  T s2 = sa > sb ? sb : sa;
  const T one = (T)1;
  // mixed form: the fast FP32 quotient (about 2 ulp; every denominator here is far inside
  // its range), which costs a fraction of the IEEE division's instruction sequence
  if constexpr (sizeof(T) == 4) {
    if (s1 < tre) return vg2 * __fdividef(s1 - s2, s1 + s2) * (__fdividef(s1 * s1, s1 + tre) - __fdividef(s2 * s2, s2 + tre));
    if (s1 < one) {
      T e = __fdividef(s2, s1);
      const T ya = (T)1.6;
      return vg2 * s1 * ((T)2 * ya - (one + e) + __fdividef((T)2, one + e) * ((T)(1.0 / 2.6) + __fdividef(e * e * e, ya + e)));
    }
    return vg2 * (__fdividef(one, one + s1) + __fdividef(one, one + s2));
  }
  if (s1 < tre) return vg2 * (s1 - s2) / (s1 + s2) * (s1 * s1 / (s1 + tre) - s2 * s2 / (s2 + tre));
  if (s1 < one) {
    T e = s2 / s1;
    const T ya = (T)1.6;
    return vg2 * s1 * ((T)2 * ya - (one + e) + (T)2 / (one + e) * (one / (one + ya) + e * e * e / (ya + e)));
  }
  return vg2 * (one / (one + s1) + one / (one + s2));
}

template <typename T>
struct PairOut {
  T c0, c1;       // effective channel rates in units of the per-particle prefactor
  T ncoll, psi;
  int outcome;    // 0 sticking, 1 erosion (c0 remnant, c1 debris), 2 fragmentation
};

// One ordered pair (i, j) at i's position (Sect. 2.5.2).  Rates come out in units of
// a per-particle prefactor: physical mode q = Nq_j (s_i+s_j)^2 dv with
// lambda = q pi/(4 V_i) (Nq_j = N_j, or N_j 2^-64 in FP32); test modes
// q = (m0/m_j) K_ij with lambda = q / (t0 N_K).
template <typename T>
__device__ __forceinline__ PairOut<T> pair_channels(const Query<T>& q, T s_j, T m_j, T Nq_j, T inv_m_j) {
  PairOut<T> o;
  const T one = (T)1;
  T psi;
  if constexpr (sizeof(T) == 8) psi = m_j / q.m; else psi = m_j * q.inv_m;
  T ncoll = one;
  if (psi <= (T)1e-6) { if constexpr (sizeof(T) == 4) ncoll = floorf(__fdividef(1e-4f, psi)); else ncoll = floor((T)1e-4 / psi); }
  T rate;
  int outcome;
  if (q.mode == GD_KERNEL_PHYSICAL) {
    T St_j = q.g * s_j;
    T aj, bj;
    if constexpr (sizeof(T) == 8) {
      aj = St_j / (one + St_j * St_j);
      bj = one / (one + St_j * St_j);
    } else {
      bj = __fdividef(one, one + St_j * St_j);
      aj = St_j * bj;
    }
    T hj = St_j < (T)0.5 ? St_j : (T)0.5;
    T dvR = q.e2 * (q.ai - aj);
    T dvZ = q.zo * (q.hi - hj);
    T dvP = q.e1 * (q.bi - bj);
    T vb;
    // mixed form: x rsqrt(x) for the FP32 roots (x > 0 here: masses and c_s are positive)
    if constexpr (sizeof(T) == 4) { const float xb = q.cB * (q.inv_m + inv_m_j); vb = xb * rsqrtf(xb); }
    else vb = sqrt(q.cB * (q.inv_m + inv_m_j));
    T dvB = q.cs < vb ? q.cs : vb;
    T t2 = turb_dv2<T>(q.St, St_j, q.Vg2, q.tRe);
    T dvt2;
    if constexpr (sizeof(T) == 8) { T dvt = sqrt(t2); dvt2 = dvt * dvt; } else { dvt2 = t2; }
    T dv;
    if constexpr (sizeof(T) == 4) { const float xd = dvR * dvR + dvZ * dvZ + dvP * dvP + dvB * dvB + dvt2; dv = xd * rsqrtf(xd); }
    else dv = sqrt(dvR * dvR + dvZ * dvZ + dvP * dvP + dvB * dvB + dvt2);
    T ss = q.s + s_j;
    rate = Nq_j * (ss * ss * dv);
    outcome = (dv < q.vfrag) ? 0 : ((psi <= (T)0.1) ? 1 : 2);
  } else {
    T Kk = one;
    if (q.mode == GD_KERNEL_LINEAR) Kk = (q.m + m_j) / q.m0;
    if (q.mode == GD_KERNEL_PRODUCT) Kk = q.m * m_j / (q.m0 * q.m0);
    rate = q.m0 * inv_m_j * Kk;
    outcome = 0;
  }
  o.psi = psi;
  o.ncoll = ncoll;
  o.outcome = outcome;
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

}  // namespace gd
