// k_misc.cu -- staggered semi-analytic push (Sect. 2.3.3), dust diffusion (Sect. 2.4),
// the common transport timestep (Sect. 2.6) and conversion of rank-space results to the
// caller's order.
#include "gd_ctx.h"
#include "gd_physics.cuh"

namespace gd {

// Sect. 2.3.3: y = (v_r, l_theta, l_phi), dy/dt = -y/t_s + y_g/t_s + f.  Drift half a step
// (angles with the old radius, then the radius), kick with the exact solution of the
// linear ODE at the midpoint, y += k (gamma (y_g - y) + f), k = (1 - e^{-gamma dt})/gamma,
// then drift the second half in mirrored order.  Gas: v_r = l_theta = 0,
// l_phi,g = sqrt(1 - 2 eta) Omega_K R * R.  Global-disk instances only.
__global__ void k_push(long long N, int n_inst, const long long* __restrict__ off,
                       const InstDev* __restrict__ P, const StateDev* __restrict__ st, double dt_in,
                       double* x, double* y, double* z, double* vr, double* lth, double* lph,
                       const double* __restrict__ s) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int b = inst_of(off, n_inst, i);
  const InstDev& p = P[b];
  if (p.geometry != GD_GEOM_DISK || p.rad) return;   // radiation: k_rad.cu
  double dt = dt_in < 0.0 ? st[P[b].unit0].dt_exe : dt_in;
  double X = x[i], Y = y[i], Zc = z[i], VR = vr[i], LT = lth[i], LP = lph[i];
  double r = sqrt(X * X + Y * Y + Zc * Zc);
  double th = acos(Zc / r);
  double ph = atan2(Y, X);
  double h = 0.5 * dt;
  double sth = sin(th);
  ph = ph + h * LP / (r * r * sth * sth);
  th = th + h * LT / (r * r);
  r = r + h * VR;
  sth = sin(th);
  double cth = cos(th);
  double fr = -p.GM / (r * r) + LT * LT / (r * r * r) + LP * LP / (r * r * r * sth * sth);
  double fth = LP * LP * cth / (r * r * sth * sth * sth);
  Gas g = gas_RZ(p, r * sth, r * cth);
  double ts = g.gst * s[i] / g.Om;
  double gam = 1.0 / ts;
  double ygph = sqrt(1.0 - 2.0 * g.eta) * g.Om * g.R * g.R;
  double k = (gam > 0.0) ? -expm1(-dt * gam) / gam : dt;
  VR = VR + k * (gam * (0.0 - VR) + fr);
  LT = LT + k * (gam * (0.0 - LT) + fth);
  LP = LP + k * (gam * (ygph - LP));
  r = r + h * VR;
  th = th + h * LT / (r * r);
  sth = sin(th);
  ph = ph + h * LP / (r * r * sth * sth);
  x[i] = r * sth * cos(ph);
  y[i] = r * sth * sin(ph);
  z[i] = r * cos(th);
  vr[i] = VR;
  lth[i] = LT;
  lph[i] = LP;
}

// Mixed form of the same step without FP64 transcendentals.  The position stays FP64 and
// each drift applies its angle increments as rotations: dphi = h l_phi / R^2 about the z
// axis and dtheta = h l_theta / r^2 in the meridional plane, through cos a - 1 =
// -2 sin^2(a/2) and sin a in FP32, then the radial step as the factor 1 + h v_r / r.  The
// kick takes the forces in FP64 from direction cosines (algebraic), the gas disk, t_s and
// the relaxation factor k in FP32, and the gas angular momentum sqrt(1 - 2 eta) sqrt(GM R)
// in FP64 so that l_phi,g - l_phi keeps its accuracy.
__global__ void k_push_f(long long N, int n_inst, const long long* __restrict__ off,
                         const InstDev* __restrict__ P, const StateDev* __restrict__ st, double dt_in,
                         double* x, double* y, double* z, double* vr, double* lth, double* lph,
                         const double* __restrict__ s) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int b = inst_of(off, n_inst, i);
  const InstDev& p = P[b];
  if (p.geometry != GD_GEOM_DISK || p.rad) return;   // radiation: k_rad.cu
  const double dt = dt_in < 0.0 ? st[P[b].unit0].dt_exe : dt_in;
  const double h = 0.5 * dt;
  double X = x[i], Y = y[i], Zc = z[i], VR = vr[i], LT = lth[i], LP = lph[i];
  drift_f(h, X, Y, Zc, VR, LT, LP, true);
  // kick at the midpoint
  const double R2 = X * X + Y * Y, R = sqrt(R2), r = sqrt(R2 + Zc * Zc);
  const double ir = 1.0 / r, sth = R * ir, cth = Zc * ir, ir2 = ir * ir;
  // f_r = -GM/r^2 + l_theta^2/r^3 + l_phi^2/(r^3 sin^2 theta), r^3 sin^2 theta = r R^2
  const double fr = (-p.GM + LT * LT * ir + LP * LP * r / R2) * ir2;
  const double fth = LP * LP * cth * ir2 / (sth * sth * sth);
  // the gas disk at the midpoint in FP32 (the forms of the FP32 diffusion coefficients)
  const float Rf = (float)R, Zf = (float)Zc;
  const float Om = sqrtf(p.f_GM / Rf) / Rf;
  const float xr = Rf / p.f_r0;
  const float cs = sqrtf((float)(kKB / (kMu * kMH)) * (p.f_T0 * powf(xr, p.f_q)));
  const float hg = cs / Om / Rf;
  const float rf = sqrtf(Rf * Rf + Zf * Zf);
  const float omr = Zf * Zf / (rf * (rf + Rf));
  const float eta = -0.5f * ((p.f_p + 0.5f * p.f_q - 1.5f) * hg * hg + p.f_q * omr);
  const float gst = 3.14159265f * p.f_rho_s / (4.0f * p.f_sigma0 * powf(xr, p.f_p)) * expf(omr / (hg * hg));
  const float gam = Om / (gst * (float)s[i]);
  const float kf = gam > 0.0f ? -expm1f(-(float)dt * gam) / gam : (float)dt;
  const double k = (double)kf, kg = (double)(kf * gam);
  const double ygph = sqrt(1.0 - 2.0 * (double)eta) * sqrt(p.GM * R);
  VR = VR - kg * VR + k * fr;
  LT = LT - kg * LT + k * fth;
  LP = LP + kg * (ygph - LP);
  drift_f(h, X, Y, Zc, VR, LT, LP, false);
  x[i] = X;
  y[i] = Y;
  z[i] = Zc;
  vr[i] = VR;
  lth[i] = LT;
  lph[i] = LP;
}

// ---------------------------------------------------------------- dust diffusion
// Sect. 2.4.  Coefficients at (R, Z) for a grain of diameter s: D_a = nu/(Sc_a (1+St^2)),
// nu = alpha c_s H_g at R, and the dt coefficients of the R and Z steps.  With
// v = (1 - R/r)/h^2 (the gas disk's vertical exponent; h^2 ~ R^(q+1)):
//   dv/dR = -Z^2/(r^3 h^2) - (q+1) v/R,  dv/dZ = R Z/(r^3 h^2),
//   dln D/dR = (q + 3/2)/R - f (dv/dR - p/R),  dln D/dZ = -f dv/dZ,  f = 2 St^2/(1+St^2),
//   dln rho_g/dR = (p - q/2 - 3/2)/R - dv/dR,  dln rho_g/dZ = -dv/dZ.
struct DiffCoef {
  double DR, DZ, Dp, aR, aZ;
};

__device__ __forceinline__ DiffCoef diff_coef(const InstDev& p, double R, double Z, double s) {
  const Gas g = gas_RZ(p, R, Z);
  const double St = g.gst * s;
  const double D = p.alpha * g.cs * g.H / (1.0 + St * St);
  const double v = (1.0 - R / g.r) / (g.h * g.h);
  const double r3h2 = g.r * g.r * g.r * (g.h * g.h);
  const double dvdR = -Z * Z / r3h2 - (p.q + 1.0) * v / R;
  const double dvdZ = R * Z / r3h2;
  const double f = 2.0 * St * St / (1.0 + St * St);
  const double chi = (double)p.diff_chi;
  DiffCoef c;
  c.DR = D / p.Sc_R;
  c.DZ = D / p.Sc_Z;
  c.Dp = D / p.Sc_phi;
  c.aR = c.DR * (1.0 / R + ((p.q + 1.5) / R - f * (dvdR - p.p / R)) + chi * ((p.p - 0.5 * p.q - 1.5) / R - dvdR));
  c.aZ = c.DZ * (-f * dvdZ - chi * dvdZ);
  return c;
}

// Two standard normals from one Philox draw (Box-Muller on the (0,1) map).
__device__ __forceinline__ void normal_pair(const InstDev& p, uint32_t i_loc, uint32_t step, uint32_t word,
                                            double& n0, double& n1) {
  const U4 w = philox(i_loc, step, 0xFFFFFFFEu, word, p.key0, p.key1);
  const double u1 = u01(w.x, w.y), u2 = u01(w.z, w.w);
  const double rad = sqrt(-2.0 * log(u1));
  double sn, cn;
  sincospi(2.0 * u2, &sn, &cn);
  n0 = rad * cn;
  n1 = rad * sn;
}

// Mixed form: the same coefficients in FP32, written in units of R so that no
// intermediate leaves the FP32 range (zeta = Z/R, rho = r/R; 1 - R/r = zeta^2/(rho(rho+1))).
// aR and aZ are the dt coefficients of the R and Z steps, as in diff_coef.
struct DiffCoefF {
  float DR, DZ, Dp, aR, aZ;
};

__device__ __forceinline__ DiffCoefF diff_coef_f(const InstDev& p, float R, float Z, float s) {
  const float zeta = Z / R;
  const float rho = sqrtf(1.0f + zeta * zeta);
  const float Om = sqrtf(p.f_GM / R) / R;
  const float xr = R / p.f_r0;
  const float T = p.f_T0 * powf(xr, p.f_q);
  const float cs = sqrtf((float)(kKB / (kMu * kMH)) * T);
  const float H = cs / Om;
  const float h2 = (H / R) * (H / R);
  const float Sigma = p.f_sigma0 * powf(xr, p.f_p);
  const float v = zeta * zeta / (rho * (rho + 1.0f)) / h2;
  const float St = 3.14159265f * p.f_rho_s / (4.0f * Sigma) * expf(v) * s;
  const float D = p.f_alpha * cs * H / (1.0f + St * St);
  const float rho3h2 = rho * rho * rho * h2;
  const float q = p.f_q, pp = p.f_p, chi = (float)p.diff_chi;
  const float R_dvdR = -(zeta * zeta / rho3h2 + (q + 1.0f) * v);
  const float R_dvdZ = zeta / rho3h2;
  const float f = 2.0f * St * St / (1.0f + St * St);
  DiffCoefF c;
  c.DR = D / (float)p.Sc_R;
  c.DZ = D / (float)p.Sc_Z;
  c.Dp = D / (float)p.Sc_phi;
  c.aR = c.DR / R * (1.0f + (q + 1.5f) - f * (R_dvdR - pp) + chi * ((pp - 0.5f * q - 1.5f) - R_dvdR));
  c.aZ = c.DZ / R * (-(f + chi) * R_dvdZ);
  return c;
}

// Mixed form: two standard normals in FP32 from the same uniforms as the FP64 form
// ((k + 1/2) 2^-52 with k = (a >> 6) 2^26 + (b >> 6)), rounded once to FP32.
__device__ __forceinline__ void normal_pair_f(const InstDev& p, uint32_t i_loc, uint32_t step, uint32_t word,
                                              float& n0, float& n1) {
  const U4 w = philox(i_loc, step, 0xFFFFFFFEu, word, p.key0, p.key1);
  const float u1 = fmaf((float)(w.x >> 6), 0x1p-26f, ((float)(w.y >> 6) + 0.5f) * 0x1p-52f);
  const float u2 = fmaf((float)(w.z >> 6), 0x1p-26f, ((float)(w.w >> 6) + 0.5f) * 0x1p-52f);
  const float rad = sqrtf(-2.0f * logf(u1));
  float sn, cn;
  sincospif(2.0f * u2, &sn, &cn);
  n0 = rad * cn;
  n1 = rad * sn;
}

// Mixed form without velocities: FP32 draws and coefficients, the displacement applied to
// the FP64 position without FP64 transcendentals -- the rotation by dphi through
// cos dphi - 1 = -2 sin^2(dphi/2) and sin dphi, the radial step as the factor 1 + dR/R.
// With velocities, their Cartesian vector is kept and (v_r, l_theta, l_phi) re-projected at
// the new position in FP64 from the direction cosines of the two positions (cos phi = x/R,
// sin theta = R/r, ...), with no transcendental function.
__global__ void k_diffuse_f(long long N, int n_inst, const long long* __restrict__ off,
                            const InstDev* __restrict__ P, const StateDev* __restrict__ st, double dt_in,
                            long long step, double* x, double* y, double* z, double* vr, double* lth,
                            double* lph, const double* __restrict__ s) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int b = inst_of(off, n_inst, i);
  const InstDev& p = P[b];
  const float dt = (float)(dt_in < 0.0 ? st[P[b].unit0].dt_exe : dt_in);
  const uint32_t il = (uint32_t)(i - p.off);
  float zR, zZ, zP, unused;
  normal_pair_f(p, il, (uint32_t)step, 0u, zR, zZ);
  normal_pair_f(p, il, (uint32_t)step, 1u, zP, unused);
  const double X = x[i], Y = y[i], Z = z[i];
  const float sf = (float)s[i];
  if (p.geometry == GD_GEOM_PATCH) {
    const DiffCoefF c = diff_coef_f(p, (float)(p.r0 + X), (float)Z, sf);
    double xn = X + (double)(sqrtf(2.0f * c.DR * dt) * zR + c.aR * dt);
    double yn = Y + (double)(sqrtf(2.0f * c.Dp * dt) * zP);
    xn -= p.box_x * floor((xn + 0.5 * p.box_x) / p.box_x);
    yn -= p.box_y * floor((yn + 0.5 * p.box_y) / p.box_y);
    x[i] = xn;
    y[i] = yn;
    z[i] = Z + (double)(sqrtf(2.0f * c.DZ * dt) * zZ + c.aZ * dt);
    return;
  }
  const float Xf = (float)X, Yf = (float)Y;
  const float Rf = sqrtf(Xf * Xf + Yf * Yf);
  float dR, dZ = 0.0f, dph = 0.0f;
  if (p.diff_mode == GD_DIFF_RING) {
    const float g = Rf / (float)p.r0;
    const float D = (float)p.D0 * g * g;
    dR = sqrtf(2.0f * D * dt) * zR + D / Rf * (3.0f + (float)p.diff_chi * (float)p.p) * dt;
  } else {
    const DiffCoefF c = diff_coef_f(p, Rf, (float)Z, sf);
    dR = sqrtf(2.0f * c.DR * dt) * zR + c.aR * dt;
    dZ = sqrtf(2.0f * c.DZ * dt) * zZ + c.aZ * dt;
    dph = sqrtf(2.0f * c.Dp * dt) * zP / Rf;
  }
  const float sh = sinf(0.5f * dph);
  const double cm1 = (double)(-2.0f * sh * sh), s1 = (double)sinf(dph);
  const double xr = X + (cm1 * X - s1 * Y), yr = Y + (cm1 * Y + s1 * X);
  const double k = (double)(dR / Rf);
  const double xn = xr + k * xr, yn = yr + k * yr, zn = Z + (double)dZ;
  x[i] = xn;
  y[i] = yn;
  z[i] = zn;
  if (vr && lth && lph) {
    const double R2 = X * X + Y * Y, R = sqrt(R2), r = sqrt(R2 + Z * Z);
    const double iR = 1.0 / R, ir = 1.0 / r;
    const double sth = R * ir, cth = Z * ir, cp = X * iR, sp = Y * iR;
    const double vth = lth[i] * ir, vph = lph[i] * iR, v_r = vr[i];
    const double vx = v_r * sth * cp + vth * cth * cp - vph * sp;
    const double vy = v_r * sth * sp + vth * cth * sp + vph * cp;
    const double vz = v_r * cth - vth * sth;
    const double Rn2 = xn * xn + yn * yn, Rn = sqrt(Rn2), rn = sqrt(Rn2 + zn * zn);
    const double iRn = 1.0 / Rn, irn = 1.0 / rn;
    const double sthn = Rn * irn, cthn = zn * irn, cpn = xn * iRn, spn = yn * iRn;
    vr[i] = vx * sthn * cpn + vy * sthn * spn + vz * cthn;
    lth[i] = rn * (vx * cthn * cpn + vy * cthn * spn - vz * sthn);
    lph[i] = Rn * (-vx * spn + vy * cpn);
  }
}

// One Euler-Maruyama step per particle (caller order), every instance.
__global__ void k_diffuse(long long N, int n_inst, const long long* __restrict__ off,
                          const InstDev* __restrict__ P, const StateDev* __restrict__ st, double dt_in,
                          long long step, double* x, double* y, double* z, double* vr, double* lth,
                          double* lph, const double* __restrict__ s) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int b = inst_of(off, n_inst, i);
  const InstDev& p = P[b];
  const double dt = dt_in < 0.0 ? st[P[b].unit0].dt_exe : dt_in;
  const uint32_t il = (uint32_t)(i - p.off);
  double zR, zZ, zP, unused;
  normal_pair(p, il, (uint32_t)step, 0u, zR, zZ);
  normal_pair(p, il, (uint32_t)step, 1u, zP, unused);
  if (p.geometry == GD_GEOM_PATCH) {
    const DiffCoef c = diff_coef(p, p.r0 + x[i], z[i], s[i]);
    double xn = x[i] + (sqrt(2.0 * c.DR * dt) * zR + c.aR * dt);
    double yn = y[i] + sqrt(2.0 * c.Dp * dt) * zP;
    xn -= p.box_x * floor((xn + 0.5 * p.box_x) / p.box_x);
    yn -= p.box_y * floor((yn + 0.5 * p.box_y) / p.box_y);
    x[i] = xn;
    y[i] = yn;
    z[i] = z[i] + (sqrt(2.0 * c.DZ * dt) * zZ + c.aZ * dt);
    return;
  }
  const double X = x[i], Y = y[i], Z = z[i];
  const double R = sqrt(X * X + Y * Y);
  const double ph = atan2(Y, X);
  double dR, dZ = 0.0, dph = 0.0;
  if (p.diff_mode == GD_DIFF_RING) {
    const double D = p.D0 * (R / p.r0) * (R / p.r0);
    dR = sqrt(2.0 * D * dt) * zR + D / R * (3.0 + (double)p.diff_chi * p.p) * dt;
  } else {
    const DiffCoef c = diff_coef(p, R, Z, s[i]);
    dR = sqrt(2.0 * c.DR * dt) * zR + c.aR * dt;
    dZ = sqrt(2.0 * c.DZ * dt) * zZ + c.aZ * dt;
    dph = sqrt(2.0 * c.Dp * dt) * zP / R;
  }
  double Rn = R + dR, phn = ph + dph;
  const double Zn = Z + dZ;
  if (Rn < 0.0) { Rn = -Rn; phn += kPi; }
  double spn, cpn;
  sincos(phn, &spn, &cpn);
  if (vr && lth && lph) {
    // keep the Cartesian velocity; its spherical components in the new basis
    const double r = sqrt(R * R + Z * Z), sth = R / r, cth = Z / r;
    double sp, cp;
    sincos(ph, &sp, &cp);
    const double vth = lth[i] / r, vph = lph[i] / (r * sth);
    const double vx = vr[i] * sth * cp + vth * cth * cp - vph * sp;
    const double vy = vr[i] * sth * sp + vth * cth * sp + vph * cp;
    const double vz = vr[i] * cth - vth * sth;
    const double rn = sqrt(Rn * Rn + Zn * Zn), sthn = Rn / rn, cthn = Zn / rn;
    vr[i] = vx * sthn * cpn + vy * sthn * spn + vz * cthn;
    lth[i] = rn * (vx * cthn * cpn + vy * cthn * spn - vz * sthn);
    lph[i] = rn * sthn * (-vx * spn + vy * cpn);
  }
  x[i] = Rn * cpn;
  y[i] = Rn * spn;
  z[i] = Zn;
}

// ---------------------------------------------------------------- transport timestep
// Sect. 2.6: the local limit dt_i of one particle; +infinity when no limit applies.
__device__ __forceinline__ double local_dt(const InstDev& p, const gd_dt_rule& r, double x, double y,
                                           double z, double s, bool has_v, double vr, double lth,
                                           double lph) {
  const double R = p.geometry == GD_GEOM_PATCH ? p.r0 + x : sqrt(x * x + y * y);
  const Gas g = gas_RZ(p, R, z);
  double dt = __longlong_as_double(0x7FF0000000000000ll);
  if (r.f_orb > 0.0) dt = fmin(dt, r.f_orb * 2.0 * kPi / g.Om);
  const double dx = r.dx_H * g.H;
  if (r.c_adv > 0.0 && has_v && p.geometry == GD_GEOM_DISK) {
    const double rr = sqrt(R * R + z * z);
    const double ur = vr, uth = lth / rr, uph = lph / R - g.Om * R;
    const double u = sqrt(ur * ur + uth * uth + uph * uph);
    if (u > 0.0) dt = fmin(dt, r.c_adv * dx / u);
  }
  if (r.c_diff > 0.0) {
    double D;
    if (p.diff_mode == GD_DIFF_RING) {
      D = p.D0 * (R / p.r0) * (R / p.r0);
    } else {
      const DiffCoef c = diff_coef(p, R, z, s);
      D = fmax(c.DR, fmax(c.DZ, c.Dp));
    }
    if (D > 0.0) dt = fmin(dt, (r.c_diff * dx) * (r.c_diff * dx) / (2.0 * D));
  }
  return dt;
}

// Mixed form: the same limits in FP32 (the gas disk as in diff_coef_f), fast FP32
// quotients.  The azimuthal speed relative to the Keplerian one, l_phi / R - v_K,
// cancels for prograde orbits: it is formed as ((l_phi^2 - GM R) / R^2) / (l_phi / R + v_K)
// with l_phi^2 - GM R in FP64 (scaled by 1/R^2 into the FP32 range), so that it keeps
// its relative accuracy down to the rounding of l_phi itself.
__device__ __forceinline__ float local_dt_f(const InstDev& p, const gd_dt_rule& r, double x, double y,
                                            double z, float s, bool has_v, double vr, double lth,
                                            double lph) {
  const float R = p.geometry == GD_GEOM_PATCH ? (float)(p.r0 + x)
                                              : sqrtf((float)x * (float)x + (float)y * (float)y);
  const float Z = (float)z;
  const float vK = sqrtf(__fdividef(p.f_GM, R));
  const float Om = __fdividef(vK, R);
  const float T = p.f_T0 * powf(__fdividef(R, p.f_r0), p.f_q);
  const float cs = sqrtf((float)(kKB / (kMu * kMH)) * T);
  const float H = __fdividef(cs, Om);
  float dt = __int_as_float(0x7F800000);
  if (r.f_orb > 0.0) dt = fminf(dt, __fdividef((float)(r.f_orb * 2.0 * kPi), Om));
  const float dx = (float)r.dx_H * H;
  if (r.c_adv > 0.0 && has_v && p.geometry == GD_GEOM_DISK) {
    const float rr = sqrtf(R * R + Z * Z);
    const float lR = __fdividef((float)lph, R);
    float uph;
    if (lph > 0.0) {
      const double Rd = sqrt(x * x + y * y);
      const float dl2 = (float)((lph * lph - p.GM * Rd) * (double)__fdividef(1.0f, R * R));
      uph = __fdividef(dl2, lR + vK);
    } else {
      uph = lR - vK;
    }
    const float ur = (float)vr, uth = __fdividef((float)lth, rr);
    const float u = sqrtf(ur * ur + uth * uth + uph * uph);
    if (u > 0.0f) dt = fminf(dt, __fdividef((float)r.c_adv * dx, u));
  }
  if (r.c_diff > 0.0) {
    float D;
    if (p.diff_mode == GD_DIFF_RING) {
      const float g = __fdividef(R, p.f_r0);
      D = (float)p.D0 * g * g;
    } else {
      const DiffCoefF c = diff_coef_f(p, R, Z, s);
      D = fmaxf(c.DR, fmaxf(c.DZ, c.Dp));
    }
    const float cdx = (float)r.c_diff * dx;
    if (D > 0.0f) dt = fminf(dt, __fdividef(cdx * cdx, 2.0f * D));
  }
  return dt;
}

// Grid-stride over the particles (caller order); each block's minimum joins the
// context's with one atomicMin on the bit pattern (positive doubles and +infinity
// order as their bits).  A dt_i that is NaN or not > 0 sets *bad instead.
template <bool kMixed>
__global__ void __launch_bounds__(256) k_timestep(long long N, int n_inst, const long long* __restrict__ off,
                                                  const InstDev* __restrict__ P, gd_dt_rule r,
                                                  const double* __restrict__ x, const double* __restrict__ y,
                                                  const double* __restrict__ z, const double* __restrict__ s,
                                                  const double* __restrict__ vr, const double* __restrict__ lth,
                                                  const double* __restrict__ lph, double* dti_out,
                                                  unsigned long long* d_min, unsigned long long* d_bad) {
  const bool has_v = vr && lth && lph;
  double m = __longlong_as_double(0x7FF0000000000000ll);
  bool bad = false;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = inst_of(off, n_inst, i);
    double t;
    if constexpr (kMixed)
      t = (double)local_dt_f(P[b], r, x[i], y[i], z[i], (float)s[i], has_v, has_v ? vr[i] : 0.0,
                             has_v ? lth[i] : 0.0, has_v ? lph[i] : 0.0);
    else
      t = local_dt(P[b], r, x[i], y[i], z[i], s[i], has_v, has_v ? vr[i] : 0.0, has_v ? lth[i] : 0.0,
                   has_v ? lph[i] : 0.0);
    if (dti_out) dti_out[i] = t;
    if (t > 0.0) m = fmin(m, t);
    else bad = true;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  __shared__ double wm[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wm[w] = m;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(d_bad, 1ull);
  if (threadIdx.x == 0) {
    double bm = wm[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) bm = fmin(bm, wm[k]);
    atomicMin(d_min, (unsigned long long)__double_as_longlong(bm));
  }
}

cudaError_t launch_timestep(gd_ctx* c, const gd_dt_rule& r, double* dti_out, unsigned long long* d_min,
                            unsigned long long* d_bad) {
  time_begin(c, 6);
  long long blocks = (c->N + 255) / 256;
  if (blocks > 8LL * c->num_sms) blocks = 8LL * c->num_sms;
  if (blocks < 1) blocks = 1;
  if (c->precision == GD_MIXED)
    k_timestep<true><<<(int)blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, r, c->x, c->y,
                                                         c->z, c->s, c->vr, c->lth, c->lph, dti_out, d_min, d_bad);
  else
    k_timestep<false><<<(int)blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, r, c->x, c->y,
                                                          c->z, c->s, c->vr, c->lth, c->lph, dti_out, d_min, d_bad);
  time_end(c);
  c->launches += 1;
  return cudaGetLastError();
}

__global__ void k_out_knn(long long N, int K, const int* __restrict__ rank_of, const int* __restrict__ perm,
                          const int* __restrict__ nbr, const double* __restrict__ dist, int* nbr_out,
                          double* d_out) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * K) return;
  long long i = t / K;
  int k = (int)(t - i * K);
  int r = rank_of[i];
  if (nbr_out) nbr_out[t] = perm[nbr[(long long)r * K + k]];
  if (d_out && k == 0) d_out[i] = dist[r];
}

__global__ void k_out_lam(long long N, const int* __restrict__ rank_of, const double* __restrict__ lam,
                          double* out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = lam[rank_of[i]];
}

cudaError_t launch_push(gd_ctx* c, double dt) {
  if (c->any_rad) {
    cudaError_t e = launch_push_rad(c, dt);
    if (e != cudaSuccess) return e;
  }
  if (!c->any_plain_push) {
    c->moved = true;
    return cudaSuccess;
  }
  time_begin(c, 5);
  int blocks = (int)((c->N + 255) / 256);
  if (c->precision == GD_MIXED)
    k_push_f<<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_state, dt, c->x, c->y,
                                            c->z, c->vr, c->lth, c->lph, c->s);
  else
    k_push<<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_state, dt, c->x, c->y,
                                          c->z, c->vr, c->lth, c->lph, c->s);
  time_end(c);
  c->launches += 1;
  c->moved = true;
  return cudaGetLastError();
}

cudaError_t launch_diffuse(gd_ctx* c, double dt) {
  time_begin(c, 7);
  const int blocks = (int)((c->N + 255) / 256);
  if (c->precision == GD_MIXED)
    k_diffuse_f<<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_state, dt,
                                               c->diff_step, c->x, c->y, c->z, c->vr, c->lth, c->lph, c->s);
  else
    k_diffuse<<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_state, dt,
                                             c->diff_step, c->x, c->y, c->z, c->vr, c->lth, c->lph, c->s);
  time_end(c);
  c->launches += 1;
  c->diff_step += 1;
  c->moved = true;
  return cudaGetLastError();
}

cudaError_t launch_outputs_knn(gd_ctx* c, int* nbr_out, double* d_out) {
  if (!nbr_out && !d_out) return cudaSuccess;
  long long n = c->N * c->K;
  k_out_knn<<<(int)((n + 255) / 256), 256, 0, c->stream>>>(c->N, c->K, c->d_rank_of, c->d_perm, c->d_nbr,
                                                           c->d_dist, nbr_out, d_out);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_outputs_lam(gd_ctx* c, double* lam_out) {
  if (!lam_out) return cudaSuccess;
  k_out_lam<<<(int)((c->N + 255) / 256), 256, 0, c->stream>>>(c->N, c->d_rank_of, c->d_lam, lam_out);
  c->launches += 1;
  return cudaGetLastError();
}

}  // namespace gd
