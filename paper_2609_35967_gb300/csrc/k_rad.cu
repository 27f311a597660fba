// k_rad.cu -- radiation pressure and Poynting-Robertson drag (Sect. 2.3.2) in the staggered
// semi-analytic step (Sect. 2.3.3), and the optical depth grid they see.
//
// One radiation step is five kernels:
//   k_rad_drift   first half drift of every particle of an instance with beta0 > 0; the
//                 midpoint goes to d_mid and, for instances with a grid, the particle's cell
//                 and kappa(s) M to d_tau_ci / d_tau_q, with the instance's largest kappa M
//                 (atomicMax on its bits);
//   k_tau_deposit each particle's kappa M in 128-bit fixed point, scaled by 2^(60 - e) for
//                 the instance's largest value < 2^e, added to its cell (two 64-bit words,
//                 the carry counted in the high word): exact, so independent of order;
//   k_tau_cells   one thread per cell: its sum over its volume times dr (the accumulators
//                 cleared for the next use);
//   k_tau_columns one thread per column: the radial prefix of those increments at the faces;
//   k_rad_kick    tau interpolated at the midpoint, the kick with the radiation force and the
//                 P-R damping, the second half drift;
// then k_rad_clock advances each instance's taper clock by its dt.
#include "gd_ctx.h"
#include "gd_physics.cuh"

namespace gd {

constexpr double kCLight = 2.99792458e10;     // speed of light [cm s^-1]
constexpr double kTwoPi = 2.0 * kPi;

// ---------------------------------------------------------------- grid geometry
// phi folded into [-pi, pi): ph - 2 pi floor((ph + pi) / 2 pi), correctly rounded steps
__device__ __forceinline__ double fold_phi(double ph) {
  const double f = floor(__ddiv_rn(__dadd_rn(ph, kPi), kTwoPi));
  return __dsub_rn(ph, __dmul_rn(kTwoPi, f));
}

// Local cell (radial cell i times the columns, plus the column j * nphi + k) of a point at
// grid radius rad, mu and phi; -1 outside the grid.  The same correctly rounded steps as the
// oracle's, so that both take the same cell.
__device__ __forceinline__ int tau_cell64(const InstDev& p, double rad, double mu, double phi) {
  const double dr = __ddiv_rn(__dsub_rn(p.tau_rmax, p.tau_rmin), (double)p.tau_nr);
  const double u = __ddiv_rn(__dsub_rn(rad, p.tau_rmin), dr);
  if (!(u >= 0.0) || !(u < (double)p.tau_nr)) return -1;
  const int i = (int)floor(u);
  int j = 0;
  if (p.tau_geom != GD_TAU_2D) {
    const double dmu = __ddiv_rn(2.0 * p.tau_mu, (double)p.tau_nm);
    const double w = __ddiv_rn(__dadd_rn(mu, p.tau_mu), dmu);
    if (!(w >= 0.0) || !(w < (double)p.tau_nm)) return -1;
    j = (int)floor(w);
  }
  const double dphi = __ddiv_rn(kTwoPi, (double)p.tau_np);
  int k = (int)floor(__ddiv_rn(__dadd_rn(phi, kPi), dphi));
  k = min(max(k, 0), p.tau_np - 1);
  return i * (p.tau_nm * p.tau_np) + j * p.tau_np + k;
}

// A cell coordinate estimated in FP32 with absolute error at most E (in cells): its floor
// when no integer lies within E, else -2 (undecided).
__device__ __forceinline__ int certain_floor(float v, float E) {
  const float f = floorf(v);
  return (v - f > E && (f + 1.0f) - v > E) ? (int)f : -2;
}

// Mixed form: the cell of a Cartesian FP64 point from FP32 coordinates where their error
// bounds decide it, else from the FP64 coordinates (the same cell in both cases).
__device__ __forceinline__ int tau_cell_mixed(const InstDev& p, double X, double Y, double Z) {
  const double R2 = X * X + Y * Y;
  const double r2 = p.tau_geom == GD_TAU_2D ? R2 : R2 + Z * Z;
  const float rf = sqrtf((float)r2);
  const float u = (rf - p.f_tau_rmin) / p.f_tau_dr;
  if (u < -p.f_eu || u >= (float)p.tau_nr + p.f_eu) return -1;
  int i = certain_floor(u, p.f_eu);
  int j = 0;
  if (i >= 0 && p.tau_geom != GD_TAU_2D) {
    const float w = ((float)Z / rf + p.f_tau_mu) / p.f_tau_dmu;
    if (w < -p.f_ew || w >= (float)p.tau_nm + p.f_ew) return -1;
    j = certain_floor(w, p.f_ew);
  }
  int k = 0;
  if (i >= 0 && j >= 0) {
    const float v = (atan2f((float)Y, (float)X) + 3.14159265f) / p.f_tau_dphi;
    k = certain_floor(v, p.f_ev);
    if (k >= 0) k = min(k, p.tau_np - 1);
  }
  if (i < 0 || j < 0 || k < 0) {
    // undecided in FP32: the FP64 coordinates of k_tau_bin
    const double R2r = __dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y));
    if (p.tau_geom == GD_TAU_2D) return tau_cell64(p, __dsqrt_rn(R2r), 0.0, atan2(Y, X));
    const double r = __dsqrt_rn(__dadd_rn(R2r, __dmul_rn(Z, Z)));
    return tau_cell64(p, r, __ddiv_rn(Z, r), atan2(Y, X));
  }
  if (i >= p.tau_nr || j >= p.tau_nm) return -1;
  return i * (p.tau_nm * p.tau_np) + j * p.tau_np + k;
}

// tau at grid radius rad, mu, phi from the faces T of the instance ([face][column]).
__device__ __forceinline__ double tau_interp64(const InstDev& p, const double* __restrict__ T, double rad,
                                               double mu, double phi) {
  const int nr = p.tau_nr, nm = p.tau_nm, np = p.tau_np, ncol = nm * np;
  const double dr = (p.tau_rmax - p.tau_rmin) / nr;
  const double u = (rad - p.tau_rmin) / dr;
  if (!(u > 0.0)) return 0.0;
  int i;
  double fr = 0.0;
  if (u >= (double)nr) {
    i = nr;
  } else {
    i = (int)floor(u);
    fr = u - (double)i;
  }
  int j0 = 0, j1 = 0;
  double fm = 0.0;
  if (nm > 1) {
    const double w = (mu + p.tau_mu) / (2.0 * p.tau_mu / nm) - 0.5;
    if (w <= 0.0) {
      j0 = j1 = 0;
    } else if (w >= (double)(nm - 1)) {
      j0 = j1 = nm - 1;
    } else {
      j0 = (int)floor(w);
      j1 = j0 + 1;
      fm = w - (double)j0;
    }
  }
  const double v = (phi + kPi) / (kTwoPi / np) - 0.5;
  const double kf = floor(v);
  const double fp = v - kf;
  const int k0 = (((int)kf % np) + np) % np, k1 = (k0 + 1) % np;
  const int cols[4] = {j0 * np + k0, j0 * np + k1, j1 * np + k0, j1 * np + k1};
  const double w4[4] = {(1.0 - fm) * (1.0 - fp), (1.0 - fm) * fp, fm * (1.0 - fp), fm * fp};
  const double* Ti = T + (long long)i * ncol;
  double tau = 0.0;
  for (int c = 0; c < 4; ++c) {
    const double t0 = __ldg(&Ti[cols[c]]);
    const double tc = i >= nr ? t0 : t0 + fr * (__ldg(&Ti[ncol + cols[c]]) - t0);
    tau = tau + w4[c] * tc;
  }
  return tau;
}

// The same in FP32 (mixed form).
__device__ __forceinline__ float tau_interp32(const InstDev& p, const double* __restrict__ T, float rad,
                                              float mu, float phi) {
  const int nr = p.tau_nr, nm = p.tau_nm, np = p.tau_np, ncol = nm * np;
  const float u = (rad - p.f_tau_rmin) / p.f_tau_dr;
  if (!(u > 0.0f)) return 0.0f;
  int i;
  float fr = 0.0f;
  if (u >= (float)nr) {
    i = nr;
  } else {
    i = min((int)floorf(u), nr - 1);
    fr = u - (float)i;
  }
  int j0 = 0, j1 = 0;
  float fm = 0.0f;
  if (nm > 1) {
    const float w = (mu + p.f_tau_mu) / p.f_tau_dmu - 0.5f;
    if (w <= 0.0f) {
      j0 = j1 = 0;
    } else if (w >= (float)(nm - 1)) {
      j0 = j1 = nm - 1;
    } else {
      j0 = min((int)floorf(w), nm - 2);
      j1 = j0 + 1;
      fm = w - (float)j0;
    }
  }
  const float v = (phi + 3.14159265f) / p.f_tau_dphi - 0.5f;
  const float kf = floorf(v);
  const float fp = v - kf;
  const int k0 = (((int)kf % np) + np) % np, k1 = (k0 + 1) % np;
  const int cols[4] = {j0 * np + k0, j0 * np + k1, j1 * np + k0, j1 * np + k1};
  const float w4[4] = {(1.0f - fm) * (1.0f - fp), (1.0f - fm) * fp, fm * (1.0f - fp), fm * fp};
  const double* Ti = T + (long long)i * ncol;
  float tau = 0.0f;
  for (int c = 0; c < 4; ++c) {
    const float t0 = (float)__ldg(&Ti[cols[c]]);
    const float tc = i >= nr ? t0 : t0 + fr * ((float)__ldg(&Ti[ncol + cols[c]]) - t0);
    tau += w4[c] * tc;
  }
  return tau;
}

// The taper xi^2 (3 - 2 xi), xi = min(max(t / t_beta, 0), 1); 1 without a time scale.
__device__ __forceinline__ double rad_taper(const InstDev& p, double t) {
  if (!(p.t_beta > 0.0)) return 1.0;
  double xi = t / p.t_beta;
  xi = xi < 0.0 ? 0.0 : (xi > 1.0 ? 1.0 : xi);
  return xi * xi * (3.0 - 2.0 * xi);
}

// Records a particle's deposit (its cell, -1 for none, and kappa(s) M); returns the bits of
// kappa M (0: none) for the instance maximum.
__device__ __forceinline__ unsigned long long deposit_note(const InstDev& p, long long i, int cell, double s,
                                                           double M, int* __restrict__ ci,
                                                           double* __restrict__ q) {
  ci[i] = cell;
  if (cell < 0) return 0ull;
  const double v = p.kappa0 * (p.rad_s0 / s) * M;
  q[i] = v;
  return (unsigned long long)__double_as_longlong(v);
}

// The instance maximum of the deposits' bits (positive doubles order as integers).  Every
// thread of the 256-thread block calls it: a block inside one instance reduces over warps
// and shared memory to one atomicMax; a block across an instance boundary takes one per lane.
__device__ __forceinline__ void block_max(long long N, int n_inst, const long long* __restrict__ off, int b,
                                          unsigned long long v, unsigned long long* __restrict__ qmax) {
  __shared__ unsigned long long sm[8];
  const long long i0 = (long long)blockIdx.x * blockDim.x;
  const int b_lo = inst_of(off, n_inst, i0);
  const int b_hi = inst_of(off, n_inst, min(N - 1, i0 + (long long)blockDim.x - 1));
  if (b_lo != b_hi) {
    if (v) atomicMax(&qmax[b], v);
    return;
  }
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0ull;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, sm[w]);
    if (m) atomicMax(&qmax[b_lo], m);
  }
}

// ---------------------------------------------------------------- kernels
// First half drift (FP64: spherical coordinates as the plain step; mixed: rotations of the
// FP64 position) of the instances with radiation forces; the midpoint to mid and, with a
// grid, the deposit's cell and kappa M.  Every other particle gets ci = -1.
template <bool kMixed>
__global__ void __launch_bounds__(256) k_rad_drift(long long N, int n_inst, const long long* __restrict__ off,
                                                   const InstDev* __restrict__ P, const StateDev* __restrict__ st,
                                                   double dt_in, const double* __restrict__ x,
                                                   const double* __restrict__ y, const double* __restrict__ z,
                                                   const double* __restrict__ vr, const double* __restrict__ lth,
                                                   const double* __restrict__ lph, const double* __restrict__ s,
                                                   const double* __restrict__ M, double* __restrict__ mid,
                                                   int* __restrict__ ci, double* __restrict__ q,
                                                   unsigned long long* __restrict__ qmax) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = inst_of(off, n_inst, min(i, N - 1));
  const InstDev& p = P[b];
  unsigned long long v = 0ull;
  if (i < N && !(p.rad && p.geometry == GD_GEOM_DISK)) ci[i] = -1;
  if (i < N && p.rad && p.geometry == GD_GEOM_DISK) {
    const double dt = dt_in < 0.0 ? st[p.unit0].dt_exe : dt_in;
    const double h = 0.5 * dt;
    double X = x[i], Y = y[i], Zc = z[i];
    const double VR = vr[i], LT = lth[i], LP = lph[i];
    int cell = -1;
    if (kMixed) {
      drift_f(h, X, Y, Zc, VR, LT, LP, true);
      mid[i] = X;
      mid[N + i] = Y;
      mid[2 * N + i] = Zc;
      if (p.tau_on) cell = tau_cell_mixed(p, X, Y, Zc);
    } else {
      double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y)), __dmul_rn(Zc, Zc)));
      double th = acos(Zc / r);
      double ph = atan2(Y, X);
      const double sth = sin(th);
      ph = __dadd_rn(ph, __ddiv_rn(__dmul_rn(h, LP), __dmul_rn(__dmul_rn(__dmul_rn(r, r), sth), sth)));
      th = __dadd_rn(th, __ddiv_rn(__dmul_rn(h, LT), __dmul_rn(r, r)));
      r = __dadd_rn(r, __dmul_rn(h, VR));
      mid[i] = r;
      mid[N + i] = th;
      mid[2 * N + i] = ph;
      if (p.tau_on) {
        const double rad = p.tau_geom == GD_TAU_2D ? __dmul_rn(r, sin(th)) : r;
        const double mu = p.tau_geom == GD_TAU_2D ? 0.0 : cos(th);
        cell = tau_cell64(p, rad, mu, fold_phi(ph));
      }
    }
    v = deposit_note(p, i, cell, s[i], M[i], ci, q);
  }
  block_max(N, n_inst, off, b, v, qmax);
}

// Cells of the particles at their current positions (gd_optical_depth), FP64 coordinates.
__global__ void __launch_bounds__(256) k_tau_bin(long long N, int n_inst, const long long* __restrict__ off,
                                                 const InstDev* __restrict__ P, const double* __restrict__ x,
                                                 const double* __restrict__ y, const double* __restrict__ z,
                                                 const double* __restrict__ s, const double* __restrict__ M,
                                                 int* __restrict__ ci, double* __restrict__ q,
                                                 unsigned long long* __restrict__ qmax) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = inst_of(off, n_inst, min(i, N - 1));
  const InstDev& p = P[b];
  unsigned long long v = 0ull;
  if (i < N) {
    int cell = -1;
    if (p.tau_on) {
      const double X = x[i], Y = y[i], Zc = z[i];
      const double R2 = __dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y));
      if (p.tau_geom == GD_TAU_2D) {
        cell = tau_cell64(p, __dsqrt_rn(R2), 0.0, atan2(Y, X));
      } else {
        const double r = __dsqrt_rn(__dadd_rn(R2, __dmul_rn(Zc, Zc)));
        cell = tau_cell64(p, r, __ddiv_rn(Zc, r), atan2(Y, X));
      }
    }
    v = deposit_note(p, i, cell, s[i], M[i], ci, q);
  }
  block_max(N, n_inst, off, b, v, qmax);
}

// Each particle's kappa M into its cell: 128-bit fixed point, q 2^(60 - e) rounded to an
// integer below 2^60 (e: the exponent of the instance's largest q), low word by atomicAdd,
// its wrap-around (the carry) counted in the high word.
__global__ void __launch_bounds__(256) k_tau_deposit(long long N, int n_inst, const long long* __restrict__ off,
                                                     const InstDev* __restrict__ P, const int* __restrict__ ci,
                                                     const double* __restrict__ q,
                                                     const unsigned long long* __restrict__ qmax,
                                                     unsigned long long* __restrict__ acc) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int c = ci[i];
  if (c < 0) return;
  const int b = inst_of(off, n_inst, i);
  int e;
  frexp(__longlong_as_double((long long)qmax[b]), &e);
  const unsigned long long v = __double2ull_rn(ldexp(q[i], 60 - e));
  unsigned long long* a = acc + 2 * (P[b].tau_cell0 + c);
  const unsigned long long old = atomicAdd(&a[0], v);
  if (old + v < old) atomicAdd(&a[1], 1ull);
}

// One thread per cell: its increment (kappa rho_d)_i dr = (sum_i / V_i) dr into the slot of
// its outer face, with the oracle's correctly rounded steps for the volume; the cell's
// accumulators cleared for the next use.
__global__ void __launch_bounds__(256) k_tau_cells(long long n_cells, int n_inst,
                                                   const long long* __restrict__ cell_off,
                                                   const InstDev* __restrict__ P,
                                                   const unsigned long long* __restrict__ qmax,
                                                   unsigned long long* __restrict__ acc, double* __restrict__ T) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_cells) return;
  const int b = inst_of(cell_off, n_inst, g);
  const InstDev& p = P[b];
  const long long l = g - cell_off[b];
  const int ncol = p.tau_nm * p.tau_np;
  const int i = (int)(l / ncol), col = (int)(l % ncol);
  int e;
  frexp(__longlong_as_double((long long)qmax[b]), &e);
  unsigned long long* a = acc + 2 * (p.tau_cell0 + l);
  const unsigned long long lo = a[0], hi = a[1];
  a[0] = 0ull;
  a[1] = 0ull;
  const double A = ldexp(__dadd_rn(__dmul_rn((double)hi, 18446744073709551616.0), (double)lo), e - 60);
  const double dr = __ddiv_rn(__dsub_rn(p.tau_rmax, p.tau_rmin), (double)p.tau_nr);
  const double dphi = __ddiv_rn(kTwoPi, (double)p.tau_np);
  const double r_lo = __dadd_rn(p.tau_rmin, __dmul_rn((double)i, dr));
  const double r_hi = __dadd_rn(p.tau_rmin, __dmul_rn((double)(i + 1), dr));
  double V;
  if (p.tau_geom == GD_TAU_2D) {
    const Gas gs = gas_RZ(p, __dadd_rn(p.tau_rmin, __dmul_rn((double)i + 0.5, dr)), 0.0);
    V = __dmul_rn(__dmul_rn(__ddiv_rn(__dsub_rn(__dmul_rn(r_hi, r_hi), __dmul_rn(r_lo, r_lo)), 2.0), dphi),
                  __dmul_rn(sqrt(2.0 * kPi), gs.H));
  } else {
    const double dmu = __ddiv_rn(2.0 * p.tau_mu, (double)p.tau_nm);
    const double c3 = __dsub_rn(__dmul_rn(__dmul_rn(r_hi, r_hi), r_hi), __dmul_rn(__dmul_rn(r_lo, r_lo), r_lo));
    V = __dmul_rn(__dmul_rn(__ddiv_rn(c3, 3.0), dmu), dphi);
  }
  T[p.tau_face0 + (long long)(i + 1) * ncol + col] = __dmul_rn(__ddiv_rn(A, V), dr);
}

// One thread per column: T_0 = 0, T_{i+1} = T_i + increment_i, in the oracle's order; the
// increments are read eight at a time ahead of their adds.
__global__ void __launch_bounds__(128) k_tau_columns(long long n_cols, int n_inst,
                                                     const long long* __restrict__ col_off,
                                                     const InstDev* __restrict__ P, double* __restrict__ T) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_cols) return;
  const int b = inst_of(col_off, n_inst, g);
  const InstDev& p = P[b];
  const int col = (int)(g - col_off[b]);
  const int nr = p.tau_nr, ncol = p.tau_nm * p.tau_np;
  double* Tc = T + p.tau_face0 + col;
  Tc[0] = 0.0;
  double sum = 0.0;
  for (int i0 = 1; i0 <= nr; i0 += 8) {
    double inc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) inc[u] = i0 + u <= nr ? Tc[(long long)(i0 + u) * ncol] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (i0 + u <= nr) {
        sum = __dadd_rn(sum, inc[u]);
        Tc[(long long)(i0 + u) * ncol] = sum;
      }
    }
  }
}

// The kick at the midpoint with the radiation force and the P-R damping, and the second
// half drift (Sect. 2.3.2-2.3.3).
template <bool kMixed>
__global__ void __launch_bounds__(256) k_rad_kick(long long N, int n_inst, const long long* __restrict__ off,
                                                  const InstDev* __restrict__ P, const StateDev* __restrict__ st,
                                                  double dt_in, const double* __restrict__ mid,
                                                  const double* __restrict__ T, const double* __restrict__ trad,
                                                  double* x, double* y, double* z, double* vr, double* lth,
                                                  double* lph, const double* __restrict__ s) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int b = inst_of(off, n_inst, i);
  const InstDev& p = P[b];
  if (!p.rad || p.geometry != GD_GEOM_DISK) return;
  const double dt = dt_in < 0.0 ? st[p.unit0].dt_exe : dt_in;
  const double h = 0.5 * dt;
  const double taper = rad_taper(p, trad[b] + h);
  const double* Tb = T + p.tau_face0;
  double VR = vr[i], LT = lth[i], LP = lph[i];
  const double si = s[i];
  if (kMixed) {
    double X = mid[i], Y = mid[N + i], Zc = mid[2 * N + i];
    const double R2 = X * X + Y * Y, R = sqrt(R2), r = sqrt(R2 + Zc * Zc);
    const double ir = 1.0 / r, sth = R * ir, cth = Zc * ir, ir2 = ir * ir;
    float tau = 0.0f;
    if (p.tau_on)
      tau = tau_interp32(p, Tb, p.tau_geom == GD_TAU_2D ? (float)R : (float)r,
                         p.tau_geom == GD_TAU_2D ? 0.0f : (float)cth, atan2f((float)Y, (float)X));
    const float be = (float)taper * (p.f_beta0 * (p.f_rad_s0 / (float)si)) * expf(-tau);
    const double fr = (-p.GM * (1.0 - (double)be) + LT * LT * ir + LP * LP * r / R2) * ir2;
    const double fth = LP * LP * cth * ir2 / (sth * sth * sth);
    // the gas disk at the midpoint in FP32, as the plain mixed step
    const float Rf = (float)R, Zf = (float)Zc;
    const float Om = sqrtf(p.f_GM / Rf) / Rf;
    const float xr = Rf / p.f_r0;
    const float cs = sqrtf((float)(kKB / (kMu * kMH)) * (p.f_T0 * powf(xr, p.f_q)));
    const float hg = cs / Om / Rf;
    const float rf = sqrtf(Rf * Rf + Zf * Zf);
    const float omr = Zf * Zf / (rf * (rf + Rf));
    const float eta = -0.5f * ((p.f_p + 0.5f * p.f_q - 1.5f) * hg * hg + p.f_q * omr);
    const float gst = 3.14159265f * p.f_rho_s / (4.0f * p.f_sigma0 * powf(xr, p.f_p)) * expf(omr / (hg * hg));
    const float gam = Om / (gst * (float)si);
    const float gpr = p.rad_pr ? be * (p.f_GM * (float)ir2) * (float)(1.0 / kCLight) : 0.0f;
    const float g_r = gam + 2.0f * gpr, g_t = gam + gpr;
    const float k_r = g_r > 0.0f ? -expm1f(-(float)dt * g_r) / g_r : (float)dt;
    const float k_t = g_t > 0.0f ? -expm1f(-(float)dt * g_t) / g_t : (float)dt;
    const double ygph = sqrt(1.0 - 2.0 * (double)eta) * sqrt(p.GM * R);
    VR = VR - (double)(k_r * g_r) * VR + (double)k_r * fr;
    LT = LT - (double)(k_t * g_t) * LT + (double)k_t * fth;
    LP = LP + (double)(k_t * gam) * (ygph - LP) - (double)(k_t * gpr) * LP;
    drift_f(h, X, Y, Zc, VR, LT, LP, false);
    x[i] = X;
    y[i] = Y;
    z[i] = Zc;
  } else {
    double r = mid[i], th = mid[N + i], ph = mid[2 * N + i];
    double sth = sin(th);
    const double cth = cos(th);
    double tau = 0.0;
    if (p.tau_on)
      tau = tau_interp64(p, Tb, p.tau_geom == GD_TAU_2D ? r * sth : r, p.tau_geom == GD_TAU_2D ? 0.0 : cth,
                         fold_phi(ph));
    const double be = taper * (p.beta0 * (p.rad_s0 / si)) * exp(-tau);
    const double fr = -(1.0 - be) * p.GM / (r * r) + LT * LT / (r * r * r) + LP * LP / (r * r * r * sth * sth);
    const double fth = LP * LP * cth / (r * r * sth * sth * sth);
    const double gpr = p.rad_pr ? be * p.GM / (kCLight * r * r) : 0.0;
    const Gas g = gas_RZ(p, r * sth, r * cth);
    const double gam = 1.0 / (g.gst * si / g.Om);
    const double ygph = sqrt(1.0 - 2.0 * g.eta) * g.Om * g.R * g.R;
    const double g_r = gam + 2.0 * gpr, g_t = gam + gpr;
    const double k_r = g_r > 0.0 ? -expm1(-dt * g_r) / g_r : dt;
    const double k_t = g_t > 0.0 ? -expm1(-dt * g_t) / g_t : dt;
    VR = VR + k_r * (fr - g_r * VR);
    LT = LT + k_t * (fth - g_t * LT);
    LP = LP + k_t * (gam * ygph - g_t * LP);
    r = r + h * VR;
    th = th + h * LT / (r * r);
    sth = sin(th);
    ph = ph + h * LP / (r * r * sth * sth);
    x[i] = r * sth * cos(ph);
    y[i] = r * sth * sin(ph);
    z[i] = r * cos(th);
  }
  vr[i] = VR;
  lth[i] = LT;
  lph[i] = LP;
}

// Each instance's taper clock forward by its dt.
__global__ void k_rad_clock(int n_inst, const InstDev* __restrict__ P, const StateDev* __restrict__ st,
                            double dt_in, double* __restrict__ trad) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_inst) return;
  trad[b] += dt_in < 0.0 ? st[P[b].unit0].dt_exe : dt_in;
}

// tau at each particle's current position (FP64), 0 for instances without a grid.
__global__ void __launch_bounds__(256) k_tau_eval(long long N, int n_inst, const long long* __restrict__ off,
                                                  const InstDev* __restrict__ P, const double* __restrict__ T,
                                                  const double* __restrict__ x, const double* __restrict__ y,
                                                  const double* __restrict__ z, double* __restrict__ tau_out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int b = inst_of(off, n_inst, i);
  const InstDev& p = P[b];
  double tau = 0.0;
  if (p.tau_on) {
    const double X = x[i], Y = y[i], Zc = z[i];
    const double R2 = __dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y));
    if (p.tau_geom == GD_TAU_2D) {
      tau = tau_interp64(p, T + p.tau_face0, __dsqrt_rn(R2), 0.0, atan2(Y, X));
    } else {
      const double r = __dsqrt_rn(__dadd_rn(R2, __dmul_rn(Zc, Zc)));
      tau = tau_interp64(p, T + p.tau_face0, r, __ddiv_rn(Zc, r), atan2(Y, X));
    }
  }
  tau_out[i] = tau;
}

// The faces in the interface layout, [column][face] per instance, instances in order.
__global__ void k_tau_grid_out(long long n_faces, int n_inst, const InstDev* __restrict__ P,
                               const long long* __restrict__ face_off, const double* __restrict__ T,
                               double* __restrict__ out) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_faces) return;
  const int b = inst_of(face_off, n_inst, g);
  const InstDev& p = P[b];
  const long long l = g - face_off[b];
  const int ncol = p.tau_nm * p.tau_np;
  const long long col = l / (p.tau_nr + 1), f = l % (p.tau_nr + 1);
  out[g] = T[p.tau_face0 + f * ncol + col];
}

// ---------------------------------------------------------------- launchers
static cudaError_t tau_sums(gd_ctx* c) {
  const int blocks = (int)((c->N + 255) / 256);
  k_tau_deposit<<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_tau_ci, c->d_tau_q,
                                               c->d_tau_max, c->d_tau_acc);
  k_tau_cells<<<(int)((c->tau_cells + 255) / 256), 256, 0, c->stream>>>(
      c->tau_cells, c->n_inst, c->d_cell_off, c->d_inst, c->d_tau_max, c->d_tau_acc, c->d_tau_T);
  k_tau_columns<<<(int)((c->tau_cols + 127) / 128), 128, 0, c->stream>>>(c->tau_cols, c->n_inst, c->d_col_off,
                                                                        c->d_inst, c->d_tau_T);
  c->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_push_rad(gd_ctx* c, double dt) {
  time_begin(c, 5);
  const int blocks = (int)((c->N + 255) / 256);
  cudaError_t e = cudaSuccess;
  if (c->any_tau) e = cudaMemsetAsync(c->d_tau_max, 0, sizeof(unsigned long long) * c->n_inst, c->stream);
  if (e != cudaSuccess) {
    time_end(c);
    return e;
  }
  if (c->precision == GD_MIXED)
    k_rad_drift<true><<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_state, dt, c->x,
                                                     c->y, c->z, c->vr, c->lth, c->lph, c->s, c->M, c->d_mid,
                                                     c->d_tau_ci, c->d_tau_q, c->d_tau_max);
  else
    k_rad_drift<false><<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_state, dt, c->x,
                                                      c->y, c->z, c->vr, c->lth, c->lph, c->s, c->M, c->d_mid,
                                                      c->d_tau_ci, c->d_tau_q, c->d_tau_max);
  c->launches += 1;
  if (c->any_tau) {
    e = tau_sums(c);
    if (e != cudaSuccess) {
      time_end(c);
      return e;
    }
  }
  if (c->precision == GD_MIXED)
    k_rad_kick<true><<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_state, dt, c->d_mid,
                                                    c->d_tau_T, c->d_trad, c->x, c->y, c->z, c->vr, c->lth,
                                                    c->lph, c->s);
  else
    k_rad_kick<false><<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_state, dt,
                                                     c->d_mid, c->d_tau_T, c->d_trad, c->x, c->y, c->z, c->vr,
                                                     c->lth, c->lph, c->s);
  k_rad_clock<<<(c->n_inst + 127) / 128, 128, 0, c->stream>>>(c->n_inst, c->d_inst, c->d_state, dt, c->d_trad);
  c->launches += 2;
  time_end(c);
  c->moved = true;
  return cudaGetLastError();
}

cudaError_t launch_optical_depth(gd_ctx* c, double* tau_out, double* grid_out) {
  const int blocks = (int)((c->N + 255) / 256);
  cudaError_t e = cudaMemsetAsync(c->d_tau_max, 0, sizeof(unsigned long long) * c->n_inst, c->stream);
  if (e != cudaSuccess) return e;
  k_tau_bin<<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->x, c->y, c->z, c->s, c->M,
                                           c->d_tau_ci, c->d_tau_q, c->d_tau_max);
  c->launches += 1;
  e = tau_sums(c);
  if (e != cudaSuccess) return e;
  if (tau_out) {
    k_tau_eval<<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_tau_T, c->x, c->y, c->z,
                                              tau_out);
    c->launches += 1;
  }
  if (grid_out && c->tau_out_faces > 0) {
    k_tau_grid_out<<<(int)((c->tau_out_faces + 255) / 256), 256, 0, c->stream>>>(
        c->tau_out_faces, c->n_inst, c->d_inst, c->d_face_off, c->d_tau_T, grid_out);
    c->launches += 1;
  }
  return cudaGetLastError();
}

}  // namespace gd
