// k_misc.cu -- staggered semi-analytic push (Sect. 2.3.3), per-instance reductions for
// gd_stats, and conversion of rank-space results to the caller's order.
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
  if (p.geometry != GD_GEOM_DISK) return;
  double dt = dt_in < 0.0 ? st[b].dt_exe : dt_in;
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
  time_begin(c, 5);
  int blocks = (int)((c->N + 255) / 256);
  k_push<<<blocks, 256, 0, c->stream>>>(c->N, c->n_inst, c->d_off, c->d_inst, c->d_state, dt, c->x, c->y,
                                         c->z, c->vr, c->lth, c->lph, c->s);
  time_end(c);
  c->launches += 1;
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
