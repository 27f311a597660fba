/*
 * gdo.c -- plain, serial, FP64 CPU oracle of the GameDev collision step.
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or run it.  It is
 * written from the paper ("GameDev: GPU-accelerated model for dust
 * evolution", Sect. 2 and Appendix A) and shares nothing with the CUDA
 * library.  Build with -ffp-contract=off so that every expression is
 * evaluated as written.
 *
 * Parity pins (tests/test_oracle_*.py): Philox known-answer vectors,
 * exhaustive K-NN enumeration with lattice ties, the monodisperse closed
 * form of the rate, quadrature of the fragment moments, a hand-computed
 * two-bin interval, the constant-kernel Smoluchowski mean mass, exact
 * conservation of the represented mass, and the drag-free Kepler orbit.
 * The turbulent relative speed is "parity unpinned" against GameDev itself:
 * the paper cites Ormel & Cuzzi (2007) without printing its branches; only
 * its limits are pinned.
 */
#include "gdo.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Physical constants, cgs (reading: the paper gives no values). */
#define GDO_PI    3.14159265358979323846
#define GDO_KB    1.380649e-16      /* Boltzmann constant [erg/K] */
#define GDO_MH    1.6735575e-24     /* hydrogen mass [g] */
#define GDO_MU    2.34              /* mean molecular weight */
#define GDO_G     6.674e-8          /* gravitational constant [cgs] */
#define GDO_SIGH2 2e-15             /* H2 collision cross-section [cm^2] */

/* ------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw (SC'11), "Parallel random
 * numbers: as easy as 1, 2, 3".  Round: two 32x32->64 products of counter
 * words 0 and 2 with the multipliers; the new counter is
 * (hi1^c1^k0, lo1, hi0^c3^k1, lo0); the key is bumped by the Weyl
 * constants before every round after the first.  (Reading: the paper does
 * not name its generator; the draws are keyed by (seed, particle, interval,
 * draw) as the method needs.) */
void gdo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on the open interval (0,1) from two 32-bit words: 26 bits of each
 * make an integer k < 2^52, and u = (k + 1/2) 2^-52 is exact in FP64. */
double gdo_u01(uint32_t a, uint32_t b) {
  uint64_t k = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
  return ((double)k + 0.5) * 0x1p-52;
}

/* ------------------------------------------------------------------ */
/* Analytic gas disk, Sect. 2.2: Sigma_g = Sigma_0 (R/R_0)^p,
 * T = T_0 (R/R_0)^q (so h_g ~ R^((q+1)/2)), c_s = sqrt(k_B T/(mu m_H)),
 * Omega_K = sqrt(G M_star/R^3), H_g = c_s/Omega_K, h_g = H_g/R,
 * rho_g = Sigma_g/(sqrt(2 pi) H_g) exp(-(1-R/r)/h_g^2),
 * eta = -[(p + q/2 - 3/2) h_g^2 + q (1 - R/r)]/2.
 * Epstein Stokes number (Sect. 2.3.1): St = (pi rho_o s / (4 Sigma_g))
 * exp((1-R/r)/h_g^2); gst is St per unit diameter.  Molecular viscosity and
 * the Reynolds number Re = alpha c_s H_g / nu_mol with
 * nu_mol = v_th lambda_mfp / 2, v_th = sqrt(8/pi) c_s,
 * lambda_mfp = mu m_H/(rho_g sigma_H2) (reading: needed by the turbulent
 * relative speed, Sect. 2.5.2). */
static void gas_RZ(const gdo_params* P, double R, double Z, gdo_gas* g) {
  double r = sqrt(R * R + Z * Z);
  double Om = sqrt(GDO_G * P->M_star / (R * R * R));
  double T = P->T0 * pow(R / P->r0, P->q);
  double cs = sqrt(GDO_KB * T / (GDO_MU * GDO_MH));
  double H = cs / Om;
  double h = H / R;
  double Sigma = P->sigma0 * pow(R / P->r0, P->p);
  double vert = (1.0 - R / r) / (h * h);
  double rho = Sigma / (sqrt(2.0 * GDO_PI) * H) * exp(-vert);
  double eta = -0.5 * ((P->p + 0.5 * P->q - 1.5) * h * h + P->q * (1.0 - R / r));
  double vth = sqrt(8.0 / GDO_PI) * cs;
  double lmfp = GDO_MU * GDO_MH / (rho * GDO_SIGH2);
  double numol = 0.5 * vth * lmfp;
  g->R = R; g->Z = Z; g->r = r; g->Om = Om; g->T = T; g->cs = cs; g->H = H; g->h = h;
  g->Sigma = Sigma; g->rho_g = rho; g->eta = eta;
  g->Re = P->alpha * cs * H / numol;
  g->gst = GDO_PI * P->rho_s / (4.0 * Sigma) * exp(vert);
}

/* Position to (R, Z): a local patch sits at R = R_0 + x (reading: x is the
 * radial offset, y the azimuthal one), a global disk uses cylindrical
 * R = sqrt(x^2 + y^2) (Sect. 2.1). */
void gdo_gas_at(const gdo_params* P, double x, double y, double z, gdo_gas* g) {
  double R = (P->geometry == GDO_PATCH) ? P->r0 + x : sqrt(x * x + y * y);
  /* vertically integrated models (radial-azimuthal, radial) see the midplane */
  if (P->model == GDO_MODEL_RPHI || P->model == GDO_MODEL_R) z = 0.0;
  gas_RZ(P, R, z, g);
}

/* Coordinates of the neighbour search, Sect. 2.5.1: 3D positions; the
 * meridional plane (R, Z) of a 2D radial-polar model; the midplane (x, y) of a
 * vertically integrated model; R alone in a 1D radial model. */
static void model_coords(const gdo_params* P, double x, double y, double z, double* X, double* Y,
                         double* Z) {
  switch (P->model) {
    case GDO_MODEL_RZ: *X = sqrt(x * x + y * y); *Y = z; *Z = 0.0; break;
    case GDO_MODEL_RPHI: *X = x; *Y = y; *Z = 0.0; break;
    case GDO_MODEL_R: *X = sqrt(x * x + y * y); *Y = 0.0; *Z = 0.0; break;
    default: *X = x; *Y = y; *Z = z; break;
  }
}

/* m = pi rho_o s^3 / 6, Sect. 2 (s is the diameter). */
double gdo_grain_mass(const gdo_params* P, double s) {
  return GDO_PI * P->rho_s * s * s * s / 6.0;
}

/* ------------------------------------------------------------------ */
/* K nearest neighbours of particle i by brute force (Sect. 2.5.1): every
 * other particle j is ranked by (d^2, j) with d^2 = (dx dx + dy dy) + dz dz in
 * the model's coordinates (model_coords), minimum image in the periodic x and y
 * of a patch.  Reading: the particle
 * itself always takes slot 0 (it is included at zero distance), the K-1
 * nearest others follow in ascending index order, and no maximum search
 * scale applies.  *d receives the distance to the farthest retained
 * neighbour. */
int gdo_knn_one(const gdo_params* P, int64_t n, const double* x, const double* y,
                const double* z, int64_t i, int32_t* nbr, double* d) {
  int L = P->K - 1;
  if (L < 0 || n < P->K) return -1;
  double* bd = (double*)malloc(sizeof(double) * (L > 0 ? L : 1));
  int64_t* bj = (int64_t*)malloc(sizeof(int64_t) * (L > 0 ? L : 1));
  int cnt = 0;
  double xi, yi, zi;
  model_coords(P, x[i], y[i], z[i], &xi, &yi, &zi);
  for (int64_t j = 0; j < n; ++j) {
    if (j == i) continue;
    double xj, yj, zj;
    model_coords(P, x[j], y[j], z[j], &xj, &yj, &zj);
    double dx = xj - xi;
    double dy = yj - yi;
    double dz = zj - zi;
    if (P->geometry == GDO_PATCH) {
      if (dx > 0.5 * P->box_x) dx -= P->box_x;
      else if (dx < -0.5 * P->box_x) dx += P->box_x;
      if (dy > 0.5 * P->box_y) dy -= P->box_y;
      else if (dy < -0.5 * P->box_y) dy += P->box_y;
    }
    double d2 = (dx * dx + dy * dy) + dz * dz;
    if (L == 0) continue;
    if (cnt == L && !(d2 < bd[L - 1] || (d2 == bd[L - 1] && j < bj[L - 1]))) continue;
    int pos = (cnt < L) ? cnt : L - 1;
    while (pos > 0 && (d2 < bd[pos - 1] || (d2 == bd[pos - 1] && j < bj[pos - 1]))) {
      bd[pos] = bd[pos - 1];
      bj[pos] = bj[pos - 1];
      --pos;
    }
    bd[pos] = d2;
    bj[pos] = j;
    if (cnt < L) ++cnt;
  }
  *d = (L > 0) ? sqrt(bd[L - 1]) : 0.0;
  /* ascending index order after the particle itself */
  for (int a = 1; a < L; ++a) {
    int64_t v = bj[a];
    int b = a;
    while (b > 0 && bj[b - 1] > v) { bj[b] = bj[b - 1]; --b; }
    bj[b] = v;
  }
  nbr[0] = (int32_t)i;
  for (int a = 0; a < L; ++a) nbr[1 + a] = (int32_t)bj[a];
  free(bd);
  free(bj);
  return 0;
}

/* Sampling measure, Sect. 2.5.1: V = 4 pi d^3 / 3; near a domain boundary
 * the part outside is removed treating the boundary as locally flat.
 * Reading: for the global disk each radial edge at distance 0 < h < d
 * removes the spherical cap pi (d-h)^2 (2d+h) / 3; patches are periodic in
 * x, y and unbounded in z, so they need no correction.  Reduced models: the
 * sampled area (a disk of radius d in the meridional plane or the midplane, an
 * annulus in 1D) times 2 pi R (2D radial-polar: a toroidal volume) or times
 * the vertical length sqrt(2 pi (H_i^2 + H_j^2)) of the Gaussian average
 * (vertically integrated models), so that lambda_ij = N_j K_ij / V_i keeps
 * its form.  R: the particle's cylindrical radius. */
double gdo_volume(const gdo_params* P, double d, double R) {
  if (P->model == GDO_MODEL_3D) {
    double V = 4.0 * GDO_PI * d * d * d / 3.0;
    if (P->geometry == GDO_DISK) {
      double h = R - P->R_in;
      if (h > 0.0 && h < d) V -= GDO_PI * (d - h) * (d - h) * (2.0 * d + h) / 3.0;
      h = P->R_out - R;
      if (h > 0.0 && h < d) V -= GDO_PI * (d - h) * (d - h) * (2.0 * d + h) / 3.0;
    }
    return V;
  }
  /* reduced models (Sect. 2.5.1) */
  double A;
  if (P->model == GDO_MODEL_R) {
    /* the annulus [R - d, R + d], clipped at the disk's edges */
    double lo = R - d > P->R_in ? R - d : P->R_in;
    double hi = R + d < P->R_out ? R + d : P->R_out;
    A = GDO_PI * (hi * hi - lo * lo);
  } else {
    /* the disk of radius d; a radial edge at distance 0 < h < d, taken as a
     * straight line, removes the circular segment d^2 acos(h/d) - h sqrt(d^2 - h^2) */
    A = GDO_PI * d * d;
    if (P->geometry == GDO_DISK) {
      double h = R - P->R_in;
      if (h > 0.0 && h < d) A -= d * d * acos(h / d) - h * sqrt(d * d - h * h);
      h = P->R_out - R;
      if (h > 0.0 && h < d) A -= d * d * acos(h / d) - h * sqrt(d * d - h * h);
    }
  }
  if (P->model == GDO_MODEL_RZ) return A * 2.0 * GDO_PI * R;   /* toroidal volume */
  /* vertically integrated: lambda_ij = N_j K_ij / (A sqrt(2 pi (H_i^2 + H_j^2)));
   * reading: H_i = H_j = H_g(R_i), at i's position like every pair quantity */
  gdo_gas g;
  gas_RZ(P, R, 0.0, &g);
  return A * sqrt(2.0 * GDO_PI * (g.H * g.H + g.H * g.H));
}

/* ------------------------------------------------------------------ */
/* Fragment moments, Sect. 2.5.3: <J> and <J^2> of J = |ln(s'/s_i)| over
 * U ~ U(0,1) with s' = [sqrt(s_min) + U (sqrt(s_i) - sqrt(s_min))]^2.
 * With a = sqrt(s_min/s_i), the integrals give
 *   <J>   = 2 (1 - a + a ln a) / (1 - a),
 *   <J^2> = 4 (2 - a ln^2 a + 2 a ln a - 2 a) / (1 - a).
 * Near a = 1 the closed forms cancel; for dd = 1 - a < 1e-3 the Taylor
 * series of the same integrals is used (coefficients 2/(k(k+1)) for <J>). */
void gdo_frag_moments(double s_i, double s_min, double* j1, double* j2) {
  double a = sqrt(s_min / s_i);
  if (!(a < 1.0)) { *j1 = 0.0; *j2 = 0.0; return; }
  double dd = 1.0 - a;
  if (dd < 1e-3) {
    *j1 = dd * (1.0 + dd * (1.0 / 3.0 + dd * (1.0 / 6.0 + dd * (1.0 / 10.0 +
          dd * (1.0 / 15.0 + dd * (1.0 / 21.0))))));
    *j2 = dd * dd * (4.0 / 3.0 + dd * (1.0 + dd * (11.0 / 15.0 + dd * (5.0 / 9.0 +
          dd * (137.0 / 315.0 + dd * (7.0 / 20.0))))));
    return;
  }
  double la = log(a);
  *j1 = 2.0 * (1.0 - a + a * la) / (1.0 - a);
  *j2 = 4.0 * (2.0 - a * la * la + 2.0 * a * la - 2.0 * a) / (1.0 - a);
}

/* Turbulent relative speed squared.  The paper adopts Ormel & Cuzzi (2007)
 * (Sect. 2.5.2) without printing it.  Reading (parity unpinned against
 * GameDev): the three closed-form regimes of Ormel & Cuzzi, with stopping
 * times in units of the large-eddy turnover time 1/Omega (that is, St),
 * t_eta = Re^-1/2, St1 >= St2, eps = St2/St1, V_g^2 = (3/2) alpha c_s^2:
 *   St1 < Re^-1/2 :  V_g^2 (St1-St2)/(St1+St2) (St1^2/(St1+t_eta) - St2^2/(St2+t_eta))
 *   St1 < 1       :  V_g^2 St1 (2 y_a - (1+eps) + 2/(1+eps) (1/(1+y_a) + eps^3/(y_a+eps))), y_a = 1.6
 *   St1 >= 1      :  V_g^2 (1/(1+St1) + 1/(1+St2)). */
double gdo_turb_dv2(double St_a, double St_b, double Vg2, double Re) {
  double St1 = St_a > St_b ? St_a : St_b;
  double St2 = St_a > St_b ? St_b : St_a;
  double teta = 1.0 / sqrt(Re);
  if (St1 < teta) {
    return Vg2 * (St1 - St2) / (St1 + St2) *
           (St1 * St1 / (St1 + teta) - St2 * St2 / (St2 + teta));
  }
  if (St1 < 1.0) {
    double e = St2 / St1;
    double ya = 1.6;
    return Vg2 * St1 *
           (2.0 * ya - (1.0 + e) + 2.0 / (1.0 + e) * (1.0 / (1.0 + ya) + e * e * e / (ya + e)));
  }
  return Vg2 * (1.0 / (1.0 + St1) + 1.0 / (1.0 + St2));
}

/* One ordered pair (i, j), every quantity at i's position (Sect. 2.5.2):
 *   Delta v^2 = dv_R^2 + dv_Z^2 + dv_phi^2 + dv_B^2 + dv_t^2 with
 *   dv_R   = 2 eta R Omega (St_i/(1+St_i^2) - St_j/(1+St_j^2)),
 *   dv_Z   = Z Omega (min(St_i, 0.5) - min(St_j, 0.5)),
 *   dv_phi = eta R Omega (1/(1+St_i^2) - 1/(1+St_j^2)),
 *   dv_B   = min(c_s, sqrt(8 k_B T/pi (1/m_i + 1/m_j))),
 * the kernel K_ij = pi (s_i+s_j)^2 Delta v / 4 and the rate
 * lambda_ij = N_j K_ij / V_i (Sect. 2.5.1).  In the Appendix A test modes
 * K_ij is 1, (m_i+m_j)/m_0 or m_i m_j/m_0^2 and
 * lambda_ij = (1/t_0)(1/N_K)(m_0/m_j) K_ij (V_i = 1), sticking only.
 * Outcome (Sect. 2.5.2): sticking if Delta v < v_frag, else erosion if
 * psi = m_j/m_i <= 0.1, else fragmentation.  Grouping
 * N_coll = floor(1e-4/psi) for psi <= 1e-6, else 1.  Effective channel
 * rates, in this order (reading: the paper fixes no order):
 *   sticking  : lambda/N_coll                (m' = m_i + N_coll m_j)
 *   erosion   : (1-psi) lambda/N_coll (rem.) (m' = m_i - N_coll m_j),
 *               psi lambda (debris)          (m' = m_j)
 *   fragment  : lambda                       (s' from Eq. frag)
 * and J = |ln(s'/s_i)| = |ln(m'/m_i)|/3 for the deterministic outcomes. */
void gdo_pair(const gdo_params* P, const gdo_gas* g, double s_i, double m_i, double s_j,
              double m_j, double N_j, double V_i, gdo_pair_t* o) {
  memset(o, 0, sizeof(*o));
  double lam;
  int outcome;
  o->psi = m_j / m_i;
  o->ncoll = (o->psi <= 1e-6) ? floor(1e-4 / o->psi) : 1.0;
  if (P->kernel_mode == GDO_PHYSICAL) {
    double St_i = g->gst * s_i;
    double St_j = g->gst * s_j;
    o->dvR = 2.0 * g->eta * g->R * g->Om * (St_i / (1.0 + St_i * St_i) - St_j / (1.0 + St_j * St_j));
    double hi = St_i < 0.5 ? St_i : 0.5;
    double hj = St_j < 0.5 ? St_j : 0.5;
    o->dvZ = g->Z * g->Om * (hi - hj);
    o->dvphi = g->eta * g->R * g->Om * (1.0 / (1.0 + St_i * St_i) - 1.0 / (1.0 + St_j * St_j));
    double vb = sqrt(8.0 * GDO_KB * g->T / GDO_PI * (1.0 / m_i + 1.0 / m_j));
    o->dvB = g->cs < vb ? g->cs : vb;
    double Vg2 = 1.5 * P->alpha * g->cs * g->cs;
    o->dvt = sqrt(gdo_turb_dv2(St_i, St_j, Vg2, g->Re));
    o->dv = sqrt(o->dvR * o->dvR + o->dvZ * o->dvZ + o->dvphi * o->dvphi + o->dvB * o->dvB +
                 o->dvt * o->dvt);
    o->Kij = GDO_PI * (s_i + s_j) * (s_i + s_j) * o->dv / 4.0;
    lam = N_j * o->Kij / V_i;
    outcome = (o->dv < P->v_frag) ? 0 : ((o->psi <= 0.1) ? 1 : 2);
  } else {
    double Kk = 1.0;
    if (P->kernel_mode == GDO_LINEAR) Kk = (m_i + m_j) / P->m0;
    if (P->kernel_mode == GDO_PRODUCT) Kk = m_i * m_j / (P->m0 * P->m0);
    o->Kij = Kk;
    lam = (1.0 / P->t0) * (1.0 / (double)P->K) * (P->m0 / m_j) * Kk;
    outcome = 0;
  }
  o->lam = lam;
  o->outcome = outcome;
  if (outcome == 0) {
    o->c[0] = lam / o->ncoll;
    o->J1[0] = log1p(o->ncoll * o->psi) / 3.0;
    o->J2[0] = o->J1[0] * o->J1[0];
  } else if (outcome == 1) {
    o->c[0] = (1.0 - o->psi) * lam / o->ncoll;
    o->J1[0] = fabs(log1p(-o->ncoll * o->psi) / 3.0);
    o->J2[0] = o->J1[0] * o->J1[0];
    o->c[1] = o->psi * lam;
    o->J1[1] = fabs(log(o->psi) / 3.0);
    o->J2[1] = o->J1[1] * o->J1[1];
  } else {
    o->c[0] = lam;
    gdo_frag_moments(s_i, P->s_min, &o->J1[0], &o->J2[0]);
  }
}

/* ------------------------------------------------------------------ */
/* Controller bins (Sect. 2.5.3 and its footnote).  Reading: fine
 * logarithmic bins of a third of an octave (log10(2)/3 ~ 0.1 dex) with edges
 * at s = 2^e {1/2, 2^(1/3)/2, 2^(2/3)/2}; the bin is found exactly from the
 * binary exponent and mantissa of s, so no rounding of a logarithm can move
 * a particle across an edge.  Fine bin t - GDO_TMIN, clamped to
 * [0, GDO_NFINE). */
int gdo_fine_bin(double s) {
  int e;
  double mant = frexp(s, &e);               /* s = mant 2^e, mant in [1/2, 1) */
  int t = 3 * e + (mant >= 0x1.428a2f98d728bp-1) + (mant >= 0x1.965fea53d6e3dp-1);
  t -= GDO_TMIN;
  if (t < 0) t = 0;
  if (t > GDO_NFINE - 1) t = GDO_NFINE - 1;
  return t;
}

/* Interval choice, Sect. 2.5.3: mass-weighted moments per controller bin
 *   A_b = sum_{i in b} M_i sum_o lambda*_io <J_io> / sum_{i in b} M_i,
 *   B_b likewise with <J_io^2>,
 *   dt_req = min(dt_remain, dt_fn_max, min_b eps C / A_b, min_b eps^2 C^2 / B_b),
 * and dt_exe = dt_coll / 2^k for the smallest k >= 0 with dt_exe <= dt_req
 * (repeated halving).  Reading: adjacent occupied fine bins are merged in
 * ascending size until each group holds at least max(N_K, 64) particles, a
 * remainder below that joins the group before it; bins with A_b = 0 (or
 * B_b = 0) do not constrain; one spatial group per instance. */
void gdo_choose_interval(const gdo_params* P, int64_t n, const double* s, const double* M,
                         const double* mA, const double* mB, gdo_state* st,
                         int32_t* group_of) {
  gdo_choose_interval_ab(P, n, s, M, mA, mB, st, group_of, NULL, NULL);
}

/* The request of one interval choice: controller bins, A_b and B_b, dt_req and the level k
 * of repeated halving (dt_exe = dt_coll 2^-k) the rule above gives, capped by the time
 * left.  Leaves st unchanged but for n_groups, near_dt and the floor status. */
static int request_level(const gdo_params* P, int64_t n, const double* s, const double* M,
                         const double* mA, const double* mB, gdo_state* st, int32_t* group_of,
                         double* A_b, double* B_b, double* dt_req_out) {
  int64_t cnt[GDO_NFINE];
  int gid[GDO_NFINE];
  double sM[GDO_NFINE], sA[GDO_NFINE], sB[GDO_NFINE];
  memset(cnt, 0, sizeof(cnt));
  for (int64_t i = 0; i < n; ++i) cnt[gdo_fine_bin(s[i])]++;
  int64_t thr = P->K > 64 ? P->K : 64;
  int ng = 0;
  int64_t acc = 0;
  for (int f = 0; f < GDO_NFINE; ++f) {
    gid[f] = -1;
    if (cnt[f] == 0) continue;
    gid[f] = ng;
    acc += cnt[f];
    if (acc >= thr) { ng++; acc = 0; }
  }
  if (acc > 0) {
    if (ng > 0) {
      for (int f = 0; f < GDO_NFINE; ++f)
        if (gid[f] == ng) gid[f] = ng - 1;
    } else {
      ng = 1;
    }
  }
  for (int g = 0; g < GDO_NFINE; ++g) { sM[g] = 0.0; sA[g] = 0.0; sB[g] = 0.0; }
  for (int64_t i = 0; i < n; ++i) {
    int g = gid[gdo_fine_bin(s[i])];
    sM[g] += M[i];
    sA[g] += M[i] * mA[i];
    sB[g] += M[i] * mB[i];
    if (group_of) group_of[i] = g;
  }
  double C = P->audit ? st->C : 1.0;
  /* The time left in the collision step is kept as an exact integer count of
   * dt_coll / 2^60 ticks: every executed interval is dt_coll / 2^k, so the
   * step then ends exactly (an FP64 difference such as dt_coll - dt_coll/4
   * is not always representable). */
  if (st->remain_ticks <= 0) st->remain_ticks = (int64_t)1 << 60;
  double remain = ldexp((double)st->remain_ticks, -60) * P->dt_coll;
  double dt_cap = remain < P->dt_fn_max ? remain : P->dt_fn_max;
  double dt_ab = HUGE_VAL;     /* the moment constraints (floating sums) */
  for (int g = 0; g < GDO_NFINE; ++g) {
    if (A_b) A_b[g] = 0.0;
    if (B_b) B_b[g] = 0.0;
  }
  for (int g = 0; g < ng; ++g) {
    double A = sA[g] / sM[g];
    double B = sB[g] / sM[g];
    if (A_b) A_b[g] = A;
    if (B_b) B_b[g] = B;
    if (A > 0.0) { double t = P->eps * C / A; if (t < dt_ab) dt_ab = t; }
    if (B > 0.0) { double t = P->eps * P->eps * C * C / B; if (t < dt_ab) dt_ab = t; }
  }
  double dt_req = dt_ab < dt_cap ? dt_ab : dt_cap;
  double dt = P->dt_coll;
  int k = 0;
  while (k < 60 && (dt > dt_req || ((int64_t)1 << (60 - k)) > st->remain_ticks)) {
    dt = 0.5 * dt;
    ++k;
  }
  if (dt > dt_req) st->status |= GDO_ST_DT_FLOOR;
  /* near tie: a moment constraint that binds within 1e-10 of a halving edge */
  if (dt_ab <= dt_cap * (1.0 + 1e-10) &&
      (fabs(dt - dt_ab) <= 1e-10 * dt_ab || fabs(2.0 * dt - dt_ab) <= 1e-10 * dt_ab))
    st->near_dt++;
  st->n_groups = ng;
  *dt_req_out = dt_req;
  return k;
}

/* Executes the interval dt_coll 2^-k: the time left drops by its exact tick count. */
static void commit_level(const gdo_params* P, gdo_state* st, int k, double dt_req) {
  st->dt_req = dt_req;
  st->dt_exe = ldexp(P->dt_coll, -k);
  st->remain_ticks -= (int64_t)1 << (60 - k);
}

void gdo_choose_interval_ab(const gdo_params* P, int64_t n, const double* s, const double* M,
                            const double* mA, const double* mB, gdo_state* st,
                            int32_t* group_of, double* A_b, double* B_b) {
  double dt_req;
  int k = request_level(P, n, s, M, mA, mB, st, group_of, A_b, B_b, &dt_req);
  commit_level(P, st, k, dt_req);
  if (st->remain_ticks == 0) st->remain_ticks = (int64_t)1 << 60;
  st->dt_remain = ldexp((double)st->remain_ticks, -60) * P->dt_coll;
}

/* Post-interval audit of the safety factor C (Sect. 2.5.3; the paper names
 * audits without giving a rule).  Reading: if any controller bin's realised
 * mass-weighted mean of sum_events |ln(s'/s)| exceeds 2 eps C, C <- max(1/4,
 * C/2); otherwise C <- min(1, 1.25 C).  With audit off C stays 1. */
void gdo_audit(const gdo_params* P, int64_t n, const double* M, const double* jsum,
               const int32_t* group_of, int32_t n_groups, gdo_state* st) {
  if (!P->audit) { st->C = 1.0; return; }
  double sM[GDO_NFINE], sJ[GDO_NFINE];
  for (int g = 0; g < GDO_NFINE; ++g) { sM[g] = 0.0; sJ[g] = 0.0; }
  for (int64_t i = 0; i < n; ++i) {
    sM[group_of[i]] += M[i];
    sJ[group_of[i]] += M[i] * jsum[i];
  }
  double thr = 2.0 * P->eps * st->C;
  int exceed = 0;
  for (int g = 0; g < n_groups; ++g) {
    double Rg = sJ[g] / sM[g];
    if (fabs(Rg - thr) <= 1e-10 * thr) st->near_audit++;
    if (Rg > thr) exceed = 1;
  }
  if (exceed) st->C = (0.5 * st->C > 0.25) ? 0.5 * st->C : 0.25;
  else st->C = (1.25 * st->C < 1.0) ? 1.25 * st->C : 1.0;
}

/* Channel rates of particle i against its frozen neighbourhood: slot-major,
 * channel-minor, summed left to right (the same order is the cumulative
 * rate used for partner selection). */
static double channels(const gdo_params* P, const gdo_gas* g, const int32_t* nbr, double V_i,
                       double s, double m, const double* s0, const double* m0,
                       const double* N0, double* ch, gdo_pair_t* prs) {
  double tot = 0.0;
  for (int k = 0; k < P->K; ++k) {
    int32_t j = nbr[k];
    gdo_pair(P, g, s, m, s0[j], m0[j], N0[j], V_i, &prs[k]);
    ch[2 * k] = prs[k].c[0];
    ch[2 * k + 1] = prs[k].c[1];
    tot = tot + ch[2 * k];
    tot = tot + ch[2 * k + 1];
  }
  return tot;
}

/* Monte Carlo sampling of one particle over one frozen interval,
 * Sect. 2.5.3: waiting times dt_w = -ln U / lambda*_i (Gillespie 1975);
 * stop once t + dt_w exceeds dt_exe; otherwise the partner channel is the
 * smallest c with U_s lambda*_i < C_c (cumulative rates in list order,
 * probability lambda*_ij / lambda*_i), the outcome follows Sect. 2.5.2, only
 * particle i changes, M_i is kept and N_i' = M_i/m_i'.  Partners keep the
 * properties frozen at the start of the interval (reading: the self slot's
 * partner too), i's own rates are recomputed after every event.
 * Draws: Philox key = seed, counter (i, interval, e, 0) gives (U_w, U_s) from
 * words (0,1) and (2,3); the fragment U of event e comes from counter
 * (i, interval, e, 1), words (0,1).  Near ties (|t + dt_w - dt_exe| or
 * |U_s lambda* - C_c| within 1e-10 relative) are counted. */
int gdo_sample_one(const gdo_params* P, const gdo_gas* g, int64_t i, const int32_t* nbr,
                   double V_i, const double* s0, const double* m0, const double* N0,
                   double M_i, double dt_exe, int64_t interval, double* s_io,
                   int32_t* ev_count, uint32_t* ev_hash, int32_t* near, double* jsum,
                   int64_t* status) {
  int K = P->K;
  double* ch = (double*)malloc(sizeof(double) * 2 * K);
  gdo_pair_t* prs = (gdo_pair_t*)malloc(sizeof(gdo_pair_t) * K);
  uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
  double s = *s_io;
  double m = gdo_grain_mass(P, s);
  double t = 0.0, J = 0.0;
  int32_t e = 0, nn = 0;
  uint32_t hash = 0;
  double tot = channels(P, g, nbr, V_i, s, m, s0, m0, N0, ch, prs);
  if (!isfinite(tot)) *status |= GDO_ST_NONFINITE;
  while (tot > 0.0) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)interval, (uint32_t)e, 0u}, w[4];
    gdo_philox4x32_10(ctr, key, w);
    double uw = gdo_u01(w[0], w[1]);
    double us = gdo_u01(w[2], w[3]);
    double dtw = -log(uw) / tot;
    if (fabs((t + dtw) - dt_exe) < 1e-10 * dt_exe) nn++;
    if (t + dtw > dt_exe) break;
    t = t + dtw;
    double target = us * tot;
    double cum = 0.0;
    int sel = -1, last = -1;
    for (int c = 0; c < 2 * K; ++c) {
      cum = cum + ch[c];
      if (ch[c] > 0.0) {
        last = c;
        if (fabs(target - cum) < 1e-10 * tot) nn++;
      }
      if (sel < 0 && target < cum) sel = c;
    }
    if (sel < 0) { sel = last; nn++; }
    int slot = sel / 2, cc = sel % 2;
    int32_t j = nbr[slot];
    const gdo_pair_t* pr = &prs[slot];
    double m_new, s_new;
    if (pr->outcome == 0) {
      m_new = m + pr->ncoll * m0[j];
      s_new = cbrt(6.0 * m_new / (GDO_PI * P->rho_s));
    } else if (pr->outcome == 1 && cc == 0) {
      m_new = m - pr->ncoll * m0[j];
      s_new = cbrt(6.0 * m_new / (GDO_PI * P->rho_s));
    } else if (pr->outcome == 1) {
      m_new = m0[j];
      s_new = s0[j];
    } else {
      uint32_t c2[4] = {(uint32_t)i, (uint32_t)interval, (uint32_t)e, 1u}, w2[4];
      gdo_philox4x32_10(c2, key, w2);
      double U = gdo_u01(w2[0], w2[1]);
      double a = sqrt(P->s_min), b = sqrt(s);
      double xr = a + U * (b - a);
      s_new = xr * xr;
      m_new = gdo_grain_mass(P, s_new);
    }
    J += fabs(log(s_new / s));
    s = s_new;
    m = m_new;
    hash = hash * 31u + (uint32_t)(sel + 1);
    ++e;
    if (e >= P->max_events) { *status |= GDO_ST_EVENT_CAP; break; }
    tot = channels(P, g, nbr, V_i, s, m, s0, m0, N0, ch, prs);
    if (!isfinite(tot)) *status |= GDO_ST_NONFINITE;
  }
  (void)M_i;   /* M_i is never written; N_i' = M_i / m_i' follows from s */
  *s_io = s;
  if (ev_count) *ev_count = e;
  if (ev_hash) *ev_hash = hash;
  if (near) *near = nn;
  if (jsum) *jsum = J;
  free(ch);
  free(prs);
  return 0;
}

/* Rates of a set of query particles against lists given as input (the
 * oracle's own lists): lambda*_i, sum_o lambda* <J>, sum_o lambda* <J^2>. */
int gdo_rates_subset(const gdo_params* P, int64_t n, const double* x, const double* y,
                     const double* z, const double* s, const double* M, int64_t nq,
                     const int64_t* q, const int32_t* nbr, const double* d, double* lam,
                     double* mA, double* mB, double* chan) {
  int K = P->K;
  for (int64_t t = 0; t < nq; ++t) {
    int64_t i = q[t];
    gdo_gas g;
    gdo_gas_at(P, x[i], y[i], z[i], &g);
    double V = (P->kernel_mode == GDO_PHYSICAL) ? gdo_volume(P, d[t], g.R) : 1.0;
    double mi = gdo_grain_mass(P, s[i]);
    double L = 0.0, A = 0.0, B = 0.0;
    for (int k = 0; k < K; ++k) {
      int32_t j = nbr[t * K + k];
      double mj = gdo_grain_mass(P, s[j]);
      gdo_pair_t pr;
      gdo_pair(P, &g, s[i], mi, s[j], mj, M[j] / mj, V, &pr);
      for (int c = 0; c < 2; ++c) {
        L = L + pr.c[c];
        A = A + pr.c[c] * pr.J1[c];
        B = B + pr.c[c] * pr.J2[c];
        if (chan) chan[(t * K + k) * 2 + c] = pr.c[c];
      }
    }
    if (lam) lam[t] = L;
    if (mA) mA[t] = A;
    if (mB) mB[t] = B;
  }
  (void)n;
  return 0;
}

/* Sampling of a set of query particles over one interval of length dt_exe,
 * partners frozen at the start values s0 (the oracle's own lists). */
int gdo_sample_subset(const gdo_params* P, int64_t n, const double* x, const double* y,
                      const double* z, const double* s0, const double* M, int64_t nq,
                      const int64_t* q, const int32_t* nbr, const double* d, double dt_exe,
                      int64_t interval, double* s_q, int32_t* ev_count, uint32_t* ev_hash,
                      int32_t* near, double* jsum, int64_t* status) {
  int K = P->K;
  double* m0 = (double*)malloc(sizeof(double) * n);
  double* N0 = (double*)malloc(sizeof(double) * n);
  for (int64_t j = 0; j < n; ++j) {
    m0[j] = gdo_grain_mass(P, s0[j]);
    N0[j] = M[j] / m0[j];
  }
  for (int64_t t = 0; t < nq; ++t) {
    int64_t i = q[t];
    gdo_gas g;
    gdo_gas_at(P, x[i], y[i], z[i], &g);
    double V = (P->kernel_mode == GDO_PHYSICAL) ? gdo_volume(P, d[t], g.R) : 1.0;
    s_q[t] = s0[i];
    gdo_sample_one(P, &g, i, nbr + t * K, V, s0, m0, N0, M[i], dt_exe, interval, &s_q[t],
                   ev_count ? &ev_count[t] : NULL, ev_hash ? &ev_hash[t] : NULL,
                   near ? &near[t] : NULL, jsum ? &jsum[t] : NULL, status);
  }
  free(m0);
  free(N0);
  return 0;
}

/* One whole frozen-neighbour interval of one instance (Sect. 2.5): K-NN,
 * measures, the frozen snapshot, rates and moments, the interval choice,
 * sampling of every particle and the audit.  s is updated in place; M is
 * only read. */
int gdo_interval_step(const gdo_params* P, int64_t n, const double* x, const double* y,
                      const double* z, double* s, const double* M, gdo_state* st,
                      gdo_outputs* out) {
  int K = P->K;
  if (n < K || K < 1) { st->status |= GDO_ST_KNN; return -1; }
  gdo_gas* gas = (gdo_gas*)malloc(sizeof(gdo_gas) * n);
  int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * n * K);
  double* d = (double*)malloc(sizeof(double) * n);
  double* V = (double*)malloc(sizeof(double) * n);
  double* s0 = (double*)malloc(sizeof(double) * n);
  double* m0 = (double*)malloc(sizeof(double) * n);
  double* N0 = (double*)malloc(sizeof(double) * n);
  double* mA = (double*)malloc(sizeof(double) * n);
  double* mB = (double*)malloc(sizeof(double) * n);
  double* jsum = (double*)malloc(sizeof(double) * n);
  int32_t* grp = (int32_t*)malloc(sizeof(int32_t) * n);
  double* ch = (double*)malloc(sizeof(double) * 2 * K);
  gdo_pair_t* prs = (gdo_pair_t*)malloc(sizeof(gdo_pair_t) * K);

  for (int64_t i = 0; i < n; ++i) {
    gdo_gas_at(P, x[i], y[i], z[i], &gas[i]);
    s0[i] = s[i];
    m0[i] = gdo_grain_mass(P, s[i]);
    N0[i] = M[i] / m0[i];
  }
  for (int64_t i = 0; i < n; ++i) {
    gdo_knn_one(P, n, x, y, z, i, nbr + i * K, &d[i]);
    V[i] = (P->kernel_mode == GDO_PHYSICAL) ? gdo_volume(P, d[i], gas[i].R) : 1.0;
  }
  for (int64_t i = 0; i < n; ++i) {
    double L = channels(P, &gas[i], nbr + i * K, V[i], s0[i], m0[i], s0, m0, N0, ch, prs);
    double A = 0.0, B = 0.0;
    for (int k = 0; k < K; ++k)
      for (int c = 0; c < 2; ++c) {
        A = A + prs[k].c[c] * prs[k].J1[c];
        B = B + prs[k].c[c] * prs[k].J2[c];
      }
    mA[i] = A;
    mB[i] = B;
    if (!isfinite(L)) st->status |= GDO_ST_NONFINITE;
    if (out && out->lam) out->lam[i] = L;
    if (out && out->chan) memcpy(out->chan + i * 2 * K, ch, sizeof(double) * 2 * K);
  }
  st->near_dt = 0;
  st->near_audit = 0;
  gdo_choose_interval_ab(P, n, s0, M, mA, mB, st, grp, out ? out->A_b : NULL,
                         out ? out->B_b : NULL);
  st->events = 0;
  st->near_draw = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t ec = 0, nn = 0;
    uint32_t hh = 0;
    gdo_sample_one(P, &gas[i], i, nbr + i * K, V[i], s0, m0, N0, M[i], st->dt_exe,
                   st->interval, &s[i], &ec, &hh, &nn, &jsum[i], &st->status);
    st->events += ec;
    st->near_draw += nn;
    if (out && out->ev_count) out->ev_count[i] = ec;
    if (out && out->ev_hash) out->ev_hash[i] = hh;
    if (out && out->near) out->near[i] = nn;
  }
  gdo_audit(P, n, M, jsum, grp, st->n_groups, st);
  st->interval++;
  if (out) {
    if (out->nbr) memcpy(out->nbr, nbr, sizeof(int32_t) * n * K);
    if (out->d) memcpy(out->d, d, sizeof(double) * n);
    if (out->V) memcpy(out->V, V, sizeof(double) * n);
    if (out->mA) memcpy(out->mA, mA, sizeof(double) * n);
    if (out->mB) memcpy(out->mB, mB, sizeof(double) * n);
    if (out->jsum) memcpy(out->jsum, jsum, sizeof(double) * n);
  }
  free(gas); free(nbr); free(d); free(V); free(s0); free(m0); free(N0);
  free(mA); free(mB); free(jsum); free(grp); free(ch); free(prs);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Spatial groups, Sect. 2.5.3 (the domain split into groups that keep their own
 * frozen-neighbour intervals; interacting groups' intervals at most 16 apart;
 * scheduled intervals are kept, so a refinement may wait). */

/* Group of a particle.  Reading: G equal-width groups, radial annuli of a disk over
 * [R_in, R_out) with R = sqrt(x^2 + y^2), slabs of a patch over x in [-box_x/2,
 * box_x/2); positions beyond the edges join the first or last group. */
int32_t gdo_group_of(const gdo_params* P, int32_t G, double x, double y) {
  double u;
  if (P->geometry == GDO_DISK) {
    double R = sqrt(x * x + y * y);
    u = (R - P->R_in) / (P->R_out - P->R_in);
  } else {
    u = (x + 0.5 * P->box_x) / P->box_x;
  }
  double f = floor(u * (double)G);
  if (!(f >= 0.0)) return 0;           /* also a NaN position */
  if (f >= (double)G) return G - 1;
  return (int32_t)f;
}

void gdo_groups_reset(const gdo_params* P, int32_t G, gdo_groups* S) {
  memset(S, 0, sizeof(*S));
  S->n_groups = G;
  for (int g = 0; g < GDO_MAXG; ++g) {
    S->level[g] = -1;
    S->k_req[g] = -1;
    S->st[g].C = 1.0;
    S->st[g].dt_remain = P->dt_coll;
    S->st[g].remain_ticks = 0;         /* no step begun */
  }
}

void gdo_groups_assign(const gdo_params* P, int64_t n, const double* x, const double* y,
                       const int32_t* nbr, int32_t* group_of, gdo_groups* S) {
  const int G = S->n_groups;
  for (int g = 0; g < GDO_MAXG; ++g) {
    S->members[g] = 0;
    S->inter[g] = 0;
  }
  for (int64_t i = 0; i < n; ++i) {
    group_of[i] = gdo_group_of(P, G, x[i], y[i]);
    S->members[group_of[i]]++;
  }
  /* g and h interact when a list of g holds a particle of h, or one of h a particle of g */
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < P->K; ++k) {
      int32_t h = group_of[nbr[i * P->K + k]], g = group_of[i];
      if (h != g) {
        S->inter[g] |= (uint64_t)1 << h;
        S->inter[h] |= (uint64_t)1 << g;
      }
    }
}

/* Levels of the active groups of one round.  Reading of the ratio-16 rule with
 * scheduled intervals kept:
 *  - an active group must end inside the collision step: at least its level k_fit;
 *  - an inactive interacting group h is in the middle of its interval, which is kept:
 *    the active group takes a level within 4 of level[h] (a coarser request is
 *    refined to level[h] - 4, a finer one waits at level[h] + 4: a delayed
 *    refinement), except that ending inside the step wins (counted as a break);
 *  - among active interacting groups the finest-allowed levels follow the chains of
 *    interactions (hi[g] <= hi[h] + 4), then each takes its request within [lo, hi]
 *    and the coarser of two interacting groups is refined until they are within 4.
 * Both passes are monotone iterations to their fixed points, so their order does not
 * matter. */
void gdo_schedule(int32_t G, const uint64_t* inter, const int64_t* members, const int32_t* active,
                  const int32_t* k_req, const int32_t* k_fit, int32_t* level, int64_t* delayed,
                  int64_t* breaks) {
  int lo[GDO_MAXG], hi[GDO_MAXG], k[GDO_MAXG];
  for (int g = 0; g < G; ++g) {
    if (!active[g]) continue;
    lo[g] = k_fit[g];
    hi[g] = 60;
    for (int h = 0; h < G; ++h) {
      if (h == g || active[h] || members[h] == 0 || level[h] < 0) continue;
      if (!((inter[g] >> h) & 1)) continue;
      if (level[h] - 4 > lo[g]) lo[g] = level[h] - 4;
      if (level[h] + 4 < hi[g]) hi[g] = level[h] + 4;
    }
    if (hi[g] < lo[g]) hi[g] = lo[g];
  }
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int g = 0; g < G; ++g) {
      if (!active[g]) continue;
      for (int h = 0; h < G; ++h) {
        if (h == g || !active[h] || !((inter[g] >> h) & 1)) continue;
        int cap = hi[h] + 4 > lo[g] ? hi[h] + 4 : lo[g];
        if (cap < hi[g]) { hi[g] = cap; changed = 1; }
      }
    }
  }
  for (int g = 0; g < G; ++g) {
    if (!active[g]) continue;
    int kk = k_req[g] < hi[g] ? k_req[g] : hi[g];
    k[g] = kk > lo[g] ? kk : lo[g];
  }
  changed = 1;
  while (changed) {
    changed = 0;
    for (int g = 0; g < G; ++g) {
      if (!active[g]) continue;
      for (int h = 0; h < G; ++h) {
        if (h == g || !active[h] || !((inter[g] >> h) & 1)) continue;
        if (k[g] < k[h] - 4) { k[g] = k[h] - 4; changed = 1; }
      }
    }
  }
  for (int g = 0; g < G; ++g) {
    if (!active[g]) continue;
    if (k[g] < k_req[g]) (*delayed)++;
    level[g] = k[g];
  }
  for (int g = 0; g < G; ++g)
    for (int h = g + 1; h < G; ++h) {
      if (!((inter[g] >> h) & 1) || level[g] < 0 || level[h] < 0) continue;
      if (!active[g] && !active[h]) continue;
      if (level[g] - level[h] > 4 || level[h] - level[g] > 4) (*breaks)++;
    }
}

int gdo_group_round(const gdo_params* P, int64_t n, const int32_t* nbr, const double* V,
                    const gdo_gas* gas, double* s, double* s0, const double* M,
                    const int32_t* group_of, gdo_groups* S, gdo_outputs* out) {
  const int G = S->n_groups;
  const int K = P->K;
  const int64_t full = (int64_t)1 << 60;
  int new_step = 1;
  for (int g = 0; g < G; ++g)
    if (S->members[g] > 0 && S->st[g].remain_ticks > 0) new_step = 0;
  if (new_step)
    for (int g = 0; g < G; ++g) {
      S->st[g].remain_ticks = full;
      S->level[g] = -1;             /* a new step: no interval scheduled */
    }
  /* the clock of the round: the earliest end of a scheduled interval */
  int64_t t = full;
  for (int g = 0; g < G; ++g)
    if (S->members[g] > 0 && S->st[g].remain_ticks > 0 && full - S->st[g].remain_ticks < t)
      t = full - S->st[g].remain_ticks;
  for (int g = 0; g < G; ++g)
    S->active[g] = S->members[g] > 0 && S->st[g].remain_ticks > 0 &&
                   full - S->st[g].remain_ticks == t;
  S->t = t;
  /* the active groups broadcast: their sizes enter the partner snapshot */
  for (int64_t i = 0; i < n; ++i)
    if (S->active[group_of[i]]) s0[i] = s[i];
  double* m0 = (double*)malloc(sizeof(double) * n);
  double* N0 = (double*)malloc(sizeof(double) * n);
  for (int64_t j = 0; j < n; ++j) {
    m0[j] = gdo_grain_mass(P, s0[j]);
    N0[j] = M[j] / m0[j];
  }
  double* ch = (double*)malloc(sizeof(double) * 2 * K);
  gdo_pair_t* prs = (gdo_pair_t*)malloc(sizeof(gdo_pair_t) * K);
  double* gs = (double*)malloc(sizeof(double) * n);
  double* gM = (double*)malloc(sizeof(double) * n);
  double* gA = (double*)malloc(sizeof(double) * n);
  double* gB = (double*)malloc(sizeof(double) * n);
  double* gJ = (double*)malloc(sizeof(double) * n);
  int32_t* gbin = (int32_t*)malloc(sizeof(int32_t) * n);
  int32_t* cbin = (int32_t*)malloc(sizeof(int32_t) * n);   /* controller bin of each particle */
  int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * n);
  int32_t k_fit[GDO_MAXG], k_req[GDO_MAXG];
  double dt_req[GDO_MAXG];
  /* rates, moments and the request of each active group (members in index order) */
  for (int g = 0; g < G; ++g) {
    k_fit[g] = 0;
    k_req[g] = 0;
    if (!S->active[g]) continue;
    gdo_state* st = &S->st[g];
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (group_of[i] != g) continue;
      double L = channels(P, &gas[i], nbr + i * K, V[i], s0[i], m0[i], s0, m0, N0, ch, prs);
      double A = 0.0, B = 0.0;
      for (int kk = 0; kk < K; ++kk)
        for (int c = 0; c < 2; ++c) {
          A = A + prs[kk].c[c] * prs[kk].J1[c];
          B = B + prs[kk].c[c] * prs[kk].J2[c];
        }
      if (!isfinite(L)) st->status |= GDO_ST_NONFINITE;
      if (out && out->lam) out->lam[i] = L;
      idx[m] = i;
      gs[m] = s0[i];
      gM[m] = M[i];
      gA[m] = A;
      gB[m] = B;
      ++m;
    }
    st->near_dt = 0;
    st->near_audit = 0;
    k_req[g] = request_level(P, m, gs, gM, gA, gB, st, gbin, NULL, NULL, &dt_req[g]);
    for (int64_t t2 = 0; t2 < m; ++t2) cbin[idx[t2]] = gbin[t2];
    while (k_fit[g] < 60 && ((int64_t)1 << (60 - k_fit[g])) > st->remain_ticks) k_fit[g]++;
    S->k_req[g] = k_req[g];
  }
  gdo_schedule(G, S->inter, S->members, S->active, k_req, k_fit, S->level, &S->delayed,
               &S->breaks);
  /* each active group commits its interval, samples it and audits it */
  for (int g = 0; g < G; ++g) {
    if (!S->active[g]) continue;
    gdo_state* st = &S->st[g];
    commit_level(P, st, S->level[g], dt_req[g]);
    st->dt_remain = ldexp((double)st->remain_ticks, -60) * P->dt_coll;
    st->events = 0;
    st->near_draw = 0;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (group_of[i] != g) continue;
      int32_t ec = 0, nn = 0;
      uint32_t hh = 0;
      double J = 0.0;
      gdo_sample_one(P, &gas[i], i, nbr + i * K, V[i], s0, m0, N0, M[i], st->dt_exe,
                     st->interval, &s[i], &ec, &hh, &nn, &J, &st->status);
      st->events += ec;
      st->near_draw += nn;
      if (out && out->ev_count) out->ev_count[i] = ec;
      if (out && out->ev_hash) out->ev_hash[i] = hh;
      if (out && out->near) out->near[i] = nn;
      if (out && out->jsum) out->jsum[i] = J;
      gM[m] = M[i];
      gJ[m] = J;
      gbin[m] = cbin[i];     /* the controller bins of the interval's choice */
      ++m;
    }
    gdo_audit(P, m, gM, gJ, gbin, st->n_groups, st);
    st->interval++;
    S->intervals[g]++;
  }
  S->rounds++;
  free(m0); free(N0); free(ch); free(prs); free(gs); free(gM); free(gA); free(gB);
  free(gJ); free(gbin); free(cbin); free(idx);
  return new_step;
}

int gdo_collide_groups(const gdo_params* P, int64_t n, const double* x, const double* y,
                       const double* z, double* s, const double* M, gdo_groups* S,
                       int32_t max_rounds) {
  int K = P->K;
  if (n < K || K < 1) return -1;
  gdo_gas* gas = (gdo_gas*)malloc(sizeof(gdo_gas) * n);
  int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * n * K);
  double* d = (double*)malloc(sizeof(double) * n);
  double* V = (double*)malloc(sizeof(double) * n);
  double* s0 = (double*)malloc(sizeof(double) * n);
  int32_t* grp = (int32_t*)malloc(sizeof(int32_t) * n);
  for (int64_t i = 0; i < n; ++i) {
    gdo_gas_at(P, x[i], y[i], z[i], &gas[i]);
    s0[i] = s[i];
  }
  for (int64_t i = 0; i < n; ++i) {
    gdo_knn_one(P, n, x, y, z, i, nbr + i * K, &d[i]);
    V[i] = (P->kernel_mode == GDO_PHYSICAL) ? gdo_volume(P, d[i], gas[i].R) : 1.0;
  }
  /* members and interaction masks follow the positions and lists of this step; the
   * groups' clocks, levels and C carry over */
  gdo_groups_assign(P, n, x, y, nbr, grp, S);
  int rc = -2;
  for (int r = 0; r < max_rounds; ++r) {
    gdo_group_round(P, n, nbr, V, gas, s, s0, M, grp, S, NULL);
    int done = 1;
    for (int g = 0; g < S->n_groups; ++g)
      if (S->members[g] > 0 && S->st[g].remain_ticks > 0) done = 0;
    if (done) { rc = r + 1; break; }
  }
  free(gas); free(nbr); free(d); free(V); free(s0); free(grp);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Staggered semi-analytic step, Sect. 2.3.3, for y = (v_r, l_theta, l_phi):
 * dy/dt = -Gamma y + y_g/t_s + f with Gamma = 1/t_s (no radiation),
 * f_r = -G M_star/r^2 + l_theta^2/r^3 + l_phi^2/(r^3 sin^2 theta),
 * f_theta = l_phi^2 cos theta/(r^2 sin^3 theta), f_phi = 0.
 * Reading (the paper gives the equation, not the update): drift half a step,
 * kick with the exact solution of the linear ODE at the midpoint,
 *   y <- y + k (gamma (y_g - y) + f),  k = (1 - e^{-gamma dt})/gamma (k = dt
 * when drag is off), then drift the second half in mirrored order (radius
 * first), which makes the step time-symmetric and a leapfrog without drag.
 * Gas velocity: v_r = l_theta = 0, l_phi,g = sqrt(1 - 2 eta) Omega_K R * R
 * (Sect. 2.2). */
void gdo_push_one(const gdo_params* P, int32_t drag, double dt, double* x, double* y,
                  double* z, double* vr, double* lth, double* lph, double s) {
  double r = sqrt(*x * *x + *y * *y + *z * *z);
  double th = acos(*z / r);
  double ph = atan2(*y, *x);
  double h = 0.5 * dt;
  double st = sin(th);
  ph = ph + h * *lph / (r * r * st * st);
  th = th + h * *lth / (r * r);
  r = r + h * *vr;
  st = sin(th);
  double ct = cos(th);
  double GM = GDO_G * P->M_star;
  double fr = -GM / (r * r) + *lth * *lth / (r * r * r) + *lph * *lph / (r * r * r * st * st);
  double fth = *lph * *lph * ct / (r * r * st * st * st);
  double gam = 0.0, ygph = 0.0;
  if (drag) {
    gdo_gas g;
    gas_RZ(P, r * st, r * ct, &g);
    double ts = g.gst * s / g.Om;
    gam = 1.0 / ts;
    ygph = sqrt(1.0 - 2.0 * g.eta) * g.Om * g.R * g.R;
  }
  double k = (gam > 0.0) ? -expm1(-dt * gam) / gam : dt;
  *vr = *vr + k * (gam * (0.0 - *vr) + fr);
  *lth = *lth + k * (gam * (0.0 - *lth) + fth);
  *lph = *lph + k * (gam * (ygph - *lph));
  r = r + h * *vr;
  th = th + h * *lth / (r * r);
  st = sin(th);
  ph = ph + h * *lph / (r * r * st * st);
  *x = r * st * cos(ph);
  *y = r * st * sin(ph);
  *z = r * cos(th);
}

/* The step above for n particles. */
void gdo_push(const gdo_params* P, int32_t drag, double dt, int64_t n, double* x, double* y,
              double* z, double* vr, double* lth, double* lph, const double* s) {
  for (int64_t i = 0; i < n; ++i)
    gdo_push_one(P, drag, dt, &x[i], &y[i], &z[i], &vr[i], &lth[i], &lph[i], s[i]);
}

/* ------------------------------------------------------------------ */
/* Radiation forces, Sect. 2.3.2.  beta(s) and kappa(s) scale as (s/s_0)^-1
 * (Eqs. beta, kappa); beta0 and kappa0 are set independently (the paper allows it),
 * s_0 is a diameter like every s here. */
#define GDO_C_LIGHT 2.99792458e10   /* speed of light [cm s^-1] */

/* sizeof(gdo_params), for the Python mirror's layout check */
int64_t gdo_params_size(void) { return (int64_t)sizeof(gdo_params); }

double gdo_rad_beta(const gdo_params* P, double s) { return P->beta0 * (P->rad_s0 / s); }

double gdo_rad_kappa(const gdo_params* P, double s) { return P->kappa0 * (P->rad_s0 / s); }

/* Sect. 2.3.2: the taper xi^2 (3 - 2 xi), xi = min(max(t / t_beta, 0), 1); no taper
 * (factor 1) when t_beta <= 0 (reading). */
double gdo_rad_taper(const gdo_params* P, double t) {
  if (!(P->t_beta > 0.0)) return 1.0;
  double xi = t / P->t_beta;
  if (xi < 0.0) xi = 0.0;
  if (xi > 1.0) xi = 1.0;
  return xi * xi * (3.0 - 2.0 * xi);
}

/* The optical depth grid (Sect. 2.3.2, Eqs. tau_3d and tau_2d).  Readings, the paper
 * naming neither the grid nor the deposit:
 *  - 3D form: cells uniform in r over [tau_rmin, tau_rmax), in mu = cos theta over
 *    [-tau_mu, tau_mu) and in phi over [-pi, pi); 2D form: uniform in R and phi, one
 *    polar cell.  A column is one (mu, phi) cell, j * nphi + k.
 *  - Each particle adds kappa(s_i) M_i to the cell that holds it (nearest grid point);
 *    particles outside the grid add nothing.  The cell's kappa rho_d is that sum over the
 *    cell volume, (r_hi^3 - r_lo^3)/3 dmu dphi, or in the 2D form kappa Sigma_d /
 *    (sqrt(2 pi) H_g) with Sigma_d over the area (R_hi^2 - R_lo^2)/2 dphi and H_g at the
 *    cell's mid radius.
 *  - tau is the integral from the grid's inner edge (no interior extinction): T at
 *    the radial faces of each column, T_0 = 0, T_{i+1} = T_i + (kappa rho_d)_i dr, stored
 *    as T[column * (nr + 1) + i].
 *  - At a point, tau is linear in r between the faces of its column (the exact integral
 *    of the binned density) and bilinear between the centres of the four nearest
 *    columns (clamped at the polar edges, periodic in phi); zero inside tau_rmin, the
 *    outer face beyond tau_rmax. */
static int tau_nmu(const gdo_params* P) { return P->tau_geom == GDO_TAU_2D ? 1 : P->tau_nmu; }

int64_t gdo_tau_size(const gdo_params* P) {
  if (P->tau_nr <= 0) return 0;
  return (int64_t)tau_nmu(P) * P->tau_nphi * (P->tau_nr + 1);
}

/* phi folded into [-pi, pi) */
static double fold_phi(double ph) { return ph - 2.0 * GDO_PI * floor((ph + GDO_PI) / (2.0 * GDO_PI)); }

/* cell of a point given by its grid radius (r or R), mu and phi; -1 outside */
static int64_t tau_cell(const gdo_params* P, double rad, double mu, double phi) {
  int nr = P->tau_nr, nm = tau_nmu(P), np = P->tau_nphi;
  double dr = (P->tau_rmax - P->tau_rmin) / nr;
  double u = (rad - P->tau_rmin) / dr;
  if (!(u >= 0.0) || !(u < (double)nr)) return -1;
  int64_t i = (int64_t)floor(u);
  int64_t j = 0;
  if (P->tau_geom != GDO_TAU_2D) {
    double dmu = 2.0 * P->tau_mu / nm;
    double w = (mu + P->tau_mu) / dmu;
    if (!(w >= 0.0) || !(w < (double)nm)) return -1;
    j = (int64_t)floor(w);
  }
  double dphi = 2.0 * GDO_PI / np;
  int64_t k = (int64_t)floor((phi + GDO_PI) / dphi);
  if (k >= np) k = np - 1;
  if (k < 0) k = 0;
  return (j * np + k) * (nr + 1) + i;   /* index of the cell's inner face */
}

/* builds T from the points (rad, mu, phi) of n particles, their sizes and masses */
static void tau_build(const gdo_params* P, int64_t n, const double* rad, const double* mu,
                      const double* phi, const double* s, const double* M, double* T) {
  int nr = P->tau_nr, nm = tau_nmu(P), np = P->tau_nphi;
  int64_t size = gdo_tau_size(P);
  for (int64_t c = 0; c < size; ++c) T[c] = 0.0;
  /* the sums of kappa M, each kept at its cell's inner face slot for now */
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = tau_cell(P, rad[i], mu[i], phi[i]);
    if (c >= 0) T[c] += gdo_rad_kappa(P, s[i]) * M[i];
  }
  double dr = (P->tau_rmax - P->tau_rmin) / nr;
  double dmu = 2.0 * P->tau_mu / nm;
  double dphi = 2.0 * GDO_PI / np;
  for (int64_t col = 0; col < (int64_t)nm * np; ++col) {
    double* Tc = T + col * (nr + 1);
    double acc = 0.0;
    for (int i = 0; i < nr; ++i) {
      double r_lo = P->tau_rmin + i * dr, r_hi = P->tau_rmin + (i + 1) * dr;
      double V;
      if (P->tau_geom == GDO_TAU_2D) {
        gdo_gas g;
        gas_RZ(P, P->tau_rmin + (i + 0.5) * dr, 0.0, &g);
        V = (r_hi * r_hi - r_lo * r_lo) / 2.0 * dphi * (sqrt(2.0 * GDO_PI) * g.H);
      } else {
        V = (r_hi * r_hi * r_hi - r_lo * r_lo * r_lo) / 3.0 * dmu * dphi;
      }
      double kr = Tc[i] / V;
      Tc[i] = acc;
      acc = acc + kr * dr;
    }
    Tc[nr] = acc;
  }
}

/* tau at a point given by its grid radius, mu and phi */
static double tau_interp(const gdo_params* P, const double* T, double rad, double mu, double phi) {
  int nr = P->tau_nr, nm = tau_nmu(P), np = P->tau_nphi;
  if (nr <= 0) return 0.0;
  double dr = (P->tau_rmax - P->tau_rmin) / nr;
  double u = (rad - P->tau_rmin) / dr;
  if (!(u > 0.0)) return 0.0;
  int64_t i = 0;
  double fr = 0.0;
  if (u >= (double)nr) {
    i = nr;
  } else {
    i = (int64_t)floor(u);
    fr = u - (double)i;
  }
  int64_t j0 = 0, j1 = 0;
  double fm = 0.0;
  if (nm > 1) {
    double dmu = 2.0 * P->tau_mu / nm;
    double w = (mu + P->tau_mu) / dmu - 0.5;
    if (w <= 0.0) {
      j0 = j1 = 0;
    } else if (w >= (double)(nm - 1)) {
      j0 = j1 = nm - 1;
    } else {
      j0 = (int64_t)floor(w);
      j1 = j0 + 1;
      fm = w - (double)j0;
    }
  }
  double dphi = 2.0 * GDO_PI / np;
  double v = (phi + GDO_PI) / dphi - 0.5;
  double kf = floor(v);
  double fp = v - kf;
  int64_t k0 = ((int64_t)kf % np + np) % np, k1 = (k0 + 1) % np;
  int64_t cols[4] = {j0 * np + k0, j0 * np + k1, j1 * np + k0, j1 * np + k1};
  double w4[4] = {(1.0 - fm) * (1.0 - fp), (1.0 - fm) * fp, fm * (1.0 - fp), fm * fp};
  double tau = 0.0;
  for (int c = 0; c < 4; ++c) {
    const double* Tc = T + cols[c] * (nr + 1);
    double tc = (i >= nr) ? Tc[nr] : Tc[i] + fr * (Tc[i + 1] - Tc[i]);
    tau = tau + w4[c] * tc;
  }
  return tau;
}

/* grid coordinates of a Cartesian point: (r, z/r, phi) in 3D, (R, 0, phi) in 2D */
static void tau_coords(const gdo_params* P, double x, double y, double z, double* rad, double* mu,
                       double* phi) {
  if (P->tau_geom == GDO_TAU_2D) {
    *rad = sqrt(x * x + y * y);
    *mu = 0.0;
  } else {
    *rad = sqrt(x * x + y * y + z * z);
    *mu = z / *rad;
  }
  *phi = atan2(y, x);
}

/* T from the particles at their positions (x, y, z). */
void gdo_tau_grid(const gdo_params* P, int64_t n, const double* x, const double* y,
                  const double* z, const double* s, const double* M, double* T) {
  if (P->tau_nr <= 0) return;
  double* c = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) tau_coords(P, x[i], y[i], z[i], &c[i], &c[n + i], &c[2 * n + i]);
  tau_build(P, n, c, c + n, c + 2 * n, s, M, T);
  free(c);
}

double gdo_tau_at(const gdo_params* P, const double* T, double x, double y, double z) {
  double rad, mu, phi;
  tau_coords(P, x, y, z, &rad, &mu, &phi);
  return tau_interp(P, T, rad, mu, phi);
}

/* The staggered step of gdo_push_one with radiation forces (Sect. 2.3.2-2.3.3):
 *  f_r = -(1 - beta e^-tau) GM/r^2 + l_theta^2/r^3 + l_phi^2/(r^3 sin^2 theta),
 *  gamma_PR = beta e^-tau GM/(c r^2), gamma_r = 1/t_s + 2 gamma_PR,
 *  gamma_theta = gamma_phi = 1/t_s + gamma_PR, and each component of
 *  dy/dt = -gamma y + y_g/t_s + f advanced exactly for fixed coefficients:
 *  y += k (f + y_g/t_s - gamma y), k = (1 - e^{-gamma dt})/gamma.
 * beta e^-tau carries the taper at the kick's time t + dt/2.  Readings: tau is built
 * from every particle at the midpoint of the first drift (the positions the kick sees)
 * and interpolated at each particle's own midpoint; mid holds (r, theta, phi) of all n
 * particles between the two passes, T the grid (gdo_tau_size doubles). */
void gdo_push_rad(const gdo_params* P, int32_t drag, double dt, double t, int64_t n, double* x,
                  double* y, double* z, double* vr, double* lth, double* lph, const double* s,
                  const double* M, double* T, double* mid) {
  double h = 0.5 * dt;
  double* mr = mid;
  double* mth = mid + n;
  double* mph = mid + 2 * n;
  for (int64_t i = 0; i < n; ++i) {
    double r = sqrt(x[i] * x[i] + y[i] * y[i] + z[i] * z[i]);
    double th = acos(z[i] / r);
    double ph = atan2(y[i], x[i]);
    double st = sin(th);
    ph = ph + h * lph[i] / (r * r * st * st);
    th = th + h * lth[i] / (r * r);
    r = r + h * vr[i];
    mr[i] = r;
    mth[i] = th;
    mph[i] = ph;
  }
  int grid = P->tau_nr > 0 && P->kappa0 > 0.0;
  if (grid) {
    double* c = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
      double st = sin(mth[i]);
      c[i] = (P->tau_geom == GDO_TAU_2D) ? mr[i] * st : mr[i];
      c[n + i] = (P->tau_geom == GDO_TAU_2D) ? 0.0 : cos(mth[i]);
      c[2 * n + i] = fold_phi(mph[i]);
    }
    tau_build(P, n, c, c + n, c + 2 * n, s, M, T);
    free(c);
  }
  double GM = GDO_G * P->M_star;
  double taper = gdo_rad_taper(P, t + h);
  for (int64_t i = 0; i < n; ++i) {
    double r = mr[i], th = mth[i], ph = mph[i];
    double st = sin(th);
    double ct = cos(th);
    double tau = 0.0;
    if (grid)
      tau = tau_interp(P, T, (P->tau_geom == GDO_TAU_2D) ? r * st : r, (P->tau_geom == GDO_TAU_2D) ? 0.0 : ct,
                       fold_phi(ph));
    double be = taper * gdo_rad_beta(P, s[i]) * exp(-tau);
    double fr = -(1.0 - be) * GM / (r * r) + lth[i] * lth[i] / (r * r * r) +
                lph[i] * lph[i] / (r * r * r * st * st);
    double fth = lph[i] * lph[i] * ct / (r * r * st * st * st);
    double gpr = P->rad_pr ? be * GM / (GDO_C_LIGHT * r * r) : 0.0;
    double gam = 0.0, ygph = 0.0;
    if (drag) {
      gdo_gas g;
      gas_RZ(P, r * st, r * ct, &g);
      double ts = g.gst * s[i] / g.Om;
      gam = 1.0 / ts;
      ygph = sqrt(1.0 - 2.0 * g.eta) * g.Om * g.R * g.R;
    }
    double g_r = gam + 2.0 * gpr, g_t = gam + gpr;
    double k_r = (g_r > 0.0) ? -expm1(-dt * g_r) / g_r : dt;
    double k_t = (g_t > 0.0) ? -expm1(-dt * g_t) / g_t : dt;
    vr[i] = vr[i] + k_r * (fr - g_r * vr[i]);
    lth[i] = lth[i] + k_t * (fth - g_t * lth[i]);
    lph[i] = lph[i] + k_t * (gam * ygph - g_t * lph[i]);
    r = r + h * vr[i];
    th = th + h * lth[i] / (r * r);
    st = sin(th);
    ph = ph + h * lph[i] / (r * r * st * st);
    x[i] = r * st * cos(ph);
    y[i] = r * st * sin(ph);
    z[i] = r * cos(th);
  }
}

/* ------------------------------------------------------------------ */
/* Dust diffusion, Sect. 2.4.  The diffusion tensor is diagonal in the local
 * cylindrical basis, D_a = nu / (Sc_a (1 + St^2)) with nu = alpha c_s H_g at R
 * (Sect. 2.2), and one Euler-Maruyama step displaces a particle by
 *   dR   = sqrt(2 D_R dt) zeta_R + (D_R/R + dD_R/dR + chi D_R dln rho_g/dR) dt
 *   dZ   = sqrt(2 D_Z dt) zeta_Z + (dD_Z/dZ + chi D_Z dln rho_g/dZ) dt
 *   dphi = sqrt(2 D_phi dt) zeta_phi / R     (the phi derivatives vanish: the
 *          disk is axisymmetric).
 * Reading: with the analytic disk of gas_RZ, ln nu = (q + 3/2) ln R + const,
 * ln St = const + ln s - ln Sigma_g + v with v = (1 - R/r)/h_g^2, h_g^2 ~ R^(q+1),
 * ln rho_g = ln Sigma_g - ln H_g - v + const, so
 *   dv/dR = -Z^2/(r^3 h^2) - (q+1) v / R,   dv/dZ = R Z/(r^3 h^2),
 *   dln D/dR = (q + 3/2)/R - f (-p/R + dv/dR),   dln D/dZ = -f dv/dZ,
 *   dln rho_g/dR = (p - q/2 - 3/2)/R - dv/dR,    dln rho_g/dZ = -dv/dZ,
 * with f = 2 St^2/(1 + St^2).
 * out: D_R, D_Z, D_phi, drift_R, drift_Z (the dt coefficients above), and
 * dln rho_g/dR, dln rho_g/dZ. */
void gdo_diff_coeffs(const gdo_params* P, double R, double Z, double s, double out[7]) {
  gdo_gas g;
  gas_RZ(P, R, Z, &g);
  double St = g.gst * s;
  double nu = P->alpha * g.cs * g.H;
  double D = nu / (1.0 + St * St);
  double v = (1.0 - R / g.r) / (g.h * g.h);
  double r3h2 = g.r * g.r * g.r * g.h * g.h;
  double dvdR = -Z * Z / r3h2 - (P->q + 1.0) * v / R;
  double dvdZ = R * Z / r3h2;
  double f = 2.0 * St * St / (1.0 + St * St);
  double dlnD_dR = (P->q + 1.5) / R - f * (-P->p / R + dvdR);
  double dlnD_dZ = -f * dvdZ;
  double dlnrho_dR = (P->p - 0.5 * P->q - 1.5) / R - dvdR;
  double dlnrho_dZ = -dvdZ;
  double chi = (double)P->diff_chi;
  double DR = D / P->Sc_R, DZ = D / P->Sc_Z, Dp = D / P->Sc_phi;
  out[0] = DR;
  out[1] = DZ;
  out[2] = Dp;
  out[3] = DR * (1.0 / R + dlnD_dR + chi * dlnrho_dR);
  out[4] = DZ * (dlnD_dZ + chi * dlnrho_dZ);
  out[5] = dlnrho_dR;
  out[6] = dlnrho_dZ;
}

/* Two standard normals from one Philox draw (Box-Muller on the (0,1) map). */
static void normals(const gdo_params* P, uint32_t i_loc, int64_t step, uint32_t word, double* n0,
                    double* n1) {
  uint32_t ctr[4] = {i_loc, (uint32_t)step, 0xFFFFFFFEu, word};
  uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
  uint32_t w[4];
  gdo_philox4x32_10(ctr, key, w);
  double u1 = gdo_u01(w[0], w[1]), u2 = gdo_u01(w[2], w[3]);
  double rad = sqrt(-2.0 * log(u1));
  *n0 = rad * cos(2.0 * GDO_PI * u2);
  *n1 = rad * sin(2.0 * GDO_PI * u2);
}

/* One Euler-Maruyama diffusion step of length dt for particles 0..n-1 of one
 * instance (Sect. 2.4).  Draws: Philox4x32-10 with the instance key and counter
 * (i, step, 0xFFFFFFFE, 0) for zeta_R, zeta_Z and (i, step, 0xFFFFFFFE, 1) for
 * zeta_phi (reading: a counter space of its own, apart from the sampler's and
 * the initial conditions').
 * Global disk: the displacement is applied in (R, phi, Z) and the position
 * rewritten in Cartesian; when velocities are given, their Cartesian vector is
 * kept and (v_r, l_theta, l_phi) recomputed in the basis at the new position
 * (reading of "recalculate the stored velocity components").  Local patch:
 * x += dR, y += R dphi, z += dZ with the periodic wrap.  Ring test (Sect. 3.2):
 * radial only, D = D0 (R/R_0)^2, drift D/R + dD/dR + chi D p / R, phi and Z
 * unchanged. */
void gdo_diffuse(const gdo_params* P, double dt, int64_t step, int64_t n, double* x, double* y,
                 double* z, double* vr, double* lth, double* lph, const double* s) {
  for (int64_t i = 0; i < n; ++i) {
    double zR, zZ, zP, unused;
    normals(P, (uint32_t)i, step, 0u, &zR, &zZ);
    normals(P, (uint32_t)i, step, 1u, &zP, &unused);
    if (P->geometry == GDO_PATCH) {
      double R = P->r0 + x[i];
      double c[7];
      gdo_diff_coeffs(P, R, z[i], s[i], c);
      double dR = sqrt(2.0 * c[0] * dt) * zR + c[3] * dt;
      double dZ = sqrt(2.0 * c[1] * dt) * zZ + c[4] * dt;
      double dy = sqrt(2.0 * c[2] * dt) * zP;
      double xn = x[i] + dR, yn = y[i] + dy;
      xn -= P->box_x * floor((xn + 0.5 * P->box_x) / P->box_x);
      yn -= P->box_y * floor((yn + 0.5 * P->box_y) / P->box_y);
      x[i] = xn;
      y[i] = yn;
      z[i] = z[i] + dZ;
      continue;
    }
    double R = sqrt(x[i] * x[i] + y[i] * y[i]);
    double ph = atan2(y[i], x[i]);
    double Z = z[i];
    double dR, dZ = 0.0, dph = 0.0;
    if (P->diff_mode == GDO_DIFF_RING) {
      double D = P->D0 * (R / P->r0) * (R / P->r0);
      dR = sqrt(2.0 * D * dt) * zR + D / R * (3.0 + (double)P->diff_chi * P->p) * dt;
    } else {
      double c[7];
      gdo_diff_coeffs(P, R, Z, s[i], c);
      dR = sqrt(2.0 * c[0] * dt) * zR + c[3] * dt;
      dZ = sqrt(2.0 * c[1] * dt) * zZ + c[4] * dt;
      dph = sqrt(2.0 * c[2] * dt) * zP / R;
    }
    double Rn = R + dR, phn = ph + dph, Zn = Z + dZ;
    if (Rn < 0.0) { Rn = -Rn; phn += GDO_PI; }
    double xn = Rn * cos(phn), yn = Rn * sin(phn);
    if (vr && lth && lph) {
      /* Cartesian velocity from (v_r, l_theta = r^2 dtheta/dt, l_phi = r^2 sin^2 theta dphi/dt) */
      double r = sqrt(R * R + Z * Z), st = R / r, ct = Z / r, cp = cos(ph), sp = sin(ph);
      double vth = lth[i] / r, vph = lph[i] / (r * st);
      double vx = vr[i] * st * cp + vth * ct * cp - vph * sp;
      double vy = vr[i] * st * sp + vth * ct * sp + vph * cp;
      double vz = vr[i] * ct - vth * st;
      double rn = sqrt(Rn * Rn + Zn * Zn), stn = Rn / rn, ctn = Zn / rn, cpn = cos(phn), spn = sin(phn);
      vr[i] = vx * stn * cpn + vy * stn * spn + vz * ctn;
      lth[i] = rn * (vx * ctn * cpn + vy * ctn * spn - vz * stn);
      lph[i] = rn * stn * (-vx * spn + vy * cpn);
    }
    x[i] = xn;
    y[i] = yn;
    z[i] = Zn;
  }
}

/* Sect. 2.6: the local timestep Delta t_i of particle i, the most restrictive of
 * the limits set by orbital motion and by the deterministic and diffusive
 * displacements against the local grid spacing.  Reading (the paper names the
 * limits, not their form or constants):
 *   orbital:        f_orb * 2 pi / Omega_K(R_i)
 *   deterministic:  c_adv * dx_i / |u_i|, u_i the velocity relative to the local
 *                   circular Keplerian motion, (v_r, l_theta / r, l_phi / R - Omega_K R);
 *                   global-disk particles with velocities only (patches do not move)
 *   diffusive:      (c_diff * dx_i)^2 / (2 D_i), D_i the largest of the directional
 *                   coefficients of Sect. 2.4 (ring test: D0 (R/R_0)^2)
 * with dx_i = dx_H * H_g(R_i): the analytic gas disk has no grid, so the caller
 * states its resolution in local gas scale heights.  A limit whose coefficient is
 * <= 0, or whose rate is zero, is off; a particle with no limit gives +infinity.
 * v: NULL or {v_r, l_theta, l_phi}. */
double gdo_local_dt(const gdo_params* P, const gdo_dt_rule* rule, double x, double y, double z,
                    double s, const double* v) {
  double R = P->geometry == GDO_PATCH ? P->r0 + x : sqrt(x * x + y * y);
  double Z = z;
  gdo_gas g;
  gas_RZ(P, R, Z, &g);
  double dt = INFINITY;
  if (rule->f_orb > 0.0) {
    double t_orb = rule->f_orb * 2.0 * GDO_PI / g.Om;
    if (t_orb < dt) dt = t_orb;
  }
  double dx = rule->dx_H * g.H;
  if (rule->c_adv > 0.0 && v != NULL && P->geometry == GDO_DISK) {
    double r = sqrt(R * R + Z * Z);
    double u_r = v[0];
    double u_th = v[1] / r;
    double u_ph = v[2] / R - g.Om * R;
    double u = sqrt(u_r * u_r + u_th * u_th + u_ph * u_ph);
    if (u > 0.0) {
      double t_adv = rule->c_adv * dx / u;
      if (t_adv < dt) dt = t_adv;
    }
  }
  if (rule->c_diff > 0.0) {
    double D;
    if (P->diff_mode == GDO_DIFF_RING) {
      D = P->D0 * (R / P->r0) * (R / P->r0);
    } else {
      double c[7];
      gdo_diff_coeffs(P, R, Z, s, c);
      D = c[0];
      if (c[1] > D) D = c[1];
      if (c[2] > D) D = c[2];
    }
    if (D > 0.0) {
      double t_diff = (rule->c_diff * dx) * (rule->c_diff * dx) / (2.0 * D);
      if (t_diff < dt) dt = t_diff;
    }
  }
  return dt;
}

/* Sect. 2.6: Delta t = min(Delta t_max, Delta t_out, min_i Delta t_i) over the
 * particles 0..n-1 of one instance (a context of several instances takes the
 * minimum over them).  dti: NULL or [n], each particle's Delta t_i. */
double gdo_timestep(const gdo_params* P, const gdo_dt_rule* rule, int64_t n, const double* x,
                    const double* y, const double* z, const double* s, const double* vr,
                    const double* lth, const double* lph, double* dti) {
  double dt = rule->dt_max < rule->dt_out ? rule->dt_max : rule->dt_out;
  for (int64_t i = 0; i < n; ++i) {
    double v[3];
    const double* vp = NULL;
    if (vr != NULL && lth != NULL && lph != NULL) {
      v[0] = vr[i];
      v[1] = lth[i];
      v[2] = lph[i];
      vp = v;
    }
    double t = gdo_local_dt(P, rule, x[i], y[i], z[i], s[i], vp);
    if (dti != NULL) dti[i] = t;
    if (t < dt) dt = t;
  }
  return dt;
}
