// gd_common.cuh -- device-side types and helpers shared by the library's kernels.
//
// Layout in HBM (library-owned, one context):
//   rank space  : particles sorted by (instance, cell); rank r of instance b lies in
//                 [off[b], off[b+1]) like the caller's indices.  perm[r] is the caller
//                 index, rank_of[i] its inverse.
//   Pos64[r]    : {x, y, z, caller index}            32 B  (FP64 K-NN, re-rank)
//   float4 pos32: {x, y, z relative to the own cell origin, packed cell (11+11+10 bits)} 16 B
//   Snap64[r]   : {s, m, N, 1/m} frozen at the interval start        32 B
//   float4 snap32: {s, m, N 2^-64, 1/m} frozen, FP32                 16 B
//   nbr[r*K+k]  : ranks of the K neighbours, slot 0 = self, others by ascending caller index
//   cell_start  : exclusive scan of per-cell counts, instance grids concatenated
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "gd.h"

namespace gd {

constexpr double kPi = 3.14159265358979323846;
constexpr double kKB = 1.380649e-16;     // Boltzmann constant [erg/K]
constexpr double kMH = 1.6735575e-24;    // hydrogen mass [g]
constexpr double kMu = 2.34;             // mean molecular weight
constexpr double kG = 6.674e-8;          // gravitational constant
constexpr double kSigH2 = 2e-15;         // H2 cross-section [cm^2]
constexpr int kNFine = 96;               // fine controller bins per instance
constexpr int kTMin = -72;               // fine bin of index 0: third-octave t = -72
constexpr int kMaxK = 256;

// Per-instance parameters as the kernels read them (derived once at create).
struct InstDev {
  int geometry, kernel_mode, audit, model;
  double r0, sigma0, p, T0, q, alpha, GM, rho_s, s_min, v_frag, eps, dt_coll, dt_fn_max;
  double R_in, R_out, box_x, box_y, t0, m0, cell_size;
  uint32_t key0, key1;
  long long off, n;
  double k6;          // 6 / (pi rho_s)
  double mk;          // pi rho_s / 6
  // FP32 copies of the parameters the mixed form's per-particle gas disk uses
  float f_r0, f_GM, f_T0, f_q, f_p, f_sigma0, f_alpha, f_rho_s, f_vfrag, f_m0, f_smin;
  // dust diffusion (Sect. 2.4)
  int diff_mode, diff_chi;
  double Sc_R, Sc_Z, Sc_phi, D0;
  // spatial groups (Sect. 2.5.3): n_sg groups, whose states are units unit0 .. unit0 + n_sg - 1
  // of the state and bin arrays (unit0 = b when no instance has more than one group)
  int n_sg, unit0;
  // radiation forces and the optical depth grid (Sect. 2.3.2)
  int rad;             // 1: beta0 > 0 (the push takes the radiation step)
  int tau_on;          // 1: the instance has a grid (tau_nr > 0, kappa0 > 0)
  int rad_pr, tau_geom, tau_nr, tau_nm, tau_np, pad_rad;   // tau_nm = 1 in the 2D form
  double beta0, kappa0, rad_s0, t_beta, tau_rmin, tau_rmax, tau_mu;
  long long tau_cell0, tau_face0;   // the instance's first cell / face in the concatenated arrays
  // FP32 copies for the mixed form, and the error bounds (in cells) of its FP32 grid
  // coordinates u (radial), w (polar) and v (azimuthal)
  float f_beta0, f_rad_s0, f_tau_rmin, f_tau_dr, f_tau_mu, f_tau_dmu, f_tau_dphi;
  float f_eu, f_ew, f_ev;
};

constexpr int kMaxSG = 64;               // spatial groups per instance (one 64-bit mask each)

// Mixed-form sampler: a heavy particle whose time decision the FP32 bounds leave open is
// settled by a deferred FP64 pass from its logged events, its states spread over the SMs.
struct DeferRec {
  long long r;       // rank
  long long lbase;   // first entry of its event log
  long long sbase;   // first entry of its states
  int n;             // logged events (states 0 .. n)
  int ok;            // 0: no room for its states (the particle is replayed in line)
};
struct DState {
  double s, m;       // diameter and mass after k events (the FP64 form's arithmetic)
  double lam, dt;    // lambda*_i at the state and the waiting time drawn from it
  double J, ncoll;   // |ln s'/s| of the event leaving the state; the chosen pair's N_coll
  int sset;          // 1: s is set, 0: s = cbrt(6 m / (pi rho_o)) (formed by the state pass)
  int chosen, j, outcome;   // the FP64 choice at the state
  int np, nc;        // near ties of the pairs' thresholds and of the channel choice
  int bad;           // the logged choice differs from the FP64 one
  int pad;
};

// Coordinates of the neighbour search in the instance's collision model (Sect. 2.5.1):
// 3D positions, the meridional plane (R, Z, 0), the midplane (x, y, 0) or (R, 0, 0).  R is
// the correctly rounded sqrt(x*x + y*y) without contraction, as the oracle forms it.
__device__ __forceinline__ void model_pos(int model, double x, double y, double z, double& X, double& Y,
                                          double& Z) {
  if (model == GD_MODEL_3D) { X = x; Y = y; Z = z; return; }
  if (model == GD_MODEL_RPHI) { X = x; Y = y; Z = 0.0; return; }
  X = __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
  Y = model == GD_MODEL_RZ ? z : 0.0;
  Z = 0.0;
}

// Spatial group of a position (Sect. 2.5.3): G equal-width radial annuli of a disk over
// [R_in, R_out) by R = sqrt(x^2 + y^2), or slabs of a patch over x in [-box_x/2, box_x/2);
// beyond the edges (and for a NaN) the first or last group.  Correctly rounded operations
// without contraction, as the oracle forms them.
__device__ __forceinline__ int group_of(const InstDev& p, double x, double y) {
  double u;
  if (p.geometry == GD_GEOM_DISK) {
    const double R = __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
    u = __ddiv_rn(__dadd_rn(R, -p.R_in), __dadd_rn(p.R_out, -p.R_in));
  } else {
    u = __ddiv_rn(__dadd_rn(x, __dmul_rn(0.5, p.box_x)), p.box_x);
  }
  const double f = floor(__dmul_rn(u, (double)p.n_sg));
  if (!(f >= 0.0)) return 0;
  if (f >= (double)p.n_sg) return p.n_sg - 1;
  return (int)f;
}

// Uniform cell grid of one instance, rebuilt every interval from the data bounds.
struct GridDev {
  double lo[3];      // origin
  double cs[3];      // cell edge per axis
  double inv[3];     // 1 / cs
  double box[3];     // periodic extent (x, y of a patch), 0 otherwise
  double ctr[3];     // origin of the FP32 mirror coordinates
  double X32;        // bound on |coordinate| + periodic extents (FP64 rounding of the mirror)
  float cs32[3];     // cell edges and their inverses in FP32 (search bookkeeping)
  float inv32[3];
  float E32;         // absolute error bound of FP32 cell-relative distances [cm]
  int dim[3];
  int periodic;      // x and y periodic (patch)
  long long cell_off;
};

// Mutable per-instance state (device resident).
struct StateDev {
  double C, dt_exe, dt_req, dt_remain;
  long long remain_ticks;   // exact time left: units of dt_coll / 2^60
  long long interval_cur;   // Philox interval counter of the current interval
  long long interval_next;
  long long events, events_total, near_draw, near_dt, near_audit;
  long long knn_redo;       // mixed K-NN queries redone in FP64
  long long rate_redo;      // mixed rates redone in FP64
  long long sample_redo;    // mixed sampling replayed in FP64
  long long sample_deferred;  // of those, settled by the deferred FP64 pass
  double tau;               // length of the current collision step (0: dt_coll)
  int hold;                 // 1: idle once the current collision step is used up (gd_collide)
  int pad_hold;
  unsigned int status;
  int n_groups;             // controller bins of the last interval choice
  // spatial groups (Sect. 2.5.3); a unit is one group of one instance.  The per-instance
  // round counters live in the instance's first unit.
  int active;               // 1: the unit takes part in the current round (always 1 with one group)
  int level;                // k of the scheduled (or last) interval, -1: none in this step
  int k_req;                // level requested in the current round
  int pad_sg;
  long long members;        // particles of the unit
  long long intervals;      // intervals the unit executed
  unsigned long long inter; // bit h: the unit interacts with group h of its instance
  long long rounds, delayed, breaks, clock;
  // bounds of the data (ordered-integer encodings of doubles), min then max, x y z
  unsigned long long bmin[3], bmax[3];
};

// Fine-bin sums of one instance (doubles; counts exact below 2^53), in this order (the
// tile reduction addresses them as quantity q of the block cnt, sM, sA, sB, sJ, sE, spec), and
// the controller bins of the last interval choice: the fine bins' group ids and each group's
// A_b and B_b.  sE is not a sum: the largest relative error bound of the mixed form's FP32
// moment contributions in the bin (0 in the FP64 form).  spec: the size spectrum of the last
// gd_stats, sum of M_i over the particles whose current diameter lies in the bin.
constexpr int kBinQ = 7;          // cnt, sM, sA, sB, sJ, sE, spec
struct BinsDev {
  double cnt[kNFine], sM[kNFine], sA[kNFine], sB[kNFine], sJ[kNFine], sE[kNFine], spec[kNFine];
  double gA[kNFine], gB[kNFine];
  int gid[kNFine];
  int ngroups;
  int pad;
};

// Per-block tiles of the per-particle passes: tile t covers [lo, hi) of one instance (at
// most kTile particles, never straddling an instance).  The tile table is derived from the
// offsets: block t belongs to the instance whose tile range contains t.
constexpr int kTile = 4096;
struct TileMap {
  const long long* off;
  int n_inst;
  const long long* tile_off;   // [n_inst + 1] first tile of each instance
};

__device__ __forceinline__ bool tile_range(const TileMap& tm, int tile, int& b, long long& lo, long long& hi) {
  int l = 0, h = tm.n_inst - 1;
  while (l < h) {
    int mid = (l + h + 1) >> 1;
    if (tm.tile_off[mid] <= tile) l = mid; else h = mid - 1;
  }
  b = l;
  long long t = tile - tm.tile_off[b];
  lo = tm.off[b] + t * kTile;
  hi = min(lo + kTile, tm.off[b + 1]);
  return lo < hi;
}

// One particle's contribution to the fine-bin sums of the interval choice (FP64 form):
// M_i, M_i pref sum_o lambda*_io <J_io>, likewise <J_io^2>, and the fine bin.  The mixed
// form holds the same in a float4 (M, MA, MB, w) whose w packs the fine bin in its low 7
// bits and, above them, the particle's relative error bound of its FP32 rates and moments
// rounded up (pack_ebin / ebin_bin / ebin_err).
struct Contrib64 {
  double M, MA, MB;
  long long fbin;
};

__device__ __forceinline__ float pack_ebin(float err, int bin) {
  const float e = fminf(fmaxf(err, 0.0f), 1.0f);
  const unsigned up = (__float_as_uint(e) + 127u) & ~127u;     // rounded up to 2^-16 relative
  return __uint_as_float(up | (unsigned)bin);
}
__device__ __forceinline__ int ebin_bin(float w) { return (int)(__float_as_uint(w) & 127u); }
__device__ __forceinline__ float ebin_err(float w) { return __uint_as_float(__float_as_uint(w) & ~127u); }

struct Pos64 {
  double x, y, z;
  long long j;
};

struct Snap64 {
  double s, m, N, inv_m;
};

// ---------------------------------------------------------------- small helpers
__device__ __forceinline__ int inst_of(const long long* __restrict__ off, int n_inst, long long r) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(&off[mid]) <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Order-preserving map of doubles to unsigned 64-bit integers (for atomic min/max).
__device__ __forceinline__ unsigned long long dbl_ord(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double ord_dbl(unsigned long long o) {
  unsigned long long b = (o >> 63) ? (o & 0x7FFFFFFFFFFFFFFFull) : ~o;
  union { unsigned long long u; double d; } c;
  c.u = b;
  return c.d;
}

// Fine controller bin: thirds of an octave, edges at 2^e {1/2, 2^(1/3)/2, 2^(2/3)/2}
// taken from the exponent and mantissa bits of s (s > 0, normal).
__device__ __forceinline__ int fine_bin(double s) {
  unsigned long long b = (unsigned long long)__double_as_longlong(s);
  int e = (int)((b >> 52) & 0x7FF) - 1022;                   // s = mant 2^e, mant in [1/2, 1)
  double mant = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFull) |
                                                 0x3FE0000000000000ull));
  // mant and both edges share the exponent of [1/2, 1): compare their mantissa bits
  const unsigned long long mb = (unsigned long long)__double_as_longlong(mant) & 0x000FFFFFFFFFFFFFull;
  const unsigned long long e1 = (unsigned long long)__double_as_longlong(0x1.428a2f98d728bp-1) & 0x000FFFFFFFFFFFFFull;
  const unsigned long long e2 = (unsigned long long)__double_as_longlong(0x1.965fea53d6e3dp-1) & 0x000FFFFFFFFFFFFFull;
  int t = 3 * e + (mb >= e1 ? 1 : 0) + (mb >= e2 ? 1 : 0);
  t -= kTMin;
  return t < 0 ? 0 : (t > kNFine - 1 ? kNFine - 1 : t);
}

// Cell index of a coordinate along one axis of an instance grid; periodic axes wrap.
__device__ __forceinline__ int axis_cell(const GridDev& g, int a, double v) {
  double t = floor((v - g.lo[a]) * g.inv[a]);
  int d = g.dim[a];
  if (g.box[a] > 0.0) {
    t = fmin(fmax(t, -1e15), 1e15);
    long long k = (long long)t;
    k %= d;
    if (k < 0) k += d;
    return (int)k;
  }
  return t < 0.0 ? 0 : (t >= (double)d ? d - 1 : (int)t);
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al. (SC'11): 10 rounds of two 32x32 products, counter permutation
// (hi1^c1^k0, lo1, hi0^c3^k1, lo0), key bumped by the Weyl constants between rounds.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

// (k + 1/2) 2^-52 with k built from 26 bits of each word: exact, in (0, 1).
__device__ __forceinline__ double u01(uint32_t a, uint32_t b) {
  unsigned long long k = ((unsigned long long)(a >> 6) << 26) | (unsigned long long)(b >> 6);
  return (double)(2ull * k + 1ull) * 0x1p-53;   // = (k + 1/2) 2^-52, exactly
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ double warp_incl_scan(double v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = __dadd_rn(v, t);
  }
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void set_status(StateDev* st, unsigned bits) {
  atomicOr(&st->status, bits);
}

}  // namespace gd
