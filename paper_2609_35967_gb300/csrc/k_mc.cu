// k_mc.cu -- pair rates, controller bins, interval choice, event sampling and audit
// (Sect. 2.5.1-2.5.3).  Rate kernel and sampler share one pair function and one warp
// scan, so lambda*_i used for the interval and for the first waiting time is the same
// number.
//
// Work mapping: a warp takes 32 consecutive ranks.  Per-particle FP64 work (gas disk,
// Stokes numbers, fragment moments, Philox draws, logs) runs lane = particle; the K
// pair evaluations of each particle run lane = slot (S = ceil(K/32) slots per lane),
// reading one coalesced neighbour row and gathering frozen partner snapshots that sit
// nearby in cell order.
#include <climits>

#include "gd_ctx.h"
#include "gd_physics.cuh"

namespace gd {

constexpr unsigned FULLM = 0xffffffffu;

struct McArgs {
  long long N;
  int K, n_inst;
  const long long* off;
  const InstDev* P;
  StateDev* st;
  BinsDev* bins;
  const Pos64* pos64;
  const Snap64* snap64;
  const float4* snap32;
  const double* Mr;
  const double* V;
  const int* nbr;
  const int* perm;
  double* lam;
  double* chan_out;
  double* s_out;
  int* ev_count;
  unsigned* ev_hash;
  int* near_out;
  long long max_events;
  unsigned long long* work;   // sampler: next chunk of 32 ranks (zeroed before the launch)
  const float4* gx;           // mixed form: FP32 (R, Z, M) and the fine bin of each rank
  const float* pref32;        // mixed form: FP32 rate prefactor of each rank
  void* contrib;              // rank order: fine-bin contribution of each particle (rate kernel)
  int* redo;                  // mixed form: ranks whose rates or sampling are redone in FP64
  unsigned long long* redo_n; //   (their number; zeroed before the launch)
  const int* list;            // FP64 list mode: the ranks to process
  const unsigned long long* list_n;
  double* MJ;                 // caller order: M_i times the realised sum of |ln s'/s| (sampler)
  double* part;               // per-tile fine-bin partial sums [kBinQ][kNFine][n_tiles]
  long long n_tiles;
  const int* unit_r;          // spatial groups: unit of each rank (nullptr: the unit is the instance)
  const int* act;             // spatial groups: the round's ranks (rate kernel and sampler take only
  const unsigned long long* act_n;   //   these; nullptr: every rank)
  const int* unit_inst;       // spatial groups: instance of each unit
  const int* heavy;           // sampler: particles expecting more than kHeavy events, one warp each
  const unsigned long long* heavy_n; //   first (their number; nullptr: no such list)
  // mixed form: the heavy particles' event logs and the deferred FP64 settlement (nullptr: none)
  int4* dlog;
  long long dlog_cap;
  unsigned long long* dctr;   // [3]: log entries reserved, particles deferred, state entries reserved
  DeferRec* defer;
  int defer_cap;
  DState* dstate;
  long long dstate_cap;
};

// Particles expecting more events than this in an interval (lambda*_i dt_exe) are sampled one
// per warp ahead of the chunks of 32: their long serial event chains start first and never
// share a warp with another chain.
constexpr double kHeavy = 16.0;

// Per-particle quantities that do not depend on the live diameter.  The pair parameters
// are held in the pair precision T, so the mixed form converts them once per particle.
template <typename T>
struct Fixed {
  T gst, e2, e1, zo, cs, cB, Vg2, tRe, vfrag, m0, smin;
  T ferr;             // mixed form: common relative error bound of the FP32 gas constants
  T prefT;            // the prefactor in the pair precision
  double pref;        // lambda = pref * (pair rate in kernel units)
  double rho_s, s_min, M;
  double k6;          // 6 / (pi rho_s): s^3 = k6 m
  double mk;          // pi rho_s / 6: m = mk s^3
  int mode;
};

template <typename T>
__device__ __forceinline__ Fixed<T> make_fixed(const InstDev& P, const Gas& g, double V, double M, int K) {
  Fixed<T> f;
  f.gst = g.gst;
  f.e2 = 2.0 * g.eta * g.R * g.Om;
  f.e1 = g.eta * g.R * g.Om;
  f.zo = g.Z * g.Om;
  f.cs = g.cs;
  f.cB = 8.0 * kKB * g.T / kPi;
  f.Vg2 = 1.5 * P.alpha * g.cs * g.cs;
  f.tRe = 1.0 / sqrt(g.Re);
  f.vfrag = P.v_frag;
  f.m0 = P.m0;
  f.smin = P.s_min;
  f.ferr = (T)0;
  f.pref = rate_prefactor(P, V, K, sizeof(T) == 4);
  f.prefT = (T)f.pref;
  f.rho_s = P.rho_s;
  f.s_min = P.s_min;
  f.M = M;
  f.k6 = 6.0 / (kPi * P.rho_s);
  f.mk = kPi * P.rho_s / 6.0;
  f.mode = P.kernel_mode;
  return f;
}

// Mixed form: the same quantities in FP32 from the particle's FP32 gas coordinates
// (R, Z, M, fine bin) and FP32 prefactor, both written once per build; they only feed FP32
// pair arithmetic.  Omega = sqrt(GM/R)/R keeps R^3 out of the FP32 range, and
// 1 - R/r = Z^2/(r (r + R)) avoids the cancellation of the literal form.
// ferr bounds the relative error these constants share, counted operation by operation
// from R and Z rounded once (u each) with the documented ulp bounds of expf (2) and rsqrtf
// (2) and 8 ulp taken for powf: the Stokes factor (15 + 27.5 v) u with v the vertical
// exponent (its own error 27.5 u amplified v times by exp), Re^-1/2 (27 + 14 v) u, c_s 6 u,
// V_g^2 14.5 u, the drift speeds 5 u plus eta's (21 |A| + 7 |B|) / |A + B| u, A and B its two
// terms, and 1.5 u per unit of |p|, |q| from the radius ratio; the largest, doubled.
__device__ __forceinline__ Fixed<float> make_fixed_f32(const InstDev& P, float4 gx, float pref) {
  const float R = gx.x, Z = gx.y;
  const float r = sqrtf(R * R + Z * Z);
  const float Om = sqrtf(P.f_GM / R) / R;
  const float xr = R / P.f_r0;
  const float T = P.f_T0 * powf(xr, P.f_q);
  const float cs = sqrtf((float)(kKB / (kMu * kMH)) * T);
  const float H = cs / Om;
  const float h = H / R;
  const float Sigma = P.f_sigma0 * powf(xr, P.f_p);
  const float omr = Z * Z / (r * (r + R));
  const float vert = omr / (h * h);
  const float rho = Sigma / (2.5066283f * H) * expf(-vert);
  const float eA = (P.f_p + 0.5f * P.f_q - 1.5f) * h * h, eB = P.f_q * omr;
  const float eta = -0.5f * (eA + eB);
  const float numol = 0.5f * 1.5957691f * cs * ((float)(kMu * kMH / kSigH2) / rho);
  Fixed<float> f;
  f.gst = 3.14159265f * P.f_rho_s / (4.0f * Sigma) * expf(vert);
  f.e2 = 2.0f * eta * R * Om;
  f.e1 = eta * R * Om;
  f.zo = Z * Om;
  f.cs = cs;
  f.cB = (float)(8.0 * kKB / kPi) * T;
  f.Vg2 = 1.5f * P.f_alpha * cs * cs;
  f.tRe = rsqrtf(P.f_alpha * cs * H / numol);
  f.vfrag = P.f_vfrag;
  f.m0 = P.f_m0;
  f.smin = P.f_smin;
  {
    const float pw = 1.5f * fmaxf(fabsf(P.f_p), fabsf(P.f_q));
    const float fe_eta = __fdividef(21.f * fabsf(eA) + 7.f * fabsf(eB), fmaxf(fabsf(eA + eB), 1e-30f)) + 6.f;
    const float fe = fmaxf(fe_eta, 27.f + 28.f * vert) + pw;
    f.ferr = 2.f * fe * kU32;
  }
  f.prefT = pref;
  f.pref = (double)pref;
  f.rho_s = P.rho_s;
  f.s_min = P.s_min;
  f.M = (double)gx.z;
  f.k6 = P.k6;
  f.mk = P.mk;
  f.mode = P.kernel_mode;
  return f;
}

// Mixed form from FP64-accurate constants: the FP64 fixed part rounded once to FP32, so the
// common relative error of the gas constants is their rounding (u/2 each; 2u is taken).
// The sampler uses it for particles that expect many events, whose many decisions it makes
// far easier to certify.
__device__ __forceinline__ Fixed<float> fixed_f32_of(const Fixed<double>& d, float pref32) {
  Fixed<float> f;
  f.gst = (float)d.gst; f.e2 = (float)d.e2; f.e1 = (float)d.e1; f.zo = (float)d.zo;
  f.cs = (float)d.cs; f.cB = (float)d.cB; f.Vg2 = (float)d.Vg2; f.tRe = (float)d.tRe;
  f.vfrag = (float)d.vfrag; f.m0 = (float)d.m0; f.smin = (float)d.smin;
  f.ferr = 2.f * kU32;
  f.prefT = pref32;
  f.pref = (double)pref32;
  f.rho_s = d.rho_s; f.s_min = d.s_min; f.M = d.M; f.k6 = d.k6; f.mk = d.mk;
  f.mode = d.mode;
  return f;
}

// The gas at a particle from its search coordinates (Pos64): the 2D radial-polar model
// holds (R, Z, 0); the others hold positions whose R and Z the gas disk reads directly
// (the vertically integrated models have Z = 0, the midplane).
__device__ __forceinline__ Gas gas_of(const InstDev& P, const Pos64& p) {
  return P.model == GD_MODEL_RZ ? gas_RZ(P, p.x, p.y) : gas_at(P, p.x, p.y, p.z);
}

// <J>, <J^2> of a fragmentation in FP32 (mixed form; they only feed the bin moments).
__device__ __forceinline__ void frag_moments_f32(float s_i, float s_min, float& j1, float& j2) {
  const float a = sqrtf(s_min / s_i);
  if (!(a < 1.0f)) { j1 = 0.0f; j2 = 0.0f; return; }
  const float dd = 1.0f - a;
  if (dd < 1e-2f) {
    j1 = dd * (1.0f + dd * (1.0f / 3.0f + dd * (1.0f / 6.0f + dd * (1.0f / 10.0f))));
    j2 = dd * dd * (4.0f / 3.0f + dd * (1.0f + dd * (11.0f / 15.0f + dd * (5.0f / 9.0f))));
    return;
  }
  const float la = logf(a);
  j1 = 2.0f * (1.0f - a + a * la) / (1.0f - a);
  j2 = 4.0f * (2.0f - a * la * la + 2.0f * a * la - 2.0f * a) / (1.0f - a);
}

// Mixed-form query from the FP32 diameter and mass with the IEEE quotient: the rate kernel
// and the sampler's first evaluation of a particle both build it here, so both see the same
// pair rates.
__device__ __forceinline__ Query<float> live_query_f32(const Fixed<float>& f, float sf, float mf) {
  Query<float> q;
  const float St = f.gst * sf;
  const float bi = 1.0f / (1.0f + St * St);
  q.s = sf; q.m = mf; q.inv_m = 1.0f / mf;
  q.St = St;
  q.ai = St * bi;
  q.bi = bi;
  q.hi = St < 0.5f ? St : 0.5f;
  q.g = f.gst;
  q.e2 = f.e2; q.e1 = f.e1; q.zo = f.zo;
  q.cs = f.cs; q.cB = f.cB; q.Vg2 = f.Vg2; q.tRe = f.tRe;
  q.vfrag = f.vfrag; q.m0 = f.m0;
  q.ferr = f.ferr;
  q.mode = f.mode;
  return q;
}

// Query of a live particle (s, m) from the fixed part.  FP64 form: FP64 throughout; mixed
// form: FP32 from the rounded s and m.
template <typename T>
__device__ __forceinline__ Query<T> live_query(const Fixed<T>& f, double s, double m) {
  if constexpr (sizeof(T) == 8) {
    Query<T> q;
    double St = f.gst * s;
    q.s = s; q.m = m; q.inv_m = 1.0 / m;
    q.St = St;
    q.ai = St / (1.0 + St * St);
    q.bi = 1.0 / (1.0 + St * St);
    q.hi = St < 0.5 ? St : 0.5;
    q.g = f.gst;
    q.e2 = f.e2; q.e1 = f.e1; q.zo = f.zo;
    q.cs = f.cs; q.cB = f.cB; q.Vg2 = f.Vg2; q.tRe = f.tRe;
    q.vfrag = f.vfrag; q.m0 = f.m0;
    q.ferr = 0.0;
    q.mode = f.mode;
    return q;
  } else {
    return live_query_f32(f, (float)s, (float)m);
  }
}

// Mixed-form query from the FP32 diameter and mass.
__device__ __forceinline__ Query<float> live_query_f(const Fixed<float>& f, float sf, float mf) {
  Query<float> q;
  const float St = f.gst * sf;
  const float bi = __fdividef(1.0f, 1.0f + St * St);
  q.s = sf; q.m = mf; q.inv_m = __fdividef(1.0f, mf);
  q.St = St;
  q.ai = St * bi;
  q.bi = bi;
  q.hi = St < 0.5f ? St : 0.5f;
  q.g = f.gst;
  q.e2 = f.e2; q.e1 = f.e1; q.zo = f.zo;
  q.cs = f.cs; q.cB = f.cB; q.Vg2 = f.Vg2; q.tRe = f.tRe;
  q.vfrag = f.vfrag; q.m0 = f.m0;
  q.ferr = f.ferr;
  q.mode = f.mode;
  return q;
}

template <typename T>
__device__ __forceinline__ Query<T> shfl_query(const Query<T>& a, int src) {
  Query<T> q;
  q.s = __shfl_sync(FULLM, a.s, src); q.m = __shfl_sync(FULLM, a.m, src);
  q.inv_m = __shfl_sync(FULLM, a.inv_m, src); q.St = __shfl_sync(FULLM, a.St, src);
  q.ai = __shfl_sync(FULLM, a.ai, src); q.bi = __shfl_sync(FULLM, a.bi, src);
  q.hi = __shfl_sync(FULLM, a.hi, src); q.g = __shfl_sync(FULLM, a.g, src);
  q.e2 = __shfl_sync(FULLM, a.e2, src); q.e1 = __shfl_sync(FULLM, a.e1, src);
  q.zo = __shfl_sync(FULLM, a.zo, src); q.cs = __shfl_sync(FULLM, a.cs, src);
  q.cB = __shfl_sync(FULLM, a.cB, src); q.Vg2 = __shfl_sync(FULLM, a.Vg2, src);
  q.tRe = __shfl_sync(FULLM, a.tRe, src); q.vfrag = __shfl_sync(FULLM, a.vfrag, src);
  q.m0 = __shfl_sync(FULLM, a.m0, src); q.mode = __shfl_sync(FULLM, a.mode, src);
  q.ferr = __shfl_sync(FULLM, a.ferr, src);
  return q;
}

template <typename T>
__device__ __forceinline__ Fixed<T> shfl_fixed(const Fixed<T>& a, int src) {
  Fixed<T> f;
  f.gst = __shfl_sync(FULLM, a.gst, src);
  f.e2 = __shfl_sync(FULLM, a.e2, src);
  f.e1 = __shfl_sync(FULLM, a.e1, src);
  f.zo = __shfl_sync(FULLM, a.zo, src);
  f.cs = __shfl_sync(FULLM, a.cs, src);
  f.cB = __shfl_sync(FULLM, a.cB, src);
  f.Vg2 = __shfl_sync(FULLM, a.Vg2, src);
  f.tRe = __shfl_sync(FULLM, a.tRe, src);
  f.vfrag = __shfl_sync(FULLM, a.vfrag, src);
  f.m0 = __shfl_sync(FULLM, a.m0, src);
  f.smin = __shfl_sync(FULLM, a.smin, src);
  f.ferr = __shfl_sync(FULLM, a.ferr, src);
  f.prefT = __shfl_sync(FULLM, a.prefT, src);
  f.pref = __shfl_sync(FULLM, a.pref, src);
  f.rho_s = __shfl_sync(FULLM, a.rho_s, src);
  f.s_min = __shfl_sync(FULLM, a.s_min, src);
  f.M = __shfl_sync(FULLM, a.M, src);
  f.k6 = __shfl_sync(FULLM, a.k6, src);
  f.mk = __shfl_sync(FULLM, a.mk, src);
  f.mode = __shfl_sync(FULLM, a.mode, src);
  return f;
}

// Partner snapshot in the pair precision.
template <typename T> struct Partner { T s, m, Nq, inv_m; };

template <typename T>
__device__ __forceinline__ Partner<T> load_partner(const McArgs& A, int j) {
  Partner<T> p;
  if constexpr (sizeof(T) == 8) {
    const double2* pp = reinterpret_cast<const double2*>(A.snap64 + j);
    double2 a = __ldg(pp), b = __ldg(pp + 1);
    p.s = a.x; p.m = a.y; p.Nq = b.x; p.inv_m = b.y;
  } else {
    float4 v = __ldg(A.snap32 + j);
    p.s = v.x; p.m = v.y; p.Nq = v.z; p.inv_m = v.w;
  }
  return p;
}

// Neighbour ranks of the S slots of this lane in the row of rank rp (-1 past K).
template <int S>
__device__ __forceinline__ void load_row_slots(const McArgs& A, long long rp, int lane, int (&jr)[S]) {
  const int* row = A.nbr + rp * A.K;
#pragma unroll
  for (int t = 0; t < S; ++t) {
    const int k = lane * S + t;
    jr[t] = k < A.K ? __ldg(row + k) : -1;
  }
}

template <typename T, int S>
__device__ __forceinline__ void load_partners(const McArgs& A, const int (&jr)[S], Partner<T> (&pt)[S]) {
#pragma unroll
  for (int t = 0; t < S; ++t)
    if (jr[t] >= 0) pt[t] = load_partner<T>(A, jr[t]);
}

// Channel rates of the S slots of this lane from loaded partners, plus the lane's
// sequential sum in FP64 (slot-major, channel-minor).  Mixed form: a grouped pair whose
// N_coll the FP32 values cannot certify takes it from the FP64 masses (m64: the query's).
template <typename T, int S>
__device__ __forceinline__ double channels_of(const McArgs& A, const Query<T>& q, double m64, const int (&jr)[S],
                                              const Partner<T> (&pt)[S], T (&c0)[S], T (&c1)[S],
                                              PairOut<T> (&po)[S]) {
  double v = 0.0;
#pragma unroll
  for (int t = 0; t < S; ++t) {
    c0[t] = (T)0; c1[t] = (T)0;
    po[t].outcome = 0; po[t].ncoll = (T)1; po[t].psi = (T)0;
    if (jr[t] >= 0) {
      po[t] = pair_channels<T>(q, pt[t].s, pt[t].m, pt[t].Nq, pt[t].inv_m);
      if constexpr (sizeof(T) == 4) {
        if (po[t].group64) regroup64(po[t], m64, A.snap64[jr[t]].m);
      }
      c0[t] = po[t].c0;
      c1[t] = po[t].c1;
      v = __dadd_rn(v, (double)c0[t]);
      v = __dadd_rn(v, (double)c1[t]);
    }
  }
  return v;
}

template <typename T, int S>
__device__ __forceinline__ double lane_channels(const McArgs& A, const Query<T>& q, double m64, long long rp,
                                                int lane, T (&c0)[S], T (&c1)[S], int (&jr)[S], PairOut<T> (&po)[S]) {
  Partner<T> pt[S];
  load_row_slots<S>(A, rp, lane, jr);
  load_partners<T, S>(A, jr, pt);
  return channels_of<T, S>(A, q, m64, jr, pt, c0, c1, po);
}

// s^3 = 6 m / (pi rho_o).  The mixed form multiplies by the per-particle constant.
template <typename T>
__device__ __forceinline__ double cube_of(const Fixed<T>& f, double m) {
  if constexpr (sizeof(T) == 8) return 6.0 * m / (kPi * f.rho_s); else return m * f.k6;
}

// This lane's channel rates summed in FP32 (slot order), for the mixed form's FP32 prefix.
template <int S>
__device__ __forceinline__ float lane_sumf(const float (&c0)[S], const float (&c1)[S], const int (&jr)[S]) {
  float v = 0.0f;
#pragma unroll
  for (int t = 0; t < S; ++t)
    if (jr[t] >= 0) { v += c0[t]; v += c1[t]; }
  return v;
}
template <int S>
__device__ __forceinline__ float lane_sumf(const double (&)[S], const double (&)[S], const int (&)[S]) { return 0.0f; }

__device__ __forceinline__ float warp_incl_scanf(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float t = __shfl_up_sync(FULLM, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Diameter from s^3 = x.  FP64 form: cbrt.  Mixed form: the FP32 cube root y refined by
// one Newton step for y^3 = x, y <- y - (y^3 - x)/(3 y^2), with the residual in FP64 and
// the 1/(3 y^2) factor in FP32: ~1e-13 relative for a handful of FP64 instructions.
template <typename T>
__device__ __forceinline__ double diameter_of(double x) {
  if constexpr (sizeof(T) == 8) {
    return cbrt(x);
  } else {
    const float yf = cbrtf((float)x);
    const double y = (double)yf;
    const float c = (float)(y * y * y - x) * __frcp_rn(3.0f * yf * yf);
    return y - (double)c;
  }
}

// -ln U for U = (k + 1/2) 2^-52, k = (a >> 6) 2^26 + (b >> 6) (the u01 map), in FP32
// without FP64 instructions.  For U >= 1/2 it is -log1p(-(1 - U)) with 1 - U formed from
// the complement of k, so short waits keep their relative accuracy.
__device__ __forceinline__ float neg_log_u01_f32(uint32_t a, uint32_t b) {
  const uint32_t hi = a >> 6, lo = b >> 6;
  if (hi >= (1u << 25)) {
    const float v = fmaf((float)((1u << 26) - 1u - hi), 0x1p26f, (float)((1u << 26) - 1u - lo) + 0.5f) * 0x1p-52f;
    return -log1pf(-v);
  }
  return -logf(fmaf((float)hi, 0x1p26f, (float)lo + 0.5f) * 0x1p-52f);
}

// Waiting time -ln(U_w) / lambda*_i.  FP64 form: FP64 throughout.  Mixed form: FP32
// (lambda*_i is an FP32 sum of FP32 rates); the caller accumulates it in FP64.
template <typename T>
__device__ __forceinline__ double waiting_time(uint32_t a, uint32_t b, double lam) {
  if constexpr (sizeof(T) == 8) {
    return -log(u01(a, b)) / lam;
  } else {
    const float nl = neg_log_u01_f32(a, b);
    const float lf = (float)lam;
    if (lf > 1e-30f && lf < 1e30f) return (double)__fdividef(nl, lf);
    return (double)nl / lam;
  }
}

// ---------------------------------------------------------------- fixed-order bin sums
// Fine-bin accumulation of one warp in a fixed order: the lanes holding particles of the
// same fine bin (one match group) sum the group's values in ascending lane order, and the
// group's lowest lane adds the sums to the warp's own accumulators acc[k * kNFine + bin].
// A warp's batches come in a fixed order, so no sum depends on scheduling (no float atomics).
// fbin < 0: the lane adds nothing.
template <typename Acc, int NV>
__device__ __forceinline__ void warp_bin_add(Acc* acc, int* cnt, int fbin, const Acc (&v)[NV], int lane) {
  const int key = fbin >= 0 ? fbin : kNFine + lane;
  const unsigned grp = __match_any_sync(FULLM, key);
  const int npop = __popc(grp);
  const int nmax = (int)__reduce_max_sync(FULLM, (unsigned)npop);
  Acc sum[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) sum[k] = (Acc)0;
  unsigned m = grp;
  for (int i = 0; i < nmax; ++i) {
    const int src = m ? __ffs(m) - 1 : lane;
    m &= m - 1u;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const Acc t = __shfl_sync(FULLM, v[k], src);
      if (i < npop) sum[k] += t;
    }
  }
  if (fbin >= 0 && lane == __ffs(grp) - 1) {
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k * kNFine + fbin] += sum[k];
    if (cnt) cnt[fbin] += npop;
  }
  __syncwarp();
}

// ---------------------------------------------------------------- rate kernel
// Lane = particle (consecutive threads take consecutive ranks): each thread walks
// its own neighbour row (the row stays in L1 across the walk), evaluates the K pairs in slot
// order and sums lambda*_i and the moments sum lambda* <J>, sum lambda* <J^2> in registers
// (FP64 form: the channel rates in the oracle's order, slot by slot, remnant before debris).
// Each particle's contribution to the fine-bin sums (M, M pref sum lambda* <J>, likewise
// <J^2>, and its fine bin) is written in rank order; k_bins_tile adds them up in caller order.
// Mixed form: FP32 throughout the particle's work, from its FP32 gas coordinates, snapshot
// and prefactor.
// One particle's lambda*_i and fine-bin contribution; returns false when a pair's threshold
// decision is uncertified (mixed form).  err: mixed form, bound on the relative error of the
// FP32 lambda*_i and moments -- the pairs' absolute error bounds derr_k c_k summed and divided
// by the sums they bound (lambda*_i and both moments; the largest of the three), plus the
// FP32 sums' and the moments' roundings; 0 in the FP64 form.  A pair of nearly equal grains
// can have a large relative bound (St_i - St_j cancels in FP32) but then has a tiny rate.
template <typename T>
__device__ __forceinline__ bool rate_particle(const McArgs& A, const InstDev& P, long long r, double& lam,
                                              T (&v)[3], int& fbin, float& err) {
  Fixed<T> fx;
  Query<T> q;
  T j1, j2;
  if constexpr (sizeof(T) == 8) {
    const Pos64 p = A.pos64[r];
    const Snap64 sn = A.snap64[r];
    Gas g = gas_of(P, p);
    fx = make_fixed<double>(P, g, A.V[r], A.Mr[r], A.K);
    frag_moments(sn.s, P.s_min, j1, j2);
    q = live_query<T>(fx, sn.s, sn.m);
    fbin = fine_bin(sn.s);
  } else {
    const float4 g4 = A.gx[r];
    const float4 sn = A.snap32[r];
    fx = make_fixed_f32(P, g4, A.pref32[r]);
    frag_moments_f32(sn.x, fx.smin, j1, j2);
    q = live_query_f32(fx, sn.x, sn.y);
    fbin = __float_as_int(g4.w);
  }
  const int* row = A.nbr + r * A.K;
  const long long ci = A.chan_out ? (long long)A.perm[r] * A.K : 0;
  T tot = (T)0, la = (T)0, lb = (T)0;
  bool cert = true;
  float et = 0.0f, ea = 0.0f, eb = 0.0f;   // mixed form: absolute error bounds of the sums
  // partners loaded one slot ahead of the pair being evaluated
  int jn = __ldg(row);
  Partner<T> pn = load_partner<T>(A, jn);
  for (int k = 0; k < A.K; ++k) {
    const Partner<T> pt = pn;
    const int jn_cur = jn;
    if (k + 1 < A.K) { jn = __ldg(row + k + 1); pn = load_partner<T>(A, jn); }
    PairOut<T> po = pair_channels<T>(q, pt.s, pt.m, pt.Nq, pt.inv_m);
    if constexpr (sizeof(T) == 4) {
      if (po.group64) regroup64(po, A.snap64[r].m, A.snap64[jn_cur].m);
    }
    if constexpr (sizeof(T) == 8) { tot = __dadd_rn(tot, po.c0); tot = __dadd_rn(tot, po.c1); }
    else { tot += po.c0; tot += po.c1; cert = cert && po.cert; }
    T a, bb;
    pair_moments<T>(po, j1, j2, a, bb);
    la += a;
    lb += bb;
    if constexpr (sizeof(T) == 4) {
      et = fmaf((float)po.derr, po.c0 + po.c1, et);
      ea = fmaf((float)po.derr, a, ea);
      eb = fmaf((float)po.derr, bb, eb);
    }
    if (A.chan_out) {
      A.chan_out[(ci + k) * 2] = fx.pref * (double)po.c0;
      A.chan_out[(ci + k) * 2 + 1] = fx.pref * (double)po.c1;
    }
  }
  if constexpr (sizeof(T) == 8) {
    lam = fx.pref * tot;
    v[0] = fx.M;
    v[1] = fx.M * (fx.pref * la);
    v[2] = fx.M * (fx.pref * lb);
    err = 0.0f;
  } else {
    const float rl = tot > 0.0f ? __fdividef(et, tot) : 0.0f;
    const float ra = la > 0.0f ? __fdividef(ea, la) : 0.0f;
    const float rb = lb > 0.0f ? __fdividef(eb, lb) : 0.0f;
    err = fmaxf(rl, fmaxf(ra, rb)) * 1.0001f + (2.f * A.K + 16.f) * kU32;
    const float lf = fx.prefT * tot;
    lam = (lf > 1e-30f && lf < 1e30f) ? (double)lf : fx.pref * (double)tot;
    const float Mf = A.gx[r].z;
    v[0] = Mf;
    v[1] = Mf * (fx.prefT * la);
    v[2] = Mf * (fx.prefT * lb);
  }
  return cert;
}

template <typename T>
__device__ __forceinline__ void rates_one(const McArgs& A, const InstDev& P, long long r, int u) {
  double lam;
  T v[3];
  int fbin;
  float err;
  const bool cert = rate_particle<T>(A, P, r, lam, v, fbin, err);
  if constexpr (sizeof(T) == 8) {
    Contrib64 c;
    c.M = v[0]; c.MA = v[1]; c.MB = v[2]; c.fbin = fbin;
    static_cast<Contrib64*>(A.contrib)[r] = c;
  } else {
    static_cast<float4*>(A.contrib)[r] = make_float4(v[0], v[1], v[2], pack_ebin(err, fbin));
    // a threshold decision the FP32 values cannot certify: the particle's rates are redone
    // in FP64 (k_rates_redo)
    if (!cert) {
      A.redo[atomicAdd(A.redo_n, 1ull)] = (int)r;
      atomicAdd((unsigned long long*)&A.st[u].rate_redo, 1ull);
    }
  }
  A.lam[r] = lam;
  if (!isfinite(lam)) set_status(&A.st[u], GD_ST_NONFINITE);
}

// A grid-stride loop over the ranks (consecutive threads, consecutive ranks), filling every
// SM whatever the number of particles; with spatial groups over the round's list only.
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 4 : 6) k_rates(McArgs A) {
  const long long n = A.act ? (long long)*A.act_n : A.N;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    if (A.act) {
      const long long r = A.act[t];
      const int u = A.unit_r[r];
      rates_one<T>(A, A.P[A.unit_inst[u]], r, u);
    } else {
      const int b = inst_of(A.off, A.n_inst, t);
      rates_one<T>(A, A.P[b], t, b);
    }
  }
}

// Mixed form: the particles k_rates could not certify, redone in FP64 (the FP64 form's
// arithmetic), their lambda*_i and fine-bin contributions written over the FP32 ones.
__global__ void __launch_bounds__(128) k_rates_redo(McArgs A) {
  // a warp per listed particle, lane = slot: the serial FP64 pair loop of one thread would
  // make the few listed particles the kernel's whole duration
  const int lane = threadIdx.x & 31;
  const long long total = (long long)*A.list_n;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total; t += nw) {
    const long long r = A.list[t];
    const int b = inst_of(A.off, A.n_inst, r);
    const InstDev& P = A.P[b];
    const Pos64 p = A.pos64[r];
    const Snap64 sn = A.snap64[r];
    Gas g = gas_of(P, p);
    const Fixed<double> fx = make_fixed<double>(P, g, A.V[r], A.Mr[r], A.K);
    double j1, j2;
    frag_moments(sn.s, P.s_min, j1, j2);
    const Query<double> q = live_query<double>(fx, sn.s, sn.m);
    const int* row = A.nbr + r * A.K;
    const long long ci = A.chan_out ? (long long)A.perm[r] * A.K : 0;
    double tot = 0.0, la = 0.0, lb = 0.0;
    for (int k = lane; k < A.K; k += 32) {
      const Partner<double> pt = load_partner<double>(A, __ldg(row + k));
      const PairOut<double> po = pair_channels<double>(q, pt.s, pt.m, pt.Nq, pt.inv_m);
      tot += po.c0 + po.c1;
      double a, bb;
      pair_moments<double>(po, j1, j2, a, bb);
      la += a;
      lb += bb;
      if (A.chan_out) {
        A.chan_out[(ci + k) * 2] = fx.pref * po.c0;
        A.chan_out[(ci + k) * 2 + 1] = fx.pref * po.c1;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tot += __shfl_xor_sync(FULLM, tot, o);
      la += __shfl_xor_sync(FULLM, la, o);
      lb += __shfl_xor_sync(FULLM, lb, o);
    }
    if (lane == 0) {
      const double lam = fx.pref * tot;
      // FP64 values rounded to FP32: half a unit of their last place
      static_cast<float4*>(A.contrib)[r] =
          make_float4((float)fx.M, (float)(fx.M * (fx.pref * la)), (float)(fx.M * (fx.pref * lb)),
                      pack_ebin(2.f * kU32, fine_bin(sn.s)));
      A.lam[r] = lam;
      if (!isfinite(lam)) set_status(&A.st[A.unit_r ? A.unit_r[r] : b], GD_ST_NONFINITE);
    }
  }
}

// Fine-bin partial sums of one tile of CALLER indices (count, M, M A, M B), each particle's
// contribution gathered from its rank: the rank order inside a cell follows the counting
// sort's atomics, the caller order does not, so the sums are the same in every run.  Warps
// add in the fixed order of warp_bin_add (FP64 form in FP64, mixed form in FP32), the warps'
// sums are added in warp order in FP64.
template <typename T>
__global__ void __launch_bounds__(128) k_bins_tile(TileMap tm, const int* __restrict__ rank_of,
                                                   const void* __restrict__ contrib, double* part,
                                                   long long n_tiles, const int* __restrict__ gperm,
                                                   const StateDev* __restrict__ st) {
  constexpr int NW = 4;
  __shared__ T acc[NW][3 * kNFine];
  __shared__ int cnt[NW][kNFine];
  __shared__ unsigned emax[kNFine];   // bits of non-negative floats: their order as integers
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int b;
  long long lo, hi;
  // grouped: tiles of units (read through gperm), past the last tile or of an idle unit: none
  if (!tile_range(tm, blockIdx.x, b, lo, hi)) return;
  if (gperm && !st[b].active) return;
  for (int t = threadIdx.x; t < NW * 3 * kNFine; t += blockDim.x) (&acc[0][0])[t] = (T)0;
  for (int t = threadIdx.x; t < NW * kNFine; t += blockDim.x) (&cnt[0][0])[t] = 0;
  for (int t = threadIdx.x; t < kNFine; t += blockDim.x) emax[t] = 0u;
  __syncthreads();
  for (long long base = lo; base < hi; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    int fb = -1;
    T v[3] = {(T)0, (T)0, (T)0};
    if (i < hi) {
      const int r = rank_of[gperm ? gperm[i] : i];
      if constexpr (sizeof(T) == 8) {
        const Contrib64 c = static_cast<const Contrib64*>(contrib)[r];
        v[0] = c.M; v[1] = c.MA; v[2] = c.MB;
        fb = (int)c.fbin;
      } else {
        const float4 c = static_cast<const float4*>(contrib)[r];
        v[0] = c.x; v[1] = c.y; v[2] = c.z;
        fb = ebin_bin(c.w);
        atomicMax(&emax[fb], __float_as_uint(ebin_err(c.w)));   // a maximum: any order
      }
    }
    warp_bin_add<T, 3>(&acc[w][0], &cnt[w][0], fb, v, lane);
  }
  __syncthreads();
  for (int f = threadIdx.x; f < kNFine; f += blockDim.x) {
    part[(5LL * kNFine + f) * n_tiles + blockIdx.x] = (double)__uint_as_float(emax[f]);
    double c = 0.0, sM = 0.0, sA = 0.0, sB = 0.0;
    for (int ww = 0; ww < NW; ++ww) {
      c += (double)cnt[ww][f];
      sM += (double)acc[ww][f];
      sA += (double)acc[ww][kNFine + f];
      sB += (double)acc[ww][2 * kNFine + f];
    }
    part[(0LL * kNFine + f) * n_tiles + blockIdx.x] = c;
    part[(1LL * kNFine + f) * n_tiles + blockIdx.x] = sM;
    part[(2LL * kNFine + f) * n_tiles + blockIdx.x] = sA;
    part[(3LL * kNFine + f) * n_tiles + blockIdx.x] = sB;
  }
}

// Fine-bin sums of M_i J_i of the interval (the realised |ln s'/s| of each particle's
// events, caller order) per tile of caller indices, in the same fixed order; quantity 4 of
// the tile partials.  The fine bin is that of the particle's size at the interval start.
template <bool kMixed>
__global__ void __launch_bounds__(128) k_jbins(TileMap tm, const int* __restrict__ rank_of,
                                               const void* __restrict__ contrib, const double* __restrict__ MJ,
                                               double* part, long long n_tiles, const int* __restrict__ gperm,
                                               const StateDev* __restrict__ st) {
  constexpr int NW = 4;
  __shared__ double acc[NW][kNFine];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int b;
  long long lo, hi;
  if (!tile_range(tm, blockIdx.x, b, lo, hi)) return;
  if (gperm && !st[b].active) return;
  for (int t = threadIdx.x; t < NW * kNFine; t += blockDim.x) (&acc[0][0])[t] = 0.0;
  __syncthreads();
  for (long long base = lo; base < hi; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    double v[1] = {0.0};
    int fb = -1;
    if (i < hi) {
      const long long ci = gperm ? gperm[i] : i;
      v[0] = MJ[ci];
      if (v[0] != 0.0) {
        const int r = rank_of[ci];
        if (kMixed) fb = ebin_bin(static_cast<const float4*>(contrib)[r].w);
        else fb = (int)static_cast<const Contrib64*>(contrib)[r].fbin;
      }
    }
    warp_bin_add<double, 1>(&acc[w][0], nullptr, fb, v, lane);
  }
  __syncthreads();
  for (int f = threadIdx.x; f < kNFine; f += blockDim.x) {
    double sJ = 0.0;
    for (int ww = 0; ww < NW; ++ww) sJ += acc[ww][f];
    part[(4LL * kNFine + f) * n_tiles + blockIdx.x] = sJ;
  }
}

// The size spectrum: sum of M_i per fine bin of the current diameter s_i, per tile of caller
// indices in the fixed order of warp_bin_add; quantity 6 of the tile partials.
__global__ void __launch_bounds__(128) k_spec_tile(TileMap tm, const double* __restrict__ s,
                                                   const double* __restrict__ M, double* part, long long n_tiles) {
  constexpr int NW = 4;
  __shared__ double acc[NW][kNFine];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < NW * kNFine; t += blockDim.x) (&acc[0][0])[t] = 0.0;
  __syncthreads();
  int b;
  long long lo, hi;
  tile_range(tm, blockIdx.x, b, lo, hi);
  for (long long base = lo; base < hi; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    double v[1] = {0.0};
    int fb = -1;
    if (i < hi) { v[0] = M[i]; fb = fine_bin(s[i]); }
    warp_bin_add<double, 1>(&acc[w][0], nullptr, fb, v, lane);
  }
  __syncthreads();
  for (int f = threadIdx.x; f < kNFine; f += blockDim.x) {
    double sp = 0.0;
    for (int ww = 0; ww < NW; ++ww) sp += acc[ww][f];
    part[(6LL * kNFine + f) * n_tiles + blockIdx.x] = sp;
  }
}

// Per-instance fine-bin sums from the tile partials, in a fixed order: one warp per
// (quantity, bin); lane l adds the instance's tiles l, l + 32, ... in order, then the lanes'
// sums meet in a fixed butterfly (quantity 5, an error bound, takes the maximum instead).
// Quantities q0 .. q0 + nq - 1 of BinsDev (cnt, sM, sA, sB, sJ, sE) except skip_q are
// overwritten.
__global__ void k_bins_reduce(const long long* __restrict__ tile_off, const double* __restrict__ part,
                              long long n_tiles, int q0, int nq, int skip_q, BinsDev* bins,
                              const InstDev* __restrict__ P, const StateDev* __restrict__ st) {
  // blocks over units (st given: idle units are skipped), or over instances whose sums go to
  // their first unit (P given)
  const int b = blockIdx.x;
  if (st && !st[b].active) return;
  const int lane = threadIdx.x & 31;
  const int pair = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (pair >= nq * kNFine) return;
  const int q = q0 + pair / kNFine, f = pair % kNFine;
  if (q == skip_q) return;
  const double* src = part + ((long long)q * kNFine + f) * n_tiles;
  double v = 0.0;
  if (q == 5) {
    for (long long t = tile_off[b] + lane; t < tile_off[b + 1]; t += 32) v = fmax(v, src[t]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  } else {
    for (long long t = tile_off[b] + lane; t < tile_off[b + 1]; t += 32) v += src[t];
    v = warp_sum(v);
  }
  if (lane == 0) (&bins[P ? P[b].unit0 : b].cnt[0])[q * kNFine + f] = v;
}

// ---------------------------------------------------------------- interval choice
// One block per unit (an instance, or one spatial group of it): the fine bins are read into
// shared memory by all threads, then one thread merges them into controller bins (>= max(K, 64) particles, ascending, a
// remainder joins the previous bin), forms A_b and B_b in one ascending pass, and halves
// dt_coll with the exact tick count of the time left.  A near tie of the interval choice is
// a binding moment within 1e-10 (FP64 form) of a halving edge; in the mixed form within
// 1.5 times the error bound of the binding bin's FP32 moments (their largest per-particle
// bound plus 64 u of summation), at least 2e-5.
__global__ void k_interval(const InstDev* __restrict__ P, StateDev* st, BinsDev* bins, int n_units,
                           const int* __restrict__ unit_inst, int K, int no_audit, int mixed) {
  __shared__ double cnt[kNFine], sM[kNFine], sA[kNFine], sB[kNFine], sE[kNFine];
  __shared__ double gM[kNFine], gA[kNFine], gB[kNFine], gE[kNFine];
  __shared__ int gid[kNFine];
  const int b = blockIdx.x;    // the unit
  if (b >= n_units) return;
  const InstDev& p = P[unit_inst ? unit_inst[b] : b];
  StateDev& S = st[b];
  if (p.n_sg > 1 && !S.active) {
    // a spatial group in the middle of its interval: idle in this round
    if (threadIdx.x == 0) { S.dt_exe = 0.0; S.events = 0; }
    return;
  }
  BinsDev& Bn = bins[b];
  for (int f = threadIdx.x; f < kNFine; f += blockDim.x) {
    cnt[f] = Bn.cnt[f]; sM[f] = Bn.sM[f]; sA[f] = Bn.sA[f]; sB[f] = Bn.sB[f]; sE[f] = Bn.sE[f];
    gM[f] = 0.0; gA[f] = 0.0; gB[f] = 0.0; gE[f] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double thr = K > 64 ? K : 64;
  int ng = 0;
  double acc = 0.0;
  for (int f = 0; f < kNFine; ++f) {
    gid[f] = -1;
    if (cnt[f] == 0.0) continue;
    gid[f] = ng;
    acc += cnt[f];
    if (acc >= thr) { ng++; acc = 0.0; }
  }
  if (acc > 0.0) {
    if (ng > 0) { for (int f = 0; f < kNFine; ++f) if (gid[f] == ng) gid[f] = ng - 1; }
    else ng = 1;
  }
  for (int f = 0; f < kNFine; ++f) {
    const int g = gid[f];
    if (g < 0) continue;
    gM[g] += sM[f]; gA[g] += sA[f]; gB[g] += sB[f];
    gE[g] = fmax(gE[g], sE[f]);
  }
  for (int f = 0; f < kNFine; ++f) Bn.gid[f] = gid[f];
  Bn.ngroups = ng;
  const double C = (p.audit && !no_audit) ? S.C : 1.0;
  const double dtc = S.tau > 0.0 ? S.tau : p.dt_coll;
  if (S.hold && S.remain_ticks <= 0) {
    // a bounded collision step (gd_collide) that is used up: idle until the next one
    S.dt_exe = 0.0;
    S.events = 0;
    return;
  }
  if (S.remain_ticks <= 0) S.remain_ticks = 1LL << 60;
  const double remain = ldexp((double)S.remain_ticks, -60) * dtc;
  const double dt_cap = remain < p.dt_fn_max ? remain : p.dt_fn_max;
  double dt_ab = HUGE_VAL, e_bind = 0.0;
  for (int g = 0; g < kNFine; ++g) { Bn.gA[g] = 0.0; Bn.gB[g] = 0.0; }
  for (int g = 0; g < ng; ++g) {
    const double A = gA[g] / gM[g], Bm = gB[g] / gM[g];
    Bn.gA[g] = A;
    Bn.gB[g] = Bm;
    if (A > 0.0) { const double t = p.eps * C / A; if (t < dt_ab) { dt_ab = t; e_bind = gE[g]; } }
    if (Bm > 0.0) { const double t = p.eps * p.eps * C * C / Bm; if (t < dt_ab) { dt_ab = t; e_bind = gE[g]; } }
  }
  const double tie = mixed ? fmax(2e-5, 1.5 * (e_bind + 64.0 * 0x1p-24)) : 1e-10;
  const double dt_req = dt_ab < dt_cap ? dt_ab : dt_cap;
  double dt = dtc;
  int k = 0;
  while (k < 60 && (dt > dt_req || (1LL << (60 - k)) > S.remain_ticks)) { dt = 0.5 * dt; ++k; }
  if (dt > dt_req) S.status |= GD_ST_DT_FLOOR;
  if (dt_ab <= dt_cap * (1.0 + tie) &&
      (fabs(dt - dt_ab) <= tie * dt_ab || fabs(2.0 * dt - dt_ab) <= tie * dt_ab))
    S.near_dt++;
  S.n_groups = ng;
  if (p.n_sg > 1) {
    // a spatial group: the level is its request, k_schedule decides and commits
    S.dt_req = dt_req;
    S.k_req = k;
    return;
  }
  S.dt_req = dt_req;
  S.dt_exe = dt;
  S.level = k;
  S.k_req = k;
  S.remain_ticks -= 1LL << (60 - k);
  if (S.remain_ticks == 0 && !S.hold) S.remain_ticks = 1LL << 60;
  S.dt_remain = ldexp((double)S.remain_ticks, -60) * dtc;
  S.interval_cur = S.interval_next;
  S.interval_next = S.interval_next + 1;
  S.events = 0;
  S.intervals++;
}

// ---------------------------------------------------------------- sampler
// Mixed form: one event decision settled with the FP64 form's arithmetic (warp-cooperative,
// lane = slot; called by the whole warp): the FP64 gas disk at the particle, its channel
// rates at the current state (s, m) against the frozen partners, their inclusive prefix and
// lambda*_i; with choose, the channel the FP64 prefix selects for the draw (uw0, uw1) and its
// partner, outcome, N_coll and psi.  Near ties are counted at the FP64 tolerance (1e-10).
// Rare (only decisions the FP32 values cannot certify), so it is kept out of line.
// lambda*_i of rank r at its snapshot state as the FP64 rate kernel forms it -- its pair
// terms summed in slot order -- with the pairs evaluated by the whole warp (lane = slot) and
// the sum taken in that order through shuffles (every lane returns it).
template <int S>
__device__ __forceinline__ double lam0_fp64(const McArgs& A, long long r, int lane) {
  const int b = inst_of(A.off, A.n_inst, r);
  const InstDev& P = A.P[b];
  const Snap64 sn = A.snap64[r];
  const Gas g = gas_of(P, A.pos64[r]);
  const Fixed<double> f = make_fixed<double>(P, g, A.V[r], A.Mr[r], A.K);
  const Query<double> q = live_query<double>(f, sn.s, sn.m);
  double c0[S], c1[S];
  int jr[S];
  PairOut<double> po[S];
  lane_channels<double, S>(A, q, sn.m, r, lane, c0, c1, jr, po);
  double tot = 0.0;
  for (int src = 0; src < 32; ++src) {
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const double a = __shfl_sync(FULLM, c0[t], src);
      const double bb = __shfl_sync(FULLM, c1[t], src);
      if (src * S + t < A.K) {
        tot = __dadd_rn(tot, a);
        tot = __dadd_rn(tot, bb);
      }
    }
  }
  return f.pref * tot;
}

struct Fp64Pick {
  int chosen, j, outcome, near;
  int near_pair;      // the near ties of the pairs' thresholds alone (part of near)
  double ncoll, psi, lam;
};

template <int S>
__device__ __noinline__ Fp64Pick fp64_event(const McArgs& A, long long rp, int bp, double s, double m,
                                            unsigned uw0, unsigned uw1, bool choose, int lane) {
  const InstDev& P = A.P[bp];
  Gas g = gas_of(P, A.pos64[rp]);
  const Fixed<double> f = make_fixed<double>(P, g, A.V[rp], A.Mr[rp], A.K);
  const Query<double> q = live_query<double>(f, s, m);
  double c0[S], c1[S];
  int jr[S];
  PairOut<double> po[S];
  const double v = lane_channels<double, S>(A, q, m, rp, lane, c0, c1, jr, po);
  int near = 0;
#pragma unroll
  for (int t = 0; t < S; ++t)
    if (jr[t] >= 0 && !po[t].cert) near++;
  int near_pair = near;
  const double incl = warp_incl_scan(v, lane);
  const double tot = __shfl_sync(FULLM, incl, 31);
  Fp64Pick r;
  r.lam = f.pref * tot;
  r.chosen = -1; r.j = -1; r.outcome = 0; r.ncoll = 1.0; r.psi = 0.0;
  if (choose) {
    const double target = u01(uw0, uw1) * tot;
    const double tie = 1e-10 * tot;
    double cum = __shfl_up_sync(FULLM, incl, 1);
    if (lane == 0) cum = 0.0;
    int sel = INT_MAX, lastnz = -1;
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const int k = lane * S + t;
      if (jr[t] < 0) continue;
      cum = __dadd_rn(cum, c0[t]);
      if (c0[t] > 0.0) {
        lastnz = 2 * k;
        if (fabs(target - cum) < tie) near++;
        if (sel == INT_MAX && target < cum) sel = 2 * k;
      }
      cum = __dadd_rn(cum, c1[t]);
      if (c1[t] > 0.0) {
        lastnz = 2 * k + 1;
        if (fabs(target - cum) < tie) near++;
        if (sel == INT_MAX && target < cum) sel = 2 * k + 1;
      }
    }
    int chosen = sel;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) chosen = min(chosen, __shfl_xor_sync(FULLM, chosen, o));
    if (chosen == INT_MAX) {
      int ln = lastnz;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ln = max(ln, __shfl_xor_sync(FULLM, ln, o));
      chosen = ln;
      if (lane == 0) near++;
    }
    r.chosen = chosen;
    if (chosen >= 0) {
      const int slot = chosen >> 1, owner = slot / S, tsl = slot % S;
      int jo = jr[0], oc = po[0].outcome;
      double nco = po[0].ncoll, pso = po[0].psi;
#pragma unroll
      for (int t = 1; t < S; ++t)
        if (t == tsl) { jo = jr[t]; oc = po[t].outcome; nco = po[t].ncoll; pso = po[t].psi; }
      r.j = __shfl_sync(FULLM, jo, owner);
      r.outcome = __shfl_sync(FULLM, oc, owner);
      r.ncoll = __shfl_sync(FULLM, nco, owner);
      r.psi = __shfl_sync(FULLM, pso, owner);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    near += __shfl_xor_sync(FULLM, near, o);
    near_pair += __shfl_xor_sync(FULLM, near_pair, o);
  }
  r.near = near;
  r.near_pair = near_pair;
  return r;
}

// The FP64 form's update of (s, m) by one event of outcome `outcome` on channel ch with the
// frozen partner pj (Sect. 2.5.2, Eq. frag); sset = 0: s is left to s_of_m64 (s must be set
// for a fragmentation).  Shared by the FP64 sampler and the deferred settlement so that both
// form the same states.
__device__ __forceinline__ double s_of_m64(double rho_s, double m) { return cbrt(6.0 * m / (kPi * rho_s)); }

__device__ __forceinline__ void event64(double rho_s, double s_min, unsigned k0, unsigned k1, const Snap64& pj,
                                        int ch, int outcome, double ncoll, unsigned il, unsigned iv, unsigned e,
                                        double& s, double& m, int& sset) {
  if (outcome == 0) {
    m = __fma_rn(ncoll, pj.m, m);
    sset = 0;
  } else if (outcome == 1 && ch == 0) {
    m = __fma_rn(-ncoll, pj.m, m);
    sset = 0;
  } else if (outcome == 1) {
    m = pj.m;
    s = pj.s;
    sset = 1;
  } else {
    const U4 w2 = philox(il, iv, e, 1u, k0, k1);
    const double U = u01(w2.x, w2.y);
    const double a = sqrt(s_min), bq = sqrt(s);
    const double xr = __fma_rn(U, bq - a, a);
    s = xr * xr;
    m = kPi * rho_s * s * s * s / 6.0;
    sset = 1;
  }
}

// Heavy particles with fewer logged events than this keep the in-line FP64 replay.
constexpr int kDeferMin = 32;

// Work items are taken from a counter: first the heavy particles (more than kHeavy events
// expected), one per warp, then chunks of 32 ranks (lane = particle): event counts are
// heavy-tailed, so a static assignment would leave warps idle behind the busiest chunks.
// Each lane draws its particle's first waiting time from lambda*_i; the particles with an
// event are then taken one at a time by the whole warp (lane = slot): the channel rates, the
// partner channel from their inclusive prefix (warp scan), the outcome, the own rates
// refreshed against the frozen partners, the next waiting time, until the waiting times
// pass dt_exe.
//
// FP64 form: FP64 throughout.  A draw within 1e-10 of a channel boundary or of dt_exe, and a
// pair within 1e-10 of an outcome, grouping or turbulence-regime threshold, is counted as a
// near tie of the particle.
//
// Mixed form: FP32 channel rates, FP64 masses, fragment sizes and waiting-time sums.  Every
// decision is certified to be the one the FP64 form takes, from error bounds:
//  * each pair's thresholds (pair_channels), and its channel rates within their bound derr;
//  * the FP32 prefix within eta = max derr + (2S + 7) u of the FP64 prefix (lambda*_i of the
//    rate kernel within the bound it packed with the particle's fine bin), the FP32 target
//    U_s lambda* within 1.5 u more: the channel is certified when the target lies more than
//    1.5 (2 eta + 3 u) lambda* inside it;
//  * each FP32 waiting time within eta + 8 u (the logarithm 4 u, the quotient 2 u, the
//    prefactor's rounding) of the FP64 one: the running error bound of the time sum, and the
//    decision against dt_exe certified when t + dt_w lies more than 1.5 times that bound
//    (plus 1e-14 dt_exe) from dt_exe.
// A particle with any uncertified decision writes nothing: the same warp replays it at once
// with the FP64 form's sampler (replay64, lambda*_i formed afresh with the rate kernel's FP64
// arithmetic), which writes its results.  The mixed form therefore reproduces the FP64 form's
// event sequences except where the replay meets an FP64 near tie.
// The heavy particles of the interval: lambda*_i dt_exe > kHeavy (the same product the
// sampler's chunks test), listed in any order (each is sampled on its own).
__global__ void k_heavy(McArgs A, int* __restrict__ heavy, unsigned long long* heavy_n) {
  const long long total = A.act ? (long long)*A.act_n : A.N;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = A.act ? A.act[t] : t;
    const int u = A.unit_r ? A.unit_r[r] : inst_of(A.off, A.n_inst, r);
    if (A.lam[r] * A.st[u].dt_exe > kHeavy) heavy[atomicAdd(heavy_n, 1ull)] = (int)r;
  }
}

// One work item of the sampler (a chunk of 32 particles, lane = particle, or one particle
// for the whole warp): the first waiting times, then each event particle's chain with the
// warp (lane = slot), then the results.  fresh: lambda*_i is lam_fresh, formed in FP64 by
// the caller (the replay), rather than read from the rate kernel.
template <int S>
__device__ __noinline__ void replay64(McArgs A, long long r, int lane);

template <typename T, int S>
__device__ __forceinline__ void sample_item(const McArgs& A, const int lane, const bool one, const bool fresh,
                                            const long long r, bool valid, const double lam_fresh = 0.0) {
  constexpr bool kMixed = sizeof(T) == 4;
  const float u = kU32;
  int b = 0, ub = 0;   // instance and unit (spatial group) of the particle
  double lam = 0.0, dtw = 0.0, us = 0.0, dt_exe = 0.0;
  unsigned ival = 0, i_loc = 0, key0 = 0, key1 = 0, usw0 = 0, usw1 = 0;
  bool ev = false, replay = false, deferred = false;
  int nn = 0;
  float eta_lam = 0.0f;   // mixed form: error bound of the first waiting time
  if (valid) {
    b = inst_of(A.off, A.n_inst, r);
    ub = A.unit_r ? A.unit_r[r] : b;
    dt_exe = A.st[ub].dt_exe;     // 0 for a group idle in this round: no event
    // a heavy particle of a chunk is sampled by its own warp (the list of k_heavy)
    if (!one && A.heavy_n && A.lam[r] * dt_exe > kHeavy) valid = false;
  }
  if (valid) {
    const InstDev& P = A.P[b];
    ival = (unsigned)A.st[ub].interval_cur;
    key0 = P.key0;
    key1 = P.key1;
    i_loc = (unsigned)(A.perm[r] - P.off);
    if (dt_exe > 0.0) {   // else idle: a held instance or a spatial group between rounds
      lam = fresh ? lam_fresh : A.lam[r];
      U4 w = philox(i_loc, ival, 0u, 0u, key0, key1);
      usw0 = w.z;
      usw1 = w.w;
      if constexpr (!kMixed) us = u01(w.z, w.w);
      if (lam > 0.0 && isfinite(lam)) {
        dtw = waiting_time<T>(w.x, w.y, lam);
        if constexpr (kMixed) {
          // lambda*_i's bound from the rate kernel, the logarithm, quotient and roundings
          eta_lam = ebin_err(reinterpret_cast<const float*>(A.contrib)[4 * r + 3]) + 8.f * u;
          const float dd = (float)(dtw - dt_exe);
          replay = !(fabsf(dd) > 1.5f * eta_lam * (float)dtw * 1.0001f + 1e-14f * (float)dt_exe);
        } else {
          if (fabs(dtw - dt_exe) < 1e-10 * dt_exe) nn++;
        }
        ev = !(dtw > dt_exe) && !replay;
      }
    }
  }
  unsigned emask = __ballot_sync(FULLM, ev);
  // per-lane fixed quantities of every particle of the chunk (lane = particle)
  Fixed<T> fx;
  double s_i = 1.0, m_i = 1.0;
  if (valid && ev) {
    const InstDev& P = A.P[b];
    const Snap64 sn = A.snap64[r];
    s_i = sn.s;
    m_i = sn.m;
    if constexpr (!kMixed) {
      Gas g = gas_of(P, A.pos64[r]);
      fx = make_fixed<double>(P, g, A.V[r], A.Mr[r], A.K);
    } else if (lam * dt_exe > 32.0) {
      // many events expected: FP64-accurate gas constants keep every bound of the
      // particle's many decisions near the FP32 rounding
      Gas g = gas_of(P, A.pos64[r]);
      fx = fixed_f32_of(make_fixed<double>(P, g, A.V[r], A.Mr[r], A.K), A.pref32[r]);
    } else {
      fx = make_fixed_f32(P, A.gx[r], A.pref32[r]);
    }
  } else {
    fx = Fixed<T>{};
    fx.mode = 0;
  }
  int my_e = 0;
  unsigned my_h = 0u;
  double my_MJ = 0.0, my_s = s_i;
  while (emask) {
    const int p = __ffs(emask) - 1;
    emask &= emask - 1;
    const long long rp = __shfl_sync(FULLM, r, p);
    const Fixed<T> f = shfl_fixed<T>(fx, p);
    double s = __shfl_sync(FULLM, s_i, p), m = __shfl_sync(FULLM, m_i, p);
    double t = __shfl_sync(FULLM, dtw, p);
    double u_s = __shfl_sync(FULLM, us, p);
    unsigned uw0 = __shfl_sync(FULLM, usw0, p), uw1 = __shfl_sync(FULLM, usw1, p);   // words of U_s
    const double dte = __shfl_sync(FULLM, dt_exe, p);
    const unsigned iv = __shfl_sync(FULLM, ival, p), il = __shfl_sync(FULLM, i_loc, p);
    const unsigned k0 = __shfl_sync(FULLM, key0, p), k1 = __shfl_sync(FULLM, key1, p);
    const int bp = __shfl_sync(FULLM, b, p);
    const int up = __shfl_sync(FULLM, ub, p);
    // mixed form, a heavy particle: its events are logged so that a time decision the FP32
    // bounds leave open can be settled by the deferred FP64 pass instead of a serial replay
    long long lbase = 0;
    int lcap = 0;
    if constexpr (kMixed) {
      if (one && A.dlog) {
        long long bl = 0;
        int cl = 0;
        if (lane == 0) {
          cl = (int)fmin(fmin((double)A.max_events, 2.0 * ceil(lam * dte) + 64.0), 1073741824.0);
          bl = (long long)atomicAdd(&A.dctr[0], (unsigned long long)cl);
          if (bl + cl > A.dlog_cap) cl = 0;
        }
        lbase = __shfl_sync(FULLM, bl, 0);
        lcap = __shfl_sync(FULLM, cl, 0);
      }
    }
    // mixed form: FP32 copies of per-particle constants for the per-event FP32 steps
    const float k6f = (float)f.k6, preff = f.prefT;
    float sf = (float)s;      // mixed form: the FP32 diameter the pair rates use
    bool s_stale = false;     // mixed form: s lags m after a sticking or erosion event
    // mixed form: error bound of the time sum t (FP32; the sum itself is FP64)
    float terr = (float)t * __shfl_sync(FULLM, eta_lam, p);
    const float dtef = (float)dte;
    bool unc = false;         // mixed form: an uncertified decision (warp-uniform)
    bool tunc = false;        // mixed form: that decision is the time sum's against dt_exe
    int e = 0, near_ch = 0, near_u = 0;   // per-lane ties, warp-uniform ties
    unsigned h = 0u;
    T J = (T)0;
    T c0[S], c1[S];
    int jr[S];
    PairOut<T> po[S];
    Query<T> q = live_query<T>(f, s, m);
    // the row and the frozen partners are the same for every event of the particle: loaded
    // once, so that an event's pair refresh waits on no dependent pair of loads
    Partner<T> pt[S];
    load_row_slots<S>(A, rp, lane, jr);
    load_partners<T, S>(A, jr, pt);
    double v = channels_of<T, S>(A, q, m, jr, pt, c0, c1, po);
    double incl = 0.0, tot = 0.0;
    float inclf = 0.0f, totf = 0.0f, eta = 0.0f;
    bool bad64 = false;       // mixed form: a pair's decision is uncertified at this state
    // certification (mixed) or near ties (FP64) of the pairs' threshold decisions
    // mixed form: eta bounds the relative error of the FP32 prefix and of lambda*_i -- the
    // pairs' absolute bounds derr c summed over the warp, over lambda*, plus the sums'
    // rounding
    auto pairs_checked = [&]() {
      int bad = 0;
      float de = 0.0f, cs = 0.0f;
#pragma unroll
      for (int t2 = 0; t2 < S; ++t2)
        if (jr[t2] >= 0) {
          bad += po[t2].cert ? 0 : 1;
          if constexpr (kMixed) {
            de = fmaf((float)po[t2].derr, (float)(c0[t2] + c1[t2]), de);
            cs += (float)(c0[t2] + c1[t2]);
          }
        }
      if constexpr (kMixed) {
        bad64 = __any_sync(FULLM, bad != 0);
        de = warp_sumf(de);
        cs = warp_sumf(cs);
        eta = (cs > 0.0f ? __fdividef(de, cs) * 1.0001f : 0.0f) + (2.f * S + 7.f) * u;
      } else {
        near_ch += bad;
      }
    };
    // the particle's FP64 diameter (mixed form: formed from the FP64 mass when it lags)
    auto s_exact = [&]() { return (kMixed && s_stale) ? diameter_of<T>(cube_of<T>(f, m)) : s; };
    pairs_checked();
    if constexpr (!kMixed) {
      incl = warp_incl_scan(v, lane);
      tot = __shfl_sync(FULLM, incl, 31);
    } else {
      inclf = warp_incl_scanf(lane_sumf<S>(c0, c1, jr), lane);
      totf = __shfl_sync(FULLM, inclf, 31);
    }
    for (;;) {
      if (unc) break;
      // partner channel: the first cumulative rate above U_s lambda*
      int chosen = INT_MAX, j = -1, outcome = 0;
      T ncoll_t = (T)1, psi_t = (T)0;
      bool from_po = true;
      if constexpr (kMixed) {
        bool ok = false;
        if (!bad64) {
          const float tf = fmaf((float)(uw0 >> 6), 0x1p26f, (float)(uw1 >> 6) + 0.5f) * 0x1p-52f * totf;
          const float mg = 1.5f * (2.f * eta + 3.f * u) * totf;
          float cumf = __shfl_up_sync(FULLM, inclf, 1);
          if (lane == 0) cumf = 0.0f;
          int sel = INT_MAX;
          float blo = 0.0f, bhi = 0.0f;
#pragma unroll
          for (int t2 = 0; t2 < S; ++t2) {
            const int k = lane * S + t2;
            if (jr[t2] < 0) continue;
            const float b0 = cumf;
            cumf += c0[t2];
            if (c0[t2] > 0.0f && sel == INT_MAX && tf < cumf) { sel = 2 * k; blo = b0; bhi = cumf; }
            const float b1 = cumf;
            cumf += c1[t2];
            if (c1[t2] > 0.0f && sel == INT_MAX && tf < cumf) { sel = 2 * k + 1; blo = b1; bhi = cumf; }
          }
          chosen = sel;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) chosen = min(chosen, __shfl_xor_sync(FULLM, chosen, o));
          if (chosen != INT_MAX) {
            const int own = (chosen >> 1) / S;
            const bool in = (bhi - tf > mg) && (blo == 0.0f || tf - blo > mg);
            ok = __shfl_sync(FULLM, in, own);
          }
        }
        if (!ok) {
          // the FP32 values cannot certify this choice: the FP64 form's choice at this state
          const Fp64Pick pk = fp64_event<S>(A, rp, bp, s_exact(), m, uw0, uw1, true, lane);
          near_u += pk.near;
          chosen = pk.chosen;
          j = pk.j;
          outcome = pk.outcome;
          ncoll_t = (T)pk.ncoll;
          psi_t = (T)pk.psi;
          from_po = false;
        }
      } else {
        const double target = u_s * tot;
        const double tie_ch = 1e-10 * tot;
        double cum = __shfl_up_sync(FULLM, incl, 1);
        if (lane == 0) cum = 0.0;
        int sel = INT_MAX, lastnz = -1;
#pragma unroll
        for (int t2 = 0; t2 < S; ++t2) {
          int k = lane * S + t2;
          if (jr[t2] < 0) continue;
          cum = __dadd_rn(cum, (double)c0[t2]);
          if (c0[t2] > (T)0) {
            lastnz = 2 * k;
            if (fabs(target - cum) < tie_ch) near_ch++;
            if (sel == INT_MAX && target < cum) sel = 2 * k;
          }
          cum = __dadd_rn(cum, (double)c1[t2]);
          if (c1[t2] > (T)0) {
            lastnz = 2 * k + 1;
            if (fabs(target - cum) < tie_ch) near_ch++;
            if (sel == INT_MAX && target < cum) sel = 2 * k + 1;
          }
        }
        chosen = sel;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) chosen = min(chosen, __shfl_xor_sync(FULLM, chosen, o));
        if (chosen == INT_MAX) {
          int ln = lastnz;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) ln = max(ln, __shfl_xor_sync(FULLM, ln, o));
          chosen = ln;
          near_u++;
        }
      }
      if (chosen < 0) break;
      const int ch = chosen & 1;
      if (from_po) {
        // partner data and outcome from the owning lane
        const int slot = chosen >> 1;
        const int owner = slot / S, tsl = slot % S;
        int jo = jr[0], oc = po[0].outcome;
        T nco = po[0].ncoll, pso = po[0].psi;
#pragma unroll
        for (int t2 = 1; t2 < S; ++t2)
          if (t2 == tsl) { jo = jr[t2]; oc = po[t2].outcome; nco = po[t2].ncoll; pso = po[t2].psi; }
        j = __shfl_sync(FULLM, jo, owner);
        outcome = __shfl_sync(FULLM, oc, owner);
        ncoll_t = __shfl_sync(FULLM, nco, owner);
        psi_t = __shfl_sync(FULLM, pso, owner);
      }
      if constexpr (kMixed) {
        if (e < lcap && lane == 0) A.dlog[lbase + e] = make_int4(chosen, j, outcome, (int)ncoll_t);
      }
      const double ncoll = (double)ncoll_t;
      const Snap64 pj = A.snap64[j];
      double m_new, s_new = s;
      float Jf = 0.0f;   // mixed form: |ln s'/s| of the event from the pair's FP32 psi
      if constexpr (!kMixed) {
        int sset;
        m_new = m;
        event64(f.rho_s, f.s_min, k0, k1, pj, ch, outcome, ncoll, il, iv, (unsigned)e, s_new, m_new, sset);
        if (!sset) s_new = s_of_m64(f.rho_s, m_new);
      } else if (outcome == 0) {
        // mixed form: the pair rates only need the FP32 diameter; the FP64-accurate one is
        // formed when it is needed (a fragmentation, an FP64 decision, the particle's end)
        m_new = fma(ncoll, pj.m, m);
        sf = cbrtf((float)m_new * k6f);
        s_stale = true;
        Jf = log1pf((float)ncoll_t * (float)psi_t) * (1.0f / 3.0f);
      } else if (outcome == 1 && ch == 0) {
        m_new = fma(-ncoll, pj.m, m);
        sf = cbrtf((float)m_new * k6f);
        s_stale = true;
        Jf = fabsf(log1pf(-(float)ncoll_t * (float)psi_t)) * (1.0f / 3.0f);
      } else if (outcome == 1) {
        m_new = pj.m;
        s_new = pj.s;
        sf = (float)s_new;
        s_stale = false;
        Jf = fabsf(logf((float)psi_t)) * (1.0f / 3.0f);
      } else {
        // fragmentation (Eq. frag): the size from the draw in FP64 in both forms
        U4 w2 = philox(il, iv, (unsigned)e, 1u, k0, k1);
        if (s_stale) { s = diameter_of<T>(cube_of<T>(f, m)); s_stale = false; }
        const double U = u01(w2.x, w2.y);
        const double a = sqrt(f.s_min), bq = sqrt(s);
        const double xr = a + U * (bq - a);
        s_new = xr * xr;
        m_new = f.mk * (s_new * s_new * s_new);
        sf = (float)s_new;
        Jf = 2.0f * fabsf(logf((float)(xr / bq)));
      }
      if constexpr (!kMixed) J += fabs(log(s_new / s));
      else J += Jf;
      s = s_new;
      m = m_new;
      h = h * 31u + (unsigned)(chosen + 1);
      ++e;
      if (e >= A.max_events) { if (lane == 0) set_status(&A.st[up], GD_ST_EVENT_CAP); break; }
      // the next event's draws depend only on its counter: formed before the pair refresh, so
      // that their integer work fills the refresh's latencies
      U4 w = philox(il, iv, (unsigned)e, 0u, k0, k1);
      if constexpr (!kMixed) q = live_query<T>(f, s, m);
      else q = live_query_f(f, sf, (float)m);
      v = channels_of<T, S>(A, q, m, jr, pt, c0, c1, po);
      pairs_checked();
      if constexpr (!kMixed) {
        incl = warp_incl_scan(v, lane);
        tot = __shfl_sync(FULLM, incl, 31);
      } else {
        inclf = warp_incl_scanf(lane_sumf<S>(c0, c1, jr), lane);
        totf = __shfl_sync(FULLM, inclf, 31);
      }
      double lam_now = 0.0;   // FP64 lambda*_i (FP64 form; mixed form at an uncertified state)
      if constexpr (!kMixed) {
        lam_now = f.pref * tot;
      } else if (bad64) {
        const Fp64Pick pk = fp64_event<S>(A, rp, bp, s_exact(), m, 0u, 0u, false, lane);
        near_u += pk.near;
        lam_now = pk.lam;
      }
      if (!kMixed || bad64) {
        if (!(lam_now > 0.0) || !isfinite(lam_now)) {
          if (lane == 0 && !(lam_now == 0.0)) set_status(&A.st[up], GD_ST_NONFINITE);
          break;
        }
      } else if (!(totf > 0.0f) || !isfinite(totf)) {
        if (totf == 0.0f) break;
        unc = true;
        break;
      }
      uw0 = w.z;
      uw1 = w.w;
      if constexpr (!kMixed) u_s = u01(w.z, w.w);
      double dt2;
      if constexpr (!kMixed) {
        dt2 = waiting_time<T>(w.x, w.y, lam_now);
        if (fabs((t + dt2) - dte) < 1e-10 * dte) near_u++;
      } else {
        if (bad64) {
          dt2 = waiting_time<double>(w.x, w.y, lam_now);   // exact up to FP64 rounding
        } else {
          // lambda* = pref * totf in FP32 when it is in range (the FP32 wait is formed
          // from it anyway), else in FP64
          const float lf = preff * totf;
          const float nl = neg_log_u01_f32(w.x, w.y);
          float d2;
          if (lf > 1e-30f && lf < 1e30f) { d2 = __fdividef(nl, lf); dt2 = (double)d2; }
          else { dt2 = (double)nl / (f.pref * (double)totf); d2 = (float)dt2; }
          terr = fmaf(d2, (eta + 8.f * u) * 1.0001f, terr);
        }
        // the time sum's decision: certified, or the particle is replayed in FP64 (one FP64
        // difference, compared in FP32 with a margin far above its rounding)
        const double tn = t + dt2;
        const float dd = (float)(tn - dte);
        if (!(fabsf(dd) > 1.5f * terr * 1.0001f + 1e-14f * dtef)) { unc = true; tunc = true; break; }
        if (dd > 0.0f) break;
        t = tn;
        continue;
      }
      if (t + dt2 > dte) break;
      t = t + dt2;
    }
    if constexpr (kMixed) {
      if (!unc && s_stale) s = diameter_of<T>(cube_of<T>(f, m));
    }
    // mixed form: a heavy particle whose time decision stayed open with all its events
    // logged goes to the deferred FP64 pass (its states then need e + 1 state entries)
    bool dfr = false;
    if constexpr (kMixed) {
      if (tunc && one && e >= kDeferMin && e <= lcap && A.defer) {
        int okd = 0;
        if (lane == 0) {
          const unsigned long long d = atomicAdd(&A.dctr[1], 1ull);
          if (d < (unsigned long long)A.defer_cap) {
            const unsigned long long sb = atomicAdd(&A.dctr[2], (unsigned long long)(e + 1));
            DeferRec rec;
            rec.r = rp;
            rec.lbase = lbase;
            rec.sbase = (long long)sb;
            rec.n = e;
            rec.ok = sb + (unsigned long long)(e + 1) <= (unsigned long long)A.dstate_cap ? 1 : 0;
            A.defer[d] = rec;
            okd = rec.ok;
          }
        }
        dfr = __shfl_sync(FULLM, okd, 0) != 0;
      }
    }
    int near_tot = near_ch;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) near_tot += __shfl_xor_sync(FULLM, near_tot, o);
    near_tot += near_u;
    if (lane == p) {
      replay = unc && !dfr;
      deferred = dfr;
      my_e = e; my_h = h; nn += near_tot; my_MJ = f.M * (double)J; my_s = s;
    }
  }
  if constexpr (kMixed) {
    // the particles with an uncertified decision: replayed at once by the FP64 form (the
    // whole warp, one particle after another), which writes their results
    unsigned rep = __ballot_sync(FULLM, valid && replay);
    if (valid && (replay || deferred)) atomicAdd((unsigned long long*)&A.st[ub].sample_redo, 1ull);
    while (rep) {
      const int p = __ffs(rep) - 1;
      rep &= rep - 1u;
      replay64<S>(A, __shfl_sync(FULLM, r, p), lane);
    }
  }
  if (valid) {
    if (replay || deferred) {
      // written by the FP64 replay or the deferred pass
    } else {
      const int ci = A.perm[r];
      if (my_e > 0) {
        A.s_out[ci] = my_s;
        atomicAdd((unsigned long long*)&A.st[ub].events, (unsigned long long)my_e);
      }
      A.MJ[ci] = my_MJ;
      if (nn) atomicAdd((unsigned long long*)&A.st[ub].near_draw, (unsigned long long)nn);
      if (A.ev_count) {
        A.ev_count[ci] = my_e;
        A.ev_hash[ci] = my_h;
        A.near_out[ci] = nn;
      }
    }
  }
}

// The FP64 replay of one particle the mixed pass could not certify: the FP64 form's sampler
// for that particle alone (its lambda*_i in FP64, every decision in FP64), run by the whole
// warp.  Kept out of line: rare, and its registers stay apart from the mixed pass's.
template <int S>
__device__ __noinline__ void replay64(McArgs A, long long r, int lane) {
  const double lam0 = lam0_fp64<S>(A, r, lane);
  sample_item<double, S>(A, lane, true, true, r, lane == 0, lam0);
}

// ---------------------------------------------------------------- deferred FP64 settlement
// Mixed form.  A heavy particle whose time decision the FP32 bounds left open has had every
// channel decision certified or settled in FP64, so its states (s, m after k events) follow
// from its logged choices with the FP64 form's arithmetic, and the FP64 waiting times of all
// its states can be formed at once, a warp per state spread over the SMs, where the in-line
// replay takes them one after another on one SM:
//   k_defer_chain   the mass chain of each deferred particle (a warp each, the log read
//                   32 entries at a time);
//   k_defer_states  each state's lambda*_i (state 0: the rate kernel's FP64 arithmetic),
//                   waiting time, FP64 choice, near ties and |ln s'/s| (a warp per state);
//   k_defer_finish  the FP64 form's time sum in order, the chain continued in FP64 past the
//                   logged events where the FP64 times say so, the particle's results (a
//                   warp per particle; a choice that differs from the log falls back to the
//                   in-line replay).
// The results are the FP64 replay's: the same states, quantities and sums in the same order.
__device__ __forceinline__ int defer_count(const McArgs& A) {
  const unsigned long long n = A.dctr[1];
  return n < (unsigned long long)A.defer_cap ? (int)n : A.defer_cap;
}

// A warp per deferred particle: each lane loads one event's log entry and partner, the
// chain then runs through the chunk by shuffles (every lane the same values), lane i
// storing the state after event i of the chunk.
__global__ void __launch_bounds__(32) k_defer_chain(McArgs A) {
  const int lane = threadIdx.x;
  const int d = blockIdx.x;
  if (d >= defer_count(A)) return;
  const DeferRec rec = A.defer[d];
  if (!rec.ok) return;
  const long long r = rec.r;
  const int b = inst_of(A.off, A.n_inst, r);
  const InstDev& P = A.P[b];
  const int ub = A.unit_r ? A.unit_r[r] : b;
  const unsigned il = (unsigned)(A.perm[r] - P.off), iv = (unsigned)A.st[ub].interval_cur;
  const Snap64 sn = A.snap64[r];
  double s = sn.s, m = sn.m;
  int sset = 1;
  DState* St = A.dstate + rec.sbase;
  if (lane == 0) {
    St[0].s = s;
    St[0].m = m;
    St[0].sset = 1;
  }
  for (int base = 0; base < rec.n; base += 32) {
    const int k = base + lane;
    int4 L = make_int4(0, 0, 0, 0);
    double pm = 0.0, ps = 0.0;
    if (k < rec.n) {
      L = A.dlog[rec.lbase + k];
      const Snap64 pj = A.snap64[L.y];
      pm = pj.m;
      ps = pj.s;
    }
    const int cnt = min(32, rec.n - base);
    for (int i = 0; i < cnt; ++i) {
      const int ch = __shfl_sync(FULLM, L.x, i) & 1;
      const int oc = __shfl_sync(FULLM, L.z, i);
      const double nc = (double)__shfl_sync(FULLM, L.w, i);
      Snap64 pj;
      pj.m = __shfl_sync(FULLM, pm, i);
      pj.s = __shfl_sync(FULLM, ps, i);
      pj.N = 0.0;
      pj.inv_m = 0.0;
      if (oc == 2 && !sset) {   // a fragmentation starts from the FP64 diameter
        s = s_of_m64(P.rho_s, m);
        sset = 1;
      }
      event64(P.rho_s, P.s_min, P.key0, P.key1, pj, ch, oc, nc, il, iv, (unsigned)(base + i), s, m, sset);
      if (lane == i) {
        St[base + i + 1].s = s;
        St[base + i + 1].m = m;
        St[base + i + 1].sset = sset;
      }
    }
  }
}

template <int S>
__global__ void __launch_bounds__(256) k_defer_states(McArgs A) {
  const int lane = threadIdx.x & 31;
  const int nd = defer_count(A);
  for (int d = blockIdx.y; d < nd; d += gridDim.y) {
    const DeferRec rec = A.defer[d];
    if (!rec.ok) continue;
    const long long r = rec.r;
    const int b = inst_of(A.off, A.n_inst, r);
    const InstDev& P = A.P[b];
    const int ub = A.unit_r ? A.unit_r[r] : b;
    const unsigned il = (unsigned)(A.perm[r] - P.off), iv = (unsigned)A.st[ub].interval_cur;
    const int wpb = blockDim.x >> 5;
    for (int k = blockIdx.x * wpb + (threadIdx.x >> 5); k <= rec.n; k += gridDim.x * wpb) {
      DState* Sk = A.dstate + rec.sbase + k;
      const double m = Sk->m;
      const double s = Sk->sset ? Sk->s : s_of_m64(P.rho_s, m);
      const U4 w = philox(il, iv, (unsigned)k, 0u, P.key0, P.key1);
      const Fp64Pick pk = fp64_event<S>(A, r, b, s, m, w.z, w.w, true, lane);
      double lam = pk.lam;
      // the first waiting time takes lambda*_i as the rate kernel forms it
      if (k == 0) lam = lam0_fp64<S>(A, r, lane);
      double dt = 0.0;
      if (lam > 0.0 && isfinite(lam)) dt = waiting_time<double>(w.x, w.y, lam);
      double J = 0.0;
      int bad = 0;
      if (k < rec.n) {
        const int4 L = A.dlog[rec.lbase + k];
        bad = L.x != pk.chosen ? 1 : 0;
        const DState& Sn = A.dstate[rec.sbase + k + 1];
        const double s1 = Sn.sset ? Sn.s : s_of_m64(P.rho_s, Sn.m);
        J = fabs(log(s1 / s));
      }
      if (lane == 0) {
        Sk->lam = lam;
        Sk->dt = dt;
        Sk->J = J;
        Sk->ncoll = pk.ncoll;
        Sk->chosen = pk.chosen;
        Sk->j = pk.j;
        Sk->outcome = pk.outcome;
        Sk->np = pk.near_pair;
        Sk->nc = pk.near - pk.near_pair;
        Sk->bad = bad;
      }
    }
  }
}

template <int S>
__global__ void __launch_bounds__(32) k_defer_finish(McArgs A) {
  const int lane = threadIdx.x;
  const int d = blockIdx.x;
  if (d >= defer_count(A)) return;
  const DeferRec rec = A.defer[d];
  if (!rec.ok) return;
  const long long r = rec.r;
  const DState* St = A.dstate + rec.sbase;
  int bad = 0;
  for (int k = lane; k < rec.n; k += 32) bad |= St[k].bad;
  if (__any_sync(FULLM, bad != 0)) {
    replay64<S>(A, r, lane);
    return;
  }
  const int b = inst_of(A.off, A.n_inst, r);
  const InstDev& P = A.P[b];
  const int ub = A.unit_r ? A.unit_r[r] : b;
  const unsigned il = (unsigned)(A.perm[r] - P.off), iv = (unsigned)A.st[ub].interval_cur;
  const double dte = A.st[ub].dt_exe;
  // the records of the logged states, 32 at a time: lane i holds state cb + i, and every lane
  // takes state k's fields by shuffles, so the walk below is uniform over the warp
  int cb = -1;
  double c_lam = 0.0, c_dt = 0.0, c_J = 0.0;
  int c_np = 0, c_nc = 0, c_ch = -1;
  double lam, dt, Jk;
  int np, nc, ch;
  auto rec_of = [&](int k) {
    const int base = k & ~31;
    if (base != cb) {
      cb = base;
      const int q = base + lane;
      if (q <= rec.n) {
        const DState& x = St[q];
        c_lam = x.lam; c_dt = x.dt; c_J = x.J; c_np = x.np; c_nc = x.nc; c_ch = x.chosen;
      }
    }
    const int src = k - base;
    lam = __shfl_sync(FULLM, c_lam, src);
    dt = __shfl_sync(FULLM, c_dt, src);
    Jk = __shfl_sync(FULLM, c_J, src);
    np = __shfl_sync(FULLM, c_np, src);
    nc = __shfl_sync(FULLM, c_nc, src);
    ch = __shfl_sync(FULLM, c_ch, src);
  };
  int nn = 0, e = 0;
  unsigned h = 0u;
  double J = 0.0;
  rec_of(0);
  double t = dt;
  bool any = false;
  if (lam > 0.0 && isfinite(lam)) {
    if (fabs(t - dte) < 1e-10 * dte) nn++;
    any = !(t > dte);
  }
  // past the logged events: the state's (s, m) and its choice's partner, outcome and N_coll
  double s = 0.0, m = 0.0, cn = 1.0;
  int cj = -1, co = 0;
  bool past = false;
  if (any) {
    nn += np;
    for (;;) {
      // the event at the current state (its FP64 choice)
      nn += nc;
      if (ch < 0) break;
      h = h * 31u + (unsigned)(ch + 1);
      if (e < rec.n) {
        J += Jk;
      } else {
        if (!past) {
          const DState& x = St[rec.n];
          m = x.m;
          s = x.sset ? x.s : s_of_m64(P.rho_s, x.m);
          cj = x.j;
          co = x.outcome;
          cn = x.ncoll;
          past = true;
        }
        double s1 = s, m1 = m;
        int ss1 = 1;
        event64(P.rho_s, P.s_min, P.key0, P.key1, A.snap64[cj], ch & 1, co, cn, il, iv, (unsigned)e, s1, m1, ss1);
        if (!ss1) s1 = s_of_m64(P.rho_s, m1);
        J += fabs(log(s1 / s));
        s = s1;
        m = m1;
      }
      ++e;
      if (e >= A.max_events) {
        if (lane == 0) set_status(&A.st[ub], GD_ST_EVENT_CAP);
        break;
      }
      // the new state: from the state pass, or formed here past the logged events
      if (e <= rec.n) {
        rec_of(e);
      } else {
        const U4 w = philox(il, iv, (unsigned)e, 0u, P.key0, P.key1);
        const Fp64Pick pk = fp64_event<S>(A, r, b, s, m, w.z, w.w, true, lane);
        lam = pk.lam;
        dt = (pk.lam > 0.0 && isfinite(pk.lam)) ? waiting_time<double>(w.x, w.y, pk.lam) : 0.0;
        np = pk.near_pair;
        nc = pk.near - pk.near_pair;
        ch = pk.chosen;
        cj = pk.j;
        co = pk.outcome;
        cn = pk.ncoll;
      }
      nn += np;
      if (!(lam > 0.0) || !isfinite(lam)) {
        if (lane == 0 && !(lam == 0.0)) set_status(&A.st[ub], GD_ST_NONFINITE);
        break;
      }
      if (fabs((t + dt) - dte) < 1e-10 * dte) nn++;
      if (t + dt > dte) break;
      t = t + dt;
    }
  }
  if (!past) {   // the final diameter: that of the state reached
    const DState& x = St[e];
    s = x.sset ? x.s : s_of_m64(P.rho_s, x.m);
  }
  if (lane == 0) {
    const int ci = A.perm[r];
    atomicAdd((unsigned long long*)&A.st[ub].sample_deferred, 1ull);
    if (e > 0) {
      A.s_out[ci] = s;
      atomicAdd((unsigned long long*)&A.st[ub].events, (unsigned long long)e);
    }
    A.MJ[ci] = A.Mr[r] * J;
    if (nn) atomicAdd((unsigned long long*)&A.st[ub].near_draw, (unsigned long long)nn);
    if (A.ev_count) {
      A.ev_count[ci] = e;
      A.ev_hash[ci] = h;
      A.near_out[ci] = nn;
    }
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(64, sizeof(T) == 8 ? 4 : 7) k_sample(McArgs A) {
  const int lane = threadIdx.x & 31;
  // spatial groups: the round's ranks only (A.act), 32 to a chunk like the full range
  const long long total = A.act ? (long long)*A.act_n : A.N;
  // work items from one counter: first the heavy particles one per warp, then chunks of 32
  // ranks without them
  const long long n_heavy = A.heavy_n ? (long long)*A.heavy_n : 0;
  const long long n_items = n_heavy + (total + 31) / 32;
  auto next_item = [&]() {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(A.work, 1ull);
    return (long long)__shfl_sync(FULLM, c, 0);
  };
  for (long long item = next_item(); item < n_items; item = next_item()) {
    const bool one = item < n_heavy;   // one particle for the whole warp
    const long long base = one ? 0 : (item - n_heavy) * 32;
    const bool valid = one ? lane == 0 : base + lane < total;
    const long long r = !valid ? 0
                        : one ? (long long)A.heavy[item]
                        : A.act ? (long long)A.act[base + lane] : base + lane;
    sample_item<T, S>(A, lane, one, false, r, valid);
  }
}

// ---------------------------------------------------------------- bounded collision steps
// gd_collide: every instance starts a collision step of length tau and idles once it is
// used up, until the next call.
// hold = 0 with tau = 0 returns the instances to collision steps of dt_coll.
__global__ void k_step_begin(const InstDev* __restrict__ P, StateDev* st, int n_units, const int* __restrict__ unit_inst,
                             double tau, int hold) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;   // the unit
  if (b >= n_units) return;
  st[b].tau = tau;
  st[b].hold = hold;
  st[b].remain_ticks = 1LL << 60;
  st[b].level = -1;
  st[b].dt_remain = tau > 0.0 ? tau : P[unit_inst ? unit_inst[b] : b].dt_coll;
}

// *flag = 1 when every unit (instance, or spatial group with members) has used up its
// collision step.
__global__ void k_step_done(const StateDev* st, int n_units, int* flag) {
  __shared__ int open;
  if (threadIdx.x == 0) open = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < n_units; b += blockDim.x)
    if (st[b].remain_ticks > 0 && st[b].members > 0) open = 1;
  __syncthreads();
  if (threadIdx.x == 0) *flag = open ? 0 : 1;
}

// ---------------------------------------------------------------- audit
// One block per instance: realised mass-weighted sum of |ln(s'/s)| per controller bin
// against 2 eps C; C halves (>= 1/4) on excess, else grows by 1.25 (<= 1).  Clears the
// fine bins for the next interval.
__global__ void k_audit(const InstDev* __restrict__ P, StateDev* st, BinsDev* bins, int n_units,
                        const int* __restrict__ unit_inst, int no_audit, double tie) {
  __shared__ double sM[kNFine], sJ[kNFine], gM[kNFine], gJ[kNFine];
  __shared__ int gid[kNFine];
  const int b = blockIdx.x;    // the unit
  if (b >= n_units) return;
  const InstDev& p = P[unit_inst ? unit_inst[b] : b];
  BinsDev& Bn = bins[b];
  for (int f = threadIdx.x; f < kNFine; f += blockDim.x) {
    sM[f] = Bn.sM[f]; sJ[f] = Bn.sJ[f]; gid[f] = Bn.gid[f];
    gM[f] = 0.0; gJ[f] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0 && st[b].dt_exe > 0.0) {   // an idle (held) interval leaves C alone
    StateDev& S = st[b];
    if (p.audit && !no_audit) {
      for (int f = 0; f < kNFine; ++f)
        if (gid[f] >= 0) { gM[gid[f]] += sM[f]; gJ[gid[f]] += sJ[f]; }
      const double thr = 2.0 * p.eps * S.C;
      bool exceed = false;
      for (int g = 0; g < Bn.ngroups; ++g) {
        const double Rg = gJ[g] / gM[g];
        if (fabs(Rg - thr) <= tie * thr) S.near_audit++;
        if (Rg > thr) exceed = true;
      }
      S.C = exceed ? fmax(0.25, 0.5 * S.C) : fmin(1.0, 1.25 * S.C);
    } else {
      S.C = 1.0;
    }
    S.events_total += S.events;
  }
  __syncthreads();
  for (int f = threadIdx.x; f < kNFine; f += blockDim.x) {
    Bn.cnt[f] = 0.0; Bn.sM[f] = 0.0; Bn.sA[f] = 0.0; Bn.sB[f] = 0.0; Bn.sJ[f] = 0.0;
  }
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_step_begin(gd_ctx* c, double tau, int hold) {
  k_step_begin<<<(c->U + 127) / 128, 128, 0, c->stream>>>(c->d_inst, c->d_state, c->U, c->d_unit_inst, tau, hold);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_step_done(gd_ctx* c, int* d_flag) {
  k_step_done<<<1, 256, 0, c->stream>>>(c->d_state, c->U, d_flag);
  c->launches += 1;
  return cudaGetLastError();
}

static McArgs mc_args(gd_ctx* c) {
  McArgs A;
  A.N = c->N;
  A.K = c->K;
  A.n_inst = c->n_inst;
  A.off = c->d_off;
  A.P = c->d_inst;
  A.st = c->d_state;
  A.bins = c->d_bins;
  A.pos64 = c->d_pos64;
  A.snap64 = c->d_snap64;
  A.snap32 = c->d_snap32;
  A.Mr = c->d_Mr;
  A.V = c->d_V;
  A.nbr = c->d_nbr;
  A.perm = c->d_perm;
  A.lam = c->d_lam;
  A.chan_out = nullptr;
  A.s_out = c->s;
  A.ev_count = nullptr;
  A.ev_hash = nullptr;
  A.near_out = nullptr;
  A.max_events = c->max_events;
  A.work = nullptr;
  A.gx = c->d_gx;
  A.pref32 = c->d_pref32;
  A.contrib = c->d_contrib;
  A.redo = c->d_redo;
  A.redo_n = nullptr;
  A.list = nullptr;
  A.list_n = nullptr;
  A.MJ = c->d_MJ;
  A.part = c->d_part;
  A.n_tiles = c->n_btiles;
  A.unit_r = c->grouped ? c->d_unit_r : nullptr;
  A.act = c->grouped ? c->d_act : nullptr;
  A.act_n = c->grouped ? c->d_counters + 10 : nullptr;
  A.unit_inst = c->d_unit_inst;
  A.heavy = nullptr;
  A.heavy_n = nullptr;
  A.dlog = c->d_dlog;
  A.dlog_cap = c->dlog_cap;
  A.dctr = c->d_counters + 12;
  A.defer = c->d_defer;
  A.defer_cap = c->defer_cap;
  A.dstate = c->d_dstate;
  A.dstate_cap = c->dstate_cap;
  return A;
}

// Per-unit sums of quantities q0 .. q0 + nq - 1 from the fine-bin tile partials (8 warps a
// block; idle spatial groups skipped).
static void bins_reduce(gd_ctx* c, int q0, int nq, int skip_q) {
  dim3 grid(c->U, (nq * kNFine + 7) / 8);
  k_bins_reduce<<<grid, 256, 0, c->stream>>>(c->grouped ? c->d_utile_off : c->d_tile_off, c->d_part, c->n_btiles,
                                             q0, nq, skip_q, c->d_bins, nullptr,
                                             c->grouped ? c->d_state : nullptr);
}

// The rate kernel's grid: one wave of the blocks its register budget lets an SM hold -- 6 of
// 128 threads in the mixed form (80 registers without spills ran 1.60 ms on the 2^22 disk
// against 1.64 with 64 and 8 blocks), 4 in the FP64 form (a second, partial wave of the
// grid-stride loop made the FP64 rates a third slower).
static int rate_grid(const gd_ctx* c) { return c->num_sms * (c->precision == GD_MIXED ? 6 : 4); }

cudaError_t launch_rates(gd_ctx* c, double* chan_out) {
  McArgs A = mc_args(c);
  A.chan_out = chan_out;
  const int* gperm = c->grouped ? c->d_gperm : nullptr;
  time_begin(c, 2);
  // one block per tile, lane = particle: any K
  if (c->precision == GD_MIXED) {
    // particles the FP32 rates cannot certify are listed (counter 5) and redone in FP64
    A.redo_n = c->d_counters + 5;
    cudaMemsetAsync(A.redo_n, 0, sizeof(unsigned long long), c->stream);
    k_rates<float><<<rate_grid(c), 128, 0, c->stream>>>(A);
    McArgs B = A;
    B.list = c->d_redo;
    B.list_n = A.redo_n;
    k_rates_redo<<<c->num_sms * 2, 128, 0, c->stream>>>(B);
    k_bins_tile<float><<<c->n_btiles, 128, 0, c->stream>>>(bins_map(c), c->d_rank_of, c->d_contrib, c->d_part,
                                                           c->n_btiles, gperm, c->d_state);
    c->launches += 1;
  } else {
    k_rates<double><<<rate_grid(c), 128, 0, c->stream>>>(A);
    k_bins_tile<double><<<c->n_btiles, 128, 0, c->stream>>>(bins_map(c), c->d_rank_of, c->d_contrib, c->d_part,
                                                            c->n_btiles, gperm, c->d_state);
  }
  bins_reduce(c, 0, 6, 4);     // count, M, M A, M B and the error bound; sJ after sampling
  time_end(c);
  c->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_interval(gd_ctx* c) {
  time_begin(c, 3);
  k_interval<<<c->U, 128, 0, c->stream>>>(c->d_inst, c->d_state, c->d_bins, c->U, c->d_unit_inst, c->K,
                                          (c->flags & GD_FLAG_NO_AUDIT) ? 1 : 0,
                                          c->precision == GD_MIXED ? 1 : 0);
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_schedule(c);
  time_end(c);
  return e;
}

template <typename T, int S>
static void sample_launch(gd_ctx* c, const McArgs& A) {
  // 64-thread blocks: the register budget of this kernel then still fills the SM
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample<T, S>, 64, 0);
  if (per_sm < 1) per_sm = 1;
  long long chunks = (A.N + 31) / 32;
  long long blocks = (long long)c->num_sms * per_sm;
  if (blocks > (chunks + 1) / 2) blocks = (chunks + 1) / 2;
  if (blocks < 1) blocks = 1;
  k_sample<T, S><<<(int)blocks, 64, 0, c->stream>>>(A);
}

// The deferred FP64 settlement after the mixed sampler: 32 blocks of 8 warps per deferred
// particle for its states (each warp a state at a time; 32 particles at once, the grid
// striding over more), then a warp per particle.
template <int S>
static void defer_launch(gd_ctx* c, const McArgs& A) {
  k_defer_chain<<<c->defer_cap, 32, 0, c->stream>>>(A);
  k_defer_states<S><<<dim3(32, 32), 256, 0, c->stream>>>(A);
  k_defer_finish<S><<<c->defer_cap, 32, 0, c->stream>>>(A);
  c->launches += 3;
}

template <typename T>
static void sample_t(gd_ctx* c, McArgs& A) {
  int S = (c->K + 31) / 32;
  A.work = c->d_counters;
  // the heavy particles first, one warp each (counter 11 counts them)
  unsigned long long* hn = c->d_counters + 11;
  cudaMemsetAsync(hn, 0, sizeof(unsigned long long), c->stream);
  k_heavy<<<c->num_sms * 8, 256, 0, c->stream>>>(A, c->d_heavy, hn);
  c->launches += 1;
  A.heavy = c->d_heavy;
  A.heavy_n = hn;
  cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long), c->stream);
  if (sizeof(T) == 4 && A.dlog) cudaMemsetAsync(A.dctr, 0, 3 * sizeof(unsigned long long), c->stream);
  switch (S) {
    case 1: sample_launch<T, 1>(c, A); break;
    case 2: sample_launch<T, 2>(c, A); break;
    case 3: sample_launch<T, 3>(c, A); break;
    case 4: sample_launch<T, 4>(c, A); break;
    default: sample_launch<T, 8>(c, A); break;
  }
  if (sizeof(T) == 4 && A.dlog) {
    switch (S) {
      case 1: defer_launch<1>(c, A); break;
      case 2: defer_launch<2>(c, A); break;
      case 3: defer_launch<3>(c, A); break;
      case 4: defer_launch<4>(c, A); break;
      default: defer_launch<8>(c, A); break;
    }
  }
}

cudaError_t launch_sample(gd_ctx* c, int* ev_count, unsigned* ev_hash, int* near) {
  McArgs A = mc_args(c);
  A.ev_count = ev_count;
  A.ev_hash = ev_hash;
  A.near_out = near;
  if (ev_count == nullptr || ev_hash == nullptr || near == nullptr) {
    A.ev_count = nullptr;
  }
  time_begin(c, 4);
  if (c->grouped && A.ev_count) {
    // the sampler visits only the round's particles: the others report no event
    cudaMemsetAsync(ev_count, 0, sizeof(int) * c->N, c->stream);
    cudaMemsetAsync(ev_hash, 0, sizeof(unsigned) * c->N, c->stream);
    cudaMemsetAsync(near, 0, sizeof(int) * c->N, c->stream);
  }
  if (c->precision == GD_MIXED) sample_t<float>(c, A); else sample_t<double>(c, A);
  time_end(c);
  c->launches += 1;
  return cudaGetLastError();
}

// The size spectrum of every instance into BinsDev::spec (gd_stats).
cudaError_t launch_spectrum(gd_ctx* c) {
  k_spec_tile<<<c->n_tiles, 128, 0, c->stream>>>(tile_map(c), c->s, c->M, c->d_part, c->n_btiles);
  // per instance, into its first unit
  dim3 grid(c->n_inst, (kNFine + 7) / 8);
  k_bins_reduce<<<grid, 256, 0, c->stream>>>(c->d_tile_off, c->d_part, c->n_btiles, 6, 1, -1, c->d_bins,
                                             c->d_inst, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_audit(gd_ctx* c) {
  time_begin(c, 3);
  const int* gperm = c->grouped ? c->d_gperm : nullptr;
  if (c->precision == GD_MIXED)
    k_jbins<true><<<c->n_btiles, 128, 0, c->stream>>>(bins_map(c), c->d_rank_of, c->d_contrib, c->d_MJ, c->d_part,
                                                      c->n_btiles, gperm, c->d_state);
  else
    k_jbins<false><<<c->n_btiles, 128, 0, c->stream>>>(bins_map(c), c->d_rank_of, c->d_contrib, c->d_MJ, c->d_part,
                                                       c->n_btiles, gperm, c->d_state);
  bins_reduce(c, 4, 1, -1);
  k_audit<<<c->U, 128, 0, c->stream>>>(c->d_inst, c->d_state, c->d_bins, c->U, c->d_unit_inst,
                                       (c->flags & GD_FLAG_NO_AUDIT) ? 1 : 0,
                                       c->precision == GD_MIXED ? 2e-5 : 1e-10);
  time_end(c);
  c->launches += 3;
  return cudaGetLastError();
}

}  // namespace gd
