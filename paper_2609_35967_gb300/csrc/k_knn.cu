// k_knn.cu -- K nearest neighbours over the device cell list (Sect. 2.5.1).
//
// A warp owns a chunk of 32 consecutive query ranks (neighbouring cells) and works in
// three phases:
//  A  per query, warp-cooperative: scan every cell row that meets a ball of radius rho
//     around the query (rows are contiguous rank ranges, so loads are coalesced), keep a
//     register top list over the lanes (slot g in lane g % 32, register g / 32) ordered by
//     (key, index), and accept rho once the ball provably holds the K-1 nearest others.
//     All search bookkeeping (cell ranges, slab distances, radii) is FP32/INT in the
//     query's cell-relative frame with conservative margins.
//       FP64 form : key = bits of d^2 = (dx dx + dy dy) + dz dz in FP64 (no FMA, minimum
//                   image), ties by caller index: the oracle's order exactly.
//       mixed form: key = FP32 d^2 from cell-relative FP32 coordinates; with
//                   |sqrt(D32) - d| <= 10u sqrt(D32) + E (u = 2^-24) keys below T_lo are
//                   certain members and keys up to T_hi form a band that phase B ranks
//                   exactly in FP64.  A band that overflows the list or the band buffer,
//                   or a periodic axis covered whole, sends the query to the FP64 form.
//  B  lane = query: the FP64 arithmetic (band re-rank, d_i = sqrt(d^2), V_i with the
//     flat-boundary caps), so FP64 instructions carry 32 queries each.
//  C  per query: members sorted by caller index (bitonic over the lanes), written as
//     ranks after the particle itself.
#include <climits>

#include "gd_ctx.h"
#include "gd_physics.cuh"

namespace gd {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kBand = 8;          // band entries resolved in phase B per query
constexpr int kWarps = 8;         // warps per block

struct KnnArgs {
  long long N;
  int K, n_inst;
  const long long* off;
  const InstDev* P;
  const GridDev* grid;
  const int* cstart;
  const Pos64* pos64;
  const float4* pos32;
  const int* perm;
  int* nbr;
  double* dist;
  double* V;
  StateDev* st;
};

template <typename KT> __device__ __forceinline__ KT kmax_();
template <> __device__ __forceinline__ unsigned long long kmax_<unsigned long long>() { return ~0ull; }
template <> __device__ __forceinline__ unsigned kmax_<unsigned>() { return ~0u; }

template <typename KT>
__device__ __forceinline__ bool kless(KT ka, int ja, KT kb, int jb) {
  return ka < kb || (ka == kb && ja < jb);
}

// Sorted list of 32*KPL (key, tie index, rank) entries spread over the warp.
template <int KPL, typename KT>
struct TopList {
  KT k[KPL];
  int j[KPL];
  int r[KPL];

  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int t = 0; t < KPL; ++t) { k[t] = kmax_<KT>(); j[t] = INT_MAX; r[t] = -1; }
  }
  __device__ __forceinline__ void get(int g, KT& kk, int& jj) const {
    KT kv = k[0];
    int jv = j[0];
#pragma unroll
    for (int t = 1; t < KPL; ++t)
      if (t == (g >> 5)) { kv = k[t]; jv = j[t]; }
    kk = __shfl_sync(FULL, kv, g & 31);
    jj = __shfl_sync(FULL, jv, g & 31);
  }
  __device__ __forceinline__ void insert(KT nk, int nj, int nr, int lane) {
    int p = 0;
#pragma unroll
    for (int t = 0; t < KPL; ++t) p += __popc(__ballot_sync(FULL, kless(k[t], j[t], nk, nj)));
#pragma unroll
    for (int t = KPL - 1; t >= 0; --t) {
      KT uk = __shfl_up_sync(FULL, k[t], 1);
      int uj = __shfl_up_sync(FULL, j[t], 1);
      int ur = __shfl_up_sync(FULL, r[t], 1);
      if (t > 0) {
        const int tp = t > 0 ? t - 1 : 0;
        KT ck = __shfl_sync(FULL, k[tp], 31);
        int cj = __shfl_sync(FULL, j[tp], 31);
        int cr = __shfl_sync(FULL, r[tp], 31);
        if (lane == 0) { uk = ck; uj = cj; ur = cr; }
      }
      int g = t * 32 + lane;
      if (g > p) { k[t] = uk; j[t] = uj; r[t] = ur; }
      else if (g == p) { k[t] = nk; j[t] = nj; r[t] = nr; }
    }
  }
};

// Bitonic sort of 32*KPL (j, r) pairs by j, element e = t*32 + lane.
template <int KPL>
__device__ __forceinline__ void sort_by_index(int (&jj)[KPL], int (&rr)[KPL], int lane) {
  constexpr int S = 32 * KPL;
#pragma unroll
  for (int k = 2; k <= S; k <<= 1) {
#pragma unroll
    for (int s = k >> 1; s > 0; s >>= 1) {
      if (s >= 32) {
        const int rs = s >> 5;
#pragma unroll
        for (int t = 0; t < KPL; ++t) {
          const int tp = t ^ rs;
          if (tp > t) {
            int e = t * 32 + lane;
            bool up = (e & k) == 0;
            bool sw = up ? (jj[t] > jj[tp]) : (jj[t] < jj[tp]);
            if (sw) {
              int a = jj[t]; jj[t] = jj[tp]; jj[tp] = a;
              a = rr[t]; rr[t] = rr[tp]; rr[tp] = a;
            }
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < KPL; ++t) {
          int e = t * 32 + lane;
          int pj = __shfl_xor_sync(FULL, jj[t], s);
          int pr = __shfl_xor_sync(FULL, rr[t], s);
          bool up = (e & k) == 0;
          bool lower = (lane & s) == 0;
          bool take = (lower == up) ? (pj < jj[t]) : (pj > jj[t]);
          if (take) { jj[t] = pj; rr[t] = pr; }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- geometry (FP32 / INT)
struct QueryPos {
  double x, y, z;     // FP64 position (FP64 keys)
  int ix, iy, iz;     // own cell
  float fx, fy, fz;   // position inside the own cell [cm]
};

struct Grid32 {
  float cs[3], inv[3];
  int dim[3];
  bool per;           // x and y periodic
  long long cell_off;
};

// Conservative cell range [lo, hi] (unwrapped on periodic axes) of the slab
// |coordinate - query| <= rs along one axis; full = a periodic axis covered whole.
__device__ __forceinline__ void axis_range32(const Grid32& G, int a, int ia, float fa, float rs, int& lo,
                                             int& hi, bool& full) {
  const float m = rs * 1.00001f + G.cs[a] * 1e-5f;
  float t0 = floorf((fa - m) * G.inv[a]);
  float t1 = floorf((fa + m) * G.inv[a]);
  const int d = G.dim[a];
  t0 = fmaxf(t0, -4.0e6f);
  t1 = fminf(t1, 4.0e6f);
  lo = ia + (int)t0;
  hi = ia + (int)t1;
  full = false;
  if (G.per && a < 2) {
    if (hi - lo + 1 >= d) { lo = 0; hi = d - 1; full = true; }
  } else {
    lo = lo < 0 ? 0 : lo;
    hi = hi > d - 1 ? d - 1 : hi;
  }
}

// Lower bound of the distance from the query to the slab of (unwrapped) cell k.
__device__ __forceinline__ float slab_dist32(const Grid32& G, int a, int ia, float fa, int k) {
  float d;
  if (k < ia) d = (float)(ia - k - 1) * G.cs[a] + fa;
  else if (k > ia) d = (float)(k - ia) * G.cs[a] - fa;
  else d = 0.0f;
  return fmaxf(d * 0.99999f - G.cs[a] * 1e-5f, 0.0f);
}

__device__ __forceinline__ int floordiv(int a, int d) {
  int q = a / d;
  return (a % d != 0 && ((a < 0) != (d < 0))) ? q - 1 : q;
}

// Visits the stored rank ranges [ra, rb) of every cell row within rs of the query:
// visit(ra, rb, x_shift_cells, dy_cells, dz_cells).  Returns true when a periodic axis
// was covered whole (the FP32 cell offsets are then ambiguous).
template <class F>
__device__ __forceinline__ bool scan_ball(const Grid32& G, const int* __restrict__ cstart, const QueryPos& Q,
                                          float rs, F&& visit) {
  bool amb = false;
  int lz, hz, ly, hy;
  bool fz, fy;
  axis_range32(G, 2, Q.iz, Q.fz, rs, lz, hz, fz);
  axis_range32(G, 1, Q.iy, Q.fy, rs, ly, hy, fy);
  if (fy && G.per) amb = true;
  const float rs2 = rs * rs * 1.00002f;
  const int dimx = G.dim[0], dimy = G.dim[1];
  for (int iz = lz; iz <= hz; ++iz) {
    const float dz = slab_dist32(G, 2, Q.iz, Q.fz, iz);
    if (dz * dz > rs2) continue;
    for (int iyu = ly; iyu <= hy; ++iyu) {
      const float dy = fy ? 0.0f : slab_dist32(G, 1, Q.iy, Q.fy, iyu);
      const float dyz2 = dy * dy + dz * dz;
      if (dyz2 > rs2) continue;
      int iy = iyu;
      if (G.per) { iy %= dimy; if (iy < 0) iy += dimy; }
      const float xr = sqrtf(fmaxf(rs2 - dyz2, 0.0f));
      int lx, hx;
      bool fx;
      axis_range32(G, 0, Q.ix, Q.fx, xr, lx, hx, fx);
      if (lx > hx) continue;
      if (fx && G.per) amb = true;
      const long long rowc = G.cell_off + (long long)dimx * (iy + (long long)dimy * iz);
      int kx = 0, a0 = lx, e0 = hx;
      if (G.per && !fx) {
        kx = floordiv(lx, dimx);
        a0 = lx - kx * dimx;
        e0 = hx - kx * dimx;
      }
      const int e1 = e0 < dimx ? e0 : dimx - 1;
      visit(__ldg(&cstart[rowc + a0]), __ldg(&cstart[rowc + e1 + 1]), kx * dimx, iyu - Q.iy, iz - Q.iz);
      if (e0 >= dimx)
        visit(__ldg(&cstart[rowc]), __ldg(&cstart[rowc + (e0 - dimx) + 1]), (kx + 1) * dimx,
              iyu - Q.iy, iz - Q.iz);
    }
  }
  return amb;
}

// Offers one candidate per lane; lanes below the threshold are inserted in lane order.
template <int KPL, typename KT, class R>
__device__ __forceinline__ void offer(TopList<KPL, KT>& Lst, KT ck, int cj, int cr, KT& wk, int& wj,
                                      int lane, R&& refresh) {
  unsigned m = __ballot_sync(FULL, kless(ck, cj, wk, wj));
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1;
    const KT nk = __shfl_sync(FULL, ck, src);
    const int nj = __shfl_sync(FULL, cj, src);
    const int nr = __shfl_sync(FULL, cr, src);
    if (kless(nk, nj, wk, wj)) {
      Lst.insert(nk, nj, nr, lane);
      refresh();
    }
  }
}

__device__ __forceinline__ double sample_volume(const InstDev& P, double d, double x, double y) {
  if (P.kernel_mode != GD_KERNEL_PHYSICAL) return 1.0;
  double V = 4.0 * kPi * d * d * d / 3.0;
  if (P.geometry == GD_GEOM_DISK) {
    double R = sqrt(x * x + y * y);
    double h = R - P.R_in;
    if (h > 0.0 && h < d) V -= kPi * (d - h) * (d - h) * (2.0 * d + h) / 3.0;
    h = P.R_out - R;
    if (h > 0.0 && h < d) V -= kPi * (d - h) * (d - h) * (2.0 * d + h) / 3.0;
  }
  return V;
}

__device__ __forceinline__ float rho_start(const Grid32& G, const int* __restrict__ cstart, const QueryPos& Q,
                                           int L) {
  int n = 0, nc = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    int iz = Q.iz + dz;
    if (iz < 0 || iz >= G.dim[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      int iy = Q.iy + dy;
      if (G.per) { iy %= G.dim[1]; if (iy < 0) iy += G.dim[1]; }
      else if (iy < 0 || iy >= G.dim[1]) continue;
      int x0 = Q.ix - 1, x1 = Q.ix + 1;
      if (!G.per) { x0 = x0 < 0 ? 0 : x0; x1 = x1 >= G.dim[0] ? G.dim[0] - 1 : x1; }
      for (int ix = x0; ix <= x1; ++ix) {
        int xw = ix;
        if (G.per) { xw %= G.dim[0]; if (xw < 0) xw += G.dim[0]; }
        long long c = G.cell_off + xw + (long long)G.dim[0] * (iy + (long long)G.dim[1] * iz);
        n += __ldg(&cstart[c + 1]) - __ldg(&cstart[c]);
        ++nc;
      }
    }
  }
  const float csmax = fmaxf(G.cs[0], fmaxf(G.cs[1], G.cs[2]));
  if (n <= 1) return 2.0f * csmax;
  // density in units of csmax^3 (a cell volume in cm^3 can exceed the FP32 range)
  const float vcell = (G.cs[0] / csmax) * (G.cs[1] / csmax) * (G.cs[2] / csmax);
  const float nd = (float)(n - 1) / ((float)nc * vcell);
  const float r = 1.2f * csmax * cbrtf(3.0f * (float)L / (4.0f * 3.14159265f * nd));
  return fminf(fmaxf(r, 1e-3f * csmax), 4.0f * csmax * (float)(G.dim[0] + G.dim[1] + G.dim[2]));
}

__device__ __forceinline__ float grow(float rho, int found, int L) {
  float g = cbrtf(1.3f * (float)L / (float)(found > 0 ? found : 1));
  return rho * fminf(fmaxf(g, 1.25f), 3.0f);
}

// Minimum-image FP64 d^2 of rank r from the query: the oracle's expression.
__device__ __forceinline__ double d2_fp64(const Pos64* __restrict__ pos64, int r, double qx, double qy,
                                          double qz, double bx, double by, long long& j) {
  const double2* pp = reinterpret_cast<const double2*>(pos64 + r);
  double2 a = __ldg(pp), b = __ldg(pp + 1);
  double dx = a.x - qx, dy = a.y - qy, dz = b.x - qz;
  if (bx > 0.0) {
    if (dx > 0.5 * bx) dx -= bx; else if (dx < -0.5 * bx) dx += bx;
    if (dy > 0.5 * by) dy -= by; else if (dy < -0.5 * by) dy += by;
  }
  j = __double_as_longlong(b.y);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Phase-A result of one query, kept in shared memory for phases B and C.
struct QInfo {
  int state;          // 0 done (row, d, V written), 1 FP64 members written, 2 mixed band pending
  int p_lo;           // certain members written to the row
  int nb;             // band entries
  int need;           // band entries to select
  unsigned long long d2max;   // FP64 form: bits of the (K-1)-th d^2
  int band[kBand];
};

// FP64-key search for one query (the plain form, and the fallback of the mixed form).
// Writes the unsorted members to the row and the (K-1)-th d^2; returns false on failure.
template <int KPL>
__device__ bool query_fp64(const KnnArgs& A, const Grid32& G, const GridDev& Gd, const QueryPos& Q, long long q,
                           int lane, float rho, QInfo& qi) {
  const int L = A.K - 1;
  TopList<KPL, unsigned long long> Lst;
  const double bx = Gd.box[0], by = Gd.box[1];
  const float diag = sqrtf((float)G.dim[0] * G.dim[0] * G.cs[0] * G.cs[0] +
                           (float)G.dim[1] * G.dim[1] * G.cs[1] * G.cs[1] +
                           (float)G.dim[2] * G.dim[2] * G.cs[2] * G.cs[2]);
  for (int att = 0; att < 64; ++att) {
    Lst.reset();
    unsigned long long wk = ~0ull;
    int wj = INT_MAX;
    const double rho2 = (double)rho * (double)rho;
    auto refresh = [&]() { Lst.get(L - 1, wk, wj); };
    scan_ball(G, A.cstart, Q, rho, [&](int ra, int rb, int, int, int) {
      for (int base = ra; base < rb; base += 32) {
        const int r = base + lane;
        unsigned long long ck = ~0ull;
        int cj = INT_MAX;
        if (r < rb && r != (int)q) {
          long long jj;
          const double d2 = d2_fp64(A.pos64, r, Q.x, Q.y, Q.z, bx, by, jj);
          if (d2 <= rho2) { ck = (unsigned long long)__double_as_longlong(d2); cj = (int)jj; }
        }
        offer(Lst, ck, cj, r, wk, wj, lane, refresh);
      }
    });
    unsigned long long kL;
    int jL;
    Lst.get(L - 1, kL, jL);
    if (kL != ~0ull) {
      int* row = A.nbr + q * (long long)A.K;
#pragma unroll
      for (int t = 0; t < KPL; ++t) {
        int g = t * 32 + lane;
        if (g < L) row[1 + g] = Lst.r[t];
      }
      if (lane == 0) { qi.state = 1; qi.d2max = kL; }
      return true;
    }
    int found = 0;
#pragma unroll
    for (int t = 0; t < KPL; ++t) found += __popc(__ballot_sync(FULL, Lst.k[t] != ~0ull));
    if (rho > 2.0f * diag) break;
    rho = grow(rho, found, L);
  }
  return false;
}

// FP32-key search with the FP64 band; returns false when the query needs the FP64 form.
template <int KPL>
__device__ bool query_mixed(const KnnArgs& A, const Grid32& G, const GridDev& Gd, const QueryPos& Q, long long q,
                            int lane, float& rho, QInfo& qi) {
  const int L = A.K - 1;
  constexpr int S = 32 * KPL;
  if (S < L + 1) return false;
  TopList<KPL, unsigned> Lst;
  const float E = Gd.E32;
  const float rel = 10.0f * 5.9604645e-8f;
  const float Ef = 4.02f * E, E2f = 4.02f * E * E;
  const float diag = sqrtf((float)G.dim[0] * G.dim[0] * G.cs[0] * G.cs[0] +
                           (float)G.dim[1] * G.dim[1] * G.cs[1] * G.cs[1] +
                           (float)G.dim[2] * G.dim[2] * G.cs[2] * G.cs[2]);
  for (int att = 0; att < 64; ++att) {
    Lst.reset();
    unsigned wk = ~0u;
    int wj = INT_MAX;
    const float rf = (rho * (1.0f + rel) + E) * 1.000001f;
    const float rhof2 = rf * rf * 1.000001f;
    // insertion threshold: the last list slot, or a bound above T_hi of the current
    // (K-1)-th key, whichever is lower
    auto refresh = [&]() {
      unsigned kS, kL;
      int jS, jL;
      Lst.get(S - 1, kS, jS);
      Lst.get(L - 1, kL, jL);
      wk = kS;
      wj = jS;
      if (kL != ~0u) {
        const float tau = __uint_as_float(kL);
        const float tins = (tau * (1.0f + 12.0f * rel) + Ef * sqrtf(tau) + E2f) * 1.00001f;
        const unsigned tb = __float_as_uint(tins);
        if (tb < wk) { wk = tb; wj = INT_MAX; }
      }
    };
    const float csx = G.cs[0], csy = G.cs[1], csz = G.cs[2];
    const bool amb = scan_ball(G, A.cstart, Q, rho, [&](int ra, int rb, int xsh, int dyc, int dzc) {
      const float offy = (float)dyc * csy, offz = (float)dzc * csz;
      for (int base = ra; base < rb; base += 32) {
        const int r = base + lane;
        unsigned ck = ~0u;
        int cj = INT_MAX;
        if (r < rb && r != (int)q) {
          const float4 p = __ldg(A.pos32 + r);
          const int ixj = __float_as_int(p.w) & 2047;
          const float dx = (p.x - Q.fx) + (float)(ixj + xsh - Q.ix) * csx;
          const float dy = (p.y - Q.fy) + offy;
          const float dz = (p.z - Q.fz) + offz;
          const float D = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          if (D <= rhof2) { ck = __float_as_uint(D); cj = r; }
        }
        offer(Lst, ck, cj, cj, wk, wj, lane, refresh);
      }
    });
    if (amb) return false;
    unsigned kL;
    int jL;
    Lst.get(L - 1, kL, jL);
    if (kL == ~0u) {
      int found = 0;
#pragma unroll
      for (int t = 0; t < KPL; ++t) found += __popc(__ballot_sync(FULL, Lst.k[t] != ~0u));
      if (rho > 2.0f * diag) return false;
      rho = grow(rho, found, L);
      continue;
    }
    // FP32 bounds with relative margins far above their own rounding
    const float sq = sqrtf(__uint_as_float(kL));
    const float hi_tau = (sq * (1.0f + rel) * 1.000001f + E) * 1.00001f;
    if (hi_tau > rho) {
      if (rho > 2.0f * diag) return false;
      rho = fmaxf(rho * 1.25f, hi_tau * 1.02f);
      continue;
    }
    const float lo_tau = (sq * (1.0f - rel) * 0.999999f - E) * 0.99999f;
    const float tlo = (lo_tau - E) / (1.0f + rel);
    const float thi = (hi_tau + E) / (1.0f - rel);
    const unsigned Tlo = tlo > 0.0f ? __float_as_uint(tlo * tlo * 0.9999f) : 0u;
    const unsigned Thi = __float_as_uint(thi * thi * 1.0001f);
    unsigned kS;
    int jS;
    Lst.get(S - 1, kS, jS);
    if (!(kS > Thi)) return false;       // the band may extend past the list
    int p_lo = 0, p_hi = 0;
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      p_lo += __popc(__ballot_sync(FULL, Lst.k[t] < Tlo));
      p_hi += __popc(__ballot_sync(FULL, Lst.k[t] <= Thi));
    }
    const int nb = p_hi - p_lo;
    if (nb > kBand) return false;
    int* row = A.nbr + q * (long long)A.K;
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      const int g = t * 32 + lane;
      if (g < p_lo) row[1 + g] = Lst.r[t];
      else if (g < p_hi) qi.band[g - p_lo] = Lst.r[t];
    }
    if (lane == 0) {
      qi.state = 2;
      qi.p_lo = p_lo;
      qi.nb = nb;
      qi.need = L - p_lo;
    }
    return true;
  }
  return false;
}

template <int KPL, bool kMixed>
__global__ void __launch_bounds__(kWarps * 32) k_knn(KnnArgs A) {
  __shared__ QInfo info[kWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int L = A.K - 1;
  for (long long base = warp * 32; base < A.N; base += nwarps * 32) {
    // ---- phase A: per query, warp-cooperative FP32/INT search
    for (int qi_ = 0; qi_ < 32; ++qi_) {
      const long long q = base + qi_;
      if (q >= A.N) break;
      QInfo& qi = info[w][qi_];
      const int b = inst_of(A.off, A.n_inst, q);
      const GridDev& Gd = A.grid[b];
      Grid32 G;
#pragma unroll
      for (int a = 0; a < 3; ++a) { G.cs[a] = Gd.cs32[a]; G.inv[a] = Gd.inv32[a]; G.dim[a] = Gd.dim[a]; }
      G.per = Gd.periodic != 0;
      G.cell_off = Gd.cell_off;
      QueryPos Q;
      const float4 f = __ldg(A.pos32 + q);
      const int pk = __float_as_int(f.w);
      Q.ix = pk & 2047;
      Q.iy = (pk >> 11) & 2047;
      Q.iz = (pk >> 22) & 1023;
      Q.fx = f.x; Q.fy = f.y; Q.fz = f.z;
      const double2* pp = reinterpret_cast<const double2*>(A.pos64 + q);
      const double2 a0 = __ldg(pp), a1 = __ldg(pp + 1);
      Q.x = a0.x; Q.y = a0.y; Q.z = a1.x;
      float rho = rho_start(G, A.cstart, Q, L);
      bool done = false;
      if (kMixed) done = query_mixed<KPL>(A, G, Gd, Q, q, lane, rho, qi);
      if (!done) done = query_fp64<KPL>(A, G, Gd, Q, q, lane, rho, qi);
      if (!done) {
        // no acceptable radius: keep the row valid (the particle against itself), V = 1
        int* row = A.nbr + q * (long long)A.K;
        for (int k = lane; k < A.K; k += 32) row[k] = (int)q;
        if (lane == 0) {
          qi.state = 0;
          A.dist[q] = 0.0;
          A.V[q] = 1.0;
          set_status(&A.st[b], GD_ST_KNN);
        }
      }
    }
    __syncwarp();
    // ---- phase B: lane = query, the FP64 arithmetic
    {
      const long long q = base + lane;
      if (q < A.N) {
        QInfo& qi = info[w][lane];
        if (qi.state != 0) {
          const int b = inst_of(A.off, A.n_inst, q);
          const GridDev& Gd = A.grid[b];
          const double2* pp = reinterpret_cast<const double2*>(A.pos64 + q);
          const double2 a0 = __ldg(pp), a1 = __ldg(pp + 1);
          double d2max;
          if (qi.state == 1) {
            d2max = __longlong_as_double((long long)qi.d2max);
          } else {
            // exact FP64 keys of the band, the `need` smallest by (d^2, index)
            double bd[kBand];
            long long bj[kBand];
            for (int t = 0; t < qi.nb; ++t)
              bd[t] = d2_fp64(A.pos64, qi.band[t], a0.x, a0.y, a1.x, Gd.box[0], Gd.box[1], bj[t]);
            int* row = A.nbr + q * (long long)A.K;
            int wr = 1 + qi.p_lo;
            d2max = 0.0;
            for (int t = 0; t < qi.nb; ++t) {
              int rank = 0;
              for (int u = 0; u < qi.nb; ++u)
                if (bd[u] < bd[t] || (bd[u] == bd[t] && bj[u] < bj[t])) rank++;
              if (rank < qi.need) {
                row[wr++] = qi.band[t];
                d2max = fmax(d2max, bd[t]);
              }
            }
          }
          const double d = sqrt(d2max);
          A.dist[q] = d;
          A.V[q] = sample_volume(A.P[b], d, a0.x, a0.y);
        }
      }
    }
    __syncwarp();
    // ---- phase C: members by ascending caller index
    for (int qi_ = 0; qi_ < 32; ++qi_) {
      const long long q = base + qi_;
      if (q >= A.N) break;
      if (info[w][qi_].state == 0) continue;
      int* row = A.nbr + q * (long long)A.K;
      int jj[KPL], rr[KPL];
#pragma unroll
      for (int t = 0; t < KPL; ++t) {
        const int g = t * 32 + lane;
        if (g < L) { rr[t] = row[1 + g]; jj[t] = __ldg(&A.perm[rr[t]]); }
        else { rr[t] = -1; jj[t] = INT_MAX; }
      }
      sort_by_index<KPL>(jj, rr, lane);
#pragma unroll
      for (int t = 0; t < KPL; ++t) {
        const int g = t * 32 + lane;
        if (g < L) row[1 + g] = rr[t];
      }
      if (lane == 0) row[0] = (int)q;
    }
    __syncwarp();
  }
}

template <int KPL, bool kMixed>
static cudaError_t launch_knn_t(gd_ctx* c, const KnnArgs& A) {
  const int bs = kWarps * 32;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_knn<KPL, kMixed>, bs, 0);
  if (per_sm < 1) per_sm = 1;
  long long chunks = (A.N + 31) / 32;
  long long want = (chunks + kWarps - 1) / kWarps;
  long long blocks = (long long)c->num_sms * per_sm;
  if (blocks > want) blocks = want;
  if (blocks < 1) blocks = 1;
  k_knn<KPL, kMixed><<<(int)blocks, bs, 0, c->stream>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_knn(gd_ctx* c) {
  KnnArgs A;
  A.N = c->N;
  A.K = c->K;
  A.n_inst = c->n_inst;
  A.off = c->d_off;
  A.P = c->d_inst;
  A.grid = c->d_grid;
  A.cstart = c->d_cell_start;
  A.pos64 = c->d_pos64;
  A.pos32 = c->d_pos32;
  A.perm = c->d_perm;
  A.nbr = c->d_nbr;
  A.dist = c->d_dist;
  A.V = c->d_V;
  A.st = c->d_state;
  const bool mixed = c->precision == GD_MIXED;
  const int kpl = (c->K + 31) / 32;   // room for K-1 members and at least one band slot
  time_begin(c, 1);
  cudaError_t e;
  if (kpl <= 1) e = mixed ? launch_knn_t<1, true>(c, A) : launch_knn_t<1, false>(c, A);
  else if (kpl <= 2) e = mixed ? launch_knn_t<2, true>(c, A) : launch_knn_t<2, false>(c, A);
  else if (kpl <= 4) e = mixed ? launch_knn_t<4, true>(c, A) : launch_knn_t<4, false>(c, A);
  else e = mixed ? launch_knn_t<8, true>(c, A) : launch_knn_t<8, false>(c, A);
  time_end(c);
  c->launches += 1;
  return e;
}

}  // namespace gd
