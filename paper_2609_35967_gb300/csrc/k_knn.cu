// k_knn.cu -- K nearest neighbours over the device cell list (Sect. 2.5.1).
//
// One warp per query particle.  The warp scans every cell row that intersects a ball
// of radius rho around the query (rows are contiguous rank ranges, so loads are
// coalesced), keeps a register top list distributed over the lanes (slot g lives in
// lane g % 32, register g / 32) ordered by (key, index), and accepts rho once the ball
// provably contains the K-1 nearest others; otherwise rho grows and the scan repeats.
//
//  FP64 form : key = bits of d^2 = (dx dx + dy dy) + dz dz (FP64, no FMA, minimum image),
//              ties by caller index -- exactly the oracle's order.
//  mixed form: key = FP32 d^2 from cell-relative FP32 coordinates.  An error bound
//              |sqrt(D32) - d| <= rel sqrt(D32) + E (rel = 10 u, E = 16 u cell + FP64
//              rounding, u = 2^-24) gives thresholds T_lo < T_hi around the (K-1)-th key:
//              keys below T_lo are certain members, keys up to T_hi form the band whose
//              members are re-ranked exactly in FP64.  Any doubt (band not held in the
//              list, a periodic axis fully covered) falls back to the FP64 form.
// Members are then sorted by caller index (bitonic over the lanes) and written as
// ranks after the particle itself; d_i and the sampling measure V_i follow.
#include <climits>

#include "gd_ctx.h"
#include "gd_physics.cuh"

namespace gd {

constexpr unsigned FULL = 0xffffffffu;

struct KnnArgs {
  long long N;
  int K, n_inst;
  const long long* off;
  const InstDev* P;
  const GridDev* grid;
  const int* cstart;
  const Pos64* pos64;
  const float4* pos32;
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

// Sorted list of 32*KPL (key, index, rank) entries spread over the warp.
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

// ---------------------------------------------------------------- geometry
struct QueryPos {
  double x, y, z;     // raw position
  double xw, yw;      // wrapped into the periodic box
  int ix, iy, iz;     // own cell
  float fx, fy, fz;   // FP32 cell-relative coordinates (mixed form)
};

__device__ __forceinline__ void axis_range(const GridDev& G, int a, double qa, double rs, int& lo,
                                           int& hi, bool& full) {
  double t0 = floor((qa - rs - G.lo[a]) * G.inv[a]);
  double t1 = floor((qa + rs - G.lo[a]) * G.inv[a]);
  int d = G.dim[a];
  full = false;
  if (G.box[a] > 0.0) {
    if (t1 - t0 + 1.0 >= (double)d) { lo = 0; hi = d - 1; full = true; return; }
    lo = (int)t0;
    hi = (int)t1;
  } else {
    t0 = fmax(t0, 0.0);
    t1 = fmin(t1, (double)(d - 1));
    lo = (int)t0;
    hi = (int)t1;
  }
}

__device__ __forceinline__ double slab_dist(const GridDev& G, int a, double qa, int k) {
  double l = G.lo[a] + k * G.cs[a];
  double h = l + G.cs[a];
  return fmax(0.0, fmax(l - qa, qa - h));
}

__device__ __forceinline__ int floordiv(int a, int d) {
  int q = a / d;
  return (a % d != 0 && ((a < 0) != (d < 0))) ? q - 1 : q;
}

// Visits every stored rank range [ra, rb) of the cell rows within distance rs of the
// query: visit(ra, rb, x_shift_cells, dy_cells, dz_cells).  Returns true when a periodic
// axis had to be covered whole (FP32 offsets are then ambiguous).
template <class F>
__device__ __forceinline__ bool scan_ball(const GridDev& G, const int* __restrict__ cstart,
                                          const QueryPos& Q, double rs, F&& visit) {
  bool amb = false;
  int lz, hz, ly, hy;
  bool fz, fy;
  axis_range(G, 2, Q.z, rs, lz, hz, fz);
  axis_range(G, 1, Q.yw, rs, ly, hy, fy);
  if (fy && G.box[1] > 0.0) amb = true;
  const double rs2 = rs * rs;
  const int dimx = G.dim[0], dimy = G.dim[1];
  for (int iz = lz; iz <= hz; ++iz) {
    double dz = slab_dist(G, 2, Q.z, iz);
    if (dz > rs) continue;
    for (int iyu = ly; iyu <= hy; ++iyu) {
      double dy = slab_dist(G, 1, Q.yw, iyu);
      double dyz2 = dy * dy + dz * dz;
      if (dyz2 > rs2) continue;
      int iy = iyu;
      if (G.box[1] > 0.0) { iy %= dimy; if (iy < 0) iy += dimy; }
      double xr = sqrt(fmax(rs2 - dyz2, 0.0));
      int lx, hx;
      bool fx;
      axis_range(G, 0, Q.xw, xr, lx, hx, fx);
      if (lx > hx) continue;
      if (fx && G.box[0] > 0.0) amb = true;
      long long rowc = G.cell_off + (long long)dimx * (iy + (long long)dimy * iz);
      int kx = 0, a0 = lx, e0 = hx;
      if (G.box[0] > 0.0 && !fx) {
        kx = floordiv(lx, dimx);
        a0 = lx - kx * dimx;
        e0 = hx - kx * dimx;
      }
      int e1 = e0 < dimx ? e0 : dimx - 1;
      visit(__ldg(&cstart[rowc + a0]), __ldg(&cstart[rowc + e1 + 1]), kx * dimx, iyu - Q.iy, iz - Q.iz);
      if (e0 >= dimx)
        visit(__ldg(&cstart[rowc]), __ldg(&cstart[rowc + (e0 - dimx) + 1]), (kx + 1) * dimx,
              iyu - Q.iy, iz - Q.iz);
    }
  }
  return amb;
}

// Offers one candidate per lane; lanes below the threshold are inserted in lane order.
template <int KPL, typename KT>
__device__ __forceinline__ void offer(TopList<KPL, KT>& Lst, KT ck, int cj, int cr, KT& wk, int& wj,
                                      int lane, int slot_thr) {
  unsigned m = __ballot_sync(FULL, kless(ck, cj, wk, wj));
  while (m) {
    int src = __ffs(m) - 1;
    m &= m - 1;
    KT nk = __shfl_sync(FULL, ck, src);
    int nj = __shfl_sync(FULL, cj, src);
    int nr = __shfl_sync(FULL, cr, src);
    if (kless(nk, nj, wk, wj)) {
      Lst.insert(nk, nj, nr, lane);
      Lst.get(slot_thr, wk, wj);
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

template <int KPL>
__device__ __forceinline__ void write_list(const KnnArgs& A, long long q, int L, int (&jj)[KPL],
                                           int (&rr)[KPL], int lane, double d, const InstDev& P,
                                           const QueryPos& Q) {
  sort_by_index<KPL>(jj, rr, lane);
  int* row = A.nbr + q * (long long)A.K;
#pragma unroll
  for (int t = 0; t < KPL; ++t) {
    int e = t * 32 + lane;
    if (e < L) row[1 + e] = rr[t];
  }
  if (lane == 0) {
    row[0] = (int)q;
    A.dist[q] = d;
    A.V[q] = sample_volume(P, d, Q.x, Q.y);
  }
}

__device__ __forceinline__ double rho_start(const GridDev& G, const int* __restrict__ cstart,
                                            const QueryPos& Q, int L) {
  int n = 0, nc = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    int iz = Q.iz + dz;
    if (iz < 0 || iz >= G.dim[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      int iy = Q.iy + dy;
      if (G.box[1] > 0.0) { iy %= G.dim[1]; if (iy < 0) iy += G.dim[1]; }
      else if (iy < 0 || iy >= G.dim[1]) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        int ix = Q.ix + dx;
        if (G.box[0] > 0.0) { ix %= G.dim[0]; if (ix < 0) ix += G.dim[0]; }
        else if (ix < 0 || ix >= G.dim[0]) continue;
        long long c = G.cell_off + ix + (long long)G.dim[0] * (iy + (long long)G.dim[1] * iz);
        n += __ldg(&cstart[c + 1]) - __ldg(&cstart[c]);
        ++nc;
      }
    }
  }
  double csmax = fmax(G.cs[0], fmax(G.cs[1], G.cs[2]));
  if (n <= 1) return 2.0 * csmax;
  double nd = (double)(n - 1) / (nc * G.cs[0] * G.cs[1] * G.cs[2]);
  return 1.2 * cbrt(3.0 * L / (4.0 * kPi * nd));
}

// ---------------------------------------------------------------- FP64 form
template <int KPL>
__device__ void query_fp64(const KnnArgs& A, const GridDev& G, const InstDev& P, const QueryPos& Q,
                           long long q, int lane, double rho, StateDev* st) {
  const int L = A.K - 1;
  TopList<KPL, unsigned long long> Lst;
  double diag = sqrt(G.cs[0] * G.cs[0] * G.dim[0] * G.dim[0] + G.cs[1] * G.cs[1] * G.dim[1] * G.dim[1] +
                     G.cs[2] * G.cs[2] * G.dim[2] * G.dim[2]);
  for (int att = 0; att < 64; ++att) {
    Lst.reset();
    unsigned long long wk = ~0ull;
    int wj = INT_MAX;
    const double rho2 = rho * rho;
    const double rs = rho * (1.0 + 1e-9);
    const double bx = G.box[0], by = G.box[1];
    scan_ball(G, A.cstart, Q, rs, [&](int ra, int rb, int, int, int) {
      for (int base = ra; base < rb; base += 32) {
        int r = base + lane;
        unsigned long long ck = ~0ull;
        int cj = INT_MAX;
        if (r < rb && r != (int)q) {
          const double2* pp = reinterpret_cast<const double2*>(A.pos64 + r);
          double2 a = __ldg(pp), b = __ldg(pp + 1);
          double dx = a.x - Q.x, dy = a.y - Q.y, dz = b.x - Q.z;
          if (bx > 0.0) {
            if (dx > 0.5 * bx) dx -= bx; else if (dx < -0.5 * bx) dx += bx;
            if (dy > 0.5 * by) dy -= by; else if (dy < -0.5 * by) dy += by;
          }
          double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
          if (d2 <= rho2) {
            ck = (unsigned long long)__double_as_longlong(d2);
            cj = (int)__double_as_longlong(b.y);
          }
        }
        offer(Lst, ck, cj, r, wk, wj, lane, L - 1);
      }
    });
    unsigned long long kL;
    int jL;
    Lst.get(L - 1, kL, jL);
    if (kL != ~0ull) {
      int jj[KPL], rr[KPL];
#pragma unroll
      for (int t = 0; t < KPL; ++t) {
        bool in = t * 32 + lane < L;
        jj[t] = in ? Lst.j[t] : INT_MAX;
        rr[t] = in ? Lst.r[t] : -1;
      }
      write_list<KPL>(A, q, L, jj, rr, lane, sqrt(__longlong_as_double((long long)kL)), P, Q);
      return;
    }
    int found = 0;
#pragma unroll
    for (int t = 0; t < KPL; ++t) found += __popc(__ballot_sync(FULL, Lst.k[t] != ~0ull));
    if (rho > 2.0 * diag) break;
    double g = cbrt(1.3 * L / (double)(found > 0 ? found : 1));
    rho *= fmin(fmax(g, 1.25), 3.0);
  }
  // no acceptable radius: keep the row valid (the particle against itself only), V = 1
  int* row = A.nbr + q * (long long)A.K;
  for (int k = lane; k < A.K; k += 32) row[k] = (int)q;
  if (lane == 0) {
    A.dist[q] = 0.0;
    A.V[q] = 1.0;
    set_status(st, GD_ST_KNN);
  }
}

// ---------------------------------------------------------------- mixed form
template <int KPL>
__device__ bool query_mixed(const KnnArgs& A, const GridDev& G, const InstDev& P, const QueryPos& Q,
                            long long q, int lane, double& rho) {
  const int L = A.K - 1;
  constexpr int S = 32 * KPL;
  if (S < L + 1) return false;
  TopList<KPL, unsigned> Lst;
  const double u = 0x1p-24;
  const double csmax = fmax(G.cs[0], fmax(G.cs[1], G.cs[2]));
  const double E = 16.0 * u * csmax + 32.0 * 0x1p-53 * G.X32;
  const double rel = 10.0 * u;
  const float Ef = (float)(4.02 * E), E2f = (float)(4.02 * E * E);
  const float csx = (float)G.cs[0], csy = (float)G.cs[1], csz = (float)G.cs[2];
  double diag = sqrt(G.cs[0] * G.cs[0] * G.dim[0] * G.dim[0] + G.cs[1] * G.cs[1] * G.dim[1] * G.dim[1] +
                     G.cs[2] * G.cs[2] * G.dim[2] * G.dim[2]);
  for (int att = 0; att < 64; ++att) {
    Lst.reset();
    unsigned wk = ~0u;
    int wj = INT_MAX;
    const double rf = rho * (1.0 + rel) + E;
    const float rhof2 = __double2float_ru(rf * rf * (1.0 + 1e-9));
    const double rs = rho * (1.0 + 1e-9);
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
        float tau = __uint_as_float(kL);
        float tins = tau * (float)(1.0 + 12.0 * rel) + Ef * sqrtf(tau) + E2f;
        unsigned tb = __float_as_uint(tins) + 4u;
        if (tb < wk) { wk = tb; wj = INT_MAX; }
      }
    };
    bool amb = scan_ball(G, A.cstart, Q, rs, [&](int ra, int rb, int xsh, int dyc, int dzc) {
      const float offy = (float)dyc * csy, offz = (float)dzc * csz;
      for (int base = ra; base < rb; base += 32) {
        int r = base + lane;
        unsigned ck = ~0u;
        int cj = INT_MAX;
        if (r < rb && r != (int)q) {
          float4 p = __ldg(A.pos32 + r);
          int ixj = __float_as_int(p.w) & 2047;
          float dx = (p.x - Q.fx) + (float)(ixj + xsh - Q.ix) * csx;
          float dy = (p.y - Q.fy) + offy;
          float dz = (p.z - Q.fz) + offz;
          float D = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          if (D <= rhof2) { ck = __float_as_uint(D); cj = r; }
        }
        unsigned m = __ballot_sync(FULL, kless(ck, cj, wk, wj));
        while (m) {
          int src = __ffs(m) - 1;
          m &= m - 1;
          unsigned nk = __shfl_sync(FULL, ck, src);
          int nj = __shfl_sync(FULL, cj, src);
          if (kless(nk, nj, wk, wj)) {
            Lst.insert(nk, nj, nj, lane);
            refresh();
          }
        }
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
      if (rho > 2.0 * diag) return false;
      double g = cbrt(1.3 * L / (double)(found > 0 ? found : 1));
      rho *= fmin(fmax(g, 1.25), 3.0);
      continue;
    }
    const double sq = sqrt((double)__uint_as_float(kL));
    const double hi_tau = sq * (1.0 + rel) + E;
    if (hi_tau > rho) {
      if (rho > 2.0 * diag) return false;
      rho = fmax(rho * 1.25, hi_tau * 1.02);
      continue;
    }
    const double lo_tau = sq * (1.0 - rel) - E;
    const double tlo = (lo_tau - E) / (1.0 + rel);
    const double thi = (hi_tau + E) / (1.0 - rel);
    const unsigned Tlo = tlo > 0.0 ? __float_as_uint(__double2float_rd(tlo * tlo * (1.0 - 1e-12))) : 0u;
    const unsigned Thi = __float_as_uint(__double2float_ru(thi * thi * (1.0 + 1e-12)));
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
    const int need = L - p_lo;
    // exact FP64 keys of the band entries
    unsigned long long bk[KPL];
    int bj[KPL];
    double bd[KPL];
    const double bx = G.box[0], by = G.box[1];
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      int g = t * 32 + lane;
      bk[t] = ~0ull;
      bj[t] = INT_MAX;
      bd[t] = 0.0;
      if (g >= p_lo && g < p_hi) {
        const double2* pp = reinterpret_cast<const double2*>(A.pos64 + Lst.r[t]);
        double2 a = __ldg(pp), b = __ldg(pp + 1);
        double dx = a.x - Q.x, dy = a.y - Q.y, dz = b.x - Q.z;
        if (bx > 0.0) {
          if (dx > 0.5 * bx) dx -= bx; else if (dx < -0.5 * bx) dx += bx;
          if (dy > 0.5 * by) dy -= by; else if (dy < -0.5 * by) dy += by;
        }
        double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        bk[t] = (unsigned long long)__double_as_longlong(d2);
        bj[t] = (int)__double_as_longlong(b.y);
        bd[t] = d2;
      }
    }
    // rank of each band entry among the band by (d^2, index)
    int rank[KPL];
#pragma unroll
    for (int t = 0; t < KPL; ++t) rank[t] = 0;
    for (int g2 = p_lo; g2 < p_hi; ++g2) {
      unsigned long long ok = bk[0];
      int oj = bj[0];
#pragma unroll
      for (int t = 1; t < KPL; ++t)
        if (t == (g2 >> 5)) { ok = bk[t]; oj = bj[t]; }
      ok = __shfl_sync(FULL, ok, g2 & 31);
      oj = __shfl_sync(FULL, oj, g2 & 31);
#pragma unroll
      for (int t = 0; t < KPL; ++t)
        if (kless(ok, oj, bk[t], bj[t])) rank[t]++;
    }
    double d2max = 0.0;
    int jj[KPL], rr[KPL];
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      int g = t * 32 + lane;
      jj[t] = INT_MAX;
      rr[t] = -1;
      if (g < p_lo) {
        rr[t] = Lst.r[t];
        jj[t] = (int)__ldg(&A.pos64[rr[t]].j);
      } else if (g < p_hi && rank[t] < need) {
        rr[t] = Lst.r[t];
        jj[t] = bj[t];
        d2max = fmax(d2max, bd[t]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2max = fmax(d2max, __shfl_xor_sync(FULL, d2max, o));
    write_list<KPL>(A, q, L, jj, rr, lane, sqrt(d2max), P, Q);
    return true;
  }
  return false;
}

template <int KPL, bool kMixed>
__global__ void __launch_bounds__(256) k_knn(KnnArgs A) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long q = warp; q < A.N; q += nwarps) {
    const int b = inst_of(A.off, A.n_inst, q);
    const GridDev G = A.grid[b];
    const InstDev P = A.P[b];
    QueryPos Q;
    const double2* pp = reinterpret_cast<const double2*>(A.pos64 + q);
    double2 a = __ldg(pp), c = __ldg(pp + 1);
    Q.x = a.x; Q.y = a.y; Q.z = c.x;
    Q.xw = Q.x; Q.yw = Q.y;
    if (G.box[0] > 0.0) Q.xw = Q.x - G.box[0] * floor((Q.x - G.lo[0]) / G.box[0]);
    if (G.box[1] > 0.0) Q.yw = Q.y - G.box[1] * floor((Q.y - G.lo[1]) / G.box[1]);
    Q.ix = axis_cell(G, 0, Q.x);
    Q.iy = axis_cell(G, 1, Q.y);
    Q.iz = axis_cell(G, 2, Q.z);
    if (kMixed) {
      float4 f = __ldg(A.pos32 + q);
      Q.fx = f.x; Q.fy = f.y; Q.fz = f.z;
    } else {
      Q.fx = Q.fy = Q.fz = 0.f;
    }
    double rho = rho_start(G, A.cstart, Q, A.K - 1);
    bool done = false;
    if (kMixed) done = query_mixed<KPL>(A, G, P, Q, q, lane, rho);
    if (!done) query_fp64<KPL>(A, G, P, Q, q, lane, rho, &A.st[b]);
  }
}

template <int KPL, bool kMixed>
static cudaError_t launch_knn_t(gd_ctx* c, const KnnArgs& A) {
  int bs = c->knn_block;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_knn<KPL, kMixed>, bs, 0);
  if (per_sm < 1) per_sm = 1;
  long long want = (A.N * 32 + bs - 1) / bs;
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
  A.nbr = c->d_nbr;
  A.dist = c->d_dist;
  A.V = c->d_V;
  A.st = c->d_state;
  bool mixed = c->precision == GD_MIXED;
  int kpl = (c->K + 31) / 32;   // room for K-1 members and at least one band slot
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
