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

// Candidate ranks of every cell row within rs of the query, in 32-wide batches flattened
// across rows.  Rows are set up one per lane (their cell_start loads are in flight
// together), a warp scan lays the rows' rank ranges end to end, and each lane of a batch
// finds its row by a binary search over the lanes.  visit(valid, r, x_shift_cells,
// dy_cells, dz_cells) sees every candidate once.  Returns true when a periodic axis was
// covered whole (the FP32 cell offsets are then ambiguous).
template <class F>
__device__ __forceinline__ bool scan_ball(const Grid32& G, const int* __restrict__ cstart, const QueryPos& Q,
                                          float rs, int lane, F&& visit) {
  bool amb = false;
  int lz, hz, ly, hy;
  bool fz, fy;
  axis_range32(G, 2, Q.iz, Q.fz, rs, lz, hz, fz);
  axis_range32(G, 1, Q.iy, Q.fy, rs, ly, hy, fy);
  if (fy && G.per) amb = true;
  const float rs2 = rs * rs * 1.00002f;
  const int dimx = G.dim[0], dimy = G.dim[1];
  const int ny = hy - ly + 1, nz = hz - lz + 1;
  const int nrows = (ny > 0 && nz > 0) ? ny * nz : 0;
  for (int r0 = 0; r0 < nrows; r0 += 32) {
    const int row = r0 + lane;
    int ra0 = 0, c0 = 0, ra1 = 0, c1 = 0, sh0 = 0, sh1 = 0, dyc = 0, dzc = 0;
    bool rowamb = false;
    if (row < nrows) {
      const int iz = lz + row / ny, iyu = ly + row % ny;
      const float dz = slab_dist32(G, 2, Q.iz, Q.fz, iz);
      const float dy = fy ? 0.0f : slab_dist32(G, 1, Q.iy, Q.fy, iyu);
      const float dyz2 = dy * dy + dz * dz;
      if (dyz2 <= rs2) {
        int iy = iyu;
        if (G.per) { iy %= dimy; if (iy < 0) iy += dimy; }
        const float xr = sqrtf(fmaxf(rs2 - dyz2, 0.0f));
        int lx, hx;
        bool fx;
        axis_range32(G, 0, Q.ix, Q.fx, xr, lx, hx, fx);
        if (lx <= hx) {
          if (fx && G.per) rowamb = true;
          const long long rowc = G.cell_off + (long long)dimx * (iy + (long long)dimy * iz);
          int kx = 0, a0 = lx, e0 = hx;
          if (G.per && !fx) {
            kx = floordiv(lx, dimx);
            a0 = lx - kx * dimx;
            e0 = hx - kx * dimx;
          }
          const int e1 = e0 < dimx ? e0 : dimx - 1;
          ra0 = __ldg(&cstart[rowc + a0]);
          c0 = __ldg(&cstart[rowc + e1 + 1]) - ra0;
          sh0 = kx * dimx;
          if (e0 >= dimx) {
            ra1 = __ldg(&cstart[rowc]);
            c1 = __ldg(&cstart[rowc + (e0 - dimx) + 1]) - ra1;
            sh1 = (kx + 1) * dimx;
          }
          dyc = iyu - Q.iy;
          dzc = iz - Q.iz;
        }
      }
    }
    if (__any_sync(FULL, rowamb)) amb = true;
    const int cnt = c0 + c1;
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    const int excl = inc - cnt;
    const int total = __shfl_sync(FULL, inc, 31);
    for (int f0 = 0; f0 < total; f0 += 32) {
      const int f = f0 + lane;
      int o = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int c = o + step;
        const int ex = __shfl_sync(FULL, excl, c & 31);
        if (c < 32 && ex <= f) o = c;
      }
      const int oex = __shfl_sync(FULL, excl, o), oc0 = __shfl_sync(FULL, c0, o);
      const int ora0 = __shfl_sync(FULL, ra0, o), ora1 = __shfl_sync(FULL, ra1, o);
      const int osh0 = __shfl_sync(FULL, sh0, o), osh1 = __shfl_sync(FULL, sh1, o);
      const int ody = __shfl_sync(FULL, dyc, o), odz = __shfl_sync(FULL, dzc, o);
      const int loc = f - oex;
      const bool first = loc < oc0;
      visit(f < total, first ? ora0 + loc : ora1 + (loc - oc0), first ? osh0 : osh1, ody, odz);
    }
  }
  return amb;
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

// Radius estimate from the particle count of the 27 cells around the query (lane c < 27
// loads cell c, so the loads are in flight together).
__device__ __forceinline__ float rho_start(const Grid32& G, const int* __restrict__ cstart, const QueryPos& Q,
                                           int L, int lane) {
  int n = 0, nc = 0;
  if (lane < 27) {
    const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
    int ix = Q.ix + dx, iy = Q.iy + dy;
    const int iz = Q.iz + dz;
    bool ok = iz >= 0 && iz < G.dim[2];
    if (G.per) {
      ix %= G.dim[0]; if (ix < 0) ix += G.dim[0];
      iy %= G.dim[1]; if (iy < 0) iy += G.dim[1];
    } else {
      ok = ok && ix >= 0 && ix < G.dim[0] && iy >= 0 && iy < G.dim[1];
    }
    if (ok) {
      const long long c = G.cell_off + ix + (long long)G.dim[0] * (iy + (long long)G.dim[1] * iz);
      n = __ldg(&cstart[c + 1]) - __ldg(&cstart[c]);
      nc = 1;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(FULL, n, o);
    nc += __shfl_xor_sync(FULL, nc, o);
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

// Candidates inside the search ball of one query, in shared memory (per warp).
template <int KB>
struct CandBuf {
  unsigned long long key[32 * KB];   // FP64 form: bits of d^2; mixed: (bits of the FP32 D) << 32 | rank
  int j[32 * KB];                    // FP64 form: tie index (caller index)
  int r[32 * KB];                    // FP64 form: rank
};

// Compare-exchange of register pairs (t, t ^ RS) inside each lane, block direction from
// the element index e = t*32 + lane.
template <int RS, int KB>
__device__ __forceinline__ void cas_regs(int nreg, int kk, unsigned long long (&k)[KB], int (&j)[KB],
                                         int (&r)[KB], int lane) {
#pragma unroll
  for (int t = 0; t < KB; ++t) {
    const int tp = t ^ RS;
    if (tp > t && tp < KB && t < nreg && tp < nreg) {
      const bool up = ((t * 32 + lane) & kk) == 0;
      const bool gt = kless(k[tp], j[tp], k[t], j[t]);
      if (up == gt) {
        unsigned long long a = k[t]; k[t] = k[tp]; k[tp] = a;
        int c = j[t]; j[t] = j[tp]; j[tp] = c;
        c = r[t]; r[t] = r[tp]; r[tp] = c;
      }
    }
  }
}

// Bitonic sort, ascending by (key, j), of the first 32*nreg register entries (nreg a power
// of two <= KB).  The stage loops run at run time and only the per-register bodies are
// unrolled, which keeps the code small (the search is otherwise instruction-cache bound).
template <int KB>
__device__ __forceinline__ void sort_cand(int nreg, unsigned long long (&k)[KB], int (&j)[KB], int (&r)[KB],
                                          int lane) {
  const int S = 32 * nreg;
#pragma unroll 1
  for (int kk = 2; kk <= S; kk <<= 1) {
#pragma unroll 1
    for (int s = kk >> 1; s > 0; s >>= 1) {
      if (s >= 32) {
        const int rs = s >> 5;
        if (rs == 1) cas_regs<1, KB>(nreg, kk, k, j, r, lane);
        else if (rs == 2) cas_regs<2, KB>(nreg, kk, k, j, r, lane);
        else if (rs == 4) cas_regs<4, KB>(nreg, kk, k, j, r, lane);
        else if (rs == 8) cas_regs<8, KB>(nreg, kk, k, j, r, lane);
        else cas_regs<16, KB>(nreg, kk, k, j, r, lane);
      } else {
        const bool lower = (lane & s) == 0;
#pragma unroll
        for (int t = 0; t < KB; ++t) {
          if (t < nreg) {
            const unsigned long long pk = __shfl_xor_sync(FULL, k[t], s);
            const int pj = __shfl_xor_sync(FULL, j[t], s);
            const int pr = __shfl_xor_sync(FULL, r[t], s);
            const bool up = ((t * 32 + lane) & kk) == 0;
            const bool pless = kless(pk, pj, k[t], j[t]);
            const bool pgreater = kless(k[t], j[t], pk, pj);
            if ((lower == up) ? pless : pgreater) { k[t] = pk; j[t] = pj; r[t] = pr; }
          }
        }
      }
    }
  }
}

template <int KB>
__device__ __forceinline__ void sort_any(int n, unsigned long long (&k)[KB], int (&j)[KB], int (&r)[KB], int lane) {
  int nreg = 1;
  while (32 * nreg < n && nreg < KB) nreg <<= 1;
  sort_cand<KB>(nreg, k, j, r, lane);
}

// Mixed form: the same bitonic network on packed keys (FP32 D bits << 32 | rank), which
// are distinct, so one 64-bit comparison orders them by (D, rank).
template <int RS, int KB>
__device__ __forceinline__ void cas_packed(int nreg, int kk, unsigned long long (&k)[KB], int lane) {
#pragma unroll
  for (int t = 0; t < KB; ++t) {
    const int tp = t ^ RS;
    if (tp > t && tp < KB && t < nreg && tp < nreg) {
      const bool up = ((t * 32 + lane) & kk) == 0;
      if (up == (k[tp] < k[t])) { unsigned long long a = k[t]; k[t] = k[tp]; k[tp] = a; }
    }
  }
}

template <int KB>
__device__ __forceinline__ void sort_packed(int n, unsigned long long (&k)[KB], int lane) {
  int nreg = 1;
  while (32 * nreg < n && nreg < KB) nreg <<= 1;
  const int S = 32 * nreg;
#pragma unroll 1
  for (int kk = 2; kk <= S; kk <<= 1) {
#pragma unroll 1
    for (int s = kk >> 1; s > 0; s >>= 1) {
      if (s >= 32) {
        const int rs = s >> 5;
        if (rs == 1) cas_packed<1, KB>(nreg, kk, k, lane);
        else if (rs == 2) cas_packed<2, KB>(nreg, kk, k, lane);
        else if (rs == 4) cas_packed<4, KB>(nreg, kk, k, lane);
        else if (rs == 8) cas_packed<8, KB>(nreg, kk, k, lane);
        else cas_packed<16, KB>(nreg, kk, k, lane);
      } else {
        const bool lower = (lane & s) == 0;
#pragma unroll
        for (int t = 0; t < KB; ++t) {
          if (t < nreg) {
            const unsigned long long pk = __shfl_xor_sync(FULL, k[t], s);
            const bool up = ((t * 32 + lane) & kk) == 0;
            // keep the smaller of the pair in the lower lane of an ascending block
            if ((lower == up) == (pk < k[t])) k[t] = pk;
          }
        }
      }
    }
  }
}

template <typename KT, int KB>
__device__ __forceinline__ void get_entry(const unsigned long long (&k)[KB], int g, unsigned long long& out) {
  unsigned long long v = k[0];
#pragma unroll
  for (int t = 1; t < KB; ++t)
    if (t == (g >> 5)) v = k[t];
  out = __shfl_sync(FULL, v, g & 31);
}

// Search of one query.  Candidates inside rho go to the warp's buffer, are sorted, and
// the K-1 nearest taken; FP64 form: exact keys, the members and the (K-1)-th d^2 are
// final; mixed form: certain members and the FP64 band are left to phase B.  Returns
// false when the query must be redone (mixed: in the FP64 form; FP64: failed).
template <int KB, bool kMixed>
__device__ __forceinline__ bool query_buf(const KnnArgs& A, const Grid32& G, const GridDev& Gd, const QueryPos& Q, long long q,
                          int lane, float& rho, QInfo& qi, CandBuf<KB>& buf, float& dk) {
  constexpr int CAP = 32 * KB;
  const int L = A.K - 1;
  const float E = Gd.E32;
  const float rel = 10.0f * 5.9604645e-8f;
  const double bx = Gd.box[0], by = Gd.box[1];
  const float csx = G.cs[0], csy = G.cs[1], csz = G.cs[2];
  const float diag = sqrtf((float)G.dim[0] * G.dim[0] * G.cs[0] * G.cs[0] +
                           (float)G.dim[1] * G.dim[1] * G.cs[1] * G.cs[1] +
                           (float)G.dim[2] * G.dim[2] * G.cs[2] * G.cs[2]);
  float r_lo = 0.0f, r_hi = 0.0f;    // radii known to hold too few / too many candidates
  for (int att = 0; att < 64; ++att) {
    int n_in = 0;
    const double rho2 = (double)rho * (double)rho;
    const float rf = (rho * (1.0f + 2.0f * rel) + 2.0f * E) * 1.000001f;
    const float rhof2 = rf * rf * 1.000001f;
    const bool amb = scan_ball(G, A.cstart, Q, rho, lane, [&](bool valid, int r, int xsh, int dyc, int dzc) {
      bool in = false;
      unsigned long long key = 0;
      int tj = 0;
      if (valid && r != (int)q) {
        if (kMixed) {
          const float4 p = __ldg(A.pos32 + r);
          const int ixj = __float_as_int(p.w) & 2047;
          const float dx = (p.x - Q.fx) + (float)(ixj + xsh - Q.ix) * csx;
          const float dy = (p.y - Q.fy) + (float)dyc * csy;
          const float dz = (p.z - Q.fz) + (float)dzc * csz;
          const float D = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          in = D <= rhof2;
          key = ((unsigned long long)__float_as_uint(D) << 32) | (unsigned)r;
        } else {
          long long jj;
          const double d2 = d2_fp64(A.pos64, r, Q.x, Q.y, Q.z, bx, by, jj);
          in = d2 <= rho2;
          key = (unsigned long long)__double_as_longlong(d2);
          tj = (int)jj;
        }
      }
      const unsigned m = __ballot_sync(FULL, in);
      const int pos = n_in + __popc(m & ((1u << lane) - 1u));
      if (in && pos < CAP) {
        buf.key[pos] = key;
        if (!kMixed) { buf.j[pos] = tj; buf.r[pos] = r; }
      }
      n_in += __popc(m);
    });
    if (kMixed && amb) return false;
    if (n_in < L) {
      if (rho > 2.0f * diag) return false;
      r_lo = rho;
      rho = r_hi > 0.0f ? sqrtf(r_lo * r_hi) : grow(rho, n_in, L);
      continue;
    }
    if (n_in > CAP) {
      r_hi = rho;
      rho = r_lo > 0.0f ? sqrtf(r_lo * r_hi) : rho * fmaxf(cbrtf(0.7f * (float)CAP / (float)n_in), 0.3f);
      continue;
    }
    __syncwarp();
    unsigned long long k[KB];
    int j[KB], r[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int e = t * 32 + lane;
      if (kMixed) {
        k[t] = e < n_in ? buf.key[e] : ~0ull;
      } else if (e < n_in) {
        k[t] = buf.key[e]; j[t] = buf.j[e]; r[t] = buf.r[e];
      } else {
        k[t] = ~0ull; j[t] = INT_MAX; r[t] = -1;
      }
    }
    __syncwarp();
    if (kMixed) {
      sort_packed<KB>(n_in, k, lane);
#pragma unroll
      for (int t = 0; t < KB; ++t) { r[t] = (int)(unsigned)k[t]; k[t] >>= 32; }
    } else {
      sort_any<KB>(n_in, k, j, r, lane);
    }
    unsigned long long kL;
    get_entry<unsigned long long, KB>(k, L - 1, kL);
    int* row = A.nbr + q * (long long)A.K;
    if (!kMixed) {
#pragma unroll
      for (int t = 0; t < KB; ++t) {
        const int e = t * 32 + lane;
        if (e < L) row[1 + e] = r[t];
      }
      if (lane == 0) { qi.state = 1; qi.d2max = kL; }
      dk = sqrtf((float)__longlong_as_double((long long)kL));   // radius hint only
      return true;
    }
    // FP32 bounds with relative margins far above their own rounding
    const float sq = sqrtf(__uint_as_float((unsigned)kL));
    const float hi_tau = (sq * (1.0f + rel) * 1.000001f + E) * 1.00001f;
    if (hi_tau > rho) {
      if (rho > 2.0f * diag) return false;
      r_lo = 0.0f;
      r_hi = 0.0f;
      rho = hi_tau * 1.02f;
      continue;
    }
    const float lo_tau = (sq * (1.0f - rel) * 0.999999f - E) * 0.99999f;
    const float tlo = (lo_tau - E) / (1.0f + rel);
    const float thi = (hi_tau + E) / (1.0f - rel);
    const unsigned long long Tlo = tlo > 0.0f ? (unsigned long long)__float_as_uint(tlo * tlo * 0.99999f) : 0ull;
    const unsigned long long Thi = (unsigned long long)__float_as_uint(thi * thi * 1.00001f);
    if (Thi > (unsigned long long)__float_as_uint(rhof2)) return false;   // band reaches past the ball
    int p_lo = 0, p_hi = 0;
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      p_lo += __popc(__ballot_sync(FULL, k[t] < Tlo));
      p_hi += __popc(__ballot_sync(FULL, k[t] <= Thi));
    }
    const int nb = p_hi - p_lo;
    if (nb > kBand || p_lo > L - 1) return false;
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      const int e = t * 32 + lane;
      if (e < p_lo) row[1 + e] = r[t];
      else if (e < p_hi) qi.band[e - p_lo] = r[t];
    }
    if (lane == 0) {
      qi.state = 2;
      qi.p_lo = p_lo;
      qi.nb = nb;
      qi.need = L - p_lo;
    }
    dk = sq;
    return true;
  }
  return false;
}

template <int KPL> struct KnnShape {
  static constexpr int KB = KPL <= 2 ? 4 : 2 * KPL;       // buffer of 32*KB candidates (>= 2K)
  static constexpr int WPB = KPL <= 2 ? 8 : (KPL <= 4 ? 4 : 2);
  static constexpr int MINB = KPL <= 1 ? 3 : 1;           // blocks per SM the registers allow
};

template <int KPL, bool kMixed>
__global__ void __launch_bounds__(KnnShape<KPL>::WPB * 32, KnnShape<KPL>::MINB) k_knn(KnnArgs A) {
  constexpr int KB = KnnShape<KPL>::KB, WPB = KnnShape<KPL>::WPB;
  __shared__ QInfo info[WPB][32];
  __shared__ CandBuf<KB> buf[WPB];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int L = A.K - 1;
  for (long long base = warp * 32; base < A.N; base += nwarps * 32) {
    // ---- phase A: per query, warp-cooperative FP32/INT search
    int prev_b = -1;
    float prev_dk = 0.0f;
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
      // the previous query of the chunk in the same cell gives a close radius
      // the previous query of the chunk (a neighbour in cell order) gives a close radius
      float rho = (prev_b == b && prev_dk > 0.0f) ? 1.15f * prev_dk : rho_start(G, A.cstart, Q, L, lane);
      float dk = 0.0f;
      bool done = false;
      if (kMixed) done = query_buf<KB, true>(A, G, Gd, Q, q, lane, rho, qi, buf[w], dk);
      if (!done) done = query_buf<KB, false>(A, G, Gd, Q, q, lane, rho, qi, buf[w], dk);
      prev_b = b;
      prev_dk = done ? dk : 0.0f;
      if (!done) {
        // no acceptable radius: keep the row valid (the particle against itself) with an
        // infinite measure, so the particle gets no rate; the status reports it
        int* row = A.nbr + q * (long long)A.K;
        for (int k = lane; k < A.K; k += 32) row[k] = (int)q;
        if (lane == 0) {
          qi.state = 0;
          A.dist[q] = 0.0;
          A.V[q] = __longlong_as_double(0x7FF0000000000000ll);
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
    // ---- phase C: members by ascending caller index.  The rows and caller indices of
    // kG queries are loaded before any of them is sorted, so their latencies overlap.
    constexpr int kG = KPL <= 1 ? 4 : (KPL <= 2 ? 2 : 1);
    for (int q0 = 0; q0 < 32; q0 += kG) {
      int jj[kG][KPL], rr[kG][KPL];
      bool live[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        const long long q = base + q0 + g;
        live[g] = q < A.N && info[w][q0 + g].state != 0;
#pragma unroll
        for (int t = 0; t < KPL; ++t) {
          const int e = t * 32 + lane;
          rr[g][t] = (live[g] && e < L) ? A.nbr[q * (long long)A.K + 1 + e] : -1;
        }
      }
#pragma unroll
      for (int g = 0; g < kG; ++g)
#pragma unroll
        for (int t = 0; t < KPL; ++t) jj[g][t] = rr[g][t] >= 0 ? __ldg(&A.perm[rr[g][t]]) : INT_MAX;
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        if (!live[g]) continue;
        const long long q = base + q0 + g;
        int* row = A.nbr + q * (long long)A.K;
        sort_by_index<KPL>(jj[g], rr[g], lane);
#pragma unroll
        for (int t = 0; t < KPL; ++t) {
          const int e = t * 32 + lane;
          if (e < L) row[1 + e] = rr[g][t];
        }
        if (lane == 0) row[0] = (int)q;
      }
    }
    __syncwarp();
  }
}

template <int KPL, bool kMixed>
static cudaError_t launch_knn_t(gd_ctx* c, const KnnArgs& A) {
  constexpr int kWarps = KnnShape<KPL>::WPB;
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
