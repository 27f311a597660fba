// k_knn.cu -- K nearest neighbours over the device cell list (Sect. 2.5.1).
//
// Lane = query.  Consecutive threads take consecutive query ranks (neighbouring cells),
// and every thread runs the whole search of its own particle.  The only shared resource
// is the warp's slice of shared memory, where lane l keeps its candidates: word w of
// entry e at [(w * CAP + e) * 33 + l], so lanes touching the same entry, or one lane
// walking its entries, never share a bank.
//
//  radius : 1.001 x the particle's d_i of the previous build when there is one (exact
//           when the particles did not move; after a push the radius search corrects it),
//           else an estimate from the particle count of the 27 cells around it;
//  scan   : the cell rows that meet the ball are produced row by row and consumed
//           candidate by candidate in one loop (the cell starts of the next row are
//           loaded while the current row is scanned); keys inside the ball are kept;
//  radius : grows or shrinks (bisection between radii known to hold too few / too many
//           candidates) until the ball holds between K-1 and CAP other particles;
//  keys   : FP64 form -- d^2 = (dx dx + dy dy) + dz dz in FP64 (no FMA, minimum image),
//           ties by caller index: the oracle's order exactly.
//           Mixed form -- FP32 D from cell-relative FP32 coordinates, ties by rank; with
//           |sqrt(D) - d| <= 10u sqrt(D) + E (u = 2^-24) keys below T_lo are certain
//           members and keys up to T_hi form a band ranked exactly in FP64.  A band wider
//           than kBand, a periodic axis covered whole, or no acceptable radius puts the
//           query on a list that the FP64 form then redoes.
//  output : d_i = sqrt of the (K-1)-th d^2, V_i with the flat-boundary caps, and the row:
//           the particle itself, then its members by ascending caller index.
#include <climits>

#include "gd_ctx.h"
#include "gd_physics.cuh"

namespace gd {

constexpr int kBand = 8;          // band entries resolved in FP64 per mixed query
constexpr int kPad = 33;          // words per entry row of a warp's buffer (32 lanes + 1)

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
  const int* rank_of;
  int* nbr;
  double* dist;
  double* V;
  float* pref32;                  // mixed form: FP32 rate prefactor (NULL in the FP64 form)
  double* dprev;                  // caller order: d_i of the last build (0: unknown)
  StateDev* st;
  int* redo;                      // mixed form: queries the FP64 form redoes
  unsigned long long* redo_n;
  const int* list;                // FP64 redo pass: the queries to process
  const unsigned long long* list_n;
  float rfac;                     // first radius = rfac d_i of the last build
};

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

// One row segment: cells [ca, cb) of the concatenated cell arrays, the x shift of a
// periodic wrap (cells) and the row's y and z offsets from the query cell.
struct Seg {
  long long ca, cb;
  int xsh, dyc, dzc;
};

// Rows (z outer, y inner) of the ball of radius rs around the query, one segment per
// call (a row wrapped across a periodic x edge gives two).
struct RowIter {
  int lz, hz, ly, hy;
  int iz, iyu;
  bool fy, pending;
  float rs2;
  Seg pend;
};

__device__ __forceinline__ void rows_begin(const Grid32& G, const QueryPos& Q, float rs, RowIter& it, bool& amb) {
  bool fz;
  axis_range32(G, 2, Q.iz, Q.fz, rs, it.lz, it.hz, fz);
  axis_range32(G, 1, Q.iy, Q.fy, rs, it.ly, it.hy, it.fy);
  if (it.fy && G.per) amb = true;
  it.iz = it.lz;
  it.iyu = it.ly;
  it.pending = false;
  it.rs2 = rs * rs * 1.00002f;
  if (it.hy < it.ly) it.iz = it.hz + 1;   // empty
}

__device__ __forceinline__ bool rows_next(const Grid32& G, const QueryPos& Q, RowIter& it, Seg& s, bool& amb) {
  if (it.pending) {
    it.pending = false;
    s = it.pend;
    if (++it.iyu > it.hy) { it.iyu = it.ly; ++it.iz; }
    return true;
  }
  const int dimx = G.dim[0], dimy = G.dim[1];
  while (it.iz <= it.hz) {
    const int iz = it.iz, iyu = it.iyu;
    bool got = false;
    const float dz = slab_dist32(G, 2, Q.iz, Q.fz, iz);
    const float dy = it.fy ? 0.0f : slab_dist32(G, 1, Q.iy, Q.fy, iyu);
    const float dyz2 = dy * dy + dz * dz;
    if (dyz2 <= it.rs2) {
      const float xr = sqrtf(fmaxf(it.rs2 - dyz2, 0.0f));
      int lx, hx;
      bool fx;
      axis_range32(G, 0, Q.ix, Q.fx, xr, lx, hx, fx);
      if (lx <= hx) {
        if (fx && G.per) amb = true;
        int iy = iyu;
        if (G.per) { iy %= dimy; if (iy < 0) iy += dimy; }
        const long long rowc = G.cell_off + (long long)dimx * (iy + (long long)dimy * iz);
        int kx = 0, a0 = lx, e0 = hx;
        if (G.per && !fx) {
          kx = floordiv(lx, dimx);
          a0 = lx - kx * dimx;
          e0 = hx - kx * dimx;
        }
        const int e1 = e0 < dimx ? e0 : dimx - 1;
        s.ca = rowc + a0;
        s.cb = rowc + e1 + 1;
        s.xsh = kx * dimx;
        s.dyc = iyu - Q.iy;
        s.dzc = iz - Q.iz;
        if (e0 >= dimx) {
          it.pending = true;
          it.pend.ca = rowc;
          it.pend.cb = rowc + (e0 - dimx) + 1;
          it.pend.xsh = (kx + 1) * dimx;
          it.pend.dyc = s.dyc;
          it.pend.dzc = s.dzc;
          return true;             // the row advances after its second segment
        }
        got = true;
      }
    }
    if (++it.iyu > it.hy) { it.iyu = it.ly; ++it.iz; }
    if (got) return true;
  }
  return false;
}

__device__ __forceinline__ double sample_volume_reduced(const InstDev& P, double d, double x, double y);

__device__ __forceinline__ double sample_volume(const InstDev& P, double d, double x, double y) {
  if (P.kernel_mode != GD_KERNEL_PHYSICAL) return 1.0;
  if (P.model != GD_MODEL_3D) return sample_volume_reduced(P, d, x, y);
  double V = 4.0 * kPi * d * d * d / 3.0;
  if (P.geometry == GD_GEOM_DISK) {
    const double R2 = x * x + y * y;
    const double a = P.R_in + d, bo = P.R_out - d;
    // clear of both edges by a relative 1e-12, far above the rounding of R2 and of the
    // squares: no cap applies and R is not needed
    if (R2 > a * a * (1.0 + 1e-12) && bo > 0.0 && R2 < bo * bo * (1.0 - 1e-12)) return V;
    double R = sqrt(R2);
    double h = R - P.R_in;
    if (h > 0.0 && h < d) V -= kPi * (d - h) * (d - h) * (2.0 * d + h) / 3.0;
    h = P.R_out - R;
    if (h > 0.0 && h < d) V -= kPi * (d - h) * (d - h) * (2.0 * d + h) / 3.0;
  }
  return V;
}

// Reduced models (Sect. 2.5.1), (x, y) the query's coordinates in its model: the sampled
// area (a disk of radius d less the circular segments beyond a radial edge taken as a
// straight line; the 1D annulus [R - d, R + d] clipped at the edges) times 2 pi R (2D
// radial-polar: a toroidal volume) or times the vertical length sqrt(2 pi (H_i^2 + H_j^2))
// of the Gaussian average with H_i = H_j = H_g(R_i) (vertically integrated models).
__device__ __forceinline__ double sample_volume_reduced(const InstDev& P, double d, double x, double y) {
  double R;
  if (P.geometry == GD_GEOM_PATCH) R = P.r0 + x;
  else if (P.model == GD_MODEL_RPHI) R = __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
  else R = x;
  double A;
  if (P.model == GD_MODEL_R) {
    const double lo = R - d > P.R_in ? R - d : P.R_in;
    const double hi = R + d < P.R_out ? R + d : P.R_out;
    A = kPi * (hi * hi - lo * lo);
  } else {
    A = kPi * d * d;
    if (P.geometry == GD_GEOM_DISK) {
      double h = R - P.R_in;
      if (h > 0.0 && h < d) A -= d * d * acos(h / d) - h * sqrt(d * d - h * h);
      h = P.R_out - R;
      if (h > 0.0 && h < d) A -= d * d * acos(h / d) - h * sqrt(d * d - h * h);
    }
  }
  if (P.model == GD_MODEL_RZ) return A * 2.0 * kPi * R;
  const Gas g = gas_RZ(P, R, 0.0);
  return A * sqrt(2.0 * kPi * (g.H * g.H + g.H * g.H));
}

// Radius estimate from the particle count of the 27 cells around the query.
__device__ __forceinline__ float rho_start(const Grid32& G, const int* __restrict__ cstart, const QueryPos& Q,
                                           int L) {
  int n = 0, nc = 0;
  for (int c = 0; c < 27; ++c) {
    const int dx = c % 3 - 1, dy = (c / 3) % 3 - 1, dz = c / 9 - 1;
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
      const long long cc = G.cell_off + ix + (long long)G.dim[0] * (iy + (long long)G.dim[1] * iz);
      n += __ldg(&cstart[cc + 1]) - __ldg(&cstart[cc]);
      nc += 1;
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

__device__ __forceinline__ float grow(float rho, int found, int L, int cap) {
  // few found: the count says little, so grow by at least a quarter
  const float g = cbrtf(0.5f * (float)(L + cap) / (float)(found > 0 ? found : 1));
  return rho * fminf(fmaxf(g, 4 * found >= L ? 1.01f : 1.25f), 3.0f);
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

// ---------------------------------------------------------------- the lane's buffer
// kMixed: word 0 = bits of the FP32 D, word 1 = rank.  FP64: words 0/1 = low/high bits of
// d^2, word 2 = caller index.  Entries compare as (key, tie) with unsigned integers
// (non-negative floats order like their bit patterns).
template <int CAP, bool kMixed>
struct LaneBuf {
  static constexpr int NW = kMixed ? 2 : 3;
  uint32_t* b;
  __device__ __forceinline__ uint32_t& w(int word, int e) const { return b[(word * CAP + e) * kPad]; }
  __device__ __forceinline__ unsigned long long key(int e) const {
    if (kMixed) return ((unsigned long long)w(0, e) << 32) | w(1, e);
    return ((unsigned long long)w(1, e) << 32) | w(0, e);
  }
  __device__ __forceinline__ void swap(int a, int b2) const {
#pragma unroll
    for (int k = 0; k < NW; ++k) { const uint32_t t = w(k, a); w(k, a) = w(k, b2); w(k, b2) = t; }
  }
  // Leaves the L smallest of entries [0, n) in [0, L) (any order) by moving the largest
  // remaining entry to the tail n - L times (the radius keeps n - L small); returns the
  // index of the largest of them, the L-th smallest.
  __device__ __forceinline__ int select(int n, int L) const {
    for (int m = n; m > L; --m) {
      const int im = argmax(m);
      if (im != m - 1) swap(im, m - 1);
    }
    return argmax(L);
  }
  // index of the largest of entries [0, m), the running maximum kept in registers
  __device__ __forceinline__ int argmax(int m) const {
    int im = 0;
    unsigned long long km = key(0);
    uint32_t jm = kMixed ? 0u : w(2, 0);
    for (int e = 1; e < m; ++e) {
      const unsigned long long ke = key(e);
      if (kMixed) {
        if (ke > km) { km = ke; im = e; }
      } else {
        const uint32_t je = w(2, e);
        if (ke > km || (ke == km && je > jm)) { km = ke; jm = je; im = e; }
      }
    }
    return im;
  }
};

// Candidates of the ball of radius rho; keys inside it go to the buffer (the first CAP of
// them).  Returns how many were inside.
// kRow1: a one-row grid (the 1D radial model) packs the x cell in all the bits of w.
template <int CAP, bool kMixed, bool kRow1>
__device__ __forceinline__ int scan_ball(const KnnArgs& A, const Grid32& G, const GridDev& Gd, const QueryPos& Q,
                                         long long q, float rho, const LaneBuf<CAP, kMixed>& buf, bool& amb) {
  const float rel = 10.0f * 5.9604645e-8f;
  const float E = Gd.E32;
  const float rf = (rho * (1.0f + 2.0f * rel) + 2.0f * E) * 1.000001f;
  const float rhof2 = rf * rf * 1.000001f;
  const double rho2 = (double)rho * (double)rho;
  const double bx = Gd.box[0], by = Gd.box[1];
  const int* __restrict__ cstart = A.cstart;
  RowIter it;
  rows_begin(G, Q, rho, it, amb);
  // rows in order; the cell starts of the next row are loaded before the current row is
  // scanned.  Neighbouring queries mostly share their rows, so the lanes of a warp walk
  // the same candidates together.
  Seg cur, nxt;
  cur.xsh = cur.dyc = cur.dzc = 0;
  bool has_cur = rows_next(G, Q, it, cur, amb);
  int ca = 0, cb = 0;
  if (has_cur) { ca = __ldg(cstart + cur.ca); cb = __ldg(cstart + cur.cb); }
  int n_in = 0;
  while (has_cur) {
    nxt.xsh = nxt.dyc = nxt.dzc = 0;
    const bool has_nxt = rows_next(G, Q, it, nxt, amb);
    int na = 0, nb = 0;
    if (has_nxt) { na = __ldg(cstart + nxt.ca); nb = __ldg(cstart + nxt.cb); }
    const float dycf = (float)cur.dyc * G.cs[1], dzcf = (float)cur.dzc * G.cs[2];
    const int xoff = cur.xsh - Q.ix;
    if (kMixed) {
      // four candidates per step, their loads issued together
      for (int r0 = ca; r0 < cb; r0 += 4) {
        float4 p[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = r0 + u < cb ? __ldg(A.pos32 + r0 + u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = r0 + u;
          if (r >= cb || r == (int)q) continue;
          const int ixj = __float_as_int(p[u].w) & (kRow1 ? 0x7FFFFFFF : 2047);
          const float dx = (p[u].x - Q.fx) + (float)(ixj + xoff) * G.cs[0];
          const float dy = (p[u].y - Q.fy) + dycf;
          const float dz = (p[u].z - Q.fz) + dzcf;
          const float D = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          if (D <= rhof2) {
            if (n_in < CAP) { buf.w(0, n_in) = __float_as_uint(D); buf.w(1, n_in) = (uint32_t)r; }
            ++n_in;
          }
        }
      }
    } else {
    for (int r = ca; r < cb; ++r) {
      if (r == (int)q) continue;
      {
        long long jj;
        const double d2 = d2_fp64(A.pos64, r, Q.x, Q.y, Q.z, bx, by, jj);
        if (d2 <= rho2) {
          if (n_in < CAP) {
            const unsigned long long kb = (unsigned long long)__double_as_longlong(d2);
            buf.w(0, n_in) = (uint32_t)kb;
            buf.w(1, n_in) = (uint32_t)(kb >> 32);
            if (LaneBuf<CAP, kMixed>::NW > 2) buf.w(2, n_in) = (uint32_t)jj;
          }
          ++n_in;
        }
      }
    }
    }
    cur = nxt;
    ca = na;
    cb = nb;
    has_cur = has_nxt;
  }
  return n_in;
}

// Search of one query.  On success the buffer holds the members in entries [0, L)
// (unsorted) -- the mixed form their ranks (word 1), the FP64 form their caller indices
// (word 0) -- and d2max is the (K-1)-th d^2.  The output gathers the rest itself.
// Returns false when no acceptable radius was found (mixed: also when the FP32 keys
// cannot decide the members).
template <int CAP, bool kMixed, bool kRow1>
__device__ bool lane_query(const KnnArgs& A, const Grid32& G, const GridDev& Gd, const QueryPos& Q, long long q,
                           float rho, const LaneBuf<CAP, kMixed>& buf, double& d2max) {
  const int L = A.K - 1;
  const float E = Gd.E32;
  const float rel = 10.0f * 5.9604645e-8f;
  const double bx = Gd.box[0], by = Gd.box[1];
  const float diag = sqrtf((float)G.dim[0] * G.dim[0] * G.cs[0] * G.cs[0] +
                           (float)G.dim[1] * G.dim[1] * G.cs[1] * G.cs[1] +
                           (float)G.dim[2] * G.dim[2] * G.cs[2] * G.cs[2]);
  float r_lo = 0.0f, r_hi = 0.0f;    // radii known to hold too few / too many candidates
  for (int att = 0; att < 64; ++att) {
    bool amb = false;
    const int n_in = scan_ball<CAP, kMixed, kRow1>(A, G, Gd, Q, q, rho, buf, amb);
    if (kMixed && amb) return false;
    // a radius that held too few or too many is rescaled by the count towards the middle
    // of the acceptable range [L, CAP] (count ~ rho^3), then bisected once both are known
    if (n_in < L) {
      if (rho > 2.0f * diag) return false;
      r_lo = rho;
      rho = r_hi > 0.0f ? sqrtf(r_lo * r_hi) : grow(rho, n_in, L, CAP);
      continue;
    }
    if (n_in > CAP) {
      r_hi = rho;
      rho = r_lo > 0.0f ? sqrtf(r_lo * r_hi) : rho * fmaxf(cbrtf(0.5f * (float)(L + CAP) / (float)n_in), 0.3f);
      continue;
    }
    const int iL = buf.select(n_in, L);
    if (!kMixed) {
      // exact keys: the L smallest are the members
      d2max = __longlong_as_double((long long)(((unsigned long long)buf.w(1, iL) << 32) | buf.w(0, iL)));
      for (int e = 0; e < L; ++e) buf.w(0, e) = buf.w(2, e);
      return true;
    }
    // FP32 bounds with relative margins far above their own rounding
    const float sq = sqrtf(__uint_as_float(buf.w(0, iL)));
    const float hi_tau = (sq * (1.0f + rel) * 1.000001f + E) * 1.00001f;
    if (hi_tau > rho) {
      if (rho > 2.0f * diag) return false;
      r_lo = 0.0f;
      r_hi = 0.0f;
      rho = hi_tau * 1.02f;
      continue;
    }
    const float rf = (rho * (1.0f + 2.0f * rel) + 2.0f * E) * 1.000001f;
    const float rhof2 = rf * rf * 1.000001f;
    const float lo_tau = (sq * (1.0f - rel) * 0.999999f - E) * 0.99999f;
    const float tlo = (lo_tau - E) / (1.0f + rel);
    const float thi = (hi_tau + E) / (1.0f - rel);
    const uint32_t Tlo = tlo > 0.0f ? __float_as_uint(tlo * tlo * 0.99999f) : 0u;
    const uint32_t Thi = __float_as_uint(thi * thi * 1.00001f);
    if (Thi > __float_as_uint(rhof2)) return false;   // band reaches past the ball
    // certain members (key < T_lo) compacted to the front; band ranks set aside
    int p_lo = 0, nb = 0;
    int br[kBand];
    for (int e = 0; e < n_in; ++e) {
      const uint32_t k = buf.w(0, e);
      if (k < Tlo) {
        buf.w(1, p_lo++) = buf.w(1, e);
      } else if (k <= Thi) {
        if (nb == kBand) return false;
        br[nb++] = (int)buf.w(1, e);
      }
    }
    const int need = L - p_lo;
    if (need < 1 || need > nb) return false;
    // exact FP64 keys of the band, the `need` smallest by (d^2, caller index); the keys
    // are compared as bit patterns (non-negative doubles order like them), on the integer
    // units rather than the FP64 pipe
    unsigned long long bd[kBand];
    long long bj[kBand];
    for (int t = 0; t < nb; ++t)
      bd[t] = (unsigned long long)__double_as_longlong(d2_fp64(A.pos64, br[t], Q.x, Q.y, Q.z, bx, by, bj[t]));
    unsigned long long kmax = 0;
    int wr = p_lo;
    for (int t = 0; t < nb; ++t) {
      int rank = 0;
      for (int u = 0; u < nb; ++u)
        if (bd[u] < bd[t] || (bd[u] == bd[t] && bj[u] < bj[t])) rank++;
      if (rank < need) {
        buf.w(1, wr++) = (uint32_t)br[t];
        kmax = kmax > bd[t] ? kmax : bd[t];
      }
    }
    d2max = __longlong_as_double((long long)kmax);
    return true;
  }
  return false;
}

// Ascending sort of 32 keys held in registers (bitonic network, fully unrolled).
__device__ __forceinline__ void bitonic32(uint32_t (&c)[32]) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const uint32_t a = c[i], b = c[l];
          const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
          if ((i & k) == 0) { c[i] = lo; c[l] = hi; } else { c[i] = hi; c[l] = lo; }
        }
      }
    }
  }
}

template <int CAP> struct KnnShape {
  // warps per block: buffers (2 words mixed, 3 FP64) of up to four warps within about
  // 100 KB of shared memory per block
  static constexpr int bytes(bool mixed) { return (mixed ? 2 : 3) * CAP * kPad * 4; }
  static constexpr int wpb(bool mixed) {
    return bytes(mixed) * 4 <= 104 * 1024 ? 4 : (bytes(mixed) * 2 <= 104 * 1024 ? 2 : 1);
  }
};

// kRow1: a context of 1D radial instances (their one-row grids pack the x cell in all the
// bits of w; the 1D model cannot share a context with the others).
template <int CAP, bool kMixed, bool kRow1>
__global__ void __launch_bounds__(128, CAP <= 40 && kMixed ? 6 : 4) k_knn(KnnArgs A) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  LaneBuf<CAP, kMixed> buf;
  buf.b = smem + (size_t)w * LaneBuf<CAP, kMixed>::NW * CAP * kPad + lane;
  const int L = A.K - 1;
  const long long total = A.list ? (long long)*A.list_n : A.N;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const long long q = A.list ? (long long)A.list[t] : t;
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
    Q.ix = kRow1 ? pk : pk & 2047;
    Q.iy = kRow1 ? 0 : (pk >> 11) & 2047;
    Q.iz = kRow1 ? 0 : (pk >> 22) & 1023;
    Q.fx = f.x; Q.fy = f.y; Q.fz = f.z;
    const double2* pp = reinterpret_cast<const double2*>(A.pos64 + q);
    const double2 a0 = __ldg(pp), a1 = __ldg(pp + 1);
    Q.x = a0.x; Q.y = a0.y; Q.z = a1.x;
    const int ci = (int)__double_as_longlong(a1.y);   // caller index
    // radius: the last build's d_i when known, else the neighbourhood's density
    const double dp = A.dprev[ci];
    const float csmax = fmaxf(G.cs[0], fmaxf(G.cs[1], G.cs[2]));
    float rho = (dp > 0.0 && dp < 1e30) ? A.rfac * (float)dp : 0.0f;
    if (!(rho > 1e-4f * csmax)) rho = rho_start(G, A.cstart, Q, L);
    double d2max = 0.0;
    const bool ok = lane_query<CAP, kMixed, kRow1>(A, G, Gd, Q, q, rho, buf, d2max);
    int* row = A.nbr + q * (long long)A.K;
    if (ok) {
      row[0] = (int)q;
      // Sort keys: the caller index.  In the mixed form, when the caller indices leave
      // room, it carries the member's buffer entry in its low kEB bits, so that the rank is
      // read back from shared memory instead of gathered from rank_of (2^22 disk, K = 32:
      // 5.14 -> 4.94 ms per build; with the 40-entry buffer the gathers had measured
      // slightly faster).
      constexpr int kEB = CAP <= 64 ? 6 : CAP <= 128 ? 7 : CAP <= 256 ? 8 : 9;
      const bool packed = kMixed && A.N <= (1LL << (32 - kEB));
      auto sort_key = [&](int e) -> uint32_t {
        if (!kMixed) return buf.w(0, e);
        const uint32_t c = (uint32_t)__ldg(&A.perm[buf.w(1, e)]);
        return packed ? (c << kEB) | (uint32_t)e : c;
      };
      auto rank_of_key = [&](uint32_t k) -> int {
        return packed ? (int)buf.w(1, (int)(k & ((1u << kEB) - 1u))) : __ldg(&A.rank_of[k]);
      };
      if constexpr (CAP <= 40) {
        // K <= 32: the members' sort keys ordered in registers
        uint32_t cs[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) cs[e] = e < L ? sort_key(e) : 0xFFFFFFFFu;
        bitonic32(cs);
#pragma unroll
        for (int e = 0; e < 31; ++e)
          if (e < L) row[1 + e] = rank_of_key(cs[e]);
      } else if constexpr (CAP == 64) {
        // K <= 48: each half of the members' sort keys ordered in registers and put back
        // in word 0 (word 1 keeps the mixed form's ranks), then the halves merged
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          uint32_t cs[32];
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int i = 32 * h + e;
            cs[e] = i < L ? sort_key(i) : 0xFFFFFFFFu;
          }
          bitonic32(cs);
#pragma unroll
          for (int e = 0; e < 32; ++e) buf.w(0, 32 * h + e) = cs[e];
        }
        const int n1 = L < 32 ? L : 32;
        int i = 0, j = 32;
        uint32_t a = buf.w(0, 0), bq = buf.w(0, 32);   // past a half's members: 0xFFFFFFFF
        for (int k = 0; k < L; ++k) {
          const bool first = a < bq;
          const uint32_t key = first ? a : bq;
          if (first) { ++i; a = i < n1 ? buf.w(0, i) : 0xFFFFFFFFu; }
          else { ++j; bq = j < L ? buf.w(0, j) : 0xFFFFFFFFu; }
          if (packed) row[1 + k] = rank_of_key(key);
          else buf.w(1, k) = key;
        }
        if (!packed) {
#pragma unroll 4
          for (int k = 0; k < L; ++k) row[1 + k] = __ldg(&A.rank_of[buf.w(1, k)]);
        }
      } else {
        // K > 48: runs of 32 members' sort keys ordered in registers and put back in word
        // 0 (word 1 keeps the mixed form's ranks), then the runs merged
        constexpr int NR = (CAP + 31) / 32;
#pragma unroll 1
        for (int h = 0; h < NR && 32 * h < L; ++h) {
          uint32_t cs[32];
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int i = 32 * h + e;
            cs[e] = i < L ? sort_key(i) : 0xFFFFFFFFu;
          }
          bitonic32(cs);
#pragma unroll
          for (int e = 0; e < 32; ++e)
            if (32 * h + e < L) buf.w(0, 32 * h + e) = cs[e];
        }
        uint32_t hd[NR];      // each run's next key (0xFFFFFFFF when it is used up)
        int ps[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) {
          ps[c] = 32 * c;
          hd[c] = ps[c] < L ? buf.w(0, ps[c]) : 0xFFFFFFFFu;
        }
        for (int k = 0; k < L; ++k) {
          uint32_t key = hd[0];
          int bi = 0;
#pragma unroll
          for (int c = 1; c < NR; ++c)
            if (hd[c] < key) { key = hd[c]; bi = c; }
#pragma unroll
          for (int c = 0; c < NR; ++c) {
            if (c == bi) {
              ++ps[c];
              const int end = 32 * c + 32 < L ? 32 * c + 32 : L;
              hd[c] = ps[c] < end ? buf.w(0, ps[c]) : 0xFFFFFFFFu;
            }
          }
          if (packed) row[1 + k] = rank_of_key(key);
          else buf.w(1, k) = key;
        }
        if (!packed) {
#pragma unroll 4
          for (int k = 0; k < L; ++k) row[1 + k] = __ldg(&A.rank_of[buf.w(1, k)]);
        }
      }
      const double d = sqrt(d2max);
      A.dist[q] = d;
      const double Vq = sample_volume(A.P[b], d, Q.x, Q.y);
      A.V[q] = Vq;
      if (A.pref32) A.pref32[q] = (float)rate_prefactor(A.P[b], Vq, A.K, true);
      A.dprev[ci] = d;
    } else if (kMixed) {
      // the FP64 form redoes it
      const unsigned long long slot = atomicAdd(A.redo_n, 1ull);
      A.redo[slot] = (int)q;
      atomicAdd((unsigned long long*)&A.st[A.P[b].unit0].knn_redo, 1ull);
    } else {
      // no acceptable radius: keep the row valid (the particle against itself) with an
      // infinite measure, so the particle gets no rate; the status reports it
      for (int k = 0; k < A.K; ++k) row[k] = (int)q;
      A.dist[q] = 0.0;
      A.V[q] = __longlong_as_double(0x7FF0000000000000ll);
      if (A.pref32) A.pref32[q] = 0.0f;
      A.dprev[ci] = 0.0;
      set_status(&A.st[A.P[b].unit0], GD_ST_KNN);
    }
  }
}

template <int CAP, bool kMixed, bool kRow1>
static cudaError_t launch_knn_t(gd_ctx* c, const KnnArgs& A) {
  constexpr int kWarps = KnnShape<CAP>::wpb(kMixed);
  const int bs = kWarps * 32;
  const int smem = kWarps * KnnShape<CAP>::bytes(kMixed);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_knn<CAP, kMixed, kRow1>, bs, smem);
  if (per_sm < 1) per_sm = 1;
  long long blocks = (long long)c->num_sms * per_sm;
  if (!A.list) {
    const long long want = (A.N + bs - 1) / bs;
    if (blocks > want) blocks = want;
  }
  if (blocks < 1) blocks = 1;
  k_knn<CAP, kMixed, kRow1><<<(int)blocks, bs, smem, c->stream>>>(A);
  return cudaGetLastError();
}

template <int CAP, bool kMixed>
static cudaError_t prepare_t() {
  constexpr int kWarps = KnnShape<CAP>::wpb(kMixed);
  const int smem = kWarps * KnnShape<CAP>::bytes(kMixed);
  cudaError_t e = cudaFuncSetAttribute(k_knn<CAP, kMixed, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_knn<CAP, kMixed, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

template <bool kMixed>
static cudaError_t prepare_cap(int K) {
  if (K <= 32) return prepare_t<34, kMixed>();
  if (K <= 48) return prepare_t<64, kMixed>();
  if (K <= 80) return prepare_t<96, kMixed>();
  if (K <= 128) return prepare_t<144, kMixed>();
  return prepare_t<272, kMixed>();
}

// Shared-memory opt-in of the neighbour kernels this context launches (once, before any
// launch or graph capture).
cudaError_t knn_prepare(gd_ctx* c) {
  cudaError_t e = prepare_cap<false>(c->K);
  if (e == cudaSuccess && c->precision == GD_MIXED) e = prepare_cap<true>(c->K);
  // the wider buffer of a build after particles moved (K <= 32)
  if (e == cudaSuccess && c->K <= 32) e = prepare_cap<false>(48);
  if (e == cudaSuccess && c->K <= 32 && c->precision == GD_MIXED) e = prepare_cap<true>(48);
  return e;
}

template <int CAP, bool kMixed>
static cudaError_t launch_both(gd_ctx* c, const KnnArgs& A) {
  return c->any_model_r ? launch_knn_t<CAP, kMixed, true>(c, A) : launch_knn_t<CAP, kMixed, false>(c, A);
}

template <bool kMixed>
static cudaError_t launch_cap(gd_ctx* c, const KnnArgs& A, bool wide) {
  // buffer capacity: the K-1 members plus room for the radius margin.  Static builds start
  // at 1.001 d_i, so for K <= 32 a 34-entry buffer holds the ball, and its 36 KB per block
  // with at most 80 registers lets 6 blocks share an SM (a 40-entry buffer allowed 5: 5.53
  // against 5.18 ms per build of the 2^22 disk); after particles moved, the K-th distance
  // is uncertain and K <= 32 takes the 64-entry buffer
  if (c->K <= 32) return wide ? launch_both<64, kMixed>(c, A) : launch_both<34, kMixed>(c, A);
  if (c->K <= 48) return launch_both<64, kMixed>(c, A);
  if (c->K <= 80) return launch_both<96, kMixed>(c, A);
  if (c->K <= 128) return launch_both<144, kMixed>(c, A);
  return launch_both<272, kMixed>(c, A);
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
  A.rank_of = c->d_rank_of;
  A.nbr = c->d_nbr;
  A.dist = c->d_dist;
  A.V = c->d_V;
  A.pref32 = c->d_pref32;
  A.dprev = c->d_dprev;
  A.st = c->d_state;
  A.redo = c->d_redo;
  A.redo_n = c->d_counters + 1;
  A.list = nullptr;
  A.list_n = nullptr;
  // static particles: d_i of the last build is exact, and 1.001 d_i (with the search's own
  // rounding margins) holds the K-1 others and little else: the scan's overscan shrinks with
  // the ball (1.02 d_i took 6.11 ms per build of the 2^22 disk, 1.001 d_i 5.59 ms); after a
  // move the K-th distance scatters around it, so the first radius aims at the middle of the
  // buffer's range instead
  const bool wide = c->moved;
  A.rfac = c->moved ? 1.045f : 1.001f;
  c->moved = false;
  time_begin(c, 1);
  cudaError_t e = cudaSuccess;
  if (c->precision == GD_MIXED) {
    e = cudaMemsetAsync(A.redo_n, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = launch_cap<true>(c, A, wide);
    // the queries the FP32 keys could not decide, in the FP64 form
    KnnArgs B = A;
    B.list = c->d_redo;
    B.list_n = A.redo_n;
    if (e == cudaSuccess) e = launch_cap<false>(c, B, wide);
    c->launches += 2;
  } else {
    e = launch_cap<false>(c, A, wide);
    c->launches += 1;
  }
  time_end(c);
  return e;
}

}  // namespace gd
