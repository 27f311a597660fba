// k_cells.cu -- device cell list: per-instance bounds and grid, counting sort by cell,
// and the frozen partner snapshot of the interval (Sect. 2.5.1, 2.5.3).
//
// A counting sort replaces the paper's KD-tree / Morton hierarchy: every particle gets
// the cell of its instance's uniform grid, cells are counted with atomics, an exclusive
// scan gives cell starts, and a scatter writes the particle, in cell order, into the
// rank-space arrays that the neighbour, rate and sampling kernels stream through.
#include <vector>

#include "gd_ctx.h"
#include "gd_physics.cuh"

namespace gd {

constexpr int kScanTile = 2048;   // cells per block in the scan

// ---------------------------------------------------------------- stats
// Sums of M, M m and M s per instance (a10): per-tile partials over a fixed stride and a
// fixed tree, then each instance's partials in tile order.  Every launch adds in the same
// order, so the result is bitwise reproducible.
__device__ __forceinline__ void block_tree3(double (&sh)[3][256], double a0, double a1, double a2) {
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = a2;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_stats_tile(TileMap tm, const InstDev* __restrict__ P,
                                                    const double* __restrict__ s, const double* __restrict__ M,
                                                    double* part) {
  __shared__ double sh[3][256];
  int b;
  long long lo, hi;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  if (tile_range(tm, blockIdx.x, b, lo, hi)) {
    const InstDev& p = P[b];
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const double si = s[i], Mi = M[i];
      a0 += Mi;
      a1 += Mi * grain_mass(p, si);
      a2 += Mi * si;
    }
  }
  block_tree3(sh, a0, a1, a2);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) part[3 * (long long)blockIdx.x + k] = sh[k][0];
}

__global__ void __launch_bounds__(256) k_stats_inst(const long long* __restrict__ tile_off,
                                                    const double* __restrict__ part, double* out) {
  __shared__ double sh[3][256];
  const int b = blockIdx.x;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (long long t = tile_off[b] + threadIdx.x; t < tile_off[b + 1]; t += blockDim.x) {
    a0 += part[3 * t];
    a1 += part[3 * t + 1];
    a2 += part[3 * t + 2];
  }
  block_tree3(sh, a0, a1, a2);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) out[3 * b + k] = sh[k][0];
}

// ---------------------------------------------------------------- bounds
__global__ void k_bounds(TileMap tm, const InstDev* __restrict__ P, const double* __restrict__ x,
                         const double* __restrict__ y, const double* __restrict__ z, StateDev* st) {
  int b;
  long long lo, hi;
  if (!tile_range(tm, blockIdx.x, b, lo, hi)) return;
  const int model = P[b].model;
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0, 0, 0};
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double X, Y, Z;
    model_pos(model, x[i], y[i], z[i], X, Y, Z);
    unsigned long long o[3] = {dbl_ord(X), dbl_ord(Y), dbl_ord(Z)};
#pragma unroll
    for (int a = 0; a < 3; ++a) { mn[a] = min(mn[a], o[a]); mx[a] = max(mx[a], o[a]); }
  }
  __shared__ unsigned long long smn[3][32], smx[3][32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
      mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
    }
    if (lane == 0) { smn[a][w] = mn[a]; smx[a][w] = mx[a]; }
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    int a = threadIdx.x;
    unsigned long long m0 = ~0ull, m1 = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { m0 = min(m0, smn[a][k]); m1 = max(m1, smx[a][k]); }
    atomicMin(&st[P[b].unit0].bmin[a], m0);
    atomicMax(&st[P[b].unit0].bmax[a], m1);
  }
}

// ---------------------------------------------------------------- grid choice
// Derived fields of a grid from its origin, edges, dimensions and periodic box: the FP32
// copies and the bound E32 of the FP32 distance error.
__device__ __forceinline__ void grid_finish(GridDev& g, bool per) {
  double X = 0.0;
  for (int a = 0; a < 3; ++a) X = fmax(X, 0.5 * g.cs[a] * g.dim[a]);
  if (per) X += fmax(g.box[0], g.box[1]);
  g.X32 = X;
  double csmax = 0.0;
  for (int a = 0; a < 3; ++a) {
    g.cs32[a] = (float)g.cs[a];
    g.inv32[a] = (float)g.inv[a];
    csmax = fmax(csmax, g.cs[a]);
  }
  // |sqrt(D32) - d| <= 10 u sqrt(D32) + E, u = 2^-24: cell-relative FP32 coordinates
  // (<= u cell each), the FP32 cell offsets, and the FP64 rounding of the mirror
  g.E32 = (float)((16.0 * 0x1p-24 * csmax + 32.0 * 0x1p-53 * X) * 1.0001);
  g.periodic = per ? 1 : 0;
}

// Uniform grid of one instance over its data bounds (patch: the periodic box in x and
// y): cell edge from the instance or cell_factor (V_box / n)^(1/3), times grow, the x edge
// divided by xsplit.  Returns the number of cells (cell_off is left to the caller).
__device__ long long grid_of(const InstDev& P, const StateDev& S, double cell_factor, int xsplit, double grow,
                             GridDev& g) {
  double lo[3], ext[3];
  for (int a = 0; a < 3; ++a) {
    const double mn = ord_dbl(S.bmin[a]), mx = ord_dbl(S.bmax[a]);
    lo[a] = mn;
    ext[a] = mx - mn;
  }
  const bool per = P.geometry == GD_GEOM_PATCH;
  if (per) { lo[0] = -0.5 * P.box_x; ext[0] = P.box_x; lo[1] = -0.5 * P.box_y; ext[1] = P.box_y; }
  const double tiny = 1e-300;
  double vol = 1.0, emax = 0.0;
  for (int a = 0; a < 3; ++a) emax = fmax(emax, ext[a]);
  for (int a = 0; a < 3; ++a) vol *= fmax(ext[a], 1e-6 * emax + tiny);
  double c;
  if (P.cell_size > 0.0) {
    c = P.cell_size;
  } else if (P.model == GD_MODEL_3D) {
    c = cell_factor * cbrt(vol / (double)P.n);
  } else {
    // reduced models: the points span 2 (RZ, RPHI) or 1 (R) axes
    double span = 1.0;
    int D = 0;
    for (int a = 0; a < 3; ++a)
      if (ext[a] > 1e-9 * emax) { span *= ext[a]; ++D; }
    const double per = span / (double)P.n;
    c = cell_factor * (D >= 3 ? cbrt(per) : D == 2 ? sqrt(per) : D == 1 ? per : 1.0);
    if (!(c > 0.0)) c = emax + tiny;
  }
  c *= grow;
  long long cells = 1;
  for (int a = 0; a < 3; ++a) {
    const bool pa = per && a < 2;
    const double e = pa ? ext[a] : ext[a] * (1.0 + 1e-9) + 1e-12 * emax + tiny;
    const double ca = a == 0 ? c / xsplit : c;
    const double dimd = pa ? floor(e / ca) : ceil(e / ca);
    // per-axis cell limits: the FP32 mirror packs the cell coordinates as 11 + 11 + 10
    // bits; the 1D radial model has y = z = 0 and gives x all the bits
    const double cap = P.model == GD_MODEL_R ? (a == 0 ? 16777216.0 : 1.0) : (a < 2 ? 2048.0 : 1024.0);
    const int dim = (int)fmin(fmax(dimd, 1.0), cap);
    g.lo[a] = lo[a];
    g.cs[a] = e / dim;
    g.inv[a] = dim / e;
    g.dim[a] = dim;
    g.box[a] = pa ? ext[a] : 0.0;
    g.ctr[a] = lo[a] + 0.5 * e;
    cells *= dim;
  }
  grid_finish(g, per);
  return cells;
}

__device__ __forceinline__ long long block_sum64(long long v, long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  long long t = 0;
  for (int k = 0; k < nw; ++k) t += sh[k];
  __syncthreads();
  return t;
}

// One block: every thread takes instances b = tid, tid + blockDim, ...  The grids of all
// instances for a common growth factor; while the total exceeds the capacity every edge
// grows.  Then the concatenated cell offsets (a block scan in chunks of blockDim
// instances) and the bounds reset for the next build.
__global__ void k_grid(const InstDev* __restrict__ P, StateDev* st, GridDev* grid, int n_inst,
                       double cell_factor, int xsplit, long long cell_cap, unsigned long long* used) {
  __shared__ long long sh[33];
  const int tid = threadIdx.x, nthr = blockDim.x;
  double grow = 1.0;
  bool fits = false;
  for (int attempt = 0; attempt < 40; ++attempt) {
    long long mine = 0;
    for (int b = tid; b < n_inst; b += nthr) {
      GridDev g;
      mine += grid_of(P[b], st[P[b].unit0], cell_factor, xsplit, grow, g);
    }
    const long long total = block_sum64(mine, sh);
    if (total <= cell_cap) { fits = true; break; }
    grow *= 1.1 * cbrt((double)total / (double)cell_cap);
  }
  if (fits) {
    long long carry = 0;
    for (int base = 0; base < n_inst; base += nthr) {
      const int b = base + tid;
      GridDev g;
      const long long cells = b < n_inst ? grid_of(P[b], st[P[b].unit0], cell_factor, xsplit, grow, g) : 0;
      // exclusive scan of the chunk's cell counts
      long long inc = cells;
      const int lane = tid & 31, w = tid >> 5, nw = nthr >> 5;
      for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      __syncthreads();
      if (lane == 31) sh[w] = inc;
      __syncthreads();
      long long before = 0, chunk = 0;
      for (int k = 0; k < nw; ++k) {
        if (k < w) before += sh[k];
        chunk += sh[k];
      }
      if (b < n_inst) {
        g.cell_off = carry + before + inc - cells;
        grid[b] = g;
      }
      carry += chunk;
    }
    if (tid == 0) *used = (unsigned long long)carry;
  } else {
    // capacity exhausted: one cell per instance keeps every index in bounds (the search
    // stays exact, only slower) and the status reports it
    for (int b = tid; b < n_inst; b += nthr) {
      GridDev g;
      grid_of(P[b], st[P[b].unit0], cell_factor, xsplit, grow, g);
      for (int a = 0; a < 3; ++a) {
        const double e = g.cs[a] * g.dim[a];
        g.dim[a] = 1;
        g.cs[a] = e;
        g.inv[a] = 1.0 / e;
      }
      grid_finish(g, P[b].geometry == GD_GEOM_PATCH);
      g.cell_off = b;
      grid[b] = g;
      set_status(&st[P[b].unit0], GD_ST_CAPACITY);
    }
    if (tid == 0) *used = (unsigned long long)n_inst;
  }
  __syncthreads();
  for (int b = tid; b < n_inst; b += nthr)
    for (int a = 0; a < 3; ++a) { st[P[b].unit0].bmin[a] = ~0ull; st[P[b].unit0].bmax[a] = 0ull; }
}

__global__ void k_cell_count(TileMap tm, const InstDev* __restrict__ P, const GridDev* __restrict__ grid,
                             const double* __restrict__ x, const double* __restrict__ y,
                             const double* __restrict__ z, int* __restrict__ count, int* __restrict__ cell_of,
                             int* __restrict__ slot, long long cell_cap) {
  int b;
  long long lo, hi;
  if (!tile_range(tm, blockIdx.x, b, lo, hi)) return;
  const GridDev g = grid[b];
  const int model = P[b].model;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double X, Y, Z;
    model_pos(model, x[i], y[i], z[i], X, Y, Z);
    int ix = axis_cell(g, 0, X), iy = axis_cell(g, 1, Y), iz = axis_cell(g, 2, Z);
    long long c = g.cell_off + ix + (long long)g.dim[0] * (iy + (long long)g.dim[1] * iz);
    if (c >= cell_cap) c = cell_cap - 1;    // only after a capacity failure (status set)
    cell_of[i] = (int)c;
    slot[i] = atomicAdd(&count[c], 1);
  }
}

// ---------------------------------------------------------------- exclusive scan
__device__ __forceinline__ int block_excl_scan(int v, int* sh, int& total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    int s = lane < nw ? sh[lane] : 0;
    int si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += t;
    }
    if (lane < nw) sh[lane] = si - s;
    if (lane == 31) sh[32] = si;
  }
  __syncthreads();
  total = sh[32];
  int r = inc - v + sh[w];
  __syncthreads();
  return r;
}

// phase 1: per-tile sums
// The scan covers the cells the grid uses (k_grid writes their number to *used); tiles
// past it only report a zero sum.
__global__ void k_scan_reduce(const int* __restrict__ in, const unsigned long long* __restrict__ used,
                              int* __restrict__ sums) {
  const long long n = (long long)*used;
  long long base = (long long)blockIdx.x * kScanTile;
  if (base > n) { if (threadIdx.x == 0) sums[blockIdx.x] = 0; return; }
  int acc = 0;
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
    long long i = base + k;
    if (i < n) acc += in[i];
  }
  __shared__ int sh[33];
  int total;
  block_excl_scan(acc, sh, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// phase 2: exclusive scan of the tile sums (one block)
__global__ void k_scan_sums(int* sums, int nt) {
  __shared__ int sh[33];
  int carry = 0;
  for (int base = 0; base < nt; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < nt ? sums[i] : 0;
    int total;
    int e = block_excl_scan(v, sh, total);
    if (i < nt) sums[i] = e + carry;
    carry += total;
  }
}

// phase 3: scan inside each tile plus its offset; out[0..n] (out[n] = the total)
__global__ void k_scan_final(const int* __restrict__ in, const unsigned long long* __restrict__ used,
                             const int* __restrict__ sums, int* __restrict__ out) {
  const long long n = (long long)*used;
  long long base = (long long)blockIdx.x * kScanTile;
  if (base > n) return;
  constexpr int per = kScanTile / 256;
  int v[per];
  int acc = 0;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    long long i = base + threadIdx.x * per + k;
    v[k] = i < n ? in[i] : 0;
    acc += v[k];
  }
  __shared__ int sh[33];
  int total;
  int e = block_excl_scan(acc, sh, total) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < per; ++k) {
    long long i = base + threadIdx.x * per + k;
    if (i <= n) out[i] = e;
    e += v[k];
  }
}

// Zeroes the counts of the cells the grid uses (and the end entry).
__global__ void k_zero_counts(int* __restrict__ count, const unsigned long long* __restrict__ used) {
  const long long n = (long long)*used;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (long long)gridDim.x * blockDim.x)
    count[i] = 0;
}

// ---------------------------------------------------------------- scatter + snapshot
// Frozen partner properties of one particle at rank r (Sect. 2.5.3): s, m, N = M/m, 1/m,
// the represented mass, and the mixed form's FP32 copy (N scaled by 2^-64).
template <bool kMixed>
__device__ __forceinline__ void put_snapshot(const InstDev& p, long long r, double si, double Mi,
                                             Snap64* __restrict__ snap64, float4* __restrict__ snap32,
                                             double* __restrict__ Mr) {
  const double m = grain_mass(p, si);
  const double im = 1.0 / m;
  const double N = Mi * im;
  Snap64 sn;
  sn.s = si; sn.m = m; sn.N = N; sn.inv_m = im;
  snap64[r] = sn;
  Mr[r] = Mi;
  if (kMixed) snap32[r] = make_float4((float)si, (float)m, (float)(N * 0x1p-64), (float)im);
}

// The gas disk's (R, Z) of a particle from its search coordinates (model_pos): a patch sits
// at R = R_0 + x; the 2D radial-polar and 1D models search (R, Z, 0) and (R, 0, 0); the 3D
// and radial-azimuthal models hold (x, y, z) and (x, y, 0).
__device__ __forceinline__ void gas_coords(const InstDev& p, double X, double Y, double Z, double& R, double& Zg) {
  if (p.geometry == GD_GEOM_PATCH) R = p.r0 + X;
  else if (p.model == GD_MODEL_RZ || p.model == GD_MODEL_R) R = X;
  else R = sqrt(X * X + Y * Y);
  Zg = p.model == GD_MODEL_RZ ? Y : Z;
}

// The snapshot alone, at unchanged ranks (positions did not move since the last build); the
// mixed form's FP32 (R, Z, M) stay, its fine bin follows the new size.
template <bool kMixed>
__global__ void k_snapshot(TileMap tm, const InstDev* __restrict__ P, const double* __restrict__ s,
                           const double* __restrict__ M, const int* __restrict__ rank_of,
                           Snap64* __restrict__ snap64, float4* __restrict__ snap32, double* __restrict__ Mr,
                           float4* __restrict__ gx) {
  int b;
  long long lo, hi;
  if (!tile_range(tm, blockIdx.x, b, lo, hi)) return;
  const InstDev p = P[b];
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int r = rank_of[i];
    put_snapshot<kMixed>(p, r, s[i], M[i], snap64, snap32, Mr);
    if (kMixed) reinterpret_cast<float*>(gx + r)[3] = __int_as_float(fine_bin(s[i]));
  }
}

// Spatial groups: the round's particles (the list act) broadcast -- their live sizes become
// the sizes partners read (sb, caller order) -- and their snapshot entries follow; the other
// particles' entries keep their last broadcast.
template <bool kMixed>
__global__ void k_broadcast_snapshot(const unsigned long long* __restrict__ total, const int* __restrict__ act,
                                     const long long* __restrict__ off, int n_inst, const InstDev* __restrict__ P,
                                     const int* __restrict__ perm, const double* __restrict__ s,
                                     double* __restrict__ sb, const double* __restrict__ M,
                                     Snap64* __restrict__ snap64, float4* __restrict__ snap32,
                                     double* __restrict__ Mr, float4* __restrict__ gx) {
  const long long n = (long long)*total;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = act[t];
    const int ci = perm[r];
    const double si = s[ci];
    sb[ci] = si;
    put_snapshot<kMixed>(P[inst_of(off, n_inst, r)], r, si, M[ci], snap64, snap32, Mr);
    if (kMixed) reinterpret_cast<float*>(gx + r)[3] = __int_as_float(fine_bin(si));
  }
}

template <bool kMixed>
__global__ void k_scatter(TileMap tm, const InstDev* __restrict__ P, const GridDev* __restrict__ grid,
                          const double* __restrict__ x, const double* __restrict__ y,
                          const double* __restrict__ z, const double* __restrict__ s,
                          const double* __restrict__ M, const int* __restrict__ cell_of,
                          const int* __restrict__ slot, const int* __restrict__ start,
                          int* __restrict__ perm, int* __restrict__ rank_of, Pos64* __restrict__ pos64,
                          float4* __restrict__ pos32, Snap64* __restrict__ snap64,
                          float4* __restrict__ snap32, double* __restrict__ Mr, float4* __restrict__ gx) {
  int b;
  long long lo, hi;
  if (!tile_range(tm, blockIdx.x, b, lo, hi)) return;
  const InstDev p = P[b];
  const GridDev g = grid[b];
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    int r = start[cell_of[i]] + slot[i];
    double xi, yi, zi;
    model_pos(p.model, x[i], y[i], z[i], xi, yi, zi);
    const double si = s[i], Mi = M[i];
    perm[r] = (int)i;
    rank_of[i] = r;
    Pos64 q;
    q.x = xi; q.y = yi; q.z = zi; q.j = i;
    pos64[r] = q;
    put_snapshot<kMixed>(p, r, si, Mi, snap64, snap32, Mr);
    if (kMixed) {
      double R, Zg;
      gas_coords(p, xi, yi, zi, R, Zg);
      gx[r] = make_float4((float)R, (float)Zg, (float)Mi, __int_as_float(fine_bin(si)));
    }
    {
      // FP32 mirror relative to the particle's own cell origin (|coord| <= cell edge),
      // cell coordinates packed in w (11 + 11 + 10 bits); periodic axes use the
      // wrapped coordinate so that the cell and the offset agree.
      // the cell from its index (integer work instead of three FP64 floors)
      const int rem = cell_of[i] - (int)g.cell_off;
      const int ix = rem % g.dim[0], iy = (rem / g.dim[0]) % g.dim[1], iz = rem / (g.dim[0] * g.dim[1]);
      double xw = xi, yw = yi;
      if (g.box[0] > 0.0) xw = xi - g.box[0] * floor((xi - g.lo[0]) / g.box[0]);
      if (g.box[1] > 0.0) yw = yi - g.box[1] * floor((yi - g.lo[1]) / g.box[1]);
      float fx = (float)(xw - (g.lo[0] + ix * g.cs[0]));
      float fy = (float)(yw - (g.lo[1] + iy * g.cs[1]));
      float fz = (float)(zi - (g.lo[2] + iz * g.cs[2]));
      pos32[r] = make_float4(fx, fy, fz, __int_as_float(ix | (iy << 11) | (iz << 22)));
    }
  }
}

}  // namespace gd

// ---------------------------------------------------------------- launcher
namespace gd {

int num_tiles(gd_ctx* c) { return c->n_tiles; }

std::vector<long long> tile_table(const std::vector<long long>& off) {
  std::vector<long long> t(off.size(), 0);
  for (size_t b = 0; b + 1 < off.size(); ++b) t[b + 1] = t[b] + (off[b + 1] - off[b] + kTile - 1) / kTile;
  return t;
}

// The sizes partners read: the live sizes, or with spatial groups each particle's size as its
// group last broadcast it.
static const double* partner_sizes(gd_ctx* c) { return c->grouped ? c->d_sb : c->s; }

// Partner snapshot refresh at unchanged ranks (gd_collide's later intervals).
cudaError_t launch_snapshot(gd_ctx* c) {
  time_begin(c, 0);
  const int nt = num_tiles(c);
  const double* s = partner_sizes(c);
  if (c->precision == GD_MIXED)
    k_snapshot<true><<<nt, 256, 0, c->stream>>>(tile_map(c), c->d_inst, s, c->M, c->d_rank_of, c->d_snap64,
                                                c->d_snap32, c->d_Mr, c->d_gx);
  else
    k_snapshot<false><<<nt, 256, 0, c->stream>>>(tile_map(c), c->d_inst, s, c->M, c->d_rank_of, c->d_snap64,
                                                 c->d_snap32, c->d_Mr, c->d_gx);
  time_end(c);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_broadcast_snapshot(gd_ctx* c) {
  time_begin(c, 0);
  const unsigned long long* total = c->d_counters + 10;
  const int grid = c->num_sms * 8;
  if (c->precision == GD_MIXED)
    k_broadcast_snapshot<true><<<grid, 256, 0, c->stream>>>(total, c->d_act, c->d_off, c->n_inst, c->d_inst,
                                                            c->d_perm, c->s, c->d_sb, c->M, c->d_snap64,
                                                            c->d_snap32, c->d_Mr, c->d_gx);
  else
    k_broadcast_snapshot<false><<<grid, 256, 0, c->stream>>>(total, c->d_act, c->d_off, c->n_inst, c->d_inst,
                                                             c->d_perm, c->s, c->d_sb, c->M, c->d_snap64,
                                                             c->d_snap32, c->d_Mr, c->d_gx);
  time_end(c);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_stats(gd_ctx* c, double* d_sums) {
  time_begin(c, 6);
  double* part = d_sums + 3 * (long long)c->n_inst;
  k_stats_tile<<<c->n_tiles, 256, 0, c->stream>>>(tile_map(c), c->d_inst, c->s, c->M, part);
  k_stats_inst<<<c->n_inst, 256, 0, c->stream>>>(c->d_tile_off, part, d_sums);
  time_end(c);
  return cudaGetLastError();
}

cudaError_t launch_cells(gd_ctx* c) {
  TileMap tm = tile_map(c);
  int nt = num_tiles(c);
  cudaStream_t st = c->stream;
  time_begin(c, 0);
  k_bounds<<<nt, 256, 0, st>>>(tm, c->d_inst, c->x, c->y, c->z, c->d_state);
  // cells in use (written by k_grid): the zeroing and the scan stop there
  unsigned long long* used = c->d_counters + 2;
  k_grid<<<1, 256, 0, st>>>(c->d_inst, c->d_state, c->d_grid, c->n_inst, c->cell_factor, c->cell_xsplit,
                           c->cell_cap, used);
  const long long ncell = c->cell_cap;
  k_zero_counts<<<c->num_sms * 8, 256, 0, st>>>(c->d_cell_count, used);
  k_cell_count<<<nt, 256, 0, st>>>(tm, c->d_inst, c->d_grid, c->x, c->y, c->z, c->d_cell_count, c->d_cell_of,
                                   c->d_slot, c->cell_cap);
  int nst = (int)((ncell + kScanTile) / kScanTile);   // tiles of cells [0, ncell] (end entry included)
  k_scan_reduce<<<nst, 256, 0, st>>>(c->d_cell_count, used, c->d_scan_tmp);
  k_scan_sums<<<1, 1024, 0, st>>>(c->d_scan_tmp, nst);
  k_scan_final<<<nst, 256, 0, st>>>(c->d_cell_count, used, c->d_scan_tmp, c->d_cell_start);
  const double* s = partner_sizes(c);
  if (c->precision == GD_MIXED)
    k_scatter<true><<<nt, 256, 0, st>>>(tm, c->d_inst, c->d_grid, c->x, c->y, c->z, s, c->M,
                                        c->d_cell_of, c->d_slot, c->d_cell_start, c->d_perm,
                                        c->d_rank_of, c->d_pos64, c->d_pos32, c->d_snap64,
                                        c->d_snap32, c->d_Mr, c->d_gx);
  else
    k_scatter<false><<<nt, 256, 0, st>>>(tm, c->d_inst, c->d_grid, c->x, c->y, c->z, s, c->M,
                                         c->d_cell_of, c->d_slot, c->d_cell_start, c->d_perm,
                                         c->d_rank_of, c->d_pos64, c->d_pos32, c->d_snap64,
                                         c->d_snap32, c->d_Mr, c->d_gx);
  time_end(c);
  c->launches += 8;
  return cudaGetLastError();
}

}  // namespace gd
