// gd_noalloc.cu -- gd_neighbors_fixed: the neighbour search of one instance with its
// scratch in a fixed device array, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host program that has already reserved the
// device's memory for its own pool (a new allocation would fail or fragment it), or a
// latency-bound loop that cannot afford cudaMalloc's implicit device synchronisation.
// This entry point allocates nothing.  Its scratch (cell counts and starts, cell-ordered
// positions, the grid) lives in one file-scope __device__ array of GD_FIXED_SCRATCH_BYTES
// bytes, which every GPU that loads the library holds until the process exits.
//
// The result is the same as gd_build_neighbors' nbr_out / d_out for a one-instance
// FP64 context: slot 0 the particle itself, then the K-1 nearest others by (d^2, index)
// in ascending index order; d = distance to the farthest of them.
#include <cmath>
#include <climits>
#include <mutex>

#include "gd_common.cuh"

namespace gdfix {

using gd::dbl_ord;
using gd::ord_dbl;

constexpr long long kMaxN = GD_FIXED_MAX_PARTICLES;
constexpr long long kMaxCells = 4 * kMaxN;
constexpr int kMaxK = GD_FIXED_MAX_K;
constexpr unsigned FULL = 0xffffffffu;

struct FixGrid {
  double lo[3], cs[3], inv[3], box[3];
  int dim[3];
  int per;
  unsigned long long bmin[3], bmax[3];
};

struct FixPos {
  double x, y, z;
  long long j;
};

constexpr size_t a256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffGrid = 0;
constexpr size_t kOffCount = a256(sizeof(FixGrid));
constexpr size_t kOffStart = kOffCount + a256(sizeof(int) * (kMaxCells + 1));
constexpr size_t kOffCell = kOffStart + a256(sizeof(int) * (kMaxCells + 1));
constexpr size_t kOffSlot = kOffCell + a256(sizeof(int) * kMaxN);
constexpr size_t kOffPos = kOffSlot + a256(sizeof(int) * kMaxN);
constexpr size_t kBytes = kOffPos + a256(sizeof(FixPos) * kMaxN);
static_assert(kBytes == GD_FIXED_SCRATCH_BYTES, "GD_FIXED_SCRATCH_BYTES must match the layout");

// The fixed scratch.  Host code must not use this name as an address: it is a host-side
// stand-in.  The device address comes from cudaGetSymbolAddress (see scratch_address).
static __device__ __align__(256) unsigned char g_scratch[kBytes];

struct Ptr {
  FixGrid* grid;
  int* count;
  int* start;
  int* cell;
  int* slot;
  FixPos* pos;
};

__device__ __forceinline__ Ptr ptrs(unsigned char* b) {
  return Ptr{reinterpret_cast<FixGrid*>(b + kOffGrid), reinterpret_cast<int*>(b + kOffCount),
             reinterpret_cast<int*>(b + kOffStart), reinterpret_cast<int*>(b + kOffCell),
             reinterpret_cast<int*>(b + kOffSlot), reinterpret_cast<FixPos*>(b + kOffPos)};
}

// every call starts from zero counts and empty bounds
__global__ void fk_clear(unsigned char* b) {
  Ptr p = ptrs(b);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t <= kMaxCells;
       t += (long long)gridDim.x * blockDim.x)
    p.count[t] = 0;
  if (blockIdx.x == 0 && threadIdx.x < 3) {
    p.grid->bmin[threadIdx.x] = ~0ull;
    p.grid->bmax[threadIdx.x] = 0ull;
  }
}

__global__ void fk_bounds(unsigned char* b, const double* __restrict__ x, const double* __restrict__ y,
                          const double* __restrict__ z, long long n) {
  Ptr p = ptrs(b);
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0, 0, 0};
  if (i < n) {
    unsigned long long o[3] = {dbl_ord(x[i]), dbl_ord(y[i]), dbl_ord(z[i])};
    for (int a = 0; a < 3; ++a) { mn[a] = o[a]; mx[a] = o[a]; }
  }
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[a] = min(mn[a], __shfl_xor_sync(FULL, mn[a], o));
      mx[a] = max(mx[a], __shfl_xor_sync(FULL, mx[a], o));
    }
  }
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 3; ++a) { atomicMin(&p.grid->bmin[a], mn[a]); atomicMax(&p.grid->bmax[a], mx[a]); }
}

// One thread: a uniform grid over the bounds (patch: the periodic box in x and y), at
// most kMaxCells cells.  The cell edge starts from cell_size or (volume / n)^(1/3), made
// finite and positive (coincident particles give a zero volume), and grows until the grid
// fits; if it still does not fit (a cell_size far below the extent, or non-finite bounds),
// one cell per axis keeps every cell index inside the scratch arrays, and the search stays
// exact, only slower.
__global__ void fk_grid(unsigned char* b, int geometry, double box_x, double box_y, double cell_size,
                        long long n) {
  Ptr p = ptrs(b);
  FixGrid& g = *p.grid;
  double lo[3], ext[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = ord_dbl(g.bmin[a]);
    ext[a] = ord_dbl(g.bmax[a]) - lo[a];
  }
  const bool per = geometry == GD_GEOM_PATCH;
  if (per) { lo[0] = -0.5 * box_x; ext[0] = box_x; lo[1] = -0.5 * box_y; ext[1] = box_y; }
  double emax = fmax(ext[0], fmax(ext[1], ext[2]));
  double vol = 1.0;
  for (int a = 0; a < 3; ++a) vol *= fmax(ext[a], 1e-6 * emax + 1e-300);
  double c = cell_size > 0.0 ? cell_size : cbrt(vol / (double)n);
  if (!(c > 0.0) || !isfinite(c)) c = emax > 0.0 && isfinite(emax) ? emax : 1.0;
  long long cells = 0;
  bool finite = true;
  for (int attempt = 0; attempt < 60; ++attempt) {
    cells = 1;
    finite = true;
    for (int a = 0; a < 3; ++a) {
      const bool pa = per && a < 2;
      const double e = pa ? ext[a] : ext[a] * (1.0 + 1e-9) + 1e-12 * emax + 1e-300;
      const double dd = pa ? floor(e / c) : ceil(e / c);
      const int dim = (int)fmin(fmax(dd, 1.0), 4096.0);
      g.lo[a] = lo[a];
      g.cs[a] = e / dim;
      g.inv[a] = dim / e;
      g.box[a] = pa ? ext[a] : 0.0;
      g.dim[a] = dim;
      cells *= dim;
      finite = finite && isfinite(g.lo[a]) && isfinite(g.cs[a]) && isfinite(g.inv[a]);
    }
    if (cells <= kMaxCells) break;
    c *= 2.0;
  }
  if (cells > kMaxCells || !finite) {
    for (int a = 0; a < 3; ++a) {
      const bool pa = per && a < 2;
      const double e = pa ? ext[a] : ext[a] * (1.0 + 1e-9) + 1e-12 * emax + 1e-300;
      g.lo[a] = isfinite(lo[a]) ? lo[a] : 0.0;
      g.cs[a] = isfinite(e) && e > 0.0 ? e : 1.0;
      g.inv[a] = 1.0 / g.cs[a];
      g.dim[a] = 1;
    }
  }
  g.per = per ? 1 : 0;
}

__device__ __forceinline__ int fcell(const FixGrid& g, int a, double v) {
  double t = floor((v - g.lo[a]) * g.inv[a]);
  const int d = g.dim[a];
  if (g.box[a] > 0.0) {
    t = fmin(fmax(t, -1e15), 1e15);
    long long k = (long long)t % d;
    if (k < 0) k += d;
    return (int)k;
  }
  return t < 0.0 ? 0 : (t >= (double)d ? d - 1 : (int)t);
}

__global__ void fk_count(unsigned char* b, const double* __restrict__ x, const double* __restrict__ y,
                         const double* __restrict__ z, long long n) {
  Ptr p = ptrs(b);
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const FixGrid& g = *p.grid;
  const int c = fcell(g, 0, x[i]) + g.dim[0] * (fcell(g, 1, y[i]) + g.dim[1] * fcell(g, 2, z[i]));
  p.cell[i] = c;
  p.slot[i] = atomicAdd(&p.count[c], 1);
}

// One block: exclusive scan of the counts of every cell of the grid.
__global__ void fk_scan(unsigned char* b) {
  Ptr p = ptrs(b);
  const FixGrid& g = *p.grid;
  const long long cells = (long long)g.dim[0] * g.dim[1] * g.dim[2];
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (long long base = 0; base < cells; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    const int v = i < cells ? p.count[i] : 0;
    int inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
      int s = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
      int si = s;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, si, o);
        if (lane >= o) si += t;
      }
      wsum[lane] = si - s;
    }
    __syncthreads();
    if (i < cells) p.start[i] = carry + wsum[w] + inc - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += wsum[w] + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) p.start[cells] = carry;
}

__global__ void fk_scatter(unsigned char* b, const double* __restrict__ x, const double* __restrict__ y,
                           const double* __restrict__ z, long long n) {
  Ptr p = ptrs(b);
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = p.start[p.cell[i]] + p.slot[i];
  p.pos[r] = FixPos{x[i], y[i], z[i], i};
}

template <int KPL>
__device__ __forceinline__ void fsort(int (&jj)[KPL], int lane) {
  constexpr int S = 32 * KPL;
  for (int k = 2; k <= S; k <<= 1)
    for (int s = k >> 1; s > 0; s >>= 1) {
      if (s >= 32) {
#pragma unroll
        for (int t = 0; t < KPL; ++t) {
          const int tp = t ^ (s >> 5);
          if (tp > t) {
            const bool up = ((t * 32 + lane) & k) == 0;
            if (up ? (jj[t] > jj[tp]) : (jj[t] < jj[tp])) { int a = jj[t]; jj[t] = jj[tp]; jj[tp] = a; }
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < KPL; ++t) {
          const int pj = __shfl_xor_sync(FULL, jj[t], s);
          const bool up = ((t * 32 + lane) & k) == 0;
          const bool lower = (lane & s) == 0;
          if ((lower == up) ? (pj < jj[t]) : (pj > jj[t])) jj[t] = pj;
        }
      }
    }
}

// Warp per query (cell order): exact FP64 keys (d^2 bits, index), ball scan over the cell
// rows with a growing radius until the ball holds the K-1 nearest others.
template <int KPL>
__global__ void __launch_bounds__(256) fk_knn(unsigned char* b, long long n, int K, int32_t* nbr_out,
                                              double* d_out) {
  Ptr p = ptrs(b);
  const FixGrid& g = *p.grid;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const int L = K - 1;
  for (long long q = warp; q < n; q += nw) {
    const FixPos Q = p.pos[q];
    double qxw = Q.x, qyw = Q.y;
    if (g.box[0] > 0.0) qxw = Q.x - g.box[0] * floor((Q.x - g.lo[0]) / g.box[0]);
    if (g.box[1] > 0.0) qyw = Q.y - g.box[1] * floor((Q.y - g.lo[1]) / g.box[1]);
    const double qw[3] = {qxw, qyw, Q.z};
    const double csmax = fmax(g.cs[0], fmax(g.cs[1], g.cs[2]));
    double rho = csmax;
    unsigned long long lk[KPL];
    int lj[KPL];
    bool ok = false;
    for (int att = 0; att < 80 && !ok; ++att) {
      for (int t = 0; t < KPL; ++t) { lk[t] = ~0ull; lj[t] = INT_MAX; }
      unsigned long long wk = ~0ull;
      int wj = INT_MAX;
      const double rs = rho * (1.0 + 1e-9);
      const double rho2 = rho * rho;
      int lo[3], hi[3];
      bool full[3];
      for (int a = 0; a < 3; ++a) {
        const double t0 = floor((qw[a] - rs - g.lo[a]) * g.inv[a]);
        const double t1 = floor((qw[a] + rs - g.lo[a]) * g.inv[a]);
        full[a] = false;
        if (g.box[a] > 0.0) {
          if (t1 - t0 + 1.0 >= g.dim[a]) { lo[a] = 0; hi[a] = g.dim[a] - 1; full[a] = true; }
          else { lo[a] = (int)t0; hi[a] = (int)t1; }
        } else {
          lo[a] = (int)fmax(t0, 0.0);
          hi[a] = (int)fmin(t1, (double)(g.dim[a] - 1));
        }
      }
      for (int iz = lo[2]; iz <= hi[2]; ++iz)
        for (int iyu = lo[1]; iyu <= hi[1]; ++iyu) {
          int iy = iyu;
          if (g.box[1] > 0.0) { iy %= g.dim[1]; if (iy < 0) iy += g.dim[1]; }
          for (int ixu = lo[0]; ixu <= hi[0]; ++ixu) {
            int ix = ixu;
            if (g.box[0] > 0.0) { ix %= g.dim[0]; if (ix < 0) ix += g.dim[0]; }
            const int c = ix + g.dim[0] * (iy + g.dim[1] * iz);
            const int ra = p.start[c], rb = p.start[c + 1];
            for (int base = ra; base < rb; base += 32) {
              const int r = base + lane;
              unsigned long long ck = ~0ull;
              int cj = INT_MAX;
              if (r < rb && r != (int)q) {
                const FixPos C = p.pos[r];
                double dx = C.x - Q.x, dy = C.y - Q.y, dz = C.z - Q.z;
                if (g.box[0] > 0.0) {
                  if (dx > 0.5 * g.box[0]) dx -= g.box[0]; else if (dx < -0.5 * g.box[0]) dx += g.box[0];
                  if (dy > 0.5 * g.box[1]) dy -= g.box[1]; else if (dy < -0.5 * g.box[1]) dy += g.box[1];
                }
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                if (d2 <= rho2) { ck = (unsigned long long)__double_as_longlong(d2); cj = (int)C.j; }
              }
              unsigned m = __ballot_sync(FULL, ck < wk || (ck == wk && cj < wj));
              while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const unsigned long long nk = __shfl_sync(FULL, ck, src);
                const int nj = __shfl_sync(FULL, cj, src);
                if (!(nk < wk || (nk == wk && nj < wj))) continue;
                int pos = 0;
                for (int t = 0; t < KPL; ++t)
                  pos += __popc(__ballot_sync(FULL, lk[t] < nk || (lk[t] == nk && lj[t] < nj)));
                for (int t = KPL - 1; t >= 0; --t) {
                  unsigned long long uk = __shfl_up_sync(FULL, lk[t], 1);
                  int uj = __shfl_up_sync(FULL, lj[t], 1);
                  const int tp = t > 0 ? t - 1 : 0;
                  const unsigned long long ck2 = __shfl_sync(FULL, lk[tp], 31);
                  const int cj2 = __shfl_sync(FULL, lj[tp], 31);
                  if (lane == 0 && t > 0) { uk = ck2; uj = cj2; }
                  const int gi = t * 32 + lane;
                  if (gi > pos) { lk[t] = uk; lj[t] = uj; }
                  else if (gi == pos) { lk[t] = nk; lj[t] = nj; }
                }
                unsigned long long kv = lk[0];
                int jv = lj[0];
                for (int t = 1; t < KPL; ++t)
                  if (t == ((L - 1) >> 5)) { kv = lk[t]; jv = lj[t]; }
                wk = __shfl_sync(FULL, kv, (L - 1) & 31);
                wj = __shfl_sync(FULL, jv, (L - 1) & 31);
              }
            }
          }
        }
      if (wk != ~0ull) {
        ok = true;
        int jj[KPL];
        for (int t = 0; t < KPL; ++t) jj[t] = (t * 32 + lane < L) ? lj[t] : INT_MAX;
        fsort<KPL>(jj, lane);
        int32_t* row = nbr_out + Q.j * (long long)K;
        for (int t = 0; t < KPL; ++t)
          if (t * 32 + lane < L) row[1 + t * 32 + lane] = jj[t];
        if (lane == 0) {
          row[0] = (int32_t)Q.j;
          if (d_out) d_out[Q.j] = sqrt(__longlong_as_double((long long)wk));
        }
      } else {
        rho *= 1.5;
      }
    }
    if (!ok) {
      int32_t* row = nbr_out + Q.j * (long long)K;
      for (int k = lane; k < K; k += 32) row[k] = -1;
      if (lane == 0 && d_out) d_out[Q.j] = -1.0;
    }
  }
}

// Device address of the fixed array, looked up once per device (with that device current)
// and kept for the life of the process: a cudaDeviceReset, which replaces the device's
// primary context, leaves the kept address stale, so the library is not used across one.
static std::mutex g_mu;
static void* g_addr[256];

static gd_status scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return GD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return GD_ERR_CUDA;
    g_addr[dev] = ptr;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return GD_OK;
}

}  // namespace gdfix

extern "C" gd_status gd_neighbors_fixed(const double* x, const double* y, const double* z, int64_t n,
                                        int32_t K, const gd_instance_params* params, int32_t* nbr_out,
                                        double* d_out, void* stream) {
  using namespace gdfix;
  if (!x || !y || !z || !params || !nbr_out) return GD_ERR_ARG;
  if (K < 2 || K > kMaxK || n < K) return GD_ERR_ARG;
  if (n > kMaxN) return GD_ERR_CAPACITY;
  if (params->geometry != GD_GEOM_PATCH && params->geometry != GD_GEOM_DISK) return GD_ERR_ARG;
  if (params->geometry == GD_GEOM_PATCH && !(params->box_x > 0.0 && params->box_y > 0.0)) return GD_ERR_ARG;
  if (params->model != GD_MODEL_3D) return GD_ERR_ARG;   // 3D positions only
  unsigned char* base = nullptr;
  gd_status st = scratch_address(&base);
  if (st != GD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = (int)((n + 255) / 256);
  fk_clear<<<256, 256, 0, s>>>(base);
  fk_bounds<<<nb, 256, 0, s>>>(base, x, y, z, n);
  fk_grid<<<1, 1, 0, s>>>(base, params->geometry, params->box_x, params->box_y, params->cell_size, n);
  fk_count<<<nb, 256, 0, s>>>(base, x, y, z, n);
  fk_scan<<<1, 1024, 0, s>>>(base);
  fk_scatter<<<nb, 256, 0, s>>>(base, x, y, z, n);
  const int kb = (int)((n * 32 + 255) / 256);
  if (K <= 32) fk_knn<1><<<kb, 256, 0, s>>>(base, n, K, nbr_out, d_out);
  else fk_knn<2><<<kb, 256, 0, s>>>(base, n, K, nbr_out, d_out);
  return cudaGetLastError() == cudaSuccess ? GD_OK : GD_ERR_CUDA;
}
