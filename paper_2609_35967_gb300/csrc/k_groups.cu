// k_groups.cu -- spatial groups (Sect. 2.5.3): the units (one group of one instance), their
// members in a fixed order, the interaction masks, the rounds (which groups broadcast and
// take a new interval) and the schedule of their levels under the ratio-16 rule.
//
// A unit's fine-bin sums run over its caller indices in ascending order (d_gperm), in tiles
// that never straddle a unit, so that every reduction keeps a fixed order.  The group of a
// particle, its unit's members and the masks are taken at each neighbour build (positions are
// frozen inside a collision step).
#include "gd_ctx.h"

namespace gd {

// Per caller tile of an instance: each particle's unit, and the tile's count of each group.
__global__ void __launch_bounds__(256) k_group_assign(TileMap tm, const InstDev* __restrict__ P,
                                                      const double* __restrict__ x, const double* __restrict__ y,
                                                      int* __restrict__ unit_i, int* __restrict__ tcount) {
  __shared__ int cnt[kMaxSG];
  int b;
  long long lo, hi;
  if (!tile_range(tm, blockIdx.x, b, lo, hi)) return;
  const InstDev& p = P[b];
  for (int g = threadIdx.x; g < kMaxSG; g += blockDim.x) cnt[g] = 0;
  __syncthreads();
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int g = p.n_sg > 1 ? group_of(p, x[i], y[i]) : 0;
    unit_i[i] = p.unit0 + g;
    atomicAdd(&cnt[g], 1);    // integer counts: the same in every run
  }
  __syncthreads();
  for (int g = threadIdx.x; g < kMaxSG; g += blockDim.x) tcount[(long long)blockIdx.x * kMaxSG + g] = cnt[g];
}

// One block, a warp per unit: its members over its instance's tiles, then its first position
// in d_gperm (the instance's offset plus the members of its lower groups) and, by a warp scan
// over the tiles in order, each tile's first position for the unit; the units' fine-bin tile
// offsets (thread 0, in unit order); the interaction masks cleared for the new lists.
__global__ void k_group_scan(const InstDev* __restrict__ P, const long long* __restrict__ tile_off,
                             const int* __restrict__ unit_inst, int U, const int* __restrict__ tcount,
                             long long* __restrict__ tbase, long long* __restrict__ uoff,
                             long long* __restrict__ utile_off, StateDev* st, long long N) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int u = threadIdx.x >> 5; u < U; u += nw) {
    const int b = unit_inst[u], g = u - P[b].unit0;
    long long m = 0;
    for (long long t = tile_off[b] + lane; t < tile_off[b + 1]; t += 32) m += tcount[t * kMaxSG + g];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    if (lane == 0) {
      st[u].members = m;
      st[u].inter = 0ull;
    }
  }
  __syncthreads();
  for (int u = threadIdx.x >> 5; u < U; u += nw) {
    const int b = unit_inst[u], u0 = P[b].unit0, g = u - u0;
    long long base = P[b].off;
    for (int h = 0; h < g; ++h) base += st[u0 + h].members;
    if (lane == 0) uoff[u] = base;
    for (long long t0 = tile_off[b]; t0 < tile_off[b + 1]; t0 += 32) {
      const long long t = t0 + lane;
      const long long c = t < tile_off[b + 1] ? tcount[t * kMaxSG + g] : 0;
      long long incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (t < tile_off[b + 1]) tbase[t * kMaxSG + g] = base + incl - c;
      base += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int u = 0; u < U; ++u) {
      utile_off[u] = t;
      t += (st[u].members + kTile - 1) / kTile;
    }
    utile_off[U] = t;
    uoff[U] = N;
  }
}

// Per rank tile: the tile's count of each group (the ranks of an instance are tiled like its
// caller indices).
__global__ void __launch_bounds__(256) k_unit_count(TileMap tm, const InstDev* __restrict__ P,
                                                    const int* __restrict__ unit_r, int* __restrict__ tcount) {
  __shared__ int cnt[kMaxSG];
  int b;
  long long lo, hi;
  if (!tile_range(tm, blockIdx.x, b, lo, hi)) return;
  const int u0 = P[b].unit0;
  for (int g = threadIdx.x; g < kMaxSG; g += blockDim.x) cnt[g] = 0;
  __syncthreads();
  for (long long r = lo + threadIdx.x; r < hi; r += blockDim.x) atomicAdd(&cnt[unit_r[r] - u0], 1);
  __syncthreads();
  for (int g = threadIdx.x; g < kMaxSG; g += blockDim.x) tcount[(long long)blockIdx.x * kMaxSG + g] = cnt[g];
}

// Per tile of positions i (caller indices, or ranks): i's position in the unit-ordered
// permutation perm (stable: ascending i inside its unit) and, with rank_of given, its unit in
// rank order.  Chunks of blockDim particles; inside a warp equal groups are ranked by
// __match_any_sync, the warps of a chunk in warp order.
__global__ void __launch_bounds__(128) k_group_scatter(TileMap tm, const InstDev* __restrict__ P,
                                                       const int* __restrict__ unit_i,
                                                       const long long* __restrict__ tbase,
                                                       const int* __restrict__ rank_of, int* __restrict__ gperm,
                                                       int* __restrict__ unit_r) {
  constexpr int NW = 4;
  __shared__ long long run[kMaxSG];
  __shared__ int wcnt[NW][kMaxSG];
  int b;
  long long lo, hi;
  if (!tile_range(tm, blockIdx.x, b, lo, hi)) return;
  const int u0 = P[b].unit0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int g = threadIdx.x; g < kMaxSG; g += blockDim.x) run[g] = tbase[(long long)blockIdx.x * kMaxSG + g];
  for (int t = threadIdx.x; t < NW * kMaxSG; t += blockDim.x) (&wcnt[0][0])[t] = 0;
  __syncthreads();
  for (long long base = lo; base < hi; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    const bool valid = i < hi;
    const int ui = valid ? unit_i[i] : -1;
    const int g = valid ? ui - u0 : -1;
    const unsigned same = __match_any_sync(0xffffffffu, g);
    const int before = __popc(same & ((1u << lane) - 1u));
    if (valid && before == 0) wcnt[w][g] = __popc(same);
    __syncthreads();
    if (valid) {
      long long pos = run[g] + before;
      for (int ww = 0; ww < w; ++ww) pos += wcnt[ww][g];
      gperm[pos] = (int)i;
      if (rank_of) unit_r[rank_of[i]] = ui;
    }
    __syncthreads();
    for (int gg = threadIdx.x; gg < kMaxSG; gg += blockDim.x) {
      int add = 0;
      for (int ww = 0; ww < NW; ++ww) { add += wcnt[ww][gg]; wcnt[ww][gg] = 0; }
      run[gg] += add;
    }
    __syncthreads();
  }
}

// Interaction masks from the lists: bit h of unit u when a list of u holds a particle of
// group h of the same instance (made symmetric by the schedule).  An OR: any order.
__global__ void k_group_inter(long long N, int K, const int* __restrict__ nbr, const int* __restrict__ unit_r,
                              const int* __restrict__ unit_inst, const InstDev* __restrict__ P, StateDev* st) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int u = unit_r[r];
  const int u0 = P[unit_inst[u]].unit0;
  unsigned long long m = 0ull;
  for (int k = 1; k < K; ++k) {
    const int v = unit_r[nbr[r * K + k]];
    if (v != u) m |= 1ull << (v - u0);
  }
  if (m) atomicOr(&st[u].inter, m);
}

// One thread per instance with groups: a round.  A step whose groups all reached its end
// starts the next one (or, in a bounded collision step, idles); the round's clock is the
// earliest end of a scheduled interval, and its groups are those ending there.
__global__ void k_round_begin(const InstDev* __restrict__ P, StateDev* st, int n_inst) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_inst) return;
  const InstDev& p = P[b];
  if (p.n_sg <= 1) return;
  StateDev* S = st + p.unit0;
  const int G = p.n_sg;
  const long long full = 1LL << 60;
  bool open = false;
  for (int g = 0; g < G; ++g)
    if (S[g].members > 0 && S[g].remain_ticks > 0) open = true;
  if (!open) {
    if (S[0].hold) {
      for (int g = 0; g < G; ++g) S[g].active = 0;
      return;
    }
    for (int g = 0; g < G; ++g) { S[g].remain_ticks = full; S[g].level = -1; }
  }
  long long t = full;
  for (int g = 0; g < G; ++g)
    if (S[g].members > 0 && S[g].remain_ticks > 0 && full - S[g].remain_ticks < t) t = full - S[g].remain_ticks;
  for (int g = 0; g < G; ++g)
    S[g].active = (S[g].members > 0 && S[g].remain_ticks > 0 && full - S[g].remain_ticks == t) ? 1 : 0;
  S[0].clock = t;
  S[0].rounds++;
}

// One thread per instance with groups: the levels of the round's groups from their requests
// (k_interval), then their intervals committed.
//  - lo: the group ends inside the collision step (level k_fit at least) and is within 4 of
//    every interacting group in the middle of its interval; hi: no finer than 4 levels
//    beyond such a group (a delayed refinement), but never below lo (the step's end wins);
//  - among the round's interacting groups hi[g] <= hi[h] + 4 (not below lo[g]), iterated to
//    its fixed point; each group takes its request within [lo, hi];
//  - the coarser of two interacting groups of the round is refined until within 4.
// Both iterations are monotone, so their fixed points do not depend on the order.
__global__ void k_schedule(const InstDev* __restrict__ P, StateDev* st, int n_inst) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_inst) return;
  const InstDev& p = P[b];
  if (p.n_sg <= 1) return;
  StateDev* S = st + p.unit0;
  const int G = p.n_sg;
  unsigned long long inter[kMaxSG];
  for (int g = 0; g < G; ++g) inter[g] = S[g].inter;
  for (int g = 0; g < G; ++g)
    for (int h = 0; h < G; ++h)
      if ((S[h].inter >> g) & 1ull) inter[g] |= 1ull << h;
  int lo[kMaxSG], hi[kMaxSG], k[kMaxSG];
  bool any = false;
  for (int g = 0; g < G; ++g) {
    lo[g] = 0; hi[g] = 60; k[g] = S[g].level;
    if (!S[g].active) continue;
    any = true;
    int kf = 0;
    while (kf < 60 && (1LL << (60 - kf)) > S[g].remain_ticks) ++kf;
    lo[g] = kf;
    for (int h = 0; h < G; ++h) {
      if (h == g || S[h].active || S[h].members == 0 || S[h].level < 0) continue;
      if (!((inter[g] >> h) & 1ull)) continue;
      lo[g] = max(lo[g], S[h].level - 4);
      hi[g] = min(hi[g], S[h].level + 4);
    }
    if (hi[g] < lo[g]) hi[g] = lo[g];
  }
  if (!any) return;
  for (bool changed = true; changed;) {
    changed = false;
    for (int g = 0; g < G; ++g) {
      if (!S[g].active) continue;
      for (int h = 0; h < G; ++h) {
        if (h == g || !S[h].active || !((inter[g] >> h) & 1ull)) continue;
        const int cap = max(hi[h] + 4, lo[g]);
        if (cap < hi[g]) { hi[g] = cap; changed = true; }
      }
    }
  }
  for (int g = 0; g < G; ++g)
    if (S[g].active) k[g] = max(lo[g], min(S[g].k_req, hi[g]));
  for (bool changed = true; changed;) {
    changed = false;
    for (int g = 0; g < G; ++g) {
      if (!S[g].active) continue;
      for (int h = 0; h < G; ++h) {
        if (h == g || !S[h].active || !((inter[g] >> h) & 1ull)) continue;
        if (k[g] < k[h] - 4) { k[g] = k[h] - 4; changed = true; }
      }
    }
  }
  long long delayed = 0, breaks = 0;
  for (int g = 0; g < G; ++g) {
    if (!S[g].active) continue;
    if (k[g] < S[g].k_req) ++delayed;
    StateDev& Sg = S[g];
    const double dtc = Sg.tau > 0.0 ? Sg.tau : p.dt_coll;
    Sg.level = k[g];
    Sg.dt_exe = ldexp(dtc, -k[g]);
    Sg.remain_ticks -= 1LL << (60 - k[g]);
    Sg.dt_remain = ldexp((double)Sg.remain_ticks, -60) * dtc;
    Sg.interval_cur = Sg.interval_next;
    Sg.interval_next = Sg.interval_next + 1;
    Sg.events = 0;
    Sg.intervals++;
  }
  for (int g = 0; g < G; ++g)
    for (int h = g + 1; h < G; ++h) {
      if (!((inter[g] >> h) & 1ull) || S[g].level < 0 || S[h].level < 0) continue;
      if (!S[g].active && !S[h].active) continue;
      if (abs(S[g].level - S[h].level) > 4) ++breaks;
    }
  S[0].delayed += delayed;
  S[0].breaks += breaks;
}

// One block: the offsets of the round's particles in the compacted list, unit by unit (units
// idle in the round take none), and their total in *total.
__global__ void k_active_scan(const StateDev* __restrict__ st, int U, long long* __restrict__ aoff,
                              unsigned long long* total) {
  __shared__ long long wsum[32];
  __shared__ long long carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < U; base += blockDim.x) {
    const int u = base + threadIdx.x;
    const long long v = (u < U && st[u].active) ? st[u].members : 0;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    long long before = carry;
    for (int k = 0; k < w; ++k) before += wsum[k];
    if (u < U) aoff[u] = before + incl - v;
    __syncthreads();
    if (threadIdx.x == 0) for (int k = 0; k < nw; ++k) carry += wsum[k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    aoff[U] = carry;
    *total = (unsigned long long)carry;
  }
}

// The round's particles as one list of ranks, unit by unit in rank order: position p of the
// unit-ordered rank permutation goes to the list when its unit takes part in the round.
__global__ void k_active_gather(long long N, int U, const long long* __restrict__ uoff,
                                const long long* __restrict__ aoff, const StateDev* __restrict__ st,
                                const int* __restrict__ rperm, int* __restrict__ act) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int l = 0, h = U - 1;
  while (l < h) {
    const int mid = (l + h + 1) >> 1;
    if (uoff[mid] <= p) l = mid; else h = mid - 1;
  }
  // l: the last unit starting at or before p (an empty unit shares its start with the next)
  if (!st[l].active) return;
  act[aoff[l] + (p - uoff[l])] = rperm[p];
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_groups(gd_ctx* c) {
  if (!c->grouped) return cudaSuccess;
  time_begin(c, 0);
  k_group_assign<<<c->n_tiles, 256, 0, c->stream>>>(tile_map(c), c->d_inst, c->x, c->y, c->d_unit_i, c->d_tcount);
  k_group_scan<<<1, 1024, 0, c->stream>>>(c->d_inst, c->d_tile_off, c->d_unit_inst, c->U, c->d_tcount, c->d_tbase,
                                          c->d_uoff, c->d_utile_off, c->d_state, c->N);
  k_group_scatter<<<c->n_tiles, 128, 0, c->stream>>>(tile_map(c), c->d_inst, c->d_unit_i, c->d_tbase,
                                                     c->d_rank_of, c->d_gperm, c->d_unit_r);
  // the ranks by unit, for the round lists
  k_unit_count<<<c->n_tiles, 256, 0, c->stream>>>(tile_map(c), c->d_inst, c->d_unit_r, c->d_tcount);
  k_group_scan<<<1, 1024, 0, c->stream>>>(c->d_inst, c->d_tile_off, c->d_unit_inst, c->U, c->d_tcount, c->d_tbase,
                                          c->d_uoff, c->d_utile_off, c->d_state, c->N);
  k_group_scatter<<<c->n_tiles, 128, 0, c->stream>>>(tile_map(c), c->d_inst, c->d_unit_r, c->d_tbase, nullptr,
                                                     c->d_rperm, nullptr);
  time_end(c);
  c->launches += 6;
  return cudaGetLastError();
}

cudaError_t launch_group_inter(gd_ctx* c) {
  if (!c->grouped) return cudaSuccess;
  time_begin(c, 1);
  k_group_inter<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(c->N, c->K, c->d_nbr, c->d_unit_r,
                                                                      c->d_unit_inst, c->d_inst, c->d_state);
  time_end(c);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_round_begin(gd_ctx* c) {
  if (!c->grouped) return cudaSuccess;
  time_begin(c, 3);
  k_round_begin<<<(c->n_inst + 127) / 128, 128, 0, c->stream>>>(c->d_inst, c->d_state, c->n_inst);
  unsigned long long* total = c->d_counters + 10;
  k_active_scan<<<1, 1024, 0, c->stream>>>(c->d_state, c->U, c->d_aoff, total);
  k_active_gather<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(c->N, c->U, c->d_uoff, c->d_aoff,
                                                                        c->d_state, c->d_rperm, c->d_act);
  time_end(c);
  c->launches += 3;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_broadcast_snapshot(c);
  return e;
}

cudaError_t launch_schedule(gd_ctx* c) {
  if (!c->grouped) return cudaSuccess;
  k_schedule<<<(c->n_inst + 127) / 128, 128, 0, c->stream>>>(c->d_inst, c->d_state, c->n_inst);
  c->launches += 1;
  return cudaGetLastError();
}

}  // namespace gd
