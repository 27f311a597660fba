// gd_ctx.h -- host-side context of the library and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "gd_common.cuh"

struct gd_ctx {
  // configuration
  int n_inst = 0, K = 0, precision = 0, flags = 0;
  long long N = 0;
  double cell_factor = 1.0;
  int cell_xsplit = 1;                  // x cells per cell edge (rows are y-z lines; finer x
                                        // cells trim each row's x range at no extra row cost)
  long long max_events = 65536;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  std::vector<long long> h_off;
  std::vector<gd_instance_params> h_params;
  bool any_disk = false;
  bool any_model_r = false;             // the instances use the 1D radial model (all of them)

  // caller-owned particle arrays (device)
  double *x = nullptr, *y = nullptr, *z = nullptr, *s = nullptr;
  const double* M = nullptr;
  double *vr = nullptr, *lth = nullptr, *lph = nullptr;

  // library-owned device memory
  long long* d_off = nullptr;           // [n_inst + 1]
  long long* d_tile_off = nullptr;      // [n_inst + 1] first per-particle tile of each instance
  int n_tiles = 0;
  gd::InstDev* d_inst = nullptr;        // [n_inst]
  gd::GridDev* d_grid = nullptr;        // [n_inst]
  gd::StateDev* d_state = nullptr;      // [n_inst]
  gd::BinsDev* d_bins = nullptr;        // [n_inst]
  long long cell_cap = 0;               // capacity of the concatenated cell arrays
  int* d_cell_count = nullptr;          // [cell_cap + 1]
  int* d_cell_start = nullptr;          // [cell_cap + 1]
  int* d_scan_tmp = nullptr;            // block sums of the scan
  int* d_cell_of = nullptr;             // [N] cell of each caller index
  int* d_slot = nullptr;                // [N] position inside the cell
  int* d_perm = nullptr;                // [N] rank -> caller index
  int* d_rank_of = nullptr;             // [N] caller index -> rank
  gd::Pos64* d_pos64 = nullptr;         // [N]
  float4* d_pos32 = nullptr;            // [N]
  gd::Snap64* d_snap64 = nullptr;       // [N]
  float4* d_snap32 = nullptr;           // [N]
  double* d_Mr = nullptr;               // [N] M in rank order
  double* d_dist = nullptr;             // [N] d_i, rank order
  double* d_dprev = nullptr;            // [N] d_i of the last build, caller order (0: none)
  int* d_redo = nullptr;                // [N] mixed K-NN: queries the FP64 form redoes
  int* d_heavy = nullptr;               // [N] sampler: the particles sampled one per warp first
  double* d_V = nullptr;                // [N] V_i, rank order
  double* d_lam = nullptr;              // [N] lambda*_i, rank order
  int* d_nbr = nullptr;                 // [N*K] ranks
  float4* d_gx = nullptr;               // [N] mixed form: FP32 (R, Z, M) and the fine bin (bits)
  float* d_pref32 = nullptr;            // [N] mixed form: FP32 rate prefactor
  void* d_contrib = nullptr;            // [N] rank order: each particle's fine-bin contribution
                                        // (FP64 form gd::Contrib64, mixed form float4)
  double* d_MJ = nullptr;               // [N] caller order: M_i times the interval's realised
                                        // sum of |ln s'/s|
  double* d_part = nullptr;             // [kBinQ * kNFine * n_btiles] per-tile fine-bin partial sums
  unsigned long long* d_counters = nullptr;  // [16] spare device counters
  // mixed form: the heavy particles' event logs and the deferred FP64 settlement
  int4* d_dlog = nullptr;               // [dlog_cap] (chosen, j, outcome, N_coll) per event
  long long dlog_cap = 0;
  gd::DeferRec* d_defer = nullptr;      // [defer_cap]
  int defer_cap = 0;
  gd::DState* d_dstate = nullptr;       // [dstate_cap]
  long long dstate_cap = 0;
  double* d_sums = nullptr;             // [3 * (n_inst + n_tiles)] gd_stats sums, then per-tile partials

  // spatial groups (Sect. 2.5.3).  Units: one state and bin entry per group of each
  // instance, instance b's at unit0(b) ..; U = n_inst when no instance has more than one.
  int U = 0;
  bool grouped = false;                 // some instance has more than one group
  std::vector<int> h_unit0;             // [n_inst]
  int n_btiles = 0;                     // tiles of the fine-bin passes (n_tiles, or
                                        // n_tiles + U over the units when grouped)
  // grouped contexts only:
  int* d_unit_i = nullptr;              // [N] caller order: unit of each particle
  int* d_unit_r = nullptr;              // [N] rank order: unit of each particle
  int* d_gperm = nullptr;               // [N] caller indices ordered by (unit, index)
  long long* d_uoff = nullptr;          // [U + 1] first position of each unit in d_gperm
  long long* d_utile_off = nullptr;     // [U + 1] first fine-bin tile of each unit
  int* d_unit_inst = nullptr;           // [U] instance of each unit
  int* d_tcount = nullptr;              // [n_tiles * kMaxSG] particles of each group per caller tile
  long long* d_tbase = nullptr;         // [n_tiles * kMaxSG] their first position in d_gperm
  double* d_sb = nullptr;               // [N] caller order: each particle's last broadcast size
  int* d_rperm = nullptr;               // [N] ranks ordered by (unit, rank)
  int* d_act = nullptr;                 // [N] the round's ranks (units taking part), unit by unit
  long long* d_aoff = nullptr;          // [U + 1] each unit's first entry in d_act

  // radiation forces and the optical depth grid (Sect. 2.3.2)
  bool any_rad = false;                 // some instance has beta0 > 0
  bool any_plain_push = false;          // some disk instance has none (the plain step)
  bool any_tau = false;                 // some instance has a grid
  long long tau_cols = 0;               // grid columns of all instances
  long long tau_cells = 0;              // grid cells of all instances
  long long tau_faces = 0;              // radial faces times columns, all instances
  long long* d_col_off = nullptr;       // [n_inst + 1] first column of each instance
  long long* d_cell_off = nullptr;      // [n_inst + 1] first cell of each instance
  unsigned long long* d_tau_acc = nullptr;   // [2 * tau_cells] 128-bit fixed-point cell sums
                                        // (low, high word), [radial cell][column] per instance
  double* d_tau_T = nullptr;            // [tau_faces] tau at the faces, [face][column]
  unsigned long long* d_tau_max = nullptr;   // [n_inst] largest kappa M (bits) of the deposit
  int* d_tau_ci = nullptr;              // [N] cell of each particle's deposit (-1: none)
  double* d_tau_q = nullptr;            // [N] its kappa M
  double* d_mid = nullptr;              // [3 N] the first drift's midpoints of the radiation
                                        // step ((r, theta, phi) FP64 form, (x, y, z) mixed)
  double* d_trad = nullptr;             // [n_inst] the taper's clock
  long long tau_out_faces = 0;          // faces of gd_optical_depth's grid output
  long long* d_face_off = nullptr;      // [n_inst + 1] each instance's first output face

  // sequencing: 0 nothing, 1 neighbours built, 2 rates done
  int phase = 0;
  long long intervals = 0;
  long long launches = 0;
  long long diff_step = 0;              // gd_diffuse calls so far (Philox counter word 1)
  bool lists_valid = false;             // neighbour lists built (gd_collide may reuse them)
  bool moved = false;                   // particles moved since the last neighbour build

  // timing
  static constexpr int kSlots = 8;
  double ms[kSlots] = {0};
  long long calls[kSlots] = {0};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  std::vector<int> ev_slot;
  size_t ev_used = 0;

  // graph replay of one interval
  cudaGraphExec_t graph_exec = nullptr;
  int graph_push = -1;
  long long graph_kernel_count = 0;     // kernel nodes of the captured interval
};

namespace gd {
inline TileMap tile_map(const gd_ctx* c) {
  TileMap tm;
  tm.off = c->d_off;
  tm.n_inst = c->n_inst;
  tm.tile_off = c->d_tile_off;
  return tm;
}

// Tiles of the fine-bin passes: the instances' caller-index tiles, or (grouped) tiles of each
// unit's caller indices in ascending order, read through d_gperm.
inline TileMap bins_map(const gd_ctx* c) {
  if (!c->grouped) return tile_map(c);
  TileMap tm;
  tm.off = c->d_uoff;
  tm.n_inst = c->U;
  tm.tile_off = c->d_utile_off;
  return tm;
}

// launchers (each returns cudaGetLastError() of its launches)
cudaError_t launch_cells(gd_ctx* c);
cudaError_t launch_knn(gd_ctx* c);
cudaError_t knn_prepare(gd_ctx* c);
cudaError_t launch_rates(gd_ctx* c, double* chan_out);
cudaError_t launch_interval(gd_ctx* c);
cudaError_t launch_sample(gd_ctx* c, int* ev_count, unsigned* ev_hash, int* near);
cudaError_t launch_audit(gd_ctx* c);
cudaError_t launch_push(gd_ctx* c, double dt);
cudaError_t launch_push_rad(gd_ctx* c, double dt);     // instances with radiation forces
cudaError_t launch_optical_depth(gd_ctx* c, double* tau_out, double* grid_out);
cudaError_t launch_diffuse(gd_ctx* c, double dt);
cudaError_t launch_timestep(gd_ctx* c, const gd_dt_rule& r, double* dti_out, unsigned long long* d_min,
                            unsigned long long* d_bad);
cudaError_t launch_snapshot(gd_ctx* c);
cudaError_t launch_groups(gd_ctx* c);          // units, their members and d_gperm (after the cells)
cudaError_t launch_group_inter(gd_ctx* c);     // interaction masks (after the lists)
cudaError_t launch_round_begin(gd_ctx* c);     // the round's groups, their broadcast and snapshot
cudaError_t launch_schedule(gd_ctx* c);
cudaError_t launch_broadcast_snapshot(gd_ctx* c);   // the round's broadcast and its snapshot entries        // levels of the round's groups (after k_interval)
cudaError_t launch_step_begin(gd_ctx* c, double tau, int hold);
cudaError_t launch_step_done(gd_ctx* c, int* d_flag);
cudaError_t launch_stats(gd_ctx* c, double* d_sums);
cudaError_t launch_spectrum(gd_ctx* c);
cudaError_t launch_outputs_knn(gd_ctx* c, int* nbr_out, double* d_out);
cudaError_t launch_outputs_lam(gd_ctx* c, double* lam_out);

std::vector<long long> tile_table(const std::vector<long long>& off);

// event timing around a launch (no-op unless GD_FLAG_TIMING)
void time_begin(gd_ctx* c, int slot);
void time_end(gd_ctx* c);
}  // namespace gd
