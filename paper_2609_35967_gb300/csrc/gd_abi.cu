// gd_abi.cu -- the C ABI of include/gd.h: argument checks, the library-owned memory
// plan, call sequencing, per-kernel event timing, CUDA-graph replay and gd_stats.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gd_ctx.h"

namespace gd {

void time_begin(gd_ctx* c, int slot) {
  if (!(c->flags & GD_FLAG_TIMING)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c->stream, &cs);
  if (cs != cudaStreamCaptureStatusNone) { c->ev_slot.push_back(-1); return; }
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
    c->ev_pool.push_back({a, b});
  }
  cudaEventRecord(c->ev_pool[c->ev_used].first, c->stream);
  c->ev_slot.push_back(slot);
}

void time_end(gd_ctx* c) {
  if (!(c->flags & GD_FLAG_TIMING)) return;
  if (c->ev_slot.empty()) return;
  if (c->ev_slot.back() < 0) { c->ev_slot.pop_back(); return; }
  cudaEventRecord(c->ev_pool[c->ev_used].second, c->stream);
  c->ev_used++;
}

static void collect_timing(gd_ctx* c) {
  size_t k = 0;
  for (size_t i = 0; i < c->ev_slot.size() && k < c->ev_used; ++i) {
    int slot = c->ev_slot[i];
    if (slot < 0) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[k].first, c->ev_pool[k].second) == cudaSuccess) {
      c->ms[slot] += ms;
      c->calls[slot] += 1;
    }
    ++k;
  }
  c->ev_slot.clear();
  c->ev_used = 0;
}

}  // namespace gd

using namespace gd;

static gd_status cuda_err(cudaError_t e) { return e == cudaSuccess ? GD_OK : GD_ERR_CUDA; }

template <typename T>
static cudaError_t dalloc(T** p, size_t n) {
  if (n == 0) n = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

static void free_all(gd_ctx* c) {
  void* ptrs[] = {c->d_off, c->d_tile_off, c->d_inst, c->d_grid, c->d_state, c->d_bins, c->d_cell_count,
                  c->d_cell_start, c->d_scan_tmp, c->d_cell_of, c->d_slot, c->d_perm, c->d_rank_of,
                  c->d_pos64, c->d_pos32, c->d_snap64, c->d_snap32, c->d_Mr, c->d_dist, c->d_V,
                  c->d_lam, c->d_nbr, c->d_counters, c->d_sums, c->d_dprev, c->d_redo, c->d_gx,
                  c->d_pref32, c->d_contrib, c->d_MJ, c->d_part, c->d_heavy, c->d_unit_i, c->d_unit_r, c->d_gperm,
                  c->d_uoff, c->d_utile_off, c->d_unit_inst, c->d_tcount, c->d_tbase, c->d_sb, c->d_rperm, c->d_act, c->d_aoff,
                  c->d_col_off, c->d_tau_acc, c->d_tau_T, c->d_tau_max, c->d_tau_ci, c->d_tau_q, c->d_mid,
                  c->d_trad, c->d_face_off, c->d_cell_off, c->d_dlog, c->d_defer, c->d_dstate};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& e : c->ev_pool) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  c->ev_pool.clear();
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
}

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// The instance's radiation parameters as the kernels read them, with the error bounds (in
// cells, four times the sum of the rounding errors' bounds) of the mixed form's FP32 grid
// coordinates: u = (r - r_min)/dr from sqrtf of the FP64 r^2, w = (z/r + mu_max)/dmu,
// v = (atan2f(y, x) + pi)/dphi (atan2f within 3 ulp).
static void fill_rad(InstDev& d, const gd_instance_params& p, long long cell0, long long face0) {
  d.rad = p.geometry == GD_GEOM_DISK && p.beta0 > 0.0;
  d.tau_on = p.tau_nr > 0 && p.kappa0 > 0.0;
  d.rad_pr = p.rad_pr;
  d.tau_geom = p.tau_geom;
  d.tau_nr = d.tau_on ? p.tau_nr : 0;
  d.tau_nm = d.tau_on ? (p.tau_geom == GD_TAU_2D ? 1 : p.tau_nmu) : 1;
  d.tau_np = d.tau_on ? p.tau_nphi : 1;
  d.beta0 = p.beta0; d.kappa0 = p.kappa0; d.rad_s0 = p.rad_s0; d.t_beta = p.t_beta;
  d.tau_rmin = p.tau_rmin; d.tau_rmax = p.tau_rmax; d.tau_mu = p.tau_mu;
  d.tau_cell0 = cell0;
  d.tau_face0 = face0;
  d.f_beta0 = (float)p.beta0;
  d.f_rad_s0 = (float)p.rad_s0;
  if (!d.tau_on) return;
  const double dr = (p.tau_rmax - p.tau_rmin) / d.tau_nr;
  const double dmu = p.tau_geom == GD_TAU_2D ? 1.0 : 2.0 * p.tau_mu / d.tau_nm;
  const double dphi = 2.0 * kPi / d.tau_np;
  d.f_tau_rmin = (float)p.tau_rmin;
  d.f_tau_dr = (float)dr;
  d.f_tau_mu = (float)p.tau_mu;
  d.f_tau_dmu = (float)dmu;
  d.f_tau_dphi = (float)dphi;
  d.f_eu = (float)(4.0 * ((1.8e-7 * p.tau_rmax + 6e-8 * p.tau_rmin) / dr + 1.2e-7 * d.tau_nr) + 1e-5);
  d.f_ew = (float)(4.0 * (4.2e-7 / dmu + 1.2e-7 * d.tau_nm) + 1e-5);
  d.f_ev = (float)(4.0 * (1.2e-6 / dphi + 1.2e-7 * d.tau_np) + 1e-5);
}

// Radiation forces and the optical depth grid (Sect. 2.3.2): global disks only; a grid of
// at most 2^28 cells per instance.
static bool rad_params_ok(const gd_instance_params& p) {
  const bool any = p.beta0 != 0.0 || p.kappa0 != 0.0 || p.rad_pr != 0 || p.tau_nr != 0;
  if (!any) return true;
  if (p.geometry != GD_GEOM_DISK) return false;
  if (!(p.beta0 >= 0.0) || !std::isfinite(p.beta0) || !(p.kappa0 >= 0.0) || !std::isfinite(p.kappa0)) return false;
  if ((p.beta0 > 0.0 || p.kappa0 > 0.0) && !finite_pos(p.rad_s0)) return false;
  if (p.rad_pr != 0 && p.rad_pr != 1) return false;
  if (!std::isfinite(p.t_beta) || !std::isfinite(p.t_start)) return false;
  if (p.tau_nr < 0) return false;
  if (p.tau_nr > 0) {
    if (p.tau_geom != GD_TAU_3D && p.tau_geom != GD_TAU_2D) return false;
    const long long nm = p.tau_geom == GD_TAU_2D ? 1 : p.tau_nmu;
    if (nm < 1 || p.tau_nphi < 1) return false;
    if ((long long)p.tau_nr * nm * p.tau_nphi > (1LL << 28)) return false;
    if (!(p.tau_rmin >= 0.0) || !(p.tau_rmax > p.tau_rmin) || !std::isfinite(p.tau_rmax)) return false;
    if (p.tau_geom == GD_TAU_3D && !(p.tau_mu > 0.0 && p.tau_mu <= 1.0)) return false;
  }
  return true;
}

extern "C" gd_status gd_create(gd_ctx** out, const gd_config* cfg) {
  if (!out) return GD_ERR_ARG;
  *out = nullptr;
  if (!cfg || cfg->n_instances < 1 || !cfg->offsets || !cfg->params) return GD_ERR_ARG;
  if (cfg->K < 2 || cfg->K > kMaxK) return GD_ERR_ARG;
  if (cfg->precision != GD_FP64 && cfg->precision != GD_MIXED) return GD_ERR_ARG;
  if (!cfg->x || !cfg->y || !cfg->z || !cfg->s || !cfg->M) return GD_ERR_ARG;
  const int n = cfg->n_instances;
  if (cfg->offsets[0] != 0) return GD_ERR_ARG;
  for (int b = 0; b < n; ++b) {
    if (cfg->offsets[b + 1] - cfg->offsets[b] < cfg->K) return GD_ERR_ARG;
    const gd_instance_params& p = cfg->params[b];
    if (p.geometry != GD_GEOM_PATCH && p.geometry != GD_GEOM_DISK) return GD_ERR_ARG;
    if (p.kernel_mode < GD_KERNEL_PHYSICAL || p.kernel_mode > GD_KERNEL_PRODUCT) return GD_ERR_ARG;
    if (!finite_pos(p.r0) || !finite_pos(p.sigma0) || !finite_pos(p.T0) || !finite_pos(p.M_star) ||
        !finite_pos(p.rho_s) || !finite_pos(p.s_min) || !finite_pos(p.eps) || !finite_pos(p.dt_coll) ||
        !finite_pos(p.dt_fn_max) || !(p.alpha >= 0.0) || !(p.v_frag > 0.0))
      return GD_ERR_ARG;
    if (p.geometry == GD_GEOM_PATCH && (!finite_pos(p.box_x) || !finite_pos(p.box_y))) return GD_ERR_ARG;
    if (p.geometry == GD_GEOM_DISK && !(p.R_out > p.R_in)) return GD_ERR_ARG;
    if (p.diff_mode != GD_DIFF_PHYSICAL && p.diff_mode != GD_DIFF_RING) return GD_ERR_ARG;
    if (p.model < GD_MODEL_3D || p.model > GD_MODEL_R) return GD_ERR_ARG;
    if ((p.model == GD_MODEL_RZ || p.model == GD_MODEL_R) && p.geometry != GD_GEOM_DISK) return GD_ERR_ARG;
    // the 1D model's one-row grids take their own neighbour kernel: all or none
    if ((p.model == GD_MODEL_R) != (cfg->params[0].model == GD_MODEL_R)) return GD_ERR_ARG;
    if (p.diff_chi != 0 && p.diff_chi != 1) return GD_ERR_ARG;
    if (p.diff_mode == GD_DIFF_RING && !(p.D0 >= 0.0 && std::isfinite(p.D0) && p.r0 > 0.0)) return GD_ERR_ARG;
    if (p.kernel_mode != GD_KERNEL_PHYSICAL && (!finite_pos(p.t0) || !finite_pos(p.m0))) return GD_ERR_ARG;
    if (p.spatial_groups < 0 || p.spatial_groups > kMaxSG) return GD_ERR_ARG;
    if (!rad_params_ok(p)) return GD_ERR_ARG;
  }
  const long long N = cfg->offsets[n];
  if (N >= (1LL << 31) - 1 || (long long)N * cfg->K >= (1LL << 40)) return GD_ERR_ARG;

  gd_ctx* c = new (std::nothrow) gd_ctx();
  if (!c) return GD_ERR_OOM;
  c->n_inst = n;
  c->K = cfg->K;
  c->precision = cfg->precision;
  c->flags = cfg->flags;
  c->N = N;
  c->cell_factor = cfg->cell_factor > 0.0 ? cfg->cell_factor : 1.0;
  c->cell_xsplit = cfg->cell_xsplit > 0 ? cfg->cell_xsplit : 1;
  if (c->cell_xsplit != 1 && c->cell_xsplit != 2 && c->cell_xsplit != 4) { delete c; return GD_ERR_ARG; }
  c->max_events = cfg->max_events_per_interval > 0 ? cfg->max_events_per_interval : 65536;
  c->stream = static_cast<cudaStream_t>(cfg->stream);
  c->x = cfg->x; c->y = cfg->y; c->z = cfg->z; c->s = cfg->s; c->M = cfg->M;
  c->vr = cfg->vr; c->lth = cfg->lth; c->lph = cfg->lph;
  c->h_off.assign(cfg->offsets, cfg->offsets + n + 1);
  c->h_params.assign(cfg->params, cfg->params + n);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete c;
    return GD_ERR_CUDA;
  }

  std::vector<long long> tiles = tile_table(c->h_off);
  c->n_tiles = (int)tiles.back();
  // units: one per spatial group of each instance
  c->h_unit0.resize(n);
  std::vector<int> unit_inst;
  for (int b = 0; b < n; ++b) {
    const int G = cfg->params[b].spatial_groups > 1 ? cfg->params[b].spatial_groups : 1;
    c->h_unit0[b] = (int)unit_inst.size();
    for (int g = 0; g < G; ++g) unit_inst.push_back(b);
    if (G > 1) c->grouped = true;
  }
  c->U = (int)unit_inst.size();
  c->n_btiles = c->grouped ? c->n_tiles + c->U : c->n_tiles;
  c->cell_cap = 16 * N + 64LL * n + 1024;
  long long nst = (c->cell_cap + 2048) / 2048 + 1;   // scan tiles of cells [0, cell_cap]

  bool ok = true;
  ok &= dalloc(&c->d_off, n + 1) == cudaSuccess;
  ok &= dalloc(&c->d_tile_off, n + 1) == cudaSuccess;
  ok &= dalloc(&c->d_inst, n) == cudaSuccess;
  ok &= dalloc(&c->d_grid, n) == cudaSuccess;
  ok &= dalloc(&c->d_state, c->U) == cudaSuccess;
  ok &= dalloc(&c->d_bins, c->U) == cudaSuccess;
  ok &= dalloc(&c->d_cell_count, c->cell_cap + 1) == cudaSuccess;
  ok &= dalloc(&c->d_cell_start, c->cell_cap + 1) == cudaSuccess;
  ok &= dalloc(&c->d_scan_tmp, nst) == cudaSuccess;
  ok &= dalloc(&c->d_cell_of, N) == cudaSuccess;
  ok &= dalloc(&c->d_slot, N) == cudaSuccess;
  ok &= dalloc(&c->d_perm, N) == cudaSuccess;
  ok &= dalloc(&c->d_rank_of, N) == cudaSuccess;
  ok &= dalloc(&c->d_pos64, N) == cudaSuccess;
  ok &= dalloc(&c->d_snap64, N) == cudaSuccess;
  ok &= dalloc(&c->d_pos32, N) == cudaSuccess;
  if (c->precision == GD_MIXED) ok &= dalloc(&c->d_snap32, N) == cudaSuccess;
  ok &= dalloc(&c->d_Mr, N) == cudaSuccess;
  ok &= dalloc(&c->d_dist, N) == cudaSuccess;
  ok &= dalloc(&c->d_dprev, N) == cudaSuccess;
  ok &= dalloc(&c->d_redo, N) == cudaSuccess;
  ok &= dalloc(&c->d_heavy, N) == cudaSuccess;
  ok &= dalloc(&c->d_V, N) == cudaSuccess;
  ok &= dalloc(&c->d_lam, N) == cudaSuccess;
  ok &= dalloc(&c->d_nbr, (size_t)N * c->K) == cudaSuccess;
  if (c->precision == GD_MIXED) {
    ok &= dalloc(&c->d_gx, N) == cudaSuccess;
    ok &= dalloc(&c->d_pref32, N) == cudaSuccess;
    // the heavy particles' event logs (about 2 lambda*_i dt_exe + 64 entries each) and
    // the deferred FP64 settlement's records and states
    c->dlog_cap = std::min(std::max(1LL << 20, N), 1LL << 23);
    c->defer_cap = 256;
    c->dstate_cap = 1LL << 18;
    ok &= dalloc(&c->d_dlog, c->dlog_cap) == cudaSuccess;
    ok &= dalloc(&c->d_defer, c->defer_cap) == cudaSuccess;
    ok &= dalloc(&c->d_dstate, c->dstate_cap) == cudaSuccess;
  }
  ok &= dalloc(reinterpret_cast<Contrib64**>(&c->d_contrib), N) == cudaSuccess;
  ok &= dalloc(&c->d_MJ, N) == cudaSuccess;
  ok &= dalloc(&c->d_part, (size_t)kBinQ * kNFine * c->n_btiles) == cudaSuccess;
  if (c->grouped) {
    ok &= dalloc(&c->d_unit_i, N) == cudaSuccess;
    ok &= dalloc(&c->d_unit_r, N) == cudaSuccess;
    ok &= dalloc(&c->d_gperm, N) == cudaSuccess;
    ok &= dalloc(&c->d_uoff, c->U + 1) == cudaSuccess;
    ok &= dalloc(&c->d_utile_off, c->U + 1) == cudaSuccess;
    ok &= dalloc(&c->d_unit_inst, c->U) == cudaSuccess;
    ok &= dalloc(&c->d_tcount, (size_t)c->n_tiles * kMaxSG) == cudaSuccess;
    ok &= dalloc(&c->d_tbase, (size_t)c->n_tiles * kMaxSG) == cudaSuccess;
    ok &= dalloc(&c->d_sb, N) == cudaSuccess;
    ok &= dalloc(&c->d_rperm, N) == cudaSuccess;
    ok &= dalloc(&c->d_act, N) == cudaSuccess;
    ok &= dalloc(&c->d_aoff, c->U + 1) == cudaSuccess;
  }
  ok &= dalloc(&c->d_counters, 16) == cudaSuccess;
  ok &= dalloc(&c->d_sums, 3 * ((size_t)n + c->n_tiles)) == cudaSuccess;
  // radiation forces and the optical depth grid
  std::vector<long long> col_off(n + 1, 0), face_off(n + 1, 0), cell0(n, 0), face0(n, 0);
  for (int b = 0; b < n; ++b) {
    const gd_instance_params& p = cfg->params[b];
    const bool tau_on = p.tau_nr > 0 && p.kappa0 > 0.0;
    const long long nm = p.tau_geom == GD_TAU_2D ? 1 : p.tau_nmu;
    const long long ncol = tau_on ? nm * p.tau_nphi : 0;
    if (p.beta0 > 0.0) c->any_rad = true;
    if (tau_on) c->any_tau = true;
    cell0[b] = c->tau_cells;
    face0[b] = c->tau_faces;
    col_off[b + 1] = col_off[b] + ncol;
    face_off[b + 1] = face_off[b] + ncol * (tau_on ? p.tau_nr + 1 : 0);
    c->tau_cells += ncol * (tau_on ? p.tau_nr : 0);
    c->tau_faces += ncol * (tau_on ? p.tau_nr + 1 : 0);
  }
  c->tau_cols = col_off[n];
  c->tau_out_faces = face_off[n];
  c->any_plain_push = !c->any_rad;
  for (int b = 0; b < n; ++b)
    if (cfg->params[b].geometry == GD_GEOM_DISK && !(cfg->params[b].beta0 > 0.0)) c->any_plain_push = true;
  if (c->any_rad || c->any_tau) {
    ok &= dalloc(&c->d_tau_max, n) == cudaSuccess;
    ok &= dalloc(&c->d_tau_ci, N) == cudaSuccess;
    ok &= dalloc(&c->d_tau_q, N) == cudaSuccess;
    ok &= dalloc(&c->d_trad, n) == cudaSuccess;
    ok &= dalloc(&c->d_col_off, n + 1) == cudaSuccess;
    ok &= dalloc(&c->d_face_off, n + 1) == cudaSuccess;
    ok &= dalloc(&c->d_cell_off, n + 1) == cudaSuccess;
    ok &= dalloc(&c->d_tau_acc, 2 * (size_t)c->tau_cells) == cudaSuccess;
    ok &= dalloc(&c->d_tau_T, c->tau_faces) == cudaSuccess;
  }
  if (c->any_rad) ok &= dalloc(&c->d_mid, 3 * (size_t)N) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return GD_ERR_OOM;
  }

  std::vector<InstDev> inst(n);
  std::vector<StateDev> st(c->U);
  for (int b = 0; b < n; ++b) {
    const gd_instance_params& p = c->h_params[b];
    InstDev& d = inst[b];
    std::memset(&d, 0, sizeof(d));
    d.geometry = p.geometry;
    d.kernel_mode = p.kernel_mode;
    d.audit = p.audit;
    d.model = p.model;
    d.r0 = p.r0; d.sigma0 = p.sigma0; d.p = p.p; d.T0 = p.T0; d.q = p.q; d.alpha = p.alpha;
    d.GM = kG * p.M_star;
    d.rho_s = p.rho_s; d.s_min = p.s_min; d.v_frag = p.v_frag; d.eps = p.eps;
    d.dt_coll = p.dt_coll; d.dt_fn_max = p.dt_fn_max; d.R_in = p.R_in; d.R_out = p.R_out;
    d.box_x = p.box_x; d.box_y = p.box_y; d.t0 = p.t0; d.m0 = p.m0; d.cell_size = p.cell_size;
    d.key0 = (uint32_t)p.seed;
    d.key1 = (uint32_t)(p.seed >> 32);
    d.k6 = 6.0 / (kPi * p.rho_s);
    d.mk = kPi * p.rho_s / 6.0;
    d.f_r0 = (float)p.r0; d.f_GM = (float)d.GM; d.f_T0 = (float)p.T0; d.f_q = (float)p.q;
    d.f_p = (float)p.p; d.f_sigma0 = (float)p.sigma0; d.f_alpha = (float)p.alpha;
    d.f_rho_s = (float)p.rho_s; d.f_vfrag = (float)p.v_frag; d.f_m0 = (float)p.m0;
    d.f_smin = (float)p.s_min;
    d.diff_mode = p.diff_mode;
    d.diff_chi = p.diff_chi;
    d.Sc_R = p.Sc_R > 0.0 ? p.Sc_R : 1.0;
    d.Sc_Z = p.Sc_Z > 0.0 ? p.Sc_Z : 1.0;
    d.Sc_phi = p.Sc_phi > 0.0 ? p.Sc_phi : 1.0;
    d.D0 = p.D0;
    d.off = c->h_off[b];
    d.n = c->h_off[b + 1] - c->h_off[b];
    d.n_sg = p.spatial_groups > 1 ? p.spatial_groups : 1;
    d.unit0 = c->h_unit0[b];
    fill_rad(d, p, cell0[b], face0[b]);
    if (p.geometry == GD_GEOM_DISK) c->any_disk = true;
    if (p.model == GD_MODEL_R) c->any_model_r = true;
    for (int g = 0; g < d.n_sg; ++g) {
      StateDev& s = st[d.unit0 + g];
      std::memset(&s, 0, sizeof(s));
      s.C = 1.0;
      s.remain_ticks = 1LL << 60;
      s.dt_remain = p.dt_coll;
      s.active = 1;
      s.level = -1;
      s.members = d.n_sg > 1 ? 0 : d.n;   // groups: counted at each build
      for (int a = 0; a < 3; ++a) { s.bmin[a] = ~0ull; s.bmax[a] = 0ull; }
    }
  }
  cudaStream_t str = c->stream;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_off, c->h_off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_tile_off, tiles.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_inst, inst.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_state, st.data(), sizeof(StateDev) * c->U, cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_bins, 0, sizeof(BinsDev) * c->U, str);
  if (c->grouped) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_unit_inst, unit_inst.data(), sizeof(int) * c->U, cudaMemcpyHostToDevice, str);
    // nothing broadcast yet: the partners' sizes start as the caller's
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_sb, c->s, sizeof(double) * N, cudaMemcpyDeviceToDevice, str);
  }
  // host tables of the radiation grid (kept until the stream synchronises below)
  std::vector<double> t0(n);
  std::vector<long long> cell_off(cell0.begin(), cell0.end());
  cell_off.push_back(c->tau_cells);
  if (c->any_rad || c->any_tau) {
    for (int b = 0; b < n; ++b) t0[b] = c->h_params[b].t_start;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_trad, t0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, str);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_col_off, col_off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, str);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_face_off, face_off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, str);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_cell_off, cell_off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, str);
    if (e == cudaSuccess && c->tau_cells > 0)
      e = cudaMemsetAsync(c->d_tau_acc, 0, sizeof(unsigned long long) * 2 * c->tau_cells, str);
    if (e == cudaSuccess && c->tau_faces > 0) e = cudaMemsetAsync(c->d_tau_T, 0, sizeof(double) * c->tau_faces, str);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * 16, str);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_dprev, 0, sizeof(double) * N, str);
  if (e == cudaSuccess) e = knn_prepare(c);
  if (e == cudaSuccess) e = cudaStreamSynchronize(str);
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    return GD_ERR_CUDA;
  }
  *out = c;
  return GD_OK;
}

extern "C" gd_status gd_destroy(gd_ctx* c) {
  if (!c) return GD_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  return GD_OK;
}

static gd_status do_build(gd_ctx* c, int32_t* nbr_out, double* d_out) {
  cudaError_t e = launch_cells(c);
  if (e == cudaSuccess) e = launch_groups(c);
  if (e == cudaSuccess) e = launch_knn(c);
  if (e == cudaSuccess) e = launch_group_inter(c);
  if (e == cudaSuccess) e = launch_outputs_knn(c, nbr_out, d_out);
  if (e != cudaSuccess) return GD_ERR_CUDA;
  c->phase = 1;
  c->lists_valid = true;
  return GD_OK;
}

static gd_status do_rates(gd_ctx* c, double* lam_out, double* chan_out) {
  // spatial groups: the round's groups broadcast and the partner snapshot follows
  cudaError_t e = launch_round_begin(c);
  if (e == cudaSuccess) e = launch_rates(c, chan_out);
  if (e == cudaSuccess) e = launch_interval(c);
  if (e == cudaSuccess) e = launch_outputs_lam(c, lam_out);
  if (e != cudaSuccess) return GD_ERR_CUDA;
  c->phase = 2;
  return GD_OK;
}

static gd_status do_sample(gd_ctx* c, int32_t* ev_count, uint32_t* ev_hash, int32_t* near) {
  cudaError_t e = launch_sample(c, ev_count, ev_hash, near);
  if (e == cudaSuccess) e = launch_audit(c);
  if (e != cudaSuccess) return GD_ERR_CUDA;
  c->phase = 0;
  c->intervals++;
  return GD_OK;
}

extern "C" gd_status gd_build_neighbors(gd_ctx* c, int32_t* nbr_out, double* d_out) {
  if (!c) return GD_ERR_ARG;
  return do_build(c, nbr_out, d_out);
}

extern "C" gd_status gd_collision_rates(gd_ctx* c, double* lambda_out, double* chan_out) {
  if (!c) return GD_ERR_ARG;
  if (c->phase != 1) return GD_ERR_STATE;
  return do_rates(c, lambda_out, chan_out);
}

extern "C" gd_status gd_sample_collisions(gd_ctx* c, int32_t* ev_count_out, uint32_t* ev_hash_out,
                                          int32_t* near_out) {
  if (!c) return GD_ERR_ARG;
  if (c->phase != 2) return GD_ERR_STATE;
  if ((ev_count_out != nullptr) != (ev_hash_out != nullptr) || (ev_count_out != nullptr) != (near_out != nullptr))
    return GD_ERR_ARG;
  return do_sample(c, ev_count_out, ev_hash_out, near_out);
}

extern "C" gd_status gd_push_staggered(gd_ctx* c, double dt) {
  if (!c) return GD_ERR_ARG;
  if (!c->vr || !c->lth || !c->lph) return GD_ERR_ARG;
  if (!std::isfinite(dt)) return GD_ERR_ARG;
  if (dt < 0.0 && c->grouped) return GD_ERR_ARG;   // groups have no common dt_exe
  c->lists_valid = false;           // positions move: gd_collide must build again
  return cuda_err(launch_push(c, dt));
}

extern "C" gd_status gd_diffuse(gd_ctx* c, double dt) {
  if (!c) return GD_ERR_ARG;
  if (!std::isfinite(dt)) return GD_ERR_ARG;
  if (dt < 0.0 && c->grouped) return GD_ERR_ARG;
  c->lists_valid = false;           // positions move: gd_collide must build again
  return cuda_err(launch_diffuse(c, dt));
}

extern "C" gd_status gd_optical_depth(gd_ctx* c, double* tau_out, double* grid_out) {
  if (!c) return GD_ERR_ARG;
  if (!c->any_tau) return GD_ERR_ARG;
  return cuda_err(launch_optical_depth(c, tau_out, grid_out));
}

extern "C" gd_status gd_collide(gd_ctx* c, double tau, int32_t reuse_lists, int32_t max_intervals,
                                int32_t* n_intervals_out) {
  if (n_intervals_out) *n_intervals_out = 0;
  if (!c || !(tau > 0.0) || !std::isfinite(tau) || max_intervals < 1) return GD_ERR_ARG;
  if (c->phase != 0) return GD_ERR_STATE;
  int* d_flag = reinterpret_cast<int*>(c->d_counters + 4);
  gd_status s = cuda_err(launch_step_begin(c, tau, 1));
  int n = 0, done = 0;
  while (s == GD_OK && n < max_intervals) {
    // positions are frozen within the step: the lists are built once (or kept from the
    // last step), later intervals only refresh the partner snapshot
    if (n == 0 && !(reuse_lists && c->lists_valid)) {
      s = do_build(c, nullptr, nullptr);
    } else {
      // (with spatial groups do_rates refreshes the snapshot after the round's broadcast)
      if (!c->grouped) s = cuda_err(launch_snapshot(c));
      c->phase = 1;
    }
    if (s == GD_OK) s = do_rates(c, nullptr, nullptr);
    if (s == GD_OK) s = do_sample(c, nullptr, nullptr, nullptr);
    if (s != GD_OK) break;
    ++n;
    cudaError_t e = launch_step_done(c, d_flag);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&done, d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { s = GD_ERR_CUDA; break; }
    if (done) break;
  }
  // back to open-ended collision steps of dt_coll
  const gd_status r = cuda_err(launch_step_begin(c, 0.0, 0));
  if (s == GD_OK) s = r;
  if (n_intervals_out) *n_intervals_out = n;
  if (s == GD_OK && !done) s = GD_ERR_TIMEOUT;
  return s;
}

extern "C" gd_status gd_step(gd_ctx* c, double dt, int32_t reuse_lists, int32_t* n_intervals_out) {
  if (n_intervals_out) *n_intervals_out = 0;
  if (!c || !(dt > 0.0) || !std::isfinite(dt)) return GD_ERR_ARG;
  if (c->phase != 0) return GD_ERR_STATE;
  const int32_t kMaxIntervals = 1 << 20;
  int32_t n1 = 0, n2 = 0;
  gd_status s = gd_collide(c, 0.5 * dt, reuse_lists, kMaxIntervals, &n1);
  if (s == GD_OK) s = cuda_err(launch_diffuse(c, 0.5 * dt));
  if (s == GD_OK && c->vr && c->lth && c->lph) s = cuda_err(launch_push(c, dt));
  if (s == GD_OK) s = cuda_err(launch_diffuse(c, 0.5 * dt));
  if (s == GD_OK) s = gd_collide(c, 0.5 * dt, 0, kMaxIntervals, &n2);
  if (n_intervals_out) *n_intervals_out = n1 + n2;
  return s;
}

extern "C" gd_status gd_timestep(gd_ctx* c, const gd_dt_rule* r, double* dt_out_host, double* dti_out) {
  if (dt_out_host) *dt_out_host = 0.0;
  if (!c || !r || !dt_out_host) return GD_ERR_ARG;
  if (!(r->dt_max > 0.0) || !(r->dt_out > 0.0)) return GD_ERR_ARG;
  if (!std::isfinite(r->f_orb) || !std::isfinite(r->c_adv) || !std::isfinite(r->c_diff)) return GD_ERR_ARG;
  if ((r->c_adv > 0.0 || r->c_diff > 0.0) && !(r->dx_H > 0.0 && std::isfinite(r->dx_H))) return GD_ERR_ARG;
  unsigned long long* d_min = c->d_counters + 8;
  unsigned long long* d_bad = c->d_counters + 9;
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(d_min, 0xFF, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess && c->N > 0) e = launch_timestep(c, *r, dti_out, d_min, d_bad);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_min, sizeof h, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return GD_ERR_CUDA;
  double dt = r->dt_max < r->dt_out ? r->dt_max : r->dt_out;
  if (h[0] != ~0ull) {
    double m;
    std::memcpy(&m, &h[0], sizeof m);
    if (m < dt) dt = m;
  }
  *dt_out_host = dt;
  return h[1] ? GD_ERR_NONFINITE : GD_OK;
}

extern "C" gd_status gd_run_intervals(gd_ctx* c, int32_t n, int32_t push) {
  if (!c || n < 0) return GD_ERR_ARG;
  if (push && (!c->vr || !c->lth || !c->lph || c->grouped)) return GD_ERR_ARG;
  if (c->phase != 0) return GD_ERR_STATE;
  if (n == 0) return GD_OK;
  bool can_graph = c->stream != nullptr && !(c->flags & GD_FLAG_TIMING);
  if (!can_graph) {
    for (int i = 0; i < n; ++i) {
      gd_status s = do_build(c, nullptr, nullptr);
      if (s == GD_OK) s = do_rates(c, nullptr, nullptr);
      if (s == GD_OK) s = do_sample(c, nullptr, nullptr, nullptr);
      if (s == GD_OK && push) s = cuda_err(launch_push(c, -1.0));
      if (s != GD_OK) return s;
    }
    return GD_OK;
  }
  if (!c->graph_exec || c->graph_push != (push ? 1 : 0)) {
    if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
    cudaGraph_t g = nullptr;
    long long l0 = c->launches;
    // the captured build is replayed after the previous interval's push
    c->moved = push != 0;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GD_ERR_CUDA;
    gd_status s = do_build(c, nullptr, nullptr);
    if (s == GD_OK) s = do_rates(c, nullptr, nullptr);
    if (s == GD_OK) s = do_sample(c, nullptr, nullptr, nullptr);
    if (s == GD_OK && push) s = cuda_err(launch_push(c, -1.0));
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->intervals -= 1;          // the capture executed nothing
    c->launches = l0;
    c->graph_kernel_count = 0;
    if (s != GD_OK || e != cudaSuccess) { if (g) cudaGraphDestroy(g); return s != GD_OK ? s : GD_ERR_CUDA; }
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    for (size_t i = 0; i < nn; ++i) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
        c->graph_kernel_count++;
    }
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { c->graph_exec = nullptr; return GD_ERR_CUDA; }
    c->graph_push = push ? 1 : 0;
  }
  for (int i = 0; i < n; ++i) {
    if (cudaGraphLaunch(c->graph_exec, c->stream) != cudaSuccess) return GD_ERR_CUDA;
    c->intervals++;
    c->launches += c->graph_kernel_count;
  }
  c->phase = 0;
  return GD_OK;
}

extern "C" gd_status gd_stats(gd_ctx* c, gd_stats_t* out, gd_instance_stats* inst_out) {
  if (!c || !out) return GD_ERR_ARG;
  if (launch_stats(c, c->d_sums) != cudaSuccess) return GD_ERR_CUDA;
  if (inst_out && launch_spectrum(c) != cudaSuccess) return GD_ERR_CUDA;
  std::vector<StateDev> st(c->U);
  std::vector<BinsDev> bins(inst_out ? c->U : 0);
  if (inst_out && cudaMemcpyAsync(bins.data(), c->d_bins, sizeof(BinsDev) * c->U, cudaMemcpyDeviceToHost,
                                  c->stream) != cudaSuccess)
    return GD_ERR_CUDA;
  std::vector<double> sums(3 * (size_t)c->n_inst);
  std::vector<double> trad(c->n_inst, 0.0);
  if (inst_out && c->d_trad &&
      cudaMemcpyAsync(trad.data(), c->d_trad, sizeof(double) * c->n_inst, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return GD_ERR_CUDA;
  if (inst_out && !c->d_trad)
    for (int b = 0; b < c->n_inst; ++b) trad[b] = c->h_params[b].t_start;
  cudaError_t e = cudaMemcpyAsync(st.data(), c->d_state, sizeof(StateDev) * c->U, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sums.data(), c->d_sums, sizeof(double) * sums.size(), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return GD_ERR_CUDA;
  collect_timing(c);
  std::memset(out, 0, sizeof(*out));
  out->intervals = c->intervals;
  out->launches = c->launches;
  out->n_instances = c->n_inst;
  for (int k = 0; k < gd_ctx::kSlots; ++k) { out->kernel_ms[k] = c->ms[k]; out->kernel_calls[k] = c->calls[k]; }
  for (int b = 0; b < c->n_inst; ++b) {
    // an instance's units: one, or its spatial groups (C, dt and interval of group 0;
    // events and ties summed; status OR-ed)
    const int u0 = c->h_unit0[b], u1 = b + 1 < c->n_inst ? c->h_unit0[b + 1] : c->U;
    const StateDev& s = st[u0];
    long long events = 0, events_total = 0, near_draw = 0, near_dt = 0, near_audit = 0;
    unsigned status = 0;
    for (int u = u0; u < u1; ++u) {
      const StateDev& g = st[u];
      events += g.events;
      events_total += g.events_total;
      near_draw += g.near_draw;
      near_dt += g.near_dt;
      near_audit += g.near_audit;
      status |= g.status;
      out->knn_redo += g.knn_redo;
      out->rate_redo += g.rate_redo;
      out->sample_redo += g.sample_redo;
      out->sample_deferred += g.sample_deferred;
    }
    out->events += events_total;
    out->near_draw += near_draw;
    out->near_dt += near_dt;
    out->near_audit += near_audit;
    out->status |= status;
    if (inst_out) {
      gd_instance_stats& o = inst_out[b];
      std::memset(&o, 0, sizeof(o));
      o.C = s.C; o.dt_exe = s.dt_exe; o.dt_req = s.dt_req; o.dt_remain = s.dt_remain;
      o.sum_M = sums[3 * b]; o.sum_Mm = sums[3 * b + 1]; o.sum_Ms = sums[3 * b + 2];
      o.interval = s.interval_next;
      o.events = events;
      o.events_total = events_total;
      o.near_draw = near_draw; o.near_dt = near_dt; o.near_audit = near_audit;
      o.status = status;
      o.n_groups = s.n_groups;
      std::memcpy(o.spectrum, bins[u0].spec, sizeof(o.spectrum));
      o.t_rad = trad[b];
    }
  }
  if (out->status & GD_ST_NONFINITE) return GD_ERR_NONFINITE;
  if (out->status & GD_ST_EVENT_CAP) return GD_ERR_EVENT_CAP;
  if (out->status & GD_ST_CAPACITY) return GD_ERR_CAPACITY;
  if (out->status & GD_ST_TIMEOUT) return GD_ERR_TIMEOUT;
  return GD_OK;
}

extern "C" gd_status gd_controller_bins(gd_ctx* c, int32_t instance, double* A_out, double* B_out,
                                        int32_t* n_groups_out) {
  if (!c || instance < 0 || instance >= c->n_inst) return GD_ERR_ARG;
  BinsDev h;
  cudaError_t e = cudaMemcpyAsync(&h, c->d_bins + c->h_unit0[instance], sizeof(BinsDev), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return GD_ERR_CUDA;
  if (A_out) std::memcpy(A_out, h.gA, sizeof(h.gA));
  if (B_out) std::memcpy(B_out, h.gB, sizeof(h.gB));
  if (n_groups_out) *n_groups_out = h.ngroups;
  return GD_OK;
}

extern "C" gd_status gd_group_stats(gd_ctx* c, int32_t instance, int32_t group, gd_group_stats_t* out) {
  if (!c || !out || instance < 0 || instance >= c->n_inst) return GD_ERR_ARG;
  const int u0 = c->h_unit0[instance], u1 = instance + 1 < c->n_inst ? c->h_unit0[instance + 1] : c->U;
  if (group < 0 || group >= u1 - u0) return GD_ERR_ARG;
  StateDev h[2];
  cudaError_t e = cudaMemcpyAsync(&h[0], c->d_state + u0, sizeof(StateDev), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h[1], c->d_state + u0 + group, sizeof(StateDev), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return GD_ERR_CUDA;
  const StateDev& g = h[1];
  std::memset(out, 0, sizeof(*out));
  out->C = g.C;
  out->dt_exe = g.dt_exe;
  out->dt_req = g.dt_req;
  out->clock = (1LL << 60) - g.remain_ticks;
  out->members = g.members;
  out->intervals = g.intervals;
  out->events_total = g.events_total;
  out->near_dt = g.near_dt;
  out->near_draw = g.near_draw;
  out->interacts = g.inter;
  out->level = g.level;
  out->k_req = g.k_req;
  out->active = g.active;
  out->n_groups = g.n_groups;
  out->status = g.status;
  out->rounds = h[0].rounds;
  out->delayed = h[0].delayed;
  out->breaks = h[0].breaks;
  out->round_clock = h[0].clock;
  return GD_OK;
}

extern "C" gd_status gd_autotune(gd_ctx* c, double* factor_out, int32_t* xsplit_out) {
  if (!c) return GD_ERR_ARG;
  if (c->phase != 0 && c->phase != 1) return GD_ERR_STATE;
  static const double kFactors[] = {0.5, 0.6, 0.7, 0.8, 1.0, 1.2, 1.4};
  static const int kSplits[] = {1, 2, 4};
  const int saved_flags = c->flags;
  c->flags &= ~GD_FLAG_TIMING;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) { c->flags = saved_flags; return GD_ERR_CUDA; }
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); c->flags = saved_flags; return GD_ERR_CUDA; }
  double best = c->cell_factor;
  int best_split = c->cell_xsplit;
  float best_ms = 1e30f;
  gd_status st = GD_OK;
  for (int k = 0; k < 21 && st == GD_OK; ++k) {
    const double f = kFactors[k / 3];
    c->cell_factor = f;
    c->cell_xsplit = kSplits[k % 3];
    cudaError_t e = launch_cells(c);                  // warm-up: grid and lists for this size
    if (e == cudaSuccess) e = launch_knn(c);
    if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
    if (e == cudaSuccess) e = launch_cells(c);
    if (e == cudaSuccess) e = launch_knn(c);
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { st = GD_ERR_CUDA; break; }
    if (ms < best_ms) { best_ms = ms; best = f; best_split = c->cell_xsplit; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->flags = saved_flags;
  c->cell_factor = best;
  c->cell_xsplit = best_split;
  c->phase = 0;
  c->lists_valid = false;      // the ranks changed: the next collision step builds again
  if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; c->graph_push = -1; }
  if (factor_out) *factor_out = best;
  if (xsplit_out) *xsplit_out = best_split;
  return st;
}

extern "C" const char* gd_status_string(gd_status code) {
  switch (code) {
    case GD_OK: return "ok";
    case GD_ERR_ARG: return "invalid argument";
    case GD_ERR_CUDA: return "CUDA runtime error";
    case GD_ERR_OOM: return "device allocation failed";
    case GD_ERR_CAPACITY: return "library buffer capacity exceeded";
    case GD_ERR_NONFINITE: return "non-finite rate";
    case GD_ERR_EVENT_CAP: return "event cap reached";
    case GD_ERR_TIMEOUT: return "bounded device wait gave up";
    case GD_ERR_STATE: return "calls out of order";
  }
  return "unknown status";
}
