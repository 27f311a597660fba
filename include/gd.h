/*
 * gd.h -- C ABI of the GB300 collision-step library (libgd.so).
 *
 * One call sequence advances every instance by one frozen-neighbour interval
 * of the representative-particle Monte Carlo of "GameDev: GPU-accelerated
 * model for dust evolution" (Sect. 2.5):
 *
 *   gd_build_neighbors    K nearest neighbours over a device cell list,
 *                         sampling measures                      (Sect. 2.5.1)
 *   gd_collision_rates    pair rates lambda_ij = n_ij K_ij, outcome channels,
 *                         controller-bin moments and the executed interval
 *                                                        (Sect. 2.5.1-2.5.3)
 *   gd_sample_collisions  Gillespie sampling of events against the frozen
 *                         neighbourhood, mass/weight updates      (Sect. 2.5.3)
 *   gd_push_staggered     staggered semi-analytic trajectory step (Sect. 2.3.3),
 *                         with radiation forces                   (Sect. 2.3.2)
 *   gd_optical_depth      the optical depth grid of the radiation forces
 *                                                                 (Sect. 2.3.2)
 *   gd_stats              reductions and counters (the only call that
 *                         synchronises the stream)
 *
 * Conventions
 *  - Units: cgs.  s is the grain diameter, M the represented particle mass
 *    (constant), N = M/m with m = pi rho_o s^3 / 6 (Sect. 2).
 *  - Particles of all instances are concatenated (CSR): instance b owns the
 *    global indices [offsets[b], offsets[b+1]).  Every pointer to particle
 *    data is a DEVICE pointer owned by the caller, who must keep it alive for
 *    the life of the context; the library reads and writes it in place
 *    (s, and x, y, z, vr, lth, lph in gd_push_staggered) and never writes M.
 *  - The library owns its scratch (cell lists, neighbour lists in cell order,
 *    frozen snapshots, controller bins, per-instance state); gd_create
 *    allocates it with cudaMalloc, gd_destroy frees it.
 *  - Every call except gd_stats and gd_destroy only enqueues work on the
 *    context's stream and is asynchronous.  Argument and sequencing errors
 *    return at once; errors found on the device set sticky status bits that
 *    gd_stats reports (GD_ST_*).  No call aborts the process or traps the GPU.
 *  - Optional *_out pointers are caller DEVICE buffers (NULL: not written).
 */
#ifndef GD_H
#define GD_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gd_ctx gd_ctx;

typedef enum {
  GD_OK = 0,
  GD_ERR_ARG = -1,       /* invalid argument                                  */
  GD_ERR_CUDA = -2,      /* a CUDA runtime call failed                         */
  GD_ERR_OOM = -3,       /* device allocation failed                           */
  GD_ERR_CAPACITY = -4,  /* a library-owned buffer is too small                */
  GD_ERR_NONFINITE = -5, /* a rate was NaN or infinite                         */
  GD_ERR_EVENT_CAP = -6, /* a particle reached max_events_per_interval         */
  GD_ERR_TIMEOUT = -7,   /* a bounded device wait gave up                      */
  GD_ERR_STATE = -8      /* calls out of order (e.g. rates before neighbours)   */
} gd_status;

/* precision of the path */
enum {
  GD_FP64 = 0,   /* every step in FP64                                         */
  GD_MIXED = 1   /* FP32 distances (FP64 re-rank at the K boundary), FP32 pair
                    rates; FP64 prefix sums, waiting times, masses and weights  */
};

enum { GD_GEOM_PATCH = 0, GD_GEOM_DISK = 1 };
enum { GD_DIFF_PHYSICAL = 0, GD_DIFF_RING = 1 };   /* gd_diffuse models */
/* Collision models of Sect. 2.5.1 by the dimensions they resolve.  The neighbour
 * search runs in the model's coordinates and V_i is the model's measure:
 *   GD_MODEL_3D   (x, y, z); V = 4 pi d^3 / 3 (spherical caps at disk edges)
 *   GD_MODEL_RZ   2D radial-polar, the meridional plane (R, Z); V = A 2 pi R,
 *                 A = pi d^2 minus the circular segments beyond a radial edge
 *   GD_MODEL_RPHI 2D radial-azimuthal, vertically integrated, the midplane (x, y);
 *                 V = A sqrt(2 pi (H_i^2 + H_j^2)) with H_i = H_j = H_g(R_i)
 *   GD_MODEL_R    1D radial, R; V = pi (R_hi^2 - R_lo^2) over [R - d, R + d]
 *                 clipped at the edges, times the same vertical length; a
 *                 context holds 1D instances only or none (GD_ERR_ARG)
 * The vertically integrated models (RPHI, R) evaluate the gas and the pair
 * speeds in the midplane.  gd_push_staggered, gd_diffuse and gd_timestep move
 * and limit the 3D positions whatever the model. */
enum { GD_MODEL_3D = 0, GD_MODEL_RZ = 1, GD_MODEL_RPHI = 2, GD_MODEL_R = 3 };
/* Optical depth forms of Sect. 2.3.2: along r from the 3D dust density (Eq. tau_3d);
 * along R in the midplane from the surface density over sqrt(2 pi) H_g (Eq. tau_2d). */
enum { GD_TAU_3D = 0, GD_TAU_2D = 1 };
enum { GD_KERNEL_PHYSICAL = 0, GD_KERNEL_CONSTANT = 1, GD_KERNEL_LINEAR = 2,
       GD_KERNEL_PRODUCT = 3 };

/* sticky device status bits */
enum {
  GD_ST_EVENT_CAP = 1 << 0,  /* a particle reached max_events_per_interval      */
  GD_ST_DT_FLOOR = 1 << 1,   /* requested interval below dt_coll / 2^60          */
  GD_ST_NONFINITE = 1 << 2,  /* NaN or infinite rate                             */
  GD_ST_KNN = 1 << 3,        /* neighbour search could not find K-1 others       */
  GD_ST_CAPACITY = 1 << 4,   /* cell grid exceeded its capacity                  */
  GD_ST_TIMEOUT = 1 << 5     /* a bounded device wait gave up                    */
};

/* flags of gd_config.flags */
enum {
  GD_FLAG_TIMING = 1 << 0,   /* time every kernel with CUDA events (gd_stats)   */
  GD_FLAG_NO_AUDIT = 1 << 1  /* keep the safety factor C at 1 in all instances  */
};

/* Per-instance parameters (Sect. 2.2 gas disk, Sect. 2.5 collision model). */
typedef struct {
  int32_t geometry;    /* GD_GEOM_PATCH: local patch, x radial / y azimuthal
                          offsets in [-box/2, box/2), both periodic, z free;
                          GD_GEOM_DISK: global disk, R = sqrt(x^2+y^2)        */
  int32_t kernel_mode; /* GD_KERNEL_*: physical kernel or an Appendix A test
                          kernel (V_i = 1, lambda_ij = (1/t0)(1/N_K)(m0/m_j) K) */
  int32_t audit;       /* 1: adaptive safety factor C; 0: C = 1              */
  int32_t model;       /* GD_MODEL_*: dimensions the collision model resolves
                          (Sect. 2.5.1); RZ and R need GD_GEOM_DISK          */
  double r0;           /* reference radius R_0 (patch: its radius) [cm]      */
  double sigma0;       /* gas surface density at R_0 [g cm^-2]               */
  double p;            /* Sigma_g ~ R^p                                      */
  double T0;           /* temperature at R_0 [K]                             */
  double q;            /* T ~ R^q                                            */
  double alpha;        /* viscosity parameter                                */
  double M_star;       /* stellar mass [g]                                   */
  double rho_s;        /* grain internal density rho_o [g cm^-3]             */
  double s_min;        /* minimum fragment diameter [cm]                     */
  double v_frag;       /* fragmentation speed [cm s^-1]                      */
  double eps;          /* interval tolerance epsilon                         */
  double dt_coll;      /* collision timestep [s]                             */
  double dt_fn_max;    /* maximum frozen-neighbour interval [s]              */
  double R_in, R_out;  /* global disk radial edges [cm] (flat-boundary caps)  */
  double box_x, box_y; /* patch periodic extents [cm]                        */
  double t0, m0;       /* test-kernel unit time and mass                     */
  double cell_size;    /* cell edge [cm]; <= 0: chosen from the data          */
  uint64_t seed;       /* Philox key of the instance                         */
  int32_t diff_mode;   /* gd_diffuse: GD_DIFF_PHYSICAL, D = nu/(Sc (1+St^2))
                          with nu = alpha c_s H_g (Sect. 2.4); GD_DIFF_RING, the
                          ring test of Sect. 3.2: radial only, D = D0 (R/R_0)^2 */
  int32_t diff_chi;    /* 1: concentration diffusion (drift along ln rho_g);
                          0: density diffusion                                */
  double Sc_R, Sc_Z, Sc_phi;  /* Schmidt numbers of the three directions
                                 (<= 0: 1)                                    */
  double D0;           /* ring test: D at R_0 [cm^2 s^-1]                     */
  int32_t spatial_groups;  /* G, 0 or 1: one group; 2 .. 64: the instance is split
                              into G spatial groups of equal width (Sect. 2.5.3),
                              radial annuli of a disk over [R_in, R_out) by
                              R = sqrt(x^2 + y^2), slabs of a patch over x in
                              [-box_x/2, box_x/2) (beyond the edges: the first or
                              last group); see gd_group_stats                    */
  int32_t pad_sg;
  /* Radiation forces (Sect. 2.3.2; global disks, gd_push_staggered) and the optical
   * depth grid (gd_push_staggered, gd_optical_depth).  beta(s) = beta0 s0/s and
   * kappa(s) = kappa0 s0/s with s0 = rad_s0; beta0 = 0: the push has no radiation
   * forces; kappa0 = 0 or tau_nr = 0: tau = 0.                                  */
  double beta0;        /* radiation pressure over gravity at diameter rad_s0     */
  double kappa0;       /* opacity at rad_s0 for the optical depth [cm^2 g^-1]     */
  double rad_s0;       /* reference diameter s0 [cm] (> 0 when beta0 or kappa0 is) */
  double t_beta;       /* taper time scale [s]: forces times xi^2 (3 - 2 xi),
                          xi = min(max(t / t_beta, 0), 1) at the kick's time;
                          <= 0: no taper                                         */
  int32_t rad_pr;      /* 1: Poynting-Robertson drag                             */
  int32_t tau_geom;    /* GD_TAU_3D or GD_TAU_2D                                 */
  int32_t tau_nr;      /* grid cells in r (3D) or R (2D); 0: no grid             */
  int32_t tau_nmu;     /* 3D: cells in mu = cos theta over [-tau_mu, tau_mu)     */
  int32_t tau_nphi;    /* cells in phi over [-pi, pi)                            */
  int32_t pad_tau;
  double tau_rmin, tau_rmax;  /* radial extent of the grid [cm]                  */
  double tau_mu;       /* 3D: polar extent, 0 < tau_mu <= 1                      */
  double t_start;      /* the taper's clock at gd_create [s]; every push of a
                          context with radiation forces advances it by its dt    */
} gd_instance_params;

typedef struct {
  int32_t n_instances;
  int32_t K;                   /* N_K, neighbours including the particle itself, 2..256 */
  int32_t precision;           /* GD_FP64 or GD_MIXED                         */
  int32_t flags;               /* GD_FLAG_*                                   */
  const int64_t* offsets;      /* HOST [n_instances + 1], offsets[0] = 0      */
  const gd_instance_params* params;  /* HOST [n_instances]                   */
  double* x;                   /* DEVICE [N] positions [cm]                   */
  double* y;
  double* z;
  double* s;                   /* DEVICE [N] diameters [cm], updated in place */
  const double* M;             /* DEVICE [N] particle masses [g], read only    */
  double* vr;                  /* DEVICE [N] or NULL: v_r      (push only)    */
  double* lth;                 /* DEVICE [N] or NULL: l_theta  (push only)    */
  double* lph;                 /* DEVICE [N] or NULL: l_phi    (push only)    */
  void* stream;                /* cudaStream_t; NULL = legacy default stream  */
  int64_t max_events_per_interval;   /* per particle; <= 0: 65536              */
  double cell_factor;          /* cell edge = factor (V_box/N)^(1/3) when the
                                  instance gives none; <= 0: 1                 */
  int32_t cell_xsplit;         /* cell x edge = the y/z edge divided by 1, 2 or 4;
                                  0: 1                                         */
  int32_t pad1;
} gd_config;

/* Library-wide counters (gd_stats). */
typedef struct {
  int64_t intervals;           /* completed gd_sample_collisions calls         */
  int64_t events;              /* all events so far                            */
  int64_t near_draw;           /* draws within the tie tolerance of a rate or
                                  time boundary (1e-10 FP64 form, 2e-5 mixed)  */
  int64_t near_dt;             /* interval choices within the tolerance of an edge */
  int64_t near_audit;          /* audit decisions within the tolerance of the threshold */
  int64_t launches;            /* kernels launched by the path so far (the two
                                  reductions of gd_stats itself not included) */
  uint32_t status;             /* OR of every instance's GD_ST_* bits          */
  int32_t n_instances;
  double kernel_ms[8];         /* GD_FLAG_TIMING: summed kernel time by step:
                                  0 cells, 1 knn, 2 rates, 3 interval, 4 sample,
                                  5 push, 6 stats/other, 7 diffusion           */
  int64_t kernel_calls[8];     /* launches timed in each slot                  */
  int64_t knn_redo;            /* mixed form: neighbour searches the FP32 keys
                                  could not decide, redone in FP64 (all builds) */
  int64_t rate_redo;           /* mixed form: particles whose pair rates the FP32
                                  error bounds could not certify, redone in FP64 */
  int64_t sample_redo;         /* mixed form: particles with an uncertified sampling
                                  decision, replayed in FP64 (all intervals) */
  int64_t sample_deferred;     /* of those, heavy particles whose open time decision
                                  the deferred FP64 pass settled from their logged
                                  events (all intervals) */
} gd_stats_t;

/* Per-instance state and reductions (gd_stats). */
typedef struct {
  double C;                    /* safety factor                                */
  double dt_exe;               /* executed interval of the last call [s]       */
  double dt_req;               /* requested interval of the last call [s]      */
  double dt_remain;            /* time left in the collision timestep [s]      */
  double sum_M;                /* sum of M_i                                   */
  double sum_Mm;               /* sum of M_i m_i (mass-weighted mean mass numerator) */
  double sum_Ms;               /* sum of M_i s_i                               */
  int64_t interval;            /* intervals executed                           */
  int64_t events;              /* events of the last interval                  */
  int64_t events_total;
  int64_t near_draw, near_dt, near_audit;
  uint32_t status;             /* GD_ST_* bits of this instance                */
  int32_t n_groups;            /* controller bins of the last interval         */
  double spectrum[96];         /* size spectrum: sum of M_i over the particles whose
                                  diameter lies in fine log-size bin f, which covers
                                  s in [2^((f - 75)/3), 2^((f - 74)/3)) cm (a third of an
                                  octave, ~0.1 dex; the first and last bins also take
                                  the sizes below and above); summed in a fixed order */
  double t_rad;                /* the radiation taper's clock [s] (t_start plus the
                                  pushes' dt in a context with radiation forces) */
} gd_instance_stats;

/* Creates a context over caller-owned particle arrays (see gd_config): the
 * representative particles of Sect. 2 (position, diameter s_i, particle mass M_i)
 * of one or more instances, each with the gas disk of Sect. 2.2 and the
 * collision-model parameters of Sect. 2.5.  Checks every argument (each instance
 * must hold at least K = N_K particles, Sect. 2.5.1), copies the parameter tables
 * to the device and allocates the library's scratch.
 * Returns GD_ERR_ARG, GD_ERR_OOM or GD_ERR_CUDA on failure (*out = NULL). */
gd_status gd_create(gd_ctx** out, const gd_config* cfg);

/* Waits for the context's stream, frees everything the library allocated (a
 * service of the library; the paper has no counterpart). */
gd_status gd_destroy(gd_ctx* ctx);

/* Sect. 2.5.1: bins every particle into a per-instance uniform cell grid
 * (counting sort by cell), then finds each particle's N_K nearest particles
 * of its instance, itself included at zero distance (minimum image across a
 * patch's periodic edges), ranked by (d^2, index) with
 * d^2 = (dx dx + dy dy) + dz dz in FP64.  Lists hold the particle itself in
 * slot 0 and the other K-1 in ascending index order (the channel order used
 * for sampling).  Also computes d_i (distance to the farthest retained
 * neighbour), the sampling measure V_i = 4 pi d_i^3 / 3 minus flat-boundary
 * caps at a global disk's radial edges (Sect. 2.5.1), and freezes the partner
 * properties (s, m, N) for the interval (Sect. 2.5.3).
 * nbr_out: DEVICE int32 [N*K] or NULL, global particle indices, row i for
 * particle i.  d_out: DEVICE double [N] or NULL. */
gd_status gd_build_neighbors(gd_ctx* ctx, int32_t* nbr_out, double* d_out);

/* Sect. 2.5.1-2.5.3: for every particle and slot, the relative speed
 * (radial drift, settling, azimuthal, Brownian and turbulent terms at the
 * query particle's position), K_ij = pi (s_i+s_j)^2 dv / 4,
 * lambda_ij = N_j K_ij / V_i, the outcome (sticking / erosion / fragmentation)
 * with grouping N_coll, the effective channel rates lambda*_ij and
 * lambda*_i = sum_j lambda*_ij; then the controller-bin moments A_b, B_b and,
 * per instance, dt_req = min(dt_remain, dt_fn_max, eps C / A_b,
 * eps^2 C^2 / B_b) and dt_exe = dt_coll / 2^k (smallest k with dt_exe <=
 * dt_req).  Requires gd_build_neighbors since the last sampling.
 * lambda_out: DEVICE double [N] or NULL: lambda*_i.
 * chan_out: DEVICE double [N*K*2] or NULL: lambda*_ij per slot and channel. */
gd_status gd_collision_rates(gd_ctx* ctx, double* lambda_out, double* chan_out);

/* Sect. 2.5.3: each particle draws waiting times -ln U / lambda*_i until they
 * exceed dt_exe; each event picks a channel with probability
 * lambda*_ij / lambda*_i, applies the outcome to the particle alone (M kept,
 * N' = M/m'), and refreshes the particle's own rates against the frozen
 * partners.  Draws: Philox4x32-10, key = instance seed, counter =
 * (index within instance, interval, event, 0|1).  Writes the new diameters
 * into cfg.s and runs the post-interval audit of C.  Requires
 * gd_collision_rates since the last build.
 * ev_count_out, ev_hash_out, near_out: DEVICE [N] or NULL: events of each
 * particle, a hash of its chosen channel sequence, and its near ties. */
gd_status gd_sample_collisions(gd_ctx* ctx, int32_t* ev_count_out, uint32_t* ev_hash_out,
                               int32_t* near_out);

/* Sect. 2.3.3: one staggered semi-analytic step of length dt (dt < 0: each
 * instance's last dt_exe) for every particle of every global-disk instance:
 * drift half a step, exact linear-drag kick toward the gas velocity with
 * gravity and the angular-momentum forces at the midpoint, drift the second
 * half in mirrored order.  Needs vr, lth, lph in the config.  GD_MIXED: the
 * drifts rotate the FP64 position by FP32 angle increments (about z by
 * h l_phi / R^2, in the meridional plane by h l_theta / r^2) and scale it by
 * 1 + h v_r / r; the forces are FP64, the gas disk and the drag factor FP32. */
gd_status gd_push_staggered(gd_ctx* ctx, double dt);
/*
 * With radiation forces (an instance with beta0 > 0; Sect. 2.3.2) the same step adds
 *   f_RP = beta e^-tau GM/r^2 r_hat to the kick's radial force, and with rad_pr the
 *   Poynting-Robertson damping gamma_PR = beta e^-tau GM/(c r^2) to the drag rates:
 *   gamma_r = 1/t_s + 2 gamma_PR, gamma_theta = gamma_phi = 1/t_s + gamma_PR, each
 *   component advanced exactly for fixed rates, y += k (f + y_g/t_s - gamma y),
 *   k = (1 - e^{-gamma dt})/gamma;
 * beta e^-tau carries the taper at the instance clock + dt/2.  tau is rebuilt every
 * push from all particles at the midpoint of the first drift (the grid of
 * gd_optical_depth) and interpolated at each particle's midpoint.  Such a push is
 * four kernels (first drift with the deposit, column sums, kick with the second
 * drift, clock); instances without beta0 take the plain step.  GD_MIXED: the cell of
 * the deposit is decided in FP32 where certified (FP64 near a cell edge), tau is
 * interpolated in FP32, the radiation factors are FP32 and the forces FP64.
 */

/* Sect. 2.3.2: the optical depth of every instance with a grid (tau_nr > 0 and
 * kappa0 > 0) from the particles at their current positions.  Readings of the paper,
 * which names neither grid nor deposit:
 *  - cells uniform in r over [tau_rmin, tau_rmax), in mu = z/r over
 *    [-tau_mu, tau_mu) and in phi = atan2(y, x) over [-pi, pi) (3D); in R and phi
 *    with one polar cell (2D); a column is one (mu, phi) cell, j * tau_nphi + k;
 *  - each particle adds kappa(s) M to the cell holding it (none outside the grid);
 *    the cell's kappa rho_d is that sum over the cell volume (r_hi^3 - r_lo^3)/3
 *    dmu dphi, or kappa Sigma_d / (sqrt(2 pi) H_g) over the area
 *    (R_hi^2 - R_lo^2)/2 dphi with H_g at the cell's mid radius (2D);
 *  - tau at the radial faces: T_0 = 0, T_{i+1} = T_i + (kappa rho_d)_i dr (no
 *    extinction inside tau_rmin);
 *  - at a point: linear in r between its column's faces, bilinear between the
 *    centres of the four nearest columns (clamped at the polar edges, periodic in
 *    phi), 0 inside tau_rmin and the outer face beyond tau_rmax.
 * The cell sums are exact (128-bit fixed point with the scale of the instance's
 * largest kappa M, 2^-60 of it) and independent of scheduling.
 * tau_out: DEVICE [N] or NULL: tau at each particle (0 for instances without a grid).
 * grid_out: DEVICE or NULL: T of the instances with a grid, in instance order, each
 *   as [column][face] = tau_nmu' * tau_nphi * (tau_nr + 1) doubles (tau_nmu' = 1 in 2D).
 * Returns GD_ERR_ARG if no instance has a grid.  Asynchronous. */
gd_status gd_optical_depth(gd_ctx* ctx, double* tau_out, double* grid_out);

/* Sect. 2.4: one Euler-Maruyama dust diffusion step of length dt (dt < 0: each
 * instance's last dt_exe) for every particle.  The tensor is diagonal in the
 * local cylindrical basis, D_a = nu/(Sc_a (1 + St^2)); the step is
 *   dR = sqrt(2 D_R dt) zeta_R + (D_R/R + dD_R/dR + chi D_R dln rho_g/dR) dt,
 *   dZ = sqrt(2 D_Z dt) zeta_Z + (dD_Z/dZ + chi D_Z dln rho_g/dZ) dt,
 *   dphi = sqrt(2 D_phi dt) zeta_phi / R,
 * with the derivatives of the analytic gas disk and zeta from Philox4x32-10
 * (key = instance seed, counter = (index in the instance, call number,
 * 0xFFFFFFFE, 0 or 1), Box-Muller).  Global disk: applied in (R, phi, Z); with
 * velocities in the config their Cartesian vector is kept and (v_r, l_theta,
 * l_phi) are recomputed at the new position.  Local patch: x += dR,
 * y += R dphi, z += dZ, wrapped.  GD_DIFF_RING: radial only with D = D0 (R/R_0)^2.
 * GD_MIXED: FP32 draws and coefficients, the displacement applied to the FP64
 * position (a rotation by dphi and the factor 1 + dR/R), the velocities
 * re-projected in FP64 from the direction cosines of the two positions.
 * Positions are written in place (x, y, z; vr, lth, lph when given).
 * Returns GD_ERR_ARG for a non-finite dt.  Asynchronous. */
gd_status gd_diffuse(gd_ctx* ctx, double dt);

/* Sect. 2.5.3 with a bounded collision step: every instance runs frozen-neighbour
 * intervals (build or reuse the lists, rates, interval choice, sampling, audit)
 * over a collision step of length tau (in place of dt_coll), the intervals
 * halving tau exactly, and idles once its step is used up; the call returns
 * when every instance has finished.  Positions are frozen during the step, so
 * the neighbour lists are built once: by the first interval, or not at all
 * when reuse_lists != 0 and the particles have not moved since the last build
 * (the caller's promise for its own changes; a gd_diffuse or gd_push_staggered
 * call since the last build makes the step build anyway).  Later intervals refresh only the partner snapshot.
 * Synchronises the stream after every interval (the number of intervals is
 * data dependent).  max_intervals bounds the loop: GD_ERR_TIMEOUT when it is
 * reached first.  n_intervals_out: HOST or NULL.  Afterwards the instances are
 * back to collision steps of dt_coll.  GD_ERR_ARG for tau <= 0 or non-finite,
 * GD_ERR_STATE between a build and its sampling. */
gd_status gd_collide(gd_ctx* ctx, double tau, int32_t reuse_lists, int32_t max_intervals,
                     int32_t* n_intervals_out);

/* Sect. 2.6: one numerical timestep of length dt in the symmetric split
 * C(dt/2) D(dt/2) T(dt) D(dt/2) C(dt/2): collisions (gd_collide), diffusion
 * (gd_diffuse), transport (gd_push_staggered, when the config has velocities;
 * patch instances do not move).  The first C reuses the lists of the previous
 * call's last C when reuse_lists != 0 (nothing moves between the two); the last
 * C rebuilds them.  n_intervals_out: HOST or NULL, the intervals of both C. */
gd_status gd_step(gd_ctx* ctx, double dt, int32_t reuse_lists, int32_t* n_intervals_out);

/* Sect. 2.6: the common transport timestep of every particle of the context,
 *   dt = min(dt_max, dt_out, min_i dt_i),
 * dt_i the most restrictive local limit of particle i (the paper names the
 * limits, orbital motion and the deterministic and diffusive displacements
 * against the local grid spacing, not their form; this is the form taken):
 *   orbital        f_orb * 2 pi / Omega_K(R_i)
 *   deterministic  c_adv * dx_i / |u_i|, u_i = (v_r, l_theta / r, l_phi / R -
 *                  Omega_K R) the velocity relative to the local circular Keplerian
 *                  motion; global-disk particles of a config with velocities only
 *   diffusive      (c_diff * dx_i)^2 / (2 D_i), D_i the largest directional
 *                  coefficient of gd_diffuse's model at the particle
 * with dx_i = dx_H * H_g(R_i) (the analytic disk has no grid: the caller states
 * its resolution in local gas scale heights).  A limit whose coefficient is <= 0
 * is off.  GD_FP64: FP64 throughout; GD_MIXED: each dt_i in FP32 (a few ulps of
 * the gas disk's powers and exponential; the deterministic limit's azimuthal
 * speed l_phi / R - sqrt(GM / R) from an FP64 difference of squares, so that
 * it does not cancel), the minimum exact over the FP32 values.  dt_out_host: HOST, required, receives
 * dt.  dti_out: DEVICE [N] caller order, or NULL, receives every dt_i (+infinity
 * where no limit applies).  Synchronises the stream.  GD_ERR_ARG for a missing
 * rule, dt_max or dt_out not > 0, a non-finite coefficient, or dx_H not > 0 and
 * finite with c_adv or c_diff on; GD_ERR_NONFINITE when some dt_i is NaN or not
 * > 0 (dt is still written, from the other particles). */
typedef struct {
  double dt_max;       /* prescribed maximum timestep [s]                      */
  double dt_out;       /* time left before the next output [s] (HUGE_VAL: none) */
  double f_orb;        /* orbital limit, fraction of the local Keplerian period */
  double dx_H;         /* local grid spacing in local gas scale heights        */
  double c_adv;        /* deterministic displacement per step, in spacings     */
  double c_diff;       /* diffusive displacement sqrt(2 D dt), in spacings     */
} gd_dt_rule;
gd_status gd_timestep(gd_ctx* ctx, const gd_dt_rule* rule, double* dt_out_host, double* dti_out);

/* Synchronises the stream, reduces per-instance sums and copies counters: the
 * mass bookkeeping of Sect. 2.5.2 (sum M_i, which no call writes, and sum M_i m_i,
 * sum M_i s_i with N_i = M_i / m_i), the size spectrum, the interval state of
 * Sect. 2.5.3 (C, dt_exe, dt_req, time left) and the event and near-tie counts.
 * out: HOST, required.  inst_out: HOST [n_instances] or NULL.
 * Returns the first device error as a gd_status (GD_OK if none). */
gd_status gd_stats(gd_ctx* ctx, gd_stats_t* out, gd_instance_stats* inst_out);

/* Sect. 2.5.3: the controller bins of one instance's last interval choice.  A_b and B_b
 * are the mass-weighted means over a bin's particles of sum_o lambda*_io <J_io> and of
 * sum_o lambda*_io <J_io^2> (J = |ln(s'/s)| of each outcome channel o), the bins in
 * ascending size; dt_req took min_b eps C / A_b and min_b eps^2 C^2 / B_b.  The fine-bin
 * sums behind them are formed in a fixed order, so they do not depend on scheduling.
 * Synchronises the stream.  instance: 0 .. n_instances - 1 (else GD_ERR_ARG).
 * A_out, B_out: HOST [96] or NULL, bins past n_groups are 0; n_groups_out: HOST or NULL. */
gd_status gd_controller_bins(gd_ctx* ctx, int32_t instance, double* A_out, double* B_out,
                             int32_t* n_groups_out);

/* Sect. 2.5.3, spatial groups (instances with spatial_groups = G > 1).  Each group
 * keeps its own controller bins, safety factor C, interval level k (dt_exe =
 * dt_coll 2^-k), clock and Philox interval counter.  Two groups interact when a
 * neighbour list of one holds a particle of the other.  On such an instance one
 * interval call (gd_collision_rates + gd_sample_collisions, one interval of
 * gd_collide or gd_run_intervals) is one ROUND: the groups whose scheduled interval
 * ends earliest broadcast their particles' sizes into the partner snapshot (the
 * others' particles keep being read as they last broadcast them), request a level by
 * the single-group rule, and are scheduled:
 *   - a group ends inside the collision step (its remaining time bounds its level);
 *   - against an interacting group in the middle of its interval (which is kept)
 *     the level stays within 4 (a ratio of 16): a coarser request is refined, a
 *     finer one waits at that group's level + 4 (a delayed refinement) -- the
 *     collision step's end wins over the ratio (counted in breaks);
 *   - interacting groups of the same round: finest-allowed levels propagate along
 *     the interactions (+4 per step), each group takes its request within its
 *     bounds, then the coarser of two interacting groups is refined until they are
 *     within 4.
 * Then the round's groups sample their intervals and audit them; the other groups'
 * particles are idle (no events).  The step ends when every group reached its end;
 * the next round starts the next step with every group.  Positions (and so groups
 * and interactions) are taken at the neighbour build and stay frozen in the step.
 * gd_push_staggered and gd_diffuse with dt < 0, and gd_run_intervals with push, take
 * no grouped instance (GD_ERR_ARG).  gd_instance_stats of a grouped instance: C,
 * dt_exe, dt_req, dt_remain and interval of group 0, events and ties summed over the
 * groups, status OR-ed. */
typedef struct {
  double C;                    /* safety factor of the group                    */
  double dt_exe;               /* its last executed interval [s] (0 when the
                                  group was idle in the last round)             */
  double dt_req;               /* its last requested interval [s]               */
  int64_t clock;               /* its time in the step, ticks of dt_coll / 2^60:
                                  the end of its scheduled interval            */
  int64_t members;             /* particles of the group at the last build      */
  int64_t intervals;           /* intervals the group executed                  */
  int64_t events_total;        /* its events so far                             */
  int64_t near_dt, near_draw;  /* its ties (interval choice; draws)             */
  uint64_t interacts;          /* bit h: the group interacts with group h       */
  int32_t level;               /* k of its scheduled (or last) interval; -1 none */
  int32_t k_req;               /* k it requested in its last round              */
  int32_t active;              /* 1: it took part in the last round             */
  int32_t n_groups;            /* its controller bins                           */
  uint32_t status;             /* its GD_ST_* bits                              */
  int32_t pad;
  /* per instance (the same in every group of it) */
  int64_t rounds;              /* rounds so far                                 */
  int64_t delayed;             /* requests held coarser by a scheduled interval */
  int64_t breaks;              /* interacting pairs left more than 16 apart     */
  int64_t round_clock;         /* clock of the last round (ticks)               */
} gd_group_stats_t;

/* The state of group `group` of instance `instance` (both 0-based; a one-group
 * instance has group 0 only).  Synchronises the stream.  out: HOST, required.
 * GD_ERR_ARG for an index out of range. */
gd_status gd_group_stats(gd_ctx* ctx, int32_t instance, int32_t group, gd_group_stats_t* out);

/* Runs n whole intervals (build, rates, sample and, if push != 0, push with
 * dt_exe) by replaying a CUDA graph of one interval captured on first use
 * (captures again if the arguments change); on instances with spatial groups an
 * interval is a round.  Asynchronous. */
gd_status gd_run_intervals(gd_ctx* ctx, int32_t n, int32_t push);

/* Autotuner: times the cell binning and neighbour search (gd_build_neighbors'
 * kernels) on the current positions for a set of cell shapes -- the y and z edge
 * is factor * (V_box / N)^(1/3) for factor in {0.5, 0.6, 0.7, 0.8, 1.0, 1.2, 1.4},
 * the x edge that divided by 1, 2 or 4 -- with CUDA events, and keeps the fastest
 * for the context (instances with an explicit cell_size keep their edge).  Results never depend on the choice: the lists
 * are exact for any cell size.  Synchronises the stream; call it before
 * gd_run_intervals captures its graph.  Leaves the context ready for
 * gd_build_neighbors.  factor_out, xsplit_out: HOST or NULL, receive the chosen
 * factor and x division. */
gd_status gd_autotune(gd_ctx* ctx, double* factor_out, int32_t* xsplit_out);

/* Static string for a gd_status code. */
const char* gd_status_string(gd_status code);

/* ---------------------------------------------------------------------------
 * No-allocation neighbour search (this entry point has no counterpart in the
 * paper; it is a service to callers).
 *
 * For callers that cannot allocate device memory at run time: a host program
 * that has already reserved the GPU's memory for its own pool, or a
 * latency-bound loop that cannot take cudaMalloc's implicit synchronisation.
 * gd_neighbors_fixed calls no cudaMalloc, cudaFree or allocating library
 * routine.  Its scratch is one fixed device array of GD_FIXED_SCRATCH_BYTES
 * bytes inside libgd.so, which every GPU that loads the library holds until
 * the process exits.
 *
 * It computes, for ONE instance, the lists gd_build_neighbors would return
 * (FP64 keys, minimum image in a patch): nbr_out row i = i, then the K-1
 * nearest others by (d^2, index) in ascending index order; d_out[i] = distance
 * to the farthest of them.  x, y, z: DEVICE [n]; nbr_out: DEVICE int32 [n*K];
 * d_out: DEVICE [n] or NULL; params: HOST, only geometry, box_x, box_y and
 * cell_size are read; stream: cudaStream_t (NULL = legacy default stream).
 *
 * Limits: n <= GD_FIXED_MAX_PARTICLES (else GD_ERR_CAPACITY, nothing runs),
 * 2 <= K <= GD_FIXED_MAX_K and K <= n, params->model == GD_MODEL_3D (else
 * GD_ERR_ARG).  A query whose search finds no K-1 others within its bounded
 * number of radius growths (a non-finite coordinate) gets a row of -1 and
 * d_out = -1; the call is asynchronous and still returns GD_OK, so a caller that
 * can meet such input checks row[0] >= 0 after synchronising.
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and keeps it for the life of the
 * process; make that first call before any stream capture, and do not use the
 * library across a cudaDeviceReset, which would leave the kept address stale.
 * All calls share the one array, which keeps the last call's contents (each call
 * clears what must start at zero): calls that overlap on the GPU -- on different
 * streams, or from different threads -- race, so serialise them.  Asynchronous
 * on the stream like the other calls.
 * ------------------------------------------------------------------------- */
#define GD_FIXED_MAX_PARTICLES 65536
#define GD_FIXED_MAX_K 64
#define GD_FIXED_SCRATCH_BYTES 4719360
gd_status gd_neighbors_fixed(const double* x, const double* y, const double* z, int64_t n,
                             int32_t K, const gd_instance_params* params, int32_t* nbr_out,
                             double* d_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
