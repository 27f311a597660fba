/*
 * gdo.h -- plain, serial, FP64 CPU oracle of the GameDev collision step
 * (representative-particle Monte Carlo with frozen neighbourhoods).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load, call or run this code.
 * It shares no code, header, table or constant with the CUDA library; it is
 * written from the paper's definitions, step by step, with no blocking,
 * fusion or reordering beyond what those definitions state.
 *
 * Units are cgs throughout.  Every function cites the paper passage it
 * follows (section / equation names of "GameDev: GPU-accelerated model for
 * dust evolution").  Where the paper is silent the reading taken is marked
 * "reading:"; the same reading is implemented, independently, on the GPU.
 *
 * Compile with -ffp-contract=off: no fused multiply-adds, so every FP64
 * expression is evaluated exactly as written (left to right).
 */
#ifndef GDO_H
#define GDO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { GDO_PATCH = 0, GDO_DISK = 1 };
enum { GDO_PHYSICAL = 0, GDO_CONSTANT = 1, GDO_LINEAR = 2, GDO_PRODUCT = 3 };
enum { GDO_DIFF_PHYSICAL = 0, GDO_DIFF_RING = 1 };  /* dust diffusion models (Sect. 2.4, 3.2) */
/* resolved dimensions of the collision model (Sect. 2.5.1): 3D; 2D radial-polar
 * (meridional plane); 2D radial-azimuthal, vertically integrated; 1D radial */
enum { GDO_MODEL_3D = 0, GDO_MODEL_RZ = 1, GDO_MODEL_RPHI = 2, GDO_MODEL_R = 3 };
enum { GDO_NFINE = 96, GDO_TMIN = -72 };          /* fine controller bins */
/* optical depth forms of Sect. 2.3.2: from the 3D dust density along rays of r; in the
 * midplane of a vertically integrated model, along R */
enum { GDO_TAU_3D = 0, GDO_TAU_2D = 1 };

/* status bits (sticky) */
enum {
  GDO_ST_EVENT_CAP = 1 << 0,   /* a particle hit max_events in one interval */
  GDO_ST_DT_FLOOR  = 1 << 1,   /* requested interval below dt_coll / 2^60 */
  GDO_ST_NONFINITE = 1 << 2,   /* a rate was NaN or infinite */
  GDO_ST_KNN       = 1 << 3    /* instance holds fewer than K particles */
};

typedef struct {
  int32_t geometry;     /* GDO_PATCH: local periodic patch (x,y periodic), GDO_DISK: global disk */
  int32_t kernel_mode;  /* GDO_PHYSICAL or one of the Appendix A test kernels */
  int32_t K;            /* N_K, neighbours including the particle itself */
  int32_t audit;        /* 1: adaptive safety factor C, 0: C fixed at 1 */
  double r0;            /* reference radius R_0 [cm] (patch: its centre radius) */
  double sigma0;        /* gas surface density at R_0 [g cm^-2] */
  double p;             /* surface-density power-law index */
  double T0;            /* gas temperature at R_0 [K] */
  double q;             /* temperature power-law index */
  double alpha;         /* viscosity parameter */
  double M_star;        /* stellar mass [g] */
  double rho_s;         /* grain internal density rho_o [g cm^-3] */
  double s_min;         /* minimum fragment diameter [cm] */
  double v_frag;        /* fragmentation speed [cm s^-1] */
  double eps;           /* interval tolerance epsilon */
  double dt_coll;       /* collision timestep Delta t_coll [s] */
  double dt_fn_max;     /* maximum frozen-neighbour interval [s] */
  double R_in, R_out;   /* global disk radial edges [cm] */
  double box_x, box_y;  /* patch periodic extents [cm]; positions in [-box/2, box/2) */
  double t0, m0;        /* test-kernel unit time [s] and unit mass [g] */
  uint64_t seed;        /* Philox key */
  int64_t max_events;   /* per particle and interval */
  int32_t diff_mode;    /* GDO_DIFF_PHYSICAL: D = nu/(Sc (1+St^2)) from the gas disk;
                           GDO_DIFF_RING: the ring test, radial only, D = D0 (R/R_0)^2 */
  int32_t diff_chi;     /* 1: concentration diffusion (drift along ln rho_g), 0: density */
  double Sc_R, Sc_Z, Sc_phi;  /* Schmidt numbers of the three directions */
  double D0;            /* ring test: D at R_0 [cm^2 s^-1] */
  int32_t model;        /* GDO_MODEL_*: which dimensions the neighbour search and the
                           sampling measure resolve (RZ and R: global disks only) */
  int32_t pad_model;
  /* radiation forces and the optical depth (Sect. 2.3.2; global disks) */
  double beta0;         /* beta at the reference diameter rad_s0; 0: no radiation forces */
  double kappa0;        /* opacity at rad_s0 for the optical depth [cm^2 g^-1]; 0: tau = 0 */
  double rad_s0;        /* reference diameter s_0 of beta(s) and kappa(s) [cm] */
  double t_beta;        /* taper time scale [s]; <= 0: no taper */
  int32_t rad_pr;       /* 1: Poynting-Robertson drag */
  int32_t tau_geom;     /* GDO_TAU_3D or GDO_TAU_2D */
  int32_t tau_nr, tau_nmu, tau_nphi, pad_tau;  /* grid cells: radial, polar (in cos theta),
                                                  azimuthal; tau_nr = 0: tau = 0 */
  double tau_rmin, tau_rmax;  /* radial extent of the grid [cm] (r in 3D, R in 2D) */
  double tau_mu;        /* 3D grid: cos theta in [-tau_mu, tau_mu] */
} gdo_params;

typedef struct {
  double C;             /* adaptive safety factor, starts at 1 */
  double dt_remain;     /* time left in the current collision timestep (derived from remain_ticks) */
  double dt_exe;        /* executed interval of the last call */
  double dt_req;        /* requested interval of the last call */
  int64_t remain_ticks; /* time left, exactly, in units of dt_coll / 2^60 */
  int64_t interval;     /* Philox interval counter of the next interval */
  int64_t events;       /* events in the last interval */
  int64_t near_draw;    /* near ties of draws against rate / time boundaries */
  int64_t near_dt;      /* near ties of dt_req against a halving boundary */
  int64_t near_audit;   /* near ties of the audit threshold */
  int64_t status;       /* GDO_ST_* bits */
  int32_t n_groups;     /* merged controller bins of the last call */
  int32_t pad;
} gdo_state;

/* Gas and particle-independent quantities at one position (Sect. 2.2, 2.3.1). */
typedef struct {
  double R, Z, r, Om, T, cs, H, h, Sigma, rho_g, eta, Re, gst;
} gdo_gas;

/* Everything the rate model gives for one ordered pair (i, j) (Sect. 2.5.1-2.5.3). */
typedef struct {
  double dvR, dvZ, dvphi, dvB, dvt, dv, Kij, lam;
  double psi, ncoll;
  int32_t outcome;      /* 0 sticking, 1 erosion, 2 fragmentation */
  int32_t pad;
  double c[2];          /* effective channel rates lambda*_ij (second is 0 unless erosion) */
  double J1[2], J2[2];  /* <J> and <J^2> of each channel */
} gdo_pair_t;

/* Optional per-particle outputs of one interval (any pointer may be NULL). */
typedef struct {
  int32_t* nbr;      /* [n*K] neighbour list: slot 0 the particle itself, then ascending index */
  double*  d;        /* [n]   distance to the farthest retained neighbour */
  double*  V;        /* [n]   sampling measure V_i */
  double*  lam;      /* [n]   lambda*_i at the start of the interval */
  double*  mA;       /* [n]   sum_o lambda*_io <J_io> */
  double*  mB;       /* [n]   sum_o lambda*_io <J_io^2> */
  double*  chan;     /* [n*K*2] channel rates lambda*_ij at the start of the interval */
  int32_t* ev_count; /* [n]   events of the interval */
  uint32_t* ev_hash; /* [n]   hash of the chosen (slot, channel) sequence */
  int32_t* near;     /* [n]   near ties met while sampling the particle */
  double*  jsum;     /* [n]   realised sum of |ln(s'/s)| over the interval's events */
  double*  A_b;      /* [GDO_NFINE] A_b of each controller bin of the interval choice
                        (entries past n_groups are 0) */
  double*  B_b;      /* [GDO_NFINE] B_b likewise */
} gdo_outputs;

void   gdo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double gdo_u01(uint32_t a, uint32_t b);
void   gdo_gas_at(const gdo_params* P, double x, double y, double z, gdo_gas* g);
int    gdo_knn_one(const gdo_params* P, int64_t n, const double* x, const double* y,
                   const double* z, int64_t i, int32_t* nbr, double* d);
double gdo_volume(const gdo_params* P, double d, double R);
double gdo_grain_mass(const gdo_params* P, double s);
void   gdo_frag_moments(double s_i, double s_min, double* j1, double* j2);
double gdo_turb_dv2(double St_a, double St_b, double Vg2, double Re);
void   gdo_pair(const gdo_params* P, const gdo_gas* g, double s_i, double m_i,
                double s_j, double m_j, double N_j, double V_i, gdo_pair_t* out);
int    gdo_fine_bin(double s);
void   gdo_choose_interval(const gdo_params* P, int64_t n, const double* s, const double* M,
                           const double* mA, const double* mB, gdo_state* st, int32_t* group_of);
/* The same, also returning A_b and B_b of every controller bin (NULL: not written). */
void   gdo_choose_interval_ab(const gdo_params* P, int64_t n, const double* s, const double* M,
                              const double* mA, const double* mB, gdo_state* st, int32_t* group_of,
                              double* A_b, double* B_b);
void   gdo_audit(const gdo_params* P, int64_t n, const double* M, const double* jsum,
                 const int32_t* group_of_particle, int32_t n_groups, gdo_state* st);
int    gdo_sample_one(const gdo_params* P, const gdo_gas* g, int64_t i, const int32_t* nbr,
                      double V_i, const double* s0, const double* m0, const double* N0,
                      double M_i, double dt_exe, int64_t interval, double* s_io,
                      int32_t* ev_count, uint32_t* ev_hash, int32_t* near, double* jsum,
                      int64_t* status);
int    gdo_interval_step(const gdo_params* P, int64_t n, const double* x, const double* y,
                         const double* z, double* s, const double* M, gdo_state* st,
                         gdo_outputs* out);
int    gdo_rates_subset(const gdo_params* P, int64_t n, const double* x, const double* y,
                        const double* z, const double* s, const double* M, int64_t nq,
                        const int64_t* q, const int32_t* nbr, const double* d,
                        double* lam, double* mA, double* mB, double* chan);
int    gdo_sample_subset(const gdo_params* P, int64_t n, const double* x, const double* y,
                         const double* z, const double* s0, const double* M, int64_t nq,
                         const int64_t* q, const int32_t* nbr, const double* d, double dt_exe,
                         int64_t interval, double* s_q, int32_t* ev_count, uint32_t* ev_hash,
                         int32_t* near, double* jsum, int64_t* status);
void   gdo_push_one(const gdo_params* P, int32_t drag, double dt, double* x, double* y,
                    double* z, double* vr, double* lth, double* lph, double s);
void   gdo_push(const gdo_params* P, int32_t drag, double dt, int64_t n, double* x, double* y,
                double* z, double* vr, double* lth, double* lph, const double* s);
/* ---- Radiation forces and the optical depth, Sect. 2.3.2 ------------------------ */
int64_t gdo_params_size(void);
double gdo_rad_beta(const gdo_params* P, double s);
double gdo_rad_kappa(const gdo_params* P, double s);
double gdo_rad_taper(const gdo_params* P, double t);
int64_t gdo_tau_size(const gdo_params* P);
void   gdo_tau_grid(const gdo_params* P, int64_t n, const double* x, const double* y,
                    const double* z, const double* s, const double* M, double* T);
double gdo_tau_at(const gdo_params* P, const double* T, double x, double y, double z);
void   gdo_push_rad(const gdo_params* P, int32_t drag, double dt, double t, int64_t n, double* x,
                    double* y, double* z, double* vr, double* lth, double* lph, const double* s,
                    const double* M, double* T, double* mid);
/* ---- Spatial groups, Sect. 2.5.3 ------------------------------------------------
 * Reading: an instance is split into G spatial groups of equal width, radial annuli
 * of a disk in R (R_in .. R_out) or slabs of a patch in x; each group has its own
 * controller bins, safety factor C, interval level k (dt_coll 2^-k), clock and Philox
 * interval counter.  Groups interact when a particle of one has a particle of the
 * other in its neighbour list.  A round takes the groups whose scheduled interval ends
 * earliest: they broadcast their particles' sizes into the partner snapshot, request a
 * level, are scheduled (the ratio-16 rule, delayed refinements) and sample their new
 * interval.  The step ends once every group reached dt_coll. */
enum { GDO_MAXG = 64 };
typedef struct {
  int32_t n_groups;           /* G (1 .. GDO_MAXG) */
  int32_t pad;
  int64_t t;                  /* clock of the last round, ticks of dt_coll / 2^60 */
  int64_t rounds;             /* rounds so far */
  int64_t delayed;            /* requests held coarser by a scheduled interval (ratio 16) */
  int64_t breaks;             /* interacting pairs left more than 16 apart (the step's end won) */
  int32_t level[GDO_MAXG];    /* level of the group's scheduled (or last) interval; -1: none yet */
  int32_t k_req[GDO_MAXG];    /* level the group requested in its last round */
  int32_t active[GDO_MAXG];   /* 1: the group took part in the last round */
  int32_t pad2;
  int64_t members[GDO_MAXG];  /* particles of the group */
  int64_t intervals[GDO_MAXG];/* intervals the group executed */
  uint64_t inter[GDO_MAXG];   /* bit h of inter[g]: groups g and h interact (symmetric) */
  gdo_state st[GDO_MAXG];     /* per-group interval state (C, clock via remain_ticks, ...) */
} gdo_groups;

int32_t gdo_group_of(const gdo_params* P, int32_t G, double x, double y);
/* A fresh set of G groups (C = 1, no step begun). */
void   gdo_groups_reset(const gdo_params* P, int32_t G, gdo_groups* S);
/* Group of every particle, members and interaction masks from the neighbour lists. */
void   gdo_groups_assign(const gdo_params* P, int64_t n, const double* x, const double* y,
                         const int32_t* nbr, int32_t* group_of, gdo_groups* S);
/* Levels of the active groups from their requests (see gdo.c). */
void   gdo_schedule(int32_t G, const uint64_t* inter, const int64_t* members,
                    const int32_t* active, const int32_t* k_req, const int32_t* k_fit,
                    int32_t* level, int64_t* delayed, int64_t* breaks);
/* One round (lists, V and gas of every particle given; s live sizes, s0 the partner
 * snapshot, both updated).  Returns 1 if the round started a new collision step. */
int    gdo_group_round(const gdo_params* P, int64_t n, const int32_t* nbr, const double* V,
                       const gdo_gas* gas, double* s, double* s0, const double* M,
                       const int32_t* group_of, gdo_groups* S, gdo_outputs* out);
/* A whole collision step: lists once, then rounds until every group reached dt_coll. */
int    gdo_collide_groups(const gdo_params* P, int64_t n, const double* x, const double* y,
                          const double* z, double* s, const double* M, gdo_groups* S,
                          int32_t max_rounds);

/* The common transport timestep of Sect. 2.6 (reading; see gdo_local_dt). */
typedef struct {
  double dt_max;        /* prescribed maximum timestep Delta t_max [s] */
  double dt_out;        /* time left before the next output Delta t_out [s] */
  double f_orb;         /* orbital limit: Delta t_i <= f_orb * 2 pi / Omega_K(R_i); <= 0: off */
  double dx_H;          /* local grid spacing Delta x_i = dx_H * H_g(R_i) */
  double c_adv;         /* deterministic displacement |u_i| dt <= c_adv Delta x_i; <= 0: off */
  double c_diff;        /* diffusive displacement sqrt(2 D_i dt) <= c_diff Delta x_i; <= 0: off */
} gdo_dt_rule;

void   gdo_diff_coeffs(const gdo_params* P, double R, double Z, double s, double out[7]);
void   gdo_diffuse(const gdo_params* P, double dt, int64_t step, int64_t n, double* x, double* y,
                   double* z, double* vr, double* lth, double* lph, const double* s);
double gdo_local_dt(const gdo_params* P, const gdo_dt_rule* rule, double x, double y, double z,
                    double s, const double* v);
double gdo_timestep(const gdo_params* P, const gdo_dt_rule* rule, int64_t n, const double* x,
                    const double* y, const double* z, const double* s, const double* vr,
                    const double* lth, const double* lph, double* dti);

#ifdef __cplusplus
}
#endif
#endif
