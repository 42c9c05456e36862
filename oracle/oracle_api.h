/* Oracle C interface (test infrastructure only).
 *
 * The oracle is a plain, serial, FP64 CPU implementation of the paper's
 * event generator: LO e+e- -> q qbar matrix element (App. B), the Sudakov veto
 * algorithm with competing emissions (Sec. 2, App. A, App. C), a massless
 * final-state dipole shower, and the Durham / thrust / heavy-jet-mass
 * observables (Sec. 3.1).  It exists to check the CUDA path: only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It shares
 * no code with the CUDA library; the only thing both sides agree on is the
 * published Philox4x32-10 definition and the draw-index scheme.
 *
 * Momentum arrays are (E, px, py, pz) per parton, in GeV, row-major.
 * Every function returns 0 on success and a negative value on bad arguments.
 */
#ifndef GAPS_ORACLE_API_H
#define GAPS_ORACLE_API_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_params {
  double sqrt_s;         /* centre-of-mass energy, GeV */
  double alphas_mz;      /* alpha_s(m_Z) */
  double t_cutoff;       /* shower cutoff t_C, GeV^2 */
  uint64_t seed;         /* Philox key */
  int32_t n_flavours;    /* active quark flavours, 1..5 */
  int32_t fixed_alphas;  /* 1: alpha_s(t) = alpha_s^over = alpha_s(m_Z) (test mode) */
  int32_t capacity;      /* partons per event before the overflow flag, 2..1024 */
  int32_t max_steps;     /* veto cycles per event before the step-limit flag */
  int32_t max_emissions; /* stop after this many accepted emissions (0 = no limit; tests) */
  int32_t mutation;      /* planted mistakes for pin-sensitivity tests (0 = none) */
  int32_t trial_mode;    /* 0: one trial per (dipole, kernel) (App. A listing); 1: one trial per
                            dipole with the kernels' summed overestimate, the kernel drawn in
                            proportion to its share: the same distribution, since the first of
                            independent exponential trials is one trial with the summed rate whose
                            kind has probability rate / sum (App. A generates one per kind) */
} oracle_params;

typedef struct oracle_event_out {
  double weight;     /* ME weight, pb */
  double t_first;    /* scale of the first accepted emission (0 if none) */
  double t_final;    /* last winner scale (t_C if the event ended at the cutoff) */
  uint64_t hash;     /* FNV-1a over the per-step decision words */
  int64_t n_trials;  /* trial emissions generated */
  int32_t me_flavour;
  int32_t n_partons;
  int32_t status;    /* 1 done, 2 overflow, 3 step limit */
  int32_t n_steps;   /* veto cycles, including the final one that found no winner */
  int32_t n_emissions;
  int32_t n_winners; /* cycles with a trial above t_C */
  int32_t valid;     /* validation error bits (0 = valid) */
  int32_t n_dipoles; /* dipoles evaluated (colour-connected, Q^2 >= 4 t_C), summed over cycles */
} oracle_event_out;

/* Status codes of an event. */
enum { ORACLE_DONE = 1, ORACLE_OVERFLOW = 2, ORACLE_STEP_LIMIT = 3 };

/* Planted mistakes (tests only). */
enum {
  ORACLE_MUT_NO_JACOBIAN = 1 << 0,   /* drop (1-y) in the veto ratio */
  ORACLE_MUT_Z_UNIFORM = 1 << 1,     /* z uniform instead of inverting I^over */
  ORACLE_MUT_NO_RECOIL = 1 << 2,     /* spectator keeps its momentum */
  ORACLE_MUT_COLOUR_SWAP = 1 << 3,   /* new gluon's colour lines swapped */
  ORACLE_MUT_ALPHAS_OVER = 1 << 4,   /* alpha_s^over = alpha_s(m_Z) with running coupling */
  ORACLE_MUT_ME_NO_INTERF = 1 << 5,  /* drop the gamma-Z interference terms */
  ORACLE_MUT_DURHAM_MAX = 1 << 6,    /* max(E_i^2, E_j^2) in the Durham measure */
  ORACLE_MUT_THRUST_NOSIGNS = 1 << 7,/* only P + p_j + p_k in the thrust search */
  ORACLE_MUT_KT_SIGN = 1 << 8,       /* +k_perp on both daughters */
  ORACLE_MUT_Z_SWAP = 1 << 9,        /* daughters' momentum fractions exchanged */
  ORACLE_MUT_HJM_LIGHT = 1 << 10,    /* lighter hemisphere mass */
  ORACLE_MUT_TRIAL_RESTART = 1 << 11,/* a vetoed trial restarts from the old scale */
  ORACLE_MUT_KERNEL_UNIFORM = 1 << 12,/* per-dipole trials: kernel drawn uniformly, not by its share */
  ORACLE_MUT_BROAD_DOT = 1 << 13,    /* broadening from |p . n_T| instead of |p x n_T| */
  ORACLE_MUT_NF_MINUS_ONE = 1 << 14, /* a gluon gets g -> q qbar kernels for flavours 1..n_f-1 only */
  ORACLE_MUT_PAIR_UNIFORM = 1 << 15, /* both kernels of a trial slot take the slot's first uniform */
  ORACLE_MUT_GG_FULL = 1 << 16       /* g -> gg without the half weight of a gluon's two dipoles */
};

/* Histogram layout: 6 observables x (100 bins + underflow + overflow) x
 * (sum w, sum w^2, entries). */
enum { ORACLE_N_OBS = 8, ORACLE_N_BINS = 100, ORACLE_HIST_ROW = 102 };

int oracle_check_params(const oracle_params* p);

/* Generate, shower and analyse events first_event .. first_event+n_events-1.
 * Outputs may be NULL.  mom: [n_events][capacity][4]; info: [n_events][capacity][3]
 * (flavour, colour, anticolour); obs: [n_events][8] (y23, y34, y45, y56, 1-T,
 * rho_H, B_T, B_W; -1 where undefined); hist: [8][102][3], accumulated over the events
 * that ended at the cutoff.  n_threads <= 1 runs serially. */
int oracle_run(const oracle_params* p, uint32_t first_event, int64_t n_events, int n_threads,
               oracle_event_out* out, double* mom, int32_t* info, double* obs, double* hist);

/* The shower of oracle_run started from a given parton state instead of the
 * matrix element (tests: pins of the shower from states with gluons).
 * n_init partons (2 <= n_init <= capacity), mom [n_init][4] (E, px, py, pz),
 * info [n_init][3] (flavour, colour, anticolour; colour lines numbered
 * below 1000).  Every event first_event + j starts from this state at
 * t0 = s with weight 1, next colour line = the largest line + 1, and runs
 * with p's settings (max_emissions applies).  Outputs as oracle_run (may be
 * NULL): out, mom_out [n_events][capacity][4], info_out
 * [n_events][capacity][3]. */
int oracle_run_from_state(const oracle_params* p, int n_init, const double* mom, const int32_t* info,
                          uint32_t first_event, int64_t n_events, int n_threads, oracle_event_out* out,
                          double* mom_out, int32_t* info_out);

/* Building blocks, exported so the tests can pin each one on its own. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void oracle_uniform_pair(uint64_t seed, uint32_t event, uint32_t step, uint32_t slot,
                         uint32_t purpose, double out[2]);
double oracle_dsigma_dcos(const oracle_params* p, int flavour, double cos_theta);
double oracle_alphas(const oracle_params* p, double t);
double oracle_alphas_over(const oracle_params* p);
/* kind: 0 = q->qg, 1 = g->gg, 2 = g->qqbar (one flavour) */
double oracle_kernel_value(int kind, double z, double y);
double oracle_kernel_estimate(int kind, double z);
double oracle_kernel_integral(int kind, double zm, double zp);
double oracle_kernel_generate_z(int kind, double zm, double zp, double u, int mutation);
int oracle_splitting_map(const double pij[4], const double pk[4], double z, double y, double phi,
                         int mutation, double pi_out[4], double pj_out[4], double pk_out[4]);
int oracle_durham(int n, const double* mom, double s, int mutation, double y_out[4]);
int oracle_thrust(int n, const double* mom, int mutation, double out[4]);
int oracle_event_shapes(int n, const double* mom, double s, int mutation, double out[8]);
int oracle_validate(int n, const double* mom, const int32_t* info, double sqrt_s);

#ifdef __cplusplus
}
#endif
#endif
