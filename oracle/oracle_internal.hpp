// Internal declarations shared by the oracle's translation units.
// Test infrastructure only (see oracle_api.h).
#pragma once
#include <cstdint>
#include <vector>

#include "oracle_api.h"
#include "physics.hpp"

namespace oracle {

struct Parton {
  Vec4 p;
  int flav;  // PDG: +-1..5 quarks, 21 gluon
  int col;   // colour line index (0 = none)
  int acol;  // anticolour line index (0 = none)
};

struct Event {
  std::vector<Parton> partons;
  double weight = 0.0;
  int me_flavour = 0;
  double t = 0.0;
  double t_first = 0.0;
  int status = 0;
  int n_steps = 0;
  int n_emissions = 0;
  int n_winners = 0;
  int64_t n_trials = 0;
  int n_dipoles = 0;
  uint64_t hash = 0;
  int next_colour = 0;
};

// Stage 1: the LO matrix element (App. B).
void generate_me(const oracle_params& p, uint32_t event_id, Event& ev);
// Stage 2: the serial veto-algorithm shower (Sec. 2, App. A, App. C).
void shower(const oracle_params& p, uint32_t event_id, Event& ev);
// Stage 3: observables (Sec. 3.1).
void durham(const std::vector<Vec4>& moms, double s, int mutation, double y_out[4]);
double thrust(const std::vector<Vec4>& moms, int mutation, Vec4* axis);
void event_shapes(const std::vector<Vec4>& moms, double s, int mutation, double out[8]);
// Per-event validation bits (momentum, on-shell, colour, flavour).
int validate(const std::vector<Parton>& partons, double sqrt_s);

// Histogram binning shared by the oracle's own runner.
constexpr int kNObs = ORACLE_N_OBS;
constexpr int kNBins = ORACLE_N_BINS;
constexpr int kRow = ORACLE_HIST_ROW;
void histogram_fill(double* hist, const double obs[8], double w);

}  // namespace oracle
