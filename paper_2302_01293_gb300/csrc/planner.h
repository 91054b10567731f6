// Host planner interface (see planner.cpp).
#pragma once

#include <cstdint>
#include <functional>
#include <vector>

#include "../../include/qlp_bls.h"

namespace qlp {

struct StarPlanHost {
  int32_t status = 0;
  int64_t n_valid = 0;
  double t_ref = 0.0;
  double baseline = 0.0;
  double pmin = 0.0;
  double pmax = 0.0;
  double rho_kg = 0.0;
  std::vector<double> tp, y, dy;   // valid points, t' = t - t_ref (unless ext_tp is set)
  // the valid points in a caller's arrays instead (batch planner with staging arrays)
  const double* ext_tp = nullptr;
  const double* ext_y = nullptr;
  const double* ext_dy = nullptr;
  const double* tp_data() const { return ext_tp ? ext_tp : tp.data(); }
  const double* y_data() const { return ext_tp ? ext_y : y.data(); }
  const double* dy_data() const { return ext_tp ? ext_dy : dy.data(); }
  std::vector<double> freqs;       // trial frequencies (1/day)
  std::vector<double> qmins;       // q_min at each frequency
  std::vector<int32_t> nbins;      // nbins at each frequency
  int32_t nbins_max = 0;
  int32_t nbins_min = 0;
  double nbins_sum = 0.0;          // sum of nbins over the grid
  // spread of the normalised weights w = dy^-2 / sum dy^-2 and of w (y - ybar):
  // the largest over the mean (the exact path's integer scale follows the largest)
  double w_spread = 0.0;
  double wd_spread = 0.0;
  // largest |w (y - ybar)| of a point and largest |sum over the points before t of
  // w (y - ybar)| over t (normalised weights): the 32-bit exact tables need the
  // second to stay within a small multiple of the first
  double wd_max = 0.0;
  double y_exc = 0.0;
  double ymax = 0.0;               // max over f of T f nbins(f)
  int32_t sturges_nb = 0;
  // cell path: cells of width h (just below the smallest point spacing) hold at
  // most one point each; cells_ok when that holds for the FP64 cell assignment
  bool cells_ok = false;
  double cell_h = 0.0;
  int64_t n_cells = 0;
  double cells_work = 0.0;         // sum over f of the bin edges across the baseline
  double bin_dmax = 0.0;           // longest bin duration 1/(f nbins) over the grid (days)
  int32_t grid_k0 = -1;            // coarse grid: bin index of the first (lowest) frequency
  bool head_ok = false;            // valid, sorted points and Pmin < Pmax: the star gets a grid
  bool points_done = false;        // the point analysis (weight spreads, cells) has run
};

// The part of a star's plan that depends on its points only (validity, t_ref,
// baseline, Pmin and Pmax, weight spreads, cells), kept by a plan so that a plan of
// the same stars on other frequencies need not scan the points again.
struct StarPoints {
  int32_t status = 0;              // the head's status when head_ok is false
  bool head_ok = false;
  int64_t n_valid = 0;
  double t_ref = 0.0, baseline = 0.0, pmin = 0.0, pmax = 0.0, rho_kg = 0.0;
  double w_spread = 0.0, wd_spread = 0.0, wd_max = 0.0, y_exc = 0.0;
  bool cells_ok = false;
  double cell_h = 0.0;
  int64_t n_cells = 0;
};

// Arrays that receive a star's valid points (t', y, dy), at least as long as its
// raw point count; entries past the valid count are set to zero.
struct PointDst {
  double* tp = nullptr;
  double* y = nullptr;
  double* dy = nullptr;
};

// Frequency windows [lo, hi] of one star (1/day) that restrict its grid.
struct Windows {
  const double* lo = nullptr;
  const double* hi = nullptr;
  int64_t n = 0;
};

int64_t cell_of(double tp, double h);

int n_q_of(const qlp_bls_params& p);
double q_min_of(double f, double rho_kg, const qlp_bls_params& p);
int nbins_of(double qmin, const qlp_bls_params& p);
double pmin_of(double rho_kg, const qlp_bls_params& p);
double pmax_of(const double* tp, int64_t n, const qlp_bls_params& p);
int sturges_of(int64_t n);
void plan_one(const qlp_bls_params& p, const double* t, const double* y, const double* dy, int64_t n,
              double rho, StarPlanHost* out, const Windows* win = nullptr, const PointDst* dst = nullptr);
// Runs fn(s) for every star s on the planner's threads (p.n_threads, 0 = all cores).
void parallel_stars(const qlp_bls_params& p, int32_t n_stars, const std::function<void(int32_t)>& fn);

// The point analysis of a planned star (running it first if its grid came out
// empty or over the cap, which skips it); the star's point arrays must still exist.
StarPoints points_of(StarPlanHost& s);
// The plans of stars whose point analysis is known, on the grids of p (windows as
// in plan_all); the same grids and bins as plan_all on the stars' points.
void plan_all_from(const qlp_bls_params& p, int32_t n_stars, const StarPoints* pts,
                   std::vector<StarPlanHost>* out, const int64_t* win_off = nullptr,
                   const double* win_lo = nullptr, const double* win_hi = nullptr);

void plan_all(const qlp_bls_params& p, int32_t n_stars, const int64_t* offsets, const double* t,
              const double* y, const double* dy, const double* rho, std::vector<StarPlanHost>* out,
              const int64_t* win_off = nullptr, const double* win_lo = nullptr,
              const double* win_hi = nullptr, const PointDst* dst = nullptr);

}  // namespace qlp
