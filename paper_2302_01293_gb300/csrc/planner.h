// Host planner interface (see planner.cpp).
#pragma once

#include <cstdint>
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
  std::vector<double> tp, y, dy;   // valid points, t' = t - t_ref
  std::vector<double> freqs;       // trial frequencies (1/day)
  std::vector<double> qmins;       // q_min at each frequency
  int32_t nbins_max = 0;
  double ymax = 0.0;               // max over f of T f nbins(f)
  int32_t sturges_nb = 0;
};

int n_q_of(const qlp_bls_params& p);
double q_min_of(double f, double rho_kg, const qlp_bls_params& p);
int nbins_of(double qmin, const qlp_bls_params& p);
double pmin_of(double rho_kg, const qlp_bls_params& p);
double pmax_of(const double* tp, int64_t n, const qlp_bls_params& p);
int sturges_of(int64_t n);
void plan_one(const qlp_bls_params& p, const double* t, const double* y, const double* dy, int64_t n,
              double rho, StarPlanHost* out);
void plan_all(const qlp_bls_params& p, int32_t n_stars, const int64_t* offsets, const double* t,
              const double* y, const double* dy, const double* rho, std::vector<StarPlanHost>* out);

}  // namespace qlp
