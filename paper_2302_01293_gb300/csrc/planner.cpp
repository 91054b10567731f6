// Host planner (Sec. 2.1 of arXiv:2302.01293): per-star validation, period
// limits, Keplerian duration range and trial-frequency grid, in FP64.
// Compiled with -ffp-contract=off: every product and sum is rounded on its own,
// so the grid is reproducible bit for bit from its definition.
//
//  * rho: the TIC density, or the solar density rho_default when it is missing;
//  * Pmin: the period where a = pmin_aR R*, from Kepler's third law with
//    M = 4/3 pi R*^3 rho (R* cancels): Pmin = sqrt(3 pi (a/R*)^3 / (G rho));
//  * Pmax: the longest continuous stretch of data (stretches split at gaps
//    longer than gap_days = one TESS sector), or half of it when there is a
//    single stretch;
//  * q_circ(f) = asin(min(1, R*/a)) / pi, a/R* = (G rho P^2 / (3 pi))^(1/3): the
//    duration fraction of a central circular orbit; searched durations
//    [qmin_fac, qmax_fac] x q_circ;
//  * grid: f_0 = 1/Pmax, f_{k+1} = f_k + q_min(f_k) / (samples_per_peak T),
//    T = t_max - t_min, while f <= 1/Pmin;
//  * bins: nbins(f) = ceil(noverlap / q_min(f)).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <exception>
#include <mutex>
#include <pthread.h>
#include <thread>
#include <utility>
#include <vector>

#include "planner.h"

namespace qlp {

namespace {
constexpr double kG = 6.67430e-11;  // m^3 kg^-1 s^-2
constexpr double kDay = 86400.0;
constexpr double kPi = 3.141592653589793;
}  // namespace

int n_q_of(const qlp_bls_params& p) {
  return (int)std::floor(std::log(p.qmax_fac / p.qmin_fac) / p.dlogq + 1e-9) + 1;
}

double q_min_of(double f, double rho_kg, const qlp_bls_params& p) {
  const double ps = kDay / f;
  const double x = kG * rho_kg * ps * ps / (3.0 * kPi);
  const double a_r = std::cbrt(x);
  const double q_circ = std::asin(std::min(1.0, 1.0 / a_r)) / kPi;
  return p.qmin_fac * q_circ;
}

int nbins_of(double qmin, const qlp_bls_params& p) { return (int)std::ceil(p.noverlap / qmin); }

double pmin_of(double rho_kg, const qlp_bls_params& p) {
  const double a3 = p.pmin_aR * p.pmin_aR * p.pmin_aR;
  return std::sqrt(3.0 * kPi * a3 / (kG * rho_kg)) / kDay;
}

double pmax_of(const double* tp, int64_t n, const qlp_bls_params& p) {
  int64_t start = 0;
  int stretches = 1;
  double longest = 0.0;
  for (int64_t i = 1; i < n; ++i) {
    if (tp[i] - tp[i - 1] > p.gap_days) {
      longest = std::max(longest, tp[i - 1] - tp[start]);
      start = i;
      ++stretches;
    }
  }
  longest = std::max(longest, tp[n - 1] - tp[start]);
  if (stretches == 1) return (tp[n - 1] - tp[0]) / 2.0;
  return longest;
}

// Cell of a point: u = floor(t'/h), adjusted so that t' - u h (FP64) lies in [0, h).
int64_t cell_of(double tp, double h) {
  double q = std::floor(tp / h);
  const double r = tp - q * h;
  if (r < 0.0) q -= 1.0;
  else if (r >= h) q += 1.0;
  return (int64_t)q;
}

int sturges_of(int64_t n) { return (int)std::floor(1.0 + 3.322 * std::log10((double)n) + 0.5); }

namespace {

// Validation, t' = t - t_min, Pmin and Pmax. False when the star gets no grid
// (its status says why).
bool plan_head(const qlp_bls_params& p, const double* t, const double* y, const double* dy, int64_t n,
               double rho, StarPlanHost& s, const PointDst* dst) {
  s = StarPlanHost();
  const double rho_gcc = (std::isfinite(rho) && rho > 0.0) ? rho : p.rho_default;
  s.rho_kg = rho_gcc * 1000.0;
  // valid points (finite, dy > 0), checked for non-decreasing t as they are kept
  int64_t i0 = 0;
  while (i0 < n && !(std::isfinite(t[i0]) && std::isfinite(y[i0]) && std::isfinite(dy[i0]) && dy[i0] > 0.0)) ++i0;
  double *otp, *oy, *ody;
  if (dst) {
    otp = dst->tp;
    oy = dst->y;
    ody = dst->dy;
    s.ext_tp = otp;
    s.ext_y = oy;
    s.ext_dy = ody;
  } else {
    s.tp.resize((size_t)(n - i0));
    s.y.resize((size_t)(n - i0));
    s.dy.resize((size_t)(n - i0));
    otp = s.tp.data();
    oy = s.y.data();
    ody = s.dy.data();
  }
  const double t_ref = i0 < n ? t[i0] : 0.0;
  int64_t m = 0;
  bool sorted = true;
  double t_prev = t_ref;
  for (int64_t i = i0; i < n; ++i) {
    if (std::isfinite(t[i]) && std::isfinite(y[i]) && std::isfinite(dy[i]) && dy[i] > 0.0) {
      sorted = sorted && !(t[i] < t_prev);
      t_prev = t[i];
      otp[m] = t[i] - t_ref;
      oy[m] = y[i];
      ody[m] = dy[i];
      ++m;
    }
  }
  if (dst) {
    for (int64_t i = m; i < n; ++i) otp[i] = oy[i] = ody[i] = 0.0;
  } else {
    s.tp.resize((size_t)m);
    s.y.resize((size_t)m);
    s.dy.resize((size_t)m);
  }
  if (m < 2) { s.status = QLP_STAR_TOO_FEW; s.n_valid = m; return false; }
  if (!sorted) { s.status = QLP_STAR_UNSORTED; s.n_valid = m; return false; }
  s.n_valid = m;
  s.t_ref = t_ref;
  s.baseline = otp[m - 1];
  s.pmin = pmin_of(s.rho_kg, p);
  s.pmax = pmax_of(otp, m, p);
  if (!(s.baseline > 0.0) || !(s.pmin < s.pmax)) { s.status = QLP_STAR_EMPTY_GRID; return false; }
  s.head_ok = true;
  return true;
}

// The coarse grid's periods, coarse_pmin (coarse_pmax / coarse_pmin)^(k / (bins - 1))
// for k = 0 .. bins - 1: the same for every star, so a batch computes them once.
std::vector<double> coarse_period_table(const qlp_bls_params& p) {
  std::vector<double> per((size_t)std::max(p.coarse_bins, 0));
  const double ratio = p.coarse_pmax / p.coarse_pmin;
  for (int k = 0; k < p.coarse_bins; ++k)
    per[(size_t)k] = p.coarse_pmin * std::pow(ratio, (double)k / (double)(p.coarse_bins - 1));
  return per;
}

// The frequencies and q_min of one star: the coarse log-period grid (its periods
// from coarse_per when given), the spacing rule inside windows, or the spacing rule
// over [1/Pmax, 1/Pmin].
void grid_one(const qlp_bls_params& p, StarPlanHost& s, const Windows* win, const double* coarse_per = nullptr) {
  auto add = [&](double f) {  // returns q_min(f)
    const double q = q_min_of(f, s.rho_kg, p);
    s.freqs.push_back(f);
    s.qmins.push_back(q);
    return q;
  };
  if (p.grid_mode == 1) {
    // coarse log-period grid, increasing frequency = decreasing bin index
    const double ratio = p.coarse_pmax / p.coarse_pmin;
    for (int k = p.coarse_bins - 1; k >= 0; --k) {
      const double per = coarse_per ? coarse_per[k]
                                    : p.coarse_pmin * std::pow(ratio, (double)k / (double)(p.coarse_bins - 1));
      if (per < s.pmin || per > s.pmax) continue;
      if (s.grid_k0 < 0) s.grid_k0 = k;
      add(1.0 / per);
    }
  } else if (win) {
    // windows: the spacing rule walked from each merged window's low edge,
    // clipped to [1/Pmax, 1/Pmin]
    std::vector<std::pair<double, double>> w;
    for (int64_t i = 0; i < win->n; ++i)
      if (win->lo[i] <= win->hi[i]) w.emplace_back(win->lo[i], win->hi[i]);
    std::sort(w.begin(), w.end());
    std::vector<std::pair<double, double>> merged;
    for (const auto& iv : w) {
      if (!merged.empty() && iv.first <= merged.back().second)
        merged.back().second = std::max(merged.back().second, iv.second);
      else
        merged.push_back(iv);
    }
    const double fmin = 1.0 / s.pmax, fmax = 1.0 / s.pmin;
    const double denom = p.samples_per_peak * s.baseline;
    for (const auto& iv : merged) {
      double f = std::max(iv.first, fmin);
      const double end = std::min(iv.second, fmax);
      while (f <= end) f = f + add(f) / denom;
    }
  } else {
    const double fmax = 1.0 / s.pmin;
    const double denom = p.samples_per_peak * s.baseline;
    double f = 1.0 / s.pmax;
    while (f <= fmax) f = f + add(f) / denom;
  }
}

// The plain grids of up to kChains stars at once. Each star's recurrence is a
// chain of dependent steps (a cube root, an arcsine and four divisions each), so
// one chain leaves the core mostly waiting; stepping several independent chains
// in one loop lets it overlap them. Every chain performs exactly the operations
// of the one-star loop above, so the grids are the same bit for bit.
constexpr int kChains = 8;
void grid_chains(const qlp_bls_params& p, StarPlanHost* const* st, int n) {
  double f[kChains], fmax[kChains], denom[kChains];
  bool on[kChains];
  int left = 0;
  for (int j = 0; j < kChains; ++j) {
    on[j] = false;
    if (j >= n) continue;
    fmax[j] = 1.0 / st[j]->pmin;
    denom[j] = p.samples_per_peak * st[j]->baseline;
    f[j] = 1.0 / st[j]->pmax;
    on[j] = f[j] <= fmax[j];
    left += on[j] ? 1 : 0;
    if (on[j]) {
      // room for the grid at once: with q_min about proportional to f^(2/3) the steps
      // number denom (3 / q(f0)) f0^(2/3) (fmax^(1/3) - f0^(1/3)); the arcsine makes
      // q_min grow faster near Pmin, so this overestimates a little (only the vectors'
      // capacity depends on it)
      const double q0 = q_min_of(f[j], st[j]->rho_kg, p);
      const double est = denom[j] * 3.0 / q0 * std::cbrt(f[j] * f[j]) * (std::cbrt(fmax[j]) - std::cbrt(f[j]));
      if (est > 0.0 && est < 1.0e8) {
        st[j]->freqs.reserve((size_t)(est * 1.02) + 64);
        st[j]->qmins.reserve((size_t)(est * 1.02) + 64);
      }
    }
  }
  while (left > 0) {
    for (int j = 0; j < kChains; ++j) {
      if (!on[j]) continue;
      StarPlanHost& s = *st[j];
      const double q = q_min_of(f[j], s.rho_kg, p);
      s.freqs.push_back(f[j]);
      s.qmins.push_back(q);
      f[j] = f[j] + q / denom[j];
      if (!(f[j] <= fmax[j])) {
        on[j] = false;
        --left;
      }
    }
  }
}

// Bins and the grid's sums, the nbins cap and Sturges' bin count; the bin edges
// across the baseline and the longest bin duration into *edges_out, *dmax_out.
// False when the grid is empty or over the cap (the status says which).
bool tail_grid(const qlp_bls_params& p, StarPlanHost& s, double* edges_out, double* dmax_out) {
  double edges = 0.0, dmax = 0.0, fnb_min = 0.0;
  const size_t nf = s.freqs.size();
  s.nbins.resize(nf);
  for (size_t k = 0; k < nf; ++k) {
    const double f = s.freqs[k];
    const int nb = nbins_of(s.qmins[k], p);
    s.nbins[k] = nb;
    s.nbins_max = std::max(s.nbins_max, nb);
    s.nbins_min = k == 0 ? nb : std::min(s.nbins_min, nb);
    s.nbins_sum += (double)nb;
    const double y = s.baseline * f * (double)nb;
    s.ymax = std::max(s.ymax, y);
    edges += std::floor(y) + 3.0;
    fnb_min = k == 0 ? f * (double)nb : std::min(fnb_min, f * (double)nb);
  }
  // longest bin duration: max of 1 / (f nbins) = 1 / min(f nbins) (division is monotonic)
  if (nf > 0) dmax = 1.0 / fnb_min;
  if (s.freqs.empty()) { s.status = QLP_STAR_EMPTY_GRID; return false; }
  if (s.nbins_max > p.nbins_cap) {
    s.status = QLP_STAR_NBINS_CAP;
    s.freqs.clear();
    s.qmins.clear();
    s.nbins.clear();
    return false;
  }
  s.sturges_nb = sturges_of((int64_t)s.freqs.size());
  *edges_out = edges;
  *dmax_out = dmax;
  return true;
}

// The weight spreads and the cell width of a star (its points only).
void tail_points(StarPlanHost& s) {
  const int64_t m = s.n_valid;
  const double* tp = s.tp_data();
  const double* yv = s.y_data();
  const double* dyv = s.dy_data();
  // weight spreads and the running sum of w (y - ybar) (FP64; only routing decisions
  // depend on them, so the sums are plain and the weights are not normalised): each
  // point's 1 / dy^2 once, kept in this thread's scratch for the second pass
  {
    thread_local std::vector<double> inv_s;
    if (inv_s.size() < (size_t)m) inv_s.resize((size_t)m);
    double* inv = inv_s.data();
    double isum = 0.0, iysum = 0.0, imax = 0.0;
    for (int64_t i = 0; i < m; ++i) {
      const double v = 1.0 / (dyv[i] * dyv[i]);
      inv[i] = v;
      isum += v;
      iysum += v * yv[i];
      imax = std::max(imax, v);
    }
    const double ybar = iysum / isum;
    // the running sum of w (y - ybar) and its largest magnitude (it ends near zero).
    // The device's weighted mean differs from this one by the FP64 sums' rounding,
    // below 2^-37 max|y| for 2^16 points, which moves every running sum by as much:
    // an excursion below 2^-28 max|y| is reported as 0 (no 32-bit table)
    double dsum = 0.0, dmax = 0.0, run = 0.0, exc = 0.0, yabs = 0.0;
    for (int64_t i = 0; i < m; ++i) {
      const double d = (yv[i] - ybar) * inv[i];
      dsum += std::fabs(d);
      dmax = std::max(dmax, std::fabs(d));
      run += d;
      exc = std::max(exc, std::fabs(run));
      yabs = std::max(yabs, std::fabs(yv[i]));
    }
    s.w_spread = imax / (isum / (double)m);
    s.wd_spread = dsum > 0.0 ? dmax / (dsum / (double)m) : 0.0;
    s.wd_max = dmax / isum;
    s.y_exc = (exc / isum >= std::ldexp(yabs, -28)) ? exc / isum : 0.0;
  }

  // cell path: smallest spacing, cells just narrower, one point per cell
  double min_gap = INFINITY;
  for (int64_t i = 1; i < m; ++i) min_gap = std::min(min_gap, tp[i] - tp[i - 1]);
  if (min_gap > 0.0 && std::isfinite(min_gap) && s.baseline / min_gap < 4.0e6) {
    const double h = min_gap * 0.999;
    bool ok = true;
    int64_t prev = -1;
    for (int64_t i = 0; i < m && ok; ++i) {
      const int64_t u = cell_of(tp[i], h);
      ok = u > prev;
      prev = u;
    }
    if (ok) {
      s.cells_ok = true;
      s.cell_h = h;
      s.n_cells = prev + 1;
    }
  }
  s.points_done = true;
}

// Bins and the grid's sums, the nbins cap, Sturges' bin count, the weight
// spreads and the cell table.
void plan_tail(const qlp_bls_params& p, StarPlanHost& s) {
  double edges = 0.0, dmax = 0.0;
  if (!tail_grid(p, s, &edges, &dmax)) return;
  tail_points(s);
  if (s.cells_ok) {
    s.cells_work = edges;
    s.bin_dmax = dmax;
  }
}

}  // namespace

void plan_one(const qlp_bls_params& p, const double* t, const double* y, const double* dy, int64_t n,
              double rho, StarPlanHost* out, const Windows* win, const PointDst* dst) {
  StarPlanHost& s = *out;
  if (!plan_head(p, t, y, dy, n, rho, s, dst)) return;
  grid_one(p, s, win);
  plan_tail(p, s);
}

namespace {

// Process-wide pool of host worker threads for the planner: started on first
// use, one fewer than the cores (the calling thread works too). A job is a range
// of task indices taken one at a time from an atomic counter, so stars of very
// different grid lengths balance across threads. One job runs at a time; a call
// that finds the pool busy (another host thread planning) starts threads of its
// own instead.
class HostPool {
 public:
  static HostPool& get() {
    // never destroyed (workers may outlive static teardown); a forked child, which
    // has none of the parent's threads, starts a pool of its own
    static std::once_flag once;
    std::call_once(once, [] { pthread_atfork(nullptr, nullptr, [] { instance().store(nullptr); }); });
    HostPool* p = instance().load();
    if (!p) {
      std::lock_guard<std::mutex> lk(create_mu());
      p = instance().load();
      if (!p) {
        p = new HostPool();
        instance().store(p);
      }
    }
    return *p;
  }
  int workers() const { return (int)th_.size(); }
  // Runs the job; an exception thrown by fn (on any thread) ends the job early and
  // is rethrown here once every thread has left it.
  bool try_run(int32_t n_tasks, int helpers, const std::function<void(int32_t)>& fn) {
    std::unique_lock<std::mutex> job(job_mu_, std::try_to_lock);
    if (!job.owns_lock()) return false;
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &fn;
      n_tasks_ = n_tasks;
      next_.store(0);
      err_ = nullptr;
      helpers_ = std::min(helpers, workers());
      active_ = helpers_;
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::exception_ptr err;
    {
      std::unique_lock<std::mutex> lk(mu_);
      done_cv_.wait(lk, [&] { return active_ == 0; });
      fn_ = nullptr;
      err = err_;
      err_ = nullptr;
    }
    if (err) std::rethrow_exception(err);
    return true;
  }

 private:
  HostPool() {
    const int n = std::max(0, (int)std::thread::hardware_concurrency() - 1);
    for (int i = 0; i < n; ++i) th_.emplace_back([this, i] { loop(i); });
    for (auto& x : th_) x.detach();
  }
  void work() {
    try {
      for (int32_t k = next_.fetch_add(1); k < n_tasks_; k = next_.fetch_add(1)) (*fn_)(k);
    } catch (...) {
      std::lock_guard<std::mutex> lk(mu_);
      if (!err_) err_ = std::current_exception();
      next_.store(n_tasks_);  // the other threads take no further task
    }
  }
  void loop(int idx) {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
        if (idx >= helpers_) continue;  // this job asked for fewer threads
      }
      work();
      std::lock_guard<std::mutex> lk(mu_);
      if (--active_ == 0) done_cv_.notify_all();
    }
  }
  static std::atomic<HostPool*>& instance() {
    static std::atomic<HostPool*> p{nullptr};
    return p;
  }
  static std::mutex& create_mu() {
    static std::mutex m;
    return m;
  }
  std::vector<std::thread> th_;
  std::mutex job_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int32_t)>* fn_ = nullptr;
  int32_t n_tasks_ = 0;
  std::atomic<int32_t> next_{0};
  int helpers_ = 0, active_ = 0;
  uint64_t gen_ = 0;
  std::exception_ptr err_;
};

}  // namespace

void parallel_stars(const qlp_bls_params& p, int32_t n_stars, const std::function<void(int32_t)>& fn) {
  int nth = p.n_threads > 0 ? p.n_threads : (int)std::thread::hardware_concurrency();
  nth = std::max(1, std::min(nth, std::max(1, n_stars)));
  if (nth == 1) {
    for (int32_t s = 0; s < n_stars; ++s) fn(s);
    return;
  }
  if (HostPool::get().try_run(n_stars, nth - 1, fn)) return;
  // the pool is busy with another caller's job: threads of this call's own
  std::vector<std::thread> th;
  std::vector<std::exception_ptr> err((size_t)nth);
  th.reserve((size_t)nth);
  for (int i = 0; i < nth; ++i)
    th.emplace_back([&, i]() {
      try {
        for (int32_t s = i; s < n_stars; s += nth) fn(s);
      } catch (...) {
        err[(size_t)i] = std::current_exception();
      }
    });
  for (auto& x : th) x.join();
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

void plan_all(const qlp_bls_params& p, int32_t n_stars, const int64_t* offsets, const double* t,
              const double* y, const double* dy, const double* rho, std::vector<StarPlanHost>* out,
              const int64_t* win_off, const double* win_lo, const double* win_hi, const PointDst* dst) {
  out->assign((size_t)n_stars, StarPlanHost());
  // star s's points go to the caller's arrays at its raw offset, when given
  auto dst_of = [&](int32_t s, PointDst* d) -> const PointDst* {
    if (!dst) return nullptr;
    const int64_t o = offsets[s] - offsets[0];
    d->tp = dst->tp + o;
    d->y = dst->y + o;
    d->dy = dst->dy + o;
    return d;
  };
  if (win_off || p.grid_mode == 1) {
    const std::vector<double> cper = p.grid_mode == 1 ? coarse_period_table(p) : std::vector<double>();
    parallel_stars(p, n_stars, [&](int32_t s) {
      const int64_t a = offsets[s], b = offsets[s + 1];
      const double r = rho ? rho[s] : NAN;
      Windows w;
      if (win_off) {
        w.lo = win_lo + win_off[s];
        w.hi = win_hi + win_off[s];
        w.n = win_off[s + 1] - win_off[s];
      }
      PointDst d;
      StarPlanHost& h = (*out)[(size_t)s];
      if (!plan_head(p, t + a, y + a, dy + a, b - a, r, h, dst_of(s, &d))) return;
      grid_one(p, h, win_off ? &w : nullptr, cper.empty() ? nullptr : cper.data());
      plan_tail(p, h);
    });
    return;
  }
  // plain grids: groups of kChains consecutive stars, their recurrences interleaved
  const int32_t n_groups = (n_stars + kChains - 1) / kChains;
  parallel_stars(p, n_groups, [&](int32_t g) {
    StarPlanHost* st[kChains];
    int n = 0;
    const int32_t s1 = std::min(n_stars, (g + 1) * kChains);
    for (int32_t s = g * kChains; s < s1; ++s) {
      const int64_t a = offsets[s], b = offsets[s + 1];
      StarPlanHost& h = (*out)[(size_t)s];
      PointDst d;
      if (plan_head(p, t + a, y + a, dy + a, b - a, rho ? rho[s] : NAN, h, dst_of(s, &d))) st[n++] = &h;
    }
    grid_chains(p, st, n);
    for (int j = 0; j < n; ++j) plan_tail(p, *st[j]);
  });
}

StarPoints points_of(StarPlanHost& s) {
  StarPoints o;
  o.head_ok = s.head_ok;
  o.status = s.head_ok ? 0 : s.status;
  o.n_valid = s.n_valid;
  o.t_ref = s.t_ref;
  o.baseline = s.baseline;
  o.pmin = s.pmin;
  o.pmax = s.pmax;
  o.rho_kg = s.rho_kg;
  if (!s.head_ok) return o;
  if (!s.points_done) tail_points(s);  // the grid was empty or over the cap
  o.w_spread = s.w_spread;
  o.wd_spread = s.wd_spread;
  o.wd_max = s.wd_max;
  o.y_exc = s.y_exc;
  o.cells_ok = s.cells_ok;
  o.cell_h = s.cell_h;
  o.n_cells = s.n_cells;
  return o;
}

void plan_all_from(const qlp_bls_params& p, int32_t n_stars, const StarPoints* pts,
                   std::vector<StarPlanHost>* out, const int64_t* win_off, const double* win_lo,
                   const double* win_hi) {
  out->assign((size_t)n_stars, StarPlanHost());
  const std::vector<double> cper = p.grid_mode == 1 ? coarse_period_table(p) : std::vector<double>();
  parallel_stars(p, n_stars, [&](int32_t st) {
    const StarPoints& q = pts[st];
    StarPlanHost& s = (*out)[(size_t)st];
    s.n_valid = q.n_valid;
    s.rho_kg = q.rho_kg;
    if (!q.head_ok) {  // the head's outcome: no grid (status as the head set it)
      s.status = q.status;
      if (q.status == QLP_STAR_EMPTY_GRID) {
        s.t_ref = q.t_ref;
        s.baseline = q.baseline;
        s.pmin = q.pmin;
        s.pmax = q.pmax;
      }
      return;
    }
    s.t_ref = q.t_ref;
    s.baseline = q.baseline;
    s.pmin = q.pmin;
    s.pmax = q.pmax;
    s.head_ok = true;
    Windows w;
    if (win_off) {
      w.lo = win_lo + win_off[st];
      w.hi = win_hi + win_off[st];
      w.n = win_off[st + 1] - win_off[st];
    }
    grid_one(p, s, win_off ? &w : nullptr, cper.empty() ? nullptr : cper.data());
    double edges = 0.0, dmax = 0.0;
    if (!tail_grid(p, s, &edges, &dmax)) return;
    s.w_spread = q.w_spread;
    s.wd_spread = q.wd_spread;
    s.wd_max = q.wd_max;
    s.y_exc = q.y_exc;
    s.points_done = true;
    if (q.cells_ok) {
      s.cells_ok = true;
      s.cell_h = q.cell_h;
      s.n_cells = q.n_cells;
      s.cells_work = edges;
      s.bin_dmax = dmax;
    }
  });
}

}  // namespace qlp
