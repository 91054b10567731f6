// qlp_bls_search_multi: several candidates per star by iterative masking (an
// extension: the paper reports one candidate per star). Each round runs the
// whole search (plan, BLS, S/N, best, post-BLS statistics of Sec. 2.2) on the
// points still kept, then removes the points within one fitted transit duration
// of the candidate's mid-transit times, |dt| < q P (dt the signed distance from
// the nearest mid-transit time, from the fitted epoch and q when the fit ran,
// else from the BLS box). A star leaves the loop when a round finds nothing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "qlp_internal.h"

namespace {

struct Scratch {
  std::vector<void*> ptrs;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() { release(); }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
    ptrs.clear();
  }
  template <typename T>
  int get(T** p, size_t count) {
    void* v = nullptr;
    const cudaError_t e = cudaMallocAsync(&v, (count ? count : 1) * sizeof(T), s);
    if (e != cudaSuccess) {
      qlp::record_cuda_error(e, "cudaMallocAsync");
      return QLP_ERR_NOMEM;
    }
    ptrs.push_back(v);
    *p = (T*)v;
    return QLP_OK;
  }
};

}  // namespace

extern "C" int qlp_bls_search_multi(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets,
                                    const double* t, const double* y, const double* dy, const double* rho,
                                    const double* rstar, int32_t n_planets, void* stream, qlp_bls_best* best_host,
                                    qlp_bls_cand_stats* stats_host, int32_t* n_found) {
  if (!p || n_stars < 0 || n_planets < 1 || !best_host || !stats_host || !offsets) return QLP_ERR_ARG;
  if (n_stars == 0) return QLP_OK;
  for (int32_t s = 0; s < n_stars; ++s)
    if (offsets[s + 1] < offsets[s]) return QLP_ERR_ARG;
  const int64_t npt = offsets[n_stars];
  if (npt > 0 && (!t || !y || !dy)) return QLP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint8_t> keep((size_t)npt, 1);
  std::vector<uint8_t> active((size_t)n_stars, 1);
  if (n_found)
    for (int32_t s = 0; s < n_stars; ++s) n_found[s] = 0;
  std::vector<int64_t> off((size_t)n_stars + 1);
  std::vector<double> tc, yc, dyc;
  tc.reserve((size_t)npt);
  yc.reserve((size_t)npt);
  dyc.reserve((size_t)npt);
  for (int32_t it = 0; it < n_planets; ++it) {
    // the points still kept (stars that found nothing keep none)
    tc.clear();
    yc.clear();
    dyc.clear();
    off[0] = 0;
    for (int32_t s = 0; s < n_stars; ++s) {
      if (active[(size_t)s])
        for (int64_t i = offsets[s]; i < offsets[s + 1]; ++i)
          if (keep[(size_t)i]) {
            tc.push_back(t[i]);
            yc.push_back(y[i]);
            dyc.push_back(dy[i]);
          }
      off[(size_t)s + 1] = (int64_t)tc.size();
    }
    qlp_bls_plan_t* pl = nullptr;
    int rc = qlp_bls_plan(p, n_stars, off.data(), tc.data(), yc.data(), dyc.data(), rho, rstar, stream, &pl);
    if (rc) return rc;
    int64_t nf = 0;
    qlp_bls_plan_info(pl, &nf, nullptr, nullptr, nullptr, nullptr, nullptr);
    Scratch sc(st);
    float *sr = nullptr, *sb = nullptr, *rb = nullptr, *snr = nullptr;
    uint8_t* q = nullptr;
    uint32_t* k = nullptr;
    qlp_bls_best* best = nullptr;
    qlp_bls_cand_stats* stats = nullptr;
    if ((rc = sc.get(&sr, (size_t)nf)) || (rc = sc.get(&sb, (size_t)nf)) || (rc = sc.get(&rb, (size_t)nf)) ||
        (rc = sc.get(&snr, (size_t)nf)) || (rc = sc.get(&q, (size_t)nf)) || (rc = sc.get(&k, (size_t)nf)) ||
        (rc = sc.get(&best, (size_t)n_stars)) || (rc = sc.get(&stats, (size_t)n_stars))) {
      qlp_bls_plan_destroy(pl);
      return rc;
    }
    if (!(rc = qlp_bls_search(pl, stream, sr, q, k, sb, rb)) &&
        !(rc = qlp_bls_snr(pl, stream, sr, q, k, sb, rb, snr, best)))
      rc = qlp_bls_candidate_stats(pl, stream, best, stats);
    qlp_bls_best* bh = best_host + (size_t)it * n_stars;
    qlp_bls_cand_stats* sh = stats_host + (size_t)it * n_stars;
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaMemcpyAsync(bh, best, sizeof(qlp_bls_best) * (size_t)n_stars, cudaMemcpyDeviceToHost, st);
    if (!rc && e == cudaSuccess)
      e = cudaMemcpyAsync(sh, stats, sizeof(qlp_bls_cand_stats) * (size_t)n_stars, cudaMemcpyDeviceToHost, st);
    if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(st);
    int32_t flags = 0;
    if (!rc && e == cudaSuccess) rc = qlp_bls_device_status(pl, stream, &flags);
    sc.release();
    qlp_bls_plan_destroy(pl);
    if (e != cudaSuccess) return qlp::record_cuda_error(e, "multi-planet round");
    if (rc) return rc;
    // mask the found transits
    for (int32_t s = 0; s < n_stars; ++s) {
      if (!active[(size_t)s]) continue;
      const qlp_bls_best& b = bh[s];
      if (b.f_idx < 0) {
        active[(size_t)s] = 0;
        continue;
      }
      if (n_found) n_found[s] += 1;
      const qlp_bls_cand_stats& c = sh[s];
      const bool fitted = c.status == QLP_STATS_OK || c.status == QLP_STATS_NOT_CONVERGED;
      const double t0 = fitted ? c.t0 : b.t0;
      const double width = (fitted ? c.q : b.q) * b.period;
      for (int64_t i = offsets[s]; i < offsets[s + 1]; ++i) {
        if (!keep[(size_t)i]) continue;
        const double u = t[i] - t0;
        const double n = std::floor(u / b.period + 0.5);
        const double dt = u - b.period * n;
        if (std::fabs(dt) < width) keep[(size_t)i] = 0;
      }
    }
  }
  return QLP_OK;
}
