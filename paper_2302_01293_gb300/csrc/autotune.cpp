// qlp_bls_autotune: launch-shape tuner for the search. The results of the
// search do not depend on these settings (every setting gives the FP64 bins of
// Sec. 2.1's BLS); only its speed does. Candidates are timed with CUDA events on
// an evenly spaced sample of the batch's stars and the fastest is kept in a
// process-wide cache keyed by the device, the fixed options and a coarse
// signature of the workload (log2 of the star count and of the median and
// largest star lengths).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "qlp_internal.h"

namespace {

using Key = std::tuple<int, int, int, int, int, int, int, int, int, int, int>;

std::mutex g_mu;
std::map<Key, qlp_bls_params> g_cache;

int ilog2(double x) { return x >= 1.0 ? (int)std::lround(std::log2(x)) : -1; }

struct Outs {
  float *sr = nullptr, *s = nullptr, *r = nullptr;
  uint8_t* q = nullptr;
  uint32_t* k = nullptr;
  ~Outs() {
    cudaFree(sr); cudaFree(s); cudaFree(r); cudaFree(q); cudaFree(k);
  }
};

}  // namespace

extern "C" int qlp_bls_autotune(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets,
                                const double* t, const double* y, const double* dy, const double* rho,
                                const double* rstar, int32_t sample_stars, void* stream, qlp_bls_params* out,
                                int32_t* cached) {
  if (!p || !out || n_stars < 0 || !offsets || sample_stars < 1) return QLP_ERR_ARG;
  for (int32_t s = 0; s < n_stars; ++s)
    if (offsets[s + 1] < offsets[s]) return QLP_ERR_ARG;
  *out = *p;
  if (cached) *cached = 0;
  if (n_stars == 0) return QLP_OK;

  std::vector<int64_t> len((size_t)n_stars);
  for (int32_t s = 0; s < n_stars; ++s) len[(size_t)s] = offsets[s + 1] - offsets[s];
  std::vector<int64_t> sorted = len;
  std::nth_element(sorted.begin(), sorted.begin() + n_stars / 2, sorted.end());
  const int64_t med = sorted[(size_t)n_stars / 2];
  const int64_t mx = *std::max_element(len.begin(), len.end());
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return qlp::record_cuda_error(e, "cudaGetDevice");
  const Key key{dev, p->sum_mode, p->phase_mode, p->method, p->grid_mode, p->warps_per_block, p->chunk_freqs,
                p->cell_window, ilog2((double)n_stars), ilog2((double)med), ilog2((double)mx)};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *out = it->second;
      if (cached) *cached = 1;
      return QLP_OK;
    }
  }

  // evenly spaced sample of stars
  const int32_t ns = std::min(n_stars, sample_stars);
  std::vector<int64_t> soff(1, 0);
  std::vector<double> st, sy, sdy, srho, srs;
  for (int32_t i = 0; i < ns; ++i) {
    const int32_t s = (int32_t)(((int64_t)i * n_stars) / ns);
    st.insert(st.end(), t + offsets[s], t + offsets[s + 1]);
    sy.insert(sy.end(), y + offsets[s], y + offsets[s + 1]);
    sdy.insert(sdy.end(), dy + offsets[s], dy + offsets[s + 1]);
    srho.push_back(rho ? rho[s] : NAN);
    srs.push_back(rstar ? rstar[s] : 1.0);
    soff.push_back((int64_t)st.size());
  }

  // candidates: only the settings the caller left to the library
  std::vector<qlp_bls_params> cand;
  const std::vector<int> warps = p->warps_per_block ? std::vector<int>{p->warps_per_block}
                                                    : std::vector<int>{0, 16, 8};
  const std::vector<int> chunk_mul = p->chunk_freqs ? std::vector<int>{0} : std::vector<int>{0, 4, 16};
  const std::vector<int> windows = p->cell_window ? std::vector<int>{p->cell_window} : std::vector<int>{0, 2048};
  for (int w : warps)
    for (int c : chunk_mul)
      for (int cw : windows) {
        qlp_bls_params q = *p;
        q.warps_per_block = w;
        q.chunk_freqs = c ? c * (w ? w : 32) : p->chunk_freqs;
        q.cell_window = cw;
        cand.push_back(q);
      }

  cudaStream_t sm = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return qlp::record_cuda_error(e, "cudaEventCreate");
  }
  Outs o;
  int64_t cap = -1;
  float best_ms = INFINITY;
  int rc = QLP_OK;
  bool any_windowed = false;
  for (size_t ci = 0; ci < cand.size() && rc == QLP_OK; ++ci) {
    const qlp_bls_params& q = cand[ci];
    if (q.cell_window != p->cell_window && !any_windowed) continue;  // no star needs windows
    qlp_bls_plan_t* pl = nullptr;
    rc = qlp_bls_plan(&q, ns, soff.data(), st.data(), sy.data(), sdy.data(), srho.data(), srs.data(), stream, &pl);
    if (rc == QLP_ERR_UNSUPPORTED) { rc = QLP_OK; continue; }  // launch shape does not fit: skip
    if (rc) break;
    int32_t nwin = 0;
    qlp_bls_plan_stats(pl, nullptr, nullptr, nullptr, nullptr, &nwin);
    if (ci == 0) any_windowed = nwin > 0;
    int64_t nf = 0;
    qlp_bls_plan_info(pl, &nf, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (cap < 0) {
      cap = std::max<int64_t>(nf, 1);
      if (cudaMalloc(&o.sr, 4 * cap) || cudaMalloc(&o.s, 4 * cap) || cudaMalloc(&o.r, 4 * cap) ||
          cudaMalloc(&o.q, cap) || cudaMalloc(&o.k, 4 * cap)) {
        qlp::record_cuda_error(cudaGetLastError(), "cudaMalloc");
        qlp_bls_plan_destroy(pl);
        rc = QLP_ERR_NOMEM;
        break;
      }
    }
    float ms = INFINITY;
    for (int rep = 0; rep < 3 && rc == QLP_OK; ++rep) {  // first run warms up
      if ((e = cudaEventRecord(e0, sm)) != cudaSuccess) { rc = qlp::record_cuda_error(e, "event"); break; }
      rc = qlp_bls_search(pl, stream, o.sr, o.q, o.k, o.s, o.r);
      if (rc) break;
      if ((e = cudaEventRecord(e1, sm)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
        rc = qlp::record_cuda_error(e, "event");
        break;
      }
      float v = 0.f;
      cudaEventElapsedTime(&v, e0, e1);
      if (rep > 0) ms = std::min(ms, v);
    }
    int32_t flags = 0;
    if (rc == QLP_OK) rc = qlp_bls_device_status(pl, stream, &flags);
    qlp_bls_plan_destroy(pl);
    if (rc) break;
    if (ms < best_ms) {
      best_ms = ms;
      *out = q;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = *out;
  return QLP_OK;
}
