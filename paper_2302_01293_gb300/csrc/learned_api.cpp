// qlp_bls_search_learned: the learned period proposal end to end behind one C
// call. A coarse BLS spectrum on the log-period grid (grid_mode 1) and its S/N
// feed the network; the top-k bins of its logits become frequency windows
// [1/P(k + w), 1/P(k - w)]; the paper's own grid (Sec. 2.1) is searched only inside
// them and scored with the coarse spectrum's trend and sigma_SR (Sec. 2.2 item 1).
// Every numeric stage is a kernel of this library; this file sequences the calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "qlp_internal.h"

namespace {

struct DevBufs {
  std::vector<void*> ptrs;
  cudaStream_t s;
  explicit DevBufs(cudaStream_t st) : s(st) {}
  ~DevBufs() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  int get(T** p, size_t count) {
    *p = nullptr;
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

struct PlanGuard {
  qlp_bls_plan_t* p = nullptr;
  ~PlanGuard() {
    if (p) qlp_bls_plan_destroy(p);
  }
};

// Device outputs of one search + S/N.
struct Spectrum {
  float *sr, *s, *r, *snr;
  uint8_t* qidx;
  uint32_t* kbin;
  qlp_bls_best* best;
};

int alloc_spectrum(DevBufs& b, int64_t nf, int32_t n_stars, Spectrum* o) {
  int rc;
  if ((rc = b.get(&o->sr, (size_t)nf)) || (rc = b.get(&o->s, (size_t)nf)) || (rc = b.get(&o->r, (size_t)nf)) ||
      (rc = b.get(&o->snr, (size_t)nf)) || (rc = b.get(&o->qidx, (size_t)nf)) ||
      (rc = b.get(&o->kbin, (size_t)nf)) || (rc = b.get(&o->best, (size_t)n_stars)))
    return rc;
  return QLP_OK;
}

}  // namespace

extern "C" int qlp_bls_search_learned(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets,
                                      const double* t, const double* y, const double* dy,
                                      const double* rho, const double* rstar, qlp_cnn_t* net, int32_t k,
                                      double half_width, void* stream, qlp_bls_best* best_host,
                                      int32_t* bins_host) {
  if (!p || !net || !best_host || n_stars < 0 || k < 1 || !(half_width > 0.0)) return QLP_ERR_ARG;
  if (n_stars == 0) return QLP_OK;
  int32_t max_batch = 0, len = 0;
  int rc = qlp_cnn_shape(net, &max_batch, &len);
  if (rc) return rc;
  if (len != p->coarse_bins || k > len) return QLP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  DevBufs buf(st);

  // coarse spectrum, its S/N and trend records, and the network input
  qlp_bls_params pc = *p;
  pc.grid_mode = 1;
  PlanGuard cp;
  if ((rc = qlp_bls_plan(&pc, n_stars, offsets, t, y, dy, rho, rstar, stream, &cp.p))) return rc;
  int64_t nfc = 0;
  if ((rc = qlp_bls_plan_info(cp.p, &nfc, nullptr, nullptr, nullptr, nullptr, nullptr))) return rc;
  Spectrum c{};
  double* trend = nullptr;
  uint16_t* x0 = nullptr;  // BF16 [n_stars][len][2]
  float* logits = nullptr;
  int32_t* bins = nullptr;
  if ((rc = alloc_spectrum(buf, nfc, n_stars, &c)) || (rc = buf.get(&trend, (size_t)n_stars * QLP_TREND_DOUBLES)) ||
      (rc = buf.get(&x0, (size_t)n_stars * len * 2)) || (rc = buf.get(&logits, (size_t)max_batch * len)) ||
      (rc = buf.get(&bins, (size_t)n_stars * k)))
    return rc;
  if ((rc = qlp_bls_search(cp.p, stream, c.sr, c.qidx, c.kbin, c.s, c.r))) return rc;
  if ((rc = qlp_bls_snr_trend(cp.p, stream, c.sr, c.qidx, c.kbin, c.s, c.r, nullptr, trend, c.snr, c.best)))
    return rc;
  if ((rc = qlp_bls_coarse_tensor(cp.p, stream, c.snr, len, x0))) return rc;

  // proposals: the network's top-k bins per star
  for (int32_t a = 0; a < n_stars; a += max_batch) {
    const int32_t nb = n_stars - a < max_batch ? n_stars - a : max_batch;
    const uint16_t* xb = x0 + (size_t)a * len * 2;
    if ((rc = qlp_cnn_forward(net, xb, nb, logits, stream))) return rc;
    if ((rc = qlp_cnn_topk(logits, xb, nb, len, k, bins + (size_t)a * k, stream))) return rc;
  }
  std::vector<int32_t> hb((size_t)n_stars * k);
  cudaError_t e = cudaMemcpyAsync(hb.data(), bins, sizeof(int32_t) * hb.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return qlp::record_cuda_error(e, "proposal download");
  if (bins_host)
    for (size_t i = 0; i < hb.size(); ++i) bins_host[i] = hb[i];

  // windows in frequency around each proposed bin: P(x) = pmin (pmax/pmin)^(x/(bins-1))
  const double ratio = p->coarse_pmax / p->coarse_pmin;
  auto period = [&](double x) { return p->coarse_pmin * std::pow(ratio, x / (double)(len - 1)); };
  std::vector<int64_t> woff((size_t)n_stars + 1, 0);
  std::vector<double> wlo, whi;
  for (int32_t s = 0; s < n_stars; ++s) {
    for (int32_t i = 0; i < k; ++i) {
      const int32_t kb = hb[(size_t)s * k + i];
      if (kb < 0) continue;
      wlo.push_back(1.0 / period((double)kb + half_width));
      whi.push_back(1.0 / period((double)kb - half_width));
    }
    woff[(size_t)s + 1] = (int64_t)wlo.size();
  }

  // full-resolution grid inside the windows, scored with the coarse trend
  qlp_bls_params pr = *p;
  pr.grid_mode = 0;
  PlanGuard rp;
  if ((rc = qlp_bls_plan_windows(&pr, n_stars, offsets, t, y, dy, rho, rstar, woff.data(), wlo.data(), whi.data(),
                                 stream, &rp.p)))
    return rc;
  int64_t nfr = 0;
  if ((rc = qlp_bls_plan_info(rp.p, &nfr, nullptr, nullptr, nullptr, nullptr, nullptr))) return rc;
  Spectrum r{};
  if ((rc = alloc_spectrum(buf, nfr, n_stars, &r))) return rc;
  if ((rc = qlp_bls_search(rp.p, stream, r.sr, r.qidx, r.kbin, r.s, r.r))) return rc;
  if ((rc = qlp_bls_snr_trend(rp.p, stream, r.sr, r.qidx, r.kbin, r.s, r.r, trend, nullptr, r.snr, r.best)))
    return rc;
  e = cudaMemcpyAsync(best_host, r.best, sizeof(qlp_bls_best) * (size_t)n_stars, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return qlp::record_cuda_error(e, "result download");
  // device error flags of both plans and of the network's tensor-core waits
  int32_t f1 = 0, f2 = 0, f3 = 0;
  const int r1 = qlp_bls_device_status(cp.p, stream, &f1);
  const int r2 = qlp_bls_device_status(rp.p, stream, &f2);
  const int r3 = qlp_cnn_loss(net, nullptr, &f3, stream);
  for (int x : {r1, r2, r3})
    if (x && x != QLP_ERR_DEVICE) return x;
  return (f1 | f2 | f3) ? QLP_ERR_DEVICE : QLP_OK;
}
