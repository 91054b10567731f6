// qlp_bls_search_learned: the learned period proposal end to end behind one C
// call. A coarse BLS spectrum on the log-period grid (grid_mode 1) and its S/N
// feed the network; the top-k bins of its logits become frequency windows
// [1/P(k + w), 1/P(k - w)]; the paper's own grid (Sec. 2.1) is searched only inside
// them and scored with the coarse spectrum's trend and sigma_SR (Sec. 2.2 item 1).
// Every numeric stage is a kernel of this library; this file sequences the calls.
#include <cuda_runtime.h>

#include <algorithm>
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

// P(x) = coarse_pmin (coarse_pmax / coarse_pmin)^(x / (coarse_bins - 1)): the period
// of (fractional) coarse bin x.
double coarse_period(const qlp_bls_params& p, double x) {
  return p.coarse_pmin * std::pow(p.coarse_pmax / p.coarse_pmin, x / (double)(p.coarse_bins - 1));
}

bool coarse_ok(const qlp_bls_params* p) {
  return p && p->coarse_bins >= 2 && p->coarse_pmin > 0.0 && p->coarse_pmax > p->coarse_pmin;
}

// Frequency windows [1/P(k + w), 1/P(k - w)] around every valid (k >= 0) proposed bin,
// star by star; offsets[s] .. offsets[s + 1] - 1 are star s's windows.
void proposal_windows(const qlp_bls_params& p, int32_t n_stars, const int32_t* bins, int32_t k, double w,
                      std::vector<int64_t>* off, std::vector<double>* lo, std::vector<double>* hi) {
  off->assign((size_t)n_stars + 1, 0);
  lo->clear();
  hi->clear();
  for (int32_t s = 0; s < n_stars; ++s) {
    for (int32_t i = 0; i < k; ++i) {
      const int32_t kb = bins[(size_t)s * k + i];
      if (kb < 0) continue;
      lo->push_back(1.0 / coarse_period(p, (double)kb + w));
      hi->push_back(1.0 / coarse_period(p, (double)kb - w));
    }
    (*off)[(size_t)s + 1] = (int64_t)lo->size();
  }
}

}  // namespace

extern "C" int qlp_bls_coarse_periods(const qlp_bls_params* p, int32_t n, const double* x, double* periods) {
  if (!coarse_ok(p) || n < 0 || (n > 0 && (!x || !periods))) return QLP_ERR_ARG;
  for (int32_t i = 0; i < n; ++i) periods[i] = coarse_period(*p, x[i]);
  return QLP_OK;
}

extern "C" int qlp_bls_coarse_bins(const qlp_bls_params* p, int32_t n, const double* periods, int32_t* bins) {
  if (!coarse_ok(p) || n < 0 || (n > 0 && (!periods || !bins))) return QLP_ERR_ARG;
  const double scale = (double)(p->coarse_bins - 1) / std::log(p->coarse_pmax / p->coarse_pmin);
  for (int32_t i = 0; i < n; ++i) {
    if (!(periods[i] > 0.0)) {
      bins[i] = -1;
      continue;
    }
    const double xb = std::nearbyint(scale * std::log(periods[i] / p->coarse_pmin));
    bins[i] = (xb >= 0.0 && xb <= (double)(p->coarse_bins - 1)) ? (int32_t)xb : -1;
  }
  return QLP_OK;
}

extern "C" int qlp_bls_proposal_windows(const qlp_bls_params* p, int32_t n_stars, const int32_t* bins, int32_t k,
                                        double half_width, int64_t* win_offsets, double* win_lo, double* win_hi,
                                        int64_t capacity) {
  if (!coarse_ok(p) || n_stars < 0 || k < 1 || !(half_width > 0.0) || (n_stars > 0 && !bins) || !win_offsets)
    return QLP_ERR_ARG;
  std::vector<int64_t> off;
  std::vector<double> lo, hi;
  proposal_windows(*p, n_stars, bins, k, half_width, &off, &lo, &hi);
  std::copy(off.begin(), off.end(), win_offsets);
  if (!win_lo && !win_hi) return QLP_OK;
  if (!win_lo || !win_hi || capacity < (int64_t)lo.size()) return QLP_ERR_ARG;
  std::copy(lo.begin(), lo.end(), win_lo);
  std::copy(hi.begin(), hi.end(), win_hi);
  return QLP_OK;
}

namespace {

// One chunk of stars on the learned path: its coarse plan and spectrum, the
// network's proposals, and its refine plan and spectrum.
struct LearnedChunk {
  int32_t s0 = 0, ns = 0;
  PlanGuard cp, rp;
  Spectrum c{}, r{};
  double* trend = nullptr;
  uint16_t* x0 = nullptr;
  int32_t* bins = nullptr;
  cudaEvent_t proposed = nullptr;  // the chunk's proposals are in `bins`
  ~LearnedChunk() {
    if (proposed) cudaEventDestroy(proposed);
  }
};

}  // namespace

extern "C" int qlp_bls_search_learned(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets,
                                      const double* t, const double* y, const double* dy,
                                      const double* rho, const double* rstar, qlp_cnn_t* net, int32_t k,
                                      double half_width, void* stream, qlp_bls_best* best_host,
                                      int32_t* bins_host) {
  if (!p || !best_host || n_stars < 0 || k < 1 || !(half_width > 0.0) || !coarse_ok(p)) return QLP_ERR_ARG;
  if (n_stars == 0) return QLP_OK;
  if (!offsets) return QLP_ERR_ARG;
  int32_t max_batch = 0, len = p->coarse_bins;
  int rc = net ? qlp_cnn_shape(net, &max_batch, &len) : QLP_OK;
  if (rc) return rc;
  if (len != p->coarse_bins || k > len) return QLP_ERR_ARG;
  // Chunks of whole stars with about equal points, in a two-stage pipeline: while
  // the device searches chunk c's coarse spectrum and runs the network on it, the
  // host plans chunk c + 1's coarse grid and then chunk c - 1's refine grid. Plans
  // upload and synchronise on their own stream; coarse work and the network run on
  // one stream, the refine searches on another.
  const int64_t npts = offsets[n_stars] - offsets[0];
  const int nch = n_stars >= 1024 ? std::min(8, n_stars / 256) : 1;
  cudaStream_t st_in = (cudaStream_t)stream;
  cudaStream_t st_up = nullptr, st_c = nullptr, st_r = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st_up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st_c, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st_r, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (st_up) cudaStreamDestroy(st_up);
    if (st_c) cudaStreamDestroy(st_c);
    return qlp::record_cuda_error(e, "cudaStreamCreate");
  }
  // the caller's stream's earlier work (the network's weights) comes first
  cudaEvent_t ev_in = nullptr;
  e = cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev_in, st_in);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st_c, ev_in, 0);
  if (ev_in) cudaEventDestroy(ev_in);
  std::vector<LearnedChunk> ch((size_t)nch);
  {
    DevBufs buf_c(st_c), buf_r(st_r);
    float* logits = nullptr;
    qlp_bls_params pc = *p;
    pc.grid_mode = 1;
    qlp_bls_params pr = *p;
    pr.grid_mode = 0;
    if (e != cudaSuccess) rc = qlp::record_cuda_error(e, "stream order");
    if (rc == QLP_OK && net) rc = buf_c.get(&logits, (size_t)max_batch * len);

    // stage 1 of chunk c: coarse plan (host), spectrum, S/N, network input, proposals
    auto coarse = [&](int c) -> int {
      LearnedChunk& q = ch[(size_t)c];
      const int64_t o0 = offsets[q.s0];
      std::vector<int64_t> off((size_t)q.ns + 1);
      for (int32_t i = 0; i <= q.ns; ++i) off[(size_t)i] = offsets[q.s0 + i] - o0;
      int r2 = qlp_bls_plan(&pc, q.ns, off.data(), t + o0, y + o0, dy + o0, rho ? rho + q.s0 : nullptr,
                            rstar ? rstar + q.s0 : nullptr, st_up, &q.cp.p);
      if (r2) return r2;
      int64_t nfc = 0;
      if ((r2 = qlp_bls_plan_info(q.cp.p, &nfc, nullptr, nullptr, nullptr, nullptr, nullptr))) return r2;
      if ((r2 = alloc_spectrum(buf_c, nfc, q.ns, &q.c)) || (r2 = buf_c.get(&q.trend, (size_t)q.ns * QLP_TREND_DOUBLES)) ||
          (r2 = buf_c.get(&q.x0, (size_t)q.ns * len * QLP_CNN_IN_CH)) || (r2 = buf_c.get(&q.bins, (size_t)q.ns * k)))
        return r2;
      if ((r2 = qlp_bls_search(q.cp.p, st_c, q.c.sr, q.c.qidx, q.c.kbin, q.c.s, q.c.r))) return r2;
      if ((r2 = qlp_bls_snr_trend(q.cp.p, st_c, q.c.sr, q.c.qidx, q.c.kbin, q.c.s, q.c.r, nullptr, q.trend, q.c.snr,
                                  q.c.best)))
        return r2;
      if (net) {
        if ((r2 = qlp_bls_coarse_tensor(q.cp.p, st_c, q.c.snr, len, q.x0, nullptr))) return r2;
        for (int32_t a = 0; a < q.ns; a += max_batch) {
          const int32_t nb = q.ns - a < max_batch ? q.ns - a : max_batch;
          const uint16_t* xb = q.x0 + (size_t)a * len * QLP_CNN_IN_CH;
          if ((r2 = qlp_cnn_forward(net, xb, nb, logits, st_c))) return r2;
          if ((r2 = qlp_cnn_topk(logits, xb, nb, len, k, q.bins + (size_t)a * k, st_c))) return r2;
        }
      } else {  // without the network: the top-k coarse bins by S/N
        float* rows = nullptr;
        if ((r2 = buf_c.get(&rows, (size_t)q.ns * len))) return r2;
        if ((r2 = qlp_bls_coarse_tensor(q.cp.p, st_c, q.c.snr, len, q.x0, rows))) return r2;
        if ((r2 = qlp_cnn_topk(rows, q.x0, q.ns, len, k, q.bins, st_c))) return r2;
      }
      cudaError_t e2 = cudaEventCreateWithFlags(&q.proposed, cudaEventDisableTiming);
      if (e2 == cudaSuccess) e2 = cudaEventRecord(q.proposed, st_c);
      return e2 == cudaSuccess ? QLP_OK : qlp::record_cuda_error(e2, "proposal event");
    };
    // stage 2 of chunk c: windows around the proposals, refine plan (host), search,
    // S/N from the coarse trend
    auto refine = [&](int c) -> int {
      LearnedChunk& q = ch[(size_t)c];
      cudaError_t e2 = cudaEventSynchronize(q.proposed);
      std::vector<int32_t> hb((size_t)q.ns * k);
      if (e2 == cudaSuccess)
        e2 = cudaMemcpyAsync(hb.data(), q.bins, sizeof(int32_t) * hb.size(), cudaMemcpyDeviceToHost, st_up);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st_up);
      if (e2 != cudaSuccess) return qlp::record_cuda_error(e2, "proposal download");
      if (bins_host)
        for (size_t i = 0; i < hb.size(); ++i) bins_host[(size_t)q.s0 * k + i] = hb[i];
      // windows in frequency around each proposed bin
      std::vector<int64_t> woff;
      std::vector<double> wlo, whi;
      proposal_windows(*p, q.ns, hb.data(), k, half_width, &woff, &wlo, &whi);
      // the refine plan from the coarse plan: its stars' point analysis and device points
      int r2 = qlp_bls_plan_windows_from(q.cp.p, &pr, woff.data(), wlo.data(), whi.data(), st_up, &q.rp.p);
      if (r2) return r2;
      int64_t nfr = 0;
      if ((r2 = qlp_bls_plan_info(q.rp.p, &nfr, nullptr, nullptr, nullptr, nullptr, nullptr))) return r2;
      if ((r2 = alloc_spectrum(buf_r, nfr, q.ns, &q.r))) return r2;
      if ((r2 = qlp_bls_search(q.rp.p, st_r, q.r.sr, q.r.qidx, q.r.kbin, q.r.s, q.r.r))) return r2;
      return qlp_bls_snr_trend(q.rp.p, st_r, q.r.sr, q.r.qidx, q.r.kbin, q.r.s, q.r.r, q.trend, nullptr, q.r.snr,
                               q.r.best);
    };

    int32_t s0 = 0;
    for (int c = 0; c < nch; ++c) {  // chunk boundaries by points
      int32_t s1 = n_stars;
      if (c < nch - 1) {
        const int64_t goal = offsets[0] + npts * (c + 1) / nch;
        s1 = s0;
        while (s1 < n_stars && offsets[s1] < goal) ++s1;
        s1 = std::max(s1, std::min(n_stars, s0 + 1));
      }
      ch[(size_t)c].s0 = s0;
      ch[(size_t)c].ns = s1 - s0;
      s0 = s1;
    }
    for (int c = 0; c <= nch && rc == QLP_OK; ++c) {
      if (c < nch && ch[(size_t)c].ns > 0) rc = coarse(c);
      if (rc == QLP_OK && c >= 1 && ch[(size_t)(c - 1)].ns > 0) rc = refine(c - 1);
    }
    if (rc == QLP_OK) {
      e = cudaStreamSynchronize(st_r);
      for (const LearnedChunk& q : ch) {
        if (e != cudaSuccess || q.ns == 0) continue;
        e = cudaMemcpyAsync(best_host + q.s0, q.r.best, sizeof(qlp_bls_best) * (size_t)q.ns, cudaMemcpyDeviceToHost,
                            st_up);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(st_up);
      if (e != cudaSuccess) rc = qlp::record_cuda_error(e, "result download");
    }
    // device error flags of every plan and of the network's tensor-core waits
    int32_t fl = 0;
    for (const LearnedChunk& q : ch) {
      if (rc != QLP_OK) break;
      for (qlp_bls_plan_t* pp : {q.cp.p, q.rp.p}) {
        if (!pp) continue;
        int32_t f = 0;
        const int x = qlp_bls_device_status(pp, st_r, &f);
        if (x && x != QLP_ERR_DEVICE) rc = x;
        fl |= f;
      }
    }
    if (rc == QLP_OK) {
      int32_t f3 = 0;
      const int r3 = net ? qlp_cnn_loss(net, nullptr, &f3, st_c) : QLP_OK;
      if (r3 && r3 != QLP_ERR_DEVICE) rc = r3;
      fl |= f3;
      if (rc == QLP_OK && fl) rc = QLP_ERR_DEVICE;
    }
    cudaStreamSynchronize(st_c);
    cudaStreamSynchronize(st_r);
  }  // buffers freed (stream-ordered) before the streams go
  for (cudaStream_t x : {st_up, st_c, st_r}) {
    cudaStreamSynchronize(x);
    cudaStreamDestroy(x);
  }
  return rc;
}
