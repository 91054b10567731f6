// qlp_bls_search_static: the BLS search of one star without any device memory
// allocation, for callers that are not allowed to call cudaMalloc (for example
// code running inside a framework that owns every device allocation, or a
// process whose memory pool is fixed before work starts). The paper has no
// counterpart of this entry point.
//
// The scratch memory the search needs beyond its inputs and outputs (the
// prepared point records, the frequency table, the work queue and its head)
// lives in one file-scope __device__ array of QLP_STATIC_SCRATCH_BYTES. Every
// GPU that loads the library holds that array until the process exits. Host
// code must not use the array's name as a device address: on the first call on
// each device (with that device current) its address is looked up once with
// cudaGetSymbolAddress and cached.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "planner.h"
#include "qlp_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[QLP_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Fill the star record, interleave (f, q_min), build the work queue and clear
// the queue head and error word (the scratch keeps the previous call's bytes).
__global__ void static_setup_kernel(qlp::StarDev* star, int32_t n_pts, int32_t n_f, double baseline,
                                    const double* f, const double* qmin, double2* fq,
                                    qlp::WorkItem* items, int32_t n_items, int32_t chunk,
                                    int32_t* ctl) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  if (tid == 0) {
    qlp::StarDev s{};
    s.pt_off = 0;
    s.pad_off = 0;
    s.f_off = 0;
    s.n_pts = n_pts;
    s.n_f = n_f;
    s.status = 0;
    s.sturges_nb = 0;
    s.fp64_phase = 0;
    s.t_ref = 0.0;
    s.baseline = baseline;
    *star = s;
    ctl[0] = 0;
    ctl[1] = 0;
  }
  for (int i = tid; i < n_f; i += stride) fq[i] = make_double2(f[i], qmin[i]);
  for (int i = tid; i < n_items; i += stride) {
    qlp::WorkItem w{};
    w.star = 0;
    w.f_begin = i * chunk;
    w.f_count = min(chunk, n_f - i * chunk);
    items[i] = w;
  }
}

int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QLP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return QLP_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return QLP_OK;
}

}  // namespace

extern "C" int qlp_bls_search_static(const qlp_bls_params* pin, int32_t n, const double* tp,
                                     const double* y, const double* dy, double baseline,
                                     int32_t n_f, const double* freqs, const double* qmins,
                                     void* stream, float* sr, uint8_t* qidx, uint32_t* phase_bin,
                                     float* s_best, float* r_best, int32_t* flags) {
  qlp_bls_params p;
  if (pin) p = *pin; else qlp_bls_params_default(&p);
  if (n < 2 || n_f < 1 || !tp || !y || !dy || !freqs || !qmins || !sr) return QLP_ERR_ARG;
  if (!(baseline > 0.0) || !(p.noverlap >= 1.0) || !(p.dlogq > 0.0) || !(p.qmin_fac > 0.0) ||
      !(p.qmax_fac >= p.qmin_fac))
    return QLP_ERR_ARG;
  if (p.phase_mode < 0 || p.phase_mode > 2 || p.sum_mode < 0 || p.sum_mode > 3) return QLP_ERR_ARG;
  // one shared histogram per frequency only: the per-duration variant needs the cell path
  if (p.bin_mode != QLP_BIN_SHARED) return QLP_ERR_UNSUPPORTED;
  // this entry point folds every point; it runs QLP_SUM_FIXED as compensated sums
  const int sum_mode = p.sum_mode == QLP_SUM_PLAIN ? QLP_SUM_PLAIN : QLP_SUM_COMP;
  if (p.warps_per_block != 0 && p.warps_per_block != 4 && p.warps_per_block != 8 &&
      p.warps_per_block != 16 && p.warps_per_block != 32)
    return QLP_ERR_ARG;
  const int nq = qlp::n_q_of(p);
  if (nq < 1 || nq > qlp::kMaxQ) return QLP_ERR_UNSUPPORTED;
  if ((p.noverlap + 1.0) * std::exp((nq - 1) * p.dlogq) + 0.5 >= (double)qlp::kMPad)
    return QLP_ERR_UNSUPPORTED;

  // sizes from the host grid; the FP32 fold needs T f nbins < 2^22, else FP64
  int nbins_max = 1;
  double ymax = 0.0;
  for (int32_t k = 0; k < n_f; ++k) {
    if (!(qmins[k] > 0.0) || !(freqs[k] > 0.0)) return QLP_ERR_ARG;
    const int nb = qlp::nbins_of(qmins[k], p);
    nbins_max = std::max(nbins_max, nb);
    ymax = std::max(ymax, baseline * freqs[k] * (double)nb);
  }
  if (nbins_max > p.nbins_cap) return QLP_ERR_ARG;
  const int64_t npad = ((int64_t)n + 31) & ~(int64_t)31;

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QLP_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QLP_ERR_CUDA;

  // launch shape, as the planned path chooses it
  const int NA = (sum_mode == QLP_SUM_COMP) ? 4 : 2;
  const int hist_stride = ((nbins_max + qlp::kMPad + 31) / 32) * 32;
  const int smem_max = qlp::bls_max_smem_per_block();
  if (smem_max <= 0) return QLP_ERR_CUDA;
  const int budget = smem_max - 1024;
  int warps = p.warps_per_block ? std::min(p.warps_per_block, 16) : 8;  // as qlp_bls_plan: 32 is for cells
  auto hist_bytes = [&](int w) { return (size_t)w * NA * hist_stride * 4 + (size_t)w * qlp::kMaxQ * 4; };
  while (warps > 4 && hist_bytes(warps) > (size_t)budget / 2) warps /= 2;
  const size_t hb = (hist_bytes(warps) + 15) & ~(size_t)15;
  if (hb + 32 * 16 > (size_t)budget) return QLP_ERR_UNSUPPORTED;
  int tile = (int)(((size_t)budget - hb) / 16 / 32 * 32);
  tile = std::min<int64_t>(tile, npad);
  if (p.tile_points > 0) tile = std::min(tile, std::max(32, (p.tile_points / 32) * 32));
  const size_t smem = hb + (size_t)tile * 16;
  const int per_sm = qlp::bls_blocks_per_sm(p.phase_mode, sum_mode, warps, smem);
  if (per_sm < 1) return QLP_ERR_UNSUPPORTED;
  const int blocks = sms * per_sm;
  int chunk = p.chunk_freqs;
  if (chunk <= 0) {
    const int rounds = std::max(1, std::min(16, (int)std::floor((double)n_f / (8.0 * blocks * warps))));
    chunk = rounds * warps;
  }
  const int32_t n_items = (n_f + chunk - 1) / chunk;

  // scratch layout
  size_t off = 0;
  const size_t o_ctl = off; off = align256(off + 2 * sizeof(int32_t));
  const size_t o_star = off; off = align256(off + sizeof(qlp::StarDev));
  const size_t o_f = off; off = align256(off + sizeof(double) * (size_t)n_f);
  const size_t o_q = off; off = align256(off + sizeof(double) * (size_t)n_f);
  const size_t o_fq = off; off = align256(off + sizeof(double2) * (size_t)n_f);
  const size_t o_items = off; off = align256(off + sizeof(qlp::WorkItem) * (size_t)n_items);
  const size_t o_pts = off; off = align256(off + sizeof(float4) * (size_t)npad);
  const size_t o_tpd = off; off = align256(off + sizeof(double) * (size_t)npad);
  if (off > (size_t)QLP_STATIC_SCRATCH_BYTES) return QLP_ERR_ARG;

  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  unsigned char* sb = static_cast<unsigned char*>(base);
  int32_t* ctl = reinterpret_cast<int32_t*>(sb + o_ctl);
  qlp::StarDev* star = reinterpret_cast<qlp::StarDev*>(sb + o_star);
  double* f_d = reinterpret_cast<double*>(sb + o_f);
  double* q_d = reinterpret_cast<double*>(sb + o_q);
  double2* fq = reinterpret_cast<double2*>(sb + o_fq);
  qlp::WorkItem* items = reinterpret_cast<qlp::WorkItem*>(sb + o_items);
  float4* pts = reinterpret_cast<float4*>(sb + o_pts);
  double* tpd = reinterpret_cast<double*>(sb + o_tpd);

  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(f_d, freqs, sizeof(double) * (size_t)n_f, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(q_d, qmins, sizeof(double) * (size_t)n_f, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return QLP_ERR_CUDA;
  static_setup_kernel<<<64, 256, 0, st>>>(star, n, n_f, baseline, f_d, q_d, fq, items, n_items, chunk, ctl);
  if (cudaGetLastError() != cudaSuccess) return QLP_ERR_CUDA;

  qlp::PrepArgs pa{};
  pa.stars = star;
  pa.tp = tp;
  pa.y = y;
  pa.dy = dy;
  pa.pts = pts;
  pa.tpd = tpd;
  pa.tile_pts = tile;
  pa.n_stars = 1;
  if (qlp::launch_prep(pa, stream)) return QLP_ERR_CUDA;

  qlp::BlsArgs a{};
  a.stars = star;
  a.fq = fq;
  a.items = items;
  a.n_items = n_items;
  a.nq = nq;
  a.pts = pts;
  a.tpd = tpd;
  a.cursor = ctl;
  a.err = ctl + 1;
  a.sr = sr;
  a.qidx = qidx;
  a.kbin = phase_bin;
  a.sbest = s_best;
  a.rbest = r_best;
  a.noverlap = p.noverlap;
  for (int j = 0; j < qlp::kMaxQ; ++j) a.E[j] = j < nq ? std::exp(j * p.dlogq) : 0.0;
  a.tile_pts = tile;
  a.hist_stride = hist_stride;
  a.tile_off = (uint32_t)hb;
  const int phase = (ymax >= 4194304.0) ? QLP_PHASE_FP64 : p.phase_mode;
  if (qlp::launch_bls(a, phase, sum_mode, warps, blocks, smem, stream)) return QLP_ERR_CUDA;
  // the kernel's error bits (histogram guard, work-queue bound) for the caller
  if (flags && cudaMemcpyAsync(flags, ctl + 1, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return QLP_ERR_CUDA;
  return QLP_OK;
}
