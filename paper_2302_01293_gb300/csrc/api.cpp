// C-ABI entry points of libqlpbls (declared in include/qlp_bls.h): plan assembly,
// device buffers, work queue, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "planner.h"
#include "qlp_internal.h"

using namespace qlp;

namespace {

thread_local std::string g_cuda_err;

int cuda_fail(cudaError_t e, const char* what) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  g_cuda_err = buf;
  return QLP_ERR_CUDA;
}

#define QLP_CK(call)                                                    \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);                 \
  } while (0)

}  // namespace

// Records a CUDA failure for qlp_last_cuda_error (other translation units).
int qlp::record_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

namespace qlp {

// Device-memory budget of the library's own allocations (plans and networks): a cap
// on the bytes they hold at once, 0 = none. An allocation that would pass it fails
// before cudaMalloc is called, as an out-of-memory cudaMalloc would.
static std::atomic<int64_t> g_budget{0};
static std::atomic<int64_t> g_held{0};

bool budget_take(size_t bytes) {
  const int64_t cap = g_budget.load();
  int64_t cur = g_held.load();
  for (;;) {
    if (cap > 0 && cur + (int64_t)bytes > cap) return false;
    if (g_held.compare_exchange_weak(cur, cur + (int64_t)bytes)) return true;
  }
}

void budget_give(size_t bytes) { g_held.fetch_sub((int64_t)bytes); }

}  // namespace qlp

namespace {

// Host exceptions (allocation failures in the planner's containers) end at the C
// boundary as error codes.
template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return QLP_ERR_NOMEM;
  } catch (...) {
    return QLP_ERR_ARG;
  }
}

template <typename T>
int dev_alloc(T** p, size_t count, size_t* held) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (!budget_take(count * sizeof(T))) return QLP_ERR_NOMEM;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    budget_give(count * sizeof(T));
    cuda_fail(e, "cudaMalloc");
    return QLP_ERR_NOMEM;
  }
  *held = count * sizeof(T);
  return QLP_OK;
}

// One device allocation for a set of buffers (cheaper to make and to free than
// one per buffer); every buffer starts on a 256-byte boundary.
struct DevArena {
  struct Req {
    void** p;
    size_t bytes;
  };
  std::vector<Req> reqs;
  template <typename T>
  DevArena& add(T** p, size_t count) {
    reqs.push_back({reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T)});
    return *this;
  }
  int commit(void** base, size_t* held) {
    size_t total = 0;
    for (const Req& r : reqs) total += (r.bytes + 255) & ~(size_t)255;
    total = std::max<size_t>(total, 256);
    if (!budget_take(total)) return QLP_ERR_NOMEM;
    void* b = nullptr;
    const cudaError_t e = cudaMalloc(&b, total);
    if (e != cudaSuccess) {
      budget_give(total);
      cuda_fail(e, "cudaMalloc");
      return QLP_ERR_NOMEM;
    }
    *base = b;
    *held = total;
    size_t off = 0;
    for (const Req& r : reqs) {
      *r.p = static_cast<char*>(b) + off;
      off += (r.bytes + 255) & ~(size_t)255;
    }
    return QLP_OK;
  }
};

}  // namespace

struct qlp_bls_plan {
  qlp_bls_params p{};
  int32_t n_stars = 0;
  int32_t nq = 0;
  double E[kMaxQ] = {};
  // host copy
  std::vector<int32_t> status;
  std::vector<int64_t> f_off;     // n_stars + 1
  std::vector<double> freqs;      // all stars
  int64_t n_points = 0;       // valid points of the batch
  int64_t n_pts_alloc = 0;    // raw points: device point arrays (star s at its raw offset)
  double work = 0.0;              // sum N_s * n_f,s
  double work_points = 0.0;       // point-frequency pairs folded by the point path
  double work_cells = 0.0;        // point-frequency pairs served by the cell path
  double edges = 0.0;             // bin edges the cell path evaluates
  int32_t nbins_max = 0;
  // launch shape
  int warps = 8;
  int blocks = 0;
  int tile_pts = 0;
  int hist_stride = 0;
  uint32_t tile_off = 0;
  size_t smem = 0;
  int32_t n_items = 0;
  // cell path launch shape
  int c_warps = 8;
  int c_blocks = 0;
  size_t c_smem = 0;
  int32_t c_items = 0;
  int32_t n_cell_stars = 0;
  int32_t n_windowed = 0;
  // exact cell path launch shape
  int f_blocks = 0;
  size_t f_smem = 0;
  int32_t f_items = 0;
  int32_t f_whole = 0;            // the first f_whole of them on whole tables, the rest windowed
  int32_t n_fixed_stars = 0;
  int32_t fixed_max_pts = 0;
  bool fixed_windowed = false;    // some exact-path star is searched in time windows
  longlong2* d_ws = nullptr;      // exact-path bin-sum workspace, ws_block entries per block:
  int64_t ws_block = 1;           // a row of the largest bin count per warp (the exact rescoring of
                                  // each best box), or a windowed item's rows if larger
  int32_t fixed_nb_max = 0;       // largest bin count of an exact-path star
  double edges_fixed = 0.0;
  double bins_fixed = 0.0;       // sum of nbins over the exact path's frequencies
  int32_t n_narrow_stars = 0;    // of the exact path's stars, those on the 32-bit table
  double edges_narrow = 0.0, bins_narrow = 0.0;
  double times[4] = {};          // seconds: host grid, host staging, device allocation, upload
  // device
  StarDev* d_stars = nullptr;
  double2* d_fq = nullptr;
  WorkItem* d_items = nullptr;    // per-point items, then cell items
  double* d_tp = nullptr;
  double* d_y = nullptr;
  double* d_dy = nullptr;
  float4* d_pts = nullptr;
  double* d_tpd = nullptr;
  int32_t* d_cell_stars = nullptr;
  double2* d_cpre = nullptr;
  uint32_t* d_dt = nullptr;
  float2* d_loc = nullptr;
  float4* d_base = nullptr;
  int32_t* d_gidx = nullptr;
  int32_t* d_fixed_stars = nullptr;
  FixedStar* d_fx = nullptr;
  FreqRec* d_frec = nullptr;
  int32_t* d_ctl = nullptr;       // [0] per-point queue head, [1] cell queue head, [2] error flags,
                                  // [3] exact cell queue head (whole tables), [4] the same (windowed)
  // search + S/N captured as one CUDA graph (qlp_bls_graph_capture)
  // slot parts-1: parts = 1 search, 2 S/N, 3 both
  WinRec* d_wrec = nullptr;      // candidate statistics scratch (allocated on first use)
  int32_t* d_sorder = nullptr;   // and the statistics' launch order
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t kev[2] = {};        // qlp_bls_kernel_timing: around the main search kernel
  // recorded after the plan's last device work (control words, per-frequency
  // records): searches wait for it on their own stream, so building a plan does
  // not wait for kernels that occupy the GPU
  cudaEvent_t ready = nullptr;
  void* d_arena = nullptr;        // the one allocation holding the plan's buffers
  size_t arena_bytes = 0, wrec_bytes = 0, sorder_bytes = 0;  // device bytes held against the budget
  // owners of device memory: this plan's arena (freed, and its bytes given back, when
  // the last holder lets go) and, for a plan made from another one, that plan's
  // arena, which holds the points d_tp, d_y, d_dy this plan reads
  std::shared_ptr<void> arena_ref, points_ref;
  std::vector<StarPoints> pinfo;  // each star's point analysis (for plans made from this one)
  std::vector<int64_t> pt_off0;   // offsets of the stars' points, from 0
  bool ready_seen = false;        // the host has seen `ready` complete
  cudaGraph_t graph[3] = {};
  cudaGraphExec_t gexec[3] = {};
};

static void free_plan(qlp_bls_plan_t* pl) {
  if (!pl) return;
  if (pl->ready) {
    cudaEventSynchronize(pl->ready);
    cudaEventDestroy(pl->ready);
  }
  for (int i = 0; i < 3; ++i) {
    if (pl->gexec[i]) cudaGraphExecDestroy(pl->gexec[i]);
    if (pl->graph[i]) cudaGraphDestroy(pl->graph[i]);
  }
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  if (pl->kev[0]) cudaEventDestroy(pl->kev[0]);
  if (pl->kev[1]) cudaEventDestroy(pl->kev[1]);
  pl->arena_ref.reset();  // every buffer below but d_wrec and d_sorder lives in it
  pl->points_ref.reset();
  cudaFree(pl->d_wrec);
  cudaFree(pl->d_sorder);
  budget_give(pl->wrec_bytes + pl->sorder_bytes);
  delete pl;
}

extern "C" {

void qlp_bls_params_default(qlp_bls_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->samples_per_peak = 2.0;
  p->dlogq = 0.1;
  p->noverlap = 3.0;
  p->qmin_fac = 0.5;
  p->qmax_fac = 2.0;
  p->pmin_aR = 2.0;
  p->gap_days = 27.4;
  p->rho_default = 1.41;
  p->nbins_cap = 8192;
  p->phase_mode = QLP_PHASE_DF;
  p->sum_mode = QLP_SUM_FIXED;
  p->mad_mode = QLP_MAD_RAW;
  p->chunk_freqs = 0;
  p->warps_per_block = 0;
  p->n_threads = 0;
  p->method = 0;
  p->grid_mode = 0;
  p->coarse_bins = 4096;
  p->cell_window = 0;
  p->coarse_pmin = 0.1;
  p->coarse_pmax = 400.0;
  p->bin_mode = QLP_BIN_SHARED;
  p->work_loop_bound = 0;
}

const char* qlp_strerror(int code) {
  switch (code) {
    case QLP_OK: return "ok";
    case QLP_ERR_ARG: return "invalid argument";
    case QLP_ERR_CUDA: return "CUDA runtime error";
    case QLP_ERR_NOMEM: return "out of memory";
    case QLP_ERR_DEVICE: return "device-side bound hit";
    case QLP_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown error";
  }
}

const char* qlp_last_cuda_error(void) { return g_cuda_err.c_str(); }

static int check_params(const qlp_bls_params& p) {
  if (!(p.samples_per_peak > 0) || !(p.dlogq > 0) || !(p.noverlap >= 1) || !(p.qmin_fac > 0) ||
      !(p.qmax_fac >= p.qmin_fac) || !(p.pmin_aR > 0) || !(p.gap_days > 0) || !(p.rho_default > 0) ||
      p.nbins_cap < 2)
    return QLP_ERR_ARG;
  if (p.phase_mode < 0 || p.phase_mode > 2 || p.sum_mode < 0 || p.sum_mode > 3 || p.mad_mode < 0 ||
      p.mad_mode > 1 || p.tile_points < 0 || p.chunk_freqs < 0 || p.method < 0 || p.method > 2 ||
      p.grid_mode < 0 || p.grid_mode > 1 || p.cell_window < 0 || p.bin_mode < 0 || p.bin_mode > 1 ||
      p.work_loop_bound < 0 ||
      (p.bin_mode == QLP_BIN_PER_Q && (p.noverlap != std::floor(p.noverlap) || p.phase_mode == QLP_PHASE_FP32 ||
                                       p.method == 1)) ||
      (p.grid_mode == 1 && (p.coarse_bins < 2 || !(p.coarse_pmin > 0) || !(p.coarse_pmax > p.coarse_pmin))))
    return QLP_ERR_ARG;
  if (p.warps_per_block != 0 && p.warps_per_block != 4 && p.warps_per_block != 8 &&
      p.warps_per_block != 16 && p.warps_per_block != 32)
    return QLP_ERR_ARG;
  const int nq = n_q_of(p);
  if (nq < 1 || nq > kMaxQ) return QLP_ERR_UNSUPPORTED;
  // widest window: q_min e^{(nq-1) dlogq} nbins + 1/2 with q_min nbins < noverlap + 1
  const double mmax = (p.noverlap + 1.0) * std::exp((nq - 1) * p.dlogq) + 0.5;
  if (mmax >= (double)kMPad) return QLP_ERR_UNSUPPORTED;
  return QLP_OK;
}

// Arguments of the exact cell path's preparation kernels.
static PrepFixedArgs fixed_args(const qlp_bls_plan_t* pl) {
  PrepFixedArgs pf{};
  pf.stars = pl->d_stars;
  pf.fixed_stars = pl->d_fixed_stars;
  pf.n = pl->n_fixed_stars;
  pf.nq = pl->nq;
  pf.tp = pl->d_tp;
  pf.y = pl->d_y;
  pf.dy = pl->d_dy;
  pf.fq = pl->d_fq;
  pf.ipre = reinterpret_cast<longlong2*>(pl->d_cpre);
  pf.dt = pl->d_dt;
  pf.loc = reinterpret_cast<int2*>(pl->d_loc);
  pf.base = reinterpret_cast<longlong2*>(pl->d_base);
  pf.gidx = pl->d_gidx;
  pf.fx = pl->d_fx;
  pf.frec = pl->d_frec;
  pf.noverlap = pl->p.noverlap;
  for (int j = 0; j < kMaxQ; ++j) pf.E[j] = pl->E[j];
  pf.nb_cap = pl->p.nbins_cap;
  pf.max_pts = pl->fixed_max_pts;
  pf.err = pl->d_ctl + 2;
  return pf;
}

static int plan_impl(const qlp_bls_params* pin, int32_t n_stars, const int64_t* offsets, const double* t,
                     const double* y, const double* dy, const double* rho, const double* rstar,
                     const int64_t* win_off, const double* win_lo, const double* win_hi, void* stream,
                     qlp_bls_plan_t** out_plan, const qlp_bls_plan_t* from = nullptr);

int qlp_bls_plan(const qlp_bls_params* pin, int32_t n_stars, const int64_t* offsets, const double* t,
                 const double* y, const double* dy, const double* rho, const double* rstar,
                 void* stream, qlp_bls_plan_t** out_plan) {
  if (out_plan) *out_plan = nullptr;
  return guarded([&] {
    return plan_impl(pin, n_stars, offsets, t, y, dy, rho, rstar, nullptr, nullptr, nullptr, stream, out_plan);
  });
}

int qlp_bls_plan_windows(const qlp_bls_params* pin, int32_t n_stars, const int64_t* offsets,
                         const double* t, const double* y, const double* dy, const double* rho,
                         const double* rstar, const int64_t* win_offsets, const double* win_flo,
                         const double* win_fhi, void* stream, qlp_bls_plan_t** out_plan) {
  if (!win_offsets || (n_stars > 0 && win_offsets[n_stars] > 0 && (!win_flo || !win_fhi)))
    return QLP_ERR_ARG;
  for (int32_t s = 0; s < n_stars; ++s)
    if (win_offsets[s + 1] < win_offsets[s]) return QLP_ERR_ARG;
  qlp_bls_params p;
  if (pin) p = *pin; else qlp_bls_params_default(&p);
  if (p.grid_mode != 0) return QLP_ERR_ARG;
  if (out_plan) *out_plan = nullptr;
  return guarded([&] {
    return plan_impl(&p, n_stars, offsets, t, y, dy, rho, rstar, win_offsets, win_flo, win_fhi, stream, out_plan);
  });
}

int qlp_bls_plan_windows_from(const qlp_bls_plan_t* base, const qlp_bls_params* pin,
                              const int64_t* win_offsets, const double* win_flo, const double* win_fhi,
                              void* stream, qlp_bls_plan_t** out_plan) {
  if (out_plan) *out_plan = nullptr;
  if (!base || !win_offsets) return QLP_ERR_ARG;
  const int32_t n_stars = base->n_stars;
  if (n_stars > 0 && win_offsets[n_stars] > 0 && (!win_flo || !win_fhi)) return QLP_ERR_ARG;
  for (int32_t s = 0; s < n_stars; ++s)
    if (win_offsets[s + 1] < win_offsets[s]) return QLP_ERR_ARG;
  qlp_bls_params p;
  if (pin) p = *pin; else qlp_bls_params_default(&p);
  if (p.grid_mode != 0) return QLP_ERR_ARG;
  // the point analysis depends on these: they must be the base plan's
  if (!(p.rho_default == base->p.rho_default) || !(p.pmin_aR == base->p.pmin_aR) ||
      !(p.gap_days == base->p.gap_days))
    return QLP_ERR_ARG;
  return guarded([&] {
    return plan_impl(&p, n_stars, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, win_offsets, win_flo,
                     win_fhi, stream, out_plan, base);
  });
}

static int plan_impl(const qlp_bls_params* pin, int32_t n_stars, const int64_t* offsets, const double* t,
                     const double* y, const double* dy, const double* rho, const double* rstar,
                     const int64_t* win_off, const double* win_lo, const double* win_hi, void* stream,
                     qlp_bls_plan_t** out_plan, const qlp_bls_plan_t* from) {
  (void)rstar;
  if (!out_plan) return QLP_ERR_ARG;
  *out_plan = nullptr;
  qlp_bls_params p;
  if (pin) p = *pin; else qlp_bls_params_default(&p);
  int rc = check_params(p);
  if (rc) return rc;
  if (from) {  // the stars and points of `from`: its offsets and point analysis
    if (n_stars != from->n_stars) return QLP_ERR_ARG;
    offsets = from->pt_off0.data();
  }
  if (n_stars < 0 || (n_stars > 0 && !offsets)) return QLP_ERR_ARG;
  if (n_stars > 0 && !from) {
    if (offsets[0] != 0) return QLP_ERR_ARG;
    for (int32_t s = 0; s < n_stars; ++s)
      if (offsets[s + 1] < offsets[s]) return QLP_ERR_ARG;
    if (offsets[n_stars] > 0 && (!t || !y || !dy)) return QLP_ERR_ARG;
  }

  using clk = std::chrono::steady_clock;
  const auto c0 = clk::now();
  // the valid points go straight into the upload arrays, each star at its raw
  // offset (a star's entries past its valid count are zero and never read)
  const int64_t npt_raw = n_stars > 0 ? offsets[n_stars] - offsets[0] : 0;
  const size_t npt_alloc = (size_t)std::max<int64_t>(npt_raw, 1);
  std::unique_ptr<double[]> tp_all, y_all, dy_all;
  std::vector<StarPlanHost> sp;
  std::vector<StarPoints> pinfo;
  if (from) {  // the grids only: the points were validated, analysed and uploaded by `from`
    plan_all_from(p, n_stars, from->pinfo.data(), &sp, win_off, win_lo, win_hi);
    pinfo = from->pinfo;
  } else {
    tp_all.reset(new (std::nothrow) double[npt_alloc]);
    y_all.reset(new (std::nothrow) double[npt_alloc]);
    dy_all.reset(new (std::nothrow) double[npt_alloc]);
    if (!tp_all || !y_all || !dy_all) return QLP_ERR_NOMEM;
    PointDst pdst;
    pdst.tp = tp_all.get();
    pdst.y = y_all.get();
    pdst.dy = dy_all.get();
    plan_all(p, n_stars, offsets, t, y, dy, rho, &sp, win_off, win_lo, win_hi, &pdst);
    pinfo.resize((size_t)n_stars);
    parallel_stars(p, n_stars, [&](int32_t s) { pinfo[(size_t)s] = points_of(sp[(size_t)s]); });
  }
  const auto c1 = clk::now();

  qlp_bls_plan_t* pl = new (std::nothrow) qlp_bls_plan_t();
  if (!pl) return QLP_ERR_NOMEM;
  pl->pinfo = std::move(pinfo);
  pl->pt_off0.resize((size_t)n_stars + 1, 0);
  for (int32_t s = 0; s <= n_stars; ++s) pl->pt_off0[(size_t)s] = n_stars > 0 ? offsets[s] - offsets[0] : 0;
  pl->times[0] = std::chrono::duration<double>(c1 - c0).count();
  pl->p = p;
  pl->n_stars = n_stars;
  pl->n_pts_alloc = npt_raw;
  pl->nq = n_q_of(p);
  for (int j = 0; j < pl->nq; ++j) pl->E[j] = std::exp(j * p.dlogq);

  // the per-point and windowed cell kernels run compensated sums under QLP_SUM_FIXED
  const int sum_old = p.sum_mode == QLP_SUM_PLAIN ? QLP_SUM_PLAIN : QLP_SUM_COMP;
  const int NA = (sum_old == QLP_SUM_COMP) ? 4 : 2;
  const int smem_max = bls_max_smem_per_block();
  if (smem_max <= 0) { delete pl; return cuda_fail(cudaGetLastError(), "device query"); }
  const int budget = smem_max - 1024;
  auto round32 = [](int64_t x) { return ((x + 31) / 32) * 32; };
  auto align16 = [](size_t x) { return (x + 15) & ~(size_t)15; };

  // method per star: the cell path needs one point per cell, its table and
  // histograms in shared memory, and fewer bin edges than point-frequency pairs
  const int cw = p.warps_per_block ? p.warps_per_block : 32;
  // the table plus at least one warp's histogram for the star's largest bin count
  auto cell_smem = [&](int64_t cells, int nbmax) {
    return (size_t)cells_hist_offset((int)cells, cw) + (size_t)NA * (size_t)round32(nbmax + kMPad) * 4;
  };
  // A table longer than shared memory is cut into windows of win_cells cells;
  // window w owns the cells from w win_cells and stages from the 32-aligned cell
  // below its start to win_ovl cells past its end (one bin duration plus the
  // cells an edge and the point after it can reach).
  struct CellWin {
    int32_t n_win = 1, cells = 0, ovl = 0, cap = 0;
  };
  std::vector<int32_t> method((size_t)n_stars, kMethodPoints);
  std::vector<CellWin> cwin((size_t)n_stars);
  for (int32_t s = 0; s < n_stars; ++s) {
    const StarPlanHost& h = sp[(size_t)s];
    if (h.status != 0 || !h.cells_ok || p.method == 1 || p.phase_mode == QLP_PHASE_FP32) continue;
    CellWin& W = cwin[(size_t)s];
    const double ovl = std::ceil(h.bin_dmax / h.cell_h) + 4.0;
    // the edge step D/h must stay below 2^8 cells: the compensated kernel holds it
    // in 8.56 fixed point, the exact one in 24.40 (32.32 for whole tables)
    if (!(ovl < 1.0e6) || !(h.bin_dmax / h.cell_h < 255.0)) continue;
    W.ovl = (int32_t)ovl;
    const bool whole = p.cell_window > 0 ? p.cell_window >= h.n_cells
                                          : cell_smem(h.n_cells + 1, h.nbins_max) <= (size_t)budget;
    if (whole) {
      W.cells = (int32_t)h.n_cells;
      W.cap = (int32_t)h.n_cells + 1;
    } else {
      int64_t c = p.cell_window;
      if (c <= 0) {  // the largest multiple of 32 whose staged window fills at most half the budget
        c = 32;
        while (cells_hist_offset((int)(c + 32 + W.ovl + 33), cw) <= (size_t)budget / 2) c += 32;
      }
      W.cells = (int32_t)c;
      W.cap = (int32_t)std::min<int64_t>(h.n_cells + 1, c + W.ovl + 33);
      W.n_win = (int32_t)((h.n_cells + c - 1) / c);
    }
    const bool old_fits = cell_smem(W.cap, h.nbins_max) <= (size_t)budget;
    const double pp_work = (double)h.freqs.size() * (double)round32(h.n_valid);
    // exact path: at least 32 bins, at most 2^14 cycles and 2^21 points (the integer
    // prefix sums stay below 2^62), no weight or weighted residual above 256 times
    // the star's mean (the integer scale follows the largest one: a single extreme
    // point would coarsen every other point's weight); the whole table and the
    // warps' rings in shared memory, or else windows of the table (bin sums through
    // a global workspace)
    const bool fixed_ok = (p.sum_mode == QLP_SUM_FIXED || p.sum_mode == QLP_SUM_FIXED64) &&
                          p.bin_mode == QLP_BIN_SHARED && h.nbins_min >= 32 &&
                          h.w_spread <= 256.0 && h.wd_spread <= 256.0 &&
                          h.baseline * h.freqs.back() <= 16384.0 && h.n_valid <= ((int64_t)1 << 21) &&
                          (size_t)32 * 16 * ((h.nbins_max + 31) / 32) <= (size_t)kFixedWsBlock * 16;
    if (fixed_ok && (p.method == 2 || h.cells_work < 2.0 * pp_work)) {
      const bool fwhole = p.cell_window > 0 ? p.cell_window >= h.n_cells
                                            : (size_t)fixed_smem_bytes((int)h.n_cells + 1) <= (size_t)budget;
      CellWin F{1, (int32_t)h.n_cells, (int32_t)ovl, (int32_t)h.n_cells + 1};
      if (!fwhole) {
        int64_t c = p.cell_window;
        if (c <= 0) {  // the largest multiple of 32 whose staged window fits
          c = 32;
          while (fixed_window_smem_bytes((int)(c + 32 + F.ovl + 34)) <= (size_t)budget) c += 32;
        }
        F.cells = (int32_t)c;
        F.cap = (int32_t)std::min<int64_t>(h.n_cells + 1, c + F.ovl + 33);
        F.n_win = (int32_t)((h.n_cells + c - 1) / c);
      }
      if ((size_t)(F.n_win > 1 ? fixed_window_smem_bytes(F.cap + 1) : fixed_smem_bytes(F.cap + 1)) <= (size_t)budget) {
        method[(size_t)s] = kMethodFixed;
        W = F;
        continue;
      }
    }
    if (!old_fits) continue;
    if (p.method == 2 || p.bin_mode == QLP_BIN_PER_Q || h.cells_work < pp_work) method[(size_t)s] = kMethodCells;
  }
  // the per-point kernel holds NA histogram arrays of round32(nbins + kMPad) floats per
  // warp in shared memory, at least 4 warps and one 32-point tile beside them: a star
  // left on that path with more bins than they hold is flagged, not searched
  {
    const int64_t rows = ((int64_t)budget - 32 * 16 - 4 * kMaxQ * 4) / (4LL * NA * 4);
    const int32_t pp_nb_cap = (int32_t)(rows / 32 * 32) - kMPad;
    for (int32_t s = 0; s < n_stars; ++s)
      if (sp[(size_t)s].status == 0 && method[(size_t)s] == kMethodPoints && sp[(size_t)s].nbins_max > pp_nb_cap)
        sp[(size_t)s].status |= QLP_STAR_NBINS_CAP;
  }
  if (p.bin_mode == QLP_BIN_PER_Q)  // per-duration histograms exist on the cell path only
    for (int32_t s = 0; s < n_stars; ++s)
      if (sp[(size_t)s].status == 0 && method[(size_t)s] != kMethodCells) sp[(size_t)s].status = QLP_STAR_UNSUPPORTED;

  // flat host arrays
  std::vector<StarDev> stars((size_t)n_stars);
  pl->status.resize((size_t)n_stars);
  pl->f_off.assign((size_t)n_stars + 1, 0);
  int64_t npt = 0, npad = 0, nf = 0, ncell = 0, nbase = 0, ncpre = 0;
  int32_t max_npts = 0, nb_pp = 0, nb_c = 0;
  int64_t cells_cap = 0;
  std::vector<int32_t> cell_stars, fixed_stars;
  int64_t fixed_ncs = 0;   // cells (with the sentinel) of the largest whole table
  size_t fixed_wsmem = 0;  // shared memory of the largest time window
  for (int32_t s = 0; s < n_stars; ++s) {
    const StarPlanHost& h = sp[(size_t)s];
    StarDev& d = stars[(size_t)s];
    std::memset(&d, 0, sizeof(d));
    const bool ok = h.status == 0;
    d.pt_off = offsets[s] - offsets[0];
    d.pad_off = npad;
    d.f_off = nf;
    d.n_pts = ok ? (int32_t)h.n_valid : 0;
    d.n_f = ok ? (int32_t)h.freqs.size() : 0;
    d.status = h.status;
    d.sturges_nb = h.sturges_nb;
    d.fp64_phase = (h.ymax >= 4194304.0) ? 1 : 0;   // 2^22: beyond the FP32 remainder range
    d.method = method[(size_t)s];
    d.t_ref = h.t_ref;
    d.baseline = h.baseline;
    d.grid_k0 = h.grid_k0;
    pl->status[(size_t)s] = h.status;
    npt += d.n_pts;
    nf += d.n_f;
    pl->f_off[(size_t)s + 1] = nf;
    if (ok) pl->work += (double)d.n_pts * (double)d.n_f;
    if (ok && (d.method == kMethodCells || d.method == kMethodFixed)) {
      pl->work_cells += (double)d.n_pts * (double)d.n_f;
      pl->edges += h.cells_work;
      d.h = h.cell_h;
      d.n_cells = (int32_t)h.n_cells;
      d.n_win = cwin[(size_t)s].n_win;
      d.win_cells = cwin[(size_t)s].cells;
      d.win_ovl = cwin[(size_t)s].ovl;
      d.win_cap = cwin[(size_t)s].cap;
      // the 32-bit exact table: whole table, at most 2^16 points (the w scale F leaves
      // 2^17 for the roundings), the running sum of w d within 64 times the largest
      // |w d|, so that its y scale (2^-30 of the running sum's range) is at most 4 times
      // coarser than the 64-bit table's (2^-25 of the largest |w d|); a white-noise star
      // of N points reaches about sqrt(N) / 4 of it
      d.narrow = (d.method == kMethodFixed && d.n_win <= 1 && p.sum_mode == QLP_SUM_FIXED &&
                  h.n_valid <= 65536 && h.y_exc > 0.0 && h.y_exc <= 64.0 * h.wd_max)
                     ? 1
                     : 0;
      d.y_exc = h.y_exc;
      if (d.n_win > 1) pl->n_windowed++;
      d.cell_off = ncell;
      d.base_off = nbase;
      d.cpre_off = ncpre;
      ncell += (h.n_cells + 1 + 3) & ~3;  // every star's table starts at a 16-byte boundary
      nbase += (h.n_cells + 1 + 31) / 32;
      ncpre += d.n_pts + 1;
      if (d.method == kMethodFixed) {
        fixed_stars.push_back(s);
        pl->fixed_max_pts = std::max(pl->fixed_max_pts, d.n_pts);
        if (d.n_win > 1)
          fixed_wsmem = std::max<size_t>(fixed_wsmem, fixed_window_smem_bytes(d.win_cap + 1));
        else
          fixed_ncs = std::max<int64_t>(fixed_ncs, h.n_cells + 1);
        if (d.n_win > 1) pl->fixed_windowed = true;
        pl->fixed_nb_max = std::max(pl->fixed_nb_max, h.nbins_max);
        pl->edges_fixed += h.cells_work;
        pl->bins_fixed += h.nbins_sum;
        if (d.narrow) {
          pl->n_narrow_stars++;
          pl->edges_narrow += h.cells_work;
          pl->bins_narrow += h.nbins_sum;
        }
      } else {
        cells_cap = std::max<int64_t>(cells_cap, h.n_cells + 1);
        nb_c = std::max(nb_c, h.nbins_max);
        cell_stars.push_back(s);
      }
    } else if (ok) {
      pl->work_points += (double)d.n_pts * (double)d.n_f;
      npad += ((int64_t)d.n_pts + 31) & ~(int64_t)31;
      max_npts = std::max(max_npts, d.n_pts);
      nb_pp = std::max(nb_pp, h.nbins_max);
    }
    if (ok) pl->nbins_max = std::max(pl->nbins_max, h.nbins_max);
  }
  pl->n_points = npt;
  pl->n_cell_stars = (int32_t)(cell_stars.size() + fixed_stars.size());
  pl->n_fixed_stars = (int32_t)fixed_stars.size();
  // frequency staging without zero fill, filled star by star in parallel
  const size_t nf_alloc = (size_t)std::max<int64_t>(nf, 1);
  std::unique_ptr<double2[]> fq(new (std::nothrow) double2[nf_alloc]);
  if (!fq) { delete pl; return QLP_ERR_NOMEM; }
  pl->freqs.resize((size_t)nf);
  parallel_stars(p, n_stars, [&](int32_t s) {
    const StarPlanHost& h = sp[(size_t)s];
    const StarDev& d = stars[(size_t)s];
    for (int32_t k = 0; k < d.n_f; ++k) {
      fq[(size_t)(d.f_off + k)] = make_double2(h.freqs[(size_t)k], h.qmins[(size_t)k]);
      pl->freqs[(size_t)(d.f_off + k)] = h.freqs[(size_t)k];
    }
  });

  int dev = 0, sms = 0;
  QLP_CK(cudaGetDevice(&dev));
  QLP_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  // per-point launch shape: histograms per warp, then the largest point tile that fits
  pl->hist_stride = (int)round32(std::max(nb_pp, 1) + kMPad);
  int warps = p.warps_per_block ? std::min(p.warps_per_block, 16) : 8;
  auto hist_bytes = [&](int w) { return (size_t)w * NA * pl->hist_stride * 4 + (size_t)w * kMaxQ * 4; };
  while (warps > 4 && hist_bytes(warps) > (size_t)budget / 2) warps /= 2;
  const size_t hb = align16(hist_bytes(warps));
  if (hb + 32 * 16 > (size_t)budget) { delete pl; return QLP_ERR_UNSUPPORTED; }
  int tile = (int)(((size_t)budget - hb) / 16 / 32 * 32);
  tile = std::min<int>(tile, (int)round32(std::max(max_npts, 1)));
  if (p.tile_points > 0) tile = std::min(tile, std::max(32, (p.tile_points / 32) * 32));
  pl->warps = warps;
  pl->tile_pts = tile;
  pl->tile_off = (uint32_t)hb;
  pl->smem = hb + (size_t)tile * 16;
  int per_sm = bls_blocks_per_sm(p.phase_mode, sum_old, warps, pl->smem);
  if (per_sm < 1) { delete pl; return QLP_ERR_UNSUPPORTED; }
  pl->blocks = sms * per_sm;

  // cell launch shape: the whole shared-memory budget; each work item gets the
  // histogram stride of its own largest bin count and as many warps as fit
  (void)cells_cap;
  (void)nb_c;
  if (!cell_stars.empty()) {
    pl->c_warps = cw;
    pl->c_smem = (size_t)budget;
    const int cper = cells_blocks_per_sm(sum_old, cw, pl->c_smem);
    if (cper < 1) { delete pl; return QLP_ERR_UNSUPPORTED; }
    pl->c_blocks = sms * cper;
  }
  if (!fixed_stars.empty()) {
    pl->f_smem = std::max<size_t>(fixed_ncs > 0 ? fixed_smem_bytes((int)fixed_ncs) : 0, fixed_wsmem);
    const int fper = fixed_blocks_per_sm(pl->f_smem);
    if (fper < 1) { delete pl; return QLP_ERR_UNSUPPORTED; }
    pl->f_blocks = sms * fper;
  }

  // exact-path workspace per block: one row of the largest bin count per warp (the
  // whole-table stars' bin sums), or the largest rows of a windowed item (its bins per
  // frequency), whichever is larger (set below, once the items are cut)
  int64_t win_rows_max = 0;

  // work items: (star, chunk of frequencies), longest first, one queue per path
  auto make_items = [&](int32_t meth, int w, int blocks, std::vector<WorkItem>* outv) {
    int64_t nf_m = 0;
    for (int32_t s = 0; s < n_stars; ++s)
      if (stars[(size_t)s].method == meth) nf_m += stars[(size_t)s].n_f;
    int chunk = p.chunk_freqs;
    if (chunk <= 0) {
      int rounds = (int)std::floor((double)nf_m / (8.0 * std::max(blocks, 1) * w));
      rounds = std::max(1, std::min(rounds, 16));
      chunk = rounds * w;
    }
    std::vector<WorkItem> items;
    std::vector<double> cost;
    for (int32_t s = 0; s < n_stars; ++s) {
      const StarDev& d = stars[(size_t)s];
      if (d.method != meth) continue;
      const StarPlanHost& h = sp[(size_t)s];
      int ck = chunk;
      int32_t ws_stride = 0;
      if (meth == kMethodFixed && d.n_win > 1) {  // rows of round32(nbins) bins in the block's workspace
        // long items: every item stages all of its star's windows once, so the fewer
        // items the less staging; at most kFixedWinRows entries per block
        ws_stride = (int32_t)round32(h.nbins_max);
        ck = std::max(1, std::min(ck, (int)(kFixedWinRows / ws_stride)));
        win_rows_max = std::max<int64_t>(win_rows_max, (int64_t)std::min(ck, d.n_f) * ws_stride);
      }
      for (int32_t b = 0; b < d.n_f; b += ck) {
        WorkItem wi{};
        wi.star = s;
        wi.f_begin = b;
        wi.f_count = std::min(ck, d.n_f - b);
        if (meth == kMethodFixed) wi.pad0 = ws_stride;
        if (meth == kMethodCells) {
          int nbm = 1;
          for (int32_t k = b; k < b + wi.f_count; ++k) nbm = std::max(nbm, h.nbins[(size_t)k]);
          const int hs32 = (int)(round32(nbm + kMPad) / 32);
          const size_t avail = (size_t)budget - cells_hist_offset(d.win_cap, cw);
          const int wact = (int)std::min<size_t>((size_t)cw, avail / ((size_t)NA * hs32 * 32 * 4));
          wi.pad0 = hs32 | (std::max(wact, 1) << 16);
        }
        items.push_back(wi);
        const int mid = b + wi.f_count / 2;
        const double nbm = (double)h.nbins[(size_t)mid];
        const double per_f = meth != kMethodPoints ? h.baseline * h.freqs[(size_t)mid] * nbm + 3.0 * nbm
                                                   : (double)d.n_pts + 3.0 * nbm;
        cost.push_back((double)wi.f_count * per_f);
      }
    }
    std::vector<int32_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return cost[(size_t)a] > cost[(size_t)b]; });
    for (size_t i = 0; i < order.size(); ++i) outv->push_back(items[(size_t)order[i]]);
    return (int32_t)order.size();
  };
  std::vector<WorkItem> sorted;
  pl->n_items = make_items(kMethodPoints, warps, pl->blocks, &sorted);
  pl->c_items = make_items(kMethodCells, cw, pl->c_blocks, &sorted);
  pl->f_items = make_items(kMethodFixed, kFixedWarps, pl->f_blocks, &sorted);
  {  // whole-table items first, then the windowed ones (separate launches), each longest first
    const auto fb = sorted.end() - pl->f_items;
    const auto mid = std::stable_partition(
        fb, sorted.end(), [&](const WorkItem& w) { return stars[(size_t)w.star].n_win <= 1; });
    pl->f_whole = (int32_t)(mid - fb);
  }
  if (!fixed_stars.empty())
    pl->ws_block = std::max<int64_t>((int64_t)kFixedWarps * (round32(pl->fixed_nb_max) + kFixedPendRows),
                                     win_rows_max);

  // device buffers
  const auto c2 = clk::now();
  pl->times[1] = std::chrono::duration<double>(c2 - c1).count();
  cudaStream_t st = (cudaStream_t)stream;
  DevArena arena;
  arena.add(&pl->d_stars, (size_t)n_stars)
      .add(&pl->d_fq, nf_alloc)
      .add(&pl->d_items, sorted.size())
      .add(&pl->d_tp, from ? (size_t)1 : npt_alloc)
      .add(&pl->d_y, from ? (size_t)1 : npt_alloc)
      .add(&pl->d_dy, from ? (size_t)1 : npt_alloc)
      .add(&pl->d_pts, (size_t)npad)
      .add(&pl->d_tpd, (size_t)npad)
      .add(&pl->d_cell_stars, cell_stars.size())
      .add(&pl->d_cpre, (size_t)ncpre)
      .add(&pl->d_dt, (size_t)ncell)
      .add(&pl->d_loc, (size_t)ncell)
      .add(&pl->d_gidx, (size_t)ncell)
      .add(&pl->d_base, (size_t)nbase)
      .add(&pl->d_fixed_stars, fixed_stars.size())
      .add(&pl->d_fx, (size_t)n_stars)
      .add(&pl->d_frec, fixed_stars.empty() ? (size_t)1 : nf_alloc)
      .add(&pl->d_ws, fixed_stars.empty() ? (size_t)1 : (size_t)pl->f_blocks * (size_t)pl->ws_block)
      .add(&pl->d_ctl, 5);
  if ((rc = arena.commit(&pl->d_arena, &pl->arena_bytes))) {
    free_plan(pl);
    return rc;
  }
  {
    const size_t ab = pl->arena_bytes;
    pl->arena_ref = std::shared_ptr<void>(pl->d_arena, [ab](void* b) {
      cudaFree(b);
      budget_give(ab);
    });
  }
  if (from) {  // the points stay in `from`'s arena, held as long as this plan lives
    pl->d_tp = from->d_tp;
    pl->d_y = from->d_y;
    pl->d_dy = from->d_dy;
    pl->points_ref = from->points_ref ? from->points_ref : from->arena_ref;
  }
  const auto c3 = clk::now();
  pl->times[2] = std::chrono::duration<double>(c3 - c2).count();
  cudaError_t e = cudaSuccess;
  if (n_stars > 0) e = cudaMemcpyAsync(pl->d_stars, stars.data(), sizeof(StarDev) * (size_t)n_stars, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nf > 0) e = cudaMemcpyAsync(pl->d_fq, fq.get(), sizeof(double2) * (size_t)nf, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !sorted.empty()) e = cudaMemcpyAsync(pl->d_items, sorted.data(), sizeof(WorkItem) * sorted.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !cell_stars.empty()) e = cudaMemcpyAsync(pl->d_cell_stars, cell_stars.data(), sizeof(int32_t) * cell_stars.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !fixed_stars.empty()) e = cudaMemcpyAsync(pl->d_fixed_stars, fixed_stars.data(), sizeof(int32_t) * fixed_stars.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && npt_raw > 0 && !from) e = cudaMemcpyAsync(pl->d_tp, tp_all.get(), sizeof(double) * (size_t)npt_raw, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && npt_raw > 0 && !from) e = cudaMemcpyAsync(pl->d_y, y_all.get(), sizeof(double) * (size_t)npt_raw, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && npt_raw > 0 && !from) e = cudaMemcpyAsync(pl->d_dy, dy_all.get(), sizeof(double) * (size_t)npt_raw, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host staging arrays die at return
  // the rest runs on the device after the uploads without the host waiting for it
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_ctl, 0, 5 * sizeof(int32_t), st);
  if (e == cudaSuccess && !fixed_stars.empty()) {  // per-frequency records of the exact path
    const int le = launch_freq_recs(fixed_args(pl), stream);
    if (le) e = (cudaError_t)le;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(pl->ready, st);
  if (e != cudaSuccess) {
    free_plan(pl);
    return cuda_fail(e, "plan upload");
  }
  pl->times[3] = std::chrono::duration<double>(clk::now() - c3).count();
  *out_plan = pl;
  return QLP_OK;
}

int qlp_bls_plan_info(const qlp_bls_plan_t* pl, int64_t* n_freq_total, int64_t* freq_offsets,
                      double* freqs, int32_t* star_status, int64_t* n_points, double* work) {
  if (!pl) return QLP_ERR_ARG;
  if (n_freq_total) *n_freq_total = pl->f_off.back();
  if (freq_offsets) std::memcpy(freq_offsets, pl->f_off.data(), sizeof(int64_t) * pl->f_off.size());
  if (freqs && !pl->freqs.empty()) std::memcpy(freqs, pl->freqs.data(), sizeof(double) * pl->freqs.size());
  if (star_status && !pl->status.empty()) std::memcpy(star_status, pl->status.data(), sizeof(int32_t) * pl->status.size());
  if (n_points) *n_points = pl->n_points;
  if (work) *work = pl->work;
  return QLP_OK;
}

int qlp_bls_plan_stats(const qlp_bls_plan_t* pl, double* work_points, double* work_cells,
                       double* edges, int32_t* n_cell_stars, int32_t* n_windowed) {
  if (!pl) return QLP_ERR_ARG;
  if (n_windowed) *n_windowed = pl->n_windowed;
  if (work_points) *work_points = pl->work_points;
  if (work_cells) *work_cells = pl->work_cells;
  if (edges) *edges = pl->edges;
  if (n_cell_stars) *n_cell_stars = pl->n_cell_stars;
  return QLP_OK;
}

// Records a timing event of the main search kernel; inside a stream capture the
// record becomes an event node of the graph.
static cudaError_t record_kev(qlp_bls_plan_t* pl, int i, cudaStream_t st) {
  if (!pl->kev[i]) return cudaSuccess;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(pl->kev[i], st, cudaEventRecordExternal)
                                             : cudaEventRecord(pl->kev[i], st);
}

// The kernel the timing events bracket: the exact cell kernel when it has work,
// else the compensated cell kernel, else the per-point kernel.
static int timed_kernel(const qlp_bls_plan_t* pl) {
  return pl->f_items > 0 ? kMethodFixed : pl->c_items > 0 ? kMethodCells : kMethodPoints;
}

int qlp_bls_kernel_timing(qlp_bls_plan_t* pl, int32_t enable) {
  if (!pl) return QLP_ERR_ARG;
  for (int i = 0; i < 2; ++i) {
    if (enable && !pl->kev[i]) QLP_CK(cudaEventCreate(&pl->kev[i]));
    if (!enable && pl->kev[i]) {
      cudaEventDestroy(pl->kev[i]);
      pl->kev[i] = nullptr;
    }
  }
  return QLP_OK;
}

int qlp_bls_kernel_time(qlp_bls_plan_t* pl, float* ms, int32_t* kernel) {
  if (!pl || !ms || !pl->kev[0]) return QLP_ERR_ARG;
  QLP_CK(cudaEventSynchronize(pl->kev[1]));
  QLP_CK(cudaEventElapsedTime(ms, pl->kev[0], pl->kev[1]));
  if (kernel) *kernel = timed_kernel(pl);
  return QLP_OK;
}

int qlp_bls_plan_times(const qlp_bls_plan_t* pl, double* seconds4) {
  if (!pl || !seconds4) return QLP_ERR_ARG;
  for (int i = 0; i < 4; ++i) seconds4[i] = pl->times[i];
  return QLP_OK;
}

int qlp_bls_plan_exact_stats(const qlp_bls_plan_t* pl, int32_t* n_exact_stars, double* exact_edges,
                             double* exact_bins) {
  if (!pl) return QLP_ERR_ARG;
  if (n_exact_stars) *n_exact_stars = pl->n_fixed_stars;
  if (exact_edges) *exact_edges = pl->edges_fixed;
  if (exact_bins) *exact_bins = pl->bins_fixed;
  return QLP_OK;
}

int qlp_bls_plan_narrow_stats(const qlp_bls_plan_t* pl, int32_t* n_narrow_stars, double* narrow_edges,
                              double* narrow_bins) {
  if (!pl) return QLP_ERR_ARG;
  if (n_narrow_stars) *n_narrow_stars = pl->n_narrow_stars;
  if (narrow_edges) *narrow_edges = pl->edges_narrow;
  if (narrow_bins) *narrow_bins = pl->bins_narrow;
  return QLP_OK;
}

int qlp_bls_plan_launches(const qlp_bls_plan_t* pl, int32_t* n_search_launches) {
  if (!pl || !n_search_launches) return QLP_ERR_ARG;
  int32_t n = 0;
  if (pl->n_items > 0) n += 2;
  if (pl->c_items > 0) n += 2;
  if (pl->f_items > 0) n += 1 + (pl->f_whole > 0) + (pl->f_items > pl->f_whole);
  *n_search_launches = n;
  return QLP_OK;
}

// Orders `stream` after the plan's own device work (see `ready`). A stream capture
// may not wait on work outside it: qlp_bls_graph_capture and qlp_bls_device_status
// wait on the host first; a capture of the caller's own that starts before either
// (or before a stream synchronisation seen here) is refused.
static cudaError_t wait_plan_ready(qlp_bls_plan_t* pl, cudaStream_t st) {
  if (!pl->ready || pl->ready_seen) return cudaSuccess;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
  return cudaStreamWaitEvent(st, pl->ready, 0);
}

// Host wait for the plan's own device work.
static cudaError_t sync_plan_ready(qlp_bls_plan_t* pl) {
  if (!pl->ready || pl->ready_seen) return cudaSuccess;
  const cudaError_t e = cudaEventSynchronize(pl->ready);
  if (e == cudaSuccess) pl->ready_seen = true;
  return e;
}

int qlp_bls_search(qlp_bls_plan_t* pl, void* stream, float* sr, uint8_t* qidx, uint32_t* phase_bin,
                   float* s_best, float* r_best) {
  if (!pl) return QLP_ERR_ARG;
  if (pl->f_off.back() > 0 && !sr) return QLP_ERR_ARG;
  if (pl->n_stars == 0 || pl->f_off.back() == 0) return QLP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  QLP_CK(wait_plan_ready(pl, st));
  QLP_CK(cudaMemsetAsync(pl->d_ctl, 0, 2 * sizeof(int32_t), st));
  QLP_CK(cudaMemsetAsync(pl->d_ctl + 3, 0, 2 * sizeof(int32_t), st));
  int e = 0;
  if (pl->n_items > 0) {
    PrepArgs pa{};
    pa.stars = pl->d_stars;
    pa.tp = pl->d_tp;
    pa.y = pl->d_y;
    pa.dy = pl->d_dy;
    pa.pts = pl->d_pts;
    pa.tpd = pl->d_tpd;
    pa.tile_pts = pl->tile_pts;
    pa.n_stars = pl->n_stars;
    e = launch_prep(pa, stream);
    if (e) return cuda_fail((cudaError_t)e, "prep launch");
    BlsArgs a{};
    a.stars = pl->d_stars;
    a.fq = pl->d_fq;
    a.items = pl->d_items;
    a.n_items = pl->n_items;
    a.loop_bound = pl->p.work_loop_bound;
    a.nq = pl->nq;
    a.pts = pl->d_pts;
    a.tpd = pl->d_tpd;
    a.cursor = pl->d_ctl;
    a.err = pl->d_ctl + 2;
    a.sr = sr;
    a.qidx = qidx;
    a.kbin = phase_bin;
    a.sbest = s_best;
    a.rbest = r_best;
    a.noverlap = pl->p.noverlap;
    for (int j = 0; j < kMaxQ; ++j) a.E[j] = pl->E[j];
    a.tile_pts = pl->tile_pts;
    a.hist_stride = pl->hist_stride;
    a.tile_off = pl->tile_off;
    if (timed_kernel(pl) == kMethodPoints) QLP_CK(record_kev(pl, 0, st));
    e = launch_bls(a, pl->p.phase_mode, pl->p.sum_mode == QLP_SUM_PLAIN ? QLP_SUM_PLAIN : QLP_SUM_COMP, pl->warps,
                   pl->blocks, pl->smem, stream);
    if (e) return cuda_fail((cudaError_t)e, "search launch");
    if (timed_kernel(pl) == kMethodPoints) QLP_CK(record_kev(pl, 1, st));
  }
  if (pl->c_items > 0) {
    PrepCellsArgs pc{};
    pc.stars = pl->d_stars;
    pc.cell_stars = pl->d_cell_stars;
    pc.n = pl->n_cell_stars - pl->n_fixed_stars;  // the compensated kernel's stars (d_cell_stars)
    pc.tp = pl->d_tp;
    pc.y = pl->d_y;
    pc.dy = pl->d_dy;
    pc.cpre = pl->d_cpre;
    pc.dt = pl->d_dt;
    pc.loc = pl->d_loc;
    pc.base = pl->d_base;
    pc.gidx = pl->d_gidx;
    e = launch_prep_cells(pc, stream);
    if (e) return cuda_fail((cudaError_t)e, "cell prep launch");
    CellArgs c{};
    c.stars = pl->d_stars;
    c.fq = pl->d_fq;
    c.items = pl->d_items + pl->n_items;
    c.n_items = pl->c_items;
    c.loop_bound = pl->p.work_loop_bound;
    c.nq = pl->nq;
    c.tp = pl->d_tp;
    c.dt = pl->d_dt;
    c.loc = pl->d_loc;
    c.base = pl->d_base;
    c.gidx = pl->d_gidx;
    c.cursor = pl->d_ctl + 1;
    c.err = pl->d_ctl + 2;
    c.sr = sr;
    c.qidx = qidx;
    c.kbin = phase_bin;
    c.sbest = s_best;
    c.rbest = r_best;
    c.noverlap = pl->p.noverlap;
    c.per_q = pl->p.bin_mode == QLP_BIN_PER_Q ? 1 : 0;
    c.m_perq = (int32_t)pl->p.noverlap;
    for (int j = 0; j < kMaxQ; ++j) c.E[j] = pl->E[j];
    if (timed_kernel(pl) == kMethodCells) QLP_CK(record_kev(pl, 0, st));
    e = launch_cells(c, pl->p.sum_mode == QLP_SUM_PLAIN ? QLP_SUM_PLAIN : QLP_SUM_COMP, pl->c_warps, pl->c_blocks,
                     pl->c_smem, stream);
    if (e) return cuda_fail((cudaError_t)e, "cell search launch");
    if (timed_kernel(pl) == kMethodCells) QLP_CK(record_kev(pl, 1, st));
  }
  if (pl->f_items > 0) {
    const PrepFixedArgs pf = fixed_args(pl);
    e = launch_prep_fixed(pf, stream);
    if (e) return cuda_fail((cudaError_t)e, "exact cell prep launch");
    FixedArgs fa{};
    fa.stars = pl->d_stars;
    fa.fx = pl->d_fx;
    fa.fq = pl->d_fq;
    fa.frec = pl->d_frec;
    fa.loop_bound = pl->p.work_loop_bound;
    fa.nq = pl->nq;
    fa.tp = pl->d_tp;
    fa.dt = pl->d_dt;
    fa.loc = reinterpret_cast<const int2*>(pl->d_loc);
    fa.base = reinterpret_cast<const longlong2*>(pl->d_base);
    fa.gidx = pl->d_gidx;
    fa.err = pl->d_ctl + 2;
    fa.sr = sr;
    fa.qidx = qidx;
    fa.kbin = phase_bin;
    fa.sbest = s_best;
    fa.rbest = r_best;
    fa.stride4 = 4;
    fa.ws = pl->d_ws;
    fa.ws_block = pl->ws_block;
    QLP_CK(record_kev(pl, 0, st));
    for (int k = 0; k < 2; ++k) {  // whole tables, then windowed ones
      const int32_t n_k = k ? pl->f_items - pl->f_whole : pl->f_whole;
      if (n_k == 0) continue;
      fa.items = pl->d_items + pl->n_items + pl->c_items + (k ? pl->f_whole : 0);
      fa.n_items = n_k;
      fa.cursor = pl->d_ctl + 3 + k;
      e = launch_cells_fixed(fa, k == 1, pl->f_blocks, pl->f_smem, stream);
      if (e) return cuda_fail((cudaError_t)e, "exact cell search launch");
    }
    QLP_CK(record_kev(pl, 1, st));
  }
  return QLP_OK;
}

int qlp_bls_snr_trend(qlp_bls_plan_t* pl, void* stream, const float* sr, const uint8_t* qidx,
                      const uint32_t* phase_bin, const float* s_best, const float* r_best,
                      const double* trend_in, double* trend_out, float* snr, qlp_bls_best* best);

int qlp_bls_snr(qlp_bls_plan_t* pl, void* stream, const float* sr, const uint8_t* qidx,
                const uint32_t* phase_bin, const float* s_best, const float* r_best, float* snr,
                qlp_bls_best* best) {
  return qlp_bls_snr_trend(pl, stream, sr, qidx, phase_bin, s_best, r_best, nullptr, nullptr, snr, best);
}

int qlp_bls_coarse_tensor(qlp_bls_plan_t* pl, void* stream, const float* snr, int32_t n_bins, void* out,
                          float* snr_rows) {
  if (!pl || !out || n_bins <= 0 || (pl->f_off.back() > 0 && !snr)) return QLP_ERR_ARG;
  if (pl->p.grid_mode != 1 || n_bins != pl->p.coarse_bins) return QLP_ERR_ARG;
  // harmonic offsets on the log-period grid: the bins of 2P and 3P lie d2 and d3 above
  const double per_bin = std::log(pl->p.coarse_pmax / pl->p.coarse_pmin) / (double)(n_bins - 1);
  const int d2 = (int)std::nearbyint(std::log(2.0) / per_bin), d3 = (int)std::nearbyint(std::log(3.0) / per_bin);
  const int e = launch_coarse_tensor(pl->d_stars, pl->n_stars, snr, n_bins, out, snr_rows, d2, d3, stream);
  return e ? cuda_fail((cudaError_t)e, "coarse tensor launch") : QLP_OK;
}

int qlp_cnn_topk(const float* logits, const void* x0, int32_t batch, int32_t len, int32_t k, int32_t* out,
                 void* stream) {
  if (!logits || !x0 || !out || batch < 0 || len <= 0 || k <= 0 || k > len) return QLP_ERR_ARG;
  const int e = launch_topk(logits, x0, batch, len, k, out, stream);
  return e ? cuda_fail((cudaError_t)e, "topk launch") : QLP_OK;
}

int qlp_bls_snr_trend(qlp_bls_plan_t* pl, void* stream, const float* sr, const uint8_t* qidx,
                      const uint32_t* phase_bin, const float* s_best, const float* r_best,
                      const double* trend_in, double* trend_out, float* snr, qlp_bls_best* best) {
  if (!pl) return QLP_ERR_ARG;
  if (pl->n_stars > 0 && !best) return QLP_ERR_ARG;
  if (pl->f_off.back() > 0 && (!sr || !qidx || !phase_bin || !s_best || !r_best || !snr)) return QLP_ERR_ARG;
  if (pl->n_stars == 0) return QLP_OK;
  QLP_CK(wait_plan_ready(pl, (cudaStream_t)stream));
  SnrArgs a{};
  a.stars = pl->d_stars;
  a.fq = pl->d_fq;
  a.sr = sr;
  a.qidx = qidx;
  a.kbin = phase_bin;
  a.sbest = s_best;
  a.rbest = r_best;
  a.snr = snr;
  a.best = best;
  a.trend_in = trend_in;
  a.trend_out = trend_out;
  a.err = pl->d_ctl + 2;
  a.noverlap = pl->p.noverlap;
  for (int j = 0; j < kMaxQ; ++j) a.E[j] = pl->E[j];
  a.nq = pl->nq;
  a.mad_mode = pl->p.mad_mode;
  a.n_stars = pl->n_stars;
  a.per_q = pl->p.bin_mode == QLP_BIN_PER_Q ? 1 : 0;
  a.m_perq = (int32_t)pl->p.noverlap;
  const int e = launch_snr(a, stream);
  if (e) return cuda_fail((cudaError_t)e, "snr launch");
  return QLP_OK;
}

int qlp_bls_device_status(qlp_bls_plan_t* pl, void* stream, int32_t* flags) {
  if (!pl || !flags) return QLP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  QLP_CK(cudaStreamSynchronize(st));
  QLP_CK(sync_plan_ready(pl));
  int32_t v = 0;
  QLP_CK(cudaMemcpy(&v, pl->d_ctl + 2, sizeof(int32_t), cudaMemcpyDeviceToHost));
  *flags = v;
  QLP_CK(cudaMemset(pl->d_ctl + 2, 0, sizeof(int32_t)));
  return v ? QLP_ERR_DEVICE : QLP_OK;
}

static int bls_run_host_impl(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets, const double* t,
                             const double* y, const double* dy, const double* rho, const double* rstar,
                             float* sr_host, float* snr_host, int64_t sr_capacity, qlp_bls_best* best_host,
                             int64_t* n_freq_total_out) {
  if (!best_host && n_stars > 0) return QLP_ERR_ARG;
  if (n_stars < 0 || (n_stars > 0 && !offsets)) return QLP_ERR_ARG;
  // The batch runs in chunks of whole stars: the host plans chunk k + 1 (the grid
  // and tables, on all cores) while the device searches chunk k. The first and
  // the last chunk hold half the points of the others, so that the device starts
  // early and the last search after the host's work is short. Uploads use one
  // stream, the searches another; results come back after the last launch.
  const int64_t npts = n_stars > 0 ? offsets[n_stars] - offsets[0] : 0;
  const int nch = n_stars >= 1024 ? 9 : 1;
  struct Chunk {
    qlp_bls_plan_t* pl = nullptr;
    int32_t s0 = 0, ns = 0;
    int64_t nf = 0;
    float *sr = nullptr, *snr = nullptr, *s = nullptr, *r = nullptr;
    uint8_t* q = nullptr;
    uint32_t* k = nullptr;
    qlp_bls_best* best = nullptr;
    void* mem = nullptr;  // one allocation holding the outputs above
    size_t mem_bytes = 0;
  };
  std::vector<Chunk> ch;
  cudaStream_t st_up = nullptr, st_run = nullptr;
  QLP_CK(cudaStreamCreateWithFlags(&st_up, cudaStreamNonBlocking));
  cudaError_t ce = cudaStreamCreateWithFlags(&st_run, cudaStreamNonBlocking);
  if (ce != cudaSuccess) {
    cudaStreamDestroy(st_up);
    return cuda_fail(ce, "cudaStreamCreate");
  }
  int rc = QLP_OK;
  int32_t s0 = 0;
  for (int c = 0; c < nch && rc == QLP_OK && (s0 < n_stars || (c == 0 && n_stars == 0)); ++c) {
    int32_t s1 = n_stars;
    if (c < nch - 1) {  // end of chunk c at (c + 1/2) of nch - 1 equal shares of the points
      const int64_t goal = offsets[0] + npts * (2 * c + 1) / (2 * (nch - 1));
      s1 = s0;
      while (s1 < n_stars && offsets[s1] < goal) ++s1;
      s1 = std::max(s1, std::min(n_stars, s0 + 1));
    }
    Chunk k;
    k.s0 = s0;
    k.ns = s1 - s0;
    std::vector<int64_t> off((size_t)k.ns + 1);
    for (int32_t i = 0; i <= k.ns; ++i) off[(size_t)i] = n_stars > 0 ? offsets[s0 + i] - offsets[s0] : 0;
    const int64_t o0 = n_stars > 0 ? offsets[s0] : 0;
    rc = qlp_bls_plan(p, k.ns, off.data(), t ? t + o0 : nullptr, y ? y + o0 : nullptr, dy ? dy + o0 : nullptr,
                      rho ? rho + s0 : nullptr, rstar ? rstar + s0 : nullptr, st_up, &k.pl);
    if (rc) break;
    k.nf = k.pl->f_off.back();
    ch.push_back(k);
    Chunk& b = ch.back();
    DevArena outs;
    outs.add(&b.sr, (size_t)b.nf)
        .add(&b.snr, (size_t)b.nf)
        .add(&b.s, (size_t)b.nf)
        .add(&b.r, (size_t)b.nf)
        .add(&b.q, (size_t)b.nf)
        .add(&b.k, (size_t)b.nf)
        .add(&b.best, (size_t)b.ns);
    if ((rc = outs.commit(&b.mem, &b.mem_bytes))) break;
    if ((rc = qlp_bls_search(b.pl, st_run, b.sr, b.q, b.k, b.s, b.r)) != QLP_OK) break;
    if ((rc = qlp_bls_snr(b.pl, st_run, b.sr, b.q, b.k, b.s, b.r, b.snr, b.best)) != QLP_OK) break;
    s0 = s1;
  }
  int64_t nf_tot = 0;
  for (const Chunk& k : ch) nf_tot += k.nf;
  if (n_freq_total_out) *n_freq_total_out = nf_tot;
  const bool fits = nf_tot <= sr_capacity;
  if (rc == QLP_OK) {
    cudaError_t e = cudaStreamSynchronize(st_run);
    int64_t f0 = 0;
    for (const Chunk& k : ch) {
      if (e == cudaSuccess && k.ns > 0)
        e = cudaMemcpy(best_host + k.s0, k.best, sizeof(qlp_bls_best) * (size_t)k.ns, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && sr_host && fits && k.nf > 0)
        e = cudaMemcpy(sr_host + f0, k.sr, sizeof(float) * (size_t)k.nf, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && snr_host && fits && k.nf > 0)
        e = cudaMemcpy(snr_host + f0, k.snr, sizeof(float) * (size_t)k.nf, cudaMemcpyDeviceToHost);
      f0 += k.nf;
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "result download");
    for (const Chunk& k : ch) {
      if (rc != QLP_OK) break;
      int32_t flags = 0;
      rc = qlp_bls_device_status(k.pl, st_run, &flags);
    }
    if (rc == QLP_OK && (sr_host || snr_host) && !fits) rc = QLP_ERR_ARG;
  }
  cudaStreamSynchronize(st_run);
  for (Chunk& k : ch) {
    cudaFree(k.mem);
    budget_give(k.mem_bytes);
    qlp_bls_plan_destroy(k.pl);
  }
  cudaStreamDestroy(st_up);
  cudaStreamDestroy(st_run);
  return rc;
}

int qlp_bls_run_host(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets, const double* t,
                     const double* y, const double* dy, const double* rho, const double* rstar,
                     float* sr_host, float* snr_host, int64_t sr_capacity, qlp_bls_best* best_host,
                     int64_t* n_freq_total_out) {
  return guarded([&] {
    return bls_run_host_impl(p, n_stars, offsets, t, y, dy, rho, rstar, sr_host, snr_host, sr_capacity, best_host,
                             n_freq_total_out);
  });
}

static int bls_star_grid_impl(const qlp_bls_params* pin, int64_t n, const double* t, const double* y,
                              const double* dy, double rho, int64_t n_win, const double* win_flo,
                              const double* win_fhi, int32_t* status, double* pmin, double* pmax,
                              double* t_ref, double* baseline, double* freqs, double* qmins,
                              int64_t capacity, int64_t* n_f_out) {
  if (!n_f_out || n < 0 || (n > 0 && (!t || !y || !dy))) return QLP_ERR_ARG;
  if (win_flo && (n_win < 0 || (n_win > 0 && !win_fhi))) return QLP_ERR_ARG;
  qlp_bls_params p;
  if (pin) p = *pin; else qlp_bls_params_default(&p);
  const int rc = check_params(p);
  if (rc) return rc;
  if (win_flo && p.grid_mode != 0) return QLP_ERR_ARG;
  StarPlanHost h;
  Windows w;
  w.lo = win_flo;
  w.hi = win_fhi;
  w.n = n_win;
  plan_one(p, t, y, dy, n, rho, &h, win_flo ? &w : nullptr);
  if (status) *status = h.status;
  if (pmin) *pmin = h.pmin;
  if (pmax) *pmax = h.pmax;
  if (t_ref) *t_ref = h.t_ref;
  if (baseline) *baseline = h.baseline;
  const int64_t nf = h.status == 0 ? (int64_t)h.freqs.size() : 0;
  *n_f_out = nf;
  if ((freqs || qmins) && capacity < nf) return QLP_ERR_ARG;
  if (freqs && nf) std::memcpy(freqs, h.freqs.data(), sizeof(double) * (size_t)nf);
  if (qmins && nf) std::memcpy(qmins, h.qmins.data(), sizeof(double) * (size_t)nf);
  return QLP_OK;
}

int qlp_bls_star_grid(const qlp_bls_params* pin, int64_t n, const double* t, const double* y,
                      const double* dy, double rho, int64_t n_win, const double* win_flo,
                      const double* win_fhi, int32_t* status, double* pmin, double* pmax,
                      double* t_ref, double* baseline, double* freqs, double* qmins,
                      int64_t capacity, int64_t* n_f_out) {
  return guarded([&] {
    return bls_star_grid_impl(pin, n, t, y, dy, rho, n_win, win_flo, win_fhi, status, pmin, pmax, t_ref, baseline,
                              freqs, qmins, capacity, n_f_out);
  });
}

static int bls_batch_grid_impl(const qlp_bls_params* pin, int32_t n_stars, const int64_t* offsets, const double* t,
                               const double* y, const double* dy, const double* rho, int32_t* star_status,
                               int64_t* freq_offsets, double* freqs, int64_t capacity) {
  if (n_stars < 0 || !freq_offsets || (n_stars > 0 && (!offsets || !t || !y || !dy))) return QLP_ERR_ARG;
  for (int32_t s = 0; s < n_stars; ++s)
    if (offsets[s + 1] < offsets[s]) return QLP_ERR_ARG;
  qlp_bls_params p;
  if (pin) p = *pin; else qlp_bls_params_default(&p);
  const int rc = check_params(p);
  if (rc) return rc;
  std::vector<StarPlanHost> sp;
  plan_all(p, n_stars, offsets, t, y, dy, rho, &sp);
  freq_offsets[0] = 0;
  for (int32_t s = 0; s < n_stars; ++s) {
    const StarPlanHost& h = sp[(size_t)s];
    if (star_status) star_status[s] = h.status;
    freq_offsets[s + 1] = freq_offsets[s] + (h.status == 0 ? (int64_t)h.freqs.size() : 0);
  }
  if (!freqs) return QLP_OK;
  if (capacity < freq_offsets[n_stars]) return QLP_ERR_ARG;
  for (int32_t s = 0; s < n_stars; ++s) {
    const int64_t k = freq_offsets[s + 1] - freq_offsets[s];
    if (k) std::memcpy(freqs + freq_offsets[s], sp[(size_t)s].freqs.data(), sizeof(double) * (size_t)k);
  }
  return QLP_OK;
}

int qlp_bls_batch_grid(const qlp_bls_params* pin, int32_t n_stars, const int64_t* offsets, const double* t,
                       const double* y, const double* dy, const double* rho, int32_t* star_status,
                       int64_t* freq_offsets, double* freqs, int64_t capacity) {
  return guarded([&] {
    return bls_batch_grid_impl(pin, n_stars, offsets, t, y, dy, rho, star_status, freq_offsets, freqs, capacity);
  });
}

void qlp_bls_plan_destroy(qlp_bls_plan_t* pl) { free_plan(pl); }

int qlp_set_device_budget(int64_t bytes) {
  if (bytes < 0) return QLP_ERR_ARG;
  g_budget.store(bytes);
  return QLP_OK;
}

int64_t qlp_device_bytes_held(void) { return g_held.load(); }

int qlp_bls_top_peaks(const qlp_bls_plan_t* pl, void* stream, const float* snr, int32_t n_peaks, double sep,
                      int32_t* out) {
  if (!pl || n_peaks < 1 || n_peaks > 64 || !(sep >= 0.0)) return QLP_ERR_ARG;
  if (pl->n_stars > 0 && (!out || (pl->f_off.back() > 0 && !snr))) return QLP_ERR_ARG;
  const int e = launch_peaks(pl->d_stars, pl->n_stars, pl->d_fq, snr, n_peaks, sep, out, stream);
  return e ? cuda_fail((cudaError_t)e, "peaks launch") : QLP_OK;
}

int qlp_bls_candidate_stats(qlp_bls_plan_t* pl, void* stream, const qlp_bls_best* best, qlp_bls_cand_stats* out) {
  if (!pl) return QLP_ERR_ARG;
  if (pl->n_stars > 0 && (!best || !out)) return QLP_ERR_ARG;
  if (pl->n_stars == 0) return QLP_OK;
  if (!pl->d_wrec) {
    const int rc = dev_alloc(&pl->d_wrec, (size_t)std::max<int64_t>(pl->n_pts_alloc, 1), &pl->wrec_bytes);
    if (rc) return rc;
  }
  if (!pl->d_sorder) {
    const int rc = dev_alloc(&pl->d_sorder, (size_t)pl->n_stars, &pl->sorder_bytes);
    if (rc) return rc;
  }
  StatsArgs a{};
  a.stars = pl->d_stars;
  a.n_stars = pl->n_stars;
  a.tp = pl->d_tp;
  a.y = pl->d_y;
  a.dy = pl->d_dy;
  a.best = best;
  a.out = out;
  a.wrec = pl->d_wrec;
  a.order = pl->d_sorder;
  const int e = launch_stats(a, stream);
  return e ? cuda_fail((cudaError_t)e, "stats launch") : QLP_OK;
}

int qlp_bls_graph_capture(qlp_bls_plan_t* pl, int32_t parts, float* sr, uint8_t* qidx, uint32_t* phase_bin,
                          float* s_best, float* r_best, float* snr, qlp_bls_best* best) {
  if (!pl || parts < 1 || parts > 3) return QLP_ERR_ARG;
  if (pl->f_off.back() > 0 && (!sr || !qidx || !phase_bin || !s_best || !r_best)) return QLP_ERR_ARG;
  if ((parts & 2) && ((pl->f_off.back() > 0 && !snr) || (pl->n_stars > 0 && !best))) return QLP_ERR_ARG;
  if (!pl->cap_stream) QLP_CK(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
  QLP_CK(sync_plan_ready(pl));
  const int slot = parts - 1;
  if (pl->gexec[slot]) { cudaGraphExecDestroy(pl->gexec[slot]); pl->gexec[slot] = nullptr; }
  if (pl->graph[slot]) { cudaGraphDestroy(pl->graph[slot]); pl->graph[slot] = nullptr; }
  QLP_CK(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = QLP_OK;
  if (parts & 1) rc = qlp_bls_search(pl, pl->cap_stream, sr, qidx, phase_bin, s_best, r_best);
  if (rc == QLP_OK && (parts & 2)) rc = qlp_bls_snr(pl, pl->cap_stream, sr, qidx, phase_bin, s_best, r_best, snr, best);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
  if (rc != QLP_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  pl->graph[slot] = g;
  QLP_CK(cudaGraphInstantiate(&pl->gexec[slot], g, 0));
  return QLP_OK;
}

int qlp_bls_graph_launch(qlp_bls_plan_t* pl, int32_t parts, void* stream) {
  if (!pl || parts < 1 || parts > 3 || !pl->gexec[parts - 1]) return QLP_ERR_ARG;
  QLP_CK(cudaGraphLaunch(pl->gexec[parts - 1], (cudaStream_t)stream));
  return QLP_OK;
}

}  // extern "C"
