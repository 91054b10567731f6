// Internal layouts shared by the host planner, the C-ABI glue and the kernels.
#pragma once

#include <cstdint>

#include <cuda_runtime_api.h>
#include <vector_types.h>

#include "../../include/qlp_bls.h"

namespace qlp {

constexpr int kMaxQ = 16;        // largest number of durations (nq) supported
constexpr int kMPad = 16;        // histogram wrap padding (>= largest m_j)
constexpr int kMaxSturges = 40;  // largest Sturges bin count the S/N kernel handles

// One star as the device sees it.
struct StarDev {
  int64_t pt_off;      // first valid point in the raw arrays (t', y, dy)
  int64_t pad_off;     // first slot in the prepared, tile-transposed arrays
  int64_t f_off;       // first entry in the per-frequency arrays
  int32_t n_pts;       // valid points N
  int32_t n_f;         // trial frequencies
  int32_t status;      // QLP_STAR_* flags from the planner
  int32_t sturges_nb;  // S/N trend bins, round(1 + 3.322 log10 n_f)
  int32_t fp64_phase;  // 1: fold this star in FP64 whatever the phase mode
  int32_t method;      // kMethodPoints or kMethodCells
  double t_ref;        // t_min of the valid points
  double baseline;     // t_max - t_min
  // cell path (method == kMethodCells): time axis cut into cells of width h,
  // each holding at most one point; cells 0 .. n_cells-1 cover [0, n_cells h),
  // cell n_cells is a sentinel past the last point
  double h;
  int32_t n_cells;
  int32_t grid_k0;     // coarse grid: bin index of the star's first (lowest) frequency
  int64_t cell_off;    // first entry in the per-cell arrays (n_cells + 1 entries)
  int64_t base_off;    // first entry in the per-32-cell base array
  int64_t cpre_off;    // first entry in the prefix-sum array (N + 1 entries)
  // time windows of the cell table when it does not fit in shared memory at once:
  // window w owns cells [w win_cells, (w+1) win_cells) and stages them from the
  // 32-aligned cell below its start to win_ovl cells past its end
  int32_t n_win;
  int32_t win_cells;
  int32_t win_ovl;
  int32_t win_cap;     // cells the shared table holds (one window, or the whole table)
  // exact path, whole table: 1 = the 32-bit table (prefix sums of round(w F) and
  // round(w d 2^ky) as 32-bit words, no group bases), with y_exc the planner's largest
  // |prefix of w d| from which the y scale follows; 0 = the 64-bit table
  int32_t narrow;
  double y_exc;
};

constexpr int32_t kMethodPoints = 0;
constexpr int32_t kMethodCells = 1;
constexpr int32_t kMethodFixed = 2;   // cell path with exact fixed-point prefix sums (fixed_kernels.cu)

// (star, frequency chunk) unit of the device work queue.
struct WorkItem {
  int32_t star;
  int32_t f_begin;     // first frequency, relative to the star
  int32_t f_count;
  int32_t pad0;        // cell path: histogram stride / 32 (low 16 bits), active warps (high 16)
};

struct BlsArgs {
  const StarDev* stars;
  const double2* fq;       // per frequency: (f, q_min)
  const WorkItem* items;
  int32_t n_items;
  int32_t loop_bound;  // 0 = n_items; else each block's work loop stops after loop_bound + 1 pops
  int32_t nq;
  const float4* pts;       // prepared points: (t'_hi, t'_lo, w d, w)
  const double* tpd;       // prepared points: t' in FP64 (same slots)
  int32_t* cursor;         // work-queue head (zeroed before the launch)
  int32_t* err;            // device error flags
  float* sr;
  uint8_t* qidx;
  uint32_t* kbin;
  float* sbest;
  float* rbest;
  double noverlap;
  double E[kMaxQ];         // exp(j dlogq)
  int32_t tile_pts;        // points per shared-memory tile (multiple of 32)
  int32_t hist_stride;     // floats per histogram array of one warp (>= nbins_max + kMPad)
  uint32_t tile_off;       // byte offset of the point tile in dynamic shared memory
  int32_t pad0;
};

// Cell search (cells_kernels.cu): boundaries of phase bins instead of points.
struct CellArgs {
  const StarDev* stars;
  const double2* fq;
  const WorkItem* items;
  int32_t n_items;
  int32_t loop_bound;  // 0 = n_items; else each block's work loop stops after loop_bound + 1 pops
  int32_t nq;
  const double* tp;        // raw t' (CSR by pt_off), for the exact decision near ties
  const uint32_t* dt;      // per cell: its point's offset, 2^-32 of the cell; 0xFFFFFFFF if empty
  const float2* loc;       // per cell: prefix sums (w, w d) before the cell, minus the block base
  const float4* base;      // per 32 cells: block base prefix sums as (w_hi, w_lo, y_hi, y_lo)
  const int32_t* gidx;     // per cell: index of the first point at or after the cell start
  int32_t* cursor;
  int32_t* err;
  float* sr;
  uint8_t* qidx;
  uint32_t* kbin;
  float* sbest;
  float* rbest;
  double noverlap;
  double E[kMaxQ];
  int32_t per_q;           // QLP_BIN_PER_Q: one histogram of bins q_j / noverlap per duration j
  int32_t m_perq;          // bins per box in that mode (noverlap)
};

// Exact cell path (fixed_kernels.cu). Per star: the point weights and weighted
// residuals as integers, w_int = round(w 2^kw) and y_int = round(w d 2^ky), with
// kw, ky chosen so that any 32 consecutive points sum to less than 2^30 in
// magnitude; the prefix sums of these integers are exact.
struct FixedStar {
  long long w_tot;   // sum of w_int over the star (the prefix sum at the sentinel cell)
  long long y_tot;   // sum of y_int
  int32_t kw, ky;    // w_int = round(w 2^kw) (64-bit table), y_int = round(w d 2^ky)
  float scw;         // FP32 scale of the w sums: 2^-kw, or 1 / w_tot on the 32-bit table
  int32_t narrow;    // 1: the star's table is the 32-bit one (w_int = round(w F))
};

// Per trial frequency of an exact-path star, derived once from (f, q_min) in FP64
// with the same operations as the other search kernels.
struct __align__(16) FreqRec {
  unsigned long long K;      // bin duration D = 1/(f nbins) in cells, 2^-40 fixed point
  unsigned long long jlow;   // per box width w (bins): the lowest duration index j with m_j = w,
                             // 4 bits at bit 4 (w - 1)
  int32_t nb;                // phase bins; 0 when unsupported (SR 0 and the nbins flag)
  uint32_t band_q;           // guard band around each edge, 2^-32 of a cell
  uint32_t gq_bstar;         // last edge g_end = gq nbins + b*: gq << 13 | b* (b* < nbins <= 8192)
  uint32_t wmask;            // box widths present: bit w - 1 for a width of w bins
};

struct PrepFixedArgs {
  const StarDev* stars;
  const int32_t* fixed_stars;  // stars on the exact cell path
  int32_t n;
  int32_t nq;
  const double* tp;
  const double* y;
  const double* dy;
  const double2* fq;
  longlong2* ipre;             // integer prefix sums before each point, N + 1 per star
  uint32_t* dt;
  int2* loc;                   // per cell: prefix sums minus the 32-cell group base (int32 each)
  longlong2* base;             // per 32 cells: the group's prefix sums (int64 each)
  int32_t* gidx;
  FixedStar* fx;
  FreqRec* frec;
  double noverlap;
  double E[kMaxQ];
  int32_t nb_cap;
  int32_t max_pts;             // most points of a star in the list (shared memory of the prep)
  int32_t* err;                // device error bits (kErrRange)
};

struct FixedArgs {
  const StarDev* stars;
  const FixedStar* fx;
  const double2* fq;
  const FreqRec* frec;
  const WorkItem* items;
  int32_t n_items;
  int32_t loop_bound;  // 0 = n_items; else each block's work loop stops after loop_bound + 1 pops
  int32_t nq;
  const double* tp;
  const uint32_t* dt;
  const int2* loc;             // layout as in PrepFixedArgs: base + loc = prefix sum
  const longlong2* base;
  const int32_t* gidx;
  int32_t* cursor;
  int32_t* err;
  float* sr;
  uint8_t* qidx;
  uint32_t* kbin;
  float* sbest;
  float* rbest;
  uint32_t stride4;            // 4 (bytes of a table entry; a run-time value on purpose)
  int32_t pad0;
  longlong2* ws;               // time-windowed stars: per block, bin-sum rows of ws_block entries
  int64_t ws_block;
};

struct PrepCellsArgs {
  const StarDev* stars;
  const int32_t* cell_stars;  // stars on the cell path
  int32_t n;
  int32_t pad0;
  const double* tp;
  const double* y;
  const double* dy;
  double2* cpre;              // prefix sums (sum w, sum w d) before each point, N + 1 per star
  uint32_t* dt;
  float2* loc;
  float4* base;
  int32_t* gidx;
};

struct PrepArgs {
  const StarDev* stars;
  const double* tp;        // t - t_ref, valid points, CSR by pt_off
  const double* y;
  const double* dy;
  float4* pts;
  double* tpd;
  int32_t tile_pts;
  int32_t n_stars;
};

// Trend record of one star (the S/N kernel writes or reads it): node count,
// sigma_SR, median, the bin centres and bin medians of the median-binned trend.
constexpr int kTrendDoubles = 4 + 2 * kMaxSturges;

struct SnrArgs {
  const StarDev* stars;
  const double2* fq;
  const float* sr;
  const uint8_t* qidx;
  const uint32_t* kbin;
  const float* sbest;
  const float* rbest;
  float* snr;
  qlp_bls_best* best;
  int32_t* err;
  double* trend_out;         // per star kTrendDoubles, or null
  const double* trend_in;    // per star: use this trend and sigma instead of computing them
  double noverlap;
  double E[kMaxQ];
  int32_t nq;
  int32_t mad_mode;
  int32_t n_stars;
  int32_t per_q;             // QLP_BIN_PER_Q: box j is m_perq bins of histogram j
  int32_t m_perq;
};

// device error flags
constexpr int32_t kErrQueueBound = 1;   // work loop exceeded its iteration bound
constexpr int32_t kErrNbins = 2;        // a frequency needed more bins than the histogram holds
static_assert(kErrQueueBound == QLP_DEVERR_QUEUE && kErrNbins == QLP_DEVERR_NBINS, "device error bits");
constexpr int32_t kErrSturges = 4;      // more S/N bins than the kernel supports
constexpr int32_t kErrSelect = 8;       // median selection failed to converge
constexpr int32_t kErrMmaWait = 16;     // a tensor-core completion wait hit its bound
constexpr int32_t kErrCopyWait = 32;    // a bulk copy into shared memory did not complete in its bound
static_assert(kErrCopyWait == QLP_DEVERR_COPY, "device error bits");
constexpr int32_t kErrRange = 64;       // a 32-bit exact table's w d prefix sum left its range
static_assert(kErrRange == QLP_DEVERR_RANGE, "device error bits");

// launchers (bls_kernels.cu / snr_kernel.cu); return cudaError_t as int
int launch_prep(const PrepArgs& a, void* stream);
int launch_bls(const BlsArgs& a, int phase_mode, int sum_mode, int warps, int blocks,
               size_t smem_bytes, void* stream);
int launch_snr(const SnrArgs& a, void* stream);
int launch_coarse_tensor(const StarDev* stars, int n_stars, const float* snr, int n_bins, void* out,
                         float* snr_rows, int d2, int d3, void* stream);
int launch_topk(const float* logits, const void* x0, int batch, int len, int k, int32_t* out, void* stream);
int launch_prep_cells(const PrepCellsArgs& a, void* stream);
int launch_cells(const CellArgs& a, int sum_mode, int warps, int blocks, size_t smem, void* stream);
int launch_prep_fixed(const PrepFixedArgs& a, void* stream);
int launch_freq_recs(const PrepFixedArgs& a, void* stream);
int launch_cells_fixed(const FixedArgs& a, bool windowed, int blocks, size_t smem, void* stream);
// shared memory of the exact cell kernel for a table of ncs cells (incl. sentinel)
uint32_t fixed_smem_bytes(int ncs);
// shared memory of a time window of ncs cells (its table; pass B's rings overlay it)
uint32_t fixed_window_smem_bytes(int ncs);
uint32_t fixed_prep_smem_bytes(int n_pts);
int fixed_blocks_per_sm(size_t smem);
constexpr int kFixedWarps = 32;
constexpr int64_t kFixedWsBlock = 131072;  // bound on a block's whole-table rows: 32 warps x round32(nbins)
constexpr int64_t kFixedWinRows = 524288;  // workspace entries (16 B) a windowed item may take per block
constexpr int64_t kFixedPendRows = 64;     // workspace entries (16 B) per warp past its row: 32 pending boxes
// bytes of shared memory before the histograms of the cell kernel for a star with
// ncs cells (incl. sentinel) and nw warps
// One point of a candidate's fit window: t', P n for its transit index n at the
// starting epoch (the product the model's dt = (t' - T0) - P n uses), y and the
// point's weight (1/dy)^2. 32 bytes: the windows of the stars in flight stay in L2
// across the fit's iterations.
struct __align__(16) WinRec {
  double t, pn, y, w;
};

struct StatsArgs {
  const StarDev* stars;
  int32_t n_stars;
  const double* tp;
  const double* y;
  const double* dy;
  const qlp_bls_best* best;
  qlp_bls_cand_stats* out;
  WinRec* wrec;  // scratch: fit-window points, CSR by pt_off
  int32_t* order;  // scratch [n_stars]: the CTAs' stars, the longest fits first (or null: star = CTA)
};
int launch_peaks(const StarDev* stars, int n_stars, const double2* fq, const float* snr, int n_peaks, double sep,
                 int32_t* out, void* stream);
int launch_stats(const StatsArgs& a, void* stream);
int record_cuda_error(cudaError_t e, const char* what);
// the library's device-memory budget (qlp_set_device_budget): take before a
// cudaMalloc of a plan or network buffer (false = over the budget), give back on free
bool budget_take(size_t bytes);
void budget_give(size_t bytes);
uint32_t cells_hist_offset(int ncs, int nw);
int cells_blocks_per_sm(int sum_mode, int warps, size_t smem);
int bls_max_smem_per_block();
int launch_conv64(const void* x, const void* wpack, const float* bias, const void* mask, void* y,
                  int32_t* err, int batch, int len, int relu, void* stream);
int launch_pack_w64(const float* w, void* out, int transpose, void* stream);
int conv64_smem_bytes();
int bls_blocks_per_sm(int phase_mode, int sum_mode, int warps, size_t smem_bytes);

}  // namespace qlp
