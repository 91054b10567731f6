/*
 * qlp_bls.h -- C ABI of the GB300 (sm_103a) batched Keplerian-constrained BLS
 * transit search of "QLP Data Release Notes 003: GPU-based Transit Search"
 * (Kunimoto et al., arXiv:2302.01293).
 *
 * The library searches many stars at once. Per star it builds the search plan
 * of Sec. 2.1 (Pmin, Pmax, Keplerian duration range, frequency grid), computes
 * the BLS signal residue SR(f) on every trial frequency (Sec. 2.1 and Eq. 1's
 * SR), the spectral S/N of Eq. 1 with the Sturges median-binned trend and the
 * 1.4826 MAD scale (Sec. 2.2 item 1), and the best candidate (P, T0, q, depth)
 * used as the initial guess of the trapezoid fit (Sec. 2.2 item 2).
 *
 * Conventions shared by every entry point:
 *  - Return value: 0 (QLP_OK) on success, a negative QLP_ERR_* code when the
 *    whole call failed; qlp_strerror() names it. Problems of a single star are
 *    not call errors: they are reported in that star's status flags
 *    (QLP_STAR_*), and such a star gets no frequencies and no candidate.
 *  - Host pointers are read during the call only and stay owned by the caller.
 *  - Device pointers are caller-allocated CUDA global memory on the current
 *    device; results are written asynchronously on the given stream
 *    (a cudaStream_t passed as void*, NULL = legacy default stream) and are
 *    valid once that stream has been synchronised.
 *  - A plan is library-owned (qlp_bls_plan_destroy frees it). Calls on one plan
 *    must not overlap; different plans are independent.
 *  - Units: t in days, y relative flux, dy its 1-sigma error, rho in g/cm^3,
 *    R* in solar radii, frequencies in 1/day.
 */
#ifndef QLP_BLS_H
#define QLP_BLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define QLP_OK               0
#define QLP_ERR_ARG         -1  /* null pointer, negative size, non-monotone offsets, bad params */
#define QLP_ERR_CUDA        -2  /* a CUDA runtime call failed (message via qlp_last_cuda_error) */
#define QLP_ERR_NOMEM       -3  /* host or device allocation failed */
#define QLP_ERR_DEVICE      -4  /* a device-side bound was hit (iteration limit, capacity) */
#define QLP_ERR_UNSUPPORTED -5  /* option combination not built into this library */

/* Device error bits, as qlp_bls_device_status and qlp_bls_search_static report them. */
#define QLP_DEVERR_QUEUE     1  /* a persistent work loop hit its iteration bound */
#define QLP_DEVERR_NBINS     2  /* a frequency needed more bins than the histogram holds */
#define QLP_DEVERR_SNR_BINS  4  /* more S/N (Sturges) bins than supported */
#define QLP_DEVERR_COPY     32  /* an asynchronous copy into shared memory did not complete
                                   within its bound (the frequencies it fed are not valid) */
#define QLP_DEVERR_RANGE    64  /* a star's 32-bit exact table got a prefix sum of w d outside
                                   its 32-bit range (the planner's bound did not hold; that
                                   star's results are not valid) */

/* ---- per-star status flags (qlp_bls_plan_info star_status, qlp_bls_best.status) ---- */
#define QLP_STAR_UNSORTED    1  /* t decreases somewhere (after dropping invalid points) */
#define QLP_STAR_TOO_FEW     2  /* fewer than 2 valid points */
#define QLP_STAR_EMPTY_GRID  4  /* Pmin >= Pmax or zero baseline: nothing to search */
#define QLP_STAR_NBINS_CAP   8  /* some frequency needs more phase bins than nbins_cap, or than the
                                   shared-memory histograms of the star's search path hold */
#define QLP_STAR_ZERO_MAD   16  /* sigma_SR = 0: S/N undefined, no candidate */
#define QLP_STAR_UNSUPPORTED 32 /* the star cannot be searched with these options (bin_mode
                                   QLP_BIN_PER_Q needs the cell path: one point per cell) */

/* ---- options ---- */
#define QLP_PHASE_FP64  0  /* fold x = t'f and its bin in FP64, the oracle's exact sequence */
#define QLP_PHASE_DF    1  /* double-float (hi/lo FP32) fold; bins identical to FP64:
                              points within a guard band of a bin edge are re-folded in FP64 */
#define QLP_PHASE_FP32  2  /* plain FP32 fold (precision study only; bins may differ) */

#define QLP_BIN_SHARED  0  /* Sec. 2.1 footnote reading: one histogram of bins q_min / noverlap
                              per frequency; every duration q_j is a window of m_j of its bins */
#define QLP_BIN_PER_Q   1  /* variant: a histogram of bins q_j / noverlap for each duration q_j
                              (ceil(noverlap / q_j) bins), each box a window of noverlap bins
                              (noverlap must be an integer); reported j and k refer to
                              histogram j. Cell path only. */

#define QLP_SUM_PLAIN   0  /* FP32 histogram sums */
#define QLP_SUM_COMP    1  /* FP32 sums with the rounding error of every shared-memory add
                              captured exactly (TwoSum) and added back (compensated) */
#define QLP_SUM_FIXED   2  /* exact sums (default): per star the weights w and w (y - ybar) are
                              rounded once to integers and every bin and box sum is an exact
                              integer sum of those; the chosen box's s, r and 1 - r reach FP32
                              as double-float (hi, lo) numbers. Two table widths: a star whose
                              whole table fits in shared memory, with at most 65,536 points and
                              a running sum of w d that stays within 64 times its largest
                              single |w d|, takes 32-bit prefix sums of round(w F), F = 2^32 -
                              2^17 (r = the ratio of two integer sums), and of round(w d 2^ky),
                              ky the largest with every prefix below 2^30; the other stars
                              take round(w 2^kw) and round(w d 2^ky) with per-star scales that
                              keep 32 consecutive points below 2^30, summed in 64 bits. Used on
                              the cell path (whole tables or time windows); the per-point path
                              uses QLP_SUM_COMP. */
#define QLP_SUM_FIXED64 3  /* as QLP_SUM_FIXED with the 64-bit tables for every star */

#define QLP_MAD_RAW     0  /* sigma_SR = 1.4826 median|SR - median(SR)| (the paper's wording) */
#define QLP_MAD_RESID   1  /* same on the detrended residual SR - trend */

typedef struct qlp_bls_params {
  double samples_per_peak;  /* 2     (Sec. 2.1 footnote) frequency step = q_min/(spp * T) */
  double dlogq;             /* 0.1   (Sec. 2.1 footnote) natural-log step of the duration grid */
  double noverlap;          /* 3     (Sec. 2.1 footnote) finest phase bin = q_min / noverlap */
  double qmin_fac;          /* 0.5   (Sec. 2.1) shortest duration / circular-orbit duration */
  double qmax_fac;          /* 2.0   (Sec. 2.1) longest duration / circular-orbit duration */
  double pmin_aR;           /* 2     (Sec. 2.1) Pmin where a = pmin_aR R* (3 for Sectors 59-60) */
  double gap_days;          /* 27.4  (Sec. 2.1) a gap longer than one sector splits stretches */
  double rho_default;       /* 1.41  (Sec. 2.1) solar density (g/cm^3) when rho is missing */
  int32_t nbins_cap;        /* largest phase-bin count a star may need (default 8192) */
  int32_t phase_mode;       /* QLP_PHASE_* (default QLP_PHASE_DF) */
  int32_t sum_mode;         /* QLP_SUM_*   (default QLP_SUM_FIXED) */
  int32_t mad_mode;         /* QLP_MAD_*   (default QLP_MAD_RAW) */
  int32_t chunk_freqs;      /* frequencies per work item, 0 = chosen by the planner */
  int32_t warps_per_block;  /* 0 = chosen by the planner; else 4, 8, 16 or 32 (32: cell path only,
                               the point path uses at most 16) */
  int32_t n_threads;        /* host threads for planning, 0 = all cores */
  int32_t tile_points;      /* points per shared-memory tile, 0 = as many as fit (multiple of 32) */
  int32_t method;           /* 0 = per star, the cheaper of the two search paths (default);
                               1 = fold every point; 2 = bin edges on the cell table wherever the
                               star allows it (same results: both give the FP64 bins) */
  int32_t grid_mode;        /* 0 = the frequency grid of Sec. 2.1 (default); 1 = the coarse grid of
                               the learned proposal: coarse_bins periods log-spaced from coarse_pmin
                               to coarse_pmax, P_k = pmin (pmax/pmin)^(k/(bins-1)), those within the
                               star's [Pmin, Pmax], in increasing frequency */
  int32_t coarse_bins;      /* 4096 */
  int32_t cell_window;      /* cell path: cells of the time table a block holds in shared memory at
                               once, 0 = the whole table when it fits, else as many as fill half
                               of it; a star whose table is longer is searched window by window */
  double coarse_pmin;       /* 0.1 d */
  double coarse_pmax;       /* 400 d */
  int32_t bin_mode;         /* QLP_BIN_* (default QLP_BIN_SHARED) */
  int32_t work_loop_bound;  /* 0 = each persistent search kernel's work loop may run as many
                               iterations as there are work items (default); n > 0 = a block
                               stops after n + 1 queue pops and raises QLP_DEVERR_QUEUE
                               (watchdog and failure-injection setting; results of items not
                               taken are left unwritten, and qlp_bls_search returns
                               QLP_ERR_DEVICE through qlp_bls_device_status) */
} qlp_bls_params;

/* Best candidate of one star: the frequency of maximum S/N and its BLS box. */
typedef struct qlp_bls_best {
  int64_t f_idx;   /* index in the star's frequency grid; -1 = no candidate */
  double f;        /* 1/day */
  double period;   /* days, 1/f */
  double t0;       /* first mid-box time >= t_min of the star (days) */
  double q;        /* box duration / period = m / nbins */
  double depth;    /* -s / (r (1 - r)), flux units; positive for a dip */
  double sr;       /* SR at f_idx */
  double snr;      /* S/N at f_idx */
  int32_t j;       /* duration index of the box (0 .. nq-1) */
  int32_t k;       /* first phase bin of the box */
  int32_t m;       /* bins covered by the box */
  int32_t nbins;   /* phase bins at f */
  int32_t status;  /* QLP_STAR_* flags of the star */
  int32_t pad;
} qlp_bls_best;

typedef struct qlp_bls_plan qlp_bls_plan_t;

/* Fill *p with the paper's settings (Sec. 2.1) and the library defaults. */
void qlp_bls_params_default(qlp_bls_params* p);

/*
 * qlp_bls_plan -- Sec. 2.1: per-star search plan, uploaded to the device.
 *  p        parameters (see qlp_bls_params); NULL = defaults.
 *  n_stars  number of stars (>= 0).
 *  offsets  host int64[n_stars + 1], non-decreasing, offsets[0] = 0: star s owns
 *           points offsets[s] .. offsets[s+1]-1 of t, y and dy.
 *  t, y, dy host double[offsets[n_stars]]: time (days), flux, 1-sigma error.
 *           Points with a non-finite value or dy <= 0 are dropped; the rest of
 *           a star must be sorted by t (else QLP_STAR_UNSORTED).
 *  rho      host double[n_stars] stellar density (g/cm^3); NULL, NaN or <= 0
 *           use p->rho_default.
 *  rstar    host double[n_stars] stellar radius (R_sun) or NULL. The period
 *           limits and durations depend on rho only (R* cancels in a/R*); it
 *           is accepted and kept for the caller.
 *  stream   cudaStream_t for the uploads (NULL = default stream).
 *  out_plan receives the plan (library-owned). On error *out_plan = NULL.
 * Host-side work: validation, Pmin (a = pmin_aR R*), Pmax (longest continuous
 * stretch, or half of it when no gap exceeds gap_days), the frequency grid
 * f_{k+1} = f_k + q_min(f_k)/(spp T) from 1/Pmax to 1/Pmin in FP64, and the
 * device work list; multithreaded over stars. Returns once the uploads are
 * complete (the host arrays may then be reused); the plan's last device work
 * (control words, per-frequency records) may still be queued on `stream`, and
 * every later call on the plan orders itself after it on its own stream.
 */
int qlp_bls_plan(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets,
                 const double* t, const double* y, const double* dy,
                 const double* rho, const double* rstar, void* stream,
                 qlp_bls_plan_t** out_plan);

/*
 * qlp_bls_plan_info -- sizes and the host copy of the plan. Any output may be NULL.
 *  n_freq_total  total number of trial frequencies over all stars.
 *  freq_offsets  int64[n_stars + 1]: star s owns spectrum entries
 *                freq_offsets[s] .. freq_offsets[s+1]-1 of every per-frequency array.
 *  freqs         double[n_freq_total] trial frequencies (1/day).
 *  star_status   int32[n_stars] QLP_STAR_* flags.
 *  n_points      int64: total valid points (the sum of N_s).
 *  work          double: sum over stars of N_s * n_f,s (point-frequency pairs).
 */
int qlp_bls_plan_info(const qlp_bls_plan_t* plan, int64_t* n_freq_total, int64_t* freq_offsets,
                      double* freqs, int32_t* star_status, int64_t* n_points, double* work);

/*
 * qlp_bls_plan_stats -- how the plan splits the work between the two search
 * paths (both give the same FP64-binned results, Sec. 2.1). Any output may be NULL.
 *  work_points   point-frequency pairs of stars whose points are folded one by one.
 *  work_cells    point-frequency pairs of stars searched by bin edges on the cell table.
 *  edges         bin edges the cell path evaluates (sum over its stars and
 *                frequencies of floor(T f nbins) + 3).
 *  n_cell_stars  stars on the cell path.
 *  n_windowed    of those, stars whose cell table is searched in several time
 *                windows (a table longer than one block's shared memory).
 */
int qlp_bls_plan_stats(const qlp_bls_plan_t* plan, double* work_points, double* work_cells,
                       double* edges, int32_t* n_cell_stars, int32_t* n_windowed);

/*
 * qlp_bls_plan_exact_stats -- the part of the cell path that runs with exact
 * integer sums (QLP_SUM_FIXED, Sec. 2.1's binned BLS with the bins' weights summed
 * exactly). Any output may be NULL.
 *  n_exact_stars  stars searched by the exact cell kernel (counted in n_cell_stars too).
 *  exact_edges    bin edges those stars evaluate (counted in edges too).
 *  exact_bins     sum of nbins over those stars' trial frequencies (box start positions
 *                 the sweep scores).
 * Returns QLP_ERR_ARG for a NULL plan.
 */
int qlp_bls_plan_exact_stats(const qlp_bls_plan_t* plan, int32_t* n_exact_stars, double* exact_edges,
                             double* exact_bins);

/*
 * qlp_bls_plan_narrow_stats -- of the exact path's stars, those whose table holds
 * 32-bit prefix sums (QLP_SUM_FIXED; see there for which stars). Any output may be NULL.
 *  n_narrow_stars  stars on the 32-bit table (counted in n_exact_stars too).
 *  narrow_edges    bin edges those stars evaluate (counted in exact_edges too).
 *  narrow_bins     sum of nbins over their trial frequencies (counted in exact_bins too).
 * Returns QLP_ERR_ARG for a NULL plan.
 */
int qlp_bls_plan_narrow_stats(const qlp_bls_plan_t* plan, int32_t* n_narrow_stars, double* narrow_edges,
                              double* narrow_bins);

/*
 * qlp_bls_plan_launches -- how many kernels one qlp_bls_search of the plan launches:
 * per search path in use its preparation kernel and its search kernel, the exact
 * path's search kernel as two launches when the plan has both whole-table and
 * time-windowed stars on it (one per kind of table). S/N is not counted.
 *  n_search_launches  output, host pointer.
 * Returns QLP_ERR_ARG for a NULL plan or output.
 */
int qlp_bls_plan_launches(const qlp_bls_plan_t* plan, int32_t* n_search_launches);

/*
 * qlp_bls_plan_times -- measurement aid (no counterpart in the paper): wall-clock
 * seconds the plan's construction spent in four phases, written to seconds4[0..3]:
 * the host grid and per-star plans (Sec. 2.1 rules, all stars in parallel), the
 * host staging of flat arrays and work items, device allocation, and the uploads
 * up to their completion (the plan-time kernels are queued after them).
 * QLP_ERR_ARG for a NULL plan or array.
 */
int qlp_bls_plan_times(const qlp_bls_plan_t* plan, double* seconds4);

/*
 * qlp_bls_kernel_timing -- measurement aid (no counterpart in the paper): with
 * enable != 0 the plan creates two CUDA events that every later qlp_bls_search on
 * it records just before and after its main kernel (the exact cell kernel when the
 * plan has exact-path stars, else the compensated cell kernel, else the per-point
 * kernel), also inside a graph captured afterwards (as event nodes); enable = 0
 * destroys them. Returns QLP_ERR_CUDA if an event cannot be created.
 * qlp_bls_kernel_time -- waits for the end event and returns, in *ms, the time
 * between the two events of the most recent search (or graph replay), and in
 * *kernel (may be NULL) which kernel they bracket: 0 per-point, 1 compensated cell,
 * 2 exact cell. QLP_ERR_ARG when timing is not enabled.
 */
int qlp_bls_kernel_timing(qlp_bls_plan_t* plan, int32_t enable);
int qlp_bls_kernel_time(qlp_bls_plan_t* plan, float* ms, int32_t* kernel);

/*
 * qlp_bls_search -- Sec. 2.1 / Eq. 1's SR: binned BLS residue at every trial frequency.
 * For each star and trial frequency f the light curve is folded (x = (t - t_min) f,
 * bin = floor(frac(x) nbins)), the weights w = dy^-2/sum(dy^-2) and w (y - ybar)
 * are histogrammed, and every cyclic window of m_j bins (durations q_j =
 * q_min e^{j dlogq}) is scored v = s^2 / (r (1 - r)), r = sum w, s = sum w (y - ybar).
 * All outputs are caller-owned device arrays of n_freq_total entries, in the
 * order of qlp_bls_plan_info's freq_offsets:
 *  sr        float: SR(f) = max v (0 when no window has 0 < r < 1).
 *  qidx      uint8: duration index j of the maximum (ties: lowest j, then lowest
 *            start bin); 255 when no window is valid. May be NULL.
 *  phase_bin uint32: first bin k of that window; 0xFFFFFFFF when none. May be NULL.
 *  s_best, r_best  float: s and r of that window. May be NULL.
 * Runs one persistent kernel over a device work queue of (star, frequency-chunk)
 * items, ordered on `stream` after the plan's own device work. Returns
 * QLP_ERR_DEVICE if a device bound was hit. Inside a stream capture of the
 * caller's own it returns QLP_ERR_CUDA unless the plan's own device work is
 * known to be complete (after qlp_bls_device_status or qlp_bls_graph_capture on
 * this plan); qlp_bls_graph_capture handles that itself.
 */
int qlp_bls_search(qlp_bls_plan_t* plan, void* stream, float* sr, uint8_t* qidx,
                   uint32_t* phase_bin, float* s_best, float* r_best);

/*
 * qlp_bls_snr -- Sec. 2.2 item 1, Eq. 1 with the two changes the paper makes:
 * S/N(f) = (SR(f) - trend(f)) / sigma_SR, trend = the spectrum median-binned in
 * N = round(1 + 3.322 log10 n) equal-width frequency bins and linearly
 * interpolated, sigma_SR = 1.4826 MAD; then the best candidate per star.
 *  sr, qidx, phase_bin, s_best, r_best  device arrays written by qlp_bls_search
 *            (all required here).
 *  snr       device float[n_freq_total] output.
 *  best      device qlp_bls_best[n_stars] output.
 */
int qlp_bls_snr(qlp_bls_plan_t* plan, void* stream, const float* sr, const uint8_t* qidx,
                const uint32_t* phase_bin, const float* s_best, const float* r_best,
                float* snr, qlp_bls_best* best);

/*
 * Learned-proposal variants (not in the paper):
 * qlp_bls_plan_windows -- as qlp_bls_plan (grid_mode 0 only), with trial
 *   frequencies only inside the star's windows: star s owns windows
 *   win_offsets[s] .. win_offsets[s+1]-1 of win_flo / win_fhi (host doubles, 1/day,
 *   inclusive). Overlapping or touching windows are merged; in each merged window,
 *   clipped to [1/Pmax, 1/Pmin], the Sec. 2.1 spacing f <- f + q_min(f)/(spp T)
 *   is walked from the window's low edge while f stays inside it. A star with no
 *   frequency inside its windows gets QLP_STAR_EMPTY_GRID.
 * qlp_bls_plan_windows_from -- the same windowed plan for the stars of an existing
 *   plan `base` (any grid mode), without their points: it takes base's validation,
 *   t_ref, Pmin, Pmax, weight spreads and cell widths, and searches base's device
 *   copy of the points (the grids, bins, paths and results are those of
 *   qlp_bls_plan_windows on the same arrays). p must be grid_mode 0 and have
 *   base's rho_default, pmin_aR and gap_days, else QLP_ERR_ARG. The new plan keeps
 *   base's device memory alive until both are destroyed (either may go first);
 *   base must not be destroyed while the call runs.
 * qlp_bls_snr_trend -- qlp_bls_snr with an optional per-star trend record
 *   (QLP_TREND_DOUBLES doubles: node count, sigma_SR, median, bin centres, bin
 *   medians) written to trend_out, or, when trend_in is given, the S/N computed
 *   from that trend and sigma instead of the spectrum's own (device arrays,
 *   n_stars records, same star order).
 * qlp_bls_coarse_tensor -- for a grid_mode 1 plan: the network input, device BF16
 *   [n_stars][n_bins][QLP_CNN_IN_CH]; on the star's searched coarse bin k channel 0
 *   is a(k) = asinh(S/N(k) / 4) and channel 1 is 1; channels 2-5 are a() at the
 *   bins of the periods 2P, P/2, 3P and P/3, k + d2, k - d2, k + d3, k - d3 with
 *   d_h = round((coarse_bins - 1) ln h / ln(coarse_pmax / coarse_pmin)) (0 where
 *   that bin is off the grid or not searched); every channel is 0 on bins not
 *   searched. n_bins must equal coarse_bins. snr_rows (device FP32
 *   [n_stars][n_bins], may be NULL) receives the S/N itself on the searched bins
 *   and 0 elsewhere (the ranking of the search without the network).
 * qlp_cnn_topk -- indices (device int32 [batch][k]) of the k largest logits of each
 *   row among bins whose x0 (BF16 [batch][len][QLP_CNN_IN_CH]) channel 1 is
 *   positive, largest first (ties: the lower bin); -1 past the last valid bin.
 */
#define QLP_TREND_DOUBLES 84
#define QLP_CNN_IN_CH 6   /* channels of the network input (qlp_bls_coarse_tensor) */
int qlp_bls_plan_windows(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets,
                         const double* t, const double* y, const double* dy, const double* rho,
                         const double* rstar, const int64_t* win_offsets, const double* win_flo,
                         const double* win_fhi, void* stream, qlp_bls_plan_t** out_plan);
int qlp_bls_plan_windows_from(const qlp_bls_plan_t* base, const qlp_bls_params* p,
                              const int64_t* win_offsets, const double* win_flo, const double* win_fhi,
                              void* stream, qlp_bls_plan_t** out_plan);
int qlp_bls_snr_trend(qlp_bls_plan_t* plan, void* stream, const float* sr, const uint8_t* qidx,
                      const uint32_t* phase_bin, const float* s_best, const float* r_best,
                      const double* trend_in, double* trend_out, float* snr, qlp_bls_best* best);
int qlp_bls_coarse_tensor(qlp_bls_plan_t* plan, void* stream, const float* snr, int32_t n_bins,
                          void* out, float* snr_rows);
/*
 * Coarse-grid arithmetic of the learned path, on the host (the same functions
 * qlp_bls_search_learned uses), for callers that sequence its stages themselves:
 * qlp_bls_coarse_periods -- periods[i] = coarse_pmin (coarse_pmax / coarse_pmin)^
 *   (x[i] / (coarse_bins - 1)) for (fractional) coarse bin positions x.
 * qlp_bls_coarse_bins -- the nearest coarse bin of each period (rounded half to
 *   even), -1 outside [0, coarse_bins) or for a period <= 0.
 * qlp_bls_proposal_windows -- frequency windows [1/P(k + half_width), 1/P(k -
 *   half_width)] around every valid (>= 0) bin k of bins (int32 [n_stars][k]),
 *   star by star: win_offsets (int64 [n_stars + 1]) always; win_lo / win_hi
 *   (double [capacity]) when given, QLP_ERR_ARG if capacity < win_offsets[n_stars].
 */
int qlp_bls_coarse_periods(const qlp_bls_params* p, int32_t n, const double* x, double* periods);
int qlp_bls_coarse_bins(const qlp_bls_params* p, int32_t n, const double* periods, int32_t* bins);
int qlp_bls_proposal_windows(const qlp_bls_params* p, int32_t n_stars, const int32_t* bins, int32_t k,
                             double half_width, int64_t* win_offsets, double* win_lo, double* win_hi,
                             int64_t capacity);
int qlp_cnn_topk(const float* logits, const void* x0, int32_t batch, int32_t len, int32_t k,
                 int32_t* out, void* stream);

/*
 * qlp_bls_run_host -- the whole path from host buffers to host results:
 * plan + upload, search, S/N, download. Arguments as for qlp_bls_plan; outputs
 * are host arrays: sr_host and snr_host float[n_freq_total] (may be NULL; the
 * caller sizes them from a previous plan of the same input or passes NULL),
 * best_host qlp_bls_best[n_stars] (required). Device memory is allocated and
 * freed inside the call. A batch of 1,024 stars or more runs in chunks of whole
 * stars (9, the first and the last with half the points of the others): the
 * host plans the next chunk while the device searches the previous ones.
 * *n_freq_total_out (may be NULL) receives the size.
 * If sr_host/snr_host are given they must hold sr_capacity floats; a larger
 * spectrum returns QLP_ERR_ARG after best_host is written.
 */
int qlp_bls_run_host(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets,
                     const double* t, const double* y, const double* dy,
                     const double* rho, const double* rstar,
                     float* sr_host, float* snr_host, int64_t sr_capacity,
                     qlp_bls_best* best_host, int64_t* n_freq_total_out);

/*
 * qlp_bls_device_status -- synchronise `stream`, return the device error flags
 * accumulated by this plan's kernels since the last call in *flags (QLP_DEVERR_*:
 * 1 the work loop hit its iteration bound, 2 a frequency needed more bins than the
 * shared histogram holds, 4 more S/N bins than supported, 32 a bulk copy of a star's
 * cell table into shared memory did not complete within its bound, 64 a 32-bit exact
 * table's prefix sum left its range) and clear them.
 * Returns QLP_ERR_DEVICE when any flag was set, else QLP_OK.
 */
int qlp_bls_device_status(qlp_bls_plan_t* plan, void* stream, int32_t* flags);

void qlp_bls_plan_destroy(qlp_bls_plan_t* plan);

/*
 * qlp_set_device_budget -- a cap on the device bytes the library's plans and
 * networks may hold at once (0 = none, the default; negative = QLP_ERR_ARG). A
 * qlp_bls_plan / qlp_cnn_create / qlp_bls_candidate_stats allocation that would
 * pass it fails before any device memory is taken and returns QLP_ERR_NOMEM,
 * exactly as an out-of-memory cudaMalloc would; everything the failing call
 * took before is released. It serves capacity control and host-side failure
 * injection (the allocation failure path is tested this way, with no GPU fault).
 * qlp_device_bytes_held -- the bytes those objects hold now.
 */
int qlp_set_device_budget(int64_t bytes);
int64_t qlp_device_bytes_held(void);

/*
 * qlp_bls_autotune -- choose the search's launch settings for a batch (an
 * implementation concern; the paper has no counterpart). Settings in *p left at
 * 0 (warps_per_block, chunk_freqs, cell_window) are tried over a small candidate
 * set; each candidate plans and searches an evenly spaced sample of up to
 * sample_stars stars (host arrays as for qlp_bls_plan) on `stream`, timed with
 * CUDA events (best of two runs after one warm-up). *out gets *p with the fastest
 * candidate's settings; results of a search never depend on them. The choice is
 * cached for the process, keyed by the device, p's other options and log2 of
 * the star count and of the median and longest star; *cached (optional) is 1
 * when the cache answered. Synchronises `stream`. Device errors as for the search.
 */
int qlp_bls_autotune(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets,
                     const double* t, const double* y, const double* dy, const double* rho,
                     const double* rstar, int32_t sample_stars, void* stream, qlp_bls_params* out,
                     int32_t* cached);

/*
 * qlp_bls_top_peaks -- the n_peaks strongest peaks of each star's S/N spectrum
 * (an extension: the paper keeps one candidate per star). Repeatedly the largest
 * S/N (ties: the lowest index) among the frequencies not excluded yet is taken,
 * and every frequency with |f / f_pick - 1| < sep is excluded (sep = 0.01 keeps
 * peaks 1 % apart in period). out: device int32 [n_stars][n_peaks], indices in
 * the star's grid, strongest first, -1 past the last. snr: device S/N from
 * qlp_bls_snr of this plan. 1 <= n_peaks <= 64.
 */
int qlp_bls_top_peaks(const qlp_bls_plan_t* plan, void* stream, const float* snr, int32_t n_peaks,
                      double sep, int32_t* out);

/*
 * qlp_bls_candidate_stats -- post-BLS statistics of every star's best candidate
 * (Sec. 2.2 items 2-5): a trapezoid fit with the period fixed to the BLS period
 * (epoch, depth, q, ingress fraction q_in, out-of-transit level z; points within
 * two BLS durations of the transit centre, weights dy^-2, 1e-6 <= q <= 1 and
 * 1e-3 <= q_in <= 0.5, Levenberg-Marquardt from the BLS box), white and red noise
 * of the residuals on the transit-duration timescale, the signal-to-pink noise
 * of Eq. 2 with the depth replaced by the trapezoid's mean depth
 * depth (1 - q_in), the point and transit counts, and the detection criteria
 * (at least two transits, S/N_pink > 9, S/N > 9).
 *  best  device qlp_bls_best[n_stars] from qlp_bls_snr / qlp_bls_snr_trend of this plan.
 *  out   device qlp_bls_cand_stats[n_stars].
 * The first call allocates a scratch array of 32 bytes per point of the plan
 * (kept by the plan). Runs on `stream`; results are valid after it.
 */
#define QLP_STATS_OK             0
#define QLP_STATS_NO_CANDIDATE   1  /* the star has no best candidate */
#define QLP_STATS_FEW_POINTS     2  /* fewer than 6 points within two durations of the transits */
#define QLP_STATS_NOT_CONVERGED  4  /* 100 iterations without meeting the stopping rule */
typedef struct qlp_bls_cand_stats {
  double t0;          /* fitted epoch: a mid-transit time (days, same scale as t) */
  double depth;       /* fitted depth delta: model y = z - delta s */
  double q;           /* fitted duration / period */
  double q_in;        /* fitted ingress duration / transit duration */
  double z;           /* fitted out-of-transit level */
  double chi2;        /* weighted chi^2 over the fit window */
  double sigma_w;     /* RMS of the residuals of all points */
  double sigma_r;     /* red noise on the timescale of one fitted duration */
  double depth_mean;  /* depth (1 - q_in): the trapezoid's mean depth over the transit */
  double snr_pink;    /* depth_mean / sqrt(sigma_w^2 / n_in + sigma_r^2 / n_transits) */
  int32_t n_fit;      /* points in the fit window */
  int32_t n_in;       /* points in transit (within half a fitted duration of a mid-transit time) */
  int32_t n_before;   /* points 0.5 to 2 durations before a mid-transit time */
  int32_t n_after;    /* points 0.5 to 2 durations after a mid-transit time */
  int32_t n_transits; /* transits with data within 0.5 durations of their mid-transit time */
  int32_t iterations; /* Levenberg-Marquardt iterations */
  int32_t status;     /* QLP_STATS_* */
  int32_t detected;   /* 1 when the detection criteria hold */
} qlp_bls_cand_stats;
int qlp_bls_candidate_stats(qlp_bls_plan_t* plan, void* stream, const qlp_bls_best* best,
                            qlp_bls_cand_stats* out);

/*
 * qlp_bls_search_multi -- several candidates per star by iterative masking (an
 * extension: the paper reports one candidate per star). Round r runs the whole
 * search (qlp_bls_plan, qlp_bls_search, qlp_bls_snr, qlp_bls_candidate_stats) on
 * the points still kept, then removes every point within one fitted transit
 * duration of the candidate's mid-transit times, |dt| < q P (fitted epoch and q
 * when the fit ran, else the BLS box); a star that finds nothing stops.
 * Arguments as for qlp_bls_plan (host arrays); outputs are host arrays:
 *  best_host   qlp_bls_best[n_planets][n_stars] (f_idx -1 after a star stopped),
 *  stats_host  qlp_bls_cand_stats[n_planets][n_stars],
 *  n_found     int32[n_stars] candidates per star (optional).
 * Device memory is allocated on `stream` and freed per round; synchronises it.
 */
int qlp_bls_search_multi(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets,
                         const double* t, const double* y, const double* dy, const double* rho,
                         const double* rstar, int32_t n_planets, void* stream, qlp_bls_best* best_host,
                         qlp_bls_cand_stats* stats_host, int32_t* n_found);

/*
 * qlp_bls_graph_capture -- record calls of this plan, with these output buffers
 * (device, as for qlp_bls_search / qlp_bls_snr), as a CUDA graph kept by the
 * plan: parts = 1 one qlp_bls_search, 2 one qlp_bls_snr, 3 the search followed by
 * the S/N (snr and best may be NULL for parts = 1). Each value of parts has its
 * own slot; capturing again replaces that slot's graph. It first waits on the
 * host for the plan's own device work; nothing runs on the GPU during the
 * capture, which uses a private stream of the plan.
 * qlp_bls_graph_launch -- replay the graph of slot `parts` on `stream` (any
 * stream, including the legacy default one): the same work and results as the
 * recorded calls, from one launch call. QLP_ERR_ARG if that slot is empty.
 * The output buffers must stay allocated while a graph may run; replays on
 * different streams must not overlap (they share the plan's work queues).
 */
int qlp_bls_graph_capture(qlp_bls_plan_t* plan, int32_t parts, float* sr, uint8_t* qidx,
                          uint32_t* phase_bin, float* s_best, float* r_best, float* snr,
                          qlp_bls_best* best);
int qlp_bls_graph_launch(qlp_bls_plan_t* plan, int32_t parts, void* stream);

/*
 * qlp_bls_star_grid -- host only, no device work: the Sec. 2.1 plan of one star,
 * exactly as qlp_bls_plan builds it (same code), for inspection and checks.
 *  n, t, y, dy   the star's points (host double[n]); rho as for qlp_bls_plan.
 *  status, pmin, pmax, t_ref, baseline   outputs, each may be NULL.
 *  n_win, win_flo, win_fhi  optional frequency windows as for qlp_bls_plan_windows
 *                (win_flo NULL = the whole grid).
 *  freqs, qmins  host double[capacity] trial frequencies and their q_min (may be NULL).
 *  n_f_out       number of trial frequencies (required).
 * Returns QLP_ERR_ARG when freqs/qmins are given and capacity < *n_f_out (the
 * scalars and *n_f_out are still written).
 */
int qlp_bls_star_grid(const qlp_bls_params* p, int64_t n, const double* t, const double* y,
                      const double* dy, double rho, int64_t n_win, const double* win_flo,
                      const double* win_fhi, int32_t* status, double* pmin, double* pmax,
                      double* t_ref, double* baseline, double* freqs, double* qmins,
                      int64_t capacity, int64_t* n_f_out);

/*
 * qlp_bls_batch_grid -- host only, no device work: the Sec. 2.1 trial-frequency
 * grids of a batch, built by the batch planner qlp_bls_plan uses (all host
 * threads, the recurrences of several stars stepped together; every grid equals
 * its one-star definition bit for bit).
 *  n_stars, offsets, t, y, dy, rho   the batch, as for qlp_bls_plan.
 *  star_status   host int32[n_stars] per-star status (may be NULL).
 *  freq_offsets  host int64[n_stars + 1] (required): star s owns
 *                freqs[freq_offsets[s] .. freq_offsets[s + 1]); stars with a
 *                non-zero status own none.
 *  freqs         host double[capacity] (may be NULL).
 * Returns QLP_ERR_ARG when freqs is given and capacity < freq_offsets[n_stars]
 * (freq_offsets and star_status are still written).
 */
int qlp_bls_batch_grid(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets, const double* t,
                       const double* y, const double* dy, const double* rho, int32_t* star_status,
                       int64_t* freq_offsets, double* freqs, int64_t capacity);

/*
 * qlp_bls_search_static -- the paper has no counterpart of this entry point.
 * The BLS search of ONE star (qlp_bls_search's results for that star) without
 * allocating any device memory, for callers that may not call cudaMalloc: code
 * that runs inside a host framework which owns every device allocation, or a
 * service whose device memory is fixed before work starts.
 * The scratch the search needs (prepared points, frequency table, work queue)
 * is a library-owned static device array of QLP_STATIC_SCRATCH_BYTES (16 MiB),
 * present on every GPU that loads the library until the process exits. A call
 * whose sizes do not fit (about 24 bytes per point plus 32 bytes per trial
 * frequency, e.g. 300,000 points and 200,000 frequencies) returns QLP_ERR_ARG.
 * The first call on each device looks up the array's device address with that
 * device current; make that first call before any stream capture. All calls
 * share the one array and it keeps the previous call's contents (each call
 * clears what must start at zero): calls that overlap on the GPU (different
 * streams or threads) race, so serialise them.
 *  p            parameters (NULL = defaults); nbins_cap, phase/sum mode, warps,
 *               chunk and tile options apply as for qlp_bls_plan.
 *  n            number of valid points (>= 2).
 *  tp, y, dy    device double[n], caller-owned: t' = t - t_min sorted ascending,
 *               flux and 1-sigma error of the star's valid points (as
 *               qlp_bls_star_grid keeps them).
 *  baseline     t'[n-1] (days).
 *  n_f, freqs, qmins  host double[n_f]: the star's trial frequencies and their
 *               q_min, e.g. from qlp_bls_star_grid.
 *  stream       cudaStream_t (NULL = default stream).
 *  sr, qidx, phase_bin, s_best, r_best  device outputs of n_f entries, as for
 *               qlp_bls_search (qidx, phase_bin, s_best, r_best may be NULL). A
 *               frequency the kernel could not search (its bin count beyond the
 *               histogram it sized) keeps sr = 0, qidx = 255, phase_bin =
 *               0xFFFFFFFF and raises QLP_DEVERR_NBINS in flags.
 *  flags        device int32 (may be NULL): receives, on `stream`, this call's
 *               device error bits (0 = clean; QLP_DEVERR_NBINS, QLP_DEVERR_QUEUE),
 *               the same bits qlp_bls_device_status reports for a plan.
 * Only the shared histogram of Sec. 2.1 (bin_mode QLP_BIN_SHARED): any other
 * bin_mode returns QLP_ERR_UNSUPPORTED. warps_per_block 32 runs as 16, as the
 * point path of qlp_bls_plan does.
 * Asynchronous on `stream`; results and flags are valid after it is synchronised.
 */
#define QLP_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
int qlp_bls_search_static(const qlp_bls_params* p, int32_t n, const double* tp, const double* y,
                          const double* dy, double baseline, int32_t n_f, const double* freqs,
                          const double* qmins, void* stream, float* sr, uint8_t* qidx,
                          uint32_t* phase_bin, float* s_best, float* r_best, int32_t* flags);

/* ---------------------------------------------------------------- learned path
 * Not in the paper: a small 1-D CNN proposes period windows from a coarse BLS
 * spectrum. The layers below are its building blocks (all device pointers,
 * caller-owned, asynchronous on `stream`).
 *
 * qlp_cnn_pack_w64 -- w: FP32 [9][64][64] weights (tap, out channel, in channel);
 *   wpack: 73,728-byte device buffer at a 16-byte boundary receiving them as BF16 in
 *   the tensor-core layout (per tap 64 rows of 128 bytes, 128-byte swizzle);
 *   transpose = 1 packs the input-gradient form W'[k][ci][co] = W[8-k][co][ci].
 * qlp_cnn_conv64 -- y[b][l][co] = epi(sum_k sum_ci W[k][co][ci] x[b][l+k-4][ci]) for
 *   BF16 channels-last x, y [batch][len][64], len a multiple of 128, zero padding;
 *   epi adds bias (FP32 [64], or NULL), applies ReLU when relu != 0, and zeroes
 *   entries where mask (BF16 [batch][len][64], or NULL) is not positive. err: a
 *   device int32 that receives QLP error bits (16 = a tensor-core wait hit its bound).
 *   x, wpack and y start at 16-byte boundaries (else QLP_ERR_ARG).
 */
int qlp_cnn_pack_w64(const float* w, void* wpack, int32_t transpose, void* stream);
/*
 * qlp_cnn_conv64_wgrad -- weight and bias gradients of one 64 -> 64 layer on the
 * tensor cores: out[(kk 64 + co) 64 + ci] = sum_p dy[p][co] x[p + kk - 4][ci]
 * (zero outside each sample), out[9 64 64 + co] = sum_p dy[p][co]; dy and x BF16
 * [batch][len][64] (device), len a multiple of 128, out FP32 [36928] (device).
 * workspace: device FP32 of qlp_cnn_wgrad64_workspace(batch, len) floats.
 * Device wait timeouts set bit 16 in *err (device int32).
 */
int64_t qlp_cnn_wgrad64_workspace(int32_t batch, int32_t len);
int qlp_cnn_conv64_wgrad(const void* dy, const void* x, float* workspace, float* out, int32_t batch,
                         int32_t len, int32_t* err, void* stream);
int qlp_cnn_conv64(const void* x, const void* wpack, const float* bias, const void* mask, void* y,
                   int32_t batch, int32_t len, int32_t relu, int32_t* err, void* stream);

/*
 * The network: input x0 BF16 [batch][len][QLP_CNN_IN_CH] (as qlp_bls_coarse_tensor
 * writes it: the coarse S/N, the valid-bin mask, the S/N at the bins of 2P, P/2, 3P
 * and P/3), conv(6->64)+ReLU, 4 x [conv(64->64)+ReLU], conv(64->1): one logit per
 * bin, kernel 9, zero padding, len a multiple of 128.
 * Parameters (FP32, qlp_cnn_n_params() of them) in the order
 *   W1 [9][64][6], b1 [64], (W_k [9][64][64], b_k [64]) for k = 2..5, W6 [9][64], b6,
 * with W[tap][out channel][in channel]. Weights are the FP32 masters of Adam; the
 * 64->64 layers compute with BF16 copies on the tensor cores, activations are
 * BF16, accumulation FP32.
 * qlp_cnn_create     network for batches of up to max_batch, He-normal initial
 *                    weights from `seed` (counter-based generator), output bias -4.
 * qlp_cnn_forward    logits (device FP32 [batch][len], may be NULL: kept inside).
 * qlp_cnn_backward   forward, then the weighted BCE with logits averaged over
 *                    batch x len (labels device FP32 [batch][len] in {0, 1};
 *                    positives weighted by pos_weight) and every parameter
 *                    gradient, kept inside the network.
 * qlp_cnn_adam_step  Adam (beta 0.9, 0.999, eps 1e-8, bias-corrected) on the masters.
 * qlp_cnn_train_step backward + Adam.
 * qlp_cnn_loss       synchronises `stream`; last loss and the device error bits.
 * qlp_cnn_get_params / qlp_cnn_set_params  host copies of the parameters (and of
 *                    the last gradients); set resets Adam's moments.
 */
typedef struct qlp_cnn qlp_cnn_t;
int32_t qlp_cnn_n_params(void);
int qlp_cnn_create(int32_t max_batch, int32_t len, uint64_t seed, qlp_cnn_t** out);
void qlp_cnn_destroy(qlp_cnn_t* net);
int qlp_cnn_set_params(qlp_cnn_t* net, const float* host, void* stream);
int qlp_cnn_get_params(const qlp_cnn_t* net, float* host, float* grads_host, void* stream);
int qlp_cnn_forward(qlp_cnn_t* net, const void* x0, int32_t batch, float* logits, void* stream);
int qlp_cnn_backward(qlp_cnn_t* net, const void* x0, const float* labels, int32_t batch,
                     float pos_weight, void* stream);
int qlp_cnn_adam_step(qlp_cnn_t* net, float lr, void* stream);
int qlp_cnn_train_step(qlp_cnn_t* net, const void* x0, const float* labels, int32_t batch,
                       float pos_weight, float lr, void* stream);
int qlp_cnn_loss(qlp_cnn_t* net, float* loss_host, int32_t* err_host, void* stream);
const char* qlp_cnn_last_error(void);

/*
 * qlp_cnn_get_tensor  host copy of a tensor the last forward / backward kept, for
 *                checks of each layer on its own inputs: which = QLP_CNN_ACT (BF16
 *                [batch][len][64] output of layer 1..5 after its ReLU),
 *                QLP_CNN_GACT (BF16 [batch][len][64] loss gradient of the
 *                pre-activation of layer 1..5), QLP_CNN_LOGIT (FP32 [batch][len]
 *                logits; layer ignored) or QLP_CNN_DLOGIT (FP32 [batch][len] loss
 *                gradient of the logits). batch <= max_batch rows are copied into
 *                host (bytes >= the tensor's size, else QLP_ERR_ARG); synchronises
 *                `stream`.
 * qlp_cnn_shape  the max_batch and len the network was created with.
 * qlp_cnn_save   checkpoint to a file: the parameters, Adam's two moment vectors
 *                and its step count (FP32 little-endian after a short header);
 *                synchronises `stream`. QLP_ERR_ARG when the file cannot be written.
 * qlp_cnn_load   restore a checkpoint written by qlp_cnn_save into a network of
 *                any max_batch and len (the parameters do not depend on them);
 *                training resumes where it stopped. QLP_ERR_ARG for a missing file
 *                or one of another layout; the network is unchanged then.
 */
#define QLP_CNN_ACT 0
#define QLP_CNN_GACT 1
#define QLP_CNN_LOGIT 2
#define QLP_CNN_DLOGIT 3
int qlp_cnn_get_tensor(const qlp_cnn_t* net, int32_t which, int32_t layer, int32_t batch, void* host,
                       int64_t bytes, void* stream);
int qlp_cnn_shape(const qlp_cnn_t* net, int32_t* max_batch, int32_t* len);
int qlp_cnn_save(const qlp_cnn_t* net, const char* path, void* stream);
int qlp_cnn_load(qlp_cnn_t* net, const char* path, void* stream);

/*
 * qlp_bls_search_learned -- the learned period proposal (an addition to the
 * paper: it narrows the full-grid search of Sec. 2.1 to the periods a network
 * proposes). From host light curves (arguments as for qlp_bls_plan):
 *   1. the coarse spectrum: plan with grid_mode 1 (p's coarse_* fields), search,
 *      S/N with its trend record (Sec. 2.2 item 1), the network input tensor;
 *   2. the network's logits and each star's top-k valid coarse bins;
 *   3. frequency windows [1/P(k_b + half_width), 1/P(k_b - half_width)] around each
 *      proposed bin k_b, P(x) = coarse_pmin (coarse_pmax/coarse_pmin)^(x/(coarse_bins-1));
 *   4. the paper's grid (grid_mode 0) restricted to those windows, searched, and
 *      scored with the coarse trend and sigma_SR.
 * net must have len == coarse_bins; net = NULL ranks the coarse bins by their S/N
 * itself instead (the same path without the network, its ablation). best_host
 * (n_stars records, required) gets the
 * best candidate of step 4 (f_idx indexes the windowed grid; a star with no grid
 * frequency in its windows gets f_idx -1 and QLP_STAR_EMPTY_GRID). bins_host
 * (int32 [n_stars][k], optional) gets the proposed bins, -1 past a star's last
 * valid bin. Device scratch is allocated on `stream` and freed before return; the
 * call synchronises `stream`. QLP_ERR_DEVICE when a kernel raised an error flag.
 */
int qlp_bls_search_learned(const qlp_bls_params* p, int32_t n_stars, const int64_t* offsets,
                           const double* t, const double* y, const double* dy, const double* rho,
                           const double* rstar, qlp_cnn_t* net, int32_t k, double half_width,
                           void* stream, qlp_bls_best* best_host, int32_t* bins_host);

/* Static description of a return code. */
const char* qlp_strerror(int code);

/* Text of the last CUDA error seen by the library in this thread ("" if none). */
const char* qlp_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QLP_BLS_H */
