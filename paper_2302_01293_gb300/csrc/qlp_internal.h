// Internal layouts shared by the host planner, the C-ABI glue and the kernels.
#pragma once

#include <cstdint>

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
  int32_t pad0;
  double t_ref;        // t_min of the valid points
  double baseline;     // t_max - t_min
};

// (star, frequency chunk) unit of the device work queue.
struct WorkItem {
  int32_t star;
  int32_t f_begin;     // first frequency, relative to the star
  int32_t f_count;
  int32_t pad0;
};

struct BlsArgs {
  const StarDev* stars;
  const double2* fq;       // per frequency: (f, q_min)
  const WorkItem* items;
  int32_t n_items;
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
  double noverlap;
  double E[kMaxQ];
  int32_t nq;
  int32_t mad_mode;
  int32_t n_stars;
  int32_t pad0;
};

// device error flags
constexpr int32_t kErrQueueBound = 1;   // work loop exceeded its iteration bound
constexpr int32_t kErrNbins = 2;        // a frequency needed more bins than the histogram holds
constexpr int32_t kErrSturges = 4;      // more S/N bins than the kernel supports
constexpr int32_t kErrSelect = 8;       // median selection failed to converge

// launchers (bls_kernels.cu / snr_kernel.cu); return cudaError_t as int
int launch_prep(const PrepArgs& a, void* stream);
int launch_bls(const BlsArgs& a, int phase_mode, int sum_mode, int warps, int blocks,
               size_t smem_bytes, void* stream);
int launch_snr(const SnrArgs& a, void* stream);
int bls_max_smem_per_block();
int bls_blocks_per_sm(int phase_mode, int sum_mode, int warps, size_t smem_bytes);

}  // namespace qlp
