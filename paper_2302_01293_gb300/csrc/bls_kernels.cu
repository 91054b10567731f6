// Point preparation (K1) and the persistent BLS search kernel (K2) for sm_103a.
//
// K1 (BLS normalisation, Kovacs et al. 2002, as adopted in Sec. 2.1 of
// arXiv:2302.01293): per star W = sum dy^-2, w = dy^-2 / W, ybar = sum w y and the
// packed point (t'_hi, t'_lo, w (y - ybar), w), t' = t - t_min split into a
// double-float pair, written in a tile-transposed order so that in every tile of
// `tile_pts` points lane l of a warp walks the contiguous run of points
// l*S .. l*S+S-1 (S = tile rows) with conflict-free 16-byte shared loads.
//
// K2 (Sec. 2.1, Eq. 1's SR): a persistent kernel; each CTA pops (star,
// frequency-chunk) items from a device queue, stages the star's points in shared
// memory, and each warp takes one trial frequency at a time:
//   fold    g = floor(t' f nbins) (global bin index), bin b = g mod nbins;
//           double-float product with a guard band: a point whose fractional bin
//           coordinate lies within the band of an edge is re-folded with the
//           exact FP64 sequence x = t' f, b = floor(frac(x) nbins), so the bin
//           equals the FP64 one;
//   bin     consecutive points of a lane fall in the same bin for a while (the
//           lane's points are contiguous in time), so runs are summed in
//           registers and flushed to the warp's shared histogram with one
//           atomic add per run and array (optionally with the exact TwoSum error
//           of each add kept in a second array);
//   boxes   every cyclic window of m_j bins, s^2 / (r (1 - r)), maximum with ties
//           to the lowest duration index and then the lowest start bin, reduced
//           over the warp by shuffles.
#include <cuda_runtime.h>

#include <cstdint>

#include "bls_device.cuh"
#include "qlp_internal.h"

namespace qlp {

// ------------------------------------------------------------------ K1 prep

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double tot = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < nw; ++i) tot += red[i];
  return tot;
}

__global__ void __launch_bounds__(256) prep_kernel(const PrepArgs a) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  const StarDev st = a.stars[s];
  const int n = st.n_pts;
  if (n <= 0 || st.method != kMethodPoints) return;
  const double* tp = a.tp + st.pt_off;
  const double* y = a.y + st.pt_off;
  const double* dy = a.dy + st.pt_off;

  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += 1.0 / (dy[i] * dy[i]);
  const double wsum = block_sum_d(acc, red);
  acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += (1.0 / (dy[i] * dy[i])) / wsum * y[i];
  const double ybar = block_sum_d(acc, red);

  const int npad = (n + 31) & ~31;
  const int TP = a.tile_pts;
  for (int p = threadIdx.x; p < npad; p += blockDim.x) {
    const int ti = p / TP;
    const int q = p - ti * TP;
    const int tile_n = min(TP, npad - ti * TP);
    const int S = tile_n >> 5;
    const int slot = ti * TP + (q % S) * 32 + q / S;
    const int src = p < n ? p : n - 1;
    const double t = tp[src];
    float w = 0.f, wd = 0.f;
    if (p < n) {
      const double ww = (1.0 / (dy[p] * dy[p])) / wsum;
      w = (float)ww;
      wd = (float)(ww * (y[p] - ybar));
    }
    const float th = __double2float_rn(t);
    const float tl = __double2float_rn(t - (double)th);
    a.pts[st.pad_off + slot] = make_float4(th, tl, wd, w);
    a.tpd[st.pad_off + slot] = t;
  }
}

int launch_prep(const PrepArgs& a, void* stream) {
  if (a.n_stars <= 0) return 0;
  prep_kernel<<<a.n_stars, 256, 0, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ K2 search

template <int PHASE, int SUM, int NW>
__global__ void __launch_bounds__(NW * 32) bls_kernel(const BlsArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NA = (SUM == QLP_SUM_COMP) ? 4 : 2;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int HS = a.hist_stride;
  float* hw = reinterpret_cast<float*>(smem) + (size_t)warp * NA * HS;
  float* hy = hw + HS;
  float* hwc = hw + 2 * HS;
  float* hyc = hw + 3 * HS;
  int* mtab = reinterpret_cast<int*>(smem + (size_t)NW * NA * HS * sizeof(float)) + warp * kMaxQ;
  unsigned char* tile = smem + a.tile_off;
  const int TP = a.tile_pts;
  const int nq = a.nq;

  __shared__ int s_item;
  __shared__ int s_star;
  __shared__ int s_tile;
  if (threadIdx.x == 0) { s_star = -1; s_tile = -1; }

  bool done = false;
  const int iter_lim = a.loop_bound > 0 ? min(a.loop_bound, a.n_items) : a.n_items;
  for (int iter = 0; iter <= iter_lim; ++iter) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.cursor, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= a.n_items) { done = true; break; }
    const WorkItem wi = a.items[it];
    const StarDev st = a.stars[wi.star];
    const int n = st.n_pts;
    const int npad = (n + 31) & ~31;
    const int n_tiles = (npad + TP - 1) / TP;
    const bool star_fp64 = (PHASE == QLP_PHASE_FP64) || (st.fp64_phase != 0);

    for (int r0 = 0; r0 < wi.f_count; r0 += NW) {
      const int fl = r0 + warp;
      bool active = fl < wi.f_count;
      const int64_t fidx = st.f_off + wi.f_begin + (active ? fl : 0);
      double f = 0.0;
      int nb = 1;
      float Fh = 0.f, Fl = 0.f, fh = 0.f, band = 0.f;
      if (active) {
        const double2 fq = a.fq[fidx];
        f = fq.x;
        nb = (int)ceil(__ddiv_rn(a.noverlap, fq.y));
        if (nb + kMPad > HS || nb < 1) {
          if (lane == 0) {
            atomicOr(a.err, kErrNbins);
            a.sr[fidx] = 0.f;
            if (a.qidx) a.qidx[fidx] = 255;
            if (a.kbin) a.kbin[fidx] = 0xffffffffu;
            if (a.sbest) a.sbest[fidx] = 0.f;
            if (a.rbest) a.rbest[fidx] = 0.f;
          }
          active = false;
        } else {
          if (lane < nq)
            mtab[lane] = max(1, (int)floor(__dadd_rn(__dmul_rn(__dmul_rn(fq.y, a.E[lane]),
                                                                (double)nb), 0.5)));
          const double F = __dmul_rn(f, (double)nb);
          Fh = __double2float_rn(F);
          Fl = __double2float_rn(__dsub_rn(F, (double)Fh));
          fh = __double2float_rn(f);
          // guard band (bin units): rounding of the FP32 remainder (<= 2^-20 for |r| < 8)
          // plus the double-float and FP64 product errors (<= 2^-40 of the largest t'f nbins)
          band = (float)(9.5367431640625e-07 + 9.094947017729282e-13 * __dmul_rn(st.baseline, F));
          for (int i = lane; i < nb + kMPad; i += 32) {
            hw[i] = 0.f;
            hy[i] = 0.f;
            if (SUM == QLP_SUM_COMP) { hwc[i] = 0.f; hyc[i] = 0.f; }
          }
        }
      }
      __syncwarp();

      for (int ti = 0; ti < n_tiles; ++ti) {
        const int tile_n = min(TP, npad - ti * TP);
        if (s_star != wi.star || s_tile != ti) {  // block-uniform
          __syncthreads();
          const int64_t g0 = st.pad_off + (int64_t)ti * TP;
          if (PHASE == QLP_PHASE_FP64) {
            double* dt = reinterpret_cast<double*>(tile);
            float2* dv = reinterpret_cast<float2*>(tile + (size_t)TP * sizeof(double));
            for (int i = threadIdx.x; i < tile_n; i += NW * 32) {
              dt[i] = a.tpd[g0 + i];
              const float4 p = a.pts[g0 + i];
              dv[i] = make_float2(p.z, p.w);
            }
          } else {
            float4* dp = reinterpret_cast<float4*>(tile);
            for (int i = threadIdx.x; i < tile_n; i += NW * 32) dp[i] = a.pts[g0 + i];
          }
          if (threadIdx.x == 0) { s_star = wi.star; s_tile = ti; }
          __syncthreads();
        }
        if (!active) continue;

        const int S = tile_n >> 5;
        const int64_t gbase = st.pad_off + (int64_t)ti * TP;
        RunAcc<SUM> acc;
        acc.reset();
        int bcur = -1;
        int gc = 0;  // first global bin of the lane's current cycle
        // kU points per lane per step: their folds are independent (ILP); the
        // run/flush logic then consumes them in time order.
        for (int k0 = 0; k0 < S; k0 += kU) {
          float wv[kU], wdv[kU];
          int gv[kU];
          bool need[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int k = k0 + u < S ? k0 + u : k0;  // in-bounds slot; results unused past S
            const int slot = k * 32 + lane;
            need[u] = false;
            if (PHASE == QLP_PHASE_FP64) {
              const double t = reinterpret_cast<const double*>(tile)[slot];
              const float2 v = reinterpret_cast<const float2*>(tile + (size_t)TP * sizeof(double))[slot];
              wdv[u] = v.x;
              wv[u] = v.y;
              int c;
              const int bb = fold_fp64(t, f, nb, &c);
              gv[u] = c * nb + bb;
            } else if (PHASE == QLP_PHASE_FP32) {
              const float4 p = reinterpret_cast<const float4*>(tile)[slot];
              wdv[u] = p.z;
              wv[u] = p.w;
              const float x = __fmul_rn(p.x, fh);
              const float fr = __fsub_rn(x, floorf(x));
              gv[u] = min(nb - 1, (int)__fmul_rn(fr, (float)nb));
            } else {
              const float4 p = reinterpret_cast<const float4*>(tile)[slot];
              wdv[u] = p.z;
              wv[u] = p.w;
              // y = t' F as an unevaluated pair (ph, e); F = f nbins as (Fh, Fl)
              const float ph = __fmul_rn(p.x, Fh);
              float e = __fmaf_rn(p.x, Fh, -ph);
              e = __fmaf_rn(p.x, Fl, e);
              e = __fmaf_rn(p.y, Fh, e);
              const float m1 = __fadd_rn(ph, kMagic);
              const float pr = __fsub_rn(m1, kMagic);           // round(ph)
              const float r = __fadd_rn(__fsub_rn(ph, pr), e);  // y - round(ph), |r| < 2
              const float m2 = __fadd_rn(r, kMagic);
              const float rn = __fsub_rn(m2, kMagic);           // round(r)
              int ri = __float_as_int(m2) - kMagicBits;
              if (rn > r) ri -= 1;                              // floor(r)
              gv[u] = (__float_as_int(m1) - kMagicBits) + ri;
              need[u] = star_fp64 || (fabsf(__fsub_rn(r, rn)) <= band);
            }
          }
          if (PHASE == QLP_PHASE_DF) {
            bool anyn = false;
#pragma unroll
            for (int u = 0; u < kU; ++u) anyn |= need[u];
            if (__any_sync(0xffffffffu, anyn)) {  // rare: re-fold near-edge points in FP64
#pragma unroll
              for (int u = 0; u < kU; ++u) {
                const int k = k0 + u < S ? k0 + u : k0;
                if (need[u]) gv[u] = exact_global_bin(a.tpd + gbase + k * 32 + lane, f, nb);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            if (k0 + u >= S) break;  // warp-uniform
            int b;
            if (PHASE == QLP_PHASE_FP32) {
              b = gv[u];
            } else {
              const int g = max(gv[u], 0);  // t' >= 0: the global bin is never negative
              b = g - gc;
              const bool next = b >= nb;    // the lane moved on by one cycle: common
              b = next ? b - nb : b;
              gc = next ? gc + nb : gc;
              if ((unsigned)b >= (unsigned)nb) {  // first point or a gap of cycles: rare
                gc = (g / nb) * nb;
                b = g - gc;
              }
            }
            const bool ch = b != bcur;
            flush_run<SUM>(hw, hy, hwc, hyc, bcur, acc, ch && bcur >= 0);
            acc.add(ch, wv[u], wdv[u]);
            bcur = b;
          }
        }
        flush_run<SUM>(hw, hy, hwc, hyc, bcur, acc, bcur >= 0);
      }
      if (!active) continue;
      __syncwarp();

      sweep_store<SUM>(hw, hy, hwc, hyc, mtab, nq, nb, lane, fidx, a.sr, a.qidx, a.kbin, a.sbest,
                       a.rbest);
    }
  }
  if (!done && threadIdx.x == 0) atomicOr(a.err, kErrQueueBound);
}

template <int PHASE, int SUM, int NW>
static int launch_t(const BlsArgs& a, int blocks, size_t smem, void* stream) {
  auto kern = bls_kernel<PHASE, SUM, NW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  kern<<<blocks, NW * 32, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

template <int PHASE, int SUM, int NW>
static int occupancy_t(size_t smem) {
  auto kern = bls_kernel<PHASE, SUM, NW>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NW * 32, smem) != cudaSuccess) return 0;
  return nb;
}

#define QLP_DISPATCH(FN, ...)                                                          \
  switch (phase_mode * 100 + sum_mode * 10 + (warps == 4 ? 0 : warps == 8 ? 1 : 2)) { \
    case 0: return FN<0, 0, 4>(__VA_ARGS__);                                           \
    case 1: return FN<0, 0, 8>(__VA_ARGS__);                                           \
    case 2: return FN<0, 0, 16>(__VA_ARGS__);                                          \
    case 10: return FN<0, 1, 4>(__VA_ARGS__);                                          \
    case 11: return FN<0, 1, 8>(__VA_ARGS__);                                          \
    case 12: return FN<0, 1, 16>(__VA_ARGS__);                                         \
    case 100: return FN<1, 0, 4>(__VA_ARGS__);                                         \
    case 101: return FN<1, 0, 8>(__VA_ARGS__);                                         \
    case 102: return FN<1, 0, 16>(__VA_ARGS__);                                        \
    case 110: return FN<1, 1, 4>(__VA_ARGS__);                                         \
    case 111: return FN<1, 1, 8>(__VA_ARGS__);                                         \
    case 112: return FN<1, 1, 16>(__VA_ARGS__);                                        \
    case 200: return FN<2, 0, 4>(__VA_ARGS__);                                         \
    case 201: return FN<2, 0, 8>(__VA_ARGS__);                                         \
    case 202: return FN<2, 0, 16>(__VA_ARGS__);                                        \
    case 210: return FN<2, 1, 4>(__VA_ARGS__);                                         \
    case 211: return FN<2, 1, 8>(__VA_ARGS__);                                         \
    case 212: return FN<2, 1, 16>(__VA_ARGS__);                                        \
    default: break;                                                                    \
  }

int launch_bls(const BlsArgs& a, int phase_mode, int sum_mode, int warps, int blocks,
               size_t smem_bytes, void* stream) {
  QLP_DISPATCH(launch_t, a, blocks, smem_bytes, stream)
  return (int)cudaErrorInvalidValue;
}

int bls_blocks_per_sm(int phase_mode, int sum_mode, int warps, size_t smem_bytes) {
  QLP_DISPATCH(occupancy_t, smem_bytes)
  return 0;
}

int bls_max_smem_per_block() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return v;
}

}  // namespace qlp
