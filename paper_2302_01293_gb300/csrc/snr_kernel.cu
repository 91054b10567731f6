// Spectral S/N and best candidate (K3), one CTA per star, for sm_103a.
//
// Sec. 2.2 item 1 of arXiv:2302.01293, Eq. 1 with the paper's two changes:
//   trend(f)  the SR spectrum median-binned into N = round(1 + 3.322 log10 n)
//             equal-width frequency bins (Sturges), bin medians placed at the bin
//             centres and linearly interpolated (constant beyond the end centres);
//   sigma_SR  1.4826 x median |SR - median(SR)| (or of the detrended residual);
//   S/N(f)    (SR(f) - trend(f)) / sigma_SR;
// then the best candidate at the first maximum of S/N (Sec. 2.2 item 2 takes its
// BLS box as the initial P, T0, q and depth).
// Medians are exact order statistics of the FP32 spectrum, found by a 4-pass
// 8-bit radix select over order-preserving integer keys, all selections of one
// pass sharing a pass over the spectrum (shared-memory digit histograms).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "qlp_internal.h"

namespace qlp {

constexpr int kSnrThreads = 512;
constexpr int kMaxTargets = 2 * (kMaxSturges + 1);

__device__ __forceinline__ uint32_t fkey(float v) {
  const uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fdekey(uint32_t k) {
  const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

// Sturges bin of spectrum entry k: min(N-1, floor((f_k - f_0) N / span)).
__device__ __forceinline__ int sturges_bin(double f, double f0, double span, int nbin) {
  if (!(span > 0.0)) return 0;
  const int i = (int)floor(__ddiv_rn(__dmul_rn(__dsub_rn(f, f0), (double)nbin), span));
  return min(nbin - 1, i);
}

struct SnrShared {
  int lo[kMaxSturges + 1];     // first spectrum index of each Sturges bin (lo[N] = n)
  double xs[kMaxSturges];      // centres of the non-empty bins
  double ys[kMaxSturges];      // their medians
  int nx;
  uint32_t prefix[kMaxTargets];
  int rank[kMaxTargets];
  uint32_t mask;
  double med, sigma;
  float best_v[kSnrThreads / 32];
  int best_i[kSnrThreads / 32];
};

// Trend at frequency f from the (xs, ys) nodes, np.interp semantics.
__device__ __forceinline__ double trend_at(const SnrShared& sh, double f) {
  const int nx = sh.nx;
  if (f <= sh.xs[0]) return sh.ys[0];
  if (f >= sh.xs[nx - 1]) return sh.ys[nx - 1];
  int lo = 0, hi = nx - 1;  // xs[lo] <= f < xs[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (sh.xs[mid] <= f) lo = mid; else hi = mid;
  }
  const double slope = __ddiv_rn(__dsub_rn(sh.ys[lo + 1], sh.ys[lo]), __dsub_rn(sh.xs[lo + 1], sh.xs[lo]));
  return __dadd_rn(sh.ys[lo], __dmul_rn(slope, __dsub_rn(f, sh.xs[lo])));
}

__device__ __forceinline__ int bin_of_index(const SnrShared& sh, int k, int nbin) {
  int lo = 0, hi = nbin;  // lo[lo] <= k < lo[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (sh.lo[mid] <= k) lo = mid; else hi = mid;
  }
  return lo;
}

// Radix selection of the rank[t]-th smallest key for targets t in [0, nt);
// KeyOf(k, &key, &tgt0, &ntg) gives entry k's key and its targets tgt0 .. tgt0+ntg-1
// plus the two global targets handled by `global_t` (-1 = none).
template <typename KeyOf>
__device__ void radix_select(SnrShared& sh, uint32_t* hist, int nt, int n, KeyOf key_of) {
  for (int t = threadIdx.x; t < nt; t += blockDim.x) sh.prefix[t] = 0u;
  if (threadIdx.x == 0) sh.mask = 0u;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int i = threadIdx.x; i < nt * 256; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const uint32_t mask = sh.mask;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      uint32_t key;
      int t0, t1;
      key_of(k, &key, &t0, &t1);
      const uint32_t dig = (key >> shift) & 255u;
      if (t0 >= 0) {
        if ((key & mask) == sh.prefix[t0]) atomicAdd(&hist[t0 * 256 + dig], 1u);
        if ((key & mask) == sh.prefix[t0 + 1]) atomicAdd(&hist[(t0 + 1) * 256 + dig], 1u);
      }
      if (t1 >= 0) {
        if ((key & mask) == sh.prefix[t1]) atomicAdd(&hist[t1 * 256 + dig], 1u);
        if ((key & mask) == sh.prefix[t1 + 1]) atomicAdd(&hist[(t1 + 1) * 256 + dig], 1u);
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
      int r = sh.rank[t];
      if (r < 0) continue;
      uint32_t d = 0;
      for (; d < 256; ++d) {
        const int c = (int)hist[t * 256 + d];
        if (r < c) break;
        r -= c;
      }
      sh.rank[t] = r;
      sh.prefix[t] |= (d & 255u) << shift;
    }
    __syncthreads();
    if (threadIdx.x == 0) sh.mask |= 255u << shift;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSnrThreads) snr_kernel(const SnrArgs a) {
  extern __shared__ __align__(16) uint32_t hist[];
  __shared__ SnrShared sh;
  const int s = blockIdx.x;
  const StarDev st = a.stars[s];
  const int n = st.n_f;
  qlp_bls_best* out = a.best + s;

  if (n <= 0 || st.status != 0) {
    if (threadIdx.x == 0 && a.trend_out)
      for (int i = 0; i < kTrendDoubles; ++i) a.trend_out[(size_t)s * kTrendDoubles + i] = 0.0;
    if (threadIdx.x == 0) {
      out->f_idx = -1;
      out->f = out->period = out->t0 = out->q = out->depth = out->sr = out->snr = 0.0;
      out->j = out->k = out->m = out->nbins = -1;
      out->status = st.status;
      out->pad = 0;
    }
    return;
  }
  const int nbin = st.sturges_nb;
  if (nbin < 1 || nbin > kMaxSturges) {
    if (threadIdx.x == 0) {
      atomicOr(a.err, kErrSturges);
      out->f_idx = -1;
      out->status = st.status;
    }
    return;
  }
  const float* sr = a.sr + st.f_off;
  const double2* fq = a.fq + st.f_off;
  float* snr = a.snr + st.f_off;
  const double f0 = fq[0].x;
  const double span = __dsub_rn(fq[n - 1].x, f0);

  if (a.trend_in) {
    // S/N from a given trend and sigma (the refined search of the learned proposal)
    const double* tr = a.trend_in + (size_t)s * kTrendDoubles;
    for (int i = threadIdx.x; i < kMaxSturges; i += blockDim.x) {
      sh.xs[i] = tr[4 + i];
      sh.ys[i] = tr[4 + kMaxSturges + i];
    }
    if (threadIdx.x == 0) {
      sh.nx = (int)tr[0];
      sh.sigma = tr[1];
      sh.med = tr[2];
    }
    __syncthreads();
    if (sh.nx < 1) {
      if (threadIdx.x == 0) {
        out->f_idx = -1;
        out->status = st.status | QLP_STAR_ZERO_MAD;
        out->f = out->period = out->t0 = out->q = out->depth = out->sr = out->snr = 0.0;
        out->j = out->k = out->m = out->nbins = -1;
        out->pad = 0;
      }
      for (int k = threadIdx.x; k < n; k += blockDim.x) snr[k] = 0.f;
      return;
    }
  } else {
  // bin boundaries: lo[i] = first k with bin(k) >= i
  for (int i = threadIdx.x; i <= nbin; i += blockDim.x) {
    int lo = 0, hi = n;
    if (i == 0) hi = 0;
    else if (i == nbin) lo = n;
    else {
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sturges_bin(fq[mid].x, f0, span, nbin) >= i) hi = mid; else lo = mid + 1;
      }
    }
    sh.lo[i] = lo;
  }
  __syncthreads();

  // medians of every bin (targets 2i, 2i+1) and of the whole spectrum (2N, 2N+1)
  const int tg = 2 * nbin;
  for (int i = threadIdx.x; i <= nbin; i += blockDim.x) {
    const int c = (i < nbin) ? sh.lo[i + 1] - sh.lo[i] : n;
    sh.rank[2 * i] = c > 0 ? (c - 1) / 2 : -1;
    sh.rank[2 * i + 1] = c > 0 ? c / 2 : -1;
  }
  __syncthreads();
  radix_select(sh, hist, tg + 2, n, [&](int k, uint32_t* key, int* t0, int* t1) {
    *key = fkey(sr[k]);
    *t0 = 2 * bin_of_index(sh, k, nbin);
    *t1 = tg;
  });
  if (threadIdx.x == 0) {
    int nx = 0;
    for (int i = 0; i < nbin; ++i) {
      if (sh.lo[i + 1] - sh.lo[i] <= 0) continue;
      const double v0 = (double)fdekey(sh.prefix[2 * i]);
      const double v1 = (double)fdekey(sh.prefix[2 * i + 1]);
      sh.xs[nx] = __dadd_rn(f0, __ddiv_rn(__dmul_rn((double)i + 0.5, span), (double)nbin));
      sh.ys[nx] = __dmul_rn(0.5, __dadd_rn(v0, v1));
      ++nx;
    }
    sh.nx = nx;
    sh.med = __dmul_rn(0.5, __dadd_rn((double)fdekey(sh.prefix[tg]), (double)fdekey(sh.prefix[tg + 1])));
  }
  __syncthreads();

  if (a.mad_mode == QLP_MAD_RESID) {
    // median of the residual SR - trend first
    if (threadIdx.x == 0) { sh.rank[0] = (n - 1) / 2; sh.rank[1] = n / 2; }
    __syncthreads();
    radix_select(sh, hist, 2, n, [&](int k, uint32_t* key, int* t0, int* t1) {
      *key = fkey((float)__dsub_rn((double)sr[k], trend_at(sh, fq[k].x)));
      *t0 = 0;
      *t1 = -1;
    });
    if (threadIdx.x == 0)
      sh.med = __dmul_rn(0.5, __dadd_rn((double)fdekey(sh.prefix[0]), (double)fdekey(sh.prefix[1])));
    __syncthreads();
  }
  if (threadIdx.x == 0) { sh.rank[0] = (n - 1) / 2; sh.rank[1] = n / 2; }
  __syncthreads();
  const bool resid = a.mad_mode == QLP_MAD_RESID;
  radix_select(sh, hist, 2, n, [&](int k, uint32_t* key, int* t0, int* t1) {
    double v = (double)sr[k];
    if (resid) v = __dsub_rn(v, trend_at(sh, fq[k].x));
    *key = fkey((float)fabs(__dsub_rn(v, sh.med)));
    *t0 = 0;
    *t1 = -1;
  });
  if (threadIdx.x == 0) {
    const double mad = __dmul_rn(0.5, __dadd_rn((double)fdekey(sh.prefix[0]), (double)fdekey(sh.prefix[1])));
    sh.sigma = __dmul_rn(1.4826, mad);
    if (a.trend_out) {
      double* tr = a.trend_out + (size_t)s * kTrendDoubles;
      tr[0] = (double)sh.nx;
      tr[1] = sh.sigma;
      tr[2] = sh.med;
      tr[3] = 0.0;
      for (int i = 0; i < kMaxSturges; ++i) {
        tr[4 + i] = i < sh.nx ? sh.xs[i] : 0.0;
        tr[4 + kMaxSturges + i] = i < sh.nx ? sh.ys[i] : 0.0;
      }
    }
  }
  __syncthreads();
  }  // trend computed here
  const double sigma = sh.sigma;

  // S/N and its first maximum
  float bv = -3.0e38f;
  int bi = n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    float v = 0.f;
    if (sigma > 0.0) v = (float)__ddiv_rn(__dsub_rn((double)sr[k], trend_at(sh, fq[k].x)), sigma);
    snr[k] = v;
    if (v > bv) { bv = v; bi = k; }   // k increases: first maximum per thread
  }
  for (int off = 16; off > 0; off >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sh.best_v[warp] = bv; sh.best_i[warp] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      if (sh.best_v[w] > bv || (sh.best_v[w] == bv && sh.best_i[w] < bi)) { bv = sh.best_v[w]; bi = sh.best_i[w]; }
    }
    out->status = st.status;
    out->pad = 0;
    const int j = (bi < n) ? (int)a.qidx[st.f_off + bi] : 255;
    if (!(sigma > 0.0) || bi >= n || j >= a.nq) {
      if (!(sigma > 0.0)) out->status |= QLP_STAR_ZERO_MAD;
      out->f_idx = -1;
      out->f = out->period = out->t0 = out->q = out->depth = out->sr = out->snr = 0.0;
      out->j = out->k = out->m = out->nbins = -1;
    } else {
      const double f = fq[bi].x;
      const double qmin = fq[bi].y;
      // shared histogram: nbins(q_min) and the window m_j; per-duration histograms:
      // nbins(q_j) bins of q_j / noverlap and a window of noverlap bins
      const int nb = a.per_q ? (int)ceil(__ddiv_rn(a.noverlap, __dmul_rn(qmin, a.E[j])))
                             : (int)ceil(__ddiv_rn(a.noverlap, qmin));
      const int m = a.per_q ? a.m_perq
                            : max(1, (int)floor(__dadd_rn(__dmul_rn(__dmul_rn(qmin, a.E[j]), (double)nb), 0.5)));
      const int kb = (int)a.kbin[st.f_off + bi];
      const double period = __ddiv_rn(1.0, f);
      const double mid = __ddiv_rn(__dadd_rn((double)kb, __dmul_rn(0.5, (double)m)), (double)nb);
      const double r = (double)a.rbest[st.f_off + bi];
      const double sv = (double)a.sbest[st.f_off + bi];
      out->f_idx = bi;
      out->f = f;
      out->period = period;
      out->t0 = __dadd_rn(st.t_ref, __dmul_rn(period, __dsub_rn(mid, floor(mid))));
      out->q = __ddiv_rn((double)m, (double)nb);
      out->depth = -__ddiv_rn(sv, __dmul_rn(r, __dsub_rn(1.0, r)));
      out->sr = (double)sr[bi];
      out->snr = (double)bv;
      out->j = j;
      out->k = kb;
      out->m = m;
      out->nbins = nb;
    }
  }
}

// Coarse spectrum of the learned proposal as the network input: out[s][k] =
// (asinh(S/N / 4), 1) for the star's searched coarse bins k (entry i of its
// spectrum is bin grid_k0 - i), (0, 0) elsewhere; BF16 [n_stars][n_bins][2]. The
// monotone asinh compression keeps the ordering of the S/N while bounding the
// range the network sees (S/N from -5 to 10^4 maps to about -1.1 to 8.5).
// The network input per coarse bin k: a(k) = asinh(S/N / 4) and 1 on searched bins,
// then a() at the harmonic bins k + d2, k - d2, k + d3, k - d3 (periods 2P, P/2, 3P,
// P/3), 0 off the grid or on bins not searched; with snr_rows, also the FP32 S/N
// itself per bin (0 elsewhere) in [star][bin] rows. Pass 1 writes channels 0 and 1;
// after the block barrier pass 2 copies channel 0 of the harmonic bins (the same
// BF16 values).
__global__ void coarse_tensor_kernel(const StarDev* stars, const float* snr, int n_bins, __nv_bfloat16* out,
                                     float* snr_rows, int d2, int d3) {
  constexpr int C = QLP_CNN_IN_CH;
  const int s = blockIdx.x;
  const StarDev st = stars[s];
  __nv_bfloat16* row = out + (size_t)s * n_bins * C;
  float* srow = snr_rows ? snr_rows + (size_t)s * n_bins : nullptr;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int k = threadIdx.x; k < n_bins; k += blockDim.x) {
    row[C * k] = zero;
    row[C * k + 1] = zero;
    if (srow) srow[k] = 0.f;
  }
  __syncthreads();
  if (st.status == 0) {
    for (int i = threadIdx.x; i < st.n_f; i += blockDim.x) {
      const int k = st.grid_k0 - i;
      if (k < 0 || k >= n_bins) continue;
      const float v = snr[st.f_off + i];
      row[C * k] = __float2bfloat16_rn(asinhf(0.25f * v));
      row[C * k + 1] = __float2bfloat16_rn(1.f);
      if (srow) srow[k] = v;
    }
  }
  __syncthreads();
  const int dk[4] = {d2, -d2, d3, -d3};
  for (int k = threadIdx.x; k < n_bins; k += blockDim.x) {
    const bool here = __bfloat162float(row[C * k + 1]) > 0.f;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int kh = k + dk[h];
      row[C * k + 2 + h] = (here && kh >= 0 && kh < n_bins) ? row[C * kh] : zero;
    }
  }
}

int launch_coarse_tensor(const StarDev* stars, int n_stars, const float* snr, int n_bins, void* out,
                         float* snr_rows, int d2, int d3, void* stream) {
  if (n_stars <= 0) return 0;
  coarse_tensor_kernel<<<n_stars, 256, 0, (cudaStream_t)stream>>>(stars, snr, n_bins,
                                                                   static_cast<__nv_bfloat16*>(out), snr_rows,
                                                                   d2, d3);
  return (int)cudaGetLastError();
}

// The k largest logits of each row among valid bins (x0 channel 1 > 0, rows of
// QLP_CNN_IN_CH channels), largest
// first, ties to the lower bin; -1 when fewer than k bins are valid.
__global__ void __launch_bounds__(256) topk_kernel(const float* logits, const __nv_bfloat16* x0, int len,
                                                   int k, int32_t* out) {
  extern __shared__ unsigned char taken[];
  __shared__ float bv[8];
  __shared__ int bi[8];
  const int s = blockIdx.x;
  const float* z = logits + (size_t)s * len;
  const __nv_bfloat16* m = x0 + (size_t)s * len * QLP_CNN_IN_CH;
  for (int i = threadIdx.x; i < len; i += blockDim.x)
    taken[i] = __bfloat162float(m[QLP_CNN_IN_CH * i + 1]) > 0.f ? 0 : 1;
  __syncthreads();
  for (int r = 0; r < k; ++r) {
    float v = -3.0e38f;
    int idx = len;
    for (int i = threadIdx.x; i < len; i += blockDim.x)
      if (!taken[i] && (z[i] > v || (z[i] == v && i < idx))) { v = z[i]; idx = i; }
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = v; bi[threadIdx.x >> 5] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < 8; ++w)
        if (bv[w] > v || (bv[w] == v && bi[w] < idx)) { v = bv[w]; idx = bi[w]; }
      out[(size_t)s * k + r] = idx < len ? idx : -1;
      if (idx < len) taken[idx] = 1;
    }
    __syncthreads();
  }
}

int launch_topk(const float* logits, const void* x0, int batch, int len, int k, int32_t* out, void* stream) {
  if (batch <= 0) return 0;
  topk_kernel<<<batch, 256, len, (cudaStream_t)stream>>>(logits, static_cast<const __nv_bfloat16*>(x0), len, k,
                                                          out);
  return (int)cudaGetLastError();
}

// The n strongest S/N peaks of each star: repeatedly the largest S/N (ties: the
// lowest index) among the frequencies not excluded yet, then every frequency
// with |f / f_pick - 1| < sep is excluded. The ratio is monotone along the
// ascending grid, so each exclusion is one index range, found by binary search.
constexpr int kMaxPeaks = 64;

__device__ __forceinline__ bool near_pick(double f, double fp, double sep) {
  return fabs(__dsub_rn(__ddiv_rn(f, fp), 1.0)) < sep;
}

__global__ void __launch_bounds__(256) peaks_kernel(const StarDev* stars, const double2* fq, const float* snr,
                                                    int n_peaks, double sep, int32_t* out) {
  __shared__ int s_lo[kMaxPeaks], s_hi[kMaxPeaks];
  __shared__ float bv[8];
  __shared__ int bi[8];
  __shared__ int s_pick;
  const int s = blockIdx.x;
  const StarDev st = stars[s];
  const int nf = st.n_f;
  const float* v = snr + st.f_off;
  const double2* f = fq + st.f_off;
  int32_t* o = out + (size_t)s * n_peaks;
  for (int r = threadIdx.x; r < n_peaks; r += blockDim.x) o[r] = -1;
  for (int r = 0; r < n_peaks; ++r) {
    float best = 0.f;
    int bidx = 0x7fffffff;
    for (int k = threadIdx.x; k < nf; k += blockDim.x) {
      bool ex = false;
      for (int i = 0; i < r; ++i) ex |= (k >= s_lo[i] && k <= s_hi[i]);
      if (ex) continue;
      const float x = v[k];
      if (bidx == 0x7fffffff || x > best || (x == best && k < bidx)) { best = x; bidx = k; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
      if (oi != 0x7fffffff && (bidx == 0x7fffffff || ov > best || (ov == best && oi < bidx))) {
        best = ov;
        bidx = oi;
      }
    }
    if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < 8; ++w)
        if (bi[w] != 0x7fffffff && (bidx == 0x7fffffff || bv[w] > best || (bv[w] == best && bi[w] < bidx))) {
          best = bv[w];
          bidx = bi[w];
        }
      s_pick = bidx;
      if (bidx != 0x7fffffff) {
        o[r] = bidx;
        const double fp = f[bidx].x;
        int a = 0, b = bidx;  // first index near the pick
        while (a < b) {
          const int m = (a + b) >> 1;
          if (near_pick(f[m].x, fp, sep)) b = m; else a = m + 1;
        }
        s_lo[r] = a;
        a = bidx;
        b = nf - 1;  // last index near the pick
        while (a < b) {
          const int m = (a + b + 1) >> 1;
          if (near_pick(f[m].x, fp, sep)) a = m; else b = m - 1;
        }
        s_hi[r] = a;
      }
    }
    __syncthreads();
    if (s_pick == 0x7fffffff) break;
  }
}

int launch_peaks(const StarDev* stars, int n_stars, const double2* fq, const float* snr, int n_peaks, double sep,
                 int32_t* out, void* stream) {
  if (n_stars <= 0) return 0;
  if (n_peaks < 1 || n_peaks > kMaxPeaks) return (int)cudaErrorInvalidValue;
  peaks_kernel<<<n_stars, 256, 0, (cudaStream_t)stream>>>(stars, fq, snr, n_peaks, sep, out);
  return (int)cudaGetLastError();
}

int launch_snr(const SnrArgs& a, void* stream) {
  if (a.n_stars <= 0) return 0;
  const size_t smem = (size_t)kMaxTargets * 256 * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(snr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  snr_kernel<<<a.n_stars, kSnrThreads, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace qlp
