// Exact cell path of the BLS search (sm_103a): integer prefix sums at the bin
// edges, accumulated per phase bin in registers, and a streaming box sweep.
//
// Notation as in cells_kernels.cu: a trial frequency f with nbins bins has its
// phase-bin edges at tau_G = G D, D = 1/(f nbins), G = 0 .. g_end, and with the
// prefix sums C(tau) of (w, w d) over the points before tau every histogram bin
// of Sec. 2.1's BLS is a sum of differences C(tau_{G+1}) - C(tau_G) over the
// cycles. Here the weights are integers, w_int = round(w 2^kw) and
// y_int = round(w d 2^ky) (kw, ky per star), so every C is an exact 64-bit
// integer and the differences telescope: with
//     S[b] = sum over G = b (mod nbins), 0 <= G <= g_end, of C(tau_G)
// the cumulative histogram U[x] = sum_{b < x} H[b mod nbins] is
//     U[x] = S[x mod nbins] + ([b* < x mod nbins] + floor(x / nbins)) C_end
// up to a constant, where b* = g_end mod nbins and C_end = C(tau_{g_end}) is
// the star's total, and the box of m bins starting at bin k sums to
// U[k + m] - U[k]. So a lane owns one bin b, walks its edges b, b + nbins, ...
// (one per cycle) and adds C(tau_G) to a register: no histogram in shared
// memory, no atomics, no exchange between lanes, and the result does not depend
// on the order of the additions.
//
// K0x freq_rec_kernel (plan time): one FreqRec per trial frequency (bins, the
// edge step in 2^-40 cells, guard band, last edge, the box widths present and
// the lowest duration index of each).
// K1x prep_fixed_kernel (1 CTA per exact-path star): weights and the weighted
// mean in FP64 as the other prep kernels, the integer weights, their exact
// prefix sums and the per-cell tables (offset of the cell's point, prefix sums at
// the cell start as a 64-bit group base plus a 32-bit local part; the local part
// of w d carries a bias of 2^30, so that both local parts are non-negative and
// widen to 64 bits with a zero high word; the sums take the bias off once).
// K2x cells_fixed_kernel: persistent; work queue of (star, frequency chunk); the
// star's table in shared memory (three contiguous arrays, staged by bulk
// asynchronous copies on an mbarrier); warps take the item's frequencies one at a time.
// Per frequency the bins are handled 32 at a time (lane = bin): the lanes' S
// values become U, the exact differences H[x] = U[x + 1] - U[x] are scaled to FP32
// (w, w d) pairs and written to a per-warp ring of four 32-bin blocks (bin x at
// x mod 128); the sweep of the boxes starting in blocks 2j and 2j + 1 (two start
// bins per lane) runs once block 2j + 2 is in the ring. Stars whose table does not fit in shared memory take
// their edges window by window into a global workspace first (windowed_item), in a
// launch of their own.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "bls_device.cuh"
#include "qlp_internal.h"

namespace qlp {

constexpr int kRing = 128;  // float2 per warp: H of the last four blocks of 32 bins, at (bin mod 128)
constexpr long long kLocBias = 1ll << 30;  // added to the w d local parts of the cell table
constexpr long long kNarrowBias = 1ll << 31;  // added to the w d prefix sums of the 32-bit table
constexpr double kNarrowF = 4294836224.0;     // 2^32 - 2^17: the w scale of the 32-bit table
// prefix sums at a cell: the group base plus the local parts, widened from 32 bits with
// a zero high word (the w d part still carries kLocBias, taken off per sum of edges)
__device__ __forceinline__ void add_cell(long long& aw, long long& ay, const longlong2& bs, const int2& lc) {
  aw += bs.x + (long long)(uint32_t)lc.x;
  ay += bs.y + (long long)(uint32_t)lc.y;
}
// cells staged past the sentinel (copies of it): every edge G <= g_end lies before
// T + 2 D, at most 2 x 255 + 1 cells past the table, so the loop needs no clamp
constexpr int kPadCells = 544;

// Byte offsets of the table arrays in shared memory: dt (4 B per cell), loc (8 B
// per cell), base (16 B per 32 cells), then the rings.
__host__ __device__ __forceinline__ uint32_t fixed_loc_off(int ncs) { return ((uint32_t)ncs * 4u + 15u) & ~15u; }
__host__ __device__ __forceinline__ uint32_t fixed_base_off(int ncs) {
  return fixed_loc_off(ncs) + (((uint32_t)ncs * 8u + 15u) & ~15u);
}
__host__ __device__ __forceinline__ uint32_t fixed_ring_off(int ncs) {
  return fixed_base_off(ncs) + ((((uint32_t)ncs + 31u) / 32u * 16u + 15u) & ~15u);
}

// ------------------------------------------------------------------ K1x

__device__ __forceinline__ double block_sum(double v, double* red) {  // blockDim.x a multiple of 32, at most 512
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = fmax(s, red[i]);
  return s;
}

// Scale exponent k with v 2^k < 2^25 for every |v| <= vmax (so that 32 such
// integers sum to less than 2^30 in magnitude).
__device__ __forceinline__ int fixed_exponent(double vmax) {
  if (!(vmax > 0.0)) return 0;
  int e = 0;
  frexp(vmax, &e);  // vmax < 2^e
  return max(-100, min(25 - e, 100));
}

// Dynamic shared memory of prep_fixed_kernel for a star of n points: 1/dy^2 (FP64)
// and the cell of every point, cached for stars of at most kPrepCachePts points.
constexpr int kPrepCachePts = 18000;
__host__ __device__ __forceinline__ uint32_t prep_fixed_smem(int n) { return (uint32_t)min(n, kPrepCachePts) * 12u; }

__global__ void __launch_bounds__(512) prep_fixed_kernel(const PrepFixedArgs a) {
  extern __shared__ __align__(16) unsigned char psm[];
  __shared__ double red[16];
  __shared__ long long scan_w[512], scan_y[512];
  const int s = a.fixed_stars[blockIdx.x];
  const StarDev st = a.stars[s];
  const int n = st.n_pts;
  if (n <= 0) return;
  const double* tp = a.tp + st.pt_off;
  const double* y = a.y + st.pt_off;
  const double* dy = a.dy + st.pt_off;
  const int tid = threadIdx.x;
  const int nc = st.n_cells;
  const double h = st.h;
  const bool cache = n <= kPrepCachePts;  // block-uniform
  double* s_inv = reinterpret_cast<double*>(psm);
  int* s_cell = reinterpret_cast<int*>(psm + 8u * (uint32_t)(cache ? n : 0));
  auto inv_of = [&](int i) { return cache ? s_inv[i] : 1.0 / (dy[i] * dy[i]); };
  auto cell_at = [&](int i) { return cache ? s_cell[i] : cell_of(tp[i], h); };

  // weights w = dy^-2 / sum dy^-2 and the weighted mean (FP64); each point's
  // inverse variance and cell once (kept in shared memory when the star fits)
  double acc = 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    const double inv = 1.0 / (dy[i] * dy[i]);
    if (cache) {
      s_inv[i] = inv;
      s_cell[i] = cell_of(tp[i], h);
    }
    acc += inv;
  }
  const double rws = 1.0 / block_sum(acc, red);
  acc = 0.0;
  for (int i = tid; i < n; i += blockDim.x) acc += inv_of(i) * rws * y[i];
  const double ybar = block_sum(acc, red);
  double mw = 0.0, md = 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    const double w = inv_of(i) * rws;
    mw = fmax(mw, w);
    md = fmax(md, fabs(w * (y[i] - ybar)));
  }
  mw = block_max(mw, red);
  md = block_max(md, red);
  // 64-bit table: scales that keep 32 consecutive points below 2^30. 32-bit table:
  // w_int = round(w F) with F = 2^32 - 2^17, so that the N <= 2^16 roundings leave the
  // total below 2^32 (r is then the ratio of two integer sums), and the largest y scale
  // that keeps every point's |y_int| (this kernel's largest |w d|) and every prefix sum
  // of y_int (the planner's largest running sum; this kernel's lies within 2^-9 of it,
  // and the roundings add at most 2^15) below 2^30
  const bool narrow = st.narrow != 0;
  int kw = fixed_exponent(mw), ky = fixed_exponent(md);
  if (narrow) {
    int e1 = 0, e2 = 0;
    frexp(st.y_exc * 1.00390625, &e1);  // y_exc (1 + 2^-8) < 2^e1
    frexp(md * 1.00390625, &e2);
    kw = 0;
    ky = max(-100, min(30 - max(e1, e2), 100));
  }
  const double pw = narrow ? kNarrowF : ldexp(1.0, kw), py = ldexp(1.0, ky);

  // exact prefix sums of the integer weights: contiguous segment per thread,
  // exclusive scan of the segment totals
  const int L = (n + blockDim.x - 1) / blockDim.x;
  const int i0 = min(n, tid * L), i1 = min(n, i0 + L);
  long long sw = 0, sy = 0;
  for (int i = i0; i < i1; ++i) {
    const double w = inv_of(i) * rws;
    const long long wi = __double2ll_rn(w * pw), yi = __double2ll_rn(w * (y[i] - ybar) * py);
    sw += wi;
    sy += yi;
    // both below 2^25 in magnitude: kept in the point's cache slot (its 1/dy^2 is no
    // longer needed) for the prefix pass below
    if (cache) reinterpret_cast<int2*>(s_inv)[i] = make_int2((int)(uint32_t)wi, (int)yi);
  }
  scan_w[tid] = sw;
  scan_y[tid] = sy;
  __syncthreads();
  if (tid < 32) {  // exclusive scan of the segment totals: 16 per lane, then the warp
    const int per = (int)blockDim.x / 32;
    long long lw = 0, ly = 0;
    for (int k = 0; k < per; ++k) {
      lw += scan_w[tid * per + k];
      ly += scan_y[tid * per + k];
    }
    long long xw = lw, xy = ly;  // inclusive warp scan of the lane totals
    for (int o = 1; o < 32; o <<= 1) {
      const long long tw = __shfl_up_sync(0xffffffffu, xw, o);
      const long long ty = __shfl_up_sync(0xffffffffu, xy, o);
      if (tid >= o) {
        xw += tw;
        xy += ty;
      }
    }
    long long rw = xw - lw, ry = xy - ly;  // exclusive
    for (int k = 0; k < per; ++k) {
      const long long tw = scan_w[tid * per + k], ty = scan_y[tid * per + k];
      scan_w[tid * per + k] = rw;
      scan_y[tid * per + k] = ry;
      rw += tw;
      ry += ty;
    }
    if (tid == 31) {
      a.ipre[st.cpre_off + n] = make_longlong2(rw, ry);
      FixedStar f;
      f.w_tot = rw;
      f.y_tot = ry;
      f.kw = kw;
      f.ky = ky;
      f.scw = narrow ? (float)(1.0 / (double)rw) : __int_as_float((127 - kw) << 23);  // 1 / w_tot or 2^-kw
      f.narrow = narrow ? 1 : 0;
      a.fx[s] = f;
    }
  }
  __syncthreads();
  long long cw = scan_w[tid], cy = scan_y[tid];
  // the 32-bit table keeps every prefix of w_int below 2^32 and of y_int below 2^30 in
  // magnitude by its scales; a sum past its word's range would wrap: raise the error bit
  // (the star's results are then void)
  auto wraps = [&](long long w, long long y) { return w >= (1ll << 32) || y >= kNarrowBias || y <= -kNarrowBias; };
  bool out_of_range = narrow && wraps(cw, cy);
  for (int i = i0; i < i1; ++i) {
    a.ipre[st.cpre_off + i] = make_longlong2(cw, cy);
    if (cache) {
      const int2 v = reinterpret_cast<const int2*>(s_inv)[i];
      cw += (long long)(uint32_t)v.x;
      cy += v.y;
    } else {
      const double w = inv_of(i) * rws;
      cw += __double2ll_rn(w * pw);
      cy += __double2ll_rn(w * (y[i] - ybar) * py);
    }
    out_of_range = out_of_range || (narrow && wraps(cw, cy));
  }
  if (out_of_range) atomicOr(a.err, kErrRange);
  __syncthreads();

  // first point at or after each cell start: point i fills cells (cell(i-1), cell(i)]
  int32_t* first = a.gidx + st.cell_off;
  for (int i = tid; i <= n; i += blockDim.x) {
    const int up = (i == 0) ? -1 : cell_at(i - 1);
    const int ui = (i == n) ? nc : cell_at(i);
    for (int c = up + 1; c <= ui && c <= nc; ++c) first[c] = i;
  }
  __syncthreads();
  // 1/h: the point's offset in its cell, (t' - u h) / h, by a multiplication; with the
  // product's rounding it stays within (T/h + 3) 2^-53 cells of the exact offset, inside
  // the guard band's allowance of 2 (T/h) 2^-53 cells for the cell offsets
  const double rh = 1.0 / h;
  for (int u = tid; u <= nc; u += blockDim.x) {
    const int f = first[u];
    const bool in_cell = (u < nc) && (f < n) && (cell_at(f) == u);
    uint32_t q = 0xffffffffu;  // the cell's point as a 32-bit fraction of the cell, empty = all ones
    if (in_cell) {
      const double fr = __dmul_rn(__dsub_rn(tp[f], __dmul_rn((double)u, h)), rh);
      q = (uint32_t)fmin(floor(__dmul_rn(fr, 4294967296.0)), 4294967294.0);
    }
    a.dt[st.cell_off + u] = q;
    const longlong2 c = a.ipre[st.cpre_off + f];
    if (narrow) {  // the prefix sums themselves: w below 2^32, |y| below 2^30 + 2^15, biased by 2^31
      a.loc[st.cell_off + u] = make_int2((int)(uint32_t)c.x, (int)(uint32_t)(c.y + kNarrowBias));
      continue;
    }
    const longlong2 cb = a.ipre[st.cpre_off + first[u & ~31]];
    // at most 31 points of weights below 2^25 lie between the group start and the
    // cell: both local parts are below 2^30 in magnitude
    a.loc[st.cell_off + u] = make_int2((int)(c.x - cb.x), (int)(c.y - cb.y + kLocBias));
    if ((u & 31) == 0) a.base[st.base_off + (u >> 5)] = cb;
  }
}

// K0x freq_rec_kernel (1 CTA per exact-path star, at plan time): one FreqRec per
// trial frequency. It depends on the grid and the star's cell width only, not on
// the fluxes, so a plan computes it once for all its searches.
__global__ void __launch_bounds__(256) freq_rec_kernel(const PrepFixedArgs a) {
  const int s = a.fixed_stars[blockIdx.x];
  const StarDev st = a.stars[s];
  const double h = st.h;
  const int tid = threadIdx.x;
  // per trial frequency: the same FP64 operations as the other search kernels
  for (int k = tid; k < st.n_f; k += blockDim.x) {
    const int64_t fidx = st.f_off + k;
    const double2 fq = a.fq[fidx];
    FreqRec r;
    r.K = 0ull;
    r.jlow = 0ull;
    r.nb = 0;
    r.band_q = 0u;
    r.gq_bstar = 0u;
    r.wmask = 0u;
    const int nb = (int)ceil(__ddiv_rn(a.noverlap, fq.y));
    if (nb >= 32 && nb <= min(a.nb_cap, 8192)) {
      const double F = __dmul_rn(fq.x, (double)nb);
      const double D = __ddiv_rn(1.0, F);  // bin duration (days)
      const double yT = __dmul_rn(st.baseline, F);
      const int g_end = (int)floor(yT) + 2;  // edges 0 .. g_end; tau_{g_end} > T
      r.gq_bstar = ((uint32_t)(g_end / nb) << 13) | (uint32_t)(g_end % nb);
      r.K = __double2ull_rn(__dmul_rn(__ddiv_rn(D, h), 1099511627776.0));  // D/h < 2^8 in 2^-40 units
      // guard band in 2^-32 cell units, twice the sum of the bounds on: the FP64 fold's
      // error, (T F + nbins) 2^-53 bins = (T F + nbins) (D/h) 2^-21 units; the edge step's
      // rounding, 2^-41 cells per edge (g_end 2^-9 units); the FP64 cell offsets of the
      // points and of D/h, (T/h) 2^-20 units; and the two 32-bit truncations
      r.band_q = (uint32_t)fmin(
          __dmul_rn(__dmul_rn(__dadd_rn(yT, (double)nb), __ddiv_rn(D, h)), 9.5367431640625e-07) +
              (double)(g_end >> 8) + __dmul_rn(__ddiv_rn(st.baseline, h), 3.814697265625e-06) + 16.0,
          1073741824.0);
      // box widths m_j and, per width, its lowest j (m_j is non-decreasing in j)
      unsigned long long jl = 0ull;
      uint32_t wm = 0u;
      for (int j = a.nq - 1; j >= 0; --j) {
        const int m = min(15, max(1, (int)floor(__dadd_rn(__dmul_rn(__dmul_rn(fq.y, a.E[j]), (double)nb), 0.5))));
        wm |= 1u << (m - 1);
        jl = (jl & ~(0xfull << (4 * (m - 1)))) | ((unsigned long long)j << (4 * (m - 1)));
      }
      r.jlow = jl;
      r.wmask = wm;
      r.nb = nb;
    }
    a.frec[fidx] = r;
  }
}

int launch_freq_recs(const PrepFixedArgs& a, void* stream) {
  if (a.n <= 0) return 0;
  freq_rec_kernel<<<a.n, 256, 0, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

int launch_prep_fixed(const PrepFixedArgs& a, void* stream) {
  if (a.n <= 0) return 0;
  const int smem = (int)prep_fixed_smem(a.max_pts);
  cudaError_t e = cudaFuncSetAttribute(prep_fixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  prep_fixed_kernel<<<a.n, 512, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

uint32_t fixed_prep_smem_bytes(int n_pts) { return prep_fixed_smem(n_pts); }

// ------------------------------------------------------------------ K2x

// Box sweep of the two start bins ka (even) and ka + 1 over the ring (H[x] at ring[x mod
// 128]): the lane's running sums of both starts are (w, w d) pairs, added as packed FP32
// pairs; a start at or past the last bin begins at r = 4, so that it never scores (every
// window of the ring sums to more than -2 in w). Every width w = o + 1 present is scored
// s^2 / (r (1 - r)) for 0 < r < 1 and compared division-free with the lane's best so far.
// An exact FP32 tie keeps the lane's earlier candidate: within a pair of blocks the
// narrower width, then the lower start; across the lane's pairs (disjoint boxes, tied
// only by a coincidence of their FP32 sums) the earlier pair. Ties between lanes go to
// the lower duration index, then the lower start (the warp argmax).
template <bool ALL>
__device__ __forceinline__ void sweep_pair(const float2* ring, int ka, bool ain, bool bin, int mmax, uint32_t wmask,
                                           float& bs2, float& bd, int& bkey) {
  constexpr int NO = ALL ? 11 : 15;
  auto ld = [&](int t) { return *reinterpret_cast<const float4*>(ring + ((ka + 2 * t) & 127)); };
  auto score = [&](const float2 acc, int key) {
    const float dd = __fmaf_rn(-acc.x, acc.x, acc.x);  // r (1 - r)
    const float s2 = __fmul_rn(acc.y, acc.y);
    const float lhs = __fmul_rn(s2, bd), rhs = __fmul_rn(bs2, dd);
    const bool better = dd > 0.f && lhs > rhs;
    bs2 = better ? s2 : bs2;
    bd = better ? dd : bd;
    bkey = better ? key : bkey;
  };
  float2 A = make_float2(ain ? 0.f : 4.f, 0.f), B = make_float2(bin ? 0.f : 4.f, 0.f);
  float4 cur = ld(0);
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    if (ALL || o < mmax) {
      if ((o & 1) == 0) {  // A += H[ka + o], B += H[ka + o + 1]
        A = __fadd2_rn(A, make_float2(cur.x, cur.y));
        B = __fadd2_rn(B, make_float2(cur.z, cur.w));
      } else {
        const float4 nxt = ld((o + 1) >> 1);
        A = __fadd2_rn(A, make_float2(cur.z, cur.w));
        B = __fadd2_rn(B, make_float2(nxt.x, nxt.y));
        cur = nxt;
      }
      if (ALL ? o >= 2 : ((wmask >> o) & 1u) != 0u) {
        score(A, (o << 16) | ka);
        score(B, (o << 16) | (ka + 1));
      }
    }
  }
}

// This warp's row of exact bin sums in the block's workspace: ws_block / kFixedWarps
// entries, at least the bins of every whole-table star of the plan, then the warp's
// kFixedPendRows entries of pending boxes (pend_rows).
__device__ __forceinline__ longlong2* warp_row(const FixedArgs& a) {
  return a.ws + (size_t)blockIdx.x * (size_t)a.ws_block +
         (size_t)(threadIdx.x >> 5) * (size_t)(a.ws_block / kFixedWarps);
}
__device__ __forceinline__ longlong2* pend_rows(const FixedArgs& a) {
  return warp_row(a) + (a.ws_block / kFixedWarps - kFixedPendRows);
}

// A whole-table frequency's chosen box, left by lane 0 for rescoring: its exact
// integer sums (w, w d) and, in the second half, (frequency in the item, the packed
// (j, width, k) word, s^2, r (1 - r)) of the FP32 sweep; s^2 < 0 when no box counts.
__device__ __forceinline__ void put_pending(longlong2* rows, int p, long long dw, long long dy, int fl,
                                            uint32_t key, float s2, float d) {
  int4* r = reinterpret_cast<int4*>(rows) + 2 * p;
  r[0] = make_int4((int)(uint32_t)dw, (int)(dw >> 32), (int)(uint32_t)dy, (int)(dy >> 32));
  r[1] = make_int4(fl, (int)key, __float_as_int(s2), __float_as_int(d));
}

// Lane t scores the t-th pending box again from its exact sums in double-float
// arithmetic (r and 1 - r over the star's total on the 32-bit table, scaled by 2^-kw
// on the 64-bit one; s scaled by 2^-ky) and stores it: the rescoring of up to 32
// frequencies takes one instruction stream (lane 0 alone, one frequency at a time,
// took 2.7 % of the launch). f0 is the item's first frequency.
__device__ __forceinline__ void flush_pending(const FixedArgs& a, const FixedStar& fx, int64_t f0,
                                              const longlong2* rows, int n, int lane) {
  __syncwarp();  // lane 0's records are visible to the warp
  if (lane < n) {
    const int4 r0 = reinterpret_cast<const int4*>(rows)[2 * lane];
    const int4 r1 = reinterpret_cast<const int4*>(rows)[2 * lane + 1];
    const long long dw = (long long)(((unsigned long long)(uint32_t)r0.y << 32) | (uint32_t)r0.x);
    const long long dy = (long long)(((unsigned long long)(uint32_t)r0.w << 32) | (uint32_t)r0.z);
    const uint32_t key = (uint32_t)r1.y;
    BoxBest bb;
    bb.s2 = __int_as_float(r1.z);
    bb.d = __int_as_float(r1.w);
    bb.s = 0.f;
    bb.r = 0.f;
    const bool nobox = bb.s2 < 0.f;
    bb.j = nobox ? 255 : (int)(key >> 20);
    bb.k = nobox ? -1 : (int)(key & 0xffffu);
    bb.xv = false;
    if (!nobox) {
      if (fx.narrow) {  // r = dw / w_tot and 1 - r = (w_tot - dw) / w_tot, both sums below 2^32
        const DF wt = df_from_ll_scaled(fx.w_tot, 0);
        bb.xr = df_div(df_from_ll_scaled(dw, 0), wt);
        bb.xq = df_div(df_from_ll_scaled(fx.w_tot - dw, 0), wt);
      } else {
        // kw lies in [24, 46] on this path: the largest weight is at most 1 and at least
        // 1/N with N <= 2^21 points, and w_max 2^kw lies in [2^24, 2^25)
        const int kw = min(max(fx.kw, 0), 62);
        bb.xr = df_from_ll_scaled(dw, kw);
        bb.xq = df_from_ll_scaled((1ll << kw) - dw, kw);  // 1 - r
      }
      bb.xs = df_from_ll_scaled(dy, fx.ky);
      bb.xv = true;
    }
    store_box(bb, 0, f0 + r1.x, a.sr, a.qidx, a.kbin, a.sbest, a.rbest);
  }
  __syncwarp();  // the records are read before the warp writes new ones
}

// One trial frequency on a warp: the bin sums S (from the staged table's edges, or
// from the window passes' workspace row when WS), then per block of 32 bins U, the
// FP32 histogram records in the ring and the sweep, the warp argmax and the store.
// The row srow holds the exact bin sums S of the frequency (the window passes'
// workspace row when WS, else this warp's row (warp_row), written here block by block), so that
// the box the FP32 sweep chose is scored once more from its exact integer sums: at
// once when WS, else from the pending record put at prow[pend] (fl: the frequency
// within the item) and rescored in the caller's next flush_pending.
template <bool WS, bool NARROW>
__device__ __forceinline__ void run_frequency(const FixedArgs& a, int64_t fidx, const FreqRec& R,
                                              const FixedStar& fx, const unsigned char* smem,
                                              uint32_t loc_off, uint32_t base_off, int nc, float2* ring,
                                              int lane, float scw, float scy, const double* tp,
                                              const int32_t* gidx, uint32_t st4, uint32_t st8, uint32_t st16,
                                              longlong2* srow, longlong2* prow, int& pend, int fl) {
  const int nb = R.nb;
  const double f = a.fq[fidx].x;  // for the exact decision near ties
  const uint32_t wmask = R.wmask;
  const int mmax = 32 - __clz(wmask);
  const bool all_widths = wmask == 0x7fcu;  // exactly 3 .. 11 bins
  const int gq = (int)(R.gq_bstar >> 13), bstar = (int)(R.gq_bstar & 8191u);
  const int g_end = gq * nb + bstar;
  // edge step in 32.32 fixed point, so that the cell and the position in it are the
  // two halves of G K with no shift. Rounding the 24.40 step to it adds at most
  // 2^-33 cells per step, G / 2 units of 2^-32 cells at edge G: the guard band
  // grows by twice that at the last edge (g_end < 2^27: at most 16384 cycles of
  // 8192 bins; so the band stays below 2^31)
  const unsigned long long K32 = (R.K + 128ull) >> 8;
  const uint32_t k_lo = (uint32_t)K32, k_hi = (uint32_t)(K32 >> 32);
  const uint32_t band_q = R.band_q + (uint32_t)g_end;
  const int nblk = (nb + 31) >> 5;

  long long h0w = 0, h0y = 0;  // U of bins 0..31 (the wrap-around values)
  long long pw = 0, py = 0;    // U of the previous block
  float bs2 = 0.f, bd = 1.f;   // best box of this lane: s^2, r (1 - r) and its key
  int bkey = 0x7fffffff;
  // block i: U of bins 32 i + lane; then the histogram of block i - 1 and, for odd
  // i >= 3, the sweep of blocks i - 3 and i - 2 (boxes of up to 15 bins starting in them)
  const int i_last = (((nblk + 1) >> 1) << 1) + 1;  // the sweep of the last pair of blocks
  for (int i = 0; i <= i_last; ++i) {
    const int x = (i << 5) + lane;
    long long uw = 0, uy = 0;
    if constexpr (WS) {  // bin sums from the window passes
      if ((i << 5) < nb) {
        if (x < nb) {
          const longlong2 sv = srow[x];
          uw = sv.x + (bstar < x ? fx.w_tot : 0);
          uy = sv.y + (bstar < x ? fx.y_tot : 0);
        }
      }
    } else {
      if ((i << 5) < nb) {  // warp-uniform: lanes x < nb own bin x
        // edges G = G0, G0 + nb, ... <= g_end (one per cycle). The edge at t' = 0
        // (G = 0) is skipped: no point lies before it. A block of r <= 16 bins spreads
        // each bin's cycles over P = 32 / r lanes (phase ph: cycles ph, ph + P, ...),
        // summed by shuffles afterwards. Idle lanes walk a real bin's edges
        // (discarded), so that every edge stays inside the staged table.
        const int r = nb - (i << 5);
        const bool split = r <= 16;
        int P = 1, ph = 0, xb = x;
        if (split) {
          P = 32 / r;
          ph = lane / r;
          xb = (i << 5) + (lane - ph * r);
        }
        const bool idle = split ? ph >= P : x >= nb;
        const int G0 = idle ? (i << 5) : (xb == 0 ? nb : xb + ph * nb);
        const int gstep = P * nb;
        // the w sums of the 32-bit table in wrapping 32-bit words: every bin and box sum
        // of w lies in [0, 2^32), so sums modulo 2^32 give them exactly
        using WAcc = std::conditional_t<NARROW, uint32_t, long long>;
        WAcc aw = 0;
        long long ay = 0;
        // the smallest (dq - fr + band) mod 2^32 over the lane's edges: some edge lies
        // within the guard band of its cell's point exactly when it is <= 2 band
        uint32_t nmin = 0xffffffffu;
        // every lane takes cnt edges; only in the last one may a lane be past g_end
        const int cnt0 = gq + ((i << 5) > bstar ? 0 : 1);
        const int cnt = split ? (cnt0 + P - 1) / P : cnt0;  // no division in full blocks
        // tau_G / h in 32.32 fixed point, X = G K (below 2^54: the cell index u < 2^22),
        // stepped by gstep K from edge to edge (the same bits as the product)
        auto xpos = [&](int G) {
          return (unsigned long long)(uint32_t)G * k_lo + ((unsigned long long)((uint32_t)G * k_hi) << 32);
        };
        const unsigned long long XS = xpos(gstep);
        unsigned long long X = xpos(G0);
        auto edge = [&](unsigned long long X, bool valid, bool clamp) {
          // cell u and position fr (2^-32 of a cell)
          int u = (int)(uint32_t)(X >> 32);
          if (clamp) u = min(u, nc);
          const uint32_t fr = (uint32_t)X;
          const uint32_t dq = *reinterpret_cast<const uint32_t*>(smem + (uint32_t)u * st4);
          nmin = min(nmin, dq - fr + band_q);
          const int v = u + (dq < fr ? 1 : 0);  // past the cell's point if it lies before tau_G
          const int2 lc = *reinterpret_cast<const int2*>(smem + loc_off + (uint32_t)v * st8);
          if constexpr (NARROW) {  // the 32-bit prefix sums themselves
            if (valid) {
              aw += (uint32_t)lc.x;
              ay += (long long)(uint32_t)lc.y;
            }
          } else {
            const longlong2 bs = *reinterpret_cast<const longlong2*>(smem + base_off + (uint32_t)(v >> 5) * st16);
            if (valid) add_cell(aw, ay, bs, lc);
          }
        };
        int c = 0;
        for (; c + 4 < cnt; c += 4) {
          const unsigned long long X1 = X + XS, X2 = X1 + XS, X3 = X2 + XS;
          edge(X, true, false);
          edge(X1, true, false);
          edge(X2, true, false);
          edge(X3, true, false);
          X = X3 + XS;
        }
        for (; c + 1 < cnt; ++c) {
          edge(X, true, false);
          X += XS;
        }
        const bool last = G0 + (cnt - 1) * gstep <= g_end;
        edge(X, last, true);
        ay -= (long long)(cnt - (last ? 0 : 1)) * (NARROW ? kNarrowBias : kLocBias);  // the bias of the edges taken
        bool near = nmin <= 2u * band_q;  // an edge within the guard band of its cell's point
        if (split) {  // warp-uniform: add the other phases of each bin into lanes 0 .. r-1
          for (int q = 1; q < P; ++q) {
            const WAcc ow = __shfl_down_sync(0xffffffffu, aw, q * r);
            const long long oy = __shfl_down_sync(0xffffffffu, ay, q * r);
            const bool on = __shfl_down_sync(0xffffffffu, near ? 1 : 0, q * r) != 0;
            if (lane < r) {
              aw += ow;
              ay += oy;
              near = near || on;
            }
          }
        }
        // lanes past the last bin accumulated nothing meaningful
        if (x >= nb) {
          aw = 0;
          ay = 0;
          near = false;
        }
        if (__any_sync(0xffffffffu, near)) {  // rare: redo the bin, near-ties by the exact FP64 fold
          if (near) {
            aw = 0;
            ay = 0;
            for (int g = x == 0 ? nb : x; g <= g_end; g += nb) {
              const unsigned long long X =
                  (unsigned long long)(uint32_t)g * k_lo + ((unsigned long long)((uint32_t)g * k_hi) << 32);
              const int u = min((int)(uint32_t)(X >> 32), nc);
              const uint32_t fr = (uint32_t)X;
              const uint32_t dq = reinterpret_cast<const uint32_t*>(smem)[u];
              int sel = dq < fr ? 1 : 0;
              if (dq != 0xffffffffu && (uint32_t)(dq - fr + band_q) <= 2u * band_q)
                sel = exact_before(tp, gidx[u], f, nb, g);
              const int v = u + sel;
              const int2 lc = reinterpret_cast<const int2*>(smem + loc_off)[v];
              if constexpr (NARROW) {
                aw += (uint32_t)lc.x;
                ay += (long long)(uint32_t)lc.y - kNarrowBias;
              } else {
                const longlong2 bs = reinterpret_cast<const longlong2*>(smem + base_off)[v >> 5];
                add_cell(aw, ay, bs, lc);
                ay -= kLocBias;
              }
            }
          }
        }
        if (x < nb) warp_row(a)[x] = make_longlong2((long long)aw, ay);  // S of bin x, for the rescoring below
        if (bstar < x) {
          aw += (WAcc)fx.w_tot;
          ay += fx.y_tot;
        }
        uw = (long long)aw;
        uy = ay;
      }
    }
    if ((i << 5) + 31 >= nb) {  // warp-uniform: lanes x >= nb take U[x - nb] + total
      const int src = (x - nb) & 31;  // x - nb < 32 for every value the sweep uses
      const long long ow = __shfl_sync(0xffffffffu, h0w, src);
      const long long oy = __shfl_sync(0xffffffffu, h0y, src);
      if (x >= nb) {
        uw = ow + fx.w_tot;
        uy = oy + fx.y_tot;
      }
    }
    if (i == 0) {
      h0w = uw;
      h0y = uy;
    } else {
      // histogram of block i - 1: H[x] = U[x + 1] - U[x], exact, then FP32. Lane x takes
      // U[x + 1] from lane x + 1's previous block, lane 31 from lane 0's current one.
      const int src = (lane + 1) & 31;
      float2 hv;
      if constexpr (NARROW) {
        // the 32-bit table's bin sums: the w sum lies in [0, 2^32) (a part of the star's
        // total below 2^32), so the difference of the low words is exact; the w d sum
        // goes through 32 bits when every lane's fits (the same rounding either way)
        const uint32_t nw32 = __shfl_sync(0xffffffffu, (uint32_t)(lane == 0 ? uw : pw), src);
        const long long ny = __shfl_sync(0xffffffffu, lane == 0 ? uy : py, src);
        const uint32_t hw = nw32 - (uint32_t)pw;
        const long long hy = ny - py;
        float fy;
        if (__all_sync(0xffffffffu, hy == (long long)(int)hy)) fy = __int2float_rn((int)hy);
        else fy = __ll2float_rn(hy);
        hv = make_float2(__fmul_rn(__uint2float_rn(hw), scw), __fmul_rn(fy, scy));
      } else {
        const long long nw = __shfl_sync(0xffffffffu, lane == 0 ? uw : pw, src);
        const long long ny = __shfl_sync(0xffffffffu, lane == 0 ? uy : py, src);
        hv = make_float2(__fmul_rn(__ll2float_rn(nw - pw), scw), __fmul_rn(__ll2float_rn(ny - py), scy));
      }
      ring[(((i - 1) & 3) << 5) + lane] = hv;
    }
    pw = uw;
    py = uy;
    __syncwarp();
    if (i >= 3 && ((i - 3) & 1) == 0) {  // sweep blocks i - 3 and i - 2: boxes starting at their bins
      const int ka = ((i - 3) << 5) + 2 * lane;
      if (all_widths) sweep_pair<true>(ring, ka, ka < nb, ka + 1 < nb, mmax, wmask, bs2, bd, bkey);
      else sweep_pair<false>(ring, ka, ka < nb, ka + 1 < nb, mmax, wmask, bs2, bd, bkey);
    }
    __syncwarp();
  }
  const bool none = bkey == 0x7fffffff;
  bs2 = none ? -1.f : bs2;
  const int bo = bkey >> 16;
  // the lowest duration index of each width, read again here rather than kept live
  const unsigned long long jlow = a.frec[fidx].jlow;
  // (j, width, k) in one word: j in bits 20-23, the width index in 16-19, k in 0-15;
  // one j has one width, so the word orders as (j, k) does
  uint32_t key = none ? 0xffffffffu
                      : ((uint32_t)((jlow >> (4 * bo)) & 15ull) << 20) | ((uint32_t)bo << 16) | (uint32_t)(bkey & 0xffff);
  for (int off = 16; off > 0; off >>= 1) {
    const float o_s2 = __shfl_xor_sync(0xffffffffu, bs2, off);
    const float o_d = __shfl_xor_sync(0xffffffffu, bd, off);
    const uint32_t o_key = __shfl_xor_sync(0xffffffffu, key, off);
    // strict: larger s^2 / d, then the lower (j, k); s^2 < 0 is no box
    bool take;
    if (o_s2 < 0.f) take = false;
    else if (bs2 < 0.f) take = true;
    else {
      const float lhs = o_s2 * bd, rhs = bs2 * o_d;
      take = lhs != rhs ? lhs > rhs : o_key < key;
    }
    if (take) {
      bs2 = o_s2; bd = o_d; key = o_key;
    }
  }
  const bool nobox = bs2 < 0.f;
  const int bj = nobox ? 255 : (int)(key >> 20);
  const int bk = nobox ? -1 : (int)(key & 0xffffu);
  const int bm = nobox ? 0 : (int)((key >> 16) & 15u) + 1;  // bins of the box
  if constexpr (!WS) {  // whole tables: the box's exact sums wait for a batch rescoring
    if (lane == 0) {
      long long dw = 0, dy = 0;
      if (bk >= 0) {  // U[bk + bm] - U[bk] as below
        const int k2 = bk + bm;
        const int k2m = k2 >= nb ? k2 - nb : k2;
        const longlong2* row = warp_row(a);
        const longlong2 a0 = row[bk], a1 = row[k2m];
        const long long nwrap = (bstar < k2m ? 1 : 0) + (k2 >= nb ? 1 : 0) - (bstar < bk ? 1 : 0);
        dw = a1.x - a0.x + nwrap * fx.w_tot;
        dy = a1.y - a0.y + nwrap * fx.y_tot;
        if (NARROW) dw = (long long)(uint32_t)dw;  // the rows hold the w sums modulo 2^32
      }
      put_pending(prow, pend, dw, dy, fl, key, bs2, bd);
    }
    ++pend;
    return;
  }
  BoxBest bb;
  bb.s2 = bs2; bb.d = bd; bb.s = 0.f; bb.r = 0.f; bb.j = bj; bb.k = bk;
  bb.xv = false;
  if (lane == 0 && bk >= 0) {
    // the chosen box [bk, bk + bm) from the exact integer sums: U[bk + bm] - U[bk],
    // U[x] = S[x mod nb] + ([b* < x mod nb] + floor(x / nb)) C_end; the difference is
    // a box sum (below 2^46), so it and 2^kw - it split into exact float pairs
    const int k2 = bk + bm;
    const int k2m = k2 >= nb ? k2 - nb : k2;
    const longlong2* row = WS ? srow : warp_row(a);
    const longlong2 a0 = row[bk], a1 = row[k2m];
    const long long nwrap = (bstar < k2m ? 1 : 0) + (k2 >= nb ? 1 : 0) - (bstar < bk ? 1 : 0);
    long long dw = a1.x - a0.x + nwrap * fx.w_tot;
    const long long dy = a1.y - a0.y + nwrap * fx.y_tot;
    if (NARROW) {  // r = dw / w_tot and 1 - r = (w_tot - dw) / w_tot, both sums below 2^32
      dw = (long long)(uint32_t)dw;  // the rows hold the w sums modulo 2^32
      const DF wt = df_from_ll_scaled(fx.w_tot, 0);
      bb.xr = df_div(df_from_ll_scaled(dw, 0), wt);
      bb.xq = df_div(df_from_ll_scaled(fx.w_tot - dw, 0), wt);
    } else {
      // kw lies in [24, 46] on this path: the largest weight is at most 1 and at least
      // 1/N with N <= 2^21 points, and w_max 2^kw lies in [2^24, 2^25)
      const int kw = min(max(fx.kw, 0), 62);
      bb.xr = df_from_ll_scaled(dw, kw);
      bb.xq = df_from_ll_scaled((1ll << kw) - dw, kw);  // 1 - r
    }
    bb.xs = df_from_ll_scaled(dy, fx.ky);
    bb.xv = true;
  }
  store_box(bb, lane, fidx, a.sr, a.qidx, a.kbin, a.sbest, a.rbest);
}

// One work item of a star whose table is longer than shared memory. Pass A, window
// by window (the window's cells staged once for all the item's frequencies): every
// warp adds, for each of its frequencies and bins, the prefix sums C(tau_G) of the
// window's edges G (the edges of a window are those in [ceil(w C h F),
// ceil((w+1) C h F)), the same FP64 expression on both sides of each boundary, so
// the windows partition them) to the bin's row of this block's workspace. Pass B:
// each frequency runs the block pipeline from its row.
template <int NW, bool STEP>
__device__ void windowed_item(const FixedArgs& a, const WorkItem& wi, const StarDev& st, const FixedStar& fx,
                              unsigned char* smem, int warp, int lane, uint32_t st4, uint32_t st8, uint32_t st16) {
  const int nc = st.n_cells;
  const int cap = st.win_cap + 1;  // staged cells of a window, plus one past its end
  const uint32_t loc_off = fixed_loc_off(cap), base_off = fixed_base_off(cap);
  // pass B reads the workspace rows only: its rings overlay the window's table
  float2* ring = reinterpret_cast<float2*>(smem) + warp * kRing;
  const int stride = wi.pad0;      // workspace row length (bins)
  longlong2* ws = a.ws + (size_t)blockIdx.x * (size_t)a.ws_block;
  const double h = st.h;
  const double* tp = a.tp + st.pt_off;
  const int32_t* gidx = a.gidx + st.cell_off;
  const uint32_t* s_dt = reinterpret_cast<const uint32_t*>(smem);
  for (int w = 0; w < st.n_win; ++w) {
    const int cstart = w * st.win_cells;
    const int lo = (w == 0) ? 0 : ((cstart - 1) >> 5) << 5;
    const int hi = (w == st.n_win - 1) ? nc : min(nc, (w + 1) * st.win_cells + st.win_ovl);
    const int n_loc = hi - lo + 1;
    __syncthreads();  // the previous window's passes are done
    {
      uint32_t* d_dt = reinterpret_cast<uint32_t*>(smem);
      int2* d_loc = reinterpret_cast<int2*>(smem + loc_off);
      longlong2* d_base = reinterpret_cast<longlong2*>(smem + base_off);
      const int2 lnc = a.loc[st.cell_off + nc];
      for (int i = threadIdx.x; i <= n_loc; i += NW * 32) {  // n_loc + 1 cells
        const int c = lo + i;
        d_dt[i] = c <= nc ? a.dt[st.cell_off + c] : 0xffffffffu;
        d_loc[i] = c <= nc ? a.loc[st.cell_off + c] : ((c >> 5) == (nc >> 5) ? lnc : make_int2(0, (int)kLocBias));
      }
      for (int i = threadIdx.x; i < (n_loc + 32) / 32; i += NW * 32) {
        const int g = (lo >> 5) + i;
        d_base[i] = g <= (nc >> 5) ? a.base[st.base_off + g] : make_longlong2(fx.w_tot, fx.y_tot);
      }
    }
    __syncthreads();
    for (int fl = warp; fl < wi.f_count; fl += NW) {
      const int64_t fidx = st.f_off + wi.f_begin + fl;
      const FreqRec R = a.frec[fidx];
      const int nb = R.nb;
      if (nb == 0) continue;  // reported by pass B
      const double f = a.fq[fidx].x;
      const double Fq = __dmul_rn(f, (double)nb);
      const int gq = (int)(R.gq_bstar >> 13), bstar = (int)(R.gq_bstar & 8191u);
      const int g_end = gq * nb + bstar;
      const int gs = (w == 0) ? 0 : (int)ceil(__dmul_rn(__dmul_rn((double)cstart, h), Fq));
      const int ge = (w == st.n_win - 1) ? g_end + 1
                                          : (int)ceil(__dmul_rn(__dmul_rn((double)((w + 1) * st.win_cells), h), Fq));
      const uint32_t k_lo = (uint32_t)R.K, k_hi = (uint32_t)(R.K >> 32);
      const unsigned long long XS =  // nb K: the step from a bin's edge to its next
          STEP ? (unsigned long long)(uint32_t)nb * k_lo + ((unsigned long long)((uint32_t)nb * k_hi) << 32) : 0ull;
      const uint32_t band_q = R.band_q;
      longlong2* row = ws + (size_t)fl * (size_t)stride;
      // this bin's edges in [gs, ge): cycles c0 = max(0, ceil((gs - x) / nb)) .. c1 =
      // floor((ge - 1 - x) / nb) for x = 32 i + lane. With A = gs + nb - 1 - 32 i = qa nb + ra
      // and B = ge - 1 - 32 i = qb nb + rb (0 <= ra, rb < nb) and lane < 32 <= nb, they are
      // qa - [lane > ra] (at least 0) and qb - [lane > rb] (below 0: no edge); (q, r) step
      // down by 32 bins per block with at most one borrow, so the divisions are once per
      // window and frequency
      int qa = (gs + nb - 1) / nb, ra = (gs + nb - 1) - qa * nb;
      int qb, rb;
      if (ge - 1 >= 0) {
        qb = (ge - 1) / nb;
        rb = (ge - 1) - qb * nb;
      } else {
        qb = -1;
        rb = ge - 1 + nb;
      }
      for (int i = 0; (i << 5) < nb; ++i) {
        const int x = (i << 5) + lane;
        const bool inb = x < nb;
        // the edge at t' = 0 is skipped
        int c0 = max(0, qa - (lane > ra ? 1 : 0));
        if (x == 0 && c0 == 0) c0 = 1;
        const int c1 = qb - (lane > rb ? 1 : 0);
        ra -= 32;
        if (ra < 0) {
          ra += nb;
          --qa;
        }
        rb -= 32;
        if (rb < 0) {
          rb += nb;
          --qb;
        }
        const int cntl = inb ? max(0, c1 - c0 + 1) : 0;
        const int cmax = __reduce_max_sync(0xffffffffu, (unsigned)cntl);
        long long aw = 0, ay = 0;
        bool near = false;
        // tau_G / h in 24.40 fixed point: G K modulo 2^64, by the product (STEP false)
        // or stepped by nb K from edge to edge (the same bits)
        const int G0 = x + c0 * nb;
        unsigned long long X =
            (unsigned long long)(uint32_t)G0 * k_lo + ((unsigned long long)((uint32_t)G0 * k_hi) << 32);
        for (int k = 0; k < cmax; ++k, X += XS) {
          const bool valid = k < cntl;
          if constexpr (!STEP) {
            const int G = x + (c0 + k) * nb;
            X = (unsigned long long)(uint32_t)G * k_lo + ((unsigned long long)((uint32_t)G * k_hi) << 32);
          }
          const int ul = min(max((int)((uint32_t)(X >> 32) >> 8) - lo, 0), n_loc - 1);  // staged cell
          const uint32_t fr = (uint32_t)(X >> 8);
          const uint32_t dq = *reinterpret_cast<const uint32_t*>(smem + (uint32_t)ul * st4);
          near = near || (valid && (uint32_t)(dq - fr + band_q) <= 2u * band_q);
          const int v = ul + (dq < fr ? 1 : 0);
          const int2 lc = *reinterpret_cast<const int2*>(smem + loc_off + (uint32_t)v * st8);
          const longlong2 bs = *reinterpret_cast<const longlong2*>(smem + base_off + (uint32_t)(v >> 5) * st16);
          if (valid) add_cell(aw, ay, bs, lc);
        }
        ay -= (long long)cntl * kLocBias;
        if (__any_sync(0xffffffffu, near)) {  // rare: redo, near-ties by the exact FP64 fold
          if (near) {
            aw = 0;
            ay = 0;
            for (int c = c0; c <= c1; ++c) {
              const int G = x + c * nb;
              const unsigned long long X =
                  (unsigned long long)(uint32_t)G * k_lo + ((unsigned long long)((uint32_t)G * k_hi) << 32);
              const int ul = min(max((int)((uint32_t)(X >> 32) >> 8) - lo, 0), n_loc - 1);
              const uint32_t fr = (uint32_t)(X >> 8);
              const uint32_t dq = s_dt[ul];
              int sel = dq < fr ? 1 : 0;
              if (dq != 0xffffffffu && (uint32_t)(dq - fr + band_q) <= 2u * band_q)
                sel = exact_before(tp, gidx[lo + ul], f, nb, G);
              const int v = ul + sel;
              const int2 lc = reinterpret_cast<const int2*>(smem + loc_off)[v];
              const longlong2 bs = reinterpret_cast<const longlong2*>(smem + base_off)[v >> 5];
              add_cell(aw, ay, bs, lc);
              ay -= kLocBias;
            }
          }
        }
        if (inb) {
          if (w == 0) {
            row[x] = make_longlong2(aw, ay);
          } else {
            const longlong2 o = row[x];
            row[x] = make_longlong2(o.x + aw, o.y + ay);
          }
        }
      }
    }
  }
  __syncthreads();  // every window's sums are in the workspace
  const float scw = fx.scw;
  const float scy = __int_as_float((127 - fx.ky) << 23);
  for (int fl = warp; fl < wi.f_count; fl += NW) {
    const int64_t fidx = st.f_off + wi.f_begin + fl;
    const FreqRec R = a.frec[fidx];
    if (R.nb == 0) {
      if (lane == 0) {
        atomicOr(a.err, kErrNbins);
        a.sr[fidx] = 0.f;
        if (a.qidx) a.qidx[fidx] = 255;
        if (a.kbin) a.kbin[fidx] = 0xffffffffu;
        if (a.sbest) a.sbest[fidx] = 0.f;
        if (a.rbest) a.rbest[fidx] = 0.f;
      }
      continue;
    }
    int no_pend = 0;
    run_frequency<true, false>(a, fidx, R, fx, smem, loc_off, base_off, nc, ring, lane, scw, scy, tp, gidx, st4, st8,
                               st16, ws + (size_t)fl * (size_t)stride, nullptr, no_pend, fl);
  }
}

// Bulk asynchronous copy global -> shared of `bytes` (a multiple of 16; both addresses
// 16-byte aligned), completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          (uint32_t)__cvta_generic_to_shared(dst)),
      "l"(src), "r"(bytes), "r"((uint32_t)__cvta_generic_to_shared(bar))
      : "memory");
}
constexpr uint32_t kCopyWaitLimit = 1u << 24;  // polls of a table copy (each ends after ~1 us at most)

// WIN: a launch of the time-windowed tables' items alone (the edge positions of
// pass A stepped from edge to edge); else a launch that takes either kind (the plan
// gives it the whole tables' items; pass A forms each edge's position by its product)
template <int NW, bool WIN>
__global__ void __launch_bounds__(NW * 32, 1) cells_fixed_kernel(const FixedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  __shared__ int s_item, s_star, s_next;
  __shared__ __align__(8) uint64_t s_tbar;  // completion of a table's bulk copies
  uint32_t tphase = 0;                       // its phase (thread 0)
  if (threadIdx.x == 0) {
    s_star = -1;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&s_tbar))
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // element strides as run-time values, so that the table addresses are formed by
  // integer multiply-adds rather than by the (busier) integer logic pipe
  const uint32_t st4 = a.stride4, st8 = 2u * a.stride4, st16 = 4u * a.stride4;

  bool done = false;
  const int iter_lim = a.loop_bound > 0 ? min(a.loop_bound, a.n_items) : a.n_items;
  for (int iter = 0; iter <= iter_lim; ++iter) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_item = atomicAdd(a.cursor, 1);
      s_next = 0;
    }
    __syncthreads();
    const int it = s_item;
    if (it >= a.n_items) { done = true; break; }
    const WorkItem wi = a.items[it];
    const StarDev st = a.stars[wi.star];
    const FixedStar fx = a.fx[wi.star];
    if (WIN && st.n_win <= 1) {  // block-uniform; the plan never hands this launch a whole table
      if (threadIdx.x == 0) atomicOr(a.err, kErrNbins);
      continue;
    }
    if (st.n_win > 1) {  // block-uniform: a table longer than shared memory
      windowed_item<NW, WIN>(a, wi, st, fx, smem, warp, lane, st4, st8, st16);
      if (threadIdx.x == 0) s_star = -1;  // shared memory no longer holds a whole table
      continue;
    }
    const int nc = st.n_cells;  // sentinel cell index
    const int ncp = nc + 1 + kPadCells;
    const uint32_t loc_off = fixed_loc_off(ncp), base_off = fixed_base_off(ncp);
    float2* ring = reinterpret_cast<float2*>(smem + fixed_ring_off(ncp)) + warp * kRing;
    if (s_star != wi.star) {  // block-uniform: stage the star's table and its padding
      uint32_t* d_dt = reinterpret_cast<uint32_t*>(smem);
      int2* d_loc = reinterpret_cast<int2*>(smem + loc_off);
      longlong2* d_base = reinterpret_cast<longlong2*>(smem + base_off);
      // cells [0, nb4) and groups [0, ng) by bulk copies (the table starts at a 16-byte
      // boundary: cell_off is a multiple of 4), the rest of the table and the padding by
      // the threads; the two parts do not overlap
      // (the 32-bit table has no group bases: its padding cells repeat the sentinel's sums)
      const bool narrow = fx.narrow != 0;
      const int nb4 = (nc + 1) & ~3, ng = narrow ? 0 : (nc >> 5) + 1;
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // after the last item's reads
        const uint32_t bytes = (uint32_t)nb4 * 12u + (uint32_t)ng * 16u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&s_tbar)), "r"(bytes)
                     : "memory");
        if (nb4 > 0) {
          bulk_g2s(d_dt, a.dt + st.cell_off, (uint32_t)nb4 * 4u, &s_tbar);
          bulk_g2s(d_loc, a.loc + st.cell_off, (uint32_t)nb4 * 8u, &s_tbar);
        }
        if (ng > 0) bulk_g2s(d_base, a.base + st.base_off, (uint32_t)ng * 16u, &s_tbar);
      }
      const int2 lnc = a.loc[st.cell_off + nc];
      for (int i = nb4 + (int)threadIdx.x; i < ncp; i += NW * 32) {
        const bool in = i <= nc;
        d_dt[i] = in ? a.dt[st.cell_off + i] : 0xffffffffu;
        d_loc[i] = in ? a.loc[st.cell_off + i]
                      : ((narrow || (i >> 5) == (nc >> 5)) ? lnc : make_int2(0, (int)kLocBias));
      }
      if (!narrow)
        for (int i = ng + (int)threadIdx.x; i < (ncp + 31) / 32; i += NW * 32)
          d_base[i] = make_longlong2(fx.w_tot, fx.y_tot);
      if (threadIdx.x == 0) {  // bounded wait for the copies
        bool ok = false;
        for (uint32_t k = 0; k < kCopyWaitLimit && !ok; ++k) {
          uint32_t done;
          asm volatile(
              "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
              "selp.u32 %0, 1, 0, p;\n\t}"
              : "=r"(done)
              : "r"((uint32_t)__cvta_generic_to_shared(&s_tbar)), "r"(tphase)
              : "memory");
          ok = done != 0;
        }
        if (!ok) atomicOr(a.err, kErrCopyWait);
        tphase ^= 1u;
        s_star = ok ? wi.star : -1;
      }
      __syncthreads();
    }
    const float scw = fx.scw;  // 2^-kw, or 1 / w_tot on the 32-bit table
    const float scy = __int_as_float((127 - fx.ky) << 23);  // 2^-ky (|ky| <= 100)
    const double* tp = a.tp + st.pt_off;
    const int32_t* gidx = a.gidx + st.cell_off;

    longlong2* const prow = pend_rows(a);
    const int64_t f0 = st.f_off + wi.f_begin;
    int pend = 0;  // boxes waiting in prow for their rescoring (warp-uniform)
    for (int fi = 0; fi <= wi.f_count; ++fi) {  // bounded: each pass takes one frequency
      int fl = 0;
      if (lane == 0) fl = atomicAdd(&s_next, 1);
      fl = __shfl_sync(0xffffffffu, fl, 0);
      if (fl >= wi.f_count) break;
      const int64_t fidx = st.f_off + wi.f_begin + fl;
      const FreqRec R = a.frec[fidx];
      const int nb = R.nb;
      if (nb == 0) {
        if (lane == 0) {
          atomicOr(a.err, kErrNbins);
          a.sr[fidx] = 0.f;
          if (a.qidx) a.qidx[fidx] = 255;
          if (a.kbin) a.kbin[fidx] = 0xffffffffu;
          if (a.sbest) a.sbest[fidx] = 0.f;
          if (a.rbest) a.rbest[fidx] = 0.f;
        }
        continue;
      }
      if (fx.narrow)  // block-uniform
        run_frequency<false, true>(a, fidx, R, fx, smem, loc_off, base_off, nc, ring, lane, scw, scy, tp, gidx, st4,
                                   st8, st16, nullptr, prow, pend, fl);
      else
        run_frequency<false, false>(a, fidx, R, fx, smem, loc_off, base_off, nc, ring, lane, scw, scy, tp, gidx, st4,
                                    st8, st16, nullptr, prow, pend, fl);
      if (pend == 32) {
        flush_pending(a, fx, f0, prow, pend, lane);
        pend = 0;
      }
    }
    if (pend > 0) flush_pending(a, fx, f0, prow, pend, lane);
  }
  if (!done && threadIdx.x == 0) atomicOr(a.err, kErrQueueBound);
}

uint32_t fixed_smem_bytes(int ncs) { return fixed_ring_off(ncs + kPadCells) + (uint32_t)kFixedWarps * kRing * 8u; }
uint32_t fixed_window_smem_bytes(int ncs) {
  return fixed_ring_off(ncs) > (uint32_t)kFixedWarps * kRing * 8u ? fixed_ring_off(ncs) : (uint32_t)kFixedWarps * kRing * 8u;
}

int launch_cells_fixed(const FixedArgs& a, bool windowed, int blocks, size_t smem, void* stream) {
  auto kern = windowed ? cells_fixed_kernel<kFixedWarps, true> : cells_fixed_kernel<kFixedWarps, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  kern<<<blocks, kFixedWarps * 32, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

int fixed_blocks_per_sm(size_t smem) {  // the fewer of the two instantiations'
  int nmin = 0;
  for (int k = 0; k < 2; ++k) {
    auto kern = k ? cells_fixed_kernel<kFixedWarps, true> : cells_fixed_kernel<kFixedWarps, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kFixedWarps * 32, smem) != cudaSuccess) return 0;
    nmin = (k == 0 || nb < nmin) ? nb : nmin;
  }
  return nmin;
}

}  // namespace qlp
