// Cell path of the BLS search (sm_103a): bins from prefix sums at bin edges.
//
// For a trial frequency f with nbins bins, let F = f nbins; the phase-bin edges
// fall at times tau_G = G / F (G = 0, 1, ...: the global bin index of the fold
// x = t' f, b = floor(frac(x) nbins) in Sec. 2.1's BLS). A point belongs to global
// bin g when tau_g <= t' < tau_{g+1}, so with the prefix sums
// C(tau) = (sum of w, sum of w d over points with t' < tau) every histogram bin is
//     H[b] = sum over G = b mod nbins of C(tau_{G+1}) - C(tau_G),
// one term per (cycle, bin) instead of one per point. For light curves sampled
// much faster than a bin lasts (TESS 200-s cadence: 3-30 points per bin and
// cycle) this is 3-10x less work than folding every point, needs no atomics and
// is deterministic.
//
// C(tau) in O(1): the star's time axis is cut into cells of width h just below
// the smallest point spacing, so each cell holds at most one point. Per cell the
// table keeps C at the cell start (a per-32-cell double-float base plus an FP32
// local part) and the offset dt of its point (a 32-bit fraction of the cell); an
// edge's cell and position come from tau/h = G D/h in 2^-56 fixed point, so
//     C(tau) = C(cell u start) + [dt_u < tau - u h] (w, w d) = C(start of cell u + [..]).
// Near ties (|dt_u - (tau - u h)| within a guard band) are decided exactly by the
// FP64 fold of that point: "point before edge G" is "its FP64 global bin < G".
//
// K1c prep_cells_kernel (1 CTA per cell-path star): weights as prep_kernel, FP64
// prefix sums, the per-cell tables. K2c cells_kernel: persistent, work queue of
// (star, frequency chunk), the star's tables staged in shared memory, one warp
// per frequency, lanes on 32 consecutive edges (31 bins) per step; then the same
// box sweep as the per-point kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "bls_device.cuh"
#include "qlp_internal.h"

namespace qlp {

// ------------------------------------------------------------------ K1c

__global__ void __launch_bounds__(256) prep_cells_kernel(const PrepCellsArgs a) {
  __shared__ double red[32];
  __shared__ double scan_w[256], scan_y[256];
  const int s = a.cell_stars[blockIdx.x];
  const StarDev st = a.stars[s];
  const int n = st.n_pts;
  if (n <= 0) return;
  const double* tp = a.tp + st.pt_off;
  const double* y = a.y + st.pt_off;
  const double* dy = a.dy + st.pt_off;
  const int tid = threadIdx.x;

  double acc = 0.0;
  for (int i = tid; i < n; i += blockDim.x) acc += 1.0 / (dy[i] * dy[i]);
  // block sum (FP64)
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  double wsum = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) wsum += red[i];
  __syncthreads();
  acc = 0.0;
  for (int i = tid; i < n; i += blockDim.x) acc += (1.0 / (dy[i] * dy[i])) / wsum * y[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  double ybar = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) ybar += red[i];

  // prefix sums before each point: contiguous segment per thread, scan of totals
  const int L = (n + blockDim.x - 1) / blockDim.x;
  const int i0 = min(n, tid * L), i1 = min(n, i0 + L);
  double sw = 0.0, sy = 0.0;
  for (int i = i0; i < i1; ++i) {
    const double ww = (1.0 / (dy[i] * dy[i])) / wsum;
    sw += ww;
    sy += ww * (y[i] - ybar);
  }
  scan_w[tid] = sw;
  scan_y[tid] = sy;
  __syncthreads();
  if (tid == 0) {  // exclusive scan of 256 segment totals (FP64, sequential)
    double rw = 0.0, ry = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) {
      const double tw = scan_w[k], ty = scan_y[k];
      scan_w[k] = rw;
      scan_y[k] = ry;
      rw += tw;
      ry += ty;
    }
    a.cpre[st.cpre_off + n] = make_double2(rw, ry);
  }
  __syncthreads();
  double cw = scan_w[tid], cy = scan_y[tid];
  for (int i = i0; i < i1; ++i) {
    a.cpre[st.cpre_off + i] = make_double2(cw, cy);
    const double ww = (1.0 / (dy[i] * dy[i])) / wsum;
    cw += ww;
    cy += ww * (y[i] - ybar);
  }

  // first point at or after each cell start: point i fills cells (cell(i-1), cell(i)]
  const int nc = st.n_cells;
  const double h = st.h;
  int32_t* first = a.gidx + st.cell_off;
  for (int i = tid; i <= n; i += blockDim.x) {
    const int up = (i == 0) ? -1 : cell_of(tp[i - 1], h);
    const int ui = (i == n) ? nc : cell_of(tp[i], h);
    for (int c = up + 1; c <= ui && c <= nc; ++c) first[c] = i;
  }
  __syncthreads();
  for (int u = tid; u <= nc; u += blockDim.x) {
    const int f = first[u];
    const bool in_cell = (u < nc) && (f < n) && (cell_of(tp[f], h) == u);
    // offset of the cell's point as a 32-bit fraction of the cell, empty = 0xFFFFFFFF
    uint32_t q = 0xffffffffu;
    if (in_cell) {
      const double fr = __ddiv_rn(__dsub_rn(tp[f], __dmul_rn((double)u, h)), h);
      q = (uint32_t)fmin(floor(__dmul_rn(fr, 4294967296.0)), 4294967294.0);
    }
    a.dt[st.cell_off + u] = q;
    const double2 c = a.cpre[st.cpre_off + f];
    const double2 cb = a.cpre[st.cpre_off + first[u & ~31]];
    a.loc[st.cell_off + u] = make_float2(__double2float_rn(c.x - cb.x), __double2float_rn(c.y - cb.y));
    if ((u & 31) == 0) {
      const float wh = __double2float_rn(cb.x), yh = __double2float_rn(cb.y);
      a.base[st.base_off + (u >> 5)] =
          make_float4(wh, __double2float_rn(cb.x - (double)wh), yh, __double2float_rn(cb.y - (double)yh));
    }
  }
}

int launch_prep_cells(const PrepCellsArgs& a, void* stream) {
  if (a.n <= 0) return 0;
  prep_cells_kernel<<<a.n, 256, 0, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ K2c

// Shared-memory layout of one star's cell table followed by the per-warp
// duration tables and histograms (the histogram stride is chosen per work item).
struct CellSmem {
  uint32_t loc, base, mtab, hist;
};
__host__ __device__ __forceinline__ CellSmem cell_smem_layout(int ncs, int nw) {
  CellSmem l;
  l.loc = ((uint32_t)ncs * 4u + 15u) & ~15u;
  l.base = l.loc + (((uint32_t)ncs * 8u + 15u) & ~15u);
  l.mtab = l.base + ((((uint32_t)ncs + 31u) / 32u * 16u + 15u) & ~15u);
  l.hist = l.mtab + (uint32_t)nw * kMaxQ * 4u;
  return l;
}

// C(tau_G) for one edge: prefix sums (w, w d) of the points before tau_G = G D,
// as (block base hi, lo; local part) for w and for w d.
struct EdgeC {
  float bwh, bwl, byh, byl, lw, ly;
};

// Prefix sums at edge G from the staged table window [lo, lo + n_loc): cells
// outside it are clamped (only lanes whose result is discarded reach them).
__device__ __forceinline__ EdgeC edge_prefix(int G, bool valid, uint32_t k_lo, uint32_t k_hi, int nc,
                                             int lo, int n_loc, uint32_t band_q, const uint32_t* s_dt,
                                             const float2* s_loc, const float4* s_base,
                                             const double* tp, const int32_t* gidx, double f,
                                             int nb) {
  // tau_G / h in 2^-56 fixed point: G (32 bits) x K (64 bits) -> 96 bits
  const unsigned long long lo64 = (unsigned long long)(uint32_t)G * k_lo;
  const unsigned long long hi64 = (unsigned long long)(uint32_t)G * k_hi + (lo64 >> 32);
  const int u = (int)min((unsigned long long)nc, hi64 >> 24);          // cell (global)
  const uint32_t fr = ((uint32_t)hi64 << 8) | ((uint32_t)lo64 >> 24);  // position in the cell, 2^-32
  const int ul = min(max(u - lo, 0), n_loc - 1);                        // cell in the window
  const uint32_t dq = s_dt[ul];
  int sel = dq < fr ? 1 : 0;                                             // the cell's point is before tau
  const bool need = valid && (dq != 0xffffffffu) && (uint32_t)(dq - fr + band_q) <= 2u * band_q;
  if (__any_sync(0xffffffffu, need)) {  // rare: decide by the exact FP64 fold
    if (need) sel = exact_before(tp, gidx[lo + ul], f, nb, G);
  }
  const int vl = min(ul + sel, n_loc - 1);
  const float2 lc = s_loc[vl];
  const float4 bs = s_base[vl >> 5];  // lo is a multiple of 32
  EdgeC c;
  c.bwh = bs.x; c.bwl = bs.y; c.byh = bs.z; c.byl = bs.w; c.lw = lc.x; c.ly = lc.y;
  return c;
}

// Piece between this lane's edge and the next lane's: (w, w d) of the points in
// one (cycle, bin).
__device__ __forceinline__ float2 edge_piece(const EdgeC& c) {
  const float nbwh = __shfl_down_sync(0xffffffffu, c.bwh, 1);
  const float nbwl = __shfl_down_sync(0xffffffffu, c.bwl, 1);
  const float nbyh = __shfl_down_sync(0xffffffffu, c.byh, 1);
  const float nbyl = __shfl_down_sync(0xffffffffu, c.byl, 1);
  const float nlw = __shfl_down_sync(0xffffffffu, c.lw, 1);
  const float nly = __shfl_down_sync(0xffffffffu, c.ly, 1);
  const float pw = __fadd_rn(__fadd_rn(__fsub_rn(nbwh, c.bwh), __fsub_rn(nbwl, c.bwl)), __fsub_rn(nlw, c.lw));
  const float py = __fadd_rn(__fadd_rn(__fsub_rn(nbyh, c.byh), __fsub_rn(nbyl, c.byl)), __fsub_rn(nly, c.ly));
  return make_float2(pw, py);
}

template <int SUM>
__device__ __forceinline__ void add_piece(typename PackedBin<SUM>::T* h, int b, float2 pc, bool own, bool p) {
  if (!p) return;
  if (own) {  // lanes 0..30 hold distinct bins
    typename PackedBin<SUM>::T v = h[b];
    if constexpr (SUM == QLP_SUM_COMP) {
      float sN = __fadd_rn(v.x, pc.x);
      v.y = __fadd_rn(v.y, two_sum_err(v.x, pc.x, sN));
      v.x = sN;
      sN = __fadd_rn(v.z, pc.y);
      v.w = __fadd_rn(v.w, two_sum_err(v.z, pc.y, sN));
      v.z = sN;
    } else {
      v.x = __fadd_rn(v.x, pc.x);
      v.y = __fadd_rn(v.y, pc.y);
    }
    h[b] = v;
  } else {
    float* f = reinterpret_cast<float*>(h + b);
    atomicAdd(f, pc.x);
    atomicAdd(f + (SUM == QLP_SUM_COMP ? 2 : 1), pc.y);
  }
}

template <int SUM, int NW>
__global__ void __launch_bounds__(NW * 32) cells_kernel(const CellArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NA = (SUM == QLP_SUM_COMP) ? 4 : 2;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int nq = a.nq;
  const uint32_t* s_dt = reinterpret_cast<const uint32_t*>(smem);

  __shared__ int s_item;
  __shared__ int s_star;
  __shared__ int s_win;
  if (threadIdx.x == 0) { s_star = -1; s_win = -1; }

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
    const int nc = st.n_cells;  // sentinel index
    const int n_win = st.n_win;
    const CellSmem L = cell_smem_layout(st.win_cap, NW);
    const float2* s_loc = reinterpret_cast<const float2*>(smem + L.loc);
    const float4* s_base = reinterpret_cast<const float4*>(smem + L.base);
    // per item: histogram stride (multiple of 32 floats) and the warps that fit
    const int HS = (wi.pad0 & 0xffff) * 32;
    const int wact = wi.pad0 >> 16;
    int* mtab = reinterpret_cast<int*>(smem + L.mtab) + warp * kMaxQ;
    using HT = typename PackedBin<SUM>::T;
    HT* hist = reinterpret_cast<HT*>(reinterpret_cast<float*>(smem + L.hist) + (size_t)warp * NA * HS);
    const double* tp = a.tp + st.pt_off;
    const int32_t* gidx = a.gidx + st.cell_off;
    const double h = st.h;

    for (int r0 = 0; r0 < wi.f_count; r0 += wact) {  // every warp runs every round (barriers)
      const int fl = r0 + warp;
      const bool active = warp < wact && fl < wi.f_count;
      const int64_t fidx = st.f_off + wi.f_begin + (active ? fl : 0);
      // one pass over the shared histogram, or one per duration (per-duration bins)
      const int n_pass = a.per_q ? nq : 1;
      BoxBest acc;
      acc.s2 = -1.f; acc.d = 1.f; acc.s = 0.f; acc.r = 0.f; acc.j = 255; acc.k = -1;
      acc.xv = false;
      bool failed = false;
      for (int pass = 0; pass < n_pass; ++pass) {
        double f = 0.0, F = 1.0;
        int nb = 1, g_end = 0;
        uint32_t k_lo = 0, k_hi = 0, band_q = 0;
        bool go = active && !failed;
        if (go) {
          const double2 fq = a.fq[fidx];
          f = fq.x;
          const double qb = a.per_q ? __dmul_rn(fq.y, a.E[pass]) : fq.y;  // bin = qb / noverlap
          nb = (int)ceil(__ddiv_rn(a.noverlap, qb));
          if (nb + kMPad > HS || nb < 1) {
            if (lane == 0) atomicOr(a.err, kErrNbins);
            go = false;
            failed = true;
          } else {
            if (a.per_q) {
              if (lane == 0) mtab[0] = a.m_perq;
            } else if (lane < nq) {
              mtab[lane] = max(1, (int)floor(__dadd_rn(__dmul_rn(__dmul_rn(fq.y, a.E[lane]), (double)nb), 0.5)));
            }
            for (int i = lane; i < nb + kMPad; i += 32) hist[i] = HT{};
            F = __dmul_rn(f, (double)nb);
            const double D = __ddiv_rn(1.0, F);  // bin duration (days)
            const double yT = __dmul_rn(st.baseline, F);
            g_end = (int)floor(yT) + 2;  // edges 0 .. g_end; tau_{g_end} > T
            // edge step in cells, 2^-56 fixed point (D/h < 2^8)
            const unsigned long long K = __double2ull_rn(__dmul_rn(__ddiv_rn(D, h), 72057594037927936.0));
            k_lo = (uint32_t)K;
            k_hi = (uint32_t)(K >> 32);
            // guard band in 2^-32 cell units: the FP64 fold's and this fixed-point edge's
            // errors (2^-20 + 2^-40 T F bins, converted) plus the table's quantisation
            band_q = (uint32_t)fmin(
                __dmul_rn(__ddiv_rn(__dmul_rn(9.5367431640625e-07 + 9.094947017729282e-13 * yT, D), h),
                          4294967296.0) + 64.0, 1073741824.0);
          }
        }
        __syncwarp();
        const bool own = nb >= 31;  // the 31 pieces of one chunk fall in distinct bins
        const int step = 31 % nb;

        for (int w = 0; w < n_win; ++w) {
          const int cstart = w * st.win_cells;  // first cell owned by window w
          const int lo = (n_win == 1) ? 0 : max(0, ((cstart - 1) >> 5) << 5);
          const int hi = (w == n_win - 1) ? nc : min(nc, (w + 1) * st.win_cells + st.win_ovl);
          const int n_loc = hi - lo + 1;
          if (s_star != wi.star || s_win != w) {  // block-uniform
            __syncthreads();
            uint32_t* d_dt = reinterpret_cast<uint32_t*>(smem);
            float2* d_loc = reinterpret_cast<float2*>(smem + L.loc);
            float4* d_base = reinterpret_cast<float4*>(smem + L.base);
            for (int i = threadIdx.x; i < n_loc; i += NW * 32) {
              d_dt[i] = a.dt[st.cell_off + lo + i];
              d_loc[i] = a.loc[st.cell_off + lo + i];
            }
            const int b0 = lo >> 5, b1 = hi >> 5;
            for (int i = threadIdx.x; i <= b1 - b0; i += NW * 32) d_base[i] = a.base[st.base_off + b0 + i];
            if (threadIdx.x == 0) { s_star = wi.star; s_win = w; }
            __syncthreads();
          }
          if (!go) continue;
          // pieces [gs, ge) of this window: edges from the first at or after its start
          const int gs = (w == 0) ? 0 : (int)ceil(__dmul_rn(__dmul_rn((double)cstart, h), F));
          const int ge = (w == n_win - 1) ? g_end
                                          : (int)ceil(__dmul_rn(__dmul_rn((double)((w + 1) * st.win_cells), h), F));
          int b = (gs + lane) % nb;  // bin of this lane's piece in the first chunk
          for (int g0 = gs; g0 < ge; g0 += 62) {
            // two chunks of 31 pieces in flight: edges g0 .. g0+31 and g0+31 .. g0+62
            const EdgeC c0 = edge_prefix(g0 + lane, g0 + lane <= ge, k_lo, k_hi, nc, lo, n_loc, band_q, s_dt,
                                         s_loc, s_base, tp, gidx, f, nb);
            const EdgeC c1 = edge_prefix(g0 + 31 + lane, g0 + 31 + lane <= ge, k_lo, k_hi, nc, lo, n_loc,
                                         band_q, s_dt, s_loc, s_base, tp, gidx, f, nb);
            const float2 p0 = edge_piece(c0);
            const float2 p1 = edge_piece(c1);
            int b1 = b + step;
            if (b1 >= nb) b1 -= nb;
            add_piece<SUM>(hist, b, p0, own, lane < 31 && g0 + lane < ge);
            add_piece<SUM>(hist, b1, p1, own, lane < 31 && g0 + 31 + lane < ge);
            b = b1 + step;
            if (b >= nb) b -= nb;
          }
        }
        if (go) {
          __syncwarp();
          BoxBest bb = sweep_best_packed<SUM>(hist, mtab, a.per_q ? 1 : nq, nb, lane);
          if (a.per_q && bb.s2 >= 0.f) bb.j = pass;  // the duration of this histogram
          // across passes: a later (longer) duration must beat the earlier ones strictly
          if (beats(bb.s2, bb.d, bb.j, bb.k, acc.s2, acc.d, acc.j, acc.k)) acc = bb;
          __syncwarp();
        }
      }
      if (active) {
        if (failed) {
          if (lane == 0) {
            a.sr[fidx] = 0.f;
            if (a.qidx) a.qidx[fidx] = 255;
            if (a.kbin) a.kbin[fidx] = 0xffffffffu;
            if (a.sbest) a.sbest[fidx] = 0.f;
            if (a.rbest) a.rbest[fidx] = 0.f;
          }
        } else {
          store_box(acc, lane, fidx, a.sr, a.qidx, a.kbin, a.sbest, a.rbest);
        }
      }
    }
  }
  if (!done && threadIdx.x == 0) atomicOr(a.err, kErrQueueBound);
}

template <int SUM, int NW>
static int launch_cells_t(const CellArgs& a, int blocks, size_t smem, void* stream) {
  auto kern = cells_kernel<SUM, NW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  kern<<<blocks, NW * 32, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

template <int SUM, int NW>
static int occ_cells_t(size_t smem) {
  auto kern = cells_kernel<SUM, NW>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NW * 32, smem) != cudaSuccess) return 0;
  return nb;
}

#define QLP_CELLS_DISPATCH(FN, ...)                                                   \
  switch (sum_mode * 10 + (warps == 4 ? 0 : warps == 8 ? 1 : warps == 16 ? 2 : 3)) { \
    case 0: return FN<0, 4>(__VA_ARGS__);                                             \
    case 1: return FN<0, 8>(__VA_ARGS__);                                             \
    case 2: return FN<0, 16>(__VA_ARGS__);                                            \
    case 3: return FN<0, 32>(__VA_ARGS__);                                            \
    case 10: return FN<1, 4>(__VA_ARGS__);                                            \
    case 11: return FN<1, 8>(__VA_ARGS__);                                            \
    case 12: return FN<1, 16>(__VA_ARGS__);                                           \
    case 13: return FN<1, 32>(__VA_ARGS__);                                           \
    default: break;                                                                   \
  }

int launch_cells(const CellArgs& a, int sum_mode, int warps, int blocks, size_t smem, void* stream) {
  QLP_CELLS_DISPATCH(launch_cells_t, a, blocks, smem, stream)
  return (int)cudaErrorInvalidValue;
}

uint32_t cells_hist_offset(int ncs, int nw) { return cell_smem_layout(ncs, nw).hist; }

int cells_blocks_per_sm(int sum_mode, int warps, size_t smem) {
  QLP_CELLS_DISPATCH(occ_cells_t, smem)
  return 0;
}

}  // namespace qlp
