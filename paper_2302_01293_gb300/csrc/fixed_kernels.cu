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
// K1x prep_fixed_kernel (1 CTA per exact-path star): weights and the weighted
// mean in FP64 as the other prep kernels, the integer weights, their exact
// prefix sums, the per-cell tables (offset of the cell's point, prefix sums at
// the cell start as a 64-bit group base plus a 32-bit local part), and one
// FreqRec per trial frequency (bins, the edge step in 2^-56 cells, guard band,
// last edge, the bins m_j of each duration).
// K2x cells_fixed_kernel: persistent; work queue of (star, frequency chunk); the
// star's table in shared memory; warps take the item's frequencies one at a time.
// Per frequency the bins are handled 32 at a time (lane = bin): the lanes'
// S values become U, converted to a double-float (hi, lo) pair per quantity and
// written to a per-warp ring of two 32-bin blocks (plus a copy of the even block
// behind the odd one, so that block i and i+1 are always contiguous); the sweep
// of block i - 1 runs as soon as block i is in the ring.
#include <cuda_runtime.h>

#include <cstdint>

#include "bls_device.cuh"
#include "qlp_internal.h"

namespace qlp {

constexpr int kRing = 96;  // float2 per warp: blocks 2i and 2i+1, then a copy of block 2i

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

__device__ __forceinline__ double block_sum256(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

__device__ __forceinline__ double block_max256(double v, double* red) {
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

__global__ void __launch_bounds__(256) prep_fixed_kernel(const PrepFixedArgs a) {
  __shared__ double red[8];
  __shared__ long long scan_w[256], scan_y[256];
  const int s = a.fixed_stars[blockIdx.x];
  const StarDev st = a.stars[s];
  const int n = st.n_pts;
  if (n <= 0) return;
  const double* tp = a.tp + st.pt_off;
  const double* y = a.y + st.pt_off;
  const double* dy = a.dy + st.pt_off;
  const int tid = threadIdx.x;

  // weights w = dy^-2 / sum dy^-2 and the weighted mean (FP64)
  double acc = 0.0;
  for (int i = tid; i < n; i += blockDim.x) acc += 1.0 / (dy[i] * dy[i]);
  const double wsum = block_sum256(acc, red);
  acc = 0.0;
  for (int i = tid; i < n; i += blockDim.x) acc += (1.0 / (dy[i] * dy[i])) / wsum * y[i];
  const double ybar = block_sum256(acc, red);
  double mw = 0.0, md = 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    const double w = (1.0 / (dy[i] * dy[i])) / wsum;
    mw = fmax(mw, w);
    md = fmax(md, fabs(w * (y[i] - ybar)));
  }
  mw = block_max256(mw, red);
  md = block_max256(md, red);
  const int kw = fixed_exponent(mw), ky = fixed_exponent(md);
  const double pw = ldexp(1.0, kw), py = ldexp(1.0, ky);

  // exact prefix sums of the integer weights: contiguous segment per thread,
  // exclusive scan of the segment totals
  const int L = (n + blockDim.x - 1) / blockDim.x;
  const int i0 = min(n, tid * L), i1 = min(n, i0 + L);
  long long sw = 0, sy = 0;
  for (int i = i0; i < i1; ++i) {
    const double w = (1.0 / (dy[i] * dy[i])) / wsum;
    sw += __double2ll_rn(w * pw);
    sy += __double2ll_rn(w * (y[i] - ybar) * py);
  }
  scan_w[tid] = sw;
  scan_y[tid] = sy;
  __syncthreads();
  if (tid == 0) {
    long long rw = 0, ry = 0;
    for (int k = 0; k < (int)blockDim.x; ++k) {
      const long long tw = scan_w[k], ty = scan_y[k];
      scan_w[k] = rw;
      scan_y[k] = ry;
      rw += tw;
      ry += ty;
    }
    a.ipre[st.cpre_off + n] = make_longlong2(rw, ry);
    FixedStar f;
    f.w_tot = rw;
    f.y_tot = ry;
    f.kw = kw;
    f.ky = ky;
    a.fx[s] = f;
  }
  __syncthreads();
  long long cw = scan_w[tid], cy = scan_y[tid];
  for (int i = i0; i < i1; ++i) {
    a.ipre[st.cpre_off + i] = make_longlong2(cw, cy);
    const double w = (1.0 / (dy[i] * dy[i])) / wsum;
    cw += __double2ll_rn(w * pw);
    cy += __double2ll_rn(w * (y[i] - ybar) * py);
  }
  __syncthreads();

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
    uint32_t q = 0xffffffffu;  // the cell's point as a 32-bit fraction of the cell, empty = all ones
    if (in_cell) {
      const double fr = __ddiv_rn(__dsub_rn(tp[f], __dmul_rn((double)u, h)), h);
      q = (uint32_t)fmin(floor(__dmul_rn(fr, 4294967296.0)), 4294967294.0);
    }
    a.dt[st.cell_off + u] = q;
    const longlong2 c = a.ipre[st.cpre_off + f];
    const longlong2 cb = a.ipre[st.cpre_off + first[u & ~31]];
    a.loc[st.cell_off + u] = make_int2((int)(c.x - cb.x), (int)(c.y - cb.y));
    if ((u & 31) == 0) a.base[st.base_off + (u >> 5)] = cb;
  }

  // per trial frequency: the same FP64 operations as the other search kernels
  for (int k = tid; k < st.n_f; k += blockDim.x) {
    const int64_t fidx = st.f_off + k;
    const double2 fq = a.fq[fidx];
    FreqRec r;
    r.K = 0ull;
    r.mpack = 0ull;
    r.nb = 0;
    r.band_q = 0u;
    r.g_end = 0;
    r.pad = 0;
    const int nb = (int)ceil(__ddiv_rn(a.noverlap, fq.y));
    if (nb >= 32 && nb <= a.nb_cap) {
      const double F = __dmul_rn(fq.x, (double)nb);
      const double D = __ddiv_rn(1.0, F);  // bin duration (days)
      const double yT = __dmul_rn(st.baseline, F);
      r.g_end = (int)floor(yT) + 2;  // edges 0 .. g_end; tau_{g_end} > T
      r.K = __double2ull_rn(__dmul_rn(__ddiv_rn(D, h), 72057594037927936.0));
      // guard band in 2^-32 cell units: the FP64 fold's and the fixed-point edge's
      // errors (2^-20 + 2^-40 T F bins, converted) plus the table's quantisation
      r.band_q = (uint32_t)fmin(
          __dmul_rn(__ddiv_rn(__dmul_rn(9.5367431640625e-07 + 9.094947017729282e-13 * yT, D), h), 4294967296.0) +
              64.0,
          1073741824.0);
      unsigned long long mp = 0ull;
      for (int j = 0; j < a.nq; ++j) {
        const int m = max(1, (int)floor(__dadd_rn(__dmul_rn(__dmul_rn(fq.y, a.E[j]), (double)nb), 0.5)));
        mp |= (unsigned long long)min(m, 15) << (4 * j);
      }
      r.mpack = mp;
      r.nb = nb;
    }
    a.frec[fidx] = r;
  }
}

int launch_prep_fixed(const PrepFixedArgs& a, void* stream) {
  if (a.n <= 0) return 0;
  prep_fixed_kernel<<<a.n, 256, 0, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ K2x

template <int NW>
__global__ void __launch_bounds__(NW * 32, 1) cells_fixed_kernel(const FixedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  __shared__ int s_item, s_star, s_next;
  if (threadIdx.x == 0) s_star = -1;

  bool done = false;
  for (int iter = 0; iter <= a.n_items; ++iter) {
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
    const int nc = st.n_cells;  // sentinel cell index
    const int ncs = nc + 1;
    const uint32_t* s_dt = reinterpret_cast<const uint32_t*>(smem);
    const int2* s_loc = reinterpret_cast<const int2*>(smem + fixed_loc_off(ncs));
    const longlong2* s_base = reinterpret_cast<const longlong2*>(smem + fixed_base_off(ncs));
    float2* ring = reinterpret_cast<float2*>(smem + fixed_ring_off(ncs)) + warp * kRing;
    if (s_star != wi.star) {  // block-uniform: stage the star's table
      uint32_t* d_dt = reinterpret_cast<uint32_t*>(smem);
      int2* d_loc = reinterpret_cast<int2*>(smem + fixed_loc_off(ncs));
      longlong2* d_base = reinterpret_cast<longlong2*>(smem + fixed_base_off(ncs));
      for (int i = threadIdx.x; i < ncs; i += NW * 32) {
        d_dt[i] = a.dt[st.cell_off + i];
        d_loc[i] = a.loc[st.cell_off + i];
      }
      for (int i = threadIdx.x; i < (ncs + 31) / 32; i += NW * 32) d_base[i] = a.base[st.base_off + i];
      __syncthreads();
      if (threadIdx.x == 0) s_star = wi.star;
    }
    const FixedStar fx = a.fx[wi.star];
    const float scw = __int_as_float((127 - fx.kw) << 23);  // 2^-kw (|kw| <= 100)
    const float scy = __int_as_float((127 - fx.ky) << 23);
    const double* tp = a.tp + st.pt_off;
    const int32_t* gidx = a.gidx + st.cell_off;

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
      const double f = a.fq[fidx].x;  // for the exact decision near ties
      const int g_end = R.g_end;
      const uint32_t band_q = R.band_q;
      // widths present (bit w-1 for a box of w bins) and the lowest duration index j
      // of each width (4 bits per width); m_j is non-decreasing in j
      uint32_t wmask = 0u;
      unsigned long long jlow = 0ull;
      int mmax = 1;
      for (int j = a.nq - 1; j >= 0; --j) {
        const int m = (int)((R.mpack >> (4 * j)) & 15ull);
        wmask |= 1u << (m - 1);
        jlow = (jlow & ~(0xfull << (4 * (m - 1)))) | ((unsigned long long)j << (4 * (m - 1)));
        mmax = max(mmax, m);
      }
      const int bstar = g_end % nb;
      const uint32_t k_lo = (uint32_t)R.K, k_hi = (uint32_t)(R.K >> 32);
      // nb K as a 96-bit step [stp_h : stp_m : stp_l]
      const unsigned long long p0 = (unsigned long long)(uint32_t)nb * k_lo;
      const unsigned long long p1 = (unsigned long long)(uint32_t)nb * k_hi + (p0 >> 32);
      const uint32_t stp_l = (uint32_t)p0, stp_m = (uint32_t)p1, stp_h = (uint32_t)(p1 >> 32);
      const int nblk = (nb + 31) >> 5;

      long long h0w = 0, h0y = 0;  // U of bins 0..31 (the wrap-around values)
      long long pw = 0, py = 0;    // U of the previous block
      float bs2 = -1.f, bd = 1.f, bsv = 0.f, brv = 0.f;
      int bo = 255, bk = -1;       // best box: width - 1 and start bin
      // block i: U of bins 32 i + lane; then the histogram of block i - 1 and the
      // sweep of block i - 2 (boxes of up to 15 bins starting in it)
      for (int i = 0; i <= nblk + 1; ++i) {
        const int x = (i << 5) + lane;
        long long uw = 0, uy = 0;
        if ((i << 5) < nb) {  // warp-uniform: lanes x < nb own bin x
          // edges G = G0, G0 + nb, ... <= g_end; the edge at t' = 0 (G = 0) is skipped:
          // no point lies before it, its prefix sum is exactly 0
          const int G0 = x == 0 ? nb : x;
          // X = G0 K in 96 bits [xh : xm : xl]
          const unsigned long long q0 = (unsigned long long)(uint32_t)G0 * k_lo;
          const unsigned long long q1 = (unsigned long long)(uint32_t)G0 * k_hi + (q0 >> 32);
          uint32_t xl = (uint32_t)q0, xm = (uint32_t)q1, xh = (uint32_t)(q1 >> 32);
          long long aw = 0, ay = 0;
          bool near = false;  // some edge of this lane lies within the guard band of its cell's point
          // all lanes take cnt edges; only in the last one may a lane be past g_end
          const int cnt = (g_end - (i << 5)) / nb + 1;
          auto edge = [&](bool valid) {
            const int u = min((int)__funnelshift_r(xm, xh, 24), nc);  // cell of tau_G
            const uint32_t fr = __funnelshift_r(xl, xm, 24);           // position in it, 2^-32
            const uint32_t dq = s_dt[u];
            near = near || (uint32_t)(dq - fr + band_q) <= 2u * band_q;
            const int v = u + (dq < fr ? 1 : 0);  // past the cell's point if it lies before tau_G
            const int2 lc = s_loc[v];
            const longlong2 bs = s_base[v >> 5];
            if (valid) {
              aw += bs.x + (long long)lc.x;
              ay += bs.y + (long long)lc.y;
            }
            asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
                : "+r"(xl), "+r"(xm), "+r"(xh)
                : "r"(stp_l), "r"(stp_m), "r"(stp_h));
          };
          int c = 0;
          for (; c + 2 < cnt; c += 2) {
            edge(true);
            edge(true);
          }
          if (c + 1 < cnt) edge(true);
          edge(G0 + (cnt - 1) * nb <= g_end);
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
              for (int g = G0; g <= g_end; g += nb) {
                const unsigned long long r0 = (unsigned long long)(uint32_t)g * k_lo;
                const unsigned long long r1 = (unsigned long long)(uint32_t)g * k_hi + (r0 >> 32);
                const int u = min((int)(r1 >> 24), nc);
                const uint32_t fr = ((uint32_t)r1 << 8) | ((uint32_t)r0 >> 24);
                const uint32_t dq = s_dt[u];
                int sel = dq < fr ? 1 : 0;
                if (dq != 0xffffffffu && (uint32_t)(dq - fr + band_q) <= 2u * band_q)
                  sel = exact_before(tp, gidx[u], f, nb, g);
                const int v = u + sel;
                aw += s_base[v >> 5].x + (long long)s_loc[v].x;
                ay += s_base[v >> 5].y + (long long)s_loc[v].y;
              }
            }
          }
          if (bstar < x) {
            aw += fx.w_tot;
            ay += fx.y_tot;
          }
          uw = aw;
          uy = ay;
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
          // histogram of block i - 1: H[x] = U[x + 1] - U[x], exact, then FP32
          long long nw = __shfl_down_sync(0xffffffffu, pw, 1);
          long long ny = __shfl_down_sync(0xffffffffu, py, 1);
          const long long fw = __shfl_sync(0xffffffffu, uw, 0);
          const long long fy = __shfl_sync(0xffffffffu, uy, 0);
          if (lane == 31) {
            nw = fw;
            ny = fy;
          }
          const float2 hv = make_float2(__fmul_rn(__ll2float_rn(nw - pw), scw), __fmul_rn(__ll2float_rn(ny - py), scy));
          ring[(((i - 1) & 1) << 5) + lane] = hv;
          if (!((i - 1) & 1)) ring[64 + lane] = hv;
        }
        pw = uw;
        py = uy;
        __syncwarp();
        if (i >= 2) {  // sweep block i - 2: running sums over its boxes' bins
          const int k = ((i - 2) << 5) + lane;
          const float2* rb = ring + (((i - 2) & 1) << 5) + lane;
          const bool kin = k < nb;
          float rw = 0.f, ry = 0.f;
#pragma unroll
          for (int o = 0; o < 15; ++o) {
            if (o < mmax) {
              const float2 hv = rb[o];
              rw = __fadd_rn(rw, hv.x);
              ry = __fadd_rn(ry, hv.y);
              if (((wmask >> o) & 1u) && kin && rw > 0.f && rw < 1.f) {
                const float dd = __fmul_rn(rw, __fsub_rn(1.f, rw));
                const float s2 = __fmul_rn(ry, ry);
                const float lhs = __fmul_rn(s2, bd), rhs = __fmul_rn(bs2, dd);
                // larger score, or equal with a narrower box (= lower j); this lane visits
                // k in increasing order and the widths increasing per k
                if (lhs > rhs || (lhs == rhs && o < bo)) {
                  bs2 = s2; bd = dd; bsv = ry; brv = rw; bo = o; bk = k;
                }
              }
            }
          }
        }
        __syncwarp();
      }
      int bj = bo < 16 ? (int)((jlow >> (4 * bo)) & 15ull) : 255;
      for (int off = 16; off > 0; off >>= 1) {
        const float o_s2 = __shfl_xor_sync(0xffffffffu, bs2, off);
        const float o_d = __shfl_xor_sync(0xffffffffu, bd, off);
        const float o_s = __shfl_xor_sync(0xffffffffu, bsv, off);
        const float o_r = __shfl_xor_sync(0xffffffffu, brv, off);
        const int o_j = __shfl_xor_sync(0xffffffffu, bj, off);
        const int o_k = __shfl_xor_sync(0xffffffffu, bk, off);
        if (beats(o_s2, o_d, o_j, o_k, bs2, bd, bj, bk)) {
          bs2 = o_s2; bd = o_d; bsv = o_s; brv = o_r; bj = o_j; bk = o_k;
        }
      }
      BoxBest bb;
      bb.s2 = bs2; bb.d = bd; bb.s = bsv; bb.r = brv; bb.j = bj; bb.k = bk;
      store_box(bb, lane, fidx, a.sr, a.qidx, a.kbin, a.sbest, a.rbest);
    }
  }
  if (!done && threadIdx.x == 0) atomicOr(a.err, kErrQueueBound);
}

uint32_t fixed_smem_bytes(int ncs) { return fixed_ring_off(ncs) + (uint32_t)kFixedWarps * kRing * 8u; }

int launch_cells_fixed(const FixedArgs& a, int blocks, size_t smem, void* stream) {
  auto kern = cells_fixed_kernel<kFixedWarps>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  kern<<<blocks, kFixedWarps * 32, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

int fixed_blocks_per_sm(size_t smem) {
  auto kern = cells_fixed_kernel<kFixedWarps>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kFixedWarps * 32, smem) != cudaSuccess) return 0;
  return nb;
}

}  // namespace qlp
