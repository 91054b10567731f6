// Device helpers shared by the search kernels (per-point and cell paths).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "qlp_internal.h"

namespace qlp {

// FP64 fold exactly as the plain definition: x = t' f, b = min(nb-1, floor(frac(x) nb)).
__device__ __forceinline__ int fold_fp64(double t, double f, int nb, int* cyc) {
  const double x = __dmul_rn(t, f);
  const double c = floor(x);
  const double ph = __dsub_rn(x, c);
  int b = (int)floor(__dmul_rn(ph, (double)nb));
  if (b > nb - 1) b = nb - 1;
  *cyc = (int)c;
  return b;
}

// Out-of-line so that the rare re-fold is a real branch, never predicated into the loop.
static __device__ __noinline__ int exact_global_bin(const double* tptr, double f, int nb) {
  int c;
  const int b = fold_fp64(*tptr, f, nb, &c);
  return c * nb + b;
}

// Cell path: cell of a point: u = floor(t'/h) adjusted so that t' - u h (in FP64) is in [0, h).
__device__ __forceinline__ int cell_of(double t, double h) {
  double q = floor(__ddiv_rn(t, h));
  const double r = __dsub_rn(t, __dmul_rn(q, h));
  if (r < 0.0) q -= 1.0;
  else if (r >= h) q += 1.0;
  return (int)q;
}

// Exact "point of cell u lies before edge G" from the FP64 fold of that point.
static __device__ __noinline__ int exact_before(const double* tp, int i, double f, int nb, int G) {
  int c;
  const int b = fold_fp64(tp[i], f, nb, &c);
  return (c * nb + b) < G ? 1 : 0;
}

constexpr int kU = 4;
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: adding it rounds |x| < 2^22 to an integer
constexpr int kMagicBits = 0x4B400000;

// Shared-memory float reductions issued under a predicate (no branch): a lane
// whose run did not end this step takes no part.
__device__ __forceinline__ void red_add_if(float* addr, float v, bool p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(addr);
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q red.shared.add.f32 [%0], %1;\n\t}"
               :: "r"(a), "f"(v), "r"((int)p) : "memory");
}
__device__ __forceinline__ float atom_add_if(float* addr, float v, bool p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(addr);
  float old = 0.f;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q atom.shared.add.f32 %0, [%1], %2;\n\t}"
               : "+f"(old) : "r"(a), "f"(v), "r"((int)p) : "memory");
  return old;
}

// Exact rounding error of a + b (TwoSum, Knuth).
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float bb = __fsub_rn(s, a);
  return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int SUM>
struct RunAcc {
  float aw, ay, cw, cy;
  __device__ __forceinline__ void reset() { aw = ay = cw = cy = 0.f; }
  // start a new run with (w, wd) when `fresh`, else add them to the current run
  __device__ __forceinline__ void add(bool fresh, float w, float wd) {
    const float bw = fresh ? 0.f : aw, by = fresh ? 0.f : ay;
    const float sw = __fadd_rn(bw, w), sy = __fadd_rn(by, wd);
    if (SUM == QLP_SUM_COMP) {
      cw = __fadd_rn(fresh ? 0.f : cw, two_sum_err(bw, w, sw));
      cy = __fadd_rn(fresh ? 0.f : cy, two_sum_err(by, wd, sy));
    }
    aw = sw;
    ay = sy;
  }
};

// Add a finished run to bin b of the warp's histogram (when p); in COMP mode the
// rounding error of each shared add, recovered from the value it replaced, goes to
// the compensation arrays together with the run's own error terms.
template <int SUM>
__device__ __forceinline__ void flush_run(float* hw, float* hy, float* hwc, float* hyc, int b,
                                          const RunAcc<SUM>& acc, bool p) {
  if (SUM == QLP_SUM_COMP) {
    const float ow = atom_add_if(hw + b, acc.aw, p);
    const float oy = atom_add_if(hy + b, acc.ay, p);
    const float ew = two_sum_err(ow, acc.aw, __fadd_rn(ow, acc.aw));
    const float ey = two_sum_err(oy, acc.ay, __fadd_rn(oy, acc.ay));
    red_add_if(hwc + b, __fadd_rn(ew, acc.cw), p);
    red_add_if(hyc + b, __fadd_rn(ey, acc.cy), p);
  } else {
    red_add_if(hw + b, acc.aw, p);
    red_add_if(hy + b, acc.ay, p);
  }
}

// Double-float numbers (hi + lo, |lo| <= ulp(hi) / 2) on the FP32 pipes: the
// error-free sum and product (Knuth's TwoSum, Dekker's product through one FMA)
// and the pair arithmetic built on them carry about 44 bits, so that a value
// computed from exact sums rounds to FP32 within half an ulp and a hair, without
// the FP64 units (1/64 of the FP32 rate here).
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact: p + e = a.hi b.hi
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// x / y rounded to FP32: the quotient of the leading parts, corrected once by the
// remainder x - q y (the product q y.hi split exactly by one FMA).
__device__ __forceinline__ float df_div_to_float(DF x, DF y) {
  const float q = __fdiv_rn(x.hi, y.hi);
  const float p = __fmul_rn(q, y.hi);
  const float pe = __fmaf_rn(q, y.hi, -p);
  const float rem = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo), __fmul_rn(q, y.lo));
  return __fadd_rn(q, __fdiv_rn(rem, y.hi));
}

// x / y as a double-float number: the same quotient and one correction, kept as the
// pair's low part.
__device__ __forceinline__ DF df_div(DF x, DF y) {
  const float q = __fdiv_rn(x.hi, y.hi);
  const float p = __fmul_rn(q, y.hi);
  const float pe = __fmaf_rn(q, y.hi, -p);
  const float rem = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo), __fmul_rn(q, y.lo));
  return df_fast_two_sum(q, __fdiv_rn(rem, y.hi));
}

// An integer of magnitude below 2^48 as an exact pair, times 2^-k (k in [-100, 100]).
__device__ __forceinline__ DF df_from_ll_scaled(long long v, int k) {
  const float hi = __ll2float_rn(v);
  const float lo = __ll2float_rn(v - (long long)hi);  // |v - hi| < 2^24: exact
  const float sc = __int_as_float((127 - (k >> 1)) << 23), sc2 = __int_as_float((127 - (k - (k >> 1))) << 23);
  return DF{__fmul_rn(__fmul_rn(hi, sc), sc2), __fmul_rn(__fmul_rn(lo, sc), sc2)};
}

// A frequency's best box: the FP32 score terms the sweep compared, and, on lane 0,
// s, r and 1 - r of that box again as double-float numbers (from the exact integer
// sums, or from the histogram's bins with their compensation terms); xv = false
// when they were not taken.
struct BoxBest {
  float s2, d, s, r;
  int j, k;
  DF xs, xr, xq;
  bool xv;
};

// s, r and 1 - r of the box [k, k + m) summed as double-float numbers over a
// histogram's bins (wrap-padded, so k + m - 1 < nb + kMPad), compensation terms
// included.
template <typename F>
__device__ __forceinline__ void box_sums_df(F bin, int k, int m, BoxBest& b) {
  DF sw{0.f, 0.f}, sy{0.f, 0.f};
  for (int o = 0; o < m; ++o) {
    const float4 v = bin(k + o);  // (w, w-compensation, w d, w d-compensation)
    sw = df_add(sw, df_two_sum(v.x, v.y));
    sy = df_add(sy, df_two_sum(v.z, v.w));
  }
  b.xs = sy;
  b.xr = sw;
  b.xq = df_add(DF{1.f, 0.f}, DF{-sw.hi, -sw.lo});
  b.xv = true;
}

// Lane 0 stores a frequency's best box: j, k, and SR = s^2 / (r (1 - r)), s, r of
// that box from its FP64 sums, each rounded once to FP32 (the FP32 sweep's own
// values when the FP64 sums are absent or give no positive r (1 - r)); SR 0, j 255,
// k 0xFFFFFFFF when no window was valid.
__device__ __forceinline__ void store_box(const BoxBest& b, int lane, int64_t fidx, float* sr, uint8_t* qidx,
                                          uint32_t* kbin, float* sbest, float* rbest) {
  if (lane != 0) return;
  const bool none = b.s2 < 0.f;
  float v = none ? 0.f : __fdiv_rn(b.s2, b.d), sv = b.s, rv = b.r;
  if (!none && b.xv && b.xr.hi > 0.f && b.xq.hi > 0.f) {  // 0 < r < 1
    v = df_div_to_float(df_mul(b.xs, b.xs), df_mul(b.xr, b.xq));
    sv = __fadd_rn(b.xs.hi, b.xs.lo);
    rv = __fadd_rn(b.xr.hi, b.xr.lo);
  }
  sr[fidx] = v;
  if (qidx) qidx[fidx] = none ? (uint8_t)255 : (uint8_t)b.j;
  if (kbin) kbin[fidx] = none ? 0xffffffffu : (uint32_t)b.k;
  if (sbest) sbest[fidx] = none ? 0.f : sv;
  if (rbest) rbest[fidx] = none ? 0.f : rv;
}

// Strict "a beats b": larger s^2/d, then lower j, then lower k; s2 < 0 = no box.
__device__ __forceinline__ bool beats(float s2a, float da, int ja, int ka, float s2b, float db,
                                      int jb, int kb) {
  if (s2a < 0.f) return false;
  if (s2b < 0.f) return true;
  const float lhs = s2a * db, rhs = s2b * da;
  if (lhs != rhs) return lhs > rhs;
  if (ja != jb) return ja < jb;
  return ka < kb;
}

// Box sweep over one frequency's histogram (wrap-padded by kMPad bins) and the
// warp argmax: every cyclic window of m_j bins (widths from mtab), score
// s^2 / (r (1 - r)) for 0 < r < 1; ties to the lower j, then the lower start bin.
// Lane 0 stores SR, j, k, s, r (SR = 0, j = 255, k = 0xFFFFFFFF when no window
// is valid).
template <int SUM>
__device__ __forceinline__ void sweep_store(float* hw, float* hy, float* hwc, float* hyc,
                                            const int* mtab, int nq, int nb, int lane,
                                            int64_t fidx, float* sr, uint8_t* qidx,
                                            uint32_t* kbin, float* sbest, float* rbest) {
  // wrap padding: window k .. k+m-1 reads bins k+o mod nb
  for (int i = lane; i < kMPad; i += 32) {
    const int src = i % nb;
    hw[nb + i] = hw[src];
    hy[nb + i] = hy[src];
    if (SUM == QLP_SUM_COMP) { hwc[nb + i] = hwc[src]; hyc[nb + i] = hyc[src]; }
  }
  __syncwarp();

  // widths present (bit o: some duration covers o+1 bins) and, per width, the
  // lowest duration index j with it (4 bits each)
  uint32_t wmask = 0u;
  unsigned long long jlow = 0ull;
  for (int j = nq - 1; j >= 0; --j) {
    const int o = mtab[j] - 1;
    wmask |= 1u << o;
    jlow = (jlow & ~(0xfull << (4 * o))) | ((unsigned long long)j << (4 * o));
  }
  const int mmax = mtab[nq - 1];
  float bs2 = -1.f, bd = 1.f, bsv = 0.f, brv = 0.f;
  int bj = 255, bk = -1;
  for (int k = lane; k < nb; k += 32) {
    float rw = 0.f, ry = 0.f, rwc = 0.f, ryc = 0.f;
    for (int o = 0; o < mmax; ++o) {
      rw = __fadd_rn(rw, hw[k + o]);
      ry = __fadd_rn(ry, hy[k + o]);
      if (SUM == QLP_SUM_COMP) {
        rwc = __fadd_rn(rwc, hwc[k + o]);
        ryc = __fadd_rn(ryc, hyc[k + o]);
      }
      if ((wmask >> o) & 1u) {
        const int j = (int)((jlow >> (4 * o)) & 0xfull);
        const float r = (SUM == QLP_SUM_COMP) ? __fadd_rn(rw, rwc) : rw;
        const float sv = (SUM == QLP_SUM_COMP) ? __fadd_rn(ry, ryc) : ry;
        if (r > 0.f && r < 1.f) {
          const float d = __fmul_rn(r, __fsub_rn(1.f, r));
          const float s2 = __fmul_rn(sv, sv);
          if (beats(s2, d, j, k, bs2, bd, bj, bk)) {
            bs2 = s2; bd = d; bsv = sv; brv = r; bj = j; bk = k;
          }
        }
      }
    }
  }
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
  BoxBest b;
  b.s2 = bs2; b.d = bd; b.s = bsv; b.r = brv; b.j = bj; b.k = bk;
  b.xv = false;
  if (lane == 0 && bk >= 0)
    box_sums_df([&](int i) {
      return make_float4(hw[i], SUM == QLP_SUM_COMP ? hwc[i] : 0.f, hy[i], SUM == QLP_SUM_COMP ? hyc[i] : 0.f);
    }, bk, mtab[bj], b);
  store_box(b, lane, fidx, sr, qidx, kbin, sbest, rbest);
}

// Histogram of the cell path: one record per bin, (w, w-compensation, w d,
// w d-compensation) as float4 in COMP mode, (w, w d) as float2 in PLAIN mode, so
// that a bin's update and the sweep's read are one 16- or 8-byte access.
template <int SUM>
struct PackedBin {
  using T = float2;
  __device__ static float w(const T& v) { return v.x; }
  __device__ static float y(const T& v) { return v.y; }
  __device__ static float wc(const T&) { return 0.f; }
  __device__ static float yc(const T&) { return 0.f; }
};
template <>
struct PackedBin<QLP_SUM_COMP> {
  using T = float4;
  __device__ static float w(const T& v) { return v.x; }
  __device__ static float y(const T& v) { return v.z; }
  __device__ static float wc(const T& v) { return v.y; }
  __device__ static float yc(const T& v) { return v.w; }
};

// The box sweep over a packed histogram: the same window sums, in the same
// order, as sweep_store over separate arrays (bit-identical results); every lane
// returns the warp's best box.
template <int SUM>
__device__ __forceinline__ BoxBest sweep_best_packed(typename PackedBin<SUM>::T* h, const int* mtab, int nq, int nb,
                                                     int lane) {
  using PB = PackedBin<SUM>;
  for (int i = lane; i < kMPad; i += 32) h[nb + i] = h[i % nb];
  __syncwarp();
  uint32_t wmask = 0u;
  unsigned long long jlow = 0ull;
  for (int j = nq - 1; j >= 0; --j) {
    const int o = mtab[j] - 1;
    wmask |= 1u << o;
    jlow = (jlow & ~(0xfull << (4 * o))) | ((unsigned long long)j << (4 * o));
  }
  const int mmax = mtab[nq - 1];
  float bs2 = -1.f, bd = 1.f, bsv = 0.f, brv = 0.f;
  int bj = 255, bk = -1;
  for (int k = lane; k < nb; k += 32) {
    float rw = 0.f, ry = 0.f, rwc = 0.f, ryc = 0.f;
    for (int o = 0; o < mmax; ++o) {
      const typename PB::T v = h[k + o];
      rw = __fadd_rn(rw, PB::w(v));
      ry = __fadd_rn(ry, PB::y(v));
      if (SUM == QLP_SUM_COMP) {
        rwc = __fadd_rn(rwc, PB::wc(v));
        ryc = __fadd_rn(ryc, PB::yc(v));
      }
      if ((wmask >> o) & 1u) {
        const int j = (int)((jlow >> (4 * o)) & 0xfull);
        const float r = (SUM == QLP_SUM_COMP) ? __fadd_rn(rw, rwc) : rw;
        const float sv = (SUM == QLP_SUM_COMP) ? __fadd_rn(ry, ryc) : ry;
        if (r > 0.f && r < 1.f) {
          const float d = __fmul_rn(r, __fsub_rn(1.f, r));
          const float s2 = __fmul_rn(sv, sv);
          if (beats(s2, d, j, k, bs2, bd, bj, bk)) {
            bs2 = s2; bd = d; bsv = sv; brv = r; bj = j; bk = k;
          }
        }
      }
    }
  }
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
  BoxBest o;
  o.s2 = bs2; o.d = bd; o.s = bsv; o.r = brv; o.j = bj; o.k = bk;
  o.xv = false;
  if (lane == 0 && bk >= 0)
    box_sums_df([&](int i) {
      const typename PB::T v = h[i];
      return make_float4(PB::w(v), PB::wc(v), PB::y(v), PB::yc(v));
    }, bk, mtab[bj], o);
  return o;
}


}  // namespace qlp
