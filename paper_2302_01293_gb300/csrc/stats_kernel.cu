// Post-BLS statistics of each star's best candidate (Sec. 2.2 items 2-5 of
// arXiv:2302.01293), one CTA per star, FP64:
//  * trapezoid model y = z - delta s(a), a = distance from the nearest
//    mid-transit time (period fixed to the BLS period), s = 1 on the flat
//    bottom a <= D/2 - q_in D, linear to 0 at a = D/2, 0 outside (D = q P);
//  * fit of (T0, delta, q, q_in, z) by Levenberg-Marquardt on the points within
//    two BLS durations of the transit centre (weights dy^-2), bounds
//    1e-6 <= q <= 1, 1e-3 <= q_in <= 0.5, start from the BLS box (q_in = 0.1,
//    z = weighted mean of the window outside the box): solve
//    (A + lam diag(max(A_ii, 1e-12 max A_jj))) h = J^T r (A = J^T J) by Gaussian
//    elimination with partial pivoting, clip to the bounds, accept when chi^2
//    falls (lam / 10) else lam x 10; stop after an accepted step with a relative
//    decrease below 1e-10 or lam > 1e10 (converged), or after 100 iterations;
//  * residuals of the fitted model over all points: sigma_w = RMS; sigma_r from
//    the residuals averaged in time bins of one fitted duration,
//    sigma_r^2 = max(0, mean square of the bin averages - sigma_w^2 / mean points
//    per occupied bin);
//  * S/N_pink = delta (1 - q_in) / sqrt(sigma_w^2 / n_in + sigma_r^2 / N_t)
//    (Eq. 2 with the depth replaced by the trapezoid's mean depth), n_in points
//    with a < D/2, N_t transits with a point at a <= D/2; points before
//    (-2D <= dt < -D/2) and after (D/2 < dt <= 2D) transit;
//  * detected = N_t >= 2 and S/N_pink > 9 and S/N > 9.
// The model's region decisions use explicitly rounded FP64 operations (no
// contraction), in the order the definition states them; the quotients they
// round down (the nearest transit index, the residual time bin) come from a
// reciprocal and fall back to the exact division wherever the two could round
// differently. Point sums are taken per thread over contiguous index ranges and
// combined in a fixed order, so the results do not depend on scheduling.
//
// GB300 executes FP64 at 1/64 of the FP32 rate, so the cost of this kernel is its
// count of FP64 operations per point: the fit's pass over a flat-bottom or
// outside point takes eight (the point's phase, residual and five sums; the
// weight 1/dy^2 and the (z, z) curvature, the sum of all weights, are taken once),
// and region tests compare FP64 bit patterns on the integer pipe.
#include <cuda_runtime.h>

#include <cstdint>

#include "qlp_internal.h"

namespace qlp {

namespace {

constexpr int kThreads = 64;
constexpr int kWarps = kThreads / 32;
constexpr int kRampBuf = 64;  // queued ramp points per warp (a batch of 32 is taken at 32)
constexpr int kSums = 21;  // chi^2, g[5], A upper triangle [15]
constexpr double kQinMin = 1e-3, kQMin = 1e-6, kQinInit = 0.1;
constexpr double kLam0 = 1e-3, kRtol = 1e-10, kLamMax = 1e10;
constexpr int kMaxIt = 100;

// |v| of a double as its bit pattern: for non-negative doubles the order of the
// patterns (as integers) is the order of the values
__device__ __forceinline__ long long mag(double v) { return __double_as_longlong(v) & 0x7fffffffffffffffll; }

// floor(fl(fl(num / den) + add)), add = 0.5 (HALF) or 0, from rden = fl(1 / den).
// fl(num rden) lies within 3 2^-53 |num / den| of fl(num / den); below 2^20 in
// magnitude that is under 2^-31, and with the rounding of the sum the two floors
// agree unless the sum lies within 2^-30 of an integer. There, and for larger
// quotients, the quotient is taken exactly.
template <bool HALF>
__device__ __forceinline__ double floor_quot(double num, double den, double rden) {
  const double q = __dmul_rn(num, rden);
  const double b = HALF ? __dadd_rn(q, 0.5) : q;
  const double nn = floor(b);
  const double fr = __dsub_rn(b, nn);  // in [0, 1), accurate to 2^-53
  if (fr > 0x1p-30 && fr < 1.0 - 0x1p-30 && fabs(b) < 0x1p20) return nn;
  const double qe = __ddiv_rn(num, den);
  return floor(HALF ? __dadd_rn(qe, 0.5) : qe);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of n values per thread (n <= kSums) into tot[0 .. n-1] in shared
// memory (warp sums, then one thread per value adds the warps' partials in order).
__device__ __forceinline__ void block_sums(const double* v, int n, double (*red)[kSums], double* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < n; ++i) {
    const double w = warp_sum(v[i]);
    if (lane == 0) red[warp][i] = w;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[w][threadIdx.x];
    tot[threadIdx.x] = t;
  }
  __syncthreads();
}

__device__ __forceinline__ void clip(double* x) {
  x[2] = fmin(fmax(x[2], kQMin), 1.0);
  x[3] = fmin(fmax(x[3], kQinMin), 0.5);
}

__device__ __forceinline__ double shfl_d(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Gaussian elimination with partial pivoting of the 5 x 5 system m h = b by one warp;
// false if singular. Lane 6 r + j holds entry (r, j) of the augmented matrix [m | b]
// (lanes 30 and 31 repeat lanes 24 and 25). Every entry goes through the same
// operations in the same order as in the serial elimination (pivot: the first row of
// the largest |m[r][c]|; m[r][j] -= (m[r][c] / m[c][c]) m[c][j]), and the back
// substitution runs in that order on every lane, so h is the serial result. The
// warp issues each step once for all entries: on GB300 a single thread's FP64
// instruction takes the pipe as long as a full warp's.
__device__ bool solve5_warp(double v, int r, int j, double* h) {
  for (int c = 0; c < 5; ++c) {
    int p = c;
    double best = shfl_d(v, 6 * c + c);
    for (int rr = c + 1; rr < 5; ++rr) {
      const double o = shfl_d(v, 6 * rr + c);
      if (fabs(o) > fabs(best)) {
        best = o;
        p = rr;
      }
    }
    if (best == 0.0) return false;
    const double vc = shfl_d(v, 6 * c + j), vp = shfl_d(v, 6 * p + j);
    if (r == c) v = vp;
    else if (r == p) v = vc;
    const double piv = shfl_d(v, 6 * c + c);
    const double rc = shfl_d(v, 6 * r + c);
    const double cj = shfl_d(v, 6 * c + j);
    if (r > c && j >= c) v = __dsub_rn(v, __dmul_rn(__ddiv_rn(rc, piv), cj));
  }
  double u[5][6];
#pragma unroll
  for (int rr = 0; rr < 5; ++rr)
#pragma unroll
    for (int jj = rr; jj < 6; ++jj) u[rr][jj] = shfl_d(v, 6 * rr + jj);
#pragma unroll
  for (int c = 4; c >= 0; --c) {
    double acc = u[c][5];
#pragma unroll
    for (int jj = c + 1; jj < 5; ++jj) acc = __dsub_rn(acc, __dmul_rn(u[c][jj], h[jj]));
    h[c] = __ddiv_rn(acc, u[c][c]);
  }
  return true;
}

}  // namespace

// Launch order of the statistics CTAs: stars by decreasing estimated fit cost (its
// window holds about 4 q n points), so that the longest fits start first rather
// than trail the launch. Half-octave buckets of q n; the order inside a bucket is
// free (each star's results do not depend on it). One CTA.
constexpr int kOrderBuckets = 64;
__global__ void __launch_bounds__(1024) stats_order_kernel(const StatsArgs a) {
  __shared__ int cnt[kOrderBuckets], pos[kOrderBuckets];
  if (threadIdx.x < kOrderBuckets) cnt[threadIdx.x] = 0;
  __syncthreads();
  auto bucket = [&](int s) {
    const double key = a.best[s].f_idx >= 0 ? a.best[s].q * (double)a.stars[s].n_pts : 0.0;
    const int e = key > 1.0 ? min((int)(2.0 * log2(key)), kOrderBuckets - 1) : 0;
    return kOrderBuckets - 1 - e;  // the largest first
  };
  for (int s = threadIdx.x; s < a.n_stars; s += blockDim.x) atomicAdd(&cnt[bucket(s)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = 0; k < kOrderBuckets; ++k) {
      pos[k] = run;
      run += cnt[k];
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < a.n_stars; s += blockDim.x) a.order[atomicAdd(&pos[bucket(s)], 1)] = s;
}

__global__ void __launch_bounds__(kThreads, 6) stats_kernel(const StatsArgs a) {
  __shared__ double red[kWarps][kSums];
  __shared__ double s_part[kThreads][kSums + 1];  // per-thread sums of the fit's pass
  __shared__ double s_q[kThreads / 32][kSums];
  __shared__ int s_ramp[kWarps][kRampBuf];
  __shared__ double s_tot[kSums];  // block totals of the last reduction
  __shared__ double s_cur[kSums];  // chi^2, g, A at the accepted parameters (thread 0)
  __shared__ double s_x[5];
  __shared__ double s_lam;         // the damping (thread 0 updates it, warp 0 reads it)
  __shared__ double s_wsum;        // sum of the window points' weights 1/dy^2
  __shared__ int s_go;
  __shared__ int s_cnt[kThreads];
  // run partials for the binned residuals and the transit count (bins as the bit
  // patterns of their non-negative FP64 indices)
  __shared__ long long s_hbin[kThreads], s_tbin[kThreads], s_kf[kThreads], s_kl[kThreads];
  __shared__ double s_hsum[kThreads], s_tsum[kThreads];
  __shared__ int s_hcnt[kThreads], s_tcnt[kThreads], s_runs[kThreads], s_kd[kThreads];

  const int s = a.order ? a.order[blockIdx.x] : (int)blockIdx.x;
  const int tid = threadIdx.x;
  const StarDev st = a.stars[s];
  const qlp_bls_best bb = a.best[s];
  qlp_bls_cand_stats* out = a.out + s;
  const int n = st.n_pts;
  if (bb.f_idx < 0 || n <= 0) {
    if (tid == 0) {
      *out = qlp_bls_cand_stats{};
      out->status = QLP_STATS_NO_CANDIDATE;
    }
    return;
  }
  const double* tp = a.tp + st.pt_off;
  const double* yv = a.y + st.pt_off;
  const double* dyv = a.dy + st.pt_off;
  WinRec* wrec = a.wrec + st.pt_off;
  const double period = bb.period;
  const double r_period = 1.0 / period;
  const double t0p = __dsub_rn(bb.t0, st.t_ref);
  const double q0 = bb.q;
  const long long lim_b = mag(__dmul_rn(2.0, __dmul_rn(q0, period)));
  const long long half0_b = mag(__dmul_rn(0.5, __dmul_rn(q0, period)));
  const int seg = (n + kThreads - 1) / kThreads;
  const int i0 = min(n, tid * seg), i1 = min(n, i0 + seg);
  // |dt| of point i from the candidate's epoch (t', y, dy in time order; t' >= 0)
  auto dt0_of = [&](int i, double& pn) {
    const double u = __dsub_rn(tp[i], t0p);
    pn = __dmul_rn(period, floor_quot<true>(u, period, r_period));
    return mag(__dsub_rn(u, pn));
  };

  // 1. the fit window (ordered compaction) and the initial out-of-transit level
  int c = 0;
  double v[4];
  for (int i = 0; i < 4; ++i) v[i] = 0.0;
  for (int i = i0; i < i1; ++i) {
    double pn;
    const long long db = dt0_of(i, pn);
    if (db <= lim_b) {
      ++c;
      const double w = __ddiv_rn(1.0, __dmul_rn(dyv[i], dyv[i]));
      v[0] += w * yv[i];
      v[1] += w;
      if (db > half0_b) {
        v[2] += w * yv[i];
        v[3] += w;
      }
    }
  }
  s_cnt[tid] = c;
  block_sums(v, 4, red, s_tot);
  if (tid == 0) {  // exclusive scan of the per-thread counts
    int run = 0;
    for (int t = 0; t < kThreads; ++t) {
      const int x = s_cnt[t];
      s_cnt[t] = run;
      run += x;
    }
    s_go = run;
    s_x[0] = t0p;
    s_x[1] = bb.depth;
    s_x[2] = q0;
    s_x[3] = kQinInit;
    s_x[4] = s_tot[3] > 0.0 ? s_tot[2] / s_tot[3] : s_tot[0] / s_tot[1];
    clip(s_x);
  }
  __syncthreads();
  const int nwin = s_go;
  {
    int o = s_cnt[tid];
    double ws = 0.0;
    for (int i = i0; i < i1; ++i) {
      double pn;
      if (dt0_of(i, pn) <= lim_b) {
        const double inv = __ddiv_rn(1.0, dyv[i]);
        const double w = __dmul_rn(inv, inv);  // the (z, z) term of J^T J, as its product
        wrec[o++] = WinRec{tp[i], pn, yv[i], w};
        ws += w;
      }
    }
    block_sums(&ws, 1, red, &s_wsum);
  }
  if (nwin < 6) {
    if (tid == 0) {
      *out = qlp_bls_cand_stats{};
      out->status = QLP_STATS_FEW_POINTS;
      out->n_fit = nwin;
    }
    return;
  }
  __syncthreads();

  // 2. Levenberg-Marquardt (thread 0 keeps the state; every pass is block-wide)
  const int wseg = (nwin + kThreads - 1) / kThreads;
  const int w0 = min(nwin, tid * wseg), w1 = min(nwin, w0 + wseg);
  // The model at s_x and its derivatives. Only points on a ramp have nonzero
  // derivatives in T0, q and q_in; flat-bottom points add to the (delta, z) block
  // and outside points to z alone, in place. Ramp points are queued per warp and
  // taken 32 at a time by all lanes, so that the long ramp branch runs once per 32
  // ramp points instead of whenever one lane meets one; its divisions are
  // multiplications by reciprocals taken once per evaluation. The region
  // decisions keep the FP64 expressions of the model's definition.
  //
  // On a ramp every derivative is 1/dy times a factor: phi = (c0 sg, -s, r_q a,
  // r_qin s, 1) with sg = sign(dt), c0 = -delta / t_in, r_q = -delta / (q_in q^2 P)
  // and r_qin = delta / q_in, so J^T J and J^T r over the ramp points follow from
  // nine weighted sums of 1, sg, s, a and their products and three of r / dy times
  // sg, s, a; the factors c0, r_q, r_qin multiply the block totals once.
  enum { kChi, kG4, kWeF, kWF, kGsg, kGs, kGa, kRw, kRsg, kRsgs, kRsga, kRss, kRsa, kRs, kRaa, kRa, kAcc };
  const int lane = tid & 31, warp_id = tid >> 5;
  int* rl = s_ramp[warp_id];
  auto evaluate = [&]() {  // at s_x: chi^2, J^T r, J^T J into s_tot
    double acc[kAcc];
    double x[5];
    for (int i = 0; i < 5; ++i) x[i] = s_x[i];
    const double d = __dmul_rn(x[2], period);
    const double t_in = __dmul_rn(x[3], d);
    const double half = __dmul_rn(0.5, d);
    const double edge = __dsub_rn(half, t_in);
    const double hp = __dmul_rn(0.5, period);
    const double r_tin = 1.0 / t_in;
    const double m_flat = __dsub_rn(x[4], x[1]);  // the model on the flat bottom
    for (int i = 0; i < kAcc; ++i) acc[i] = 0.0;
    const long long hp_b = mag(hp), edge_b = mag(edge), half_b = mag(half);
    auto dt_of = [&](const WinRec& pt) {
      const double u = __dsub_rn(pt.t, x[0]);
      double dt = __dsub_rn(u, pt.pn);
      if (mag(dt) > hp_b) {  // the epoch moved by half a period: the nearest transit changed
        const double nn = floor(__dadd_rn(__ddiv_rn(u, period), 0.5));
        dt = __dsub_rn(u, __dmul_rn(period, nn));
      }
      return dt;
    };
    auto ramp_batch = [&](int cnt) {  // lanes < cnt take the queued ramp points rl[lane]
      if (lane < cnt) {
        const WinRec pt = wrec[rl[lane]];
        const double dt = dt_of(pt);
        const bool neg = __double_as_longlong(dt) < 0;  // sg = -1 (a ramp point has dt != 0)
        const double aa = fabs(dt);
        const double sv = __dmul_rn(__dsub_rn(half, aa), r_tin);
        const double e = __dsub_rn(pt.y, __dsub_rn(x[4], __dmul_rn(x[1], sv)));
        const double ir = pt.w * e;  // r / dy
        acc[kChi] += ir * e;
        acc[kG4] += ir;
        acc[kGsg] += neg ? -ir : ir;
        acc[kGs] += sv * ir;
        acc[kGa] += aa * ir;
        const double ws = pt.w * sv, wa = pt.w * aa;
        acc[kRw] += pt.w;
        acc[kRsg] += neg ? -pt.w : pt.w;
        acc[kRsgs] += neg ? -ws : ws;
        acc[kRsga] += neg ? -wa : wa;
        acc[kRss] += ws * sv;
        acc[kRsa] += ws * aa;
        acc[kRs] += ws;
        acc[kRaa] += wa * aa;
        acc[kRa] += wa;
      }
    };
    int nr = 0;  // queued ramp points of this warp (warp-uniform)
    for (int k = 0; k < wseg; ++k) {  // the same trip count on every lane
      const int wi = w0 + k;
      bool on_ramp = false;
      if (wi < w1) {
        const WinRec pt = wrec[wi];
        const long long ab = mag(dt_of(pt));
        on_ramp = ab > edge_b && ab < half_b;
        if (!on_ramp) {  // flat bottom (s = 1) or outside (s = 0): one path, no divergence
          const bool flat = ab <= edge_b;  // dm/ddelta = -s, dm/dz = 1
          const double e = __dsub_rn(pt.y, flat ? m_flat : x[4]);
          const double we = __dmul_rn(pt.w, e);  // r / dy with r = e / dy
          acc[kChi] += we * e;                   // r^2
          acc[kG4] += we;                        // g4 = sum r / dy
          acc[kWeF] += flat ? we : 0.0;          // -g1 over the flat bottom
          acc[kWF] += flat ? pt.w : 0.0;         // A11 and -A14 over the flat bottom
        }
      }
      const unsigned mk = __ballot_sync(0xffffffffu, on_ramp);
      if (on_ramp) rl[nr + __popc(mk & ((1u << lane) - 1u))] = wi;
      nr += __popc(mk);
      if (nr >= 32) {
        __syncwarp();
        ramp_batch(32);
        const int rest = nr - 32;
        const int moved = lane < rest ? rl[32 + lane] : 0;
        __syncwarp();
        if (lane < rest) rl[lane] = moved;
        __syncwarp();
        nr = rest;
      }
    }
    __syncwarp();
    if (nr > 0) ramp_batch(nr);
    __syncwarp();
    // block sums through shared memory: each thread of the first kAcc x 4 sums one
    // value over 32 threads; then every entry of chi^2, g and A adds the 4 quarters
    // of the sums it takes, in order, and applies the factors
    for (int i = 0; i < kAcc; ++i) s_part[tid][i] = acc[i];
    __syncthreads();
    if (tid < kAcc * (kThreads / 32)) {
      const int v = tid % kAcc, qq = tid / kAcc;
      double sum = 0.0;
      for (int r = 0; r < 32; ++r) sum += s_part[32 * qq + r][v];
      s_q[qq][v] = sum;
    }
    __syncthreads();
    if (tid < kSums) {
      auto T = [&](int v) {
        double sum = 0.0;
        for (int qq = 0; qq < kThreads / 32; ++qq) sum += s_q[qq][v];
        return sum;
      };
      const double c0 = -x[1] * r_tin;
      const double r_q = -x[1] / (x[3] * x[2] * x[2] * period);  // d(-delta s)/dq per unit a
      const double r_qin = x[1] / x[3];
      double v = 0.0;
      switch (tid) {
        case 0: v = T(kChi); break;
        case 1: v = c0 * T(kGsg); break;                 // g0
        case 2: v = -(T(kWeF) + T(kGs)); break;          // g1
        case 3: v = r_q * T(kGa); break;                 // g2
        case 4: v = r_qin * T(kGs); break;               // g3
        case 5: v = T(kG4); break;                       // g4
        case 6: v = c0 * c0 * T(kRw); break;             // A00
        case 7: v = -c0 * T(kRsgs); break;               // A01
        case 8: v = c0 * r_q * T(kRsga); break;          // A02
        case 9: v = c0 * r_qin * T(kRsgs); break;        // A03
        case 10: v = c0 * T(kRsg); break;                // A04
        case 11: v = T(kRss) + T(kWF); break;            // A11
        case 12: v = -r_q * T(kRsa); break;              // A12
        case 13: v = -r_qin * T(kRss); break;            // A13
        case 14: v = -(T(kRs) + T(kWF)); break;          // A14
        case 15: v = r_q * r_q * T(kRaa); break;         // A22
        case 16: v = r_q * r_qin * T(kRsa); break;       // A23
        case 17: v = r_q * T(kRa); break;                // A24
        case 18: v = r_qin * r_qin * T(kRss); break;     // A33
        case 19: v = r_qin * T(kRs); break;              // A34
        default: v = s_wsum; break;                      // A44: every window point's weight
      }
      s_tot[tid] = v;
    }
    __syncthreads();
  };
  double xa[5];
  evaluate();
  if (tid == 0) {
    for (int i = 0; i < kSums; ++i) s_cur[i] = s_tot[i];
    s_lam = kLam0;
  }
  for (int i = 0; i < 5; ++i) xa[i] = s_x[i];
  __syncthreads();  // warp 0 reads s_cur and s_lam
  int it = 0;
  bool conv = false;
  while (it < kMaxIt) {  // block-uniform: s_go decides
    ++it;
    if (tid < 32) {  // warp 0: the damped normal equations and their solution
      // entry (r, j) of [A + lam diag(max(A_kk, 1e-12 max A_jj)) | g] on lane 6 r + j;
      // A's upper triangle is stored row by row after chi^2 and g
      const int r = min(lane / 6, 4), j = lane % 6;
      const int k = min(r, j), l = max(r, j);
      double v = j == 5 ? s_cur[1 + r] : s_cur[6 + 5 * k - k * (k - 1) / 2 + (l - k)];
      double dmax = 0.0;
      for (int kk = 0; kk < 5; ++kk) dmax = fmax(dmax, s_cur[6 + 5 * kk - kk * (kk - 1) / 2]);
      if (r == j) v = __dadd_rn(v, __dmul_rn(s_lam, fmax(v, __dmul_rn(1e-12, dmax))));
      double h[5];
      const bool ok = solve5_warp(v, r, j, h);
      if (tid == 0) {
        if (ok) {
          for (int kk = 0; kk < 5; ++kk) s_x[kk] = __dadd_rn(xa[kk], h[kk]);
          clip(s_x);
        }
        s_go = ok ? 1 : 0;
      }
    }
    __syncthreads();
    const bool ok = s_go != 0;
    if (ok) evaluate();
    if (tid == 0) {
      int act = 0;  // 0 continue, 1 stop
      if (ok && s_tot[0] < s_cur[0]) {
        const double rel = s_cur[0] > 0.0 ? (s_cur[0] - s_tot[0]) / s_cur[0] : 0.0;
        for (int i = 0; i < kSums; ++i) s_cur[i] = s_tot[i];
        for (int i = 0; i < 5; ++i) xa[i] = s_x[i];
        s_lam /= 10.0;
        if (rel < kRtol) { conv = true; act = 1; }
      } else {
        s_lam *= 10.0;
        if (s_lam > kLamMax) { conv = true; act = 1; }
      }
      for (int i = 0; i < 5; ++i) s_x[i] = xa[i];
      s_go = act;
    }
    __syncthreads();
    if (s_go) break;
  }

  // 3. residuals over every point at the fitted parameters
  double x[5];
  for (int i = 0; i < 5; ++i) x[i] = s_x[i];
  const double D = __dmul_rn(x[2], period);
  const double r_D = 1.0 / D;
  const double hD = __dmul_rn(0.5, D), tD = __dmul_rn(2.0, D);
  const double t_in = __dmul_rn(x[3], D);
  const double edge = __dsub_rn(hD, t_in);
  const double m_flat = __dsub_rn(x[4], x[1]);
  const long long hD_b = mag(hD), tD_b = mag(tD), edge_b = mag(edge);
  double r2 = 0.0, sb2 = 0.0;
  int n_in = 0, n_before = 0, n_after = 0, runs = 0;
  long long cbin = -1, hbin = -1;
  double csum = 0.0, hsum = 0.0;
  int ccnt = 0, hcnt = 0;
  bool have_head = false;
  long long kf = 0, kl = 0;  // first and last transit index seen (valid when kd > 0)
  int kd = 0;
  for (int i = i0; i < i1; ++i) {
    // the model (Sec. 2.2 item 2) at t'_i: nearest transit, distance, trapezoid
    const double u = __dsub_rn(tp[i], x[0]);
    const double nn = floor_quot<true>(u, period, r_period);
    const double dt = __dsub_rn(u, __dmul_rn(period, nn));
    const long long ab = mag(dt);
    const bool neg = __double_as_longlong(dt) < 0;  // sign bit (ab > hD_b excludes -0)
    double m;
    if (ab <= edge_b) m = m_flat;
    else if (ab < hD_b) m = __dsub_rn(x[4], __dmul_rn(x[1], __ddiv_rn(__dsub_rn(hD, fabs(dt)), t_in)));
    else m = x[4];
    const double r = __dsub_rn(yv[i], m);
    r2 += r * r;
    n_in += ab < hD_b;
    n_before += neg && ab > hD_b && ab <= tD_b;
    n_after += !neg && ab > hD_b && ab <= tD_b;
    if (ab <= hD_b) {
      const long long k = (long long)nn;
      if (kd == 0 || kl != k) {  // indices do not decrease along t
        if (kd == 0) kf = k;
        kl = k;
        ++kd;
      }
    }
    // the residual's time bin floor(t' / D) (t' >= 0: the bit pattern orders and identifies it)
    const long long b = __double_as_longlong(floor_quot<false>(tp[i], D, r_D));
    if (ccnt > 0 && b != cbin) {  // close the current run
      if (!have_head) { have_head = true; hbin = cbin; hsum = csum; hcnt = ccnt; }
      else { const double mu = csum / ccnt; sb2 += mu * mu; ++runs; }
      ccnt = 0;
      csum = 0.0;
    }
    cbin = b;
    csum += r;
    ++ccnt;
  }
  s_hbin[tid] = have_head ? hbin : cbin;
  s_hsum[tid] = have_head ? hsum : csum;
  s_hcnt[tid] = have_head ? hcnt : ccnt;
  s_tbin[tid] = have_head ? cbin : -1;  // the last run when it differs from the head
  s_tsum[tid] = have_head ? csum : 0.0;
  s_tcnt[tid] = have_head ? ccnt : 0;
  s_runs[tid] = runs;
  s_kf[tid] = kf;
  s_kl[tid] = kl;
  s_kd[tid] = kd;
  const double part[2] = {r2, sb2};
  block_sums(part, 2, red, s_tot);
  int cnt3[3] = {n_in, n_before, n_after};
  for (int i = 0; i < 3; ++i) {
    double vv = (double)cnt3[i];
    vv = warp_sum(vv);
    if ((tid & 31) == 0) red[tid >> 5][2 + i] = vv;
  }
  __syncthreads();
  if (tid == 0) {
    double cn[3] = {0.0, 0.0, 0.0};
    for (int w = 0; w < kWarps; ++w)
      for (int i = 0; i < 3; ++i) cn[i] += red[w][2 + i];
    // merge the run partials in thread order
    double sbm = s_tot[1];
    long long nb_occ = 0;
    for (int t = 0; t < kThreads; ++t) nb_occ += s_runs[t];
    long long carry_bin = -1;
    double carry_sum = 0.0;
    int carry_cnt = 0;
    auto flush = [&]() {
      if (carry_cnt > 0) { const double mu = carry_sum / carry_cnt; sbm += mu * mu; ++nb_occ; }
      carry_cnt = 0;
      carry_sum = 0.0;
    };
    for (int t = 0; t < kThreads; ++t) {
      if (s_hcnt[t] == 0) continue;  // no points
      if (carry_cnt > 0 && s_hbin[t] == carry_bin) { carry_sum += s_hsum[t]; carry_cnt += s_hcnt[t]; }
      else { flush(); carry_bin = s_hbin[t]; carry_sum = s_hsum[t]; carry_cnt = s_hcnt[t]; }
      if (s_tcnt[t] > 0) { flush(); carry_bin = s_tbin[t]; carry_sum = s_tsum[t]; carry_cnt = s_tcnt[t]; }
    }
    flush();
    // transits: distinct indices over threads, adjacent duplicates removed
    int nt = 0;
    long long last = -1;
    bool have = false;
    for (int t = 0; t < kThreads; ++t) {
      if (s_kd[t] == 0) continue;
      nt += s_kd[t];
      if (have && s_kf[t] == last) --nt;
      last = s_kl[t];
      have = true;
    }
    const double sw = sqrt(s_tot[0] / n);
    const double nb_mean = (double)n / (double)nb_occ;
    const double sb2m = sbm / (double)nb_occ;
    const double sr = sqrt(fmax(0.0, sb2m - sw * sw / nb_mean));
    const int n_in_t = (int)cn[0];
    const double depth_mean = x[1] * (1.0 - x[3]);
    const double den = (n_in_t ? sw * sw / n_in_t : 0.0) + (nt ? sr * sr / nt : 0.0);
    qlp_bls_cand_stats o{};
    o.t0 = x[0] + st.t_ref;
    o.depth = x[1];
    o.q = x[2];
    o.q_in = x[3];
    o.z = x[4];
    o.chi2 = s_cur[0];
    o.sigma_w = sw;
    o.sigma_r = sr;
    o.depth_mean = depth_mean;
    o.snr_pink = (n_in_t && nt && den > 0.0) ? depth_mean / sqrt(den) : 0.0;
    o.n_fit = nwin;
    o.n_in = n_in_t;
    o.n_before = (int)cn[1];
    o.n_after = (int)cn[2];
    o.n_transits = nt;
    o.iterations = it;
    o.status = conv ? QLP_STATS_OK : QLP_STATS_NOT_CONVERGED;
    o.detected = (nt >= 2 && o.snr_pink > 9.0 && bb.snr > 9.0) ? 1 : 0;
    *out = o;
  }
}

int launch_stats(const StatsArgs& a, void* stream) {
  if (a.n_stars <= 0) return 0;
  if (a.order) stats_order_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(a);
  stats_kernel<<<a.n_stars, kThreads, 0, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace qlp
