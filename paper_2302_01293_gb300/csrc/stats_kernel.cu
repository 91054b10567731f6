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
// contraction), in the order the definition states them. Point sums are taken
// per thread over contiguous index ranges and combined in a fixed order, so the
// results do not depend on scheduling.
#include <cuda_runtime.h>

#include <cstdint>

#include "qlp_internal.h"

namespace qlp {

namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kRampBuf = 64;  // queued ramp points per warp (a batch of 32 is taken at 32)
constexpr int kSums = 21;  // chi^2, g[5], A upper triangle [15]
constexpr double kQinMin = 1e-3, kQMin = 1e-6, kQinInit = 0.1;
constexpr double kLam0 = 1e-3, kRtol = 1e-10, kLamMax = 1e10;
constexpr int kMaxIt = 100;

struct Model {
  double dt, a, s, m;
  long long k;
  bool ramp;
};

__device__ __forceinline__ Model model_at(double t, const double* x, double period) {
  Model o;
  const double u = __dsub_rn(t, x[0]);
  const double n = floor(__dadd_rn(__ddiv_rn(u, period), 0.5));
  o.k = (long long)n;
  o.dt = __dsub_rn(u, __dmul_rn(period, n));
  o.a = fabs(o.dt);
  const double d = __dmul_rn(x[2], period);
  const double t_in = __dmul_rn(x[3], d);
  const double half = __dmul_rn(0.5, d);
  const double edge = __dsub_rn(half, t_in);
  if (o.a <= edge) {
    o.s = 1.0;
    o.ramp = false;
  } else if (o.a < half) {
    o.s = __ddiv_rn(__dsub_rn(half, o.a), t_in);
    o.ramp = true;
  } else {
    o.s = 0.0;
    o.ramp = false;
  }
  o.m = __dsub_rn(x[4], __dmul_rn(x[1], o.s));
  return o;
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

// Gaussian elimination with partial pivoting of the 5 x 5 system m h = b; false if singular.
__device__ bool solve5(double (*m)[6], double* h) {
  for (int c = 0; c < 5; ++c) {
    int p = c;
    for (int r = c + 1; r < 5; ++r)
      if (fabs(m[r][c]) > fabs(m[p][c])) p = r;
    if (m[p][c] == 0.0) return false;
    if (p != c)
      for (int j = 0; j < 6; ++j) {
        const double t = m[c][j];
        m[c][j] = m[p][j];
        m[p][j] = t;
      }
    for (int r = c + 1; r < 5; ++r) {
      const double f = __ddiv_rn(m[r][c], m[c][c]);
      for (int j = c; j < 6; ++j) m[r][j] = __dsub_rn(m[r][j], __dmul_rn(f, m[c][j]));
    }
  }
  for (int c = 4; c >= 0; --c) {
    double acc = m[c][5];
    for (int j = c + 1; j < 5; ++j) acc = __dsub_rn(acc, __dmul_rn(m[c][j], h[j]));
    h[c] = __ddiv_rn(acc, m[c][c]);
  }
  return true;
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 3) stats_kernel(const StatsArgs a) {
  __shared__ double red[kWarps][kSums];
  __shared__ double s_part[kThreads][kSums + 1];  // per-thread normal-equation sums
  __shared__ double s_q[kThreads / 32][kSums];
  __shared__ int s_ramp[kWarps][kRampBuf];
  __shared__ double s_tot[kSums];  // block totals of the last reduction
  __shared__ double s_cur[kSums];  // chi^2, g, A at the accepted parameters (thread 0)
  __shared__ double s_m[5][6];     // the damped normal equations (thread 0)
  __shared__ double s_x[5];
  __shared__ int s_go;
  __shared__ int s_cnt[kThreads];
  // run partials for the binned residuals and the transit count
  __shared__ long long s_hbin[kThreads], s_tbin[kThreads], s_kf[kThreads], s_kl[kThreads];
  __shared__ double s_hsum[kThreads], s_tsum[kThreads];
  __shared__ int s_hcnt[kThreads], s_tcnt[kThreads], s_runs[kThreads], s_kd[kThreads];

  const int s = blockIdx.x;
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
  const double t0p = __dsub_rn(bb.t0, st.t_ref);
  const double q0 = bb.q;
  const double lim = __dmul_rn(2.0, __dmul_rn(q0, period));
  const double half0 = __dmul_rn(0.5, __dmul_rn(q0, period));
  const int seg = (n + kThreads - 1) / kThreads;
  const int i0 = min(n, tid * seg), i1 = min(n, i0 + seg);

  // 1. the fit window (ordered compaction) and the initial out-of-transit level
  int c = 0;
  double v[4];
  for (int i = 0; i < 4; ++i) v[i] = 0.0;
  for (int i = i0; i < i1; ++i) {
    const double u = __dsub_rn(tp[i], t0p);
    const double nn = floor(__dadd_rn(__ddiv_rn(u, period), 0.5));
    const double dt = fabs(__dsub_rn(u, __dmul_rn(period, nn)));
    if (dt <= lim) {
      ++c;
      const double w = __ddiv_rn(1.0, __dmul_rn(dyv[i], dyv[i]));
      v[0] += w * yv[i];
      v[1] += w;
      if (dt > half0) {
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
    for (int i = i0; i < i1; ++i) {
      const double u = __dsub_rn(tp[i], t0p);
      const double nn = floor(__dadd_rn(__ddiv_rn(u, period), 0.5));
      const double dt = fabs(__dsub_rn(u, __dmul_rn(period, nn)));
      if (dt <= lim) wrec[o++] = WinRec{tp[i], yv[i], __ddiv_rn(1.0, dyv[i]), __dmul_rn(period, nn)};
    }
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
  const int lane = tid & 31, warp_id = tid >> 5;
  int* rl = s_ramp[warp_id];
  auto evaluate = [&]() {  // at s_x: chi^2, J^T r, J^T J into s_tot
    double sums[kSums];
    double x[5];
    for (int i = 0; i < 5; ++i) x[i] = s_x[i];
    const double d = __dmul_rn(x[2], period);
    const double t_in = __dmul_rn(x[3], d);
    const double half = __dmul_rn(0.5, d);
    const double edge = __dsub_rn(half, t_in);
    const double hp = __dmul_rn(0.5, period);
    const double r_tin = 1.0 / t_in;
    const double m_flat = __dsub_rn(x[4], x[1]);  // the model on the flat bottom
    const double r_q = -x[1] / (x[3] * x[2] * x[2] * period);  // d(-delta s)/dq per unit a
    const double r_qin = x[1] / x[3];
    for (int i = 0; i < kSums; ++i) sums[i] = 0.0;
    // |v| of a double as its bit pattern: for non-negative doubles the order of the
    // patterns (as integers) is the order of the values, so the region tests below
    // take the integer pipe instead of the FP64 one
    auto mag = [](double v) { return __double_as_longlong(v) & 0x7fffffffffffffffll; };
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
        const double aa = fabs(dt);
        const double inv = pt.inv;
        const double sv = __dmul_rn(__dsub_rn(half, aa), r_tin);
        const double r = __dmul_rn(__dsub_rn(pt.y, __dsub_rn(x[4], __dmul_rn(x[1], sv))), inv);
        const double sg = dt > 0.0 ? 1.0 : (dt < 0.0 ? -1.0 : 0.0);
        double j[5];
        j[0] = -x[1] * sg * r_tin * inv;
        j[1] = -sv * inv;
        j[2] = r_q * aa * inv;
        j[3] = r_qin * sv * inv;
        j[4] = inv;
        sums[0] += r * r;
        for (int k = 0; k < 5; ++k) sums[1 + k] += j[k] * r;
        int p = 6;
        for (int k = 0; k < 5; ++k)
          for (int l = k; l < 5; ++l) sums[p++] += j[k] * j[l];
      }
    };
    int nr = 0;  // queued ramp points of this warp (warp-uniform)
    for (int k = 0; k < wseg; ++k) {  // the same trip count on every lane
      const int wi = w0 + k;
      bool on_ramp = false;
      if (wi < w1) {
        const WinRec pt = wrec[wi];  // t', y, 1/dy, P n of the starting epoch
        const long long ab = mag(dt_of(pt));
        const double inv = pt.inv;
        on_ramp = ab > edge_b && ab < half_b;
        if (!on_ramp) {  // flat bottom (s = 1) or outside (s = 0): one path, no divergence
          const bool flat = ab <= edge_b;  // dm/ddelta = -s, dm/dz = 1
          const double r = __dmul_rn(__dsub_rn(pt.y, flat ? m_flat : x[4]), inv);
          const double fs = flat ? 1.0 : 0.0;
          const double ir = inv * r, i2 = inv * inv;
          sums[0] += r * r;
          sums[2] -= fs * ir;
          sums[5] += ir;
          sums[6 + 5] += fs * i2;   // A11
          sums[6 + 8] -= fs * i2;   // A14
          sums[6 + 14] += i2;       // A44
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
    // block sums through shared memory: each thread of the first kSums x 4 sums one
    // value over 32 threads, then kSums threads add the 4 quarters in order
    for (int i = 0; i < kSums; ++i) s_part[tid][i] = sums[i];
    __syncthreads();
    if (tid < kSums * (kThreads / 32)) {
      const int v = tid % kSums, qq = tid / kSums;
      double acc = 0.0;
      for (int r = 0; r < 32; ++r) acc += s_part[32 * qq + r][v];
      s_q[qq][v] = acc;
    }
    __syncthreads();
    if (tid < kSums) {
      double acc = 0.0;
      for (int qq = 0; qq < kThreads / 32; ++qq) acc += s_q[qq][tid];
      s_tot[tid] = acc;
    }
    __syncthreads();
  };
  double xa[5];
  evaluate();
  if (tid == 0)
    for (int i = 0; i < kSums; ++i) s_cur[i] = s_tot[i];
  for (int i = 0; i < 5; ++i) xa[i] = s_x[i];
  double lam = kLam0;
  int it = 0;
  bool conv = false;
  while (it < kMaxIt) {  // block-uniform: s_go decides
    ++it;
    if (tid == 0) {
      int p = 6;
      for (int k = 0; k < 5; ++k)
        for (int l = k; l < 5; ++l) s_m[k][l] = s_m[l][k] = s_cur[p++];
      double dmax = 0.0;
      for (int k = 0; k < 5; ++k) dmax = fmax(dmax, s_m[k][k]);
      for (int k = 0; k < 5; ++k) {
        s_m[k][k] = __dadd_rn(s_m[k][k], __dmul_rn(lam, fmax(s_m[k][k], __dmul_rn(1e-12, dmax))));
        s_m[k][5] = s_cur[1 + k];
      }
      double h[5];
      const bool ok = solve5(s_m, h);
      if (ok) {
        for (int k = 0; k < 5; ++k) s_x[k] = __dadd_rn(xa[k], h[k]);
        clip(s_x);
      }
      s_go = ok ? 1 : 0;
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
        lam /= 10.0;
        if (rel < kRtol) { conv = true; act = 1; }
      } else {
        lam *= 10.0;
        if (lam > kLamMax) { conv = true; act = 1; }
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
  const double hD = __dmul_rn(0.5, D), tD = __dmul_rn(2.0, D);
  double r2 = 0.0, sb2 = 0.0;
  int n_in = 0, n_before = 0, n_after = 0, runs = 0;
  long long cbin = -1, hbin = -1;
  double csum = 0.0, hsum = 0.0;
  int ccnt = 0, hcnt = 0;
  bool have_head = false;
  long long kf = 0, kl = 0;  // first and last transit index seen (valid when kd > 0)
  int kd = 0;
  for (int i = i0; i < i1; ++i) {
    const Model md = model_at(tp[i], x, period);
    const double r = __dsub_rn(yv[i], md.m);
    r2 += r * r;
    n_in += md.a < hD;
    n_before += (md.dt >= -tD) && (md.dt < -hD);
    n_after += (md.dt > hD) && (md.dt <= tD);
    if (md.a <= hD && (kd == 0 || kl != md.k)) {  // indices do not decrease along t
      if (kd == 0) kf = md.k;
      kl = md.k;
      ++kd;
    }
    const long long b = (long long)floor(__ddiv_rn(tp[i], D));
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
  stats_kernel<<<a.n_stars, kThreads, 0, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace qlp
