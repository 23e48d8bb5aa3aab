// Tile body and final stage of the DBaS-Log-MPPI step; shared by the plain
// one-launch-per-controller kernel and the batched persistent kernel.
#pragma once

#include "mppi_device.cuh"

namespace dbm {

constexpr int kTmaPolls = 1 << 22;
constexpr long long kTmaWaitCycles = 4000000000ll;  // about 2 s at 2 GHz

// Obstacle staging: 1 = bulk TMA copy into shared memory (mbarrier
// completion), 0 = coalesced loads by all threads.
#ifndef DBM_STAGE_TMA
#define DBM_STAGE_TMA 1
#endif


// Savitzky-Golay weights (Algorithm 1's SGF) for a window of W steps and
// polynomials of degree p: w[q W + i] is the weight of window sample i in
// the least-squares fit's value at window position q.  The fit is the
// orthogonal projection onto the polynomials of degree <= p, so
//   w[q W + i] = sum_{k<=p} G_k(x_q) G_k(x_i) / h_k,
// with G_k the monic discrete orthogonal (Gram) polynomials on the centred
// abscissae x = -(W-1)/2 .. (W-1)/2, built by their three-term recurrence
// G_{k+1}(x) = x G_k(x) - b_k G_{k-1}(x), b_k = k^2 (W^2 - k^2) / (4 (4k^2 - 1)),
// and h_k = sum_x G_k(x)^2 = b_k h_{k-1}, h_0 = W (the discrete Chebyshev
// polynomials; e.g. Gorry, Anal. Chem. 62 (1990)).  FP64, one entry per
// thread; p < W.
__device__ inline void sgf_weights(float* w, int W, int p, int tid, int nthreads) {
  const double c = 0.5 * (W - 1), WW = (double)W * W;
  for (int e = tid; e < W * W; e += nthreads) {
    const int q = e / W, i = e - q * W;
    const double xq = q - c, xi = i - c;
    double gq0 = 1.0, gi0 = 1.0, gq1 = xq, gi1 = xi;  // G_0, G_1
    double h = W;
    double acc = 1.0 / h;
    if (p >= 1) {
      h *= (WW - 1.0) / 12.0;
      acc += gq1 * gi1 / h;
    }
    for (int k = 1; k < p; ++k) {
      const double b = (double)k * k * (WW - (double)k * k) / (4.0 * (4.0 * k * k - 1.0));
      const double gq2 = xq * gq1 - b * gq0, gi2 = xi * gi1 - b * gi0;
      const int k1 = k + 1;
      h *= (double)k1 * k1 * (WW - (double)k1 * k1) / (4.0 * (4.0 * k1 * k1 - 1.0));
      acc += gq2 * gi2 / h;
      gq0 = gq1; gq1 = gq2;
      gi0 = gi1; gi1 = gi2;
    }
    w[e] = (float)acc;
  }
}

// Constants of the controller that never change: the unrolled DBaS weights
// c_s (scaled by R_B) and their sums, and the smoothing weights.  One CTA, at
// creation (and on every call of the allocation-free entry point).
__device__ inline void init_constants(const CtrlDesc& D, int tid, int nthreads) {
  const int T = D.T;
  const double g = D.gamma_bas;
  for (int t = tid; t < T; t += nthreads) {
    // step t produces x_{t+1}: c_{t+1} = (1 - g^(T - t)) / (1 - g)
    double c = (1.0 - pow(g, (double)(T - t))) / (1.0 - g);
    D.cw[t] = (float)(D.R_B_d * c);
  }
  if (tid == 0) {
    double gT = pow(g, (double)T);
    D.st->g1 = g * (1.0 - gT) / (1.0 - g);
    D.st->csum = (T - D.st->g1) / (1.0 - g);
  }
  if (D.sgf_wp)
    sgf_weights(D.cw + sgf_table_offset(T), D.sgf_wp & 0xff, D.sgf_wp >> 8, tid, nthreads);
}

// Per-step constants that depend only on the controller state (U, S_e), for
// a state the host has set: chol(S_e Sigma) = sqrt(S_e) chol(Sigma), u_t in
// FP32, a'_t = gamma Sigma^-1 u_t (the step divides it by S_e: a_t = gamma
// (S_e Sigma)^-1 u_t) and C0 = sum_t u_t . a_t, the part of the control cost
// of Eq. 9 (Algorithm 1 form gamma u^T (S_e Sigma)^-1 v) that every sample
// shares.  The final stage forms the same constants after each shift.
// Usrc: the sequence; Se_src: S_e, read after the first barrier; red: >= 32
// doubles of shared memory.
__device__ inline void prep_constants(const CtrlDesc& D, const double* Usrc, const double* Se_src,
                                      double* red, int tid, int nthreads) {
  DevState* st = D.st;
  const int T = D.T;
  __syncthreads();
  const float Se = (float)*Se_src;
  const float inv_Se = 1.0f / Se;
  if (tid == 0) {
    const float r = sqrtf(Se);
    st->L00 = r * (float)D.Lsig[0];
    st->L10 = r * (float)D.Lsig[1];
    st->L11 = r * (float)D.Lsig[2];
  }
  const float M00 = (float)D.Sinv[0], M01 = (float)D.Sinv[1];
  const float M10 = (float)D.Sinv[2], M11 = (float)D.Sinv[3];
  FF c0 = {0.0f, 0.0f};
  for (int t = tid; t < T; t += nthreads) {
    const float u0 = (float)Usrc[2 * t], u1 = (float)Usrc[2 * t + 1];
    const float a0 = fmaf(M00, u0, M01 * u1), a1 = fmaf(M10, u0, M11 * u1);
    D.cU[t] = make_float2(u0, u1);
    D.cA[t] = make_float2(a0, a1);
    ff_add_prod(c0, u0, a0, 0.0f);
    ff_add_prod(c0, u1, a1, 0.0f);
  }
  c0 = warp_sum_ff(c0);
  float* redf = reinterpret_cast<float*>(red);
  if ((tid & 31) == 0) {
    redf[2 * (tid >> 5)] = c0.hi;
    redf[2 * (tid >> 5) + 1] = c0.lo;
  }
  __syncthreads();
  if (tid < 32) {
    FF sum = tid < (nthreads >> 5) ? FF{redf[2 * tid], redf[2 * tid + 1]} : FF{0.0f, 0.0f};
    sum = warp_sum_ff(sum);
    if (tid == 0) st->C0 = (double)((sum.hi + sum.lo) * inv_Se);
  }
  __syncthreads();
}

// One trajectory of T explicit-Euler steps (Eq. 1, 12, 14) under the
// controls V[t * vs], from the initial state x_init (position rebased to the
// origin), evaluated by the 32 lanes of one warp: lanes take steps
// t = t0 + lane in segments of 32, and every state component is a prefix sum
// over steps of increments that depend only on components earlier in the
// chain
//   unicycle:          theta -> (cos, sin) -> (x, y)
//   quadrotor (6):     phidot -> phi -> (cos, sin) -> (ydot, zdot) -> (y, z)
//   Ackermann:         v -> theta -> (cos, sin) -> (x, y)
//   quadrotor (5):     theta -> (cos, sin) -> (vx, vz) -> (x, z)
// so each segment is a few warp scans, carried from segment to segment.  The
// pose after step t is written to pose[t * ps] as (x, y, cos, sin) of the
// heading.  With COST the lane also adds to `cost` its steps' stage cost
// q(x_{t+1}) and control cost a_t . (v_t - u_t) of Eq. 9 (Algorithm 1 form,
// the sample-independent part u_t . a_t excluded), and phi(x_T): summed in
// FP32 over the lane's ceil(T / 32) steps, then added to the float pair once.
template <int MODEL, bool COST>
__device__ void scan_trajectory(const CtrlDesc& D, int T, const float2* V, int vs,
                                const float* __restrict__ x_init, float4* pose, int ps,
                                const float2* __restrict__ Uf, const float2* __restrict__ Af,
                                const float* __restrict__ xrf, FF& cost, int lane,
                                float* x1 = nullptr) {
  const float dt = D.dt;
  if constexpr (MODEL == 0) {
    float cth = x_init[2], cx = x_init[0], cy = x_init[1];
    float cs_, cc_;
    sincosf(cth, &cs_, &cc_);
    float lc = 0.0f;  // this lane's few stage terms, in FP32
    for (int t0 = 0; t0 < T; t0 += 32) {
      const int t = t0 + lane;
      const bool valid = t < T;
      const float2 v = valid ? V[t * vs] : make_float2(0.0f, 0.0f);
      const float th_a = cth + warp_incl_scan(v.y * dt, lane);
      float sa, ca;
      sincosf(th_a, &sa, &ca);
      const float cb = from_prev_lane(ca, cc_, lane), sb = from_prev_lane(sa, cs_, lane);
      const float vdt = v.x * dt;
      const float xa = cx + warp_incl_scan(vdt * cb, lane);
      const float ya = cy + warp_incl_scan(vdt * sb, lane);
      if (x1 && t == 0) {
        x1[0] = xa;
        x1[1] = ya;
        x1[2] = th_a;
      }
      if (valid) {
        pose[t * ps] = make_float4(xa, ya, ca, sa);
        if constexpr (COST) {
          const float* xr = xrf + (t + 1) * 3;
          const float e0 = xa - xr[0], e1 = ya - xr[1], e2 = th_a - xr[2];
          const float2 u = Uf[t], a = Af[t];
          lc += fmaf(D.Q[0] * e0, e0, fmaf(D.Q[1] * e1, e1, fmaf(D.Q[2] * e2, e2,
                     fmaf(a.x, v.x - u.x, a.y * (v.y - u.y)))));
          if (t == T - 1) {
            const float* xT = xrf + T * 3;
            const float f0 = xa - xT[0], f1 = ya - xT[1], f2 = th_a - xT[2];
            lc += fmaf(D.Qf[0] * f0, f0, fmaf(D.Qf[1] * f1, f1, D.Qf[2] * f2 * f2));
          }
        }
      }
      cth = lane31(th_a);
      cc_ = lane31(ca);
      cs_ = lane31(sa);
      cx = lane31(xa);
      cy = lane31(ya);
    }
    if constexpr (COST) ff_add(cost, lc);
  } else if constexpr (MODEL == 2) {
    // Ackermann (Eq. 14): speed -> heading (rate v tan(steer) / L) ->
    // (cos, sin) -> position, each a prefix sum over the segment's steps
    float cx = x_init[0], cy = x_init[1], cth = x_init[2], cv = x_init[3];
    float cs_, cc_;
    sincosf(cth, &cs_, &cc_);
    const float kth = D.k_turn * dt;  // 1 / L
    float lc = 0.0f;
    for (int t0 = 0; t0 < T; t0 += 32) {
      const int t = t0 + lane;
      const bool valid = t < T;
      const float2 v = valid ? V[t * vs] : make_float2(0.0f, 0.0f);
      const float v_a = cv + warp_incl_scan(v.y * dt, lane);  // v_{t+1}
      const float v_b = from_prev_lane(v_a, cv, lane);       // v_t
      const float th_a = cth + warp_incl_scan(v_b * tanf(v.x) * kth, lane);
      float sa, ca;
      sincosf(th_a, &sa, &ca);
      const float cb = from_prev_lane(ca, cc_, lane), sb = from_prev_lane(sa, cs_, lane);
      const float vdt = v_b * dt;
      const float xa = cx + warp_incl_scan(vdt * cb, lane);
      const float ya = cy + warp_incl_scan(vdt * sb, lane);
      if (x1 && t == 0) {
        x1[0] = xa;
        x1[1] = ya;
        x1[2] = th_a;
        x1[3] = v_a;
      }
      if (valid) {
        pose[t * ps] = make_float4(xa, ya, ca, sa);
        if constexpr (COST) {
          const float xs[4] = {xa, ya, th_a, v_a};
          const float* xr = xrf + (t + 1) * 4;
          float q = 0.0f;
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            const float e = xs[d] - xr[d];
            q = fmaf(D.Q[d] * e, e, q);
          }
          const float2 u = Uf[t], a = Af[t];
          lc += fmaf(a.x, v.x - u.x, fmaf(a.y, v.y - u.y, q));
          if (t == T - 1) {
            const float* xT = xrf + T * 4;
            float f = 0.0f;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
              const float e = xs[d] - xT[d];
              f = fmaf(D.Qf[d] * e, e, f);
            }
            lc += f;
          }
        }
      }
      cv = lane31(v_a);
      cth = lane31(th_a);
      cc_ = lane31(ca);
      cs_ = lane31(sa);
      cx = lane31(xa);
      cy = lane31(ya);
    }
    if constexpr (COST) ff_add(cost, lc);
  } else if constexpr (MODEL == 3) {
    // the paper's planar quadrotor (Eq. 12): pitch (rate omega) -> (cos,
    // sin) -> velocities (thrust m g + u_t) -> position
    float cx = x_init[0], cz = x_init[1], cth = x_init[2];
    float cvx = x_init[3], cvz = x_init[4];
    float cs_, cc_;
    sincosf(cth, &cs_, &cc_);
    float lc = 0.0f;
    for (int t0 = 0; t0 < T; t0 += 32) {
      const int t = t0 + lane;
      const bool valid = t < T;
      const float2 v = valid ? V[t * vs] : make_float2(0.0f, 0.0f);
      const float th_a = cth + warp_incl_scan(v.x * dt, lane);  // theta_{t+1}
      float sa, ca;
      sincosf(th_a, &sa, &ca);
      const float cb = from_prev_lane(ca, cc_, lane), sb = from_prev_lane(sa, cs_, lane);
      const float acc = fmaf(v.y, D.inv_mass, D.g);  // (m g + u_t) / m
      const float vx_a = cvx + warp_incl_scan(-acc * sb * dt, lane);
      const float vz_a = cvz + warp_incl_scan(fmaf(acc, cb, -D.g) * dt, lane);
      const float vx_b = from_prev_lane(vx_a, cvx, lane), vz_b = from_prev_lane(vz_a, cvz, lane);
      const float x_a = cx + warp_incl_scan(vx_b * dt, lane);
      const float z_a = cz + warp_incl_scan(vz_b * dt, lane);
      if (x1 && t == 0) {
        x1[0] = x_a;
        x1[1] = z_a;
        x1[2] = th_a;
        x1[3] = vx_a;
        x1[4] = vz_a;
      }
      if (valid) {
        pose[t * ps] = make_float4(x_a, z_a, ca, sa);
        if constexpr (COST) {
          const float xs[5] = {x_a, z_a, th_a, vx_a, vz_a};
          const float* xr = xrf + (t + 1) * 5;
          float q = 0.0f;
#pragma unroll
          for (int d = 0; d < 5; ++d) {
            const float e = xs[d] - xr[d];
            q = fmaf(D.Q[d] * e, e, q);
          }
          const float2 u = Uf[t], a = Af[t];
          lc += fmaf(a.x, v.x - u.x, fmaf(a.y, v.y - u.y, q));
          if (t == T - 1) {
            const float* xT = xrf + T * 5;
            float f = 0.0f;
#pragma unroll
            for (int d = 0; d < 5; ++d) {
              const float e = xs[d] - xT[d];
              f = fmaf(D.Qf[d] * e, e, f);
            }
            lc += f;
          }
        }
      }
      cth = lane31(th_a);
      cc_ = lane31(ca);
      cs_ = lane31(sa);
      cvx = lane31(vx_a);
      cvz = lane31(vz_a);
      cx = lane31(x_a);
      cz = lane31(z_a);
    }
    if constexpr (COST) ff_add(cost, lc);
  } else {
    float cy = x_init[0], cz = x_init[1], cph = x_init[2];
    float cvy = x_init[3], cvz = x_init[4], cw = x_init[5];
    float cs_, cc_;
    sincosf(cph, &cs_, &cc_);
    const float kw = D.k_turn * dt;  // arm / I
    float lc = 0.0f;
    for (int t0 = 0; t0 < T; t0 += 32) {
      const int t = t0 + lane;
      const bool valid = t < T;
      const float2 v = valid ? V[t * vs] : make_float2(0.0f, 0.0f);
      const float w_a = cw + warp_incl_scan((v.y - v.x) * kw, lane);  // phidot_{t+1}
      const float w_b = from_prev_lane(w_a, cw, lane);                // phidot_t
      const float ph_a = cph + warp_incl_scan(w_b * dt, lane);        // phi_{t+1}
      float sa, ca;
      sincosf(ph_a, &sa, &ca);
      const float cb = from_prev_lane(ca, cc_, lane), sb = from_prev_lane(sa, cs_, lane);
      const float acc = fmaf(v.x + v.y, D.inv_mass, D.g);  // (F1 + F2) / m
      const float vy_a = cvy + warp_incl_scan(-acc * sb * dt, lane);
      const float vz_a = cvz + warp_incl_scan(fmaf(acc, cb, -D.g) * dt, lane);
      const float vy_b = from_prev_lane(vy_a, cvy, lane), vz_b = from_prev_lane(vz_a, cvz, lane);
      const float y_a = cy + warp_incl_scan(vy_b * dt, lane);
      const float z_a = cz + warp_incl_scan(vz_b * dt, lane);
      if (x1 && t == 0) {
        x1[0] = y_a;
        x1[1] = z_a;
        x1[2] = ph_a;
        x1[3] = vy_a;
        x1[4] = vz_a;
        x1[5] = w_a;
      }
      if (valid) {
        pose[t * ps] = make_float4(y_a, z_a, ca, sa);
        if constexpr (COST) {
          const float xs[6] = {y_a, z_a, ph_a, vy_a, vz_a, w_a};
          const float* xr = xrf + (t + 1) * 6;
          float q = 0.0f;
#pragma unroll
          for (int d = 0; d < 6; ++d) {
            const float e = xs[d] - xr[d];
            q = fmaf(D.Q[d] * e, e, q);
          }
          const float2 u = Uf[t], a = Af[t];
          lc += fmaf(a.x, v.x - u.x, fmaf(a.y, v.y - u.y, q));
          if (t == T - 1) {
            const float* xT = xrf + T * 6;
            float f = 0.0f;
#pragma unroll
            for (int d = 0; d < 6; ++d) {
              const float e = xs[d] - xT[d];
              f = fmaf(D.Qf[d] * e, e, f);
            }
            lc += f;
          }
        }
      }
      cw = lane31(w_a);
      cph = lane31(ph_a);
      cc_ = lane31(ca);
      cs_ = lane31(sa);
      cvy = lane31(vy_a);
      cvz = lane31(vz_a);
      cy = lane31(y_a);
      cz = lane31(z_a);
    }
    if constexpr (COST) ff_add(cost, lc);
  }
}

// The grid map in the tile's frame, whose origin is the measured position
// (x0g[0], x0g[1]).  FP64, so one thread builds it (grid_shared) and the
// others read it from shared memory.
__device__ __forceinline__ GridView grid_view(const CtrlDesc& D, const double* __restrict__ x0g) {
  const DevState* st = D.st;
  GridView gv;
  gv.g = st->grid;
  gv.nx = st->grid_nx;
  gv.ny = st->grid_ny;
  gv.inv_res = st->grid_inv_res;
  if (!gv.g) return gv;
  // x0's grid coordinates, bounded so that the cell fits an int (beyond the
  // bound every point lies off the map and clamps to its edge anyway)
  const double u = fmin(fmax((x0g[0] - st->grid_ox) / st->grid_res, -1073741824.0), 1073741824.0);
  const double v = fmin(fmax((x0g[1] - st->grid_oy) / st->grid_res, -1073741824.0), 1073741824.0);
  const double fu = floor(u), fv = floor(v);
  gv.ci = (int)fu;
  gv.cj = (int)fv;
  gv.ru = (float)(u - fu);
  gv.rv = (float)(v - fv);
  return gv;
}

// The CTA's copy of its grid view (only the grid kernels instantiate it).
__device__ __forceinline__ GridView& grid_shared() {
  __shared__ GridView s;
  return s;
}

// Algorithm 1's SGF on the merged column sums, in place: hi[2t + d] becomes
// the smoothed sum and lo[2t + d] zero.  The filter is linear, so smoothing
// the sums before their common 1 / Z scale is smoothing the update.  Window
// start s = clamp(t - W/2, 0, T - W); t sits at position t - s of it.
// buf: 2T floats of free shared memory.  Called by every thread of the CTA.
__device__ __forceinline__ void sgf_columns(const float* __restrict__ w, int W, int T, float* hi,
                                           float* lo, float* buf, int tid, int nthreads) {
  const int ncol = 2 * T, half = W >> 1;
  __syncthreads();
  for (int c = tid; c < ncol; c += nthreads) buf[c] = hi[c] + lo[c];
  __syncthreads();
  for (int c = tid; c < ncol; c += nthreads) {
    const int t = c >> 1, d = c & 1;
    const int s = min(max(t - half, 0), T - W);
    const float* wq = w + (t - s) * W;
    const float* y = buf + 2 * s + d;
    float a = 0.0f;
    for (int i = 0; i < W; ++i) a = fmaf(wq[i], y[2 * i], a);
    hi[c] = a;
    lo[c] = 0.0f;
  }
  __syncthreads();
}

// Final stage (one CTA per controller per step): U* from the merged sums
// (Eq. 4), Algorithm 1's receding-horizon shift (u_t <- u*_{t+1}, the last
// entry kept), the nominal rollout of U* over the horizon for C_B, S_e
// (Eq. 10, C_B floored at 0 inside the logarithm) and the state update.  The
// next step's constants that do not depend on S_e (u_t in FP32, a'_t = gamma
// Sigma^-1 u_t and sum_t u_t . a'_t) are formed with the shift, one step per
// thread; S_e enters afterwards through L, C0 and the 1 / S_e that the next
// step applies to a'_t.
// One CTA runs this alone at the end of the step, so its length is a chain
// of latencies: the measured position comes from the tile's scratch (no
// memory round trip), and the lanes of a warp meet (__syncwarp) before the
// shuffles of a reduction that follows a loop they left at different
// steps.  Each thread forms u*_t and u*_{t+1} itself, which is faster here
// than forming each entry once and reading the neighbour after a barrier
// (that costs another barrier and more code, which a step run after an L2
// flush fetches from memory).
template <int MODEL, int NPOS, bool GRID = false>
__device__ void final_stage(const CtrlDesc& D, char* smem, const SmemLayout& L, TileScratch& ts,
                            double* out, const GridView* gv = nullptr) {
  const int tid = threadIdx.x, nthreads = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int T = D.T, P = D.P;
  const double* Us = reinterpret_cast<const double*>(smem + L.Us);  // the step's U
  float2* Usf = reinterpret_cast<float2*>(smem + L.Usf);
  const float* col_hi = reinterpret_cast<const float*>(smem + L.colhi);
  const float* col_lo = reinterpret_cast<const float*>(smem + L.collo);
  float4* pose_nom = reinterpret_cast<float4*>(smem + L.region);
  float* b_nom = reinterpret_cast<float*>(smem + L.region + 16 * T);
  const float2* shp = reinterpret_cast<const float2*>(smem + L.shp);
  const float4* obs4 = reinterpret_cast<const float4*>(smem + L.obs4);
  const float* cw = reinterpret_cast<const float*>(smem + L.cw);
  const float* xi = reinterpret_cast<const float*>(smem + L.xi);
  float* redf = reinterpret_cast<float*>(smem + L.red);
  // Z >= 1 (the minimum's own weight is 1), so its float reciprocal and the
  // float quotient carry the update to about 1e-7 relative
  const float invZ = 1.0f / (ts.Z.hi + ts.Z.lo);
  const float M00 = (float)D.Sinv[0], M01 = (float)D.Sinv[1];
  const float M10 = (float)D.Sinv[2], M11 = (float)D.Sinv[3];
  FF c0 = {0.0f, 0.0f};
  double us0[2] = {0.0, 0.0};  // u*_0, kept by thread 0
  for (int t = tid; t < T; t += nthreads) {
    const int tn = t + 1 < T ? t + 1 : T - 1;
    double us[2], un[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const int c = 2 * t + d, cn = 2 * tn + d;
      us[d] = fmin(fmax(Us[c] + (double)((col_hi[c] + col_lo[c]) * invZ), D.umin_d[d]), D.umax_d[d]);
      un[d] = fmin(fmax(Us[cn] + (double)((col_hi[cn] + col_lo[cn]) * invZ), D.umin_d[d]), D.umax_d[d]);
      D.Ustar[c] = us[d];
      D.U[c] = un[d];
    }
    if (t == 0) {
      us0[0] = us[0];
      us0[1] = us[1];
    }
    Usf[t] = make_float2((float)us[0], (float)us[1]);
    const float v0 = (float)un[0], v1 = (float)un[1];
    const float a0 = fmaf(M00, v0, M01 * v1), a1 = fmaf(M10, v0, M11 * v1);
    D.cU[t] = make_float2(v0, v1);
    D.cA[t] = make_float2(a0, a1);
    ff_add_prod(c0, v0, a0, 0.0f);
    ff_add_prod(c0, v1, a1, 0.0f);
  }
  __syncwarp();
  c0 = warp_sum_ff(c0);
  if (lane == 0) {
    redf[2 * warp] = c0.hi;
    redf[2 * warp + 1] = c0.lo;
  }
  __syncthreads();
  float* x1 = reinterpret_cast<float*>(smem + L.scH);  // per-sample sums are consumed
  if (tid < 32) {
    FF none = {0.0f, 0.0f};
    scan_trajectory<MODEL, false>(D, T, Usf, 1, xi, pose_nom, 1, nullptr, nullptr, nullptr, none,
                                  lane, x1);
  }
  __syncthreads();
  barrier_flat<GRID>(T * P, P, D.J, pose_nom, shp, obs4, D.h_eps, b_nom, tid, nthreads, gv);
  __syncthreads();
  if (tid < 32) {
    FF a = {0.0f, 0.0f};
    for (int t = lane; t < T; t += 32) {
      float b = 0.0f;  // the step's P shape-point sums
      for (int p = 0; p < P; ++p) b += fabsf(b_nom[t * P + p]);
      ff_add_prod(a, cw[t], b, 0.0f);
    }
    __syncwarp();
    a = warp_sum_ff(a);
    FF cs = lane < (nthreads >> 5) ? FF{redf[2 * lane], redf[2 * lane + 1]} : FF{0.0f, 0.0f};
    cs = warp_sum_ff(cs);
    if (tid == 0) {
      DevState* st = D.st;
      const double CB = (double)a.hi + (double)a.lo + ts.Kconst;
      // Eq. 10, C_B floored at 0 inside the logarithm
      const float arg = (float)(2.718281828459045 + fmax(CB, 0.0));
      const double S_e_next = D.mu_coarse > 0.0 ? D.mu_coarse * (double)logf(arg) : 1.0;
      const float Se = (float)S_e_next, r = sqrtf(Se), inv_Se = 1.0f / Se;
      st->L00 = r * (float)D.Lsig[0];
      st->L10 = r * (float)D.Lsig[1];
      st->L11 = r * (float)D.Lsig[2];
      st->C0 = (double)((cs.hi + cs.lo) * inv_Se);
      st->rho = ts.base + ((double)ts.rho.hi + (double)ts.rho.lo);
      st->Z = (double)ts.Z.hi + (double)ts.Z.lo;
      st->CB_star = CB;
      st->beta_used = ts.beta0;
      st->beta_d = ts.beta_d;
      st->S_e_used = ts.S_e_used;
      st->u0[0] = us0[0];
      st->u0[1] = us0[1];
      if (D.host_out) {  // what mppi_get_control reads, straight to host memory
        D.host_out->u0[0] = us0[0];
        D.host_out->u0[1] = us0[1];
        D.host_out->status = *reinterpret_cast<volatile int*>(&st->status);
        __threadfence_system();
        *reinterpret_cast<volatile int*>(&D.host_out->seq) = (int)(uint32_t)(ts.iter + 1ull);
      }
      constexpr int n = Dyn<MODEL>::n;
      double xn[6] = {0, 0, 0, 0, 0, 0};
      xn[0] = ts.x0[0] + (double)x1[0];  // back from the frame centred on x0
      xn[1] = ts.x0[1] + (double)x1[1];
      for (int d = 2; d < n; ++d) xn[d] = (double)x1[d];
      for (int d = 0; d < 6; ++d) st->x1[d] = xn[d];
      if (out) {  // batched launches: u0 then the predicted state, 8 doubles
        out[0] = us0[0];
        out[1] = us0[1];
        for (int d = 0; d < 6; ++d) out[2 + d] = xn[d];
      }
      st->S_e = S_e_next;
      st->beta = ts.beta0;
      st->first = 0;
      st->iter = ts.iter + 1ull;
    }
  }
}

// One tile of one controller.  ts.mbar must be initialised; mbar_phase is
// each thread's own copy of the parity of the barrier's next completion.
// BATCHED: the tile runs in the persistent batch kernel, which takes the
// one-batch form of merge_partials and the odd row stride of row_stride;
// the one-controller kernels take the pipelined merge and SP = S.  Both
// choices were measured per kernel; the results are the same bit for bit.
// GRID: the grid map's terms are compiled in (taken when D.st->grid is set).
// SGF: the Savitzky-Golay pass is compiled in (taken when D.sgf_wp is set).
// The batch kernels carry it, and the one-controller kernels have a form
// with it and one without, so that controllers that do not smooth run code
// with no trace of it.
// The one-controller kernels inline the body (run_tile_inl), so the
// descriptor stays the kernel's own parameter: its fields are read from the
// parameter bank, and no store in the body can alias them.  The batch
// kernels call it out of line (run_tile), which keeps their four-model
// switch small.
template <int MODEL, int NPOS, bool BATCHED, bool SGF = BATCHED, bool GRID = false>
__device__ __forceinline__ void run_tile_inl(const CtrlDesc& D, int tile,
                                             const double* __restrict__ x0g,
                                             const double* __restrict__ xrefg, char* smem,
                                             TileScratch& ts, uint32_t& mbar_phase,
                                             double* u0_out = nullptr) {
  constexpr int n = Dyn<MODEL>::n;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
  const int T = D.T, S = D.S, P = D.P, J = D.J, K = D.K;
  const int SP = row_stride(S, BATCHED);  // row stride of the (t, s) arrays
  const SmemLayout L = smem_layout(T, S, P, J, n, D.nscl, nwarps, BATCHED);
  float4* obs4 = reinterpret_cast<float4*>(smem + L.obs4);
  float4* pose = reinterpret_cast<float4*>(smem + L.pose);
  float2* uB = reinterpret_cast<float2*>(smem + L.pose);  // overlays pose, stride 2
  float2* V = reinterpret_cast<float2*>(smem + L.V);
  float2* Uf = reinterpret_cast<float2*>(smem + L.Uf);
  float2* Af = reinterpret_cast<float2*>(smem + L.Af);
  float* xrf = reinterpret_cast<float*>(smem + L.xrf);
  float2* shp = reinterpret_cast<float2*>(smem + L.shp);
  float* eS = reinterpret_cast<float*>(smem + L.eS);
  float* cw = reinterpret_cast<float*>(smem + L.cw);
  float* scH = reinterpret_cast<float*>(smem + L.scH);
  float* scL = reinterpret_cast<float*>(smem + L.scL);
  unsigned char* collf = reinterpret_cast<unsigned char*>(smem + L.collf);
  float* xi = reinterpret_cast<float*>(smem + L.xi);
  double* red = reinterpret_cast<double*>(smem + L.red);
  DevState* st = D.st;
  const int k0 = tile * S;

  // ---- prologue: stage obstacles (TMA bulk copy), per-step constants
  __syncthreads();  // previous use of shared memory by this CTA is over
#if DBM_STAGE_TMA
  if (tid == 0 && J > 0)
    tma_bulk_g2s(smem + L.region, D.obst, (uint32_t)align_up(24 * J, 16), &ts.mbar);
#endif
  if (tid < P) shp[tid] = make_float2(D.shape[2 * tid], D.shape[2 * tid + 1]);
  // Loads ahead of stores: the shared-memory stores below go through
  // pointers that the compiler cannot tell apart from the global arrays read
  // here, so a load written after a store is issued only once that store's
  // data has arrived, and interleaved loads and stores pay one memory round
  // trip each.  Written in this order, the state words and the sequence's
  // constants take one round trip and the reference rows (kXrefBatch per
  // thread at a time) one more.  Issuing the reference loads before the
  // constants' stores as well saves that second trip but costs registers
  // that the 14-point barrier loop needs: slower at 14 points per thread.
  const double ox = x0g[0], oy = x0g[1];
  const double x0t = tid < n ? x0g[tid] : 0.0;
  double* Us = reinterpret_cast<double*>(smem + L.Us);
  const double S_e = st->S_e;
  const unsigned long long iter = tid == 0 ? st->iter : 0ull;
  const float inv_Se = 1.0f / (float)S_e;  // a_t = a'_t / S_e
  for (int t = tid; t < T; t += nthreads) {
    const float2 u = D.cU[t], a = D.cA[t];
    const float w = D.cw[t];
    const double v0 = D.U[2 * t], v1 = D.U[2 * t + 1];
    Uf[t] = u;
    Af[t] = make_float2(a.x * inv_Se, a.y * inv_Se);
    cw[t] = w;
    Us[2 * t] = v0;  // for the final stage, should this CTA run it
    Us[2 * t + 1] = v1;
  }
  {
    constexpr int kXrefBatch = 4;
    const int NX = (T + 1) * n;
    for (int i0 = tid; i0 < NX; i0 += kXrefBatch * nthreads) {
      double v[kXrefBatch];
#pragma unroll
      for (int r = 0; r < kXrefBatch; ++r) {
        const int i = i0 + r * nthreads;
        v[r] = i < NX ? xrefg[i] : 0.0;
      }
#pragma unroll
      for (int r = 0; r < kXrefBatch; ++r) {
        const int i = i0 + r * nthreads, d = i % n;
        if (i < NX) xrf[i] = (float)(d == 0 ? v[r] - ox : d == 1 ? v[r] - oy : v[r]);
      }
    }
  }
  if (tid < n) xi[tid] = tid < 2 ? 0.0f : (float)x0t;
  if (tid == 0) {  // read early: only the final stage uses them
    ts.S_e_used = S_e;
    ts.iter = iter;
    ts.x0[0] = ox;
    ts.x0[1] = oy;
    if constexpr (GRID) grid_shared() = grid_view(D, x0g);  // read after the next barrier
  }
  if (J > 0) {
#if DBM_STAGE_TMA
    bool ok = mbar_wait(&ts.mbar, mbar_phase, kTmaPolls, kTmaWaitCycles);
    if (!ok) {
      if (tid == 0) atomicExch(&st->status, kStatusTimeout);
      mbar_wait(&ts.mbar, mbar_phase, kTmaPolls, kTmaWaitCycles);
    }
    mbar_phase ^= 1u;  // every thread flips its own copy
    const double* raw = reinterpret_cast<const double*>(smem + L.region);
#else
    const double* raw = D.obst;
#endif
    // the raw (region) and converted (obs4) areas are distinct
    for (int j = tid; j < J; j += nthreads) {
      double cx = raw[3 * j], cy = raw[3 * j + 1], r = raw[3 * j + 2];
      obs4[j] = make_float4((float)(cx - ox), (float)(cy - oy), -(float)(r * r), 0.0f);
    }
  }
  __syncthreads();
  // barrier at the goal pose (beta_d of Eq. 7) and at the measured pose
  float gx = (float)(D.x_goal[0] - ox), gy = (float)(D.x_goal[1] - oy);
  float gs, gc, xs, xc;
  sincosf((float)D.x_goal[2], &gs, &gc);
  sincosf((float)x0g[2], &xs, &xc);
  float bd = 0.0f, b0 = 0.0f;
  if constexpr (GRID) {
    const GridView gv = grid_shared();
    if (gv.g) {
      for (int p = tid; p < P; p += nthreads) {
        const float2 sh = shp[p];
        bd += 1.0f / fmaxf(grid_h(gv, fmaf(gc, sh.x, fmaf(-gs, sh.y, gx)),
                                  fmaf(gs, sh.x, fmaf(gc, sh.y, gy))), D.h_eps);
        b0 += 1.0f / fmaxf(grid_h(gv, fmaf(xc, sh.x, -xs * sh.y), fmaf(xs, sh.x, xc * sh.y)),
                           D.h_eps);
      }
    }
  }
  for (int i = tid; i < P * J; i += nthreads) {
    int p = i / J, j = i - p * J;
    float2 sh = shp[p];
    float4 o = obs4[j];
    float X = fmaf(gc, sh.x, fmaf(-gs, sh.y, gx)), Y = fmaf(gs, sh.x, fmaf(gc, sh.y, gy));
    float dx = X - o.x, dy = Y - o.y;
    bd += 1.0f / fmaxf(fmaf(dx, dx, fmaf(dy, dy, o.z)), D.h_eps);
    X = fmaf(xc, sh.x, -xs * sh.y);
    Y = fmaf(xs, sh.x, xc * sh.y);
    dx = X - o.x;
    dy = Y - o.y;
    b0 += 1.0f / fmaxf(fmaf(dx, dx, fmaf(dy, dy, o.z)), D.h_eps);
  }
  {
    float v0 = warp_sum_f(bd), v1 = warp_sum_f(b0);
    if (lane == 0) {
      reinterpret_cast<float*>(red)[2 * warp] = v0;
      reinterpret_cast<float*>(red)[2 * warp + 1] = v1;
    }
  }

  // ---- noise: every (sample, step) draw, kept as the clamped control
  {
    const uint32_t it_lo = (uint32_t)(st->iter & 0xffffffffull);
    const uint32_t it_hi = (uint32_t)(st->iter >> 32);
    const float L00 = st->L00, L10 = st->L10, L11 = st->L11;
    const float lo0 = D.umin[0], hi0 = D.umax[0], lo1 = D.umin[1], hi1 = D.umax[1];
    // item i = t S + s, stored at t SP + s; (t, s) stepped by nthreads
    // without a division
    const int dt = nthreads / S, ds = nthreads - dt * S;
    int t = tid / S, s = tid - t * S;
#pragma unroll 2
    for (int i = tid; i < T * S; i += nthreads) {
      const uint4 r = philox4x32_10(make_uint4((uint32_t)(k0 + s), (uint32_t)t, it_lo, it_hi),
                                    D.key0, D.key1);
      const float2 du = nln_draw(r, L00, L10, L11, D.ln_mu, D.ln_sigma);
      const float2 u = Uf[t];
      V[t * SP + s] =
          make_float2(fminf(fmaxf(u.x + du.x, lo0), hi0), fminf(fmaxf(u.y + du.y, lo1), hi1));
      t += dt;
      s += ds;
      if (s >= S) {
        s -= S;
        ++t;
      }
    }
  }
  __syncthreads();
  // (one lane of the last warp, which has the fewest samples below)
  if (tid == nthreads - 32) {
    float fbd = 0.0f, fb0 = 0.0f;
    for (int w = 0; w < nwarps; ++w) {
      fbd += reinterpret_cast<const float*>(red)[2 * w];
      fb0 += reinterpret_cast<const float*>(red)[2 * w + 1];
    }
    const double sbd = fbd, sb0 = fb0;
    double beta0 = st->first ? sb0 : sb0 + D.gamma_bas * (st->beta - sbd);
    ts.beta_d = sbd;
    ts.beta0 = beta0;
    // sample-independent part of sum_t R_B w_t (unrolled Eq. 7)
    ts.Kconst = D.R_B_d * (beta0 * st->g1 - D.gamma_bas * sbd * st->csum);
    ts.base = st->C0 + ts.Kconst;
  }

  // ---- dynamics and stage/control costs: one warp per sample
  for (int s = warp; s < S; s += nwarps) {
    FF c = {0.0f, 0.0f};
    scan_trajectory<MODEL, true>(D, T, V + s, SP, xi, pose + s, SP, Uf, Af, xrf, c, lane);
    c = warp_sum_ff(c);
    if (lane == 0) {
      scH[s] = c.hi;
      scL[s] = c.lo;
    }
  }
  __syncthreads();

  // ---- fused barrier over all (step, sample) units, sums over the poses
  if constexpr (GRID) {
    const GridView gv = grid_shared();
    barrier_units<NPOS, BATCHED, true>(T * S, S, P, J, pose, shp, obs4, D.h_eps, uB, 2, tid,
                                       nthreads, &gv);
  } else {
    barrier_units<NPOS, BATCHED>(T * S, S, P, J, pose, shp, obs4, D.h_eps, uB, 2, tid, nthreads);
  }
  __syncthreads();

  // ---- barrier-state and collision costs: one warp per sample; costs are
  // kept relative to base = C0 + Kconst (the same for every sample of the
  // controller, so it cancels in the weights)
  float* relH = reinterpret_cast<float*>(smem + L.scH);
  float* relL = reinterpret_cast<float*>(smem + L.scL);
  for (int s = warp; s < S; s += nwarps) {
    FF b = {0.0f, 0.0f};
    bool coll = false;
    for (int t = lane; t < T; t += 32) {
      const float2 v = uB[2 * (t * SP + s)];
      const bool cl = __float_as_int(v.x) < 0;
      ff_add_prod(b, cw[t], fabsf(v.x), v.y);
      if (cl) ff_add(b, D.C_coll);
      coll |= cl;
    }
    b = warp_sum_ff(b);
    coll = __any_sync(0xffffffffu, coll);
    if (lane == 0) {
      FF c = {scH[s], scL[s]};
      c = ff_norm(ff_sum(c, b));
      relH[s] = c.hi;
      relL[s] = c.lo;
      collf[s] = coll ? 1 : 0;
    }
  }
  __syncthreads();

  // ---- tile weights (Eq. 4 relative to the tile's own minimum)
  if (warp == 0) {
    const bool valid = (lane < S) && (k0 + lane < K);
    const FF Sk = valid ? FF{relH[lane], relL[lane]} : FF{__int_as_float(0x7f800000), 0.0f};
    const FF rho_c = warp_min_ff(Sk);
    const float e = valid ? expf(-ff_diff(Sk, rho_c) * D.inv_lambda_f) : 0.0f;
    const FF z = ff_norm(warp_sum_ff(FF{e, 0.0f}));
    eS[lane] = e;
    if (lane == 0) {
      D.part_rz[tile] = make_float4(rho_c.hi, rho_c.lo, z.hi, z.lo);
      atomicMax(&D.counters[D.nGroups + 1 + tile / D.GT], min_key(rho_c.hi));
    }
    if (valid) {
      D.costs[k0 + lane] = ts.base + ((double)Sk.hi + (double)Sk.lo);
      D.coll[k0 + lane] = collf[lane];
    }
  }
  __syncthreads();
  {
    // one thread per column (t, d): sum over the tile's samples, whose
    // weights eS are zero past K
    float* prow = D.part + (size_t)tile * 2 * T;
    for (int c = tid; c < 2 * T; c += nthreads) {
      const int t = c >> 1;
      const float* Vt = reinterpret_cast<const float*>(V + t * SP) + (c & 1);
      const float u = reinterpret_cast<const float*>(Uf + t)[c & 1];
      float a = 0.0f;
      for (int s = 0; s < S; ++s) a = fmaf(eS[s], Vt[2 * s] - u, a);
      prow[c] = a;
    }
  }

  // ---- two-level last-arriver merge.  The CTA's writes are published by
  // one thread: barrier, fence, ticket; the last arriver fences again before
  // the barrier that releases its threads to read the others' partials.  The
  // merge reads (and clears) the group's minimum word, the exact minimum of
  // its members' rho.
  __syncthreads();
  const int g = tile / D.GT;
  const int m0 = g * D.GT;
  const int members = min(D.GT, D.nTiles - m0);
  unsigned* minw = D.counters + D.nGroups + 1;
  if (tid == 0) {
    __threadfence();
    unsigned tk = atomicAdd(&D.counters[g], 1u);
    ts.flag = (tk == (unsigned)(members - 1));
    if (ts.flag) {
      __threadfence();
      D.counters[g] = 0u;
    }
  }
  __syncthreads();
  if (!ts.flag) return;
  float* scl = reinterpret_cast<float*>(smem + L.scl);
  float* col_hi = reinterpret_cast<float*>(smem + L.colhi);
  float* col_lo = reinterpret_cast<float*>(smem + L.collo);
  const int ncol = 2 * T;
  FF* mbuf = reinterpret_cast<FF*>(smem + L.region);
  float2* zi = reinterpret_cast<float2*>(smem + L.region + merge_buf_bytes(ncol, nthreads));
  merge_partials<!BATCHED>(members, D.part_rz + m0, D.part + (size_t)m0 * ncol, ncol, &minw[g],
                           D.inv_lambda_f, scl, zi, mbuf, &ts.ref, &ts.Z, col_hi, col_lo, tid,
                           nthreads);
  if (D.nGroups > 1) {
    for (int c = tid; c < ncol; c += nthreads) D.gpart[(size_t)g * ncol + c] = col_hi[c] + col_lo[c];
    if (tid == 0) {
      D.gpart_rz[g] = make_float4(ts.ref, 0.0f, ts.Z.hi, ts.Z.lo);
      atomicMax(&minw[D.nGroups], min_key(ts.ref));
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      unsigned tk = atomicAdd(&D.counters[D.nGroups], 1u);
      ts.flag = (tk == (unsigned)(D.nGroups - 1));
      if (ts.flag) {
        __threadfence();
        D.counters[D.nGroups] = 0u;
      }
    }
    __syncthreads();
    if (!ts.flag) return;
    merge_partials<!BATCHED>(D.nGroups, D.gpart_rz, D.gpart, ncol, &minw[D.nGroups],
                             D.inv_lambda_f, scl, zi, mbuf, &ts.ref, &ts.Z, col_hi, col_lo, tid,
                             nthreads);
  }
  if constexpr (SGF) {
    if (D.sgf_wp)
      sgf_columns(D.cw + sgf_table_offset(T), D.sgf_wp & 0xff, T, col_hi, col_lo,
                  reinterpret_cast<float*>(smem + L.region), tid, nthreads);
  }
  if (tid == 0) ts.rho = FF{ts.ref, 0.0f};
  if constexpr (GRID) {
    const GridView gv = grid_shared();
    final_stage<MODEL, NPOS, true>(D, smem, L, ts, u0_out, &gv);
  } else {
    final_stage<MODEL, NPOS>(D, smem, L, ts, u0_out);
  }
}

template <int MODEL, int NPOS, bool BATCHED, bool SGF = BATCHED, bool GRID = false>
__device__ __noinline__ void run_tile(const CtrlDesc& D, int tile, const double* __restrict__ x0g,
                                      const double* __restrict__ xrefg, char* smem,
                                      TileScratch& ts, uint32_t& mbar_phase,
                                      double* u0_out = nullptr) {
  run_tile_inl<MODEL, NPOS, BATCHED, SGF, GRID>(D, tile, x0g, xrefg, smem, ts, mbar_phase, u0_out);
}

}  // namespace dbm
