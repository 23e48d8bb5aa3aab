// Tile body and final stage of the DBaS-Log-MPPI step; shared by the plain
// one-launch-per-controller kernel and the batched persistent kernel.
#pragma once

#include "mppi_device.cuh"

namespace dbm {

constexpr int kTmaPolls = 1 << 22;

// Per-step constants that depend only on the controller state (U, S_e):
// the Cholesky factor of S_e Sigma, a_t = gamma (S_e Sigma)^-1 u_t, u_t in
// FP32, and C0 = sum_t u_t . a_t, the part of the control cost of Eq. 9
// (Algorithm 1 form gamma u^T (S_e Sigma)^-1 v) that every sample shares.
// Run by one CTA after each shift, and by a one-CTA kernel after the host
// sets the state.  red: >= 40 doubles of shared memory.
__device__ inline void prep_constants(const CtrlDesc& D, double* red, int tid, int nthreads) {
  DevState* st = D.st;
  const int T = D.T;
  __syncthreads();
  if (tid == 0) {
    double Se = st->S_e;
    double a = Se * D.sigma[0], b = Se * D.sigma[1], c = Se * D.sigma[2], d = Se * D.sigma[3];
    double l00 = sqrt(fmax(a, 0.0));
    double l10 = l00 > 0.0 ? c / l00 : 0.0;
    double l11 = sqrt(fmax(d - l10 * l10, 0.0));
    st->L00 = (float)l00;
    st->L10 = (float)l10;
    st->L11 = (float)l11;
    double det = a * d - b * c;
    double gi = D.gamma_ctrl != 0.0 ? D.gamma_ctrl / det : 0.0;
    red[32] = gi * d;
    red[33] = -gi * b;
    red[34] = -gi * c;
    red[35] = gi * a;
  }
  __syncthreads();
  const double M00 = red[32], M01 = red[33], M10 = red[34], M11 = red[35];
  double c0 = 0.0;
  for (int t = tid; t < T; t += nthreads) {
    double u0 = D.U[2 * t], u1 = D.U[2 * t + 1];
    double a0 = M00 * u0 + M01 * u1, a1 = M10 * u0 + M11 * u1;
    D.cU[t] = make_float2((float)u0, (float)u1);
    D.cA[t] = make_float2((float)a0, (float)a1);
    c0 += u0 * a0 + u1 * a1;
  }
  c0 = warp_sum_d(c0);
  if ((tid & 31) == 0) red[tid >> 5] = c0;
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int w = 0; w < (nthreads >> 5); ++w) sum += red[w];
    st->C0 = sum;
  }
  __syncthreads();
}

// Final stage (one CTA per controller per step): U* from the merged sums
// (Eq. 4), nominal rollout of U* for C_B (Algorithm 1, "for t = 1..T"),
// S_e (Eq. 10, C_B floored at 0 inside the logarithm), shift, state update.
template <int MODEL, int NPOS>
__device__ void final_stage(const CtrlDesc& D, char* smem, const SmemLayout& L, TileScratch& ts,
                            double rho, double Z, const double* __restrict__ x0g) {
  constexpr int n = Dyn<MODEL>::n;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const int T = D.T, P = D.P;
  double* Us = reinterpret_cast<double*>(smem + L.Us);
  const float* col_hi = reinterpret_cast<const float*>(smem + L.colhi);
  const float* col_lo = reinterpret_cast<const float*>(smem + L.collo);
  float4* pose_nom = reinterpret_cast<float4*>(smem + L.region);
  float* posB_nom = reinterpret_cast<float*>(smem + L.region + 16 * T);
  const float2* shp = reinterpret_cast<const float2*>(smem + L.shp);
  const float4* obs4 = reinterpret_cast<const float4*>(smem + L.obs4);
  const double invZ = 1.0 / Z;
  for (int c = tid; c < 2 * T; c += nthreads) {
    int d = c & 1;
    double du = ((double)col_hi[c] + (double)col_lo[c]) * invZ;
    double u = D.U[c] + du;
    u = fmin(fmax(u, D.umin_d[d]), D.umax_d[d]);
    Us[c] = u;
    D.Ustar[c] = u;
  }
  __syncthreads();
  if (tid == 0) {
    float x[n];
    x[0] = 0.0f;
    x[1] = 0.0f;
#pragma unroll
    for (int d = 2; d < n; ++d) x[d] = (float)x0g[d];
    float sn, cs;
    sincosf(x[2], &sn, &cs);
    for (int t = 0; t < T; ++t) {
      Dyn<MODEL>::step(x, cs, sn, (float)Us[2 * t], (float)Us[2 * t + 1], D);
      pose_nom[t] = make_float4(x[0], x[1], cs, sn);
    }
  }
  __syncthreads();
  barrier_positions<NPOS>(T * P, 1, P, D.J, pose_nom, shp, obs4, D.h_eps, posB_nom, tid, nthreads);
  __syncthreads();
  if (tid == 0) {
    float w = (float)ts.beta0;
    FF cb = {0.0f, 0.0f};
    for (int t = 0; t < T; ++t) {
      float b = 0.0f;
      for (int p = 0; p < P; ++p) b += fabsf(posB_nom[t * P + p]);
      w = fmaf(D.gamma_bas_f, w - ts.beta_d_f, b);
      ff_add(cb, D.R_B * w);
    }
    double CB = (double)cb.hi + (double)cb.lo;
    DevState* st = D.st;
    double S_e_used = st->S_e;
    double S_e_next = D.mu_coarse > 0.0 ? D.mu_coarse * log(2.718281828459045 + fmax(CB, 0.0)) : 1.0;
    st->rho = rho;
    st->Z = Z;
    st->CB_star = CB;
    st->beta_used = ts.beta0;
    st->beta_d = ts.beta_d;
    st->S_e_used = S_e_used;
    st->u0[0] = Us[0];
    st->u0[1] = Us[1];
    st->S_e = S_e_next;
    st->beta = ts.beta0;
    st->first = 0;
    st->iter = st->iter + 1ull;
  }
  // shift (Algorithm 1, last loop): u_{t-1} <- u*_t, the last entry kept
  for (int c = tid; c < 2 * T; c += nthreads) {
    int t = c >> 1, d = c & 1;
    D.U[c] = (t + 1 < T) ? Us[2 * (t + 1) + d] : Us[2 * (T - 1) + d];
  }
  __threadfence_block();
  prep_constants(D, reinterpret_cast<double*>(smem + L.red), tid, nthreads);
}

// One tile of one controller.  ts.mbar must be initialised; ts.mbar_phase is
// the parity of its next completion.
template <int MODEL, int NPOS>
__device__ void run_tile(const CtrlDesc& D, int tile, const double* __restrict__ x0g,
                         const double* __restrict__ xrefg, char* smem, TileScratch& ts) {
  constexpr int n = Dyn<MODEL>::n;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
  const int T = D.T, S = D.S, P = D.P, J = D.J, TC = D.TC, K = D.K;
  const SmemLayout L = smem_layout(T, S, TC, P, J, n, D.nscl);
  float4* obs4 = reinterpret_cast<float4*>(smem + L.obs4);
  float4* pose = reinterpret_cast<float4*>(smem + L.pose);
  float2* dU = reinterpret_cast<float2*>(smem + L.dU);
  float* posB = reinterpret_cast<float*>(smem + L.posB);
  float2* Uf = reinterpret_cast<float2*>(smem + L.Uf);
  float2* Af = reinterpret_cast<float2*>(smem + L.Af);
  float* xrf = reinterpret_cast<float*>(smem + L.xrf);
  float2* shp = reinterpret_cast<float2*>(smem + L.shp);
  float* eS = reinterpret_cast<float*>(smem + L.eS);
  double* red = reinterpret_cast<double*>(smem + L.red);
  DevState* st = D.st;
  const int k0 = tile * S;

  // ---- prologue: stage obstacles (TMA bulk copy), per-step constants
  __syncthreads();  // previous use of shared memory by this CTA is over
  if (tid == 0 && J > 0)
    tma_bulk_g2s(smem + L.region, D.obst, (uint32_t)align_up(24 * J, 16), &ts.mbar);
  if (tid < P) shp[tid] = make_float2(D.shape[2 * tid], D.shape[2 * tid + 1]);
  const double ox = x0g[0], oy = x0g[1];
  for (int t = tid; t < T; t += nthreads) {
    Uf[t] = D.cU[t];
    Af[t] = D.cA[t];
  }
  for (int i = tid; i < (T + 1) * n; i += nthreads) {
    int d = i % n;
    double v = xrefg[i];
    if (d == 0) v -= ox;
    if (d == 1) v -= oy;
    xrf[i] = (float)v;
  }
  if (J > 0) {
    bool ok = mbar_wait(&ts.mbar, ts.mbar_phase, kTmaPolls);
    if (!ok) {
      if (tid == 0) atomicExch(&st->status, kStatusTimeout);
      mbar_wait(&ts.mbar, ts.mbar_phase, kTmaPolls);
    }
    ts.mbar_phase ^= 1u;
    const double* raw = reinterpret_cast<const double*>(smem + L.region);
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
      red[2 * warp] = (double)v0;
      red[2 * warp + 1] = (double)v1;
    }
  }
  // noise of chunk 0, all threads
  const uint32_t it_lo = (uint32_t)(st->iter & 0xffffffffull), it_hi = (uint32_t)(st->iter >> 32);
  const float L00 = st->L00, L10 = st->L10, L11 = st->L11;
  auto draw_chunk = [&](int c, int first, int count) {
    int t0 = c * TC;
    int TCc = min(TC, T - t0);
    for (int i = tid - first; i < TCc * S; i += count) {
      int tl = i / S, s = i - tl * S;
      int t = t0 + tl;
      uint4 r = philox4x32_10(make_uint4((uint32_t)(k0 + s), (uint32_t)t, it_lo, it_hi), D.key0,
                              D.key1);
      dU[t * S + s] = nln_draw(r, L00, L10, L11, D.ln_mu, D.ln_sigma);
    }
  };
  draw_chunk(0, 0, nthreads);
  __syncthreads();
  if (tid == 0) {
    double sbd = 0.0, sb0 = 0.0;
    for (int w = 0; w < nwarps; ++w) {
      sbd += red[2 * w];
      sb0 += red[2 * w + 1];
    }
    ts.beta_d = sbd;
    ts.beta_d_f = (float)sbd;
    ts.C0 = st->C0;
    ts.beta0 = st->first ? sb0 : sb0 + D.gamma_bas * (st->beta - sbd);
  }
  __syncthreads();

  // ---- rollout over chunks
  float x[n];
  float cs = 1.0f, sn = 0.0f, w = 0.0f;
  FF acc1 = {0.0f, 0.0f}, acc2 = {0.0f, 0.0f};
  bool coll = false;
  if (warp == 0) {
    x[0] = 0.0f;
    x[1] = 0.0f;
#pragma unroll
    for (int d = 2; d < n; ++d) x[d] = (float)x0g[d];
    sincosf(x[2], &sn, &cs);
    w = (float)ts.beta0;
  }
  const float gb = D.gamma_bas_f, bdf = ts.beta_d_f;
  auto recur_chunk = [&](int c) {
    int t0 = c * TC;
    int TCc = min(TC, T - t0);
    for (int tl = 0; tl < TCc; ++tl) {
      float b = 0.0f;
      bool cl = false;
      const float* pb = posB + (tl * S + lane) * P;
      for (int p = 0; p < P; ++p) {
        float v = pb[p];
        cl |= (__float_as_int(v) < 0);
        b += fabsf(v);
      }
      w = fmaf(gb, w - bdf, b);
      ff_add(acc2, D.R_B * w);
      if (cl) ff_add(acc2, D.C_coll);
      coll |= cl;
    }
  };
  const int nchunks = (T + TC - 1) / TC;
  for (int c = 0; c < nchunks; ++c) {
    const int t0 = c * TC;
    const int TCc = min(TC, T - t0);
    if (warp == 0) {
      if (lane < S) {
        if (c > 0) recur_chunk(c - 1);
        for (int tl = 0; tl < TCc; ++tl) {
          int t = t0 + tl;
          float2 u = Uf[t];
          float2 du = dU[t * S + lane];
          float v0 = fminf(fmaxf(u.x + du.x, D.umin[0]), D.umax[0]);
          float v1 = fminf(fmaxf(u.y + du.y, D.umin[1]), D.umax[1]);
          float e0 = v0 - u.x, e1 = v1 - u.y;
          dU[t * S + lane] = make_float2(e0, e1);
          Dyn<MODEL>::step(x, cs, sn, v0, v1, D);
          pose[tl * S + lane] = make_float4(x[0], x[1], cs, sn);
          const float* xr = xrf + (t + 1) * n;
          float q = 0.0f;
#pragma unroll
          for (int d = 0; d < n; ++d) {
            float e = x[d] - xr[d];
            q = fmaf(D.Q[d] * e, e, q);
          }
          float2 a = Af[t];
          ff_add(acc1, q);
          ff_add(acc1, fmaf(a.x, e0, a.y * e1));
        }
      }
    } else if (c + 1 < nchunks) {
      draw_chunk(c + 1, 32, nthreads - 32);
    }
    __syncthreads();
    barrier_positions<NPOS>(TCc * S * P, S, P, J, pose, shp, obs4, D.h_eps, posB, tid, nthreads);
    __syncthreads();
  }

  // ---- per-sample cost, tile weights
  if (warp == 0) {
    double Sk = __longlong_as_double(0x7ff0000000000000ll);
    const bool valid = (lane < S) && (k0 + lane < K);
    if (lane < S) {
      recur_chunk(nchunks - 1);
      const float* xr = xrf + T * n;
      float phi = 0.0f;
#pragma unroll
      for (int d = 0; d < n; ++d) {
        float e = x[d] - xr[d];
        phi = fmaf(D.Qf[d] * e, e, phi);
      }
      double s = (double)acc1.hi + (double)acc2.hi;
      s += (double)acc1.lo + (double)acc2.lo;
      s += ts.C0 + (double)phi;
      if (valid) Sk = s;
    }
    double rho_c = warp_min_d(Sk);
    float e = valid ? expf(-(float)((Sk - rho_c) * D.inv_lambda)) : 0.0f;
    double Zc = warp_sum_d((double)e);
    eS[lane] = e;
    if (valid) {
      D.costs[k0 + lane] = Sk;
      D.coll[k0 + lane] = coll ? 1 : 0;
    }
    if (lane == 0) D.part_rz[tile] = make_double2(rho_c, Zc);
  }
  __syncthreads();
  {
    float* prow = D.part + (size_t)tile * 2 * T;
    for (int t = warp; t < T; t += nwarps) {
      float e = eS[lane];
      float2 du = lane < S ? dU[t * S + lane] : make_float2(0.0f, 0.0f);
      float a = warp_sum_f(e * du.x);
      float b = warp_sum_f(e * du.y);
      if (lane == 0) reinterpret_cast<float2*>(prow)[t] = make_float2(a, b);
    }
  }

  // ---- two-level last-arriver merge: every writer fences, then one ticket
  __threadfence();
  __syncthreads();
  const int g = tile / D.GT;
  const int m0 = g * D.GT;
  const int members = min(D.GT, D.nTiles - m0);
  if (tid == 0) {
    unsigned tk = atomicAdd(&D.counters[g], 1u);
    ts.flag = (tk == (unsigned)(members - 1));
  }
  __syncthreads();
  if (!ts.flag) return;
  __threadfence();
  float* scl = reinterpret_cast<float*>(smem + L.scl);
  float* col_hi = reinterpret_cast<float*>(smem + L.colhi);
  float* col_lo = reinterpret_cast<float*>(smem + L.collo);
  double* mres = red + 100;
  const int ncol = 2 * T;
  merge_partials(members, D.part_rz + m0, D.part + (size_t)m0 * ncol, ncol, D.lambda, scl, mres,
                 mres + 1, col_hi, col_lo, red, tid, nthreads);
  for (int c = tid; c < ncol; c += nthreads) D.gpart[(size_t)g * ncol + c] = col_hi[c] + col_lo[c];
  if (tid == 0) {
    D.gpart_rz[g] = make_double2(mres[0], mres[1]);
    D.counters[g] = 0u;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    unsigned tk = atomicAdd(&D.counters[D.nGroups], 1u);
    ts.flag = (tk == (unsigned)(D.nGroups - 1));
  }
  __syncthreads();
  if (!ts.flag) return;
  __threadfence();
  merge_partials(D.nGroups, D.gpart_rz, D.gpart, ncol, D.lambda, scl, mres, mres + 1, col_hi,
                 col_lo, red, tid, nthreads);
  if (tid == 0) D.counters[D.nGroups] = 0u;
  final_stage<MODEL, NPOS>(D, smem, L, ts, mres[0], mres[1], x0g);
}

}  // namespace dbm
