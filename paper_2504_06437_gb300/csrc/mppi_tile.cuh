// Tile body and final stage of the DBaS-Log-MPPI step; shared by the plain
// one-launch-per-controller kernel and the batched persistent kernel.
#pragma once

#include "mppi_device.cuh"

namespace dbm {

constexpr int kTmaPolls = 1 << 22;

// Obstacle staging: 1 = bulk TMA copy into shared memory (mbarrier
// completion), 0 = coalesced loads by all threads.
#ifndef DBM_STAGE_TMA
#define DBM_STAGE_TMA 1
#endif

// TwoProd: c * b = ph + pe exactly, added to the float pair.
__device__ __forceinline__ void ff_add_prod(FF& a, float c, float bh, float bl) {
  float ph = c * bh;
  float pe = fmaf(c, bh, -ph);
  ff_add(a, ph);
  a.lo += fmaf(c, bl, pe);
}

// Constants of the controller that never change: the unrolled DBaS weights
// c_s (scaled by R_B) and their sums.  One CTA, at creation.
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
}

// Per-step constants that depend only on the controller state (U, S_e):
// chol(S_e Sigma) = sqrt(S_e) chol(Sigma), a_t = gamma (S_e Sigma)^-1 u_t
// = (gamma Sigma^-1 / S_e) u_t, u_t in FP32, and C0 = sum_t u_t . a_t, the
// part of the control cost of Eq. 9 (Algorithm 1 form
// gamma u^T (S_e Sigma)^-1 v) that every sample shares.  Run by one CTA after
// each shift, and by a one-CTA kernel after the host sets the state.
// red: >= 32 doubles of shared memory.
__device__ inline void prep_constants(const CtrlDesc& D, double* red, int tid, int nthreads) {
  DevState* st = D.st;
  const int T = D.T;
  __syncthreads();
  const double Se = st->S_e;
  const double inv_Se = 1.0 / Se;
  if (tid == 0) {
    const double r = sqrt(Se);
    st->L00 = (float)(r * D.Lsig[0]);
    st->L10 = (float)(r * D.Lsig[1]);
    st->L11 = (float)(r * D.Lsig[2]);
  }
  const double M00 = D.Sinv[0] * inv_Se, M01 = D.Sinv[1] * inv_Se;
  const double M10 = D.Sinv[2] * inv_Se, M11 = D.Sinv[3] * inv_Se;
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

// Barrier-state cost of one trajectory from its unit sums uB[0..T): the
// sample-dependent part sum_s R_B c_s b_s, spread over the lanes of one warp
// (all lanes call it), plus the FP64 constant.
__device__ __forceinline__ double dbas_cost_warp(const float2* uB, const float* cw, int T,
                                                 double Kconst, int lane) {
  FF a = {0.0f, 0.0f};
  for (int t = lane; t < T; t += 32) {
    float2 v = uB[t];
    ff_add_prod(a, cw[t], fabsf(v.x), v.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF b;
    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
    b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
    a = ff_sum(a, b);
  }
  return (double)a.hi + (double)a.lo + Kconst;
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
  float2* Usf = reinterpret_cast<float2*>(smem + L.Usf);
  const float* col_hi = reinterpret_cast<const float*>(smem + L.colhi);
  const float* col_lo = reinterpret_cast<const float*>(smem + L.collo);
  float4* pose_nom = reinterpret_cast<float4*>(smem + L.region);
  float2* uB_nom = reinterpret_cast<float2*>(smem + L.region + 16 * T);
  const float2* shp = reinterpret_cast<const float2*>(smem + L.shp);
  const float4* obs4 = reinterpret_cast<const float4*>(smem + L.obs4);
  const float* cw = reinterpret_cast<const float*>(smem + L.cw);
  const double invZ = 1.0 / Z;
  for (int c = tid; c < 2 * T; c += nthreads) {
    int d = c & 1;
    double du = ((double)col_hi[c] + (double)col_lo[c]) * invZ;
    double u = D.U[c] + du;
    u = fmin(fmax(u, D.umin_d[d]), D.umax_d[d]);
    Us[c] = u;
    reinterpret_cast<float*>(Usf)[c] = (float)u;
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
      const float2 u = Usf[t];
      Dyn<MODEL>::step(x, cs, sn, u.x, u.y, D);
      pose_nom[t] = make_float4(x[0], x[1], cs, sn);
    }
  }
  __syncthreads();
  barrier_units<NPOS>(T, P, D.J, pose_nom, shp, obs4, D.h_eps, uB_nom, tid, nthreads);
  __syncthreads();
  if (tid < 32) {
    const double CB = dbas_cost_warp(uB_nom, cw, T, ts.Kconst, tid);
    if (tid == 0) {
      DevState* st = D.st;
      const double S_e_used = st->S_e;
      // Eq. 10, C_B floored at 0 inside the logarithm
      const float arg = (float)(2.718281828459045 + fmax(CB, 0.0));
      const double S_e_next = D.mu_coarse > 0.0 ? D.mu_coarse * (double)logf(arg) : 1.0;
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
  }
  // shift (Algorithm 1, last loop): u_{t-1} <- u*_t, the last entry kept
  for (int c = tid; c < 2 * T; c += nthreads) {
    int t = c >> 1, d = c & 1;
    D.U[c] = (t + 1 < T) ? Us[2 * (t + 1) + d] : Us[2 * (T - 1) + d];
  }
  __threadfence_block();
  prep_constants(D, reinterpret_cast<double*>(smem + L.red), tid, nthreads);
}

// One tile of one controller.  ts.mbar must be initialised; mbar_phase is
// each thread's own copy of the parity of the barrier's next completion.
template <int MODEL, int NPOS>
__device__ void run_tile(const CtrlDesc& D, int tile, const double* __restrict__ x0g,
                         const double* __restrict__ xrefg, char* smem, TileScratch& ts,
                         uint32_t& mbar_phase) {
  constexpr int n = Dyn<MODEL>::n;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
  const int T = D.T, S = D.S, P = D.P, J = D.J, TC = D.TC, K = D.K;
  const SmemLayout L = smem_layout(T, S, TC, P, J, n, D.nscl, nwarps);
  float4* obs4 = reinterpret_cast<float4*>(smem + L.obs4);
  float4* pose = reinterpret_cast<float4*>(smem + L.pose);
  float2* dU = reinterpret_cast<float2*>(smem + L.dU);
  float2* uB = reinterpret_cast<float2*>(smem + L.posB);
  float2* Uf = reinterpret_cast<float2*>(smem + L.Uf);
  float2* Af = reinterpret_cast<float2*>(smem + L.Af);
  float* xrf = reinterpret_cast<float*>(smem + L.xrf);
  float2* shp = reinterpret_cast<float2*>(smem + L.shp);
  float* eS = reinterpret_cast<float*>(smem + L.eS);
  float* cw = reinterpret_cast<float*>(smem + L.cw);
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
  const double ox = x0g[0], oy = x0g[1];
  for (int t = tid; t < T; t += nthreads) {
    Uf[t] = D.cU[t];
    Af[t] = D.cA[t];
    cw[t] = D.cw[t];
  }
  for (int i = tid; i < (T + 1) * n; i += nthreads) {
    int d = i % n;
    double v = xrefg[i];
    if (d == 0) v -= ox;
    if (d == 1) v -= oy;
    xrf[i] = (float)v;
  }
  if (J > 0) {
#if DBM_STAGE_TMA
    bool ok = mbar_wait(&ts.mbar, mbar_phase, kTmaPolls);
    if (!ok) {
      if (tid == 0) atomicExch(&st->status, kStatusTimeout);
      mbar_wait(&ts.mbar, mbar_phase, kTmaPolls);
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
    double beta0 = st->first ? sb0 : sb0 + D.gamma_bas * (st->beta - sbd);
    ts.beta_d = sbd;
    ts.beta0 = beta0;
    // sample-independent part of sum_t R_B w_t (unrolled Eq. 7)
    ts.Kconst = D.R_B_d * (beta0 * st->g1 - D.gamma_bas * sbd * st->csum);
  }
  __syncthreads();

  // ---- rollout over chunks
  float x[n];
  float cs = 1.0f, sn = 0.0f;
  FF acc1 = {0.0f, 0.0f}, acc2 = {0.0f, 0.0f};
  bool coll = false;
  if (warp == 0) {
    x[0] = 0.0f;
    x[1] = 0.0f;
#pragma unroll
    for (int d = 2; d < n; ++d) x[d] = (float)x0g[d];
    sincosf(x[2], &sn, &cs);
  }
  // barrier-state and collision costs of chunk c from its unit sums
  auto recur_chunk = [&](int c) {
    int t0 = c * TC;
    int TCc = min(TC, T - t0);
    for (int tl = 0; tl < TCc; ++tl) {
      float2 v = uB[tl * S + lane];
      bool cl = __float_as_int(v.x) < 0;
      ff_add_prod(acc2, cw[t0 + tl], fabsf(v.x), v.y);
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
    barrier_units<NPOS>(TCc * S, P, J, pose, shp, obs4, D.h_eps, uB, tid, nthreads);
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
      s += st->C0 + ts.Kconst + (double)phi;
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
    if (lane == 0) {
      D.part_rz[tile] = make_double2(rho_c, Zc);
      __threadfence();
    }
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
    if (lane == 0) __threadfence();  // the writers of the tile's partials
  }

  // ---- two-level last-arriver merge: the writers fenced, then one ticket
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
  FF* mbuf = reinterpret_cast<FF*>(smem + L.region);
  double* mres = red + 100;
  const int ncol = 2 * T;
  merge_partials(members, D.part_rz + m0, D.part + (size_t)m0 * ncol, ncol, D.inv_lambda, scl,
                 mres, mres + 1, col_hi, col_lo, mbuf, red, tid, nthreads);
  bool wrote = false;
  for (int c = tid; c < ncol; c += nthreads) {
    D.gpart[(size_t)g * ncol + c] = col_hi[c] + col_lo[c];
    wrote = true;
  }
  if (tid == 0) {
    D.gpart_rz[g] = make_double2(mres[0], mres[1]);
    D.counters[g] = 0u;
    wrote = true;
  }
  if (wrote) __threadfence();
  __syncthreads();
  if (tid == 0) {
    unsigned tk = atomicAdd(&D.counters[D.nGroups], 1u);
    ts.flag = (tk == (unsigned)(D.nGroups - 1));
  }
  __syncthreads();
  if (!ts.flag) return;
  __threadfence();
  merge_partials(D.nGroups, D.gpart_rz, D.gpart, ncol, D.inv_lambda, scl, mres, mres + 1, col_hi,
                 col_lo, mbuf, red, tid, nthreads);
  if (tid == 0) D.counters[D.nGroups] = 0u;
  final_stage<MODEL, NPOS>(D, smem, L, ts, mres[0], mres[1], x0g);
}

}  // namespace dbm
