// Device side of the DBaS-Log-MPPI step (arXiv 2504.06437), sm_103a.
//
// One controller's K samples are cut into tiles of S <= 32 samples; a CTA
// processes one tile (plain step: one CTA per tile; batched step: persistent
// CTAs pull (controller, tile) work items).  Per tile, for each chunk of TC
// time steps:
//   warps 1..   draw the NLN perturbations of the next chunk (Eq. 11) from
//               Philox4x32-10 with counter (k, t, iter) -- no noise crosses HBM;
//   warp 0      (lane = sample) clamps v = u + du, steps the dynamics (Eq. 1,
//               8), accumulates the stage and control costs (Eq. 9), and runs
//               the DBaS recursion (Eq. 7) of the previous chunk;
//   all warps   evaluate the fused barrier sum over every (step, sample)
//               unit, its P shape points and every obstacle (Eq. 5, 13/15):
//               each thread keeps whole units (NPOS world points) in
//               registers, streams the obstacle set from shared memory
//               (broadcast reads) and sums each unit's points exactly into a
//               float pair.
// After the horizon the tile forms its own min-shifted exponentiated weights
// and weighted perturbation sums (the numerator and denominator of Eq. 4
// relative to the tile's own minimum).  Tiles are combined by a two-level
// last-arriver reduction (atomic tickets, no spinning): the last CTA of each
// group of tiles merges the group, and the last group merger forms U*,
// runs the nominal rollout of U* for C_B (Algorithm 1), sets S_e (Eq. 10) and
// shifts the sequence.
//
// The DBaS recursion of Eq. 7, w_t = b_t + gamma (w_{t-1} - beta_d), is
// linear, so its cost sum is evaluated in unrolled form:
//   sum_{t=1..T} w_t = sum_s c_s b_s + beta_0 g1 - gamma beta_d csum,
//   c_s = (1 - gamma^(T-s+1)) / (1 - gamma),  g1 = gamma (1 - gamma^T) / (1 - gamma),
//   csum = sum_s c_s,
// which removes the rounding of the running state w; the sample-independent
// part is formed once in FP64.
//
// Precision: the rollout runs in FP32 in a frame whose origin is the
// measured position (obstacles and reference are moved into it in FP64 then
// rounded), so coordinates stay small; the per-sample cost is accumulated as
// an unevaluated float pair (TwoSum / TwoProd), the parts of the cost common
// to all samples are added in FP64, the normaliser and the tile minima are
// FP64, and the cross-tile sums of weighted perturbations are compensated
// FP32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dbm {

constexpr int kMaxShape = 8;
constexpr int kMaxN = 6;
constexpr int kStatusOk = 0;
constexpr int kStatusTimeout = 1;

// Controller state resident on the device between steps.
struct DevState {
  double S_e;        // exploration rate used by the next step
  double beta;       // barrier state of the last measured state
  double rho, Z;     // last step: global minimum cost and normaliser
  double CB_star;    // last step: barrier cost of the nominal rollout of U*
  double beta_used;  // last step: barrier state the rollouts started from
  double beta_d;     // last step: barrier summed at the goal pose
  double S_e_used;   // last step: exploration rate of the draws
  double u0[2];      // last step: u*_0
  double C0;         // sum_t gamma u_t^T (S_e Sigma)^-1 u_t of the next step
  double csum, g1;   // DBaS unrolling constants (see above)
  float L00, L10, L11, pad;  // chol(S_e Sigma) of the next step
  unsigned long long iter;  // Philox counter words 2..3
  int first;         // 1 until the first step
  int status;        // kStatus*
};

// Everything a CTA needs to process one tile of one controller.
struct CtrlDesc {
  int model, K, T, J, P, n;
  int S, TC, NPOS, nTiles, GT, nGroups;
  float dt, h_eps, gamma_bas_f, R_B, C_coll, ln_mu, ln_sigma;
  float umin[2], umax[2];
  float Q[kMaxN], Qf[kMaxN];
  float shape[2 * kMaxShape];
  float g, inv_mass, arm_over_I;
  double lambda, inv_lambda, mu_coarse, gamma_ctrl, gamma_bas, R_B_d;
  double umin_d[2], umax_d[2];
  int nscl;
  double sigma[4];
  double Lsig[3];            // chol(Sigma): l00, l10, l11
  double Sinv[4];            // gamma * Sigma^-1 (row-major; zero when gamma = 0)
  double x_goal[kMaxN];
  uint32_t key0, key1;
  double* U;                 // T x 2 nominal sequence
  float2* cU;                // T: U in FP32 for the next step
  float2* cA;                // T: gamma (S_e Sigma)^-1 u_t in FP32
  float* cw;                 // T: R_B c_{t+1}, weight of step t's barrier sum
  DevState* st;
  const double* obst;        // J x 3 (cx, cy, r), padded to 16 bytes
  const double* x0;          // n (may be overridden per launch)
  const double* xref;        // (T+1) x n
  float* part;               // nTiles x 2T tile weighted sums
  double2* part_rz;          // nTiles x (rho_c, Z_c)
  float* gpart;              // nGroups x 2T
  double2* gpart_rz;         // nGroups
  unsigned* counters;        // nGroups + 1 tickets (zero between steps)
  double* costs;             // K
  uint8_t* coll;             // K
  double* Ustar;             // T x 2
};

// Shared-memory layout of one tile; host and device compute it alike.
// region: per-chunk poses + whole-horizon perturbations + per-position
// barrier partials, reused as the raw obstacle staging buffer before the
// rollout and as the nominal-rollout buffers in the final stage.
struct SmemLayout {
  int obs4, region, dU, pose, posB, Uf, Af, red, Us, Usf, colhi, collo, scl, xrf, shp, eS, cw,
      total;
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(int T, int S, int TC, int P, int J, int n,
                                                  int nscl, int nwarps) {
  SmemLayout L;
  int off = 0;
  L.obs4 = off;
  off += 16 * (J > 0 ? J : 1);
  off = align_up(off, 16);
  L.region = off;
  int pose_b = 16 * TC * S;
  int dU_b = 8 * T * S;
  int uB_b = 8 * TC * S;
  int main_b = pose_b + dU_b + uB_b;
  int raw_b = align_up(24 * J, 16);
  int nom_b = 16 * T + 8 * T;
  int merge_b = 8 * 2 * T * nwarps;  // per-warp float-pair column sums of a merge
  int reg = main_b;
  if (raw_b > reg) reg = raw_b;
  if (nom_b > reg) reg = nom_b;
  if (merge_b > reg) reg = merge_b;
  L.pose = off;
  L.dU = off + pose_b;
  L.posB = off + pose_b + dU_b;
  off += align_up(reg, 16);
  L.red = off;
  off += 8 * 4 * 32;
  L.Us = off;
  off += 16 * T;
  L.Usf = off;
  off += 8 * T;
  L.Uf = off;
  off += 8 * T;
  L.Af = off;
  off += 8 * T;
  L.colhi = off;
  off += 8 * T;
  L.collo = off;
  off += 8 * T;
  L.scl = off;
  off += 4 * (nscl > 32 ? nscl : 32);
  L.xrf = off;
  off += 4 * (T + 1) * n;
  off = align_up(off, 8);
  L.shp = off;
  off += 8 * kMaxShape;
  L.eS = off;
  off += 4 * 32;
  L.cw = off;
  off += 4 * T;
  L.total = align_up(off, 16);
  return L;
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 from the published description (Salmon et al., SC'11):
// ten rounds of two 32x32->64 multiplies with the key bumped by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a0 = 0xD2511F53u, a1 = 0xCD9E8D57u;
    uint32_t hi0 = __umulhi(a0, c.x), lo0 = a0 * c.x;
    uint32_t hi1 = __umulhi(a1, c.z), lo1 = a1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Top 23 bits of r as an odd multiple of 2^-24: exactly representable.
__device__ __forceinline__ float unit_open(uint32_t r) {
  return __uint2float_rn((r >> 8) | 1u) * 5.9604644775390625e-8f;
}

// One NLN perturbation (Eq. 11): (chol(S_e Sigma) z_n) .* exp(mu + sigma z_ln).
__device__ __forceinline__ float2 nln_draw(uint4 r, float L00, float L10, float L11,
                                           float ln_mu, float ln_sigma) {
  float u0 = unit_open(r.x), u1 = unit_open(r.y), u2 = unit_open(r.z), u3 = unit_open(r.w);
  float ra = sqrtf(-2.0f * logf(u0));
  float sa, ca;
  sincospif(2.0f * u1, &sa, &ca);
  float rb = sqrtf(-2.0f * logf(u2));
  float sb, cb;
  sincospif(2.0f * u3, &sb, &cb);
  float zn0 = ra * ca, zn1 = ra * sa;
  float g0 = expf(ln_mu + ln_sigma * (rb * cb));
  float g1 = expf(ln_mu + ln_sigma * (rb * sb));
  return make_float2(L00 * zn0 * g0, (L10 * zn0 + L11 * zn1) * g1);
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Unevaluated float pair accumulated with Knuth's TwoSum.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ void ff_add(FF& a, float x) {
  float s = __fadd_rn(a.hi, x);
  float bp = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, e);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------ mbarrier / TMA
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Bulk (non-tensor) TMA copy global -> shared, completion on the mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                             uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bounded wait on an mbarrier phase; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int max_polls) {
  uint32_t a = smem_u32(bar);
  for (int i = 0; i < max_polls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// ------------------------------------------------------------------ dynamics
// State in registers; (cs, sn) are cos/sin of the current heading and are
// refreshed to the new heading by each step (they also place the shape points).
template <int MODEL>
struct Dyn;

template <>
struct Dyn<0> {  // unicycle (x, y, theta), u = (v, omega)
  static constexpr int n = 3;
  __device__ __forceinline__ static void step(float* x, float& cs, float& sn, float v0, float v1,
                                              const CtrlDesc& D) {
    float vdt = v0 * D.dt;
    x[0] = fmaf(vdt, cs, x[0]);
    x[1] = fmaf(vdt, sn, x[1]);
    x[2] = fmaf(v1, D.dt, x[2]);
    sincosf(x[2], &sn, &cs);
  }
};

template <>
struct Dyn<1> {  // planar quadrotor (y, z, phi, ydot, zdot, phidot), u = thrust deviations
  static constexpr int n = 6;
  __device__ __forceinline__ static void step(float* x, float& cs, float& sn, float v0, float v1,
                                              const CtrlDesc& D) {
    float dt = D.dt;
    float acc = fmaf(v0 + v1, D.inv_mass, D.g);  // (F1 + F2) / m
    float y = fmaf(x[3], dt, x[0]);
    float z = fmaf(x[4], dt, x[1]);
    float ph = fmaf(x[5], dt, x[2]);
    float vy = fmaf(-acc * sn, dt, x[3]);
    float vz = fmaf(fmaf(acc, cs, -D.g), dt, x[4]);
    float w = fmaf((v1 - v0) * D.arm_over_I, dt, x[5]);
    x[0] = y;
    x[1] = z;
    x[2] = ph;
    x[3] = vy;
    x[4] = vz;
    x[5] = w;
    sincosf(ph, &sn, &cs);
  }
};

// ------------------------------------------------------------ tile kernel body
struct TileScratch {
  uint64_t mbar;
  int flag;
  double beta0, beta_d, Kconst;
};

// Fused barrier over nunits (step, sample) units; unit u has pose pose[u]
// and P shape points shp[0..P).  Each thread takes NPOS / P whole units at a
// time (NPOS >= P), keeps their world points in registers and streams every
// obstacle: h = |p - c|^2 - r^2 evaluated as fma(dx, dx, fma(dy, dy, -r^2)),
// term 1 / max(h, h_eps) by the approximate reciprocal.  A unit's points are
// summed exactly (TwoSum) into (hi, lo); the sign bit of hi marks a unit in
// which some h <= 0 (collision).
template <int NPOS>
__device__ __forceinline__ void barrier_units(int nunits, int P, int J,
                                              const float4* __restrict__ pose,
                                              const float2* __restrict__ shp,
                                              const float4* __restrict__ obs4, float h_eps,
                                              float2* __restrict__ uB, int tid, int nthreads) {
  const int upt = NPOS / P;  // units per thread per round
  const int used = upt * P;
  for (int ub = tid * upt; ub < nunits; ub += nthreads * upt) {
    float X[NPOS], Y[NPOS], acc[NPOS], mn[NPOS];
    int uu = 0, p = 0;
#pragma unroll
    for (int i = 0; i < NPOS; ++i) {
      const int u = ub + uu;
      const bool ok = (i < used) && (u < nunits);
      const float4 ps = pose[ok ? u : ub];
      const float2 sh = shp[ok ? p : 0];
      X[i] = fmaf(ps.z, sh.x, fmaf(-ps.w, sh.y, ps.x));
      Y[i] = fmaf(ps.w, sh.x, fmaf(ps.z, sh.y, ps.y));
      acc[i] = 0.0f;
      mn[i] = __int_as_float(0x7f800000);
      if (++p == P) {
        p = 0;
        ++uu;
      }
    }
    for (int j = 0; j < J; ++j) {
      const float4 o = obs4[j];
#pragma unroll
      for (int i = 0; i < NPOS; ++i) {
        float dx = X[i] - o.x;
        float dy = Y[i] - o.y;
        float h = fmaf(dx, dx, fmaf(dy, dy, o.z));
        mn[i] = fminf(mn[i], h);
        acc[i] += rcp_approx(fmaxf(h, h_eps));
      }
    }
    FF f = {0.0f, 0.0f};
    bool coll = false;
    uu = 0;
    p = 0;
#pragma unroll
    for (int i = 0; i < NPOS; ++i) {
      if (i < used) {
        ff_add(f, acc[i]);
        coll |= (mn[i] <= 0.0f);
        if (++p == P) {
          const int u = ub + uu;
          if (u < nunits) uB[u] = make_float2(coll ? -f.hi : f.hi, f.lo);
          f.hi = 0.0f;
          f.lo = 0.0f;
          coll = false;
          p = 0;
          ++uu;
        }
      }
    }
  }
}

// Two float pairs added exactly up to the final rounding of the low part.
__device__ __forceinline__ FF ff_sum(FF a, FF b) {
  FF r = a;
  ff_add(r, b.hi);
  r.lo += b.lo;
  return r;
}

// Merge n partial results (rho_i, Z_i, cols_i[ncol]) taken relative to their
// own minima into one relative to the common minimum: the log-sum-exp merge
// of Eq. 4's numerator and denominator.  Warp w takes sources w, w + nwarps,
// ...; lane l takes columns l, l + 32, ... (ncol <= 32 * kMaxColsPerLane), so
// every load instruction reads a contiguous row segment and many rows are in
// flight at once; the per-warp float-pair sums are then added in warp order.
// All threads of the CTA call it.  buf: nwarps x ncol float pairs.
// Outputs in shared memory: *rho_out, *Z_out, col_hi/col_lo[ncol].
constexpr int kMaxColsPerLane = 16;  // 2 T <= 512
__device__ inline void merge_partials(int n, const double2* rz, const float* cols, int ncol,
                                      double inv_lambda, float* scl, double* rho_out,
                                      double* Z_out, float* col_hi, float* col_lo, FF* buf,
                                      double* red, int tid, int nthreads) {
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
  if (warp == 0) {
    double r = __longlong_as_double(0x7ff0000000000000ll);
    for (int i = lane; i < n; i += 32) r = fmin(r, __ldcg(&rz[i].x));
    r = warp_min_d(r);
    double z = 0.0;
    for (int i = lane; i < n; i += 32) {
      double2 v = __ldcg(&rz[i]);
      float s = expf(-(float)((v.x - r) * inv_lambda));
      scl[i] = s;
      z += v.y * (double)s;
    }
    z = warp_sum_d(z);
    if (lane == 0) {
      *rho_out = r;
      *Z_out = z;
    }
  }
  __syncthreads();
  FF acc[kMaxColsPerLane];
#pragma unroll
  for (int j = 0; j < kMaxColsPerLane; ++j) acc[j].hi = acc[j].lo = 0.0f;
  const int nj = (ncol + 31) / 32;
  for (int i = warp; i < n; i += nwarps) {
    const float s = scl[i];
    const float* row = cols + (size_t)i * ncol;
    float v[kMaxColsPerLane];
#pragma unroll
    for (int j = 0; j < kMaxColsPerLane; ++j) {
      int c = lane + 32 * j;
      v[j] = (j < nj && c < ncol) ? __ldcg(row + c) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < kMaxColsPerLane; ++j)
      if (j < nj) ff_add(acc[j], v[j] * s);
  }
#pragma unroll
  for (int j = 0; j < kMaxColsPerLane; ++j) {
    int c = lane + 32 * j;
    if (j < nj && c < ncol) buf[warp * ncol + c] = acc[j];
  }
  __syncthreads();
  for (int c = tid; c < ncol; c += nthreads) {
    FF a = buf[c];
    for (int w = 1; w < nwarps; ++w) a = ff_sum(a, buf[w * ncol + c]);
    col_hi[c] = a.hi;
    col_lo[c] = a.lo;
  }
  (void)red;
  __syncthreads();
}

}  // namespace dbm
