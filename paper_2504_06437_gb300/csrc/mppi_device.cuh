// Device side of the DBaS-Log-MPPI step (arXiv 2504.06437), sm_103a.
//
// One controller's K samples are cut into tiles of S <= 32 samples; a CTA
// processes one tile (plain step: one CTA per tile; batched step: persistent
// CTAs pull (controller, tile) work items).  Per tile:
//   noise      all threads draw the NLN perturbations of every (sample, step)
//              (Eq. 11) from Philox4x32-10 with counter (k, t, iter) -- no
//              noise crosses HBM -- and keep the clamped controls v = u + du;
//   dynamics   one warp per sample, lanes over steps: explicit Euler for both
//              models is triangular (heading rate -> heading -> velocities
//              -> positions), so a whole trajectory is a few warp prefix
//              scans over time, segment by segment, with one sincos per step;
//              the warp also sums the stage and control costs (Eq. 9);
//   barrier    all threads evaluate the fused barrier sum over every
//              (step, sample) unit, its P shape points and every obstacle
//              (Eq. 5, 13/15): each thread keeps whole units (NPOS world
//              points) in registers as packed pairs, streams the obstacle
//              set from shared memory (broadcast reads), evaluates two points
//              per packed two-lane FP32 instruction, adds two obstacles per
//              approximate reciprocal, and sums each unit's points exactly
//              into a float pair, written over the unit's pose;
//   costs      one warp per sample adds the barrier-state and collision costs;
//   partials   the tile's minimum cost, its exponentiated weights, their sum Z
//              and the 2T weighted column sums of the perturbations (Eq. 4);
//   merge      the last tile to finish (a ticket per group of tiles) merges
//              the partials log-sum-exp style against the exact minimum over
//              the tiles, then runs the final stage (U*, nominal rollout, S_e,
//              shift).
// The one-controller kernels exist in a 96- and an 80-register form (the
// host picks per launch); the batch kernel's tiles take a padded row stride
// and the one-batch merge (BATCHED in run_tile).  All forms give the same
// results bit for bit.
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
// rounded), so coordinates stay small; the per-sample cost is an unevaluated
// float pair (TwoSum / TwoProd) relative to a base, the part of the cost
// common to all samples, formed in FP64; the minima, the normaliser Z and the
// weighted sums of perturbations are float pairs, merged across tiles with
// float-pair arithmetic; U* is formed in FP64 from them.
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
  double x1[6];      // last step: state after applying u*_0 (model prediction)
  double C0;         // sum_t gamma u_t^T (S_e Sigma)^-1 u_t of the next step
  double csum, g1;   // DBaS unrolling constants (see above)
  float L00, L10, L11, pad;  // chol(S_e Sigma) of the next step
  unsigned long long iter;  // Philox counter words 2..3
  int first;         // 1 until the first step
  int status;        // kStatus*
  // grid map, set by the host (mppi_set_grid) and read by the grid form of
  // the step kernels: signed distances (m), sample (i, j) at
  // (grid_ox + i res, grid_oy + j res), stored at grid[j grid_nx + i]; or null
  const float* grid;
  int grid_nx, grid_ny;
  double grid_ox, grid_oy, grid_res;
  float grid_inv_res, grid_pad;
};

// Outputs of a step that the host reads after every step, written by the
// final stage straight into mapped pinned host memory (one-controller
// contexts; null elsewhere).  seq is stored last, after a system-scope
// fence, so a host that sees the step's seq also sees its u0 and status.
struct HostOut {
  double u0[2];  // u*_0
  int status;    // kStatus*
  int seq;       // low 32 bits of the step's iteration counter + 1
};

// Everything a CTA needs to process one tile of one controller.
struct CtrlDesc {
  int model, K, T, J, P, n;
  int S, NPOS, nTiles, GT, nGroups;
  float dt, h_eps, gamma_bas_f, R_B, C_coll, ln_mu, ln_sigma;
  float umin[2], umax[2];
  float Q[kMaxN], Qf[kMaxN];
  float shape[2 * kMaxShape];
  float g, inv_mass;
  float k_turn;              // arm / I (6-state quadrotor) or 1 / wheelbase (Ackermann)
  float inv_lambda_f;
  double lambda, inv_lambda, mu_coarse, gamma_ctrl, gamma_bas, R_B_d;
  double umin_d[2], umax_d[2];
  int nscl;
  int sgf_wp;                // Savitzky-Golay window | order << 8, 0 = off (weights: cw)
  double sigma[4];
  double Lsig[3];            // chol(Sigma): l00, l10, l11
  double Sinv[4];            // gamma * Sigma^-1 (row-major; zero when gamma = 0)
  double x_goal[kMaxN];
  uint32_t key0, key1;
  double* U;                 // T x 2 nominal sequence
  float2* cU;                // T: U in FP32 for the next step
  float2* cA;                // T: gamma Sigma^-1 u_t in FP32 (divided by S_e where used)
  float* cw;                 // T: R_B c_{t+1}, weight of step t's barrier sum (then the
                             // smoothing weights, see sgf_table_offset)
  DevState* st;
  const double* obst;        // J x 3 (cx, cy, r), padded to 16 bytes
  const double* x0;          // n (may be overridden per launch)
  const double* xref;        // (T+1) x n
  float* part;               // nTiles x 2T tile weighted sums
  float4* part_rz;           // nTiles x (rho_c hi, lo, Z_c hi, lo), rho relative to base
  float* gpart;              // nGroups x 2T
  float4* gpart_rz;          // nGroups
  unsigned* counters;        // 2 (nGroups + 1): tickets, then minimum words (zero between steps)
  double* costs;             // K
  uint8_t* coll;             // K
  double* Ustar;             // T x 2
  HostOut* host_out;         // device alias of the host mirror, or null
};

// The Savitzky-Golay weights (W x W floats, row q: the fit's value at window
// position q) follow the T barrier weights cw at the next 16-byte boundary
// of the same buffer, when the controller smooths its update.
__host__ __device__ inline int sgf_table_offset(int T) { return (T + 3) & ~3; }

// Shared-memory layout of one tile; host and device compute it alike.
// region: poses (overwritten in place by the unit barrier sums) and clamped
// controls of the whole horizon; reused as the raw obstacle staging buffer
// before the rollout, as the per-warp column sums of a merge and as the
// nominal-rollout buffers in the final stage.
struct SmemLayout {
  int obs4, region, pose, V, red, Us, Usf, Uf, Af, colhi, collo, scl, xrf, shp, eS, cw, Sk, scH,
      scL, collf, xi, total;
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Tile merge geometry (merge_partials): row groups over the CTA's threads
// and the bytes of their float-pair column sums.
constexpr int kMergeLoads = 16;   // float2 loads in flight per thread
constexpr int kMergeGroups = 32;  // row groups at most
__host__ __device__ inline int merge_row_groups(int ncol, int nthreads) {
  const int ncp = ncol / 2;
  int rg = ncp > 0 ? nthreads / ncp : nthreads;
  if (rg < 1) rg = 1;
  if (rg > kMergeGroups) rg = kMergeGroups;
  return rg;
}
__host__ __device__ inline int merge_buf_bytes(int ncol, int nthreads) {
  return align_up(8 * merge_row_groups(ncol, nthreads) * (ncol + 1), 16);  // + Z
}

// Row stride of the tile's (step, sample) arrays (poses, clamped controls,
// unit sums): element (t, s) sits at t SP + s.  The rollout scans and the
// per-sample cost loops step through a sample's row with lanes on
// consecutive t, so an even S folds the lanes' float4 and float2 accesses
// onto a few banks (S = 32: all onto one).  The persistent batch kernel
// rounds SP up to an odd number, which spreads them (a 64-controller mix
// at S = 32: 3.31 -> 3.00 ms); the one-controller kernels keep SP = S,
// which measured faster there (their autotuned S avoid the worst strides).
__host__ __device__ inline int row_stride(int S, bool batched) { return batched ? (S | 1) : S; }

__host__ __device__ inline SmemLayout smem_layout(int T, int S, int P, int J, int n, int nscl,
                                                  int nwarps, bool batched) {
  SmemLayout L;
  int off = 0;
  L.obs4 = off;
  off += 16 * (J > 0 ? J : 1);
  off = align_up(off, 16);
  L.region = off;
  const int SP = row_stride(S, batched);
  int main_b = 16 * T * SP + 8 * T * SP;
  int raw_b = align_up(24 * J, 16);
  int nom_b = 16 * T + 4 * T * P;
  int merge_b = merge_buf_bytes(2 * T, 32 * nwarps) + 8 * (nscl > 1 ? nscl : 1);
  int reg = main_b;
  if (raw_b > reg) reg = raw_b;
  if (nom_b > reg) reg = nom_b;
  if (merge_b > reg) reg = merge_b;
  L.pose = off;
  L.V = off + 16 * T * SP;
  off += align_up(reg, 16);
  L.red = off;
  off += 8 * 4 * 32;
  L.Us = off;
  off += 16 * T;
  L.Sk = off;
  off += 8 * 32;
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
  L.scH = off;
  off += 4 * 32;
  L.scL = off;
  off += 4 * 32;
  L.xi = off;
  off += 4 * kMaxN;
  L.collf = off;
  off += 32;
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

// Square root by the approximate instruction (relative error about one ulp).
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One NLN perturbation (Eq. 11): (chol(S_e Sigma) z_n) .* exp(mu + sigma z_ln).
// Box-Muller radii sqrt(-2 ln u) with u >= 2^-24 and 1 - u >= 2^-24, so the
// argument of the square root is at least 1.1e-7; the log-normal factor's
// exponent is bounded by |mu| + 5.8 sigma, where the intrinsic exponential is
// within a few ulp.
__device__ __forceinline__ float2 nln_draw(uint4 r, float L00, float L10, float L11,
                                           float ln_mu, float ln_sigma) {
  float u0 = unit_open(r.x), u1 = unit_open(r.y), u2 = unit_open(r.z), u3 = unit_open(r.w);
  float ra = sqrt_approx(-2.0f * logf(u0));
  float sa, ca;
  sincospif(2.0f * u1, &sa, &ca);
  float rb = sqrt_approx(-2.0f * logf(u2));
  float sb, cb;
  sincospif(2.0f * u3, &sb, &cb);
  float zn0 = ra * ca, zn1 = ra * sa;
  float g0 = __expf(ln_mu + ln_sigma * (rb * cb));
  float g1 = __expf(ln_mu + ln_sigma * (rb * sb));
  return make_float2(L00 * zn0 * g0, (L10 * zn0 + L11 * zn1) * g1);
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// min(a, b, c) in one instruction (three-input PTX min, sm_100 and later);
// exact, as min(min(a, b), c).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float y;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
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

// TwoProd: c * (bh + bl) = ph + pe (+ c bl) added to the float pair.
__device__ __forceinline__ void ff_add_prod(FF& a, float c, float bh, float bl) {
  float ph = c * bh;
  float pe = fmaf(c, bh, -ph);
  ff_add(a, ph);
  a.lo += fmaf(c, bl, pe);
}

// Renormalise a float pair so that |lo| <= ulp(hi) / 2 (Fast2Sum).
__device__ __forceinline__ FF ff_norm(FF a) {
  const float s = __fadd_rn(a.hi, a.lo);
  return FF{s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}
// Lexicographic order of normalised float pairs = order of their values.
__device__ __forceinline__ bool ff_less(FF a, FF b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
// (a - b) rounded to float, for normalised pairs a >= b.
__device__ __forceinline__ float ff_diff(FF a, FF b) {
  return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}
__device__ __forceinline__ FF warp_min_ff(FF a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF b;
    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
    b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
    if (ff_less(b, a)) a = b;
  }
  return a;
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
// One arrival on an mbarrier (no transaction bytes).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait on an mbarrier phase: at most max_polls tries and max_cycles
// SM clock cycles (a try may suspend the thread for a while); false if a
// bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int max_polls,
                                          long long max_cycles) {
  uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (int i = 0; i < max_polls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > max_cycles) break;
  }
  return false;
}

// ------------------------------------------------------------------ dynamics
// State dimension of each model (the Euler steps themselves are evaluated in
// scan form, see scan_trajectory).
// Models: 0 unicycle, 1 planar quadrotor (6 states, two thrusts), 2 Ackermann
// vehicle (Eq. 14), 3 the paper's planar quadrotor (5 states, Eq. 12).
template <int MODEL>
struct Dyn {
  static constexpr int n = MODEL == 0 ? 3 : MODEL == 1 ? 6 : MODEL == 2 ? 4 : 5;
};

// ------------------------------------------------------------ tile kernel body
struct TileScratch {
  uint64_t mbar;
  int flag;
  double beta0, beta_d, Kconst, base;  // base = C0 + Kconst
  FF rho, Z;                           // merge results
  float ref;                           // common reference of a merge (minimum of the sources' rho)
  double S_e_used, S_e_next;           // exploration rate of this step and the next
  unsigned long long iter;             // iteration counter of this step
  double x0[2];                        // measured position: origin of the tile's frame
};

// The grid map as a tile reads it.  The tile's frame is centred on the
// measured position x0, whose grid coordinates are split (in FP64) into the
// integer cell (ci, cj) and the remainder (ru, rv) in [0, 1): a point X of
// the tile's frame has grid coordinate ci + (ru + X / res), and the FP32
// part stays small, so its rounding is that of a few cells, not of the
// whole map.
struct GridView {
  const float* g;
  int nx, ny, ci, cj;
  float ru, rv, inv_res;
};

// One axis of the lookup: cell index in [0, n - 2] and weight in [0, 1] of
// grid coordinate c + l, with the coordinate clamped to [0, n - 1] first.
// The first clamp bounds l to just beyond the map (fminf / fmaxf return the
// number when the other operand is NaN), so the index is finite for any
// input.
__device__ __forceinline__ int grid_axis(int c, float l, int n, float& f) {
  l = fminf(fmaxf(l, (float)(-1 - c)), (float)(n - c));
  const float fl = floorf(l);
  int i = c + (int)fl;
  f = l - fl;
  if (i < 0) {
    i = 0;
    f = 0.0f;
  } else if (i >= n - 1) {
    i = n - 2;
    f = 1.0f;
  }
  return i;
}

// The grid map's h at a point of the tile's frame (Sec. V-C grid map):
// bilinear interpolation of the four samples around it, the grid
// coordinates first clamped to [0, nx - 1] x [0, ny - 1]; nx, ny >= 2.
__device__ __forceinline__ float grid_h(const GridView& gv, float X, float Y) {
  float fx, fy;
  const int i = grid_axis(gv.ci, fmaf(X, gv.inv_res, gv.ru), gv.nx, fx);
  const int j = grid_axis(gv.cj, fmaf(Y, gv.inv_res, gv.rv), gv.ny, fy);
  const float* r0 = gv.g + (size_t)j * gv.nx + i;
  const float* r1 = r0 + gv.nx;
  const float g00 = __ldg(r0), g10 = __ldg(r0 + 1), g01 = __ldg(r1), g11 = __ldg(r1 + 1);
  const float a = fmaf(fx, g10 - g00, g00), b = fmaf(fx, g11 - g01, g01);
  return fmaf(fy, b - a, a);
}

// Fused barrier over nunits = T S (step, sample) units; unit u = t S + s has
// its pose at pose[t SP + s] (SP = row_stride(S, BATCHED)) and P shape
// points shp[0..P).  Each thread takes NPOS / P whole units at a
// time (NPOS >= P), units base + k nthreads + tid (k < NPOS / P) so that
// neighbouring lanes read neighbouring poses, keeps their world points in
// registers and streams every
// obstacle: h = |p - c|^2 - r^2 evaluated as fma(dx, dx, fma(dy, dy, -r^2)),
// terms 1 / max(h, h_eps) added two obstacles at a time as (h1 + h2) / (h1 h2)
// with the approximate reciprocal.  The points are held in packed pairs and
// the subtractions, fmas, sums and products are packed two-lane FP32
// instructions (each lane the same round-to-nearest operation as the scalar
// one, so the results are the scalar loop's bit for bit): one issue slot
// for two points, where the loop is bound by instruction issue.  A unit's
// points are summed exactly (TwoSum) into (hi, lo), stored at
// uB[u * ustride]; the sign bit of hi marks a unit in which some h <= 0
// (collision).  A thread reads the poses of its units before it writes their
// sums, so uB may overlay pose.  GRID: each point also adds the grid map's
// term (grid_h) and counts its h in the collision test.
template <int NPOS, bool BATCHED, bool GRID = false>
__device__ __forceinline__ void barrier_units(int nunits, int S, int P, int J, const float4* pose,
                                              const float2* __restrict__ shp,
                                              const float4* __restrict__ obs4, float h_eps,
                                              float2* uB, int ustride, int tid, int nthreads,
                                              const GridView* gv = nullptr) {
  // unit u = t S + s lives at t SP + s = u + (SP - S) floor(u / S); the
  // quotient by one multiply-high with m = ceil(2^32 / S), exact while
  // u (m S - 2^32) < 2^32 (here u < T S <= 2^13 and m S - 2^32 < S <= 32)
  const unsigned pad = (unsigned)(row_stride(S, BATCHED) - S);
  const unsigned mS = pad ? 0xffffffffu / (unsigned)S + 1u : 0u;
  auto at = [&](int u) {
    if constexpr (BATCHED) return (int)((unsigned)u + pad * __umulhi((unsigned)u, mS));
    else return u;
  };
  static_assert(NPOS % 2 == 0, "points are held in packed pairs");
  constexpr int NP2 = NPOS / 2;
  const int upt = NPOS / P;  // units per thread per round
  const int used = upt * P;
  for (int ub = tid; ub < nunits; ub += nthreads * upt) {  // ub: this round's first unit
    float2 X2[NP2], Y2[NP2], acc2[NP2];  // points 2k and 2k + 1
    float mn[NPOS];
    int uu = 0, p = 0;
#pragma unroll
    for (int i = 0; i < NPOS; ++i) {
      const int u = ub + uu * nthreads;
      const bool ok = (i < used) && (u < nunits);
      const float4 ps = pose[at(ok ? u : ub)];
      const float2 sh = shp[ok ? p : 0];
      const float X = fmaf(ps.z, sh.x, fmaf(-ps.w, sh.y, ps.x));
      const float Y = fmaf(ps.w, sh.x, fmaf(ps.z, sh.y, ps.y));
      if (i & 1) {
        X2[i >> 1].y = X;
        Y2[i >> 1].y = Y;
      } else {
        X2[i >> 1].x = X;
        Y2[i >> 1].x = Y;
      }
      mn[i] = __int_as_float(0x7f800000);
      if (++p == P) {
        p = 0;
        ++uu;
      }
    }
#pragma unroll
    for (int k = 0; k < NP2; ++k) acc2[k] = make_float2(0.0f, 0.0f);
    // obstacles in pairs: 1/h1 + 1/h2 = (h1 + h2) / (h1 h2), one reciprocal
    // for two terms (h1 h2 stays finite for |p - c| < 4e9 m and h_eps >= 1e-18);
    // with more points per thread the pair's temporaries would not fit
    int j = 0;
    if constexpr (NPOS <= 8)
    for (; j + 1 < J; j += 2) {
      const float4 o = obs4[j], q = obs4[j + 1];
      const float2 nox = make_float2(-o.x, -o.x), noy = make_float2(-o.y, -o.y);
      const float2 noz = make_float2(o.z, o.z);
      const float2 nqx = make_float2(-q.x, -q.x), nqy = make_float2(-q.y, -q.y);
      const float2 nqz = make_float2(q.z, q.z);
#pragma unroll
      for (int k = 0; k < NP2; ++k) {
        const float2 dx = __fadd2_rn(X2[k], nox), dy = __fadd2_rn(Y2[k], noy);
        const float2 ex = __fadd2_rn(X2[k], nqx), ey = __fadd2_rn(Y2[k], nqy);
        float2 h1 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, noz));
        float2 h2 = __ffma2_rn(ex, ex, __ffma2_rn(ey, ey, nqz));
        mn[2 * k] = fmin3(mn[2 * k], h1.x, h2.x);
        mn[2 * k + 1] = fmin3(mn[2 * k + 1], h1.y, h2.y);
        h1 = make_float2(fmaxf(h1.x, h_eps), fmaxf(h1.y, h_eps));
        h2 = make_float2(fmaxf(h2.x, h_eps), fmaxf(h2.y, h_eps));
        const float2 pr = __fmul2_rn(h1, h2);
        const float2 r = make_float2(rcp_approx(pr.x), rcp_approx(pr.y));
        acc2[k] = __ffma2_rn(__fadd2_rn(h1, h2), r, acc2[k]);
      }
    }
    for (; j < J; ++j) {
      const float4 o = obs4[j];
      const float2 nox = make_float2(-o.x, -o.x), noy = make_float2(-o.y, -o.y);
      const float2 noz = make_float2(o.z, o.z);
#pragma unroll
      for (int k = 0; k < NP2; ++k) {
        const float2 dx = __fadd2_rn(X2[k], nox), dy = __fadd2_rn(Y2[k], noy);
        const float2 h = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, noz));
        mn[2 * k] = fminf(mn[2 * k], h.x);
        mn[2 * k + 1] = fminf(mn[2 * k + 1], h.y);
        acc2[k] = __fadd2_rn(acc2[k], make_float2(rcp_approx(fmaxf(h.x, h_eps)),
                                                  rcp_approx(fmaxf(h.y, h_eps))));
      }
    }
    if constexpr (GRID) {
      if (gv->g) {
#pragma unroll
        for (int k = 0; k < NP2; ++k) {
          const float hx = grid_h(*gv, X2[k].x, Y2[k].x), hy = grid_h(*gv, X2[k].y, Y2[k].y);
          mn[2 * k] = fminf(mn[2 * k], hx);
          mn[2 * k + 1] = fminf(mn[2 * k + 1], hy);
          acc2[k] = __fadd2_rn(acc2[k], make_float2(rcp_approx(fmaxf(hx, h_eps)),
                                                    rcp_approx(fmaxf(hy, h_eps))));
        }
      }
    }
    FF f = {0.0f, 0.0f};
    bool coll = false;
    uu = 0;
    p = 0;
#pragma unroll
    for (int i = 0; i < NPOS; ++i) {
      if (i < used) {
        ff_add(f, (i & 1) ? acc2[i >> 1].y : acc2[i >> 1].x);
        coll |= (mn[i] <= 0.0f);
        if (++p == P) {
          const int u = ub + uu * nthreads;
          if (u < nunits) uB[(size_t)at(u) * ustride] = make_float2(coll ? -f.hi : f.hi, f.lo);
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

// Sum of a float pair over the 32 lanes (fixed butterfly order).
__device__ __forceinline__ FF warp_sum_ff(FF a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF b;
    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
    b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
    a = ff_sum(a, b);
  }
  return a;
}

// Minimum of floats by an integer atomic: key(f) = ~u(f), u the
// order-preserving unsigned image of f, so that a larger key is a smaller f
// and 0 (the cleared word) is below every key of a number.  atomicMax over
// keys is an exact, order-independent minimum.
__device__ __forceinline__ unsigned min_key(float f) {
  const int i = __float_as_int(f);
  return ~((unsigned)(i >= 0 ? i : i ^ 0x7fffffff) ^ 0x80000000u);
}
__device__ __forceinline__ float key_min(unsigned k) {
  const int i = (int)(~k ^ 0x80000000u);
  return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

// Merge n partial results (rho_i, Z_i, cols_i[ncol]), each taken relative to
// its own minimum rho_i, into one relative to ref = min_i rho_i.hi: the
// log-sum-exp merge of Eq. 4's numerator and denominator.  ref is read from
// *minw, the key (min_key) into which every source put its rho_i.hi with an
// atomic maximum before its ticket; thread 0 clears the word for the next
// step once every thread has read it, and stores ref at *ref_out.  Source i
// is scaled by s_i = exp(-(rho_i - ref) / lambda) <= 1.  Every load of the
// merge (the word, a thread's first source row, its column pairs) is issued
// before the first of them is used: one memory round trip, which is most of
// what a merge costs when one CTA runs it alone at the end of a step.  The
// ncol columns are read as ncp = ncol / 2 float pairs: thread tid takes the
// cell (row group rg, column pair cp) = (tid / ncp, tid % ncp), i.e. rows
// rg, rg + RG, ... of that pair, up to kMergeLoads rows in flight; the
// threads with cp = 0 also add s_i Z_i.  The row groups are then added in
// order.  All threads of the CTA call it.
// PIPELINED: the rows in flight are two batches of kMergeLoads / 2, the next
// loading while one is added; otherwise one batch of kMergeLoads, added
// before the next is loaded.  Both add the rows in the same order (the same
// bits).  The two-batch form is faster in the one-controller step kernels
// (a 256-sample step: 24.2 against 26.4 us); the one-batch form in the
// persistent batch kernel (64 mixed controllers: 3.31 against 4.04 ms).
// Shared memory: scl (n floats), zi (n float2), buf (merge_buf_bytes).
// Outputs in shared memory: *Z_out, col_hi/col_lo[ncol].
template <bool PIPELINED>
__device__ inline void merge_partials(int n, const float4* rz, const float* cols, int ncol,
                                      unsigned* minw, float inv_lambda, float* scl, float2* zi,
                                      FF* buf, float* ref_out, FF* Z_out, float* col_hi,
                                      float* col_lo, int tid, int nthreads) {
  const int ncp = ncol >> 1;
  const int RG = merge_row_groups(ncol, nthreads);
  const int ncell = RG * ncp;
  const int ldb = ncol + 1;  // buf row: the columns, then Z
  const float2* cols2 = reinterpret_cast<const float2*>(cols);
  constexpr int KB = PIPELINED ? kMergeLoads / 2 : kMergeLoads;
  float2 va[KB], vb[KB];  // vb: the second batch (PIPELINED only)
  auto load = [&](float2 (&v)[KB], int cell, int r0) {
    const int rg = cell / ncp, cp = cell - rg * ncp;
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int i = rg + (r0 + q) * RG;
      v[q] = (cell < ncell && i < n) ? __ldcg(cols2 + (size_t)i * ncp + cp) : make_float2(0.0f, 0.0f);
    }
  };
  auto add = [&](const float2 (&v)[KB], int rg, int cp, int r0, FF& a0, FF& a1, FF& z) {
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int i = rg + (r0 + q) * RG;
      if (i < n) {
        const float sc = scl[i];
        ff_add(a0, v[q].x * sc);
        ff_add(a1, v[q].y * sc);
        if (cp == 0) {
          const float2 zz = zi[i];
          ff_add_prod(z, sc, zz.x, zz.y);
        }
      }
    }
  };
  const unsigned kmin = __ldcg(minw);
  const float4 c0 = tid < n ? __ldcg(rz + tid) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  load(va, tid, 0);
  if constexpr (PIPELINED) load(vb, tid, KB);
  const float ref = key_min(kmin);
  if (tid < n) {
    scl[tid] = expf(-((c0.x - ref) + c0.y) * inv_lambda);
    zi[tid] = make_float2(c0.z, c0.w);
  }
  for (int i = tid + nthreads; i < n; i += nthreads) {  // more sources than threads
    const float4 c = __ldcg(rz + i);
    scl[i] = expf(-((c.x - ref) + c.y) * inv_lambda);
    zi[i] = make_float2(c.z, c.w);
  }
  __syncthreads();
  if (tid == 0) {
    *ref_out = ref;
    *minw = 0u;
  }
  for (int cell = tid; cell < ncell; cell += nthreads) {
    const int rg = cell / ncp, cp = cell - rg * ncp;
    FF a0 = {0.0f, 0.0f}, a1 = {0.0f, 0.0f}, z = {0.0f, 0.0f};
    if constexpr (PIPELINED) {
      for (int r0 = 0;; r0 += 2 * KB) {
        add(va, rg, cp, r0, a0, a1, z);
        if (rg + (r0 + KB) * RG >= n) break;
        if (rg + (r0 + 2 * KB) * RG < n) load(va, cell, r0 + 2 * KB);
        add(vb, rg, cp, r0 + KB, a0, a1, z);
        if (rg + (r0 + 2 * KB) * RG >= n) break;
        if (rg + (r0 + 3 * KB) * RG < n) load(vb, cell, r0 + 3 * KB);
      }
    } else {
      for (int r0 = 0;; r0 += KB) {
        add(va, rg, cp, r0, a0, a1, z);
        if (rg + (r0 + KB) * RG >= n) break;
        load(va, cell, r0 + KB);
      }
    }
    buf[rg * ldb + 2 * cp] = a0;
    buf[rg * ldb + 2 * cp + 1] = a1;
    if (cp == 0) buf[rg * ldb + ncol] = z;
    if (cell + nthreads < ncell) {
      load(va, cell + nthreads, 0);
      if constexpr (PIPELINED) load(vb, cell + nthreads, KB);
    }
  }
  __syncthreads();
  for (int c = tid; c <= ncol; c += nthreads) {
    FF a = buf[c];
    for (int g = 1; g < RG; ++g) a = ff_sum(a, buf[g * ldb + c]);
    if (c < ncol) {
      col_hi[c] = a.hi;
      col_lo[c] = a.lo;
    } else {
      *Z_out = ff_norm(a);
    }
  }
  __syncthreads();
}

// Fused barrier over npos positions, one position per thread at a time
// (position i = unit i / P, shape point i % P): the fully parallel form used
// for the single nominal trajectory.  out[i] = +-sum_j 1/max(h, h_eps), the
// sign bit marking some h <= 0.  GRID: plus the grid map's term.
template <bool GRID = false>
__device__ __forceinline__ void barrier_flat(int npos, int P, int J, const float4* __restrict__ pose,
                                             const float2* __restrict__ shp,
                                             const float4* __restrict__ obs4, float h_eps,
                                             float* __restrict__ out, int tid, int nthreads,
                                             const GridView* gv = nullptr) {
  for (int i = tid; i < npos; i += nthreads) {
    const int u = i / P, p = i - u * P;
    const float4 ps = pose[u];
    const float2 sh = shp[p];
    const float X = fmaf(ps.z, sh.x, fmaf(-ps.w, sh.y, ps.x));
    const float Y = fmaf(ps.w, sh.x, fmaf(ps.z, sh.y, ps.y));
    float acc = 0.0f, mn = __int_as_float(0x7f800000);
    for (int j = 0; j < J; ++j) {
      const float4 o = obs4[j];
      float dx = X - o.x, dy = Y - o.y;
      float h = fmaf(dx, dx, fmaf(dy, dy, o.z));
      mn = fminf(mn, h);
      acc += rcp_approx(fmaxf(h, h_eps));
    }
    if constexpr (GRID) {
      if (gv->g) {
        const float h = grid_h(*gv, X, Y);
        mn = fminf(mn, h);
        acc += rcp_approx(fmaxf(h, h_eps));
      }
    }
    out[i] = mn <= 0.0f ? -acc : acc;
  }
}

// Warp inclusive prefix sum over the 32 lanes.
__device__ __forceinline__ float warp_incl_scan(float v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    float y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}
// The value of lane - 1; lane 0 receives `first`.
__device__ __forceinline__ float from_prev_lane(float v, float first, int lane) {
  float y = __shfl_up_sync(0xffffffffu, v, 1);
  return lane == 0 ? first : y;
}
__device__ __forceinline__ float lane31(float v) { return __shfl_sync(0xffffffffu, v, 31); }

}  // namespace dbm
