// C ABI of the DBaS-Log-MPPI step (declared in include/dbasmppi.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <deque>
#include <mutex>
#include <thread>
#include <new>
#include <vector>

#include "../../include/dbasmppi.h"
#include "kernels.cuh"

using namespace dbm;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(MPPI_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                  __FILE__, __LINE__);                                                   \
  } while (0)

// ------------------------------------------------------------------ kernels

__global__ void prep_kernel(const __grid_constant__ CtrlDesc D, int init) {
  __shared__ double red[64];
  if (init) init_constants(D, threadIdx.x, blockDim.x);
  prep_constants(D, D.U, &D.st->S_e, red, threadIdx.x, blockDim.x);
}

__global__ void weights_kernel(const double* __restrict__ costs, int K,
                               const DevState* __restrict__ st, double inv_lambda,
                               double* __restrict__ w) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K) w[k] = exp(-(costs[k] - st->rho) * inv_lambda) / st->Z;
}

// Raw Philox words and NLN draws of the device generator for k < K, t < T.
// One CTA waits on a fresh mbarrier (see mppi_debug_wait_probe).
__global__ void wait_probe_kernel(long long max_cycles, int arrive, int* expired) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_arrive(&bar);
  const bool ok = mbar_wait(&bar, 0u, 1 << 30, max_cycles);
  if (threadIdx.x == 0) *expired = ok ? 0 : 1;
}

__global__ void draws_kernel(int K, int T, uint32_t k0, uint32_t k1, uint32_t it_lo, uint32_t it_hi,
                             float L00, float L10, float L11, float ln_mu, float ln_sigma,
                             uint32_t* __restrict__ raw, float* __restrict__ du) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K * T) return;
  int k = i / T, t = i - k * T;
  uint4 r = philox4x32_10(make_uint4((uint32_t)k, (uint32_t)t, it_lo, it_hi), k0, k1);
  if (raw) reinterpret_cast<uint4*>(raw)[i] = r;
  if (du) reinterpret_cast<float2*>(du)[i] = nln_draw(r, L00, L10, L11, ln_mu, ln_sigma);
}

using StepFn = void (*)(CtrlDesc, const double*, const double*);

StepFn pick_kernel(int model, int npos, bool r80) {
  // [model][points 8 / 14][register form 96 / 80]
  static const StepFn table[MPPI_NUM_MODELS][2][2] = {
      {{step_u8, step_u8_r80}, {step_u14, step_u14_r80}},
      {{step_q8, step_q8_r80}, {step_q14, step_q14_r80}},
      {{step_a8, step_a8_r80}, {step_a14, step_a14_r80}},
      {{step_p8, step_p8_r80}, {step_p14, step_p14_r80}}};
  return table[model][npos == 14 ? 1 : 0][r80 ? 1 : 0];
}

// Forms of the step kernels beyond the plain one (96-register form, separate
// instantiations, so the plain kernels carry no trace of them): kFormSgf
// smooths the update (Savitzky-Golay), kFormGrid adds the grid map's barrier
// terms and smooths when asked.
constexpr int kFormPlain = 0, kFormSgf = 1, kFormGrid = 2;
StepFn pick_form_kernel(int form, int model, int npos) {
  static const StepFn table[2][MPPI_NUM_MODELS][2] = {
      {{step_u8_sgf, step_u14_sgf}, {step_q8_sgf, step_q14_sgf},
       {step_a8_sgf, step_a14_sgf}, {step_p8_sgf, step_p14_sgf}},
      {{step_u8_grid, step_u14_grid}, {step_q8_grid, step_q14_grid},
       {step_a8_grid, step_a14_grid}, {step_p8_grid, step_p14_grid}}};
  return table[form == kFormGrid ? 1 : 0][model][npos == 14 ? 1 : 0];
}

// World points a barrier thread holds: whole units of P points each; the
// instantiated sizes are 8, 14 and 16, picked to waste the fewest slots.
int pick_npos(int P) {
  const int opts[2] = {8, 14};
  int best = 16;
  double best_waste = 2.0;
  for (int o : opts) {
    if (o < P) continue;
    double waste = (double)(o - (o / P) * P) / o;
    if (waste < best_waste - 1e-12) {
      best_waste = waste;
      best = o;
    }
  }
  return best;
}

int state_dim(int model) {
  switch (model) {
    case MPPI_QUAD2D: return 6;
    case MPPI_ACKERMANN: return 4;
    case MPPI_QUAD5: return 5;
    default: return 3;
  }
}

bool finite_all(const double* a, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// One obstacle (cx, cy, r): finite, r >= 0, and within MPPI_MAX_COORD of the
// origin (which keeps the barrier's paired products h1 h2 finite in FP32).
int check_obstacle(const double* o, int j) {
  if (!finite_all(o, 3)) return fail(MPPI_EINVAL, "obstacle %d is not finite", j);
  if (o[2] < 0) return fail(MPPI_EINVAL, "obstacle %d has a negative radius", j);
  if (std::fabs(o[0]) > MPPI_MAX_COORD || std::fabs(o[1]) > MPPI_MAX_COORD || o[2] > MPPI_MAX_COORD)
    return fail(MPPI_EINVAL, "obstacle %d lies beyond %g m", j, (double)MPPI_MAX_COORD);
  return 0;
}

int validate(const mppi_params* p) {
  if (!p) return fail(MPPI_EINVAL, "params is NULL");
  if (p->model < 0 || p->model >= MPPI_NUM_MODELS)
    return fail(MPPI_EINVAL, "unknown model %d", p->model);
  if (p->K < 1 || p->K > MPPI_MAX_K) return fail(MPPI_EINVAL, "K=%d out of [1, %d]", p->K, MPPI_MAX_K);
  if (p->T < 1 || p->T > MPPI_MAX_T) return fail(MPPI_EINVAL, "T=%d out of [1, %d]", p->T, MPPI_MAX_T);
  if (p->n_shape < 1 || p->n_shape > MPPI_MAX_SHAPE)
    return fail(MPPI_EINVAL, "n_shape=%d out of [1, %d]", p->n_shape, MPPI_MAX_SHAPE);
  const double sc[] = {p->dt,      p->lambda,     p->ln_mu, p->ln_sigma, p->mu_coarse,
                       p->gamma_ctrl, p->gamma_bas, p->R_B,   p->C_coll,   p->h_eps,
                       p->mass,    p->inertia,    p->arm,   p->gravity, p->wheelbase};
  if (!finite_all(sc, 15) || !finite_all(p->sigma, 4) || !finite_all(p->Q, 6) ||
      !finite_all(p->Qf, 6) || !finite_all(p->u_min, 2) || !finite_all(p->u_max, 2) ||
      !finite_all(p->x_goal, 6) || !finite_all(p->shape, 2 * p->n_shape))
    return fail(MPPI_EINVAL, "non-finite parameter");
  if (!(p->dt > 0)) return fail(MPPI_EINVAL, "dt must be > 0");
  if (!(p->lambda > 0)) return fail(MPPI_EINVAL, "lambda must be > 0");
  if (!(p->gamma_bas > 0 && p->gamma_bas < 1)) return fail(MPPI_EINVAL, "gamma_bas must be in (0,1)");
  if (!(p->h_eps >= MPPI_MIN_H_EPS)) return fail(MPPI_EINVAL, "h_eps must be >= %g", MPPI_MIN_H_EPS);
  if (p->ln_sigma < 0) return fail(MPPI_EINVAL, "ln_sigma must be >= 0");
  for (int d = 0; d < 2; ++d)
    if (p->u_min[d] > p->u_max[d]) return fail(MPPI_EINVAL, "u_min > u_max");
  const double* S = p->sigma;
  if (S[1] != S[2]) return fail(MPPI_EINVAL, "Sigma must be symmetric");
  double det = S[0] * S[3] - S[1] * S[2];
  if (S[0] < 0 || S[3] < 0 || det < 0) return fail(MPPI_EINVAL, "Sigma must be positive semi-definite");
  if (p->gamma_ctrl != 0 && !(S[0] > 0 && det > 0))
    return fail(MPPI_EINVAL, "Sigma must be positive definite when gamma_ctrl != 0");
  if (p->model == MPPI_QUAD2D && !(p->mass > 0 && p->inertia > 0))
    return fail(MPPI_EINVAL, "quadrotor mass and inertia must be > 0");
  if (p->model == MPPI_QUAD5 && !(p->mass > 0))
    return fail(MPPI_EINVAL, "quadrotor mass must be > 0");
  if (p->model == MPPI_ACKERMANN) {
    if (!(p->wheelbase > 0)) return fail(MPPI_EINVAL, "wheelbase must be > 0");
    // tan(steering) of Eq. 14 is finite only inside (-pi/2, pi/2)
    if (!(p->u_min[0] > -1.5707963267948966 && p->u_max[0] < 1.5707963267948966))
      return fail(MPPI_EINVAL, "steering limits must lie inside (-pi/2, pi/2)");
  }
  if (p->sgf_window != 0) {
    const int w = p->sgf_window, o = p->sgf_order;
    if (w < 3 || w % 2 != 1 || w > MPPI_SGF_MAX_WINDOW || w > p->T)
      return fail(MPPI_EINVAL, "sgf_window=%d must be 0 or odd in [3, min(%d, T)]", w,
                  MPPI_SGF_MAX_WINDOW);
    if (o < 0 || o >= w || o > MPPI_SGF_MAX_ORDER)
      return fail(MPPI_EINVAL, "sgf_order=%d must be in [0, min(%d, sgf_window - 1)]", o,
                  MPPI_SGF_MAX_ORDER);
  }
  return MPPI_OK;
}

// Bytes of the buffer of the barrier weights cw: T floats, then, when the
// update is smoothed, the W x W Savitzky-Golay weights (sgf_table_offset).
size_t cw_bytes(const mppi_params* p) {
  if (p->sgf_window <= 0) return sizeof(float) * (size_t)p->T;
  return sizeof(float) * ((size_t)sgf_table_offset(p->T) + (size_t)p->sgf_window * p->sgf_window);
}

// Tiles merged by one CTA: all of them in one level up to 256 tiles, else
// groups of at least 32 so that at most 64 group results remain.
int group_size(int nTiles) {
  if (nTiles <= 256) return nTiles;
  int GT = (nTiles + 63) / 64;
  return GT < 32 ? 32 : GT;
}

int g_num_sms = 0;

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

// Largest dynamic shared memory a step kernel may request: the opt-in
// per-block maximum less the kernel's static shared memory.
int max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (v <= 0) v = 48 * 1024;
  cudaFuncAttributes fa;
  size_t stat = 0;
  if (cudaFuncGetAttributes(&fa, step_q14) == cudaSuccess) stat = fa.sharedSizeBytes;
  else cudaGetLastError();
  return v - (int)align_up((int)stat + 64, 128);
}

// Step kernel of a launch: the 96-register form, or the 80-register form
// (_r80) when the grid spans more than one wave of the 96-register form and
// the lower cap raises the CTAs resident per SM.  The shared-memory limit
// of a model's step kernels is raised once per device; the last decision per
// device is kept, so a repeated configuration costs no occupancy query
// (the allocation-free entry point calls this every step).
constexpr int kMaxPickDevices = 64;
struct PickMemo {
  int model, npos, threads, smem, nTiles;
  StepFn fn;
};
std::mutex g_pick_mu;
bool g_step_attr[kMaxPickDevices][MPPI_NUM_MODELS] = {};
bool g_form_attr[kMaxPickDevices][2][MPPI_NUM_MODELS] = {};
PickMemo g_pick_memo[kMaxPickDevices] = {};

int choose_step_kernel(int model, int npos, int threads, int smem, int nTiles, int form,
                       StepFn* out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxPickDevices) return fail(MPPI_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_pick_mu);
  if (form != kFormPlain) {
    bool& done = g_form_attr[dev][form == kFormGrid ? 1 : 0][model];
    if (!done) {
      const int lim = max_smem_optin();
      for (int np : {8, 14})
        CK(cudaFuncSetAttribute(pick_form_kernel(form, model, np),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
      done = true;
    }
    *out = pick_form_kernel(form, model, npos);
    return MPPI_OK;
  }
  // only this model's kernels: with lazy module loading, touching a kernel
  // loads its module, and the models a process never steps stay unloaded
  if (!g_step_attr[dev][model]) {
    const int lim = max_smem_optin();
    for (int np : {8, 14})
      for (bool r80 : {false, true})
        CK(cudaFuncSetAttribute(pick_kernel(model, np, r80),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    g_step_attr[dev][model] = true;
  }
  PickMemo& m = g_pick_memo[dev];
  if (m.fn && m.model == model && m.npos == npos && m.threads == threads && m.smem == smem &&
      m.nTiles == nTiles) {
    *out = m.fn;
    return MPPI_OK;
  }
  const StepFn hi = pick_kernel(model, npos, false), lo = pick_kernel(model, npos, true);
  int occ_hi = 0, occ_lo = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_hi, hi, threads, smem));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_lo, lo, threads, smem));
  const StepFn fn = (occ_lo > occ_hi && (long)nTiles > (long)occ_hi * num_sms()) ? lo : hi;
  m = PickMemo{model, npos, threads, smem, nTiles, fn};
  *out = fn;
  return MPPI_OK;
}

}  // namespace

// ------------------------------------------------------------------ context

struct mppi_ctx {
  mppi_params p;
  mppi_tiling tl;
  int n = 3;
  int Jcap = 0;
  int smem = 0;
  CtrlDesc D;
  StepFn fn = nullptr;
  double* d_U = nullptr;
  float2* d_cU = nullptr;
  float2* d_cA = nullptr;
  float* d_cw = nullptr;   // cw, then the smoothing weights when the update is smoothed
  float* d_grid = nullptr; // the grid map, when one is set
  DevState* d_st = nullptr;
  double* d_obst = nullptr;
  double* d_in = nullptr;  // x0 (n) then xref ((T+1) n)
  float* d_part = nullptr;
  float4* d_part_rz = nullptr;
  float* d_gpart = nullptr;
  float4* d_gpart_rz = nullptr;
  unsigned* d_cnt = nullptr;
  double* d_costs = nullptr;
  uint8_t* d_coll = nullptr;
  double* d_Ustar = nullptr;
  double* d_w = nullptr;
  // Host inputs of mppi_step: two mapped pinned staging buffers, used in
  // turn; the kernel reads x0 and xref from them over the host link (their
  // device aliases in h_in_dev), so no copy is staged before the launch.  A
  // buffer is rewritten only after the kernel that read it has finished
  // (in_ev, recorded after that launch).
  double* h_in[2] = {nullptr, nullptr};
  double* h_in_dev[2] = {nullptr, nullptr};
  cudaEvent_t in_ev[2] = {nullptr, nullptr};
  bool in_ev_pending[2] = {false, false};
  int in_next = 0;
  DevState* h_st = nullptr; // pinned readback
  double* h_U = nullptr;    // pinned readback
  HostOut* h_out = nullptr;      // mapped mirror of u0 and status, written by the step
  HostOut* h_out_dev = nullptr;  // its device alias
  cudaStream_t own = nullptr;
  cudaStream_t last = nullptr;
  bool stepped = false;
  bool mirrored = false;  // the last step writes the host mirror (mppi_step)
  uint64_t iter = 0;  // iteration counter of the device state after the steps enqueued so far
};

namespace {

// The form of step kernel a context needs: the grid map's when it has one,
// else the smoothing form when it smooths, else the plain one.
int step_form(const mppi_ctx* c) {
  if (c->d_grid) return kFormGrid;
  return c->p.sgf_window > 0 ? kFormSgf : kFormPlain;
}

void free_ctx(mppi_ctx* c) {
  if (!c) return;
  if (c->last) cudaStreamSynchronize(c->last);
  cudaFree(c->d_U);
  cudaFree(c->d_cU);
  cudaFree(c->d_cA);
  cudaFree(c->d_cw);
  cudaFree(c->d_grid);
  cudaFree(c->d_st);
  cudaFree(c->d_obst);
  cudaFree(c->d_in);
  cudaFree(c->d_part);
  cudaFree(c->d_part_rz);
  cudaFree(c->d_gpart);
  cudaFree(c->d_gpart_rz);
  cudaFree(c->d_cnt);
  cudaFree(c->d_costs);
  cudaFree(c->d_coll);
  cudaFree(c->d_Ustar);
  cudaFree(c->d_w);
  for (int b = 0; b < 2; ++b) {
    cudaFreeHost(c->h_in[b]);
    if (c->in_ev[b]) cudaEventDestroy(c->in_ev[b]);
  }
  cudaFreeHost(c->h_st);
  cudaFreeHost(c->h_U);
  cudaFreeHost(c->h_out);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
}

// Launch shape: S samples per CTA, chosen so the grid covers the SMs at
// least twice when K allows, then shrunk until the tile's shared memory
// (whole-horizon poses and controls, obstacles) fits.
int choose_tiling(const mppi_params* p, const mppi_tiling* req, int J, mppi_tiling* out,
                  int* smem_out, bool batched = false) {
  const int sms = num_sms();
  const int n = state_dim(p->model);
  mppi_tiling t = {0, 0, 0, 0};
  if (req) t = *req;
  const bool fixed_S = t.samples_per_cta > 0;
  if (!fixed_S) {
    long want = ((long)p->K + 2L * sms - 1) / (2L * sms);
    t.samples_per_cta = (int)(want < 1 ? 1 : (want > 32 ? 32 : want));
  }
  if (t.samples_per_cta > 32) return fail(MPPI_EINVAL, "samples_per_cta must be <= 32");
  if (t.threads <= 0) t.threads = 256;
  if (t.threads != 64 && t.threads != 128 && t.threads != 256 && t.threads != 512)
    return fail(MPPI_EINVAL, "threads must be 64, 128, 256 or 512");
  if (t.positions_per_thread <= 0) t.positions_per_thread = pick_npos(p->n_shape);
  if (t.positions_per_thread != 8 && t.positions_per_thread != 14)
    return fail(MPPI_EINVAL, "positions_per_thread must be 8 or 14");
  if (t.positions_per_thread < p->n_shape)
    return fail(MPPI_EINVAL, "positions_per_thread must be >= n_shape");
  t.chunk_steps = 0;
  const int limit = max_smem_optin();
  for (;;) {
    const int nTiles = (p->K + t.samples_per_cta - 1) / t.samples_per_cta;
    const int GT = group_size(nTiles);
    const int nGroups = (nTiles + GT - 1) / GT;
    const int nscl = GT > nGroups ? GT : nGroups;
    SmemLayout L =
        smem_layout(p->T, t.samples_per_cta, p->n_shape, J, n, nscl, t.threads / 32, batched);
    if (L.total <= limit) {
      *smem_out = L.total;
      break;
    }
    if (t.samples_per_cta > 1 && !fixed_S) {
      t.samples_per_cta = (t.samples_per_cta + 1) / 2;
    } else {
      return fail(MPPI_EINVAL, "problem needs %d bytes of shared memory per CTA (limit %d)",
                  L.total, limit);
    }
  }
  *out = t;
  return MPPI_OK;
}

// Fill the descriptor from the parameters and the device buffers.
void fill_desc(mppi_ctx* c) {
  const mppi_params* p = &c->p;
  CtrlDesc& D = c->D;
  memset(&D, 0, sizeof(D));
  D.model = p->model;
  D.K = p->K;
  D.T = p->T;
  D.J = 0;
  D.P = p->n_shape;
  D.n = c->n;
  D.S = c->tl.samples_per_cta;
  D.NPOS = c->tl.positions_per_thread;
  D.nTiles = (p->K + D.S - 1) / D.S;
  D.GT = group_size(D.nTiles);
  D.nGroups = (D.nTiles + D.GT - 1) / D.GT;
  D.nscl = D.GT > D.nGroups ? D.GT : D.nGroups;
  D.dt = (float)p->dt;
  D.h_eps = (float)p->h_eps;
  D.gamma_bas_f = (float)p->gamma_bas;
  D.R_B = (float)p->R_B;
  D.C_coll = (float)p->C_coll;
  D.ln_mu = (float)p->ln_mu;
  D.ln_sigma = (float)p->ln_sigma;
  for (int d = 0; d < 2; ++d) {
    D.umin[d] = (float)p->u_min[d];
    D.umax[d] = (float)p->u_max[d];
    D.umin_d[d] = p->u_min[d];
    D.umax_d[d] = p->u_max[d];
  }
  for (int d = 0; d < kMaxN; ++d) {
    D.Q[d] = d < c->n ? (float)p->Q[d] : 0.0f;
    D.Qf[d] = d < c->n ? (float)p->Qf[d] : 0.0f;
    D.x_goal[d] = d < c->n ? p->x_goal[d] : 0.0;
  }
  for (int i = 0; i < 2 * kMaxShape; ++i)
    D.shape[i] = i < 2 * p->n_shape ? (float)p->shape[i] : 0.0f;
  D.g = (float)p->gravity;
  D.inv_mass = (p->model == MPPI_QUAD2D || p->model == MPPI_QUAD5) ? (float)(1.0 / p->mass) : 0.0f;
  D.k_turn = p->model == MPPI_QUAD2D      ? (float)(p->arm / p->inertia)
             : p->model == MPPI_ACKERMANN ? (float)(1.0 / p->wheelbase)
                                          : 0.0f;
  D.lambda = p->lambda;
  D.inv_lambda = 1.0 / p->lambda;
  D.inv_lambda_f = (float)(1.0 / p->lambda);
  D.mu_coarse = p->mu_coarse;
  D.gamma_ctrl = p->gamma_ctrl;
  D.gamma_bas = p->gamma_bas;
  D.R_B_d = p->R_B;
  for (int i = 0; i < 4; ++i) D.sigma[i] = p->sigma[i];
  {
    // chol(Sigma) and gamma Sigma^-1 (PSD checked by validate; inverse only
    // needed, and only defined, when gamma_ctrl != 0)
    const double* S = p->sigma;
    double l00 = std::sqrt(S[0] > 0 ? S[0] : 0.0);
    double l10 = l00 > 0 ? S[2] / l00 : 0.0;
    double r = S[3] - l10 * l10;
    D.Lsig[0] = l00;
    D.Lsig[1] = l10;
    D.Lsig[2] = std::sqrt(r > 0 ? r : 0.0);
    double det = S[0] * S[3] - S[1] * S[2];
    double gi = p->gamma_ctrl != 0 ? p->gamma_ctrl / det : 0.0;
    D.Sinv[0] = gi * S[3];
    D.Sinv[1] = -gi * S[1];
    D.Sinv[2] = -gi * S[2];
    D.Sinv[3] = gi * S[0];
  }
  D.key0 = (uint32_t)(p->seed & 0xffffffffull);
  D.key1 = (uint32_t)(p->seed >> 32);
  D.U = c->d_U;
  D.cU = c->d_cU;
  D.cA = c->d_cA;
  D.cw = c->d_cw;
  D.st = c->d_st;
  D.obst = c->d_obst;
  D.x0 = c->d_in;
  D.xref = c->d_in + c->n;
  D.part = c->d_part;
  D.part_rz = c->d_part_rz;
  D.gpart = c->d_gpart;
  D.gpart_rz = c->d_gpart_rz;
  D.counters = c->d_cnt;
  D.costs = c->d_costs;
  D.coll = c->d_coll;
  D.Ustar = c->d_Ustar;
  D.host_out = c->h_out_dev;  // null for the batch slots and the static entry point
  D.sgf_wp = p->sgf_window > 0 ? p->sgf_window | (p->sgf_order << 8) : 0;
}

int check_status(mppi_ctx* c) {
  if (c->h_st->status == kStatusTimeout)
    return fail(MPPI_ETIMEOUT, "a bounded device wait (obstacle staging) expired");
  return MPPI_OK;
}

}  // namespace

extern "C" {

const char* mppi_last_error(void) { return g_err; }

int mppi_create_tiled(const mppi_params* p, const double* u_init, const mppi_tiling* tiling,
                      mppi_ctx** out) {
  if (!out) return fail(MPPI_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(p);
  if (rc) return rc;
  if (u_init && !finite_all(u_init, 2 * p->T)) return fail(MPPI_EINVAL, "non-finite u_init");
  mppi_ctx* c = new (std::nothrow) mppi_ctx();
  if (!c) return fail(MPPI_ENOMEM, "host allocation failed");
  c->p = *p;
  c->n = state_dim(p->model);
  rc = choose_tiling(p, tiling, 0, &c->tl, &c->smem);
  if (rc) {
    delete c;
    return rc;
  }
  const int T = p->T, K = p->K, n = c->n;
  const int nTiles = (K + c->tl.samples_per_cta - 1) / c->tl.samples_per_cta;
  const int GT = group_size(nTiles);
  const int nGroups = (nTiles + GT - 1) / GT;
#define ALLOC(ptr, bytes)                                                          \
  do {                                                                             \
    if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) {                      \
      cudaGetLastError();                                                          \
      free_ctx(c);                                                                 \
      return fail(MPPI_ENOMEM, "cudaMalloc of %zu bytes failed", (size_t)(bytes)); \
    }                                                                              \
  } while (0)
  ALLOC(c->d_U, sizeof(double) * 2 * T);
  ALLOC(c->d_cU, sizeof(float2) * T);
  ALLOC(c->d_cA, sizeof(float2) * T);
  ALLOC(c->d_cw, cw_bytes(p));
  ALLOC(c->d_st, sizeof(DevState));
  ALLOC(c->d_obst, 16);
  c->Jcap = 0;
  ALLOC(c->d_in, sizeof(double) * (n + (T + 1) * n));
  ALLOC(c->d_part, sizeof(float) * (size_t)nTiles * 2 * T);
  ALLOC(c->d_part_rz, sizeof(float4) * nTiles);
  ALLOC(c->d_gpart, sizeof(float) * (size_t)nGroups * 2 * T);
  ALLOC(c->d_gpart_rz, sizeof(float4) * nGroups);
  ALLOC(c->d_cnt, sizeof(unsigned) * 2 * (nGroups + 1));
  ALLOC(c->d_costs, sizeof(double) * K);
  ALLOC(c->d_coll, K);
  ALLOC(c->d_Ustar, sizeof(double) * 2 * T);
  ALLOC(c->d_w, sizeof(double) * K);
#undef ALLOC
  const size_t in_bytes = sizeof(double) * (n + (T + 1) * n);
  for (int b = 0; b < 2; ++b) {
    if (cudaHostAlloc((void**)&c->h_in[b], in_bytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&c->h_in_dev[b], c->h_in[b], 0) != cudaSuccess) {
      cudaGetLastError();
      free_ctx(c);
      return fail(MPPI_ENOMEM, "mapped pinned host allocation failed");
    }
  }
  if (cudaHostAlloc((void**)&c->h_out, sizeof(HostOut), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&c->h_out_dev, c->h_out, 0) != cudaSuccess) {
    cudaGetLastError();
    free_ctx(c);
    return fail(MPPI_ENOMEM, "mapped pinned host allocation failed");
  }
  memset(c->h_out, 0, sizeof(HostOut));
  if (cudaMallocHost((void**)&c->h_st, sizeof(DevState)) != cudaSuccess ||
      cudaMallocHost((void**)&c->h_U, sizeof(double) * 2 * T) != cudaSuccess) {
    cudaGetLastError();
    free_ctx(c);
    return fail(MPPI_ENOMEM, "pinned host allocation failed");
  }
  if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->in_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->in_ev[1], cudaEventDisableTiming) != cudaSuccess) {
    free_ctx(c);
    return fail(MPPI_ECUDA, "stream/event creation failed");
  }
  c->last = c->own;
  fill_desc(c);
  rc = choose_step_kernel(p->model, c->tl.positions_per_thread, c->tl.threads, c->smem, nTiles,
                          p->sgf_window > 0 ? kFormSgf : kFormPlain,
                          &c->fn);
  if (rc) {
    free_ctx(c);
    return rc;
  }
  // initial state: U, S_e = mu ln(e + 0) (Eq. 10 with C_B = 0), first call
  DevState st;
  memset(&st, 0, sizeof(st));
  st.S_e = p->mu_coarse > 0 ? p->mu_coarse : 1.0;
  st.first = 1;
  double* U0 = c->h_U;
  for (int i = 0; i < 2 * T; ++i) U0[i] = u_init ? u_init[i] : 0.0;
  if (cudaMemcpy(c->d_U, U0, sizeof(double) * 2 * T, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_st, &st, sizeof(DevState), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->d_cnt, 0, sizeof(unsigned) * 2 * (nGroups + 1)) != cudaSuccess) {
    free_ctx(c);
    return fail(MPPI_ECUDA, "initial upload failed");
  }
  prep_kernel<<<1, 256, 0, c->own>>>(c->D, 1);
  if (cudaStreamSynchronize(c->own) != cudaSuccess) {
    free_ctx(c);
    return fail(MPPI_ECUDA, "prep kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  *out = c;
  return MPPI_OK;
}

int mppi_create(const mppi_params* p, const double* u_init, mppi_ctx** out) {
  return mppi_create_tiled(p, u_init, nullptr, out);
}

int mppi_set_obstacles(mppi_ctx* c, const double* cxcyr, int32_t J) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  if (J < 0 || J > MPPI_MAX_OBSTACLES)
    return fail(MPPI_EINVAL, "J=%d out of [0, %d]", J, MPPI_MAX_OBSTACLES);
  if (J > 0 && !cxcyr) return fail(MPPI_EINVAL, "obstacles pointer is NULL");
  for (int j = 0; j < J; ++j) {
    if (int rc = check_obstacle(cxcyr + 3 * j, j)) return rc;
  }
  mppi_tiling t;
  int smem = 0;
  int rc = choose_tiling(&c->p, &c->tl, J, &t, &smem);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->last));
  const size_t bytes = (size_t)align_up(24 * (J > 0 ? J : 1), 16);
  if (J > c->Jcap) {
    double* nb = nullptr;
    if (cudaMalloc((void**)&nb, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(MPPI_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    cudaFree(c->d_obst);
    c->d_obst = nb;
    c->Jcap = J;
  }
  if (J > 0) {
    CK(cudaMemset(c->d_obst, 0, bytes));
    CK(cudaMemcpy(c->d_obst, cxcyr, sizeof(double) * 3 * J, cudaMemcpyHostToDevice));
  }
  if (t.samples_per_cta != c->tl.samples_per_cta)
    return fail(MPPI_EINVAL, "obstacle set too large for the controller's tile shape");
  StepFn fn = nullptr;
  rc = choose_step_kernel(c->p.model, t.positions_per_thread, t.threads, smem, c->D.nTiles,
                          step_form(c), &fn);
  if (rc) return rc;
  c->tl = t;
  c->smem = smem;
  c->fn = fn;
  c->D.J = J;
  c->D.obst = c->d_obst;
  return MPPI_OK;
}

namespace {
int check_grid(const float* sdf, int32_t nx, int32_t ny, double ox, double oy, double res) {
  if (!sdf) return fail(MPPI_EINVAL, "grid pointer is NULL");
  if (nx < 2 || ny < 2 || nx > MPPI_MAX_GRID_SIDE || ny > MPPI_MAX_GRID_SIDE ||
      (int64_t)nx * ny > MPPI_MAX_GRID_SAMPLES)
    return fail(MPPI_EINVAL, "grid of %d x %d samples: each side in [2, %d], at most %d samples",
                nx, ny, MPPI_MAX_GRID_SIDE, MPPI_MAX_GRID_SAMPLES);
  if (!(res > 0) || !std::isfinite(res) || !std::isfinite(ox) || !std::isfinite(oy))
    return fail(MPPI_EINVAL, "grid origin must be finite and its cell size finite and > 0");
  for (size_t i = 0; i < (size_t)nx * ny; ++i)
    if (!std::isfinite(sdf[i])) return fail(MPPI_EINVAL, "grid value %zu is not finite", i);
  return MPPI_OK;
}
}  // namespace

int mppi_set_grid(mppi_ctx* c, const float* sdf, int32_t nx, int32_t ny, double ox, double oy,
                  double res) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  const bool off = nx == 0 && ny == 0;
  if (!off) {
    if (int rc = check_grid(sdf, nx, ny, ox, oy, res)) return rc;
  }
  StepFn fn = nullptr;
  int rc = choose_step_kernel(c->p.model, c->tl.positions_per_thread, c->tl.threads, c->smem,
                              c->D.nTiles,
                              off ? (c->p.sgf_window > 0 ? kFormSgf : kFormPlain) : kFormGrid, &fn);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->last));  // no step in flight reads the old map
  float* nb = nullptr;
  if (!off) {
    const size_t bytes = sizeof(float) * (size_t)nx * ny;
    if (cudaMalloc((void**)&nb, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(MPPI_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    if (cudaMemcpy(nb, sdf, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(nb);
      return fail(MPPI_ECUDA, "grid upload failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
  }
  // the map's fields of the device state (no kernel writes them)
  DevState* hs = c->h_st;
  hs->grid = nb;
  hs->grid_nx = off ? 0 : nx;
  hs->grid_ny = off ? 0 : ny;
  hs->grid_ox = off ? 0.0 : ox;
  hs->grid_oy = off ? 0.0 : oy;
  hs->grid_res = off ? 0.0 : res;
  hs->grid_inv_res = off ? 0.0f : (float)(1.0 / res);
  hs->grid_pad = 0.0f;
  const size_t o = offsetof(DevState, grid);
  if (cudaMemcpy(reinterpret_cast<char*>(c->d_st) + o, reinterpret_cast<char*>(hs) + o,
                 sizeof(DevState) - o, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(nb);
    return fail(MPPI_ECUDA, "grid upload failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  cudaFree(c->d_grid);
  c->d_grid = nb;
  c->fn = fn;
  return MPPI_OK;
}

namespace {
// Enqueue one step.  mirror: the final stage writes u0, the status and the
// fenced sequence word to the mapped host mirror (mppi_step, whose caller
// reads the control on the host); the device-input entry point leaves it
// out, since the system-scope fence adds the host link's round trip to the
// kernel's retirement.
int launch_step(mppi_ctx* c, const double* x0, const double* xref, void* stream, bool mirror) {
  cudaStream_t s = stream ? (cudaStream_t)stream : c->own;
  if (mirror) {
    c->fn<<<c->D.nTiles, c->tl.threads, c->smem, s>>>(c->D, x0, xref);
  } else {
    CtrlDesc D = c->D;
    D.host_out = nullptr;
    c->fn<<<c->D.nTiles, c->tl.threads, c->smem, s>>>(D, x0, xref);
  }
  CK(cudaGetLastError());
  c->last = s;
  c->stepped = true;
  c->mirrored = mirror;
  ++c->iter;
  return MPPI_OK;
}
}  // namespace

int mppi_step_device(mppi_ctx* c, const double* d_x0, const double* d_xref, void* stream) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  if (!d_x0 || !d_xref) return fail(MPPI_EINVAL, "device x0 / xref must not be NULL");
  return launch_step(c, d_x0, d_xref, stream, false);
}

int mppi_step(mppi_ctx* c, const double* x0, const double* xref, void* stream) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  if (!x0) return fail(MPPI_EINVAL, "x0 is NULL");
  const int n = c->n, T = c->p.T;
  if (!finite_all(x0, n)) return fail(MPPI_EINVAL, "x0 is not finite");
  if (xref && !finite_all(xref, (T + 1) * n)) return fail(MPPI_EINVAL, "xref is not finite");
  cudaStream_t s = stream ? (cudaStream_t)stream : c->own;
  const int b = c->in_next;
  if (c->in_ev_pending[b]) CK(cudaEventSynchronize(c->in_ev[b]));  // its reader has finished
  double* h = c->h_in[b];
  memcpy(h, x0, sizeof(double) * n);
  if (xref) {
    memcpy(h + n, xref, sizeof(double) * (T + 1) * n);
  } else {
    for (int t = 0; t <= T; ++t) memcpy(h + n + t * n, c->p.x_goal, sizeof(double) * n);
  }
  const int rc = launch_step(c, c->h_in_dev[b], c->h_in_dev[b] + n, s, true);
  if (rc) return rc;
  CK(cudaEventRecord(c->in_ev[b], s));
  c->in_ev_pending[b] = true;
  c->in_next = b ^ 1;
  return MPPI_OK;
}

int mppi_get_control(mppi_ctx* c, double* u0, double* U) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  if (!c->stepped) return fail(MPPI_ESTATE, "no step has run");
  // u0 and the status word come from the mapped mirror the step's final
  // stage wrote; only U, when asked for, is copied
  if (!U && c->mirrored) {
    // the last step's final stage stores seq after its u0 and status (and a
    // system-scope fence): once seq shows that step, the mirror holds its
    // output, without waiting for the kernel to retire.  The stream is
    // polled now and then, so a step that ended without writing (an error)
    // falls through to the synchronisation below, which reports it.
    const int want = (int)(uint32_t)c->iter;
    volatile int* seq = &c->h_out->seq;
    for (unsigned n = 1;; ++n) {
      if (*seq == want) {
        std::atomic_thread_fence(std::memory_order_acquire);
        const volatile HostOut* o = c->h_out;
        if (o->status == kStatusTimeout)
          return fail(MPPI_ETIMEOUT, "a bounded device wait (obstacle staging) expired");
        if (u0) {
          u0[0] = o->u0[0];
          u0[1] = o->u0[1];
        }
        return MPPI_OK;
      }
      if ((n & 1023u) == 0u && cudaStreamQuery(c->last) != cudaErrorNotReady) break;
    }
  }
  if (U) CK(cudaMemcpyAsync(c->h_U, c->d_U, sizeof(double) * 2 * c->p.T, cudaMemcpyDeviceToHost, c->last));
  // a step with device inputs wrote no mirror: u0 and the status come from
  // the device state
  if (!c->mirrored)
    CK(cudaMemcpyAsync(c->h_st, c->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, c->last));
  CK(cudaStreamSynchronize(c->last));
  const int status = c->mirrored ? c->h_out->status : c->h_st->status;
  if (status == kStatusTimeout)
    return fail(MPPI_ETIMEOUT, "a bounded device wait (obstacle staging) expired");
  if (u0) {
    u0[0] = c->mirrored ? c->h_out->u0[0] : c->h_st->u0[0];
    u0[1] = c->mirrored ? c->h_out->u0[1] : c->h_st->u0[1];
  }
  if (U) memcpy(U, c->h_U, sizeof(double) * 2 * c->p.T);
  return MPPI_OK;
}

int mppi_get_debug(mppi_ctx* c, double* costs, uint8_t* collided, double* weights, double* Ustar,
                   double* scalars) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  if (!c->stepped) return fail(MPPI_ESTATE, "no step has run");
  const int K = c->p.K, T = c->p.T;
  cudaStream_t s = c->last;
  if (weights) {
    weights_kernel<<<(K + 255) / 256, 256, 0, s>>>(c->d_costs, K, c->d_st, 1.0 / c->p.lambda, c->d_w);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(c->h_st, c->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (costs) CK(cudaMemcpy(costs, c->d_costs, sizeof(double) * K, cudaMemcpyDeviceToHost));
  if (collided) CK(cudaMemcpy(collided, c->d_coll, K, cudaMemcpyDeviceToHost));
  if (weights) CK(cudaMemcpy(weights, c->d_w, sizeof(double) * K, cudaMemcpyDeviceToHost));
  if (Ustar) CK(cudaMemcpy(Ustar, c->d_Ustar, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost));
  if (scalars) {
    const DevState& st = *c->h_st;
    scalars[0] = st.rho;
    scalars[1] = st.Z;
    scalars[2] = st.CB_star;
    scalars[3] = st.S_e;
    scalars[4] = st.beta_used;
    scalars[5] = st.beta_d;
    scalars[6] = st.S_e_used;
    scalars[7] = (double)st.iter;
  }
  return check_status(c);
}

int mppi_io_bytes(mppi_ctx* c, uint64_t* h2d, uint64_t* d2h) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  if (h2d) *h2d = sizeof(double) * (uint64_t)(c->n + (c->p.T + 1) * c->n);
  if (d2h) *d2h = sizeof(HostOut);  // u0 and the status word, written by the step
  return MPPI_OK;
}

int mppi_get_tiling(mppi_ctx* c, mppi_tiling* t, int32_t* n_ctas) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  if (t) *t = c->tl;
  if (n_ctas) *n_ctas = c->D.nTiles;
  return MPPI_OK;
}

int mppi_get_kernel_regs(mppi_ctx* c, int32_t* regs_cap) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  if (!regs_cap) return fail(MPPI_EINVAL, "regs_cap is NULL");
  const bool r80 = c->fn == pick_kernel(c->p.model, c->tl.positions_per_thread, true);
  *regs_cap = r80 ? DBM_STEP_MAXNREG_R80 : DBM_STEP_MAXNREG;
  return MPPI_OK;
}

int mppi_get_state(mppi_ctx* c, double* U, double* S_e, double* beta, int32_t* first,
                   uint64_t* iter) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  CK(cudaStreamSynchronize(c->last));
  CK(cudaMemcpy(c->h_st, c->d_st, sizeof(DevState), cudaMemcpyDeviceToHost));
  if (U) CK(cudaMemcpy(U, c->d_U, sizeof(double) * 2 * c->p.T, cudaMemcpyDeviceToHost));
  if (S_e) *S_e = c->h_st->S_e;
  if (beta) *beta = c->h_st->beta;
  if (first) *first = c->h_st->first;
  if (iter) *iter = c->h_st->iter;
  return MPPI_OK;
}

int mppi_set_state(mppi_ctx* c, const double* U, double S_e, double beta, int32_t first,
                   uint64_t iter) {
  if (!c) return fail(MPPI_ESTATE, "context is NULL");
  if (!U || !finite_all(U, 2 * c->p.T)) return fail(MPPI_EINVAL, "U missing or not finite");
  if (!std::isfinite(S_e) || !(S_e > 0) || !std::isfinite(beta))
    return fail(MPPI_EINVAL, "S_e must be finite and > 0, beta finite");
  CK(cudaStreamSynchronize(c->last));
  CK(cudaMemcpy(c->h_st, c->d_st, sizeof(DevState), cudaMemcpyDeviceToHost));
  DevState st = *c->h_st;
  st.S_e = S_e;
  st.beta = beta;
  st.first = first ? 1 : 0;
  st.iter = iter;
  st.status = 0;
  c->iter = iter;
  CK(cudaMemcpy(c->d_U, U, sizeof(double) * 2 * c->p.T, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_st, &st, sizeof(DevState), cudaMemcpyHostToDevice));
  prep_kernel<<<1, 256, 0, c->own>>>(c->D, 0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->own));
  return MPPI_OK;
}

extern "C" int mppi_debug_wait_probe(int64_t max_cycles, int32_t arrive) {
  if (max_cycles < 1 || max_cycles > 4000000000ll)
    return fail(MPPI_EINVAL, "max_cycles must be in [1, 4e9]");
  int* d = nullptr;
  CK(cudaMalloc((void**)&d, sizeof(int)));
  wait_probe_kernel<<<1, 32>>>((long long)max_cycles, arrive ? 1 : 0, d);
  int h = -1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(MPPI_ECUDA, "wait probe: %s", cudaGetErrorString(e));
  if (h != 0) return fail(MPPI_ETIMEOUT, "the bounded device wait expired (probe)");
  return MPPI_OK;
}

int mppi_debug_draws(const mppi_params* p, double S_e, uint64_t iter, int32_t K, int32_t T,
                     uint32_t* raw, float* du) {
  int rc = validate(p);
  if (rc) return rc;
  if (K < 1 || T < 1 || (long)K * T > (1L << 26)) return fail(MPPI_EINVAL, "K*T out of range");
  if (!(S_e > 0)) return fail(MPPI_EINVAL, "S_e must be > 0");
  double a = S_e * p->sigma[0], c = S_e * p->sigma[2], d = S_e * p->sigma[3];
  double l00 = std::sqrt(a > 0 ? a : 0.0);
  double l10 = l00 > 0 ? c / l00 : 0.0;
  double r = d - l10 * l10;
  double l11 = std::sqrt(r > 0 ? r : 0.0);
  const size_t N = (size_t)K * T;
  uint32_t* d_raw = nullptr;
  float* d_du = nullptr;
  CK(cudaMalloc((void**)&d_raw, N * 16));
  if (cudaMalloc((void**)&d_du, N * 8) != cudaSuccess) {
    cudaFree(d_raw);
    return fail(MPPI_ENOMEM, "cudaMalloc failed");
  }
  draws_kernel<<<(unsigned)((N + 255) / 256), 256>>>(
      K, T, (uint32_t)(p->seed & 0xffffffffull), (uint32_t)(p->seed >> 32),
      (uint32_t)(iter & 0xffffffffull), (uint32_t)(iter >> 32), (float)l00, (float)l10, (float)l11,
      (float)p->ln_mu, (float)p->ln_sigma, d_raw, d_du);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && raw) e = cudaMemcpy(raw, d_raw, N * 16, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && du) e = cudaMemcpy(du, d_du, N * 8, cudaMemcpyDeviceToHost);
  cudaFree(d_raw);
  cudaFree(d_du);
  if (e != cudaSuccess) return fail(MPPI_ECUDA, "draws failed: %s", cudaGetErrorString(e));
  return MPPI_OK;
}

int mppi_destroy(mppi_ctx* c) {
  free_ctx(c);
  return MPPI_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Allocation-free step.  For callers that may not allocate device memory once
// they run: real-time control loops that must keep every step's latency
// bounded (cudaMalloc can block and synchronise the device), and host
// programs whose device memory is owned by another allocator.  Everything
// the step needs beyond its inputs and outputs lives in this fixed array,
// which every GPU that loads the library keeps until the process exits.

namespace {

constexpr size_t kStaticScratchBytes = 8u << 20;  // 8 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxStaticDevices = 64;
unsigned char* g_static_base[kMaxStaticDevices] = {nullptr};  // device address, per device
std::mutex g_static_mu;  // guards the set-up of g_static_base

// Device-side copy of the caller's controller state into the scratch state
// block, ticket counters and minimum words cleared, constants derived; the caller's ctl is
// {S_e, beta, first, iter, status}.
__global__ void static_prologue(const __grid_constant__ CtrlDesc D, const double* __restrict__ ctl,
                                int n_counters) {
  __shared__ double red[64];
  if (threadIdx.x == 0) {
    D.st->S_e = ctl[0];
    D.st->beta = ctl[1];
    D.st->first = ctl[2] != 0.0 ? 1 : 0;
    D.st->iter = (unsigned long long)ctl[3];
    D.st->status = 0;
  }
  for (int i = threadIdx.x; i < n_counters; i += blockDim.x) D.counters[i] = 0u;
  __syncthreads();
  init_constants(D, threadIdx.x, blockDim.x);
  prep_constants(D, D.U, &D.st->S_e, red, threadIdx.x, blockDim.x);
}

__global__ void static_epilogue(const DevState* __restrict__ st, double* __restrict__ ctl,
                                double* __restrict__ u0) {
  if (threadIdx.x == 0) {
    ctl[0] = st->S_e;
    ctl[1] = st->beta;
    ctl[2] = st->first;
    ctl[3] = (double)st->iter;
    ctl[4] = st->status;
    u0[0] = st->u0[0];
    u0[1] = st->u0[1];
  }
}

size_t carve(size_t* off, size_t bytes) {
  size_t at = *off;
  *off += (bytes + 255) & ~(size_t)255;
  return at;
}

}  // namespace

extern "C" int mppi_step_static(const mppi_params* p, const double* d_obst, int32_t J,
                                const double* d_x0, const double* d_xref, double* d_U,
                                double* d_ctl, double* d_u0, double* d_costs, void* stream) {
  int rc = validate(p);
  if (rc) return rc;
  if (J < 0 || J > MPPI_MAX_OBSTACLES)
    return fail(MPPI_EINVAL, "J=%d out of [0, %d]", J, MPPI_MAX_OBSTACLES);
  if ((J > 0 && !d_obst) || !d_x0 || !d_xref || !d_U || !d_ctl || !d_u0)
    return fail(MPPI_EINVAL, "a required device pointer is NULL");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxStaticDevices) return fail(MPPI_EINVAL, "device %d out of range", dev);
  unsigned char* base = nullptr;
  {
    // set-up, once per device, with that device current; the lock makes the
    // first calls of several host threads safe
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_base[dev]) {
      void* a = nullptr;
      CK(cudaGetSymbolAddress(&a, g_static_scratch));
      g_static_base[dev] = (unsigned char*)a;
    }
    base = g_static_base[dev];
  }
  mppi_ctx c;  // on the stack: only its descriptor logic is used
  c.p = *p;
  c.n = state_dim(p->model);
  rc = choose_tiling(p, nullptr, J, &c.tl, &c.smem);
  if (rc) return rc;
  const int T = p->T, K = p->K;
  const int nTiles = (K + c.tl.samples_per_cta - 1) / c.tl.samples_per_cta;
  const int GT = group_size(nTiles);
  const int nGroups = (nTiles + GT - 1) / GT;
  StepFn fn = nullptr;  // picked before anything is launched
  rc = choose_step_kernel(p->model, c.tl.positions_per_thread, c.tl.threads, c.smem, nTiles,
                          p->sgf_window > 0 ? kFormSgf : kFormPlain, &fn);
  if (rc) return rc;
  size_t off = 0;
  const size_t o_st = carve(&off, sizeof(DevState));
  const size_t o_cU = carve(&off, sizeof(float2) * T);
  const size_t o_cA = carve(&off, sizeof(float2) * T);
  const size_t o_cw = carve(&off, cw_bytes(p));
  const size_t o_obst = carve(&off, (size_t)align_up(24 * (J > 0 ? J : 1), 16));
  const size_t o_part = carve(&off, sizeof(float) * (size_t)nTiles * 2 * T);
  const size_t o_prz = carve(&off, sizeof(float4) * nTiles);
  const size_t o_gpart = carve(&off, sizeof(float) * (size_t)nGroups * 2 * T);
  const size_t o_grz = carve(&off, sizeof(float4) * nGroups);
  const size_t o_cnt = carve(&off, sizeof(unsigned) * 2 * (nGroups + 1));
  const size_t o_costs = d_costs ? 0 : carve(&off, sizeof(double) * K);
  const size_t o_coll = carve(&off, (size_t)K);
  const size_t o_Ustar = carve(&off, sizeof(double) * 2 * T);
  if (off > kStaticScratchBytes)
    return fail(MPPI_EINVAL, "step needs %zu bytes of static scratch, the limit is %zu", off,
                kStaticScratchBytes);
  cudaStream_t s = (cudaStream_t)stream;
  c.d_U = d_U;
  c.d_cU = (float2*)(base + o_cU);
  c.d_cA = (float2*)(base + o_cA);
  c.d_cw = (float*)(base + o_cw);
  c.d_st = (DevState*)(base + o_st);
  c.d_obst = (double*)(base + o_obst);
  c.d_in = nullptr;
  c.d_part = (float*)(base + o_part);
  c.d_part_rz = (float4*)(base + o_prz);
  c.d_gpart = (float*)(base + o_gpart);
  c.d_gpart_rz = (float4*)(base + o_grz);
  c.d_cnt = (unsigned*)(base + o_cnt);
  c.d_costs = d_costs ? d_costs : (double*)(base + o_costs);
  c.d_coll = (uint8_t*)(base + o_coll);
  c.d_Ustar = (double*)(base + o_Ustar);
  fill_desc(&c);
  c.D.J = J;
  if (J > 0)
    CK(cudaMemcpyAsync(c.d_obst, d_obst, sizeof(double) * 3 * J, cudaMemcpyDeviceToDevice, s));
  static_prologue<<<1, 256, 0, s>>>(c.D, d_ctl, 2 * (nGroups + 1));
  CK(cudaGetLastError());
  fn<<<c.D.nTiles, c.tl.threads, c.smem, s>>>(c.D, d_x0, d_xref);
  CK(cudaGetLastError());
  static_epilogue<<<1, 32, 0, s>>>(c.d_st, d_ctl, d_u0);
  CK(cudaGetLastError());
  return MPPI_OK;
}

// ------------------------------------------------------------------------
// Autotuner: time the candidate launch shapes on the problem itself and keep
// the fastest.  Candidates: every samples-per-CTA value 1..32 (those giving
// at most 16 CTAs per SM): neighbouring values trade how the last wave of
// CTAs fills the SMs against how fully the tile's units fill the barrier's
// register slots, a discrete trade-off settled here by measurement; threads
// in {128, 256, 512}; world points per barrier thread in {8, 14} (whole
// units).
// Each candidate runs on a scratch controller: two warm-up steps, two steps
// that estimate its step time, then max(iters, steps filling about 2 ms)
// timed steps (CUDA events).  The controller state is reset so every
// candidate sees the same inputs.
constexpr float kTuneWindowUs = 2000.0f;  // device time timed per candidate, at least
constexpr int kTuneMaxReps = 400;
constexpr int kTuneMaxRepsFlushed = 40;  // each flushed step also writes the flush buffer

extern "C" int mppi_autotune(const mppi_params* p, const double* cxcyr, int32_t J, int32_t iters,
                             mppi_tiling* best, float* best_us) {
  return mppi_autotune_flush(p, cxcyr, J, nullptr, 0, 0, 0.0, 0.0, 0.0, iters, 0, best, best_us);
}

extern "C" int mppi_autotune_grid(const mppi_params* p, const double* cxcyr, int32_t J,
                                  const float* sdf, int32_t nx, int32_t ny, double ox, double oy,
                                  double res, int32_t iters, mppi_tiling* best, float* best_us) {
  return mppi_autotune_flush(p, cxcyr, J, sdf, nx, ny, ox, oy, res, iters, 0, best, best_us);
}

extern "C" int mppi_autotune_flush(const mppi_params* p, const double* cxcyr, int32_t J,
                                   const float* sdf, int32_t nx, int32_t ny, double ox, double oy,
                                   double res, int32_t iters, uint64_t flush_bytes,
                                   mppi_tiling* best, float* best_us) {
  int rc = validate(p);
  if (rc) return rc;
  if (sdf && (rc = check_grid(sdf, nx, ny, ox, oy, res))) return rc;
  if (!best) return fail(MPPI_EINVAL, "best is NULL");
  if (flush_bytes > ((uint64_t)4 << 30)) return fail(MPPI_EINVAL, "flush_bytes above 4 GiB");
  if (iters < 1) iters = 5;
  // with flush_bytes, each timed step runs alone after a write of that many
  // bytes (an L2 flush when it exceeds the L2), as a caller that steps once
  // per control period sees it
  void* flush = nullptr;
  if (flush_bytes && cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(MPPI_ENOMEM, "cudaMalloc of the %llu-byte flush buffer failed",
                (unsigned long long)flush_bytes);
  }
  const int sms = num_sms();
  int S_opts[32];
  for (int i = 0; i < 32; ++i) S_opts[i] = i + 1;
  const int NT_opts[3] = {128, 256, 512};
  const int NP_opts[2] = {8, 14};
  const int n = state_dim(p->model);
  double* x0 = new double[(size_t)n * (p->T + 2)];
  for (int d = 0; d < n; ++d) x0[d] = p->x_goal[d];
  for (int t = 0; t <= p->T; ++t)
    for (int d = 0; d < n; ++d) x0[n + t * n + d] = p->x_goal[d];
  float best_t = 1e30f;
  mppi_tiling best_tl = {0, 0, 0, 0};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int S : S_opts) {
    const long nT = ((long)p->K + S - 1) / S;
    if (S > p->K && S != S_opts[0]) continue;
    if (nT > 16L * sms * 4 && S < 32) continue;  // far too many tiny tiles
    for (int NT : NT_opts)
      for (int NP : NP_opts) {
        if (NP < p->n_shape) continue;
        mppi_tiling t = {S, NT, NP, 0};
        mppi_ctx* c = nullptr;
        if (mppi_create_tiled(p, nullptr, &t, &c) != MPPI_OK) continue;
        if (mppi_set_obstacles(c, cxcyr, J) != MPPI_OK || c->tl.samples_per_cta != S ||
            (sdf && mppi_set_grid(c, sdf, nx, ny, ox, oy, res) != MPPI_OK)) {
          mppi_destroy(c);
          continue;
        }
        bool ok = true;
        for (int w = 0; w < 2 && ok; ++w) ok = mppi_step(c, x0, x0 + n, nullptr) == MPPI_OK;
        if (ok) ok = cudaStreamSynchronize(c->own) == cudaSuccess;
        // the timed steps read their inputs from device memory
        if (ok)
          ok = cudaMemcpy(c->d_in, x0, sizeof(double) * n * (p->T + 2), cudaMemcpyHostToDevice) ==
               cudaSuccess;
        // timed steps: at least `iters`, and enough to cover kTuneWindowUs of
        // device time (estimated from two steps), so that microsecond-scale
        // steps are not ranked on launch jitter
        int reps = iters;
        float ms = 0.0f;
        for (int pass = 0; pass < 2 && ok; ++pass) {
          const int k = pass == 0 ? 2 : reps;
          if (flush) {  // each step alone, after the flush, its own events
            ms = 0.0f;
            for (int i = 0; i < k && ok; ++i) {
              float one = 0.0f;
              ok = cudaMemsetAsync(flush, i & 0xff, flush_bytes, c->own) == cudaSuccess &&
                   cudaEventRecord(e0, c->own) == cudaSuccess &&
                   mppi_step_device(c, c->d_in, c->d_in + n, nullptr) == MPPI_OK &&
                   cudaEventRecord(e1, c->own) == cudaSuccess &&
                   cudaEventSynchronize(e1) == cudaSuccess &&
                   cudaEventElapsedTime(&one, e0, e1) == cudaSuccess;
              ms += one;
            }
          } else {
            cudaEventRecord(e0, c->own);
            for (int i = 0; i < k && ok; ++i)
              ok = mppi_step_device(c, c->d_in, c->d_in + n, nullptr) == MPPI_OK;
            cudaEventRecord(e1, c->own);
            ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
            if (ok) cudaEventElapsedTime(&ms, e0, e1);
          }
          if (pass == 0 && ok) {
            const float est_us = 1000.0f * ms / 2.0f;
            const float want = est_us > 0.0f ? kTuneWindowUs / est_us : (float)kTuneMaxReps;
            reps = std::max(iters, std::min(flush ? kTuneMaxRepsFlushed : kTuneMaxReps, (int)want + 1));
          }
        }
        mppi_destroy(c);
        if (!ok) {
          cudaGetLastError();
          continue;
        }
        const float us = 1000.0f * ms / reps;
        if (us < best_t) {
          best_t = us;
          best_tl = t;
        }
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(flush);
  delete[] x0;
  if (best_tl.samples_per_cta == 0) return fail(MPPI_ECUDA, "no launch shape ran");
  *best = best_tl;
  if (best_us) *best_us = best_t;
  return MPPI_OK;
}

// ------------------------------------------------------------------------
// Batched execution: controllers of mixed model, K, T and obstacle count
// stepped together by one persistent launch.  Each controller keeps its
// state in a slot carved from one device pool (admission by memory).  A
// step packs, in one pinned block, a header, the step table (slot and input
// offsets of each stepped controller), the work items (controller, tile) in
// longest-first order and the packed x0 / xref; one host-to-device copy, one
// persistent kernel whose CTAs pull work items from an atomic counter, one
// device-to-host copy of the u0.  The sequence is captured in a CUDA graph
// and replayed while the set of stepped controllers stays the same.

namespace {

struct BatchSlot {
  bool used = false;
  mppi_params p;
  mppi_tiling tl;
  int n = 3, J = 0, Jcap = 0, smem = 0;
  size_t off = 0, bytes = 0;   // pool range
  size_t obst_off = 0;         // pool offset of the obstacle area
  CtrlDesc D;
  double tile_cost = 0.0;      // work estimate of one tile
};

}  // namespace

// One launch lane: staging, outputs, stream state and captured graph of
// one in-flight batched step.  A batch has one lane for mppi_batch_step; the
// serving runtime keeps several so that steps overlap on the device.
struct BatchLane {
  unsigned char* h_stage = nullptr;
  unsigned char* d_stage = nullptr;
  size_t stage_cap = 0;
  double* h_out = nullptr;  // 8 doubles per stepped controller: u0, predicted x1
  double* d_out = nullptr;
  int out_cap = 0;
  int n_last = 0;
  cudaStream_t last = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<int> graph_key;  // stepped slots the graph was captured for
  size_t graph_bytes = 0;
  int graph_smem = 0, graph_grid = 0;
  // buffers outgrown by a larger step, freed with the lane: cudaFree and
  // cudaFreeHost wait for the whole device, which would stall a scheduler
  // that keeps other lanes' work in flight
  std::vector<void*> retired_host, retired_dev;
};

struct mppi_batch {
  int max_ctrl = 0;
  unsigned char* pool = nullptr;
  size_t pool_bytes = 0;
  std::vector<std::pair<size_t, size_t>> free_list;  // (offset, size), sorted
  std::vector<BatchSlot> slots;
  CtrlDesc* d_descs = nullptr;
  BatchLane lane;
  cudaStream_t own = nullptr;
  int use_graph = 1;
  int max_smem = 0;
  mppi_batch_policy pol = {{32, 32, 32, 32}, {0, 0, 0, 0}};
};

namespace {

bool pool_alloc(mppi_batch* b, size_t bytes, size_t* off) {
  bytes = (bytes + 255) & ~(size_t)255;
  for (size_t i = 0; i < b->free_list.size(); ++i) {
    auto& f = b->free_list[i];
    if (f.second >= bytes) {
      *off = f.first;
      f.first += bytes;
      f.second -= bytes;
      if (f.second == 0) b->free_list.erase(b->free_list.begin() + i);
      return true;
    }
  }
  return false;
}

void pool_free(mppi_batch* b, size_t off, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  b->free_list.push_back({off, bytes});
  std::sort(b->free_list.begin(), b->free_list.end());
  std::vector<std::pair<size_t, size_t>> merged;
  for (auto& f : b->free_list) {
    if (!merged.empty() && merged.back().first + merged.back().second == f.first)
      merged.back().second += f.second;
    else
      merged.push_back(f);
  }
  b->free_list.swap(merged);
}

void drop_lane_graph(BatchLane& L) {
  if (L.gexec) cudaGraphExecDestroy(L.gexec);
  if (L.graph) cudaGraphDestroy(L.graph);
  L.gexec = nullptr;
  L.graph = nullptr;
  L.graph_key.clear();
}
void drop_graph(mppi_batch* b) { drop_lane_graph(b->lane); }

void free_lane(BatchLane& L) {
  if (L.last) cudaStreamSynchronize(L.last);
  drop_lane_graph(L);
  cudaFreeHost(L.h_stage);
  cudaFree(L.d_stage);
  cudaFreeHost(L.h_out);
  cudaFree(L.d_out);
  for (void* p : L.retired_host) cudaFreeHost(p);
  for (void* p : L.retired_dev) cudaFree(p);
  L = BatchLane();
}

// Make room for a step of `bytes` of staging and n outputs; outgrown buffers
// are retired, not freed (see BatchLane).
int lane_reserve(BatchLane& L, size_t bytes, int n) {
  if (bytes > L.stage_cap) {
    drop_lane_graph(L);
    if (L.h_stage) L.retired_host.push_back(L.h_stage);
    if (L.d_stage) L.retired_dev.push_back(L.d_stage);
    L.h_stage = nullptr;
    L.d_stage = nullptr;
    size_t cap = std::max(bytes, (size_t)1 << 16) * 2;
    if (cudaMallocHost((void**)&L.h_stage, cap) != cudaSuccess ||
        cudaMalloc((void**)&L.d_stage, cap) != cudaSuccess) {
      cudaGetLastError();
      L.stage_cap = 0;
      return fail(MPPI_ENOMEM, "staging allocation failed");
    }
    L.stage_cap = cap;
  }
  if (n > L.out_cap) {
    drop_lane_graph(L);
    if (L.h_out) L.retired_host.push_back(L.h_out);
    if (L.d_out) L.retired_dev.push_back(L.d_out);
    L.h_out = nullptr;
    L.d_out = nullptr;
    int cap = std::max(n, 64) * 2;
    if (cudaMallocHost((void**)&L.h_out, sizeof(double) * 8 * cap) != cudaSuccess ||
        cudaMalloc((void**)&L.d_out, sizeof(double) * 8 * cap) != cudaSuccess) {
      cudaGetLastError();
      L.out_cap = 0;
      return fail(MPPI_ENOMEM, "output allocation failed");
    }
    L.out_cap = cap;
  }
  return MPPI_OK;
}

// Device bytes of one slot (laid out in this order by slot_layout).
size_t slot_bytes(const mppi_params* p, const mppi_tiling* t, int Jcap) {
  const int T = p->T, K = p->K;
  const int nTiles = (K + t->samples_per_cta - 1) / t->samples_per_cta;
  const int GT = group_size(nTiles);
  const int nGroups = (nTiles + GT - 1) / GT;
  size_t off = 0;
  carve(&off, sizeof(double) * 2 * T);
  carve(&off, sizeof(float2) * T);
  carve(&off, sizeof(float2) * T);
  carve(&off, cw_bytes(p));
  carve(&off, sizeof(DevState));
  carve(&off, sizeof(float) * (size_t)nTiles * 2 * T);
  carve(&off, sizeof(float4) * nTiles);
  carve(&off, sizeof(float) * (size_t)nGroups * 2 * T);
  carve(&off, sizeof(float4) * nGroups);
  carve(&off, sizeof(unsigned) * 2 * (nGroups + 1));
  carve(&off, sizeof(double) * K);
  carve(&off, (size_t)K);
  carve(&off, sizeof(double) * 2 * T);
  carve(&off, (size_t)align_up(24 * (Jcap > 0 ? Jcap : 1), 16));
  return off;
}

void slot_layout(mppi_batch* b, BatchSlot& s, mppi_ctx* c) {
  const mppi_params* p = &s.p;
  const int T = p->T, K = p->K;
  const int nTiles = (K + s.tl.samples_per_cta - 1) / s.tl.samples_per_cta;
  const int GT = group_size(nTiles);
  const int nGroups = (nTiles + GT - 1) / GT;
  unsigned char* base = b->pool + s.off;
  size_t off = 0;
  c->d_U = (double*)(base + carve(&off, sizeof(double) * 2 * T));
  c->d_cU = (float2*)(base + carve(&off, sizeof(float2) * T));
  c->d_cA = (float2*)(base + carve(&off, sizeof(float2) * T));
  c->d_cw = (float*)(base + carve(&off, cw_bytes(p)));
  c->d_st = (DevState*)(base + carve(&off, sizeof(DevState)));
  c->d_part = (float*)(base + carve(&off, sizeof(float) * (size_t)nTiles * 2 * T));
  c->d_part_rz = (float4*)(base + carve(&off, sizeof(float4) * nTiles));
  c->d_gpart = (float*)(base + carve(&off, sizeof(float) * (size_t)nGroups * 2 * T));
  c->d_gpart_rz = (float4*)(base + carve(&off, sizeof(float4) * nGroups));
  c->d_cnt = (unsigned*)(base + carve(&off, sizeof(unsigned) * 2 * (nGroups + 1)));
  c->d_costs = (double*)(base + carve(&off, sizeof(double) * K));
  c->d_coll = (uint8_t*)(base + carve(&off, (size_t)K));
  c->d_Ustar = (double*)(base + carve(&off, sizeof(double) * 2 * T));
  s.obst_off = s.off + carve(&off, (size_t)align_up(24 * (s.Jcap > 0 ? s.Jcap : 1), 16));
  c->d_obst = (double*)(b->pool + s.obst_off);
  c->d_in = nullptr;
}

int batch_max_smem(mppi_batch* b) {
  if (b->max_smem == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    size_t stat = 0;
    if (cudaFuncGetAttributes(&fa, batch_kernel_all) == cudaSuccess) stat = fa.sharedSizeBytes;
    else cudaGetLastError();
    if (cudaFuncGetAttributes(&fa, batch_kernel) == cudaSuccess && fa.sharedSizeBytes > stat)
      stat = fa.sharedSizeBytes;
    else cudaGetLastError();
    b->max_smem = v - align_up((int)stat + 64, 128);
    cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, b->max_smem);
    cudaFuncSetAttribute(batch_kernel_all, cudaFuncAttributeMaxDynamicSharedMemorySize, b->max_smem);
  }
  return b->max_smem;
}

// Fill slot s's descriptor (device pointers into the pool) and upload it.
int batch_write_desc(mppi_batch* b, int slot) {
  BatchSlot& s = b->slots[slot];
  mppi_ctx c;
  c.p = s.p;
  c.n = s.n;
  c.tl = s.tl;
  slot_layout(b, s, &c);
  fill_desc(&c);
  c.D.J = s.J;
  s.D = c.D;
  CK(cudaMemcpy(b->d_descs + slot, &s.D, sizeof(CtrlDesc), cudaMemcpyHostToDevice));
  return MPPI_OK;
}

}  // namespace

extern "C" {

int mppi_batch_create(int32_t max_ctrl, size_t pool_bytes, mppi_batch** out) {
  if (!out) return fail(MPPI_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_ctrl < 1 || max_ctrl > (1 << 20)) return fail(MPPI_EINVAL, "max_ctrl out of range");
  if (pool_bytes < (1u << 20)) return fail(MPPI_EINVAL, "pool must be at least 1 MiB");
  mppi_batch* b = new (std::nothrow) mppi_batch();
  if (!b) return fail(MPPI_ENOMEM, "host allocation failed");
  b->max_ctrl = max_ctrl;
  b->slots.resize(max_ctrl);
  if (cudaMalloc((void**)&b->pool, pool_bytes) != cudaSuccess ||
      cudaMalloc((void**)&b->d_descs, sizeof(CtrlDesc) * max_ctrl) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->pool);
    cudaFree(b->d_descs);
    delete b;
    return fail(MPPI_ENOMEM, "device allocation of the batch pool failed");
  }
  b->pool_bytes = pool_bytes;
  b->free_list.push_back({0, pool_bytes});
  batch_max_smem(b);
  *out = b;
  return MPPI_OK;
}

int mppi_batch_add(mppi_batch* b, const mppi_params* p, const double* u_init,
                   const mppi_tiling* tiling, const double* cxcyr, int32_t J, int32_t* slot_out) {
  if (!b) return fail(MPPI_ESTATE, "batch is NULL");
  if (!slot_out) return fail(MPPI_EINVAL, "slot is NULL");
  int rc = validate(p);
  if (rc) return rc;
  if (u_init && !finite_all(u_init, 2 * p->T)) return fail(MPPI_EINVAL, "non-finite u_init");
  if (J < 0 || J > MPPI_MAX_OBSTACLES)
    return fail(MPPI_EINVAL, "J=%d out of [0, %d]", J, MPPI_MAX_OBSTACLES);
  if (J > 0 && !cxcyr) return fail(MPPI_EINVAL, "obstacles pointer is NULL");
  for (int j = 0; j < J; ++j) {
    if (int rc = check_obstacle(cxcyr + 3 * j, j)) return rc;
  }
  int slot = -1;
  for (int i = 0; i < b->max_ctrl; ++i)
    if (!b->slots[i].used) {
      slot = i;
      break;
    }
  if (slot < 0) return fail(MPPI_ENOMEM, "all %d slots are in use", b->max_ctrl);
  BatchSlot& s = b->slots[slot];
  s = BatchSlot();
  s.p = *p;
  s.n = state_dim(p->model);
  mppi_tiling req = {0, kBatchThreads, 0, 0};
  if (tiling) {
    req = *tiling;
    req.threads = kBatchThreads;
  } else {  // the batch's policy for this model
    req.samples_per_cta = b->pol.samples_per_cta[p->model];
    req.positions_per_thread = b->pol.positions_per_thread[p->model];
    if (req.positions_per_thread > 0 && req.positions_per_thread < p->n_shape)
      req.positions_per_thread = 0;
  }
  if (req.samples_per_cta <= 0) req.samples_per_cta = 32;
  if (req.samples_per_cta > p->K) req.samples_per_cta = p->K;
  int smem = 0;
  rc = choose_tiling(p, &req, J, &s.tl, &smem, true);
  if (rc) return rc;
  if (smem > batch_max_smem(b)) return fail(MPPI_EINVAL, "controller too large for the batch kernel");
  s.J = J;
  s.Jcap = J;
  s.bytes = slot_bytes(p, &s.tl, s.Jcap);
  if (!pool_alloc(b, s.bytes, &s.off))
    return fail(MPPI_ENOMEM, "admission refused: the slot needs %zu bytes of the batch pool",
                s.bytes);
  s.used = true;
  s.smem = smem;
  rc = batch_write_desc(b, slot);
  if (rc) {
    pool_free(b, s.off, s.bytes);
    s.used = false;
    return rc;
  }
  DevState st;
  memset(&st, 0, sizeof(st));
  st.S_e = p->mu_coarse > 0 ? p->mu_coarse : 1.0;
  st.first = 1;
  std::vector<double> U(2 * p->T, 0.0);
  if (u_init) memcpy(U.data(), u_init, sizeof(double) * 2 * p->T);
  const int nGroups = s.D.nGroups;
  bool up = cudaMemcpy(s.D.U, U.data(), sizeof(double) * 2 * p->T, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(s.D.st, &st, sizeof(DevState), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(s.D.counters, 0, sizeof(unsigned) * 2 * (nGroups + 1)) == cudaSuccess;
  if (up && J > 0)
    up = cudaMemset(b->pool + s.obst_off, 0, (size_t)align_up(24 * J, 16)) == cudaSuccess &&
         cudaMemcpy(b->pool + s.obst_off, cxcyr, sizeof(double) * 3 * J, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!up) {
    pool_free(b, s.off, s.bytes);
    s.used = false;
    return fail(MPPI_ECUDA, "slot initialisation failed");
  }
  prep_kernel<<<1, 256, 0, b->own>>>(s.D, 1);
  if (cudaStreamSynchronize(b->own) != cudaSuccess) {
    pool_free(b, s.off, s.bytes);
    s.used = false;
    return fail(MPPI_ECUDA, "slot prep failed");
  }
  s.tile_cost = (double)s.tl.samples_per_cta * p->T * (8.0 * p->n_shape * (J > 0 ? J : 1) + 135.0);
  drop_graph(b);
  *slot_out = slot;
  return MPPI_OK;
}

int mppi_batch_set_obstacles(mppi_batch* b, int32_t slot, const double* cxcyr, int32_t J) {
  if (!b) return fail(MPPI_ESTATE, "batch is NULL");
  if (slot < 0 || slot >= b->max_ctrl || !b->slots[slot].used)
    return fail(MPPI_EINVAL, "slot %d is not in use", slot);
  if (J < 0 || J > MPPI_MAX_OBSTACLES)
    return fail(MPPI_EINVAL, "J=%d out of [0, %d]", J, MPPI_MAX_OBSTACLES);
  if (J > 0 && !cxcyr) return fail(MPPI_EINVAL, "obstacles pointer is NULL");
  for (int j = 0; j < J; ++j) {
    if (int rc = check_obstacle(cxcyr + 3 * j, j)) return rc;
  }
  BatchSlot& s = b->slots[slot];
  mppi_tiling t;
  int smem = 0;
  int rc = choose_tiling(&s.p, &s.tl, J, &t, &smem, true);
  if (rc) return rc;
  if (smem > batch_max_smem(b)) return fail(MPPI_EINVAL, "obstacle set too large");
  if (b->lane.last) CK(cudaStreamSynchronize(b->lane.last));
  if (J > s.Jcap) {
    // grow the slot: a new range holding the state and the larger obstacle area
    const size_t nbytes = slot_bytes(&s.p, &s.tl, J);
    size_t noff = 0;
    if (!pool_alloc(b, nbytes, &noff))
      return fail(MPPI_ENOMEM, "admission refused: %zu bytes for the obstacle set", nbytes);
    CK(cudaMemcpy(b->pool + noff, b->pool + s.off, s.bytes, cudaMemcpyDeviceToDevice));
    pool_free(b, s.off, s.bytes);
    s.off = noff;
    s.bytes = nbytes;
    s.Jcap = J;
  }
  s.J = J;
  s.smem = smem;
  rc = batch_write_desc(b, slot);
  if (rc) return rc;
  if (J > 0) {
    CK(cudaMemset(b->pool + s.obst_off, 0, (size_t)align_up(24 * J, 16)));
    CK(cudaMemcpy(b->pool + s.obst_off, cxcyr, sizeof(double) * 3 * J, cudaMemcpyHostToDevice));
  }
  s.tile_cost = (double)s.tl.samples_per_cta * s.p.T * (8.0 * s.p.n_shape * (J > 0 ? J : 1) + 135.0);
  drop_graph(b);
  return MPPI_OK;
}

int mppi_batch_remove(mppi_batch* b, int32_t slot) {
  if (!b) return fail(MPPI_ESTATE, "batch is NULL");
  if (slot < 0 || slot >= b->max_ctrl || !b->slots[slot].used)
    return fail(MPPI_EINVAL, "slot %d is not in use", slot);
  if (b->lane.last) CK(cudaStreamSynchronize(b->lane.last));
  BatchSlot& s = b->slots[slot];
  pool_free(b, s.off, s.bytes);
  s.used = false;
  drop_graph(b);
  return MPPI_OK;
}

}  // extern "C"

namespace {

// One batched step of the listed slots on lane L and stream st: pack, copy
// in, launch, copy out; graph replay when allowed and the composition is the
// one captured.  Slot bookkeeping must not change concurrently.  share < 1
// caps the persistent kernel's CTAs at that fraction of the resident CTAs
// the GPU holds (the serving runtime leaves the rest of the SMs to its other
// size class); results do not depend on it.
int lane_step(mppi_batch* b, BatchLane& L, const int32_t* slots, int32_t n, const double* x0s,
              const double* const* xrefs, cudaStream_t st, bool allow_graph, double share = 1.0) {
  size_t n_items = 0, n_in = 0;
  int smem = 0;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) {
    const int sl = slots[i];
    if (sl < 0 || sl >= b->max_ctrl || !b->slots[sl].used)
      return fail(MPPI_EINVAL, "slot %d is not in use", sl);
    for (int k = 0; k < i; ++k)
      if (slots[k] == sl) return fail(MPPI_EINVAL, "slot %d listed twice", sl);
    const BatchSlot& s = b->slots[sl];
    n_items += s.D.nTiles;
    n_in += (size_t)s.n * (s.p.T + 2);
    smem = std::max(smem, s.smem);
    order[i] = i;
  }
  const size_t head = sizeof(BatchHdr) + sizeof(StepEntry) * n + sizeof(WorkItem) * n_items;
  const size_t inputs_off = (head + 15) & ~(size_t)15;
  const size_t bytes = inputs_off + sizeof(double) * n_in;
  if (L.last) CK(cudaStreamSynchronize(L.last));
  if (int rc = lane_reserve(L, bytes, n)) return rc;
  // pack: header, step table, longest-first work items, inputs
  BatchHdr* hdr = (BatchHdr*)L.h_stage;
  StepEntry* steps = (StepEntry*)(L.h_stage + sizeof(BatchHdr));
  WorkItem* items = (WorkItem*)(steps + n);
  double* in = (double*)(L.h_stage + inputs_off);
  std::sort(order.begin(), order.end(), [&](int a, int c) {
    return b->slots[slots[a]].tile_cost > b->slots[slots[c]].tile_cost;
  });
  size_t w = 0, d = 0;
  for (int i = 0; i < n; ++i) {
    const BatchSlot& s = b->slots[slots[i]];
    const int nn = s.n, T = s.p.T;
    const double* x0 = x0s + (size_t)i * 6;
    if (!finite_all(x0, nn)) return fail(MPPI_EINVAL, "x0 of slot %d is not finite", slots[i]);
    steps[i].slot = slots[i];
    steps[i].x0_off = (int)d;
    memcpy(in + d, x0, sizeof(double) * nn);
    d += nn;
    steps[i].xref_off = (int)d;
    const double* xr = xrefs ? xrefs[i] : nullptr;
    if (xr && !finite_all(xr, (T + 1) * nn))
      return fail(MPPI_EINVAL, "xref of slot %d is not finite", slots[i]);
    for (int t = 0; t <= T; ++t)
      for (int k = 0; k < nn; ++k) in[d + t * nn + k] = xr ? xr[t * nn + k] : s.p.x_goal[k];
    d += (size_t)(T + 1) * nn;
  }
  for (int oi = 0; oi < n; ++oi) {
    const int i = order[oi];
    const BatchSlot& s = b->slots[slots[i]];
    for (int t = 0; t < s.D.nTiles; ++t) items[w++] = WorkItem{i, t};
  }
  hdr->n_steps = n;
  hdr->n_items = (int)n_items;
  hdr->next = 0u;
  hdr->inputs_off = (int)inputs_off;
  // batch_kernel covers the unicycle and the 6-state quadrotor; a step that
  // holds the Ackermann vehicle or the 5-state quadrotor takes batch_kernel_all
  bool all_models = false;
  for (int i = 0; i < n; ++i) all_models = all_models || b->slots[slots[i]].p.model >= 2;
  const auto kernel = all_models ? batch_kernel_all : batch_kernel;
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kBatchThreads, smem));
  if (occ < 1) return fail(MPPI_EINVAL, "batch needs %d bytes of shared memory per CTA", smem);
  int grid = (int)std::min<size_t>((size_t)num_sms() * occ, n_items);
  if (share < 1.0) grid = std::max(1, std::min(grid, (int)(share * num_sms() * occ)));
  std::vector<int> key(slots, slots + n);
  const bool same = allow_graph && L.gexec && key == L.graph_key && bytes == L.graph_bytes &&
                    smem == L.graph_smem && grid == L.graph_grid && st == L.last;
  if (same) {
    CK(cudaGraphLaunch(L.gexec, st));
  } else {
    drop_lane_graph(L);
    if (allow_graph) CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    // every call checked; once a capture has begun it is ended on every path
    cudaError_t e = cudaMemcpyAsync(L.d_stage, L.h_stage, bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      kernel<<<grid, kBatchThreads, smem, st>>>(b->d_descs, L.d_stage, L.d_out);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(L.h_out, L.d_out, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost, st);
    if (allow_graph) {
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(st, &g);
      if (e == cudaSuccess) e = ec;
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(MPPI_ECUDA, "batched step capture failed: %s", cudaGetErrorString(e));
      }
      L.graph = g;
      e = cudaGraphInstantiate(&L.gexec, L.graph, 0);
      if (e != cudaSuccess) {
        cudaGetLastError();
        drop_lane_graph(L);
        return fail(MPPI_ECUDA, "batched step graph instantiation failed: %s",
                    cudaGetErrorString(e));
      }
      L.graph_key = key;
      L.graph_bytes = bytes;
      L.graph_smem = smem;
      L.graph_grid = grid;
      CK(cudaGraphLaunch(L.gexec, st));
    } else if (e != cudaSuccess) {
      return fail(MPPI_ECUDA, "batched step launch failed: %s", cudaGetErrorString(e));
    }
  }
  L.last = st;
  L.n_last = n;
  return MPPI_OK;
}

}  // namespace

extern "C" {

int mppi_batch_step(mppi_batch* b, const int32_t* slots, int32_t n, const double* x0s,
                    const double* const* xrefs, void* stream) {
  if (!b) return fail(MPPI_ESTATE, "batch is NULL");
  if (n < 0 || (n > 0 && (!slots || !x0s))) return fail(MPPI_EINVAL, "bad slot list");
  cudaStream_t st = stream ? (cudaStream_t)stream : b->own;
  if (n == 0) return MPPI_OK;
  return lane_step(b, b->lane, slots, n, x0s, xrefs, st, b->use_graph != 0);
}

int mppi_batch_get_controls(mppi_batch* b, double* u0s, int32_t n) {
  if (!b) return fail(MPPI_ESTATE, "batch is NULL");
  BatchLane& L = b->lane;
  if (n != L.n_last) return fail(MPPI_EINVAL, "n=%d but the last step had %d controllers", n, L.n_last);
  if (L.last) CK(cudaStreamSynchronize(L.last));
  for (int i = 0; u0s && i < n; ++i) {
    u0s[2 * i] = L.h_out[8 * i];
    u0s[2 * i + 1] = L.h_out[8 * i + 1];
  }
  return MPPI_OK;
}

int mppi_batch_get_state(mppi_batch* b, int32_t slot, double* U, double* costs, double* scalars) {
  if (!b) return fail(MPPI_ESTATE, "batch is NULL");
  if (slot < 0 || slot >= b->max_ctrl || !b->slots[slot].used)
    return fail(MPPI_EINVAL, "slot %d is not in use", slot);
  if (b->lane.last) CK(cudaStreamSynchronize(b->lane.last));
  const BatchSlot& s = b->slots[slot];
  if (U) CK(cudaMemcpy(U, s.D.U, sizeof(double) * 2 * s.p.T, cudaMemcpyDeviceToHost));
  if (costs) CK(cudaMemcpy(costs, s.D.costs, sizeof(double) * s.p.K, cudaMemcpyDeviceToHost));
  if (scalars) {
    DevState st;
    CK(cudaMemcpy(&st, s.D.st, sizeof(DevState), cudaMemcpyDeviceToHost));
    scalars[0] = st.rho;
    scalars[1] = st.Z;
    scalars[2] = st.CB_star;
    scalars[3] = st.S_e;
    scalars[4] = st.beta_used;
    scalars[5] = st.beta_d;
    scalars[6] = st.S_e_used;
    scalars[7] = (double)st.iter;
    if (st.status == kStatusTimeout)
      return fail(MPPI_ETIMEOUT, "a bounded device wait (obstacle staging) expired");
  }
  return MPPI_OK;
}

int mppi_batch_info(mppi_batch* b, int32_t slot, mppi_tiling* t, uint64_t* bytes,
                    uint64_t* pool_free_bytes) {
  if (!b) return fail(MPPI_ESTATE, "batch is NULL");
  if (slot >= 0) {
    if (slot >= b->max_ctrl || !b->slots[slot].used)
      return fail(MPPI_EINVAL, "slot %d is not in use", slot);
    if (t) *t = b->slots[slot].tl;
    if (bytes) *bytes = b->slots[slot].bytes;
  }
  if (pool_free_bytes) {
    size_t f = 0;
    for (auto& e : b->free_list) f += e.second;
    *pool_free_bytes = f;
  }
  return MPPI_OK;
}

int mppi_batch_set_graph(mppi_batch* b, int32_t enable) {
  if (!b) return fail(MPPI_ESTATE, "batch is NULL");
  if (b->lane.last) CK(cudaStreamSynchronize(b->lane.last));
  drop_graph(b);
  b->use_graph = enable ? 1 : 0;
  return MPPI_OK;
}

int mppi_batch_set_policy(mppi_batch* b, const mppi_batch_policy* pol) {
  if (!b) return fail(MPPI_ESTATE, "batch is NULL");
  if (!pol) return fail(MPPI_EINVAL, "policy is NULL");
  for (int m = 0; m < MPPI_NUM_MODELS; ++m) {
    if (pol->samples_per_cta[m] < 1 || pol->samples_per_cta[m] > 32)
      return fail(MPPI_EINVAL, "samples_per_cta must be in 1..32");
    const int np = pol->positions_per_thread[m];
    if (np != 0 && np != 8 && np != 14)
      return fail(MPPI_EINVAL, "positions_per_thread must be 0, 8 or 14");
  }
  b->pol = *pol;
  return MPPI_OK;
}

int mppi_batch_get_policy(const mppi_batch* b, mppi_batch_policy* pol) {
  if (!b) return fail(MPPI_ESTATE, "batch is NULL");
  if (!pol) return fail(MPPI_EINVAL, "policy is NULL");
  *pol = b->pol;
  return MPPI_OK;
}

int mppi_batch_destroy(mppi_batch* b) {
  if (!b) return MPPI_OK;
  free_lane(b->lane);
  cudaFree(b->pool);
  cudaFree(b->d_descs);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
  return MPPI_OK;
}

// Time `iters` batched steps of n controllers added under policy pol to a
// fresh batch of pool_bytes; false if a controller does not fit.
static bool time_policy(const mppi_params* ps, const double* const* cxcyrs, const int32_t* Js,
                        int32_t n, int32_t iters, size_t pool_bytes, const mppi_batch_policy& pol,
                        const std::vector<double>& x0s, float* ms_out, int* rc_out) {
  mppi_batch* b = nullptr;
  *rc_out = mppi_batch_create(n, pool_bytes, &b);
  if (*rc_out) return false;
  bool ok = mppi_batch_set_policy(b, &pol) == MPPI_OK;
  std::vector<int32_t> slots(n);
  for (int i = 0; i < n && ok; ++i) {
    const int rc = mppi_batch_add(b, &ps[i], nullptr, nullptr, cxcyrs ? cxcyrs[i] : nullptr,
                                  Js ? Js[i] : 0, &slots[i]);
    if (rc) {
      *rc_out = rc;
      ok = false;
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ok) ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  for (int w = 0; w < 2 && ok; ++w)
    ok = mppi_batch_step(b, slots.data(), n, x0s.data(), nullptr, nullptr) == MPPI_OK;
  if (ok) ok = cudaStreamSynchronize(b->own) == cudaSuccess;
  if (ok) {
    cudaEventRecord(e0, b->own);
    for (int i = 0; i < iters && ok; ++i)
      ok = mppi_batch_step(b, slots.data(), n, x0s.data(), nullptr, nullptr) == MPPI_OK;
    cudaEventRecord(e1, b->own);
    ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.0f;
    if (ok) cudaEventElapsedTime(&ms, e0, e1);
    *ms_out = ms / (float)iters;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  mppi_batch_destroy(b);
  return ok;
}

int mppi_batch_autotune(const mppi_params* ps, const double* const* cxcyrs, const int32_t* Js,
                        int32_t n, int32_t iters, size_t pool_bytes, mppi_batch_policy* best,
                        float* best_ms) {
  if (!ps || n < 1 || !best) return fail(MPPI_EINVAL, "bad controller list or output");
  if (iters < 1) iters = 3;
  std::vector<double> x0s((size_t)6 * n, 0.0);  // n x 6, each from its goal state
  for (int i = 0; i < n; ++i) {
    if (int rc = validate(&ps[i])) return rc;
    for (int d = 0; d < 6; ++d) x0s[(size_t)i * 6 + d] = ps[i].x_goal[d];
  }
  mppi_batch_policy cur = {{32, 32, 32, 32}, {0, 0, 0, 0}};
  float cur_ms = 0.0f;
  int rc = 0;
  if (!time_policy(ps, cxcyrs, Js, n, iters, pool_bytes, cur, x0s, &cur_ms, &rc))
    return rc ? rc : fail(MPPI_ECUDA, "timing the default policy failed");
  const int S_opts[3] = {8, 16, 32};
  const int NP_opts[2] = {8, 14};
  for (int m = 0; m < MPPI_NUM_MODELS; ++m) {
    bool present = false;
    for (int i = 0; i < n; ++i) present = present || ps[i].model == m;
    if (!present) continue;
    for (int S : S_opts)
      for (int NP : NP_opts) {
        mppi_batch_policy cand = cur;
        cand.samples_per_cta[m] = S;
        cand.positions_per_thread[m] = NP;
        if (S == cur.samples_per_cta[m] && NP == cur.positions_per_thread[m]) continue;
        float ms = 0.0f;
        int crc = 0;
        if (time_policy(ps, cxcyrs, Js, n, iters, pool_bytes, cand, x0s, &ms, &crc) && ms < cur_ms) {
          cur = cand;
          cur_ms = ms;
        }
        cudaGetLastError();
      }
  }
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return MPPI_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Serving runtime: continuous batching of control-step requests from many
// robots.  Robots join by taking a slot of the device pool (admission by
// memory); their warm-start sequence, generator counter, exploration rate
// and barrier state stay on the device between requests.  Requests are sorted
// by size into two classes, each with its own queue and lanes: a lane is one
// batched step in flight on its own stream.  When a lane is free it launches
// one persistent batch of the requests queued in its class, oldest first, up
// to the class's work cap, so requests that arrive while others run join the
// next batch and the batches of both classes overlap on the device.  The
// large-request lanes cap their kernels' CTAs at a share of the GPU, which
// leaves SMs free for the small requests: a small request does not wait for
// a running batch of large ones.  Completions carry u*_0, the model's
// prediction of the next state, the latency from submission, and its split
// into time queued (submission to launch) and the batch's device time.

namespace {

struct ServerReq {
  int robot;
  int cls;                   // size class: 0 small, 1 large
  double ops;                // work estimate (FP32 operations)
  double x0[6];
  std::vector<double> xref;  // empty: goal repeated
  std::chrono::steady_clock::time_point t0, t_launch;
};

struct ServerDone {
  int robot;
  double out[8];  // u0[2], x1[6]
  double latency, queue, device;
  int cls;
  int status;
};

// A request published to the resident kernel's rings (device-queue mode).
struct RingReq {
  ServerReq r;
  int rq = 0;              // request slot of the rings
  unsigned seq = 0;        // its sequence number (done word: seq + 1)
  int cls = 0;
  double ops = 0.0;
  unsigned item_begin = 0;  // its items: [item_begin, item_begin + nTiles) of its class
  std::chrono::steady_clock::time_point t_publish;
  bool done = false;
};

// The resident kernel's rings and the scheduler's view of them; only the
// scheduler thread touches it after set-up.
struct ServeState {
  bool ready = false;
  ServeHdr* h_hdr = nullptr;
  ServeHdr* d_hdr = nullptr;
  WorkItem* h_items[2] = {nullptr, nullptr};
  WorkItem* d_items[2] = {nullptr, nullptr};
  ServeReq* h_reqs = nullptr;
  ServeReq* d_reqs = nullptr;
  double* h_in = nullptr;
  double* d_in = nullptr;
  double* h_out = nullptr;
  double* d_out = nullptr;
  unsigned* h_done = nullptr;
  unsigned* d_done = nullptr;
  unsigned* d_next = nullptr;  // device memory: items claimed per class
  unsigned cap_items = 0;
  int cap_reqs = 0, in_stride = 0, max_dyn = 0;
  unsigned pub[2] = {0, 0};  // items published per class
  double flight_ops[2] = {0.0, 0.0};  // work published and not yet complete, per class
  unsigned seq = 0;
  std::chrono::steady_clock::time_point last_busy;  // last pass with work queued or in flight
  std::vector<int> free_rq;
  std::deque<RingReq> flight[2];  // published requests per class, in publish order
  int n_flight = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool running = false, closing = false, failed = false;
  int k_smem = 0;
  bool k_all = false;
};

// Work of one step of a slot: K T (7 P J + 135) FP32 operations (the
// barrier's pairs dominate), the measure the size classes and caps use.
double slot_ops(const BatchSlot& s) {
  return (double)s.p.K * s.p.T * (7.0 * s.p.n_shape * s.J + 135.0);
}

}  // namespace

struct mppi_server {
  mppi_batch* b = nullptr;
  int max_robots = 0;
  std::vector<BatchLane> lanes;
  std::vector<int> lane_cls;  // class a lane serves
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev_start, events;  // per lane: launch and completion
  std::vector<std::vector<ServerReq>> inflight;
  std::vector<char> lane_busy;
  std::mutex mu;       // queues, completions, robot flags and the policy
  std::mutex slot_mu;  // the pool's slot bookkeeping (join, leave), apart from the
                       // scheduler so that a join's uploads never stall a launch
  std::deque<ServerReq> queue[2];
  std::deque<ServerDone> done;
  std::vector<char> joined, busy;
  mppi_server_policy pol;
  std::thread worker;
  std::atomic<bool> stop{false};
  std::atomic<unsigned long long> batches{0}, requests{0};
  std::atomic<int> n_inflight{0};
  int device = 0;  // the device current at mppi_server_create, where the pool lives
  int max_slot_smem = 0;  // largest shared memory of a joined robot's tiles (never lowered)
  bool any_all = false;   // a joined robot needs the four-model kernel (never cleared)
  ServeState ring;        // device-queue mode
  std::atomic<bool> dq{false};  // the policy's device_queue, read by the scheduler
  char err[512] = "";
};

namespace {

// Lane roles under a policy: with small_ops_max > 0 and two or more lanes,
// the first small_lanes serve the small class and the rest the large class;
// otherwise every lane serves one queue (class 0).
void assign_lanes(mppi_server* sv) {
  const int n = (int)sv->lanes.size();
  const bool classes = sv->pol.small_ops_max > 0 && n >= 2;
  int ns = classes ? std::min(std::max(sv->pol.small_lanes, 1), n - 1) : n;
  for (int i = 0; i < n; ++i) sv->lane_cls[i] = i < ns ? 0 : 1;
}

// ---- device-queue mode: the resident kernel's rings

constexpr unsigned kRingItems = 1u << 21;  // items per class ring (a power of two)
// The resident kernel's CTAs exit when the host closes the kernel, which it
// does after kServeIdleClose with nothing queued or in flight (CTAs leaving
// one by one would leave a running kernel with too few CTAs for the work
// that arrives next).  On the device each idle wait is still bounded:
// kServeIdlePolls polls kServeIdleNs apart, about 2 s, after which a CTA
// exits on its own.
constexpr int kServeIdlePolls = 400000;
constexpr int kServeIdleNs = 5000;
constexpr double kServeIdleClose = 3e-4;  // seconds

template <class T>
bool mapped_alloc(T** h, T** d, size_t n) {
  if (cudaHostAlloc((void**)h, sizeof(T) * n, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)d, *h, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  memset(*h, 0, sizeof(T) * n);
  return true;
}

// Stop the resident kernel (if any) and release the rings.
void ring_free(ServeState& R) {
  if (R.running) {
    *reinterpret_cast<volatile unsigned*>(&R.h_hdr->closed) = 1u;
    cudaStreamSynchronize(R.stream);
    R.running = false;
  }
  cudaFreeHost(R.h_hdr);
  for (int c = 0; c < 2; ++c) cudaFreeHost(R.h_items[c]);
  cudaFreeHost(R.h_reqs);
  cudaFreeHost(R.h_in);
  cudaFreeHost(R.h_out);
  cudaFreeHost(R.h_done);
  cudaFree(R.d_next);
  if (R.ev) cudaEventDestroy(R.ev);
  if (R.stream) cudaStreamDestroy(R.stream);
  R = ServeState();
}

// Rings for up to max_robots requests in flight (one per robot).
int ring_alloc(mppi_server* sv) {
  ServeState& R = sv->ring;
  if (R.ready) return MPPI_OK;
  R.cap_items = kRingItems;
  R.cap_reqs = sv->max_robots;
  R.in_stride = (MPPI_MAX_T + 2) * kMaxN;
  bool ok = mapped_alloc(&R.h_hdr, &R.d_hdr, 1) && mapped_alloc(&R.h_items[0], &R.d_items[0], R.cap_items) &&
            mapped_alloc(&R.h_items[1], &R.d_items[1], R.cap_items) &&
            mapped_alloc(&R.h_reqs, &R.d_reqs, (size_t)R.cap_reqs) &&
            mapped_alloc(&R.h_in, &R.d_in, (size_t)R.cap_reqs * R.in_stride) &&
            mapped_alloc(&R.h_out, &R.d_out, (size_t)R.cap_reqs * 8) &&
            mapped_alloc(&R.h_done, &R.d_done, (size_t)R.cap_reqs);
  ok = ok && cudaMalloc((void**)&R.d_next, 2 * sizeof(unsigned)) == cudaSuccess &&
       cudaMemset(R.d_next, 0, 2 * sizeof(unsigned)) == cudaSuccess &&
       cudaStreamCreateWithFlags(&R.stream, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&R.ev, cudaEventDisableTiming) == cudaSuccess;
  if (ok) {
    // dynamic shared memory the serving kernels may take beside their own
    // static staging of the inputs
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    size_t stat = 0;
    for (auto k : {serve_kernel, serve_kernel_all})
      if (cudaFuncGetAttributes(&fa, k) == cudaSuccess && fa.sharedSizeBytes > stat)
        stat = fa.sharedSizeBytes;
    R.max_dyn = optin - align_up((int)stat + 64, 128);
    ok = R.max_dyn > 0 &&
         cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, R.max_dyn) ==
             cudaSuccess &&
         cudaFuncSetAttribute(serve_kernel_all, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              R.max_dyn) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    ring_free(R);
    return fail(MPPI_ENOMEM, "device queue: allocation of its rings failed");
  }
  for (int i = R.cap_reqs - 1; i >= 0; --i) R.free_rq.push_back(i);
  R.ready = true;
  return MPPI_OK;
}

// One pass of the device-queue scheduler: completions, publication of
// queued requests, and a launch of the resident kernel when work is
// published and none runs.  Returns whether anything happened.
bool ring_step(mppi_server* sv, bool dev_ok) {
  ServeState& R = sv->ring;
  bool did = false;
  if (R.running) {
    const cudaError_t q = cudaEventQuery(R.ev);
    if (q != cudaErrorNotReady) {
      R.running = false;
      R.closing = false;  // a request held back for a larger kernel is published below
      if (q != cudaSuccess) {
        R.failed = true;
        snprintf(sv->err, sizeof(sv->err), "resident serving kernel: %s", cudaGetErrorString(q));
        cudaGetLastError();
      }
      did = true;
    }
  }
  const auto now = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> g(sv->mu);
  // completions: a done word equal to the request's sequence number + 1
  // follows its outputs (system-scope fence in the kernel)
  if (R.n_flight > 0) {
    for (int c = 0; c < 2; ++c) {
      for (RingReq& x : R.flight[c]) {
        if (x.done) continue;
        const bool ok = *reinterpret_cast<volatile unsigned*>(&R.h_done[x.rq]) == x.seq + 1u;
        if (!ok && !(R.failed && !R.running)) continue;
        std::atomic_thread_fence(std::memory_order_acquire);
        ServerDone d;
        d.robot = x.r.robot;
        for (int k = 0; k < 8; ++k) d.out[k] = ok ? R.h_out[8 * (size_t)x.rq + k] : NAN;
        d.latency = std::chrono::duration<double>(now - x.r.t0).count();
        d.queue = std::chrono::duration<double>(x.t_publish - x.r.t0).count();
        d.device = std::chrono::duration<double>(now - x.t_publish).count();
        d.cls = x.cls;
        d.status = ok ? MPPI_OK : MPPI_ECUDA;
        sv->done.push_back(d);
        sv->busy[x.r.robot] = 0;
        sv->n_inflight--;
        sv->requests++;
        x.done = true;
        R.free_rq.push_back(x.rq);
        R.n_flight--;
        R.flight_ops[c] -= x.ops;
        if (R.n_flight == 0) R.flight_ops[0] = R.flight_ops[1] = 0.0;  // no drift
        did = true;
      }
      while (!R.flight[c].empty() && R.flight[c].front().done) R.flight[c].pop_front();
    }
  }
  // publication, small class first: each request's inputs and entry, then
  // its items, then (release) the class's published count
  bool pub_any[2] = {false, false};
  for (int c = 0; c < 2 && !R.failed; ++c) {
    std::deque<ServerReq>& qu = sv->queue[c];
    // the requests held on the host are published least work first (the
    // age limit first), up to the class's cap on published, unfinished work
    const double cap = c == 0 ? sv->pol.batch_ops_small : sv->pol.batch_ops_large;
    if (sv->pol.shortest_first && qu.size() > 1) {
      const double lim = sv->pol.max_wait_s;
      std::stable_sort(qu.begin(), qu.end(), [&](const ServerReq& a, const ServerReq& b2) {
        const bool oa = lim > 0 && std::chrono::duration<double>(now - a.t0).count() > lim;
        const bool ob = lim > 0 && std::chrono::duration<double>(now - b2.t0).count() > lim;
        if (oa != ob) return oa;
        if (oa) return a.t0 < b2.t0;
        return a.ops < b2.ops;
      });
    }
    while (!qu.empty() && !R.closing) {
      ServerReq& r = qu.front();
      if (cap > 0 && R.flight_ops[c] > 0 && R.flight_ops[c] + r.ops > cap) break;
      const BatchSlot& s = sv->b->slots[r.robot];
      const unsigned nt = (unsigned)s.D.nTiles;
      if (s.smem > R.max_dyn) {  // cannot run in the serving kernel at all
        ServerDone d;
        d.robot = r.robot;
        for (int k = 0; k < 8; ++k) d.out[k] = NAN;
        d.latency = d.queue = std::chrono::duration<double>(now - r.t0).count();
        d.device = 0.0;
        d.cls = c;
        d.status = MPPI_EINVAL;
        sv->done.push_back(d);
        sv->busy[r.robot] = 0;
        sv->n_inflight--;
        qu.pop_front();
        continue;
      }
      if (R.running && (s.smem > R.k_smem || (s.p.model >= 2 && !R.k_all))) {
        // the running kernel was launched for smaller tiles or fewer models:
        // let it finish what it has claimed, then launch one that fits
        R.closing = true;
        *reinterpret_cast<volatile unsigned*>(&R.h_hdr->closed) = 1u;
        break;
      }
      const unsigned wm = R.flight[c].empty() ? R.pub[c] : R.flight[c].front().item_begin;
      if (R.free_rq.empty() || R.pub[c] + nt - wm > R.cap_items) break;  // rings full
      const int rq = R.free_rq.back();
      R.free_rq.pop_back();
      const int n = s.n, T = s.p.T;
      double* in = R.h_in + (size_t)rq * R.in_stride;
      memcpy(in, r.x0, sizeof(double) * n);
      if (!r.xref.empty()) {
        memcpy(in + n, r.xref.data(), sizeof(double) * (size_t)(T + 1) * n);
      } else {
        for (int t = 0; t <= T; ++t) memcpy(in + n + (size_t)t * n, s.p.x_goal, sizeof(double) * n);
      }
      R.h_reqs[rq] = ServeReq{r.robot, n, n * (T + 2), R.seq};
      WorkItem* items = R.h_items[c];
      for (unsigned t = 0; t < nt; ++t)
        items[(R.pub[c] + t) & (R.cap_items - 1u)] = WorkItem{rq, (int)t};
      RingReq x;
      x.r = std::move(r);
      x.rq = rq;
      x.seq = R.seq++;
      x.cls = c;
      x.ops = x.r.ops;
      x.item_begin = R.pub[c];
      x.t_publish = now;
      R.flight_ops[c] += x.ops;
      R.pub[c] += nt;
      R.flight[c].push_back(std::move(x));
      R.n_flight++;
      qu.pop_front();
      pub_any[c] = true;
      did = true;
    }
  }
  if (R.failed) {  // a failed kernel leaves nothing to run the queued requests
    for (int c = 0; c < 2; ++c) {
      for (ServerReq& r : sv->queue[c]) {
        ServerDone d;
        d.robot = r.robot;
        for (int k = 0; k < 8; ++k) d.out[k] = NAN;
        d.latency = d.queue = std::chrono::duration<double>(now - r.t0).count();
        d.device = 0.0;
        d.cls = c;
        d.status = MPPI_ECUDA;
        sv->done.push_back(d);
        sv->busy[r.robot] = 0;
        sv->n_inflight--;
        did = true;
      }
      sv->queue[c].clear();
    }
  }
  if (pub_any[0] || pub_any[1]) {
    std::atomic_thread_fence(std::memory_order_seq_cst);
    for (int c = 0; c < 2; ++c)
      if (pub_any[c]) *reinterpret_cast<volatile unsigned*>(&R.h_hdr->published[c]) = R.pub[c];
  }
  // close the kernel once it has had nothing to do for a while
  const bool busy = R.n_flight > 0 || !sv->queue[0].empty() || !sv->queue[1].empty();
  if (busy) R.last_busy = now;
  if (R.running && !R.closing && !busy &&
      std::chrono::duration<double>(now - R.last_busy).count() > kServeIdleClose) {
    R.closing = true;
    *reinterpret_cast<volatile unsigned*>(&R.h_hdr->closed) = 1u;
    did = true;
  }
  // launch when work is published and no kernel runs
  if (!R.running && R.n_flight > 0 && dev_ok && !R.failed) {
    *reinterpret_cast<volatile unsigned*>(&R.h_hdr->closed) = 0u;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    R.closing = false;
    const int smem = std::min(std::max(sv->max_slot_smem, 16), R.max_dyn);
    const bool all = sv->any_all;
    const auto kernel = all ? serve_kernel_all : serve_kernel;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kBatchThreads, smem) != cudaSuccess ||
        occ < 1) {
      cudaGetLastError();
      R.failed = true;
      snprintf(sv->err, sizeof(sv->err), "resident serving kernel does not fit (%d bytes)", smem);
      return true;
    }
    // one CTA slot stays free, so a joining robot's set-up kernel can run
    const int grid = std::max(1, num_sms() * occ - 1);
    ServeRing ring;
    ring.hdr = R.d_hdr;
    ring.items[0] = R.d_items[0];
    ring.items[1] = R.d_items[1];
    ring.reqs = R.d_reqs;
    ring.inputs = R.d_in;
    ring.out = R.d_out;
    ring.done = R.d_done;
    ring.next = R.d_next;
    ring.cap_items = R.cap_items;
    ring.in_stride = R.in_stride;
    ring.idle_polls = kServeIdlePolls;
    ring.idle_ns = kServeIdleNs;
    kernel<<<grid, kBatchThreads, smem, R.stream>>>(sv->b->d_descs, ring);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(R.ev, R.stream) != cudaSuccess) {
      R.failed = true;
      snprintf(sv->err, sizeof(sv->err), "resident serving kernel launch failed");
      cudaGetLastError();
      return true;
    }
    R.running = true;
    R.k_smem = smem;
    R.k_all = all;
    sv->batches++;
    did = true;
  }
  return did;
}

void server_loop(mppi_server* sv) {
  // a new host thread starts on device 0: take the server's device, where
  // its pool, streams and events were made, before any other CUDA call
  const bool dev_ok = cudaSetDevice(sv->device) == cudaSuccess;
  if (!dev_ok) cudaGetLastError();  // every request then completes with MPPI_ECUDA
  std::vector<int32_t> slots;
  std::vector<double> x0s;
  std::vector<const double*> xr;
  while (!sv->stop.load()) {
    if (sv->dq.load()) {
      if (!ring_step(sv, dev_ok)) std::this_thread::sleep_for(std::chrono::microseconds(10));
      continue;
    }
    bool did = false;
    for (size_t i = 0; i < sv->lanes.size(); ++i) {
      if (!sv->lane_busy[i]) continue;
      cudaError_t q = cudaEventQuery(sv->events[i]);
      if (q == cudaErrorNotReady) continue;
      const auto now = std::chrono::steady_clock::now();
      float dev_ms = 0.0f;
      if (q == cudaSuccess && cudaEventElapsedTime(&dev_ms, sv->ev_start[i], sv->events[i]) != cudaSuccess) {
        cudaGetLastError();
        dev_ms = 0.0f;
      }
      std::lock_guard<std::mutex> g(sv->mu);
      const double* out = sv->lanes[i].h_out;
      for (size_t j = 0; j < sv->inflight[i].size(); ++j) {
        const ServerReq& r = sv->inflight[i][j];
        ServerDone d;
        d.robot = r.robot;
        for (int k = 0; k < 8; ++k) d.out[k] = q == cudaSuccess ? out[8 * j + k] : NAN;
        d.latency = std::chrono::duration<double>(now - r.t0).count();
        d.queue = std::chrono::duration<double>(r.t_launch - r.t0).count();
        d.device = 1e-3 * dev_ms;
        d.cls = r.cls;
        d.status = q == cudaSuccess ? MPPI_OK : MPPI_ECUDA;
        sv->done.push_back(d);
        sv->busy[r.robot] = 0;
      }
      sv->n_inflight -= (int)sv->inflight[i].size();
      sv->requests += sv->inflight[i].size();
      sv->inflight[i].clear();
      sv->lane_busy[i] = 0;
      did = true;
    }
    for (size_t i = 0; i < sv->lanes.size(); ++i) {
      if (sv->lane_busy[i]) continue;
      std::vector<ServerReq>& batch = sv->inflight[i];  // only this thread touches it
      double share = 1.0;
      {
        std::lock_guard<std::mutex> g(sv->mu);
        const int c = sv->lane_cls[i];
        std::deque<ServerReq>& qu = sv->queue[c];
        if (qu.empty()) continue;
        // the oldest requests of the class, up to the class's work cap (a
        // request above the cap goes alone)
        const double cap = c == 0 ? sv->pol.batch_ops_small : sv->pol.batch_ops_large;
        batch.clear();
        double work = 0.0;
        const auto t_launch = std::chrono::steady_clock::now();
        if (sv->pol.shortest_first) {
          // requests queued past the age limit first (oldest first), then
          // the least work first; stable, so equal work keeps queue order
          std::stable_sort(qu.begin(), qu.end(), [&](const ServerReq& a, const ServerReq& b2) {
            const double lim = sv->pol.max_wait_s;
            const bool oa = lim > 0 && std::chrono::duration<double>(t_launch - a.t0).count() > lim;
            const bool ob = lim > 0 && std::chrono::duration<double>(t_launch - b2.t0).count() > lim;
            if (oa != ob) return oa;
            if (oa) return a.t0 < b2.t0;
            return a.ops < b2.ops;
          });
        }
        while (!qu.empty() && (batch.empty() || cap <= 0 || work + qu.front().ops <= cap)) {
          work += qu.front().ops;
          batch.push_back(std::move(qu.front()));
          batch.back().t_launch = t_launch;
          qu.pop_front();
        }
        // the large class's kernels leave the small class its share of the
        // SMs whenever the small class has lanes of its own
        bool shared = false;
        for (size_t k = 0; k < sv->lanes.size(); ++k) shared = shared || sv->lane_cls[k] != c;
        share = (c == 1 && shared) ? sv->pol.large_share : 1.0;
      }
      // pack and launch outside the lock: submissions and polls go on
      const int n = (int)batch.size();
      slots.resize(n);
      x0s.assign((size_t)n * 6, 0.0);
      xr.resize(n);
      for (int j = 0; j < n; ++j) {
        slots[j] = batch[j].robot;
        memcpy(&x0s[(size_t)j * 6], batch[j].x0, sizeof(double) * 6);
        xr[j] = batch[j].xref.empty() ? nullptr : batch[j].xref.data();
      }
      int rc = MPPI_OK;
      if (!dev_ok)
        rc = fail(MPPI_ECUDA, "cudaSetDevice(%d) failed in the scheduler thread", sv->device);
      if (rc == MPPI_OK && cudaEventRecord(sv->ev_start[i], sv->streams[i]) != cudaSuccess)
        rc = fail(MPPI_ECUDA, "event record failed");
      if (rc == MPPI_OK)
        rc = lane_step(sv->b, sv->lanes[i], slots.data(), n, x0s.data(), xr.data(), sv->streams[i],
                       false, share);
      if (rc == MPPI_OK && cudaEventRecord(sv->events[i], sv->streams[i]) != cudaSuccess)
        rc = fail(MPPI_ECUDA, "event record failed");
      if (rc != MPPI_OK) {
        std::lock_guard<std::mutex> g(sv->mu);
        snprintf(sv->err, sizeof(sv->err), "%s", g_err);
        const auto now = std::chrono::steady_clock::now();
        for (const ServerReq& r : batch) {
          ServerDone d;
          d.robot = r.robot;
          for (int k = 0; k < 8; ++k) d.out[k] = NAN;
          d.latency = std::chrono::duration<double>(now - r.t0).count();
          d.queue = d.latency;
          d.device = 0.0;
          d.cls = r.cls;
          d.status = rc;
          sv->done.push_back(d);
          sv->busy[r.robot] = 0;
        }
        sv->n_inflight -= n;
        batch.clear();
        continue;
      }
      sv->lane_busy[i] = 1;
      sv->batches++;
      did = true;
    }
    if (!did) std::this_thread::sleep_for(std::chrono::microseconds(10));
  }
}

}  // namespace

extern "C" {

int mppi_server_create(int32_t max_robots, size_t pool_bytes, int32_t lanes, mppi_server** out) {
  if (!out) return fail(MPPI_EINVAL, "out is NULL");
  *out = nullptr;
  if (lanes < 1 || lanes > 8) return fail(MPPI_EINVAL, "lanes must be in [1, 8]");
  mppi_server* sv = new (std::nothrow) mppi_server();
  if (!sv) return fail(MPPI_ENOMEM, "host allocation failed");
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return fail(MPPI_ECUDA, "cudaGetDevice failed");
  }
  int rc = mppi_batch_create(max_robots, pool_bytes, &sv->b);
  if (rc) {
    delete sv;
    return rc;
  }
  sv->max_robots = max_robots;
  sv->lanes.resize(lanes);
  sv->lane_cls.assign(lanes, 0);
  sv->streams.assign(lanes, nullptr);
  sv->ev_start.assign(lanes, nullptr);
  sv->events.assign(lanes, nullptr);
  sv->inflight.resize(lanes);
  sv->lane_busy.assign(lanes, 0);
  sv->joined.assign(max_robots, 0);
  sv->busy.assign(max_robots, 0);
  sv->pol = mppi_server_policy{0.0, 1, 0, 0.75, 0.0, 0.0, 0.0, 0, 0};  // one class, oldest first
  assign_lanes(sv);
  // staging for a step of every robot at once (step table, inputs, a
  // generous work list), made now so that the scheduler never has to grow it
  const size_t stage0 = std::min<size_t>((size_t)64 << 20, ((size_t)1 << 20) + (size_t)max_robots * (16u << 10));
  for (int i = 0; i < lanes; ++i) {
    if (lane_reserve(sv->lanes[i], stage0, max_robots) != MPPI_OK ||
        cudaStreamCreateWithFlags(&sv->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sv->ev_start[i]) != cudaSuccess ||
        cudaEventCreate(&sv->events[i]) != cudaSuccess) {
      cudaGetLastError();
      for (int k = 0; k <= i; ++k) {
        free_lane(sv->lanes[k]);
        if (sv->ev_start[k]) cudaEventDestroy(sv->ev_start[k]);
        if (sv->events[k]) cudaEventDestroy(sv->events[k]);
        if (sv->streams[k]) cudaStreamDestroy(sv->streams[k]);
      }
      mppi_batch_destroy(sv->b);
      delete sv;
      return fail(MPPI_ECUDA, "stream/event creation failed");
    }
  }
  sv->worker = std::thread(server_loop, sv);
  *out = sv;
  return MPPI_OK;
}

int mppi_server_set_policy(mppi_server* sv, const mppi_server_policy* pol) {
  if (!sv) return fail(MPPI_ESTATE, "server is NULL");
  if (!pol) return fail(MPPI_EINVAL, "policy is NULL");
  if (!std::isfinite(pol->small_ops_max) || pol->small_ops_max < 0 ||
      !std::isfinite(pol->batch_ops_small) || pol->batch_ops_small < 0 ||
      !std::isfinite(pol->batch_ops_large) || pol->batch_ops_large < 0)
    return fail(MPPI_EINVAL, "work thresholds must be finite and >= 0");
  if (!(pol->large_share > 0.0 && pol->large_share <= 1.0))
    return fail(MPPI_EINVAL, "large_share must be in (0, 1]");
  if (pol->small_lanes < 1) return fail(MPPI_EINVAL, "small_lanes must be >= 1");
  if (pol->shortest_first != 0 && pol->shortest_first != 1)
    return fail(MPPI_EINVAL, "shortest_first must be 0 or 1");
  if (!std::isfinite(pol->max_wait_s) || pol->max_wait_s < 0)
    return fail(MPPI_EINVAL, "max_wait_s must be finite and >= 0");
  if (pol->device_queue != 0 && pol->device_queue != 1)
    return fail(MPPI_EINVAL, "device_queue must be 0 or 1");
  std::lock_guard<std::mutex> g(sv->mu);
  if (sv->n_inflight.load() != 0)
    return fail(MPPI_ESTATE, "requests are queued or in flight: set the policy while idle");
  if (pol->device_queue) {
    if (int rc = ring_alloc(sv)) return rc;
  }
  sv->pol = *pol;
  assign_lanes(sv);
  sv->dq = pol->device_queue != 0;
  return MPPI_OK;
}

int mppi_server_get_policy(mppi_server* sv, mppi_server_policy* pol, int32_t* lane_classes) {
  if (!sv) return fail(MPPI_ESTATE, "server is NULL");
  std::lock_guard<std::mutex> g(sv->mu);
  if (pol) *pol = sv->pol;
  if (lane_classes)
    for (size_t i = 0; i < sv->lane_cls.size(); ++i) lane_classes[i] = sv->lane_cls[i];
  return MPPI_OK;
}

int mppi_server_join(mppi_server* sv, const mppi_params* p, const double* u_init,
                     const double* cxcyr, int32_t J, int32_t* robot) {
  if (!sv) return fail(MPPI_ESTATE, "server is NULL");
  if (!robot) return fail(MPPI_EINVAL, "robot is NULL");
  std::lock_guard<std::mutex> gs(sv->slot_mu);
  int32_t slot = -1;
  // a free slot is read by no launch, so the scheduler runs on meanwhile
  int rc = mppi_batch_add(sv->b, p, u_init, nullptr, cxcyr, J, &slot);
  if (rc) return rc;
  std::lock_guard<std::mutex> g(sv->mu);
  sv->joined[slot] = 1;
  sv->busy[slot] = 0;
  sv->max_slot_smem = std::max(sv->max_slot_smem, sv->b->slots[slot].smem);
  sv->any_all = sv->any_all || p->model >= 2;
  *robot = slot;
  return MPPI_OK;
}

int mppi_server_leave(mppi_server* sv, int32_t robot) {
  if (!sv) return fail(MPPI_ESTATE, "server is NULL");
  std::lock_guard<std::mutex> gs(sv->slot_mu);
  {
    std::lock_guard<std::mutex> g(sv->mu);
    if (robot < 0 || robot >= sv->max_robots || !sv->joined[robot])
      return fail(MPPI_EINVAL, "robot %d has not joined", robot);
    if (sv->busy[robot]) return fail(MPPI_ESTATE, "robot %d has a request in flight", robot);
    sv->joined[robot] = 0;  // no request can be queued for it from here on
  }
  return mppi_batch_remove(sv->b, robot);
}

int mppi_server_submit(mppi_server* sv, int32_t robot, const double* x0, const double* xref) {
  if (!sv) return fail(MPPI_ESTATE, "server is NULL");
  if (!x0) return fail(MPPI_EINVAL, "x0 is NULL");
  ServerReq r;
  r.robot = robot;
  r.t0 = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> g(sv->mu);
  if (robot < 0 || robot >= sv->max_robots || !sv->joined[robot])
    return fail(MPPI_EINVAL, "robot %d has not joined", robot);
  if (sv->busy[robot]) return fail(MPPI_ESTATE, "robot %d already has a request", robot);
  const BatchSlot& s = sv->b->slots[robot];
  for (int k = 0; k < 6; ++k) r.x0[k] = k < s.n ? x0[k] : 0.0;
  if (!finite_all(r.x0, s.n)) return fail(MPPI_EINVAL, "x0 is not finite");
  if (xref) {
    r.xref.assign(xref, xref + (size_t)(s.p.T + 1) * s.n);
    if (!finite_all(r.xref.data(), (int)r.xref.size())) return fail(MPPI_EINVAL, "xref is not finite");
  }
  r.ops = slot_ops(s);
  bool two = sv->pol.device_queue != 0 && sv->pol.small_ops_max > 0;
  for (int c : sv->lane_cls) two = two || c == 1;
  r.cls = (two && r.ops > sv->pol.small_ops_max) ? 1 : 0;
  sv->busy[robot] = 1;
  sv->n_inflight++;
  sv->queue[r.cls].push_back(std::move(r));
  return MPPI_OK;
}

int mppi_server_poll_timed(mppi_server* sv, int32_t max, int32_t* robots, double* u0s, double* x1s,
                           double* latency_s, double* queue_s, double* device_s,
                           int32_t* size_class, int32_t* status, int32_t* n_out) {
  if (!sv) return fail(MPPI_ESTATE, "server is NULL");
  if (!n_out) return fail(MPPI_EINVAL, "n_out is NULL");
  std::lock_guard<std::mutex> g(sv->mu);
  int n = 0;
  while (n < max && !sv->done.empty()) {
    const ServerDone& d = sv->done.front();
    if (robots) robots[n] = d.robot;
    if (u0s) {
      u0s[2 * n] = d.out[0];
      u0s[2 * n + 1] = d.out[1];
    }
    if (x1s)
      for (int k = 0; k < 6; ++k) x1s[6 * n + k] = d.out[2 + k];
    if (latency_s) latency_s[n] = d.latency;
    if (queue_s) queue_s[n] = d.queue;
    if (device_s) device_s[n] = d.device;
    if (size_class) size_class[n] = d.cls;
    if (status) status[n] = d.status;
    sv->done.pop_front();
    ++n;
  }
  *n_out = n;
  return MPPI_OK;
}

int mppi_server_poll(mppi_server* sv, int32_t max, int32_t* robots, double* u0s, double* x1s,
                     double* latency_s, int32_t* status, int32_t* n_out) {
  return mppi_server_poll_timed(sv, max, robots, u0s, x1s, latency_s, nullptr, nullptr, nullptr,
                                status, n_out);
}

int mppi_server_stats(mppi_server* sv, uint64_t* batches, uint64_t* requests, int32_t* pending,
                      uint64_t* pool_free_bytes) {
  if (!sv) return fail(MPPI_ESTATE, "server is NULL");
  if (batches) *batches = sv->batches.load();
  if (requests) *requests = sv->requests.load();
  if (pending) *pending = sv->n_inflight.load();
  if (pool_free_bytes) {
    std::lock_guard<std::mutex> g(sv->slot_mu);
    size_t f = 0;
    for (auto& e : sv->b->free_list) f += e.second;
    *pool_free_bytes = f;
  }
  return MPPI_OK;
}

int mppi_server_destroy(mppi_server* sv) {
  if (!sv) return MPPI_OK;
  sv->stop = true;
  if (sv->worker.joinable()) sv->worker.join();
  ring_free(sv->ring);
  for (size_t i = 0; i < sv->lanes.size(); ++i) {
    free_lane(sv->lanes[i]);
    cudaEventDestroy(sv->ev_start[i]);
    cudaEventDestroy(sv->events[i]);
    cudaStreamDestroy(sv->streams[i]);
  }
  mppi_batch_destroy(sv->b);
  delete sv;
  return MPPI_OK;
}

}  // extern "C"
