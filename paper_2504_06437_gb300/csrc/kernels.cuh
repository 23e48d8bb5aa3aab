// Kernels of the DBaS-Log-MPPI library, defined in separate translation
// units (compiled in parallel) and launched from the host code in
// dbasmppi.cu.
#pragma once

#include "../../include/dbasmppi.h"
#include "mppi_tile.cuh"

namespace dbm {

// Register cap of the one-controller step kernels: 96 lets five 128-thread
// CTAs (20 warps) share an SM where the uncapped allocation fits four.  The
// merge and the final stage, which run once per launch, are what would
// otherwise raise the kernel's allocation.
#ifndef DBM_STEP_MAXNREG
#define DBM_STEP_MAXNREG 96
#endif

// Register cap of the second form of the step kernels (suffix _r80), taken
// for grids of several waves when it raises the CTAs resident per SM: 80
// lets six 128-thread CTAs share an SM (24 warps instead of 20), which hides
// more of the barrier loop's pipe latency.  It spills a little, so the
// 96-register form stays the choice for single-wave grids.
#ifndef DBM_STEP_MAXNREG_R80
#define DBM_STEP_MAXNREG_R80 80
#endif

// One step of one controller: one CTA per tile (MODEL: 0 unicycle (u),
// 1 planar quadrotor with two thrusts (q), 2 Ackermann vehicle (a), 3 the
// paper's 5-state planar quadrotor (p); 8 or 14 world points per barrier
// thread).
__global__ void step_u8(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                        const double* __restrict__ xref);
__global__ void step_u14(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                         const double* __restrict__ xref);
__global__ void step_q8(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                        const double* __restrict__ xref);
__global__ void step_q14(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                         const double* __restrict__ xref);
__global__ void step_a8(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                        const double* __restrict__ xref);
__global__ void step_a14(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                         const double* __restrict__ xref);
__global__ void step_p8(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                        const double* __restrict__ xref);
__global__ void step_p14(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                         const double* __restrict__ xref);
__global__ void step_u8_r80(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                            const double* __restrict__ xref);
__global__ void step_u14_r80(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);
__global__ void step_q8_r80(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                            const double* __restrict__ xref);
__global__ void step_q14_r80(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);
__global__ void step_a8_r80(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                            const double* __restrict__ xref);
__global__ void step_a14_r80(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);
__global__ void step_p8_r80(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                            const double* __restrict__ xref);
__global__ void step_p14_r80(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);

// The same with Savitzky-Golay smoothing of the update compiled in (suffix
// _sgf, 96-register form), launched only for controllers that smooth.
__global__ void step_u8_sgf(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                            const double* __restrict__ xref);
__global__ void step_u14_sgf(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);
__global__ void step_q8_sgf(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                            const double* __restrict__ xref);
__global__ void step_q14_sgf(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);
__global__ void step_a8_sgf(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                            const double* __restrict__ xref);
__global__ void step_a14_sgf(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);
__global__ void step_p8_sgf(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                            const double* __restrict__ xref);
__global__ void step_p14_sgf(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);

// The same with the grid map's terms compiled in (suffix _grid; smoothing
// too), launched only for controllers that have a grid map.
__global__ void step_u8_grid(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);
__global__ void step_u14_grid(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                              const double* __restrict__ xref);
__global__ void step_q8_grid(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);
__global__ void step_q14_grid(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                              const double* __restrict__ xref);
__global__ void step_a8_grid(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);
__global__ void step_a14_grid(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                              const double* __restrict__ xref);
__global__ void step_p8_grid(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                             const double* __restrict__ xref);
__global__ void step_p14_grid(const __grid_constant__ CtrlDesc D, const double* __restrict__ x0,
                              const double* __restrict__ xref);

// Batched step: persistent CTAs pull (controller, tile) work items.
struct WorkItem {
  int ctrl;  // index into the step table
  int tile;
};
struct StepEntry {
  int slot;
  int x0_off;  // offsets, in doubles, into the packed inputs
  int xref_off;
  int pad;
};
struct BatchHdr {
  int n_steps, n_items;
  unsigned next;
  int inputs_off;  // byte offset of the packed inputs
};
constexpr int kBatchThreads = 256;
__global__ void batch_kernel(const CtrlDesc* __restrict__ descs, unsigned char* stage,
                             double* __restrict__ u0_out);
// The same over all four models (launched when a step holds model 2 or 3).
__global__ void batch_kernel_all(const CtrlDesc* __restrict__ descs, unsigned char* stage,
                                 double* __restrict__ u0_out);

// Resident serving kernel (serve_kernel, serve_kernel_all): persistent CTAs
// pull (request, tile) items that the host publishes while the kernel runs.
// The rings live in mapped pinned host memory: the host writes a request's
// entry, inputs and items, then (release) raises its class's published
// count; a CTA reads the count with a system-scope acquire, claims the next
// item of the small class if any, else of the large class, with a CAS on a
// device counter, and runs the tile.  The CTA whose tile completes a request
// writes u0 and the predicted state to the request's output slot, fences at
// system scope, then stores the request's number + 1 in its done word.  With
// nothing to claim a CTA polls until the host sets `closed`, at most
// idle_polls times idle_ns apart (a bound that ends the wait should the host
// never close the kernel).
struct __align__(8) ServeHdr {
  unsigned published[2];  // items published per class (0 small, 1 large); monotonic
  unsigned closed;        // nonzero: stop claiming and exit
  unsigned pad;
};
// One published request: the robot's pool slot, where its reference starts
// in its inputs, how many input doubles there are, and its sequence number.
struct ServeReq {
  int slot;
  int xref_off;
  int n_in;
  unsigned seq;
};
struct ServeRing {
  const ServeHdr* hdr;          // mapped host memory (device alias)
  const WorkItem* items[2];     // per class, cap_items entries (a power of two);
                                // WorkItem.ctrl = request slot
  const ServeReq* reqs;         // per request slot
  const double* inputs;         // request slot * in_stride: x0 (n) then xref ((T+1) n)
  double* out;                  // request slot * 8: u0 then the predicted state
  unsigned* done;               // request slot: sequence number + 1 once complete
  unsigned* next;               // device memory: items claimed per class
  unsigned cap_items;
  int in_stride;                // doubles per request slot of `inputs`
  int idle_polls, idle_ns;
};
constexpr int kServeInputMax = (MPPI_MAX_T + 2) * kMaxN;  // doubles staged per item

// Both classes' published counts in one system-scope acquire load (the two
// words are adjacent and 8-byte aligned; each is monotonic, so a read that
// catches one updated and not the other is still a valid view).
__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0: claim the next item, small class first; the class, or -1 when
// the bounded idle wait ran out or the host closed the kernel.
__device__ __forceinline__ int serve_claim(const ServeRing& R, unsigned* idx) {
  for (int poll = 0; poll <= R.idle_polls; ++poll) {
    const unsigned long long both = ld_acquire_sys_u64(R.hdr->published);
    for (int c = 0; c < 2; ++c) {
      const unsigned pub = (unsigned)(c == 0 ? both : both >> 32);
      unsigned cur = *reinterpret_cast<volatile unsigned*>(&R.next[c]);
      while ((int)(pub - cur) > 0) {  // an item is published and unclaimed
        const unsigned prev = atomicCAS(&R.next[c], cur, cur + 1u);
        if (prev == cur) {
          *idx = cur;
          return c;
        }
        cur = prev;  // another CTA took it: the next one, if any
      }
    }
    if (*reinterpret_cast<const volatile unsigned*>(&R.hdr->closed)) return -1;
    if (poll < R.idle_polls) __nanosleep(R.idle_ns);
  }
  return -1;
}

__global__ void serve_kernel(const CtrlDesc* __restrict__ descs, ServeRing R);
__global__ void serve_kernel_all(const CtrlDesc* __restrict__ descs, ServeRing R);

__device__ __forceinline__ int npos_code(int npos) { return npos == 14 ? 1 : 0; }

// The loop of the resident serving kernels; ALL: the four models (else the
// unicycle and the 6-state quadrotor).  Everything the host may rewrite
// while the kernel runs is read past the L1 (volatile or .cg loads): the
// ring entries, the inputs (staged into shared memory, which run_tile then
// reads), and the descriptor of a slot that a robot joining later reuses.
// Controller state that an earlier request's final stage wrote is read after
// the claim's system-scope acquire and a fence, so it is the latest.
template <bool ALL>
__device__ __forceinline__ void serve_body(const CtrlDesc* __restrict__ descs, const ServeRing& R) {
  extern __shared__ __align__(16) char smem[];
  __shared__ TileScratch ts;
  __shared__ CtrlDesc Ds;
  __shared__ int s_cls;
  __shared__ unsigned s_idx;
  __shared__ __align__(16) double s_in[kServeInputMax];
  const int tid = threadIdx.x;
  if (tid == 0) mbar_init(&ts.mbar);
  __syncthreads();
  uint32_t phase = 0u;
  for (;;) {
    if (tid == 0) s_cls = serve_claim(R, &s_idx);
    __syncthreads();
    const int cls = s_cls;
    if (cls < 0) break;
    __threadfence();
    const WorkItem* wp = R.items[cls] + (s_idx & (R.cap_items - 1u));
    const int rq = *reinterpret_cast<const volatile int*>(&wp->ctrl);
    const int tile = *reinterpret_cast<const volatile int*>(&wp->tile);
    const ServeReq* ep = R.reqs + rq;
    const int slot = *reinterpret_cast<const volatile int*>(&ep->slot);
    const int xref_off = *reinterpret_cast<const volatile int*>(&ep->xref_off);
    const int n_in = *reinterpret_cast<const volatile int*>(&ep->n_in);
    const unsigned seq = *reinterpret_cast<const volatile unsigned*>(&ep->seq);
    const int* src = reinterpret_cast<const int*>(descs + slot);
    int* dst = reinterpret_cast<int*>(&Ds);
    for (int i = tid; i < (int)(sizeof(CtrlDesc) / 4); i += blockDim.x) dst[i] = __ldcg(src + i);
    const volatile double* in = R.inputs + (size_t)rq * R.in_stride;
    for (int i = tid; i < n_in; i += blockDim.x) s_in[i] = in[i];
    __syncthreads();
    double* uo = R.out + 8 * (size_t)rq;
    const double* x0 = s_in;
    const double* xref = s_in + xref_off;
    switch (Ds.model * 2 + npos_code(Ds.NPOS)) {
      case 0: run_tile<0, 8, true>(Ds, tile, x0, xref, smem, ts, phase, uo); break;
      case 1: run_tile<0, 14, true>(Ds, tile, x0, xref, smem, ts, phase, uo); break;
      case 2: run_tile<1, 8, true>(Ds, tile, x0, xref, smem, ts, phase, uo); break;
      case 3: run_tile<1, 14, true>(Ds, tile, x0, xref, smem, ts, phase, uo); break;
      default:
        if constexpr (ALL) {
          switch (Ds.model * 2 + npos_code(Ds.NPOS)) {
            case 4: run_tile<2, 8, true>(Ds, tile, x0, xref, smem, ts, phase, uo); break;
            case 5: run_tile<2, 14, true>(Ds, tile, x0, xref, smem, ts, phase, uo); break;
            case 6: run_tile<3, 8, true>(Ds, tile, x0, xref, smem, ts, phase, uo); break;
            default: run_tile<3, 14, true>(Ds, tile, x0, xref, smem, ts, phase, uo); break;
          }
        }
        break;
    }
    // the CTA that ran the final stage publishes the request's completion
    // after its outputs (written by thread 0 in the final stage)
    if (tid == 0 && ts.flag) {
      __threadfence_system();
      *reinterpret_cast<volatile unsigned*>(R.done + rq) = seq + 1u;
    }
    __syncthreads();  // Ds, s_in, s_cls and s_idx are reused by the next item
  }
}

// Body of the one-controller step kernels.
template <int MODEL, int NPOS, bool SGF = false, bool GRID = false>
__device__ __forceinline__ void step_body(const CtrlDesc& D, const double* __restrict__ x0,
                                          const double* __restrict__ xref) {
  extern __shared__ __align__(16) char smem[];
  __shared__ TileScratch ts;
  if (threadIdx.x == 0) mbar_init(&ts.mbar);
  __syncthreads();
  uint32_t phase = 0u;
  run_tile_inl<MODEL, NPOS, false, SGF, GRID>(D, blockIdx.x, x0, xref, smem, ts, phase);
}

}  // namespace dbm
