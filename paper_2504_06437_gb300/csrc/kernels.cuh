// Kernels of the DBaS-Log-MPPI library, defined in separate translation
// units (compiled in parallel) and launched from the host code in
// dbasmppi.cu.
#pragma once

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
