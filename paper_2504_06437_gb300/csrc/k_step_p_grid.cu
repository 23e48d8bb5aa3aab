// One-controller step kernels of the 5-state planar quadrotor (Eq. 12) with
// the grid map's barrier terms (and Savitzky-Golay smoothing) compiled in.
#include "kernels.cuh"

namespace dbm {

__global__ void __maxnreg__(DBM_STEP_MAXNREG) step_p8_grid(const __grid_constant__ CtrlDesc D,
                                                        const double* __restrict__ x0,
                                                        const double* __restrict__ xref) {
  step_body<3, 8, true, true>(D, x0, xref);
}

__global__ void __maxnreg__(DBM_STEP_MAXNREG) step_p14_grid(const __grid_constant__ CtrlDesc D,
                                                         const double* __restrict__ x0,
                                                         const double* __restrict__ xref) {
  step_body<3, 14, true, true>(D, x0, xref);
}

}  // namespace dbm
