// One-controller step kernels of the paper's 5-state planar quadrotor (Eq. 12).
#include "kernels.cuh"

namespace dbm {

__global__ void __maxnreg__(DBM_STEP_MAXNREG) step_p8(const __grid_constant__ CtrlDesc D,
                                                     const double* __restrict__ x0,
                                                     const double* __restrict__ xref) {
  step_body<3, 8>(D, x0, xref);
}

__global__ void __maxnreg__(DBM_STEP_MAXNREG) step_p14(const __grid_constant__ CtrlDesc D,
                                                      const double* __restrict__ x0,
                                                      const double* __restrict__ xref) {
  step_body<3, 14>(D, x0, xref);
}

}  // namespace dbm
