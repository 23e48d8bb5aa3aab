// One-controller step kernels of the paper's 5-state planar quadrotor (Eq. 12), 80-register form
// (see DBM_STEP_MAXNREG_R80).
#include "kernels.cuh"

namespace dbm {

__global__ void __maxnreg__(DBM_STEP_MAXNREG_R80) step_p8_r80(const __grid_constant__ CtrlDesc D,
                                                     const double* __restrict__ x0,
                                                     const double* __restrict__ xref) {
  step_body<3, 8>(D, x0, xref);
}

__global__ void __maxnreg__(DBM_STEP_MAXNREG_R80) step_p14_r80(const __grid_constant__ CtrlDesc D,
                                                      const double* __restrict__ x0,
                                                      const double* __restrict__ xref) {
  step_body<3, 14>(D, x0, xref);
}

}  // namespace dbm
