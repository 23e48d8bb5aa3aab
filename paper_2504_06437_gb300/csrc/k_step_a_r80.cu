// One-controller step kernels of the Ackermann vehicle (Eq. 14), 80-register form
// (see DBM_STEP_MAXNREG_R80).
#include "kernels.cuh"

namespace dbm {

__global__ void __maxnreg__(DBM_STEP_MAXNREG_R80) step_a8_r80(const __grid_constant__ CtrlDesc D,
                                                     const double* __restrict__ x0,
                                                     const double* __restrict__ xref) {
  step_body<2, 8>(D, x0, xref);
}

__global__ void __maxnreg__(DBM_STEP_MAXNREG_R80) step_a14_r80(const __grid_constant__ CtrlDesc D,
                                                      const double* __restrict__ x0,
                                                      const double* __restrict__ xref) {
  step_body<2, 14>(D, x0, xref);
}

}  // namespace dbm
