// One-controller step kernels of the planar quadrotor model.
#include "kernels.cuh"

namespace dbm {

__global__ void __maxnreg__(DBM_STEP_MAXNREG) step_q8(const __grid_constant__ CtrlDesc D,
                                                const double* __restrict__ x0,
                                                const double* __restrict__ xref) {
  step_body<1, 8>(D, x0, xref);
}

__global__ void __maxnreg__(DBM_STEP_MAXNREG) step_q14(const __grid_constant__ CtrlDesc D,
                                                 const double* __restrict__ x0,
                                                 const double* __restrict__ xref) {
  step_body<1, 14>(D, x0, xref);
}

}  // namespace dbm
