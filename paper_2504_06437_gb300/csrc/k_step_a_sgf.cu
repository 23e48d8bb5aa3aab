// One-controller step kernels of the Ackermann vehicle (Eq. 14) with
// Savitzky-Golay smoothing of the update (Algorithm 1's SGF).
#include "kernels.cuh"

namespace dbm {

__global__ void __maxnreg__(DBM_STEP_MAXNREG) step_a8_sgf(const __grid_constant__ CtrlDesc D,
                                                       const double* __restrict__ x0,
                                                       const double* __restrict__ xref) {
  step_body<2, 8, true>(D, x0, xref);
}

__global__ void __maxnreg__(DBM_STEP_MAXNREG) step_a14_sgf(const __grid_constant__ CtrlDesc D,
                                                        const double* __restrict__ x0,
                                                        const double* __restrict__ xref) {
  step_body<2, 14, true>(D, x0, xref);
}

}  // namespace dbm
