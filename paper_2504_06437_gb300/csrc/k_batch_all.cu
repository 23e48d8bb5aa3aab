// Batched step kernel for batches that hold the Ackermann vehicle or the
// 5-state quadrotor: the loop of batch_kernel (k_batch.cu) over all four
// models.  It is a translation unit of its own so that its tile
// instantiations, compiled under its register bound, are not the ones
// batch_kernel calls: the host launches batch_kernel, unchanged, whenever a
// step holds only unicycles and 6-state quadrotors.
#include "kernels.cuh"

namespace dbm {

// At least two resident CTAs per SM: without the bound the allocation would
// follow the largest of its eight tile instantiations (249 registers, one
// CTA per SM).
__global__ void __launch_bounds__(kBatchThreads, 2) batch_kernel_all(
    const CtrlDesc* __restrict__ descs, unsigned char* stage, double* __restrict__ u0_out) {
  extern __shared__ __align__(16) char smem[];
  __shared__ TileScratch ts;
  __shared__ CtrlDesc Ds;
  __shared__ int s_item;
  BatchHdr* hdr = reinterpret_cast<BatchHdr*>(stage);
  const StepEntry* steps = reinterpret_cast<const StepEntry*>(stage + sizeof(BatchHdr));
  const WorkItem* items = reinterpret_cast<const WorkItem*>(steps + hdr->n_steps);
  const double* inputs = reinterpret_cast<const double*>(stage + hdr->inputs_off);
  const int tid = threadIdx.x;
  if (tid == 0) mbar_init(&ts.mbar);
  __syncthreads();
  uint32_t phase = 0u;
  const int n_items = hdr->n_items;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(&hdr->next, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const WorkItem w = items[it];
    const StepEntry e = steps[w.ctrl];
    const int* src = reinterpret_cast<const int*>(descs + e.slot);
    int* dst = reinterpret_cast<int*>(&Ds);
    for (int i = tid; i < (int)(sizeof(CtrlDesc) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    const double* x0 = inputs + e.x0_off;
    const double* xref = inputs + e.xref_off;
    double* uo = u0_out + 8 * w.ctrl;  // u0 and the predicted next state
    // the batched form of the tile: see run_tile
    switch (Ds.model * 2 + npos_code(Ds.NPOS)) {
      case 0: run_tile<0, 8, true>(Ds, w.tile, x0, xref, smem, ts, phase, uo); break;
      case 1: run_tile<0, 14, true>(Ds, w.tile, x0, xref, smem, ts, phase, uo); break;
      case 2: run_tile<1, 8, true>(Ds, w.tile, x0, xref, smem, ts, phase, uo); break;
      case 3: run_tile<1, 14, true>(Ds, w.tile, x0, xref, smem, ts, phase, uo); break;
      case 4: run_tile<2, 8, true>(Ds, w.tile, x0, xref, smem, ts, phase, uo); break;
      case 5: run_tile<2, 14, true>(Ds, w.tile, x0, xref, smem, ts, phase, uo); break;
      case 6: run_tile<3, 8, true>(Ds, w.tile, x0, xref, smem, ts, phase, uo); break;
      default: run_tile<3, 14, true>(Ds, w.tile, x0, xref, smem, ts, phase, uo); break;
    }
    __syncthreads();  // Ds and s_item are reused by the next item
  }
}

// Resident serving kernel over the same tile instantiations (see
// serve_body in kernels.cuh).
__global__ void __launch_bounds__(kBatchThreads, 2) serve_kernel_all(const CtrlDesc* __restrict__ descs,
                                                              ServeRing R) {
  serve_body<true>(descs, R);
}

}  // namespace dbm
