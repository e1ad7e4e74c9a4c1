// Kernel instantiations for the D3Q19 fluid lattice (with D3Q7 scalars),
// BGK collision, FP32 state storage.
#include "albm_kernels.cuh"

namespace albm {

bool kernels_d3q19_bgk_f32(int nscalars, KernelSet* out) {
  return pick_scalars<D3Q19, false, float, 2>(nscalars, out);
}

}  // namespace albm
