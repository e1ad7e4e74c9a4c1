// Kernel instantiations for the D2Q9 fluid lattice (with D2Q9 scalars),
// BGK and MRT collision, FP32 state storage.
#include "albm_kernels.cuh"

namespace albm {

bool kernels_d2q9_f32(bool mrt, int nscalars, KernelSet* out) {
  return mrt ? pick_scalars<D2Q9, true, float, 1>(nscalars, out)
             : pick_scalars<D2Q9, false, float, 1>(nscalars, out);
}

}  // namespace albm
