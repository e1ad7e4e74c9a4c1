// Kernel instantiations for the D2Q9 fluid lattice (with D2Q9 scalars),
// BGK and MRT collision, FP16 state storage.
#include "albm_kernels.cuh"

namespace albm {

bool kernels_d2q9_f16(bool mrt, int nscalars, KernelSet* out) {
  return mrt ? pick_scalars<D2Q9, true, __half, 1>(nscalars, out)
             : pick_scalars<D2Q9, false, __half, 1>(nscalars, out);
}

}  // namespace albm
