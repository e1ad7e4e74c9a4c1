// Kernel instantiations for the D2Q9 fluid lattice (with D2Q9 scalars).
#include "albm_kernels.cuh"

namespace albm {

template <int NS, bool MRT>
static bool pick(int precision, KernelSet* out) {
  switch (precision) {
    case 0: *out = Launch<D2Q9, NS, MRT, float>::set(); return true;
    case 1: *out = Launch<D2Q9, NS, MRT, __nv_bfloat16>::set(); return true;
    case 2: *out = Launch<D2Q9, NS, MRT, __half>::set(); return true;
    default: return false;
  }
}

bool kernels_d2q9(int collision, int nscalars, int precision, KernelSet* out) {
  const bool mrt = collision == 1;
  switch (nscalars) {
    case 0: return mrt ? pick<0, true>(precision, out) : pick<0, false>(precision, out);
    case 1: return mrt ? pick<1, true>(precision, out) : pick<1, false>(precision, out);
    default: return false;
  }
}

}  // namespace albm
