// Kernel instantiations for the D3Q19 fluid lattice (with D3Q7 scalars), MRT.
#include "albm_kernels.cuh"

namespace albm {

template <int NS>
static bool pick_mrt(int precision, KernelSet* out) {
  switch (precision) {
    case 0: *out = Launch<D3Q19, NS, true, float>::set(); return true;
    case 1: *out = Launch<D3Q19, NS, true, __nv_bfloat16>::set(); return true;
    case 2: *out = Launch<D3Q19, NS, true, __half>::set(); return true;
    default: return false;
  }
}

bool kernels_d3q19_mrt(int nscalars, int precision, KernelSet* out) {
  switch (nscalars) {
    case 0: return pick_mrt<0>(precision, out);
    case 1: return pick_mrt<1>(precision, out);
    case 2: return pick_mrt<2>(precision, out);
    default: return false;
  }
}

}  // namespace albm
