// Kernel instantiations for the D3Q19 fluid lattice (with D3Q7 scalars), BGK.
#include "albm_kernels.cuh"

namespace albm {

template <int NS>
static bool pick_bgk(int precision, KernelSet* out) {
  switch (precision) {
    case 0: *out = Launch<D3Q19, NS, false, float>::set(); return true;
    case 1: *out = Launch<D3Q19, NS, false, __nv_bfloat16>::set(); return true;
    case 2: *out = Launch<D3Q19, NS, false, __half>::set(); return true;
    default: return false;
  }
}

bool kernels_d3q19_bgk(int nscalars, int precision, KernelSet* out) {
  switch (nscalars) {
    case 0: return pick_bgk<0>(precision, out);
    case 1: return pick_bgk<1>(precision, out);
    case 2: return pick_bgk<2>(precision, out);
    default: return false;
  }
}

}  // namespace albm
