// Instantiations of the large-N (9..24 sites) engine kernel, plain and scaled hierarchies.
#include "heom_large.cuh"
#include "heom_internal.h"

namespace heom {

const void* large_kernel(bool fp64, bool cplx, bool scaled) {
  if (scaled) {
    if (fp64) return cplx ? (const void*)heom_large_kernel<double, false, true, true>
                          : (const void*)heom_large_kernel<double, false, false, true>;
    return cplx ? (const void*)heom_large_kernel<float, true, true, true>
                : (const void*)heom_large_kernel<float, true, false, true>;
  }
  if (fp64) return cplx ? (const void*)heom_large_kernel<double, false, true>
                        : (const void*)heom_large_kernel<double, false, false>;
  return cplx ? (const void*)heom_large_kernel<float, true, true> : (const void*)heom_large_kernel<float, true, false>;
}

}  // namespace heom
