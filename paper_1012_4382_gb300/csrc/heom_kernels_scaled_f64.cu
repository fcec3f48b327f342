// Instantiations of the N <= 8 engine kernel for scaled hierarchies (HEOM_FLAG_SCALED):
// FP64, load views only (node_threads >= 3), real and complex Hamiltonians.
#include "heom_engine.cuh"
#include "heom_internal.h"

namespace heom {

const void* engine_kernel_scaled_f64(int N, bool cplx) {
  switch (N) {
    case 1: return cplx ? (const void*)heom_engine_kernel<1, double, false, true, false, true>
                     : (const void*)heom_engine_kernel<1, double, false, false, false, true>;
    case 2: return cplx ? (const void*)heom_engine_kernel<2, double, false, true, false, true>
                     : (const void*)heom_engine_kernel<2, double, false, false, false, true>;
    case 3: return cplx ? (const void*)heom_engine_kernel<3, double, false, true, false, true>
                     : (const void*)heom_engine_kernel<3, double, false, false, false, true>;
    case 4: return cplx ? (const void*)heom_engine_kernel<4, double, false, true, false, true>
                     : (const void*)heom_engine_kernel<4, double, false, false, false, true>;
    case 5: return cplx ? (const void*)heom_engine_kernel<5, double, false, true, false, true>
                     : (const void*)heom_engine_kernel<5, double, false, false, false, true>;
    case 6: return cplx ? (const void*)heom_engine_kernel<6, double, false, true, false, true>
                     : (const void*)heom_engine_kernel<6, double, false, false, false, true>;
    case 7: return cplx ? (const void*)heom_engine_kernel<7, double, false, true, false, true>
                     : (const void*)heom_engine_kernel<7, double, false, false, false, true>;
    case 8: return cplx ? (const void*)heom_engine_kernel<8, double, false, true, false, true>
                     : (const void*)heom_engine_kernel<8, double, false, false, false, true>;
    default: return nullptr;
  }
}

}  // namespace heom
