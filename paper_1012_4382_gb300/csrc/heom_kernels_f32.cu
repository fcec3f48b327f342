// FP32 (auxiliaries) / FP64 (root node, eta) instantiations of the N <= 8
// engine kernel.
#include "heom_engine.cuh"
#include "heom_internal.h"

namespace heom {

const void* engine_kernel_f32(int N) {
  switch (N) {
    case 1: return (const void*)heom_engine_kernel<1, float, true>;
    case 2: return (const void*)heom_engine_kernel<2, float, true>;
    case 3: return (const void*)heom_engine_kernel<3, float, true>;
    case 4: return (const void*)heom_engine_kernel<4, float, true>;
    case 5: return (const void*)heom_engine_kernel<5, float, true>;
    case 6: return (const void*)heom_engine_kernel<6, float, true>;
    case 7: return (const void*)heom_engine_kernel<7, float, true>;
    case 8: return (const void*)heom_engine_kernel<8, float, true>;
    default: return nullptr;
  }
}

}  // namespace heom
