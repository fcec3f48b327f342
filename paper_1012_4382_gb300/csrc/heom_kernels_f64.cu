// FP64 instantiations of the N <= 8 engine kernel (one translation unit per
// precision so the two compile in parallel).
#include "heom_engine.cuh"
#include "heom_internal.h"

namespace heom {

const void* engine_kernel_f64(int N) {
  switch (N) {
    case 1: return (const void*)heom_engine_kernel<1, double, false>;
    case 2: return (const void*)heom_engine_kernel<2, double, false>;
    case 3: return (const void*)heom_engine_kernel<3, double, false>;
    case 4: return (const void*)heom_engine_kernel<4, double, false>;
    case 5: return (const void*)heom_engine_kernel<5, double, false>;
    case 6: return (const void*)heom_engine_kernel<6, double, false>;
    case 7: return (const void*)heom_engine_kernel<7, double, false>;
    case 8: return (const void*)heom_engine_kernel<8, double, false>;
    default: return nullptr;
  }
}

}  // namespace heom
