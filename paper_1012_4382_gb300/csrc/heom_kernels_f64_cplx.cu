// Instantiations of the N <= 8 engine kernel: FP64, complex Hamiltonian.
// (One translation unit per precision and Hamiltonian kind so they compile in parallel.)
#include "heom_engine.cuh"
#include "heom_internal.h"

namespace heom {

const void* engine_kernel_f64_cplx(int N, bool reg) {
  switch (N) {
    case 1: return reg ? (const void*)heom_engine_kernel<1, double, false, true, true>
                    : (const void*)heom_engine_kernel<1, double, false, true, false>;
    case 2: return reg ? (const void*)heom_engine_kernel<2, double, false, true, true>
                    : (const void*)heom_engine_kernel<2, double, false, true, false>;
    case 3: return reg ? (const void*)heom_engine_kernel<3, double, false, true, true>
                    : (const void*)heom_engine_kernel<3, double, false, true, false>;
    case 4: return reg ? (const void*)heom_engine_kernel<4, double, false, true, true>
                    : (const void*)heom_engine_kernel<4, double, false, true, false>;
    case 5: return reg ? (const void*)heom_engine_kernel<5, double, false, true, true>
                    : (const void*)heom_engine_kernel<5, double, false, true, false>;
    case 6: return reg ? (const void*)heom_engine_kernel<6, double, false, true, true>
                    : (const void*)heom_engine_kernel<6, double, false, true, false>;
    case 7: return reg ? (const void*)heom_engine_kernel<7, double, false, true, true>
                    : (const void*)heom_engine_kernel<7, double, false, true, false>;
    case 8: return reg ? (const void*)heom_engine_kernel<8, double, false, true, true>
                    : (const void*)heom_engine_kernel<8, double, false, true, false>;
    default: return nullptr;
  }
}

}  // namespace heom
