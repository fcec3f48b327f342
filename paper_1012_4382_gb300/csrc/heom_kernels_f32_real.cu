// Instantiations of the N <= 8 engine kernel: FP32 auxiliaries with FP64 root, real Hamiltonian.
// (One translation unit per precision and Hamiltonian kind so they compile in parallel.)
#include "heom_engine.cuh"
#include "heom_internal.h"

namespace heom {

const void* engine_kernel_f32_real(int N, bool reg) {
  switch (N) {
    case 1: return reg ? (const void*)heom_engine_kernel<1, float, true, false, true>
                    : (const void*)heom_engine_kernel<1, float, true, false, false>;
    case 2: return reg ? (const void*)heom_engine_kernel<2, float, true, false, true>
                    : (const void*)heom_engine_kernel<2, float, true, false, false>;
    case 3: return reg ? (const void*)heom_engine_kernel<3, float, true, false, true>
                    : (const void*)heom_engine_kernel<3, float, true, false, false>;
    case 4: return reg ? (const void*)heom_engine_kernel<4, float, true, false, true>
                    : (const void*)heom_engine_kernel<4, float, true, false, false>;
    case 5: return reg ? (const void*)heom_engine_kernel<5, float, true, false, true>
                    : (const void*)heom_engine_kernel<5, float, true, false, false>;
    case 6: return reg ? (const void*)heom_engine_kernel<6, float, true, false, true>
                    : (const void*)heom_engine_kernel<6, float, true, false, false>;
    case 7: return reg ? (const void*)heom_engine_kernel<7, float, true, false, true>
                    : (const void*)heom_engine_kernel<7, float, true, false, false>;
    case 8: return reg ? (const void*)heom_engine_kernel<8, float, true, false, true>
                    : (const void*)heom_engine_kernel<8, float, true, false, false>;
    default: return nullptr;
  }
}


}  // namespace heom
