// Instantiations of the distributed-shared-memory engine kernel (mixed precision,
// real Hamiltonian); a translation unit of its own so it compiles in parallel.
#include "heom_engine.cuh"
#include "heom_internal.h"

namespace heom {

const void* smem_kernel_f32_real(int N, bool reg) {
  switch (N) {
    case 1: return reg ? (const void*)heom_smem_kernel<1, false, true>
                    : (const void*)heom_smem_kernel<1, false, false>;
    case 2: return reg ? (const void*)heom_smem_kernel<2, false, true>
                    : (const void*)heom_smem_kernel<2, false, false>;
    case 3: return reg ? (const void*)heom_smem_kernel<3, false, true>
                    : (const void*)heom_smem_kernel<3, false, false>;
    case 4: return reg ? (const void*)heom_smem_kernel<4, false, true>
                    : (const void*)heom_smem_kernel<4, false, false>;
    case 5: return reg ? (const void*)heom_smem_kernel<5, false, true>
                    : (const void*)heom_smem_kernel<5, false, false>;
    case 6: return reg ? (const void*)heom_smem_kernel<6, false, true>
                    : (const void*)heom_smem_kernel<6, false, false>;
    case 7: return reg ? (const void*)heom_smem_kernel<7, false, true>
                    : (const void*)heom_smem_kernel<7, false, false>;
    case 8: return reg ? (const void*)heom_smem_kernel<8, false, true>
                    : (const void*)heom_smem_kernel<8, false, false>;
    default: return nullptr;
  }
}
}  // namespace heom
