// Instantiations of the distributed-shared-memory engine kernel (mixed precision,
// complex Hamiltonian); a translation unit of its own so it compiles in parallel.
#include "heom_engine.cuh"
#include "heom_internal.h"

namespace heom {

const void* smem_kernel_f32_cplx(int N, bool reg) {
  switch (N) {
    case 1: return reg ? (const void*)heom_smem_kernel<1, true, true>
                    : (const void*)heom_smem_kernel<1, true, false>;
    case 2: return reg ? (const void*)heom_smem_kernel<2, true, true>
                    : (const void*)heom_smem_kernel<2, true, false>;
    case 3: return reg ? (const void*)heom_smem_kernel<3, true, true>
                    : (const void*)heom_smem_kernel<3, true, false>;
    case 4: return reg ? (const void*)heom_smem_kernel<4, true, true>
                    : (const void*)heom_smem_kernel<4, true, false>;
    case 5: return reg ? (const void*)heom_smem_kernel<5, true, true>
                    : (const void*)heom_smem_kernel<5, true, false>;
    case 6: return reg ? (const void*)heom_smem_kernel<6, true, true>
                    : (const void*)heom_smem_kernel<6, true, false>;
    case 7: return reg ? (const void*)heom_smem_kernel<7, true, true>
                    : (const void*)heom_smem_kernel<7, true, false>;
    case 8: return reg ? (const void*)heom_smem_kernel<8, true, true>
                    : (const void*)heom_smem_kernel<8, true, false>;
    default: return nullptr;
  }
}
}  // namespace heom
