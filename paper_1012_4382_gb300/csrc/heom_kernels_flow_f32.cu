// Instantiations of the dataflow engine (launch mode 3) for N = 1..8, mixed precision (float auxiliaries, float-float root).
// (One translation unit per precision so they compile in parallel.)
#include "heom_flow.cuh"
#include "heom_internal.h"

namespace heom {

const void* flow_kernel_f32(int N, bool cplx) {
  switch (N) {
    case 1: return cplx ? (const void*)heom_flow_kernel<1, float, true, true> : (const void*)heom_flow_kernel<1, float, true, false>;
    case 2: return cplx ? (const void*)heom_flow_kernel<2, float, true, true> : (const void*)heom_flow_kernel<2, float, true, false>;
    case 3: return cplx ? (const void*)heom_flow_kernel<3, float, true, true> : (const void*)heom_flow_kernel<3, float, true, false>;
    case 4: return cplx ? (const void*)heom_flow_kernel<4, float, true, true> : (const void*)heom_flow_kernel<4, float, true, false>;
    case 5: return cplx ? (const void*)heom_flow_kernel<5, float, true, true> : (const void*)heom_flow_kernel<5, float, true, false>;
    case 6: return cplx ? (const void*)heom_flow_kernel<6, float, true, true> : (const void*)heom_flow_kernel<6, float, true, false>;
    case 7: return cplx ? (const void*)heom_flow_kernel<7, float, true, true> : (const void*)heom_flow_kernel<7, float, true, false>;
    case 8: return cplx ? (const void*)heom_flow_kernel<8, float, true, true> : (const void*)heom_flow_kernel<8, float, true, false>;
    default: return nullptr;
  }
}

}  // namespace heom
