// Instantiations of the dataflow engine (launch mode 3) for N = 1..8, double precision.
// (One translation unit per precision so they compile in parallel.)
#include "heom_flow.cuh"
#include "heom_internal.h"

namespace heom {

const void* flow_kernel_f64(int N, bool cplx) {
  switch (N) {
    case 1: return cplx ? (const void*)heom_flow_kernel<1, double, false, true> : (const void*)heom_flow_kernel<1, double, false, false>;
    case 2: return cplx ? (const void*)heom_flow_kernel<2, double, false, true> : (const void*)heom_flow_kernel<2, double, false, false>;
    case 3: return cplx ? (const void*)heom_flow_kernel<3, double, false, true> : (const void*)heom_flow_kernel<3, double, false, false>;
    case 4: return cplx ? (const void*)heom_flow_kernel<4, double, false, true> : (const void*)heom_flow_kernel<4, double, false, false>;
    case 5: return cplx ? (const void*)heom_flow_kernel<5, double, false, true> : (const void*)heom_flow_kernel<5, double, false, false>;
    case 6: return cplx ? (const void*)heom_flow_kernel<6, double, false, true> : (const void*)heom_flow_kernel<6, double, false, false>;
    case 7: return cplx ? (const void*)heom_flow_kernel<7, double, false, true> : (const void*)heom_flow_kernel<7, double, false, false>;
    case 8: return cplx ? (const void*)heom_flow_kernel<8, double, false, true> : (const void*)heom_flow_kernel<8, double, false, false>;
    default: return nullptr;
  }
}

}  // namespace heom
