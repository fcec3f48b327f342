// Instantiations of the dataflow engine (launch mode 3) for N = 1..8, mixed precision (float auxiliaries, float-float root).
// One node per thread for every N and H; with real H and N >= 4 also 2 to 6
// nodes per thread (hierarchies too large for one node per thread).
// (One translation unit per precision so they compile in parallel.)
#include "heom_flow.cuh"
#include "heom_internal.h"

namespace heom {

namespace {
template <int N, typename R, bool MIXED>
const void* flow_pick(bool cplx, int npt) {
  if (npt == 1)
    return cplx ? (const void*)heom_flow_kernel<N, R, MIXED, true, 1> : (const void*)heom_flow_kernel<N, R, MIXED, false, 1>;
  if constexpr (N >= 4) {
    if (cplx) return nullptr;
    switch (npt) {
      case 2: return (const void*)heom_flow_kernel<N, R, MIXED, false, 2>;
      case 3: return (const void*)heom_flow_kernel<N, R, MIXED, false, 3>;
      case 4: return (const void*)heom_flow_kernel<N, R, MIXED, false, 4>;
      case 5: return (const void*)heom_flow_kernel<N, R, MIXED, false, 5>;
      case 6: return (const void*)heom_flow_kernel<N, R, MIXED, false, 6>;
      default: return nullptr;
    }
  }
  return nullptr;
}
}  // namespace

const void* flow_kernel_f32(int N, bool cplx, int npt) {
  switch (N) {
    case 1: return flow_pick<1, float, true>(cplx, npt);
    case 2: return flow_pick<2, float, true>(cplx, npt);
    case 3: return flow_pick<3, float, true>(cplx, npt);
    case 4: return flow_pick<4, float, true>(cplx, npt);
    case 5: return flow_pick<5, float, true>(cplx, npt);
    case 6: return flow_pick<6, float, true>(cplx, npt);
    case 7: return flow_pick<7, float, true>(cplx, npt);
    case 8: return flow_pick<8, float, true>(cplx, npt);
    default: return nullptr;
  }
}

}  // namespace heom
