// Private declarations shared by the translation units of libheom.
#pragma once

#include <cstdint>
#include <vector>

namespace heom {

// Engine kernel entry points for N = 1..8 (nullptr otherwise); reg selects
// the register-resident node view.
const void* engine_kernel_f64_real(int N, bool reg);
const void* engine_kernel_f64_cplx(int N, bool reg);
const void* engine_kernel_f32_real(int N, bool reg);
const void* engine_kernel_f32_cplx(int N, bool reg);
// Scaled hierarchies (HEOM_FLAG_SCALED), N = 1..8, load views only.
const void* engine_kernel_scaled_f64(int N, bool cplx);
const void* engine_kernel_scaled_f32(int N, bool cplx);
// Large-N engine (9..24 sites).
const void* large_kernel(bool fp64, bool cplx, bool scaled);
// Dataflow engine (launch mode 3, one hierarchy on the whole GPU), N = 1..8,
// npt nodes per thread (nullptr where that count is not built).
const void* flow_kernel_f32(int N, bool cplx, int npt);
const void* flow_kernel_f64(int N, bool cplx, int npt);
inline const void* flow_kernel(bool fp64, bool cplx, int N, int npt = 1) {
  return fp64 ? flow_kernel_f64(N, cplx, npt) : flow_kernel_f32(N, cplx, npt);
}
// Distributed-shared-memory engine (mixed precision only).
const void* smem_kernel_f32_real(int N, bool reg);
const void* smem_kernel_f32_cplx(int N, bool reg);
inline const void* smem_kernel(bool cplx, bool reg, int N) {
  return cplx ? smem_kernel_f32_cplx(N, reg) : smem_kernel_f32_real(N, reg);
}
// nullptr where there is no such kernel (N > 8, or a scaled register view)
inline const void* engine_kernel(bool fp64, bool cplx, bool reg, int N, bool scaled = false) {
  if (scaled) {
    if (reg) return nullptr;
    return fp64 ? engine_kernel_scaled_f64(N, cplx) : engine_kernel_scaled_f32(N, cplx);
  }
  if (fp64) return cplx ? engine_kernel_f64_cplx(N, reg) : engine_kernel_f64_real(N, reg);
  return cplx ? engine_kernel_f32_cplx(N, reg) : engine_kernel_f32_real(N, reg);
}

// Hierarchy index builder (heom_index.cpp).
int64_t num_nodes(int N, int K);  // -1 on overflow beyond int64
struct Index {
  int N = 0, K = 0;
  int64_t M = 0;
  std::vector<int32_t> multi;  // [M][N]
  std::vector<int32_t> up;     // [M][N]
  std::vector<int32_t> down;   // [M][N]
};
void build_index(int N, int K, Index& out);
int64_t rank_of(const int32_t* n, int N, int K);
// Writes the element-major tables up[j*Mpad + i] and the packed down links
// (n_j << 24 | index) without allocating; returns the number of nodes.
int64_t write_packed_tables(int N, int K, int Mpad, int32_t* up, int32_t* dn);

}  // namespace heom
