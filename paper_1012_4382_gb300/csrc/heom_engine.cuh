// heom_engine.cuh -- device side of libheom: the fused right-hand-side + RK4
// stage kernel for hierarchies with N <= 8 sites.
//
// Method (Kreisbeck et al., arXiv:1012.4382, App. A2 Eqs. labsevena/lab8, App. B):
//   d sigma_n/dt = -i (H_eff sigma_n - sigma_n H_eff^+) - (sum_j n_j gamma_j) sigma_n
//                  + sum_j i V_j^x sigma_{n+e_j} + sum_j n_j theta_j sigma_{n-e_j}
//   H_eff = H - (i/2) diag(Gamma_RC + Gamma_phot)            (App. A1, end)
//   theta_j X = i alpha_j V_j^x X + beta_j V_j^o X,  alpha = 2 lambda k_B T, beta = lambda gamma
//   V_j = |j><j|, so (V_j^x X)_ab = (d_aj - d_bj) X_ab and (V_j^o X)_ab = (d_aj + d_bj) X_ab.
//
// Storage.  Every sigma_n is Hermitian (the right-hand side maps Hermitian
// matrices to Hermitian ones), so a node is stored as N*N reals: element
// (a, b) of the packed matrix P holds Re sigma_ab for a <= b and Im sigma_ba
// for a > b.  Arrays are element-major ("structure of arrays"):
// w[p * Mpad + n] is packed element p of node n, so a warp that handles 32
// consecutive nodes reads and writes every element with one 128-byte
// (float) or 256-byte (double) transaction, and neighbour gathers
// w[p * Mpad + up_j(n)] touch ascending, nearly contiguous addresses because
// n -> n + e_j preserves the lexicographic order inside a level.
//
// Time stepping.  The right-hand side is linear and autonomous, so classic
// RK4 (App. B) is the degree-4 Taylor polynomial of h L.  It is evaluated in
// Horner form, which gives the same result up to rounding with three arrays
// (y, wa, wb) instead of four and 11 instead of 18 node-array sweeps per step:
//   stage 0: wa = y + (h/4) L y      stage 1: wb = y + (h/3) L wa
//   stage 2: wa = y + (h/2) L wb     stage 3: y  = y + h L wa
// The efficiency integral eta' = sum_m Gamma_RC,m rho_mm is the extra row of
// the augmented linear system; its RK4 update is exactly
// eta += h * sum_m Gamma_RC,m (wa_0)_mm with wa the stage-3 input, and the
// same holds for the radiative loss with Gamma_phot.
//
// Parallel decomposition.  A "team" (one thread-block cluster, or the whole
// grid) owns one hierarchy at a time.  Nodes are grouped in blocks of 32
// (one warp lane per node); each node block is split into G "unit groups"
// (1 <= G <= 32): warp (block, g) computes the packed elements whose unit
// index u satisfies u % G == g.  Units are the N(N-1)/2 off-diagonal pairs
// (two packed reals each) and the N diagonal entries.  With G <= 2 a thread
// loads its node's whole packed matrix into registers once (RegView); with
// larger G each unit loads the elements it needs (LoadView), so many short
// threads share a node.  All index arithmetic on the packed matrix is resolved
// at compile time.  Between RK4 stages the team synchronises with a hardware
// cluster barrier (release/acquire at cluster scope) or a software grid
// barrier with a bounded wait.  In mixed precision the root node rho is
// split into one work item per unit, each run by one lane of its own warp,
// so that its double-precision accumulations (FP64 runs at 1/64 of the FP32
// rate on this GPU) proceed in parallel rather than in one serial chain.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

namespace heom {

constexpr int kMaxSmallN = 8;
constexpr int kMaxSites = 24;
constexpr int kStatusTimeout = 1;
constexpr int kStatusNonFinite = 2;  // a population, the trace, eta or the loss came out NaN or infinite
constexpr uint64_t kBarrierLimitNs = 2000000000ull;  // a stage barrier gives up after 2 s

// Per-instance device descriptor (host fills it; see heom_runtime.cu).
struct Inst {
  int32_t N, K, M, Mpad;
  int32_t complex_h, terminator;
  int32_t wstride;     // scaled hierarchy: K + 2, the row length of wsc
  int32_t pad1;
  const int32_t* up;   // [N][Mpad] index of n + e_j or -1
  const int32_t* dn;   // [N][Mpad] (n_j << 24) | index of n - e_j, or -1
  void* y;             // [N*N][Mpad] packed state, element-major (R)
  void* wa;            // stage buffers, same layout
  void* wb;
  // mixed precision: the root node rho in float-float, N*N (hi, lo) float
  // pairs per buffer (y0, wa0, wb0); its hi parts are also kept in column 0 of
  // y, wa, wb for the neighbours
  void* y0;
  void* w0a;
  void* w0b;
  const void* coef;    // flat coefficient block, see CoefLayout below
  const void* ngam;    // [Mpad] sum_j n_j gamma_j per node (R)
  const void* wsc;     // scaled hierarchy (HEOM_FLAG_SCALED): link weights (R), see scaled_up; else null
  double* acc;         // [8] eta, loss, xi = int eta dt, elapsed time (fs), steps done by the last call
                       // (read at the start of a call, written at its end)
  void* parts;         // [32] slots of kPartBytes: partial (eta, loss, xi) sums per unit group,
                       // float-float x3 (mixed) or double x3
  double* out_pops;    // [nout][N] populations (may be null)
  double* out_el;      // [nout][2] eta, loss (may be null)
  int* done;           // set to 1 (system-wide release) when the instance is finished (may be null)
  int64_t nsteps;
  int64_t out_every;
  double dt;
  double hd[4];        // Horner steps h/4, h/3, h/2, h
  float hh[4], hl[4];  // the same as float-float pairs (hi, lo)
  float ec[4 * kMaxSites];  // per site a: h*Gamma_RC,a (hi, lo), h*Gamma_phot,a (hi, lo)
  float xc[2 * kMaxSites];  // per site a: (h^2/2)*Gamma_RC,a (hi, lo)
  double stop_trace;        // > 0: stop after the first step whose site population is below it
};

// Bytes of one running-sum slot in Inst::parts.
constexpr int kPartBytes = 32;

// Coefficient block (host writes it with the same layout; 16-byte aligned):
//   R J[N][JS]    real part of H off the diagonal (rad/fs), zero diagonal; rows padded
//                 to JS = 4*ceil(N/4) entries; exactly symmetric
//   R Ji[N][JS]   imaginary part of H, same padding; exactly antisymmetric
//   R site[N][4]  per site a: eps_a = H_aa minus the mean diagonal (rad/fs),
//                 goff_a = (Gamma_RC,a + Gamma_phot,a)/2 + c_a (1/fs), alpha_a = 2 lambda_a k_B T,
//                 beta_a = lambda_a gamma_a (rad^2/fs^2); c_a is the low-temperature
//                 correction rate (0 when off), which damps only off-diagonal elements
//   R gam[N]      gamma_a (rad/fs)
//   R gd[N]       (Gamma_RC,a + Gamma_phot,a)/2, the damping of the diagonal element a
//   then, 16-byte aligned: double trap[N], double recomb[N] (1/fs)
template <typename R>
struct CoefLayout {
  __host__ __device__ static constexpr int JS(int N) { return (N + 3) / 4 * 4; }
  __host__ __device__ static constexpr int J(int N) { return 0; }
  __host__ __device__ static constexpr int Ji(int N) { return N * JS(N); }
  __host__ __device__ static constexpr int site(int N) { return 2 * N * JS(N); }
  __host__ __device__ static constexpr int gam(int N) { return 2 * N * JS(N) + 4 * N; }
  __host__ __device__ static constexpr int gd(int N) { return 2 * N * JS(N) + 5 * N; }
  __host__ __device__ static constexpr int reals(int N) { return 2 * N * JS(N) + 6 * N; }
  // byte offset of the double arrays
  __host__ __device__ static constexpr int dbl_offset(int N) {
    return ((reals(N) * (int)sizeof(R) + 15) / 16) * 16;
  }
  __host__ __device__ static constexpr int bytes(int N) { return dbl_offset(N) + 2 * N * 8; }
};

struct EngineArgs {
  const Inst* insts;
  const int32_t* team_first;  // [nteams + 1]
  const int32_t* team_list;   // instance ids, team by team
  int32_t G;                  // unit groups per node (power of two)
  int32_t logG;
  int32_t mode;               // 0: cluster teams, 1: whole grid is one team
  int32_t team_ctas;          // CTAs per team in mode 0
  unsigned* gsync;            // grid barrier counter (mode 1), zero at launch
  int* status;                // error bits
};

// ---------------------------------------------------------------- helpers

template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// pair index u -> (a, b), a < b, in the order (0,1),(0,2),...,(1,2),...
__host__ __device__ constexpr int pair_a(int N, int u) {
  int a = 0;
  while (u >= N - 1 - a) { u -= N - 1 - a; ++a; }
  return a;
}
__host__ __device__ constexpr int pair_b(int N, int u) {
  int a = 0;
  while (u >= N - 1 - a) { u -= N - 1 - a; ++a; }
  return a + 1 + u;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// Spins until *p has reached target (acquire loads).  The comparison is made
// on the wrapped difference, (int)(*p - target) < 0 means "not yet", so it
// stays right when the 32-bit counter and target pass 2^32 during a long
// launch (the counter never lags the target by 2^31 or more).  Gives up after
// limit_ns of global time, sets kStatusTimeout in *status and returns false;
// also returns false as soon as another thread has set that bit.
__device__ __forceinline__ bool bounded_wait_geq(const unsigned* p, unsigned target, uint64_t limit_ns, int* status) {
  const uint64_t t0 = global_timer_ns();
  unsigned spins = 0;
  while ((int)(ld_acquire_gpu(p) - target) < 0) {
    if ((++spins & 1023u) == 0) {
      if (ld_volatile(status) & kStatusTimeout) return false;
      if (global_timer_ns() - t0 > limit_ns) {
        atomicOr(status, kStatusTimeout);
        return false;
      }
    }
  }
  return true;
}

// Barrier between RK4 stages.  Returns false when a bounded wait expired
// (grid mode only); the caller then leaves the kernel.
__device__ __forceinline__ bool team_barrier(const EngineArgs& A, unsigned& epoch) {
  if (A.mode == 0) {
    if (A.team_ctas == 1) {
      __syncthreads();
    } else {
      asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
    return true;
  }
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned target = epoch * gridDim.x;
    red_release_gpu_add(A.gsync, 1u);
    s_ok = bounded_wait_geq(A.gsync, target, kBarrierLimitNs, A.status) ? 1 : 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------ node views
//
// A view gives the unit code everything it touches for one node n in one RK4
// stage, with every index known at compile time:
//   P<p>()        packed element p = k*N + l of the node's stage input
//   Up<j>(), Dn<j>()  link handles of n + e_j, n - e_j (-1: no link)
//   Nj<j>()       n_j
//   G<p>(h)       packed element p of the linked node h's stage input
//   Y<p>(), St<p>(v)  the node's y element, and the store of its stage output
// Global views address the element-major arrays in device memory; shared
// views address one thread-block cluster's distributed shared memory, where
// each CTA holds a contiguous slice of the nodes and link handles are
// shared::cluster addresses.  "Reg" views load the node's whole packed matrix
// into registers once; "Load" views load each element where a unit uses it.

// Loads *a when q holds, else returns 0; predicated, so that gathers of
// absent neighbours need no branch.
__device__ __forceinline__ float ld_global_or0(const float* a, bool q) {
  float v = 0.f;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.f32 %0, [%1];\n\t}"
               : "+f"(v)
               : "l"(a), "r"((unsigned)q));
  return v;
}
__device__ __forceinline__ double ld_global_or0(const double* a, bool q) {
  double v = 0.0;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.f64 %0, [%1];\n\t}"
               : "+d"(v)
               : "l"(a), "r"((unsigned)q));
  return v;
}
template <typename R>
struct GlobalArrays {
  const R* __restrict__ win;
  R* __restrict__ wout;
  const R* __restrict__ y;
  const int32_t* __restrict__ up;
  const int32_t* __restrict__ dn;
  int Mp;
};

template <int N, typename R, bool REG>
struct GlobalView {
  const R* __restrict__ win;  // column n of the input
  const R* __restrict__ base;  // input, for gathers
  R* __restrict__ wout;
  const R* __restrict__ y;
  const int32_t* __restrict__ upt;
  const int32_t* __restrict__ dnt;
  int Mp;
  R sg[REG ? N * N : 1];
  int upr[REG ? N : 1], dnr[REG ? N : 1];
  __device__ __forceinline__ GlobalView(const GlobalArrays<R>& a, int n)
      : win(a.win + n), base(a.win), wout(a.wout + n), y(a.y + n), upt(a.up + n), dnt(a.dn + n), Mp(a.Mp) {
    if constexpr (REG) {
#pragma unroll
      for (int p = 0; p < N * N; ++p) sg[p] = win[p * Mp];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        upr[j] = upt[j * Mp];
        dnr[j] = dnt[j * Mp];
      }
    }
  }
  template <int p>
  __device__ __forceinline__ R P() const {
    if constexpr (REG) return sg[p];
    else return win[p * Mp];
  }
  template <int j>
  __device__ __forceinline__ int Up() const {
    if constexpr (REG) return upr[j];
    else return upt[j * Mp];
  }
  template <int j>
  __device__ __forceinline__ int DnRaw() const {
    if constexpr (REG) return dnr[j];
    else return dnt[j * Mp];
  }
  template <int j>
  __device__ __forceinline__ int Dn() const {
    const int d = DnRaw<j>();
    return d < 0 ? -1 : (d & 0xFFFFFF);
  }
  template <int j>
  __device__ __forceinline__ R Nj() const {
    const int d = DnRaw<j>();
    return d < 0 ? R(0) : R(d >> 24);
  }
  template <int p>
  __device__ __forceinline__ R G(int h) const { return base[p * Mp + h]; }
  // element p of node h, or 0 when h == -1 (no link)
  template <int p>
  __device__ __forceinline__ R G0(int h) const { return ld_global_or0(base + (p * Mp + h), h != -1); }
  template <int p>
  __device__ __forceinline__ R Y() const { return y[p * Mp]; }
  template <int p>
  __device__ __forceinline__ void St(R v) const { wout[p * Mp] = v; }
  // the same with run-time indices (load views)
  __device__ __forceinline__ R Pr(int p) const { return win[p * Mp]; }
  __device__ __forceinline__ int Upr(int j) const { return upt[j * Mp]; }
  __device__ __forceinline__ int Dnr(int j) const {
    const int d = dnt[j * Mp];
    return d < 0 ? -1 : (d & 0xFFFFFF);
  }
  __device__ __forceinline__ R Njr(int j) const {
    const int d = dnt[j * Mp];
    return d < 0 ? R(0) : R(d >> 24);
  }
  __device__ __forceinline__ R Gr(int p, int h) const { return base[p * Mp + h]; }
  __device__ __forceinline__ R Yr(int p) const { return y[p * Mp]; }
  __device__ __forceinline__ void Str(int p, R v) const { wout[p * Mp] = v; }
};

__device__ __forceinline__ float ld_dsmem_f32_or0(unsigned addr, bool q) {
  float v = 0.f;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.shared::cluster.f32 %0, [%1];\n\t}"
               : "+f"(v)
               : "r"(addr), "r"((unsigned)q)
               : "memory");
  return v;
}

__device__ __forceinline__ float ld_dsmem_f32(unsigned addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ unsigned map_to_rank(unsigned smem_addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr), "r"(rank));
  return r;
}
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Shared-memory slice of one CTA: arrays [N*N][B] (floats), link tables
// [N][B] of handles, n_j [N][B] (bytes), damping [B].  A handle is the
// shared::cluster address of element (0, l) of the first array in the owning
// CTA; element p of the array at byte offset o is at handle + o + 4*p*B,
// because each CTA's shared memory is one contiguous range of the cluster
// window and every CTA uses the same layout.
struct SmemArrays {
  const float* win;
  float* wout;
  const float* y;
  const unsigned* up;
  const unsigned* dn;
  const unsigned char* nj;
  const float* ngam;
  unsigned win_off;  // byte offset of the stage input from the start of the dynamic shared memory
  int B;
};

template <int N, bool REG>
struct SmemView {
  const float* win;
  float* wout;
  const float* y;
  const unsigned* upt;
  const unsigned* dnt;
  const unsigned char* njt;
  unsigned win_off;
  int B;
  float sg[REG ? N * N : 1];
  __device__ __forceinline__ SmemView(const SmemArrays& a, int l)
      : win(a.win + l), wout(a.wout + l), y(a.y + l), upt(a.up + l), dnt(a.dn + l), njt(a.nj + l),
        win_off(a.win_off), B(a.B) {
    if constexpr (REG) {
#pragma unroll
      for (int p = 0; p < N * N; ++p) sg[p] = win[p * B];
    }
  }
  template <int p>
  __device__ __forceinline__ float P() const {
    if constexpr (REG) return sg[p];
    else return win[p * B];
  }
  template <int j>
  __device__ __forceinline__ int Up() const { return (int)upt[j * B]; }
  template <int j>
  __device__ __forceinline__ int Dn() const { return (int)dnt[j * B]; }
  template <int j>
  __device__ __forceinline__ float Nj() const { return (float)njt[j * B]; }
  template <int p>
  __device__ __forceinline__ float G(int h) const {
    return ld_dsmem_f32((unsigned)h + win_off + (unsigned)(p * B * 4));
  }
  template <int p>
  __device__ __forceinline__ float G0(int h) const {
    return ld_dsmem_f32_or0((unsigned)h + win_off + (unsigned)(p * B * 4), h != -1);
  }
  template <int p>
  __device__ __forceinline__ float Y() const { return y[p * B]; }
  template <int p>
  __device__ __forceinline__ void St(float v) const { wout[p * B] = v; }
  // the same with run-time indices (load views)
  __device__ __forceinline__ float Pr(int p) const { return win[p * B]; }
  __device__ __forceinline__ int Upr(int j) const { return (int)upt[j * B]; }
  __device__ __forceinline__ int Dnr(int j) const { return (int)dnt[j * B]; }
  __device__ __forceinline__ float Njr(int j) const { return (float)njt[j * B]; }
  __device__ __forceinline__ float Gr(int p, int h) const {
    return ld_dsmem_f32((unsigned)h + win_off + (unsigned)(p * B * 4));
  }
  __device__ __forceinline__ float Yr(int p) const { return y[p * B]; }
  __device__ __forceinline__ void Str(int p, float v) const { wout[p * B] = v; }
};

// S = Re sigma (symmetric), A = Im sigma (antisymmetric) from the packed view
template <int N, int k, int l, class V>
__device__ __forceinline__ auto Sv(const V& v) {
  if constexpr (k <= l) return v.template P<k * N + l>();
  else return v.template P<l * N + k>();
}
template <int N, int k, int l, class V, typename R>
__device__ __forceinline__ R Av(const V& v) {
  if constexpr (k < l) return v.template P<l * N + k>();
  else if constexpr (k > l) return -v.template P<k * N + l>();
  else return R(0);
}

// ------------------------------------------------------------ float-float
//
// FP64 runs at 1/64 of the FP32 rate on this GPU (a double-precision warp
// instruction occupies a sub-partition's FP64 unit for 64 cycles whatever the
// number of active lanes), so the mixed-precision kernels keep rho's RK4
// accumulation and the eta integral in float-float: an unevaluated sum
// hi + lo of two floats, carried with the error-free transformations TwoSum
// (Knuth) and TwoProduct-by-FMA (Dekker/Ogita-Rump-Oishi).  Each operation
// below is exact up to a relative 2^-48; no double-precision instruction runs
// in the stage loop.

struct FF {
  float h, l;
};

// y + (ah + al) * r
__device__ __forceinline__ FF ff_axpy(FF y, float ah, float al, float r) {
  const float p = ah * r;
  const float e = fmaf(ah, r, -p) + al * r;  // error of the product, plus the low part of a
  const float s = y.h + p;                    // TwoSum(y.h, p) = (s, t)
  const float bp = s - y.h;
  float t = (y.h - (s - bp)) + (p - bp);
  t += y.l + e;
  const float h = s + t;                      // FastTwoSum renormalisation
  return FF{h, t - (h - s)};
}

// a + b
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.h + b.h;
  const float bp = s - a.h;
  float t = (a.h - (s - bp)) + (b.h - bp);
  t += a.l + b.l;
  const float h = s + t;
  return FF{h, t - (h - s)};
}

// (ch + cl) * (x.h + x.l)
__device__ __forceinline__ FF ff_mul(float ch, float cl, FF x) {
  const float p = ch * x.h;
  const float e = fmaf(ch, x.h, -p) + (ch * x.l + cl * x.h);
  const float h = p + e;
  return FF{h, e - (h - p)};
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.h + (double)a.l; }

// Running eta and loss sums of one thread (the owner of some of the root's
// diagonal units): float-float in the mixed kernels, double in the FP64 ones.
template <typename R>
struct EtaAcc;
//
// xi = int eta dt (for the trapping time <t> = t eta - xi, Eq. trappingtime
// integrated by parts) is one more component of the augmented system:
// RK4 on (y, eta, xi) gives xi += h eta + (h^2/2) sum_a Gamma_a (w_b)_aa with
// w_b the stage-2 input (y + h/3 L y + h^2/12 L^2 y).  Each owner adds its
// share: h e (its own running eta sum, before this step's update) and its
// diagonals of w_b; h eta at the start of the call is added once at the end.
template <>
struct EtaAcc<float> {
  FF e{0.f, 0.f}, l{0.f, 0.f}, x{0.f, 0.f};
  // contribution of diagonal a of the root's stage-3 input w: h Gamma_a w
  __device__ __forceinline__ void add(const Inst& I, int a, FF w) {
    e = ff_add(e, ff_mul(I.ec[4 * a], I.ec[4 * a + 1], w));
    l = ff_add(l, ff_mul(I.ec[4 * a + 2], I.ec[4 * a + 3], w));
  }
  // contribution of diagonal a of the root's stage-2 input w: (h^2/2) Gamma_a w
  __device__ __forceinline__ void add_xi(const Inst& I, int a, FF w) {
    x = ff_add(x, ff_mul(I.xc[2 * a], I.xc[2 * a + 1], w));
  }
  // once per step, before the step's eta update: xi += h e
  __device__ __forceinline__ void step_xi(const Inst& I) { x = ff_add(x, ff_mul(I.hh[3], I.hl[3], e)); }
  __device__ __forceinline__ void store(const Inst& I, int slot) const {
    float* p = static_cast<float*>(I.parts) + (kPartBytes / 4) * slot;
    p[0] = e.h;
    p[1] = e.l;
    p[2] = l.h;
    p[3] = l.l;
    p[4] = x.h;
    p[5] = x.l;
  }
};
template <>
struct EtaAcc<double> {
  double e = 0.0, l = 0.0, x = 0.0;
  __device__ __forceinline__ void add(const Inst& I, const double* cfd, int N, int a, double w) {
    e += I.dt * cfd[a] * w;
    l += I.dt * cfd[N + a] * w;
  }
  __device__ __forceinline__ void add_xi(const Inst& I, const double* cfd, int a, double w) {
    x += 0.5 * I.dt * I.dt * cfd[a] * w;
  }
  __device__ __forceinline__ void step_xi(const Inst& I) { x += I.dt * e; }
  __device__ __forceinline__ void store(const Inst& I, int slot) const {
    double* p = static_cast<double*>(I.parts) + (kPartBytes / 8) * slot;
    p[0] = e;
    p[1] = l;
    p[2] = x;
  }
};

// eta and loss at the current step: the value at the start of the call plus
// every owner's running sum (read through L2: the owners wrote them before
// the last stage barrier).
template <typename R>
__device__ __forceinline__ void eta_total(const Inst& I, int nslots, double acc0, double acc1, double& e, double& l,
                                          double* xs = nullptr) {
  if constexpr (sizeof(R) == 4) {
    FF se{0.f, 0.f}, sl{0.f, 0.f}, sx{0.f, 0.f};
    const float* p = static_cast<const float*>(I.parts);
    constexpr int S = kPartBytes / 4;
    for (int k = 0; k < nslots; ++k) {
      se = ff_add(se, FF{__ldcg(p + S * k), __ldcg(p + S * k + 1)});
      sl = ff_add(sl, FF{__ldcg(p + S * k + 2), __ldcg(p + S * k + 3)});
      if (xs) sx = ff_add(sx, FF{__ldcg(p + S * k + 4), __ldcg(p + S * k + 5)});
    }
    e = acc0 + ff_to_double(se);
    l = acc1 + ff_to_double(sl);
    if (xs) *xs = ff_to_double(sx);
  } else {
    double se = 0.0, sl = 0.0, sx = 0.0;
    const double* p = static_cast<const double*>(I.parts);
    constexpr int S = kPartBytes / 8;
    for (int k = 0; k < nslots; ++k) {
      se += __ldcg(p + S * k);
      sl += __ldcg(p + S * k + 1);
      sx += __ldcg(p + S * k + 2);
    }
    e = acc0 + se;
    l = acc1 + sl;
    if (xs) *xs = sx;
  }
}

// Raises kStatusNonFinite (reported as HEOM_ENONFINITE) when v is NaN or
// infinite: a run that diverged must not come back as a success.
__device__ __forceinline__ void flag_nonfinite(int* status, double v) {
  if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
}

// The eta and loss row `row` (lead thread, one stage after the output step,
// once the team barrier has ordered the owners' sums and the population row).
// Every output row is also checked for NaN or infinity: the populations of
// the row, eta and the loss.
template <typename R>
__device__ __forceinline__ void eta_write_row(const Inst& I, int nslots, double acc0, double acc1, int64_t row,
                                              int* status) {
  double e, l;
  eta_total<R>(I, nslots, acc0, acc1, e, l);
  flag_nonfinite(status, e);
  flag_nonfinite(status, l);
  if (I.out_pops)
    for (int a = 0; a < I.N; ++a) flag_nonfinite(status, __ldcg(I.out_pops + row * I.N + a));
  if (!I.out_el) return;
  I.out_el[2 * row] = e;
  I.out_el[2 * row + 1] = l;
}

template <typename R>
struct StageCoef {
  R h;         // Horner step of this stage (R precision)
  float hl;    // low part of the float-float step (mixed root)
  FF* root_in;   // mixed: the root's float-float stage input
  FF* root_out;  // mixed: the root's float-float stage output
  const FF* root_y;  // mixed: the root's float-float y
};

// Loads M consecutive coefficients (M a multiple of 4, 16-byte aligned) as
// vectors.
template <int M, typename R>
__device__ __forceinline__ void load_row(const R* __restrict__ p, R* out) {
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int i = 0; i < M / 4; ++i) {
      const float4 v = reinterpret_cast<const float4*>(p)[i];
      out[4 * i] = v.x;
      out[4 * i + 1] = v.y;
      out[4 * i + 2] = v.z;
      out[4 * i + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < M / 2; ++i) {
      const double2 v = reinterpret_cast<const double2*>(p)[i];
      out[2 * i] = v.x;
      out[2 * i + 1] = v.y;
    }
  }
}

// Link weights of the scaled hierarchy.  The auxiliaries are stored as
// sigma~_n = sigma_n / S(n), S(n) = prod_j sqrt(n_j! s_j^{n_j}) with s_j the
// modulus of the bath amplitude 2 lambda_j kT - i lambda_j gamma_j (Shi et
// al., J. Chem. Phys. 130, 084105 (2009); the paper's introduction names the
// scaled hierarchy).  In these variables the up link of site j carries
// S(n+e_j)/S(n) = sqrt((n_j+1) s_j) and the down link n_j S(n-e_j)/S(n) =
// sqrt(n_j / s_j); the host tabulates both per site and n_j:
// w[j * 2S + n] = sqrt((n+1) s_j), w[j * 2S + S + n] = sqrt(n / s_j), S = K + 2.
template <typename R>
__device__ __forceinline__ R scaled_up(const R* __restrict__ w, int S, int j, R nj) {
  return __ldg(w + j * 2 * S + (int)nj);
}
template <typename R>
__device__ __forceinline__ R scaled_dn(const R* __restrict__ w, int S, int j, R nj) {
  return __ldg(w + j * 2 * S + S + (int)nj);
}

// Right-hand side of unit u (pair (a, b) or diagonal a) of one node.
// Returns the real part in re and, for pairs, the imaginary part in im.
// J is symmetric and Ji antisymmetric, so all the coefficients of a unit sit
// in rows a and b and in the site records of a and b.  tc[j] is the
// terminator factor (n_j + 1) / (ngam + gamma_j) of a leaf node (term), 0
// elsewhere.  BF: branch-free form -- absent neighbours read as 0 (predicated
// loads), n_j is 0 where there is no down link and the terminator terms are
// always evaluated, so the compiler may issue the loads of several units
// ahead of their arithmetic; worth it where a thread runs many units of a
// node and arithmetic is cheap (FP32, unit groups G <= 2).  Otherwise each
// term is skipped where it is absent, which saves FP64 instructions (1/64
// rate) and the latency of unneeded loads when a thread runs one unit.
// SC: scaled hierarchy, link weights from wsc (row length ws); branching form only.
template <int N, int u, typename R, bool CPLX, bool BF, bool SC, class V>
__device__ __forceinline__ void unit_rhs(const V& v, const R* __restrict__ cf, R ngam, bool term, const R* tc, R& re,
                                         R& im, const R* __restrict__ wsc, int ws) {
  static_assert(!(SC && BF), "the scaled hierarchy uses the branching form");
  using L = CoefLayout<R>;
  constexpr int NP = N * (N - 1) / 2;
  constexpr int JS = L::JS(N);
  re = R(0);
  im = R(0);
  if constexpr (u < NP) {
    constexpr int a = pair_a(N, u);
    constexpr int b = pair_b(N, u);
    constexpr int pab = a * N + b, pba = b * N + a;
    // rows a and b of J and the site records of a and b, as vectors
    R jr[2 * JS], sa[4], sb[4];
    load_row<JS>(cf + L::J(N) + a * JS, jr);       // J(a, k)
    load_row<JS>(cf + L::J(N) + b * JS, jr + JS);  // J(b, k) = J(k, b)
    auto ja = [&](int k) -> R { return jr[k]; };
    auto jb = [&](int k) -> R { return jr[JS + k]; };
    load_row<4>(cf + L::site(N) + 4 * a, sa);
    load_row<4>(cf + L::site(N) + 4 * b, sb);
    const R x = v.template P<pab>();   // Re sigma_ab
    const R yi = v.template P<pba>();  // Im sigma_ab
    // -i[J, sigma]: Re += [J, A]_ab, Im -= [J, S]_ab
    static_for<0, N>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (k != a) {
        if constexpr (k != b) re += ja(k) * Av<N, k, b, V, R>(v);
        im -= ja(k) * Sv<N, k, b>(v);
      }
      if constexpr (k != b) {
        if constexpr (k != a) re -= Av<N, a, k, V, R>(v) * jb(k);
        im += Sv<N, a, k>(v) * jb(k);
      }
    });
    if constexpr (CPLX) {
      // -i[i Ji, sigma] = [Ji, S] + i [Ji, A], with Ji(k, b) = -Ji(b, k)
      R ir[2 * JS];
      load_row<JS>(cf + L::Ji(N) + a * JS, ir);
      load_row<JS>(cf + L::Ji(N) + b * JS, ir + JS);
      auto ia = [&](int k) -> R { return ir[k]; };
      auto ib = [&](int k) -> R { return ir[JS + k]; };
      static_for<0, N>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if constexpr (k != a) {
          re += ia(k) * Sv<N, k, b>(v);
          if constexpr (k != b) im += ia(k) * Av<N, k, b, V, R>(v);
        }
        if constexpr (k != b) {
          re += Sv<N, a, k>(v) * ib(k);
          if constexpr (k != a) im += Av<N, a, k, V, R>(v) * ib(k);
        }
      });
    }
    // -i (eps_a - eps_b) sigma_ab, anti-Hermitian part and damping
    const R d = sa[0] - sb[0];
    const R c = ngam + sa[1] + sb[1];
    re += d * yi - c * x;
    im -= d * x + c * yi;
    const R al_a = sa[2], be_a = sa[3];
    const R al_b = sb[2], be_b = sb[3];
    // up-couplings i V_j^x sigma_{n+e_j}: j = a gives +i, j = b gives -i
    const int ua = v.template Up<a>();
    const int ub = v.template Up<b>();
    // down-couplings n_j theta_j sigma_{n-e_j}
    const int da = v.template Dn<a>();
    const int db = v.template Dn<b>();
    if constexpr (BF) {
      const R uar = v.template G0<pab>(ua), uai = v.template G0<pba>(ua);
      const R ubr = v.template G0<pab>(ub), ubi = v.template G0<pba>(ub);
      const R dar = v.template G0<pab>(da), dai = v.template G0<pba>(da);
      const R dbr = v.template G0<pab>(db), dbi = v.template G0<pba>(db);
      re += ubi - uai;
      im += uar - ubr;
      // terminator: sigma_{n+e_j} ~ (n_j+1)/(ngam+gamma_j) theta_j sigma_n, then i V_j^x of it
      const R ca = tc[a], cb = tc[b];
      re += ca * (-al_a * x - be_a * yi) + cb * (-al_b * x + be_b * yi);
      im += ca * (-al_a * yi + be_a * x) + cb * (-al_b * yi - be_b * x);
      const R n_a = v.template Nj<a>();
      const R n_b = v.template Nj<b>();
      re += n_a * (be_a * dar - al_a * dai) + n_b * (be_b * dbr + al_b * dbi);
      im += n_a * (al_a * dar + be_a * dai) + n_b * (be_b * dbi - al_b * dbr);
    } else {
      if (ua != -1) {
        R gr = v.template G<pba>(ua), gi = v.template G<pab>(ua);
        if constexpr (SC) {
          const R w = scaled_up(wsc, ws, a, v.template Nj<a>());
          gr *= w;
          gi *= w;
        }
        re -= gr;
        im += gi;
      }
      if (ub != -1) {
        R gr = v.template G<pba>(ub), gi = v.template G<pab>(ub);
        if constexpr (SC) {
          const R w = scaled_up(wsc, ws, b, v.template Nj<b>());
          gr *= w;
          gi *= w;
        }
        re += gr;
        im -= gi;
      }
      if (term) {
        const R ca = (v.template Nj<a>() + R(1)) / (ngam + cf[L::gam(N) + a]);
        const R cb = (v.template Nj<b>() + R(1)) / (ngam + cf[L::gam(N) + b]);
        re += ca * (-al_a * x - be_a * yi) + cb * (-al_b * x + be_b * yi);
        im += ca * (-al_a * yi + be_a * x) + cb * (-al_b * yi - be_b * x);
      }
      if (da != -1) {
        const R n_a = SC ? scaled_dn(wsc, ws, a, v.template Nj<a>()) : v.template Nj<a>();
        const R yr = v.template G<pab>(da);
        const R yy = v.template G<pba>(da);
        re += n_a * (be_a * yr - al_a * yy);
        im += n_a * (al_a * yr + be_a * yy);
      }
      if (db != -1) {
        const R n_b = SC ? scaled_dn(wsc, ws, b, v.template Nj<b>()) : v.template Nj<b>();
        const R yr = v.template G<pab>(db);
        const R yy = v.template G<pba>(db);
        re += n_b * (be_b * yr + al_b * yy);
        im += n_b * (be_b * yy - al_b * yr);
      }
    }
  } else {
    constexpr int a = u - NP;
    constexpr int paa = a * N + a;
    R jr[JS], sa[4];
    load_row<JS>(cf + L::J(N) + a * JS, jr);
    auto ja = [&](int k) -> R { return jr[k]; };
    load_row<4>(cf + L::site(N) + 4 * a, sa);
    const R x = v.template P<paa>();
    static_for<0, N>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (k != a) re += R(2) * ja(k) * Av<N, k, a, V, R>(v);
    });
    if constexpr (CPLX) {
      R ir[JS];
      load_row<JS>(cf + L::Ji(N) + a * JS, ir);
      auto ia = [&](int k) -> R { return ir[k]; };
      static_for<0, N>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if constexpr (k != a) re += R(2) * ia(k) * Sv<N, k, a>(v);
      });
    }
    re -= (ngam + R(2) * cf[L::gd(N) + a]) * x;
    const int da = v.template Dn<a>();
    if constexpr (BF) {
      re += R(2) * v.template Nj<a>() * sa[3] * v.template G0<paa>(da);
    } else {
      if (da != -1) {
        const R n_a = SC ? scaled_dn(wsc, ws, a, v.template Nj<a>()) : v.template Nj<a>();
        re += R(2) * n_a * sa[3] * v.template G<paa>(da);
      }
    }
  }
}

// Output steps are tracked with a counter (no 64-bit division in the loop):
// now is true at steps whose end is an output row, row is that row.
struct OutStep {
  bool now;
  int64_t row;
};

// Does unit u belong to this item's group?  GS > 0: the group is u % GS ==
// GI, known at compile time; GS == 0: the runtime mask umask decides.
template <int GS, int GI, int u>
__host__ __device__ constexpr bool in_group(uint64_t umask) {
  if constexpr (GS > 0) return (u % GS) == GI;
  else return (umask >> u) & 1ull;
}

// Shared-memory scratch of one warp for the staged outputs of the global
// engine: element p of lane l at stg[p * 32 + l]; per CTA the root's
// float-float stage outputs and its population row.
template <typename R>
struct Staging {
  R* stg;        // this lane's column
  FF* root_ff;   // [N*N]
  double* pops;  // [N]
};

// All units of one node in this item's group, one RK4 stage.  For the root
// node of the mixed path the Horner update w = y + h r runs in float-float
// on the root's own buffers, and the hi part is stored for the neighbours.
// At the last stage the owner of the root's diagonal unit a adds
// h Gamma_a x_aa to its running eta and loss sums (the extra rows of the
// augmented RK4 system, x being the stage input).  ROOT: the node may be the
// root (only the item holding node 0 needs that code).  With staging the
// results first go to shared memory and are copied out after the last unit,
// so no global store separates the loads of one unit from those of the next
// (STG; without it the results are stored where they are computed).
template <int N, typename R, bool MIXED, bool CPLX, int GS, int GI, bool ROOT, bool STG, bool BF, bool SC, class V>
__device__ __forceinline__ void node_units(const Inst& I, const R* __restrict__ cf, const double* __restrict__ cfd,
                                           const StageCoef<R>& P, const V& v, R ngam, int s, bool root,
                                           uint64_t umask, OutStep os, EtaAcc<R>& ea, const Staging<R>& sg) {
  using L = CoefLayout<R>;
  constexpr int NP = N * (N - 1) / 2;
  constexpr int U = NP + N;
  constexpr bool stage_out = STG;
  // terminator factors: precomputed for the branch-free form, else computed where used
  R tc[BF ? N : 1];
#pragma unroll
  for (int j = 0; j < (BF ? N : 1); ++j) tc[j] = R(0);
  const bool term = I.terminator && v.template Up<0>() == -1;
  if constexpr (BF) {
    if (term) {
      static_for<0, N>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        tc[j] = (v.template Nj<j>() + R(1)) / (ngam + cf[L::gam(N) + j]);
      });
    }
  }
  const bool out_row = ROOT && (s == 3) && root && I.out_pops && os.now;
  auto put = [&](auto pc, R w) {
    constexpr int p = decltype(pc)::value;
    if constexpr (stage_out) sg.stg[p * 32] = w;
    else v.template St<p>(w);
  };

  static_for<0, U>([&](auto uc) {
    constexpr int u = decltype(uc)::value;
    if constexpr (GS > 0) {
      if constexpr (!in_group<GS, GI, u>(0)) return;
    } else {
      if (!in_group<0, 0, u>(umask)) return;
    }
    R re, im;
    unit_rhs<N, u, R, CPLX, BF, SC>(v, cf, ngam, term, tc, re, im, static_cast<const R*>(I.wsc), I.wstride);
    if constexpr (u < NP) {
      constexpr int a = pair_a(N, u);
      constexpr int b = pair_b(N, u);
      constexpr int pr = a * N + b, pi = b * N + a;
      R wr, wi;
      if constexpr (ROOT && MIXED) {
        if (root) {
          const FF fr = ff_axpy(P.root_y[pr], P.h, P.hl, re);
          const FF fi = ff_axpy(P.root_y[pi], P.h, P.hl, im);
          if constexpr (stage_out) {
            sg.root_ff[pr] = fr;
            sg.root_ff[pi] = fi;
          } else {
            P.root_out[pr] = fr;
            P.root_out[pi] = fi;
          }
          wr = fr.h;
          wi = fi.h;
        } else {
          wr = v.template Y<pr>() + P.h * re;
          wi = v.template Y<pi>() + P.h * im;
        }
      } else {
        wr = v.template Y<pr>() + P.h * re;
        wi = v.template Y<pi>() + P.h * im;
      }
      put(std::integral_constant<int, pr>{}, wr);
      put(std::integral_constant<int, pi>{}, wi);
    } else {
      constexpr int a = u - NP;
      constexpr int pd = a * N + a;
      R w;
      [[maybe_unused]] double pop = 0.0;
      if constexpr (ROOT && MIXED) {
        if (root) {
          if (s == 3) ea.add(I, a, P.root_in[pd]);
          if (s == 2) ea.add_xi(I, a, P.root_in[pd]);
          const FF f = ff_axpy(P.root_y[pd], P.h, P.hl, re);
          if constexpr (stage_out) sg.root_ff[pd] = f;
          else P.root_out[pd] = f;
          w = f.h;
          if (out_row) pop = ff_to_double(f);
        } else {
          w = v.template Y<pd>() + P.h * re;
        }
      } else {
        if constexpr (ROOT && !MIXED) {
          if (root && s == 3) ea.add(I, cfd, N, a, (double)v.template P<pd>());
          if (root && s == 2) ea.add_xi(I, cfd, a, (double)v.template P<pd>());
        }
        w = v.template Y<pd>() + P.h * re;
        if constexpr (ROOT) {
          if (out_row) pop = (double)w;
        }
      }
      put(std::integral_constant<int, pd>{}, w);
      if constexpr (ROOT) {
        if (out_row) {
          if constexpr (stage_out) sg.pops[a] = pop;
          else I.out_pops[os.row * N + a] = pop;
        }
      }
    }
  });

  if constexpr (stage_out) {
    static_for<0, U>([&](auto uc) {
      constexpr int u = decltype(uc)::value;
      if constexpr (GS > 0) {
        if constexpr (!in_group<GS, GI, u>(0)) return;
      } else {
        if (!in_group<0, 0, u>(umask)) return;
      }
      if constexpr (u < NP) {
        constexpr int pr = pair_a(N, u) * N + pair_b(N, u), pi = pair_b(N, u) * N + pair_a(N, u);
        v.template St<pr>(sg.stg[pr * 32]);
        v.template St<pi>(sg.stg[pi * 32]);
        if constexpr (ROOT && MIXED) {
          if (root) {
            P.root_out[pr] = sg.root_ff[pr];
            P.root_out[pi] = sg.root_ff[pi];
          }
        }
      } else {
        constexpr int a = u - NP;
        constexpr int pd = a * N + a;
        v.template St<pd>(sg.stg[pd * 32]);
        if constexpr (ROOT) {
          if constexpr (MIXED) {
            if (root) P.root_out[pd] = sg.root_ff[pd];
          }
          if (out_row) I.out_pops[os.row * N + a] = sg.pops[a];
        }
      }
    });
  }
}

// ------------------------------------------------ run-time indexed units
//
// With load views (G > 2 unit groups) a warp runs one or a few units of its
// nodes per stage, and different warps run different units.  Compile-time
// unrolled unit bodies would then put the code of all N(N+1)/2 units in the
// instruction stream of one SM (tens of KB, more than the instruction cache
// holds); these versions run one compact body with the unit's (a, b) known at
// run time.  Same arithmetic as unit_rhs (branching form).
__device__ __forceinline__ void unit_pair_of(int N, int u, int& a, int& b) {
  a = 0;
  while (u >= N - 1 - a) {
    u -= N - 1 - a;
    ++a;
  }
  b = a + 1 + u;
}

template <int N, typename R, bool CPLX, bool SC, class V>
__device__ __forceinline__ void unit_rhs_rt(const V& v, const R* __restrict__ cf, R ngam, bool term, int a, int b,
                                            R& re, R& im, const R* __restrict__ wsc, int ws) {
  using L = CoefLayout<R>;
  constexpr int JS = L::JS(N);
  // packed element (k, l): Re sigma_kl for k <= l, Im sigma_lk for k > l
  auto S = [&](int k, int l) -> R { return k <= l ? v.Pr(k * N + l) : v.Pr(l * N + k); };
  auto A = [&](int k, int l) -> R { return k < l ? v.Pr(l * N + k) : (k > l ? -v.Pr(k * N + l) : R(0)); };
  re = R(0);
  im = R(0);
  const R* ja = cf + L::J(N) + a * JS;  // J(a, k)
  const R* jb = cf + L::J(N) + b * JS;  // J(b, k) = J(k, b)
  const R* sa = cf + L::site(N) + 4 * a;
  if (a != b) {
    const R* sb = cf + L::site(N) + 4 * b;
    const int pab = a * N + b, pba = b * N + a;
    const R x = v.Pr(pab), yi = v.Pr(pba);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const R jak = ja[k], jbk = jb[k];
      re += jak * A(k, b) - A(a, k) * jbk;
      im += S(a, k) * jbk - jak * S(k, b);
      if constexpr (CPLX) {
        const R iak = cf[L::Ji(N) + a * JS + k], ibk = cf[L::Ji(N) + b * JS + k];
        re += iak * S(k, b) + S(a, k) * ibk;
        im += iak * A(k, b) + A(a, k) * ibk;
      }
    }
    const R d = sa[0] - sb[0];
    const R c = ngam + sa[1] + sb[1];
    re += d * yi - c * x;
    im -= d * x + c * yi;
    const R al_a = sa[2], be_a = sa[3], al_b = sb[2], be_b = sb[3];
    const int ua = v.Upr(a), ub = v.Upr(b);
    if (ua != -1) {
      R gr = v.Gr(pba, ua), gi = v.Gr(pab, ua);
      if constexpr (SC) {
        const R w = scaled_up(wsc, ws, a, v.Njr(a));
        gr *= w;
        gi *= w;
      }
      re -= gr;
      im += gi;
    }
    if (ub != -1) {
      R gr = v.Gr(pba, ub), gi = v.Gr(pab, ub);
      if constexpr (SC) {
        const R w = scaled_up(wsc, ws, b, v.Njr(b));
        gr *= w;
        gi *= w;
      }
      re += gr;
      im -= gi;
    }
    if (term) {
      const R ca = (v.Njr(a) + R(1)) / (ngam + cf[L::gam(N) + a]);
      const R cb = (v.Njr(b) + R(1)) / (ngam + cf[L::gam(N) + b]);
      re += ca * (-al_a * x - be_a * yi) + cb * (-al_b * x + be_b * yi);
      im += ca * (-al_a * yi + be_a * x) + cb * (-al_b * yi - be_b * x);
    }
    const int da = v.Dnr(a), db = v.Dnr(b);
    if (da != -1) {
      const R n_a = SC ? scaled_dn(wsc, ws, a, v.Njr(a)) : v.Njr(a);
      const R yr = v.Gr(pab, da), yy = v.Gr(pba, da);
      re += n_a * (be_a * yr - al_a * yy);
      im += n_a * (al_a * yr + be_a * yy);
    }
    if (db != -1) {
      const R n_b = SC ? scaled_dn(wsc, ws, b, v.Njr(b)) : v.Njr(b);
      const R yr = v.Gr(pab, db), yy = v.Gr(pba, db);
      re += n_b * (be_b * yr + al_b * yy);
      im += n_b * (be_b * yy - al_b * yr);
    }
  } else {
    const int paa = a * N + a;
    const R x = v.Pr(paa);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      re += R(2) * ja[k] * A(k, a);
      if constexpr (CPLX) re += R(2) * cf[L::Ji(N) + a * JS + k] * S(k, a);
    }
    re -= (ngam + R(2) * cf[L::gd(N) + a]) * x;
    const int da = v.Dnr(a);
    if (da != -1) re += R(2) * (SC ? scaled_dn(wsc, ws, a, v.Njr(a)) : v.Njr(a)) * sa[3] * v.Gr(paa, da);
  }
}

// node_units for load views: the units in umask, one compact body.
template <int N, typename R, bool MIXED, bool CPLX, bool SC, class V>
__device__ __forceinline__ void node_units_rt(const Inst& I, const R* __restrict__ cf,
                                              const double* __restrict__ cfd, const StageCoef<R>& P, const V& v,
                                              R ngam, int s, bool root, uint64_t umask, OutStep os,
                                              EtaAcc<R>& ea) {
  constexpr int NP = N * (N - 1) / 2;
  const bool term = I.terminator && v.Upr(0) == -1;
  const bool out_row = (s == 3) && root && I.out_pops && os.now;
#pragma unroll 1
  for (uint64_t m = umask; m; m &= m - 1) {
    const int u = __ffsll((long long)m) - 1;
    int a, b;
    if (u < NP) unit_pair_of(N, u, a, b);
    else a = b = u - NP;
    R re, im;
    unit_rhs_rt<N, R, CPLX, SC>(v, cf, ngam, term, a, b, re, im, static_cast<const R*>(I.wsc), I.wstride);
    const int pr = a * N + b, pi = b * N + a;
    if (MIXED && root) {
      if constexpr (MIXED) {
        if (a == b && s == 3) ea.add(I, a, P.root_in[pr]);
        if (a == b && s == 2) ea.add_xi(I, a, P.root_in[pr]);
        const FF wr = ff_axpy(P.root_y[pr], P.h, P.hl, re);
        P.root_out[pr] = wr;
        v.Str(pr, wr.h);
        if (a != b) {
          const FF wi = ff_axpy(P.root_y[pi], P.h, P.hl, im);
          P.root_out[pi] = wi;
          v.Str(pi, wi.h);
        } else if (out_row) {
          I.out_pops[os.row * N + a] = ff_to_double(wr);
        }
      }
    } else {
      if constexpr (!MIXED) {
        if (root && a == b && s == 3) ea.add(I, cfd, N, a, (double)v.Pr(pr));
        if (root && a == b && s == 2) ea.add_xi(I, cfd, a, (double)v.Pr(pr));
      }
      const R w = v.Yr(pr) + P.h * re;
      v.Str(pr, w);
      if (a != b) v.Str(pi, v.Yr(pi) + P.h * im);
      else if (out_row) I.out_pops[os.row * N + a] = (double)w;
    }
  }
}

// ------------------------------------- one unit per warp, links in registers
//
// When every warp owns at most one item and every unit group holds one unit
// (G >= N(N+1)/2: the single-instance grid launch), the node, the unit and
// its links are the same in every stage of the call.  They are read once
// into registers, so a stage issues only the loads of stage values, all of
// them independent: one trip to L2 instead of two (links, then neighbours).
template <typename R>
struct CachedUnit {
  bool valid = false, term = false, root = false;
  int n = 0, a = 0, b = 0;
  int ua = -1, ub = -1, da = -1, db = -1;
  R na = R(0), nb = R(0), ng = R(0);
};

template <int N, typename R>
struct CachedView {
  const R* __restrict__ win;
  const R* __restrict__ base;
  R* __restrict__ wout;
  const R* __restrict__ y;
  int Mp;
  const CachedUnit<R>& c;
  __device__ __forceinline__ CachedView(const GlobalArrays<R>& g, const CachedUnit<R>& cu)
      : win(g.win + cu.n), base(g.win), wout(g.wout + cu.n), y(g.y + cu.n), Mp(g.Mp), c(cu) {}
  __device__ __forceinline__ R Pr(int p) const { return win[p * Mp]; }
  // links are asked for the unit's own sites only
  __device__ __forceinline__ int Upr(int j) const { return j == c.a ? c.ua : c.ub; }
  __device__ __forceinline__ int Dnr(int j) const { return j == c.a ? c.da : c.db; }
  __device__ __forceinline__ R Njr(int j) const { return j == c.a ? c.na : c.nb; }
  __device__ __forceinline__ R Gr(int p, int h) const { return base[p * Mp + h]; }
  __device__ __forceinline__ R Yr(int p) const { return y[p * Mp]; }
  __device__ __forceinline__ void Str(int p, R v) const { wout[p * Mp] = v; }
};

template <int N, typename R>
__device__ __forceinline__ CachedUnit<R> cache_unit(const Inst& I, int warp, int G, int lane) {
  constexpr int NP = N * (N - 1) / 2;
  constexpr int U = NP + N;
  CachedUnit<R> c;
  const int nblk = (I.M + 31) >> 5;
  if (warp >= nblk * G) return c;
  const int nb = warp / G, g = warp - nb * G;
  const int n = (nb << 5) + lane;
  if (n >= I.M || g >= U) return c;
  c.valid = true;
  c.n = n;
  if (g < NP) unit_pair_of(N, g, c.a, c.b);
  else c.a = c.b = g - NP;
  const int Mp = I.Mpad;
  c.ua = I.up[c.a * Mp + n];
  c.ub = I.up[c.b * Mp + n];
  const int ra = I.dn[c.a * Mp + n], rb = I.dn[c.b * Mp + n];
  c.da = ra < 0 ? -1 : (ra & 0xFFFFFF);
  c.db = rb < 0 ? -1 : (rb & 0xFFFFFF);
  c.na = ra < 0 ? R(0) : R(ra >> 24);
  c.nb = rb < 0 ? R(0) : R(rb >> 24);
  c.ng = static_cast<const R*>(I.ngam)[n];
  c.term = I.terminator && I.up[n] < 0;
  c.root = n == 0;
  return c;
}

// The one unit of a cached item, one RK4 stage (the per-unit part of node_units_rt).
template <int N, typename R, bool MIXED, bool CPLX, bool SC>
__device__ __forceinline__ void cached_unit_stage(const Inst& I, const R* __restrict__ cf,
                                                  const double* __restrict__ cfd, const StageCoef<R>& P,
                                                  const CachedView<N, R>& v, const CachedUnit<R>& c, int s,
                                                  OutStep os, EtaAcc<R>& ea) {
  const int a = c.a, b = c.b;
  const bool out_row = (s == 3) && c.root && I.out_pops && os.now;
  const int pr = a * N + b, pi = b * N + a;
  // every load of the stage before the arithmetic: y values, and for the root
  // its float-float y and stage input
  const R ypr = v.Yr(pr), ypi = a != b ? v.Yr(pi) : R(0);
  FF ry_r{0.f, 0.f}, ry_i{0.f, 0.f}, rin{0.f, 0.f};
  if constexpr (MIXED) {
    if (c.root) {
      ry_r = P.root_y[pr];
      if (a != b) ry_i = P.root_y[pi];
      else rin = P.root_in[pr];
    }
  }
  R re, im;
  unit_rhs_rt<N, R, CPLX, SC>(v, cf, c.ng, c.term, a, b, re, im, static_cast<const R*>(I.wsc), I.wstride);
  if (MIXED && c.root) {
    if constexpr (MIXED) {
      if (a == b && s == 3) ea.add(I, a, rin);
      if (a == b && s == 2) ea.add_xi(I, a, rin);
      const FF wr = ff_axpy(ry_r, P.h, P.hl, re);
      P.root_out[pr] = wr;
      v.Str(pr, wr.h);
      if (a != b) {
        const FF wi = ff_axpy(ry_i, P.h, P.hl, im);
        P.root_out[pi] = wi;
        v.Str(pi, wi.h);
      } else if (out_row) {
        I.out_pops[os.row * N + a] = ff_to_double(wr);
      }
    }
  } else {
    if constexpr (!MIXED) {
      if (c.root && a == b && s == 3) ea.add(I, cfd, N, a, (double)v.Pr(pr));
      if (c.root && a == b && s == 2) ea.add_xi(I, cfd, a, (double)v.Pr(pr));
    }
    const R w = ypr + P.h * re;
    v.Str(pr, w);
    if (a != b) v.Str(pi, ypi + P.h * im);
    else if (out_row) I.out_pops[os.row * N + a] = (double)w;
  }
}

// Row 0 of the outputs (the state at the start of the call).
template <int N, typename R, bool MIXED>
__device__ __forceinline__ void write_row0(const Inst& I) {
  if (I.out_pops)
    for (int a = 0; a < N; ++a)
      I.out_pops[a] = MIXED ? ff_to_double(static_cast<const FF*>(I.y0)[a * N + a])
                            : (double)static_cast<const R*>(I.y)[(a * N + a) * I.Mpad];
  if (I.out_el) {
    I.out_el[0] = I.acc[0];
    I.out_el[1] = I.acc[1];
  }
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Marks an instance finished for a host that polls its flag (host-mapped
// memory): every output write of the team happened before the team barrier
// that precedes this call; the system-scope fence orders them before the flag.
__device__ __forceinline__ void signal_done(const Inst& I) {
  if (!I.done) return;
  __threadfence_system();
  *reinterpret_cast<volatile int*>(I.done) = 1;
}

template <typename R>
__device__ __forceinline__ void load_instance(const EngineArgs& A, int li, Inst& s_inst, unsigned char* s_coef) {
  __syncthreads();
  if (threadIdx.x == 0) s_inst = A.insts[A.team_list[li]];
  __syncthreads();
  const int nb = CoefLayout<R>::bytes(s_inst.N);
  const unsigned char* src = static_cast<const unsigned char*>(s_inst.coef);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s_coef[i] = src[i];
  __syncthreads();
}

// Horner RK4: 0: wa = y + h/4 L y; 1: wb = y + h/3 L wa; 2: wa = y + h/2 L wb; 3: y = y + h L wa.
// Buffer selectors: 0 = y, 1 = wa, 2 = wb.
__device__ __forceinline__ void stage_buffers(int s, int& in_sel, int& out_sel) {
  in_sel = (s == 0) ? 0 : (s == 2 ? 2 : 1);
  out_sel = (s == 1) ? 2 : (s == 3 ? 0 : 1);
}

template <typename R>
__device__ __forceinline__ StageCoef<R> stage_coef(const Inst& I, int s, int in_sel, int out_sel) {
  StageCoef<R> P;
  if constexpr (sizeof(R) == 4) {
    P.h = I.hh[s];
    P.hl = I.hl[s];
  } else {
    P.h = I.hd[s];
    P.hl = 0.f;
  }
  FF* roots[3] = {static_cast<FF*>(I.y0), static_cast<FF*>(I.w0a), static_cast<FF*>(I.w0b)};
  P.root_in = roots[in_sel];
  P.root_out = roots[out_sel];
  P.root_y = roots[0];
  return P;
}

// The owner threads of the root's diagonal units publish their running sums
// (after the last stage of output steps and of the final step); one thread
// writes the eta row one stage later, once the team barrier has ordered them.
struct EtaRows {
  int64_t pending = -1;
  double acc0 = 0.0, acc1 = 0.0;
};

// The stop rule: true when the site population of the root after the step
// just finished is below I.stop_trace.  Every CTA of the team evaluates it
// from the same memory after the stage barrier, so all take the same branch.
template <typename R, bool MIXED>
__device__ __forceinline__ bool stop_now(const Inst& I, int N, int* s_flag) {
  if (threadIdx.x == 0) {
    double tr = 0.0;
    if constexpr (MIXED) {
      FF sum{0.f, 0.f};
      const float* y0 = static_cast<const float*>(I.y0);
      for (int a = 0; a < N; ++a) sum = ff_add(sum, FF{__ldcg(y0 + 2 * (a * N + a)), __ldcg(y0 + 2 * (a * N + a) + 1)});
      tr = ff_to_double(sum);
    } else {
      const R* y = static_cast<const R*>(I.y);
      for (int a = 0; a < N; ++a) tr += (double)__ldcg(y + (size_t)(a * N + a) * I.Mpad);
    }
    *s_flag = tr < I.stop_trace;
  }
  __syncthreads();
  const bool r = *s_flag != 0;
  __syncthreads();
  return r;
}

// End of an instance, lead thread: the last eta row, NaN rows after a stop,
// and the totals (eta, loss, xi, elapsed time, steps done) for the next call.
template <typename R>
__device__ __forceinline__ void finish_instance(const Inst& I, int nslots, const EtaRows& rows, int64_t done,
                                                int64_t orow, int N, int* status) {
  if (rows.pending >= 0) eta_write_row<R>(I, nslots, rows.acc0, rows.acc1, rows.pending, status);
  // the site populations at the end of the call, whether or not rows were asked for
  for (int a = 0; a < N; ++a) {
    if constexpr (sizeof(R) == 4) {
      const float* y0 = static_cast<const float*>(I.y0);
      flag_nonfinite(status, (double)__ldcg(y0 + 2 * (a * N + a)) + (double)__ldcg(y0 + 2 * (a * N + a) + 1));
    } else {
      flag_nonfinite(status, (double)__ldcg(static_cast<const R*>(I.y) + (size_t)(a * N + a) * I.Mpad));
    }
  }
  if (done < I.nsteps) {
    const int64_t nout = I.nsteps / I.out_every + 1;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t r = orow; r < nout; ++r) {
      if (I.out_pops)
        for (int a = 0; a < N; ++a) I.out_pops[r * N + a] = nan;
      if (I.out_el) {
        I.out_el[2 * r] = nan;
        I.out_el[2 * r + 1] = nan;
      }
    }
  }
  if (done > 0) {
    double e, l, xs;
    eta_total<R>(I, nslots, rows.acc0, rows.acc1, e, l, &xs);
    flag_nonfinite(status, e);
    flag_nonfinite(status, l);
    I.acc[2] += (double)done * I.dt * rows.acc0 + xs;
    I.acc[3] += (double)done * I.dt;
    I.acc[0] = e;
    I.acc[1] = l;
  }
  I.acc[4] = (double)done;
}

// ------------------------------------------------------ global-memory engine

// Dynamic shared memory of the global engine: with FP32 register views (unit
// groups G <= 2, many units per item) the output staging of every warp,
// [N*N][32] floats each; none otherwise.
__host__ __device__ constexpr int engine_dyn_bytes(int N, int block, int rsize, bool reg) {
  return (reg && rsize == 4) ? (block / 32) * N * N * 32 * rsize : 0;
}

// SC: scaled hierarchy (link weights from Inst::wsc); not with the FP32
// register view, whose branch-free units take no weights.
template <int N, typename R, bool MIXED, bool CPLX, bool REG, bool SC = false>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 256 : 512, (sizeof(R) == 8 && !REG) ? 2 : 1)
    heom_engine_kernel(EngineArgs A) {
  static_assert(!(SC && REG && sizeof(R) == 4), "no scaled FP32 register view");
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ __align__(16) unsigned char s_coef[CoefLayout<R>::bytes(kMaxSmallN) + 64];
  __shared__ FF s_rootff[kMaxSmallN * kMaxSmallN];
  __shared__ double s_pops[kMaxSmallN];
  __shared__ Inst s_inst;
  __shared__ int s_stop;
  __shared__ uint64_t s_umask[32];
  constexpr int U = N * (N - 1) / 2 + N;
  constexpr int NP = N * (N - 1) / 2;

  int team, rank, team_size;
  if (A.mode == 0) {
    team = blockIdx.x / A.team_ctas;
    rank = blockIdx.x - team * A.team_ctas;
    team_size = A.team_ctas;
  } else {
    team = 0;
    rank = blockIdx.x;
    team_size = gridDim.x;
  }
  const int wpc = blockDim.x >> 5;
  // Team-wide warp index.  FP64: interleaved over the CTAs, so that when the
  // items of a stage are fewer than the team's warps they spread over every
  // SM's FP64 units (FMO-like depth 6: 11.1 -> 8.5 us per stage).  FP32:
  // consecutive per CTA, so the unit groups of a node block share an SM and
  // its L1 (interleaving measured 4.3 -> 5.6 us there).
  const int warp = sizeof(R) == 8 ? (threadIdx.x >> 5) * team_size + rank : rank * wpc + (threadIdx.x >> 5);
  const int W = team_size * wpc;
  const int lane = threadIdx.x & 31;
  const int G = A.G;
  if (threadIdx.x < 32) {
    uint64_t m = 0;
    for (int u = 0; u < U; ++u)
      if (u % G == (int)threadIdx.x) m |= 1ull << u;
    s_umask[threadIdx.x] = m;
  }
  // this thread's parts slot: the smallest group g whose root item it runs
  // and that owns a diagonal unit (-1: none)
  int slot = -1;
  if (lane == 0)
    for (int g = 0; g < G; ++g)
      if (g % W == warp) {
        bool diag = false;
        for (int a = 0; a < N; ++a) diag |= ((NP + a) % G) == g;
        if (diag) {
          slot = g;
          break;
        }
      }
  const bool lead = (warp == 0 && lane == 0);
  const int nslots = G < 32 ? G : 32;
  unsigned epoch = 0;
  const Staging<R> sg{reinterpret_cast<R*>(dsm) + (threadIdx.x >> 5) * (N * N * 32) + lane, s_rootff, s_pops};

  for (int li = A.team_first[team]; li < A.team_first[team + 1]; ++li) {
    load_instance<R>(A, li, s_inst, s_coef);
    const Inst& I = s_inst;
    const R* cf = reinterpret_cast<const R*>(s_coef);
    const double* cfd = reinterpret_cast<const double*>(s_coef + CoefLayout<R>::dbl_offset(N));
    const R* ngam = static_cast<const R*>(I.ngam);
    const int nblk = (I.M + 31) >> 5;
    const int items = nblk * G;
    EtaAcc<R> ea;
    EtaRows rows;
    rows.acc0 = I.acc[0];
    rows.acc1 = I.acc[1];
    if (lead) {
      write_row0<N, R, MIXED>(I);
      for (int k = 0; k < nslots; ++k) ea.store(I, k);  // zero every running-sum slot of this instance
    }
    if (!team_barrier(A, epoch)) return;

    R* arr[3] = {static_cast<R*>(I.y), static_cast<R*>(I.wa), static_cast<R*>(I.wb)};
    // FP32 load views with one unit per warp: the unit and its links stay in registers
    constexpr bool CACHE_OK = !REG && sizeof(R) == 4;
    const bool cached = CACHE_OK && G >= N * (N + 1) / 2 && items <= W;
    CachedUnit<R> cu;
    if (CACHE_OK && cached) cu = cache_unit<N, R>(I, warp, G, lane);
    int64_t next_out = I.out_every, orow = 1, done = I.nsteps;
    for (int64_t t = 0; t < I.nsteps; ++t) {
      const OutStep os{t + 1 == next_out, orow};
      if (os.now) {
        next_out += I.out_every;
        ++orow;
      }
#pragma unroll 1
      for (int s = 0; s < 4; ++s) {
        if (s == 0 && rows.pending >= 0) {
          if (lead) eta_write_row<R>(I, nslots, rows.acc0, rows.acc1, rows.pending, A.status);
          rows.pending = -1;
        }
        int in_sel, out_sel;
        stage_buffers(s, in_sel, out_sel);
        const StageCoef<R> P = stage_coef<R>(I, s, in_sel, out_sel);
        GlobalArrays<R> ga{arr[in_sel], arr[out_sel], arr[0], I.up, I.dn, I.Mpad};
        if constexpr (CACHE_OK) {
          if (cached) {
            if (cu.valid) cached_unit_stage<N, R, MIXED, CPLX, SC>(I, cf, cfd, P, CachedView<N, R>(ga, cu), cu, s, os, ea);
          }
        }
        for (int it = warp; it < items && !(CACHE_OK && cached); it += W) {
          const int nb = it / G;
          const int g = it - nb * G;
          const int n = (nb << 5) + lane;
          if (n >= I.M) continue;
          const GlobalView<N, R, REG> v(ga, n);
          const R ng = ngam[n];
          // FP32 register views: staged, branch-free units (see unit_rhs), and the
          // root's code only in the items that hold it.  Other views run one
          // instantiation for every item (measured faster: a second copy of the
          // unit code costs more in instruction fetch than the root branches).
          constexpr bool BF = REG && sizeof(R) == 4;
          if constexpr (!REG && sizeof(R) == 4) {
            node_units_rt<N, R, MIXED, CPLX, SC>(I, cf, cfd, P, v, ng, s, n == 0, s_umask[g], os, ea);
          } else if constexpr (!BF) {
            node_units<N, R, MIXED, CPLX, 0, 0, true, false, false, SC>(I, cf, cfd, P, v, ng, s, n == 0,
                                                                        s_umask[g], os, ea, sg);
          } else if (nb == 0) {
            node_units<N, R, MIXED, CPLX, 0, 0, true, true, true, false>(I, cf, cfd, P, v, ng, s, n == 0,
                                                                         s_umask[g], os, ea, sg);
          } else if (G == 1) {
            node_units<N, R, MIXED, CPLX, 1, 0, false, true, true, false>(I, cf, cfd, P, v, ng, s, false, 0, os, ea,
                                                                          sg);
          } else if (g == 0) {  // G == 2
            node_units<N, R, MIXED, CPLX, 2, 0, false, true, true, false>(I, cf, cfd, P, v, ng, s, false, 0, os, ea,
                                                                          sg);
          } else {
            node_units<N, R, MIXED, CPLX, 2, 1, false, true, true, false>(I, cf, cfd, P, v, ng, s, false, 0, os, ea,
                                                                          sg);
          }
        }
        if (s == 2 && slot >= 0) ea.step_xi(I);
        if (s == 3 && slot >= 0 && (os.now || t + 1 == I.nsteps)) ea.store(I, slot);
        if (!team_barrier(A, epoch)) return;
      }
      if (os.now) rows.pending = os.row;
      if (I.stop_trace > 0.0 && t + 1 < I.nsteps && stop_now<R, MIXED>(I, N, &s_stop)) {
        if (slot >= 0) ea.store(I, slot);
        done = t + 1;
        if (!team_barrier(A, epoch)) return;
        break;
      }
    }
    if (lead) finish_instance<R>(I, nslots, rows, done, orow, N, A.status);
    if (!team_barrier(A, epoch)) return;
    if (lead) signal_done(I);
  }
}

// ------------------------------------------- distributed-shared-memory engine
//
// Mixed precision only.  One thread-block cluster of C CTAs holds a whole
// hierarchy in its distributed shared memory: CTA r owns nodes
// [r*B, r*B + B) and keeps y, wa and wb of those nodes, their link handles,
// n_j and damping in its own shared memory.  Own elements are read from local
// shared memory, neighbours with ld.shared::cluster; the stage barrier is the
// hardware cluster barrier, whose release/acquire orders the shared-memory
// writes of one stage before the reads of the next.  y is copied in from and
// back to device memory once per call.

// Dynamic shared memory of one CTA for a slice of B nodes.
__host__ __device__ constexpr int smem_dyn_bytes(int N, int B) {
  return (3 * N * N + 2 * N + 1) * 4 * B + N * B;
}

template <int N, bool CPLX, bool REG>
__global__ void __launch_bounds__(512) heom_smem_kernel(EngineArgs A, int B) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ __align__(16) unsigned char s_coef[CoefLayout<float>::bytes(kMaxSmallN) + 64];
  __shared__ Inst s_inst;
  __shared__ int s_stop;
  __shared__ uint64_t s_umask[32];
  constexpr int U = N * (N - 1) / 2 + N;
  constexpr int NP = N * (N - 1) / 2;
  constexpr int NN = N * N;

  unsigned rank, C;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(C));
  const int team = blockIdx.x / C;
  const int wpc = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int G = A.G;
  if (threadIdx.x < 32) {
    uint64_t m = 0;
    for (int u = 0; u < U; ++u)
      if (u % G == (int)threadIdx.x) m |= 1ull << u;
    s_umask[threadIdx.x] = m;
  }
  int slot = -1;
  if (rank == 0 && lane == 0)
    for (int g = 0; g < G; ++g)
      if (g % wpc == warp) {
        bool diag = false;
        for (int a = 0; a < N; ++a) diag |= ((NP + a) % G) == g;
        if (diag) {
          slot = g;
          break;
        }
      }
  const bool lead = (rank == 0 && threadIdx.x == 0);
  const int nslots = G < 32 ? G : 32;
  float* sy = reinterpret_cast<float*>(dsm);
  float* swa = sy + NN * B;
  float* swb = swa + NN * B;
  unsigned* sup = reinterpret_cast<unsigned*>(swb + NN * B);
  unsigned* sdn = sup + N * B;
  float* sng = reinterpret_cast<float*>(sdn + N * B);
  unsigned char* snj = reinterpret_cast<unsigned char*>(sng + B);
  float* arr[3] = {sy, swa, swb};
  const unsigned base = smem_u32(dsm);

  for (int li = A.team_first[team]; li < A.team_first[team + 1]; ++li) {
    load_instance<float>(A, li, s_inst, s_coef);
    const Inst& I = s_inst;
    const float* cf = reinterpret_cast<const float*>(s_coef);
    const double* cfd = reinterpret_cast<const double*>(s_coef + CoefLayout<float>::dbl_offset(N));
    const int Mp = I.Mpad;
    const int n0 = (int)rank * B;
    const int nloc = max(0, min(B, I.M - n0));
    // fill this CTA's slice
    const float* gy = static_cast<const float*>(I.y);
    for (int idx = threadIdx.x; idx < NN * B; idx += blockDim.x) {
      const int p = idx / B, l = idx - (idx / B) * B;
      sy[idx] = l < nloc ? gy[p * Mp + n0 + l] : 0.f;
    }
    for (int idx = threadIdx.x; idx < N * B; idx += blockDim.x) {
      const int j = idx / B, l = idx - (idx / B) * B;
      unsigned hu = 0xFFFFFFFFu, hd = 0xFFFFFFFFu;
      unsigned char nj = 0;
      if (l < nloc) {
        const int m = I.up[j * Mp + n0 + l];
        if (m >= 0) hu = map_to_rank(base + (unsigned)(m % B) * 4u, (unsigned)(m / B));
        const int d = I.dn[j * Mp + n0 + l];
        if (d >= 0) {
          const int md = d & 0xFFFFFF;
          hd = map_to_rank(base + (unsigned)(md % B) * 4u, (unsigned)(md / B));
          nj = (unsigned char)(d >> 24);
        }
      }
      sup[idx] = hu;
      sdn[idx] = hd;
      snj[idx] = nj;
    }
    for (int l = threadIdx.x; l < B; l += blockDim.x)
      sng[l] = l < nloc ? static_cast<const float*>(I.ngam)[n0 + l] : 0.f;
    EtaAcc<float> ea;
    EtaRows rows;
    rows.acc0 = I.acc[0];
    rows.acc1 = I.acc[1];
    if (lead) {
      write_row0<N, float, true>(I);
      for (int k = 0; k < nslots; ++k) ea.store(I, k);  // zero every running-sum slot of this instance
    }
    cluster_sync_all();

    const int nblk = (nloc + 31) >> 5;
    const int items = nblk * G;
    int64_t next_out = I.out_every, orow = 1, done = I.nsteps;
    for (int64_t t = 0; t < I.nsteps; ++t) {
      const OutStep os{t + 1 == next_out, orow};
      if (os.now) {
        next_out += I.out_every;
        ++orow;
      }
#pragma unroll 1
      for (int s = 0; s < 4; ++s) {
        if (s == 0 && rows.pending >= 0) {
          if (lead) eta_write_row<float>(I, nslots, rows.acc0, rows.acc1, rows.pending, A.status);
          rows.pending = -1;
        }
        int in_sel, out_sel;
        stage_buffers(s, in_sel, out_sel);
        const StageCoef<float> P = stage_coef<float>(I, s, in_sel, out_sel);
        SmemArrays sa{arr[in_sel], arr[out_sel], sy, sup, sdn, snj, sng,
                      (unsigned)(in_sel * NN * B * 4), B};
        for (int it = warp; it < items; it += wpc) {
          const int nb = it / G;
          const int g = it - nb * G;
          const int l = (nb << 5) + lane;
          if (l >= nloc) continue;
          const SmemView<N, REG> v(sa, l);
          node_units<N, float, true, CPLX, 0, 0, true, false, false, false>(I, cf, cfd, P, v, sng[l], s, rank == 0 && l == 0,
                                                                     s_umask[g], os, ea,
                                                                     Staging<float>{nullptr, nullptr, nullptr});
        }
        if (s == 2 && slot >= 0) ea.step_xi(I);
        if (s == 3 && slot >= 0 && (os.now || t + 1 == I.nsteps)) ea.store(I, slot);
        cluster_sync_all();
      }
      if (os.now) rows.pending = os.row;
      if (I.stop_trace > 0.0 && t + 1 < I.nsteps && stop_now<float, true>(I, N, &s_stop)) {
        if (slot >= 0) ea.store(I, slot);
        done = t + 1;
        cluster_sync_all();
        break;
      }
    }
    if (lead) finish_instance<float>(I, nslots, rows, done, orow, N, A.status);
    // write the slice of y back
    float* gyw = static_cast<float*>(I.y);
    for (int idx = threadIdx.x; idx < NN * B; idx += blockDim.x) {
      const int p = idx / B, l = idx - (idx / B) * B;
      if (l < nloc) gyw[p * Mp + n0 + l] = sy[idx];
    }
    cluster_sync_all();  // no CTA reuses or leaves its slice while others may still read it
    if (lead) signal_done(I);
  }
}

}  // namespace heom
