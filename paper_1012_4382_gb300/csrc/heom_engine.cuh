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

// Per-instance device descriptor (host fills it; see heom_runtime.cu).
struct Inst {
  int32_t N, K, M, Mpad;
  int32_t complex_h, terminator, pad0, pad1;
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
  double* acc;         // [2] eta and loss integrals (read at the start of a call, written at its end)
  void* parts;         // [32] partial (eta, loss) sums per unit group: float-float x2 (mixed) or double x2
  double* out_pops;    // [nout][N] populations (may be null)
  double* out_el;      // [nout][2] eta, loss (may be null)
  int* done;           // set to 1 (system-wide release) when the instance is finished (may be null)
  int64_t nsteps;
  int64_t out_every;
  double dt;
  double hd[4];        // Horner steps h/4, h/3, h/2, h
  float hh[4], hl[4];  // the same as float-float pairs (hi, lo)
  float ec[4 * kMaxSites];  // per site a: h*Gamma_RC,a (hi, lo), h*Gamma_phot,a (hi, lo)
};

// Coefficient block (host writes it with the same layout):
//   R J[N*N]     real part of H off the diagonal (rad/fs), zero diagonal
//   R Ji[N*N]    imaginary part of H (antisymmetric)
//   R eps[N]     diagonal of H minus its mean
//   R ghalf[N]   (Gamma_RC + Gamma_phot) / 2   (1/fs)
//   R alpha[N]   2 lambda k_B T                (rad^2/fs^2)
//   R beta[N]    lambda gamma                  (rad^2/fs^2)
//   R gam[N]     gamma                         (rad/fs)
//   then, 8-byte aligned: double trap[N], double recomb[N] (1/fs)
template <typename R>
struct CoefLayout {
  __host__ __device__ static constexpr int J(int N) { return 0; }
  __host__ __device__ static constexpr int Ji(int N) { return N * N; }
  __host__ __device__ static constexpr int eps(int N) { return 2 * N * N; }
  __host__ __device__ static constexpr int ghalf(int N) { return 2 * N * N + N; }
  __host__ __device__ static constexpr int alpha(int N) { return 2 * N * N + 2 * N; }
  __host__ __device__ static constexpr int beta(int N) { return 2 * N * N + 3 * N; }
  __host__ __device__ static constexpr int gam(int N) { return 2 * N * N + 4 * N; }
  __host__ __device__ static constexpr int reals(int N) { return 2 * N * N + 5 * N; }
  // byte offset of the double arrays
  __host__ __device__ static constexpr int dbl_offset(int N) {
    return ((reals(N) * (int)sizeof(R) + 7) / 8) * 8;
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
    int ok = 1;
    const uint64_t t0 = global_timer_ns();
    unsigned spins = 0;
    while (ld_acquire_gpu(A.gsync) < target) {
      if ((++spins & 1023u) == 0) {
        if (ld_volatile(A.status) & kStatusTimeout) { ok = 0; break; }
        if (global_timer_ns() - t0 > 2000000000ull) {  // 2 s without the team arriving
          atomicOr(A.status, kStatusTimeout);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
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
  template <int p>
  __device__ __forceinline__ R Y() const { return y[p * Mp]; }
  template <int p>
  __device__ __forceinline__ void St(R v) const { wout[p * Mp] = v; }
};

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
  __device__ __forceinline__ float Y() const { return y[p * B]; }
  template <int p>
  __device__ __forceinline__ void St(float v) const { wout[p * B] = v; }
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
template <>
struct EtaAcc<float> {
  FF e{0.f, 0.f}, l{0.f, 0.f};
  // contribution of diagonal a of the root's stage-3 input x: h Gamma_a x
  __device__ __forceinline__ void add(const Inst& I, int a, FF x) {
    e = ff_add(e, ff_mul(I.ec[4 * a], I.ec[4 * a + 1], x));
    l = ff_add(l, ff_mul(I.ec[4 * a + 2], I.ec[4 * a + 3], x));
  }
  __device__ __forceinline__ void store(const Inst& I, int slot) const {
    float* p = static_cast<float*>(I.parts) + 4 * slot;
    p[0] = e.h;
    p[1] = e.l;
    p[2] = l.h;
    p[3] = l.l;
  }
};
template <>
struct EtaAcc<double> {
  double e = 0.0, l = 0.0;
  __device__ __forceinline__ void add(const Inst& I, const double* cfd, int N, int a, double x) {
    e += I.dt * cfd[a] * x;
    l += I.dt * cfd[N + a] * x;
  }
  __device__ __forceinline__ void store(const Inst& I, int slot) const {
    double* p = static_cast<double*>(I.parts) + 2 * slot;
    p[0] = e;
    p[1] = l;
  }
};

// eta and loss at the current step: the value at the start of the call plus
// every owner's running sum (read through L2: the owners wrote them before
// the last stage barrier).
template <typename R>
__device__ __forceinline__ void eta_total(const Inst& I, int nslots, double acc0, double acc1, double& e, double& l) {
  if constexpr (sizeof(R) == 4) {
    FF se{0.f, 0.f}, sl{0.f, 0.f};
    const float* p = static_cast<const float*>(I.parts);
    for (int k = 0; k < nslots; ++k) {
      se = ff_add(se, FF{__ldcg(p + 4 * k), __ldcg(p + 4 * k + 1)});
      sl = ff_add(sl, FF{__ldcg(p + 4 * k + 2), __ldcg(p + 4 * k + 3)});
    }
    e = acc0 + ff_to_double(se);
    l = acc1 + ff_to_double(sl);
  } else {
    double se = 0.0, sl = 0.0;
    const double* p = static_cast<const double*>(I.parts);
    for (int k = 0; k < nslots; ++k) {
      se += __ldcg(p + 2 * k);
      sl += __ldcg(p + 2 * k + 1);
    }
    e = acc0 + se;
    l = acc1 + sl;
  }
}

template <typename R>
__device__ __forceinline__ void eta_write_row(const Inst& I, int nslots, double acc0, double acc1, int64_t row) {
  if (!I.out_el) return;
  double e, l;
  eta_total<R>(I, nslots, acc0, acc1, e, l);
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

// Right-hand side of unit u (pair (a, b) or diagonal a) of one node.
// Returns the real part in re and, for pairs, the imaginary part in im.
template <int N, int u, typename R, bool CPLX, class V>
__device__ __forceinline__ void unit_rhs(const V& v, const R* __restrict__ cf, R ngam, bool term, R& re, R& im) {
  using L = CoefLayout<R>;
  constexpr int NP = N * (N - 1) / 2;
  re = R(0);
  im = R(0);
  if constexpr (u < NP) {
    constexpr int a = pair_a(N, u);
    constexpr int b = pair_b(N, u);
    constexpr int pab = a * N + b, pba = b * N + a;
    const R x = v.template P<pab>();   // Re sigma_ab
    const R yi = v.template P<pba>();  // Im sigma_ab
    // -i[J, sigma]: Re += [J, A]_ab, Im -= [J, S]_ab
    static_for<0, N>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (k != a) {
        const R jak = cf[L::J(N) + a * N + k];
        if constexpr (k != b) re += jak * Av<N, k, b, V, R>(v);
        im -= jak * Sv<N, k, b>(v);
      }
      if constexpr (k != b) {
        const R jkb = cf[L::J(N) + k * N + b];
        if constexpr (k != a) re -= Av<N, a, k, V, R>(v) * jkb;
        im += Sv<N, a, k>(v) * jkb;
      }
    });
    if constexpr (CPLX) {
      // -i[i Ji, sigma] = [Ji, S] + i [Ji, A]
      static_for<0, N>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if constexpr (k != a) {
          const R jak = cf[L::Ji(N) + a * N + k];
          re += jak * Sv<N, k, b>(v);
          if constexpr (k != b) im += jak * Av<N, k, b, V, R>(v);
        }
        if constexpr (k != b) {
          const R jkb = cf[L::Ji(N) + k * N + b];
          re -= Sv<N, a, k>(v) * jkb;
          if constexpr (k != a) im -= Av<N, a, k, V, R>(v) * jkb;
        }
      });
    }
    // -i (eps_a - eps_b) sigma_ab, anti-Hermitian part and damping
    const R d = cf[L::eps(N) + a] - cf[L::eps(N) + b];
    const R c = ngam + cf[L::ghalf(N) + a] + cf[L::ghalf(N) + b];
    re += d * yi - c * x;
    im -= d * x + c * yi;
    const R al_a = cf[L::alpha(N) + a], be_a = cf[L::beta(N) + a];
    const R al_b = cf[L::alpha(N) + b], be_b = cf[L::beta(N) + b];
    // up-couplings i V_j^x sigma_{n+e_j}: j = a gives +i, j = b gives -i
    const int ua = v.template Up<a>();
    const int ub = v.template Up<b>();
    if (ua != -1) {
      re -= v.template G<pba>(ua);
      im += v.template G<pab>(ua);
    }
    if (ub != -1) {
      re += v.template G<pba>(ub);
      im -= v.template G<pab>(ub);
    }
    if (term) {
      // sigma_{n+e_j} ~ (n_j+1)/(ngam+gamma_j) theta_j sigma_n, then i V_j^x of it
      const R ca = (v.template Nj<a>() + R(1)) / (ngam + cf[L::gam(N) + a]);
      const R cb = (v.template Nj<b>() + R(1)) / (ngam + cf[L::gam(N) + b]);
      re += ca * (-al_a * x - be_a * yi) + cb * (-al_b * x + be_b * yi);
      im += ca * (-al_a * yi + be_a * x) + cb * (-al_b * yi - be_b * x);
    }
    // down-couplings n_j theta_j sigma_{n-e_j}
    const int da = v.template Dn<a>();
    const int db = v.template Dn<b>();
    if (da != -1) {
      const R n_a = v.template Nj<a>();
      const R yr = v.template G<pab>(da);
      const R yy = v.template G<pba>(da);
      re += n_a * (be_a * yr - al_a * yy);
      im += n_a * (al_a * yr + be_a * yy);
    }
    if (db != -1) {
      const R n_b = v.template Nj<b>();
      const R yr = v.template G<pab>(db);
      const R yy = v.template G<pba>(db);
      re += n_b * (be_b * yr + al_b * yy);
      im += n_b * (be_b * yy - al_b * yr);
    }
  } else {
    constexpr int a = u - NP;
    constexpr int paa = a * N + a;
    const R x = v.template P<paa>();
    static_for<0, N>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (k != a) re += R(2) * cf[L::J(N) + a * N + k] * Av<N, k, a, V, R>(v);
    });
    if constexpr (CPLX) {
      static_for<0, N>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if constexpr (k != a) re += R(2) * cf[L::Ji(N) + a * N + k] * Sv<N, k, a>(v);
      });
    }
    re -= (ngam + R(2) * cf[L::ghalf(N) + a]) * x;
    const int da = v.template Dn<a>();
    if (da != -1) re += R(2) * v.template Nj<a>() * cf[L::beta(N) + a] * v.template G<paa>(da);
  }
}

// Output steps are tracked with a counter (no 64-bit division in the loop):
// now is true at steps whose end is an output row, row is that row.
struct OutStep {
  bool now;
  int64_t row;
};

// All units of one node that belong to the unit mask, one RK4 stage.  For
// the root node of the mixed path the Horner update w = y + h r runs in
// float-float on the root's own buffers, and the hi part is stored for the
// neighbours.  At the last stage the owner of the root's diagonal unit a adds
// h Gamma_a x_aa to its running eta and loss sums (the extra rows of the
// augmented RK4 system, x being the stage input).
template <int N, typename R, bool MIXED, bool CPLX, class V>
__device__ __forceinline__ void node_units(const Inst& I, const R* __restrict__ cf, const double* __restrict__ cfd,
                                           const StageCoef<R>& P, const V& v, R ngam, int s, bool root,
                                           uint64_t umask, OutStep os, EtaAcc<R>& ea) {
  constexpr int NP = N * (N - 1) / 2;
  constexpr int U = NP + N;
  const bool term = I.terminator && (v.template Up<0>() == -1);
  const bool out_row = (s == 3) && root && I.out_pops && os.now;

  static_for<0, U>([&](auto uc) {
    constexpr int u = decltype(uc)::value;
    if (!((umask >> u) & 1ull)) return;
    R re, im;
    unit_rhs<N, u, R, CPLX>(v, cf, ngam, term, re, im);
    if constexpr (u < NP) {
      constexpr int a = pair_a(N, u);
      constexpr int b = pair_b(N, u);
      constexpr int pr = a * N + b, pi = b * N + a;
      if (MIXED && root) {
        if constexpr (MIXED) {
          const FF wr = ff_axpy(P.root_y[pr], P.h, P.hl, re);
          const FF wi = ff_axpy(P.root_y[pi], P.h, P.hl, im);
          P.root_out[pr] = wr;
          P.root_out[pi] = wi;
          v.template St<pr>(wr.h);
          v.template St<pi>(wi.h);
        }
      } else {
        v.template St<pr>(v.template Y<pr>() + P.h * re);
        v.template St<pi>(v.template Y<pi>() + P.h * im);
      }
    } else {
      constexpr int a = u - NP;
      constexpr int pd = a * N + a;
      if (MIXED && root) {
        if constexpr (MIXED) {
          if (s == 3) ea.add(I, a, P.root_in[pd]);
          const FF w = ff_axpy(P.root_y[pd], P.h, P.hl, re);
          P.root_out[pd] = w;
          v.template St<pd>(w.h);
          if (out_row) I.out_pops[os.row * N + a] = ff_to_double(w);
        }
      } else {
        if constexpr (!MIXED) {
          if (root && s == 3) ea.add(I, cfd, N, a, (double)v.template P<pd>());
        }
        const R vv = v.template Y<pd>() + P.h * re;
        v.template St<pd>(vv);
        if (out_row) I.out_pops[os.row * N + a] = (double)vv;
      }
    }
  });
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

// ------------------------------------------------------ global-memory engine

template <int N, typename R, bool MIXED, bool CPLX, bool REG>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 256 : 512) heom_engine_kernel(EngineArgs A) {
  __shared__ __align__(16) unsigned char s_coef[CoefLayout<R>::bytes(kMaxSmallN) + 64];
  __shared__ Inst s_inst;
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
  const int warp = rank * wpc + (threadIdx.x >> 5);
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
    int64_t next_out = I.out_every, orow = 1;
    for (int64_t t = 0; t < I.nsteps; ++t) {
      const OutStep os{t + 1 == next_out, orow};
      if (os.now) {
        next_out += I.out_every;
        ++orow;
      }
#pragma unroll 1
      for (int s = 0; s < 4; ++s) {
        if (s == 0 && rows.pending >= 0) {
          if (lead) eta_write_row<R>(I, nslots, rows.acc0, rows.acc1, rows.pending);
          rows.pending = -1;
        }
        int in_sel, out_sel;
        stage_buffers(s, in_sel, out_sel);
        const StageCoef<R> P = stage_coef<R>(I, s, in_sel, out_sel);
        GlobalArrays<R> ga{arr[in_sel], arr[out_sel], arr[0], I.up, I.dn, I.Mpad};
        for (int it = warp; it < items; it += W) {
          const int nb = it / G;
          const int g = it - nb * G;
          const int n = (nb << 5) + lane;
          if (n >= I.M) continue;
          const GlobalView<N, R, REG> v(ga, n);
          node_units<N, R, MIXED, CPLX>(I, cf, cfd, P, v, ngam[n], s, n == 0, s_umask[g], os, ea);
        }
        if (s == 3 && slot >= 0 && (os.now || t + 1 == I.nsteps)) ea.store(I, slot);
        if (!team_barrier(A, epoch)) return;
      }
      if (os.now) rows.pending = os.row;
    }
    if (lead) {
      if (rows.pending >= 0) eta_write_row<R>(I, nslots, rows.acc0, rows.acc1, rows.pending);
      if (I.nsteps > 0) {
        double e, l;
        eta_total<R>(I, nslots, rows.acc0, rows.acc1, e, l);
        I.acc[0] = e;
        I.acc[1] = l;
      }
    }
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
    int64_t next_out = I.out_every, orow = 1;
    for (int64_t t = 0; t < I.nsteps; ++t) {
      const OutStep os{t + 1 == next_out, orow};
      if (os.now) {
        next_out += I.out_every;
        ++orow;
      }
#pragma unroll 1
      for (int s = 0; s < 4; ++s) {
        if (s == 0 && rows.pending >= 0) {
          if (lead) eta_write_row<float>(I, nslots, rows.acc0, rows.acc1, rows.pending);
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
          node_units<N, float, true, CPLX>(I, cf, cfd, P, v, sng[l], s, rank == 0 && l == 0, s_umask[g], os, ea);
        }
        if (s == 3 && slot >= 0 && (os.now || t + 1 == I.nsteps)) ea.store(I, slot);
        cluster_sync_all();
      }
      if (os.now) rows.pending = os.row;
    }
    if (lead) {
      if (rows.pending >= 0) eta_write_row<float>(I, nslots, rows.acc0, rows.acc1, rows.pending);
      if (I.nsteps > 0) {
        double e, l;
        eta_total<float>(I, nslots, rows.acc0, rows.acc1, e, l);
        I.acc[0] = e;
        I.acc[1] = l;
      }
    }
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

// ------------------------------------------------------------ large-N engine
//
// Hierarchies with 9..24 sites (N is a run-time argument).  A CTA stages a
// tile of 32 consecutive nodes' packed matrices in shared memory (element-
// major, one lane per node, so every access is bank-conflict free); warp w
// then computes the units u = w, w + nwarps, ... of all 32 nodes, reading the
// node's own elements from shared memory and its neighbours' from device
// memory.  Teams and barriers are those of the small-N engine.

struct LargeUnit {
  unsigned char a, b;
};

template <typename R, bool MIXED, bool CPLX>
__global__ void __launch_bounds__(256) heom_large_kernel(EngineArgs A) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ Inst s_inst;
  __shared__ LargeUnit s_units[kMaxSites * (kMaxSites + 1) / 2];

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
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int slot = (rank == 0 && lane == 0) ? warp : -1;  // tile 0 is on rank 0; warp w owns units w, w + nwarps, ...
  const bool lead = (rank == 0 && threadIdx.x == 0);
  unsigned epoch = 0;

  for (int li = A.team_first[team]; li < A.team_first[team + 1]; ++li) {
    __syncthreads();
    if (threadIdx.x == 0) s_inst = A.insts[A.team_list[li]];
    __syncthreads();
    const Inst& I = s_inst;
    const int N = I.N;
    const int NN = N * N;
    const int NP = N * (N - 1) / 2;
    const int U = NP + N;
    using L = CoefLayout<R>;
    // shared memory: tile [NN][32] | coefficients
    R* tile = reinterpret_cast<R*>(dsm);
    unsigned char* cbytes = dsm + (size_t)NN * 32 * sizeof(R);
    const int cb = L::bytes(N);
    for (int i = threadIdx.x; i < cb; i += blockDim.x) cbytes[i] = static_cast<const unsigned char*>(I.coef)[i];
    for (int u = threadIdx.x; u < U; u += blockDim.x) {
      int a, b;
      if (u < NP) {
        int r = u;
        a = 0;
        while (r >= N - 1 - a) { r -= N - 1 - a; ++a; }
        b = a + 1 + r;
      } else {
        a = b = u - NP;
      }
      s_units[u].a = (unsigned char)a;
      s_units[u].b = (unsigned char)b;
    }
    __syncthreads();
    const R* cf = reinterpret_cast<const R*>(cbytes);
    const double* cfd = reinterpret_cast<const double*>(cbytes + L::dbl_offset(N));
    const R* ngam = static_cast<const R*>(I.ngam);
    const int Mp = I.Mpad;
    const int ntiles = (I.M + 31) >> 5;
    EtaAcc<R> ea;
    EtaRows rows;
    rows.acc0 = I.acc[0];
    rows.acc1 = I.acc[1];
    if (lead) {
      if (I.out_pops)
        for (int a = 0; a < N; ++a)
          I.out_pops[a] = MIXED ? ff_to_double(static_cast<const FF*>(I.y0)[a * N + a])
                                : (double)static_cast<const R*>(I.y)[(a * N + a) * Mp];
      if (I.out_el) {
        I.out_el[0] = I.acc[0];
        I.out_el[1] = I.acc[1];
      }
    }
    if (lead)
      for (int k = 0; k < nwarps; ++k) ea.store(I, k);  // zero every running-sum slot of this instance
    if (!team_barrier(A, epoch)) return;
    R* arr[3] = {static_cast<R*>(I.y), static_cast<R*>(I.wa), static_cast<R*>(I.wb)};
    int64_t next_out = I.out_every, orow = 1;
    for (int64_t t = 0; t < I.nsteps; ++t) {
      const OutStep os{t + 1 == next_out, orow};
      if (os.now) {
        next_out += I.out_every;
        ++orow;
      }
#pragma unroll 1
      for (int s = 0; s < 4; ++s) {
        if (s == 0 && rows.pending >= 0) {
          if (lead) eta_write_row<R>(I, nwarps, rows.acc0, rows.acc1, rows.pending);
          rows.pending = -1;
        }
        int in_sel, out_sel;
        stage_buffers(s, in_sel, out_sel);
        const StageCoef<R> P = stage_coef<R>(I, s, in_sel, out_sel);
        const R h = P.h;
        const R* __restrict__ win = arr[in_sel];
        R* __restrict__ wout = arr[out_sel];
        const R* __restrict__ yv = arr[0];
        for (int tl = rank; tl < ntiles; tl += team_size) {
          const int n0 = tl << 5;
          __syncthreads();
          for (int i = threadIdx.x; i < NN * 32; i += blockDim.x) {
            const int p = i >> 5, l = i & 31;
            tile[i] = (n0 + l < I.M) ? win[p * Mp + n0 + l] : R(0);
          }
          __syncthreads();
          const int n = n0 + lane;
          const bool live = n < I.M;
          const bool root = (n == 0);
          const R ng = live ? ngam[n] : R(0);
          const bool term = live && I.terminator && I.up[n] < 0;
          auto Pk = [&](int k, int l) -> R { return tile[(k * N + l) * 32 + lane]; };
          auto S = [&](int k, int l) -> R { return k <= l ? Pk(k, l) : Pk(l, k); };
          auto Aim = [&](int k, int l) -> R { return k < l ? Pk(l, k) : (k > l ? -Pk(k, l) : R(0)); };
          for (int u = warp; u < U && live; u += nwarps) {
            const int a = s_units[u].a, b = s_units[u].b;
            R re = R(0), im = R(0);
            const int da_raw = I.dn[a * Mp + n];
            const int da = da_raw < 0 ? -1 : (da_raw & 0xFFFFFF);
            const R na = da_raw < 0 ? R(0) : R(da_raw >> 24);
            if (a != b) {
              const R x = Pk(a, b), yi = Pk(b, a);
              for (int k = 0; k < N; ++k) {
                const R jak = cf[L::J(N) + a * N + k];
                const R jkb = cf[L::J(N) + k * N + b];
                re += jak * Aim(k, b) - Aim(a, k) * jkb;
                im += S(a, k) * jkb - jak * S(k, b);
                if (CPLX) {
                  const R iak = cf[L::Ji(N) + a * N + k];
                  const R ikb = cf[L::Ji(N) + k * N + b];
                  re += iak * S(k, b) - S(a, k) * ikb;
                  im += iak * Aim(k, b) - Aim(a, k) * ikb;
                }
              }
              const R d = cf[L::eps(N) + a] - cf[L::eps(N) + b];
              const R c = ng + cf[L::ghalf(N) + a] + cf[L::ghalf(N) + b];
              re += d * yi - c * x;
              im -= d * x + c * yi;
              const R al_a = cf[L::alpha(N) + a], be_a = cf[L::beta(N) + a];
              const R al_b = cf[L::alpha(N) + b], be_b = cf[L::beta(N) + b];
              const int upa = I.up[a * Mp + n];
              const int upb = I.up[b * Mp + n];
              if (upa >= 0) {
                re -= win[(b * N + a) * Mp + upa];
                im += win[(a * N + b) * Mp + upa];
              }
              if (upb >= 0) {
                re += win[(b * N + a) * Mp + upb];
                im -= win[(a * N + b) * Mp + upb];
              }
              const int db_raw = I.dn[b * Mp + n];
              const R nb = db_raw < 0 ? R(0) : R(db_raw >> 24);
              if (term) {
                const R ca = (na + R(1)) / (ng + cf[L::gam(N) + a]);
                const R cbf = (nb + R(1)) / (ng + cf[L::gam(N) + b]);
                re += ca * (-al_a * x - be_a * yi) + cbf * (-al_b * x + be_b * yi);
                im += ca * (-al_a * yi + be_a * x) + cbf * (-al_b * yi - be_b * x);
              }
              if (da >= 0) {
                const R yr = win[(a * N + b) * Mp + da];
                const R yy = win[(b * N + a) * Mp + da];
                re += na * (be_a * yr - al_a * yy);
                im += na * (al_a * yr + be_a * yy);
              }
              if (db_raw >= 0) {
                const int db = db_raw & 0xFFFFFF;
                const R yr = win[(a * N + b) * Mp + db];
                const R yy = win[(b * N + a) * Mp + db];
                re += nb * (be_b * yr + al_b * yy);
                im += nb * (be_b * yy - al_b * yr);
              }
            } else {
              const R x = Pk(a, a);
              for (int k = 0; k < N; ++k) {
                if (k == a) continue;
                re += R(2) * cf[L::J(N) + a * N + k] * Aim(k, a);
                if (CPLX) re += R(2) * cf[L::Ji(N) + a * N + k] * S(k, a);
              }
              re -= (ng + R(2) * cf[L::ghalf(N) + a]) * x;
              if (da >= 0) re += R(2) * na * cf[L::beta(N) + a] * win[(a * N + a) * Mp + da];
            }
            // Horner update w = y + h r (root in float-float for mixed precision)
            const int pr = a * N + b, pi = b * N + a;
            if (MIXED && root) {
              if constexpr (MIXED) {
                if (a == b && s == 3) ea.add(I, a, P.root_in[pr]);
                const FF wr = ff_axpy(P.root_y[pr], P.h, P.hl, re);
                P.root_out[pr] = wr;
                wout[pr * Mp] = wr.h;
                if (a != b) {
                  const FF wi = ff_axpy(P.root_y[pi], P.h, P.hl, im);
                  P.root_out[pi] = wi;
                  wout[pi * Mp] = wi.h;
                } else if (s == 3 && I.out_pops && os.now) {
                  I.out_pops[os.row * N + a] = ff_to_double(wr);
                }
              }
            } else {
              if constexpr (!MIXED) {
                if (root && a == b && s == 3) ea.add(I, cfd, N, a, (double)Pk(a, a));
              }
              const R vr = yv[pr * Mp + n] + h * re;
              wout[pr * Mp + n] = vr;
              if (a != b) {
                wout[pi * Mp + n] = yv[pi * Mp + n] + h * im;
              } else if (root && s == 3 && I.out_pops && os.now) {
                I.out_pops[os.row * N + a] = (double)vr;
              }
            }
          }
        }
        if (s == 3 && slot >= 0 && (os.now || t + 1 == I.nsteps)) ea.store(I, slot);
        if (!team_barrier(A, epoch)) return;
      }
      if (os.now) rows.pending = os.row;
    }
    if (lead) {
      if (rows.pending >= 0) eta_write_row<R>(I, nwarps, rows.acc0, rows.acc1, rows.pending);
      if (I.nsteps > 0) {
        double e, l;
        eta_total<R>(I, nwarps, rows.acc0, rows.acc1, e, l);
        I.acc[0] = e;
        I.acc[1] = l;
      }
    }
    if (!team_barrier(A, epoch)) return;
    if (lead) signal_done(I);
  }
}

__host__ __device__ constexpr int large_smem_bytes(int N, int rsize) {
  return N * N * 32 * rsize + ((2 * N * N + 5 * N) * rsize + 7) / 8 * 8 + 2 * N * 8;
}

}  // namespace heom
