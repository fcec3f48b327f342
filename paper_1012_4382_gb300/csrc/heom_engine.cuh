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
// handled by one warp per stage (root_task) so that its double-precision
// accumulation runs with all 32 lanes active.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

namespace heom {

constexpr int kMaxSmallN = 8;
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
  double* y0;          // [N*N] packed root node in double (mixed precision only)
  double* w0a;
  double* w0b;
  const void* coef;    // flat coefficient block, see CoefLayout below
  const void* ngam;    // [Mpad] sum_j n_j gamma_j per node (R)
  double* acc;         // [2] eta and loss integrals
  double* out_pops;    // [nout][N] populations (may be null)
  double* out_el;      // [nout][2] eta, loss (may be null)
  int64_t nsteps;
  int64_t out_every;
  double dt;
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
// A view gives the unit code access to one node's packed matrix P (packed
// element p = k*N + l) and to its links, with every index known at compile
// time.  RegView loads the whole matrix into registers once (cheapest in
// instructions when one thread computes many units of its node); LoadView
// loads each element where a unit needs it (fewest instructions per unit when
// many threads share a node).

template <int N, typename R>
struct RegView {
  R sg[N * N];
  int up[N], dn[N];
  R nj[N];
  __device__ __forceinline__ RegView(const R* __restrict__ w, const int32_t* __restrict__ upt,
                                     const int32_t* __restrict__ dnt, int Mp, int n) {
#pragma unroll
    for (int p = 0; p < N * N; ++p) sg[p] = w[p * Mp + n];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      up[j] = upt[j * Mp + n];
      const int d = dnt[j * Mp + n];
      dn[j] = d < 0 ? -1 : (d & 0xFFFFFF);
      nj[j] = d < 0 ? R(0) : R(d >> 24);
    }
  }
  template <int p>
  __device__ __forceinline__ R P() const { return sg[p]; }
  template <int j>
  __device__ __forceinline__ int Up() const { return up[j]; }
  template <int j>
  __device__ __forceinline__ int Dn() const { return dn[j]; }
  template <int j>
  __device__ __forceinline__ R Nj() const { return nj[j]; }
};

template <int N, typename R>
struct LoadView {
  const R* __restrict__ w;
  const int32_t* __restrict__ upt;
  const int32_t* __restrict__ dnt;
  int Mp;
  __device__ __forceinline__ LoadView(const R* __restrict__ w_, const int32_t* __restrict__ upt_,
                                      const int32_t* __restrict__ dnt_, int Mp_, int n)
      : w(w_ + n), upt(upt_ + n), dnt(dnt_ + n), Mp(Mp_) {}
  template <int p>
  __device__ __forceinline__ R P() const { return w[p * Mp]; }
  template <int j>
  __device__ __forceinline__ int Up() const { return upt[j * Mp]; }
  template <int j>
  __device__ __forceinline__ int Dn() const {
    const int d = dnt[j * Mp];
    return d < 0 ? -1 : (d & 0xFFFFFF);
  }
  template <int j>
  __device__ __forceinline__ R Nj() const {
    const int d = dnt[j * Mp];
    return d < 0 ? R(0) : R(d >> 24);
  }
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

template <typename R>
struct StagePtrs {
  const R* win;
  R* wout;
  const R* y;
  double* out64;  // root output in double (mixed)
  R h;
  double hd;
};

// Right-hand side of unit u (pair (a, b) or diagonal a) of one node.
// Returns the real part in re and, for pairs, the imaginary part in im.
template <int N, int u, typename R, bool CPLX, class V>
__device__ __forceinline__ void unit_rhs(const V& v, const R* __restrict__ cf, const R* __restrict__ win, int Mp,
                                         R ngam, bool term, R& re, R& im) {
  using L = CoefLayout<R>;
  constexpr int NP = N * (N - 1) / 2;
  re = R(0);
  im = R(0);
  if constexpr (u < NP) {
    constexpr int a = pair_a(N, u);
    constexpr int b = pair_b(N, u);
    const R x = v.template P<a * N + b>();   // Re sigma_ab
    const R yi = v.template P<b * N + a>();  // Im sigma_ab
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
    if (ua >= 0) {
      re -= win[(b * N + a) * Mp + ua];
      im += win[(a * N + b) * Mp + ua];
    }
    if (ub >= 0) {
      re += win[(b * N + a) * Mp + ub];
      im -= win[(a * N + b) * Mp + ub];
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
    if (da >= 0) {
      const R n_a = v.template Nj<a>();
      const R yr = win[(a * N + b) * Mp + da];
      const R yy = win[(b * N + a) * Mp + da];
      re += n_a * (be_a * yr - al_a * yy);
      im += n_a * (al_a * yr + be_a * yy);
    }
    if (db >= 0) {
      const R n_b = v.template Nj<b>();
      const R yr = win[(a * N + b) * Mp + db];
      const R yy = win[(b * N + a) * Mp + db];
      re += n_b * (be_b * yr + al_b * yy);
      im += n_b * (be_b * yy - al_b * yr);
    }
  } else {
    constexpr int a = u - NP;
    const R x = v.template P<a * N + a>();
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
    if (da >= 0) re += R(2) * v.template Nj<a>() * cf[L::beta(N) + a] * win[(a * N + a) * Mp + da];
  }
}

// All units of node n that belong to the unit mask, one RK4 stage.
template <int N, typename R, bool MIXED, bool CPLX, class V>
__device__ __forceinline__ void node_units(const Inst& I, const R* __restrict__ cf, const double* __restrict__ cfd,
                                           const StagePtrs<R>& P, const V& v, int s, int n, uint64_t umask,
                                           int64_t step_done) {
  constexpr int NP = N * (N - 1) / 2;
  constexpr int U = NP + N;
  const int Mp = I.Mpad;
  const R* __restrict__ win = P.win;
  R* __restrict__ wout = P.wout;
  const R* __restrict__ yv = P.y;
  const R ngam = static_cast<const R*>(I.ngam)[n];
  const bool term = I.terminator && (v.template Up<0>() < 0);
  const bool out_row = (s == 3) && (n == 0) && I.out_pops && ((step_done + 1) % I.out_every) == 0;

  // eta and loss (plain FP64 path; the mixed path does this in root_task)
  if (!MIXED && s == 3 && n == 0 && (umask & 1ull)) {
    double e = 0.0, l = 0.0;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const double x = (double)win[(m * N + m) * Mp];
      e += cfd[m] * x;
      l += cfd[N + m] * x;
    }
    I.acc[0] += I.dt * e;
    I.acc[1] += I.dt * l;
    if (I.out_el && ((step_done + 1) % I.out_every) == 0) {
      const int64_t o = (step_done + 1) / I.out_every;
      I.out_el[2 * o] = I.acc[0];
      I.out_el[2 * o + 1] = I.acc[1];
    }
  }

  static_for<0, U>([&](auto uc) {
    constexpr int u = decltype(uc)::value;
    if (!((umask >> u) & 1ull)) return;
    R re, im;
    unit_rhs<N, u, R, CPLX>(v, cf, win, Mp, ngam, term, re, im);
    if constexpr (u < NP) {
      constexpr int a = pair_a(N, u);
      constexpr int b = pair_b(N, u);
      constexpr int pr = a * N + b, pi = b * N + a;
      wout[pr * Mp + n] = yv[pr * Mp + n] + P.h * re;
      wout[pi * Mp + n] = yv[pi * Mp + n] + P.h * im;
    } else {
      constexpr int a = u - NP;
      constexpr int pd = a * N + a;
      const R val = yv[pd * Mp + n] + P.h * re;
      wout[pd * Mp + n] = val;
      if (out_row) I.out_pops[((step_done + 1) / I.out_every) * N + a] = (double)val;
    }
  });
}

// Mixed precision: the root node (rho itself) is computed by one warp, one
// unit per lane, and accumulated in double with all lanes active (FP64 runs
// at 1/64 of the FP32 rate here, so it must not serialise on one lane).
template <int N, bool CPLX>
__device__ __forceinline__ void root_task(const Inst& I, const float* __restrict__ cf, const double* __restrict__ cfd,
                                          const StagePtrs<float>& P, int s, int lane, int64_t step_done) {
  using L = CoefLayout<float>;
  constexpr int NP = N * (N - 1) / 2;
  constexpr int U = NP + N;
  const int Mp = I.Mpad;
  const float* __restrict__ win = P.win;  // float copy of the root sits at column 0
  const bool out_step = ((step_done + 1) % I.out_every) == 0;
  if (s == 3) {
    // eta and loss: the extra rows of the augmented RK4 system, from the
    // stage-3 input of the root (in double)
    double e = 0.0, l = 0.0;
    if (lane < N) {
      const double x = I.w0a[lane * N + lane];
      e = cfd[lane] * x;
      l = cfd[N + lane] * x;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      e += __shfl_down_sync(0xffffffffu, e, off);
      l += __shfl_down_sync(0xffffffffu, l, off);
    }
    if (lane == 0) {
      I.acc[0] += I.dt * e;
      I.acc[1] += I.dt * l;
      if (I.out_el && out_step) {
        const int64_t o = (step_done + 1) / I.out_every;
        I.out_el[2 * o] = I.acc[0];
        I.out_el[2 * o + 1] = I.acc[1];
      }
    }
  }
  auto Pk = [&](int k, int l) -> float { return win[(k * N + l) * Mp]; };
  auto S = [&](int k, int l) -> float { return k <= l ? Pk(k, l) : Pk(l, k); };
  auto A = [&](int k, int l) -> float { return k < l ? Pk(l, k) : (k > l ? -Pk(k, l) : 0.f); };
  const bool term = I.terminator && I.up[0] < 0;  // depth 0: the root is the last level
  for (int uu = lane; uu < U; uu += 32) {
    float re = 0.f, im = 0.f;
    int a, b;
    if (uu < NP) {
      int r = uu;
      a = 0;
      while (r >= N - 1 - a) { r -= N - 1 - a; ++a; }
      b = a + 1 + r;
      const float x = Pk(a, b), yi = Pk(b, a);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        if (k != a) {
          const float jak = cf[L::J(N) + a * N + k];
          re += jak * A(k, b);
          im -= jak * S(k, b);
        }
        if (k != b) {
          const float jkb = cf[L::J(N) + k * N + b];
          re -= A(a, k) * jkb;
          im += S(a, k) * jkb;
        }
        if (CPLX) {
          if (k != a) {
            const float jak = cf[L::Ji(N) + a * N + k];
            re += jak * S(k, b);
            im += jak * A(k, b);
          }
          if (k != b) {
            const float jkb = cf[L::Ji(N) + k * N + b];
            re -= S(a, k) * jkb;
            im -= A(a, k) * jkb;
          }
        }
      }
      const float d = cf[L::eps(N) + a] - cf[L::eps(N) + b];
      const float c = cf[L::ghalf(N) + a] + cf[L::ghalf(N) + b];
      re += d * yi - c * x;
      im -= d * x + c * yi;
      const int ua = I.up[a * Mp], ub = I.up[b * Mp];
      if (ua >= 0) {
        re -= win[(b * N + a) * Mp + ua];
        im += win[(a * N + b) * Mp + ua];
      }
      if (ub >= 0) {
        re += win[(b * N + a) * Mp + ub];
        im -= win[(a * N + b) * Mp + ub];
      }
      if (term) {
        const float al_a = cf[L::alpha(N) + a], be_a = cf[L::beta(N) + a];
        const float al_b = cf[L::alpha(N) + b], be_b = cf[L::beta(N) + b];
        const float ca = 1.f / cf[L::gam(N) + a];
        const float cb = 1.f / cf[L::gam(N) + b];
        re += ca * (-al_a * x - be_a * yi) + cb * (-al_b * x + be_b * yi);
        im += ca * (-al_a * yi + be_a * x) + cb * (-al_b * yi - be_b * x);
      }
    } else {
      a = b = uu - NP;
      const float x = Pk(a, a);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        if (k != a) {
          re += 2.f * cf[L::J(N) + a * N + k] * A(k, a);
          if (CPLX) re += 2.f * cf[L::Ji(N) + a * N + k] * S(k, a);
        }
      }
      re -= 2.f * cf[L::ghalf(N) + a] * x;
    }
    // accumulate in double: w = y0 + h r
    const int pr = a * N + b;
    const double vr = I.y0[pr] + P.hd * (double)re;
    P.out64[pr] = vr;
    P.wout[pr * Mp] = (float)vr;
    if (a != b) {
      const int pi = b * N + a;
      const double vi = I.y0[pi] + P.hd * (double)im;
      P.out64[pi] = vi;
      P.wout[pi * Mp] = (float)vi;
    } else if (s == 3 && I.out_pops && out_step) {
      I.out_pops[((step_done + 1) / I.out_every) * N + a] = vr;
    }
  }
}

// Row 0 of the outputs (the state at the start of the call).
template <int N, typename R, bool MIXED>
__device__ __forceinline__ void write_row0(const Inst& I) {
  if (I.out_pops)
    for (int a = 0; a < N; ++a)
      I.out_pops[a] = MIXED ? I.y0[a * N + a] : (double)static_cast<const R*>(I.y)[(a * N + a) * I.Mpad];
  if (I.out_el) {
    I.out_el[0] = I.acc[0];
    I.out_el[1] = I.acc[1];
  }
}

template <int N, typename R, bool MIXED, bool CPLX, bool REG>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 256 : 512) heom_engine_kernel(EngineArgs A) {
  __shared__ __align__(16) unsigned char s_coef[CoefLayout<R>::bytes(kMaxSmallN) + 64];
  __shared__ Inst s_inst;
  __shared__ uint64_t s_umask[32];
  constexpr int U = N * (N - 1) / 2 + N;

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
  unsigned epoch = 0;

  for (int li = A.team_first[team]; li < A.team_first[team + 1]; ++li) {
    __syncthreads();
    if (threadIdx.x == 0) s_inst = A.insts[A.team_list[li]];
    __syncthreads();
    {
      const int nb = CoefLayout<R>::bytes(N);
      const unsigned char* src = static_cast<const unsigned char*>(s_inst.coef);
      for (int i = threadIdx.x; i < nb; i += blockDim.x) s_coef[i] = src[i];
    }
    __syncthreads();
    const Inst& I = s_inst;
    const R* cf = reinterpret_cast<const R*>(s_coef);
    const double* cfd = reinterpret_cast<const double*>(s_coef + CoefLayout<R>::dbl_offset(N));
    const int nblk = (I.M + 31) >> 5;
    const int items = nblk * G;
    const int nitems = items + (MIXED ? 1 : 0);  // the mixed path adds one root task

    if (warp == 0 && lane == 0) write_row0<N, R, MIXED>(I);

    R* y = static_cast<R*>(I.y);
    R* wa = static_cast<R*>(I.wa);
    R* wb = static_cast<R*>(I.wb);
    const double dt = I.dt;
    for (int64_t t = 0; t < I.nsteps; ++t) {
#pragma unroll 1
      for (int s = 0; s < 4; ++s) {
        StagePtrs<R> P;
        P.y = y;
        if (s == 0) { P.win = y;  P.wout = wa; P.out64 = I.w0a; P.hd = 0.25 * dt; }
        else if (s == 1) { P.win = wa; P.wout = wb; P.out64 = I.w0b; P.hd = dt / 3.0; }
        else if (s == 2) { P.win = wb; P.wout = wa; P.out64 = I.w0a; P.hd = 0.5 * dt; }
        else { P.win = wa; P.wout = y;  P.out64 = I.y0; P.hd = dt; }
        P.h = (R)P.hd;
        for (int it = warp; it < nitems; it += W) {
          if (MIXED && it == items) {
            if constexpr (MIXED) root_task<N, CPLX>(I, cf, cfd, P, s, lane, t);
            continue;
          }
          const int nb = it / G;
          const int g = it - nb * G;
          const int n = (nb << 5) + lane;
          if (n >= I.M || (MIXED && n == 0)) continue;
          const uint64_t um = s_umask[g];
          if constexpr (REG) {
            const RegView<N, R> v(P.win, I.up, I.dn, I.Mpad, n);
            node_units<N, R, MIXED, CPLX>(I, cf, cfd, P, v, s, n, um, t);
          } else {
            const LoadView<N, R> v(P.win, I.up, I.dn, I.Mpad, n);
            node_units<N, R, MIXED, CPLX>(I, cf, cfd, P, v, s, n, um, t);
          }
        }
        if (!team_barrier(A, epoch)) return;
      }
    }
  }
}

}  // namespace heom
