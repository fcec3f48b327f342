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
// (one warp lane per node); each node block is split into G "unit groups":
// warp (block, g) computes the packed elements whose unit index u satisfies
// u % G == g.  Units are the N(N-1)/2 off-diagonal pairs (two packed reals
// each) and the N diagonal entries.  Every thread keeps its node's whole
// packed matrix in registers; all index arithmetic on it is resolved at
// compile time.  Between RK4 stages the team synchronises with a hardware
// cluster barrier (release/acquire at cluster scope) or a software grid
// barrier with a bounded wait.
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
  const void* coef;    // flat coefficient block, see coef_layout below
  double* acc;         // [2] eta and loss integrals
  double* out_pops;    // [nout][N] populations (may be null)
  double* out_el;      // [nout][2] eta, loss (may be null)
  int64_t nsteps;
  int64_t out_every;
  double dt;
  double pad2;
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

// ------------------------------------------------------------ node update

template <typename R>
struct StagePtrs {
  const R* win;
  R* wout;
  const R* y;
  double* out64;  // root output in double (mixed)
  R h;
  double hd;
};

// One node (n), one unit group (g of G), one RK4 stage (s).
template <int N, typename R, bool MIXED>
__device__ __forceinline__ void node_update(const Inst& I, const R* __restrict__ cf, const double* __restrict__ cfd,
                                            const StagePtrs<R>& P, int s, int n, int g, int G, int64_t step_done) {
  using L = CoefLayout<R>;
  constexpr int NN = N * N;
  constexpr int NP = N * (N - 1) / 2;
  constexpr int U = NP + N;
  const int Mp = I.Mpad;
  const R* __restrict__ win = P.win;

  R sg[NN];
#pragma unroll
  for (int p = 0; p < NN; ++p) sg[p] = win[(size_t)p * Mp + n];

  int up[N], dn[N];
  R nj[N];
  R ngam = R(0);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    up[j] = I.up[(size_t)j * Mp + n];
    const int d = I.dn[(size_t)j * Mp + n];
    dn[j] = d < 0 ? -1 : (d & 0xFFFFFF);
    nj[j] = d < 0 ? R(0) : R(d >> 24);
    ngam += nj[j] * cf[L::gam(N) + j];
  }
  const bool last_level = up[0] < 0;
  const bool term = last_level && I.terminator;
  const bool cplx = I.complex_h != 0;
  const bool root = (n == 0);

  // eta and loss: RK4 update with the stage-3 input of the root node.
  if (s == 3 && root && g == 0) {
    double e = 0.0, l = 0.0;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const double x = MIXED ? I.w0a[m * N + m] : (double)sg[m * N + m];
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

  auto S = [&](int k, int l) -> R { return k <= l ? sg[k * N + l] : sg[l * N + k]; };
  auto A = [&](int k, int l) -> R { return k < l ? sg[l * N + k] : (k > l ? -sg[k * N + l] : R(0)); };
  auto Jr = [&](int k, int l) -> R { return cf[L::J(N) + k * N + l]; };
  auto Jim = [&](int k, int l) -> R { return cf[L::Ji(N) + k * N + l]; };

  auto store = [&](int p, R r, bool is_diag_a, int a) {
    if (MIXED && root) {
      const double v = I.y0[p] + P.hd * (double)r;
      P.out64[p] = v;
      P.wout[(size_t)p * Mp] = (R)v;
      if (s == 3 && is_diag_a && I.out_pops && ((step_done + 1) % I.out_every) == 0)
        I.out_pops[((step_done + 1) / I.out_every) * N + a] = v;
    } else {
      const R v = P.y[(size_t)p * Mp + n] + P.h * r;
      P.wout[(size_t)p * Mp + n] = v;
      if (s == 3 && root && is_diag_a && I.out_pops && ((step_done + 1) % I.out_every) == 0)
        I.out_pops[((step_done + 1) / I.out_every) * N + a] = (double)v;
    }
  };

  static_for<0, U>([&](auto uc) {
    constexpr int u = decltype(uc)::value;
    if ((u & (G - 1)) != g) return;
    if constexpr (u < NP) {
      constexpr int a = pair_a(N, u);
      constexpr int b = pair_b(N, u);
      const R x = sg[a * N + b];   // Re sigma_ab
      const R yi = sg[b * N + a];  // Im sigma_ab
      R re = R(0), im = R(0);
      // -i[J, sigma]: Re += [J, A]_ab, Im -= [J, S]_ab
      static_for<0, N>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if constexpr (k != a) {
          const R jak = Jr(a, k);
          if constexpr (k != b) re += jak * A(k, b);
          im -= jak * S(k, b);
        }
        if constexpr (k != b) {
          const R jkb = Jr(k, b);
          if constexpr (k != a) re -= A(a, k) * jkb;
          im += S(a, k) * jkb;
        }
      });
      if (cplx) {
        // -i[i Ji, sigma] = [Ji, S] + i [Ji, A]
        static_for<0, N>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          if constexpr (k != a) {
            const R jak = Jim(a, k);
            re += jak * S(k, b);
            if constexpr (k != b) im += jak * A(k, b);
          }
          if constexpr (k != b) {
            const R jkb = Jim(k, b);
            re -= S(a, k) * jkb;
            if constexpr (k != a) im -= A(a, k) * jkb;
          }
        });
      }
      // -i (eps_a - eps_b) sigma_ab and the anti-Hermitian + damping terms
      const R d = cf[L::eps(N) + a] - cf[L::eps(N) + b];
      const R c = ngam + cf[L::ghalf(N) + a] + cf[L::ghalf(N) + b];
      re += d * yi - c * x;
      im -= d * x + c * yi;
      const R al_a = cf[L::alpha(N) + a], be_a = cf[L::beta(N) + a];
      const R al_b = cf[L::alpha(N) + b], be_b = cf[L::beta(N) + b];
      // up-couplings i V_j^x sigma_{n+e_j}: only j = a (+i) and j = b (-i) act on (a, b)
      if (up[a] >= 0) {
        const R xr = win[(size_t)(a * N + b) * Mp + up[a]];
        const R xi = win[(size_t)(b * N + a) * Mp + up[a]];
        re -= xi;
        im += xr;
      }
      if (up[b] >= 0) {
        const R xr = win[(size_t)(a * N + b) * Mp + up[b]];
        const R xi = win[(size_t)(b * N + a) * Mp + up[b]];
        re += xi;
        im -= xr;
      }
      if (term) {
        // sigma_{n+e_j} ~ (n_j+1)/(ngam+gamma_j) theta_j sigma_n, then i V_j^x of it
        const R ca = (nj[a] + R(1)) / (ngam + cf[L::gam(N) + a]);
        const R cb = (nj[b] + R(1)) / (ngam + cf[L::gam(N) + b]);
        re += ca * (-al_a * x - be_a * yi) + cb * (-al_b * x + be_b * yi);
        im += ca * (-al_a * yi + be_a * x) + cb * (-al_b * yi - be_b * x);
      }
      // down-couplings n_j theta_j sigma_{n-e_j}
      if (dn[a] >= 0) {
        const R yr = win[(size_t)(a * N + b) * Mp + dn[a]];
        const R yy = win[(size_t)(b * N + a) * Mp + dn[a]];
        re += nj[a] * (be_a * yr - al_a * yy);
        im += nj[a] * (al_a * yr + be_a * yy);
      }
      if (dn[b] >= 0) {
        const R yr = win[(size_t)(a * N + b) * Mp + dn[b]];
        const R yy = win[(size_t)(b * N + a) * Mp + dn[b]];
        re += nj[b] * (be_b * yr + al_b * yy);
        im += nj[b] * (be_b * yy - al_b * yr);
      }
      store(a * N + b, re, false, a);
      store(b * N + a, im, false, a);
    } else {
      constexpr int a = u - NP;
      const R x = sg[a * N + a];
      R re = R(0);
      static_for<0, N>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if constexpr (k != a) re += R(2) * Jr(a, k) * A(k, a);
      });
      if (cplx) {
        static_for<0, N>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          if constexpr (k != a) re += R(2) * Jim(a, k) * S(k, a);
        });
      }
      re -= (ngam + R(2) * cf[L::ghalf(N) + a]) * x;
      if (dn[a] >= 0) re += R(2) * nj[a] * cf[L::beta(N) + a] * win[(size_t)(a * N + a) * Mp + dn[a]];
      store(a * N + a, re, true, a);
    }
  });
}

// Row 0 of the outputs (state at the start of the call), written by the
// owners of the root's diagonal units.
template <int N, typename R, bool MIXED>
__device__ __forceinline__ void write_row0(const Inst& I, int g, int G) {
  constexpr int NP = N * (N - 1) / 2;
  if (I.out_pops) {
    for (int a = 0; a < N; ++a) {
      if (((NP + a) & (G - 1)) != g) continue;
      const double v = MIXED ? I.y0[a * N + a] : (double)static_cast<const R*>(I.y)[(size_t)(a * N + a) * I.Mpad];
      I.out_pops[a] = v;
    }
  }
  if (g == 0 && I.out_el) {
    I.out_el[0] = I.acc[0];
    I.out_el[1] = I.acc[1];
  }
}

template <int N, typename R, bool MIXED>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 256 : 512) heom_engine_kernel(EngineArgs A) {
  __shared__ __align__(16) unsigned char s_coef[CoefLayout<R>::bytes(kMaxSmallN) + 64];
  __shared__ Inst s_inst;

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
    const int units = nblk << A.logG;

    for (int g = 0; g < G; ++g)
      if (warp == (g % W) && lane == 0) write_row0<N, R, MIXED>(I, g, G);

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
        for (int u = warp; u < units; u += W) {
          const int nb = u >> A.logG;
          const int g = u & (G - 1);
          const int n = (nb << 5) + lane;
          if (n < I.M) node_update<N, R, MIXED>(I, cf, cfd, P, s, n, g, G, t);
        }
        if (!team_barrier(A, epoch)) return;
      }
    }
  }
}

}  // namespace heom
