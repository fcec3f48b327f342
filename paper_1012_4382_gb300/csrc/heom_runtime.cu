// heom_runtime.cu -- host runtime and C ABI of libheom (declared in include/heom.h).
//
// Owns contexts and batches: parameter validation, unit conversion and
// coefficient precompute, node tables, device memory, launch shapes, the
// persistent engine launches and the small utility kernels that move rho and
// the full state in and out.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <set>
#include <tuple>
#include <cmath>
#include <deque>
#include <cstdarg>
#include <cstdio>
#include <climits>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <vector>

#include "heom.h"
#include "heom_flow.cuh"
#include "heom_large.cuh"
#include "heom_internal.h"

using heom::CoefLayout;
using heom::EngineArgs;
using heom::Inst;

namespace {

// ------------------------------------------------------------------ ranges
//
// NVTX ranges (header-only NVTX v3: no-ops unless a profiler is attached)
// around the library's host calls that queue device work, so that a timeline
// shows which call a launch belongs to.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------------ errors

thread_local std::string t_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

#define CUDA_TRY(x)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (x);                                                                \
    if (e_ != cudaSuccess) return fail(HEOM_ECUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

#define TRY(x)                   \
  do {                           \
    int r_ = (x);                \
    if (r_ != HEOM_OK) return r_; \
  } while (0)

// --------------------------------------------------------------- constants
// Unit conversion: an energy or rate nu in cm^-1 is the angular frequency
// 2 pi c nu; with c in cm/fs this is rad/fs (hbar = 1).
constexpr double kPi = 3.14159265358979323846;
constexpr double kSpeedOfLightCmPerFs = 2.99792458e-5;
constexpr double kCmToRadPerFs = 2.0 * kPi * kSpeedOfLightCmPerFs;
constexpr double kBoltzmannCmPerK = 0.6950348004;  // k_B / (h c)
constexpr double kPerPsToPerFs = 1e-3;
// per-instance totals carried between calls: eta, loss, xi = int eta dt,
// elapsed time (fs), steps done by the last call, spare
constexpr int kAccDoubles = 8;

// ------------------------------------------------------------------ memory

struct Hooks {
  heom_alloc_fn alloc = nullptr;
  heom_free_fn release = nullptr;
  void* user = nullptr;
};
std::mutex g_hooks_mu;
Hooks g_hooks;

Hooks current_hooks() {
  std::lock_guard<std::mutex> lk(g_hooks_mu);
  return g_hooks;
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  Hooks hooks;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  int alloc(size_t n, const Hooks& h) {
    release();
    hooks = h;
    if (n == 0) n = 16;
    if (hooks.alloc) {
      p = hooks.alloc(n, hooks.user);
      if (!p) return fail(HEOM_ENOMEM, "device allocation of %zu bytes failed (allocator hook)", n);
    } else {
      cudaError_t e = cudaMalloc(&p, n);
      if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? HEOM_ENOMEM : HEOM_ECUDA, "cudaMalloc(%zu): %s", n,
                    cudaGetErrorString(e));
      }
    }
    bytes = n;
    return HEOM_OK;
  }
  void release() {
    if (!p) return;
    if (hooks.release)
      hooks.release(p, bytes, hooks.user);
    else
      cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct PinnedBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~PinnedBuf() {
    if (p) cudaFreeHost(p);
  }
  int ensure(size_t n) {
    if (n <= bytes) return HEOM_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    CUDA_TRY(cudaHostAlloc(&p, n, cudaHostAllocDefault));
    bytes = n;
    return HEOM_OK;
  }
};

// ------------------------------------------------------------- utilities

// The root node of the mixed path is kept in float-float (hi, lo) pairs.
__device__ __forceinline__ float2 to_ff(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// One thread waits, through the stage barrier's bounded wait, for a counter
// that nothing raises (the self-test of heom_selftest_bounded_wait).  The
// counter holds 2^32 - 1 and the target is 1, i.e. two arrivals past the point
// where the 32-bit count wraps: a plain "counter < target" test would let the
// wait through at once, the wrapped comparison keeps it waiting.
__global__ void bounded_wait_probe_kernel(const unsigned* counter, int* status, uint64_t limit_ns) {
  if (threadIdx.x == 0 && blockIdx.x == 0) heom::bounded_wait_geq(counter, 1u, limit_ns, status);
}

template <typename R>
__global__ void set_root_kernel(R* y, int Mpad, float2* y0, const double* rho, int N, double* acc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N * N) {
    const int a = p / N, b = p - (p / N) * N;
    double v;
    if (a < b)
      v = rho[2 * (a * N + b)];
    else if (a > b)
      v = rho[2 * (b * N + a) + 1];
    else
      v = rho[2 * (a * N + a)];
    y[(size_t)p * Mpad] = (R)v;
    if (y0) y0[p] = to_ff(v);
  }
  if (p == 0)
    for (int k = 0; k < kAccDoubles; ++k) acc[k] = 0.0;
}

// packed element-major state -> full complex matrices [M][N][N]
template <typename R>
__global__ void unpack_state_kernel(const R* y, int Mpad, int64_t M, int N, const float2* y0, double* out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int NN = N * N;
  if (idx >= M * NN) return;
  const int64_t n = idx / NN;
  const int e = (int)(idx - n * NN);
  const int a = e / N, b = e - (e / N) * N;
  auto P = [&](int k, int l) -> double {
    if (n == 0 && y0) return (double)y0[k * N + l].x + (double)y0[k * N + l].y;
    return (double)y[(size_t)(k * N + l) * Mpad + n];
  };
  double re, im;
  if (a < b) {
    re = P(a, b);
    im = P(b, a);
  } else if (a > b) {
    re = P(b, a);
    im = -P(a, b);
  } else {
    re = P(a, a);
    im = 0.0;
  }
  out[2 * idx] = re;
  out[2 * idx + 1] = im;
}

template <typename R>
__global__ void pack_state_kernel(const double* in, R* y, int Mpad, int64_t M, int N, float2* y0) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int NN = N * N;
  if (idx >= M * NN) return;
  const int64_t n = idx / NN;
  const int p = (int)(idx - n * NN);
  const int a = p / N, b = p - (p / N) * N;
  const double* m = in + 2 * n * NN;
  double v;
  if (a < b)
    v = m[2 * (a * N + b)];
  else if (a > b)
    v = m[2 * (b * N + a) + 1];
  else
    v = m[2 * (a * N + a)];
  y[(size_t)p * Mpad + n] = (R)v;
  if (n == 0 && y0) y0[p] = to_ff(v);
}

int launch_blocks(int64_t work, int threads) { return (int)((work + threads - 1) / threads); }

// Largest element modulus of every node's matrix (packed, element-major):
// out[n] = max_ab |sigma_n,ab|, one thread per node.
template <typename R>
__global__ void node_max_kernel(const R* y, int Mpad, int64_t M, int N, double* out) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= M) return;
  double mx = 0.0;
  for (int a = 0; a < N; ++a) {
    mx = fmax(mx, fabs((double)y[(size_t)(a * N + a) * Mpad + n]));
    for (int b = a + 1; b < N; ++b) {
      const double re = (double)y[(size_t)(a * N + b) * Mpad + n], im = (double)y[(size_t)(b * N + a) * Mpad + n];
      mx = fmax(mx, sqrt(re * re + im * im));
    }
  }
  out[n] = mx;
}

// Device-side bounds and consistency check of a node table pair ([N][Mpad]
// int32, element-major like the state; dn packs n_j in its top byte), run on
// the tables every kernel will read, before any propagation reads them.  For
// node n < M and site j: an up link is -1 or a later node u < M whose down
// link on site j is n with n_j(u) = n_j(n) + 1; a down link is -1 or an
// earlier node d with n_j >= 1 whose up link on site j is n; padding nodes
// (M <= n < Mpad) have no links.  A neighbour's entry is read only after its
// index has been found in range.  bad[0] receives the smallest offending node.
__global__ void table_check_kernel(const int32_t* up, const int32_t* dn, int M, int Mpad, int N, int* bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * Mpad) return;
  const int j = (int)(t / Mpad), n = (int)(t - (int64_t)j * Mpad);
  const int32_t u = up[t], d = dn[t];
  bool ok;
  if (n >= M) {
    ok = u == -1 && d == -1;
  } else {
    ok = d == -1 || (d >= 0 && (d >> 24) >= 1 && (d & 0xFFFFFF) < n);
    const int nj = d >= 0 ? (d >> 24) : 0;
    if (ok && d >= 0) ok = up[(int64_t)j * Mpad + (d & 0xFFFFFF)] == n;
    if (ok && u != -1) {
      ok = u > n && u < M;
      if (ok) {
        const int32_t back = dn[(int64_t)j * Mpad + u];
        ok = back >= 0 && (back & 0xFFFFFF) == n && (back >> 24) == nj + 1;
      }
    }
  }
  if (!ok) atomicMin(bad, n);
}

// Runs table_check_kernel on device tables; HEOM_OK, or `code` naming the
// first offending node (bad_node may be NULL).
int check_node_tables(const int32_t* up, const int32_t* dn, int64_t M, int Mpad, int N, cudaStream_t stream,
                      const Hooks& hooks, int code, int64_t* bad_node) {
  DevBuf flag;
  TRY(flag.alloc(sizeof(int), hooks));
  const int none = INT_MAX;
  CUDA_TRY(cudaMemcpyAsync(flag.p, &none, sizeof(int), cudaMemcpyHostToDevice, stream));
  const int64_t work = (int64_t)N * Mpad;
  if (work > 0)
    table_check_kernel<<<launch_blocks(work, 256), 256, 0, stream>>>(up, dn, (int)M, Mpad, N, flag.as<int>());
  CUDA_TRY(cudaGetLastError());
  int bad = none;
  CUDA_TRY(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (bad_node) *bad_node = bad == none ? -1 : bad;
  if (bad != none)
    return fail(code, "node tables (N=%d, %lld nodes) failed the device check at node %d", N, (long long)M, bad);
  return HEOM_OK;
}

// --------------------------------------------------------------- structures

struct Tables {
  int N = 0, K = 0;
  int64_t M = 0;
  int Mpad = 0;
  std::vector<int32_t> multi;  // host copy of the multi-indices [M][N]
  DevBuf up, dn;
};

// Node tables keyed by (N, K); one cache per context, or one shared by all
// requests of a server.
typedef std::map<std::pair<int, int>, std::shared_ptr<Tables>> TableCache;

struct Instance {
  int N = 0, K = 0;
  int64_t M = 0;
  int Mpad = 0;
  int complex_h = 0, terminator = 0;
  int scaled = 0;            // HEOM_FLAG_SCALED: link weights follow the coefficient block
  size_t wsc_offset = 0;     // byte offset of the weights in coef
  std::shared_ptr<Tables> tab;
  DevBuf y, wa, wb, root64, coef, acc, stage, ngam;
  std::vector<unsigned char> coef_host;
  // dataflow engine (launch mode 3, N <= 8): the model's coefficients in double
  // (see flow_table), the device copy of the unit table, the tagged stage
  // buffers and the next call's first tag
  std::vector<double> flow_src;
  DevBuf flow_units, flow_tags;
  unsigned flow_tag = 0;
};

struct LaunchCfg {
  int mode = 0;       // 0: cluster teams on device memory, 1: whole grid, 2: cluster teams on shared
                      // memory, 3: whole grid, dataflow (block = nodes per CTA x units of a node)
  int team_ctas = 1;
  int block = 256;
  int G = 1;
};

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// Lowest-order quantum (low-temperature) correction of bath a, 1/fs, when
// HEOM_FLAG_LOW_TEMP is set (else 0).  The Matsubara terms k >= 1 of the
// Drude-Lorentz correlation function, c_k exp(-nu_k t) with nu_k = 2 pi k kT
// and c_k = 4 lambda gamma kT nu_k / (nu_k^2 - gamma^2), taken as
// delta(t) c_k / nu_k, give the local term -c_a V_a^x V_a^x sigma_n with
// c_a = sum_k c_k / nu_k = 2 lambda kT / gamma - lambda cot(gamma / (2 kT)).
// V_a^x V_a^x damps the elements (a, b) and (b, a), b != a, and leaves the
// diagonal alone, so c_a enters the off-diagonal damping only.
double low_temp_rate(const heom_params& p, int a) {
  if (!(p.flags & HEOM_FLAG_LOW_TEMP)) return 0.0;
  const double kT = kBoltzmannCmPerK * p.T_kelvin * kCmToRadPerFs;
  const double lam = p.lambda[a] * kCmToRadPerFs;
  const double gam = p.gamma[a] * kCmToRadPerFs;
  const double x = gam / (2.0 * kT);
  return 2.0 * lam * kT / gam - lam * std::cos(x) / std::sin(x);
}

// Coefficient block of CoefLayout<R> for a validated parameter set, written
// into out (CoefLayout<R>::bytes(N) bytes; no heap).  J is taken from the
// upper triangle of H and mirrored, so it is exactly symmetric and Ji
// exactly antisymmetric, as the kernels assume.
template <typename R>
void write_coefficients(const heom_params& p, unsigned char* out, int* complex_h) {
  using L = CoefLayout<R>;
  const int N = p.N;
  const int JS = L::JS(N);
  memset(out, 0, L::bytes(N));
  R* c = reinterpret_cast<R*>(out);
  double* cd = reinterpret_cast<double*>(out + L::dbl_offset(N));
  double diag[heom::kMaxSites];
  double mean = 0.0;
  for (int a = 0; a < N; ++a) {
    diag[a] = p.H[2 * (a * N + a)] + (p.add_reorg_to_H ? p.lambda[a] : 0.0);
    mean += diag[a];
  }
  mean /= N;
  int cplx = 0;
  for (int a = 0; a < N; ++a)
    for (int b = a + 1; b < N; ++b) {
      const R re = (R)(p.H[2 * (a * N + b)] * kCmToRadPerFs);
      const double im = p.H[2 * (a * N + b) + 1];
      const R ri = (R)(im * kCmToRadPerFs);
      c[L::J(N) + a * JS + b] = re;
      c[L::J(N) + b * JS + a] = re;
      c[L::Ji(N) + a * JS + b] = ri;
      c[L::Ji(N) + b * JS + a] = -ri;
      if (im != 0.0) cplx = 1;
    }
  const double kT = kBoltzmannCmPerK * p.T_kelvin * kCmToRadPerFs;
  for (int a = 0; a < N; ++a) {
    const double lam = p.lambda[a] * kCmToRadPerFs;
    const double gam = p.gamma[a] * kCmToRadPerFs;
    const double tr = p.trap_rate ? p.trap_rate[a] * kPerPsToPerFs : 0.0;
    const double rc = p.recomb_rate ? p.recomb_rate[a] * kPerPsToPerFs : 0.0;
    R* st = c + L::site(N) + 4 * a;
    st[0] = (R)((diag[a] - mean) * kCmToRadPerFs);
    st[1] = (R)(0.5 * (tr + rc) + low_temp_rate(p, a));
    c[L::gd(N) + a] = (R)(0.5 * (tr + rc));
    st[2] = (R)(2.0 * lam * kT);
    st[3] = (R)(lam * gam);
    c[L::gam(N) + a] = (R)gam;
    cd[a] = tr;
    cd[N + a] = rc;
  }
  *complex_h = cplx;
}

// Scale s_a of the scaled hierarchy (HEOM_FLAG_SCALED), rad^2/fs^2: the
// modulus of the bath amplitude 2 lambda kT - i lambda gamma whose powers the
// auxiliaries are divided by, sigma~_n = sigma_n / prod_j sqrt(n_j! s_j^{n_j})
// (Shi et al., J. Chem. Phys. 130, 084105 (2009)); 1 for a site without a
// bath, whose auxiliaries stay zero whatever the scale.
double scaled_hierarchy_scale(const heom_params& p, int a) {
  const double kT = kBoltzmannCmPerK * p.T_kelvin * kCmToRadPerFs;
  const double lam = p.lambda[a] * kCmToRadPerFs;
  const double gam = p.gamma[a] * kCmToRadPerFs;
  const double s = std::hypot(2.0 * lam * kT, lam * gam);
  return s > 0.0 ? s : 1.0;
}

// The coefficient block into a host vector (the instance's copy of its
// coefficients); for a scaled hierarchy followed, 16-byte aligned, by the link
// weights w[j][0][n] = sqrt((n+1) s_j) (up link of site j at n_j = n) and
// w[j][1][n] = sqrt(n / s_j) (down link), n = 0..K+1, whose byte offset goes
// to *wsc_offset (0 when unscaled).
template <typename R>
void fill_coefficients(const heom_params& p, std::vector<unsigned char>& out, int* complex_h, size_t* wsc_offset) {
  const size_t base = CoefLayout<R>::bytes(p.N);
  *wsc_offset = 0;
  if (!(p.flags & HEOM_FLAG_SCALED)) {
    out.assign(base, 0);
    write_coefficients<R>(p, out.data(), complex_h);
    return;
  }
  const size_t off = (base + 15) / 16 * 16;
  const int S = p.K + 2;
  out.assign(off + sizeof(R) * 2 * (size_t)S * p.N, 0);
  write_coefficients<R>(p, out.data(), complex_h);
  R* w = reinterpret_cast<R*>(out.data() + off);
  for (int j = 0; j < p.N; ++j) {
    const double sj = scaled_hierarchy_scale(p, j);
    for (int n = 0; n < S; ++n) {
      w[(size_t)j * 2 * S + n] = (R)std::sqrt((n + 1) * sj);
      w[(size_t)j * 2 * S + S + n] = (R)std::sqrt(n / sj);
    }
  }
  *wsc_offset = off;
}

// ------------------------------------------------------- dataflow unit table
//
// flow_src holds, in rad/fs and 1/fs: J[N][N] = Re H off the diagonal, Ji[N][N]
// = Im H, eps[N] (mean-shifted site energies), goff[N] = (Gamma_RC + Gamma_phot)/2
// + c (the off-diagonal damping, c the low-temperature correction), gd[N] =
// (Gamma_RC + Gamma_phot)/2, alpha[N] = 2 lambda k_B T, beta[N] = lambda gamma,
// gamma[N], scale[N] (s_j of the scaled hierarchy).
void fill_flow_src(const heom_params& p, std::vector<double>& v) {
  const int N = p.N;
  v.assign((size_t)2 * N * N + 7 * N, 0.0);
  double* J = v.data();
  double* Ji = J + N * N;
  double* eps = Ji + N * N;
  double *goff = eps + N, *gd = goff + N, *al = gd + N, *be = al + N, *ga = be + N, *sc = ga + N;
  double mean = 0.0;
  for (int a = 0; a < N; ++a) mean += p.H[2 * (a * N + a)] + (p.add_reorg_to_H ? p.lambda[a] : 0.0);
  mean /= N;
  for (int a = 0; a < N; ++a)
    for (int b = a + 1; b < N; ++b) {
      J[a * N + b] = J[b * N + a] = p.H[2 * (a * N + b)] * kCmToRadPerFs;
      Ji[a * N + b] = p.H[2 * (a * N + b) + 1] * kCmToRadPerFs;
      Ji[b * N + a] = -Ji[a * N + b];
    }
  const double kT = kBoltzmannCmPerK * p.T_kelvin * kCmToRadPerFs;
  for (int a = 0; a < N; ++a) {
    const double lam = p.lambda[a] * kCmToRadPerFs, gam = p.gamma[a] * kCmToRadPerFs;
    const double tr = p.trap_rate ? p.trap_rate[a] * kPerPsToPerFs : 0.0;
    const double rc = p.recomb_rate ? p.recomb_rate[a] * kPerPsToPerFs : 0.0;
    eps[a] = (p.H[2 * (a * N + a)] + (p.add_reorg_to_H ? p.lambda[a] : 0.0) - mean) * kCmToRadPerFs;
    gd[a] = 0.5 * (tr + rc);
    goff[a] = gd[a] + low_temp_rate(p, a);
    al[a] = 2.0 * lam * kT;
    be[a] = lam * gam;
    ga[a] = gam;
    sc[a] = scaled_hierarchy_scale(p, a);
  }
}

// The own-node part of unit (a, b) of the right-hand side applied to a packed
// node P (element (k, l): Re sigma_kl for k <= l, Im sigma_lk for k > l):
// -i[H_eff, sigma]_ab with the site-energy differences and the trap, decay and
// low-temperature damping, without the node's sum_j n_j gamma_j.
void flow_unit_apply(int N, const double* src, int a, int b, const double* P, double& re, double& im) {
  const double* J = src;
  const double* Ji = J + N * N;
  const double *eps = Ji + N * N, *goff = eps + N, *gd = goff + N;
  auto S = [&](int k, int l) { return k <= l ? P[k * N + l] : P[l * N + k]; };
  auto A = [&](int k, int l) { return k < l ? P[l * N + k] : (k > l ? -P[k * N + l] : 0.0); };
  re = im = 0.0;
  if (a != b) {
    for (int k = 0; k < N; ++k) {
      const double jak = J[a * N + k], jbk = J[b * N + k], iak = Ji[a * N + k], ibk = Ji[b * N + k];
      re += jak * A(k, b) - A(a, k) * jbk + iak * S(k, b) + S(a, k) * ibk;
      im += S(a, k) * jbk - jak * S(k, b) + iak * A(k, b) + A(a, k) * ibk;
    }
    const double x = P[a * N + b], yi = P[b * N + a];
    const double d = eps[a] - eps[b], c = goff[a] + goff[b];
    re += d * yi - c * x;
    im -= d * x + c * yi;
  } else {
    for (int k = 0; k < N; ++k) re += 2.0 * J[a * N + k] * A(k, a) + 2.0 * Ji[a * N + k] * S(k, a);
    re -= 2.0 * gd[a] * P[a * N + a];
  }
}

// Unit table of the dataflow engine: FlowUnit[U] (pairs in the kernels' order,
// then diagonals) followed by FlowSite[N].  Each unit's linear form is read
// off flow_unit_apply on the unit vectors of the packed node.
int flow_table(const Instance& in, std::vector<unsigned char>& out) {
  const int N = in.N, NN = N * N, NP = N * (N - 1) / 2, U = NP + N;
  const double* src = in.flow_src.data();
  const int nre = heom::flow_nre(N, in.complex_h != 0), nim = heom::flow_nim(N, in.complex_h != 0);
  out.assign(sizeof(heom::FlowUnit) * U + sizeof(heom::FlowSite) * N, 0);
  heom::FlowUnit* fu = reinterpret_cast<heom::FlowUnit*>(out.data());
  std::vector<double> P(NN, 0.0), cr(NN), ci(NN);
  for (int u = 0; u < U; ++u) {
    int a, b;
    if (u < NP) {
      a = 0;
      int r = u;
      while (r >= N - 1 - a) {
        r -= N - 1 - a;
        ++a;
      }
      b = a + 1 + r;
    } else {
      a = b = u - NP;
    }
    for (int p = 0; p < NN; ++p) {
      P[p] = 1.0;
      flow_unit_apply(N, src, a, b, P.data(), cr[p], ci[p]);
      P[p] = 0.0;
    }
    heom::FlowUnit& f = fu[u];
    f.a = (uint8_t)a;
    f.b = (uint8_t)b;
    const int pab = a * N + b, pba = b * N + a;
    auto fill = [&](const std::vector<double>& c, uint8_t* idx, double* w, int cap, bool any) -> bool {
      for (int i = 0; i < cap; ++i) {
        idx[i] = (uint8_t)pab;
        w[i] = 0.0;
      }
      if (!any) return true;
      // slot 0: x; slot 1: yi (pairs only: the kernel adds the node's terms there)
      idx[0] = (uint8_t)pab;
      w[0] = c[pab];
      int k = 1;
      if (a != b) {
        idx[1] = (uint8_t)pba;
        w[1] = c[pba];
        k = 2;
      }
      for (int p = 0; p < NN; ++p) {
        if (p == pab || p == pba || c[p] == 0.0) continue;
        if (k >= cap) return false;
        idx[k] = (uint8_t)p;
        w[k] = c[p];
        ++k;
      }
      return true;
    };
    if (!fill(cr, f.ire, f.cre, nre, true) || !fill(ci, f.iim, f.cim, nim, a != b))
      return fail(HEOM_ECUDA, "dataflow unit table: unit (%d,%d) has more terms than its kernel holds", a, b);
  }
  heom::FlowSite* fs = reinterpret_cast<heom::FlowSite*>(out.data() + sizeof(heom::FlowUnit) * U);
  const double* al = src + 2 * NN + 3 * N;
  for (int a = 0; a < N; ++a) {
    fs[a].alpha = al[a];
    fs[a].beta = al[N + a];
    fs[a].gamma = al[2 * N + a];
    fs[a].scale = al[3 * N + a];
  }
  return HEOM_OK;
}

int validate(const heom_params* p, int idx) {
  if (!p) return fail(HEOM_EINVAL, "params[%d] is NULL", idx);
  if (p->N < 1 || p->N > HEOM_MAX_SITES) return fail(HEOM_EINVAL, "params[%d]: N=%d outside 1..%d", idx, p->N, HEOM_MAX_SITES);
  if (p->K < 0 || p->K > 255) return fail(HEOM_EINVAL, "params[%d]: K=%d outside 0..255", idx, p->K);
  const int64_t M = heom::num_nodes(p->N, p->K);
  if (M < 0 || M > HEOM_MAX_NODES)
    return fail(HEOM_EINVAL, "params[%d]: C(N+K,K) nodes exceed %d", idx, HEOM_MAX_NODES);
  if (!p->H || !p->lambda || !p->gamma) return fail(HEOM_EINVAL, "params[%d]: H, lambda and gamma are required", idx);
  if (!(p->T_kelvin > 0.0) || !std::isfinite(p->T_kelvin)) return fail(HEOM_EINVAL, "params[%d]: T must be > 0", idx);
  if (p->precision != HEOM_FP64 && p->precision != HEOM_FP32_MIXED)
    return fail(HEOM_EINVAL, "params[%d]: unknown precision %d", idx, p->precision);
  if (p->terminator != HEOM_TERM_NONE && p->terminator != HEOM_TERM_MARKOV)
    return fail(HEOM_EINVAL, "params[%d]: unknown terminator %d", idx, p->terminator);
  if (p->add_reorg_to_H != 0 && p->add_reorg_to_H != 1)
    return fail(HEOM_EINVAL, "params[%d]: add_reorg_to_H must be 0 or 1", idx);
  if (p->flags & ~(HEOM_FLAG_LOW_TEMP | HEOM_FLAG_SCALED))
    return fail(HEOM_EINVAL, "params[%d]: unknown flags 0x%x", idx, p->flags);
  const int N = p->N;
  double scale = 0.0;
  for (int i = 0; i < 2 * N * N; ++i) {
    if (!std::isfinite(p->H[i])) return fail(HEOM_EINVAL, "params[%d]: H has a non-finite entry", idx);
    scale = std::max(scale, std::fabs(p->H[i]));
  }
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      const double dr = p->H[2 * (a * N + b)] - p->H[2 * (b * N + a)];
      const double di = p->H[2 * (a * N + b) + 1] + p->H[2 * (b * N + a) + 1];
      if (std::fabs(dr) > 1e-12 * std::max(1.0, scale) || std::fabs(di) > 1e-12 * std::max(1.0, scale))
        return fail(HEOM_EINVAL, "params[%d]: H is not Hermitian at (%d,%d)", idx, a, b);
    }
  for (int a = 0; a < N; ++a) {
    if (!(p->lambda[a] >= 0.0) || !std::isfinite(p->lambda[a]))
      return fail(HEOM_EINVAL, "params[%d]: lambda[%d] must be finite and >= 0", idx, a);
    if (!(p->gamma[a] > 0.0) || !std::isfinite(p->gamma[a]))
      return fail(HEOM_EINVAL, "params[%d]: gamma[%d] must be finite and > 0", idx, a);
    if (p->trap_rate && (!(p->trap_rate[a] >= 0.0) || !std::isfinite(p->trap_rate[a])))
      return fail(HEOM_EINVAL, "params[%d]: trap_rate[%d] must be finite and >= 0", idx, a);
    if (p->recomb_rate && (!(p->recomb_rate[a] >= 0.0) || !std::isfinite(p->recomb_rate[a])))
      return fail(HEOM_EINVAL, "params[%d]: recomb_rate[%d] must be finite and >= 0", idx, a);
  }
  if (p->flags & HEOM_FLAG_LOW_TEMP)
    for (int a = 0; a < N; ++a)
      if (!std::isfinite(low_temp_rate(*p, a)))
        return fail(HEOM_EINVAL, "params[%d]: the low-temperature correction of site %d is not finite", idx, a);
  return HEOM_OK;
}

// Horner steps and the eta/loss step factors of one call, in double and as
// float-float pairs (the mixed kernels run no double-precision arithmetic).
void fill_steps(Inst& d, double dt, const double* rates /* trap[N], recomb[N] in 1/fs */) {
  const double h[4] = {0.25 * dt, dt / 3.0, 0.5 * dt, dt};
  for (int s = 0; s < 4; ++s) {
    d.hd[s] = h[s];
    d.hh[s] = (float)h[s];
    d.hl[s] = (float)(h[s] - (double)d.hh[s]);
  }
  for (int a = 0; a < d.N; ++a) {
    const double et = dt * rates[a], el = dt * rates[d.N + a];
    d.ec[4 * a] = (float)et;
    d.ec[4 * a + 1] = (float)(et - (double)d.ec[4 * a]);
    d.ec[4 * a + 2] = (float)el;
    d.ec[4 * a + 3] = (float)(el - (double)d.ec[4 * a + 2]);
    const double ex = 0.5 * dt * dt * rates[a];
    d.xc[2 * a] = (float)ex;
    d.xc[2 * a + 1] = (float)(ex - (double)d.xc[2 * a]);
  }
}

int validate_rho(const double* rho, int N) {
  if (!rho) return fail(HEOM_EINVAL, "rho0 is NULL");
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      const double re = rho[2 * (a * N + b)], im = rho[2 * (a * N + b) + 1];
      if (!std::isfinite(re) || !std::isfinite(im)) return fail(HEOM_EINVAL, "rho0 has a non-finite entry");
      if (std::fabs(re - rho[2 * (b * N + a)]) > 1e-12 || std::fabs(im + rho[2 * (b * N + a) + 1]) > 1e-12)
        return fail(HEOM_EINVAL, "rho0 is not Hermitian at (%d,%d)", a, b);
    }
  return HEOM_OK;
}

}  // namespace

// ------------------------------------------------------------------ engine

struct Engine {
  int prec = HEOM_FP64;
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  Hooks hooks;
  std::vector<std::unique_ptr<Instance>> inst;
  std::shared_ptr<TableCache> tables = std::make_shared<TableCache>();
  std::map<int, LaunchCfg> cfg;  // per N
  double stop_trace = 0.0;        // the stop rule (0: off)
  const uint8_t* subset_keep = nullptr;  // while a filtered context is created: its node flags
  const uint8_t* const* subset_keeps = nullptr;  // while a filtered batch is created: per instance (may hold NULL)
  bool pageable_args = false;     // stage launch descriptors from pageable memory (servers)
  std::vector<unsigned char> h_args_pageable;
  // per-instance output destinations and cadences (servers); empty = contiguous buffers
  std::vector<double*> ovr_pops, ovr_el;
  std::vector<int*> ovr_done;
  std::vector<int64_t> ovr_every;
  DevBuf d_args, d_status, d_gsync, d_out;
  PinnedBuf h_args;
  cudaEvent_t args_done = nullptr;
  bool args_pending = false;
  // set while a CUDA graph of one propagate call is being built: the launch
  // descriptors go to *graph_args (copied before the capture starts) and the
  // launches are captured into *graph_out instead of being run
  DevBuf* graph_args = nullptr;
  cudaGraph_t* graph_out = nullptr;

  ~Engine() {
    if (args_done) {
      cudaEventSynchronize(args_done);
      cudaEventDestroy(args_done);
    }
    if (stream) cudaStreamSynchronize(stream);
  }

  size_t rsize() const { return prec == HEOM_FP64 ? sizeof(double) : sizeof(float); }
  // the FP64 kernels are compiled for at most 256 threads per block (register budget)
  int max_block() const { return prec == HEOM_FP64 ? 256 : 512; }

  int ensure_device() {
    int cur = -1;
    CUDA_TRY(cudaGetDevice(&cur));
    if (cur != device) CUDA_TRY(cudaSetDevice(device));
    return HEOM_OK;
  }

  int init(const heom_params* params, int count, void* s, const Hooks* hooks_override = nullptr,
           std::shared_ptr<TableCache> shared_tables = nullptr) {
    if (shared_tables) tables = shared_tables;
    if (count < 1) return fail(HEOM_EINVAL, "count must be >= 1");
    if (!params) return fail(HEOM_EINVAL, "params is NULL");
    for (int i = 0; i < count; ++i) TRY(validate(&params[i], i));
    prec = params[0].precision;
    for (int i = 1; i < count; ++i)
      if (params[i].precision != prec) return fail(HEOM_EINVAL, "params[%d]: all instances need the same precision", i);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1) {
      cudaGetLastError();
      return fail(HEOM_ECUDA, "no usable CUDA device (%s)", cudaGetErrorString(e));
    }
    CUDA_TRY(cudaGetDevice(&device));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    stream = static_cast<cudaStream_t>(s);
    hooks = hooks_override ? *hooks_override : current_hooks();
    CUDA_TRY(cudaEventCreateWithFlags(&args_done, cudaEventDisableTiming));
    TRY(d_status.alloc(sizeof(int) * 4, hooks));
    TRY(d_gsync.alloc(sizeof(unsigned) * 4, hooks));
    CUDA_TRY(cudaMemsetAsync(d_status.p, 0, sizeof(int) * 4, stream));
    for (int i = 0; i < count; ++i) {
      subset_keep = subset_keeps ? subset_keeps[i] : subset_keep;
      TRY(add_instance(params[i]));
    }
    for (auto& in : inst)
      if (!cfg.count(in->N)) cfg[in->N] = default_cfg(in->N, count);
    // rho(0) = |0><0| everywhere
    std::vector<double> rho;
    for (int i = 0; i < count; ++i) {
      const int N = inst[i]->N;
      rho.assign(2 * N * N, 0.0);
      rho[0] = 1.0;
      TRY(set_rho0_host(i, rho.data()));
    }
    CUDA_TRY(cudaStreamSynchronize(stream));
    return HEOM_OK;
  }

  // Default launch shape for the instances with N sites.  Scaled hierarchies
  // (N <= 8) need a load view (node_threads >= 3) in mode 0 or 1: where any
  // instance of this N is scaled the plain default is moved there.
  LaunchCfg default_cfg(int N, int count) const {
    LaunchCfg c = default_cfg_plain(N, count);
    bool sc = false;
    for (auto& in : inst) sc |= (in->N == N && in->scaled);
    if (sc && N <= heom::kMaxSmallN) {
      if (c.mode == 2) c.mode = 0;
      const int U = N * (N + 1) / 2;
      if (c.G <= 2) c.G = std::max(3, std::min(8, U));
    }
    return c;
  }

  LaunchCfg default_cfg_plain(int N, int count) const {
    LaunchCfg c;
    int64_t Mmax = 0;
    for (auto& in : inst)
      if (in->N == N) Mmax = std::max<int64_t>(Mmax, in->M);
    if (N > heom::kMaxSmallN) {
      c.block = 256;
      c.G = 1;
      if (count == 1 && Mmax >= 1024) {
        c.mode = 1;
      } else {
        c.mode = 0;
        c.team_ctas = count == 1 ? 8 : 2;
      }
      return c;
    }
    if (count == 1) {
      // one hierarchy of 256 nodes or more: the dataflow engine (mode 3), when all its
      // CTAs fit on the GPU at once.  Nodes per CTA, measured on the FMO-like N = 7,
      // depth 6 hierarchy and a filtered version of it (1225 nodes): in mixed precision
      // CTAs of about 336 threads (12 nodes at N = 7: 1.25 us per stage for both, 1.45-2.3
      // with 5-11 or 13 nodes); in FP64, bound by the FP64 pipe, the nodes spread evenly
      // over all SMs, S = ceil(M / SMs)
      // Beyond what one node per thread holds (about 1976 nodes at N = 7), each thread
      // carries npt = 2..6 nodes of its unit (real H, N >= 4; CTAs of at most 256 threads,
      // the nodes spread evenly): the fewest nodes per thread with which all CTAs fit.
      if (Mmax >= 256) {
        const int U = N * (N + 1) / 2;
        bool cplx_any = false;
        for (auto& in : inst) cplx_any |= (in->N == N && in->complex_h);
        for (int npt = 1; npt <= heom::kFlowMaxNpt; ++npt) {
          const int maxthr = npt == 1 ? heom::kFlowMaxThreads : heom::kFlowMaxThreadsMulti;
          const int64_t even = (Mmax + (int64_t)sms * npt - 1) / ((int64_t)sms * npt);
          const int S = (int)std::min<int64_t>(
              maxthr / U, npt > 1 ? even : (prec == HEOM_FP64 ? even : std::max<int64_t>(336 / U, even)));
          const void* k = heom::flow_kernel(prec == HEOM_FP64, cplx_any, N, npt);
          if (S < 1 || !k) continue;
          const int dyn = heom::flow_smem_bytes(N, S * npt, (int)rsize());
          int per_sm = 0;
          if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess &&
              cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, S * U, dyn) == cudaSuccess &&
              (int64_t)per_sm * sms >= (Mmax + S * npt - 1) / (S * npt)) {
            c.mode = 3;
            c.block = S * U;
            c.G = 1;
            c.team_ctas = npt;
            return c;
          }
          cudaGetLastError();
        }
      }
      if ((prec == HEOM_FP64 && Mmax >= 256) || (prec == HEOM_FP32_MIXED && Mmax >= 1024)) {
        // the grid engine: unit groups and CTA size as the autotuner picks them for the
        // N = 7 trap hierarchies of depth 8, 10 and 12 (6435, 19448, 50388 nodes; 202, 608
        // and 1575 blocks of 32 nodes): load views of 8 groups while the node blocks are
        // few, the register view (2 groups) once they fill the GPU.  Measured against 32
        // groups, 1000 steps: mixed 38.9 / 66.8 / 87.1 ms instead of 40.2 / 95.5 / 236.8,
        // FP64 76.4 / 184.8 / 481 instead of 93.2 / 246.5 / 621
        const int64_t nb = (Mmax + 31) / 32;
        c.mode = 1;
        c.team_ctas = 1;
        if (N < 4) {
          c.block = max_block();
          c.G = 2;
        } else if (prec == HEOM_FP64) {
          c.G = nb < 400 ? 8 : 2;
          c.block = nb < 1000 ? 128 : 256;
        } else {
          c.G = nb < 1000 ? 8 : 2;
          c.block = c.G == 8 ? 512 : 256;
        }
      } else {
        c.mode = 0;
        c.block = 256;
        c.G = N >= 4 ? 8 : 2;
        const int64_t units = ((Mmax + 31) / 32) * c.G;
        const int64_t warps = c.block / 32;
        int ctas = (int)std::min<int64_t>(16, std::max<int64_t>(1, (units + warps - 1) / warps));
        int p2 = 1;
        while (p2 < ctas) p2 <<= 1;
        c.team_ctas = std::min(16, p2);
        if (prec == HEOM_FP32_MIXED) {
          // the hierarchy in the cluster's shared memory, ~128 nodes per CTA
          int ct = 1;
          while (ct < 16 && (ct * 128 < Mmax || heom::smem_dyn_bytes(N, smem_slice(Mmax, ct)) > max_dyn_smem())) ct <<= 1;
          if (heom::smem_dyn_bytes(N, smem_slice(Mmax, ct)) <= max_dyn_smem()) {
            c.mode = 2;
            c.team_ctas = ct;
            c.block = 512;
            c.G = 4;
          }
        }
      }
    } else {
      // many hierarchies: small teams so that every instance runs at once
      c.mode = 0;
      c.block = max_block();
      c.G = 2;
      c.team_ctas = 2;
      if (prec == HEOM_FP32_MIXED && heom::smem_dyn_bytes(N, smem_slice(Mmax, 1)) <= max_dyn_smem()) {
        c.mode = 2;
        c.team_ctas = 1;
      }
    }
    return c;
  }

  int add_instance(const heom_params& p) {
    auto in = std::make_unique<Instance>();
    in->N = p.N;
    in->K = p.K;
    in->M = heom::num_nodes(p.N, p.K);
    in->Mpad = (int)((in->M + 31) / 32 * 32);
    in->terminator = p.terminator;
    in->scaled = (p.flags & HEOM_FLAG_SCALED) ? 1 : 0;
    if (p.N <= heom::kMaxSmallN) fill_flow_src(p, in->flow_src);
    if (prec == HEOM_FP64)
      fill_coefficients<double>(p, in->coef_host, &in->complex_h, &in->wsc_offset);
    else
      fill_coefficients<float>(p, in->coef_host, &in->complex_h, &in->wsc_offset);
    auto key = std::make_pair(p.N, p.K);
    auto it = tables->find(key);
    if (subset_keep) {
      // a filtered hierarchy: private tables over the kept nodes
      auto t = std::make_shared<Tables>();
      TRY(build_subset_tables(p, subset_keep, *t));
      in->M = t->M;
      in->Mpad = t->Mpad;
      in->tab = t;
    } else if (it == tables->end()) {
      auto t = std::make_shared<Tables>();
      t->N = p.N;
      t->K = p.K;
      t->M = in->M;
      t->Mpad = in->Mpad;
      heom::Index idx;
      heom::build_index(p.N, p.K, idx);
      t->multi = idx.multi;
      std::vector<int32_t> up((size_t)p.N * t->Mpad, -1), dn((size_t)p.N * t->Mpad, -1);
      for (int64_t n = 0; n < t->M; ++n)
        for (int j = 0; j < p.N; ++j) {
          up[(size_t)j * t->Mpad + n] = idx.up[(size_t)n * p.N + j];
          const int32_t d = idx.down[(size_t)n * p.N + j];
          const int32_t nj = idx.multi[(size_t)n * p.N + j];
          dn[(size_t)j * t->Mpad + n] = d < 0 ? -1 : ((nj << 24) | d);
        }
      TRY(t->up.alloc(up.size() * 4, hooks));
      TRY(t->dn.alloc(dn.size() * 4, hooks));
      CUDA_TRY(cudaMemcpyAsync(t->up.p, up.data(), up.size() * 4, cudaMemcpyHostToDevice, stream));
      CUDA_TRY(cudaMemcpyAsync(t->dn.p, dn.data(), dn.size() * 4, cudaMemcpyHostToDevice, stream));
      TRY(check_node_tables(t->up.as<int32_t>(), t->dn.as<int32_t>(), t->M, t->Mpad, p.N, stream, hooks,
                            HEOM_EINTERNAL, nullptr));
      (*tables)[key] = t;
      in->tab = t;
    } else {
      in->tab = it->second;
    }
    {
      // sum_j n_j gamma_j per node (rad/fs), from the node multi-indices
      const std::vector<int32_t>& multi = in->tab->multi;
      std::vector<unsigned char> ng((size_t)in->Mpad * rsize(), 0);
      for (int64_t n = 0; n < in->M; ++n) {
        double v = 0.0;
        for (int j = 0; j < p.N; ++j) v += multi[(size_t)n * p.N + j] * (p.gamma[j] * kCmToRadPerFs);
        if (prec == HEOM_FP64)
          reinterpret_cast<double*>(ng.data())[n] = v;
        else
          reinterpret_cast<float*>(ng.data())[n] = (float)v;
      }
      TRY(in->ngam.alloc(ng.size(), hooks));
      CUDA_TRY(cudaMemcpyAsync(in->ngam.p, ng.data(), ng.size(), cudaMemcpyHostToDevice, stream));
      CUDA_TRY(cudaStreamSynchronize(stream));
    }
    const size_t arr = (size_t)p.N * p.N * in->Mpad * rsize();
    TRY(in->y.alloc(arr, hooks));
    TRY(in->wa.alloc(arr, hooks));
    TRY(in->wb.alloc(arr, hooks));
    // three root buffers of N*N float-float pairs, then the 32 (eta, loss, xi) partial-sum slots
    TRY(in->root64.alloc(3 * 8 * p.N * p.N + 32 * heom::kPartBytes, hooks));
    TRY(in->coef.alloc(in->coef_host.size(), hooks));
    TRY(in->acc.alloc(kAccDoubles * sizeof(double), hooks));
    TRY(in->stage.alloc(2 * sizeof(double) * p.N * p.N, hooks));
    CUDA_TRY(cudaMemcpyAsync(in->coef.p, in->coef_host.data(), in->coef_host.size(), cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaMemsetAsync(in->y.p, 0, arr, stream));
    CUDA_TRY(cudaMemsetAsync(in->acc.p, 0, kAccDoubles * sizeof(double), stream));
    CUDA_TRY(cudaStreamSynchronize(stream));  // coef_host must outlive the copy
    inst.push_back(std::move(in));
    return HEOM_OK;
  }

  // Node tables of the hierarchy restricted to the nodes with keep[i] != 0
  // (heom_build_index order): the kept nodes in their order, links to removed
  // nodes dropped (-1), the set checked to hold the root and to be closed
  // downwards (every n - e_j of a kept n kept).
  int build_subset_tables(const heom_params& p, const uint8_t* keep, Tables& t) {
    const int N = p.N;
    heom::Index idx;
    heom::build_index(N, p.K, idx);
    const int64_t Mfull = idx.M;
    if (!keep[0]) return fail(HEOM_EINVAL, "the filtered hierarchy must keep the root node (node 0)");
    std::vector<int32_t> sub(Mfull, -1);
    int64_t M = 0;
    for (int64_t i = 0; i < Mfull; ++i)
      if (keep[i]) {
        for (int j = 0; j < N; ++j) {
          const int32_t d = idx.down[(size_t)i * N + j];
          if (d >= 0 && !keep[d])
            return fail(HEOM_EINVAL, "the node set is not closed downwards: node %lld is kept, its n - e_%d (node %d) "
                                     "is not", (long long)i, j, d);
        }
        sub[i] = (int32_t)M++;
      }
    t.N = N;
    t.K = p.K;
    t.M = M;
    t.Mpad = (int)((M + 31) / 32 * 32);
    t.multi.assign((size_t)M * N, 0);
    std::vector<int32_t> up((size_t)N * t.Mpad, -1), dn((size_t)N * t.Mpad, -1);
    for (int64_t i = 0; i < Mfull; ++i) {
      const int32_t si = sub[i];
      if (si < 0) continue;
      for (int j = 0; j < N; ++j) {
        t.multi[(size_t)si * N + j] = idx.multi[(size_t)i * N + j];
        const int32_t u = idx.up[(size_t)i * N + j];
        up[(size_t)j * t.Mpad + si] = u >= 0 ? sub[u] : -1;
        const int32_t d = idx.down[(size_t)i * N + j];
        const int32_t nj = idx.multi[(size_t)i * N + j];
        dn[(size_t)j * t.Mpad + si] = d < 0 ? -1 : ((nj << 24) | sub[d]);
      }
    }
    TRY(t.up.alloc(up.size() * 4, hooks));
    TRY(t.dn.alloc(dn.size() * 4, hooks));
    CUDA_TRY(cudaMemcpyAsync(t.up.p, up.data(), up.size() * 4, cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaMemcpyAsync(t.dn.p, dn.data(), dn.size() * 4, cudaMemcpyHostToDevice, stream));
    return check_node_tables(t.up.as<int32_t>(), t.dn.as<int32_t>(), t.M, t.Mpad, N, stream, hooks, HEOM_EINTERNAL,
                             nullptr);
  }

  // root buffer `which` (0: y0, 1: wa0, 2: wb0) of the mixed path, N*N float2
  float2* root_ptr(const Instance& in, int which) const {
    if (prec == HEOM_FP64) return nullptr;
    return in.root64.as<float2>() + (size_t)which * in.N * in.N;
  }
  void* parts_ptr(const Instance& in) const { return in.root64.as<unsigned char>() + (size_t)3 * 8 * in.N * in.N; }

  int set_rho0_device(int i, const double* d_rho) {
    Instance& in = *inst[i];
    const size_t arr = (size_t)in.N * in.N * in.Mpad * rsize();
    CUDA_TRY(cudaMemsetAsync(in.y.p, 0, arr, stream));
    const int NN = in.N * in.N;
    if (prec == HEOM_FP64)
      set_root_kernel<double><<<launch_blocks(NN, 128), 128, 0, stream>>>(in.y.as<double>(), in.Mpad, nullptr, d_rho,
                                                                         in.N, in.acc.as<double>());
    else
      set_root_kernel<float><<<launch_blocks(NN, 128), 128, 0, stream>>>(in.y.as<float>(), in.Mpad, root_ptr(in, 0),
                                                                        d_rho, in.N, in.acc.as<double>());
    CUDA_TRY(cudaGetLastError());
    return HEOM_OK;
  }

  int set_rho0_host(int i, const double* rho) {
    Instance& in = *inst[i];
    TRY(validate_rho(rho, in.N));
    CUDA_TRY(cudaMemcpyAsync(in.stage.p, rho, sizeof(double) * 2 * in.N * in.N, cudaMemcpyHostToDevice, stream));
    return set_rho0_device(i, in.stage.as<double>());
  }

  // Output offsets (rows) of instance i for a call with these step counts.
  static int64_t nout_of(int64_t nsteps, int64_t out_every) { return nsteps / out_every + 1; }

  int propagate(const double* dt, const int64_t* nsteps, int64_t out_every, double* d_pops, double* d_el) {
    NvtxRange range("heom propagate");
    TRY(ensure_device());
    if (out_every < 1) return fail(HEOM_EINVAL, "out_every must be >= 1");
    const int count = (int)inst.size();
    for (int i = 0; i < count; ++i) {
      if (nsteps[i] < 0) return fail(HEOM_EINVAL, "nsteps[%d] < 0", i);
      if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return fail(HEOM_EINVAL, "dt[%d] must be > 0", i);
    }
    // descriptors for every instance
    std::vector<Inst> hi(count);
    int64_t pop_off = 0, row_off = 0;
    for (int i = 0; i < count; ++i) {
      Instance& in = *inst[i];
      Inst& d = hi[i];
      memset(&d, 0, sizeof(d));
      d.N = in.N;
      d.K = in.K;
      d.M = (int32_t)in.M;
      d.Mpad = in.Mpad;
      d.complex_h = in.complex_h;
      d.terminator = in.terminator;
      d.up = in.tab->up.as<int32_t>();
      d.dn = in.tab->dn.as<int32_t>();
      d.y = in.y.p;
      d.wa = in.wa.p;
      d.wb = in.wb.p;
      d.y0 = root_ptr(in, 0);
      d.w0a = root_ptr(in, 1);
      d.w0b = root_ptr(in, 2);
      d.parts = parts_ptr(in);
      fill_steps(d, dt[i], reinterpret_cast<const double*>(in.coef_host.data() +
                                                           (prec == HEOM_FP64 ? CoefLayout<double>::dbl_offset(in.N)
                                                                              : CoefLayout<float>::dbl_offset(in.N))));
      d.coef = in.coef.p;
      d.ngam = in.ngam.p;
      d.wsc = in.scaled ? in.coef.as<unsigned char>() + in.wsc_offset : nullptr;
      d.wstride = in.K + 2;
      d.acc = in.acc.as<double>();
      d.out_pops = d_pops ? d_pops + pop_off : nullptr;
      d.out_el = d_el ? d_el + 2 * row_off : nullptr;
      d.nsteps = nsteps[i];
      d.out_every = out_every;
      if (!ovr_pops.empty()) {
        d.out_pops = ovr_pops[i];
        d.out_el = ovr_el[i];
        d.done = ovr_done[i];
        d.out_every = ovr_every[i];
      }
      d.dt = dt[i];
      d.stop_trace = stop_trace;
      const int64_t nout = nout_of(nsteps[i], out_every);
      pop_off += nout * in.N;
      row_off += nout;
    }
    // group by N, assign instances to teams (longest first, least loaded team)
    struct Group {
      int N;
      int cplx;
      int sc;          // scaled hierarchies

      int B = 0;       // nodes per CTA (mode 2)
      int dyn = 0;     // dynamic shared memory per CTA
      LaunchCfg c;
      int nteams;
      std::vector<int32_t> first, list;
    };
    std::vector<Group> groups;
    std::map<std::tuple<int, int, int>, std::vector<int>> byN;
    for (int i = 0; i < count; ++i)
      byN[std::make_tuple(inst[i]->N, inst[i]->complex_h, inst[i]->scaled)].push_back(i);
    for (auto& kv : byN) {
      Group g;
      g.N = std::get<0>(kv.first);
      g.cplx = std::get<1>(kv.first);
      g.sc = std::get<2>(kv.first);
      g.c = cfg[g.N];
      std::vector<int>& ids = kv.second;
      if (g.N > heom::kMaxSmallN) {
        if (g.c.mode == 2) return fail(HEOM_EINVAL, "launch mode 2 supports at most %d sites", heom::kMaxSmallN);
        g.dyn = heom::large_smem_bytes(g.N, (int)rsize());
      } else if (g.c.mode == 2) {
        int64_t Mmax = 0;
        for (int id : ids) Mmax = std::max<int64_t>(Mmax, inst[id]->M);
        g.B = smem_slice(Mmax, g.c.team_ctas);
        g.dyn = heom::smem_dyn_bytes(g.N, g.B);
        if (g.dyn > max_dyn_smem())
          return fail(HEOM_EINVAL,
                      "launch mode 2: %lld nodes of N=%d need %d bytes of shared memory per CTA with %d CTAs "
                      "(at most %d); use more team CTAs or mode 0",
                      (long long)Mmax, g.N, g.dyn, g.c.team_ctas, max_dyn_smem());
      } else {
        g.dyn = heom::engine_dyn_bytes(g.N, g.c.block, (int)rsize(), g.c.G <= 2);
      }
      if (!kernel_for(g.N, g.cplx, g.sc, g.c))
        return fail(HEOM_EUNSUPPORTED, "no engine kernel for N=%d, launch mode %d, node_threads %d%s", g.N, g.c.mode,
                    g.c.G, no_kernel_reason(g.N, g.sc));
      if (g.c.mode == 3 && count != 1)
        return fail(HEOM_EUNSUPPORTED, "launch mode 3 (dataflow) propagates a single hierarchy, not a batch");
      if (g.c.mode == 1 || g.c.mode == 3) {
        g.nteams = 1;
      } else {
        int maxc = max_active_teams(g.N, g.cplx, g.sc, g.c, g.dyn);
        if (maxc < 1) return HEOM_ECUDA;
        g.nteams = std::max(1, std::min<int>((int)ids.size(), maxc));
      }
      std::vector<std::vector<int32_t>> lists(g.nteams);
      std::sort(ids.begin(), ids.end(), [&](int a, int b) {
        return (double)inst[a]->M * (double)nsteps[a] > (double)inst[b]->M * (double)nsteps[b];
      });
      typedef std::pair<double, int> Load;
      std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
      for (int t = 0; t < g.nteams; ++t) pq.push(Load(0.0, t));
      for (int id : ids) {
        Load l = pq.top();
        pq.pop();
        lists[l.second].push_back(id);
        l.first += (double)inst[id]->M * (double)std::max<int64_t>(nsteps[id], 1);
        pq.push(l);
      }
      g.first.push_back(0);
      for (int t = 0; t < g.nteams; ++t) {
        for (int32_t id : lists[t]) g.list.push_back(id);
        g.first.push_back((int32_t)g.list.size());
      }
      groups.push_back(std::move(g));
    }
    // stage descriptors and team lists in one pinned buffer, one copy
    size_t bytes = sizeof(Inst) * count;
    std::vector<size_t> off_first(groups.size()), off_list(groups.size());
    for (size_t k = 0; k < groups.size(); ++k) {
      off_first[k] = bytes;
      bytes += sizeof(int32_t) * groups[k].first.size();
      off_list[k] = bytes;
      bytes += sizeof(int32_t) * groups[k].list.size();
      bytes = (bytes + 15) / 16 * 16;
    }
    if (graph_args) {
      for (auto& g : groups)
        if (g.c.mode == 1 || g.c.mode == 3) return fail(HEOM_EUNSUPPORTED, "CUDA graphs take launch modes 0 and 2");
      std::vector<unsigned char> hg(bytes, 0);
      memcpy(hg.data(), hi.data(), sizeof(Inst) * count);
      for (size_t k = 0; k < groups.size(); ++k) {
        memcpy(hg.data() + off_first[k], groups[k].first.data(), sizeof(int32_t) * groups[k].first.size());
        memcpy(hg.data() + off_list[k], groups[k].list.data(), sizeof(int32_t) * groups[k].list.size());
      }
      TRY(graph_args->alloc(bytes, hooks));
      CUDA_TRY(cudaStreamSynchronize(stream));
      CUDA_TRY(cudaMemcpy(graph_args->p, hg.data(), bytes, cudaMemcpyHostToDevice));
      unsigned char* gdb = graph_args->as<unsigned char>();
      // capture on a private stream (the context's stream may be the legacy
      // default stream, which cannot be captured); launches go there meanwhile
      cudaStream_t cs = nullptr;
      CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      const cudaStream_t saved = stream;
      stream = cs;
      const cudaError_t be = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (be != cudaSuccess) {
        stream = saved;
        cudaStreamDestroy(cs);
        return fail(HEOM_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(be));
      }
      int rc = HEOM_OK;
      for (size_t k = 0; k < groups.size() && rc == HEOM_OK; ++k) {
        Group& g = groups[k];
        EngineArgs A;
        A.insts = reinterpret_cast<const Inst*>(gdb);
        A.team_first = reinterpret_cast<const int32_t*>(gdb + off_first[k]);
        A.team_list = reinterpret_cast<const int32_t*>(gdb + off_list[k]);
        A.G = g.c.G;
        A.logG = ilog2(g.c.G);
        A.mode = g.c.mode;
        A.team_ctas = g.c.team_ctas;
        A.gsync = d_gsync.as<unsigned>();
        A.status = d_status.as<int>();
        rc = launch(g.N, g.cplx, g.sc, g.c, g.nteams, A, g.B, g.dyn);
      }
      cudaGraph_t graph = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
      stream = saved;
      cudaStreamDestroy(cs);
      if (rc != HEOM_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != HEOM_OK ? rc : fail(HEOM_ECUDA, "stream capture: %s", cudaGetErrorString(ce));
      }
      *graph_out = graph;
      return HEOM_OK;
    }
    if (args_pending) {
      CUDA_TRY(cudaEventSynchronize(args_done));
      args_pending = false;
    }
    unsigned char* hb = nullptr;
    if (pageable_args) {
      h_args_pageable.resize(bytes);
      hb = h_args_pageable.data();
    } else {
      TRY(h_args.ensure(bytes));
      hb = static_cast<unsigned char*>(h_args.p);
    }
    if (d_args.bytes < bytes) TRY(d_args.alloc(bytes * 2, hooks));
    memcpy(hb, hi.data(), sizeof(Inst) * count);
    for (size_t k = 0; k < groups.size(); ++k) {
      memcpy(hb + off_first[k], groups[k].first.data(), sizeof(int32_t) * groups[k].first.size());
      memcpy(hb + off_list[k], groups[k].list.data(), sizeof(int32_t) * groups[k].list.size());
    }
    CUDA_TRY(cudaMemcpyAsync(d_args.p, hb, bytes, cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaEventRecord(args_done, stream));
    args_pending = true;
    unsigned char* db = d_args.as<unsigned char>();
    for (size_t k = 0; k < groups.size(); ++k) {
      Group& g = groups[k];
      EngineArgs A;
      A.insts = reinterpret_cast<const Inst*>(db);
      A.team_first = reinterpret_cast<const int32_t*>(db + off_first[k]);
      A.team_list = reinterpret_cast<const int32_t*>(db + off_list[k]);
      A.G = g.c.G;
      A.logG = ilog2(g.c.G);
      A.mode = g.c.mode;
      A.team_ctas = g.c.team_ctas;
      A.gsync = d_gsync.as<unsigned>();
      A.status = d_status.as<int>();
      if (g.c.mode == 3) {
        TRY(launch_flow(*inst[g.list[0]], g.c, A.insts + g.list[0], A.status, nsteps[g.list[0]]));
        continue;
      }
      TRY(launch(g.N, g.cplx, g.sc, g.c, g.nteams, A, g.B, g.dyn));
    }
    return HEOM_OK;
  }

  // Nodes per CTA of the dataflow engine for a block of `block` threads.
  static int flow_nodes_per_cta(int N, int block) { return std::max(1, block / (N * (N + 1) / 2)); }

  // The dataflow engine (mode 3) on one instance: the unit table and the
  // tagged stage buffers on first use, the tag base, one cooperative launch.
  int launch_flow(Instance& in, const LaunchCfg& c, const Inst* d_inst, int* d_status, int64_t nsteps) {
    NvtxRange range("heom dataflow launch");
    const int N = in.N, U = N * (N + 1) / 2, NN = N * N;
    const bool fp64 = prec == HEOM_FP64;
    const int npt = c.team_ctas;  // nodes per thread
    const void* k = heom::flow_kernel(fp64, in.complex_h != 0, N, npt);
    if (!k)
      return fail(HEOM_EUNSUPPORTED,
                  "launch mode 3 takes at most %d sites, and more than one node per thread only with real H "
                  "and 4..%d sites (asked: %d nodes per thread)", heom::kMaxSmallN, heom::kMaxSmallN, npt);
    if (nsteps > (int64_t)1 << 29) return fail(HEOM_EINVAL, "launch mode 3 takes at most 2^29 steps per call");
    const int S = flow_nodes_per_cta(N, c.block);
    const int threads = S * U;
    const int maxthr = npt == 1 ? heom::kFlowMaxThreads : heom::kFlowMaxThreadsMulti;
    if (threads > maxthr)
      return fail(HEOM_EINVAL, "launch mode 3: %d nodes x %d units exceed %d threads", S, U, maxthr);
    const int SL = S * npt;  // nodes of a CTA's slice
    const int grid = (int)((in.M + SL - 1) / SL);
    const int dyn = heom::flow_smem_bytes(N, SL, (int)rsize());
    const long long wd = fp64 ? 2 : 1;
    const long long stride = (long long)NN * in.Mpad * wd;
    if (!in.flow_tags.p) {
      std::vector<unsigned char> tab;
      TRY(flow_table(in, tab));
      TRY(in.flow_units.alloc(tab.size(), hooks));
      CUDA_TRY(cudaMemcpy(in.flow_units.p, tab.data(), tab.size(), cudaMemcpyHostToDevice));
      TRY(in.flow_tags.alloc(sizeof(unsigned long long) * (3 * stride + heom::kFlowRing), hooks));
      CUDA_TRY(cudaMemsetAsync(in.flow_tags.p, 0, in.flow_tags.bytes, stream));
      in.flow_tag = 0;
    }
    const unsigned need = (unsigned)(4 * nsteps + 2);
    if (in.flow_tag > 0xF0000000u - need) {
      // the 32-bit tags would wrap: clear the buffers and start again from 0
      CUDA_TRY(cudaMemsetAsync(in.flow_tags.p, 0, in.flow_tags.bytes, stream));
      in.flow_tag = 0;
    }
    CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, dyn));
    if ((int64_t)per_sm * sms < grid)
      return fail(HEOM_EINVAL,
                  "launch mode 3: %d CTAs of %d nodes (%d threads) cannot all be resident (%d per SM); use "
                  "more nodes per CTA or per thread, or another mode",
                  grid, SL, threads, per_sm);
    heom::FlowArgs F;
    F.inst = d_inst;
    F.units = in.flow_units.as<heom::FlowUnit>();
    F.tags = in.flow_tags.as<unsigned long long>();
    F.tag_stride = stride;
    F.ring = F.tags + 3 * stride;
    F.status = d_status;
    F.S = S;
    F.tag0 = in.flow_tag;
    in.flow_tag += need;
    void* args[] = {&F};
    CUDA_TRY(cudaLaunchCooperativeKernel(k, dim3(grid), dim3(threads), args, dyn, stream));
    return HEOM_OK;
  }

  // The kernel of a launch shape, or nullptr where none is built: mode 2 for
  // FP64 or N > 8; scaled hierarchies in mode 2 or with the register view
  // (node_threads <= 2) for N <= 8.
  const void* kernel_for(int N, int cplx, int sc, const LaunchCfg& c) const {
    if (c.mode == 3)
      return N > heom::kMaxSmallN ? nullptr : heom::flow_kernel(prec == HEOM_FP64, cplx != 0, N, c.team_ctas);
    if (N > heom::kMaxSmallN) return c.mode == 2 ? nullptr : heom::large_kernel(prec == HEOM_FP64, cplx != 0, sc != 0);
    if (c.mode == 2) return (prec == HEOM_FP64 || sc) ? nullptr : heom::smem_kernel(cplx != 0, c.G <= 2, N);
    return heom::engine_kernel(prec == HEOM_FP64, cplx != 0, c.G <= 2, N, sc != 0);
  }
  static const char* no_kernel_reason(int N, int sc) {
    if (sc && N <= heom::kMaxSmallN) return " (scaled hierarchies take modes 0 and 1 with node_threads >= 3)";
    return "";
  }

  // Nodes per CTA when a cluster of `ctas` CTAs holds M nodes (mode 2).
  static int smem_slice(int64_t M, int ctas) {
    const int64_t per = (M + ctas - 1) / ctas;
    return (int)((per + 31) / 32 * 32);
  }
  // Dynamic shared memory a CTA of the shared-memory engine may use.
  int max_dyn_smem() const {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    return optin - 4096;  // the kernel's static shared memory
  }

  // Teams of this shape that fit on the GPU at once; 0 on error (message set).
  int max_active_teams(int N, int cplx, int sc, const LaunchCfg& c, int dyn = 0) {
    const void* k = kernel_for(N, cplx, sc, c);
    if (!k) {
      fail(HEOM_EUNSUPPORTED, "no engine kernel for N=%d, launch mode %d, node_threads %d%s", N, c.mode, c.G,
           no_kernel_reason(N, sc));
      return 0;
    }
    if (c.team_ctas > 8) CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    if (dyn > 0) CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(c.team_ctas);
    lc.blockDim = dim3(c.block);
    lc.dynamicSmemBytes = dyn;
    lc.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c.team_ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&n, k, &lc);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(HEOM_ECUDA, "cudaOccupancyMaxActiveClusters(N=%d, ctas=%d, block=%d): %s", N, c.team_ctas, c.block,
           cudaGetErrorString(e));
      return 0;
    }
    if (n < 1) fail(HEOM_ECUDA, "launch shape N=%d ctas=%d block=%d cannot be resident", N, c.team_ctas, c.block);
    return n;
  }

  int launch(int N, int cplx, int sc, const LaunchCfg& c, int nteams, EngineArgs& A, int B = 0, int dyn = 0) {
    NvtxRange range(c.mode == 1 ? "heom grid launch" : "heom cluster launch");
    const void* k = kernel_for(N, cplx, sc, c);
    if (!k)
      return fail(HEOM_EUNSUPPORTED, "no engine kernel for N=%d, launch mode %d, node_threads %d%s", N, c.mode, c.G,
                  no_kernel_reason(N, sc));
    if (c.mode == 1) {
      int per_sm = 0;
      if (dyn > 0) CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
      CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, c.block, dyn));
      if (per_sm < 1) return fail(HEOM_ECUDA, "block of %d threads cannot be resident", c.block);
      const int grid = per_sm * sms;
      CUDA_TRY(cudaMemsetAsync(A.gsync, 0, sizeof(unsigned), stream));
      void* args[] = {&A, &B};
      CUDA_TRY(cudaLaunchCooperativeKernel(k, dim3(grid), dim3(c.block), args, dyn, stream));
      return HEOM_OK;
    }
    if (c.team_ctas > 8) CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    if (dyn > 0) CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(nteams * c.team_ctas);
    lc.blockDim = dim3(c.block);
    lc.dynamicSmemBytes = dyn;
    lc.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c.team_ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    void* args[] = {&A, &B};
    CUDA_TRY(cudaLaunchKernelExC(&lc, k, args));
    return HEOM_OK;
  }

  int check_status() {
    int st = 0;
    CUDA_TRY(cudaStreamSynchronize(stream));
    CUDA_TRY(cudaMemcpy(&st, d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
      CUDA_TRY(cudaMemset(d_status.p, 0, sizeof(int)));
      if (st & heom::kStatusTimeout)
        return fail(HEOM_ETIMEOUT, "a grid barrier wait expired on the device; the call's results are invalid");
      if (st & heom::kStatusNonFinite)
        return fail(HEOM_ENONFINITE,
                    "the propagation produced a NaN or infinite population, eta or loss (a diverging run or a "
                    "non-finite initial state)");
      return fail(HEOM_ECUDA, "device status 0x%x", st);
    }
    return HEOM_OK;
  }

  // host-side blocking propagate with host outputs
  int propagate_host(const double* dt, const int64_t* nsteps, int64_t out_every, double* pops, double* eta,
                     double* trace) {
    if (out_every < 1) return fail(HEOM_EINVAL, "out_every must be >= 1");
    int64_t pop_total = 0, rows = 0;
    for (size_t i = 0; i < inst.size(); ++i) {
      if (nsteps[i] < 0) return fail(HEOM_EINVAL, "nsteps[%zu] < 0", i);
      const int64_t nout = nout_of(nsteps[i], out_every);
      pop_total += nout * inst[i]->N;
      rows += nout;
    }
    const bool want = pops || eta || trace;
    double* dp = nullptr;
    double* de = nullptr;
    if (want) {
      const size_t need = sizeof(double) * (pop_total + 2 * rows);
      if (d_out.bytes < need) TRY(d_out.alloc(need, hooks));
      dp = d_out.as<double>();
      de = dp + pop_total;
    }
    TRY(propagate(dt, nsteps, out_every, dp, de));
    TRY(check_status());
    if (!want) return HEOM_OK;
    std::vector<double> hp(pop_total), he(2 * rows);
    CUDA_TRY(cudaMemcpy(hp.data(), dp, sizeof(double) * pop_total, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(he.data(), de, sizeof(double) * 2 * rows, cudaMemcpyDeviceToHost));
    if (pops) memcpy(pops, hp.data(), sizeof(double) * pop_total);
    int64_t po = 0, ro = 0;
    for (size_t i = 0; i < inst.size(); ++i) {
      const int64_t nout = nout_of(nsteps[i], out_every);
      const int N = inst[i]->N;
      for (int64_t o = 0; o < nout; ++o) {
        if (eta) eta[ro + o] = he[2 * (ro + o)];
        if (trace) {
          double s = 0.0;
          for (int a = 0; a < N; ++a) s += hp[po + o * N + a];
          trace[ro + o] = s;
        }
      }
      po += nout * N;
      ro += nout;
    }
    return HEOM_OK;
  }

  int trapping_time(double* tmean, int64_t* steps) {
    TRY(ensure_device());
    CUDA_TRY(cudaStreamSynchronize(stream));
    for (size_t i = 0; i < inst.size(); ++i) {
      double v[5];
      CUDA_TRY(cudaMemcpy(v, inst[i]->acc.p, sizeof(v), cudaMemcpyDeviceToHost));
      if (tmean) tmean[i] = v[3] * v[0] - v[2];
      if (steps) steps[i] = (int64_t)v[4];
    }
    return HEOM_OK;
  }

  int efficiency(double* eta, double* loss) {
    TRY(ensure_device());
    CUDA_TRY(cudaStreamSynchronize(stream));
    for (size_t i = 0; i < inst.size(); ++i) {
      double v[2];
      CUDA_TRY(cudaMemcpy(v, inst[i]->acc.p, sizeof(v), cudaMemcpyDeviceToHost));
      if (eta) eta[i] = v[0];
      if (loss) loss[i] = v[1];
    }
    return HEOM_OK;
  }

  int get_states(int i, int64_t nodes, double* out, bool only_root) {
    TRY(ensure_device());
    Instance& in = *inst[i];
    const int64_t M = only_root ? 1 : in.M;
    const size_t bytes = sizeof(double) * 2 * (size_t)M * in.N * in.N;
    DevBuf tmp;
    TRY(tmp.alloc(bytes, hooks));
    const int64_t work = M * in.N * in.N;
    if (prec == HEOM_FP64)
      unpack_state_kernel<double><<<launch_blocks(work, 256), 256, 0, stream>>>(in.y.as<double>(), in.Mpad, M, in.N,
                                                                               nullptr, tmp.as<double>());
    else
      unpack_state_kernel<float><<<launch_blocks(work, 256), 256, 0, stream>>>(in.y.as<float>(), in.Mpad, M, in.N,
                                                                              root_ptr(in, 0), tmp.as<double>());
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(stream));
    CUDA_TRY(cudaMemcpy(out, tmp.p, bytes, cudaMemcpyDeviceToHost));
    (void)nodes;
    return HEOM_OK;
  }

  int set_state(int i, const double* in_state, const double* extra) {
    TRY(ensure_device());
    Instance& in = *inst[i];
    const size_t bytes = sizeof(double) * 2 * (size_t)in.M * in.N * in.N;
    for (int64_t n = 0; n < in.M; ++n) {
      int r = validate_rho(in_state + 2 * (size_t)n * in.N * in.N, in.N);
      if (r != HEOM_OK) return fail(HEOM_EINVAL, "state of node %lld is not Hermitian", (long long)n);
    }
    DevBuf tmp;
    TRY(tmp.alloc(bytes, hooks));
    CUDA_TRY(cudaMemcpyAsync(tmp.p, in_state, bytes, cudaMemcpyHostToDevice, stream));
    const int64_t work = in.M * in.N * in.N;
    if (prec == HEOM_FP64)
      pack_state_kernel<double><<<launch_blocks(work, 256), 256, 0, stream>>>(tmp.as<double>(), in.y.as<double>(),
                                                                             in.Mpad, in.M, in.N, nullptr);
    else
      pack_state_kernel<float><<<launch_blocks(work, 256), 256, 0, stream>>>(tmp.as<double>(), in.y.as<float>(),
                                                                            in.Mpad, in.M, in.N, root_ptr(in, 0));
    CUDA_TRY(cudaGetLastError());
    double acc[kAccDoubles] = {extra ? extra[0] : 0.0, extra ? extra[1] : 0.0};
    CUDA_TRY(cudaMemcpyAsync(in.acc.p, acc, sizeof(acc), cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    return HEOM_OK;
  }
};

struct heom_ctx {
  Engine e;
};
struct heom_batch {
  Engine e;
};

// One captured propagate call of a batch (heom_batch_graph_create).
struct heom_graph {
  Engine* e = nullptr;
  DevBuf args;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~heom_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

// ------------------------------------------------------------------- C ABI

extern "C" {

const char* heom_last_error(void) { return t_err.c_str(); }

int heom_selftest_bounded_wait(double limit_ms, int32_t* timed_out, double* waited_ms) {
  if (!(limit_ms > 0.0) || !(limit_ms <= 1000.0)) return fail(HEOM_EINVAL, "limit_ms must be in (0, 1000]");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(HEOM_ECUDA, "no usable CUDA device (%s)", cudaGetErrorString(e));
  }
  unsigned char* buf = nullptr;  // counter (stays at 2^32 - 1) and status word
  CUDA_TRY(cudaMalloc(&buf, 256));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = 0;
  float ms = 0.f;
  cudaError_t ce = cudaMemset(buf, 0, 256);
  if (ce == cudaSuccess) ce = cudaMemset(buf, 0xFF, sizeof(unsigned));
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce == cudaSuccess) ce = cudaEventRecord(e0, 0);
  if (ce == cudaSuccess) {
    bounded_wait_probe_kernel<<<1, 32>>>(reinterpret_cast<unsigned*>(buf), reinterpret_cast<int*>(buf + 128),
                                         (uint64_t)(limit_ms * 1e6));
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaEventRecord(e1, 0);
  if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
  if (ce == cudaSuccess) ce = cudaMemcpy(&st, buf + 128, sizeof(int), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (ce != cudaSuccess) return fail(HEOM_ECUDA, "bounded-wait self-test: %s", cudaGetErrorString(ce));
  if (timed_out) *timed_out = (st & heom::kStatusTimeout) ? 1 : 0;
  if (waited_ms) *waited_ms = ms;
  return HEOM_OK;
}

int heom_num_nodes(int32_t N, int32_t K, int64_t* out) {
  if (!out) return fail(HEOM_EINVAL, "out is NULL");
  if (N < 1 || N > HEOM_MAX_SITES) return fail(HEOM_EINVAL, "N=%d outside 1..%d", N, HEOM_MAX_SITES);
  if (K < 0) return fail(HEOM_EINVAL, "K=%d < 0", K);
  const int64_t M = heom::num_nodes(N, K);
  if (M < 0 || M > HEOM_MAX_NODES) return fail(HEOM_EINVAL, "C(N+K,K) exceeds %d nodes", HEOM_MAX_NODES);
  *out = M;
  return HEOM_OK;
}

int heom_build_index(int32_t N, int32_t K, int32_t* multi, int32_t* up, int32_t* down) {
  int64_t M = 0;
  TRY(heom_num_nodes(N, K, &M));
  heom::Index idx;
  heom::build_index(N, K, idx);
  const size_t n = (size_t)M * N;
  if (multi) memcpy(multi, idx.multi.data(), n * 4);
  if (up) memcpy(up, idx.up.data(), n * 4);
  if (down) memcpy(down, idx.down.data(), n * 4);
  return HEOM_OK;
}

int heom_set_allocator(heom_alloc_fn alloc, heom_free_fn release, void* user) {
  if ((alloc == nullptr) != (release == nullptr)) return fail(HEOM_EINVAL, "set both hooks or neither");
  std::lock_guard<std::mutex> lk(g_hooks_mu);
  g_hooks.alloc = alloc;
  g_hooks.release = release;
  g_hooks.user = user;
  return HEOM_OK;
}

int heom_create(const heom_params* params, void* cuda_stream, heom_ctx** out) {
  if (!out) return fail(HEOM_EINVAL, "out is NULL");
  *out = nullptr;
  auto c = std::make_unique<heom_ctx>();
  TRY(c->e.init(params, 1, cuda_stream));
  *out = c.release();
  return HEOM_OK;
}

int heom_create_subset(const heom_params* params, const uint8_t* keep, void* cuda_stream, heom_ctx** out) {
  if (!out) return fail(HEOM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!keep) return fail(HEOM_EINVAL, "keep is NULL");
  TRY(validate(params, 0));
  if (params->terminator != HEOM_TERM_NONE)
    return fail(HEOM_EUNSUPPORTED, "a filtered hierarchy takes the plain truncation (HEOM_TERM_NONE)");
  auto c = std::make_unique<heom_ctx>();
  c->e.subset_keep = keep;
  const int rc = c->e.init(params, 1, cuda_stream);
  c->e.subset_keep = nullptr;
  TRY(rc);
  *out = c.release();
  return HEOM_OK;
}

int heom_node_magnitudes(heom_ctx* ctx, double* node_max) {
  if (!ctx || !node_max) return fail(HEOM_EINVAL, "ctx or node_max is NULL");
  Engine& e = ctx->e;
  TRY(e.ensure_device());
  Instance& in = *e.inst[0];
  const size_t need = sizeof(double) * (size_t)in.M;
  if (e.d_out.bytes < need) TRY(e.d_out.alloc(need, e.hooks));
  if (e.prec == HEOM_FP64)
    node_max_kernel<double><<<launch_blocks(in.M, 256), 256, 0, e.stream>>>(in.y.as<double>(), in.Mpad, in.M, in.N,
                                                                          e.d_out.as<double>());
  else
    node_max_kernel<float><<<launch_blocks(in.M, 256), 256, 0, e.stream>>>(in.y.as<float>(), in.Mpad, in.M, in.N,
                                                                         e.d_out.as<double>());
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(e.stream));
  CUDA_TRY(cudaMemcpy(node_max, e.d_out.p, need, cudaMemcpyDeviceToHost));
  return HEOM_OK;
}

int heom_check_node_tables(const int32_t* d_up, const int32_t* d_dn, int64_t M, int32_t Mpad, int32_t N,
                           int64_t* bad_node) {
  if (bad_node) *bad_node = -1;
  if (!d_up || !d_dn) return fail(HEOM_EINVAL, "d_up or d_dn is NULL");
  if (N < 1 || N > HEOM_MAX_SITES) return fail(HEOM_EINVAL, "N must be 1..%d", HEOM_MAX_SITES);
  if (M < 1 || Mpad < M || M > HEOM_MAX_NODES)
    return fail(HEOM_EINVAL, "need 1 <= M <= Mpad and M <= %d", HEOM_MAX_NODES);
  return check_node_tables(d_up, d_dn, M, Mpad, N, 0, Hooks(), HEOM_EINVAL, bad_node);
}

int heom_filter_select(int32_t N, int32_t K, const double* node_max, double delta, uint8_t* keep) {
  int64_t M = 0;
  TRY(heom_num_nodes(N, K, &M));
  if (!node_max || !keep) return fail(HEOM_EINVAL, "node_max or keep is NULL");
  if (!(delta >= 0.0)) return fail(HEOM_EINVAL, "delta must be >= 0 (not NaN)");
  heom::Index idx;
  heom::build_index(N, K, idx);
  for (int64_t i = 0; i < M; ++i) keep[i] = (i == 0 || !(node_max[i] < delta)) ? 1 : 0;
  // close downwards: nodes are ordered by level, so one pass from the deepest suffices
  for (int64_t i = M - 1; i > 0; --i)
    if (keep[i])
      for (int j = 0; j < N; ++j) {
        const int32_t d = idx.down[(size_t)i * N + j];
        if (d >= 0) keep[d] = 1;
      }
  return HEOM_OK;
}

void heom_destroy(heom_ctx* ctx) { delete ctx; }

int heom_set_rho0(heom_ctx* ctx, const double* rho0) {
  if (!ctx) return fail(HEOM_EINVAL, "ctx is NULL");
  TRY(ctx->e.ensure_device());
  TRY(ctx->e.set_rho0_host(0, rho0));
  CUDA_TRY(cudaStreamSynchronize(ctx->e.stream));
  return HEOM_OK;
}

int heom_set_rho0_device(heom_ctx* ctx, const double* d_rho0) {
  if (!ctx || !d_rho0) return fail(HEOM_EINVAL, "ctx or d_rho0 is NULL");
  TRY(ctx->e.ensure_device());
  return ctx->e.set_rho0_device(0, d_rho0);
}

int heom_propagate(heom_ctx* ctx, double dt_fs, int64_t nsteps, int64_t out_every, double* pops_out,
                   double* trace_out, double* eta_out) {
  if (!ctx) return fail(HEOM_EINVAL, "ctx is NULL");
  TRY(ctx->e.ensure_device());
  return ctx->e.propagate_host(&dt_fs, &nsteps, out_every, pops_out, eta_out, trace_out);
}

int heom_propagate_device(heom_ctx* ctx, double dt_fs, int64_t nsteps, int64_t out_every, double* d_pops,
                          double* d_eta_loss) {
  if (!ctx) return fail(HEOM_EINVAL, "ctx is NULL");
  return ctx->e.propagate(&dt_fs, &nsteps, out_every, d_pops, d_eta_loss);
}

int heom_synchronize(heom_ctx* ctx) {
  if (!ctx) return fail(HEOM_EINVAL, "ctx is NULL");
  TRY(ctx->e.ensure_device());
  return ctx->e.check_status();
}

int heom_efficiency(heom_ctx* ctx, double* eta_out, double* loss_out) {
  if (!ctx || !eta_out) return fail(HEOM_EINVAL, "ctx or eta_out is NULL");
  return ctx->e.efficiency(eta_out, loss_out);
}

int heom_trapping_time(heom_ctx* ctx, double* t_mean_fs, int64_t* steps_done) {
  if (!ctx || !t_mean_fs) return fail(HEOM_EINVAL, "ctx or t_mean_fs is NULL");
  return ctx->e.trapping_time(t_mean_fs, steps_done);
}

int heom_set_stop(heom_ctx* ctx, double stop_trace) {
  if (!ctx) return fail(HEOM_EINVAL, "ctx is NULL");
  if (!(stop_trace >= 0.0) || !std::isfinite(stop_trace)) return fail(HEOM_EINVAL, "stop_trace must be finite and >= 0");
  ctx->e.stop_trace = stop_trace;
  return HEOM_OK;
}

int heom_get_rho(heom_ctx* ctx, double* rho_out) {
  if (!ctx || !rho_out) return fail(HEOM_EINVAL, "ctx or rho_out is NULL");
  return ctx->e.get_states(0, 1, rho_out, true);
}

int heom_get_state(heom_ctx* ctx, double* state_out, double* extra) {
  if (!ctx || !state_out) return fail(HEOM_EINVAL, "ctx or state_out is NULL");
  TRY(ctx->e.get_states(0, ctx->e.inst[0]->M, state_out, false));
  if (extra) TRY(ctx->e.efficiency(&extra[0], &extra[1]));
  return HEOM_OK;
}

int heom_set_state(heom_ctx* ctx, const double* state_in, const double* extra) {
  if (!ctx || !state_in) return fail(HEOM_EINVAL, "ctx or state_in is NULL");
  return ctx->e.set_state(0, state_in, extra);
}

int heom_ctx_num_nodes(const heom_ctx* ctx, int64_t* out) {
  if (!ctx || !out) return fail(HEOM_EINVAL, "ctx or out is NULL");
  *out = ctx->e.inst[0]->M;
  return HEOM_OK;
}

int heom_set_launch(heom_ctx* ctx, int32_t mode, int32_t team_ctas, int32_t block_threads, int32_t node_threads) {
  if (!ctx) return fail(HEOM_EINVAL, "ctx is NULL");
  LaunchCfg& c = ctx->e.cfg[ctx->e.inst[0]->N];
  LaunchCfg n = c;
  if (mode >= 0) n.mode = mode;
  if (team_ctas > 0) n.team_ctas = team_ctas;
  if (block_threads > 0) n.block = block_threads;
  if (node_threads > 0) n.G = node_threads;
  if (n.mode < 0 || n.mode > 3) return fail(HEOM_EINVAL, "mode must be 0, 1, 2 or 3");
  if ((n.mode == 3) != (c.mode == 3)) {
    // a block size or team size (nodes per thread in mode 3) of the other family of
    // engines does not carry over: take that family's default
    const int N = ctx->e.inst[0]->N;
    const int U = N * (N + 1) / 2;
    if (block_threads <= 0) n.block = n.mode == 3 ? std::max(U, heom::kFlowMaxThreads / U * U) : ctx->e.max_block();
    if (team_ctas <= 0) n.team_ctas = 1;
  }
  if (n.mode == 2 && ctx->e.prec == HEOM_FP64) return fail(HEOM_EINVAL, "mode 2 (shared memory) needs HEOM_FP32_MIXED");
  const int N = ctx->e.inst[0]->N;
  if (N > heom::kMaxSmallN && (n.mode == 2 || n.mode == 3 || n.block > 256))
    return fail(HEOM_EINVAL, "hierarchies with more than %d sites take modes 0 and 1 with at most 256 threads",
                heom::kMaxSmallN);
  if (n.team_ctas < 1 || n.team_ctas > 16) return fail(HEOM_EINVAL, "team_ctas must be 1..16");
  if (n.mode == 3) {
    // block_threads: the CTA size asked for; a CTA runs block_threads / U unit rows
    // (U = N(N+1)/2) of team_ctas nodes each (nodes per thread, 1..kFlowMaxNpt)
    const int U = N * (N + 1) / 2;
    if (n.team_ctas > heom::kFlowMaxNpt)
      return fail(HEOM_EINVAL, "mode 3: team_ctas (nodes per thread) must be 1..%d", heom::kFlowMaxNpt);
    const int maxthr = n.team_ctas == 1 ? heom::kFlowMaxThreads : heom::kFlowMaxThreadsMulti;
    if (n.block < U || n.block > maxthr)
      return fail(HEOM_EINVAL, "mode 3: block_threads must be %d..%d with %d nodes per thread (at least one node "
                  "of %d units)", U, maxthr, n.team_ctas, U);
  } else {
    const int maxb = ctx->e.max_block();
    if (n.block < 64 || n.block > maxb || n.block % 32)
      return fail(HEOM_EINVAL, "block_threads must be 64..%d, multiple of 32", maxb);
  }
  if (n.G < 1 || n.G > 32) return fail(HEOM_EINVAL, "node_threads must be 1..32");
  c = n;
  return HEOM_OK;
}

int heom_get_launch(const heom_ctx* ctx, int32_t* mode, int32_t* team_ctas, int32_t* block_threads,
                    int32_t* node_threads) {
  if (!ctx) return fail(HEOM_EINVAL, "ctx is NULL");
  const LaunchCfg& c = ctx->e.cfg.at(ctx->e.inst[0]->N);
  if (mode) *mode = c.mode;
  if (team_ctas) *team_ctas = c.team_ctas;
  if (block_threads) *block_threads = c.block;
  if (node_threads) *node_threads = c.G;
  return HEOM_OK;
}

int heom_autotune(heom_ctx* ctx, int64_t trial_steps, double* best_us_per_step) {
  NvtxRange range("heom autotune");
  if (!ctx) return fail(HEOM_EINVAL, "ctx is NULL");
  if (trial_steps < 1) return fail(HEOM_EINVAL, "trial_steps must be >= 1");
  Engine& e = ctx->e;
  TRY(e.ensure_device());
  Instance& in = *e.inst[0];
  // snapshot the state
  const size_t arr = (size_t)in.N * in.N * in.Mpad * e.rsize();
  DevBuf sy, sr, sa;
  TRY(sy.alloc(arr, e.hooks));
  TRY(sr.alloc(in.root64.bytes, e.hooks));
  TRY(sa.alloc(in.acc.bytes, e.hooks));
  CUDA_TRY(cudaMemcpyAsync(sy.p, in.y.p, arr, cudaMemcpyDeviceToDevice, e.stream));
  CUDA_TRY(cudaMemcpyAsync(sr.p, in.root64.p, in.root64.bytes, cudaMemcpyDeviceToDevice, e.stream));
  CUDA_TRY(cudaMemcpyAsync(sa.p, in.acc.p, in.acc.bytes, cudaMemcpyDeviceToDevice, e.stream));
  std::vector<LaunchCfg> cands;
  const bool large = in.N > heom::kMaxSmallN;
  for (int G : {1, 2, 4, 8, 16, 32}) {
    if (large && G > 1) break;
    for (int block : {128, 256, 512})
      for (int ctas : {1, 2, 4, 8, 16}) {
        if (block > e.max_block() || (large && block != 256)) continue;
        LaunchCfg c;
        c.mode = 0;
        c.team_ctas = ctas;
        c.block = block;
        c.G = G;
        const int64_t units = ((in.M + 31) / 32) * G;
        if ((int64_t)ctas * block / 32 > 4 * units && ctas > 1) continue;  // mostly idle warps
        cands.push_back(c);
      }
    for (int block : {128, 256, 512}) {
      if (block > e.max_block() || (large && block != 256)) continue;
      LaunchCfg c;
      c.mode = 1;
      c.block = block;
      c.G = G;
      cands.push_back(c);
    }
    if (!large && G == 1) {
      // the dataflow engine: S nodes per unit row and npt nodes per thread (its unit
      // groups are fixed: one thread per unit); shapes whose CTAs cannot all be resident
      // are refused by the launch
      const int U = in.N * (in.N + 1) / 2;
      for (int npt = 1; npt <= heom::kFlowMaxNpt; ++npt) {
        if (!heom::flow_kernel(e.prec == HEOM_FP64, in.complex_h != 0, in.N, npt)) continue;
        const int maxthr = npt == 1 ? heom::kFlowMaxThreads : heom::kFlowMaxThreadsMulti;
        for (int S : {4, 6, 8, 9, 10, 12, 13, 16, 24, 32, 64}) {
          if (S * U > maxthr) continue;
          LaunchCfg c;
          c.mode = 3;
          c.block = S * U;
          c.G = 1;
          c.team_ctas = npt;
          cands.push_back(c);
        }
      }
    }
    if (e.prec == HEOM_FP32_MIXED && !large)
      for (int block : {256, 512})
        for (int ctas : {1, 2, 4, 8, 16}) {
          LaunchCfg c;
          c.mode = 2;
          c.team_ctas = ctas;
          c.block = block;
          c.G = G;
          if (heom::smem_dyn_bytes(in.N, Engine::smem_slice(in.M, ctas)) > e.max_dyn_smem()) continue;
          const int64_t units = ((Engine::smem_slice(in.M, ctas) + 31) / 32) * G;
          if (block / 32 > 4 * units && ctas > 1) continue;
          cands.push_back(c);
        }
  }
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  const LaunchCfg saved = e.cfg[in.N];
  LaunchCfg best = saved;
  float best_ms = 1e30f;
  const double dt = 1.0;
  for (const LaunchCfg& c : cands) {
    e.cfg[in.N] = c;
    const int dyn = large ? heom::large_smem_bytes(in.N, (int)e.rsize())
                          : (c.mode == 2 ? heom::smem_dyn_bytes(in.N, Engine::smem_slice(in.M, c.team_ctas))
                                         : heom::engine_dyn_bytes(in.N, c.block, (int)e.rsize(), c.G <= 2));
    if (c.mode != 1 && c.mode != 3 && e.max_active_teams(in.N, in.complex_h, in.scaled, c, dyn) < 1) {
      t_err.clear();
      continue;
    }
    int64_t warm = 1;
    if (e.propagate(&dt, &warm, 1, nullptr, nullptr) != HEOM_OK) { t_err.clear(); continue; }
    cudaEventRecord(e0, e.stream);
    if (e.propagate(&dt, &trial_steps, trial_steps, nullptr, nullptr) != HEOM_OK) { t_err.clear(); continue; }
    cudaEventRecord(e1, e.stream);
    if (e.check_status() != HEOM_OK) { t_err.clear(); continue; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e.cfg[in.N] = best;
  CUDA_TRY(cudaMemcpyAsync(in.y.p, sy.p, arr, cudaMemcpyDeviceToDevice, e.stream));
  CUDA_TRY(cudaMemcpyAsync(in.root64.p, sr.p, in.root64.bytes, cudaMemcpyDeviceToDevice, e.stream));
  CUDA_TRY(cudaMemcpyAsync(in.acc.p, sa.p, in.acc.bytes, cudaMemcpyDeviceToDevice, e.stream));
  CUDA_TRY(cudaStreamSynchronize(e.stream));
  if (best_us_per_step) *best_us_per_step = best_ms * 1e3 / (double)trial_steps;
  if (best_ms >= 1e30f) return fail(HEOM_ECUDA, "no launch shape ran");
  return HEOM_OK;
}

int heom_batch_create(const heom_params* params, int32_t count, void* cuda_stream, heom_batch** out) {
  if (!out) return fail(HEOM_EINVAL, "out is NULL");
  *out = nullptr;
  auto b = std::make_unique<heom_batch>();
  TRY(b->e.init(params, count, cuda_stream));
  *out = b.release();
  return HEOM_OK;
}

int heom_batch_create_subset(const heom_params* params, const uint8_t* const* keep, int32_t count, void* cuda_stream,
                             heom_batch** out) {
  if (!out) return fail(HEOM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!keep) return fail(HEOM_EINVAL, "keep is NULL");
  if (!params || count < 1) return fail(HEOM_EINVAL, "params is NULL or count < 1");
  for (int i = 0; i < count; ++i)
    if (keep[i] && params[i].terminator != HEOM_TERM_NONE)
      return fail(HEOM_EUNSUPPORTED, "params[%d]: a filtered hierarchy takes the plain truncation", i);
  auto b = std::make_unique<heom_batch>();
  b->e.subset_keeps = keep;
  const int rc = b->e.init(params, count, cuda_stream);
  b->e.subset_keeps = nullptr;
  b->e.subset_keep = nullptr;
  TRY(rc);
  *out = b.release();
  return HEOM_OK;
}

int heom_batch_num_nodes(const heom_batch* b, int32_t i, int64_t* out) {
  if (!b || !out) return fail(HEOM_EINVAL, "batch or out is NULL");
  if (i < 0 || i >= (int)b->e.inst.size()) return fail(HEOM_EINVAL, "instance %d out of range", i);
  *out = b->e.inst[i]->M;
  return HEOM_OK;
}

int heom_batch_node_magnitudes(heom_batch* b, int32_t i, double* node_max) {
  if (!b || !node_max) return fail(HEOM_EINVAL, "batch or node_max is NULL");
  if (i < 0 || i >= (int)b->e.inst.size()) return fail(HEOM_EINVAL, "instance %d out of range", i);
  Engine& e = b->e;
  TRY(e.ensure_device());
  Instance& in = *e.inst[i];
  const size_t need = sizeof(double) * (size_t)in.M;
  if (e.d_out.bytes < need) TRY(e.d_out.alloc(need, e.hooks));
  if (e.prec == HEOM_FP64)
    node_max_kernel<double><<<launch_blocks(in.M, 256), 256, 0, e.stream>>>(in.y.as<double>(), in.Mpad, in.M, in.N,
                                                                          e.d_out.as<double>());
  else
    node_max_kernel<float><<<launch_blocks(in.M, 256), 256, 0, e.stream>>>(in.y.as<float>(), in.Mpad, in.M, in.N,
                                                                         e.d_out.as<double>());
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(e.stream));
  CUDA_TRY(cudaMemcpy(node_max, e.d_out.p, need, cudaMemcpyDeviceToHost));
  return HEOM_OK;
}

int heom_batch_count(const heom_batch* b, int32_t* count) {
  if (!b || !count) return fail(HEOM_EINVAL, "batch or count is NULL");
  *count = (int32_t)b->e.inst.size();
  return HEOM_OK;
}

int heom_batch_set_rho0(heom_batch* b, const double* rho0_all) {
  if (!b || !rho0_all) return fail(HEOM_EINVAL, "batch or rho0_all is NULL");
  TRY(b->e.ensure_device());
  size_t off = 0;
  for (size_t i = 0; i < b->e.inst.size(); ++i) {
    TRY(b->e.set_rho0_host((int)i, rho0_all + off));
    CUDA_TRY(cudaStreamSynchronize(b->e.stream));  // the staging copy reads rho0_all
    off += 2 * (size_t)b->e.inst[i]->N * b->e.inst[i]->N;
  }
  return HEOM_OK;
}

int heom_batch_propagate(heom_batch* b, const double* dt_fs, const int64_t* nsteps, int64_t out_every,
                         double* pops_out, double* eta_out) {
  if (!b || !dt_fs || !nsteps) return fail(HEOM_EINVAL, "batch, dt_fs or nsteps is NULL");
  TRY(b->e.ensure_device());
  return b->e.propagate_host(dt_fs, nsteps, out_every, pops_out, eta_out, nullptr);
}

int heom_batch_propagate_device(heom_batch* b, const double* dt_fs, const int64_t* nsteps, int64_t out_every,
                                double* d_pops, double* d_eta_loss) {
  if (!b || !dt_fs || !nsteps) return fail(HEOM_EINVAL, "batch, dt_fs or nsteps is NULL");
  TRY(b->e.ensure_device());
  return b->e.propagate(dt_fs, nsteps, out_every, d_pops, d_eta_loss);
}

int heom_batch_synchronize(heom_batch* b) {
  if (!b) return fail(HEOM_EINVAL, "batch is NULL");
  TRY(b->e.ensure_device());
  return b->e.check_status();
}

int heom_batch_efficiency(heom_batch* b, double* eta_out, double* loss_out) {
  if (!b) return fail(HEOM_EINVAL, "batch is NULL");
  return b->e.efficiency(eta_out, loss_out);
}

int heom_batch_trapping_time(heom_batch* b, double* t_mean_fs, int64_t* steps_done) {
  if (!b || !t_mean_fs) return fail(HEOM_EINVAL, "batch or t_mean_fs is NULL");
  return b->e.trapping_time(t_mean_fs, steps_done);
}

int heom_batch_set_stop(heom_batch* b, double stop_trace) {
  if (!b) return fail(HEOM_EINVAL, "batch is NULL");
  if (!(stop_trace >= 0.0) || !std::isfinite(stop_trace)) return fail(HEOM_EINVAL, "stop_trace must be finite and >= 0");
  b->e.stop_trace = stop_trace;
  return HEOM_OK;
}

int heom_batch_graph_create(heom_batch* b, const double* dt_fs, const int64_t* nsteps, int64_t out_every,
                            double* d_pops, double* d_eta_loss, heom_graph** out) {
  if (!b || !dt_fs || !nsteps || !out) return fail(HEOM_EINVAL, "batch, dt_fs, nsteps or out is NULL");
  *out = nullptr;
  TRY(b->e.ensure_device());
  std::unique_ptr<heom_graph> g(new heom_graph());
  g->e = &b->e;
  b->e.graph_args = &g->args;
  b->e.graph_out = &g->graph;
  const int rc = b->e.propagate(dt_fs, nsteps, out_every, d_pops, d_eta_loss);
  b->e.graph_args = nullptr;
  b->e.graph_out = nullptr;
  if (rc != HEOM_OK) return rc;
  CUDA_TRY(cudaGraphInstantiate(&g->exec, g->graph, 0));
  *out = g.release();
  return HEOM_OK;
}

int heom_graph_launch(heom_graph* g) {
  if (!g || !g->exec) return fail(HEOM_EINVAL, "graph is NULL");
  TRY(g->e->ensure_device());
  CUDA_TRY(cudaGraphLaunch(g->exec, g->e->stream));
  return HEOM_OK;
}

void heom_graph_destroy(heom_graph* g) { delete g; }

int heom_batch_get_rho(heom_batch* b, int32_t i, double* rho_out) {
  if (!b || !rho_out) return fail(HEOM_EINVAL, "batch or rho_out is NULL");
  if (i < 0 || i >= (int32_t)b->e.inst.size()) return fail(HEOM_EINVAL, "instance %d out of range", i);
  return b->e.get_states(i, 1, rho_out, true);
}

int heom_batch_set_launch(heom_batch* b, int32_t mode, int32_t team_ctas, int32_t block_threads,
                          int32_t node_threads) {
  if (!b) return fail(HEOM_EINVAL, "batch is NULL");
  if (mode >= 0 && mode != 0 && mode != 2) return fail(HEOM_EINVAL, "batch launch mode must be 0 or 2");
  if (mode == 2 && b->e.prec == HEOM_FP64) return fail(HEOM_EINVAL, "mode 2 (shared memory) needs HEOM_FP32_MIXED");
  for (auto& kv : b->e.cfg) {
    LaunchCfg n = kv.second;
    if (mode >= 0) n.mode = mode;
    if (team_ctas > 0) n.team_ctas = team_ctas;
    if (block_threads > 0) n.block = block_threads;
    if (node_threads > 0) n.G = node_threads;
    if (n.team_ctas < 1 || n.team_ctas > 16) return fail(HEOM_EINVAL, "team_ctas must be 1..16");
    const int maxb = b->e.max_block();
    if (n.block < 64 || n.block > maxb || n.block % 32)
      return fail(HEOM_EINVAL, "block_threads must be 64..%d, multiple of 32", maxb);
    if (n.G < 1 || n.G > 32) return fail(HEOM_EINVAL, "node_threads must be 1..32");
    kv.second = n;
  }
  return HEOM_OK;
}

int heom_batch_autotune(heom_batch* b, int64_t trial_steps, double* best_ms) {
  if (!b) return fail(HEOM_EINVAL, "batch is NULL");
  if (trial_steps < 1) return fail(HEOM_EINVAL, "trial_steps must be >= 1");
  Engine& e = b->e;
  TRY(e.ensure_device());
  // snapshot every instance's state (y, root and running-sum buffers, accumulators)
  const int count = (int)e.inst.size();
  std::vector<DevBuf> sy(count), sr(count), sa(count);
  for (int i = 0; i < count; ++i) {
    Instance& in = *e.inst[i];
    const size_t arr = (size_t)in.N * in.N * in.Mpad * e.rsize();
    TRY(sy[i].alloc(arr, e.hooks));
    TRY(sr[i].alloc(in.root64.bytes, e.hooks));
    TRY(sa[i].alloc(in.acc.bytes, e.hooks));
    CUDA_TRY(cudaMemcpyAsync(sy[i].p, in.y.p, arr, cudaMemcpyDeviceToDevice, e.stream));
    CUDA_TRY(cudaMemcpyAsync(sr[i].p, in.root64.p, in.root64.bytes, cudaMemcpyDeviceToDevice, e.stream));
    CUDA_TRY(cudaMemcpyAsync(sa[i].p, in.acc.p, in.acc.bytes, cudaMemcpyDeviceToDevice, e.stream));
  }
  // candidates: cluster teams on device memory, and on distributed shared memory in mixed precision;
  // one shape for every site count of the batch
  std::vector<LaunchCfg> cands;
  for (int mode : {0, 2}) {
    if (mode == 2 && e.prec != HEOM_FP32_MIXED) continue;
    for (int block : {256, 512}) {
      if (block > e.max_block()) continue;
      for (int ctas : {1, 2, 4, 8, 16})
        for (int G : {1, 2, 4, 8}) {
          LaunchCfg c;
          c.mode = mode;
          c.team_ctas = ctas;
          c.block = block;
          c.G = G;
          cands.push_back(c);
        }
    }
  }
  const std::map<int, LaunchCfg> saved = e.cfg;
  std::map<int, LaunchCfg> best = saved;
  float best_t = 1e30f;
  std::vector<double> dt(count, 1.0);
  std::vector<int64_t> one(count, 1), steps(count, trial_steps);
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  for (const LaunchCfg& c : cands) {
    for (auto& kv : e.cfg) kv.second = c;
    // the shape must run every instance (too little shared memory, no kernel: skipped)
    if (e.propagate(dt.data(), one.data(), 1, nullptr, nullptr) != HEOM_OK || e.check_status() != HEOM_OK) {
      cudaGetLastError();
      t_err.clear();
      continue;
    }
    cudaEventRecord(e0, e.stream);
    if (e.propagate(dt.data(), steps.data(), trial_steps, nullptr, nullptr) != HEOM_OK) {
      cudaGetLastError();
      t_err.clear();
      continue;
    }
    cudaEventRecord(e1, e.stream);
    if (e.check_status() != HEOM_OK) {
      t_err.clear();
      continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_t) {
      best_t = ms;
      best = e.cfg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e.cfg = best;
  for (int i = 0; i < count; ++i) {
    Instance& in = *e.inst[i];
    const size_t arr = (size_t)in.N * in.N * in.Mpad * e.rsize();
    CUDA_TRY(cudaMemcpyAsync(in.y.p, sy[i].p, arr, cudaMemcpyDeviceToDevice, e.stream));
    CUDA_TRY(cudaMemcpyAsync(in.root64.p, sr[i].p, in.root64.bytes, cudaMemcpyDeviceToDevice, e.stream));
    CUDA_TRY(cudaMemcpyAsync(in.acc.p, sa[i].p, in.acc.bytes, cudaMemcpyDeviceToDevice, e.stream));
  }
  CUDA_TRY(cudaStreamSynchronize(e.stream));
  if (best_t >= 1e30f) {
    e.cfg = saved;
    return fail(HEOM_ECUDA, "no launch shape ran");
  }
  if (best_ms) *best_ms = best_t;
  return HEOM_OK;
}

int heom_batch_get_launch(const heom_batch* b, int32_t N, int32_t* mode, int32_t* team_ctas, int32_t* block_threads,
                          int32_t* node_threads) {
  if (!b) return fail(HEOM_EINVAL, "batch is NULL");
  auto it = b->e.cfg.find(N);
  if (it == b->e.cfg.end()) return fail(HEOM_EINVAL, "the batch has no instance with N=%d", N);
  const LaunchCfg& c = it->second;
  if (mode) *mode = c.mode;
  if (team_ctas) *team_ctas = c.team_ctas;
  if (block_threads) *block_threads = c.block;
  if (node_threads) *node_threads = c.G;
  return HEOM_OK;
}

void heom_batch_destroy(heom_batch* b) { delete b; }

}  // extern "C"

// ----------------------------------------------------- allocation-free entry
//
// heom_propagate_static: one complete propagation that allocates nothing.
// Callers that cannot call cudaMalloc (code running under a device-memory
// budget fixed up front, or inside a host framework that owns every device
// allocation) get all of the working memory from the file-scope array below:
// the node tables, the coefficient block, the state and both RK4 stage
// buffers, the launch descriptor and the status words.  The caller passes the
// input rho(0) and the output buffers.  Host-side staging uses a static host
// array under a mutex, so no heap memory is taken either.

namespace {

__device__ __align__(256) unsigned char g_heom_static_scratch[HEOM_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
int32_t g_static_host_tables[HEOM_STATIC_SCRATCH_BYTES / 8];  // up and down tables, at most half the area

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Device address of the static area on the current device.  Looked up on
// every call (with that device current): the lookup allocates nothing once
// the module is loaded, and a cached address would go stale if the
// application reset the device and the module were loaded again elsewhere.
// Caller holds g_static_mu.
int static_scratch_address(void** out) {
  void* p = nullptr;
  CUDA_TRY(cudaGetSymbolAddress(&p, g_heom_static_scratch));
  if (!p) return fail(HEOM_ECUDA, "cudaGetSymbolAddress returned NULL for the static area");
  *out = p;
  return HEOM_OK;
}

}  // namespace

extern "C" int heom_propagate_static(const heom_params* params, const double* d_rho0, double dt_fs, int64_t nsteps,
                                     int64_t out_every, double* d_pops, double* d_eta_loss, double* d_rho_out,
                                     void* cuda_stream) {
  TRY(validate(params, 0));
  if (params->N > heom::kMaxSmallN)
    return fail(HEOM_EINVAL, "the allocation-free entry point takes at most %d sites", heom::kMaxSmallN);
  if (params->flags & HEOM_FLAG_SCALED)
    return fail(HEOM_EUNSUPPORTED, "the allocation-free entry point does not take HEOM_FLAG_SCALED");
  if (!d_rho0) return fail(HEOM_EINVAL, "d_rho0 is NULL");
  if (nsteps < 0) return fail(HEOM_EINVAL, "nsteps < 0");
  if (out_every < 1) return fail(HEOM_EINVAL, "out_every must be >= 1");
  if (!(dt_fs > 0.0) || !std::isfinite(dt_fs)) return fail(HEOM_EINVAL, "dt_fs must be > 0");
  const heom_params& p = *params;
  const int N = p.N;
  const bool fp64 = p.precision == HEOM_FP64;
  const size_t rs = fp64 ? sizeof(double) : sizeof(float);
  const int64_t M = heom::num_nodes(N, p.K);
  const int Mpad = (int)((M + 31) / 32 * 32);
  // layout of the static area
  const size_t o_inst = 0;
  const size_t o_team = align256(o_inst + sizeof(Inst));
  const size_t o_status = align256(o_team + 4 * sizeof(int32_t));
  const size_t o_gsync = o_status + 4 * sizeof(int);
  const size_t o_acc = align256(o_gsync + 4 * sizeof(unsigned));
  const size_t o_coef = align256(o_acc + kAccDoubles * sizeof(double));
  const size_t coef_bytes = fp64 ? CoefLayout<double>::bytes(N) : CoefLayout<float>::bytes(N);
  const size_t o_root = align256(o_coef + coef_bytes);
  const size_t o_up = align256(o_root + 3 * 8 * N * N + 32 * heom::kPartBytes);
  const size_t tab_bytes = sizeof(int32_t) * (size_t)N * Mpad;
  const size_t o_dn = align256(o_up + tab_bytes);
  const size_t o_ngam = align256(o_dn + tab_bytes);
  const size_t ngam_bytes = (size_t)Mpad * rs;
  const size_t arr = (size_t)N * N * Mpad * rs;
  const size_t o_y = align256(o_ngam + ngam_bytes);
  const size_t o_wa = align256(o_y + arr);
  const size_t o_wb = align256(o_wa + arr);
  const size_t total = align256(o_wb + arr);
  if (total > HEOM_STATIC_SCRATCH_BYTES)
    return fail(HEOM_EINVAL,
                "N=%d, K=%d (%lld nodes) needs %zu bytes of working memory; the static area holds %u bytes",
                N, p.K, (long long)M, total, (unsigned)HEOM_STATIC_SCRATCH_BYTES);
  if (2 * tab_bytes + ngam_bytes > sizeof(g_static_host_tables))
    return fail(HEOM_EINVAL, "node tables exceed the staging area");

  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  {
    // the host staging below is pageable memory that a captured graph could not
    // replay, and the call waits for its own work: no stream capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(stream, &cs);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      return fail(HEOM_EUNSUPPORTED, "the allocation-free entry point cannot run while a stream capture is active (%s)",
                  cudaGetErrorString(ce));
    }
    if (cs != cudaStreamCaptureStatusNone)
      return fail(HEOM_EUNSUPPORTED, "the allocation-free entry point cannot be captured into a CUDA graph");
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  void* base_v = nullptr;
  TRY(static_scratch_address(&base_v));
  unsigned char* base = static_cast<unsigned char*>(base_v);

  // host staging: tables, coefficients, descriptor (no heap)
  int32_t* h_up = g_static_host_tables;
  int32_t* h_dn = g_static_host_tables + (size_t)N * Mpad;
  if (heom::write_packed_tables(N, p.K, Mpad, h_up, h_dn) != M) return fail(HEOM_EINVAL, "table construction failed");
  // sum_j n_j gamma_j per node, from the packed down links (n_j in the top byte)
  unsigned char* h_ngam = reinterpret_cast<unsigned char*>(h_dn + (size_t)N * Mpad);
  for (int64_t n = 0; n < Mpad; ++n) {
    double v = 0.0;
    for (int j = 0; j < N; ++j) {
      const int32_t dv = h_dn[(size_t)j * Mpad + n];
      if (dv >= 0) v += (dv >> 24) * (p.gamma[j] * kCmToRadPerFs);
    }
    if (fp64)
      reinterpret_cast<double*>(h_ngam)[n] = v;
    else
      reinterpret_cast<float*>(h_ngam)[n] = (float)v;
  }
  alignas(8) unsigned char h_coef[CoefLayout<double>::bytes(heom::kMaxSmallN)];
  int complex_h = 0;
  if (fp64)
    write_coefficients<double>(p, h_coef, &complex_h);
  else
    write_coefficients<float>(p, h_coef, &complex_h);

  Inst d;
  memset(&d, 0, sizeof(d));
  d.N = N;
  d.K = p.K;
  d.M = (int32_t)M;
  d.Mpad = Mpad;
  d.complex_h = complex_h;
  d.terminator = p.terminator;
  d.up = reinterpret_cast<const int32_t*>(base + o_up);
  d.dn = reinterpret_cast<const int32_t*>(base + o_dn);
  d.y = base + o_y;
  d.wa = base + o_wa;
  d.wb = base + o_wb;
  float2* root = reinterpret_cast<float2*>(base + o_root);
  d.y0 = fp64 ? nullptr : root;
  d.w0a = fp64 ? nullptr : root + N * N;
  d.w0b = fp64 ? nullptr : root + 2 * N * N;
  d.parts = base + o_root + 3 * 8 * N * N;
  d.coef = base + o_coef;
  d.ngam = base + o_ngam;
  d.acc = reinterpret_cast<double*>(base + o_acc);
  d.out_pops = d_pops;
  d.out_el = d_eta_loss;
  d.nsteps = nsteps;
  d.out_every = out_every;
  d.dt = dt_fs;
  fill_steps(d, dt_fs, reinterpret_cast<const double*>(h_coef + (fp64 ? CoefLayout<double>::dbl_offset(N)
                                                                       : CoefLayout<float>::dbl_offset(N))));
  const int32_t team[4] = {0, 1, 0, 0};  // team_first = {0, 1}, team_list = {0}

  // one team (a thread-block cluster) for the single hierarchy
  const int block = 256;
  const int G = N >= 4 ? 8 : 2;
  const int64_t units = ((M + 31) / 32) * G;
  int ctas = (int)std::min<int64_t>(16, std::max<int64_t>(1, (units + block / 32 - 1) / (block / 32)));
  int p2 = 1;
  while (p2 < ctas) p2 <<= 1;
  ctas = std::min(16, p2);
  const void* k = heom::engine_kernel(fp64, complex_h != 0, G <= 2, N);
  if (!k) return fail(HEOM_EUNSUPPORTED, "no engine kernel for N=%d", N);
  const int dyn = heom::engine_dyn_bytes(N, block, fp64 ? 8 : 4, G <= 2);
  if (dyn > 0) CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  for (;;) {
    if (ctas > 8) CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    lc = cudaLaunchConfig_t{};
    lc.gridDim = dim3(ctas);
    lc.blockDim = dim3(block);
    lc.dynamicSmemBytes = dyn;
    lc.stream = stream;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int nclusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k, &lc);
    if (e == cudaSuccess && nclusters >= 1) break;
    cudaGetLastError();
    if (ctas == 1) return fail(HEOM_ECUDA, "no resident launch shape for N=%d", N);
    ctas >>= 1;
  }

  // everything that must start at zero: status and barrier words, the state
  CUDA_TRY(cudaMemsetAsync(base + o_status, 0, o_acc - o_status, stream));
  CUDA_TRY(cudaMemsetAsync(base + o_y, 0, arr, stream));
  CUDA_TRY(cudaMemcpyAsync(base + o_coef, h_coef, coef_bytes, cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(base + o_up, h_up, tab_bytes, cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(base + o_dn, h_dn, tab_bytes, cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(base + o_ngam, h_ngam, ngam_bytes, cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(base + o_inst, &d, sizeof(d), cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(base + o_team, team, sizeof(team), cudaMemcpyHostToDevice, stream));
  const int NN = N * N;
  if (fp64)
    set_root_kernel<double><<<launch_blocks(NN, 128), 128, 0, stream>>>(static_cast<double*>(d.y), Mpad, nullptr,
                                                                       d_rho0, N, d.acc);
  else
    set_root_kernel<float><<<launch_blocks(NN, 128), 128, 0, stream>>>(static_cast<float*>(d.y), Mpad,
                                                                      static_cast<float2*>(d.y0), d_rho0, N, d.acc);
  CUDA_TRY(cudaGetLastError());

  EngineArgs A;
  A.insts = reinterpret_cast<const Inst*>(base + o_inst);
  A.team_first = reinterpret_cast<const int32_t*>(base + o_team);
  A.team_list = reinterpret_cast<const int32_t*>(base + o_team) + 2;
  A.G = G;
  A.logG = ilog2(G);
  A.mode = 0;
  A.team_ctas = ctas;
  A.gsync = reinterpret_cast<unsigned*>(base + o_gsync);
  A.status = reinterpret_cast<int*>(base + o_status);
  void* args[] = {&A};
  CUDA_TRY(cudaLaunchKernelExC(&lc, k, args));
  if (d_rho_out) {
    if (fp64)
      unpack_state_kernel<double><<<launch_blocks(NN, 128), 128, 0, stream>>>(static_cast<double*>(d.y), Mpad, 1, N,
                                                                             nullptr, d_rho_out);
    else
      unpack_state_kernel<float><<<launch_blocks(NN, 128), 128, 0, stream>>>(static_cast<float*>(d.y), Mpad, 1, N,
                                                                            static_cast<const float2*>(d.y0),
                                                                            d_rho_out);
    CUDA_TRY(cudaGetLastError());
  }
  // wait for this call's work and report its status word (a non-finite result)
  CUDA_TRY(cudaStreamSynchronize(stream));
  int st = 0;
  CUDA_TRY(cudaMemcpy(&st, base + o_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & heom::kStatusTimeout)
    return fail(HEOM_ETIMEOUT, "a device-side wait expired; the call's results are invalid");
  if (st & heom::kStatusNonFinite)
    return fail(HEOM_ENONFINITE, "the propagation produced a NaN or infinite population, eta or loss");
  if (st) return fail(HEOM_ECUDA, "device status 0x%x", st);
  return HEOM_OK;
}

// ------------------------------------------------------------------ server
//
// Continuous batching of propagation requests of different sizes.  The server
// owns one device buffer (its device-memory budget), one pinned host buffer
// for results, and a few CUDA streams.  Each heom_server_progress() call
//   * marks finished every running request whose done flag the GPU has set
//     (its populations and eta rows are written straight into pinned host
//     memory by the kernel, so they are complete at that point),
//   * retires every launch whose device work has ended (its device memory goes
//     back to the budget, its stream is free), and
//   * admits the queued requests, in arrival order, that fit in the budget into
//     new launches on free streams, one per (precision, N, team shape): one
//     team of CTAs per request, all of them running concurrently with each
//     other and with earlier launches (a launch larger than the GPU holds runs
//     its requests in turn inside the launch).
// So requests that arrive while others run are admitted at the next progress
// call and overlap with them on the device; each request completes on its own
// as soon as its block finishes.  Node tables are cached per (N, K).

namespace {

// First-fit allocator over one contiguous buffer, with coalescing on release.
struct Arena {
  unsigned char* base = nullptr;
  size_t bytes = 0;
  std::map<size_t, size_t> free_blocks;  // offset -> size
  std::map<size_t, size_t> used_blocks;  // offset -> size
  size_t in_use = 0;

  void init(void* b, size_t n) {
    base = static_cast<unsigned char*>(b);
    bytes = n;
    free_blocks.clear();
    used_blocks.clear();
    free_blocks[0] = n;
    in_use = 0;
  }
  void* alloc(size_t n) {
    n = (n + 255) / 256 * 256;
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second < n) continue;
      const size_t off = it->first, sz = it->second;
      free_blocks.erase(it);
      if (sz > n) free_blocks[off + n] = sz - n;
      used_blocks[off] = n;
      in_use += n;
      return base + off;
    }
    return nullptr;
  }
  void release(void* p) {
    if (!p) return;
    const size_t off = static_cast<size_t>(static_cast<unsigned char*>(p) - base);
    auto u = used_blocks.find(off);
    if (u == used_blocks.end()) return;
    size_t start = off, size = u->second;
    in_use -= size;
    used_blocks.erase(u);
    auto next = free_blocks.lower_bound(start);
    if (next != free_blocks.end() && next->first == start + size) {
      size += next->second;
      free_blocks.erase(next);
    }
    auto prev = free_blocks.lower_bound(start);
    if (prev != free_blocks.begin()) {
      --prev;
      if (prev->first + prev->second == start) {
        start = prev->first;
        size += prev->second;
        free_blocks.erase(prev);
      }
    }
    free_blocks[start] = size;
  }
};

void* arena_alloc_hook(size_t n, void* user) { return static_cast<Arena*>(user)->alloc(n); }
void arena_free_hook(void* p, size_t, void* user) { static_cast<Arena*>(user)->release(p); }

enum { kReqQueued = 0, kReqRunning = 1, kReqDone = 2, kReqCancelled = 3, kReqFailed = 4 };

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t id = 0;
  int state = kReqQueued;
  heom_params p;
  std::vector<double> H, lam, gam, trap, recomb, rho0;
  double dt = 1.0;
  int64_t nsteps = 0, out_every = 1, nout = 1;
  size_t need = 0;
  unsigned char* host = nullptr;  // pinned: pops [nout*N], (eta, loss) [nout*2], done flag
  int launch = -1;                // index of the launch running it
  LaunchCfg cfg;                  // launch shape, chosen at admission
  bool released = false;          // released by the caller while its launch still runs
  std::vector<double> pops, el;
  double t_submit = 0, t_start = 0, t_done = 0;
  std::string err;
  int err_code = HEOM_ECUDA;      // code heom_server_result returns for a failed request
  size_t host_bytes() const { return sizeof(double) * (size_t)nout * (p.N + 2) + 64; }
  double* h_pops() const { return reinterpret_cast<double*>(host); }
  double* h_el() const { return reinterpret_cast<double*>(host) + nout * p.N; }
  int* h_done() const { return reinterpret_cast<int*>(host + sizeof(double) * (size_t)nout * (p.N + 2)); }
};

struct Launch {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  std::unique_ptr<Engine> eng;
  std::vector<int64_t> reqs;
  bool busy = false;
};

// Device bytes a request needs, rounded like the arena rounds (tables counted
// when they are not cached yet).
size_t request_bytes(const heom_params& p, bool tables_cached) {
  auto r = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t rs = p.precision == HEOM_FP64 ? 8 : 4;
  const int64_t M = heom::num_nodes(p.N, p.K);
  const size_t Mpad = (size_t)((M + 31) / 32 * 32);
  const size_t NN = (size_t)p.N * p.N;
  size_t coef = rs == 8 ? CoefLayout<double>::bytes(p.N) : CoefLayout<float>::bytes(p.N);
  if (p.flags & HEOM_FLAG_SCALED) coef = (coef + 15) / 16 * 16 + rs * 2 * (size_t)(p.K + 2) * p.N;
  size_t b = 3 * r(NN * Mpad * rs) + r(Mpad * rs) + r(3 * 8 * NN + 32 * heom::kPartBytes) + r(coef) +
             r(kAccDoubles * 8) + r(2 * 8 * NN);
  if (!tables_cached) b += 2 * r(4 * (size_t)p.N * Mpad);
  return b;
}

}  // namespace

struct heom_server {
  std::mutex mu;
  DevBuf dev;
  Arena arena;   // device budget
  void* host_mem = nullptr;
  Arena harena;  // pinned host results
  Hooks hooks;
  std::vector<Launch> launches;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::deque<int64_t> queue;
  int64_t next_id = 1;
  std::shared_ptr<TableCache> tables = std::make_shared<TableCache>();
  int device = 0;

  ~heom_server() {
    for (auto& l : launches)
      if (l.s) cudaStreamSynchronize(l.s);
    for (auto& l : launches) l.eng.reset();  // engines give their blocks back to the arena
    tables.reset();
    for (auto& l : launches) {
      if (l.done) cudaEventDestroy(l.done);
      if (l.s) cudaStreamDestroy(l.s);
    }
    if (host_mem) cudaFreeHost(host_mem);
  }

  // Team of a request: about 256 nodes per CTA (1..16 CTAs), the hierarchy in
  // the team's shared memory when it fits.
  static int team_for(int64_t M) {
    int c = 1;
    while (c < 16 && (int64_t)c * 256 < M) c <<= 1;
    return c;
  }
  // Launch shape of a request.  Scaled hierarchies (N <= 8) take a load view
  // in device memory.  (Smaller teams -- 2 CTAs, or the fewest whose shared
  // memory holds the hierarchy -- were measured slower on the serving trace:
  // the largest requests' service time then sets the makespan.)
  static LaunchCfg launch_for(int prec, int N, int64_t M, int max_dyn, bool scaled) {
    LaunchCfg c;
    c.mode = 0;
    c.team_ctas = team_for(M);
    c.block = prec == HEOM_FP64 ? 256 : 512;
    c.G = 2;
    if (scaled && N <= heom::kMaxSmallN) {
      c.G = std::max(3, std::min(8, N * (N + 1) / 2));
      return c;
    }
    if (prec == HEOM_FP32_MIXED && N <= heom::kMaxSmallN &&
        heom::smem_dyn_bytes(N, Engine::smem_slice(M, c.team_ctas)) <= max_dyn)
      c.mode = 2;
    return c;
  }
  int max_dyn_smem() const {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    return optin - 4096;
  }

  int start_launch(int li, const std::vector<int64_t>& ids) {
    Launch& L = launches[li];
    auto eng = std::make_unique<Engine>();
    eng->pageable_args = true;
    std::vector<heom_params> ps;
    for (int64_t id : ids) ps.push_back(reqs[id]->p);
    int rc = eng->init(ps.data(), (int)ps.size(), L.s, &hooks, tables);
    if (rc != HEOM_OK) return rc;
    // every request of a launch has the same shape (the group key holds it)
    for (auto& in : eng->inst) eng->cfg[in->N] = reqs[ids[0]]->cfg;
    std::vector<double> dts;
    std::vector<int64_t> steps;
    for (size_t k = 0; k < ids.size(); ++k) {
      Request& q = *reqs[ids[k]];
      TRY(eng->set_rho0_host((int)k, q.rho0.data()));
      *q.h_done() = 0;
      eng->ovr_pops.push_back(q.h_pops());
      eng->ovr_el.push_back(q.h_el());
      eng->ovr_done.push_back(q.h_done());
      eng->ovr_every.push_back(q.out_every);
      dts.push_back(q.dt);
      steps.push_back(q.nsteps);
    }
    rc = eng->propagate(dts.data(), steps.data(), 1, nullptr, nullptr);
    if (rc != HEOM_OK) return rc;
    CUDA_TRY(cudaEventRecord(L.done, L.s));
    const double t = now_s();
    for (int64_t id : ids) {
      Request& q = *reqs[id];
      q.state = kReqRunning;
      q.launch = li;
      q.t_start = t;
    }
    L.eng = std::move(eng);
    L.reqs = ids;
    L.busy = true;
    return HEOM_OK;
  }

  // Marks a request whose block has finished: done, or failed when a row of
  // its results is NaN or infinite (a diverging run).
  static void finish_request(Request& q) {
    q.pops.assign(q.h_pops(), q.h_pops() + q.nout * q.p.N);
    q.el.assign(q.h_el(), q.h_el() + 2 * q.nout);
    q.state = kReqDone;
    for (double v : q.pops)
      if (!std::isfinite(v)) q.state = kReqFailed;
    for (double v : q.el)
      if (!std::isfinite(v)) q.state = kReqFailed;
    if (q.state == kReqFailed) {
      q.err = "non-finite populations or eta: the propagation diverged";
      q.err_code = HEOM_ENONFINITE;
    }
  }

  int progress(int32_t* completed) {
    NvtxRange range("heom server progress");
    int done = 0;
    // requests whose block has finished
    for (auto& L : launches) {
      if (!L.busy) continue;
      for (int64_t id : L.reqs) {
        Request& q = *reqs[id];
        if (q.state != kReqRunning) continue;
        if (*reinterpret_cast<volatile int*>(q.h_done()) != 0) {
          finish_request(q);
          q.t_done = now_s();
          ++done;
        }
      }
    }
    // launches whose device work has ended
    for (auto& L : launches) {
      if (!L.busy) continue;
      cudaError_t e = cudaEventQuery(L.done);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) cudaGetLastError();
      for (int64_t id : L.reqs) {
        Request& q = *reqs[id];
        if (q.state == kReqRunning) {
          if (e == cudaSuccess && *reinterpret_cast<volatile int*>(q.h_done()) != 0) {
            // finished between the flag scan above and this event query
            finish_request(q);
          } else {  // the launch ended without the request's flag: it failed
            q.state = kReqFailed;
            q.err = e != cudaSuccess ? cudaGetErrorString(e) : "launch ended before the request finished";
          }
          q.t_done = now_s();
          ++done;
        }
        harena.release(q.host);
        q.host = nullptr;
        q.launch = -1;
      }
      for (int64_t id : L.reqs)
        if (reqs[id]->released) reqs.erase(id);
      L.eng.reset();
      L.reqs.clear();
      L.busy = false;
    }
    // admit queued requests, in arrival order, while they fit in the budget;
    // each launch holds requests of one precision, site count and team shape
    // and takes one free stream.  A request whose group would need a stream
    // when none is left keeps its place in the queue, and later requests that
    // join a group already formed go ahead of it (it gets the next free stream).
    std::vector<int> free_streams;
    for (size_t k = 0; k < launches.size(); ++k)
      if (!launches[k].busy) free_streams.push_back((int)k);
    std::map<std::tuple<int, int, int, int, int>, std::vector<int64_t>> groups;
    std::vector<std::tuple<int, int, int, int, int>> order;
    std::deque<int64_t> skipped;
    if (free_streams.empty()) {
      if (completed) *completed = done;
      return HEOM_OK;
    }
    size_t budget = arena.in_use;
    std::set<std::pair<int, int>> new_tables;
    const int max_dyn = max_dyn_smem();
    while (!queue.empty()) {
      Request& q = *reqs[queue.front()];
      const auto tkey = std::make_pair(q.p.N, q.p.K);
      const bool cached = tables->count(tkey) != 0 || new_tables.count(tkey) != 0;
      const size_t need = request_bytes(q.p, cached) + 8192;
      if (budget + need > arena.bytes) break;
      const int64_t M = heom::num_nodes(q.p.N, q.p.K);
      const bool sc = (q.p.flags & HEOM_FLAG_SCALED) != 0;
      const LaunchCfg c = launch_for(q.p.precision, q.p.N, M, max_dyn, sc);
      const auto gkey = std::make_tuple(q.p.precision, q.p.N, c.team_ctas, c.mode, (int)sc);
      if (!groups.count(gkey)) {
        if (groups.size() == free_streams.size()) {  // no stream for a new group
          skipped.push_back(q.id);
          queue.pop_front();
          continue;
        }
        order.push_back(gkey);
      }
      q.host = static_cast<unsigned char*>(harena.alloc(q.host_bytes()));
      if (!q.host) break;
      q.cfg = c;
      budget += need;
      new_tables.insert(tkey);
      groups[gkey].push_back(q.id);
      queue.pop_front();
    }
    for (auto it = skipped.rbegin(); it != skipped.rend(); ++it) queue.push_front(*it);
    for (size_t g = 0; g < order.size(); ++g) {
      const int li = free_streams[g];
      std::vector<int64_t>& ids = groups[order[g]];
      const int rc = start_launch(li, ids);
      if (rc != HEOM_OK) {
        Launch& L = launches[li];
        L.eng.reset();
        for (auto it = ids.rbegin(); it != ids.rend(); ++it) {
          Request& q = *reqs[*it];
          harena.release(q.host);
          q.host = nullptr;
          if (rc == HEOM_ENOMEM) {
            queue.push_front(*it);
          } else {
            q.state = kReqFailed;
            q.err = t_err;
          }
        }
      }
    }
    if (completed) *completed = done;
    return HEOM_OK;
  }
};

extern "C" {

int heom_server_create(size_t device_bytes, size_t host_bytes, int32_t streams, heom_server** out) {
  if (!out) return fail(HEOM_EINVAL, "out is NULL");
  *out = nullptr;
  if (streams < 1 || streams > 64) return fail(HEOM_EINVAL, "streams must be 1..64");
  if (device_bytes < (1u << 20)) return fail(HEOM_EINVAL, "device_bytes must be at least 1 MiB");
  if (host_bytes < (1u << 16)) return fail(HEOM_EINVAL, "host_bytes must be at least 64 KiB");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(HEOM_ECUDA, "no usable CUDA device (%s)", cudaGetErrorString(e));
  }
  auto s = std::make_unique<heom_server>();
  CUDA_TRY(cudaGetDevice(&s->device));
  TRY(s->dev.alloc(device_bytes, Hooks()));
  s->arena.init(s->dev.p, s->dev.bytes);
  CUDA_TRY(cudaHostAlloc(&s->host_mem, host_bytes, cudaHostAllocMapped | cudaHostAllocPortable));
  s->harena.init(s->host_mem, host_bytes);
  s->hooks.alloc = arena_alloc_hook;
  s->hooks.release = arena_free_hook;
  s->hooks.user = &s->arena;
  s->launches.resize(streams);
  for (auto& l : s->launches) {
    CUDA_TRY(cudaStreamCreateWithFlags(&l.s, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming));
  }
  *out = s.release();
  return HEOM_OK;
}

void heom_server_destroy(heom_server* s) { delete s; }

int heom_server_submit(heom_server* s, const heom_params* params, const double* rho0, double dt_fs, int64_t nsteps,
                       int64_t out_every, int64_t* request_id) {
  if (!s || !request_id) return fail(HEOM_EINVAL, "server or request_id is NULL");
  TRY(validate(params, 0));
  if (params->N > heom::kMaxSmallN) return fail(HEOM_EUNSUPPORTED, "the server takes at most %d sites", heom::kMaxSmallN);
  TRY(validate_rho(rho0, params->N));
  if (nsteps < 0) return fail(HEOM_EINVAL, "nsteps < 0");
  if (out_every < 1) return fail(HEOM_EINVAL, "out_every must be >= 1");
  if (!(dt_fs > 0.0) || !std::isfinite(dt_fs)) return fail(HEOM_EINVAL, "dt_fs must be > 0");
  std::lock_guard<std::mutex> lk(s->mu);
  auto q = std::make_unique<Request>();
  const int N = params->N;
  q->p = *params;
  q->H.assign(params->H, params->H + 2 * N * N);
  q->lam.assign(params->lambda, params->lambda + N);
  q->gam.assign(params->gamma, params->gamma + N);
  if (params->trap_rate) q->trap.assign(params->trap_rate, params->trap_rate + N);
  if (params->recomb_rate) q->recomb.assign(params->recomb_rate, params->recomb_rate + N);
  q->p.H = q->H.data();
  q->p.lambda = q->lam.data();
  q->p.gamma = q->gam.data();
  q->p.trap_rate = params->trap_rate ? q->trap.data() : nullptr;
  q->p.recomb_rate = params->recomb_rate ? q->recomb.data() : nullptr;
  q->rho0.assign(rho0, rho0 + 2 * N * N);
  q->dt = dt_fs;
  q->nsteps = nsteps;
  q->out_every = out_every;
  q->nout = nsteps / out_every + 1;
  q->need = request_bytes(q->p, false) + 8192;
  if (q->need > s->arena.bytes)
    return fail(HEOM_ENOMEM, "request needs %zu device bytes; the server's budget is %zu", q->need, s->arena.bytes);
  if (q->host_bytes() > s->harena.bytes)
    return fail(HEOM_ENOMEM, "request needs %zu bytes of pinned host memory for its results; the server has %zu",
                q->host_bytes(), s->harena.bytes);
  q->id = s->next_id++;
  q->t_submit = now_s();
  *request_id = q->id;
  s->queue.push_back(q->id);
  s->reqs[q->id] = std::move(q);
  return HEOM_OK;
}

int heom_server_progress(heom_server* s, int32_t* completed) {
  if (!s) return fail(HEOM_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != s->device) CUDA_TRY(cudaSetDevice(s->device));
  return s->progress(completed);
}

int heom_server_status(heom_server* s, int64_t id, int32_t* state) {
  if (!s || !state) return fail(HEOM_EINVAL, "server or state is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second->released) return fail(HEOM_EINVAL, "unknown request %lld", (long long)id);
  *state = it->second->state;
  return HEOM_OK;
}

int heom_server_result(heom_server* s, int64_t id, double* pops_out, double* eta_out, double* loss_out,
                       double* times_out) {
  if (!s) return fail(HEOM_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(HEOM_EINVAL, "unknown request %lld", (long long)id);
  Request& q = *it->second;
  if (q.state == kReqFailed) return fail(q.err_code, "request %lld failed: %s", (long long)id, q.err.c_str());
  if (q.state != kReqDone) return fail(HEOM_EINVAL, "request %lld is not finished", (long long)id);
  if (pops_out) memcpy(pops_out, q.pops.data(), sizeof(double) * q.pops.size());
  for (int64_t o = 0; o < q.nout; ++o) {
    if (eta_out) eta_out[o] = q.el[2 * o];
    if (loss_out) loss_out[o] = q.el[2 * o + 1];
  }
  if (times_out) {
    times_out[0] = q.t_start - q.t_submit;
    times_out[1] = q.t_done - q.t_submit;
  }
  return HEOM_OK;
}

int heom_server_release(heom_server* s, int64_t id) {
  if (!s) return fail(HEOM_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second->released) return fail(HEOM_EINVAL, "unknown request %lld", (long long)id);
  const int st = it->second->state;
  if (st == kReqQueued || st == kReqRunning) return fail(HEOM_EINVAL, "request %lld is still active", (long long)id);
  if (it->second->host) {
    it->second->released = true;  // its launch still runs; forgotten when the launch retires
  } else {
    s->reqs.erase(it);
  }
  return HEOM_OK;
}

int heom_server_cancel(heom_server* s, int64_t id) {
  if (!s) return fail(HEOM_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(HEOM_EINVAL, "unknown request %lld", (long long)id);
  if (it->second->state != kReqQueued)
    return fail(HEOM_EINVAL, "request %lld is not queued (only queued requests can be cancelled)", (long long)id);
  it->second->state = kReqCancelled;
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (*q == id) {
      s->queue.erase(q);
      break;
    }
  return HEOM_OK;
}

int heom_server_stats(heom_server* s, int64_t* queued, int64_t* running, int64_t* bytes_in_use) {
  if (!s) return fail(HEOM_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t r = 0;
  for (auto& kv : s->reqs)
    if (kv.second->state == kReqRunning) ++r;
  if (queued) *queued = (int64_t)s->queue.size();
  if (running) *running = r;
  if (bytes_in_use) *bytes_in_use = (int64_t)s->arena.in_use;
  return HEOM_OK;
}

}  // extern "C"
