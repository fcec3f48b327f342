// heom_flow.cuh -- the dataflow engine for one hierarchy with N <= 8 sites
// (launch mode 3): the whole GPU, no grid-wide barrier.
//
// Method: the same right-hand side and Horner-form RK4 as heom_engine.cuh
// (App. A2 Eqs. labsevena/lab8, App. A1, App. B), with trapping as the
// anti-Hermitian part of H_eff.
//
// Decomposition.  CTA c owns the SL = S * NPT consecutive nodes
// [c*SL, c*SL + SL) and keeps their three stage arrays (y, wa, wb) in shared
// memory for the whole call, node-major: element p of local node l at
// l*N*N + p.  Thread (u, l) of the CTA computes unit u (an off-diagonal pair
// (a, b), two packed reals, or a diagonal a) of the local nodes k*S + l,
// k = 0..NPT-1, in every stage (NPT nodes per thread, 1 by default).  The part of a unit's right-hand side
// that involves its own node -- the commutator with H_eff, the site-energy
// differences, the trap/decay and low-temperature damping -- is a fixed
// linear form in at most NRE (real part) and NIM (imaginary part) packed
// elements of the node; the host evaluates it once per unit and the thread
// keeps the nonzero coefficients and element indices in registers.  The
// node-dependent parts (the hierarchy damping -sum_j n_j gamma_j, the
// terminator at the last level, the up and down link weights, including the
// scaled hierarchy's) are folded into the same registers at the start of the
// call.  A stage is then a short sparse dot product over shared memory plus
// at most four neighbour pairs.
//
// Exchange.  Neighbour values go through global memory as 64-bit words that
// carry the stage they belong to: (tag << 32 | float bits) in FP32, two such
// words (low and high halves of the double) in FP64.  A thread gathers the
// words of its links n +- e_a, n +- e_b and waits (bounded) until every tag is
// the one of the previous stage, so it waits exactly for the values it reads,
// and no flag, fence or barrier crosses CTAs.  The dependence is symmetric
// (unit (a, b) of n reads element (a, b) of n +- e_a, n +- e_b, and unit (a, b)
// of each of those reads element (a, b) of n), so a writer of stage s + 1 has
// always seen every reader of its stage-s value finish: three tagged buffers
// (y, wa, wb) in the Horner rotation are enough.  Diagonal units also wait on
// their up link, whose weight is zero, to keep that symmetry.  Within a CTA
// the stages are separated by __syncthreads.
//
// Tags: the call starts at tag0; the initial y carries tag0 + 1 and the output
// of step t, stage s carries tag0 + 4t + s + 2, so stage s of step t waits for
// tag0 + 4t + s + 1.  The host advances tag0 by 4 nsteps + 2 per call and
// clears the buffers before the 32-bit tags would wrap, so a stale word never
// carries an expected tag.
#pragma once

#include "heom_engine.cuh"

namespace heom {

constexpr int kFlowMaxE = 28;   // 4N - 4 at N = 8
constexpr int kFlowRing = 64;   // stop-rule decisions kept in flight
// Threads per CTA the kernels are compiled for: at most 168 registers a thread,
// so that a CTA of 13 nodes at N = 7 (364 threads) fits one SM; real-H kernels
// do not spill at this budget.
constexpr int kFlowMaxThreads = 384;
// Threads per CTA of the kernels whose threads carry several nodes (NPT > 1):
// eight warps, two per SM sub-partition, so that a thread may hold 255
// registers (with ten or twelve warps some sub-partition holds three, and its
// register file allows 168).
constexpr int kFlowMaxThreadsMulti = 256;
constexpr int kFlowMaxNpt = 6;

// One unit's own-node linear form (host-built).  Slot 0 of both lists is the
// unit's own real element x = P[a*N + b]; for a pair, slot 1 is its imaginary
// element yi = P[b*N + a] (the node-dependent terms are added to these two
// slots); the other slots hold the remaining elements with a nonzero weight,
// and unused slots have weight 0.
struct FlowUnit {
  uint8_t ire[kFlowMaxE];
  uint8_t iim[kFlowMaxE];
  uint8_t a, b, pad[6];
  double cre[kFlowMaxE];
  double cim[kFlowMaxE];
};
// Per-site bath data in double (host-built, after the units).
struct FlowSite {
  double alpha, beta, gamma, scale;  // 2 lambda k_B T, lambda gamma, gamma, s_j of the scaled hierarchy
};

struct FlowArgs {
  const Inst* inst;                  // the one instance
  const FlowUnit* units;             // [U] then FlowSite[N]
  unsigned long long* tags;          // tagged y, wa, wb, one after the other: [N*N][Mpad] words each
                                     // (FP64: pairs of words)
  long long tag_stride;              // words from one tagged buffer to the next
  unsigned long long* ring;          // [kFlowRing] stop decisions
  int* status;
  int S;                             // nodes per CTA
  unsigned tag0;
};

__host__ __device__ constexpr int flow_nre(int N, bool cplx) {
  return (cplx ? 4 * N - 4 : 2 * N - 2) < 2 ? 2 : (cplx ? 4 * N - 4 : 2 * N - 2);
}
__host__ __device__ constexpr int flow_nim(int N, bool cplx) {
  return (cplx ? 4 * N - 4 : 2 * N) < 2 ? 2 : (cplx ? 4 * N - 4 : 2 * N);
}
// Dynamic shared memory of a CTA whose slice holds S nodes.
__host__ __device__ constexpr int flow_smem_bytes(int N, int S, int rsize) { return 3 * S * N * N * rsize; }

// ------------------------------------------------------------ tagged words

__device__ __forceinline__ void flow_store(unsigned long long* p, float v, unsigned tag) {
  const unsigned long long w = ((unsigned long long)tag << 32) | __float_as_uint(v);
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w));
}
__device__ __forceinline__ void flow_store(unsigned long long* p, double v, unsigned tag) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned long long t = (unsigned long long)tag << 32;
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(t | (b & 0xFFFFFFFFull)),
               "l"(t | (b >> 32)));
}

// A gathered word (FP32) or pair of words (FP64) and its check.
template <typename R>
struct FlowWord;
template <>
struct FlowWord<float> {
  unsigned long long w = 0;
  __device__ __forceinline__ void load(const unsigned long long* p) {
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p));
  }
  __device__ __forceinline__ bool ok(unsigned tag) const { return (unsigned)(w >> 32) == tag; }
  __device__ __forceinline__ float value() const { return __uint_as_float((unsigned)w); }
};
template <>
struct FlowWord<double> {
  unsigned long long lo = 0, hi = 0;
  __device__ __forceinline__ void load(const unsigned long long* p) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "l"(p));
  }
  __device__ __forceinline__ bool ok(unsigned tag) const {
    return (unsigned)(lo >> 32) == tag && (unsigned)(hi >> 32) == tag;
  }
  __device__ __forceinline__ double value() const {
    return __hiloint2double((int)(unsigned)hi, (int)(unsigned)lo);
  }
};
template <typename R>
__host__ __device__ constexpr int flow_words() {
  return sizeof(R) == 8 ? 2 : 1;
}

// The eta and loss row `row` from the diagonal owners' running sums in shared
// memory (the same sums, in the same order, as eta_total reads from the parts
// slots), and the check of the row for NaN or infinity; the population row
// is the root's diagonal of the step's y, also in shared memory.
template <typename R, bool MIXED>
__device__ __forceinline__ void flow_eta_row(const Inst& I, const EtaAcc<R>* ea, const FF* trace_ff,
                                             const double* trace_d, int N, double acc0, double acc1, int64_t row,
                                             int* status) {
  double e, l;
  if constexpr (sizeof(R) == 4) {
    FF se{0.f, 0.f}, sl{0.f, 0.f};
    for (int k = 0; k < N; ++k) {
      se = ff_add(se, ea[k].e);
      sl = ff_add(sl, ea[k].l);
    }
    e = acc0 + ff_to_double(se);
    l = acc1 + ff_to_double(sl);
  } else {
    double se = 0.0, sl = 0.0;
    for (int k = 0; k < N; ++k) {
      se += ea[k].e;
      sl += ea[k].l;
    }
    e = acc0 + se;
    l = acc1 + sl;
  }
  flag_nonfinite(status, e);
  flag_nonfinite(status, l);
  for (int k = 0; k < N; ++k) flag_nonfinite(status, MIXED ? ff_to_double(trace_ff[k]) : trace_d[k]);
  if (!I.out_el) return;
  I.out_el[2 * row] = e;
  I.out_el[2 * row + 1] = l;
}

// ------------------------------------------------------------------ kernel
//
// NPT nodes per thread: thread (u, l) of CTA c computes unit u of the nodes
// c*S*NPT + k*S + l, k = 0..NPT-1 (the lanes of a warp stay consecutive nodes
// of one unit for every k, so the exchange keeps its coalescing).  A thread
// first runs the own-node parts and issues the gathers of all its nodes
// (independent chains the compiler interleaves), then waits for and updates
// them node by node, so one exchange latency covers all of its nodes.
// NPT = 1 runs the steps in the same order as a plain one-node-per-thread
// kernel.
template <int N, typename R, bool MIXED, bool CPLX, int NPT = 1>
__global__ void __launch_bounds__(NPT == 1 ? kFlowMaxThreads : kFlowMaxThreadsMulti) heom_flow_kernel(FlowArgs A) {
  constexpr int NN = N * N;
  constexpr int NP = N * (N - 1) / 2;
  constexpr int U = NP + N;
  constexpr int NRE = flow_nre(N, CPLX);
  constexpr int NIM = flow_nim(N, CPLX);
  constexpr int WD = flow_words<R>();
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ Inst s_inst;
  __shared__ int s_abort, s_stop;
  // the root node (CTA 0, local node 0): float-float y and stage outputs of the
  // mixed path, and the eta/loss/xi running sums of its diagonal owners
  __shared__ FF s_ry[kMaxSmallN * kMaxSmallN], s_rw[kMaxSmallN];
  __shared__ EtaAcc<R> s_ea[kMaxSmallN];
  __shared__ FF s_trace_ff[kMaxSmallN];
  __shared__ double s_trace_d[kMaxSmallN];

  const int S = A.S;        // threads per unit: nodes of one row of the slice
  const int SL = S * NPT;   // nodes of the CTA's slice
  const int u = threadIdx.x / S;
  const int l = threadIdx.x - u * S;
  if (threadIdx.x == 0) {
    s_inst = *A.inst;
    s_abort = 0;
    s_stop = 0;
  }
  __syncthreads();
  const Inst& I = s_inst;
  const int M = I.M, Mp = I.Mpad;
  int nd[NPT];
  bool valid[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    nd[k] = blockIdx.x * SL + k * S + l;
    valid[k] = u < U && nd[k] < M;
  }
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  R* const sb = reinterpret_cast<R*>(dsm);  // stage buffer k at sb + k * SL * NN

  // ---- the thread's unit and its linear form (shared by its nodes); per node
  // the slots 0 and 1 of both forms (where the node's damping and terminator
  // enter), the links and the link weights
  int a = 0, b = 0, pab = 0, pba = 0;
  uint32_t ire4[(NRE + 3) / 4], iim4[(NIM + 3) / 4];
  R cre[NRE], cim[NIM];
  R c0r[NPT], c1r[NPT], c0i[NPT], c1i[NPT];
  int hl[NPT][4];  // up a, up b, down a, down b
  R cu_a[NPT], cu_b[NPT], pd_a[NPT], qd_a[NPT], pd_b[NPT], qd_b[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    c0r[k] = c1r[k] = c0i[k] = c1i[k] = R(0);
    cu_a[k] = cu_b[k] = pd_a[k] = qd_a[k] = pd_b[k] = qd_b[k] = R(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) hl[k][j] = -1;
  }
  const bool root = valid[0] && nd[0] == 0;  // only node 0 of a thread can be the root
  if (valid[0]) {
    const FlowUnit& fu = A.units[u];
    const FlowSite* fs = reinterpret_cast<const FlowSite*>(A.units + U);
    a = fu.a;
    b = fu.b;
    pab = a * N + b;
    pba = b * N + a;
#pragma unroll
    for (int i = 0; i < (NRE + 3) / 4; ++i) {
      uint32_t w = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (4 * i + k < NRE) w |= (uint32_t)fu.ire[4 * i + k] << (8 * k);
      ire4[i] = w;
    }
#pragma unroll
    for (int i = 0; i < (NIM + 3) / 4; ++i) {
      uint32_t w = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (4 * i + k < NIM) w |= (uint32_t)fu.iim[4 * i + k] << (8 * k);
      iim4[i] = w;
    }
    double dre[NRE], dim[NIM];
#pragma unroll
    for (int i = 0; i < NRE; ++i) dre[i] = fu.cre[i];
#pragma unroll
    for (int i = 0; i < NIM; ++i) dim[i] = fu.cim[i];
#pragma unroll
    for (int i = 0; i < NRE; ++i) cre[i] = (R)dre[i];
#pragma unroll
    for (int i = 0; i < NIM; ++i) cim[i] = (R)dim[i];
    const FlowSite sa = fs[a], sbs = fs[b];
    const bool scaled = I.wsc != nullptr;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      if (!valid[k]) continue;
      const int n = nd[k];
      // node data: links, n_a, n_b, sum_j n_j gamma_j, last level
      const int ra = I.dn[a * Mp + n], rb = I.dn[b * Mp + n];
      const int ua = I.up[a * Mp + n], ub = I.up[b * Mp + n];
      const double na = ra < 0 ? 0.0 : (double)(ra >> 24), nb = rb < 0 ? 0.0 : (double)(rb >> 24);
      const double ng = (double)static_cast<const R*>(I.ngam)[n];
      const bool leaf = I.up[n] < 0;
      double x0r = dre[0], x1r = dre[1], x0i = dim[0], x1i = dim[1];
      x0r -= ng;  // hierarchy damping -sum_j n_j gamma_j on x (and on yi below)
      if (a != b) {
        x1i -= ng;
        if (I.terminator && leaf) {
          // sigma_{n+e_j} ~ (n_j+1)/(ngam+gamma_j) theta_j sigma_n, then i V_j^x of it (j = a, b)
          const double ca = (na + 1.0) / (ng + sa.gamma), cb = (nb + 1.0) / (ng + sbs.gamma);
          x0r += -ca * sa.alpha - cb * sbs.alpha;
          x1r += -ca * sa.beta + cb * sbs.beta;
          x0i += ca * sa.beta - cb * sbs.beta;
          x1i += -ca * sa.alpha - cb * sbs.alpha;
        }
        // up links i V_j^x sigma_{n+e_j}: re += cu Im(up), im -= cu Re(up); weight 1, or
        // sqrt((n_j+1) s_j) in the scaled hierarchy
        hl[k][0] = ua;
        hl[k][1] = ub;
        cu_a[k] = (R)(-(scaled ? sqrt((na + 1.0) * sa.scale) : 1.0));
        cu_b[k] = (R)(scaled ? sqrt((nb + 1.0) * sbs.scale) : 1.0);
        // down links n_j theta_j sigma_{n-e_j}: re += p Re - q Im, im += q Re + p Im
        hl[k][2] = ra < 0 ? -1 : (ra & 0xFFFFFF);
        hl[k][3] = rb < 0 ? -1 : (rb & 0xFFFFFF);
        const double wa = scaled ? sqrt(na / sa.scale) : na, wb = scaled ? sqrt(nb / sbs.scale) : nb;
        pd_a[k] = (R)(wa * sa.beta);
        qd_a[k] = (R)(wa * sa.alpha);
        pd_b[k] = (R)(wb * sbs.beta);
        qd_b[k] = (R)(-wb * sbs.alpha);
      } else {
        // the up link carries no weight for a diagonal; it is still waited on (see above)
        hl[k][0] = ua;
        hl[k][2] = ra < 0 ? -1 : (ra & 0xFFFFFF);
        const double wa = scaled ? sqrt(na / sa.scale) : na;
        pd_a[k] = (R)(2.0 * wa * sa.beta);
      }
      c0r[k] = (R)x0r;
      c1r[k] = (R)x1r;
      c0i[k] = (R)x0i;
      c1i[k] = (R)x1i;
    }
  }
  const bool pair = a != b;

  // ---- the state: own elements in registers (the Horner base), slice in shared memory
  R y_r[NPT], y_i[NPT];
  const R* gy = static_cast<const R*>(I.y);
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    y_r[k] = y_i[k] = R(0);
    if (!valid[k]) continue;
    const int oab = pab * Mp + nd[k], oba = pba * Mp + nd[k];
    y_r[k] = gy[oab];
    y_i[k] = pair ? gy[oba] : R(0);
    R* own = sb + (k * S + l) * NN;
    own[pab] = y_r[k];
    if (pair) own[pba] = y_i[k];
    flow_store(A.tags + WD * oab, y_r[k], A.tag0 + 1);
    if (pair) flow_store(A.tags + WD * oba, y_i[k], A.tag0 + 1);
  }
  if constexpr (MIXED) {
    if (root) {
      const FF* y0 = static_cast<const FF*>(I.y0);
      s_ry[pab] = y0[pab];
      if (pair) s_ry[pba] = y0[pba];
    }
  }
  if (root && !pair) s_ea[a] = EtaAcc<R>{};
  EtaRows rows;
  rows.acc0 = I.acc[0];
  rows.acc1 = I.acc[1];
  const bool diag_root = root && !pair;  // owner of the root's diagonal a: eta slot a, sums in s_ea[a]
  const double* cfd = reinterpret_cast<const double*>(static_cast<const unsigned char*>(I.coef) +
                                                      CoefLayout<R>::dbl_offset(N));
  if (lead) {
    write_row0<N, R, MIXED>(I);
    const EtaAcc<R> zero{};
    for (int k = 0; k < N; ++k) zero.store(I, k);  // zero every running-sum slot
  }
  __syncthreads();

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
        if (lead) flow_eta_row<R, MIXED>(I, s_ea, s_trace_ff, s_trace_d, N, rows.acc0, rows.acc1, rows.pending, A.status);
        rows.pending = -1;
      }
      const int in_sel = (s == 0) ? 0 : (s == 2 ? 2 : 1);
      const int out_sel = (s == 1) ? 2 : (s == 3 ? 0 : 1);
      const unsigned want = A.tag0 + 4u * (unsigned)t + (unsigned)s + 1u;
      const unsigned long long* tin = A.tags + in_sel * A.tag_stride;
      R re[NPT], im[NPT];
      FlowWord<R> gr[NPT][4], gi[NPT][4];
      bool aborted = false;
      // the own-node part (shared memory), then the neighbours: by the time the
      // gathers reach L2 their producers have mostly stored (measured: equal in
      // FP32, 15 % faster in FP64 than gathering first)
      auto own_and_gather = [&](auto kc) {
        constexpr int k = decltype(kc)::value;
        re[k] = R(0);
        im[k] = R(0);
        if (!valid[k]) return;
        const R* sin = sb + in_sel * SL * NN + (k * S + l) * NN;
#pragma unroll
        for (int i = 0; i < NRE; ++i)
          re[k] += (i == 0 ? c0r[k] : (i == 1 ? c1r[k] : cre[i])) * sin[(ire4[i / 4] >> (8 * (i % 4))) & 0xFF];
        if (pair) {  // a diagonal has no imaginary part; its units fill the last warps of a CTA
#pragma unroll
          for (int i = 0; i < NIM; ++i)
            im[k] += (i == 0 ? c0i[k] : (i == 1 ? c1i[k] : cim[i])) * sin[(iim4[i / 4] >> (8 * (i % 4))) & 0xFF];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (hl[k][j] >= 0) {
            gr[k][j].load(tin + WD * (pab * Mp + hl[k][j]));
            gi[k][j].load(tin + WD * (pba * Mp + hl[k][j]));
          }
      };
      // wait, bounded, until every gathered word of node k carries the previous stage's tag
      auto wait_words = [&](auto kc) -> bool {
        constexpr int k = decltype(kc)::value;
        bool ready = true;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (hl[k][j] >= 0) ready = ready & gr[k][j].ok(want) & gi[k][j].ok(want);
        if (ready) return true;
        uint64_t t0 = 0;
        for (unsigned spins = 1;; ++spins) {
          // reload every word that is not there yet, then check them all
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (hl[k][j] >= 0) {
              if (!gr[k][j].ok(want)) gr[k][j].load(tin + WD * (pab * Mp + hl[k][j]));
              if (!gi[k][j].ok(want)) gi[k][j].load(tin + WD * (pba * Mp + hl[k][j]));
            }
          ready = true;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (hl[k][j] >= 0) ready = ready & gr[k][j].ok(want) & gi[k][j].ok(want);
          if (ready) return true;
          if ((spins & 255u) == 0) {
            if (ld_volatile(A.status) & kStatusTimeout) {
              s_abort = 1;
              return false;
            }
            const uint64_t now = global_timer_ns();
            if (t0 == 0) {
              t0 = now;
            } else if (now - t0 > kBarrierLimitNs) {
              atomicOr(A.status, kStatusTimeout);
              s_abort = 1;
              return false;
            }
          }
        }
      };
      // the neighbour terms, the Horner update and the stores of node k
      auto finish = [&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const R ur = gr[k][0].value(), ui = gi[k][0].value(), vr = gr[k][1].value(), vi = gi[k][1].value();
        const R dr = gr[k][2].value(), di = gi[k][2].value(), er = gr[k][3].value(), ei = gi[k][3].value();
        // absent links were never loaded and read as 0
        R rr = re[k], mm = im[k];
        rr += cu_a[k] * ui + cu_b[k] * vi + pd_a[k] * dr - qd_a[k] * di + pd_b[k] * er - qd_b[k] * ei;
        mm += -cu_a[k] * ur - cu_b[k] * vr + qd_a[k] * dr + pd_a[k] * di + qd_b[k] * er + pd_b[k] * ei;
        R w_r, w_i;
        const unsigned tag_out = want + 1u;
        const bool rt = k == 0 && root;
        if (MIXED && rt) {
          if constexpr (MIXED) {
            const float hh = I.hh[s], hlo = I.hl[s];
            if (!pair) {
              // eta, loss and xi rows of the augmented system: the float-float stage input
              if (s == 3) s_ea[a].add(I, a, s_rw[a]);
              if (s == 2) s_ea[a].add_xi(I, a, s_rw[a]);
            }
            const FF fr = ff_axpy(s_ry[pab], hh, hlo, rr);
            const FF fi = pair ? ff_axpy(s_ry[pba], hh, hlo, mm) : FF{0.f, 0.f};
            w_r = fr.h;
            w_i = fi.h;
            if (!pair) s_rw[a] = fr;
            if (s == 3) {
              s_ry[pab] = fr;
              if (pair) s_ry[pba] = fi;
              if (!pair && os.now && I.out_pops) I.out_pops[os.row * N + a] = ff_to_double(fr);
            }
          }
        } else {
          if constexpr (!MIXED) {
            if (rt && !pair) {
              const R* sin = sb + in_sel * SL * NN + (k * S + l) * NN;
              if (s == 3) s_ea[a].add(I, cfd, N, a, (double)sin[pab]);
              if (s == 2) s_ea[a].add_xi(I, cfd, a, (double)sin[pab]);
            }
          }
          const R h = sizeof(R) == 8 ? (R)I.hd[s] : (R)I.hh[s];
          w_r = y_r[k] + h * rr;
          w_i = y_i[k] + h * mm;
          if (s == 3 && rt && !pair && os.now && I.out_pops) I.out_pops[os.row * N + a] = (double)w_r;
        }
        R* sout = sb + out_sel * SL * NN + (k * S + l) * NN;
        unsigned long long* tout = A.tags + out_sel * A.tag_stride;
        const int oab = pab * Mp + nd[k], oba = pba * Mp + nd[k];
        sout[pab] = w_r;
        flow_store(tout + WD * oab, w_r, tag_out);
        if (pair) {
          sout[pba] = w_i;
          flow_store(tout + WD * oba, w_i, tag_out);
        }
        if (s == 3) {
          y_r[k] = w_r;
          y_i[k] = w_i;
        }
        if (k == 0 && diag_root) {
          if (s == 2) s_ea[a].step_xi(I);
          if (s == 3) {
            if (os.now || t + 1 == I.nsteps) s_ea[a].store(I, a);
            if constexpr (MIXED) s_trace_ff[a] = s_ry[pab];
            else s_trace_d[a] = (double)w_r;
          }
        }
      };
      // every node's own-node part and gathers first (independent chains the
      // compiler interleaves), then the waits and updates node by node
      static_for<0, NPT>([&](auto kc) { own_and_gather(kc); });
      static_for<0, NPT>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if (valid[k] && !aborted) {
          if (wait_words(kc)) finish(kc);
          else aborted = true;
        }
      });
      __syncthreads();
      if (s_abort) return;
    }
    if (os.now) rows.pending = os.row;
    if (I.stop_trace > 0.0 && t + 1 < I.nsteps) {
      // the stop rule: CTA 0 holds the root and decides; every CTA waits for the decision of this step
      const unsigned dtag = A.tag0 + (unsigned)t + 1u;
      unsigned long long* slot = A.ring + (t % kFlowRing);
      if (threadIdx.x == 0) {
        if (blockIdx.x == 0) {
          double tr = 0.0;
          if constexpr (MIXED) {
            FF sum{0.f, 0.f};
            for (int k = 0; k < N; ++k) sum = ff_add(sum, s_trace_ff[k]);
            tr = ff_to_double(sum);
          } else {
            for (int k = 0; k < N; ++k) tr += s_trace_d[k];
          }
          const unsigned long long w = ((unsigned long long)dtag << 32) | (tr < I.stop_trace ? 1ull : 0ull);
          asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(slot), "l"(w));
          s_stop = (int)(w & 1ull);
        } else {
          unsigned long long w = 0;
          uint64_t t0 = 0;
          for (unsigned spins = 1;; ++spins) {
            asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(slot));
            if ((unsigned)(w >> 32) == dtag) break;
            if ((spins & 255u) == 0) {
              if (ld_volatile(A.status) & kStatusTimeout) {
                s_abort = 1;
                break;
              }
              const uint64_t now = global_timer_ns();
              if (t0 == 0) {
                t0 = now;
              } else if (now - t0 > kBarrierLimitNs) {
                atomicOr(A.status, kStatusTimeout);
                s_abort = 1;
                break;
              }
            }
          }
          s_stop = (int)(w & 1ull);
        }
      }
      __syncthreads();
      if (s_abort) return;
      if (s_stop) {
        if (diag_root) s_ea[a].store(I, a);
        done = t + 1;
        break;
      }
    }
  }
  // the state back to device memory (packed, element-major; the root also in float-float)
  R* gyw = static_cast<R*>(I.y);
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    if (!valid[k]) continue;
    gyw[pab * Mp + nd[k]] = y_r[k];
    if (pair) gyw[pba * Mp + nd[k]] = y_i[k];
  }
  if constexpr (MIXED) {
    if (root) {
      FF* y0 = static_cast<FF*>(I.y0);
      y0[pab] = s_ry[pab];
      if (pair) y0[pba] = s_ry[pba];
    }
  }
  __syncthreads();
  if (lead) finish_instance<R>(I, N, rows, done, orow, N, A.status);
}

}  // namespace heom
