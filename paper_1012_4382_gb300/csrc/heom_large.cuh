// Large-N engine of the HEOM RK4 propagation (9..24 sites): see the comment
// below.  Shares the descriptors, coefficient layout, barriers, eta sums and
// stop rule of heom_engine.cuh.
#pragma once

#include "heom_engine.cuh"

namespace heom {

// ------------------------------------------------------------ large-N engine
//
// Hierarchies with 9..24 sites (N is a run-time argument).  A CTA stages a
// tile of 16 consecutive nodes' matrices in shared memory, element-major with
// the 16 nodes innermost; two lanes share a node (lane = 2 x node + half), so
// a warp covers the 16 nodes and every shared-memory access is free of bank
// conflicts (the two lanes of a node read the same word).  The node's outputs
// are cut into 4 x 4 blocks (a in A, b in B, A <= B, the upper triangle);
// warp w computes blocks w, w + nwarps, ... of all 16 nodes, each lane two
// rows of a block.  Within a block the commutator is a small matrix product:
// for each k the thread reads sigma_ak for its two rows and sigma_kb for the
// four columns, row k of J, and does 32 multiply-adds.  Neighbours are read
// from device memory.  Teams and barriers are those of the small-N engine.
//
// FP32 keeps Re sigma and Im sigma in the tile as full, zero-padded
// 4 ceil(N/4)-square matrices (no selects in the product loop); FP64 keeps
// the packed matrix.  The 16-node tile (74 KB at N = 24) lets two FP32 CTAs share
// an SM, so one CTA's loads overlap the other's arithmetic.
constexpr int kLargeTile = 16;

// SC: scaled hierarchy, link weights from Inst::wsc (see scaled_up).
template <typename R, bool MIXED, bool CPLX, bool SC = false>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) heom_large_kernel(EngineArgs A) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ Inst s_inst;
  __shared__ int s_stop;
  constexpr int TN = kLargeTile;

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
  const int node = lane >> 1, half = lane & 1;
  // tile 0 is on rank 0; its node 0 is the root, on lanes 0 and 1 of every warp
  const int nslots = 2 * nwarps;
  const int slot = (rank == 0 && lane < 2) ? 2 * warp + lane : -1;
  const bool lead = (rank == 0 && threadIdx.x == 0);
  unsigned epoch = 0;

  for (int li = A.team_first[team]; li < A.team_first[team + 1]; ++li) {
    __syncthreads();
    if (threadIdx.x == 0) s_inst = A.insts[A.team_list[li]];
    __syncthreads();
    const Inst& I = s_inst;
    const int N = I.N;
    const int NN = N * N;
    using L = CoefLayout<R>;
    const int JS = L::JS(N);  // = 4 * number of blocks per side
    const int NB = JS / 4;
    const int nblk = NB * (NB + 1) / 2;
    constexpr bool FULL = sizeof(R) == 4;
    R* tile = reinterpret_cast<R*>(dsm);
    R* tileA = tile + JS * JS * TN;
    unsigned char* cbytes = dsm + (size_t)(FULL ? 2 * JS * JS : NN) * TN * sizeof(R);
    const int cb = L::bytes(N);
    for (int i = threadIdx.x; i < cb; i += blockDim.x) cbytes[i] = static_cast<const unsigned char*>(I.coef)[i];
    if (FULL)
      for (int i = threadIdx.x; i < 2 * JS * JS * TN; i += blockDim.x) tile[i] = R(0);  // padding stays 0
    __syncthreads();
    const R* cf = reinterpret_cast<const R*>(cbytes);
    const double* cfd = reinterpret_cast<const double*>(cbytes + L::dbl_offset(N));
    const R* ngam = static_cast<const R*>(I.ngam);
    const int Mp = I.Mpad;
    const int ntiles = (I.M + TN - 1) / TN;
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
      for (int k = 0; k < nslots; ++k) ea.store(I, k);  // zero every running-sum slot of this instance
    }
    if (!team_barrier(A, epoch)) return;
    R* arr[3] = {static_cast<R*>(I.y), static_cast<R*>(I.wa), static_cast<R*>(I.wb)};
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
        const R h = P.h;
        const R* __restrict__ win = arr[in_sel];
        R* __restrict__ wout = arr[out_sel];
        const R* __restrict__ yv = arr[0];
        for (int tl = rank; tl < ntiles; tl += team_size) {
          const int n0 = tl * TN;
          __syncthreads();
          {
            // thread t copies (element, node) pairs e = t, t + blockDim, ...,
            // element e / 16 of node e % 16; 8 loads in flight before their
            // stores; (r, c) of the packed element is stepped along.
            const int jn = threadIdx.x & (TN - 1);
            const bool lv = n0 + jn < I.M;
            const int pstep = blockDim.x / TN;
            int r0 = 0, c0 = threadIdx.x / TN;
            while (c0 >= N) { c0 -= N; ++r0; }
            for (int p0 = threadIdx.x / TN; p0 < NN; p0 += 8 * pstep) {
              R v[8];
              int rr[8], cc[8];
              int r = r0, c = c0;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const int pp = p0 + q * pstep;
                rr[q] = r;
                cc[q] = c;
                v[q] = ld_global_or0(win + (pp * Mp + n0 + jn), lv && pp < NN);
                c += pstep;
                while (c >= N) { c -= N; ++r; }
              }
              r0 = r;
              c0 = c;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const int pp = p0 + q * pstep;
                if (pp >= NN) break;
                if constexpr (FULL) {
                  // packed (r, c): Re sigma_rc for r <= c, Im sigma_cr for r > c
                  const int rq = rr[q], cq = cc[q];
                  if (rq < cq) {
                    tile[(rq * JS + cq) * TN + jn] = v[q];
                    tile[(cq * JS + rq) * TN + jn] = v[q];
                  } else if (rq > cq) {
                    tileA[(cq * JS + rq) * TN + jn] = v[q];
                    tileA[(rq * JS + cq) * TN + jn] = -v[q];
                  } else {
                    tile[(rq * JS + rq) * TN + jn] = v[q];
                  }
                } else {
                  tile[pp * TN + jn] = v[q];
                }
              }
            }
          }
          __syncthreads();
          const int n = n0 + node;
          if (n >= I.M) continue;
          const bool root = (n == 0);
          const R ng = ngam[n];
          const bool term = I.terminator && I.up[n] < 0;
          // packed element (i, j) of this lane's node; 0 outside the N x N matrix
          auto Pk = [&](int i, int j) -> R { return (i < N && j < N) ? tile[(i * N + j) * TN + node] : R(0); };
          // Re sigma_ij and Im sigma_ij (FULL tile: no bounds checks, padding is 0)
          auto Sf = [&](int i, int j) -> R { return tile[(i * JS + j) * TN + node]; };
          auto Af = [&](int i, int j) -> R { return tileA[(i * JS + j) * TN + node]; };
          auto Re_ = [&](int i, int j) -> R { return FULL ? Sf(i, j) : Pk(i <= j ? i : j, i <= j ? j : i); };
          auto Im_ = [&](int i, int j) -> R {
            return FULL ? Af(i, j) : (i < j ? Pk(j, i) : (i > j ? -Pk(i, j) : R(0)));
          };
          for (int bk = warp; bk < nblk; bk += nwarps) {
            // block index -> (A0, B0), A0 <= B0; this lane's rows A0 + 2 half + {0, 1}
            int ab = 0, rem = bk;
            while (rem >= NB - ab) { rem -= NB - ab; ++ab; }
            const int A0 = 4 * ab + 2 * half, B0 = 4 * (ab + rem);
            // A diagonal block (the same for the whole warp) keeps only its 10 entries
            // with b >= a: in FP64, whose pipe bounds this kernel, the two lanes of a
            // node take rows {0, 3} and {1, 2} of it, five entries each, instead of rows
            // {0, 1} and {2, 3} with eight products each (about 11 % of the product work
            // of a 24-site node); FP32 is bound by the neighbour gathers and keeps the
            // plain blocks
            const bool dblk = sizeof(R) == 8 && rem == 0;
            const int ra0 = dblk ? 4 * ab + half : A0, ra1 = dblk ? 4 * ab + 3 - half : A0 + 1;
            R re[2][4], im[2][4];
            R rd[5], id[5];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) re[i][j] = im[i][j] = R(0);
#pragma unroll
            for (int e = 0; e < 5; ++e) rd[e] = id[e] = R(0);
            // -i[H, sigma] with the real part J (symmetric) and imaginary part Ji (antisymmetric) of H:
            //   Re += sum_k J(a,k) A(k,b) - A(a,k) J(k,b);  Im -= sum_k J(a,k) S(k,b) - S(a,k) J(k,b)
            //   Re += sum_k Ji(a,k) S(k,b) - S(a,k) Ji(k,b); Im += sum_k Ji(a,k) A(k,b) - A(a,k) Ji(k,b)
            // with S = Re sigma, A = Im sigma; J(a,k) = J(k,a) is read from row k.
#pragma unroll 2
            for (int k = 0; k < N; ++k) {
              R ja[2], jb[4];
              ja[0] = cf[L::J(N) + k * JS + ra0];
              ja[1] = cf[L::J(N) + k * JS + ra1];
              load_row<4>(cf + L::J(N) + k * JS + B0, jb);
              R sak[2], aak[2], skb[4], akb[4];
#pragma unroll
              for (int i = 0; i < 2; ++i) {
                sak[i] = Re_(i ? ra1 : ra0, k);
                aak[i] = Im_(i ? ra1 : ra0, k);
              }
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                skb[j] = Re_(B0 + j, k);    // S(k, b) = S(b, k)
                akb[j] = -Im_(B0 + j, k);   // A(k, b) = -A(b, k)
              }
              if (dblk) {
                // the five entries (row r, column c) of this lane, picked by selects:
                // half 0: (0,0) (0,1) (0,2) (0,3) (1,3); half 1: (0,1) (0,2) (0,3) (1,2) (1,3)
                const bool hf = half != 0;
                const R J0[5] = {ja[0], ja[0], ja[0], hf ? ja[1] : ja[0], ja[1]};
                const R S0[5] = {sak[0], sak[0], sak[0], hf ? sak[1] : sak[0], sak[1]};
                const R A0v[5] = {aak[0], aak[0], aak[0], hf ? aak[1] : aak[0], aak[1]};
                const R JB[5] = {hf ? jb[1] : jb[0], hf ? jb[2] : jb[1], hf ? jb[3] : jb[2], hf ? jb[2] : jb[3], jb[3]};
                const R SB[5] = {hf ? skb[1] : skb[0], hf ? skb[2] : skb[1], hf ? skb[3] : skb[2], hf ? skb[2] : skb[3],
                                 skb[3]};
                const R AB[5] = {hf ? akb[1] : akb[0], hf ? akb[2] : akb[1], hf ? akb[3] : akb[2], hf ? akb[2] : akb[3],
                                 akb[3]};
#pragma unroll
                for (int e = 0; e < 5; ++e) {
                  rd[e] = fma(J0[e], AB[e], rd[e]);
                  rd[e] = fma(-A0v[e], JB[e], rd[e]);
                  id[e] = fma(-J0[e], SB[e], id[e]);
                  id[e] = fma(S0[e], JB[e], id[e]);
                }
                if constexpr (CPLX) {
                  R ia[2], ib[4];
                  ia[0] = cf[L::Ji(N) + k * JS + ra0];
                  ia[1] = cf[L::Ji(N) + k * JS + ra1];
                  load_row<4>(cf + L::Ji(N) + k * JS + B0, ib);
                  const R I0[5] = {ia[0], ia[0], ia[0], hf ? ia[1] : ia[0], ia[1]};
                  const R IB[5] = {hf ? ib[1] : ib[0], hf ? ib[2] : ib[1], hf ? ib[3] : ib[2], hf ? ib[2] : ib[3], ib[3]};
#pragma unroll
                  for (int e = 0; e < 5; ++e) {
                    rd[e] = fma(-I0[e], SB[e], rd[e]);
                    rd[e] = fma(-S0[e], IB[e], rd[e]);
                    id[e] = fma(-I0[e], AB[e], id[e]);
                    id[e] = fma(-A0v[e], IB[e], id[e]);
                  }
                }
                continue;
              }
              // explicit multiply-add chains: two FMAs per output and term (written as
              // x += a*b - c*d the compiler keeps a separate multiply and add, 1.5x the
              // FP64 instructions of this loop)
#pragma unroll
              for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  re[i][j] = fma(ja[i], akb[j], re[i][j]);
                  re[i][j] = fma(-aak[i], jb[j], re[i][j]);
                  im[i][j] = fma(-ja[i], skb[j], im[i][j]);
                  im[i][j] = fma(sak[i], jb[j], im[i][j]);
                }
              if constexpr (CPLX) {
                R ia[2], ib[4];  // row k of Ji: Ji(k, a) = -Ji(a, k)
                ia[0] = cf[L::Ji(N) + k * JS + ra0];
                ia[1] = cf[L::Ji(N) + k * JS + ra1];
                load_row<4>(cf + L::Ji(N) + k * JS + B0, ib);
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                  for (int j = 0; j < 4; ++j) {
                    re[i][j] = fma(-ia[i], skb[j], re[i][j]);
                    re[i][j] = fma(-sak[i], ib[j], re[i][j]);
                    im[i][j] = fma(-ia[i], akb[j], im[i][j]);
                    im[i][j] = fma(-aak[i], ib[j], im[i][j]);
                  }
              }
            }
            if (dblk) {
              // the five entries into their places of the 2 x 4 block (rows ra0, ra1); the
              // places not set hold entries with b < a, which the epilogue drops
              const bool hf = half != 0;
              re[0][0] = rd[0];
              im[0][0] = id[0];
              re[0][1] = hf ? rd[0] : rd[1];
              im[0][1] = hf ? id[0] : id[1];
              re[0][2] = hf ? rd[1] : rd[2];
              im[0][2] = hf ? id[1] : id[2];
              re[0][3] = hf ? rd[2] : rd[3];
              im[0][3] = hf ? id[2] : id[3];
              re[1][2] = rd[3];
              im[1][2] = id[3];
              re[1][3] = rd[4];
              im[1][3] = id[4];
            }
            // links of the block's rows and columns
            int ua[2], ub[4], da[2], db[4];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int a = q ? ra1 : ra0;
              ua[q] = a < N ? I.up[a * Mp + n] : -1;
              da[q] = a < N ? I.dn[a * Mp + n] : -1;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int b = B0 + q;
              ub[q] = b < N ? I.up[b * Mp + n] : -1;
              db[q] = b < N ? I.dn[b * Mp + n] : -1;
            }
            // terminator factors (n_j + 1) / (ngam + gamma_j) of the block's rows and columns (leaf nodes)
            R tca[2], tcb[4];
#pragma unroll
            for (int q = 0; q < 2; ++q) tca[q] = R(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) tcb[q] = R(0);
            if (term) {
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const int a = min(q ? ra1 : ra0, N - 1);
                tca[q] = ((da[q] < 0 ? R(0) : R(da[q] >> 24)) + R(1)) / (ng + cf[L::gam(N) + a]);
              }
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int b = min(B0 + q, N - 1);
                tcb[q] = ((db[q] < 0 ? R(0) : R(db[q] >> 24)) + R(1)) / (ng + cf[L::gam(N) + b]);
              }
            }
            // Per row and pair of columns: the local, neighbour and terminator
            // terms of two outputs and their y values are loaded before their
            // stores.
#pragma unroll
            for (int ij = 0; ij < 4; ++ij) {
              const int i = ij >> 1, j0 = 2 * (ij & 1);
              R yr[4], yim[4];
              const int a = i ? ra1 : ra0;
              const int ac = a < N ? a : N - 1;  // clamped for addressing; outputs with a >= N are dropped
              const R* sa = cf + L::site(N) + 4 * ac;
              const R eps_a = sa[0], gh_a = sa[1], al_a = sa[2], be_a = sa[3];
              R na = da[i] < 0 ? R(0) : R(da[i] >> 24);
              const int dai = da[i] < 0 ? -1 : (da[i] & 0xFFFFFF);
              R wua = R(1);  // up-link weight of row a (scaled hierarchy)
              if constexpr (SC) {
                wua = scaled_up(static_cast<const R*>(I.wsc), I.wstride, ac, na);
                na = scaled_dn(static_cast<const R*>(I.wsc), I.wstride, ac, na);
              }
              const R ca = tca[i];
#pragma unroll
              for (int j = j0; j < j0 + 2; ++j) {
                const int b = B0 + j;
                const int bc = b < N ? b : N - 1;
                const bool keep = a < N && b < N && b >= a;
                const int pr = ac * N + bc, pi = bc * N + ac;
                yr[j] = ld_global_or0(yv + (pr * Mp + n), keep);
                yim[j] = ld_global_or0(yv + (pi * Mp + n), keep && a != b);
                const R* sb = cf + L::site(N) + 4 * bc;
                const R eps_b = sb[0], gh_b = sb[1], al_b = sb[2], be_b = sb[3];
                const R x = Re_(a, b), yi = Im_(a, b);
                const int dbj = db[j] < 0 ? -1 : (db[j] & 0xFFFFFF);
                R nb = db[j] < 0 ? R(0) : R(db[j] >> 24);
                R wub = R(1);
                if constexpr (SC) {
                  wub = scaled_up(static_cast<const R*>(I.wsc), I.wstride, bc, nb);
                  nb = scaled_dn(static_cast<const R*>(I.wsc), I.wstride, bc, nb);
                }
                // up-couplings i V_j^x sigma_{n+e_j}: j = a gives +i, j = b gives -i
                const R uar = ld_global_or0(win + (pr * Mp + ua[i]), keep && a != b && ua[i] >= 0);
                const R uai = ld_global_or0(win + (pi * Mp + ua[i]), keep && a != b && ua[i] >= 0);
                const R ubr = ld_global_or0(win + (pr * Mp + ub[j]), keep && a != b && ub[j] >= 0);
                const R ubi = ld_global_or0(win + (pi * Mp + ub[j]), keep && a != b && ub[j] >= 0);
                // down-couplings n_j theta_j sigma_{n-e_j}
                const R dar = ld_global_or0(win + (pr * Mp + dai), keep && dai >= 0);
                const R dai_ = ld_global_or0(win + (pi * Mp + dai), keep && a != b && dai >= 0);
                const R dbr = ld_global_or0(win + (pr * Mp + dbj), keep && a != b && dbj >= 0);
                const R dbi = ld_global_or0(win + (pi * Mp + dbj), keep && a != b && dbj >= 0);
                R r = re[i][j], m = im[i][j];
                if (a != b) {
                  // the same terms as the small-N units, as multiply-add chains
                  const R d = eps_a - eps_b;
                  const R c = ng + gh_a + gh_b;
                  r = fma(d, yi, r);
                  r = fma(-c, x, r);
                  m = fma(-d, x, m);
                  m = fma(-c, yi, m);
                  if constexpr (SC) {
                    r = fma(wub, ubi, r);
                    r = fma(-wua, uai, r);
                    m = fma(wua, uar, m);
                    m = fma(-wub, ubr, m);
                  } else {
                    r += ubi - uai;
                    m += uar - ubr;
                  }
                  if (I.terminator) {
                    const R cbf = tcb[j];
                    r += ca * (-al_a * x - be_a * yi) + cbf * (-al_b * x + be_b * yi);
                    m += ca * (-al_a * yi + be_a * x) + cbf * (-al_b * yi - be_b * x);
                  }
                  const R nbe_a = na * be_a, nal_a = na * al_a, nbe_b = nb * be_b, nal_b = nb * al_b;
                  r = fma(nbe_a, dar, r);
                  r = fma(-nal_a, dai_, r);
                  r = fma(nbe_b, dbr, r);
                  r = fma(nal_b, dbi, r);
                  m = fma(nal_a, dar, m);
                  m = fma(nbe_a, dai_, m);
                  m = fma(nbe_b, dbi, m);
                  m = fma(-nal_b, dbr, m);
                } else {
                  r -= (ng + R(2) * cf[L::gd(N) + ac]) * x;
                  r += R(2) * na * be_a * dar;
                }
                re[i][j] = r;
                im[i][j] = m;
              }
              // Horner update w = y + h r and the stores (root in float-float for mixed precision)
#pragma unroll
              for (int j = j0; j < j0 + 2; ++j) {
                const int b = B0 + j;
                if (a >= N || b >= N || b < a) continue;
                const int pr = a * N + b, pi = b * N + a;
                const R r = re[i][j], m = im[i][j];
                if (MIXED && root) {
                  if constexpr (MIXED) {
                    if (a == b && s == 3) ea.add(I, a, P.root_in[pr]);
                    if (a == b && s == 2) ea.add_xi(I, a, P.root_in[pr]);
                    const FF wr = ff_axpy(P.root_y[pr], P.h, P.hl, r);
                    P.root_out[pr] = wr;
                    wout[pr * Mp] = wr.h;
                    if (a != b) {
                      const FF wi = ff_axpy(P.root_y[pi], P.h, P.hl, m);
                      P.root_out[pi] = wi;
                      wout[pi * Mp] = wi.h;
                    } else if (s == 3 && I.out_pops && os.now) {
                      I.out_pops[os.row * N + a] = ff_to_double(wr);
                    }
                  }
                } else {
                  if constexpr (!MIXED) {
                    if (root && a == b && s == 3) ea.add(I, cfd, N, a, (double)Re_(a, a));
                    if (root && a == b && s == 2) ea.add_xi(I, cfd, a, (double)Re_(a, a));
                  }
                  const R vr = yr[j] + h * r;
                  wout[pr * Mp + n] = vr;
                  if (a != b) {
                    wout[pi * Mp + n] = yim[j] + h * m;
                  } else if (root && s == 3 && I.out_pops && os.now) {
                    I.out_pops[os.row * N + a] = (double)vr;
                  }
                }
              }
            }
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

__host__ __device__ constexpr int large_smem_bytes(int N, int rsize) {
  // FP32: unpacked Re and Im tiles of (4 ceil(N/4))^2 x 16 nodes; FP64: the packed tile N^2 x 16
  return rsize == 8 ? N * N * kLargeTile * 8 + CoefLayout<double>::bytes(N)
                    : 2 * CoefLayout<float>::JS(N) * CoefLayout<float>::JS(N) * kLargeTile * 4 +
                          CoefLayout<float>::bytes(N);
}

}  // namespace heom
