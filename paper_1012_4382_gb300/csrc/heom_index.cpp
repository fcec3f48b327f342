// heom_index.cpp -- hierarchy index builder of libheom (host code).
//
// The hierarchy holds one auxiliary matrix sigma_n for every multi-index
// n in N^N with |n| = sum_j n_j <= K; there are C(N+K, K) of them (App. B,
// N_tot), and each is coupled to its 2N neighbours n +- e_j (App. B).
//
// Order: by level |n|, then lexicographically descending (larger n_1 first,
// then larger n_2, ...).  This order is translation invariant, so for every j
// the map n -> n + e_j is increasing inside a level; node blocks of 32
// consecutive nodes therefore gather from ascending, nearly contiguous
// neighbour indices.
//
// Neighbours are found by combinatorial ranking: the rank of n is the number
// of multi-indices on lower levels, C(|n| - 1 + N, N), plus the number of
// compositions of |n| into N parts that precede n in the descending order,
// sum_j sum_{v = n_j+1}^{R_j} C(R_j - v + N - j - 2, N - j - 2),
// R_j = |n| - n_1 - ... - n_{j-1}.
#include <cstdint>
#include <vector>

#include "heom_internal.h"

namespace heom {

namespace {

// C(n, k) with saturation at INT64_MAX.
int64_t binom(int64_t n, int64_t k) {
  if (k < 0 || n < 0 || k > n) return 0;
  if (k > n - k) k = n - k;
  __int128 r = 1;
  for (int64_t i = 1; i <= k; ++i) {
    r = r * (n - k + i) / i;
    if (r > (__int128)INT64_MAX) return INT64_MAX;
  }
  return (int64_t)r;
}

// number of compositions of L into P >= 0 parts
int64_t compositions(int L, int P) {
  if (P == 0) return L == 0 ? 1 : 0;
  return binom((int64_t)L + P - 1, P - 1);
}

void enumerate_level(int N, int level, int j, int remaining, std::vector<int32_t>& cur, std::vector<int32_t>& out) {
  if (j == N - 1) {
    cur[j] = remaining;
    out.insert(out.end(), cur.begin(), cur.end());
    cur[j] = 0;
    return;
  }
  for (int v = remaining; v >= 0; --v) {
    cur[j] = v;
    enumerate_level(N, level, j + 1, remaining - v, cur, out);
  }
  cur[j] = 0;
}

}  // namespace

int64_t num_nodes(int N, int K) {
  if (N < 1 || K < 0) return -1;
  const int64_t c = binom((int64_t)N + K, K);
  return c == INT64_MAX ? -1 : c;
}

int64_t rank_of(const int32_t* n, int N, int K) {
  int L = 0;
  for (int j = 0; j < N; ++j) {
    if (n[j] < 0) return -1;
    L += n[j];
  }
  if (L > K) return -1;
  int64_t r = L > 0 ? binom((int64_t)L - 1 + N, N) : 0;
  int R = L;
  for (int j = 0; j < N - 1; ++j) {
    for (int v = R; v > n[j]; --v) r += compositions(R - v, N - j - 1);
    R -= n[j];
  }
  return r;
}

void build_index(int N, int K, Index& out) {
  out.N = N;
  out.K = K;
  out.M = num_nodes(N, K);
  out.multi.clear();
  out.multi.reserve((size_t)out.M * N);
  std::vector<int32_t> cur(N, 0);
  for (int level = 0; level <= K; ++level) enumerate_level(N, level, 0, level, cur, out.multi);
  out.up.assign((size_t)out.M * N, -1);
  out.down.assign((size_t)out.M * N, -1);
  std::vector<int32_t> nb(N);
  for (int64_t i = 0; i < out.M; ++i) {
    const int32_t* n = &out.multi[(size_t)i * N];
    int L = 0;
    for (int j = 0; j < N; ++j) L += n[j];
    for (int j = 0; j < N; ++j) {
      for (int k = 0; k < N; ++k) nb[k] = n[k];
      if (L < K) {
        nb[j] += 1;
        out.up[(size_t)i * N + j] = (int32_t)rank_of(nb.data(), N, K);
        nb[j] -= 1;
      }
      if (n[j] > 0) {
        nb[j] -= 1;
        out.down[(size_t)i * N + j] = (int32_t)rank_of(nb.data(), N, K);
      }
    }
  }
}

}  // namespace heom

namespace heom {

namespace {

struct TableWriter {
  int N, K, Mpad;
  int32_t* up;
  int32_t* dn;
  int64_t next;
  int32_t cur[32];
};

void write_level(TableWriter& w, int j, int remaining, int level) {
  if (j == w.N - 1) {
    w.cur[j] = remaining;
    const int64_t i = w.next++;
    int32_t nb[32];
    for (int k = 0; k < w.N; ++k) nb[k] = w.cur[k];
    for (int k = 0; k < w.N; ++k) {
      int32_t u = -1, d = -1;
      if (level < w.K) {
        nb[k] += 1;
        u = (int32_t)rank_of(nb, w.N, w.K);
        nb[k] -= 1;
      }
      if (w.cur[k] > 0) {
        nb[k] -= 1;
        d = (w.cur[k] << 24) | (int32_t)rank_of(nb, w.N, w.K);
        nb[k] += 1;
      }
      w.up[(size_t)k * w.Mpad + i] = u;
      w.dn[(size_t)k * w.Mpad + i] = d;
    }
    w.cur[j] = 0;
    return;
  }
  for (int v = remaining; v >= 0; --v) {
    w.cur[j] = v;
    write_level(w, j + 1, remaining - v, level);
  }
  w.cur[j] = 0;
}

}  // namespace

int64_t write_packed_tables(int N, int K, int Mpad, int32_t* up, int32_t* dn) {
  if (N < 1 || N > 32 || K < 0) return -1;
  TableWriter w;
  w.N = N;
  w.K = K;
  w.Mpad = Mpad;
  w.up = up;
  w.dn = dn;
  w.next = 0;
  for (int k = 0; k < 32; ++k) w.cur[k] = 0;
  for (int level = 0; level <= K; ++level) write_level(w, 0, level, level);
  for (int k = 0; k < N; ++k)
    for (int64_t i = w.next; i < Mpad; ++i) {
      up[(size_t)k * Mpad + i] = -1;
      dn[(size_t)k * Mpad + i] = -1;
    }
  return w.next;
}

}  // namespace heom
