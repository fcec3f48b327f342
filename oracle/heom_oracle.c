/*
 * heom_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU reference ("the oracle") for the hybrid
 * master-equation / hierarchical-equations-of-motion (ME-HEOM) propagation of
 * Kreisbeck, Kramer, Rodriguez and Hein, "High-performance solution of
 * hierarchical equations of motions for studying energy-transfer in
 * light-harvesting complexes" (arXiv:1012.4382).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header, table or helper with the CUDA
 * path, and the CUDA path never calls it.
 *
 * What it computes, written out as the paper defines it:
 *   * the reduced density matrix lives on the N exciton sites plus the
 *     electronic ground state |0> and the reaction-centre state |RC>
 *     (Sec. "Model", the (N+2)x(N+2) = 9x9 matrix for N = 7);
 *   * H_ex = sum_m (eps_m [+ lambda_m]) |m><m| + sum_{m>n} J_mn (|m><n| + h.c.),
 *     E_0 = 0 (Eq. H_ex); E_RC = 0 (the paper gives no value; it never enters
 *     populations);
 *   * radiative decay sum_m Gamma_phot D(|0><m|) and trapping
 *     sum_m Gamma_RC D(|RC><m|) in Lindblad form, D(L)x = L x L^+ - {L^+L, x}/2
 *     (App. A1, Eqs. lab2 and lab3);
 *   * one Drude-Lorentz bath per site, V_m = |m><m|, high-temperature
 *     correlation functions (App. A2, Eq. gamma and the S, chi forms);
 *   * the hierarchy of App. A2, Eqs. labsevena and lab8:
 *       d sigma_n/dt = -i[H_ex, sigma_n] + (Lindblad terms) sigma_n
 *                      - sum_m n_m gamma_m sigma_n
 *                      + sum_m i V_m^x sigma_{n+e_m}
 *                      + sum_m n_m theta_m sigma_{n-e_m},
 *       theta_m = i ( 2 lambda_m k_B T V_m^x  -  i lambda_m gamma_m V_m^o ),
 *     with sigma_0 = rho, all other sigma zero at t = 0, truncated at
 *     |n| = N_max (end of App. A2);
 *   * classic 4th-order Runge-Kutta in time (App. B);
 *   * the efficiency eta = <RC| rho |RC> (Eq. eta) read off the RC element of
 *     rho itself, and the radiative loss read off <0| rho |0>;
 *   * the trapping time <t> = int_0^t t' d<RC|rho|RC>/dt' dt' (Eq.
 *     trappingtime), evaluated as t eta(t) - int_0^t eta dt' (integration by
 *     parts, exact for the integrals), where xi = int eta dt is one more
 *     component of the RK4 system (xi' = <RC|rho|RC>);
 *   * the stop rule of Sec. "Trapping time": propagation ends at t_max, the
 *     first step at which the population left on the sites has dropped below
 *     a threshold (1e-5 in the paper).
 *   * optionally the scaled hierarchy the paper points to in its introduction
 *     (the "scaled version of the HEOM"; the formula is not printed there):
 *     the auxiliaries are rescaled, sigma~_n = sigma_n / S(n) with
 *     S(n) = prod_j sqrt(n_j! s_j^{n_j}) and s_j = |2 lambda_j kT - i lambda_j gamma_j|
 *     the modulus of the bath's correlation amplitude (1 where lambda_j = 0;
 *     the rescaling of Shi et
 *     al., J. Chem. Phys. 130, 084105 (2009)).  Substituting sigma_n = S(n)
 *     sigma~_n into the hierarchy gives the same equations with the up link
 *     weighted by S(n+e_j)/S(n) = sqrt((n_j+1) s_j) and the down link's n_j
 *     replaced by n_j S(n-e_j)/S(n) = sqrt(n_j / s_j).  S(0) = 1, so rho is the
 *     same; the terminator term is local and unchanged.
 *
 * Readings of the paper taken here (each one is also listed in the design notes):
 *   * damping sign: lab8 prints "+ sum n_m gamma_m" inside the bracket; the
 *     hierarchy is only stable with a minus sign, which is the Ishizaki-Fleming
 *     form the paper says it follows.  The oracle uses "- sum n_m gamma_m".
 *   * temperature factor in theta_m: the printed 2 lambda / (k_B T hbar^2) is
 *     dimensionally inconsistent; the oracle uses 2 lambda k_B T / hbar^2, the
 *     high-temperature limit of the real part of the Drude-Lorentz correlation
 *     function at t = 0.
 *   * optional truncation terminator (the paper only says "truncate"): for
 *     |n| = N_max, sigma_{n+e_j} is replaced by
 *     (n_j + 1) theta_j sigma_n / (sum_k n_k gamma_k + gamma_j).
 *
 * Units: energies in cm^-1 are converted to angular frequencies in rad/fs with
 * 2 pi c, c = 2.99792458e-5 cm/fs; k_B = 0.6950348004 cm^-1/K; rates in ps^-1
 * are divided by 1000 to give fs^-1; hbar = 1.
 *
 * Nothing here is blocked, fused or reordered beyond the equations above:
 * every commutator is two full complex matrix products, every projector
 * super-operator is applied element by element from its definition.
 * The node loop of the right-hand side may run on several OpenMP threads; each
 * node is written by exactly one thread, so the result does not depend on the
 * thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_PI 3.14159265358979323846
static const double OR_C_CM_PER_FS = 2.99792458e-5;  /* speed of light */
static const double OR_KB_CM_PER_K = 0.6950348004;   /* Boltzmann constant / (h c) */

static double cm_to_rad_per_fs(double x) { return 2.0 * OR_PI * OR_C_CM_PER_FS * x; }

/* Parameters as the caller gives them (paper units).  The field order is
 * mirrored by the ctypes structure in oracle/__init__.py. */
typedef struct {
  int32_t N;               /* number of exciton sites */
  int32_t K;               /* truncation depth N_max */
  const double* H;         /* N*N complex (re, im interleaved), row-major, cm^-1 */
  const double* lambda;    /* N reorganisation energies, cm^-1 */
  const double* gamma;     /* N bath correlation rates, cm^-1 */
  double T;                /* temperature, K */
  const double* trap;      /* N trapping rates Gamma_RC (ps^-1) or NULL */
  const double* recomb;    /* N radiative decay rates Gamma_phot (ps^-1) or NULL */
  int32_t terminator;      /* 0: plain truncation, 1: Markovian terminator */
  int32_t add_reorg;       /* 1: eps_m -> eps_m + lambda_m (Eq. H_ex) */
  int32_t low_temp;        /* 1: lowest-order quantum (low-temperature) correction */
  int32_t scaled;          /* 1: scaled auxiliaries sigma~_n = sigma_n / S(n) (see the header) */
  const unsigned char* keep; /* NULL, or one flag per node in the order of oracle_multi_indices: a node
                                with flag 0 is removed from the hierarchy (its matrix stays zero, so
                                every link to it contributes nothing) -- the filtered hierarchy */
} oracle_params;

/* ---------------------------------------------------------------------- */
/* Hierarchy of multi-indices n in N^N with |n| <= K                        */
/* (App. B: the number of sigma-matrices is (N + N_max)! / (N! N_max!))     */
/* ---------------------------------------------------------------------- */

typedef struct {
  int N, K;
  long nodes;
  int* idx;     /* nodes * N multi-indices, sorted by (level, lexicographic ascending) */
  long* plus;   /* nodes * N: node of n + e_j, or -1 when |n| = K */
  long* minus;  /* nodes * N: node of n - e_j, or -1 when n_j = 0 */
} hierarchy;

static int g_cmp_N;  /* width used by the qsort/bsearch comparator */

static int level_of(const int* n, int N) {
  int s = 0;
  for (int j = 0; j < N; ++j) s += n[j];
  return s;
}

static int cmp_multi(const void* pa, const void* pb) {
  const int* a = (const int*)pa;
  const int* b = (const int*)pb;
  int la = level_of(a, g_cmp_N), lb = level_of(b, g_cmp_N);
  if (la != lb) return la < lb ? -1 : 1;
  for (int j = 0; j < g_cmp_N; ++j)
    if (a[j] != b[j]) return a[j] < b[j] ? -1 : 1;
  return 0;
}

/* Depth-first listing of every n with sum(n) <= K. */
static void list_rec(int N, int K, int j, int used, int* cur, int* out, long* count) {
  if (j == N) {
    memcpy(out + (*count) * N, cur, sizeof(int) * N);
    (*count)++;
    return;
  }
  for (int v = 0; v <= K - used; ++v) {
    cur[j] = v;
    list_rec(N, K, j + 1, used + v, cur, out, count);
  }
  cur[j] = 0;
}

/* C(N+K, K) computed by counting, to stay independent of any closed form. */
static long count_rec(int N, int K, int j, int used) {
  if (j == N) return 1;
  long c = 0;
  for (int v = 0; v <= K - used; ++v) c += count_rec(N, K, j + 1, used + v);
  return c;
}

static void hier_free(hierarchy* h) {
  free(h->idx);
  free(h->plus);
  free(h->minus);
  memset(h, 0, sizeof(*h));
}

static int hier_build(hierarchy* h, int N, int K) {
  memset(h, 0, sizeof(*h));
  h->N = N;
  h->K = K;
  h->nodes = count_rec(N, K, 0, 0);
  h->idx = (int*)malloc(sizeof(int) * (size_t)h->nodes * N);
  h->plus = (long*)malloc(sizeof(long) * (size_t)h->nodes * N);
  h->minus = (long*)malloc(sizeof(long) * (size_t)h->nodes * N);
  int* cur = (int*)calloc((size_t)N, sizeof(int));
  if (!h->idx || !h->plus || !h->minus || !cur) {
    free(cur);
    hier_free(h);
    return -1;
  }
  long count = 0;
  list_rec(N, K, 0, 0, cur, h->idx, &count);
  g_cmp_N = N;
  qsort(h->idx, (size_t)h->nodes, sizeof(int) * N, cmp_multi);
  for (long i = 0; i < h->nodes; ++i) {
    const int* n = h->idx + i * N;
    int lev = level_of(n, N);
    for (int j = 0; j < N; ++j) {
      memcpy(cur, n, sizeof(int) * N);
      cur[j] += 1;
      long p = -1;
      if (lev < K) {
        const int* hit = (const int*)bsearch(cur, h->idx, (size_t)h->nodes, sizeof(int) * N, cmp_multi);
        p = hit ? (long)((hit - h->idx) / N) : -1;
      }
      h->plus[i * N + j] = p;
      memcpy(cur, n, sizeof(int) * N);
      long m = -1;
      if (n[j] > 0) {
        cur[j] -= 1;
        const int* hit = (const int*)bsearch(cur, h->idx, (size_t)h->nodes, sizeof(int) * N, cmp_multi);
        m = hit ? (long)((hit - h->idx) / N) : -1;
      }
      h->minus[i * N + j] = m;
    }
  }
  free(cur);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* The model in rad/fs on the (N+2)-dimensional space                       */
/* basis: 0..N-1 = sites |m>, N = ground |0>, N+1 = reaction centre |RC>   */
/* ---------------------------------------------------------------------- */

typedef struct {
  int N, D;          /* D = N + 2 */
  cplx* H;           /* D*D system Hamiltonian */
  double* lam;       /* N, rad/fs */
  double* gam;       /* N, rad/fs */
  double kT;         /* rad/fs */
  double* g_rc;      /* N, fs^-1 */
  double* g_phot;    /* N, fs^-1 */
  double* ltc;       /* N, fs^-1: low-temperature correction rate per bath (0: off) */
  double* scale;     /* N, rad^2/fs^2: s_j of the scaled hierarchy, or NULL (unscaled) */
  int terminator;
  const unsigned char* keep; /* the caller's node flags (oracle_params.keep), or NULL: every node */
  hierarchy hier;
} model;

static void model_free(model* m) {
  free(m->H);
  free(m->lam);
  free(m->gam);
  free(m->g_rc);
  free(m->g_phot);
  free(m->ltc);
  free(m->scale);
  hier_free(&m->hier);
  memset(m, 0, sizeof(*m));
}

static int model_build(model* m, const oracle_params* p) {
  memset(m, 0, sizeof(*m));
  if (!p || p->N < 1 || p->K < 0 || !p->H || !p->lambda || !p->gamma || !(p->T > 0)) return -1;
  int N = p->N, D = N + 2;
  m->N = N;
  m->D = D;
  m->H = (cplx*)calloc((size_t)D * D, sizeof(cplx));
  m->lam = (double*)calloc((size_t)N, sizeof(double));
  m->gam = (double*)calloc((size_t)N, sizeof(double));
  m->g_rc = (double*)calloc((size_t)N, sizeof(double));
  m->g_phot = (double*)calloc((size_t)N, sizeof(double));
  m->ltc = (double*)calloc((size_t)N, sizeof(double));
  if (!m->H || !m->lam || !m->gam || !m->g_rc || !m->g_phot || !m->ltc) {
    model_free(m);
    return -1;
  }
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      double re = p->H[2 * (a * N + b)], im = p->H[2 * (a * N + b) + 1];
      m->H[a * D + b] = cm_to_rad_per_fs(re) + I * cm_to_rad_per_fs(im);
    }
  for (int a = 0; a < N; ++a) {
    if (p->add_reorg) m->H[a * D + a] += cm_to_rad_per_fs(p->lambda[a]);
    m->lam[a] = cm_to_rad_per_fs(p->lambda[a]);
    m->gam[a] = cm_to_rad_per_fs(p->gamma[a]);
    m->g_rc[a] = p->trap ? p->trap[a] * 1e-3 : 0.0;
    m->g_phot[a] = p->recomb ? p->recomb[a] * 1e-3 : 0.0;
  }
  m->kT = cm_to_rad_per_fs(OR_KB_CM_PER_K * p->T);
  m->terminator = p->terminator;
  m->keep = p->keep;
  /* Lowest-order quantum correction (the paper cites Ishizaki-Fleming for it):
   * the Drude-Lorentz correlation function has, besides the exp(-gamma t)
   * term kept in the hierarchy, Matsubara terms
   *   c_k exp(-nu_k t),  nu_k = 2 pi k kT,  c_k = 4 lambda gamma kT nu_k / (nu_k^2 - gamma^2),  k >= 1.
   * Taking exp(-nu_k t) ~ delta(t) / nu_k turns them into the local term
   *   - sum_j ltc_j V_j^x V_j^x sigma_n,  ltc_j = sum_k c_k / nu_k,
   * and with sum_{k>=1} 1/(k^2 - x^2) = 1/(2 x^2) - pi cot(pi x) / (2 x)
   * the sum is ltc_j = 2 lambda_j kT / gamma_j - lambda_j cot(gamma_j / (2 kT)). */
  if (p->low_temp)
    for (int a = 0; a < N; ++a) {
      const double x = m->gam[a] / (2.0 * m->kT);
      m->ltc[a] = 2.0 * m->lam[a] * m->kT / m->gam[a] - m->lam[a] * cos(x) / sin(x);
    }
  if (p->scaled) {
    m->scale = (double*)calloc((size_t)N, sizeof(double));
    if (!m->scale) {
      model_free(m);
      return -1;
    }
    /* s_j = |c_j|, c_j = 2 lambda_j kT - i lambda_j gamma_j */
    /* s_j = |c_j|, c_j = 2 lambda_j kT - i lambda_j gamma_j; a site without a
     * bath (lambda_j = 0) never feeds its auxiliaries, and any s_j > 0 is a
     * valid rescaling there: s_j = 1 */
    for (int a = 0; a < N; ++a) {
      m->scale[a] = cabs(2.0 * m->lam[a] * m->kT - I * m->lam[a] * m->gam[a]);
      if (!(m->scale[a] > 0)) m->scale[a] = 1.0;
    }
  }
  if (hier_build(&m->hier, N, p->K) != 0) {
    model_free(m);
    return -1;
  }
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Super-operators, each written from its definition                       */
/* ---------------------------------------------------------------------- */

/* out += c * (-i) [H, x]  (two full matrix products) */
static void add_commutator(const model* m, const cplx* x, cplx* out) {
  int D = m->D;
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      cplx hx = 0, xh = 0;
      for (int k = 0; k < D; ++k) {
        hx += m->H[a * D + k] * x[k * D + b];
        xh += x[a * D + k] * m->H[k * D + b];
      }
      out[a * D + b] += -I * (hx - xh);
    }
}

/* out += rate * D(|t><s|) x  with D(L)x = L x L^+ - (L^+ L x + x L^+ L)/2.
 * For L = |t><s|: L x L^+ = x_ss |t><t| and L^+ L = |s><s|. */
static void add_lindblad(int D, int t, int s, double rate, const cplx* x, cplx* out) {
  if (rate == 0.0) return;
  out[t * D + t] += rate * x[s * D + s];
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      double proj = 0.0;
      if (a == s) proj += 0.5;
      if (b == s) proj += 0.5;
      if (proj != 0.0) out[a * D + b] -= rate * proj * x[a * D + b];
    }
}

/* out += c * V_m^x x = c (V_m x - x V_m), V_m = |m><m| */
static void add_Vcomm(int D, int m, cplx c, const cplx* x, cplx* out) {
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      double v = (a == m ? 1.0 : 0.0) - (b == m ? 1.0 : 0.0);
      if (v != 0.0) out[a * D + b] += c * v * x[a * D + b];
    }
}

/* out += c * V_m^o x = c (V_m x + x V_m) */
static void add_Vanti(int D, int m, cplx c, const cplx* x, cplx* out) {
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      double v = (a == m ? 1.0 : 0.0) + (b == m ? 1.0 : 0.0);
      if (v != 0.0) out[a * D + b] += c * v * x[a * D + b];
    }
}

/* out += c * theta_m x,  theta_m = i (2 lambda_m kT V_m^x - i lambda_m gamma_m V_m^o) */
static void add_theta(const model* m, int j, cplx c, const cplx* x, cplx* out) {
  add_Vcomm(m->D, j, c * I * 2.0 * m->lam[j] * m->kT, x, out);
  add_Vanti(m->D, j, c * m->lam[j] * m->gam[j], x, out);
}

/* The whole right-hand side (Eqs. labsevena, lab8) for one node. */
static void rhs_node(const model* m, long i, const cplx* state, cplx* out, cplx* scratch) {
  int N = m->N, D = m->D;
  size_t DD = (size_t)D * D;
  const hierarchy* h = &m->hier;
  const int* n = h->idx + i * N;
  const cplx* x = state + i * DD;
  cplx* o = out + i * DD;
  for (size_t e = 0; e < DD; ++e) o[e] = 0;
  if (m->keep && !m->keep[i]) return; /* removed from the (filtered) hierarchy */

  /* -i [H_ex, sigma_n] */
  add_commutator(m, x, o);
  /* radiative decay to |0> and trapping to |RC> in Lindblad form */
  for (int s = 0; s < N; ++s) {
    add_lindblad(D, N, s, m->g_phot[s], x, o);
    add_lindblad(D, N + 1, s, m->g_rc[s], x, o);
  }
  /* - sum_j ltc_j V_j^x (V_j^x sigma_n): the low-temperature correction */
  for (int j = 0; j < N; ++j) {
    if (m->ltc[j] == 0.0) continue;
    for (size_t e = 0; e < DD; ++e) scratch[e] = 0;
    add_Vcomm(D, j, 1.0, x, scratch);
    add_Vcomm(D, j, -m->ltc[j], scratch, o);
  }
  /* - sum_m n_m gamma_m sigma_n */
  double ngam = 0.0;
  for (int j = 0; j < N; ++j) ngam += n[j] * m->gam[j];
  for (size_t e = 0; e < DD; ++e) o[e] -= ngam * x[e];
  for (int j = 0; j < N; ++j) {
    /* link weights: 1 and n_j, or sqrt((n_j+1) s_j) and sqrt(n_j / s_j) when scaled */
    const double w_up = m->scale ? sqrt((n[j] + 1) * m->scale[j]) : 1.0;
    const double w_dn = m->scale ? sqrt(n[j] / m->scale[j]) : (double)n[j];
    /* + i V_j^x sigma_{n+e_j} */
    long up = h->plus[i * N + j];
    if (up >= 0) {
      add_Vcomm(D, j, I * w_up, state + up * DD, o);
    } else if (m->terminator == 1 && level_of(n, N) == h->K) {
      /* sigma_{n+e_j} ~ (n_j + 1) theta_j sigma_n / (sum_k n_k gamma_k + gamma_j) */
      for (size_t e = 0; e < DD; ++e) scratch[e] = 0;
      add_theta(m, j, (double)(n[j] + 1) / (ngam + m->gam[j]), x, scratch);
      add_Vcomm(D, j, I, scratch, o);
    }
    /* + n_j theta_j sigma_{n-e_j} */
    long dn = h->minus[i * N + j];
    if (dn >= 0) add_theta(m, j, w_dn, state + dn * DD, o);
  }
}

static void rhs_all(const model* m, const cplx* state, cplx* out, cplx* scratch_all) {
  long nodes = m->hier.nodes;
  size_t DD = (size_t)m->D * m->D;
  long i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < nodes; ++i) {
#ifdef _OPENMP
    cplx* scratch = scratch_all + (size_t)omp_get_thread_num() * DD;
#else
    cplx* scratch = scratch_all;
#endif
    rhs_node(m, i, state, out, scratch);
  }
}

static int max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Exported functions                                                      */
/* ---------------------------------------------------------------------- */

int oracle_num_threads(void) { return max_threads(); }

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Number of nodes of the hierarchy, by counting. */
long long oracle_num_nodes(int N, int K) {
  if (N < 1 || K < 0) return -1;
  return (long long)count_rec(N, K, 0, 0);
}

/* Multi-indices of all nodes in the oracle's own order (nodes*N ints). */
int oracle_multi_indices(int N, int K, int* out) {
  hierarchy h;
  if (hier_build(&h, N, K) != 0) return -1;
  memcpy(out, h.idx, sizeof(int) * (size_t)h.nodes * N);
  hier_free(&h);
  return 0;
}

/* Applies the right-hand side once to a full state vector.
 * state_in/state_out: nodes * (N+2)^2 complex, node order of
 * oracle_multi_indices, basis order sites, |0>, |RC>. */
int oracle_rhs(const oracle_params* p, const double* state_in, double* state_out) {
  model m;
  if (model_build(&m, p) != 0) return -1;
  size_t DD = (size_t)m.D * m.D;
  cplx* scratch = (cplx*)calloc(DD * (size_t)max_threads(), sizeof(cplx));
  if (!scratch) {
    model_free(&m);
    return -1;
  }
  rhs_all(&m, (const cplx*)state_in, (cplx*)state_out, scratch);
  free(scratch);
  model_free(&m);
  return 0;
}

/* Classic RK4 propagation from rho(0) (N*N complex on the sites; ground and RC
 * start empty, all auxiliary matrices start at zero).
 *
 * Outputs at steps 0, out_every, 2*out_every, ... (nout = nsteps/out_every + 1):
 *   pops_out  [nout*N]  Re <m|rho|m>              (may be NULL)
 *   trace_out [nout]    sum_m Re <m|rho|m>        (may be NULL)
 *   eta_out   [nout]    Re <RC|rho|RC>            (may be NULL)
 *   loss_out  [nout]    Re <0|rho|0>              (may be NULL)
 *   tmean_out [nout]    trapping time <t> up to that step, fs (may be NULL)
 * and at the end:
 *   rho_out   [N*N complex] site block of rho     (may be NULL)
 *   state_out [nodes*(N+2)^2 complex] every node  (may be NULL)
 *   steps_done            steps taken             (may be NULL)
 * stop_trace > 0 ends the propagation after the first step whose site
 * population sum_m Re <m|rho|m> is below stop_trace (t_max); output rows of
 * later steps are set to NaN.
 * Returns 0 on success, -1 on bad input or allocation failure. */
int oracle_propagate_ex(const oracle_params* p, const double* rho0, double dt_fs, long long nsteps,
                        long long out_every, double stop_trace, double* pops_out, double* trace_out,
                        double* eta_out, double* loss_out, double* tmean_out, double* rho_out, double* state_out,
                        long long* steps_done) {
  if (!rho0 || nsteps < 0 || out_every < 1 || !(dt_fs > 0)) return -1;
  model m;
  if (model_build(&m, p) != 0) return -1;
  int N = m.N, D = m.D;
  long nodes = m.hier.nodes;
  size_t DD = (size_t)D * D, total = DD * (size_t)nodes;
  cplx* y = (cplx*)calloc(total, sizeof(cplx));
  cplx* k = (cplx*)calloc(total, sizeof(cplx));
  cplx* z = (cplx*)calloc(total, sizeof(cplx));
  cplx* acc = (cplx*)calloc(total, sizeof(cplx));
  cplx* scratch = (cplx*)calloc(DD * (size_t)max_threads(), sizeof(cplx));
  if (!y || !k || !z || !acc || !scratch) {
    free(y); free(k); free(z); free(acc); free(scratch);
    model_free(&m);
    return -1;
  }
  /* sigma_0 = rho(0) on the site block; node 0 is n = (0,...,0) */
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) y[a * D + b] = rho0[2 * (a * N + b)] + I * rho0[2 * (a * N + b) + 1];

  const double h = dt_fs;
  const size_t rc = (size_t)(N + 1) * D + (N + 1); /* <RC|rho|RC> in node 0 */
  double xi = 0.0;                                 /* int_0^t <RC|rho|RC> dt' */
  long long o = 0, step;
  const long long nout = nsteps / out_every + 1;
  for (step = 0; step <= nsteps; ++step) {
    double tr = 0.0;
    for (int a = 0; a < N; ++a) tr += creal(y[a * D + a]);
    if (step % out_every == 0) {
      for (int a = 0; a < N; ++a)
        if (pops_out) pops_out[o * N + a] = creal(y[a * D + a]);
      if (trace_out) trace_out[o] = tr;
      if (eta_out) eta_out[o] = creal(y[rc]);
      if (loss_out) loss_out[o] = creal(y[N * D + N]);
      if (tmean_out) tmean_out[o] = (double)step * h * creal(y[rc]) - xi;
      ++o;
    }
    if (step == nsteps) break;
    if (step > 0 && stop_trace > 0 && tr < stop_trace) break;
    size_t e;
    /* k1 = f(y) */
    double xk = creal(y[rc]);
    rhs_all(&m, y, k, scratch);
    for (e = 0; e < total; ++e) { acc[e] = y[e] + (h / 6.0) * k[e]; z[e] = y[e] + (h / 2.0) * k[e]; }
    /* k2 = f(y + h/2 k1) */
    xk += 2.0 * creal(z[rc]);
    rhs_all(&m, z, k, scratch);
    for (e = 0; e < total; ++e) { acc[e] += (h / 3.0) * k[e]; z[e] = y[e] + (h / 2.0) * k[e]; }
    /* k3 = f(y + h/2 k2) */
    xk += 2.0 * creal(z[rc]);
    rhs_all(&m, z, k, scratch);
    for (e = 0; e < total; ++e) { acc[e] += (h / 3.0) * k[e]; z[e] = y[e] + h * k[e]; }
    /* k4 = f(y + h k3) */
    xk += creal(z[rc]);
    rhs_all(&m, z, k, scratch);
    for (e = 0; e < total; ++e) y[e] = acc[e] + (h / 6.0) * k[e];
    xi += (h / 6.0) * xk;
  }
  if (steps_done) *steps_done = step < nsteps ? step : nsteps;
  for (; o < nout; ++o) { /* rows after the stop */
    for (int a = 0; a < N; ++a)
      if (pops_out) pops_out[o * N + a] = NAN;
    if (trace_out) trace_out[o] = NAN;
    if (eta_out) eta_out[o] = NAN;
    if (loss_out) loss_out[o] = NAN;
    if (tmean_out) tmean_out[o] = NAN;
  }
  if (rho_out)
    for (int a = 0; a < N; ++a)
      for (int b = 0; b < N; ++b) {
        rho_out[2 * (a * N + b)] = creal(y[a * D + b]);
        rho_out[2 * (a * N + b) + 1] = cimag(y[a * D + b]);
      }
  if (state_out) memcpy(state_out, y, sizeof(cplx) * total);
  free(y); free(k); free(z); free(acc); free(scratch);
  model_free(&m);
  return 0;
}

/* The same without the trapping time and the stop rule. */
int oracle_propagate(const oracle_params* p, const double* rho0, double dt_fs, long long nsteps, long long out_every,
                     double* pops_out, double* trace_out, double* eta_out, double* loss_out, double* rho_out,
                     double* state_out) {
  return oracle_propagate_ex(p, rho0, dt_fs, nsteps, out_every, 0.0, pops_out, trace_out, eta_out, loss_out, NULL,
                             rho_out, state_out, NULL);
}
