/*
 * redfield.c -- TEST AND COMPARISON INFRASTRUCTURE ONLY (CPU).
 *
 * The secular Redfield model that Kreisbeck, Kramer, Rodriguez and Hein
 * (arXiv:1012.4382) compare the HEOM with (App. A1, "Secular Redfield
 * approximation"), written out from its definitions in plain C, FP64:
 *
 *   d rho/dt = -i [H_ex, rho]
 *              + sum_{m, omega} gamma_m(omega) D(V_m(omega)) rho          (Eq. lab6, Lamb shift dropped)
 *              + sum_m Gamma_phot,m D(|0><m|) rho                          (Eq. lab2)
 *              + sum_m Gamma_RC,m  D(|RC><m|) rho                          (Eq. lab3)
 *
 * with D(L) rho = L rho L^+ - (L^+ L rho + rho L^+ L)/2, the exciton basis
 * H_ex |M> = E_M |M>, |M> = sum_m c_m(M) |m>, and the exciton operators
 * V_m(omega) = sum_{M,N: E_M - E_N = omega} c_m*(M) c_m(N) |M><N|.  Each
 * ordered pair (M, N), M != N, is taken as its own Bohr frequency (exact
 * degeneracies of Bohr frequencies do not occur for the seeded Hamiltonians);
 * omega = 0 collects the diagonal, V_m(0) = sum_M |c_m(M)|^2 |M><M|.
 *
 * Rates, with the paper's sign convention (omega = E_M - E_N < 0 is a
 * downhill jump, which emits into the bath) and the Drude-Lorentz spectral
 * density J_m(w) = 2 lambda_m w gamma_m / (w^2 + gamma_m^2):
 *   bath_form 0 (the paper's Bose-Einstein form):
 *     gamma(omega) = 2 J(-omega) (n(-omega) + 1)   omega < 0
 *                    2 k_B T J'(0)                  omega = 0   (= 4 lambda k_B T / gamma)
 *                    2 J(omega) n(omega)            omega > 0,  n(w) = 1 / (exp(w / k_B T) - 1)
 *   bath_form 1 (the high-temperature bath the HEOM of App. A2 uses,
 *     <u(t) u(0)> = (2 lambda k_B T - i lambda gamma) exp(-gamma t)):
 *     gamma(omega) = 2 Re int_0^inf e^{-i omega t} <u(t) u(0)> dt
 *                  = (4 lambda k_B T gamma - 2 lambda gamma omega) / (gamma^2 + omega^2),
 *     the first two terms of the Bose form's expansion in omega / k_B T.
 * Reading: the paper prints 2 pi J instead of 2 J.  With its own bath
 * (the HEOM's correlation function above) the omega = 0 rate is
 * 2 Re int_0^inf <u(t) u(0)> dt = 4 lambda k_B T / gamma, while 2 pi k_B T J'(0)
 * is pi times that; the rates here are normalised to the HEOM's bath, so that
 * both methods describe the same system-bath coupling (pinned by the
 * weak-coupling agreement with the HEOM oracle in the tests).
 *
 * The state is the (N+2) x (N+2) density matrix in the basis {|M>, |0>, |RC>}
 * (excitons, ground state, reaction centre); eta = <RC|rho|RC>, the loss
 * <0|rho|0>.  Integration: classic 4th-order Runge-Kutta (as the HEOM, App. B).
 * Units: cm^-1 -> rad/fs by 2 pi c, c = 2.99792458e-5 cm/fs; k_B = 0.6950348004
 * cm^-1/K; ps^-1 / 1000 = fs^-1; hbar = 1.
 *
 * Only the test suite may load this library; nothing of the CUDA path calls it.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double kPi = 3.14159265358979323846;
static const double kCm = 2.0 * 3.14159265358979323846 * 2.99792458e-5; /* cm^-1 -> rad/fs */
static const double kBoltz = 0.6950348004;                              /* cm^-1 per K */

typedef struct {
  int N;
  const double* H;      /* N*N complex interleaved (re, im), cm^-1, Hermitian */
  const double* lam;    /* N, cm^-1 */
  const double* gam;    /* N, cm^-1 */
  double T;             /* K */
  const double* trap;   /* N, ps^-1, or NULL */
  const double* recomb; /* N, ps^-1, or NULL */
  int add_reorg;        /* 1: lambda_m added to H_mm (Eq. H_ex) */
  int bath_form;        /* 0: Bose-Einstein rates; 1: the HEOM's high-temperature bath */
} redfield_params;

/* ------------------------------------------------------- Hermitian eigen */

/* Cyclic Jacobi method for a Hermitian n x n matrix A (row-major, destroyed).
 * Each rotation first turns A_pq real with a phase on column q, then zeroes
 * it with a real plane rotation; V accumulates the unitary, so that on exit
 * A = V^+ H V is diagonal: E[k] = A_kk, eigenvector k = column k of V.
 * Eigenpairs are returned in ascending order. */
static int herm_jacobi(int n, cplx* A, double* E, cplx* V) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, scale = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a = cabs(A[i * n + j]);
        if (i != j) off += a * a;
        else scale += a * a;
      }
    if (off <= 1e-30 * (scale > 0.0 ? scale : 1.0)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double b = cabs(A[p * n + q]);
        if (b == 0.0) continue;
        const cplx ph = A[p * n + q] / b; /* A_pq = b e^{i phi} */
        const double a = creal(A[p * n + p]), d = creal(A[q * n + q]);
        const double zeta = (d - a) / (2.0 * b);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        /* U = diag(1, conj(ph)) R with R = [[c, s], [-s, c]] on (p, q) */
        const cplx upp = c, upq = s, uqp = -s * conj(ph), uqq = c * conj(ph);
        for (int k = 0; k < n; ++k) { /* A <- A U (columns p, q) */
          const cplx x = A[k * n + p], y = A[k * n + q];
          A[k * n + p] = x * upp + y * uqp;
          A[k * n + q] = x * upq + y * uqq;
        }
        for (int k = 0; k < n; ++k) { /* A <- U^+ A (rows p, q) */
          const cplx x = A[p * n + k], y = A[q * n + k];
          A[p * n + k] = conj(upp) * x + conj(uqp) * y;
          A[q * n + k] = conj(upq) * x + conj(uqq) * y;
        }
        A[p * n + q] = 0.0;
        A[q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) { /* V <- V U */
          const cplx x = V[k * n + p], y = V[k * n + q];
          V[k * n + p] = x * upp + y * uqp;
          V[k * n + q] = x * upq + y * uqq;
        }
      }
  }
  for (int i = 0; i < n; ++i) E[i] = creal(A[i * n + i]);
  /* ascending order (selection sort; n <= 24) */
  for (int i = 0; i < n; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (E[j] < E[m]) m = j;
    if (m != i) {
      const double te = E[i];
      E[i] = E[m];
      E[m] = te;
      for (int k = 0; k < n; ++k) {
        const cplx tv = V[k * n + i];
        V[k * n + i] = V[k * n + m];
        V[k * n + m] = tv;
      }
    }
  }
  return 0;
}

/* Site Hamiltonian in rad/fs (Eq. H_ex). */
static void site_hamiltonian(const redfield_params* p, cplx* H) {
  const int N = p->N;
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      double re = p->H[2 * (a * N + b)], im = p->H[2 * (a * N + b) + 1];
      if (a == b && p->add_reorg) re += p->lam[a];
      H[a * N + b] = (re + I * im) * kCm;
    }
}

/* Exciton energies E[M] (rad/fs, ascending) and V[m*N + M] = c_m(M). */
int redfield_spectrum(const redfield_params* p, double* E, double* V) {
  const int N = p->N;
  if (N < 1 || N > 24) return -1;
  cplx* A = malloc(sizeof(cplx) * N * N);
  cplx* W = malloc(sizeof(cplx) * N * N);
  if (!A || !W) {
    free(A);
    free(W);
    return -2;
  }
  site_hamiltonian(p, A);
  herm_jacobi(N, A, E, W);
  for (int i = 0; i < N * N; ++i) {
    V[2 * i] = creal(W[i]);
    V[2 * i + 1] = cimag(W[i]);
  }
  free(A);
  free(W);
  return 0;
}

/* --------------------------------------------------------------- rates */

/* gamma_m(omega) of site m (rad/fs in, 1/fs out), see the header. */
static double rate(const redfield_params* p, int m, double omega) {
  const double kT = kBoltz * p->T * kCm;
  const double lam = p->lam[m] * kCm, g = p->gam[m] * kCm;
  if (p->bath_form == 1) return (4.0 * lam * kT * g - 2.0 * lam * g * omega) / (g * g + omega * omega);
  if (omega == 0.0) return 4.0 * lam * kT / g;
  const double w = fabs(omega);
  const double J = 2.0 * lam * w * g / (w * w + g * g);
  const double n = 1.0 / expm1(w / kT);
  return omega < 0.0 ? 2.0 * J * (n + 1.0) : 2.0 * J * n;
}

/* W[M*N + K] (M != K): the rate of the jump K -> M, sum_m gamma_m(E_M - E_K)
 * |c_m(M)|^2 |c_m(K)|^2 (1/fs); W[M*N + M] = 0.  deph[m] = gamma_m(0). */
int redfield_rates(const redfield_params* p, double* Wout, double* deph) {
  const int N = p->N;
  double* E = malloc(sizeof(double) * N);
  double* V = malloc(sizeof(double) * 2 * N * N);
  if (!E || !V || redfield_spectrum(p, E, V) != 0) {
    free(E);
    free(V);
    return -1;
  }
  for (int M = 0; M < N; ++M)
    for (int K = 0; K < N; ++K) {
      double w = 0.0;
      if (M != K)
        for (int m = 0; m < N; ++m) {
          const double cM = V[2 * (m * N + M)] * V[2 * (m * N + M)] + V[2 * (m * N + M) + 1] * V[2 * (m * N + M) + 1];
          const double cK = V[2 * (m * N + K)] * V[2 * (m * N + K)] + V[2 * (m * N + K) + 1] * V[2 * (m * N + K) + 1];
          w += rate(p, m, E[M] - E[K]) * cM * cK;
        }
      Wout[M * N + K] = w;
    }
  if (deph)
    for (int m = 0; m < N; ++m) deph[m] = rate(p, m, 0.0);
  free(E);
  free(V);
  return 0;
}

/* ---------------------------------------------------------- propagation */

typedef struct {
  int N, d;
  double* E;              /* exciton energies, rad/fs */
  cplx* c;                /* c[m*N + M] = c_m(M) */
  double* W;              /* jump rates, redfield_rates */
  double* wout;           /* wout[K] = sum_M W[M][K], the total rate out of K */
  double* deph;           /* gamma_m(0) */
  double* a;              /* a[m*N + M] = |c_m(M)|^2, the diagonal of V_m(0) */
  double *gtrap, *gdec;   /* Gamma_RC,m and Gamma_phot,m, 1/fs */
} model;

static void model_free(model* m) {
  free(m->E);
  free(m->c);
  free(m->W);
  free(m->wout);
  free(m->deph);
  free(m->a);
  free(m->gtrap);
  free(m->gdec);
}

static int model_build(const redfield_params* p, model* m) {
  const int N = p->N;
  memset(m, 0, sizeof(*m));
  m->N = N;
  m->d = N + 2;
  m->E = malloc(sizeof(double) * N);
  m->c = malloc(sizeof(cplx) * N * N);
  m->W = malloc(sizeof(double) * N * N);
  m->wout = calloc(N, sizeof(double));
  m->deph = malloc(sizeof(double) * N);
  m->a = malloc(sizeof(double) * N * N);
  m->gtrap = malloc(sizeof(double) * N);
  m->gdec = malloc(sizeof(double) * N);
  double* V = malloc(sizeof(double) * 2 * N * N);
  if (!m->E || !m->c || !m->W || !m->wout || !m->deph || !m->a || !m->gtrap || !m->gdec || !V) {
    free(V);
    model_free(m);
    return -2;
  }
  if (redfield_spectrum(p, m->E, V) != 0 || redfield_rates(p, m->W, m->deph) != 0) {
    free(V);
    model_free(m);
    return -1;
  }
  for (int i = 0; i < N * N; ++i) {
    m->c[i] = V[2 * i] + I * V[2 * i + 1];
    m->a[i] = creal(m->c[i] * conj(m->c[i]));
  }
  free(V);
  for (int K = 0; K < N; ++K)
    for (int M = 0; M < N; ++M) m->wout[K] += m->W[M * N + K];
  for (int j = 0; j < N; ++j) {
    m->gtrap[j] = p->trap ? p->trap[j] * 1e-3 : 0.0;
    m->gdec[j] = p->recomb ? p->recomb[j] * 1e-3 : 0.0;
  }
  return 0;
}

/* The right-hand side for rho in the basis {|M>, |0>, |RC>} (indices 0..N-1, N, N+1). */
static void rhs(const model* m, const cplx* r, cplx* out) {
  const int N = m->N, d = m->d;
  /* -i [H, rho]: the exciton energies, 0 for |0> and |RC> */
  for (int K = 0; K < d; ++K)
    for (int L = 0; L < d; ++L) {
      const double eK = K < N ? m->E[K] : 0.0, eL = L < N ? m->E[L] : 0.0;
      out[K * d + L] = -I * (eK - eL) * r[K * d + L];
    }
  /* jumps K -> M (omega != 0): W[M][K] (rho_KK |M><M| - {|K><K|, rho} / 2) */
  for (int M = 0; M < N; ++M)
    for (int K = 0; K < N; ++K)
      if (M != K) out[M * d + M] += m->W[M * N + K] * r[K * d + K];
  for (int K = 0; K < d; ++K)
    for (int L = 0; L < d; ++L) {
      const double wK = K < N ? m->wout[K] : 0.0, wL = L < N ? m->wout[L] : 0.0;
      out[K * d + L] -= 0.5 * (wK + wL) * r[K * d + L];
    }
  /* omega = 0: gamma_m(0) D(V_m(0)), V_m(0) = sum_M |c_m(M)|^2 |M><M| */
  for (int K = 0; K < d; ++K)
    for (int L = 0; L < d; ++L) {
      double s = 0.0;
      for (int j = 0; j < N; ++j) {
        const double aK = K < N ? m->a[j * N + K] : 0.0, aL = L < N ? m->a[j * N + L] : 0.0;
        s += m->deph[j] * (aK * aL - 0.5 * (aK * aK + aL * aL));
      }
      out[K * d + L] += s * r[K * d + L];
    }
  /* trapping and radiative decay: Gamma D(|X><j|) rho = Gamma (<j|rho|j> |X><X| - {|j><j|, rho} / 2) */
  for (int j = 0; j < N; ++j) {
    const double gt = m->gtrap[j], gd = m->gdec[j];
    if (gt == 0.0 && gd == 0.0) continue;
    const cplx* cj = m->c + j * N;
    cplx pj = 0.0; /* <j|rho|j> = sum_KL c_j(K) rho_KL conj(c_j(L)) */
    for (int K = 0; K < N; ++K)
      for (int L = 0; L < N; ++L) pj += cj[K] * r[K * d + L] * conj(cj[L]);
    out[(N + 1) * d + (N + 1)] += gt * pj;
    out[N * d + N] += gd * pj;
    /* {P, rho} with P_KL = conj(c_j(K)) c_j(L) on the exciton block */
    for (int K = 0; K < d; ++K)
      for (int L = 0; L < d; ++L) {
        cplx s = 0.0;
        if (K < N)
          for (int Q = 0; Q < N; ++Q) s += conj(cj[K]) * cj[Q] * r[Q * d + L];
        if (L < N)
          for (int Q = 0; Q < N; ++Q) s += r[K * d + Q] * conj(cj[Q]) * cj[L];
        out[K * d + L] -= 0.5 * (gt + gd) * s;
      }
  }
}

/* Classic RK4 from rho(0) (site basis, N*N complex interleaved) for nsteps
 * steps of dt fs.  Rows at steps 0, out_every, ...: pops[row*N + m] = <m|rho|m>,
 * trace[row] = sum_m pops, eta[row] = <RC|rho|RC>, loss[row] = <0|rho|0>
 * (each may be NULL).  Returns 0, or < 0 on bad input / no memory. */
int redfield_propagate(const redfield_params* p, const double* rho0, double dt, long long nsteps, long long out_every,
                       double* pops, double* trace, double* eta, double* loss) {
  if (!p || !rho0 || !(dt > 0.0) || nsteps < 0 || out_every < 1) return -1;
  model m;
  const int rc = model_build(p, &m);
  if (rc != 0) return rc;
  const int N = m.N, d = m.d, D = d * d;
  cplx* y = calloc(D, sizeof(cplx));
  cplx* k = malloc(sizeof(cplx) * D);
  cplx* z = malloc(sizeof(cplx) * D);
  cplx* acc = malloc(sizeof(cplx) * D);
  if (!y || !k || !z || !acc) {
    free(y);
    free(k);
    free(z);
    free(acc);
    model_free(&m);
    return -2;
  }
  /* rho(0) into the exciton basis: <K|rho|L> = sum_mn conj(c_m(K)) rho_mn c_n(L) */
  for (int K = 0; K < N; ++K)
    for (int L = 0; L < N; ++L) {
      cplx s = 0.0;
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b)
          s += conj(m.c[a * N + K]) * (rho0[2 * (a * N + b)] + I * rho0[2 * (a * N + b) + 1]) * m.c[b * N + L];
      y[K * d + L] = s;
    }
  long long row = 0;
  for (long long t = 0; t <= nsteps; ++t) {
    if (t % out_every == 0) {
      double tr = 0.0;
      for (int j = 0; j < N; ++j) {
        cplx pj = 0.0;
        for (int K = 0; K < N; ++K)
          for (int L = 0; L < N; ++L) pj += m.c[j * N + K] * y[K * d + L] * conj(m.c[j * N + L]);
        if (pops) pops[row * N + j] = creal(pj);
        tr += creal(pj);
      }
      if (trace) trace[row] = tr;
      if (eta) eta[row] = creal(y[(N + 1) * d + (N + 1)]);
      if (loss) loss[row] = creal(y[N * d + N]);
      ++row;
    }
    if (t == nsteps) break;
    /* classic RK4: c = 0, 1/2, 1/2, 1; b = 1/6, 1/3, 1/3, 1/6 */
    static const double cs[4] = {0.0, 0.5, 0.5, 1.0}, bs[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    memcpy(acc, y, sizeof(cplx) * D);
    memcpy(z, y, sizeof(cplx) * D);
    for (int s = 0; s < 4; ++s) {
      rhs(&m, z, k);
      for (int i = 0; i < D; ++i) acc[i] += bs[s] * dt * k[i];
      if (s < 3)
        for (int i = 0; i < D; ++i) z[i] = y[i] + cs[s + 1] * dt * k[i];
    }
    memcpy(y, acc, sizeof(cplx) * D);
  }
  free(y);
  free(k);
  free(z);
  free(acc);
  model_free(&m);
  (void)kPi;
  return 0;
}
