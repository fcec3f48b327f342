/*
 * heom.h -- C ABI of libheom, a GB300 (sm_103a) implementation of the
 * hierarchical equations of motion (HEOM) for excitonic energy transfer with
 * trapping, as set up by Kreisbeck, Kramer, Rodriguez and Hein,
 * "High-performance solution of hierarchical equations of motions for studying
 * energy-transfer in light-harvesting complexes" (arXiv:1012.4382).
 *
 * What the library computes (paper passages in brackets):
 *   * system: N exciton sites with a Hermitian Hamiltonian H (Sec. "Model",
 *     Eq. H_ex); one Drude-Lorentz bath per site with reorganisation energy
 *     lambda_m and correlation rate gamma_m in the high-temperature form
 *     (App. A2, Eq. gamma and the S(t), chi(t) forms);
 *   * trapping into the reaction centre at rate Gamma_RC,m and radiative decay
 *     to the ground state at rate Gamma_phot,m (App. A1, Eqs. lab2, lab3),
 *     carried as the anti-Hermitian part -(i/2) diag(Gamma_RC + Gamma_phot) of
 *     an effective Hamiltonian, which the paper states is equivalent
 *     (App. A1, end);
 *   * the hierarchy of auxiliary density matrices sigma_n, |n| <= K = N_max
 *     (App. A2, Eqs. labsevena and lab8, truncation at its end), propagated
 *     with 4th-order Runge-Kutta (App. B);
 *   * the efficiency eta = <RC|rho(t)|RC> (Eq. eta), obtained as the time
 *     integral of sum_m Gamma_RC,m <m|rho|m> integrated by the same RK4, and
 *     the radiative loss <0|rho|0> likewise;
 *   * the trapping time <t> (Eq. trappingtime) and the t_max stop rule of the
 *     section on trapping times (heom_trapping_time, heom_set_stop);
 *   * optionally, the lowest-order quantum correction to the high-temperature
 *     baths (HEOM_FLAG_LOW_TEMP), and the scaled hierarchy the introduction
 *     mentions (HEOM_FLAG_SCALED).
 * Readings taken where the paper is ambiguous: damping term
 * -sum_m n_m gamma_m sigma_n (the printed sign in lab8 would be unstable);
 * theta_m = i (2 lambda_m k_B T V_m^x - i lambda_m gamma_m V_m^o) (the printed
 * temperature factor is dimensionally inconsistent).
 *
 * Units at this boundary: energies and couplings in cm^-1, rates in ps^-1,
 * temperature in K, time in fs.  Complex arrays are interleaved (re, im)
 * doubles, row-major.
 *
 * Ownership: every pointer argument is owned by the caller and only read or
 * written during the call (or, for the *_device variants, until the work
 * queued on the context's stream has finished).  Contexts own all device
 * memory they allocate; it stays resident between calls (App. B keeps the
 * sigma-matrices on the GPU and copies only rho out).
 *
 * Errors: every function returns HEOM_OK (0) or a positive HEOM_E* code and
 * sets a thread-local message readable with heom_last_error().  Nothing throws
 * across this boundary.  There is no CPU fallback: without a usable CUDA
 * device, functions that need one return HEOM_ECUDA.
 */
#ifndef HEOM_H
#define HEOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define HEOM_OK 0
#define HEOM_EINVAL 1       /* invalid argument (message says which) */
#define HEOM_ENOMEM 2       /* host or device allocation failed */
#define HEOM_ECUDA 3        /* CUDA runtime error or no usable device */
#define HEOM_ETIMEOUT 4     /* a bounded device-side wait expired; results of that call are invalid */
#define HEOM_EUNSUPPORTED 5 /* valid request this build does not implement (message says what) */
#define HEOM_ENONFINITE 6   /* a population, the trace, eta or the loss came out NaN or infinite (checked at
                               every output row and at the end of each propagate call): the run diverged,
                               e.g. a time step too large for the bath rates, or the initial state was not
                               finite; the call's results are not usable */
#define HEOM_EINTERNAL 7    /* an internal consistency check failed (the library's own node tables did not
                               pass heom_check_node_tables' test after upload); message says where */

/* precision of the propagation */
#define HEOM_FP64 0         /* every array and every operation in double precision */
#define HEOM_FP32_MIXED 1   /* auxiliary matrices and right-hand side in float; rho's RK4
                               accumulation and the eta and loss integrals in float-float
                               (about 48-bit significand; FP64 runs at 1/64 of the FP32 rate
                               on GB300); populations, eta and loss returned in double */

/* truncation of the hierarchy at |n| = K (the paper only says "truncate") */
#define HEOM_TERM_NONE 0    /* sigma_{n+e_j} = 0 beyond the last level */
#define HEOM_TERM_MARKOV 1  /* sigma_{n+e_j} ~ (n_j+1) theta_j sigma_n / (sum_k n_k gamma_k + gamma_j) */

/* heom_params.flags */
#define HEOM_FLAG_LOW_TEMP 1 /* lowest-order quantum correction to the high-temperature baths (the
                                paper includes it, citing Ishizaki and Fleming, without giving it):
                                -sum_j c_j V_j^x V_j^x sigma_n on every node, c_j the Markovian
                                weight of the Matsubara terms, 2 lambda_j k_B T / gamma_j -
                                lambda_j cot(gamma_j / (2 k_B T)) (hbar = 1) */
#define HEOM_FLAG_SCALED 2   /* scaled hierarchy (the paper's introduction names it, citing Zhu et al.,
                                without the formula): the auxiliaries are stored as
                                sigma~_n = sigma_n / prod_j sqrt(n_j! s_j^{n_j}), s_j = |2 lambda_j k_B T
                                - i lambda_j gamma_j| (1 where lambda_j = 0), the rescaling of Shi et al.,
                                J. Chem. Phys. 130, 084105 (2009).  The up link of site j then carries
                                sqrt((n_j+1) s_j) and the down link sqrt(n_j / s_j) instead of 1 and n_j;
                                rho, eta, loss and <t> are unchanged up to rounding, while the
                                auxiliaries of different depths become of comparable size (the
                                first step towards filtering small ones, which this library does
                                not do).  heom_get_state/heom_set_state exchange sigma~_n.  For
                                N <= 8 not with the register node view (node_threads 1 or 2) nor
                                with mode 2: the default launch shape avoids them, and a launch
                                shape set to them fails at propagate time with HEOM_EUNSUPPORTED */

/* largest supported number of sites and of hierarchy nodes per instance */
#define HEOM_MAX_SITES 24
#define HEOM_MAX_NODES 16777215

typedef struct heom_params {
  int32_t N;                 /* number of sites, 1..HEOM_MAX_SITES */
  int32_t K;                 /* hierarchy depth N_max, >= 0 */
  const double* H;           /* N*N complex Hamiltonian (cm^-1), must be Hermitian */
  const double* lambda;      /* N reorganisation energies (cm^-1), >= 0 */
  const double* gamma;       /* N bath correlation rates (cm^-1), > 0 */
  double T_kelvin;           /* temperature (K), > 0 */
  const double* trap_rate;   /* N trapping rates Gamma_RC (ps^-1), >= 0; NULL = none */
  const double* recomb_rate; /* N radiative decay rates Gamma_phot (ps^-1), >= 0; NULL = none */
  int32_t precision;         /* HEOM_FP64 or HEOM_FP32_MIXED */
  int32_t terminator;        /* HEOM_TERM_NONE or HEOM_TERM_MARKOV */
  int32_t add_reorg_to_H;    /* 0: H used as given; 1: lambda_m added to H_mm (Eq. H_ex) */
  int32_t flags;             /* 0 or an OR of HEOM_FLAG_LOW_TEMP and HEOM_FLAG_SCALED */
} heom_params;

typedef struct heom_ctx heom_ctx;     /* one propagated hierarchy */
typedef struct heom_batch heom_batch; /* many independent hierarchies */

/* ---------------------------------------------------------------- host-only */

/* Number of hierarchy nodes C(N+K, K) (App. B, N_tot).  HEOM_EINVAL when N is
 * outside 1..HEOM_MAX_SITES, K < 0, or the count exceeds HEOM_MAX_NODES. */
int heom_num_nodes(int32_t N, int32_t K, int64_t* out);

/* Writes the library's node order and neighbour tables (App. B: each sigma
 * has 2N neighbours).  Nodes are ordered by level |n|, then lexicographically
 * descending (n_1 first); node 0 is n = 0.  For nodes i and sites j:
 *   multi[i*N + j] = n_j,
 *   up[i*N + j]    = index of n + e_j, or -1 when |n| = K,
 *   down[i*N + j]  = index of n - e_j, or -1 when n_j = 0.
 * Each output may be NULL.  Arrays hold nodes*N int32 values. */
int heom_build_index(int32_t N, int32_t K, int32_t* multi, int32_t* up, int32_t* down);

/* Device-side bounds and consistency check of node tables in the layout the
 * kernels read (App. B: sigma_n couples to sigma_{n+e_j} and sigma_{n-e_j}):
 * d_up and d_dn are DEVICE int32 arrays [N][Mpad], element (j, n) at
 * j*Mpad + n; d_up holds the index of n + e_j or -1, d_dn holds
 * (n_j << 24) | index of n - e_j, or -1 when n_j = 0.  The test, per node
 * n < M and site j: an up link is -1 or a later node u < M whose down link on
 * site j is n with n_j(u) = n_j(n) + 1; a down link is -1 or an earlier node
 * with n_j >= 1 whose up link on site j is n; nodes M..Mpad-1 have no links.
 * A linked entry is read only after its index is found in range, so corrupt
 * tables are read in bounds.  Every context, batch and server runs this test
 * on the tables it uploads (full or filtered) and fails with HEOM_EINTERNAL if
 * they do not pass.  Returns HEOM_OK, or HEOM_EINVAL with *bad_node (may be
 * NULL) = the smallest offending node (-1 when the tables pass).  Blocking, on
 * the legacy default stream; the arrays are only read. */
int heom_check_node_tables(const int32_t* d_up, const int32_t* d_dn, int64_t M, int32_t Mpad, int32_t N,
                           int64_t* bad_node);

/* Device memory hooks.  When set, every device allocation of the library goes
 * through alloc/release (e.g. a framework's caching allocator); otherwise
 * cudaMalloc/cudaFree are used.  alloc returns NULL on failure.  Set before
 * creating contexts; contexts keep the hooks they were created with. */
typedef void* (*heom_alloc_fn)(size_t bytes, void* user);
typedef void (*heom_free_fn)(void* ptr, size_t bytes, void* user);
int heom_set_allocator(heom_alloc_fn alloc, heom_free_fn release, void* user);

/* Thread-local description of the last error on this thread ("" if none). */
const char* heom_last_error(void);

/* Self-test of the bounded device-side wait that every grid-wide stage
 * barrier uses (the wait behind HEOM_ETIMEOUT): one thread on the current
 * device waits for a counter that nothing raises, with a limit of limit_ms
 * (0 < limit_ms <= 1000) instead of the barrier's 2 s.  The counter is preset
 * to 2^32 - 1 and the awaited count is 1, past the 32-bit wrap, so the probe
 * also shows that the wait compares counts in a wrap-safe way.  *timed_out (may be
 * NULL) is 1 when the wait gave up and raised its status bit, as it must;
 * *waited_ms (may be NULL) is the probe's device time.  Nothing is faulted:
 * the kernel returns and the device stays usable.  HEOM_ECUDA without a
 * device.  Blocking; allocates and frees 256 device bytes. */
int heom_selftest_bounded_wait(double limit_ms, int32_t* timed_out, double* waited_ms);

/* ------------------------------------------------------- single hierarchy */

/* Creates a context: validates params, converts units, builds the node tables,
 * allocates the device state on the current CUDA device and sets rho(0) =
 * |0><0| (site index 0).  Paper: the system Hamiltonian H_ex of Sec. "Model"
 * (Eq. H_ex; lambda_m added to the site energies only with add_reorg_to_H);
 * the trapping and radiative-decay rates of App. A1 (Eqs. lab2, lab3), taken
 * in the equivalent anti-Hermitian form -(i/2) diag(Gamma_RC + Gamma_phot) of
 * H that the end of App. A1 states; the bath coefficients of App. A2
 * (theta_m, Eq. labsevena) and the hierarchy of all n with |n| <= K = N_max
 * (Eq. lab8 and the truncation at the end of App. A2), C(N+K, K) nodes with
 * 2N neighbour links each (App. B).  cuda_stream is a cudaStream_t (NULL: the legacy
 * default stream); all device work of the context is ordered on it.  The
 * params and their arrays may be freed after the call. */
int heom_create(const heom_params* params, void* cuda_stream, heom_ctx** out);

/* Sets rho(0) from a host N*N complex Hermitian matrix (|rho - rho^+| must be
 * <= 1e-12 elementwise, else HEOM_EINVAL), zeroes every auxiliary matrix
 * (App. A2: "the sigma-matrices are initially set to zero") and the eta and
 * loss integrals.  Blocking. */
int heom_set_rho0(heom_ctx* ctx, const double* rho0);

/* Same from a device buffer of N*N complex doubles; asynchronous on the
 * context's stream, no host synchronisation, no validation of hermiticity. */
int heom_set_rho0_device(heom_ctx* ctx, const double* d_rho0);

/* Advances the state by nsteps RK4 steps of dt_fs and records, at steps
 * 0, out_every, 2*out_every, ... of this call (nout = nsteps/out_every + 1
 * rows), the site populations pops_out[nout*N], their sum trace_out[nout]
 * and eta_out[nout] (each may be NULL).  Resumable: a later call continues
 * from the state this one left.  Blocking; returns HEOM_ETIMEOUT if a device
 * wait expired and HEOM_ENONFINITE if a row came out NaN or infinite.
 * Paper: every step is one 4th-order Runge-Kutta step (App. B) of the whole
 * hierarchy, Eq. lab8 with the damping sign read as -sum_m n_m gamma_m, the
 * up links i V_m^x sigma_{n+e_m}, the down links n_m theta_m sigma_{n-e_m}
 * (Eq. labsevena) and the commutator with the non-Hermitian H of App. A1;
 * the sigma matrices stay on the device between calls and only the
 * populations and eta are copied out (App. B); eta is the integral of
 * Eq. eta carried as an extra row of the RK4 system. */
int heom_propagate(heom_ctx* ctx, double dt_fs, int64_t nsteps, int64_t out_every, double* pops_out,
                   double* trace_out, double* eta_out);

/* Same with device output buffers d_pops[nout*N] and d_eta_loss[nout*2]
 * ((eta, loss) per row); either may be NULL.  Asynchronous on the context's
 * stream; call heom_synchronize() to wait and to collect device errors. */
int heom_propagate_device(heom_ctx* ctx, double dt_fs, int64_t nsteps, int64_t out_every, double* d_pops,
                          double* d_eta_loss);

/* Waits for the context's stream and reports HEOM_ETIMEOUT / HEOM_ENONFINITE /
 * HEOM_ECUDA raised by work queued since the last check. */
int heom_synchronize(heom_ctx* ctx);

/* eta = <RC|rho|RC> (Eq. eta) and the radiative loss <0|rho|0> at the current
 * time; loss_out may be NULL.  Blocking. */
int heom_efficiency(heom_ctx* ctx, double* eta_out, double* loss_out);

/* Trapping time <t> = int_0^t t' d<RC|rho|RC>/dt' dt' (Eq. trappingtime,
 * Sec. "Trapping time for different reorganization energies") up to the
 * current time t (fs from the last heom_set_rho0), evaluated as
 * t eta(t) - int_0^t eta dt' with the integral carried as one more component
 * of the RK4 system.  steps_done (may be NULL) receives the number of steps
 * the last propagate call took (fewer than asked when the stop rule ended it).
 * heom_set_state restarts the integral (t and int eta dt' set to 0).
 * Blocking. */
int heom_trapping_time(heom_ctx* ctx, double* t_mean_fs, int64_t* steps_done);

/* The stop rule of the same section: with stop_trace > 0, the following
 * propagate calls end after the first step whose site population
 * sum_m Re <m|rho|m> is below stop_trace (t_max; the paper uses 1e-5).  The
 * check runs after every step but the last of a call; output rows of later
 * steps are set to NaN.  0 (the default) turns it off; negative or non-finite
 * values are HEOM_EINVAL. */
int heom_set_stop(heom_ctx* ctx, double stop_trace);

/* Current reduced density matrix on the sites, N*N complex.  Blocking.
 * Paper: rho = sigma_0, the root of the hierarchy (App. A2), copied from the
 * device, where the hierarchy lives (App. B). */
int heom_get_rho(heom_ctx* ctx, double* rho_out);

/* Full state for checkpoints and checks: every node's N*N complex matrix in
 * the order of heom_build_index (nodes*N*N complex doubles), plus eta and
 * loss in extra[2] (may be NULL).  heom_set_state restores it exactly
 * (FP64) or to float rounding (auxiliaries in HEOM_FP32_MIXED).  Blocking. */
int heom_get_state(heom_ctx* ctx, double* state_out, double* extra);
int heom_set_state(heom_ctx* ctx, const double* state_in, const double* extra);

/* Number of nodes of the context's hierarchy. */
int heom_ctx_num_nodes(const heom_ctx* ctx, int64_t* out);

/* Launch shape.  mode 0: one thread-block cluster of `team_ctas` CTAs
 * (1..16) per hierarchy, state in device memory, hardware cluster barriers
 * between RK4 stages; mode 1: the whole GPU per hierarchy (cooperative launch,
 * software grid barrier with a bounded wait); mode 2 (HEOM_FP32_MIXED only):
 * like mode 0 but the whole hierarchy lives in the cluster's distributed
 * shared memory during the call (HEOM_EINVAL at propagate time if it does
 * not fit in team_ctas CTAs); mode 3 (N <= 8, single hierarchies): the
 * dataflow engine -- the whole GPU, no grid barrier: each CTA keeps a slice
 * of nodes in shared memory, one thread per unit (an off-diagonal pair or a
 * diagonal element) of a node, and neighbour values travel as stage-tagged
 * words that a thread waits for (bounded, HEOM_ETIMEOUT) one by one.  In
 * mode 3 team_ctas is the number of nodes each thread carries, 1..6 (more
 * than one: real H and 4..8 sites only, HEOM_EUNSUPPORTED otherwise), which
 * lets a hierarchy of up to about 6800 nodes (N = 7) run with all CTAs
 * resident.  Mode 3 is the default for one hierarchy of 256 nodes or more
 * when all its CTAs fit on the GPU at once with some number of nodes per
 * thread (the fewest that fit).  block_threads: multiple of 32, 64..512
 * (64..256 for HEOM_FP64, whose kernels are compiled for that register budget);
 * in mode 3 the CTA size, at most 384 with one node per thread and 256 with
 * more, of which every N(N+1)/2 threads make a row of team_ctas nodes (N = 7,
 * one node per thread: 12 nodes in 336 threads); a call whose CTAs cannot all
 * be resident fails with HEOM_EINVAL.  Switching between mode 3 and the
 * other modes without giving team_ctas or block_threads resets them to that
 * family's default.  node_threads: threads sharing one node's matrix, 1..32
 * (1 or 2 keep the node's matrix in registers; not used by mode 3).  A
 * negative mode or a non-positive value keeps the current setting. */
int heom_set_launch(heom_ctx* ctx, int32_t mode, int32_t team_ctas, int32_t block_threads, int32_t node_threads);
int heom_get_launch(const heom_ctx* ctx, int32_t* mode, int32_t* team_ctas, int32_t* block_threads,
                    int32_t* node_threads);

/* Autotuner: times `trial_steps` steps for each candidate launch shape on
 * this context's hierarchy, keeps the fastest and restores the state it
 * found.  best_us_per_step may be NULL. */
int heom_autotune(heom_ctx* ctx, int64_t trial_steps, double* best_us_per_step);

/* ------------------------------------------------- filtered hierarchies */

/* The introduction names the scaled HEOM as the way to need fewer auxiliary
 * matrices (citing Zhu et al.; no formula is given).  In the scaled
 * hierarchy (HEOM_FLAG_SCALED) auxiliaries of every depth are of comparable
 * size, so the ones that stay small can be left out: the library selects a
 * node set from their magnitudes and propagates the hierarchy restricted to
 * it with the same engines (the node tables shrink; nothing else changes).
 *
 * heom_node_magnitudes: node_max[i] = max_ab |sigma_i,ab| (sigma~ for a scaled
 * context) of the context's current state, i in the order of
 * heom_build_index (of the subset for a filtered context).  Blocking.
 *
 * heom_filter_select (host only; delta >= 0, infinity keeping the root alone,
 * HEOM_EINVAL for a negative or NaN delta): keep[i] = 1 for every node with
 * node_max[i] >= delta, the root, and every n - e_j of a kept n (closed downwards, so that
 * each kept auxiliary stays linked to rho through kept nodes); node_max and
 * keep hold one value per node of the full hierarchy C(N+K, K), in
 * heom_build_index order.  Typical use: propagate the full scaled hierarchy
 * for a pilot time, take the elementwise maximum of heom_node_magnitudes over
 * a few snapshots, select, and continue on the filtered context.  The error
 * of the filtered propagation shrinks with delta (FMO-like N = 7, depth 6,
 * 2 ps pilot, delta = 1e-5: 71 % of the nodes kept, populations within
 * 1.7e-6 over 10 ps).
 *
 * heom_create_subset: heom_create on the hierarchy restricted to the nodes with
 * keep[i] != 0 (keep as above, one flag per node of the full hierarchy).  The
 * set must contain the root and be closed downwards (HEOM_EINVAL otherwise);
 * links to removed nodes are truncated like links beyond depth K, and only
 * the plain truncation is supported (HEOM_EUNSUPPORTED with HEOM_TERM_MARKOV).
 * heom_ctx_num_nodes, heom_get_state and heom_set_state then count and order
 * the kept nodes only (in heom_build_index order). */
int heom_node_magnitudes(heom_ctx* ctx, double* node_max);
int heom_filter_select(int32_t N, int32_t K, const double* node_max, double delta, uint8_t* keep);
int heom_create_subset(const heom_params* params, const uint8_t* keep, void* cuda_stream, heom_ctx** out);

/* Releases the context and its device memory (NULL-safe).  Paper: the
 * device-resident sigma matrices and neighbour tables of App. B. */
void heom_destroy(heom_ctx* ctx);

/* -------------------------------------------------------------- batches */

/* count independent hierarchies propagated together: every instance with
 * the same N runs in one persistent launch, one thread-block cluster per
 * instance at a time.  All instances must have the same precision.
 * Instances start from rho(0) = |0><0|.  Each instance is the model of
 * heom_create (Sec. "Model", App. A1, App. A2); the batch itself has no
 * counterpart in the paper, which propagates one hierarchy at a time
 * (its parameter scans of Secs. 3-5 are such batches). */
int heom_batch_create(const heom_params* params, int32_t count, void* cuda_stream, heom_batch** out);
int heom_batch_count(const heom_batch* b, int32_t* count);

/* A batch of filtered hierarchies (see heom_create_subset): keep[i] holds the
 * node flags of instance i over its full hierarchy, or NULL for the full
 * hierarchy.  heom_batch_num_nodes gives an instance's node count and
 * heom_batch_node_magnitudes its per-node max |sigma_ab| (as
 * heom_node_magnitudes; blocking). */
int heom_batch_create_subset(const heom_params* params, const uint8_t* const* keep, int32_t count, void* cuda_stream,
                             heom_batch** out);
int heom_batch_num_nodes(const heom_batch* b, int32_t i, int64_t* out);
int heom_batch_node_magnitudes(heom_batch* b, int32_t i, double* node_max);

/* rho0_all: the count initial matrices concatenated (sum_i N_i^2 complex). */
int heom_batch_set_rho0(heom_batch* b, const double* rho0_all);

/* Advances instance i by nsteps[i] steps of dt_fs[i] (arrays of count;
 * nsteps may hold 0).  Outputs, each may be NULL, concatenated over
 * instances: pops_out rows of N_i (nout_i = nsteps[i]/out_every + 1 rows per
 * instance), eta_out nout_i values per instance.  Blocking. */
int heom_batch_propagate(heom_batch* b, const double* dt_fs, const int64_t* nsteps, int64_t out_every,
                         double* pops_out, double* eta_out);

/* Asynchronous form with device outputs at the same offsets (d_eta_loss holds
 * two doubles per row). */
int heom_batch_propagate_device(heom_batch* b, const double* dt_fs, const int64_t* nsteps, int64_t out_every,
                                double* d_pops, double* d_eta_loss);
int heom_batch_synchronize(heom_batch* b);

/* eta_out[count], loss_out[count] (may be NULL); blocking. */
int heom_batch_efficiency(heom_batch* b, double* eta_out, double* loss_out);
/* Per instance, as heom_trapping_time / heom_set_stop: t_mean_fs[count],
 * steps_done[count] (may be NULL); the stop rule applies to every instance. */
int heom_batch_trapping_time(heom_batch* b, double* t_mean_fs, int64_t* steps_done);
int heom_batch_set_stop(heom_batch* b, double stop_trace);
int heom_batch_get_rho(heom_batch* b, int32_t i, double* rho_out);

/* Launch shape of the batch's persistent launches (see heom_set_launch;
 * mode 0 or 2, negative keeps the current mode). */
int heom_batch_set_launch(heom_batch* b, int32_t mode, int32_t team_ctas, int32_t block_threads,
                          int32_t node_threads);
/* Autotuner for a batch: times `trial_steps` steps of every instance for each
 * candidate shape (mode 0 and, in HEOM_FP32_MIXED, mode 2; 256 or 512
 * threads; 1-16 team CTAs; node_threads 1-8), one shape for all site counts;
 * shapes that cannot run every instance are skipped.  Keeps the fastest,
 * restores the state it found and returns that shape's time in *best_ms (may
 * be NULL).  Holds a copy of the batch's state meanwhile. */
int heom_batch_autotune(heom_batch* b, int64_t trial_steps, double* best_ms);

/* The launch shape used for the batch's instances with N sites (one launch
 * per site count); HEOM_EINVAL when the batch has no such instance.  Each
 * output may be NULL. */
int heom_batch_get_launch(const heom_batch* b, int32_t N, int32_t* mode, int32_t* team_ctas, int32_t* block_threads,
                          int32_t* node_threads);

void heom_batch_destroy(heom_batch* b);

/* CUDA graph of one batch propagate call (no counterpart in the paper: a
 * serving-side way to replay a fixed persistent launch without host work).
 * heom_batch_graph_create captures what heom_batch_propagate_device(b, dt_fs,
 * nsteps, out_every, d_pops, d_eta_loss) would launch -- step counts, time
 * steps, output pointers and launch shapes are fixed in the graph -- without
 * running it.  Each heom_graph_launch then runs that propagation once more on
 * the batch's stream (asynchronously; heom_batch_synchronize waits), continuing
 * from the current state and overwriting the same output rows; heom_batch_set_rho0
 * between launches restarts the instances.  Launch modes 0 and 2 only (mode 1
 * gives HEOM_EUNSUPPORTED).  The batch must outlive its graphs; later
 * heom_batch_set_launch / heom_batch_set_stop calls do not change a graph.
 * heom_graph_destroy is NULL-safe. */
typedef struct heom_graph heom_graph;
int heom_batch_graph_create(heom_batch* b, const double* dt_fs, const int64_t* nsteps, int64_t out_every,
                            double* d_pops, double* d_eta_loss, heom_graph** out);
int heom_graph_launch(heom_graph* g);
void heom_graph_destroy(heom_graph* g);

/* -------------------------------------------------------------- serving */

/* Continuous batching of propagation requests (N <= 8).  The server owns a
 * device-memory budget (device_bytes, allocated once), a pinned host buffer
 * for results (host_bytes) and `streams` CUDA streams.  heom_server_submit
 * queues a request; each heom_server_progress call
 *   - marks finished every running request whose thread block has ended (the
 *     kernel writes its populations and eta rows straight into pinned host
 *     memory and then raises a flag there),
 *   - retires launches whose device work has ended, returning their memory
 *     and stream, and
 *   - admits the queued requests that fit in the budget, in arrival order,
 *     into new launches on free streams, one per (precision, N, team shape):
 *     one team of thread blocks per request.  A request whose launch would
 *     need a stream when none is free keeps its place; later requests that
 *     join a launch formed in the same call go ahead of it.
 * So requests that arrive while others run start at the next progress call
 * and overlap with them on the device, and each completes as soon as its own
 * block is done.  Node tables are cached per (N, K).  Calls are serialised by
 * an internal mutex; heom_server_progress never blocks on the device.
 * Request states: 0 queued, 1 running, 2 done, 3 cancelled, 4 failed. */
typedef struct heom_server heom_server;
int heom_server_create(size_t device_bytes, size_t host_bytes, int32_t streams, heom_server** out);

/* Queues one propagation from rho0 (host N*N complex Hermitian) of nsteps
 * steps of dt_fs with outputs every out_every steps.  HEOM_ENOMEM if the
 * request can never fit in the budgets; HEOM_EINVAL for malformed input.
 * params and rho0 are copied. */
int heom_server_submit(heom_server* s, const heom_params* params, const double* rho0, double dt_fs, int64_t nsteps,
                       int64_t out_every, int64_t* request_id);

/* Retires finished requests and launches and admits queued requests;
 * completed (may be NULL) receives the number of requests finished by this
 * call. */
int heom_server_progress(heom_server* s, int32_t* completed);
int heom_server_status(heom_server* s, int64_t request_id, int32_t* state);

/* Results of a finished request: pops_out[nout*N], eta_out[nout],
 * loss_out[nout] (each may be NULL), times_out[2] = seconds from submission
 * to launch and to the progress call that saw it finish.  A failed request
 * (state 4) returns HEOM_ENONFINITE when its rows came out NaN or infinite,
 * HEOM_ECUDA when its launch failed. */
int heom_server_result(heom_server* s, int64_t request_id, double* pops_out, double* eta_out, double* loss_out,
                       double* times_out);

/* Forgets a finished, failed or cancelled request. */
int heom_server_release(heom_server* s, int64_t request_id);

/* Cancels a queued request (running requests cannot be cancelled). */
int heom_server_cancel(heom_server* s, int64_t request_id);
int heom_server_stats(heom_server* s, int64_t* queued, int64_t* running, int64_t* bytes_in_use);

/* Waits for all device work of the server, then frees everything. */
void heom_server_destroy(heom_server* s);

/* --------------------------------------------- allocation-free propagation */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot call cudaMalloc -- code that runs under a device-memory budget fixed
 * before it starts, or inside a host framework that owns every device
 * allocation -- and so cannot create a heom_ctx.
 *
 * One complete propagation from rho(0), like heom_create + heom_set_rho0 +
 * heom_propagate_device on a fresh context, that allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine, no host heap.  All
 * device working memory (node tables, coefficients, the state and both RK4
 * stage buffers, launch descriptor, status words) lives in one file-scope
 * device array of HEOM_STATIC_SCRATCH_BYTES, which every GPU that loads the
 * library holds until the process exits.  Problems that need more than that
 * (N = 7: up to depth 8 in HEOM_FP64 and depth 9 in HEOM_FP32_MIXED; N = 8:
 * depth 6 and 7) are
 * rejected with HEOM_EINVAL and a message giving the bytes needed; only
 * N <= 8 is supported, and HEOM_FLAG_SCALED is not (HEOM_EUNSUPPORTED).
 *
 * Inputs: params (host, read during the call) and d_rho0, a device buffer of
 * N*N complex doubles whose upper triangle and diagonal define the Hermitian
 * rho(0).  Outputs (device, each may be NULL): d_pops[nout*N],
 * d_eta_loss[nout*2] with nout = nsteps/out_every + 1 (rows as in
 * heom_propagate_device), and d_rho_out[N*N complex], rho at the end.
 * The work runs on cuda_stream (a cudaStream_t; NULL = legacy default
 * stream), after the work queued there before the call.  The call is
 * blocking: it waits for its own work to finish and returns its status --
 * HEOM_ENONFINITE when the run produced NaN or infinite values, HEOM_ETIMEOUT
 * when a device-side wait expired -- so the outputs are complete when it
 * returns HEOM_OK.  Because it stages its inputs from host memory that does
 * not outlive the call and waits for the device, it returns HEOM_EUNSUPPORTED
 * when cuda_stream is being captured into a CUDA graph.
 *
 * The address of the static array on the current device is looked up on
 * every call (cudaGetSymbolAddress, with that device current; this allocates
 * nothing).  Every call shares the one array, which keeps the last call's
 * contents; each call clears what must start at zero.  A call holds a
 * process-wide lock until its work has finished, so calls from several host
 * threads run one after another; work that reached the array while a call ran
 * (nothing in this library does) would race with it and corrupt its
 * results. */
#define HEOM_STATIC_SCRATCH_BYTES (8u << 20)
int heom_propagate_static(const heom_params* params, const double* d_rho0, double dt_fs, int64_t nsteps,
                          int64_t out_every, double* d_pops, double* d_eta_loss, double* d_rho_out,
                          void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* HEOM_H */
