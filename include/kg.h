/*
 * kg.h -- C ABI of the GB300 library for linear-scaling Kubo-Greenwood quantum
 * transport (Fan, Uppstu, Siro and Harju, arXiv 1307.0288).
 *
 * The library evaluates, on one GB300 GPU (sm_103a), the Chebyshev recursion
 * T_{n+1}(H~) = 2 H~ T_n(H~) - T_{n-1}(H~) (Eq. 38) applied to complex vectors through
 * the nearest-neighbour graphene tight-binding Hamiltonian (Eq. 13), and from it
 *   - the Chebyshev (KPM) moments C_n = <phi_L|T_n(H~)|phi_R> (Eq. 46, Algorithm 5),
 *   - the Chebyshev-Bessel propagator U(+-dt) and commutator [X, U(dt)]
 *     (Eqs. 36-37, Algorithms 6-7),
 *   - the velocity auto-correlation (VAC) and mean-square-displacement (MSD)
 *     moments per correlation time (Eqs. 33-34, 42-44, Algorithms 2-3),
 * plus the host-side energy sums and running conductivities (Eqs. 6, 9, 11, 29-31, 35).
 *
 * Conventions for every entry point:
 *   - Complex vectors are arrays of (re, im) double pairs.  A block of R vectors over
 *     N sites is laid out [N][R][2] (site-major, vector-minor).
 *   - A pointer argument named "host or device" may point to host memory or to CUDA
 *     device memory of the Hamiltonian's device; the library detects which.  The
 *     library never takes ownership of caller buffers and never keeps a pointer to
 *     them after the call returns.
 *   - Every call is synchronous: when it returns, outputs are complete.
 *   - No exception crosses the ABI.  A negative kg_status is an error; kg_last_error()
 *     then returns a message (per calling thread).  After KG_ECUDA the CUDA context
 *     may be unusable; destroy the handle.
 *   - There is no CPU fallback: without a usable CUDA device every GPU entry point
 *     returns KG_ENODEV.
 *
 * Units: energies eV, lengths nm, times fs (time steps are given in units of
 * hbar/gamma0), hbar = 0.6582119569 eV fs, velocities nm/fs.
 */
#ifndef KG_H
#define KG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int kg_status;
#define KG_OK 0
#define KG_EINVAL (-1)    /* invalid argument (message says which) */
#define KG_ENOMEM (-2)    /* device or host allocation failed */
#define KG_ECUDA (-3)     /* a CUDA call failed */
#define KG_ETIMEOUT (-4)  /* a bounded device-side wait gave up */
#define KG_ENUMERIC (-5)  /* NaN or Inf found in results */
#define KG_ENODEV (-6)    /* no usable CUDA device */

/* Message for the last error on the calling thread ("" if none). */
const char* kg_last_error(void);

/* ABI version of this header (increments on incompatible change). */
#define KG_ABI_VERSION 1
int kg_abi_version(void);

/* ------------------------------------------------------------------------- */
/* Lattice and Hamiltonian (Sec. 2)                                           */
/* ------------------------------------------------------------------------- */

#define KG_SHEET 0  /* 2D graphene, periodic in x and y, transport along x (zigzag)  */
#define KG_ZGNR 1   /* zigzag ribbon, periodic in x, open in y, transport along x     */
#define KG_AGNR 2   /* armchair ribbon, periodic in y, open in x, transport along y   */
#define KG_SHEET_OPEN_X 3  /* sheet open along the transport direction x (periodic in y):
                            * the non-periodic boundary of Sec. 5.1's length study      */

/* Sample geometry (Sec. 2): nx dimer lines along the zigzag direction, ny zigzag
 * chains; N = nx * ny carbon sites, site (i, j) numbered n = j * nx + i.  Position
 * x = i sqrt(3) a / 2, y = j 3a/2 + (a/2 when i + j is odd).  Periodic directions
 * need an even extent >= 4.  H = -gamma0 sum_<mn> |m><n| (Eq. 13) plus optional
 * on-site energies; the library works with H~ = H / emax_ev, so emax_ev must bound
 * the spectrum (|E| < emax_ev), e.g. 1.05 (3 gamma0 + W/2) for Anderson width W. */
typedef struct {
    int32_t kind;       /* KG_SHEET, KG_ZGNR, KG_AGNR or KG_SHEET_OPEN_X */
    int32_t reserved;   /* must be 0 */
    int64_t nx;         /* N_x */
    int64_t ny;         /* N_y */
    double gamma0_ev;   /* hopping gamma0 (2.7 in the paper) */
    double bond_nm;     /* carbon-carbon distance a (0.142 in the paper) */
    double emax_ev;     /* spectral scale E_max > 0 */
} kg_lattice;

typedef struct kg_hamiltonian kg_hamiltonian;

/* Builds H~ on the current CUDA device and keeps it there (owned by the handle).
 *   vacancies   host, n_vacancies distinct site numbers in [0, N) of removed atoms
 *               (Sec. 2, random single vacancies); may be NULL when n_vacancies = 0.
 *               A removed atom keeps no bonds and carries no amplitude.
 *   onsite_ev   host [N] on-site energies eps_n in eV (Anderson disorder), or NULL.
 *   cuda_stream cudaStream_t every later call on this handle is issued on (NULL =
 *               the legacy default stream).
 *   out         receives the handle; free it with kg_destroy_hamiltonian.
 * Errors: KG_EINVAL (bad sizes, duplicate or out-of-range vacancy, |eps| or
 * 3 gamma0 + max|eps| not below emax_ev), KG_ENOMEM, KG_ECUDA, KG_ENODEV. */
kg_status kg_build_hamiltonian(const kg_lattice* lattice, const int64_t* vacancies,
                               int64_t n_vacancies, const double* onsite_ev,
                               void* cuda_stream, kg_hamiltonian** out);

/* Sizes of a built Hamiltonian: N, N - N_v, E_max, and Omega = L_x L_y in nm^2. */
kg_status kg_hamiltonian_info(const kg_hamiltonian* h, int64_t* n_sites, int64_t* n_active,
                              double* emax_ev, double* area_nm2);

/* Releases the handle and all device memory it owns.  NULL is ignored. */
void kg_destroy_hamiltonian(kg_hamiltonian* h);

/* Host-only (no GPU needed): the neighbour list the library builds for a lattice, as
 * the paper's NL_nk table (Sec. 3.2, Algorithm 8) in slot-major order: idx_out[k*N + n]
 * is neighbour k of site n, or -1 if absent (open edge or removed atom).  Slot 0 is
 * (i-1, j), slot 1 is (i+1, j), slot 2 the bond to the neighbouring chain.  idx_out is
 * host [3][N] int32, caller-owned. */
kg_status kg_lattice_neighbors(const kg_lattice* lattice, const int64_t* vacancies,
                               int64_t n_vacancies, int32_t* idx_out);

/* ------------------------------------------------------------------------- */
/* Seeded synthetic inputs (host only, no GPU needed)                         */
/* ------------------------------------------------------------------------- */
/* The random numbers the method draws (Sec. 2: random single vacancies; Anderson
 * on-site energies uniform in [-W/2, W/2]; Sec. 3.1.1: random-phase vectors
 * phi_n = exp(i theta_n), theta_n uniform in [0, 2 pi)), from SplitMix64 (Steele, Lea
 * and Flood, OOPSLA 2014) in counter mode: key = mix64(seed + stream G),
 * x_k = mix64(key + (k + 1) G), G = 0x9E3779B97F4A7C15, arithmetic modulo 2^64;
 * uniform u_k = (x_k >> 11) 2^-53.  Streams: 0 vacancies, 1 Anderson energies, 16 + r
 * random vector r.  With these a C caller builds the same seeded workloads as the
 * Python input module: kg_n_vacancies -> kg_vacancy_sites -> kg_anderson_onsite ->
 * kg_build_hamiltonian, then kg_random_phase_vectors -> kg_dos_moments / kg_vac /
 * kg_msd.  Words, vacancy sites, energies and phases are bit-identical to that module;
 * cos and sin are the C library's.  All buffers are host memory, caller-owned;
 * errors: KG_EINVAL. */

/* SplitMix64 words x_start .. x_start + count - 1 of one stream into out[count]. */
kg_status kg_splitmix64(uint64_t seed, uint64_t stream, int64_t start, int64_t count, uint64_t* out);
/* N_v = round(n N), rounded half to even, for a concentration 0 <= n <= 1. */
kg_status kg_n_vacancies(int64_t n_sites, double concentration, int64_t* n_vac);
/* n_vac distinct sites of [0, N) (N < 2^31 - 1), sorted ascending, into out[n_vac]: a partial
 * Fisher-Yates shuffle whose step k swaps positions k and k + floor(w_k (N - k) / 2^32),
 * w_k the top 32 bits of word k of stream 0. */
kg_status kg_vacancy_sites(int64_t n_sites, int64_t n_vac, uint64_t seed, int64_t* out);
/* out_ev[n] = W (u_n - 1/2) in eV from stream 1, n < N. */
kg_status kg_anderson_onsite(int64_t n_sites, double w_ev, uint64_t seed, double* out_ev);
/* out [N][R][2] (interleaved complex, site-major as the moment entry points take it):
 * phi_n^(r) = (cos theta, sin theta), theta = 2 pi u_n of stream 16 + r, and 0 on the
 * n_vacancies removed sites (in [0, N)). */
kg_status kg_random_phase_vectors(int64_t n_sites, int n_vectors, uint64_t seed, const int64_t* vacancies,
                                  int64_t n_vacancies, double* out);

/* ------------------------------------------------------------------------- */
/* Moments and time evolution on the GPU                                      */
/* ------------------------------------------------------------------------- */

#define KG_FP64 0   /* complex128 vectors, FP64 recursion; moment sums see below */
#define KG_C64 1    /* complex64 vectors, FP32 recursion, compensated sums combined in FP64 */

/* Precision of the moments.  KG_FP64 runs the Chebyshev recursion and the time evolution
 * in FP64; the inner products of the moments are formed in double-float arithmetic on
 * the FP32 pipe (each FP64 factor split exactly into a float head and tail, products by
 * FMA TwoProduct, per-thread TwoSum/FastTwoSum pairs) and combined across threads and
 * blocks in FP64, about 2^-45 relative per term.  This holds for vector entries of
 * magnitude in [2^-63, 2^63) (random-phase vectors and their Chebyshev iterates are
 * O(1)); smaller entries contribute less accurately (nothing below 2^-126), and larger
 * ones overflow.  Every entry point that returns moments checks them and fails with
 * KG_ENUMERIC when one is NaN or infinite (NaN/Inf inputs, or entries >= 2^63);
 * kg_dos_moments_noalloc included (it returns after its stream completes). */

typedef struct {
    int32_t n_moments;   /* M >= 1: moments C_0 .. C_{M-1} (Eqs. 32-34) */
    int32_t n_vectors;   /* R: random vectors processed together, 1..64 (power of 2) */
    int32_t n_times;     /* N_c >= 1: correlation times t_m = m dt, m = 0..N_c-1 */
    int32_t precision;   /* KG_FP64 or KG_C64 */
    double dt;           /* correlation time step, units of hbar / gamma0 */
    double bessel_tol;   /* truncation of Eqs. 36-37: first omitted |J_m| < tol (1e-15) */
} kg_run;

/* DOS moments C_n^DOS = <phi|T_n(H~)|phi> (Eq. 32, Algorithm 5) for each of the R
 * vectors.  phi: host or device [N][R][2] (Sec. 3.1.1: random vectors with
 * <phi|phi> = N - N_v, zero on removed atoms).  mu_out: host or device [R][M][2],
 * caller-owned.  Uses run->n_moments, n_vectors, precision. */
kg_status kg_dos_moments(kg_hamiltonian* h, const kg_run* run, const double* phi,
                         double* mu_out);

/* VAC moments C_n^VAC(t_m) = <phi_L|T_n(H~)|phi_R> with |phi_L> = V U^dagger(t_m)|phi>,
 * |phi_R> = U^dagger(t_m) V |phi> (Eq. 33, Algorithm 2), t_m = m dt, advanced with
 * Eqs. 42-43.  V = (i/hbar)[H, X] (Eq. 15), so the moments are in (nm/fs)^2.
 * phi: host or device [N][R][2].  mu_out: host or device [R][N_c][M][2]. */
kg_status kg_vac(kg_hamiltonian* h, const kg_run* run, const double* phi, double* mu_out);

/* MSD moments C_n^MSD(t_m) = <phi_L|T_n(H~)|phi_L> with |phi_L> = [X, U(t_m)]|phi>
 * (Eq. 34, Algorithm 3), advanced with Eq. 44; in nm^2.  C^MSD(t_0) = 0.
 * phi: host or device [N][R][2].  mu_out: host or device [R][N_c][M][2]. */
kg_status kg_msd(kg_hamiltonian* h, const kg_run* run, const double* phi, double* mu_out);

/* Resumable time loops, for checkpointing long runs (the paper has no counterpart; its time
 * loops, Algorithms 2-3, carry exactly this state from one t_m to the next).  Each call
 * advances the loop state by run->n_times steps of run->dt and returns the moments at the
 * n_times new times; chaining calls reproduces one long run bit for bit.
 *   kg_msd_resume: state (psi, xi) = (U(t) phi, [X, U(t)] phi) (Eq. 44); xi NULL means a
 *     fresh start at t = 0 (psi = phi, xi = 0).
 *   kg_vac_resume: state (a, b) = (U^dagger(t) phi, U^dagger(t) V phi) (Eqs. 42-43); b NULL
 *     means a fresh start (a = phi, b = V phi).
 * psi, xi, a, b: host or device [N][R][2] complex128 (also for KG_C64, where the state is
 * converted on the way in and out).  mu_out: host or device [R][N_c][M][2], the moments at
 * t + dt .. t + N_c dt.  psi_out/xi_out (a_out/b_out): host or device [N][R][2], caller-owned,
 * both or neither (NULL: the final state is not returned); they may be the input buffers.
 * Every time loop checks that U(dt) kept the norm of psi (a): KG_ENUMERIC when it drifts by
 * more than 1e-10 (FP64) or 1e-3 (KG_C64) relative, e.g. for a far too loose bessel_tol.
 * The time loops (kg_vac, kg_msd and these) run the norm check, the non-finite check and the
 * copy of the moments behind one stream synchronisation; on KG_ENUMERIC mu_out holds the
 * offending moments. */
kg_status kg_msd_resume(kg_hamiltonian* h, const kg_run* run, const double* psi, const double* xi,
                        double* mu_out, double* psi_out, double* xi_out);
kg_status kg_vac_resume(kg_hamiltonian* h, const kg_run* run, const double* a, const double* b,
                        double* mu_out, double* a_out, double* b_out);

/* Fourier moments F_n = <phi|U(n dtau)|phi>, n = -N_m .. N_m (Eq. 25, Algorithm 4), with
 * the Nyquist step dtau = pi hbar for the scaled Hamiltonian (Sec. 4.2), i.e. U(dtau) =
 * exp(-i pi H~) applied n times forward and n times backward.  run->n_moments is N_m,
 * run->bessel_tol truncates the series of U(dtau); KG_FP64 only.
 * phi: host or device [N][R][2].  f_out: host or device [R][2 N_m + 1][2], index n + N_m. */
kg_status kg_ftm_dos_moments(kg_hamiltonian* h, const kg_run* run, const double* phi, double* f_out);

#define KG_OP_H 0    /* out = H~ in                                  (Algorithm 8) */
#define KG_OP_XH 1   /* out = [X, H~] in, (X_n - X_m) H~_nm, in nm    (Eq. 15)     */
#define KG_OP_V 2    /* out = V in = (i/hbar)[H, X] in, in nm/fs      (Eq. 15)     */

/* One sparse product on R vectors.  in, out: device [N][R][2] (distinct buffers). */
kg_status kg_apply(kg_hamiltonian* h, int op, const double* in_dev, double* out_dev,
                   int n_vectors);

#define KG_U_FORWARD 0    /* out = U(+dt) in = exp(-i H dt / hbar) in  (Eq. 36, Algorithm 6) */
#define KG_U_BACKWARD 1   /* out = U(-dt) in = U(dt)^dagger in         (Eq. 36, Algorithm 6) */
#define KG_U_COMMUTATOR 2 /* out = [X, U(dt)] in, in nm                (Eq. 37, Algorithm 7) */

/* One Chebyshev-Bessel time step of length dt (units of hbar/gamma0) on R vectors.
 * in, out: device [N][R][2] (distinct buffers). */
kg_status kg_evolve(kg_hamiltonian* h, double dt, int which, double bessel_tol,
                    const double* in_dev, double* out_dev, int n_vectors);

/* ------------------------------------------------------------------------- */
/* Batched instances in one persistent launch                                */
/* ------------------------------------------------------------------------- */

/* DOS moments (Eq. 32, Algorithm 5) of n_h independent Hamiltonians at once, e.g. many
 * ribbons of different widths, lengths and disorder, R random vectors each.  All members
 * must live on the current device and use transport along x (sheet or ZGNR).  The
 * members are concatenated into one block-diagonal table; one persistent kernel runs
 * every Chebyshev step of every member, each CTA waiting (bounded) only for the CTAs
 * that hold its sites' neighbours; the call's device work is captured once in a CUDA
 * graph and replayed.  The block width (vectors per thread group: 8..64) is chosen by a
 * measured autotuner on the first call for a given member set and R.
 *   hs       n_h member handles (one batch is cached per process for the same list and R;
 *            calls must not run concurrently from several host threads).
 *   run      n_moments M, n_vectors R (power of two <= 64), precision KG_FP64.
 *   phis     n_h pointers, host or device, member i's vectors [N_i][R][2].
 *   mu_out   host or device [n_h][R][M][2].
 * KG_ETIMEOUT if a CTA's wait for its neighbours gave up (the context stays usable);
 * KG_ENUMERIC if a moment is not finite. */
kg_status kg_batched_dos_moments(kg_hamiltonian* const* hs, int n_h, const kg_run* run,
                                 const double* const* phis, double* mu_out);

/* Result of the autotuner for the cached batch.  It measures every (block width, CTA
 * budget) pair: widths 8..64 (vectors one thread group covers per pass) and a budget of one
 * occupancy wave of CTAs or half of one (the tile schedule: how many site ranges the
 * members are cut into).  Returns the chosen width, its time per recursion step (ms) and
 * CTA count, and up to max_log measured trials (width, CTAs, ms per step). */
kg_status kg_batched_tuning(int* block_width, double* ms_per_step, int* n_ctas, int max_log,
                            int* log_width, int* log_ctas, double* log_ms);

/* Frees the cached batch (its device memory and graphs). */
kg_status kg_batched_release(void);

/* Test hook for failure detection: every workspace allocation of a handle larger than
 * `bytes` fails with KG_ENOMEM as if the device were out of memory (0 = no cap).  Injects
 * allocation failures on the host; the handle stays usable once the cap is lifted. */
kg_status kg_test_alloc_cap(uint64_t bytes);

/* Execution option for small instances (the recursion loops of Algorithms 5-7; no new
 * arithmetic).  When one recursion step needs at most 16 CTAs (up to 8192 site-vectors,
 * R <= 16), a launch per step costs more than the step, so by default (enable = 1) the
 * steps run in launches of a single thread-block cluster that keeps the vectors in its
 * shared memory and separates the steps with the cluster's hardware barrier: up to 256
 * moment steps per launch, and the whole Chebyshev-Bessel series of a time step (up to
 * 96 terms, all chains) in one launch.  The Chebyshev vectors and the propagated vectors
 * are bitwise those of one launch per step; the moments' inner products are summed in
 * another order (double-float sums; the two paths agree within 1e-12 of the largest
 * moment).  enable = 0 selects one launch per step for every size.  Process-wide; takes
 * effect on the next call. */
kg_status kg_set_small_persistent(int enable);

/* Test hook for failure detection: CTA `cta` of the cached batch stops publishing its
 * step flags after step 0, so its neighbours' bounded waits run out and the next
 * kg_batched_dos_moments returns KG_ETIMEOUT.  -1 turns the hook off. */
kg_status kg_batched_test_stall(int cta);

/* ------------------------------------------------------------------------- */
/* Surrogate MLP for sigma(E, t) (not part of the paper)                      */
/* ------------------------------------------------------------------------- */

/* A small network trained on sigma(E, t) curves the method generates, used to predict
 * ensemble-averaged sigma(E, t) across vacancy concentrations (the method itself stays
 * the fallback and the reference for its error).  Architecture: 3 inputs -> 4 hidden layers
 * of 256 GELU units (tanh form) -> 1 output; BF16 weights and activations at the matrix-multiply
 * inputs with FP32 accumulation (the 256 x 256 layers on the tcgen05 tensor cores),
 * FP32 master weights, Adam (beta1 0.9, beta2 0.999, eps 1e-8), loss = mean (y - t)^2.
 * Flat FP32 parameter layout (KG_MLP_PARAMS values): W1 [256][3], b1 [256], then for
 * layers 2..4 W [256][256] ([out][in]) and b [256], then W5 [256], b5 [1]. */
#define KG_MLP_PARAMS 198657
typedef struct kg_mlp kg_mlp;

/* Uploads the initial parameters (host or device, caller-owned) to the current device;
 * every later call is issued on cuda_stream. */
kg_status kg_mlp_create(const float* params, void* cuda_stream, kg_mlp** out);
void kg_mlp_destroy(kg_mlp* m);
/* Current FP32 parameters into params (host or device [KG_MLP_PARAMS]). */
kg_status kg_mlp_get_params(kg_mlp* m, float* params);
/* Inference: y [n] for inputs x [n][3] (host or device; device arrays are read and written
 * in place, so they must hold n x 3 and n floats).  Returns after the stream completes, with
 * one synchronisation.  One persistent kernel runs the
 * whole network on the tensor cores.  Layer 1 takes its FP32 inputs and weights as two BF16
 * terms each and b1 as three (W1 x + b1 to about 2^-16 relative); the training passes
 * evaluate layer 1 in FP32 on the CUDA cores.  The two differ by less than the BF16
 * rounding of the activations. */
kg_status kg_mlp_forward(kg_mlp* m, const float* x, int64_t n, float* y);
/* Loss and FP32 gradient (host or device [KG_MLP_PARAMS], may be NULL) of one batch. */
kg_status kg_mlp_gradients(kg_mlp* m, const float* x, const float* t, int64_t n, float* grad,
                           double* loss);
/* One Adam step on the batch (x [n][3], targets t [n]); loss before the step (may be NULL). */
kg_status kg_mlp_train_step(kg_mlp* m, const float* x, const float* t, int64_t n, float lr,
                            double* loss);
/* Number of kernels this handle has launched. */
kg_status kg_mlp_launches(kg_mlp* m, int64_t* launches);
/* CUDA-event timing of the tensor-core GEMM launches: enable (1) / disable (0) and reset;
 * read the summed GEMM time (ms), launch count and their 2MNK flops since the reset. */
kg_status kg_mlp_timing_enable(kg_mlp* m, int enable);
kg_status kg_mlp_timing_read(kg_mlp* m, double* gemm_ms, int64_t* gemm_launches, double* gemm_flop);
/* Test hook: D [rows][256] (FP32, device) = A [rows][k] * B [256][k]^T on the tensor cores,
 * A and B BF16 device arrays, k a multiple of 64. */
kg_status kg_mlp_gemm_test(const void* a_dev, const void* b_dev, int64_t rows, int k, float* d_dev);

/* DOS moments without device memory allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (their device memory is owned by a host framework's allocator, or they
 * must not allocate once they are serving).  It computes the same moments as
 * kg_dos_moments (C_n = <phi|T_n(H~)|phi>, n < M, for R vectors) but builds no
 * kg_hamiltonian and allocates nothing: its scratch space is one file-scope device
 * array of KG_NOALLOC_SCRATCH_BYTES, reserved when the library's device code is
 * loaded on a GPU and held there until the process exits.
 *   idx_dev     device int32 [3][N], the neighbour table of kg_lattice_neighbors
 *               (slot-major, -1 where absent).
 *   onsite_dev  device double [N], scaled on-site energies eps_n / E_max, or NULL.
 *               Precondition: 3|hopping| + max_n |onsite_n| < 1, so that the spectrum
 *               of H~ lies inside [-1, 1] (Eqs. 32-34); checked on the device before the
 *               recursion, KG_EINVAL otherwise.  kg_build_hamiltonian sets the on-site
 *               energy of removed sites to 0; pass 0 there too.  (When phi is 0 on the
 *               removed sites, as the random-phase vectors of Sec. 3.1.1 are, the value
 *               there does not enter the moments; a nonzero phi entry on a removed
 *               site would add a spurious delta(E - eps_n) term.)
 *   n_sites     N.   hopping: the scaled hopping -gamma0 / E_max (0 < |h| < 1/3).
 *   n_vectors   R, a power of two in 1..64.   n_moments: M >= 1.
 *   phi_dev     device [N][R][2] random vectors;  mu_dev: device [R][M][2] output.
 *   cuda_stream stream the work is issued on; the call returns after it completes.
 *               The caller's tensors are neither freed nor kept.  Moments that are
 *               NaN or infinite give KG_ENUMERIC.
 * Scratch needed: 12 N + 48 (N + 1) R bytes plus about 0.5 MB x R of partial sums;
 * larger problems are rejected with KG_EINVAL and a message giving both sizes.
 * The first call on a device looks up the array's device address (with that device
 * current).  The call synchronises its stream, so it cannot be captured into a CUDA
 * graph.  Every call shares the
 * one array and overwrites it, so calls that overlap on the GPU (several streams or
 * host threads at once) race; serialise them. */
#define KG_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
kg_status kg_dos_moments_noalloc(const int32_t* idx_dev, const double* onsite_dev, int64_t n_sites,
                                 double hopping, int n_vectors, int n_moments,
                                 const double* phi_dev, double* mu_dev, void* cuda_stream);

/* ------------------------------------------------------------------------- */
/* Timing counters (filled by the GPU entry points above)                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    double kpm_ms;          /* CUDA-event time of the moment recursions (Algorithm 5) */
    double evolve_ms;       /* CUDA-event time of the time-evolution steps (Algorithms 6-7) */
    int64_t kpm_launches;   /* fused moment-step kernel launches */
    int64_t evolve_launches;/* fused evolution-step kernel launches */
    int64_t other_launches; /* every other kernel launched (copies, V, reductions) */
    double kpm_site_steps;  /* site x vector x recursion-step updates in the moment loops */
    double evolve_site_steps;/* same for the evolution loops (all chains) */
} kg_timing;

/* Enables (1) or disables (0) CUDA-event timing of the phases; resets the counters. */
kg_status kg_timing_enable(kg_hamiltonian* h, int enable);
/* Reads the counters accumulated since the last kg_timing_enable (synchronises). */
kg_status kg_timing_read(kg_hamiltonian* h, kg_timing* out);

/* Measured FP64 fused multiply-add throughput of the current device (not in the paper:
 * the denominator of the FP64 recursion's ALU roofline).  Runs `repeats` (1..100)
 * launches of a kernel in which every thread of four 256-thread CTAs per SM advances
 * eight independent FP64 FMA chains for a fixed number of iterations (no waits, no
 * memory traffic beyond one store per thread), each timed with CUDA events; writes the
 * best rate in FMA instructions per second (thread-level: one DFMA = 2 flops) to
 * *fma_per_s.  Allocates and frees a small device buffer; synchronous.
 * Errors: KG_EINVAL (repeats out of range, null output), KG_ECUDA. */
kg_status kg_fp64_fma_rate(int repeats, double* fma_per_s);

/* ------------------------------------------------------------------------- */
/* Host-side helpers (FP64, no GPU needed)                                    */
/* ------------------------------------------------------------------------- */

/* J_m(tau), m = 0..n_terms-1, of the series Eqs. 36-37, with n_terms = the smallest
 * m > tau with |J_m(tau)| < tol (evaluated by Bessel's integral, A&S 9.1.21, with the
 * periodic trapezoidal rule).  j_out: host, capacity max_terms.  Returns KG_EINVAL if
 * max_terms is too small. */
kg_status kg_bessel_series(double tau, double tol, int max_terms, double* j_out,
                           int* n_terms);

/* Jackson damping g_n, n < M (Eq. 35).  g_out: host [M]. */
kg_status kg_jackson(int n_moments, double* g_out);

/* Chebyshev sum of Eqs. 29-31 on physical energies:
 *   out[s][e] = 2 / (pi Omega E_max sqrt(1 - E~^2)) sum_n g_n (2 - delta_n0) T_n(E~) mu[s][n],
 * E~ = energies_ev[e] / emax_ev (|E~| < 1), g_n Jackson (Eq. 35).  mu: host [n_sets][M]
 * (real parts of the moments, averaged over random vectors); out: host [n_sets][n_e]
 * in 1/(eV nm^2) times the moments' unit. */
kg_status kg_kpm_sum(const double* mu, int n_sets, int n_moments, const double* energies_ev,
                     int n_e, double emax_ev, double area_nm2, double* out);

/* FTM density of states, Eq. 22 with the Hanning window of Eq. 28 (w_n = (1 +
 * cos(pi n/(N_m+1)))/2) and dtau = pi hbar / E_max:
 *   out[s][e] = 1/(E_max Omega) sum_n w_n Re[exp(i pi n E/E_max) f[s][n + N_m]].
 * f: host [n_sets][2 N_m + 1][2] (complex moments, averaged over vectors); out: host
 * [n_sets][n_e] in 1/(eV nm^2). */
kg_status kg_ftm_sum(const double* f, int n_sets, int n_m, const double* energies_ev, int n_e,
                     double emax_ev, double area_nm2, double* out);

#define KG_SIGMA_GK 0   /* Eq. 6: e^2 int_0^t rho C_vv dt' (trapezoid)            */
#define KG_SIGMA_E1 1   /* Eq. 9: e^2 d(rho DX^2)/(2 dt) (central differences)    */
#define KG_SIGMA_E2 2   /* Eq. 11: e^2 rho DX^2 / (2 t), 0 at t = 0               */

/* Running conductivity in units of e^2/h on the grid t_m = m dt_fs.
 *   density: host [N_c][n_e], rho C_vv (for KG_SIGMA_GK, in 1/(eV fs^2)) or
 *            rho DX^2 (for E1/E2, in 1/eV), e.g. from kg_kpm_sum.
 *   out:     host [N_c][n_e]. */
kg_status kg_conductivity(int formula, const double* density, int n_times, int n_e,
                          double dt_fs, double* out);

/* Ballistic regime (Sec. 5.1): DX^2 = (rho DX^2) / rho (Eq. 10), length L = 2 sqrt(DX^2)
 * (Eq. 50) in nm and conductance G = (W / L) sigma^E1 (Eq. 51) in e^2/h, with sigma^E1 from
 * Eq. 9.  rho: host [n_e] (1/(eV nm^2)); rho_dx2: host [N_c][n_e] (1/eV); width_nm: the
 * sample width W across the transport direction; outputs host [N_c][n_e]; 0 where L = 0. */
kg_status kg_ballistic(const double* rho, const double* rho_dx2, int n_times, int n_e, double dt_fs,
                       double width_nm, double* length_out, double* g_out);

/* Semi-classical conductivity (Sec. 5.2): max_out[e] = max_{t > 0} sigma(E, t) (Eq. 53);
 * avg_out[e] = (1/(t2 - t1)) int_{t1}^{t2} sigma(E, t) dt (Eq. 54), trapezoid over the grid
 * times t_m = m dt_fs inside [t1, t2].  sigma: host [N_c][n_e]; either output may be NULL. */
kg_status kg_sigma_sc(const double* sigma, int n_times, int n_e, double dt_fs, double t1_fs,
                      double t2_fs, double* max_out, double* avg_out);

/* Pade [m/n] fit of a late-time MSD (Sec. 5.3, Eq. 58), y(t) = sum_{j=0}^{m} a_j t^j /
 * (1 + sum_{k=1}^{n} b_k t^k) (the printed denominator sum from k = 0 is read as k = 1),
 * by linear least squares on y (1 + sum b_k t^k) = sum a_j t^j.  coef_out: host
 * [m + 1 + n] = (a_0..a_m, b_1..b_n).  KG_EINVAL when n_points < m + 1 + n. */
kg_status kg_pade_fit(const double* t, const double* y, int n_points, int m, int n, double* coef_out);

/* The fit of Eq. 58 with every denominator coefficient b_k >= 0, so the approximant has no
 * pole for t >= 0 (the free linearised fit can put one among flat, noisy late-time data),
 * and on the true residual sum (R(t_i) - y_i)^2 rather than the linearised one.  Starting
 * points come from Sanathanan-Koerner reweighting of the bounded linearised problem (rows
 * divided by the previous pass's denominator until the weights settle; every pass solved
 * exactly over the 2^n sets of b_k held at 0), begun from four weight profiles
 * (1 + |t| / s)^-n, s = infinity, t_max, t_max / 10, t_max / 100; each is refined by
 * projected Levenberg-Marquardt and the smallest residual wins.  n <= 8.  Not in the paper:
 * a safeguard of the Eq. 58 fit.  Same layout and errors as kg_pade_fit. */
kg_status kg_pade_fit_positive(const double* t, const double* y, int n_points, int m, int n,
                               double* coef_out);

/* Value and derivative d/dt of the fitted approximant (for sigma^E1 = e^2 rho d(DX^2)/(2 dt)). */
kg_status kg_pade_eval(const double* coef, int m, int n, const double* t, int n_points,
                       double* value_out, double* deriv_out);

#ifdef __cplusplus
}
#endif

#endif /* KG_H */
