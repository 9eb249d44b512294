/*
 * spfc.h -- C interface of the GB300 BDF2-SAV Fourier pseudo-spectral solver
 * for the square phase field crystal (SPFC) equation.
 *
 * The problem (Sec. 1, eqs. energy-SPFC and equation-SPFC): on a periodic box
 * [0,L]^d, d = 2 or 3, evolve the density phi by the H^{-1} gradient flow
 *     phi_t = Delta mu,  mu = -div(beta |grad phi|^2 grad phi) + a phi + 2 Delta phi + Delta^2 phi,
 * a = 1 - eps > 0, of the energy
 *     E(phi) = int a/2 phi^2 + beta/4 |grad phi|^4 - |grad phi|^2 + 1/2 (Delta phi)^2.
 * (The paper fixes beta = 1.) Space: Fourier collocation on N points per axis
 * (Sec. 2.1). Time: the second-order BDF2 scheme with a scalar auxiliary
 * variable r = sqrt(E_1) (eq. scheme-SAV-1), E_1 = int beta/4 |grad phi|^4 -
 * |grad phi|^2 + (1 + 1/beta), solved per step by the scalar elimination of
 * Sec. 2.3 (eqs. solver-1 .. solver-6): a few FFTs, diagonal solves with the
 * positive symbol 3/2 + dt |k|^2 (a + |k|^4), and global inner products.
 *
 * Conventions shared by all calls
 *  - Every call returns an spfc_status; on failure spfc_last_error() gives a
 *    message. A device-side failure (non-finite value or an infeasible scalar
 *    system in the SAV solve) is latched on the GPU, stops further steps, and
 *    is reported by the next call that synchronises (spfc_energy, spfc_mass,
 *    spfc_sav_scalars, spfc_get_field, spfc_sync).
 *  - Real fields are float64, row-major with x fastest: index x + N*(y + N*z).
 *  - Pointers flagged *_on_device are CUDA device pointers on the handle's
 *    device; they are only read or written during the call (on the handle's
 *    stream, which is synchronised before the call returns). Host pointers
 *    are plain memory and are likewise not retained.
 *  - The handle owns all of its device memory (allocated in spfc_create,
 *    released in spfc_destroy) and launches all work on the stream given at
 *    creation. A handle must not be used from two threads at once.
 *  - The GPU supports N in {16, 32, 64, 128, 256, 512} (2D) and
 *    {16, 32, 64, 128} (3D), the same N on every axis.
 */
#ifndef SPFC_H
#define SPFC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spfc_s* spfc_t;

typedef enum {
  SPFC_OK = 0,
  SPFC_EINVAL = 1,     /* invalid argument */
  SPFC_ENOMEM = 2,     /* device allocation failed */
  SPFC_ECUDA = 3,      /* CUDA runtime error */
  SPFC_ENONFINITE = 4, /* non-finite value or infeasible SAV scalar system (latched on device) */
  SPFC_ETIMEOUT = 5,   /* a bounded device-side wait expired */
  SPFC_ESTATE = 6      /* call out of order (e.g. step before init) */
} spfc_status;

/* Start-up of the two-level scheme. */
typedef enum {
  SPFC_START_BDF1 = 0,  /* one first-order SAV step from phi^0 (not printed in the paper) */
  SPFC_START_GHOST = 1, /* phi^{-1} = phi^0 - dt Delta_N mu^0, eq. scheme-SAV-initial-1 */
  SPFC_START_COPY = 2   /* phi^{-1} = phi^0, the restart rule of Sec. 5.2 */
} spfc_start;

typedef enum {
  SPFC_FP64 = 0,      /* all arithmetic in float64 */
  SPFC_FP32_BULK = 1  /* FFTs and pointwise work in float32; the sums of E_1 and of the inner
                         products accumulated in float-float (two float32 words, about 2^-48
                         relative) per thread and per block, then in float64 across blocks;
                         E_1, S, gamma, eta, theta, the scalar solve, r and the zero mode
                         (mass) in float64 */
} spfc_precision;

/* Create a solver for one run.
 * d: 2 or 3; n[d]: points per axis (x first, all equal); L[d]: box lengths (x first);
 * eps: a = 1 - eps must be > 0; beta > 0; dt > 0; precision: spfc_precision;
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) on the current device.
 * Cites: Sec. 1 (problem), Sec. 2.1 (grid), eq. scheme-SAV-1 (scheme).
 * Errors: SPFC_EINVAL for unsupported sizes or parameters, SPFC_ENOMEM, SPFC_ECUDA. */
int spfc_create(int d, const int* n, const double* L, double eps, double beta, double dt,
                int precision, void* cuda_stream, spfc_t* out);

/* Kernel launch schedules compiled for a grid: the tile shapes of the
 * two-kernel step (row pass, then the column pass with its grid barrier;
 * six for N >= 128, one below) and the persistent step: every step of a
 * spfc_step call in one cooperative launch (row pass, column forward pass,
 * scalar solve, update and the next column inverse pass behind bounded grid
 * barriers), as schedule 6 for N >= 128 (8 values per FFT lane), 7 for
 * N >= 128 (4 values per lane, twice the threads) and 1 below. spfc_create
 * uses the grid's default, the autotuner's choice measured on GB300 (2D
 * float32: 512 -> 6, 256 and 128 -> 7, 16..64 -> 1; 2D float64: 512 -> 6,
 * 128 and 256 -> 5, otherwise 0), as does spfc_create_scheduled with
 * schedule = -1; a schedule in [0, spfc_num_schedules(d, n)) picks one
 * explicitly, which is how the autotuner times the choices. All schedules
 * compute the same step; results agree to rounding. spfc_schedule returns
 * the handle's schedule. */
int spfc_num_schedules(int d, int n);
int spfc_create_scheduled(int d, const int* n, const double* L, double eps, double beta, double dt,
                          int precision, void* cuda_stream, int schedule, spfc_t* out);
int spfc_schedule(spfc_t h);

/* Load phi^0 (N^d float64 values) and start the scheme with `mode` (spfc_start).
 * After BDF1 the handle holds (phi^1, phi^0, r^1, r^0); after GHOST/COPY it
 * holds (phi^0, phi^{-1}, r^0, r^{-1}) with r = sqrt(E_{1,N}) as in the line
 * after eq. scheme-SAV-initial-2. */
int spfc_init(spfc_t h, const double* phi0, int phi0_on_device, int mode);

/* Start from a seeded noise field, generated on the device: phi0[j] = mean +
 * amp (2 u_j - 1) at flat grid index j (x fastest), u_j = (x_j >> 11) 2^-53
 * with x_j output j of SplitMix64 (Steele, Lea & Flood 2014) seeded with
 * `seed`, i.e. the finaliser applied to seed + (j + 1) 0x9E3779B97F4A7C15.
 * The paper's initial data (Sec. 5.2) is mean = 0, amp = 0.05. Then as
 * spfc_init with `mode`. Allocates and frees one temporary device field;
 * synchronises. SPFC_EINVAL for a non-finite mean or amp or a bad mode. */
int spfc_init_random(spfc_t h, double mean, double amp, uint64_t seed, int mode);

/* Set the two time levels and auxiliary scalars directly: phi = phi^n,
 * phi_prev = phi^{n-1}, r = r^n, r_prev = r^{n-1} (used for restarts and
 * for per-step comparisons from a given state). */
int spfc_set_state(spfc_t h, const double* phi, const double* phi_prev, double r, double r_prev,
                   int on_device);

/* Advance nsteps >= 0 steps of eq. scheme-SAV-1 (asynchronous on the stream;
 * a latched device failure is returned by the next synchronising call). */
int spfc_step(spfc_t h, int64_t nsteps);

/* Energies of the current state (synchronising):
 * E_orig = E_N(phi^n) (eq. energy-discrete-spectral, with beta),
 * E_mod  = the modified energy of eq. discrete energy,
 * E_breve = a/2 ||phi||^2 + 1/2 ||Delta_N phi||^2 + r^2 (Sec. 5.2). Any pointer may be NULL. */
int spfc_energy(spfc_t h, double* E_orig, double* E_mod, double* E_breve);

/* mass = <phi, 1> = h^d sum phi (invariant, Theorem SPFC solvability); mean = mass / |Omega|.
 * Either pointer may be NULL. */
int spfc_mass(spfc_t h, double* mass, double* mean);

/* Scalars of the current state and of the last SAV solve (synchronising):
 * out[0] = r^n, out[1] = r^{n-1}, out[2] = xi = r^n / sqrt(E_1), out[3] = gamma =
 * <N, A^{-1} Delta N> (<= 0, eq. solver-5), out[4] = E_1 at the extrapolation,
 * out[5] = the steps taken since init, and of the last solve out[6] = eta =
 * <N, A^{-1}(2 phi^n - phi^{n-1}/2)>, out[7] = theta = <N, 2 phi^n - phi^{n-1}/2>,
 * out[8] = 1 - dt gamma / (2 E_1), out[9] = LHS (eq. solver-4). All of them
 * are float64 on both precision paths. `nout` entries (<= 10) are written. */
int spfc_sav_scalars(spfc_t h, double* out, int nout);

/* Copy phi^n (which = 0) or phi^{n-1} (which = 1) to `out` (N^d float64 values). */
int spfc_get_field(spfc_t h, double* out, int out_on_device, int which);

/* Change dt and restart the two-level scheme with phi^{n-1} = phi^n (Sec. 5.2). */
int spfc_dt_change(spfc_t h, double dt_new);

/* Stabilised scheme (Sec. 5.2, the remedy for rough initial data): the
 * dt-multiplied equation (a) gains - A dt Delta_N (phi^{n+1} - phi^n) on its
 * left side, i.e. the symbol A_N becomes 3/2 + dt |k|^2 (a + |k|^4) + A dt |k|^2
 * and the right-hand side gains - A dt Delta_N phi^n; the r-equation is
 * unchanged. A >= 0 (0, the default, is the scheme of Sec. 2). Set before
 * spfc_init it also applies to the start-up step; set later it applies to the
 * steps that follow (a pending update is completed first). Checkpoints record
 * A and spfc_load requires the same A. SPFC_EINVAL for a negative or
 * non-finite A. */
int spfc_set_stabilization(spfc_t h, double A);

/* Optional phi^4 term (the local part of the PFC free energy, Sec. 1): E_1
 * gains gamma3/4 ||phi||_4^4, so that E_1 >= |Omega| still holds, and the
 * nonlinear chemical potential N_N gains gamma3 phi^3 with its mean removed
 * (its zero mode never enters the mass-conserving scheme). The SAV scheme of
 * Sec. 2.2-2.3 is otherwise unchanged. gamma3 >= 0; 0, the default, is the
 * SPFC model. Single runs in 2D and 3D (the batched ensemble runs SPFC). With
 * gamma3 > 0 a 2D step takes three kernels (the lazy form) instead of two, a
 * 3D step keeps its six, and the first call allocates one more half-spectrum
 * work array (SPFC_ENOMEM if that fails). Set before spfc_init
 * it also applies to the start-up step; set later it applies to the steps
 * that follow (a pending update is completed first). Checkpoints record gamma3
 * and spfc_load requires the same value. SPFC_EINVAL for a negative or
 * non-finite gamma3. */
int spfc_set_gamma3(spfc_t h, double gamma3);

/* The PFC model of Sec. 1 (eq. energy-PFC: gamma3/4 phi^4 in place of
 * beta/4 |grad phi|^4; gamma3 = 1 is the paper's) on the same scheme, with a
 * split of its own, since without the |grad phi|^4 term the SPFC split has no
 * lower bound: L_N = a + (1 + Delta_N)^2 (symbol a + (1 - |k|^2)^2 > 0, so
 * A_N = 3/2 + dt |k|^2 (a + (1 - |k|^2)^2)), E_1 = gamma3/4 ||phi||_4^4 -
 * 1/2 ||phi||^2 + (1 + 1/(4 gamma3)) |Omega| >= |Omega|, N_N = gamma3 phi^3 -
 * phi (mean removed). gamma3 > 0 switches it on, 0 switches back to SPFC (the
 * beta given at creation). 2D single runs; a step is the lazy three-pass form.
 * spfc_energy then returns E_N = the PFC energy, the modified energy with
 * this L_N, and E_breve = 1/2 ||L_N^{1/2} phi||^2 + r^2. Set before spfc_init
 * it also applies to the start-up step; set later it applies to the steps
 * that follow (a pending update is completed first). Checkpoints record the
 * model. spfc_set_gamma3 is refused while it is on. SPFC_EINVAL for a
 * negative or non-finite gamma3, or a 3D handle with gamma3 > 0. */
int spfc_set_pfc(spfc_t h, double gamma3);

/* Write / read a checkpoint: the exact device state (both spectral levels in the
 * handle's precision, r^n, r^{n-1}, the step count) plus the grid and parameters.
 * A resumed run continues bit-identically. spfc_load rejects a file whose grid,
 * precision, L, dt, eps, beta, stabiliser A or gamma3 differ from the
 * handle's (SPFC_EINVAL). */
int spfc_save(spfc_t h, const char* path);
int spfc_load(spfc_t h, const char* path);

/* Per-step scalar records without host synchronisation (the paper has no
 * counterpart; it serves callers that follow r, xi, gamma and E_1 every step
 * without stalling the stream): host_ring is page-locked host memory that the
 * device can address (cudaHostAlloc / cudaMallocHost, or pinned torch
 * tensors, under unified addressing) holding `capacity` records of 8 float64
 * values. Every committed step of this handle (every solve of eqs. solver-2 to
 * solver-6, the start-up included) writes, from the device, record
 * steps % capacity = {steps since init, r^{n+1}, r^n, xi, gamma, E_1,
 * alpha = dt r^{n+1}/sqrt(E_1), device status}. Records are complete once the
 * stream has been synchronised (spfc_sync or any synchronising call); the
 * caller owns the memory and must keep it alive until the ring is removed
 * (host_ring = NULL) or the handle destroyed. The setting survives
 * spfc_init, spfc_set_state and spfc_load. SPFC_EINVAL for a capacity < 1
 * or memory the device cannot address. Synchronises the stream. */
int spfc_set_scalar_ring(spfc_t h, double* host_ring, int64_t capacity);

/* Wait for the handle's stream and report any latched device status. */
int spfc_sync(spfc_t h);

/* Per-kernel timing: when enabled (on != 0), spfc_step launches its kernels
 * one by one with CUDA events around each (no graph), and
 * spfc_kernel_times() returns, per kernel class, the number of launches and
 * the summed device milliseconds since the last reset (synchronising).
 * names[i] receives a static string. Returns the number of classes. */
int spfc_set_timing(spfc_t h, int on);
int spfc_kernel_times(spfc_t h, int max, const char** names, int64_t* launches, double* ms);

/* Device memory held by the handle, in bytes. */
int64_t spfc_device_bytes(spfc_t h);

/* Self-test of failure detection (the paper has no counterpart): runs the
 * bounded device-side waits of the grid barriers (the fused column pass's,
 * then the persistent step's acquire polls) on a counter that starts at 0
 * and that nothing advances, each for at most `polls` polls (~100 ns each,
 * polls <= 2^24). Returns SPFC_ETIMEOUT when the waits ran out (target > 0),
 * SPFC_OK when they were already satisfied (target == 0), SPFC_EINVAL for a
 * bad poll count, SPFC_ECUDA if the two disagree. The context stays usable
 * either way. */
int spfc_wait_selftest(unsigned long long target, long long polls, void* cuda_stream);

/* Measured float64 FMA throughput of the current device in GFLOP/s (one FMA
 * = 2 flops), the arithmetic roofline of the float64 step (the paper has no
 * counterpart): 4 x SM-count blocks of 256 threads, each thread 8
 * independent chains of 4096 FMAs, best of three timed launches after one
 * warm-up (CUDA events on cuda_stream, synchronising). Allocates and frees
 * one small output buffer. SPFC_EINVAL for a NULL pointer, SPFC_ENOMEM,
 * SPFC_ECUDA. */
int spfc_fp64_fma_rate(double* gflops, void* cuda_stream);

void spfc_destroy(spfc_t h);

/* ---------------------------------------------------------------------------
 * Batched ensemble: many independent 2D runs of uneven grid sizes and
 * parameters stepped together (each run is the scheme of spfc_create).
 * Runs of equal N share batched kernel launches; the size classes run as
 * parallel branches of one CUDA graph per step. The paper runs single grids;
 * the runs here do not interact.
 * ------------------------------------------------------------------------- */
typedef struct spfc_batch_s* spfc_batch_t;

/* nruns runs; per run: n[r] in {16..512} (power of two), square box of side
 * L[r], eps[r] (1 - eps > 0), beta[r] > 0; dt and precision shared. */
int spfc_batch_create(int nruns, const int* n, const double* L, const double* eps, const double* beta, double dt,
                      int precision, void* cuda_stream, spfc_batch_t* out);
/* As spfc_batch_create, with the tile shape of each grid-size class chosen:
 * schedules[r] (nruns values, NULL for every default) is the Shape schedule
 * of run r's class, -1 for the default of its size and precision (float32:
 * 4 from N = 256, else 0; float64: 5 from N = 128, else 0); runs of one grid
 * size must give the same value. The schedules a class can be built with
 * (spfc_batch_schedule_valid): 0, 2, 4 and 5 from N = 128, 0 below. Every
 * schedule computes the same steps (results agree to rounding); the
 * autotuner times them. SPFC_EINVAL for a schedule not compiled for its
 * size or runs of one size that disagree. */
int spfc_batch_create_scheduled(int nruns, const int* n, const double* L, const double* eps, const double* beta,
                                double dt, int precision, void* cuda_stream, const int* schedules,
                                spfc_batch_t* out);
/* 1 if a batch class of grid size n can be built with `schedule`, else 0. */
int spfc_batch_schedule_valid(int n, int schedule);
/* The schedule of the batch's class of grid size n (-1: no such class). */
int spfc_batch_schedule(spfc_batch_t b, int n);
/* Start run `run` from phi0 (host, n[run]^2 float64 values) with spfc_start `mode`. */
int spfc_batch_init(spfc_batch_t b, int run, const double* phi0, int mode);
/* Set both time levels and the auxiliary scalars of one run directly, as
 * spfc_set_state does for a single run: phi = phi^n, phi_prev = phi^{n-1}
 * (host, n[run]^2 float64 values each, x fastest), r = r^n, r_prev =
 * r^{n-1} (eq. scheme-SAV-1 advances from this state). Used for restarts and
 * for per-step comparisons from a given state. Synchronises the batch's
 * stream. SPFC_EINVAL for a bad run index, a NULL field or a non-finite r. */
int spfc_batch_set_state(spfc_batch_t b, int run, const double* phi, const double* phi_prev, double r,
                         double r_prev);
/* The optional phi^4 term of one run (as spfc_set_gamma3: gamma3/4 ||phi||_4^4
 * in E_1, gamma3 phi^3 with its mean removed in N; gamma3 >= 0, 0 the
 * default). A grid-size class with any run that has the term steps with
 * passes that carry it (one more half-spectrum work array per run of the
 * class, allocated on first need; runs with gamma3 = 0 there add zeros).
 * Set before spfc_batch_init it also applies to that run's start-up; set
 * later it applies to the following steps. Synchronises the batch's stream.
 * SPFC_EINVAL for a bad run index or a negative or non-finite gamma3,
 * SPFC_ENOMEM if the work array cannot be allocated. */
int spfc_batch_set_gamma3(spfc_batch_t b, int run, double gamma3);
/* Advance every run by nsteps (asynchronous; a run whose device status
 * latches an error stops, the others continue). */
int spfc_batch_step(spfc_batch_t b, int64_t nsteps);
int spfc_batch_sync(spfc_batch_t b);
/* phi^n (which = 0) or phi^{n-1} (which = 1) of one run to host memory. */
int spfc_batch_get_field(spfc_batch_t b, int run, double* out, int which);
/* out[0..8): r^n, r^{n-1}, xi, gamma, E_1, steps, mean of phi, device status. */
int spfc_batch_scalars(spfc_batch_t b, int run, double* out, int nout);
/* E3 = {E_N, modified energy, E_breve} of one run (as spfc_energy). */
int spfc_batch_energy(spfc_batch_t b, int run, double* E3);
/* Total grid points over all runs. */
int64_t spfc_batch_points(spfc_batch_t b);
void spfc_batch_destroy(spfc_batch_t b);
const char* spfc_batch_last_error(spfc_batch_t b);

/* ---------------------------------------------------------------------------
 * Learned surrogate: a Fourier neural operator (Li et al. 2020; the paper has
 * none) mapping (phi^{n-1}, phi^n, eps, beta) on an n x n periodic grid to
 * phi^{n+K}: lift 4 -> width, `layers` spectral-conv layers (truncated DFT
 * to kx < modes1 and |ky| <= modes2 as BF16 tensor-core GEMMs, per-mode
 * complex channel mixing, inverse truncated DFT, 1x1 conv, GELU), projection
 * width -> proj -> 1, output phi^n + 0.1 (d - mean d) (mass kept exactly).
 * Weights: float32 master and bfloat16 copy; products in BF16 with float32
 * accumulation, on the fifth-generation tensor cores (tcgen05.mma with the
 * accumulator in tensor memory). Fields are float32 device arrays
 * [batch][n][n]. The products' device-side waits are bounded: one that runs
 * out latches a status word of the handle, and the tile it was computing is
 * left unwritten. spfc_fno_loss_grad, which synchronises, reports it as
 * SPFC_ETIMEOUT; spfc_fno_predict does not synchronise, so the next
 * spfc_fno_predict or spfc_fno_loss_grad call reports it. Every call after
 * that returns SPFC_ETIMEOUT too.
 * ------------------------------------------------------------------------- */
typedef struct spfc_fno_s* spfc_fno_t;

int spfc_fno_create(int n, int width, int modes1, int modes2, int layers, int proj, int max_batch,
                    void* cuda_stream, spfc_fno_t* out);
int64_t spfc_fno_num_params(spfc_fno_t f);
/* parameters as float32 host arrays in the documented order (lift, layers, projection) */
int spfc_fno_set_params(spfc_fno_t f, const float* host);
int spfc_fno_get_params(spfc_fno_t f, float* host);
/* out = phi^{n+K} prediction; eps, beta: host arrays of `batch` values */
int spfc_fno_predict(spfc_fno_t f, int batch, const float* phi_n, const float* phi_nm1, const double* eps,
                     const double* beta, float* out);
/* Mean-square loss against target (device), gradient kept on the device for
 * spfc_fno_adam_step and optionally copied to grad_host. */
int spfc_fno_loss_grad(spfc_fno_t f, int batch, const float* phi_n, const float* phi_nm1, const double* eps,
                       const double* beta, const float* target, double* loss, float* grad_host);
int spfc_fno_adam_step(spfc_fno_t f, float lr, float beta1, float beta2, float epsilon, float weight_decay);
void spfc_fno_destroy(spfc_fno_t f);
const char* spfc_fno_last_error(spfc_fno_t f);
/* Self-test of the network's tensor-core product (no paper counterpart):
 * C[b] = A[b] B[b] for b < batch, A M x K, B K x N, C M x N, all float32 host
 * arrays, row-major, batches contiguous. The product rounds A and B to
 * bfloat16 (nearest even) and accumulates in float32; splits > 1 sums K in
 * `splits` chunks in a fixed order. flags: 1 = A stored as bfloat16 on the
 * device, 2 = A stored column-major, 4 = B stored column-major (the storage
 * only; the arguments stay row-major), 8 = a test of the wait bound: after
 * its product, each tile waits for an mbarrier phase that nothing completes,
 * so the wait runs out after about a second, latches the status and the
 * tile is left unwritten (C undefined); the call returns SPFC_ETIMEOUT and
 * the context stays usable. Synchronises the stream. SPFC_EINVAL for bad
 * sizes (each array <= 2^26 elements, splits <= 1024) or flags, SPFC_ETIMEOUT
 * if a bounded wait ran out. */
int spfc_gemm_selftest(int M, int N, int K, int batch, int splits, int flags, const float* A, const float* B,
                       float* C, void* cuda_stream);
/* Weight file: magic "SPFCFNO1", int32 {n, width, modes1, modes2, layers,
 * proj}, int64 parameter count, then the float32 parameters in the order of
 * spfc_fno_set_params. spfc_fno_load requires a network of the same shape
 * (SPFC_EINVAL otherwise, the weights unchanged) and resets Adam's moments
 * as spfc_fno_set_params does. */
int spfc_fno_save(spfc_fno_t f, const char* path);
int spfc_fno_load(spfc_fno_t f, const char* path);

/* The surrogate's jump-with-fallback loop, `jumps` rounds over `nruns` runs.
 * The paper has no counterpart: the network is an accelerator of the SAV
 * scheme, which stays its fallback and its judge. Each round:
 *  1. one call of the network predicts phi^{n+K} of every run from
 *     (phi^n, phi^{n-1}, eps, beta);
 *  2. energy test: the jump is rejected, and the run takes K plain SAV steps
 *     instead, if the modified energy (eq. discrete energy) of the restarted
 *     prediction exceeds that of the run's live two-level state (phi^n,
 *     phi^{n-1}, r^n, r^{n-1}). After the copy restart with r = sqrt(E_1) the
 *     former is E_N(prediction) + C_beta |Omega| (E_N of eq.
 *     energy-discrete-spectral with the run's phi^4 term);
 *  3. every check_every rounds (round j with j % check_every == 0; 0: never)
 *     a surviving prediction is compared with K plain steps that run's twin
 *     takes from the same state (phi^n, phi^{n-1}, r^n, r^{n-1}); rel-L2 above
 *     tol rejects the jump and the run takes the twin's state;
 *  4. an accepted prediction restarts the run with the copy start (Sec. 5.2:
 *     phi^{n+K-1} := phi^{n+K}, r = sqrt(E_1)).
 * net: a network of grid size n <= 256 (the energy test's limit), nruns <= its
 *    largest batch; runs of the PFC model (spfc_set_pfc) are refused;
 * runs: nruns initialised 2D handles on square n x n grids (their eps and
 *    beta feed the network), owned by the caller;
 * twins: nruns further 2D handles, distinct and none of them a run, each with
 *    its run's grid, parameters and precision, used as scratch for the
 *    checks (their state is overwritten); may be NULL when check_every == 0;
 * counts (host, 5 values, nullable): rounds x runs, accepted, rejected by
 *    energy, rejected by check, checks made;
 * decisions (host, jumps x nruns, row-major by round, nullable): 0 accepted,
 *    1 rejected by energy, 2 rejected by check;
 * check_err (host, jumps x nruns, nullable): rel-L2 of each checked jump, NaN
 *    where no check was made.
 * Synchronous (the handles' and the network's streams are synchronised).
 * Errors: SPFC_EINVAL, SPFC_ESTATE, SPFC_ENOMEM, SPFC_ECUDA, SPFC_ENONFINITE;
 * after an error during the rounds the runs may be partly advanced and
 * counts is not written. Message in spfc_surrogate_last_error(). */
int spfc_surrogate_advance(spfc_fno_t net, spfc_t* runs, spfc_t* twins, int nruns, int K, int jumps, int check_every,
                           double tol, int64_t* counts, int8_t* decisions, double* check_err);
const char* spfc_surrogate_last_error(void);

/* Allocation-free energy diagnostics of one 2D field (float64).
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory -- code whose device memory is owned by another allocator or
 * a fixed budget, and code that must not risk the device synchronisation
 * that cudaMalloc / cudaFree can cause. It allocates nothing: its scratch
 * lives in one fixed device array of about 1.6 MB inside the library, which
 * every GPU that loads the library holds until the process exits.
 * n: points per axis, one of 16, 32, 64, 128, 256 (larger N is rejected with
 *    SPFC_EINVAL: the scratch array is sized for 256 x 256);
 * L[2]: box lengths; eps, beta as in spfc_create;
 * phi_dev: the field, n*n float64 values on the current device (x fastest);
 * out[3] (host): E_N(phi) (eq. energy-discrete-spectral), 1/2 ||L_N^{1/2} phi||^2,
 *    and the mass h^2 sum phi;
 * cuda_stream: the stream to run on (synchronised before returning).
 * Every call looks up the scratch array's device address on the current
 * device and reads an 8-byte marker from it (synchronously); the first call
 * in a device context (the first on a device, or the first after
 * cudaDeviceReset) also writes a twiddle table and the marker into it. Make
 * that first call before any stream capture. All calls share the one array
 * and leave their contents in it; calls that overlap on the GPU (other host
 * threads, other streams) race and must be serialised by the caller.
 * Errors: SPFC_EINVAL, SPFC_ECUDA, SPFC_ENONFINITE; message in
 * spfc_noalloc_last_error(). */
int spfc_field_energy_noalloc(int n, const double* L, double eps, double beta, const double* phi_dev,
                              double* out, void* cuda_stream);
const char* spfc_noalloc_last_error(void);

/* Message of the last failed call on this handle (or of the last failed
 * spfc_create on this thread when h is NULL). Never NULL. */
const char* spfc_last_error(spfc_t h);

#ifdef __cplusplus
}
#endif

#endif /* SPFC_H */
