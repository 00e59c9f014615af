/*
 * ed.h -- C ABI of the GB300 time-dependent Hubbard exact-diagonalisation
 * library (libhubbard_ed.so).
 *
 * The library implements the hot path of Innerberger, Worm, Prauhart, Kauch,
 * "Electron-light interaction in nonequilibrium: exact diagonalization for
 * time dependent Hubbard Hamiltonians" (arXiv:2005.13498): the Hubbard
 * Hamiltonian H(t) with Peierls phases (Sec. 2.1-2.2, Eqs. (1), (3)) in one
 * (n_up, n_dn) sector (Sec. 2.3, 3.1), applied matrix-free on the GPU inside a
 * Lanczos approximation of exp(-i tau H(t_mid)) v (Sec. 3.4, Algorithm 6;
 * fixed dimension by default, or with the algorithm's adaptive exit) for the
 * exponential midpoint rule (Eq. (32)) or a fourth-order commutator-free
 * scheme, with the observables of Sec. 3.5, the nonequilibrium Green's
 * functions of Eq. (15) and the spectral function of Eq. (37).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Sites are 0..Ns-1 (Ns <= 16).  A spin configuration is an Ns-bit word,
 *   bit i = occupation of site i.  Each spin basis lists all words with n
 *   set bits in ascending integer order; this is the order of the fermionic
 *   hash of Eq. (36).  A sector vector is a dim_up x dim_dn matrix Psi stored
 *   row-major: element (r_up, r_dn) at offset r_up * dim_dn + r_dn.
 * - Complex vectors are interleaved (re, im): ED_C128 = two float64 per
 *   element, ED_C64 = two float32 per element.  ED_C64 keeps every Lanczos
 *   scalar (inner products, norms, the tridiagonal matrix and its
 *   exponential) in float64; only vectors and the apply run in float32.
 * - Fermion sign: modes are ordered all up sites, then all down sites; a hop
 *   p -> q of one spin picks up (-1)^(occupied sites of that spin strictly
 *   between p and q) (Eqs. (7)-(8), (26)).  The paper's site-interleaved mode
 *   order differs by a diagonal +-1 gauge that leaves every observable here
 *   unchanged.
 * - Hopping p -> q on bond b has matrix element -t_b exp(-i A(t).d_b) times
 *   the fermion sign, the reverse hop the complex conjugate (Eq. (3) with a
 *   uniform vector potential, e = 1); d_b = r_q - r_p.
 * - Pointers to vectors may be device pointers (CUDA memory allocated by the
 *   caller) or, where a call says so, host pointers; the library detects which
 *   and copies host data in and out itself.  All other arrays are host memory.
 * - Streams: `stream` is a cudaStream_t passed as void*; NULL = the legacy
 *   default stream.  Calls on one context must not run concurrently from
 *   several host threads.
 * - Devices: a context's tables go to the device that is current at its
 *   first GPU call.  Every later GPU call on it must run with that device
 *   current (else ED_ERR_STATE, nothing launched), and device vectors passed
 *   to it must live on that device (else ED_ERR_ARG).
 * - Errors: every call returns an ed_status; no C++ exception crosses the
 *   ABI.  ed_last_error() returns a human-readable message for the last
 *   failing call on that context (or on any context when ctx is NULL).
 * - Ownership: the context owns its tables and workspace; caller-provided
 *   vectors stay owned by the caller and are never freed by the library.
 */
#ifndef HUBBARD_ED_H
#define HUBBARD_ED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ed_ctx ed_ctx;

typedef enum {
  ED_OK = 0,
  ED_ERR_ARG = 1,          /* invalid argument (bad sector, null pointer, ...)   */
  ED_ERR_CUDA = 2,         /* a CUDA runtime call failed                          */
  ED_ERR_OOM = 3,          /* device allocation failed or exceeds the workspace cap */
  ED_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up                  */
  ED_ERR_UNSUPPORTED = 5,  /* outside the supported range (Ns > 16, m > 64, ...)   */
  ED_ERR_STATE = 6,        /* call order violated (e.g. apply before set_lattice)  */
  ED_ERR_NUMERIC = 7       /* non-finite value detected in a norm or coefficient   */
} ed_status;

typedef enum { ED_C128 = 0, ED_C64 = 1 } ed_dtype;

/* Time-stepping scheme of ed_propagate / ed_spectral_propagate.
 * ED_MIDPOINT: the exponential midpoint rule of Eq. (32), one Krylov step of
 *   Algorithm 6 per time step with H at the midpoint (second order).
 * ED_CFET4: the fourth-order commutator-free exponential propagator (the
 *   family named in Sec. 3.4; the two-exponential form of Alvermann and
 *   Fehske, J. Comput. Phys. 230, 5930 (2011)):
 *     psi(t+dt) = exp(-i dt (a1 H1 + a2 H2)) exp(-i dt (a2 H1 + a1 H2)) psi(t),
 *   H_k = H(t + c_k dt), c_{1,2} = 1/2 -+ sqrt(3)/6, a_{1,2} = (3 -+ 2 sqrt(3))/12;
 *   two Krylov steps of length dt/2 per time step.                            */
typedef enum { ED_MIDPOINT = 0, ED_CFET4 = 1 } ed_integrator;

/* Vector potential of the pump pulse, entering every bond through its phase
 * A(t).d_b (Eq. (3)); dir is used as given (not normalised).
 * shape ED_PULSE_SIN_GAUSS (0):
 *   A(t) = A0 exp(-(t-t0)^2/(2 sigma^2)) sin(omega (t - t0)) dir,
 *   a Gaussian-enveloped oscillation like the field pulse of Eq. (2); the
 *   workloads define their pulses by A(t) directly.
 * shape ED_PULSE_COS_PHASE (1): the paper's simplified phase of Eq. (4),
 *   A(t) = -A0 [cos(omega (t - t0)) - b] exp(-(t-t0)^2/(2 sigma^2)) dir,
 *   so that a hop p -> q with dir.d_b = 1 carries exactly the factor
 *   f(t) = exp(i a [cos(omega (t - t_p)) - b] exp(-(t-t_p)^2/(2 sigma^2)))
 *   with a = A0, t_p = t0 (b = cos(omega t0) makes f(0) = 1).
 * A zero-initialised shape/b gives the first form.                            */
typedef enum { ED_PULSE_SIN_GAUSS = 0, ED_PULSE_COS_PHASE = 1 } ed_pulse_shape;
typedef struct {
  double A0, omega, sigma, t0;
  double dir[3];
  double b;        /* ED_PULSE_COS_PHASE only                                 */
  int shape;       /* ed_pulse_shape                                          */
  int reserved;    /* must be 0                                               */
} ed_pulse;

/* Optional per-step outputs of ed_propagate (all host arrays, each nullable). */
typedef struct {
  double* docc;    /* [n_steps+1] <d>(t_n) = (1/Ns) sum_k w_d[k] |psi_k|^2,
                      Eq. (13) through the weight vector of Sec. 3.5; not
                      divided by |psi|^2                                       */
  double* norm2;   /* [n_steps+1] |psi(t_n)|^2                                 */
  double* energy;  /* [n_steps+1] E(t_n) = (1/Ns) <psi|H(t_n)|psi>, Eq. (14);
                      costs one extra apply per step                          */
  double* delta;   /* [n_steps] a-posteriori estimate delta of Algorithm 6 for
                      the step's Krylov approximation (a diagnostic unless
                      ed_set_krylov_tol enabled the adaptive exit)             */
  int32_t* m_eff;  /* [n_steps] Krylov dimension used (< m after a breakdown
                      or the adaptive exit); with ED_CFET4 the larger of the
                      step's two Krylov steps, likewise delta                   */
  int32_t profile; /* nonzero: launch kernels one by one (no CUDA graph) with
                      a CUDA event pair around every launch on the launching
                      stream, and report per-kind device time below           */
  double* kernel_ms;        /* [ED_KERNEL_KINDS] summed event time per kind  */
  int64_t* kernel_launches; /* [ED_KERNEL_KINDS] launches per kind           */
} ed_observables;

/* Kernel kinds reported by the profile mode, in this order.                  */
#define ED_KERNEL_KINDS 6
/* 0 apply (fused H x_j with the three-term recurrence and <v_j, w>),
 * 1 update (x_{j+1} = w - alpha_j v_j and |x_{j+1}|), 2 small exponential,
 * 3 combine (psi = beta V y with <d> and |psi|^2), 4 energy apply,
 * 5 Green's-function overlaps.                                               */

/* Create a context for the sector H^{n_up}_{n_dn}(Ns) (Sec. 3.1, Eq. (18)):
 * enumerates both spin bases and their ranks on the host.
 * Errors: ED_ERR_ARG if out == NULL or n_up/n_dn outside 0..Ns;
 * ED_ERR_UNSUPPORTED if Ns < 1 or Ns > 16.  On error *out is set to NULL.   */
ed_status ed_build_basis(ed_ctx** out, int Ns, int n_up, int n_dn);

/* Sector shape: dim_up = C(Ns, n_up), dim_dn = C(Ns, n_dn) (Eq. (18)).       */
ed_status ed_dims(const ed_ctx* ctx, int64_t* dim_up, int64_t* dim_dn);

/* Copy the spin basis words (ascending) of spin 0 (up) or 1 (down) into
 * words[dim_spin] (host).  Used to check the basis against other codes.       */
ed_status ed_get_basis(const ed_ctx* ctx, int spin, uint32_t* words);

/* Define the lattice and interaction (Sec. 2.1, Eq. (1); Sec. 3.2-3.3).
 * Bond b joins sites p[b] != q[b] with hopping magnitude t_hop[b] and
 * displacement d[3b..3b+2] = r_q - r_p (minimum image across a periodic wrap).
 * U is the on-site repulsion; eps (nullable, Ns entries) adds
 * eps_i (n_i,up + n_i,dn) (eps_i = -v_ii of the paper).  Builds the per-spin
 * connection tables (target rank, bond class and orientation, fermion sign;
 * the O(N_nz) hop-emulation construction suggested in Sec. 3.3) and uploads
 * them to the current CUDA device.  May be called again to change the lattice.
 * Bonds listed twice add up.  Errors: ED_ERR_ARG for a bad site index,
 * p == q, a non-finite value or more than 128 distinct (t, d) bond classes;
 * ED_ERR_CUDA / ED_ERR_OOM for device failures.                             */
ed_status ed_set_lattice(ed_ctx* ctx, int n_bonds, const int32_t* p,
                         const int32_t* q, const double* t_hop,
                         const double* d, double U, const double* eps);

/* Set the static vector potential A (3 doubles) used by ed_apply_H and
 * ed_double_occupation-side energy queries.  Default A = 0.                  */
ed_status ed_set_field(ed_ctx* ctx, const double A[3]);

/* Copy the connection table of spin 0/1 to host arrays for inspection:
 * off[dim+1] (row offsets) and ent[off[dim]] packed entries
 * (bits 0-15 target rank, bits 16-23 group = 2*class + orientation,
 * bit 31 fermion sign (1 = negative)); n_classes receives the number of bond
 * classes.  Either array may be NULL to query sizes only (*nnz_out).          */
ed_status ed_get_table(const ed_ctx* ctx, int spin, int32_t* off,
                       uint32_t* ent, int64_t* nnz_out, int32_t* n_classes);

/* w = H(A) v for nvec vectors stored back to back (each dim_up*dim_dn
 * elements), A from ed_set_field.  v and w are DEVICE pointers of the given
 * dtype and must not overlap.  Asynchronous on `stream`.
 * Errors: ED_ERR_STATE before ed_set_lattice, ED_ERR_ARG for NULL / host
 * pointers or nvec < 1.                                                      */
ed_status ed_apply_H(ed_ctx* ctx, const void* v, void* w, ed_dtype dtype,
                     int nvec, void* stream);

/* Ground state of H(A = 0) (Sec. 3.4, "Ground state"): float64 Lanczos with
 * full reorthogonalisation and explicit restarts (replacing the paper's
 * shifted power iteration, Algorithms 4-5), started from a seeded
 * pseudo-random vector.  psi (DEVICE or host, complex128, unit norm on
 * return, phase-fixed so that its largest-magnitude element is real and
 * positive) receives the eigenvector, *E0 the eigenvalue; resid_out
 * (nullable) receives |H psi - E0 psi|.  Stops when the residual is below
 * tol * max(1, |E0|) or after max_iter applies (then returns ED_OK with the
 * best estimate; check resid_out).                                           */
ed_status ed_ground_state(ed_ctx* ctx, void* psi, double* E0, double tol,
                          int max_iter, uint64_t seed, double* resid_out);

/* Propagate psi from t_start over n_steps steps of the exponential midpoint
 * rule (Eq. (32)): psi <- exp(-i dt H(t_n + dt/2)) psi, t_n = t_start + n dt,
 * each exponential by m Lanczos steps (Algorithm 6 with fixed m, breakdown
 * exit when beta_j <= tol * max(1, max|alpha|, max beta), tol = 1e-13 for
 * ED_C128 and 1e-6 for ED_C64).  psi (DEVICE or host pointer of `dtype`) is
 * updated in place; a host psi is back in place when the call returns.  A
 * pinned host psi (cudaHostAlloc, or cudaHostRegister with mapping) is read
 * and written by a kernel over the host link, any other host memory through
 * a staged copy.  After an error a host psi holds the state as far as the
 * steps got (pinned) or is unchanged (other host memory).
 * obs (nullable) receives observables at t_0..t_{n_steps}.
 * One step is captured as a CUDA graph and replayed.  Requires 1 <= m <= 64.
 * Errors: ED_ERR_ARG, ED_ERR_STATE, ED_ERR_UNSUPPORTED (m > 64),
 * ED_ERR_NUMERIC (non-finite norm), ED_ERR_CUDA / ED_ERR_OOM.                */
ed_status ed_propagate(ed_ctx* ctx, void* psi, ed_dtype dtype,
                       const ed_pulse* pulse, double t_start, double dt,
                       int n_steps, int m, const ed_observables* obs,
                       void* stream);

/* <d> = (1/Ns) sum_k w_d[k] |psi_k|^2 (Sec. 3.5, Eq. (13)) and, if d_site is
 * not NULL, the per-site values <n_i,up n_i,dn> (Ns entries).  psi is a DEVICE
 * or host pointer.  Synchronous.                                             */
ed_status ed_double_occupation(ed_ctx* ctx, const void* psi, ed_dtype dtype,
                               double* d_avg, double* d_site);

/* Double occupancy without any device allocation: the same results as
 * ed_double_occupation (average and, if d_site is not NULL, per-site values),
 * for callers that must not allocate device memory while they run -- for
 * example inside a loop whose device memory is fixed up front, or in a host
 * application that enforces its own device-memory budget.  The paper has no
 * counterpart; this is a deployment variant of the reduction above.
 *   - Scratch: a fixed array of 139,400 bytes inside the library (one per
 *     device that loads it, held until the process exits) replaces the
 *     per-call partial-sum buffers.  The sector may have at most 67,108,864
 *     elements (dim_up * dim_dn); larger sectors are rejected with
 *     ED_ERR_UNSUPPORTED before anything runs.
 *   - psi must be a DEVICE pointer of `dtype`; the context's tables must
 *     already be on the device (any earlier GPU call on this context puts them
 *     there), else ED_ERR_STATE.  The call itself allocates nothing: no
 *     cudaMalloc, cudaFree or allocating library routine.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call uses the same array, whose contents persist between calls;
 *     nothing in it needs to start at zero (each call overwrites every slot
 *     it reads).  Calls that overlap on the GPU (other streams, other host
 *     threads) race on the array and must not be issued.
 *   - Runs on `stream` and synchronises it before returning (the results are
 *     host values).                                                          */
ed_status ed_double_occupation_static(ed_ctx* ctx, const void* psi, ed_dtype dtype,
                                      double* d_avg, double* d_site, void* stream);

/* Nonequilibrium Green's functions of Eq. (15) with reference time 0
 * (Sec. 2.5, 3.7): for every site i and spin s, phi = c_is psi0 and
 * phi' = c^+_is psi0 are built in the sectors with one electron fewer / more
 * (the hash lookup of Sec. 3.7), then phi, phi' and psi0 itself are propagated
 * together by the midpoint rule (pulse, dt, m as in ed_propagate) in one
 * batched launch per kernel, and after every step
 *   G_less[n][i][s]  = i <c_is psi(t_n)| phi_is(t_n)>,
 *   G_great[n][i][s] = -i <c^+_is psi(t_n)| phi'_is(t_n)>,
 * n = 0..n_steps.  psi0 (DEVICE or host, complex128, in ctxN's sector) is not
 * modified.  G_less / G_great are host arrays of (n_steps+1)*Ns*2 complex128
 * (interleaved re, im); an entry whose target sector does not exist is 0.
 * dtype selects the vector precision of the propagation (ED_C64: float32
 * vectors with float64 Lanczos scalars and float64 overlaps).                */
ed_status ed_spectral_propagate(ed_ctx* ctxN, const void* psi0,
                                ed_dtype dtype, const ed_pulse* pulse,
                                double dt, int n_steps, int m,
                                double* G_less, double* G_great, void* stream);

/* ed_spectral_propagate with the reference time t_ref of Eq. (15) instead of
 * 0: psi0 is the state psi(t_ref) (e.g. the ground state propagated to t_ref
 * with ed_propagate and the same pulse), and G_less[n] / G_great[n] are the
 * Green's functions at times (t_ref, t_ref + n dt), the pulse evaluated at
 * the absolute times.  Same arguments, outputs and errors otherwise.        */
ed_status ed_spectral_propagate_at(ed_ctx* ctxN, const void* psi0, double t_ref,
                                   ed_dtype dtype, const ed_pulse* pulse,
                                   double dt, int n_steps, int m,
                                   double* G_less, double* G_great, void* stream);

/* Broadened Fourier transform of Eq. (37) (Sec. 3.7), on the host:
 *   A[f][j] = (1/pi) Im int_0^{T} e^{-eps t} e^{i nu_f t} G_j(t) dt,
 * T = n_steps dt, by the trapezoid rule over the samples G_j(k dt),
 * k = 0..n_steps.  G: host array [n_steps+1][n_series] complex128
 * (interleaved re, im), e.g. G_less or G_great of ed_spectral_propagate with
 * n_series = 2 Ns; nu: host [n_nu]; A: host [n_nu][n_series].  A(nu, t) of
 * the paper is the sum of the A of G_less and of G_great.  ED_ERR_ARG for
 * NULL pointers, sizes < 1, dt <= 0 or eps < 0.                              */
ed_status ed_spectral_function(const double* G, int n_steps, int n_series, double dt,
                               double eps, const double* nu, int n_nu, double* A);

/* Apply c_is (create = 0) or c^+_is (create = 1) to psi of ctx's sector and
 * write the result into out (a vector of ctx_dst's sector, which must be
 * (n_up-+1, n_dn) for s = 0 or (n_up, n_dn-+1) for s = 1 on the same Ns).
 * Sign (-1)^(occupied modes before (i, s)), Eqs. (7)-(8).  DEVICE pointers,
 * asynchronous on stream.                                                    */
ed_status ed_apply_fermion_op(ed_ctx* ctx, ed_ctx* ctx_dst, int site, int spin,
                              int create, const void* psi, void* out,
                              ed_dtype dtype, void* stream);

/* Adaptive Krylov dimension (the a-posteriori exit of Algorithm 6, Sec. 3.4)
 * for the ed_propagate and ed_spectral_propagate calls made on ctx after
 * this one.  tol = 0 (the default): every step uses exactly m Lanczos
 * vectors (unless the Krylov space breaks down).  tol > 0: m becomes the
 * maximum; after Lanczos step j < m the step's approximation
 * y^(j) = exp(-i tau T_j) e_1 is compared with y^(j-1) (zero-padded; y^(0) =
 * 0): delta = |y^(j) - y^(j-1)| / |y^(j)|, epsilon = min(1 + |y^(j)|,
 * delta / (1 - delta) |y^(j)|) for delta < 1 and 1 + |y^(j)| otherwise, and
 * the step ends with dimension j once epsilon < tol or beta_j < tol * alpha,
 * alpha = max(1, |alpha_k|, beta_k over the steps before) as the estimate of
 * |H|.  The dimension used in each step is reported in observables->m_eff.
 * The check of step j runs while the next Lanczos pass proceeds, so one pass
 * past the exit is computed and discarded.  ED_ERR_ARG for a negative or
 * non-finite tol.                                                            */
ed_status ed_set_krylov_tol(ed_ctx* ctx, double tol);

/* Select the time-stepping scheme (ed_integrator) for the ed_propagate and
 * ed_spectral_propagate calls made on ctx after this one (default
 * ED_MIDPOINT).  With ED_CFET4, n_steps, dt, m, the observables and the
 * Green's functions keep their meaning per time step: docc, norm2 and energy
 * are recorded at t_start + n dt, and m_eff / delta report the larger value of
 * the step's two Krylov steps.  ED_ERR_ARG for an unknown scheme.            */
ed_status ed_set_integrator(ed_ctx* ctx, ed_integrator scheme);

/* The hopping coefficients a propagation of this context uses (host
 * computation, no GPU work): for every Krylov sub-step s of n_steps time
 * steps from t_start (n_sub = n_steps sub-steps for ED_MIDPOINT, at the
 * midpoints t_start + (n + 1/2) dt of Eq. (32); n_sub = 2 n_steps for
 * ED_CFET4, in the order they act) and every bond b,
 * coef[2 (s n_bonds + b)] + i coef[.. + 1] is the matrix element of the hop
 * p_b -> q_b, -t_b exp(-i A(t) . d_b) with the Peierls phase of Eqs. (1)
 * and (3) (for CFET4 the combination of its two field times that the
 * sub-step applies).  The reverse hop carries the conjugate.  *n_sub and
 * *tau (both nullable) receive the number of sub-steps and the sub-step
 * length the Krylov exponential uses with them (dt, or dt / 2 for CFET4).
 * coef is a host buffer of 2 n_sub n_bonds doubles, or NULL to query n_sub
 * only.  pulse may be NULL (A = 0).  ED_ERR_STATE before ed_set_lattice;
 * ED_ERR_ARG for n_steps < 1, a non-finite t_start or dt, or invalid pulse
 * parameters.                                                               */
ed_status ed_step_coefficients(ed_ctx* ctx, const ed_pulse* pulse, double t_start,
                               double dt, int n_steps, double* coef, int* n_sub,
                               double* tau);

/* The small exponential of Algorithm 6 on the current GPU: for each of
 * `batch` real symmetric tridiagonal matrices T_b of order n (1 <= n <= 64;
 * diagonal alpha[b n .. b n + n), off-diagonal beta[b (n-1) ..]),
 * y[b n + i] = (exp(-i tau T_b) e_1)_i as (re, im) pairs, computed by the
 * float64 device routine the propagation's exponential kernel runs (shifted
 * Taylor series with sub-steps).  Host buffers (alpha: batch n doubles, beta:
 * batch (n - 1), may be NULL for n = 1; y: 2 batch n doubles); the call
 * copies them to and from the device and returns when y is written.
 * ED_ERR_ARG for sizes out of range, NULL buffers or non-finite inputs;
 * ED_ERR_CUDA if the device work fails.                                     */
ed_status ed_tridiag_expm(int batch, int n, const double* alpha, const double* beta,
                          double tau, double* y);

/* Kernel configurations of H v (the matrix-vector product inside Lanczos,
 * Eq. (18) applied as T_up (x) 1 + 1 (x) T_dn + diagonal, Sec. 3.2).  Each
 * entry of the library's table fixes the precision, the rows of Psi one
 * thread block owns (rows_per_cta), the column pairs per thread, the target
 * thread blocks per SM, and whether the product runs as one kernel (split =
 * 0: the T_up rows are gathered across the matrix) or as a T_up pass
 * followed by a row pass for the diagonal and T_dn (split = 1; the T_up pass
 * either stages column blocks of all rows in shared memory or gathers rows
 * one chunk of columns at a time, for vectors larger than the L2), and
 * whether an extra producer warp stages the T_up source-row chunks in shared
 * memory with TMA bulk copies (tma = 1; used only for even dim_dn and
 * 16-byte aligned vectors), and whether a thread block takes one row u of
 * rows_per_cta vectors of one sector instead of rows_per_cta rows of one
 * vector (multi_vector = 1: for batches such as the c / c+ propagations of
 * Sec. 3.7, where the T_dn tables and the entry list of u then serve those
 * vectors together; the autotuner does not pick these entries, which
 * measured slower than one-vector blocks on the batches, so they run only
 * when pinned with ed_set_apply_config).
 * ed_apply_config_count returns the number of entries; ed_apply_config_info
 * describes entry `config` (ED_ERR_ARG if out of range; any output pointer
 * may be NULL).                                                              */
int ed_apply_config_count(void);
ed_status ed_apply_config_info(int config, int* fp64, int* rows_per_cta,
                               int* pairs_per_thread, int* ctas_per_sm,
                               int* split, int* tma, int* multi_vector);

/* Process-wide choice of the H v configuration for every propagation,
 * ed_apply_H plan and ground-state solve set up after the call (contexts
 * rebuild their plans when it changes).  config = -1 (the default): an
 * autotuner times the feasible entries once per precision and sector shape
 * (sectors under 2^20 elements keep the first feasible entry); otherwise the
 * given entry is used, and calls whose precision or sector it does not fit
 * fail with ED_ERR_CUDA and a message naming it.  ED_ERR_ARG if config is
 * not -1 and not a table index.                                             */
ed_status ed_set_apply_config(int config);

/* The configuration the context's propagation engine (*propagate) and its
 * ed_apply_H plan (*apply) use, or -1 where none has been set up yet.        */
ed_status ed_get_apply_config(const ed_ctx* ctx, int* propagate, int* apply);

/* Cap on the device memory that the Krylov workspace of this context's
 * ed_propagate and ed_spectral_propagate engines (the propagated states the
 * library owns, the m - 1 stored Krylov vectors and one scratch vector per
 * propagated vector) and of its ed_ground_state solves (the restart basis)
 * may take; 0 (the default) = no cap.  A call whose workspace would exceed the
 * cap returns ED_ERR_OOM before allocating anything; a smaller cap set later
 * makes the next call rebuild (and re-check) its workspace.  Tables and the
 * few kilobytes of per-call bookkeeping are not counted.  ED_ERR_ARG for a
 * negative size.  (No passage of the paper: a deployment control.)          */
ed_status ed_set_workspace_limit(ed_ctx* ctx, int64_t bytes);

/* Test hook for the bounded device-side waits (process-wide; applies to the
 * propagation engines, ed_apply_H plans and ground-state solves set up after
 * the call, which rebuild when it changes).  The TMA configurations of the
 * H v kernel (tma = 1 in ed_apply_config_info) wait on shared-memory
 * barriers for the T_up row copies of a producer warp; every such wait gives
 * up after wait_polls polls (0 = the default, 2^22), records ED_ERR_TIMEOUT
 * in the vector's status and lets the kernel finish, so that the context
 * stays usable.  withhold_copy >= 0 makes the producer of every thread block
 * stop before that copy (counted from 0 per block) instead of issuing it, so
 * that the consumers' wait for it runs out: ed_propagate and
 * ed_spectral_propagate then return ED_ERR_TIMEOUT (ed_apply_H runs
 * asynchronously and does not read the status).  No copy is left in flight
 * when a block ends.  withhold_copy = -1 (the default) turns the hook off.
 * ED_ERR_ARG for withhold_copy < -1 or wait_polls outside 0..2^32-1.
 * (No passage of the paper: a check of the library's own failure path.)    */
ed_status ed_set_wait_fault(int withhold_copy, int64_t wait_polls);

/* Bytes of device memory the context currently holds (tables + workspace).  */
ed_status ed_device_bytes(const ed_ctx* ctx, int64_t* bytes);

/* Release the context and all device memory it owns.  NULL is accepted.      */
ed_status ed_destroy(ed_ctx* ctx);

/* Message of the last failing call on ctx (ctx may be NULL).  Never NULL.    */
const char* ed_last_error(const ed_ctx* ctx);

/* Library version string.                                                    */
const char* ed_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HUBBARD_ED_H */
