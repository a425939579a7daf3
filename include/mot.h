/*
 * mot.h - C ABI of the GB300 MOT-JVIE marching library (arXiv 2407.03323).
 *
 * The library marches the contrast-current-density volume integral equation in time
 * (Sec. 2, Eqs. MOTInversion and PnMOT):
 *
 *     Z_0 J_n = E_n - P_{n-1},     P_{n-1} = sum_{l=1}^{ell} Z_l J_{n-l},
 *
 * on a uniform voxel grid, with the history P evaluated by zero-padded 3D FFTs
 * (Sec. 3, Eq. PnFFTMOT, App. A), the FIR regularisation Z_n + delta_n I (Sec. 6.1)
 * and a conjugate-gradient solve of the near-field operator Z_0 each step.
 *
 * Conventions for every call:
 *  - Units: c0 = 1, eps0 = 1.  Voxels are cubes of edge h with c0 dt = h (the
 *    paper's setting, Sec. 5.2); any other h/dt is rejected with MOT_ERR_ARG.
 *  - Voxel index m = u + U (v + V w), 0-based (Sec. 2.2).  Vectors over unknowns are
 *    "AoS": element [m][b], b = x, y, z (Eqs. CurrentVector, ExcitationVector).
 *  - Time steps are 1-based as in the paper: the first unknown is J_1 and J_n = 0
 *    for n <= 0 (the incident field arrives after t = 0, Sec. 2.1).
 *  - The caller owns every buffer it passes; the library copies what it keeps and
 *    never frees caller memory.  Pointer arguments may be host or device pointers
 *    where stated; the library tells them apart with cudaPointerGetAttributes.
 *  - Every call returns a mot_status.  On error, mot_last_error(ctx) returns a
 *    message.  A context stays usable after MOT_ERR_ARG / MOT_ERR_NOT_CONVERGED /
 *    MOT_ERR_UNSTABLE; after MOT_ERR_CUDA or MOT_ERR_TIMEOUT it is in
 *    MOT_ERR_STATE and only mot_last_error / mot_get_info / mot_get_levels /
 *    mot_destroy work.
 *  - Calls on one context are not thread safe; separate contexts are independent.
 */
#ifndef MOT_H
#define MOT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mot_ctx mot_ctx;

typedef enum {
    MOT_OK = 0,
    MOT_ERR_ARG = 1,            /* invalid argument (message says which)            */
    MOT_ERR_OOM = 2,            /* device allocation failed                         */
    MOT_ERR_CUDA = 3,           /* CUDA runtime error                               */
    MOT_ERR_NOT_CONVERGED = 4,  /* CG did not reach its tolerance within max_iter    */
    MOT_ERR_UNSTABLE = 5,       /* NaN/Inf or runaway growth of ||J_n|| (Sec. 5.2)   */
    MOT_ERR_TIMEOUT = 6,        /* a device-side wait ran out of its budget          */
    MOT_ERR_STATE = 7           /* context unusable (earlier device fault)           */
} mot_status;

typedef enum {
    MOT_FP64 = 0,          /* every stage in FP64                                    */
    MOT_FP32_HISTORY = 1   /* FFTs, spectra and lag MAC in FP32 with compensated
                              accumulation; element quadrature, Z_0, FIR state and
                              the solution J stay FP64; the CG residual is formed in
                              double-float (float pairs, ~48 bits)                  */
} mot_precision;

typedef enum {
    MOT_HISTORY_DIRECT = 0,  /* every lag 1..ell multiplied per step in the spatial
                                spectral domain (Sec. 3, Eq. PnFFTMOT)                */
    MOT_HISTORY_BLOCKED = 1, /* lags >= B by block Toeplitz products with temporal
                                FFTs (Secs. 4-5); lags < B as in DIRECT.  Levels of
                                length S = B, 2B, ... over lags [S, 2S); where at
                                most half of the last one's lags [a, 2a) are <= ell,
                                it is replaced by the shortest level S' = B 2^j over
                                lags [a, a + S') that reaches ell; mot_get_levels   */
    MOT_HISTORY_BLOCKED_DOUBLING = 2  /* the blocked scheme with every level over
                                [S, 2S), the last one included                       */
} mot_history_scheme;

/*
 * mot_create - build a marching context (setup; not part of the per-step path).
 *
 * Computes ell (Eq. Ell), chi_m = (eps_m - 1)/eps_m (Eq. TDJVIE), the interaction
 * elements G_l(d) = K^face_l(d) - delta_ab K^vol_l(d) for lags 0..ell by FP64
 * quadrature on the GPU (Eq. Z; K^vol_l = int C_d T''(l - r)/(4 pi r),
 * K^face_l^ab = int (d_a d_b C_d) T(l - r)/(4 pi r), C_d the autocorrelation of two
 * voxels at offset d, T the quadratic B-spline basis), their zero-padded spatial
 * spectra (App. A), and allocates the rings.
 *
 *  grid[3]   U, V, W voxels along x, y, z (each >= 1)
 *  h[3]      voxel edges; must be equal
 *  dt        time step; must satisfy c0 dt = h (c0 = 1)
 *  eps_r     host pointer, U*V*W relative permittivities (>= 1), m order; copied
 *  fir_taps  host pointer to delta_0..delta_{n_taps-1} (Z_n + delta_n I, Sec. 6.1);
 *            may be NULL when n_taps = 0; copied
 *  precision mot_precision
 *  scheme    mot_history_scheme
 *  block     block size B for the blocked schemes (power of two, 2..ell), else 0
 *  out       receives the context (NULL on failure)
 * Errors: MOT_ERR_ARG, MOT_ERR_OOM, MOT_ERR_CUDA.  On failure *out is NULL and the
 * message is available from mot_last_error(NULL).
 */
mot_status mot_create(const int grid[3], const double h[3], double dt,
                      const double* eps_r, const double* fir_taps, int n_taps,
                      int precision, int scheme, int block, mot_ctx** out);

/*
 * mot_create_padded - mot_create with the zero-padded FFT lengths chosen by the caller
 * (App. A: any length >= 2 N - 1 per axis makes the circular convolution of the
 * history equal the linear one, so the march is the same up to rounding): fft_len[a]
 * for grid axis a (u, v, w), each even, 7-smooth (radices 2, 3, 5, 7), >= 2 grid[a] - 1
 * and <= 4096; NULL gives mot_create's choice (the smallest such length).  A tuner
 * picks lengths with a compiled four-step codelet (64, 96, 210) or the smallest one by
 * timing.  Errors as mot_create (MOT_ERR_ARG for an invalid length).
 */
mot_status mot_create_padded(const int grid[3], const double h[3], double dt,
                             const double* eps_r, const double* fir_taps, int n_taps,
                             int precision, int scheme, int block, const int fft_len[3],
                             mot_ctx** out);

/*
 * mot_create_shared - a second, independent marching state on the setup of `src`:
 * the same grid, eps_r, FIR taps, precision, history scheme and solver settings, with
 * the element table, kernel and level spectra, geometry and solver setup shared
 * read-only (not recomputed, not copied).  For several excitations of one scatterer
 * marched side by side (each context has its own stream, rings and solver vectors).
 * `src` (or the context it shares from) must outlive every context shared from it.
 *  out   receives the new context (NULL on error; mot_last_error(NULL) explains)
 * Errors: MOT_ERR_ARG, MOT_ERR_STATE (src unusable), MOT_ERR_OOM, MOT_ERR_CUDA.
 */
mot_status mot_create_shared(mot_ctx* src, mot_ctx** out);

/* Release every device and host resource of the context.  NULL is a no-op. */
void mot_destroy(mot_ctx* ctx);

/*
 * mot_set_excitation - stage tested excitation samples E_n (Eq. E) for the next
 * n_steps calls-worth of steps.
 *
 *  n_steps   number of time steps provided (>= 1)
 *  E         [n_steps][M][3] doubles, E_{n0+1} first where n0 is the number of steps
 *            already marched; host or device pointer; copied into a device staging
 *            buffer, which is reallocated if n_steps exceeds its capacity
 *  stream    cudaStream_t to use, or NULL for the context's stream
 * Steps without staged excitation are marched with E = 0.
 * A host E is copied in ~64 MB chunks on a staging stream of the context, and
 * mot_march waits only for the chunk of the step it is about to solve, so the copy
 * overlaps the march.  Pageable host memory is captured before this call returns;
 * page-locked (pinned) host memory is read while the copy runs, so keep it unchanged
 * until mot_march has returned from the steps that consume it.
 * A device E is copied on `stream`, ordered like the caller's own work there.
 */
mot_status mot_set_excitation(mot_ctx* ctx, int n_steps, const double* E, void* stream);

/*
 * mot_plane_wave - tested modulated-Gaussian plane wave (Eq. E) computed on the GPU:
 *   E^b_{m,n} = chi_m p_b (1/V) int_{V_m} sin(2 pi f_c tau) exp(-tau^2/(2 sigma_t^2)) dV,
 *   tau = n dt - t0 - r . k_hat   (voxel m occupies [u, u+1] x [v, v+1] x [w, w+1] h).
 *  k_hat, p_hat  unit propagation and polarisation vectors (host, 3 doubles each)
 *  f_c, sigma_t, t0   pulse parameters in units of dt
 *  n_first   first time index n (1-based); n_steps samples are produced
 *  E_out     [n_steps][M][3] doubles, host or device pointer
 */
mot_status mot_plane_wave(mot_ctx* ctx, const double k_hat[3], const double p_hat[3],
                          double f_c, double sigma_t, double t0, int n_first, int n_steps,
                          double* E_out, void* stream);

/*
 * mot_plane_wave_static - mot_plane_wave into HOST memory without allocating device
 * memory.  The paper has no counterpart: this is a library service for callers that
 * must not allocate during a call (a process whose own pool reserves the device's
 * memory up front, so a cudaMalloc could fail mid-run; a loop that cannot absorb the
 * device-wide synchronisation of cudaFree).  mot_plane_wave stages a host result in a
 * device buffer it allocates per call; this variant stages it in one fixed device
 * array of 2^21 doubles (16 MiB) per device.
 *  arguments  as mot_plane_wave; E_out must be host memory ([n_steps][M][3] doubles,
 *             pageable or pinned), else MOT_ERR_ARG
 *  limits     3 * M * n_steps <= 2^21, else MOT_ERR_ARG naming both numbers; split
 *             longer requests over several calls (n_first advances by n_steps)
 *  set-up     the first call on a device resolves the array's address there (and may
 *             load the module): make it before any stream capture on that device
 *  device     runs on the device the context was created on, whichever device is
 *             current; the caller's current device is restored before returning
 *  zeroing    none needed: every staged element is written before it is copied out
 *  races      one array per device per process: calls that overlap in time (several
 *             host threads, any contexts on the same device) overwrite each other's
 *             staging data and must be serialised by the caller
 *  Returns after the result is in E_out (the stream is synchronised).
 */
mot_status mot_plane_wave_static(mot_ctx* ctx, const double k_hat[3], const double p_hat[3],
                                 double f_c, double sigma_t, double t0, int n_first,
                                 int n_steps, double* E_out, void* stream);

/*
 * mot_march - advance the march by n_steps time steps.
 *  J_out     [n_steps][M][3] doubles receiving J_{n0+1} .. J_{n0+n_steps} (host or
 *            device pointer), or NULL to keep the result on the device only; a host
 *            J_out is filled through a 3-slot device ring whose device-to-host copies
 *            run on a copy stream while the next steps compute, and is complete when
 *            the call returns
 *  stream    cudaStream_t or NULL
 * Errors: MOT_ERR_NOT_CONVERGED (CG exceeded max_iter; J of that step is the last
 * iterate), MOT_ERR_UNSTABLE (NaN/Inf or ||J_n|| above the growth limit; see
 * mot_get_info for the step), MOT_ERR_CUDA.
 */
mot_status mot_march(mot_ctx* ctx, int n_steps, double* J_out, void* stream);

/*
 * mot_eval_history - evaluate P_{n-1} = sum_{l=1}^{ell} Z_l J_{n-l} (Eq. PnMOT,
 * FIR taps included) for a caller-given past, through the same FFT / lag-MAC path
 * the march uses.  The march state is reset (n0 = 0) before and after.
 *  n_hist    number of past steps given (1..ell); older ones are zero
 *  J_hist    [n_hist][M][3], J_{n-1} first (host or device)
 *  P_out     [M][3] (host or device)
 */
mot_status mot_eval_history(mot_ctx* ctx, int n_hist, const double* J_hist, double* P_out,
                            void* stream);

/*
 * mot_adjoint - gradient of an objective O(J_1 .. J_N) with respect to eps_r per voxel,
 * by the adjoint march: the transposed system of Eq. MatrixEquation solved backwards
 * in time, Z_0^T lambda_n = g_n - sum_{l>=1} Z_l^T lambda_{n+l}, n = N .. 1, with
 * g_n = dO/dJ_n and Z_l^T lambda = (T(l)/eps + delta_l) lambda - G_l * (chi lambda)
 * (G_l is symmetric).  The gradient is
 *     dO/deps_m = (1/eps_m^2) sum_n lambda_{n,m} . (1/chi_m) sum_l (T(l) + delta_l) J_{n-l,m},
 * the chi-derivative of the forward rows (Eq. Z, Eq. E) simplified with the forward
 * equation itself; it is defined for voxels with eps_m > 1 and set to 0 where eps_m = 1.
 *  n_steps   N
 *  J         [N][M][3] forward currents J_1 .. J_N (from mot_march; host or device)
 *  dO_dJ     [N][M][3] g_n (host or device)
 *  grad_eps  [M] output (host or device)
 *  lambda    [N][M][3] optional output of lambda_1 .. lambda_N, or NULL
 *  stream    cudaStream_t or NULL
 * The march state is reset before and after; the same context (precision, history
 * scheme, FIR taps, solver settings) serves forward and adjoint.
 * Errors: MOT_ERR_ARG, MOT_ERR_OOM, MOT_ERR_NOT_CONVERGED, MOT_ERR_CUDA.
 */
mot_status mot_adjoint(mot_ctx* ctx, int n_steps, const double* J, const double* dO_dJ,
                       double* grad_eps, double* lambda, void* stream);

/*
 * The adjoint march in segments (checkpointed gradients).  mot_adjoint is one segment
 * of these.  Row m of the gradient at step n reads J_{n-l,m} for l < L = max(taps, 2)
 * only, so a segment needs the currents of its own steps and L - 1 before them, which
 * the caller may recompute from a checkpoint (mot_restart) instead of keeping all N.
 *
 * mot_adjoint_begin - open an adjoint run of N = n_total forward steps on the context
 *   (resets the march state; mot_march / mot_eval_history / mot_restart are refused
 *   until mot_adjoint_end).
 * mot_adjoint_run - advance by n_count adjoint steps: forward steps n_hi down to
 *   n_lo = n_hi - n_count + 1, where n_hi = N - (adjoint steps done so far).
 *  J_win      [win_count][M][3] currents J_{win_first} .. (host or device); must cover
 *             steps max(1, n_lo - L + 1) .. n_hi
 *  dO_dJ      [n_count][M][3] g_n for n = n_lo .. n_hi (host or device)
 *  lambda     [n_count][M][3] optional output of lambda_{n_lo} .. lambda_{n_hi}, or NULL
 * mot_adjoint_end - close the run; with grad_eps non-NULL (all N steps done) write
 *   dO/deps [M] (host or device) as for mot_adjoint; NULL abandons the run.
 * Errors: MOT_ERR_ARG (no open run, coverage, steps left), MOT_ERR_OOM,
 * MOT_ERR_NOT_CONVERGED / MOT_ERR_UNSTABLE (the run stays open), MOT_ERR_CUDA.
 */
mot_status mot_adjoint_begin(mot_ctx* ctx, int n_total, void* stream);
mot_status mot_adjoint_run(mot_ctx* ctx, int n_count, const double* J_win, int win_first,
                           int win_count, const double* dO_dJ, double* lambda, void* stream);
mot_status mot_adjoint_end(mot_ctx* ctx, double* grad_eps, void* stream);

/*
 * mot_restart - continue a march from a saved history: afterwards the next mot_march
 * step is n0 + 1, exactly as if J_1 .. J_n0 had been marched (the history sum of
 * Eq. PnMOT reaches back ell steps, so the last ell currents determine every later
 * step; the spectral ring and the far-level accumulators are rebuilt by replaying the
 * history path over them).
 *  n0      steps already marched (>= 0; 0 restarts from rest)
 *  n_hist  currents given, min(n0, ell) <= n_hist <= n0
 *  J_hist  [n_hist][M][3] J_{n0-n_hist+1} .. J_n0 (host or device)
 * Staged excitation is cleared (stage E_{n0+1}.. with mot_set_excitation).
 * Errors: MOT_ERR_ARG, MOT_ERR_OOM, MOT_ERR_CUDA.
 */
mot_status mot_restart(mot_ctx* ctx, int n0, int n_hist, const double* J_hist, void* stream);

/*
 * mot_get_table - copy interaction elements G_l^{ab}(d) of lags l0..l0+n_lags-1 on
 * the octant d in [0,U-1]x[0,V-1]x[0,W-1] to host memory.
 *  out  host pointer, [n_lags][6][W][V][U] doubles, component order xx, yy, zz,
 *       xy, xz, yz; other octants follow by parity (diagonal even in each d_i, the
 *       (a, b) component odd in d_a and d_b)
 */
mot_status mot_get_table(mot_ctx* ctx, int l0, int n_lags, double* out);

/*
 * mot_get_spectrum - copy the spatial spectrum of lag l (1..ell) on the octant of
 * frequencies k_i in [0, P_i/2]:  Ghat_l^{ab}(k) = sum_d G_l^{ab}(d) exp(-2 pi i k.d/P)
 * (real by the parity of G; App. A with the circulant embedding of size P_i).
 *  out  host pointer, [6][Pw/2+1][Pv/2+1][Pu/2+1] doubles (unnormalised)
 */
mot_status mot_get_spectrum(mot_ctx* ctx, int l, double* out);

/*
 * Positive definite stability analysis (Sec. 5.1, Eq. Dn).  The PDSA matrices
 *     D_n = sum_{i=0}^{n} (-1)^i C(ell - i, n - i) Z_i,   n = 0..ell,
 * (D_0 = Z_0, D_ell = sum_i (-1)^i Z_i = Z(z = -1)) all positive definite keep every
 * companion-matrix eigenvalue on the negative real axis inside the unit circle.  The
 * functions below work on the scaled operator
 *     A_n = diag(1/chi) D_n / C(ell, n)
 * restricted to the active voxels (eps_r > 1; the other rows only hold their own
 * diagonal and a current that stays zero).  A_n is symmetric and has the signs of
 * D_n's eigenvalues; its Z_i include this context's FIR taps (Sec. 6.1), so
 * D_ell^delta = D_ell + delta I (Eq. Regularization) is analysed by creating the
 * context with the taps.  The Toeplitz part sum_i c_i G_i is applied as one spatial
 * FFT convolution on the padded grid (App. A).  FP64 contexts only (MOT_ERR_ARG
 * otherwise); the context's stream is used and the calls are synchronous.  The
 * operator of the last (n, flags) is cached in the context (a [noct][6] FP64 kernel
 * spectrum, an [M] diagonal and FFT scratch, freed by mot_destroy).
 *  n      0 <= n <= ell
 *  flags  0, or MOT_PDSA_FP32_SPECTRUM: every lag's spectrum Ghat_i (i >= 1) is
 *         rounded to FP32 before it is summed, as the FP32-history direct scheme
 *         multiplies it, so the analysis includes that finite-precision error
 *         (the perturbation N of Eq. DellFinitePrecision)
 * Errors: MOT_ERR_ARG (bad n, flags, pointer, precision), MOT_ERR_OOM, MOT_ERR_CUDA.
 */
#define MOT_PDSA_FP32_SPECTRUM 1

/*
 * mot_pdsa_apply - y = A_n x.
 *  x, y  [M][3] doubles, host or device; entries of voxels with eps_r = 1 are ignored
 *        in x and returned 0 in y
 */
mot_status mot_pdsa_apply(mot_ctx* ctx, int n, int flags, const double* x, double* y);

/*
 * mot_pdsa_bounds - rigorous bracket of the spectrum of A_n from the circulant
 * embedding of its Toeplitz part (Weyl's inequality and Cauchy interlacing):
 *  out  host pointer, 5 doubles: [0] lower bound of lambda_min(A_n), [1] upper bound
 *       of lambda_max(A_n), [2] min and [3] max eigenvalue of the 3x3 blocks of the
 *       padded kernel spectrum, [4] the largest chi over active voxels
 * A positive out[0] proves D_n positive definite; a negative one decides nothing.
 */
mot_status mot_pdsa_bounds(mot_ctx* ctx, int n, int flags, double out[5]);

/*
 * mot_pdsa_lanczos - extreme eigenvalues of A_n by k Lanczos steps on the device from
 * a start vector drawn from `seed`.
 *  flags   MOT_PDSA_FP32_SPECTRUM as above; MOT_PDSA_FULL_REORTH keeps the basis and
 *          reorthogonalises every step against it (device memory (k + 1) 3M doubles),
 *          else the plain three-term recurrence runs (memory 4 x 3M doubles; k may
 *          exceed the dimension: lost orthogonality only repeats converged Ritz values)
 *  k       steps (>= 1); fewer are taken when the Krylov space becomes invariant
 *  n_out   how many of the smallest Ritz values to return in ritz (ascending)
 *  ritz    host pointer, n_out doubles (may be NULL when n_out = 0)
 *  info    host pointer, 2 ints: [0] Ritz values written, [1] steps taken
 *  extreme host pointer, 4 doubles: smallest Ritz value, its residual norm
 *          ||A y - theta y||, largest Ritz value, its residual norm; each lies within
 *          its residual of an eigenvalue of A_n
 * The smallest Ritz value is an upper bound of lambda_min(A_n) (to rounding of order
 * k eps ||A_n|| without reorthogonalisation): a clearly negative value proves that D_n
 * is not positive definite.
 */
#define MOT_PDSA_FULL_REORTH 2
mot_status mot_pdsa_lanczos(mot_ctx* ctx, int n, int flags, int k, unsigned long long seed,
                            int n_out, double* ritz, int info[2], double extreme[4]);

/*
 * mot_truncate_table - the truncated MOT-JVIE of the finite-precision experiment
 * (Sec. 6): every tabulated element G_l^{ab}(d) of a history lag l >= 1 is replaced
 * by the nearest multiple of eps_trunc (ties to even) and the spectra derived from the
 * table are recomputed.  The lag-0 elements (the stencil of the Z_0 solve) are kept.
 * Call on a fresh context (no step marched, not created by or shared with
 * mot_create_shared).
 * Errors: MOT_ERR_ARG (eps_trunc not finite and > 0, context marched or shared),
 *         MOT_ERR_CUDA.
 */
mot_status mot_truncate_table(mot_ctx* ctx, double eps_trunc);

/*
 * mot_fir_magnitude - FIR-regularisation magnitude |sum_n exp(-i n theta) delta_n|
 * (Eq. FIRmagnitude) of the taps delta_0..delta_{n_taps-1} at n_theta normalised
 * frequencies theta (host arrays; out host, n_theta doubles).  Host computation, no
 * device use.  Errors: MOT_ERR_ARG (negative counts, NULL arrays).
 */
mot_status mot_fir_magnitude(const double* taps, int n_taps, int n_theta, const double* theta,
                             double* out);

/*
 * mot_frequency_response - |H^alpha|(r, f) of Eq. Halpha at n_probe probe voxels from
 * their time series, on the device (Sec. 7.1).  The series J_n (n = 1..n_steps, time
 * t_n = n dt) is tapered by a half cosine over its last fraction `taper` (the samples
 * n > n_steps - floor(taper n_steps) weigh 0.5 (1 + cos(pi (n - n_flat) / (n_steps -
 * n_flat)))), transformed as j(f) = dt sum_n w_n J_n exp(-2 pi i f t_n), and divided by
 * (eps_r - 1) |e^i(f)| with the amplitude spectrum of the modulated Gaussian pulse
 * sin(2 pi f_c tau) exp(-tau^2 / (2 sigma_t^2)) (eps0 = c0 = 1):
 *     |e^i(f)| = sigma_t sqrt(2 pi) / 2 |exp(-2 pi^2 sigma_t^2 (f - f_c)^2)
 *                                       - exp(-2 pi^2 sigma_t^2 (f + f_c)^2)|.
 *  J          [n_steps][n_probe][3] doubles, host or device
 *  taper      in [0, 1)
 *  eps_probe  host, n_probe values of eps_r (> 1) at the probes
 *  freqs      host, n_freq frequencies (cycles per unit time, c0 = h = 1)
 *  H          host, [n_freq][n_probe][3] doubles
 *  j_hat      host or NULL, [n_freq][n_probe][3] complex (re, im) doubles
 * Synchronous on the default stream.  Errors: MOT_ERR_ARG, MOT_ERR_OOM, MOT_ERR_CUDA.
 */
mot_status mot_frequency_response(int n_steps, int n_probe, const double* J, double dt,
                                  double taper, const double* eps_probe, double f_c,
                                  double sigma_t, int n_freq, const double* freqs, double* H,
                                  double* j_hat);

/* Grid facts and the last march's diagnostics.  Any pointer may be NULL.
 *  ell, P[3]            lags and padded FFT sizes
 *  n_done               steps marched so far
 *  last_norm            ||J_{n_done}||_2
 *  fail_step            step index of the first UNSTABLE/NOT_CONVERGED event, or 0
 *  last_cg_iters        CG iterations of the last step                             */
mot_status mot_get_info(const mot_ctx* ctx, int* ell, int P[3], int* n_done,
                        double* last_norm, int* fail_step, int* last_cg_iters);

/*
 * mot_get_levels - the far levels of the blocked schemes (Secs. 4-5): level k has
 * length S[k] (it fires at every step n with (n - 1) mod S[k] = 0, a temporal FFT of
 * length 2 S[k]) and covers lags lag0[k] .. lag0[k] + S[k] - 1; lags 1 .. B - 1 are
 * the near lags.  The firing pattern repeats every max S[k] steps (the period that
 * mot_set_graph requires).
 *  max_levels  capacity of S and lag0 (at most 8 levels exist)
 *  n_levels    receives the number of levels (0 for MOT_HISTORY_DIRECT)
 *  S, lag0     host arrays of max_levels ints, or NULL; the first
 *              min(n_levels, max_levels) entries are written
 * Errors: MOT_ERR_ARG (ctx or n_levels NULL, max_levels < 0); MOT_ERR_STATE after a
 * CUDA error (the values are still written).
 */
mot_status mot_get_levels(const mot_ctx* ctx, int max_levels, int* n_levels, int* S, int* lag0);

/*
 * mot_level_plan - the far levels that a context with this block size, ell and history
 * scheme would use (the plan of mot_get_levels, Secs. 4-5), computed on the host with
 * no context and no device.
 *  block       block size B (power of two >= 2; ignored for MOT_HISTORY_DIRECT)
 *  ell         number of history lags (>= 1; mot_create derives it from the grid, Eq. Ell)
 *  scheme      mot_history_scheme
 *  max_levels, n_levels, S, lag0   as for mot_get_levels
 * Errors: MOT_ERR_ARG (bad argument, or more than 8 levels needed: raise B); the message
 * is available from mot_last_error(NULL).
 */
mot_status mot_level_plan(int block, int ell, int scheme, int max_levels, int* n_levels, int* S,
                          int* lag0);

/* Set per-step solver/monitor parameters.  tol: the FP64 residual of the Z_0 solve
 * must fall below tol ||rhs / chi|| (default 1e-13 for MOT_FP64, 3e-8 for
 * MOT_FP32_HISTORY, whose history already carries ~2e-7 relative error); max_iter:
 * cap on the inner (FP32) iterations per step (default 200); growth_limit: a step
 * whose ||J_n|| exceeds growth_limit times the largest norm seen so far is reported
 * as MOT_ERR_UNSTABLE (default 1e12). */
mot_status mot_set_solver(mot_ctx* ctx, double tol, int max_iter, double growth_limit);

/* Counters of mot_march calls since the last mot_set_profiling (or creation).
 *  launches      kernels launched by mot_march
 *  mac_launches  of which lag multiply-accumulate kernels
 *  steps         time steps marched
 *  cg_iters      total CG iterations
 *  far_launches  of which block Toeplitz (temporal FFT) kernels, blocked scheme
 *  ms_*          summed CUDA-event durations of the phases, recorded on the stream
 *                mot_march ran on, only while profiling is enabled: forward FFT of
 *                J_{n-1}, far-lag block products (blocked scheme), near-lag MAC,
 *                inverse FFT, rhs + solve                                          */
typedef struct {
    long long launches;
    long long mac_launches;
    long long far_launches;
    long long steps;
    long long cg_iters;
    double ms_fft_fwd;
    double ms_far;
    double ms_mac;
    double ms_fft_inv;
    double ms_solve;
    long long graph_launches;        /* periods launched as one CUDA graph (mot_set_graph) */
    long long graph_instantiations;  /* executable graphs built (first period, or after an
                                        in-place update was refused)                     */
} mot_stats;

/*
 * Several right-hand sides of one scatterer (the n_rhs dimension of the excitation):
 * the excitations E^(r) of Eq. E for r < n_rhs, marched by Eq. MOTInversion with the
 * same Z_l, each its own march state.
 * mot_set_excitation_rhs - stage E for the context's n_rhs right-hand sides.  E is
 *   [r][n_steps][M][3] (host or device, read during the call or on the stream as for
 *   mot_set_excitation): right-hand side 0 is the context itself, the others are
 *   contexts sharing its setup (made here, owned and destroyed with it).  n_rhs may
 *   change only before the first step.  Errors: MOT_ERR_ARG (n_rhs outside 1..4096,
 *   n_steps < 1, NULL E, ctx made by mot_create_shared, n_rhs changed after marching),
 *   MOT_ERR_OOM, MOT_ERR_CUDA.
 * mot_march_rhs - march every right-hand side n_steps steps, the steps of all of them
 *   interleaved on their own streams (all on `stream` when it is not NULL); J_out is
 *   [r][n_steps][M][3] (host or device) or NULL.  Returns the first failing right-hand
 *   side's status (mot_last_error names it); each one's monitor state is its own
 *   (mot_rhs_context + mot_get_info).  Graph-captured periods are not used here.
 * mot_rhs_context - the context of right-hand side k (k = 0: ctx itself), owned by ctx,
 *   for per-right-hand-side queries (mot_get_info, mot_get_stats, mot_restart ...);
 *   mot_destroy on it does nothing (it is destroyed with ctx).
 *   Errors: MOT_ERR_ARG (k outside 0..n_rhs - 1).
 * mot_set_solver on ctx applies to all its right-hand sides.
 */
mot_status mot_set_excitation_rhs(mot_ctx* ctx, int n_rhs, int n_steps, const double* E,
                                  void* stream);
mot_status mot_march_rhs(mot_ctx* ctx, int n_steps, double* J_out, void* stream);
mot_status mot_rhs_context(mot_ctx* ctx, int k, mot_ctx** out);

/*
 * mot_set_graph - march whole periods as CUDA graphs (no counterpart in the paper:
 * launch overhead).  With steps_per_graph = Q > 0, mot_march captures the launches of
 * Q consecutive steps (every step's history transform, far-level firings, near-lag
 * MAC, inverse transform, epilogue and solve of Eqs. PnFFTMOT and MOTInversion) into a
 * graph and launches it as one unit.  A period starts at a step n with (n - 1) mod Q = 0
 * and n >= 2, where every level fires, so the graphs of all periods hold the same
 * kernels in the same order: the first is instantiated, the later ones update it in
 * place (ring slots, step index, excitation and output pointers).  Steps outside whole
 * periods are launched one by one.  Results are identical to mot_march without graphs.
 * Used only when the excitation is on the device (or fully staged), J_out is NULL or a
 * device pointer, profiling is off and the stream is not a default stream; otherwise
 * mot_march launches step by step.  Q = 0 turns graphs off.
 * Errors: MOT_ERR_ARG (Q < 0 or Q > 65536; with a blocked scheme Q not a multiple of
 * the longest level's length, see mot_get_levels).
 */
mot_status mot_set_graph(mot_ctx* ctx, int steps_per_graph);

/* Enable (1) or disable (0) per-phase event timing in mot_march and reset the
 * counters.  Timing adds five event records per step. */
mot_status mot_set_profiling(mot_ctx* ctx, int enable);

/* Copy the counters (see mot_stats) to *out (host pointer). */
mot_status mot_get_stats(const mot_ctx* ctx, mot_stats* out);

/*
 * Probe field: the scattered field at probe voxels, for objectives such as the
 * time-gated field energy around the scatterer.  A probe is a voxel of the grid's
 * lattice, inside or outside the grid (lattice indices (u, v, w), any integers); its
 * field is the tested, voxel-averaged field of Eq. E at that virtual vacuum voxel, which
 * the march's own interaction elements give (Eq. Z; no local term in vacuum):
 *     E^s_p(t_n) = sum_{l>=0} sum_m G_l(r_p - r_m) J_{n-l,m},
 * and its transpose, the source of the adjoint march for an objective of E^s,
 *     g_{k,m} = sum_{l>=0} sum_p G_l(r_p - r_m) W_{k+l,p}      (G_l is symmetric).
 *
 * mot_probe_setup - compute the element windows of every probe-voxel pair on the
 *   device (the quadrature of mot_create on the distinct sorted offsets) and keep them
 *   in the context: P x M x 6 x 8 doubles (2.7 GB for 64 probes on a 48^3 grid).
 *   probes  host, [n_probes][3] ints (u, v, w); replaces an earlier probe set
 *   Errors: MOT_ERR_ARG (counts, pointers, probes so far away that the offset table
 *   exceeds 2^28 entries), MOT_ERR_OOM, MOT_ERR_CUDA.
 * mot_probe_field - E = the probe field of the currents J.
 *   J  [n_steps][M][3] J_1 .. J_{n_steps} (host or device);  E  [n_steps][P][3]
 *   (host or device).  Synchronous on `stream` (or the context's stream).
 * mot_probe_transpose - g = the transposed probe operator applied to W.
 *   W  [n_steps][P][3] (host or device);  g  [n_steps][M][3] (host or device).
 * FP64 throughout.  Errors: MOT_ERR_ARG (no probes, counts, NULL), MOT_ERR_OOM,
 * MOT_ERR_CUDA.
 */
mot_status mot_probe_setup(mot_ctx* ctx, int n_probes, const int* probes);
mot_status mot_probe_field(mot_ctx* ctx, int n_steps, const double* J, double* E, void* stream);
mot_status mot_probe_transpose(mot_ctx* ctx, int n_steps, const double* W, double* g,
                               void* stream);

/*
 * mot_fma_peak - measure the current device's sustained FMA rate (no counterpart in the
 * paper: the denominator of the roofline of kernels bound by arithmetic rather than
 * memory, such as the FP64 history kernels on GPUs whose FP64 rate is a fraction of
 * their FP32 rate).  One launch of independent FMA chains on every SM, timed with CUDA
 * events on the default stream after a warm-up launch; synchronous.
 *  fp64   1: double-precision FMAs, 0: single precision
 *  iters  FMA iterations per chain (>= 1); choose it for a launch of ~0.1 s
 *  ms     receives the launch's duration in milliseconds
 *  flops  receives the floating-point operations it performed (2 per FMA)
 * Errors: MOT_ERR_ARG (NULL outputs, iters < 1), MOT_ERR_OOM, MOT_ERR_CUDA.
 */
mot_status mot_fma_peak(int fp64, int iters, float* ms, double* flops);

/*
 * mot_barrier_check - exercise the bounded wait of the grid barrier that the solve
 * kernel (the CG of Eq. MOTInversion) uses between its passes (no counterpart in the
 * paper: a failure guard).  One cooperative launch of n_blocks blocks on the current
 * device passes `rounds` barriers; block `absent` (0 <= absent < n_blocks; -1: none)
 * returns without arriving, so the other blocks' wait runs out after budget_s seconds
 * of SM clock and the launch ends with a timeout instead of hanging.  Synchronous.
 *  passed         receives the number of blocks that passed every round
 *  timeout_round  receives the round (1-based) at which the wait ran out, 0 if none
 * Returns MOT_OK, MOT_ERR_TIMEOUT (the wait ran out), MOT_ERR_ARG (n_blocks above what
 * can be resident at once, rounds outside 1..2^20, budget_s outside (0, 10], NULL
 * outputs), MOT_ERR_OOM, MOT_ERR_CUDA.  The solve reports the same timeout of one of
 * its barriers (2 s budget) as MOT_ERR_TIMEOUT from mot_march / mot_adjoint_run, with
 * the step in mot_last_error, and the context becomes unusable (MOT_ERR_STATE).
 */
mot_status mot_barrier_check(int n_blocks, int rounds, int absent, double budget_s,
                             int* passed, int* timeout_round);

/* Last error message of ctx, or of the last failed mot_create when ctx is NULL. */
const char* mot_last_error(const mot_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MOT_H */
