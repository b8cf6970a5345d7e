/*
 * gmmnlse.h -- C ABI of the B300 (sm_103a) solver for the generalized
 * multimode nonlinear Schroedinger equation (GMMNLSE) by the massively
 * parallel algorithm (MPA).
 *
 * Method: Wright et al., "Multimode Nonlinear Fiber Optics: Massively
 * Parallel Numerical Solver, Tutorial and Outlook", arXiv:1708.05324.
 *   - the equation solved is Eq. 1 (Sec. III) with S^K, S^R of Eq. 2;
 *   - the solver is the MPA of Sec. III.D: the interaction-picture change of
 *     variables (Eq. cov), the integral form (Eq. MPA_eq), a long step
 *     L = M dz split into M substeps solved together by fixed-point iteration
 *     with the trapezoid rule over z'.
 *
 * Conventions (all arrays row-major, FP64, owned by the caller; the library
 * copies what it keeps):
 *   - Fields vary as exp(-i w t).  The spectrum is
 *     A~(w_q) = sum_k A(t_k) exp(+i w_q t_k), w_q = 2 pi q / T in FFT order
 *     (q < Nt/2, else q - Nt), T = Nt dt.  D_w = i beta_p(w).
 *   - Time samples t_k = (k - Nt/2) dt for A0/Aout; h_R at t_k = k dt.
 *   - Complex arrays are interleaved (re, im) doubles: [N][Nt][2].
 *
 * Every call returns an int status: GMMNLSE_OK (0), GMMNLSE_PENDING (1, poll
 * only) or a negative GMMNLSE_E_* code.  No call aborts the process; CUDA
 * failures are reported as GMMNLSE_E_CUDA.  All calls are thread-safe except
 * that one context must not run two gmmnlse_propagate calls at once (use the
 * server for concurrency).
 */
#ifndef GMMNLSE_H
#define GMMNLSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GMMNLSE_OK                0
#define GMMNLSE_PENDING           1
#define GMMNLSE_E_INVALID        -1  /* bad argument (shape, NaN input, null) */
#define GMMNLSE_E_NOMEM          -2  /* device allocation failed / over budget */
#define GMMNLSE_E_UNSUPPORTED    -3  /* valid input outside what is built */
#define GMMNLSE_E_NOT_CONVERGED  -4  /* max_iter reached above tol */
#define GMMNLSE_E_NONFINITE      -5  /* NaN/Inf appeared in the field */
#define GMMNLSE_E_CUDA           -6  /* a CUDA call failed */
#define GMMNLSE_E_BUSY           -7  /* server queue full */
#define GMMNLSE_E_CANCELLED      -8  /* request cancelled at server shutdown */

/* Arithmetic of the MPA iteration.  The running field between long steps,
 * the dispersion phase beta*z (reduced mod 2 pi), the convergence norm and
 * the energy / photon-number sums are FP64 in every mode. */
typedef enum gmmnlse_precision {
    GMMNLSE_FP64 = 0,       /* everything FP64 */
    GMMNLSE_FP32 = 1,       /* FFTs, contraction and iterates FP32 */
    GMMNLSE_MIXED_BF16 = 2, /* FP32, coupling contraction on tensor cores in
                               BF16 with hi/lo split operands, FP32 accumulate,
                               for every N = 9..64 with Nt a multiple of 128
                               (Nt not a multiple of 128 with N > 8:
                               GMMNLSE_E_UNSUPPORTED); for N <= 8 the FP32
                               register contraction, faster there */
    GMMNLSE_MIXED_FP16 = 3, /* as MIXED_BF16 with FP16 hi/lo operands, each
                               scaled by a power of two into FP16 range (exact
                               to undo); N and Nt limits as MIXED_BF16 */
    GMMNLSE_MIXED_TF32 = 4  /* as MIXED_BF16 with TF32 hi/lo operands (FP32
                               range, 11-bit significands: three products
                               leave ~2^-21 relative); same limits */
} gmmnlse_precision;

typedef struct gmmnlse_params {
    int N;               /* number of modes, 1 <= N <= 64 */
    int Nt;              /* time samples: power of two, 16 <= Nt <= 16384
                            (FP64 at 16384: every transform of the iterates
                            over a 4-block cluster; not on the no-alloc
                            entry point) */
    double dt;           /* sample spacing [s] */
    double lambda0;      /* centre wavelength [m] (omega0 = 2 pi c / lambda0) */
    double n2;           /* nonlinear index [m^2/W] */
    int self_steepening; /* 1: factor (1 + w/w0) of Eq. MPA_eq; 0: factor 1 */
    int precision;       /* gmmnlse_precision */
    int max_iter;        /* cap on updates per long step (0 -> 50) */
    int fixed_iters;     /* > 0: exactly this many updates per long step,
                            tol ignored (for bit-comparable runs) */
    int device;          /* CUDA device ordinal */
    void* stream;        /* cudaStream_t for gmmnlse_propagate; NULL -> a
                            stream owned by the context */
    int io_device;       /* 1: A0/Aout of gmmnlse_propagate are device
                            pointers (FP64 complex, same layout) */
} gmmnlse_params;

typedef struct gmmnlse_stats {
    double z;             /* fiber position reached [m] */
    int long_steps;       /* long steps completed */
    int iters_total;      /* MPA updates over all long steps */
    int iters_min;        /* fewest updates in one long step */
    int iters_max;        /* most updates in one long step */
    int iter_hist[33];    /* [k]: long steps that took k updates (k >= 32 in [32]) */
    double eps_max;       /* largest final convergence measure of a long step */
    double eps_last;      /* final convergence measure of the last long step */
    double energy_in;     /* dt sum_{p,k} |A_p(t_k)|^2 of A0 [J] */
    double energy_out;    /* the same of Aout [J] */
    double photons_in;    /* sum_{p,q: w0+w_q>0} |A~_p(w_q)|^2 / (w0 + w_q) of A0 */
    double photons_out;   /* the same of Aout */
    double ms;            /* device time of the propagation [ms] */
    int coupling_rank;    /* rank r of the coupling G = X W the contraction
                             used (N > 8, S^R = S^K, r <= 3K/4), else
                             K = N(N+1)/2 (the dense reduced matrix).  The
                             factorisation drops columns below 1e-12 (FP64)
                             or 1e-9 (FP32, mixed) of the largest column of
                             G, under the rounding of the contraction; the
                             environment variable GMMNLSE_DENSE=1 at create
                             keeps the dense matrix */
} gmmnlse_stats;

typedef struct gmmnlse_ctx gmmnlse_ctx;
typedef struct gmmnlse_server gmmnlse_server;

/*
 * gmmnlse_create -- upload a fiber (Eq. 1 coefficients) to the device.
 *
 *   prm   problem size, physical constants, precision, device, stream.
 *   beta  [N][Nt] rad/m in FFT order, already in the frame of mode 1: the
 *         Taylor-series dispersion of Eq. 1, beta_p(w) = db0_p + db1_p w +
 *         sum_{n>=2} beta_n^(p) w^n / n!, so that D_w = i beta_p(w)
 *         (Sec. III.D).  Host pointer.
 *   SK    [N][N][N][N] Kerr coupling S^K_plmn [1/m^2] (Eq. 2).  Host.
 *   SR    [N][N][N][N] Raman coupling S^R_plmn, or NULL (then S^R = S^K).
 *   fR    Raman fraction f_R of Eq. 1 (0 <= fR < 1).
 *   hR    [Nt] Raman response h_R(t_k), t_k = k dt [1/s], normalised by the
 *         caller; NULL allowed when fR == 0.  Host.
 *   out   receives the context.
 *
 * S^K and S^R must be real and symmetric under p<->l and m<->n, as Eq. 2
 * makes them; otherwise GMMNLSE_E_UNSUPPORTED.  Non-finite inputs or a
 * non-power-of-two Nt give GMMNLSE_E_INVALID.  The context owns its device
 * memory until gmmnlse_destroy; it is read-only after creation and may be
 * shared by concurrent server requests.
 * With N <= 8 and the contraction on the CUDA cores, create compiles a
 * contraction kernel for the context's nonzero coupling entries (NVRTC,
 * opened at run time; about 0.1 s); if that cannot be done the dense
 * register kernel runs instead.  GMMNLSE_NZ=0 in the environment keeps the
 * dense kernel; GMMNLSE_NZ=require makes a failed build GMMNLSE_E_CUDA.
 */
int gmmnlse_create(const gmmnlse_params* prm, const double* beta, const double* SK,
                   const double* SR, double fR, const double* hR, gmmnlse_ctx** out);

/*
 * gmmnlse_create_general -- the same, with complex coupling tensors and no
 * symmetry assumed: Eq. 1 as written, without the single-polarization,
 * real-profile simplification of Eq. 2 (complex or vector mode fields, a
 * complex mode basis such as circularly polarized or orbital-angular-
 * momentum modes).
 *
 *   SK    [N][N][N][N][2] S^K_plmn as (re, im) pairs [1/m^2].  Host.
 *   SR    [N][N][N][N][2] S^R_plmn, or NULL (then S^R = S^K).  Host.
 *   other arguments as for gmmnlse_create.
 *
 * The bracket is evaluated as sum_l A_l R_pl with the complex R_pl =
 * sum_mn S_plmn A_m A_n^* formed from the N^2 real rows of the pair
 * products (Re A_m A_n^* for m <= n, Im A_m A_n^* for m < n) and, with
 * f_R > 0, their convolutions with h_R.  Precision GMMNLSE_FP64 or
 * GMMNLSE_FP32 (the contraction on the CUDA cores) and N <= 32; otherwise
 * GMMNLSE_E_UNSUPPORTED.  gmmnlse_set_gain_saturation (non-zero) and
 * gmmnlse_propagate_noalloc return GMMNLSE_E_UNSUPPORTED on such a context;
 * everything else (gmmnlse_propagate, the RK4IP comparator, the linear
 * terms, the server) takes it as any other.
 */
int gmmnlse_create_general(const gmmnlse_params* prm, const double* beta, const double* SK,
                           const double* SR, double fR, const double* hR, gmmnlse_ctx** out);

/* Free a context and all its device memory.  NULL is accepted. */
int gmmnlse_destroy(gmmnlse_ctx* ctx);

/*
 * gmmnlse_propagate -- propagate A0 over a fiber of length L (Sec. III.D).
 *
 *   A0    [N][Nt] complex launched field A_p(0, t_k) [sqrt(W)]; host pointer
 *         unless prm.io_device.
 *   L     fiber length [m]; must be a whole number of dz (to 1e-9 relative).
 *   dz    substep Delta z [m].
 *   M     substeps per long step (L_long = M dz); the last long step is
 *         shorter when M does not divide L/dz.  1 <= M <= 64.
 *   tol   convergence threshold on eps = ||psi^(n+1) - psi^(n)||_2 /
 *         ||psi^(n+1)||_2 over all substeps, modes and frequencies.
 *   Aout  [N][Nt] complex output A_p(L, t_k); may alias A0.
 *   st    optional statistics (NULL allowed).
 *
 * Synchronous: returns after Aout is written.  On GMMNLSE_E_NOT_CONVERGED
 * or GMMNLSE_E_NONFINITE, Aout holds the field at the end of the last
 * completed long step and st->z says where that is.
 */
int gmmnlse_propagate(gmmnlse_ctx* ctx, const double* A0, double L, double dz, int M,
                      double tol, double* Aout, gmmnlse_stats* st);

/*
 * gmmnlse_set_linear_coupling -- add linear mode coupling to the right-hand
 * side of Eq. 1 (Sec. IV, "Linear mode coupling including disorder"):
 * C_p = i sum_n Q_np A_n, with Q constant along the fiber.
 *
 *   Q   [N][N] real, Q[n][p] = Q_np [1/m] (row n, column p), host pointer;
 *       NULL removes the term.  Copied; the caller keeps its array.
 *
 * The term joins the integrand of the MPA and the nonlinear operator of
 * gmmnlse_propagate_rk4ip, in the context's precision.  Q symmetric keeps
 * the total energy (i Q^T anti-Hermitian); any real Q is accepted.
 * Call it between propagations: it waits for the context's stream and
 * retires the context's captured graphs; server requests on this context
 * must not be in flight.  gmmnlse_propagate_noalloc returns
 * GMMNLSE_E_UNSUPPORTED while a Q is set.  gmmnlse_set_coupling_profile
 * makes Q depend on z.  Non-finite entries give
 * GMMNLSE_E_INVALID; a failed device allocation GMMNLSE_E_NOMEM.
 */
int gmmnlse_set_linear_coupling(gmmnlse_ctx* ctx, const double* Q);

/*
 * gmmnlse_set_gain -- add small-signal gain to the right-hand side of Eq. 1:
 * the term g_p A_p, the lowest order of the gain of Sec. IV ("Saturating
 * gain"; its saturation is gmmnlse_set_gain_saturation).
 *
 *   g   [N] field gain g_p [1/m] per mode (energy grows as exp(2 g_p z)
 *       alone), host pointer; NULL removes the term.  Copied.
 *
 * Same rules as gmmnlse_set_linear_coupling: both terms may be set at once;
 * call between propagations; gmmnlse_propagate_noalloc returns
 * GMMNLSE_E_UNSUPPORTED while either is set; non-finite g gives
 * GMMNLSE_E_INVALID.
 */
int gmmnlse_set_gain(gmmnlse_ctx* ctx, const double* g);

/*
 * gmmnlse_set_gain_saturation -- add the saturation of the gain to the
 * right-hand side of Eq. 1, the first-order term of Sec. IV ("Saturating
 * gain"): - sat sum_{l,m,n} S^R_plmn A_l(t) int A_m(tau) A_n^*(tau) dtau,
 * the integral over the time window at the current z (dt sum_k), beside the
 * small-signal gain g_p A_p of gmmnlse_set_gain.
 *
 *   sat  the coefficient of the term (the paper's 1/I_sat, read as carrying
 *        the units that make the term a rate of A: [1/(J m)] with S^R in
 *        1/m^2); 0 removes the term.  S^R is the context's (S^K when it was
 *        created without one).
 *
 * For an S^R of Eq. 2 (real, symmetric) the term is - sat sum_l R_pl A_l with
 * the real symmetric R_pl = sum_mn S^R_plmn int A_m A_n^* dtau, constant in
 * time within a substep: per substep the library forms the FP64 time
 * integrals of the pair products, R_pl, and adds the term to the MPA's
 * integrand (and to the RK4IP operator).  Same rules as
 * gmmnlse_set_linear_coupling (call between propagations; the allocation-
 * free entry point refuses it).  Negative or non-finite sat gives
 * GMMNLSE_E_INVALID; the device copy of S^R (8 K P bytes) GMMNLSE_E_NOMEM if
 * it cannot be allocated.
 */
int gmmnlse_set_gain_saturation(gmmnlse_ctx* ctx, double sat);

/*
 * gmmnlse_set_coupling_profile -- a longitudinal profile of the linear mode
 * coupling (Sec. IV, "Linear mode coupling including disorder": an index
 * perturbation eps(x, y) f(z) gives Q_np(z) = Q_np f(z), e.g. a long-period
 * grating's cos(2 pi z / period) or a sampled disorder record).
 *
 *   f      [count] samples f(z_k) at z_k = k fdz from the fiber's start,
 *          host pointer (copied), linearly interpolated between samples and
 *          held at f[count - 1] beyond the last; NULL removes the profile
 *          (f = 1).
 *   fdz    sample spacing [m].
 *
 * Multiplies the Q of gmmnlse_set_linear_coupling (no effect without one) at
 * every substep's position z (the MPA) or stage position (RK4IP).  Same rules
 * as gmmnlse_set_linear_coupling; count < 1, fdz <= 0 or non-finite samples
 * give GMMNLSE_E_INVALID.
 */
int gmmnlse_set_coupling_profile(gmmnlse_ctx* ctx, const double* f, int count, double fdz);

/*
 * gmmnlse_overlap_tensor -- the mode overlap tensor of Eq. 2 from mode
 * profiles on a grid, computed on the GPU: S_plmn = int F_p F_l F_m F_n dA /
 * sqrt(int F_p^2 dA int F_l^2 dA int F_m^2 dA int F_n^2 dA), the integrals
 * as sums over the grid cells (one FP64 Gram GEMM of the N(N+1)/2 pair
 * products F_m F_n over the cells, then spread with the norms).
 *
 *   device  CUDA device to run on.
 *   F       [N][G] real mode profiles (any scale), host pointer.
 *   N       modes, 1..64.   G  grid cells (>= 1).   dA  cell area [m^2].
 *   S       [N][N][N][N] output [1/m^2], host pointer, ready for
 *           gmmnlse_create (real and fully symmetric up to rounding).
 *
 * Synchronous; allocates device memory for the call (8 (N G + K^2) bytes,
 * K = N(N+1)/2; GMMNLSE_E_NOMEM if that fails).  Non-finite F, a profile
 * that is zero everywhere, or bad sizes give GMMNLSE_E_INVALID.
 */
int gmmnlse_overlap_tensor(int device, const double* F, int N, long long G, double dA, double* S);

/*
 * gmmnlse_propagate_rk4ip -- the split-step comparator of the MPA (Sec. III.D,
 * Fig. 3): fourth-order Runge-Kutta in the interaction picture (RK4IP), one
 * step of h after another, each step four evaluations of the nonlinear
 * operator N(A~) = i (n2 w0/c) s(w) F{bracket of Eq. 1 at F^-1 A~} made by
 * the same transform, pair/Raman and contraction kernels as the MPA, and
 * exp(i beta h/2) applied three times.
 *
 *   A0, Aout, st  as for gmmnlse_propagate (host unless prm.io_device).
 *   L     fiber length [m]; a whole number of h (to 1e-9 relative).
 *   h     step [m].
 *
 * The field between steps is FP64; N runs in the context's precision.
 * st->long_steps = steps of h, st->iters_total = evaluations of N (4 per
 * step), the energy / photon sums and st->ms as for gmmnlse_propagate.
 * Synchronous.  Allocates 48 bytes per mode and sample of device memory for
 * the call (GMMNLSE_E_NOMEM if that fails).  Non-finite A0 gives
 * GMMNLSE_E_INVALID; a non-finite result GMMNLSE_E_NONFINITE.
 */
int gmmnlse_propagate_rk4ip(gmmnlse_ctx* ctx, const double* A0, double L, double h, double* Aout,
                            gmmnlse_stats* st);

/*
 * gmmnlse_choose_m -- pick the substeps per long step M that propagates
 * fastest from this field (Sec. III.D: the M of largest speed-up depends on
 * how z_NL compares with dz; the paper gives no rule, so it is measured).
 *
 *   A0          [N][Nt] complex field to start from, as for
 *               gmmnlse_propagate (host unless prm.io_device); not changed.
 *   dz, tol     substep and tolerance of the propagation to come.
 *   candidates  [count] values of M to try, each 1..64.
 *   trial_substeps  length of every trial in substeps (the same fiber
 *               piece, trial_substeps * dz, for each candidate; a remainder
 *               long step is taken when M does not divide it).
 *   scratch     [N][Nt] complex buffer on the same side as A0; receives the
 *               trial fields (contents undefined on return).
 *   sec_per_substep  optional [count] output: device seconds per substep of
 *               each candidate's timed trial, +inf where the trial failed.
 *   M_best      receives the fastest candidate.
 *
 * Each candidate propagates the piece twice, untimed then timed with CUDA
 * events on the context's stream, largest M first (the workspace is sized
 * once).  Costs 2 * count trials; synchronous.  Every M converges to the
 * same field up to tol, since the M coupled trapezoid equations of a long
 * step are the implicit trapezoid taken substep after substep.  Returns
 * GMMNLSE_E_INVALID for bad arguments or a non-finite A0; a candidate whose
 * trial fails (GMMNLSE_E_NOT_CONVERGED, ...) is skipped, and if all fail the
 * last trial's status is returned.
 */
int gmmnlse_choose_m(gmmnlse_ctx* ctx, const double* A0, double dz, double tol,
                     const int* candidates, int count, int trial_substeps, double* scratch,
                     double* sec_per_substep, int* M_best);

/* The step sizes chosen by gmmnlse_choose_step. */
typedef struct gmmnlse_step {
    double dz;       /* substep [m]: L divided by a whole number */
    int M;           /* substeps per long step, 1..64 */
    double z_nl;     /* nonlinear length 1 / (gamma0 max_p S^K_pppp P0) [m] */
    double z_im;     /* intermode beat length 1 / max_p |db0_p| [m] (inf: one mode group) */
    double err_est;  /* step-doubling estimate of the relative L2 error over L at
                        the last trial dz (0 when rtol = 0) */
    int trials;      /* trial propagations made */
} gmmnlse_step;

/*
 * gmmnlse_choose_step -- choose the substep dz and the substeps per long step
 * M from the problem's length scales (Sec. III.D: the long step L_long =
 * M dz << z_NL and the substep dz << z_IM, the nonlinear length and the
 * intermode beat length), refined to an accuracy target.
 *
 *   A0       [N][Nt] launched field (host unless prm.io_device); not changed.
 *   L        fiber length [m].
 *   rtol     target relative L2 error of the field at L; 0 keeps the length-
 *            scale rule alone: dz = min(z_NL / 200, z_IM / 10) (the paper's
 *            usual z_NL / dz of about 200; one tenth of the beat length).
 *   tol      iteration tolerance of the trial propagations.
 *   scratch  [2][N][Nt] complex buffer on the same side as A0 (trial fields).
 *   out      the choice.
 *
 * With rtol > 0 the library propagates a trial piece (one nonlinear length,
 * or L if shorter) at dz and dz/2: the trapezoid rule is second order, so
 * (4/3) |A(dz) - A(dz/2)| / |A(dz/2)| estimates the error of A(dz), scaled
 * linearly to L; dz shrinks (at most 4 rounds) until that meets rtol, and
 * never exceeds the length-scale rule.  Then dz = L / ceil(L / dz) and
 * M = floor(z_NL / (10 dz)), clamped to 1..64 and to the substep count.
 * z_NL takes the peak power P0 = max_t sum_p |A_p(t)|^2 and gamma0 =
 * n2 omega0 / c; db0_p = beta_p(0) - beta_1(0) of the context's beta.
 * Synchronous.  GMMNLSE_E_INVALID for bad arguments, a zero or non-finite
 * field, or n2 <= 0; a failing trial's status is returned.
 */
int gmmnlse_choose_step(gmmnlse_ctx* ctx, const double* A0, double L, double rtol, double tol,
                        double* scratch, gmmnlse_step* out);

/*
 * gmmnlse_propagate_noalloc -- gmmnlse_propagate without any memory
 * allocation.  (An addition of this library: the paper has no counterpart.)
 *
 * For callers that cannot have a library allocate device memory: latency-
 * critical loops that cannot take the device-wide synchronisation of
 * cudaMalloc/cudaFree, and programs whose device memory is all owned by
 * their own pool allocator (a framework's caching allocator, a service with
 * a fixed memory budget per GPU).  It runs the same transforms and
 * trapezoid as gmmnlse_propagate with the dense CUDA-core contraction (no
 * tensor cores, no low-rank coupling; st->coupling_rank = K), a host-driven
 * iteration loop that reads the loop state back after every iteration (the
 * call is synchronous), no graphs and no events, with the workspace in one
 * static device array of 32 MiB that every GPU loading the library holds
 * until the process exits.
 *
 *   ctx   a context made beforehand with gmmnlse_create (that call allocates).
 *   A0    [N][Nt] complex128 input field in DEVICE memory of the context's
 *         device (whatever prm.io_device says); Aout the same for the
 *         output.  Any other pointer gives GMMNLSE_E_INVALID.
 *   L, dz, M, tol, st as for gmmnlse_propagate (st->ms is 0).
 *
 * An FP64 context with Nt = 16384 is rejected with GMMNLSE_E_UNSUPPORTED
 * (this entry point has one-block transforms only), and so is a context
 * with a linear coupling or gain set.
 * A problem whose workspace does not fit in the 32 MiB array is rejected with
 * GMMNLSE_E_NOMEM before any work, and gmmnlse_last_error() says so.  (For
 * FP32, N = 6, Nt = 8192, M = 10 with Raman just fits.)  The first call on a
 * device sets that device up (it sets the attributes of this entry point's
 * kernels); make that first call before any stream capture.  Every call
 * looks up the array's device address.
 * All calls share the one array, which keeps what the last call left in it:
 * the entry point resets every part that must start from zero.  Two calls
 * whose work overlaps on the GPU (different streams, or different threads
 * with different contexts on one device) race on the array and give wrong
 * results: serialise them.
 */
int gmmnlse_propagate_noalloc(gmmnlse_ctx* ctx, const double* A0, double L, double dz, int M,
                              double tol, double* Aout, gmmnlse_stats* st);

/* Static, human-readable text for a status code. */
const char* gmmnlse_strerror(int status);

/* Text of the last CUDA failure seen by the calling thread (for
 * GMMNLSE_E_CUDA); empty if none.  Valid until the thread's next call. */
const char* gmmnlse_last_error(void);

/*
 * gmmnlse_profile -- time each kernel of one MPA iteration of this context
 * (Sec. III.D: phase x inverse FFT; pair products + Raman convolution;
 * coupling contraction; forward FFT x integrand prefactor; trapezoid +
 * convergence sums and decision; long-step advance; with the low-rank
 * coupling, slot 1 is the Raman convolution of the rows of Z = W U and slot
 * 2 both GEMMs of the contraction) on the workspace of its last
 * gmmnlse_propagate, which must have used at least M substeps.  Each kernel
 * is launched reps times back to back (after one untimed launch) on the
 * context's stream between two CUDA events.  ms[6] receives the mean duration of each kernel
 * [ms]; bytes[6] its algorithmic bytes per launch (each operand read or
 * written once).  Leaves the workspace iterate in an arbitrary state (the
 * next gmmnlse_propagate starts afresh).
 */
int gmmnlse_profile(gmmnlse_ctx* ctx, int M, int reps, double* ms, double* bytes);

/* Device bytes one in-flight propagation of this context with M substeps
 * keeps resident (its workspace). */
size_t gmmnlse_request_bytes(const gmmnlse_ctx* ctx, int M);

/*
 * Serving: continuous batching of propagation requests.
 *
 * gmmnlse_server_create(hbm_budget, max_inflight, out): a server whose
 * workspaces together hold at most hbm_budget device bytes (as
 * gmmnlse_request_bytes counts one propagation's; every workspace the
 * server keeps, in use or idle for reuse, counts) and that runs at most
 * max_inflight requests at once.  Requests beyond that wait in a queue and
 * are admitted, first fit, as earlier ones finish.
 *
 * Same-shape requests are packed: requests on one context with the same M
 * that run whole long steps (L a whole number of M dz; any dz, tol and
 * field) and no linear coupling, gain or saturation share a workspace of
 * min(max_inflight, 16) slots (the environment variable GMMNLSE_PACK_SLOTS
 * at server creation overrides it; 1 turns packing off), and one launch (a CUDA graph captured once
 * per workspace) advances all of them by one long step, every kernel of the
 * MPA iteration over all slots at once; a request joins or leaves between
 * launches.  Each slot keeps its own convergence, so its result equals that
 * of gmmnlse_propagate on the same input.  Other requests run alone, each on
 * its own stream.  Idle workspaces are freed, oldest first, when a new one
 * would not fit the budget.
 *
 * gmmnlse_submit copies A0 (host) and returns at once with a ticket.  The
 * context must outlive the request.  GMMNLSE_E_BUSY if 65536 requests are
 * queued; GMMNLSE_E_NOMEM if one request alone exceeds the budget.
 *
 * gmmnlse_poll(server, ticket, Aout, st): GMMNLSE_PENDING while the request
 * runs; otherwise its final status, with Aout (host, [N][Nt] complex) and st
 * (NULL allowed) filled as gmmnlse_propagate would.  A finished ticket is
 * released by the poll that reports it; polling it again is
 * GMMNLSE_E_INVALID.
 *
 * gmmnlse_cancel(server, ticket): a request that has not started is
 * cancelled (its poll returns GMMNLSE_E_CANCELLED); GMMNLSE_E_BUSY if it is
 * already running (it then completes normally), GMMNLSE_OK if it has ended.
 *
 * gmmnlse_server_resident_bytes(server, now, peak): the device bytes the
 * server's workspaces hold now and the most they have held (either may be
 * NULL); never above hbm_budget.
 *
 * gmmnlse_server_destroy waits for admitted requests, cancels queued ones
 * and frees the server.
 */
int gmmnlse_server_create(size_t hbm_budget, int max_inflight, gmmnlse_server** out);
int gmmnlse_submit(gmmnlse_server* srv, gmmnlse_ctx* ctx, const double* A0, double L,
                   double dz, int M, double tol, uint64_t* ticket);
int gmmnlse_poll(gmmnlse_server* srv, uint64_t ticket, double* Aout, gmmnlse_stats* st);
int gmmnlse_cancel(gmmnlse_server* srv, uint64_t ticket);
int gmmnlse_server_resident_bytes(gmmnlse_server* srv, size_t* now, size_t* peak);
int gmmnlse_server_destroy(gmmnlse_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* GMMNLSE_H */
