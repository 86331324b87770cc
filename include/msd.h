/*
 * msd.h -- C ABI of the GB300 multiple-scattering-by-disks library (libmsd.so).
 *
 * The library solves the truncated Fourier-Galerkin boundary-integral system
 * for M disks (paper: mu-diff, arXiv 1409.8186, section 5, eq. for
 * L rho = -U and its sound-hard counterpart) on one GPU, with the
 * block-Toeplitz matrix-vector product of section 5 as the hot path.
 * Around it: plane-wave and point-source right-hand sides (Prop. 4.1,
 * section 4.3), the far field (section 4.4) and near field (Prop. 4.3), the
 * adjoint gradient of a far-field misfit, other integral equations as
 * combinations of I, L, M, N, D (sections 3 and 4.2), penetrable obstacles
 * and the time-reversal matrix (section 7).
 *
 * Notation (section 4.1): disk p has centre O_p, radius a_p and a boundary
 * condition flag; every disk of a configuration carries the Fourier modes
 * m = -N..N (n = 2N+1 per disk).  A configuration with M disks has
 * N_tot = M*n unknowns; several configurations may be batched in one
 * problem, their unknowns concatenated in configuration order.
 *
 * Vector layout (all vectors in this ABI): element (row, r) at index
 * row*R + r, row = row_offset(config) + p*n + (m + N), r = right-hand side
 * (incidence angle) index.  Complex numbers are interleaved (re, im):
 * complex128 = two doubles, complex64 = two floats.
 *
 * Pointers.  Arguments named *_host are host memory owned by the caller and
 * only read (or written) during the call.  Arguments documented "host or
 * device" may point to either; the library asks the CUDA runtime which it is
 * and stages host buffers through device memory itself.  Device results are
 * written asynchronously on the problem's stream unless stated otherwise;
 * host results are complete when the call returns.  The caller keeps
 * ownership of every buffer it passes; the library owns its work buffers
 * and frees them in msd_destroy.
 *
 * Errors.  Every call returns an msd_status.  Negative values mean no
 * result was produced; msd_last_error() then describes the failure (per
 * thread).  Positive values (from the solver) mean a result was produced
 * but the stopping test was not met.  Nothing aborts the process and no
 * C++ exception crosses this boundary.  Every device-side wait or loop in
 * the library is bounded.
 */
#ifndef MSD_H
#define MSD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct msd_problem msd_problem;

typedef enum {
    MSD_OK = 0,              /* converged / completed                               */
    MSD_NOT_CONVERGED = 1,   /* iteration limit reached before the tolerance        */
    MSD_STAGNATED = 3,       /* refinement stopped reducing the FP64 residual        */
    /* Matlab's gmres FLAG 2 (section 6.2: the preconditioner is ill-conditioned)
     * has no positive code here.  The single-scattering preconditioner is the
     * block diagonal of self blocks (section 5), which are diagonal in the
     * Fourier modes, so it is singular exactly when one mode's self block
     * vanishes (a sound-hard disk with k a_p at a zero of J_m; a resonance of a
     * formulation's combination).  The library finds that when it forms the
     * per-row factors -- msd_create, msd_update_geometry, msd_set_formulation,
     * msd_set_formulation_kind, msd_set_penetrable -- and returns
     * MSD_ERR_NONFINITE there, before any solve; a solve never returns 2. */
    MSD_ERR_ARG = -1,        /* invalid argument (sizes, null pointers, N range)     */
    MSD_ERR_OVERLAP = -2,    /* two disks of one configuration intersect             */
    MSD_ERR_CUDA = -3,       /* a CUDA runtime call failed                            */
    MSD_ERR_OOM = -4,        /* device allocation failed                              */
    MSD_ERR_NONFINITE = -5,  /* a NaN/Inf appeared in an input or an iterate          */
    MSD_ERR_RANGE = -6       /* a Hankel generator exceeds the complex64 range        */
} msd_status;

enum { MSD_DIRICHLET = 0, MSD_NEUMANN = 1 };          /* sound-soft / sound-hard   */
enum { MSD_FP64 = 0, MSD_MIXED = 1, MSD_FP32 = 2 };   /* arithmetic of a product   */
enum { MSD_GEN_AUTO = 0, MSD_GEN_STREAMED = 1, MSD_GEN_RECOMPUTE = 2 };

/* Largest truncation order accepted (modes -N..N, n <= 111): every product
 * kernel runs it (the FP64 CUDA-core kernel covers at most 16 warps x 7
 * modes per target disk; above N ~ 50 it stages one source at a time).
 * Eq. (Np) of section 5 reaches it at k a ~ 39 for eps = 1e-10. */
#define MSD_MAX_N 55

/* Solver options (section 5 and the restarted GMRES call of section 6.2:
 * RESTART, TOL, MAXIT).  Zero-initialised fields take the defaults in
 * brackets. */
typedef struct {
    double tol;        /* stop when ||P^-1(b - A x)|| / ||P^-1 b|| <= tol   [1e-10]   */
    int restart;       /* GMRES restart length m          [auto: as long as HBM allows] */
    int maxit;         /* limit on Arnoldi steps over the whole solve       [3000]    */
    int max_refine;    /* MSD_MIXED: limit on FP64 refinement sweeps        [60]      */
    double inner_tol;  /* MSD_MIXED: relative tolerance of each FP32 sweep  [5e-6]    */
    int precision;     /* MSD_FP64 (all FP64) or MSD_MIXED                  [FP64]    */
    int gen_mode;      /* MSD_GEN_*: generators stored in HBM or recomputed [auto]    */
    double reorth;     /* second Gram-Schmidt pass when the first leaves less than
                          this fraction of ||w||^2 (in (0, 1]; 1: always)  [0.5]     */
} msd_opts;

/* Per-system statistics (one per configuration and right-hand side). */
typedef struct {
    int flag;          /* MSD_OK, MSD_NOT_CONVERGED or MSD_STAGNATED                    */
    int iters;         /* Arnoldi steps taken by this system (all sweeps)               */
    int refine_steps;  /* FP64 residual evaluations after the first (MSD_MIXED)         */
    int reserved;
    double relres;     /* final FP64 relative residual of the preconditioned system     */
    double true_relres;/* ||b - A rho|| / ||b|| of the unpreconditioned system, from the
                          final residual and the diagonal preconditioner (section 5);
                          -1 for adjoint solves and for R > 64                          */
    double solve_ms;   /* wall time of the whole call (host clock), every system       */
} msd_stats;

/* Create a problem.  Section 4.1 (geometry), section 5 (truncation).
 *   C            number of batched configurations (>= 1)
 *   disk_off     [C+1] host: configuration c owns disks disk_off[c]..disk_off[c+1]-1
 *   centres      [disk_off[C]][2] host: O_p = (x, y)
 *   radii        [disk_off[C]] host: a_p > 0
 *   bc           [disk_off[C]] host: MSD_DIRICHLET or MSD_NEUMANN per disk
 *   k            [C] host: wavenumber per configuration (> 0)
 *   N            [C] host: truncation order per configuration (1..MSD_MAX_N)
 *   cuda_stream  cudaStream_t used for every later call (NULL: legacy stream)
 *   out          receives the problem handle
 * Copies the geometry to the device and evaluates the Bessel diagonals of
 * section 4.2 (kernel K1).  Returns MSD_ERR_OVERLAP if two disks of one
 * configuration intersect. */
msd_status msd_create(int C, const int* disk_off, const double* centres,
                      const double* radii, const int8_t* bc, const double* k,
                      const int* N, void* cuda_stream, msd_problem** out);

void msd_destroy(msd_problem* pb);

/* Total unknowns (sum over configurations of M*n) and the row offset of a
 * configuration; -1 on a bad handle or index. */
int64_t msd_num_unknowns(const msd_problem* pb);
int64_t msd_row_offset(const msd_problem* pb, int config);

/* Section 4.2: the diagonals J^p, J'^p, H^p, H'^p at k a_p for every unknown
 * row, as complex128 [4][N_tot] (J and J' carry zero imaginary parts).
 * out: host or device, caller-allocated. */
msd_status msd_disk_diagonals(msd_problem* pb, void* out);

/* Section 4.2: the Toeplitz generators g^pq_l = H^(1)_l(k b_pq) e^{i l alpha_pq},
 * l = -2N..2N, of configuration `config` (kernel K2), as complex128
 * [q][p][l + 2N] (M*M*(4N+1) values, zeros on p == q).  These are the
 * entries of (S^pq)^T: (S^pq)^T_mn = g^pq_{n-m}.  out: host or device. */
msd_status msd_pair_generators(msd_problem* pb, int config, void* out);

/* Prop. 4.1 and section 5: the preconditioned plane-wave right-hand side
 * P^-1(-U) (Dirichlet rows) or P^-1(-dU) (Neumann rows), complex128
 * [N_tot][R].  betas: [C][R] host incidence angles (kernel K5).
 * out: host or device. */
msd_status msd_rhs_planewave(msd_problem* pb, int R, const double* betas_host, void* out);

/* Section 5 (hot path, kernel K3): y = P^-1 A x, the single-scattering
 * left-preconditioned operator, applied to R columns at once:
 *   y^p_m = x^p_m + l^p_m sum_{q != p} sum_n g^pq_{n-m} r^q_n x^q_n,
 * with r^q_n = sqrt(a_q) J_n(k a_q), l^p_m = 1/(sqrt(a_p) H_m(k a_p))
 * (Dirichlet) or J'_m/(sqrt(a_p) J_m H'_m) (Neumann).
 *   precision  MSD_FP64: x, y complex128; MSD_FP32: complex64 with FP32
 *              accumulation (the inner product of MSD_MIXED solves)
 *   x, y       device, [N_tot][R]; byte ranges that overlap in any way are
 *              rejected with MSD_ERR_ARG
 * Asynchronous on the problem's stream. */
msd_status msd_matvec(msd_problem* pb, int R, int precision, const void* x_dev, void* y_dev);

/* The same product as msd_matvec, for callers that must not allocate device
 * memory at the time of the call: a serving process that reserves its whole
 * device-memory budget at start-up, or a latency-critical caller for which
 * the implicit device-wide synchronisation of cudaMalloc/cudaFree is not
 * acceptable.  The paper has no counterpart; it is a property of this
 * library's memory management only.
 *   pb         a problem whose generators of this precision already exist
 *              (after one msd_matvec or msd_solve_planewaves call with that
 *              precision; otherwise MSD_ERR_ARG)
 *   x, y       device, [N_tot][R], as for msd_matvec; byte ranges that
 *              overlap in any way are rejected with MSD_ERR_ARG
 * The tile shape is the cost model's choice for (R, precision), not the
 * autotuned one (tuning would need timing buffers and a synchronisation).
 * The call allocates nothing: its work list, scaled input and per-split
 * partial sums live in one 32 MiB device array that the library declares
 * at file scope (every GPU that loads the library holds it until the
 * process exits).  A problem whose 2 * N_tot * R values (complex128 or
 * complex64) plus work list exceed 32 MiB is rejected with MSD_ERR_ARG.
 * The first call on a device looks up the device address of that array
 * (cudaGetSymbolAddress), so that first call should come before any stream
 * capture.  Every call shares the array and overwrites what it reads before
 * reading it; calls whose execution overlaps on the GPU (other streams,
 * other problems) race on it and must be serialised by the caller.
 * Asynchronous on the problem's stream. */
msd_status msd_matvec_noalloc(msd_problem* pb, int R, int precision, const void* x_dev, void* y_dev);

/* Section 5 / section 6.2: solve A rho = -U for R plane waves per
 * configuration with left-preconditioned restarted GMRES on the device
 * (x0 = 0), FP64 throughout (MSD_FP64) or FP32 inner sweeps with FP64
 * residuals and corrections (MSD_MIXED).  A mixed sweep stops when its
 * residual estimate falls below inner_tol times its starting FP64 residual,
 * but not below opts->tol (relative), or below half of it when the sweep
 * started within twice the tolerance; systems that have converged drop out
 * of the remaining products and projections of the batch.
 *   betas_host  [C][R] incidence angles
 *   opts        may be NULL (defaults)
 *   rho_out     host or device, complex128 [N_tot][R]: the density
 *               coefficients rho^p_m (identical for A and P^-1 A)
 *   stats_host  may be NULL, else [C*R] (system index c*R + r)
 * Synchronises the stream.  Returns MSD_OK when every system met opts->tol,
 * MSD_NOT_CONVERGED / MSD_STAGNATED otherwise (rho_out still written). */
msd_status msd_solve_planewaves(msd_problem* pb, int R, const double* betas_host,
                                const msd_opts* opts, void* rho_out, msd_stats* stats_host);

/* Section 4.4: far field a_L(theta_t) = (a_L(theta_t))^T rho for every
 * configuration, sample angle and column (kernel K6).
 *   rho     host or device, complex128 [N_tot][R]
 *   thetas  [T] host sample angles (shared by all configurations)
 *   F_out   host or device, complex128 [C][T][R] */
msd_status msd_farfield(msd_problem* pb, const void* rho, int R, int T,
                        const double* thetas_host, void* F_out);

/* Far-field misfit and its gradient (adjoint method).  The misfit is
 *   J_c = sum_{t, r} |F_c(theta_t; beta_r) - Ftarget_c[t][r]|^2
 * per configuration c, with F the far field a_L of section 4.4 for the plane
 * waves of Prop. 4.1 (densities from the section 5 system).  The gradient is
 * taken with respect to every disk centre, every radius and each k, through
 * one forward solve, one adjoint solve with (P^-1 A)^H, the raw Toeplitz sums
 * of both, a per-pair correlation contracted with the derivatives of the
 * separation generators, and per-row terms (kernel K7).  The paper itself
 * computes fields only; the misfit is this library's differentiation target.
 *   betas_host   [C][R] incidence angles
 *   thetas_host  [T] far-field sample angles
 *   F_target     host or device, complex128 [C][T][R]
 *   opts         solver options for both solves (default tol 1e-12; NULL ok)
 *   J_out        host or device [C] (may be NULL)
 *   dO           host or device [disk_off[C]][2] dJ/dO_p (may be NULL)
 *   da           host or device [disk_off[C]] dJ/da_p (may be NULL)
 *   dk           host or device [C] dJ/dk_c (may be NULL)
 * Returns MSD_NOT_CONVERGED / MSD_STAGNATED (no gradient written) when a
 * solve misses its tolerance.  Synchronises the stream. */
msd_status msd_grad_farfield_misfit(msd_problem* pb, int R, const double* betas_host, int T,
                                    const double* thetas_host, const void* F_target, const msd_opts* opts,
                                    double* J_out, double* dO, double* da, double* dk);

/* Replace the geometry of every configuration (same disk counts, N and
 * boundary flags) and recompute the Bessel diagonals (K1) and any stored
 * Toeplitz generators (K2).  Any argument may be NULL to keep it.
 *   centres  host or device, [disk_off[C]][2]
 *   radii    host or device, [disk_off[C]]
 *   k_host   host, [C]
 * The disks are not re-checked for overlap.  Synchronises the stream. */
msd_status msd_update_geometry(msd_problem* pb, const double* centres, const double* radii,
                               const double* k_host);

/* Kernel timing of the block-Toeplitz product.  enable = 1 starts recording
 * a CUDA event pair around every K3 kernel launched on the problem's
 * stream (the column scaling and the split reduction around it are
 * excluded), enable = 0 stops, enable = -1 only reads.  On return the
 * totals since the last start: summed kernel time in ms, number of
 * launches, algorithmic flops (8 per complex multiply-add of the
 * off-diagonal blocks) and algorithmic bytes (generators of every ordered
 * pair plus x and y) of those launches.  Any output may be NULL.
 * Synchronises on the recorded events. */
msd_status msd_matvec_timing(msd_problem* pb, int enable, double* kernel_ms, int64_t* launches,
                             double* flops, double* bytes);

/* Point sources (section 4.3, point-source proposition): the incident wave
 * is the Green's function u_inc(x) = (i/4) H_0(k |x - s|) of a source s
 * outside every disk; its trace coefficients are U^p_m = d'^p_m J_m(k a_p)
 * (Dirichlet rows; k d'^p_m J_m'(k a_p) on Neumann rows) with
 * d'^p_m = (i/4) sqrt(2 pi a_p) H_m(k b) e^{-i m phi}, (b, phi) the polar
 * coordinates of s - O_p (kernel K5').
 *   sources  [C][R][2] host: source (x, y) of column r of configuration c
 * msd_rhs_pointsource: out (host or device, complex128 [N_tot][R]) = P^-1(-U),
 *   the preconditioned right-hand side, as msd_rhs_planewave.
 * msd_solve_pointsources: as msd_solve_planewaves with these right-hand sides.
 * A source on or inside a disk gives non-finite coefficients
 * (MSD_ERR_NONFINITE from the solve). */
msd_status msd_rhs_pointsource(msd_problem* pb, int R, const double* sources, void* out);
msd_status msd_solve_pointsources(msd_problem* pb, int R, const double* sources, const msd_opts* opts,
                                  void* rho_out, msd_stats* stats_host);

/* Prop. 4.3: the scattered field at points x outside the disks,
 *   u(x)[r] = sum_p sum_m rho^p_m[r] (i pi a_p / 2) J_m(k a_p) H_m(k r_p)
 *             e^{i m theta_p} / sqrt(2 pi a_p),
 * (r_p, theta_p) the polar coordinates of x - O_p, for configuration
 * `config` of the problem (kernel K8).
 *   rho     host or device, complex128 [N_tot][R] (all configurations)
 *   P       number of points
 *   points  host or device, double [P][2] (x, y)
 *   u_out   host or device, complex128 [P][R]
 * Points inside a disk of the configuration get 0 (the expansion holds
 * outside the disks only).  Far point-disk pairs (k r_p > 20 and N <= k r_p)
 * evaluate the Hankel functions in FP32 after an FP64 phase (relative error
 * ~1e-6 of the field); near pairs in FP64.  Synchronises the stream when
 * u_out is host memory. */
msd_status msd_nearfield(msd_problem* pb, int config, const void* rho, int R, int64_t P, const double* points,
                         void* u_out);

/* Penetrable obstacles (section 7, Example II, the transmission problem):
 * the wavenumber is k+ (the problem's k) outside the disks and k- inside,
 * and u+ = L+ rho+ outside, u- = L- rho- inside (single layers at k+ and
 * k-).  The unknowns (rho+, rho-) solve
 *   L+ rho+ - L- rho- = -U,
 *   (-I/2 + N+) rho+ - mu (I/2 + N-) rho- = -dU,
 * i.e. u+ + u_inc = u- and d_n(u+ + u_inc) = mu d_n u- on every circle
 * (mu per disk: the section 7 contrast of the normal derivatives).  The
 * (2, 2) block carries the minus sign of the interior jump relation of
 * Prop. 3.2 (printed without it).  Every row is preconditioned by the
 * 2 x 2 self block of its mode, and a product runs the block-Toeplitz
 * kernel once with the generators at k+ and once at k-.
 * msd_set_penetrable:
 *   k_minus  host [C] interior wavenumbers (> 0), NULL switches the mode off
 *   mu       host [disk_off[C]] contrasts (> 0), NULL for all 1
 *   needs the default formulation; MSD_ERR_NONFINITE when a 2 x 2 self
 *   block is singular.  Keeps internal problems for the interior
 *   wavenumber and the solver layout until switched off or destroyed.
 * msd_penetrable_matvec: (y+, y-) = B^-1 A (x+, x-), B the 2 x 2 self
 *   blocks; x+-, y+- device complex128 [N_tot][R]; MSD_FP64 only.
 * msd_solve_penetrable: plane waves (Prop. 4.1, at k+) betas_host [C][R];
 *   rho_plus, rho_minus host or device complex128 [N_tot][R]; options and
 *   statistics as msd_solve_planewaves (true_relres not computed, -1).
 *   The exterior scattered field of the solution is msd_farfield /
 *   msd_nearfield of rho_plus.
 * msd_solve_penetrable_pointsources: the same with the point-source
 *   incident waves (i/4) H_0(k+ |x - s|) of section 4.3, sources [C][R][2]
 *   host (outside every disk). */
msd_status msd_set_penetrable(msd_problem* pb, const double* k_minus, const double* mu);
msd_status msd_penetrable_matvec(msd_problem* pb, int R, int precision, const void* xp, const void* xm, void* yp,
                                 void* ym);
msd_status msd_solve_penetrable(msd_problem* pb, int R, const double* betas_host, const msd_opts* opts,
                                void* rho_plus, void* rho_minus, msd_stats* stats_host);
msd_status msd_solve_penetrable_pointsources(msd_problem* pb, int R, const double* sources, const msd_opts* opts,
                                             void* rho_plus, void* rho_minus, msd_stats* stats_host);

/* The interior field of penetrable obstacles (section 7, Example II):
 * u-(x) = L- rho- (x) for points x inside a disk of configuration `config`,
 * the single layers of every circle at the interior wavenumber k-; for x
 * inside disk p the circle of p takes its interior expansion
 * (i pi a_p/2) H_m(k- a_p) J_m(k- r_p) e^{i m theta_p} rho-^p_m / sqrt(2 pi a_p),
 * the other circles their exterior one with H_m(k- r_q) (Prop. 4.3 at k-).
 * With u+ from msd_nearfield(rho_plus) and the incident wave, this gives the
 * total field everywhere (u+ + u_inc outside, u- inside).
 *   rho_minus  host or device, complex128 [N_tot][R] (msd_solve_penetrable)
 *   points     host or device, double [P][2]
 *   u_out      host or device, complex128 [P][R]; 0 at points outside every disk
 * Needs msd_set_penetrable.  FP64.  Synchronises the stream when u_out is
 * host memory. */
msd_status msd_penetrable_interior_field(msd_problem* pb, int config, const void* rho_minus, int R, int64_t P,
                                         const double* points, void* u_out);

/* Integral-equation formulation (sections 3, 4.2, 5): replaces the default
 * rows (EFIE L rho = -U on sound-soft disks, (-I/2 + N) rho = -dU on
 * sound-hard ones, u = L rho) by linear combinations of the identity and
 * the four boundary integral operators of section 4.2,
 *   rows of disks with boundary condition c:
 *     (w_I I + w_L L + w_M M + w_N N + w_D D) dens = -(w_U U + w_dU dU),
 *   fields (far field section 4.4, near field Prop. 4.3):
 *     u = w_L' L dens + w_M' M dens,
 * for every configuration of the problem.  Examples (Dirichlet rows):
 * CFIE  w_L = alpha eta, w_I = (1 - alpha)/2, w_N = 1 - alpha,
 *       w_U = alpha eta, w_dU = 1 - alpha, u = L dens;
 * Brakhage-Werner  w_I = 1/2, w_L = -eta, w_M = -1, w_U = 1,
 *       u = -(eta L + M) dens.
 * The off-diagonal blocks of M, N, D use the same generators g^pq as L
 * with J' in place of J on the source side (M, D) and/or the target side
 * (N, D); the D diagonal is -(i pi k^2 a/2) J' H' (the normal derivative of
 * the double-layer potential of Prop. 4.3; printed with the opposite sign)
 * and the double-layer far field carries -i e^{-i pi/4} sqrt(k a)/2.
 * Every solve, product, right-hand side, far field, near field and time-
 * reversal call then uses the formulation, preconditioned by its own
 * diagonal self blocks; products always use stored generators.
 *   op_weights   double [2][5][2]: per boundary condition (MSD_DIRICHLET,
 *                MSD_NEUMANN) the complex weights (re, im) of I, L, M, N, D;
 *                NULL restores the default rows
 *   rhs_weights  double [2][2][2]: per boundary condition the weights of U, dU
 *   rep_weights  double [2][2]: the weights of L and M in the representation
 * Returns MSD_ERR_NONFINITE when the self block of the combination vanishes
 * for some mode (a resonance of that formulation at k a_p; the EFIE at a
 * zero of J_m, for instance), and the formulation is left set.  The
 * gradient (msd_grad_farfield_misfit) and msd_matvec_noalloc need the
 * default rows (MSD_ERR_ARG otherwise).  Synchronises the stream. */
msd_status msd_set_formulation(msd_problem* pb, const double* op_weights, const double* rhs_weights,
                               const double* rep_weights);

/* The named formulations of section 3, with their weights formed by the
 * library (for every configuration of the problem):
 *   MSD_FORM_EFIE  sound-soft rows L rho = -U
 *   MSD_FORM_MFIE  sound-soft rows (I/2 + N) rho = -dU
 *   MSD_FORM_CFIE  sound-soft rows [alpha eta L + (1 - alpha)(I/2 + N)] rho
 *                  = -(alpha eta U + (1 - alpha) dU)   (section 5 CFIE system)
 *   (these three: sound-hard rows (-I/2 + N) rho = -dU, field u = L rho)
 *   MSD_FORM_BWIE  Brakhage-Werner, u = -(eta L + M) psi: sound-soft rows
 *                  (I/2 - eta L - M) psi = -U, sound-hard rows the normal
 *                  trace (eta I/2 - eta N - D) psi = -dU
 * msd_set_formulation_kind:
 *   alpha  CFIE weight, 0 <= alpha <= 1 (ignored by the other kinds)
 *   eta    NULL: eta = i k of each configuration; else host double[2]
 *          (re, im) for every configuration.  CFIE and Brakhage-Werner need
 *          Im(eta) != 0 (section 3), else MSD_ERR_ARG.
 *   Otherwise as msd_set_formulation (MSD_ERR_NONFINITE at a resonance of
 *   the combination; synchronises the stream).
 * msd_formulation_weights: the same weights in the layout of
 *   msd_set_formulation, for inspection or editing; needs no problem and no
 *   GPU.  eta NULL means i k (k > 0 then needed for CFIE and BWIE).  Any
 *   output may be NULL. */
enum { MSD_FORM_EFIE = 0, MSD_FORM_MFIE = 1, MSD_FORM_CFIE = 2, MSD_FORM_BWIE = 3 };
msd_status msd_set_formulation_kind(msd_problem* pb, int kind, double alpha, const double* eta);
msd_status msd_formulation_weights(int kind, double alpha, const double* eta, double k, double* op_weights,
                                   double* rhs_weights, double* rep_weights);

/* Time reversal, DORT (section 7, far-field mirror): for every
 * configuration the mirror emits the plane waves of incidence
 * alpha_j = 2 pi j / n_alpha (j = 0..n_alpha-1) and measures the far field
 * a_L of section 4.4 in the opposite directions alpha_i + pi.  With
 *   F[i][j] = a_L(alpha_i + pi; alpha_j)   (densities from one batched solve
 *             of the section 5 system with n_alpha right-hand sides)
 * the time-reversal matrix is T = conj(F)^T F (Hermitian, positive
 * semi-definite) and eig holds its eigenvalues, largest first (Householder
 * tridiagonalisation and Sturm bisection on the device, absolute error a
 * small multiple of 1e-16 ||T||).  No quadrature weight h_alpha is applied.
 *   n_alpha  1..MSD_MAX_DORT mirror angles
 *   opts     solver options of the batched solve (NULL: defaults)
 *   F_out    NULL or host/device complex128 [C][n_alpha][n_alpha]
 *   T_out    NULL or host/device complex128 [C][n_alpha][n_alpha]
 *   eig_out  host or device double [C][n_alpha]
 *   stats_host  NULL or [C*n_alpha] (system c*n_alpha + j)
 * Returns the status of the solve (MSD_NOT_CONVERGED / MSD_STAGNATED still
 * write every output).  Synchronises the stream. */
#define MSD_MAX_DORT 2048
msd_status msd_dort(msd_problem* pb, int n_alpha, const msd_opts* opts, void* F_out, void* T_out, void* eig_out,
                    msd_stats* stats_host);

/* The second half of msd_dort for far-field matrices the caller supplies
 * (computed elsewhere or measured by a mirror): T = conj(F)^T F and its
 * eigenvalues, largest first, for each of the problem's C configurations
 * (only the problem's stream and work buffers are used).
 *   F        host or device complex128 [C][n_alpha][n_alpha], row i the
 *            receiving direction, column j the emitting one
 *   T_out    NULL or host/device complex128 [C][n_alpha][n_alpha]
 *   eig_out  host or device double [C][n_alpha]
 * Synchronises the stream. */
msd_status msd_dort_eigen(msd_problem* pb, int n_alpha, const void* F, void* T_out, void* eig_out);

/* Eigenvectors of the time-reversal matrix (section 7: the eigenvectors of
 * T = conj(F)^T F for its significant eigenvalues are the mirror signals
 * that focus on one obstacle each, see msd_herglotz_wave): for each of the
 * problem's C configurations, T and its eigenvalues as msd_dort_eigen, then
 * the eigenvectors of the K largest eigenvalues: inverse iteration on the
 * real tridiagonal form of T (orthogonalised within clusters of eigenvalues
 * closer than 1e-3 of the norm bound), mapped back through the phase
 * similarity and the Householder reflections of the reduction.
 *   F        host or device complex128 [C][n_alpha][n_alpha]
 *   K        1..n_alpha eigenvectors (largest eigenvalues first)
 *   eig_out  NULL or host/device double [C][n_alpha]
 *   vec_out  host or device complex128 [C][K][n_alpha]: unit 2-norm, the
 *            entry of largest modulus real and positive (an eigenvector is
 *            fixed up to a phase; vectors of a multiple eigenvalue span its
 *            eigenspace)
 * Synchronises the stream. */
msd_status msd_dort_eigenvectors(msd_problem* pb, int n_alpha, const void* F, int K, void* eig_out, void* vec_out);

/* The discrete Herglotz wave of section 7 emitted by the mirror of n_alpha
 * transducers at the angles alpha_j = 2 pi j / n_alpha, for K parameter
 * vectors g (for instance eigenvectors of the time-reversal matrix), at
 * the wavenumber k of configuration `config`:
 *   u[p][r] = (2 pi / n_alpha) sum_j g[r][j] exp(i k (x_p cos alpha_j + y_p sin alpha_j)).
 *   g       host or device complex128 [K][n_alpha]
 *   points  host or device double [P][2]
 *   u_out   host or device complex128 [P][K]
 * FP64.  Synchronises the stream when u_out is host memory. */
msd_status msd_herglotz_wave(msd_problem* pb, int config, int n_alpha, int K, const void* g, int64_t P,
                             const double* points, void* u_out);

/* Per-disk truncation orders (section 5: disk p keeps the modes
 * -N_p..N_p, the blocks of the truncated system are (2N_p+1) x (2N_q+1);
 * eq. (Np) gives N_p from k a_p).  Vectors keep the layout [N_tot][R] of the
 * configurations' N: the rows of modes |m| > N_p of disk p become an
 * identity block with a zero right-hand side that no product couples to the
 * other rows, so every solve leaves them zero (GMRES from x0 = 0) and their
 * densities add nothing to a far or near field.  On the other rows the
 * solution is that of the system truncated at N_p on every disk; a product
 * returns y = x on the dropped rows.  The kernels still run the padded
 * blocks; msd_matvec_timing counts the flops and bytes of the truncated
 * blocks.
 *   Np  host int [disk_off[C]], 0 <= Np[d] <= N of the disk's configuration;
 *       NULL restores N on every disk
 * Needs the default rows: MSD_ERR_ARG with a formulation or penetrable
 * obstacles (and msd_set_formulation, msd_set_formulation_kind,
 * msd_set_penetrable and msd_grad_farfield_misfit refuse while orders are
 * set).  Synchronises the stream. */
msd_status msd_set_truncation(msd_problem* pb, const int* Np);

/* Generators of the forward products (the Toeplitz storage of section 5).
 *   MSD_GEN_STREAMED (default): the 4N+1 values of every ordered pair are
 *     stored in HBM (complex128, plus complex64 for FP32 products) and read
 *     by every product.
 *   MSD_GEN_RECOMPUTE: no stored array; every product evaluates the
 *     generators again (kernel K2), chunk by chunk, into a work buffer of
 *     about chunk_bytes (0: 64 MiB, sized to stay in L2) that the product
 *     kernel reads at once.  The stored arrays are freed.
 *   MSD_GEN_AUTO: streamed if both stored copies fit in half the free
 *     device memory, else recompute (decided now).
 * Applies to msd_matvec and to msd_solve_planewaves (whose opts.gen_mode,
 * when not MSD_GEN_AUTO, overrides it for that solve).  The gradient and
 * msd_pair_generators always use (and build) the stored arrays.  A complex64
 * range overflow of a generator (MSD_ERR_RANGE) is checked once per
 * geometry on the first recomputed FP32 product.  Synchronises the stream. */
msd_status msd_set_generator_mode(msd_problem* pb, int mode, int64_t chunk_bytes);

/* Tile shape of the block-Toeplitz product kernel (an implementation
 * choice; the paper fixes none).  The kernel gives each thread a register
 * window of KB consecutive modes and each CTA a tile of 32 target disks by
 * RT columns; the sources of a tile are split into nsplit ranges.  On the
 * first product of a given (R, precision) the library times every shape
 * that fits (autotuner; the first product therefore synchronises the
 * stream, so make it before any stream capture) unless the environment sets
 * MSD_AUTOTUNE=0 (cost-model choice) or msd_set_tile fixed one.
 *
 * msd_plan_info: the shape used for (R, precision), precision MSD_FP64 or
 *   MSD_FP32, creating the plan (and tuning) if needed.  out[4] receives
 *   {KB (encoded as for msd_set_tile), RT, nsplit, number of shapes timed
 *   (0: not tuned)}; tuned_ms (may
 *   be NULL) the kernel time of the chosen shape in the tuning run (0 if
 *   not tuned).  Needs the generators of that precision (builds them).
 * msd_set_tile: fix the shape (KB, RT) for later products of (R, precision)
 *   of this problem, replacing any plan made before.  MSD_ERR_ARG if
 *   (KB, RT) is not one of the instantiated shapes that fit (FP64: KB 4..7,
 *   RT 1; FP32: KB 4..9, RT in {1,2,4,8,16} dividing R, at most 16 warps
 *   per CTA, shared memory <= 226 KB; FP32 KB + 100 selects the same window
 *   with each complex multiply-add issued as two paired FP32 FMAs, and with
 *   RT = 1, KB + 200 / KB + 300 the same windows in a kernel without CTA
 *   barriers in its source loop (stages released per warp, source values
 *   read from global memory); KB = 0,
 *   RT in {16, 32, 64} dividing R: the tensor-core kernel that expands the
 *   Toeplitz blocks in shared memory; RT = 8 with KB = 0 or 1, R a multiple
 *   of 8: the shift-GEMM tensor-core kernel, one dense GEMM over the source
 *   disks per shift d = n - m, with mode blocks of <= 8 two per CTA (KB = 0)
 *   or one block of <= 16 modes per CTA (KB = 1); it serves the forward
 *   products of the default rows with stored generators, every other product
 *   of a problem pinned to it takes the cost-model shape).  KB reported by
 *   msd_plan_info uses the same encoding. */
msd_status msd_plan_info(msd_problem* pb, int R, int precision, int* out, double* tuned_ms);
msd_status msd_set_tile(msd_problem* pb, int R, int precision, int KB, int RT);

/* Test hook for the error path of the bounded device waits (no GPU fault
 * is involved).  While on != 0 (process-wide; off by default), every launch
 * of a kernel with such a wait -- the tensor-core product's pipeline and the
 * time-reversal grid barrier -- waits once, with a limit of about 10 us,
 * for a condition that nothing fulfils: the kernel records the expiry, lets
 * its own MMAs finish (the tensor-core kernel waits for them as usual),
 * frees its TMEM, writes no result and returns.  The call that synchronises
 * on that work then returns MSD_ERR_CUDA (solves and msd_matvec_timing for
 * products, msd_dort / msd_dort_eigen for the barrier); an msd_matvec alone
 * is asynchronous and leaves the report to the next such call.  With the
 * hook off again the next call works normally. */
void msd_test_expire_waits(int on);

/* Total number of CUDA kernels launched by this library in this process. */
int64_t msd_kernel_launches(void);

/* Description of the last failure on the calling thread ("" if none). */
const char* msd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MSD_H */
