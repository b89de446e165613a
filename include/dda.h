/*
 * dda.h -- C ABI of the GB300 discrete-dipole-approximation (DDA) solver.
 *
 * The library solves A P = E (the DDSCAT 7.3 guide, Sec. "Choice of Iterative
 * Algorithm", eq. AP=E) for N polarizable points on a cubic lattice: E is the
 * incident field at the occupied sites, P the unknown dipole moments and A the
 * 3N x 3N interaction matrix, (A P)_j = alpha_j^{-1} P_j - sum_{l != j}
 * G(r_j - r_l) P_l.  The product A.P is evaluated as a zero-padded 3-D FFT
 * convolution of the three polarization components with the six unique
 * components of the lattice Green tensor (Sec. "Choice of FFT Algorithm"), on
 * the GPU, and the system is solved by BiCGSTAB (the PIM method behind the
 * guide's PBCGST option).
 *
 * Conventions (all calls):
 *  - Lattice units: d = 1; "kd" is k d with k the wavenumber in the ambient
 *    medium; refractive indices m are relative to the ambient medium (Sec.
 *    "Application to Targets in Dielectric Media").
 *  - A target box is nx * ny * nz sites; site (ix, iy, iz) has flat index
 *    ix + nx*(iy + ny*iz) and sits at r = (ix - (nx-1)/2, iy - (ny-1)/2,
 *    iz - (nz-1)/2) (origin at the box centre).  Vectors over the N occupied
 *    sites are stored in flat-index order.
 *  - Complex numbers are two consecutive doubles (re, im).
 *  - Every pointer argument is a HOST pointer unless stated; the library copies
 *    what it needs and never keeps a caller's pointer after the call returns.
 *  - No call throws; each returns a dda_status.  dda_last_error() gives a
 *    human-readable detail for the calling thread's last failing call.
 *  - One dda_target must not be used from two threads at once; distinct
 *    targets may be used concurrently (each call runs on its own stream).
 *  - Without a usable CUDA device every compute call returns DDA_ERR_CUDA;
 *    there is no CPU fallback.
 */
#ifndef DDA_H
#define DDA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DDA_OK = 0,
  DDA_ERR_INVALID_ARG = 1, /* a size, pointer or option is out of range        */
  DDA_ERR_OOM = 2,         /* device allocation failed (nothing is leaked)     */
  DDA_ERR_CUDA = 3,        /* CUDA error, or no device                         */
  DDA_ERR_NOCONV = 4,      /* max_iter reached; outputs hold the last iterate  */
  DDA_ERR_BREAKDOWN = 5,   /* Krylov breakdown (rho, omega or sigma = 0, NaN)  */
  DDA_ERR_TIMEOUT = 6      /* a bounded device wait ran out                    */
} dda_status;

/* Polarizability prescriptions (Sec. "Choice of DDA Method").
 *  CM : Clausius-Mossotti alpha_CM = 3/(4 pi) (m^2-1)/(m^2+2) with the
 *       radiative-reaction correction alpha = alpha_CM / (1 - (2/3) i (kd)^3 alpha_CM).
 *  LDR: LATTDR, alpha = alpha_CM / {1 + alpha_CM [(b1 + m^2 b2 + m^2 b3 S)(kd)^2
 *       - (2/3) i (kd)^3]}, S = sum_j (khat_j e_j)^2, with the Draine & Goodman
 *       (1993) coefficients; depends on each incident direction and polarization.
 *  FCD: FLTRCD, alpha = alpha_CM / {1 - alpha_CM [(4/3)(kd)^2 + (2/(3 pi))
 *       ln((pi-kd)/(pi+kd)) (kd)^3 + (2/3) i (kd)^3]} (Sec. "Filtered Coupled
 *       Dipole", read with the sign and (kd)^3 factor that make a lossless
 *       material absorb nothing), and the interaction tensor is the filtered one,
 *       (k^2 + grad grad) of the outgoing Green function with spatial
 *       frequencies above pi/d removed.
 *  GKDLDR: the lattice dispersion relation as corrected by Gutkowicz-Krusin &
 *       Draine (2004), the guide's recommended option (Sec. "Point Dipoles:
 *       Options LATTDR and GKDLDR"): a polarizability TENSOR, diagonal on the
 *       lattice axes, alpha_a = alpha_CM / {1 + alpha_CM [(b1 + m^2 b2 +
 *       m^2 b3 khat_a^2)(kd)^2 - (2/3) i (kd)^3]} for a = x, y, z, with LATTDR's
 *       coefficients; it depends on each incident direction, not on the
 *       polarization, and makes the infinite lattice carry a wave of index m
 *       for both transverse polarizations.
 *  CM, LDR and GKDLDR use the point-dipole tensor
 *       G(r) P = e^{ikr}/r^3 {k^2 r^2 (rhat x P) x rhat + (1-ikr)[3 rhat(rhat.P) - P]}. */
typedef enum {
  DDA_POL_CM = 0,
  DDA_POL_LDR = 1,
  DDA_POL_FCD = 2,
  DDA_POL_GKDLDR = 3
} dda_pol_method;

/* Arithmetic of the solve.
 *  FP64        : every step in FP64.
 *  FP32        : FFT convolution and Krylov vectors in complex FP32, inner
 *                products and norms accumulated in FP64; the reported residual
 *                is still the FP64 true residual of the result.
 *  FP32_REFINED: FP64 iterative refinement around FP32 inner BiCGSTAB solves:
 *                r = E - A P in FP64, solve A d = r in FP32 to inner_tol,
 *                P += d in FP64, until ||E - A P|| / ||E|| <= tol (the guide's
 *                single/double precision discussion, Sec. "Single vs. Double
 *                Precision", motivates keeping the accuracy-critical parts in FP64). */
typedef enum {
  DDA_PREC_FP64 = 0,
  DDA_PREC_FP32 = 1,
  DDA_PREC_FP32_REFINED = 2,
  DDA_PREC_DF64 = 3      /* dda_matvec only: FP64 vectors, FFT passes in double-float
                            arithmetic (the refinement's residual operator)        */
} dda_precision;

/* Krylov method of the solve (the guide's CMETHD choice, Sec. "Choice of
 * Iterative Algorithm").
 *  BICGSTAB : BiCGSTAB (van der Vorst 1992), the guide's PBCGST: two matvecs
 *             per iteration; stops on the recursive residual.
 *  QMR      : quasi-minimal residual for complex-symmetric A (Freund 1992),
 *             the guide's QMRCCG: one matvec per iteration on the bilinear
 *             form x^T y (A = A^T for the DDA matrix); stops when the bound
 *             tau_k sqrt(k+1) >= ||E - A P_k|| reaches tol ||E||.  Where
 *             r^T r vanishes (|r^T r| <= 1e-10 ||r||^2 in FP64, 1e-5 in FP32;
 *             e.g. circularly polarized light, E . E = 0) it cannot go on; those
 *             right-hand sides are finished by BiCGSTAB from QMR's iterate.
 *  BICGSTAB2: BiCGstab(2) (Sleijpen & van der Vorst 1993), the guide's PBCGS2
 *             and its recommended method: four matvecs per cycle with a
 *             two-dimensional minimal-residual step; a cycle counts as two
 *             iterations; stops on the recursive residual checked after each
 *             cycle (breakdowns finish with BiCGSTAB as for QMR).
 *  GPBICG   : GPBi-CG (Zhang 1997), the guide's GPBICG: two matvecs per
 *             iteration; each iteration minimises the residual over a
 *             two-parameter (zeta, eta) update (eta = 0 gives BiCGSTAB); stops
 *             on the recursive residual (breakdowns finish with BiCGSTAB).
 *  PETRKP   : conjugate gradients on the normal equations A^H A P = A^H E
 *             (Petravic & Kuo-Petravic 1979), the guide's PETRKP: two matvecs
 *             per iteration (A p and A^H r = conj(A conj(r)), since A = A^T);
 *             slow but monotone in ||E - A P||, on which it stops.
 * Every method's reported residual is the FP64 true residual of the result. */
typedef enum {
  DDA_SOLVER_BICGSTAB = 0,
  DDA_SOLVER_QMR = 1,
  DDA_SOLVER_BICGSTAB2 = 2,
  DDA_SOLVER_GPBICG = 3,
  DDA_SOLVER_PETRKP = 4
} dda_solver;

typedef struct dda_target dda_target; /* opaque, library-owned */

/* Create a target from an occupancy grid.
 *  occ : nx*ny*nz bytes, nonzero = occupied site.
 *  comp: nx*ny*nz bytes, composition 1..ncomp at occupied sites (ignored
 *        elsewhere); NULL means composition 1 everywhere.
 *  m   : ncomp complex refractive indices (interleaved re, im), relative to the
 *        ambient medium (Sec. "Target Geometry: The Target Frame": a target is the list of
 *        occupied sites with their composition).
 *  out : receives the new target; freed with dda_target_destroy.
 * Limits: 1 <= nx, ny, nz <= 4096, 1 <= ncomp <= 255, at least one occupied
 * site.  Device memory for the target (composition grid, site list) is
 * allocated here; the Green-tensor transform is built on the first solve or
 * matvec for a given (kd, method) and kept until the next different one. */
dda_status dda_target_create(int nx, int ny, int nz, const uint8_t* occ,
                             const uint8_t* comp, int ncomp, const double* m,
                             dda_target** out);

/* Select the polarizability prescription used by later solves (default LDR). */
dda_status dda_set_polarizability(dda_target* t, dda_pol_method method);

/* y = A x for one incident wave (the hot loop's operator, eq. AP=E).
 *  kd        : k d (> 0, < pi for FCD).
 *  khat, e   : incident direction [3] and polarization [3][2] (LDR reads both,
 *              GKDLDR khat only; may be NULL otherwise).
 *  x, y      : [N][3][2] on the occupied sites in flat-index order (host).
 *  precision : DDA_PREC_FP64, DDA_PREC_DF64 (FP64 vectors, double-float FFT
 *              passes) or DDA_PREC_FP32 (FP32_REFINED acts as FP32). */
dda_status dda_matvec(dda_target* t, double kd, const double* khat, const double* e,
                      const double* x, double* y, dda_precision precision);

/* y = A x like dda_matvec, for callers that cannot allocate device memory.
 * The paper has no counterpart: this is an integration variant of the same
 * FFT-convolution matvec.  Some callers must not call cudaMalloc/cudaFree at
 * this point: code that runs under another framework's memory manager which
 * owns the device heap, latency-critical serving loops (cudaFree synchronizes
 * the whole device and stalls every stream), and real-time loops that forbid
 * allocation after start-up.  This entry point allocates nothing; its FFT
 * scratch and alpha^{-1} table live in one fixed 64 MiB file-scope device array
 * of the library, which every GPU that loads the library holds until exit.
 *  x_dev, y_dev : DEVICE pointers, caller-allocated, box layout [3][nz][ny][nx]
 *                 complex (float2 for DDA_PREC_FP32, double2 for DDA_PREC_FP64),
 *                 x zero on vacant sites; y must not alias x.  y is written on
 *                 every box site (0 on vacant ones).
 *  kd, khat, e  : as dda_matvec.  The Green-tensor transform for (kd, current
 *                 method) must already exist on the target (a previous
 *                 dda_matvec or dda_solve with the same kd builds it, which does
 *                 allocate); otherwise DDA_ERR_INVALID_ARG.
 *  cuda_stream  : cudaStream_t to run on, or NULL for the target's own stream;
 *                 the call returns after the work on that stream has finished.
 * Limit: 3*nz*Ly*Lx complex values of the chosen precision must fit in 64 MiB
 * minus 12 KiB (with L = 2n: cubic boxes up to 88^3 in FP32, 70^3 in FP64);
 * larger targets get DDA_ERR_INVALID_ARG with the sizes in dda_last_error().
 * The 64 MiB are committed on a device when the first target is created there:
 * dda_target_create looks up the array's device address (which loads the part
 * of the library that holds it), so this call does not.  CUDA loads each kernel
 * on its first launch; a dda_matvec with the same precision beforehand (as the
 * Green-transform rule above already asks) has launched them all.  The call is
 * synchronous: it returns after its work on the stream has finished.  All calls
 * on a device share the array and see whatever the previous call left there
 * (nothing in it needs to start at zero): calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialized by the caller. */
dda_status dda_matvec_noalloc(dda_target* t, double kd, const double* khat, const double* e,
                              const void* x_dev, void* y_dev, dda_precision precision,
                              void* cuda_stream);

typedef struct {
  double kd;             /* k d in the ambient medium                           */
  int n_inc;             /* number of incident directions (orientations) >= 1   */
  const double* khat;    /* [n_inc][3] unit propagation vectors, target frame   */
  const double* yhat;    /* [n_inc][3] Lab-Frame y axis in the target frame, for
                            the scattering basis; NULL = normalized Re(e01)    */
  const double* e01;     /* [n_inc][3][2] first polarization (normalized by the
                            library); e02 = khat x conj(e01)                    */
  int npol;              /* 1 or 2 polarizations per direction                  */
  double tol;            /* stop when ||E - A P|| / ||E|| <= tol (FP64)          */
  int max_iter;          /* cap on Krylov iterations per RHS (all sweeps)       */
  dda_precision precision;
  double inner_tol;      /* FP32_REFINED inner tolerance.  > 0: that tolerance
                            in every sweep; 0: adaptive, each sweep reduces the
                            residual by what the target still needs,
                            max(tol/(2 * current rel. residual), 1e-5); < 0: the
                            same with the floor -inner_tol in place of 1e-5   */
  int n_dirs;            /* scattering directions besides forward (>= 0)        */
  const double* dirs;    /* [n_dirs][2] (theta_s, phi_s) radians in the Lab Frame
                            (x_LF = khat, y_LF = yhat): n = x cos(theta) +
                            y sin(theta) cos(phi) + z sin(theta) sin(phi)       */
  const double* P0;      /* optional warm start [n_inc*npol][N][3][2] or NULL   */
  int profile;           /* nonzero: time each FFT-matvec pass with CUDA events   */
  int solver;            /* dda_solver: DDA_SOLVER_BICGSTAB (0, default), _QMR,
                            _BICGSTAB2, _GPBICG or _PETRKP; unknown values:
                            DDA_ERR_INVALID_ARG                                 */
  int fp64_residual;     /* FP32_REFINED only: 0 (default) computes the refinement's
                            residuals E - A P with FP64 box vectors and FFT passes in
                            double-float arithmetic (pairs of FP32 values, ~48 bits,
                            run at FP32 rates); 1 uses FP64 arithmetic throughout */
  void* cuda_stream;     /* optional cudaStream_t of the caller (created on the
                            target's device; not cudaStreamLegacy/PerThread:
                            DDA_ERR_INVALID_ARG).  dda_solve then enqueues all its
                            device work on that stream -- after whatever the caller
                            queued there before -- and returns once it has finished;
                            the stream must not be under capture.  NULL: the
                            target's own stream.  dda_nearfield ignores it.        */
} dda_solve_params;

/* Results.  Every array is caller-allocated HOST memory; a NULL pointer means
 * "not requested".  Right-hand side index rhs = inc*npol + pol. */
typedef struct {
  double* P;       /* [n_rhs][N][3][2] dipole moments (|E_0| = 1)                  */
  double* Qext;    /* [n_rhs] extinction efficiency C_ext / (pi a_eff^2)           */
  double* Qabs;    /* [n_rhs] absorption efficiency                                 */
  double* Qsca;    /* [n_rhs] Q_ext - Q_abs                                         */
  double* famp;    /* [n_inc][n_dirs+1][2 (m)][npol (l)][2] scattering amplitudes
                      f_ml (Sec. "Scattering by Finite Targets: The Mueller Matrix", eq. f_ml_def);
                      direction 0 is forward                                         */
  int* iters;      /* [n_rhs] Krylov iterations (inner iterations when refined)     */
  double* resid;   /* [n_rhs] final FP64 true relative residual ||E - A P|| / ||E||  */
  int* sweeps;     /* [n_rhs] FP64 refinement sweeps (1 when not refined)           */
  double t_setup_ms;   /* Green-tensor transform build in this call (0 if cached) */
  double t_solve_ms;   /* solve, observables and copies (device events)           */
  int64_t matvecs;     /* RHS-matvecs executed (FP32 + FP64)                      */
  int64_t matvecs_fp64;
  /* with params->profile: device time (ms) and launch count of the five matvec
     passes, [precision 0 = FP32, 1 = FP64][pass: x fwd, y fwd, z fwd+multiply+
     inverse, y inv, x inv + diagonal], summed over the call                       */
  double kernel_ms[10];
  int64_t kernel_calls[10];
  int64_t launches;    /* CUDA kernels this call launched                          */
} dda_solve_result;

/* Solve A P = E for every incident direction and polarization of params as one
 * batch of right-hand sides (they share A unless the polarizability is LDR,
 * where only alpha differs per RHS), then compute Q_ext, Q_abs (Sec. "What
 * Does It Calculate?"; Q = C / (pi a_eff^2), a_eff = (3N/4pi)^(1/3) d) and
 * f_ml for the forward direction and params->dirs.  Returns DDA_ERR_NOCONV if
 * some RHS did not reach tol within max_iter (results hold the last iterate). */
dda_status dda_solve(dda_target* t, const dda_solve_params* params,
                     dda_solve_result* result);

/* Free a target and all its device memory.  NULL is ignored. */
void dda_target_destroy(dda_target* t);

/* Static string for a status code. */
const char* dda_status_string(dda_status s);

/* Detail of the calling thread's last failing call ("" if none). */
const char* dda_last_error(void);

/* Choose the launch schedule of the five FFT-matvec passes for this target by
 * timing candidates on the device (x-pass lines per CTA, y/z column tiles, the
 * z row pitch and whether the z pass stages its Green-transform rows in shared
 * memory), for batches of n_rhs right-hand sides, in FP32 and FP64.  Results
 * are cached per (precision, box, grid, n_rhs) for the process, and appended to
 * the file named by the environment variable DDA_TUNE_FILE when it is set (and
 * read from it first).  Builds the Green-tensor transform for kd if needed.
 * Without this call the library uses a fixed rule. */
dda_status dda_autotune(dda_target* t, double kd, int n_rhs);

/* The schedule in use: out8 = {x lines, y tile, z tile, z row pitch, z kind,
 * threads per CTA of the x, y and z passes} for DDA_PREC_FP64 or (otherwise)
 * FP32.  z kind: 0 / 1 -- one column tile of one right-hand side per CTA, Ghat
 * read through L2 / staged in shared memory; 2 / 3 -- the FP32 column-pair
 * kernel (two columns per thread, both rows of an octant row and every
 * right-hand side per CTA, its own radix-8 plan; Ghat through L2 / staged);
 * 6 / 7 -- the same with each pass's column tile moved by TMA tensor copies. */
dda_status dda_target_schedule(const dda_target* t, int precision, int* out8);

/* Set the schedule of DDA_PREC_FP64 or (otherwise) FP32 explicitly, in the
 * layout dda_target_schedule returns (for instance one saved from an earlier
 * dda_autotune).  Values outside x lines 1..64, y tile 1..64, z tile 2/4/8/16,
 * z pitch 3*tile..3*tile+8, z kind 0/1/2/3/6/7, threads 32..256 (multiples of
 * 32; up to 384 for the FP32 z pass when the target's z length has a compiled
 * radix plan for that tile; exactly 384 for kinds 2..7, which need FP32, an
 * even Lx, Lz of 64, 128, 288 or 512 and tile 4 or 8, and for 6/7 nz <= 256),
 * or needing more than 200 KB of shared memory: DDA_ERR_INVALID_ARG.  Kinds
 * 0/1 and 2/3 factor the z transform differently (the same transform, results
 * equal to FP32 rounding); otherwise the schedule changes tiling and launch
 * shape only, not the arithmetic. */
dda_status dda_set_schedule(dda_target* t, int precision, const int* in8);

/* Kernels launched by this library since the process started (all threads). */
int64_t dda_launch_count(void);

/* Near field (the guide's NRFLD option, Sec. "Near-Field Calculations"): the
 * field of the solved dipoles in and around the target, on an extended box.
 * The box adds round(ext[2a] * n_a) lattice layers below and round(ext[2a+1] *
 * n_a) above the target's box along axis a (ext = r1..r6 of the guide: -x, +x,
 * -y, +y, -z, +z; each in [0, 64]); every axis of the result is at most 1024.
 * dda_nearfield_box returns the extended dimensions dims[3] = (nx', ny', nz')
 * and the target's offset lo[3] inside them (sizing only, no GPU work). */
dda_status dda_nearfield_box(const dda_target* t, const double* ext, int* dims, int* lo);

/* Fields on every site of the extended box for the incidences in p (kd, n_inc,
 * khat, e01, npol as given to dda_solve; the other fields of p are ignored):
 *  P       : [n_rhs][N][3][2] dipole moments returned by dda_solve (host).
 *  E_sca   : field radiated by all dipoles except the one at the site,
 *            sum_{l != j} G(r_j - r_l) P_l (G as in the solve: point dipole, or
 *            the filtered tensor for FCD).
 *  E_inc   : the incident wave at the site (phase origin: the target's centre).
 *  E_macro : macroscopic field, 3/(eps_j + 2) (E_inc + E_sca) on target sites
 *            (eps_j = m_j^2, eq. macro_vs_micro), E_inc + E_sca in vacuum.
 *  B_inc   : magnetic field of the incident wave, khat x E_inc (Gaussian units).
 *  B_sca   : magnetic field of all dipoles except the site's own (the guide's
 *            NRFLD = 2), sum_{l != j} h(r_j - r_l) x P_l with h = -i k g'(r) rhat
 *            for the scalar Green function g of the solve (point e^{ikr}/r,
 *            or the filtered one for FCD); B = H for mu = 1.
 * Outputs are caller-allocated HOST arrays [n_rhs][3][nz'][ny'][nx'][2]
 * (component-major, x fastest); NULL skips one.  At target sites a converged
 * P satisfies P_j = alpha_j (E_inc + E_sca)_j up to the solve's tolerance.
 * The extended box (its own Green-tensor transform, FP64 workspace) is kept
 * on the target and reused while ext and kd stay the same. */
dda_status dda_nearfield(dda_target* t, const dda_solve_params* p, const double* P,
                         const double* ext, double* E_inc, double* E_sca, double* E_macro,
                         double* B_inc, double* B_sca);

/* ---- Scattering matrices and averages (Sec. "Averaging over Scattering
 * Directions", "Scattering by Finite Targets: The Mueller Matrix",
 * "Orientational Averaging").  Host-side helpers; no GPU needed except for
 * dda_orient_average. ---------------------------------------------------- */

/* The guide's set of scattering directions for averages over scattering angle
 * at size parameter x = k a_eff and ETASCA eta (theta at equal steps of
 * s = theta + theta/(theta + theta0), theta0 = 2 pi/(1 + x); N_phi(j) equally
 * spaced azimuths from 0) and the solid angle Omega of each (they sum to 4 pi).
 * Writes min(n, capacity) entries of theta_phi [n][2] (radians, Lab Frame) and
 * omega [n] (either may be NULL) and returns n; -1 for x <= 0 or eta < 1e-3. */
int64_t dda_scattering_directions(double x, double eta, int64_t capacity, double* theta_phi,
                                  double* omega);

/* Amplitude matrix S_1..S_4 and Mueller matrix S_ij (Bohren & Huffman) from the
 * f_ml that dda_solve returns, for n directions:
 *  f       : [n][2 (m)][2 (l)][2] f_ml of the two incident polarizations.
 *  e01_lab : [3][2] incident polarization 1 in the Lab Frame (x component 0;
 *            normalised here); e02 = x_LF x e01^*.
 *  phi_s   : [n] azimuth of each direction's scattering plane (radians).
 *  S       : [n][4][2] S_1..S_4, or NULL;  M : [n][4][4] S_ij row-major, or NULL.
 * DDA_ERR_INVALID_ARG for a null input with n > 0 or an e01_lab along x_LF. */
dda_status dda_mueller(int64_t n, const double* f, const double* e01_lab, const double* phi_s,
                       double* S, double* M);

/* Orientation samples (Sec. "Sampling in Theta, Phi, and beta"): range = (beta
 * min, max, Theta min, max, Phi min, max) radians, n = (NBETA, NTHETA, NPHI),
 * each 1..4096.  beta and Phi at interval midpoints; Theta uniform in
 * cos(Theta) (midpoints for even NTHETA, end points for odd).  Weights: wbeta
 * [NBETA] = 1/NBETA; wthetaphi [NTHETA][NPHI] = 1/(NTHETA NPHI) for even
 * NTHETA, Simpson weights (1, 4, 2, ..., 4, 1)/(3 (NTHETA - 1) NPHI) for odd
 * (each set sums to 1). */
dda_status dda_orientation_grid(const double* range, const int* n, double* beta, double* theta,
                                double* phi, double* wbeta, double* wthetaphi);

typedef struct {
  double kd;
  double range[6];          /* beta, Theta, Phi (min, max), radians                     */
  int n[3];                 /* NBETA, NTHETA, NPHI                                      */
  const double* e01_lab;    /* [3][2] incident polarization 1, Lab Frame; NULL = y_LF    */
  double tol;
  int max_iter;
  dda_precision precision;
  int solver;               /* dda_solver                                               */
  double eta;               /* > 0: averages over scattering directions (ETASCA)        */
  int n_sel;                /* Lab-Frame directions for the Mueller matrix              */
  const double* sel;        /* [n_sel][2] (theta_s, phi_s) radians                      */
  int max_rhs;              /* right-hand sides per batched solve; 0 = all at once      */
} dda_orient_params;

typedef struct {
  /* orientation averages for incident polarization l = 0 (e01), 1 (e02)               */
  double Qext[2], Qabs[2], Qsca[2];   /* Q_sca = Q_ext - Q_abs                         */
  double Qpha[2];                     /* (2 pi/k^2) Re f_ll(0) / (pi a_eff^2)          */
  double Qsca_int[2];                 /* quadrature of dC_sca/dOmega (eta > 0)         */
  double g[2][3];                     /* <n_LF> weighted by dC_sca/dOmega: g(1..3)     */
  double cos2[2];                     /* <cos^2 theta_s>                               */
  double Qbk[2];                      /* dC_sca/dOmega(theta = pi) / (pi a_eff^2)      */
  double* mueller;                    /* [n_sel][4][4] averaged S_ij, caller's; or NULL */
  int n_orient;                       /* orientations solved (NBETA NTHETA NPHI)       */
  int64_t n_sca;                      /* directions in the angular averages            */
  int64_t iters;                      /* Krylov iterations, all right-hand sides       */
  double t_solve_ms;                  /* sum of the solves' device times               */
} dda_orient_result;

/* Average over target orientations (Sec. "Orientational Averaging"): every
 * (beta, Theta, Phi) of the grid is an incidence of a batched solve (k along
 * x_LF, polarizations e01_lab and x_LF x e01_lab^*, written in the Target Frame
 * through the orientation), weighted by wbeta * wthetaphi.  Each orientation
 * is solved: the guide's shortcut of combining two polarizations for other Phi
 * holds only when alpha does not depend on the polarization (LDR's does).
 * g and <cos^2> are averaged with weights Q_sca_int.  Returns the first
 * non-OK status of the solves (DDA_ERR_NOCONV keeps the averages). */
dda_status dda_orient_average(dda_target* t, const dda_orient_params* p, dda_orient_result* r);

/* Number of occupied sites N of a target (-1 for NULL). */
int64_t dda_target_num_dipoles(const dda_target* t);

/* Upper bound on the device bytes dda_solve(t, params) allocates on the target
 * besides its creation arrays and a Green transform it already holds: the
 * solve's workspace and, when the transform for (kd, method) is not built
 * yet, its transient build grids (admission control); -1 on bad arguments. */
int64_t dda_solve_hbm_bytes(const dda_target* t, const dda_solve_params* params);

/* Upper bound on the device bytes a NEW target of this shape holds at the
 * peak of its first dda_solve(params): creation arrays, the kept Green
 * transform, its transient build grids and the workspace.  Host-only (no
 * device work, no allocation), so a scheduler can admit a request before the
 * target exists.  method: dda_pol_method.  -1 on bad arguments. */
int64_t dda_estimate_solve_bytes(int nx, int ny, int nz, int64_t n_dipoles, int ncomp,
                                 int method, const dda_solve_params* params);

/* Device bytes target t holds now (creation arrays, Green transforms,
 * workspace kept from earlier solves, near-field box); -1 for NULL. */
int64_t dda_target_device_bytes(const dda_target* t);

/* FFT grid chosen for a target: the smallest 2^a 3^b 5^c lengths >= 2n-1 per
 * axis (Sec. "Choice of FFT Algorithm": the guide's GPFA grid sizes). */
dda_status dda_target_grid(const dda_target* t, int* Lx, int* Ly, int* Lz);

#ifdef __cplusplus
}
#endif

#endif /* DDA_H */
