// Host-side launchers of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dda_common.cuh"

namespace dda {

// Count one kernel launch of this library (process-wide, for reporting).
void note_launch();
long long launch_count();

// Shared memory of the inverse x pass with nl lines: the lines (Lx x (nl+1)
// complex), the x and rhat chunks (nl nx complex each) and the sites'
// composition bytes (nl nx, rounded up to 16).
inline size_t x_inv_smem_bytes(int Lx, int nl, int nx, size_t csize) {
  return (size_t)Lx * (nl + 1) * csize + (size_t)2 * nl * nx * csize +
         (((size_t)nl * nx + 15) & ~(size_t)15);
}

struct MatvecLaunch {
  int x_lines, x_threads; size_t x_smem, xinv_smem;
  int y_tile, y_threads; size_t y_smem;
  int z_tile, z_ps, z_threads; size_t z_smem;
  bool z_gs;   // Ghat tile staged in shared memory
  int z_pair;  // FP32: the column-pair z kernel (k_fft_z_pairs); 2: with TMA tiles
};

template <typename T> MatvecLaunch plan_matvec(const OpView<T>& op);
template <typename T> cudaError_t configure_matvec_kernels(const MatvecLaunch& L);
// Time candidate schedules of each pass on live buffers and keep the fastest in L.
template <typename T>
cudaError_t autotune_matvec(const OpView<T>& op, MatvecLaunch& L, int R, const cplx_t<T>* x,
                            cplx_t<T>* y, cplx_t<T>* scratch, cudaStream_t st);
// y = A x for R right-hand sides (box layout); scratch holds R*3*nz*Ly*Lx.
// With ev (6 events), the five passes are bracketed by events for profiling
// (recorded as external events, so they also time passes inside CUDA graphs).
constexpr int kMatvecPasses = 5;
template <typename T>
cudaError_t launch_matvec(const OpView<T>& op, const MatvecLaunch& L, int R,
                          const cplx_t<T>* x, cplx_t<T>* y, cplx_t<T>* scratch,
                          const int* active, cudaStream_t st,
                          const cudaEvent_t* ev = nullptr);

// y_j = sum_{l != j} G(r_j - r_l) x_l on every box site, vacant ones included:
// the field radiated by the dipoles x (same five passes, FP64 only).  With
// magnetic, op.ghat holds the transform of h (components 0..2) and the
// product is h x x (the magnetic field B of the dipoles).
template <typename T>
cudaError_t launch_field(const OpView<T>& op, const MatvecLaunch& L, int R,
                         const cplx_t<T>* x, cplx_t<T>* y, cplx_t<T>* scratch,
                         cudaStream_t st, bool magnetic = false);

// y = A x with FP64 box vectors and the FFT passes in double-float arithmetic
// (scratch: df64c, same size as the FP64 scratch); the schedule of the FP64
// passes applies (same element size).  FP64-level accuracy at FP32 rates.
cudaError_t launch_matvec_df(const OpView<df64>& op, const MatvecLaunch& L, int R,
                             const double2* x, double2* y, df64c* scratch, const int* active,
                             cudaStream_t st, const cudaEvent_t* ev = nullptr);
cudaError_t configure_matvec_kernels_df();
// Ghat octant FP64 -> df64 (n complex values)
cudaError_t launch_split_df(int64_t n, const double2* in, df64c* out, cudaStream_t st);

// x pass forward only (box rows -> spectral rows), used by the setup transforms.
template <typename T>
cudaError_t launch_x_fwd(const OpView<T>& op, const MatvecLaunch& L, int R,
                         const cplx_t<T>* x, cplx_t<T>* out, cudaStream_t st);

// ---- Green tensor ----------------------------------------------------------
// Fill the 6 components of G on the full FFT grid (FP64), parity-mirrored.
// kind: bit 0 = filtered (FCD) scalar Green function; bit 1 = the magnetic
// vector h (B = h x P) in components 0..2 instead of G (3..5 stay zero).
cudaError_t launch_green_fill(int nx, int ny, int nz, int Lx, int Ly, int Lz, double kd,
                              int kind, double2* grid6, cudaStream_t st);
// Forward 3-D FFT of `count` full grids in place (FP64, unpruned).
cudaError_t launch_fft3d_full(const OpView<double>& op, const MatvecLaunch& L, int count,
                              double2* grids, double2* tmp, cudaStream_t st);
// Copy the octant of the transformed grids (frequency k of an axis sits at
// position pos[k]), scaled by 1/(Lx Ly Lz), to FP64 and FP32 (g32 may be null).
cudaError_t launch_green_octant(int Lx, int Ly, int Lz, const int* posx, const int* posy,
                                const int* posz, const double2* grid6, double2* g64,
                                float2* g32, cudaStream_t st);

// ---- Krylov / vector kernels -----------------------------------------------
struct KState {
  double2 rho, rho_old, alpha, omega, beta;
  double bnorm2, rnorm2, tol2;
  int active_unused;
  int iters, status, max_iter;
  // QMR (complex symmetric): quasi-residual norm tau, rotation parameter
  // theta, and the coefficients of the update d <- qa1 d + qa2 q, x <- x + d
  // that each iteration leaves for the next one's first pass
  double tau, theta;
  double2 qa1, qa2;
  double rho_floor;  // |r^T r| <= rho_floor ||r||^2 counts as a breakdown
};

enum { KS_RUN = 0, KS_CONV = 1, KS_NOCONV = 2, KS_BREAKDOWN = 3 };

// True when the FP32 z pass of this axis plan and z tile runs a compiled-plan
// kernel (matvec_fixed.cu), which takes up to 384 threads per CTA.
bool z_fixed_applies(const AxisPlan& P, int tile);
// The column-pair FP32 z kernel applies: Lz with a compiled pair plan (64, 128,
// 288, 512), Lx even, tile 4 or 8; it always runs kZPairThreads threads.
bool z_pair_applies(int Lz, int Lx, int tile);
constexpr int kZPairThreads = 384;
// Dynamic shared memory of the column-pair z kernel (with the Ghat tile if gs).
size_t zpair_smem_bytes(int Lz, int tile, bool gs);
// The column-pair kernel's TMA variant applies as well: nz <= 256 (a box
// dimension), 2 nz <= Lz, and a driver that encodes tensor maps.
bool z_pair_tma_applies(int Lz, int Lx, int nz, int tile);

// A vector pass that finishes one of the Krylov scalar steps in its last
// block (instead of a separate one-block kernel).  Up to kFoldSingle blocks
// per RHS, the last block to finish sums all partials and runs the step.
// Beyond that the blocks are counted in two levels, so that no counter takes
// more than a few hundred tickets per pass and no block sums more than ~1024
// partials: groups of at least 64 consecutive blocks (at most kFoldGroups
// groups), the last block of a group sums the group's partials into `gsum`,
// and the last group to finish sums the group sums and runs the step.  `counter` holds per RHS one word for
// the groups and kFoldGroups words for the blocks ([R][1 + kFoldGroups], zero
// between passes; the finishing blocks re-arm them); `gsum` [R][kFoldGroups][4].
enum { FOLD_NONE = 0, FOLD_ALPHA = 1, FOLD_OMEGA = 2, FOLD_RHO = 3, FOLD_QSIGMA = 4,
       FOLD_QMR = 5 };
constexpr int kFoldGroups = 1024;
constexpr int kFoldSingle = 2048;  // up to this many blocks: one level
struct FoldArgs {
  KState* ks = nullptr;
  int* active = nullptr;
  unsigned* counter = nullptr;
  int step = FOLD_NONE;
  double* gsum = nullptr;
};
// bytes of the counters and group sums of R right-hand sides (counters first,
// the sums at fold_gsum_offset)
inline size_t fold_gsum_offset(int R) {
  return ((sizeof(unsigned) * (size_t)R * (1 + kFoldGroups)) + 255) & ~(size_t)255;
}
inline size_t fold_bytes(int R) {
  return fold_gsum_offset(R) + sizeof(double) * 4 * (size_t)R * kFoldGroups;
}

// Matvecs fused with BiCGSTAB steps (same five passes as launch_matvec):
//  launch_matvec_p: p <- r + beta (p - omega v); v = A p; partials of <rhat, v>
//                   ([R][nblk][2])
//  launch_matvec_s: s <- r - alpha v; t = A s; partials of <t, s>, <t, t>
//                   ([R][nblk][4])
// nblk = matvec_partial_blocks(op, L).
template <typename T> int matvec_partial_blocks(const OpView<T>& op, const MatvecLaunch& L);
template <typename T>
cudaError_t launch_matvec_p(const OpView<T>& op, const MatvecLaunch& L, int R,
                            const cplx_t<T>* r, cplx_t<T>* p, cplx_t<T>* v,
                            const cplx_t<T>* rhat, cplx_t<T>* scratch, const KState* ks,
                            double* partials, const int* active, cudaStream_t st,
                            const cudaEvent_t* ev = nullptr, FoldArgs fold = FoldArgs());
template <typename T>
cudaError_t launch_matvec_s(const OpView<T>& op, const MatvecLaunch& L, int R,
                            const cplx_t<T>* r, const cplx_t<T>* v, cplx_t<T>* s_vec,
                            cplx_t<T>* t_vec, cplx_t<T>* scratch, const KState* ks,
                            double* partials, const int* active, cudaStream_t st,
                            const cudaEvent_t* ev = nullptr, FoldArgs fold = FoldArgs());

// QMR for complex-symmetric A (one matvec per iteration):
//  launch_matvec_q: the pending d/x update, q <- r + beta q; t = A q; partials
//                   of q^T t ([R][nblk][2])
template <typename T>
cudaError_t launch_matvec_q(const OpView<T>& op, const MatvecLaunch& L, int R,
                            const cplx_t<T>* r, cplx_t<T>* q, cplx_t<T>* d, cplx_t<T>* x,
                            cplx_t<T>* t_vec, cplx_t<T>* scratch, const KState* ks,
                            double* partials, const int* active, cudaStream_t st,
                            const cudaEvent_t* ev = nullptr, FoldArgs fold = FoldArgs());

struct RhsTables {            // per-RHS incident-wave data (device)
  const double2* pol;         // [R][3] polarization vector
  const double2* phx;         // [R][nx] exp(i k khat_x x)
  const double2* phy;         // [R][ny]
  const double2* phz;         // [R][nz]
};

// b = E_inc on occupied sites (box layout), in precision T.
template <typename T>
cudaError_t launch_einc(int nx, int ny, int nz, const uint8_t* comp, RhsTables tb, int R,
                        cplx_t<T>* b, cudaStream_t st);

int reduce_blocks(int64_t n);

// BiCGSTAB building blocks (all R RHS per launch; inactive RHS are skipped).
template <typename T>
cudaError_t launch_bicg_init(int64_t n, int R, const cplx_t<T>* b, const cplx_t<T>* ax,
                             cplx_t<T>* r, cplx_t<T>* rhat, cplx_t<T>* p, cplx_t<T>* v,
                             double* partials, cudaStream_t st);
cudaError_t launch_state_init(int R, int nblk, const double* partials, KState* ks,
                              int* active, double tol, int max_iter, cudaStream_t st);
// Body end of a device-side iteration loop: ctl[0] += 1, and the while-node's
// condition h stays set while any active[r] != 0 and ctl[0] < ctl[1].
cudaError_t launch_loop_continue(cudaGraphConditionalHandle h, const int* active, int R,
                                 int* ctl, cudaStream_t st);
cudaError_t launch_scalar_alpha(int R, int nblk, const double* partials, KState* ks,
                                int* active, cudaStream_t st);
template <typename T>
cudaError_t launch_update_xr(int64_t n, int R, cplx_t<T>* x, cplx_t<T>* r,
                             const cplx_t<T>* p, const cplx_t<T>* s, const cplx_t<T>* t,
                             const cplx_t<T>* rhat, double* partials, const KState* ks,
                             const int* active, cudaStream_t st, FoldArgs fold = FoldArgs());
cudaError_t launch_scalar_rho(int R, int nblk, const double* partials, KState* ks,
                              int* active, cudaStream_t st);

// QMR building blocks.
//  qmr_init:    r = b - ax (ax may be null), q = d = 0; partials of ||r||^2,
//               ||b||^2, r^T r ([R][nblk][4])
//  qmr_state:   tau = ||r||, theta = 0, rho = r^T r, beta = 0, no pending update;
//               |r^T r| <= rho_floor ||r||^2 (now or later) is a breakdown
//  (alpha = rho / (q^T t) runs in the last block of the matvec, FOLD_QSIGMA)
//  qmr_update_r: r -= alpha t; partials of ||r||^2, r^T r ([R][nblk][4]); its
//               last block runs the rotation, pending update coefficients,
//               convergence on the quasi-residual bound tau sqrt(k+1) <= tol
//               ||b|| and beta (FOLD_QMR)
//  qmr_flush:   apply the last pending update (all RHS)
template <typename T>
cudaError_t launch_qmr_init(int64_t n, int R, const cplx_t<T>* b, const cplx_t<T>* ax,
                            cplx_t<T>* r, cplx_t<T>* q, cplx_t<T>* d, double* partials,
                            cudaStream_t st);
cudaError_t launch_qmr_state(int R, int nblk, const double* partials, KState* ks,
                             int* active, double tol, int max_iter, double rho_floor,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_qmr_update_r(int64_t n, int R, cplx_t<T>* r, const cplx_t<T>* t,
                                double* partials, const KState* ks, const int* active,
                                cudaStream_t st, FoldArgs fold = FoldArgs());
template <typename T>
cudaError_t launch_qmr_flush(int64_t n, int R, cplx_t<T>* x, cplx_t<T>* d,
                             const cplx_t<T>* q, const KState* ks, cudaStream_t st);

// BiCGstab(2) building blocks (bicgstab2.cu).  launch_bs2_vec `which`:
//  0: u0 = r0 - beta u0            1: r0 -= alpha u1
//  2: x += alpha u0, u0 = r0 - beta u0, u1 = r1 - beta u1
//  3: r0 -= alpha u1, r1 -= alpha u2, x += alpha u0
//  4: Gram partials ||r1||^2, ||r2||^2, <r1,r2>, <r1,r0>, <r2,r0> ([R][nblk][8])
//  5: minimal-residual update with partials <rt, r0>, ||r0||^2 ([R][nblk][4])
// launch_bs2_scalar phases: see bicgstab2.cu.
template <typename T>
cudaError_t launch_bs2_vec(int which, int64_t n, int R, cplx_t<T>* x, cplx_t<T>* r0,
                           cplx_t<T>* r1, cplx_t<T>* r2, cplx_t<T>* u0, cplx_t<T>* u1,
                           cplx_t<T>* u2, const cplx_t<T>* rt, double* partials,
                           const KState* ks, const int* active, cudaStream_t st);
cudaError_t launch_bs2_scalar(int phase, int R, int nblk, const double* partials, KState* ks,
                              int* active, cudaStream_t st);

// GPBi-CG building blocks (gpbicg.cu), vectors of R RHS ([R][n] each).
// launch_gp_vec `which`:
//  0: p = r + beta (p - u), w = At + beta q
//  1: t' = r - alpha q, y = t - t' - alpha w, u = t - r + beta u, t = t'
//  2: partials <At,t>, <At,At>, <y,y>, <At,y>, <y,t> ([R][nblk][8])
//  3: u, z, x, r updates with partials <rt, r>, ||r||^2 ([R][nblk][4], the
//     layout launch_scalar_rho reads)
// launch_gp_zeta: zeta -> KState.omega, eta -> KState.qa1.
template <typename T> struct GpVecs {
  cplx_t<T>*x, *r, *p, *q, *t, *at, *y, *u, *z, *w;
  const cplx_t<T>* rt;
};
template <typename T>
cudaError_t launch_gp_vec(int which, int64_t n, int R, const GpVecs<T>& v, double* partials,
                          const KState* ks, const int* active, cudaStream_t st);
cudaError_t launch_gp_zeta(int R, int nblk, const double* partials, KState* ks, int* active,
                           cudaStream_t st);
// Conjugate gradients on the normal equations (gpbicg.cu).  launch_cg_vec
// `which`: 0: c = conj(r) (active may be NULL);  1: partials ||w||^2;
//  2: x += alpha p, r -= alpha w, c = conj(r), partials ||r||^2;
//  3: partials ||m||^2;  4: p = conj(m);  5: p = conj(m) + beta p
// (partials [R][nblk][1]).  launch_cg_scalar phases: see gpbicg.cu.
template <typename T>
cudaError_t launch_cg_vec(int which, int64_t n, int R, cplx_t<T>* x, cplx_t<T>* r,
                          cplx_t<T>* p, const cplx_t<T>* w, cplx_t<T>* c, const cplx_t<T>* m,
                          double* partials, const KState* ks, const int* active,
                          cudaStream_t st);
cudaError_t launch_cg_scalar(int phase, int R, int nblk, const double* partials, KState* ks,
                             int* active, cudaStream_t st);
// y = A x with the epilogue partials <rhat, y> ([R][nblk][2], nblk =
// matvec_partial_blocks): a plain input with the XOUT_RV epilogue.
template <typename T>
cudaError_t launch_matvec_rv(const OpView<T>& op, const MatvecLaunch& L, int R,
                             const cplx_t<T>* x, cplx_t<T>* y, const cplx_t<T>* rhat,
                             cplx_t<T>* scratch, double* partials, const int* active,
                             cudaStream_t st, const cudaEvent_t* ev = nullptr);

// ---- refinement helpers -----------------------------------------------------
// partials of ||v||^2 per RHS (FP64 vector)
cudaError_t launch_norm2(int64_t n, int R, const double2* v, double* partials,
                         cudaStream_t st);
// out[r] = sum of partials (fixed order)
cudaError_t launch_finalize_sums(int R, int nblk, int nval, const double* partials,
                                 double* out, cudaStream_t st);
// r = b - ax (FP64)
cudaError_t launch_residual(int64_t n, int R, const double2* b, const double2* ax,
                            double2* r, cudaStream_t st);
// r32 = r64 * scale[r]  (scale = 1/||r|| per RHS)
cudaError_t launch_scale_to_f32(int64_t n, int R, const double2* r64, const double* norms,
                                float2* r32, const int* active, cudaStream_t st);
// x64 += d32 * norm[r]
cudaError_t launch_accumulate(int64_t n, int R, double2* x64, const float2* d32,
                              const double* norms, const int* active, cudaStream_t st);
// precision casts
cudaError_t launch_f64_to_f32(int64_t n, const double2* a, float2* b, cudaStream_t st);
cudaError_t launch_f32_to_f64(int64_t n, const float2* a, double2* b, cudaStream_t st);

// ---- site gather / scatter (box layout <-> site list) ------------------------
cudaError_t launch_sites_to_box(int64_t N, int64_t nbox, int R, const int64_t* site,
                                const double2* v, double2* box, cudaStream_t st);
cudaError_t launch_box_to_sites(int64_t N, int64_t nbox, int R, const int64_t* site,
                                const double2* box, double2* v, cudaStream_t st);

// ---- observables --------------------------------------------------------------
// partial sums per RHS: [Im(E^*.P), |P|^2 * w(comp)] (w per RHS per comp),
// written as [R][nblk][2]
cudaError_t launch_cross_sections(int nx, int ny, int nz, const uint8_t* comp, RhsTables tb,
                                  int R, const double2* P, const double* wabs, int ncomp1,
                                  double* partials, int nblk, cudaStream_t st);
// near field on a box: E_inc from the per-RHS tables on every site (phases
// relative to the solved target's origin), E_tot = E_inc + E_sca, and the
// macroscopic field fac[comp] * E_tot (fac[0] = 1 for vacant sites), and
// B_inc = khat x E_inc (khat: [R][3]).  Outputs may be null; layout [R][3][nbox].
cudaError_t launch_nearfield_post(int nx, int ny, int nz, const uint8_t* comp, RhsTables tb,
                                  int R, const double2* esca, const double2* fac,
                                  const double* khat, double2* einc, double2* emacro,
                                  double2* binc, cudaStream_t st);
// far-field sums F[d][r][3] = sum_j P_j exp(-i k n_d . r_j), partials per block
cudaError_t launch_farfield(int nx, int ny, int nz, const uint8_t* comp, int R, int D,
                            const double2* P, const double2* fphx, const double2* fphy,
                            const double2* fphz, double* partials, int nblk,
                            cudaStream_t st);

}  // namespace dda
