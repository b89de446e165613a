// C ABI of the DDA library: targets, the Green-tensor transform cache, the
// BiCGSTAB drivers (FP64, FP32, FP32 with FP64 refinement) and observables.
// See include/dda.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dda.h"
#include "dda_ops.h"

using namespace dda;
using cd = std::complex<double>;

#include <atomic>
namespace {
// Device address of the allocation-free matvec's static scratch array on a
// device (defined with the array, below dda_matvec_noalloc's helpers).
cudaError_t static_scratch_address(int dev, void** out);
}  // namespace

static std::atomic<long long> g_launches{0};
void dda::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long dda::launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static dda_status fail(dda_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

struct CudaFail {
  cudaError_t e;
  const char* what;
};

#define CK(expr)                                                   \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) throw CudaFail{_e, #expr};              \
  } while (0)

static dda_status from_cuda(const CudaFail& f) {
  cudaGetLastError();  // clear sticky-free errors
  std::string msg = std::string(f.what) + ": " + cudaGetErrorString(f.e);
  if (f.e == cudaErrorMemoryAllocation) return fail(DDA_ERR_OOM, msg);
  return fail(DDA_ERR_CUDA, msg);
}

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void ensure(size_t n) {
    if (n <= bytes) return;
    release();
    if (n == 0) return;
    CK(cudaMalloc(&p, n));
    bytes = n;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename X> X* as() const { return reinterpret_cast<X*>(p); }
};

// ---------------------------------------------------------------------------
// FFT plans (Stockham radix sequence and twiddles, host side)
// ---------------------------------------------------------------------------
static bool is_smooth(int n) {
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

// smallest 2^a 3^b 5^c >= m (the guide's GPFA lengths)
static int smooth_at_least(int m) {
  int n = std::max(1, m);
  while (!is_smooth(n)) ++n;
  return n;
}

// Radices of L, largest first: 16s, then one 8/4/2 for the rest of the powers
// of two, then 3s and 5s; a trailing 16 is split into 4 x 4 so that the last
// stage (which the z pass runs forward, multiplies and runs back in registers
// for three components at once) has radix <= 8.
static std::vector<int> factor_radices(int L) {
  int a = 0, n = L;
  while (n % 2 == 0) { n /= 2; ++a; }
  std::vector<int> r;
  int q = a / 4, rem = a % 4;
  for (int i = 0; i < q; ++i) r.push_back(16);
  if (rem == 1) {
    if (q >= 1) { r.back() = 8; r.push_back(4); }   // 16*2 -> 8*4
    else r.push_back(2);
  } else if (rem == 2) {
    r.push_back(4);
  } else if (rem == 3) {
    r.push_back(8);
  }
  while (n % 3 == 0) { n /= 3; r.push_back(3); }
  while (n % 5 == 0) { n /= 5; r.push_back(5); }
  if (!r.empty() && r.back() == 16) { r.back() = 4; r.push_back(4); }
  return r;
}

// In-place plan: stage t has radix rs[t], block B_t = L / (rs[0]...rs[t-1]) and
// twiddles exp(-2 pi i j m / B_t), j < B_t/rs[t], m = 1..rs[t]-1.  Also returns
// which frequency ends up at each position after the forward (decimation in
// frequency) transform: position sum_t m_t S_t holds sum_t m_t N_t with
// S_t = B_t/rs[t] and N_t = rs[0]...rs[t-1].
static AxisPlan make_plan_radices(int L, const std::vector<int>& rs,
                                  std::vector<long double>& twr, std::vector<long double>& twi,
                                  std::vector<int>& k_at);

static AxisPlan make_plan(int L, std::vector<long double>& twr, std::vector<long double>& twi,
                          std::vector<int>& k_at) {
  return make_plan_radices(L, factor_radices(L), twr, twi, k_at);
}

// The radix plan the column-pair z kernel compiles for a z length (radices of
// at most 8, which keeps its registers low), or an empty list.
static std::vector<int> pair_plan_radices(int L) {
  switch (L) {
    case 64: return {8, 8};
    case 128: return {8, 4, 4};
    case 288: return {8, 4, 3, 3};
    case 512: return {8, 8, 8};
    default: return {};
  }
}

static AxisPlan make_plan_radices(int L, const std::vector<int>& rs,
                                  std::vector<long double>& twr, std::vector<long double>& twi,
                                  std::vector<int>& k_at) {
  AxisPlan P{};
  P.L = L;
  P.nstage = (int)rs.size();
  int B = L, off = 0;
  twr.clear(); twi.clear();
  const long double two_pi = 6.283185307179586476925286766559L;
  std::vector<int> S(P.nstage), Nt(P.nstage);
  int nprod = 1;
  for (int t = 0; t < P.nstage; ++t) {
    const int R = rs[t];
    const int Sp = B / R;
    P.radix[t] = R;
    P.blk[t] = B;
    P.tw_off[t] = off;
    P.sdiv[t] = ((1ull << 36) + (unsigned long long)Sp - 1) / (unsigned long long)Sp;
    for (int j = 0; j < Sp; ++j)
      for (int m = 1; m < R; ++m) {
        const long long num = ((long long)j * m) % (long long)B;
        const long double ang = -two_pi * (long double)num / (long double)B;
        twr.push_back(cosl(ang));
        twi.push_back(sinl(ang));
      }
    off += Sp * (R - 1);
    S[t] = Sp;
    Nt[t] = nprod;
    nprod *= R;
    B = Sp;
  }
  P.tw_len = off;
  k_at.assign(L, 0);
  for (int pos = 0; pos < L; ++pos) {
    int q = pos, k = 0;
    for (int t = 0; t < P.nstage; ++t) {
      const int m = q / S[t];
      q -= m * S[t];
      k += m * Nt[t];
    }
    k_at[pos] = k;
  }
  return P;
}

// ---------------------------------------------------------------------------
// target
// ---------------------------------------------------------------------------
struct Workspace {
  int R = 0;
  // FP64
  DevBuf b64, x64, r64, rh64, p64, v64, s64, t64, scr64;
  // FP32
  DevBuf x32, r32, rh32, p32, v32, s32, t32, scr32, b32;
  DevBuf partials, ks, active, active_outer, norms, sums;
  DevBuf pol, ph, ainv64, ainv32, ainvdf, wabs, fph, sitebuf;
  DevBuf extra64, extra32;  // extra Krylov vectors of BiCGstab(2), GPBi-CG (on first use)
  DevBuf fold;              // per-RHS block counters of the passes that end a scalar step
  template <class F> void each(F f) {
    for (DevBuf* b : {&b64, &x64, &r64, &rh64, &p64, &v64, &s64, &t64, &scr64, &x32, &r32,
                      &rh32, &p32, &v32, &s32, &t32, &scr32, &b32, &partials, &ks, &active,
                      &active_outer, &norms, &sums, &pol, &ph, &ainv64, &ainv32, &ainvdf, &wabs, &fph,
                      &extra64, &extra32, &fold,
                      &sitebuf})
      f(*b);
  }
  void release_all() { each([](DevBuf& b) { b.release(); }); }
  int64_t bytes() {
    int64_t n = 0;
    each([&n](DevBuf& b) { n += (int64_t)b.bytes; });
    return n;
  }
};

// Per-pass CUDA-event timing of the matvec kernels (enabled per solve).  Event
// sets: [slot][matvec 0/1] for the iterations between two convergence checks,
// plus one set for the FP64 residual matvecs.
constexpr int kCheckEvery = 4;  // BiCGSTAB iterations between host convergence checks

struct Profiler {
  bool on = false;
  bool created = false;
  cudaEvent_t ev[kCheckEvery][2][kMatvecPasses + 1];
  cudaEvent_t evr[kMatvecPasses + 1];
  double ms[2][kMatvecPasses];
  long long calls[2][kMatvecPasses];
  void reset() {
    for (int p = 0; p < 2; ++p)
      for (int i = 0; i < kMatvecPasses; ++i) { ms[p][i] = 0.0; calls[p][i] = 0; }
  }
  void create() {
    if (created) return;
    for (auto& slot : ev)
      for (auto& set : slot)
        for (auto& e : set) CK(cudaEventCreate(&e));
    for (auto& e : evr) CK(cudaEventCreate(&e));
    created = true;
  }
  void destroy() {
    if (!created) return;
    for (auto& slot : ev)
      for (auto& set : slot)
        for (auto& e : set) cudaEventDestroy(e);
    for (auto& e : evr) cudaEventDestroy(e);
    created = false;
  }
  const cudaEvent_t* iter_set(int slot, int k) const { return on ? ev[slot][k] : nullptr; }
  const cudaEvent_t* resid_set() const { return on ? evr : nullptr; }
  void add(int p, const cudaEvent_t* e) {
    for (int i = 0; i < kMatvecPasses; ++i) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e[i], e[i + 1]));
      ms[p][i] += t;
      calls[p][i] += 1;
    }
  }
  // after a synchronize: add the times of the first `nslots` iteration slots
  // (`nmv` matvecs per iteration)
  void harvest_iters(int p, int nslots, int nmv = 2) {
    if (!on) return;
    for (int sl = 0; sl < nslots; ++sl)
      for (int k = 0; k < nmv; ++k) add(p, ev[sl][k]);
  }
  void harvest_resid() {
    if (on) add(1, evr);
  }
};

// An instantiated CUDA graph of one block of BiCGSTAB iterations.
struct IterGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> sig;
  long long kernels = 0;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    sig.clear();
  }
};

// A device-side loop over blocks of iterations: a CUDA graph whose while-node
// runs the block (captured once) until every right-hand side is frozen or a
// cap on the blocks is reached, so a whole solve is one graph launch.
struct LoopGraph {
  IterGraph g;
  long long body_kernels = 0;  // kernels per body run (incl. the loop test)
};

struct dda_target {
  int nx = 0, ny = 0, nz = 0;
  int64_t nbox = 0, N = 0;
  int ncomp = 0;
  std::vector<cd> m;
  dda_pol_method method = DDA_POL_LDR;
  int Lx = 0, Ly = 0, Lz = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  DevBuf comp, site, tw64, tw32, twdf, perm;  // perm: k_at x|y|z, then pos x|y|z
  DevBuf twzp;  // FP32 z twiddles of the column-pair kernel's plan (when it has one)
  DevBuf zerr;  // one int: a kernel's bounded wait on a copy ran out
  AxisPlan px{}, py{}, pz{};
  int twoff[3] = {0, 0, 0};
  // Green transform cache
  bool have_green = false;
  double green_kd = 0.0;
  int green_filtered = -1;
  DevBuf g64, g32, gdf;  // Ghat octant: FP64, FP32, double-float
  // transform of the magnetic vector h (near-field B), built on demand
  bool have_h = false;
  double h_kd = 0.0;
  int h_filtered = -1;
  DevBuf h64;
  MatvecLaunch L32{}, L64{};
  bool kernels_configured = false;
  Workspace ws;
  Profiler prof;
  IterGraph graphs[2];  // FP32, FP64 (for the solver that ran last)
  LoopGraph loops[2];   // the same blocks as device-side loops
  DevBuf loopctl;       // [2] ints: blocks run, block cap
  int loopctl_host[2] = {0, 0};
  int schedule_gen = 0;  // bumped when the launch schedule changes
  // near field: the target embedded in an extended box (vacant around it)
  dda_target* nf = nullptr;
  int nf_lo[3] = {0, 0, 0}, nf_n[3] = {0, 0, 0};
};

static int64_t octant_size(const dda_target* t) {
  return (int64_t)(t->Lx / 2 + 1) * (t->Ly / 2 + 1) * (t->Lz / 2 + 1);
}

template <typename T>
static OpView<T> make_view(const dda_target* t, const void* ghat, const void* ainv,
                           const void* tw) {
  OpView<T> v{};
  v.nx = t->nx; v.ny = t->ny; v.nz = t->nz;
  v.Lx = t->Lx; v.Ly = t->Ly; v.Lz = t->Lz;
  v.Hx = t->Lx / 2 + 1; v.Hy = t->Ly / 2 + 1; v.Hz = t->Lz / 2 + 1;
  v.nbox = t->nbox;
  v.comp = t->comp.as<uint8_t>();
  v.ghat = reinterpret_cast<const cplx_t<T>*>(ghat);
  v.ainv = reinterpret_cast<const cplx_t<T>*>(ainv);
  v.ncomp1 = t->ncomp + 1;
  const cplx_t<T>* tb = reinterpret_cast<const cplx_t<T>*>(tw);
  v.twx = tb + t->twoff[0];
  v.twy = tb + t->twoff[1];
  v.twz = tb + t->twoff[2];
  const int* pm = t->perm.as<int>();
  v.kx_at = pm;
  v.ky_at = pm + t->Lx;
  v.kz_at = pm + t->Lx + t->Ly;
  v.ypos_at = pm + (t->Lx + t->Ly + t->Lz) + t->Lx;
  v.twz_pair = t->twzp.as<float2>();
  v.zerr = t->zerr.as<int>();
  v.px = t->px; v.py = t->py; v.pz = t->pz;
  auto magic = [](int d) { return ((1ull << 36) + (unsigned long long)d - 1) / (unsigned long long)d; };
  v.div_nx = magic(v.nx); v.div_ny = magic(v.ny); v.div_nz = magic(v.nz); v.div_Lx = magic(v.Lx);
  return v;
}

// Fill a tensor on the full grid (kind: see launch_green_fill), transform it
// (FP64, unpruned) and keep one octant in g64 (and g32 when given).
static void build_transform(dda_target* t, double kd, int kind, DevBuf& g64, DevBuf* g32) {
  const int64_t M = (int64_t)t->Lx * t->Ly * t->Lz;
  const int64_t H = octant_size(t);
  DevBuf full, tmp;
  try {
    full.ensure(sizeof(double2) * 6 * M);
    tmp.ensure(sizeof(double2) * 6 * M);
    g64.ensure(sizeof(double2) * 6 * H);
    if (g32) g32->ensure(sizeof(float2) * 6 * H);
    CK(launch_green_fill(t->nx, t->ny, t->nz, t->Lx, t->Ly, t->Lz, kd, kind,
                         full.as<double2>(), t->stream));
    // the full grid seen as a "box" of 2 RHS x 3 components: nothing is pruned
    OpView<double> op = make_view<double>(t, nullptr, nullptr, t->tw64.p);
    op.nx = t->Lx; op.ny = t->Ly; op.nz = t->Lz;
    op.nbox = M;
    op.comp = nullptr;
    auto magic = [](int d) { return ((1ull << 36) + (unsigned long long)d - 1) / (unsigned long long)d; };
    op.div_nx = magic(op.nx); op.div_ny = magic(op.ny); op.div_nz = magic(op.nz);
    MatvecLaunch L = plan_matvec<double>(op);
    CK(configure_matvec_kernels<double>(L));
    CK(launch_fft3d_full(op, L, 6, full.as<double2>(), tmp.as<double2>(), t->stream));
    const int* pos = t->perm.as<int>() + (t->Lx + t->Ly + t->Lz);
    CK(launch_green_octant(t->Lx, t->Ly, t->Lz, pos, pos + t->Lx, pos + t->Lx + t->Ly,
                           tmp.as<double2>(), g64.as<double2>(),
                           g32 ? g32->as<float2>() : nullptr, t->stream));
    CK(cudaStreamSynchronize(t->stream));
  } catch (...) {
    full.release();
    tmp.release();
    throw;
  }
  full.release();
  tmp.release();
}

static void build_green(dda_target* t, double kd, int filtered) {
  if (t->have_green && t->green_kd == kd && t->green_filtered == filtered) return;
  t->have_green = false;
  build_transform(t, kd, filtered, t->g64, &t->g32);
  t->gdf.ensure(sizeof(df64c) * 6 * (size_t)octant_size(t));
  CK(launch_split_df(6 * octant_size(t), t->g64.as<double2>(), t->gdf.as<df64c>(), t->stream));
  t->have_green = true;
  t->green_kd = kd;
  t->green_filtered = filtered;
}

static void build_magnetic(dda_target* t, double kd, int filtered) {
  if (t->have_h && t->h_kd == kd && t->h_filtered == filtered) return;
  t->have_h = false;
  build_transform(t, kd, filtered | 2, t->h64, nullptr);
  t->have_h = true;
  t->h_kd = kd;
  t->h_filtered = filtered;
}

// ---------------------------------------------------------------------------
// polarizabilities and incident-wave tables (host, FP64)
// ---------------------------------------------------------------------------
static const double kLdrB1 = -1.8915316, kLdrB2 = 0.1648469, kLdrB3 = -1.7700004;

static cd alpha_of(dda_pol_method meth, cd m, double kd, const double* khat, const cd* e) {
  const double pi = 3.14159265358979323846;
  const cd m2 = m * m;
  const cd a0 = 3.0 / (4.0 * pi) * (m2 - 1.0) / (m2 + 2.0);
  const cd I(0.0, 1.0);
  const double k3 = kd * kd * kd;
  if (meth == DDA_POL_CM) return a0 / (1.0 - (2.0 / 3.0) * I * k3 * a0);
  if (meth == DDA_POL_LDR) {
    double S = 0.0, en = 0.0;
    for (int c = 0; c < 3; ++c) en += std::norm(e[c]);
    for (int c = 0; c < 3; ++c) S += khat[c] * khat[c] * std::norm(e[c]) / en;
    return a0 / (1.0 + a0 * ((kLdrB1 + m2 * kLdrB2 + m2 * kLdrB3 * S) * kd * kd -
                             (2.0 / 3.0) * I * k3));
  }
  const double lg = std::log((pi - kd) / (pi + kd));
  return a0 / (1.0 - a0 * ((4.0 / 3.0) * kd * kd + (2.0 / (3.0 * pi)) * lg * k3 +
                           (2.0 / 3.0) * I * k3));
}

// The polarizability tensor's diagonal on the lattice axes x, y, z.  GKDLDR
// (Sec. "Point Dipoles: Options LATTDR and GKDLDR"; Gutkowicz-Krusin & Draine
// 2004): alpha_a = alpha_CM / {1 + alpha_CM [(b1 + m^2 b2 + m^2 b3 khat_a^2)
// (kd)^2 - (2/3) i (kd)^3]} -- the lattice dispersion relation satisfied for
// both transverse polarizations of a wave along khat (LATTDR's S replaced by
// khat_a^2 on each axis); it does not depend on the polarization.  The scalar
// prescriptions put their alpha on all three axes.
static void alpha3_of(dda_pol_method meth, cd m, double kd, const double* khat, const cd* e,
                      cd out[3]) {
  if (meth != DDA_POL_GKDLDR) {
    out[0] = out[1] = out[2] = alpha_of(meth, m, kd, khat, e);
    return;
  }
  const double pi = 3.14159265358979323846;
  const cd m2 = m * m;
  const cd a0 = 3.0 / (4.0 * pi) * (m2 - 1.0) / (m2 + 2.0);
  const cd I(0.0, 1.0);
  const double k3 = kd * kd * kd;
  for (int a = 0; a < 3; ++a)
    out[a] = a0 / (1.0 + a0 * ((kLdrB1 + m2 * kLdrB2 + m2 * kLdrB3 * khat[a] * khat[a]) * kd * kd -
                               (2.0 / 3.0) * I * k3));
}

// One right-hand side's alpha^{-1} table, [ncomp+1][3] (entry 0 unused, 0):
// FP64 and FP32 copies and, when wabs is given, the absorption weights
// -Im(alpha^{-1}) - (2/3) k^3 of C_abs on each axis.
static void ainv_table(const dda_target* t, double kd, const double* khat, const cd* e,
                       double2* a64, float2* a32, double* wabs) {
  for (int a = 0; a < 3; ++a) {
    a64[a] = make_double2(0, 0);
    a32[a] = make_float2(0, 0);
    if (wabs) wabs[a] = 0.0;
  }
  for (int c = 1; c <= t->ncomp; ++c) {
    cd al[3];
    alpha3_of(t->method, t->m[c - 1], kd, khat, e, al);
    for (int a = 0; a < 3; ++a) {
      const cd v = 1.0 / al[a];
      a64[3 * c + a] = make_double2(v.real(), v.imag());
      a32[3 * c + a] = make_float2((float)v.real(), (float)v.imag());
      if (wabs) wabs[3 * c + a] = -v.imag() - (2.0 / 3.0) * kd * kd * kd;
    }
  }
}

struct Incidence {
  double khat[3];
  double yhat[3];
  cd e[2][3];  // e01, e02
};

static dda_status make_incidence(const dda_solve_params* p, int i, Incidence& inc) {
  const double* k = p->khat + 3 * i;
  double kn = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
  if (!(kn > 0.0) || !std::isfinite(kn)) return fail(DDA_ERR_INVALID_ARG, "khat is zero");
  for (int c = 0; c < 3; ++c) inc.khat[c] = k[c] / kn;
  double en = 0.0;
  cd e1[3];
  for (int c = 0; c < 3; ++c) {
    e1[c] = cd(p->e01[6 * i + 2 * c], p->e01[6 * i + 2 * c + 1]);
    en += std::norm(e1[c]);
  }
  if (!(en > 0.0) || !std::isfinite(en)) return fail(DDA_ERR_INVALID_ARG, "e01 is zero");
  en = std::sqrt(en);
  for (int c = 0; c < 3; ++c) e1[c] /= en;
  // e01 must be transverse
  cd ke = 0.0;
  for (int c = 0; c < 3; ++c) ke += inc.khat[c] * e1[c];
  if (std::abs(ke) > 1e-6) return fail(DDA_ERR_INVALID_ARG, "e01 is not perpendicular to khat");
  const double* x = inc.khat;
  cd c1[3] = {std::conj(e1[0]), std::conj(e1[1]), std::conj(e1[2])};
  cd e2[3] = {x[1] * c1[2] - x[2] * c1[1], x[2] * c1[0] - x[0] * c1[2],
              x[0] * c1[1] - x[1] * c1[0]};
  for (int c = 0; c < 3; ++c) { inc.e[0][c] = e1[c]; inc.e[1][c] = e2[c]; }
  double y[3];
  if (p->yhat) {
    for (int c = 0; c < 3; ++c) y[c] = p->yhat[3 * i + c];
  } else {
    for (int c = 0; c < 3; ++c) y[c] = e1[c].real();
    double yn = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    if (yn < 1e-12)
      for (int c = 0; c < 3; ++c) y[c] = e1[c].imag();
  }
  // orthonormalize y against khat
  double d = y[0] * x[0] + y[1] * x[1] + y[2] * x[2];
  for (int c = 0; c < 3; ++c) y[c] -= d * x[c];
  double yn = std::sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
  if (!(yn > 1e-9)) return fail(DDA_ERR_INVALID_ARG, "yhat is parallel to khat");
  for (int c = 0; c < 3; ++c) inc.yhat[c] = y[c] / yn;
  return DDA_OK;
}

// per-axis phase table exp(i s kd u (i - (n-1)/2)) for i < n
static void axis_phase(int n, double kd, double u, double sgn, std::vector<double2>& out) {
  for (int i = 0; i < n; ++i) {
    const double arg = sgn * kd * u * (i - 0.5 * (n - 1));
    out.push_back(make_double2(std::cos(arg), std::sin(arg)));
  }
}

// Runs blocks of iterations (enqueue() queues one block) on the device until
// no right-hand side is active or max_blocks blocks have run, as ONE launch of
// a CUDA graph with a while-node (built on first use, rebuilt when `sig`
// changes); then refreshes hact.  Returns the blocks run.  Without profiling
// only: event records are not allowed inside a while-node's body.
template <class ENQ>
static int run_device_loop(dda_target* t, int slot, const std::vector<uintptr_t>& sig,
                           int max_blocks, std::vector<int>& hact, const ENQ& enqueue) {
  cudaStream_t st = t->stream;
  int* act = t->ws.active.as<int>();
  const int R = (int)hact.size();
  t->loopctl.ensure(2 * sizeof(int));
  int* ctl = t->loopctl.as<int>();
  LoopGraph& lg = t->loops[slot];
  if (lg.g.exec && lg.g.sig != sig) lg.g.reset();
  if (!lg.g.exec) {
    cudaGraph_t graph = nullptr;
    CK(cudaGraphCreate(&graph, 0));
    try {
      cudaGraphConditionalHandle h;
      CK(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams np{};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      CK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
      cudaGraph_t body = np.conditional.phGraph_out[0];
      const long long before = launch_count();
      CK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal));
      try {
        enqueue();
        CK(launch_loop_continue(h, act, R, ctl, st));
      } catch (...) {
        cudaGraph_t broken = nullptr;
        cudaStreamEndCapture(st, &broken);
        throw;
      }
      cudaGraph_t captured = nullptr;
      CK(cudaStreamEndCapture(st, &captured));
      lg.body_kernels = launch_count() - before;
      note_launches(-lg.body_kernels);  // captured, not run
      CK(cudaGraphInstantiate(&lg.g.exec, graph, 0));
    } catch (...) {
      cudaGraphDestroy(graph);
      throw;
    }
    cudaGraphDestroy(graph);
    lg.g.sig = sig;
  }
  t->loopctl_host[0] = 0;
  t->loopctl_host[1] = max_blocks;
  CK(cudaMemcpyAsync(ctl, t->loopctl_host, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaGraphLaunch(lg.g.exec, st));
  CK(cudaMemcpyAsync(t->loopctl_host, ctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hact.data(), act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int blocks = t->loopctl_host[0];
  note_launches(lg.body_kernels * blocks);
  return blocks;
}

// ---------------------------------------------------------------------------
// BiCGSTAB driver, R RHS in lockstep on the device.  Returns the number of
// iterations per RHS through `its` and the status per RHS.
// ---------------------------------------------------------------------------
template <typename T> struct Vecs {
  cplx_t<T>*b, *x, *r, *rh, *p, *v, *s, *t, *scr;
};

template <typename T>
static void bicgstab(dda_target* t, const OpView<T>& op, const MatvecLaunch& L, int R,
                     const Vecs<T>& V, bool x_nonzero, double tol, int max_iter,
                     std::vector<int>& its, std::vector<int>& status, int64_t& matvecs) {
  Workspace& w = t->ws;
  const int64_t n = 3 * t->nbox;
  const int nblk = reduce_blocks(n);
  double* part = w.partials.as<double>();
  KState* ks = w.ks.as<KState>();
  int* act = w.active.as<int>();
  cudaStream_t st = t->stream;
  if (x_nonzero) {
    CK(launch_matvec<T>(op, L, R, V.x, V.s, V.scr, nullptr, st));
    matvecs += R;
    CK(launch_bicg_init<T>(n, R, V.b, V.s, V.r, V.rh, V.p, V.v, part, st));
  } else {
    CK(launch_bicg_init<T>(n, R, V.b, nullptr, V.r, V.rh, V.p, V.v, part, st));
  }
  CK(launch_state_init(R, nblk, part, ks, act, tol, max_iter, st));
  // the scalar steps alpha, omega, rho run in the last block of the pass that
  // produces their sums (block counters start at zero and are re-armed there)
  w.fold.ensure(fold_bytes(R));
  unsigned* cnt = w.fold.as<unsigned>();
  double* gsum = reinterpret_cast<double*>(w.fold.as<char>() + fold_gsum_offset(R));
  CK(cudaMemsetAsync(cnt, 0, fold_gsum_offset(R), st));
  FoldArgs fa{ks, act, cnt, FOLD_ALPHA, gsum}, fo{ks, act, cnt, FOLD_OMEGA, gsum},
      fr{ks, act, cnt, FOLD_RHO, gsum};
  std::vector<int> hact(R);
  CK(cudaMemcpyAsync(hact.data(), act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int nact = 0;
  for (int a : hact) nact += a;
  int iter = 0;
  const int nblk_mv = matvec_partial_blocks<T>(op, L);
  // one block of nq iterations: every pointer and scalar lives in device memory,
  // so the same launch sequence is valid for every block of the solve
  auto enqueue_block = [&](int nq) {
    for (int q = 0; q < nq; ++q) {
      // p <- r + beta (p - omega v); v = A p; <rhat, v>
      CK(launch_matvec_p<T>(op, L, R, V.r, V.p, V.v, V.rh, V.scr, ks, part, act, st,
                            t->prof.iter_set(q, 0), fa));
      // s <- r - alpha v; t = A s; <t, s>, <t, t>
      CK(launch_matvec_s<T>(op, L, R, V.r, V.v, V.s, V.t, V.scr, ks, part, act, st,
                            t->prof.iter_set(q, 1), fo));
      // x += alpha p + omega s; r = s - omega t; <rhat, r>, <r, r>
      CK(launch_update_xr<T>(n, R, V.x, V.r, V.p, V.s, V.t, V.rh, part, ks, act, st, fr));
    }
  };
  // A full block is captured once into a CUDA graph and replayed; the graph is
  // rebuilt only when a pointer, the batch size or the profiling mode changes.
  std::vector<uintptr_t> sig = {(uintptr_t)sizeof(T), (uintptr_t)R, (uintptr_t)t->prof.on,
                                (uintptr_t)V.r, (uintptr_t)V.p, (uintptr_t)V.v,
                                (uintptr_t)V.rh, (uintptr_t)V.s, (uintptr_t)V.t,
                                (uintptr_t)V.x, (uintptr_t)V.scr, (uintptr_t)ks,
                                (uintptr_t)part, (uintptr_t)act, (uintptr_t)op.ghat,
                                (uintptr_t)op.ainv, (uintptr_t)nblk_mv, (uintptr_t)nblk,
                                (uintptr_t)cnt, (uintptr_t)t->schedule_gen};
  IterGraph& g = t->graphs[sizeof(T) == 4 ? 0 : 1];
  if (g.exec && g.sig != sig) g.reset();
  if (!g.exec) {
    const long long before = launch_count();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue_block(kCheckEvery);
    } catch (...) {
      cudaGraph_t broken = nullptr;
      cudaStreamEndCapture(st, &broken);  // leave capture mode before reporting
      if (broken) cudaGraphDestroy(broken);
      throw;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamEndCapture(st, &graph));
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ie);
    g.kernels = launch_count() - before;
    note_launches(-g.kernels);  // captured, not run
    g.sig = sig;
  }
  // without per-pass profiling the full blocks run as one device-side loop
  // (a single graph launch); the host loop below then only runs a remainder
  // shorter than a block, or every block when profiling
  if (!t->prof.on && nact > 0 && max_iter - iter >= kCheckEvery) {
    std::vector<uintptr_t> wsig = sig;
    wsig.push_back(7);
    const int nb = run_device_loop(t, sizeof(T) == 4 ? 0 : 1, wsig,
                                   (max_iter - iter) / kCheckEvery, hact,
                                   [&]() { enqueue_block(kCheckEvery); });
    iter += nb * kCheckEvery;
    nact = 0;
    for (int a : hact) nact += a;
  }
  while (nact > 0 && iter < max_iter) {
    // kCheckEvery iterations are queued back to back; a converged RHS is frozen
    // on the device by its active flag, so the extra iterations cost nothing
    const int nq = std::min(kCheckEvery, max_iter - iter);
    if (nq == kCheckEvery) {
      CK(cudaGraphLaunch(g.exec, st));
      note_launches(g.kernels);
    } else {
      enqueue_block(nq);
    }
    CK(cudaMemcpyAsync(hact.data(), act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    t->prof.harvest_iters(sizeof(T) == 4 ? 0 : 1, nq);
    nact = 0;
    for (int a : hact) nact += a;
    iter += nq;
  }
  std::vector<KState> hks(R);
  CK(cudaMemcpyAsync(hks.data(), ks, sizeof(KState) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  its.resize(R);
  status.resize(R);
  for (int r = 0; r < R; ++r) {
    matvecs += 2 * (int64_t)hks[r].iters;  // frozen RHS do no work
    its[r] = hks[r].iters;
    status[r] = hks[r].status == KS_RUN ? KS_NOCONV : hks[r].status;
  }
}

// ---------------------------------------------------------------------------
// QMR driver for complex-symmetric A (one matvec per iteration), R RHS in
// lockstep like bicgstab(): q lives in V.p, d in V.s, t in V.t.
// ---------------------------------------------------------------------------
template <typename T>
static void qmr(dda_target* t, const OpView<T>& op, const MatvecLaunch& L, int R,
                const Vecs<T>& V, bool x_nonzero, double tol, int max_iter,
                std::vector<int>& its, std::vector<int>& status, int64_t& matvecs) {
  Workspace& w = t->ws;
  const int64_t n = 3 * t->nbox;
  const int nblk = reduce_blocks(n);
  double* part = w.partials.as<double>();
  KState* ks = w.ks.as<KState>();
  int* act = w.active.as<int>();
  cudaStream_t st = t->stream;
  cplx_t<T>* q = V.p;
  cplx_t<T>* d = V.s;
  if (x_nonzero) {
    CK(launch_matvec<T>(op, L, R, V.x, V.t, V.scr, nullptr, st));
    matvecs += R;
    CK(launch_qmr_init<T>(n, R, V.b, V.t, V.r, q, d, part, st));
  } else {
    CK(launch_qmr_init<T>(n, R, V.b, nullptr, V.r, q, d, part, st));
  }
  // r^T r at the rounding level of the vectors' precision is numerically zero:
  // a relative 1e-10 in FP64, 1e-5 in FP32 (where the products of FP32 values
  // leave |r^T r| ~ 1e-7 ||r||^2 even when it vanishes exactly)
  const double rho_floor = sizeof(T) == 4 ? 1e-5 : 1e-10;
  CK(launch_qmr_state(R, nblk, part, ks, act, tol, max_iter, rho_floor, st));
  std::vector<int> hact(R);
  CK(cudaMemcpyAsync(hact.data(), act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int nact = 0;
  for (int a : hact) nact += a;
  int iter = 0;
  const int nblk_mv = matvec_partial_blocks<T>(op, L);
  // sigma/alpha and the rotation step run in the last block of the pass that
  // produces their sums
  w.fold.ensure(fold_bytes(R));
  unsigned* cnt = w.fold.as<unsigned>();
  double* gsum = reinterpret_cast<double*>(w.fold.as<char>() + fold_gsum_offset(R));
  CK(cudaMemsetAsync(cnt, 0, fold_gsum_offset(R), st));
  const FoldArgs fs{ks, act, cnt, FOLD_QSIGMA, gsum}, fq{ks, act, cnt, FOLD_QMR, gsum};
  auto enqueue_block = [&](int nq) {
    for (int k = 0; k < nq; ++k) {
      // pending d/x update, q <- r + beta q; t = A q; q^T t; alpha
      CK(launch_matvec_q<T>(op, L, R, V.r, q, d, V.x, V.t, V.scr, ks, part, act, st,
                            t->prof.iter_set(k, 0), fs));
      // r -= alpha t; ||r||^2, r^T r; rotation and the next pending update
      CK(launch_qmr_update_r<T>(n, R, V.r, V.t, part, ks, act, st, fq));
    }
  };
  std::vector<uintptr_t> sig = {(uintptr_t)1000 + sizeof(T), (uintptr_t)R, (uintptr_t)t->prof.on,
                                (uintptr_t)V.r, (uintptr_t)q, (uintptr_t)d, (uintptr_t)V.t,
                                (uintptr_t)V.x, (uintptr_t)V.scr, (uintptr_t)ks,
                                (uintptr_t)part, (uintptr_t)act, (uintptr_t)op.ghat,
                                (uintptr_t)op.ainv, (uintptr_t)nblk_mv, (uintptr_t)nblk,
                                (uintptr_t)cnt, (uintptr_t)t->schedule_gen};
  IterGraph& g = t->graphs[sizeof(T) == 4 ? 0 : 1];
  if (g.exec && g.sig != sig) g.reset();
  if (!g.exec) {
    const long long before = launch_count();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue_block(kCheckEvery);
    } catch (...) {
      cudaGraph_t broken = nullptr;
      cudaStreamEndCapture(st, &broken);
      if (broken) cudaGraphDestroy(broken);
      throw;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamEndCapture(st, &graph));
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ie);
    g.kernels = launch_count() - before;
    note_launches(-g.kernels);
    g.sig = sig;
  }
  // without per-pass profiling the full blocks run as one device-side loop
  // (a single graph launch); the host loop below then only runs a remainder
  // shorter than a block, or every block when profiling
  if (!t->prof.on && nact > 0 && max_iter - iter >= kCheckEvery) {
    std::vector<uintptr_t> wsig = sig;
    wsig.push_back(7);
    const int nb = run_device_loop(t, sizeof(T) == 4 ? 0 : 1, wsig,
                                   (max_iter - iter) / kCheckEvery, hact,
                                   [&]() { enqueue_block(kCheckEvery); });
    iter += nb * kCheckEvery;
    nact = 0;
    for (int a : hact) nact += a;
  }
  while (nact > 0 && iter < max_iter) {
    const int nq = std::min(kCheckEvery, max_iter - iter);
    if (nq == kCheckEvery) {
      CK(cudaGraphLaunch(g.exec, st));
      note_launches(g.kernels);
    } else {
      enqueue_block(nq);
    }
    CK(cudaMemcpyAsync(hact.data(), act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    t->prof.harvest_iters(sizeof(T) == 4 ? 0 : 1, nq, 1);
    nact = 0;
    for (int a : hact) nact += a;
    iter += nq;
  }
  // the last iteration's d/x update
  CK(launch_qmr_flush<T>(n, R, V.x, d, q, ks, st));
  std::vector<KState> hks(R);
  CK(cudaMemcpyAsync(hks.data(), ks, sizeof(KState) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  its.resize(R);
  status.resize(R);
  for (int r = 0; r < R; ++r) {
    matvecs += (int64_t)hks[r].iters;
    its[r] = hks[r].iters;
    status[r] = hks[r].status == KS_RUN ? KS_NOCONV : hks[r].status;
  }
}

// ---------------------------------------------------------------------------
// BiCGstab(2) driver (the guide's PBCGS2), R RHS in lockstep: r0 in V.r, the
// shadow vector in V.rh, u0, u1, u2 in V.p, V.v, V.s, r1 in V.t, r2 in an
// extra workspace vector.  Each cycle (two iterations, four matvecs) is one
// fixed launch sequence; two cycles are captured per CUDA graph.
// ---------------------------------------------------------------------------
template <typename T>
static void bicgstab2(dda_target* t, const OpView<T>& op, const MatvecLaunch& L, int R,
                      const Vecs<T>& V, bool x_nonzero, double tol, int max_iter,
                      std::vector<int>& its, std::vector<int>& status, int64_t& matvecs) {
  Workspace& w = t->ws;
  const int64_t n = 3 * t->nbox;
  const int nblk = reduce_blocks(n);
  double* part = w.partials.as<double>();
  KState* ks = w.ks.as<KState>();
  int* act = w.active.as<int>();
  cudaStream_t st = t->stream;
  DevBuf& xb = sizeof(T) == 4 ? w.extra32 : w.extra64;
  xb.ensure(sizeof(cplx_t<T>) * n * R);
  cplx_t<T>* r2 = xb.as<cplx_t<T>>();
  cplx_t<T>*r0 = V.r, *rt = V.rh, *u0 = V.p, *u1 = V.v, *u2 = V.s, *r1 = V.t;
  if (x_nonzero) {
    CK(launch_matvec<T>(op, L, R, V.x, V.s, V.scr, nullptr, st));
    matvecs += R;
    CK(launch_bicg_init<T>(n, R, V.b, V.s, r0, rt, u0, u1, part, st));
  } else {
    CK(launch_bicg_init<T>(n, R, V.b, nullptr, r0, rt, u0, u1, part, st));
  }
  CK(launch_state_init(R, nblk, part, ks, act, tol, max_iter, st));
  CK(launch_bs2_scalar(6, R, nblk, part, ks, act, st));
  std::vector<int> hact(R);
  CK(cudaMemcpyAsync(hact.data(), act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int nact = 0;
  for (int a : hact) nact += a;
  const int nblk_mv = matvec_partial_blocks<T>(op, L);
  constexpr int kCycles = kCheckEvery / 2;  // two iterations per cycle
  auto vec = [&](int which) {
    CK(launch_bs2_vec<T>(which, n, R, V.x, r0, r1, r2, u0, u1, u2, rt, part, ks, act, st));
  };
  auto enqueue_block = [&](int ncyc) {
    for (int c = 0; c < ncyc; ++c) {
      CK(launch_bs2_scalar(0, R, nblk, part, ks, act, st));          // beta, rho0
      vec(0);                                                        // u0 = r0 - beta u0
      CK(launch_matvec_rv<T>(op, L, R, u0, u1, rt, V.scr, part, act, st,
                             t->prof.iter_set(2 * c, 0)));           // u1 = A u0
      CK(launch_scalar_alpha(R, nblk_mv, part, ks, act, st));        // alpha
      vec(1);                                                        // r0 -= alpha u1
      CK(launch_matvec_rv<T>(op, L, R, r0, r1, rt, V.scr, part, act, st,
                             t->prof.iter_set(2 * c, 1)));           // r1 = A r0
      CK(launch_bs2_scalar(2, R, nblk_mv, part, ks, act, st));      // beta, rho0
      vec(2);                                                        // x, u0, u1
      CK(launch_matvec_rv<T>(op, L, R, u1, u2, rt, V.scr, part, act, st,
                             t->prof.iter_set(2 * c + 1, 0)));       // u2 = A u1
      CK(launch_scalar_alpha(R, nblk_mv, part, ks, act, st));        // alpha
      vec(3);                                                        // r0, r1, x
      CK(launch_matvec<T>(op, L, R, r1, r2, V.scr, act, st,
                          t->prof.iter_set(2 * c + 1, 1)));          // r2 = A r1
      vec(4);                                                        // Gram partials
      CK(launch_bs2_scalar(4, R, nblk, part, ks, act, st));          // g1, g2, omega
      vec(5);                                                        // MR update
      CK(launch_bs2_scalar(5, R, nblk, part, ks, act, st));          // convergence
    }
  };
  std::vector<uintptr_t> sig = {(uintptr_t)2000 + sizeof(T), (uintptr_t)R, (uintptr_t)t->prof.on,
                                (uintptr_t)r0, (uintptr_t)rt, (uintptr_t)u0, (uintptr_t)u1,
                                (uintptr_t)u2, (uintptr_t)r1, (uintptr_t)r2, (uintptr_t)V.x,
                                (uintptr_t)V.scr, (uintptr_t)ks, (uintptr_t)part,
                                (uintptr_t)act, (uintptr_t)op.ghat, (uintptr_t)op.ainv,
                                (uintptr_t)nblk_mv, (uintptr_t)nblk,
                                (uintptr_t)t->schedule_gen};
  IterGraph& g = t->graphs[sizeof(T) == 4 ? 0 : 1];
  if (g.exec && g.sig != sig) g.reset();
  if (!g.exec) {
    const long long before = launch_count();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue_block(kCycles);
    } catch (...) {
      cudaGraph_t broken = nullptr;
      cudaStreamEndCapture(st, &broken);
      if (broken) cudaGraphDestroy(broken);
      throw;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamEndCapture(st, &graph));
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ie);
    g.kernels = launch_count() - before;
    note_launches(-g.kernels);
    g.sig = sig;
  }
  int iter = 0;
  if (!t->prof.on && nact > 0) {
    std::vector<uintptr_t> wsig = sig;
    wsig.push_back(7);
    const int nb = run_device_loop(t, sizeof(T) == 4 ? 0 : 1, wsig,
                                   (max_iter + 2 * kCycles - 1) / (2 * kCycles), hact,
                                   [&]() { enqueue_block(kCycles); });
    iter += nb * 2 * kCycles;
    nact = 0;
    for (int a : hact) nact += a;
  }
  while (nact > 0 && iter < max_iter) {
    CK(cudaGraphLaunch(g.exec, st));
    note_launches(g.kernels);
    CK(cudaMemcpyAsync(hact.data(), act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    t->prof.harvest_iters(sizeof(T) == 4 ? 0 : 1, kCheckEvery, 2);
    nact = 0;
    for (int a : hact) nact += a;
    iter += 2 * kCycles;
  }
  std::vector<KState> hks(R);
  CK(cudaMemcpyAsync(hks.data(), ks, sizeof(KState) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  its.resize(R);
  status.resize(R);
  for (int r = 0; r < R; ++r) {
    matvecs += 2 * (int64_t)hks[r].iters;
    its[r] = hks[r].iters;
    status[r] = hks[r].status == KS_RUN ? KS_NOCONV : hks[r].status;
  }
}

// Runs one block of iterations as a CUDA graph (captured on first use, rebuilt
// when `sig` changes) until every RHS is frozen on the device.  `per_block`
// iterations of `nmv` matvecs each are enqueued by `enqueue`.
template <typename T, class ENQ>
static void run_graph_loop(dda_target* t, const std::vector<uintptr_t>& sig, int per_block,
                           int nmv, int max_iter, int nact, std::vector<int>& hact,
                           const ENQ& enqueue) {
  cudaStream_t st = t->stream;
  int* act = t->ws.active.as<int>();
  const int R = (int)hact.size();
  IterGraph& g = t->graphs[sizeof(T) == 4 ? 0 : 1];
  if (g.exec && g.sig != sig) g.reset();
  if (!g.exec) {
    const long long before = launch_count();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue();
    } catch (...) {
      cudaGraph_t broken = nullptr;
      cudaStreamEndCapture(st, &broken);
      if (broken) cudaGraphDestroy(broken);
      throw;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamEndCapture(st, &graph));
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ie);
    g.kernels = launch_count() - before;
    note_launches(-g.kernels);
    g.sig = sig;
  }
  int iter = 0;
  if (!t->prof.on && nact > 0) {
    std::vector<uintptr_t> wsig = sig;
    wsig.push_back(7);
    const int nb = run_device_loop(t, sizeof(T) == 4 ? 0 : 1, wsig,
                                   (max_iter + per_block - 1) / per_block, hact, enqueue);
    iter += nb * per_block;
    nact = 0;
    for (int a : hact) nact += a;
  }
  while (nact > 0 && iter < max_iter) {
    CK(cudaGraphLaunch(g.exec, st));
    note_launches(g.kernels);
    CK(cudaMemcpyAsync(hact.data(), act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    t->prof.harvest_iters(sizeof(T) == 4 ? 0 : 1, per_block, nmv);
    nact = 0;
    for (int a : hact) nact += a;
    iter += per_block;
  }
}

static void finish_states(dda_target* t, int R, int nmv, std::vector<int>& its,
                          std::vector<int>& status, int64_t& matvecs) {
  std::vector<KState> hks(R);
  CK(cudaMemcpyAsync(hks.data(), t->ws.ks.as<KState>(), sizeof(KState) * R,
                     cudaMemcpyDeviceToHost, t->stream));
  CK(cudaStreamSynchronize(t->stream));
  its.resize(R);
  status.resize(R);
  for (int r = 0; r < R; ++r) {
    matvecs += nmv * (int64_t)hks[r].iters;
    its[r] = hks[r].iters;
    status[r] = hks[r].status == KS_RUN ? KS_NOCONV : hks[r].status;
  }
}

static int active_count(dda_target* t, std::vector<int>& hact) {
  CK(cudaMemcpyAsync(hact.data(), t->ws.active.as<int>(), sizeof(int) * hact.size(),
                     cudaMemcpyDeviceToHost, t->stream));
  CK(cudaStreamSynchronize(t->stream));
  int nact = 0;
  for (int a : hact) nact += a;
  return nact;
}

// ---------------------------------------------------------------------------
// GPBi-CG driver (the guide's GPBICG), R RHS in lockstep: r, the shadow vector,
// p, q = A p, t and At = A t in V.r, V.rh, V.p, V.v, V.t, V.s; y, u, z, w in
// four extra workspace vectors.  Iterations (two matvecs each) are captured
// kCheckEvery per CUDA graph.
// ---------------------------------------------------------------------------
template <typename T>
static void gpbicg(dda_target* t, const OpView<T>& op, const MatvecLaunch& L, int R,
                   const Vecs<T>& V, bool x_nonzero, double tol, int max_iter,
                   std::vector<int>& its, std::vector<int>& status, int64_t& matvecs) {
  using C = cplx_t<T>;
  Workspace& w = t->ws;
  const int64_t n = 3 * t->nbox;
  const int nblk = reduce_blocks(n);
  double* part = w.partials.as<double>();
  KState* ks = w.ks.as<KState>();
  int* act = w.active.as<int>();
  cudaStream_t st = t->stream;
  DevBuf& xb = sizeof(T) == 4 ? w.extra32 : w.extra64;
  xb.ensure(4 * sizeof(C) * n * R);
  C* ex = xb.as<C>();
  const GpVecs<T> g{V.x, V.r, V.p, V.v, V.t, V.s, ex, ex + n * R, ex + 2 * n * R,
                    ex + 3 * n * R, V.rh};
  if (x_nonzero) {
    CK(launch_matvec<T>(op, L, R, V.x, V.s, V.scr, nullptr, st));
    matvecs += R;
    CK(launch_bicg_init<T>(n, R, V.b, V.s, V.r, V.rh, V.p, V.v, part, st));
  } else {
    CK(launch_bicg_init<T>(n, R, V.b, nullptr, V.r, V.rh, V.p, V.v, part, st));
  }
  CK(launch_state_init(R, nblk, part, ks, act, tol, max_iter, st));
  // t, At, u and z start at zero (p and q are zeroed by the set-up, beta = 0)
  const size_t vb = sizeof(C) * n * R;
  CK(cudaMemsetAsync(g.t, 0, vb, st));
  CK(cudaMemsetAsync(g.at, 0, vb, st));
  CK(cudaMemsetAsync(g.u, 0, vb, st));
  CK(cudaMemsetAsync(g.z, 0, vb, st));
  std::vector<int> hact(R);
  const int nact = active_count(t, hact);
  const int nblk_mv = matvec_partial_blocks<T>(op, L);
  auto enqueue = [&]() {
    for (int q = 0; q < kCheckEvery; ++q) {
      CK(launch_gp_vec<T>(0, n, R, g, part, ks, act, st));                 // p, w
      CK(launch_matvec_rv<T>(op, L, R, g.p, g.q, g.rt, V.scr, part, act, st,
                             t->prof.iter_set(q, 0)));                      // q = A p
      CK(launch_scalar_alpha(R, nblk_mv, part, ks, act, st));               // alpha
      CK(launch_gp_vec<T>(1, n, R, g, part, ks, act, st));                 // t, y, u
      CK(launch_matvec<T>(op, L, R, g.t, g.at, V.scr, act, st,
                          t->prof.iter_set(q, 1)));                         // At = A t
      CK(launch_gp_vec<T>(2, n, R, g, part, ks, act, st));                 // 2x2 sums
      CK(launch_gp_zeta(R, nblk, part, ks, act, st));                      // zeta, eta
      CK(launch_gp_vec<T>(3, n, R, g, part, ks, act, st));                 // u, z, x, r
      CK(launch_scalar_rho(R, nblk, part, ks, act, st));                   // beta, convergence
    }
  };
  const std::vector<uintptr_t> sig = {
      (uintptr_t)3000 + sizeof(T), (uintptr_t)R, (uintptr_t)t->prof.on, (uintptr_t)V.x,
      (uintptr_t)V.r, (uintptr_t)V.rh, (uintptr_t)V.p, (uintptr_t)V.v, (uintptr_t)V.t,
      (uintptr_t)V.s, (uintptr_t)ex, (uintptr_t)V.scr, (uintptr_t)ks, (uintptr_t)part,
      (uintptr_t)act, (uintptr_t)op.ghat, (uintptr_t)op.ainv, (uintptr_t)nblk_mv,
      (uintptr_t)nblk, (uintptr_t)t->schedule_gen};
  run_graph_loop<T>(t, sig, kCheckEvery, 2, max_iter, nact, hact, enqueue);
  finish_states(t, R, 2, its, status, matvecs);
}

// ---------------------------------------------------------------------------
// Conjugate gradients on the normal equations (the guide's PETRKP), R RHS in
// lockstep: r, c = conj(r), p, w = A p and m = A c in V.r, V.rh, V.p, V.v, V.s.
// ---------------------------------------------------------------------------
template <typename T>
static void cgnr(dda_target* t, const OpView<T>& op, const MatvecLaunch& L, int R,
                 const Vecs<T>& V, bool x_nonzero, double tol, int max_iter,
                 std::vector<int>& its, std::vector<int>& status, int64_t& matvecs) {
  Workspace& w = t->ws;
  const int64_t n = 3 * t->nbox;
  const int nblk = reduce_blocks(n);
  double* part = w.partials.as<double>();
  KState* ks = w.ks.as<KState>();
  int* act = w.active.as<int>();
  cudaStream_t st = t->stream;
  cplx_t<T>*r = V.r, *c = V.rh, *p = V.p, *wv = V.v, *m = V.s;
  if (x_nonzero) {
    CK(launch_matvec<T>(op, L, R, V.x, V.s, V.scr, nullptr, st));
    matvecs += R;
    CK(launch_bicg_init<T>(n, R, V.b, V.s, r, c, p, wv, part, st));
  } else {
    CK(launch_bicg_init<T>(n, R, V.b, nullptr, r, c, p, wv, part, st));
  }
  CK(launch_state_init(R, nblk, part, ks, act, tol, max_iter, st));
  auto vec = [&](int which) {
    CK(launch_cg_vec<T>(which, n, R, V.x, r, p, wv, c, m, part, ks, act, st));
  };
  // p = A^H r = conj(A conj(r)), gamma = ||p||^2
  vec(0);
  CK(launch_matvec<T>(op, L, R, c, m, V.scr, act, st));
  vec(3);
  CK(launch_cg_scalar(0, R, nblk, part, ks, act, st));
  vec(4);
  std::vector<int> hact(R);
  const int nact = active_count(t, hact);
  matvecs += nact;
  auto enqueue = [&]() {
    for (int q = 0; q < kCheckEvery; ++q) {
      CK(launch_matvec<T>(op, L, R, p, wv, V.scr, act, st, t->prof.iter_set(q, 0)));  // w = A p
      vec(1);                                                          // ||w||^2
      CK(launch_cg_scalar(1, R, nblk, part, ks, act, st));             // alpha
      vec(2);                                                          // x, r, c = conj(r)
      CK(launch_cg_scalar(2, R, nblk, part, ks, act, st));             // convergence
      CK(launch_matvec<T>(op, L, R, c, m, V.scr, act, st, t->prof.iter_set(q, 1)));  // m = A c
      vec(3);                                                          // ||m||^2
      CK(launch_cg_scalar(3, R, nblk, part, ks, act, st));             // beta, gamma
      vec(5);                                                          // p = conj(m) + beta p
    }
  };
  const std::vector<uintptr_t> sig = {
      (uintptr_t)4000 + sizeof(T), (uintptr_t)R, (uintptr_t)t->prof.on, (uintptr_t)V.x,
      (uintptr_t)r, (uintptr_t)c, (uintptr_t)p, (uintptr_t)wv, (uintptr_t)m,
      (uintptr_t)V.scr, (uintptr_t)ks, (uintptr_t)part, (uintptr_t)act, (uintptr_t)op.ghat,
      (uintptr_t)op.ainv, (uintptr_t)nblk, (uintptr_t)t->schedule_gen};
  run_graph_loop<T>(t, sig, kCheckEvery, 2, max_iter, nact, hact, enqueue);
  finish_states(t, R, 2, its, status, matvecs);
}

// Krylov solve with the requested method.  QMR's bilinear Lanczos process
// breaks down when r^T r vanishes for r != 0 (circularly polarized incident
// light makes E . E = 0 at every site), and BiCGstab(2) when its 2x2
// minimal-residual system is singular; such right-hand sides are finished by
// BiCGSTAB from the last iterate (the others are already converged there and
// take no further iterations).
template <typename T>
static void krylov(int solver, dda_target* t, const OpView<T>& op, const MatvecLaunch& L,
                   int R, const Vecs<T>& V, bool x_nonzero, double tol, int max_iter,
                   std::vector<int>& its, std::vector<int>& status, int64_t& matvecs) {
  if (solver == DDA_SOLVER_BICGSTAB) {
    bicgstab<T>(t, op, L, R, V, x_nonzero, tol, max_iter, its, status, matvecs);
    return;
  }
  if (solver == DDA_SOLVER_QMR)
    qmr<T>(t, op, L, R, V, x_nonzero, tol, max_iter, its, status, matvecs);
  else if (solver == DDA_SOLVER_GPBICG)
    gpbicg<T>(t, op, L, R, V, x_nonzero, tol, max_iter, its, status, matvecs);
  else if (solver == DDA_SOLVER_PETRKP)
    cgnr<T>(t, op, L, R, V, x_nonzero, tol, max_iter, its, status, matvecs);
  else
    bicgstab2<T>(t, op, L, R, V, x_nonzero, tol, max_iter, its, status, matvecs);
  bool broke = false;
  int left = max_iter;
  for (int r = 0; r < R; ++r)
    if (status[r] == KS_BREAKDOWN) { broke = true; left = std::min(left, max_iter - its[r]); }
  if (!broke || left < 1) return;
  std::vector<int> its2, st2;
  bicgstab<T>(t, op, L, R, V, true, tol, left, its2, st2, matvecs);
  for (int r = 0; r < R; ++r) {
    its[r] += its2[r];
    status[r] = st2[r];
  }
}

// ---------------------------------------------------------------------------
// Near field on an extended box (the guide's NRFLD option, Sec. "Near-Field
// Calculations"): the solved dipoles radiate into a box that adds
// round(r_i n) vacant layers on each side of the target's box.
// ---------------------------------------------------------------------------
static dda_status nearfield_box(const dda_target* t, const double* ext, int n[3], int lo[3]) {
  if (!ext) return fail(DDA_ERR_INVALID_ARG, "ext is NULL");
  const int nb[3] = {t->nx, t->ny, t->nz};
  for (int a = 0; a < 3; ++a) {
    const double rl = ext[2 * a], rh = ext[2 * a + 1];
    if (!(rl >= 0.0) || !(rh >= 0.0) || !std::isfinite(rl) || !std::isfinite(rh) ||
        rl > 64.0 || rh > 64.0)
      return fail(DDA_ERR_INVALID_ARG, "ext values must be finite, in [0, 64]");
    lo[a] = (int)std::lround(rl * nb[a]);
    const int hi = (int)std::lround(rh * nb[a]);
    n[a] = nb[a] + lo[a] + hi;
    if (n[a] > 1024) return fail(DDA_ERR_INVALID_ARG, "extended box exceeds 1024 sites per axis");
  }
  return DDA_OK;
}

// exp(i kd u x) at the extended box's sites, x measured from the solved target's
// origin (its box centroid): x = i - lo - (n_target - 1)/2
static void axis_phase_ext(int n_ext, int lo, int n_tgt, double kd, double u,
                           std::vector<double2>& out) {
  for (int i = 0; i < n_ext; ++i) {
    const double arg = kd * u * ((i - lo) - 0.5 * (n_tgt - 1));
    out.push_back(make_double2(std::cos(arg), std::sin(arg)));
  }
}

static dda_status ensure_nearfield_target(dda_target* t, const int n[3], const int lo[3]) {
  if (t->nf && t->nf_n[0] == n[0] && t->nf_n[1] == n[1] && t->nf_n[2] == n[2] &&
      t->nf_lo[0] == lo[0] && t->nf_lo[1] == lo[1] && t->nf_lo[2] == lo[2]) {
    t->nf->method = t->method;
    return DDA_OK;
  }
  if (t->nf) dda_target_destroy(t->nf);
  t->nf = nullptr;
  std::vector<uint8_t> c0(t->nbox);
  CK(cudaMemcpy(c0.data(), t->comp.p, t->nbox, cudaMemcpyDeviceToHost));
  const int64_t nb = (int64_t)n[0] * n[1] * n[2];
  std::vector<uint8_t> c1(nb, 0);
  for (int z = 0; z < t->nz; ++z)
    for (int y = 0; y < t->ny; ++y)
      for (int x = 0; x < t->nx; ++x)
        c1[((int64_t)(z + lo[2]) * n[1] + (y + lo[1])) * n[0] + (x + lo[0])] =
            c0[((int64_t)z * t->ny + y) * t->nx + x];
  std::vector<double> m;
  for (const cd& v : t->m) { m.push_back(v.real()); m.push_back(v.imag()); }
  dda_target* f = nullptr;
  const dda_status s = dda_target_create(n[0], n[1], n[2], c1.data(), c1.data(), t->ncomp,
                                         m.data(), &f);
  if (s != DDA_OK) return s;
  f->method = t->method;
  t->nf = f;
  for (int a = 0; a < 3; ++a) { t->nf_n[a] = n[a]; t->nf_lo[a] = lo[a]; }
  return DDA_OK;
}

// ---------------------------------------------------------------------------
// workspace sizing
// ---------------------------------------------------------------------------
static int64_t workspace_bytes(const dda_target* t, int R, dda_precision prec, int ndir) {
  const int64_t nv = 3 * t->nbox * (int64_t)R;
  const int64_t ns = 3 * (int64_t)t->nz * t->Ly * t->Lx * R;
  int64_t b = 0;
  const bool f32 = prec != DDA_PREC_FP64;
  // FP64: b, x, r (+ the 5 Krylov vectors and scratch if FP64 solve)
  b += 3 * nv * 16;
  if (!f32) b += 5 * nv * 16;
  b += ns * 16;  // FP64 scratch (final/true residual matvec)
  if (f32) b += 8 * nv * 8 + ns * 8;
  const int nblk = std::max(reduce_blocks(3 * t->nbox), 3 * t->nz * t->ny);
  // Krylov partials [R][nblk][<= 8]; far field, one incidence at a time:
  // [2][ndir+1][fblk][6]
  const int fblk = std::min(reduce_blocks(t->nbox), 304);
  b += std::max((int64_t)8 * R * nblk, (int64_t)12 * (ndir + 1) * fblk) * 8;
  b += (int64_t)R * (sizeof(KState) + 64) + (int64_t)R * (t->nx + t->ny + t->nz + 8) * 16;
  b += (int64_t)fold_bytes(R);  // scalar-step counters and group sums
  b += (int64_t)(ndir + 1) * (t->nx + t->ny + t->nz) * 16 + t->N * (int64_t)R * 48;
  return b;
}

static void configure(dda_target* t);

static void ensure_workspace(dda_target* t, int R, dda_precision prec, int ndir) {
  configure(t);
  Workspace& w = t->ws;
  const int64_t nv = 3 * t->nbox * (int64_t)R;
  const int64_t ns = 3 * (int64_t)t->nz * t->Ly * t->Lx * R;
  const bool f32 = prec != DDA_PREC_FP64;
  w.b64.ensure(nv * 16); w.x64.ensure(nv * 16); w.r64.ensure(nv * 16);
  w.scr64.ensure(ns * 16);
  if (!f32) {
    w.rh64.ensure(nv * 16); w.p64.ensure(nv * 16); w.v64.ensure(nv * 16);
    w.s64.ensure(nv * 16); w.t64.ensure(nv * 16);
  } else {
    w.x32.ensure(nv * 8); w.r32.ensure(nv * 8); w.rh32.ensure(nv * 8); w.p32.ensure(nv * 8);
    w.v32.ensure(nv * 8); w.s32.ensure(nv * 8); w.t32.ensure(nv * 8); w.b32.ensure(nv * 8);
    w.scr32.ensure(ns * 8);
  }
  const int rows = 3 * t->nz * t->ny;
  const int nblk = std::max({reduce_blocks(3 * t->nbox), (rows + t->L32.x_lines - 1) / t->L32.x_lines,
                             (rows + t->L64.x_lines - 1) / t->L64.x_lines});
  const int fblk = std::min(reduce_blocks(t->nbox), 304);
  w.partials.ensure((size_t)std::max((int64_t)8 * R * nblk, (int64_t)12 * (ndir + 1) * fblk) * 8);
  w.ks.ensure(sizeof(KState) * R);
  w.active.ensure(sizeof(int) * R);
  w.active_outer.ensure(sizeof(int) * R);
  w.norms.ensure(sizeof(double) * R);
  w.sums.ensure(sizeof(double) * 6 * (size_t)std::max(R, 2 * (ndir + 1)));
  w.pol.ensure(sizeof(double2) * 3 * R);
  w.ph.ensure(sizeof(double2) * (size_t)R * (t->nx + t->ny + t->nz));
  w.ainv64.ensure(sizeof(double2) * (size_t)R * (t->ncomp + 1) * 3);
  w.ainv32.ensure(sizeof(float2) * (size_t)R * (t->ncomp + 1) * 3);
  w.ainvdf.ensure(sizeof(df64c) * (size_t)R * (t->ncomp + 1) * 3);
  w.wabs.ensure(sizeof(double) * (size_t)R * (t->ncomp + 1) * 3);
  w.fph.ensure(sizeof(double2) * (size_t)(ndir + 1) * (t->nx + t->ny + t->nz));
  w.sitebuf.ensure(sizeof(double2) * 3 * (size_t)t->N * R);
  w.R = R;
}

static void configure(dda_target* t) {
  if (t->kernels_configured) return;
  OpView<float> v32 = make_view<float>(t, t->g32.p, nullptr, t->tw32.p);
  OpView<double> v64 = make_view<double>(t, t->g64.p, nullptr, t->tw64.p);
  t->L32 = plan_matvec<float>(v32);
  t->L64 = plan_matvec<double>(v64);
  CK(configure_matvec_kernels<float>(t->L32));
  CK(configure_matvec_kernels<double>(t->L64));
  CK(configure_matvec_kernels_df());
  t->kernels_configured = true;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* dda_status_string(dda_status s) {
  switch (s) {
    case DDA_OK: return "ok";
    case DDA_ERR_INVALID_ARG: return "invalid argument";
    case DDA_ERR_OOM: return "out of device memory";
    case DDA_ERR_CUDA: return "CUDA error";
    case DDA_ERR_NOCONV: return "not converged";
    case DDA_ERR_BREAKDOWN: return "BiCGSTAB breakdown";
    case DDA_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* dda_last_error(void) { return g_last_error.c_str(); }

int64_t dda_launch_count(void) { return (int64_t)launch_count(); }

int64_t dda_target_num_dipoles(const dda_target* t) { return t ? t->N : -1; }

dda_status dda_target_grid(const dda_target* t, int* Lx, int* Ly, int* Lz) {
  if (!t || !Lx || !Ly || !Lz) return fail(DDA_ERR_INVALID_ARG, "null argument");
  *Lx = t->Lx; *Ly = t->Ly; *Lz = t->Lz;
  return DDA_OK;
}

void dda_target_destroy(dda_target* t) {
  if (!t) return;
  if (t->nf) dda_target_destroy(t->nf);
  t->nf = nullptr;
  cudaSetDevice(t->device);
  if (t->stream) cudaStreamSynchronize(t->stream);
  t->ws.release_all();
  t->comp.release(); t->site.release(); t->tw64.release(); t->tw32.release(); t->twdf.release();
  t->twzp.release();
  t->zerr.release();
  t->perm.release();
  t->g64.release(); t->g32.release(); t->gdf.release(); t->h64.release();
  t->prof.destroy();
  t->graphs[0].reset();
  t->graphs[1].reset();
  t->loops[0].g.reset();
  t->loops[1].g.reset();
  t->loopctl.release();
  if (t->ev0) cudaEventDestroy(t->ev0);
  if (t->ev1) cudaEventDestroy(t->ev1);
  if (t->stream) cudaStreamDestroy(t->stream);
  delete t;
}

dda_status dda_target_create(int nx, int ny, int nz, const uint8_t* occ, const uint8_t* comp,
                             int ncomp, const double* m, dda_target** out) {
  g_last_error.clear();
  if (!out) return fail(DDA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 1024 || nz > 1024)
    return fail(DDA_ERR_INVALID_ARG, "box dimensions must be in 1..1024");
  if (!occ) return fail(DDA_ERR_INVALID_ARG, "occ is NULL");
  if (ncomp < 1 || ncomp > 255 || !m) return fail(DDA_ERR_INVALID_ARG, "ncomp must be 1..255 with m");
  const int64_t nbox = (int64_t)nx * ny * nz;
  std::vector<uint8_t> cgrid(nbox);
  std::vector<int64_t> sites;
  for (int64_t i = 0; i < nbox; ++i) {
    if (occ[i]) {
      const int c = comp ? comp[i] : 1;
      if (c < 1 || c > ncomp) return fail(DDA_ERR_INVALID_ARG, "composition out of 1..ncomp");
      cgrid[i] = (uint8_t)c;
      sites.push_back(i);
    } else {
      cgrid[i] = 0;
    }
  }
  if (sites.empty()) return fail(DDA_ERR_INVALID_ARG, "target has no occupied site");
  for (int c = 0; c < 2 * ncomp; ++c)
    if (!std::isfinite(m[c])) return fail(DDA_ERR_INVALID_ARG, "refractive index not finite");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(DDA_ERR_CUDA, "no CUDA device");
  }
  dda_target* t = new dda_target();
  try {
    CK(cudaGetDevice(&t->device));
    t->nx = nx; t->ny = ny; t->nz = nz;
    t->nbox = nbox;
    t->N = (int64_t)sites.size();
    t->ncomp = ncomp;
    for (int c = 0; c < ncomp; ++c) t->m.push_back(cd(m[2 * c], m[2 * c + 1]));
    t->Lx = smooth_at_least(2 * nx - 1);
    t->Ly = smooth_at_least(2 * ny - 1);
    t->Lz = smooth_at_least(2 * nz - 1);
    CK(cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking));
    {
      // Resolve the static scratch array of dda_matvec_noalloc here, where
      // allocating is allowed: the lookup loads the module that holds it and
      // commits its device memory (once per device), so that the
      // allocation-free entry point itself never does.
      void* scratch = nullptr;
      CK(static_scratch_address(t->device, &scratch));
    }
    CK(cudaEventCreate(&t->ev0));
    CK(cudaEventCreate(&t->ev1));
    t->comp.ensure(nbox);
    CK(cudaMemcpy(t->comp.p, cgrid.data(), nbox, cudaMemcpyHostToDevice));
    t->site.ensure(sizeof(int64_t) * sites.size());
    CK(cudaMemcpy(t->site.p, sites.data(), sizeof(int64_t) * sites.size(),
                  cudaMemcpyHostToDevice));
    // plans and twiddles for the three axes, one table per precision
    std::vector<double2> t64;
    std::vector<float2> t32;
    std::vector<float4> tdf;
    std::vector<int> kat;
    const int Ls[3] = {t->Lx, t->Ly, t->Lz};
    AxisPlan* ps[3] = {&t->px, &t->py, &t->pz};
    std::vector<int> posall;
    for (int a = 0; a < 3; ++a) {
      std::vector<long double> wr, wi;
      std::vector<int> ka;
      *ps[a] = make_plan(Ls[a], wr, wi, ka);
      std::vector<int> pa(Ls[a]);
      for (int q = 0; q < Ls[a]; ++q) pa[ka[q]] = q;
      kat.insert(kat.end(), ka.begin(), ka.end());
      posall.insert(posall.end(), pa.begin(), pa.end());
      t->twoff[a] = (int)t64.size();
      for (size_t i = 0; i < wr.size(); ++i) {
        t64.push_back(make_double2((double)wr[i], (double)wi[i]));
        t32.push_back(make_float2((float)wr[i], (float)wi[i]));
        // double-float: hi = nearest float, lo = float of the remainder (long double)
        const float rh = (float)wr[i], ih = (float)wi[i];
        tdf.push_back(make_float4(rh, (float)(wr[i] - (long double)rh), ih,
                                  (float)(wi[i] - (long double)ih)));
      }
    }
    if (t64.empty()) {
      t64.push_back(make_double2(1, 0)); t32.push_back(make_float2(1, 0));
      tdf.push_back(make_float4(1, 0, 0, 0));
    }
    t->tw64.ensure(sizeof(double2) * t64.size());
    t->tw32.ensure(sizeof(float2) * t32.size());
    t->twdf.ensure(sizeof(float4) * tdf.size());
    CK(cudaMemcpy(t->tw64.p, t64.data(), sizeof(double2) * t64.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t->tw32.p, t32.data(), sizeof(float2) * t32.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t->twdf.p, tdf.data(), sizeof(float4) * tdf.size(), cudaMemcpyHostToDevice));
    kat.insert(kat.end(), posall.begin(), posall.end());
    t->perm.ensure(sizeof(int) * kat.size());
    CK(cudaMemcpy(t->perm.p, kat.data(), sizeof(int) * kat.size(), cudaMemcpyHostToDevice));
    t->zerr.ensure(sizeof(int));
    CK(cudaMemset(t->zerr.p, 0, sizeof(int)));
    // twiddles of the column-pair z kernel's own radix plan (FP32)
    const std::vector<int> prs = pair_plan_radices(t->Lz);
    if (!prs.empty()) {
      std::vector<long double> wr, wi;
      std::vector<int> ka;
      make_plan_radices(t->Lz, prs, wr, wi, ka);
      std::vector<float2> tp(std::max<size_t>(1, wr.size()), make_float2(1, 0));
      for (size_t i = 0; i < wr.size(); ++i) tp[i] = make_float2((float)wr[i], (float)wi[i]);
      t->twzp.ensure(sizeof(float2) * tp.size());
      CK(cudaMemcpy(t->twzp.p, tp.data(), sizeof(float2) * tp.size(), cudaMemcpyHostToDevice));
    }
  } catch (const CudaFail& f) {
    dda_status s = from_cuda(f);
    dda_target_destroy(t);
    return s;
  }
  *out = t;
  return DDA_OK;
}

dda_status dda_set_polarizability(dda_target* t, dda_pol_method method) {
  if (!t) return fail(DDA_ERR_INVALID_ARG, "target is NULL");
  if (method != DDA_POL_CM && method != DDA_POL_LDR && method != DDA_POL_FCD &&
      method != DDA_POL_GKDLDR)
    return fail(DDA_ERR_INVALID_ARG, "unknown polarizability method");
  t->method = method;
  return DDA_OK;
}

int64_t dda_solve_hbm_bytes(const dda_target* t, const dda_solve_params* p) {
  if (!t || !p || p->n_inc < 1 || (p->npol != 1 && p->npol != 2) || p->n_dirs < 0) return -1;
  const int R = p->n_inc * p->npol;
  int64_t b = workspace_bytes(t, R, p->precision, p->n_dirs);
  // the method's extra Krylov vectors (BiCGstab(2): r2; GPBi-CG: y, u, z, w)
  const int nextra = p->solver == DDA_SOLVER_BICGSTAB2 ? 1 : p->solver == DDA_SOLVER_GPBICG ? 4 : 0;
  b += (int64_t)nextra * 3 * t->nbox * R * (p->precision == DDA_PREC_FP64 ? 16 : 8);
  const int filtered = t->method == DDA_POL_FCD ? 1 : 0;
  if (!(t->have_green && t->green_kd == p->kd && t->green_filtered == filtered)) {
    const int64_t M = (int64_t)t->Lx * t->Ly * t->Lz;
    b += 2 * 6 * M * 16;                            // transient setup grids
    b += 6 * octant_size(t) * (16 + 8 + 16);        // the kept octant (FP64, FP32, df)
  }
  return b;
}

// Device bytes a target holds now: resident arrays, Green transforms,
// workspace and its near-field box.
static int64_t held_bytes(dda_target* t) {
  int64_t b = 0;
  for (const DevBuf* d : {&t->comp, &t->site, &t->tw64, &t->tw32, &t->twdf, &t->twzp, &t->perm,
                          &t->g64, &t->g32, &t->gdf, &t->h64})
    b += (int64_t)d->bytes;
  b += t->ws.bytes();
  if (t->nf) b += held_bytes(t->nf);
  return b;
}

int64_t dda_target_device_bytes(const dda_target* t) {
  return t ? held_bytes(const_cast<dda_target*>(t)) : -1;
}

int64_t dda_estimate_solve_bytes(int nx, int ny, int nz, int64_t n_dipoles, int ncomp,
                                 int method, const dda_solve_params* p) {
  if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 1024 || nz > 1024 || ncomp < 1 ||
      ncomp > 255 || method < DDA_POL_CM || method > DDA_POL_GKDLDR)
    return -1;
  const int64_t nbox = (int64_t)nx * ny * nz;
  if (n_dipoles < 1 || n_dipoles > nbox) return -1;
  // a host-only description of the target (nothing is allocated)
  dda_target d;
  d.nx = nx; d.ny = ny; d.nz = nz;
  d.nbox = nbox;
  d.N = n_dipoles;
  d.ncomp = ncomp;
  d.method = (dda_pol_method)method;
  d.Lx = smooth_at_least(2 * nx - 1);
  d.Ly = smooth_at_least(2 * ny - 1);
  d.Lz = smooth_at_least(2 * nz - 1);
  // workspace, transient build grids and the kept transform
  const int64_t solve = dda_solve_hbm_bytes(&d, p);
  if (solve < 0) return -1;
  const int64_t Lsum = (int64_t)d.Lx + d.Ly + d.Lz;
  // dda_target_create: composition grid, site list, twiddles (FP64, FP32,
  // double-float) and the frequency/position tables
  const int64_t created = nbox + 8 * n_dipoles + Lsum * (16 + 8 + 16) + 2 * Lsum * 4 + 3 * 256;
  return created + solve;
}

// The incident direction and polarization a single-wave call needs for the
// target's polarizability (LDR reads both, GKDLDR the direction only).
static dda_status incidence_of(const dda_target* t, const double* khat, const double* e,
                               double kh[3], cd ev[3]) {
  const bool need_k = t->method == DDA_POL_LDR || t->method == DDA_POL_GKDLDR;
  const bool need_e = t->method == DDA_POL_LDR;
  if (!need_k) return DDA_OK;
  if (!khat || (need_e && !e)) return fail(DDA_ERR_INVALID_ARG, "LDR needs khat and e, GKDLDR khat");
  const double kn = std::sqrt(khat[0] * khat[0] + khat[1] * khat[1] + khat[2] * khat[2]);
  if (!(kn > 0)) return fail(DDA_ERR_INVALID_ARG, "khat is zero");
  for (int c = 0; c < 3; ++c) {
    kh[c] = khat[c] / kn;
    if (need_e) ev[c] = cd(e[2 * c], e[2 * c + 1]);
  }
  return DDA_OK;
}

static dda_status check_kd(const dda_target* t, double kd) {
  if (!(kd > 0.0) || !std::isfinite(kd)) return fail(DDA_ERR_INVALID_ARG, "kd must be > 0");
  if (t->method == DDA_POL_FCD && !(kd < 3.14159265358979323846))
    return fail(DDA_ERR_INVALID_ARG, "FCD needs kd < pi");
  return DDA_OK;
}

dda_status dda_matvec(dda_target* t, double kd, const double* khat, const double* e,
                      const double* x, double* y, dda_precision precision) {
  g_last_error.clear();
  if (!t || !x || !y) return fail(DDA_ERR_INVALID_ARG, "null argument");
  dda_status s = check_kd(t, kd);
  if (s != DDA_OK) return s;
  double kh[3] = {1, 0, 0};
  cd ev[3] = {0.0, 1.0, 0.0};
  s = incidence_of(t, khat, e, kh, ev);
  if (s != DDA_OK) return s;
  try {
    CK(cudaSetDevice(t->device));
    const int filtered = t->method == DDA_POL_FCD ? 1 : 0;
    build_green(t, kd, filtered);
    const bool dfp = precision == DDA_PREC_DF64;
    const bool f32 = precision != DDA_PREC_FP64 && !dfp;
    ensure_workspace(t, 1, f32 ? DDA_PREC_FP32 : DDA_PREC_FP64, 0);
    configure(t);
    Workspace& w = t->ws;
    std::vector<double2> ai(3 * (t->ncomp + 1));
    std::vector<float2> ai32(3 * (t->ncomp + 1));
    ainv_table(t, kd, kh, ev, ai.data(), ai32.data(), nullptr);
    cudaStream_t st = t->stream;
    CK(cudaMemcpyAsync(w.ainv64.p, ai.data(), sizeof(double2) * ai.size(),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w.ainv32.p, ai32.data(), sizeof(float2) * ai32.size(),
                       cudaMemcpyHostToDevice, st));
    const int64_t N = t->N, nbox = t->nbox;
    CK(cudaMemcpyAsync(w.sitebuf.p, x, sizeof(double2) * 3 * N, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w.x64.p, 0, sizeof(double2) * 3 * nbox, st));
    CK(launch_sites_to_box(N, nbox, 1, t->site.as<int64_t>(), w.sitebuf.as<double2>(),
                           w.x64.as<double2>(), st));
    if (dfp) {
      std::vector<float4> aidf(ai.size());
      for (size_t i = 0; i < ai.size(); ++i) {
        const df64 re(ai[i].x), im(ai[i].y);
        aidf[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
      }
      CK(cudaMemcpyAsync(w.ainvdf.p, aidf.data(), sizeof(float4) * aidf.size(),
                         cudaMemcpyHostToDevice, st));
      OpView<df64> op = make_view<df64>(t, t->gdf.p, w.ainvdf.p, t->twdf.p);
      CK(launch_matvec_df(op, t->L64, 1, w.x64.as<double2>(), w.r64.as<double2>(),
                          reinterpret_cast<df64c*>(w.scr64.p), nullptr, st));
    } else if (!f32) {
      OpView<double> op = make_view<double>(t, t->g64.p, w.ainv64.p, t->tw64.p);
      CK(launch_matvec<double>(op, t->L64, 1, w.x64.as<double2>(), w.r64.as<double2>(),
                               w.scr64.as<double2>(), nullptr, st));
    } else {
      OpView<float> op = make_view<float>(t, t->g32.p, w.ainv32.p, t->tw32.p);
      CK(launch_f64_to_f32(3 * nbox, w.x64.as<double2>(), w.x32.as<float2>(), st));
      CK(launch_matvec<float>(op, t->L32, 1, w.x32.as<float2>(), w.r32.as<float2>(),
                              w.scr32.as<float2>(), nullptr, st));
      CK(launch_f32_to_f64(3 * nbox, w.r32.as<float2>(), w.r64.as<double2>(), st));
    }
    CK(launch_box_to_sites(N, nbox, 1, t->site.as<int64_t>(), w.r64.as<double2>(),
                           w.sitebuf.as<double2>(), st));
    CK(cudaMemcpyAsync(y, w.sitebuf.p, sizeof(double2) * 3 * N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  } catch (const CudaFail& f) {
    return from_cuda(f);
  }
  return DDA_OK;
}

dda_status dda_solve(dda_target* t, const dda_solve_params* p, dda_solve_result* res) {
  g_last_error.clear();
  if (!t || !p || !res) return fail(DDA_ERR_INVALID_ARG, "null argument");
  dda_status s = check_kd(t, p->kd);
  if (s != DDA_OK) return s;
  if (p->n_inc < 1 || !p->khat || !p->e01) return fail(DDA_ERR_INVALID_ARG, "need n_inc >= 1, khat, e01");
  if (p->npol != 1 && p->npol != 2) return fail(DDA_ERR_INVALID_ARG, "npol must be 1 or 2");
  if (!(p->tol > 0.0) || p->max_iter < 1) return fail(DDA_ERR_INVALID_ARG, "tol > 0 and max_iter >= 1");
  if (p->n_dirs < 0 || (p->n_dirs > 0 && !p->dirs)) return fail(DDA_ERR_INVALID_ARG, "bad dirs");
  if (p->precision != DDA_PREC_FP64 && p->precision != DDA_PREC_FP32 &&
      p->precision != DDA_PREC_FP32_REFINED)
    return fail(DDA_ERR_INVALID_ARG, "unknown precision");
  if (p->solver < DDA_SOLVER_BICGSTAB || p->solver > DDA_SOLVER_PETRKP)
    return fail(DDA_ERR_INVALID_ARG, "unknown solver");
  const int R = p->n_inc * p->npol;
  if (R > 4096) return fail(DDA_ERR_INVALID_ARG, "at most 4096 right-hand sides");
  if (p->cuda_stream == (void*)cudaStreamLegacy || p->cuda_stream == (void*)cudaStreamPerThread)
    return fail(DDA_ERR_INVALID_ARG,
                "cuda_stream must be a created stream (not the legacy or per-thread default)");
  std::vector<Incidence> incs(p->n_inc);
  for (int i = 0; i < p->n_inc; ++i) {
    s = make_incidence(p, i, incs[i]);
    if (s != DDA_OK) return s;
  }
  const double kd = p->kd;
  const int64_t N = t->N, nbox = t->nbox;
  const int64_t n = 3 * nbox;
  const int D = p->n_dirs + 1;
  dda_status result_status = DDA_OK;
  // With a caller's stream every launch, copy and graph of this call goes to
  // that stream instead of the target's own one (restored on return).
  struct StreamSwap {
    dda_target* t;
    cudaStream_t saved;
    StreamSwap(dda_target* tt, void* s) : t(tt), saved(tt->stream) {
      if (s) t->stream = (cudaStream_t)s;
    }
    ~StreamSwap() { t->stream = saved; }
  } stream_swap(t, p->cuda_stream);
  try {
    CK(cudaSetDevice(t->device));
    cudaStream_t st = t->stream;
    const int filtered = t->method == DDA_POL_FCD ? 1 : 0;
    CK(cudaEventRecord(t->ev0, st));
    build_green(t, kd, filtered);
    CK(cudaEventRecord(t->ev1, st));
    CK(cudaEventSynchronize(t->ev1));
    float setup_ms = 0.f;
    CK(cudaEventElapsedTime(&setup_ms, t->ev0, t->ev1));
    ensure_workspace(t, R, p->precision, p->n_dirs);
    configure(t);
    Workspace& w = t->ws;
    const long long launches0 = launch_count();
    t->prof.on = p->profile != 0;
    if (t->prof.on) t->prof.create();
    t->prof.reset();
    CK(cudaEventRecord(t->ev0, st));
    // ---- per-RHS tables ----
    const int nc1 = t->ncomp + 1;
    // alpha^{-1} tables [R][ncomp+1][3]: one entry per lattice axis
    std::vector<double2> pol(3 * R), ph, ai(3 * R * nc1), fph;
    std::vector<float2> ai32(3 * R * nc1);
    std::vector<double> wabs(3 * R * nc1, 0.0);
    const double k3 = kd * kd * kd;
    for (int i = 0; i < p->n_inc; ++i)
      for (int l = 0; l < p->npol; ++l) {
        const int r = i * p->npol + l;
        for (int c = 0; c < 3; ++c)
          pol[3 * r + c] = make_double2(incs[i].e[l][c].real(), incs[i].e[l][c].imag());
        const size_t o = (size_t)3 * r * nc1;
        ainv_table(t, kd, incs[i].khat, incs[i].e[l], ai.data() + o, ai32.data() + o,
                   wabs.data() + o);
      }
    // phases: all x tables, then y, then z
    for (int r = 0; r < R; ++r) axis_phase(t->nx, kd, incs[r / p->npol].khat[0], 1.0, ph);
    for (int r = 0; r < R; ++r) axis_phase(t->ny, kd, incs[r / p->npol].khat[1], 1.0, ph);
    for (int r = 0; r < R; ++r) axis_phase(t->nz, kd, incs[r / p->npol].khat[2], 1.0, ph);
    CK(cudaMemcpyAsync(w.pol.p, pol.data(), sizeof(double2) * pol.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w.ph.p, ph.data(), sizeof(double2) * ph.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w.ainv64.p, ai.data(), sizeof(double2) * ai.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w.ainv32.p, ai32.data(), sizeof(float2) * ai32.size(), cudaMemcpyHostToDevice, st));
    std::vector<float4> aidf(ai.size());
    for (size_t i = 0; i < ai.size(); ++i) {
      const df64 re(ai[i].x), im(ai[i].y);
      aidf[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    CK(cudaMemcpyAsync(w.ainvdf.p, aidf.data(), sizeof(float4) * aidf.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w.wabs.p, wabs.data(), sizeof(double) * wabs.size(), cudaMemcpyHostToDevice, st));
    RhsTables tb;
    tb.pol = w.pol.as<double2>();
    tb.phx = w.ph.as<double2>();
    tb.phy = tb.phx + (size_t)R * t->nx;
    tb.phz = tb.phy + (size_t)R * t->ny;
    // ---- b = E_inc, x = P0 or 0 ----
    CK(launch_einc<double>(t->nx, t->ny, t->nz, t->comp.as<uint8_t>(), tb, R,
                           w.b64.as<double2>(), st));
    bool x_nonzero = false;
    CK(cudaMemsetAsync(w.x64.p, 0, sizeof(double2) * n * R, st));
    if (p->P0) {
      CK(cudaMemcpyAsync(w.sitebuf.p, p->P0, sizeof(double2) * 3 * N * R, cudaMemcpyHostToDevice, st));
      CK(launch_sites_to_box(N, nbox, R, t->site.as<int64_t>(), w.sitebuf.as<double2>(),
                             w.x64.as<double2>(), st));
      x_nonzero = true;
    }
    OpView<double> op64 = make_view<double>(t, t->g64.p, w.ainv64.p, t->tw64.p);
    OpView<float> op32 = make_view<float>(t, t->g32.p, w.ainv32.p, t->tw32.p);
    OpView<df64> opdf = make_view<df64>(t, t->gdf.p, w.ainvdf.p, t->twdf.p);
    // the refinement's residuals r = E - A x: FFT passes in double-float
    // arithmetic (FP64-level accuracy at FP32 rates) unless FP64 is requested
    const bool df_resid = p->precision == DDA_PREC_FP32_REFINED && !p->fp64_residual;
    auto resid_matvec = [&](const cudaEvent_t* ev) {
      if (df_resid)
        CK(launch_matvec_df(opdf, t->L64, R, w.x64.as<double2>(), w.r64.as<double2>(),
                            reinterpret_cast<df64c*>(w.scr64.p), nullptr, st, ev));
      else
        CK(launch_matvec<double>(op64, t->L64, R, w.x64.as<double2>(), w.r64.as<double2>(),
                                 w.scr64.as<double2>(), nullptr, st, ev));
    };
    std::vector<int> its_total(R, 0), sweeps(R, 0), status(R, KS_RUN);
    int64_t matvecs = 0, matvecs64 = 0;
    const int nblk = reduce_blocks(n);
    double* part = w.partials.as<double>();
    std::vector<double> bn2(R), rn2(R);
    bool resid_fresh = false;  // rn2 already holds ||b - A x||^2 of the final x (FP64)
    // ||b||^2 per RHS
    CK(launch_norm2(n, R, w.b64.as<double2>(), part, st));
    CK(launch_finalize_sums(R, nblk, 1, part, w.sums.as<double>(), st));
    CK(cudaMemcpyAsync(bn2.data(), w.sums.p, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));

    if (p->precision == DDA_PREC_FP64) {
      Vecs<double> V{w.b64.as<double2>(), w.x64.as<double2>(), w.r64.as<double2>(),
                     w.rh64.as<double2>(), w.p64.as<double2>(), w.v64.as<double2>(),
                     w.s64.as<double2>(), w.t64.as<double2>(), w.scr64.as<double2>()};
      std::vector<int> its;
      krylov<double>(p->solver, t, op64, t->L64, R, V, x_nonzero, p->tol, p->max_iter, its,
                     status, matvecs);
      matvecs64 = matvecs;
      for (int r = 0; r < R; ++r) { its_total[r] = its[r]; sweeps[r] = 1; }
    } else if (p->precision == DDA_PREC_FP32) {
      Vecs<float> V{w.b32.as<float2>(), w.x32.as<float2>(), w.r32.as<float2>(),
                    w.rh32.as<float2>(), w.p32.as<float2>(), w.v32.as<float2>(),
                    w.s32.as<float2>(), w.t32.as<float2>(), w.scr32.as<float2>()};
      CK(launch_f64_to_f32(n * R, w.b64.as<double2>(), V.b, st));
      CK(launch_f64_to_f32(n * R, w.x64.as<double2>(), V.x, st));
      std::vector<int> its;
      krylov<float>(p->solver, t, op32, t->L32, R, V, x_nonzero, p->tol, p->max_iter, its,
                    status, matvecs);
      CK(launch_f32_to_f64(n * R, V.x, w.x64.as<double2>(), st));
      for (int r = 0; r < R; ++r) { its_total[r] = its[r]; sweeps[r] = 1; }
    } else {
      // FP64 iterative refinement around FP32 BiCGSTAB
      // inner tolerance: the caller's, or adaptive -- reduce the residual only as far
      // as the outer target needs (half of tol / current relative residual), but no
      // further than FP32 arithmetic can carry the inner solve (by default 1e-5; a
      // negative inner_tol sets another floor)
      const double kInnerFloor = p->inner_tol < 0 ? -p->inner_tol : 1e-5;
      Vecs<float> V{w.b32.as<float2>(), w.x32.as<float2>(), w.r32.as<float2>(),
                    w.rh32.as<float2>(), w.p32.as<float2>(), w.v32.as<float2>(),
                    w.s32.as<float2>(), w.t32.as<float2>(), w.scr32.as<float2>()};
      std::vector<int> outer_act(R, 1);
      std::vector<double> prev(R, 0.0);
      bool first = true;
      for (int sweep = 0; sweep < 30; ++sweep) {
        // r = b - A x (FP64); skipped when x = 0
        if (first && !x_nonzero) {
          CK(cudaMemcpyAsync(w.r64.p, w.b64.p, sizeof(double2) * n * R, cudaMemcpyDeviceToDevice, st));
        } else {
          resid_matvec(t->prof.resid_set());
          matvecs += R; matvecs64 += R;
          CK(launch_residual(n, R, w.b64.as<double2>(), w.r64.as<double2>(),
                             w.r64.as<double2>(), st));
        }
        first = false;
        CK(launch_norm2(n, R, w.r64.as<double2>(), part, st));
        CK(launch_finalize_sums(R, nblk, 1, part, w.norms.as<double>(), st));
        CK(cudaMemcpyAsync(rn2.data(), w.norms.p, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (!(sweep == 0 && !x_nonzero)) t->prof.harvest_resid();
        resid_fresh = true;
        int nact = 0;
        for (int r = 0; r < R; ++r) {
          if (!outer_act[r]) continue;
          if (rn2[r] <= p->tol * p->tol * bn2[r]) { outer_act[r] = 0; status[r] = KS_CONV; continue; }
          if (!std::isfinite(rn2[r])) { outer_act[r] = 0; status[r] = KS_BREAKDOWN; continue; }
          if (its_total[r] >= p->max_iter || (sweep > 0 && rn2[r] > 0.25 * prev[r])) {
            // out of iterations, or the last sweep stagnated
            outer_act[r] = 0;
            status[r] = KS_NOCONV;
            continue;
          }
          prev[r] = rn2[r];
          ++nact;
        }
        if (nact == 0) break;
        CK(cudaMemcpyAsync(w.active_outer.p, outer_act.data(), sizeof(int) * R,
                           cudaMemcpyHostToDevice, st));
        // inner: A d = r / ||r|| in FP32 (converged RHS get a zero right-hand side)
        CK(launch_scale_to_f32(n, R, w.r64.as<double2>(), w.norms.as<double>(), V.b,
                               w.active_outer.as<int>(), st));
        CK(cudaMemsetAsync(V.x, 0, sizeof(float2) * n * R, st));
        std::vector<int> its, st_in;
        int cap = 0;
        for (int r = 0; r < R; ++r)
          if (outer_act[r]) cap = std::max(cap, p->max_iter - its_total[r]);
        double inner_tol = p->inner_tol;
        if (!(inner_tol > 0)) {
          inner_tol = 1.0;
          for (int r = 0; r < R; ++r)
            if (outer_act[r] && rn2[r] > 0)
              inner_tol = std::min(inner_tol, 0.5 * p->tol * std::sqrt(bn2[r] / rn2[r]));
          inner_tol = std::max(inner_tol, kInnerFloor);
        }
        krylov<float>(p->solver, t, op32, t->L32, R, V, false, inner_tol, std::max(1, cap),
                      its, st_in, matvecs);
        for (int r = 0; r < R; ++r) {
          if (!outer_act[r]) continue;
          its_total[r] += its[r];
          sweeps[r] += 1;
          status[r] = st_in[r] == KS_BREAKDOWN ? KS_BREAKDOWN : KS_RUN;
          if (st_in[r] == KS_BREAKDOWN && its[r] == 0) outer_act[r] = 0;
        }
        CK(launch_accumulate(n, R, w.x64.as<double2>(), V.x, w.norms.as<double>(),
                             w.active_outer.as<int>(), st));
        resid_fresh = false;
      }
      for (int r = 0; r < R; ++r)
        if (status[r] == KS_RUN) status[r] = KS_NOCONV;
    }

    // ---- true residual (FP64) of the result, unless the refinement loop's last
    //      residual already belongs to the final iterate ----
    const bool final_matvec = !resid_fresh;
    if (final_matvec) {
      resid_matvec(t->prof.resid_set());
      matvecs += R; matvecs64 += R;
      CK(launch_residual(n, R, w.b64.as<double2>(), w.r64.as<double2>(), w.r64.as<double2>(),
                         st));
      CK(launch_norm2(n, R, w.r64.as<double2>(), part, st));
      CK(launch_finalize_sums(R, nblk, 1, part, w.norms.as<double>(), st));
      CK(cudaMemcpyAsync(rn2.data(), w.norms.p, sizeof(double) * R, cudaMemcpyDeviceToHost,
                         st));
    }

    // ---- observables ----
    CK(launch_cross_sections(t->nx, t->ny, t->nz, t->comp.as<uint8_t>(), tb, R,
                             w.x64.as<double2>(), w.wabs.as<double>(), nc1, part, nblk, st));
    std::vector<double> qs(2 * R);
    CK(launch_finalize_sums(R, nblk, 2, part, w.sums.as<double>(), st));
    CK(cudaMemcpyAsync(qs.data(), w.sums.p, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (final_matvec) t->prof.harvest_resid();
    std::vector<double> ff;
    if (res->famp) {
      ff.resize((size_t)p->n_inc * D * p->npol * 6);
      const int fblk = std::min(reduce_blocks(nbox), 304);
      for (int i = 0; i < p->n_inc; ++i) {
        fph.clear();
        std::vector<double2> fx, fy, fz;
        const double* x = incs[i].khat;
        const double* y = incs[i].yhat;
        const double zz[3] = {x[1] * y[2] - x[2] * y[1], x[2] * y[0] - x[0] * y[2],
                              x[0] * y[1] - x[1] * y[0]};
        for (int d = 0; d < D; ++d) {
          const double th = d == 0 ? 0.0 : p->dirs[2 * (d - 1)];
          const double phi = d == 0 ? 0.0 : p->dirs[2 * (d - 1) + 1];
          double nv[3];
          for (int c = 0; c < 3; ++c)
            nv[c] = x[c] * std::cos(th) + y[c] * std::sin(th) * std::cos(phi) +
                    zz[c] * std::sin(th) * std::sin(phi);
          axis_phase(t->nx, kd, nv[0], -1.0, fx);
          axis_phase(t->ny, kd, nv[1], -1.0, fy);
          axis_phase(t->nz, kd, nv[2], -1.0, fz);
        }
        fph.insert(fph.end(), fx.begin(), fx.end());
        fph.insert(fph.end(), fy.begin(), fy.end());
        fph.insert(fph.end(), fz.begin(), fz.end());
        CK(cudaMemcpyAsync(w.fph.p, fph.data(), sizeof(double2) * fph.size(),
                           cudaMemcpyHostToDevice, st));
        const double2* dfx = w.fph.as<double2>();
        const double2* dfy = dfx + (size_t)D * t->nx;
        const double2* dfz = dfy + (size_t)D * t->ny;
        const double2* Pi = w.x64.as<double2>() + (size_t)i * p->npol * n;
        CK(launch_farfield(t->nx, t->ny, t->nz, t->comp.as<uint8_t>(), p->npol, D, Pi, dfx,
                           dfy, dfz, part, fblk, st));
        CK(launch_finalize_sums(p->npol * D, fblk, 6, part, w.sums.as<double>(), st));
        CK(cudaMemcpyAsync(ff.data() + (size_t)i * D * p->npol * 6, w.sums.p,
                           sizeof(double) * D * p->npol * 6, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
      }
    }
    if (res->P) {
      CK(launch_box_to_sites(N, nbox, R, t->site.as<int64_t>(), w.x64.as<double2>(),
                             w.sitebuf.as<double2>(), st));
      CK(cudaMemcpyAsync(res->P, w.sitebuf.p, sizeof(double2) * 3 * N * R,
                         cudaMemcpyDeviceToHost, st));
    }
    CK(cudaEventRecord(t->ev1, st));
    CK(cudaEventSynchronize(t->ev1));
    float solve_ms = 0.f;
    CK(cudaEventElapsedTime(&solve_ms, t->ev0, t->ev1));

    // ---- outputs ----
    const double pi = 3.14159265358979323846;
    const double aeff = std::cbrt(3.0 * (double)N / (4.0 * pi));
    const double geo = pi * aeff * aeff;
    for (int r = 0; r < R; ++r) {
      const double qe = 4.0 * pi * kd * qs[2 * r] / geo;
      const double qa = 4.0 * pi * kd * qs[2 * r + 1] / geo;
      if (res->Qext) res->Qext[r] = qe;
      if (res->Qabs) res->Qabs[r] = qa;
      if (res->Qsca) res->Qsca[r] = qe - qa;
      if (res->iters) res->iters[r] = its_total[r];
      if (res->sweeps) res->sweeps[r] = sweeps[r];
      if (res->resid) res->resid[r] = bn2[r] > 0 ? std::sqrt(rn2[r] / bn2[r]) : 0.0;
    }
    if (res->famp) {
      // sums layout per incidence: [(d*npol + l)][6] -> famp[i][d][m][l][2]
      for (int i = 0; i < p->n_inc; ++i) {
        const double* x = incs[i].khat;
        const double* y = incs[i].yhat;
        const double zz[3] = {x[1] * y[2] - x[2] * y[1], x[2] * y[0] - x[0] * y[2],
                              x[0] * y[1] - x[1] * y[0]};
        for (int d = 0; d < D; ++d) {
          const double th = d == 0 ? 0.0 : p->dirs[2 * (d - 1)];
          const double phi = d == 0 ? 0.0 : p->dirs[2 * (d - 1) + 1];
          double eth[3], eph[3];
          for (int c = 0; c < 3; ++c) {
            eth[c] = -x[c] * std::sin(th) + y[c] * std::cos(th) * std::cos(phi) +
                     zz[c] * std::cos(th) * std::sin(phi);
            eph[c] = -y[c] * std::sin(phi) + zz[c] * std::cos(phi);
          }
          for (int l = 0; l < p->npol; ++l) {
            const double* F = ff.data() + ((size_t)i * D * p->npol + (size_t)d * p->npol + l) * 6;
            for (int mm = 0; mm < 2; ++mm) {
              const double* e = mm == 0 ? eth : eph;
              double re = 0, im = 0;
              for (int c = 0; c < 3; ++c) { re += e[c] * F[2 * c]; im += e[c] * F[2 * c + 1]; }
              double* o = res->famp + ((((size_t)i * D + d) * 2 + mm) * p->npol + l) * 2;
              o[0] = k3 * re;
              o[1] = k3 * im;
            }
          }
        }
      }
    }
    res->t_setup_ms = setup_ms;
    res->t_solve_ms = solve_ms;
    for (int pp = 0; pp < 2; ++pp)
      for (int i = 0; i < kMatvecPasses; ++i) {
        res->kernel_ms[pp * kMatvecPasses + i] = t->prof.ms[pp][i];
        res->kernel_calls[pp * kMatvecPasses + i] = t->prof.calls[pp][i];
      }
    res->launches = launch_count() - launches0;
    t->prof.on = false;
    res->matvecs = matvecs;
    res->matvecs_fp64 = matvecs64;
    for (int r = 0; r < R; ++r) {
      if (status[r] == KS_BREAKDOWN) result_status = DDA_ERR_BREAKDOWN;
      else if (status[r] != KS_CONV && result_status == DDA_OK) result_status = DDA_ERR_NOCONV;
    }
    if (result_status == DDA_ERR_BREAKDOWN) g_last_error = "BiCGSTAB breakdown on some RHS";
    if (result_status == DDA_ERR_NOCONV) g_last_error = "some RHS did not reach tol";
    // a pass whose bounded wait on a TMA copy ran out stopped early: the
    // results are not to be trusted
    int zerr = 0;
    CK(cudaMemcpy(&zerr, t->zerr.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (zerr) {
      CK(cudaMemset(t->zerr.p, 0, sizeof(int)));
      result_status = DDA_ERR_TIMEOUT;
      g_last_error = "a z-pass copy (TMA) did not complete within its bounded wait";
    }
  } catch (const CudaFail& f) {
    return from_cuda(f);
  }
  return result_status;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Schedule autotuning with a process-wide cache (optionally persisted in the
// file named by DDA_TUNE_FILE: one line per key, "key : x_lines y_tile z_tile
// z_pitch z_stage x_threads y_threads z_threads").
// ---------------------------------------------------------------------------
constexpr int kScheduleLen = 8;
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

namespace {
std::mutex g_tune_mu;
std::map<std::string, std::vector<int>> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const dda_target* t, int prec, int R) {
  std::ostringstream k;
  k << (prec ? "f64" : "f32") << ' ' << t->nx << ' ' << t->ny << ' ' << t->nz << ' ' << t->Lx
    << ' ' << t->Ly << ' ' << t->Lz << ' ' << R;
  return k.str();
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* f = std::getenv("DDA_TUNE_FILE");
  if (!f) return;
  std::ifstream in(f);
  std::string line;
  while (std::getline(in, line)) {
    const size_t c = line.find(':');
    if (c == std::string::npos) continue;
    std::istringstream v(line.substr(c + 1));
    std::vector<int> vals;
    int x;
    while (v >> x) vals.push_back(x);
    std::string key = line.substr(0, c);
    while (!key.empty() && key.back() == ' ') key.pop_back();
    if (vals.size() == (size_t)kScheduleLen) g_tune[key] = vals;
  }
}

void tune_store_locked(const std::string& key, const std::vector<int>& v) {
  g_tune[key] = v;
  const char* f = std::getenv("DDA_TUNE_FILE");
  if (!f) return;
  std::ofstream out(f, std::ios::app);
  out << key << " :";
  for (int x : v) out << ' ' << x;
  out << '\n';
}

template <typename T>
void apply_schedule(const dda_target* t, MatvecLaunch& L, const std::vector<int>& v) {
  using C = cplx_t<T>;
  L.x_threads = v[5];
  L.y_threads = v[6];
  L.z_threads = v[7];
  L.x_lines = v[0];
  L.x_smem = (size_t)t->Lx * (v[0] + 1) * sizeof(C);
  L.xinv_smem = x_inv_smem_bytes(t->Lx, v[0], t->nx, sizeof(C));
  L.y_tile = v[1];
  L.y_smem = (size_t)t->Ly * v[1] * sizeof(C);
  L.z_tile = v[2];
  L.z_ps = v[3];
  // z staging 2, 3: the column-pair kernel, Ghat through L2 (2) or staged (3);
  // +4: its column tiles moved by TMA
  L.z_pair = v[4] >= 6 ? 2 : v[4] >= 2 ? 1 : 0;
  L.z_gs = v[4] == 1 || v[4] == 3 || v[4] == 7;
  const int Hz = t->Lz / 2 + 1;
  L.z_smem = (((size_t)t->Lz * L.z_ps * sizeof(C) + 15) & ~(size_t)15) +
             (L.z_gs ? (size_t)6 * Hz * L.z_tile * sizeof(C) : 0);
}

std::vector<int> schedule_of(const MatvecLaunch& L) {
  return {L.x_lines, L.y_tile, L.z_tile, L.z_ps,
          (L.z_pair ? 2 : 0) + (L.z_pair == 2 ? 4 : 0) + (L.z_gs ? 1 : 0),
          L.x_threads, L.y_threads, L.z_threads};
}
}  // namespace

extern "C" {

dda_status dda_nearfield_box(const dda_target* t, const double* ext, int* dims, int* lo) {
  g_last_error.clear();
  if (!t || !dims || !lo) return fail(DDA_ERR_INVALID_ARG, "null argument");
  return nearfield_box(t, ext, dims, lo);
}

dda_status dda_nearfield(dda_target* t, const dda_solve_params* p, const double* P,
                         const double* ext, double* E_inc, double* E_sca, double* E_macro,
                         double* B_inc, double* B_sca) {
  g_last_error.clear();
  if (!t || !p || !P) return fail(DDA_ERR_INVALID_ARG, "null argument");
  dda_status s = check_kd(t, p->kd);
  if (s != DDA_OK) return s;
  if (p->n_inc < 1 || !p->khat || !p->e01) return fail(DDA_ERR_INVALID_ARG, "need n_inc >= 1, khat, e01");
  if (p->npol != 1 && p->npol != 2) return fail(DDA_ERR_INVALID_ARG, "npol must be 1 or 2");
  const int R = p->n_inc * p->npol;
  if (R > 4096) return fail(DDA_ERR_INVALID_ARG, "at most 4096 right-hand sides");
  int n[3], lo[3];
  s = nearfield_box(t, ext, n, lo);
  if (s != DDA_OK) return s;
  std::vector<Incidence> incs(p->n_inc);
  for (int i = 0; i < p->n_inc; ++i) {
    s = make_incidence(p, i, incs[i]);
    if (s != DDA_OK) return s;
  }
  try {
    CK(cudaSetDevice(t->device));
    s = ensure_nearfield_target(t, n, lo);
    if (s != DDA_OK) return s;
    dda_target* f = t->nf;
    cudaStream_t st = f->stream;
    build_green(f, p->kd, t->method == DDA_POL_FCD ? 1 : 0);
    ensure_workspace(f, R, DDA_PREC_FP64, 0);
    Workspace& w = f->ws;
    const int64_t N = f->N, nb = f->nbox;
    // dipoles of the solved target, in the extended box
    CK(cudaMemcpyAsync(w.sitebuf.p, P, sizeof(double2) * 3 * N * R, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w.x64.p, 0, sizeof(double2) * 3 * nb * R, st));
    CK(launch_sites_to_box(N, nb, R, f->site.as<int64_t>(), w.sitebuf.as<double2>(),
                           w.x64.as<double2>(), st));
    // E_sca = sum_{l != j} G(r_j - r_l) P_l on every site
    OpView<double> op = make_view<double>(f, f->g64.p, w.ainv64.p, f->tw64.p);
    CK(launch_field<double>(op, f->L64, R, w.x64.as<double2>(), w.r64.as<double2>(),
                            w.scr64.as<double2>(), st));
    // incident wave (phases from the solved target's origin) and macroscopic field
    std::vector<double2> pol(3 * R), ph;
    for (int i = 0; i < p->n_inc; ++i)
      for (int l = 0; l < p->npol; ++l)
        for (int c = 0; c < 3; ++c)
          pol[3 * (i * p->npol + l) + c] =
              make_double2(incs[i].e[l][c].real(), incs[i].e[l][c].imag());
    const int nt[3] = {t->nx, t->ny, t->nz};
    for (int a = 0; a < 3; ++a)
      for (int r = 0; r < R; ++r)
        axis_phase_ext(n[a], lo[a], nt[a], p->kd, incs[r / p->npol].khat[a], ph);
    std::vector<double> kh(3 * R);
    for (int r = 0; r < R; ++r)
      for (int c = 0; c < 3; ++c) kh[3 * r + c] = incs[r / p->npol].khat[c];
    std::vector<double2> fac(t->ncomp + 1);
    fac[0] = make_double2(1.0, 0.0);
    for (int c = 1; c <= t->ncomp; ++c) {
      const cd e = t->m[c - 1] * t->m[c - 1];
      const cd v = 3.0 / (e + 2.0);
      fac[c] = make_double2(v.real(), v.imag());
    }
    CK(cudaMemcpyAsync(w.pol.p, pol.data(), sizeof(double2) * pol.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w.ph.p, ph.data(), sizeof(double2) * ph.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w.ainv64.p, fac.data(), sizeof(double2) * fac.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w.sums.p, kh.data(), sizeof(double) * kh.size(), cudaMemcpyHostToDevice, st));
    RhsTables tb;
    tb.pol = w.pol.as<double2>();
    tb.phx = w.ph.as<double2>();
    tb.phy = tb.phx + (size_t)R * n[0];
    tb.phz = tb.phy + (size_t)R * n[1];
    CK(launch_nearfield_post(n[0], n[1], n[2], f->comp.as<uint8_t>(), tb, R,
                             w.r64.as<double2>(), w.ainv64.as<double2>(), w.sums.as<double>(),
                             E_inc ? w.b64.as<double2>() : nullptr,
                             E_macro ? w.t64.as<double2>() : nullptr,
                             B_inc ? w.v64.as<double2>() : nullptr, st));
    const size_t bytes = sizeof(double2) * 3 * nb * R;
    if (E_sca) CK(cudaMemcpyAsync(E_sca, w.r64.p, bytes, cudaMemcpyDeviceToHost, st));
    if (E_inc) CK(cudaMemcpyAsync(E_inc, w.b64.p, bytes, cudaMemcpyDeviceToHost, st));
    if (E_macro) CK(cudaMemcpyAsync(E_macro, w.t64.p, bytes, cudaMemcpyDeviceToHost, st));
    if (B_inc) CK(cudaMemcpyAsync(B_inc, w.v64.p, bytes, cudaMemcpyDeviceToHost, st));
    if (B_sca) {
      // B_sca = sum_l h(r_j - r_l) x P_l with the magnetic vector's transform
      build_magnetic(f, p->kd, t->method == DDA_POL_FCD ? 1 : 0);
      OpView<double> oph = make_view<double>(f, f->h64.p, w.ainv64.p, f->tw64.p);
      CK(launch_field<double>(oph, f->L64, R, w.x64.as<double2>(), w.s64.as<double2>(),
                              w.scr64.as<double2>(), st, true));
      CK(cudaMemcpyAsync(B_sca, w.s64.p, bytes, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
  } catch (const CudaFail& e) {
    return from_cuda(e);
  }
  return DDA_OK;
}

dda_status dda_autotune(dda_target* t, double kd, int n_rhs) {
  g_last_error.clear();
  if (!t || n_rhs < 1 || n_rhs > 4096) return fail(DDA_ERR_INVALID_ARG, "bad arguments");
  dda_status s = check_kd(t, kd);
  if (s != DDA_OK) return s;
  try {
    CK(cudaSetDevice(t->device));
    build_green(t, kd, t->method == DDA_POL_FCD ? 1 : 0);
    ensure_workspace(t, n_rhs, DDA_PREC_FP32_REFINED, 0);  // FP32 and FP64 matvec buffers
    Workspace& w = t->ws;
    for (int prec = 0; prec < 2; ++prec) {
      const std::string key = tune_key(t, prec, n_rhs);
      std::vector<int> v;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) v = it->second;
      }
      if (v.empty()) {
        if (prec == 0) {
          OpView<float> op = make_view<float>(t, t->g32.p, w.ainv32.p, t->tw32.p);
          MatvecLaunch L = t->L32;
          CK(autotune_matvec<float>(op, L, n_rhs, w.x32.as<float2>(), w.r32.as<float2>(),
                                    w.scr32.as<float2>(), t->stream));
          v = schedule_of(L);
        } else {
          OpView<double> op = make_view<double>(t, t->g64.p, w.ainv64.p, t->tw64.p);
          MatvecLaunch L = t->L64;
          CK(autotune_matvec<double>(op, L, n_rhs, w.x64.as<double2>(), w.r64.as<double2>(),
                                     w.scr64.as<double2>(), t->stream));
          v = schedule_of(L);
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_store_locked(key, v);
      }
      if (prec == 0) apply_schedule<float>(t, t->L32, v);
      else apply_schedule<double>(t, t->L64, v);
    }
    t->schedule_gen += 1;
    ensure_workspace(t, n_rhs, DDA_PREC_FP32_REFINED, 0);  // partial-sum blocks may grow
    CK(cudaStreamSynchronize(t->stream));
  } catch (const CudaFail& f) {
    return from_cuda(f);
  }
  return DDA_OK;
}

dda_status dda_set_schedule(dda_target* t, int precision, const int* in8) {
  g_last_error.clear();
  if (!t || !in8) return fail(DDA_ERR_INVALID_ARG, "null argument");
  const int xl = in8[0], yt = in8[1], zt = in8[2], zp = in8[3], zg = in8[4];
  const bool f64 = precision == DDA_PREC_FP64;
  const size_t cs = f64 ? sizeof(double2) : sizeof(float2);
  if (xl < 1 || xl > 64 || yt < 1 || yt > 64 || (zt != 2 && zt != 4 && zt != 8 && zt != 16) ||
      zp < 3 * zt || zp > 3 * zt + 8 || zg < 0 || zg > 7 || zg == 4 || zg == 5)
    return fail(DDA_ERR_INVALID_ARG, "schedule: x lines 1..64, y tile 1..64, z tile 2/4/8/16, "
                                     "z pitch 3*tile..3*tile+8, z staging 0, 1, 2, 3, 6 or 7");
  if (zg >= 2 && (f64 || !z_pair_applies(t->Lz, t->Lx, zt) || in8[7] != kZPairThreads))
    return fail(DDA_ERR_INVALID_ARG, "schedule: z staging 2/3/6/7 (column-pair z kernel) needs "
                                     "FP32, an even Lx, Lz of 64, 128, 288 or 512, tile 4 or 8 "
                                     "and 384 threads");
  if (zg >= 6 && !z_pair_tma_applies(t->Lz, t->Lx, t->nz, zt))
    return fail(DDA_ERR_INVALID_ARG, "schedule: z staging 6/7 (TMA tiles) needs nz <= 256");
  for (int i = 5; i < 8; ++i) {
    // the FP32 z pass of a compiled radix plan (and the column-pair one) takes
    // up to 384 threads
    const int tmax =
        (i == 7 && !f64 && (z_fixed_applies(t->pz, zt) || zg >= 2)) ? 384 : 256;
    if (in8[i] < 32 || in8[i] > tmax || in8[i] % 32)
      return fail(DDA_ERR_INVALID_ARG, "schedule: threads per CTA must be a multiple of 32 in "
                                       "32..256 (FP32 z pass of a compiled plan: ..384)");
  }
  const size_t xinv = (size_t)t->Lx * (xl + 1) * cs + (size_t)2 * xl * t->nx * cs;
  const size_t ysm = (size_t)t->Ly * yt * cs;
  // a compiled-plan z kernel uses its own pitch, 3 tile (+1 below 128 B rows)
  const int zpc = (!f64 && z_fixed_applies(t->pz, zt))
                      ? std::max(zp, 3 * zt + (zt * (int)cs < 128 ? 1 : 0)) : zp;
  const size_t zsm = zg >= 2 ? zpair_smem_bytes(t->Lz, zt, zg == 3 || zg == 7)
                             : (((size_t)t->Lz * zpc * cs + 15) & ~(size_t)15) +
                                   (zg ? (size_t)6 * (t->Lz / 2 + 1) * zt * cs : 0);
  if (xinv > 200 * 1024 || ysm > 200 * 1024 || zsm > 200 * 1024)
    return fail(DDA_ERR_INVALID_ARG, "schedule: a pass would need more than 200 KB of shared memory");
  try {
    CK(cudaSetDevice(t->device));
    configure(t);
    const std::vector<int> v(in8, in8 + kScheduleLen);
    if (f64) apply_schedule<double>(t, t->L64, v);
    else apply_schedule<float>(t, t->L32, v);
    ++t->schedule_gen;
  } catch (const CudaFail& e) {
    return from_cuda(e);
  }
  return DDA_OK;
}

dda_status dda_target_schedule(const dda_target* t, int precision, int* out8) {
  if (!t || !out8) return fail(DDA_ERR_INVALID_ARG, "null argument");
  const MatvecLaunch& L = precision == DDA_PREC_FP64 ? t->L64 : t->L32;
  const std::vector<int> v = schedule_of(L);
  for (int i = 0; i < kScheduleLen; ++i) out8[i] = v[i];
  return DDA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free matvec: the same five-pass FFT convolution as dda_matvec, with
// its spectral scratch (and the alpha^{-1} table) in a fixed file-scope device
// array instead of memory this library allocates.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;  // 64 MiB per device
constexpr size_t kStaticAinvBytes = 12288;           // 256 x 3 complex FP64 entries

// Held by every GPU that loads this library, until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_ptr[64] = {nullptr};

// Device address of g_static_scratch on the current device (looked up once
// per device; the host-side symbol itself is not a device address).
cudaError_t static_scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" {

dda_status dda_matvec_noalloc(dda_target* t, double kd, const double* khat, const double* e,
                              const void* x_dev, void* y_dev, dda_precision precision,
                              void* cuda_stream) {
  g_last_error.clear();
  if (!t || !x_dev || !y_dev) return fail(DDA_ERR_INVALID_ARG, "null argument");
  if (x_dev == y_dev) return fail(DDA_ERR_INVALID_ARG, "x and y must not alias");
  if (precision == DDA_PREC_DF64)
    return fail(DDA_ERR_INVALID_ARG, "DDA_PREC_DF64 is not offered without allocation");
  dda_status s = check_kd(t, kd);
  if (s != DDA_OK) return s;
  const bool f32 = precision != DDA_PREC_FP64;
  const size_t elem = f32 ? sizeof(float2) : sizeof(double2);
  const size_t need = (size_t)3 * t->nz * t->Ly * t->Lx * elem;
  if (need > kStaticScratchBytes - kStaticAinvBytes) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "target needs %zu bytes of FFT scratch; the static area holds %zu "
             "(at most 3*nz*Ly*Lx complex values of the chosen precision)",
             need, kStaticScratchBytes - kStaticAinvBytes);
    return fail(DDA_ERR_INVALID_ARG, msg);
  }
  if (t->ncomp + 1 > 256) return fail(DDA_ERR_INVALID_ARG, "too many compositions");
  const int filtered = t->method == DDA_POL_FCD ? 1 : 0;
  if (!t->have_green || t->green_kd != kd || t->green_filtered != filtered || !t->kernels_configured)
    return fail(DDA_ERR_INVALID_ARG,
                "the Green-tensor transform for this kd and method is not built: call "
                "dda_matvec or dda_solve once with them first (building it allocates)");
  double kh[3] = {1, 0, 0};
  cd ev[3] = {0.0, 1.0, 0.0};
  s = incidence_of(t, khat, e, kh, ev);
  if (s != DDA_OK) return s;
  try {
    CK(cudaSetDevice(t->device));
    void* base = nullptr;
    CK(static_scratch_address(t->device, &base));  // resolved by dda_target_create
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : t->stream;
    unsigned char* area = reinterpret_cast<unsigned char*>(base);
    // alpha^{-1} per composition and lattice axis (entry 0 unused) at the
    // start of the area
    double2 ai64[3 * 256];
    float2 ai32[3 * 256];
    ainv_table(t, kd, kh, ev, ai64, ai32, nullptr);
    const size_t nai = (size_t)3 * (t->ncomp + 1);
    // the spectral scratch needs no clearing: every element the passes read was
    // written earlier in the same call
    if (f32) {
      CK(cudaMemcpyAsync(area, ai32, sizeof(float2) * nai, cudaMemcpyHostToDevice, st));
      OpView<float> op = make_view<float>(t, t->g32.p, area, t->tw32.p);
      CK(launch_matvec<float>(op, t->L32, 1, reinterpret_cast<const float2*>(x_dev),
                              reinterpret_cast<float2*>(y_dev),
                              reinterpret_cast<float2*>(area + kStaticAinvBytes), nullptr, st));
    } else {
      CK(cudaMemcpyAsync(area, ai64, sizeof(double2) * nai, cudaMemcpyHostToDevice, st));
      OpView<double> op = make_view<double>(t, t->g64.p, area, t->tw64.p);
      CK(launch_matvec<double>(op, t->L64, 1, reinterpret_cast<const double2*>(x_dev),
                               reinterpret_cast<double2*>(y_dev),
                               reinterpret_cast<double2*>(area + kStaticAinvBytes), nullptr,
                               st));
    }
    CK(cudaStreamSynchronize(st));
  } catch (const CudaFail& f) {
    return from_cuda(f);
  }
  return DDA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Orientation averages (Sec. "Orientational Averaging")
// ---------------------------------------------------------------------------
#include "scattering.h"

extern "C" {

dda_status dda_orient_average(dda_target* t, const dda_orient_params* p, dda_orient_result* r) {
  g_last_error.clear();
  if (!t || !p || !r) return fail(DDA_ERR_INVALID_ARG, "null argument");
  for (int a = 0; a < 3; ++a)
    if (p->n[a] < 1 || p->n[a] > 4096) return fail(DDA_ERR_INVALID_ARG, "NBETA, NTHETA, NPHI must be 1..4096");
  if (p->n_sel < 0 || (p->n_sel > 0 && !p->sel)) return fail(DDA_ERR_INVALID_ARG, "bad sel");
  if (p->max_rhs < 0) return fail(DDA_ERR_INVALID_ARG, "max_rhs must be >= 0");
  dda_status s = check_kd(t, p->kd);
  if (s != DDA_OK) return s;
  const double pi = 3.14159265358979323846;
  // incident polarization in the Lab Frame
  cd el[3] = {0.0, 1.0, 0.0};
  if (p->e01_lab)
    for (int c = 0; c < 3; ++c) el[c] = cd(p->e01_lab[2 * c], p->e01_lab[2 * c + 1]);
  double en = std::norm(el[0]) + std::norm(el[1]) + std::norm(el[2]);
  if (!(en > 0.0) || std::abs(el[0]) > 1e-6 * std::sqrt(en))
    return fail(DDA_ERR_INVALID_ARG, "e01_lab must be nonzero and transverse to x_LF");
  for (int c = 0; c < 3; ++c) el[c] /= std::sqrt(en);
  // orientations and weights
  const int nb = p->n[0], nt = p->n[1], np = p->n[2];
  std::vector<double> beta(nb), theta(nt), phi(np), wb(nb), wa((size_t)nt * np);
  dda::orientation_grid(p->range, p->n, beta.data(), theta.data(), phi.data(), wb.data(),
                        wa.data());
  struct Ori { double b, th, ph, w; };
  std::vector<Ori> ori;
  for (int ib = 0; ib < nb; ++ib)
    for (int it = 0; it < nt; ++it)
      for (int ip = 0; ip < np; ++ip)
        ori.push_back({beta[ib], theta[it], phi[ip], wb[ib] * wa[(size_t)it * np + ip]});
  // scattering directions: the averaging set, then the selected ones
  const double aeff = std::cbrt(3.0 * (double)t->N / (4.0 * pi));
  const double geo = pi * aeff * aeff;
  std::vector<double> sth, sph, som;
  if (p->eta > 0) {
    if (p->eta < 1e-3) return fail(DDA_ERR_INVALID_ARG, "eta must be >= 1e-3");
    dda::scattering_directions(p->kd * aeff, p->eta, sth, sph, som);
  }
  const int64_t nsca = (int64_t)sth.size();
  const int D = (int)nsca + p->n_sel;
  std::vector<double> dirs(2 * (size_t)D);
  for (int64_t i = 0; i < nsca; ++i) { dirs[2 * i] = sth[i]; dirs[2 * i + 1] = sph[i]; }
  for (int i = 0; i < p->n_sel; ++i) {
    dirs[2 * (nsca + i)] = p->sel[2 * i];
    dirs[2 * (nsca + i) + 1] = p->sel[2 * i + 1];
  }
  // accumulators
  double Qe[2] = {0, 0}, Qa[2] = {0, 0}, Qs[2] = {0, 0}, Qp[2] = {0, 0};
  double Qi[2] = {0, 0}, G[2][3] = {{0, 0, 0}, {0, 0, 0}}, C2[2] = {0, 0}, Qb[2] = {0, 0};
  std::vector<double> mu((size_t)16 * p->n_sel, 0.0);
  int64_t iters = 0;
  double tsolve = 0.0;
  dda_status worst = DDA_OK;
  const int per = p->max_rhs > 0 ? std::max(1, p->max_rhs / 2) : (int)ori.size();
  const double k2 = p->kd * p->kd;
  for (size_t o0 = 0; o0 < ori.size(); o0 += per) {
    const int ni = (int)std::min<size_t>(per, ori.size() - o0);
    std::vector<double> kh(3 * ni), yh(3 * ni), e1(6 * ni);
    for (int i = 0; i < ni; ++i) {
      double x[3], y[3], z[3];
      dda::lab_axes(ori[o0 + i].th, ori[o0 + i].ph, ori[o0 + i].b, x, y, z);
      for (int c = 0; c < 3; ++c) {
        kh[3 * i + c] = x[c];
        yh[3 * i + c] = y[c];
        const cd e = el[1] * y[c] + el[2] * z[c];
        e1[6 * i + 2 * c] = e.real();
        e1[6 * i + 2 * c + 1] = e.imag();
      }
    }
    dda_solve_params sp{};
    sp.kd = p->kd; sp.n_inc = ni; sp.khat = kh.data(); sp.yhat = yh.data(); sp.e01 = e1.data();
    sp.npol = 2; sp.tol = p->tol; sp.max_iter = p->max_iter; sp.precision = p->precision;
    sp.inner_tol = 0.0; sp.n_dirs = D; sp.dirs = D ? dirs.data() : nullptr; sp.P0 = nullptr;
    sp.profile = 0; sp.solver = p->solver;
    const int R = 2 * ni;
    std::vector<double> qe(R), qa(R), qs(R), fa((size_t)ni * (D + 1) * 2 * 2 * 2), rs(R);
    std::vector<int> it(R), sw(R);
    dda_solve_result sr{};
    sr.Qext = qe.data(); sr.Qabs = qa.data(); sr.Qsca = qs.data(); sr.famp = fa.data();
    sr.iters = it.data(); sr.resid = rs.data(); sr.sweeps = sw.data();
    s = dda_solve(t, &sp, &sr);
    if (s != DDA_OK && s != DDA_ERR_NOCONV) return s;
    if (worst == DDA_OK) worst = s;
    tsolve += sr.t_solve_ms;
    for (int i = 0; i < R; ++i) iters += it[i];
    // famp[i][d][m][l] complex
    auto F = [&](int i, int d, int m, int l) {
      const size_t o = ((((size_t)i * (D + 1) + d) * 2 + m) * 2 + l) * 2;
      return cd(fa[o], fa[o + 1]);
    };
    std::vector<cd> f1(nsca), f2(nsca);
    for (int i = 0; i < ni; ++i) {
      const double w = ori[o0 + i].w;
      for (int l = 0; l < 2; ++l) {
        const int rr = 2 * i + l;
        Qe[l] += w * qe[rr];
        Qa[l] += w * qa[rr];
        Qs[l] += w * qs[rr];
        Qp[l] += w * (2.0 * pi / k2) * F(i, 0, l, l).real() / geo;
        if (nsca) {
          for (int64_t d = 0; d < nsca; ++d) { f1[d] = F(i, 1 + (int)d, 0, l); f2[d] = F(i, 1 + (int)d, 1, l); }
          const dda::AngularAverages av = dda::angular_averages(
              nsca, f1.data(), f2.data(), sth.data(), sph.data(), som.data(), p->kd, aeff);
          Qi[l] += w * av.Qsca;
          for (int c = 0; c < 3; ++c) G[l][c] += w * av.Qsca * av.g[c];
          C2[l] += w * av.Qsca * av.cos2;
          Qb[l] += w * av.Qbk;
        }
      }
      for (int sidx = 0; sidx < p->n_sel; ++sidx) {
        cd ff[2][2], S4[4];
        for (int m = 0; m < 2; ++m)
          for (int l = 0; l < 2; ++l) ff[m][l] = F(i, 1 + (int)nsca + sidx, m, l);
        dda::amplitude_matrix(ff, el, p->sel[2 * sidx + 1], S4);
        double M[16];
        dda::mueller_matrix(S4, M);
        for (int q = 0; q < 16; ++q) mu[(size_t)16 * sidx + q] += w * M[q];
      }
    }
  }
  for (int l = 0; l < 2; ++l) {
    r->Qext[l] = Qe[l]; r->Qabs[l] = Qa[l]; r->Qsca[l] = Qs[l]; r->Qpha[l] = Qp[l];
    r->Qsca_int[l] = Qi[l];
    for (int c = 0; c < 3; ++c) r->g[l][c] = Qi[l] > 0 ? G[l][c] / Qi[l] : 0.0;
    r->cos2[l] = Qi[l] > 0 ? C2[l] / Qi[l] : 0.0;
    r->Qbk[l] = Qb[l];
  }
  if (r->mueller) std::copy(mu.begin(), mu.end(), r->mueller);
  r->n_orient = (int)ori.size();
  r->n_sca = nsca;
  r->iters = iters;
  r->t_solve_ms = tsolve;
  return worst;
}

}  // extern "C"
