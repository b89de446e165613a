// FP32 FFT-matvec passes compiled for fixed radix plans (fft_plan.cuh): the
// plans of the grid lengths 64 = 16x4, 128 = 16x8 and 512 = 16x8x4 and those
// of the 48x96x144 ellipsoid's grid, 96 = 8x4x3 (x), 192 = 16x4x3 (y) and
// 288 = 8x4x3x3 (z).  The variants live in their own translation unit so the
// build compiles them in parallel with the generic kernels; any other plan,
// tile or precision takes the generic kernels.
#include <cstring>
#include <type_traits>

#include "matvec_impl.cuh"
#include "zpass_pair.cuh"

namespace dda {

namespace {

using P16x4 = FixedPlan<16, 4>;
using P16x8 = FixedPlan<16, 8>;
using P16x8x4 = FixedPlan<16, 8, 4>;
using P8x4x3 = FixedPlan<8, 4, 3>;
using P16x4x3 = FixedPlan<16, 4, 3>;
using P8x4x3x3 = FixedPlan<8, 4, 3, 3>;

template <class P> bool is_plan(const AxisPlan& a) {
  if (a.nstage != P::NS || a.L != P::L) return false;
  for (int t = 0; t < P::NS; ++t)
    if (a.radix[t] != P::radix(t)) return false;
  return true;
}

template <class... Ps> struct PlanList {};

template <class F, class P, class... Ps>
bool dispatch_plan(const AxisPlan& a, PlanList<P, Ps...>, F&& f) {
  if (is_plan<P>(a)) {
    f(P{});
    return true;
  }
  if constexpr (sizeof...(Ps) > 0) return dispatch_plan(a, PlanList<Ps...>{}, f);
  else return false;
}

using XPlans = PlanList<P16x8, P16x4, P16x8x4, P8x4x3>;
using YPlans = PlanList<P16x8, P16x4, P16x8x4, P16x4x3>;
using ZPlans = PlanList<P16x8, P16x4, P16x8x4, P8x4x3x3>;

template <int V> using IC = std::integral_constant<int, V>;

// z tiles compiled per plan: every tile for two-stage plans, 4 and 8 otherwise
template <class P> constexpr bool z_tile_compiled(int tile) {
  return P::NS == 2 ? (tile == 2 || tile == 4 || tile == 8 || tile == 16)
                    : (tile == 4 || tile == 8);
}

template <class P, class F> void for_z_variants(F&& f) {
  if constexpr (P::NS == 2) {
    f(IC<2>{}, IC<0>{}); f(IC<2>{}, IC<1>{});
    f(IC<16>{}, IC<0>{}); f(IC<16>{}, IC<1>{});
  }
  f(IC<4>{}, IC<0>{}); f(IC<4>{}, IC<1>{});
  f(IC<8>{}, IC<0>{}); f(IC<8>{}, IC<1>{});
}

template <class F> void for_y_variants(F&& f) {
  f(IC<8>{}, IC<0>{}); f(IC<16>{}, IC<0>{}); f(IC<32>{}, IC<0>{});
  f(IC<8>{}, IC<1>{}); f(IC<16>{}, IC<1>{}); f(IC<32>{}, IC<1>{});
}

cudaError_t set_smem(const void* k) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace

bool z_fixed_plan(const AxisPlan& a) {
  return dispatch_plan(a, ZPlans{}, [](auto) {});
}

bool z_fixed_applies(const AxisPlan& a, int tile) {
  bool ok = false;
  dispatch_plan(a, ZPlans{}, [&](auto plan) { ok = z_tile_compiled<decltype(plan)>(tile); });
  return ok;
}

// the column-pair z kernel's own plans (radices <= 8; twiddles in op.twz_pair)
using QP64 = FixedPlan<8, 8>;
using QP128 = FixedPlan<8, 4, 4>;
using QP288 = FixedPlan<8, 4, 3, 3>;
using QP512 = FixedPlan<8, 8, 8>;
using PairPlans = PlanList<QP64, QP128, QP288, QP512>;

template <class F, class P, class... Ps>
bool dispatch_length(int L, PlanList<P, Ps...>, F&& f) {
  if (L == P::L) {
    f(P{});
    return true;
  }
  if constexpr (sizeof...(Ps) > 0) return dispatch_length(L, PlanList<Ps...>{}, f);
  else return false;
}

bool z_pair_applies(int Lz, int Lx, int tile) {
  return (tile == 4 || tile == 8) && Lx % 2 == 0 &&
         dispatch_length(Lz, PairPlans{}, [](auto) {});
}

size_t zpair_smem_bytes(int Lz, int tile, bool gs) {
  return (size_t)zpair_row(Lz, Lz, tile) * sizeof(float4) +
         (gs ? (size_t)tile * zpair_gstride(Lz / 2 + 1, tile) * sizeof(float2) : 0);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library links the runtime only); resolved once.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

bool z_pair_tma_applies(int Lz, int Lx, int nz, int tile) {
  return z_pair_applies(Lz, Lx, tile) && nz <= 256 && 2 * nz <= Lz && encode_fn() != nullptr;
}

bool encode_zpair_map(CUtensorMap* map, const float2* scratch, int Lx, int Ly, int nz, int R,
                      int tile) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || ((uintptr_t)scratch & 15) || Lx % 2) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)Lx, (cuuint64_t)Ly, (cuuint64_t)nz, (cuuint64_t)3 * R};
  const cuuint64_t strides[3] = {(cuuint64_t)Lx * 8, (cuuint64_t)Ly * Lx * 8,
                                 (cuuint64_t)nz * Ly * Lx * 8};
  const cuuint32_t box[4] = {(cuuint32_t)tile, 1, (cuuint32_t)nz, 3};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<float2*>(scratch), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool launch_z_fixed(const OpView<float>& op, const MatvecLaunch& L, int R, float2* scratch,
                    const int* active, cudaStream_t st) {
  bool done = false;
  if (L.z_pair) {
    if (!z_pair_applies(op.Lz, op.Lx, L.z_tile) || !op.twz_pair) return false;
    dispatch_length(op.Lz, PairPlans{}, [&](auto plan) {
      using P = decltype(plan);
      constexpr int NT = kZPairThreads;
      const dim3 gz((op.Lx + L.z_tile - 1) / L.z_tile, op.Ly / 2 + 1);
      CUtensorMap map;
      std::memset(&map, 0, sizeof map);
      const bool tma = L.z_pair == 2 && z_pair_tma_applies(op.Lz, op.Lx, op.nz, L.z_tile) &&
                       encode_zpair_map(&map, scratch, op.Lx, op.Ly, op.nz, R, L.z_tile);
      auto go = [&](auto tile) {
        constexpr int TT = decltype(tile)::value;
        if (tma) {
          if (L.z_gs)
            k_fft_z_pairs<TT, P, true, NT, true><<<gz, NT, zpair_smem<TT, P, true>(), st>>>(
                op, scratch, R, active, map);
          else
            k_fft_z_pairs<TT, P, false, NT, true><<<gz, NT, zpair_smem<TT, P, false>(), st>>>(
                op, scratch, R, active, map);
        } else {
          if (L.z_gs)
            k_fft_z_pairs<TT, P, true, NT, false><<<gz, NT, zpair_smem<TT, P, true>(), st>>>(
                op, scratch, R, active, map);
          else
            k_fft_z_pairs<TT, P, false, NT, false><<<gz, NT, zpair_smem<TT, P, false>(), st>>>(
                op, scratch, R, active, map);
        }
        done = true;
      };
      if (L.z_tile == 4) go(IC<4>{});
      else go(IC<8>{});
    });
    return done;
  }
  dispatch_plan(op.pz, ZPlans{}, [&](auto plan) {
    using P = decltype(plan);
    if (!z_tile_compiled<P>(L.z_tile)) return;
    const dim3 gz((op.Lx + L.z_tile - 1) / L.z_tile, op.Ly, R);
    for_z_variants<P>([&](auto tile, auto gs) {
      constexpr int TT = decltype(tile)::value;
      constexpr bool GG = decltype(gs)::value != 0;
      if (done || TT != L.z_tile || GG != L.z_gs) return;
      k_fft_z_mul_p<TT, GG, P><<<gz, L.z_threads, zp_smem<TT, GG>(op), st>>>(op, scratch,
                                                                            active);
      done = true;
    });
  });
  return done;
}

bool launch_y_fixed(bool inv, const OpView<float>& op, const MatvecLaunch& L, int R,
                    float2* scratch, const int* active, cudaStream_t st) {
  bool done = false;
  dispatch_plan(op.py, YPlans{}, [&](auto plan) {
    using P = decltype(plan);
    const dim3 gy((op.Lx + L.y_tile - 1) / L.y_tile, 3 * op.nz, R);
    for_y_variants([&](auto tile, auto iv) {
      constexpr int TT = decltype(tile)::value;
      constexpr bool INV = decltype(iv)::value != 0;
      if (done || TT != L.y_tile || INV != inv) return;
      k_fft_y_p<TT, INV, P><<<gy, L.y_threads, L.y_smem, st>>>(op, scratch, active);
      done = true;
    });
  });
  return done;
}

template <int XIN>
bool launch_x_fwd_fixed(const OpView<float>& op, const MatvecLaunch& L, int R, const float2* x,
                        float2* scratch, const int* active, XinArgs<float> xa, cudaStream_t st) {
  return dispatch_plan(op.px, XPlans{}, [&](auto plan) {
    using P = decltype(plan);
    const int rows = 3 * op.nz * op.ny;
    const dim3 gx((rows + L.x_lines - 1) / L.x_lines, R);
    k_fft_x_fwd<float, XIN, P><<<gx, L.x_threads, L.x_smem, st>>>(
        op, x, scratch, L.x_lines, div_magic(L.x_lines), active, xa);
  });
}

template <int XOUT>
bool launch_x_inv_fixed(const OpView<float>& op, const MatvecLaunch& L, int R,
                        const float2* scratch, const float2* x, float2* y, const int* active,
                        const float2* rhat, double* partials, cudaStream_t st, FoldArgs fold) {
  return dispatch_plan(op.px, XPlans{}, [&](auto plan) {
    using P = decltype(plan);
    const int rows = 3 * op.nz * op.ny;
    const dim3 gx((rows + L.x_lines - 1) / L.x_lines, R);
    k_fft_x_inv<float, XOUT, P><<<gx, L.x_threads, L.xinv_smem, st>>>(
        op, scratch, x, y, L.x_lines, div_magic(L.x_lines), active, rhat, partials, fold);
  });
}

template bool launch_x_fwd_fixed<XIN_PLAIN>(const OpView<float>&, const MatvecLaunch&, int,
                                            const float2*, float2*, const int*, XinArgs<float>,
                                            cudaStream_t);
template bool launch_x_fwd_fixed<XIN_P>(const OpView<float>&, const MatvecLaunch&, int,
                                        const float2*, float2*, const int*, XinArgs<float>,
                                        cudaStream_t);
template bool launch_x_fwd_fixed<XIN_S>(const OpView<float>&, const MatvecLaunch&, int,
                                        const float2*, float2*, const int*, XinArgs<float>,
                                        cudaStream_t);
template bool launch_x_fwd_fixed<XIN_Q>(const OpView<float>&, const MatvecLaunch&, int,
                                        const float2*, float2*, const int*, XinArgs<float>,
                                        cudaStream_t);
#define DDA_XINV(M)                                                                             \
  template bool launch_x_inv_fixed<M>(const OpView<float>&, const MatvecLaunch&, int,          \
                                      const float2*, const float2*, float2*, const int*,      \
                                      const float2*, double*, cudaStream_t, FoldArgs);
DDA_XINV(XOUT_PLAIN)
DDA_XINV(XOUT_RV)
DDA_XINV(XOUT_TS)
DDA_XINV(XOUT_QT)
#undef DDA_XINV

cudaError_t configure_fixed_kernels() {
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  auto zcfg = [&](auto plan) {
    using P = decltype(plan);
    for_z_variants<P>([&](auto tile, auto gs) {
      constexpr int TT = decltype(tile)::value;
      constexpr bool GG = decltype(gs)::value != 0;
      ok(set_smem((const void*)k_fft_z_mul_p<TT, GG, P>));
    });
  };
  zcfg(P16x8{}); zcfg(P16x4{}); zcfg(P16x8x4{}); zcfg(P8x4x3x3{});
  auto zpcfg = [&](auto plan) {
    using P = decltype(plan);
    constexpr int NT = kZPairThreads;
    ok(set_smem((const void*)k_fft_z_pairs<4, P, false, NT, false>));
    ok(set_smem((const void*)k_fft_z_pairs<8, P, false, NT, false>));
    ok(set_smem((const void*)k_fft_z_pairs<4, P, true, NT, false>));
    ok(set_smem((const void*)k_fft_z_pairs<8, P, true, NT, false>));
    ok(set_smem((const void*)k_fft_z_pairs<4, P, false, NT, true>));
    ok(set_smem((const void*)k_fft_z_pairs<8, P, false, NT, true>));
    ok(set_smem((const void*)k_fft_z_pairs<4, P, true, NT, true>));
    ok(set_smem((const void*)k_fft_z_pairs<8, P, true, NT, true>));
  };
  zpcfg(QP64{}); zpcfg(QP128{}); zpcfg(QP288{}); zpcfg(QP512{});
  auto ycfg = [&](auto plan) {
    using P = decltype(plan);
    for_y_variants([&](auto tile, auto iv) {
      constexpr int TT = decltype(tile)::value;
      constexpr bool INV = decltype(iv)::value != 0;
      ok(set_smem((const void*)k_fft_y_p<TT, INV, P>));
    });
  };
  ycfg(P16x8{}); ycfg(P16x4{}); ycfg(P16x8x4{}); ycfg(P16x4x3{});
  auto xcfg = [&](auto plan) {
    using P = decltype(plan);
    ok(set_smem((const void*)k_fft_x_fwd<float, XIN_PLAIN, P>));
    ok(set_smem((const void*)k_fft_x_fwd<float, XIN_P, P>));
    ok(set_smem((const void*)k_fft_x_fwd<float, XIN_S, P>));
    ok(set_smem((const void*)k_fft_x_fwd<float, XIN_Q, P>));
    ok(set_smem((const void*)k_fft_x_inv<float, XOUT_PLAIN, P>));
    ok(set_smem((const void*)k_fft_x_inv<float, XOUT_RV, P>));
    ok(set_smem((const void*)k_fft_x_inv<float, XOUT_TS, P>));
    ok(set_smem((const void*)k_fft_x_inv<float, XOUT_QT, P>));
  };
  xcfg(P16x8{}); xcfg(P16x4{}); xcfg(P16x8x4{}); xcfg(P8x4x3{});
  return e;
}

}  // namespace dda
