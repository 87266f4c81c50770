// Kernel launch wrappers; included after euler_kernels.cuh by each
// (type, dimension) translation unit.
#pragma once
#include <type_traits>

#include "euler_ops.h"
#include "stage2d_f32.cuh"
#include "stage2d_march.cuh"
#include "stage3d_march.cuh"

namespace amrgpu {

namespace detail {

template <int ND, int B>
constexpr int stage_threads() { return ND == 1 ? 128 : 256; }

template <typename real, int ND, int B, int FLUX>
cudaError_t stage_launch(const StageArgs<real>& a, const Geometry& G, cudaStream_t s) {
  if (a.nleaves == 0) return cudaSuccess;
  if constexpr (ND == 3) {
    constexpr int LPB = 256 / (B * B);
    size_t smem = sizeof(Stage3DSmem<real, B>);
    int grid = (a.nleaves + LPB - 1) / LPB;
    stage_kernel_3d<real, B, FLUX><<<grid, 256, smem, s>>>(a, G);
  } else {
    constexpr int T = stage_threads<ND, B>();
    constexpr int NC = ND == 1 ? B : B * B;
    constexpr int LPB = T / NC;
    int grid = (a.nleaves + LPB - 1) / LPB;
    stage_kernel_12<real, ND, B, FLUX><<<grid, T, 0, s>>>(a, G);
  }
  return cudaGetLastError();
}

// persistent grid: resident CTAs per SM x SMs, computed once per kernel outside any capture
template <int B, int FLUX, int LIM>
int& stage2d_f32_grid() {
  static int g = 0;
  return g;
}

// march kernel (16^2 leaves): resident CTAs x SMs per stage kind and warps per CTA (2, 4, 8)
template <int FLUX, int LIM>
int (&march_caps())[3][3] {
  static int c[3][3] = {};
  return c;
}
constexpr int march_nw_index(int nw) { return nw == 2 ? 0 : (nw == 4 ? 1 : 2); }
constexpr size_t march_smem(int nw) { return (size_t)nw * sizeof(MarchSmem) + 128; }

template <int FLUX, int LIM, int SK, bool P>
cudaError_t march_prepare_kind(int sms) {
  cudaError_t e = cudaFuncSetAttribute(stage2d_march_kernel<FLUX, LIM, SK, P>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march_smem(kMarchMaxWarps));
  if constexpr (P) {  // resident-CTA counts (one CTA per leaf group otherwise: none needed)
    for (int nw : {2, 4, 8}) {
      int per = 0;
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, stage2d_march_kernel<FLUX, LIM, SK, P>, 32 * nw,
                                                          march_smem(nw));
      march_caps<FLUX, LIM>()[SK][march_nw_index(nw)] = sms * (per > 0 ? per : 1);
    }
  }
  return e;
}

template <int B, int FLUX, int LIM>
cudaError_t stage2d_f32_prepare_one() {
  int dev, sms, per;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if constexpr (B == 16) {  // dynamic shared memory and resident-CTA counts of the march kernels
    if (e == cudaSuccess) e = march_prepare_kind<FLUX, LIM, kStageFirst, false>(sms);
    if (e == cudaSuccess) e = march_prepare_kind<FLUX, LIM, kStageFirst, true>(sms);
    if (e == cudaSuccess) e = march_prepare_kind<FLUX, LIM, kStageMid, false>(sms);
    if (e == cudaSuccess) e = march_prepare_kind<FLUX, LIM, kStageMid, true>(sms);
    if (e == cudaSuccess) e = march_prepare_kind<FLUX, LIM, kStageLast, true>(sms);
  } else if (e == cudaSuccess) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, stage2d_f32_kernel<B, FLUX, LIM>, 256, 0);
    if (e == cudaSuccess) stage2d_f32_grid<B, FLUX, LIM>() = sms * (per > 0 ? per : 1);
  }
  return e;
}

template <int B, int FLUX>
cudaError_t stage2d_f32_prepare(int lim) {
  switch (lim) {
    case LIM_MINMOD: return stage2d_f32_prepare_one<B, FLUX, LIM_MINMOD>();
    case LIM_VANLEER: return stage2d_f32_prepare_one<B, FLUX, LIM_VANLEER>();
    case LIM_KOREN: return stage2d_f32_prepare_one<B, FLUX, LIM_KOREN>();
    case LIM_MC: return stage2d_f32_prepare_one<B, FLUX, LIM_MC>();
    case LIM_CADA: return stage2d_f32_prepare_one<B, FLUX, LIM_CADA>();
    default: return stage2d_f32_prepare_one<B, FLUX, LIM_NONE>();
  }
}

template <int B, int FLUX, int LIM>
void stage2d_f32_go(const StageArgs<float>& a, const Geometry& G, cudaStream_t s) {
  if constexpr (B == 16) {
    const int kind = a.fuse_reduce ? kStageLast : (a.stage1 ? kStageFirst : kStageMid);
    const int nw = kind == kStageLast ? kMarchWarps : (a.march_nw == 2 || a.march_nw == 8 ? a.march_nw : 4);
    const bool persist = a.march_persist > 0;
    const int ngroups = (a.nleaves + nw - 1) / nw;
    const int cap = march_caps<FLUX, LIM>()[kind][march_nw_index(nw)];
    const int grid = persist && cap > 0 && cap < ngroups ? cap : ngroups;
    const CUtensorMap& tm = *static_cast<const CUtensorMap*>(a.tmap_us);
    if (kind == kStageLast)
      stage2d_march_kernel<FLUX, LIM, kStageLast, true><<<grid, 32 * nw, march_smem(nw), s>>>(a, G, tm);
    else if (kind == kStageFirst && persist)
      stage2d_march_kernel<FLUX, LIM, kStageFirst, true><<<grid, 32 * nw, march_smem(nw), s>>>(a, G, tm);
    else if (kind == kStageFirst)
      stage2d_march_kernel<FLUX, LIM, kStageFirst, false><<<grid, 32 * nw, march_smem(nw), s>>>(a, G, tm);
    else if (persist)
      stage2d_march_kernel<FLUX, LIM, kStageMid, true><<<grid, 32 * nw, march_smem(nw), s>>>(a, G, tm);
    else
      stage2d_march_kernel<FLUX, LIM, kStageMid, false><<<grid, 32 * nw, march_smem(nw), s>>>(a, G, tm);
    return;
  }
  constexpr int LPB = 256 / (B * B);
  int nslots = (a.nleaves + LPB - 1) / LPB;
  int cap = stage2d_f32_grid<B, FLUX, LIM>();
  int grid = cap > 0 && cap < nslots ? cap : nslots;
  stage2d_f32_kernel<B, FLUX, LIM><<<grid, 256, 0, s>>>(a, G);
}

template <int B, int FLUX>
cudaError_t stage2d_f32_launch(const StageArgs<float>& a, const Geometry& G, cudaStream_t s) {
  if (B == 16 && !a.tmap_us) return cudaErrorInvalidValue;  // the march kernel needs the state's tensor map
  switch (a.limiter) {
    case LIM_MINMOD: stage2d_f32_go<B, FLUX, LIM_MINMOD>(a, G, s); break;
    case LIM_VANLEER: stage2d_f32_go<B, FLUX, LIM_VANLEER>(a, G, s); break;
    case LIM_KOREN: stage2d_f32_go<B, FLUX, LIM_KOREN>(a, G, s); break;
    case LIM_MC: stage2d_f32_go<B, FLUX, LIM_MC>(a, G, s); break;
    case LIM_CADA: stage2d_f32_go<B, FLUX, LIM_CADA>(a, G, s); break;
    default: stage2d_f32_go<B, FLUX, LIM_NONE>(a, G, s); break;
  }
  return cudaGetLastError();
}

// float32 3D, 16^3 leaves: xy pass (4 CTAs of 4 warps per leaf), then z pass (kZRows rows of
// the leaf per CTA; 4 with the fused reduction).  Rows per CTA measured on the blast step:
// 2 rows (6 CTAs of 2 warps per SM) 0.74 ms, 4 rows (3 CTAs of 4 warps) 0.70 ms.
constexpr int kZRows = 4;

template <int FLUX, int LIM>
void stage3d_f32_go(const StageArgs<float>& a, const Geometry& G, cudaStream_t s) {
  const int grid = a.nleaves * 4;
  stage3d_xy_kernel<FLUX, LIM><<<grid, 128, kXy3Smem, s>>>(a, G);
  if (a.fuse_reduce)
    stage3d_z_kernel<FLUX, LIM, true><<<grid, 128, kZSmem, s>>>(a, G);
  else
    stage3d_z_kernel<FLUX, LIM, false, kZRows>
        <<<a.nleaves * (16 / kZRows), 32 * kZRows, ZGeom<kZRows>::Smem, s>>>(a, G);
}

template <int FLUX>
cudaError_t stage3d_f32_launch(const StageArgs<float>& a, const Geometry& G, cudaStream_t s) {
  switch (a.limiter) {
    case LIM_MINMOD: stage3d_f32_go<FLUX, LIM_MINMOD>(a, G, s); break;
    case LIM_VANLEER: stage3d_f32_go<FLUX, LIM_VANLEER>(a, G, s); break;
    case LIM_KOREN: stage3d_f32_go<FLUX, LIM_KOREN>(a, G, s); break;
    case LIM_MC: stage3d_f32_go<FLUX, LIM_MC>(a, G, s); break;
    case LIM_CADA: stage3d_f32_go<FLUX, LIM_CADA>(a, G, s); break;
    default: stage3d_f32_go<FLUX, LIM_NONE>(a, G, s); break;
  }
  return cudaGetLastError();
}

template <int FLUX, int LIM>
cudaError_t stage3d_z_prepare() {
  cudaError_t e = cudaFuncSetAttribute(stage3d_z_kernel<FLUX, LIM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kZSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stage3d_z_kernel<FLUX, LIM, false, kZRows>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ZGeom<kZRows>::Smem);
  return e;
}

template <int FLUX>
cudaError_t stage3d_f32_prepare(int lim) {
  cudaError_t e = lim == LIM_MINMOD    ? stage3d_z_prepare<FLUX, LIM_MINMOD>()
                  : lim == LIM_VANLEER ? stage3d_z_prepare<FLUX, LIM_VANLEER>()
                  : lim == LIM_KOREN   ? stage3d_z_prepare<FLUX, LIM_KOREN>()
                  : lim == LIM_MC      ? stage3d_z_prepare<FLUX, LIM_MC>()
                  : lim == LIM_CADA    ? stage3d_z_prepare<FLUX, LIM_CADA>()
                                       : stage3d_z_prepare<FLUX, LIM_NONE>();
  if (e != cudaSuccess) return e;
  switch (lim) {
    case LIM_MINMOD:
      return cudaFuncSetAttribute(stage3d_xy_kernel<FLUX, LIM_MINMOD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kXy3Smem);
    case LIM_VANLEER:
      return cudaFuncSetAttribute(stage3d_xy_kernel<FLUX, LIM_VANLEER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kXy3Smem);
    case LIM_KOREN:
      return cudaFuncSetAttribute(stage3d_xy_kernel<FLUX, LIM_KOREN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kXy3Smem);
    case LIM_MC:
      return cudaFuncSetAttribute(stage3d_xy_kernel<FLUX, LIM_MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kXy3Smem);
    case LIM_CADA:
      return cudaFuncSetAttribute(stage3d_xy_kernel<FLUX, LIM_CADA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kXy3Smem);
    default:
      return cudaFuncSetAttribute(stage3d_xy_kernel<FLUX, LIM_NONE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kXy3Smem);
  }
}

// opt in to the 3D kernel's dynamic shared memory (outside any stream capture)
template <typename real, int ND, int B, int FLUX>
cudaError_t stage_prepare(int lim) {
  if constexpr (std::is_same<real, float>::value && ND == 2) return stage2d_f32_prepare<B, FLUX>(lim);
  if constexpr (ND == 3) {
    if constexpr (std::is_same<real, float>::value && B == 16) {
      cudaError_t e = stage3d_f32_prepare<FLUX>(lim);
      if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(stage_kernel_3d<real, B, FLUX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(Stage3DSmem<real, B>));
  }
  return cudaSuccess;
}

template <typename real, int ND, int B>
cudaError_t stage_b(int flux, const StageArgs<real>& a, const Geometry& G, cudaStream_t s) {
  if constexpr (std::is_same<real, float>::value && ND == 2) {
    if (a.nleaves == 0) return cudaSuccess;
    switch (flux) {
      case FLUX_TVDLF: return stage2d_f32_launch<B, FLUX_TVDLF>(a, G, s);
      case FLUX_HLL: return stage2d_f32_launch<B, FLUX_HLL>(a, G, s);
      default: return stage2d_f32_launch<B, FLUX_HLLC>(a, G, s);
    }
  }
  if constexpr (std::is_same<real, float>::value && ND == 3 && B == 16) {
    if (a.nleaves == 0) return cudaSuccess;
    switch (flux) {
      case FLUX_TVDLF: return stage3d_f32_launch<FLUX_TVDLF>(a, G, s);
      case FLUX_HLL: return stage3d_f32_launch<FLUX_HLL>(a, G, s);
      default: return stage3d_f32_launch<FLUX_HLLC>(a, G, s);
    }
  }
  switch (flux) {
    case FLUX_TVDLF: return stage_launch<real, ND, B, FLUX_TVDLF>(a, G, s);
    case FLUX_HLL: return stage_launch<real, ND, B, FLUX_HLL>(a, G, s);
    default: return stage_launch<real, ND, B, FLUX_HLLC>(a, G, s);
  }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }
// resident CTAs of the float32 reduction walk: 3 per SM of the current device
inline int reduce_ctas() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      n = 3 * sms;
    else
      n = 3 * 152;
  }
  return n;
}

}  // namespace detail

#define AMRGPU_BSWITCH(B, CALL) ((B) == 16 ? CALL(16) : CALL(8))

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::stage(int B, int flux, const StageArgs<real>& a, const Geometry& G,
                                      cudaStream_t s) {
#define CALL(BB) detail::stage_b<real, ND, BB>(flux, a, G, s)
  return AMRGPU_BSWITCH(B, CALL);
#undef CALL
}

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::prepare(int B, int flux, int lim) {
#define CALL(BB)                                                                             \
  (flux == FLUX_TVDLF ? detail::stage_prepare<real, ND, BB, FLUX_TVDLF>(lim)                \
                      : (flux == FLUX_HLL ? detail::stage_prepare<real, ND, BB, FLUX_HLL>(lim) \
                                          : detail::stage_prepare<real, ND, BB, FLUX_HLLC>(lim)))
  return AMRGPU_BSWITCH(B, CALL);
#undef CALL
}

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::reduce(int B, const real* U, const int* level, const Geometry& G, DevCtl* ctl,
                                       double* partials, double* gpart, unsigned* gcount, int nleaves,
                                       int advance, cudaStream_t s) {
  if (nleaves == 0) return cudaSuccess;
#define CALL(BB)                                                                                   \
  ([&]() {                                                                                         \
    constexpr int NC = Tile<ND, BB>::NC;                                                           \
    constexpr int LPB = ReduceShape<NC>::LPB;                                                      \
    if constexpr (sizeof(real) == 4 && NC % 1024 == 0)                                             \
      reduce_split_kernel<ND, BB><<<std::min(nleaves * (NC / 1024), detail::reduce_ctas()), 256, 0, s>>>( \
          reinterpret_cast<const float*>(U), level, G, ctl, partials, gpart, gcount, nleaves, advance); \
    else                                                                                           \
      reduce_kernel<real, ND, BB><<<(nleaves + LPB - 1) / LPB, 256, 0, s>>>(U, level, G, ctl, partials, \
                                                                           gpart, gcount, nleaves, advance); \
    return cudaGetLastError();                                                                     \
  }())
  return AMRGPU_BSWITCH(B, CALL);
#undef CALL
}

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::ghost_fill(int B, const real* U, real* slabs, const SlabDesc* desc, int nslabs,
                                           cudaStream_t s) {
  if (nslabs == 0) return cudaSuccess;
#define CALL(BB)                                                                                  \
  ([&]() {                                                                                        \
    ghost_fill_kernel<real, ND, BB><<<nslabs, GhostShape<ND, BB>::THREADS, 0, s>>>(U, slabs, desc, nslabs); \
    return cudaGetLastError();                                                                    \
  }())
  return AMRGPU_BSWITCH(B, CALL);
#undef CALL
}

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::reflux(int B, real* out, const real* fflux, const RefluxRec* rec, int nrec,
                                       const int* level, const Geometry& G, const DevCtl* ctl, real beta,
                                       cudaStream_t s) {
  if (nrec == 0) return cudaSuccess;
#define CALL(BB)                                                                                   \
  ([&]() {                                                                                         \
    long long n = (long long)nrec * (ND + 2) * Tile<ND, BB>::NT;                                   \
    reflux_kernel<real, ND, BB><<<detail::blocks_for(n, 256), 256, 0, s>>>(out, fflux, rec, nrec, level, G, \
                                                                           ctl, beta);             \
    return cudaGetLastError();                                                                     \
  }())
  return AMRGPU_BSWITCH(B, CALL);
#undef CALL
}

// shared memory of the staged estimator for the selected variables, 0 where it does not apply
// (1D, or more than 200 KB)
template <typename real, int ND, int B>
size_t lohner_tile_smem(unsigned mask) {
  if constexpr (ND < 2) {
    return 0;
  } else {
    int nsel = 0;
    for (int v = 0; v < ND + 2; ++v) nsel += (mask >> v) & 1u;
    size_t pt = ND == 2 ? (size_t)(B + 2) * (B + 2) : (size_t)(B + 2) * (B + 2) * (B + 2);
    size_t bytes = (size_t)nsel * pt * sizeof(real);
    return nsel > 0 && bytes <= 200 * 1024 ? bytes : 0;
  }
}

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::lohner(int B, const real* U, const real* slabs, const int* nb, double gamma,
                                       double eps, unsigned mask, double* err, int nleaves, cudaStream_t s) {
  if (nleaves == 0) return cudaSuccess;
#define CALL(BB)                                                                                   \
  ([&]() {                                                                                         \
    constexpr int NC = Tile<ND, BB>::NC;                                                           \
    constexpr int LPB = NC >= 256 ? 1 : 256 / NC;                                                  \
    const size_t smem = lohner_tile_smem<real, ND, BB>(mask);                                            \
    if constexpr (ND >= 2) if (smem > 0) {                                                         \
      if (smem > 48 * 1024) {                                                                      \
        cudaError_t e = cudaFuncSetAttribute(lohner_tile_kernel<real, ND, BB>,                     \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                            \
      }                                                                                            \
      lohner_tile_kernel<real, ND, BB><<<nleaves, 256, smem, s>>>(U, slabs, nb, gamma, eps, mask, err, nleaves); \
      return cudaGetLastError();                                                                   \
    }                                                                                              \
    lohner_kernel<real, ND, BB><<<(nleaves + LPB - 1) / LPB, 256, 0, s>>>(U, slabs, nb, gamma, eps, mask, err, \
                                                                         nleaves);                 \
    return cudaGetLastError();                                                                     \
  }())
  return AMRGPU_BSWITCH(B, CALL);
#undef CALL
}

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::regrid(int B, const real* Uold, real* Unew, const real* slabs, const int* nb,
                                       const RegridOp* ops, int nnew, cudaStream_t s) {
  if (nnew == 0) return cudaSuccess;
#define CALL(BB)                                                                                   \
  ([&]() {                                                                                         \
    long long n = (long long)nnew * Tile<ND, BB>::NC;                                              \
    regrid_kernel<real, ND, BB><<<detail::blocks_for(n, 256), 256, 0, s>>>(Uold, Unew, slabs, nb, ops, nnew); \
    return cudaGetLastError();                                                                     \
  }())
  return AMRGPU_BSWITCH(B, CALL);
#undef CALL
}

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::set_state(int B, const double* W, real* U, long long nleaves, int primitive,
                                          double gamma, cudaStream_t s) {
  int lognc = 0;
  while ((1 << lognc) < B) ++lognc;  // block sizes are powers of two
  lognc *= ND;
  long long n = nleaves << lognc;
  if (n == 0) return cudaSuccess;
  set_state_kernel<real, ND><<<detail::blocks_for(n / 2, 256), 256, 0, s>>>(W, U, n, lognc, primitive, gamma);
  return cudaGetLastError();
}

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::read_state(const real* U, double* out, long long n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  read_state_kernel<real><<<detail::blocks_for(n, 256), 256, 0, s>>>(U, out, n);
  return cudaGetLastError();
}

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::face_ghosts(int B, const real* U, const real* slabs, const int* nb, int leaf,
                                            double* out, cudaStream_t s) {
#define CALL(BB)                                                                                   \
  ([&]() {                                                                                         \
    int n = (ND + 2) * 2 * ND * 2 * Tile<ND, BB>::NT;                                             \
    face_ghost_dump_kernel<real, ND, BB><<<detail::blocks_for(n, 256), 256, 0, s>>>(U, slabs, nb, leaf, out); \
    return cudaGetLastError();                                                                     \
  }())
  return AMRGPU_BSWITCH(B, CALL);
#undef CALL
}

}  // namespace amrgpu
