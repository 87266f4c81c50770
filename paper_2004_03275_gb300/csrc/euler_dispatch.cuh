// Kernel launch wrappers; included after euler_kernels.cuh by each
// (type, dimension) translation unit.
#pragma once
#include "euler_ops.h"

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

// opt in to the 3D kernel's dynamic shared memory (outside any stream capture)
template <typename real, int ND, int B, int FLUX>
cudaError_t stage_prepare() {
  if constexpr (ND == 3)
    return cudaFuncSetAttribute(stage_kernel_3d<real, B, FLUX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(Stage3DSmem<real, B>));
  return cudaSuccess;
}

template <typename real, int ND, int B>
cudaError_t stage_b(int flux, const StageArgs<real>& a, const Geometry& G, cudaStream_t s) {
  switch (flux) {
    case FLUX_TVDLF: return stage_launch<real, ND, B, FLUX_TVDLF>(a, G, s);
    case FLUX_HLL: return stage_launch<real, ND, B, FLUX_HLL>(a, G, s);
    default: return stage_launch<real, ND, B, FLUX_HLLC>(a, G, s);
  }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

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
cudaError_t EulerOps<real, ND>::prepare(int B, int flux) {
#define CALL(BB)                                                                          \
  (flux == FLUX_TVDLF ? detail::stage_prepare<real, ND, BB, FLUX_TVDLF>()                \
                      : (flux == FLUX_HLL ? detail::stage_prepare<real, ND, BB, FLUX_HLL>() \
                                          : detail::stage_prepare<real, ND, BB, FLUX_HLLC>()))
  return AMRGPU_BSWITCH(B, CALL);
#undef CALL
}

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::reduce(int B, const real* U, const int* level, const Geometry& G, DevCtl* ctl,
                                       double* partials, int nleaves, int advance, cudaStream_t s) {
  if (nleaves == 0) return cudaSuccess;
#define CALL(BB)                                                                                   \
  ([&]() {                                                                                         \
    constexpr int NC = Tile<ND, BB>::NC;                                                           \
    constexpr int LPB = NC >= 256 ? 1 : 256 / NC;                                                  \
    reduce_kernel<real, ND, BB><<<(nleaves + LPB - 1) / LPB, 256, 0, s>>>(U, level, G, ctl, partials, \
                                                                         nleaves, advance);        \
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
    long long n = (long long)nslabs * (ND + 2) * 2 * Tile<ND, BB>::NT;                            \
    ghost_fill_kernel<real, ND, BB><<<detail::blocks_for(n, 256), 256, 0, s>>>(U, slabs, desc, nslabs); \
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

template <typename real, int ND>
cudaError_t EulerOps<real, ND>::lohner(int B, const real* U, const real* slabs, const int* nb, double gamma,
                                       double eps, unsigned mask, double* err, int nleaves, cudaStream_t s) {
  if (nleaves == 0) return cudaSuccess;
#define CALL(BB)                                                                                   \
  ([&]() {                                                                                         \
    constexpr int NC = Tile<ND, BB>::NC;                                                           \
    constexpr int LPB = NC >= 256 ? 1 : 256 / NC;                                                  \
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
  int nc = 1;
  for (int d = 0; d < ND; ++d) nc *= B;
  long long n = nleaves * nc;
  if (n == 0) return cudaSuccess;
  set_state_kernel<real, ND><<<detail::blocks_for(n, 256), 256, 0, s>>>(W, U, n, nc, primitive, gamma);
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
