// Launch wrappers of the Euler device code, one explicit instantiation per
// (arithmetic type, dimension) translation unit.  Host code includes only this.
#pragma once
#include "common.cuh"

namespace amrgpu {

template <typename real, int ND>
struct EulerOps {
  static cudaError_t prepare(int B, int flux, int limiter);
  static cudaError_t stage(int B, int flux, const StageArgs<real>& a, const Geometry& G, cudaStream_t s);
  static cudaError_t reduce(int B, const real* U, const int* level, const Geometry& G, DevCtl* ctl,
                            double* partials, double* gpart, unsigned* gcount, int nleaves, int advance,
                            cudaStream_t s);
  static cudaError_t ghost_fill(int B, const real* U, real* slabs, const SlabDesc* desc, int nslabs,
                                cudaStream_t s);
  // rec: records grouped by coarse leaf, faces ascending within a group ([first, last) of each)
  static cudaError_t reflux(int B, real* out, const real* fflux, const RefluxRec* rec, int nrec,
                            const int* level, const Geometry& G, const DevCtl* ctl, real beta, cudaStream_t s);
  static cudaError_t lohner(int B, const real* U, const real* slabs, const int* nb, double gamma, double eps,
                            unsigned mask, double* err, int nleaves, cudaStream_t s);
  static cudaError_t regrid(int B, const real* Uold, real* Unew, const real* slabs, const int* nb,
                            const RegridOp* ops, int nnew, cudaStream_t s);
  static cudaError_t set_state(int B, const double* W, real* U, long long nleaves, int primitive, double gamma,
                               cudaStream_t s);
  static cudaError_t read_state(const real* U, double* out, long long n, cudaStream_t s);
  static cudaError_t face_ghosts(int B, const real* U, const real* slabs, const int* nb, int leaf, double* out,
                                 cudaStream_t s);
};

// tiny control kernels (ctl_kernels.cu)
cudaError_t ctl_set_t_end(DevCtl* ctl, double t_end, cudaStream_t s);
cudaError_t ctl_set_t(DevCtl* ctl, double t, cudaStream_t s);

}  // namespace amrgpu
