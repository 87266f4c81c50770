// Tiny control kernels of the Euler solver.
#include "euler_ops.h"

namespace amrgpu {

__global__ void set_t_end_kernel(DevCtl* ctl, double t_end) { ctl->t_end = t_end; }

cudaError_t ctl_set_t_end(DevCtl* ctl, double t_end, cudaStream_t s) {
  set_t_end_kernel<<<1, 1, 0, s>>>(ctl, t_end);
  return cudaGetLastError();
}

}  // namespace amrgpu
