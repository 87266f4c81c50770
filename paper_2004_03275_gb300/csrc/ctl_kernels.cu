// Tiny control kernels of the Euler solver.
#include "euler_ops.h"

namespace amrgpu {

// Both setters also rewrite the float copy of the step's dt (DevCtl::dt_stepf).
__global__ void set_t_end_kernel(DevCtl* ctl, double t_end) {
  ctl->t_end = t_end;
  ctl->dt_stepf = (float)step_dt(ctl->t, ctl->dt_cfl, t_end);
}
__global__ void set_t_kernel(DevCtl* ctl, double t) {
  ctl->t = t;
  ctl->dt_stepf = (float)step_dt(t, ctl->dt_cfl, ctl->t_end);
}

cudaError_t ctl_set_t_end(DevCtl* ctl, double t_end, cudaStream_t s) {
  set_t_end_kernel<<<1, 1, 0, s>>>(ctl, t_end);
  return cudaGetLastError();
}
cudaError_t ctl_set_t(DevCtl* ctl, double t, cudaStream_t s) {
  set_t_kernel<<<1, 1, 0, s>>>(ctl, t);
  return cudaGetLastError();
}

}  // namespace amrgpu
