// Explicit instantiation of the Euler device code for double, 2D.
#include "euler_kernels.cuh"
#include "euler_dispatch.cuh"

template struct amrgpu::EulerOps<double, 2>;
