// Explicit instantiation of the Euler device code for double, 3D.
#include "euler_kernels.cuh"
#include "euler_dispatch.cuh"

template struct amrgpu::EulerOps<double, 3>;
