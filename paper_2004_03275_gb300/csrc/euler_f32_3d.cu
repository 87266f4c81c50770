// Explicit instantiation of the Euler device code for float, 3D.
#include "euler_kernels.cuh"
#include "euler_dispatch.cuh"

template struct amrgpu::EulerOps<float, 3>;
