// Explicit instantiation of the Euler device code for float, 2D.
#include "euler_kernels.cuh"
#include "stage2d_f32.cuh"
#include "euler_dispatch.cuh"

template struct amrgpu::EulerOps<float, 2>;
