// Entry points of the batched multigrid (mg.cu) for other units of this library; not part
// of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "../../include/amrvac_gb300.h"

// Enqueue one complete solve of h onto stream s, which must be capturing a graph: b and x
// (device arrays of mg_num_unknowns doubles; x: guess in, solution out) are copied in, the
// solve runs with its device-side convergence loop, and x is copied back.
int mg_capture_solve(mg_handle* h, const double* b, double* x, cudaStream_t s);

// Device array of the V-cycles of each instance in the handle's last solve, and the number
// of kernels one iteration of its device-side loop launches.
const int* mg_device_cycles(const mg_handle* h);
long long mg_loop_kernels(const mg_handle* h);
