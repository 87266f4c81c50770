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

// Inference of the learned-guess network (cnn.cu) on stream s without a final
// synchronisation; the network's own pending work is ordered before it, and the network's
// later work after it, by events.  Arguments as cnn_forward.
int cnn_forward_async(cnn_handle* h, const float* in, int N, int D, int H, int W, float* out, cudaStream_t s);
