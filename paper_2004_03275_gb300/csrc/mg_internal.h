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
// synchronisation; the network's own pending work is ordered before it by an event.  Arguments
// as cnn_forward; fused: the single-pass inference kernel where it applies (2D, sides multiples
// of 32 and 16), which allocates nothing, else the layer-by-layer network.
int cnn_forward_async(cnn_handle* h, const float* in, int N, int D, int H, int W, float* out, cudaStream_t s,
                      bool fused);

// The fused inference path: whether it applies to an image shape, and its single launch on
// stream s with no event and no allocation (usable inside a stream capture; the caller orders
// the network's own stream, cnn_own_stream, around it).  The kernel reads the network's packed
// weights and biases, whose device buffers live as long as the handle.
bool cnn_fused_applies(const cnn_handle* h, int D, int H, int W);
cudaStream_t cnn_own_stream(const cnn_handle* h);
int cnn_enqueue_fused(cnn_handle* h, const float* in, int N, int H, int W, float* out, cudaStream_t s);
