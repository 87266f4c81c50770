// CFL step and conserved totals of a uniform block grid, computed without any
// device allocation: the reduction's scratch (per-leaf partial sums, group
// sums, counters and the control block) lives in one file-scope __device__
// array of fixed size instead of memory obtained from cudaMalloc.
//
// For callers that cannot allocate device memory themselves, e.g. code that
// runs under a fixed memory budget handed out by an enclosing framework's pool
// allocator (which forbids cudaMalloc beside it), or a latency-critical loop
// where the implicit synchronisation of cudaMalloc is not acceptable.  The
// address of the array is looked up once per device and kept for the life of
// the process: the call must not be used across a reset of that device.
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

#include "../../include/amrvac_gb300.h"
#include "euler_kernels.cuh"

namespace amrgpu {
namespace {

constexpr long long kNoAllocMaxLeaves = AMR_NOALLOC_MAX_LEAVES;
constexpr long long kNoAllocGroups = kNoAllocMaxLeaves / kGroupCTAs + 2;

struct NoAllocScratch {
  DevCtl ctl;
  double partials[kNoAllocMaxLeaves * 5];
  double gpart[kNoAllocGroups * 5];
  unsigned gcount[kNoAllocGroups];
};

// The scratch: every GPU that loads this library holds one copy until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the scratch on the current device (looked up once per device).
cudaError_t scratch_address(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = reinterpret_cast<NoAllocScratch*>(g_scratch_addr[dev]);
  return cudaSuccess;
}

// Same reduction as reduce_kernel for a grid whose leaves are all on level 1.
template <int ND, int B>
__global__ void __launch_bounds__(256) reduce_uniform_kernel(const double* __restrict__ U, Geometry G,
                                                             NoAllocScratch* S, int nleaves) {
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC;
  constexpr int CPT = NC >= 256 ? NC / 256 : 1;
  constexpr int LPB = NC >= 256 ? 1 : 256 / NC;
  const int lb = threadIdx.x / (NC / CPT), tc = threadIdx.x % (NC / CPT);
  const int leaf = blockIdx.x * LPB + lb;
  const double gam = G.gamma, gm1 = gam - 1.0;
  double rate = 0.0;
  double sums[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) sums[v] = 0.0;
  int bad = 0;
  if (leaf < nleaves) {
    double dx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) dx[d] = G.dx[1][d];
    for (int c = tc; c < NC; c += NC / CPT) {
      double Uc[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Uc[v] = U[((size_t)leaf * NV + v) * NC + c];
      rate = fmax(rate, cell_rate<double, ND>(Uc, gam, gm1, dx, &bad));
#pragma unroll
      for (int v = 0; v < NV; ++v) sums[v] += Uc[v] * G.dV[1];
    }
  }
  block_reduce_finish<double, NV, 256>(rate, sums, blockIdx.x * LPB, LPB, lb, G, &S->ctl, S->partials, S->gpart,
                                       S->gcount, nleaves, false, 0.0, bad);
}

template <int ND, int B>
void launch_uniform(const double* U, const Geometry& G, NoAllocScratch* S, int nleaves, cudaStream_t s) {
  constexpr int NC = Tile<ND, B>::NC;
  constexpr int LPB = NC >= 256 ? 1 : 256 / NC;
  reduce_uniform_kernel<ND, B><<<(nleaves + LPB - 1) / LPB, 256, 0, s>>>(U, G, S, nleaves);
}

}  // namespace
}  // namespace amrgpu

using namespace amrgpu;

extern "C" int amr_reduce_noalloc(const amr_config* cfg, const double* U, long long nleaves, double* dt_cfl,
                                  double* totals) {
  if (!cfg || !U || !dt_cfl || !totals) return AMR_ERR_INVALID_ARG;
  const int nd = cfg->ndim, B = cfg->block_nx;
  if (nd < 1 || nd > 3 || (B != 8 && B != 16) || !(cfg->gamma > 1.0) || !(cfg->cfl > 0.0)) return AMR_ERR_INVALID_ARG;
  long long nbase = 1;
  for (int d = 0; d < nd; ++d) {
    if (cfg->base_nblocks[d] < 1 || !(cfg->xmax[d] > cfg->xmin[d])) return AMR_ERR_INVALID_ARG;
    nbase *= cfg->base_nblocks[d];
  }
  if (nleaves != nbase) return AMR_ERR_INVALID_ARG;  // a uniform level-1 grid of base_nblocks leaves
  if (nleaves < 1 || nleaves > AMR_NOALLOC_MAX_LEAVES) return AMR_ERR_CAPACITY;
  cudaStream_t stream = (cudaStream_t)cfg->stream;
  NoAllocScratch* S = nullptr;
  if (scratch_address(&S) != cudaSuccess) return AMR_ERR_CUDA;
  Geometry G{};
  G.ndim = nd;
  G.bnx = B;
  G.nleaves = (int)nleaves;
  G.gamma = cfg->gamma;
  G.cfl = cfg->cfl;
  double dV = 1.0;
  for (int d = 0; d < 3; ++d) {
    G.dx[1][d] = d < nd ? (cfg->xmax[d] - cfg->xmin[d]) / ((double)cfg->base_nblocks[d] * B) : 1.0;
    if (d < nd) dV = dV * G.dx[1][d];
  }
  G.dV[1] = dV;
  // the scratch keeps the previous call's contents: reset what must start at zero
  DevCtl c0{};
  c0.cfl = cfg->cfl;
  c0.t_end = 1e300;
  if (cudaMemcpyAsync(&S->ctl, &c0, sizeof(DevCtl), cudaMemcpyHostToDevice, stream) != cudaSuccess) return AMR_ERR_CUDA;
  if (cudaMemsetAsync(S->gcount, 0, sizeof(S->gcount), stream) != cudaSuccess) return AMR_ERR_CUDA;
  if (nd == 1) {
    if (B == 16) launch_uniform<1, 16>(U, G, S, (int)nleaves, stream);
    else launch_uniform<1, 8>(U, G, S, (int)nleaves, stream);
  } else if (nd == 2) {
    if (B == 16) launch_uniform<2, 16>(U, G, S, (int)nleaves, stream);
    else launch_uniform<2, 8>(U, G, S, (int)nleaves, stream);
  } else {
    if (B == 16) launch_uniform<3, 16>(U, G, S, (int)nleaves, stream);
    else launch_uniform<3, 8>(U, G, S, (int)nleaves, stream);
  }
  if (cudaGetLastError() != cudaSuccess) return AMR_ERR_CUDA;
  DevCtl out{};
  if (cudaMemcpyAsync(&out, &S->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return AMR_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return AMR_ERR_CUDA;
  *dt_cfl = out.dt_cfl;
  for (int v = 0; v < nd + 2; ++v) totals[v] = out.totals[v];
  return (out.status & 1) ? AMR_ERR_NONPHYSICAL : AMR_OK;
}
