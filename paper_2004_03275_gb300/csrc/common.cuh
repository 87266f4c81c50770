// Shared device-side types of the amrvac_gb300 library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace amrgpu {

constexpr int kMaxLevel = 16;
constexpr int kGroupCTAs = 64;  // CTAs per first-level group of the two-level reduction finish

// Device control block of one solver: time, CFL step, reductions.  Written only
// by the last CTA of a reduction pass (no spin waits anywhere).
struct DevCtl {
  double t;          // current time
  double t_end;      // end time of the current run
  double dt_cfl;     // cfl / max signal rate of the current state
  double dt_last;    // dt of the last completed step
  double cfl;
  unsigned long long smax_bits;  // running max of the signal rate (bit pattern, >= 0)
  unsigned int done;             // CTAs finished in the current reduction pass
  int status;                    // bit 0: non-physical state met
  long long steps;
  double totals[5];
  float dt_stepf;    // (float) of the current step's dt, min(dt_cfl, t_end - t): rewritten by every
                     // writer of t, t_end and dt_cfl, so that float32 kernels read the step's dt
                     // without float64 instructions (GB300 runs float64 at 1/64 of the float32 rate)
};

// dt of a step from the time, the CFL step and the end time: the CFL step clipped to t_end
__host__ __device__ __forceinline__ double step_dt(double t, double dt_cfl, double t_end) {
  return t + dt_cfl > t_end ? t_end - t : dt_cfl;
}

// Ghost slab of one leaf face at a level jump.
struct SlabDesc {
  int target;   // leaf owning the ghosts
  int face;     // 2*dim + side
  int kind;     // 0: restriction from finer leaves, 1: prolongation from a coarser leaf
  int src[4];   // kind 0: fine leaf per tangential quadrant (q1 + 2 q2); kind 1: src[0] coarse leaf
  int off[2];   // kind 1: tangential offset of the target inside the coarse face (coarse cells)
};

// Coarse side of a level jump: replace the coarse face flux by the mean of the fine ones.
struct RefluxRec {
  int coarse;   // coarse leaf
  int face;     // its face
  int cslot;    // face-flux slot written by the coarse leaf
  int fslot[4]; // face-flux slots of the fine leaves per tangential quadrant
  int first;    // the records of the same coarse leaf: [first, last), faces ascending
  int last;
};

// New leaf after a regrid.
struct RegridOp {
  int kind;     // 0 copy, 1 prolong from parent, 2 restrict from children
  int src[8];   // copy/prolong: src[0] old leaf; restrict: children in x-fastest order
  int child;    // prolong: child offset bits (x | y<<1 | z<<2)
};

struct Geometry {
  int ndim, bnx, nleaves;
  double gamma, cfl;
  double dx[kMaxLevel + 1][3];
  double dV[kMaxLevel + 1];
  // float copies for the float32 kernels (float32 code touches no float64 unit in the cell loop)
  float gammaf;
  float dxf[kMaxLevel + 1][3];
  float idxf[kMaxLevel + 1][3];
};

// SSPRK stage combination alpha*U^n + beta*T, where T = U^(s) - dt div F and alpha + beta = 1
// in every stage of SSPRK2/3 (Sec. 2.4).  Float: written T + alpha (U^n - T), so that the
// rounded coefficients (1/3 and 2/3 round to floats whose sum is 1 + 3e-8) cannot scale the
// state up a little every step; T == U^n gives U^n exactly.  Double: the plain form, in the
// oracle's operation order (the double coefficients sum to 1 - 6e-17).
__device__ __forceinline__ float ssp_combine(float alpha, float, float u0, float t) { return t + alpha * (u0 - t); }
__device__ __forceinline__ double ssp_combine(double alpha, double beta, double u0, double t) {
  return alpha * u0 + beta * t;
}

// ------------------------------------------------------------ stage args --
template <typename real>
struct StageArgs {
  const real* Us;      // U^(s), read with halos
  const real* U0;      // U^n, read pointwise
  real* out;           // U^(s+1)
  const int* nb;       // [leaf][2*ndim] neighbour codes
  const real* slabs;   // [slab][var][2][nt]
  const int* level;    // [leaf]
  const int* ffx;      // [leaf][2*ndim] face-flux slot or -1
  real* fflux;         // [slot][var][nt]
  real* scratch;       // float32 3D 16^3 leaves: x + y flux differences, laid out like the state
  const void* tmap_us; // float32 2D 16^2 leaves: host pointer to the TMA tensor map of Us ([leaf*4+var][256])
  DevCtl* ctl;
  double* partials;    // [leaf][var]
  double* gpart;       // [group of CTAs][var]
  unsigned* gcount;    // [group of CTAs], zero between passes
  real alpha, beta;    // out = ssp_combine(alpha, beta, U0, Us - dt*div); stage1: out = Us - dt*div
  int stage1;
  int fuse_reduce;     // fold max rate / totals / time update into this pass
  int has_ffx;
  int limiter;
  int nleaves;
  int march_nw;        // float32 2D 16^2 march kernel, first and middle stages: warps (leaves) per CTA
  int march_persist;   // ... and whether a grid of resident CTAs loops over the leaf groups
};

}  // namespace amrgpu
