// Device code of the block-tree finite-volume Euler update, templated on the
// arithmetic type.  Included by one translation unit per (type, dimension);
// float units are compiled with fast division/sqrt, double units without FMA
// contraction so that every rounding follows the written order.
//
// Paper (arXiv:2004.03275): Sec. 1.1 variables and flux split; Sec. 1.2 signal
// speeds (phys_get_cmax/cbounds), TVDLF and HLL; Sec. 2.4 HLLC; Sec. 2.3.1
// limited reconstruction (Koren); Sec. 2.3.2 / 2.4 SSP Runge-Kutta; Sec. 1.3
// block tree with refinement ratio 2 and a Lohner-type estimator.
//
// State layout: U[leaf][var][cell], cell = i + B*(j + B*k), leaves in Morton
// order.  A leaf's face ghosts (two layers) come from a same-level neighbour's
// interior, from a ghost slab filled at a level jump, or from the leaf itself
// (zero-gradient outflow).
#pragma once
#include "common.cuh"

namespace amrgpu {

enum { FLUX_TVDLF = 0, FLUX_HLL = 1, FLUX_HLLC = 2 };
enum { LIM_MINMOD = 0, LIM_VANLEER = 1, LIM_KOREN = 2, LIM_NONE = 3, LIM_MC = 4, LIM_CADA = 5 };

// ------------------------------------------------------------------ physics --
template <typename real, int ND>
__device__ __forceinline__ void cons_to_prim(const real* U, real* V, real gm1) {
  real rho = U[0];
  real msq = real(0);
#pragma unroll
  for (int d = 0; d < ND; ++d) msq = msq + U[1 + d] * U[1 + d];
  V[0] = rho;
#pragma unroll
  for (int d = 0; d < ND; ++d) V[1 + d] = U[1 + d] / rho;
  V[ND + 1] = gm1 * (U[ND + 1] - (real(0.5) * msq) / rho);
}

template <typename real, int ND>
__device__ __forceinline__ void prim_to_cons(const real* V, real* U, real gm1) {
  real rho = V[0];
  real vsq = real(0);
#pragma unroll
  for (int d = 0; d < ND; ++d) vsq = vsq + V[1 + d] * V[1 + d];
  U[0] = rho;
#pragma unroll
  for (int d = 0; d < ND; ++d) U[1 + d] = rho * V[1 + d];
  U[ND + 1] = V[ND + 1] / gm1 + (real(0.5) * rho) * vsq;
}

template <typename real>
__device__ __forceinline__ real dsqrt(real x) { return sqrt(x); }

// flux of the state V (conserved U precomputed) normal to `dir`
template <typename real, int ND>
__device__ __forceinline__ void phys_flux(int dir, const real* V, const real* U, real* F) {
  real un = V[1 + dir];
  real p = V[ND + 1];
  F[0] = U[1 + dir];
#pragma unroll
  for (int e = 0; e < ND; ++e) {
    F[1 + e] = U[1 + e] * un;
    if (e == dir) F[1 + e] = F[1 + e] + p;
  }
  F[ND + 1] = (U[ND + 1] + p) * un;
}

// Approximate Riemann fluxes.  Wave-speed bounds: Davis estimates
// S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R); HLLC with
// Toro's contact speed S*; TVDLF with c_max = max(|u| + c).
template <typename real, int ND, int FLUX>
__device__ __forceinline__ void riemann(int dir, const real* VL, const real* VR, real gam, real gm1, real* F) {
  constexpr int NV = ND + 2;
  real UL[NV], UR[NV], FL[NV], FR[NV];
  prim_to_cons<real, ND>(VL, UL, gm1);
  prim_to_cons<real, ND>(VR, UR, gm1);
  phys_flux<real, ND>(dir, VL, UL, FL);
  phys_flux<real, ND>(dir, VR, UR, FR);
  real uL = VL[1 + dir], uR = VR[1 + dir];
  real cL = dsqrt(gam * VL[ND + 1] / VL[0]);
  real cR = dsqrt(gam * VR[ND + 1] / VR[0]);
  if (FLUX == FLUX_TVDLF) {
    real cmax = fmax(fabs(uL) + cL, fabs(uR) + cR);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = real(0.5) * (FL[v] + FR[v]) - (real(0.5) * cmax) * (UR[v] - UL[v]);
    return;
  }
  real SL = fmin(uL - cL, uR - cR);
  real SR = fmax(uL + cL, uR + cR);
  if (SL >= real(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = FL[v];
    return;
  }
  if (SR <= real(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = FR[v];
    return;
  }
  if (FLUX == FLUX_HLL) {
    real inv = real(1) / (SR - SL);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = (SR * FL[v] - SL * FR[v] + (SL * SR) * (UR[v] - UL[v])) * inv;
    return;
  }
  real rL = VL[0], rR = VR[0], pL = VL[ND + 1], pR = VR[ND + 1];
  real aL = rL * (SL - uL), aR = rR * (SR - uR);
  real Sstar = (pR - pL + aL * uL - aR * uR) / (aL - aR);
  bool left = Sstar >= real(0);
  real Vk[NV], Uk[NV], Fk[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    Vk[v] = left ? VL[v] : VR[v];
    Uk[v] = left ? UL[v] : UR[v];
    Fk[v] = left ? FL[v] : FR[v];
  }
  real Sk = left ? SL : SR;
  real ak = left ? aL : aR;
  real uk = Vk[1 + dir], pk = Vk[ND + 1], rk = Vk[0];
  real fac = ak / (Sk - Sstar);
  real Us[NV];
  Us[0] = fac;
#pragma unroll
  for (int e = 0; e < ND; ++e) Us[1 + e] = fac * (e == dir ? Sstar : Vk[1 + e]);
  Us[ND + 1] = fac * (Uk[ND + 1] / rk + (Sstar - uk) * (Sstar + pk / ak));
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = Fk[v] + Sk * (Us[v] - Uk[v]);
}

// Limited slopes of a cell from a = q_i - q_{i-1}, b = q_{i+1} - q_i:
// s- towards i-1/2, s+ towards i+1/2 (face values q_i -+ s/2).  minmod, van Leer,
// monotonized central: one symmetric slope.  Koren (1993): the third-order kappa = 1/3
// face values q_i + (a + 2b)/6, q_i - (2a + b)/6 limited into the TVD region.  Cada and
// Torrilhon (2009), the third-order limiter of Sec. 2.3.1: theta = a/b, offset phi(theta) b/2
// with phi = max(0, min(phi_3, max(-theta, min(2 theta, phi_3, 3/2)))), phi_3 = (2 + theta)/3,
// and its mirror image towards i-1/2; it keeps a slope where a and b differ in sign.
template <typename real>
__device__ __forceinline__ void limited_slopes(int lim, real a, real b, real& sm, real& sp) {
  bool same = (a > real(0) && b > real(0)) || (a < real(0) && b < real(0));
  if (lim == LIM_CADA) {
    real A = fabs(a), Bb = fabs(b), up = real(0), dn = real(0);
    if (same) {
      up = fmin(fmin(real(2) * A, (A + real(2) * Bb) / real(3)), real(1.5) * Bb);
      dn = fmin(fmin(real(2) * Bb, (real(2) * A + Bb) / real(3)), real(1.5) * A);
    } else if (a != real(0) && b != real(0)) {
      up = fmax(real(0), fmin((real(2) * Bb - A) / real(3), A));
      dn = fmax(real(0), fmin((real(2) * A - Bb) / real(3), Bb));
    }
    sp = (b > real(0)) ? up : -up;
    sm = (a > real(0)) ? dn : -dn;
    return;
  }
  if (lim == LIM_NONE || !same) {
    sm = real(0);
    sp = real(0);
    return;
  }
  if (lim == LIM_MINMOD) {
    real s = (a > real(0)) ? fmin(a, b) : fmax(a, b);
    sm = s;
    sp = s;
  } else if (lim == LIM_VANLEER) {
    real s = (real(2) * a * b) / (a + b);
    sm = s;
    sp = s;
  } else if (lim == LIM_MC) {  // monotonized central: minmod((a+b)/2, 2a, 2b)
    real A = fabs(a), Bb = fabs(b);
    real s = fmin(fmin(real(0.5) * (A + Bb), real(2) * A), real(2) * Bb);
    sm = (a > real(0)) ? s : -s;
    sp = sm;
  } else {  // Koren
    real A = fabs(a), Bb = fabs(b);
    real up = fmin(fmin(real(2) * A, (A + real(2) * Bb) / real(3)), real(2) * Bb);
    real dn = fmin(fmin(real(2) * Bb, (real(2) * A + Bb) / real(3)), real(2) * A);
    sp = (b > real(0)) ? up : -up;
    sm = (a > real(0)) ? dn : -dn;
  }
}

template <typename real>
__device__ __forceinline__ real minmod2(real a, real b) {
  if (a > real(0) && b > real(0)) return fmin(a, b);
  if (a < real(0) && b < real(0)) return fmax(a, b);
  return real(0);
}

// Face state pair from the primitive values of cells f-2, f-1, f, f+1 along a line;
// first-order fallback when a reconstructed density or pressure is not positive.
template <typename real, int ND>
__device__ __forceinline__ void face_states(int lim, const real (*W)[ND + 2], real* VL, real* VR) {
  constexpr int NV = ND + 2;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    real smL, spL, smR, spR;
    limited_slopes<real>(lim, W[1][v] - W[0][v], W[2][v] - W[1][v], smL, spL);
    limited_slopes<real>(lim, W[2][v] - W[1][v], W[3][v] - W[2][v], smR, spR);
    VL[v] = W[1][v] + real(0.5) * spL;
    VR[v] = W[2][v] - real(0.5) * smR;
  }
  if (!(VL[0] > real(0)) || !(VR[0] > real(0)) || !(VL[ND + 1] > real(0)) || !(VR[ND + 1] > real(0))) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      VL[v] = W[1][v];
      VR[v] = W[2][v];
    }
  }
}

// ------------------------------------------------------------- reductions --
template <typename real>
struct MaxKey;
template <>
struct MaxKey<double> {
  static __device__ unsigned long long enc(double s) { return (unsigned long long)__double_as_longlong(s); }
  static __device__ double dec(unsigned long long b) { return __longlong_as_double((long long)b); }
};
template <>
struct MaxKey<float> {
  static __device__ unsigned long long enc(float s) { return (unsigned long long)__float_as_uint(s); }
  static __device__ double dec(unsigned long long b) { return (double)__uint_as_float((unsigned int)b); }
};

// dt of the current step: the CFL step clipped to t_end (same on every CTA; step_dt in common.cuh)
__device__ __forceinline__ double stage_dt(const DevCtl* ctl) { return step_dt(ctl->t, ctl->dt_cfl, ctl->t_end); }
// DevCtl::dt_stepf from the current t, dt_cfl and t_end (one thread, after it changed one of them)
__device__ __forceinline__ void refresh_dt_step(volatile DevCtl* c) {
  c->dt_stepf = (float)step_dt(c->t, c->dt_cfl, c->t_end);
}

// dt of the current step computed once per CTA (thread 0) and shared: keeps
// float64 arithmetic out of the per-cell path of the float32 kernels.
__device__ __forceinline__ double cta_stage_dt(const DevCtl* ctl, float* dtf) {
  __shared__ double s_dt;
  __shared__ float s_dtf;
  if (threadIdx.x == 0) {
    double d = stage_dt(ctl);
    s_dt = d;
    s_dtf = (float)d;
  }
  __syncthreads();
  if (dtf) *dtf = s_dtf;
  return s_dt;
}

// float32 kernels: the step's dt as a float, read once per CTA and shared (the barrier is
// part of the contract, as in cta_stage_dt); no float64 instruction is issued
__device__ __forceinline__ float cta_stage_dtf(const DevCtl* ctl) {
  __shared__ float s_dtf;
  if (threadIdx.x == 0) s_dtf = *reinterpret_cast<const volatile float*>(&ctl->dt_stepf);
  __syncthreads();
  return s_dtf;
}

template <typename real>
__device__ __forceinline__ real geo_dx(const Geometry& G, int lev, int d);
template <>
__device__ __forceinline__ double geo_dx<double>(const Geometry& G, int lev, int d) { return G.dx[lev][d]; }
template <>
__device__ __forceinline__ float geo_dx<float>(const Geometry& G, int lev, int d) { return G.dxf[lev][d]; }
template <typename real>
__device__ __forceinline__ real geo_gamma(const Geometry& G);
template <>
__device__ __forceinline__ double geo_gamma<double>(const Geometry& G) { return G.gamma; }
template <>
__device__ __forceinline__ float geo_gamma<float>(const Geometry& G) { return G.gammaf; }

// Signal rate sum_d (|v_d| + c)/dx_d of one cell (Sec. 1.2, phys_get_cmax);
// marks non-physical states.
template <typename real, int ND>
__device__ __forceinline__ real cell_rate(const real* U, real gam, real gm1, const real* dx, int* bad) {
  real V[ND + 2];
  cons_to_prim<real, ND>(U, V, gm1);
  if (!(V[0] > real(0)) || !(V[ND + 1] > real(0))) *bad = 1;
  real cs = dsqrt(gam * V[ND + 1] / V[0]);
  real s = real(0);
#pragma unroll
  for (int d = 0; d < ND; ++d) s = s + (fabs(V[1 + d]) + cs) / dx[d];
  return s;
}

// Fixed-order block sum of NV doubles held by every thread (butterfly per warp,
// warps in order); the result is valid in thread 0.
template <int NV, int NTHREADS>
__device__ __forceinline__ void block_sum_fixed(double* acc) {
  __shared__ double wred[NTHREADS / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
  if (lane == 0)
#pragma unroll
    for (int v = 0; v < NV; ++v) wred[warp][v] = acc[v];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = wred[0][v];
    for (int w = 1; w < NTHREADS / 32; ++w)
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += wred[w][v];
  }
}

// Totals, dt_cfl = cfl / smax and, when `advance`, t += dt (one thread).
template <typename real, int NV>
__device__ __forceinline__ void publish_reduction(DevCtl* ctl, const double* acc, bool advance, double dt) {
  volatile DevCtl* c = ctl;
  for (int v = 0; v < NV; ++v) c->totals[v] = acc[v];
  unsigned long long bits = atomicAdd(&ctl->smax_bits, 0ull);
  double smax = MaxKey<real>::dec(bits);
  if (advance) {
    c->t = c->t + dt;
    c->dt_last = dt;
    c->steps = c->steps + 1;
  }
  c->dt_cfl = c->cfl / smax;
  refresh_dt_step(c);
  c->smax_bits = 0ull;
  c->done = 0u;
}

// Two-level finish of a reduction pass.  The last CTA to finish in each group of
// kGroupCTAs CTAs sums that group's per-leaf partials (fixed order) into gpart;
// the last group to finish sums the group partials (fixed order), sets the
// totals, dt_cfl = cfl/smax and, when `advance`, t += dt.  Every thread of every
// CTA calls this after its CTA's partials and atomicMax are issued.  No CTA
// waits on another; counters are reset by the CTA that consumed them.
// fence_all = false: the threads that wrote the CTA's partials have already
// issued their fence, so the others skip it.  dt_from_ctl: the step's dt is read
// from the control block by the finishing thread (float32 kernels carry only its
// float copy; t, dt_cfl and t_end do not change before this finish).
template <typename real, int NV, int NTHREADS>
__device__ void last_cta_finish(DevCtl* ctl, const double* partials, double* gpart, unsigned* gcount,
                                int nleaves, int lpb, bool advance, double dt, bool fence_all = true,
                                bool dt_from_ctl = false) {
  __shared__ bool flag;
  const int g = blockIdx.x / kGroupCTAs;
  const int ngroups = (gridDim.x + kGroupCTAs - 1) / kGroupCTAs;
  const int gsize = min(kGroupCTAs, (int)gridDim.x - g * kGroupCTAs);
  if (fence_all) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) flag = atomicAdd(&gcount[g], 1u) == (unsigned)(gsize - 1);
  __syncthreads();
  if (!flag) return;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  // the group's CTAs processed slots s = g*kGroupCTAs + i + k*gridDim (i < gsize, k >= 0),
  // each slot holding lpb consecutive leaves; summed in a fixed order
  const int nslots = (nleaves + lpb - 1) / lpb;
  const int nj = gsize * ((nslots + (int)gridDim.x - 1) / (int)gridDim.x);
  for (int j = threadIdx.x; j < nj; j += NTHREADS) {
    int s = g * kGroupCTAs + (j % gsize) + (j / gsize) * (int)gridDim.x;
    if (s >= nslots) continue;
    for (int q = 0; q < lpb; ++q) {
      int l = s * lpb + q;
      if (l < nleaves)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += __ldcg(&partials[(size_t)l * NV + v]);
    }
  }
  block_sum_fixed<NV, NTHREADS>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) gpart[(size_t)g * NV + v] = acc[v];
    gcount[g] = 0u;
    __threadfence();
    flag = atomicAdd(&ctl->done, 1u) == (unsigned)(ngroups - 1);
  }
  __syncthreads();
  if (!flag) return;
  __threadfence();
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  for (int q = threadIdx.x; q < ngroups; q += NTHREADS)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += __ldcg(&gpart[(size_t)q * NV + v]);
  __syncthreads();  // wred reuse
  block_sum_fixed<NV, NTHREADS>(acc);
  if (threadIdx.x == 0) {
    if (dt_from_ctl) {
      const volatile DevCtl* c = ctl;
      dt = step_dt(c->t, c->dt_cfl, c->t_end);
    }
    publish_reduction<real, NV>(ctl, acc, advance, dt);
  }
}

// One-level finish for a grid whose CTAs each wrote one row of NV partials (row = blockIdx.x):
// the last CTA to arrive sums the rows in a fixed order (thread t: rows t, t + NTHREADS, ...;
// then the block sum) and publishes.  One counter atomic, one fence and one pass over the
// partials, against two of each in last_cta_finish: for a few hundred CTAs this shortens the
// serial tail at the end of the launch.  The caller fences its partials before the barrier.
template <typename real, int NV, int NTHREADS>
__device__ void last_cta_finish_flat(DevCtl* ctl, const double* partials, bool advance, double dt) {
  __shared__ bool flag;
  __syncthreads();
  if (threadIdx.x == 0) flag = atomicAdd(&ctl->done, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!flag) return;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  for (int r = threadIdx.x; r < (int)gridDim.x; r += NTHREADS)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += __ldcg(&partials[(size_t)r * NV + v]);
  block_sum_fixed<NV, NTHREADS>(acc);
  if (threadIdx.x == 0) publish_reduction<real, NV>(ctl, acc, advance, dt);
}

// Block-wide reduction of (max rate, per-variable FP64 sums) and the last-CTA
// finalisation: totals = fixed-order sum of per-leaf partials, dt_cfl = cfl/smax,
// and, when `advance`, t += dt of the step just taken.  Deterministic for any
// CTA schedule; no CTA ever waits on another.
template <typename real, int NV, int NTHREADS>
__device__ void block_reduce_finish(real rate, const double* sums, int leaf_first, int nleaf_cta,
                                    int leaf_of_thread, const Geometry& G, DevCtl* ctl, double* partials,
                                    double* gpart, unsigned* gcount, int nleaves, bool advance, double dt,
                                    int bad) {
  __shared__ double red[NTHREADS / 32][4][NV];  // per warp, per local leaf (<= 4), per var
  __shared__ real wmax[NTHREADS / 32];
  __shared__ int sbad;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  if (bad) sbad = 1;
  // max rate
  real m = rate;
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) wmax[warp] = m;
  // sums per local leaf: a warp covers one leaf when leaves have >= 32 cells per CTA slot
  double s[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) s[v] = sums[v];
  // leaves of a CTA are contiguous groups of threads of equal size >= 16 cells; reduce within
  // groups of width gw = NTHREADS / nleaf_cta (power of two) by butterflies limited to the group
  int gw = NTHREADS / nleaf_cta;
  int lim = gw < 32 ? gw : 32;
  for (int o = lim / 2; o > 0; o >>= 1)
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
  if (gw >= 32) {
    if (lane == 0)
#pragma unroll
      for (int v = 0; v < NV; ++v) red[warp][0][v] = s[v];
  } else {
    if ((threadIdx.x % gw) == 0)
#pragma unroll
      for (int v = 0; v < NV; ++v) red[warp][(threadIdx.x % 32) / gw][v] = s[v];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    real mm = wmax[0];
    for (int w = 1; w < NTHREADS / 32; ++w) mm = fmax(mm, wmax[w]);
    atomicMax(&ctl->smax_bits, MaxKey<real>::enc(mm));
    if (sbad) atomicOr(&ctl->status, 1);
  }
  if (threadIdx.x < nleaf_cta) {
    int l = leaf_first + threadIdx.x;
    if (l < nleaves) {
      double acc[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = 0.0;
      if (gw >= 32) {
        int wpl = gw / 32;
        for (int w = 0; w < wpl; ++w)
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] += red[threadIdx.x * wpl + w][0][v];
      } else {
        int lpw = 32 / gw;
        int w = threadIdx.x / lpw, q = threadIdx.x % lpw;
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = red[w][q][v];
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) partials[(size_t)l * NV + v] = acc[v];
    }
  }
  __threadfence();
  __syncthreads();  // partials written and red[] consumed before it is reused below
  last_cta_finish<real, NV, NTHREADS>(ctl, partials, gpart, gcount, nleaves, nleaf_cta, advance, dt);
}

// ------------------------------------------------------------ ghost fetch --
template <int ND, int B>
__device__ __forceinline__ int compose_cell(int d, int n, int t) {
  if (ND == 1) return n;
  if (ND == 2) return d == 0 ? n + B * t : t + B * n;
  int t1 = t % B, t2 = t / B;
  if (d == 0) return n + B * (t1 + B * t2);
  if (d == 1) return t1 + B * (n + B * t2);
  return t1 + B * (t2 + B * n);
}

template <int ND, int B>
struct Tile {
  static constexpr int NV = ND + 2;
  static constexpr int NC = ND == 1 ? B : (ND == 2 ? B * B : B * B * B);
  static constexpr int NT = ND == 1 ? 1 : (ND == 2 ? B : B * B);
};

// conserved value of ghost (face f = 2d+side, layer m, tangential t, var v) of leaf b
template <typename real, int ND, int B>
__device__ __forceinline__ real fetch_ghost(const real* __restrict__ U, const real* __restrict__ slabs,
                                            const int* __restrict__ nb, int b, int f, int m, int t, int v) {
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC, NT = Tile<ND, B>::NT;
  int code = __ldg(&nb[b * 2 * ND + f]);
  int d = f >> 1, side = f & 1;
  if (code >= 0) {
    int n = side == 0 ? B - 1 - m : m;
    return U[((size_t)code * NV + v) * NC + compose_cell<ND, B>(d, n, t)];
  }
  if (code == -1) {
    int n = side == 0 ? 0 : B - 1;
    return U[((size_t)b * NV + v) * NC + compose_cell<ND, B>(d, n, t)];
  }
  int s = -2 - code;
  return slabs[(((size_t)s * NV + v) * 2 + m) * NT + t];
}

// ======================================================= 1D and 2D stages ==
// One thread per cell; a CTA takes LPB leaves.  Primitive values of each leaf
// plus its face ghosts are staged in shared memory, every face flux is computed
// once, then each cell forms its flux difference and the SSPRK combination.
template <typename real, int ND, int B, int FLUX>
__global__ void __launch_bounds__(ND == 1 ? 128 : 256)
stage_kernel_12(StageArgs<real> a, Geometry G) {
  constexpr int THREADS = ND == 1 ? 128 : 256;
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC, NT = Tile<ND, B>::NT;
  constexpr int LPB = THREADS / NC;
  constexpr int P = B + 4;
  constexpr int PP = ND == 1 ? P : P * P;
  constexpr int NFX = ND == 1 ? (B + 1) : B * (B + 1);  // faces per direction per leaf
  __shared__ real W[LPB][NV][PP];
  __shared__ real FXs[LPB][ND][NV][NFX];

  float dtf;
  const double dt = cta_stage_dt(a.ctl, &dtf);
  if (!(dt > 0.0)) return;
  const real dtr = sizeof(real) == 4 ? (real)dtf : (real)dt;
  const real gam = geo_gamma<real>(G), gm1 = gam - real(1);
  const int lb = threadIdx.x / NC, tc = threadIdx.x % NC;
  const int leaf = blockIdx.x * LPB + lb;
  const bool active = leaf < a.nleaves;
  const int ic = tc % B, jc = ND == 2 ? tc / B : 0;

  real Uc[NV];
  if (active) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Uc[v] = a.Us[((size_t)leaf * NV + v) * NC + tc];
    real Vc[NV];
    cons_to_prim<real, ND>(Uc, Vc, gm1);
    int pidx = ND == 1 ? ic + 2 : (jc + 2) * P + (ic + 2);
#pragma unroll
    for (int v = 0; v < NV; ++v) W[lb][v][pidx] = Vc[v];
    // face ghosts: 2*ND faces x 2 layers x NT cells
    constexpr int NH = 2 * ND * 2 * NT;
    for (int h = tc; h < NH; h += NC) {
      int f = h / (2 * NT), m = (h / NT) % 2, t = h % NT;
      real Ug[NV], Vg[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Ug[v] = fetch_ghost<real, ND, B>(a.Us, a.slabs, a.nb, leaf, f, m, t, v);
      cons_to_prim<real, ND>(Ug, Vg, gm1);
      int d = f >> 1, side = f & 1;
      int n = side == 0 ? -1 - m : B + m;
      int pi, pj;
      if (d == 0) { pi = n; pj = t; } else { pi = t; pj = n; }
      int q = ND == 1 ? pi + 2 : (pj + 2) * P + (pi + 2);
#pragma unroll
      for (int v = 0; v < NV; ++v) W[lb][v][q] = Vg[v];
    }
  }
  __syncthreads();
  const int lim = a.limiter;
  if (active) {
    for (int idx = tc; idx < ND * NFX; idx += NC) {
      int dim = idx / NFX, fl = idx % NFX;
      int fi, fj;  // face index along dim, row
      if (ND == 1) { fi = fl; fj = 0; }
      else if (dim == 0) { fi = fl % (B + 1); fj = fl / (B + 1); }
      else { fi = fl % (B + 1); fj = fl / (B + 1); }
      real Wl[4][NV];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        int c = fi - 2 + s;
        int q = ND == 1 ? c + 2 : (dim == 0 ? (fj + 2) * P + (c + 2) : (c + 2) * P + (fj + 2));
#pragma unroll
        for (int v = 0; v < NV; ++v) Wl[s][v] = W[lb][v][q];
      }
      real VL[NV], VR[NV], F[NV];
      face_states<real, ND>(lim, Wl, VL, VR);
      riemann<real, ND, FLUX>(dim, VL, VR, gam, gm1, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) FXs[lb][dim][v][fl] = F[v];
      if (a.has_ffx && (fi == 0 || fi == B)) {
        int face = 2 * dim + (fi == 0 ? 0 : 1);
        int slot = a.ffx[leaf * 2 * ND + face];
        if (slot >= 0) {
#pragma unroll
          for (int v = 0; v < NV; ++v) a.fflux[((size_t)slot * NV + v) * NT + fj] = F[v];
        }
      }
    }
  }
  __syncthreads();
  real rate = real(0);
  double sums[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) sums[v] = 0.0;
  int bad = 0;
  if (active) {
    const int lev = a.level[leaf];
    real dx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) dx[d] = geo_dx<real>(G, lev, d);
    real Un[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      real div = real(0);
      {
        int lo = ND == 1 ? ic : jc * (B + 1) + ic;
        div = div + (FXs[lb][0][v][lo + 1] - FXs[lb][0][v][lo]) / dx[0];
      }
      if (ND == 2)  // y faces are stored per column: (face index jc, column ic)
        div = div + (FXs[lb][ND - 1][v][ic * (B + 1) + jc + 1] - FXs[lb][ND - 1][v][ic * (B + 1) + jc]) / dx[1];
      real tmp = Uc[v] - dtr * div;
      Un[v] = a.stage1 ? tmp : ssp_combine(a.alpha, a.beta, a.U0[((size_t)leaf * NV + v) * NC + tc], tmp);
      a.out[((size_t)leaf * NV + v) * NC + tc] = Un[v];
    }
    if (a.fuse_reduce) {
      rate = cell_rate<real, ND>(Un, gam, gm1, dx, &bad);
      double dV = G.dV[lev];
#pragma unroll
      for (int v = 0; v < NV; ++v) sums[v] = (double)Un[v] * dV;
    }
  }
  if (a.fuse_reduce)
    block_reduce_finish<real, NV, THREADS>(rate, sums, blockIdx.x * LPB, LPB, lb, G, a.ctl, a.partials,
                                           a.gpart, a.gcount, a.nleaves, true, dt, bad);
}

// ============================================================ 3D stage ==
// One thread per (i, j) column of a leaf, marching in k.  Shared memory holds a
// ring of four primitive planes (k-1 .. k+2, with x/y face ghosts for interior
// planes), the x and y face fluxes of plane k and the z flux of face k-1/2.
template <typename real, int B>
struct Stage3DSmem {
  static constexpr int NV = 5, P = B + 4, LPB = 256 / (B * B);
  real W[LPB][4][NV][P * P];
  real FX[LPB][2][NV][B * (B + 1)];
  real FZ[LPB][NV][B * B];
};

template <typename real, int B, int FLUX>
__global__ void __launch_bounds__(256) stage_kernel_3d(StageArgs<real> a, Geometry G) {
  constexpr int NV = 5, NC = B * B * B, NT = B * B, P = B + 4, COLS = B * B;
  constexpr int LPB = 256 / COLS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Stage3DSmem<real, B>& S = *reinterpret_cast<Stage3DSmem<real, B>*>(smem_raw);

  float dtf;
  const double dt = cta_stage_dt(a.ctl, &dtf);
  if (!(dt > 0.0)) return;
  const real dtr = sizeof(real) == 4 ? (real)dtf : (real)dt;
  const real gam = geo_gamma<real>(G), gm1 = gam - real(1);
  const int lb = threadIdx.x / COLS, tc = threadIdx.x % COLS;
  const int leaf = blockIdx.x * LPB + lb;
  const bool active = leaf < a.nleaves;
  const int ic = tc % B, jc = tc / B;
  const int lim = a.limiter;
  const int lev = active ? a.level[leaf] : 1;
  real dx[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) dx[d] = geo_dx<real>(G, lev, d);

  // load plane z (-2 .. B+1) of this leaf into ring slot; interior planes get x/y ghosts
  auto load_plane = [&](int z, real (&Ucol)[NV], bool keep) {
    real* Wp = &S.W[lb][(z + 4) & 3][0][0];
    real Uv[NV], Vv[NV];
    if (z >= 0 && z < B) {
      int cell = tc + COLS * z;
#pragma unroll
      for (int v = 0; v < NV; ++v) Uv[v] = a.Us[((size_t)leaf * NV + v) * NC + cell];
      if (keep)
#pragma unroll
        for (int v = 0; v < NV; ++v) Ucol[v] = Uv[v];
    } else {
      int f = z < 0 ? 4 : 5;
      int m = z < 0 ? -1 - z : z - B;
#pragma unroll
      for (int v = 0; v < NV; ++v) Uv[v] = fetch_ghost<real, 3, B>(a.Us, a.slabs, a.nb, leaf, f, m, tc, v);
    }
    cons_to_prim<real, 3>(Uv, Vv, gm1);
#pragma unroll
    for (int v = 0; v < NV; ++v) Wp[v * P * P + (jc + 2) * P + (ic + 2)] = Vv[v];
    if (z >= 0 && z < B) {
      // x/y ghosts of this plane: faces 0..3, 2 layers, B cells along the other in-plane axis
      for (int h = tc; h < 4 * 2 * B; h += COLS) {
        int f = h / (2 * B), m = (h / B) % 2, s = h % B;
        int d = f >> 1, side = f & 1;
        int t = d == 0 ? s + B * z : s + B * z;  // tangential (t1 = other in-plane axis, t2 = z)
        real Ug[NV], Vg[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) Ug[v] = fetch_ghost<real, 3, B>(a.Us, a.slabs, a.nb, leaf, f, m, t, v);
        cons_to_prim<real, 3>(Ug, Vg, gm1);
        int n = side == 0 ? -1 - m : B + m;
        int pi = d == 0 ? n : s, pj = d == 0 ? s : n;
#pragma unroll
        for (int v = 0; v < NV; ++v) Wp[v * P * P + (pj + 2) * P + (pi + 2)] = Vg[v];
      }
    }
  };

  auto zflux = [&](int kface, real* F) {  // face between cells kface-1 and kface
    real Wl[4][NV];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const real* Wp = &S.W[lb][(kface - 2 + s + 4) & 3][0][0];
#pragma unroll
      for (int v = 0; v < NV; ++v) Wl[s][v] = Wp[v * P * P + (jc + 2) * P + (ic + 2)];
    }
    real VL[NV], VR[NV];
    face_states<real, 3>(lim, Wl, VL, VR);
    riemann<real, 3, FLUX>(2, VL, VR, gam, gm1, F);
  };

  real Uk0[NV], Uk1[NV], Uk2[NV];  // conserved values of planes k, k+1, k+2 of this column
  real rate = real(0);
  double sums[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) sums[v] = 0.0;
  int bad = 0;

  if (active) {
    load_plane(-2, Uk2, false);
    load_plane(-1, Uk2, false);
    load_plane(0, Uk0, true);
    load_plane(1, Uk1, true);
  }
  __syncthreads();
  if (active) {
    real F[NV];
    zflux(0, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) S.FZ[lb][v][tc] = F[v];
    if (a.has_ffx) {
      int slot = a.ffx[leaf * 6 + 4];
      if (slot >= 0)
#pragma unroll
        for (int v = 0; v < NV; ++v) a.fflux[((size_t)slot * NV + v) * NT + tc] = F[v];
    }
  }
  for (int k = 0; k < B; ++k) {
    // ring: slot of plane k-2 is reused for plane k+2
    __syncthreads();
    if (active) load_plane(k + 2, Uk2, k + 2 < B);
    __syncthreads();
    real Fz[NV];
    if (active) {
      zflux(k + 1, Fz);
      if (a.has_ffx && k == B - 1) {
        int slot = a.ffx[leaf * 6 + 5];
        if (slot >= 0)
#pragma unroll
          for (int v = 0; v < NV; ++v) a.fflux[((size_t)slot * NV + v) * NT + tc] = Fz[v];
      }
      // x and y faces of plane k
      const real* Wp = &S.W[lb][(k + 4) & 3][0][0];
      for (int idx = tc; idx < 2 * B * (B + 1); idx += COLS) {
        int dim = idx / (B * (B + 1)), fl = idx % (B * (B + 1));
        int fi = fl % (B + 1), fj = fl / (B + 1);
        real Wl[4][NV];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          int c = fi - 2 + s;
          int q = dim == 0 ? (fj + 2) * P + (c + 2) : (c + 2) * P + (fj + 2);
#pragma unroll
          for (int v = 0; v < NV; ++v) Wl[s][v] = Wp[v * P * P + q];
        }
        real VL[NV], VR[NV], F[NV];
        face_states<real, 3>(lim, Wl, VL, VR);
        riemann<real, 3, FLUX>(dim, VL, VR, gam, gm1, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) S.FX[lb][dim][v][fl] = F[v];
        if (a.has_ffx && (fi == 0 || fi == B)) {
          int slot = a.ffx[leaf * 6 + 2 * dim + (fi == 0 ? 0 : 1)];
          if (slot >= 0)
#pragma unroll
            for (int v = 0; v < NV; ++v) a.fflux[((size_t)slot * NV + v) * NT + fj + B * k] = F[v];
        }
      }
    }
    __syncthreads();
    if (active) {
      const real* Uk = Uk0;
      int cell = tc + COLS * k;
      real Un[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real div = real(0);
        div = div + (S.FX[lb][0][v][jc * (B + 1) + ic + 1] - S.FX[lb][0][v][jc * (B + 1) + ic]) / dx[0];
        div = div + (S.FX[lb][1][v][ic * (B + 1) + jc + 1] - S.FX[lb][1][v][ic * (B + 1) + jc]) / dx[1];
        div = div + (Fz[v] - S.FZ[lb][v][tc]) / dx[2];
        real tmp = Uk[v] - dtr * div;
        Un[v] = a.stage1 ? tmp : ssp_combine(a.alpha, a.beta, a.U0[((size_t)leaf * NV + v) * NC + cell], tmp);
        a.out[((size_t)leaf * NV + v) * NC + cell] = Un[v];
        S.FZ[lb][v][tc] = Fz[v];
      }
      if (a.fuse_reduce) {
        rate = fmax(rate, cell_rate<real, 3>(Un, gam, gm1, dx, &bad));
        double dV = G.dV[lev];
#pragma unroll
        for (int v = 0; v < NV; ++v) sums[v] += (double)Un[v] * dV;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Uk0[v] = Uk1[v];
        Uk1[v] = Uk2[v];
      }
    }
  }
  if (a.fuse_reduce)
    block_reduce_finish<real, NV, 256>(rate, sums, blockIdx.x * LPB, LPB, lb, G, a.ctl, a.partials, a.gpart,
                                       a.gcount, a.nleaves, true, dt, bad);
}

// ========================================================= reduce kernel ==
// Max signal rate and FP64 totals of the current state (after set_state, a
// regrid, or the refluxed last stage of a step on a tree with level jumps).
// Shape of a 256-thread CTA: CPT cells per thread, TPL threads per leaf, LPB leaves per
// CTA (16^2 leaves: 4 cells per thread and 4 leaves per CTA, so that the block-wide
// reduction is amortised over 1024 cells).
template <int NC>
struct ReduceShape {
  static constexpr int CPT = NC == 256 ? 4 : (NC > 256 ? NC / 256 : 1);
  static constexpr int TPL = NC / CPT;
  static constexpr int LPB = 256 / TPL;
};

// error-free sum a + b = s + e (TwoSum, Knuth), accumulated into the pair (hi, lo)
__device__ __forceinline__ void twosum_acc(float& hi, float& lo, float x) {
  const float s = hi + x, bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

// (hi, lo) += (h2, l2) for float-float accumulators (TwoSum of the high parts)
__device__ __forceinline__ void ff_acc(float& hi, float& lo, float h2, float l2) {
  const float s = hi + h2, bb = s - hi;
  lo = lo + l2 + ((hi - (s - bb)) + (h2 - bb));
  hi = s;
}

template <typename real, int ND, int B>
__global__ void __launch_bounds__(256) reduce_kernel(const real* __restrict__ U, const int* __restrict__ level,
                                                     Geometry G, DevCtl* ctl, double* partials, double* gpart,
                                                     unsigned* gcount, int nleaves, int advance) {
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC;
  constexpr int TPL = ReduceShape<NC>::TPL, LPB = ReduceShape<NC>::LPB;
  const int lb = threadIdx.x / TPL, tc = threadIdx.x % TPL;
  const int leaf = blockIdx.x * LPB + lb;
  const real gam = geo_gamma<real>(G), gm1 = gam - real(1);
  real rate = real(0);
  double sums[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) sums[v] = 0.0;
  int bad = 0;
  double dt = cta_stage_dt(ctl, nullptr);
  if (leaf < nleaves) {
    int lev = level[leaf];
    real dx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) dx[d] = geo_dx<real>(G, lev, d);
    // float32 state: per-thread sums as float-float pairs (TwoSum), widened once per thread,
    // so the float64 pipe (GB300's scarcest) is not touched per cell; float64 state: plain sums
    float hi[NV], lo[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) hi[v] = lo[v] = 0.f;
    // cells tc, tc + TPL, ... in that order; the loads of RB consecutive cells of the thread are
    // issued together so that a thread keeps RB x NV loads in flight
    constexpr int CPT = NC / TPL, RB = CPT % 4 == 0 && sizeof(real) == 4 ? 4 : (CPT % 2 == 0 ? 2 : 1);
    static_assert(NC % (RB * TPL) == 0, "cells per thread split into whole batches");
    const real* Ul = U + (size_t)leaf * NV * NC;
    for (int c0 = tc; c0 < NC; c0 += RB * TPL) {
      real Ub[RB][NV];
#pragma unroll
      for (int k = 0; k < RB; ++k)
#pragma unroll
        for (int v = 0; v < NV; ++v) Ub[k][v] = Ul[(size_t)v * NC + c0 + k * TPL];
#pragma unroll
      for (int k = 0; k < RB; ++k) {
        rate = fmax(rate, cell_rate<real, ND>(Ub[k], gam, gm1, dx, &bad));
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if constexpr (sizeof(real) == 4) twosum_acc(hi[v], lo[v], Ub[k][v]);
          else sums[v] += (double)Ub[k][v];
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if constexpr (sizeof(real) == 4) sums[v] = (double)hi[v] + (double)lo[v];
      sums[v] *= G.dV[lev];  // one cell volume per leaf
    }
  }
  block_reduce_finish<real, NV, 256>(rate, sums, blockIdx.x * LPB, LPB, lb, G, ctl, partials, gpart, gcount,
                                     nleaves, advance != 0, dt, bad);
}

// Float32 reduction for leaves of >= 1024 cells.  Items are quarters (NC / 1024 parts) of
// leaves; a grid of resident CTAs walks them (CTA b takes items b, b + grid, ...), four
// consecutive cells per thread read as one float4 per variable, the next item's loads issued
// before the current one is reduced.  Cell values are scaled by the exact power of two
// dV(level) / dV(1) so that one float-float (TwoSum) sum per thread and variable serves every
// level; the sums stay float-float through the warp butterflies and the fixed-order combination
// of the warps, and one thread widens the CTA's sums to float64 and scales them by dV(1)
// (GB300's float64 pipe is too narrow for per-thread float64 work).  Each CTA writes one
// partial; the two-level finish sums the partials in CTA order, so the result depends on the
// grid size only.
template <int ND, int B>
__global__ void __launch_bounds__(256, 3) reduce_split_kernel(const float* __restrict__ U, const int* __restrict__ level,
                                                           Geometry G, DevCtl* ctl, double* partials, double* gpart,
                                                           unsigned* gcount, int nleaves, int advance) {
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC, CPL = NC / 1024;
  static_assert(NC % 1024 == 0, "four cells per thread, 256 threads per CTA");
  __shared__ float red[8][2 * NV + 1];
  __shared__ int sbad;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int items = nleaves * CPL;
  auto load = [&](int it, float4* q) {
    const int leaf = it / CPL, part = it - leaf * CPL;
    const float* Ul = U + (size_t)leaf * NV * NC + (part * 256 + threadIdx.x) * 4;
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = __ldg(reinterpret_cast<const float4*>(Ul + (size_t)v * NC));
  };
  float4 q[NV], qn[NV];
  int it = blockIdx.x;
  if (it < items) load(it, q);
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();  // orders sbad (the step's dt, when advancing, is read by the finishing thread)
  const float gam = G.gammaf, gm1 = gam - 1.f;
  float rate = 0.f, hi[NV], lo[NV];
  int bad = 0;
#pragma unroll
  for (int v = 0; v < NV; ++v) hi[v] = lo[v] = 0.f;
  for (; it < items; it += gridDim.x) {
    const int nx = it + (int)gridDim.x;
    if (nx < items) load(nx, qn);
    const int lev = level[it / CPL];
    const float vscale = __int_as_float((127 - ND * (lev - 1)) << 23);  // dV(lev) / dV(1), exact
    float dx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) dx[d] = geo_dx<float>(G, lev, d);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float Uc[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Uc[v] = k == 0 ? q[v].x : k == 1 ? q[v].y : k == 2 ? q[v].z : q[v].w;
      rate = fmaxf(rate, cell_rate<float, ND>(Uc, gam, gm1, dx, &bad));
#pragma unroll
      for (int v = 0; v < NV; ++v) twosum_acc(hi[v], lo[v], Uc[v] * vscale);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = qn[v];
  }
  if (bad) sbad = 1;
  for (int o = 16; o > 0; o >>= 1) {
    rate = fmaxf(rate, __shfl_xor_sync(0xffffffffu, rate, o));
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float h2 = __shfl_xor_sync(0xffffffffu, hi[v], o), l2 = __shfl_xor_sync(0xffffffffu, lo[v], o);
      ff_acc(hi[v], lo[v], h2, l2);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) red[warp][v] = hi[v], red[warp][NV + v] = lo[v];
    red[warp][2 * NV] = rate;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = red[0][2 * NV];
    for (int w = 1; w < 8; ++w) {
      mm = fmaxf(mm, red[w][2 * NV]);
#pragma unroll
      for (int v = 0; v < NV; ++v) ff_acc(hi[v], lo[v], red[w][v], red[w][NV + v]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) partials[(size_t)blockIdx.x * NV + v] = ((double)hi[v] + (double)lo[v]) * G.dV[1];
    __threadfence();  // the partial is visible before the group counter counts this CTA
    atomicMax(&ctl->smax_bits, MaxKey<float>::enc(mm));
    if (sbad) atomicOr(&ctl->status, 1);
  }
  last_cta_finish<float, NV, 256>(ctl, partials, gpart, gcount, (int)gridDim.x, 1, advance != 0, 0.0, false, true);
}

// ====================================================== ghost slab fill ==
// One CTA per slab.  Restriction: mean of the 2^ndim fine cells (x-fastest sum).
// Prolongation: q_p + 1/4 sum_e sigma_e s_e, minmod slopes; normal inner
// neighbour = restriction of the target leaf; tangential neighbours outside the
// coarse leaf give s_e = 0.  The face direction D is a template parameter so that
// every cell index is formed in registers; runs of consecutive x cells are read as
// one vector (4 fine layers of an x face, x pairs otherwise).

// n consecutive values at p (p aligned to n * sizeof(real), or to 16 bytes for double)
template <typename real>
__device__ __forceinline__ void ld_run4(const real* p, real* o) {
  if constexpr (sizeof(real) == 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = a.x, o[1] = a.y, o[2] = a.z, o[3] = a.w;
  } else {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
  }
}
template <typename real>
__device__ __forceinline__ void ld_run2(const real* p, real* o) {
  if constexpr (sizeof(real) == 4) {
    const float2 a = __ldg(reinterpret_cast<const float2*>(p));
    o[0] = a.x, o[1] = a.y;
  } else {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = a.x, o[1] = a.y;
  }
}
template <typename real>
__device__ __forceinline__ void st_run2(real* p, real a, real b) {
  if constexpr (sizeof(real) == 4) *reinterpret_cast<float2*>(p) = make_float2(a, b);
  else *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

// the tangential dimensions of face direction D (E1 < E2; -1 where ND has none)
template <int ND, int D>
struct FaceDims {
  static constexpr int E1 = ND < 2 ? -1 : (D == 0 ? 1 : 0);
  static constexpr int E2 = ND < 3 ? -1 : (D == 2 ? 1 : 2);
};

template <int ND, int B, int D>
__device__ __forceinline__ int face_cell(int n, int a1, int a2) {
  constexpr int E1 = FaceDims<ND, D>::E1, E2 = FaceDims<ND, D>::E2;
  int x[3] = {0, 0, 0};
  x[D] = n;
  if constexpr (E1 >= 0) x[E1] = a1;
  if constexpr (E2 >= 0) x[E2] = a2;
  return x[0] + B * (x[1] + B * x[2]);
}

// restriction ghosts of one (tangential cell t, variable v) of a slab, both layers
template <typename real, int ND, int B, int D>
__device__ __forceinline__ void ghost_restrict(const real* __restrict__ U, real* __restrict__ slab,
                                               const SlabDesc& S, int t, int v) {
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC, NT = Tile<ND, B>::NT;
  constexpr int E1 = FaceDims<ND, D>::E1, E2 = FaceDims<ND, D>::E2;
  constexpr int NA = E1 >= 0 ? 2 : 1, NB = E2 >= 0 ? 2 : 1;
  const int side = S.face & 1;
  const int t1 = E1 >= 0 ? t % B : 0, t2 = E2 >= 0 ? t / B : 0;
  const int q1 = t1 / (B / 2), q2 = t2 / (B / 2);
  const real* Uf = U + ((size_t)S.src[q1 + 2 * q2] * NV + v) * NC;
  const int f1 = 2 * t1 - q1 * B, f2 = 2 * t2 - q2 * B;  // first fine cell along E1, E2
  const int n0 = side == 0 ? B - 4 : 0;                  // the four fine layers next to the face
  real c[4][2][2];  // [normal layer n0 + k][offset along E1][offset along E2]
  if constexpr (D == 0) {
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        real r[4];
        ld_run4(Uf + face_cell<ND, B, D>(n0, f1 + a, f2 + b), r);
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k][a][b] = r[k];
      }
  } else {  // E1 = 0: fine x pairs
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        real r[2];
        ld_run2(Uf + face_cell<ND, B, D>(n0 + k, f1, f2 + b), r);
        c[k][0][b] = r[0], c[k][1][b] = r[1];
      }
  }
  // mean over the 2^ND fine cells of the layer pair starting at normal offset kb, x fastest
  auto mean = [&](int kb) {
    real sum = real(0);
#pragma unroll
    for (int o = 0; o < (1 << ND); ++o) {
      const int k = kb + ((o >> D) & 1);
      const int a = E1 >= 0 ? (o >> E1) & 1 : 0, b = E2 >= 0 ? (o >> E2) & 1 : 0;
      sum = sum + c[k][a][b];
    }
    return sum * (real(1) / real(1 << ND));
  };
  const real lo = mean(0), hi = mean(2);
  // layer m = 0 is the one next to the face: fine layers B-2, B-1 (side 0) or 0, 1 (side 1)
  slab[((size_t)v * 2 + 0) * NT + t] = side == 0 ? hi : lo;
  slab[((size_t)v * 2 + 1) * NT + t] = side == 0 ? lo : hi;
}

// prolongation ghosts of one (coarse face cell qc, variable v): 2 layers x 2^(ND-1) fine cells
template <typename real, int ND, int B, int D>
__device__ __forceinline__ void ghost_prolong(const real* __restrict__ U, real* __restrict__ slab,
                                              const SlabDesc& S, int qc, int v) {
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC, NT = Tile<ND, B>::NT, HB = B / 2;
  constexpr int E1 = FaceDims<ND, D>::E1, E2 = FaceDims<ND, D>::E2;
  constexpr int NA = E1 >= 0 ? 2 : 1, NB = E2 >= 0 ? 2 : 1;
  const int side = S.face & 1;
  const int c1 = E1 >= 0 ? qc % HB : 0, c2 = E2 >= 0 ? qc / HB : 0;  // the target's coarse cell
  const int p1 = S.off[0] + c1, p2 = S.off[1] + c2;                  // the coarse cell in its leaf
  const int pn = side == 0 ? B - 1 : 0;
  const real* Uc = U + ((size_t)S.src[0] * NV + v) * NC;
  const real* Ut = U + ((size_t)S.target * NV + v) * NC;
  const real qp = __ldg(Uc + face_cell<ND, B, D>(pn, p1, p2));
  const real away = __ldg(Uc + face_cell<ND, B, D>(side == 0 ? pn - 1 : pn + 1, p1, p2));
  // restriction of the target's fine cells next to the face (normal inner neighbour)
  const int fn = side == 0 ? 0 : B - 2;
  real g[2][2][2];  // [normal offset][offset along E1][offset along E2]
  if constexpr (D == 0) {
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        real r[2];
        ld_run2(Ut + face_cell<ND, B, D>(fn, 2 * c1 + a, 2 * c2 + b), r);
        g[0][a][b] = r[0], g[1][a][b] = r[1];
      }
  } else {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        real r[2];
        ld_run2(Ut + face_cell<ND, B, D>(fn + k, 2 * c1, 2 * c2 + b), r);
        g[k][0][b] = r[0], g[k][1][b] = r[1];
      }
  }
  real inner = real(0);
#pragma unroll
  for (int o = 0; o < (1 << ND); ++o) {
    const int k = (o >> D) & 1;
    const int a = E1 >= 0 ? (o >> E1) & 1 : 0, b = E2 >= 0 ? (o >> E2) & 1 : 0;
    inner = inner + g[k][a][b];
  }
  inner = inner * (real(1) / real(1 << ND));
  real sl[3] = {real(0), real(0), real(0)};
  sl[D] = side == 0 ? minmod2(qp - away, inner - qp) : minmod2(qp - inner, away - qp);
  if constexpr (E1 >= 0) {
    const bool ok = p1 >= 1 && p1 + 1 < B;
    sl[E1] = ok ? minmod2(qp - __ldg(Uc + face_cell<ND, B, D>(pn, p1 - 1, p2)),
                          __ldg(Uc + face_cell<ND, B, D>(pn, p1 + 1, p2)) - qp)
                : real(0);
  }
  if constexpr (E2 >= 0) {
    const bool ok = p2 >= 1 && p2 + 1 < B;
    sl[E2] = ok ? minmod2(qp - __ldg(Uc + face_cell<ND, B, D>(pn, p1, p2 - 1)),
                          __ldg(Uc + face_cell<ND, B, D>(pn, p1, p2 + 1)) - qp)
                : real(0);
  }
  // fine ghost (layer m, offsets a, b along E1, E2): sigma_e = +1 on the upper fine half
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      real val[2];
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        real acc = real(0);
#pragma unroll
        for (int e = 0; e < ND; ++e) {
          real sg;
          if (e == D) sg = (side == 0) == (m == 0) ? real(1) : real(-1);
          else sg = ((e == E1 ? a : b) == 1) ? real(1) : real(-1);
          acc = acc + sg * sl[e];
        }
        val[a] = qp + real(0.25) * acc;
      }
      real* o = slab + ((size_t)v * 2 + m) * NT;
      if constexpr (NA == 2) st_run2(o + (2 * c1) + B * (2 * c2 + b), val[0], val[1]);
      else o[0] = val[0];
    }
}

template <int ND, int B>
struct GhostShape {
  static constexpr int NV = ND + 2, HB = B / 2;
  static constexpr int NCC = ND == 1 ? 1 : (ND == 2 ? HB : HB * HB);  // coarse cells of a prolongation slab
  static constexpr int THREADS = (NCC * NV + 31) / 32 * 32;
};

template <typename real, int ND, int B>
__global__ void __launch_bounds__(GhostShape<ND, B>::THREADS)
ghost_fill_kernel(const real* __restrict__ U, real* __restrict__ slabs, const SlabDesc* __restrict__ desc,
                  int nslabs) {
  constexpr int NV = ND + 2, NT = Tile<ND, B>::NT;
  constexpr int NCC = GhostShape<ND, B>::NCC, NTH = GhostShape<ND, B>::THREADS;
  const int s = blockIdx.x;
  if (s >= nslabs) return;
  const SlabDesc S = desc[s];
  real* slab = slabs + (size_t)s * NV * 2 * NT;
  const int d = S.face >> 1;
  if (S.kind == 0) {
    // (tangential cell, variable) items, NT * NV of them, strided over the CTA
#pragma unroll
    for (int i = 0; i < (NT * NV + NTH - 1) / NTH; ++i) {
      const int q = threadIdx.x + i * NTH;
      if (q < NT * NV) {
        const int t = q % NT, v = q / NT;
        if (d == 0) ghost_restrict<real, ND, B, 0>(U, slab, S, t, v);
        else if constexpr (ND >= 2) {
          if (d == 1) ghost_restrict<real, ND, B, 1>(U, slab, S, t, v);
          else if constexpr (ND == 3) ghost_restrict<real, ND, B, 2>(U, slab, S, t, v);
        }
      }
    }
    return;
  }
  const int q = threadIdx.x;
  if (q >= NCC * NV) return;
  const int qc = q % NCC, v = q / NCC;
  if (d == 0) ghost_prolong<real, ND, B, 0>(U, slab, S, qc, v);
  else if constexpr (ND >= 2) {
    if (d == 1) ghost_prolong<real, ND, B, 1>(U, slab, S, qc, v);
    else if constexpr (ND == 3) ghost_prolong<real, ND, B, 2>(U, slab, S, qc, v);
  }
}

// ================================================================ reflux ==
// Coarse cell next to a level jump: out += +-beta*dt/dx_c*(mean fine flux - coarse flux).
template <typename real, int ND, int B>
__device__ __forceinline__ real reflux_corr(const real* __restrict__ fflux, const RefluxRec& R, int t, int v,
                                            real dxc, real dtr, real beta) {
  constexpr int NV = ND + 2, NT = Tile<ND, B>::NT;
  int d = R.face >> 1;
  int e1 = -1, e2 = -1;
  for (int e = 0; e < ND; ++e)
    if (e != d) {
      if (e1 < 0) e1 = e; else e2 = e;
    }
  int t1 = e1 >= 0 ? t % B : 0, t2 = e2 >= 0 ? t / B : 0;
  int q1 = t1 / (B / 2), q2 = t2 / (B / 2);
  int fs = R.fslot[q1 + 2 * q2];
  real sum = real(0);
  int n2 = ND > 2 ? 2 : 1, n1 = ND > 1 ? 2 : 1;
  for (int o2 = 0; o2 < n2; ++o2)
    for (int o1 = 0; o1 < n1; ++o1) {
      int f1 = 2 * t1 + o1 - q1 * B, f2 = 2 * t2 + o2 - q2 * B;
      int tf = ND == 1 ? 0 : (ND == 2 ? f1 : f1 + B * f2);
      sum = sum + fflux[((size_t)fs * NV + v) * NT + tf];
    }
  real mean = sum * (real(1) / real(1 << (ND - 1)));
  real Fc = fflux[((size_t)R.cslot * NV + v) * NT + t];
  return beta * dtr * (mean - Fc) / dxc;
}

// One thread per (record, variable, tangential cell).  A cell at a leaf edge or corner
// borders level jumps through several faces of its leaf: the thread of the first such
// record (faces ascending, i.e. x before y before z) applies all of them in that
// order and the others skip the cell, so every cell has one writer.
template <typename real, int ND, int B>
__global__ void reflux_kernel(real* __restrict__ out, const real* __restrict__ fflux, const RefluxRec* __restrict__ rec,
                              int nrec, const int* __restrict__ level, Geometry G, const DevCtl* ctl, real beta) {
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC, NT = Tile<ND, B>::NT;
  long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float dtf;
  double dt = cta_stage_dt(ctl, &dtf);
  if (gid >= (long long)nrec * NV * NT) return;
  if (!(dt > 0.0)) return;
  const real dtr = sizeof(real) == 4 ? (real)dtf : (real)dt;
  int t = gid % NT, v = (gid / NT) % NV, r = gid / (NT * NV);
  const RefluxRec R = rec[r];
  const int cell = compose_cell<ND, B>(R.face >> 1, (R.face & 1) ? B - 1 : 0, t);
  const int x[3] = {cell % B, ND > 1 ? (cell / B) % B : 0, ND > 2 ? cell / (B * B) : 0};
  auto touches = [&](int face) { return x[face >> 1] == ((face & 1) ? B - 1 : 0); };
  for (int k = R.first; k < r; ++k)
    if (touches(rec[k].face)) return;
  const int lev = level[R.coarse];
  const size_t o = ((size_t)R.coarse * NV + v) * NC + cell;
  real val = out[o];
  for (int k = r; k < R.last; ++k) {
    const RefluxRec K = rec[k];
    if (k > r && !touches(K.face)) continue;
    const int dk = K.face >> 1;
    // tangential index of the cell on face dk (the inverse of compose_cell)
    const int tk = ND == 1 ? 0 : (ND == 2 ? x[dk == 0 ? 1 : 0] : (dk == 0 ? x[1] + B * x[2] : (dk == 1 ? x[0] + B * x[2] : x[0] + B * x[1])));
    const real corr = reflux_corr<real, ND, B>(fflux, K, tk, v, geo_dx<real>(G, lev, dk), dtr, beta);
    val = (K.face & 1) == 0 ? val + corr : val - corr;
  }
  out[o] = val;
}

// ============================================================ estimator ==
// Lohner-type estimator per direction: |q+ - 2 q0 + q-| over |q+ - q0| + |q0 - q-|
// + eps (|q+| + 2|q0| + |q-|), squares summed over directions, sqrt; max over the
// selected primitive variables and the leaf's cells.  Evaluated in float64.
template <typename real, int ND, int B>
__global__ void __launch_bounds__(256) lohner_kernel(const real* __restrict__ U, const real* __restrict__ slabs,
                                                     const int* __restrict__ nb, double gamma, double eps,
                                                     unsigned mask, double* err, int nleaves) {
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC;
  constexpr int TPL = NC >= 256 ? 256 : NC;  // threads per leaf
  constexpr int LPB = 256 / TPL;
  const int lb = threadIdx.x / TPL, tc = threadIdx.x % TPL;
  const int leaf = blockIdx.x * LPB + lb;
  double emax = 0.0;
  const double gm1 = gamma - 1.0;
  if (leaf < nleaves) {
    for (int c = tc; c < NC; c += TPL) {
      int ci[3] = {c % B, ND > 1 ? (c / B) % B : 0, ND > 2 ? c / (B * B) : 0};
      double Uq[NV], Vc[NV], Vm[3][NV], Vp[3][NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Uq[v] = (double)U[((size_t)leaf * NV + v) * NC + c];
      cons_to_prim<double, ND>(Uq, Vc, gm1);
      for (int d = 0; d < ND; ++d) {
        for (int s = 0; s < 2; ++s) {
          int cc[3] = {ci[0], ci[1], ci[2]};
          cc[d] += s == 0 ? -1 : 1;
          double Un[NV];
          if (cc[d] < 0 || cc[d] >= B) {
            int f = 2 * d + (cc[d] < 0 ? 0 : 1);
            int t = 0, k = 0;
            for (int e = 0; e < ND; ++e)
              if (e != d) {
                t += ci[e] * (k == 0 ? 1 : B);
                ++k;
              }
#pragma unroll
            for (int v = 0; v < NV; ++v) Un[v] = (double)fetch_ghost<real, ND, B>(U, slabs, nb, leaf, f, 0, t, v);
          } else {
            int cn = cc[0] + B * (cc[1] + B * cc[2]);
#pragma unroll
            for (int v = 0; v < NV; ++v) Un[v] = (double)U[((size_t)leaf * NV + v) * NC + cn];
          }
          cons_to_prim<double, ND>(Un, s == 0 ? Vm[d] : Vp[d], gm1);
        }
      }
      double ecell = 0.0;
      for (int v = 0; v < NV; ++v) {
        if (!((mask >> v) & 1u)) continue;
        double num = 0.0, den = 0.0;
        for (int d = 0; d < ND; ++d) {
          double qm = Vm[d][v], q0 = Vc[v], qp = Vp[d][v];
          double d2 = qp - 2.0 * q0 + qm;
          double d1 = fabs(qp - q0) + fabs(q0 - qm) + eps * (fabs(qp) + 2.0 * fabs(q0) + fabs(qm));
          num = num + d2 * d2;
          den = den + d1 * d1;
        }
        double e = den > 0.0 ? sqrt(num / den) : 0.0;
        ecell = fmax(ecell, e);
      }
      emax = fmax(emax, ecell);
    }
  }
  // max within the leaf's threads
  __shared__ double sm[256];
  sm[threadIdx.x] = emax;
  __syncthreads();
  for (int w = TPL / 2; w > 0; w >>= 1) {
    if (tc < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
    __syncthreads();
  }
  if (tc == 0 && leaf < nleaves) err[leaf] = sm[threadIdx.x];
}

// Same estimator with each primitive value computed once: one CTA per leaf converts the leaf's
// cells and its face ghosts (layer 0) to primitive variables, keeps the nsel selected ones in
// a (B+2)^ND shared tile, then evaluates every cell from the tile.  On a float64 state the
// values and the arithmetic are those of lohner_kernel (which converts each cell up to 2 ND + 1
// times), so the result is the same bit for bit; a float32 state is evaluated in float32
// (GB300's float64 pipe made the float64 evaluation most of a regrid).  Dynamic shared memory
// nsel (B+2)^ND values of the state's type.
template <typename real, int ND, int B>
__global__ void __launch_bounds__(256) lohner_tile_kernel(const real* __restrict__ U, const real* __restrict__ slabs,
                                                          const int* __restrict__ nb, double gamma, double eps,
                                                          unsigned mask, double* err, int nleaves) {
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC, NT = Tile<ND, B>::NT, P1 = B + 2;
  constexpr int PT = ND == 2 ? P1 * P1 : P1 * P1 * P1;
  static_assert(ND >= 2, "2D and 3D leaves");
  extern __shared__ __align__(16) unsigned char lohner_smem[];
  using acc = real;  // float32 state: float32 estimator; float64 state: float64 (bit-exact with the oracle)
  acc* ptile = reinterpret_cast<acc*>(lohner_smem);  // [selected variable][(B+2)^ND], cell (i, j, k) at i+1 + P1 (j+1 + P1 (k+1))
  __shared__ acc wmax[8];
  const int leaf = blockIdx.x;
  if (leaf >= nleaves) return;
  int sel[NV], nsel = 0;
#pragma unroll
  for (int v = 0; v < NV; ++v)
    if ((mask >> v) & 1u) sel[nsel++] = v;
  const acc gm1 = acc(gamma) - acc(1), epsa = acc(eps);
  auto at = [&](int i, int j, int k) { return (i + 1) + P1 * ((j + 1) + (ND == 3 ? P1 * (k + 1) : 0)); };
  for (int c = threadIdx.x; c < NC; c += blockDim.x) {
    const int i = c % B, j = (c / B) % B, k = ND == 3 ? c / (B * B) : 0;
    acc Uq[NV], V[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Uq[v] = (acc)U[((size_t)leaf * NV + v) * NC + c];
    cons_to_prim<acc, ND>(Uq, V, gm1);
    for (int q = 0; q < nsel; ++q) ptile[q * PT + at(i, j, k)] = V[sel[q]];
  }
  for (int g = threadIdx.x; g < 2 * ND * NT; g += blockDim.x) {
    const int f = g / NT, t = g % NT, d = f >> 1, side = f & 1;
    int ci[3] = {0, 0, 0}, kk = 0;  // tangential coordinates in increasing direction order
    for (int e = 0; e < ND; ++e)
      if (e != d) {
        ci[e] = kk == 0 ? t % B : t / B;
        ++kk;
      }
    ci[d] = side == 0 ? -1 : B;
    acc Un[NV], V[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Un[v] = (acc)fetch_ghost<real, ND, B>(U, slabs, nb, leaf, f, 0, t, v);
    cons_to_prim<acc, ND>(Un, V, gm1);
    for (int q = 0; q < nsel; ++q) ptile[q * PT + at(ci[0], ci[1], ci[2])] = V[sel[q]];
  }
  __syncthreads();
  acc emax = acc(0);
  for (int c = threadIdx.x; c < NC; c += blockDim.x) {
    const int i = c % B, j = (c / B) % B, k = ND == 3 ? c / (B * B) : 0;
    acc ecell = acc(0);
    for (int q = 0; q < nsel; ++q) {
      const acc* P = ptile + q * PT;
      acc num = acc(0), den = acc(0);
      for (int d = 0; d < ND; ++d) {
        const int m[3] = {i - (d == 0), j - (d == 1), k - (d == 2)}, pp[3] = {i + (d == 0), j + (d == 1), k + (d == 2)};
        const acc qm = P[at(m[0], m[1], m[2])], q0 = P[at(i, j, k)], qp = P[at(pp[0], pp[1], pp[2])];
        acc d2 = qp - acc(2) * q0 + qm;
        acc d1 = fabs(qp - q0) + fabs(q0 - qm) + epsa * (fabs(qp) + acc(2) * fabs(q0) + fabs(qm));
        num = num + d2 * d2;
        den = den + d1 * d1;
      }
      acc e = den > acc(0) ? sqrt(num / den) : acc(0);
      ecell = fmax(ecell, e);
    }
    emax = fmax(emax, ecell);
  }
  for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = emax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) emax = fmax(emax, wmax[w]);
    err[leaf] = (double)emax;
  }
}

// =============================================================== regrid ==
// New leaf state: copy, limited prolongation from the old parent (its face
// ghosts give the slopes at its edges), or restriction from the old children.
template <typename real, int ND, int B>
__global__ void regrid_kernel(const real* __restrict__ Uold, real* __restrict__ Unew, const real* __restrict__ slabs,
                              const int* __restrict__ nb, const RegridOp* __restrict__ ops, int nnew) {
  constexpr int NV = ND + 2, NC = Tile<ND, B>::NC;
  long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)nnew * NC) return;
  int c = gid % NC;
  int nl = gid / NC;
  RegridOp op = ops[nl];
  int ci[3] = {c % B, ND > 1 ? (c / B) % B : 0, ND > 2 ? c / (B * B) : 0};
  for (int v = 0; v < NV; ++v) {
    real val;
    if (op.kind == 0) {
      val = Uold[((size_t)op.src[0] * NV + v) * NC + c];
    } else if (op.kind == 1) {
      int P = op.src[0];
      int pc[3] = {0, 0, 0};
      real sg[3];
      for (int e = 0; e < ND; ++e) {
        int oe = (op.child >> e) & 1;
        int f = oe * B + ci[e];
        pc[e] = f >> 1;
        sg[e] = (f & 1) ? real(1) : real(-1);
      }
      auto pval = [&](const int* q) -> real {
        for (int e = 0; e < ND; ++e) {
          if (q[e] < 0 || q[e] >= B) {
            int face = 2 * e + (q[e] < 0 ? 0 : 1);
            int t = 0, k = 0;
            for (int g = 0; g < ND; ++g)
              if (g != e) {
                t += q[g] * (k == 0 ? 1 : B);
                ++k;
              }
            return fetch_ghost<real, ND, B>(Uold, slabs, nb, P, face, 0, t, v);
          }
        }
        return Uold[((size_t)P * NV + v) * NC + q[0] + B * (q[1] + B * q[2])];
      };
      real qp = pval(pc);
      real acc = real(0);
      for (int e = 0; e < ND; ++e) {
        int m[3] = {pc[0], pc[1], pc[2]}, p[3] = {pc[0], pc[1], pc[2]};
        m[e] -= 1;
        p[e] += 1;
        real s = minmod2(qp - pval(m), pval(p) - qp);
        acc = acc + sg[e] * s;
      }
      val = qp + real(0.25) * acc;
    } else {
      int o[3] = {0, 0, 0};
      for (int e = 0; e < ND; ++e) o[e] = (2 * ci[e]) / B;
      int child = op.src[o[0] | (o[1] << 1) | (o[2] << 2)];
      real sum = real(0);
      for (int q = 0; q < (1 << ND); ++q) {
        int f[3] = {0, 0, 0};
        for (int e = 0; e < ND; ++e) f[e] = 2 * ci[e] - o[e] * B + ((q >> e) & 1);
        sum = sum + Uold[((size_t)child * NV + v) * NC + f[0] + B * (f[1] + B * f[2])];
      }
      val = sum * (real(1) / real(1 << ND));
    }
    Unew[((size_t)nl * NV + v) * NC + c] = val;
  }
}

// ============================================================ state I/O ==
// W may be device memory or pinned host memory read in place (zero copy); cells per leaf
// nc = 2^lognc >= 2.  Each thread converts two neighbouring cells with 16-byte loads, so
// that reads over the host link come in whole-sector requests.
template <typename real, int ND>
__global__ void set_state_kernel(const double* __restrict__ W, real* __restrict__ U, long long ncells_total, int lognc,
                                 int primitive, double gamma) {
  constexpr int NV = ND + 2;
  const long long pair = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gid = 2 * pair;
  if (gid >= ncells_total) return;
  const int nc = 1 << lognc;
  const long long leaf = gid >> lognc;
  const int c = (int)(gid & (nc - 1));
  double in[2][NV], o[2][NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double2 w = *reinterpret_cast<const double2*>(&W[(leaf * NV + v) * nc + c]);
    in[0][v] = w.x;
    in[1][v] = w.y;
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (primitive) prim_to_cons<double, ND>(in[k], o[k], gamma - 1.0);
    else
#pragma unroll
      for (int v = 0; v < NV; ++v) o[k][v] = in[k][v];
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    U[(leaf * NV + v) * nc + c] = (real)o[0][v];
    U[(leaf * NV + v) * nc + c + 1] = (real)o[1][v];
  }
}

// out may be device memory or pinned host memory written in place (zero copy).  One value
// per thread: over the host link, many 8-byte stores in flight measured 0.72 ms for 134 MB,
// two 16-byte stores per thread 1.6 ms.
template <typename real>
__global__ void read_state_kernel(const real* __restrict__ U, double* __restrict__ out, long long n) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid < n) out[gid] = (double)U[gid];
}

template <typename real, int ND, int B>
__global__ void face_ghost_dump_kernel(const real* __restrict__ U, const real* __restrict__ slabs,
                                       const int* __restrict__ nb, int leaf, double* out) {
  constexpr int NV = ND + 2, NT = Tile<ND, B>::NT;
  int gid = blockIdx.x * blockDim.x + threadIdx.x;
  int total = NV * 2 * ND * 2 * NT;
  if (gid >= total) return;
  int t = gid % NT, m = (gid / NT) % 2, f = (gid / (2 * NT)) % (2 * ND), v = gid / (2 * NT * 2 * ND);
  out[gid] = (double)fetch_ghost<real, ND, B>(U, slabs, nb, leaf, f, m, t, v);
}

}  // namespace amrgpu
