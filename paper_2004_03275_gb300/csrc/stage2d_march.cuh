// Float32 2D stage kernel for 16^2 leaves: one warp per leaf, directional marches.
//
// Same method as the other stage kernels (limited MUSCL on primitive variables,
// HLL/HLLC/TVDLF flux, SSPRK combination; Sec. 1.1, 1.2, 2.3-2.4), organised so
// that the stencil work of each direction stays in registers:
//   1. the warp loads the leaf (coalesced 16-byte loads) and its two-cell face
//      ghosts, converts every cell to primitive values once and stores them as
//      float4 in a shared tile T[20][21] (rows and columns -2..17, odd row stride);
//   2. x march: lane (row j, half h) walks columns h*8-2 .. h*8+9 of row j keeping
//      a three-cell window; at each step it forms the limited slope of one cell,
//      its two face values, the flux through one face and, one step later, the
//      flux difference of a cell, which goes to a shared array E[16][17];
//   3. y march: lane (column i, half h) walks rows h*8-2 .. h*8+9 of column i the
//      same way and finishes each cell: flux differences of both directions, the
//      SSPRK combination with U^(s) and U^n (coalesced scalar loads), the store,
//      and on the last stage the signal rate and the conserved totals.
// Every lane does identical work in every phase (the leaf-boundary faces are the
// first or last faces of a march), there is no block-wide barrier inside a leaf,
// and the two access patterns of T and E hit distinct banks (strides 21 and 17).
// Per cell: 1.5 primitive conversions (ghosts included), 1.25 slopes and 1.125
// fluxes per direction.
//
// Conserved totals on the last stage: every thread accumulates its cells in
// float-float (TwoSum), scaled by 4^-(level-1) so that all levels share one unit
// (dV halves exactly per level and per dimension); each warp adds its lanes by a
// fixed float-float butterfly, one warp adds the CTA's warps in order into one
// float64 partial per variable, and the last CTA to finish sums the partials in
// CTA order (one level up to kFlatFinishMax CTAs, else the two-level finish).  The
// result is deterministic for a given tree.
#pragma once
#include "stage2d_f32.cuh"
#include "tma.cuh"

namespace amrgpu {

constexpr int kMarchWarps = 4;     // warps (= leaves) per CTA of the last stage (its reduction's thread count)
constexpr int kMarchMaxWarps = 8;  // largest CTA of the first and middle stages (launch parameter)
constexpr int kFlatFinishMax = 4096;  // last stage: one-level finish up to this many CTAs

struct MarchSmem {
  float4 E[16][17];  // x flux differences of the interior cells, E[j][i]; before the x march it
                     // receives the leaf's conserved values [var][cell] from one TMA tensor copy
  float4 pad[4];     // keeps every warp's E 128-byte aligned (TMA destination)
  float4 T[20][21];  // primitive values, T[r+2][c+2], r, c in -2..17 (corners unused)
};
static_assert(sizeof(MarchSmem) % 128 == 0, "per-warp block must keep E 128-byte aligned");
constexpr unsigned kLeafBytes = 4 * 256 * 4;  // one 16^2 leaf, 4 variables, float32
constexpr int kTmaWaitLimit = 1 << 20;

namespace march {

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ float4 prim(float r, float mx, float my, float e, float gm1) {
  float ir = f32::rcp(r);
  float vx = mx * ir, vy = my * ir;
  return make_float4(r, vx, vy, gm1 * (e - 0.5f * (mx * vx + my * vy)));
}

// lower (toward -d) and upper (toward +d) face values of the cell w0 from its differences to the
// cell below, dm = w0 - wm, and to the cell above, dp = wp - w0; the limiter runs on the variable
// pairs (rho, v_x) and (v_y, p) with packed arithmetic
template <int LIM>
__device__ __forceinline__ void faces(const float4& w0, const float4& dm, const float4& dp, float4& lo, float4& hi) {
  using namespace f32;
  float2 hm, hp;
  const float2 a0 = make_float2(w0.x, w0.y), a1 = make_float2(w0.z, w0.w);
  half_slopes2<LIM>(make_float2(dm.x, dm.y), make_float2(dp.x, dp.y), hm, hp);
  const float2 l0 = sub2(a0, hm), h0 = add2(a0, hp);
  half_slopes2<LIM>(make_float2(dm.z, dm.w), make_float2(dp.z, dp.w), hm, hp);
  const float2 l1 = sub2(a1, hm), h1 = add2(a1, hp);
  lo = make_float4(l0.x, l0.y, l1.x, l1.y);
  hi = make_float4(h0.x, h0.y, h1.x, h1.y);
}

__device__ __forceinline__ float4 diff(const float4& a, const float4& b) {  // a - b, packed
  const float2 d0 = f32::sub2(make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 d1 = f32::sub2(make_float2(a.z, a.w), make_float2(b.z, b.w));
  return make_float4(d0.x, d0.y, d1.x, d1.y);
}

// flux through the face between cells a (left) and b (right) from face states L, R;
// first order (the cell values) if a reconstructed density or pressure is not
// positive (a warp-uniform branch, taken only when some lane needs it).  Result in
// variable order (rho, m_x, m_y, E).
template <int FLUX, bool ISY>
__device__ __forceinline__ void flux(float4 L, float4 R, const float4& a, const float4& b, float gam, float igm1,
                                     float* F) {
  const bool ok = L.x > 0.f && R.x > 0.f && L.w > 0.f && R.w > 0.f;
  if (__any_sync(0xffffffffu, !ok)) {
    if (!ok) {
      L = a;
      R = b;
    }
  }
  float G[4];
  if (ISY) {
    f32::flux2<FLUX>(L.x, L.z, L.y, L.w, R.x, R.z, R.y, R.w, gam, igm1, G);
    F[0] = G[0];
    F[1] = G[2];
    F[2] = G[1];
    F[3] = G[3];
  } else {
    f32::flux2<FLUX>(L.x, L.y, L.z, L.w, R.x, R.y, R.z, R.w, gam, igm1, G);
    F[0] = G[0];
    F[1] = G[1];
    F[2] = G[2];
    F[3] = G[3];
  }
}

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  float s = hi + x, bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

// TwoSum accumulation of a variable pair, packed; each element as two_sum_add
__device__ __forceinline__ void two_sum_add2(float2& hi, float2& lo, float2 x) {
  using namespace f32;
  const float2 s = add2(hi, x), bb = sub2(s, hi);
  lo = add2(lo, add2(sub2(hi, sub2(s, bb)), sub2(x, bb)));
  hi = s;
}

__device__ __forceinline__ void ff_add(float& hi, float& lo, float h2, float l2) {
  float s = hi + h2, bb = s - hi;
  float e = (hi - (s - bb)) + (h2 - bb);
  lo = lo + l2 + e;
  hi = s;
}

}  // namespace march

// SK: stage kind, fixed at compile time so every kernel carries only its own path
enum { kStageFirst = 0, kStageMid = 1, kStageLast = 2 };

// Launch: block 32 x NW threads (NW warps = leaves per CTA; the last stage takes
// kMarchWarps), dynamic shared memory NW x sizeof(MarchSmem) + 128 bytes of alignment
// slack; grid = leaf groups, or fewer CTAs that loop over the groups (persistent).  Every
// choice gives the same state bit for bit (the per-cell arithmetic does not depend on it).
// PERSIST: CTAs loop over the leaf groups (the last stage always does; its grid may still
// cover every group); without it each CTA takes one group and the kernel has no loop.
template <int FLUX, int LIM, int SK, bool PERSIST>
__global__ void __launch_bounds__(32 * kMarchMaxWarps, 2)
    stage2d_march_kernel(const __grid_constant__ StageArgs<float> a, const __grid_constant__ Geometry G,
                         const __grid_constant__ CUtensorMap tmU) {
  constexpr int B = 16, NC = B * B, NV = 4;
  constexpr bool FIRST = SK == kStageFirst, LAST = SK == kStageLast;
  // The leaf's conserved values arrive by one TMA tensor copy per leaf in the persistent
  // last stage, and by coalesced 16-byte loads of all 32 lanes in the other stages: the
  // copy measured ~1 us faster per launch in the former and ~3.5 us slower in the latter
  // (one 4 KB copy per warp against 256 requests in flight).
  constexpr bool TMA = LAST;
  extern __shared__ __align__(128) unsigned char march_smem_raw[];
  MarchSmem* S = reinterpret_cast<MarchSmem*>(march_smem_raw +
                                              ((128u - (tma::smem_addr(march_smem_raw) & 127u)) & 127u));
  __shared__ uint64_t tbar[kMarchMaxWarps];
  __shared__ float wrate[kMarchMaxWarps];
  __shared__ float wtot[2][kMarchWarps][4];  // last stage: per warp (hi, lo) of each variable
  __shared__ int sbad;
  const int NW = LAST ? kMarchWarps : (int)(blockDim.x >> 5);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lo16 = lane & 15, h = lane >> 4;
  MarchSmem& M = S[warp];
  if (threadIdx.x == 0) sbad = 0;  // before the barrier inside cta_stage_dt
  if (TMA && lane == 0) tma::bar_init(&tbar[warp], 1);
  __syncwarp();
  unsigned phase = 0;

  // Leaf groups (NW consecutive leaves, one per warp): CTA b takes groups b, b + gridDim.x,
  // ... in that order (one group when the grid covers them all).  On the last stage the
  // per-thread totals are so summed in a fixed order and the finish runs once per CTA.
  const int ngroups = (a.nleaves + NW - 1) / NW;
  int grp = blockIdx.x;
  int leaf = grp * NW + warp;
  bool active = leaf < a.nleaves;
  float gu[4][NV];
  float4 u[NV][2];
  int lev = 1;
  // ---- 1a. global loads of a leaf: its conserved values by one TMA tensor copy into E
  // (rows leaf*4 .. leaf*4+3 of the state viewed as [leaf*4 + var][256 cells]), and one
  // ghost cell per face and lane (layer m = h, tangential index t = lo16; faces x-, x+,
  // y-, y+).  Those of the first leaf are issued before the CTA's dt barrier.
  auto load_leaf = [&]() {
    if constexpr (TMA) {
      tma::fence_async_smem();  // every lane's earlier reads and writes of E come before the copy
      __syncwarp();
      if (lane == 0) {
        tma::bar_expect(&tbar[warp], kLeafBytes);
        tma::load_2d(&M.E[0][0], &tmU, 0, leaf * NV, &tbar[warp]);
      }
    } else {
      const float* Ul = a.Us + (size_t)leaf * NV * NC;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float4* p = reinterpret_cast<const float4*>(Ul + v * NC + lo16 * B + h * 8);
        u[v][0] = __ldg(p);
        u[v][1] = __ldg(p + 1);
      }
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int code = __ldg(&a.nb[leaf * 4 + f]);
      const int d = f >> 1, side = f & 1, m = h, t = lo16;
      const float* src;
      int stride;
      if (code >= -1) {
        int n = code >= 0 ? (side == 0 ? B - 1 - m : m) : (side == 0 ? 0 : B - 1);
        int cell = d == 0 ? n + B * t : t + B * n;
        src = a.Us + (size_t)(code >= 0 ? code : leaf) * NV * NC + cell;
        stride = NC;
      } else {
        src = a.slabs + ((size_t)(-2 - code) * NV * 2 + m) * B + t;
        stride = 2 * B;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) gu[f][v] = __ldg(&src[v * stride]);
    }
    lev = __ldg(&a.level[leaf]);
    // U^n of this leaf is read only by the y march, late: ask for it in L2 now (one 128-byte
    // line per lane), so that those loads find it there instead of in DRAM
    if (!FIRST) march::prefetch_l2(a.U0 + (size_t)leaf * NV * NC + lane * 32);
    // persistent last stage: the next group's leaf too, whose copy is issued only after this one
    if (LAST || PERSIST) {
      const int nl = (grp + (int)gridDim.x) * NW + warp;
      if (nl < a.nleaves) march::prefetch_l2(a.Us + (size_t)nl * NV * NC + lane * 32);
    }
  };
  if (active) load_leaf();
  // the first and middle stages read the float copy of dt (no float64 instruction); the last
  // stage, a few resident CTAs, keeps the float64 dt for its finish (fewer registers live)
  float dt;
  double dtd = 0.0;
  if constexpr (LAST) dtd = cta_stage_dt(a.ctl, &dt);
  else dt = cta_stage_dtf(a.ctl);
  if (!(dt > 0.f)) {  // no step to take; the first leaf's copy must land before the exit
    if (TMA && active) tma::bar_wait(&tbar[warp], phase, kTmaWaitLimit);
    return;
  }
  const float gam = G.gammaf, gm1 = gam - 1.f, igm1 = 1.f / gm1;

  float rate = 0.f;
  int bad = 0;
  float2 th[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, tl[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};

  while (true) {
    if (TMA && active) {
      bool landed = tma::bar_wait(&tbar[warp], phase, kTmaWaitLimit);
      if (!landed) {  // the copy did not land: report, wait once more for it, skip the leaf
        if (lane == 0) atomicOr(&a.ctl->status, 2);
        landed = tma::bar_wait(&tbar[warp], phase, kTmaWaitLimit);
        active = false;
      }
      if (landed) phase ^= 1u;
    }
    if (active) {
      const float* Ul = a.Us + (size_t)leaf * NV * NC;
      // ---- 1b. primitive tile
      {
        if constexpr (TMA) {
          const float4* e4 = reinterpret_cast<const float4*>(&M.E[0][0]);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            u[v][0] = e4[(v * NC + lo16 * B + h * 8) / 4];
            u[v][1] = e4[(v * NC + lo16 * B + h * 8) / 4 + 1];
          }
          __syncwarp();  // every lane has its cells before the tile (and later E) is written
        }
        float4* trow = &M.T[lo16 + 2][h * 8 + 2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          trow[4 * q + 0] = march::prim(u[0][q].x, u[1][q].x, u[2][q].x, u[3][q].x, gm1);
          trow[4 * q + 1] = march::prim(u[0][q].y, u[1][q].y, u[2][q].y, u[3][q].y, gm1);
          trow[4 * q + 2] = march::prim(u[0][q].z, u[1][q].z, u[2][q].z, u[3][q].z, gm1);
          trow[4 * q + 3] = march::prim(u[0][q].w, u[1][q].w, u[2][q].w, u[3][q].w, gm1);
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const int d = f >> 1, side = f & 1, m = h, t = lo16;
          int r, c;
          if (d == 0) {
            r = t;
            c = side == 0 ? -1 - m : B + m;
          } else {
            c = t;
            r = side == 0 ? -1 - m : B + m;
          }
          M.T[r + 2][c + 2] = march::prim(gu[f][0], gu[f][1], gu[f][2], gu[f][3], gm1);
        }
      }
      __syncwarp();

      const float idx = G.idxf[lev][0], idy = G.idxf[lev][1];
      const int c0 = h * 8;

      // ---- 2. x march along row j = lo16: flux differences of columns c0..c0+7 -> E
      {
        const int j = lo16;
        const float4* row = &M.T[j + 2][2];  // row[c] = W(c, j)
        float4 wm = row[c0 - 2], w0 = row[c0 - 1], wp = row[c0], wnext = row[c0 + 1];
        float4 dm = march::diff(w0, wm), dp = march::diff(wp, w0);
        float4 lo, hiPrev;
        march::faces<LIM>(w0, dm, dp, lo, hiPrev);  // cell c0-1: its upper face value
        wm = w0;
        w0 = wp;
        dm = dp;
        float Fp[NV];
#pragma unroll
        for (int k = 0; k <= 8; ++k) {
          const int cc = c0 + k;  // cell whose slope is formed; face cc-1/2
          wp = wnext;
          if (k < 8) wnext = row[cc + 2];
          dp = march::diff(wp, w0);
          float4 hi;
          march::faces<LIM>(w0, dm, dp, lo, hi);
          float F[NV];
          march::flux<FLUX, false>(hiPrev, lo, wm, w0, gam, igm1, F);
          if (a.has_ffx && ((h == 0 && k == 0) || (h == 1 && k == 8))) {
            int slot = a.ffx[leaf * 4 + h];
            if (slot >= 0)
#pragma unroll
              for (int v = 0; v < NV; ++v) a.fflux[((size_t)slot * NV + v) * B + j] = F[v];
          }
          if (k > 0)
            M.E[j][cc - 1] = march::diff(make_float4(F[0], F[1], F[2], F[3]), make_float4(Fp[0], Fp[1], Fp[2], Fp[3]));
#pragma unroll
          for (int v = 0; v < NV; ++v) Fp[v] = F[v];
          hiPrev = hi;
          wm = w0;
          w0 = wp;
          dm = dp;
        }
      }
      __syncwarp();

      // ---- 3. y march along column i = lo16, then the cell update of rows c0..c0+7
      {
        const int i = lo16;
        const float4* col = &M.T[2][i + 2];  // col[r * 21] = W(i, r)
        constexpr int RS = 21;
        float4 wm = col[(c0 - 2) * RS], w0 = col[(c0 - 1) * RS], wp = col[c0 * RS], wnext = col[(c0 + 1) * RS];
        float4 dm = march::diff(w0, wm), dp = march::diff(wp, w0);
        float4 lo, hiPrev;
        march::faces<LIM>(w0, dm, dp, lo, hiPrev);
        wm = w0;
        w0 = wp;
        dm = dp;
        float Fp[NV];
        const float* U0l = a.U0 + (size_t)leaf * NV * NC;
        float* Ol = a.out + (size_t)leaf * NV * NC;
        const float vscale = __int_as_float((127 - 2 * (lev - 1)) << 23);  // 4^-(lev-1), exact
        // U^(s) and U^n of the next cell to update, loaded one march step ahead
        float un[NV], u0n[NV], un2[NV], u0n2[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          un[v] = __ldg(&Ul[v * NC + c0 * B + i]);
          u0n[v] = FIRST ? 0.f : __ldg(&U0l[v * NC + c0 * B + i]);
          un2[v] = __ldg(&Ul[v * NC + (c0 + 1) * B + i]);
          u0n2[v] = FIRST ? 0.f : __ldg(&U0l[v * NC + (c0 + 1) * B + i]);
        }
#pragma unroll
        for (int k = 0; k <= 8; ++k) {
          const int rr = c0 + k;  // cell whose slope is formed; face rr-1/2
          wp = wnext;
          if (k < 8) wnext = col[(rr + 2) * RS];
          dp = march::diff(wp, w0);
          float4 hi;
          march::faces<LIM>(w0, dm, dp, lo, hi);
          float F[NV];
          march::flux<FLUX, true>(hiPrev, lo, wm, w0, gam, igm1, F);
          if (a.has_ffx && ((h == 0 && k == 0) || (h == 1 && k == 8))) {
            int slot = a.ffx[leaf * 4 + 2 + h];
            if (slot >= 0)
#pragma unroll
              for (int v = 0; v < NV; ++v) a.fflux[((size_t)slot * NV + v) * B + i] = F[v];
          }
          if (k > 0) {
            const int r = rr - 1, q = r * B + i;
            const float4 e = M.E[r][i];
            const float ex[NV] = {e.x, e.y, e.z, e.w};
            float uc[NV], u0c[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              uc[v] = un[v];
              u0c[v] = u0n[v];
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              un[v] = un2[v];
              u0n[v] = u0n2[v];
            }
            if (k < 7)
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                un2[v] = __ldg(&Ul[v * NC + q + 2 * B]);
                u0n2[v] = FIRST ? 0.f : __ldg(&U0l[v * NC + q + 2 * B]);
              }
            // div = E_x idx + (F - F_prev) idy; T = U^(s) - dt div; SSPRK: T + alpha (U^n - T); on the
            // variable pairs (rho, m_x) and (m_y, E), packed
            float Un[NV];
#pragma unroll
            for (int w = 0; w < 2; ++w) {
              using namespace f32;
              const float2 dF = sub2(make_float2(F[2 * w], F[2 * w + 1]), make_float2(Fp[2 * w], Fp[2 * w + 1]));
              const float2 div = fma2(make_float2(ex[2 * w], ex[2 * w + 1]), bc2(idx), mul2(dF, bc2(idy)));
              const float2 tmp = fma2(bc2(-dt), div, make_float2(uc[2 * w], uc[2 * w + 1]));
              const float2 un2 =
                  FIRST ? tmp : fma2(bc2(a.alpha), sub2(make_float2(u0c[2 * w], u0c[2 * w + 1]), tmp), tmp);
              Un[2 * w] = un2.x;
              Un[2 * w + 1] = un2.y;
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) Ol[v * NC + q] = Un[v];
            if constexpr (LAST) {
              float ir = f32::rcp(Un[0]);
              const float2 vv = f32::mul2(make_float2(Un[1], Un[2]), f32::bc2(ir));
              const float vx = vv.x, vy = vv.y;
              float p = gm1 * (Un[3] - 0.5f * (Un[1] * vx + Un[2] * vy));
              if (!(Un[0] > 0.f) || !(p > 0.f)) bad = 1;
              float cs = sqrtf(gam * p * ir);
              rate = fmaxf(rate, (fabsf(vx) + cs) * idx + (fabsf(vy) + cs) * idy);
#pragma unroll
              for (int w = 0; w < 2; ++w)
                march::two_sum_add2(th[w], tl[w], f32::mul2(make_float2(Un[2 * w], Un[2 * w + 1]), f32::bc2(vscale)));
            }
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) Fp[v] = F[v];
          hiPrev = hi;
          wm = w0;
          w0 = wp;
          dm = dp;
        }
      }
    }
    if constexpr (!LAST && !PERSIST) return;
    grp += gridDim.x;
    if (grp >= ngroups) break;
    leaf = grp * NW + warp;
    active = leaf < a.nleaves;
    __syncwarp();  // every lane of this warp is done with its tile and E before the next leaf
    if (active) load_leaf();
  }

  if constexpr (LAST) {
    // ---- last stage: CTA max rate, CTA totals (fixed order), finish
    for (int o = 16; o > 0; o >>= 1) rate = fmaxf(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    // each warp adds its 32 lanes' (hi, lo) pairs by a fixed butterfly (both partners of an
    // exchange get the same bits: TwoSum's error term is exact whatever the operand order)
    float hv[NV] = {th[0].x, th[0].y, th[1].x, th[1].y}, lv[NV] = {tl[0].x, tl[0].y, tl[1].x, tl[1].y};
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hv[v], o), l2 = __shfl_xor_sync(0xffffffffu, lv[v], o);
        march::ff_add(hv[v], lv[v], h2, l2);
      }
    if (lane == 0) {
      wrate[warp] = rate;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        wtot[0][warp][v] = hv[v];
        wtot[1][warp][v] = lv[v];
      }
    }
    if (bad) sbad = 1;
    __syncthreads();
    if (warp == 0) {
      if (lane < NV) {  // lane v: the warps' pairs in warp order
        float hh = wtot[0][0][lane], ll = wtot[1][0][lane];
        for (int w = 1; w < kMarchWarps; ++w) march::ff_add(hh, ll, wtot[0][w][lane], wtot[1][w][lane]);
        a.partials[(size_t)blockIdx.x * NV + lane] = ((double)hh + (double)ll) * G.dV[1];
      }
      __threadfence();  // the partials are visible before the counter counts this CTA
      if (lane == 0) {
        float mm = wrate[0];
        for (int w = 1; w < kMarchWarps; ++w) mm = fmaxf(mm, wrate[w]);
        atomicMax(&a.ctl->smax_bits, MaxKey<float>::enc(mm));
        if (sbad) atomicOr(&a.ctl->status, 1);
      }
    }
    if (gridDim.x <= kFlatFinishMax)
      last_cta_finish_flat<float, NV, 32 * kMarchWarps>(a.ctl, a.partials, true, dtd);
    else
      last_cta_finish<float, NV, 32 * kMarchWarps>(a.ctl, a.partials, a.gpart, a.gcount, (int)gridDim.x, 1, true, dtd,
                                                   false);
  }
}

}  // namespace amrgpu
