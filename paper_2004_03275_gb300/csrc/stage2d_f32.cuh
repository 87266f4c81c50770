// Float32 2D stage kernel (the batched fast path).
//
// Same method as the generic kernel (limited MUSCL on primitive variables,
// HLL/HLLC/TVDLF flux, SSPRK combination; Sec. 1.1, 1.2, 2.3-2.4), arranged to
// do each piece of work once:
//   A. the leaf and its face ghosts -> primitive values, once per cell;
//   B. one limited slope per cell, variable and direction; the two face values
//      of each cell go to shared memory;
//   C. one Riemann flux per face (branch-free HLLC evaluated on the upwind side
//      of the contact only), written over the face values it consumed;
//   D. flux difference and SSPRK combination; on the last stage, the max signal
//      rate and the conserved totals (compensated float-float block sums, one
//      float64 value per leaf and variable) for the CFL step.
// Persistent CTAs of 256 threads walk the leaves (one 16^2 leaf, or four 8^2
// leaves, per iteration) and prefetch the next leaf's cells into registers while
// the current one is computed.  Shared-memory layouts are chosen so that every
// access pattern of a warp hits distinct banks.
#pragma once
#include "euler_kernels.cuh"

namespace amrgpu {
namespace f32 {

__device__ __forceinline__ float rcp(float x) { return __fdividef(1.f, x); }

// Packed pairs: one f32x2 add / multiply / multiply-add (Blackwell) does two lanes of float32
// work, each element rounded as the scalar operation would be.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once (b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sel2(bool cx, bool cy, float2 a, float2 b) {
  return make_float2(cx ? a.x : b.x, cy ? a.y : b.y);
}

// s- / s+ times one half: the offsets from the cell value to its two face values
template <int LIM>
__device__ __forceinline__ void half_slopes(float a, float b, float& hm, float& hp) {
  if (LIM == LIM_NONE) {
    hm = 0.f;
    hp = 0.f;
  } else if (LIM == LIM_MINMOD) {
    float s = (a > 0.f) ? fminf(a, b) : fmaxf(a, b);
    s = (a * b > 0.f) ? 0.5f * s : 0.f;
    hm = s;
    hp = s;
  } else if (LIM == LIM_VANLEER) {  // (2ab/(a+b))/2
    float ab = a * b;
    float s = ab * rcp(a + b);
    s = (ab > 0.f) ? s : 0.f;
    hm = s;
    hp = s;
  } else if (LIM == LIM_MC) {  // minmod((a+b)/2, 2a, 2b) / 2
    float s = fminf(fminf(0.25f * fabsf(a + b), fabsf(a)), fabsf(b));
    s = (a * b > 0.f) ? copysignf(s, a) : 0.f;
    hm = s;
    hp = s;
  } else if (LIM == LIM_CADA) {  // Cada and Torrilhon (2009), halved; see limited_slopes
    const float A = fabsf(a), B = fabsf(b), ab = a * b;
    const float up = ab > 0.f ? fminf(fminf(A, (A + 2.f * B) * (1.f / 6.f)), 0.75f * B)
                              : fmaxf(0.f, fminf((2.f * B - A) * (1.f / 6.f), 0.5f * A));
    const float dn = ab > 0.f ? fminf(fminf(B, (2.f * A + B) * (1.f / 6.f)), 0.75f * A)
                              : fmaxf(0.f, fminf((2.f * A - B) * (1.f / 6.f), 0.5f * B));
    hp = ab != 0.f ? copysignf(up, b) : 0.f;
    hm = ab != 0.f ? copysignf(dn, a) : 0.f;
  } else {  // Koren: kappa = 1/3 face values limited into the TVD region, halved
    float A = fabsf(a), B = fabsf(b);
    float up = fminf(fminf(A, (A + 2.f * B) * (1.f / 6.f)), B);
    float dn = fminf(fminf(B, (2.f * A + B) * (1.f / 6.f)), A);
    bool same = a * b > 0.f;
    hp = same ? copysignf(up, b) : 0.f;
    hm = same ? copysignf(dn, a) : 0.f;
  }
}

// half_slopes for two variables at once (same limiters, packed arithmetic where it applies)
template <int LIM>
__device__ __forceinline__ void half_slopes2(float2 a, float2 b, float2& hm, float2& hp) {
  if (LIM == LIM_NONE) {
    hm = bc2(0.f);
    hp = bc2(0.f);
  } else if (LIM == LIM_MINMOD) {
    const float2 ab = mul2(a, b);
    float2 s = make_float2(a.x > 0.f ? fminf(a.x, b.x) : fmaxf(a.x, b.x), a.y > 0.f ? fminf(a.y, b.y) : fmaxf(a.y, b.y));
    s = sel2(ab.x > 0.f, ab.y > 0.f, mul2(s, bc2(0.5f)), bc2(0.f));
    hm = s;
    hp = s;
  } else if (LIM == LIM_VANLEER) {  // (2ab/(a+b))/2
    const float2 ab = mul2(a, b), d = add2(a, b);
    float2 s = mul2(ab, make_float2(rcp(d.x), rcp(d.y)));
    s = sel2(ab.x > 0.f, ab.y > 0.f, s, bc2(0.f));
    hm = s;
    hp = s;
  } else if (LIM == LIM_MC) {  // minmod((a+b)/2, 2a, 2b) / 2
    const float2 ab = mul2(a, b), q = mul2(add2(a, b), bc2(0.25f));
    float2 s = make_float2(fminf(fminf(fabsf(q.x), fabsf(a.x)), fabsf(b.x)), fminf(fminf(fabsf(q.y), fabsf(a.y)), fabsf(b.y)));
    s = sel2(ab.x > 0.f, ab.y > 0.f, make_float2(copysignf(s.x, a.x), copysignf(s.y, a.y)), bc2(0.f));
    hm = s;
    hp = s;
  } else if (LIM == LIM_CADA) {  // Cada and Torrilhon (2009), halved; per element as half_slopes
    half_slopes<LIM_CADA>(a.x, b.x, hm.x, hp.x);
    half_slopes<LIM_CADA>(a.y, b.y, hm.y, hp.y);
  } else {  // Koren: kappa = 1/3 face values (a + 2b)/6 up, (2a + b)/6 down, limited
    const float2 ab = mul2(a, b);
    const float2 A = make_float2(fabsf(a.x), fabsf(a.y)), B = make_float2(fabsf(b.x), fabsf(b.y));
    const float2 u6 = fma2(B, bc2(1.f / 3.f), mul2(A, bc2(1.f / 6.f)));
    const float2 d6 = fma2(A, bc2(1.f / 3.f), mul2(B, bc2(1.f / 6.f)));
    const float2 up = make_float2(fminf(fminf(A.x, u6.x), B.x), fminf(fminf(A.y, u6.y), B.y));
    const float2 dn = make_float2(fminf(fminf(B.x, d6.x), A.x), fminf(fminf(B.y, d6.y), A.y));
    const bool sx = ab.x > 0.f, sy = ab.y > 0.f;
    hp = sel2(sx, sy, make_float2(copysignf(up.x, b.x), copysignf(up.y, b.y)), bc2(0.f));
    hm = sel2(sx, sy, make_float2(copysignf(dn.x, a.x), copysignf(dn.y, a.y)), bc2(0.f));
  }
}

// sound speed c = sqrt(gamma p / rho), formed as (gamma p) / sqrt(gamma p rho): one
// special-function operation instead of a reciprocal and a square root
__device__ __forceinline__ float sound(float r, float p, float gam) {
  const float gp = gam * p;
  return gp * rsqrtf(gp * r);
}

// Riemann flux normal to x of the local frame (u normal, w tangential).
template <int FLUX>
__device__ __forceinline__ void flux2(float rL, float uL, float wL, float pL, float rR, float uR, float wR, float pR,
                                      float gam, float igm1, float* F) {
  const float cL = sound(rL, pL, gam), cR = sound(rR, pR, gam);
  if (FLUX == FLUX_TVDLF) {
    float EL = pL * igm1 + 0.5f * rL * (uL * uL + wL * wL);
    float ER = pR * igm1 + 0.5f * rR * (uR * uR + wR * wR);
    float mL = rL * uL, mR = rR * uR;
    float c = fmaxf(fabsf(uL) + cL, fabsf(uR) + cR);
    F[0] = 0.5f * (mL + mR) - 0.5f * c * (rR - rL);
    F[1] = 0.5f * (mL * uL + pL + mR * uR + pR) - 0.5f * c * (mR - mL);
    F[2] = 0.5f * (mL * wL + mR * wR) - 0.5f * c * (rR * wR - rL * wL);
    F[3] = 0.5f * ((EL + pL) * uL + (ER + pR) * uR) - 0.5f * c * (ER - EL);
    return;
  }
  float SL = fminf(uL - cL, uR - cR);
  float SR = fmaxf(uL + cL, uR + cR);
  if (FLUX == FLUX_HLL) {
    float EL = pL * igm1 + 0.5f * rL * (uL * uL + wL * wL);
    float ER = pR * igm1 + 0.5f * rR * (uR * uR + wR * wR);
    float mL = rL * uL, mR = rR * uR;
    float FL[4] = {mL, mL * uL + pL, mL * wL, (EL + pL) * uL};
    float FR[4] = {mR, mR * uR + pR, mR * wR, (ER + pR) * uR};
    float UL[4] = {rL, mL, rL * wL, EL};
    float UR[4] = {rR, mR, rR * wR, ER};
    float inv = rcp(SR - SL);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float h = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) * inv;
      F[v] = SL >= 0.f ? FL[v] : (SR <= 0.f ? FR[v] : h);
    }
    return;
  }
  // HLLC on the upwind side K of the contact only: F_K, plus S_K (U*_K - U_K) inside the fan
  float aL = rL * (SL - uL), aR = rR * (SR - uR);
  float Ss = (pR - pL + aL * uL - aR * uR) * rcp(aL - aR);
  const bool left = SL >= 0.f || (SR > 0.f && Ss >= 0.f), fan = SL < 0.f && SR > 0.f;
  float rK = left ? rL : rR, uK = left ? uL : uR, wK = left ? wL : wR, pK = left ? pL : pR;
  float SK = left ? SL : SR;
  float EK = pK * igm1 + 0.5f * rK * (uK * uK + wK * wK);
  float mK = rK * uK, eK = EK + pK;
  const float2 FK01 = make_float2(mK, mK * uK + pK), FK23 = make_float2(mK * wK, eK * uK);
  // U*_K - U_K with d = S* - u_K, q = 1 / (S_K - S*), g = d q (so that rho* = rho_K (1 + g)):
  //   (rho_K g, rho_K d + rho_K g S*, rho_K g w_K, d (q (E_K + p_K) + rho* S*)),
  // the star state of the fan with no division by rho_K and no difference of near-equal terms.
  // Outside the fan q and the wave-speed factor are zero, so the flux is F_K exactly.
  const float q = fan ? rcp(SK - Ss) : 0.f, s = fan ? SK : 0.f;
  const float d = Ss - uK, g0 = rK * (d * q);
  const float2 dU01 = make_float2(g0, g0 * Ss + rK * d), dU23 = make_float2(g0 * wK, d * (q * eK + (rK + g0) * Ss));
  const float2 F01 = fma2(bc2(s), dU01, FK01), F23 = fma2(bc2(s), dU23, FK23);
  F[0] = F01.x;
  F[1] = F01.y;
  F[2] = F23.x;
  F[3] = F23.y;
}

}  // namespace f32

// Shared memory of one leaf slot.
//  W  [v][(j+2)*B + i], j in [-2, B+2), i in [0, B): interior columns and the
//     y-ghost rows (row stride B: the rows a warp touches are contiguous);
//  HX [v][c][j]: the x-ghost columns c = 0..3 <-> i = -2, -1, B, B+1;
//  X  [v][f*S + j]: x faces f = 0..B of row j;  Y [v][i*S + f]: y faces of column i;
//     S = B + 2 (even, = 2 mod 4 for B = 16): the faces a warp touches split over
//     even and odd banks.  XL/YL hold the left/lower states, then the fluxes.
template <int B>
struct Stage2DF32Smem {
  static constexpr int LPB = 256 / (B * B), S = B + 2, NF = (B + 1) * S;
  float W[LPB][4][(B + 4) * B];
  float HX[LPB][4][4][B];
  float XL[LPB][4][NF], XR[LPB][4][NF], YL[LPB][4][NF], YR[LPB][4][NF];
};

template <int B>
__device__ __forceinline__ float wcell(const Stage2DF32Smem<B>& S, int lb, int v, int i, int j) {
  if (i < 0) return S.HX[lb][v][i + 2][j];
  if (i >= B) return S.HX[lb][v][i - B + 2][j];
  return S.W[lb][v][(j + 2) * B + i];
}

// Flux of face `fi` of line `line` (x: row; y: column), written over the left
// state it consumed; fluxes on a level jump also go to the reflux buffer.
template <int B, int FLUX, bool ISY>
__device__ __forceinline__ void face_flux(Stage2DF32Smem<B>& S, const StageArgs<float>& a, int lb, int leaf,
                                          int line, int fi, float gam, float igm1) {
  constexpr int SS = B + 2, NF = (B + 1) * SS, NV = 4;
  constexpr int VN = ISY ? 2 : 1, VT = ISY ? 1 : 2;  // normal / tangential velocity
  float (*Lb)[NF] = ISY ? S.YL[lb] : S.XL[lb];
  const float (*Rb)[NF] = ISY ? S.YR[lb] : S.XR[lb];
  const int o = ISY ? line * SS + fi : fi * SS + line;
  float rL = Lb[0][o], uL = Lb[VN][o], wL = Lb[VT][o], pL = Lb[3][o];
  float rR = Rb[0][o], uR = Rb[VN][o], wR = Rb[VT][o], pR = Rb[3][o];
  if (!(rL > 0.f) || !(rR > 0.f) || !(pL > 0.f) || !(pR > 0.f)) {  // first-order fallback
    int il = ISY ? line : fi - 1, jl = ISY ? fi - 1 : line;
    int ir = ISY ? line : fi, jr = ISY ? fi : line;
    rL = wcell(S, lb, 0, il, jl); uL = wcell(S, lb, VN, il, jl); wL = wcell(S, lb, VT, il, jl);
    pL = wcell(S, lb, 3, il, jl);
    rR = wcell(S, lb, 0, ir, jr); uR = wcell(S, lb, VN, ir, jr); wR = wcell(S, lb, VT, ir, jr);
    pR = wcell(S, lb, 3, ir, jr);
  }
  float F[4];
  f32::flux2<FLUX>(rL, uL, wL, pL, rR, uR, wR, pR, gam, igm1, F);
  Lb[0][o] = F[0];
  Lb[VN][o] = F[1];
  Lb[VT][o] = F[2];
  Lb[3][o] = F[3];
  if (a.has_ffx && (fi == 0 || fi == B)) {
    int slot = a.ffx[leaf * 4 + 2 * (ISY ? 1 : 0) + (fi == 0 ? 0 : 1)];
    if (slot >= 0) {
      a.fflux[((size_t)slot * NV + 0) * B + line] = F[0];
      a.fflux[((size_t)slot * NV + VN) * B + line] = F[1];
      a.fflux[((size_t)slot * NV + VT) * B + line] = F[2];
      a.fflux[((size_t)slot * NV + 3) * B + line] = F[3];
    }
  }
}

// cells of one leaf slot held in registers: the thread's own cell (U, U0) and,
// for the first 8B threads, one face-ghost cell
struct Prefetch {
  float U[4], U0[4], G[4];
};

template <int B>
__device__ __forceinline__ void prefetch(const StageArgs<float>& a, int leaf, int tc, Prefetch& p) {
  constexpr int NC = B * B;
  if (leaf >= a.nleaves) return;
#pragma unroll
  for (int v = 0; v < 4; ++v) p.U[v] = a.Us[((size_t)leaf * 4 + v) * NC + tc];
  if (!a.stage1)
#pragma unroll
    for (int v = 0; v < 4; ++v) p.U0[v] = a.U0[((size_t)leaf * 4 + v) * NC + tc];
  if (tc < 8 * B) {
    int f = tc / (2 * B), m = (tc / B) & 1, t = tc % B;
#pragma unroll
    for (int v = 0; v < 4; ++v) p.G[v] = fetch_ghost<float, 2, B>(a.Us, a.slabs, a.nb, leaf, f, m, t, v);
  }
}

template <int B, int FLUX, int LIM>
__global__ void __launch_bounds__(256, 5) stage2d_f32_kernel(StageArgs<float> a, Geometry G) {
  constexpr int NV = 4, NC = B * B, LPB = 256 / NC;
  __shared__ Stage2DF32Smem<B> S;
  __shared__ float wmax[8];
  __shared__ int sbad;
  const float dt = cta_stage_dtf(a.ctl);
  if (!(dt > 0.f)) return;
  const float gam = G.gammaf, gm1 = gam - 1.f, igm1 = 1.f / gm1;
  const int lb = threadIdx.x / NC, tc = threadIdx.x % NC;
  const int ic = tc % B, jc = tc / B;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nslots = (a.nleaves + LPB - 1) / LPB;

  float rate = 0.f;
  int bad = 0;
  if (threadIdx.x == 0) sbad = 0;

  Prefetch cur;
  int slot = blockIdx.x;
  prefetch<B>(a, slot * LPB + lb, tc, cur);
  for (; slot < nslots; slot += gridDim.x) {
    const int leaf = slot * LPB + lb;
    const bool active = leaf < a.nleaves;
    float Uc[NV], Un0[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Uc[v] = cur.U[v];
      Un0[v] = cur.U0[v];
    }
    float Gc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Gc[v] = cur.G[v];
    // ---- A: primitive values of the cell and of one ghost cell
    __syncthreads();  // previous iteration done with the shared arrays
    if (active) {
      float ir = f32::rcp(Uc[0]);
      float vx = Uc[1] * ir, vy = Uc[2] * ir;
      int q = (jc + 2) * B + ic;
      S.W[lb][0][q] = Uc[0];
      S.W[lb][1][q] = vx;
      S.W[lb][2][q] = vy;
      S.W[lb][3][q] = gm1 * (Uc[3] - 0.5f * (Uc[1] * vx + Uc[2] * vy));
      if (tc < 8 * B) {
        int f = tc / (2 * B), m = (tc / B) & 1, t = tc % B;
        float irg = f32::rcp(Gc[0]);
        float gx = Gc[1] * irg, gy = Gc[2] * irg;
        float V[4] = {Gc[0], gx, gy, gm1 * (Gc[3] - 0.5f * (Gc[1] * gx + Gc[2] * gy))};
        if (f < 2) {  // x ghost column
          int c = f == 0 ? 1 - m : 2 + m;
#pragma unroll
          for (int v = 0; v < NV; ++v) S.HX[lb][v][c][t] = V[v];
        } else {
          int row = f == 2 ? -1 - m : B + m;
#pragma unroll
          for (int v = 0; v < NV; ++v) S.W[lb][v][(row + 2) * B + t] = V[v];
        }
      }
    }
    // prefetch the next slot while this one is computed
    if (slot + gridDim.x < nslots) prefetch<B>(a, (slot + gridDim.x) * LPB + lb, tc, cur);
    __syncthreads();

    // ---- B: slopes once per cell and direction; face values
    if (active) {
      const int q = (jc + 2) * B + ic;
      constexpr int SS = B + 2;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* Wv = S.W[lb][v];
        float c = Wv[q];
        float l = ic > 0 ? Wv[q - 1] : S.HX[lb][v][1][jc];
        float r = ic < B - 1 ? Wv[q + 1] : S.HX[lb][v][2][jc];
        float hm, hp;
        f32::half_slopes<LIM>(c - l, r - c, hm, hp);
        S.XR[lb][v][ic * SS + jc] = c - hm;
        S.XL[lb][v][(ic + 1) * SS + jc] = c + hp;
        f32::half_slopes<LIM>(c - Wv[q - B], Wv[q + B] - c, hm, hp);
        S.YR[lb][v][ic * SS + jc] = c - hm;
        S.YL[lb][v][ic * SS + jc + 1] = c + hp;
      }
      // the adjacent ghost layer needs its normal slope for the boundary faces
      if (tc < 4 * B) {
        int f = tc / B, t = tc % B;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float hm, hp;
          if (f == 0) {
            float c = S.HX[lb][v][1][t];
            f32::half_slopes<LIM>(c - S.HX[lb][v][0][t], S.W[lb][v][(t + 2) * B] - c, hm, hp);
            S.XL[lb][v][0 * SS + t] = c + hp;
          } else if (f == 1) {
            float c = S.HX[lb][v][2][t];
            f32::half_slopes<LIM>(c - S.W[lb][v][(t + 2) * B + B - 1], S.HX[lb][v][3][t] - c, hm, hp);
            S.XR[lb][v][B * SS + t] = c - hm;
          } else if (f == 2) {
            const float* Wv = S.W[lb][v];
            float c = Wv[1 * B + t];
            f32::half_slopes<LIM>(c - Wv[t], Wv[2 * B + t] - c, hm, hp);
            S.YL[lb][v][t * SS + 0] = c + hp;
          } else {
            const float* Wv = S.W[lb][v];
            float c = Wv[(B + 2) * B + t];
            f32::half_slopes<LIM>(c - Wv[(B + 1) * B + t], Wv[(B + 3) * B + t] - c, hm, hp);
            S.YR[lb][v][t * SS + B] = c - hm;
          }
        }
      }
    }
    __syncthreads();

    // ---- C: one flux per face; x faces face-fastest, y faces line-fastest
    if (active) {
      face_flux<B, FLUX, false>(S, a, lb, leaf, jc, ic, gam, igm1);
      face_flux<B, FLUX, true>(S, a, lb, leaf, ic, jc, gam, igm1);
      if (tc < B) face_flux<B, FLUX, false>(S, a, lb, leaf, tc, B, gam, igm1);
      else if (tc < 2 * B) face_flux<B, FLUX, true>(S, a, lb, leaf, tc - B, B, gam, igm1);
    }
    __syncthreads();

    // ---- D: flux difference, SSPRK combination, last-stage reductions
    float Un[NV];
    if (active) {
      const int lev = a.level[leaf];
      const float idx = G.idxf[lev][0], idy = G.idxf[lev][1];
      constexpr int SS = B + 2;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float div = (S.XL[lb][v][(ic + 1) * SS + jc] - S.XL[lb][v][ic * SS + jc]) * idx +
                    (S.YL[lb][v][ic * SS + jc + 1] - S.YL[lb][v][ic * SS + jc]) * idy;
        float tmp = Uc[v] - dt * div;
        Un[v] = a.stage1 ? tmp : ssp_combine(a.alpha, a.beta, Un0[v], tmp);
        a.out[((size_t)leaf * NV + v) * NC + tc] = Un[v];
      }
      if (a.fuse_reduce) {
        float ir = f32::rcp(Un[0]);
        float vx = Un[1] * ir, vy = Un[2] * ir;
        float p = gm1 * (Un[3] - 0.5f * (Un[1] * vx + Un[2] * vy));
        if (!(Un[0] > 0.f) || !(p > 0.f)) bad = 1;
        float c = sqrtf(gam * p * ir);
        rate = fmaxf(rate, (fabsf(vx) + c) * idx + (fabsf(vy) + c) * idy);
      }
    }
    if (a.fuse_reduce) {
      // per (leaf, variable) one warp adds the leaf's cells in float-float
      __syncthreads();  // XR is reused for the values
      float* vals = &S.XR[0][0][0];  // [LPB][NV][NC] fits in XR
      if (active)
#pragma unroll
        for (int v = 0; v < NV; ++v) vals[(lb * NV + v) * NC + tc] = Un[v];
      __syncthreads();
      for (int pidx = warp; pidx < LPB * NV; pidx += 8) {
        int l2 = pidx / NV, v = pidx % NV;
        int lf = slot * LPB + l2;
        if (lf >= a.nleaves) continue;
        float hi = 0.f, lo = 0.f;
        for (int c = lane; c < NC; c += 32) {
          float x = vals[(l2 * NV + v) * NC + c];
          float s = hi + x, bb = s - hi;
          lo += (hi - (s - bb)) + (x - bb);
          hi = s;
        }
        for (int o = 16; o > 0; o >>= 1) {
          float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2v = __shfl_xor_sync(0xffffffffu, lo, o);
          float s = hi + h2, bb = s - hi;
          float e = (hi - (s - bb)) + (h2 - bb);
          lo = lo + l2v + e;
          hi = s;
        }
        if (lane == 0) a.partials[(size_t)lf * NV + v] = ((double)hi + (double)lo) * G.dV[a.level[lf]];
      }
    }
  }
  if (!a.fuse_reduce) return;
  float m = rate;
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) wmax[warp] = m;
  __syncthreads();
  if (bad) sbad = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = wmax[0];
    for (int w = 1; w < 8; ++w) mm = fmaxf(mm, wmax[w]);
    atomicMax(&a.ctl->smax_bits, MaxKey<float>::enc(mm));
    if (sbad) atomicOr(&a.ctl->status, 1);
  }
  last_cta_finish<float, NV, 256>(a.ctl, a.partials, a.gpart, a.gcount, a.nleaves, LPB, true, 0.0, true, true);
}

}  // namespace amrgpu
