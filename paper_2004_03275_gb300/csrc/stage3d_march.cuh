// Float32 3D stage for 16^3 leaves as two directional-march kernels.
//
// Same method as the other stage kernels (limited MUSCL on primitive variables,
// HLL/HLLC/TVDLF flux, SSPRK combination; Sec. 1.1, 1.2, 2.3-2.4).  A 16^3 leaf
// with its ghosts does not fit in shared memory with five variables, so the stage
// is split in two passes over the leaf:
//   xy pass: one warp per (leaf, z-plane), the 2D march (primitive tile of the plane
//     with its x and y ghosts, x march then y march with register windows); it
//     writes D = (F_{i+1/2} - F_{i-1/2}) / dx + (G_{j+1/2} - G_{j-1/2}) / dy per
//     cell and variable to a scratch array laid out like the state;
//   z pass: lane (i, half) of warp j walks planes half*8-2 .. half*8+9 of the
//     pencil (i, j), keeping the conserved and primitive values of a three-cell
//     window in registers, forms the z fluxes, and finishes each cell:
//     out = alpha U^n + beta (U - dt (D + (H_{k+1/2} - H_{k-1/2}) / dz)), plus on
//     the last stage the CFL rate and the conserved totals.
// Every lane does the same work; there is no shared memory in the z pass and no
// block-wide barrier inside either pass except the z pass's dt and finish.
// Variables: U = (rho, m_x, m_y, m_z, E), W = (rho, v_x, v_y, v_z, p).
#pragma once
#include "stage2d_march.cuh"

namespace amrgpu {

namespace f32 {

// Riemann flux normal to x of the local frame (u normal; v, w tangential), result in
// the local order (mass, normal momentum, tangential momenta v then w, energy).
template <int FLUX>
__device__ __forceinline__ void flux3(float rL, float uL, float vL, float wL, float pL, float rR, float uR, float vR,
                                      float wR, float pR, float gam, float igm1, float* F) {
  const float cL = sound(rL, pL, gam), cR = sound(rR, pR, gam);
  if (FLUX == FLUX_TVDLF) {
    float EL = pL * igm1 + 0.5f * rL * (uL * uL + vL * vL + wL * wL);
    float ER = pR * igm1 + 0.5f * rR * (uR * uR + vR * vR + wR * wR);
    float mL = rL * uL, mR = rR * uR;
    float c = fmaxf(fabsf(uL) + cL, fabsf(uR) + cR);
    F[0] = 0.5f * (mL + mR) - 0.5f * c * (rR - rL);
    F[1] = 0.5f * (mL * uL + pL + mR * uR + pR) - 0.5f * c * (mR - mL);
    F[2] = 0.5f * (mL * vL + mR * vR) - 0.5f * c * (rR * vR - rL * vL);
    F[3] = 0.5f * (mL * wL + mR * wR) - 0.5f * c * (rR * wR - rL * wL);
    F[4] = 0.5f * ((EL + pL) * uL + (ER + pR) * uR) - 0.5f * c * (ER - EL);
    return;
  }
  float SL = fminf(uL - cL, uR - cR);
  float SR = fmaxf(uL + cL, uR + cR);
  if (FLUX == FLUX_HLL) {
    float EL = pL * igm1 + 0.5f * rL * (uL * uL + vL * vL + wL * wL);
    float ER = pR * igm1 + 0.5f * rR * (uR * uR + vR * vR + wR * wR);
    float mL = rL * uL, mR = rR * uR;
    float FL[5] = {mL, mL * uL + pL, mL * vL, mL * wL, (EL + pL) * uL};
    float FR[5] = {mR, mR * uR + pR, mR * vR, mR * wR, (ER + pR) * uR};
    float UL[5] = {rL, mL, rL * vL, rL * wL, EL};
    float UR[5] = {rR, mR, rR * vR, rR * wR, ER};
    float inv = rcp(SR - SL);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      float h = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) * inv;
      F[v] = SL >= 0.f ? FL[v] : (SR <= 0.f ? FR[v] : h);
    }
    return;
  }
  // HLLC on the upwind side K of the contact only; U*_K - U_K in the form of flux2
  float aL = rL * (SL - uL), aR = rR * (SR - uR);
  float Ss = (pR - pL + aL * uL - aR * uR) * rcp(aL - aR);
  const bool left = SL >= 0.f || (SR > 0.f && Ss >= 0.f), fan = SL < 0.f && SR > 0.f;
  float rK = left ? rL : rR, uK = left ? uL : uR, vK = left ? vL : vR, wK = left ? wL : wR, pK = left ? pL : pR;
  float SK = left ? SL : SR;
  float EK = pK * igm1 + 0.5f * rK * (uK * uK + vK * vK + wK * wK);
  float mK = rK * uK, eK = EK + pK;
  const float2 FK01 = make_float2(mK, mK * uK + pK), FK23 = make_float2(mK * vK, mK * wK);
  const float q = fan ? rcp(SK - Ss) : 0.f, s = fan ? SK : 0.f;
  const float d = Ss - uK, g0 = rK * (d * q);
  const float2 dU01 = make_float2(g0, g0 * Ss + rK * d), dU23 = make_float2(g0 * vK, g0 * wK);
  const float2 F01 = fma2(bc2(s), dU01, FK01), F23 = fma2(bc2(s), dU23, FK23);
  F[0] = F01.x;
  F[1] = F01.y;
  F[2] = F23.x;
  F[3] = F23.y;
  F[4] = s * (d * (q * eK + (rK + g0) * Ss)) + eK * uK;
}

}  // namespace f32

namespace march3 {

// primitive (rho, v_x, v_y, v_z, p) of a conserved cell
__device__ __forceinline__ void prim5(const float* u, float gm1, float* w) {
  float ir = f32::rcp(u[0]);
  float vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  w[0] = u[0];
  w[1] = vx;
  w[2] = vy;
  w[3] = vz;
  w[4] = gm1 * (u[4] - 0.5f * (u[1] * vx + u[2] * vy + u[3] * vz));
}

// the two face values of the middle cell: (rho, v_x) and (v_y, v_z) as packed pairs, p alone
template <int LIM>
__device__ __forceinline__ void faces5(const float* wm, const float* w0, const float* wp, float* lo, float* hi) {
  using namespace f32;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float2 m = make_float2(wm[2 * q], wm[2 * q + 1]), c = make_float2(w0[2 * q], w0[2 * q + 1]);
    const float2 p = make_float2(wp[2 * q], wp[2 * q + 1]);
    float2 hm, hp;
    half_slopes2<LIM>(sub2(c, m), sub2(p, c), hm, hp);
    const float2 l = sub2(c, hm), h = add2(c, hp);
    lo[2 * q] = l.x, lo[2 * q + 1] = l.y;
    hi[2 * q] = h.x, hi[2 * q + 1] = h.y;
  }
  float hm, hp;
  f32::half_slopes<LIM>(w0[4] - wm[4], wp[4] - w0[4], hm, hp);
  lo[4] = w0[4] - hm;
  hi[4] = w0[4] + hp;
}

// flux through a face normal to direction D (0 x, 1 y, 2 z) from face states L, R (W
// order), first order from the cell values a, b if a reconstructed density or
// pressure is not positive; result in variable order (rho, m_x, m_y, m_z, E)
template <int FLUX, int D>
__device__ __forceinline__ void flux(const float* Lf, const float* Rf, const float* a, const float* b, float gam,
                                     float igm1, float* F) {
  const bool fo = !(Lf[0] > 0.f) || !(Rf[0] > 0.f) || !(Lf[4] > 0.f) || !(Rf[4] > 0.f);
  const float* L = fo ? a : Lf;
  const float* R = fo ? b : Rf;
  constexpr int N = 1 + D, T1 = D == 0 ? 2 : 1, T2 = D == 2 ? 2 : 3;
  float G[5];
  f32::flux3<FLUX>(L[0], L[N], L[T1], L[T2], L[4], R[0], R[N], R[T1], R[T2], R[4], gam, igm1, G);
  F[0] = G[0];
  F[N] = G[1];
  F[T1] = G[2];
  F[T2] = G[3];
  F[4] = G[4];
}

}  // namespace march3

struct Xy3Smem {
  float4 T[20][21];  // (rho, v_x, v_y, p) of the plane, T[j+2][i+2], i, j in -2..17
  float Tz[20][21];  // v_z
  float4 E[16][17];  // x flux differences (rho, m_x, m_y, E) / dx, E[j][i]
  float Ez[16][17];  // m_z
};

__device__ __forceinline__ float4 pick4(const float* w) { return make_float4(w[0], w[1], w[2], w[4]); }
__device__ __forceinline__ void unpick(const float4& q, float z, float* w) {
  w[0] = q.x;
  w[1] = q.y;
  w[2] = q.z;
  w[3] = z;
  w[4] = q.w;
}

// ---- xy pass: one warp per (leaf, plane k), 4 planes per CTA; launch bounds for 3 CTAs per SM
// (up to 168 registers: no spill; measured 2 % faster over a blast step than 4 CTAs at 128)
constexpr size_t kXy3Smem = 4 * sizeof(Xy3Smem);  // dynamic shared memory of the xy pass (55 KB)

template <int FLUX, int LIM>
__global__ void __launch_bounds__(128, 3) stage3d_xy_kernel(StageArgs<float> a, Geometry G) {
  constexpr int B = 16, NC = B * B * B, NV = 5, NT = B * B;
  extern __shared__ __align__(16) unsigned char xy3_smem[];
  Xy3Smem* S = reinterpret_cast<Xy3Smem*>(xy3_smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int leaf = blockIdx.x >> 2, k = ((blockIdx.x & 3) << 2) + warp;
  if (leaf >= a.nleaves) return;
  const int lo16 = lane & 15, h = lane >> 4;
  Xy3Smem& M = S[warp];
  const float gam = G.gammaf, gm1 = gam - 1.f, igm1 = 1.f / gm1;
  const float* Ul = a.Us + (size_t)leaf * NV * NC;
  // ---- plane cells: row lo16, columns h*8..h*8+7
  {
    float4 u[NV][2];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float4* p = reinterpret_cast<const float4*>(Ul + v * NC + k * NT + lo16 * B + h * 8);
      u[v][0] = __ldg(p);
      u[v][1] = __ldg(p + 1);
    }
    float4* trow = &M.T[lo16 + 2][h * 8 + 2];
    float* zrow = &M.Tz[lo16 + 2][h * 8 + 2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float c[NV], w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) c[v] = e == 0 ? u[v][q].x : e == 1 ? u[v][q].y : e == 2 ? u[v][q].z : u[v][q].w;
        march3::prim5(c, gm1, w);
        trow[4 * q + e] = pick4(w);
        zrow[4 * q + e] = w[3];
      }
    }
  }
  // ---- x and y ghosts of the plane: face f, layer m = h, in-plane tangential index lo16
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int code = __ldg(&a.nb[leaf * 6 + f]);
    const int d = f >> 1, side = f & 1, m = h, t = lo16;
    const int t3 = t + B * k;  // tangential index on the face: (j, k) for x faces, (i, k) for y faces
    const float* src;
    int stride;
    if (code >= -1) {
      int n = code >= 0 ? (side == 0 ? B - 1 - m : m) : (side == 0 ? 0 : B - 1);
      int cell = d == 0 ? n + B * t + NT * k : t + B * n + NT * k;
      src = a.Us + (size_t)(code >= 0 ? code : leaf) * NV * NC + cell;
      stride = NC;
    } else {
      src = a.slabs + ((size_t)(-2 - code) * NV * 2 + m) * NT + t3;
      stride = 2 * NT;
    }
    float c[NV], w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = __ldg(&src[v * stride]);
    march3::prim5(c, gm1, w);
    int r, cc;
    if (d == 0) {
      r = t;
      cc = side == 0 ? -1 - m : B + m;
    } else {
      cc = t;
      r = side == 0 ? -1 - m : B + m;
    }
    M.T[r + 2][cc + 2] = pick4(w);
    M.Tz[r + 2][cc + 2] = w[3];
  }
  __syncwarp();
  const int lev = __ldg(&a.level[leaf]);
  const float idx = G.idxf[lev][0], idy = G.idxf[lev][1];
  const int c0 = h * 8;

  // ---- x march along row j = lo16 -> E
  {
    const int j = lo16;
    auto W = [&](int c, float* w) { unpick(M.T[j + 2][c + 2], M.Tz[j + 2][c + 2], w); };
    float wm[NV], w0[NV], wp[NV], lo[NV], hiPrev[NV], Fp[NV];
    W(c0 - 2, wm);
    W(c0 - 1, w0);
    W(c0, wp);
    march3::faces5<LIM>(wm, w0, wp, lo, hiPrev);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wm[v] = w0[v];
      w0[v] = wp[v];
    }
#pragma unroll
    for (int kk = 0; kk <= 8; ++kk) {
      const int cc = c0 + kk;
      W(cc + 1, wp);
      float hi[NV], F[NV];
      march3::faces5<LIM>(wm, w0, wp, lo, hi);
      march3::flux<FLUX, 0>(hiPrev, lo, wm, w0, gam, igm1, F);
      if (a.has_ffx && ((h == 0 && kk == 0) || (h == 1 && kk == 8))) {
        int slot = a.ffx[leaf * 6 + h];
        if (slot >= 0)
#pragma unroll
          for (int v = 0; v < NV; ++v) a.fflux[((size_t)slot * NV + v) * NT + j + B * k] = F[v];
      }
      if (kk > 0) {
        M.E[j][cc - 1] = make_float4((F[0] - Fp[0]) * idx, (F[1] - Fp[1]) * idx, (F[2] - Fp[2]) * idx,
                                     (F[4] - Fp[4]) * idx);
        M.Ez[j][cc - 1] = (F[3] - Fp[3]) * idx;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Fp[v] = F[v];
        hiPrev[v] = hi[v];
        wm[v] = w0[v];
        w0[v] = wp[v];
      }
    }
  }
  __syncwarp();
  // ---- y march along column i = lo16 -> D of rows c0..c0+7
  {
    const int i = lo16;
    auto W = [&](int r, float* w) { unpick(M.T[r + 2][i + 2], M.Tz[r + 2][i + 2], w); };
    float* Dl = a.scratch + (size_t)leaf * NV * NC + k * NT;
    float wm[NV], w0[NV], wp[NV], lo[NV], hiPrev[NV], Fp[NV];
    W(c0 - 2, wm);
    W(c0 - 1, w0);
    W(c0, wp);
    march3::faces5<LIM>(wm, w0, wp, lo, hiPrev);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wm[v] = w0[v];
      w0[v] = wp[v];
    }
#pragma unroll
    for (int kk = 0; kk <= 8; ++kk) {
      const int rr = c0 + kk;
      W(rr + 1, wp);
      float hi[NV], F[NV];
      march3::faces5<LIM>(wm, w0, wp, lo, hi);
      march3::flux<FLUX, 1>(hiPrev, lo, wm, w0, gam, igm1, F);
      if (a.has_ffx && ((h == 0 && kk == 0) || (h == 1 && kk == 8))) {
        int slot = a.ffx[leaf * 6 + 2 + h];
        if (slot >= 0)
#pragma unroll
          for (int v = 0; v < NV; ++v) a.fflux[((size_t)slot * NV + v) * NT + i + B * k] = F[v];
      }
      if (kk > 0) {
        const int r = rr - 1, q = r * B + i;
        const float4 e = M.E[r][i];
        const float ez = M.Ez[r][i];
        Dl[0 * NC + q] = e.x + (F[0] - Fp[0]) * idy;
        Dl[1 * NC + q] = e.y + (F[1] - Fp[1]) * idy;
        Dl[2 * NC + q] = e.z + (F[2] - Fp[2]) * idy;
        Dl[3 * NC + q] = ez + (F[3] - Fp[3]) * idy;
        Dl[4 * NC + q] = e.w + (F[4] - Fp[4]) * idy;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Fp[v] = F[v];
        hiPrev[v] = hi[v];
        wm[v] = w0[v];
        w0[v] = wp[v];
      }
    }
  }
}

// ---- z pass: ZR rows per CTA (16 / ZR CTAs per leaf); warp w of CTA b handles row
// j = (b % (16 / ZR)) ZR + w of leaf b / (16 / ZR); lane (i, half)
// z-pass staging: U^(s), D and U^n of the CTA's ZR rows of the leaf for all 16 planes,
// [array][var][plane][row][i] with a plane stride of 16 ZR + 2 floats, so that the two
// half-warps (planes k and k + 8) fall on different banks
template <int ZR>
struct ZGeom {
  static constexpr int Plane = 16 * ZR + 2, Var = 16 * Plane;
  static constexpr size_t Smem = 3 * 5 * Var * sizeof(float);  // 63.4 KB for 4 rows
};
constexpr size_t kZSmem = ZGeom<4>::Smem;

template <int FLUX, int LIM, bool LAST, int ZR = 4>
__global__ void __launch_bounds__(32 * ZR, 12 / ZR) stage3d_z_kernel(StageArgs<float> a, Geometry G) {
  constexpr int B = 16, NC = B * B * B, NV = 5, NT = B * B;
  constexpr int kZPlane = ZGeom<ZR>::Plane, kZVar = ZGeom<ZR>::Var, CPL = 16 / ZR;
  static_assert(!LAST || ZR == 4, "the fused reduction writes 4 partials per leaf");
  __shared__ float red[ZR][2 * NV + 1];
  __shared__ int sbad;
  extern __shared__ __align__(16) float zst[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int leaf = blockIdx.x / CPL, j0 = (blockIdx.x % CPL) * ZR, j = j0 + warp;
  const bool active = leaf < a.nleaves;
  const int i = lane & 15, h = lane >> 4, c0 = h * 8;
  if (threadIdx.x == 0) sbad = 0;
  // ---- stage U^(s), D and U^n of rows j0..j0+3 (64 contiguous floats per variable and plane)
  if (active) {
    // thread t: 16-byte column q = t mod 4 ZR of planes k0 = t / 4 ZR and k0 + 8, every array and
    // variable
    const int q = threadIdx.x % (4 * ZR), k0 = threadIdx.x / (4 * ZR);
    const size_t lb = (size_t)leaf * NV * NC + j0 * B + k0 * NT;
    const float* src3[3] = {a.Us, a.scratch, a.U0};
#pragma unroll
    for (int arr = 0; arr < 3; ++arr) {
      if (arr == 2 && a.stage1) break;
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const float4 x4 = __ldg(reinterpret_cast<const float4*>(src3[arr] + lb + (size_t)v * NC + p * 8 * NT) + q);
          float2* dst = reinterpret_cast<float2*>(zst + (arr * NV + v) * kZVar + (k0 + 8 * p) * kZPlane + 4 * q);
          dst[0] = make_float2(x4.x, x4.y);
          dst[1] = make_float2(x4.z, x4.w);
        }
    }
  }
  // ghost cells of the pencil beyond its z faces: h = 0 takes planes -2, -1 (face z-),
  // h = 1 planes 16, 17 (face z+); g[0] is the layer next to the leaf, g[1] the outer one
  float gz[2][NV];
  if (active) {
    const int f = 4 + h, code = __ldg(&a.nb[leaf * 6 + f]);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const float* src;
      int stride;
      if (code >= -1) {
        int n = code >= 0 ? (h == 0 ? B - 1 - m : m) : (h == 0 ? 0 : B - 1);
        src = a.Us + (size_t)(code >= 0 ? code : leaf) * NV * NC + i + B * j + NT * n;
        stride = NC;
      } else {
        src = a.slabs + ((size_t)(-2 - code) * NV * 2 + m) * NT + i + B * j;
        stride = 2 * NT;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) gz[m][v] = __ldg(&src[v * stride]);
    }
  }
  const float dt = cta_stage_dtf(a.ctl);  // its barrier also publishes the staged arrays
  if (!(dt > 0.f)) return;
  const float gam = G.gammaf, gm1 = gam - 1.f, igm1 = 1.f / gm1;
  float rate = 0.f;
  int bad = 0;
  float th[NV] = {0.f, 0.f, 0.f, 0.f, 0.f}, tl[NV] = {0.f, 0.f, 0.f, 0.f, 0.f};
  if (active) {
    const int lev = __ldg(&a.level[leaf]);
    const float idx = G.idxf[lev][0], idy = G.idxf[lev][1], idz = G.idxf[lev][2];
    const float vscale = __int_as_float((127 - 3 * (lev - 1)) << 23);  // 8^-(lev-1), exact
    const int col = i + B * j;
    const float* sU = zst + 0 * NV * kZVar + warp * 16 + i;  // + v * kZVar + k * kZPlane
    const float* sD = zst + 1 * NV * kZVar + warp * 16 + i;
    const float* sU0 = zst + 2 * NV * kZVar + warp * 16 + i;
    // conserved cell of plane kk of the pencil (ghost planes from gz)
    auto cellU = [&](int kk, float* u) {
      if (kk < 0 || kk >= B) {
        const bool outer = kk == -2 || kk == B + 1;
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = outer ? gz[1][v] : gz[0][v];
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = sU[v * kZVar + kk * kZPlane];
      }
    };
    float* Ol = a.out + (size_t)leaf * NV * NC + col;
    float up[NV], wm[NV], w0[NV], wp[NV], lo[NV], hiPrev[NV], Fp[NV];
    cellU(c0 - 2, up);
    march3::prim5(up, gm1, wm);
    cellU(c0 - 1, up);
    march3::prim5(up, gm1, w0);
    cellU(c0, up);
    march3::prim5(up, gm1, wp);
    march3::faces5<LIM>(wm, w0, wp, lo, hiPrev);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wm[v] = w0[v];
      w0[v] = wp[v];
    }
    float un[NV];
    cellU(c0 + 1, un);
#pragma unroll
    for (int kk = 0; kk <= 8; ++kk) {
      const int cc = c0 + kk;  // plane whose slope is formed; face cc-1/2
#pragma unroll
      for (int v = 0; v < NV; ++v) up[v] = un[v];
      if (kk < 8) cellU(cc + 2, un);
      march3::prim5(up, gm1, wp);
      float hi[NV], F[NV];
      march3::faces5<LIM>(wm, w0, wp, lo, hi);
      march3::flux<FLUX, 2>(hiPrev, lo, wm, w0, gam, igm1, F);
      if (a.has_ffx && ((h == 0 && kk == 0) || (h == 1 && kk == 8))) {
        int slot = a.ffx[leaf * 6 + 4 + h];
        if (slot >= 0)
#pragma unroll
          for (int v = 0; v < NV; ++v) a.fflux[((size_t)slot * NV + v) * NT + col] = F[v];
      }
      if (kk > 0) {
        const int r = cc - 1;  // plane of the cell finished now
        float uc[NV], dc[NV], u0c[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          uc[v] = sU[v * kZVar + r * kZPlane];
          dc[v] = sD[v * kZVar + r * kZPlane];
          u0c[v] = a.stage1 ? 0.f : sU0[v * kZVar + r * kZPlane];
        }
        // Un = U - dt (D + (F - Fp) / dz), then the SSPRK combination T + alpha (U^n - T);
        // variables (0, 1) and (2, 3) as packed pairs, 4 alone
        float Un[NV];
        {
          using namespace f32;
          const float2 mdt = bc2(-dt), iz = bc2(idz), al = bc2(a.alpha);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int v = 2 * q;
            const float2 div = fma2(sub2(make_float2(F[v], F[v + 1]), make_float2(Fp[v], Fp[v + 1])), iz,
                                    make_float2(dc[v], dc[v + 1]));
            float2 t = fma2(mdt, div, make_float2(uc[v], uc[v + 1]));
            if (!a.stage1) t = fma2(al, sub2(make_float2(u0c[v], u0c[v + 1]), t), t);
            Un[v] = t.x, Un[v + 1] = t.y;
          }
          const float tmp = uc[4] - dt * (dc[4] + (F[4] - Fp[4]) * idz);
          Un[4] = a.stage1 ? tmp : ssp_combine(a.alpha, a.beta, u0c[4], tmp);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) Ol[v * NC + r * NT] = Un[v];
        if constexpr (LAST) {
          float wn[NV];
          march3::prim5(Un, gm1, wn);
          if (!(Un[0] > 0.f) || !(wn[4] > 0.f)) bad = 1;
          float cs = sqrtf(gam * wn[4] * f32::rcp(Un[0]));
          rate = fmaxf(rate, (fabsf(wn[1]) + cs) * idx + (fabsf(wn[2]) + cs) * idy + (fabsf(wn[3]) + cs) * idz);
#pragma unroll
          for (int v = 0; v < NV; ++v) march::two_sum_add(th[v], tl[v], Un[v] * vscale);
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Fp[v] = F[v];
        hiPrev[v] = hi[v];
        wm[v] = w0[v];
        w0[v] = wp[v];
      }
    }
  }
  if constexpr (LAST) {
    // ---- last stage: CTA max rate, CTA totals (fixed order), two-level finish
    for (int o = 16; o > 0; o >>= 1) {
      rate = fmaxf(rate, __shfl_xor_sync(0xffffffffu, rate, o));
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float h2 = __shfl_xor_sync(0xffffffffu, th[v], o), l2 = __shfl_xor_sync(0xffffffffu, tl[v], o);
        march::ff_add(th[v], tl[v], h2, l2);
      }
    }
    if (lane == 0) {
      red[warp][2 * NV] = rate;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        red[warp][v] = th[v];
        red[warp][NV + v] = tl[v];
      }
    }
    if (bad) sbad = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
      float mm = red[0][2 * NV], hh[NV], ll[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        hh[v] = red[0][v];
        ll[v] = red[0][NV + v];
      }
      for (int w = 1; w < 4; ++w) {
        mm = fmaxf(mm, red[w][2 * NV]);
#pragma unroll
        for (int v = 0; v < NV; ++v) march::ff_add(hh[v], ll[v], red[w][v], red[w][NV + v]);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) a.partials[(size_t)blockIdx.x * NV + v] = ((double)hh[v] + (double)ll[v]) * G.dV[1];
      __threadfence();  // the partials are visible before the group counter counts this CTA
      atomicMax(&a.ctl->smax_bits, MaxKey<float>::enc(mm));
      if (sbad) atomicOr(&a.ctl->status, 1);
    }
    last_cta_finish<float, NV, 128>(a.ctl, a.partials, a.gpart, a.gcount, (int)gridDim.x, 1, true, 0.0, false, true);
  }
}

}  // namespace amrgpu
