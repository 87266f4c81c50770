// Batched geometric multigrid for (lambda - lap_h) x = b on periodic or zero-flux
// (Neumann) grids, and the reaction-diffusion steps built on it.
//
// Paper: Sec. 2.5.1, Eq. (diff-helmholtz): the implicit diffusion stage is a
// Helmholtz problem solved by geometric multigrid (Sec. 1.4, linear cost);
// Eq. (imex): IMEX trapezoidal scheme; Eq. (splitting): the split scheme;
// Eqs. (gray-scott), (schnakenberg): reaction terms; Sec. 2.5.2: iterate until
// the maximum residual is below a fraction of the right-hand side, Neumann
// boundaries for the Schnakenberg runs.
//
// Neumann boundaries: a boundary face carries no flux, so a boundary cell sums
// only its in-domain neighbours and its diagonal is lambda + count / h^2 (the
// reciprocal diagonals are tabulated per level and per number of missing
// neighbours); the prolongation puts the weight of a coarse neighbour beyond the
// boundary on the parent.
//
// Layout: every multigrid instance owns a chain of levels (side n, n/2, ...,
// coarsest when the side is odd or <= coarse_max); level arrays of all
// instances are packed in one buffer per quantity.  Work is described by
// per-depth chunk lists (instance, first index, count), so one launch per
// sweep covers every instance deep enough for that depth.  The float64
// iterate X and right-hand side B live on level 0; V-cycles run on the
// correction in `real` (float or double): R = B - A X (float64) -> V-cycle on
// A e = R -> X += e (defect correction).  The coarsest level is solved with a
// precomputed dense inverse, applied in float64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/amrvac_gb300.h"
#include "mg_internal.h"

namespace mggpu {

constexpr int kMaxLev = 16;
constexpr int kChunk = 256;

struct Chunk {
  int inst, lev;
  long long start;
  int count;
};

struct InstDev {
  int nlev;
  int n[kMaxLev];
  long long off[kMaxLev];  // offsets into the level buffers
  double ih2[kMaxLev];
  float ih2f[kMaxLev];
  double lam;
  float lamf;
  float lamlo;    // lambda - lamf (float-float lambda for the level-0 defect update)
  float ih2lo0;   // ih2[0] - ih2f[0]
  double idiag[kMaxLev][7];     // 1 / (lambda + (2 ndim - m) / h^2) for m neighbours beyond a
  float idiagf[kMaxLev][7];     // Neumann boundary (m = 0 inside and on periodic grids)
  long long off0;          // offset into X / B
  long long inv_off;       // offset into the coarsest inverse matrices
  int dsm;                 // 2D: first depth whose V-cycle part runs in shared memory, or -1
};

struct MgState {
  const InstDev* inst;
  double* X;
  const double* B;
  double* R;                  // float32 V-cycles: level-0 float64 defect B - A X, kept up to date
  unsigned long long* rnorm;  // max |R| bits per instance
  double* bnorm;              // max |B| per instance
  double* lastres;            // last max |R| per instance
  double* initres;            // max |R| of the initial guess per instance
  int* active;                // instance still iterating
  int* cycles;
  int* failed;
  int* any;                   // any instance active (for the host)
  int* iters;                 // loop iterations of the current solve (device-side loop cap)
  const double* inv;          // dense inverses of the coarsest operators
  const float* invf;          // the same rounded to float32 (float32 cycles solve in float32)
  int ndim;
  int neu;                    // Neumann (zero-flux) boundaries, else periodic
  double rtol;
  int max_cycles;
};

template <typename real>
struct Lvl {
  real* x;
  real* b;
};

// cell coordinates of index t of an n^nd grid (setup keeps n^nd below 2^31, so the
// divisions are 32-bit)
__device__ __forceinline__ void cell_of(long long t, int n, int nd, int* c) {
  unsigned u = (unsigned)t, un = (unsigned)n;
  unsigned r = u / un;
  c[0] = (int)(u - r * un);
  if (nd > 2) {
    unsigned z = r / un;
    c[1] = (int)(r - z * un);
    c[2] = (int)z;
  } else {
    c[1] = nd > 1 ? (int)r : 0;
    c[2] = 0;
  }
}

// max of a non-negative double over the block, as its bit pattern (the order of the
// bit patterns of non-negative doubles is their numeric order), one atomic per block
__device__ __forceinline__ void block_max_atomic(unsigned long long m, unsigned long long* dst) {
  __shared__ unsigned long long wm[32];
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wm[w] > m ? wm[w] : m;
    if (m) atomicMax(dst, m);
  }
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ long long lin(const int* c, int n) {
  return (long long)c[0] + (long long)n * ((long long)c[1] + (long long)n * c[2]);
}

// neighbour index i (at most one cell outside [0, n)): the periodic image, or the cell
// itself (ci) beyond a Neumann boundary, where the prolongation uses the parent
__device__ __forceinline__ int nbr_or_self(int i, int ci, int n, bool neu) {
  return i < 0 ? (neu ? ci : i + n) : (i >= n ? (neu ? ci : i - n) : i);
}

// sum of the neighbours, ordered x-, x+, y-, y+, z-, z+: all 2 ndim on a periodic grid
// (images across the boundary), only the in-domain ones on a Neumann grid (NEU); *miss gets
// the number left out
template <bool NEU, typename T>
__device__ __forceinline__ T nbsum(const T* x, const int* c, int n, int nd, int* miss) {
  if constexpr (!NEU) {
    *miss = 0;
    int q[3] = {c[0], c[1], c[2]};
    q[0] = wrapi(c[0] - 1, n);
    T s = x[lin(q, n)];
    q[0] = wrapi(c[0] + 1, n);
    s = s + x[lin(q, n)];
    q[0] = c[0];
    if (nd > 1) {
      q[1] = wrapi(c[1] - 1, n);
      s = s + x[lin(q, n)];
      q[1] = wrapi(c[1] + 1, n);
      s = s + x[lin(q, n)];
      q[1] = c[1];
    }
    if (nd > 2) {
      q[2] = wrapi(c[2] - 1, n);
      s = s + x[lin(q, n)];
      q[2] = wrapi(c[2] + 1, n);
      s = s + x[lin(q, n)];
    }
    return s;
  } else {
    T s = T(0);
    int m = 0;
    for (int d = 0; d < nd; ++d) {
#pragma unroll
      for (int side = -1; side <= 1; side += 2) {
        int q[3] = {c[0], c[1], c[2]};
        int t = c[d] + side;
        if (t < 0 || t >= n) {
          ++m;
          continue;
        }
        q[d] = t;
        s = s + x[lin(q, n)];
      }
    }
    *miss = m;
    return s;
  }
}

template <typename real>
__device__ __forceinline__ real ih2_of(const InstDev& I, int l);
template <>
__device__ __forceinline__ double ih2_of<double>(const InstDev& I, int l) { return I.ih2[l]; }
template <>
__device__ __forceinline__ float ih2_of<float>(const InstDev& I, int l) { return I.ih2f[l]; }
template <typename real>
__device__ __forceinline__ real idiag_of(const InstDev& I, int l, int miss);
template <>
__device__ __forceinline__ double idiag_of<double>(const InstDev& I, int l, int miss) { return I.idiag[l][miss]; }
template <>
__device__ __forceinline__ float idiag_of<float>(const InstDev& I, int l, int miss) { return I.idiagf[l][miss]; }
template <typename real>
__device__ __forceinline__ real lam_of(const InstDev& I);
template <>
__device__ __forceinline__ double lam_of<double>(const InstDev& I) { return I.lam; }
template <>
__device__ __forceinline__ float lam_of<float>(const InstDev& I) { return I.lamf; }

// IEEE-754 widening and narrowing between float32 and float64 by bit manipulation, on the
// integer units (GB300's float64 pipe is ~1/64 of its float32 rate and bounds the defect
// correction).  Widening is exact, subnormals included.  Narrowing truncates the 29 dropped
// mantissa bits and flushes values below the float normal range to zero, which is enough for
// the right-hand side of a correction equation.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f), e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  unsigned long long bits;
  if (e == 0u) {
    if (m == 0u) {
      bits = sign;  // signed zero
    } else {        // subnormal: m 2^-149 = 2^(p-149) (m / 2^p), p = position of the leading one
      const int p = 31 - __clz(m);
      bits = sign | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
    }
  } else if (e == 0xffu) {
    bits = sign | (0x7ffull << 52) | ((unsigned long long)m << 29);  // infinity, NaN (payload kept)
  } else {
    bits = sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  }
  return __longlong_as_double((long long)bits);
}
template <typename real>
__device__ __forceinline__ real narrow(double d);
template <>
__device__ __forceinline__ double narrow<double>(double d) { return d; }
template <>
__device__ __forceinline__ float narrow<float>(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ffu) - 896;  // float exponent field
  const unsigned m = (unsigned)((b >> 29) & 0x7fffffull);
  unsigned u;
  if (e <= 0) u = sign;                                                             // below 2^-126: zero
  else if (e >= 255) u = sign | 0x7f800000u | ((b & 0xfffffffffffffull) ? 0x400000u : 0u);  // overflow, inf, NaN
  else u = sign | ((unsigned)e << 23) | m;
  return __uint_as_float(u);
}

// ---------------------------------------------------------------- kernels --
// max |B| per instance (level-0 chunks)
__global__ void bnorm_kernel(MgState S, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];
  unsigned long long m = 0ull;
  if (threadIdx.x < C.count) {
    const InstDev& I = S.inst[C.inst];
    m = (unsigned long long)__double_as_longlong(fabs(S.B[I.off0 + C.start + threadIdx.x]));
  }
  block_max_atomic(m, &S.rnorm[C.inst]);
}

__global__ void bnorm_finish_kernel(MgState S, int ninst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *S.iters = 0;
  if (i >= ninst) return;
  S.bnorm[i] = __longlong_as_double((long long)S.rnorm[i]);
  S.rnorm[i] = 0ull;
  S.active[i] = 1;
  S.cycles[i] = 0;
  S.failed[i] = 0;
}

// float64 residual R = B - (lambda X - lap X) on level 0 -> rhs of the correction,
// correction zeroed, per-instance max |R|
template <typename real, bool NEU>
__global__ void residual64_kernel(MgState S, Lvl<real> L, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];
  if (!S.active[C.inst]) return;
  unsigned long long m = 0ull;
  const InstDev& I = S.inst[C.inst];
  if (threadIdx.x < C.count) {
    long long t = C.start + threadIdx.x;
    int n = I.n[0];
    int c[3];
    cell_of(t, n, S.ndim, c);
    const double* X = S.X + I.off0;
    double x = X[t];
    // r = B + ih2 (nbsum - count x) - lambda x in three fused multiply-adds: the float64
    // unit is GB300's scarcest pipe, so the residual uses as few float64 operations as it can
    int miss;
    const double s = nbsum<NEU>(X, c, n, S.ndim, &miss);
    const double mcount = NEU ? (double)(miss - 2 * S.ndim) : (S.ndim == 3 ? -6.0 : -4.0);
    double r = fma(fma(mcount, x, s), I.ih2[0], S.B[I.off0 + t]);
    r = fma(-I.lam, x, r);
    if constexpr (sizeof(real) == 4) S.R[I.off0 + t] = r;
    L.b[I.off[0] + t] = narrow<real>(r);
    L.x[I.off[0] + t] = real(0);
    m = (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffull;  // |r| as bits
  }
  block_max_atomic(m, &S.rnorm[C.inst]);
}

// convergence test per instance (the paper's max-residual rule)
// cond != 0: the kernel runs inside a graph's device-side while loop and sets the loop
// condition (some instance still iterating); the loop also stops after max_cycles + 1 checks
// whatever the flags say, so it always ends.
__global__ void check_kernel(MgState S, int ninst, cudaGraphConditionalHandle hc, int cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < ninst; i += blockDim.x) {
    if (!S.active[i]) continue;
    double rn = __longlong_as_double((long long)S.rnorm[i]);
    S.rnorm[i] = 0ull;
    S.lastres[i] = rn;
    if (S.cycles[i] == 0) S.initres[i] = rn;
    if (rn <= S.rtol * S.bnorm[i]) {
      S.active[i] = 0;
    } else if (S.cycles[i] >= S.max_cycles) {
      S.active[i] = 0;
      S.failed[i] = 1;
    } else {
      S.cycles[i] += 1;
      atomicOr(&any, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *S.any = any;
    if (cond) {
      const int it = ++*S.iters;
      cudaGraphSetConditional(hc, (any && it <= S.max_cycles + 1) ? 1u : 0u);
    }
  }
}

// red-black Gauss-Seidel sweep of one colour: x = (b + nbsum * ih2) / (lambda + count ih2)
template <typename real, bool NEU>
__global__ void smooth_kernel(MgState S, Lvl<real> L, const Chunk* ch, int colour) {
  Chunk C = ch[blockIdx.x];
  if (!S.active[C.inst] || threadIdx.x >= C.count) return;
  const InstDev& I = S.inst[C.inst];
  const int l = C.lev, n = I.n[l], nd = S.ndim;
  unsigned t = (unsigned)(C.start + threadIdx.x);  // index among the cells of this colour
  unsigned half = (unsigned)n / 2u;
  int c[3];
  unsigned row = t / half;
  int ii = (int)(t - row * half);
  unsigned z = row / (unsigned)n;
  c[1] = nd > 1 ? (int)(row - z * (unsigned)n) : 0;
  c[2] = nd > 2 ? (int)z : 0;
  c[0] = 2 * ii + ((c[1] + c[2] + colour) & 1);
  real* x = L.x + I.off[l];
  const real* b = L.b + I.off[l];
  real ih2 = ih2_of<real>(I, l);
  long long q = lin(c, n);
  int miss;
  const real sn = nbsum<NEU>(x, c, n, nd, &miss);
  x[q] = (b[q] + sn * ih2) * idiag_of<real>(I, l, NEU ? miss : 0);
}

// One full red-black sweep of a 2D level, one warp per strip of kStripW columns and
// H rows (H per depth from the strip-height tuner, carried in the chunk's count).  Lane k
// holds the column pair (x0 - 2 + 2k, x0 - 1 + 2k) (periodic): one red and one black cell
// per row, read and written as one float2 / double2 (swept levels have an even side and
// level offsets are multiples of 4 cells, so pairs are aligned and never straddle the
// periodic wrap); lanes 0 and 31 are halo.  Walking the strip's rows, a lane keeps three
// rows of old values and three rows of red-updated values in registers (loads run kPre
// rows ahead): at row s it updates the red cell of row s + 1 (old black neighbours: its
// own rows s and s + 2, its own black cell and one from the lane beside it), then the
// black cell of row s (red-updated neighbours: its rows s - 1 and s + 1, its own red cell
// and one from the lane beside it), and stores row s.  It reads one iterate array and
// writes the other, so no warp sees another's writes; the updates and their arithmetic
// (neighbour sums in the order x-, x+, y-, y+) are those of two in-place colour sweeps.
// NEU (zero-flux boundaries): cells outside the domain read as 0 and are never updated,
// so they add nothing to a neighbour sum, and a boundary cell divides by its own diagonal
// lambda + count / h^2.  XZERO: the first sweep of a correction, whose initial iterate is
// zero (not read).
constexpr int kStripW = 60, kStripHMax = 64, kPre = 4;

inline int strip_height(int n) { return std::min(kStripHMax, std::max(8, n / 32)); }

// Autotuner of the strip height H of the 2D sweep, per depth of the batch: candidate heights,
// and the process-wide cache of the measured choice keyed by (sides, precision, boundary kind).
constexpr int kStripCandidates[] = {4, 8, 16, 32, 64};
inline std::map<std::string, int>& strip_cache() {
  static std::map<std::string, int> m;
  return m;
}
inline std::mutex& strip_cache_mutex() {
  static std::mutex m;
  return m;
}
constexpr unsigned kFull = 0xffffffffu;

template <typename real>
struct Pair;
template <>
struct Pair<float> {
  using T = float2;
};
template <>
struct Pair<double> {
  using T = double2;
};

struct StripGeom {
  int n, ca, cw, x0, y0, y1;
  bool out_lane;
};

// strip `start` of a level of (even) side n with strips of H rows, seen by lane `lane`
__device__ __forceinline__ StripGeom strip_geom(int n, long long start, int H, int lane) {
  StripGeom g;
  const int nsx = (n + kStripW - 1) / kStripW;
  const int sx = (int)(start % nsx), sy = (int)(start / nsx);
  g.n = n;
  g.x0 = sx * kStripW;
  g.y0 = sy * H;
  g.y1 = min(g.y0 + H, n);
  g.ca = g.x0 - 2 + 2 * lane;  // the pair's first column before the periodic wrap
  g.cw = ((g.ca % n) + n) % n;
  g.out_lane = lane >= 1 && lane <= 30 && g.ca < n;
  return g;
}

__device__ __forceinline__ int wrap_row(int r, int n) { return r < 0 ? r + n : (r >= n ? r - n : r); }

template <typename real, bool NEU, bool XZERO = false>
__global__ void __launch_bounds__(128)
    sweep2d_kernel(MgState S, const real* __restrict__ xin, real* __restrict__ xout, const real* __restrict__ bl,
                   const Chunk* ch, int nch) {
  using V2 = typename Pair<real>::T;
  const int lane = threadIdx.x & 31;
  const int wi = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (wi >= nch) return;
  const Chunk C = ch[wi];
  if (!S.active[C.inst]) return;
  const InstDev& I = S.inst[C.inst];
  const int l = C.lev;
  const StripGeom g = strip_geom(I.n[l], C.start, C.count, lane);
  const int n = g.n, ca = g.ca, cw = g.cw;
  const real* x = xin + I.off[l];
  const real* b = bl + I.off[l];
  real* xo = xout + I.off[l];
  const real ih2 = ih2_of<real>(I, l), idg = idiag_of<real>(I, l, 0);
  // rows stay within one period of [0, n) when n > H + kPre + 2; else a full modulo
  const bool one_wrap = n > C.count + kPre + 2;
  auto rowof = [&](int r) { return one_wrap ? wrap_row(r, n) : ((r % n) + n) % n; };
  const bool colin = ca >= 0 && ca < n;  // the pair lies in the domain (both or neither: n even)
  auto inside = [&](int r) { return !NEU || (colin && r >= 0 && r < n); };
  auto ld2 = [&](const real* p, int r) { return *reinterpret_cast<const V2*>(p + rowof(r) * n + cw); };
  auto ldx = [&](int r) {
    if constexpr (XZERO) return V2{real(0), real(0)};
    else return inside(r) ? ld2(x, r) : V2{real(0), real(0)};
  };
  auto ldb = [&](int r) { return ld2(b, r); };
  // reciprocal diagonal of the pair's cell in column ca + e, row r
  auto idg_at = [&](int e, int r) {
    if constexpr (!NEU) return idg;
    const int c = ca + e;
    const int m = (c == 0) + (c == n - 1) + (r == 0) + (r == n - 1);
    return idiag_of<real>(I, l, m);
  };
  // red update of row r from old rows om, o0 (row r), op: the red cell is the first of the
  // pair on even rows (n even: the parity of r is that of its periodic image), the second on
  // odd ones; the black cell keeps o0
  auto red = [&](V2 om, V2 o0, V2 op, V2 bb, int r) {
    V2 out;
    if ((r & 1) == 0) {
      const real lft = __shfl_up_sync(kFull, o0.y, 1);
      out = V2{(bb.x + (lft + o0.y + om.x + op.x) * ih2) * idg_at(0, r), o0.y};
    } else {
      const real rgt = __shfl_down_sync(kFull, o0.x, 1);
      out = V2{o0.x, (bb.y + (o0.x + rgt + om.y + op.y) * ih2) * idg_at(1, r)};
    }
    return inside(r) ? out : V2{real(0), real(0)};
  };
  const int y0 = g.y0, y1 = g.y1;
  // old rows y0-2 .. y0+1, red rows y0-1 and y0
  V2 o_a = ldx(y0 - 2), o_b = ldx(y0 - 1), o_c = ldx(y0), o_d = ldx(y0 + 1);
  V2 b_c = ldb(y0 - 1), b_d = ldb(y0);
  V2 r_m = red(o_a, o_b, o_c, b_c, y0 - 1);
  V2 r_0 = red(o_b, o_c, o_d, b_d, y0);
  V2 b_0 = b_d;
  // prefetch ring: old rows s+2 .. s+1+kPre and right-hand sides of rows s+1 .. s+kPre
  V2 px[kPre], pb[kPre];
#pragma unroll
  for (int k = 0; k < kPre; ++k) {
    px[k] = y0 + 2 + k <= y1 + 1 ? ldx(y0 + 2 + k) : V2{real(0), real(0)};
    pb[k] = y0 + 1 + k <= y1 ? ldb(y0 + 1 + k) : V2{real(0), real(0)};
  }
  V2 o_s = o_c, o_s1 = o_d;  // old rows s, s+1
#pragma unroll 4
  for (int s = y0; s < y1; ++s) {
    const V2 o_s2 = px[0], b_s1 = pb[0];
#pragma unroll
    for (int k = 0; k + 1 < kPre; ++k) {
      px[k] = px[k + 1];
      pb[k] = pb[k + 1];
    }
    px[kPre - 1] = s + 2 + kPre <= y1 + 1 ? ldx(s + 2 + kPre) : V2{real(0), real(0)};
    pb[kPre - 1] = s + 1 + kPre <= y1 ? ldb(s + 1 + kPre) : V2{real(0), real(0)};
    const V2 r_p = red(o_s, o_s1, o_s2, b_s1, s + 1);
    // black cell of row s: the second of the pair on even rows, the first on odd ones
    V2 outv;
    if ((s & 1) == 0) {
      const real rgt = __shfl_down_sync(kFull, r_0.x, 1);
      outv = V2{r_0.x, (b_0.y + (r_0.x + rgt + r_m.y + r_p.y) * ih2) * idg_at(1, s)};
    } else {
      const real lft = __shfl_up_sync(kFull, r_0.y, 1);
      outv = V2{(b_0.x + (lft + r_0.y + r_m.x + r_p.x) * ih2) * idg_at(0, s), r_0.y};
    }
    if (g.out_lane) *reinterpret_cast<V2*>(xo + s * n + ca) = outv;
    r_m = r_0;
    r_0 = r_p;
    b_0 = b_s1;
    o_s = o_s1;
    o_s1 = o_s2;
  }
}

// copy of one strip (after an odd number of sweeps)
template <typename real>
__global__ void __launch_bounds__(128) copy2d_kernel(MgState S, const real* __restrict__ xin, real* __restrict__ xout,
                                                     const Chunk* ch, int nch) {
  using V2 = typename Pair<real>::T;
  const int lane = threadIdx.x & 31;
  const int wi = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (wi >= nch) return;
  const Chunk C = ch[wi];
  if (!S.active[C.inst]) return;
  const InstDev& I = S.inst[C.inst];
  const StripGeom g = strip_geom(I.n[C.lev], C.start, C.count, lane);
  if (!g.out_lane) return;
  const long long o = I.off[C.lev];
  for (int s = g.y0; s < g.y1; ++s)
    *reinterpret_cast<V2*>(xout + o + s * g.n + g.ca) = *reinterpret_cast<const V2*>(xin + o + s * g.n + g.ca);
}

// 2D prolongation, one thread per coarse cell writing its four fine children
// 2D residual and restriction of coarse cell (ci, cj): the 4 x 4 patch of fine iterate values
// around its 2 x 2 children (corners excepted) is loaded once, then each child's residual
// b - (lambda x - lap x) is formed with the neighbour sum in the order x-, x+, y-, y+ (as
// nbsum) and the four are summed in x-fastest order (as resrestrict_kernel).  x, b: the fine
// level (global or shared memory); nf its side.
template <typename real, bool NEU>
__device__ __forceinline__ real restrict_cell2d(const real* x, const real* b, int nf, int ci, int cj, real ih2,
                                                real lam) {
  const int x0 = 2 * ci, y0 = 2 * cj;
  // patch columns x0-1 .. x0+2 and rows y0-1 .. y0+2: periodic images, or -1 outside a
  // zero-flux boundary
  const int col[4] = {x0 > 0 ? x0 - 1 : (NEU ? -1 : nf - 1), x0, x0 + 1, x0 + 2 < nf ? x0 + 2 : (NEU ? -1 : 0)};
  const int row[4] = {y0 > 0 ? y0 - 1 : (NEU ? -1 : nf - 1), y0, y0 + 1, y0 + 2 < nf ? y0 + 2 : (NEU ? -1 : 0)};
  real P[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const bool corner = (r == 0 || r == 3) && (c == 0 || c == 3);
      P[r][c] = (!corner && row[r] >= 0 && col[c] >= 0) ? x[row[r] * nf + col[c]] : real(0);
    }
  real sum = real(0);
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int a = o & 1, bb = o >> 1, r = 1 + bb, c = 1 + a;
    const real xv = P[r][c];
    int miss = 0;
    real sn;
    if constexpr (!NEU) {
      sn = P[r][c - 1];
      sn = sn + P[r][c + 1];
      sn = sn + P[r - 1][c];
      sn = sn + P[r + 1][c];
    } else {
      sn = real(0);
      if (col[c - 1] >= 0) sn = sn + P[r][c - 1]; else ++miss;
      if (col[c + 1] >= 0) sn = sn + P[r][c + 1]; else ++miss;
      if (row[r - 1] >= 0) sn = sn + P[r - 1][c]; else ++miss;
      if (row[r + 1] >= 0) sn = sn + P[r + 1][c]; else ++miss;
    }
    const real lap = (sn - real(4 - miss) * xv) * ih2;
    sum = sum + (b[row[r] * nf + col[c]] - (lam * xv - lap));
  }
  return sum * real(0.25);
}

// 2D residual and restriction, one thread per coarse cell
template <typename real, bool NEU>
__global__ void resrestrict2d_kernel(MgState S, Lvl<real> L, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];
  if (!S.active[C.inst] || threadIdx.x >= C.count) return;
  const InstDev& I = S.inst[C.inst];
  const int l = C.lev;
  const int nc = I.n[l + 1], nf = I.n[l];
  const unsigned t = (unsigned)C.start + threadIdx.x;  // coarse cell
  const int cj = (int)(t / (unsigned)nc), ci = (int)(t - (unsigned)cj * (unsigned)nc);
  L.b[I.off[l + 1] + t] =
      restrict_cell2d<real, NEU>(L.x + I.off[l], L.b + I.off[l], nf, ci, cj, ih2_of<real>(I, l), lam_of<real>(I));
  L.x[I.off[l + 1] + t] = real(0);
}

// 2D prolongation of coarse cell (ci, cj) of ec (side nc) onto its four children in xf (side
// nf): bilinear weights 9/16, 3/16, 3/16, 1/16 in the order (x, y) = (0,0), (1,0), (0,1), (1,1),
// the coarse cell itself beyond a zero-flux boundary
template <typename real, bool NEU>
__device__ __forceinline__ void prolong_cell2d(const real* ec, real* xf, int nc, int nf, int ci, int cj) {
  real v[3][3];
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
    for (int di = -1; di <= 1; ++di)
      v[dj + 1][di + 1] = ec[nbr_or_self(cj + dj, cj, nc, NEU) * nc + nbr_or_self(ci + di, ci, nc, NEU)];
  // each row pair of children as one vector (nf even, level offsets multiples of 4 cells)
  using V2 = typename Pair<real>::T;
#pragma unroll
  for (int b2 = 0; b2 < 2; ++b2) {
    const int sy = b2 ? 1 : -1;
    real acc[2];
#pragma unroll
    for (int a2 = 0; a2 < 2; ++a2) {
      const int sx = a2 ? 1 : -1;
      acc[a2] = real(0);
      acc[a2] = acc[a2] + real(0.5625) * v[1][1];
      acc[a2] = acc[a2] + real(0.1875) * v[1][1 + sx];
      acc[a2] = acc[a2] + real(0.1875) * v[1 + sy][1];
      acc[a2] = acc[a2] + real(0.0625) * v[1 + sy][1 + sx];
    }
    V2* q = reinterpret_cast<V2*>(xf + (2 * cj + b2) * nf + 2 * ci);
    const V2 o = *q;
    *q = V2{o.x + acc[0], o.y + acc[1]};
  }
}

template <typename real, bool NEU>
__global__ void prolong2d_kernel(MgState S, Lvl<real> L, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];
  if (!S.active[C.inst] || threadIdx.x >= C.count) return;
  const InstDev& I = S.inst[C.inst];
  const int l = C.lev;
  const int nf = I.n[l], nc = I.n[l + 1];
  unsigned t = (unsigned)(C.start + threadIdx.x);  // coarse cell
  int cj = (int)(t / (unsigned)nc), ci = (int)(t - (unsigned)cj * (unsigned)nc);
  prolong_cell2d<real, NEU>(L.x + I.off[l + 1], L.x + I.off[l], nc, nf, ci, cj);
}

// residual of level l restricted to level l+1 (mean of the 2^ndim children), x_{l+1} = 0
template <typename real, bool NEU>
__global__ void resrestrict_kernel(MgState S, Lvl<real> L, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];
  if (!S.active[C.inst] || threadIdx.x >= C.count) return;
  const InstDev& I = S.inst[C.inst];
  const int l = C.lev, nd = S.ndim;  // chunk enumerates cells of level l+1
  const int nc = I.n[l + 1], nf = I.n[l];
  long long t = C.start + threadIdx.x;
  int cc[3];
  cell_of(t, nc, nd, cc);
  const real* x = L.x + I.off[l];
  const real* b = L.b + I.off[l];
  real ih2 = ih2_of<real>(I, l), lam = lam_of<real>(I);
  real sum = real(0);
  for (int o = 0; o < (1 << nd); ++o) {
    int f[3] = {2 * cc[0] + (o & 1), nd > 1 ? 2 * cc[1] + ((o >> 1) & 1) : 0, nd > 2 ? 2 * cc[2] + ((o >> 2) & 1) : 0};
    long long q = lin(f, nf);
    real xv = x[q];
    int miss;
    const real sn = nbsum<NEU>(x, f, nf, nd, &miss);
    real lap = (sn - real(2 * nd - (NEU ? miss : 0)) * xv) * ih2;
    sum = sum + (b[q] - (lam * xv - lap));
  }
  L.b[I.off[l + 1] + t] = sum * (real(1) / real(1 << nd));
  L.x[I.off[l + 1] + t] = real(0);
}

// cell-centred (bi/tri)linear prolongation of level l+1 added to level l
template <typename real, bool NEU>
__global__ void prolong_kernel(MgState S, Lvl<real> L, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];
  if (!S.active[C.inst] || threadIdx.x >= C.count) return;
  const InstDev& I = S.inst[C.inst];
  const int l = C.lev, nd = S.ndim;
  const int nf = I.n[l], nc = I.n[l + 1];
  long long t = C.start + threadIdx.x;
  int f[3];
  cell_of(t, nf, nd, f);
  int P[3] = {f[0] >> 1, f[1] >> 1, f[2] >> 1};
  int sg[3] = {(f[0] & 1) ? 1 : -1, (f[1] & 1) ? 1 : -1, (f[2] & 1) ? 1 : -1};
  const real* ec = L.x + I.off[l + 1];
  real acc = real(0);
  int cz = nd > 2 ? 2 : 1, cy = nd > 1 ? 2 : 1;
  for (int z = 0; z < cz; ++z)
    for (int y = 0; y < cy; ++y)
      for (int xx = 0; xx < 2; ++xx) {
        constexpr bool neu = NEU;
        int q[3] = {nbr_or_self(P[0] + xx * sg[0], P[0], nc, neu), nd > 1 ? nbr_or_self(P[1] + y * sg[1], P[1], nc, neu) : 0,
                    nd > 2 ? nbr_or_self(P[2] + z * sg[2], P[2], nc, neu) : 0};
        real w = xx ? real(0.25) : real(0.75);
        if (nd > 1) w = w * (y ? real(0.25) : real(0.75));
        if (nd > 2) w = w * (z ? real(0.25) : real(0.75));
        acc = acc + w * ec[lin(q, nc)];
      }
  real* x = L.x + I.off[l] + t;
  *x = *x + acc;
}

// coarsest level: x = inverse(A) b, float64, a warp per row
// float32 cycles: the float32 inverse and float32 sums (the correction is float32 anyway, and
// GB300's float64 pipe made the float64 product the slowest kernel of the coarse levels)
__device__ __forceinline__ float coarse_row(const float* A, int r, int m, const float* b, int lane) {
  float acc = 0.f;
  for (int c = lane; c < m; c += 32) acc = fmaf(A[(size_t)r * m + c], b[c], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}
__device__ __forceinline__ double coarse_row(const double* A, int r, int m, const double* b, int lane) {
  double acc = 0.0;
  for (int c = lane; c < m; c += 32) acc += A[(size_t)r * m + c] * b[c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

template <typename real>
__global__ void coarse_kernel(MgState S, Lvl<real> L, const int* insts, const int* rows0, int nitems) {
  int item = blockIdx.x;
  if (item >= nitems) return;
  int i = insts[item];
  if (!S.active[i]) return;
  const InstDev& I = S.inst[i];
  int l = I.nlev - 1, n = I.n[l];
  int m = n;
  for (int d = 1; d < S.ndim; ++d) m *= n;
  const real* b = L.b + I.off[l];
  real* x = L.x + I.off[l];
  const real* A;
  if constexpr (sizeof(real) == 4) A = S.invf + I.inv_off;
  else A = S.inv + I.inv_off;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = rows0[item] + warp; r < min(m, rows0[item] + 64); r += blockDim.x / 32) {
    const real acc = coarse_row(A, r, m, b, lane);
    if (lane == 0) x[r] = acc;
  }
}

// The coarse part of a 2D V-cycle of one instance in shared memory, one CTA per instance:
// depths I.dsm .. nlev - 1 (sides up to 64).  It takes the
// right-hand side of depth dsm from the restriction above it and returns the correction of
// that depth, doing in between what the per-depth kernels do, in their order and with their
// arithmetic: nu1 red-black sweeps from a zero correction (each an in-place red pass, then a
// black pass, as the strip sweep computes them), residual and restriction, the dense solve
// of the coarsest level, then prolongation and nu2 sweeps back up.  A block barrier separates
// the passes.  Shared layout per depth: x, then b, each padded to 4 cells.
constexpr int kCoarseThreads = 1024;
constexpr int kCoarseSideF32 = 64, kCoarseSideF64 = 64;  // largest side of its first depth

template <typename real, bool NEU>
__global__ void __launch_bounds__(kCoarseThreads)
    coarse2d_kernel(MgState S, Lvl<real> L, const int* insts, int nu1, int nu2) {
  extern __shared__ __align__(16) unsigned char cv_smem[];
  real* sm = reinterpret_cast<real*>(cv_smem);
  const int i = insts[blockIdx.x];
  if (!S.active[i]) return;
  const InstDev& I = S.inst[i];
  const int d0 = I.dsm, nl = I.nlev, tid = threadIdx.x;
  __shared__ int so[kMaxLev];  // shared offset of each depth's x
  if (tid == 0) {
    int o = 0;
    for (int l = d0; l < nl; ++l) {
      so[l] = o;
      o += 2 * ((I.n[l] * I.n[l] + 3) & ~3);
    }
  }
  __syncthreads();
  auto X = [&](int l) { return sm + so[l]; };
  auto Bv = [&](int l) { return sm + so[l] + ((I.n[l] * I.n[l] + 3) & ~3); };
  {
    const int m = I.n[d0] * I.n[d0];
    const real* bg = L.b + I.off[d0];
    for (int c = tid; c < m; c += kCoarseThreads) {
      Bv(d0)[c] = bg[c];
      X(d0)[c] = real(0);
    }
  }
  __syncthreads();
  // one red-black sweep of depth l in place: cells (c + r) even, then odd; neighbour sums in
  // the order x-, x+, y-, y+, cells beyond a zero-flux boundary read as zero
  // threads as 16 rows x 64 cells of one colour (a side of at most 128)
  const int tx = tid & 63, ty = tid >> 6;
  auto sweep = [&](int l) {
    const int n = I.n[l], hn = n / 2;
    real* x = X(l);
    const real* b = Bv(l);
    const real ih2 = ih2_of<real>(I, l), idg = idiag_of<real>(I, l, 0);
    for (int colour = 0; colour < 2; ++colour) {
      for (int r = ty; r < n; r += kCoarseThreads / 64)
        for (int k = tx; k < hn; k += 64) {
          const int c = 2 * k + ((r + colour) & 1);
          const int cm = c > 0 ? c - 1 : n - 1, cp = c + 1 < n ? c + 1 : 0;
          const int rm = r > 0 ? r - 1 : n - 1, rp = r + 1 < n ? r + 1 : 0;
          real lft = x[r * n + cm], rgt = x[r * n + cp], dn = x[rm * n + c], up = x[rp * n + c];
          real d = idg;
          if constexpr (NEU) {
            lft = c > 0 ? lft : real(0);
            rgt = c + 1 < n ? rgt : real(0);
            dn = r > 0 ? dn : real(0);
            up = r + 1 < n ? up : real(0);
            d = idiag_of<real>(I, l, (c == 0) + (c == n - 1) + (r == 0) + (r == n - 1));
          }
          x[r * n + c] = (b[r * n + c] + (lft + rgt + dn + up) * ih2) * d;
        }
      __syncthreads();
    }
  };
  for (int l = d0; l + 1 < nl; ++l) {
    for (int s2 = 0; s2 < nu1; ++s2) sweep(l);
    const int nc = I.n[l + 1];
    for (int t = tid; t < nc * nc; t += kCoarseThreads) {
      const int cj = t / nc, ci = t - cj * nc;
      Bv(l + 1)[t] = restrict_cell2d<real, NEU>(X(l), Bv(l), I.n[l], ci, cj, ih2_of<real>(I, l), lam_of<real>(I));
      X(l + 1)[t] = real(0);
    }
    __syncthreads();
  }
  {
    const int m = I.n[nl - 1] * I.n[nl - 1];
    const real* A;
    if constexpr (sizeof(real) == 4) A = S.invf + I.inv_off;
    else A = S.inv + I.inv_off;
    const int warp = tid >> 5, lane = tid & 31;
    for (int r = warp; r < m; r += kCoarseThreads / 32) {
      const real acc = coarse_row(A, r, m, Bv(nl - 1), lane);
      if (lane == 0) X(nl - 1)[r] = acc;
    }
    __syncthreads();
  }
  for (int l = nl - 2; l >= d0; --l) {
    const int nc = I.n[l + 1];
    for (int t = tid; t < nc * nc; t += kCoarseThreads) {
      const int cj = t / nc, ci = t - cj * nc;
      prolong_cell2d<real, NEU>(X(l + 1), X(l), nc, I.n[l], ci, cj);
    }
    __syncthreads();
    for (int s2 = 0; s2 < nu2; ++s2) sweep(l);
  }
  {
    const int m = I.n[d0] * I.n[d0];
    real* xg = L.x + I.off[d0];
    for (int c = tid; c < m; c += kCoarseThreads) xg[c] = X(d0)[c];
  }
}

template <typename real>
__global__ void correct64_kernel(MgState S, Lvl<real> L, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];
  if (!S.active[C.inst] || threadIdx.x >= C.count) return;
  const InstDev& I = S.inst[C.inst];
  long long t = C.start + threadIdx.x;
  const real e = L.x[I.off[0] + t];
  if constexpr (sizeof(real) == 4)
    S.X[I.off0 + t] = S.X[I.off0 + t] + widen(e);
  else
    S.X[I.off0 + t] = S.X[I.off0 + t] + e;
}

// float-float arithmetic (Dekker / Knuth error-free transformations) for the defect update.
// The _rn intrinsics keep every product and sum rounded on its own: a multiply-add
// contraction would break the exactness the transformations rely on.
struct FF {
  float hi, lo;
};
// a + b exactly as s + err (TwoSum), err folded into the low part, renormalised
__device__ __forceinline__ FF ff_add(FF a, float b) {
  const float s = __fadd_rn(a.hi, b);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  const float lo = __fadd_rn(a.lo, err);
  const float hi = __fadd_rn(s, lo);
  return {hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}
__device__ __forceinline__ FF ff_sub(FF a, FF b) {
  FF r = ff_add(a, -b.hi);
  return ff_add(r, -b.lo);
}
// a (c.hi + c.lo) for a float-float a and a float-float constant c (TwoProd by fma)
__device__ __forceinline__ FF ff_mul(FF a, float chi, float clo) {
  const float p = __fmul_rn(a.hi, chi);
  float e = __fmaf_rn(a.hi, chi, -p);
  e = __fmaf_rn(a.hi, clo, e);
  e = __fmaf_rn(a.lo, chi, e);
  const float hi = __fadd_rn(p, e);
  return {hi, __fsub_rn(e, __fsub_rn(hi, p))};
}

// Update of the float64 defect after a float32 V-cycle, fused with the correction:
// X += e and R -= A e, with e the level-0 correction and A = lambda - lap_h.  Since A is
// linear, R stays B - A X; A e is formed in float-float from the float values of e (error
// ~2^-44 of its largest term, far below the stopping tolerance), so the only float64
// operations per cell are the two updates and one widening add.  R replaces the float64
// re-evaluation of the stencil of X, which kept GB300's float64 pipe busy.  e is not zeroed
// here (its neighbours are still being read): in 2D the next cycle's first pre-sweep starts
// from zero without reading it, in 3D zero0_kernel follows.
constexpr int kUpdCells = 4;  // cells per thread of update64_kernel: chunks of kUpdCells * kChunk cells

// the defect update of one cell from its correction e and the float-float sum of its cnt
// neighbours' corrections; returns |r| as bits
__device__ __forceinline__ unsigned long long upd_cell(const InstDev& I, double* X, double* R, float& bout, unsigned t,
                                                       float e, FF sum, int cnt) {
  const float ce = __fmul_rn((float)cnt, e);  // cnt e exactly as ce + ce_err
  const float ce_err = __fmaf_rn((float)cnt, e, -ce);
  sum = ff_add(sum, -ce);
  sum = ff_add(sum, -ce_err);
  const FF lap = ff_mul(sum, I.ih2f[0], I.ih2lo0);
  const FF le = ff_mul(FF{e, 0.f}, I.lamf, I.lamlo);
  const FF ae = ff_sub(le, lap);
  X[t] = __dadd_rn(X[t], widen(e));
  const double r = __dsub_rn(R[t], __dadd_rn(widen(ae.hi), widen(ae.lo)));
  R[t] = r;
  bout = narrow<float>(r);
  return (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffull;
}

template <bool NEU, int ND>
__global__ void __launch_bounds__(kChunk) update64_kernel(MgState S, Lvl<float> L, const Chunk* ch) {
  const Chunk C = ch[blockIdx.x];
  if (!S.active[C.inst]) return;
  const InstDev& I = S.inst[C.inst];
  const int n = I.n[0];
  const unsigned un = (unsigned)n, plane = un * un;
  const float* E = L.x + I.off[0];
  float* Bf = L.b + I.off[0];
  double* X = S.X + I.off0;
  double* R = S.R + I.off0;
  unsigned long long m = 0ull;
  if (ND == 2 && (n & 3) == 0) {
    // four consecutive cells of one row per thread (a side divisible by 4; level offsets are
    // multiples of 4 cells): the row's corrections and those of the rows below and above as
    // one float4 each, plus the cells left and right of the four
    const int j4 = 4 * (int)threadIdx.x;
    if (j4 < C.count) {
      const unsigned t0 = (unsigned)C.start + (unsigned)j4;
      const unsigned r = t0 / un, c0 = t0 - r * un;
      const bool hasdn = r > 0u, hasup = r + 1u < un, hasl = c0 > 0u, hasr = c0 + 4u < un;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 e4 = *reinterpret_cast<const float4*>(E + t0);
      const float4 d4 = (NEU && !hasdn) ? z4 : *reinterpret_cast<const float4*>(E + (hasdn ? t0 - un : t0 + (un - 1u) * un));
      const float4 u4 = (NEU && !hasup) ? z4 : *reinterpret_cast<const float4*>(E + (hasup ? t0 + un : t0 - (un - 1u) * un));
      const float lft = (NEU && !hasl) ? 0.f : E[hasl ? t0 - 1u : t0 + un - 1u];
      const float rgt = (NEU && !hasr) ? 0.f : E[hasr ? t0 + 4u : t0 + 4u - un];
      const float ev[6] = {lft, e4.x, e4.y, e4.z, e4.w, rgt};
      const float dv[4] = {d4.x, d4.y, d4.z, d4.w}, uv[4] = {u4.x, u4.y, u4.z, u4.w};
      float bo[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // neighbours in the order x-, x+, y-, y+ (cells beyond a zero-flux boundary left out)
        FF sum{0.f, 0.f};
        int cnt = 0;
        if (!(NEU && q == 0 && !hasl)) sum = ff_add(sum, ev[q]), ++cnt;
        if (!(NEU && q == 3 && !hasr)) sum = ff_add(sum, ev[q + 2]), ++cnt;
        if (!(NEU && !hasdn)) sum = ff_add(sum, dv[q]), ++cnt;
        if (!(NEU && !hasup)) sum = ff_add(sum, uv[q]), ++cnt;
        const unsigned long long rb = upd_cell(I, X, R, bo[q], t0 + q, ev[q + 1], sum, cnt);
        m = rb > m ? rb : m;
      }
      *reinterpret_cast<float4*>(Bf + t0) = make_float4(bo[0], bo[1], bo[2], bo[3]);
    }
  } else {
    // cells start + threadIdx.x + k kChunk: each access of the k loop is coalesced
#pragma unroll
    for (int k = 0; k < kUpdCells; ++k) {
      const int j = threadIdx.x + k * kChunk;
      if (j >= C.count) break;
      const unsigned t = (unsigned)C.start + (unsigned)j;
      const unsigned qr = t / un;
      const unsigned c[3] = {t - qr * un, ND > 2 ? qr % un : qr, ND > 2 ? t / plane : 0u};
      const unsigned stride[3] = {1u, un, plane};
      const float e = E[t];
      // lap e * h^2 = sum of the neighbours (x-, x+, y-, y+, z-, z+) - count e, in float-float
      FF sum{0.f, 0.f};
      int cnt = 0;
#pragma unroll
      for (int d = 0; d < ND; ++d) {
#pragma unroll
        for (int side = -1; side <= 1; side += 2) {
          unsigned q;
          if (side < 0) {
            if (c[d] == 0u) {
              if (NEU) continue;
              q = t + (un - 1u) * stride[d];
            } else {
              q = t - stride[d];
            }
          } else {
            if (c[d] == un - 1u) {
              if (NEU) continue;
              q = t - (un - 1u) * stride[d];
            } else {
              q = t + stride[d];
            }
          }
          sum = ff_add(sum, E[q]);
          ++cnt;
        }
      }
      float bo;
      const unsigned long long rb = upd_cell(I, X, R, bo, t, e, sum, cnt);
      Bf[t] = bo;
      m = rb > m ? rb : m;
    }
  }
  block_max_atomic(m, &S.rnorm[C.inst]);
}

// level-0 correction zeroed for the next V-cycle (after update64_kernel has read it)
__global__ void zero0_kernel(MgState S, Lvl<float> L, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];
  if (!S.active[C.inst] || threadIdx.x >= C.count) return;
  L.x[S.inst[C.inst].off[0] + C.start + threadIdx.x] = 0.f;
}

// per-step log of a device-side solve: entry [step % cap][instance] = V-cycles, or
// -1 - cycles where the instance did not converge; then the step counter advances
__global__ void log_kernel(MgState S, int ninst, int* log, int* step, int cap) {
  const int row = *step % cap;
  for (int i = threadIdx.x; i < ninst; i += blockDim.x)
    log[(size_t)row * ninst + i] = S.failed[i] ? -1 - S.cycles[i] : S.cycles[i];
  __syncthreads();
  if (threadIdx.x == 0) *step = *step + 1;
}

// ------------------------------------------------------ reaction-diffusion --
// Eq. (gray-scott): F0_u = -u v^2 + F(1-u), F0_v = u v^2 - (F+k) v.
// Eq. (schnakenberg): F0_u = kappa (a - u + u^2 v), F0_v = kappa (b - u^2 v).
// IMEX, Eq. (imex): stage 1 B = lambda g, g = w + dt F0(w) + dt/2 D lap w, X = w (guess),
//   Fn = F0(w) + D lap w kept for stage 2; after the solve w += dt/2 [Fn + F(w*)].
// Split, Eqs. (splitting), (diff-helmholtz): B = lambda w*, X = w* = w + dt F0(w); after
//   the solve w = X.
// Explicit: three-stage SSP Runge-Kutta on F = F0 + D lap w, one kernel per stage.
struct RdArgs {
  const InstDev* inst;  // multigrid instances: species s of instance i is s*ninst + i
  int ninst, ndim, model, neu;
  double F, k, kappa, a, b, dt, D[2], lam[2];
  double* u;
  double* v;            // state, packed like level 0 of one species
  double* X;            // multigrid iterate (2 species); explicit: stage 1 state
  double* B;            // multigrid right-hand side; explicit: stage 2 state
  double* Fn;           // F(w_n) per species
};

__device__ __forceinline__ void reaction(const RdArgs& A, double u, double v, double* fu, double* fv) {
  if (A.model == RD_SCHNAKENBERG) {
    double uuv = (u * u) * v;
    *fu = A.kappa * ((A.a - u) + uuv);
    *fv = A.kappa * (A.b - uuv);
  } else {
    double uvv = (u * v) * v;
    *fu = -uvv + A.F * (1.0 - u);
    *fv = uvv - (A.F + A.k) * v;
  }
}

// (sum of in-domain neighbours - count x) / h^2 on level 0
__device__ __forceinline__ double rd_lap(const RdArgs& A, const double* x, const int* c, int n, long long t,
                                         double ih2) {
  int miss;
  double s = A.neu ? nbsum<true>(x, c, n, A.ndim, &miss) : nbsum<false>(x, c, n, A.ndim, &miss);
  return (s - (double)(2 * A.ndim - miss) * x[t]) * ih2;
}

template <int SCHEME>
__global__ void rd_rhs_kernel(RdArgs A, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];  // chunks over level 0 of species-0 instances
  if (threadIdx.x >= C.count) return;
  const InstDev& I0 = A.inst[C.inst];
  const InstDev& I1 = A.inst[C.inst + A.ninst];
  long long t = C.start + threadIdx.x;
  int n = I0.n[0], c[3];
  cell_of(t, n, A.ndim, c);
  long long o = I0.off0;  // species-0 offset equals the state offset
  const double* u = A.u + o;
  const double* v = A.v + o;
  double fu, fv;
  reaction(A, u[t], v[t], &fu, &fv);
  if constexpr (SCHEME == RD_SPLIT) {
    double us = u[t] + A.dt * fu, vs = v[t] + A.dt * fv;
    A.B[I0.off0 + t] = A.lam[0] * us;
    A.B[I1.off0 + t] = A.lam[1] * vs;
    A.X[I0.off0 + t] = us;
    A.X[I1.off0 + t] = vs;
  } else {
    double lu = rd_lap(A, u, c, n, t, I0.ih2[0]);
    double lv = rd_lap(A, v, c, n, t, I0.ih2[0]);
    double gu = (u[t] + A.dt * fu) + ((0.5 * A.dt) * A.D[0]) * lu;
    double gv = (v[t] + A.dt * fv) + ((0.5 * A.dt) * A.D[1]) * lv;
    A.B[I0.off0 + t] = A.lam[0] * gu;
    A.B[I1.off0 + t] = A.lam[1] * gv;
    A.X[I0.off0 + t] = u[t];
    A.X[I1.off0 + t] = v[t];
    A.Fn[I0.off0 + t] = fu + A.D[0] * lu;
    A.Fn[I1.off0 + t] = fv + A.D[1] * lv;
  }
}

// after the solve: IMEX w_{n+1} = w_n + dt/2 [F(w_n) + F(w*)]; split w_{n+1} = X
template <int SCHEME>
__global__ void rd_finish_kernel(RdArgs A, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];
  if (threadIdx.x >= C.count) return;
  const InstDev& I0 = A.inst[C.inst];
  const InstDev& I1 = A.inst[C.inst + A.ninst];
  long long t = C.start + threadIdx.x;
  long long o = I0.off0;
  const double* us = A.X + I0.off0;
  const double* vs = A.X + I1.off0;
  if constexpr (SCHEME == RD_SPLIT) {
    A.u[o + t] = us[t];
    A.v[o + t] = vs[t];
  } else {
    int n = I0.n[0], c[3];
    cell_of(t, n, A.ndim, c);
    double fu, fv;
    reaction(A, us[t], vs[t], &fu, &fv);
    double lu = rd_lap(A, us, c, n, t, I0.ih2[0]);
    double lv = rd_lap(A, vs, c, n, t, I0.ih2[0]);
    double Fu = fu + A.D[0] * lu, Fv = fv + A.D[1] * lv;
    A.u[o + t] = A.u[o + t] + (0.5 * A.dt) * (A.Fn[I0.off0 + t] + Fu);
    A.v[o + t] = A.v[o + t] + (0.5 * A.dt) * (A.Fn[I1.off0 + t] + Fv);
  }
}

// Explicit step, stage S of the three-stage SSP Runge-Kutta scheme (w = state u, v):
//   S = 0: X = w + dt F(w);  S = 1: B = 3/4 w + 1/4 (X + dt F(X));
//   S = 2: w = 1/3 w + 2/3 (B + dt F(B)).
// Stage 2 overwrites w in place: each cell reads only its own w and neighbours of B.
template <int S>
__global__ void rd_explicit_kernel(RdArgs A, const Chunk* ch) {
  Chunk C = ch[blockIdx.x];
  if (threadIdx.x >= C.count) return;
  const InstDev& I0 = A.inst[C.inst];
  const InstDev& I1 = A.inst[C.inst + A.ninst];
  long long t = C.start + threadIdx.x;
  int n = I0.n[0], c[3];
  cell_of(t, n, A.ndim, c);
  const long long o = I0.off0;
  const double* su = S == 0 ? A.u + o : (S == 1 ? A.X + I0.off0 : A.B + I0.off0);
  const double* sv = S == 0 ? A.v + o : (S == 1 ? A.X + I1.off0 : A.B + I1.off0);
  double fu, fv;
  reaction(A, su[t], sv[t], &fu, &fv);
  const double Fu = fu + A.D[0] * rd_lap(A, su, c, n, t, I0.ih2[0]);
  const double Fv = fv + A.D[1] * rd_lap(A, sv, c, n, t, I0.ih2[0]);
  const double eu = su[t] + A.dt * Fu, ev = sv[t] + A.dt * Fv;
  if constexpr (S == 0) {
    A.X[I0.off0 + t] = eu;
    A.X[I1.off0 + t] = ev;
  } else if constexpr (S == 1) {
    A.B[I0.off0 + t] = 0.75 * A.u[o + t] + 0.25 * eu;
    A.B[I1.off0 + t] = 0.75 * A.v[o + t] + 0.25 * ev;
  } else {
    A.u[o + t] = (1.0 / 3.0) * A.u[o + t] + (2.0 / 3.0) * eu;
    A.v[o + t] = (1.0 / 3.0) * A.v[o + t] + (2.0 / 3.0) * ev;
  }
}

// ------------------------------------------------------- learned guess --
// Residual of the previous-step guess at cell p of one instance-species, B - A w_n with
// A = lambda - lap_h (Eq. (diff-helmholtz)), normalised by the operator's diagonal scale
// 2 ndim / h^2 and by the target scale: with target t = (w* - w_n) / scale the network
// then learns t = A_hat^-1 rho_hat, A_hat = A h^2 / (2 ndim).  Periodic wrap, or zero
// flux (neighbours outside the domain dropped from the sum and from the diagonal).
__device__ __forceinline__ double rd_guess_residual(const InstDev& I, const double* __restrict__ B,
                                                    const double* __restrict__ w, long long p, int ndim, int neu,
                                                    double inv_scale) {
  const int n = I.n[0];
  int c[3] = {(int)(p % n), ndim > 1 ? (int)((p / n) % n) : 0, ndim > 2 ? (int)(p / ((long long)n * n)) : 0};
  long long stride = 1;
  double nb = 0.0;
  int cnt = 0;
  for (int d = 0; d < ndim; ++d) {
    if (c[d] > 0) {
      nb += w[p - stride];
      ++cnt;
    } else if (!neu) {
      nb += w[p + (long long)(n - 1) * stride];
      ++cnt;
    }
    if (c[d] < n - 1) {
      nb += w[p + stride];
      ++cnt;
    } else if (!neu) {
      nb += w[p - (long long)(n - 1) * stride];
      ++cnt;
    }
    stride *= n;
  }
  const double ih2 = I.ih2[0];
  double Aw = I.lam * w[p] - (nb - cnt * w[p]) * ih2;
  return (B[I.off0 + p] - Aw) * inv_scale / (2.0 * ndim * ih2);
}

// The same residual as the network's input, in float32 from float32 copies of w_n and B made
// by bit narrowing (no float64 unit work: GB300's float64 rate is ~1/64 of float32).  B and
// lambda w_n nearly cancel: with the narrowing's 2^-23 relative error the result keeps about
// max|B| 2^-22 absolute accuracy, far below the bf16 resolution of the network's input (2^-9
// of the residual's own size) wherever the residual is above 1e-4 of max|B|.
__device__ __forceinline__ float rd_guess_residual_f(const InstDev& I, const double* __restrict__ B,
                                                     const double* __restrict__ w, long long p, int ndim, int neu,
                                                     float inv_scale) {
  const int n = I.n[0];
  int c[3] = {(int)(p % n), ndim > 1 ? (int)((p / n) % n) : 0, ndim > 2 ? (int)(p / ((long long)n * n)) : 0};
  long long stride = 1;
  float nb = 0.f;
  int cnt = 0;
  for (int d = 0; d < ndim; ++d) {
    if (c[d] > 0) {
      nb += narrow<float>(w[p - stride]);
      ++cnt;
    } else if (!neu) {
      nb += narrow<float>(w[p + (long long)(n - 1) * stride]);
      ++cnt;
    }
    if (c[d] < n - 1) {
      nb += narrow<float>(w[p + stride]);
      ++cnt;
    } else if (!neu) {
      nb += narrow<float>(w[p - (long long)(n - 1) * stride]);
      ++cnt;
    }
    stride *= n;
  }
  const float ih2 = I.ih2f[0], wp = narrow<float>(w[p]);
  const float Aw = I.lamf * wp - (nb - (float)cnt * wp) * ih2;
  return (narrow<float>(B[I.off0 + p]) - Aw) * (inv_scale / (2.f * (float)ndim * ih2));
}

// network input of one instance as float [5][cells]: (u_n, v_n, c2, c3, dt) with
// (c2, c3) = (u*_prev, v*_prev) (RD_GUESS_IN_PREV) or the normalised residuals of the
// previous-step guess (RD_GUESS_IN_RESIDUAL); float64 values narrowed on the integer units
__global__ void rd_cnn_input_kernel(const InstDev* __restrict__ inst, int iu, int iv, const double* __restrict__ B,
                                    const double* __restrict__ wn, const double* __restrict__ pin, long long cells,
                                    long long n0, float dt, int kind, int ndim, int neu, double inv_scale,
                                    float* __restrict__ cin) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n0) return;
  const InstDev& Iu = inst[iu];
  const long long off = Iu.off0;
  cin[0 * n0 + t] = narrow<float>(wn[off + t]);
  cin[1 * n0 + t] = narrow<float>(wn[cells + off + t]);
  if (kind == RD_GUESS_IN_RESIDUAL) {
    cin[2 * n0 + t] = rd_guess_residual_f(Iu, B, wn + off, t, ndim, neu, (float)inv_scale);
    cin[3 * n0 + t] = rd_guess_residual_f(inst[iv], B, wn + cells + off, t, ndim, neu, (float)inv_scale);
  } else {
    cin[2 * n0 + t] = narrow<float>(pin[off + t]);
    cin[3 * n0 + t] = narrow<float>(pin[cells + off + t]);
  }
  cin[4 * n0 + t] = dt;
}

// multigrid guess X = w_n + scale * network output (per species): the network
// predicts the increment over the previous-step guess (formed in float32, widened exactly)
__global__ void rd_cnn_guess_kernel(const InstDev* __restrict__ inst, int iu, int iv, const float* __restrict__ cout,
                                    long long n0, double scale, double* __restrict__ X, const double* __restrict__ wn,
                                    long long cells) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n0) return;
  const InstDev& Iu = inst[iu];
  const InstDev& Iv = inst[iv];
  const float sf = (float)scale;
  X[Iu.off0 + t] = __dadd_rn(wn[Iu.off0 + t], widen(sf * cout[t]));
  X[Iv.off0 + t] = __dadd_rn(wn[cells + Iu.off0 + t], widen(sf * cout[n0 + t]));
}

// training pairs: crops of the network input (as rd_cnn_input_kernel) and target (w* - w_n) / scale
struct CropArgs {
  const InstDev* inst;
  const int* cinst;
  const int* corner;  // [ncrops][3]
  int ninst, ndim, crop, ncrops;
  long long cells;
  const double* wn;
  const double* pin;
  const double* X;
  const double* B;
  float dt;
  double inv_scale;
  int kind, neu;
  float* in;
  float* tgt;
};

__global__ void rd_crop_kernel(CropArgs A) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long cp = 1;
  for (int d = 0; d < A.ndim; ++d) cp *= A.crop;
  if (t >= cp * A.ncrops) return;
  int k = (int)(t / cp);
  long long q = t % cp;
  int i = A.cinst[k];
  const InstDev& Iu = A.inst[i];
  const InstDev& Iv = A.inst[i + A.ninst];
  int n = Iu.n[0];
  int c[3] = {(int)(q % A.crop), A.ndim > 1 ? (int)((q / A.crop) % A.crop) : 0,
              A.ndim > 2 ? (int)(q / ((long long)A.crop * A.crop)) : 0};
  int g[3] = {0, 0, 0};
  for (int d = 0; d < A.ndim; ++d) g[d] = (A.corner[3 * k + d] + c[d]) % n;
  long long p = (long long)g[0] + (long long)n * ((long long)g[1] + (long long)n * g[2]);
  long long off = Iu.off0;  // species-0 offset = state offset
  float* in = A.in + (long long)k * 5 * cp;
  in[0 * cp + q] = (float)A.wn[off + p];
  in[1 * cp + q] = (float)A.wn[A.cells + off + p];
  if (A.kind == RD_GUESS_IN_RESIDUAL) {
    in[2 * cp + q] = (float)rd_guess_residual(Iu, A.B, A.wn + off, p, A.ndim, A.neu, A.inv_scale);
    in[3 * cp + q] = (float)rd_guess_residual(Iv, A.B, A.wn + A.cells + off, p, A.ndim, A.neu, A.inv_scale);
  } else {
    in[2 * cp + q] = (float)A.pin[off + p];
    in[3 * cp + q] = (float)A.pin[A.cells + off + p];
  }
  in[4 * cp + q] = A.dt;
  float* tg = A.tgt + (long long)k * 2 * cp;
  tg[q] = (float)((A.X[Iu.off0 + p] - A.wn[off + p]) * A.inv_scale);
  tg[cp + q] = (float)((A.X[Iv.off0 + p] - A.wn[A.cells + off + p]) * A.inv_scale);
}

// ------------------------------------------------------------------ host --
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// Dense inverse of the operator (lambda - lap_h), periodic or Neumann (a neighbour beyond
// the boundary is left out of the row and of its diagonal count), by Gauss-Jordan with
// partial pivoting (host, float64).
bool dense_inverse(int nd, int n, double L, double lambda, bool neu, std::vector<double>& inv) {
  int m = 1;
  for (int d = 0; d < nd; ++d) m *= n;
  double h = L / n, ih2 = 1.0 / (h * h);
  std::vector<double> A((size_t)m * m, 0.0);
  inv.assign((size_t)m * m, 0.0);
  for (int r = 0; r < m; ++r) {
    int c[3] = {r % n, nd > 1 ? (r / n) % n : 0, nd > 2 ? r / (n * n) : 0};
    int count = 0;
    for (int d = 0; d < nd; ++d)
      for (int s = -1; s <= 1; s += 2) {
        int q[3] = {c[0], c[1], c[2]};
        if (neu && (q[d] + s < 0 || q[d] + s >= n)) continue;
        q[d] = (q[d] + s + n) % n;
        int cidx = q[0] + n * (q[1] + n * q[2]);
        A[(size_t)r * m + cidx] -= ih2;
        ++count;
      }
    A[(size_t)r * m + r] += lambda + count * ih2;
    inv[(size_t)r * m + r] = 1.0;
  }
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int r = col + 1; r < m; ++r)
      if (std::fabs(A[(size_t)r * m + col]) > std::fabs(A[(size_t)piv * m + col])) piv = r;
    if (A[(size_t)piv * m + col] == 0.0) return false;
    if (piv != col)
      for (int k = 0; k < m; ++k) {
        std::swap(A[(size_t)piv * m + k], A[(size_t)col * m + k]);
        std::swap(inv[(size_t)piv * m + k], inv[(size_t)col * m + k]);
      }
    double d = 1.0 / A[(size_t)col * m + col];
    for (int k = 0; k < m; ++k) {
      A[(size_t)col * m + k] *= d;
      inv[(size_t)col * m + k] *= d;
    }
    for (int r = 0; r < m; ++r) {
      if (r == col) continue;
      double f = A[(size_t)r * m + col];
      if (f == 0.0) continue;
      for (int k = 0; k < m; ++k) {
        A[(size_t)r * m + k] -= f * A[(size_t)col * m + k];
        inv[(size_t)r * m + k] -= f * inv[(size_t)col * m + k];
      }
    }
  }
  return true;
}

void add_chunks(std::vector<Chunk>& v, int inst, int lev, long long count) {
  for (long long s = 0; s < count; s += kChunk) v.push_back(Chunk{inst, lev, s, (int)std::min<long long>(kChunk, count - s)});
}

// kernel kinds of one V-cycle (mg_profile_vcycle)
enum MgKind {
  kMgSweep = 0,        // 2D red-black sweep (one tiled pass per sweep)
  kMgCopy = 1,         // 2D copy after an odd number of sweeps
  kMgSmooth = 2,       // 3D red-black half sweep (one colour)
  kMgResRestrict = 3,  // residual and restriction to the next depth
  kMgCoarse = 4,       // coarsest-level direct solve
  kMgProlong = 5,      // prolongation of the correction
  kMgUpdate = 6,       // float32 cycles: X += e, R -= A e (float-float)
  kMgZero = 7,         // float32 cycles: zero the level-0 correction
  kMgCorrect = 8,      // float64 cycles: X += e
  kMgResidual = 9,     // float64 cycles: new level-0 defect
  kMgCoarseCycle = 10  // 2D: the coarse depths of the cycle in shared memory
};

struct Mg {
  int nd = 2, ninst = 0, nu1 = 2, nu2 = 2, max_cycles = 50, precision = AMR_FP32;
  bool neu = false;  // Neumann (zero-flux) boundaries, else periodic
  double rtol = 1e-10, Lside = 1.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<InstDev> insts;
  int maxdepth = 0;
  long long n0 = 0, nlevtot = 0;
  // chunk lists: level 0 cells; per depth: colour cells, coarse cells, fine cells
  std::vector<Chunk> ch0;
  std::vector<Chunk> ch0q;  // level 0 in chunks of kUpdCells * kChunk cells (update64_kernel)
  std::vector<std::vector<Chunk>> ch_half, ch_coarse, ch_fine, ch_tile;
  std::vector<int> coarse_inst, coarse_row0;
  DevBuf d_yl;  // 2D: second iterate array for the tiled sweeps
  DevBuf d_R;  // float32 V-cycles: level-0 float64 defect
  DevBuf d_inst, d_X, d_B, d_xl, d_bl, d_rnorm, d_bnorm, d_lastres, d_initres, d_active, d_cycles, d_failed, d_any, d_inv, d_invf;
  DevBuf d_iters;
  cudaStream_t cstream = nullptr;   // captures the body of the device-side solve loop
  cudaGraphExec_t sgraph = nullptr; // one whole solve (device-side convergence loop)
  long long solve_loop_kernels = 0; // kernels per iteration of that loop
  DevBuf d_ch0, d_ch0q, d_chall, d_cinst, d_crow0, d_sinst;
  std::vector<int> smem_inst;  // 2D instances whose coarse depths run in shared memory
  size_t smem_bytes = 0;       // the largest such instance's levels
  // per-depth kernels run on depths 0 .. per_depth_end - 1 of an instance
  static int per_depth_end(const InstDev& I) { return I.dsm >= 0 ? I.dsm : I.nlev - 1; }
  std::vector<size_t> off_half, off_coarse, off_fine, off_tile;
  int* h_any = nullptr;
  cudaGraphExec_t vgraph = nullptr;
  long long launches = 0;
  bool solved = false;  // a solve has run: the level-0 defect and the level arrays are set
  // measurement: while prof_ev is set, every kernel enqueue_vcycle launches is followed by an
  // event on the stream (prof_ev[0] is recorded before the first), and its kind is kept
  std::vector<cudaEvent_t>* prof_ev = nullptr;
  std::vector<int>* prof_kind = nullptr;
  void mark(int kind) {
    ++launches;
    if (!prof_ev) return;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) == cudaSuccess) {
      cudaEventRecord(e, stream);
      prof_ev->push_back(e);
      prof_kind->push_back(kind);
    }
  }
  int vcycle_kernels = 0;

  ~Mg() {
    if (vgraph) cudaGraphExecDestroy(vgraph);
    if (sgraph) cudaGraphExecDestroy(sgraph);
    if (cstream) cudaStreamDestroy(cstream);
    if (h_any) cudaFreeHost(h_any);
    if (own_stream) cudaStreamDestroy(stream);
  }
  int fail(int code, const std::string& m) {
    err = m;
    return code;
  }
  int cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return AMR_OK;
    err = std::string("CUDA error ") + cudaGetErrorString(e) + " in " + what;
    return e == cudaErrorMemoryAllocation ? AMR_ERR_OOM : AMR_ERR_CUDA;
  }

  MgState state() const {
    MgState S{};
    S.inst = d_inst.as<InstDev>();
    S.X = d_X.as<double>();
    S.B = d_B.as<double>();
    S.R = d_R.as<double>();
    S.rnorm = d_rnorm.as<unsigned long long>();
    S.bnorm = d_bnorm.as<double>();
    S.lastres = d_lastres.as<double>();
    S.initres = d_initres.as<double>();
    S.active = d_active.as<int>();
    S.cycles = d_cycles.as<int>();
    S.failed = d_failed.as<int>();
    S.any = d_any.as<int>();
    S.iters = d_iters.as<int>();
    S.inv = d_inv.as<double>();
    S.invf = d_invf.as<float>();
    S.ndim = nd;
    S.neu = neu ? 1 : 0;
    S.rtol = rtol;
    S.max_cycles = max_cycles;
    return S;
  }

  int setup(int ndim, int n_inst, const int* n_cells, const double* lambda, double L, int nu1_, int nu2_, int maxc,
            double rtol_, int coarse_max, int prec, int bc, void* strm) {
    if (ndim < 2 || ndim > 3 || n_inst < 1 || !n_cells || !lambda || !(L > 0) || nu1_ < 0 || nu2_ < 0 ||
        maxc < 0 || !(rtol_ > 0) || coarse_max < 1 || (prec != AMR_FP32 && prec != AMR_FP64) ||
        (bc != MG_BC_PERIODIC && bc != MG_BC_NEUMANN))
      return fail(AMR_ERR_INVALID_ARG, "invalid multigrid configuration");
    nd = ndim;
    neu = bc == MG_BC_NEUMANN;
    ninst = n_inst;
    nu1 = nu1_;
    nu2 = nu2_;
    max_cycles = maxc;
    rtol = rtol_;
    Lside = L;
    precision = prec;
    stream = (cudaStream_t)strm;
    if (!stream) {
      if (int rc = cuda(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking), "stream")) return rc;
      own_stream = true;
    }
    insts.resize(n_inst);
    long long off = 0, off0 = 0, invoff = 0;
    std::vector<std::vector<double>> invs(n_inst);
    for (int i = 0; i < n_inst; ++i) {
      int n = n_cells[i];
      if (n < 1 || !(lambda[i] > 0)) return fail(AMR_ERR_INVALID_ARG, "instance size or lambda");
      if (std::pow((double)n, ndim) >= 2147483648.0) return fail(AMR_ERR_INVALID_ARG, "instance above 2^31 cells");
      InstDev& I = insts[i];
      std::memset(&I, 0, sizeof(I));
      I.lam = lambda[i];
      I.lamf = (float)lambda[i];
      I.lamlo = (float)(lambda[i] - (double)I.lamf);
      I.off0 = off0;
      long long cells0 = 1;
      for (int d = 0; d < nd; ++d) cells0 *= n;
      off0 += cells0;
      int l = 0, m = n;
      while (true) {
        if (l >= kMaxLev) return fail(AMR_ERR_INVALID_ARG, "too many levels");
        I.n[l] = m;
        I.off[l] = off;
        long long cells = 1;
        for (int d = 0; d < nd; ++d) cells *= m;
        off += (cells + 3) & ~3LL;  // every level starts at a multiple of 4 cells (aligned pairs)
        double h = L / m;
        I.ih2[l] = 1.0 / (h * h);
        I.ih2f[l] = (float)I.ih2[l];
        for (int mm = 0; mm < 7; ++mm) {
          const int count = std::max(0, 2 * nd - mm);
          I.idiag[l][mm] = 1.0 / (lambda[i] + count * I.ih2[l]);
          I.idiagf[l][mm] = (float)I.idiag[l][mm];
        }
        ++l;
        if ((m & 1) || m <= coarse_max) break;
        m /= 2;
      }
      I.nlev = l;
      I.ih2lo0 = (float)(I.ih2[0] - (double)I.ih2f[0]);
      // 2D: the depths from the first one (below 0) whose side fits the shared-memory coarse
      // cycle run in one CTA; instances with a single level keep the per-depth kernels
      I.dsm = -1;
      if (nd == 2 && l >= 2)
        for (int d = 1; d < l; ++d)
          if (I.n[d] <= (prec == AMR_FP64 ? kCoarseSideF64 : kCoarseSideF32)) {
            I.dsm = d;
            break;
          }
      maxdepth = std::max(maxdepth, l);
      int mc = I.n[l - 1];
      long long msz = 1;
      for (int d = 0; d < nd; ++d) msz *= mc;
      if (msz > 4096) return fail(AMR_ERR_INVALID_ARG, "coarsest grid too large (increase coarse_max or use sizes with more factors of 2)");
      if (!dense_inverse(nd, mc, L, lambda[i], neu, invs[i])) return fail(AMR_ERR_INVALID_ARG, "singular coarse operator");
      I.inv_off = invoff;
      invoff += msz * msz;
    }
    n0 = off0;
    nlevtot = off;
    // chunk lists
    ch0.clear();
    ch0q.clear();
    for (int i = 0; i < n_inst; ++i) {
      long long c = 1;
      for (int d = 0; d < nd; ++d) c *= insts[i].n[0];
      add_chunks(ch0, i, 0, c);
      for (long long s0 = 0; s0 < c; s0 += kUpdCells * kChunk)
        ch0q.push_back(Chunk{i, 0, s0, (int)std::min<long long>(kUpdCells * kChunk, c - s0)});
    }
    ch_half.assign(maxdepth, {});
    ch_coarse.assign(maxdepth, {});
    ch_fine.assign(maxdepth, {});
    ch_tile.assign(maxdepth, {});
    coarse_inst.clear();
    coarse_row0.clear();
    smem_inst.clear();
    smem_bytes = 0;
    for (int i = 0; i < n_inst; ++i) {
      const InstDev& I = insts[i];
      for (int l = 0; l < per_depth_end(I); ++l) {
        long long cf = 1, cc = 1;
        for (int d = 0; d < nd; ++d) {
          cf *= I.n[l];
          cc *= I.n[l + 1];
        }
        add_chunks(ch_half[l], i, l, cf / 2);
        add_chunks(ch_coarse[l], i, l, cc);
        add_chunks(ch_fine[l], i, l, cf);
      }
      if (I.dsm >= 0) {
        smem_inst.push_back(i);
        size_t cells = 0;
        for (int l = I.dsm; l < I.nlev; ++l) cells += 2 * ((I.n[l] * I.n[l] + 3) & ~3);
        smem_bytes = std::max(smem_bytes, cells * (precision == AMR_FP64 ? 8 : 4));
        continue;
      }
      long long m = 1;
      for (int d = 0; d < nd; ++d) m *= I.n[I.nlev - 1];
      for (long long r = 0; r < m; r += 64) {
        coarse_inst.push_back(i);
        coarse_row0.push_back((int)r);
      }
    }
    // device buffers
    size_t wb = precision == AMR_FP64 ? 8 : 4;
    int rc;
    if ((rc = cuda(d_inst.alloc(insts.size() * sizeof(InstDev)), "alloc")) ||
        (rc = cuda(d_X.alloc(n0 * 8), "alloc X")) || (rc = cuda(d_B.alloc(n0 * 8), "alloc B")) ||
        (precision != AMR_FP64 && (rc = cuda(d_R.alloc(n0 * 8), "alloc R"))) ||
        (rc = cuda(d_xl.alloc(nlevtot * wb), "alloc levels")) || (rc = cuda(d_bl.alloc(nlevtot * wb), "alloc levels")) ||
        (nd == 2 && (rc = cuda(d_yl.alloc(nlevtot * wb), "alloc levels"))) ||
        (rc = cuda(d_rnorm.alloc(n_inst * 8), "alloc")) || (rc = cuda(d_bnorm.alloc(n_inst * 8), "alloc")) ||
        (rc = cuda(d_lastres.alloc(n_inst * 8), "alloc")) || (rc = cuda(d_initres.alloc(n_inst * 8), "alloc")) ||
        (rc = cuda(d_active.alloc(n_inst * 4), "alloc")) ||
        (rc = cuda(d_cycles.alloc(n_inst * 4), "alloc")) || (rc = cuda(d_failed.alloc(n_inst * 4), "alloc")) ||
        (rc = cuda(d_any.alloc(4), "alloc")) || (rc = cuda(d_iters.alloc(4), "alloc")) ||
        (rc = cuda(d_inv.alloc(invoff * 8), "alloc inverse")) ||
        (rc = cuda(d_invf.alloc(invoff * 4), "alloc inverse")))
      return rc;
    if ((rc = cuda(cudaMallocHost(&h_any, 4), "host alloc"))) return rc;
    // host-to-device copy of a table (empty tables copy nothing)
    auto upload = [&](void* dst, const void* src, size_t bytes) {
      return bytes ? cuda(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice), "copy table") : AMR_OK;
    };
    if ((rc = upload(d_inst.p, insts.data(), insts.size() * sizeof(InstDev)))) return rc;
    {
      std::vector<float> f;
      for (int i = 0; i < n_inst; ++i) {
        if ((rc = upload(d_inv.as<double>() + insts[i].inv_off, invs[i].data(), invs[i].size() * 8))) return rc;
        f.assign(invs[i].begin(), invs[i].end());
        if ((rc = upload(d_invf.as<float>() + insts[i].inv_off, f.data(), f.size() * 4))) return rc;
      }
    }
    if ((rc = cuda(cudaMemset(d_rnorm.p, 0, n_inst * 8), "memset"))) return rc;
    if (nd == 2) {  // strip heights: measured per level side, then the tile lists
      if ((rc = precision == AMR_FP64 ? tune_strips<double>() : tune_strips<float>())) return rc;
      for (int i = 0; i < n_inst; ++i) {
        const InstDev& I = insts[i];
        for (int l = 0; l < per_depth_end(I); ++l) {
          const int H = height_for(l, I.n[l]);
          for (int k = 0; k < tiles_of(I.n[l], H); ++k) ch_tile[l].push_back(Chunk{i, l, k, H});
        }
      }
    }
    std::vector<Chunk> all;
    off_half.assign(maxdepth, 0);
    off_coarse.assign(maxdepth, 0);
    off_fine.assign(maxdepth, 0);
    off_tile.assign(maxdepth, 0);
    for (int l = 0; l < maxdepth; ++l) {
      off_tile[l] = all.size();
      all.insert(all.end(), ch_tile[l].begin(), ch_tile[l].end());
      off_half[l] = all.size();
      all.insert(all.end(), ch_half[l].begin(), ch_half[l].end());
      off_coarse[l] = all.size();
      all.insert(all.end(), ch_coarse[l].begin(), ch_coarse[l].end());
      off_fine[l] = all.size();
      all.insert(all.end(), ch_fine[l].begin(), ch_fine[l].end());
    }
    if ((rc = cuda(d_ch0.alloc(ch0.size() * sizeof(Chunk)), "alloc")) ||
        (rc = cuda(d_ch0q.alloc(ch0q.size() * sizeof(Chunk)), "alloc")) ||
        (rc = cuda(d_chall.alloc(all.size() * sizeof(Chunk)), "alloc")) ||
        (rc = cuda(d_cinst.alloc(coarse_inst.size() * 4), "alloc")) ||
        (rc = cuda(d_crow0.alloc(coarse_row0.size() * 4), "alloc")) ||
        (rc = cuda(d_sinst.alloc(smem_inst.size() * 4), "alloc")))
      return rc;
    if ((rc = upload(d_ch0.p, ch0.data(), ch0.size() * sizeof(Chunk))) ||
        (rc = upload(d_ch0q.p, ch0q.data(), ch0q.size() * sizeof(Chunk))) ||
        (rc = upload(d_chall.p, all.data(), all.size() * sizeof(Chunk))) ||
        (rc = upload(d_cinst.p, coarse_inst.data(), coarse_inst.size() * 4)) ||
        (rc = upload(d_crow0.p, coarse_row0.data(), coarse_row0.size() * 4)) ||
        (rc = upload(d_sinst.p, smem_inst.data(), smem_inst.size() * 4)))
      return rc;
    if (!smem_inst.empty()) {
      const int sb = (int)smem_bytes;
      cudaError_t e = cudaSuccess;
      if (precision == AMR_FP64)
        e = neu ? cudaFuncSetAttribute(coarse2d_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb)
                : cudaFuncSetAttribute(coarse2d_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
      else
        e = neu ? cudaFuncSetAttribute(coarse2d_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb)
                : cudaFuncSetAttribute(coarse2d_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
      if ((rc = cuda(e, "coarse cycle shared memory"))) return rc;
    }
    return cuda(cudaDeviceSynchronize(), "setup");
  }

  template <typename real>
  Lvl<real> lvl() const {
    return Lvl<real>{d_xl.as<real>(), d_bl.as<real>()};
  }

  std::map<int, int> strip_h;  // level side -> strip height of the 2D sweep
  std::vector<int> depth_h;     // per depth: the chosen candidate height, 0 = the side-based default
  static int tiles_of(int n, int H) { return ((n + kStripW - 1) / kStripW) * ((n + H - 1) / H); }
  int height_for(int depth, int n) const { return depth_h[depth] > 0 ? depth_h[depth] : strip_height(n); }

  // Autotuner: for every depth of the batch, time the sweep of all the instances' levels of
  // that depth together, as the V-cycle launches it, with each candidate strip height (one
  // height for the whole depth, or the side-based default clamp(n/32, 8, 64)); 3 launches
  // after a warm-up, CUDA events on the stream.  The kernel reads x and writes the second
  // iterate array, so no data change, and every height gives the same iterate bit for bit:
  // the choice changes time only.  Cached per (sides of the depth, precision, boundary kind).
  template <typename real>
  int tune_strips() {
    std::vector<int> ones(ninst, 1);
    if (int rc = cuda(cudaMemcpy(d_active.p, ones.data(), ninst * sizeof(int), cudaMemcpyHostToDevice), "copy"))
      return rc;
    MgState S = state();
    Lvl<real> Lv = lvl<real>();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DevBuf dch;
    int rc = AMR_OK;
    depth_h.assign(maxdepth, 0);
    for (int l = 0; l + 1 < maxdepth && !rc; ++l) {
      std::vector<int> sides;  // instances swept at this depth
      std::vector<int> who;
      for (int i = 0; i < ninst; ++i)
        if (l < per_depth_end(insts[i])) {
          sides.push_back(insts[i].n[l]);
          who.push_back(i);
        }
      if (who.empty()) continue;
      std::string key = std::to_string(precision) + (neu ? "n" : "p");
      for (int n : sides) key += ":" + std::to_string(n);
      {
        std::lock_guard<std::mutex> g(strip_cache_mutex());
        auto it = strip_cache().find(key);
        if (it != strip_cache().end()) {
          depth_h[l] = it->second;
          continue;
        }
      }
      if (!e0 && ((rc = cuda(cudaEventCreate(&e0), "event")) || (rc = cuda(cudaEventCreate(&e1), "event")))) break;
      int best = 0;
      float tbest = 1e30f;
      for (int c = -1; c < (int)(sizeof(kStripCandidates) / sizeof(int)); ++c) {
        const int H = c < 0 ? 0 : kStripCandidates[c];
        std::vector<Chunk> t;
        for (int i : who) {
          const int n = insts[i].n[l], h = H > 0 ? H : strip_height(n);
          for (int k = 0; k < tiles_of(n, h); ++k) t.push_back(Chunk{i, l, k, h});
        }
        const int nch = (int)t.size();
        if ((rc = cuda(dch.alloc(t.size() * sizeof(Chunk)), "alloc")) ||
            (rc = cuda(cudaMemcpy(dch.p, t.data(), t.size() * sizeof(Chunk), cudaMemcpyHostToDevice), "copy")))
          break;
        const unsigned nb = (unsigned)((nch + 3) / 4);
        auto sweep = [&]() {
          if (neu)
            sweep2d_kernel<real, true><<<nb, 128, 0, stream>>>(S, Lv.x, d_yl.as<real>(), Lv.b, dch.as<Chunk>(), nch);
          else
            sweep2d_kernel<real, false><<<nb, 128, 0, stream>>>(S, Lv.x, d_yl.as<real>(), Lv.b, dch.as<Chunk>(), nch);
        };
        sweep();
        cudaEventRecord(e0, stream);
        for (int r = 0; r < 3; ++r) sweep();
        cudaEventRecord(e1, stream);
        if ((rc = cuda(cudaEventSynchronize(e1), "tuning"))) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < tbest) {
          tbest = ms;
          best = H;
        }
      }
      depth_h[l] = best;
      std::lock_guard<std::mutex> g(strip_cache_mutex());
      strip_cache()[key] = best;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!rc) rc = cuda(cudaGetLastError(), "tuning");
    if (!rc)
      for (int i = 0; i < ninst; ++i)
        for (int l = 0; l < per_depth_end(insts[i]); ++l)
          if (!strip_h.count(insts[i].n[l])) strip_h[insts[i].n[l]] = height_for(l, insts[i].n[l]);
    return rc;
  }

  template <typename real>
  int enqueue_vcycle() {
    MgState S = state();
    Lvl<real> Lv = lvl<real>();
    const Chunk* all = d_chall.as<Chunk>();
    real* Y = d_yl.as<real>();
    auto smooth = [&](int l, int sweeps, bool first) {  // `sweeps` red-black sweeps of depth l
      if (nd == 2) {
        if (ch_tile[l].empty()) return;
        const int nch = (int)ch_tile[l].size();
        const unsigned nb = (unsigned)((nch + 3) / 4);
        const Chunk* tl = all + off_tile[l];
        for (int s = 0; s < sweeps; ++s) {
          bool even = (s & 1) == 0;
          // the first pre-sweep starts from the zero correction (set by the residual, the
          // restriction or, for depth 0 of later cycles, by nobody: it is never read)
          const bool xz = first && s == 0;
          if (neu) {
            if (xz)
              sweep2d_kernel<real, true, true><<<nb, 128, 0, stream>>>(S, Lv.x, Y, Lv.b, tl, nch);
            else
              sweep2d_kernel<real, true><<<nb, 128, 0, stream>>>(S, even ? Lv.x : Y, even ? Y : Lv.x, Lv.b, tl, nch);
          } else {
            if (xz)
              sweep2d_kernel<real, false, true><<<nb, 128, 0, stream>>>(S, Lv.x, Y, Lv.b, tl, nch);
            else
              sweep2d_kernel<real, false><<<nb, 128, 0, stream>>>(S, even ? Lv.x : Y, even ? Y : Lv.x, Lv.b, tl, nch);
          }
          mark(kMgSweep);
        }
        if (sweeps & 1) {
          copy2d_kernel<real><<<nb, 128, 0, stream>>>(S, Y, Lv.x, tl, nch);
          mark(kMgCopy);
        }
        return;
      }
      if (ch_half[l].empty()) return;
      for (int s = 0; s < sweeps; ++s)
        for (int colour = 0; colour < 2; ++colour) {
          if (neu)
            smooth_kernel<real, true><<<(unsigned)ch_half[l].size(), kChunk, 0, stream>>>(S, Lv, all + off_half[l], colour);
          else
            smooth_kernel<real, false><<<(unsigned)ch_half[l].size(), kChunk, 0, stream>>>(S, Lv, all + off_half[l], colour);
          mark(kMgSmooth);
        }
    };
    for (int l = 0; l + 1 < maxdepth; ++l) {
      smooth(l, nu1, true);
      if (!ch_coarse[l].empty()) {
        const unsigned g = (unsigned)ch_coarse[l].size();
        if (nd == 2) {
          if (neu)
            resrestrict2d_kernel<real, true><<<g, kChunk, 0, stream>>>(S, Lv, all + off_coarse[l]);
          else
            resrestrict2d_kernel<real, false><<<g, kChunk, 0, stream>>>(S, Lv, all + off_coarse[l]);
        } else {
          if (neu)
            resrestrict_kernel<real, true><<<g, kChunk, 0, stream>>>(S, Lv, all + off_coarse[l]);
          else
            resrestrict_kernel<real, false><<<g, kChunk, 0, stream>>>(S, Lv, all + off_coarse[l]);
        }
        mark(kMgResRestrict);
      }
    }
    if (!coarse_inst.empty()) {
      coarse_kernel<real><<<(unsigned)coarse_inst.size(), 256, 0, stream>>>(S, Lv, d_cinst.as<int>(),
                                                                            d_crow0.as<int>(), (int)coarse_inst.size());
      mark(kMgCoarse);
    }
    if (!smem_inst.empty()) {
      const unsigned g = (unsigned)smem_inst.size();
      if (neu)
        coarse2d_kernel<real, true><<<g, kCoarseThreads, smem_bytes, stream>>>(S, Lv, d_sinst.as<int>(), nu1, nu2);
      else
        coarse2d_kernel<real, false><<<g, kCoarseThreads, smem_bytes, stream>>>(S, Lv, d_sinst.as<int>(), nu1, nu2);
      mark(kMgCoarseCycle);
    }
    for (int l = maxdepth - 2; l >= 0; --l) {
      if (nd == 2 && !ch_coarse[l].empty()) {
        if (neu)
          prolong2d_kernel<real, true><<<(unsigned)ch_coarse[l].size(), kChunk, 0, stream>>>(S, Lv, all + off_coarse[l]);
        else
          prolong2d_kernel<real, false><<<(unsigned)ch_coarse[l].size(), kChunk, 0, stream>>>(S, Lv, all + off_coarse[l]);
        mark(kMgProlong);
      } else if (nd != 2 && !ch_fine[l].empty()) {
        if (neu)
          prolong_kernel<real, true><<<(unsigned)ch_fine[l].size(), kChunk, 0, stream>>>(S, Lv, all + off_fine[l]);
        else
          prolong_kernel<real, false><<<(unsigned)ch_fine[l].size(), kChunk, 0, stream>>>(S, Lv, all + off_fine[l]);
        mark(kMgProlong);
      }
      smooth(l, nu2, false);
    }
    // the correction and the new level-0 defect: float32 cycles update R by A e; float64
    // cycles correct X and re-evaluate the residual
    if constexpr (sizeof(real) == 4) {
      {
        const unsigned g = (unsigned)ch0q.size();
        const Chunk* cq = d_ch0q.as<Chunk>();
        if (nd == 2) {
          if (neu) update64_kernel<true, 2><<<g, kChunk, 0, stream>>>(S, Lv, cq);
          else update64_kernel<false, 2><<<g, kChunk, 0, stream>>>(S, Lv, cq);
        } else if (nd == 3) {
          if (neu) update64_kernel<true, 3><<<g, kChunk, 0, stream>>>(S, Lv, cq);
          else update64_kernel<false, 3><<<g, kChunk, 0, stream>>>(S, Lv, cq);
        } else {
          if (neu) update64_kernel<true, 1><<<g, kChunk, 0, stream>>>(S, Lv, cq);
          else update64_kernel<false, 1><<<g, kChunk, 0, stream>>>(S, Lv, cq);
        }
      }
      mark(kMgUpdate);
      if (nd != 2 || nu1 == 0) {  // 2D pre-sweeps never read the correction they start from
        zero0_kernel<<<(unsigned)ch0.size(), kChunk, 0, stream>>>(S, Lv, d_ch0.as<Chunk>());
        mark(kMgZero);
      }
    } else {
      correct64_kernel<real><<<(unsigned)ch0.size(), kChunk, 0, stream>>>(S, Lv, d_ch0.as<Chunk>());
      mark(kMgCorrect);
      if (neu)
        residual64_kernel<real, true><<<(unsigned)ch0.size(), kChunk, 0, stream>>>(S, Lv, d_ch0.as<Chunk>());
      else
        residual64_kernel<real, false><<<(unsigned)ch0.size(), kChunk, 0, stream>>>(S, Lv, d_ch0.as<Chunk>());
      mark(kMgResidual);
    }
    return cuda(cudaGetLastError(), "vcycle launch");
  }

  template <typename real>
  int build_graph() {
    if (vgraph) return AMR_OK;
    cudaGraph_t g;
    if (int rc = cuda(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "capture")) return rc;
    long long before = launches;
    int rc = enqueue_vcycle<real>();
    cudaError_t ec = cudaStreamEndCapture(stream, &g);
    if (rc) return rc;
    if ((rc = cuda(ec, "end capture"))) return rc;
    vcycle_kernels = (int)(launches - before);
    launches = before;
    rc = cuda(cudaGraphInstantiate(&vgraph, g, 0), "instantiate");
    cudaGraphDestroy(g);
    return rc;
  }

  // Enqueue one whole solve on `stream` while it is being captured into a graph: the norms,
  // the first residual and check, then a conditional while node whose body (captured on
  // cstream) is one V-cycle, the residual and the check.  The check kernel sets the loop
  // condition, so the convergence loop runs on the device with no host round trip.
  template <typename real>
  int capture_solve() {
    MgState S = state();
    Lvl<real> Lv = lvl<real>();
    if (!cstream) {
      if (int rc = cuda(cudaStreamCreateWithFlags(&cstream, cudaStreamNonBlocking), "stream")) return rc;
    }
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    if (int rc = cuda(cudaStreamGetCaptureInfo(stream, &st, nullptr, &g), "capture info")) return rc;
    if (st != cudaStreamCaptureStatusActive || !g) return fail(AMR_ERR_CUDA, "solve capture outside a capture");
    cudaGraphConditionalHandle hc;
    if (int rc = cuda(cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault), "conditional handle"))
      return rc;
    bnorm_kernel<<<(unsigned)ch0.size(), kChunk, 0, stream>>>(S, d_ch0.as<Chunk>());
    bnorm_finish_kernel<<<(ninst + 255) / 256, 256, 0, stream>>>(S, ninst);
    if (neu)
      residual64_kernel<real, true><<<(unsigned)ch0.size(), kChunk, 0, stream>>>(S, Lv, d_ch0.as<Chunk>());
    else
      residual64_kernel<real, false><<<(unsigned)ch0.size(), kChunk, 0, stream>>>(S, Lv, d_ch0.as<Chunk>());
    check_kernel<<<1, 256, 0, stream>>>(S, ninst, hc, 1);
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if (int rc = cuda(cudaStreamGetCaptureInfo(stream, &st, nullptr, &g, &deps, nullptr, &ndeps), "capture info"))
      return rc;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (int rc = cuda(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp), "conditional node")) return rc;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (int rc = cuda(cudaStreamUpdateCaptureDependencies(stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
                      "capture dependencies"))
      return rc;
    if (int rc = cuda(cudaStreamBeginCaptureToGraph(cstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                      "body capture"))
      return rc;
    cudaStream_t outer = stream;
    stream = cstream;
    long long before = launches;
    int rc = enqueue_vcycle<real>();  // ends with the new defect
    check_kernel<<<1, 256, 0, stream>>>(S, ninst, hc, 1);
    solve_loop_kernels = launches - before + 1;
    launches = before;
    stream = outer;
    cudaGraph_t got = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cstream, &got);
    if (rc) return rc;
    return cuda(ec, "end body capture");
  }

  template <typename real>
  int build_solve_graph() {
    if (sgraph) return AMR_OK;
    cudaGraph_t g;
    if (int rc = cuda(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "capture")) return rc;
    int rc = capture_solve<real>();
    cudaError_t ec = cudaStreamEndCapture(stream, &g);
    if (rc) {
      if (ec == cudaSuccess) cudaGraphDestroy(g);
      return rc;
    }
    if ((rc = cuda(ec, "end capture"))) return rc;
    rc = cuda(cudaGraphInstantiate(&sgraph, g, 0), "instantiate");
    cudaGraphDestroy(g);
    return rc;
  }

  // kernels one device-side solve ran: prelude 4 (norms, first residual, check), then per loop
  // iteration (max cycles of an instance) a V-cycle ending with the new defect, and a check
  long long solve_kernels(int maxcyc) const { return 4 + (long long)maxcyc * solve_loop_kernels; }

  // X (device, float64) holds the guess; B (device) the right-hand side; both at d_X / d_B.
  // One launch of the solve graph; the host does not wait.
  template <typename real>
  int solve_graph_launch() {
    if (int rc = build_solve_graph<real>()) return rc;
    return cuda(cudaGraphLaunch(sgraph, stream), "solve graph launch");
  }
  int solve_graph_launch_any() {
    return precision == AMR_FP64 ? solve_graph_launch<double>() : solve_graph_launch<float>();
  }
  int capture_solve_any() { return precision == AMR_FP64 ? capture_solve<double>() : capture_solve<float>(); }

  // X (device, float64) holds the guess; B (device) the right-hand side; both at d_X / d_B
  // (host-polled loop: used with the learned guess, whose step syncs anyway)
  template <typename real>
  int solve_device() {
    MgState S = state();
    Lvl<real> Lv = lvl<real>();
    int rc = build_graph<real>();
    if (rc) return rc;
    bnorm_kernel<<<(unsigned)ch0.size(), kChunk, 0, stream>>>(S, d_ch0.as<Chunk>());
    bnorm_finish_kernel<<<(ninst + 255) / 256, 256, 0, stream>>>(S, ninst);
    if (neu)
      residual64_kernel<real, true><<<(unsigned)ch0.size(), kChunk, 0, stream>>>(S, Lv, d_ch0.as<Chunk>());
    else
      residual64_kernel<real, false><<<(unsigned)ch0.size(), kChunk, 0, stream>>>(S, Lv, d_ch0.as<Chunk>());
    launches += 3;
    while (true) {
      check_kernel<<<1, 256, 0, stream>>>(S, ninst, 0, 0);
      ++launches;
      if ((rc = cuda(cudaMemcpyAsync(h_any, d_any.p, 4, cudaMemcpyDeviceToHost, stream), "copy"))) return rc;
      if ((rc = cuda(cudaStreamSynchronize(stream), "sync"))) return rc;
      if (!*h_any) break;
      if ((rc = cuda(cudaGraphLaunch(vgraph, stream), "graph launch"))) return rc;  // V-cycle + new defect
      launches += vcycle_kernels;
    }
    return cuda(cudaGetLastError(), "solve");
  }

  int solve_device_any() { return precision == AMR_FP64 ? solve_device<double>() : solve_device<float>(); }

  // One V-cycle from the current defect with every instance taking part (a converged one
  // too: its active flag is set, as at the start of a solve), its kernels launched one by one
  // with an event after each; kind[i] and us[i] (microseconds between consecutive events) for
  // up to cap kernels.
  int profile_vcycle(int* kind, float* us, int cap, int* n) {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kinds;
    cudaEvent_t e0 = nullptr;
    int rc = cuda(cudaMemsetAsync(d_active.p, 1, (size_t)ninst * sizeof(int), stream), "active");  // nonzero
    if (!rc) rc = cuda(cudaEventCreate(&e0), "event");
    if (!rc) {
      ev.push_back(e0);
      rc = cuda(cudaEventRecord(e0, stream), "event");
    }
    if (!rc) {
      prof_ev = &ev;
      prof_kind = &kinds;
      rc = precision == AMR_FP64 ? enqueue_vcycle<double>() : enqueue_vcycle<float>();
      prof_ev = nullptr;
      prof_kind = nullptr;
    }
    if (!rc) rc = cuda(cudaStreamSynchronize(stream), "sync");
    if (!rc) {
      *n = (int)kinds.size();
      for (int i = 0; i < (int)kinds.size() && i < cap; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
        kind[i] = kinds[i];
        us[i] = ms * 1e3f;
      }
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    return rc;
  }

  int results(int* cycles, double* relres, bool* all_ok) {
    std::vector<int> cyc(ninst), fl(ninst);
    std::vector<double> lr(ninst), bn(ninst);
    int rc;
    if ((rc = cuda(cudaMemcpy(cyc.data(), d_cycles.p, ninst * 4, cudaMemcpyDeviceToHost), "copy")) ||
        (rc = cuda(cudaMemcpy(fl.data(), d_failed.p, ninst * 4, cudaMemcpyDeviceToHost), "copy")) ||
        (rc = cuda(cudaMemcpy(lr.data(), d_lastres.p, ninst * 8, cudaMemcpyDeviceToHost), "copy")) ||
        (rc = cuda(cudaMemcpy(bn.data(), d_bnorm.p, ninst * 8, cudaMemcpyDeviceToHost), "copy")))
      return rc;
    *all_ok = true;
    for (int i = 0; i < ninst; ++i) {
      if (cycles) cycles[i] = cyc[i];
      if (relres) relres[i] = bn[i] > 0 ? lr[i] / bn[i] : lr[i];
      if (fl[i]) *all_ok = false;
    }
    return AMR_OK;
  }
};

}  // namespace mggpu

using namespace mggpu;

struct mg_handle {
  Mg mg;
};

// Helmholtz constant of species s: 2/(dt D) for the IMEX trapezoidal stage, 1/(dt D) for
// the backward-Euler stage of the split scheme (the explicit scheme does not solve)
inline double rd_lambda(const rd_config& c, int s) {
  return (c.scheme == RD_SPLIT ? 1.0 : 2.0) / (c.dt * (s == 0 ? c.Du : c.Dv));
}

constexpr int kExplicitGraphSteps = 32;  // explicit steps per captured graph
constexpr int kLogSteps = 256;           // implicit steps per host wait (rows of the cycle log)

struct rd_handle {
  Mg mg;
  cudaGraphExec_t egraph = nullptr;  // kExplicitGraphSteps explicit steps
  cudaGraphExec_t stgraph = nullptr; // one implicit step with its device-side solve
  cudaGraphExec_t gstgraph = nullptr;  // the same with the learned guess (fused inference)
  long long guess_launches = 0;        // kernels of the learned guess in one step
  cudaEvent_t order_ev = nullptr;      // orders the network's own stream around the step replays
  DevBuf d_log, d_stepctr;           // per-step cycle log ([kLogSteps][2 n_inst]) and its counter
  void drop_guess_graph() {
    if (gstgraph) cudaGraphExecDestroy(gstgraph);
    gstgraph = nullptr;
  }
  ~rd_handle() {
    if (egraph) cudaGraphExecDestroy(egraph);
    if (stgraph) cudaGraphExecDestroy(stgraph);
    drop_guess_graph();
    if (order_ev) cudaEventDestroy(order_ev);
  }
  rd_config cfg{};
  std::vector<int> sizes;
  DevBuf d_u, d_v, d_Fn;
  DevBuf d_wn, d_prev, d_pin;  // state before the last step, last solution, solution before the last step
  DevBuf d_cin, d_cout;        // network input / output of one instance (float)
  bool have_prev = false;
  cnn_handle* guess = nullptr;
  double guess_scale = 1.0;
  int guess_inputs = RD_GUESS_IN_PREV;
  std::string err;
  long long cells = 0;
  long long maxcells = 0;
};

extern "C" {

int mg_create(const mg_config* cfg, mg_handle** out) {
  if (!cfg || !out) return AMR_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<mg_handle> h(new mg_handle());
  int rc = h->mg.setup(cfg->ndim, cfg->n_inst, cfg->n_cells, cfg->lambda, cfg->L, cfg->nu1, cfg->nu2, cfg->max_cycles,
                       cfg->rtol, cfg->coarse_max, cfg->precision, cfg->bc, cfg->stream);
  if (rc) return rc;
  *out = h.release();
  return AMR_OK;
}

int mg_destroy(mg_handle* h) {
  if (!h) return AMR_ERR_INVALID_ARG;
  delete h;
  return AMR_OK;
}

const char* mg_last_error(const mg_handle* h) { return h ? h->mg.err.c_str() : "null handle"; }

int mg_num_unknowns(const mg_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = h->mg.n0;
  return AMR_OK;
}

}  // extern "C"

int mg_capture_solve(mg_handle* h, const double* b, double* x, cudaStream_t s) {
  Mg& M = h->mg;
  cudaStream_t saved = M.stream;
  M.stream = s;
  int rc = M.cuda(cudaMemcpyAsync(M.d_B.p, b, M.n0 * 8, cudaMemcpyDeviceToDevice, s), "copy b");
  if (!rc) rc = M.cuda(cudaMemcpyAsync(M.d_X.p, x, M.n0 * 8, cudaMemcpyDeviceToDevice, s), "copy x");
  if (!rc) rc = M.capture_solve_any();
  if (!rc) rc = M.cuda(cudaMemcpyAsync(x, M.d_X.p, M.n0 * 8, cudaMemcpyDeviceToDevice, s), "copy x back");
  M.stream = saved;
  return rc;
}

const int* mg_device_cycles(const mg_handle* h) { return h->mg.d_cycles.as<int>(); }

long long mg_loop_kernels(const mg_handle* h) { return h->mg.solve_loop_kernels; }

extern "C" {

int mg_strip_height(const mg_handle* h, int side, int* height) {
  if (!h || !height) return AMR_ERR_INVALID_ARG;
  auto it = h->mg.strip_h.find(side);
  if (it == h->mg.strip_h.end()) return AMR_ERR_INVALID_ARG;
  *height = it->second;
  return AMR_OK;
}

int mg_profile_vcycle(mg_handle* h, int* kind, float* us, int cap, int* nkernels) {
  if (!h || !kind || !us || !nkernels || cap < 0) return AMR_ERR_INVALID_ARG;
  if (!h->mg.solved) return h->mg.fail(AMR_ERR_INVALID_ARG, "mg_profile_vcycle needs a prior mg_solve");
  return h->mg.profile_vcycle(kind, us, cap, nkernels);
}

int mg_kernel_launches(const mg_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = h->mg.launches;
  return AMR_OK;
}

int rd_kernel_launches(const rd_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = h->mg.launches;
  return AMR_OK;
}

int mg_solve(mg_handle* h, const double* b, double* x, int on_device, int* cycles, double* relres) {
  if (!h || !b || !x) return AMR_ERR_INVALID_ARG;
  Mg& M = h->mg;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (int rc = M.cuda(cudaMemcpyAsync(M.d_B.p, b, M.n0 * 8, k, M.stream), "copy b")) return rc;
  if (int rc = M.cuda(cudaMemcpyAsync(M.d_X.p, x, M.n0 * 8, k, M.stream), "copy x")) return rc;
  int rc = M.solve_graph_launch_any();
  if (rc) return rc;
  M.solved = true;
  cudaMemcpyKind kb = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if ((rc = M.cuda(cudaMemcpyAsync(x, M.d_X.p, M.n0 * 8, kb, M.stream), "copy x back"))) return rc;
  if ((rc = M.cuda(cudaStreamSynchronize(M.stream), "sync"))) return rc;
  bool ok;
  std::vector<int> cyc(M.ninst);
  if ((rc = M.results(cyc.data(), relres, &ok))) return rc;
  if (cycles) std::memcpy(cycles, cyc.data(), cyc.size() * sizeof(int));
  M.launches += M.solve_kernels(*std::max_element(cyc.begin(), cyc.end()));
  if (!ok) return M.fail(MG_ERR_NOT_CONVERGED, "an instance did not reach rtol within max_cycles");
  return AMR_OK;
}

int rd_create(const rd_config* cfg, rd_handle** out) {
  if (!cfg || !out || cfg->n_inst < 1 || !cfg->n_cells) return AMR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(cfg->dt > 0) || !(cfg->Du > 0) || !(cfg->Dv > 0)) return AMR_ERR_INVALID_ARG;
  if ((cfg->model != RD_GRAY_SCOTT && cfg->model != RD_SCHNAKENBERG) ||
      (cfg->scheme != RD_IMEX && cfg->scheme != RD_SPLIT && cfg->scheme != RD_EXPLICIT))
    return AMR_ERR_INVALID_ARG;
  std::unique_ptr<rd_handle> h(new rd_handle());
  h->cfg = *cfg;
  h->sizes.assign(cfg->n_cells, cfg->n_cells + cfg->n_inst);
  h->cfg.n_cells = h->sizes.data();
  // multigrid batch: species-major (u of every instance, then v)
  std::vector<int> n2(2 * cfg->n_inst);
  std::vector<double> lam(2 * cfg->n_inst);
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < cfg->n_inst; ++i) {
      n2[s * cfg->n_inst + i] = cfg->n_cells[i];
      lam[s * cfg->n_inst + i] = rd_lambda(*cfg, s);
    }
  int rc = h->mg.setup(cfg->ndim, 2 * cfg->n_inst, n2.data(), lam.data(), cfg->L, cfg->nu1, cfg->nu2, cfg->max_cycles,
                       cfg->rtol, cfg->coarse_max, cfg->precision, cfg->bc, cfg->stream);
  if (rc) return rc;
  h->cells = h->mg.insts[cfg->n_inst].off0;  // species-0 block size = cells of all instances
  for (int i = 0; i < cfg->n_inst; ++i) {
    long long c = 1;
    for (int d = 0; d < cfg->ndim; ++d) c *= cfg->n_cells[i];
    h->maxcells = std::max(h->maxcells, c);
  }
  if ((rc = h->mg.cuda(h->d_u.alloc(h->cells * 8), "alloc u")) || (rc = h->mg.cuda(h->d_v.alloc(h->cells * 8), "alloc v")) ||
      (rc = h->mg.cuda(h->d_Fn.alloc(2 * h->cells * 8), "alloc Fn")) ||
      (rc = h->mg.cuda(h->d_wn.alloc(2 * h->cells * 8), "alloc")) ||
      (rc = h->mg.cuda(h->d_prev.alloc(2 * h->cells * 8), "alloc")) ||
      (rc = h->mg.cuda(h->d_pin.alloc(2 * h->cells * 8), "alloc")) ||
      (rc = h->mg.cuda(h->d_log.alloc((size_t)kLogSteps * 2 * cfg->n_inst * sizeof(int)), "alloc")) ||
      (rc = h->mg.cuda(h->d_stepctr.alloc(sizeof(int)), "alloc")))
    return rc;
  *out = h.release();
  return AMR_OK;
}

int rd_destroy(rd_handle* h) {
  if (!h) return AMR_ERR_INVALID_ARG;
  delete h;
  return AMR_OK;
}

const char* rd_last_error(const rd_handle* h) { return h ? h->mg.err.c_str() : "null handle"; }

int rd_set_state(rd_handle* h, const double* u, const double* v, int on_device) {
  if (!h || !u || !v) return AMR_ERR_INVALID_ARG;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  Mg& M = h->mg;
  if (int rc = M.cuda(cudaMemcpyAsync(h->d_u.p, u, h->cells * 8, k, M.stream), "copy u")) return rc;
  if (int rc = M.cuda(cudaMemcpyAsync(h->d_v.p, v, h->cells * 8, k, M.stream), "copy v")) return rc;
  // the first step's "previous solution" is the state itself
  if (int rc = M.cuda(cudaMemcpyAsync(h->d_prev.p, h->d_u.p, h->cells * 8, cudaMemcpyDeviceToDevice, M.stream), "copy"))
    return rc;
  if (int rc = M.cuda(cudaMemcpyAsync(h->d_prev.as<double>() + h->cells, h->d_v.p, h->cells * 8,
                                      cudaMemcpyDeviceToDevice, M.stream), "copy"))
    return rc;
  h->have_prev = false;
  return M.cuda(cudaStreamSynchronize(M.stream), "sync");
}

int rd_read_state(rd_handle* h, double* u, double* v, int on_device) {
  if (!h || !u || !v) return AMR_ERR_INVALID_ARG;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  Mg& M = h->mg;
  if (int rc = M.cuda(cudaMemcpyAsync(u, h->d_u.p, h->cells * 8, k, M.stream), "copy u")) return rc;
  if (int rc = M.cuda(cudaMemcpyAsync(v, h->d_v.p, h->cells * 8, k, M.stream), "copy v")) return rc;
  return M.cuda(cudaStreamSynchronize(M.stream), "sync");
}

int rd_step(rd_handle* h, int nsteps, int* cycles) {
  if (!h || nsteps < 0) return AMR_ERR_INVALID_ARG;
  Mg& M = h->mg;
  const int ni = h->cfg.n_inst;
  const int scheme = h->cfg.scheme;
  RdArgs A{};
  A.inst = M.d_inst.as<InstDev>();
  A.ninst = ni;
  A.ndim = h->cfg.ndim;
  A.model = h->cfg.model;
  A.neu = h->cfg.bc == MG_BC_NEUMANN ? 1 : 0;
  A.F = h->cfg.F;
  A.k = h->cfg.k;
  A.kappa = h->cfg.kappa;
  A.a = h->cfg.a;
  A.b = h->cfg.b;
  A.dt = h->cfg.dt;
  A.D[0] = h->cfg.Du;
  A.D[1] = h->cfg.Dv;
  A.lam[0] = rd_lambda(h->cfg, 0);
  A.lam[1] = rd_lambda(h->cfg, 1);
  A.u = h->d_u.as<double>();
  A.v = h->d_v.as<double>();
  A.X = M.d_X.as<double>();
  A.B = M.d_B.as<double>();
  A.Fn = h->d_Fn.as<double>();
  // level-0 chunks of species 0 only
  unsigned nch0 = 0;
  for (const Chunk& c : M.ch0)
    if (c.inst < ni) ++nch0;
  const Chunk* ch0 = M.d_ch0.as<Chunk>();
  int rc;
  if (scheme == RD_EXPLICIT) {
    auto enqueue = [&](int k) {
      for (int s = 0; s < k; ++s) {
        rd_explicit_kernel<0><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
        rd_explicit_kernel<1><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
        rd_explicit_kernel<2><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
      }
    };
    int left = nsteps;
    if (nsteps >= kExplicitGraphSteps) {  // long runs: replay a captured graph of 32 steps
      if (!h->egraph) {
        cudaGraph_t g;
        if ((rc = M.cuda(cudaStreamBeginCapture(M.stream, cudaStreamCaptureModeThreadLocal), "capture"))) return rc;
        enqueue(kExplicitGraphSteps);
        cudaError_t ec = cudaStreamEndCapture(M.stream, &g);
        if ((rc = M.cuda(ec, "end capture"))) return rc;
        rc = M.cuda(cudaGraphInstantiate(&h->egraph, g, 0), "instantiate");
        cudaGraphDestroy(g);
        if (rc) return rc;
      }
      for (; left >= kExplicitGraphSteps; left -= kExplicitGraphSteps)
        if ((rc = M.cuda(cudaGraphLaunch(h->egraph, M.stream), "graph launch"))) return rc;
    }
    enqueue(left);
    M.launches += 3LL * nsteps;
    if (cycles) std::memset(cycles, 0, sizeof(int) * (size_t)nsteps * 2 * ni);
    if ((rc = M.cuda(cudaGetLastError(), "rd launch"))) return rc;
    return M.cuda(cudaStreamSynchronize(M.stream), "sync");
  }
  const size_t cb = (size_t)h->cells * 8;
  double* wn = h->d_wn.as<double>();
  double* prev = h->d_prev.as<double>();
  double* pin = h->d_pin.as<double>();
  // learned guess: per instance the network's input channels, one inference and the guess
  // X = w_n + scale * net, before the solve.  captured: the fused inference's single launch
  // (no event, no allocation), for a step replayed from a graph.
  auto enqueue_guess = [&](bool captured) -> int {
    for (int i = 0; i < ni; ++i) {
      const InstDev& I = M.insts[i];
      long long n0 = 1;
      for (int d = 0; d < h->cfg.ndim; ++d) n0 *= I.n[0];
      unsigned nb = (unsigned)((n0 + 255) / 256);
      rd_cnn_input_kernel<<<nb, 256, 0, M.stream>>>(M.d_inst.as<InstDev>(), i, i + ni, M.d_B.as<double>(), wn, pin,
                                                     h->cells, n0, (float)h->cfg.dt, h->guess_inputs, h->cfg.ndim,
                                                     h->cfg.bc == MG_BC_NEUMANN ? 1 : 0, 1.0 / h->guess_scale,
                                                     h->d_cin.as<float>());
      int n = I.n[0];
      int crc = captured ? cnn_enqueue_fused(h->guess, h->d_cin.as<float>(), 1, n, n, h->d_cout.as<float>(), M.stream)
                         : cnn_forward_async(h->guess, h->d_cin.as<float>(), 1, h->cfg.ndim == 3 ? n : 1, n, n,
                                             h->d_cout.as<float>(), M.stream, true);
      if (crc) return M.fail(crc, std::string("learned guess: ") + cnn_last_error(h->guess));
      rd_cnn_guess_kernel<<<nb, 256, 0, M.stream>>>(M.d_inst.as<InstDev>(), i, i + ni, h->d_cout.as<float>(), n0,
                                                    h->guess_scale, M.d_X.as<double>(), wn, h->cells);
      M.launches += 2;
    }
    return AMR_OK;
  };
  // One implicit step as a graph: (IMEX: keep w_n and the previous solution) right-hand side,
  // (learned guess), the solve with its device-side convergence loop, (IMEX: keep the
  // solution) finish, and a row of the cycle log.
  auto capture_step = [&](cudaGraphExec_t* out, bool with_guess) -> int {
    cudaGraph_t g;
    int rc2;
    if ((rc2 = M.cuda(cudaStreamBeginCapture(M.stream, cudaStreamCaptureModeThreadLocal), "capture"))) return rc2;
    int crc = AMR_OK;
    if (scheme == RD_IMEX) {
      cudaMemcpyAsync(wn, h->d_u.p, cb, cudaMemcpyDeviceToDevice, M.stream);
      cudaMemcpyAsync(wn + h->cells, h->d_v.p, cb, cudaMemcpyDeviceToDevice, M.stream);
      cudaMemcpyAsync(pin, prev, 2 * cb, cudaMemcpyDeviceToDevice, M.stream);
      rd_rhs_kernel<RD_IMEX><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
    } else {
      rd_rhs_kernel<RD_SPLIT><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
    }
    const long long l0 = M.launches;
    if (with_guess) crc = enqueue_guess(true);
    h->guess_launches = M.launches - l0;
    M.launches = l0;
    if (!crc) crc = M.capture_solve_any();
    if (scheme == RD_IMEX) {
      cudaMemcpyAsync(prev, M.d_X.p, 2 * cb, cudaMemcpyDeviceToDevice, M.stream);
      rd_finish_kernel<RD_IMEX><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
    } else {
      rd_finish_kernel<RD_SPLIT><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
    }
    log_kernel<<<1, 256, 0, M.stream>>>(M.state(), M.ninst, h->d_log.as<int>(), h->d_stepctr.as<int>(), kLogSteps);
    cudaError_t ec = cudaStreamEndCapture(M.stream, &g);
    if (crc) {
      if (ec == cudaSuccess) cudaGraphDestroy(g);
      return crc;
    }
    if ((rc2 = M.cuda(ec, "end capture"))) return rc2;
    rc2 = M.cuda(cudaGraphInstantiate(out, g, 0), "instantiate");
    cudaGraphDestroy(g);
    return rc2;
  };
  // k replays of a step graph from step s_first; the host waits once per kLogSteps steps
  auto replay = [&](cudaGraphExec_t gx, int s_first, int k_all, long long extra_launches) -> int {
    std::vector<int> log((size_t)kLogSteps * 2 * ni);
    bool failed = false;
    int rc2;
    for (int s0 = 0; s0 < k_all; s0 += kLogSteps) {
      const int k = std::min(kLogSteps, k_all - s0);
      if ((rc2 = M.cuda(cudaMemsetAsync(h->d_stepctr.p, 0, sizeof(int), M.stream), "memset"))) return rc2;
      for (int s = 0; s < k; ++s)
        if ((rc2 = M.cuda(cudaGraphLaunch(gx, M.stream), "step graph launch"))) return rc2;
      if ((rc2 = M.cuda(cudaMemcpyAsync(log.data(), h->d_log.p, (size_t)k * 2 * ni * sizeof(int),
                                        cudaMemcpyDeviceToHost, M.stream), "copy log")))
        return rc2;
      if ((rc2 = M.cuda(cudaStreamSynchronize(M.stream), "sync"))) return rc2;
      for (int s = 0; s < k; ++s) {
        int maxc = 0;
        for (int i = 0; i < 2 * ni; ++i) {
          int e = log[(size_t)s * 2 * ni + i];
          if (e < 0) {
            failed = true;
            e = -1 - e;
          }
          maxc = std::max(maxc, e);
          if (cycles) cycles[(size_t)(s_first + s0 + s) * 2 * ni + i] = e;
        }
        M.launches += 3 + extra_launches + M.solve_kernels(maxc);
      }
    }
    if (scheme == RD_IMEX && k_all > 0) h->have_prev = true;
    if (failed) return M.fail(MG_ERR_NOT_CONVERGED, "an instance did not reach rtol within max_cycles");
    return M.cuda(cudaGetLastError(), "rd step");
  };
  if (!h->guess) {
    if (!h->stgraph && (rc = capture_step(&h->stgraph, false))) return rc;
    return replay(h->stgraph, 0, nsteps, 0);
  }
  // Learned guess.  Steps replay one captured graph, like the previous-step guess, when the
  // network's fused inference applies to every instance (2D, sides multiples of 32 and 16)
  // and a previous solution exists; otherwise (and for the first step after a new state,
  // whose network inputs use w_n for the missing previous solution) steps run launch by launch.
  bool capturable = scheme == RD_IMEX;
  for (int i = 0; i < ni; ++i) {
    const int n = M.insts[i].n[0];
    capturable = capturable && cnn_fused_applies(h->guess, h->cfg.ndim == 3 ? n : 1, n, n);
  }
  const int eager = capturable ? (h->have_prev ? 0 : std::min(1, nsteps)) : nsteps;
  for (int s = 0; s < eager; ++s) {
    if (scheme == RD_IMEX) {
      // keep w_n and the previous solution (inputs of the learned guess and of training crops)
      if ((rc = M.cuda(cudaMemcpyAsync(wn, h->d_u.p, cb, cudaMemcpyDeviceToDevice, M.stream), "copy")) ||
          (rc = M.cuda(cudaMemcpyAsync(wn + h->cells, h->d_v.p, cb, cudaMemcpyDeviceToDevice, M.stream), "copy")) ||
          (rc = M.cuda(cudaMemcpyAsync(pin, h->have_prev ? prev : wn, 2 * cb, cudaMemcpyDeviceToDevice, M.stream),
                       "copy")))
        return rc;
      rd_rhs_kernel<RD_IMEX><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
    } else {
      rd_rhs_kernel<RD_SPLIT><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
    }
    ++M.launches;
    // the network runs in order on the solver's stream (no host synchronisation)
    if ((rc = enqueue_guess(false))) return rc;
    rc = M.solve_device_any();
    if (rc) return rc;
    if (scheme == RD_IMEX) {
      if ((rc = M.cuda(cudaMemcpyAsync(prev, M.d_X.p, 2 * cb, cudaMemcpyDeviceToDevice, M.stream), "copy"))) return rc;
      h->have_prev = true;
    }
    bool ok;
    std::vector<int> cyc(2 * ni);
    if ((rc = M.results(cyc.data(), nullptr, &ok))) return rc;
    if (cycles) std::memcpy(cycles + (size_t)s * 2 * ni, cyc.data(), cyc.size() * sizeof(int));
    if (!ok) return M.fail(MG_ERR_NOT_CONVERGED, "an instance did not reach rtol within max_cycles");
    if (scheme == RD_IMEX)
      rd_finish_kernel<RD_IMEX><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
    else
      rd_finish_kernel<RD_SPLIT><<<nch0, kChunk, 0, M.stream>>>(A, ch0);
    ++M.launches;
    if ((rc = M.cuda(cudaGetLastError(), "rd launch"))) return rc;
  }
  if (eager < nsteps) {
    if (!h->gstgraph && (rc = capture_step(&h->gstgraph, true))) return rc;
    // the network's pending work (weight repacks) before the replays, its later work after them
    cudaStream_t ns = cnn_own_stream(h->guess);
    if (!h->order_ev && (rc = M.cuda(cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming), "event")))
      return rc;
    if (ns && ns != M.stream &&
        ((rc = M.cuda(cudaEventRecord(h->order_ev, ns), "event")) ||
         (rc = M.cuda(cudaStreamWaitEvent(M.stream, h->order_ev, 0), "event"))))
      return rc;
    rc = replay(h->gstgraph, eager, nsteps - eager, h->guess_launches);
    if (ns && ns != M.stream) {
      int rc2;
      if ((rc2 = M.cuda(cudaEventRecord(h->order_ev, M.stream), "event")) ||
          (rc2 = M.cuda(cudaStreamWaitEvent(ns, h->order_ev, 0), "event")))
        return rc ? rc : rc2;
    }
    return rc;
  }
  return M.cuda(cudaStreamSynchronize(M.stream), "sync");
}

int rd_last_residuals(rd_handle* h, double* initial, double* final_) {
  if (!h) return AMR_ERR_INVALID_ARG;
  Mg& M = h->mg;
  std::vector<double> ir(M.ninst), lr(M.ninst), bn(M.ninst);
  int rc;
  if ((rc = M.cuda(cudaMemcpy(ir.data(), M.d_initres.p, M.ninst * 8, cudaMemcpyDeviceToHost), "copy")) ||
      (rc = M.cuda(cudaMemcpy(lr.data(), M.d_lastres.p, M.ninst * 8, cudaMemcpyDeviceToHost), "copy")) ||
      (rc = M.cuda(cudaMemcpy(bn.data(), M.d_bnorm.p, M.ninst * 8, cudaMemcpyDeviceToHost), "copy")))
    return rc;
  for (int i = 0; i < M.ninst; ++i) {
    double b = bn[i] > 0 ? bn[i] : 1.0;
    if (initial) initial[i] = ir[i] / b;
    if (final_) final_[i] = lr[i] / b;
  }
  return AMR_OK;
}

int rd_set_guess(rd_handle* h, cnn_handle* net, double scale) {
  if (!h || (net && !(scale > 0))) return AMR_ERR_INVALID_ARG;
  if (net && h->cfg.scheme != RD_IMEX) return h->mg.fail(AMR_ERR_INVALID_ARG, "the learned guess is for the IMEX scheme");
  if (net) {
    for (int n : h->sizes) {
      if (h->cfg.ndim == 2 && n % 16 != 0) return h->mg.fail(AMR_ERR_INVALID_ARG, "learned guess needs sides multiple of 16");
      if (h->cfg.ndim == 3 && n % 8 != 0) return h->mg.fail(AMR_ERR_INVALID_ARG, "learned guess needs sides multiple of 8");
    }
    int rc;
    if ((rc = h->mg.cuda(h->d_cin.alloc((size_t)h->maxcells * 5 * sizeof(float)), "alloc")) ||
        (rc = h->mg.cuda(h->d_cout.alloc((size_t)h->maxcells * 2 * sizeof(float)), "alloc")))
      return rc;
  }
  h->guess = net;
  h->guess_scale = net ? scale : 1.0;
  h->drop_guess_graph();  // its buffers, network and scale are baked into the graph
  return AMR_OK;
}

int rd_set_guess_inputs(rd_handle* h, int kind) {
  if (!h || (kind != RD_GUESS_IN_PREV && kind != RD_GUESS_IN_RESIDUAL)) return AMR_ERR_INVALID_ARG;
  h->guess_inputs = kind;
  h->drop_guess_graph();
  return AMR_OK;
}

int rd_extract_crops(rd_handle* h, int ncrops, const int* inst, const int* corner, int crop, double scale, float* in,
                     float* target) {
  if (!h || ncrops < 1 || !inst || !corner || crop < 1 || !(scale > 0) || !in || !target) return AMR_ERR_INVALID_ARG;
  if (!h->have_prev) return h->mg.fail(AMR_ERR_INVALID_ARG, "no IMEX step taken yet");
  Mg& M = h->mg;
  for (int k = 0; k < ncrops; ++k)
    if (inst[k] < 0 || inst[k] >= h->cfg.n_inst || crop > h->sizes[inst[k]]) return AMR_ERR_INVALID_ARG;
  DevBuf dinst, dcorner;
  int rc;
  if ((rc = M.cuda(dinst.alloc(ncrops * sizeof(int)), "alloc")) || (rc = M.cuda(dcorner.alloc(ncrops * 3 * sizeof(int)), "alloc")))
    return rc;
  if ((rc = M.cuda(cudaMemcpy(dinst.p, inst, ncrops * sizeof(int), cudaMemcpyHostToDevice), "copy")) ||
      (rc = M.cuda(cudaMemcpy(dcorner.p, corner, ncrops * 3 * sizeof(int), cudaMemcpyHostToDevice), "copy")))
    return rc;
  CropArgs A{};
  A.inst = M.d_inst.as<InstDev>();
  A.cinst = dinst.as<int>();
  A.corner = dcorner.as<int>();
  A.ninst = h->cfg.n_inst;
  A.ndim = h->cfg.ndim;
  A.crop = crop;
  A.ncrops = ncrops;
  A.cells = h->cells;
  A.wn = h->d_wn.as<double>();
  A.pin = h->d_pin.as<double>();
  A.X = M.d_X.as<double>();
  A.B = M.d_B.as<double>();
  A.dt = (float)h->cfg.dt;
  A.inv_scale = 1.0 / scale;
  A.kind = h->guess_inputs;
  A.neu = h->cfg.bc == MG_BC_NEUMANN ? 1 : 0;
  A.in = in;
  A.tgt = target;
  long long cp = 1;
  for (int d = 0; d < h->cfg.ndim; ++d) cp *= crop;
  rd_crop_kernel<<<(unsigned)((cp * ncrops + 255) / 256), 256, 0, M.stream>>>(A);
  ++M.launches;
  if ((rc = M.cuda(cudaGetLastError(), "crops"))) return rc;
  return M.cuda(cudaStreamSynchronize(M.stream), "sync");
}

}  // extern "C"
