// Multigrid for the Helmholtz problem (lambda - lap_h) x = b on the leaves of a 2D block
// quadtree (Sec. 1.4: the multigrid is AMR-compatible; Sec. 2.5.2 runs it on a three-level
// mesh), float64.
//
// Discretisation (the paper defers it to mg2019; these are the readings this file and the
// test oracle share):
//  * composite operator on leaf cells: 5-point stencil of the cell's level; a coarser
//    neighbour contributes g = (2/3) C^ + (1/3) f0 with C^ = C + s (C_t+ - C_t-) / 8 (linear
//    along the normal and along the face); a refined neighbour block contributes
//    (4/3) m - (1/3) f0 with m the mean of the two finer cells touching the face (flux
//    matching: the operator is conservative);
//  * level operator: the same, except that a refined same-level block contributes its own
//    level values (the means of its children);
//  * full approximation scheme over the levels: red-black Gauss-Seidel of the level
//    operator, the restriction of x and of the residual (means of 2x2 children), the
//    composite residual for leaves of the coarser level, b = r + A x there, cell-centred
//    bilinear prolongation (9/16, 3/16, 3/16, 1/16) of the coarse change, and the base grid
//    (level 1, uniform) solved in correction form, A e = b - A x from e = 0 to base_rtol of
//    max|b - A x|, by the batched uniform multigrid of mg.cu.
//
// Layout: every block of every level (leaves and refined blocks) owns B*B values of x, b,
// r, x_before and (leaves) the composite right-hand side, x fastest; a dense table per
// level maps block coordinates to block indices (-1 where the level has no block), so a
// stencil finds any neighbour cell by its global level indices.  One CTA of B*B threads per
// block; the operations are level-by-level kernels in the order of the V-cycle.  This unit
// is compiled without multiply-add contraction, so its arithmetic is the written one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/amrvac_gb300.h"
#include "mg_internal.h"

namespace mgtree {

constexpr int kMaxLev = 12;

struct TreeDev {
  int B, lmax;
  double lam;
  const int* table[kMaxLev + 1];  // level l: [ny(l)][nx(l)] block index or -1
  int nx[kMaxLev + 1], ny[kMaxLev + 1];
  double ih2[kMaxLev + 1];
  const int* leaf;  // [block] 1 for a leaf
  double* x;
  double* b;
  double* r;
  double* xold;
  double* bo;       // composite right-hand side (leaves)
};

__device__ __forceinline__ int wrapc(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// block index of global level-l cell (I, J) (periodic) and the cell's offset in the block
__device__ __forceinline__ int blk_at(const TreeDev& T, int l, int I, int J, int* off) {
  if (l < 1 || l > T.lmax) return -1;
  const int B = T.B;
  I = wrapc(I, T.nx[l] * B);
  J = wrapc(J, T.ny[l] * B);
  *off = (J % B) * B + (I % B);
  return T.table[l][(J / B) * T.nx[l] + I / B];
}

__device__ __forceinline__ bool cell(const TreeDev& T, const double* F, int l, int I, int J, double* v) {
  int off;
  const int k = blk_at(T, l, I, J, &off);
  if (k < 0) return false;
  *v = F[(size_t)k * T.B * T.B + off];
  return true;
}

// the value the stencil of a level-l cell (value f0) reads for its neighbour cell (I, J)
// across the face normal to d (side +1: the neighbour is in the + direction); leafcell:
// the composite operator at a leaf cell
__device__ double nbr(const TreeDev& T, const double* F, int l, int I, int J, int d, int side, double f0,
                      bool leafcell) {
  const int B = T.B;
  I = wrapc(I, T.nx[l] * B);
  J = wrapc(J, T.ny[l] * B);
  const int k = T.table[l][(J / B) * T.nx[l] + I / B];
  if (k >= 0) {
    const double v = F[(size_t)k * B * B + (J % B) * B + (I % B)];
    if (T.leaf[k] || !leafcell) return v;
    const int n = side > 0 ? 0 : 1;  // the children's layer nearest the face
    double a, c;
    bool ok;
    if (d == 0)
      ok = cell(T, F, l + 1, 2 * I + n, 2 * J, &a) && cell(T, F, l + 1, 2 * I + n, 2 * J + 1, &c);
    else
      ok = cell(T, F, l + 1, 2 * I, 2 * J + n, &a) && cell(T, F, l + 1, 2 * I + 1, 2 * J + n, &c);
    if (!ok) return nan("");
    const double m = 0.5 * (a + c);
    return (4.0 / 3.0) * m - (1.0 / 3.0) * f0;
  }
  const int Ic = I >> 1, Jc = J >> 1;
  double C, Cp, Cm;
  bool ok = cell(T, F, l - 1, Ic, Jc, &C);
  if (d == 0)
    ok = ok && cell(T, F, l - 1, Ic, Jc + 1, &Cp) && cell(T, F, l - 1, Ic, Jc - 1, &Cm);
  else
    ok = ok && cell(T, F, l - 1, Ic + 1, Jc, &Cp) && cell(T, F, l - 1, Ic - 1, Jc, &Cm);
  if (!ok) return nan("");
  const int t = d == 0 ? J : I;
  const double s = (t & 1) ? 1.0 : -1.0;
  const double Chat = C + (s * (Cp - Cm)) * 0.125;
  return (2.0 / 3.0) * Chat + (1.0 / 3.0) * f0;
}

struct Cell {
  int k, l, i, j, I, J;
};

__device__ __forceinline__ Cell cell_of_thread(const TreeDev& T, const int* list, int l, const int* bxy) {
  Cell c;
  c.k = list[blockIdx.x];
  c.l = l;
  c.i = threadIdx.x % T.B;
  c.j = threadIdx.x / T.B;
  c.I = bxy[2 * c.k] * T.B + c.i;
  c.J = bxy[2 * c.k + 1] * T.B + c.j;
  return c;
}

__device__ __forceinline__ double nbr_sum(const TreeDev& T, const double* F, const Cell& c, double x0, bool comp) {
  const bool lf = comp && T.leaf[c.k];
  double s = nbr(T, F, c.l, c.I - 1, c.J, 0, -1, x0, lf);
  s = s + nbr(T, F, c.l, c.I + 1, c.J, 0, +1, x0, lf);
  s = s + nbr(T, F, c.l, c.I, c.J - 1, 1, -1, x0, lf);
  s = s + nbr(T, F, c.l, c.I, c.J + 1, 1, +1, x0, lf);
  return s;
}

__device__ __forceinline__ double apply_at(const TreeDev& T, const double* F, const Cell& c, bool comp) {
  const double x0 = F[(size_t)c.k * T.B * T.B + c.j * T.B + c.i];
  const double s = nbr_sum(T, F, c, x0, comp);
  return T.lam * x0 - (s - 4.0 * x0) * T.ih2[c.l];
}

// ---------------------------------------------------------------- kernels --
// red-black Gauss-Seidel, one colour, every block of the list (level l)
__global__ void gs_kernel(TreeDev T, const int* list, const int* bxy, int l, int colour) {
  const Cell c = cell_of_thread(T, list, l, bxy);
  if (((c.I + c.J) & 1) != colour) return;
  const size_t q = (size_t)c.k * T.B * T.B + c.j * T.B + c.i;
  const double x0 = T.x[q];
  const double s = nbr_sum(T, T.x, c, x0, false);
  const double ih2 = T.ih2[l];
  T.x[q] = (T.b[q] + s * ih2) / (T.lam + 4.0 * ih2);
}

// r = b - A x (level operator) on the list
__global__ void level_residual_kernel(TreeDev T, const int* list, const int* bxy, int l) {
  const Cell c = cell_of_thread(T, list, l, bxy);
  const size_t q = (size_t)c.k * T.B * T.B + c.j * T.B + c.i;
  T.r[q] = T.b[q] - apply_at(T, T.x, c, false);
}

// leaves of the list: r = bo - A x (composite operator); then every block: b = r + A x
// (level operator).  Two kernels: the second reads x only, so the order within a kernel
// does not matter.
__global__ void composite_residual_kernel(TreeDev T, const int* list, const int* bxy, int l) {
  const Cell c = cell_of_thread(T, list, l, bxy);
  if (!T.leaf[c.k]) return;
  const size_t q = (size_t)c.k * T.B * T.B + c.j * T.B + c.i;
  T.r[q] = T.bo[q] - apply_at(T, T.x, c, true);
}

__global__ void fas_rhs_kernel(TreeDev T, const int* list, const int* bxy, int l) {
  const Cell c = cell_of_thread(T, list, l, bxy);
  const size_t q = (size_t)c.k * T.B * T.B + c.j * T.B + c.i;
  T.b[q] = T.r[q] + apply_at(T, T.x, c, false);
}

// refined blocks of the list: field = mean of the 2x2 children cells
__global__ void restrict_kernel(TreeDev T, const int* list, const int* child, int which) {
  const int k = list[blockIdx.x], B = T.B;
  const int i = threadIdx.x % B, j = threadIdx.x / B;
  double* F = which == 0 ? T.x : T.r;
  const int quad = (2 * i >= B ? 1 : 0) + 2 * (2 * j >= B ? 1 : 0);
  const int ck = child[4 * k + quad];
  const int ci = (2 * i) % B, cj = (2 * j) % B;
  const double* cf = F + (size_t)ck * B * B;
  double s = cf[cj * B + ci];
  s = s + cf[cj * B + ci + 1];
  s = s + cf[(cj + 1) * B + ci];
  s = s + cf[(cj + 1) * B + ci + 1];
  F[(size_t)k * B * B + j * B + i] = 0.25 * s;
}

__global__ void save_kernel(TreeDev T, const int* list) {
  const size_t q = (size_t)list[blockIdx.x] * T.B * T.B + threadIdx.x;
  T.xold[q] = T.x[q];
}

// e = x - xold at level-l cell (Ic, Jc), or ep where the level has no block there
__device__ __forceinline__ double corr(const TreeDev& T, int l, int Ic, int Jc, double ep) {
  int off;
  const int k = blk_at(T, l, Ic, Jc, &off);
  if (k < 0) return ep;
  const size_t q = (size_t)k * T.B * T.B + off;
  return T.x[q] - T.xold[q];
}

// blocks of level l (children of refined level-(l-1) blocks): x += bilinear(e) of level l-1
__global__ void prolong_kernel(TreeDev T, const int* list, const int* bxy, int l) {
  const Cell c = cell_of_thread(T, list, l, bxy);
  const int Ic = c.I >> 1, Jc = c.J >> 1;
  const int sx = (c.I & 1) ? 1 : -1, sy = (c.J & 1) ? 1 : -1;
  const double e0 = corr(T, l - 1, Ic, Jc, 0.0);
  double acc = 0.5625 * e0;
  acc = acc + 0.1875 * corr(T, l - 1, Ic + sx, Jc, e0);
  acc = acc + 0.1875 * corr(T, l - 1, Ic, Jc + sy, e0);
  acc = acc + 0.0625 * corr(T, l - 1, Ic + sx, Jc + sy, e0);
  const size_t q = (size_t)c.k * T.B * T.B + c.j * T.B + c.i;
  T.x[q] = T.x[q] + acc;
}

// level 1 <-> a uniform (nx B) x (ny B) array: dir 0 gathers x and b, dir 1 scatters x + e
__global__ void base_copy_kernel(TreeDev T, const int* list, const int* bxy, double* ux, double* ub, const double* ue,
                                 int dir) {
  const int k = list[blockIdx.x], B = T.B;
  const int i = threadIdx.x % B, j = threadIdx.x / B;
  const size_t g = (size_t)(bxy[2 * k + 1] * B + j) * (T.nx[1] * B) + bxy[2 * k] * B + i;
  const size_t q = (size_t)k * B * B + j * B + i;
  if (dir == 0) {
    ux[g] = T.x[q];
    ub[g] = T.b[q];
  } else {
    T.x[q] = ux[g] + ue[g];
  }
}

// base level in correction form: r = b - (lambda x - lap x) on the uniform periodic n x n
// array (neighbours x-, x+, y-, y+), written over b; e = 0
__global__ void base_residual_kernel(const double* __restrict__ ux, double* __restrict__ ub, double* __restrict__ ue,
                                     int n, double lam, double ih2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const size_t g = (size_t)j * n + i;
  const double x0 = ux[g];
  double s = ux[(size_t)j * n + (i == 0 ? n - 1 : i - 1)];
  s = s + ux[(size_t)j * n + (i == n - 1 ? 0 : i + 1)];
  s = s + ux[(size_t)(j == 0 ? n - 1 : j - 1) * n + i];
  s = s + ux[(size_t)(j == n - 1 ? 0 : j + 1) * n + i];
  ub[g] = ub[g] - (lam * x0 - (s - 4.0 * x0) * ih2);
  ue[g] = 0.0;
}

// max |bo - A x| (composite) and max |bo| over the leaves of the list, as bit patterns
__global__ void resmax_kernel(TreeDev T, const int* list, const int* bxy, int l, unsigned long long* out) {
  const Cell c = cell_of_thread(T, list, l, bxy);
  const size_t q = (size_t)c.k * T.B * T.B + c.j * T.B + c.i;
  const double r = fabs(T.bo[q] - apply_at(T, T.x, c, true));
  const double bm = fabs(T.bo[q]);
  // NaN compares as the largest bit pattern, so it cannot pass the convergence test
  unsigned long long rb = isnan(r) ? 0x7ff8000000000000ull : (unsigned long long)__double_as_longlong(r);
  atomicMax(&out[0], rb);
  atomicMax(&out[1], (unsigned long long)__double_as_longlong(bm));
}

__global__ void apply_kernel(TreeDev T, const int* list, const int* bxy, int l, double* out, const int* slot) {
  const Cell c = cell_of_thread(T, list, l, bxy);
  out[(size_t)slot[c.k] * T.B * T.B + c.j * T.B + c.i] = apply_at(T, T.x, c, true);
}

// leaf data [leaf][B*B] <-> block arrays: dir 0 loads x and bo (b too), dir 1 stores x
__global__ void leaf_copy_kernel(TreeDev T, const int* leaf_blk, const double* bsrc, double* xio, int dir) {
  const int s = blockIdx.x, k = leaf_blk[s], n = T.B * T.B;
  const size_t q = (size_t)k * n + threadIdx.x, p = (size_t)s * n + threadIdx.x;
  if (dir == 0) {
    T.x[q] = xio[p];
    if (bsrc) {
      T.bo[q] = bsrc[p];
      T.b[q] = bsrc[p];
    }
  } else {
    xio[p] = T.x[q];
  }
}

// Convergence test of the device-side solve loop: max|r| and max|b| come as bit patterns in
// red[0..1].  ctr[0] counts V-cycles and ctr[1] the base level's V-cycles (added from
// base_cyc after each cycle); res[0..1] keep the last max|r| and max|b|.  The loop goes on
// while max|r| > rtol max|b| and fewer than max_cycles cycles ran (a NaN residual stops it).
__global__ void tree_check_kernel(const unsigned long long* red, int* ctr, double* res, const int* base_cyc,
                                  double rtol, int max_cycles, int first, cudaGraphConditionalHandle hc) {
  const double rm = __longlong_as_double((long long)red[0]), bm = __longlong_as_double((long long)red[1]);
  if (first) {
    ctr[0] = 0;
    ctr[1] = 0;
  } else {
    ctr[0] += 1;
    ctr[1] += base_cyc[0];
  }
  res[0] = rm;
  res[1] = bm;
  cudaGraphSetConditional(hc, (rm > rtol * bm && ctr[0] < max_cycles) ? 1u : 0u);
}

// composite Laplacian (sum of neighbours - 4 x) / h^2 of the leaves of the list, into
// leaf-major out[slot]
__global__ void lap_kernel(TreeDev T, const int* list, const int* bxy, int l, double* out, const int* slot) {
  const Cell c = cell_of_thread(T, list, l, bxy);
  const double x0 = T.x[(size_t)c.k * T.B * T.B + c.j * T.B + c.i];
  out[(size_t)slot[c.k] * T.B * T.B + c.j * T.B + c.i] = (nbr_sum(T, T.x, c, x0, true) - 4.0 * x0) * T.ih2[l];
}

// Gray-Scott on leaf-major arrays (Eq. (gray-scott)), IMEX stage 1 (Eq. (imex)):
// b = lambda (w + dt F0 + dt/2 D lap w), Fn = F0 + D lap w, per species
struct RdtArgs {
  double Du, Dv, F, k, dt, lam_u, lam_v;
  double* u;
  double* v;
  const double* lu;
  const double* lv;
  double* bu;
  double* bv;
  double* Fn;  // [2][n]
  double* xu;  // solutions w* (guess w_n)
  double* xv;
  long long n;
};

__global__ void rdt_rhs_kernel(RdtArgs A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const double u = A.u[i], v = A.v[i];
  const double uvv = (u * v) * v;
  const double fu = -uvv + A.F * (1.0 - u);
  const double fv = uvv - (A.F + A.k) * v;
  const double gu = (u + A.dt * fu) + ((0.5 * A.dt) * A.Du) * A.lu[i];
  const double gv = (v + A.dt * fv) + ((0.5 * A.dt) * A.Dv) * A.lv[i];
  A.bu[i] = A.lam_u * gu;
  A.bv[i] = A.lam_v * gv;
  A.Fn[i] = fu + A.Du * A.lu[i];
  A.Fn[A.n + i] = fv + A.Dv * A.lv[i];
  A.xu[i] = u;
  A.xv[i] = v;
}

// stage 2: w = w + dt/2 [F(w_n) + F(w*)], lu, lv the Laplacians of w*
__global__ void rdt_finish_kernel(RdtArgs A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const double us = A.xu[i], vs = A.xv[i];
  const double uvv = (us * vs) * vs;
  const double fus = -uvv + A.F * (1.0 - us);
  const double fvs = uvv - (A.F + A.k) * vs;
  A.u[i] = A.u[i] + (0.5 * A.dt) * (A.Fn[i] + (fus + A.Du * A.lu[i]));
  A.v[i] = A.v[i] + (0.5 * A.dt) * (A.Fn[A.n + i] + (fvs + A.Dv * A.lv[i]));
}

// ------------------------------------------------------------------ regrid --
// Lohner estimator of the field in x over the leaves of the list (level l): per cell and
// direction, (q+ - 2 q0 + q-)^2 over (|q+ - q0| + |q0 - q-| + eps (|q+| + 2|q0| + |q-|))^2,
// neighbours by the level operator, E = sqrt(num / den) (0 where den = 0); the max over the
// leaf's cells goes to err[slot] as a bit pattern (non-negative doubles order like their bits)
__global__ void lohner_kernel(TreeDev T, const int* list, const int* bxy, int l, const int* slot, double eps,
                              unsigned long long* err) {
  __shared__ unsigned long long wmax[8];
  const Cell c = cell_of_thread(T, list, l, bxy);
  const double q0 = T.x[(size_t)c.k * T.B * T.B + c.j * T.B + c.i];
  double num = 0.0, den = 0.0;
  for (int d = 0; d < 2; ++d) {
    const double qm = d == 0 ? nbr(T, T.x, l, c.I - 1, c.J, 0, -1, q0, false) : nbr(T, T.x, l, c.I, c.J - 1, 1, -1, q0, false);
    const double qp = d == 0 ? nbr(T, T.x, l, c.I + 1, c.J, 0, +1, q0, false) : nbr(T, T.x, l, c.I, c.J + 1, 1, +1, q0, false);
    const double d2 = qp - 2.0 * q0 + qm;
    const double d1 = fabs(qp - q0) + fabs(q0 - qm) + eps * (fabs(qp) + 2.0 * fabs(q0) + fabs(qm));
    num = num + d2 * d2;
    den = den + d1 * d1;
  }
  const double e = den > 0.0 ? sqrt(num / den) : 0.0;
  unsigned long long m = (unsigned long long)__double_as_longlong(e);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wmax[w] > m ? wmax[w] : m;
    atomicMax(&err[slot[c.k]], m);
  }
}

__device__ __forceinline__ double minmod2(double a, double b) {
  return a * b > 0.0 ? (fabs(a) < fabs(b) ? a : b) : 0.0;
}

// How new leaf n of a regrid gets its values from the old tree (block indices of the old tree)
struct Xfer {
  int kind;  // 0: the same leaf, 1: a child of refined leaf src[0], 2: the parent of leaves src[0..3]
  int l, x, y;
  int src[4];
};

// field of the new leaf blockIdx.x (old tree's x holds the field, refined blocks restricted)
__global__ void transfer_kernel(TreeDev T, const Xfer* __restrict__ xf, double* __restrict__ out) {
  const Xfer X = xf[blockIdx.x];
  const int B = T.B, i = threadIdx.x % B, j = threadIdx.x / B;
  double* dst = out + (size_t)blockIdx.x * B * B + j * B + i;
  if (X.kind == 0) {
    *dst = T.x[(size_t)X.src[0] * B * B + j * B + i];
  } else if (X.kind == 1) {
    const int I = X.x * B + i, J = X.y * B + j, Ic = I >> 1, Jc = J >> 1, pl = X.l - 1;
    const int pk = X.src[0];
    const int pi = Ic - (X.x >> 1) * B, pj = Jc - (X.y >> 1) * B;
    const double q = T.x[(size_t)pk * B * B + pj * B + pi];
    const double qxm = nbr(T, T.x, pl, Ic - 1, Jc, 0, -1, q, false);
    const double qxp = nbr(T, T.x, pl, Ic + 1, Jc, 0, +1, q, false);
    const double qym = nbr(T, T.x, pl, Ic, Jc - 1, 1, -1, q, false);
    const double qyp = nbr(T, T.x, pl, Ic, Jc + 1, 1, +1, q, false);
    const double sx = (I & 1) ? 0.25 : -0.25, sy = (J & 1) ? 0.25 : -0.25;
    *dst = (q + sx * minmod2(q - qxm, qxp - q)) + sy * minmod2(q - qym, qyp - q);
  } else {
    const int quad = (2 * i >= B ? 1 : 0) + 2 * (2 * j >= B ? 1 : 0);
    const double* cf = T.x + (size_t)X.src[quad] * B * B;
    const int ci = (2 * i) % B, cj = (2 * j) % B;
    double sum = cf[cj * B + ci];
    sum = sum + cf[cj * B + ci + 1];
    sum = sum + cf[(cj + 1) * B + ci];
    sum = sum + cf[(cj + 1) * B + ci + 1];
    *dst = 0.25 * sum;
  }
}

// ------------------------------------------------------------------ host --
struct Buf {
  void* p = nullptr;
  ~Buf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t n) {
    if (p) cudaFree(p);
    p = nullptr;
    return cudaMalloc(&p, n ? n : 16);
  }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

struct Tree {
  mgt_config cfg{};
  int B = 8, lmax = 1;
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // host tree
  std::vector<int> lev, bx, by, isleaf, child;  // per block; child [4 per block]
  std::vector<std::vector<int>> bylev, parents;  // per level: all blocks, refined blocks
  std::vector<int> leaf_blk;                     // leaf order of the caller -> block
  std::map<long long, int> at;
  // device
  TreeDev T{};
  Buf d_x, d_b, d_r, d_xold, d_bo, d_leaf, d_bxy, d_child, d_leafblk, d_slot, d_lists, d_tables, d_red, d_ux, d_ub, d_ue;
  std::vector<size_t> off_all, off_par;  // offsets of the level lists inside d_lists
  mg_handle* base = nullptr;
  unsigned long long* h_red = nullptr;
  long long launches = 0, base_launches = 0;
  // device-side solve loop (one graph per pair of b, x arrays)
  cudaStream_t cstream = nullptr;
  cudaGraphExec_t sgraph = nullptr;
  const double* g_b = nullptr;
  double* g_x = nullptr;
  bool capturing = false;
  long long pre_kernels = 0, body_kernels = 0;
  Buf d_ctr, d_res, d_bin, d_xin;
  double* h_res = nullptr;  // pinned: [rm, bm]

  ~Tree() {
    if (sgraph) cudaGraphExecDestroy(sgraph);
    if (cstream) cudaStreamDestroy(cstream);
    if (h_res) cudaFreeHost(h_res);
    if (base) mg_destroy(base);
    if (h_red) cudaFreeHost(h_red);
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
  int nx(int l) const { return cfg.nbx << (l - 1); }
  int ny(int l) const { return cfg.nby << (l - 1); }
  static long long key(int l, int x, int y) { return ((long long)l << 48) | ((long long)y << 24) | x; }
  int find(int l, int x, int y) const {
    auto it = at.find(key(l, x, y));
    return it == at.end() ? -1 : it->second;
  }
  int add(int l, int x, int y) {
    int k = find(l, x, y);
    if (k >= 0) return k;
    k = (int)lev.size();
    lev.push_back(l);
    bx.push_back(x);
    by.push_back(y);
    isleaf.push_back(0);
    for (int q = 0; q < 4; ++q) child.push_back(-1);
    at[key(l, x, y)] = k;
    return k;
  }

  int build(const mgt_config* c, int nleaves, const int* level, const int* coords) {
    cfg = *c;
    B = c->B;
    if ((B != 8 && B != 16) || c->nbx < 1 || c->nbx != c->nby || !(c->L > 0) || !(c->lambda >= 0) || c->nu1 < 0 ||
        c->nu2 < 0 || c->max_cycles < 0 || !(c->rtol > 0) || !(c->base_rtol > 0) || nleaves < 1 || !level || !coords)
      return fail(AMR_ERR_INVALID_ARG, "invalid tree multigrid configuration");
    lmax = 1;
    for (int k = 0; k < nleaves; ++k) lmax = std::max(lmax, level[k]);
    if (lmax > kMaxLev) return fail(AMR_ERR_INVALID_ARG, "too many levels");
    for (int k = 0; k < nleaves; ++k) {
      int l = level[k], x = coords[2 * k], y = coords[2 * k + 1];
      if (l < 1 || x < 0 || y < 0 || x >= nx(l) || y >= ny(l) || find(l, x, y) >= 0)
        return fail(AMR_ERR_INVALID_ARG, "leaf outside the domain or repeated");
      int id = add(l, x, y);
      isleaf[id] = 1;
      leaf_blk.push_back(id);
      while (l > 1) {
        int p = add(l - 1, x >> 1, y >> 1);
        if (isleaf[p]) return fail(AMR_ERR_INVALID_ARG, "leaves overlap");
        child[4 * p + (x & 1) + 2 * (y & 1)] = find(l, x, y);
        --l;
        x >>= 1;
        y >>= 1;
      }
    }
    const int nblk = (int)lev.size();
    for (int k = 0; k < nblk; ++k)
      if (!isleaf[k])
        for (int q = 0; q < 4; ++q)
          if (child[4 * k + q] < 0) return fail(AMR_ERR_INVALID_ARG, "the leaves do not tile the domain");
    // 2:1 balance across faces and corners: every block position next to a leaf is covered by
    // a block of the leaf's level or by one of the level above it
    for (int k : leaf_blk) {
      const int l = lev[k];
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy) continue;
          const int X = (bx[k] + dx + nx(l)) % nx(l), Y = (by[k] + dy + ny(l)) % ny(l);
          if (find(l, X, Y) < 0 && (l == 1 || find(l - 1, X >> 1, Y >> 1) < 0))
            return fail(AMR_ERR_INVALID_ARG, "the tree is not 2:1 balanced");
        }
    }
    bylev.assign(lmax + 1, {});
    parents.assign(lmax + 1, {});
    for (int k = 0; k < nblk; ++k) {
      bylev[lev[k]].push_back(k);
      if (!isleaf[k]) parents[lev[k]].push_back(k);
    }
    if ((int)bylev[1].size() != c->nbx * c->nby) return fail(AMR_ERR_INVALID_ARG, "incomplete base level");
    return AMR_OK;
  }

  int setup(void* strm) {
    stream = (cudaStream_t)strm;
    if (!stream) {
      if (int rc = cuda(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking), "stream")) return rc;
      own_stream = true;
    }
    const int nblk = (int)lev.size();
    const size_t cells = (size_t)nblk * B * B;
    // level lists (all blocks, refined blocks) and tables
    std::vector<int> lists;
    off_all.assign(lmax + 1, 0);
    off_par.assign(lmax + 1, 0);
    for (int l = 1; l <= lmax; ++l) {
      off_all[l] = lists.size();
      lists.insert(lists.end(), bylev[l].begin(), bylev[l].end());
      off_par[l] = lists.size();
      lists.insert(lists.end(), parents[l].begin(), parents[l].end());
    }
    std::vector<int> tables;
    std::vector<size_t> toff(lmax + 1, 0);
    for (int l = 1; l <= lmax; ++l) {
      toff[l] = tables.size();
      std::vector<int> t((size_t)nx(l) * ny(l), -1);
      for (int k : bylev[l]) t[(size_t)by[k] * nx(l) + bx[k]] = k;
      tables.insert(tables.end(), t.begin(), t.end());
    }
    std::vector<int> bxy(2 * nblk), slot(nblk, -1);
    for (int k = 0; k < nblk; ++k) {
      bxy[2 * k] = bx[k];
      bxy[2 * k + 1] = by[k];
    }
    for (size_t s = 0; s < leaf_blk.size(); ++s) slot[leaf_blk[s]] = (int)s;
    const size_t nu = (size_t)nx(1) * B * ny(1) * B;
    int rc;
    if ((rc = cuda(d_x.alloc(cells * 8), "alloc")) || (rc = cuda(d_b.alloc(cells * 8), "alloc")) ||
        (rc = cuda(d_r.alloc(cells * 8), "alloc")) || (rc = cuda(d_xold.alloc(cells * 8), "alloc")) ||
        (rc = cuda(d_bo.alloc(cells * 8), "alloc")) || (rc = cuda(d_leaf.alloc(nblk * 4), "alloc")) ||
        (rc = cuda(d_bxy.alloc(bxy.size() * 4), "alloc")) || (rc = cuda(d_child.alloc(child.size() * 4), "alloc")) ||
        (rc = cuda(d_leafblk.alloc(leaf_blk.size() * 4), "alloc")) || (rc = cuda(d_slot.alloc(nblk * 4), "alloc")) ||
        (rc = cuda(d_lists.alloc(lists.size() * 4), "alloc")) || (rc = cuda(d_tables.alloc(tables.size() * 4), "alloc")) ||
        (rc = cuda(d_red.alloc(16), "alloc")) || (rc = cuda(d_ux.alloc(nu * 8), "alloc")) ||
        (rc = cuda(d_ub.alloc(nu * 8), "alloc")) || (rc = cuda(d_ue.alloc(nu * 8), "alloc")) ||
        (rc = cuda(cudaMallocHost(&h_red, 16), "host alloc")))
      return rc;
    // host-to-device copy of a table (empty tables copy nothing)
    auto upload = [&](void* dst, const void* src, size_t bytes) {
      return bytes ? cuda(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice), "copy table") : AMR_OK;
    };
    if ((rc = upload(d_leaf.p, isleaf.data(), (size_t)nblk * 4)) || (rc = upload(d_bxy.p, bxy.data(), bxy.size() * 4)) ||
        (rc = upload(d_child.p, child.data(), child.size() * 4)) ||
        (rc = upload(d_leafblk.p, leaf_blk.data(), leaf_blk.size() * 4)) ||
        (rc = upload(d_slot.p, slot.data(), (size_t)nblk * 4)) || (rc = upload(d_lists.p, lists.data(), lists.size() * 4)) ||
        (rc = upload(d_tables.p, tables.data(), tables.size() * 4)))
      return rc;
    for (Buf* z : {&d_x, &d_b, &d_r, &d_xold, &d_bo})
      if ((rc = cuda(cudaMemset(z->p, 0, cells * 8), "memset"))) return rc;
    T.B = B;
    T.lmax = lmax;
    T.lam = cfg.lambda;
    const double h1 = cfg.L / (double)(cfg.nbx * B);
    for (int l = 1; l <= lmax; ++l) {
      T.table[l] = d_tables.as<int>() + toff[l];
      T.nx[l] = nx(l);
      T.ny[l] = ny(l);
      const double h = h1 / (double)(1 << (l - 1));
      T.ih2[l] = 1.0 / (h * h);
    }
    T.leaf = d_leaf.as<int>();
    T.x = d_x.as<double>();
    T.b = d_b.as<double>();
    T.r = d_r.as<double>();
    T.xold = d_xold.as<double>();
    T.bo = d_bo.as<double>();
    // the base grid's uniform multigrid (periodic, side nbx B)
    const int nside = cfg.nbx * B;
    const double lamb = cfg.lambda;
    mg_config mc{};
    mc.ndim = 2;
    mc.n_inst = 1;
    mc.n_cells = &nside;
    mc.lambda = &lamb;
    mc.L = cfg.L;
    mc.nu1 = 2;
    mc.nu2 = 2;
    mc.max_cycles = 200;
    mc.rtol = cfg.base_rtol;
    mc.coarse_max = cfg.coarse_max;
    mc.precision = AMR_FP64;
    mc.stream = stream;
    mc.bc = MG_BC_PERIODIC;
    if ((rc = mg_create(&mc, &base))) return fail(rc, "base multigrid: could not create");
    return cuda(cudaDeviceSynchronize(), "setup");
  }

  const int* all(int l) const { return d_lists.as<int>() + off_all[l]; }
  const int* par(int l) const { return d_lists.as<int>() + off_par[l]; }
  unsigned nall(int l) const { return (unsigned)bylev[l].size(); }
  unsigned npar(int l) const { return (unsigned)parents[l].size(); }

  void restrict_all() {
    for (int l = lmax - 1; l >= 1; --l)
      if (npar(l)) {
        restrict_kernel<<<npar(l), B * B, 0, stream>>>(T, par(l), d_child.as<int>(), 0);
        ++launches;
      }
  }

  int base_solve() {
    const int* bxy = d_bxy.as<int>();
    double* ux = d_ux.as<double>();
    double* ub = d_ub.as<double>();
    double* ue = d_ue.as<double>();
    const int n = cfg.nbx * B;
    base_copy_kernel<<<nall(1), B * B, 0, stream>>>(T, all(1), bxy, ux, ub, ue, 0);
    base_residual_kernel<<<dim3((n + 127) / 128, n), 128, 0, stream>>>(ux, ub, ue, n, cfg.lambda, T.ih2[1]);
    launches += 2;
    if (capturing) {  // inside the graph of a device-side solve: the base solve is a nested loop
      if (int rc = mg_capture_solve(base, ub, ue, stream))
        return fail(rc, std::string("base multigrid: ") + mg_last_error(base));
      base_copy_kernel<<<nall(1), B * B, 0, stream>>>(T, all(1), bxy, ux, ub, ue, 1);
      ++launches;
      return AMR_OK;
    }
    int cyc;
    double rr;
    int rc = mg_solve(base, ub, ue, 1, &cyc, &rr);
    if (rc) return fail(rc, std::string("base multigrid: ") + mg_last_error(base));
    long long bl = 0;
    mg_kernel_launches(base, &bl);
    launches += bl - base_launches;
    base_launches = bl;
    base_copy_kernel<<<nall(1), B * B, 0, stream>>>(T, all(1), bxy, ux, ub, ue, 1);
    ++launches;
    return AMR_OK;
  }

  int vcycle(int l) {
    if (l == 1) return base_solve();
    const int* bxy = d_bxy.as<int>();
    const unsigned nt = (unsigned)(B * B);
    auto smooth = [&](int sweeps) {
      for (int s = 0; s < sweeps; ++s)
        for (int colour = 0; colour < 2; ++colour) {
          gs_kernel<<<nall(l), nt, 0, stream>>>(T, all(l), bxy, l, colour);
          ++launches;
        }
    };
    smooth(cfg.nu1);
    level_residual_kernel<<<nall(l), nt, 0, stream>>>(T, all(l), bxy, l);
    ++launches;
    if (npar(l - 1)) {
      restrict_kernel<<<npar(l - 1), nt, 0, stream>>>(T, par(l - 1), d_child.as<int>(), 0);
      ++launches;
    }
    save_kernel<<<nall(l - 1), nt, 0, stream>>>(T, all(l - 1));
    ++launches;
    if (npar(l - 1)) {
      restrict_kernel<<<npar(l - 1), nt, 0, stream>>>(T, par(l - 1), d_child.as<int>(), 1);
      ++launches;
    }
    composite_residual_kernel<<<nall(l - 1), nt, 0, stream>>>(T, all(l - 1), bxy, l - 1);
    fas_rhs_kernel<<<nall(l - 1), nt, 0, stream>>>(T, all(l - 1), bxy, l - 1);
    launches += 2;
    if (int rc = vcycle(l - 1)) return rc;
    prolong_kernel<<<nall(l), nt, 0, stream>>>(T, all(l), bxy, l);
    ++launches;
    smooth(cfg.nu2);
    return cuda(cudaGetLastError(), "tree V-cycle");
  }

  // enqueue: refined blocks restricted, then max |b - A x| (composite) and max |b| over the
  // leaves into d_red (bit patterns)
  int enqueue_resmax() {
    restrict_all();
    if (int rc = cuda(cudaMemsetAsync(d_red.p, 0, 16, stream), "memset")) return rc;
    const int* bxy = d_bxy.as<int>();
    for (int l = 1; l <= lmax; ++l)
      if (!leafl[l].empty()) {
        resmax_kernel<<<(unsigned)leafl[l].size(), B * B, 0, stream>>>(T, d_leafl.as<int>() + leafl_off[l], bxy, l,
                                                                        d_red.as<unsigned long long>());
        ++launches;
      }
    return AMR_OK;
  }

  // Enqueue one whole solve of device leaf-major b, x onto `stream` while it is being
  // captured: load, the first residual and check, a conditional while node whose body
  // (captured on cstream) is a V-cycle (the base solve a nested device-side loop), the
  // residual and the check, then the store of x.
  int capture_solve(const double* db, double* dx) {
    int rc;
    if (!cstream && (rc = cuda(cudaStreamCreateWithFlags(&cstream, cudaStreamNonBlocking), "stream"))) return rc;
    const unsigned nl = (unsigned)leaf_blk.size(), nt = (unsigned)(B * B);
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    if ((rc = cuda(cudaStreamGetCaptureInfo(stream, &st, nullptr, &g), "capture info"))) return rc;
    cudaGraphConditionalHandle hc;
    if ((rc = cuda(cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault), "conditional"))) return rc;
    const long long start = launches;  // captured kernels are counted when a solve runs
    long long l0 = launches;
    leaf_copy_kernel<<<nl, nt, 0, stream>>>(T, d_leafblk.as<int>(), db, dx, 0);
    ++launches;
    if ((rc = enqueue_resmax())) return rc;
    tree_check_kernel<<<1, 1, 0, stream>>>(d_red.as<unsigned long long>(), d_ctr.as<int>(), d_res.as<double>(),
                                           mg_device_cycles(base), cfg.rtol, cfg.max_cycles, 1, hc);
    ++launches;
    pre_kernels = launches - l0 + 1;  // and the final store
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if ((rc = cuda(cudaStreamGetCaptureInfo(stream, &st, nullptr, &g, &deps, nullptr, &ndeps), "capture info")))
      return rc;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((rc = cuda(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp), "conditional node"))) return rc;
    if ((rc = cuda(cudaStreamUpdateCaptureDependencies(stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
                   "capture dependencies")))
      return rc;
    if ((rc = cuda(cudaStreamBeginCaptureToGraph(cstream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeThreadLocal),
                   "body capture")))
      return rc;
    cudaStream_t outer = stream;
    stream = cstream;
    capturing = true;
    l0 = launches;
    rc = vcycle(lmax);
    if (!rc) rc = enqueue_resmax();
    if (!rc) {
      tree_check_kernel<<<1, 1, 0, stream>>>(d_red.as<unsigned long long>(), d_ctr.as<int>(), d_res.as<double>(),
                                             mg_device_cycles(base), cfg.rtol, cfg.max_cycles, 0, hc);
      ++launches;
    }
    body_kernels = launches - l0 + 4;  // and the base solve's prelude
    capturing = false;
    stream = outer;
    cudaGraph_t got = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cstream, &got);
    if (rc) return rc;
    if ((rc = cuda(ec, "end body capture"))) return rc;
    leaf_copy_kernel<<<nl, nt, 0, stream>>>(T, d_leafblk.as<int>(), nullptr, dx, 1);
    launches = start;
    return cuda(cudaGetLastError(), "solve capture");
  }

  // one device-side solve of device arrays db, dx (the graph is rebuilt when they change)
  int solve_graph(const double* db, double* dx, int* cycles, double* rmo, double* bmo) {
    int rc;
    if (!sgraph || db != g_b || dx != g_x) {
      if (sgraph) cudaGraphExecDestroy(sgraph);
      sgraph = nullptr;
      if (!d_ctr.p && ((rc = cuda(d_ctr.alloc(16), "alloc")) || (rc = cuda(d_res.alloc(16), "alloc")) ||
                       (rc = cuda(cudaMallocHost(&h_res, 4 * sizeof(double)), "host alloc"))))
        return rc;
      cudaGraph_t g;
      if ((rc = cuda(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "capture"))) return rc;
      int crc = capture_solve(db, dx);
      cudaError_t ec = cudaStreamEndCapture(stream, &g);
      if (crc) {
        if (ec == cudaSuccess) cudaGraphDestroy(g);
        return crc;
      }
      if ((rc = cuda(ec, "end capture"))) return rc;
      rc = cuda(cudaGraphInstantiate(&sgraph, g, 0), "instantiate");
      cudaGraphDestroy(g);
      if (rc) return rc;
      g_b = db;
      g_x = dx;
    }
    if ((rc = cuda(cudaGraphLaunch(sgraph, stream), "solve graph"))) return rc;
    int ctr[2];
    if ((rc = cuda(cudaMemcpyAsync(h_res, d_res.p, 16, cudaMemcpyDeviceToHost, stream), "copy")) ||
        (rc = cuda(cudaMemcpyAsync(ctr, d_ctr.p, 8, cudaMemcpyDeviceToHost, stream), "copy")) ||
        (rc = cuda(cudaStreamSynchronize(stream), "sync")))
      return rc;
    *cycles = ctr[0];
    *rmo = h_res[0];
    *bmo = h_res[1];
    launches += pre_kernels + (long long)ctr[0] * body_kernels + (long long)ctr[1] * mg_loop_kernels(base);
    return AMR_OK;
  }

  // composite residual max and max |b| over the leaves (refined blocks restricted first)
  int resmax(double* rm, double* bm) {
    restrict_all();
    if (int rc = cuda(cudaMemsetAsync(d_red.p, 0, 16, stream), "memset")) return rc;
    const int* bxy = d_bxy.as<int>();
    for (int l = 1; l <= lmax; ++l) {
      // leaves of level l only: the kernel runs on all blocks of the level and skips none, so
      // pass the leaf blocks through their own list
      if (!leafl[l].empty()) {
        resmax_kernel<<<(unsigned)leafl[l].size(), B * B, 0, stream>>>(T, d_leafl.as<int>() + leafl_off[l], bxy, l,
                                                                        d_red.as<unsigned long long>());
        ++launches;
      }
    }
    if (int rc = cuda(cudaMemcpyAsync(h_red, d_red.p, 16, cudaMemcpyDeviceToHost, stream), "copy")) return rc;
    if (int rc = cuda(cudaStreamSynchronize(stream), "sync")) return rc;
    double a, b;
    std::memcpy(&a, &h_red[0], 8);
    std::memcpy(&b, &h_red[1], 8);
    *rm = a;
    *bm = b;
    return AMR_OK;
  }

  std::vector<std::vector<int>> leafl;
  std::vector<size_t> leafl_off;
  Buf d_leafl;

  // solve with device leaf-major b and x (x: guess in, solution out)
  int solve_dev(const double* db, double* dx, int fixed_cycles, int* cycles, double* rmo, double* bmo) {
    const unsigned nl = (unsigned)leaf_blk.size(), nt = (unsigned)(B * B);
    leaf_copy_kernel<<<nl, nt, 0, stream>>>(T, d_leafblk.as<int>(), db, dx, 0);
    ++launches;
    double rm, bm;
    int rc;
    if ((rc = resmax(&rm, &bm))) return rc;
    int cyc = 0;
    while (fixed_cycles > 0 ? cyc < fixed_cycles : (rm > cfg.rtol * bm && cyc < cfg.max_cycles)) {
      if ((rc = vcycle(lmax))) return rc;
      ++cyc;
      if ((rc = resmax(&rm, &bm))) return rc;
    }
    leaf_copy_kernel<<<nl, nt, 0, stream>>>(T, d_leafblk.as<int>(), nullptr, dx, 1);
    ++launches;
    *cycles = cyc;
    *rmo = rm;
    *bmo = bm;
    return cuda(cudaGetLastError(), "tree solve");
  }

  // composite Laplacian of device leaf-major w into lap
  int lap_leaves(const double* w, double* lap) {
    const unsigned nt = (unsigned)(B * B);
    leaf_copy_kernel<<<(unsigned)leaf_blk.size(), nt, 0, stream>>>(T, d_leafblk.as<int>(), nullptr,
                                                                  const_cast<double*>(w), 0);
    ++launches;
    restrict_all();
    for (int l = 1; l <= lmax; ++l)
      if (!leafl[l].empty()) {
        lap_kernel<<<(unsigned)leafl[l].size(), nt, 0, stream>>>(T, d_leafl.as<int>() + leafl_off[l], d_bxy.as<int>(),
                                                                 l, lap, d_slot.as<int>());
        ++launches;
      }
    return cuda(cudaGetLastError(), "laplacian");
  }

  int setup_leaf_lists() {
    leafl.assign(lmax + 1, {});
    for (int k : leaf_blk) leafl[lev[k]].push_back(k);
    std::vector<int> flat;
    leafl_off.assign(lmax + 1, 0);
    for (int l = 1; l <= lmax; ++l) {
      leafl_off[l] = flat.size();
      flat.insert(flat.end(), leafl[l].begin(), leafl[l].end());
    }
    if (int rc = cuda(d_leafl.alloc(flat.size() * 4), "alloc")) return rc;
    return cuda(cudaMemcpy(d_leafl.p, flat.data(), flat.size() * 4, cudaMemcpyHostToDevice), "copy");
  }
};

}  // namespace mgtree

using namespace mgtree;

struct mgt_handle {
  Tree t;
};

extern "C" {

int mgt_create(const mgt_config* cfg, int nleaves, const int* level, const int* coords, mgt_handle** out) {
  if (!cfg || !out) return AMR_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<mgt_handle> h(new mgt_handle());
  int rc = h->t.build(cfg, nleaves, level, coords);
  if (!rc) rc = h->t.setup(cfg->stream);
  if (!rc) rc = h->t.setup_leaf_lists();
  if (rc) return rc;
  *out = h.release();
  return AMR_OK;
}

int mgt_destroy(mgt_handle* h) {
  if (!h) return AMR_ERR_INVALID_ARG;
  delete h;
  return AMR_OK;
}

const char* mgt_last_error(const mgt_handle* h) { return h ? h->t.err.c_str() : "null handle"; }

int mgt_num_leaves(const mgt_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = (long long)h->t.leaf_blk.size();
  return AMR_OK;
}

int mgt_solve(mgt_handle* h, const double* b, double* x, int on_device, int fixed_cycles, int* cycles,
              double* relres) {
  if (!h || !b || !x || fixed_cycles < 0) return AMR_ERR_INVALID_ARG;
  Tree& t = h->t;
  const size_t n = t.leaf_blk.size() * (size_t)t.B * t.B;
  double* db = const_cast<double*>(b);
  double* dx = x;
  Buf hb, hx;
  int rc;
  if (!on_device) {  // stage host arrays through device buffers
    if ((rc = t.cuda(hb.alloc(n * 8), "alloc")) || (rc = t.cuda(hx.alloc(n * 8), "alloc"))) return rc;
    cudaMemcpyAsync(hb.p, b, n * 8, cudaMemcpyHostToDevice, t.stream);
    cudaMemcpyAsync(hx.p, x, n * 8, cudaMemcpyHostToDevice, t.stream);
    db = hb.as<double>();
    dx = hx.as<double>();
  }
  double rm, bm;
  int cyc;
  if (fixed_cycles > 0) {  // a fixed number of cycles: the host-driven loop
    if ((rc = t.solve_dev(db, dx, fixed_cycles, &cyc, &rm, &bm))) return rc;
  } else {  // to rtol: the graph with the device-side loop, on the handle's own b, x arrays
    if (!t.d_bin.p && ((rc = t.cuda(t.d_bin.alloc(n * 8), "alloc")) || (rc = t.cuda(t.d_xin.alloc(n * 8), "alloc"))))
      return rc;
    cudaMemcpyAsync(t.d_bin.p, db, n * 8, cudaMemcpyDeviceToDevice, t.stream);
    cudaMemcpyAsync(t.d_xin.p, dx, n * 8, cudaMemcpyDeviceToDevice, t.stream);
    if ((rc = t.solve_graph(t.d_bin.as<double>(), t.d_xin.as<double>(), &cyc, &rm, &bm))) return rc;
    cudaMemcpyAsync(dx, t.d_xin.p, n * 8, cudaMemcpyDeviceToDevice, t.stream);
  }
  if (!on_device) cudaMemcpyAsync(x, hx.p, n * 8, cudaMemcpyDeviceToHost, t.stream);
  if ((rc = t.cuda(cudaStreamSynchronize(t.stream), "sync"))) return rc;
  if (cycles) *cycles = cyc;
  if (relres) *relres = bm > 0 ? rm / bm : rm;
  if (fixed_cycles == 0 && !(rm <= t.cfg.rtol * bm))
    return t.fail(MG_ERR_NOT_CONVERGED, "the composite residual did not reach rtol within max_cycles");
  return AMR_OK;
}

int mgt_apply(mgt_handle* h, const double* x, double* Ax, int on_device) {
  if (!h || !x || !Ax) return AMR_ERR_INVALID_ARG;
  Tree& t = h->t;
  const size_t n = t.leaf_blk.size() * (size_t)t.B * t.B;
  Buf hx, ha;
  double* dx = const_cast<double*>(x);
  double* da = Ax;
  int rc;
  if (!on_device) {
    if ((rc = t.cuda(hx.alloc(n * 8), "alloc")) || (rc = t.cuda(ha.alloc(n * 8), "alloc"))) return rc;
    cudaMemcpyAsync(hx.p, x, n * 8, cudaMemcpyHostToDevice, t.stream);
    dx = hx.as<double>();
    da = ha.as<double>();
  }
  const unsigned nt = (unsigned)(t.B * t.B);
  leaf_copy_kernel<<<(unsigned)t.leaf_blk.size(), nt, 0, t.stream>>>(t.T, t.d_leafblk.as<int>(), nullptr, dx, 0);
  t.restrict_all();
  for (int l = 1; l <= t.lmax; ++l)
    if (!t.leafl[l].empty())
      apply_kernel<<<(unsigned)t.leafl[l].size(), nt, 0, t.stream>>>(t.T, t.d_leafl.as<int>() + t.leafl_off[l],
                                                                    t.d_bxy.as<int>(), l, da, t.d_slot.as<int>());
  if (!on_device) cudaMemcpyAsync(Ax, ha.p, n * 8, cudaMemcpyDeviceToHost, t.stream);
  return t.cuda(cudaStreamSynchronize(t.stream), "sync");
}

int mgt_kernel_launches(const mgt_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = h->t.launches;
  return AMR_OK;
}

// ---------------------------------------------------- Gray-Scott on the tree --
struct rdt_handle {
  rdt_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::unique_ptr<Tree> tu, tv;  // the same leaves, lambda 2/(dt Du) and 2/(dt Dv)
  Buf d_u, d_v, d_lu, d_lv, d_bu, d_bv, d_Fn, d_xu, d_xv;
  long long n = 0;
  std::string err;
  ~rdt_handle() {
    tu.reset();
    tv.reset();
    if (own_stream) cudaStreamDestroy(stream);
  }
  int fail(int code, const std::string& m) {
    err = m;
    return code;
  }
};

// (re)build the two trees and the state buffers of h for these leaves
static int rdt_build(rdt_handle* h, int nleaves, const int* level, const int* coords) {
  const rdt_config* cfg = &h->cfg;
  const double D[2] = {cfg->Du, cfg->Dv};
  std::unique_ptr<Tree>* t[2] = {&h->tu, &h->tv};
  for (int s = 0; s < 2; ++s) {
    mgt_config mc = cfg->mg;
    mc.lambda = 2.0 / (cfg->dt * D[s]);
    mc.stream = h->stream;
    t[s]->reset(new Tree());
    Tree& tr = **t[s];
    int rc = tr.build(&mc, nleaves, level, coords);
    if (!rc) rc = tr.setup(h->stream);
    if (!rc) rc = tr.setup_leaf_lists();
    if (rc) return h->fail(rc, tr.err);
  }
  h->n = (long long)nleaves * cfg->mg.B * cfg->mg.B;
  const size_t bytes = (size_t)h->n * 8;
  for (Buf* b : {&h->d_u, &h->d_v, &h->d_lu, &h->d_lv, &h->d_bu, &h->d_bv, &h->d_xu, &h->d_xv})
    if (b->alloc(bytes) != cudaSuccess) return h->fail(AMR_ERR_OOM, "alloc");
  if (h->d_Fn.alloc(2 * bytes) != cudaSuccess) return h->fail(AMR_ERR_OOM, "alloc");
  return AMR_OK;
}

int rdt_create(const rdt_config* cfg, int nleaves, const int* level, const int* coords, rdt_handle** out) {
  if (!cfg || !out || !(cfg->dt > 0) || !(cfg->Du > 0) || !(cfg->Dv > 0)) return AMR_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<rdt_handle> h(new rdt_handle());
  h->cfg = *cfg;
  h->stream = (cudaStream_t)cfg->mg.stream;
  if (!h->stream) {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return AMR_ERR_CUDA;
    h->own_stream = true;
  }
  if (int rc = rdt_build(h.get(), nleaves, level, coords)) return rc;
  *out = h.release();
  return AMR_OK;
}

int rdt_destroy(rdt_handle* h) {
  if (!h) return AMR_ERR_INVALID_ARG;
  delete h;
  return AMR_OK;
}

const char* rdt_last_error(const rdt_handle* h) {
  if (!h) return "null handle";
  if (!h->err.empty()) return h->err.c_str();
  if (h->tu && !h->tu->err.empty()) return h->tu->err.c_str();
  return h->tv ? h->tv->err.c_str() : "";
}

int rdt_set_state(rdt_handle* h, const double* u, const double* v, int on_device) {
  if (!h || !u || !v) return AMR_ERR_INVALID_ARG;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(h->d_u.p, u, h->n * 8, k, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->d_v.p, v, h->n * 8, k, h->stream) != cudaSuccess)
    return AMR_ERR_CUDA;
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? AMR_OK : AMR_ERR_CUDA;
}

int rdt_read_state(rdt_handle* h, double* u, double* v, int on_device) {
  if (!h || !u || !v) return AMR_ERR_INVALID_ARG;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (cudaMemcpyAsync(u, h->d_u.p, h->n * 8, k, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(v, h->d_v.p, h->n * 8, k, h->stream) != cudaSuccess)
    return AMR_ERR_CUDA;
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? AMR_OK : AMR_ERR_CUDA;
}

// nsteps IMEX steps: composite Laplacians, right-hand sides, the two tree solves, finish
int rdt_step(rdt_handle* h, int nsteps, int* cycles) {
  if (!h || nsteps < 0) return AMR_ERR_INVALID_ARG;
  Tree& tu = *h->tu;
  Tree& tv = *h->tv;
  RdtArgs A{};
  A.Du = h->cfg.Du;
  A.Dv = h->cfg.Dv;
  A.F = h->cfg.F;
  A.k = h->cfg.k;
  A.dt = h->cfg.dt;
  A.lam_u = tu.cfg.lambda;
  A.lam_v = tv.cfg.lambda;
  A.u = h->d_u.as<double>();
  A.v = h->d_v.as<double>();
  A.lu = h->d_lu.as<double>();
  A.lv = h->d_lv.as<double>();
  A.bu = h->d_bu.as<double>();
  A.bv = h->d_bv.as<double>();
  A.Fn = h->d_Fn.as<double>();
  A.xu = h->d_xu.as<double>();
  A.xv = h->d_xv.as<double>();
  A.n = h->n;
  const unsigned nb = (unsigned)((h->n + 255) / 256);
  for (int s = 0; s < nsteps; ++s) {
    int rc;
    if ((rc = tu.lap_leaves(A.u, h->d_lu.as<double>())) || (rc = tv.lap_leaves(A.v, h->d_lv.as<double>())))
      return rc;
    rdt_rhs_kernel<<<nb, 256, 0, h->stream>>>(A);
    ++tu.launches;
    int cu, cv;
    double rm, bm, rm2, bm2;
    if ((rc = tu.solve_graph(A.bu, A.xu, &cu, &rm, &bm)) || (rc = tv.solve_graph(A.bv, A.xv, &cv, &rm2, &bm2)))
      return rc;
    if (cycles) {
      cycles[2 * s] = cu;
      cycles[2 * s + 1] = cv;
    }
    if (!(rm <= tu.cfg.rtol * bm) || !(rm2 <= tv.cfg.rtol * bm2))
      return h->fail(MG_ERR_NOT_CONVERGED, "a tree solve did not reach rtol within max_cycles");
    if ((rc = tu.lap_leaves(A.xu, h->d_lu.as<double>())) || (rc = tv.lap_leaves(A.xv, h->d_lv.as<double>())))
      return rc;
    rdt_finish_kernel<<<nb, 256, 0, h->stream>>>(A);
    ++tu.launches;
    if (cudaGetLastError() != cudaSuccess) return h->fail(AMR_ERR_CUDA, "launch");
  }
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? AMR_OK : AMR_ERR_CUDA;
}

int rdt_num_leaves(const rdt_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = (long long)h->tu->leaf_blk.size();
  return AMR_OK;
}

int rdt_leaves(const rdt_handle* h, int* level, int* coords, long long cap) {
  if (!h || !level || !coords) return AMR_ERR_INVALID_ARG;
  const Tree& t = *h->tu;
  if (cap < (long long)t.leaf_blk.size()) return AMR_ERR_INVALID_ARG;
  for (size_t s = 0; s < t.leaf_blk.size(); ++s) {
    const int k = t.leaf_blk[s];
    level[s] = t.lev[k];
    coords[2 * s] = t.bx[k];
    coords[2 * s + 1] = t.by[k];
  }
  return AMR_OK;
}

namespace {
struct LeafId {
  int l, x, y;
};
long long leaf_key(int l, int x, int y) { return ((long long)l << 48) | ((long long)y << 24) | x; }
// do the closed boxes of two blocks meet (periodic images included)?  Box edges in units of a
// level-lmax block.
bool boxes_meet(const LeafId& a, const LeafId& b, int nbx, int nby, int lmax) {
  const long long n[2] = {(long long)nbx << (lmax - 1), (long long)nby << (lmax - 1)};
  const long long sa = 1LL << (lmax - a.l), sb = 1LL << (lmax - b.l);
  const long long a0[2] = {a.x * sa, a.y * sa}, b0[2] = {b.x * sb, b.y * sb};
  for (int d = 0; d < 2; ++d) {
    bool hit = false;
    for (int img = -1; img <= 1 && !hit; ++img) {
      const long long off = img * n[d];
      hit = a0[d] <= b0[d] + off + sb && b0[d] + off <= a0[d] + sa;
    }
    if (!hit) return false;
  }
  return true;
}
unsigned long long zorder(const LeafId& k, int lmax) {
  unsigned long long x = (unsigned long long)k.x << (lmax - k.l), y = (unsigned long long)k.y << (lmax - k.l), z = 0;
  for (int b = 0; b < 24; ++b) z |= (((x >> b) & 1ull) << (2 * b)) | (((y >> b) & 1ull) << (2 * b + 1));
  return z;
}
}  // namespace

// Regrid: Lohner estimator of u on the GPU, the new tree on the host (refine above
// refine_tol up to max_level; coarsen sibling groups below coarsen_frac refine_tol; 2:1
// balance over faces and corners), the fields moved on the GPU (copy, minmod-sloped
// prolongation, mean restriction), then the trees rebuilt for the new leaves (Morton order).
int rdt_regrid(rdt_handle* h, double refine_tol, double coarsen_frac, double eps, int max_level, double* err_out,
               long long* nleaves_out) {
  if (!h || !(refine_tol > 0) || !(coarsen_frac >= 0) || max_level < 1 || max_level > kMaxLev)
    return AMR_ERR_INVALID_ARG;
  Tree& tu = *h->tu;
  Tree& tv = *h->tv;
  const int nl = (int)tu.leaf_blk.size(), B = tu.B, nt = B * B;
  Buf d_err;
  if (d_err.alloc((size_t)nl * 8) != cudaSuccess) return h->fail(AMR_ERR_OOM, "alloc");
  cudaMemsetAsync(d_err.p, 0, (size_t)nl * 8, h->stream);
  // fields into the old trees' x (refined blocks restricted); the estimator on u
  Tree* trees[2] = {&tu, &tv};
  const double* fields[2] = {h->d_u.as<double>(), h->d_v.as<double>()};
  long long extra = 2;  // the two transfers below
  for (int f = 0; f < 2; ++f) {
    Tree& t = *trees[f];
    leaf_copy_kernel<<<(unsigned)nl, nt, 0, h->stream>>>(t.T, t.d_leafblk.as<int>(), nullptr,
                                                        const_cast<double*>(fields[f]), 0);
    ++extra;
    t.restrict_all();
    for (int l = 1; l <= t.lmax && f == 0; ++l)
      if (!t.leafl[l].empty()) {
        lohner_kernel<<<(unsigned)t.leafl[l].size(), nt, 0, h->stream>>>(t.T, t.d_leafl.as<int>() + t.leafl_off[l],
                                                                        t.d_bxy.as<int>(), l, t.d_slot.as<int>(), eps,
                                                                        d_err.as<unsigned long long>());
        ++extra;
      }
  }
  std::vector<unsigned long long> eb(nl);
  if (cudaMemcpyAsync(eb.data(), d_err.p, (size_t)nl * 8, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return h->fail(AMR_ERR_CUDA, "estimator");
  std::vector<double> E(nl);
  for (int k = 0; k < nl; ++k) std::memcpy(&E[k], &eb[k], 8);
  if (err_out) std::memcpy(err_out, E.data(), (size_t)nl * 8);
  // the new tree
  std::vector<LeafId> old(nl);
  std::unordered_map<long long, int> where;  // old leaf -> its position in the caller's order
  for (int k = 0; k < nl; ++k) {
    const int b = tu.leaf_blk[k];
    old[k] = {tu.lev[b], tu.bx[b], tu.by[b]};
    where[leaf_key(old[k].l, old[k].x, old[k].y)] = k;
  }
  const int lmax = std::max(max_level, tu.lmax), nbx = h->cfg.mg.nbx, nby = h->cfg.mg.nby;
  std::vector<char> ref(nl);
  for (int k = 0; k < nl; ++k) ref[k] = E[k] > refine_tol && old[k].l < max_level;
  bool grew = true;
  while (grew) {  // a refined leaf's coarser neighbours are refined too
    grew = false;
    for (int a = 0; a < nl; ++a)
      if (ref[a])
        for (int b = 0; b < nl; ++b)
          if (!ref[b] && old[b].l < old[a].l && boxes_meet(old[a], old[b], nbx, nby, lmax)) {
            ref[b] = 1;
            grew = true;
          }
  }
  std::vector<LeafId> after;  // the tree once the refinements are applied
  for (int k = 0; k < nl; ++k) {
    if (!ref[k]) {
      after.push_back(old[k]);
    } else {
      for (int q = 0; q < 4; ++q) after.push_back({old[k].l + 1, 2 * old[k].x + (q & 1), 2 * old[k].y + (q >> 1)});
    }
  }
  std::unordered_map<long long, int> quiet;  // parent -> number of its children that may coarsen
  for (int k = 0; k < nl; ++k)
    if (old[k].l > 1 && !ref[k] && E[k] < coarsen_frac * refine_tol) ++quiet[leaf_key(old[k].l - 1, old[k].x >> 1, old[k].y >> 1)];
  std::unordered_map<long long, char> merge;  // parents that replace their four children
  for (const auto& kv : quiet) {
    if (kv.second != 4) continue;
    const LeafId p{(int)(kv.first >> 48), (int)(kv.first & 0xffffff), (int)((kv.first >> 24) & 0xffffff)};
    bool ok = true;
    for (const LeafId& n : after)
      if (n.l > p.l + 1 && boxes_meet(p, n, nbx, nby, lmax)) {
        ok = false;
        break;
      }
    if (ok) merge[kv.first] = 1;
  }
  std::vector<LeafId> nw;
  for (const LeafId& n : after)
    if (!(n.l > 1 && merge.count(leaf_key(n.l - 1, n.x >> 1, n.y >> 1)))) nw.push_back(n);
  for (const auto& kv : merge) nw.push_back({(int)(kv.first >> 48), (int)(kv.first & 0xffffff), (int)((kv.first >> 24) & 0xffffff)});
  std::sort(nw.begin(), nw.end(), [&](const LeafId& a, const LeafId& b) { return zorder(a, lmax) < zorder(b, lmax); });
  // how each new leaf gets its values (old blocks)
  const int nn = (int)nw.size();
  std::vector<Xfer> xf(nn);
  for (int n = 0; n < nn; ++n) {
    Xfer& X = xf[n];
    X.l = nw[n].l;
    X.x = nw[n].x;
    X.y = nw[n].y;
    auto it = where.find(leaf_key(X.l, X.x, X.y));
    if (it != where.end()) {
      X.kind = 0;
      X.src[0] = tu.leaf_blk[it->second];
      continue;
    }
    auto ip = X.l > 1 ? where.find(leaf_key(X.l - 1, X.x >> 1, X.y >> 1)) : where.end();
    if (ip != where.end()) {
      X.kind = 1;
      X.src[0] = tu.leaf_blk[ip->second];
      continue;
    }
    X.kind = 2;
    for (int q = 0; q < 4; ++q) {
      auto ic = where.find(leaf_key(X.l + 1, 2 * X.x + (q & 1), 2 * X.y + (q >> 1)));
      if (ic == where.end()) return h->fail(AMR_ERR_CUDA, "regrid: a merged parent lost a child");
      X.src[q] = tu.leaf_blk[ic->second];
    }
  }
  Buf d_xf, nu, nv;
  if (d_xf.alloc(nn * sizeof(Xfer)) != cudaSuccess || nu.alloc((size_t)nn * nt * 8) != cudaSuccess ||
      nv.alloc((size_t)nn * nt * 8) != cudaSuccess)
    return h->fail(AMR_ERR_OOM, "alloc");
  cudaMemcpyAsync(d_xf.p, xf.data(), nn * sizeof(Xfer), cudaMemcpyHostToDevice, h->stream);
  transfer_kernel<<<(unsigned)nn, nt, 0, h->stream>>>(tu.T, d_xf.as<Xfer>(), nu.as<double>());
  transfer_kernel<<<(unsigned)nn, nt, 0, h->stream>>>(tv.T, d_xf.as<Xfer>(), nv.as<double>());
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return h->fail(AMR_ERR_CUDA, "transfer");
  const long long kept = tu.launches + tv.launches + extra;
  // rebuild the trees for the new leaves and move the fields in
  std::vector<int> lv(nn), cd(2 * nn);
  for (int n = 0; n < nn; ++n) {
    lv[n] = nw[n].l;
    cd[2 * n] = nw[n].x;
    cd[2 * n + 1] = nw[n].y;
  }
  if (int rc = rdt_build(h, nn, lv.data(), cd.data())) return rc;
  h->tu->launches = kept;  // the count carries over
  cudaMemcpyAsync(h->d_u.p, nu.p, (size_t)nn * nt * 8, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(h->d_v.p, nv.p, (size_t)nn * nt * 8, cudaMemcpyDeviceToDevice, h->stream);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return h->fail(AMR_ERR_CUDA, "regrid");
  if (nleaves_out) *nleaves_out = nn;
  return AMR_OK;
}

int rdt_kernel_launches(const rdt_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = h->tu->launches + h->tv->launches;
  return AMR_OK;
}

}  // extern "C"
