// FP64 oracle: multigrid for the Helmholtz problem (lambda - lap_h) x = b on a 2D block
// quadtree (AMR), the multigrid Sec. 1.4 describes as AMR-compatible and Sec. 2.5.2 runs
// on a three-level Gray-Scott mesh.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// READING (the paper defers the method to mg2019 and defines none of it):
//  * Composite operator (the problem solved: one unknown per leaf cell).  Every leaf cell
//    uses the 5-point stencil of its own level, h_l = h_1 / 2^(l-1), with these neighbour
//    values.  Same-level leaf neighbour: its value.  Coarser neighbour (no block of that
//    level there; 2:1 balance across faces and corners): g = (2/3) C^ + (1/3) f0, the linear
//    interpolation along the normal between the coarse cell C (centre 3h/2 from the fine
//    cell f0) and f0, with C^ = C + s (C_t+ - C_t-) / 8 the coarse value moved to the
//    ghost's tangential position (s = -1 for the lower fine half of C, +1 for the upper).
//    Finer neighbour (a refined block of the same level): (4/3) m - (1/3) f0 with m the mean
//    of the two finer cells touching the face, so that the coarse face flux (4/3)(m - f0)
//    equals the sum of the two fine fluxes (2/3)(f - C^) (flux matching: the operator is
//    conservative).  All three rules reproduce linear data; the solution error is second
//    order on refined trees.
//  * Levels.  Level l holds every block at level l: leaves, and refined blocks that carry
//    the mean of their children.  The level operator is the 5-point stencil with the
//    same-level value of any level-l neighbour (refined or not) and the coarser-neighbour
//    rule above; it differs from the composite operator only at leaf cells next to refined
//    blocks.
//  * Full approximation scheme.  V-cycle at level l: nu1 red-black Gauss-Seidel sweeps of the
//    level operator; the level residual r; refined blocks of level l-1 get x = mean of their
//    children and r = mean of their children's residuals; leaves of level l-1 get r = their
//    composite residual; every block of level l-1 gets b = r + (A_{l-1} x) (level operator),
//    so the level-(l-1) problem corrects the composite one; the V-cycle at level l-1; the
//    children of refined blocks get the cell-centred bilinear prolongation (9/16, 3/16, 3/16,
//    1/16) of e = x - x_before at level l-1 (a level-(l-1) cell that does not exist reads the
//    parent cell's e); nu2 sweeps.  Level 1 (the base grid, uniform and periodic) is solved
//    in correction form: A e = b - A x from e = 0 by the uniform multigrid of mg.cpp until
//    the correction's residual is below base_rtol of max|b - A x| (a reduction factor, so
//    every cycle reduces the base error; a tolerance relative to b would stall the
//    iteration at that level), then x += e.  Gauss-Seidel colours by (I + J) parity of
//    global level-l cell indices; a fine cell next to a coarser block reads its own old
//    value through f0.
//  * Outer iteration: refined blocks are set to the means of their children (bottom up)
//    and V-cycles run from the finest level until the composite residual max|b - A x| over
//    the leaf cells is at most rtol max|b|, or a fixed number of cycles for parity tests.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "oracle.h"

namespace {

struct Blk {
  int lev, bx, by;
  bool leaf;
  int child[4];  // quadrant q = qx + 2 qy
  std::vector<double> x, b, r, xold;
  std::vector<double> bo;  // leaves: the right-hand side of the composite problem
};

struct Tree {
  int B = 8, nbx = 1, nby = 1, lmax = 1;
  double h1 = 1.0, lam = 1.0;
  std::vector<Blk> blk;
  std::map<long long, int> at;
  std::vector<std::vector<int>> bylev;  // index 1..lmax
  std::vector<int> leaf_blk;            // leaf k -> block

  int nx(int l) const { return nbx << (l - 1); }
  int ny(int l) const { return nby << (l - 1); }
  double h(int l) const { return h1 / (double)(1 << (l - 1)); }
  static long long key(int l, int bx, int by) { return ((long long)l << 48) | ((long long)by << 24) | bx; }
  int find(int l, int bx, int by) const {
    auto it = at.find(key(l, bx, by));
    return it == at.end() ? -1 : it->second;
  }
  static int wrap(int i, int n) { return ((i % n) + n) % n; }
  // value of field F at global level-l cell (I, J) (periodic); false if no level-l block there
  bool cell(int l, int I, int J, std::vector<double> Blk::*F, double* v) const {
    if (l < 1) return false;
    I = wrap(I, nx(l) * B);
    J = wrap(J, ny(l) * B);
    int k = find(l, I / B, J / B);
    if (k < 0) return false;
    *v = (blk[k].*F)[(size_t)(J % B) * B + (I % B)];
    return true;
  }
};

int build_tree(const orc_amg_config* c, int nleaves, const int* level, const int* coords, Tree* T) {
  T->B = c->B;
  T->nbx = c->nbx;
  T->nby = c->nby;
  T->h1 = c->L / (double)(c->nbx * c->B);
  T->lam = c->lambda;
  T->lmax = 1;
  for (int k = 0; k < nleaves; ++k) T->lmax = level[k] > T->lmax ? level[k] : T->lmax;
  T->bylev.assign(T->lmax + 1, {});
  auto add = [&](int l, int bx, int by) {
    int k = T->find(l, bx, by);
    if (k >= 0) return k;
    Blk b;
    b.lev = l;
    b.bx = bx;
    b.by = by;
    b.leaf = false;
    for (int q = 0; q < 4; ++q) b.child[q] = -1;
    size_t n = (size_t)T->B * T->B;
    b.x.assign(n, 0.0);
    b.b.assign(n, 0.0);
    b.r.assign(n, 0.0);
    b.xold.assign(n, 0.0);
    b.bo.assign(n, 0.0);
    T->blk.push_back(b);
    k = (int)T->blk.size() - 1;
    T->at[Tree::key(l, bx, by)] = k;
    T->bylev[l].push_back(k);
    return k;
  };
  for (int k = 0; k < nleaves; ++k) {
    int l = level[k], bx = coords[2 * k], by = coords[2 * k + 1];
    if (l < 1 || bx < 0 || by < 0 || bx >= T->nx(l) || by >= T->ny(l)) return -2;
    if (T->find(l, bx, by) >= 0) return -2;  // duplicate or overlapping
    int id = add(l, bx, by);
    T->blk[id].leaf = true;
    T->leaf_blk.push_back(id);
    while (l > 1) {  // ancestors
      int p = add(l - 1, bx >> 1, by >> 1);
      if (T->blk[p].leaf) return -2;
      T->blk[p].child[(bx & 1) + 2 * (by & 1)] = T->find(l, bx, by);
      --l;
      bx >>= 1;
      by >>= 1;
    }
  }
  // every refined block has four children, and the base level is complete
  for (const Blk& b : T->blk)
    if (!b.leaf)
      for (int q = 0; q < 4; ++q)
        if (b.child[q] < 0) return -2;
  if ((int)T->bylev[1].size() != T->nbx * T->nby) return -2;
  return 0;
}

// Value that the stencil of a level-l cell (value f0) reads for its neighbour cell (I, J)
// (global level-l indices, periodic) across the face normal to direction d (0 = x, 1 = y);
// side = +1 if the neighbour lies in the + direction, -1 otherwise.  `leaf`: the cell
// is evaluated with the composite operator (comp) and belongs to a leaf block.
//  * a level-l block holds (I, J) and it is a leaf, or not `leaf`: its value (the level
//    operator, which the multigrid levels smooth);
//  * it is refined and `leaf`: flux matching, (4/3) m - (1/3) f0 with m the
//    mean of the two level-(l+1) children cells that touch the face, so that the face flux
//    (4/3)(m - f0) equals the sum of the fine cells' fluxes through the face;
//  * no level-l block (the neighbour is coarser): g = (2/3) C^ + (1/3) f0 (see the header).
double nbr(const Tree& T, int l, int I, int J, int d, int side, double f0, std::vector<double> Blk::*F,
           bool leaf) {
  I = Tree::wrap(I, T.nx(l) * T.B);
  J = Tree::wrap(J, T.ny(l) * T.B);
  const int k = T.find(l, I / T.B, J / T.B);
  if (k >= 0) {
    const double v = (T.blk[k].*F)[(size_t)(J % T.B) * T.B + (I % T.B)];
    if (T.blk[k].leaf || !leaf) return v;
    const int n = side > 0 ? 0 : 1;  // the children's layer nearest the face
    double a, b;
    bool ok;
    if (d == 0)
      ok = T.cell(l + 1, 2 * I + n, 2 * J, F, &a) && T.cell(l + 1, 2 * I + n, 2 * J + 1, F, &b);
    else
      ok = T.cell(l + 1, 2 * I, 2 * J + n, F, &a) && T.cell(l + 1, 2 * I + 1, 2 * J + n, F, &b);
    if (!ok) return NAN;
    const double m = 0.5 * (a + b);
    return (4.0 / 3.0) * m - (1.0 / 3.0) * f0;
  }
  const int Ic = I >> 1, Jc = J >> 1;
  double C, Cp, Cm;
  bool ok = T.cell(l - 1, Ic, Jc, F, &C);
  if (d == 0) {
    ok = ok && T.cell(l - 1, Ic, Jc + 1, F, &Cp) && T.cell(l - 1, Ic, Jc - 1, F, &Cm);
  } else {
    ok = ok && T.cell(l - 1, Ic + 1, Jc, F, &Cp) && T.cell(l - 1, Ic - 1, Jc, F, &Cm);
  }
  if (!ok) return NAN;  // the tree is not 2:1 balanced
  const int t = d == 0 ? J : I;
  const double s = (t & 1) ? 1.0 : -1.0;
  const double Chat = C + (s * (Cp - Cm)) * 0.125;
  return (2.0 / 3.0) * Chat + (1.0 / 3.0) * f0;
}

// sum of the four neighbours of cell (i, j) of block b (value x0), ordered x-, x+, y-, y+;
// comp: the composite operator (flux matching at leaf cells next to refined blocks), else
// the level operator
double nbr_sum(const Tree& T, const Blk& b, int i, int j, double x0, std::vector<double> Blk::*F, bool comp) {
  const int l = b.lev, I = b.bx * T.B + i, J = b.by * T.B + j;
  const bool lf = comp && b.leaf;
  double s = nbr(T, l, I - 1, J, 0, -1, x0, F, lf);
  s = s + nbr(T, l, I + 1, J, 0, +1, x0, F, lf);
  s = s + nbr(T, l, I, J - 1, 1, -1, x0, F, lf);
  s = s + nbr(T, l, I, J + 1, 1, +1, x0, F, lf);
  return s;
}

// (A x) at cell (i, j) of block k: lambda x - (sum of the four neighbours - 4 x) / h^2
double apply_at(const Tree& T, int k, int i, int j, std::vector<double> Blk::*F, bool comp) {
  const Blk& b = T.blk[k];
  const double x0 = (b.*F)[(size_t)j * T.B + i];
  const double s = nbr_sum(T, b, i, j, x0, F, comp);
  const double ih2 = 1.0 / (T.h(b.lev) * T.h(b.lev));
  return T.lam * x0 - (s - 4.0 * x0) * ih2;
}

// refined blocks of level l get the means of their children's field F (children first)
void restrict_level(Tree& T, int l, std::vector<double> Blk::*F) {
  const int B = T.B;
  for (int k : T.bylev[l]) {
    Blk& p = T.blk[k];
    if (p.leaf) continue;
    for (int j = 0; j < B; ++j)
      for (int i = 0; i < B; ++i) {
        const int q = (2 * i >= B ? 1 : 0) + 2 * (2 * j >= B ? 1 : 0);
        const Blk& c = T.blk[p.child[q]];
        const int ci = (2 * i) % B, cj = (2 * j) % B;
        double s = (c.*F)[(size_t)cj * B + ci];
        s = s + (c.*F)[(size_t)cj * B + ci + 1];
        s = s + (c.*F)[(size_t)(cj + 1) * B + ci];
        s = s + (c.*F)[(size_t)(cj + 1) * B + ci + 1];
        (p.*F)[(size_t)j * B + i] = 0.25 * s;
      }
  }
}

void restrict_all(Tree& T) {
  for (int l = T.lmax - 1; l >= 1; --l) restrict_level(T, l, &Blk::x);
}

// one red-black Gauss-Seidel sweep over every block of level l
void gs_level(Tree& T, int l) {
  const int B = T.B;
  const double ih2 = 1.0 / (T.h(l) * T.h(l));
  for (int colour = 0; colour < 2; ++colour)
    for (int k : T.bylev[l]) {
      Blk& b = T.blk[k];
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i) {
          const int I = b.bx * B + i, J = b.by * B + j;
          if (((I + J) & 1) != colour) continue;
          const double x0 = b.x[(size_t)j * B + i];
          const double s = nbr_sum(T, b, i, j, x0, &Blk::x, false);
          b.x[(size_t)j * B + i] = (b.b[(size_t)j * B + i] + s * ih2) / (T.lam + 4.0 * ih2);
        }
    }
}

void residual_level(Tree& T, int l) {
  const int B = T.B;
  for (int k : T.bylev[l]) {
    Blk& b = T.blk[k];
    for (int j = 0; j < B; ++j)
      for (int i = 0; i < B; ++i)
        b.r[(size_t)j * B + i] = b.b[(size_t)j * B + i] - apply_at(T, k, i, j, &Blk::x, false);
  }
}

// level 1 is a uniform periodic grid: gather it, solve A e = b - A x from e = 0 with the
// uniform multigrid (relative tolerance base_rtol), scatter x + e
void base_solve(Tree& T, const orc_amg_config* c) {
  const int B = T.B, n = T.nbx * B;
  std::vector<double> x((size_t)n * n), b((size_t)n * n);
  for (int k : T.bylev[1]) {
    const Blk& blk = T.blk[k];
    for (int j = 0; j < B; ++j)
      for (int i = 0; i < B; ++i) {
        size_t g = (size_t)(blk.by * B + j) * n + blk.bx * B + i;
        x[g] = blk.x[(size_t)j * B + i];
        b[g] = blk.b[(size_t)j * B + i];
      }
  }
  // correction form: A e = b - A x from e = 0, to base_rtol of the initial base residual
  std::vector<double> r((size_t)n * n), e((size_t)n * n, 0.0);
  orc_mg_apply(2, n, c->L, c->lambda, ORC_MG_PERIODIC, x.data(), r.data());
  for (size_t i = 0; i < r.size(); ++i) r[i] = b[i] - r[i];
  orc_mg_config mc{2, n, c->L, c->lambda, 2, 2, 200, c->base_rtol, c->coarse_max, ORC_MG_PERIODIC};
  double rr;
  orc_mg_solve(&mc, r.data(), e.data(), &rr);
  for (int k : T.bylev[1]) {
    Blk& blk = T.blk[k];
    for (int j = 0; j < B; ++j)
      for (int i = 0; i < B; ++i) {
        const size_t g = (size_t)(blk.by * B + j) * n + blk.bx * B + i;
        blk.x[(size_t)j * B + i] = x[g] + e[g];
      }
  }
}

// e = x - xold at level-(l-1) cell (Ic, Jc), or e of the parent cell (Pc, Pj) if that cell
// does not exist at level l-1
double corr(const Tree& T, int l, int Ic, int Jc, double ep) {
  double a, o;
  if (!T.cell(l, Ic, Jc, &Blk::x, &a)) return ep;
  T.cell(l, Ic, Jc, &Blk::xold, &o);
  return a - o;
}

void vcycle(Tree& T, const orc_amg_config* c, int l) {
  if (l == 1) {
    base_solve(T, c);
    return;
  }
  const int B = T.B;
  for (int s = 0; s < c->nu1; ++s) gs_level(T, l);
  residual_level(T, l);
  restrict_level(T, l - 1, &Blk::x);
  for (int k : T.bylev[l - 1]) T.blk[k].xold = T.blk[k].x;
  restrict_level(T, l - 1, &Blk::r);  // r of a refined level-(l-1) block = mean residual of its children
  for (int k : T.bylev[l - 1]) {       // leaves of level l-1: their composite residual
    Blk& p = T.blk[k];
    if (!p.leaf) continue;
    for (int j = 0; j < B; ++j)
      for (int i = 0; i < B; ++i)
        p.r[(size_t)j * B + i] = p.bo[(size_t)j * B + i] - apply_at(T, k, i, j, &Blk::x, true);
  }
  for (int k : T.bylev[l - 1]) {  // FAS right-hand side of level l-1: b = r + A_{l-1} x
    Blk& p = T.blk[k];
    for (int j = 0; j < B; ++j)
      for (int i = 0; i < B; ++i)
        p.b[(size_t)j * B + i] = p.r[(size_t)j * B + i] + apply_at(T, k, i, j, &Blk::x, false);
  }
  vcycle(T, c, l - 1);
  for (int k : T.bylev[l - 1]) {
    const Blk& p = T.blk[k];
    if (p.leaf) continue;
    for (int q = 0; q < 4; ++q) {
      Blk& ch = T.blk[p.child[q]];
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i) {
          const int I = ch.bx * B + i, J = ch.by * B + j;
          const int Ic = I >> 1, Jc = J >> 1;
          const int sx = (I & 1) ? 1 : -1, sy = (J & 1) ? 1 : -1;
          const double e0 = corr(T, l - 1, Ic, Jc, 0.0);
          double acc = 0.5625 * e0;
          acc = acc + 0.1875 * corr(T, l - 1, Ic + sx, Jc, e0);
          acc = acc + 0.1875 * corr(T, l - 1, Ic, Jc + sy, e0);
          acc = acc + 0.0625 * corr(T, l - 1, Ic + sx, Jc + sy, e0);
          ch.x[(size_t)j * B + i] = ch.x[(size_t)j * B + i] + acc;
        }
    }
  }
  for (int s = 0; s < c->nu2; ++s) gs_level(T, l);
}

double leaf_residual_max(Tree& T, double* bmax) {
  restrict_all(T);
  double rm = 0.0, bm = 0.0;
  const int B = T.B;
  for (int k : T.leaf_blk) {
    const Blk& b = T.blk[k];
    for (int j = 0; j < B; ++j)
      for (int i = 0; i < B; ++i) {
        const double r = b.bo[(size_t)j * B + i] - apply_at(T, k, i, j, &Blk::x, true);
        rm = std::fmax(rm, std::fabs(r));
        bm = std::fmax(bm, std::fabs(b.bo[(size_t)j * B + i]));
      }
  }
  if (bmax) *bmax = bm;
  return rm;
}

void load(Tree& T, const double* src, std::vector<double> Blk::*F) {
  const size_t n = (size_t)T.B * T.B;
  for (size_t k = 0; k < T.leaf_blk.size(); ++k) std::memcpy((T.blk[T.leaf_blk[k]].*F).data(), src + k * n, n * 8);
}

void store(const Tree& T, double* dst) {
  const size_t n = (size_t)T.B * T.B;
  for (size_t k = 0; k < T.leaf_blk.size(); ++k) std::memcpy(dst + k * n, T.blk[T.leaf_blk[k]].x.data(), n * 8);
}

// composite Laplacian of leaf data w on the leaves: (sum of neighbours - 4 w) / h^2
void composite_lap(Tree& T, const double* w, double* lap) {
  load(T, w, &Blk::x);
  restrict_all(T);
  const int B = T.B;
  for (size_t k = 0; k < T.leaf_blk.size(); ++k) {
    const Blk& b = T.blk[T.leaf_blk[k]];
    const double ih2 = 1.0 / (T.h(b.lev) * T.h(b.lev));
    for (int j = 0; j < B; ++j)
      for (int i = 0; i < B; ++i) {
        const double x0 = b.x[(size_t)j * B + i];
        lap[k * B * B + (size_t)j * B + i] = (nbr_sum(T, b, i, j, x0, &Blk::x, true) - 4.0 * x0) * ih2;
      }
  }
}

// ---------------------------------------------------------------- regrid ---
// READING (the paper refines the Gray-Scott mesh adaptively but states no criterion; the
// Lohner estimator of Sec. 1.3 is the method's default): per leaf, the Lohner estimator of u
// (the field the paper's figure shows; v is near zero away from the pattern, where the
// filter, relative to |q|, would flag round-off), per direction, second difference over the
// sum of the two first differences plus a filter eps (|q+| + 2|q0| + |q-|), squares summed
// over the two directions, E = sqrt(num / den) (0 where den = 0); neighbours through the
// level operator's values; max over the leaf's cells.
double lohner_field(const Tree& T, int k, double eps) {
  const Blk& b = T.blk[k];
  const int B = T.B, l = b.lev;
  double emax = 0.0;
  for (int j = 0; j < B; ++j)
    for (int i = 0; i < B; ++i) {
      const int I = b.bx * B + i, J = b.by * B + j;
      const double q0 = b.x[(size_t)j * B + i];
      double num = 0.0, den = 0.0;
      for (int d = 0; d < 2; ++d) {
        const double qm = d == 0 ? nbr(T, l, I - 1, J, 0, -1, q0, &Blk::x, false) : nbr(T, l, I, J - 1, 1, -1, q0, &Blk::x, false);
        const double qp = d == 0 ? nbr(T, l, I + 1, J, 0, +1, q0, &Blk::x, false) : nbr(T, l, I, J + 1, 1, +1, q0, &Blk::x, false);
        const double d2 = qp - 2.0 * q0 + qm;
        const double d1 = std::fabs(qp - q0) + std::fabs(q0 - qm) + eps * (std::fabs(qp) + 2.0 * std::fabs(q0) + std::fabs(qm));
        num = num + d2 * d2;
        den = den + d1 * d1;
      }
      const double e = den > 0.0 ? std::sqrt(num / den) : 0.0;
      emax = std::fmax(emax, e);
    }
  return emax;
}

struct LeafKey {
  int l, x, y;
  bool operator<(const LeafKey& o) const { return l != o.l ? l < o.l : (x != o.x ? x < o.x : y < o.y); }
  bool operator==(const LeafKey& o) const { return l == o.l && x == o.x && y == o.y; }
};

// closed boxes of two blocks overlap, periodic images included (nbx x nby base blocks)
bool touches(const LeafKey& a, const LeafKey& b, int nbx, int nby, int lmax) {
  const long sa = 1L << (lmax - a.l), sb = 1L << (lmax - b.l);
  const long N[2] = {(long)nbx << (lmax - 1), (long)nby << (lmax - 1)};
  const long lo_a[2] = {a.x * sa, a.y * sa}, lo_b[2] = {b.x * sb, b.y * sb};
  for (int d = 0; d < 2; ++d) {
    bool any = false;
    for (long shift = -N[d]; shift <= N[d]; shift += N[d])
      if (lo_a[d] <= lo_b[d] + sb + shift && lo_b[d] + shift <= lo_a[d] + sa) any = true;
    if (!any) return false;
  }
  return true;
}

// Morton key of a block's lower corner at level lmax (x bits lowest): the order of new leaves
unsigned long long morton(const LeafKey& k, int lmax) {
  const unsigned long long x = (unsigned long long)k.x << (lmax - k.l), y = (unsigned long long)k.y << (lmax - k.l);
  unsigned long long m = 0;
  for (int b = 0; b < 24; ++b) m |= ((x >> b) & 1ull) << (2 * b) | ((y >> b) & 1ull) << (2 * b + 1);
  return m;
}

double minmod(double a, double b) { return a * b > 0.0 ? (std::fabs(a) < std::fabs(b) ? a : b) : 0.0; }

}  // namespace

extern "C" {

// Regrid of the reaction-diffusion quadtree (READING, see lohner_field above; the tree rules
// are those of the hydrodynamic regrid): refine a leaf with E > refine_tol below max_level;
// coarsen a group of four sibling leaves when each has E < coarsen_frac refine_tol and none
// is refined; 2:1 balance across faces and corners (periodic images included) by refining
// the coarser touching leaves of a refined leaf until none is left, and by dropping a
// coarsening whose parent would touch a leaf more than one level finer.  Transfer: kept leaves
// copy, a refined leaf's children take q + s_x/4 + s_y/4 with s the minmod of the parent's two
// one-sided differences along each direction (parent-level neighbours, level operator),
// signed by the child's half; a coarsened parent takes the means of its 2x2 children.  New
// leaves in Morton order of their lower corner at max_level.
int orc_amg_regrid(const orc_amg_config* c, int nleaves, const int* level, const int* coords, const double* u,
                   const double* v, double refine_tol, double coarsen_frac, double eps, int max_level, int cap,
                   int* new_level, int* new_coords, double* new_u, double* new_v, double* err) {
  Tree Tu, Tv;
  if (c->nbx != c->nby || build_tree(c, nleaves, level, coords, &Tu) || build_tree(c, nleaves, level, coords, &Tv))
    return -2;
  load(Tu, u, &Blk::x);
  load(Tv, v, &Blk::x);
  restrict_all(Tu);
  restrict_all(Tv);
  const int B = c->B, nb2 = B * B;
  std::vector<double> E(nleaves);
  std::vector<LeafKey> old(nleaves);
  for (int k = 0; k < nleaves; ++k) {
    E[k] = lohner_field(Tu, Tu.leaf_blk[k], eps);
    if (err) err[k] = E[k];
    old[k] = {level[k], coords[2 * k], coords[2 * k + 1]};
  }
  const int lmax = max_level > Tu.lmax ? max_level : Tu.lmax;
  std::map<LeafKey, int> idx;  // old leaf -> index
  for (int k = 0; k < nleaves; ++k) idx[old[k]] = k;
  std::vector<char> refine(nleaves, 0);
  for (int k = 0; k < nleaves; ++k) refine[k] = E[k] > refine_tol && old[k].l < max_level;
  for (bool changed = true; changed;) {  // balance the refinement
    changed = false;
    for (int a = 0; a < nleaves; ++a) {
      if (!refine[a]) continue;
      for (int b = 0; b < nleaves; ++b)
        if (!refine[b] && old[b].l < old[a].l && touches(old[a], old[b], c->nbx, c->nby, lmax)) {
          refine[b] = 1;
          changed = true;
        }
    }
  }
  std::vector<LeafKey> mid;  // the tree after refinement
  for (int k = 0; k < nleaves; ++k) {
    if (!refine[k]) {
      mid.push_back(old[k]);
      continue;
    }
    for (int q = 0; q < 4; ++q) mid.push_back({old[k].l + 1, 2 * old[k].x + (q & 1), 2 * old[k].y + (q >> 1)});
  }
  std::map<LeafKey, int> parents;  // candidate coarsenings: parent -> number of qualifying children
  for (int k = 0; k < nleaves; ++k)
    if (old[k].l > 1 && !refine[k] && E[k] < coarsen_frac * refine_tol)
      parents[{old[k].l - 1, old[k].x >> 1, old[k].y >> 1}] += 1;
  std::vector<LeafKey> coarsen;
  for (const auto& pc : parents) {
    if (pc.second != 4) continue;
    bool ok = true;
    for (const LeafKey& n : mid)
      if (n.l > pc.first.l + 1 && touches(pc.first, n, c->nbx, c->nby, lmax)) {
        ok = false;
        break;
      }
    if (ok) coarsen.push_back(pc.first);
  }
  std::vector<LeafKey> out;
  for (const LeafKey& n : mid) {
    const LeafKey p{n.l - 1, n.x >> 1, n.y >> 1};
    if (n.l > 1 && std::find(coarsen.begin(), coarsen.end(), p) != coarsen.end()) continue;
    out.push_back(n);
  }
  for (const LeafKey& p : coarsen) out.push_back(p);
  std::sort(out.begin(), out.end(),
            [&](const LeafKey& a, const LeafKey& b) { return morton(a, lmax) < morton(b, lmax); });
  if ((int)out.size() > cap) return -3;
  for (size_t n = 0; n < out.size(); ++n) {
    const LeafKey& K = out[n];
    new_level[n] = K.l;
    new_coords[2 * n] = K.x;
    new_coords[2 * n + 1] = K.y;
    for (int f = 0; f < 2; ++f) {
      const Tree& T = f == 0 ? Tu : Tv;
      double* dst = (f == 0 ? new_u : new_v) + n * nb2;
      auto it = idx.find(K);
      if (it != idx.end()) {  // kept
        std::memcpy(dst, T.blk[T.leaf_blk[it->second]].x.data(), nb2 * sizeof(double));
        continue;
      }
      const LeafKey P{K.l - 1, K.x >> 1, K.y >> 1};
      if (K.l > 1 && idx.count(P)) {  // child of a refined leaf
        const Blk& pb = T.blk[T.leaf_blk[idx[P]]];
        for (int j = 0; j < B; ++j)
          for (int i = 0; i < B; ++i) {
            const int I = K.x * B + i, J = K.y * B + j;  // fine cell, level K.l
            const int Ic = I >> 1, Jc = J >> 1;        // parent cell, level P.l
            const int pi = Ic - pb.bx * B, pj = Jc - pb.by * B;
            const double q = pb.x[(size_t)pj * B + pi];
            const double qxm = nbr(T, P.l, Ic - 1, Jc, 0, -1, q, &Blk::x, false);
            const double qxp = nbr(T, P.l, Ic + 1, Jc, 0, +1, q, &Blk::x, false);
            const double qym = nbr(T, P.l, Ic, Jc - 1, 1, -1, q, &Blk::x, false);
            const double qyp = nbr(T, P.l, Ic, Jc + 1, 1, +1, q, &Blk::x, false);
            const double sx = (I & 1) ? 0.25 : -0.25, sy = (J & 1) ? 0.25 : -0.25;
            dst[(size_t)j * B + i] = (q + sx * minmod(q - qxm, qxp - q)) + sy * minmod(q - qym, qyp - q);
          }
        continue;
      }
      // parent of coarsened leaves: means of the children
      for (int j = 0; j < B; ++j)
        for (int i = 0; i < B; ++i) {
          const int quad = (2 * i >= B ? 1 : 0) + 2 * (2 * j >= B ? 1 : 0);
          const LeafKey ch{K.l + 1, 2 * K.x + (quad & 1), 2 * K.y + (quad >> 1)};
          const Blk& cb = T.blk[T.leaf_blk[idx.at(ch)]];
          const int ci = (2 * i) % B, cj = (2 * j) % B;
          double sum = cb.x[(size_t)cj * B + ci];
          sum = sum + cb.x[(size_t)cj * B + ci + 1];
          sum = sum + cb.x[(size_t)(cj + 1) * B + ci];
          sum = sum + cb.x[(size_t)(cj + 1) * B + ci + 1];
          dst[(size_t)j * B + i] = 0.25 * sum;
        }
    }
  }
  return (int)out.size();
}

// Gray-Scott IMEX step, Eq. (imex) with Eq. (gray-scott), on the leaves of the quadtree:
// the composite Laplacian for the explicit parts and the tree multigrid for the implicit
// stage (lambda = 2/(dt D) per species, guess w_n), in the order of orc_rd_step.
int orc_amg_rd_step(const orc_amg_config* c, int nleaves, const int* level, const int* coords, double Du, double Dv,
                    double F, double k, double dt, double* u, double* v, int* cycles) {
  Tree T;
  if (c->nbx != c->nby || build_tree(c, nleaves, level, coords, &T)) return -2;
  const size_t N = (size_t)nleaves * c->B * c->B;
  std::vector<double> lu(N), lv(N), fu(N), fv(N);
  composite_lap(T, u, lu.data());
  composite_lap(T, v, lv.data());
  for (size_t i = 0; i < N; ++i) {
    double uvv = (u[i] * v[i]) * v[i];
    fu[i] = -uvv + F * (1.0 - u[i]);
    fv[i] = uvv - (F + k) * v[i];
  }
  double D[2] = {Du, Dv};
  double* w[2] = {u, v};
  std::vector<double>* R[2] = {&fu, &fv};
  std::vector<double>* Lp[2] = {&lu, &lv};
  std::vector<double> ws[2];
  int status = 0;
  for (int s = 0; s < 2; ++s) {
    orc_amg_config mc = *c;
    mc.lambda = 2.0 / (dt * D[s]);
    std::vector<double> b(N);
    for (size_t i = 0; i < N; ++i) {
      double gi = (w[s][i] + dt * (*R[s])[i]) + ((0.5 * dt) * D[s]) * (*Lp[s])[i];
      b[i] = mc.lambda * gi;
    }
    ws[s].assign(w[s], w[s] + N);
    double rr;
    int cyc = orc_amg_solve(&mc, nleaves, level, coords, b.data(), ws[s].data(), 0, &rr);
    if (cycles) cycles[s] = cyc;
    if (cyc < 0) status = -1;
  }
  std::vector<double> lus(N), lvs(N);
  composite_lap(T, ws[0].data(), lus.data());
  composite_lap(T, ws[1].data(), lvs.data());
  for (size_t i = 0; i < N; ++i) {
    double uvv = (ws[0][i] * ws[1][i]) * ws[1][i];
    double fus = -uvv + F * (1.0 - ws[0][i]);
    double fvs = uvv - (F + k) * ws[1][i];
    double Fnu = fu[i] + Du * lu[i], Fnv = fv[i] + Dv * lv[i];
    u[i] = u[i] + (0.5 * dt) * (Fnu + (fus + Du * lus[i]));
    v[i] = v[i] + (0.5 * dt) * (Fnv + (fvs + Dv * lvs[i]));
  }
  return status;
}

int orc_amg_solve(const orc_amg_config* c, int nleaves, const int* level, const int* coords, const double* b,
                  double* x, int fixed_cycles, double* relres) {
  Tree T;
  if (c->nbx != c->nby || build_tree(c, nleaves, level, coords, &T)) return -2;
  load(T, b, &Blk::bo);
  load(T, b, &Blk::b);  // the finest level has no refined blocks: its level problem is the composite one
  load(T, x, &Blk::x);
  double bm;
  double rm = leaf_residual_max(T, &bm);
  int cycles = 0;
  while (fixed_cycles > 0 ? cycles < fixed_cycles : (rm > c->rtol * bm && cycles < c->max_cycles)) {
    vcycle(T, c, T.lmax);
    ++cycles;
    rm = leaf_residual_max(T, &bm);
  }
  store(T, x);
  if (relres) *relres = bm > 0.0 ? rm / bm : rm;
  return (fixed_cycles > 0 || rm <= c->rtol * bm) ? cycles : -1;
}

int orc_amg_apply(const orc_amg_config* c, int nleaves, const int* level, const int* coords, const double* x,
                  double* Ax) {
  Tree T;
  if (c->nbx != c->nby || build_tree(c, nleaves, level, coords, &T)) return -2;
  load(T, x, &Blk::x);
  restrict_all(T);
  const int B = T.B;
  for (size_t k = 0; k < T.leaf_blk.size(); ++k)
    for (int j = 0; j < B; ++j)
      for (int i = 0; i < B; ++i) Ax[k * B * B + (size_t)j * B + i] = apply_at(T, T.leaf_blk[k], i, j, &Blk::x, true);
  return 0;
}

int orc_amg_face_ghosts(const orc_amg_config* c, int nleaves, const int* level, const int* coords, const double* x,
                        double* ghosts) {
  Tree T;
  if (c->nbx != c->nby || build_tree(c, nleaves, level, coords, &T)) return -2;
  load(T, x, &Blk::x);
  restrict_all(T);
  const int B = T.B;
  for (size_t k = 0; k < T.leaf_blk.size(); ++k) {
    const Blk& b = T.blk[T.leaf_blk[k]];
    const int l = b.lev, I0 = b.bx * B, J0 = b.by * B;
    double* g = ghosts + k * 4 * B;
    for (int t = 0; t < B; ++t) {
      g[0 * B + t] = nbr(T, l, I0 - 1, J0 + t, 0, -1, b.x[(size_t)t * B], &Blk::x, true);
      g[1 * B + t] = nbr(T, l, I0 + B, J0 + t, 0, +1, b.x[(size_t)t * B + B - 1], &Blk::x, true);
      g[2 * B + t] = nbr(T, l, I0 + t, J0 - 1, 1, -1, b.x[t], &Blk::x, true);
      g[3 * B + t] = nbr(T, l, I0 + t, J0 + B, 1, +1, b.x[(size_t)(B - 1) * B + t], &Blk::x, true);
    }
  }
  return 0;
}

}  // extern "C"
