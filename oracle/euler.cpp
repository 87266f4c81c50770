// FP64 oracle: Euler finite-volume update on a block quadtree/octree.
// TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain loops, no blocking, no
// fusion; ghost cells are found by searching the leaf set for the block that
// covers each ghost location, never through neighbour tables.
//
// Written from the paper (arXiv:2004.03275):
//  * Sec. 1.1: U = (rho, rho v, E), E = rho v^2/2 + p/(gamma-1), V = (rho, v, p).
//  * Sec. 1.2: CFL limit from the maximal signal speed (phys_get_cmax); TVDLF and
//    HLL fluxes from the speed bounds (phys_get_cbounds).
//  * Sec. 2.3.1 / 2.4: HLLC flux, limited reconstruction (Koren), three-step RK.
//  * Sec. 1.3: block tree with refinement ratio 2, Lohner-type estimator of
//    weighted second derivatives, refine when one cell exceeds the tolerance,
//    coarsen when every cell is below a fraction of it.
// Readings where the paper is silent are marked READING.
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <tuple>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct Leaf {
  int level;
  int c[3];
  std::vector<double> U;  // [var][cell]
};

typedef std::tuple<int, int, int, int> Key;

}  // namespace

struct orc_grid {
  orc_config cfg;
  int nv;      // conserved variables
  int ncell;   // cells per block
  double t;
  std::vector<Leaf> leaves;      // Morton order
  std::map<Key, int> index;      // (level, cx, cy, cz) -> leaf position
};

namespace {

// ---------------------------------------------------------------- physics --
// Sec. 1.1: primitive <-> conserved.  Operation order is fixed as written.
void prim_to_cons(int nd, double gam, const double* V, double* U) {
  double rho = V[0];
  double vsq = 0.0;
  for (int d = 0; d < nd; ++d) vsq = vsq + V[1 + d] * V[1 + d];
  U[0] = rho;
  for (int d = 0; d < nd; ++d) U[1 + d] = rho * V[1 + d];
  U[nd + 1] = V[nd + 1] / (gam - 1.0) + (0.5 * rho) * vsq;
}

void cons_to_prim(int nd, double gam, const double* U, double* V) {
  double rho = U[0];
  double msq = 0.0;
  for (int d = 0; d < nd; ++d) msq = msq + U[1 + d] * U[1 + d];
  V[0] = rho;
  for (int d = 0; d < nd; ++d) V[1 + d] = U[1 + d] / rho;
  V[nd + 1] = (gam - 1.0) * (U[nd + 1] - (0.5 * msq) / rho);
}

double sound_speed(int nd, double gam, const double* V) {
  return std::sqrt(gam * V[nd + 1] / V[0]);
}

// Sec. 1.1: flux in direction `dir` = advective part v_dir U plus the pressure
// (non-advective) part in the momentum and energy equations.
void phys_flux(int nd, int dir, double gam, const double* V, double* F) {
  double U[5];
  prim_to_cons(nd, gam, V, U);
  double un = V[1 + dir];
  double p = V[nd + 1];
  F[0] = U[1 + dir];
  for (int e = 0; e < nd; ++e) {
    F[1 + e] = U[1 + e] * un;
    if (e == dir) F[1 + e] = F[1 + e] + p;
  }
  F[nd + 1] = (U[nd + 1] + p) * un;
}

// Sec. 1.2 / 2.3 / 2.4.  READING: wave-speed bounds are the Davis estimates
// S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R); HLLC is
// Toro's form with the contact speed S*; TVDLF uses c_max = max(|u|+c).
void riemann_flux(int nd, int dir, int kind, double gam, const double* VL, const double* VR,
                  double* F) {
  const int nv = nd + 2;
  double UL[5], UR[5], FL[5], FR[5];
  prim_to_cons(nd, gam, VL, UL);
  prim_to_cons(nd, gam, VR, UR);
  phys_flux(nd, dir, gam, VL, FL);
  phys_flux(nd, dir, gam, VR, FR);
  double uL = VL[1 + dir], uR = VR[1 + dir];
  double cL = sound_speed(nd, gam, VL), cR = sound_speed(nd, gam, VR);
  if (kind == ORC_FLUX_TVDLF) {
    double cmax = std::max(std::fabs(uL) + cL, std::fabs(uR) + cR);
    for (int v = 0; v < nv; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - (0.5 * cmax) * (UR[v] - UL[v]);
    return;
  }
  double SL = std::min(uL - cL, uR - cR);
  double SR = std::max(uL + cL, uR + cR);
  if (SL >= 0.0) {
    for (int v = 0; v < nv; ++v) F[v] = FL[v];
    return;
  }
  if (SR <= 0.0) {
    for (int v = 0; v < nv; ++v) F[v] = FR[v];
    return;
  }
  if (kind == ORC_FLUX_HLL) {
    double inv = 1.0 / (SR - SL);
    for (int v = 0; v < nv; ++v)
      F[v] = (SR * FL[v] - SL * FR[v] + (SL * SR) * (UR[v] - UL[v])) * inv;
    return;
  }
  // HLLC
  double rL = VL[0], rR = VR[0], pL = VL[nd + 1], pR = VR[nd + 1];
  double aL = rL * (SL - uL), aR = rR * (SR - uR);
  double Sstar = (pR - pL + aL * uL - aR * uR) / (aL - aR);
  const double* Vk;
  const double* Uk;
  const double* Fk;
  double Sk, ak;
  if (Sstar >= 0.0) {
    Vk = VL; Uk = UL; Fk = FL; Sk = SL; ak = aL;
  } else {
    Vk = VR; Uk = UR; Fk = FR; Sk = SR; ak = aR;
  }
  double uk = Vk[1 + dir], pk = Vk[nd + 1], rk = Vk[0];
  double fac = ak / (Sk - Sstar);
  double Us[5];
  Us[0] = fac;
  for (int e = 0; e < nd; ++e) Us[1 + e] = fac * (e == dir ? Sstar : Vk[1 + e]);
  Us[nd + 1] = fac * (Uk[nd + 1] / rk + (Sstar - uk) * (Sstar + pk / ak));
  for (int v = 0; v < nv; ++v) F[v] = Fk[v] + Sk * (Us[v] - Uk[v]);
}

// READING (limiters are named in Sec. 2.3.1 / 2.4 but not written out):
// a = q_i - q_{i-1}, b = q_{i+1} - q_i; s- is used towards i-1/2, s+ towards i+1/2
// (face values q_i - s-/2 and q_i + s+/2).
//  * minmod, van Leer, monotonized central: one symmetric slope, zero at extrema.
//  * Koren (1993): the third-order upwind-biased (kappa = 1/3) face values
//    q_i + (a + 2b)/6 and q_i - (2a + b)/6, limited into the TVD region:
//    s+ = sgn(b) min(2|a|, (|a| + 2|b|)/3, 2|b|), s- = sgn(a) min(2|b|, (2|a| + |b|)/3, 2|a|),
//    zero where a b <= 0.
//  * Cada: the third-order limiter of Cada and Torrilhon (J. Comput. Phys. 228 (2009) 4118,
//    "Compact third-order limiter functions for finite volume methods"), which Sec. 2.3.1
//    uses.  With theta = a / b the face offset is phi(theta) b / 2, phi_3(theta) = (2 + theta)/3
//    the unlimited third-order function and
//      phi(theta) = max(0, min(phi_3(theta), max(-theta, min(2 theta, phi_3(theta), 1.5)))),
//    and the mirror image, theta = b / a times a, towards i-1/2.  Unlike the TVD limiters it
//    keeps a slope where a and b differ in sign (|theta| small: a one-sided extremum), bounded
//    by -theta.  READING: the limited function everywhere; the paper's switch to phi_3 near
//    smooth extrema, which depends on a dimensional radius, is not used.
void limited_slopes(int lim, double a, double b, double* sm, double* sp) {
  bool same = (a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0);
  if (lim == ORC_LIM_CADA) {
    double A = std::fabs(a), B = std::fabs(b);
    double up = 0.0, dn = 0.0;
    if (same) {
      up = std::min(std::min(2.0 * A, (A + 2.0 * B) / 3.0), 1.5 * B);
      dn = std::min(std::min(2.0 * B, (2.0 * A + B) / 3.0), 1.5 * A);
    } else if (a != 0.0 && b != 0.0) {
      up = std::max(0.0, std::min((2.0 * B - A) / 3.0, A));
      dn = std::max(0.0, std::min((2.0 * A - B) / 3.0, B));
    }
    *sp = (b > 0.0) ? up : -up;
    *sm = (a > 0.0) ? dn : -dn;
    return;
  }
  if (lim == ORC_LIM_NONE || !same) {
    *sm = 0.0;
    *sp = 0.0;
    return;
  }
  if (lim == ORC_LIM_MINMOD) {
    double s = (a > 0.0) ? std::min(a, b) : std::max(a, b);
    *sm = s;
    *sp = s;
  } else if (lim == ORC_LIM_VANLEER) {
    double s = (2.0 * a * b) / (a + b);
    *sm = s;
    *sp = s;
  } else if (lim == ORC_LIM_MC) {  // monotonized central: minmod((a+b)/2, 2a, 2b)
    double A = std::fabs(a), B = std::fabs(b);
    double s = std::min(std::min(0.5 * (A + B), 2.0 * A), 2.0 * B);
    *sm = (a > 0.0) ? s : -s;
    *sp = *sm;
  } else {  // Koren: kappa = 1/3 face values limited into the TVD region
    double A = std::fabs(a), B = std::fabs(b);
    double up = std::min(std::min(2.0 * A, (A + 2.0 * B) / 3.0), 2.0 * B);
    double dn = std::min(std::min(2.0 * B, (2.0 * A + B) / 3.0), 2.0 * A);
    *sp = (b > 0.0) ? up : -up;
    *sm = (a > 0.0) ? dn : -dn;
  }
}

// minmod of two differences, used by prolongation (READING: limited linear
// prolongation with minmod slopes).
double minmod2(double a, double b) {
  if (a > 0.0 && b > 0.0) return std::min(a, b);
  if (a < 0.0 && b < 0.0) return std::max(a, b);
  return 0.0;
}

// ------------------------------------------------------------------- tree --
int ncells_dim(const orc_grid* g, int level, int d) {
  if (d >= g->cfg.ndim) return 1;
  return g->cfg.base[d] * g->cfg.block_nx * (1 << (level - 1));
}

double cell_dx(const orc_grid* g, int level, int d) {
  return (g->cfg.xmax[d] - g->cfg.xmin[d]) / (double)ncells_dim(g, level, d);
}

uint64_t morton(const orc_grid* g, int level, const int* c) {
  int L = g->cfg.max_level;
  uint64_t X[3] = {0, 0, 0};
  for (int d = 0; d < g->cfg.ndim; ++d) X[d] = (uint64_t)c[d] << (L - level);
  uint64_t key = 0;
  for (int b = 20; b >= 0; --b)
    for (int d = g->cfg.ndim - 1; d >= 0; --d) key = (key << 1) | ((X[d] >> b) & 1u);
  return key;
}

void rebuild_index(orc_grid* g) {
  std::sort(g->leaves.begin(), g->leaves.end(), [g](const Leaf& a, const Leaf& b) {
    return morton(g, a.level, a.c) < morton(g, b.level, b.c);
  });
  g->index.clear();
  for (size_t i = 0; i < g->leaves.size(); ++i) {
    const Leaf& l = g->leaves[i];
    g->index[Key(l.level, l.c[0], l.c[1], l.c[2])] = (int)i;
  }
}

int find_leaf(const orc_grid* g, int level, const int* c) {
  if (level < 1 || level > g->cfg.max_level) return -1;
  auto it = g->index.find(Key(level, c[0], c[1], c[2]));
  return it == g->index.end() ? -1 : it->second;
}

int cell_index(const orc_grid* g, int i, int j, int k) {
  int n = g->cfg.block_nx;
  return i + n * (j + n * k);
}

// value of variable v of the leaf cell covering global cell gi (level of leaf)
double leaf_cell(const orc_grid* g, int li, const int* gi, int v) {
  const Leaf& L = g->leaves[li];
  int n = g->cfg.block_nx;
  int loc[3] = {0, 0, 0};
  for (int d = 0; d < g->cfg.ndim; ++d) loc[d] = gi[d] - L.c[d] * n;
  return L.U[(size_t)v * g->ncell + cell_index(g, loc[0], loc[1], loc[2])];
}

// mean of the 2^ndim cells of a leaf at level `lev+1` that make up coarse cell gc
// of level `lev`.  Sum order: child offsets with x fastest, then times 1/2^ndim.
double restrict_cell(const orc_grid* g, int li, const int* gc, int v) {
  int nd = g->cfg.ndim;
  double sum = 0.0;
  int nz = nd > 2 ? 2 : 1, ny = nd > 1 ? 2 : 1;
  for (int oz = 0; oz < nz; ++oz)
    for (int oy = 0; oy < ny; ++oy)
      for (int ox = 0; ox < 2; ++ox) {
        int f[3] = {2 * gc[0] + ox, nd > 1 ? 2 * gc[1] + oy : 0, nd > 2 ? 2 * gc[2] + oz : 0};
        sum = sum + leaf_cell(g, li, f, v);
      }
  return sum * (1.0 / (double)(1 << nd));
}

// wrap a global cell index of `level` into the domain (periodic dims);
// returns false if it lies outside a non-periodic boundary.
bool wrap_cell(const orc_grid* g, int level, int* gi) {
  for (int d = 0; d < g->cfg.ndim; ++d) {
    int N = ncells_dim(g, level, d);
    if (gi[d] < 0 || gi[d] >= N) {
      int side = gi[d] < 0 ? 0 : 1;
      if (g->cfg.bc[d][side] != ORC_BC_PERIODIC) return false;
      gi[d] = ((gi[d] % N) + N) % N;
    }
  }
  return true;
}

int leaf_at(const orc_grid* g, int level, const int* gi) {
  int n = g->cfg.block_nx;
  int c[3] = {0, 0, 0};
  for (int d = 0; d < g->cfg.ndim; ++d) c[d] = gi[d] / n;
  return find_leaf(g, level, c);
}

// coarse-resolution value at global cell gc of level `lev` (already wrapped):
// the covering leaf's cell if the leaf is on `lev`, the restriction of its
// children if the covering leaf is one level finer.
bool coarse_sample(const orc_grid* g, int lev, const int* gc, int v, double* out) {
  int li = leaf_at(g, lev, gc);
  if (li >= 0) {
    *out = leaf_cell(g, li, gc, v);
    return true;
  }
  int f[3] = {2 * gc[0], 2 * gc[1], 2 * gc[2]};
  li = leaf_at(g, lev + 1, f);
  if (li >= 0) {
    *out = restrict_cell(g, li, gc, v);
    return true;
  }
  return false;
}

// Ghost value for leaf `bi`, face dimension `fd`, at global cell gi of the
// leaf's level (gi lies just outside the leaf across face fd).
// READING (ghost filling between levels is not described in the paper):
//  * same level: copy;
//  * finer neighbour: mean of the 2^ndim fine cells (conservative restriction);
//  * coarser neighbour: limited linear prolongation q_p + 1/4 sum_e sigma_e s_e
//    with s_e = minmod of the coarse cell's one-sided differences; in the face
//    normal the inner neighbour is the restriction of the requesting leaf, in
//    tangential directions a neighbour outside the coarse leaf gives s_e = 0;
//  * outflow boundary: zero gradient, i.e. the leaf's own edge cell.
double ghost_value(const orc_grid* g, int bi, int fd, const int* gi_in, int v) {
  const orc_config& C = g->cfg;
  const Leaf& B = g->leaves[bi];
  int lev = B.level;
  int gi[3] = {gi_in[0], gi_in[1], gi_in[2]};
  if (!wrap_cell(g, lev, gi)) {
    int own[3] = {gi_in[0], gi_in[1], gi_in[2]};
    int n = C.block_nx;
    for (int d = 0; d < C.ndim; ++d)
      own[d] = std::min(std::max(own[d], B.c[d] * n), B.c[d] * n + n - 1);
    return leaf_cell(g, bi, own, v);
  }
  int li = leaf_at(g, lev, gi);
  if (li >= 0) return leaf_cell(g, li, gi, v);
  if (lev < C.max_level) {
    int f[3] = {2 * gi[0], 2 * gi[1], 2 * gi[2]};
    int lf = leaf_at(g, lev + 1, f);
    if (lf >= 0) return restrict_cell(g, lf, gi, v);
  }
  // coarser neighbour
  int gc[3] = {gi[0] >> 1, gi[1] >> 1, gi[2] >> 1};
  int lc = leaf_at(g, lev - 1, gc);
  if (lc < 0) return NAN;  // tree not balanced
  const Leaf& Cl = g->leaves[lc];
  int n = C.block_nx;
  double qp = leaf_cell(g, lc, gc, v);
  double acc = 0.0;
  for (int e = 0; e < C.ndim; ++e) {
    double sigma = (gi[e] & 1) ? 1.0 : -1.0;
    double q[2];
    bool ok = true;
    for (int s = 0; s < 2; ++s) {
      int nb[3] = {gc[0], gc[1], gc[2]};
      nb[e] += (s == 0 ? -1 : 1);
      int loc = nb[e] - Cl.c[e] * n;
      if (loc >= 0 && loc < n) {
        q[s] = leaf_cell(g, lc, nb, v);
      } else if (e == fd) {
        // the inner neighbour, inside the requesting leaf's region
        if (!wrap_cell(g, lev - 1, nb) || !coarse_sample(g, lev - 1, nb, v, &q[s])) ok = false;
      } else {
        ok = false;
      }
    }
    double s = ok ? minmod2(qp - q[0], q[1] - qp) : 0.0;
    acc = acc + sigma * s;
  }
  return qp + 0.25 * acc;
}

int ntang(const orc_grid* g) {
  int nt = 1;
  for (int d = 1; d < g->cfg.ndim; ++d) nt *= g->cfg.block_nx;
  return nt;
}

// global cell of tangential position t, layer m, on face (fd, side) of leaf B
void face_ghost_cell(const orc_grid* g, const Leaf& B, int fd, int side, int m, int t, int* gi) {
  int n = g->cfg.block_nx;
  int loc[3] = {0, 0, 0};
  int e1 = -1, e2 = -1;
  for (int e = 0; e < g->cfg.ndim; ++e)
    if (e != fd) {
      if (e1 < 0) e1 = e; else e2 = e;
    }
  if (e1 >= 0) loc[e1] = t % n;
  if (e2 >= 0) loc[e2] = t / n;
  loc[fd] = side == 0 ? -1 - m : n + m;
  for (int d = 0; d < 3; ++d) gi[d] = (d < g->cfg.ndim ? B.c[d] * n : 0) + loc[d];
}

// padded conserved block with face ghosts (2 layers); index (i+2, j+2, k+2)
struct Padded {
  int n, nd, P;
  std::vector<double> a;  // [var][pk][pj][pi]
  double& at(int v, int i, int j, int k) {
    int pj = nd > 1 ? j + 2 : 0, pk = nd > 2 ? k + 2 : 0;
    int Py = nd > 1 ? P : 1;
    int Pz = nd > 2 ? P : 1;
    return a[(((size_t)v * Pz + pk) * Py + pj) * P + (i + 2)];
  }
};

void fill_padded(const orc_grid* g, int bi, Padded* pd) {
  const orc_config& C = g->cfg;
  int n = C.block_nx, nd = C.ndim, nv = g->nv;
  pd->n = n;
  pd->nd = nd;
  pd->P = n + 4;
  size_t sz = (size_t)nv * pd->P * (nd > 1 ? pd->P : 1) * (nd > 2 ? pd->P : 1);
  pd->a.assign(sz, NAN);
  const Leaf& B = g->leaves[bi];
  for (int v = 0; v < nv; ++v)
    for (int k = 0; k < (nd > 2 ? n : 1); ++k)
      for (int j = 0; j < (nd > 1 ? n : 1); ++j)
        for (int i = 0; i < n; ++i) pd->at(v, i, j, k) = B.U[(size_t)v * g->ncell + cell_index(g, i, j, k)];
  int nt = ntang(g);
  for (int fd = 0; fd < nd; ++fd)
    for (int side = 0; side < 2; ++side)
      for (int m = 0; m < 2; ++m)
        for (int t = 0; t < nt; ++t) {
          int gi[3];
          face_ghost_cell(g, B, fd, side, m, t, gi);
          int loc[3];
          for (int d = 0; d < 3; ++d) loc[d] = gi[d] - (d < nd ? B.c[d] * n : 0);
          for (int v = 0; v < nv; ++v) pd->at(v, loc[0], loc[1], loc[2]) = ghost_value(g, bi, fd, gi, v);
        }
}

struct BlockFlux {
  std::vector<double> F[3];  // per dim: [var][k][j][i] with extent n+1 along that dim
};

int flux_index(int nd, int n, int dim, int v, int i, int j, int k) {
  int ni = (dim == 0) ? n + 1 : n;
  int nj = nd > 1 ? ((dim == 1) ? n + 1 : n) : 1;
  int nk = nd > 2 ? ((dim == 2) ? n + 1 : n) : 1;
  return ((v * nk + k) * nj + j) * ni + i;
}

// fluxes of one leaf at every face of its cells, from its padded state
void block_fluxes(const orc_grid* g, Padded* pd, BlockFlux* bf) {
  const orc_config& C = g->cfg;
  int n = C.block_nx, nd = C.ndim, nv = g->nv;
  for (int dim = 0; dim < nd; ++dim) {
    int ni = (dim == 0) ? n + 1 : n;
    int nj = nd > 1 ? ((dim == 1) ? n + 1 : n) : 1;
    int nk = nd > 2 ? ((dim == 2) ? n + 1 : n) : 1;
    bf->F[dim].assign((size_t)nv * ni * nj * nk, 0.0);
    for (int k = 0; k < nk; ++k)
      for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
          // face between cell (f-1) and f along dim, f = (i,j,k)[dim]
          int f[3] = {i, j, k};
          double W[4][5];  // primitive states of cells f-2 .. f+1
          for (int s = 0; s < 4; ++s) {
            int c[3] = {f[0], f[1], f[2]};
            c[dim] = f[dim] - 2 + s;
            double Uc[5];
            for (int v = 0; v < nv; ++v) Uc[v] = pd->at(v, c[0], c[1], c[2]);
            cons_to_prim(nd, C.gamma, Uc, W[s]);
          }
          double VL[5], VR[5];
          bool bad = false;
          for (int v = 0; v < nv; ++v) {
            double smL, spL, smR, spR;
            limited_slopes(C.limiter, W[1][v] - W[0][v], W[2][v] - W[1][v], &smL, &spL);
            limited_slopes(C.limiter, W[2][v] - W[1][v], W[3][v] - W[2][v], &smR, &spR);
            VL[v] = W[1][v] + 0.5 * spL;
            VR[v] = W[2][v] - 0.5 * smR;
          }
          // READING: positivity fallback to first order at this face
          if (!(VL[0] > 0.0) || !(VR[0] > 0.0) || !(VL[nd + 1] > 0.0) || !(VR[nd + 1] > 0.0)) bad = true;
          if (bad)
            for (int v = 0; v < nv; ++v) {
              VL[v] = W[1][v];
              VR[v] = W[2][v];
            }
          double F[5];
          riemann_flux(nd, dim, C.flux, C.gamma, VL, VR, F);
          for (int v = 0; v < nv; ++v) bf->F[dim][flux_index(nd, n, dim, v, i, j, k)] = F[v];
        }
  }
}

// READING (refluxing is not described in the paper; it is what keeps the
// update conservative on the tree): at a face shared with finer leaves the
// coarse leaf uses the mean of the 2^(ndim-1) fine face fluxes.
void reflux(const orc_grid* g, std::vector<BlockFlux>& fl) {
  const orc_config& C = g->cfg;
  int n = C.block_nx, nd = C.ndim, nv = g->nv;
  if (C.max_level == 1) return;
  for (size_t bi = 0; bi < g->leaves.size(); ++bi) {
    const Leaf& B = g->leaves[bi];
    if (B.level == C.max_level) continue;
    for (int fd = 0; fd < nd; ++fd)
      for (int side = 0; side < 2; ++side) {
        int nt = ntang(g);
        for (int t = 0; t < nt; ++t) {
          int gi[3];
          face_ghost_cell(g, B, fd, side, 0, t, gi);
          if (!wrap_cell(g, B.level, gi)) continue;
          if (leaf_at(g, B.level, gi) >= 0) continue;
          int f0[3] = {2 * gi[0], 2 * gi[1], 2 * gi[2]};
          int lf = leaf_at(g, B.level + 1, f0);
          if (lf < 0) continue;
          const Leaf& Fl = g->leaves[lf];
          // coarse face position in B's flux array
          int loc[3] = {0, 0, 0};
          int e1 = -1, e2 = -1;
          for (int e = 0; e < nd; ++e)
            if (e != fd) {
              if (e1 < 0) e1 = e; else e2 = e;
            }
          if (e1 >= 0) loc[e1] = t % n;
          if (e2 >= 0) loc[e2] = t / n;
          loc[fd] = side == 0 ? 0 : n;
          // fine faces: fine cells adjacent to B's face, tangential 2*g + o
          int ffd = side == 0 ? n : 0;  // fine leaf's face index along fd
          for (int v = 0; v < nv; ++v) {
            double sum = 0.0;
            int n2 = nd > 2 ? 2 : 1, n1 = nd > 1 ? 2 : 1;
            for (int o2 = 0; o2 < n2; ++o2)
              for (int o1 = 0; o1 < n1; ++o1) {
                int fl_loc[3] = {0, 0, 0};
                if (e1 >= 0) fl_loc[e1] = 2 * gi[e1] + o1 - Fl.c[e1] * n;
                if (e2 >= 0) fl_loc[e2] = 2 * gi[e2] + o2 - Fl.c[e2] * n;
                fl_loc[fd] = ffd;
                sum = sum + fl[lf].F[fd][flux_index(nd, n, fd, v, fl_loc[0], fl_loc[1], fl_loc[2])];
              }
            double mean = sum * (1.0 / (double)(1 << (nd - 1)));
            fl[bi].F[fd][flux_index(nd, n, fd, v, loc[0], loc[1], loc[2])] = mean;
          }
        }
      }
  }
}

// one SSPRK stage: out = alpha*U0 + beta*(Us - dt*div F(Us)); stage 1 when alpha == 0
void stage(orc_grid* g, const std::vector<std::vector<double>>& U0, double alpha, double beta, double dt,
           std::vector<std::vector<double>>* out) {
  const orc_config& C = g->cfg;
  int n = C.block_nx, nd = C.ndim, nv = g->nv;
  size_t nb = g->leaves.size();
  std::vector<BlockFlux> fl(nb);
  // blocks are independent here and below: a parallel run (OpenMP timing build) gives the
  // same result as the serial one, bit for bit
#pragma omp parallel for schedule(static)
  for (size_t bi = 0; bi < nb; ++bi) {
    Padded pd;
    fill_padded(g, (int)bi, &pd);
    block_fluxes(g, &pd, &fl[bi]);
  }
  reflux(g, fl);
  out->assign(nb, std::vector<double>());
#pragma omp parallel for schedule(static)
  for (size_t bi = 0; bi < nb; ++bi) {
    const Leaf& B = g->leaves[bi];
    (*out)[bi].assign((size_t)nv * g->ncell, 0.0);
    double dx[3];
    for (int d = 0; d < 3; ++d) dx[d] = cell_dx(g, B.level, d);
    for (int v = 0; v < nv; ++v)
      for (int k = 0; k < (nd > 2 ? n : 1); ++k)
        for (int j = 0; j < (nd > 1 ? n : 1); ++j)
          for (int i = 0; i < n; ++i) {
            double div = 0.0;
            for (int d = 0; d < nd; ++d) {
              int lo[3] = {i, j, k}, hi[3] = {i, j, k};
              hi[d] += 1;
              double Fp = fl[bi].F[d][flux_index(nd, n, d, v, hi[0], hi[1], hi[2])];
              double Fm = fl[bi].F[d][flux_index(nd, n, d, v, lo[0], lo[1], lo[2])];
              div = div + (Fp - Fm) / dx[d];
            }
            size_t ci = (size_t)v * g->ncell + cell_index(g, i, j, k);
            double tmp = B.U[ci] - dt * div;
            (*out)[bi][ci] = (alpha == 0.0) ? tmp : alpha * U0[bi][ci] + beta * tmp;
          }
  }
}

double max_speed(const orc_grid* g) {
  const orc_config& C = g->cfg;
  int nd = C.ndim, nv = g->nv;
  double smax = 0.0;
  const long long nb = (long long)g->leaves.size();
#pragma omp parallel for schedule(static) reduction(max : smax)
  for (long long bi = 0; bi < nb; ++bi) {
    const Leaf& B = g->leaves[bi];
    double dx[3];
    for (int d = 0; d < 3; ++d) dx[d] = cell_dx(g, B.level, d);
    for (int c = 0; c < g->ncell; ++c) {
      double U[5], V[5];
      for (int v = 0; v < nv; ++v) U[v] = B.U[(size_t)v * g->ncell + c];
      cons_to_prim(nd, C.gamma, U, V);
      double cs = sound_speed(nd, C.gamma, V);
      double s = 0.0;
      for (int d = 0; d < nd; ++d) s = s + (std::fabs(V[1 + d]) + cs) / dx[d];
      smax = std::max(smax, s);
    }
  }
  return smax;
}

// READING (Sec. 1.3 names a Lohner-type estimator of weighted second
// derivatives without the formula): per direction, second difference over
// the sum of the two first differences plus a filter eps*(|q+|+2|q0|+|q-|);
// squares summed over directions, E = sqrt(num/den); max over selected
// primitive variables and over the leaf's cells.
void lohner(const orc_grid* g, std::vector<double>* err) {
  const orc_config& C = g->cfg;
  int n = C.block_nx, nd = C.ndim, nv = g->nv;
  err->assign(g->leaves.size(), 0.0);
#pragma omp parallel for schedule(static)
  for (size_t bi = 0; bi < g->leaves.size(); ++bi) {
    Padded pd;
    fill_padded(g, (int)bi, &pd);
    double emax = 0.0;
    for (int k = 0; k < (nd > 2 ? n : 1); ++k)
      for (int j = 0; j < (nd > 1 ? n : 1); ++j)
        for (int i = 0; i < n; ++i) {
          double Vc[5], Vm[3][5], Vp[3][5];
          double U[5];
          for (int v = 0; v < nv; ++v) U[v] = pd.at(v, i, j, k);
          cons_to_prim(nd, C.gamma, U, Vc);
          for (int d = 0; d < nd; ++d) {
            int m[3] = {i, j, k}, p[3] = {i, j, k};
            m[d] -= 1;
            p[d] += 1;
            for (int v = 0; v < nv; ++v) U[v] = pd.at(v, m[0], m[1], m[2]);
            cons_to_prim(nd, C.gamma, U, Vm[d]);
            for (int v = 0; v < nv; ++v) U[v] = pd.at(v, p[0], p[1], p[2]);
            cons_to_prim(nd, C.gamma, U, Vp[d]);
          }
          double ecell = 0.0;
          for (int v = 0; v < nv; ++v) {
            if (!((C.var_mask >> v) & 1u)) continue;
            double num = 0.0, den = 0.0;
            for (int d = 0; d < nd; ++d) {
              double qm = Vm[d][v], q0 = Vc[v], qp = Vp[d][v];
              double d2 = qp - 2.0 * q0 + qm;
              double d1 = std::fabs(qp - q0) + std::fabs(q0 - qm) +
                          C.wavefilter * (std::fabs(qp) + 2.0 * std::fabs(q0) + std::fabs(qm));
              num = num + d2 * d2;
              den = den + d1 * d1;
            }
            double e = den > 0.0 ? std::sqrt(num / den) : 0.0;
            ecell = std::max(ecell, e);
          }
          emax = std::max(emax, ecell);
        }
    (*err)[bi] = emax;
  }
}

// closed-interval overlap of two blocks, with periodic images
bool touches(const orc_grid* g, const Leaf& A, int lb, const int* cb) {
  const orc_config& C = g->cfg;
  int L = C.max_level;
  for (int d = 0; d < C.ndim; ++d) {
    long loA = (long)A.c[d] << (L - A.level), hiA = (long)(A.c[d] + 1) << (L - A.level);
    long loB = (long)cb[d] << (L - lb), hiB = (long)(cb[d] + 1) << (L - lb);
    long N = (long)C.base[d] << (L - 1);
    bool hit = false;
    for (int s = -1; s <= 1; ++s) {
      if (s != 0 && C.bc[d][0] != ORC_BC_PERIODIC) continue;
      long sh = s * N;
      if (loA <= hiB + sh && loB + sh <= hiA) hit = true;
    }
    if (!hit) return false;
  }
  return true;
}

}  // namespace

// ====================================================================== API

extern "C" {

orc_grid* orc_create(const orc_config* cfg) {
  orc_grid* g = new orc_grid();
  g->cfg = *cfg;
  g->nv = cfg->ndim + 2;
  g->ncell = 1;
  for (int d = 0; d < cfg->ndim; ++d) g->ncell *= cfg->block_nx;
  g->t = 0.0;
  int bz = cfg->ndim > 2 ? cfg->base[2] : 1, by = cfg->ndim > 1 ? cfg->base[1] : 1;
  for (int z = 0; z < bz; ++z)
    for (int y = 0; y < by; ++y)
      for (int x = 0; x < cfg->base[0]; ++x) {
        Leaf l;
        l.level = 1;
        l.c[0] = x;
        l.c[1] = y;
        l.c[2] = z;
        l.U.assign((size_t)g->nv * g->ncell, 0.0);
        g->leaves.push_back(l);
      }
  rebuild_index(g);
  return g;
}

void orc_destroy(orc_grid* g) { delete g; }

int orc_num_leaves(const orc_grid* g) { return (int)g->leaves.size(); }

void orc_leaves(const orc_grid* g, int* level, int* coords) {
  for (size_t i = 0; i < g->leaves.size(); ++i) {
    level[i] = g->leaves[i].level;
    for (int d = 0; d < 3; ++d) coords[3 * i + d] = g->leaves[i].c[d];
  }
}

int orc_set_leaves(orc_grid* g, int n, const int* level, const int* coords) {
  g->leaves.clear();
  for (int i = 0; i < n; ++i) {
    Leaf l;
    l.level = level[i];
    for (int d = 0; d < 3; ++d) l.c[d] = coords[3 * i + d];
    l.U.assign((size_t)g->nv * g->ncell, 0.0);
    g->leaves.push_back(l);
  }
  rebuild_index(g);
  return (int)g->index.size() == n ? 0 : -1;
}

void orc_set_prim(orc_grid* g, const double* V) {
  int nv = g->nv;
  for (size_t b = 0; b < g->leaves.size(); ++b)
    for (int c = 0; c < g->ncell; ++c) {
      double Vc[5], Uc[5];
      for (int v = 0; v < nv; ++v) Vc[v] = V[((size_t)b * nv + v) * g->ncell + c];
      prim_to_cons(g->cfg.ndim, g->cfg.gamma, Vc, Uc);
      for (int v = 0; v < nv; ++v) g->leaves[b].U[(size_t)v * g->ncell + c] = Uc[v];
    }
}

void orc_set_cons(orc_grid* g, const double* U) {
  size_t per = (size_t)g->nv * g->ncell;
  for (size_t b = 0; b < g->leaves.size(); ++b)
    std::memcpy(g->leaves[b].U.data(), U + b * per, per * sizeof(double));
}

void orc_get_cons(const orc_grid* g, double* U) {
  size_t per = (size_t)g->nv * g->ncell;
  for (size_t b = 0; b < g->leaves.size(); ++b)
    std::memcpy(U + b * per, g->leaves[b].U.data(), per * sizeof(double));
}

void orc_set_time(orc_grid* g, double t) { g->t = t; }
double orc_time(const orc_grid* g) { return g->t; }

// Sec. 1.2: dt = CFL / max over cells of sum_d (|v_d| + c)/dx_d.
// READING: the multi-dimensional limit sums the directional rates; the last
// step is shortened to land on t_end.
double orc_dt(const orc_grid* g, double t_end) {
  double smax = max_speed(g);
  double dt = g->cfg.cfl / smax;
  if (g->t + dt > t_end) dt = t_end - g->t;
  return dt;
}

// Sec. 2.3.1 / 2.4 name a three-step SSP Runge-Kutta; READING: Shu-Osher SSPRK3
// (and the two-stage SSPRK2), same dt on all levels.
double orc_step(orc_grid* g, double t_end) {
  double dt = orc_dt(g, t_end);
  if (!(dt > 0.0)) return 0.0;
  size_t nb = g->leaves.size();
  std::vector<std::vector<double>> U0(nb), Ua, Ub;
  for (size_t b = 0; b < nb; ++b) U0[b] = g->leaves[b].U;
  auto load = [g](const std::vector<std::vector<double>>& S) {
    for (size_t b = 0; b < g->leaves.size(); ++b) g->leaves[b].U = S[b];
  };
  stage(g, U0, 0.0, 1.0, dt, &Ua);
  load(Ua);
  if (g->cfg.rk == ORC_SSPRK2) {
    stage(g, U0, 0.5, 0.5, dt, &Ub);
    load(Ub);
  } else {
    stage(g, U0, 0.75, 0.25, dt, &Ub);
    load(Ub);
    std::vector<std::vector<double>> Uc;
    stage(g, U0, 1.0 / 3.0, 2.0 / 3.0, dt, &Uc);
    load(Uc);
  }
  g->t = g->t + dt;
  return dt;
}

void orc_totals(const orc_grid* g, double* tot) {
  int nv = g->nv;
  for (int v = 0; v < nv; ++v) tot[v] = 0.0;
  for (const Leaf& B : g->leaves) {
    double dV = 1.0;
    for (int d = 0; d < g->cfg.ndim; ++d) dV = dV * cell_dx(g, B.level, d);
    for (int v = 0; v < nv; ++v) {
      double s = 0.0;
      for (int c = 0; c < g->ncell; ++c) s = s + B.U[(size_t)v * g->ncell + c];
      tot[v] = tot[v] + s * dV;
    }
  }
}

void orc_lohner(const orc_grid* g, double* err) {
  std::vector<double> e;
  lohner(g, &e);
  for (size_t i = 0; i < e.size(); ++i) err[i] = e[i];
}

void orc_face_ghosts(const orc_grid* g, int leaf, double* out) {
  const Leaf& B = g->leaves[leaf];
  int nd = g->cfg.ndim, nt = ntang(g);
  for (int v = 0; v < g->nv; ++v)
    for (int fd = 0; fd < nd; ++fd)
      for (int side = 0; side < 2; ++side)
        for (int m = 0; m < 2; ++m)
          for (int t = 0; t < nt; ++t) {
            int gi[3];
            face_ghost_cell(g, B, fd, side, m, t, gi);
            size_t o = ((((size_t)v * 2 * nd + (2 * fd + side)) * 2 + m) * nt) + t;
            out[o] = ghost_value(g, leaf, fd, gi, v);
          }
}

// Sec. 1.3: refine a leaf (ratio 2) if one cell's error exceeds refine_tol,
// coarsen a sibling group if every cell of every sibling is below
// coarsen_frac*refine_tol.  READING: 2:1 level balance across faces, edges and
// corners; refinement propagates to coarser touching leaves until balanced; a
// coarsening group is dropped if any touching leaf would end up more than one
// level finer than the new parent.  New children get the limited linear
// prolongation of the parent (parent's face ghosts give the edge slopes), a
// new parent gets the mean of its children.
int orc_regrid(orc_grid* g) {
  const orc_config& C = g->cfg;
  int nd = C.ndim, n = C.block_nx, nv = g->nv;
  size_t nb = g->leaves.size();
  std::vector<double> err;
  lohner(g, &err);
  std::vector<char> ref(nb, 0), crs(nb, 0);
  for (size_t i = 0; i < nb; ++i) {
    int lev = g->leaves[i].level;
    if (lev < C.max_level && err[i] > C.refine_tol) ref[i] = 1;
    if (lev > 1 && err[i] < C.coarsen_frac * C.refine_tol) crs[i] = 1;
  }
  bool changed = true;
  while (changed) {
    changed = false;
    for (size_t i = 0; i < nb; ++i) {
      if (!ref[i]) continue;
      for (size_t j = 0; j < nb; ++j) {
        if (ref[j] || j == i) continue;
        if (g->leaves[j].level < g->leaves[i].level &&
            touches(g, g->leaves[i], g->leaves[j].level, g->leaves[j].c)) {
          ref[j] = 1;
          changed = true;
        }
      }
    }
  }
  // coarsening groups, identified by their first child
  int nchild = 1 << nd;
  std::vector<char> merged(nb, 0);
  std::vector<int> group_first;
  for (size_t i = 0; i < nb; ++i) {
    const Leaf& A = g->leaves[i];
    if (A.level == 1) continue;
    bool first = true;
    for (int d = 0; d < nd; ++d)
      if (A.c[d] & 1) first = false;
    if (!first) continue;
    bool ok = true;
    std::vector<int> kids;
    for (int o = 0; o < nchild && ok; ++o) {
      int c[3] = {A.c[0] + (o & 1), nd > 1 ? A.c[1] + ((o >> 1) & 1) : 0, nd > 2 ? A.c[2] + ((o >> 2) & 1) : 0};
      int li = find_leaf(g, A.level, c);
      if (li < 0 || ref[li] || !crs[li]) ok = false;
      kids.push_back(li);
    }
    if (!ok) continue;
    int pc[3] = {A.c[0] >> 1, A.c[1] >> 1, A.c[2] >> 1};
    for (size_t j = 0; j < nb && ok; ++j) {
      const Leaf& Bj = g->leaves[j];
      int newlev = Bj.level + (ref[j] ? 1 : 0);
      Leaf P;
      P.level = A.level - 1;
      P.c[0] = pc[0];
      P.c[1] = pc[1];
      P.c[2] = pc[2];
      if (newlev > P.level + 1 && touches(g, P, Bj.level, Bj.c)) ok = false;
    }
    if (!ok) continue;
    group_first.push_back((int)i);
    for (int li : kids) merged[li] = 1;
  }
  // build the new leaf set
  std::vector<Leaf> out;
  // prolongation needs the old tree's face ghosts
  for (size_t i = 0; i < nb; ++i) {
    const Leaf& B = g->leaves[i];
    if (ref[i]) {
      Padded pd;
      fill_padded(g, (int)i, &pd);
      for (int o = 0; o < nchild; ++o) {
        int oo[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
        Leaf ch;
        ch.level = B.level + 1;
        for (int d = 0; d < 3; ++d) ch.c[d] = d < nd ? 2 * B.c[d] + oo[d] : 0;
        ch.U.assign((size_t)nv * g->ncell, 0.0);
        for (int k = 0; k < (nd > 2 ? n : 1); ++k)
          for (int j = 0; j < (nd > 1 ? n : 1); ++j)
            for (int ii = 0; ii < n; ++ii) {
              int fi[3] = {ii, j, k};
              int pcell[3] = {0, 0, 0};
              for (int d = 0; d < nd; ++d) pcell[d] = (oo[d] * n + fi[d]) >> 1;
              for (int v = 0; v < nv; ++v) {
                double qp = pd.at(v, pcell[0], pcell[1], pcell[2]);
                double acc = 0.0;
                for (int e = 0; e < nd; ++e) {
                  int m[3] = {pcell[0], pcell[1], pcell[2]}, p[3] = {pcell[0], pcell[1], pcell[2]};
                  m[e] -= 1;
                  p[e] += 1;
                  double s = minmod2(qp - pd.at(v, m[0], m[1], m[2]), pd.at(v, p[0], p[1], p[2]) - qp);
                  double sigma = ((oo[e] * n + fi[e]) & 1) ? 1.0 : -1.0;
                  acc = acc + sigma * s;
                }
                ch.U[(size_t)v * g->ncell + cell_index(g, ii, j, k)] = qp + 0.25 * acc;
              }
            }
        out.push_back(ch);
      }
    } else if (!merged[i]) {
      out.push_back(B);
    }
  }
  for (int fi : group_first) {
    const Leaf& A = g->leaves[fi];
    Leaf P;
    P.level = A.level - 1;
    for (int d = 0; d < 3; ++d) P.c[d] = A.c[d] >> 1;
    P.U.assign((size_t)nv * g->ncell, 0.0);
    for (int k = 0; k < (nd > 2 ? n : 1); ++k)
      for (int j = 0; j < (nd > 1 ? n : 1); ++j)
        for (int i = 0; i < n; ++i) {
          int pc[3] = {i, j, k};
          // global coarse cell on P's level
          int gc[3] = {0, 0, 0};
          for (int d = 0; d < nd; ++d) gc[d] = P.c[d] * n + pc[d];
          int child[3] = {0, 0, 0};
          for (int d = 0; d < nd; ++d) child[d] = (2 * gc[d]) / n;
          int li = find_leaf(g, A.level, child);
          for (int v = 0; v < nv; ++v)
            P.U[(size_t)v * g->ncell + cell_index(g, i, j, k)] = restrict_cell(g, li, gc, v);
        }
    out.push_back(P);
  }
  g->leaves.swap(out);
  rebuild_index(g);
  return (int)g->leaves.size();
}

// threads of the OpenMP loops over blocks and cells (1 without OpenMP); 0 leaves the default
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void orc_prim_to_cons(int ndim, double gamma, const double* V, double* U) { prim_to_cons(ndim, gamma, V, U); }
void orc_cons_to_prim(int ndim, double gamma, const double* U, double* V) { cons_to_prim(ndim, gamma, U, V); }
void orc_phys_flux(int ndim, int dir, double gamma, const double* V, double* F) {
  phys_flux(ndim, dir, gamma, V, F);
}
void orc_riemann_flux(int ndim, int dir, int flux, double gamma, const double* VL, const double* VR, double* F) {
  riemann_flux(ndim, dir, flux, gamma, VL, VR, F);
}
void orc_limited_slopes(int limiter, double a, double b, double* sm, double* sp) {
  limited_slopes(limiter, a, b, sm, sp);
}

}  // extern "C"
