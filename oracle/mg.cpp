// FP64 oracle: geometric multigrid for the Helmholtz problem of the implicit
// diffusion step, and the reaction-diffusion steps that use it.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Paper: Sec. 2.5.1, Eq. (diff-helmholtz) writes the implicit diffusion stage as
// a Helmholtz problem solved by geometric multigrid with linear cost (Sec. 1.4,
// mg2019); Eq. (imex) is the IMEX trapezoidal scheme and Eq. (splitting) the
// split scheme; Eqs. (gray-scott) and (schnakenberg) give the reaction terms.
// Sec. 2.5.2 states the stopping rule as the maximum residual relative to the
// right-hand side, and uses zero-flux (Neumann) boundaries for Schnakenberg.
//
// READING (the paper does not define the cycle; mg2019 is cited): cell-centred
// 5/7-point Laplacian, red-black Gauss-Seidel smoother (red = even i+j+k first),
// restriction = mean of the 2^ndim children, prolongation = cell-centred
// (bi/tri)linear interpolation, nu1 pre- and nu2 post-sweeps, coarsen while the
// side is even and above coarse_max, exact (dense) solve on the coarsest grid.
// Neumann boundaries: a boundary face carries no flux, so a boundary cell's
// Laplacian sums only its in-domain neighbours, (sum - count x) / h^2, on every
// level; Gauss-Seidel divides by lambda + count / h^2; the prolongation puts the
// weight of an out-of-domain coarse neighbour on the parent (zero gradient).
#include <cmath>
#include <cstring>
#include <vector>

#include "oracle.h"

namespace {

struct Grid {
  int nd, n;
  double h;
  int bc;  // ORC_MG_PERIODIC or ORC_MG_NEUMANN
  size_t size() const {
    size_t s = 1;
    for (int d = 0; d < nd; ++d) s *= (size_t)n;
    return s;
  }
};

inline int wrapi(int i, int n) { return (i % n + n) % n; }

inline size_t idx(const Grid& g, int i, int j, int k) {
  return (size_t)i + (size_t)g.n * ((size_t)j + (size_t)g.n * (size_t)k);
}

// the neighbour index i (at most one cell outside [0, n)): its periodic image, or -1
// beyond a Neumann boundary
inline int nbr(const Grid& g, int i) {
  if (i >= 0 && i < g.n) return i;
  return g.bc == ORC_MG_NEUMANN ? -1 : wrapi(i, g.n);
}

// sum of the neighbours inside the domain, ordered x-, x+, y-, y+, z-, z+, and their
// number (2 ndim on a periodic grid)
inline double nbsum(const Grid& g, const double* x, int i, int j, int k, int* count) {
  double s = 0.0;
  int m = 0;
  for (int d = 0; d < g.nd; ++d)
    for (int side = -1; side <= 1; side += 2) {
      int q[3] = {i, j, k};
      q[d] = nbr(g, q[d] + side);
      if (q[d] < 0) continue;
      s = s + x[idx(g, q[0], q[1], q[2])];
      ++m;
    }
  *count = m;
  return s;
}

// discrete Laplacian (sum of neighbours - count x) / h^2: the net diffusive flux through
// the cell's faces, none through a Neumann boundary face
void laplacian(const Grid& g, const double* x, double* out) {
  double ih2 = 1.0 / (g.h * g.h);
  int nz = g.nd > 2 ? g.n : 1, ny = g.nd > 1 ? g.n : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < g.n; ++i) {
        size_t c = idx(g, i, j, k);
        int m;
        double s = nbsum(g, x, i, j, k, &m);
        out[c] = (s - (double)m * x[c]) * ih2;
      }
}

// r = b - (lambda x - lap x)
void residual(const Grid& g, double lambda, const double* x, const double* b, double* r) {
  double ih2 = 1.0 / (g.h * g.h);
  int nz = g.nd > 2 ? g.n : 1, ny = g.nd > 1 ? g.n : 1;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < g.n; ++i) {
        size_t c = idx(g, i, j, k);
        int m;
        double s = nbsum(g, x, i, j, k, &m);
        double lap = (s - (double)m * x[c]) * ih2;
        r[c] = b[c] - (lambda * x[c] - lap);
      }
}

// one red-black Gauss-Seidel sweep: each cell solves its own row of (lambda - lap_h)
void rbgs(const Grid& g, double lambda, double* x, const double* b) {
  double ih2 = 1.0 / (g.h * g.h);
  int nz = g.nd > 2 ? g.n : 1, ny = g.nd > 1 ? g.n : 1;
  for (int colour = 0; colour < 2; ++colour)
    // a cell of one colour reads only cells of the other: any order within a colour (OpenMP
    // timing build) gives the same sweep
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < g.n; ++i) {
          if (((i + j + k) & 1) != colour) continue;
          size_t c = idx(g, i, j, k);
          int m;
          double s = nbsum(g, x, i, j, k, &m);
          x[c] = (b[c] + s * ih2) / (lambda + (double)m * ih2);
        }
}

void restrict_mean(const Grid& f, const Grid& c, const double* rf, double* bc) {
  int nz = c.nd > 2 ? c.n : 1, ny = c.nd > 1 ? c.n : 1;
  int oz = c.nd > 2 ? 2 : 1, oy = c.nd > 1 ? 2 : 1;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < c.n; ++i) {
        double s = 0.0;
        for (int z = 0; z < oz; ++z)
          for (int y = 0; y < oy; ++y)
            for (int x = 0; x < 2; ++x)
              s = s + rf[idx(f, 2 * i + x, c.nd > 1 ? 2 * j + y : 0, c.nd > 2 ? 2 * k + z : 0)];
        bc[idx(c, i, j, k)] = s * (1.0 / (double)(1 << c.nd));
      }
}

// cell-centred linear interpolation: per dimension weight 3/4 on the parent,
// 1/4 on the parent's neighbour on the child's side (the parent itself where that
// neighbour is beyond a Neumann boundary); corners in x-fastest order
void prolong_add(const Grid& c, const Grid& f, const double* ec, double* xf) {
  int nz = f.nd > 2 ? f.n : 1, ny = f.nd > 1 ? f.n : 1;
  int cz = f.nd > 2 ? 2 : 1, cy = f.nd > 1 ? 2 : 1;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < f.n; ++i) {
        int P[3] = {i >> 1, j >> 1, k >> 1};
        int S[3] = {(i & 1) ? 1 : -1, (j & 1) ? 1 : -1, (k & 1) ? 1 : -1};
        double acc = 0.0;
        for (int z = 0; z < cz; ++z)
          for (int y = 0; y < cy; ++y)
            for (int x = 0; x < 2; ++x) {
              int q[3] = {P[0] + x * S[0], f.nd > 1 ? P[1] + y * S[1] : 0, f.nd > 2 ? P[2] + z * S[2] : 0};
              for (int d = 0; d < f.nd; ++d) {
                int t = nbr(c, q[d]);
                q[d] = t < 0 ? P[d] : t;
              }
              double w = (x ? 0.25 : 0.75);
              if (f.nd > 1) w = w * (y ? 0.25 : 0.75);
              if (f.nd > 2) w = w * (z ? 0.25 : 0.75);
              acc = acc + w * ec[idx(c, q[0], q[1], q[2])];
            }
        size_t fc = idx(f, i, j, k);
        xf[fc] = xf[fc] + acc;
      }
}

// dense matrix of (lambda - lap_h): row r has lambda + count / h^2 on the diagonal and
// -1/h^2 for each in-domain neighbour (periodic images included)
void dense_matrix(const Grid& g, double lambda, std::vector<double>* A) {
  size_t N = g.size();
  A->assign(N * N, 0.0);
  double ih2 = 1.0 / (g.h * g.h);
  int nz = g.nd > 2 ? g.n : 1, ny = g.nd > 1 ? g.n : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < g.n; ++i) {
        size_t r = idx(g, i, j, k);
        int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
        int m = 0;
        for (int q = 0; q < 2 * g.nd; ++q) {
          int a = nbr(g, nb[q][0]), b = g.nd > 1 ? nbr(g, nb[q][1]) : 0, c3 = g.nd > 2 ? nbr(g, nb[q][2]) : 0;
          if (a < 0 || b < 0 || c3 < 0) continue;
          (*A)[r * N + idx(g, a, b, c3)] -= ih2;
          ++m;
        }
        (*A)[r * N + r] += lambda + (double)m * ih2;
      }
}

// Gaussian elimination with partial pivoting
int gauss_solve(size_t N, std::vector<double> A, const double* b, double* x) {
  std::vector<double> rhs(b, b + N);
  for (size_t col = 0; col < N; ++col) {
    size_t piv = col;
    for (size_t r = col + 1; r < N; ++r)
      if (std::fabs(A[r * N + col]) > std::fabs(A[piv * N + col])) piv = r;
    if (A[piv * N + col] == 0.0) return -1;
    if (piv != col) {
      for (size_t c = 0; c < N; ++c) std::swap(A[piv * N + c], A[col * N + c]);
      std::swap(rhs[piv], rhs[col]);
    }
    for (size_t r = col + 1; r < N; ++r) {
      double f = A[r * N + col] / A[col * N + col];
      if (f == 0.0) continue;
      for (size_t c = col; c < N; ++c) A[r * N + c] -= f * A[col * N + c];
      rhs[r] -= f * rhs[col];
    }
  }
  for (size_t r = N; r-- > 0;) {
    double s = rhs[r];
    for (size_t c = r + 1; c < N; ++c) s -= A[r * N + c] * x[c];
    x[r] = s / A[r * N + r];
  }
  return 0;
}

struct Hierarchy {
  std::vector<Grid> lv;
  double lambda;
  int nu1, nu2;
};

Hierarchy make_hierarchy(int nd, int n, double L, double lambda, int nu1, int nu2, int coarse_max, int bc) {
  Hierarchy H;
  H.lambda = lambda;
  H.nu1 = nu1;
  H.nu2 = nu2;
  int m = n;
  while (true) {
    Grid g{nd, m, L / (double)m, bc};
    H.lv.push_back(g);
    if ((m & 1) || m <= coarse_max) break;
    m /= 2;
  }
  return H;
}

void vcycle(const Hierarchy& H, size_t l, const double* b, double* x) {
  const Grid& g = H.lv[l];
  if (l + 1 == H.lv.size()) {
    std::vector<double> A;
    dense_matrix(g, H.lambda, &A);
    gauss_solve(g.size(), A, b, x);
    return;
  }
  for (int s = 0; s < H.nu1; ++s) rbgs(g, H.lambda, x, b);
  std::vector<double> r(g.size());
  residual(g, H.lambda, x, b, r.data());
  const Grid& c = H.lv[l + 1];
  std::vector<double> bc(c.size()), ec(c.size(), 0.0);
  restrict_mean(g, c, r.data(), bc.data());
  vcycle(H, l + 1, bc.data(), ec.data());
  prolong_add(c, g, ec.data(), x);
  for (int s = 0; s < H.nu2; ++s) rbgs(g, H.lambda, x, b);
}

double maxabs(const double* a, size_t n) {
  double m = 0.0;
  for (size_t i = 0; i < n; ++i) m = std::fmax(m, std::fabs(a[i]));
  return m;
}

// reaction terms F0 at one cell: Eq. (gray-scott) F0_u = -u v^2 + F (1 - u),
// F0_v = u v^2 - (F + k) v; Eq. (schnakenberg) F0_u = kappa (a - u + u^2 v),
// F0_v = kappa (b - u^2 v)
void reaction(const orc_rd_config* c, double u, double v, double* fu, double* fv) {
  if (c->model == ORC_RD_SCHNAKENBERG) {
    double uuv = (u * u) * v;
    *fu = c->kappa * ((c->a - u) + uuv);
    *fv = c->kappa * (c->b - uuv);
  } else {
    double uvv = (u * v) * v;
    *fu = -uvv + c->F * (1.0 - u);
    *fv = uvv - (c->F + c->k) * v;
  }
}

// full right-hand side F(w) = F0(w) + D lap_h w of both species
void rd_rhs(const orc_rd_config* c, const Grid& g, const double* u, const double* v, double* Fu, double* Fv) {
  size_t N = g.size();
  std::vector<double> lu(N), lv(N);
  laplacian(g, u, lu.data());
  laplacian(g, v, lv.data());
  for (size_t i = 0; i < N; ++i) {
    double fu, fv;
    reaction(c, u[i], v[i], &fu, &fv);
    Fu[i] = fu + c->Du * lu[i];
    Fv[i] = fv + c->Dv * lv[i];
  }
}

}  // namespace

extern "C" {

void orc_mg_apply(int ndim, int n, double L, double lambda, int bc, const double* x, double* Ax) {
  Grid g{ndim, n, L / (double)n, bc};
  std::vector<double> zero(g.size(), 0.0), r(g.size());
  residual(g, lambda, x, zero.data(), r.data());
  for (size_t i = 0; i < g.size(); ++i) Ax[i] = -r[i];
}

void orc_laplacian(int ndim, int n, double L, int bc, const double* x, double* out) {
  Grid g{ndim, n, L / (double)n, bc};
  laplacian(g, x, out);
}

void orc_mg_vcycle(const orc_mg_config* c, const double* r, double* e) {
  Hierarchy H = make_hierarchy(c->ndim, c->n, c->L, c->lambda, c->nu1, c->nu2, c->coarse_max, c->bc);
  std::memset(e, 0, sizeof(double) * H.lv[0].size());
  vcycle(H, 0, r, e);
}

int orc_mg_solve(const orc_mg_config* c, const double* b, double* x, double* relres) {
  Hierarchy H = make_hierarchy(c->ndim, c->n, c->L, c->lambda, c->nu1, c->nu2, c->coarse_max, c->bc);
  const Grid& g = H.lv[0];
  size_t N = g.size();
  std::vector<double> r(N);
  double bn = maxabs(b, N);
  residual(g, c->lambda, x, b, r.data());
  double rn = maxabs(r.data(), N);
  int cycles = 0;
  while (rn > c->rtol * bn && cycles < c->max_cycles) {
    vcycle(H, 0, b, x);
    ++cycles;
    residual(g, c->lambda, x, b, r.data());
    rn = maxabs(r.data(), N);
  }
  if (relres) *relres = bn > 0.0 ? rn / bn : rn;
  return rn <= c->rtol * bn ? cycles : -1;
}

int orc_dense_solve(int ndim, int n, double L, double lambda, int bc, const double* b, double* x) {
  Grid g{ndim, n, L / (double)n, bc};
  std::vector<double> A;
  dense_matrix(g, lambda, &A);
  return gauss_solve(g.size(), A, b, x);
}

void orc_rd_reaction(double F, double k, int n, const double* u, const double* v, double* fu, double* fv) {
  orc_rd_config c{};
  c.model = ORC_RD_GRAY_SCOTT;
  c.F = F;
  c.k = k;
  for (int i = 0; i < n; ++i) reaction(&c, u[i], v[i], &fu[i], &fv[i]);
}

void orc_rd_reaction_schnakenberg(double kappa, double a, double b, int n, const double* u, const double* v,
                                  double* fu, double* fv) {
  orc_rd_config c{};
  c.model = ORC_RD_SCHNAKENBERG;
  c.kappa = kappa;
  c.a = a;
  c.b = b;
  for (int i = 0; i < n; ++i) reaction(&c, u[i], v[i], &fu[i], &fv[i]);
}

// One step of the configured scheme (Sec. 2.5.1).
//  IMEX, Eq. (imex): w* = w_n + dt F0(w_n) + dt/2 [F1(w_n) + F1(w*)] (Helmholtz solve with
//    lambda = 2/(dt D) and right-hand side lambda g, g = w_n + dt F0(w_n) + dt/2 D lap w_n),
//    then w_{n+1} = w_n + dt/2 [F(w_n) + F(w*)].  READING: the multigrid initial guess is
//    w_n; the Laplacian of w* is evaluated with the same stencil.
//  Split, Eqs. (splitting), (diff-helmholtz): w* = w_n + dt F0(w_n), then backward Euler
//    w_{n+1} = w* + dt F1(w_{n+1}), i.e. (lambda - lap) w_{n+1} = lambda w* with
//    lambda = 1/(dt D).  READING: the reaction is advanced by forward Euler (the paper
//    says only that it is handled explicitly); the multigrid initial guess is w*.
//  Explicit: READING: the three-stage SSP Runge-Kutta scheme of the hydrodynamic steps
//    (Sec. 2.4) on F = F0 + F1 (the paper's reference solution uses an explicit
//    third-order scheme): w1 = w + dt F(w), w2 = 3/4 w + 1/4 (w1 + dt F(w1)),
//    w_{n+1} = 1/3 w + 2/3 (w2 + dt F(w2)).
int orc_rd_step(const orc_rd_config* c, double* u, double* v, int* cycles) {
  Grid g{c->ndim, c->n, c->L / (double)c->n, c->bc};
  size_t N = g.size();
  double D[2] = {c->Du, c->Dv};
  double* w[2] = {u, v};
  if (cycles) cycles[0] = cycles[1] = 0;
  if (c->scheme == ORC_RD_EXPLICIT) {
    std::vector<double> Fu(N), Fv(N), u1(N), v1(N), u2(N), v2(N);
    rd_rhs(c, g, u, v, Fu.data(), Fv.data());
    for (size_t i = 0; i < N; ++i) {
      u1[i] = u[i] + c->dt * Fu[i];
      v1[i] = v[i] + c->dt * Fv[i];
    }
    rd_rhs(c, g, u1.data(), v1.data(), Fu.data(), Fv.data());
    for (size_t i = 0; i < N; ++i) {
      u2[i] = 0.75 * u[i] + 0.25 * (u1[i] + c->dt * Fu[i]);
      v2[i] = 0.75 * v[i] + 0.25 * (v1[i] + c->dt * Fv[i]);
    }
    rd_rhs(c, g, u2.data(), v2.data(), Fu.data(), Fv.data());
    for (size_t i = 0; i < N; ++i) {
      u[i] = (1.0 / 3.0) * u[i] + (2.0 / 3.0) * (u2[i] + c->dt * Fu[i]);
      v[i] = (1.0 / 3.0) * v[i] + (2.0 / 3.0) * (v2[i] + c->dt * Fv[i]);
    }
    return 0;
  }
  std::vector<double> fu(N), fv(N);
  for (size_t i = 0; i < N; ++i) reaction(c, u[i], v[i], &fu[i], &fv[i]);
  std::vector<double>* R[2] = {&fu, &fv};
  int status = 0;
  if (c->scheme == ORC_RD_SPLIT) {
    for (int s = 0; s < 2; ++s) {
      double lambda = 1.0 / (c->dt * D[s]);
      std::vector<double> ws(N), b(N);
      for (size_t i = 0; i < N; ++i) {
        ws[i] = w[s][i] + c->dt * (*R[s])[i];
        b[i] = lambda * ws[i];
      }
      orc_mg_config mc{c->ndim, c->n, c->L, lambda, c->nu1, c->nu2, c->max_cycles, c->rtol, c->coarse_max, c->bc};
      double rr;
      int cyc = orc_mg_solve(&mc, b.data(), ws.data(), &rr);
      if (cycles) cycles[s] = cyc;
      if (cyc < 0) status = -1;
      std::memcpy(w[s], ws.data(), N * sizeof(double));
    }
    return status;
  }
  std::vector<double> lu(N), lv(N);
  laplacian(g, u, lu.data());
  laplacian(g, v, lv.data());
  std::vector<double>* Lp[2] = {&lu, &lv};
  std::vector<double> ws[2];
  for (int s = 0; s < 2; ++s) {
    double lambda = 2.0 / (c->dt * D[s]);
    std::vector<double> b(N);
    for (size_t i = 0; i < N; ++i) {
      double gi = (w[s][i] + c->dt * (*R[s])[i]) + ((0.5 * c->dt) * D[s]) * (*Lp[s])[i];
      b[i] = lambda * gi;
    }
    ws[s].assign(w[s], w[s] + N);
    orc_mg_config mc{c->ndim, c->n, c->L, lambda, c->nu1, c->nu2, c->max_cycles, c->rtol, c->coarse_max, c->bc};
    double rr;
    int cyc = orc_mg_solve(&mc, b.data(), ws[s].data(), &rr);
    if (cycles) cycles[s] = cyc;
    if (cyc < 0) status = -1;
  }
  std::vector<double> fus(N), fvs(N), lus(N), lvs(N);
  for (size_t i = 0; i < N; ++i) reaction(c, ws[0][i], ws[1][i], &fus[i], &fvs[i]);
  laplacian(g, ws[0].data(), lus.data());
  laplacian(g, ws[1].data(), lvs.data());
  std::vector<double>* Rs[2] = {&fus, &fvs};
  std::vector<double>* Ls[2] = {&lus, &lvs};
  for (int s = 0; s < 2; ++s)
    for (size_t i = 0; i < N; ++i) {
      double Fn = (*R[s])[i] + D[s] * (*Lp[s])[i];
      double Fs = (*Rs[s])[i] + D[s] * (*Ls[s])[i];
      w[s][i] = w[s][i] + (0.5 * c->dt) * (Fn + Fs);
    }
  return status;
}

}  // extern "C"
