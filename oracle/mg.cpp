// FP64 oracle: geometric multigrid for the Helmholtz problem of the implicit
// diffusion step, and the Gray-Scott IMEX step that uses it.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Paper: Sec. 2.5.1, Eq. (diff-helmholtz) writes the implicit diffusion stage as
// a Helmholtz problem solved by geometric multigrid with linear cost (Sec. 1.4,
// mg2019); Eq. (imex) is the IMEX trapezoidal scheme; Eq. (gray-scott) gives
// the reaction terms.  Sec. 2.5.2 states the stopping rule as the maximum
// residual relative to the right-hand side.
//
// READING (the paper does not define the cycle; mg2019 is cited): cell-centred
// 5/7-point Laplacian on a periodic grid, red-black Gauss-Seidel smoother (red =
// even i+j+k first), restriction = mean of the 2^ndim children, prolongation =
// cell-centred (bi/tri)linear interpolation, nu1 pre- and nu2 post-sweeps,
// coarsen while the side is even and above coarse_max, exact (dense) solve on
// the coarsest grid.
#include <cmath>
#include <cstring>
#include <vector>

#include "oracle.h"

namespace {

struct Grid {
  int nd, n;
  double h;
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

// sum of the 2*ndim neighbours, ordered x-, x+, y-, y+, z-, z+
inline double nbsum(const Grid& g, const double* x, int i, int j, int k) {
  int n = g.n;
  double s = x[idx(g, wrapi(i - 1, n), j, k)] + x[idx(g, wrapi(i + 1, n), j, k)];
  if (g.nd > 1) s = s + x[idx(g, i, wrapi(j - 1, n), k)] + x[idx(g, i, wrapi(j + 1, n), k)];
  if (g.nd > 2) s = s + x[idx(g, i, j, wrapi(k - 1, n))] + x[idx(g, i, j, wrapi(k + 1, n))];
  return s;
}

// discrete Laplacian (sum of neighbours - 2 ndim x) / h^2
void laplacian(const Grid& g, const double* x, double* out) {
  double ih2 = 1.0 / (g.h * g.h);
  int nz = g.nd > 2 ? g.n : 1, ny = g.nd > 1 ? g.n : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < g.n; ++i) {
        size_t c = idx(g, i, j, k);
        out[c] = (nbsum(g, x, i, j, k) - (2.0 * g.nd) * x[c]) * ih2;
      }
}

// r = b - (lambda x - lap x)
void residual(const Grid& g, double lambda, const double* x, const double* b, double* r) {
  double ih2 = 1.0 / (g.h * g.h);
  int nz = g.nd > 2 ? g.n : 1, ny = g.nd > 1 ? g.n : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < g.n; ++i) {
        size_t c = idx(g, i, j, k);
        double lap = (nbsum(g, x, i, j, k) - (2.0 * g.nd) * x[c]) * ih2;
        r[c] = b[c] - (lambda * x[c] - lap);
      }
}

void rbgs(const Grid& g, double lambda, double* x, const double* b) {
  double ih2 = 1.0 / (g.h * g.h);
  double diag = lambda + (2.0 * g.nd) * ih2;
  int nz = g.nd > 2 ? g.n : 1, ny = g.nd > 1 ? g.n : 1;
  for (int colour = 0; colour < 2; ++colour)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < g.n; ++i) {
          if (((i + j + k) & 1) != colour) continue;
          size_t c = idx(g, i, j, k);
          x[c] = (b[c] + nbsum(g, x, i, j, k) * ih2) / diag;
        }
}

void restrict_mean(const Grid& f, const Grid& c, const double* rf, double* bc) {
  int nz = c.nd > 2 ? c.n : 1, ny = c.nd > 1 ? c.n : 1;
  int oz = c.nd > 2 ? 2 : 1, oy = c.nd > 1 ? 2 : 1;
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
// 1/4 on the parent's neighbour on the child's side; corners in x-fastest order
void prolong_add(const Grid& c, const Grid& f, const double* ec, double* xf) {
  int nz = f.nd > 2 ? f.n : 1, ny = f.nd > 1 ? f.n : 1;
  int cz = f.nd > 2 ? 2 : 1, cy = f.nd > 1 ? 2 : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < f.n; ++i) {
        int P[3] = {i >> 1, j >> 1, k >> 1};
        int S[3] = {(i & 1) ? 1 : -1, (j & 1) ? 1 : -1, (k & 1) ? 1 : -1};
        double acc = 0.0;
        for (int z = 0; z < cz; ++z)
          for (int y = 0; y < cy; ++y)
            for (int x = 0; x < 2; ++x) {
              int q[3] = {wrapi(P[0] + x * S[0], c.n), f.nd > 1 ? wrapi(P[1] + y * S[1], c.n) : 0,
                          f.nd > 2 ? wrapi(P[2] + z * S[2], c.n) : 0};
              double w = (x ? 0.25 : 0.75);
              if (f.nd > 1) w = w * (y ? 0.25 : 0.75);
              if (f.nd > 2) w = w * (z ? 0.25 : 0.75);
              acc = acc + w * ec[idx(c, q[0], q[1], q[2])];
            }
        size_t fc = idx(f, i, j, k);
        xf[fc] = xf[fc] + acc;
      }
}

// dense matrix of (lambda - lap_h) on the periodic grid
void dense_matrix(const Grid& g, double lambda, std::vector<double>* A) {
  size_t N = g.size();
  A->assign(N * N, 0.0);
  double ih2 = 1.0 / (g.h * g.h);
  int nz = g.nd > 2 ? g.n : 1, ny = g.nd > 1 ? g.n : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < g.n; ++i) {
        size_t r = idx(g, i, j, k);
        (*A)[r * N + r] += lambda + (2.0 * g.nd) * ih2;
        int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
        for (int q = 0; q < 2 * g.nd; ++q) {
          size_t c = idx(g, wrapi(nb[q][0], g.n), g.nd > 1 ? wrapi(nb[q][1], g.n) : 0,
                         g.nd > 2 ? wrapi(nb[q][2], g.n) : 0);
          (*A)[r * N + c] -= ih2;
        }
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

Hierarchy make_hierarchy(int nd, int n, double L, double lambda, int nu1, int nu2, int coarse_max) {
  Hierarchy H;
  H.lambda = lambda;
  H.nu1 = nu1;
  H.nu2 = nu2;
  int m = n;
  while (true) {
    Grid g{nd, m, L / (double)m};
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

}  // namespace

extern "C" {

void orc_mg_apply(int ndim, int n, double L, double lambda, const double* x, double* Ax) {
  Grid g{ndim, n, L / (double)n};
  std::vector<double> zero(g.size(), 0.0), r(g.size());
  residual(g, lambda, x, zero.data(), r.data());
  for (size_t i = 0; i < g.size(); ++i) Ax[i] = -r[i];
}

void orc_laplacian(int ndim, int n, double L, const double* x, double* out) {
  Grid g{ndim, n, L / (double)n};
  laplacian(g, x, out);
}

void orc_mg_vcycle(const orc_mg_config* c, const double* r, double* e) {
  Hierarchy H = make_hierarchy(c->ndim, c->n, c->L, c->lambda, c->nu1, c->nu2, c->coarse_max);
  std::memset(e, 0, sizeof(double) * H.lv[0].size());
  vcycle(H, 0, r, e);
}

int orc_mg_solve(const orc_mg_config* c, const double* b, double* x, double* relres) {
  Hierarchy H = make_hierarchy(c->ndim, c->n, c->L, c->lambda, c->nu1, c->nu2, c->coarse_max);
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

int orc_dense_solve(int ndim, int n, double L, double lambda, const double* b, double* x) {
  Grid g{ndim, n, L / (double)n};
  std::vector<double> A;
  dense_matrix(g, lambda, &A);
  return gauss_solve(g.size(), A, b, x);
}

// Eq. (gray-scott): F0_u = -u v^2 + F (1 - u), F0_v = u v^2 - (F + k) v
void orc_rd_reaction(double F, double k, int n, const double* u, const double* v, double* fu,
                     double* fv) {
  for (int i = 0; i < n; ++i) {
    double uvv = (u[i] * v[i]) * v[i];
    fu[i] = -uvv + F * (1.0 - u[i]);
    fv[i] = uvv - (F + k) * v[i];
  }
}

// Eq. (imex): w* = w_n + dt F0(w_n) + dt/2 [F1(w_n) + F1(w*)]  (Helmholtz solve with
// lambda = 2/(dt D) and right-hand side lambda g, g = w_n + dt F0(w_n) + dt/2 D lap w_n),
// then w_{n+1} = w_n + dt/2 [F(w_n) + F(w*)].  READING: the multigrid initial guess is
// w_n; the Laplacian of w* is evaluated with the same stencil.
int orc_rd_step(const orc_rd_config* c, double* u, double* v, int* cycles) {
  Grid g{c->ndim, c->n, c->L / (double)c->n};
  size_t N = g.size();
  std::vector<double> fu(N), fv(N), lu(N), lv(N);
  orc_rd_reaction(c->F, c->k, (int)N, u, v, fu.data(), fv.data());
  laplacian(g, u, lu.data());
  laplacian(g, v, lv.data());
  double D[2] = {c->Du, c->Dv};
  double* w[2] = {u, v};
  std::vector<double>* R[2] = {&fu, &fv};
  std::vector<double>* Lp[2] = {&lu, &lv};
  std::vector<double> ws[2];
  int status = 0;
  for (int s = 0; s < 2; ++s) {
    double lambda = 2.0 / (c->dt * D[s]);
    std::vector<double> b(N);
    for (size_t i = 0; i < N; ++i) {
      double gi = (w[s][i] + c->dt * (*R[s])[i]) + ((0.5 * c->dt) * D[s]) * (*Lp[s])[i];
      b[i] = lambda * gi;
    }
    ws[s].assign(w[s], w[s] + N);
    orc_mg_config mc{c->ndim, c->n, c->L, lambda, c->nu1, c->nu2, c->max_cycles, c->rtol, c->coarse_max};
    double rr;
    int cyc = orc_mg_solve(&mc, b.data(), ws[s].data(), &rr);
    if (cycles) cycles[s] = cyc;
    if (cyc < 0) status = -1;
  }
  std::vector<double> fus(N), fvs(N), lus(N), lvs(N);
  orc_rd_reaction(c->F, c->k, (int)N, ws[0].data(), ws[1].data(), fus.data(), fvs.data());
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
