/*
 * FP64 CPU oracle for the block-AMR finite-volume Euler update, the Helmholtz
 * multigrid solve and the Gray-Scott IMEX step of MPI-AMRVAC
 * (Keppens, Teunissen, Xia, Porth, arXiv:2004.03275).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or helper with the CUDA library; the two only see the
 * same seeded inputs.
 *
 * Everything is double precision, single threaded, compiled without FMA
 * contraction (-ffp-contract=off) so that every rounding step is the one
 * written in the source.
 *
 * Paper passages followed (section / equation):
 *   Sec. 1.1, Eq. (eq)      conservation law dU/dt + div F(U) = S
 *   Sec. 1.1                HD variables U=(rho, rho v, E), E = rho v^2/2 + p/(gamma-1),
 *                           primitive V=(rho, v, p); flux = advective vU + non-advective part
 *   Sec. 1.2                phys_get_cmax / phys_get_cbounds: CFL limit, TVDLF and HLL fluxes
 *   Sec. 2.3 / 2.4          HLLC flux, Koren limiter, three-step (SSP) Runge-Kutta
 *   Sec. 1.3                block quadtree/octree AMR, refinement ratio 2, Lohner-type
 *                           estimator, refine if one cell exceeds tol, coarsen if all
 *                           cells are below a fraction of tol
 *   Sec. 2.5.1, Eq. (diff-helmholtz), Sec. 1.4   Helmholtz problem, geometric multigrid
 *   Sec. 2.5.1, Eq. (imex)  second-order IMEX trapezoidal scheme
 *   Sec. 2.5, Eq. (gray-scott)  Gray-Scott reaction terms
 *
 * Where the paper is silent (limiter formulas, wave-speed estimates, ghost
 * filling between levels, refluxing, 2:1 balance, the smoother), the readings
 * implemented here are stated next to each function in the sources.
 */
#ifndef AMRVAC_ORACLE_H
#define AMRVAC_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FLUX_TVDLF = 0, ORC_FLUX_HLL = 1, ORC_FLUX_HLLC = 2 };
enum { ORC_LIM_MINMOD = 0, ORC_LIM_VANLEER = 1, ORC_LIM_KOREN = 2, ORC_LIM_NONE = 3, ORC_LIM_MC = 4, ORC_LIM_CADA = 5 };
enum { ORC_SSPRK2 = 2, ORC_SSPRK3 = 3 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_OUTFLOW = 1 };

typedef struct {
  int ndim;            /* 1..3 */
  int block_nx;        /* cells per block side */
  int base[3];         /* blocks per dimension on level 1 */
  int max_level;       /* 1 = uniform block grid */
  double xmin[3], xmax[3];
  double gamma, cfl;
  int flux, limiter, rk;
  int bc[3][2];        /* [dim][low/high] */
  double refine_tol, coarsen_frac, wavefilter;
  unsigned var_mask;   /* primitive variables used by the estimator: bit 0 rho .. bit ndim+1 p */
} orc_config;

typedef struct orc_grid orc_grid;

orc_grid* orc_create(const orc_config* cfg);          /* base level only, state zero */
void orc_destroy(orc_grid* g);
int orc_num_leaves(const orc_grid* g);
/* leaves in Morton order: level[n], coords[3n] (block index on its level) */
void orc_leaves(const orc_grid* g, int* level, int* coords);
/* replace the tree by the given leaves (any order; stored in Morton order); 0 on success */
int orc_set_leaves(orc_grid* g, int n, const int* level, const int* coords);
/* state layout: [leaf (Morton order)][var][cell], cell index i + nx*(j + nx*k) */
void orc_set_prim(orc_grid* g, const double* V);
void orc_set_cons(orc_grid* g, const double* U);
void orc_get_cons(const orc_grid* g, double* U);
void orc_set_time(orc_grid* g, double t);
double orc_time(const orc_grid* g);
double orc_dt(const orc_grid* g, double t_end);        /* CFL step clipped to t_end */
double orc_step(orc_grid* g, double t_end);            /* one SSPRK step; returns dt */
void orc_totals(const orc_grid* g, double* tot);       /* sum U dV per variable */
void orc_lohner(const orc_grid* g, double* err);       /* max estimator per leaf */
/* threads of the OpenMP loops over blocks and cells (the timed CPU baseline); n <= 0 keeps the
   current count; returns it (1 in a build without OpenMP).  Results do not depend on it. */
int orc_set_threads(int n);
int orc_regrid(orc_grid* g);                           /* returns new number of leaves */
/* face-ghost values of one leaf (for tests): [var][face 0..2*ndim-1][layer 0..1][tangential cells] */
void orc_face_ghosts(const orc_grid* g, int leaf, double* out);

/* single-face pieces, for pinning tests */
void orc_prim_to_cons(int ndim, double gamma, const double* V, double* U);
void orc_cons_to_prim(int ndim, double gamma, const double* U, double* V);
void orc_phys_flux(int ndim, int dir, double gamma, const double* V, double* F);
void orc_riemann_flux(int ndim, int dir, int flux, double gamma,
                      const double* VL, const double* VR, double* F);
/* limited slopes s- and s+ of cell i from its neighbours (a = q_i - q_{i-1}, b = q_{i+1} - q_i) */
void orc_limited_slopes(int limiter, double a, double b, double* sm, double* sp);

/* exact Riemann solution of the Euler equations (Toro ch. 4), sampled at xi = x/t */
int orc_exact_riemann(double gamma, const double* left, const double* right,
                      int n, const double* xi, double* out /* [n][3] rho,u,p */,
                      double* pstar, double* ustar);

/* ---- multigrid: (lambda - lap_h) x = b on an n^ndim grid of side L ----
 * Boundaries: periodic, or Neumann (zero flux: a face on the domain boundary carries no
 * diffusive flux, so a boundary cell's Laplacian has only its in-domain neighbours). */
enum { ORC_MG_PERIODIC = 0, ORC_MG_NEUMANN = 1 };
typedef struct {
  int ndim, n;      /* cells per side */
  double L, lambda;
  int nu1, nu2, max_cycles;
  double rtol;      /* stop when max|b - A x| <= rtol * max|b| */
  int coarse_max;   /* coarsen while n is even and n > coarse_max */
  int bc;           /* ORC_MG_PERIODIC or ORC_MG_NEUMANN */
} orc_mg_config;
/* x holds the initial guess on entry; returns V-cycles used (or -1 if not converged) */
int orc_mg_solve(const orc_mg_config* c, const double* b, double* x, double* relres);
void orc_mg_apply(int ndim, int n, double L, double lambda, int bc, const double* x, double* Ax);
/* one V-cycle on the correction equation A e = r, e zero on entry (test hook) */
void orc_mg_vcycle(const orc_mg_config* c, const double* r, double* e);
/* dense Gaussian elimination solve of the same system (tiny n only) */
int orc_dense_solve(int ndim, int n, double L, double lambda, int bc, const double* b, double* x);

/* ---- multigrid on a 2D block quadtree (Sec. 1.4, Sec. 2.5.2), periodic, square base of
 * nbx x nby blocks of B^2 cells, level-1 cell size L / (nbx B).  Leaves: level[k] >= 1 and
 * block coordinates coords[2k], coords[2k+1] at that level; the tree must tile the domain and
 * be 2:1 balanced across faces and corners.  Leaf data [leaf][B*B], x fastest. ---- */
typedef struct {
  int nbx, nby, B;
  double L, lambda;
  int nu1, nu2, max_cycles;
  double rtol;        /* max|b - A x| over leaf cells <= rtol max|b| */
  double base_rtol;   /* level-1 correction solve by the uniform multigrid: residual reduction */
  int coarse_max;
} orc_amg_config;
/* x: guess in, solution out.  fixed_cycles > 0 runs exactly that many V-cycles.  Returns
 * the V-cycles used, -1 if rtol was not reached, -2 for an invalid tree. */
int orc_amg_solve(const orc_amg_config* c, int nleaves, const int* level, const int* coords, const double* b,
                  double* x, int fixed_cycles, double* relres);
/* the composite operator on the leaves, and the face ghost values it uses ([leaf][4][B]:
 * faces x-, x+, y-, y+, along the face in increasing order) */
int orc_amg_apply(const orc_amg_config* c, int nleaves, const int* level, const int* coords, const double* x,
                  double* Ax);
int orc_amg_face_ghosts(const orc_amg_config* c, int nleaves, const int* level, const int* coords, const double* x,
                        double* ghosts);
/* Regrid of the reaction-diffusion quadtree: Lohner estimator of u (eps filter), refine
 * above refine_tol (up to max_level), coarsen sibling groups below coarsen_frac refine_tol, 2:1
 * balance; fields copied, prolonged (minmod slopes) or restricted.  Writes the new leaves (Morton
 * order of the lower corner at max_level), their u, v and the old leaves' estimator err[nleaves];
 * returns the new leaf count, -2 for an invalid tree, -3 if it exceeds cap. */
int orc_amg_regrid(const orc_amg_config* c, int nleaves, const int* level, const int* coords, const double* u,
                   const double* v, double refine_tol, double coarsen_frac, double eps, int max_level, int cap,
                   int* new_level, int* new_coords, double* new_u, double* new_v, double* err);
/* Gray-Scott IMEX step (Eq. (imex), Eq. (gray-scott)) on the leaves: composite Laplacian
 * for the explicit parts, the tree multigrid (lambda = 2/(dt D), guess w_n; c->lambda is
 * ignored) for the implicit stage.  cycles[2]: V-cycles per species.  0, -1 (a solve did
 * not reach rtol) or -2 (invalid tree). */
int orc_amg_rd_step(const orc_amg_config* c, int nleaves, const int* level, const int* coords, double Du, double Dv,
                    double F, double k, double dt, double* u, double* v, int* cycles);

/* ---- reaction-diffusion step (Sec. 2.5): w = (u, v), dw/dt = F0(w) + F1(w), F0 the
 * reaction terms of Eq. (gray-scott) or Eq. (schnakenberg), F1 = D lap_h w ---- */
enum { ORC_RD_GRAY_SCOTT = 0, ORC_RD_SCHNAKENBERG = 1 };
enum { ORC_RD_IMEX = 0, ORC_RD_SPLIT = 1, ORC_RD_EXPLICIT = 2 };
typedef struct {
  int ndim, n; double L;
  double Du, Dv, F, k, dt;
  int nu1, nu2, max_cycles; double rtol; int coarse_max;
  int model;              /* ORC_RD_GRAY_SCOTT (F, k) or ORC_RD_SCHNAKENBERG (kappa, a, b) */
  double kappa, a, b;
  int scheme;             /* ORC_RD_IMEX: Eq. (imex); ORC_RD_SPLIT: explicit reaction then
                             backward-Euler diffusion, Eqs. (splitting), (diff-helmholtz);
                             ORC_RD_EXPLICIT: three-stage SSP Runge-Kutta on F0 + F1 */
  int bc;                 /* ORC_MG_PERIODIC or ORC_MG_NEUMANN */
} orc_rd_config;
/* advances u, v (n^ndim each) by one step; cycles[2] receives V-cycles used per species
 * (0 for the explicit scheme) */
int orc_rd_step(const orc_rd_config* c, double* u, double* v, int* cycles);
/* reaction terms F0 and the discrete Laplacian, for pins */
void orc_rd_reaction(double F, double k, int n, const double* u, const double* v,
                     double* fu, double* fv);
void orc_rd_reaction_schnakenberg(double kappa, double a, double b, int n, const double* u, const double* v,
                                  double* fu, double* fv);
void orc_laplacian(int ndim, int n, double L, int bc, const double* x, double* out);

/* ---- learned multigrid guess: CNN 5->16->16->16->2, 3^ndim periodic convolutions ----
 * params flat: per layer W[cout][cin][tap] then b[cout]; images [N][C][D][H][W] (D = 1 in 2D) */
long long orc_cnn_num_params(int ndim);
void orc_cnn_forward(int ndim, const double* params, int N, int D, int H, int W, const double* in, double* out);
/* masked MSE (pixels at least `margin` from every edge) and its gradient; returns the loss */
double orc_cnn_loss_grad(int ndim, const double* params, int N, int D, int H, int W, int margin, const double* in,
                         const double* target, double* grad);
// kind 0 = the masked MSE above; kind 1 = operator-weighted (kappa[2] per output channel,
// margin >= 1, else -1 is returned)
double orc_cnn_loss_grad_kind(int ndim, const double* params, int N, int D, int H, int W, int margin, int kind,
                              const double* kappa, const double* in, const double* target, double* grad);
double orc_cnn_output_loss(int ndim, int N, int D, int H, int W, int margin, int kind, const double* kappa,
                           const double* out, const double* target, double* dout);
void orc_cnn_adam(long long n, double* params, const double* grad, double* m, double* v, int t, double lr,
                  double b1, double b2, double eps);
double orc_gelu(double z);
double orc_gelu_d(double z);

#ifdef __cplusplus
}
#endif
#endif
