// Exact solution of the 1D Euler Riemann problem (Toro, "Riemann Solvers and
// Numerical Methods for Fluid Dynamics", ch. 4): Newton iteration for the star
// pressure on f_L(p) + f_R(p) + (u_R - u_L) = 0, then sampling of the
// self-similar solution at xi = x/t.  TEST INFRASTRUCTURE ONLY (see oracle.h):
// it pins the finite-volume oracle on the Sod problem.
#include <cmath>

#include "oracle.h"

namespace {

struct State {
  double r, u, p, c;
};

// pressure function of one side and its derivative
void fK(double p, const State& K, double g, double* f, double* df) {
  if (p > K.p) {  // shock
    double A = 2.0 / ((g + 1.0) * K.r);
    double B = (g - 1.0) / (g + 1.0) * K.p;
    double q = std::sqrt(A / (p + B));
    *f = (p - K.p) * q;
    *df = q * (1.0 - 0.5 * (p - K.p) / (B + p));
  } else {  // rarefaction
    double pr = p / K.p;
    *f = 2.0 * K.c / (g - 1.0) * (std::pow(pr, (g - 1.0) / (2.0 * g)) - 1.0);
    *df = 1.0 / (K.r * K.c) * std::pow(pr, -(g + 1.0) / (2.0 * g));
  }
}

}  // namespace

extern "C" int orc_exact_riemann(double g, const double* left, const double* right, int n,
                                 const double* xi, double* out, double* pstar_out,
                                 double* ustar_out) {
  State L{left[0], left[1], left[2], std::sqrt(g * left[2] / left[0])};
  State R{right[0], right[1], right[2], std::sqrt(g * right[2] / right[0])};
  double du = R.u - L.u;
  if (2.0 * (L.c + R.c) / (g - 1.0) <= du) return -1;  // vacuum generated
  // primitive-variable guess, then Newton
  double p = 0.5 * (L.p + R.p) - 0.125 * du * (L.r + R.r) * (L.c + R.c);
  if (p < 1e-8) p = 1e-8;
  for (int it = 0; it < 100; ++it) {
    double fl, dfl, fr, dfr;
    fK(p, L, g, &fl, &dfl);
    fK(p, R, g, &fr, &dfr);
    double pn = p - (fl + fr + du) / (dfl + dfr);
    if (pn < 1e-12) pn = 1e-12;
    double ch = 2.0 * std::fabs(pn - p) / (pn + p);
    p = pn;
    if (ch < 1e-15) break;
  }
  double fl, dfl, fr, dfr;
  fK(p, L, g, &fl, &dfl);
  fK(p, R, g, &fr, &dfr);
  double us = 0.5 * (L.u + R.u) + 0.5 * (fr - fl);
  if (pstar_out) *pstar_out = p;
  if (ustar_out) *ustar_out = us;
  double gm = (g - 1.0) / (g + 1.0);
  for (int i = 0; i < n; ++i) {
    double S = xi[i];
    double r, u, pp;
    if (S <= us) {  // left of contact
      if (p > L.p) {
        double SL = L.u - L.c * std::sqrt((g + 1.0) / (2.0 * g) * p / L.p + (g - 1.0) / (2.0 * g));
        if (S <= SL) {
          r = L.r; u = L.u; pp = L.p;
        } else {
          r = L.r * (p / L.p + gm) / (gm * p / L.p + 1.0); u = us; pp = p;
        }
      } else {
        double SH = L.u - L.c;
        double cs = L.c * std::pow(p / L.p, (g - 1.0) / (2.0 * g));
        double ST = us - cs;
        if (S <= SH) {
          r = L.r; u = L.u; pp = L.p;
        } else if (S >= ST) {
          r = L.r * std::pow(p / L.p, 1.0 / g); u = us; pp = p;
        } else {
          double fac = 2.0 / (g + 1.0) + gm / L.c * (L.u - S);
          r = L.r * std::pow(fac, 2.0 / (g - 1.0));
          u = 2.0 / (g + 1.0) * (L.c + (g - 1.0) / 2.0 * L.u + S);
          pp = L.p * std::pow(fac, 2.0 * g / (g - 1.0));
        }
      }
    } else {  // right of contact
      if (p > R.p) {
        double SR = R.u + R.c * std::sqrt((g + 1.0) / (2.0 * g) * p / R.p + (g - 1.0) / (2.0 * g));
        if (S >= SR) {
          r = R.r; u = R.u; pp = R.p;
        } else {
          r = R.r * (p / R.p + gm) / (gm * p / R.p + 1.0); u = us; pp = p;
        }
      } else {
        double SH = R.u + R.c;
        double cs = R.c * std::pow(p / R.p, (g - 1.0) / (2.0 * g));
        double ST = us + cs;
        if (S >= SH) {
          r = R.r; u = R.u; pp = R.p;
        } else if (S <= ST) {
          r = R.r * std::pow(p / R.p, 1.0 / g); u = us; pp = p;
        } else {
          double fac = 2.0 / (g + 1.0) - gm / R.c * (R.u - S);
          r = R.r * std::pow(fac, 2.0 / (g - 1.0));
          u = 2.0 / (g + 1.0) * (-R.c + (g - 1.0) / 2.0 * R.u + S);
          pp = R.p * std::pow(fac, 2.0 * g / (g - 1.0));
        }
      }
    }
    out[3 * i] = r;
    out[3 * i + 1] = u;
    out[3 * i + 2] = pp;
  }
  return 0;
}
