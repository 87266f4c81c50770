// FP64 oracle of the learned multigrid initial guess: a small convolutional
// network, its backward pass, a masked mean-squared-error loss and Adam.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// The paper has no learned component; this network is the project's addition
// for the multigrid initial guess.  READINGS (all architectural details):
//  * 4 layers of 3^ndim periodic cross-correlations with bias, channels
//    5 -> 16 -> 16 -> 16 -> 2, GELU (erf form) after layers 1..3;
//  * parameters flat, per layer W[cout][cin][tap] (tap = x fastest over
//    offsets -1, 0, 1 per dimension) followed by b[cout];
//  * loss = mean over channels and over pixels at least `margin` cells away
//    from every image edge of (out - target)^2;
//  * or, the operator-weighted loss: the same mean of q^2 with
//    q = (1 + kappa_c) e - (1/(2 ndim)) * (sum of e over the 2 ndim face
//    neighbours), e = out - target, kappa_c per output channel.  This is the
//    residual of the guess under the diagonal-normalised Helmholtz operator
//    (lambda - lap_h) * h^2 / (2 ndim) of Eq. (diff-helmholtz) with kappa =
//    lambda h^2 / (2 ndim): for a guess X = w_n + s * out and the converged
//    solution w* = w_n + s * target, lambda g - A X = s (2 ndim / h^2) q.
//    It needs margin >= 1 (the neighbours of counted pixels lie in the image);
//  * Adam with bias correction.
#include <cmath>
#include <cstring>
#include <vector>

#include "oracle.h"

namespace {

const int kCh[5] = {5, 16, 16, 16, 2};

int ntaps(int nd) { return nd == 3 ? 27 : 9; }

long long layer_offset(int nd, int l) {
  long long o = 0;
  for (int i = 0; i < l; ++i) o += (long long)kCh[i + 1] * kCh[i] * ntaps(nd) + kCh[i + 1];
  return o;
}

struct Shape {
  int nd, N, D, H, W;  // D = 1 in 2D
  long long npix() const { return (long long)D * H * W; }
};

inline int wrap(int i, int n) { return ((i % n) + n) % n; }

// z[n][co][p] = b[co] + sum_ci sum_tap W[co][ci][tap] x[n][ci][p + off(tap)]
void conv(const Shape& s, int cin, int cout, const double* Wt, const double* b, const std::vector<double>& x,
          std::vector<double>& z) {
  int T = ntaps(s.nd);
  long long P = s.npix();
  z.assign((size_t)s.N * cout * P, 0.0);
  for (int n = 0; n < s.N; ++n)
    for (int co = 0; co < cout; ++co)
      for (int k = 0; k < s.D; ++k)
        for (int j = 0; j < s.H; ++j)
          for (int i = 0; i < s.W; ++i) {
            double acc = b[co];
            for (int ci = 0; ci < cin; ++ci)
              for (int t = 0; t < T; ++t) {
                int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = s.nd == 3 ? t / 9 - 1 : 0;
                long long q = ((long long)wrap(k + dz, s.D) * s.H + wrap(j + dy, s.H)) * s.W + wrap(i + dx, s.W);
                acc += Wt[((long long)co * cin + ci) * T + t] * x[((size_t)n * cin + ci) * P + q];
              }
            z[((size_t)n * cout + co) * P + ((long long)k * s.H + j) * s.W + i] = acc;
          }
}

double gelu(double z) { return 0.5 * z * (1.0 + std::erf(z / std::sqrt(2.0))); }
double gelu_d(double z) {
  const double inv_sqrt_2pi = 0.3989422804014327;
  return 0.5 * (1.0 + std::erf(z / std::sqrt(2.0))) + z * inv_sqrt_2pi * std::exp(-0.5 * z * z);
}

struct Acts {
  std::vector<double> x[5];  // x[0] = input, x[l] = activation after layer l (x[4] = output)
  std::vector<double> z[5];  // pre-activations z[1..4]
};

void forward(const Shape& s, const double* params, const double* in, Acts& A) {
  long long P = s.npix();
  A.x[0].assign(in, in + (size_t)s.N * kCh[0] * P);
  for (int l = 0; l < 4; ++l) {
    const double* Wt = params + layer_offset(s.nd, l);
    const double* b = Wt + (long long)kCh[l + 1] * kCh[l] * ntaps(s.nd);
    conv(s, kCh[l], kCh[l + 1], Wt, b, A.x[l], A.z[l + 1]);
    A.x[l + 1] = A.z[l + 1];
    if (l < 3)
      for (double& v : A.x[l + 1]) v = gelu(v);
  }
}

bool in_mask(const Shape& s, int k, int j, int i, int margin) {
  if (j < margin || j >= s.H - margin || i < margin || i >= s.W - margin) return false;
  if (s.nd == 3 && (k < margin || k >= s.D - margin)) return false;
  return true;
}

}  // namespace

extern "C" {

long long orc_cnn_num_params(int ndim) { return layer_offset(ndim, 4); }

void orc_cnn_forward(int ndim, const double* params, int N, int D, int H, int W, const double* in, double* out) {
  Shape s{ndim, N, ndim == 3 ? D : 1, H, W};
  Acts A;
  forward(s, params, in, A);
  std::memcpy(out, A.x[4].data(), A.x[4].size() * sizeof(double));
}

}  // extern "C"

namespace {

// masked loss of the network output and its derivative dL/d(out); kind 0 = MSE,
// kind 1 = operator-weighted (kappa[2] per output channel); margin >= 1 for kind 1
double output_loss(const Shape& s, int margin, int kind, const double* kappa, const double* out,
                   const double* target, double* dout) {
  long long P = s.npix();
  const int C = kCh[4];
  long long count = 0;
  for (int k = 0; k < s.D; ++k)
    for (int j = 0; j < s.H; ++j)
      for (int i = 0; i < s.W; ++i)
        if (in_mask(s, k, j, i, margin)) ++count;
  count *= (long long)s.N * C;
  size_t n_all = (size_t)s.N * C * P;
  for (size_t o = 0; o < n_all; ++o) dout[o] = 0.0;
  double loss = 0.0;
  if (kind == 0) {
    for (int n = 0; n < s.N; ++n)
      for (int c = 0; c < C; ++c)
        for (int k = 0; k < s.D; ++k)
          for (int j = 0; j < s.H; ++j)
            for (int i = 0; i < s.W; ++i) {
              if (!in_mask(s, k, j, i, margin)) continue;
              size_t o = ((size_t)n * C + c) * P + ((long long)k * s.H + j) * s.W + i;
              double d = out[o] - target[o];
              loss += d * d;
              dout[o] = 2.0 * d / (double)count;
            }
    return loss / (double)count;
  }
  // operator-weighted: q on the counted pixels, then dL/d(out) = (2/count) A^T q
  // (the normalised operator is symmetric), neighbours by plain index offsets
  const double nb_w = 1.0 / (2.0 * s.nd);
  auto e_at = [&](size_t base, int k, int j, int i) {
    size_t o = base + ((long long)k * s.H + j) * s.W + i;
    return out[o] - target[o];
  };
  std::vector<double> q(n_all, 0.0);
  for (int n = 0; n < s.N; ++n)
    for (int c = 0; c < C; ++c) {
      size_t base = ((size_t)n * C + c) * P;
      for (int k = 0; k < s.D; ++k)
        for (int j = 0; j < s.H; ++j)
          for (int i = 0; i < s.W; ++i) {
            if (!in_mask(s, k, j, i, margin)) continue;
            double nb = e_at(base, k, j, i - 1) + e_at(base, k, j, i + 1) + e_at(base, k, j - 1, i) +
                        e_at(base, k, j + 1, i);
            if (s.nd == 3) nb += e_at(base, k - 1, j, i) + e_at(base, k + 1, j, i);
            double qv = (1.0 + kappa[c]) * e_at(base, k, j, i) - nb_w * nb;
            q[base + ((long long)k * s.H + j) * s.W + i] = qv;
            loss += qv * qv;
          }
    }
  for (int n = 0; n < s.N; ++n)
    for (int c = 0; c < C; ++c) {
      size_t base = ((size_t)n * C + c) * P;
      for (int k = 0; k < s.D; ++k)
        for (int j = 0; j < s.H; ++j)
          for (int i = 0; i < s.W; ++i) {
            size_t o = base + ((long long)k * s.H + j) * s.W + i;
            // q is zero off the mask, and every pixel next to the mask lies in the image
            double g = (1.0 + kappa[c]) * q[o];
            if (i > 0) g -= nb_w * q[o - 1];
            if (i < s.W - 1) g -= nb_w * q[o + 1];
            if (j > 0) g -= nb_w * q[o - s.W];
            if (j < s.H - 1) g -= nb_w * q[o + s.W];
            if (s.nd == 3 && k > 0) g -= nb_w * q[o - (size_t)s.H * s.W];
            if (s.nd == 3 && k < s.D - 1) g -= nb_w * q[o + (size_t)s.H * s.W];
            dout[o] = 2.0 * g / (double)count;
          }
    }
  return loss / (double)count;
}

// loss and gradient of the masked loss with respect to every parameter
double loss_grad(int ndim, const double* params, int N, int D, int H, int W, int margin, int kind,
                 const double* kappa, const double* in, const double* target, double* grad) {
  Shape s{ndim, N, ndim == 3 ? D : 1, H, W};
  long long P = s.npix();
  int T = ntaps(ndim);
  Acts A;
  forward(s, params, in, A);
  std::vector<double> dz((size_t)s.N * kCh[4] * P, 0.0);  // dL/dz of the current layer
  double loss = output_loss(s, margin, kind, kappa, A.x[4].data(), target, dz.data());
  std::memset(grad, 0, sizeof(double) * layer_offset(ndim, 4));
  for (int l = 3; l >= 0; --l) {
    int cin = kCh[l], cout = kCh[l + 1];
    const double* Wt = params + layer_offset(ndim, l);
    double* gW = grad + layer_offset(ndim, l);
    double* gb = gW + (long long)cout * cin * T;
    std::vector<double> dx((size_t)s.N * cin * P, 0.0);
    for (int n = 0; n < s.N; ++n)
      for (int co = 0; co < cout; ++co)
        for (int k = 0; k < s.D; ++k)
          for (int j = 0; j < s.H; ++j)
            for (int i = 0; i < s.W; ++i) {
              double g = dz[((size_t)n * cout + co) * P + ((long long)k * s.H + j) * s.W + i];
              if (g == 0.0) continue;
              gb[co] += g;
              for (int ci = 0; ci < cin; ++ci)
                for (int t = 0; t < T; ++t) {
                  int ddx = t % 3 - 1, ddy = (t / 3) % 3 - 1, ddz = ndim == 3 ? t / 9 - 1 : 0;
                  long long q = ((long long)wrap(k + ddz, s.D) * s.H + wrap(j + ddy, s.H)) * s.W + wrap(i + ddx, s.W);
                  size_t xi = ((size_t)n * cin + ci) * P + q;
                  gW[((long long)co * cin + ci) * T + t] += g * A.x[l][xi];
                  dx[xi] += g * Wt[((long long)co * cin + ci) * T + t];
                }
            }
    if (l > 0) {
      // through the GELU of layer l
      for (size_t o = 0; o < dx.size(); ++o) dx[o] *= gelu_d(A.z[l][o]);
    }
    dz.swap(dx);
  }
  return loss;
}

}  // namespace

extern "C" {

// loss and gradient of the masked MSE with respect to every parameter
double orc_cnn_loss_grad(int ndim, const double* params, int N, int D, int H, int W, int margin, const double* in,
                         const double* target, double* grad) {
  return loss_grad(ndim, params, N, D, H, W, margin, 0, nullptr, in, target, grad);
}

// the same for a loss kind (0 = MSE, 1 = operator-weighted with kappa[2]); negative = invalid
double orc_cnn_loss_grad_kind(int ndim, const double* params, int N, int D, int H, int W, int margin, int kind,
                              const double* kappa, const double* in, const double* target, double* grad) {
  if (kind == 1 && margin < 1) return -1.0;
  return loss_grad(ndim, params, N, D, H, W, margin, kind, kappa, in, target, grad);
}

// the loss alone, on given network outputs: returns it and writes dL/d(out)
double orc_cnn_output_loss(int ndim, int N, int D, int H, int W, int margin, int kind, const double* kappa,
                           const double* out, const double* target, double* dout) {
  if (kind == 1 && margin < 1) return -1.0;
  Shape s{ndim, N, ndim == 3 ? D : 1, H, W};
  return output_loss(s, margin, kind, kappa, out, target, dout);
}

// one Adam step (bias-corrected), t = step number starting at 1
void orc_cnn_adam(long long n, double* params, const double* grad, double* m, double* v, int t, double lr,
                  double b1, double b2, double eps) {
  double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
  for (long long i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
    v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    params[i] -= lr * mh / (std::sqrt(vh) + eps);
  }
}

double orc_gelu(double z) { return gelu(z); }
double orc_gelu_d(double z) { return gelu_d(z); }

}  // extern "C"
