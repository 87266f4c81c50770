// Learned multigrid initial guess: a 4-layer periodic CNN (5 -> 16 -> 16 -> 16
// -> 2 channels, 3x3 or 3x3x3 taps, GELU after layers 1..3) with hand-written
// forward, backward and Adam kernels.  The paper has no learned component; the
// network predicts the implicit-diffusion solution (as a correction to the
// right-hand side g of the Helmholtz problem) that the multigrid then iterates
// to the same tolerance.
//
// Convolutions are implicit GEMMs on the tensor cores (mma m16n8k16, bf16
// operands, fp32 accumulation): M = 16 output pixels, N = 8 output channels,
// K = 16 input channels of one tap; the tile's input pixels (with a one-cell
// periodic halo) and the packed weights are staged in shared memory with a 48-byte
// stride per pixel / weight row so every fragment load of a warp hits distinct
// banks.  The same kernel computes the data gradient of a layer with the taps
// mirrored and the weight matrix transposed.  Weight gradients are accumulated
// on the fp32 cores per persistent CTA and reduced in a fixed order.
//
// Layouts: activations NHWC with 16 bf16 channels per pixel (32 bytes); the
// caller's images are [N][C][D][H][W] float32; parameters are flat float32, per
// layer W[cout][cin][tap] (tap x fastest over offsets -1, 0, 1) then b[cout].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <memory>
#include <random>
#include <string>
#include <vector>

#include "../../include/amrvac_gb300.h"
#include "mg_internal.h"

namespace cnngpu {

constexpr int kCh[5] = {5, 16, 16, 16, 2};
constexpr int CS = 24;  // bf16 stride of one pixel / weight row in shared memory

using bf16 = __nv_bfloat16;

template <int ND>
struct TD;
template <>
struct TD<2> {
  static constexpr int TZ = 1, TY = 16, TX = 16, HZ = 0, T = 9;
};
template <>
struct TD<3> {
  static constexpr int TZ = 4, TY = 8, TX = 8, HZ = 1, T = 27;
};

__host__ __device__ constexpr int ntaps(int nd) { return nd == 3 ? 27 : 9; }

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

// FWD_INFER: FWD_GELU without the pre-activation store (inference has no backward pass)
enum { FWD_GELU = 0, FWD_OUT = 1, BWD_GELU = 2, FWD_INFER = 3 };

struct ConvArgs {
  const bf16* in;     // NHWC16
  const bf16* w;      // packed [tap][npad][CS]
  const float* bias;  // forward modes
  const bf16* zprev;  // BWD_GELU: pre-activations of the layer input
  bf16* z_out;
  bf16* a_out;
  float* out;         // FWD_OUT: [N][P][2]
  bf16* dz_out;
  int N, D, H, W;
};

template <int ND>
__device__ __forceinline__ void tile_origin(int tile, int D, int H, int W, int& n, int& z0, int& y0, int& x0) {
  using T = TD<ND>;
  int tx = W / T::TX, ty = H / T::TY, tz = D / T::TZ;
  x0 = (tile % tx) * T::TX;
  tile /= tx;
  y0 = (tile % ty) * T::TY;
  tile /= ty;
  z0 = (tile % tz) * T::TZ;
  n = tile / tz;
}

// stage the tile's input pixels with a one-cell periodic halo: [SZ][SY][SX][CS]
template <int ND>
__device__ __forceinline__ void load_tile(bf16* s_in, const bf16* in, int n, int z0, int y0, int x0, int D, int H,
                                          int W) {
  using T = TD<ND>;
  constexpr int SZ = T::TZ + 2 * T::HZ, SY = T::TY + 2, SX = T::TX + 2;
  for (int r = threadIdx.x; r < SZ * SY * SX * 2; r += blockDim.x) {
    int pix = r >> 1, half = r & 1;
    int sx = pix % SX, sy = (pix / SX) % SY, sz = pix / (SX * SY);
    int gz = wrapi(z0 + sz - T::HZ, D), gy = wrapi(y0 + sy - 1, H), gx = wrapi(x0 + sx - 1, W);
    const uint4* src = reinterpret_cast<const uint4*>(in + ((((size_t)n * D + gz) * H + gy) * W + gx) * 16) + half;
    *reinterpret_cast<uint4*>(s_in + pix * CS + half * 8) = __ldg(src);
  }
}

template <int ND, int MODE>
constexpr size_t conv_smem_bytes() {
  using T = TD<ND>;
  return (size_t)((T::TZ + 2 * T::HZ) * (T::TY + 2) * (T::TX + 2) + T::T * (MODE == FWD_OUT ? 8 : 16)) * CS *
         sizeof(bf16);
}

template <int ND, int MODE>
__global__ void __launch_bounds__(256) conv_kernel(ConvArgs a) {
  using T = TD<ND>;
  constexpr int TAPS = T::T, NT = MODE == FWD_OUT ? 1 : 2, NPAD = NT * 8;
  constexpr int SY = T::TY + 2, SX = T::TX + 2, SZ = T::TZ + 2 * T::HZ;
  extern __shared__ __align__(16) unsigned char conv_smem[];
  bf16* s_in = reinterpret_cast<bf16*>(conv_smem);
  bf16* s_w = s_in + SZ * SY * SX * CS;
  int n, z0, y0, x0;
  tile_origin<ND>(blockIdx.x, a.D, a.H, a.W, n, z0, y0, x0);
  for (int r = threadIdx.x; r < TAPS * NPAD * CS / 8; r += blockDim.x)
    reinterpret_cast<uint4*>(s_w)[r] = __ldg(reinterpret_cast<const uint4*>(a.w) + r);
  load_tile<ND>(s_in, a.in, n, z0, y0, x0, a.D, a.H, a.W);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // the warp's two m-tiles: tile pixels v = 16*(2w+mt) + g (+8)
  int sp0[2], sp1[2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    int v0 = 16 * (2 * warp + mt) + g, v1 = v0 + 8;
    int x = v0 % T::TX, y = (v0 / T::TX) % T::TY, z = v0 / (T::TX * T::TY);
    sp0[mt] = ((z + T::HZ) * SY + (y + 1)) * SX + (x + 1);
    x = v1 % T::TX, y = (v1 / T::TX) % T::TY, z = v1 / (T::TX * T::TY);
    sp1[mt] = ((z + T::HZ) * SY + (y + 1)) * SX + (x + 1);
  }
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
  const uint32_t* sw32 = reinterpret_cast<const uint32_t*>(s_w);
  const uint32_t* si32 = reinterpret_cast<const uint32_t*>(s_in);
#pragma unroll 3
  for (int tap = 0; tap < TAPS; ++tap) {
    int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = ND == 3 ? tap / 9 - 1 : 0;
    int doff = (dz * SY + dy) * SX + dx;
    uint32_t b[NT][2];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      int row = tap * NPAD + nt * 8 + g;
      b[nt][0] = sw32[row * (CS / 2) + t];
      b[nt][1] = sw32[row * (CS / 2) + 4 + t];
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      uint32_t av[4];
      int p0 = sp0[mt] + doff, p1 = sp1[mt] + doff;
      av[0] = si32[p0 * (CS / 2) + t];
      av[1] = si32[p1 * (CS / 2) + t];
      av[2] = si32[p0 * (CS / 2) + 4 + t];
      av[3] = si32[p1 * (CS / 2) + 4 + t];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) mma16816(acc[mt][nt], av, b[nt]);
    }
  }
  // epilogue
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      int v = 16 * (2 * warp + mt) + g + 8 * half;
      int x = v % T::TX, y = (v / T::TX) % T::TY, z = v / (T::TX * T::TY);
      size_t gp = (((size_t)n * a.D + z0 + z) * a.H + y0 + y) * a.W + x0 + x;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        int c = nt * 8 + 2 * t;
        float v0 = acc[mt][nt][2 * half], v1 = acc[mt][nt][2 * half + 1];
        if (MODE == FWD_GELU || MODE == FWD_INFER) {
          v0 += a.bias[c];
          v1 += a.bias[c + 1];
          if (MODE == FWD_GELU)
            *reinterpret_cast<__nv_bfloat162*>(a.z_out + gp * 16 + c) = __floats2bfloat162_rn(v0, v1);
          *reinterpret_cast<__nv_bfloat162*>(a.a_out + gp * 16 + c) = __floats2bfloat162_rn(gelu(v0), gelu(v1));
        } else if (MODE == FWD_OUT) {
          if (c < 2) {
            a.out[gp * 2 + 0] = v0 + a.bias[0];
            a.out[gp * 2 + 1] = v1 + a.bias[1];
          }
        } else {
          __nv_bfloat162 zp = *reinterpret_cast<const __nv_bfloat162*>(a.zprev + gp * 16 + c);
          float2 zf = __bfloat1622float2(zp);
          *reinterpret_cast<__nv_bfloat162*>(a.dz_out + gp * 16 + c) =
              __floats2bfloat162_rn(v0 * gelu_d(zf.x), v1 * gelu_d(zf.y));
        }
      }
    }
}

// caller's [N][5][P] float32 -> NHWC16 bf16 (channels 5..15 zero)
__global__ void pack_input_kernel(const float* __restrict__ in, bf16* __restrict__ x, long long npix, long long P) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  long long n = i / P, p = i % P;
  __align__(16) bf16 v[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(c < 5 ? in[(n * 5 + c) * P + p] : 0.f);
  reinterpret_cast<uint4*>(x + i * 16)[0] = reinterpret_cast<uint4*>(v)[0];
  reinterpret_cast<uint4*>(x + i * 16)[1] = reinterpret_cast<uint4*>(v)[1];
}

// forward packing: w[tap][n = co][k = ci]; transposed packing for the data gradient:
// w[tap'][n = ci][k = co] = W[co][ci][T-1-tap'] (mirrored taps)
__global__ void pack_weights_kernel(const float* __restrict__ W, bf16* __restrict__ out, int cin, int cout, int taps,
                                    int npad, int transposed) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int total = taps * npad * CS;
  if (i >= total) return;
  int k = i % CS, row = i / CS, nn = row % npad, tap = row / npad;
  float v = 0.f;
  if (k < 16) {
    if (!transposed) {
      if (nn < cout && k < cin) v = W[((long long)nn * cin + k) * taps + tap];
    } else {
      if (k < cout && nn < cin) v = W[((long long)k * cin + nn) * taps + (taps - 1 - tap)];
    }
  }
  out[i] = __float2bfloat16_rn(v);
}

// masked MSE: loss accumulation and dL/dz of the output layer (NHWC16, channels 2.. zero)
__global__ void loss_grad_kernel(const float* __restrict__ out, const float* __restrict__ target, bf16* __restrict__ dz,
                                 float* loss, long long npix, int D, int H, int W, int margin, int ndim, float inv_count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < npix) {
    long long P = (long long)D * H * W;
    long long n = i / P, p = i % P;
    int x = (int)(p % W), y = (int)((p / W) % H), z = (int)(p / ((long long)W * H));
    bool in = x >= margin && x < W - margin && y >= margin && y < H - margin &&
              (ndim < 3 || (z >= margin && z < D - margin));
    __align__(16) bf16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
    if (in) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float d = out[i * 2 + c] - target[(n * 2 + c) * P + p];
        l += d * d;
        v[c] = __float2bfloat16_rn(2.f * d * inv_count);
      }
    }
    reinterpret_cast<uint4*>(dz + i * 16)[0] = reinterpret_cast<uint4*>(v)[0];
    reinterpret_cast<uint4*>(dz + i * 16)[1] = reinterpret_cast<uint4*>(v)[1];
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l * inv_count);
}

// operator-weighted loss, pass 1: q = (1 + kappa_c) e - (1/(2 ndim)) sum_faces e with
// e = out - target on the counted pixels (zero elsewhere), and the loss sum of q^2.
// The counted pixels lie at least one cell inside the image, so every neighbour exists.
__global__ void op_q_kernel(const float* __restrict__ out, const float* __restrict__ target, float* __restrict__ q,
                            float* loss, long long npix, int D, int H, int W, int margin, int ndim, float k0, float k1,
                            float inv_count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < npix) {
    long long P = (long long)D * H * W;
    long long n = i / P, p = i % P;
    int x = (int)(p % W), y = (int)((p / W) % H), z = (int)(p / ((long long)W * H));
    bool in = x >= margin && x < W - margin && y >= margin && y < H - margin &&
              (ndim < 3 || (z >= margin && z < D - margin));
    float qv[2] = {0.f, 0.f};
    if (in) {
      const long long HW = (long long)H * W;
      const float nbw = ndim == 3 ? 1.f / 6.f : 0.25f;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float* t = target + (n * 2 + c) * P;
        auto e = [&](long long pp, long long ii) { return out[ii * 2 + c] - t[pp]; };
        float nb = e(p - 1, i - 1) + e(p + 1, i + 1) + e(p - W, i - W) + e(p + W, i + W);
        if (ndim == 3) nb += e(p - HW, i - HW) + e(p + HW, i + HW);
        qv[c] = (1.f + (c ? k1 : k0)) * e(p, i) - nbw * nb;
        l += qv[c] * qv[c];
      }
    }
    reinterpret_cast<float2*>(q)[i] = make_float2(qv[0], qv[1]);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l * inv_count);
}

// operator-weighted loss, pass 2: dL/dz of the output layer = (2 / count) A^T q, A the
// normalised operator (symmetric); neighbours outside the image hold no q.
__global__ void op_grad_kernel(const float* __restrict__ q, bf16* __restrict__ dz, long long npix, int D, int H, int W,
                               int ndim, float k0, float k1, float inv_count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  long long P = (long long)D * H * W;
  long long p = i % P;
  int x = (int)(p % W), y = (int)((p / W) % H), z = (int)(p / ((long long)W * H));
  const long long HW = (long long)H * W;
  const float nbw = ndim == 3 ? 1.f / 6.f : 0.25f;
  const float2* q2 = reinterpret_cast<const float2*>(q);
  float2 c = q2[i];
  float2 s = make_float2(0.f, 0.f);
  auto add = [&](long long j) {
    float2 v = q2[j];
    s.x += v.x;
    s.y += v.y;
  };
  if (x > 0) add(i - 1);
  if (x < W - 1) add(i + 1);
  if (y > 0) add(i - W);
  if (y < H - 1) add(i + W);
  if (ndim == 3 && z > 0) add(i - HW);
  if (ndim == 3 && z < D - 1) add(i + HW);
  __align__(16) bf16 v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __float2bfloat16_rn(0.f);
  v[0] = __float2bfloat16_rn(2.f * inv_count * ((1.f + k0) * c.x - nbw * s.x));
  v[1] = __float2bfloat16_rn(2.f * inv_count * ((1.f + k1) * c.y - nbw * s.y));
  reinterpret_cast<uint4*>(dz + i * 16)[0] = reinterpret_cast<uint4*>(v)[0];
  reinterpret_cast<uint4*>(dz + i * 16)[1] = reinterpret_cast<uint4*>(v)[1];
}

// weight and bias gradient partials of one layer, one set per CTA (persistent over tiles):
// dW[co][ci][tap] = sum_p dz[p][co] a[p + off(tap)][ci]; db[co] = sum_p dz[p][co]
template <int ND>
__global__ void __launch_bounds__(256) dw_kernel(const bf16* __restrict__ aprev, const bf16* __restrict__ dz,
                                                 float* __restrict__ part, int cin, int cout, int N, int D, int H,
                                                 int W) {
  using T = TD<ND>;
  constexpr int TAPS = T::T, SY = T::TY + 2, SX = T::TX + 2, SZ = T::TZ + 2 * T::HZ, NP = T::TZ * T::TY * T::TX;
  __shared__ __align__(16) bf16 s_in[SZ * SY * SX * CS];
  __shared__ __align__(16) bf16 s_dz[NP * 16];
  const int co = threadIdx.x >> 4, ci = threadIdx.x & 15;
  float acc[TAPS];
#pragma unroll
  for (int k = 0; k < TAPS; ++k) acc[k] = 0.f;
  float accb = 0.f;
  int ntiles = N * (D / T::TZ) * (H / T::TY) * (W / T::TX);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int n, z0, y0, x0;
    tile_origin<ND>(tile, D, H, W, n, z0, y0, x0);
    __syncthreads();
    load_tile<ND>(s_in, aprev, n, z0, y0, x0, D, H, W);
    for (int r = threadIdx.x; r < NP * 2; r += blockDim.x) {
      int v = r >> 1, half = r & 1;
      int x = v % T::TX, y = (v / T::TX) % T::TY, z = v / (T::TX * T::TY);
      size_t gp = (((size_t)n * D + z0 + z) * H + y0 + y) * W + x0 + x;
      reinterpret_cast<uint4*>(s_dz + v * 16)[half] = __ldg(reinterpret_cast<const uint4*>(dz + gp * 16) + half);
    }
    __syncthreads();
    if (co < cout && ci < cin) {
      for (int v = 0; v < NP; ++v) {
        float d = __bfloat162float(s_dz[v * 16 + co]);
        if (ci == 0) accb += d;
        int x = v % T::TX, y = (v / T::TX) % T::TY, z = v / (T::TX * T::TY);
        int base = ((z + T::HZ) * SY + (y + 1)) * SX + (x + 1);
#pragma unroll
        for (int tap = 0; tap < TAPS; ++tap) {
          int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dzz = ND == 3 ? tap / 9 - 1 : 0;
          acc[tap] += d * __bfloat162float(s_in[(base + (dzz * SY + dy) * SX + dx) * CS + ci]);
        }
      }
    }
  }
  float* P = part + (size_t)blockIdx.x * (16 * 16 * TAPS + 16);
  for (int tap = 0; tap < TAPS; ++tap) P[(co * 16 + ci) * TAPS + tap] = acc[tap];
  if (ci == 0) P[16 * 16 * TAPS + co] = accb;
}

// fixed-order sum of the per-CTA partials into the flat gradient of one layer
__global__ void dw_reduce_kernel(const float* __restrict__ part, int nparts, float* __restrict__ grad, int cin, int cout,
                                 int taps) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int nw = cout * cin * taps;
  if (i >= nw + cout) return;
  int src;
  if (i < nw) {
    int tap = i % taps, ci = (i / taps) % cin, co = i / (taps * cin);
    src = (co * 16 + ci) * taps + tap;
  } else {
    src = 16 * 16 * taps + (i - nw);
  }
  float s = 0.f;
  for (int p = 0; p < nparts; ++p) s += part[(size_t)p * (16 * 16 * taps + 16) + src];
  grad[i] = s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// [N][P][2] -> [N][2][P]
__global__ void unpack_output_kernel(const float* __restrict__ o, float* __restrict__ out, long long npix, long long P) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  long long n = i / P, p = i % P;
  out[(n * 2 + 0) * P + p] = o[i * 2 + 0];
  out[(n * 2 + 1) * P + p] = o[i * 2 + 1];
}

// ------------------------------------------------------- fused inference --
// All four layers of the 2D network in one pass over the image: a CTA stages a
// (TX+8) x (TY+8) tile of the five input channels (bf16, periodic wrap) and keeps
// every intermediate activation in shared memory, each layer computing its output
// on a region one cell smaller per side than its input (38 x 22, 36 x 20, 34 x 18,
// then the 32 x 16 output tile for TX = 32, TY = 16), so the only global traffic is
// the float32 input and output images.  Contractions: mma m16n8k8 (layer 1, whose
// five input channels pad to K = 8) and m16n8k16 (layers 2-4), bf16 operands,
// float32 accumulation, one tap per K step (implicit GEMM, M = 16 region pixels in
// raster order); each warp keeps the layer's weight fragments of all nine taps in
// registers.  Activations in shared memory: 16 bf16 channels at a 48-byte pixel
// stride (conflict-free fragment loads); the input tile: 8 channels, 16 bytes.
//
// GELU here is the tanh form 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))
// (Hendrycks and Gimpel, 2016) with the hardware tanh approximation, in place of
// the exact erf form of the training kernels.  The form differs from the erf form
// by at most 4.7e-4 (at z = 2.70; evaluated in float64 over [-12, 12]); the
// hardware tanh adds |z|/2 times its own error, of order 2^-11.  Both are of the
// size of the bf16 rounding of the stored activations (2^-9 relative); the test of
// this kernel bounds its output against the exact-GELU layer-by-layer network.

__device__ __forceinline__ void mma1688(float* c, const uint32_t* a, uint32_t b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(b));
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// GELU (tanh form) of a pair, packed float32 arithmetic
__device__ __forceinline__ float2 gelu_tanh2(float2 z) {
  const float2 z2 = __fmul2_rn(z, z);
  const float2 u = __fmul2_rn(z, __ffma2_rn(z2, make_float2(0.0356774081f, 0.0356774081f),
                                            make_float2(0.7978845608f, 0.7978845608f)));
  const float2 hz = __fmul2_rn(z, make_float2(0.5f, 0.5f));
  return __ffma2_rn(hz, make_float2(tanh_approx(u.x), tanh_approx(u.y)), hz);
}

constexpr int kFuseTX = 32, kFuseTY = 16;  // output tile of the fused inference
constexpr int kFuseThreads = 256;

struct FusedArgs {
  const float* in;    // [N][5][H][W]
  float* out;         // [N][2][H][W]
  const bf16* w[4];   // packed [tap][npad][CS]
  const float* b[4];  // biases
  int N, H, W;
};

__host__ __device__ constexpr int fused_region(int l, int d) { return (d == 0 ? kFuseTX : kFuseTY) + 2 * (4 - l); }
__host__ __device__ constexpr int fused_pix(int l) { return fused_region(l, 0) * fused_region(l, 1); }
constexpr size_t kFusedA = (size_t)fused_pix(2) * CS > (size_t)fused_pix(0) * 8 ? (size_t)fused_pix(2) * CS
                                                                                 : (size_t)fused_pix(0) * 8;
constexpr size_t kFusedB = (size_t)fused_pix(1) * CS;
constexpr size_t kFusedSmem = (kFusedA + kFusedB) * sizeof(bf16);

// four (x4) or two (x2) 8x8 bf16 matrices from shared memory, one 16-byte row address per lane
__device__ __forceinline__ void ldsm_x4(uint32_t* r, uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t* r, uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}

// Layer L (1..4): region L-1 (in; 8 bf16 per pixel for L = 1, else CS) -> region L.  Each warp
// takes pairs of 16-pixel chunks (four independent accumulator chains); the A fragments of a
// tap come by one ldmatrix per chunk (lane = pixel row (lane & 15), K half (lane >> 4)), the
// weight fragments of all nine taps from global memory into registers once per layer.
// Hidden layers: bias, GELU, bf16 into `out` (shared); layer 4: bias, float32 into the image.
template <int L>
__device__ __forceinline__ void fused_layer(const FusedArgs& a, const bf16* s_in, bf16* s_out, int n, int x0, int y0,
                                            int warp, int lane) {
  constexpr bool LAST = L == 4, K8 = L == 1;
  constexpr int NT = LAST ? 1 : 2, NPAD = LAST ? 8 : 16, PB = K8 ? 16 : CS * 2;  // pixel stride (bytes) of `in`
  constexpr int wo = fused_region(L, 0), ho = fused_region(L, 1), wi = wo + 2, npix = wo * ho;
  constexpr int nchunks = (npix + 15) / 16;
  const int g = lane >> 2, t = lane & 3;
  const uint32_t* w32 = reinterpret_cast<const uint32_t*>(a.w[L - 1]);
  uint32_t bq[9][NT][K8 ? 1 : 2];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int row = tap * NPAD + nt * 8 + g;
      bq[tap][nt][0] = __ldg(w32 + row * (CS / 2) + t);
      if (!K8) bq[tap][nt][K8 ? 0 : 1] = __ldg(w32 + row * (CS / 2) + 4 + t);
    }
  const float* bias = a.b[L - 1];
  const float2 bb0 = make_float2(__ldg(bias + 2 * t), __ldg(bias + 2 * t + 1));
  const float2 bb1 = LAST ? bb0 : make_float2(__ldg(bias + 8 + 2 * t), __ldg(bias + 9 + 2 * t));
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(s_in) + (K8 ? 0 : (lane >> 4) * 16);
  const int r = lane & 15;
  for (int c = 2 * warp; c < nchunks; c += 2 * (kFuseThreads / 32)) {
    uint32_t prow[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int u = min(16 * (c + j) + r, npix - 1);  // rows beyond the region compute a clamped pixel
      prow[j] = sbase + ((u / wo + 1) * wi + u % wo + 1) * PB;
    }
    float acc[2][NT][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) acc[j][nt][0] = acc[j][nt][1] = acc[j][nt][2] = acc[j][nt][3] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int off = ((tap / 3 - 1) * wi + (tap % 3 - 1)) * PB;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (K8) {
          uint32_t av[2];
          ldsm_x2(av, prow[j] + off);
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) mma1688(acc[j][nt], av, bq[tap][nt][0]);
        } else {
          uint32_t av[4];
          ldsm_x4(av, prow[j] + off);
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) mma16816(acc[j][nt], av, bq[tap][nt]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int v0 = 16 * (c + j) + g, v1 = v0 + 8;
      if (LAST) {
        if (t == 0) {  // columns 0 and 1 are the two output channels
          const long long P = (long long)a.H * a.W;
          float* out = a.out + (long long)n * 2 * P;
          const long long o0 = (long long)(y0 + v0 / wo) * a.W + x0 + v0 % wo;
          const long long o1 = (long long)(y0 + v1 / wo) * a.W + x0 + v1 % wo;
          out[o0] = acc[j][0][0] + bb0.x;
          out[P + o0] = acc[j][0][1] + bb0.y;
          out[o1] = acc[j][0][2] + bb0.x;
          out[P + o1] = acc[j][0][3] + bb0.y;
        }
      } else {
        uint32_t* o32 = reinterpret_cast<uint32_t*>(s_out);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const float2 bb = nt ? bb1 : bb0;
          const float2 r0 = gelu_tanh2(__fadd2_rn(make_float2(acc[j][nt][0], acc[j][nt][1]), bb));
          const float2 r1 = gelu_tanh2(__fadd2_rn(make_float2(acc[j][nt][2], acc[j][nt][3]), bb));
          const __nv_bfloat162 h0 = __floats2bfloat162_rn(r0.x, r0.y), h1 = __floats2bfloat162_rn(r1.x, r1.y);
          if (v0 < npix) o32[v0 * (CS / 2) + nt * 4 + t] = *reinterpret_cast<const uint32_t*>(&h0);
          if (v1 < npix) o32[v1 * (CS / 2) + nt * 4 + t] = *reinterpret_cast<const uint32_t*>(&h1);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kFuseThreads, 3) cnn_fused2d_kernel(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char fused_smem[];
  bf16* s_a = reinterpret_cast<bf16*>(fused_smem);  // region 0 (8-channel input), then region 2
  bf16* s_b = s_a + kFusedA;                        // region 1, then region 3
  const int tiles_x = a.W / kFuseTX, tiles_y = a.H / kFuseTY;
  int tile = blockIdx.x;
  const int x0 = (tile % tiles_x) * kFuseTX;
  tile /= tiles_x;
  const int y0 = (tile % tiles_y) * kFuseTY;
  const int n = tile / tiles_y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // region 0: the five input channels of the tile and its 4-cell periodic halo, bf16, 8 per pixel
  {
    constexpr int w0 = fused_region(0, 0), np0 = fused_pix(0);
    const long long P = (long long)a.H * a.W;
    const float* in = a.in + (long long)n * 5 * P;
    for (int p = threadIdx.x; p < np0; p += kFuseThreads) {
      const int gx = wrapi(x0 + p % w0 - 4, a.W), gy = wrapi(y0 + p / w0 - 4, a.H);
      const long long q = (long long)gy * a.W + gx;
      float f[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) f[c] = __ldg(in + c * P + q);
      const __nv_bfloat162 h01 = __floats2bfloat162_rn(f[0], f[1]), h23 = __floats2bfloat162_rn(f[2], f[3]),
                           h4 = __floats2bfloat162_rn(f[4], 0.f);
      reinterpret_cast<uint4*>(s_a)[p] = make_uint4(*reinterpret_cast<const uint32_t*>(&h01),
                                                    *reinterpret_cast<const uint32_t*>(&h23),
                                                    *reinterpret_cast<const uint32_t*>(&h4), 0u);
    }
  }
  __syncthreads();
  fused_layer<1>(a, s_a, s_b, n, x0, y0, warp, lane);
  __syncthreads();
  fused_layer<2>(a, s_b, s_a, n, x0, y0, warp, lane);
  __syncthreads();
  fused_layer<3>(a, s_a, s_b, n, x0, y0, warp, lane);
  __syncthreads();
  fused_layer<4>(a, s_b, nullptr, n, x0, y0, warp, lane);
}

// ------------------------------------------------------------------- host --
struct Buf {
  void* p = nullptr;
  size_t n = 0;
  ~Buf() {
    if (p) cudaFree(p);
  }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

long long layer_off(int nd, int l) {
  long long o = 0;
  for (int i = 0; i < l; ++i) o += (long long)kCh[i + 1] * kCh[i] * ntaps(nd) + kCh[i + 1];
  return o;
}

}  // namespace cnngpu

using namespace cnngpu;

struct cnn_handle {
  int nd = 2;
  long long nparams = 0;
  int step = 0;
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Buf params, grad, m, v, wfwd[4], wbwd[4], loss;
  Buf x0, z[4], act[4], outp, dz[5], part, out_user;
  Buf qres;  // q of the operator-weighted loss, float2 per pixel
  long long cap_pix = 0;
  int sms = 152;
  long long launches = 0;
  int loss_kind = CNN_LOSS_MSE;
  float kappa[2] = {0.f, 0.f};

  cudaEvent_t order_ev = nullptr;  // orders inference on a caller's stream against this stream

  ~cnn_handle() {
    if (order_ev) cudaEventDestroy(order_ev);
    if (own_stream) cudaStreamDestroy(stream);
  }
  int fail(int code, const std::string& s) {
    err = s;
    return code;
  }
  int cuda(cudaError_t e, const char* w) {
    if (e == cudaSuccess) return AMR_OK;
    err = std::string("CUDA error ") + cudaGetErrorString(e) + " in " + w;
    return e == cudaErrorMemoryAllocation ? AMR_ERR_OOM : AMR_ERR_CUDA;
  }
  int taps() const { return ntaps(nd); }

  int repack() {
    for (int l = 0; l < 4; ++l) {
      int npad = l == 3 ? 8 : 16;
      int total = taps() * npad * CS;
      pack_weights_kernel<<<(total + 255) / 256, 256, 0, stream>>>(params.as<float>() + layer_off(nd, l),
                                                                   wfwd[l].as<bf16>(), kCh[l], kCh[l + 1], taps(), npad, 0);
      ++launches;
      if (l > 0) {
        int tot2 = taps() * 16 * CS;
        pack_weights_kernel<<<(tot2 + 255) / 256, 256, 0, stream>>>(params.as<float>() + layer_off(nd, l),
                                                                     wbwd[l].as<bf16>(), kCh[l], kCh[l + 1], taps(), 16, 1);
        ++launches;
      }
    }
    return cuda(cudaGetLastError(), "pack weights");
  }

  int ensure_acts(long long npix) {
    if (npix <= cap_pix) return AMR_OK;
    int rc;
    size_t b16 = (size_t)npix * 16 * sizeof(bf16);
    if ((rc = cuda(x0.ensure(b16), "alloc"))) return rc;
    for (int l = 0; l < 4; ++l)
      if ((rc = cuda(z[l].ensure(b16), "alloc")) || (rc = cuda(act[l].ensure(b16), "alloc"))) return rc;
    for (int l = 0; l < 5; ++l)
      if ((rc = cuda(dz[l].ensure(b16), "alloc"))) return rc;
    if ((rc = cuda(outp.ensure((size_t)npix * 2 * sizeof(float)), "alloc"))) return rc;
    cap_pix = npix;
    return AMR_OK;
  }

  bool shape_ok(int N, int D, int H, int W) const {
    if (N < 1 || H < 1 || W < 1) return false;
    if (nd == 2) return D == 1 && H % TD<2>::TY == 0 && W % TD<2>::TX == 0;
    return D % TD<3>::TZ == 0 && H % TD<3>::TY == 0 && W % TD<3>::TX == 0;
  }

  // infer: no pre-activations are kept (no backward pass follows)
  template <int ND>
  int forward_t(int N, int D, int H, int W, bool infer) {
    using T = TD<ND>;
    int tiles = N * (D / T::TZ) * (H / T::TY) * (W / T::TX);
    const bf16* in = x0.as<bf16>();
    for (int l = 0; l < 4; ++l) {
      ConvArgs a{};
      a.in = in;
      a.w = wfwd[l].as<bf16>();
      a.bias = params.as<float>() + layer_off(nd, l) + (long long)kCh[l + 1] * kCh[l] * taps();
      a.N = N;
      a.D = D;
      a.H = H;
      a.W = W;
      if (l < 3) {
        a.z_out = z[l].as<bf16>();
        a.a_out = act[l].as<bf16>();
        if (infer)
          conv_kernel<ND, FWD_INFER><<<tiles, 256, conv_smem_bytes<ND, FWD_INFER>(), stream>>>(a);
        else
          conv_kernel<ND, FWD_GELU><<<tiles, 256, conv_smem_bytes<ND, FWD_GELU>(), stream>>>(a);
        in = act[l].as<bf16>();
      } else {
        a.out = outp.as<float>();
        conv_kernel<ND, FWD_OUT><<<tiles, 256, conv_smem_bytes<ND, FWD_OUT>(), stream>>>(a);
      }
      ++launches;
    }
    return cuda(cudaGetLastError(), "forward");
  }

  template <int ND>
  int backward_t(int N, int D, int H, int W) {
    using T = TD<ND>;
    int tiles = N * (D / T::TZ) * (H / T::TY) * (W / T::TX);
    int parts = std::min(tiles, 2 * sms);
    int rc;
    if ((rc = cuda(part.ensure((size_t)parts * (16 * 16 * T::T + 16) * sizeof(float)), "alloc"))) return rc;
    // dz[4] = dL/dz of the output layer (from the loss kernel); dz[l] for l = 3, 2, 1
    for (int l = 3; l >= 0; --l) {
      const bf16* aprev = l == 0 ? x0.as<bf16>() : act[l - 1].as<bf16>();
      dw_kernel<ND><<<parts, 256, 0, stream>>>(aprev, dz[l + 1].as<bf16>(), part.as<float>(), kCh[l], kCh[l + 1], N, D,
                                               H, W);
      int nw = kCh[l + 1] * kCh[l] * T::T + kCh[l + 1];
      dw_reduce_kernel<<<(nw + 255) / 256, 256, 0, stream>>>(part.as<float>(), parts, grad.as<float>() + layer_off(nd, l),
                                                             kCh[l], kCh[l + 1], T::T);
      launches += 2;
      if (l > 0) {
        ConvArgs a{};
        a.in = dz[l + 1].as<bf16>();
        a.w = wbwd[l].as<bf16>();
        a.zprev = z[l - 1].as<bf16>();
        a.dz_out = dz[l].as<bf16>();
        a.N = N;
        a.D = D;
        a.H = H;
        a.W = W;
        conv_kernel<ND, BWD_GELU><<<tiles, 256, conv_smem_bytes<ND, BWD_GELU>(), stream>>>(a);
        ++launches;
      }
    }
    return cuda(cudaGetLastError(), "backward");
  }

  int forward(int N, int D, int H, int W, bool infer = false) {
    return nd == 2 ? forward_t<2>(N, D, H, W, infer) : forward_t<3>(N, D, H, W, infer);
  }
  int backward(int N, int D, int H, int W) { return nd == 2 ? backward_t<2>(N, D, H, W) : backward_t<3>(N, D, H, W); }

  int pack_input(const float* in, long long npix, long long P) {
    pack_input_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, stream>>>(in, x0.as<bf16>(), npix, P);
    ++launches;
    return cuda(cudaGetLastError(), "pack input");
  }

  // loss + gradient of the masked loss (MSE or operator-weighted) into `grad`; returns via *loss_out (host)
  int loss_and_grad(const float* in, const float* target, int N, int D, int H, int W, int margin, float* loss_out) {
    long long P = (long long)D * H * W, npix = (long long)N * P;
    int rc;
    if (loss_kind == CNN_LOSS_OPERATOR && margin < 1) return fail(AMR_ERR_INVALID_ARG, "operator loss needs margin >= 1");
    if ((rc = ensure_acts(npix))) return rc;
    if ((rc = pack_input(in, npix, P)) || (rc = forward(N, D, H, W))) return rc;
    long long cnt = 0;
    {
      long long inx = std::max(0, W - 2 * margin), iny = std::max(0, H - 2 * margin);
      long long inz = nd == 3 ? std::max(0, D - 2 * margin) : 1;
      cnt = (long long)N * 2 * inx * iny * inz;
    }
    if (cnt == 0) return fail(AMR_ERR_INVALID_ARG, "margin leaves no pixel");
    if ((rc = cuda(cudaMemsetAsync(loss.p, 0, sizeof(float), stream), "memset"))) return rc;
    unsigned grid = (unsigned)((npix + 255) / 256);
    if (loss_kind == CNN_LOSS_OPERATOR) {
      if ((rc = cuda(qres.ensure((size_t)npix * 2 * sizeof(float)), "alloc"))) return rc;
      op_q_kernel<<<grid, 256, 0, stream>>>(outp.as<float>(), target, qres.as<float>(), loss.as<float>(), npix, D, H,
                                            W, margin, nd, kappa[0], kappa[1], 1.f / (float)cnt);
      op_grad_kernel<<<grid, 256, 0, stream>>>(qres.as<float>(), dz[4].as<bf16>(), npix, D, H, W, nd, kappa[0],
                                               kappa[1], 1.f / (float)cnt);
      launches += 2;
    } else {
      loss_grad_kernel<<<grid, 256, 0, stream>>>(outp.as<float>(), target, dz[4].as<bf16>(), loss.as<float>(), npix,
                                                 D, H, W, margin, nd, 1.f / (float)cnt);
      ++launches;
    }
    if ((rc = backward(N, D, H, W))) return rc;
    if (loss_out) {
      if ((rc = cuda(cudaMemcpyAsync(loss_out, loss.p, sizeof(float), cudaMemcpyDeviceToHost, stream), "copy")))
        return rc;
      if ((rc = cuda(cudaStreamSynchronize(stream), "sync"))) return rc;
    }
    return AMR_OK;
  }
};

// inference on `stream` (NULL = the handle's own) without a final synchronisation
// the fused single-pass inference applies to 2D images whose sides tile by 32 x 16
static bool fused_ok(const cnn_handle* h, int D, int H, int W) {
  return h->nd == 2 && D == 1 && W % kFuseTX == 0 && H % kFuseTY == 0;
}

static int fused_forward(cnn_handle* h, const float* in, int N, int H, int W, float* out, cudaStream_t s) {
  FusedArgs a{};
  a.in = in;
  a.out = out;
  for (int l = 0; l < 4; ++l) {
    a.w[l] = h->wfwd[l].as<bf16>();
    a.b[l] = h->params.as<float>() + layer_off(2, l) + (long long)kCh[l + 1] * kCh[l] * 9;
  }
  a.N = N;
  a.H = H;
  a.W = W;
  const unsigned tiles = (unsigned)N * (H / kFuseTY) * (W / kFuseTX);
  cnn_fused2d_kernel<<<tiles, kFuseThreads, kFusedSmem, s>>>(a);
  ++h->launches;
  return h->cuda(cudaGetLastError(), "fused inference");
}

bool cnn_fused_applies(const cnn_handle* h, int D, int H, int W) { return h && fused_ok(h, D, H, W); }

cudaStream_t cnn_own_stream(const cnn_handle* h) { return h ? h->stream : nullptr; }

int cnn_enqueue_fused(cnn_handle* h, const float* in, int N, int H, int W, float* out, cudaStream_t s) {
  if (!h || !in || !out || N < 1 || !fused_ok(h, 1, H, W)) return AMR_ERR_INVALID_ARG;
  return fused_forward(h, in, N, H, W, out, s);
}

int cnn_forward_async(cnn_handle* h, const float* in, int N, int D, int H, int W, float* out, cudaStream_t stream,
                      bool fused) {
  if (!h || !in || !out || !h->shape_ok(N, D, H, W)) return AMR_ERR_INVALID_ARG;
  long long P = (long long)D * H * W, npix = (long long)N * P;
  if (fused && fused_ok(h, D, H, W)) {
    // no intermediate buffers (nothing to allocate): one kernel on `stream`, ordered after the
    // handle's pending work (weight repacks) by an event when the streams differ
    cudaStream_t own = h->stream;
    int rc;
    if (stream && stream != own) {
      if (!h->order_ev && (rc = h->cuda(cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming), "event")))
        return rc;
      if ((rc = h->cuda(cudaEventRecord(h->order_ev, own), "event")) ||
          (rc = h->cuda(cudaStreamWaitEvent(stream, h->order_ev, 0), "event")))
        return rc;
    }
    if ((rc = fused_forward(h, in, N, H, W, out, stream ? stream : own))) return rc;
    if (stream && stream != own &&  // the handle's later work (repacks) after this inference
        ((rc = h->cuda(cudaEventRecord(h->order_ev, stream), "event")) ||
         (rc = h->cuda(cudaStreamWaitEvent(own, h->order_ev, 0), "event"))))
      return rc;
    return AMR_OK;
  }
  cudaStream_t own = h->stream;
  int rc;
  const bool other = stream && stream != own;
  if (other) {
    // `stream` waits for the handle's pending work (weight repacks after Adam steps), and
    // the handle's stream later waits for this inference (it reads the packed weights)
    if (!h->order_ev && (rc = h->cuda(cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming), "event")))
      return rc;
    if ((rc = h->cuda(cudaEventRecord(h->order_ev, own), "event")) ||
        (rc = h->cuda(cudaStreamWaitEvent(stream, h->order_ev, 0), "event")))
      return rc;
    h->stream = stream;
  }
  if (!(rc = h->ensure_acts(npix)) && !(rc = h->pack_input(in, npix, P)) && !(rc = h->forward(N, D, H, W, true))) {
    unpack_output_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, h->stream>>>(h->outp.as<float>(), out, npix, P);
    ++h->launches;
    rc = h->cuda(cudaGetLastError(), "unpack");
  }
  h->stream = own;
  if (other && !rc) {
    if ((rc = h->cuda(cudaEventRecord(h->order_ev, stream), "event")) ||
        (rc = h->cuda(cudaStreamWaitEvent(own, h->order_ev, 0), "event")))
      return rc;
  }
  return rc;
}

extern "C" {

int cnn_create(int ndim, unsigned long long seed, void* stream, cnn_handle** out) {
  if (!out || (ndim != 2 && ndim != 3)) return AMR_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<cnn_handle> h(new cnn_handle());
  h->nd = ndim;
  h->nparams = layer_off(ndim, 4);
  h->stream = (cudaStream_t)stream;
  if (!h->stream) {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return AMR_ERR_CUDA;
    h->own_stream = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  // the 3D convolution tile and its weights exceed the 48 KB default
  if (cudaFuncSetAttribute(conv_kernel<3, FWD_GELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem_bytes<3, FWD_GELU>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_kernel<3, FWD_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem_bytes<3, FWD_OUT>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_kernel<3, FWD_INFER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem_bytes<3, FWD_INFER>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_kernel<3, BWD_GELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem_bytes<3, BWD_GELU>()) != cudaSuccess ||
      cudaFuncSetAttribute(cnn_fused2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem) !=
          cudaSuccess)
    return AMR_ERR_CUDA;
  size_t pb = (size_t)h->nparams * sizeof(float);
  int rc;
  if ((rc = h->cuda(h->params.ensure(pb), "alloc")) || (rc = h->cuda(h->grad.ensure(pb), "alloc")) ||
      (rc = h->cuda(h->m.ensure(pb), "alloc")) || (rc = h->cuda(h->v.ensure(pb), "alloc")) ||
      (rc = h->cuda(h->loss.ensure(sizeof(float)), "alloc")))
    return rc;
  for (int l = 0; l < 4; ++l) {
    int npad = l == 3 ? 8 : 16;
    if ((rc = h->cuda(h->wfwd[l].ensure((size_t)ntaps(ndim) * npad * CS * sizeof(bf16)), "alloc"))) return rc;
    if (l > 0 && (rc = h->cuda(h->wbwd[l].ensure((size_t)ntaps(ndim) * 16 * CS * sizeof(bf16)), "alloc"))) return rc;
  }
  // He-normal initialisation, zero biases
  std::vector<float> p(h->nparams, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < 4; ++l) {
    int fan_in = kCh[l] * ntaps(ndim);
    std::normal_distribution<float> nd_(0.f, std::sqrt(2.f / fan_in) * (l == 3 ? 0.1f : 1.f));
    long long o = layer_off(ndim, l);
    for (long long i = 0; i < (long long)kCh[l + 1] * kCh[l] * ntaps(ndim); ++i) p[o + i] = nd_(rng);
  }
  if ((rc = h->cuda(cudaMemcpy(h->params.p, p.data(), pb, cudaMemcpyHostToDevice), "copy")) ||
      (rc = h->cuda(cudaMemset(h->m.p, 0, pb), "memset")) || (rc = h->cuda(cudaMemset(h->v.p, 0, pb), "memset")))
    return rc;
  if ((rc = h->repack())) return rc;
  if ((rc = h->cuda(cudaStreamSynchronize(h->stream), "sync"))) return rc;
  *out = h.release();
  return AMR_OK;
}

int cnn_destroy(cnn_handle* h) {
  if (!h) return AMR_ERR_INVALID_ARG;
  delete h;
  return AMR_OK;
}

const char* cnn_last_error(const cnn_handle* h) { return h ? h->err.c_str() : "null handle"; }

int cnn_num_params(const cnn_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = h->nparams;
  return AMR_OK;
}

int cnn_set_params(cnn_handle* h, const float* p, long long n) {
  if (!h || !p || n != h->nparams) return AMR_ERR_INVALID_ARG;
  int rc;
  if ((rc = h->cuda(cudaMemcpyAsync(h->params.p, p, n * sizeof(float), cudaMemcpyHostToDevice, h->stream), "copy")))
    return rc;
  if ((rc = h->cuda(cudaMemsetAsync(h->m.p, 0, n * sizeof(float), h->stream), "memset")) ||
      (rc = h->cuda(cudaMemsetAsync(h->v.p, 0, n * sizeof(float), h->stream), "memset")))
    return rc;
  h->step = 0;
  if ((rc = h->repack())) return rc;
  return h->cuda(cudaStreamSynchronize(h->stream), "sync");
}

int cnn_get_params(cnn_handle* h, float* p, long long n) {
  if (!h || !p || n != h->nparams) return AMR_ERR_INVALID_ARG;
  int rc;
  if ((rc = h->cuda(cudaMemcpyAsync(p, h->params.p, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "copy")))
    return rc;
  return h->cuda(cudaStreamSynchronize(h->stream), "sync");
}

int cnn_forward(cnn_handle* h, const float* in, int N, int D, int H, int W, float* out) {
  int rc = cnn_forward_async(h, in, N, D, H, W, out, nullptr, false);
  if (rc) return rc;
  return h->cuda(cudaStreamSynchronize(h->stream), "sync");
}

int cnn_gradient(cnn_handle* h, const float* in, const float* target, int N, int D, int H, int W, int margin,
                 float* grad_host, float* loss) {
  if (!h || !in || !target || !h->shape_ok(N, D, H, W) || margin < 0) return AMR_ERR_INVALID_ARG;
  int rc = h->loss_and_grad(in, target, N, D, H, W, margin, loss);
  if (rc) return rc;
  if (grad_host) {
    if ((rc = h->cuda(cudaMemcpyAsync(grad_host, h->grad.p, h->nparams * sizeof(float), cudaMemcpyDeviceToHost,
                                      h->stream), "copy")))
      return rc;
    return h->cuda(cudaStreamSynchronize(h->stream), "sync");
  }
  return AMR_OK;
}

int cnn_train_step(cnn_handle* h, const float* in, const float* target, int N, int D, int H, int W, int margin, float lr,
                   float* loss) {
  if (!h || !in || !target || !h->shape_ok(N, D, H, W) || margin < 0 || !(lr > 0)) return AMR_ERR_INVALID_ARG;
  int rc = h->loss_and_grad(in, target, N, D, H, W, margin, loss);
  if (rc) return rc;
  h->step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float c1 = 1.f - std::pow(b1, (float)h->step), c2 = 1.f - std::pow(b2, (float)h->step);
  adam_kernel<<<(unsigned)((h->nparams + 255) / 256), 256, 0, h->stream>>>(
      h->params.as<float>(), h->grad.as<float>(), h->m.as<float>(), h->v.as<float>(), h->nparams, lr, b1, b2, eps, c1, c2);
  ++h->launches;
  if ((rc = h->repack())) return rc;
  if (loss) return h->cuda(cudaStreamSynchronize(h->stream), "sync");
  return h->cuda(cudaGetLastError(), "adam");
}

int cnn_set_loss(cnn_handle* h, int kind, const double* kappa) {
  if (!h) return AMR_ERR_INVALID_ARG;
  if (kind == CNN_LOSS_MSE) {
    h->loss_kind = kind;
    return AMR_OK;
  }
  if (kind != CNN_LOSS_OPERATOR || !kappa) return h->fail(AMR_ERR_INVALID_ARG, "cnn_set_loss: bad kind or kappa");
  for (int c = 0; c < 2; ++c)
    if (!(kappa[c] >= 0.0) || !std::isfinite(kappa[c])) return h->fail(AMR_ERR_INVALID_ARG, "cnn_set_loss: kappa");
  h->loss_kind = kind;
  h->kappa[0] = (float)kappa[0];
  h->kappa[1] = (float)kappa[1];
  return AMR_OK;
}

int cnn_infer(cnn_handle* h, const float* in, int N, int D, int H, int W, float* out) {
  int rc = cnn_forward_async(h, in, N, D, H, W, out, nullptr, true);
  if (rc) return rc;
  return h->cuda(cudaStreamSynchronize(h->stream), "sync");
}

// parameter file: 8-byte magic, int32 ndim, int32 0, int64 count, count float32 (host byte order)
static const char kCnnMagic[8] = {'A', 'M', 'R', 'V', 'C', 'N', 'N', '1'};

int cnn_save(cnn_handle* h, const char* path) {
  if (!h || !path) return AMR_ERR_INVALID_ARG;
  std::vector<float> p((size_t)h->nparams);
  int rc = cnn_get_params(h, p.data(), h->nparams);
  if (rc) return rc;
  FILE* f = std::fopen(path, "wb");
  if (!f) return h->fail(AMR_ERR_INVALID_ARG, std::string("cannot open ") + path);
  const int32_t hdr[2] = {h->nd, 0};
  const int64_t n = h->nparams;
  bool ok = std::fwrite(kCnnMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            std::fwrite(&n, sizeof(n), 1, f) == 1 && std::fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? AMR_OK : h->fail(AMR_ERR_INVALID_ARG, std::string("cannot write ") + path);
}

int cnn_load(cnn_handle* h, const char* path) {
  if (!h || !path) return AMR_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return h->fail(AMR_ERR_INVALID_ARG, std::string("cannot open ") + path);
  char magic[8];
  int32_t hdr[2];
  int64_t n = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCnnMagic, 8) == 0 &&
            std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(&n, sizeof(n), 1, f) == 1 && hdr[0] == h->nd &&
            n == h->nparams;
  std::vector<float> p;
  if (ok) {
    p.resize((size_t)n);
    ok = std::fread(p.data(), sizeof(float), p.size(), f) == p.size();
  }
  std::fclose(f);
  if (!ok) return h->fail(AMR_ERR_INVALID_ARG, std::string("not a parameter file of this network: ") + path);
  return cnn_set_params(h, p.data(), h->nparams);
}

int cnn_kernel_launches(const cnn_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = h->launches;
  return AMR_OK;
}

}  // extern "C"
