// Layer kernels of the 3D U-Net that predicts the PCG initial guess (no paper
// counterpart; the network is defined with the C ABI in include/tm.h): zero-padded
// 3x3x3 and 1x1x1 convolutions with bias and optional ReLU, their gradients with
// respect to input, weights and bias, 2x2x2 average pooling, nearest 2x upsampling
// and their adjoints.  Activations are N x C x X x Y x Z, FP32, contiguous; weights
// Cout x Cin x K x K x K.  Direct CUDA-core kernels: one thread per output value,
// fixed summation orders (deterministic).
#include <cuda_runtime.h>

#include "tm_internal.h"

namespace amr {

namespace {

constexpr int kT = 256;

int grid_of(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  if (g < 1) g = 1;
  if (g > 16 * device_sms()) g = 16 * device_sms();
  return (int)g;
}

// y = conv(x) + b, then ReLU if relu.  K in {1, 3}, padding K / 2.
__global__ void conv_fwd_kernel(const float *x, const float *w, const float *b, float *y, int N, int Ci, int Co,
                                int X, int Y, int Z, int K, int relu) {
  const int64_t S = (int64_t)X * Y * Z, total = (int64_t)N * Co * S;
  const int P = K / 2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % Z), j = (int)((t / Z) % Y), i = (int)((t / ((int64_t)Y * Z)) % X);
    const int o = (int)((t / S) % Co), n = (int)(t / ((int64_t)Co * S));
    float acc = b[o];
    for (int c = 0; c < Ci; ++c) {
      const float *xc = x + ((int64_t)n * Ci + c) * S;
      const float *wc = w + ((int64_t)o * Ci + c) * K * K * K;
      for (int a = 0; a < K; ++a) {
        const int ii = i + a - P;
        if (ii < 0 || ii >= X) continue;
        for (int bb = 0; bb < K; ++bb) {
          const int jj = j + bb - P;
          if (jj < 0 || jj >= Y) continue;
          for (int cc = 0; cc < K; ++cc) {
            const int kk = k + cc - P;
            if (kk < 0 || kk >= Z) continue;
            acc += wc[(a * K + bb) * K + cc] * xc[((int64_t)ii * Y + jj) * Z + kk];
          }
        }
      }
    }
    y[t] = (relu && acc < 0.0f) ? 0.0f : acc;
  }
}

// g *= (y > 0): gradient through ReLU from its output y.
__global__ void relu_bwd_kernel(const float *y, float *g, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    if (!(y[t] > 0.0f)) g[t] = 0.0f;
}

// dx (+)= conv^T(dy): dx[n,c,p] = sum_o sum_taps w[o,c,tap] dy[n,o,p - tap + P].
__global__ void conv_bwd_data_kernel(const float *dy, const float *w, float *dx, int N, int Ci, int Co, int X, int Y,
                                     int Z, int K, int accumulate) {
  const int64_t S = (int64_t)X * Y * Z, total = (int64_t)N * Ci * S;
  const int P = K / 2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % Z), j = (int)((t / Z) % Y), i = (int)((t / ((int64_t)Y * Z)) % X);
    const int c = (int)((t / S) % Ci), n = (int)(t / ((int64_t)Ci * S));
    float acc = 0.0f;
    for (int o = 0; o < Co; ++o) {
      const float *dyo = dy + ((int64_t)n * Co + o) * S;
      const float *wc = w + ((int64_t)o * Ci + c) * K * K * K;
      for (int a = 0; a < K; ++a) {
        const int ii = i - a + P;
        if (ii < 0 || ii >= X) continue;
        for (int bb = 0; bb < K; ++bb) {
          const int jj = j - bb + P;
          if (jj < 0 || jj >= Y) continue;
          for (int cc = 0; cc < K; ++cc) {
            const int kk = k - cc + P;
            if (kk < 0 || kk >= Z) continue;
            acc += wc[(a * K + bb) * K + cc] * dyo[((int64_t)ii * Y + jj) * Z + kk];
          }
        }
      }
    }
    dx[t] = accumulate ? dx[t] + acc : acc;
  }
}

// dw[o,c,tap] = sum_n sum_p dy[n,o,p] x[n,c,p + tap - P]; db[o] = sum dy[n,o,.] (when c == 0).
// One CTA per (o, c, tap); a fixed-order block reduction over (n, p).
__global__ void __launch_bounds__(kT) conv_bwd_weight_kernel(const float *x, const float *dy, float *dw, float *db,
                                                             int N, int Ci, int Co, int X, int Y, int Z, int K) {
  const int KKK = K * K * K;
  const int tap = blockIdx.x % KKK, c = (blockIdx.x / KKK) % Ci, o = blockIdx.x / (KKK * Ci);
  const int a = tap / (K * K), bb = (tap / K) % K, cc = tap % K, P = K / 2;
  const int64_t S = (int64_t)X * Y * Z;
  double acc = 0.0, accb = 0.0;
  for (int n = 0; n < N; ++n) {
    const float *dyo = dy + ((int64_t)n * Co + o) * S;
    const float *xc = x + ((int64_t)n * Ci + c) * S;
    for (int64_t p = threadIdx.x; p < S; p += kT) {
      const int k = (int)(p % Z), j = (int)((p / Z) % Y), i = (int)(p / ((int64_t)Y * Z));
      const int ii = i + a - P, jj = j + bb - P, kk = k + cc - P;
      const float g = dyo[p];
      if (ii >= 0 && ii < X && jj >= 0 && jj < Y && kk >= 0 && kk < Z)
        acc += (double)g * (double)xc[((int64_t)ii * Y + jj) * Z + kk];
      accb += (double)g;
    }
  }
  __shared__ double sa[kT], sb[kT];
  sa[threadIdx.x] = acc;
  sb[threadIdx.x] = accb;
  __syncthreads();
  for (int h = kT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sa[threadIdx.x] += sa[threadIdx.x + h];
      sb[threadIdx.x] += sb[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    dw[blockIdx.x] = (float)sa[0];
    if (c == 0 && tap == 0) db[o] = (float)sb[0];
  }
}

// 2x2x2 average pooling: (N, C, X, Y, Z) -> (N, C, X/2, Y/2, Z/2).
__global__ void pool_fwd_kernel(const float *x, float *y, int64_t NC, int X, int Y, int Z) {
  const int Xo = X / 2, Yo = Y / 2, Zo = Z / 2;
  const int64_t So = (int64_t)Xo * Yo * Zo, total = NC * So, S = (int64_t)X * Y * Z;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % Zo), j = (int)((t / Zo) % Yo), i = (int)((t / ((int64_t)Yo * Zo)) % Xo);
    const float *xc = x + (t / So) * S;
    float s = 0.0f;
    for (int d = 0; d < 8; ++d)
      s += xc[((int64_t)(2 * i + (d & 1)) * Y + (2 * j + ((d >> 1) & 1))) * Z + (2 * k + ((d >> 2) & 1))];
    y[t] = 0.125f * s;
  }
}

// Adjoint pair of pool / upsample on the fine grid (X, Y, Z):
//   mode 0 (upsample forward): out[fine] = in[coarse]
//   mode 1 (pool backward):    out[fine] (+)= in[coarse] / 8
__global__ void spread_kernel(const float *in, float *out, int64_t NC, int X, int Y, int Z, int mode,
                              int accumulate) {
  const int Xc = X / 2, Yc = Y / 2, Zc = Z / 2;
  const int64_t S = (int64_t)X * Y * Z, Sc = (int64_t)Xc * Yc * Zc, total = NC * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % Z), j = (int)((t / Z) % Y), i = (int)((t / ((int64_t)Y * Z)) % X);
    float v = in[(t / S) * Sc + ((int64_t)(i / 2) * Yc + j / 2) * Zc + k / 2];
    if (mode == 1) v *= 0.125f;
    out[t] = accumulate ? out[t] + v : v;
  }
}

// Upsample backward: out[coarse] = sum of the 8 fine children of in.
__global__ void gather8_kernel(const float *in, float *out, int64_t NC, int X, int Y, int Z) {
  const int Xc = X / 2, Yc = Y / 2, Zc = Z / 2;
  const int64_t Sc = (int64_t)Xc * Yc * Zc, total = NC * Sc, S = (int64_t)X * Y * Z;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % Zc), j = (int)((t / Zc) % Yc), i = (int)((t / ((int64_t)Yc * Zc)) % Xc);
    const float *ic = in + (t / Sc) * S;
    float s = 0.0f;
    for (int d = 0; d < 8; ++d)
      s += ic[((int64_t)(2 * i + (d & 1)) * Y + (2 * j + ((d >> 1) & 1))) * Z + (2 * k + ((d >> 2) & 1))];
    out[t] = s;
  }
}

// Copy of a channel range between two activation tensors of the same N and grid:
// dst[n, dc0 + c] (+)= src[n, sc0 + c] for c < nc.
__global__ void channels_copy_kernel(const float *src, int Cs, int sc0, float *dst, int Cd, int dc0, int nc, int N,
                                     int64_t S, int accumulate) {
  const int64_t total = (int64_t)N * nc * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t % S;
    const int c = (int)((t / S) % nc), n = (int)(t / ((int64_t)nc * S));
    const float v = src[((int64_t)n * Cs + sc0 + c) * S + p];
    float &d = dst[((int64_t)n * Cd + dc0 + c) * S + p];
    d = accumulate ? d + v : v;
  }
}

}  // namespace

cudaError_t unet_conv_fwd(const float *x, const float *w, const float *b, float *y, int N, int Ci, int Co, int X,
                          int Y, int Z, int K, bool relu, cudaStream_t s) {
  conv_fwd_kernel<<<grid_of((int64_t)N * Co * X * Y * Z), kT, 0, s>>>(x, w, b, y, N, Ci, Co, X, Y, Z, K, relu ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t unet_relu_bwd(const float *y, float *g, int64_t n, cudaStream_t s) {
  relu_bwd_kernel<<<grid_of(n), kT, 0, s>>>(y, g, n);
  return cudaGetLastError();
}
cudaError_t unet_conv_bwd(const float *x, const float *w, const float *dy, float *dx, bool dx_accumulate, float *dw,
                          float *db, int N, int Ci, int Co, int X, int Y, int Z, int K, cudaStream_t s) {
  if (dx) {
    conv_bwd_data_kernel<<<grid_of((int64_t)N * Ci * X * Y * Z), kT, 0, s>>>(dy, w, dx, N, Ci, Co, X, Y, Z, K,
                                                                             dx_accumulate ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  conv_bwd_weight_kernel<<<Co * Ci * K * K * K, kT, 0, s>>>(x, dy, dw, db, N, Ci, Co, X, Y, Z, K);
  return cudaGetLastError();
}
cudaError_t unet_pool_fwd(const float *x, float *y, int64_t NC, int X, int Y, int Z, cudaStream_t s) {
  pool_fwd_kernel<<<grid_of(NC * (X / 2) * (Y / 2) * (Z / 2)), kT, 0, s>>>(x, y, NC, X, Y, Z);
  return cudaGetLastError();
}
cudaError_t unet_spread(const float *in, float *out, int64_t NC, int X, int Y, int Z, bool pool_adjoint,
                        bool accumulate, cudaStream_t s) {
  spread_kernel<<<grid_of(NC * X * Y * Z), kT, 0, s>>>(in, out, NC, X, Y, Z, pool_adjoint ? 1 : 0, accumulate ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t unet_gather8(const float *in, float *out, int64_t NC, int X, int Y, int Z, cudaStream_t s) {
  gather8_kernel<<<grid_of(NC * (X / 2) * (Y / 2) * (Z / 2)), kT, 0, s>>>(in, out, NC, X, Y, Z);
  return cudaGetLastError();
}
cudaError_t unet_channels_copy(const float *src, int Cs, int sc0, float *dst, int Cd, int dc0, int nc, int N,
                               int64_t S, bool accumulate, cudaStream_t s) {
  channels_copy_kernel<<<grid_of((int64_t)N * nc * S), kT, 0, s>>>(src, Cs, sc0, dst, Cd, dc0, nc, N, S,
                                                                   accumulate ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace amr

// ---------------------------------------------------------------- the network
namespace amr {
namespace {

struct UnetPlan {
  int L = 0, N = 0, ci = 0, co = 0;
  int C[8] = {};
  int X[8] = {}, Y[8] = {}, Z[8] = {};
  int64_t S[8] = {};
  // parameter offsets: encoder level i (w1, b1, w2, b2), decoder level i (w1, b1, w2, b2), out (w, b)
  int64_t enc[8][4] = {}, dec[8][4] = {}, out_w = 0, out_b = 0, n_params = 0;
  // workspace offsets (floats): activations, then their gradients
  int64_t t1[8] = {}, s[8] = {}, pooled[8] = {}, up[8] = {}, cat[8] = {}, d1[8] = {}, d2[8] = {}, n_act = 0;
  std::string error;
};

bool make_plan(const tm_unet_desc *d, UnetPlan &p) {
  if (!d || d->levels < 1 || d->levels > 6 || d->c_in < 1 || d->c_out < 1 || d->n < 1) {
    p.error = "bad network description";
    return false;
  }
  p.L = d->levels;
  p.N = d->n;
  p.ci = d->c_in;
  p.co = d->c_out;
  const int div = 1 << (p.L - 1);
  if (d->x < 1 || d->y < 1 || d->z < 1 || d->x % div || d->y % div || d->z % div) {
    p.error = "grid sizes must be positive multiples of 2^(levels - 1)";
    return false;
  }
  for (int i = 0; i < p.L; ++i) {
    p.C[i] = d->channels[i];
    if (p.C[i] < 1) {
      p.error = "channels must be positive";
      return false;
    }
    p.X[i] = d->x >> i;
    p.Y[i] = d->y >> i;
    p.Z[i] = d->z >> i;
    p.S[i] = (int64_t)p.X[i] * p.Y[i] * p.Z[i];
  }
  int64_t o = 0;
  int prev = p.ci;
  for (int i = 0; i < p.L; ++i) {
    const int c = p.C[i];
    p.enc[i][0] = o; o += (int64_t)c * prev * 27;
    p.enc[i][1] = o; o += c;
    p.enc[i][2] = o; o += (int64_t)c * c * 27;
    p.enc[i][3] = o; o += c;
    prev = c;
  }
  for (int i = p.L - 2; i >= 0; --i) {
    const int c = p.C[i];
    p.dec[i][0] = o; o += (int64_t)c * (prev + c) * 27;
    p.dec[i][1] = o; o += c;
    p.dec[i][2] = o; o += (int64_t)c * c * 27;
    p.dec[i][3] = o; o += c;
    prev = c;
  }
  p.out_w = o; o += (int64_t)p.co * prev;
  p.out_b = o; o += p.co;
  p.n_params = o;
  int64_t a = 0;
  for (int i = 0; i < p.L; ++i) {
    p.t1[i] = a; a += (int64_t)p.N * p.C[i] * p.S[i];
    p.s[i] = a; a += (int64_t)p.N * p.C[i] * p.S[i];
    if (i < p.L - 1) {
      p.pooled[i] = a; a += (int64_t)p.N * p.C[i] * p.S[i + 1];
      p.up[i] = a; a += (int64_t)p.N * p.C[i + 1] * p.S[i];
      p.cat[i] = a; a += (int64_t)p.N * (p.C[i + 1] + p.C[i]) * p.S[i];
      p.d1[i] = a; a += (int64_t)p.N * p.C[i] * p.S[i];
      p.d2[i] = a; a += (int64_t)p.N * p.C[i] * p.S[i];
    }
  }
  p.n_act = a;
  return true;
}

int unet_fail(tm_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define UNET_CUDA(ctx, ...)                                                                  \
  do {                                                                                       \
    cudaError_t _e = (__VA_ARGS__);                                                          \
    if (_e != cudaSuccess) return unet_fail(ctx, TM_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// output features of decoder level i (or of the bottleneck when i == L - 1)
int64_t level_out(const UnetPlan &p, int i) { return i == p.L - 1 ? p.s[i] : p.d2[i]; }

}  // namespace
}  // namespace amr

extern "C" {

int64_t tm_unet_param_count(const tm_unet_desc *d) {
  amr::UnetPlan p;
  return amr::make_plan(d, p) ? p.n_params : -1;
}

int64_t tm_unet_workspace_floats(const tm_unet_desc *d) {
  amr::UnetPlan p;
  return amr::make_plan(d, p) ? 2 * p.n_act : -1;
}

int tm_unet_forward(tm_ctx *ctx, const tm_unet_desc *d, const float *params, const float *x, float *y, float *ws) try {
  using namespace amr;
  if (!ctx) return TM_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return unet_fail(ctx, TM_ECUDA, "cudaSetDevice");
  UnetPlan p;
  if (!make_plan(d, p)) return unet_fail(ctx, TM_EINVAL, p.error);
  if (!params || !x || !y || !ws) return unet_fail(ctx, TM_EINVAL, "null pointer");
  cudaStream_t s = ctx->stream;
  const float *in = x;
  int cin = p.ci;
  for (int i = 0; i < p.L; ++i) {
    UNET_CUDA(ctx, unet_conv_fwd(in, params + p.enc[i][0], params + p.enc[i][1], ws + p.t1[i], p.N, cin, p.C[i],
                                 p.X[i], p.Y[i], p.Z[i], 3, true, s));
    UNET_CUDA(ctx, unet_conv_fwd(ws + p.t1[i], params + p.enc[i][2], params + p.enc[i][3], ws + p.s[i], p.N, p.C[i],
                                 p.C[i], p.X[i], p.Y[i], p.Z[i], 3, true, s));
    if (i < p.L - 1) {
      UNET_CUDA(ctx, unet_pool_fwd(ws + p.s[i], ws + p.pooled[i], (int64_t)p.N * p.C[i], p.X[i], p.Y[i], p.Z[i], s));
      in = ws + p.pooled[i];
      cin = p.C[i];
    }
  }
  for (int i = p.L - 2; i >= 0; --i) {
    const int cu = p.C[i + 1], cs = p.C[i], cc = cu + cs;
    // upsampled features of the level below, then the skip features, in one tensor
    float *up = ws + p.up[i];
    UNET_CUDA(ctx, unet_spread(ws + level_out(p, i + 1), up, (int64_t)p.N * cu, p.X[i], p.Y[i], p.Z[i], false, false,
                               s));
    UNET_CUDA(ctx, unet_channels_copy(up, cu, 0, ws + p.cat[i], cc, 0, cu, p.N, p.S[i], false, s));
    UNET_CUDA(ctx, unet_channels_copy(ws + p.s[i], cs, 0, ws + p.cat[i], cc, cu, cs, p.N, p.S[i], false, s));
    UNET_CUDA(ctx, unet_conv_fwd(ws + p.cat[i], params + p.dec[i][0], params + p.dec[i][1], ws + p.d1[i], p.N, cc, cs,
                                 p.X[i], p.Y[i], p.Z[i], 3, true, s));
    UNET_CUDA(ctx, unet_conv_fwd(ws + p.d1[i], params + p.dec[i][2], params + p.dec[i][3], ws + p.d2[i], p.N, cs, cs,
                                 p.X[i], p.Y[i], p.Z[i], 3, true, s));
  }
  UNET_CUDA(ctx, unet_conv_fwd(ws + level_out(p, 0), params + p.out_w, params + p.out_b, y, p.N, p.C[0], p.co, p.X[0],
                               p.Y[0], p.Z[0], 1, false, s));
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_unet_backward(tm_ctx *ctx, const tm_unet_desc *d, const float *params, const float *x, const float *dy,
                     float *dparams, float *dx, float *ws) try {
  using namespace amr;
  if (!ctx) return TM_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return unet_fail(ctx, TM_ECUDA, "cudaSetDevice");
  UnetPlan p;
  if (!make_plan(d, p)) return unet_fail(ctx, TM_EINVAL, p.error);
  if (!params || !x || !dy || !dparams || !ws) return unet_fail(ctx, TM_EINVAL, "null pointer");
  cudaStream_t s = ctx->stream;
  float *g = ws + p.n_act;     // gradients, same layout as the activations
  const int N = p.N;
  // output 1x1x1 convolution: gradient into the top decoder output
  UNET_CUDA(ctx, unet_conv_bwd(ws + level_out(p, 0), params + p.out_w, dy, g + level_out(p, 0), false,
                               dparams + p.out_w, dparams + p.out_b, N, p.C[0], p.co, p.X[0], p.Y[0], p.Z[0], 1, s));
  for (int i = 0; i <= p.L - 2; ++i) {
    const int cu = p.C[i + 1], cs = p.C[i], cc = cu + cs;
    const int64_t nd = (int64_t)N * cs * p.S[i];
    UNET_CUDA(ctx, unet_relu_bwd(ws + p.d2[i], g + p.d2[i], nd, s));
    UNET_CUDA(ctx, unet_conv_bwd(ws + p.d1[i], params + p.dec[i][2], g + p.d2[i], g + p.d1[i], false,
                                 dparams + p.dec[i][2], dparams + p.dec[i][3], N, cs, cs, p.X[i], p.Y[i], p.Z[i], 3, s));
    UNET_CUDA(ctx, unet_relu_bwd(ws + p.d1[i], g + p.d1[i], nd, s));
    UNET_CUDA(ctx, unet_conv_bwd(ws + p.cat[i], params + p.dec[i][0], g + p.d1[i], g + p.cat[i], false,
                                 dparams + p.dec[i][0], dparams + p.dec[i][1], N, cc, cs, p.X[i], p.Y[i], p.Z[i], 3, s));
    // skip part of the concatenation -> gradient of the encoder output s[i] (the pooling part comes later)
    UNET_CUDA(ctx, unet_channels_copy(g + p.cat[i], cc, cu, g + p.s[i], cs, 0, cs, N, p.S[i], false, s));
    // upsampled part -> gradient of the level below's output (sum over the 8 fine children)
    float *gup = g + p.up[i];
    UNET_CUDA(ctx, unet_channels_copy(g + p.cat[i], cc, 0, gup, cu, 0, cu, N, p.S[i], false, s));
    UNET_CUDA(ctx, unet_gather8(gup, g + level_out(p, i + 1), (int64_t)N * cu, p.X[i], p.Y[i], p.Z[i], s));
  }
  for (int i = p.L - 1; i >= 0; --i) {
    const int c = p.C[i], cin = i == 0 ? p.ci : p.C[i - 1];
    const int64_t na = (int64_t)N * c * p.S[i];
    UNET_CUDA(ctx, unet_relu_bwd(ws + p.s[i], g + p.s[i], na, s));
    UNET_CUDA(ctx, unet_conv_bwd(ws + p.t1[i], params + p.enc[i][2], g + p.s[i], g + p.t1[i], false,
                                 dparams + p.enc[i][2], dparams + p.enc[i][3], N, c, c, p.X[i], p.Y[i], p.Z[i], 3, s));
    UNET_CUDA(ctx, unet_relu_bwd(ws + p.t1[i], g + p.t1[i], na, s));
    const float *in = i == 0 ? x : ws + p.pooled[i - 1];
    float *gin = i == 0 ? dx : g + p.pooled[i - 1];
    UNET_CUDA(ctx, unet_conv_bwd(in, params + p.enc[i][0], g + p.t1[i], gin, false, dparams + p.enc[i][0],
                                 dparams + p.enc[i][1], N, cin, c, p.X[i], p.Y[i], p.Z[i], 3, s));
    if (i > 0)   // average pooling: each fine value receives 1/8 of its coarse gradient
      UNET_CUDA(ctx, unet_spread(g + p.pooled[i - 1], g + p.s[i - 1], (int64_t)N * p.C[i - 1], p.X[i - 1], p.Y[i - 1],
                                 p.Z[i - 1], true, true, s));
  }
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

}  // extern "C"
