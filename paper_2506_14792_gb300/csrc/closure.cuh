// Learned closure: a 3x3 periodic CNN (channels 1 -> 32 -> 32 -> 32 -> 1, tanh after the first
// three layers) whose output is added to the explicit term F on the dealiased grid, so its
// weights are parameters of F (their gradient follows from the adjoint sweep, eq. 6).
//
// Arithmetic: BF16 operands (activations, weights, back-propagated signals), FP32
// accumulation and biases, tanh in FP32; the network's input (the vorticity grid) and its
// output (the correction, and the input gradient) are FP64 at the boundary with the solver.
// Layouts: grid [y][x] (the solver's row order), activations [pixel][channel] (channels
// contiguous), weights [layer][o][a][b][c] with a the x offset and b the y offset, matching the
// reference convolution y[o](x, y) = b[o] + sum W[o, c, a, b] x[c](x + a - 1, y + b - 1).
// Parameter order of the flat FP64 vector: per layer W[o][c][a][b] then b[o].
#pragma once
#include <cuda_bf16.h>

namespace spadj {
namespace cnn {

constexpr int kLayers = 4;
constexpr int kCh[kLayers + 1] = {1, 32, 32, 32, 1};
constexpr int kHid = 32;

__host__ __device__ inline int w_off(int l) {  // offset of layer l's weights in the flat vector
  int o = 0;
  const int ch[5] = {1, 32, 32, 32, 1};
  for (int k = 0; k < l; ++k) o += ch[k + 1] * ch[k] * 9 + ch[k + 1];
  return o;
}
__host__ __device__ inline int n_params() { return w_off(kLayers); }

// flat FP64 params -> BF16 weights [l][o][a][b][c] (same offsets as the flat vector) + FP32 biases
__global__ void convert_kernel(const double* __restrict__ p, __nv_bfloat16* __restrict__ wq, float* __restrict__ bq) {
  const int total = n_params();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int l = 0;
    while (l + 1 < kLayers && i >= w_off(l + 1)) ++l;
    const int ci = (l == 0) ? 1 : kHid, co = (l == kLayers - 1) ? 1 : kHid;
    const int r = i - w_off(l);
    if (r < co * ci * 9) {
      const int o = r / (ci * 9), c = (r / 9) % ci, a = (r % 9) / 3, b = r % 3;
      wq[w_off(l) + ((o * 3 + a) * 3 + b) * ci + c] = __float2bfloat16_rn((float)p[i]);
      bq[i] = 0.0f;
    } else {
      bq[i] = (float)p[i];  // bias stored at its flat offset
      wq[i] = __float2bfloat16_rn(0.0f);
    }
  }
}

// FP64 grid -> BF16 activation of the input layer (one channel)
__global__ void quantize_kernel(const double* __restrict__ g, __nv_bfloat16* __restrict__ x, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = __float2bfloat16_rn((float)g[i]);
}

// forward of layer l for `nb` members of an M x M grid (member stride M*M pixels):
// z = conv(in) + b; hidden layers store h = bf16(tanh z) and dact = 1 - tanh^2 (if non-null);
// the last layer writes the FP64 output.
__global__ void fwd_kernel(int l, int M, int nb, const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ wq,
                           const float* __restrict__ bq, __nv_bfloat16* __restrict__ h, float* __restrict__ dact,
                           double* __restrict__ out) {
  const int ci = (l == 0) ? 1 : kHid, co = (l == kLayers - 1) ? 1 : kHid;
  const long long P = (long long)M * M;
  const long long total = P * nb * co;
  const __nv_bfloat16* W = wq + w_off(l);
  const float* B = bq + w_off(l) + co * ci * 9;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(t % co);
    const long long pix = t / co;
    const long long mb = pix / P;
    const int pp = (int)(pix % P);
    const int y = pp / M, x = pp % M;
    float acc = B[o];
    for (int a = 0; a < 3; ++a) {
      const int xs = (x + a - 1 + M) % M;
      for (int b = 0; b < 3; ++b) {
        const int ys = (y + b - 1 + M) % M;
        const __nv_bfloat16* src = in + (mb * P + (long long)ys * M + xs) * ci;
        const __nv_bfloat16* w = W + ((o * 3 + a) * 3 + b) * ci;
        for (int c = 0; c < ci; ++c) acc = fmaf(__bfloat162float(w[c]), __bfloat162float(src[c]), acc);
      }
    }
    if (l < kLayers - 1) {
      const float th = tanhf(acc);
      h[pix * co + o] = __float2bfloat16_rn(th);
      if (dact) dact[pix * co + o] = 1.0f - th * th;
    } else {
      out[pix] = (double)acc;
    }
  }
}

// dz = bf16(dh * dact) (hidden layers) or bf16(g) (last layer; g FP64 grid)
__global__ void dz_kernel(long long n, const float* __restrict__ dh, const float* __restrict__ dact,
                          const double* __restrict__ g, __nv_bfloat16* __restrict__ dz) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dz[i] = __float2bfloat16_rn(g ? (float)g[i] : dh[i] * dact[i]);
}

// input gradient of layer l: din[c](x', y') = sum_{o,a,b} W[o,c,a,b] dz[o](x' - a + 1, y' - b + 1)
// (FP32 into din, or FP64 into dout for the first layer)
__global__ void dgrad_kernel(int l, int M, int nb, const __nv_bfloat16* __restrict__ dz, const __nv_bfloat16* __restrict__ wq,
                             float* __restrict__ din, double* __restrict__ dout) {
  const int ci = (l == 0) ? 1 : kHid, co = (l == kLayers - 1) ? 1 : kHid;
  const long long P = (long long)M * M;
  const long long total = P * nb * ci;
  const __nv_bfloat16* W = wq + w_off(l);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t % ci);
    const long long pix = t / ci;
    const long long mb = pix / P;
    const int pp = (int)(pix % P);
    const int y = pp / M, x = pp % M;
    float acc = 0.0f;
    for (int a = 0; a < 3; ++a) {
      const int xs = (x - a + 1 + M) % M;
      for (int b = 0; b < 3; ++b) {
        const int ys = (y - b + 1 + M) % M;
        const __nv_bfloat16* src = dz + (mb * P + (long long)ys * M + xs) * co;
        for (int o = 0; o < co; ++o)
          acc = fmaf(__bfloat162float(W[((o * 3 + a) * 3 + b) * ci + c]), __bfloat162float(src[o]), acc);
      }
    }
    if (dout) dout[pix] = (double)acc;
    else din[pix * ci + c] = acc;
  }
}

// weight gradient of layer l for each member: part[mb][w_off(l) + r] (flat FP64-vector order),
// dW[o,c,a,b] = sum_pixels in[c](x + a - 1, y + b - 1) dz[o](x, y), db[o] = sum dz[o].
// One CTA per (member, o, a, b) plus one per (member, o) for the bias; fixed reduction order.
__global__ void wgrad_kernel(int l, int M, const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ dz,
                             float* __restrict__ part, int npar) {
  const int ci = (l == 0) ? 1 : kHid, co = (l == kLayers - 1) ? 1 : kHid;
  const long long P = (long long)M * M;
  const int mb = blockIdx.y;
  const int item = blockIdx.x;  // 0 .. co*9 - 1: weights; co*9 .. co*10 - 1: biases
  __shared__ float red[256];
  float* dst = part + (long long)mb * npar + w_off(l);
  if (item < co * 9) {
    const int o = item / 9, a = (item % 9) / 3, b = item % 3;
    // thread t owns channel c = t % ci and a strided share of the pixels
    const int c = threadIdx.x % ci, lane = threadIdx.x / ci, nl = blockDim.x / ci;
    float acc = 0.0f;
    for (long long pp = lane; pp < P; pp += nl) {
      const int y = (int)(pp / M), x = (int)(pp % M);
      const int xs = (x + a - 1 + M) % M, ys = (y + b - 1 + M) % M;
      const float iv = __bfloat162float(in[((long long)mb * P + (long long)ys * M + xs) * ci + c]);
      const float dv = __bfloat162float(dz[((long long)mb * P + pp) * co + o]);
      acc = fmaf(iv, dv, acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < ci) {
      float s = 0.0f;
      for (int k = 0; k < nl; ++k) s += red[k * ci + threadIdx.x];
      dst[((o * ci + threadIdx.x) * 3 + a) * 3 + b] = s;
    }
  } else {
    const int o = item - co * 9;
    float acc = 0.0f;
    for (long long pp = threadIdx.x; pp < P; pp += blockDim.x) acc += __bfloat162float(dz[((long long)mb * P + pp) * co + o]);
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.0f;
      for (int k = 0; k < (int)blockDim.x; ++k) s += red[k];
      dst[co * ci * 9 + o] = s;
    }
  }
}

// grad_p += sum over members of the per-member partials (fixed order, FP64 accumulation)
__global__ void reduce_params_kernel(const float* __restrict__ part, int nb, int npar, double* __restrict__ gp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npar; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += (double)part[(long long)b * npar + i];
    gp[i] += s;
  }
}

}  // namespace cnn
}  // namespace spadj
