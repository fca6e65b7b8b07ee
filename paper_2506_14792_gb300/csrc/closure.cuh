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

#include "pdl.cuh"

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

// acc + sum_c x[c] w[c] over 32 BF16 channels (both 16-byte aligned; either may be in global or
// shared memory, so the loads are generic), FP32 products and sums in channel order
__device__ __forceinline__ float dot32_bf16(const __nv_bfloat16* x, const __nv_bfloat16* w, float acc) {
  const uint4* xv = reinterpret_cast<const uint4*>(x);
  const uint4* wv = reinterpret_cast<const uint4*>(w);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint4 a = xv[j], b = wv[j];
    const unsigned au[4] = {a.x, a.y, a.z, a.w}, bu[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 af = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&au[k]));
      const float2 bf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&bu[k]));
      acc = fmaf(bf.x, af.x, acc);
      acc = fmaf(bf.y, af.y, acc);
    }
  }
  return acc;
}

// two BF16 values as one 32-bit word (lo in the low half)
__device__ __forceinline__ unsigned pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// periodic neighbour index of a coordinate in [-1, M]
__device__ __forceinline__ int wrap1(int v, int M) { return v < 0 ? v + M : (v >= M ? v - M : v); }

// Thin layers (l = 0: 1 -> 32, l = 3: 32 -> 1).  Thread = (pixel q of a member, channel k) with
// the 32-wide channel fastest, so the 32-channel tensor is read and written coalesced; grid =
// (pixel-channel tiles of 256, member); 32-bit index arithmetic (a member has M^2 < 2^31 pixels).
template <int C>
__device__ __forceinline__ bool thin_index(int M, int& y, int& x, int& k) {
  const int tq = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = C == 1 ? tq : (tq >> 5);
  k = C == 1 ? 0 : (tq & 31);
  if (q >= M * M) return false;
  y = q / M;
  x = q - y * M;
  return true;
}

// forward of a thin layer: z = conv(in) + b; layer 0 stores h = bf16(tanh z) and
// dact = 1 - tanh^2 (if non-null); layer 3 writes the FP64 output.
template <int CI, int CO>
__global__ void __launch_bounds__(256) fwd_kernel(int l, int M, const __nv_bfloat16* __restrict__ in,
                                                  const __nv_bfloat16* __restrict__ wq, const float* __restrict__ bq,
                                                  __nv_bfloat16* __restrict__ h, float* __restrict__ dact,
                                                  double* __restrict__ out) {
  int y, x, o;
  if (!thin_index<CO>(M, y, x, o)) return;
  const long long base = (long long)blockIdx.y * M * M;
  const long long pix = base + (long long)y * M + x;
  const __nv_bfloat16* W = wq + w_off(l);
  float acc = bq[w_off(l) + CO * CI * 9 + o];
  for (int a = 0; a < 3; ++a) {
    const int xs = wrap1(x + a - 1, M);
    for (int b = 0; b < 3; ++b) {
      const int ys = wrap1(y + b - 1, M);
      const __nv_bfloat16* src = in + (base + (long long)ys * M + xs) * CI;
      const __nv_bfloat16* w = W + ((o * 3 + a) * 3 + b) * CI;
      if (CI == kHid) acc = dot32_bf16(src, w, acc);
      else acc = fmaf(__bfloat162float(w[0]), __bfloat162float(src[0]), acc);
    }
  }
  if (CO == kHid) {
    const float th = tanhf(acc);
    h[pix * CO + o] = __float2bfloat16_rn(th);
    if (dact) dact[pix * CO + o] = 1.0f - th * th;
  } else {
    out[pix] = (double)acc;
  }
}

// dz = bf16(dh * dact) (hidden layers) or bf16(g) (last layer; g FP64 grid)
__global__ void dz_kernel(long long n, const float* __restrict__ dh, const float* __restrict__ dact,
                          const double* __restrict__ g, __nv_bfloat16* __restrict__ dz) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dz[i] = __float2bfloat16_rn(g ? (float)g[i] : dh[i] * dact[i]);
}

// input gradient of a thin layer: din[c](x', y') = sum_{o,a,b} W[o,c,a,b] dz[o](x' - a + 1, y' - b + 1)
// (FP32 into din for layer 3, FP64 into dout for layer 0)
template <int CI, int CO>
__global__ void __launch_bounds__(256) dgrad_kernel(int l, int M, const __nv_bfloat16* __restrict__ dz,
                                                    const __nv_bfloat16* __restrict__ wq, float* __restrict__ din,
                                                    double* __restrict__ dout) {
  const __nv_bfloat16* W = wq + w_off(l);
  // for CI = 1 the weights of a tap, W[o][0][a][b] over o, as a contiguous 32-vector
  __shared__ __align__(16) __nv_bfloat16 wt[9 * kHid];
  if (CI == 1) {
    for (int i = threadIdx.x; i < 9 * CO; i += blockDim.x) wt[i] = W[(i % CO) * 9 + i / CO];
    __syncthreads();
  }
  int y, x, c;
  if (!thin_index<CI>(M, y, x, c)) return;
  const long long base = (long long)blockIdx.y * M * M;
  const long long pix = base + (long long)y * M + x;
  float acc = 0.0f;
  for (int a = 0; a < 3; ++a) {
    const int xs = wrap1(x - a + 1, M);
    for (int b = 0; b < 3; ++b) {
      const int ys = wrap1(y - b + 1, M);
      const __nv_bfloat16* src = dz + (base + (long long)ys * M + xs) * CO;
      if (CI == 1 && CO == kHid) {
        acc = dot32_bf16(src, wt + (a * 3 + b) * kHid, acc);
      } else {
        for (int o = 0; o < CO; ++o)
          acc = fmaf(__bfloat162float(W[((o * 3 + a) * 3 + b) * CI + c]), __bfloat162float(src[o]), acc);
      }
    }
  }
  if (CI == 1) dout[pix] = (double)acc;
  else din[pix * CI + c] = acc;
}

// Layer 0 forward with one thread per pixel (all 32 output channels): the pixel's nine inputs are
// read once and the 288 weights come from shared memory; the same sums in the same order as
// fwd_kernel<1, 32> (bias, then the taps a-major), written as four 16-byte BF16 stores of h and
// eight of dact.  Grid = (pixel tiles of 128, member).
__global__ void __launch_bounds__(128) fwd0_kernel(int M, const __nv_bfloat16* __restrict__ in,
                                                   const __nv_bfloat16* __restrict__ wq, const float* __restrict__ bq,
                                                   __nv_bfloat16* __restrict__ h, float* __restrict__ dact) {
  __shared__ float ws[9][kHid];
  __shared__ float bs[kHid];
  for (int i = threadIdx.x; i < 9 * kHid; i += blockDim.x) {
    const int o = i / 9, t = i - o * 9;  // W[o][0][a][b] at o * 9 + a * 3 + b
    ws[t][o] = __bfloat162float(wq[w_off(0) + i]);
  }
  if (threadIdx.x < kHid) bs[threadIdx.x] = bq[w_off(0) + kHid * 9 + threadIdx.x];
  __syncthreads();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= M * M) return;
  const int y = q / M, x = q - y * M;
  const long long base = (long long)blockIdx.y * M * M;
  const long long pix = base + q;
  float v[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      v[a * 3 + b] = __bfloat162float(in[base + (long long)wrap1(y + b - 1, M) * M + wrap1(x + a - 1, M)]);
#pragma unroll
  for (int o0 = 0; o0 < kHid; o0 += 8) {
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = bs[o0 + e];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] = fmaf(ws[t][o0 + e], v[t], acc[e]);
    float th[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) th[e] = tanhf(acc[e]);
    uint4 hv;
    hv.x = pack2(__float2bfloat16_rn(th[0]), __float2bfloat16_rn(th[1]));
    hv.y = pack2(__float2bfloat16_rn(th[2]), __float2bfloat16_rn(th[3]));
    hv.z = pack2(__float2bfloat16_rn(th[4]), __float2bfloat16_rn(th[5]));
    hv.w = pack2(__float2bfloat16_rn(th[6]), __float2bfloat16_rn(th[7]));
    *reinterpret_cast<uint4*>(h + pix * kHid + o0) = hv;
    if (dact) {
      *reinterpret_cast<float4*>(dact + pix * kHid + o0) =
          make_float4(1.0f - th[0] * th[0], 1.0f - th[1] * th[1], 1.0f - th[2] * th[2], 1.0f - th[3] * th[3]);
      *reinterpret_cast<float4*>(dact + pix * kHid + o0 + 4) =
          make_float4(1.0f - th[4] * th[4], 1.0f - th[5] * th[5], 1.0f - th[6] * th[6], 1.0f - th[7] * th[7]);
    }
  }
}

// Layer 3 input gradient with one thread per pixel (all 32 input channels): din[c] = sum over taps
// of W[0][c][a][b] dz(x - a + 1, y - b + 1), the nine dz values read once, the same sums in the
// same order as dgrad_kernel<32, 1>, written as eight 16-byte stores.
__global__ void __launch_bounds__(128) dgrad3_kernel(int M, const __nv_bfloat16* __restrict__ dz,
                                                     const __nv_bfloat16* __restrict__ wq, float* __restrict__ din,
                                                     const float* __restrict__ dact, __nv_bfloat16* __restrict__ dzo) {
  __shared__ float ws[9][kHid];
  for (int i = threadIdx.x; i < 9 * kHid; i += blockDim.x) {
    const int t = i / kHid, c = i - t * kHid;  // W[0][a][b][c] at (a * 3 + b) * 32 + c
    ws[t][c] = __bfloat162float(wq[w_off(kLayers - 1) + i]);
  }
  __syncthreads();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= M * M) return;
  const int y = q / M, x = q - y * M;
  const long long base = (long long)blockIdx.y * M * M;
  float v[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      v[a * 3 + b] = __bfloat162float(dz[base + (long long)wrap1(y - b + 1, M) * M + wrap1(x - a + 1, M)]);
  const long long o = (base + q) * kHid;
#pragma unroll
  for (int c0 = 0; c0 < kHid; c0 += 4) {
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] = fmaf(ws[t][c0 + e], v[t], acc[e]);
    if (dzo) {  // the previous layer's BF16 cotangent bf16(din * dact), the separate dz pass fused in
      const float4 d = *reinterpret_cast<const float4*>(dact + o + c0);
      uint2 zv;
      zv.x = pack2(__float2bfloat16_rn(acc[0] * d.x), __float2bfloat16_rn(acc[1] * d.y));
      zv.y = pack2(__float2bfloat16_rn(acc[2] * d.z), __float2bfloat16_rn(acc[3] * d.w));
      *reinterpret_cast<uint2*>(dzo + o + c0) = zv;
    } else {
      *reinterpret_cast<float4*>(din + o + c0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
    }
  }
}

// weight gradient of a thin layer for each member: dW[o,c,a,b] = sum_pixels in[c](x + a - 1, y + b - 1)
// dz[o](x, y), db[o] = sum dz[o], in kThinSplits row bands per member whose partials
// (scratch[member][band][r], r the flat FP64-vector index within the layer) wgrad_finish_kernel sums
// in order.  CTA = (x offset a with its three taps b, or the bias; member; band); thread t = (pixel
// lane t / 32, wide channel w = t % 32), the wide channel being o for layer 0 and c for layer 3, so
// the reads of the 32-channel tensor are coalesced and one dz load serves the three taps; a pixel
// lane takes the pixels x = lane (mod lanes) of the band's rows, and the lanes' partial sums are
// reduced in shared memory in a fixed order.
constexpr int kThinSplits = 4;
constexpr int kThinOut = 9 * kHid + kHid;  // 320 partial slots per (member, band)
template <int CI, int CO>
__global__ void __launch_bounds__(256) wgrad_kernel(int l, int M, const __nv_bfloat16* __restrict__ in,
                                                    const __nv_bfloat16* __restrict__ dz,
                                                    float* __restrict__ scratch) {
  const int mb = blockIdx.y, item = blockIdx.x, band = blockIdx.z;  // item 0..2: x offset a, 3: bias
  const int w = threadIdx.x & 31, lane = threadIdx.x >> 5, nl = blockDim.x >> 5;
  const int y0 = band * M / kThinSplits, y1 = (band + 1) * M / kThinSplits;
  __shared__ float red[3][256];
  float* dst = scratch + ((long long)mb * kThinSplits + band) * kThinOut;
  const __nv_bfloat16* inm = in + (long long)mb * M * M * CI;
  const __nv_bfloat16* dzm = dz + (long long)mb * M * M * CO;
  float acc[3] = {0.0f, 0.0f, 0.0f};  // taps (a, b = 0, 1, 2)
  if (item < 3) {
    const int a = item;
    for (int y = y0; y < y1; ++y) {
      const __nv_bfloat16* irow[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) irow[b] = inm + (long long)wrap1(y + b - 1, M) * M * CI;
      const __nv_bfloat16* drow = dzm + (long long)y * M * CO;
#pragma unroll 4
      for (int x = lane; x < M; x += nl) {
        const int xs = wrap1(x + a - 1, M);
        const float dv = __bfloat162float(CO == 1 ? drow[x] : drow[x * CO + w]);
#pragma unroll
        for (int b = 0; b < 3; ++b)
          acc[b] = fmaf(__bfloat162float(CI == 1 ? irow[b][xs] : irow[b][xs * CI + w]), dv, acc[b]);
      }
    }
  } else if (CO > 1) {  // bias of layer 0: db[o = w]
    for (int q = y0 * M + lane; q < y1 * M; q += nl) acc[0] += __bfloat162float(dzm[(long long)q * CO + w]);
  } else {  // bias of layer 3: every thread takes a strided share of the band's pixels
    for (int q = y0 * M + threadIdx.x; q < y1 * M; q += blockDim.x) acc[0] += __bfloat162float(dzm[q]);
  }
#pragma unroll
  for (int b = 0; b < 3; ++b) red[b][threadIdx.x] = acc[b];
  __syncthreads();
  if (item == 3 && CO == 1) {
    if (threadIdx.x == 0) {
      float s = 0.0f;
      for (int k = 0; k < (int)blockDim.x; ++k) s += red[0][k];
      dst[CO * CI * 9] = s;
    }
    return;
  }
  if (threadIdx.x < 32) {
    if (item == 3) {
      float s = 0.0f;
      for (int k = 0; k < nl; ++k) s += red[0][k * 32 + w];
      dst[CO * CI * 9 + w] = s;
    } else {
      const int o = (CO == 1) ? 0 : w, c = (CI == 1) ? 0 : w;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        float s = 0.0f;
        for (int k = 0; k < nl; ++k) s += red[b][k * 32 + w];
        dst[((o * CI + c) * 3 + item) * 3 + b] = s;
      }
    }
  }
}

// The same weight and bias gradients with all nine taps in one CTA per (band, member): thread =
// (pixel lane = t / 16, channel pair p = t % 16: wide channels 2p, 2p + 1, read as one BF16 pair).
// A lane walks a contiguous segment of each row of the band with the 3 x 3 input window in
// registers (three new input loads and one dz load per pixel, against four loads per tap triple
// in wgrad_kernel, whose three x offsets are separate CTAs), accumulating the 9 x 2 tap sums and
// the bias sums; the lanes' partials are then summed in shared memory in lane order into the same
// scratch slots as wgrad_kernel (weight r = k * 9 + a * 3 + b, k the wide channel; then the
// biases).  The narrow side (one channel) is loaded as a scalar by every thread of a pixel.
template <int CI, int CO>
__global__ void __launch_bounds__(256) wgrad_win_kernel(int M, const __nv_bfloat16* __restrict__ in,
                                                        const __nv_bfloat16* __restrict__ dz,
                                                        float* __restrict__ scratch) {
  static_assert((CI == 1) != (CO == 1) && CI * CO == kHid, "a thin layer: one side 1, the other 32 wide");
  constexpr bool kWideIn = CI > 1;
  const int band = blockIdx.x, mb = blockIdx.y;
  const int cp = threadIdx.x & 15, lane = threadIdx.x >> 4;
  const int y0 = band * M / kThinSplits, y1 = (band + 1) * M / kThinSplits;
  const int S = (M + 15) >> 4, x0 = lane * S, x1 = min(M, x0 + S);
  const __nv_bfloat16* inm = in + (long long)mb * M * M * CI;
  const __nv_bfloat16* dzm = dz + (long long)mb * M * M * CO;
  // value pair at pixel q of a tensor: the thread's two wide channels, or the narrow value twice
  auto ld = [&](const __nv_bfloat16* t, bool wide, int q) -> float2 {
    if (wide) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(t + (long long)q * kHid + 2 * cp));
    const float v = __bfloat162float(t[q]);
    return make_float2(v, v);
  };
  float acc[9][2], bacc[2] = {0.0f, 0.0f};
#pragma unroll
  for (int t = 0; t < 9; ++t) acc[t][0] = acc[t][1] = 0.0f;
  if (x0 < x1) {
    for (int y = y0; y < y1; ++y) {
      const int yr[3] = {wrap1(y - 1, M) * M, y * M, wrap1(y + 1, M) * M};
      float2 w[3][3];  // w[b][j]: input at row y + b - 1, column x + j - 1
      const int xl = wrap1(x0 - 1, M);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        w[b][0] = ld(inm, kWideIn, yr[b] + xl);
        w[b][1] = ld(inm, kWideIn, yr[b] + x0);
      }
      for (int x = x0; x < x1; ++x) {
        const int xn = wrap1(x + 1, M);
#pragma unroll
        for (int b = 0; b < 3; ++b) w[b][2] = ld(inm, kWideIn, yr[b] + xn);
        const float2 d = ld(dzm, !kWideIn, yr[1] + x);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            acc[a * 3 + b][0] = fmaf(w[b][a].x, d.x, acc[a * 3 + b][0]);
            acc[a * 3 + b][1] = fmaf(w[b][a].y, d.y, acc[a * 3 + b][1]);
          }
        bacc[0] += d.x;
        bacc[1] += d.y;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          w[b][0] = w[b][1];
          w[b][1] = w[b][2];
        }
      }
    }
  }
  __shared__ float red[16][16][20];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    red[lane][cp][2 * t] = acc[t][0];
    red[lane][cp][2 * t + 1] = acc[t][1];
  }
  red[lane][cp][18] = bacc[0];
  red[lane][cp][19] = bacc[1];
  __syncthreads();
  float* dst = scratch + ((long long)mb * kThinSplits + band) * kThinOut;
  const int nout = 9 * kHid + CO;  // CO biases (a narrow output has one, summed once: channel 0)
  for (int r = threadIdx.x; r < nout; r += blockDim.x) {
    int p, e;
    if (r < 9 * kHid) {
      const int k = r / 9, t = r - k * 9;
      p = k >> 1;
      e = 2 * t + (k & 1);
    } else {
      const int k = r - 9 * kHid;
      p = k >> 1;
      e = 18 + (k & 1);
    }
    float sum = 0.0f;
    for (int q = 0; q < 16; ++q) sum += red[q][p][e];
    dst[r] = sum;
  }
}

// The thin layers' single-channel FP64 outputs with the 32-channel side read in windows: the
// 32 -> 1 forward (kAdj = false: out = b + sum_{a,b,c} W[0][a][b][c] in[c](x + a - 1, y + b - 1))
// and the 1 -> 32 input gradient (kAdj = true: out = sum_{o,a,b} W[o][0][a][b] dz[o](x - a + 1,
// y - b + 1)).  CTA = (row band, member); thread = (pixel lane, channel pair) as in
// wgrad_win_kernel: a lane walks a contiguous segment of each row with the 3 x 3 window of its two
// channels in registers (three new loads per pixel) and its 18 weights in registers; the partial
// sums of a pixel's 16 channel pairs are added by a butterfly over the half-warp.  Every thread of
// a warp takes the same number of steps (a lane past the row's end works on a wrapped pixel and
// stores nothing), so the shuffles are convergent.
constexpr int kThinBands = 8;
template <bool kAdj>
__global__ void __launch_bounds__(256) thin_out_win_kernel(int M, const __nv_bfloat16* __restrict__ t32,
                                                           const __nv_bfloat16* __restrict__ wq,
                                                           const float* __restrict__ bq, double* __restrict__ out) {
  const int band = blockIdx.x, mb = blockIdx.y;
  const int cp = threadIdx.x & 15, lane = threadIdx.x >> 4;
  const int y0 = band * M / kThinBands, y1 = (band + 1) * M / kThinBands;
  const int S = (M + 15) >> 4, x0 = lane * S, xa = x0 % M;
  const int l = kAdj ? 0 : kLayers - 1;
  const __nv_bfloat16* W = wq + w_off(l);
  float wr[9][2];
#pragma unroll
  for (int t = 0; t < 9; ++t)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k = 2 * cp + e;  // W[0][a][b][k] (forward) or W[k][0][a][b] (input gradient), t = 3 a + b
      wr[t][e] = __bfloat162float(kAdj ? W[k * 9 + t] : W[t * kHid + k]);
    }
  const float bias = kAdj ? 0.0f : bq[w_off(l) + 9 * kHid];
  const __nv_bfloat16* tm = t32 + (long long)mb * M * M * kHid + 2 * cp;
  double* om = out + (long long)mb * M * M;
  auto ld = [&](int q) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(tm + (long long)q * kHid));
  };
  for (int y = y0; y < y1; ++y) {
    const int yr[3] = {wrap1(y - 1, M) * M, y * M, wrap1(y + 1, M) * M};
    float2 w[3][3];  // w[r][j]: row y + r - 1, column xc + j - 1
    int xc = xa;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      w[r][0] = ld(yr[r] + wrap1(xc - 1, M));
      w[r][1] = ld(yr[r] + xc);
    }
    for (int s = 0; s < S; ++s) {
      const int xn = wrap1(xc + 1, M);
#pragma unroll
      for (int r = 0; r < 3; ++r) w[r][2] = ld(yr[r] + xn);
      float acc = 0.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const float2 v = kAdj ? w[2 - b][2 - a] : w[b][a];
          acc = fmaf(wr[a * 3 + b][0], v.x, acc);
          acc = fmaf(wr[a * 3 + b][1], v.y, acc);
        }
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      const int x = x0 + s;
      if (cp == 0 && x < M) om[yr[1] + x] = (double)(bias + acc);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        w[r][0] = w[r][1];
        w[r][1] = w[r][2];
      }
      xc = xn;
    }
  }
}

// part[mb][w_off(l) + r] = sum over the bands of scratch[mb][band][r], in band order
__global__ void wgrad_finish_kernel(int l, const float* __restrict__ scratch, float* __restrict__ part, int npar) {
  const int mb = blockIdx.x, nr = kThinOut - (l == 0 ? 0 : kHid - 1);  // 9 * 32 weights + 32 or 1 biases
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    float s = 0.0f;
    for (int band = 0; band < kThinSplits; ++band) s += scratch[((long long)mb * kThinSplits + band) * kThinOut + r];
    part[(long long)mb * npar + w_off(l) + r] = s;
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

namespace spadj {
namespace cnn {

// ---- tensor-core kernels for the 32 -> 32 layers (BF16 mma.sync m16n8k16, FP32 accumulate) ----
//
// Implicit GEMM per member: rows = pixels, columns = 32 output channels, reduction = 9 taps x 32
// input channels (18 k-steps of 16).  A CTA of 4 warps owns 64 consecutive pixels; warp w owns
// pixels 16w..16w+15 and all four 8-column tiles.  The forward pass (dir = +1) gathers
// in[pixel shifted by (a - 1, b - 1)] with weights W[o][a][b][c]; the input gradient (dir = -1)
// gathers dz[pixel shifted by (1 - a, 1 - b)] with the transposed weights W[c][a][b][o].
// Fragment layout of m16n8k16 (bf16): A rows g = lane/4 (+8), k pairs 2(lane%4) (+8);
// B k pairs 2(lane%4) (+8), column g; C rows g (+8), column pairs 2(lane%4).

__device__ __forceinline__ void mma_bf16(float* c, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 16-byte asynchronous copy global -> shared, zero-filled (nothing read) when valid is false
__device__ __forceinline__ void cp_async16_zfill(void* smem_dst, const void* gmem_src, bool valid) {
  const unsigned s = smem_addr(smem_dst);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem_src), "r"(n) : "memory");
}

// out[p][n] = sum_{a,b,c} Wt[n][a][b][c] * in[shift(p, a, b)][c]  (+ bias, tanh for dir = +1)
// mode 0: forward hidden layer (writes h, dact); mode 1: input gradient (writes din FP32)
__global__ void __launch_bounds__(128) conv32_mma_kernel(int l, int M, int nb, int mode,
                                                         const __nv_bfloat16* __restrict__ in,
                                                         const __nv_bfloat16* __restrict__ wq,
                                                         const float* __restrict__ bq,
                                                         __nv_bfloat16* __restrict__ h, float* __restrict__ dact,
                                                         float* __restrict__ din) {
  __shared__ __nv_bfloat16 sw[32 * 9 * 32];  // weights as [n][tap][k] (k = reduction channel)
  const __nv_bfloat16* W = wq + w_off(l);
  // forward: Wt[n=o][tap][k=c] = W[o][a][b][c]; gradient: Wt[n=c][tap][k=o] = W[o][a][b][c]
  for (int i = threadIdx.x; i < 32 * 9 * 32; i += blockDim.x) {
    const int n = i / (9 * 32), tap = (i / 32) % 9, k = i % 32;
    sw[i] = mode == 0 ? W[(n * 9 + tap) * 32 + k] : W[(k * 9 + tap) * 32 + n];
  }
  __syncthreads();
  const long long P = (long long)M * M;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int g = lane / 4, t4 = lane % 4;
  const long long tiles = (P * nb + 63) / 64;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long p0 = tile * 64 + warp * 16;
    // the two pixel rows of this lane's A fragment
    long long pr[2];
    int ys[2], xs[2];
    long long mbr[2];
    bool ok[2];
    for (int r = 0; r < 2; ++r) {
      pr[r] = p0 + g + 8 * r;
      ok[r] = pr[r] < P * nb;
      const long long pc = ok[r] ? pr[r] : 0;
      mbr[r] = pc / P;
      const int pp = (int)(pc % P);
      ys[r] = pp / M;
      xs[r] = pp % M;
    }
    float acc[4][4];
    for (int nt = 0; nt < 4; ++nt)
      for (int q = 0; q < 4; ++q) acc[nt][q] = 0.0f;
    for (int tap = 0; tap < 9; ++tap) {
      const int a = tap / 3, b = tap % 3;
      const int dx = mode == 0 ? a - 1 : 1 - a, dy = mode == 0 ? b - 1 : 1 - b;
      const __nv_bfloat16* src[2];
      for (int r = 0; r < 2; ++r) {
        const int xx = (xs[r] + dx + M) % M, yy = (ys[r] + dy + M) % M;
        src[r] = in + (mbr[r] * P + (long long)yy * M + xx) * 32;
      }
      for (int kh = 0; kh < 2; ++kh) {  // 16-channel halves of the 32 input channels
        const int k0 = kh * 16 + 2 * t4;
        unsigned af[4];
        const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
        af[0] = ok[0] ? pack2(src[0][k0], src[0][k0 + 1]) : pack2(z, z);
        af[1] = ok[1] ? pack2(src[1][k0], src[1][k0 + 1]) : pack2(z, z);
        af[2] = ok[0] ? pack2(src[0][k0 + 8], src[0][k0 + 9]) : pack2(z, z);
        af[3] = ok[1] ? pack2(src[1][k0 + 8], src[1][k0 + 9]) : pack2(z, z);
        for (int nt = 0; nt < 4; ++nt) {
          const __nv_bfloat16* wr = sw + ((nt * 8 + g) * 9 + tap) * 32;
          unsigned bf[2] = {pack2(wr[k0], wr[k0 + 1]), pack2(wr[k0 + 8], wr[k0 + 9])};
          mma_bf16(acc[nt], af, bf);
        }
      }
    }
    const float* B = bq + w_off(l) + 32 * 32 * 9;
    for (int nt = 0; nt < 4; ++nt)
      for (int q = 0; q < 4; ++q) {
        const int r = q / 2;
        if (!ok[r]) continue;
        const int n = nt * 8 + 2 * t4 + (q % 2);
        const long long idx = pr[r] * 32 + n;
        if (mode == 0) {
          const float th = tanhf(acc[nt][q] + B[n]);
          h[idx] = __float2bfloat16_rn(th);
          if (dact) dact[idx] = 1.0f - th * th;
        } else {
          din[idx] = acc[nt][q];
        }
      }
  }
}

// weight gradient of a 32 -> 32 layer: dW[o][c][a][b] = sum_p dz[p][o] in[shift(p, a, b)][c].
// GEMM per tap: rows o (32 = 2 m-tiles), columns c (32 = 4 n-tiles), reduction over pixels.
// CTA = (member, tap, pixel chunk); its 4 warps split the chunk; partial sums reduced in smem and
// written to part[member][chunk]... summed over chunks in a fixed order by wgrad32_finish.
__global__ void __launch_bounds__(128) wgrad32_mma_kernel(int l, int M, const __nv_bfloat16* __restrict__ in,
                                                          const __nv_bfloat16* __restrict__ dz,
                                                          float* __restrict__ chunkbuf, int nchunk) {
  const int P = M * M;  // pixels of a member (< 2^31): 32-bit index arithmetic
  const int tap = blockIdx.y, mb = blockIdx.z, chunk = blockIdx.x;
  const int a = tap / 3, b = tap % 3;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int g = lane / 4, t4 = lane % 4;
  const int per = (P + nchunk - 1) / nchunk;
  const int pbeg = chunk * per, pend = min(P, pbeg + per);
  const __nv_bfloat16* inm = in + (long long)mb * P * 32;
  const __nv_bfloat16* dzm = dz + (long long)mb * P * 32;
  float acc[2][4][4];
  for (int mt = 0; mt < 2; ++mt)
    for (int nt = 0; nt < 4; ++nt)
      for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
  // k-steps of 16 pixels, interleaved over the 4 warps
  for (int k0 = pbeg + warp * 16; k0 < pend; k0 += 64) {
    // pixels of this lane's k pairs: k0 + 2 t4 + {0, 1} and + 8
    const int pk[4] = {k0 + 2 * t4, k0 + 2 * t4 + 1, k0 + 2 * t4 + 8, k0 + 2 * t4 + 9};
    const __nv_bfloat16* sh[4];
    const __nv_bfloat16* dzr[4];
    bool okk[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      okk[i] = pk[i] < pend;
      const int pc = okk[i] ? pk[i] : pbeg;
      const int y = pc / M, x = pc - y * M;
      sh[i] = inm + ((long long)wrap1(y + b - 1, M) * M + wrap1(x + a - 1, M)) * 32;
      dzr[i] = dzm + (long long)pc * 32;
    }
    for (int mt = 0; mt < 2; ++mt) {
      // A[o][p] = dz[p][o]: rows o = 16 mt + g (+8), k pairs = pixels
      const int o0 = mt * 16 + g, o1 = o0 + 8;
      unsigned af[4];
      af[0] = pack2(okk[0] ? dzr[0][o0] : z, okk[1] ? dzr[1][o0] : z);
      af[1] = pack2(okk[0] ? dzr[0][o1] : z, okk[1] ? dzr[1][o1] : z);
      af[2] = pack2(okk[2] ? dzr[2][o0] : z, okk[3] ? dzr[3][o0] : z);
      af[3] = pack2(okk[2] ? dzr[2][o1] : z, okk[3] ? dzr[3][o1] : z);
      for (int nt = 0; nt < 4; ++nt) {
        // B[p][c] = in[shift(p)][c]: column c = 8 nt + g, k pairs = pixels
        const int c = nt * 8 + g;
        unsigned bf[2] = {pack2(okk[0] ? sh[0][c] : z, okk[1] ? sh[1][c] : z),
                          pack2(okk[2] ? sh[2][c] : z, okk[3] ? sh[3][c] : z)};
        mma_bf16(acc[mt][nt], af, bf);
      }
    }
  }
  // reduce the 4 warps in smem (fixed order) and write the chunk's 32 x 32 block
  __shared__ float red[4][32 * 32];
  for (int mt = 0; mt < 2; ++mt)
    for (int nt = 0; nt < 4; ++nt)
      for (int q = 0; q < 4; ++q) {
        const int o = mt * 16 + g + 8 * (q / 2), c = nt * 8 + 2 * t4 + (q % 2);
        red[warp][o * 32 + c] = acc[mt][nt][q];
      }
  __syncthreads();
  float* dst = chunkbuf + (((long long)mb * 9 + tap) * nchunk + chunk) * 1024;
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) dst[i] = ((red[0][i] + red[1][i]) + red[2][i]) + red[3][i];
}

// sum the chunks of wgrad32_mma_kernel / wgrad32_halo_kernel in order into part[mb][w_off(l) + flat W
// index]; with bpart (the halo kernel's partial bias sums [mb][chunk][32]) the bias gradient too
__global__ void wgrad32_finish_kernel(int l, const float* __restrict__ chunkbuf, int nchunk, float* __restrict__ part,
                                      int npar, const float* __restrict__ bpart) {
  const int mb = blockIdx.y;
  if (bpart && blockIdx.x == 0 && threadIdx.x < 32) {
    float s = 0.0f;
    for (int k = 0; k < nchunk; ++k) s += bpart[((long long)mb * nchunk + k) * 32 + threadIdx.x];
    part[(long long)mb * npar + w_off(l) + 32 * 32 * 9 + threadIdx.x] = s;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 9 * 1024; i += gridDim.x * blockDim.x) {
    const int tap = i / 1024, oc = i % 1024, o = oc / 32, c = oc % 32;
    const float* src = chunkbuf + (((long long)mb * 9 + tap) * nchunk) * 1024 + oc;
    float s = 0.0f;
    for (int k = 0; k < nchunk; ++k) s += src[(long long)k * 1024];
    part[(long long)mb * npar + w_off(l) + (o * 32 + c) * 9 + tap] = s;
  }
}

// bias gradient of a 32-channel layer (the weights are handled by the tensor-core kernels)
__global__ void bgrad32_kernel(int l, int M, const __nv_bfloat16* __restrict__ dz, float* __restrict__ part, int npar) {
  const long long P = (long long)M * M;
  const int mb = blockIdx.y, o = blockIdx.x;
  __shared__ float red[256];
  float acc = 0.0f;
  for (long long p = threadIdx.x; p < P; p += blockDim.x) acc += __bfloat162float(dz[((long long)mb * P + p) * 32 + o]);
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int k = 0; k < (int)blockDim.x; ++k) s += red[k];
    part[(long long)mb * npar + w_off(l) + 32 * 32 * 9 + o] = s;
  }
}

}  // namespace cnn
}  // namespace spadj

namespace spadj {
namespace cnn {

// ---- fifth-generation tensor cores (tcgen05) for the 32 -> 32 layers ----------------------------
//
// Implicit GEMM D[p][n] = sum_k A[p][k] B[n][k] with rows p = 128 consecutive pixels (one tile),
// columns n = 32 output channels and reduction k = tap * 32 + channel (9 taps x 32 channels = 288),
// BF16 operands and an FP32 accumulator in tensor memory:
//  * A (the gathered, shifted activations: forward in[shift(p, a - 1, b - 1)][c], input gradient
//    dz[shift(p, 1 - a, 1 - b)][o]) and B (the weights, W[o][a][b][c] or its transpose) are staged in
//    shared memory in the canonical K-major layout without swizzle: 8 x 16-byte core matrices, the
//    core matrix of rows 8 r .. 8 r + 7 and k = 8 g .. 8 g + 7 at byte (r * 36 + g) * 128, row i of it
//    at + 16 i (leading-byte offset 128 between the two k core matrices of an MMA, stride-byte offset
//    36 * 128 between 8-row groups);
//  * one thread issues the 18 MMAs (M = 128, N = 32, K = 16) of a tile and commits them to an
//    mbarrier; every thread waits on it (bounded), reads its pixel's 32 accumulators from its lane of
//    tensor memory (tcgen05.ld 32x32b) and applies the epilogue.
// The CTA keeps its 32 tensor-memory columns (allocated by warp 0) for all tiles and frees them at
// exit.  A wait that runs out sets *err, waits once more (bounded) and ends the CTA's work.
constexpr int kTcRows = 128;        // pixels per tile (MMA M)
constexpr int kTcK = 288;           // reduction length
constexpr int kTcKg = kTcK / 8;     // k core-matrix groups
constexpr unsigned kTcSpin = 1u << 22;
constexpr size_t kTcSmem = (size_t)(kTcRows + 32) * kTcK * 2;  // A tile + B

__device__ __forceinline__ unsigned long long tc_smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  // start address, leading- and stride-byte offsets in 16-byte units; version 1 (tcgen05); no swizzle
  return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D F32, A and B BF16, both K-major, N = 32, M = 128
constexpr unsigned kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ unsigned tc_core_off(int row, int k) {  // byte offset of element (row, k)
  return (unsigned)(((row >> 3) * kTcKg + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ bool tc_wait(unsigned long long* bar, unsigned parity, int* err) {
  for (unsigned it = 0; it < kTcSpin; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    __nanosleep(32);
  }
  if (err) atomicExch(err, 1);
  return false;
}

// mode 0: forward hidden layer, out = tanh(D + b) as BF16 h and 1 - tanh^2 as FP32 dact (nullable);
// mode 1: input gradient, din = D (FP32); mode 2: pre-activation zout = D + b (FP32, for tests);
// mode 3: input gradient times the previous layer's activation derivative, written as that
// layer's BF16 cotangent h = bf16(D * dact) (dact read): the separate dz pass fused into the epilogue.
__global__ void __launch_bounds__(128) conv32_tc_kernel(int l, int M, int nb, int mode,
                                                        const __nv_bfloat16* __restrict__ in,
                                                        const __nv_bfloat16* __restrict__ wq,
                                                        const float* __restrict__ bq, __nv_bfloat16* __restrict__ h,
                                                        float* __restrict__ dact, float* __restrict__ fout,
                                                        int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char tcs[];
  __shared__ unsigned long long bar;
  __shared__ unsigned tmem_holder;
  unsigned char* sA = tcs;                              // 128 x 288 BF16, canonical K-major
  unsigned char* sB = tcs + (size_t)kTcRows * kTcK * 2; // 32 x 288 BF16, canonical K-major
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long P = (long long)M * M, npix = P * nb;
  const long long tiles = (npix + kTcRows - 1) / kTcRows;
  const __nv_bfloat16* W = wq + w_off(l);
  // B[n][k = tap * 32 + kc]: forward W[o = n][tap][c = kc]; gradient W[o = kc][tap][c = n]
  for (int i = tid; i < 32 * kTcK; i += blockDim.x) {
    const int n = i / kTcK, k = i - n * kTcK, tap = k >> 5, kc = k & 31;
    const __nv_bfloat16 v = (mode & 1) ? W[(kc * 9 + tap) * 32 + n] : W[(n * 9 + tap) * 32 + kc];
    *reinterpret_cast<__nv_bfloat16*>(sB + tc_core_off(n, k)) = v;
  }
  if (tid == 0) mbar_init(&bar, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_addr(&tmem_holder))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_holder;
  const float* Bias = bq + w_off(l) + 32 * 32 * 9;
  const unsigned aaddr = smem_addr(sA), baddr = smem_addr(sB);
  unsigned parity = 0;
  bool alive = true;
  // A gather of a tile: thread t owns row t (pixel p), 36 asynchronous 16-byte copies (8 channels
  // each) into the canonical layout; rows past the last pixel are zero-filled
  auto gather = [&](long long tile) {
    const long long p = tile * kTcRows + tid;
    const bool ok = p < npix;
    const long long pc = ok ? p : 0;
    const long long mb = pc / P;
    const int pp = (int)(pc - mb * P), y = pp / M, x = pp - y * M;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int a = tap / 3, b = tap % 3;
      const int dx = (mode & 1) ? 1 - a : a - 1, dy = (mode & 1) ? 1 - b : b - 1;
      const int xx = wrap1(x + dx, M), yy = wrap1(y + dy, M);
      const __nv_bfloat16* src = in + (mb * P + (long long)yy * M + xx) * 32;
#pragma unroll
      for (int j = 0; j < 4; ++j) cp_async16_zfill(sA + tc_core_off(tid, tap * 32 + 8 * j), src + 8 * j, ok);
    }
    cp_async_commit();
  };
  long long tile = blockIdx.x;
  if (tile < tiles) gather(tile);
  for (; tile < tiles && alive; tile += gridDim.x) {
    cp_async_wait_all();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // A complete, and every thread has read the previous tile's accumulator
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int kk = 0; kk < kTcK / 16; ++kk) {
        const unsigned long long ad = tc_smem_desc(aaddr + kk * 256, 128, kTcKg * 128);
        const unsigned long long bd = tc_smem_desc(baddr + kk * 256, 128, kTcKg * 128);
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(kk > 0 ? 1 : 0)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(&bar))
                   : "memory");
    }
    if (!tc_wait(&bar, parity, err)) {
      tc_wait(&bar, parity, nullptr);  // the tile's MMAs may still be running: wait once more
      alive = false;
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(tmem + ((unsigned)(warp * 32) << 16))
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    // the MMAs have consumed A: the next tile's gather runs under this tile's epilogue
    if (alive && tile + gridDim.x < tiles) gather(tile + gridDim.x);
    const long long p = tile * kTcRows + tid;
    if (p < npix && alive) {
      if (mode == 0) {
#pragma unroll
        for (int n = 0; n < 32; n += 8) {
          float t[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) t[e] = tanhf(__uint_as_float(r[n + e]) + Bias[n + e]);
          uint4 hv;
          hv.x = pack2(__float2bfloat16_rn(t[0]), __float2bfloat16_rn(t[1]));
          hv.y = pack2(__float2bfloat16_rn(t[2]), __float2bfloat16_rn(t[3]));
          hv.z = pack2(__float2bfloat16_rn(t[4]), __float2bfloat16_rn(t[5]));
          hv.w = pack2(__float2bfloat16_rn(t[6]), __float2bfloat16_rn(t[7]));
          *reinterpret_cast<uint4*>(h + p * 32 + n) = hv;
          if (dact) {
            *reinterpret_cast<float4*>(dact + p * 32 + n) =
                make_float4(1.0f - t[0] * t[0], 1.0f - t[1] * t[1], 1.0f - t[2] * t[2], 1.0f - t[3] * t[3]);
            *reinterpret_cast<float4*>(dact + p * 32 + n + 4) =
                make_float4(1.0f - t[4] * t[4], 1.0f - t[5] * t[5], 1.0f - t[6] * t[6], 1.0f - t[7] * t[7]);
          }
        }
      } else if (mode == 3) {  // the next layer's BF16 cotangent dz = din * dact, dact read from `dact`
#pragma unroll
        for (int n = 0; n < 32; n += 8) {
          const float4 d0 = *reinterpret_cast<const float4*>(dact + p * 32 + n);
          const float4 d1 = *reinterpret_cast<const float4*>(dact + p * 32 + n + 4);
          uint4 zv;
          zv.x = pack2(__float2bfloat16_rn(__uint_as_float(r[n]) * d0.x), __float2bfloat16_rn(__uint_as_float(r[n + 1]) * d0.y));
          zv.y = pack2(__float2bfloat16_rn(__uint_as_float(r[n + 2]) * d0.z), __float2bfloat16_rn(__uint_as_float(r[n + 3]) * d0.w));
          zv.z = pack2(__float2bfloat16_rn(__uint_as_float(r[n + 4]) * d1.x), __float2bfloat16_rn(__uint_as_float(r[n + 5]) * d1.y));
          zv.w = pack2(__float2bfloat16_rn(__uint_as_float(r[n + 6]) * d1.z), __float2bfloat16_rn(__uint_as_float(r[n + 7]) * d1.w));
          *reinterpret_cast<uint4*>(h + p * 32 + n) = zv;
        }
      } else {
        const float bs = mode == 2 ? 1.0f : 0.0f;
#pragma unroll
        for (int n = 0; n < 32; n += 4)
          *reinterpret_cast<float4*>(fout + p * 32 + n) =
              make_float4(__uint_as_float(r[n]) + bs * Bias[n], __uint_as_float(r[n + 1]) + bs * Bias[n + 1],
                          __uint_as_float(r[n + 2]) + bs * Bias[n + 2], __uint_as_float(r[n + 3]) + bs * Bias[n + 3]);
      }
    }
  }
  cp_async_wait_all();  // no copy outstanding at exit (a run cut short by a timeout)
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// The same convolutions with the operand staged once per tile instead of once per tap.  The
// member's grid is addressed through a staged index s = ys * W + xs with W = M + 2 (xs = 0 holds
// column M - 1, xs = 1..M columns 0..M-1, xs = M + 1 column 0: the periodic halo), so that every
// tap is a uniform shift of s: (b - 1) W + (a - 1) in the forward (mode 0/2), its negative for the
// input gradient (mode 1).  A tile is 128 consecutive staged indices of one member (rows at a halo
// column or past the member are computed and discarded); its operand is the staged range
// [s0 - W - 1, s0 + 128 + W + 1) of R = 2 W + 130 pixels, copied once by cp.async into
//   [chunk g = c / 8][staged pixel i] x 16 bytes,
// which is the canonical K-major layout without swizzle with rows 16 bytes apart (stride-byte
// offset 128 between 8-row groups) and the chunks R * 16 bytes apart (leading-byte offset): the
// MMA of tap t and channel half h reads A from chunk 2h at the tap's shifted first row, so the
// nine taps need no copies of their own.  The staged range of the next tile is copied into the
// other of two buffers while the current tile's MMAs and epilogue run.  Each input pixel is read
// about R / 128 = 2.5 times instead of nine.
__host__ __device__ constexpr int halo_range(int M) { return 2 * (M + 2) + 130; }
__host__ __device__ constexpr size_t halo_smem(int M) {
  return (size_t)2 * 4 * halo_range(M) * 16 + (size_t)32 * kTcK * 2;
}

// One thread's entries of a staged halo range: i = i0, i0 + step, ... < R, entry i holding the
// pixel at staged index r0 + i (row ys = floor(s / W) taken modulo M, column xs - 1 with the halo
// columns xs = 0 and M + 1 wrapped).  One floor division at the start; then the column advances by
// step and carries into the row, so the loop needs no division.  f(i, pixel) per entry.
template <class F>
__device__ __forceinline__ void halo_walk(int r0, int i, int step, int R, int W, int M, F&& f) {
  const int r = r0 + i;
  const int ys = r >= 0 ? r / W : -((W - 1 - r) / W);  // floor division (r >= -W - 1)
  int xs = r - ys * W;                                 // 0 .. W - 1
  int ym = ((ys % M) + M) % M;  // rows past the member (read only by discarded outputs) wrap too
  for (; i < R; i += step) {
    int x = xs - 1;
    x = x < 0 ? x + M : (x >= M ? x - M : x);
    f(i, ym * M + x);
    xs += step;
    while (xs >= W) {
      xs -= W;
      if (++ym == M) ym = 0;
    }
  }
}

__global__ void __launch_bounds__(128) conv32_halo_kernel(int l, int M, int nb, int mode,
                                                          const __nv_bfloat16* __restrict__ in,
                                                          const __nv_bfloat16* __restrict__ wq,
                                                          const float* __restrict__ bq, __nv_bfloat16* __restrict__ h,
                                                          float* __restrict__ dact, float* __restrict__ fout,
                                                          int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char hs[];
  __shared__ unsigned long long bar;
  __shared__ unsigned tmem_holder;
  const int W = M + 2, R = halo_range(M);
  const size_t abytes = (size_t)4 * R * 16;
  unsigned char* sA[2] = {hs, hs + abytes};
  unsigned char* sB = hs + 2 * abytes;
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long P = (long long)M * M;
  const int tpm = (M * W + kTcRows - 1) / kTcRows;  // tiles per member
  const long long tiles = (long long)tpm * nb;
  const __nv_bfloat16* Wt = wq + w_off(l);
  for (int i = tid; i < 32 * kTcK; i += blockDim.x) {
    const int n = i / kTcK, k = i - n * kTcK, tap = k >> 5, kc = k & 31;
    const __nv_bfloat16 v = (mode & 1) ? Wt[(kc * 9 + tap) * 32 + n] : Wt[(n * 9 + tap) * 32 + kc];
    *reinterpret_cast<__nv_bfloat16*>(sB + tc_core_off(n, k)) = v;
  }
  if (tid == 0) mbar_init(&bar, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_addr(&tmem_holder))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_holder;
  const float* Bias = bq + w_off(l) + 32 * 32 * 9;
  const unsigned baddr = smem_addr(sB);
  // staged range of a tile into buffer buf: entry (g, i) <- channels 8g..8g+7 of the pixel at
  // staged index s0 - W - 1 + i (rows wrap periodically)
  auto stage = [&](long long tile, int buf) {
    const long long mb = tile / tpm;
    const int s0 = (int)(tile - mb * tpm) * kTcRows;
    const __nv_bfloat16* src = in + mb * P * 32 + (tid & 3) * 8;
    unsigned char* dst = sA[buf] + (size_t)(tid & 3) * R * 16;
    // entry (g, i) for idx = 4 i + g = tid, tid + 128, ...: g = tid & 3 fixed, i steps by 32
    halo_walk(s0 - W - 1, tid >> 2, blockDim.x >> 2, R, W, M, [&](int i, int pix) {
      cp_async16_zfill(dst + (size_t)i * 16, src + (long long)pix * 32, true);
    });
    cp_async_commit();
  };
  unsigned parity = 0;
  bool alive = true;
  long long tile = blockIdx.x;
  int buf = 0;
  if (tile < tiles) stage(tile, 0);
  for (; tile < tiles && alive; tile += gridDim.x, buf ^= 1) {
    // the next tile's range into the other buffer (its last reader, the MMAs of the previous
    // tile, completed before that tile's epilogue); then wait for this tile's range only
    if (tile + gridDim.x < tiles) stage(tile + gridDim.x, buf ^ 1);
    else cp_async_commit();
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the range complete, and every thread has read the previous accumulator
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned aaddr = smem_addr(sA[buf]);
#pragma unroll 1
      for (int kk = 0; kk < kTcK / 16; ++kk) {
        const int tap = kk >> 1, half = kk & 1, a = tap / 3, b = tap % 3;
        const int sh = (b - 1) * W + (a - 1);
        const int i0 = W + 1 + ((mode & 1) ? -sh : sh);
        const unsigned long long ad = tc_smem_desc(aaddr + (unsigned)((2 * half * R + i0) * 16), (unsigned)R * 16, 128);
        const unsigned long long bd = tc_smem_desc(baddr + kk * 256, 128, kTcKg * 128);
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(kk > 0 ? 1 : 0)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(&bar))
                   : "memory");
    }
    if (!tc_wait(&bar, parity, err)) {
      tc_wait(&bar, parity, nullptr);  // the tile's MMAs may still be running: wait once more
      alive = false;
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(tmem + ((unsigned)(warp * 32) << 16))
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    // this thread's output row: staged index s0 + tid, a pixel unless at a halo column or past the member
    const long long mb = tile / tpm;
    const int so = (int)(tile - mb * tpm) * kTcRows + tid;
    const int ys = so / W, xs = so - ys * W;
    if (alive && ys < M && xs >= 1 && xs <= M) {
      const long long p = mb * P + (long long)ys * M + (xs - 1);
      if (mode == 0) {
#pragma unroll
        for (int n = 0; n < 32; n += 8) {
          float t[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) t[e] = tanhf(__uint_as_float(r[n + e]) + Bias[n + e]);
          uint4 hv;
          hv.x = pack2(__float2bfloat16_rn(t[0]), __float2bfloat16_rn(t[1]));
          hv.y = pack2(__float2bfloat16_rn(t[2]), __float2bfloat16_rn(t[3]));
          hv.z = pack2(__float2bfloat16_rn(t[4]), __float2bfloat16_rn(t[5]));
          hv.w = pack2(__float2bfloat16_rn(t[6]), __float2bfloat16_rn(t[7]));
          *reinterpret_cast<uint4*>(h + p * 32 + n) = hv;
          if (dact) {
            *reinterpret_cast<float4*>(dact + p * 32 + n) =
                make_float4(1.0f - t[0] * t[0], 1.0f - t[1] * t[1], 1.0f - t[2] * t[2], 1.0f - t[3] * t[3]);
            *reinterpret_cast<float4*>(dact + p * 32 + n + 4) =
                make_float4(1.0f - t[4] * t[4], 1.0f - t[5] * t[5], 1.0f - t[6] * t[6], 1.0f - t[7] * t[7]);
          }
        }
      } else if (mode == 3) {  // the next layer's BF16 cotangent dz = din * dact, dact read from `dact`
#pragma unroll
        for (int n = 0; n < 32; n += 8) {
          const float4 d0 = *reinterpret_cast<const float4*>(dact + p * 32 + n);
          const float4 d1 = *reinterpret_cast<const float4*>(dact + p * 32 + n + 4);
          uint4 zv;
          zv.x = pack2(__float2bfloat16_rn(__uint_as_float(r[n]) * d0.x), __float2bfloat16_rn(__uint_as_float(r[n + 1]) * d0.y));
          zv.y = pack2(__float2bfloat16_rn(__uint_as_float(r[n + 2]) * d0.z), __float2bfloat16_rn(__uint_as_float(r[n + 3]) * d0.w));
          zv.z = pack2(__float2bfloat16_rn(__uint_as_float(r[n + 4]) * d1.x), __float2bfloat16_rn(__uint_as_float(r[n + 5]) * d1.y));
          zv.w = pack2(__float2bfloat16_rn(__uint_as_float(r[n + 6]) * d1.z), __float2bfloat16_rn(__uint_as_float(r[n + 7]) * d1.w));
          *reinterpret_cast<uint4*>(h + p * 32 + n) = zv;
        }
      } else {
        const float bs = mode == 2 ? 1.0f : 0.0f;
#pragma unroll
        for (int n = 0; n < 32; n += 4)
          *reinterpret_cast<float4*>(fout + p * 32 + n) =
              make_float4(__uint_as_float(r[n]) + bs * Bias[n], __uint_as_float(r[n + 1]) + bs * Bias[n + 1],
                          __uint_as_float(r[n + 2]) + bs * Bias[n + 2], __uint_as_float(r[n + 3]) + bs * Bias[n + 3]);
      }
    }
  }
  cp_async_wait_all();  // no copy outstanding at exit
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// Weight gradient of a 32 -> 32 layer from halo-staged operands: dW[o][c][tap] =
// sum_p dz[p][o] in[p + shift(tap)][c] as warp-level BF16 MMAs (m16n8k16, FP32 accumulation) whose
// fragments are read from shared memory by ldmatrix.trans.  A tile is 128 consecutive staged
// indices of one member (the staged index space of conv32_halo_kernel); its dz rows (zero at the
// halo columns and past the member, so they add nothing) and the halo range of the input are
// copied once by cp.async as [8-channel chunk][pixel] x 16 bytes, double-buffered.  Warp t owns
// tap t: per 16 pixels it loads the A fragments (o x pixel) from the dz chunks and the B fragments
// (pixel x c) from the input chunks at the tap's shifted rows, and keeps its 32 x 32 accumulators
// in registers over the CTA's tiles.  CTA = (pixel chunk of the member's tiles, member); each warp
// writes its tap's partial block to chunkbuf[member][tap][chunk], summed by wgrad32_finish_kernel.
__device__ __forceinline__ void ldsm_x4_t(unsigned* r, const void* row_addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(row_addr)));
}
__host__ __device__ constexpr size_t wgrad_halo_smem(int M) {
  return (size_t)2 * 4 * (halo_range(M) + kTcRows) * 16;
}

__global__ void __launch_bounds__(288, 3) wgrad32_halo_kernel(int M, const __nv_bfloat16* __restrict__ in,
                                                           const __nv_bfloat16* __restrict__ dz,
                                                           float* __restrict__ chunkbuf, int nchunk,
                                                           float* __restrict__ bpart) {
  extern __shared__ __align__(128) unsigned char ws[];
  const int W = M + 2, R = halo_range(M);
  const size_t buf_bytes = (size_t)4 * (R + kTcRows) * 16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int chunk = blockIdx.x, mb = blockIdx.y;
  const long long P = (long long)M * M;
  const int tpm = (M * W + kTcRows - 1) / kTcRows;
  const int t0 = chunk * tpm / nchunk, t1 = (chunk + 1) * tpm / nchunk;
  const __nv_bfloat16* inm = in + mb * P * 32;
  const __nv_bfloat16* dzm = dz + mb * P * 32;
  // buffer b: input range [g][i] (4 x R rows), then dz [g][k] (4 x 128 rows), 16 bytes each
  auto sin = [&](int b) { return ws + b * buf_bytes; };
  auto sdz = [&](int b) { return ws + b * buf_bytes + (size_t)4 * R * 16; };
  auto stage = [&](int tile, int b) {
    const int s0 = tile * kTcRows;
    {
      const __nv_bfloat16* src = inm + (tid & 3) * 8;
      unsigned char* dst = sin(b) + (size_t)(tid & 3) * R * 16;
      halo_walk(s0 - W - 1, tid >> 2, blockDim.x >> 2, R, W, M, [&](int i, int pix) {
        cp_async16_zfill(dst + (size_t)i * 16, src + (long long)pix * 32, true);
      });
    }
    for (int idx = tid; idx < 4 * kTcRows; idx += blockDim.x) {
      const int i = idx >> 2, g = idx & 3;
      const int so = s0 + i, ys = so / W, xs = so - ys * W;
      const bool ok = ys < M && xs >= 1 && xs <= M;
      const long long pix = ok ? (long long)ys * M + (xs - 1) : 0;
      cp_async16_zfill(sdz(b) + ((size_t)g * kTcRows + i) * 16, dzm + pix * 32 + g * 8, ok);
    }
    cp_async_commit();
  };
  const int tap = warp, a = tap / 3, bb = tap % 3;
  const int i0 = W + 1 + (bb - 1) * W + (a - 1);  // the tap's first input row of a tile
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;
  // ldmatrix row of this lane: matrix lane / 8, row lane % 8
  const int lm = lane >> 3, lr = lane & 7;
  // bias gradient db[o = lane] = sum_p dz[p][o] from the same staged rows: warp w takes rows
  // w, w + 9, ... of every tile
  float bacc = 0.0f;
  int b = 0;
  if (t0 < t1) stage(t0, 0);
  for (int tile = t0; tile < t1; ++tile, b ^= 1) {
    if (tile + 1 < t1) stage(tile + 1, b ^ 1);
    else cp_async_commit();
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    const unsigned char* si = sin(b);
    const unsigned char* sd = sdz(b);
#pragma unroll 1
    for (int ks = 0; ks < kTcRows / 16; ++ks) {
      unsigned af[2][4], bf[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        // matrices: (o 0-7, k 0-7), (o 8-15, k 0-7), (o 0-7, k 8-15), (o 8-15, k 8-15) of chunks 2mt, 2mt+1
        const int g = 2 * mt + (lm & 1), k = ks * 16 + (lm >> 1) * 8 + lr;
        ldsm_x4_t(af[mt], sd + ((size_t)g * kTcRows + k) * 16);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        // matrices: (c chunk 2np, k 0-7), (2np, k 8-15), (2np+1, k 0-7), (2np+1, k 8-15)
        const int g = 2 * np + (lm >> 1), k = ks * 16 + (lm & 1) * 8 + lr;
        unsigned r4[4];
        ldsm_x4_t(r4, si + ((size_t)g * R + i0 + k) * 16);
        bf[2 * np][0] = r4[0];
        bf[2 * np][1] = r4[1];
        bf[2 * np + 1][0] = r4[2];
        bf[2 * np + 1][1] = r4[3];
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt]);
    }
    for (int k = warp; k < kTcRows; k += 9)
      bacc += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(sd + ((size_t)(lane >> 3) * kTcRows + k) * 16 +
                                                                         (lane & 7) * 2));
    __syncthreads();  // every warp is done with buffer b before the next stage overwrites it
  }
  cp_async_wait_all();
  __shared__ float bred[9][32];
  bred[warp][lane] = bacc;
  __syncthreads();
  if (warp == 0) {  // the warps' partial bias sums in warp order
    float sb = 0.0f;
    for (int w = 0; w < 9; ++w) sb += bred[w][lane];
    bpart[((long long)mb * nchunk + chunk) * 32 + lane] = sb;
  }
  const int g = lane >> 2, t4 = lane & 3;
  float* dst = chunkbuf + (((long long)mb * 9 + tap) * nchunk + chunk) * 1024;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = mt * 16 + g + 8 * (q / 2), c = nt * 8 + 2 * t4 + (q % 2);
        dst[o * 32 + c] = acc[mt][nt][q];
      }
}

}  // namespace cnn
}  // namespace spadj
