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

__device__ __forceinline__ unsigned pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
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
  const long long P = (long long)M * M;
  const int tap = blockIdx.y, mb = blockIdx.z, chunk = blockIdx.x;
  const int a = tap / 3, b = tap % 3;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int g = lane / 4, t4 = lane % 4;
  const long long per = (P + nchunk - 1) / nchunk;
  const long long pbeg = chunk * per, pend = min(P, pbeg + per);
  float acc[2][4][4];
  for (int mt = 0; mt < 2; ++mt)
    for (int nt = 0; nt < 4; ++nt)
      for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
  // k-steps of 16 pixels, interleaved over the 4 warps
  for (long long k0 = pbeg + warp * 16; k0 < pend; k0 += 64) {
    // pixels of this lane's k pairs: k0 + 2 t4 + {0, 1} and + 8
    long long pk[4] = {k0 + 2 * t4, k0 + 2 * t4 + 1, k0 + 2 * t4 + 8, k0 + 2 * t4 + 9};
    const __nv_bfloat16* sh[4];
    bool okk[4];
    for (int i = 0; i < 4; ++i) {
      okk[i] = pk[i] < pend;
      const long long pc = okk[i] ? pk[i] : pbeg;
      const int y = (int)(pc / M), x = (int)(pc % M);
      const int xx = (x + a - 1 + M) % M, yy = (y + b - 1 + M) % M;
      sh[i] = in + ((long long)mb * P + (long long)yy * M + xx) * 32;
    }
    const __nv_bfloat16* dzr[4];
    for (int i = 0; i < 4; ++i) dzr[i] = dz + ((long long)mb * P + (okk[i] ? pk[i] : pbeg)) * 32;
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

// sum the chunks of wgrad32_mma_kernel in order into part[mb][w_off(l) + flat W index]
__global__ void wgrad32_finish_kernel(int l, const float* __restrict__ chunkbuf, int nchunk, float* __restrict__ part,
                                      int npar) {
  const int mb = blockIdx.y;
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
