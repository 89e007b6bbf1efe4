// Convolutional coarse corrector (network declared in learned.cuh): BF16
// operands with FP32 accumulation for the 3x3x3 convolutions, their data
// and weight gradients, the linear up-sampling and its adjoint, the
// mean-squared loss and Adam.  The C ABI rm_net_* (include/rm.h) exposes
// the network on its own; capi.cu drives it as a coarse corrector.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/rm.h"
#include "device.cuh"
#include "learned.cuh"

namespace rmn {
namespace {

using bf16 = __nv_bfloat16;

#define CKN(x)                                                                                  \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) throw std::runtime_error(std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

__device__ __forceinline__ float tof(float v) { return v; }
__device__ __forceinline__ float tof(bf16 v) { return __bfloat162float(v); }
__device__ __forceinline__ void put(float *p, float v) { *p = v; }
__device__ __forceinline__ void put(bf16 *p, float v) { *p = __float2bfloat16_rn(v); }

// One 3x3x3 convolution (or the transpose of one) as a gather:
//   out[b, o, c_out] = bias + sum_{tap, c_in} W(c_out, tap, c_in) in[b, src(o, tap), c_in]
// forward:    src = stride * o + tap - 1 per direction
// transposed: src = (o + 1 - tap) / stride when that is an integer
// (the data gradient of the forward conv with the same weights).
struct ConvArgs {
  int cin, cout;          // reduction and output channels
  int din[3], dout[3];    // voxel dims of the tensor read and of the one written
  int stride, transposed;
  int w_so, w_sd, w_si;   // weight strides of (output channel, tap, reduction channel)
  int relu, accumulate;
};

__device__ __forceinline__ int tap_src(int o, int t, int s, int n, int transposed) {
  if (!transposed) {
    const int i = s * o + t - 1;
    return (i >= 0 && i < n) ? i : -1;
  }
  int u = o + 1 - t;
  if (u < 0) return -1;
  if (s == 2) {
    if (u & 1) return -1;
    u >>= 1;
  }
  return u < n ? u : -1;
}

__device__ __forceinline__ int pick3(int t, int a0, int a1, int a2) {
  return t == 0 ? a0 : (t == 1 ? a1 : a2);
}

// One thread per output voxel, OT output channels per block row (blockIdx.y).
// The reduction runs over units u = (c_in chunk of IC) * 3 + dz, each unit a
// plane of 9 taps; blockIdx.z takes the units [z * per, (z + 1) * per).  The
// unit's weights for the OT channels are staged in shared memory ([tap][c_in]
// [c_out], c_out fastest) and read as broadcasts.  With one split the block
// finishes the output (bias, ReLU, accumulate, store); with several (small
// grids: too few voxels to fill the GPU) it adds its FP32 partial sums to
// `part` and conv_finish_kernel finishes.
template <typename TI, typename TO, int OT, int IC>
__global__ void __launch_bounds__(128) conv_kernel(ConvArgs a, long long total, int per,
                                                   const TI *__restrict__ in,
                                                   const bf16 *__restrict__ W,
                                                   const float *__restrict__ bias,
                                                   TO *__restrict__ out, float *__restrict__ part) {
  __shared__ __align__(16) float ws[9 * IC * OT];
  const long long gv = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = gv < total;
  const int nvo = a.dout[0] * a.dout[1] * a.dout[2];
  const long long nvi = (long long)a.din[0] * a.din[1] * a.din[2];
  const long long b = live ? gv / nvo : 0;
  const int vo = live ? (int)(gv - b * nvo) : 0;
  const int ox = vo % a.dout[0], oy = (vo / a.dout[0]) % a.dout[1], oz = vo / (a.dout[0] * a.dout[1]);
  const int sx0 = tap_src(ox, 0, a.stride, a.din[0], a.transposed);
  const int sx1 = tap_src(ox, 1, a.stride, a.din[0], a.transposed);
  const int sx2 = tap_src(ox, 2, a.stride, a.din[0], a.transposed);
  const int sy0 = tap_src(oy, 0, a.stride, a.din[1], a.transposed);
  const int sy1 = tap_src(oy, 1, a.stride, a.din[1], a.transposed);
  const int sy2 = tap_src(oy, 2, a.stride, a.din[1], a.transposed);
  const int sz0 = tap_src(oz, 0, a.stride, a.din[2], a.transposed);
  const int sz1 = tap_src(oz, 1, a.stride, a.din[2], a.transposed);
  const int sz2 = tap_src(oz, 2, a.stride, a.din[2], a.transposed);
  const int o0 = blockIdx.y * OT;
  float acc[OT];
#pragma unroll
  for (int o = 0; o < OT; ++o) acc[o] = 0.f;
  const TI *base = in + b * nvi * a.cin;
  const int nunits = 3 * ((a.cin + IC - 1) / IC);
  const int u1 = min(nunits, (int)(blockIdx.z + 1) * per);
  for (int u = blockIdx.z * per; u < u1; ++u) {
    const int ic0 = (u / 3) * IC, dz = u % 3;
    const int icn = min(IC, a.cin - ic0);
    __syncthreads();
    for (int e = threadIdx.x; e < 9 * IC * OT; e += blockDim.x) {
      const int o = e % OT, i = (e / OT) % IC, d = dz * 9 + e / (OT * IC);
      float w = 0.f;
      if (i < icn && o0 + o < a.cout)
        w = __bfloat162float(W[(long long)(o0 + o) * a.w_so + (long long)d * a.w_sd +
                               (long long)(ic0 + i) * a.w_si]);
      ws[e] = w;
    }
    __syncthreads();
    const int iz = pick3(dz, sz0, sz1, sz2);
    if (!live || iz < 0) continue;
    for (int t = 0; t < 9; ++t) {
      const int ix = pick3(t % 3, sx0, sx1, sx2), iy = pick3(t / 3, sy0, sy1, sy2);
      if (ix < 0 || iy < 0) continue;
      const TI *src = base + ((long long)(iz * a.din[1] + iy) * a.din[0] + ix) * a.cin + ic0;
      const float *wr = ws + t * IC * OT;
#pragma unroll 4
      for (int i = 0; i < icn; ++i) {
        const float x = tof(src[i]);
#pragma unroll
        for (int o = 0; o < OT; ++o) acc[o] = fmaf(wr[i * OT + o], x, acc[o]);
      }
    }
  }
  if (!live) return;
  if (gridDim.z > 1) {
    float *pp = part + (long long)blockIdx.z * total * a.cout + gv * a.cout + o0;
#pragma unroll
    for (int o = 0; o < OT; ++o)
      if (o0 + o < a.cout) pp[o] = acc[o];
    return;
  }
  TO *dst = out + gv * a.cout + o0;
#pragma unroll
  for (int o = 0; o < OT; ++o) {
    if (o0 + o < a.cout) {
      float v = acc[o] + (bias ? bias[o0 + o] : 0.f);
      if (a.relu) v = fmaxf(v, 0.f);
      if (a.accumulate) v += tof(dst[o]);
      put(dst + o, v);
    }
  }
}

// out = act(sum_z part[z] + bias) (+ out): the epilogue of a split conv; the
// slices are added in a fixed order, so the result does not depend on timing
template <typename TO>
__global__ void conv_finish_kernel(long long n, int cout, int splits, const float *__restrict__ part,
                                   const float *__restrict__ bias, int relu, int accumulate,
                                   TO *__restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = 0.f;
  for (int z = 0; z < splits; ++z) v += part[(long long)z * n + i];
  v += bias ? bias[i % cout] : 0.f;
  if (relu) v = fmaxf(v, 0.f);
  if (accumulate) v += tof(out[i]);
  put(out + i, v);
}

// Weight and bias gradients of a forward conv:
//   dW[c_out][tap][c_in] += sum_{b, o} g[b, o, c_out] x[b, stride o + tap - 1, c_in],
//   db[c_out] += sum_{b, o} g[b, o, c_out].
// Block = 16 x 16 (c_in, c_out) pairs with 27 accumulators each, over a
// chunk of output voxels staged 16 at a time in shared memory; the partial
// sums of the chunks meet in FP32 atomics.
struct WgArgs {
  int ci, co;
  int din[3], dout[3];
  int stride;
};

__global__ void __launch_bounds__(256) wgrad_kernel(WgArgs a, long long total, long long chunk,
                                                    const float *__restrict__ g,
                                                    const bf16 *__restrict__ x,
                                                    float *__restrict__ dW, float *__restrict__ db) {
  __shared__ float gs[16][16];
  __shared__ float xs[16][27][16];
  __shared__ long long vb_base[16];
  __shared__ int vb_c[16][3];
  const int ti = threadIdx.x & 15, to = threadIdx.x >> 4;
  const int nti = (a.ci + 15) / 16;
  const int i0 = (blockIdx.y % nti) * 16, o0 = (blockIdx.y / nti) * 16;
  const int nvo = a.dout[0] * a.dout[1] * a.dout[2];
  const long long nvi = (long long)a.din[0] * a.din[1] * a.din[2];
  float acc[27];
#pragma unroll
  for (int d = 0; d < 27; ++d) acc[d] = 0.f;
  float accb = 0.f;
  const long long v0 = (long long)blockIdx.x * chunk;
  const long long v1 = min(total, v0 + chunk);
  for (long long vb = v0; vb < v1; vb += 16) {
    __syncthreads();
    if (threadIdx.x < 16) {
      const long long gv = vb + threadIdx.x;
      long long bb = 0;
      int vo = 0;
      if (gv < v1) {
        bb = gv / nvo;
        vo = (int)(gv - bb * nvo);
      }
      vb_base[threadIdx.x] = gv < v1 ? bb * nvi : -1;
      vb_c[threadIdx.x][0] = a.stride * (vo % a.dout[0]) - 1;
      vb_c[threadIdx.x][1] = a.stride * ((vo / a.dout[0]) % a.dout[1]) - 1;
      vb_c[threadIdx.x][2] = a.stride * (vo / (a.dout[0] * a.dout[1])) - 1;
    }
    {
      const int v = threadIdx.x >> 4, o = threadIdx.x & 15;
      const long long gv = vb + v;
      gs[v][o] = (gv < v1 && o0 + o < a.co) ? g[gv * a.co + o0 + o] : 0.f;
    }
    __syncthreads();
    for (int dv = to; dv < 16 * 27; dv += 16) {
      const int v = dv / 27, d = dv - 27 * (dv / 27);
      float val = 0.f;
      const long long bbase = vb_base[v];
      if (bbase >= 0 && i0 + ti < a.ci) {
        const int ix = vb_c[v][0] + d % 3, iy = vb_c[v][1] + (d / 3) % 3, iz = vb_c[v][2] + d / 9;
        if (ix >= 0 && ix < a.din[0] && iy >= 0 && iy < a.din[1] && iz >= 0 && iz < a.din[2])
          val = __bfloat162float(
              x[(bbase + ((long long)iz * a.din[1] + iy) * a.din[0] + ix) * a.ci + i0 + ti]);
      }
      xs[v][d][ti] = val;
    }
    __syncthreads();
#pragma unroll 2
    for (int v = 0; v < 16; ++v) {
      const float gv = gs[v][to];
      accb += gv;
#pragma unroll
      for (int d = 0; d < 27; ++d) acc[d] = fmaf(gv, xs[v][d][ti], acc[d]);
    }
  }
  if (o0 + to < a.co && i0 + ti < a.ci) {
#pragma unroll
    for (int d = 0; d < 27; ++d) atomicAdd(&dW[((long long)(o0 + to) * 27 + d) * a.ci + i0 + ti], acc[d]);
  }
  if (db && ti == 0 && blockIdx.y % nti == 0 && o0 + to < a.co) atomicAdd(&db[o0 + to], accb);
}

// Vertex-centred linear interpolation by 2 per direction (coarse dims c,
// fine dims 2c - 1): even fine index -> the coarse node, odd -> the mean of
// its two neighbours.
__global__ void up_kernel(int ch, int c0, int c1, int c2, int f0, int f1, int f2, long long total,
                          const bf16 *__restrict__ in, bf16 *__restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int c = (int)(e % ch);
  const long long gv = e / ch;
  const long long nf = (long long)f0 * f1 * f2, nc = (long long)c0 * c1 * c2;
  const long long b = gv / nf;
  const int v = (int)(gv - b * nf);
  const int fx = v % f0, fy = (v / f0) % f1, fz = v / (f0 * f1);
  const int nx = (fx & 1) ? 2 : 1, ny = (fy & 1) ? 2 : 1, nz = (fz & 1) ? 2 : 1;
  const float w = 1.f / (nx * ny * nz);
  float s = 0.f;
  for (int kz = 0; kz < nz; ++kz)
    for (int ky = 0; ky < ny; ++ky)
      for (int kx = 0; kx < nx; ++kx) {
        const int cx = (fx >> 1) + kx, cy = (fy >> 1) + ky, cz = (fz >> 1) + kz;
        s += __bfloat162float(in[((b * nc) + ((long long)cz * c1 + cy) * c0 + cx) * ch + c]);
      }
  out[e] = __float2bfloat16_rn(s * w);
}

// Adjoint of up_kernel: coarse node c collects fine 2c (weight 1) and
// 2c +- 1 (weight 1/2) per direction.
__global__ void up_adjoint_kernel(int ch, int c0, int c1, int c2, int f0, int f1, int f2,
                                  long long total, const float *__restrict__ gin,
                                  float *__restrict__ gout) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int c = (int)(e % ch);
  const long long gv = e / ch;
  const long long nf = (long long)f0 * f1 * f2, nc = (long long)c0 * c1 * c2;
  const long long b = gv / nc;
  const int v = (int)(gv - b * nc);
  const int cx = v % c0, cy = (v / c0) % c1, cz = v / (c0 * c1);
  float s = 0.f;
  for (int kz = -1; kz <= 1; ++kz) {
    const int fz = 2 * cz + kz;
    if (fz < 0 || fz >= f2) continue;
    const float wz = kz ? 0.5f : 1.f;
    for (int ky = -1; ky <= 1; ++ky) {
      const int fy = 2 * cy + ky;
      if (fy < 0 || fy >= f1) continue;
      const float wy = ky ? 0.5f : 1.f;
      for (int kx = -1; kx <= 1; ++kx) {
        const int fx = 2 * cx + kx;
        if (fx < 0 || fx >= f0) continue;
        const float wx = kx ? 0.5f : 1.f;
        s += wz * wy * wx * gin[((b * nf) + ((long long)fz * f1 + fy) * f0 + fx) * ch + c];
      }
    }
  }
  gout[e] = s;
}

__global__ void add_bf16_kernel(long long n, const bf16 *a, const bf16 *b, bf16 *c) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = __float2bfloat16_rn(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

__global__ void cast_kernel(long long n, const float *a, bf16 *b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// g *= (a > 0): the ReLU derivative, a the stored activation
__global__ void relu_mask_kernel(long long n, float *g, const bf16 *a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(__bfloat162float(a[i]) > 0.f)) g[i] = 0.f;
}

__global__ void mse_kernel(long long total, int nvox, const float *y, const float *t,
                           const uint8_t *mask, float scale, float *dy, double *loss) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < total) {
    const float m = mask[i % nvox] ? 1.f : 0.f;
    const float d = m * (y[i] - t[i]);
    dy[i] = 2.f * d * scale;
    l = d * d * scale;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, (double)l);
}

__global__ void adam_kernel(long long n, float *w, const float *g, float *m, float *v, bf16 *wb,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
}

unsigned grid1(long long n, int t) { return (unsigned)((n + t - 1) / t); }

struct Layer {
  int cin, cout, stride, lin, lout;  // channels, stride, levels of input and output
  long long woff, boff;
};

// tensor roles
enum { T_X = 0, T_E0A, T_E, T_D, T_U, T_A, T_S, T_H, T_ROLES };

}  // namespace

struct Net {
  NetSpec s{};
  cudaStream_t stream = nullptr;
  int dims[5][3] = {};
  long long nvox[5] = {};
  int ch[5] = {};
  std::vector<Layer> layers;
  long long nparams = 0;
  float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  bf16 *wbf = nullptr;
  float *part = nullptr;  // partial sums of split convolutions (largest tensor)
  int adam_t = 0;
  int batch = 0;
  // activations (BF16) and their gradients (FP32), per role and level
  bf16 *act[T_ROLES][5] = {};
  float *gact[T_ROLES][5] = {};
  std::vector<void *> allocs;
  template <typename T>
  T *alloc(size_t n) {
    void *p = nullptr;
    CKN(cudaMalloc(&p, (n ? n : 1) * sizeof(T)));
    allocs.push_back(p);
    return (T *)p;
  }
  ~Net() {
    for (void *p : allocs) cudaFree(p);
  }
};

namespace {

int add_layer(Net *n, int cin, int cout, int stride, int lin, int lout) {
  Layer L{cin, cout, stride, lin, lout, n->nparams, 0};
  n->nparams += (long long)cout * 27 * cin;
  L.boff = n->nparams;
  n->nparams += cout;
  n->layers.push_back(L);
  return (int)n->layers.size() - 1;
}

// layer indices in parameter order
struct Idx {
  int e0a, e0, head;
  int down[5], enc[5], upc[5], hc[5];
};

Idx layer_index(const NetSpec &s) {
  Idx x{};
  int i = 0;
  x.e0a = i++;
  x.e0 = i++;
  for (int l = 1; l <= s.levels; ++l) {
    x.down[l] = i++;
    x.enc[l] = i++;
  }
  for (int l = s.levels - 1; l >= 0; --l) {
    x.upc[l] = i++;
    x.hc[l] = i++;
  }
  x.head = i++;
  return x;
}

// Grids of fewer than two blocks per SM split the reduction (see
// conv_kernel) to reach about four.  part: FP32 scratch for the splits'
// slices, splits * total * cout <= (4 + 2) * kSMs * 128 * 16 floats
// (kSplitScratch), since a split grid has fewer than 2 * kSMs blocks of
// 128 voxels x 16 channels.
constexpr int kSMs = 152;
constexpr long long kSplitScratch = (4LL + 2LL) * kSMs * 128 * 16;

template <typename TI, typename TO, int OT, int IC>
void run_conv(const ConvArgs &a, int batch, const TI *in, const bf16 *W, const float *bias, TO *out,
              float *part, cudaStream_t s) {
  static_assert(OT <= 16, "split scratch bound assumes at most 16 channels per block");
  const long long total = (long long)batch * a.dout[0] * a.dout[1] * a.dout[2];
  const long long bxy = (long long)grid1(total, 128) * ((a.cout + OT - 1) / OT);
  const int nunits = 3 * ((a.cin + IC - 1) / IC);
  int splits = 1;
  if (bxy < 2 * kSMs) splits = (int)std::min<long long>(nunits, (4 * kSMs + bxy - 1) / bxy);
  const int per = (nunits + splits - 1) / splits;
  splits = (nunits + per - 1) / per;
  if (splits > 1 && (long long)splits * total * a.cout > kSplitScratch)
    throw std::runtime_error("conv split scratch too small");
  dim3 grid(grid1(total, 128), (a.cout + OT - 1) / OT, splits);
  conv_kernel<TI, TO, OT, IC><<<grid, 128, 0, s>>>(a, total, per, in, W, bias, out, part);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
  if (splits > 1) {
    const long long n = total * a.cout;
    conv_finish_kernel<TO><<<grid1(n, 256), 256, 0, s>>>(n, a.cout, splits, part, bias, a.relu,
                                                         a.accumulate, out);
    CKN(cudaGetLastError());
    rmd::add_launches(1);
  }
}

ConvArgs fwd_args(const Net *n, const Layer &L, int relu) {
  ConvArgs a{};
  a.cin = L.cin;
  a.cout = L.cout;
  for (int d = 0; d < 3; ++d) {
    a.din[d] = n->dims[L.lin][d];
    a.dout[d] = n->dims[L.lout][d];
  }
  a.stride = L.stride;
  a.transposed = 0;
  a.w_so = 27 * L.cin;
  a.w_sd = L.cin;
  a.w_si = 1;
  a.relu = relu;
  a.accumulate = 0;
  return a;
}

// data gradient of layer L: gin (level lin, cin channels) from gout (level lout, cout)
void conv_bwd_data(Net *n, const Layer &L, const float *gout, float *gin, int accumulate) {
  ConvArgs a{};
  a.cin = L.cout;
  a.cout = L.cin;
  for (int d = 0; d < 3; ++d) {
    a.din[d] = n->dims[L.lout][d];
    a.dout[d] = n->dims[L.lin][d];
  }
  a.stride = L.stride;
  a.transposed = 1;
  a.w_so = 1;
  a.w_sd = L.cin;
  a.w_si = 27 * L.cin;
  a.relu = 0;
  a.accumulate = accumulate;
  run_conv<float, float, 16, 16>(a, n->batch, gout, n->wbf + L.woff, nullptr, gin, n->part,
                                 n->stream);
}

void conv_fwd(Net *n, const Layer &L, const bf16 *in, bf16 *out) {
  run_conv<bf16, bf16, 16, 16>(fwd_args(n, L, 1), n->batch, in, n->wbf + L.woff,
                               n->master + L.boff, out, n->part, n->stream);
}

void conv_wgrad(Net *n, const Layer &L, const float *gout, const bf16 *in) {
  WgArgs a{};
  a.ci = L.cin;
  a.co = L.cout;
  for (int d = 0; d < 3; ++d) {
    a.din[d] = n->dims[L.lin][d];
    a.dout[d] = n->dims[L.lout][d];
  }
  a.stride = L.stride;
  const long long total = (long long)n->batch * n->nvox[L.lout];
  const int tiles = ((L.cin + 15) / 16) * ((L.cout + 15) / 16);
  long long blocks = std::max(1LL, std::min((total + 15) / 16, (long long)(4 * 152 / tiles) + 1));
  long long chunk = (total + blocks - 1) / blocks;
  chunk = (chunk + 15) / 16 * 16;
  blocks = (total + chunk - 1) / chunk;
  wgrad_kernel<<<dim3((unsigned)blocks, tiles), 256, 0, n->stream>>>(
      a, total, chunk, gout, in, n->grad + L.woff, n->grad + L.boff);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
}

void relu_mask(Net *n, float *g, const bf16 *a, long long count) {
  relu_mask_kernel<<<grid1(count, 256), 256, 0, n->stream>>>(count, g, a);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
}

long long tsize(const Net *n, int lvl, int c) { return (long long)n->batch * n->nvox[lvl] * c; }

uint64_t splitmix(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace

Net *create(const NetSpec &s, uint64_t seed, cudaStream_t stream) {
  if (s.levels < 0 || s.levels > 4) throw std::runtime_error("levels must be 0..4");
  if (s.width < 1 || s.width > 256 || s.in_ch < 1 || s.in_ch > 64 || s.max_batch < 1)
    throw std::runtime_error("bad network width, input channels or batch");
  for (int d = 0; d < 3; ++d)
    if (s.dims[d] < 2 || (s.dims[d] - 1) % (1 << s.levels) != 0)
      throw std::runtime_error("grid dims - 1 must be divisible by 2^levels");
  std::unique_ptr<Net> n(new Net());
  n->s = s;
  n->stream = stream;
  for (int l = 0; l <= s.levels; ++l) {
    n->nvox[l] = 1;
    for (int d = 0; d < 3; ++d) {
      n->dims[l][d] = (s.dims[d] - 1) / (1 << l) + 1;
      n->nvox[l] *= n->dims[l][d];
    }
    n->ch[l] = s.width << l;
  }
  const int L = s.levels;
  add_layer(n.get(), s.in_ch, n->ch[0], 1, 0, 0);
  add_layer(n.get(), n->ch[0], n->ch[0], 1, 0, 0);
  for (int l = 1; l <= L; ++l) {
    add_layer(n.get(), n->ch[l - 1], n->ch[l], 2, l - 1, l);
    add_layer(n.get(), n->ch[l], n->ch[l], 1, l, l);
  }
  for (int l = L - 1; l >= 0; --l) {
    add_layer(n.get(), n->ch[l + 1], n->ch[l], 1, l, l);
    add_layer(n.get(), n->ch[l], n->ch[l], 1, l, l);
  }
  add_layer(n.get(), n->ch[0], 1, 1, 0, 0);
  const size_t np = (size_t)n->nparams;
  n->master = n->alloc<float>(np);
  n->grad = n->alloc<float>(np);
  n->m = n->alloc<float>(np);
  n->v = n->alloc<float>(np);
  n->wbf = n->alloc<bf16>(np);
  CKN(cudaMemsetAsync(n->m, 0, np * sizeof(float), stream));
  CKN(cudaMemsetAsync(n->v, 0, np * sizeof(float), stream));
  const long long B = s.max_batch;
  auto both = [&](int role, int lvl, int c) {
    n->act[role][lvl] = n->alloc<bf16>((size_t)(B * n->nvox[lvl] * c));
    n->gact[role][lvl] = n->alloc<float>((size_t)(B * n->nvox[lvl] * c));
  };
  both(T_X, 0, s.in_ch);
  both(T_E0A, 0, n->ch[0]);
  for (int l = 0; l <= L; ++l) both(T_E, l, n->ch[l]);
  for (int l = 1; l <= L; ++l) both(T_D, l, n->ch[l]);
  for (int l = 0; l < L; ++l) {
    both(T_U, l, n->ch[l + 1]);
    both(T_A, l, n->ch[l]);
    both(T_S, l, n->ch[l]);
    both(T_H, l, n->ch[l]);
  }
  n->part = n->alloc<float>((size_t)kSplitScratch);
  // He-normal initial weights (Box-Muller on a SplitMix64 stream), zero biases
  std::vector<float> w(np, 0.f);
  uint64_t st = seed;
  for (const Layer &Ly : n->layers) {
    const double sd = std::sqrt(2.0 / (27.0 * Ly.cin));
    for (long long i = Ly.woff; i < Ly.boff; ++i) {
      const double u1 = ((splitmix(st) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
      const double u2 = (splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      w[i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  }
  set_params(n.get(), w.data());
  return n.release();
}

void destroy(Net *net) { delete net; }
const NetSpec &spec(const Net *net) { return net->s; }
long long num_params(const Net *net) { return net->nparams; }
float *grads(Net *net) { return net->grad; }

void get_params(const Net *n, float *host) {
  CKN(cudaStreamSynchronize(n->stream));
  CKN(cudaMemcpy(host, n->master, n->nparams * sizeof(float), cudaMemcpyDeviceToHost));
}

void set_params(Net *n, const float *host) {
  CKN(cudaStreamSynchronize(n->stream));
  CKN(cudaMemcpy(n->master, host, n->nparams * sizeof(float), cudaMemcpyHostToDevice));
  cast_kernel<<<grid1(n->nparams, 256), 256, 0, n->stream>>>(n->nparams, n->master, n->wbf);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
  CKN(cudaMemsetAsync(n->m, 0, n->nparams * sizeof(float), n->stream));
  CKN(cudaMemsetAsync(n->v, 0, n->nparams * sizeof(float), n->stream));
  n->adam_t = 0;
}

void forward(Net *n, int batch, const float *x, float *y) {
  if (batch < 1 || batch > n->s.max_batch) throw std::runtime_error("batch out of range");
  n->batch = batch;
  cudaStream_t s = n->stream;
  const int L = n->s.levels;
  const Idx ix = layer_index(n->s);
  const long long nx = tsize(n, 0, n->s.in_ch);
  cast_kernel<<<grid1(nx, 256), 256, 0, s>>>(nx, x, n->act[T_X][0]);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
  conv_fwd(n, n->layers[ix.e0a], n->act[T_X][0], n->act[T_E0A][0]);
  conv_fwd(n, n->layers[ix.e0], n->act[T_E0A][0], n->act[T_E][0]);
  for (int l = 1; l <= L; ++l) {
    conv_fwd(n, n->layers[ix.down[l]], n->act[T_E][l - 1], n->act[T_D][l]);
    conv_fwd(n, n->layers[ix.enc[l]], n->act[T_D][l], n->act[T_E][l]);
  }
  for (int l = L - 1; l >= 0; --l) {
    const bf16 *hin = (l + 1 == L) ? n->act[T_E][L] : n->act[T_H][l + 1];
    const int c = n->ch[l + 1];
    const long long tot = tsize(n, l, c);
    up_kernel<<<grid1(tot, 256), 256, 0, s>>>(c, n->dims[l + 1][0], n->dims[l + 1][1],
                                               n->dims[l + 1][2], n->dims[l][0], n->dims[l][1],
                                               n->dims[l][2], tot, hin, n->act[T_U][l]);
    CKN(cudaGetLastError());
    conv_fwd(n, n->layers[ix.upc[l]], n->act[T_U][l], n->act[T_A][l]);
    const long long ts = tsize(n, l, n->ch[l]);
    add_bf16_kernel<<<grid1(ts, 256), 256, 0, s>>>(ts, n->act[T_A][l], n->act[T_E][l], n->act[T_S][l]);
    CKN(cudaGetLastError());
    rmd::add_launches(2);
    conv_fwd(n, n->layers[ix.hc[l]], n->act[T_S][l], n->act[T_H][l]);
  }
  const Layer &H = n->layers[ix.head];
  const bf16 *hin = L > 0 ? n->act[T_H][0] : n->act[T_E][0];
  run_conv<bf16, float, 1, 64>(fwd_args(n, H, 0), batch, hin, n->wbf + H.woff, n->master + H.boff,
                               y, n->part, s);
}

void backward(Net *n, const float *dy, float *dx) {
  cudaStream_t s = n->stream;
  const int L = n->s.levels;
  const Idx ix = layer_index(n->s);
  CKN(cudaMemsetAsync(n->grad, 0, n->nparams * sizeof(float), s));
  // head
  const Layer &H = n->layers[ix.head];
  bf16 *h0 = L > 0 ? n->act[T_H][0] : n->act[T_E][0];
  float *gh0 = L > 0 ? n->gact[T_H][0] : n->gact[T_E][0];
  conv_wgrad(n, H, dy, h0);
  conv_bwd_data(n, H, dy, gh0, 0);
  relu_mask(n, gh0, h0, tsize(n, 0, n->ch[0]));
  // decoder, level 0 upwards
  for (int l = 0; l < L; ++l) {
    const Layer &Lh = n->layers[ix.hc[l]], &Lu = n->layers[ix.upc[l]];
    float *gS = n->gact[T_S][l];
    conv_wgrad(n, Lh, n->gact[T_H][l], n->act[T_S][l]);
    conv_bwd_data(n, Lh, n->gact[T_H][l], gS, 0);
    const long long ts = tsize(n, l, n->ch[l]);
    // s = a + e: the skip receives the same gradient
    CKN(cudaMemcpyAsync(n->gact[T_E][l], gS, ts * sizeof(float), cudaMemcpyDeviceToDevice, s));
    relu_mask(n, gS, n->act[T_A][l], ts);
    conv_wgrad(n, Lu, gS, n->act[T_U][l]);
    conv_bwd_data(n, Lu, gS, n->gact[T_U][l], 0);
    const int c = n->ch[l + 1];
    float *gh = (l + 1 == L) ? n->gact[T_E][L] : n->gact[T_H][l + 1];
    const long long tot = tsize(n, l + 1, c);
    up_adjoint_kernel<<<grid1(tot, 256), 256, 0, s>>>(c, n->dims[l + 1][0], n->dims[l + 1][1],
                                                       n->dims[l + 1][2], n->dims[l][0],
                                                       n->dims[l][1], n->dims[l][2], tot,
                                                       n->gact[T_U][l], gh);
    CKN(cudaGetLastError());
    rmd::add_launches(1);
    if (l + 1 < L) relu_mask(n, gh, n->act[T_H][l + 1], tot);
  }
  // encoder, deepest level first
  for (int l = L; l >= 1; --l) {
    const Layer &Le = n->layers[ix.enc[l]], &Ld = n->layers[ix.down[l]];
    float *gE = n->gact[T_E][l], *gD = n->gact[T_D][l];
    relu_mask(n, gE, n->act[T_E][l], tsize(n, l, n->ch[l]));
    conv_wgrad(n, Le, gE, n->act[T_D][l]);
    conv_bwd_data(n, Le, gE, gD, 0);
    relu_mask(n, gD, n->act[T_D][l], tsize(n, l, n->ch[l]));
    conv_wgrad(n, Ld, gD, n->act[T_E][l - 1]);
    conv_bwd_data(n, Ld, gD, n->gact[T_E][l - 1], L > 0 ? 1 : 0);
  }
  const Layer &L0 = n->layers[ix.e0a], &L1 = n->layers[ix.e0];
  if (L > 0) relu_mask(n, n->gact[T_E][0], n->act[T_E][0], tsize(n, 0, n->ch[0]));
  conv_wgrad(n, L1, n->gact[T_E][0], n->act[T_E0A][0]);
  conv_bwd_data(n, L1, n->gact[T_E][0], n->gact[T_E0A][0], 0);
  relu_mask(n, n->gact[T_E0A][0], n->act[T_E0A][0], tsize(n, 0, n->ch[0]));
  conv_wgrad(n, L0, n->gact[T_E0A][0], n->act[T_X][0]);
  if (dx) conv_bwd_data(n, L0, n->gact[T_E0A][0], dx, 0);
}

void adam(Net *n, float lr, float beta1, float beta2, float eps) {
  n->adam_t += 1;
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, n->adam_t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, n->adam_t)));
  adam_kernel<<<grid1(n->nparams, 256), 256, 0, n->stream>>>(n->nparams, n->master, n->grad, n->m,
                                                              n->v, n->wbf, lr, beta1, beta2, eps,
                                                              c1, c2);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
}

void mse(int batch, int nvox, const float *y, const float *t, const uint8_t *mask, float scale,
         float *dy, double *loss, cudaStream_t s) {
  const long long total = (long long)batch * nvox;
  mse_kernel<<<grid1(total, 256), 256, 0, s>>>(total, nvox, y, t, mask, scale, dy, loss);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
}

namespace {

__global__ void corr_pack_kernel(int nc, long long nvox, const double *cc, const int *lat2free,
                                 const float *logal, const double *scal, float *x) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  const double nn = scal[0];
  const double sc = nn > 0.0 ? sqrt((double)nc / nn) : 0.0;
  const int f = lat2free[v];
  x[2 * v] = f >= 0 ? (float)(sc * cc[f]) : 0.f;
  x[2 * v + 1] = logal[v];
}

__global__ void corr_gather_kernel(int nc, const float *y, const int *free2lat, double *cl) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < nc) cl[f] = (double)y[free2lat[f]];
}

__global__ void corr_scale_kernel(int nc, const double *cl, const double *scal, double *ce) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nc) return;
  const double b = scal[2];
  ce[f] = b > 0.0 ? (scal[1] / b) * cl[f] : 0.0;
}

__global__ void corr_normalise_kernel(int nc, const double *v, const double *scal, float *out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nc) return;
  const double nn = scal[0];
  out[f] = nn > 0.0 ? (float)(sqrt((double)nc / nn) * v[f]) : 0.f;
}

__global__ void corr_batch_kernel(int batch, int nc, long long nvox, const int *idx, const float *R,
                                  const float *T, const int *lat2free, const float *logal, float *x,
                                  float *t) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)batch * nvox) return;
  const int b = (int)(e / nvox);
  const long long v = e - (long long)b * nvox;
  const long long j = idx[b];
  const int f = lat2free[v];
  x[2 * e] = f >= 0 ? R[j * nc + f] : 0.f;
  x[2 * e + 1] = logal[v];
  t[e] = f >= 0 ? T[j * nc + f] : 0.f;
}

}  // namespace

void corr_pack(int nc, long long nvox, const double *cc, const int *lat2free, const float *logal,
               const double *scal, float *x, cudaStream_t s) {
  corr_pack_kernel<<<grid1(nvox, 256), 256, 0, s>>>(nc, nvox, cc, lat2free, logal, scal, x);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
}

void corr_gather(int nc, const float *y, const int *free2lat, double *cl, cudaStream_t s) {
  corr_gather_kernel<<<grid1(nc, 256), 256, 0, s>>>(nc, y, free2lat, cl);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
}

void corr_scale(int nc, const double *cl, const double *scal, double *ce, cudaStream_t s) {
  corr_scale_kernel<<<grid1(nc, 256), 256, 0, s>>>(nc, cl, scal, ce);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
}

void corr_normalise(int nc, const double *v, const double *scal, float *out, cudaStream_t s) {
  corr_normalise_kernel<<<grid1(nc, 256), 256, 0, s>>>(nc, v, scal, out);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
}

void corr_batch(int batch, int nc, long long nvox, const int *idx, const float *R, const float *T,
                const int *lat2free, const float *logal, float *x, float *t, cudaStream_t s) {
  const long long total = (long long)batch * nvox;
  corr_batch_kernel<<<grid1(total, 256), 256, 0, s>>>(batch, nc, nvox, idx, R, T, lat2free, logal,
                                                      x, t);
  CKN(cudaGetLastError());
  rmd::add_launches(1);
}

}  // namespace rmn

// ---------------------------------------------------------------------------
// C ABI: the network on its own (include/rm.h)
struct rm_net {
  rmn::Net *net = nullptr;
  ~rm_net() { rmn::destroy(net); }
};

namespace {
thread_local std::string g_net_error;
int net_fail(int code, const std::string &msg) {
  g_net_error = msg;
  return code;
}
}  // namespace

extern "C" {

int rm_net_create(rm_net **out, const int dims[3], int levels, int width, int in_channels,
                  int max_batch, unsigned long long seed, void *stream) {
  if (!out || !dims) return net_fail(RM_ERR_ARG, "rm_net_create: NULL argument");
  try {
    rmn::NetSpec s{{dims[0], dims[1], dims[2]}, levels, width, in_channels, max_batch};
    std::unique_ptr<rm_net> h(new rm_net());
    h->net = rmn::create(s, seed, (cudaStream_t)stream);
    *out = h.release();
  } catch (const std::exception &e) {
    return net_fail(RM_ERR_ARG, std::string("rm_net_create: ") + e.what());
  }
  return RM_OK;
}

long long rm_net_num_params(const rm_net *net) { return net ? rmn::num_params(net->net) : -1; }

int rm_net_get_params(const rm_net *net, float *params) {
  if (!net || !params) return net_fail(RM_ERR_ARG, "rm_net_get_params: NULL argument");
  try {
    rmn::get_params(net->net, params);
  } catch (const std::exception &e) {
    return net_fail(RM_ERR_CUDA, e.what());
  }
  return RM_OK;
}

int rm_net_set_params(rm_net *net, const float *params) {
  if (!net || !params) return net_fail(RM_ERR_ARG, "rm_net_set_params: NULL argument");
  try {
    rmn::set_params(net->net, params);
  } catch (const std::exception &e) {
    return net_fail(RM_ERR_CUDA, e.what());
  }
  return RM_OK;
}

int rm_net_forward(rm_net *net, int batch, const float *x, float *y) {
  if (!net || !x || !y) return net_fail(RM_ERR_ARG, "rm_net_forward: NULL argument");
  if (batch < 1 || batch > rmn::spec(net->net).max_batch)
    return net_fail(RM_ERR_ARG, "rm_net_forward: batch outside 1..max_batch");
  try {
    rmn::forward(net->net, batch, x, y);
  } catch (const std::exception &e) {
    return net_fail(RM_ERR_CUDA, e.what());
  }
  return RM_OK;
}

int rm_net_backward(rm_net *net, const float *dy, float *grad, float *dx) {
  if (!net || !dy) return net_fail(RM_ERR_ARG, "rm_net_backward: NULL argument");
  try {
    rmn::backward(net->net, dy, dx);
    if (grad)
      CKN(cudaMemcpyAsync(grad, rmn::grads(net->net), rmn::num_params(net->net) * sizeof(float),
                          cudaMemcpyDeviceToDevice, net->net->stream));
  } catch (const std::exception &e) {
    return net_fail(RM_ERR_CUDA, e.what());
  }
  return RM_OK;
}

int rm_net_adam(rm_net *net, float lr) {
  if (!net) return net_fail(RM_ERR_ARG, "rm_net_adam: NULL argument");
  try {
    rmn::adam(net->net, lr, 0.9f, 0.999f, 1e-8f);
  } catch (const std::exception &e) {
    return net_fail(RM_ERR_CUDA, e.what());
  }
  return RM_OK;
}

void rm_net_destroy(rm_net *net) { delete net; }

const char *rm_net_last_error(void) { return g_net_error.c_str(); }

}  // extern "C"
