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
#include "mbarrier.cuh"

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

// mma.sync tile constants of the weight-gradient kernel (rows padded to 40
// BF16 = 80 B so fragment reads of the 8 row groups fall in distinct banks)
constexpr int kMmaLd = 40;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return l | (h << 16);
}
__device__ __forceinline__ float tof_any(bf16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float tof_any(float v) { return v; }

// ---- tcgen05 (5th-generation tensor core) helpers, inline PTX ----------------
using rmd::mbar_init;
using rmd::mbar_wait_bounded;
using rmd::smem_u32;

// Shared-memory matrix descriptor of a K-major BF16 operand tile without
// swizzling: 8-row x 16-byte core matrices, LBO = byte distance between core
// matrices adjacent along K, SBO = between 8-row groups; bits 46-48 hold the
// descriptor version 1, swizzle mode 0.
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((saddr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ULL << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (D format 1), BF16 A
// and B (format 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr unsigned tc_idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(unsigned tmem_d, unsigned long long ad, unsigned long long bd, unsigned idesc,
                                       unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on the mbarrier once every tcgen05.mma issued so far by this thread completed
__device__ __forceinline__ void tc_commit(unsigned long long *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes (row = lane)
__device__ __forceinline__ void tc_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// a conv whose tensor-core waits gave up: set once, read and cleared by the host
__device__ int g_conv_timeout = 0;

// Tensor-core form of the same convolution (output channels >= 16): an
// implicit GEMM out[v][c_out] = sum_k A[v][k] W[c_out][k] with k = tap * c_in
// + c_in index (K = 27 c_in), A the gathered input (im2col).  Per CTA a tile
// of 128 voxels x BN output channels accumulates in tensor memory (BN FP32
// columns, TMEM rows = voxels) through tcgen05.mma (M = 128, N = BN, K = 16
// per instruction, BF16 operands) issued by one thread; the threads stage
// 32-wide K chunks of A (one voxel row each) and of W into shared memory in
// the no-swizzle K-major core-matrix layout, double-buffered: chunk i + 1 is
// gathered while the tensor core works on chunk i, and a buffer is rewritten
// only after the mbarrier that tcgen05.commit arrives on says its MMAs are
// done.  blockIdx.z takes the K chunks [z * per, (z + 1) * per) (split
// reduction for small grids, as in conv_kernel).  Every mbarrier wait is
// bounded; on timeout the CTA records it in g_conv_timeout, writes NaN for
// its outputs, waits once more for its MMAs and frees its tensor memory.
constexpr int kTcBM = 128, kTcKC = 32;
// bytes of one buffer: A (128 rows) and B (64 rows max) chunks of 32 BF16
constexpr int kTcABytes = kTcBM * kTcKC * 2, kTcBBytes = 64 * kTcKC * 2;
// 8-row group stride: kTcKC / 8 core matrices of 8 rows x 16 B along K
constexpr int kTcSBO = kTcKC / 8 * 128;
// two stages of A and B plus the barriers, padded to 28 KB: 8 CTAs per SM,
// whose 8 x 64 tensor-memory columns fill the SM's 512 exactly
constexpr int kTcSmem = 28 * 1024;
static_assert(2 * (kTcABytes + kTcBBytes) + 128 <= kTcSmem, "shared memory of the conv stages");

// byte offset of element (r, k) of a rows x kTcKC BF16 tile: 8-row groups of
// kTcSBO bytes, in each group the core matrices of 8 rows x 16 B along K
__device__ __forceinline__ int tc_off(int r, int k) {
  return (r >> 3) * kTcSBO + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

template <typename TI, typename TO, int BN>
__global__ void __launch_bounds__(128) conv_tc_kernel(ConvArgs a, long long total, int per,
                                                      const TI *__restrict__ in, const bf16 *__restrict__ W,
                                                      const float *__restrict__ bias, TO *__restrict__ out,
                                                      float *__restrict__ part) {
  static_assert(BN == 16 || BN == 32 || BN == 64, "N of the MMA tile");
  constexpr int NCOLS = BN < 32 ? 32 : BN;  // TMEM allocation: a power of two >= 32
  constexpr unsigned IDESC = tc_idesc_bf16(kTcBM, BN);
  extern __shared__ __align__(128) unsigned char tsm[];
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(tsm + 2 * (kTcABytes + kTcBBytes));
  unsigned *tmem_slot = reinterpret_cast<unsigned *>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long v0 = (long long)blockIdx.x * kTcBM;
  const int n0 = blockIdx.y * BN;
  const int K = 27 * a.cin;
  const int nkc = (K + kTcKC - 1) / kTcKC;
  const int kc0 = blockIdx.z * per, kc1 = min(nkc, kc0 + per);
  const int nvo = a.dout[0] * a.dout[1] * a.dout[2];
  const long long nvi = (long long)a.din[0] * a.din[1] * a.din[2];
  const long long gv = v0 + tid;  // the voxel (row of A) this thread stages
  const bool live = gv < total;
  const long long b = live ? gv / nvo : 0;
  const int vo = live ? (int)(gv - b * nvo) : 0;
  const int ox = vo % a.dout[0], oy = (vo / a.dout[0]) % a.dout[1], oz = vo / (a.dout[0] * a.dout[1]);
  const TI *base = in + b * nvi * a.cin;
  const bool avec = a.cin % 8 == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0;
  const bool bvec = !a.transposed && a.w_si == 1 && a.cin % 8 == 0 && a.w_so % 8 == 0 &&
                    (reinterpret_cast<uintptr_t>(W) & 15) == 0;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tmem_slot;
  bool ok = true;
  int issued = 0;  // chunks whose MMAs were issued and committed (the same in every thread)
  for (int kc = kc0; kc < kc1 && ok; ++kc) {
    const int i = kc - kc0, buf = i & 1;
    if (i >= 2 && !mbar_wait_bounded(&bar[buf], ((i - 2) >> 1) & 1)) ok = false;  // MMAs of chunk i - 2 done
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    const int k0 = kc * kTcKC;
    // A: row tid, k0 .. k0 + 63 (zero outside the input, beyond K or the voxels)
    unsigned char *As = tsm + buf * kTcABytes;
#pragma unroll
    for (int gq = 0; gq < kTcKC / 8; ++gq) {
      const int k = k0 + 8 * gq;
      uint4 pk = make_uint4(0u, 0u, 0u, 0u);
      if (avec) {
        if (live && k < K) {
          const int tap = k / a.cin, ci = k - tap * a.cin;
          const int ix = tap_src(ox, tap % 3, a.stride, a.din[0], a.transposed);
          const int iy = tap_src(oy, (tap / 3) % 3, a.stride, a.din[1], a.transposed);
          const int iz = tap_src(oz, tap / 9, a.stride, a.din[2], a.transposed);
          if (ix >= 0 && iy >= 0 && iz >= 0) {
            const TI *src = base + ((long long)(iz * a.din[1] + iy) * a.din[0] + ix) * a.cin + ci;
            if constexpr (sizeof(TI) == 2) {
              pk = *reinterpret_cast<const uint4 *>(src);
            } else {
              const float4 f0 = *reinterpret_cast<const float4 *>(src);
              const float4 f1 = *reinterpret_cast<const float4 *>(src + 4);
              pk = make_uint4(pack_bf16(f0.x, f0.y), pack_bf16(f0.z, f0.w), pack_bf16(f1.x, f1.y),
                              pack_bf16(f1.z, f1.w));
            }
          }
        }
      } else {
        float xv[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
          const int kk = k + h;
          xv[h] = 0.f;
          if (live && kk < K) {
            const int tap = kk / a.cin, ci = kk - tap * a.cin;
            const int ix = tap_src(ox, tap % 3, a.stride, a.din[0], a.transposed);
            const int iy = tap_src(oy, (tap / 3) % 3, a.stride, a.din[1], a.transposed);
            const int iz = tap_src(oz, tap / 9, a.stride, a.din[2], a.transposed);
            if (ix >= 0 && iy >= 0 && iz >= 0)
              xv[h] = tof_any(base[((long long)(iz * a.din[1] + iy) * a.din[0] + ix) * a.cin + ci]);
          }
        }
        pk = make_uint4(pack_bf16(xv[0], xv[1]), pack_bf16(xv[2], xv[3]), pack_bf16(xv[4], xv[5]),
                        pack_bf16(xv[6], xv[7]));
      }
      *reinterpret_cast<uint4 *>(As + tc_off(tid, 8 * gq)) = pk;
    }
    // B: BN rows (output channels) x 64 k
    unsigned char *Bs = tsm + 2 * kTcABytes + buf * kTcBBytes;
    for (int e = tid; e < BN * (kTcKC / 8); e += 128) {
      const int n = e / (kTcKC / 8), gq = e - n * (kTcKC / 8), co = n0 + n;
      const int k = k0 + 8 * gq;
      uint4 pk = make_uint4(0u, 0u, 0u, 0u);
      if (bvec) {
        if (co < a.cout && k < K) pk = *reinterpret_cast<const uint4 *>(W + (long long)co * a.w_so + k);
      } else {
        unsigned short w[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
          const int kk = k + h;
          bf16 wv = __float2bfloat16_rn(0.f);
          if (co < a.cout && kk < K) {
            const int tap = kk / a.cin, ci = kk - tap * a.cin;
            wv = W[(long long)co * a.w_so + (long long)tap * a.w_sd + (long long)ci * a.w_si];
          }
          w[h] = __bfloat16_as_ushort(wv);
        }
        pk = make_uint4(w[0] | ((unsigned)w[1] << 16), w[2] | ((unsigned)w[3] << 16), w[4] | ((unsigned)w[5] << 16),
                        w[6] | ((unsigned)w[7] << 16));
      }
      *reinterpret_cast<uint4 *>(Bs + tc_off(n, 8 * gq)) = pk;
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const unsigned sa = smem_u32(As), sb = smem_u32(Bs);
#pragma unroll
      for (int ks = 0; ks < kTcKC / 16; ++ks)  // K = 16 per MMA: two core matrices along K
        tc_mma(tmem, tc_desc(sa + 256 * ks, 128, kTcSBO), tc_desc(sb + 256 * ks, 128, kTcSBO), IDESC,
               (i > 0 || ks > 0) ? 1u : 0u);
      tc_commit(&bar[buf]);
    }
    issued = i + 1;
  }
  // the last commit covers every MMA before it
  const int nch = kc1 - kc0;
  if (ok && issued > 0) ok = mbar_wait_bounded(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (tid == 0) atomicExch(&g_conv_timeout, 1);
    // MMAs still in flight write this CTA's tensor memory: wait (bounded) for them
    if (issued > 0) mbar_wait_bounded(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
  }
  tc_fence_after();
  // epilogue: thread tid holds row tid (TMEM lane), columns 0 .. BN - 1
  const long long vr = v0 + tid;
  const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);
#pragma unroll
  for (int c0 = 0; c0 < BN; c0 += 16) {
    float v[16];
    tc_ld16(trow + c0, v);
    tc_wait_ld();
    if (vr < total && nch > 0) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int co = n0 + c0 + j;
        if (co >= a.cout) continue;
        const float val = ok ? v[j] : __int_as_float(0x7fc00000);
        if (gridDim.z > 1) {
          part[(long long)blockIdx.z * total * a.cout + vr * a.cout + co] = val;
        } else {
          float y = val + (bias ? bias[co] : 0.f);
          if (a.relu) y = fmaxf(y, 0.f);
          TO *dst = out + vr * a.cout + co;
          if (a.accumulate) y += tof(*dst);
          put(dst, y);
        }
      }
    } else if (vr < total && gridDim.z > 1) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int co = n0 + c0 + j;
        if (co < a.cout) part[(long long)blockIdx.z * total * a.cout + vr * a.cout + co] = 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
  }
}

// Arguments of the weight gradient of a forward conv (wgrad_mma_kernel).
struct WgArgs {
  int ci, co;
  int din[3], dout[3];
  int stride;
};

// Tensor-core weight gradient: dW[c_out][k] += sum_v g[v][c_out] A[v][k] with
// A the forward im2col (k = tap * c_in + c_in index), a GEMM with the voxels
// as its reduction: mma.sync m16n8k16 BF16 -> FP32 on a 64 (c_out) x 64 (k)
// tile per CTA (2 x 2 warps of 32 x 32), 32 voxels per step, a range of
// voxels per CTA, FP32 atomics into dW at the end.  g is staged transposed
// ([c_out][v]) and A as [k][v] (both with 40-element rows).
constexpr int kWgTile = 64, kWgV = 32;

__global__ void __launch_bounds__(128) wgrad_mma_kernel(WgArgs a, long long total, long long chunk,
                                                        const float *__restrict__ g,
                                                        const bf16 *__restrict__ x,
                                                        float *__restrict__ dW) {
  __shared__ __align__(16) bf16 Gs[kWgTile * kMmaLd];
  __shared__ __align__(16) bf16 Xs[kWgTile * kMmaLd];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gq = lane >> 2, t4 = lane & 3;
  const int wm = warp >> 1, wn = warp & 1;
  const int K = 27 * a.ci;
  const int k0 = blockIdx.y * kWgTile, c0 = blockIdx.z * kWgTile;
  const int nvo = a.dout[0] * a.dout[1] * a.dout[2];
  const long long nvi = (long long)a.din[0] * a.din[1] * a.din[2];
  const bool xvec = a.ci % 8 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0.f;
  const long long va = (long long)blockIdx.x * chunk, vb = min(total, va + chunk);
  for (long long v0 = va; v0 < vb; v0 += kWgV) {
    __syncthreads();
    // G^T: [c_out][v], zero beyond c_out or the voxel range
    for (int e = tid; e < kWgTile * kWgV; e += 128) {
      const int co = e % kWgTile, v = e / kWgTile;
      const long long gv = v0 + v;
      float val = 0.f;
      if (gv < vb && c0 + co < a.co) val = g[gv * a.co + c0 + co];
      Gs[co * kMmaLd + v] = __float2bfloat16_rn(val);
    }
    // A^T: [k][v]; 8 consecutive k share a tap when c_in % 8 == 0
    for (int e = tid; e < (kWgTile / 8) * kWgV; e += 128) {
      const int v = e % kWgV, kq = e / kWgV, kb = k0 + 8 * kq;
      const long long gv = v0 + v;
      bf16 vals[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) vals[j] = __float2bfloat16_rn(0.f);
      if (gv < vb) {
        const long long b = gv / nvo;
        const int vo = (int)(gv - b * nvo);
        const int ox = vo % a.dout[0], oy = (vo / a.dout[0]) % a.dout[1], oz = vo / (a.dout[0] * a.dout[1]);
        const bf16 *base = x + b * nvi * a.ci;
        if (xvec && kb < K) {
          const int tap = kb / a.ci, ci = kb - tap * a.ci;
          const int ix = a.stride * ox + tap % 3 - 1, iy = a.stride * oy + (tap / 3) % 3 - 1,
                    iz = a.stride * oz + tap / 9 - 1;
          if (ix >= 0 && ix < a.din[0] && iy >= 0 && iy < a.din[1] && iz >= 0 && iz < a.din[2]) {
            const uint4 pk = *reinterpret_cast<const uint4 *>(
                base + ((long long)(iz * a.din[1] + iy) * a.din[0] + ix) * a.ci + ci);
            const bf16 *pv = reinterpret_cast<const bf16 *>(&pk);
#pragma unroll
            for (int j = 0; j < 8; ++j) vals[j] = pv[j];
          }
        } else if (!xvec) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int k = kb + j;
            if (k >= K) break;
            const int tap = k / a.ci, ci = k - tap * a.ci;
            const int ix = a.stride * ox + tap % 3 - 1, iy = a.stride * oy + (tap / 3) % 3 - 1,
                      iz = a.stride * oz + tap / 9 - 1;
            if (ix >= 0 && ix < a.din[0] && iy >= 0 && iy < a.din[1] && iz >= 0 && iz < a.din[2])
              vals[j] = base[((long long)(iz * a.din[1] + iy) * a.din[0] + ix) * a.ci + ci];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) Xs[(8 * kq + j) * kMmaLd + v] = vals[j];
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kWgV; ks += 16) {
      uint32_t af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const bf16 *r0 = Gs + (wm * 32 + mt * 16 + gq) * kMmaLd + ks + 2 * t4;
        const bf16 *r8 = r0 + 8 * kMmaLd;
        af[mt][0] = *reinterpret_cast<const uint32_t *>(r0);
        af[mt][1] = *reinterpret_cast<const uint32_t *>(r8);
        af[mt][2] = *reinterpret_cast<const uint32_t *>(r0 + 8);
        af[mt][3] = *reinterpret_cast<const uint32_t *>(r8 + 8);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const bf16 *bp = Xs + (wn * 32 + nt * 8 + gq) * kMmaLd + ks + 2 * t4;
        const uint32_t b0 = *reinterpret_cast<const uint32_t *>(bp);
        const uint32_t b1 = *reinterpret_cast<const uint32_t *>(bp + 8);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          float *c = acc[mt][nt];
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
              "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
              : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
              : "r"(af[mt][0]), "r"(af[mt][1]), "r"(af[mt][2]), "r"(af[mt][3]), "r"(b0), "r"(b1));
        }
      }
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int co = c0 + wm * 32 + mt * 16 + gq + 8 * hr;
      if (co >= a.co) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
          const int k = k0 + wn * 32 + nt * 8 + 2 * t4 + hc;
          if (k < K) atomicAdd(&dW[(long long)co * K + k], acc[mt][nt][2 * hr + hc]);
        }
    }
}

// db[c_out] += sum_v g[v][c_out]: one thread per channel and voxel range
__global__ void bias_grad_kernel(int co, long long total, long long chunk, const float *__restrict__ g,
                                 float *__restrict__ db) {
  const int c = threadIdx.x;
  if (c >= co) return;
  const long long va = (long long)blockIdx.x * chunk, vb = min(total, va + chunk);
  float s = 0.f;
  for (long long v = va; v < vb; ++v) s += g[v * co + c];
  atomicAdd(&db[c], s);
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
// slices, splits * total * cout <= (4 + 2) * kSMs * 128 * 64 floats
// (kSplitScratch), since a split grid has fewer than 2 * kSMs blocks of at
// most 128 voxels x 64 channels.
constexpr int kSMs = 152;
constexpr long long kSplitScratch = (4LL + 2LL) * kSMs * 128 * 64;

// tensor-core path (output channels >= 16): BN = 16, 32 or 64 channels per CTA
template <typename TI, typename TO, int BN>
void launch_conv_tc(dim3 grid, const ConvArgs &a, long long total, int per, const TI *in, const bf16 *W,
                    const float *bias, TO *out, float *part, cudaStream_t s) {
  CKN(cudaFuncSetAttribute(conv_tc_kernel<TI, TO, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
  conv_tc_kernel<TI, TO, BN><<<grid, 128, kTcSmem, s>>>(a, total, per, in, W, bias, out, part);
}

template <typename TI, typename TO>
void run_conv_mma(const ConvArgs &a, int batch, const TI *in, const bf16 *W, const float *bias,
                  TO *out, float *part, cudaStream_t s) {
  const long long total = (long long)batch * a.dout[0] * a.dout[1] * a.dout[2];
  const int bn = a.cout <= 16 ? 16 : (a.cout <= 32 ? 32 : 64);
  const long long bxy = (long long)grid1(total, kTcBM) * ((a.cout + bn - 1) / bn);
  const int nkc = (27 * a.cin + kTcKC - 1) / kTcKC;
  int splits = 1;
  if (bxy < 2 * kSMs) splits = (int)std::min<long long>(nkc, (4 * kSMs + bxy - 1) / bxy);
  const int per = (nkc + splits - 1) / splits;
  splits = (nkc + per - 1) / per;
  if (splits > 1 && (long long)splits * total * a.cout > kSplitScratch)
    throw std::runtime_error("conv split scratch too small");
  dim3 grid(grid1(total, kTcBM), (a.cout + bn - 1) / bn, splits);
  if (bn == 16) launch_conv_tc<TI, TO, 16>(grid, a, total, per, in, W, bias, out, part, s);
  else if (bn == 32) launch_conv_tc<TI, TO, 32>(grid, a, total, per, in, W, bias, out, part, s);
  else launch_conv_tc<TI, TO, 64>(grid, a, total, per, in, W, bias, out, part, s);
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

template <typename TI, typename TO, int OT, int IC>
void run_conv(const ConvArgs &a, int batch, const TI *in, const bf16 *W, const float *bias, TO *out,
              float *part, cudaStream_t s) {
  static_assert(OT <= 16, "split scratch bound assumes at most 16 channels per block");
  if (OT == 16 && a.cout >= 16) {
    run_conv_mma<TI, TO>(a, batch, in, W, bias, out, part, s);
    return;
  }
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
  {
    // tensor cores: 64 x 64 tiles of dW (rows beyond c_out are zero), voxel
    // ranges to fill ~4 CTAs per SM
    const int kt = (27 * L.cin + kWgTile - 1) / kWgTile, ct = (L.cout + kWgTile - 1) / kWgTile;
    long long blocks = std::max(1LL, std::min((total + kWgV - 1) / kWgV,
                                              (long long)(4 * kSMs / (kt * ct)) + 1));
    long long chunk = (total + blocks - 1) / blocks;
    chunk = (chunk + kWgV - 1) / kWgV * kWgV;
    blocks = (total + chunk - 1) / chunk;
    wgrad_mma_kernel<<<dim3((unsigned)blocks, kt, ct), 128, 0, n->stream>>>(
        a, total, chunk, gout, in, n->grad + L.woff);
    CKN(cudaGetLastError());
    const int bb = (int)std::min<long long>(4 * kSMs, (total + 255) / 256);
    const long long bc = (total + bb - 1) / bb;
    bias_grad_kernel<<<(unsigned)((total + bc - 1) / bc), ((L.cout + 31) / 32) * 32, 0, n->stream>>>(
        L.cout, total, bc, gout, n->grad + L.boff);
    CKN(cudaGetLastError());
    rmd::add_launches(2);
  }
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

int conv_timeouts(cudaError_t *err) {
  int v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_conv_timeout, sizeof(int));
  if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_conv_timeout, &zero, sizeof(int));
  if (err) *err = e;
  return e == cudaSuccess ? v : 0;
}
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
