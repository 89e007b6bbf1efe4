// Convolutional coarse corrector: a small 3D U-Net on the vertex grid of
// the p = 1 coarse space, with hand-written BF16 forward and backward
// kernels (FP32 accumulation) and an Adam optimiser (learned.cu).
//
// Architecture (levels L, width C, input channels c_in, grid D_0 = dims):
//   level l has the grid D_l = (D_{l-1} - 1) / 2 + 1 and C_l = C 2^l channels
//   e0a = relu(conv(x))             c_in -> C_0      (stride 1)
//   e0  = relu(conv(e0a))           C_0  -> C_0
//   for l = 1..L:  d_l = relu(conv_2(e_{l-1}))  C_{l-1} -> C_l  (stride 2)
//                  e_l = relu(conv(d_l))        C_l -> C_l
//   h_L = e_L
//   for l = L-1..0: u_l  = up(h_{l+1})          vertex-centred linear interpolation
//                   a_l  = relu(conv(u_l))      C_{l+1} -> C_l
//                   s_l  = a_l + e_l            skip connection
//                   h_l  = relu(conv(s_l))      C_l -> C_l
//   y = conv(h_0)                   C_0 -> 1 (no activation, FP32 output)
// Every conv is 3x3x3 with zero padding; a stride-2 conv reads the input at
// 2 o + d - 1.  Parameters, in this order, one conv after another: W[co][27][ci]
// (tap d = (dz * 3 + dy) * 3 + dx for the offset (dx-1, dy-1, dz-1)), then b[co].
// Tensors are channels-last, [batch][voxel][channel], voxel = (z * ny + y) * nx + x.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rmn {

struct Net;

struct NetSpec {
  int dims[3];    // grid of level 0 (each (dims - 1) divisible by 2^levels)
  int levels;     // 0..4
  int width;      // C_0
  int in_ch;      // input channels
  int max_batch;  // buffers are sized for this many samples
};

// All functions throw std::runtime_error on a CUDA error or a bad argument.
Net *create(const NetSpec &s, uint64_t seed, cudaStream_t stream);
void destroy(Net *net);
const NetSpec &spec(const Net *net);
long long num_params(const Net *net);
void get_params(const Net *net, float *host);
void set_params(Net *net, const float *host);
// x: device [batch][V0][in_ch] FP32, y: device [batch][V0] FP32
void forward(Net *net, int batch, const float *x, float *y);
// After forward(): parameter gradients of sum(dy * y) (FP32, device, in
// the parameter order) and, if dx != NULL, the input gradient.
void backward(Net *net, const float *dy, float *dx);
// 1 if a tensor-core convolution gave up a bounded wait since the last call
// (its outputs are NaN; the flag is cleared), 0 otherwise; a CUDA error code
// in *err when reading the flag fails
int conv_timeouts(cudaError_t *err);
float *grads(Net *net);
// Adam (Kingma & Ba) on the FP32 master weights; refreshes the BF16 copy.
void adam(Net *net, float lr, float beta1, float beta2, float eps);
// Mean squared error over the masked voxels: loss += sum_b sum_v m_v (y - t)^2 * scale,
// dy = 2 m_v (y - t) * scale.  loss: device double (accumulated).
void mse(int batch, int nvox, const float *y, const float *t, const uint8_t *mask, float scale,
         float *dy, double *loss, cudaStream_t s);
// Coarse-corrector glue.  Coarse free DOF f sits at grid voxel free2lat[f];
// lat2free[v] = -1 on Dirichlet vertices.
// x[v][0] = sqrt(nc) cc[lat2free[v]] / sqrt(scal[0]) (0 on Dirichlet), x[v][1] = logal[v]
void corr_pack(int nc, long long nvox, const double *cc, const int *lat2free, const float *logal,
               const double *scal, float *x, cudaStream_t s);
// cl[f] = y[free2lat[f]]
void corr_gather(int nc, const float *y, const int *free2lat, double *cl, cudaStream_t s);
// ce = (scal[1] / scal[2]) cl if scal[2] > 0, else 0 (the A_0-energy optimal step along cl)
void corr_scale(int nc, const double *cl, const double *scal, double *ce, cudaStream_t s);
// out = sqrt(nc) v / sqrt(scal[0]) in FP32 (0 if scal[0] = 0)
void corr_normalise(int nc, const double *v, const double *scal, float *out, cudaStream_t s);
// Training batch: for b < batch, pair j = idx[b]:
// x[b][v][0] = R[j][lat2free[v]], x[b][v][1] = logal[v], t[b][v] = T[j][lat2free[v]] (0 on Dirichlet)
void corr_batch(int batch, int nc, long long nvox, const int *idx, const float *R, const float *T,
                const int *lat2free, const float *logal, float *x, float *t, cudaStream_t s);

}  // namespace rmn
