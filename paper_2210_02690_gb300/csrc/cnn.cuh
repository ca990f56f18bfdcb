// Warm-start network: a stack of 3x3 convolutions (zero padding, bias, tanh after
// every layer but the last) on the Q2 node grid of a 2D slab, trained in FP32 by
// mean-squared error and Adam.  All tensors are NCHW float arrays in device memory.
#pragma once

#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

struct stg_cnn {
  int L = 0;                 // layers
  int ch[9] = {};            // channels[0..L]
  int H = 0, W = 0, max_batch = 0;
  cudaStream_t st = nullptr;
  long long n_params = 0;
  std::vector<long long> off;  // offset of layer l's weights; bias follows at off[l] + ch[l+1]*ch[l]*9
  float* params = nullptr;
  float* grad = nullptr;
  float* m = nullptr;          // Adam moments
  float* v = nullptr;
  long long adam_t = 0;
  float* act[9] = {};          // act[0]: gathered input batch; act[l]: output of layer l
  float* g0 = nullptr;         // gradient ping-pong buffers, max_batch * max channels * H * W
  float* g1 = nullptr;
  float* tgt = nullptr;        // gathered target batch
  float* part = nullptr;       // per-tile weight-gradient partials
  long long part_floats = 0;
  double* loss_part = nullptr;  // per-block squared-error partials
  double* loss_dev = nullptr;   // one loss per training step
  int* idx = nullptr;           // sample indices of the training steps
  long long idx_cap = 0;
  std::string err;
};

namespace stg {

// Forward pass of `batch` samples x[batch][ch0][H][W] on stream st; returns the device
// pointer of the output (the network's own buffer act[L], valid until the next call).
const float* cnn_forward(stg_cnn* n, const float* x, int batch, cudaStream_t st);

// Warm-start packing kernels on the finest level of a 2D slab problem (C-ABI vectors).
void warm_features(const Geom& g, const double* Xn, const double* Xm, float sv, float sd, float* feat,
                   cudaStream_t st);
void warm_target(const Geom& g, const TimeData& td, const double* Xn, const double* Xm, const double* Xp, float sd,
                 float* tgt, cudaStream_t st);
void warm_guess(const Geom& g, const TimeData& td, const double* Xn, const double* Xm, const float* y, float sd,
                double* X0, cudaStream_t st);

// Sums of |v_n(t_n)|^2 and |v_n(t_n) - v_{n-1}(t_{n-1})|^2 over the nodal velocity entries into
// part[512], part[513] (part: 514 doubles of scratch).
void warm_sums(const Geom& g, const double* Xn, const double* Xm, double* part, cudaStream_t st);

}  // namespace stg
