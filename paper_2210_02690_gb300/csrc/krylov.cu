// FP64 vector kernels of the flexible GMRES driver (Sec. 3: GMRES iterations
// preconditioned by the V-cycle).  Orthogonalisation uses classical
// Gram-Schmidt applied twice (one fused pass computes all inner products of a
// step); reductions use a fixed grid and a fixed order, so results are
// reproducible run to run.
#include "common.cuh"
#include "kernels.cuh"

namespace stg {
namespace {

constexpr int kDotBlocks = 1216;  // 8 x 152 SMs
constexpr int kMaxVec = 32;

// Inner products of w with the m columns of V; each block writes its partial sums.  MV (>= m)
// sizes the per-thread accumulators, so short bases keep the register count (and with it the
// number of loads in flight per SM) where a long basis would not.  The per-element order of
// the sums does not depend on MV.
template <int MV>
__global__ void __launch_bounds__(256) multi_dot_partial(long long n, int m, const double* __restrict__ V,
                                                         long long ldv, const double* __restrict__ w,
                                                         double* __restrict__ partial) {
  double acc[MV];
#pragma unroll
  for (int i = 0; i < MV; ++i) acc[i] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; t + stride < n; t += 2 * stride) {  // two independent elements per pass
    const double w0 = w[t], w1 = w[t + stride];
#pragma unroll
    for (int i = 0; i < MV; ++i)
      if (i < m) acc[i] += V[i * ldv + t] * w0 + V[i * ldv + t + stride] * w1;
  }
  for (; t < n; t += stride) {
    const double wt = w[t];
#pragma unroll
    for (int i = 0; i < MV; ++i)
      if (i < m) acc[i] += V[i * ldv + t] * wt;
  }
  __shared__ double red[8][kMaxVec];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < MV; ++i) {
    if (i >= m) break;
    double v = acc[i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[wid][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < m) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][threadIdx.x];
    partial[(long long)blockIdx.x * kMaxVec + threadIdx.x] = s;
  }
}

__global__ void multi_dot_final(int m, int nblocks, const double* __restrict__ partial, double* __restrict__ h) {
  const int i = blockIdx.x;
  if (i >= m) return;
  __shared__ double red[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(long long)b * kMaxVec + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) h[i] = red[0];
}

__global__ void multi_axpy_kernel(long long n, int m, const double* __restrict__ V, long long ldv,
                                  const double* __restrict__ h, double sign, double* __restrict__ w) {
  __shared__ double hs[kMaxVec];
  if (threadIdx.x < m) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double s = 0.0;
  for (int i = 0; i < m; ++i) s += hs[i] * V[i * ldv + t];
  w[t] += sign * s;
}

__global__ void axpby_kernel(long long n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = a * x[t] + (b == 0.0 ? 0.0 : b * y[t]);
}

}  // namespace

void multi_dot(long long n, int m, const double* V, long long ldv, const double* w, double* partial, double* h,
               cudaStream_t st) {
  if (m > kMaxVec) throw Error{STG_EINVAL, "too many vectors in one orthogonalisation step"};
  // chunks of at most 8 vectors per launch (79 registers a thread); a vector's sum is the same
  // whichever chunk carries it
  for (int c = 0; c < m; c += 8) {
    const int mc = m - c < 8 ? m - c : 8;
    if (mc <= 4)
      multi_dot_partial<4><<<kDotBlocks, 256, 0, st>>>(n, mc, V + c * ldv, ldv, w, partial + c);
    else
      multi_dot_partial<8><<<kDotBlocks, 256, 0, st>>>(n, mc, V + c * ldv, ldv, w, partial + c);
    STG_LAUNCH_OK();
  }
  multi_dot_final<<<m, 256, 0, st>>>(m, kDotBlocks, partial, h);
  STG_LAUNCH_OK();
}

void multi_axpy_sub(long long n, int m, const double* V, long long ldv, const double* h, double* w, cudaStream_t st) {
  multi_axpy_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, m, V, ldv, h, -1.0, w);
  STG_LAUNCH_OK();
}

void multi_axpy_add(long long n, int m, const double* Z, long long ldz, const double* y, double* x, cudaStream_t st) {
  multi_axpy_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, m, Z, ldz, y, 1.0, x);
  STG_LAUNCH_OK();
}

void axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t st) {
  launch_k(axpby_kernel, grid_for(n, 256), 256, 0, st, n, a, x, b, y);
}

size_t dot_partial_doubles() { return (size_t)kDotBlocks * kMaxVec; }

}  // namespace stg
