// Allocation-free batched inverse of caller-supplied local matrices.
//
// Some callers cannot call cudaMalloc at the point where they need local
// inverses: host applications and frameworks that own the GPU's memory and
// hand it out only from their own pools or arenas (a stray cudaMalloc there
// fails once the pool holds the memory, or breaks the host's accounting), and
// real-time loops that forbid allocation after start-up because cudaMalloc and
// cudaFree may synchronise the device and take unbounded time.  stg_setup
// allocates everything a context needs, so it is not usable there.  This entry
// point needs no context: the caller passes the matrices and the output
// buffer, and the Gauss-Jordan working copies live in a fixed array compiled
// into the library.
//
// The kernel is a variant of the patch-inversion kernel of the smoother set-up
// (same in-place Gauss-Jordan elimination with partial pivoting, first maximal
// pivot, columns swapped back at the end); it reads dense row-major matrices
// instead of gathering J_K from an assembled operator, and its working matrix
// is always the static scratch array.
#include <string>

#include "common.cuh"

namespace stg {

void set_global_error(const std::string& msg);

namespace {

constexpr int kNoAllocMaxN = 256;
constexpr long long kNoAllocScratchDoubles = 1LL << 20;  // 1 Mi doubles = 8 MiB per device
constexpr int kMaxDevices = 64;

// Working matrices of the in-flight batch; held by every GPU that loads the library.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];
// Lowest index of a singular matrix in the current call (all bits set = none); set to
// all ones at the start of every call, lowered by atomicMin.
static __device__ __align__(256) unsigned long long g_noalloc_status[4];

// Device addresses of the two arrays, looked up once per device.
double* g_scratch_ptr[kMaxDevices];
unsigned long long* g_status_ptr[kMaxDevices];
bool g_ready[kMaxDevices];

__global__ void __launch_bounds__(256) invert_dense_kernel(int n, long long p0, const double* __restrict__ a,
                                                           double* __restrict__ a_inv, double* work,
                                                           unsigned long long* status) {
  const long long p = p0 + blockIdx.x;
  double* A = work + (long long)blockIdx.x * n * n;
  __shared__ double colj[kNoAllocMaxN];
  __shared__ int perm[kNoAllocMaxN];
  __shared__ int s_piv, s_fail;
  __shared__ double s_pval;
  const int tid = threadIdx.x, nth = blockDim.x;
  const double* src = a + p * n * n;
  for (int t = tid; t < n * n; t += nth) A[t] = src[t];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid < 32) {
      double best = -1.0;
      int bi = n;
      for (int i = j + tid; i < n; i += 32) {
        const double v = fabs(A[i * n + j]);
        if (v > best || (v == best && i < bi)) {
          best = v;
          bi = i;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        s_piv = bi;
        const double pv = bi < n ? A[bi * n + j] : 0.0;
        s_pval = pv;
        if (!(fabs(pv) > 0.0) || isinf(pv)) s_fail = 1;
        perm[j] = bi;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const int pr = s_piv;
    if (pr != j)
      for (int l = tid; l < n; l += nth) {
        const double t = A[j * n + l];
        A[j * n + l] = A[pr * n + l];
        A[pr * n + l] = t;
      }
    __syncthreads();
    for (int i = tid; i < n; i += nth) colj[i] = A[i * n + j];
    __syncthreads();
    const double inv = 1.0 / s_pval;
    for (int l = tid; l < n; l += nth) A[j * n + l] = (l == j ? 1.0 : A[j * n + l]) * inv;
    __syncthreads();
    for (int t = tid; t < n * n; t += nth) {
      const int i = t / n, l = t - i * n;
      if (i == j) continue;
      A[t] = (l == j ? 0.0 : A[t]) - colj[i] * A[j * n + l];
    }
    __syncthreads();
  }
  double* dst = a_inv + p * n * n;
  if (s_fail) {
    if (tid == 0) atomicMin(status, (unsigned long long)p);
    for (int t = tid; t < n * n; t += nth) dst[t] = 0.0;
    return;
  }
  for (int j = n - 1; j >= 0; --j) {
    const int pj = perm[j];
    if (pj != j)
      for (int i = tid; i < n; i += nth) {
        const double t = A[i * n + j];
        A[i * n + j] = A[i * n + pj];
        A[i * n + pj] = t;
      }
    __syncthreads();
  }
  for (int t = tid; t < n * n; t += nth) dst[t] = A[t];
}

}  // namespace
}  // namespace stg

extern "C" stg_status stg_invert_local_noalloc(int n, long long count, const double* a, double* a_inv,
                                               void* stream) {
  using namespace stg;
  if (n < 1 || n > kNoAllocMaxN) {
    set_global_error("stg_invert_local_noalloc: n = " + std::to_string(n) + " is outside 1.." +
                     std::to_string(kNoAllocMaxN));
    return STG_EINVAL;
  }
  if (count < 0 || (count > 0 && (!a || !a_inv))) {
    set_global_error("stg_invert_local_noalloc: negative count or null buffer");
    return STG_EINVAL;
  }
  if (count == 0) return STG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_global_error(std::string("stg_invert_local_noalloc: no usable current device: ") + cudaGetErrorString(e));
    return STG_ECUDA;
  }
  if (!g_ready[dev]) {
    // In host code the array names are host-side stand-ins; the kernel needs the device addresses.
    e = cudaGetSymbolAddress((void**)&g_scratch_ptr[dev], g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&g_status_ptr[dev], g_noalloc_status);
    if (e != cudaSuccess) {
      set_global_error(std::string("stg_invert_local_noalloc: cudaGetSymbolAddress failed: ") +
                       cudaGetErrorString(e));
      return STG_ECUDA;
    }
    g_ready[dev] = true;
  }
  double* work = g_scratch_ptr[dev];
  unsigned long long* status = g_status_ptr[dev];
  // the array keeps the previous call's value: reset it to "none" (all bits set)
  e = cudaMemsetAsync(status, 0xff, sizeof(unsigned long long), st);
  const long long slots = kNoAllocScratchDoubles / ((long long)n * n);
  for (long long p0 = 0; e == cudaSuccess && p0 < count; p0 += slots) {
    const long long cnt = count - p0 < slots ? count - p0 : slots;
    invert_dense_kernel<<<(unsigned)cnt, 256, 0, st>>>(n, p0, a, a_inv, work, status);
    e = cudaGetLastError();
  }
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_global_error(std::string("stg_invert_local_noalloc: ") + cudaGetErrorString(e));
    return STG_ECUDA;
  }
  if (h != ~0ULL) {
    set_global_error("stg_invert_local_noalloc: matrix " + std::to_string(h) + " has a zero pivot");
    return STG_ESINGULAR;
  }
  return STG_OK;
}
