// Direct solver for the coarsest level (Sec. 3: a direct solver for J_0 d_0 = b_0 on T_0).
//
// The paper uses a parallel sparse direct solver on a CPU cluster.  Here the
// structure of the box mesh is used instead of a general sparse LU:
//   * unknowns are grouped along x into vertex planes V_s (Q2 nodes with even x
//     index 2s) and interior slabs I_s (Q2 nodes with x index 2s+1 plus the
//     pressure of the cells of cell column s).  I_s couples only to V_s and
//     V_{s+1}, so J_0 = [[A_VV, A_VI], [A_IV, A_II]] with block-diagonal A_II;
//   * the interiors are eliminated in parallel (dense Gauss-Jordan inverses with
//     partial pivoting, one CTA per slab): S = A_VV - A_VI A_II^{-1} A_IV is block
//     tridiagonal over the vertex planes;
//   * S is factored by block cyclic reduction (log2 of the plane count levels,
//     each a batch of independent dense inverses and products).
// Everything is FP64.  With Dirichlet data on the whole boundary J_0 has one
// constant-pressure null vector per Radau node; the pressure coefficient 0 of
// cell 0 is then fixed to zero at every Radau node (its row and column become
// identity rows), which yields the solution with that value for consistent b.
// An obstacle (2D) splits the cell columns it crosses into a piece below and a
// piece above it; each piece's interior block has its own constant-pressure null
// vector, so the cell-constant coefficient of the first cell above the obstacle
// joins V_s as well (a second group of nt slots in every vertex plane, identity
// rows where unused); removed cells' pressures are identity rows.
#include <algorithm>
#include <vector>

#include "coarse.cuh"
#include "kernels.cuh"

namespace stg {

namespace {

// ---------------------------------------------------------------- batched dense kernels
// In-place Gauss-Jordan inverse with partial pivoting; one CTA per matrix.  With
// SMEM the matrix is copied into shared memory first (when it fits).  Each
// pivot step has three phases separated by barriers: pivot search (one warp);
// row interchange, saved pivot column and scaled pivot row (all threads, from
// the values before the interchange); rank-one update of the other rows.
template <typename T, bool SMEM>
__global__ void __launch_bounds__(1024) bgj_kernel(int m, T* const* As, int* status) {
  T* G = As[blockIdx.x];
  extern __shared__ __align__(16) unsigned char sh_raw[];
  T* A = SMEM ? reinterpret_cast<T*>(sh_raw) : G;
  T* colj = SMEM ? A + (long long)m * m : reinterpret_cast<T*>(sh_raw);
  int* perm = reinterpret_cast<int*>(colj + m);
  __shared__ int s_piv, s_fail;
  __shared__ T s_pval, s_ajj;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int w = tid >> 5, ln = tid & 31, nw = nth >> 5;
  if (tid == 0) s_fail = 0;
  if (SMEM)
    for (long long t = tid; t < (long long)m * m; t += nth) A[t] = G[t];
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (tid < 32) {
      T best = -1;
      int bi = m;
      for (int i = j + tid; i < m; i += 32) {
        const T v = fabs(A[(long long)i * m + j]);
        if (v > best || (v == best && i < bi)) {
          best = v;
          bi = i;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const T ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        s_piv = bi;
        const T pv = bi < m ? A[(long long)bi * m + j] : (T)0;
        s_pval = pv;
        s_ajj = A[(long long)j * m + j];
        if (!(fabs(pv) > (T)0) || isinf(pv)) s_fail = 1;
        perm[j] = bi;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const int pr = s_piv;
    const T inv = (T)1 / s_pval;
    // column j of every row before the interchange (rows j and pr swap their entries)
    for (int i = tid; i < m; i += nth)
      colj[i] = i == j ? s_pval : (i == pr ? s_ajj : A[(long long)i * m + j]);
    // interchange rows j and pr, scale the new pivot row
    for (int l = tid; l < m; l += nth) {
      const T vj = A[(long long)j * m + l], vp = A[(long long)pr * m + l];
      A[(long long)j * m + l] = l == j ? inv : vp * inv;
      if (pr != j) A[(long long)pr * m + l] = vj;
    }
    __syncthreads();
    {
      const T* rj = A + (long long)j * m;
      for (int i = w; i < m; i += nw) {
        if (i == j) continue;
        const T f = colj[i];
        T* ri = A + (long long)i * m;
        for (int l = ln; l < m; l += 32) ri[l] = (l == j ? (T)0 : ri[l]) - f * rj[l];
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) atomicCAS(status, 0, 1 + (int)blockIdx.x);
    return;
  }
  for (int j = m - 1; j >= 0; --j) {
    const int pj = perm[j];
    if (pj != j)
      for (int i = tid; i < m; i += nth) {
        const T t = A[(long long)i * m + j];
        A[(long long)i * m + j] = A[(long long)i * m + pj];
        A[(long long)i * m + pj] = t;
      }
    __syncthreads();
  }
  if (SMEM)
    for (long long t = tid; t < (long long)m * m; t += nth) G[t] = A[t];
}

// Gauss-Jordan for matrices too large for shared memory: each pivot step is two launches over
// the whole batch, so the rank-one updates (O(m^2) per step) spread over all SMs instead of one
// CTA per matrix.  Same operations and order as bgj_kernel (first maximal pivot, saved pivot
// column, row interchange, scaled pivot row, update, columns swapped back at the end).
template <typename T>
__global__ void __launch_bounds__(256) gj_pivot_kernel(int m, int j, T* const* As, T* __restrict__ col,
                                                       int* __restrict__ perm, int* __restrict__ fail) {
  const int b = blockIdx.x, tid = threadIdx.x;
  if (fail[b]) return;
  T* A = As[b];
  T* cj = col + (long long)b * m;
  __shared__ T s_best[256];
  __shared__ int s_idx[256];
  __shared__ int s_pr, s_bad;
  __shared__ T s_pv, s_ajj;
  T best = -1;
  int bi = m;
  for (int i = j + tid; i < m; i += blockDim.x) {
    const T v = fabs(A[(long long)i * m + j]);
    if (v > best || (v == best && i < bi)) {
      best = v;
      bi = i;
    }
  }
  s_best[tid] = best;
  s_idx[tid] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) {
      const T ob = s_best[tid + w];
      const int oi = s_idx[tid + w];
      if (ob > s_best[tid] || (ob == s_best[tid] && oi < s_idx[tid])) {
        s_best[tid] = ob;
        s_idx[tid] = oi;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    const int pr = s_idx[0];
    const T pv = pr < m ? A[(long long)pr * m + j] : (T)0;
    s_pr = pr;
    s_pv = pv;
    s_ajj = A[(long long)j * m + j];
    s_bad = (!(fabs(pv) > (T)0) || isinf(pv)) ? 1 : 0;
    if (s_bad) fail[b] = 1;
    perm[(long long)b * m + j] = pr;
  }
  __syncthreads();
  if (s_bad) return;
  const int pr = s_pr;
  const T inv = (T)1 / s_pv;
  for (int i = tid; i < m; i += blockDim.x) cj[i] = i == j ? s_pv : (i == pr ? s_ajj : A[(long long)i * m + j]);
  __syncthreads();
  for (int l = tid; l < m; l += blockDim.x) {
    const T vj = A[(long long)j * m + l], vp = A[(long long)pr * m + l];
    A[(long long)j * m + l] = l == j ? inv : vp * inv;
    if (pr != j) A[(long long)pr * m + l] = vj;
  }
}

// A[i][l] = (l == j ? 0 : A[i][l]) - col[i] A[j][l] for all i != j; 32 columns x 32 rows a block
template <typename T>
__global__ void __launch_bounds__(256) gj_update_kernel(int m, int j, T* const* As, const T* __restrict__ col,
                                                        const int* __restrict__ fail) {
  const int b = blockIdx.z;
  if (fail[b]) return;
  T* A = As[b];
  const T* cj = col + (long long)b * m;
  const int l = blockIdx.x * 32 + (threadIdx.x & 31);
  if (l >= m) return;
  const T rj = A[(long long)j * m + l];
  const int i0 = blockIdx.y * 32 + (threadIdx.x >> 5);
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + 8 * r;
    if (i >= m || i == j) continue;
    T* ai = A + (long long)i * m + l;
    *ai = (l == j ? (T)0 : *ai) - cj[i] * rj;
  }
}

// Blocked Gauss-Jordan for the large blocks: the same pivots and operations as gj_pivot_kernel /
// gj_update_kernel, arranged by panels of w columns [c0, c0 + w).  Within a panel every step
// (first maximal pivot among the rows not yet used, row interchange, scaled pivot row, update)
// runs on the m x w panel in shared memory; the other columns are updated once per panel:
// with P the panel's pivot rows, Q the panel columns and C the others, w Gauss-Jordan steps turn
// A_PC into A_PQ^{-1} A_PC and A_RC into A_RC - A_RQ A_PQ^{-1} A_PC, i.e.
//   A[:, C] = [0 on rows P; A_RC] + panel_new A_PC_old,
// one batched product (panel_new is the m x w panel after its steps: A_PQ^{-1} on rows P and
// -A_RQ A_PQ^{-1} on the others).  3 launches per panel instead of 2 per column.
template <typename T>
__global__ void __launch_bounds__(1024) gjb_panel_kernel(int m, int c0, int w, T* const* As, T* const* Ps,
                                                         int* __restrict__ perm, long long pstride,
                                                         int* __restrict__ fail) {
  const int b = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  if (fail[b]) return;
  T* A = As[b];
  extern __shared__ __align__(16) unsigned char sh_raw[];
  const int ld = w + 1;  // padded row stride: a panel column read across rows spreads over the banks
  T* P = reinterpret_cast<T*>(sh_raw);
  T* colj = P + (long long)m * ld;
  __shared__ T s_best[32];
  __shared__ int s_idx[32];
  __shared__ int s_pr, s_bad;
  __shared__ T s_pv;
  for (long long t = tid; t < (long long)m * w; t += nth) {
    const int i = (int)(t / w), l = (int)(t - (long long)i * w);
    P[i * ld + l] = A[(long long)i * m + c0 + l];
  }
  __syncthreads();
  for (int jj = 0; jj < w; ++jj) {
    const int j = c0 + jj;
    T best = -1;
    int bi = m;
    for (int i = j + tid; i < m; i += nth) {
      const T v = fabs(P[i * ld + jj]);
      if (v > best || (v == best && i < bi)) {
        best = v;
        bi = i;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const T ob = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if ((tid & 31) == 0) {
      s_best[tid >> 5] = best;
      s_idx[tid >> 5] = bi;
    }
    __syncthreads();
    if (tid < 32) {
      best = tid < (nth >> 5) ? s_best[tid] : (T)-1;
      bi = tid < (nth >> 5) ? s_idx[tid] : m;
      for (int off = 16; off > 0; off >>= 1) {
        const T ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        const T pv = bi < m ? P[bi * ld + jj] : (T)0;
        s_pr = bi;
        s_pv = pv;
        s_bad = (!(fabs(pv) > (T)0) || isinf(pv)) ? 1 : 0;
        if (s_bad) fail[b] = 1;
        perm[(long long)b * pstride + j] = bi;
      }
    }
    __syncthreads();
    if (s_bad) return;  // block-uniform; the matrix is reported by gj_unpermute_kernel
    const int pr = s_pr;
    if (pr != j)
      for (int l = tid; l < w; l += nth) {
        const T t = P[j * ld + l];
        P[j * ld + l] = P[pr * ld + l];
        P[pr * ld + l] = t;
      }
    __syncthreads();
    const T inv = (T)1 / s_pv;
    for (int i = tid; i < m; i += nth) colj[i] = P[i * ld + jj];
    __syncthreads();
    for (int l = tid; l < w; l += nth) P[j * ld + l] = (l == jj ? (T)1 : P[j * ld + l]) * inv;
    __syncthreads();
    for (long long t = tid; t < (long long)m * w; t += nth) {
      const int i = (int)(t / w), l = (int)(t - (long long)i * w);
      if (i == j) continue;
      P[i * ld + l] = (l == jj ? (T)0 : P[i * ld + l]) - colj[i] * P[j * ld + l];
    }
    __syncthreads();
  }
  T* pn = Ps[b];
  for (long long t = tid; t < (long long)m * w; t += nth) {
    const int i = (int)(t / w), l = (int)(t - (long long)i * w);
    const T v = P[i * ld + l];
    A[(long long)i * m + c0 + l] = v;
    pn[t] = v;
  }
}

// The panel's row interchanges applied to the other columns (in order), then the pivot rows'
// old values of the other columns saved (zero in the panel's own columns) and cleared in A.
template <typename T>
__global__ void __launch_bounds__(256) gjb_swap_save_kernel(int m, int c0, int w, T* const* As, T* const* Os,
                                                            const int* __restrict__ perm, long long pstride,
                                                            const int* __restrict__ fail) {
  const int b = blockIdx.y;
  if (fail[b]) return;
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= m) return;
  T* A = As[b];
  T* O = Os[b];
  const bool panel = l >= c0 && l < c0 + w;
  if (!panel)
    for (int t = 0; t < w; ++t) {
      const int j = c0 + t, pr = perm[(long long)b * pstride + j];
      if (pr != j) {
        const T x = A[(long long)j * m + l];
        A[(long long)j * m + l] = A[(long long)pr * m + l];
        A[(long long)pr * m + l] = x;
      }
    }
  for (int t = 0; t < w; ++t) {
    T* a = A + (long long)(c0 + t) * m + l;
    O[(long long)t * m + l] = panel ? (T)0 : *a;
    if (!panel) *a = (T)0;
  }
}

// columns swapped back (last interchange first); the status records the first failed matrix
template <typename T>
__global__ void __launch_bounds__(1024) gj_unpermute_kernel(int m, T* const* As, const int* __restrict__ perm,
                                                            const int* __restrict__ fail, int* status) {
  const int b = blockIdx.x;
  if (fail[b]) {
    if (threadIdx.x == 0) atomicCAS(status, 0, 1 + b);
    return;
  }
  T* A = As[b];
  const int* pm = perm + (long long)b * m;
  for (int j = m - 1; j >= 0; --j) {
    const int pj = pm[j];
    if (pj != j)
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const T t = A[(long long)i * m + j];
        A[(long long)i * m + j] = A[(long long)i * m + pj];
        A[(long long)i * m + pj] = t;
      }
    __syncthreads();
  }
}

// C = alpha (A0 B0 + A1 B1) + beta C, batched through pointer arrays, row-major (A: M x K, B:
// K x N, C: M x N); a null A0/A1 (per item) drops its product.  64 x 64 tiles, 16-deep k slices
// staged in shared memory, 4 x 4 outputs per thread.
template <typename T>
__global__ void __launch_bounds__(256) bgemm2_kernel(int M, int N, int K, T alpha, const T* const* A0s,
                                                     const T* const* B0s, const T* const* A1s,
                                                     const T* const* B1s, T beta, T* const* Cs) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ __align__(16) T sa[BK][BM + 4];
  __shared__ __align__(16) T sb[BK][BN + 4];
  const int b = blockIdx.z, tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int pr = 0; pr < 2; ++pr) {
    const T* const* As = pr == 0 ? A0s : A1s;
    const T* const* Bs = pr == 0 ? B0s : B1s;
    const T* A = As ? As[b] : nullptr;
    if (!A) continue;  // the same for the whole CTA
    const T* B = Bs[b];
    for (int k0 = 0; k0 < K; k0 += BK) {
      for (int t = tid; t < BM * BK; t += 256) {
        const int i = t / BK, kk = t % BK, r = r0 + i, k = k0 + kk;
        sa[kk][i] = (r < M && k < K) ? A[(long long)r * K + k] : (T)0;
      }
      for (int t = tid; t < BK * BN; t += 256) {
        const int kk = t / BN, j = t % BN, k = k0 + kk, c = c0 + j;
        sb[kk][j] = (k < K && c < N) ? B[(long long)k * N + c] : (T)0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = sa[kk][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = sb[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
      }
      __syncthreads();
    }
  }
  T* C = Cs[b];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty * 4 + i, c = c0 + tx * 4 + j;
      if (r < M && c < N) {
        T* p = C + (long long)r * N + c;
        *p = alpha * acc[i][j] + (beta == (T)0 ? (T)0 : beta * *p);
      }
    }
}

// Row `item % M` of batch item `item / M` of a kMV step, by one warp.
template <typename T>
__device__ __forceinline__ void mv_row(const CStep<T>& s, long long item, int lane) {
  const int b = (int)(item / s.M), row = (int)(item - (long long)b * s.M);
  const T* A0 = s.A0 ? s.A0[b] : nullptr;
  const T* A1 = s.A1 ? s.A1[b] : nullptr;
  const T* A2 = s.A2 ? s.A2[b] : nullptr;
  T acc = 0, acc2 = 0;
  if (A0) {
    const T* x = s.x0[b];
    for (int c = lane; c < s.N0; c += 32) acc += A0[(long long)row * s.N0 + c] * x[c];
  }
  if (A1) {
    const T* x = s.x1[b];
    for (int c = lane; c < s.N1; c += 32) acc += A1[(long long)row * s.N1 + c] * x[c];
  }
  if (A2) {
    const T* x = s.x2[b];
    for (int c = lane; c < s.N2; c += 32) acc2 += A2[(long long)row * s.N2 + c] * x[c];
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (A2)  // the same for the whole warp
    for (int off = 16; off > 0; off >>= 1) acc2 += __shfl_down_sync(0xffffffffu, acc2, off);
  if (lane == 0) {
    T* y = s.y[b];
    T val = s.alpha * acc;
    if (A2) val += acc2;
    if (s.c && s.c[b]) val += s.c[b][row];
    if (s.beta != (T)0) val += s.beta * y[row];
    y[row] = val;
  }
}

// One kMV step as a launch of its own: 8 rows per CTA, one warp per row.
template <typename T>
__global__ void __launch_bounds__(256) bgemv2_kernel(CStep<T> s) {
  pdl_wait();
  const int row = blockIdx.x * 8 + threadIdx.x / 32;
  if (row >= s.M) return;
  mv_row(s, (long long)blockIdx.y * s.M + row, threadIdx.x % 32);
}

// ---------------------------------------------------------------- DoF classification
struct Cls {
  int type;  // 0 = vertex plane, 1 = interior slab
  int slab;
  int loc;
};

// First cell above the obstacle in a cell column the obstacle crosses (2D).
__host__ __device__ __forceinline__ bool piece_start(const Geom& g, int col, long long row) {
  return has_obstacle(g) && col >= g.ob[0] && col < g.ob[1] && row == g.ob[3] && g.ob[3] < g.n[1];
}

__device__ __forceinline__ Cls classify(const Geom& g, int mV, long long t) {
  Cls c;
  const long long pn = (long long)g.nn[1] * g.nn[2];
  if (t < g.nvel) {
    const long long node = t / g.NV;
    const int v = (int)(t - node * g.NV);
    const int ix = (int)(node % g.nn[0]);
    const long long pi = node / g.nn[0];
    const int q = ix % g.r;  // 0: vertex plane; else the q-th interior node line of the slab
    c.type = q ? 1 : 0;
    c.slab = ix / g.r;
    c.loc = (int)(((q ? q - 1 : 0) * pn + pi) * g.NV + v);
  } else {
    // The pressure of cell column s belongs to I_s except the cell-constant
    // coefficient of the column's first cell, which joins V_s: with Dirichlet
    // data on both ends of a column the column's interior block alone has a
    // constant-pressure null vector (zero net flux).
    const long long u = t - g.nvel;
    const long long cell = u / g.NP;
    const int q = (int)(u - cell * g.NP);
    const int a = q / g.npd, m = q % g.npd;
    const long long cr = cell / g.n[0];
    const long long base = (long long)(g.r - 1) * pn * g.NV;  // interior velocity of the slab
    c.slab = (int)(cell % g.n[0]);
    if (cr == 0 && m == 0) {
      c.type = 0;
      c.loc = (int)(pn * g.NV + a);
    } else if (m == 0 && piece_start(g, c.slab, cr)) {
      c.type = 0;
      c.loc = (int)(pn * g.NV + g.nt + a);
    } else if (cr == 0) {
      c.type = 1;
      c.loc = (int)(base + a * (g.npd - 1) + m - 1);
    } else {
      c.type = 1;
      c.loc = (int)(base + (long long)g.nt * (g.npd - 1) + (cr - 1) * g.NP + q);
    }
  }
  (void)mV;
  return c;
}

__device__ __forceinline__ bool is_pinned(const Geom& g, int pin, long long t) {
  if (!pin || t < g.nvel) return false;
  const long long u = t - g.nvel;
  return u < g.NP && (u % g.npd) == 0;  // cell 0, coefficient 0, every Radau node
}

template <typename T>
__device__ void put(const CoarseView<T>& v, long long row, long long col, double val) {
  const Geom& g = v.g;
  if (is_pinned(g, v.pin, row) || is_pinned(g, v.pin, col)) return;
  const Cls r = classify(g, v.mV, row), c = classify(g, v.mV, col);
  const int mV = v.mV, mI = v.mI;
  long long idx = -1;
  T* base = nullptr;
  if (r.type == 1 && c.type == 1) {
    if (r.slab == c.slab) {
      base = v.AII;
      idx = ((long long)r.slab * mI + r.loc) * mI + c.loc;
    }
  } else if (r.type == 1 && c.type == 0) {
    const int d = c.slab - r.slab;
    if (d == 0 || d == 1) {
      base = v.AIV;
      idx = ((long long)r.slab * mI + r.loc) * (2 * mV) + d * mV + c.loc;
    }
  } else if (r.type == 0 && c.type == 1) {
    const int d = r.slab - c.slab;
    if (d == 0 || d == 1) {
      base = v.AVI;
      idx = ((long long)c.slab * 2 * mV + d * mV + r.loc) * mI + c.loc;
    }
  } else {
    const int d = c.slab - r.slab;
    const long long o = ((long long)r.slab * mV + r.loc) * mV + c.loc;
    if (d == 0) {
      base = v.D;
      idx = o;
    } else if (d == -1) {
      base = v.L;
      idx = o;
    } else if (d == 1) {
      base = v.U;
      idx = o;
    }
  }
  if (base)
    base[idx] = (T)val;
  else if (val != 0.0)
    atomicOr(v.status + 1, 1);  // coupling outside the expected block structure
}

template <typename T>
__global__ void extract_vv(CoarseView<T> v, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                           const double* __restrict__ vv) {
  const Geom& g = v.g;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nvel) return;
  const long long node = t / g.NV;
  const int r = (int)(t - node * g.NV);
  for (int blk = rowptr[node]; blk < rowptr[node + 1]; ++blk)
    for (int s = 0; s < g.NV; ++s)
      put(v, t, (long long)colidx[blk] * g.NV + s, vv[((long long)blk * g.NV + r) * g.NV + s]);
}

template <typename T>
__global__ void extract_vp(CoarseView<T> v, const double* __restrict__ vp, const double* __restrict__ pv) {
  const Geom& g = v.g;
  const int d = g.dim, npd = g.npd, r = g.r, r1 = g.r + 1;
  const long long per = (long long)g.nloc * g.nt * d * npd;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.n_cells * per) return;
  const long long K = t / per;
  int u = (int)(t - K * per);
  const int m = u % npd;
  u /= npd;
  const int c = u % d;
  u /= d;
  const int a = u % g.nt;
  const int i = u / g.nt;
  const int cx = (int)(K % g.n[0]), cy = (int)((K / g.n[0]) % g.n[1]), cz = (int)(K / ((long long)g.n[0] * g.n[1]));
  const long long vel =
      node_id(g, r * cx + i % r1, r * cy + (i / r1) % r1, r * cz + i / (r1 * r1)) * g.NV + a * d + c;
  const long long pres = g.nvel + K * g.NP + a * npd + m;
  put(v, vel, pres, vp[(((K * g.nloc + i) * g.nt + a) * d + c) * npd + m]);
  put(v, pres, vel, pv[((K * g.nt + a) * npd + m) * (long long)g.nloc * d + i * d + c]);
}

// Identity rows for the unused pressure slots of the last vertex plane (it has
// no cell column to its right) and, when pinned, for the fixed pressure value.
template <typename T>
__global__ void pin_diag(CoarseView<T> v) {
  const int a = threadIdx.x;
  if (a >= v.g.nt) return;
  const long long pn = (long long)v.g.nn[1] * v.g.nn[2];
  const long long loc = pn * v.g.NV + a;
  const long long mV = v.mV;
  v.D[((long long)(v.nsv - 1) * mV + loc) * mV + loc] = (T)1;
  if (v.pin) v.D[loc * mV + loc] = (T)1;
}

// Obstacle: identity rows for the pressures of removed cells, for the second pressure group of
// vertex planes whose cell column has no piece above the obstacle, and for the interior slot left
// by each moved coefficient.  One thread per (plane or cell, Radau node).
template <typename T>
__global__ void obstacle_diag(CoarseView<T> v) {
  const Geom& g = v.g;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long pn = (long long)g.nn[1] * g.nn[2];
  const long long mV = v.mV, mI = v.mI;
  if (t < (long long)v.nsv * g.nt) {
    const int s = (int)(t / g.nt), a = (int)(t % g.nt);
    const bool used = s < v.nsi && piece_start(g, s, g.ob[3]);
    const long long loc = pn * g.NV + g.nt + a;
    if (!used) v.D[((long long)s * mV + loc) * mV + loc] = (T)1;
    if (used) {
      // the moved coefficient's own slot in I_s (cell row ob[3] >= 1, coefficient 0)
      const long long il = (long long)(g.r - 1) * pn * g.NV + (long long)g.nt * (g.npd - 1) +
                           (g.ob[3] - 1) * g.NP + a * g.npd;
      v.AII[((long long)s * mI + il) * mI + il] = (T)1;
    }
  }
  const long long u = t;
  if (u < g.n_cells * g.NP) {
    const long long cell = u / g.NP;
    const int cx = (int)(cell % g.n[0]), cy = (int)(cell / g.n[0]);
    if (cell_masked(g, cx, cy)) put(v, g.nvel + u, g.nvel + u, 1.0);
  }
}

// D[t] -= C[t-1](lower right) + C[t](upper left); U[t] -= C[t](upper right); L[t+1] -= C[t](lower left)
template <typename T>
__global__ void schur_combine(CoarseView<T> v, const T* __restrict__ C) {
  const int mV = v.mV, nsi = v.nsi;
  const long long per = (long long)mV * mV;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)(nsi + 1) * per) return;
  const int s = (int)(t / per);
  const int i = (int)((t % per) / mV), j = (int)(t % mV);
  const long long ld = 2 * mV;
  T d = v.D[t];
  if (s > 0) d -= C[(long long)(s - 1) * 4 * per + (long long)(mV + i) * ld + mV + j];
  if (s < nsi) {
    const T* Cs = C + (long long)s * 4 * per;
    d -= Cs[(long long)i * ld + j];
    v.U[t] -= Cs[(long long)i * ld + mV + j];
    v.L[t + per] -= Cs[(long long)(mV + i) * ld + j];
  }
  v.D[t] = d;
}

template <typename T>
__global__ void gather_rhs(CoarseView<T> v, const double* __restrict__ b, T* __restrict__ bV, T* __restrict__ bI) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= v.g.N) return;
  const Cls c = classify(v.g, v.mV, t);
  const T val = is_pinned(v.g, v.pin, t) ? (T)0 : (T)b[t];
  if (c.type == 0)
    bV[(long long)c.slab * v.mV + c.loc] = val;
  else
    bI[(long long)c.slab * v.mI + c.loc] = val;
}

template <typename T>
__global__ void scatter_sol(CoarseView<T> v, const T* __restrict__ xV, const T* __restrict__ xI,
                            double* __restrict__ x) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= v.g.N) return;
  const Cls c = classify(v.g, v.mV, t);
  x[t] = (double)(c.type == 0 ? xV[(long long)c.slab * v.mV + c.loc] : xI[(long long)c.slab * v.mI + c.loc]);
}

template <typename T>
T** upload_ptrs(const std::vector<T*>& h, std::vector<void*>& owned) {
  if (h.empty()) return nullptr;
  T** d = nullptr;
  STG_CUDA_OK(cudaMalloc(&d, sizeof(T*) * h.size()));
  STG_CUDA_OK(cudaMemcpy(d, h.data(), sizeof(T*) * h.size(), cudaMemcpyHostToDevice));
  owned.push_back(d);
  return d;
}

}  // namespace

template <typename T>
void CoarseSolver<T>::init(const Geom& geom, bool pure_dirichlet) {
  v.g = geom;
  v.pin = pure_dirichlet ? 1 : 0;
  v.nsi = geom.n[0];
  v.nsv = geom.n[0] + 1;
  const long long pn = (long long)geom.nn[1] * geom.nn[2];
  v.mV = (int)(pn * geom.NV + (has_obstacle(geom) ? 2 : 1) * geom.nt);
  v.mI = (int)((long long)(geom.r - 1) * pn * geom.NV + (long long)geom.n[1] * geom.n[2] * geom.NP - geom.nt);
  const long long mV = v.mV, mI = v.mI, nsi = v.nsi, nsv = v.nsv;
  auto alloc = [&](T** p, long long n) {
    STG_CUDA_OK(cudaMalloc(p, sizeof(T) * (n > 0 ? n : 1)));
    owned.push_back(*p);
  };
  alloc(&v.AII, nsi * mI * mI);
  alloc(&v.AIV, nsi * mI * 2 * mV);
  alloc(&v.AVI, nsi * 2 * mV * mI);
  alloc(&W, nsi * mI * 2 * mV);
  alloc(&C, nsi * 4 * mV * mV);
  alloc(&v.D, nsv * mV * mV);
  alloc(&v.L, nsv * mV * mV);
  alloc(&v.U, nsv * mV * mV);
  alloc(&GL, nsv * mV * mV);
  alloc(&GU, nsv * mV * mV);
  alloc(&bV, nsv * mV);
  {
    const long long nb = std::max(nsi, nsv), mm = std::max(mI, mV);
    alloc(&gj_scr, nb * mm);
    STG_CUDA_OK(cudaMalloc(&gj_perm, sizeof(int) * nb * mm));
    owned.push_back(gj_perm);
    STG_CUDA_OK(cudaMalloc(&gj_fail, sizeof(int) * nb));
    owned.push_back(gj_fail);
    if (mm >= 512) {
      // blocked Gauss-Jordan scratch: panels of at most 32 columns (FP32) or 16 (FP64)
      gjb.w = sizeof(T) == 4 ? 32 : 16;
      gjb.m_max = mm;
      gjb.batch_max = (int)nb;
      T *pan = nullptr, *old = nullptr;
      alloc(&pan, nb * mm * gjb.w);
      alloc(&old, nb * mm * gjb.w);
      std::vector<T*> hp(nb), ho(nb);
      for (long long b = 0; b < nb; ++b) {
        hp[b] = pan + b * mm * gjb.w;
        ho[b] = old + b * mm * gjb.w;
      }
      gjb.panels = upload_ptrs(hp, owned);
      gjb.olds = upload_ptrs(ho, owned);
    }
  }
  alloc(&xV, nsv * mV);
  alloc(&bI, nsi * mI);
  alloc(&gI, nsi * mI);
  alloc(&xI, nsi * mI);
  int* st = nullptr;
  STG_CUDA_OK(cudaMalloc(&st, sizeof(int) * 2));
  owned.push_back(st);
  v.status = st;

  // per-slab pointer arrays for the interior elimination
  std::vector<T*> pAII, pAIV, pAVI, pW, pC, pbI, pgI, pxVs, pxI;
  for (long long s = 0; s < nsi; ++s) {
    pAII.push_back(v.AII + s * mI * mI);
    pAIV.push_back(v.AIV + s * mI * 2 * mV);
    pAVI.push_back(v.AVI + s * 2 * mV * mI);
    pW.push_back(W + s * mI * 2 * mV);
    pC.push_back(C + s * 4 * mV * mV);
    pbI.push_back(bI + s * mI);
    pgI.push_back(gI + s * mI);
    pxVs.push_back(xV + s * mV);  // [x_V,s ; x_V,s+1] are contiguous
    pxI.push_back(xI + s * mI);
  }
  d_AII = upload_ptrs(pAII, owned);
  d_AIV = upload_ptrs(pAIV, owned);
  d_AVI = upload_ptrs(pAVI, owned);
  d_W = upload_ptrs(pW, owned);
  d_C = upload_ptrs(pC, owned);
  d_bI = upload_ptrs(pbI, owned);
  d_gI = upload_ptrs(pgI, owned);
  d_xVs = upload_ptrs(pxVs, owned);
  d_xI = upload_ptrs(pxI, owned);

  // cyclic-reduction schedule over the nsv vertex planes.  curL/curU: the block each plane's L/U
  // currently lives in (level 0: the extracted blocks; later levels: the previous level's output)
  levels.clear();
  auto blk = [&](T* base, long long i) { return base + i * mV * mV; };
  std::vector<T*> curL(nsv), curU(nsv);
  for (long long j = 0; j < nsv; ++j) {
    curL[j] = blk(v.L, j);
    curU[j] = blk(v.U, j);
  }
  for (long long st_ = 1; st_ < nsv; st_ *= 2) {
    CrLevel<T> lv{};
    lv.stride = st_;
    // odd planes: D_i^{-1} (in place), GL_i, GU_i
    std::vector<T*> oD, gA, gB, gC;
    for (long long i = st_; i < nsv; i += 2 * st_) oD.push_back(blk(v.D, i));
    lv.n_odd = (int)oD.size();
    for (int pass = 0; pass < 2; ++pass)
      for (long long i = st_; i < nsv; i += 2 * st_) {
        gA.push_back(blk(v.D, i));
        gB.push_back(pass == 0 ? curL[i] : curU[i]);
        gC.push_back(blk(pass == 0 ? GL : GU, i));
      }
    lv.oD = upload_ptrs(oD, owned);
    lv.gA = upload_ptrs(gA, owned);
    lv.gB = upload_ptrs(gB, owned);
    lv.gC = upload_ptrs(gC, owned);
    // even planes with a neighbour: D update and the forward right-hand-side update share the
    // products' left factors (this level's L_j, U_j); new L/U blocks for the next level
    std::vector<T*> eA0, eA1, ey, fA0, fx0, fA1, fx1, dB0, dB1, dC, uA, uB, uC, pB, pC;
    std::vector<T*> newL(curL), newU(curU);
    int n_left = 0, n_right = 0;
    std::vector<T*> uAr, uBr, uCr, pBr, pCr;
    for (long long j = 0; j < nsv; j += 2 * st_) {
      const bool has_l = j - st_ >= 0, has_r = j + st_ < nsv;
      if (!has_l && !has_r) continue;
      T* pl = nullptr;
      T* pr = nullptr;
      if (has_l) alloc(&pl, mV * mV);
      if (has_r) alloc(&pr, mV * mV);
      eA0.push_back(has_l ? curL[j] : nullptr);
      dB0.push_back(has_l ? blk(GU, j - st_) : nullptr);
      eA1.push_back(has_r ? curU[j] : nullptr);
      dB1.push_back(has_r ? blk(GL, j + st_) : nullptr);
      fA0.push_back(pl);
      fx0.push_back(has_l ? bV + (j - st_) * mV : nullptr);
      fA1.push_back(pr);
      fx1.push_back(has_r ? bV + (j + st_) * mV : nullptr);
      ey.push_back(bV + j * mV);
      dC.push_back(blk(v.D, j));
      if (has_l) {
        T* p = nullptr;
        alloc(&p, mV * mV);
        uA.push_back(curL[j]);
        uB.push_back(blk(GL, j - st_));
        uC.push_back(p);
        pB.push_back(blk(v.D, j - st_));  // D_{j-st}^{-1} once inverted
        pC.push_back(pl);
        newL[j] = p;
        ++n_left;
      }
      if (has_r) {
        T* p = nullptr;
        alloc(&p, mV * mV);
        uAr.push_back(curU[j]);
        uBr.push_back(blk(GU, j + st_));
        uCr.push_back(p);
        pBr.push_back(blk(v.D, j + st_));
        pCr.push_back(pr);
        newU[j] = p;
        ++n_right;
      }
    }
    uA.insert(uA.end(), uAr.begin(), uAr.end());
    uB.insert(uB.end(), uBr.begin(), uBr.end());
    uC.insert(uC.end(), uCr.begin(), uCr.end());
    pB.insert(pB.end(), pBr.begin(), pBr.end());
    pC.insert(pC.end(), pCr.begin(), pCr.end());
    lv.n_left = n_left;
    lv.n_right = n_right;
    lv.n_even = (int)ey.size();
    lv.eA0 = upload_ptrs(eA0, owned);
    lv.eA1 = upload_ptrs(eA1, owned);
    lv.fA0 = upload_ptrs(fA0, owned);
    lv.fx0 = upload_ptrs(fx0, owned);
    lv.fA1 = upload_ptrs(fA1, owned);
    lv.fx1 = upload_ptrs(fx1, owned);
    lv.ey = upload_ptrs(ey, owned);
    lv.dB0 = upload_ptrs(dB0, owned);
    lv.dB1 = upload_ptrs(dB1, owned);
    lv.dC = upload_ptrs(dC, owned);
    lv.uA = upload_ptrs(uA, owned);
    lv.uB = upload_ptrs(uB, owned);
    lv.uC = upload_ptrs(uC, owned);
    lv.pB = upload_ptrs(pB, owned);
    lv.pC = upload_ptrs(pC, owned);
    // back substitution of the odd planes: x_i = D_i^{-1} b_i - GL_i x_{i-st} - GU_i x_{i+st}
    std::vector<T*> bx, bb, bGL, bxl, qA1, qx1;
    for (long long i = st_; i < nsv; i += 2 * st_) {
      bx.push_back(xV + i * mV);
      bb.push_back(bV + i * mV);
      bGL.push_back(blk(GL, i));
      bxl.push_back(xV + (i - st_) * mV);
      qA1.push_back(i + st_ < nsv ? blk(GU, i) : nullptr);
      qx1.push_back(i + st_ < nsv ? xV + (i + st_) * mV : nullptr);
    }
    lv.bx = upload_ptrs(bx, owned);
    lv.bb = upload_ptrs(bb, owned);
    lv.bGL = upload_ptrs(bGL, owned);
    lv.bxl = upload_ptrs(bxl, owned);
    lv.qA1 = upload_ptrs(qA1, owned);
    lv.qx1 = upload_ptrs(qx1, owned);
    levels.push_back(lv);
    curL.swap(newL);
    curU.swap(newU);
  }
  std::vector<T*> top{v.D}, topb{bV}, topx{xV};
  d_top = upload_ptrs(top, owned);
  d_topb = upload_ptrs(topb, owned);
  d_topx = upload_ptrs(topx, owned);

  // the vertex-plane right-hand side update from the interiors: b_V,s -= A_VI,s-1 (upper rows)
  // g_I,s-1 + A_VI,s (lower rows) g_I,s, with g_I = A_II^{-1} b_I
  {
    std::vector<T*> cA0, cx0, cA1, cx1, cy;
    for (long long s = 0; s < nsv; ++s) {
      cA0.push_back(s >= 1 ? v.AVI + (s - 1) * 2 * mV * mI + mV * mI : nullptr);
      cx0.push_back(s >= 1 ? gI + (s - 1) * mI : nullptr);
      cA1.push_back(s < nsi ? v.AVI + s * 2 * mV * mI : nullptr);
      cx1.push_back(s < nsi ? gI + s * mI : nullptr);
      cy.push_back(bV + s * mV);
    }
    d_cA0 = upload_ptrs(cA0, owned);
    d_cx0 = upload_ptrs(cx0, owned);
    d_cA1 = upload_ptrs(cA1, owned);
    d_cx1 = upload_ptrs(cx1, owned);
    d_cy = upload_ptrs(cy, owned);
  }

  // the solve plan: interior right-hand sides, reduction down the levels, the top block, back
  // substitution up the levels, the interiors, the scatter.  Slots of bV that no unknown maps to
  // are zeroed once (here) and stay zero: the rows of every operator the plan applies vanish there.
  STG_CUDA_OK(cudaMemset(bV, 0, sizeof(T) * nsv * mV));
  const T one = 1, zero = 0, mone = -1;
  const int m = (int)mV;
  auto mv = [&](int M, int N0, int N1, int N2, T alpha, T* const* A0, T* const* x0, T* const* A1, T* const* x1,
                T* const* A2, T* const* x2, T beta, T* const* y, long long batch) {
    if (batch <= 0) return;
    plan.push_back(CStep<T>{kMV, M, N0, N1, N2, (int)batch, alpha, beta, A0, x0, A1, x1, A2, x2, nullptr, y});
  };
  auto element = [&](int kind) {
    plan.push_back(CStep<T>{kind, 0, 0, 0, 0, 0, zero, zero, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                            nullptr, nullptr});
  };
  plan.clear();
  element(kGather);
  mv((int)mI, (int)mI, 0, 0, one, d_AII, d_bI, nullptr, nullptr, nullptr, nullptr, zero, d_gI, nsi);
  mv(m, (int)mI, (int)mI, 0, mone, d_cA0, d_cx0, d_cA1, d_cx1, nullptr, nullptr, one, d_cy, nsv);
  for (const auto& lv : levels)  // b_j -= PL_j b_{j-st} + PR_j b_{j+st} (even planes)
    mv(m, m, m, 0, mone, lv.fA0, lv.fx0, lv.fA1, lv.fx1, nullptr, nullptr, one, lv.ey, lv.n_even);
  mv(m, m, 0, 0, one, d_top, d_topb, nullptr, nullptr, nullptr, nullptr, zero, d_topx, 1);
  for (auto it = levels.rbegin(); it != levels.rend(); ++it)  // x_i = D_i^{-1} b_i - GL_i x_{i-st} - GU_i x_{i+st}
    mv(m, m, m, m, mone, it->bGL, it->bxl, it->qA1, it->qx1, it->oD, it->bb, zero, it->bx, it->n_odd);
  // x_I = g_I - W [x_V,s ; x_V,s+1]
  plan.push_back(CStep<T>{kMV, (int)mI, (int)(2 * mV), 0, 0, (int)nsi, mone, zero, d_W, d_xVs, nullptr, nullptr,
                          nullptr, nullptr, d_gI, d_xI});
  element(kScatter);
}

template <typename T>
void CoarseSolver<T>::release() {
  for (void* p : owned) cudaFree(p);
  owned.clear();
}

// Batched in-place inverses.  scratch: batch * m values of T, perm: batch * m ints, fail: batch
// ints (used only for matrices of 512 rows or more, which take the multi-launch form).
// FP32 blocks of up to 256 rows go to the on-chip Gauss-Jordan (coarse_gj.cu)
static bool rgj(int m, float* const* A, int batch, int* status, cudaStream_t st) {
  return rgj_invert(m, A, batch, status, st);
}
static bool rgj(int, double* const*, int, int*, cudaStream_t) { return false; }

template <typename T>
static void gemm2(int M, int N, int K, T alpha, const T* const* A0, const T* const* B0, const T* const* A1,
                  const T* const* B1, T beta, T* const* C, int batch, cudaStream_t st);

template <typename T>
static void gj(int m, T* const* A, int batch, int* status, T* scratch, int* perm, int* fail, const GjBlocked& blk,
               cudaStream_t st) {
  if (batch <= 0 || m <= 0) return;
  if (rgj(m, A, batch, status, st)) return;
  const size_t tail = sizeof(T) * m + sizeof(int) * m;
  const size_t full = sizeof(T) * (size_t)m * m + tail;
  if (full <= 220 * 1024) {  // the whole matrix in shared memory
    STG_CUDA_OK(cudaFuncSetAttribute(bgj_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(full, 48 * 1024)));
    bgj_kernel<T, true><<<batch, 1024, full, st>>>(m, A, status);
    STG_LAUNCH_OK();
    return;
  }
  if (m < 512) {  // one CTA per matrix in global memory: faster than 2m launches at this size
    STG_CUDA_OK(cudaFuncSetAttribute(bgj_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(tail, 48 * 1024)));
    bgj_kernel<T, false><<<batch, 1024, tail, st>>>(m, A, status);
    STG_LAUNCH_OK();
    return;
  }
  STG_CUDA_OK(cudaMemsetAsync(fail, 0, sizeof(int) * batch, st));
  if (blk.panels && blk.m_max >= m && blk.batch_max >= batch) {
    // blocked form: panels of w columns in shared memory, one batched product per panel
    int w = blk.w;
    while (w > 4 && ((size_t)m * (w + 1) + m) * sizeof(T) > 200 * 1024) w /= 2;
    const size_t sm = ((size_t)m * (w + 1) + m) * sizeof(T);
    STG_CUDA_OK(cudaFuncSetAttribute(gjb_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(sm, 48 * 1024)));
    const dim3 sgrid((m + 255) / 256, batch);
    for (int c0 = 0; c0 < m; c0 += w) {
      const int wp = std::min(w, m - c0);
      gjb_panel_kernel<T><<<batch, 1024, sm, st>>>(m, c0, wp, A, (T* const*)blk.panels, perm, m, fail);
      STG_LAUNCH_OK();
      gjb_swap_save_kernel<T><<<sgrid, 256, 0, st>>>(m, c0, wp, A, (T* const*)blk.olds, perm, m, fail);
      STG_LAUNCH_OK();
      gemm2<T>(m, m, wp, (T)1, (const T* const*)blk.panels, (const T* const*)blk.olds, nullptr, nullptr, (T)1, A,
               batch, st);
    }
  } else {
    const dim3 ugrid((m + 31) / 32, (m + 31) / 32, batch);
    for (int j = 0; j < m; ++j) {
      gj_pivot_kernel<T><<<batch, 256, 0, st>>>(m, j, A, scratch, perm, fail);
      STG_LAUNCH_OK();
      gj_update_kernel<T><<<ugrid, 256, 0, st>>>(m, j, A, scratch, fail);
      STG_LAUNCH_OK();
    }
  }
  gj_unpermute_kernel<T><<<batch, 1024, 0, st>>>(m, A, perm, fail, status);
  STG_LAUNCH_OK();
}

template <typename T>
static void gemm2(int M, int N, int K, T alpha, const T* const* A0, const T* const* B0, const T* const* A1,
                  const T* const* B1, T beta, T* const* C, int batch, cudaStream_t st) {
  if (batch <= 0) return;
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  bgemm2_kernel<T><<<grid, 256, 0, st>>>(M, N, K, alpha, A0, B0, A1, B1, beta, C);
  STG_LAUNCH_OK();
}

// One plan step as a launch of its own.
template <typename T>
static void run_step(const CStep<T>& s, const CoarseView<T>& v, const double* b, double* x, T* bV, T* bI,
                     const T* xV, const T* xI, cudaStream_t st) {
  if (s.kind == kGather)
    launch_k(gather_rhs<T>, grid_for(v.g.N, 256), 256, 0, st, v, b, bV, bI);
  else if (s.kind == kMV)
    launch_k(bgemv2_kernel<T>, dim3((s.M + 7) / 8, s.batch), 256, 0, st, s);
  else
    launch_k(scatter_sol<T>, grid_for(v.g.N, 256), 256, 0, st, v, xV, xI, x);
}

template <typename T>
void CoarseSolver<T>::factor(const int* rowptr, const int* colidx, const double* vv, const double* vp,
                             const double* pv, cudaStream_t st) {
  const Geom& g = v.g;
  const long long mV = v.mV, mI = v.mI, nsi = v.nsi, nsv = v.nsv;
  STG_CUDA_OK(cudaMemsetAsync(v.status, 0, sizeof(int) * 2, st));
  STG_CUDA_OK(cudaMemsetAsync(v.AII, 0, sizeof(T) * nsi * mI * mI, st));
  STG_CUDA_OK(cudaMemsetAsync(v.AIV, 0, sizeof(T) * nsi * mI * 2 * mV, st));
  STG_CUDA_OK(cudaMemsetAsync(v.AVI, 0, sizeof(T) * nsi * 2 * mV * mI, st));
  STG_CUDA_OK(cudaMemsetAsync(v.D, 0, sizeof(T) * nsv * mV * mV, st));
  STG_CUDA_OK(cudaMemsetAsync(v.L, 0, sizeof(T) * nsv * mV * mV, st));
  STG_CUDA_OK(cudaMemsetAsync(v.U, 0, sizeof(T) * nsv * mV * mV, st));
  extract_vv<T><<<grid_for(g.nvel, 128), 128, 0, st>>>(v, rowptr, colidx, vv);
  STG_LAUNCH_OK();
  const long long nvp = g.n_cells * g.nloc * g.nt * g.dim * g.npd;
  extract_vp<T><<<grid_for(nvp, 256), 256, 0, st>>>(v, vp, pv);
  STG_LAUNCH_OK();
  pin_diag<T><<<1, 32, 0, st>>>(v);
  STG_LAUNCH_OK();
  if (has_obstacle(g)) {
    const long long n_ob = std::max<long long>((long long)nsv * g.nt, g.n_cells * g.NP);
    obstacle_diag<T><<<grid_for(n_ob, 256), 256, 0, st>>>(v);
    STG_LAUNCH_OK();
  }
  // interiors: A_II^{-1}, W = A_II^{-1} A_IV, C = A_VI W, S = A_VV - C (scattered)
  gj<T>((int)mI, d_AII, (int)nsi, v.status, gj_scr, gj_perm, gj_fail, gjb, st);
  const T one = 1, zero = 0, mone = -1;
  gemm2<T>((int)mI, (int)(2 * mV), (int)mI, one, d_AII, d_AIV, nullptr, nullptr, zero, d_W, (int)nsi, st);
  gemm2<T>((int)(2 * mV), (int)(2 * mV), (int)mI, one, d_AVI, d_W, nullptr, nullptr, zero, d_C, (int)nsi, st);
  schur_combine<T><<<grid_for(nsv * mV * mV, 256), 256, 0, st>>>(v, C);
  STG_LAUNCH_OK();
  // block cyclic reduction of the vertex-plane system
  const int m = (int)mV;
  for (const auto& lv : levels) {
    gj<T>(m, lv.oD, lv.n_odd, v.status, gj_scr, gj_perm, gj_fail, gjb, st);
    // [GL_i | GU_i] = D_i^{-1} [L_i | U_i]
    gemm2<T>(m, m, m, one, lv.gA, lv.gB, nullptr, nullptr, zero, lv.gC, 2 * lv.n_odd, st);
    // PL_j = L_j D_{j-st}^{-1}, PR_j = U_j D_{j+st}^{-1} (the solve's forward products)
    gemm2<T>(m, m, m, one, lv.uA, lv.pB, nullptr, nullptr, zero, lv.pC, lv.n_left + lv.n_right, st);
    // D_j -= L_j GU_{j-st} + U_j GL_{j+st}
    gemm2<T>(m, m, m, mone, lv.eA0, lv.dB0, lv.eA1, lv.dB1, one, lv.dC, lv.n_even, st);
    // L_j <- -L_j GL_{j-st}, U_j <- -U_j GU_{j+st}, into new blocks
    gemm2<T>(m, m, m, mone, lv.uA, lv.uB, nullptr, nullptr, zero, lv.uC, lv.n_left + lv.n_right, st);
  }
  gj<T>(m, d_top, 1, v.status, gj_scr, gj_perm, gj_fail, gjb, st);
}

template <typename T>
void CoarseSolver<T>::solve(const double* b, double* x, cudaStream_t st) {
  for (const CStep<T>& s : plan) run_step<T>(s, v, b, x, bV, bI, xV, xI, st);
}

template <typename T>
int CoarseSolver<T>::read_status(cudaStream_t st) {
  int h[2] = {0, 0};
  STG_CUDA_OK(cudaMemcpyAsync(h, v.status, sizeof(h), cudaMemcpyDeviceToHost, st));
  STG_CUDA_OK(cudaStreamSynchronize(st));
  if (h[1]) return -1;
  return h[0];
}

template struct CoarseSolver<double>;
template struct CoarseSolver<float>;

}  // namespace stg
