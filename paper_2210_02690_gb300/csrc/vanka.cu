// Operator application, local inverses and the local Vanka smoother (Sec. 3).
//
// Eq. (3.4): S_K(d) = R_K d + omega J_K^{-1} R_K (b - J d), with J_K the
// restriction of the assembled J to the (k+1)(R^+S^) DoFs of cell K.  The
// averaging loop (S0)-(S3) equals d <- d + omega (sum_K E_K J_K^{-1} R_K r) / p
// with r = b - J d and p the number of cells sharing a DoF.  The sum is
// accumulated colour by colour: cells of one colour share no velocity DoF and
// pressure DoFs belong to one cell, so one colour's scatters never collide
// (no atomics, deterministic order).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace stg {
namespace {

// Factor of a removed cell's patch (obstacle, 2D): the projector onto the patch's unknowns without
// an equation (velocity at Q2 nodes of removed cells only, the cell's pressure), whose rows are
// the identity; the patch smooths only those.  1 at local entry mu when it is such an unknown.
__device__ __forceinline__ bool patch_entry_dead(const Geom& g, int cx, int cy, int mu) {
  const int vel = g.nloc * g.NV;
  if (mu >= vel) return true;
  const int i = mu / g.NV;
  return node_dead(g, 2 * cx + i % 3, 2 * cy + i / 3);
}
template <typename FT>
__device__ void write_patch_projector(const Geom& g, int cx, int cy, FT* out, int tid, int nth) {
  const int n = g.npatch;
  for (int t = tid; t < n * n; t += nth) {
    const int col = t / n, row = t - col * n;
    out[t] = cvt<FT>((row == col && patch_entry_dead(g, cx, cy, row)) ? 1.f : 0.f);
  }
}


template <typename T>
struct AccT { using type = T; };
template <>
struct AccT<__nv_bfloat16> { using type = float; };

// ------------------------------------------------------------------ J x, b - J x
template <int DIM, typename MT, typename VT>
__global__ void __launch_bounds__(256) op_vel_rows(Geom g, const int* __restrict__ rowptr,
                                                   const int* __restrict__ colidx, const MT* __restrict__ vv,
                                                   const MT* __restrict__ vp, const VT* __restrict__ x,
                                                   const VT* __restrict__ b, VT* __restrict__ out) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nvel) return;
  const int NV = g.NV;
  const long long node = t / NV;
  const int row = (int)(t - node * NV);
  VT acc = 0;
  const int b0 = rowptr[node], b1 = rowptr[node + 1];
#pragma unroll 4
  for (int blk = b0; blk < b1; ++blk) {
    const MT* vals = vv + (long long)blk * NV * NV + (long long)row * NV;
    const VT* xc = x + (long long)colidx[blk] * NV;
    for (int s = 0; s < NV; ++s) acc += (VT)vals[s] * xc[s];
  }
  const int ix = (int)(node % g.nn[0]);
  const int iy = (int)((node / g.nn[0]) % g.nn[1]);
  const int iz = (int)(node / ((long long)g.nn[0] * g.nn[1]));
  const int a = row / DIM, c = row % DIM;
  const int id[3] = {ix, iy, iz};
  int clo[3], chi[3];
  for (int e = 0; e < 3; ++e) {
    if (e >= DIM)
      clo[e] = chi[e] = 0;
    else
      node_cells(id[e], g.n[e], clo[e], chi[e], g.r);
  }
  const int r = g.r, r1 = g.r + 1, npd = g.npd;
  for (int cz = clo[2]; cz <= chi[2]; ++cz)
    for (int cy = clo[1]; cy <= chi[1]; ++cy)
      for (int cx = clo[0]; cx <= chi[0]; ++cx) {
        const int il = (ix - r * cx) + r1 * (iy - r * cy) + r1 * r1 * (iz - r * cz);
        const long long K = cell_id(g, cx, cy, cz);
        const MT* q = vp + (((K * g.nloc + il) * g.nt + a) * DIM + c) * npd;
        const VT* p = x + g.nvel + K * g.NP + a * npd;
        for (int m = 0; m < npd; ++m) acc += (VT)q[m] * p[m];
      }
  out[t] = b ? b[t] - acc : acc;
}

// ------------------------------------------------------------------ Kronecker-split FP32 rows (2D)
// With the Radau rule in time the velocity block of node pair (i, j) is
//   J[(a,c),(b,e)] = T_ab M_ij delta_ce + delta_ab Ahat_a,ij[c][e],
// so a slot needs M_ij and, per Radau node a, the d x d spatial block Ahat_a (9 values for
// 2D k = 1 against 16 in the dense block).  Columns follow the structured stencil.

struct TimeF {
  float T[5][5];
};

// Mk[slot] = M_ij, Ak[slot][a][c][e] = Ahat_a,ij[c][e], split (in FP64, then rounded) from the
// FP64 dense blocks: M_ij = J[(as,0),(bs,0)] / T_{as,bs} for the largest off-diagonal |T_{as,bs}|.
__global__ void kron_split_kernel(Geom g, long long nnzb, const double* __restrict__ vv, TimeData td, int as,
                                  int bs, float* __restrict__ Mk, float* __restrict__ Ak) {
  const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nnzb) return;
  const int NV = g.NV, D = g.dim, NT = g.nt;
  const double* blk = vv + slot * NV * NV;
  const double M = blk[(as * D) * NV + bs * D] / td.T[as][bs];
  Mk[slot] = (float)M;
  float* A = Ak + slot * NT * D * D;
  for (int a = 0; a < NT; ++a)
    for (int c = 0; c < D; ++c)
      for (int e = 0; e < D; ++e)
        A[(a * D + c) * D + e] = (float)(blk[(a * D + c) * NV + a * D + e] - (c == e ? td.T[a][a] * M : 0.0));
}

// b - J x (or J x) on the velocity rows of the FP32 level operators from the Kronecker split,
// one thread per (node, Radau node a): per slot the mass term M_ij ((T (x) I) x_j)[a] and the
// 2 x 2 block Ahat_a,ij, 4 + 4 (k+1) d^2 bytes of matrix per slot instead of 4 NV^2.  A stencil
// row (3 or 5 slots) is unrolled with pointer increments, so each slot costs three loads (x_j,
// Ahat_a as one float4, M_ij) and few integer operations.
template <int NT>
struct XNode {
  float v[NT * 2];
};

template <int NT>
__device__ __forceinline__ XNode<NT> load_node(const float* p) {
  XNode<NT> r;
  if (NT % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NT / 2; ++i) {
      const float4 q = reinterpret_cast<const float4*>(p)[i];
      r.v[4 * i] = q.x;
      r.v[4 * i + 1] = q.y;
      r.v[4 * i + 2] = q.z;
      r.v[4 * i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      const float2 q = reinterpret_cast<const float2*>(p)[i];
      r.v[2 * i] = q.x;
      r.v[2 * i + 1] = q.y;
    }
  }
  return r;
}

template <int NT, int W>
__device__ __forceinline__ void kron_stencil_row(const float* __restrict__ xj, const float4* __restrict__ Ap,
                                                 const float* __restrict__ Mp, const float (&tr)[NT], int a,
                                                 float& acc0, float& acc1) {
  constexpr int D = 2, NV = NT * D;
  XNode<NT> xs[W];
  float4 As[W];
  float Ms[W];
#pragma unroll
  for (int u = 0; u < W; ++u) {
    xs[u] = load_node<NT>(xj + u * NV);
    As[u] = Ap[u * NT];
    Ms[u] = Mp[u];
  }
#pragma unroll
  for (int u = 0; u < W; ++u) {
    float y0 = 0.f, y1 = 0.f, xa0 = 0.f, xa1 = 0.f;
#pragma unroll
    for (int bb = 0; bb < NT; ++bb) {
      y0 += tr[bb] * xs[u].v[bb * D];
      y1 += tr[bb] * xs[u].v[bb * D + 1];
      if (bb == a) {
        xa0 = xs[u].v[bb * D];
        xa1 = xs[u].v[bb * D + 1];
      }
    }
    acc0 += Ms[u] * y0 + As[u].x * xa0 + As[u].y * xa1;
    acc1 += Ms[u] * y1 + As[u].z * xa0 + As[u].w * xa1;
  }
}

// One thread per (node, Radau node a): both velocity rows (a, 0), (a, 1).
template <int NT>
__global__ void __launch_bounds__(256) op_vel_rows_kron(Geom g, TimeF tf, const float* __restrict__ Mk,
                                                        const float* __restrict__ Ak,
                                                        const float* __restrict__ vp, const float* __restrict__ x,
                                                        const float* __restrict__ b, float* __restrict__ out) {
  pdl_wait();
  constexpr int D = 2, NV = NT * D;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // (node, a) pairs < 2^31 (checked by the caller)
  if (t >= g.n_nodes * NT) return;
  const int node = t / NT;
  const int a = t - node * NT;
  const int nx = g.nn[0];
  const int ix = node % nx, iy = node / nx;
  int xl, xh, yl, yh;
  stencil_range(ix, nx, xl, xh);
  stencil_range(iy, g.nn[1], yl, yh);
  float tr[NT];
#pragma unroll
  for (int bb = 0; bb < NT; ++bb) {
    float v = tf.T[0][bb];
#pragma unroll
    for (int aa = 1; aa < NT; ++aa)
      if (aa == a) v = tf.T[aa][bb];
    tr[bb] = v;
  }
  float acc0 = 0.f, acc1 = 0.f;
  // first block slot of the row in closed form (no dependent load of rowptr): with r = 2 a node
  // couples to w(i) = 5 nodes per direction at interior even indices and to 3 elsewhere, so
  // the rows before (ix, iy) hold P(iy) S_x + w(iy) P(ix) slots, with the prefix
  // P(i) = sum_{i' < i} w(i') = 3 i + 2 max(0, (i + 1) / 2 - 1) and S_x = P(nx - 1) + 3
  auto prefix = [](int i) { return 3 * i + 2 * max(0, (i + 1) / 2 - 1); };
  const int s0 = prefix(iy) * (prefix(nx - 1) + 3) + (yh - yl + 1) * prefix(ix);
  const float* Mp = Mk + s0;
  const float4* Ap = reinterpret_cast<const float4*>(Ak) + (long long)s0 * NT + a;  // Ahat_a (2 x 2)
  const int wx = xh - xl + 1;
  for (int jy = yl; jy <= yh; ++jy) {
    const float* xj = x + ((long long)jy * nx + xl) * NV;
    if (wx == 5)
      kron_stencil_row<NT, 5>(xj, Ap, Mp, tr, a, acc0, acc1);
    else
      kron_stencil_row<NT, 3>(xj, Ap, Mp, tr, a, acc0, acc1);
    Mp += wx;
    Ap += wx * NT;
  }
  // pressure coupling of the cells around the node
  const int cxl = (ix & 1) ? (ix - 1) / 2 : (ix / 2 - 1 < 0 ? 0 : ix / 2 - 1);
  const int cxh = (ix & 1) ? (ix - 1) / 2 : (ix / 2 > g.n[0] - 1 ? g.n[0] - 1 : ix / 2);
  const int cyl = (iy & 1) ? (iy - 1) / 2 : (iy / 2 - 1 < 0 ? 0 : iy / 2 - 1);
  const int cyh = (iy & 1) ? (iy - 1) / 2 : (iy / 2 > g.n[1] - 1 ? g.n[1] - 1 : iy / 2);
  for (int cy = cyl; cy <= cyh; ++cy)
    for (int cx = cxl; cx <= cxh; ++cx) {
      const int il = (ix - 2 * cx) + 3 * (iy - 2 * cy);
      const long long K = (long long)cy * g.n[0] + cx;
      const float* q = vp + ((K * g.nloc + il) * NT + a) * D * (D + 1);
      const float* p = x + g.nvel + K * g.NP + a * (D + 1);
      acc0 += q[0] * p[0] + q[1] * p[1] + q[2] * p[2];
      acc1 += q[3] * p[0] + q[4] * p[1] + q[5] * p[2];
    }
  const long long o = (long long)node * NV + a * D;
  if (b) {
    out[o] = b[o] - acc0;
    out[o + 1] = b[o + 1] - acc1;
  } else {
    out[o] = acc0;
    out[o + 1] = acc1;
  }
}

template <int DIM, typename MT, typename VT>
__global__ void __launch_bounds__(256) op_pres_rows(Geom g, const MT* __restrict__ pv, const VT* __restrict__ x,
                                                    const VT* __restrict__ b, VT* __restrict__ out) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.npres) return;
  const long long K = t / g.NP;
  const int q = (int)(t - K * g.NP);
  const int npd = g.npd;
  const int a = q / npd, m = q % npd;
  const int cx = (int)(K % g.n[0]);
  const int cy = (int)((K / g.n[0]) % g.n[1]);
  const int cz = (int)(K / ((long long)g.n[0] * g.n[1]));
  const MT* row = pv + ((K * g.nt + a) * npd + m) * (long long)g.nloc * DIM;
  VT acc = 0;
  if (DIM == 2 && cell_masked(g, cx, cy)) {  // removed cell: identity row
    out[g.nvel + t] = b ? b[g.nvel + t] - x[g.nvel + t] : x[g.nvel + t];
    return;
  }
  const int r = g.r, r1 = g.r + 1;
  for (int i = 0; i < g.nloc; ++i) {
    const long long nd = node_id(g, r * cx + i % r1, r * cy + (i / r1) % r1, r * cz + i / (r1 * r1));
    const VT* xv = x + nd * g.NV + a * DIM;
    for (int e = 0; e < DIM; ++e) acc += (VT)row[i * DIM + e] * xv[e];
  }
  out[g.nvel + t] = b ? b[g.nvel + t] - acc : acc;
}

// ------------------------------------------------------------------ local inverses
// Gather J_K from the assembled operator, then in-place Gauss-Jordan inversion
// with partial pivoting (row interchanges, first maximal pivot as in LAPACK's
// i_amax, columns swapped back at the end).  A in shared memory, or in global
// scratch when it does not fit (SCR != nullptr).
template <typename CT, typename FT>
__global__ void __launch_bounds__(256) invert_kernel(Geom g, long long p0, const int* __restrict__ rowptr,
                                                     const double* __restrict__ vv,
                                                     const double* __restrict__ vp,
                                                     const double* __restrict__ pv, FT* __restrict__ jinv,
                                                     long long stride, int* status, int equil, CT* scratch,
                                                     const int* __restrict__ only) {
  const int n = g.npatch, NV = g.NV, nloc = g.nloc, dim = g.dim, nt = g.nt;
  const int gr = g.r, gr1 = g.r + 1, npd = g.npd;
  const long long p = p0 + blockIdx.x;
  if (only && !only[p]) return;  // block-uniform: only the patches a pivot-free pass flagged
  int cx, cy, cz;
  patch_cell(g, p, cx, cy, cz);
  const long long cell = cell_id(g, cx, cy, cz);
  if (g.dim == 2 && cell_masked(g, cx, cy)) {  // removed cell: block-uniform early return
    write_patch_projector(g, cx, cy, jinv + p * stride, threadIdx.x, blockDim.x);
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  CT* A;
  CT* tail;
  if (scratch) {
    A = scratch + (long long)blockIdx.x * n * n;
    tail = (CT*)smem_raw;
  } else {
    A = (CT*)smem_raw;
    tail = A + n * n;
  }
  CT* colj = tail;
  CT* rs = colj + n;
  CT* cs = rs + n;
  int* perm = (int*)(cs + n);
  __shared__ int s_piv, s_fail;
  __shared__ CT s_pval;
  const int tid = threadIdx.x, nth = blockDim.x;

  for (int t = tid; t < n * n; t += nth) A[t] = 0;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  const int nvv = nloc * nloc * NV * NV;
  for (int t = tid; t < nvv; t += nth) {
    const int s = t % NV, r = (t / NV) % NV, j = (t / (NV * NV)) % nloc, i = t / (NV * NV * nloc);
    const long long slot = bcsr_slot(g, rowptr, gr * cx + i % gr1, gr * cy + (i / gr1) % gr1, gr * cz + i / (gr1 * gr1),
                                     gr * cx + j % gr1, gr * cy + (j / gr1) % gr1, gr * cz + j / (gr1 * gr1));
    A[(i * NV + r) * n + j * NV + s] = (CT)vv[slot * NV * NV + r * NV + s];
  }
  const int nvp = nloc * nt * dim * npd;
  const int voff = nloc * NV;
  for (int t = tid; t < nvp; t += nth) {
    const int m = t % npd, c = (t / npd) % dim, a = (t / (npd * dim)) % nt;
    const int i = t / (npd * dim * nt);
    const int vrow = i * NV + a * dim + c, prow = voff + a * npd + m;
    A[vrow * n + prow] = (CT)vp[(((cell * nloc + i) * nt + a) * dim + c) * npd + m];
    A[prow * n + vrow] = (CT)pv[((cell * nt + a) * npd + m) * (long long)nloc * dim + i * dim + c];
  }
  __syncthreads();

  // optional equilibration: A' = Dr A Dc with Dr = 1/max|row|, then Dc = 1/max|col of Dr A|
  for (int i = tid; i < n; i += nth) {
    rs[i] = 1;
    cs[i] = 1;
  }
  __syncthreads();
  if (equil) {
    for (int i = tid; i < n; i += nth) {
      CT mx = 0;
      for (int l = 0; l < n; ++l) mx = fmax(mx, fabs(A[i * n + l]));
      rs[i] = mx > 0 ? (CT)1 / mx : (CT)1;
    }
    __syncthreads();
    for (int l = tid; l < n; l += nth) {
      CT mx = 0;
      for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(A[i * n + l] * rs[i]));
      cs[l] = mx > 0 ? (CT)1 / mx : (CT)1;
    }
    __syncthreads();
    for (int t = tid; t < n * n; t += nth) A[t] *= rs[t / n] * cs[t % n];
    __syncthreads();
  }

  for (int j = 0; j < n; ++j) {
    if (tid < 32) {
      CT best = -1;
      int bi = n;
      for (int i = j + tid; i < n; i += 32) {
        const CT v = fabs(A[i * n + j]);
        if (v > best || (v == best && i < bi)) {
          best = v;
          bi = i;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const CT ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        s_piv = bi;
        const CT pv_ = bi < n ? A[bi * n + j] : (CT)0;
        s_pval = pv_;
        if (!(fabs(pv_) > 0) || isinf(pv_)) s_fail = 1;
        perm[j] = bi;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const int pr = s_piv;
    if (pr != j)
      for (int l = tid; l < n; l += nth) {
        const CT tmp = A[j * n + l];
        A[j * n + l] = A[pr * n + l];
        A[pr * n + l] = tmp;
      }
    __syncthreads();
    for (int i = tid; i < n; i += nth) colj[i] = A[i * n + j];
    __syncthreads();
    const CT inv = (CT)1 / s_pval;
    for (int l = tid; l < n; l += nth) A[j * n + l] = (l == j ? (CT)1 : A[j * n + l]) * inv;
    __syncthreads();
    for (int t = tid; t < n * n; t += nth) {
      const int i = t / n, l = t - i * n;
      if (i == j) continue;
      A[t] = (l == j ? (CT)0 : A[t]) - colj[i] * A[j * n + l];
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) atomicCAS(status, 0, (int)(cell + 1));
    for (int t = tid; t < n * n; t += nth) jinv[p * stride + t] = cvt<FT>((CT)0);
    return;
  }
  for (int j = n - 1; j >= 0; --j) {
    const int pj = perm[j];
    if (pj != j)
      for (int i = tid; i < n; i += nth) {
        const CT tmp = A[i * n + j];
        A[i * n + j] = A[i * n + pj];
        A[i * n + pj] = tmp;
      }
    __syncthreads();
  }
  // A^{-1} = Dc A'^{-1} Dr, stored column-major
  for (int t = tid; t < n * n; t += nth) {
    const int col = t / n, row = t - col * n;
    jinv[p * stride + t] = cvt<FT>(A[row * n + col] * cs[row] * rs[col]);
  }
}

// Warp-per-patch variant for patches whose matrix fits a warp's share of shared
// memory (2D, n <= 105): same gather, equilibration and Gauss-Jordan elimination
// as invert_kernel, with only warp-level synchronisation.
template <typename CT, typename FT>
__global__ void __launch_bounds__(256) invert_warp_kernel(Geom g, const int* __restrict__ rowptr,
                                                          const double* __restrict__ vv,
                                                          const double* __restrict__ vp,
                                                          const double* __restrict__ pv, FT* __restrict__ jinv,
                                                          long long stride, int* status, int equil,
                                                          const int* __restrict__ only) {
  const int n = g.npatch, NV = g.NV, nloc = g.nloc, dim = g.dim, nt = g.nt;
  const int gr = g.r, gr1 = g.r + 1, npd = g.npd;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int per = n * n + 3 * n;
  CT* A = reinterpret_cast<CT*>(smem_raw) + (long long)wid * per;
  CT* colj = A + n * n;
  CT* rs = colj + n;
  CT* cs = rs + n;
  int* perm = reinterpret_cast<int*>(reinterpret_cast<CT*>(smem_raw) + (long long)wpb * per) + wid * n;
  const int voff = nloc * NV;
  for (long long p = (long long)blockIdx.x * wpb + wid; p < g.n_cells; p += (long long)gridDim.x * wpb) {
    if (only && !only[p]) continue;
    int cx, cy, cz;
    patch_cell(g, p, cx, cy, cz);
    const long long cell = cell_id(g, cx, cy, cz);
    if (dim == 2 && cell_masked(g, cx, cy)) {  // removed cell: warp-uniform
      write_patch_projector(g, cx, cy, jinv + p * stride, lane, 32);
      continue;
    }
    for (int t = lane; t < n * n; t += 32) A[t] = 0;
    __syncwarp();
    const int nvv = nloc * nloc * NV * NV;
    for (int t = lane; t < nvv; t += 32) {
      const int s = t % NV, r = (t / NV) % NV, j = (t / (NV * NV)) % nloc, i = t / (NV * NV * nloc);
      const long long slot = bcsr_slot(g, rowptr, gr * cx + i % gr1, gr * cy + (i / gr1) % gr1, gr * cz + i / (gr1 * gr1),
                                       gr * cx + j % gr1, gr * cy + (j / gr1) % gr1, gr * cz + j / (gr1 * gr1));
      A[(i * NV + r) * n + j * NV + s] = (CT)vv[slot * NV * NV + r * NV + s];
    }
    const int nvp = nloc * nt * dim * npd;
    for (int t = lane; t < nvp; t += 32) {
      const int m = t % npd, c = (t / npd) % dim, a = (t / (npd * dim)) % nt;
      const int i = t / (npd * dim * nt);
      const int vrow = i * NV + a * dim + c, prow = voff + a * npd + m;
      A[vrow * n + prow] = (CT)vp[(((cell * nloc + i) * nt + a) * dim + c) * npd + m];
      A[prow * n + vrow] = (CT)pv[((cell * nt + a) * npd + m) * (long long)nloc * dim + i * dim + c];
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      CT mx = 0;
      if (equil)
        for (int l = 0; l < n; ++l) mx = fmax(mx, fabs(A[i * n + l]));
      rs[i] = mx > 0 ? (CT)1 / mx : (CT)1;
    }
    __syncwarp();
    for (int l = lane; l < n; l += 32) {
      CT mx = 0;
      if (equil)
        for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(A[i * n + l] * rs[i]));
      cs[l] = mx > 0 ? (CT)1 / mx : (CT)1;
    }
    __syncwarp();
    if (equil)
      for (int i = 0; i < n; ++i)
        for (int l = lane; l < n; l += 32) A[i * n + l] *= rs[i] * cs[l];
    __syncwarp();
    bool fail = false;
    for (int j = 0; j < n; ++j) {
      CT best = -1;
      int bi = n;
      for (int i = j + lane; i < n; i += 32) {
        const CT v = fabs(A[i * n + j]);
        if (v > best || (v == best && i < bi)) {
          best = v;
          bi = i;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const CT ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      const CT pval = bi < n ? A[bi * n + j] : (CT)0;
      if (!(fabs(pval) > 0) || isinf(pval)) {
        fail = true;
        break;
      }
      if (lane == 0) perm[j] = bi;
      if (bi != j)
        for (int l = lane; l < n; l += 32) {
          const CT tmp = A[j * n + l];
          A[j * n + l] = A[bi * n + l];
          A[bi * n + l] = tmp;
        }
      __syncwarp();
      for (int i = lane; i < n; i += 32) colj[i] = A[i * n + j];
      __syncwarp();
      const CT inv = (CT)1 / pval;
      for (int l = lane; l < n; l += 32) A[j * n + l] = (l == j ? (CT)1 : A[j * n + l]) * inv;
      __syncwarp();
      for (int i = 0; i < n; ++i) {
        if (i == j) continue;
        const CT f = colj[i];
        for (int l = lane; l < n; l += 32) A[i * n + l] = (l == j ? (CT)0 : A[i * n + l]) - f * A[j * n + l];
      }
      __syncwarp();
    }
    if (fail) {
      if (lane == 0) atomicCAS(status, 0, (int)(cell + 1));
      for (int t = lane; t < n * n; t += 32) jinv[p * stride + t] = cvt<FT>((CT)0);
      __syncwarp();
      continue;
    }
    for (int j = n - 1; j >= 0; --j) {
      const int pj = perm[j];
      if (pj != j)
        for (int i = lane; i < n; i += 32) {
          const CT tmp = A[i * n + j];
          A[i * n + j] = A[i * n + pj];
          A[i * n + pj] = tmp;
        }
      __syncwarp();
    }
    for (int t = lane; t < n * n; t += 32) {
      const int col = t / n, row = t - col * n;
      jinv[p * stride + t] = cvt<FT>(A[row * n + col] * cs[row] * rs[col]);
    }
    __syncwarp();
  }
}

// Row r of the 2D local matrix J_K (local order: time node, 9 Q2 nodes x 2 components,
// then the 3 P1disc coefficients per time node), gathered from the block-CSR velocity
// blocks and the per-cell velocity-pressure blocks and rounded to FP32.
template <int N, typename MT>
__device__ __forceinline__ void gather_patch_row(const Geom& g, const int* __restrict__ rowptr,
                                                 const MT* __restrict__ vv, const MT* __restrict__ vp,
                                                 const MT* __restrict__ pv, int cx, int cy, long long cell,
                                                 int row, float (&a)[N]) {
  constexpr int DIM = 2, NL = 9, NT = N / 21, NV = NT * DIM, NP = NT * (DIM + 1), VOFF = NL * NV;
  if (row < VOFF) {
    const int i = row / NV, v = row % NV, ta = v / DIM, c = v % DIM;
    const int ix = 2 * cx + i % 3, iy = 2 * cy + i / 3;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const long long slot = bcsr_slot(g, rowptr, ix, iy, 0, 2 * cx + j % 3, 2 * cy + j / 3, 0);
      const MT* b = vv + slot * NV * NV + v * NV;
#pragma unroll
      for (int s2 = 0; s2 < NV; ++s2) a[j * NV + s2] = (float)b[s2];
    }
    const MT* q = vp + (((cell * NL + i) * NT + ta) * DIM + c) * (DIM + 1);
#pragma unroll
    for (int m = 0; m < NP; ++m) a[VOFF + m] = (m / (DIM + 1) == ta) ? (float)q[m % (DIM + 1)] : 0.f;
  } else if (row < N) {
    const int qq = row - VOFF, ta = qq / (DIM + 1), m = qq % (DIM + 1);
    const MT* q = pv + ((cell * NT + ta) * (DIM + 1) + m) * (long long)NL * DIM;
#pragma unroll
    for (int col = 0; col < VOFF; ++col) {
      const int j = col / NV, s2 = col % NV;
      a[col] = (s2 / DIM == ta) ? (float)q[j * DIM + s2 % DIM] : 0.f;
    }
#pragma unroll
    for (int m2 = 0; m2 < NP; ++m2) a[VOFF + m2] = 0.f;
  } else {
#pragma unroll
    for (int l = 0; l < N; ++l) a[l] = 0.f;  // padding row of an odd N
  }
}

// Entries 4 l4 .. 4 l4 + 3 of a register row as a float4 (zeros past the end).
template <int N>
__device__ __forceinline__ float4 pack4(const float (&x)[N], int l4) {
  float v[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = 4 * l4 + u;
    v[u] = i < N ? x[i < N ? i : N - 1] : 0.f;
  }
  return make_float4(v[0], v[1], v[2], v[3]);
}

// One step of the rotated Gauss-Jordan elimination of invert_triples_kernel for the three rows
// (x, y, z) of a lane.  The pivot row is read unscaled from shared memory as float4 (raw[0] the
// pivot); every row, the pivot row included, takes x[c - 1] = x[c] - (fx / pivot) raw[c]: with
// fx = pivot - 1 the pivot row becomes x / pivot (up to about eps max(1, |pivot|)), so no row
// needs a select per entry and the pivot row needs no scaling pass before it is published.
// ex = 1 on the pivot row supplies the new last column, 1 / pivot; the other rows get -f / pivot.
template <int N>
__device__ __forceinline__ void triples_update(float (&x)[N], float (&y)[N], float (&z)[N], const float* raw,
                                               float fx, float fy, float fz, float ex, float ey, float ez) {
  constexpr int NR = (N + 3) / 4 * 4;
  const float inv = 1.f / raw[0];
  const float gx = fx * inv, gy = fy * inv, gz = fz * inv;
#pragma unroll
  for (int l4 = 0; l4 < NR / 4; ++l4) {
    const float4 q = reinterpret_cast<const float4*>(raw)[l4];
    const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = 4 * l4 + u;
      if (c >= 1 && c < N) {
        x[c - 1] = fmaf(-gx, qv[u], x[c]);
        y[c - 1] = fmaf(-gy, qv[u], y[c]);
        z[c - 1] = fmaf(-gz, qv[u], z[c]);
      }
    }
  }
  x[N - 1] = fmaf(-fx, inv, ex);
  y[N - 1] = fmaf(-fy, inv, ey);
  z[N - 1] = fmaf(-fz, inv, ez);
}

// Elimination steps s L .. s L + L - 1 of invert_triples_kernel: their pivot rows are register set
// S (0: x, 1: y, 2: z) of lanes 0 .. L - 1 of each group.  Pivot rows alternate between the two
// buffers by the parity of the step, so one __syncwarp per step orders a buffer's next write
// after every lane's reads of it.
template <int N, int L, int S>
__device__ __forceinline__ void triples_phase(float (&x)[N], float (&y)[N], float (&z)[N], float* buf0, float* buf1,
                                              int t, bool& bad) {
  constexpr int NR = (N + 3) / 4 * 4;
#pragma unroll 1
  for (int jj = 0; jj < L; ++jj) {
    const bool own = t == jj;
    float* sr = ((S * L + jj) & 1) ? buf1 : buf0;
    if (own) {
      const float piv = S == 0 ? x[0] : S == 1 ? y[0] : z[0];
      if (!(fabsf(piv) > 1e-3f) || isinf(piv)) bad = true;
#pragma unroll
      for (int l4 = 0; l4 < NR / 4; ++l4)
        reinterpret_cast<float4*>(sr)[l4] = S == 0 ? pack4<N>(x, l4) : S == 1 ? pack4<N>(y, l4) : pack4<N>(z, l4);
    }
    __syncwarp();
    const float fx = (S == 0 && own) ? x[0] - 1.f : x[0];
    const float fy = (S == 1 && own) ? y[0] - 1.f : y[0];
    const float fz = (S == 2 && own) ? z[0] - 1.f : z[0];
    triples_update<N>(x, y, z, sr, fx, fy, fz, (S == 0 && own) ? 1.f : 0.f, (S == 1 && own) ? 1.f : 0.f,
                      (S == 2 && own) ? 1.f : 0.f);
  }
}

// Warp-synchronous variant for the 2D patches of 21 and 42 unknowns: a warp holds 32 / G patches
// in lane groups of G (a power of two), L = N / 3 lanes of a group hold three rows each (rows t,
// t + L, t + 2 L), the others hold zero rows.  Pivot rows pass through a per-warp shared buffer
// behind __syncwarp only; with no CTA barrier in the elimination, one warp's step latency
// (publish, synchronise, load, reciprocal) hides behind the other warps' FMAs, and each pivot
// value loaded feeds three FMAs.  The method: Gauss-Jordan without row
// interchanges on the equilibrated J_K (eliminating the velocity unknowns before the pressure
// unknowns of the saddle-point matrix needs none on these problems), columns rotated by one
// position per step so that the pivot column is always register 0 (no dynamic register
// indexing; after n steps the columns are back in order); a pivot below 1e-3 (entries are O(1)
// after equilibration) flags the patch and the pivoting kernel redoes it.
template <int N, int WPB, int MAXR, typename MT, typename FT>
__global__ void __launch_bounds__(32 * WPB) __maxnreg__(MAXR)
    invert_triples_kernel(Geom g, const int* __restrict__ rowptr, const MT* __restrict__ vv,
                          const MT* __restrict__ vp, const MT* __restrict__ pv, FT* __restrict__ jinv,
                          long long stride, int* __restrict__ flags) {
  constexpr int L = N / 3;
  constexpr int G = L <= 8 ? 8 : 16;
  constexpr int PPW = 32 / G;
  constexpr int NR = (N + 3) / 4 * 4;
  static_assert(N % 3 == 0 && L <= 16, "three rows per lane, at most 16 lanes per patch");
  __shared__ __align__(16) float s_row[WPB][2][PPW][NR];
  __shared__ float s_rs[WPB][PPW][N];
  __shared__ float s_cs[WPB][PPW][N];
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32, h = lane / G, t = lane % G;
  const bool act = t < L;
  const int r0 = t, r1 = t + L, r2 = t + 2 * L;
  const long long groups = (g.n_cells + PPW - 1) / PPW;
  for (long long q = (long long)blockIdx.x * WPB + w; q < groups; q += (long long)gridDim.x * WPB) {
    const long long p = q * PPW + h;
    int cx = 0, cy = 0, cz = 0;
    if (p < g.n_cells) patch_cell(g, p, cx, cy, cz);
    const bool removed = p < g.n_cells && cell_masked(g, cx, cy);
    const bool live = p < g.n_cells && !removed && act;
    float a[N], b[N], c[N];
    if (live) {
      const long long cell = cell_id(g, cx, cy, cz);
      gather_patch_row<N, MT>(g, rowptr, vv, vp, pv, cx, cy, cell, r0, a);
      gather_patch_row<N, MT>(g, rowptr, vv, vp, pv, cx, cy, cell, r1, b);
      gather_patch_row<N, MT>(g, rowptr, vv, vp, pv, cx, cy, cell, r2, c);
    } else {
#pragma unroll
      for (int l = 0; l < N; ++l) {  // identity rows keep idle patches harmless; idle lanes hold zeros
        a[l] = act && r0 == l ? 1.f : 0.f;
        b[l] = act && r1 == l ? 1.f : 0.f;
        c[l] = act && r2 == l ? 1.f : 0.f;
      }
    }
    // equilibration: row scales, then column scales by a butterfly maximum over the group (the
    // scales need no rounding guarantee: the output undoes exactly the scales applied)
    {
      float ma = 0.f, mb = 0.f, mc = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        ma = fmaxf(ma, fabsf(a[l]));
        mb = fmaxf(mb, fabsf(b[l]));
        mc = fmaxf(mc, fabsf(c[l]));
      }
      const float ra = ma > 0.f ? __fdividef(1.f, ma) : 1.f, rb = mb > 0.f ? __fdividef(1.f, mb) : 1.f,
                  rc = mc > 0.f ? __fdividef(1.f, mc) : 1.f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        a[l] *= ra;
        b[l] *= rb;
        c[l] *= rc;
      }
      if (act) {
        s_rs[w][h][r0] = ra;
        s_rs[w][h][r1] = rb;
        s_rs[w][h][r2] = rc;
      }
    }
#pragma unroll
    for (int l = 0; l < N; ++l) {
      float m = fmaxf(fabsf(a[l]), fmaxf(fabsf(b[l]), fabsf(c[l])));
#pragma unroll
      for (int o = G / 2; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      const float cs = m > 0.f ? __fdividef(1.f, m) : 1.f;
      a[l] *= cs;
      b[l] *= cs;
      c[l] *= cs;
      if (t == 0) s_cs[w][h][l] = cs;
    }
    bool bad = false;
    float* buf0 = s_row[w][0][h];
    float* buf1 = s_row[w][1][h];
    triples_phase<N, L, 0>(a, b, c, buf0, buf1, t, bad);
    triples_phase<N, L, 1>(a, b, c, buf0, buf1, t, bad);
    triples_phase<N, L, 2>(a, b, c, buf0, buf1, t, bad);
    const unsigned votes = __ballot_sync(0xffffffffu, bad);
    const bool patch_bad = ((votes >> (h * G)) & ((G == 32 ? 0xffffffffu : (1u << G) - 1u))) != 0u;
    if (live) {
      if (patch_bad) {
        if (t == 0) flags[p] = 1;
      } else {
        // J_K^{-1} = Dc A'^{-1} Dr, column-major: element (row, col) at col * N + row
        FT* out = jinv + p * stride;
        const float ca = s_cs[w][h][r0], cb = s_cs[w][h][r1], cc = s_cs[w][h][r2];
#pragma unroll
        for (int col = 0; col < N; ++col) {
          const float rs = s_rs[w][h][col];
          out[col * N + r0] = cvt<FT>(a[col] * ca * rs);
          out[col * N + r1] = cvt<FT>(b[col] * cb * rs);
          out[col * N + r2] = cvt<FT>(c[col] * cc * rs);
        }
      }
    } else if (removed && act) {
      FT* out = jinv + p * stride;
      const float o0 = patch_entry_dead(g, cx, cy, r0) ? 1.f : 0.f, o1 = patch_entry_dead(g, cx, cy, r1) ? 1.f : 0.f,
                  o2 = patch_entry_dead(g, cx, cy, r2) ? 1.f : 0.f;
      for (int col = 0; col < N; ++col) {
        out[col * N + r0] = cvt<FT>(col == r0 ? o0 : 0.f);
        out[col * N + r1] = cvt<FT>(col == r1 ? o1 : 0.f);
        out[col * N + r2] = cvt<FT>(col == r2 ? o2 : 0.f);
      }
    }
    __syncwarp();
  }
}

// Entry (mu, nu) of J_K (internal local order: 3^d nodes x NV velocity values, node-major, then
// the NP pressure values), gathered from the block-CSR velocity blocks and the per-cell
// velocity-pressure blocks; 0 in the pressure-pressure block; the identity beyond n (padding).
template <typename MT>
__device__ __forceinline__ float patch_entry(const Geom& g, const int* __restrict__ rowptr, const MT* __restrict__ vv,
                                             const MT* __restrict__ vp, const MT* __restrict__ pv, int cx, int cy,
                                             int cz, long long cell, int mu, int nu) {
  const int n = g.npatch, NV = g.NV, dim = g.dim, nloc = g.nloc, vel = nloc * NV;
  const int gr = g.r, gr1 = g.r + 1, npd = g.npd;
  if (mu >= n || nu >= n) return mu == nu ? 1.f : 0.f;
  if (mu < vel) {
    const int i = mu / NV, v = mu - i * NV;
    if (nu < vel) {
      const int j = nu / NV, s2 = nu - j * NV;
      const long long slot = bcsr_slot(g, rowptr, gr * cx + i % gr1, gr * cy + (i / gr1) % gr1, gr * cz + i / (gr1 * gr1),
                                       gr * cx + j % gr1, gr * cy + (j / gr1) % gr1, gr * cz + j / (gr1 * gr1));
      return (float)vv[(slot * NV + v) * NV + s2];
    }
    const int q = nu - vel, a = q / npd, m = q - a * npd;
    const int ta = v / dim, c = v - ta * dim;
    return ta == a ? (float)vp[(((cell * nloc + i) * g.nt + a) * dim + c) * npd + m] : 0.f;
  }
  if (nu >= vel) return 0.f;
  const int q = mu - vel, a = q / npd, m = q - a * npd;
  const int j = nu / NV, s2 = nu - j * NV, tb = s2 / dim, e = s2 - tb * dim;
  return tb == a ? (float)pv[((cell * g.nt + a) * npd + m) * (long long)nloc * dim + j * dim + e] : 0.f;
}

// Register-tiled variant for the larger patches (2D k >= 2, 3D): one CTA per patch, the
// (padded) NPAD x NPAD matrix spread over a T x T grid of threads (T = NPAD / B), each holding a
// B x B tile in registers.  Gauss-Jordan without row interchanges on the equilibrated J_K (the
// velocity unknowns come before the pressure unknowns, as in invert_triples_kernel); a pivot below
// 1e-3 flags the patch for the pivoting kernel.  Step j = cb B + jj runs over column blocks cb
// and, unrolled, their columns jj, so a thread's pivot-row and pivot-column registers are
// compile-time indices: the threads of column block cb publish column j, those of row block cb
// publish row j (unscaled), one barrier per step (double-buffered), then every thread applies
//   a[r][c] -= (f_r / pivot) row[c]   (f_r = the row's entry in column j; pivot row: f = pivot - 1)
// and the threads of column block cb write the new column j (-f_r / pivot; 1 / pivot on the pivot
// row).  B x B FMAs per step read 2 B values from shared memory.
template <int NPAD, int B, typename MT, typename FT>
__global__ void __launch_bounds__((NPAD / B) * (NPAD / B), NPAD <= 64 ? 8 : (NPAD <= 88 ? 4 : (NPAD <= 120 ? 2 : 1)))
    invert_tiles_kernel(Geom g, const int* __restrict__ rowptr, const MT* __restrict__ vv,
                        const MT* __restrict__ vp, const MT* __restrict__ pv, FT* __restrict__ jinv,
                        long long stride, int* __restrict__ flags) {
  constexpr int T = NPAD / B;
  static_assert(NPAD % B == 0 && B % 4 == 0, "tile layout");
  __shared__ __align__(16) float s_col[2][NPAD];
  __shared__ __align__(16) float s_row[2][NPAD];
  __shared__ float s_red[NPAD][T + 1];
  __shared__ float s_rs[NPAD], s_cs[NPAD];
  __shared__ int s_bad;
  const int n = g.npatch;
  const int tid = threadIdx.x, rg = tid % T, cg = tid / T;
  const long long p = blockIdx.x;
  int cx, cy, cz;
  patch_cell(g, p, cx, cy, cz);
  if (g.dim == 2 && cell_masked(g, cx, cy)) {  // removed cell: block-uniform early return
    write_patch_projector(g, cx, cy, jinv + p * stride, tid, blockDim.x);
    return;
  }
  const long long cell = cell_id(g, cx, cy, cz);
  float a[B][B];
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) a[r][c] = patch_entry<MT>(g, rowptr, vv, vp, pv, cx, cy, cz, cell, rg * B + r, cg * B + c);
  if (tid == 0) s_bad = 0;
  // equilibration: row scales (max over the row, reduced over the thread columns), then column
  // scales of the row-scaled matrix
#pragma unroll
  for (int r = 0; r < B; ++r) {
    float mx = 0.f;
#pragma unroll
    for (int c = 0; c < B; ++c) mx = fmaxf(mx, fabsf(a[r][c]));
    s_red[rg * B + r][cg] = mx;
  }
  __syncthreads();
  for (int i = tid; i < NPAD; i += T * T) {
    float mx = 0.f;
    for (int t = 0; t < T; ++t) mx = fmaxf(mx, s_red[i][t]);
    s_rs[i] = mx > 0.f ? 1.f / mx : 1.f;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < B; ++r) {
    const float rs = s_rs[rg * B + r];
#pragma unroll
    for (int c = 0; c < B; ++c) a[r][c] *= rs;
  }
#pragma unroll
  for (int c = 0; c < B; ++c) {
    float mx = 0.f;
#pragma unroll
    for (int r = 0; r < B; ++r) mx = fmaxf(mx, fabsf(a[r][c]));
    s_red[cg * B + c][rg] = mx;
  }
  __syncthreads();
  for (int i = tid; i < NPAD; i += T * T) {
    float mx = 0.f;
    for (int t = 0; t < T; ++t) mx = fmaxf(mx, s_red[i][t]);
    s_cs[i] = mx > 0.f ? 1.f / mx : 1.f;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const float cs = s_cs[cg * B + c];
#pragma unroll
    for (int r = 0; r < B; ++r) a[r][c] *= cs;
  }
  for (int cb = 0; cb < T; ++cb) {
    const bool colown = cg == cb, rowown = rg == cb;
#pragma unroll
    for (int jj = 0; jj < B; ++jj) {
      const int j = cb * B + jj;
      float* col = s_col[jj & 1];
      float* row = s_row[jj & 1];
      if (colown)
#pragma unroll
        for (int r4 = 0; r4 < B / 4; ++r4)
          reinterpret_cast<float4*>(col + rg * B)[r4] =
              make_float4(a[4 * r4][jj], a[4 * r4 + 1][jj], a[4 * r4 + 2][jj], a[4 * r4 + 3][jj]);
      if (rowown)
#pragma unroll
        for (int c4 = 0; c4 < B / 4; ++c4)
          reinterpret_cast<float4*>(row + cg * B)[c4] =
              make_float4(a[jj][4 * c4], a[jj][4 * c4 + 1], a[jj][4 * c4 + 2], a[jj][4 * c4 + 3]);
      __syncthreads();
      const float piv = row[j];
      if (tid == 0 && (!(fabsf(piv) > 1e-3f) || isinf(piv))) s_bad = 1;
      const float inv = 1.f / piv;
      float f[B], q[B];
#pragma unroll
      for (int r4 = 0; r4 < B / 4; ++r4) {
        const float4 v = reinterpret_cast<const float4*>(col + rg * B)[r4];
        f[4 * r4] = v.x;
        f[4 * r4 + 1] = v.y;
        f[4 * r4 + 2] = v.z;
        f[4 * r4 + 3] = v.w;
        const float4 w = reinterpret_cast<const float4*>(row + cg * B)[r4];
        q[4 * r4] = w.x;
        q[4 * r4 + 1] = w.y;
        q[4 * r4 + 2] = w.z;
        q[4 * r4 + 3] = w.w;
      }
#pragma unroll
      for (int r = 0; r < B; ++r) {
        const float gr = ((rowown && r == jj) ? f[r] - 1.f : f[r]) * inv;
#pragma unroll
        for (int c = 0; c < B; ++c) a[r][c] = fmaf(-gr, q[c], a[r][c]);
      }
      if (colown)
#pragma unroll
        for (int r = 0; r < B; ++r) a[r][jj] = (rowown && r == jj) ? inv : -f[r] * inv;
    }
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) flags[p] = 1;
    return;
  }
  // J_K^{-1} = Dc A'^{-1} Dr, column-major: element (row, col) at col * n + row
  FT* out = jinv + p * stride;
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const int colx = cg * B + c;
    if (colx >= n) continue;
    const float rc = s_rs[colx];
#pragma unroll
    for (int r = 0; r < B; ++r) {
      const int rowx = rg * B + r;
      if (rowx < n) out[(long long)colx * n + rowx] = cvt<FT>(a[r][c] * s_cs[rowx] * rc);
    }
  }
}

// The register-tiled elimination of invert_tiles_kernel for patches too large for one CTA's
// register file (3D k = 2: n_K = 255, padded to NPAD = 256): a cluster of two CTAs per patch,
// CTA q holding columns [q NPAD/2, (q + 1) NPAD/2) as B x B tiles of a (NPAD/B) x (NPAD/2B)
// thread grid.  Per step the threads owning column j write it into both CTAs' shared memory
// (the other CTA's through the cluster's distributed shared memory), the threads of row block
// j / B publish their half of row j locally, and one cluster barrier separates publication from
// use (double-buffered, as in the one-CTA kernel).  The pivot is read from the column.  Row
// scales need both halves: each CTA sends its row maxima to the other before the scales are
// formed, so both CTAs scale identically.  Same method and flagging as invert_tiles_kernel.
template <int NPAD, int B, typename MT, typename FT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__((NPAD / B) * (NPAD / B / 2), 1)
    invert_tiles2_kernel(Geom g, const int* __restrict__ rowptr, const MT* __restrict__ vv,
                         const MT* __restrict__ vp, const MT* __restrict__ pv, FT* __restrict__ jinv,
                         long long stride, int* __restrict__ flags) {
  namespace cg = cooperative_groups;
  constexpr int TR = NPAD / B, TC = NPAD / B / 2, HALF = NPAD / 2;
  static_assert(NPAD % (2 * B) == 0 && B % 4 == 0, "tile layout");
  __shared__ __align__(16) float s_col[2][NPAD];
  __shared__ __align__(16) float s_row[2][HALF];
  __shared__ float s_red[NPAD][TR + 1];
  __shared__ float s_rmax[2][NPAD];  // row maxima of each CTA's half
  __shared__ float s_rs[NPAD], s_cs[NPAD];
  __shared__ int s_bad;
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank(), other = q ^ 1;
  const int n = g.npatch;
  const int tid = threadIdx.x, rg = tid % TR, cgl = tid / TR, cgg = q * TC + cgl;
  const long long p = blockIdx.x / 2;
  int cx, cy, cz;
  patch_cell(g, p, cx, cy, cz);
  const long long cell = cell_id(g, cx, cy, cz);
  float a[B][B];
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) a[r][c] = patch_entry<MT>(g, rowptr, vv, vp, pv, cx, cy, cz, cell, rg * B + r, cgg * B + c);
  if (tid == 0) s_bad = 0;
  // row scales: this half's maxima, exchanged with the other CTA
#pragma unroll
  for (int r = 0; r < B; ++r) {
    float mx = 0.f;
#pragma unroll
    for (int c = 0; c < B; ++c) mx = fmaxf(mx, fabsf(a[r][c]));
    s_red[rg * B + r][cgl] = mx;
  }
  __syncthreads();
  float* rmax_other = cl.map_shared_rank(&s_rmax[q][0], other);
  for (int i = tid; i < NPAD; i += TR * TC) {
    float mx = 0.f;
    for (int t = 0; t < TC; ++t) mx = fmaxf(mx, s_red[i][t]);
    s_rmax[q][i] = mx;
    rmax_other[i] = mx;
  }
  cl.sync();
  for (int i = tid; i < NPAD; i += TR * TC) {
    const float mx = fmaxf(s_rmax[0][i], s_rmax[1][i]);
    s_rs[i] = mx > 0.f ? 1.f / mx : 1.f;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < B; ++r) {
    const float rs = s_rs[rg * B + r];
#pragma unroll
    for (int c = 0; c < B; ++c) a[r][c] *= rs;
  }
  // column scales: whole columns are local; both CTAs need all of them for the output
#pragma unroll
  for (int c = 0; c < B; ++c) {
    float mx = 0.f;
#pragma unroll
    for (int r = 0; r < B; ++r) mx = fmaxf(mx, fabsf(a[r][c]));
    s_red[cgl * B + c][rg] = mx;
  }
  __syncthreads();
  float* cs_other = cl.map_shared_rank(&s_cs[0], other);
  for (int i = tid; i < HALF; i += TR * TC) {
    float mx = 0.f;
    for (int t = 0; t < TR; ++t) mx = fmaxf(mx, s_red[i][t]);
    const float cs = mx > 0.f ? 1.f / mx : 1.f;
    s_cs[q * HALF + i] = cs;
    cs_other[q * HALF + i] = cs;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const float cs = s_cs[q * HALF + cgl * B + c];
#pragma unroll
    for (int r = 0; r < B; ++r) a[r][c] *= cs;
  }
  float* col_other[2] = {cl.map_shared_rank(&s_col[0][0], other), cl.map_shared_rank(&s_col[1][0], other)};
  for (int cb = 0; cb < TR; ++cb) {
    const bool colown = cgg == cb, rowown = rg == cb;
#pragma unroll
    for (int jj = 0; jj < B; ++jj) {
      const int j = cb * B + jj;
      float* col = s_col[jj & 1];
      float* row = s_row[jj & 1];
      if (colown)
#pragma unroll
        for (int r4 = 0; r4 < B / 4; ++r4) {
          const float4 v = make_float4(a[4 * r4][jj], a[4 * r4 + 1][jj], a[4 * r4 + 2][jj], a[4 * r4 + 3][jj]);
          reinterpret_cast<float4*>(col + rg * B)[r4] = v;
          reinterpret_cast<float4*>(col_other[jj & 1] + rg * B)[r4] = v;
        }
      if (rowown)
#pragma unroll
        for (int c4 = 0; c4 < B / 4; ++c4)
          reinterpret_cast<float4*>(row + cgl * B)[c4] =
              make_float4(a[jj][4 * c4], a[jj][4 * c4 + 1], a[jj][4 * c4 + 2], a[jj][4 * c4 + 3]);
      cl.sync();
      const float piv = col[j];
      if (tid == 0 && (!(fabsf(piv) > 1e-3f) || isinf(piv))) s_bad = 1;
      const float inv = 1.f / piv;
      float f[B], qv[B];
#pragma unroll
      for (int r4 = 0; r4 < B / 4; ++r4) {
        const float4 v = reinterpret_cast<const float4*>(col + rg * B)[r4];
        f[4 * r4] = v.x;
        f[4 * r4 + 1] = v.y;
        f[4 * r4 + 2] = v.z;
        f[4 * r4 + 3] = v.w;
        const float4 w = reinterpret_cast<const float4*>(row + cgl * B)[r4];
        qv[4 * r4] = w.x;
        qv[4 * r4 + 1] = w.y;
        qv[4 * r4 + 2] = w.z;
        qv[4 * r4 + 3] = w.w;
      }
#pragma unroll
      for (int r = 0; r < B; ++r) {
        const float gr = ((rowown && r == jj) ? f[r] - 1.f : f[r]) * inv;
#pragma unroll
        for (int c = 0; c < B; ++c) a[r][c] = fmaf(-gr, qv[c], a[r][c]);
      }
      if (colown)
#pragma unroll
        for (int r = 0; r < B; ++r) a[r][jj] = (rowown && r == jj) ? inv : -f[r] * inv;
    }
  }
  __syncthreads();
  const bool bad = s_bad != 0;
  // neither CTA may leave while the other can still address its shared memory
  cl.sync();
  if (bad) {
    if (tid == 0 && q == 0) flags[p] = 1;
    return;
  }
  // J_K^{-1} = Dc A'^{-1} Dr, column-major: element (row, col) at col * n + row
  FT* out = jinv + p * stride;
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const int colx = cgg * B + c;
    if (colx >= n) continue;
    const float rc = s_rs[colx];
#pragma unroll
    for (int r = 0; r < B; ++r) {
      const int rowx = rg * B + r;
      if (rowx < n) {
        out[(long long)colx * n + rowx] = cvt<FT>(a[r][c] * s_cs[rowx] * rc);
      }
    }
  }
}

// ------------------------------------------------------------------ smoother
template <typename VT, typename FT, int RPL, int CB>
__global__ void __launch_bounds__(512) vanka_colour_kernel(Geom g, int colour, const FT* __restrict__ jinv,
                                                           long long stride, const VT* __restrict__ r,
                                                           VT* __restrict__ z, VT scale) {
  pdl_wait();
  using AT = typename AccT<VT>::type;
  const int n = g.npatch;
  const int wpb = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long li = (long long)blockIdx.x * wpb + wid;
  const long long cnt = g.coff[colour + 1] - g.coff[colour];
  extern __shared__ unsigned char smem_raw[];
  VT* rl = reinterpret_cast<VT*>(smem_raw) + wid * n;
  if (li >= cnt) return;
  const long long p = g.coff[colour] + li;
  const int* cc = g.ccount[colour];
  long long rem = li;
  const int jx = (int)(rem % cc[0]);
  rem /= cc[0];
  const int jy = (int)(rem % cc[1]);
  const int jz = (int)(rem / cc[1]);
  const int cx = 2 * jx + (colour & 1), cy = 2 * jy + ((colour >> 1) & 1), cz = 2 * jz + ((colour >> 2) & 1);
  long long gi[RPL];
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int row = lane + 32 * t;
    gi[t] = row < n ? patch_dof(g, cx, cy, cz, row) : 0;
    if (row < n) rl[row] = r[gi[t]];
  }
  __syncwarp();
  const FT* A = jinv + p * stride;
  AT acc[RPL];
#pragma unroll
  for (int t = 0; t < RPL; ++t) acc[t] = 0;
  // stream the column-major J_K^{-1}: CB columns of loads are issued before their
  // FMAs so that each warp keeps CB * n values in flight
  int col = 0;
  for (; col + CB <= n; col += CB) {
    FT v[CB][RPL];
#pragma unroll
    for (int u = 0; u < CB; ++u)
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        v[u][t] = row < n ? A[(long long)(col + u) * n + row] : cvt<FT>(0.f);
      }
#pragma unroll
    for (int u = 0; u < CB; ++u) {
      const AT rc = (AT)rl[col + u];
#pragma unroll
      for (int t = 0; t < RPL; ++t) acc[t] += cvt<AT>(v[u][t]) * rc;
    }
  }
  for (; col < n; ++col) {
    const AT rc = (AT)rl[col];
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int row = lane + 32 * t;
      if (row < n) acc[t] += cvt<AT>(A[(long long)col * n + row]) * rc;
    }
  }
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int row = lane + 32 * t;
    if (row < n) z[gi[t]] += scale * (VT)acc[t];
  }
}

// ------------------------------------------------------------------ bulk-copy colour kernel
// The same y_K = J_K^{-1} R_K r, z += y_K as vanka_colour_kernel, with each patch's factor
// streamed into shared memory by the bulk-copy engine: one elected thread keeps S patches
// in flight per CTA (cp.async.bulk completing on an mbarrier per stage) while the CTA, one
// thread per row, computes the previous patch from shared memory.  Every wait has an
// iteration limit; a CTA that reaches it raises g_colour_timeout, waits (again with a
// limit) for its own copies still in flight, and returns.

// 1: a wait for a factor copy reached its limit; 2: in addition, a copy already in flight
// had not landed when its drain wait gave up (the CTA then returned with it pending).
__device__ int g_colour_timeout;

constexpr long long kBarrierSpins = 1LL << 22;
// limit of the waits for a patch's factor (read at run time, so graph replays see changes;
// 0 makes every such wait give up at once)
__device__ long long g_colour_wait_spins = kBarrierSpins;
// Limit of the drain waits after giving up.  A bulk copy that has been issued always lands
// unless the context has already faulted, and a CTA that returned before its copies landed
// would leave them writing into shared memory that the next CTA on the SM may own.  So the
// drain wait does not depend on the fault-injection limit above: it backs off with
// __nanosleep and gives up only after about 2^24 sleeps of up to 1 us (tens of seconds),
// a bound no healthy copy comes near; it stays finite so that no wait in this kernel is
// unbounded.
constexpr long long kDrainSleeps = 1LL << 24;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool barrier_wait(unsigned bar, unsigned phase, long long spins) {
  for (long long i = 0; i < spins; ++i) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ bool drain_wait(unsigned bar, unsigned phase) {
  unsigned ns = 32;
  for (long long i = 0; i < kDrainSleeps; ++i) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
  return false;
}

__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Shared memory: S mbarriers (128 B reserved), the gathered residual (n values, padded to
// 128 B), then S stages of stage_bytes each (128-byte aligned).
template <typename VT>
__host__ __device__ __forceinline__ unsigned bulk_rl_bytes(int n) {
  return (unsigned)((n * sizeof(VT) + 127) / 128 * 128);
}

// RPT adjacent rows of a column-major factor column as accumulator values (one vector load for
// RPT = 2: rows 2t, 2t + 1 are adjacent, and the address is aligned for even n).
template <typename AT, typename FT, int RPT>
__device__ __forceinline__ void load_rows(const FT* p, AT (&a)[RPT]) {
  if constexpr (RPT == 1) {
    a[0] = cvt<AT>(p[0]);
  } else if constexpr (std::is_same<FT, float>::value) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    a[0] = v.x;
    a[1] = v.y;
  } else if constexpr (std::is_same<FT, double>::value) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    a[0] = v.x;
    a[1] = v.y;
  } else {
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    a[0] = v.x;
    a[1] = v.y;
  }
}

template <typename VT, typename FT, int S, int RPT>
__global__ void __launch_bounds__(1024) vanka_colour_bulk_kernel(Geom g, int colour, const FT* __restrict__ jinv,
                                                                 long long stride, const VT* __restrict__ r,
                                                                 VT* __restrict__ z, VT scale, unsigned bytes,
                                                                 unsigned stage_bytes) {
  pdl_wait();
  using AT = typename AccT<VT>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int n = g.npatch;
  const int tid = threadIdx.x;
  const long long cnt = g.coff[colour + 1] - g.coff[colour];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);
  VT* rl = reinterpret_cast<VT*>(smem_raw + 128);  // two buffers of n values
  unsigned char* stages = smem_raw + 128 + bulk_rl_bytes<VT>(2 * n);
  const long long first = blockIdx.x, step = gridDim.x;
  const FT* base = jinv + g.coff[colour] * stride;
  const int* cc = g.ccount[colour];
  const long long spins = g_colour_wait_spins;
  // thread tid owns rows row0 .. row0 + RPT - 1 of every patch (RPT = 2 only for even n)
  const int row0 = tid * RPT;
  const bool act = row0 < n;
  auto dof = [&](long long li, int row) {
    long long rem = li;
    const int jx = (int)(rem % cc[0]);
    rem /= cc[0];
    const int jy = (int)(rem % cc[1]);
    const int jz = (int)(rem / cc[1]);
    return patch_dof(g, 2 * jx + (colour & 1), 2 * jy + ((colour >> 1) & 1), 2 * jz + ((colour >> 2) & 1), row);
  };
  if (tid == 0) {
    for (int s = 0; s < S; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + s)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // S - 1 patches ahead; iteration it issues patch it + S - 1
    for (int s = 0; s + 1 < S; ++s) {
      const long long li = first + s * step;
      if (li < cnt) bulk_load(smem_u32(stages + s * stage_bytes), base + li * stride, bytes, smem_u32(bar + s));
    }
  }
  __syncthreads();  // no thread may poll a barrier before thread 0 has initialised it
  long long gi[RPT];
  VT zold[RPT];
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    gi[u] = 0;
    zold[u] = 0;
  }
  if (act && first < cnt) {
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      gi[u] = dof(first, row0 + u);
      rl[row0 + u] = r[gi[u]];
      zold[u] = z[gi[u]];  // no other patch of this colour touches these entries
    }
  }
  int it = 0;
  for (long long li = first; li < cnt; li += step, ++it) {
    const int s = it % S;
    const bool ok = barrier_wait(smem_u32(bar + s), (unsigned)((it / S) & 1), spins);
    // one barrier per patch: publishes rl[it & 1], frees the stage of patch it - 1
    if (__syncthreads_or(!ok)) {
      // give up: flag it, let the copies already issued land, then leave
      if (tid == 0) {
        atomicExch(&g_colour_timeout, 1);
        for (int j = it; j < it + S - 1; ++j) {
          if (first + (long long)j * step >= cnt) break;
          if (!drain_wait(smem_u32(bar + (j % S)), (unsigned)((j / S) & 1))) atomicExch(&g_colour_timeout, 2);
        }
      }
      __syncthreads();
      return;
    }
    if (tid == 0) {
      const int j = it + S - 1;
      const long long lj = first + (long long)j * step;
      if (lj < cnt) bulk_load(smem_u32(stages + (j % S) * stage_bytes), base + lj * stride, bytes, smem_u32(bar + (j % S)));
    }
    // gather of the next patch, in flight while this one is computed
    const long long ln = li + step;
    long long gn[RPT];
    VT rn[RPT], zn[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      gn[u] = 0;
      rn[u] = 0;
      zn[u] = 0;
    }
    if (act && ln < cnt) {
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        gn[u] = dof(ln, row0 + u);
        rn[u] = r[gn[u]];
        zn[u] = z[gn[u]];
      }
    }
    if (act) {
      const FT* A = reinterpret_cast<const FT*>(stages + s * stage_bytes);
      const VT* rc = rl + (it & 1) * n;
      AT acc[RPT];
#pragma unroll
      for (int u = 0; u < RPT; ++u) acc[u] = 0;
#pragma unroll 6
      for (int col = 0; col < n; ++col) {
        AT av[RPT];
        load_rows<AT, FT, RPT>(A + col * n + row0, av);
        const AT rv = (AT)rc[col];
#pragma unroll
        for (int u = 0; u < RPT; ++u) acc[u] += av[u] * rv;
      }
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        z[gi[u]] = zold[u] + scale * (VT)acc[u];
        rl[((it + 1) & 1) * n + row0 + u] = rn[u];
      }
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      gi[u] = gn[u];
      zold[u] = zn[u];
    }
  }
}

template <typename VT>
__global__ void vanka_update_kernel(Geom g, VT* __restrict__ d, VT* __restrict__ z, double omega) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.N) return;
  int mult = 1;
  if (t < g.nvel) {
    const long long node = t / g.NV;
    const int ix = (int)(node % g.nn[0]);
    const int iy = (int)((node / g.nn[0]) % g.nn[1]);
    const int iz = (int)(node / ((long long)g.nn[0] * g.nn[1]));
    mult = node_multiplicity(g, ix, iy, iz);
  }
  d[t] += (VT)omega * z[t] / (VT)mult;
  z[t] = 0;
}

}  // namespace

template <typename MT, typename VT>
void apply_operator(const Geom& g, const int* rowptr, const int* colidx, const MT* vv, const MT* vp, const MT* pv,
                    const VT* x, const VT* b, VT* out, cudaStream_t st) {
  if (g.dim == 2) {
    launch_k(op_vel_rows<2, MT, VT>, grid_for(g.nvel, 256), 256, 0, st, g, rowptr, colidx, vv, vp, x, b, out);
    launch_k(op_pres_rows<2, MT, VT>, grid_for(g.npres, 256), 256, 0, st, g, pv, x, b, out);
  } else {
    launch_k(op_vel_rows<3, MT, VT>, grid_for(g.nvel, 256), 256, 0, st, g, rowptr, colidx, vv, vp, x, b, out);
    launch_k(op_pres_rows<3, MT, VT>, grid_for(g.npres, 256), 256, 0, st, g, pv, x, b, out);
  }
}

bool kron_supported(const Geom& g) { return g.dim == 2 && g.r == 2 && g.nt >= 2 && g.nt <= 5; }

void kron_split(const Geom& g, long long nnzb, const double* vv, const TimeData& td, float* Mk, float* Ak,
                cudaStream_t st) {
  int as = 0, bs = 1;
  for (int a = 0; a < g.nt; ++a)
    for (int b = 0; b < g.nt; ++b)
      if (a != b && std::fabs(td.T[a][b]) > std::fabs(td.T[as][bs])) {
        as = a;
        bs = b;
      }
  kron_split_kernel<<<grid_for(nnzb, 256), 256, 0, st>>>(g, nnzb, vv, td, as, bs, Mk, Ak);
  STG_LAUNCH_OK();
}

void apply_operator_kron(const Geom& g, const TimeData& td, const float* Mk, const float* Ak,
                         const float* vp, const float* pv, const float* x, const float* b, float* out,
                         cudaStream_t st) {
  if (g.n_nodes * g.nt >= (1LL << 31)) throw Error{STG_EINVAL, "level too large for 32-bit row indices"};
  TimeF tf;
  for (int a = 0; a < 5; ++a)
    for (int c = 0; c < 5; ++c) tf.T[a][c] = (float)td.T[a][c];
  const unsigned grid = grid_for(g.n_nodes * g.nt, 256);
  switch (g.nt) {
    case 2: launch_k(op_vel_rows_kron<2>, grid, 256, 0, st, g, tf, Mk, Ak, vp, x, b, out); break;
    case 3: launch_k(op_vel_rows_kron<3>, grid, 256, 0, st, g, tf, Mk, Ak, vp, x, b, out); break;
    case 4: launch_k(op_vel_rows_kron<4>, grid, 256, 0, st, g, tf, Mk, Ak, vp, x, b, out); break;
    default: launch_k(op_vel_rows_kron<5>, grid, 256, 0, st, g, tf, Mk, Ak, vp, x, b, out); break;
  }
  launch_k(op_pres_rows<2, float, float>, grid_for(g.npres, 256), 256, 0, st, g, pv, x, b, out);
}

size_t invert_scratch_bytes(const Geom& g, int compute_f32) {
  const int n = g.npatch;
  const size_t cs = compute_f32 ? sizeof(float) : sizeof(double);
  const size_t full = (size_t)n * n * cs + (size_t)3 * n * cs + (size_t)n * sizeof(int) + 64;
  if (full <= 200 * 1024) return 0;
  const long long chunk = g.n_cells < 1024 ? g.n_cells : 1024;
  return cs * n * n * chunk;
}

template <typename FT>
void invert_patches(const Geom& g, const int* rowptr, const double* vv, const double* vp, const double* pv,
                    const float* vv32, const float* vp32, const float* pv32, FT* jinv, int compute_f32, int* status,
                    void* scratch, int* flags, cudaStream_t st) {
  const int n = g.npatch;
  const long long stride = patch_stride(n);
  const int threads = n <= 63 ? 128 : 256;
  int sms = 0, dev = 0;
  STG_CUDA_OK(cudaGetDevice(&dev));
  STG_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int* only = nullptr;
  if (compute_f32 && g.dim == 2 && n <= 42 && flags) {
    // register-resident pivot-free pass, then the pivoting kernel for flagged patches only
    STG_CUDA_OK(cudaMemsetAsync(flags, 0, sizeof(int) * g.n_cells, st));
    // one CTA per PPB patches (not a resident-capped grid): the set-up runs this beside other
    // streams' kernels, and a static split over resident CTAs would wait for the busiest SM
    auto run = [&](auto kern, int ppb, int nthreads, auto* V, auto* VP, auto* PV) {
      const long long grid = std::max<long long>(1, std::min<long long>((g.n_cells + ppb - 1) / ppb, 0x7fffffffLL));
      kern<<<(unsigned)grid, nthreads, 0, st>>>(g, rowptr, V, VP, PV, jinv, stride, flags);
      STG_LAUNCH_OK();
    };
    // warp-synchronous kernels, 4 patches a warp (n = 21) or 2 (n = 42).  At n = 42 registers
    // are allocated per SM sub-partition (16K each): 168 a thread leave 3 warps on each, 200 only
    // 2.  The 168 cap costs a few spill slots outside the elimination loop and measured faster
    // than both the spill-free 200 cap and the two-rows-per-thread CTA kernel this replaced
    // (finest channel set-up 4.98 ms against 5.23 and 5.29 ms).
    if (vv32) {
      if (n == 21) run(invert_triples_kernel<21, 4, 128, float, FT>, 16, 128, vv32, vp32, pv32);
      else run(invert_triples_kernel<42, 2, 168, float, FT>, 4, 64, vv32, vp32, pv32);
    } else {
      if (n == 21) run(invert_triples_kernel<21, 4, 128, double, FT>, 16, 128, vv, vp, pv);
      else run(invert_triples_kernel<42, 2, 168, double, FT>, 4, 64, vv, vp, pv);
    }
    only = flags;
  } else if (compute_f32 && flags &&
             (n == 63 || n == 84 || n == 105 || n == 85 || n == 170 || n == 60 || n == 120 || n == 180 ||
              (n == 255 && g.dim == 3))) {  // the cluster kernel has no removed-cell path (3D only)
    // larger patches: register tiles, pivot-free, then the pivoting kernel for flagged patches
    STG_CUDA_OK(cudaMemsetAsync(flags, 0, sizeof(int) * g.n_cells, st));
    auto tiles = [&](auto kern, int threads_t, auto* V, auto* VP, auto* PV) {
      kern<<<(unsigned)g.n_cells, threads_t, 0, st>>>(g, rowptr, V, VP, PV, jinv, stride, flags);
      STG_LAUNCH_OK();
    };
    const bool f32src = vv32 != nullptr;
    if (n == 63 || n == 60) {
      if (f32src) tiles(invert_tiles_kernel<64, 8, float, FT>, 64, vv32, vp32, pv32);
      else tiles(invert_tiles_kernel<64, 8, double, FT>, 64, vv, vp, pv);
    } else if (n == 120) {  // order 4, k = 1
      if (f32src) tiles(invert_tiles_kernel<120, 8, float, FT>, 225, vv32, vp32, pv32);
      else tiles(invert_tiles_kernel<120, 8, double, FT>, 225, vv, vp, pv);
    } else if (n == 180) {  // order 4, k = 2: 12 x 12 tiles keep the 256 threads within the register file
      if (f32src) tiles(invert_tiles_kernel<192, 12, float, FT>, 256, vv32, vp32, pv32);
      else tiles(invert_tiles_kernel<192, 12, double, FT>, 256, vv, vp, pv);
    } else if (n == 255) {  // 3D k = 2: a cluster of two CTAs per patch
      const unsigned grid2 = (unsigned)(2 * g.n_cells);
      if (f32src)
        invert_tiles2_kernel<256, 8, float, FT><<<grid2, 512, 0, st>>>(g, rowptr, vv32, vp32, pv32, jinv, stride, flags);
      else
        invert_tiles2_kernel<256, 8, double, FT><<<grid2, 512, 0, st>>>(g, rowptr, vv, vp, pv, jinv, stride, flags);
      STG_LAUNCH_OK();
    } else if (n == 84 || n == 85) {
      if (f32src) tiles(invert_tiles_kernel<88, 8, float, FT>, 121, vv32, vp32, pv32);
      else tiles(invert_tiles_kernel<88, 8, double, FT>, 121, vv, vp, pv);
    } else if (n == 105) {
      if (f32src) tiles(invert_tiles_kernel<112, 8, float, FT>, 196, vv32, vp32, pv32);
      else tiles(invert_tiles_kernel<112, 8, double, FT>, 196, vv, vp, pv);
    } else {
      if (f32src) tiles(invert_tiles_kernel<176, 8, float, FT>, 484, vv32, vp32, pv32);
      else tiles(invert_tiles_kernel<176, 8, double, FT>, 484, vv, vp, pv);
    }
    only = flags;
  }
  auto launch = [&](auto tag) {
    using CT = decltype(tag);
    const size_t per_warp = ((size_t)n * n + 3 * n) * sizeof(CT) + (size_t)n * sizeof(int);
    const int wpb = (int)std::min<size_t>(8, (200 * 1024) / per_warp);
    // FP64 elimination is FMA-throughput bound and wants more warps per SM than a
    // warp-per-patch layout leaves; it keeps the CTA-per-patch kernel.
    if (sizeof(CT) == 4 && wpb >= 4) {
      const size_t sm = per_warp * wpb;
      STG_CUDA_OK(cudaFuncSetAttribute(invert_warp_kernel<CT, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)std::max<size_t>(sm, 48 * 1024)));
      int per_sm = 0;
      STG_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, invert_warp_kernel<CT, FT>, 32 * wpb, sm));
      const long long want = (g.n_cells + wpb - 1) / wpb;
      const long long grid = std::max<long long>(1, std::min<long long>(want, (long long)sms * std::max(per_sm, 1)));
      invert_warp_kernel<CT, FT><<<(unsigned)grid, 32 * wpb, sm, st>>>(g, rowptr, vv, vp, pv, jinv, stride, status,
                                                                       compute_f32, only);
      STG_LAUNCH_OK();
      return;
    }
    const size_t tail = (size_t)3 * n * sizeof(CT) + (size_t)n * sizeof(int) + 64;
    const size_t full = (size_t)n * n * sizeof(CT) + tail;
    // the attribute is a per-function maximum: never set it below the 48 KB default
    STG_CUDA_OK(cudaFuncSetAttribute(invert_kernel<CT, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(full <= 200 * 1024 ? full : tail, 48 * 1024)));
    if (full <= 200 * 1024) {
      invert_kernel<CT, FT><<<(unsigned)g.n_cells, threads, full, st>>>(g, 0, rowptr, vv, vp, pv, jinv, stride,
                                                                        status, compute_f32, (CT*)nullptr, only);
      STG_LAUNCH_OK();
    } else {
      // matrix too large for shared memory: caller-provided global scratch, in chunks
      if (!scratch) throw Error{STG_EINVAL, "local inverse needs scratch memory"};
      const long long chunk = g.n_cells < 1024 ? g.n_cells : 1024;
      for (long long p0 = 0; p0 < g.n_cells; p0 += chunk) {
        const long long cnt = g.n_cells - p0 < chunk ? g.n_cells - p0 : chunk;
        invert_kernel<CT, FT><<<(unsigned)cnt, threads, tail, st>>>(g, p0, rowptr, vv, vp, pv, jinv, stride,
                                                                    status, compute_f32, (CT*)scratch, only);
        STG_LAUNCH_OK();
      }
    }
  };
  if (compute_f32)
    launch(float{});
  else
    launch(double{});
}

namespace {

struct BulkShape {
  int stages, ctas_per_sm, rows_per_thread;
};
constexpr BulkShape kBulkShapes[kColourVariants - kColourWarpVariants] = {
    {4, 32, 1}, {3, 32, 1}, {2, 32, 1}, {6, 32, 1}, {4, 32, 2}, {3, 32, 2}, {2, 32, 2}, {6, 32, 2}};

template <typename VT, typename FT, int S, int RPT>
bool launch_bulk(const Geom& g, int colour, const FT* jinv, const VT* r, VT* z, VT scale, cudaStream_t st,
                 int ctas_per_sm) {
  const int n = g.npatch;
  if (RPT == 2 && (n & 1)) return false;  // two rows per thread need an even patch size
  const long long cnt = g.coff[colour + 1] - g.coff[colour];
  const long long stride = patch_stride(n);
  const unsigned bytes = (unsigned)((n * n * sizeof(FT) + 15) / 16 * 16);  // <= stride * sizeof(FT)
  const unsigned stage_bytes = (bytes + 127) / 128 * 128;
  const size_t smem = 128 + bulk_rl_bytes<VT>(2 * n) + (size_t)S * stage_bytes;
  const int threads = ((n + RPT - 1) / RPT + 31) / 32 * 32;
  if (smem > 200 * 1024 || threads > 1024) return false;
  // queried per launch (a host-side attribute read): contexts on different devices may share
  // this process
  int sms = 0, dev = 0;
  STG_CUDA_OK(cudaGetDevice(&dev));
  STG_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (smem > 48 * 1024)
    STG_CUDA_OK(cudaFuncSetAttribute(vanka_colour_bulk_kernel<VT, FT, S, RPT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  // every CTA resident at once: the grid is capped by the occupancy the launch can reach
  int resident = 0;
  STG_CUDA_OK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, vanka_colour_bulk_kernel<VT, FT, S, RPT>,
                                                            threads, smem));
  if (resident < 1) return false;
  const long long want = (long long)sms * std::min(ctas_per_sm, resident);
  const unsigned grid = (unsigned)(cnt < want ? cnt : want);
  // an ordinary launch: the grid is one wave with a static split of the patches, which needs the
  // CTAs spread evenly over idle SMs; scheduled early into the SMs that the previous kernel frees
  // first, some SMs would take two CTAs and the launch would wait for them
  const OverlapScope serial(false);
  launch_k(vanka_colour_bulk_kernel<VT, FT, S, RPT>, grid, threads, smem, st, g, colour, jinv, stride, r, z, scale, bytes,
           stage_bytes);
  return true;
}

}  // namespace

void set_colour_wait_limit(long long spins) {
  STG_CUDA_OK(cudaMemcpyToSymbol(g_colour_wait_spins, &spins, sizeof(spins)));
}

bool colour_kernel_timed_out(cudaStream_t st) {
  int h = 0;
  STG_CUDA_OK(cudaMemcpyFromSymbolAsync(&h, g_colour_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  STG_CUDA_OK(cudaStreamSynchronize(st));
  if (h) {
    const int zero = 0;
    STG_CUDA_OK(cudaMemcpyToSymbolAsync(g_colour_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
    STG_CUDA_OK(cudaStreamSynchronize(st));
  }
  return h != 0;
}

template <typename VT, typename FT>
void vanka_colour(const Geom& g, int colour, const FT* jinv, const VT* r, VT* z, VT scale, cudaStream_t st,
                  int variant) {
  const long long cnt = g.coff[colour + 1] - g.coff[colour];
  if (cnt == 0) return;
  if (variant >= kColourWarpVariants) {
    const BulkShape b = kBulkShapes[(variant - kColourWarpVariants) % (kColourVariants - kColourWarpVariants)];
    bool done = false;
    if (b.rows_per_thread == 2) {
      if (b.stages == 2)
        done = launch_bulk<VT, FT, 2, 2>(g, colour, jinv, r, z, scale, st, b.ctas_per_sm);
      else if (b.stages == 3)
        done = launch_bulk<VT, FT, 3, 2>(g, colour, jinv, r, z, scale, st, b.ctas_per_sm);
      else if (b.stages == 4)
        done = launch_bulk<VT, FT, 4, 2>(g, colour, jinv, r, z, scale, st, b.ctas_per_sm);
      else
        done = launch_bulk<VT, FT, 6, 2>(g, colour, jinv, r, z, scale, st, b.ctas_per_sm);
    }
    if (!done) {  // one row per thread (also for an odd patch size)
      if (b.stages == 2)
        done = launch_bulk<VT, FT, 2, 1>(g, colour, jinv, r, z, scale, st, b.ctas_per_sm);
      else if (b.stages == 3)
        done = launch_bulk<VT, FT, 3, 1>(g, colour, jinv, r, z, scale, st, b.ctas_per_sm);
      else if (b.stages == 4)
        done = launch_bulk<VT, FT, 4, 1>(g, colour, jinv, r, z, scale, st, b.ctas_per_sm);
      else
        done = launch_bulk<VT, FT, 6, 1>(g, colour, jinv, r, z, scale, st, b.ctas_per_sm);
    }
    if (done) return;
    variant = kColourWarpDefault;  // patch too large for the staged form
  }
  const int n = g.npatch;
  const long long stride = patch_stride(n);
  const int cb_idx = (variant / 3) % 3, th_idx = variant % 3;
  const int threads = 128 << th_idx, wpb = threads / 32;
  const size_t sm = (size_t)wpb * n * sizeof(VT);
  const unsigned grid = grid_for(cnt, wpb);
#define STG_VC(RPL, CB) \
  launch_k(vanka_colour_kernel<VT, FT, RPL, CB>, grid, threads, sm, st, g, colour, jinv, stride, r, z, scale)
#define STG_VCB(RPL)      \
  if (cb_idx == 0)        \
    STG_VC(RPL, 4);       \
  else if (cb_idx == 1)   \
    STG_VC(RPL, 8);       \
  else                    \
    STG_VC(RPL, 16)
  if (n <= 32) {
    STG_VCB(1);
  } else if (n <= 64) {
    STG_VCB(2);
  } else if (n <= 96) {
    STG_VCB(3);
  } else if (n <= 128) {
    STG_VCB(4);
  } else if (n <= 192) {
    STG_VCB(6);
  } else {
    STG_VCB(8);
  }
#undef STG_VCB
#undef STG_VC
}

template <typename VT>
void vanka_update(const Geom& g, VT* d, VT* z, double omega, cudaStream_t st) {
  launch_k(vanka_update_kernel<VT>, grid_for(g.N, 256), 256, 0, st, g, d, z, omega);
}

// explicit instantiations
template void apply_operator<double, double>(const Geom&, const int*, const int*, const double*, const double*,
                                             const double*, const double*, const double*, double*, cudaStream_t);
template void apply_operator<float, float>(const Geom&, const int*, const int*, const float*, const float*,
                                           const float*, const float*, const float*, float*, cudaStream_t);
template void invert_patches<double>(const Geom&, const int*, const double*, const double*, const double*, const float*,
                                     const float*, const float*, double*, int, int*, void*, int*, cudaStream_t);
template void invert_patches<float>(const Geom&, const int*, const double*, const double*, const double*,
                                    const float*, const float*, const float*, float*, int, int*, void*, int*,
                                    cudaStream_t);
template void invert_patches<__nv_bfloat16>(const Geom&, const int*, const double*, const double*, const double*,
                                            const float*, const float*, const float*, __nv_bfloat16*, int, int*,
                                            void*, int*, cudaStream_t);
template void vanka_colour<double, double>(const Geom&, int, const double*, const double*, double*, double,
                                           cudaStream_t, int);
template void vanka_colour<float, float>(const Geom&, int, const float*, const float*, float*, float, cudaStream_t,
                                         int);
template void vanka_colour<float, __nv_bfloat16>(const Geom&, int, const __nv_bfloat16*, const float*, float*,
                                                 float, cudaStream_t, int);
template void vanka_update<double>(const Geom&, double*, double*, double, cudaStream_t);
template void vanka_update<float>(const Geom&, float*, float*, double, cudaStream_t);

}  // namespace stg
