// On-chip Gauss-Jordan inverses of the coarse solver's FP32 slab blocks (up to 256 rows), in a
// translation unit of its own: its unrolled variants compile beside coarse.cu.
#include <algorithm>

#include "coarse.cuh"
#include "kernels.cuh"

namespace stg {

namespace {

// Gauss-Jordan inverse of an FP32 matrix held on chip, one CTA of NW warps per matrix: lane l
// of warp w holds rows l + 32 q (q < R) and columns w + NW k (k < CR + CS), column slots k < CR
// in registers and the others in a per-thread shared-memory slice (slot-major, thread-minor:
// conflict-free).  Partial pivoting without row interchanges: the pivot row p_j of column j is
// the unused row of largest |a_rj| (first such row on ties), it is scaled, and column j is
// eliminated from every other row.  After the last column, row p_j holds row j of the inverse
// of the row-permuted matrix, whose column c is column p_c of A^{-1}; the write-out puts a_{p_j c}
// at (j, p_c).  Rows are scaled lazily: row r is stored divided by sigma_r (1 until it becomes
// a pivot row, then 1 / a_pj), so the pivot row keeps its stored values (with 1 in column j)
// and every other entry takes the same fused multiply-add, a_rk -= a_rj (a_pk / a_pj), with the
// stored a_rj: no per-entry select.  One barrier a pivot step.  The warp that holds column j + 1 updates that column
// first, searches it and publishes it (with 1 / pivot) in the other half of a double buffer,
// then finishes its update: the search overlaps the rest of the CTA's update.  Each warp takes
// the pivot row's slice of its columns from its own lane p mod 32 through a per-warp buffer.
// Same pivots and operations as bgj_kernel, up to the order of equal-magnitude candidates.
template <int R, int CR, int CS, int NW>
__global__ void __launch_bounds__(32 * NW, 1) rgj_kernel(int m, float* const* As, int* status) {
  constexpr int C = CR + CS, NT = 32 * NW;
  float* G = As[blockIdx.x];
  extern __shared__ __align__(16) unsigned char sh_raw[];
  float* sp = reinterpret_cast<float*>(sh_raw) + threadIdx.x;  // slot (k, q) at ((k - CR) R + q) NT
  __shared__ float s_col[2][32 * R];
  __shared__ float s_prow[NW][C];
  __shared__ int s_piv[2];
  __shared__ float s_inv[2];
  __shared__ int s_pc[32 * R], s_pr[32 * R];  // pivot row of column c; column pivoted on row r
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  float a[R][CR > 0 ? CR : 1];
#define RGJ_GET(q, k) ((k) < CR ? a[q][(k) < CR ? (k) : 0] : sp[((k) - CR) * R * NT + (q) * NT])
#define RGJ_SET(q, k, v)                          \
  do {                                            \
    if ((k) < CR)                                 \
      a[q][(k) < CR ? (k) : 0] = (v);             \
    else                                          \
      sp[((k) - CR) * R * NT + (q) * NT] = (v);   \
  } while (0)
  unsigned used = 0;  // bit q: row lane + 32 q is a pivot row already (or padding)
  float sig[R];       // row scales (see above)
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = lane + 32 * q;
    sig[q] = 1.f;
    if (r >= m) used |= 1u << q;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const int c = w + NW * k;
      RGJ_SET(q, k, (r < m && c < m) ? G[(long long)r * m + c] : 0.f);
    }
  }
  // pivot search in column slot k of this warp; the result goes to buffer b
  auto search = [&](int k, int b) {
    float best = -1.f, val = 0.f;
    int bi = 0x7fffffff;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const float v = RGJ_GET(q, k);
      s_col[b][lane + 32 * q] = v;
      // rows of a lane ascend with q: '>' keeps the first maximum
      if (!((used >> q) & 1u) && fabsf(v) > best) {
        best = fabsf(v);
        bi = lane + 32 * q;
        val = v;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      const float ov = __shfl_xor_sync(0xffffffffu, val, off);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
        val = ov;
      }
    }
    if (lane == 0) {
      const bool ok = best > 0.f && !isinf(val);
      s_piv[b] = ok ? bi : -1;
      s_inv[b] = ok ? 1.f / val : 0.f;
    }
  };
  if (w == 0) search(0, 0);
  int buf = 0;
  bool fail = false;
#pragma unroll
  for (int kj = 0; kj < C; ++kj) {
    for (int jw = 0; jw < NW; ++jw) {
      const int j = kj * NW + jw;
      if (j >= m) break;
      __syncthreads();
      const int p = s_piv[buf];
      if (p < 0) {
        fail = true;
        break;
      }
      const float inv = s_inv[buf];
      const int pq = p >> 5, pl = p & 31;
      const bool piv_lane = lane == pl;
#pragma unroll
      for (int q = 0; q < R; ++q)
        if (q == pq && piv_lane) {
#pragma unroll
          for (int k = 0; k < C; ++k) s_prow[w][k] = (w == jw && k == kj) ? inv : RGJ_GET(q, k) * inv;
        }
      if (piv_lane) used |= 1u << pq;
      __syncwarp();
      float f[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const bool pr_here = q == pq && piv_lane;
        f[q] = pr_here ? 0.f : s_col[buf][lane + 32 * q];  // the pivot row is not updated
        if (pr_here) sig[q] = inv;
      }
      if (w == jw) {
        // column j becomes -a_rj / a_pj; the pivot row stores 1 (times sigma_p = 1 / a_pj)
#pragma unroll
        for (int q = 0; q < R; ++q) RGJ_SET(q, kj, (q == pq && piv_lane) ? 1.f : 0.f);
      }
      // the row update of column slot k: a_rk -= f_r pr_k
      auto update = [&](int k) {
        const float pk = s_prow[w][k];
#pragma unroll
        for (int q = 0; q < R; ++q) RGJ_SET(q, k, fmaf(-f[q], pk, RGJ_GET(q, k)));
      };
      // look-ahead: column j + 1 is slot kj of warp jw + 1, or slot kj + 1 of warp 0
      const bool next_here = jw + 1 < NW;
      const int la_w = next_here ? jw + 1 : 0;
      const bool la = w == la_w && j + 1 < m && (next_here || kj + 1 < C);
      if (la) {
        if (next_here) {
          update(kj);
          search(kj, buf ^ 1);
        } else if (kj + 1 < C) {
          update(kj + 1);
          search(kj + 1, buf ^ 1);
        }
      }
      const int la_k = next_here ? kj : kj + 1;
#pragma unroll
      for (int k = 0; k < CR; ++k)
        if (!(la && k == la_k)) update(k);
      if (CS > 0) {
        // shared-memory slots: all R loads of a slot are issued together, and those of the
        // next slot before the stores of this one (the stores could alias the loads otherwise)
        float cur[R], nxt[R];
#pragma unroll
        for (int q = 0; q < R; ++q) cur[q] = RGJ_GET(q, CR);
#pragma unroll
        for (int k = CR; k < C; ++k) {
          if (k + 1 < C) {
#pragma unroll
            for (int q = 0; q < R; ++q) nxt[q] = RGJ_GET(q, k + 1 < C ? k + 1 : k);
          }
          if (!(la && k == la_k)) {
            const float pk = s_prow[w][k];
#pragma unroll
            for (int q = 0; q < R; ++q) RGJ_SET(q, k, fmaf(-f[q], pk, cur[q]));
          }
#pragma unroll
          for (int q = 0; q < R; ++q) cur[q] = nxt[q];
        }
      }
      if (tid == 0) {
        s_pc[j] = p;
        s_pr[p] = j;
      }
      buf ^= 1;
    }
    if (fail) break;
  }
  if (fail) {
    if (tid == 0) atomicCAS(status, 0, 1 + (int)blockIdx.x);
    return;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = lane + 32 * q;
    if (r < m) {
      const long long row = (long long)s_pr[r] * m;
#pragma unroll
      for (int k = 0; k < C; ++k) {
        const int c = w + NW * k;
        if (c < m) G[row + s_pc[c]] = RGJ_GET(q, k) * sig[q];
      }
    }
  }
#undef RGJ_GET
#undef RGJ_SET
}

}  // namespace

// FP32 matrices of up to 256 rows: on-chip Gauss-Jordan, 16 warps a matrix (column slots of
// a thread beyond its register budget in shared memory)
template <int R, int CR, int CS, int NW>
static void launch_rgj(int m, float* const* A, int batch, int* status, cudaStream_t st) {
  const size_t smem = sizeof(float) * (size_t)CS * R * 32 * NW;
  if (smem > 48 * 1024)
    STG_CUDA_OK(cudaFuncSetAttribute(rgj_kernel<R, CR, CS, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  rgj_kernel<R, CR, CS, NW><<<batch, 32 * NW, smem, st>>>(m, A, status);
  STG_LAUNCH_OK();
}

bool rgj_invert(int m, float* const* A, int batch, int* status, cudaStream_t st) {
  switch ((m + 15) / 16) {
    case 1: launch_rgj<1, 1, 0, 16>(m, A, batch, status, st); return true;
    case 2: launch_rgj<1, 2, 0, 16>(m, A, batch, status, st); return true;
    case 3: launch_rgj<2, 3, 0, 16>(m, A, batch, status, st); return true;
    case 4: launch_rgj<2, 4, 0, 16>(m, A, batch, status, st); return true;
    case 5: launch_rgj<3, 5, 0, 16>(m, A, batch, status, st); return true;
    case 6: launch_rgj<3, 6, 0, 16>(m, A, batch, status, st); return true;
    case 7: launch_rgj<4, 7, 0, 16>(m, A, batch, status, st); return true;
    case 8: launch_rgj<4, 8, 0, 16>(m, A, batch, status, st); return true;
    case 9: launch_rgj<5, 9, 0, 16>(m, A, batch, status, st); return true;
    case 10: launch_rgj<5, 10, 0, 16>(m, A, batch, status, st); return true;
    case 11: launch_rgj<6, 11, 0, 16>(m, A, batch, status, st); return true;
    case 12: launch_rgj<6, 11, 1, 16>(m, A, batch, status, st); return true;
    case 13: launch_rgj<7, 8, 5, 16>(m, A, batch, status, st); return true;
    case 14: launch_rgj<7, 8, 6, 16>(m, A, batch, status, st); return true;
    case 15: launch_rgj<8, 7, 8, 16>(m, A, batch, status, st); return true;
    case 16: launch_rgj<8, 7, 9, 16>(m, A, batch, status, st); return true;
    default: return false;
  }
}

}  // namespace stg
