// Internal definitions shared by the sm_103a kernels of the space-time Vanka
// multigrid solver (geometry of one structured level, data layout, helpers).
//
// Internal data layout of one level (differs from the C-ABI order of X_n,
// Eq. (3.2); the entry points permute at the boundary):
//   vector  = [velocity | pressure]
//   velocity: node-major, NV = (k+1)*dim values per Q2 node, index a*dim + c
//   pressure: cell-major, NP = (k+1)*npd values per cell, index a*npd + m (npd = dim P_{r-1}:
//             dim+1 for r = 2, 10 for r = 4 in 2D)
//   Jvv     : block-CSR over Q2 nodes, dense NV x NV blocks (row (a,c), col (b,e)),
//             the columns of a row ordered (z, y, x) lexicographically over the
//             tensor-product stencil of the node
//   Jvp     : per cell and local node: [cell][i][a][c][m]   (time-diagonal)
//   Jpv     : per cell: [cell][a][m][i][c]                  (time-diagonal)
//   patch   : local order [(r+1)^d nodes x NV | NP]; npatch = (k+1)((r+1)^d d + npd)
//   J_K^{-1}: one column-major npatch x npatch matrix per cell, cells ordered by
//             colour (colour = sum_e (c_e & 1) 2^e) and lexicographically inside
//             a colour
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>

#include "stg.h"

namespace stg {

struct Geom {
  int dim, k, nt;
  int r;                // velocity order of (Q_r)^d x P_{r-1}^disc: 2, or 4 (2D)
  int npd;              // pressure coefficients of a cell per time node: dim P_{r-1}
  int n[3];             // cells per direction (1 beyond dim)
  int nn[3];            // Q2 nodes per direction (1 beyond dim)
  double lo[3], h[3];
  unsigned dirichlet;   // bit 2*dir+side
  int NV, NP, nloc, npatch;
  long long n_nodes, n_cells, nvel, npres, N;
  // cells of each colour: count per direction and offset of the colour's first patch
  int ccount[8][3];
  long long coff[9];
  // removed cells (2D obstacle) in this level's cell indices: [ob[0], ob[1]) x [ob[2], ob[3]);
  // empty (ob[1] <= ob[0]) without an obstacle
  int ob[4];
};

Geom make_geom(const stg_mesh& m, int level, int k);

// ------------------------------------------------------------------ conversions
template <typename D, typename S>
__device__ __forceinline__ D cvt(S x) { return static_cast<D>(x); }
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, float>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, double>(double x) { return __double2bfloat16(x); }

// ------------------------------------------------------------------ index helpers
__host__ __device__ __forceinline__ long long node_id(const Geom& g, int ix, int iy, int iz) {
  return ix + (long long)g.nn[0] * (iy + (long long)g.nn[1] * iz);
}
__host__ __device__ __forceinline__ long long cell_id(const Geom& g, int cx, int cy, int cz) {
  return cx + (long long)g.n[0] * (cy + (long long)g.n[1] * cz);
}
// Range of Q_r node indices coupled to node index i along one direction: a vertex line
// (i % r == 0) touches two cells (r nodes either side), an interior line the nodes of its cell.
__host__ __device__ __forceinline__ void stencil_range(int i, int nn, int& lo, int& hi, int r = 2) {
  const int q = i % r;
  const int l = q == 0 ? i - r : i - q, h = q == 0 ? i + r : i - q + r;
  lo = l < 0 ? 0 : l;
  hi = h > nn - 1 ? nn - 1 : h;
}
// Position of column node (jx,jy,jz) in the BCSR row of node (ix,iy,iz).
__host__ __device__ __forceinline__ long long bcsr_slot(const Geom& g, const int* rowptr, int ix, int iy,
                                                        int iz, int jx, int jy, int jz) {
  int xl, xh, yl, yh, zl, zh;
  stencil_range(ix, g.nn[0], xl, xh, g.r);
  stencil_range(iy, g.nn[1], yl, yh, g.r);
  stencil_range(iz, g.nn[2], zl, zh, g.r);
  const int wx = xh - xl + 1, wy = yh - yl + 1;
  return (long long)rowptr[node_id(g, ix, iy, iz)] + ((long long)(jz - zl) * wy + (jy - yl)) * wx + (jx - xl);
}
// Cell of patch index p (patches ordered by colour, then lexicographically).
__host__ __device__ __forceinline__ void patch_cell(const Geom& g, long long p, int& cx, int& cy, int& cz) {
  int col = 0;
  while (col < (1 << g.dim) - 1 && p >= g.coff[col + 1]) ++col;
  long long li = p - g.coff[col];
  const int* c = g.ccount[col];
  const int jx = (int)(li % c[0]);
  li /= c[0];
  const int jy = (int)(li % c[1]);
  const int jz = (int)(li / c[1]);
  cx = 2 * jx + (col & 1);
  cy = g.dim > 1 ? 2 * jy + ((col >> 1) & 1) : 0;
  cz = g.dim > 2 ? 2 * jz + ((col >> 2) & 1) : 0;
}
__host__ __device__ __forceinline__ long long patch_of_cell(const Geom& g, int cx, int cy, int cz) {
  const int col = (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
  const int* c = g.ccount[col];
  return g.coff[col] + (cx >> 1) + (long long)c[0] * ((cy >> 1) + (long long)c[1] * (cz >> 1));
}
// Global internal index of local patch entry mu of cell (cx,cy,cz).
__host__ __device__ __forceinline__ long long patch_dof(const Geom& g, int cx, int cy, int cz, int mu) {
  const int vel = g.nloc * g.NV;
  if (mu < vel) {
    const int i = mu / g.NV, v = mu - i * g.NV;
    if (g.r == 2) {
      const int lx = i % 3, ly = (i / 3) % 3, lz = i / 9;
      return node_id(g, 2 * cx + lx, 2 * cy + ly, 2 * cz + lz) * g.NV + v;
    }
    const int r1 = g.r + 1;
    const int lx = i % r1, ly = (i / r1) % r1, lz = i / (r1 * r1);
    return node_id(g, g.r * cx + lx, g.r * cy + ly, g.r * cz + lz) * g.NV + v;
  }
  return g.nvel + cell_id(g, cx, cy, cz) * g.NP + (mu - vel);
}
// ------------------------------------------------------------------ obstacle (2D)
__host__ __device__ __forceinline__ bool has_obstacle(const Geom& g) { return g.ob[1] > g.ob[0]; }
__host__ __device__ __forceinline__ bool cell_masked(const Geom& g, int cx, int cy) {
  return cx >= g.ob[0] && cx < g.ob[1] && cy >= g.ob[2] && cy < g.ob[3];
}
// Range of cell indices that contain Q_r node index i along one direction.
__host__ __device__ __forceinline__ void node_cells(int i, int n, int& lo, int& hi, int r = 2) {
  if (i % r) {
    lo = hi = i / r;
  } else {
    lo = i / r - 1 < 0 ? 0 : i / r - 1;
    hi = i / r > n - 1 ? n - 1 : i / r;
  }
}
// Cells containing node (ix, iy): (fluid, removed) counts.
__host__ __device__ __forceinline__ void node_cell_counts(const Geom& g, int ix, int iy, int& fluid, int& removed) {
  int xl, xh, yl, yh;
  node_cells(ix, g.n[0], xl, xh, g.r);
  node_cells(iy, g.n[1], yl, yh, g.r);
  fluid = removed = 0;
  for (int cy = yl; cy <= yh; ++cy)
    for (int cx = xl; cx <= xh; ++cx) {
      if (cell_masked(g, cx, cy))
        ++removed;
      else
        ++fluid;
    }
}
// A Q2 node of removed cells only: its velocity has no equation (identity rows).
__host__ __device__ __forceinline__ bool node_dead(const Geom& g, int ix, int iy) {
  if (!has_obstacle(g)) return false;
  int f, r;
  node_cell_counts(g, ix, iy, f, r);
  return f == 0;
}
// Face (e, side) of a remaining cell borders the obstacle.
__host__ __device__ __forceinline__ bool face_on_obstacle(const Geom& g, int cx, int cy, int e, int side) {
  if (!has_obstacle(g)) return false;
  const int nx = cx + (e == 0 ? (side ? 1 : -1) : 0), ny = cy + (e == 1 ? (side ? 1 : -1) : 0);
  if (nx < 0 || nx >= g.n[0] || ny < 0 || ny >= g.n[1]) return false;
  return cell_masked(g, nx, ny);
}

// Number of cells sharing Q2 node (ix,iy,iz): the static multiplicity p of (S2).  With an
// obstacle, the patches of the remaining cells smooth the nodes of the fluid domain, and a
// node of removed cells only is smoothed by the patches of those cells.
__host__ __device__ __forceinline__ int node_multiplicity(const Geom& g, int ix, int iy, int iz) {
  if (has_obstacle(g)) {
    int f, r;
    node_cell_counts(g, ix, iy, f, r);
    return f > 0 ? f : r;
  }
  int m = 1;
  if (ix % g.r == 0 && ix > 0 && ix < g.nn[0] - 1) m *= 2;
  if (g.dim > 1 && iy % g.r == 0 && iy > 0 && iy < g.nn[1] - 1) m *= 2;
  if (g.dim > 2 && iz % g.r == 0 && iz > 0 && iz < g.nn[2] - 1) m *= 2;
  return m;
}

inline long long patch_stride(int npatch) { return ((long long)npatch * npatch + 31) / 32 * 32; }

// ------------------------------------------------------------------ errors
struct Error {
  stg_status st;
  std::string msg;
};

#define STG_CUDA_OK(call)                                                                      \
  do {                                                                                         \
    cudaError_t e__ = (call);                                                                  \
    if (e__ != cudaSuccess)                                                                    \
      throw ::stg::Error{STG_ECUDA, std::string(#call) + " at " + __FILE__ + ":" +               \
                                        std::to_string(__LINE__) + ": " + cudaGetErrorString(e__)}; \
  } while (0)

// Every kernel launch is followed by exactly one STG_LAUNCH_OK, which also
// counts it (graph replays are counted per kernel node by the V-cycle driver).
long long& launch_counter();
#define STG_LAUNCH_OK()                    \
  do {                                     \
    STG_CUDA_OK(cudaGetLastError());       \
    ++::stg::launch_counter();             \
  } while (0)

inline unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }

// ------------------------------------------------------------------ launch overlap
// Programmatic dependent launch (sm_90+).  A kernel launched by launch_k while launch_overlap()
// is set carries the programmatic-serialisation attribute: its launch may begin before the
// previous kernel on the stream has been retired.  Every kernel launched by launch_k begins with
// pdl_wait(): griddepcontrol.wait returns once the previous grid has completed and its memory
// writes are visible, so nothing is read or written before it.  No kernel signals its dependents
// early (griddepcontrol.launch_dependents): that lets the next grid's CTAs take SM slots while
// this grid still runs, which measured 20% slower per V-cycle; the implicit signal at grid exit
// keeps only the launch latency hidden.  Without the attribute pdl_wait() does nothing, and a
// preceding memset, copy or event keeps its ordinary full dependency.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Set (per host thread) while a context with overlap_launches records or runs its V-cycle.
bool& launch_overlap();

template <typename... P, typename... A>
void launch_k(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = launch_overlap() ? 1 : 0;
  STG_CUDA_OK(cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...));
  ++launch_counter();
}

// Sets launch_overlap() for the lifetime of the guard and restores it afterwards.
struct OverlapScope {
  bool old;
  explicit OverlapScope(bool on) : old(launch_overlap()) { launch_overlap() = on; }
  ~OverlapScope() { launch_overlap() = old; }
};

}  // namespace stg
