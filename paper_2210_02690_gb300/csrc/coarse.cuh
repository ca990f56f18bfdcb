// Coarse-level direct solver: interior elimination per cell column plus block
// cyclic reduction over the vertex planes, in precision T.  See coarse.cu.
#pragma once

#include <vector>

#include "common.cuh"

namespace stg {

// In-place inverses of `batch` FP32 m x m row-major matrices (m <= 256) by the on-chip
// Gauss-Jordan kernel; status gets 1 + the first singular matrix.  Returns false (nothing
// launched) for larger m.
bool rgj_invert(int m, float* const* A, int batch, int* status, cudaStream_t st);


template <typename T>
struct CoarseView {
  Geom g;
  int pin, nsi, nsv, mV, mI;
  T *AII, *AIV, *AVI, *D, *L, *U;
  int* status;  // [0]: 1 + first singular block, [1]: unexpected coupling
};

template <typename T>
struct CrLevel {
  long long stride;
  int n_odd, n_left, n_right;
  T** oD;
  // solve lists.  Forward, even planes with a neighbour: b_j -= PL_j b_{j-st} + PR_j b_{j+st}
  // with PL_j = L_j D_{j-st}^{-1}, PR_j = U_j D_{j+st}^{-1} (so t = D^{-1} b of the odd planes is
  // never formed); backward, odd planes: x_i = D_i^{-1} b_i - GL_i x_{i-st} - GU_i x_{i+st}.
  // Absent terms are null pointers.
  int n_even;
  T **fA0, **fx0, **fA1, **fx1, **ey;
  T **bx, **bGL, **bxl, **qA1, **qx1, **bb;
  // factorisation lists: [GL_i | GU_i] = D_i^{-1} [L_i | U_i] (2 n_odd items); D_j -= L_j GU_{j-st}
  // + U_j GL_{j+st} (n_even items, A = eA0 / eA1, B = dB0 / dB1); new L_j = -L_j GL_{j-st}, new
  // U_j = -U_j GU_{j+st} (n_left + n_right items, written to this level's own blocks); PL_j, PR_j
  // (n_left + n_right items: A = uA, B = pB, C = pC)
  T **eA0, **eA1;
  T **gA, **gB, **gC, **dB0, **dB1, **dC, **uA, **uB, **uC, **pB, **pC;
};

// Scratch of the blocked Gauss-Jordan (blocks of 512+ rows): per matrix an m x w panel and a
// w x m copy of the pivot rows, addressed through device pointer arrays.
struct GjBlocked {
  void* panels = nullptr;  // T** [batch_max]
  void* olds = nullptr;    // T** [batch_max]
  int w = 32;
  long long m_max = 0;
  int batch_max = 0;
};

// One step of the coarse solve (its plan is built once, at init), one launch each:
//   kGather  b (FP64, level layout) -> vertex and interior right-hand sides bV, bI
//   kMV      y_i = alpha (A0_i x0_i + A1_i x1_i) + A2_i x2_i + c_i + beta y_i, i < batch, M rows
//            per item (Ak: M x Nk row-major); a null array, or a null entry of one, drops its
//            term
//   kScatter xV, xI -> x (FP64, level layout)
enum CoarseStepKind : int { kGather = 1, kMV = 2, kScatter = 4 };

template <typename T>
struct CStep {
  int kind, M, N0, N1, N2, batch;
  T alpha, beta;
  const T* const* A0;
  const T* const* x0;
  const T* const* A1;
  const T* const* x1;
  const T* const* A2;
  const T* const* x2;
  const T* const* c;
  T* const* y;
};

template <typename T>
struct CoarseSolver {
  CoarseView<T> v{};
  T *W = nullptr, *C = nullptr, *GL = nullptr, *GU = nullptr;
  T *bV = nullptr, *xV = nullptr, *bI = nullptr, *gI = nullptr, *xI = nullptr;
  T **d_AII = nullptr, **d_AIV = nullptr, **d_AVI = nullptr, **d_W = nullptr, **d_C = nullptr;
  T **d_bI = nullptr, **d_gI = nullptr, **d_xVs = nullptr, **d_xI = nullptr;
  T **d_cA0 = nullptr, **d_cx0 = nullptr, **d_cA1 = nullptr, **d_cx1 = nullptr, **d_cy = nullptr;
  T **d_top = nullptr, **d_topb = nullptr, **d_topx = nullptr;
  T* gj_scr = nullptr;  // Gauss-Jordan scratch for blocks too large for shared memory
  int *gj_perm = nullptr, *gj_fail = nullptr;
  GjBlocked gjb;
  std::vector<CrLevel<T>> levels;
  std::vector<void*> owned;
  // the solve as a list of steps, one launch each
  std::vector<CStep<T>> plan;

  void init(const Geom& g, bool pure_dirichlet);
  void release();
  // factor J_0 given in the internal level layout (FP64 operator), factors stored in T
  void factor(const int* rowptr, const int* colidx, const double* vv, const double* vp, const double* pv,
              cudaStream_t st);
  // x = J_0^{-1} b, both FP64 in the internal level layout, arithmetic in T
  void solve(const double* b, double* x, cudaStream_t st);
  // 0 = ok, > 0: 1 + singular block, -1: coupling outside the block structure (synchronises)
  int read_status(cudaStream_t st);

};

}  // namespace stg
