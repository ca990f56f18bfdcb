// Host-side launchers of the solver kernels (one declaration per kernel family).
#pragma once

#include "common.cuh"

namespace stg {

// Radau-Lagrange time basis on [0,1] (Sec. 3): nodes c_a, weights w_a,
// T_ab = int chi_b' chi_a + chi_a(0) chi_b(0), jump vector chi_a(0).
struct TimeData {
  double T[5][5];
  double w[5];
  double c[5];
  double jump[5];
};
TimeData time_basis(int k);

struct AsmCoef {
  double nu, tau, gamma1, gamma2;
  int newton;
};

// ---- assembly (assemble.cu)
void upload_fe_tables();
// doubles of the per-level table of w-independent element matrices (mass + one set per face class)
long long assemble_table_doubles(int dim, int k);
// vv, vp, pv = the part of the operator that does not depend on w (time coupling, viscous and
// Nitsche terms, velocity-pressure blocks), and the level's element tables; w is not read
void assemble_level(const Geom& g, const TimeData& td, const AsmCoef& cf, const double* w_int, const int* rowptr,
                    double* tab, double* vv, long long nnzb, double* vp, double* pv, cudaStream_t st);
// vv = vconst (the w = 0 assembly: time coupling, viscous, Nitsche terms) plus the terms that
// depend on w (convection, Newton when cf.newton) on the time-diagonal blocks; needs the tables
// of a previous assemble_level; leaves vp, pv as they are (they do not depend on w).
void assemble_level_w(const Geom& g, const TimeData& td, const AsmCoef& cf, const double* w_int, const int* rowptr,
                      const double* tab, const double* vconst, double* vv, long long nnzb, cudaStream_t st);

// right-hand side of Eq. (2.2) from nodal f, g (internal velocity layout) and v_prev ([node][c]);
// the mass matrix comes from the assembly table of the level (assemble_level first)
long long rhs_table_doubles(int dim);
// Q4 transfer weights and P3disc child embeddings into constant memory (order 4).
void upload_transfer4_tables();
// Force of the fluid on the obstacle at every Radau node: out[2a + c] (device), x internal.
void obstacle_forces(const Geom& g, double nu, const double* x_int, double* out, cudaStream_t st);
void assemble_rhs_level(const Geom& g, const TimeData& td, const AsmCoef& cf, const double* tab, double* rt,
                        const double* f, const double* gd, const double* vprev, double* b, cudaStream_t st);

// ---- operators, smoother and transfers (vanka.cu, transfer.cu)
// out = b - J x (has_b) or out = J x; MT = operator precision, VT = vector precision
template <typename MT, typename VT>
void apply_operator(const Geom& g, const int* rowptr, const int* colidx, const MT* vv, const MT* vp, const MT* pv,
                    const VT* x, const VT* b, VT* out, cudaStream_t st);

// Local inverses J_K^{-1} of every cell (gather from the assembled J, Gauss-Jordan
// with partial pivoting in CT precision, stored as FT). status[0] receives the
// first singular cell + 1 (0 = none).
size_t invert_scratch_bytes(const Geom& g, int compute_f32);
template <typename FT>
void invert_patches(const Geom& g, const int* rowptr, const double* vv, const double* vp, const double* pv,
                    const float* vv32, const float* vp32, const float* pv32, FT* jinv, int compute_f32, int* status,
                    void* scratch, int* flags, cudaStream_t st);

// One colour phase of the smoother: y_K = J_K^{-1} R_K r for all cells of colour
// `colour`; accumulate (averaged mode: z += y) or apply (coloured mode: z += omega y).
// variant = 3 * column-batch index (4, 8, 16 columns in flight) + CTA-size index (128, 256, 512)
// Variants 0..8: one warp per patch, loads straight from global memory (3 column-batch depths x
// 3 CTA sizes); 9..12: factors staged in shared memory by bulk copies (4 pipeline shapes), one
// row per thread; 13..16: the same shapes with two adjacent rows per thread (one vector load per
// column and row pair; even patch sizes, else they run as 9..12).
constexpr int kColourWarpVariants = 9;
constexpr int kColourVariants = 17;
constexpr int kColourWarpDefault = 4;  // 8 columns, 256 threads
constexpr int kColourDefault = 9;      // 4 stages, 8 CTAs per SM (falls back to the warp form)
template <typename VT, typename FT>
void vanka_colour(const Geom& g, int colour, const FT* jinv, const VT* r, VT* z, VT scale, cudaStream_t st,
                  int variant = kColourDefault);

// Kronecker-split FP32 velocity rows (2D, 2..5 Radau nodes): per BCSR slot M_ij and the d x d
// spatial blocks of every Radau node, split from the FP64 dense blocks.
bool kron_supported(const Geom& g);
void kron_split(const Geom& g, long long nnzb, const double* vv, const TimeData& td, float* Mk, float* Ak,
                cudaStream_t st);
void apply_operator_kron(const Geom& g, const TimeData& td, const float* Mk, const float* Ak,
                         const float* vp, const float* pv, const float* x, const float* b, float* out,
                         cudaStream_t st);

// True (and the flag cleared) when a staged colour kernel gave up waiting for a copy.
bool colour_kernel_timed_out(cudaStream_t st);
// Iteration limit of the staged colour kernel's waits for a factor copy.
void set_colour_wait_limit(long long spins);

// d += omega z / p (p = static multiplicity of (S2)); z = 0.
template <typename VT>
void vanka_update(const Geom& g, VT* d, VT* z, double omega, cudaStream_t st);

template <typename VT>
void prolongate_add(const Geom& gc, const Geom& gf, const VT* xc, VT* xf, cudaStream_t st);
template <typename VT>
void restrict_res(const Geom& gc, const Geom& gf, const VT* rf, VT* bc, cudaStream_t st);

// C-ABI order <-> internal layout
template <typename VT>
void cabi_to_internal(const Geom& g, const double* in, VT* out, cudaStream_t st);
template <typename VT>
void internal_to_cabi(const Geom& g, const VT* in, double* out, cudaStream_t st);
// velocity-only (k+1) x R C-ABI block -> internal node-major velocity
void w_to_internal(const Geom& g, const double* in, double* out, cudaStream_t st);
// X0 = last Radau-node block of X_prev repeated (C-ABI order), the slab's initial guess
void replicate_end_value(const Geom& g, const double* xp, double* x0, cudaStream_t st);
// coarse velocity at node 2g of the fine level (injection)
void inject_w(const Geom& gc, const Geom& gf, const double* wf, double* wc, cudaStream_t st);

template <typename D, typename S>
void convert(long long n, const S* in, D* out, cudaStream_t st);
// x[0 .. n) = 0 by a kernel (not a memset), so that it takes part in launch overlap.
template <typename VT>
void fill_zero(long long n, VT* x, cudaStream_t st);

// ---- BLAS-1 in FP64 (krylov.cu)
// h[i] = <V_i, w>, i < m, V row-major (m x n, leading dim ldv); partial sums per block -> h.
void multi_dot(long long n, int m, const double* V, long long ldv, const double* w, double* partial, double* h,
               cudaStream_t st);
// w -= sum_i h[i] V_i (h on the device)
void multi_axpy_sub(long long n, int m, const double* V, long long ldv, const double* h, double* w,
                    cudaStream_t st);
// x += sum_i y[i] Z_i
void multi_axpy_add(long long n, int m, const double* Z, long long ldz, const double* y, double* x,
                    cudaStream_t st);
// y = a x + b y
void axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t st);

size_t dot_partial_doubles();

}  // namespace stg
