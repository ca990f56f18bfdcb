// Grid transfer between nested levels and layout permutations.
//
// The V-cycle of Sec. 3 works on nested meshes (Sec. 2, h_l = h_{l-1}/2); the
// transfers are those of the nested spaces: prolongation P maps a coarse
// (Q2)^d x P1disc function to its coefficients on the fine mesh, restriction
// is P^T.  Along one direction a fine Q2 node at coarse reference coordinate
// -1/2 (+1/2) takes the coarse cell's nodal values with weights (3/8, 3/4,
// -1/8) ((-1/8, 3/4, 3/8)); nodes on coarse nodes take weight 1.  A child
// cell with offset s in {-1/2, +1/2}^d gets c0 + sum_e s_e c_e and c_e / 2.
// Time nodes are not coarsened.  With an obstacle (2D) the spaces are those of the fluid
// domain: P is zero on the fine unknowns outside it (Q2 nodes of removed cells only, the
// pressure of removed cells), and P^T leaves their residual out of the coarse problem.
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace stg {
namespace {

// Coarse node indices and weights feeding fine node index f along one direction.
// The weights are exact in binary, so the transfers run in the vector precision.
template <typename W>
__device__ __forceinline__ int prolong_1d(int f, int* idx, W* w) {
  if (!(f & 1)) {
    idx[0] = f >> 1;
    w[0] = (W)1;
    return 1;
  }
  const int cc = f >> 2;
  idx[0] = 2 * cc;
  idx[1] = 2 * cc + 1;
  idx[2] = 2 * cc + 2;
  if ((f & 3) == 1) {
    w[0] = (W)0.375;
    w[1] = (W)0.75;
    w[2] = (W)-0.125;
  } else {
    w[0] = (W)-0.125;
    w[1] = (W)0.75;
    w[2] = (W)0.375;
  }
  return 3;
}

// Fine node indices and weights of row c of P^T along one direction (nnf fine nodes).
template <typename W>
__device__ __forceinline__ int restrict_1d(int c, int nnf, int* idx, W* w) {
  int n = 0;
  auto add = [&](int f, W wt) {
    if (f >= 0 && f < nnf) {
      idx[n] = f;
      w[n] = wt;
      ++n;
    }
  };
  add(2 * c, (W)1);
  if (c & 1) {
    add(2 * c - 1, (W)0.75);
    add(2 * c + 1, (W)0.75);
  } else {
    add(2 * c - 1, (W)0.375);
    add(2 * c + 1, (W)0.375);
    add(2 * c - 3, (W)-0.125);
    add(2 * c + 3, (W)-0.125);
  }
  return n;
}

template <typename VT>
__global__ void prolong_vel(Geom gc, Geom gf, const VT* __restrict__ xc, VT* __restrict__ xf) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gf.nvel) return;
  const int NV = gf.NV;
  const long long node = t / NV;
  const int v = (int)(t - node * NV);
  const int f[3] = {(int)(node % gf.nn[0]), (int)((node / gf.nn[0]) % gf.nn[1]),
                    (int)(node / ((long long)gf.nn[0] * gf.nn[1]))};
  if (gf.dim == 2 && node_dead(gf, f[0], f[1])) return;
  int ix[3][3], n[3];
  VT w[3][3];
  for (int e = 0; e < 3; ++e) n[e] = prolong_1d<VT>(f[e], ix[e], w[e]);
  VT acc = 0;
  for (int c = 0; c < n[2]; ++c)
    for (int b = 0; b < n[1]; ++b)
      for (int a = 0; a < n[0]; ++a)
        acc += w[0][a] * w[1][b] * w[2][c] * xc[node_id(gc, ix[0][a], ix[1][b], ix[2][c]) * NV + v];
  xf[t] += acc;
}

template <typename VT>
__global__ void prolong_pres(Geom gc, Geom gf, const VT* __restrict__ xc, VT* __restrict__ xf) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gf.npres) return;
  const int d = gf.dim;
  const long long K = t / gf.NP;
  const int q = (int)(t - K * gf.NP);
  const int a = q / (d + 1), m = q % (d + 1);
  const int f[3] = {(int)(K % gf.n[0]), (int)((K / gf.n[0]) % gf.n[1]), (int)(K / ((long long)gf.n[0] * gf.n[1]))};
  if (d == 2 && cell_masked(gf, f[0], f[1])) return;
  const long long Kc = cell_id(gc, f[0] >> 1, f[1] >> 1, f[2] >> 1);
  const VT* c = xc + gc.nvel + Kc * gc.NP + a * (d + 1);
  VT val;
  if (m == 0) {
    val = c[0];
    for (int e = 0; e < d; ++e) val += ((f[e] & 1) ? (VT)0.5 : (VT)-0.5) * c[e + 1];
  } else {
    val = (VT)0.5 * c[m];
  }
  xf[gf.nvel + t] += val;
}

template <typename VT>
__global__ void restrict_vel(Geom gc, Geom gf, const VT* __restrict__ rf, VT* __restrict__ bc) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gc.nvel) return;
  const int NV = gc.NV;
  const long long node = t / NV;
  const int v = (int)(t - node * NV);
  const int c[3] = {(int)(node % gc.nn[0]), (int)((node / gc.nn[0]) % gc.nn[1]),
                    (int)(node / ((long long)gc.nn[0] * gc.nn[1]))};
  int ix[3][5], n[3];
  VT w[3][5];
  for (int e = 0; e < 3; ++e) n[e] = restrict_1d<VT>(c[e], gf.nn[e], ix[e], w[e]);
  VT acc = 0;
  const bool obst = gf.dim == 2 && has_obstacle(gf);
  for (int z = 0; z < n[2]; ++z)
    for (int y = 0; y < n[1]; ++y)
      for (int x = 0; x < n[0]; ++x) {
        if (obst && node_dead(gf, ix[0][x], ix[1][y])) continue;
        acc += w[0][x] * w[1][y] * w[2][z] * rf[node_id(gf, ix[0][x], ix[1][y], ix[2][z]) * NV + v];
      }
  bc[t] = acc;
}

template <typename VT>
__global__ void restrict_pres(Geom gc, Geom gf, const VT* __restrict__ rf, VT* __restrict__ bc) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gc.npres) return;
  const int d = gc.dim;
  const long long K = t / gc.NP;
  const int q = (int)(t - K * gc.NP);
  const int a = q / (d + 1), m = q % (d + 1);
  const int c[3] = {(int)(K % gc.n[0]), (int)((K / gc.n[0]) % gc.n[1]), (int)(K / ((long long)gc.n[0] * gc.n[1]))};
  VT acc = 0;
  const int nch = 1 << d;
  for (int o = 0; o < nch; ++o) {
    const int fx = 2 * c[0] + (o & 1), fy = d > 1 ? 2 * c[1] + ((o >> 1) & 1) : 0;
    const int fz = d > 2 ? 2 * c[2] + ((o >> 2) & 1) : 0;
    if (d == 2 && cell_masked(gf, fx, fy)) continue;  // removed child: P is zero there
    const VT* f = rf + gf.nvel + cell_id(gf, fx, fy, fz) * gf.NP + a * (d + 1);
    if (m == 0) {
      acc += f[0];
    } else {
      const VT s = ((o >> (m - 1)) & 1) ? (VT)0.5 : (VT)-0.5;
      acc += s * f[0] + (VT)0.5 * f[m];
    }
  }
  bc[gc.nvel + t] = acc;
}

// ---------------------------------------------------------------- order 4 (2D)
// Q4: a fine node on a coarse node takes its value; a fine node at coarse reference coordinate
// -3/4, -1/4, 1/4, 3/4 of a coarse cell takes the cell's 5 nodal values with the Q4 Lagrange
// weights there (c_W4).  P3disc: the child with offset o in {0,1}^2 gets the coefficients of
// the coarse polynomial in its own reference coordinates, xi_c = xi_f / 2 + (o - 1/2):
// binomial expansion of each monomial (c_E4[o][fine][coarse]).
__constant__ double c_W4[4][5];
__constant__ double c_E4[4][10][10];

template <typename W>
__device__ __forceinline__ int prolong4_1d(int f, int* idx, W* w) {
  if (!(f & 1)) {
    idx[0] = f >> 1;
    w[0] = (W)1;
    return 1;
  }
  const int cc = f >> 3, k = ((f - 8 * cc) - 1) >> 1;
  for (int l = 0; l < 5; ++l) {
    idx[l] = 4 * cc + l;
    w[l] = (W)c_W4[k][l];
  }
  return 5;
}

// Fine node indices and weights of coarse node c along one direction (row c of P^T).
template <typename W>
__device__ __forceinline__ int restrict4_1d(int c, int nnf, int ncells, int* idx, W* w) {
  int n = 0;
  idx[n] = 2 * c;
  w[n] = (W)1;
  ++n;
  const int cl = (c % 4 == 0) ? c / 4 - 1 : c / 4, ch = c / 4;
  for (int cc = cl; cc <= ch; ++cc) {
    if (cc < 0 || cc >= ncells) continue;
    const int l = c - 4 * cc;
    if (l < 0 || l > 4) continue;
    for (int k = 0; k < 4; ++k) {
      const int f = 8 * cc + 2 * k + 1;
      if (f < nnf) {
        idx[n] = f;
        w[n] = (W)c_W4[k][l];
        ++n;
      }
    }
  }
  return n;
}

template <typename VT>
__global__ void prolong_vel4(Geom gc, Geom gf, const VT* __restrict__ xc, VT* __restrict__ xf) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gf.nvel) return;
  const int NV = gf.NV;
  const long long node = t / NV;
  const int v = (int)(t - node * NV);
  const int fx = (int)(node % gf.nn[0]), fy = (int)(node / gf.nn[0]);
  int ix[5], iy[5];
  VT wx[5], wy[5];
  const int nx = prolong4_1d<VT>(fx, ix, wx), ny = prolong4_1d<VT>(fy, iy, wy);
  VT acc = 0;
  for (int b = 0; b < ny; ++b)
    for (int a = 0; a < nx; ++a) acc += wx[a] * wy[b] * xc[node_id(gc, ix[a], iy[b], 0) * NV + v];
  xf[t] += acc;
}

template <typename VT>
__global__ void restrict_vel4(Geom gc, Geom gf, const VT* __restrict__ rf, VT* __restrict__ bc) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gc.nvel) return;
  const int NV = gc.NV;
  const long long node = t / NV;
  const int v = (int)(t - node * NV);
  const int cx = (int)(node % gc.nn[0]), cy = (int)(node / gc.nn[0]);
  int ix[9], iy[9];
  VT wx[9], wy[9];
  const int nx = restrict4_1d<VT>(cx, gf.nn[0], gc.n[0], ix, wx);
  const int ny = restrict4_1d<VT>(cy, gf.nn[1], gc.n[1], iy, wy);
  VT acc = 0;
  for (int b = 0; b < ny; ++b)
    for (int a = 0; a < nx; ++a) acc += wx[a] * wy[b] * rf[node_id(gf, ix[a], iy[b], 0) * NV + v];
  bc[t] = acc;
}

template <typename VT>
__global__ void prolong_pres4(Geom gc, Geom gf, const VT* __restrict__ xc, VT* __restrict__ xf) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gf.npres) return;
  const long long K = t / gf.NP;
  const int q = (int)(t - K * gf.NP);
  const int a = q / 10, m = q % 10;
  const int fx = (int)(K % gf.n[0]), fy = (int)(K / gf.n[0]);
  const int o = (fx & 1) + 2 * (fy & 1);
  const VT* c = xc + gc.nvel + cell_id(gc, fx >> 1, fy >> 1, 0) * gc.NP + a * 10;
  VT val = 0;
  for (int j = 0; j < 10; ++j) val += (VT)c_E4[o][m][j] * c[j];
  xf[gf.nvel + t] += val;
}

template <typename VT>
__global__ void restrict_pres4(Geom gc, Geom gf, const VT* __restrict__ rf, VT* __restrict__ bc) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gc.npres) return;
  const long long K = t / gc.NP;
  const int q = (int)(t - K * gc.NP);
  const int a = q / 10, j = q % 10;
  const int cx = (int)(K % gc.n[0]), cy = (int)(K / gc.n[0]);
  VT acc = 0;
  for (int o = 0; o < 4; ++o) {
    const VT* f = rf + gf.nvel + cell_id(gf, 2 * cx + (o & 1), 2 * cy + (o >> 1), 0) * gf.NP + a * 10;
    for (int m = 0; m < 10; ++m) acc += (VT)c_E4[o][m][j] * f[m];
  }
  bc[gc.nvel + t] = acc;
}

__device__ __forceinline__ long long cabi_index(const Geom& g, long long t) {
  const long long R = (long long)g.dim * g.n_nodes, S = (long long)g.npd * g.n_cells;
  if (t < g.nvel) {
    const long long node = t / g.NV;
    const int v = (int)(t - node * g.NV);
    const int a = v / g.dim, c = v % g.dim;
    return a * (R + S) + node * g.dim + c;
  }
  const long long u = t - g.nvel;
  const long long cell = u / g.NP;
  const int q = (int)(u - cell * g.NP);
  const int a = q / g.npd, m = q % g.npd;
  return a * (R + S) + R + cell * g.npd + m;
}

template <typename VT>
__global__ void to_internal_kernel(Geom g, const double* __restrict__ in, VT* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.N) return;
  out[t] = (VT)in[cabi_index(g, t)];
}

template <typename VT>
__global__ void to_cabi_kernel(Geom g, const VT* __restrict__ in, double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.N) return;
  out[cabi_index(g, t)] = (double)in[t];
}

__global__ void w_to_internal_kernel(Geom g, const double* __restrict__ in, double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nvel) return;
  const long long node = t / g.NV;
  const int v = (int)(t - node * g.NV);
  const int a = v / g.dim, c = v % g.dim;
  out[t] = in[a * (long long)g.dim * g.n_nodes + node * g.dim + c];
}

__global__ void inject_w_kernel(Geom gc, Geom gf, const double* __restrict__ wf, double* __restrict__ wc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gc.nvel) return;
  const long long node = t / gc.NV;
  const int v = (int)(t - node * gc.NV);
  const int c[3] = {(int)(node % gc.nn[0]), (int)((node / gc.nn[0]) % gc.nn[1]),
                    (int)(node / ((long long)gc.nn[0] * gc.nn[1]))};
  wc[t] = wf[node_id(gf, 2 * c[0], 2 * c[1], 2 * c[2]) * gf.NV + v];
}

// X0 (C-ABI order) = the last Radau-node block of X_prev, repeated for every node.
__global__ void replicate_kernel(Geom g, const double* __restrict__ xp, double* __restrict__ x0) {
  const long long blk = g.nvel / g.nt + g.npres / g.nt;  // R + S
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.N) return;
  x0[t] = xp[(long long)(g.nt - 1) * blk + t % blk];
}

template <typename VT>
__global__ void zero_kernel(long long n, VT* __restrict__ x) {
  pdl_wait();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = (VT)0;
}

template <typename D, typename S>
__global__ void convert_kernel(long long n, const S* __restrict__ in, D* __restrict__ out) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = cvt<D>(in[t]);
}

}  // namespace

void upload_transfer4_tables() {
  // Q4 Lagrange weights at coarse reference points -3/4, -1/4, 1/4, 3/4 (nodes -1, -1/2, 0, 1/2, 1)
  double W[4][5];
  const double nodes[5] = {-1.0, -0.5, 0.0, 0.5, 1.0};
  for (int k = 0; k < 4; ++k) {
    const double x = -0.75 + 0.5 * k;
    for (int l = 0; l < 5; ++l) {
      double v = 1.0;
      for (int m = 0; m < 5; ++m)
        if (m != l) v *= (x - nodes[m]) / (nodes[l] - nodes[m]);
      W[k][l] = v;
    }
  }
  // P3 monomials (a, b) of x and y exponents, by degree, x exponent falling
  const int ex[10][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}, {3, 0}, {2, 1}, {1, 2}, {0, 3}};
  auto binom = [](int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
  };
  double E[4][10][10] = {};
  for (int o = 0; o < 4; ++o) {
    const double sx = (o & 1) - 0.5, sy = (o >> 1) - 0.5;
    for (int j = 0; j < 10; ++j) {      // coarse monomial xi_c^a eta_c^b
      const int a = ex[j][0], b = ex[j][1];
      for (int m = 0; m < 10; ++m) {    // fine monomial xi_f^i eta_f^k
        const int i = ex[m][0], k = ex[m][1];
        if (i > a || k > b) continue;
        E[o][m][j] = binom(a, i) * std::pow(0.5, i) * std::pow(sx, a - i) * binom(b, k) * std::pow(0.5, k) *
                     std::pow(sy, b - k);
      }
    }
  }
  STG_CUDA_OK(cudaMemcpyToSymbol(c_W4, W, sizeof(W)));
  STG_CUDA_OK(cudaMemcpyToSymbol(c_E4, E, sizeof(E)));
}

template <typename VT>
void prolongate_add(const Geom& gc, const Geom& gf, const VT* xc, VT* xf, cudaStream_t st) {
  if (gf.r == 4) {
    launch_k(prolong_vel4<VT>, grid_for(gf.nvel, 256), 256, 0, st, gc, gf, xc, xf);
    launch_k(prolong_pres4<VT>, grid_for(gf.npres, 256), 256, 0, st, gc, gf, xc, xf);
    return;
  }
  launch_k(prolong_vel<VT>, grid_for(gf.nvel, 256), 256, 0, st, gc, gf, xc, xf);
  launch_k(prolong_pres<VT>, grid_for(gf.npres, 256), 256, 0, st, gc, gf, xc, xf);
}

template <typename VT>
void restrict_res(const Geom& gc, const Geom& gf, const VT* rf, VT* bc, cudaStream_t st) {
  if (gf.r == 4) {
    launch_k(restrict_vel4<VT>, grid_for(gc.nvel, 256), 256, 0, st, gc, gf, rf, bc);
    launch_k(restrict_pres4<VT>, grid_for(gc.npres, 256), 256, 0, st, gc, gf, rf, bc);
    return;
  }
  launch_k(restrict_vel<VT>, grid_for(gc.nvel, 256), 256, 0, st, gc, gf, rf, bc);
  launch_k(restrict_pres<VT>, grid_for(gc.npres, 256), 256, 0, st, gc, gf, rf, bc);
}

template <typename VT>
void cabi_to_internal(const Geom& g, const double* in, VT* out, cudaStream_t st) {
  to_internal_kernel<VT><<<grid_for(g.N, 256), 256, 0, st>>>(g, in, out);
  STG_LAUNCH_OK();
}

template <typename VT>
void internal_to_cabi(const Geom& g, const VT* in, double* out, cudaStream_t st) {
  to_cabi_kernel<VT><<<grid_for(g.N, 256), 256, 0, st>>>(g, in, out);
  STG_LAUNCH_OK();
}

void w_to_internal(const Geom& g, const double* in, double* out, cudaStream_t st) {
  w_to_internal_kernel<<<grid_for(g.nvel, 256), 256, 0, st>>>(g, in, out);
  STG_LAUNCH_OK();
}

void inject_w(const Geom& gc, const Geom& gf, const double* wf, double* wc, cudaStream_t st) {
  inject_w_kernel<<<grid_for(gc.nvel, 256), 256, 0, st>>>(gc, gf, wf, wc);
  STG_LAUNCH_OK();
}

void replicate_end_value(const Geom& g, const double* xp, double* x0, cudaStream_t st) {
  replicate_kernel<<<grid_for(g.N, 256), 256, 0, st>>>(g, xp, x0);
  STG_LAUNCH_OK();
}

template <typename VT>
void fill_zero(long long n, VT* x, cudaStream_t st) {
  if (n <= 0) return;
  launch_k(zero_kernel<VT>, grid_for(n, 256), 256, 0, st, n, x);
}

template <typename D, typename S>
void convert(long long n, const S* in, D* out, cudaStream_t st) {
  if (n <= 0) return;
  launch_k(convert_kernel<D, S>, grid_for(n, 256), 256, 0, st, n, in, out);
}

template void fill_zero<double>(long long, double*, cudaStream_t);
template void fill_zero<float>(long long, float*, cudaStream_t);
template void prolongate_add<double>(const Geom&, const Geom&, const double*, double*, cudaStream_t);
template void prolongate_add<float>(const Geom&, const Geom&, const float*, float*, cudaStream_t);
template void restrict_res<double>(const Geom&, const Geom&, const double*, double*, cudaStream_t);
template void restrict_res<float>(const Geom&, const Geom&, const float*, float*, cudaStream_t);
template void cabi_to_internal<double>(const Geom&, const double*, double*, cudaStream_t);
template void cabi_to_internal<float>(const Geom&, const double*, float*, cudaStream_t);
template void internal_to_cabi<double>(const Geom&, const double*, double*, cudaStream_t);
template void internal_to_cabi<float>(const Geom&, const float*, double*, cudaStream_t);
template void convert<float, double>(long long, const double*, float*, cudaStream_t);
template void convert<double, float>(long long, const float*, double*, cudaStream_t);
template void convert<__nv_bfloat16, double>(long long, const double*, __nv_bfloat16*, cudaStream_t);

}  // namespace stg
