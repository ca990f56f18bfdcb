// Jacobian assembly on one structured level (Sec. 3, Eq. (3.3) with D_ab and B_ab).
//
// For the linearisation velocity w_a at Radau node a, the space-time block of
// test (a, i, c) and trial (b, j, e) is
//   T_ab M_ij delta_ce + delta_ab tau w_a [ (w_a . grad phi_j, phi_i) delta_ce
//       + (Newton) phi_i phi_j d_e w_a,c + nu (grad phi_j, grad phi_i) delta_ce
//       + Nitsche terms of A_h and B_GammaD (Eq. (2.1)) on Dirichlet faces ],
// the velocity-pressure blocks delta_ab tau w_a [ -(xi_m, d_c phi_i) + <xi_m, phi_i n_c> ],
// the pressure-velocity blocks delta_ab tau w_a [ (xi_m, d_e phi_j) - <phi_j n_e, xi_m> ].
// T_ab is the time-derivative plus jump matrix of the Radau-Lagrange basis.
// One CTA per cell; cells of one colour share no Q2 node, so a colour's cells
// add into disjoint BCSR blocks and the launches need no atomics.
#include "common.cuh"
#include "kernels.cuh"

namespace stg {

// 1D Q2 Lagrange values / derivatives at five points: the three Gauss points and xi = -1, +1.
__constant__ double c_L1[5][3];
__constant__ double c_D1[5][3];
__constant__ double c_X[5];
__constant__ double c_GW[3];
// order 4 (2D): the same at the 5 Gauss points and xi = -1, +1
__constant__ double c_L4[7][5];
__constant__ double c_D4[7][5];
__constant__ double c_X4[7];
__constant__ double c_GW4[5];

void upload_fe_tables() {
  const double g = std::sqrt(0.6);
  const double X[5] = {-g, 0.0, g, -1.0, 1.0};
  double L1[5][3], D1[5][3];
  for (int p = 0; p < 5; ++p) {
    const double x = X[p];
    L1[p][0] = x * (x - 1.0) / 2.0;
    L1[p][1] = 1.0 - x * x;
    L1[p][2] = x * (x + 1.0) / 2.0;
    D1[p][0] = x - 0.5;
    D1[p][1] = -2.0 * x;
    D1[p][2] = x + 0.5;
  }
  const double GW[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  STG_CUDA_OK(cudaMemcpyToSymbol(c_L1, L1, sizeof(L1)));
  STG_CUDA_OK(cudaMemcpyToSymbol(c_D1, D1, sizeof(D1)));
  STG_CUDA_OK(cudaMemcpyToSymbol(c_X, X, sizeof(X)));
  STG_CUDA_OK(cudaMemcpyToSymbol(c_GW, GW, sizeof(GW)));
  // order 4: 1D Q4 Lagrange values / derivatives (nodes -1, -1/2, 0, 1/2, 1) at the 5 Gauss points
  // and xi = -1, +1; the 5-point Gauss rule
  const double a5 = std::sqrt(5.0 - 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
  const double b5 = std::sqrt(5.0 + 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
  const double X4[7] = {-b5, -a5, 0.0, a5, b5, -1.0, 1.0};
  const double wa = (322.0 + 13.0 * std::sqrt(70.0)) / 900.0, wb = (322.0 - 13.0 * std::sqrt(70.0)) / 900.0;
  const double GW4[5] = {wb, wa, 128.0 / 225.0, wa, wb};
  const double nd[5] = {-1.0, -0.5, 0.0, 0.5, 1.0};
  double L4[7][5], D4[7][5];
  for (int p = 0; p < 7; ++p)
    for (int l = 0; l < 5; ++l) {
      double v = 1.0, dsum = 0.0;
      for (int m = 0; m < 5; ++m)
        if (m != l) v *= (X4[p] - nd[m]) / (nd[l] - nd[m]);
      for (int q = 0; q < 5; ++q) {
        if (q == l) continue;
        double t = 1.0 / (nd[l] - nd[q]);
        for (int m = 0; m < 5; ++m)
          if (m != l && m != q) t *= (X4[p] - nd[m]) / (nd[l] - nd[m]);
        dsum += t;
      }
      L4[p][l] = v;
      D4[p][l] = dsum;
    }
  STG_CUDA_OK(cudaMemcpyToSymbol(c_L4, L4, sizeof(L4)));
  STG_CUDA_OK(cudaMemcpyToSymbol(c_D4, D4, sizeof(D4)));
  STG_CUDA_OK(cudaMemcpyToSymbol(c_X4, X4, sizeof(X4)));
  STG_CUDA_OK(cudaMemcpyToSymbol(c_GW4, GW4, sizeof(GW4)));
}

namespace {

template <int DIM>
struct Pow3 { static constexpr int v = DIM == 2 ? 9 : 27; };

// Value and physical gradient of local Q2 function i at point multi-index p.
template <int DIM>
__device__ __forceinline__ void basis_at(const Geom& g, const int* p, int i, double& v, double* grad) {
  int l[3] = {i % 3, (i / 3) % 3, i / 9};
  v = 1.0;
  for (int e = 0; e < DIM; ++e) v *= c_L1[p[e]][l[e]];
  for (int e = 0; e < DIM; ++e) {
    double d = 2.0 / g.h[e] * c_D1[p[e]][l[e]];
    for (int f = 0; f < DIM; ++f)
      if (f != e) d *= c_L1[p[f]][l[f]];
    grad[e] = d;
  }
}

// Face class of a cell: bit 2e set when the cell lies on a Dirichlet face
// x_e = low, bit 2e+1 for x_e = high.  On a uniform box every w-independent
// element matrix depends only on this class.
// With an obstacle (2D) the faces of a remaining cell that border a removed cell are Dirichlet
// faces as well.
template <int DIM>
__device__ __forceinline__ unsigned face_class(const Geom& g, const int* cc) {
  unsigned faces = 0;
  for (int e = 0; e < DIM; ++e) {
    if (cc[e] == 0 && (g.dirichlet >> (2 * e) & 1u)) faces |= 1u << (2 * e);
    if (cc[e] == g.n[e] - 1 && (g.dirichlet >> (2 * e + 1) & 1u)) faces |= 1u << (2 * e + 1);
    if (DIM == 2) {
      if (face_on_obstacle(g, cc[0], cc[1], e, 0)) faces |= 1u << (2 * e);
      if (face_on_obstacle(g, cc[0], cc[1], e, 1)) faces |= 1u << (2 * e + 1);
    }
  }
  return faces;
}

// Reference values phi, physical gradients dphi and weights W|det| of the cell rule.
template <int DIM, int NQ, int NL>
__device__ void cell_tables(const Geom& g, double (*phi)[NL], double (*dphi)[NL][DIM], double* qwd) {
  for (int t = threadIdx.x; t < NQ * NL; t += blockDim.x) {
    const int q = t / NL, i = t % NL;
    int p[3] = {q % 3, (q / 3) % 3, q / 9};
    double v, gr[3];
    basis_at<DIM>(g, p, i, v, gr);
    phi[q][i] = v;
    for (int e = 0; e < DIM; ++e) dphi[q][i][e] = gr[e];
    if (i == 0) {
      double wt = 1.0;
      for (int e = 0; e < DIM; ++e) wt *= c_GW[p[e]] * g.h[e] / 2.0;
      qwd[q] = wt;
    }
  }
}

// Face rule point fq of face (e0, s0): multi-index p and weight (reference weights times face Jacobian).
template <int DIM>
__device__ __forceinline__ double face_point(const Geom& g, int e0, int s0, int fq, int* p) {
  double wt = 1.0;
  int o = 0;
  for (int d = 0; d < DIM; ++d) {
    if (d == e0) {
      p[d] = 3 + s0;
    } else {
      p[d] = (o == 0) ? fq % 3 : fq / 3;
      wt *= c_GW[p[d]] * g.h[d] / 2.0;
      ++o;
    }
  }
  return wt;
}

// Layout of the per-level table written by element_constants:
//   [mass NL^2 | 4^d face classes x (vv ND^2, vp ND(d+1), pv (d+1)ND) | phi NQ NL | dphi NQ NL d |
//    qwd NQ | pp NQ NL NL], pp[q][i][j] = W_q |det| phi_i(q) phi_j(q).
__host__ __device__ __forceinline__ long long tab_class_size(int dim, int nloc) {
  const long long nd = (long long)nloc * dim;
  return nd * nd + 2 * nd * (dim + 1);
}
__host__ __device__ __forceinline__ long long tab_extra_offset(int dim, int nloc) {
  return (long long)nloc * nloc + (1LL << (2 * dim)) * tab_class_size(dim, nloc);
}

// w-independent element matrices, one CTA per face class:
//   mass M_ij (class 0 only), viscosity nu (grad phi_j, grad phi_i) delta_ce plus the Nitsche
//   terms of A_h and B_GammaD (Eq. (2.1)), and the velocity-pressure / pressure-velocity blocks.
template <int DIM>
__global__ void __launch_bounds__(256) element_constants(Geom g, AsmCoef cf, double* __restrict__ tab) {
  constexpr int NQ = Pow3<DIM>::v;
  constexpr int NL = NQ;
  constexpr int ND = NL * DIM;
  __shared__ double phi[NQ][NL];
  __shared__ double dphi[NQ][NL][DIM];
  __shared__ double qwd[NQ];
  const unsigned faces = blockIdx.x;
  cell_tables<DIM, NQ, NL>(g, phi, dphi, qwd);
  __syncthreads();
  if (faces == 0) {
    for (int t = threadIdx.x; t < NL * NL; t += blockDim.x) {
      const int i = t / NL, j = t % NL;
      double m = 0.0;
      for (int q = 0; q < NQ; ++q) m += qwd[q] * phi[q][i] * phi[q][j];
      tab[t] = m;
    }
    double* x = tab + tab_extra_offset(DIM, NL);
    double* xphi = x;
    double* xdphi = xphi + NQ * NL;
    double* xqwd = xdphi + NQ * NL * DIM;
    double* xpp = xqwd + NQ;
    for (int t = threadIdx.x; t < NQ * NL; t += blockDim.x) {
      const int q = t / NL, i = t % NL;
      xphi[t] = phi[q][i];
      for (int e = 0; e < DIM; ++e) xdphi[t * DIM + e] = dphi[q][i][e];
    }
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) xqwd[q] = qwd[q];
    for (int t = threadIdx.x; t < NQ * NL * NL; t += blockDim.x) {
      const int q = t / (NL * NL), i = (t / NL) % NL, j = t % NL;
      xpp[t] = qwd[q] * phi[q][i] * phi[q][j];
    }
  }
  double* base = tab + NL * NL + (long long)faces * tab_class_size(DIM, NL);
  for (int t = threadIdx.x; t < ND * ND; t += blockDim.x) {
    const int I = t / ND, J = t % ND;
    const int i = I / DIM, c = I % DIM, j = J / DIM, e = J % DIM;
    double val = 0.0;
    if (c == e) {
      double visc = 0.0;
      for (int q = 0; q < NQ; ++q) {
        double d = 0.0;
        for (int f = 0; f < DIM; ++f) d += dphi[q][j][f] * dphi[q][i][f];
        visc += qwd[q] * d;
      }
      val += cf.nu * visc;
    }
    for (int f = 0; f < 2 * DIM; ++f) {
      if (!(faces >> f & 1u)) continue;
      const int e0 = f >> 1, s0 = f & 1;
      const double ns = s0 ? 1.0 : -1.0, hf = g.h[e0];
      for (int fq = 0; fq < NQ / 3; ++fq) {
        int p[3];
        const double wt = face_point<DIM>(g, e0, s0, fq, p);
        double vi, vj, gi[3], gj[3];
        basis_at<DIM>(g, p, i, vi, gi);
        basis_at<DIM>(g, p, j, vj, gj);
        const double dni = ns * gi[e0], dnj = ns * gj[e0];
        double term = 0.0;
        if (c == e) term += -cf.nu * dnj * vi - cf.nu * vj * dni + cf.gamma1 * cf.nu / hf * vj * vi;
        if (c == e0 && e == e0) term += cf.gamma2 / hf * vj * vi;
        val += wt * term;
      }
    }
    base[t] = val;
  }
  double* vpt = base + (long long)ND * ND;
  double* pvt = vpt + (long long)ND * (DIM + 1);
  for (int t = threadIdx.x; t < ND * (DIM + 1); t += blockDim.x) {
    const int I = t / (DIM + 1), m = t % (DIM + 1);
    const int i = I / DIM, c = I % DIM;
    double vol = 0.0;
    for (int q = 0; q < NQ; ++q) {
      const double xi = m == 0 ? 1.0 : c_X[(m == 1) ? q % 3 : (m == 2 ? (q / 3) % 3 : q / 9)];
      vol += qwd[q] * xi * dphi[q][i][c];
    }
    double bnd = 0.0;
    for (int f = 0; f < 2 * DIM; ++f) {
      if (!(faces >> f & 1u)) continue;
      const int e0 = f >> 1, s0 = f & 1;
      if (c != e0) continue;
      const double ns = s0 ? 1.0 : -1.0;
      for (int fq = 0; fq < NQ / 3; ++fq) {
        int p[3];
        const double wt = face_point<DIM>(g, e0, s0, fq, p);
        double vi, gi[3];
        basis_at<DIM>(g, p, i, vi, gi);
        const double xi = m == 0 ? 1.0 : c_X[p[m - 1]];
        bnd += wt * xi * vi * ns;
      }
    }
    vpt[t] = -vol + bnd;                    // -(xi_m, d_c phi_i) + <xi_m, phi_i n_c>
    pvt[m * ND + I] = vol - bnd;            // (d_c phi_i, xi_m) - <phi_i n_c, xi_m>
  }
}

// K[a][cls][(i,c),(j,e)] = T_aa M_ij delta_ce + tau w_a C[cls][(i,c),(j,e)]: the w-independent
// part of the diagonal time block a for face class cls.
template <int DIM>
__global__ void diag_blocks(Geom g, TimeData td, AsmCoef cf, const double* __restrict__ tab, double* __restrict__ K) {
  constexpr int NL = Pow3<DIM>::v;
  constexpr int ND = NL * DIM;
  const int ncls = 1 << (2 * DIM);
  const long long per = (long long)ND * ND;
  const long long total = (long long)g.nt * ncls * per;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t / (ncls * per));
    const int cls = (int)((t / per) % ncls);
    const int I = (int)((t % per) / ND), J = (int)(t % ND);
    const int i = I / DIM, c = I % DIM, j = J / DIM, e = J % DIM;
    const double* cvv = tab + NL * NL + (long long)cls * tab_class_size(DIM, NL);
    K[t] = (c == e ? td.T[a][a] * tab[i * NL + j] : 0.0) + cf.tau * td.w[a] * cvv[t % per];
  }
}

// Per-cell assembly: the convection (and Newton) matrices from w_a at the cell's
// nodes, combined with the class constants, the time matrix T_ab and the factor
// tau w_a, added into the BCSR blocks of the cell's node pairs.
// WONLY = false: the part of the operator that does not depend on w (time coupling, viscous,
// Nitsche terms, velocity-pressure blocks); w is not read.  WONLY = true: add the terms that
// depend on w (convection, Newton) to the time-diagonal blocks of an operator that already
// holds that part.
// index of the unordered pair {a, b} of 1D Q2 nodes: (0,0) 0, (0,1) 1, (0,2) 2, (1,1) 3, (1,2) 4, (2,2) 5
__device__ __forceinline__ int pair3(int a, int b) {
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

template <int DIM, bool WONLY>
__global__ void __launch_bounds__(256) assemble_cells(Geom g, int colour, TimeData td, AsmCoef cf,
                                                      const double* __restrict__ w, const int* __restrict__ rowptr,
                                                      const double* __restrict__ tab, const double* __restrict__ K,
                                                      double* __restrict__ vv, double* __restrict__ vp,
                                                      double* __restrict__ pv) {
  constexpr int NQ = Pow3<DIM>::v;
  constexpr int NL = NQ;
  constexpr int ND = NL * DIM;
  constexpr int NTMAX = DIM == 2 ? 5 : 3;
  constexpr int NTC = DIM == 2 ? NTMAX : 1;  // precomputed convection/Newton matrices in 2D only
  __shared__ double phi[NQ][NL];
  __shared__ double dphi[NQ][NL][DIM];
  __shared__ double qwd[NQ];
  __shared__ double wq[NTMAX][NQ][DIM];
  __shared__ double gw[NTMAX][NQ][DIM][DIM];
  __shared__ double cm[NTC][NL][NL];
  // 2D sum factorisation (see below): 1D weighted products per Gauss point, contractions over
  // one direction, and the Newton blocks per pair of 1D index pairs
  constexpr int S2 = DIM == 2 ? 1 : 0;  // 3D: size-1 placeholders, indices scaled by S2
  constexpr int N3 = DIM == 2 ? 3 : 1, N5 = DIM == 2 ? 5 : 1, N6 = DIM == 2 ? 6 : 1;
  __shared__ double wll[2][N3][6];           // W_q L_a(q) L_b(q), per direction, pair (a, b)
  __shared__ double wld[2][N3][3][3];        // W_q L_a(q) D_b(q), per direction
  __shared__ double sfp[NTC][N5][3][6];      // P_f(q1; p2), f = w_x, g_xx, g_xy, g_yx, g_yy
  __shared__ double sfq[NTC][N3][6];         // Q(q2; p1) for w_y
  __shared__ double nmp[NTC][N6][6][DIM * DIM];
  __shared__ int slots[NL * NL];

  const int nt = g.nt, NV = g.NV;
  int cx, cy, cz;
  patch_cell(g, g.coff[colour] + blockIdx.x, cx, cy, cz);
  const int cc[3] = {cx, cy, cz};
  const long long cell = cell_id(g, cx, cy, cz);
  if (DIM == 2 && cell_masked(g, cx, cy)) {
    // a removed cell carries no element matrices (uniform over the block: safe early return)
    if (!WONLY) {
      const int nvp0 = NL * nt * DIM * (DIM + 1);
      for (int t = threadIdx.x; t < nvp0; t += blockDim.x) {
        vp[cell * nvp0 + t] = 0.0;
        pv[cell * nvp0 + t] = 0.0;
      }
    }
    return;
  }
  const unsigned cls = face_class<DIM>(g, cc);
  const double* mass = tab;
  const double* cvv = tab + NL * NL + (long long)cls * tab_class_size(DIM, NL);
  const double* cvp = cvv + (long long)ND * ND;
  const double* cpv = cvp + (long long)ND * (DIM + 1);

  {
    const double* x = tab + tab_extra_offset(DIM, NL);
    for (int t = threadIdx.x; t < NQ * NL; t += blockDim.x) {
      const int q = t / NL, i = t % NL;
      phi[q][i] = x[t];
      for (int e = 0; e < DIM; ++e) dphi[q][i][e] = x[NQ * NL + t * DIM + e];
    }
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) qwd[q] = x[NQ * NL * (1 + DIM) + q];
    if (DIM == 2 && WONLY) {
      // 1D tables of the tensor-product rule: direction d, Gauss point q, local 1D nodes a, b
      for (int t = threadIdx.x; t < 2 * 3 * 6; t += blockDim.x) {
        const int d = t / 18, q = (t / 6) % 3, pr = t % 6;
        const int pa = pr < 3 ? 0 : (pr < 5 ? 1 : 2), pb = pr < 3 ? pr : (pr < 5 ? pr - 2 : 2);  // inverse of pair3
        wll[d][q * S2][pr] = c_GW[q] * g.h[d] / 2.0 * c_L1[q][pa] * c_L1[q][pb];
      }
      for (int t = threadIdx.x; t < 2 * 27; t += blockDim.x) {
        const int d = t / 27, q = (t / 9) % 3, a = (t / 3) % 3, b = t % 3;
        wld[d][q * S2][a][b] = c_GW[q] * g.h[d] / 2.0 * c_L1[q][a] * (2.0 / g.h[d] * c_D1[q][b]);
      }
    }
  }
  for (int t = threadIdx.x; t < NL * NL; t += blockDim.x) {
    const int i = t / NL, j = t % NL;
    slots[t] = (int)bcsr_slot(g, rowptr, 2 * cx + i % 3, 2 * cy + (i / 3) % 3, 2 * cz + i / 9, 2 * cx + j % 3,
                              2 * cy + (j / 3) % 3, 2 * cz + j / 9);
  }
  __syncthreads();
  if (WONLY) {
    for (int t = threadIdx.x; t < nt * NQ * DIM; t += blockDim.x) {
      const int a = t / (NQ * DIM), q = (t / DIM) % NQ, c = t % DIM;
      double v = 0.0, gr[3] = {0.0, 0.0, 0.0};
      for (int i = 0; i < NL; ++i) {
        const long long nd = node_id(g, 2 * cx + i % 3, 2 * cy + (i / 3) % 3, 2 * cz + i / 9);
        const double wi = w[nd * NV + a * DIM + c];
        v += phi[q][i] * wi;
        for (int e = 0; e < DIM; ++e) gr[e] += dphi[q][i][e] * wi;
      }
      wq[a][q][c] = v;
      for (int e = 0; e < DIM; ++e) gw[a][q][c][e] = gr[e];
    }
    __syncthreads();
    if (DIM == 2) {
      // Sum factorisation over the tensor-product basis phi_i(q) = L_i1(q1) L_i2(q2) and the
      // 3 x 3 Gauss rule W_q = W_q1 W_q2 (x fastest in i and q).  With the contraction over q2
      //   P_f(q1; i2 j2) = sum_q2 W_q2 L_i2 L_j2 (q2) f(q1, q2),  f in {w_x, d_e w_c},
      // and over q1 for w_y, Q(q2; i1 j1) = sum_q1 W_q1 L_i1 L_j1 (q1) w_y(q1, q2):
      //   convection (w_a . grad phi_j, phi_i) = sum_q1 W L_i1 D^x_j1 (q1) P_wx(q1; i2 j2)
      //                                          + sum_q2 W L_i2 D^y_j2 (q2) Q(q2; i1 j1),
      //   Newton (phi_j d_e w_c, phi_i) = sum_q1 W L_i1 L_j1 (q1) P_{g_ce}(q1; i2 j2),
      // the latter a function of the unordered pairs {i1, j1}, {i2, j2} only (6 x 6 values).
      for (int t = threadIdx.x; t < nt * 5 * 3 * 6; t += blockDim.x) {
        const int a = t / 90, f = (t / 18) % 5, q1 = (t / 6) % 3, pr = t % 6;
        double sum = 0.0;
        for (int q2 = 0; q2 < 3; ++q2) {
          const int q = q1 + 3 * q2;
          const double fv = f == 0 ? wq[a][q][0] : gw[a][q][(f - 1) / 2][(f - 1) % 2];
          sum += wll[1][q2 * S2][pr] * fv;
        }
        sfp[a % NTC][f * S2][q1][pr] = sum;
      }
      for (int t = threadIdx.x; t < nt * 3 * 6; t += blockDim.x) {
        const int a = t / 18, q2 = (t / 6) % 3, pr = t % 6;
        double sum = 0.0;
        for (int q1 = 0; q1 < 3; ++q1) sum += wll[0][q1 * S2][pr] * wq[a][q1 + 3 * q2][1];
        sfq[a % NTC][q2 * S2][pr] = sum;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nt * NL * NL; t += blockDim.x) {
        const int a = t / (NL * NL), i = (t / NL) % NL, j = t % NL;
        const int i1 = i % 3, i2 = i / 3, j1 = j % 3, j2 = j / 3;
        double conv = 0.0;
        for (int q = 0; q < 3; ++q)
          conv += wld[0][q * S2][i1][j1] * sfp[a % NTC][0][q][pair3(i2, j2)] +
                  wld[1][q * S2][i2][j2] * sfq[a % NTC][q * S2][pair3(i1, j1)];
        cm[a % NTC][i][j] = cf.tau * td.w[a] * conv;
      }
      if (cf.newton)
        for (int t = threadIdx.x; t < nt * 36 * DIM * DIM; t += blockDim.x) {
          const int a = t / (36 * DIM * DIM), p1 = (t / (6 * DIM * DIM)) % 6, p2 = (t / (DIM * DIM)) % 6;
          const int ce = t % (DIM * DIM);
          double sum = 0.0;
          for (int q1 = 0; q1 < 3; ++q1) sum += wll[0][q1 * S2][p1] * sfp[a % NTC][(1 + ce) * S2][q1][p2];
          nmp[a % NTC][p1 * S2][p2][ce] = cf.tau * td.w[a] * sum;
        }
      __syncthreads();
    }

    if (DIM == 2) {
      // time-diagonal entries only: (i, j, a, c, e)
      const int nd = NL * NL * nt * DIM * DIM;
      for (int t = threadIdx.x; t < nd; t += blockDim.x) {
        const int e = t % DIM, c = (t / DIM) % DIM, a = (t / (DIM * DIM)) % nt;
        const int j = (t / (DIM * DIM * nt)) % NL, i = t / (DIM * DIM * nt * NL);
        double val = cf.newton ? nmp[a % NTC][pair3(i % 3, j % 3) * S2][pair3(i / 3, j / 3)][c * DIM + e] : 0.0;
        if (c == e) val += cm[a % NTC][i][j];
        const int r = a * DIM + c, sc = a * DIM + e;
        vv[(long long)slots[i * NL + j] * NV * NV + (long long)r * NV + sc] += val;
      }
    } else {
      // one task per (i, j, a): the convection value and the d x d Newton block over the
      // quadrature points, then the d x d entries of block (a, a) of node pair (i, j)
      for (int t = threadIdx.x; t < NL * NL * nt; t += blockDim.x) {
        const int a = t % nt, j = (t / nt) % NL, i = t / (nt * NL);
        double conv = 0.0, newt[DIM][DIM];
        for (int c = 0; c < DIM; ++c)
          for (int e = 0; e < DIM; ++e) newt[c][e] = 0.0;
        for (int q = 0; q < NQ; ++q) {
          double u = 0.0;
          for (int f = 0; f < DIM; ++f) u += wq[a][q][f] * dphi[q][j][f];
          const double wpi = qwd[q] * phi[q][i];
          conv += wpi * u;
          if (cf.newton) {
            const double pp = wpi * phi[q][j];
            for (int c = 0; c < DIM; ++c)
              for (int e = 0; e < DIM; ++e) newt[c][e] += pp * gw[a][q][c][e];
          }
        }
        const double sa = cf.tau * td.w[a];
        double* blk = vv + (long long)slots[i * NL + j] * NV * NV;
        for (int c = 0; c < DIM; ++c)
          for (int e = 0; e < DIM; ++e) {
            double val = cf.newton ? newt[c][e] : 0.0;
            if (c == e) val += conv;
            blk[(long long)(a * DIM + c) * NV + a * DIM + e] += sa * val;
          }
      }
    }
    return;
  }
  // constant part (the operator at w = 0): time coupling, viscous and Nitsche terms from the
  // class tables, the velocity-pressure blocks
  const long long kper = (long long)ND * ND;
  const int ncls = 1 << (2 * DIM);
  const long long nvv = (long long)NL * NL * NV * NV;
#pragma unroll 2
  for (long long t = threadIdx.x; t < nvv; t += blockDim.x) {
    const int s = (int)(t % NV), r = (int)((t / NV) % NV);
    const int j = (int)((t / (NV * NV)) % NL), i = (int)(t / ((long long)NV * NV * NL));
    const int a = r / DIM, c = r % DIM, b = s / DIM, e = s % DIM;
    double val;
    if (a == b) {
      val = K[((long long)a * ncls + cls) * kper + (i * DIM + c) * ND + j * DIM + e];
    } else {
      val = c == e ? td.T[a][b] * mass[i * NL + j] : 0.0;
    }
    vv[(long long)slots[i * NL + j] * NV * NV + (long long)r * NV + s] += val;
  }

  // velocity-pressure [cell][i][a][c][m] and pressure-velocity [cell][a][m][i][c]
  const int nvp = NL * nt * DIM * (DIM + 1);
  for (int t = threadIdx.x; t < nvp; t += blockDim.x) {
    const int m = t % (DIM + 1), c = (t / (DIM + 1)) % DIM, a = (t / ((DIM + 1) * DIM)) % nt;
    const int i = t / ((DIM + 1) * DIM * nt);
    const double sc = cf.tau * td.w[a];
    const int I = i * DIM + c;
    vp[(((cell * NL + i) * nt + a) * DIM + c) * (DIM + 1) + m] = sc * cvp[I * (DIM + 1) + m];
    pv[((cell * nt + a) * (DIM + 1) + m) * (long long)NL * DIM + I] = sc * cpv[m * ND + I];
  }
}


// Data terms of the right-hand side of Eq. (2.2), one CTA per face class:
//   NB[(i,c),(j,e)]: B_GammaD(phi_j e_e, (phi_i e_c, 0)) = -nu <phi_j, d_n phi_i> delta_ce
//                    + gamma1 nu / h <phi_j, phi_i> delta_ce + gamma2 / h <phi_j n_e, phi_i n_c>
//   PB[m][(j,e)]  : B_GammaD(phi_j e_e, (0, xi_m)) = -<phi_j n_e, xi_m>
template <int DIM>
__global__ void __launch_bounds__(256) rhs_constants(Geom g, AsmCoef cf, double* __restrict__ rt) {
  constexpr int NQ = Pow3<DIM>::v;
  constexpr int NL = NQ;
  constexpr int ND = NL * DIM;
  const unsigned faces = blockIdx.x;
  double* nb = rt + (long long)faces * (ND * ND + (DIM + 1) * ND);
  double* pb = nb + ND * ND;
  for (int t = threadIdx.x; t < ND * ND; t += blockDim.x) {
    const int I = t / ND, J = t % ND;
    const int i = I / DIM, c = I % DIM, j = J / DIM, e = J % DIM;
    double val = 0.0;
    for (int f = 0; f < 2 * DIM; ++f) {
      if (!(faces >> f & 1u)) continue;
      const int e0 = f >> 1, s0 = f & 1;
      const double ns = s0 ? 1.0 : -1.0, hf = g.h[e0];
      for (int fq = 0; fq < NQ / 3; ++fq) {
        int p[3];
        const double wt = face_point<DIM>(g, e0, s0, fq, p);
        double vi, vj, gi[3], gj[3];
        basis_at<DIM>(g, p, i, vi, gi);
        basis_at<DIM>(g, p, j, vj, gj);
        double term = 0.0;
        if (c == e) term += -cf.nu * vj * ns * gi[e0] + cf.gamma1 * cf.nu / hf * vj * vi;
        if (c == e0 && e == e0) term += cf.gamma2 / hf * vj * vi;
        val += wt * term;
      }
    }
    nb[t] = val;
  }
  for (int t = threadIdx.x; t < (DIM + 1) * ND; t += blockDim.x) {
    const int m = t / ND, J = t % ND, j = J / DIM, e = J % DIM;
    double val = 0.0;
    for (int f = 0; f < 2 * DIM; ++f) {
      if (!(faces >> f & 1u)) continue;
      const int e0 = f >> 1, s0 = f & 1;
      if (e != e0) continue;
      const double ns = s0 ? 1.0 : -1.0;
      for (int fq = 0; fq < NQ / 3; ++fq) {
        int p[3];
        const double wt = face_point<DIM>(g, e0, s0, fq, p);
        double vj, gj[3];
        basis_at<DIM>(g, p, j, vj, gj);
        const double xi = m == 0 ? 1.0 : c_X[p[m - 1]];
        val -= wt * vj * ns * xi;
      }
    }
    pb[t] = val;
  }
}

// Right-hand side b_a = tau w_a [ M f_a + NB g_a ] + chi_a(0) M v_prev (velocity rows, added
// colour by colour) and tau w_a PB g_a (pressure rows of the cell).  f, g: nodal data in
// the internal velocity layout [node][a][c]; v_prev: [node][c]; each may be null.
template <int DIM>
__global__ void __launch_bounds__(256) assemble_rhs(Geom g, int colour, TimeData td, AsmCoef cf,
                                                    const double* __restrict__ tab,
                                                    const double* __restrict__ rt, const double* __restrict__ f,
                                                    const double* __restrict__ gd,
                                                    const double* __restrict__ vprev, double* __restrict__ b) {
  constexpr int NL = Pow3<DIM>::v;
  constexpr int ND = NL * DIM;
  __shared__ double fl[NL * 5 * DIM], gl[NL * 5 * DIM], vl[NL * DIM];
  __shared__ long long nodes[NL];
  const int nt = g.nt, NV = g.NV;
  int cx, cy, cz;
  patch_cell(g, g.coff[colour] + blockIdx.x, cx, cy, cz);
  const int cc[3] = {cx, cy, cz};
  const long long cell = cell_id(g, cx, cy, cz);
  if (DIM == 2 && cell_masked(g, cx, cy)) return;  // removed cell: no data terms (b is zeroed)
  const unsigned cls = face_class<DIM>(g, cc);
  const double* nb = rt + (long long)cls * (ND * ND + (DIM + 1) * ND);
  const double* pb = nb + ND * ND;
  for (int i = threadIdx.x; i < NL; i += blockDim.x)
    nodes[i] = node_id(g, 2 * cx + i % 3, 2 * cy + (i / 3) % 3, 2 * cz + i / 9);
  __syncthreads();
  for (int t = threadIdx.x; t < NL * NV; t += blockDim.x) {
    const int i = t / NV, v = t % NV;
    fl[t] = f ? f[nodes[i] * NV + v] : 0.0;
    gl[t] = gd ? gd[nodes[i] * NV + v] : 0.0;
  }
  for (int t = threadIdx.x; t < NL * DIM; t += blockDim.x) vl[t] = vprev ? vprev[nodes[t / DIM] * DIM + t % DIM] : 0.0;
  __syncthreads();
  for (int t = threadIdx.x; t < NL * NV; t += blockDim.x) {
    const int i = t / NV, v = t % NV, a = v / DIM, c = v % DIM;
    double mf = 0.0, mv = 0.0, ng = 0.0;
    for (int j = 0; j < NL; ++j) {
      const double mij = tab[i * NL + j];
      mf += mij * fl[j * NV + v];
      mv += mij * vl[j * DIM + c];
      for (int e = 0; e < DIM; ++e) ng += nb[(i * DIM + c) * ND + j * DIM + e] * gl[j * NV + a * DIM + e];
    }
    b[nodes[i] * NV + v] += cf.tau * td.w[a] * (mf + ng) + td.jump[a] * mv;
  }
  for (int t = threadIdx.x; t < nt * (DIM + 1); t += blockDim.x) {
    const int a = t / (DIM + 1), m = t % (DIM + 1);
    double s = 0.0;
    for (int J = 0; J < ND; ++J) s += pb[m * ND + J] * gl[(J / DIM) * NV + a * DIM + J % DIM];
    b[g.nvel + cell * g.NP + t] = cf.tau * td.w[a] * s;
  }
}

// ---------------------------------------------------------------- order 4 (2D), (Q4)^2 x P3disc
// One CTA per cell: the whole element matrix of the space-time block (time coupling, viscous,
// convection and Newton at w_a, the Nitsche terms of the cell's Dirichlet faces) by quadrature
// with the 5 x 5 Gauss rule (5 points per face), added into the cell's BCSR blocks, and the
// velocity-pressure / pressure-velocity blocks.  w = nullptr: the operator at w = 0.
// P3 monomials xi^a eta^b in the order (0,0) (1,0) (0,1) (2,0) (1,1) (0,2) (3,0) (2,1) (1,2) (0,3).
__device__ __forceinline__ double p3_monomial(int m, double x, double y) {
  const int ea[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0}, eb[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
  double v = 1.0;
  for (int i = 0; i < ea[m]; ++i) v *= x;
  for (int i = 0; i < eb[m]; ++i) v *= y;
  return v;
}

__global__ void __launch_bounds__(256) assemble_cells_q4(Geom g, int colour, TimeData td, AsmCoef cf,
                                                         const double* __restrict__ w,
                                                         const int* __restrict__ rowptr, double* __restrict__ vv,
                                                         double* __restrict__ vp, double* __restrict__ pv) {
  constexpr int NL = 25, NQ = 25, NF = 5, NPD = 10;
  __shared__ double phi[NQ][NL];
  __shared__ double dphi[NQ][NL][2];
  __shared__ double qwd[NQ];
  __shared__ double wq[5][NQ][2];
  __shared__ double gw[5][NQ][2][2];
  __shared__ int slots[NL * NL];
  const int nt = g.nt, NV = g.NV;
  int cx, cy, cz;
  patch_cell(g, g.coff[colour] + blockIdx.x, cx, cy, cz);
  const int cc[3] = {cx, cy, 0};
  const long long cell = cell_id(g, cx, cy, 0);
  const unsigned faces = face_class<2>(g, cc);
  const double hx = g.h[0], hy = g.h[1];
  for (int t = threadIdx.x; t < NQ * NL; t += blockDim.x) {
    const int q = t / NL, i = t % NL;
    const int q1 = q % 5, q2 = q / 5, i1 = i % 5, i2 = i / 5;
    phi[q][i] = c_L4[q1][i1] * c_L4[q2][i2];
    dphi[q][i][0] = 2.0 / hx * c_D4[q1][i1] * c_L4[q2][i2];
    dphi[q][i][1] = 2.0 / hy * c_L4[q1][i1] * c_D4[q2][i2];
    if (i == 0) qwd[q] = c_GW4[q1] * c_GW4[q2] * hx * hy / 4.0;
  }
  for (int t = threadIdx.x; t < NL * NL; t += blockDim.x) {
    const int i = t / NL, j = t % NL;
    slots[t] = (int)bcsr_slot(g, rowptr, 4 * cx + i % 5, 4 * cy + i / 5, 0, 4 * cx + j % 5, 4 * cy + j / 5, 0);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nt * NQ * 2; t += blockDim.x) {
    const int a = t / (NQ * 2), q = (t / 2) % NQ, c = t % 2;
    double v = 0.0, g0 = 0.0, g1 = 0.0;
    if (w)
      for (int i = 0; i < NL; ++i) {
        const double wi = w[node_id(g, 4 * cx + i % 5, 4 * cy + i / 5, 0) * NV + a * 2 + c];
        v += phi[q][i] * wi;
        g0 += dphi[q][i][0] * wi;
        g1 += dphi[q][i][1] * wi;
      }
    wq[a][q][c] = v;
    gw[a][q][c][0] = g0;
    gw[a][q][c][1] = g1;
  }
  __syncthreads();
  // one task per node pair (i, j): the scalar integrals, the Newton and Nitsche d x d blocks
  for (int t = threadIdx.x; t < NL * NL; t += blockDim.x) {
    const int i = t / NL, j = t % NL;
    double mass = 0.0, stiff = 0.0, conv[5] = {0, 0, 0, 0, 0}, newt[5][2][2] = {};
    for (int q = 0; q < NQ; ++q) {
      const double wpi = qwd[q] * phi[q][i];
      mass += wpi * phi[q][j];
      stiff += qwd[q] * (dphi[q][i][0] * dphi[q][j][0] + dphi[q][i][1] * dphi[q][j][1]);
      for (int a = 0; a < nt; ++a) {
        conv[a] += wpi * (wq[a][q][0] * dphi[q][j][0] + wq[a][q][1] * dphi[q][j][1]);
        if (cf.newton) {
          const double pp = wpi * phi[q][j];
          for (int c = 0; c < 2; ++c)
            for (int e = 0; e < 2; ++e) newt[a][c][e] += pp * gw[a][q][c][e];
        }
      }
    }
    double fs = 0.0, fn[2][2] = {{0, 0}, {0, 0}};
    for (int f = 0; f < 4; ++f) {
      if (!(faces >> f & 1u)) continue;
      const int e0 = f >> 1, s0 = f & 1;
      const double nrm = s0 ? 1.0 : -1.0, hf = g.h[e0], hl = g.h[1 - e0];
      for (int fq = 0; fq < NF; ++fq) {
        const int p0 = e0 == 0 ? 5 + s0 : fq, p1 = e0 == 1 ? 5 + s0 : fq;
        const double wt = c_GW4[fq] * hl / 2.0;
        const double vi = c_L4[p0][i % 5] * c_L4[p1][i / 5], vj = c_L4[p0][j % 5] * c_L4[p1][j / 5];
        const double di = (e0 == 0 ? 2.0 / hx * c_D4[p0][i % 5] * c_L4[p1][i / 5]
                                   : 2.0 / hy * c_L4[p0][i % 5] * c_D4[p1][i / 5]) * nrm;
        const double dj = (e0 == 0 ? 2.0 / hx * c_D4[p0][j % 5] * c_L4[p1][j / 5]
                                   : 2.0 / hy * c_L4[p0][j % 5] * c_D4[p1][j / 5]) * nrm;
        fs += wt * (-cf.nu * dj * vi - cf.nu * vj * di + cf.gamma1 * cf.nu / hf * vj * vi);
        fn[e0][e0] += wt * cf.gamma2 / hf * vj * vi;  // n n^T has the single entry (e0, e0)
      }
    }
    double* blk = vv + (long long)slots[i * NL + j] * NV * NV;
    for (int a = 0; a < nt; ++a)
      for (int b = 0; b < nt; ++b)
        for (int c = 0; c < 2; ++c)
          for (int e = 0; e < 2; ++e) {
            double val = c == e ? td.T[a][b] * mass : 0.0;
            if (a == b) {
              double sp = fn[c][e] + (cf.newton ? newt[a][c][e] : 0.0);
              if (c == e) sp += conv[a] + cf.nu * stiff + fs;
              val += cf.tau * td.w[a] * sp;
            }
            blk[(long long)(a * 2 + c) * NV + b * 2 + e] += val;
          }
  }
  // velocity-pressure [cell][i][a][c][m] and pressure-velocity [cell][a][m][i][c] (w-independent:
  // written by the set-up's call, skipped by re-linearisations, vp == nullptr)
  if (!vp) return;
  for (int t = threadIdx.x; t < NL * 2 * NPD; t += blockDim.x) {
    const int m = t % NPD, c = (t / NPD) % 2, i = t / (NPD * 2);
    double val = 0.0;
    for (int q = 0; q < NQ; ++q)
      val -= qwd[q] * p3_monomial(m, c_X4[q % 5], c_X4[q / 5]) * dphi[q][i][c];
    for (int f = 0; f < 4; ++f) {
      if (!(faces >> f & 1u)) continue;
      const int e0 = f >> 1, s0 = f & 1;
      if (e0 != c) continue;  // <xi_m n_c, phi_i> with n along e0 only
      const double nrm = s0 ? 1.0 : -1.0, hl = g.h[1 - e0];
      for (int fq = 0; fq < NF; ++fq) {
        const int p0 = e0 == 0 ? 5 + s0 : fq, p1 = e0 == 1 ? 5 + s0 : fq;
        val += c_GW4[fq] * hl / 2.0 * p3_monomial(m, c_X4[p0], c_X4[p1]) * nrm * c_L4[p0][i % 5] *
               c_L4[p1][i / 5];
      }
    }
    for (int a = 0; a < nt; ++a) {
      const double sc = cf.tau * td.w[a];
      vp[(((cell * NL + i) * nt + a) * 2 + c) * NPD + m] = sc * val;
      pv[((cell * nt + a) * NPD + m) * (long long)NL * 2 + i * 2 + c] = -sc * val;
    }
  }
}

// Identity rows of the unknowns without an equation (obstacle): I added to the diagonal block
// of every Q2 node of removed cells only (the pressure of removed cells is handled by the
// residual and the patch inversion, as the velocity-pressure blocks carry no diagonal).
__global__ void dead_node_identity(Geom g, const int* __restrict__ rowptr, double* __restrict__ vv) {
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.n_nodes) return;
  const int ix = (int)(node % g.nn[0]), iy = (int)(node / g.nn[0]);
  if (!node_dead(g, ix, iy)) return;
  const long long slot = bcsr_slot(g, rowptr, ix, iy, 0, ix, iy, 0);
  for (int r = 0; r < g.NV; ++r) vv[(slot * g.NV + r) * g.NV + r] += 1.0;
}

}  // namespace

long long assemble_table_doubles(int dim, int k) {
  const int nloc = dim == 2 ? 9 : 27, nq = nloc;
  const long long nd = (long long)nloc * dim;
  const long long base = tab_extra_offset(dim, nloc) + (long long)nq * nloc * (1 + dim) + nq + (long long)nq * nloc * nloc;
  return base + (long long)(k + 1) * (1LL << (2 * dim)) * nd * nd;  // followed by K
}

static void assemble_level_q4(const Geom& g, const TimeData& td, const AsmCoef& cf, const double* w_int,
                              const int* rowptr, double* vv, long long nnzb, double* vp, double* pv, cudaStream_t st) {
  STG_CUDA_OK(cudaMemsetAsync(vv, 0, sizeof(double) * nnzb * g.NV * g.NV, st));
  for (int col = 0; col < 4; ++col) {
    const long long cnt = g.coff[col + 1] - g.coff[col];
    if (cnt == 0) continue;
    assemble_cells_q4<<<(unsigned)cnt, 256, 0, st>>>(g, col, td, cf, w_int, rowptr, vv, vp, pv);
    STG_LAUNCH_OK();
  }
}

void assemble_level(const Geom& g, const TimeData& td, const AsmCoef& cf, const double* w_int, const int* rowptr,
                    double* tab, double* vv, long long nnzb, double* vp, double* pv, cudaStream_t st) {
  if (g.r == 4) {  // order 4: the whole operator at w_int (null: w = 0) by the generic kernel
    assemble_level_q4(g, td, cf, w_int, rowptr, vv, nnzb, vp, pv, st);
    return;
  }
  STG_CUDA_OK(cudaMemsetAsync(vv, 0, sizeof(double) * nnzb * g.NV * g.NV, st));
  const unsigned ncls = 1u << (2 * g.dim);
  const int nloc = g.dim == 2 ? 9 : 27;
  double* K = tab + assemble_table_doubles(g.dim, -1);
  if (g.dim == 2)
    element_constants<2><<<ncls, 256, 0, st>>>(g, cf, tab);
  else
    element_constants<3><<<ncls, 256, 0, st>>>(g, cf, tab);
  STG_LAUNCH_OK();
  const long long nK = (long long)g.nt * ncls * nloc * g.dim * nloc * g.dim;
  if (g.dim == 2)
    diag_blocks<2><<<grid_for(nK, 256), 256, 0, st>>>(g, td, cf, tab, K);
  else
    diag_blocks<3><<<grid_for(nK, 256), 256, 0, st>>>(g, td, cf, tab, K);
  STG_LAUNCH_OK();
  for (int col = 0; col < (1 << g.dim); ++col) {
    const long long cnt = g.coff[col + 1] - g.coff[col];
    if (cnt == 0) continue;
    if (g.dim == 2)
      assemble_cells<2, false><<<(unsigned)cnt, 128, 0, st>>>(g, col, td, cf, w_int, rowptr, tab, K, vv, vp, pv);
    else
      assemble_cells<3, false><<<(unsigned)cnt, 256, 0, st>>>(g, col, td, cf, w_int, rowptr, tab, K, vv, vp, pv);
    STG_LAUNCH_OK();
  }
  if (has_obstacle(g)) {
    dead_node_identity<<<grid_for(g.n_nodes, 256), 256, 0, st>>>(g, rowptr, vv);
    STG_LAUNCH_OK();
  }
}

void assemble_level_w(const Geom& g, const TimeData& td, const AsmCoef& cf, const double* w_int, const int* rowptr,
                      const double* tab, const double* vconst, double* vv, long long nnzb, cudaStream_t st) {
  if (g.r == 4) {
    assemble_level_q4(g, td, cf, w_int, rowptr, vv, nnzb, nullptr, nullptr, st);
    return;
  }
  STG_CUDA_OK(cudaMemcpyAsync(vv, vconst, sizeof(double) * nnzb * g.NV * g.NV, cudaMemcpyDeviceToDevice, st));
  const double* K = tab + assemble_table_doubles(g.dim, -1);
  for (int col = 0; col < (1 << g.dim); ++col) {
    const long long cnt = g.coff[col + 1] - g.coff[col];
    if (cnt == 0) continue;
    if (g.dim == 2)
      assemble_cells<2, true><<<(unsigned)cnt, 128, 0, st>>>(g, col, td, cf, w_int, rowptr, tab, K, vv, nullptr,
                                                           nullptr);
    else
      assemble_cells<3, true><<<(unsigned)cnt, 256, 0, st>>>(g, col, td, cf, w_int, rowptr, tab, K, vv, nullptr,
                                                           nullptr);
    STG_LAUNCH_OK();
  }
}

}  // namespace stg

namespace stg {

namespace {

// Force of the fluid on the obstacle (2D) at every Radau node,
//   F_a = - sum over the faces of remaining cells that border the obstacle of
//         int_F (nu grad v_h - p_h I) n dS        (n: the fluid cell's outward normal),
// with the 3-point Gauss rule per face.  One CTA; each thread takes (face, Radau node) tasks
// and the partial sums are reduced in shared memory in a fixed order.
__global__ void __launch_bounds__(256) obstacle_forces_kernel(Geom g, double nu, const double* __restrict__ x,
                                                            double* __restrict__ out) {
  constexpr int NL = 9;
  __shared__ double part[256][2 * 5];
  const int tid = threadIdx.x, nt = g.nt, NV = g.NV;
  double acc[2 * 5];
  for (int i = 0; i < 2 * 5; ++i) acc[i] = 0.0;
  // faces: (e, side, fixed cell index along e, range along the other direction)
  const int nf0 = g.ob[3] - g.ob[2], nf1 = g.ob[1] - g.ob[0];
  const int nfaces = 2 * nf0 + 2 * nf1;
  for (int task = tid; task < nfaces * nt; task += blockDim.x) {
    const int f = task / nt, a = task % nt;
    int cx, cy, e, side;
    if (f < nf0) {  // left of the obstacle: the cell's high-x face
      e = 0; side = 1; cx = g.ob[0] - 1; cy = g.ob[2] + f;
    } else if (f < 2 * nf0) {  // right of it: the low-x face
      e = 0; side = 0; cx = g.ob[1]; cy = g.ob[2] + f - nf0;
    } else if (f < 2 * nf0 + nf1) {  // below: the high-y face
      e = 1; side = 1; cx = g.ob[0] + f - 2 * nf0; cy = g.ob[2] - 1;
    } else {  // above: the low-y face
      e = 1; side = 0; cx = g.ob[0] + f - 2 * nf0 - nf1; cy = g.ob[3];
    }
    if (cx < 0 || cx >= g.n[0] || cy < 0 || cy >= g.n[1]) continue;  // obstacle on the domain boundary
    const double nrm = side ? 1.0 : -1.0;
    const long long cell = cell_id(g, cx, cy, 0);
    const double* pc = x + g.nvel + cell * g.NP + a * 3;
    for (int fq = 0; fq < 3; ++fq) {
      int pidx[3] = {0, 0, 0};
      const double wt = face_point<2>(g, e, side, fq, pidx);
      double gv[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
      for (int i = 0; i < NL; ++i) {
        double v, gr[3];
        basis_at<2>(g, pidx, i, v, gr);
        const long long nd = node_id(g, 2 * cx + i % 3, 2 * cy + i / 3, 0);
        for (int c = 0; c < 2; ++c) {
          const double vi = x[nd * NV + a * 2 + c];
          gv[c][0] += gr[0] * vi;
          gv[c][1] += gr[1] * vi;
        }
      }
      // P1disc {1, xi, eta} at the face point
      const double xi = c_X[pidx[0]], eta = c_X[pidx[1]];
      const double p = pc[0] + pc[1] * xi + pc[2] * eta;
      for (int c = 0; c < 2; ++c) {
        const double trac = nu * gv[c][e] * nrm - (c == e ? p * nrm : 0.0);
        acc[2 * a + c] -= wt * trac;
      }
    }
  }
  for (int i = 0; i < 2 * 5; ++i) part[tid][i] = acc[i];
  __syncthreads();
  if (tid < 2 * nt) {
    double sum = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) sum += part[t][tid];
    out[tid] = sum;
  }
}

}  // namespace

void obstacle_forces(const Geom& g, double nu, const double* x_int, double* out, cudaStream_t st) {
  obstacle_forces_kernel<<<1, 256, 0, st>>>(g, nu, x_int, out);
  STG_LAUNCH_OK();
}

long long rhs_table_doubles(int dim) {
  const long long nd = (long long)(dim == 2 ? 9 : 27) * dim;
  return (1LL << (2 * dim)) * (nd * nd + (dim + 1) * nd);
}

void assemble_rhs_level(const Geom& g, const TimeData& td, const AsmCoef& cf, const double* tab, double* rt,
                        const double* f, const double* gd, const double* vprev, double* b, cudaStream_t st) {
  STG_CUDA_OK(cudaMemsetAsync(b, 0, sizeof(double) * g.N, st));
  const unsigned ncls = 1u << (2 * g.dim);
  if (g.dim == 2)
    rhs_constants<2><<<ncls, 256, 0, st>>>(g, cf, rt);
  else
    rhs_constants<3><<<ncls, 256, 0, st>>>(g, cf, rt);
  STG_LAUNCH_OK();
  for (int col = 0; col < (1 << g.dim); ++col) {
    const long long cnt = g.coff[col + 1] - g.coff[col];
    if (cnt == 0) continue;
    if (g.dim == 2)
      assemble_rhs<2><<<(unsigned)cnt, 128, 0, st>>>(g, col, td, cf, tab, rt, f, gd, vprev, b);
    else
      assemble_rhs<3><<<(unsigned)cnt, 256, 0, st>>>(g, col, td, cf, tab, rt, f, gd, vprev, b);
    STG_LAUNCH_OK();
  }
}

}  // namespace stg
