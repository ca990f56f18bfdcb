// C-ABI of the solver: context, level hierarchy, V-cycle and flexible GMRES (Sec. 3).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "cnn.cuh"
#include "coarse.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace stg {

long long& launch_counter() {
  static long long n = 0;
  return n;
}

bool& launch_overlap() {
  static thread_local bool on = false;
  return on;
}

// ------------------------------------------------------------------ geometry
Geom make_geom(const stg_mesh& m, int level, int k) {
  Geom g{};
  g.dim = m.dim;
  g.k = k;
  g.nt = k + 1;
  const int f = 1 << (m.n_levels - 1 - level);
  g.r = m.order == 4 ? 4 : 2;
  g.npd = g.r == 2 ? m.dim + 1 : (m.dim == 2 ? 10 : 20);
  const int nf[3] = {m.nx, m.ny, m.dim == 3 ? m.nz : 1};
  const double lo[3] = {m.x0, m.y0, m.z0}, hi[3] = {m.x1, m.y1, m.z1};
  for (int e = 0; e < 3; ++e) {
    if (e < m.dim) {
      g.n[e] = nf[e] / f;
      g.nn[e] = g.r * g.n[e] + 1;
      g.lo[e] = lo[e];
      g.h[e] = (hi[e] - lo[e]) / g.n[e];
    } else {
      g.n[e] = 1;
      g.nn[e] = 1;
      g.lo[e] = 0.0;
      g.h[e] = 1.0;
    }
  }
  g.dirichlet = m.dirichlet_faces;
  const int fo = 1 << level;  // the obstacle box is given in coarsest-level cells
  for (int i = 0; i < 4; ++i) g.ob[i] = m.obstacle[i] * fo;
  if (g.ob[1] <= g.ob[0] || g.ob[3] <= g.ob[2]) g.ob[0] = g.ob[1] = g.ob[2] = g.ob[3] = 0;
  g.NV = g.nt * g.dim;
  g.NP = g.nt * g.npd;
  g.nloc = g.dim == 2 ? (g.r + 1) * (g.r + 1) : (g.r + 1) * (g.r + 1) * (g.r + 1);
  g.npatch = g.nloc * g.NV + g.NP;
  g.n_nodes = (long long)g.nn[0] * g.nn[1] * g.nn[2];
  g.n_cells = (long long)g.n[0] * g.n[1] * g.n[2];
  g.nvel = g.n_nodes * g.NV;
  g.npres = g.n_cells * g.NP;
  g.N = g.nvel + g.npres;
  g.coff[0] = 0;
  for (int c = 0; c < 8; ++c) {
    long long cnt = 1;
    for (int e = 0; e < 3; ++e) {
      const int p = (c >> e) & 1;
      int ce;
      if (e < g.dim)
        ce = (g.n[e] - p + 1) / 2;
      else
        ce = p ? 0 : 1;
      g.ccount[c][e] = ce;
      cnt *= ce;
    }
    if (c >= (1 << g.dim)) cnt = 0;
    g.coff[c + 1] = g.coff[c] + cnt;
  }
  return g;
}

// ------------------------------------------------------------------ time basis
namespace {
double legendre(int n, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = x;
  for (int i = 1; i < n; ++i) {
    const double p2 = ((2.0 * i + 1.0) * x * p1 - i * p0) / (i + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Sign-change roots of f on (-1, 1) by bisection to machine precision.
template <typename F>
std::vector<double> roots_in(F f) {
  std::vector<double> x;
  const int ns = 4000;
  for (int i = 0; i < ns - 1; ++i) {
    double a = -1.0 + 2.0 * i / ns, b = -1.0 + 2.0 * (i + 1) / ns;
    double fa = f(a);
    const double fb = f(b);
    if (fa == 0.0) {
      x.push_back(a);
      continue;
    }
    if (fa * fb < 0.0) {
      for (int it = 0; it < 200; ++it) {
        const double m = 0.5 * (a + b), fm = f(m);
        if (fa * fm <= 0.0) {
          b = m;
        } else {
          a = m;
          fa = fm;
        }
      }
      x.push_back(0.5 * (a + b));
    }
  }
  return x;
}

// Lagrange polynomial a at nodes c, and its derivative, in product form.
double lag(const std::vector<double>& c, int a, double s) {
  double v = 1.0;
  for (size_t b = 0; b < c.size(); ++b)
    if ((int)b != a) v *= (s - c[b]) / (c[a] - c[b]);
  return v;
}
double dlag(const std::vector<double>& c, int a, double s) {
  double d = 0.0;
  for (size_t m = 0; m < c.size(); ++m) {
    if ((int)m == a) continue;
    double t = 1.0 / (c[a] - c[m]);
    for (size_t l = 0; l < c.size(); ++l)
      if ((int)l != a && l != m) t *= (s - c[l]) / (c[a] - c[l]);
    d += t;
  }
  return d;
}
}  // namespace

TimeData time_basis(int k) {
  // right Radau points: roots of P_k - P_{k+1} on (-1, 1], mapped to [0, 1]
  std::vector<double> x = roots_in([k](double t) { return legendre(k, t) - legendre(k + 1, t); });
  x.push_back(1.0);
  if ((int)x.size() != k + 1) throw Error{STG_EINVAL, "Radau root search failed"};
  // (k+1)-point Gauss-Legendre rule on [0, 1]: exact for the degree-2k integrands below
  const int nq = k + 1;
  std::vector<double> gx = roots_in([nq](double t) { return legendre(nq, t); });
  if ((int)gx.size() != nq) throw Error{STG_EINVAL, "Gauss root search failed"};
  std::vector<double> q(nq), qw(nq);
  for (int i = 0; i < nq; ++i) {
    const double t = gx[i];
    const double dp = nq * (t * legendre(nq, t) - legendre(nq - 1, t)) / (t * t - 1.0);
    q[i] = 0.5 * (t + 1.0);
    qw[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2 / ((1 - t^2) P'(t)^2), halved for [0, 1]
  }
  TimeData td{};
  std::vector<double> c(k + 1);
  for (int a = 0; a <= k; ++a) c[a] = 0.5 * (x[a] + 1.0);
  for (int a = 0; a <= k; ++a) {
    td.c[a] = c[a];
    td.jump[a] = lag(c, a, 0.0);
    double w = 0.0;
    for (int i = 0; i < nq; ++i) w += qw[i] * lag(c, a, q[i]);
    td.w[a] = w;
  }
  for (int a = 0; a <= k; ++a)
    for (int b = 0; b <= k; ++b) {
      double t = 0.0;
      for (int i = 0; i < nq; ++i) t += qw[i] * dlag(c, b, q[i]) * lag(c, a, q[i]);
      td.T[a][b] = t + td.jump[a] * td.jump[b];
    }
  return td;
}

}  // namespace stg

using namespace stg;

// ------------------------------------------------------------------ context
struct LevelBufs {
  Geom g{};
  int* rowptr = nullptr;
  int* colidx = nullptr;
  long long nnzb = 0;
  double *vv = nullptr, *vp = nullptr, *pv = nullptr;
  float *vv32 = nullptr, *vp32 = nullptr, *pv32 = nullptr;
  double* vconst = nullptr;  // the w = 0 assembly (time coupling, viscous, Nitsche), built once
  float *mk32 = nullptr, *ak32 = nullptr;  // Kronecker-split FP32 velocity rows (F32 form, levels >= 1, 2D)
  void* jinv = nullptr;
  double* w = nullptr;
  double* asm_tab = nullptr;
  int colour_variant = kColourDefault;
  void *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr;
};

struct stg_ctx {
  stg_mesh mesh{};
  stg_options opt{};
  int k = 0;
  double nu = 0, tau = 0;
  cudaStream_t st = nullptr;
  // side stream of the set-up: the coarse factorisation overlaps the finer levels' work
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // aux stream of the set-up: the intermediate levels (assembly and inversion) run beside the
  // finest level's chain
  cudaStream_t aux = nullptr;
  cudaEvent_t aux_done = nullptr;
  TimeData td{};
  std::vector<LevelBufs> lv;
  CoarseSolver<double> coarse64;  // FP64 form
  CoarseSolver<float> coarse32;   // FP32 form: FP32 factors, FP64 iterative refinement
  double *cb64 = nullptr, *cx64 = nullptr, *cr64 = nullptr, *cd64 = nullptr;
  int* status = nullptr;
  void* inv_scratch = nullptr;
  int* inv_flags = nullptr;  // per patch: redo with pivoting
  // the same for the intermediate levels, which are inverted concurrently with the finest
  void* inv_scratch2 = nullptr;
  int* inv_flags2 = nullptr;
  // FGMRES (finest level, internal layout, FP64)
  double *V = nullptr, *Z = nullptr, *wv = nullptr, *rv = nullptr, *partial = nullptr, *hd = nullptr;
  double *vin = nullptr, *vout = nullptr, *tmp_a = nullptr, *tmp_b = nullptr;
  double* hh = nullptr;  // pinned host
  cudaGraphExec_t graph = nullptr;
  long long graph_kernels = 0;
  int graph_prof_events = 0;
  long long graph_prof_patches = 0;
  // instrumentation: CUDA events around the finest-level colour kernels
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;
  int prof_used = 0;
  double prof_ms = 0.0;
  long long prof_launches = 0, prof_patches = 0, prof_pending_patches = 0;
  // damped Newton (finest level, internal layout, FP64)
  double *nb = nullptr, *nX = nullptr, *nr = nullptr, *nC = nullptr, *nXt = nullptr;
  double *nf = nullptr, *ng = nullptr, *rhs_tab = nullptr;
  // warm start of the next slab: network input and reduction scratch
  float* wfeat = nullptr;
  double* wsum = nullptr;
  std::vector<void*> owned;
  std::string err;
  bool pure_dirichlet = false;
};

namespace {

thread_local std::string g_setup_error;

template <typename T>
T* dalloc(stg_ctx* c, long long n) {
  T* p = nullptr;
  const size_t bytes = sizeof(T) * (size_t)(n > 0 ? n : 1);
  const cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{STG_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
  }
  c->owned.push_back(p);
  return p;
}

size_t fsize(int prec) { return prec == STG_F64 ? 8 : (prec == STG_F32 ? 4 : 2); }

void build_pattern(stg_ctx* c, LevelBufs& L) {
  const Geom& g = L.g;
  std::vector<int> rowptr(g.n_nodes + 1, 0);
  std::vector<int> colidx;
  long long nnz = 0;
  for (int iz = 0; iz < g.nn[2]; ++iz)
    for (int iy = 0; iy < g.nn[1]; ++iy)
      for (int ix = 0; ix < g.nn[0]; ++ix) {
        int xl, xh, yl, yh, zl, zh;
        stencil_range(ix, g.nn[0], xl, xh, g.r);
        stencil_range(iy, g.nn[1], yl, yh, g.r);
        stencil_range(iz, g.nn[2], zl, zh, g.r);
        for (int jz = zl; jz <= zh; ++jz)
          for (int jy = yl; jy <= yh; ++jy)
            for (int jx = xl; jx <= xh; ++jx) colidx.push_back((int)node_id(g, jx, jy, jz));
        nnz += (long long)(xh - xl + 1) * (yh - yl + 1) * (zh - zl + 1);
        if (nnz > 2147483647LL) throw Error{STG_EINVAL, "level too large for 32-bit block indices"};
        rowptr[node_id(g, ix, iy, iz) + 1] = (int)nnz;
      }
  L.nnzb = nnz;
  L.rowptr = dalloc<int>(c, g.n_nodes + 1);
  L.colidx = dalloc<int>(c, nnz);
  STG_CUDA_OK(cudaMemcpy(L.rowptr, rowptr.data(), sizeof(int) * rowptr.size(), cudaMemcpyHostToDevice));
  STG_CUDA_OK(cudaMemcpy(L.colidx, colidx.data(), sizeof(int) * colidx.size(), cudaMemcpyHostToDevice));
}

bool vc64(const stg_ctx* c) { return c->opt.vcycle_prec == STG_F64; }
// FP64 coarse factors: always with the FP64 V-cycle, on request with the FP32 one
bool coarse64(const stg_ctx* c) { return vc64(c) || c->opt.coarse_prec == STG_F64; }

// Assemble every level for the finest-level linearisation velocity in F.w (internal
// layout), invert the local matrices, factor the coarse system.
void linearise_internal(stg_ctx* c) {
  const int nl = (int)c->lv.size();
  for (int l = nl - 1; l > 0; --l) inject_w(c->lv[l - 1].g, c->lv[l].g, c->lv[l].w, c->lv[l - 1].w, c->st);
  AsmCoef cf{c->nu, c->tau, c->opt.gamma1, c->opt.gamma2, c->opt.linearisation == STG_NEWTON ? 1 : 0};
  STG_CUDA_OK(cudaMemsetAsync(c->status, 0, sizeof(int) * 4, c->st));
  // three chains once w is on every level: the finest level on the main stream; the coarse
  // level and its factorisation (a chain of small, latency-bound launches) on the side stream;
  // the intermediate levels on the aux stream.  The finest chain is enqueued first; the other
  // two have the higher stream priority, so their smaller grids do not queue behind it.
  STG_CUDA_OK(cudaEventRecord(c->fork, c->st));
  STG_CUDA_OK(cudaStreamWaitEvent(c->side, c->fork, 0));
  STG_CUDA_OK(cudaStreamWaitEvent(c->aux, c->fork, 0));
  // FP32 copies of a level's operator for the FP32 V-cycle (Kronecker split where there is one)
  auto to_f32 = [&](LevelBufs& L, cudaStream_t s) {
    if (vc64(c)) return;
    if (L.vv32) convert(L.nnzb * L.g.NV * L.g.NV, L.vv, L.vv32, s);
    const long long nvp = L.g.n_cells * L.g.nloc * L.g.nt * L.g.dim * L.g.npd;
    convert(nvp, L.vp, L.vp32, s);
    convert(nvp, L.pv, L.pv32, s);
    if (L.mk32) kron_split(L.g, L.nnzb, L.vv, c->td, L.mk32, L.ak32, s);
  };
  for (int i = 0; i < nl; ++i) {
    const int l = i == 0 ? nl - 1 : i - 1;
    LevelBufs& L = c->lv[l];
    cudaStream_t s = l == 0 ? c->side : (l == nl - 1 ? c->st : c->aux);
    assemble_level_w(L.g, c->td, cf, L.w, L.rowptr, L.asm_tab, L.vconst, L.vv, L.nnzb, s);
    to_f32(L, s);
    if (l == 0) {
      if (coarse64(c))
        c->coarse64.factor(L.rowptr, L.colidx, L.vv, L.vp, L.pv, s);
      else
        c->coarse32.factor(L.rowptr, L.colidx, L.vv, L.vp, L.pv, s);
      continue;
    }
    // the finest level and the intermediate ones are inverted concurrently: separate flags
    // and scratch (the intermediate levels share theirs, in level order on the aux stream)
    int* flags = l == nl - 1 ? c->inv_flags : c->inv_flags2;
    void* scr = l == nl - 1 ? c->inv_scratch : c->inv_scratch2;
    const int fp = c->opt.factor_prec;
    // FP32/BF16 factors are computed in FP32 on the equilibrated J_K; FP64 factors in FP64
    const int cf32 = fp != STG_F64 ? 1 : 0;
    if (fp == STG_F64)
      invert_patches<double>(L.g, L.rowptr, L.vv, L.vp, L.pv, nullptr, nullptr, nullptr, (double*)L.jinv, 0, c->status,
                             scr, flags, s);
    else if (fp == STG_F32)
      invert_patches<float>(L.g, L.rowptr, L.vv, L.vp, L.pv, L.vv32, L.vp32, L.pv32, (float*)L.jinv, cf32, c->status,
                            scr, flags, s);
    else
      invert_patches<__nv_bfloat16>(L.g, L.rowptr, L.vv, L.vp, L.pv, L.vv32, L.vp32, L.pv32,
                                    (__nv_bfloat16*)L.jinv, cf32, c->status, scr, flags, s);
  }
  STG_CUDA_OK(cudaEventRecord(c->join, c->side));
  STG_CUDA_OK(cudaEventRecord(c->aux_done, c->aux));
  STG_CUDA_OK(cudaStreamWaitEvent(c->st, c->aux_done, 0));
  STG_CUDA_OK(cudaStreamWaitEvent(c->st, c->join, 0));
  int hs[4];
  STG_CUDA_OK(cudaMemcpyAsync(hs, c->status, sizeof(hs), cudaMemcpyDeviceToHost, c->st));
  STG_CUDA_OK(cudaStreamSynchronize(c->st));
  if (hs[0]) throw Error{STG_ESINGULAR, "singular local matrix J_K of cell " + std::to_string(hs[0] - 1)};
  const int cs = coarse64(c) ? c->coarse64.read_status(c->st) : c->coarse32.read_status(c->st);
  if (cs > 0) throw Error{STG_ESINGULAR, "singular block in the coarse solver (block " + std::to_string(cs - 1) + ")"};
  if (cs < 0) throw Error{STG_ECUDA, "coarse matrix coupling outside the slab block structure"};
}

void linearise(stg_ctx* c, const double* w_cabi) {
  LevelBufs& F = c->lv.back();
  w_to_internal(F.g, w_cabi, F.w, c->st);
  linearise_internal(c);
}

template <typename VT>
struct Ops;
template <>
struct Ops<double> {
  static const double* vv(const LevelBufs& L) { return L.vv; }
  static const double* vp(const LevelBufs& L) { return L.vp; }
  static const double* pv(const LevelBufs& L) { return L.pv; }
};
template <>
struct Ops<float> {
  static const float* vv(const LevelBufs& L) { return L.vv32; }
  static const float* vp(const LevelBufs& L) { return L.vp32; }
  static const float* pv(const LevelBufs& L) { return L.pv32; }
};

// Event record that also lands in a CUDA graph when the stream is being captured.
void record_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  STG_CUDA_OK(cudaStreamIsCapturing(st, &cap));
  if (cap == cudaStreamCaptureStatusActive)
    STG_CUDA_OK(cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
  else
    STG_CUDA_OK(cudaEventRecord(ev, st));
}

template <typename VT>
void residual(stg_ctx* c, const LevelBufs& L, const VT* x, const VT* b, VT* r) {
  if (std::is_same<VT, float>::value && L.mk32)
    apply_operator_kron(L.g, c->td, L.mk32, L.ak32, L.vp32, L.pv32, (const float*)x, (const float*)b,
                        (float*)r, c->st);
  else
    apply_operator<VT, VT>(L.g, L.rowptr, L.colidx, Ops<VT>::vv(L), Ops<VT>::vp(L), Ops<VT>::pv(L), x, b, r, c->st);
}

// J x (b null) or b - J x with the FP64 operator of level L.  The dense blocks stay: on GB300
// the FP64 rows are bound by FP64 throughput, and the dense block needs the fewest operations.
void apply64(stg_ctx* c, const LevelBufs& L, const double* x, const double* b, double* y) {
  apply_operator<double, double>(L.g, L.rowptr, L.colidx, L.vv, L.vp, L.pv, x, b, y, c->st);
}

template <typename VT, typename FT>
void smooth_level(stg_ctx* c, int l, int sweeps, bool x_zero) {
  LevelBufs& L = c->lv[l];
  const Geom& g = L.g;
  VT* b = (VT*)L.b;
  VT* x = (VT*)L.x;
  VT* r = (VT*)L.r;
  VT* z = (VT*)L.z;
  const FT* jinv = (const FT*)L.jinv;
  const int ncol = 1 << g.dim;
  for (int s = 0; s < sweeps; ++s) {
    // with profiling on, the colour launches of one sweep per V-cycle are bracketed by events
    // (the last post-smoothing sweep of the finest level; the last pre-smoothing sweep when
    // there is no post-smoothing): each event node is a graph node of its own, so a sample
    // keeps the timed cycle close to the uninstrumented one
    const bool prof_sweep = s == sweeps - 1 && (!x_zero || c->opt.nu2 == 0);
    if (c->opt.smoother == STG_VANKA_AVERAGED) {
      const VT* res = b;
      if (!(x_zero && s == 0)) {
        residual<VT>(c, L, x, b, r);
        res = r;
      }
      for (int col = 0; col < ncol; ++col) {
        const bool prof = prof_sweep && c->prof_on && l == (int)c->lv.size() - 1 &&
                          c->prof_used + 2 <= (int)c->prof_ev.size();
        if (prof) record_event(c->prof_ev[c->prof_used], c->st);
        vanka_colour<VT, FT>(g, col, jinv, res, z, (VT)1, c->st, L.colour_variant);
        if (prof) {
          record_event(c->prof_ev[c->prof_used + 1], c->st);
          c->prof_used += 2;
          c->prof_pending_patches += g.coff[col + 1] - g.coff[col];
        }
      }
      vanka_update<VT>(g, x, z, c->opt.omega, c->st);
    } else {
      for (int col = 0; col < ncol; ++col) {
        const VT* res = b;
        if (!(x_zero && s == 0 && col == 0)) {
          residual<VT>(c, L, x, b, r);
          res = r;
        }
        const bool prof = prof_sweep && c->prof_on && l == (int)c->lv.size() - 1 &&
                          c->prof_used + 2 <= (int)c->prof_ev.size();
        if (prof) record_event(c->prof_ev[c->prof_used], c->st);
        vanka_colour<VT, FT>(g, col, jinv, res, x, (VT)c->opt.omega, c->st, L.colour_variant);
        if (prof) {
          record_event(c->prof_ev[c->prof_used + 1], c->st);
          c->prof_used += 2;
          c->prof_pending_patches += g.coff[col + 1] - g.coff[col];
        }
      }
    }
  }
}

// x = J_0^{-1} b on FP64 vectors: the factors (FP64, or FP32 in the FP32 form) followed by
// coarse_refine steps of iterative refinement with the residual b - J_0 x computed in FP64
// (FP64 factors are refined only in the FP64 V-cycle).
void coarse_solve64(stg_ctx* c, const double* b, double* x) {
  const LevelBufs& L = c->lv[0];
  if (coarse64(c)) {
    c->coarse64.solve(b, x, c->st);
    // The FP64 V-cycle refines its FP64 solve as well: the block cyclic reduction applies
    // explicit block inverses, whose forward error grows with cond(block) (observed relative
    // residuals around 5e-14 against about 1e-16 for an LU solve); each step with the FP64
    // residual brings the solve back to LU accuracy.  FP64 factors under the FP32 V-cycle
    // are used as they are.
    if (vc64(c))
      for (int it = 0; it < c->opt.coarse_refine; ++it) {
        apply64(c, L, x, b, c->cr64);
        c->coarse64.solve(c->cr64, c->cd64, c->st);
        axpby(L.g.N, 1.0, c->cd64, 1.0, x, c->st);
      }
    return;
  }
  c->coarse32.solve(b, x, c->st);
  for (int it = 0; it < c->opt.coarse_refine; ++it) {
    apply64(c, L, x, b, c->cr64);
    c->coarse32.solve(c->cr64, c->cd64, c->st);
    axpby(L.g.N, 1.0, c->cd64, 1.0, x, c->st);
  }
}

template <typename VT>
void coarse_level(stg_ctx* c) {
  LevelBufs& L = c->lv[0];
  if (std::is_same<VT, double>::value) {
    coarse_solve64(c, (const double*)L.b, (double*)L.x);
  } else {
    convert(L.g.N, (const float*)L.b, c->cb64, c->st);
    coarse_solve64(c, c->cb64, c->cx64);
    convert(L.g.N, c->cx64, (float*)L.x, c->st);
  }
}

template <typename VT, typename FT>
void vcycle_level(stg_ctx* c, int l) {
  if (l == 0) {
    coarse_level<VT>(c);
    return;
  }
  LevelBufs& L = c->lv[l];
  LevelBufs& Lc = c->lv[l - 1];
  fill_zero<VT>(L.g.N, (VT*)L.x, c->st);
  smooth_level<VT, FT>(c, l, c->opt.nu1, true);
  residual<VT>(c, L, (const VT*)L.x, (const VT*)L.b, (VT*)L.r);
  restrict_res<VT>(Lc.g, L.g, (const VT*)L.r, (VT*)Lc.b, c->st);
  vcycle_level<VT, FT>(c, l - 1);
  prolongate_add<VT>(Lc.g, L.g, (const VT*)Lc.x, (VT*)L.x, c->st);
  smooth_level<VT, FT>(c, l, c->opt.nu2, false);
}

// V-cycle from c->vin (FP64 internal) to c->vout (FP64 internal)
void vcycle_body(stg_ctx* c) {
  const OverlapScope overlap(c->opt.overlap_launches != 0);
  LevelBufs& F = c->lv.back();
  const int top = (int)c->lv.size() - 1;
  if (vc64(c)) {
    STG_CUDA_OK(cudaMemcpyAsync(F.b, c->vin, sizeof(double) * F.g.N, cudaMemcpyDeviceToDevice, c->st));
    vcycle_level<double, double>(c, top);
    STG_CUDA_OK(cudaMemcpyAsync(c->vout, F.x, sizeof(double) * F.g.N, cudaMemcpyDeviceToDevice, c->st));
  } else {
    convert(F.g.N, c->vin, (float*)F.b, c->st);
    if (c->opt.factor_prec == STG_F32)
      vcycle_level<float, float>(c, top);
    else
      vcycle_level<float, __nv_bfloat16>(c, top);
    convert(F.g.N, (const float*)F.x, c->vout, c->st);
  }
}

// One V-cycle; with profiling on, the events of the colour kernels are read
// back after the cycle (the caller synchronises before the next one).
void run_vcycle(stg_ctx* c) {
  if (c->opt.use_graph) {
    if (!c->graph) {
      cudaGraph_t graph = nullptr;
      const long long before = launch_counter();
      const int used0 = c->prof_used;
      const long long pend0 = c->prof_pending_patches;
      STG_CUDA_OK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
      try {
        vcycle_body(c);
      } catch (...) {
        cudaStreamEndCapture(c->st, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      STG_CUDA_OK(cudaStreamEndCapture(c->st, &graph));
      c->graph_kernels = launch_counter() - before;
      launch_counter() = before;  // capturing enqueues nothing; replays are counted below
      c->graph_prof_events = c->prof_used - used0;
      c->graph_prof_patches = c->prof_pending_patches - pend0;
      c->prof_used = used0;
      c->prof_pending_patches = pend0;
      const cudaError_t e = cudaGraphInstantiate(&c->graph, graph, 0);
      cudaGraphDestroy(graph);
      STG_CUDA_OK(e);
    }
    STG_CUDA_OK(cudaGraphLaunch(c->graph, c->st));
    launch_counter() += c->graph_kernels;
    c->prof_used += c->graph_prof_events;
    c->prof_pending_patches += c->graph_prof_patches;
  } else {
    vcycle_body(c);
  }
}

// Accumulate the recorded colour-kernel times (call after the stream has drained).
void prof_collect(stg_ctx* c) {
  if (!c->prof_on || c->prof_used == 0) return;
  for (int i = 0; i + 1 < c->prof_used; i += 2) {
    float ms = 0.f;
    STG_CUDA_OK(cudaEventElapsedTime(&ms, c->prof_ev[i], c->prof_ev[i + 1]));
    c->prof_ms += ms;
    ++c->prof_launches;
  }
  c->prof_patches += c->prof_pending_patches;
  c->prof_pending_patches = 0;
  c->prof_used = 0;
}

template <typename VT>
void level_to_internal(stg_ctx* c, int l, const double* in, VT* out) {
  cabi_to_internal<VT>(c->lv[l].g, in, out, c->st);
}

void apply_fine64(stg_ctx* c, const double* x, double* y) { apply64(c, c->lv.back(), x, nullptr, y); }

double dot_host(stg_ctx* c, const double* a, const double* b) {
  const long long n = c->lv.back().g.N;
  multi_dot(n, 1, a, n, b, c->partial, c->hd, c->st);
  STG_CUDA_OK(cudaMemcpyAsync(c->hh, c->hd, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  STG_CUDA_OK(cudaStreamSynchronize(c->st));
  return c->hh[0];
}

// Flexible GMRES(m), right preconditioned by one V-cycle (Sec. 3), as a state machine so
// that one problem or a batch of problems (stepped in lock step) share the code.
struct FgState {
  stg_ctx* c = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  long long n = 0;
  int m = 0, its = 0, j = 0, jend = 0;
  double bnorm = 0.0, tol = 0.0, beta = 0.0;
  bool active = false, done = false;
  std::vector<double> H, cs, sn, gv, y;
  double& Hc(int i, int jj) { return H[(size_t)i * m + jj]; }
};

void fg_begin(FgState& S, stg_ctx* c, const double* b, double* x) {
  S.c = c;
  S.b = b;
  S.x = x;
  S.n = c->lv.back().g.N;
  S.m = c->opt.gmres_restart;
  S.H.assign((size_t)(S.m + 1) * S.m, 0.0);
  S.cs.assign(S.m, 0.0);
  S.sn.assign(S.m, 0.0);
  S.gv.assign(S.m + 1, 0.0);
  S.y.assign(S.m, 0.0);
  S.bnorm = std::sqrt(dot_host(c, b, b));
  if (!std::isfinite(S.bnorm)) throw Error{STG_EINVAL, "right-hand side contains NaN or Inf"};
  S.tol = std::max(c->opt.gmres_rtol * S.bnorm, c->opt.gmres_atol);
  S.its = 0;
  S.active = false;
  S.done = false;
}

// r = b - J x; stop or open a new restart cycle (synchronises the context's stream)
void fg_restart(FgState& S) {
  stg_ctx* c = S.c;
  apply_fine64(c, S.x, c->rv);
  axpby(S.n, 1.0, S.b, -1.0, c->rv, c->st);
  S.beta = std::sqrt(dot_host(c, c->rv, c->rv));
  if (S.beta <= S.tol || S.its >= c->opt.gmres_maxit || S.bnorm == 0.0) {
    S.done = true;
    return;
  }
  axpby(S.n, 1.0 / S.beta, c->rv, 0.0, c->V, c->st);
  std::fill(S.gv.begin(), S.gv.end(), 0.0);
  S.gv[0] = S.beta;
  S.j = 0;
  S.active = true;
}

// V-cycle input v_j
void fg_pre(FgState& S) {
  stg_ctx* c = S.c;
  STG_CUDA_OK(cudaMemcpyAsync(c->vin, c->V + (long long)S.j * S.n, sizeof(double) * S.n, cudaMemcpyDeviceToDevice,
                              c->st));
}

// z_j = V(v_j), w = J z_j, classical Gram-Schmidt twice, ||w||; the coefficients go to the host
void fg_post(FgState& S) {
  stg_ctx* c = S.c;
  const long long n = S.n;
  const int j = S.j;
  double* zj = c->Z + (long long)j * n;
  STG_CUDA_OK(cudaMemcpyAsync(zj, c->vout, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
  apply_fine64(c, zj, c->wv);
  multi_dot(n, j + 1, c->V, n, c->wv, c->partial, c->hd, c->st);
  multi_axpy_sub(n, j + 1, c->V, n, c->hd, c->wv, c->st);
  multi_dot(n, j + 1, c->V, n, c->wv, c->partial, c->hd + 32, c->st);
  multi_axpy_sub(n, j + 1, c->V, n, c->hd + 32, c->wv, c->st);
  multi_dot(n, 1, c->wv, n, c->wv, c->partial, c->hd + 64, c->st);
  STG_CUDA_OK(cudaMemcpyAsync(c->hh, c->hd, sizeof(double) * 65, cudaMemcpyDeviceToHost, c->st));
}

// after the stream has drained: Arnoldi column, Givens rotations, and at the end of a
// cycle the update x += Z y
void fg_update(FgState& S) {
  stg_ctx* c = S.c;
  const long long n = S.n;
  const int j = S.j;
  for (int i = 0; i <= j; ++i) S.Hc(i, j) = c->hh[i] + c->hh[32 + i];
  const double hn = std::sqrt(std::max(c->hh[64], 0.0));
  S.Hc(j + 1, j) = hn;
  if (hn > 0.0) axpby(n, 1.0 / hn, c->wv, 0.0, c->V + (long long)(j + 1) * n, c->st);
  for (int i = 0; i < j; ++i) {
    const double t = S.cs[i] * S.Hc(i, j) + S.sn[i] * S.Hc(i + 1, j);
    S.Hc(i + 1, j) = -S.sn[i] * S.Hc(i, j) + S.cs[i] * S.Hc(i + 1, j);
    S.Hc(i, j) = t;
  }
  const double rho = std::hypot(S.Hc(j, j), S.Hc(j + 1, j));
  S.cs[j] = rho > 0 ? S.Hc(j, j) / rho : 1.0;
  S.sn[j] = rho > 0 ? S.Hc(j + 1, j) / rho : 0.0;
  S.Hc(j, j) = rho;
  S.Hc(j + 1, j) = 0.0;
  S.gv[j + 1] = -S.sn[j] * S.gv[j];
  S.gv[j] = S.cs[j] * S.gv[j];
  ++S.its;
  S.jend = j + 1;
  S.j = j + 1;
  const bool end = std::fabs(S.gv[j + 1]) <= S.tol || S.its >= c->opt.gmres_maxit || rho == 0.0 || hn == 0.0 ||
                   S.j == S.m;
  if (!end) return;
  const int je = S.jend;
  for (int i = je - 1; i >= 0; --i) {
    double sum = S.gv[i];
    for (int l = i + 1; l < je; ++l) sum -= S.Hc(i, l) * S.y[l];
    S.y[i] = S.Hc(i, i) != 0.0 ? sum / S.Hc(i, i) : 0.0;
  }
  STG_CUDA_OK(cudaMemcpyAsync(c->hd + 96, S.y.data(), sizeof(double) * je, cudaMemcpyHostToDevice, c->st));
  multi_axpy_add(n, je, c->Z, n, c->hd + 96, S.x, c->st);
  S.active = false;
}

stg_status fg_result(const FgState& S, int* iters_out, double* rel_out) {
  if (iters_out) *iters_out = S.its;
  if (rel_out) *rel_out = S.bnorm > 0 ? S.beta / S.bnorm : 0.0;
  return S.beta <= S.tol || S.bnorm == 0.0 ? STG_OK : STG_ENOCONV;
}

const char* const kColourTimeout = "a staged smoother kernel gave up waiting for a bulk copy";

stg_status fgmres(stg_ctx* c, const double* b, double* x, int* iters_out, double* rel_out) {
  FgState S;
  fg_begin(S, c, b, x);
  for (;;) {
    if (!S.active) {
      fg_restart(S);
      if (S.done) break;
    }
    fg_pre(S);
    run_vcycle(c);
    fg_post(S);
    STG_CUDA_OK(cudaStreamSynchronize(c->st));
    prof_collect(c);
    fg_update(S);
  }
  if (colour_kernel_timed_out(c->st)) throw Error{STG_ETIMEOUT, kColourTimeout};
  return fg_result(S, iters_out, rel_out);
}

// r = b - F... precisely r = -F_n(X) = b - J_Oseen(w = v(X)) X on the finest level (the finest
// operator storage is overwritten by the Oseen Jacobian at v(X)).
double neg_residual(stg_ctx* c, const double* X, double* r) {
  LevelBufs& F = c->lv.back();
  AsmCoef cf{c->nu, c->tau, c->opt.gamma1, c->opt.gamma2, 0};
  // the velocity part of an internal vector is laid out exactly like an internal w
  assemble_level_w(F.g, c->td, cf, X, F.rowptr, F.asm_tab, F.vconst, F.vv, F.nnzb, c->st);
  apply_operator<double, double>(F.g, F.rowptr, F.colidx, F.vv, F.vp, F.pv, X, c->nb, r, c->st);
  return std::sqrt(dot_host(c, r, r));
}

// Damped Newton for F_n(X) = 0 (Sec. 3) on internal vectors; X in/out.
stg_status newton(stg_ctx* c, double* X, double rtol, double atol, int maxit, int* steps_out, int* gmres_out,
                  double* res_out) {
  LevelBufs& F = c->lv.back();
  const long long n = F.g.N;
  double nr = neg_residual(c, X, c->nr);
  if (!std::isfinite(nr)) throw Error{STG_EINVAL, "slab residual is NaN or Inf (check X, f, g and v_prev)"};
  const double tol = std::max(rtol * nr, atol);
  int steps = 0, gits = 0;
  stg_status st = STG_OK;
  while (nr > tol && steps < maxit) {
    STG_CUDA_OK(cudaMemcpyAsync(F.w, X, sizeof(double) * F.g.nvel, cudaMemcpyDeviceToDevice, c->st));
    linearise_internal(c);  // Newton Jacobian at v(X) on every level, local inverses, coarse factors
    STG_CUDA_OK(cudaMemsetAsync(c->nC, 0, sizeof(double) * n, c->st));
    int its = 0;
    double rel = 0.0;
    const stg_status ls = fgmres(c, c->nr, c->nC, &its, &rel);  // J C = -F
    gits += its;
    if (ls == STG_ENOCONV) st = STG_ENOCONV;
    double lam = 1.0, nt = 0.0;
    for (;;) {
      axpby(n, 1.0, X, 0.0, c->nXt, c->st);
      axpby(n, lam, c->nC, 1.0, c->nXt, c->st);
      nt = neg_residual(c, c->nXt, c->nr);
      if (nt < (1.0 - 1e-4 * lam) * nr || lam <= 1.0 / 16.0) break;
      lam *= 0.5;
    }
    STG_CUDA_OK(cudaMemcpyAsync(X, c->nXt, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
    nr = nt;
    ++steps;
  }
  if (steps_out) *steps_out = steps;
  if (gmres_out) *gmres_out = gits;
  if (res_out) *res_out = nr;
  if (nr > tol) return STG_ENOCONV;
  return st;
}

// Times every colour-kernel variant on one level (all colours of one sweep, `reps` times)
// and keeps the fastest; returns its time per sweep in ms.
template <typename VT, typename FT>
double tune_level(stg_ctx* c, int l, int reps) {
  LevelBufs& L = c->lv[l];
  cudaEvent_t e0, e1;
  STG_CUDA_OK(cudaEventCreate(&e0));
  STG_CUDA_OK(cudaEventCreate(&e1));
  double best = 1e30;
  int bestv = L.colour_variant;
  for (int v = 0; v < kColourVariants; ++v) {
    for (int w = 0; w < 2; ++w)  // warm-up
      for (int col = 0; col < (1 << L.g.dim); ++col)
        vanka_colour<VT, FT>(L.g, col, (const FT*)L.jinv, (const VT*)L.r, (VT*)L.z, (VT)1, c->st, v);
    STG_CUDA_OK(cudaEventRecord(e0, c->st));
    for (int rep = 0; rep < reps; ++rep)
      for (int col = 0; col < (1 << L.g.dim); ++col)
        vanka_colour<VT, FT>(L.g, col, (const FT*)L.jinv, (const VT*)L.r, (VT*)L.z, (VT)1, c->st, v);
    STG_CUDA_OK(cudaEventRecord(e1, c->st));
    STG_CUDA_OK(cudaEventSynchronize(e1));
    float ms = 0.f;
    STG_CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms / reps < best) {
      best = ms / reps;
      bestv = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  L.colour_variant = bestv;
  STG_CUDA_OK(cudaMemsetAsync(L.z, 0, (vc64(c) ? 8 : 4) * L.g.N, c->st));  // the smoother expects z = 0
  return best;
}

stg_status fail(stg_ctx* c, const Error& e) {
  if (c)
    c->err = e.msg;
  else
    g_setup_error = e.msg;
  return e.st;
}

stg_status validate(const stg_mesh* m, int k, const stg_options* o) {
  if (!m || !o) throw Error{STG_EINVAL, "null mesh or options"};
  if (m->dim != 2 && m->dim != 3) throw Error{STG_EINVAL, "dim must be 2 or 3"};
  if (m->n_levels < 1 || m->n_levels > 12) throw Error{STG_EINVAL, "n_levels must be in 1..12"};
  if (k < 0 || k > (m->dim == 2 ? 4 : 2)) throw Error{STG_EINVAL, "k out of range (2D: 0..4, 3D: 0..2)"};
  const int f = 1 << (m->n_levels - 1);
  const int n[3] = {m->nx, m->ny, m->dim == 3 ? m->nz : f};
  for (int e = 0; e < m->dim; ++e)
    if (n[e] < f || n[e] % f) throw Error{STG_EINVAL, "cells per direction must be a positive multiple of 2^(n_levels-1)"};
  const double lo[3] = {m->x0, m->y0, m->z0}, hi[3] = {m->x1, m->y1, m->z1};
  for (int e = 0; e < m->dim; ++e)
    if (!(hi[e] > lo[e])) throw Error{STG_EINVAL, "empty domain"};
  if (m->order != 0 && m->order != 2 && m->order != 4) throw Error{STG_EINVAL, "order must be 2 or 4"};
  if (m->order == 4 && m->dim != 2) throw Error{STG_EINVAL, "order 4 is supported in 2D only"};
  if (m->order == 4 && k > 2) throw Error{STG_EINVAL, "order 4 supports k = 0..2"};
  const int* ob = m->obstacle;
  if (ob[0] || ob[1] || ob[2] || ob[3]) {
    const int nc0[2] = {m->nx / f, m->ny / f};
    if (m->order == 4) throw Error{STG_EINVAL, "an obstacle is supported with order 2 only"};
    if (m->dim != 2) throw Error{STG_EINVAL, "an obstacle is supported in 2D only"};
    if (!(0 <= ob[0] && ob[0] < ob[1] && ob[1] <= nc0[0] && 0 <= ob[2] && ob[2] < ob[3] && ob[3] <= nc0[1]))
      throw Error{STG_EINVAL, "obstacle box outside the coarsest level's cells or empty"};
    if (ob[1] - ob[0] == nc0[0] || ob[3] - ob[2] == nc0[1])
      throw Error{STG_EINVAL, "an obstacle may not cut the domain in two"};
  }
  if (o->vcycle_prec == STG_F64 && o->factor_prec != STG_F64)
    throw Error{STG_EINVAL, "an FP64 V-cycle needs FP64 local inverses"};
  if (o->vcycle_prec == STG_F32 && o->factor_prec == STG_F64)
    throw Error{STG_EINVAL, "an FP32 V-cycle takes FP32 or BF16 local inverses"};
  if (o->vcycle_prec != STG_F64 && o->vcycle_prec != STG_F32) throw Error{STG_EINVAL, "bad vcycle_prec"};
  if (o->nu1 < 0 || o->nu2 < 0) throw Error{STG_EINVAL, "negative smoothing steps"};
  if (o->gmres_restart < 1 || o->gmres_restart > 30) throw Error{STG_EINVAL, "gmres_restart must be in 1..30"};
  if (o->smoother != STG_VANKA_AVERAGED && o->smoother != STG_VANKA_COLOURED) throw Error{STG_EINVAL, "bad smoother"};
  if (o->coarse_refine < 0 || o->coarse_refine > 20) throw Error{STG_EINVAL, "coarse_refine must be in 0..20"};
  if (o->coarse_prec != STG_F64 && o->coarse_prec != STG_F32)
    throw Error{STG_EINVAL, "coarse_prec must be STG_F64 or STG_F32"};
  if (o->overlap_launches != 0 && o->overlap_launches != 1) throw Error{STG_EINVAL, "overlap_launches must be 0 or 1"};
  return STG_OK;
}

}  // namespace

namespace stg {
// Error text for entry points without a context (read through stg_last_error(NULL)).
void set_global_error(const std::string& msg) { g_setup_error = msg; }
}  // namespace stg

// ------------------------------------------------------------------ C ABI
extern "C" {

stg_status stg_options_default(stg_options* o) {
  if (!o) return STG_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->linearisation = STG_NEWTON;
  o->smoother = STG_VANKA_AVERAGED;
  o->nu1 = 4;
  o->nu2 = 4;
  o->omega = 0.7;
  o->gamma1 = 35.0;
  o->gamma2 = 35.0;
  o->factor_prec = STG_F64;
  o->vcycle_prec = STG_F64;
  o->gmres_restart = 30;
  o->gmres_maxit = 200;
  o->gmres_rtol = 1e-8;
  o->gmres_atol = 0.0;
  o->use_graph = 1;
  o->coarse_refine = 1;
  o->coarse_prec = STG_F32;
  o->overlap_launches = 1;
  return STG_OK;
}

stg_status stg_setup(const stg_mesh* mesh, int k, double nu, double tau, const double* w, const stg_options* opt,
                     void* stream, stg_ctx** out) {
  if (!out) return STG_EINVAL;
  *out = nullptr;
  stg_ctx* c = nullptr;
  try {
    validate(mesh, k, opt);
    if (!w) throw Error{STG_EINVAL, "null linearisation velocity"};
    c = new (std::nothrow) stg_ctx();
    if (!c) throw Error{STG_ENOMEM, "host allocation failed"};
    c->mesh = *mesh;
    c->opt = *opt;
    c->k = k;
    c->nu = nu;
    c->tau = tau;
    c->st = (cudaStream_t)stream;
    // highest priority: the coarse factorisation and the intermediate levels are chains of
    // smaller launches whose CTAs should not queue behind the finest level's large grids
    int prio_lo = 0, prio_hi = 0;
    STG_CUDA_OK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    STG_CUDA_OK(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi));
    STG_CUDA_OK(cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, prio_hi));
    STG_CUDA_OK(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    STG_CUDA_OK(cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming));
    STG_CUDA_OK(cudaEventCreateWithFlags(&c->aux_done, cudaEventDisableTiming));
    c->td = time_basis(k);
    c->pure_dirichlet = mesh->dirichlet_faces == (1u << (2 * mesh->dim)) - 1u;
    upload_fe_tables();
    upload_transfer4_tables();
    const int nl = mesh->n_levels;
    c->lv.resize(nl);
    size_t scratch = 0, scratch2 = 0;
    const bool f64 = vc64(c);
    const size_t vts = f64 ? 8 : 4;
    for (int l = 0; l < nl; ++l) {
      LevelBufs& L = c->lv[l];
      L.g = make_geom(*mesh, l, k);
      const Geom& g = L.g;
      build_pattern(c, L);
      L.vv = dalloc<double>(c, L.nnzb * g.NV * g.NV);
      const long long nvp = g.n_cells * g.nloc * g.nt * g.dim * g.npd;
      L.vp = dalloc<double>(c, nvp);
      L.pv = dalloc<double>(c, nvp);
      if (!f64) {
        L.vp32 = dalloc<float>(c, nvp);
        L.pv32 = dalloc<float>(c, nvp);
        if (l > 0 && kron_supported(g)) {
          // the FP32 residual takes the Kronecker form, and the patch inversion rounds the
          // FP64 blocks as it gathers them: no FP32 copy of the dense blocks
          L.mk32 = dalloc<float>(c, L.nnzb);
          L.ak32 = dalloc<float>(c, L.nnzb * g.nt * g.dim * g.dim);
        } else {
          L.vv32 = dalloc<float>(c, L.nnzb * g.NV * g.NV);
        }
      }
      L.w = dalloc<double>(c, g.nvel);
      L.asm_tab = dalloc<double>(c, assemble_table_doubles(g.dim, k));
      L.vconst = dalloc<double>(c, L.nnzb * g.NV * g.NV);
      L.b = dalloc<char>(c, (long long)vts * g.N);
      L.x = dalloc<char>(c, (long long)vts * g.N);
      L.r = dalloc<char>(c, (long long)vts * g.N);
      L.z = dalloc<char>(c, (long long)vts * g.N);
      STG_CUDA_OK(cudaMemset(L.z, 0, vts * g.N));
      STG_CUDA_OK(cudaMemset(L.x, 0, vts * g.N));
      if (l > 0) {
        L.jinv = dalloc<char>(c, (long long)fsize(opt->factor_prec) * patch_stride(g.npatch) * g.n_cells);
        const int cf32 = opt->factor_prec != STG_F64 ? 1 : 0;
        if (l == mesh->n_levels - 1)
          scratch = invert_scratch_bytes(g, cf32);
        else
          scratch2 = std::max(scratch2, invert_scratch_bytes(g, cf32));
      }
    }
    if (scratch) c->inv_scratch = dalloc<char>(c, (long long)scratch);
    if (scratch2) c->inv_scratch2 = dalloc<char>(c, (long long)scratch2);
    c->inv_flags = dalloc<int>(c, c->lv.back().g.n_cells);
    if (mesh->n_levels > 2) c->inv_flags2 = dalloc<int>(c, c->lv[mesh->n_levels - 2].g.n_cells);
    if (f64 || opt->coarse_prec == STG_F64)
      c->coarse64.init(c->lv[0].g, c->pure_dirichlet);
    else
      c->coarse32.init(c->lv[0].g, c->pure_dirichlet);
    c->cb64 = dalloc<double>(c, c->lv[0].g.N);
    c->cx64 = dalloc<double>(c, c->lv[0].g.N);
    c->cr64 = dalloc<double>(c, c->lv[0].g.N);
    c->cd64 = dalloc<double>(c, c->lv[0].g.N);
    c->status = dalloc<int>(c, 4);
    const long long n = c->lv.back().g.N;
    const int m = opt->gmres_restart;
    c->V = dalloc<double>(c, (long long)(m + 1) * n);
    c->Z = dalloc<double>(c, (long long)m * n);
    c->wv = dalloc<double>(c, n);
    c->rv = dalloc<double>(c, n);
    c->vin = dalloc<double>(c, n);
    c->vout = dalloc<double>(c, n);
    c->tmp_a = dalloc<double>(c, n);
    c->tmp_b = dalloc<double>(c, n);
    c->partial = dalloc<double>(c, (long long)dot_partial_doubles());
    c->nb = dalloc<double>(c, n);
    c->nX = dalloc<double>(c, n);
    c->nr = dalloc<double>(c, n);
    c->nC = dalloc<double>(c, n);
    c->nXt = dalloc<double>(c, n);
    c->nf = dalloc<double>(c, c->lv.back().g.nvel);
    c->ng = dalloc<double>(c, c->lv.back().g.nvel);
    c->rhs_tab = dalloc<double>(c, rhs_table_doubles(mesh->dim));
    c->hd = dalloc<double>(c, 160);
    STG_CUDA_OK(cudaMallocHost(&c->hh, sizeof(double) * 160));
    // the part of every level's operator that does not depend on w: assembled once, together
    // with the element tables and the velocity-pressure blocks
    {
      const AsmCoef cf0{nu, tau, c->opt.gamma1, c->opt.gamma2, 0};
      for (LevelBufs& L : c->lv) {
        assemble_level(L.g, c->td, cf0, nullptr, L.rowptr, L.asm_tab, L.vv, L.nnzb, L.vp, L.pv, c->st);
        STG_CUDA_OK(cudaMemcpyAsync(L.vconst, L.vv, sizeof(double) * L.nnzb * L.g.NV * L.g.NV,
                                    cudaMemcpyDeviceToDevice, c->st));
      }
    }
    linearise(c, w);
    *out = c;
    return STG_OK;
  } catch (const Error& e) {
    g_setup_error = e.msg;
    if (c) stg_destroy(c);
    return e.st;
  } catch (const std::bad_alloc&) {
    g_setup_error = "host allocation failed";
    if (c) stg_destroy(c);
    return STG_ENOMEM;
  }
}

stg_status stg_update_linearisation(stg_ctx* c, const double* w) {
  if (!c || !w) return STG_EINVAL;
  try {
    linearise(c, w);
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_obstacle_forces(stg_ctx* c, const double* X, double* forces) {
  if (!c || !X || !forces) return STG_EINVAL;
  try {
    const Geom& g = c->lv.back().g;
    if (!has_obstacle(g)) throw Error{STG_EINVAL, "the mesh has no obstacle"};
    cabi_to_internal<double>(g, X, c->tmp_a, c->st);
    obstacle_forces(g, c->nu, c->tmp_a, c->hd, c->st);
    STG_CUDA_OK(cudaMemcpyAsync(c->hh, c->hd, sizeof(double) * 2 * g.nt, cudaMemcpyDeviceToHost, c->st));
    STG_CUDA_OK(cudaStreamSynchronize(c->st));
    for (int i = 0; i < 2 * g.nt; ++i) forces[i] = c->hh[i];
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_set_slab_length(stg_ctx* c, double tau) {
  if (!c) return STG_EINVAL;
  if (!(tau >= 0.0) || !std::isfinite(tau)) {
    c->err = "slab length must be finite and >= 0";
    return STG_EINVAL;
  }
  try {
    // tau scales every spatial term of D_ab and the velocity-pressure blocks: the
    // w-independent part of every level is assembled again, then the levels are
    // re-linearised at the current w (the last one set or left by the Newton iteration)
    c->tau = tau;
    const AsmCoef cf0{c->nu, tau, c->opt.gamma1, c->opt.gamma2, 0};
    for (LevelBufs& L : c->lv) {
      assemble_level(L.g, c->td, cf0, nullptr, L.rowptr, L.asm_tab, L.vv, L.nnzb, L.vp, L.pv, c->st);
      STG_CUDA_OK(cudaMemcpyAsync(L.vconst, L.vv, sizeof(double) * L.nnzb * L.g.NV * L.g.NV,
                                  cudaMemcpyDeviceToDevice, c->st));
    }
    linearise_internal(c);
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_apply_level_jacobian(stg_ctx* c, int level, const double* x, double* y) {
  if (!c || !x || !y || level < 0 || level >= (int)c->lv.size()) return STG_EINVAL;
  try {
    const LevelBufs& L = c->lv[level];
    cabi_to_internal<double>(L.g, x, c->tmp_a, c->st);
    apply64(c, L, c->tmp_a, nullptr, c->tmp_b);
    internal_to_cabi<double>(L.g, c->tmp_b, y, c->st);
    STG_CUDA_OK(cudaGetLastError());
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_apply_jacobian(stg_ctx* c, const double* x, double* y) {
  if (!c) return STG_EINVAL;
  return stg_apply_level_jacobian(c, (int)c->lv.size() - 1, x, y);
}

stg_status stg_vcycle(stg_ctx* c, const double* b, double* x) {
  if (!c || !b || !x) return STG_EINVAL;
  try {
    const Geom& g = c->lv.back().g;
    cabi_to_internal<double>(g, b, c->vin, c->st);
    run_vcycle(c);
    internal_to_cabi<double>(g, c->vout, x, c->st);
    if (c->prof_on) {
      STG_CUDA_OK(cudaStreamSynchronize(c->st));
      prof_collect(c);
    }
    if (colour_kernel_timed_out(c->st)) throw Error{STG_ETIMEOUT, kColourTimeout};
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_smooth(stg_ctx* c, int level, int sweeps, const double* b, double* x) {
  if (!c || !b || !x || level < 1 || level >= (int)c->lv.size() || sweeps < 0) return STG_EINVAL;
  try {
    LevelBufs& L = c->lv[level];
    if (vc64(c)) {
      cabi_to_internal<double>(L.g, b, (double*)L.b, c->st);
      cabi_to_internal<double>(L.g, x, (double*)L.x, c->st);
      smooth_level<double, double>(c, level, sweeps, false);
      internal_to_cabi<double>(L.g, (const double*)L.x, x, c->st);
    } else {
      cabi_to_internal<float>(L.g, b, (float*)L.b, c->st);
      cabi_to_internal<float>(L.g, x, (float*)L.x, c->st);
      if (c->opt.factor_prec == STG_F32)
        smooth_level<float, float>(c, level, sweeps, false);
      else
        smooth_level<float, __nv_bfloat16>(c, level, sweeps, false);
      internal_to_cabi<float>(L.g, (const float*)L.x, x, c->st);
    }
    if (colour_kernel_timed_out(c->st)) throw Error{STG_ETIMEOUT, kColourTimeout};
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_prolongate(stg_ctx* c, int level, const double* xc, double* xf) {
  if (!c || !xc || !xf || level < 1 || level >= (int)c->lv.size()) return STG_EINVAL;
  try {
    const Geom& gc = c->lv[level - 1].g;
    const Geom& gf = c->lv[level].g;
    cabi_to_internal<double>(gc, xc, c->tmp_a, c->st);
    cabi_to_internal<double>(gf, xf, c->tmp_b, c->st);
    prolongate_add<double>(gc, gf, c->tmp_a, c->tmp_b, c->st);
    internal_to_cabi<double>(gf, c->tmp_b, xf, c->st);
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_restrict(stg_ctx* c, int level, const double* rf, double* bc) {
  if (!c || !rf || !bc || level < 1 || level >= (int)c->lv.size()) return STG_EINVAL;
  try {
    const Geom& gc = c->lv[level - 1].g;
    const Geom& gf = c->lv[level].g;
    cabi_to_internal<double>(gf, rf, c->tmp_a, c->st);
    restrict_res<double>(gc, gf, c->tmp_a, c->tmp_b, c->st);
    internal_to_cabi<double>(gc, c->tmp_b, bc, c->st);
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_coarse_solve(stg_ctx* c, const double* b, double* x) {
  if (!c || !b || !x) return STG_EINVAL;
  try {
    const Geom& g = c->lv[0].g;
    cabi_to_internal<double>(g, b, c->tmp_a, c->st);
    coarse_solve64(c, c->tmp_a, c->tmp_b);
    internal_to_cabi<double>(g, c->tmp_b, x, c->st);
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_gmres_solve(stg_ctx* c, const double* b, double* x, int* iters, double* rel_res) {
  if (!c || !b || !x) return STG_EINVAL;
  try {
    const Geom& g = c->lv.back().g;
    cabi_to_internal<double>(g, b, c->tmp_a, c->st);
    cabi_to_internal<double>(g, x, c->tmp_b, c->st);
    const stg_status s = fgmres(c, c->tmp_a, c->tmp_b, iters, rel_res);
    internal_to_cabi<double>(g, c->tmp_b, x, c->st);
    STG_CUDA_OK(cudaStreamSynchronize(c->st));
    if (s == STG_ENOCONV) c->err = "FGMRES reached gmres_maxit";
    return s;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_newton_slab(stg_ctx* c, const double* v_prev, const double* f, const double* g, double* X,
                           double rtol, double atol, int maxit, int* newton_steps, int* gmres_iters,
                           double* residual) {
  if (!c || !X || maxit < 0 || rtol < 0 || atol < 0) return STG_EINVAL;
  if (c->lv.back().g.r != 2) {
    c->err = "stg_newton_slab needs order 2";
    return STG_EINVAL;
  }
  try {
    LevelBufs& F = c->lv.back();
    const Geom& gg = F.g;
    if (f) w_to_internal(gg, f, c->nf, c->st);
    if (g) w_to_internal(gg, g, c->ng, c->st);
    // assemble_level fills the mass matrix of the level's table used by the right-hand side
    AsmCoef cf{c->nu, c->tau, c->opt.gamma1, c->opt.gamma2, 0};
    assemble_rhs_level(gg, c->td, cf, F.asm_tab, c->rhs_tab, f ? c->nf : nullptr, g ? c->ng : nullptr, v_prev,
                       c->nb, c->st);
    cabi_to_internal<double>(gg, X, c->nX, c->st);
    const stg_status s = newton(c, c->nX, rtol, atol, maxit, newton_steps, gmres_iters, residual);
    internal_to_cabi<double>(gg, c->nX, X, c->st);
    STG_CUDA_OK(cudaStreamSynchronize(c->st));
    if (s == STG_ENOCONV) c->err = "Newton or FGMRES reached its iteration limit";
    return s;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_slab_initial_guess(stg_ctx* c, const double* X_prev, double* X0) {
  if (!c || !X_prev || !X0) return STG_EINVAL;
  try {
    replicate_end_value(c->lv.back().g, X_prev, X0, c->st);
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

namespace {

// The warm-start calls work on a 2D finest level; the network must map 2d input channels
// to d(k+1) output channels on the H x W node grid.
stg_status warm_check(stg_ctx* c, const stg_cnn* net) {
  const Geom& g = c->lv.back().g;
  if (g.dim != 2) {
    c->err = "warm start: the network works on 2D node grids";
    return STG_EINVAL;
  }
  if (net && (net->ch[0] != 2 * g.dim || net->ch[net->L] != g.dim * g.nt || net->H != g.nn[1] ||
              net->W != g.nn[0])) {
    c->err = "warm start: network channels or grid do not match the slab problem";
    return STG_EINVAL;
  }
  return STG_OK;
}

}  // namespace

stg_status stg_warm_features(stg_ctx* c, const double* X_n, const double* X_prev, float scale_v, float scale_d,
                             float* feat) {
  if (c && c->lv.back().g.r != 2) {
    c->err = "stg_warm_features needs order 2";
    return STG_EINVAL;
  }
  if (!c || !X_n || !X_prev || !feat || !(scale_v > 0.f) || !(scale_d > 0.f)) return STG_EINVAL;
  const stg_status s = warm_check(c, nullptr);
  if (s != STG_OK) return s;
  try {
    warm_features(c->lv.back().g, X_n, X_prev, scale_v, scale_d, feat, c->st);
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_warm_target(stg_ctx* c, const double* X_n, const double* X_prev, const double* X_next, float scale_d,
                           float* target) {
  if (c && c->lv.back().g.r != 2) {
    c->err = "stg_warm_target needs order 2";
    return STG_EINVAL;
  }
  if (!c || !X_n || !X_prev || !X_next || !target || !(scale_d > 0.f)) return STG_EINVAL;
  const stg_status s = warm_check(c, nullptr);
  if (s != STG_OK) return s;
  try {
    warm_target(c->lv.back().g, c->td, X_n, X_prev, X_next, scale_d, target, c->st);
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_warm_start(stg_ctx* c, stg_cnn* net, const double* X_n, const double* X_prev, float scale_v,
                          float scale_d, double* X0) {
  if (c && c->lv.back().g.r != 2) {
    c->err = "stg_warm_start needs order 2";
    return STG_EINVAL;
  }
  if (!c || !X_n || !X_prev || !X0 || !(scale_v > 0.f) || !(scale_d > 0.f)) return STG_EINVAL;
  const stg_status s = warm_check(c, net);
  if (s != STG_OK) return s;
  try {
    const Geom& g = c->lv.back().g;
    const float* y = nullptr;
    if (net) {
      if (!c->wfeat) c->wfeat = dalloc<float>(c, 2LL * g.dim * g.n_nodes);
      // the network's buffers are used on this context's stream
      STG_CUDA_OK(cudaStreamSynchronize(net->st));
      warm_features(g, X_n, X_prev, scale_v, scale_d, c->wfeat, c->st);
      y = cnn_forward(net, c->wfeat, 1, c->st);
    }
    warm_guess(g, c->td, X_n, X_prev, y, scale_d, X0, c->st);
    if (net) STG_CUDA_OK(cudaStreamSynchronize(c->st));
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_warm_scales(stg_ctx* c, const double* X_n, const double* X_prev, double* rms_v, double* rms_dv) {
  if (c && c->lv.back().g.r != 2) {
    c->err = "stg_warm_scales needs order 2";
    return STG_EINVAL;
  }
  if (!c || !X_n || !X_prev) return STG_EINVAL;
  try {
    const Geom& g = c->lv.back().g;
    if (!c->wsum) c->wsum = dalloc<double>(c, 514);
    warm_sums(g, X_n, X_prev, c->wsum, c->st);
    double h[2];
    STG_CUDA_OK(cudaMemcpyAsync(h, c->wsum + 512, sizeof(h), cudaMemcpyDeviceToHost, c->st));
    STG_CUDA_OK(cudaStreamSynchronize(c->st));
    const double R = (double)(g.nvel / g.nt);
    if (rms_v) *rms_v = std::sqrt(h[0] / R);
    if (rms_dv) *rms_dv = std::sqrt(h[1] / R);
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_get_sizes(const stg_ctx* c, int level, long long* n_dofs, long long* n_cells, int* n_patch) {
  if (!c || level < 0 || level >= (int)c->lv.size()) return STG_EINVAL;
  const Geom& g = c->lv[level].g;
  if (n_dofs) *n_dofs = g.N;
  if (n_cells) *n_cells = g.n_cells;
  if (n_patch) *n_patch = g.npatch;
  return STG_OK;
}

stg_status stg_get_local_inverse(const stg_ctx* cc, int level, long long cell, double* out) {
  stg_ctx* c = const_cast<stg_ctx*>(cc);
  if (!c || !out || level < 1 || level >= (int)c->lv.size()) return STG_EINVAL;
  const Geom& g = c->lv[level].g;
  if (cell < 0 || cell >= g.n_cells) return STG_EINVAL;
  try {
    const int n = g.npatch;
    const int cx = (int)(cell % g.n[0]), cy = (int)((cell / g.n[0]) % g.n[1]);
    const int cz = (int)(cell / ((long long)g.n[0] * g.n[1]));
    const long long p = patch_of_cell(g, cx, cy, cz);
    const size_t fs = fsize(c->opt.factor_prec);
    std::vector<unsigned char> raw((size_t)n * n * fs);
    STG_CUDA_OK(cudaStreamSynchronize(c->st));
    STG_CUDA_OK(cudaMemcpy(raw.data(), (const char*)c->lv[level].jinv + (size_t)p * patch_stride(n) * fs,
                           raw.size(), cudaMemcpyDeviceToHost));
    auto val = [&](int col, int row) -> double {
      const size_t i = (size_t)col * n + row;
      if (c->opt.factor_prec == STG_F64) return ((const double*)raw.data())[i];
      if (c->opt.factor_prec == STG_F32) return ((const float*)raw.data())[i];
      unsigned int bits = (unsigned int)((const unsigned short*)raw.data())[i] << 16;
      float f;
      std::memcpy(&f, &bits, 4);
      return f;
    };
    // paper order: a-major; nodes x comps; then pressure coefficients
    const int d = g.dim, blk = g.nloc * d + g.npd;
    auto gpu_index = [&](int mu) {
      const int a = mu / blk, r = mu % blk;
      if (r < g.nloc * d) {
        const int i = r / d, comp = r % d;
        return i * g.NV + a * d + comp;
      }
      return g.nloc * g.NV + a * g.npd + (r - g.nloc * d);
    };
    for (int r = 0; r < n; ++r)
      for (int col = 0; col < n; ++col) out[(size_t)r * n + col] = val(gpu_index(col), gpu_index(r));
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_profile(stg_ctx* c, int enable) {
  if (!c) return STG_EINVAL;
  try {
    if (enable && c->prof_ev.empty()) {
      const int per_cycle = 2 * (1 << c->mesh.dim);  // one sweep's colour launches per V-cycle
      c->prof_ev.resize(per_cycle);
      for (auto& e : c->prof_ev) STG_CUDA_OK(cudaEventCreate(&e));
    }
    if ((bool)enable != c->prof_on) {
      STG_CUDA_OK(cudaStreamSynchronize(c->st));
      if (c->graph) {  // the captured V-cycle changes with the instrumentation
        STG_CUDA_OK(cudaGraphExecDestroy(c->graph));
        c->graph = nullptr;
      }
    }
    c->prof_on = enable != 0;
    c->prof_used = 0;
    c->prof_pending_patches = 0;
    c->prof_ms = 0.0;
    c->prof_launches = 0;
    c->prof_patches = 0;
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_profile_read(const stg_ctx* c, double* total_ms, long long* launches, long long* patches) {
  if (!c) return STG_EINVAL;
  if (total_ms) *total_ms = c->prof_ms;
  if (launches) *launches = c->prof_launches;
  if (patches) *patches = c->prof_patches;
  return STG_OK;
}

long long stg_kernel_launches(void) { return launch_counter(); }

stg_status stg_autotune(stg_ctx* c, int* variant, double* sweep_ms) {
  if (!c) return STG_EINVAL;
  try {
    STG_CUDA_OK(cudaStreamSynchronize(c->st));
    double ms = 0.0;
    for (int l = 1; l < (int)c->lv.size(); ++l) {
      if (vc64(c))
        ms = tune_level<double, double>(c, l, 5);
      else if (c->opt.factor_prec == STG_F32)
        ms = tune_level<float, float>(c, l, 5);
      else
        ms = tune_level<float, __nv_bfloat16>(c, l, 5);
    }
    STG_CUDA_OK(cudaStreamSynchronize(c->st));
    if (c->graph) {  // recapture with the chosen variants
      STG_CUDA_OK(cudaGraphExecDestroy(c->graph));
      c->graph = nullptr;
    }
    if (variant) *variant = c->lv.back().colour_variant;
    if (sweep_ms) *sweep_ms = ms;
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

stg_status stg_set_wait_limit(long long spins) {
  if (spins < 0) return STG_EINVAL;
  try {
    set_colour_wait_limit(spins);
    return STG_OK;
  } catch (const Error& e) {
    g_setup_error = e.msg;
    return e.st;
  }
}

stg_status stg_get_colour_variant(const stg_ctx* c, int level, int* variant) {
  if (!c || !variant || level < 1 || level >= (int)c->lv.size()) return STG_EINVAL;
  *variant = c->lv[level].colour_variant;
  return STG_OK;
}

stg_status stg_set_colour_variant(stg_ctx* c, int level, int variant) {
  if (!c || level < 1 || level >= (int)c->lv.size() || variant < 0 || variant >= kColourVariants)
    return STG_EINVAL;
  try {
    STG_CUDA_OK(cudaStreamSynchronize(c->st));
    c->lv[level].colour_variant = variant;
    if (c->graph) {  // recapture with the new variant
      STG_CUDA_OK(cudaGraphExecDestroy(c->graph));
      c->graph = nullptr;
    }
    return STG_OK;
  } catch (const Error& e) {
    return fail(c, e);
  }
}

}  // extern "C"

struct stg_batch {
  std::vector<stg_ctx*> ctx;
  cudaStream_t main = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<long long> branch_kernels;  // kernels of each problem's V-cycle
  std::vector<cudaEvent_t> ev;
  std::vector<cudaStream_t> branch;  // one capture stream per problem
  cudaGraphConditionalHandle* handles = nullptr;  // device: the IF handle of each branch
  int* live_dev = nullptr;                        // device: 1 = run the branch in the next launch
  int* live_host = nullptr;                       // pinned staging of live_dev
};

namespace stg {

// Head of the batch graph: opens the IF node of every problem still iterating.
__global__ void set_branch_conditions(const cudaGraphConditionalHandle* h, const int* live, int n) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    for (int p = 0; p < n; ++p) cudaGraphSetConditional(h[p], live[p] ? 1u : 0u);
}

}  // namespace stg

extern "C" {

stg_status stg_batch_create(int n, stg_ctx* const* ctxs, stg_batch** out) {
  if (!out || n < 1 || !ctxs) return STG_EINVAL;
  *out = nullptr;
  stg_batch* B = new (std::nothrow) stg_batch();
  if (!B) return STG_ENOMEM;
  try {
    for (int p = 0; p < n; ++p) {
      stg_ctx* c = ctxs[p];
      if (!c || !c->st) throw Error{STG_EINVAL, "every batched context needs a non-default stream"};
      for (int q = 0; q < p; ++q)
        if (ctxs[q] == c) throw Error{STG_EINVAL, "a context appears twice in the batch"};
      if (c->prof_on) throw Error{STG_EINVAL, "turn profiling off before batching"};
      B->ctx.push_back(c);
    }
    STG_CUDA_OK(cudaStreamCreateWithFlags(&B->main, cudaStreamNonBlocking));
    B->ev.resize(n + 1);
    for (auto& e : B->ev) STG_CUDA_OK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    B->branch.resize(n, nullptr);
    for (auto& b : B->branch) STG_CUDA_OK(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
    B->branch_kernels.assign(n, 0);
    for (stg_ctx* c : B->ctx) STG_CUDA_OK(cudaStreamSynchronize(c->st));
    STG_CUDA_OK(cudaMalloc(&B->handles, sizeof(cudaGraphConditionalHandle) * n));
    STG_CUDA_OK(cudaMalloc(&B->live_dev, sizeof(int) * n));
    STG_CUDA_OK(cudaMallocHost(&B->live_host, sizeof(int) * n));
    // One graph: a head kernel that sets the conditions, then every problem's V-cycle as the
    // body of its own IF node (all bodies depend only on the head, so they run concurrently).
    // Each body is captured on a stream of its own, so the contexts' streams may coincide.
    cudaGraph_t graph = nullptr;
    STG_CUDA_OK(cudaGraphCreate(&graph, 0));
    try {
      std::vector<cudaGraphConditionalHandle> hs(n);
      for (int p = 0; p < n; ++p)
        STG_CUDA_OK(cudaGraphConditionalHandleCreate(&hs[p], graph, 0, cudaGraphCondAssignDefault));
      STG_CUDA_OK(cudaMemcpy(B->handles, hs.data(), sizeof(cudaGraphConditionalHandle) * n,
                             cudaMemcpyHostToDevice));
      cudaGraphNode_t head = nullptr;
      cudaKernelNodeParams kp = {};
      const cudaGraphConditionalHandle* hdev = B->handles;
      const int* ldev = B->live_dev;
      int nn = n;
      void* args[] = {(void*)&hdev, (void*)&ldev, (void*)&nn};
      kp.func = (void*)set_branch_conditions;
      kp.gridDim = dim3(1);
      kp.blockDim = dim3(32);
      kp.kernelParams = args;
      STG_CUDA_OK(cudaGraphAddKernelNode(&head, graph, nullptr, 0, &kp));
      for (int p = 0; p < n; ++p) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hs[p];
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        STG_CUDA_OK(cudaGraphAddNode(&node, graph, &head, nullptr, 1, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        stg_ctx* c = B->ctx[p];
        const cudaStream_t saved = c->st;
        c->st = B->branch[p];
        // branch bodies are captured with ordinary launches: programmatic edges are not
        // relied on inside conditional-node bodies
        const int saved_overlap = c->opt.overlap_launches;
        c->opt.overlap_launches = 0;
        const long long before = launch_counter();
        cudaError_t ce = cudaStreamBeginCaptureToGraph(c->st, body, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
          try {
            vcycle_body(c);
          } catch (...) {
            cudaGraph_t g2 = nullptr;
            cudaStreamEndCapture(c->st, &g2);
            c->st = saved;
            c->opt.overlap_launches = saved_overlap;
            launch_counter() = before;
            throw;
          }
          cudaGraph_t g2 = nullptr;
          ce = cudaStreamEndCapture(c->st, &g2);
        }
        c->st = saved;
        c->opt.overlap_launches = saved_overlap;
        B->branch_kernels[p] = launch_counter() - before;
        launch_counter() = before;  // capturing enqueues nothing; launches are counted per live branch
        STG_CUDA_OK(ce);
      }
      STG_CUDA_OK(cudaGraphInstantiate(&B->graph, graph, 0));
    } catch (...) {
      cudaGraphDestroy(graph);
      throw;
    }
    cudaGraphDestroy(graph);
    *out = B;
    return STG_OK;
  } catch (const Error& e) {
    g_setup_error = e.msg;
    stg_batch_destroy(B);
    return e.st;
  }
}

stg_status stg_batch_gmres_solve(stg_batch* B, const double* const* b, double* const* x, int* iters, double* rel) {
  if (!B || !b || !x) return STG_EINVAL;
  const int n = (int)B->ctx.size();
  try {
    std::vector<FgState> S(n);
    for (int p = 0; p < n; ++p) {
      stg_ctx* c = B->ctx[p];
      const Geom& g = c->lv.back().g;
      cabi_to_internal<double>(g, b[p], c->tmp_a, c->st);
      cabi_to_internal<double>(g, x[p], c->tmp_b, c->st);
      fg_begin(S[p], c, c->tmp_a, c->tmp_b);
    }
    std::vector<int> live;
    for (;;) {
      live.clear();
      for (int p = 0; p < n; ++p) {
        if (S[p].done) continue;
        if (!S[p].active) fg_restart(S[p]);
        if (!S[p].done) live.push_back(p);
      }
      if (live.empty()) break;
      for (int p = 0; p < n; ++p) B->live_host[p] = 0;
      long long kernels = 1;
      for (int p : live) {
        fg_pre(S[p]);
        STG_CUDA_OK(cudaEventRecord(B->ev[p], B->ctx[p]->st));
        STG_CUDA_OK(cudaStreamWaitEvent(B->main, B->ev[p], 0));
        B->live_host[p] = 1;
        kernels += B->branch_kernels[p];
      }
      STG_CUDA_OK(cudaMemcpyAsync(B->live_dev, B->live_host, sizeof(int) * n, cudaMemcpyHostToDevice, B->main));
      STG_CUDA_OK(cudaGraphLaunch(B->graph, B->main));  // the live problems' V-cycles, concurrently
      launch_counter() += kernels;
      STG_CUDA_OK(cudaEventRecord(B->ev[n], B->main));
      for (int p : live) {
        STG_CUDA_OK(cudaStreamWaitEvent(B->ctx[p]->st, B->ev[n], 0));
        fg_post(S[p]);
      }
      for (int p : live) {
        STG_CUDA_OK(cudaStreamSynchronize(B->ctx[p]->st));
        fg_update(S[p]);
      }
    }
    stg_status all = STG_OK;
    for (int p = 0; p < n; ++p) {
      stg_ctx* c = B->ctx[p];
      internal_to_cabi<double>(c->lv.back().g, c->tmp_b, x[p], c->st);
      const stg_status sp = fg_result(S[p], iters ? iters + p : nullptr, rel ? rel + p : nullptr);
      if (sp != STG_OK) all = sp;
    }
    for (stg_ctx* c : B->ctx) STG_CUDA_OK(cudaStreamSynchronize(c->st));
    if (colour_kernel_timed_out(B->main)) throw Error{STG_ETIMEOUT, kColourTimeout};
    return all;
  } catch (const Error& e) {
    g_setup_error = e.msg;
    return e.st;
  }
}

void stg_batch_destroy(stg_batch* B) {
  if (!B) return;
  if (B->main) cudaStreamSynchronize(B->main);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  for (auto& e : B->ev)
    if (e) cudaEventDestroy(e);
  if (B->main) cudaStreamDestroy(B->main);
  for (auto& b : B->branch)
    if (b) cudaStreamDestroy(b);
  cudaFree(B->handles);
  cudaFree(B->live_dev);
  if (B->live_host) cudaFreeHost(B->live_host);
  delete B;
}

const char* stg_last_error(const stg_ctx* c) { return c ? c->err.c_str() : g_setup_error.c_str(); }

void stg_destroy(stg_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  if (c->aux) {
    cudaStreamSynchronize(c->aux);
    cudaStreamDestroy(c->aux);
  }
  if (c->aux_done) cudaEventDestroy(c->aux_done);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (auto& e : c->prof_ev) cudaEventDestroy(e);
  c->coarse64.release();
  c->coarse32.release();
  for (void* p : c->owned) cudaFree(p);
  if (c->hh) cudaFreeHost(c->hh);
  delete c;
}

}  // extern "C"
