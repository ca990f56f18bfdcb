// Warm-start network kernels (FP32) and the C-ABI of the network object.
//
// A layer computes y[n][o][i][j] = b[o] + sum_{c,dy,dx} w[o][c][dy][dx] x[n][c][i+dy-1][j+dx-1]
// with zeros outside the image, then tanh unless it is the last layer.  Training
// minimises the mean squared error over all outputs of a batch with Adam.
//
// Kernels:
//  * conv3x3_kernel    one thread per output pixel, all output channels in registers,
//                      weights staged in shared memory as [in][tap][out] so that one
//                      float4 broadcast feeds four FMAs; the same kernel runs the
//                      backward data pass (transposed, flipped weights) with the tanh
//                      derivative of the layer input fused into its epilogue.
//  * wgrad_kernel      per tile of the image (rows x columns of one sample) the partial
//                      weight and bias gradients, tile data staged in shared memory,
//                      each (out, in) channel pair sliding a 3x3 window along a row.
//  * reduce_tiles      sums the tile partials in a fixed order (FP64), so gradients are
//                      bit-reproducible run to run.
//  * mse_kernel, adam_kernel, gather_kernel and the warm-start packing kernels.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/stg.h"
#include "cnn.cuh"

namespace stg {

void set_global_error(const std::string& msg);

namespace {

constexpr int kMaxLayers = 8;
constexpr int kMaxChannels = 32;
constexpr int kConvThreads = 128;
constexpr int kWgThreads = 256;
constexpr int kTileRows = 4;
constexpr int kTileColsMax = 64;
constexpr int kLossBlocks = 256;

// out[n][q][p] = sum_r sum_t K[r][t][q] in[n][r][p + off_t], off_t = (t/3 - 1, t%3 - 1).
// Forward:  K[r][t][q] = w[q][r][t];        out = act(acc + b[q]).
// Backward: K[r][t][q] = w[r][q][8 - t];    out = acc * (1 - a^2), a = the layer input.
template <int Q, bool BWD>
__global__ void __launch_bounds__(kConvThreads) conv3x3_kernel(const float* __restrict__ in, int nr, int nq,
                                                              const float* __restrict__ w,
                                                              const float* __restrict__ bias,
                                                              const float* __restrict__ act,
                                                              float* __restrict__ out, int B, int H, int W,
                                                              int tanh_out) {
  extern __shared__ float4 ks4[];
  float* ks = reinterpret_cast<float*>(ks4);
  for (int e = threadIdx.x; e < nr * 9 * Q; e += blockDim.x) {
    const int q = e % Q, t = (e / Q) % 9, r = e / (9 * Q);
    float v = 0.f;
    if (q < nq) v = BWD ? w[((long long)r * nq + q) * 9 + (8 - t)] : w[((long long)q * nr + r) * 9 + t];
    ks[e] = v;
  }
  __syncthreads();
  const long long HW = (long long)H * W;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= (long long)B * HW) return;
  const int n = (int)(pix / HW);
  const long long p = pix - (long long)n * HW;
  const int i = (int)(p / W), j = (int)(p - (long long)i * W);
  float acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) acc[q] = 0.f;
  const float* inn = in + (long long)n * nr * HW;
  const bool up = i > 0, dn = i + 1 < H, lf = j > 0, rt = j + 1 < W;
  for (int r = 0; r < nr; ++r) {
    const float* c = inn + r * HW + p;
    float x[9];
    x[0] = up && lf ? __ldg(c - W - 1) : 0.f;
    x[1] = up ? __ldg(c - W) : 0.f;
    x[2] = up && rt ? __ldg(c - W + 1) : 0.f;
    x[3] = lf ? __ldg(c - 1) : 0.f;
    x[4] = __ldg(c);
    x[5] = rt ? __ldg(c + 1) : 0.f;
    x[6] = dn && lf ? __ldg(c + W - 1) : 0.f;
    x[7] = dn ? __ldg(c + W) : 0.f;
    x[8] = dn && rt ? __ldg(c + W + 1) : 0.f;
    const float4* kr = ks4 + r * 9 * (Q / 4);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
#pragma unroll
      for (int q4 = 0; q4 < Q / 4; ++q4) {
        const float4 kk = kr[t * (Q / 4) + q4];
        acc[4 * q4 + 0] = fmaf(kk.x, x[t], acc[4 * q4 + 0]);
        acc[4 * q4 + 1] = fmaf(kk.y, x[t], acc[4 * q4 + 1]);
        acc[4 * q4 + 2] = fmaf(kk.z, x[t], acc[4 * q4 + 2]);
        acc[4 * q4 + 3] = fmaf(kk.w, x[t], acc[4 * q4 + 3]);
      }
    }
  }
  float* o = out + (long long)n * nq * HW + p;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if (q >= nq) break;
    float v = acc[q];
    if (!BWD) {
      v += bias[q];
      if (tanh_out) v = tanhf(v);
    } else if (act) {
      const float a = act[(long long)n * nq * HW + q * HW + p];
      v *= 1.f - a * a;
    }
    o[q * HW] = v;
  }
}

struct Tiling {
  int rows, cols, ty, tx;  // tile extent and tiles per direction
  long long tiles(int batch) const { return (long long)batch * ty * tx; }
};

Tiling tiling(int H, int W) {
  Tiling t;
  t.ty = (H + kTileRows - 1) / kTileRows;
  t.rows = (H + t.ty - 1) / t.ty;
  t.tx = (W + kTileColsMax - 1) / kTileColsMax;
  t.cols = (W + t.tx - 1) / t.tx;
  return t;
}

size_t wgrad_smem_bytes(const Tiling& t, int nc, int no) {
  const int gpitch = t.rows * t.cols + 1;
  const int xpitch = (t.rows + 2) * (t.cols + 2) + 1;
  const int P = no * nc;
  const int G = P >= kWgThreads ? 1 : kWgThreads / P;
  const size_t red = G > 1 ? (size_t)G * P * 10 : 0;
  return sizeof(float) * ((size_t)no * gpitch + (size_t)nc * xpitch + red);
}

// part[tile][(o*nc + c)*9 + t] = sum over the tile's pixels p of g[n][o][p] x[n][c][p + off_t];
// part[tile][no*nc*9 + o] = sum of g[n][o][p].  Pixels outside the image carry g = 0.
__global__ void __launch_bounds__(kWgThreads) wgrad_kernel(const float* __restrict__ x, int nc,
                                                          const float* __restrict__ g, int no, int H, int W,
                                                          Tiling tl, float* __restrict__ part) {
  extern __shared__ float sm[];
  const int RB = tl.rows, CW = tl.cols;
  const int gpitch = RB * CW + 1;
  const int xw = CW + 2, xpitch = (RB + 2) * xw + 1;
  float* gs = sm;
  float* xs = sm + no * gpitch;
  const int tile = blockIdx.x;
  const int n = tile / (tl.ty * tl.tx);
  const int ty = (tile / tl.tx) % tl.ty, tx = tile % tl.tx;
  const int y0 = ty * RB, x0 = tx * CW;
  const long long HW = (long long)H * W;
  const float* gn = g + (long long)n * no * HW;
  const float* xn = x + (long long)n * nc * HW;
  for (int e = threadIdx.x; e < no * RB * CW; e += blockDim.x) {
    const int o = e / (RB * CW), rr = (e / CW) % RB, cc = e % CW;
    const int yy = y0 + rr, xx = x0 + cc;
    gs[o * gpitch + rr * CW + cc] = (yy < H && xx < W) ? gn[o * HW + (long long)yy * W + xx] : 0.f;
  }
  for (int e = threadIdx.x; e < nc * (RB + 2) * xw; e += blockDim.x) {
    const int c = e / ((RB + 2) * xw), rr = (e / xw) % (RB + 2), cc = e % xw;
    const int yy = y0 + rr - 1, xx = x0 + cc - 1;
    xs[c * xpitch + rr * xw + cc] =
        (yy >= 0 && yy < H && xx >= 0 && xx < W) ? xn[c * HW + (long long)yy * W + xx] : 0.f;
  }
  __syncthreads();
  const int P = no * nc;
  const int G = P >= (int)blockDim.x ? 1 : (int)blockDim.x / P;
  const int nv = P * 9 + no;
  float* out = part + (long long)tile * nv;
  float* red = xs + nc * xpitch;
  for (int base = 0; base < P; base += (int)blockDim.x) {
    const int slot = threadIdx.x;
    const int pair = G == 1 ? base + slot : slot % P;
    const int grp = G == 1 ? 0 : slot / P;
    const bool active = G == 1 ? pair < P : grp < G;
    float acc[9];
    float accb = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = 0.f;
    if (active) {
      const int o = pair / nc, c = pair % nc;
      const int cb = grp * CW / G, ce = (grp + 1) * CW / G;
      const float* gp = gs + o * gpitch;
      const float* xp = xs + c * xpitch;
      for (int rr = 0; rr < RB; ++rr) {
        if (cb >= ce) break;
        const float* x0r = xp + rr * xw;  // window rows rr, rr+1, rr+2 (image rows y-1, y, y+1)
        float a0 = x0r[cb], a1 = x0r[cb + 1];
        float b0 = x0r[xw + cb], b1 = x0r[xw + cb + 1];
        float c0 = x0r[2 * xw + cb], c1 = x0r[2 * xw + cb + 1];
        for (int cc = cb; cc < ce; ++cc) {
          const float a2 = x0r[cc + 2], b2 = x0r[xw + cc + 2], c2 = x0r[2 * xw + cc + 2];
          const float gv = gp[rr * CW + cc];
          acc[0] = fmaf(gv, a0, acc[0]);
          acc[1] = fmaf(gv, a1, acc[1]);
          acc[2] = fmaf(gv, a2, acc[2]);
          acc[3] = fmaf(gv, b0, acc[3]);
          acc[4] = fmaf(gv, b1, acc[4]);
          acc[5] = fmaf(gv, b2, acc[5]);
          acc[6] = fmaf(gv, c0, acc[6]);
          acc[7] = fmaf(gv, c1, acc[7]);
          acc[8] = fmaf(gv, c2, acc[8]);
          accb += gv;
          a0 = a1;
          a1 = a2;
          b0 = b1;
          b1 = b2;
          c0 = c1;
          c1 = c2;
        }
      }
    }
    if (G == 1) {
      if (active) {
#pragma unroll
        for (int t = 0; t < 9; ++t) out[pair * 9 + t] = acc[t];
        if (pair % nc == 0) out[P * 9 + pair / nc] = accb;
      }
    } else {
      if (active) {
#pragma unroll
        for (int t = 0; t < 9; ++t) red[(grp * P + pair) * 10 + t] = acc[t];
        red[(grp * P + pair) * 10 + 9] = accb;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < P * 10; e += blockDim.x) {
        float s = 0.f;
        for (int q = 0; q < G; ++q) s += red[q * P * 10 + e];
        const int pr = e / 10, t = e % 10;
        if (t < 9)
          out[pr * 9 + t] = s;
        else if (pr % nc == 0)
          out[P * 9 + pr / nc] = s;
      }
    }
  }
}

// dst[j] = sum over tiles of part[tile][j], in tile order, FP64 accumulation.
__global__ void __launch_bounds__(256) reduce_tiles(const float* __restrict__ part, long long ntiles, int nv,
                                                    float* __restrict__ dst) {
  __shared__ double sh[8][32];
  const int jj = threadIdx.x % 32, tl = threadIdx.x / 32;
  const int j = blockIdx.x * 32 + jj;
  double s = 0.0;
  if (j < nv)
    for (long long t = tl; t < ntiles; t += 8) s += part[t * nv + j];
  sh[tl][jj] = s;
  __syncthreads();
  if (tl == 0 && j < nv) {
    double r = 0.0;
    for (int q = 0; q < 8; ++q) r += sh[q][jj];
    dst[j] = (float)r;
  }
}

// g = scale (y - t); part[block] = sum of (y - t)^2 over the block's elements.
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                                  long long M, float scale, float* __restrict__ g,
                                                  double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < M; e += (long long)gridDim.x * blockDim.x) {
    const float d = y[e] - t[e];
    g[e] = scale * d;
    s += (double)d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void mse_final(const double* __restrict__ part, int nb, double inv_m, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *out = s * inv_m;
  }
}

// theta -= lr * m_hat / (sqrt(v_hat) + eps) with m_hat = m c1, v_hat = v c2 (bias corrections).
__global__ void adam_kernel(long long n, float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gv = g[e];
  const float mv = b1 * m[e] + (1.f - b1) * gv;
  const float vv = b2 * v[e] + (1.f - b2) * gv * gv;
  m[e] = mv;
  v[e] = vv;
  th[e] -= lr * (mv * c1) / (sqrtf(vv * c2) + eps);
}

// dst[b][e] = src[idx[b]][e], e < per.
__global__ void gather_kernel(const float* __restrict__ src, const int* __restrict__ idx, int batch, long long per,
                              float* __restrict__ dst) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)batch * per) return;
  const long long b = e / per, r = e - b * per;
  dst[e] = src[(long long)idx[b] * per + r];
}

// ---------------------------------------------------------------- warm-start packing
// Slab vectors in C-ABI order: block a (Radau node) = [R nodal velocities (node-major,
// component fastest) | S P1disc coefficients]; image pixel p = node number (x fastest).

__global__ void features_kernel(Geom g, const double* __restrict__ Xn, const double* __restrict__ Xm, float sv,
                                float sd, float* __restrict__ f) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n_nodes) return;
  const long long blk = g.nvel / g.nt + g.npres / g.nt;
  const long long e0 = (long long)(g.nt - 1) * blk + p * g.dim;
  for (int c = 0; c < g.dim; ++c) {
    const double v = Xn[e0 + c];
    f[c * g.n_nodes + p] = (float)(v / sv);
    f[(g.dim + c) * g.n_nodes + p] = (float)((v - Xm[e0 + c]) / sd);
  }
}

__global__ void target_kernel(Geom g, TimeData td, const double* __restrict__ Xn, const double* __restrict__ Xm,
                              const double* __restrict__ Xp, float sd, float* __restrict__ t) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.n_nodes) return;
  const long long blk = g.nvel / g.nt + g.npres / g.nt;
  const long long e0 = (long long)(g.nt - 1) * blk + p * g.dim;
  for (int c = 0; c < g.dim; ++c) {
    const double v = Xn[e0 + c], dv = v - Xm[e0 + c];
    for (int a = 0; a < g.nt; ++a)
      t[(a * g.dim + c) * g.n_nodes + p] = (float)((Xp[a * blk + p * g.dim + c] - v - td.c[a] * dv) / sd);
  }
}

// X0 block a: velocity v_n + c_a dv (+ sd y[a*d + comp] except at nodes on Dirichlet faces,
// whose data does not change and whose errors the Nitsche penalty weights with gamma / h),
// pressure p_n + c_a (p_n - p_{n-1}).
__global__ void guess_kernel(Geom g, TimeData td, const double* __restrict__ Xn, const double* __restrict__ Xm,
                             const float* __restrict__ y, float sd, double* __restrict__ X0) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  const long long blk = g.nvel / g.nt + g.npres / g.nt;
  const long long R = g.nvel / g.nt;
  const int a = (int)(e / blk);
  const long long r = e - a * blk;
  const long long src = (long long)(g.nt - 1) * blk + r;
  const double v = Xn[src];
  double x = v + td.c[a] * (v - Xm[src]);
  if (y && r < R) {
    const long long p = r / g.dim;
    const int c = (int)(r - p * g.dim);
    const int ix = (int)(p % g.nn[0]), iy = (int)(p / g.nn[0]);
    const bool fixed = ((g.dirichlet & 1u) && ix == 0) || ((g.dirichlet & 2u) && ix == g.nn[0] - 1) ||
                       ((g.dirichlet & 4u) && iy == 0) || ((g.dirichlet & 8u) && iy == g.nn[1] - 1);
    if (!fixed) x += (double)sd * (double)y[(a * g.dim + c) * g.n_nodes + p];
  }
  X0[e] = x;
}

// part[b] / part[256 + b]: block sums of |v_n(t_n)|^2 / |v_n(t_n) - v_{n-1}(t_{n-1})|^2;
// warm_sums_final writes the totals to part[512], part[513].
__global__ void __launch_bounds__(256) warm_sums_kernel(Geom g, const double* __restrict__ Xn,
                                                        const double* __restrict__ Xm, double* __restrict__ part) {
  __shared__ double sv[256], sd[256];
  const long long blk = g.nvel / g.nt + g.npres / g.nt;
  const long long R = g.nvel / g.nt;
  const long long e0 = (long long)(g.nt - 1) * blk;
  double a = 0.0, b = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < R; e += (long long)gridDim.x * blockDim.x) {
    const double v = Xn[e0 + e], d = v - Xm[e0 + e];
    a += v * v;
    b += d * d;
  }
  sv[threadIdx.x] = a;
  sd[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sv[threadIdx.x] += sv[threadIdx.x + w];
      sd[threadIdx.x] += sd[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sv[0];
    part[256 + blockIdx.x] = sd[0];
  }
}

__global__ void warm_sums_final(double* part) {
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int b = 0; b < 256; ++b) s += part[threadIdx.x * 256 + b];
    part[512 + threadIdx.x] = s;
  }
}

template <int Q, bool BWD>
void conv_launch(const float* in, int nr, int nq, const float* w, const float* b, const float* act, float* out,
                 int B, int H, int W, int tanh_out, cudaStream_t st) {
  const size_t smem = sizeof(float) * (size_t)nr * 9 * Q;
  const long long npix = (long long)B * H * W;
  conv3x3_kernel<Q, BWD><<<grid_for(npix, kConvThreads), kConvThreads, smem, st>>>(in, nr, nq, w, b, act, out, B, H,
                                                                                   W, tanh_out);
  STG_LAUNCH_OK();
}

template <bool BWD>
void conv(const float* in, int nr, int nq, const float* w, const float* b, const float* act, float* out, int B,
          int H, int W, int tanh_out, cudaStream_t st) {
  if (nq <= 4)
    conv_launch<4, BWD>(in, nr, nq, w, b, act, out, B, H, W, tanh_out, st);
  else if (nq <= 8)
    conv_launch<8, BWD>(in, nr, nq, w, b, act, out, B, H, W, tanh_out, st);
  else if (nq <= 16)
    conv_launch<16, BWD>(in, nr, nq, w, b, act, out, B, H, W, tanh_out, st);
  else
    conv_launch<32, BWD>(in, nr, nq, w, b, act, out, B, H, W, tanh_out, st);
}

const float* layer_w(const stg_cnn* n, const float* base, int l) { return base + n->off[l]; }
const float* layer_b(const stg_cnn* n, const float* base, int l) {
  return base + n->off[l] + (long long)n->ch[l + 1] * n->ch[l] * 9;
}

const float* forward_from(stg_cnn* n, const float* x, int batch, cudaStream_t st) {
  const float* in = x;
  for (int l = 0; l < n->L; ++l) {
    conv<false>(in, n->ch[l], n->ch[l + 1], layer_w(n, n->params, l), layer_b(n, n->params, l), nullptr,
                n->act[l + 1], batch, n->H, n->W, l + 1 < n->L, st);
    in = n->act[l + 1];
  }
  return n->act[n->L];
}

// Loss and gradients of the batch whose input is x and target t; the loss lands in *loss_dev.
void gradients(stg_cnn* n, const float* x, const float* t, int batch, float* grad, double* loss_dev,
               cudaStream_t st) {
  const float* y = forward_from(n, x, batch, st);
  const long long HW = (long long)n->H * n->W;
  const long long M = (long long)batch * n->ch[n->L] * HW;
  float* g = n->g0;
  float* gnext = n->g1;
  mse_kernel<<<kLossBlocks, 256, 0, st>>>(y, t, M, (float)(2.0 / (double)M), g, n->loss_part);
  STG_LAUNCH_OK();
  mse_final<<<1, 32, 0, st>>>(n->loss_part, kLossBlocks, 1.0 / (double)M, loss_dev);
  STG_LAUNCH_OK();
  const Tiling tl = tiling(n->H, n->W);
  for (int l = n->L - 1; l >= 0; --l) {
    const int nc = n->ch[l], no = n->ch[l + 1];
    const float* xin = l == 0 ? x : n->act[l];
    const size_t smem = wgrad_smem_bytes(tl, nc, no);
    const long long ntiles = tl.tiles(batch);
    wgrad_kernel<<<(unsigned)ntiles, kWgThreads, smem, st>>>(xin, nc, g, no, n->H, n->W, tl, n->part);
    STG_LAUNCH_OK();
    const int nv = no * nc * 9 + no;
    reduce_tiles<<<(nv + 31) / 32, 256, 0, st>>>(n->part, ntiles, nv, grad + n->off[l]);
    STG_LAUNCH_OK();
    if (l > 0) {
      // gradient w.r.t. the layer input, times tanh' of that input (it is a tanh output)
      conv<true>(g, no, nc, layer_w(n, n->params, l), nullptr, n->act[l], gnext, batch, n->H, n->W, 0, st);
      float* tmp = g;
      g = gnext;
      gnext = tmp;
    }
  }
}

void adam(stg_cnn* n, const float* grad, float lr, float b1, float b2, float eps, cudaStream_t st) {
  ++n->adam_t;
  const double c1 = 1.0 / (1.0 - std::pow((double)b1, (double)n->adam_t));
  const double c2 = 1.0 / (1.0 - std::pow((double)b2, (double)n->adam_t));
  adam_kernel<<<grid_for(n->n_params, 256), 256, 0, st>>>(n->n_params, n->params, grad, n->m, n->v, lr, b1, b2, eps,
                                                          (float)c1, (float)c2);
  STG_LAUNCH_OK();
}

stg_status cnn_fail(stg_cnn* n, const Error& e) {
  if (n) n->err = e.msg;
  return e.st;
}

void release(stg_cnn* n) {
  cudaFree(n->params);
  cudaFree(n->grad);
  cudaFree(n->m);
  cudaFree(n->v);
  for (int l = 0; l <= n->L; ++l) cudaFree(n->act[l]);
  cudaFree(n->g0);
  cudaFree(n->g1);
  cudaFree(n->tgt);
  cudaFree(n->part);
  cudaFree(n->loss_part);
  cudaFree(n->loss_dev);
  cudaFree(n->idx);
}

template <typename T>
T* dalloc(long long count) {
  void* p = nullptr;
  if (count <= 0) count = 1;
  if (cudaMalloc(&p, sizeof(T) * (size_t)count) != cudaSuccess) {
    cudaGetLastError();
    throw Error{STG_ENOMEM, "cudaMalloc failed for the network buffers"};
  }
  return static_cast<T*>(p);
}

}  // namespace

const float* cnn_forward(stg_cnn* n, const float* x, int batch, cudaStream_t st) { return forward_from(n, x, batch, st); }

void warm_features(const Geom& g, const double* Xn, const double* Xm, float sv, float sd, float* feat,
                   cudaStream_t st) {
  features_kernel<<<grid_for(g.n_nodes, 256), 256, 0, st>>>(g, Xn, Xm, sv, sd, feat);
  STG_LAUNCH_OK();
}

void warm_target(const Geom& g, const TimeData& td, const double* Xn, const double* Xm, const double* Xp, float sd,
                 float* tgt, cudaStream_t st) {
  target_kernel<<<grid_for(g.n_nodes, 256), 256, 0, st>>>(g, td, Xn, Xm, Xp, sd, tgt);
  STG_LAUNCH_OK();
}

void warm_guess(const Geom& g, const TimeData& td, const double* Xn, const double* Xm, const float* y, float sd,
                double* X0, cudaStream_t st) {
  guess_kernel<<<grid_for(g.N, 256), 256, 0, st>>>(g, td, Xn, Xm, y, sd, X0);
  STG_LAUNCH_OK();
}

void warm_sums(const Geom& g, const double* Xn, const double* Xm, double* part, cudaStream_t st) {
  warm_sums_kernel<<<256, 256, 0, st>>>(g, Xn, Xm, part);
  STG_LAUNCH_OK();
  warm_sums_final<<<1, 32, 0, st>>>(part);
  STG_LAUNCH_OK();
}

}  // namespace stg

using namespace stg;

extern "C" {

stg_status stg_cnn_create(const stg_cnn_desc* d, void* stream, stg_cnn** out) {
  if (!out) return STG_EINVAL;
  *out = nullptr;
  if (!d || d->n_layers < 1 || d->n_layers > kMaxLayers || d->height < 1 || d->width < 1 || d->max_batch < 1) {
    set_global_error("stg_cnn_create: need 1..8 layers and positive height, width and max_batch");
    return STG_EINVAL;
  }
  for (int l = 0; l <= d->n_layers; ++l)
    if (d->channels[l] < 1 || d->channels[l] > kMaxChannels) {
      set_global_error("stg_cnn_create: channel counts must be in 1..32");
      return STG_EINVAL;
    }
  stg_cnn* n = new stg_cnn;
  try {
    n->L = d->n_layers;
    n->H = d->height;
    n->W = d->width;
    n->max_batch = d->max_batch;
    n->st = static_cast<cudaStream_t>(stream);
    int cmax = 0;
    long long part = 0;
    const Tiling tl = tiling(n->H, n->W);
    for (int l = 0; l <= n->L; ++l) {
      n->ch[l] = d->channels[l];
      cmax = std::max(cmax, n->ch[l]);
    }
    for (int l = 0; l < n->L; ++l) {
      n->off.push_back(n->n_params);
      n->n_params += (long long)n->ch[l + 1] * n->ch[l] * 9 + n->ch[l + 1];
      part = std::max(part, tl.tiles(n->max_batch) * ((long long)n->ch[l + 1] * n->ch[l] * 9 + n->ch[l + 1]));
      const size_t smem = wgrad_smem_bytes(tl, n->ch[l], n->ch[l + 1]);
      if (smem > 200 * 1024) throw Error{STG_EINVAL, "stg_cnn_create: layer too wide for the gradient tiles"};
      if (smem > 48 * 1024)
        STG_CUDA_OK(cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    }
    const long long HW = (long long)n->H * n->W;
    n->params = dalloc<float>(n->n_params);
    n->grad = dalloc<float>(n->n_params);
    n->m = dalloc<float>(n->n_params);
    n->v = dalloc<float>(n->n_params);
    for (int l = 0; l <= n->L; ++l) n->act[l] = dalloc<float>((long long)n->max_batch * n->ch[l] * HW);
    n->g0 = dalloc<float>((long long)n->max_batch * cmax * HW);
    n->g1 = dalloc<float>((long long)n->max_batch * cmax * HW);
    n->tgt = dalloc<float>((long long)n->max_batch * n->ch[n->L] * HW);
    n->part = dalloc<float>(part);
    n->part_floats = part;
    n->loss_part = dalloc<double>(kLossBlocks);
    n->loss_dev = dalloc<double>(1);
    STG_CUDA_OK(cudaMemsetAsync(n->params, 0, sizeof(float) * n->n_params, n->st));
    STG_CUDA_OK(cudaMemsetAsync(n->m, 0, sizeof(float) * n->n_params, n->st));
    STG_CUDA_OK(cudaMemsetAsync(n->v, 0, sizeof(float) * n->n_params, n->st));
    STG_CUDA_OK(cudaStreamSynchronize(n->st));
    *out = n;
    return STG_OK;
  } catch (const Error& e) {
    set_global_error(e.msg);
    release(n);
    delete n;
    return e.st;
  }
}

stg_status stg_cnn_n_params(const stg_cnn* n, long long* count) {
  if (!n || !count) return STG_EINVAL;
  *count = n->n_params;
  return STG_OK;
}

stg_status stg_cnn_set_params(stg_cnn* n, const float* params) {
  if (!n || !params) return STG_EINVAL;
  try {
    STG_CUDA_OK(cudaMemcpyAsync(n->params, params, sizeof(float) * n->n_params, cudaMemcpyHostToDevice, n->st));
    STG_CUDA_OK(cudaMemsetAsync(n->m, 0, sizeof(float) * n->n_params, n->st));
    STG_CUDA_OK(cudaMemsetAsync(n->v, 0, sizeof(float) * n->n_params, n->st));
    STG_CUDA_OK(cudaStreamSynchronize(n->st));
    n->adam_t = 0;
    return STG_OK;
  } catch (const Error& e) {
    return cnn_fail(n, e);
  }
}

stg_status stg_cnn_get_params(stg_cnn* n, float* params) {
  if (!n || !params) return STG_EINVAL;
  try {
    STG_CUDA_OK(cudaMemcpyAsync(params, n->params, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost, n->st));
    STG_CUDA_OK(cudaStreamSynchronize(n->st));
    return STG_OK;
  } catch (const Error& e) {
    return cnn_fail(n, e);
  }
}

stg_status stg_cnn_forward(stg_cnn* n, const float* x, float* y, int batch) {
  if (!n || !x || !y || batch < 1 || batch > n->max_batch) return STG_EINVAL;
  try {
    const float* out = forward_from(n, x, batch, n->st);
    STG_CUDA_OK(cudaMemcpyAsync(y, out, sizeof(float) * batch * n->ch[n->L] * (size_t)n->H * n->W,
                                cudaMemcpyDeviceToDevice, n->st));
    return STG_OK;
  } catch (const Error& e) {
    return cnn_fail(n, e);
  }
}

stg_status stg_cnn_gradients(stg_cnn* n, const float* x, const float* t, int batch, float* grad, double* loss) {
  if (!n || !x || !t || !grad || batch < 1 || batch > n->max_batch) return STG_EINVAL;
  try {
    gradients(n, x, t, batch, grad, n->loss_dev, n->st);
    if (loss) {
      STG_CUDA_OK(cudaMemcpyAsync(loss, n->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, n->st));
      STG_CUDA_OK(cudaStreamSynchronize(n->st));
    }
    return STG_OK;
  } catch (const Error& e) {
    return cnn_fail(n, e);
  }
}

stg_status stg_cnn_adam_step(stg_cnn* n, const float* grad, float lr, float beta1, float beta2, float eps) {
  if (!n || !grad || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps >= 0.f))
    return STG_EINVAL;
  try {
    adam(n, grad, lr, beta1, beta2, eps, n->st);
    return STG_OK;
  } catch (const Error& e) {
    return cnn_fail(n, e);
  }
}

stg_status stg_cnn_train(stg_cnn* n, const float* x_all, const float* t_all, int n_samples, const int* order,
                         int batch, int n_steps, float lr, double* losses) {
  if (!n || !x_all || !t_all || !order || n_samples < 1 || batch < 1 || batch > n->max_batch || n_steps < 0 ||
      !(lr >= 0.f))
    return STG_EINVAL;
  const long long total = (long long)batch * n_steps;
  for (long long e = 0; e < total; ++e)
    if (order[e] < 0 || order[e] >= n_samples) {
      n->err = "stg_cnn_train: sample index out of range";
      return STG_EINVAL;
    }
  try {
    if (total > n->idx_cap) {
      cudaFree(n->idx);
      n->idx = nullptr;
      n->idx = dalloc<int>(total);
      n->idx_cap = total;
    }
    STG_CUDA_OK(cudaMemcpyAsync(n->idx, order, sizeof(int) * total, cudaMemcpyHostToDevice, n->st));
    double* ldev = dalloc<double>(n_steps > 0 ? n_steps : 1);
    const long long HW = (long long)n->H * n->W;
    const long long per_x = n->ch[0] * HW, per_t = n->ch[n->L] * HW;
    try {
      for (int s = 0; s < n_steps; ++s) {
        const int* ib = n->idx + (long long)s * batch;
        gather_kernel<<<grid_for(batch * per_x, 256), 256, 0, n->st>>>(x_all, ib, batch, per_x, n->act[0]);
        STG_LAUNCH_OK();
        gather_kernel<<<grid_for(batch * per_t, 256), 256, 0, n->st>>>(t_all, ib, batch, per_t, n->tgt);
        STG_LAUNCH_OK();
        gradients(n, n->act[0], n->tgt, batch, n->grad, ldev + s, n->st);
        adam(n, n->grad, lr, 0.9f, 0.999f, 1e-8f, n->st);
      }
      if (losses && n_steps > 0)
        STG_CUDA_OK(cudaMemcpyAsync(losses, ldev, sizeof(double) * n_steps, cudaMemcpyDeviceToHost, n->st));
      STG_CUDA_OK(cudaStreamSynchronize(n->st));
    } catch (...) {
      cudaStreamSynchronize(n->st);
      cudaFree(ldev);
      throw;
    }
    cudaFree(ldev);
    return STG_OK;
  } catch (const Error& e) {
    return cnn_fail(n, e);
  }
}

const char* stg_cnn_last_error(const stg_cnn* n) { return n ? n->err.c_str() : nullptr; }

stg_status stg_cnn_destroy(stg_cnn* n) {
  if (!n) return STG_OK;
  cudaStreamSynchronize(n->st);
  release(n);
  delete n;
  return STG_OK;
}

}  // extern "C"
