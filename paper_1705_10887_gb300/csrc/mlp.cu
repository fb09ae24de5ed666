// Learned preconditioner of the pinned-Laplacian block solves L_uu X = B.
//
// The harmonic-extension solve E = L_uu^{-1} A_ub and the later solves with the same
// matrix run conjugate gradients preconditioned by M^{-1} = G^T G.  G has the sparsity of
// L_uu (the one-ring of every unknown and its diagonal); its entries are predicted by a
// small network, 6 -> 64 -> 64 -> 1 with tanh, BF16 weights and FP32 arithmetic, from six
// scale-free features of each entry:
//   [i == j,  -L_ij / L_ii,  -L_ij / L_jj,  leak_i,  leak_j,  nnz(row i) / 7],
// where leak_i = (L_ii - sum_{k != i} |L_ik|) / L_ii is the share of the diagonal that ties
// row i to the pinned landmarks.  G_ij = (delta_ij + y(f_ij)) / sqrt(L_ii): with the last
// layer at zero the network is exactly the Jacobi preconditioner, the state it starts
// from and the one it falls back to.
//
// Training uses the pairs the plain solver produces: after a first chunk of columns has
// been solved with Jacobi-preconditioned CG, the network is fitted by full-batch Adam to
// make one application of M^{-1} solve those systems well,
//   loss = sum_c w_c ||L_uu G^T G b_c - b_c||^2,   w_c = 1 / (ncols ||b_c||^2).
// The gradient reaches only entries of rows within one ring of the support of the b_c, so
// the network is evaluated and differentiated there alone.  One epoch is a CUDA graph of
// eleven kernels, replayed.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "mlp.cuh"

namespace sbha {

namespace {

constexpr int H = kMlpHidden;    // 64
constexpr int F = kMlpFeatures;  // 6
constexpr int kOffB1 = H * F;
constexpr int kOffW2 = kOffB1 + H;
constexpr int kOffB2 = kOffW2 + H * H;
constexpr int kOffW3 = kOffB2 + H;
constexpr int kOffB3 = kOffW3 + H;
constexpr int kOffW2T = (kMlpParams + 3) / 4 * 4;  // transposed W2 after the parameters (16-byte aligned)
constexpr int kParamSmem = kOffW2T + H * H;
static_assert(kOffW2 % 4 == 0 && kOffW2T % 4 == 0, "float4 rows of W2 need 16-byte alignment");

constexpr int kBwdThreads = 128;     // samples per tile of the backward kernel
constexpr int kS = kBwdThreads + 4;  // row stride of the per-sample activation arrays

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Parameters into shared memory rounded to BF16 (the network's storage precision), plus W2^T.
__device__ void load_params(const float* __restrict__ p, float* s, bool transposed) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    float v = bf16_round(p[i]);
    s[i] = v;
    if (transposed && i >= kOffW2 && i < kOffB2) {
      int o = i - kOffW2;
      s[kOffW2T + (o % H) * H + o / H] = v;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float dot_row(const float* __restrict__ w, const float (&v)[H]) {
  const float4* w4 = reinterpret_cast<const float4*>(w);
  float a = 0.f;
#pragma unroll
  for (int q = 0; q < H / 4; ++q) {
    float4 t = w4[q];
    a = fmaf(t.x, v[4 * q], a);
    a = fmaf(t.y, v[4 * q + 1], a);
    a = fmaf(t.z, v[4 * q + 2], a);
    a = fmaf(t.w, v[4 * q + 3], a);
  }
  return a;
}

__device__ __forceinline__ void layer1(const float* s, const float (&x)[F], float (&h1)[H]) {
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float a = s[kOffB1 + i];
#pragma unroll
    for (int f = 0; f < F; ++f) a = fmaf(s[i * F + f], x[f], a);
    h1[i] = tanhf(a);
  }
}

// y for N samples, one per thread.
__global__ void __launch_bounds__(128) k_mlp_forward(int64_t N, const float* __restrict__ X,
                                                     const float* __restrict__ params, float* __restrict__ Y) {
  extern __shared__ __align__(16) float smem[];
  load_params(params, smem, false);
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    asm volatile("" ::: "memory");  // weights are re-read from shared memory per sample, not held in registers
    float x[F], h1[H];
#pragma unroll
    for (int f = 0; f < F; ++f) x[f] = X[s * F + f];
    layer1(smem, x, h1);
    float y = smem[kOffB3];
#pragma unroll 4
    for (int i = 0; i < H; ++i) {
      float h2 = tanhf(smem[kOffB2 + i] + dot_row(smem + kOffW2 + i * H, h1));
      y = fmaf(smem[kOffW3 + i], h2, y);
    }
    Y[s] = y;
  }
}

// Parameter gradient sum_s dY_s d y(x_s) / d params, added to grad[].  Each CTA walks tiles of
// 128 samples (one per thread): the forward pass keeps a sample's hidden layer in registers and
// leaves the activations and back-propagated deltas in shared memory, column per sample; every
// thread then owns a fixed set of parameters and sums their per-sample terms over the tile.
__global__ void __launch_bounds__(kBwdThreads) k_mlp_backward(int64_t N, const float* __restrict__ X,
                                                              const float* __restrict__ dY,
                                                              const float* __restrict__ params,
                                                              float* __restrict__ grad) {
  extern __shared__ __align__(16) float smem[];
  float* sp = smem;              // kParamSmem
  float* h1s = sp + kParamSmem;  // [H][kS]
  float* h2s = h1s + H * kS;     // [H][kS]
  float* e2s = h2s + H * kS;     // [H][kS]  d loss / d (layer-2 pre-activation)
  float* e1s = e2s + H * kS;     // [H][kS]  d loss / d (layer-1 pre-activation)
  float* xs = e1s + H * kS;      // [F][kS]
  float* dys = xs + F * kS;      // [kS]
  float* gacc = dys + kS;        // [kMlpParams] this CTA's partial gradient
  load_params(params, sp, true);
  const int t = threadIdx.x;
  for (int o = t; o < kMlpParams; o += kBwdThreads) gacc[o] = 0.f;
  const int64_t ntile = (N + kBwdThreads - 1) / kBwdThreads;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    asm volatile("" ::: "memory");
    int64_t s = tile * kBwdThreads + t;
    bool ok = s < N;
    float x[F], h1[H], e2[H];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      x[f] = ok ? X[s * F + f] : 0.f;
      xs[f * kS + t] = x[f];
    }
    float dy = ok ? dY[s] : 0.f;
    dys[t] = dy;
    layer1(sp, x, h1);
#pragma unroll
    for (int i = 0; i < H; ++i) h1s[i * kS + t] = h1[i];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      float h2 = tanhf(sp[kOffB2 + i] + dot_row(sp + kOffW2 + i * H, h1));
      h2s[i * kS + t] = h2;
      e2[i] = dy * sp[kOffW3 + i] * (1.f - h2 * h2);
      e2s[i * kS + t] = e2[i];
    }
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
      float a = dot_row(sp + kOffW2T + j * H, e2);
      float hj = h1s[j * kS + t];
      e1s[j * kS + t] = a * (1.f - hj * hj);
    }
    __syncthreads();
    for (int o = t; o < kMlpParams; o += kBwdThreads) {
      const float* u;  // per-sample factor 1
      const float* v;  // per-sample factor 2 (nullptr: 1)
      if (o < kOffB1) {
        u = e1s + (o / F) * kS;
        v = xs + (o % F) * kS;
      } else if (o < kOffW2) {
        u = e1s + (o - kOffB1) * kS;
        v = nullptr;
      } else if (o < kOffB2) {
        u = e2s + ((o - kOffW2) / H) * kS;
        v = h1s + ((o - kOffW2) % H) * kS;
      } else if (o < kOffW3) {
        u = e2s + (o - kOffB2) * kS;
        v = nullptr;
      } else if (o < kOffB3) {
        u = dys;
        v = h2s + (o - kOffW3) * kS;
      } else {
        u = dys;
        v = nullptr;
      }
      const float4* u4 = reinterpret_cast<const float4*>(u);
      float a = 0.f;
      if (v) {
        const float4* v4 = reinterpret_cast<const float4*>(v);
#pragma unroll 8
        for (int q = 0; q < kBwdThreads / 4; ++q) {
          float4 p = u4[q], r = v4[q];
          a = fmaf(p.x, r.x, a);
          a = fmaf(p.y, r.y, a);
          a = fmaf(p.z, r.z, a);
          a = fmaf(p.w, r.w, a);
        }
      } else {
#pragma unroll 8
        for (int q = 0; q < kBwdThreads / 4; ++q) {
          float4 p = u4[q];
          a += (p.x + p.y) + (p.z + p.w);
        }
      }
      gacc[o] += a;
    }
    __syncthreads();
  }
  for (int o = t; o < kMlpParams; o += kBwdThreads) atomicAdd(grad + o, gacc[o]);
}

size_t backward_smem_bytes() { return sizeof(float) * (kParamSmem + 4 * H * kS + F * kS + kS + kMlpParams); }

unsigned backward_grid(int64_t N) {
  int64_t tiles = (N + kBwdThreads - 1) / kBwdThreads;
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(tiles, num_sms())));
}

// dY = 2 (Y - T) / N ; loss += sum (Y - T)^2 / N
__global__ void k_mse(int64_t N, const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                      double* __restrict__ loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    float e = Y[s] - T[s];
    dY[s] = 2.f * e / static_cast<float>(N);
    acc += static_cast<double>(e) * e;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / static_cast<double>(N));
}

// One Adam step on the FP32 master parameters; the step counter lives on the device so that
// the epoch can be replayed from a graph.  Launched as a single CTA.
__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, float lr, int32_t* __restrict__ step) {
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  int t = *step + 1;
  float b1t = 1.f - powf(beta1, static_cast<float>(t)), b2t = 1.f - powf(beta2, static_cast<float>(t));
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float gi = g[i];
    float a = beta1 * m1[i] + (1.f - beta1) * gi;
    float b = beta2 * m2[i] + (1.f - beta2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / b1t) / (sqrtf(b / b2t) + eps);
  }
  __syncthreads();
  if (threadIdx.x == 0) *step = t;
}

// Glorot-uniform hidden layers, zero biases, zero output layer (so that y = 0).
__global__ void k_init_params(int n, uint64_t seed, float* __restrict__ p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint64_t x = seed ^ (static_cast<uint64_t>(i) * 0x9e3779b97f4a7c15ull);
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    x ^= x >> 31;
    float r = static_cast<float>(x >> 40) * (2.f / 16777216.f) - 1.f;
    float a = 0.f;
    if (i < kOffB1) a = sqrtf(6.f / (F + H));
    else if (i >= kOffW2 && i < kOffB2) a = sqrtf(6.f / (H + H));
    p[i] = a * r;
  }
}

// ---------------------------------------------------------------- matrix side ----

// Row of every entry, 1/sqrt(diagonal), the diagonal-dominance share leak_i, and checks.
__global__ void k_rows(int64_t m, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, int32_t* __restrict__ erow, double* __restrict__ sc,
                       double* __restrict__ leak, int* __restrict__ err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0, off = 0.0;
    bool diag = false;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      erow[e] = static_cast<int32_t>(i);
      int j = col[e];
      if (j < 0 || j >= m || (e > rowptr[i] && col[e - 1] >= j)) atomicCAS(err, DERR_NONE, DERR_BAD_CSR);
      if (j == i) {
        d = val[e];
        diag = true;
      } else {
        off += fabs(val[e]);
      }
    }
    if (!diag) atomicCAS(err, DERR_NONE, DERR_BAD_CSR);
    if (!(d > 0.0)) {
      atomicCAS(err, DERR_NONE, DERR_BAD_CSR);
      d = 1.0;
    }
    sc[i] = 1.0 / sqrt(d);
    leak[i] = (d - off) / d;
  }
}

// Position of the transposed entry (binary search in the sorted row), features, and the Jacobi G.
__global__ void k_entries(int64_t m, int64_t nnz, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const int32_t* __restrict__ erow,
                          const double* __restrict__ sc, const double* __restrict__ leak, int32_t* __restrict__ tpos,
                          float* __restrict__ feat, float* __restrict__ g32, float* __restrict__ gt32,
                          double* __restrict__ g64, double* __restrict__ gt64, int* __restrict__ err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    int i = erow[e], j = col[e];
    if (j < 0 || j >= m) {  // reported by k_rows
      tpos[e] = static_cast<int32_t>(e);
      continue;
    }
    int lo = rowptr[j], hi = rowptr[j + 1] - 1, at = -1;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      int cm = col[mid];
      if (cm == i) {
        at = mid;
        break;
      }
      if (cm < i) lo = mid + 1;
      else hi = mid - 1;
    }
    if (at < 0) {
      atomicCAS(err, DERR_NONE, DERR_BAD_CSR);  // pattern not symmetric
      at = static_cast<int>(e);
    }
    tpos[e] = at;
    bool d = i == j;
    double si = sc[i], sj = sc[j];
    float* f = feat + e * F;
    f[0] = d ? 1.f : 0.f;
    f[1] = d ? 0.f : static_cast<float>(-val[e] * si * si);
    f[2] = d ? 0.f : static_cast<float>(-val[e] * sj * sj);
    f[3] = static_cast<float>(leak[i]);
    f[4] = static_cast<float>(leak[j]);
    f[5] = static_cast<float>(rowptr[i + 1] - rowptr[i]) * (1.f / 7.f);
    double g = d ? si : 0.0;
    g64[e] = g;
    gt64[e] = g;
    g32[e] = static_cast<float>(g);
    gt32[e] = static_cast<float>(g);
  }
}

// G and G^T entries from network outputs y (for the listed entries, or all when list == nullptr).
__global__ void k_set_g(int64_t count, const int32_t* __restrict__ list, const float* __restrict__ y,
                        const int32_t* __restrict__ erow, const int32_t* __restrict__ col,
                        const int32_t* __restrict__ tpos, const double* __restrict__ sc, float* __restrict__ g32,
                        float* __restrict__ gt32, double* __restrict__ g64, double* __restrict__ gt64) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = list ? list[k] : k;
    int i = erow[e];
    double g = sc[i] * ((i == col[e] ? 1.0 : 0.0) + static_cast<double>(y[k]));
    g32[e] = static_cast<float>(g);
    gt32[tpos[e]] = static_cast<float>(g);
    if (g64) {
      g64[e] = g;
      gt64[tpos[e]] = g;
    }
  }
}

// Training right-hand sides: squared column norms, per-column weights w_c = 1 / (ncols ||b_c||^2),
// an FP32 block copy, and the rows where some b_c is nonzero.
__global__ void k_colsq(int64_t m, int ncols, const double* __restrict__ B, double* __restrict__ bb) {
  __shared__ double red[256];
  int c = blockIdx.x;
  double a = 0.0;
  for (int64_t u = threadIdx.x; u < m; u += blockDim.x) {
    double v = B[((c / 32) * m + u) * 32 + (c % 32)];
    a += v * v;
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) bb[c] = red[0];
}

__global__ void k_weights(int ncp, int ncols, const double* __restrict__ bb, float* __restrict__ w) {
  for (int c = threadIdx.x; c < ncp; c += blockDim.x)
    w[c] = (c < ncols && bb[c] > 0.0) ? static_cast<float>(1.0 / (static_cast<double>(ncols) * bb[c])) : 0.f;
}

__global__ void k_rhs32(int64_t m, int nb, int ncols, const double* __restrict__ B, float* __restrict__ B32,
                        int32_t* __restrict__ supp) {
  int64_t total = static_cast<int64_t>(nb) * m * 32;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int c = static_cast<int>((q / (m * 32)) * 32 + (q % 32));
    double v = c < ncols ? B[q] : 0.0;
    B32[q] = static_cast<float>(v);
    if (supp && v != 0.0) supp[(q / 32) % m] = 1;
  }
}

// Rows within one ring of the support: their entries (all of them) are the ones trained.
__global__ void k_ring_count(int64_t m, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ supp, int32_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    bool in = false;
    for (int e = rowptr[i]; e < rowptr[i + 1] && !in; ++e) in = supp[col[e]] != 0;
    cnt[i] = in ? rowptr[i + 1] - rowptr[i] : 0;
  }
}

__global__ void k_ring_list(int64_t m, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ cnt,
                            const int32_t* __restrict__ off, const float* __restrict__ feat,
                            int32_t* __restrict__ list, float* __restrict__ Xa) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (!cnt[i]) continue;
    int k = off[i];
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e, ++k) {
      list[k] = e;
      for (int f = 0; f < F; ++f) Xa[static_cast<int64_t>(k) * F + f] = feat[static_cast<int64_t>(e) * F + f];
    }
  }
}

// R <- 2 w_c (R - T) where R holds A Z and T = A X; loss[*step] += sum_c w_c ||A Z_c - t_c||^2.
__global__ void k_resid_loss(int64_t m, const float* __restrict__ B, const float* __restrict__ w,
                             float* __restrict__ R, double* __restrict__ loss, const int32_t* __restrict__ step) {
  // CTA (x, y): column block y over the x-th share of the rows, a warp per row and a lane per column;
  // each thread sums its terms in FP32 (a few hundred of them) and the CTA reduces in FP64
  __shared__ double red[256];
  const int lane = threadIdx.x & 31;
  const float wc = w[blockIdx.y * 32 + lane];
  const int64_t base = static_cast<int64_t>(blockIdx.y) * m * 32 + lane;
  const int wpc = blockDim.x >> 5;
  float acc = 0.f;
  for (int64_t u = static_cast<int64_t>(blockIdx.x) * wpc + (threadIdx.x >> 5); u < m;
       u += static_cast<int64_t>(gridDim.x) * wpc) {
    const int64_t q = base + u * 32;
    const float r = R[q] - B[q];
    const float t = wc * r;
    acc = fmaf(t, r, acc);
    R[q] = 2.f * t;
  }
  red[threadIdx.x] = static_cast<double>(acc);
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss + (step ? *step : 0), red[0]);
}

// d loss / d y_e for the listed entries e = (i, j):
//   sc_i * sum_c [ Phi_jc Y_ic + (G Phi)_ic B_jc ]   (one warp per entry)
__global__ void k_entry_grad(int64_t count, int64_t m, int nb, const int32_t* __restrict__ list,
                             const int32_t* __restrict__ erow, const int32_t* __restrict__ col,
                             const double* __restrict__ sc, const float* __restrict__ Phi, const float* __restrict__ Y,
                             const float* __restrict__ GPhi, const float* __restrict__ B, float* __restrict__ dy) {
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = w; k < count; k += nw) {
    int64_t e = list[k];
    int64_t i = erow[e], j = col[e];
    float a = 0.f;
    for (int b = 0; b < nb; ++b) {
      int64_t oi = (b * m + i) * 32 + lane, oj = (b * m + j) * 32 + lane;
      a = fmaf(Phi[oj], Y[oi], a);
      a = fmaf(GPhi[oi], B[oj], a);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) a += __shfl_xor_sync(0xffffffffu, a, s);
    if (lane == 0) dy[k] = a * static_cast<float>(sc[i]);
  }
}

// y = A x in block layout (nb blocks of 32 columns over m rows), FP32: one warp per (row, block), a
// lane per column, eight entries' loads in flight before their FMAs (CSR order, one chain).  Used for
// fewer than four blocks, where the gather product's four-block warp accesses would leave lanes idle.
__global__ void k_bspmm(int64_t m, int nb, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                        const float* __restrict__ val, const float* __restrict__ x, float* __restrict__ y) {
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = w; q < m * nb; q += nw) {
    const int64_t b = q / m, u = q - b * m;
    const float* xb = x + b * m * 32 + lane;
    float a = 0.f;
    const int e1 = rowptr[u + 1];
    for (int e0 = rowptr[u]; e0 < e1; e0 += 8) {
      float vv[8], xv[8];
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        const bool ok = e0 + d < e1;
        vv[d] = ok ? val[e0 + d] : 0.f;
        xv[d] = ok ? xb[static_cast<int64_t>(col[e0 + d]) * 32] : 0.f;
      }
#pragma unroll
      for (int d = 0; d < 8; ++d)
        if (e0 + d < e1) a = fmaf(vv[d], xv[d], a);
    }
    y[(b * m + u) * 32 + lane] = a;
  }
}

unsigned warps_grid(int64_t warps) { return grid_for(warps * 32, 256); }

__global__ void k_check_rowptr(int64_t m, const int32_t* __restrict__ rowptr, int* __restrict__ err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    if (rowptr[i + 1] < rowptr[i]) atomicCAS(err, DERR_NONE, DERR_BAD_CSR);
}

__global__ void k_to_float(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = static_cast<float>(x[i]);
}

__global__ void k_rows_to_blocks(int64_t m, int ncols, int ncp, const double* __restrict__ B, double* __restrict__ out) {
  int64_t total = static_cast<int64_t>(ncp) * m;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = q / (m * 32), u = (q / 32) % m;
    int c = static_cast<int>(b * 32 + q % 32);
    out[q] = c < ncols ? B[u * ncols + c] : 0.0;
  }
}

}  // namespace

void check_rowptr(Ctx& c, int64_t m, const int32_t* rowptr) {
  k_check_rowptr<<<grid_for(m, 256), 256, 0, c.stream>>>(m, rowptr, c.d_err);
  c.launched("check_rowptr");
  c.check_device("CSR input");
}

void to_float(Ctx& c, int64_t n, const double* x, float* y) {
  k_to_float<<<grid_for(n, 256), 256, 0, c.stream>>>(n, x, y);
  c.launched("to_float");
}

void rows_to_blocks(Ctx& c, int64_t m, int ncols, const double* B, double* out) {
  int ncp = (ncols + 31) / 32 * 32;
  k_rows_to_blocks<<<grid_for(static_cast<int64_t>(ncp) * m, 256), 256, 0, c.stream>>>(m, ncols, ncp, B, out);
  c.launched("rows_to_blocks");
}

void mlp_gradient(Ctx& c, int64_t N, const float* X, const float* T, const float* params, float* grad,
                  double* loss) {
  SBHA_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, c.stream));
  SBHA_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), c.stream));
  if (N <= 0) return;
  float* Y = c.alloc<float>(N);
  float* dY = c.alloc<float>(N);
  k_mlp_forward<<<grid_for(N, 128), 128, sizeof(float) * kParamSmem, c.stream>>>(N, X, params, Y);
  c.launched("mlp_forward");
  k_mse<<<grid_for(N, 256, 4 * num_sms()), 256, 0, c.stream>>>(N, Y, T, dY, loss);
  c.launched("mse");
  size_t smem = backward_smem_bytes();
  SBHA_CUDA(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  k_mlp_backward<<<backward_grid(N), kBwdThreads, smem, c.stream>>>(N, X, dY, params, grad);
  c.launched("mlp_backward");
  c.free(Y);
  c.free(dY);
}

LearnedPrecond::LearnedPrecond(Ctx& ctx, int64_t m_, int64_t nnz_, const int32_t* rowptr_, const int32_t* col_,
                               const double* val_, const float* val32_)
    : c(ctx), m(m_), nnz(nnz_), rowptr(rowptr_), col(col_), val(val_), val32(val32_) {
  erow = c.alloc<int32_t>(nnz);
  sc = c.alloc<double>(m);
  double* leak = c.alloc<double>(m);
  tpos = c.alloc<int32_t>(nnz);
  feat = c.alloc<float>(nnz * F);
  g32 = c.alloc<float>(nnz);
  gt32 = c.alloc<float>(nnz);
  g64 = c.alloc<double>(nnz);
  gt64 = c.alloc<double>(nnz);
  params = c.alloc<float>(kMlpParams);
  k_rows<<<grid_for(m, 128), 128, 0, c.stream>>>(m, rowptr, col, val, erow, sc, leak, c.d_err);
  c.launched("precond_rows");
  k_entries<<<grid_for(nnz, 256), 256, 0, c.stream>>>(m, nnz, rowptr, col, val, erow, sc, leak, tpos, feat, g32, gt32,
                                                      g64, gt64, c.d_err);
  c.launched("precond_entries");
  k_init_params<<<grid_for(kMlpParams, 256), 256, 0, c.stream>>>(kMlpParams, 0x1ea2ull, params);
  c.launched("init_params");
  c.check_device("learned preconditioner");
  c.free(leak);
}

namespace {

// Device workspace of one training problem (right-hand sides B, the active entries).
struct Train {
  int nb = 0;
  int64_t na = 0;
  int32_t* list = nullptr;
  float *Xa = nullptr, *ya = nullptr, *dya = nullptr;
  float *B32 = nullptr, *w = nullptr, *Y = nullptr, *Z = nullptr, *R = nullptr, *Phi = nullptr, *GPhi = nullptr;
  float* T32 = nullptr;  // A X (the solutions' image), or B32 itself when no solutions are given
};

Train prepare(Ctx& c, const LearnedPrecond& P, const double* B, const double* X, int ncols) {
  Train t;
  int64_t m = P.m;
  t.nb = (ncols + 31) / 32;
  int ncp = t.nb * 32;
  size_t blk = static_cast<size_t>(m) * ncp;
  t.B32 = c.alloc<float>(blk);
  t.w = c.alloc<float>(ncp);
  t.Y = c.alloc<float>(blk);
  t.Z = c.alloc<float>(blk);
  t.R = c.alloc<float>(blk);
  t.Phi = c.alloc<float>(blk);
  t.GPhi = c.alloc<float>(blk);
  double* bb = c.zeros<double>(ncp);
  k_colsq<<<ncols, 256, 0, c.stream>>>(m, ncols, B, bb);
  c.launched("precond_colsq");
  k_weights<<<1, 256, 0, c.stream>>>(ncp, ncols, bb, t.w);
  c.launched("precond_weights");
  int32_t* supp = c.zeros<int32_t>(m);
  k_rhs32<<<grid_for(blk, 256), 256, 0, c.stream>>>(m, t.nb, ncols, B, t.B32, supp);
  c.launched("precond_rhs");
  int32_t* cnt = c.alloc<int32_t>(m);
  k_ring_count<<<grid_for(m, 128), 128, 0, c.stream>>>(m, P.rowptr, P.col, supp, cnt);
  c.launched("precond_ring_count");
  int32_t* off = c.alloc<int32_t>(m + 1);
  t.na = exclusive_scan(c, cnt, off, m);
  t.list = c.alloc<int32_t>(std::max<int64_t>(t.na, 1));
  t.Xa = c.alloc<float>(std::max<int64_t>(t.na, 1) * F);
  t.ya = c.alloc<float>(std::max<int64_t>(t.na, 1));
  t.dya = c.alloc<float>(std::max<int64_t>(t.na, 1));
  k_ring_list<<<grid_for(m, 128), 128, 0, c.stream>>>(m, P.rowptr, cnt, off, P.feat, t.list, t.Xa);
  c.launched("precond_ring_list");
  t.T32 = t.B32;
  if (X) {  // T = A X from the paired solutions (FP32, like the rest of the loss)
    k_rhs32<<<grid_for(blk, 256), 256, 0, c.stream>>>(m, t.nb, ncols, X, t.Z, nullptr);
    c.launched("precond_rhs");
    t.T32 = c.alloc<float>(blk);
    if (t.nb >= 4) {
      csr_block_spmm_f32(c, m, P.nnz, P.rowptr, P.col, P.val32, t.nb, t.Z, t.T32);
    } else {
      k_bspmm<<<warps_grid(m * t.nb), 256, 0, c.stream>>>(m, t.nb, P.rowptr, P.col, P.val32, t.Z, t.T32);
      c.launched("precond_bspmm");
    }
  }
  c.free(bb);
  c.free(supp);
  c.free(cnt);
  c.free(off);
  return t;
}

void release(Ctx& c, Train& t) {
  for (void* p : {static_cast<void*>(t.list), static_cast<void*>(t.Xa), static_cast<void*>(t.ya),
                  static_cast<void*>(t.dya), static_cast<void*>(t.B32), static_cast<void*>(t.w),
                  static_cast<void*>(t.Y), static_cast<void*>(t.Z), static_cast<void*>(t.R),
                  static_cast<void*>(t.Phi), static_cast<void*>(t.GPhi)})
    c.free(p);
  if (t.T32 != t.B32) c.free(t.T32);
}

// One evaluation of the loss and its gradient on stream s (no allocation: capturable).
void epoch(Ctx& c, cudaStream_t s, const LearnedPrecond& P, const Train& t, const float* params, float* grad,
           double* loss, const int32_t* step) {
  int64_t m = P.m;
  SBHA_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s));
  if (t.na > 0) {
    k_mlp_forward<<<grid_for(t.na, 128), 128, sizeof(float) * kParamSmem, s>>>(t.na, t.Xa, params, t.ya);
    c.launched("mlp_forward");
    k_set_g<<<grid_for(t.na, 256), 256, 0, s>>>(t.na, t.list, t.ya, P.erow, P.col, P.tpos, P.sc, P.g32, P.gt32,
                                                nullptr, nullptr);
    c.launched("precond_set_g");
  }
  // the sparse products through the solver's tuned gather product, issued on the epoch's stream (the
  // context's stream is switched for them and restored on every exit)
  struct StreamSwap {
    Ctx& c;
    cudaStream_t saved;
    ~StreamSwap() { c.stream = saved; }
  } swap{c, c.stream};
  c.stream = s;
  Ctx& cs = c;
  const auto product = [&](const float* val, const float* x, float* y) {
    if (t.nb >= 4) {
      csr_block_spmm_f32(cs, m, P.nnz, P.rowptr, P.col, val, t.nb, x, y);
    } else {
      k_bspmm<<<warps_grid(m * t.nb), 256, 0, s>>>(m, t.nb, P.rowptr, P.col, val, x, y);
      c.launched("precond_bspmm");
    }
  };
  product(P.g32, t.B32, t.Y);    // Y = G B
  product(P.gt32, t.Y, t.Z);     // Z = G^T Y
  product(P.val32, t.Z, t.R);    // R = A Z
  const int64_t lx = std::max<int64_t>(1, std::min<int64_t>(4 * num_sms() / std::max(t.nb, 1), (m + 7) / 8));
  k_resid_loss<<<dim3(static_cast<unsigned>(lx), t.nb), 256, 0, s>>>(m, t.T32, t.w, t.R, loss, step);
  c.launched("precond_resid_loss");
  product(P.val32, t.R, t.Phi);  // Phi = A R
  product(P.g32, t.Phi, t.GPhi);  // G Phi
  if (t.na > 0) {
    k_entry_grad<<<warps_grid(t.na), 256, 0, s>>>(t.na, m, t.nb, t.list, P.erow, P.col, P.sc, t.Phi, t.Y, t.GPhi,
                                                  t.B32, t.dya);
    c.launched("precond_entry_grad");
    k_mlp_backward<<<backward_grid(t.na), kBwdThreads, backward_smem_bytes(), s>>>(t.na, t.Xa, t.dya, params, grad);
    c.launched("mlp_backward");
  }
}

}  // namespace

void LearnedPrecond::loss_grad(const double* B, const double* X, int ncols, const float* p, float* grad,
                               double* loss) {
  SBHA_CUDA(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(backward_smem_bytes())));
  Train t = prepare(c, *this, B, X, ncols);
  SBHA_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), c.stream));
  epoch(c, c.stream, *this, t, p, grad, loss, nullptr);
  release(c, t);
}

bool LearnedPrecond::train(const double* B, const double* X, int ncols, int epochs, float lr, double* loss_first,
                           double* loss_last) {
  SBHA_CUDA(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(backward_smem_bytes())));
  trained = false;
  epochs = std::max(epochs, 1);
  Train t = prepare(c, *this, B, X, ncols);
  train_entries = t.na;
  float* grad = c.alloc<float>(kMlpParams);
  float* m1 = c.zeros<float>(kMlpParams);
  float* m2 = c.zeros<float>(kMlpParams);
  double* hist = c.zeros<double>(epochs + 1);
  int32_t* step = c.zeros<int32_t>(1);
  // capture one epoch (loss, gradient, Adam step) on a private stream and replay it
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  SBHA_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  struct Guard {
    cudaStream_t& s;
    cudaGraph_t& g;
    cudaGraphExec_t& x;
    ~Guard() {
      if (x) cudaGraphExecDestroy(x);
      if (g) cudaGraphDestroy(g);
      if (s) cudaStreamDestroy(s);
    }
  } guard{cs, graph, exec};
  int64_t before = c.launches;
  SBHA_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  epoch(c, cs, *this, t, params, grad, hist, step);
  k_adam<<<1, 1024, 0, cs>>>(kMlpParams, params, grad, m1, m2, lr, step);
  c.launched("adam");
  SBHA_CUDA(cudaStreamEndCapture(cs, &graph));
  SBHA_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  int64_t per_epoch = c.launches - before;
  c.launches = before;
  for (int e = 0; e < epochs; ++e) {
    SBHA_CUDA(cudaGraphLaunch(exec, c.stream));
    c.launches += per_epoch;
  }
  // loss of the final parameters
  epoch(c, c.stream, *this, t, params, grad, hist, step);
  std::vector<double> h(epochs + 1);
  SBHA_CUDA(cudaMemcpyAsync(h.data(), hist, sizeof(double) * (epochs + 1), cudaMemcpyDeviceToHost, c.stream));
  SBHA_CUDA(cudaStreamSynchronize(c.stream));
  if (loss_first) *loss_first = h[0];
  if (loss_last) *loss_last = h[epochs];
  release(c, t);
  for (void* p : {static_cast<void*>(grad), static_cast<void*>(m1), static_cast<void*>(m2), static_cast<void*>(hist),
                  static_cast<void*>(step)})
    c.free(p);
  // the network stalls unless it at least halves the loss of the Jacobi start: keep Jacobi then
  trained = std::isfinite(h[epochs]) && h[epochs] < 0.5 * h[0];
  if (trained) assemble();
  return trained;
}

void LearnedPrecond::assemble() {
  float* y = c.alloc<float>(nnz);
  k_mlp_forward<<<grid_for(nnz, 128), 128, sizeof(float) * kParamSmem, c.stream>>>(nnz, feat, params, y);
  c.launched("mlp_forward");
  k_set_g<<<grid_for(nnz, 256), 256, 0, c.stream>>>(nnz, nullptr, y, erow, col, tpos, sc, g32, gt32, g64, gt64);
  c.launched("precond_set_g");
  c.free(y);
}

void LearnedPrecond::poison() {
  // all-ones bit patterns are NaN in FP32 and FP64
  SBHA_CUDA(cudaMemsetAsync(g32, 0xff, sizeof(float) * nnz, c.stream));
  SBHA_CUDA(cudaMemsetAsync(gt32, 0xff, sizeof(float) * nnz, c.stream));
  SBHA_CUDA(cudaMemsetAsync(g64, 0xff, sizeof(double) * nnz, c.stream));
  SBHA_CUDA(cudaMemsetAsync(gt64, 0xff, sizeof(double) * nnz, c.stream));
}

}  // namespace sbha
