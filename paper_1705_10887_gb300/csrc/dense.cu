// Dense FP64 building blocks of the factored interpolation solve: tiled GEMMs on the
// column-block layout of the solver (column c of an m-row array at
// ((c / 32) * m + u) * 32 + c % 32) and on row-major matrices, the landmark-space
// matrices T = D_b + E^T D_u E and S = L_bb - A_bu E, and a column-parallel PCG for
// the small SPD systems T Y = S.
//
// The GEMM tile is 64 x 64 with a depth of 16, 256 threads computing 4 x 4 outputs
// each from shared-memory tiles; the operands are read through small accessor
// structs so that one kernel serves every layout.  These products are FP64 because
// their results feed the operator entries at full precision.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace sbha {

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

// column-block layout read: (row u, column col), optional row scale
struct BlockAt {
  const double* p;
  int64_t m;
  const double* scale;
  __device__ __forceinline__ double operator()(int64_t u, int64_t col) const {
    double v = p[((col >> 5) * m + u) * 32 + (col & 31)];
    return scale ? v * scale[u] : v;
  }
};
// transposed view of a block-layout array: (col, u)
struct BlockAtT {
  BlockAt b;
  __device__ __forceinline__ double operator()(int64_t col, int64_t u) const { return b(u, col); }
};
struct RowAt {
  const double* p;
  int64_t ld;
  __device__ __forceinline__ double operator()(int64_t i, int64_t j) const { return p[i * ld + j]; }
};
struct RowAtT {
  const double* p;
  int64_t ld;
  __device__ __forceinline__ double operator()(int64_t i, int64_t j) const { return p[j * ld + i]; }
};

// C(i, j) = sum_k A(i, k) B(k, j) over k in this z-slice; out(i, j, value) stores.  AI: consecutive
// threads load consecutive i of A (A is contiguous along i); otherwise along k.  LOWER: C is
// symmetric and only the tiles on or below the diagonal are computed.
template <bool AI, class AF, class BF, class OF, bool LOWER = false>
__global__ void __launch_bounds__(256) k_dgemm(int64_t M, int64_t N, int64_t K, AF A, BF B, OF out) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  if (LOWER && blockIdx.y < blockIdx.x) return;
  int64_t i0 = static_cast<int64_t>(blockIdx.y) * TM, j0 = static_cast<int64_t>(blockIdx.x) * TN;
  int64_t kper = (K + gridDim.z - 1) / gridDim.z;
  int64_t kbeg = kper * blockIdx.z, kend = min(K, kbeg + kper);
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int64_t k0 = kbeg; k0 < kend; k0 += TK) {
    for (int q = threadIdx.x; q < TK * TM; q += 256) {
      int ii = AI ? q % TM : q / TK, kk = AI ? q / TM : q % TK;
      int64_t gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < M && gk < kend) ? A(gi, gk) : 0.0;
    }
    for (int q = threadIdx.x; q < TK * TN; q += 256) {
      int jj = q % TN, kk = q / TN;
      int64_t gj = j0 + jj, gk = k0 + kk;
      Bs[kk][jj] = (gj < N && gk < kend) ? B(gk, gj) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int s = 0; s < 4; ++s) b[s] = Bs[kk][tx * 4 + s];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[r][s] = fma(a[r], b[s], acc[r][s]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int64_t gi = i0 + ty * 4 + r, gj = j0 + tx * 4 + s;
      if (gi < M && gj < N) out(gi, gj, acc[r][s]);
    }
}

// out: row-major partial slice z
struct PartialOut {
  double* p;
  int64_t M, N;
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double v) const {
    p[(static_cast<int64_t>(blockIdx.z) * M + i) * N + j] = v;
  }
};
// out: block layout with optional row scale
struct BlockOut {
  double* p;
  int64_t m;
  const double* scale;
  __device__ __forceinline__ void operator()(int64_t u, int64_t col, double v) const {
    p[((col >> 5) * m + u) * 32 + (col & 31)] = scale ? v * scale[u] : v;
  }
};
struct RowOut {
  double* p;
  int64_t ld;
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double v) const { p[i * ld + j] = v; }
};

// T = diag(db) + sum over slices.  sym: only the tiles on or below the diagonal were computed;
// element (i, j) of an upper tile is read as (j, i).
__global__ void k_sum_slices(int64_t M, int64_t N, int Z, const double* __restrict__ part,
                             const double* __restrict__ diag, double* __restrict__ out, bool sym = false) {
  int64_t total = M * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = q / N, j = q % N;
    int64_t src = (sym && i / TM < j / TN) ? j * N + i : q;
    double s = 0.0;
    for (int z = 0; z < Z; ++z) s += part[z * total + src];
    if (diag && (q / N) == (q % N)) s += diag[q / N];
    out[q] = s;
  }
}

// S_jk = Lbb_jk - sum_e a_e E(u_e, k) over the landmark's unknown neighbours (A_ub column j)
__global__ void k_schur(int l, int64_t m, const double* __restrict__ Lbb, const int32_t* __restrict__ aptr,
                        const int32_t* __restrict__ arow, const double* __restrict__ aval, const double* __restrict__ E,
                        double* __restrict__ S) {
  int64_t total = static_cast<int64_t>(l) * l;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int j = static_cast<int>(q / l), k = static_cast<int>(q % l);
    double s = Lbb[q];
    for (int e = aptr[j]; e < aptr[j + 1]; ++e) s -= aval[e] * E[((static_cast<int64_t>(k) >> 5) * m + arow[e]) * 32 + (k & 31)];
    S[q] = s;
  }
}

// ------------------------------------------------------- small dense PCG ---

// per-column dots of two row-major l x N arrays: out[j] = sum_i a_ij b_ij (w_i optional)
__global__ void k_coldot(int64_t rows, int64_t N, const double* __restrict__ a, const double* __restrict__ b,
                         const double* __restrict__ w, double* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t i = 0; i < rows; ++i) {
      double t = a[i * N + j] * b[i * N + j];
      s += w ? t * w[i] : t;
    }
    out[j] = s;
  }
}

__global__ void k_inv_diag(int64_t l, const double* __restrict__ T, double* __restrict__ dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < l; i += (int64_t)gridDim.x * blockDim.x)
    dinv[i] = 1.0 / T[i * l + i];
}

// X = 0, R = S, P = D^-1 R
__global__ void k_dpcg_init(int64_t rows, int64_t N, const double* __restrict__ S, const double* __restrict__ dinv,
                            double* __restrict__ X, double* __restrict__ R, double* __restrict__ P) {
  int64_t total = rows * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    X[q] = 0.0;
    R[q] = S[q];
    P[q] = S[q] * dinv[q / N];
  }
}

// alpha_j = rz_j / pq_j ; X += alpha P ; R -= alpha Q
__global__ void k_dpcg_xr(int64_t rows, int64_t N, const double* __restrict__ rz, const double* __restrict__ pq,
                          const int* __restrict__ act, double* __restrict__ X, double* __restrict__ R,
                          const double* __restrict__ P, const double* __restrict__ Q) {
  int64_t total = rows * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = q % N;
    if (!act[j] || pq[j] == 0.0) continue;
    double a = rz[j] / pq[j];
    X[q] += a * P[q];
    R[q] -= a * Q[q];
  }
}

// beta_j = rz_new_j / rz_j ; P = D^-1 R + beta P ; rz <- rz_new ; deactivate converged columns
__global__ void k_dpcg_p(int64_t rows, int64_t N, double* __restrict__ rz, const double* __restrict__ rz_new,
                         const double* __restrict__ rr, const double* __restrict__ bb, double tol2,
                         const double* __restrict__ dinv, int* __restrict__ act, const double* __restrict__ R,
                         double* __restrict__ P) {
  int64_t total = rows * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = q % N;
    if (!act[j] || rz[j] == 0.0) continue;
    double b = rz_new[j] / rz[j];
    P[q] = R[q] * dinv[q / N] + b * P[q];
  }
}

__global__ void k_dpcg_state(int64_t N, double* __restrict__ rz, const double* __restrict__ rz_new,
                             const double* __restrict__ rr, const double* __restrict__ bb, double tol2,
                             int* __restrict__ act, int* __restrict__ nact) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    if (!act[j]) continue;
    rz[j] = rz_new[j];
    if (rr[j] <= tol2 * bb[j]) act[j] = 0;
    else atomicAdd(nact, 1);
  }
}

__global__ void k_init_act(int64_t N, const double* __restrict__ bb, int* __restrict__ act) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
    act[j] = bb[j] > 0.0 ? 1 : 0;
}

unsigned tiles(int64_t n, int t) { return static_cast<unsigned>((n + t - 1) / t); }

}  // namespace

void weighted_gram(Ctx& c, int64_t m, int32_t l, const double* E, const double* Du, const double* Db, double* T) {
  int Z = static_cast<int>(std::min<int64_t>(32, std::max<int64_t>(1, m / 2048)));
  double* part = c.alloc<double>(static_cast<size_t>(Z) * l * l);
  BlockAt e{E, m, nullptr};
  BlockAt de{E, m, Du};
  dim3 grid(tiles(l, TN), tiles(l, TM), Z);
  // T is symmetric: the tiles on or below the diagonal, mirrored when the slices are summed
  k_dgemm<true, BlockAtT, BlockAt, PartialOut, true><<<grid, 256, 0, c.stream>>>(
      static_cast<int64_t>(l), static_cast<int64_t>(l), m, BlockAtT{e}, de, PartialOut{part, l, l});
  c.launched("dgemm_gram");
  k_sum_slices<<<grid_for(static_cast<int64_t>(l) * l, 256), 256, 0, c.stream>>>(l, l, Z, part, Db, T, true);
  c.launched("sum_slices");
  c.free(part);
}

void dgemm_rowmajor(Ctx& c, int64_t M, int64_t N, int64_t K, const double* A, const double* B, double* C) {
  int Z = static_cast<int>(std::min<int64_t>(32, std::max<int64_t>(1, K / 2048)));
  double* part = c.alloc<double>(static_cast<size_t>(Z) * M * N);
  dim3 grid(tiles(N, TN), tiles(M, TM), Z);
  k_dgemm<false><<<grid, 256, 0, c.stream>>>(M, N, K, RowAt{A, K}, RowAt{B, N}, PartialOut{part, M, N});
  c.launched("dgemm");
  k_sum_slices<<<grid_for(M * N, 256), 256, 0, c.stream>>>(M, N, Z, part, nullptr, C);
  c.launched("sum_slices");
  c.free(part);
}

void landmark_schur(Ctx& c, int64_t m, int32_t l, const double* Lbb, const int32_t* aptr, const int32_t* arow,
                    const double* aval, const double* E, double* S) {
  k_schur<<<grid_for(static_cast<int64_t>(l) * l, 256), 256, 0, c.stream>>>(l, m, Lbb, aptr, arow, aval, E, S);
  c.launched("schur");
}

// F(:, 0..N) = diag(Du) E Y(:, col0 .. col0+N) written in block layout (N columns)
void gemm_EY(Ctx& c, int64_t m, int32_t l, const double* E, const double* Y, int64_t ldy, int64_t col0, int64_t N,
             const double* Du, double* F) {
  dim3 grid(tiles(N, TN), tiles(m, TM), 1);
  k_dgemm<false><<<grid, 256, 0, c.stream>>>(m, N, static_cast<int64_t>(l), BlockAt{E, m, nullptr}, RowAt{Y + col0, ldy},
                                      BlockOut{F, m, Du});
  c.launched("dgemm_EY");
}

// V (l x N, row-major) = E^T diag(Du) X, X in block layout with N columns
void gemm_EtDX(Ctx& c, int64_t m, int32_t l, const double* E, const double* Du, const double* X, int64_t N,
               double* V) {
  int Z = static_cast<int>(std::min<int64_t>(32, std::max<int64_t>(1, m / 2048)));
  double* part = c.alloc<double>(static_cast<size_t>(Z) * l * N);
  dim3 grid(tiles(N, TN), tiles(l, TM), Z);
  k_dgemm<true><<<grid, 256, 0, c.stream>>>(static_cast<int64_t>(l), N, m, BlockAtT{BlockAt{E, m, nullptr}},
                                      BlockAt{X, m, Du}, PartialOut{part, l, N});
  c.launched("dgemm_EtDX");
  k_sum_slices<<<grid_for(static_cast<int64_t>(l) * N, 256), 256, 0, c.stream>>>(l, N, Z, part, nullptr, V);
  c.launched("sum_slices");
  c.free(part);
}

// Solves T Y = S (T SPD, l x l, row-major; S l x N) by column-parallel Jacobi-PCG to rtol.
int dense_spd_solve(Ctx& c, int32_t l, const double* T, const double* S, int64_t N, double* Y, double rtol,
                    int max_iter) {
  int64_t ln = static_cast<int64_t>(l) * N;
  double* R = c.alloc<double>(ln);
  double* P = c.alloc<double>(ln);
  double* Q = c.alloc<double>(ln);
  double* dinv = c.alloc<double>(l);
  double* rz = c.alloc<double>(N);
  double* rzn = c.alloc<double>(N);
  double* pq = c.alloc<double>(N);
  double* rr = c.alloc<double>(N);
  double* bb = c.alloc<double>(N);
  int* act = c.alloc<int>(N);
  int* nact = c.alloc<int>(1);
  unsigned g = grid_for(ln, 256);
  unsigned gn = grid_for(N, 128);
  k_inv_diag<<<grid_for(l, 128), 128, 0, c.stream>>>(l, T, dinv);
  c.launched("inv_diag");
  k_dpcg_init<<<g, 256, 0, c.stream>>>(l, N, S, dinv, Y, R, P);
  c.launched("dpcg_init");
  k_coldot<<<gn, 128, 0, c.stream>>>(l, N, R, R, dinv, rz);
  c.launched("coldot");
  k_coldot<<<gn, 128, 0, c.stream>>>(l, N, R, R, nullptr, bb);
  c.launched("coldot");
  k_init_act<<<gn, 128, 0, c.stream>>>(N, bb, act);
  c.launched("init_act");
  dim3 grid(tiles(N, TN), tiles(l, TM), 1);
  int it = 0;
  int h_nact = 1;
  while (it < max_iter) {
    for (int b = 0; b < 4 && it < max_iter; ++b, ++it) {
      // T is symmetric: read A(i, k) = T(k, i) so that consecutive threads load consecutive addresses
      k_dgemm<true><<<grid, 256, 0, c.stream>>>(static_cast<int64_t>(l), N, static_cast<int64_t>(l), RowAtT{T, l},
                                                RowAt{P, N}, RowOut{Q, N});
      c.launched("dgemm_TP");
      k_coldot<<<gn, 128, 0, c.stream>>>(l, N, P, Q, nullptr, pq);
      c.launched("coldot");
      k_dpcg_xr<<<g, 256, 0, c.stream>>>(l, N, rz, pq, act, Y, R, P, Q);
      c.launched("dpcg_xr");
      k_coldot<<<gn, 128, 0, c.stream>>>(l, N, R, R, dinv, rzn);
      c.launched("coldot");
      k_coldot<<<gn, 128, 0, c.stream>>>(l, N, R, R, nullptr, rr);
      c.launched("coldot");
      k_dpcg_p<<<g, 256, 0, c.stream>>>(l, N, rz, rzn, rr, bb, rtol * rtol, dinv, act, R, P);
      c.launched("dpcg_p");
      SBHA_CUDA(cudaMemsetAsync(nact, 0, sizeof(int), c.stream));
      k_dpcg_state<<<gn, 128, 0, c.stream>>>(N, rz, rzn, rr, bb, rtol * rtol, act, nact);
      c.launched("dpcg_state");
    }
    SBHA_CUDA(cudaMemcpyAsync(&h_nact, nact, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    SBHA_CUDA(cudaStreamSynchronize(c.stream));
    if (h_nact == 0) break;
  }
  for (void* p : {static_cast<void*>(R), static_cast<void*>(P), static_cast<void*>(Q), static_cast<void*>(dinv),
                  static_cast<void*>(rz), static_cast<void*>(rzn), static_cast<void*>(pq), static_cast<void*>(rr),
                  static_cast<void*>(bb), static_cast<void*>(act), static_cast<void*>(nact)})
    c.free(p);
  if (h_nact != 0) SBHA_THROW(SBHA_ENOCONV, "landmark-space system T Y = S did not converge");
  return it;
}


// ------------------------------------------------------ blocked Cholesky ---
//
// T = L L^T for the small SPD landmark-space matrices, right-looking with 32-wide
// panels: factor the diagonal block in one CTA, solve the panel below it, update the
// trailing lower triangle; then blocked forward and backward substitution for many
// right-hand sides.  FP64 throughout.

namespace {

constexpr int CB = 32;

__global__ void __launch_bounds__(CB * CB) k_chol_diag(int l, int k0, int kb, double* __restrict__ A, int* err) {
  __shared__ double a[CB][CB + 1];
  int tx = threadIdx.x % CB, ty = threadIdx.x / CB;
  if (ty < kb && tx < kb) a[ty][tx] = A[static_cast<int64_t>(k0 + ty) * l + k0 + tx];
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (ty == j && tx == j) {
      double d = a[j][j];
      if (!(d > 0.0)) {
        set_error(err, DERR_NOT_SPD);
        d = 1.0;
      }
      a[j][j] = sqrt(d);
    }
    __syncthreads();
    if (tx == j && ty > j && ty < kb) a[ty][j] /= a[j][j];
    __syncthreads();
    if (ty > j && tx > j && tx <= ty && ty < kb) a[ty][tx] -= a[ty][j] * a[tx][j];
    __syncthreads();
  }
  if (ty < kb && tx <= ty) A[static_cast<int64_t>(k0 + ty) * l + k0 + tx] = a[ty][tx];
}

// rows i >= k0 + kb: L[i, k0:k0+kb] = A[i, k0:k0+kb] L_kk^{-T}
__global__ void k_chol_panel(int l, int k0, int kb, double* __restrict__ A) {
  __shared__ double d[CB][CB + 1];
  for (int q = threadIdx.x; q < kb * kb; q += blockDim.x) d[q / kb][q % kb] = A[static_cast<int64_t>(k0 + q / kb) * l + k0 + q % kb];
  __syncthreads();
  for (int i = k0 + kb + blockIdx.x * blockDim.x + threadIdx.x; i < l; i += gridDim.x * blockDim.x) {
    double x[CB];
    for (int j = 0; j < kb; ++j) x[j] = A[static_cast<int64_t>(i) * l + k0 + j];
    for (int j = 0; j < kb; ++j) {
      double s = x[j];
      for (int t = 0; t < j; ++t) s -= x[t] * d[j][t];
      x[j] = s / d[j][j];
    }
    for (int j = 0; j < kb; ++j) A[static_cast<int64_t>(i) * l + k0 + j] = x[j];
  }
}

// trailing lower triangle: A[i][j] -= sum_t L[i][k0+t] L[j][k0+t], k0+kb <= j <= i < l
__global__ void k_chol_update(int l, int k0, int kb, double* __restrict__ A) {
  int i = k0 + kb + blockIdx.y * 16 + threadIdx.y;
  int j = k0 + kb + blockIdx.x * 16 + threadIdx.x;
  if (i >= l || j > i) return;
  const double* ri = A + static_cast<int64_t>(i) * l + k0;
  const double* rj = A + static_cast<int64_t>(j) * l + k0;
  double s = 0.0;
  for (int t = 0; t < kb; ++t) s += ri[t] * rj[t];
  A[static_cast<int64_t>(i) * l + j] -= s;
}

// forward: B[k0:k0+kb, c] <- L_kk^{-1} B[k0:k0+kb, c]   (thread per column)
__global__ void k_trsm_fwd_diag(int l, int64_t N, int k0, int kb, const double* __restrict__ Lc, double* __restrict__ B) {
  __shared__ double d[CB][CB + 1];
  for (int q = threadIdx.x; q < kb * kb; q += blockDim.x) d[q / kb][q % kb] = Lc[static_cast<int64_t>(k0 + q / kb) * l + k0 + q % kb];
  __syncthreads();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
    double x[CB];
    for (int j = 0; j < kb; ++j) {
      double s = B[static_cast<int64_t>(k0 + j) * N + c];
      for (int t = 0; t < j; ++t) s -= d[j][t] * x[t];
      x[j] = s / d[j][j];
    }
    for (int j = 0; j < kb; ++j) B[static_cast<int64_t>(k0 + j) * N + c] = x[j];
  }
}

// forward update: B[i, c] -= sum_t L[i, k0+t] B[k0+t, c] for i >= k0 + kb
__global__ void k_trsm_fwd_update(int l, int64_t N, int k0, int kb, const double* __restrict__ Lc, double* __restrict__ B) {
  int64_t total = static_cast<int64_t>(l - k0 - kb) * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int i = k0 + kb + static_cast<int>(q / N);
    int64_t c = q % N;
    double s = 0.0;
    for (int t = 0; t < kb; ++t) s += Lc[static_cast<int64_t>(i) * l + k0 + t] * B[static_cast<int64_t>(k0 + t) * N + c];
    B[static_cast<int64_t>(i) * N + c] -= s;
  }
}

// backward: B[k0:k0+kb, c] <- L_kk^{-T} B[k0:k0+kb, c]
__global__ void k_trsm_bwd_diag(int l, int64_t N, int k0, int kb, const double* __restrict__ Lc, double* __restrict__ B) {
  __shared__ double d[CB][CB + 1];
  for (int q = threadIdx.x; q < kb * kb; q += blockDim.x) d[q / kb][q % kb] = Lc[static_cast<int64_t>(k0 + q / kb) * l + k0 + q % kb];
  __syncthreads();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
    double x[CB];
    for (int j = kb - 1; j >= 0; --j) {
      double s = B[static_cast<int64_t>(k0 + j) * N + c];
      for (int t = j + 1; t < kb; ++t) s -= d[t][j] * x[t];
      x[j] = s / d[j][j];
    }
    for (int j = 0; j < kb; ++j) B[static_cast<int64_t>(k0 + j) * N + c] = x[j];
  }
}

// backward update: B[i, c] -= sum_t L[k0+t, i] B[k0+t, c] for i < k0
__global__ void k_trsm_bwd_update(int l, int64_t N, int k0, int kb, const double* __restrict__ Lc, double* __restrict__ B) {
  int64_t total = static_cast<int64_t>(k0) * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int i = static_cast<int>(q / N);
    int64_t c = q % N;
    double s = 0.0;
    for (int t = 0; t < kb; ++t) s += Lc[static_cast<int64_t>(k0 + t) * l + i] * B[static_cast<int64_t>(k0 + t) * N + c];
    B[static_cast<int64_t>(i) * N + c] -= s;
  }
}

}  // namespace

// Lower Cholesky factor of the SPD l x l row-major matrix T (returns a new device array).
double* cholesky(Ctx& c, int32_t l, const double* T) {
  double* A = c.alloc<double>(static_cast<size_t>(l) * l);
  SBHA_CUDA(cudaMemcpyAsync(A, T, sizeof(double) * l * l, cudaMemcpyDeviceToDevice, c.stream));
  for (int k0 = 0; k0 < l; k0 += CB) {
    int kb = std::min(CB, l - k0);
    k_chol_diag<<<1, CB * CB, 0, c.stream>>>(l, k0, kb, A, c.d_err);
    c.launched("chol_diag");
    int rest = l - k0 - kb;
    if (rest <= 0) break;
    k_chol_panel<<<grid_for(rest, 128), 128, 0, c.stream>>>(l, k0, kb, A);
    c.launched("chol_panel");
    dim3 g(tiles(rest, 16), tiles(rest, 16));
    k_chol_update<<<g, dim3(16, 16), 0, c.stream>>>(l, k0, kb, A);
    c.launched("chol_update");
  }
  c.check_device("landmark-space factorisation");
  return A;
}

// B (l x N, row-major) <- (L L^T)^{-1} B
void cholesky_solve(Ctx& c, int32_t l, const double* Lc, double* B, int64_t N) {
  for (int k0 = 0; k0 < l; k0 += CB) {
    int kb = std::min(CB, l - k0);
    k_trsm_fwd_diag<<<grid_for(N, 128), 128, 0, c.stream>>>(l, N, k0, kb, Lc, B);
    c.launched("trsm_fwd_diag");
    if (l - k0 - kb > 0) {
      k_trsm_fwd_update<<<grid_for(static_cast<int64_t>(l - k0 - kb) * N, 256), 256, 0, c.stream>>>(l, N, k0, kb, Lc, B);
      c.launched("trsm_fwd_update");
    }
  }
  int last = ((l - 1) / CB) * CB;
  for (int k0 = last; k0 >= 0; k0 -= CB) {
    int kb = std::min(CB, l - k0);
    k_trsm_bwd_diag<<<grid_for(N, 128), 128, 0, c.stream>>>(l, N, k0, kb, Lc, B);
    c.launched("trsm_bwd_diag");
    if (k0 > 0) {
      k_trsm_bwd_update<<<grid_for(static_cast<int64_t>(k0) * N, 256), 256, 0, c.stream>>>(l, N, k0, kb, Lc, B);
      c.launched("trsm_bwd_update");
    }
  }
}

}  // namespace sbha
