// Classical scaling with the sparse approximation (Sec. 3.3).
//
// The top-k eigenpairs of -1/2 J P (W.W) P^T J (n x n) are found in the landmark
// space.  With c = P^T 1 and G = (J P)^T (J P) = P^T P - c c^T / n, the operator
// T = -1/2 (W.W) G (l x l) is self-adjoint in the G inner product and its nonzero
// eigenvalues are those of the n x n matrix; an eigenvector y with y^T G y = 1 gives
// the unit eigenvector J P y.  T is applied by two dense products (G Y, then
// (W.W)(G Y), the squares formed on the fly) to a block Y of s = k + oversample
// vectors; each iteration performs a Rayleigh-Ritz step in the G inner product with
// two small symmetric eigenproblems (Jacobi, one CTA, FP64) and moves to T applied
// to the Ritz vectors (subspace iteration).  It stops when every top-k Ritz pair has a
// residual ||T x_i - theta_i x_i|| <= eig_tol theta_1 ||x_i||; T x_i is the next basis
// vector, so the check costs one pass over the block.  The embedding is
// Z = J P [y_1..y_k] diag(sqrt(max(theta, 0))) = P T_k - 1 (c^T T_k) / n.
//
// Precision: G, its centring and everything after it are FP64 (the centring cancels
// catastrophically along the ones vector).  The column sums and the Gram are summed in a
// fixed order (no atomics on values), so G is the same bit pattern on every run.
#include <algorithm>
#include <climits>
#include <memory>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace sbha {

namespace {

constexpr int SMAX = 32;       // largest subspace
constexpr int kGemmRows = 16;  // rows per CTA in the l x l by l x s products (32 CTAs at l = 500)
constexpr int kGemmK = 32;

__global__ void k_check_csr(int64_t n, int l, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int s = rowptr[i], e = rowptr[i + 1];
    if (e < s) {
      set_error(err, DERR_BAD_CSR);
      continue;
    }
    for (int a = s; a < e; ++a)
      if (col[a] < 0 || col[a] >= l) set_error(err, DERR_BAD_CSR);
  }
}

// c += P^T 1 ; G += P^T P   (warp per row, FP64 atomics: the last bits depend on scheduling).  Only the
// allocation-free sbha_mds_static uses it: the fixed-order Gram needs a transposed copy of P, whose size
// grows with n.
__global__ void k_gram(int64_t n, int l, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, double* __restrict__ c, double* __restrict__ G) {
  int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    int s = rowptr[i], e = rowptr[i + 1];
    for (int a0 = s; a0 < e; a0 += 32) {
      int a = a0 + lane;
      bool ok = a < e;
      int ca = ok ? col[a] : 0;
      double va = ok ? val[a] : 0.0;
      if (ok) atomicAdd(c + ca, va);
      for (int b0 = s; b0 < e; b0 += 32) {
        int bcnt = min(32, e - b0);
        int cb_l = (b0 + lane < e) ? col[b0 + lane] : 0;
        double vb_l = (b0 + lane < e) ? val[b0 + lane] : 0.0;
        for (int q = 0; q < bcnt; ++q) {
          int cb = __shfl_sync(0xffffffffu, cb_l, q);
          double vb = __shfl_sync(0xffffffffu, vb_l, q);
          if (ok) atomicAdd(G + static_cast<int64_t>(ca) * l + cb, va * vb);
        }
      }
    }
  }
}

// G_jk -= c_j c_k / n
__global__ void k_center(int l, double inv_n, const double* __restrict__ c, double* __restrict__ G) {
  int64_t total = static_cast<int64_t>(l) * l;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int j = static_cast<int>(q / l), k = static_cast<int>(q % l);
    G[q] -= (c[j] * c[k]) * inv_n;
  }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

__global__ void k_random_block(int l, int s, uint64_t seed, double* __restrict__ Y) {
  int64_t total = static_cast<int64_t>(l) * s;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
    Y[q] = static_cast<double>(splitmix64(seed ^ (static_cast<uint64_t>(q) * 0x2545f4914f6cdd1dull)) >> 11) *
               (2.0 / 9007199254740992.0) - 1.0;
}

// C[l x s] = alpha * op(A)[l x l] * B[l x s], op(A)_ij = A_ij or A_ij^2 (square = 1).  FP64.
__global__ void __launch_bounds__(256) k_gemm_ls(int l, int s, const double* __restrict__ A, int square,
                                                 const double* __restrict__ B, double* __restrict__ C, double alpha,
                                                 const int* __restrict__ conv_it, int it) {
  if (conv_it && *conv_it < it) return;
  __shared__ double As[kGemmRows][kGemmK + 1];
  __shared__ double Bs[kGemmK][SMAX];
  int r0 = blockIdx.x * kGemmRows;
  // thread t computes rows r0 + (t / s') ... : 256 threads cover 64 rows x s cols, (64*s)/256 outputs each
  int nout = (kGemmRows * s + 255) / 256;
  double acc[8];
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  for (int k0 = 0; k0 < l; k0 += kGemmK) {
    for (int q = threadIdx.x; q < kGemmRows * kGemmK; q += 256) {
      int rr = q / kGemmK, kk = q % kGemmK;
      int gr = r0 + rr, gk = k0 + kk;
      double a = (gr < l && gk < l) ? A[static_cast<int64_t>(gr) * l + gk] : 0.0;
      As[rr][kk] = square ? a * a : a;
    }
    for (int q = threadIdx.x; q < kGemmK * s; q += 256) {
      int kk = q / s, cc = q % s;
      int gk = k0 + kk;
      Bs[kk][cc] = gk < l ? B[static_cast<int64_t>(gk) * s + cc] : 0.0;
    }
    __syncthreads();
    for (int o = 0; o < nout; ++o) {
      int idx = threadIdx.x + o * 256;
      if (idx >= kGemmRows * s) break;
      int rr = idx / s, cc = idx % s;
      double a = acc[o];
#pragma unroll 8
      for (int kk = 0; kk < kGemmK; ++kk) a += As[rr][kk] * Bs[kk][cc];
      acc[o] = a;
    }
    __syncthreads();
  }
  for (int o = 0; o < nout; ++o) {
    int idx = threadIdx.x + o * 256;
    if (idx >= kGemmRows * s) break;
    int rr = idx / s, cc = idx % s;
    if (r0 + rr < l) C[static_cast<int64_t>(r0 + rr) * s + cc] = alpha * acc[o];
  }
}

// partial[b] = X^T Y over a tile of kGramRows rows, for two pairs: S = Y^T A1, H = A1^T A2 (s x s each)
constexpr int kGramRows = 32;
__global__ void __launch_bounds__(256) k_small_gram(int l, int s, const double* __restrict__ Y,
                                                    const double* __restrict__ A1, const double* __restrict__ A2,
                                                    double* __restrict__ part, const int* __restrict__ conv_it,
                                                    int it) {
  if (*conv_it < it) return;
  __shared__ double ys[kGramRows][SMAX], a1[kGramRows][SMAX], a2[kGramRows][SMAX];
  int r0 = blockIdx.x * kGramRows;
  for (int q = threadIdx.x; q < kGramRows * s; q += 256) {
    int rr = q / s, cc = q % s;
    int gr = r0 + rr;
    bool ok = gr < l;
    ys[rr][cc] = ok ? Y[static_cast<int64_t>(gr) * s + cc] : 0.0;
    a1[rr][cc] = ok ? A1[static_cast<int64_t>(gr) * s + cc] : 0.0;
    a2[rr][cc] = ok ? A2[static_cast<int64_t>(gr) * s + cc] : 0.0;
  }
  __syncthreads();
  double* out = part + static_cast<int64_t>(blockIdx.x) * 2 * s * s;
  for (int q = threadIdx.x; q < 2 * s * s; q += 256) {
    int which = q / (s * s), ij = q % (s * s), i = ij / s, j = ij % s;
    double acc = 0.0;
    if (which == 0)
      for (int rr = 0; rr < kGramRows; ++rr) acc += ys[rr][i] * a1[rr][j];
    else
      for (int rr = 0; rr < kGramRows; ++rr) acc += a1[rr][i] * a2[rr][j];
    out[q] = acc;
  }
}

// Cyclic Jacobi on a symmetric m x m matrix in shared memory (row-major, stride SMAX),
// parallel ordering: each round rotates m/2 disjoint index pairs.  V accumulates the rotations.
// A pair is rotated only while |a_pq| > eps sqrt(|a_pp a_qq|) (the relative threshold that keeps
// every eigenvalue to a few units of its own last place); the sweeps stop after one that rotated
// no pair, or after max_sweeps.
__device__ void block_jacobi(double (*A)[SMAX], double (*V)[SMAX], int m, double* cs, double* sn, int* pp, int* qq,
                             int max_sweeps) {
  int me = m + (m & 1);  // even count with a dummy index m if odd
  for (int q = threadIdx.x; q < SMAX * SMAX; q += blockDim.x) V[q / SMAX][q % SMAX] = (q / SMAX == q % SMAX) ? 1.0 : 0.0;
  __shared__ int s_rot;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < me - 1; ++round) {
      // round-robin pairing: fixed position 0, the others rotate
      if (threadIdx.x < me / 2) {
        int i = threadIdx.x;
        auto at = [&](int pos) { return pos == 0 ? 0 : 1 + ((pos - 1 + round) % (me - 1)); };
        int p = at(i), q = at(me - 1 - i);
        if (p > q) {
          int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[p][q];
          constexpr double eps = 2.220446049250313e-16;
          if (apq * apq > eps * eps * fabs(A[p][p] * A[q][q]) && apq != 0.0) {
            // t = tan(phi) of the annihilating rotation, t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)) with
            // theta = d / h, d = a_qq - a_pp, h = 2 a_pq, written as sgn(theta) |h| / (|d| + sqrt(d^2 + h^2)):
            // one square root and one division instead of two of each (the FP64 pipes are few)
            const double d = A[q][q] - A[p][p], h = 2.0 * apq;
            const bool pos = d == 0.0 || ((d > 0.0) == (h > 0.0));  // theta >= 0
            const double t = (pos ? 1.0 : -1.0) * fabs(h) / (fabs(d) + sqrt(d * d + h * h));
            c = rsqrt(t * t + 1.0);
            s = t * c;
            s_rot = 1;  // benign race: every writer stores 1
          } else {
            q = m;  // nothing to rotate in this pair
          }
        }
        pp[i] = p;
        qq[i] = q;
        cs[i] = c;
        sn[i] = s;
      }
      __syncthreads();
      // rows: (A_p., A_q.) <- (c A_p. - s A_q., s A_p. + c A_q.)
      for (int w = threadIdx.x; w < (me / 2) * m; w += blockDim.x) {
        int i = w / m, k = w % m;
        int p = pp[i], q = qq[i];
        if (q >= m) continue;
        double c = cs[i], s = sn[i];
        double ap = A[p][k], aq = A[q][k];
        A[p][k] = c * ap - s * aq;
        A[q][k] = s * ap + c * aq;
      }
      __syncthreads();
      // columns of A and V
      for (int w = threadIdx.x; w < (me / 2) * m; w += blockDim.x) {
        int i = w / m, k = w % m;
        int p = pp[i], q = qq[i];
        if (q >= m) continue;
        double c = cs[i], s = sn[i];
        double ap = A[k][p], aq = A[k][q];
        A[k][p] = c * ap - s * aq;
        A[k][q] = s * ap + c * aq;
        double vp = V[k][p], vq = V[k][q];
        V[k][p] = c * vp - s * vq;
        V[k][q] = s * vp + c * vq;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < me / 2; i += blockDim.x) {
        int p = pp[i], q = qq[i];
        if (q < m) {
          A[p][q] = 0.0;
          A[q][p] = 0.0;
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) break;  // read after the round's last barrier; reset only after the next one
    __syncthreads();
  }
}

// Rayleigh-Ritz in the G inner product (one CTA): S = U Sig U^T, H' = Sig^-1/2 U^T H U Sig^-1/2 = V Th V^T,
// Cm = U Sig^-1/2 V (columns by decreasing theta).
__global__ void __launch_bounds__(256) k_rayleigh_ritz(int s, int k, int nparts, const double* __restrict__ part,
                                                       double* __restrict__ Cm, double* __restrict__ theta,
                                                       const int* conv_it, int it, int* err) {
  if (*conv_it < it) return;
  __shared__ double S[SMAX][SMAX], H[SMAX][SMAX], U[SMAX][SMAX], V[SMAX][SMAX];
  __shared__ double cs[SMAX], sn[SMAX], sig[SMAX], th[SMAX];
  __shared__ int pp[SMAX], qq[SMAX], order[SMAX];
  for (int q = threadIdx.x; q < s * s; q += blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int p = 0; p < nparts; ++p) {
      a += part[static_cast<int64_t>(p) * 2 * s * s + q];
      b += part[static_cast<int64_t>(p) * 2 * s * s + s * s + q];
    }
    S[q / s][q % s] = a;
    H[q / s][q % s] = b;
  }
  __syncthreads();
  // symmetrise (rounding)
  for (int q = threadIdx.x; q < s * s; q += blockDim.x) {
    int i = q / s, j = q % s;
    if (i < j) {
      double a = 0.5 * (S[i][j] + S[j][i]);
      S[i][j] = S[j][i] = a;
      double b = 0.5 * (H[i][j] + H[j][i]);
      H[i][j] = H[j][i] = b;
    }
  }
  __syncthreads();
  block_jacobi(S, U, s, cs, sn, pp, qq, 40);
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < s; ++i) mx = fmax(mx, S[i][i]);
    int r = 0;
    for (int i = 0; i < s; ++i) {
      bool keep = S[i][i] > 1e-13 * mx && mx > 0.0;
      sig[i] = keep ? 1.0 / sqrt(S[i][i]) : 0.0;
      r += keep;
    }
    if (r < k) set_error(err, DERR_NOT_SPD);
  }
  __syncthreads();
  // H' = diag(sig) U^T H U diag(sig): first W = H U (into V as scratch), then U^T W
  for (int q = threadIdx.x; q < s * s; q += blockDim.x) {
    int i = q / s, j = q % s;
    double a = 0.0;
    for (int t = 0; t < s; ++t) a += H[i][t] * U[t][j];
    V[i][j] = a;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < s * s; q += blockDim.x) {
    int i = q / s, j = q % s;
    double a = 0.0;
    for (int t = 0; t < s; ++t) a += U[t][i] * V[t][j];
    H[i][j] = sig[i] * a * sig[j];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < s * s; q += blockDim.x) {
    int i = q / s, j = q % s;
    if (i < j) {
      double b = 0.5 * (H[i][j] + H[j][i]);
      H[i][j] = H[j][i] = b;
    }
  }
  __syncthreads();
  block_jacobi(H, V, s, cs, sn, pp, qq, 40);
  if (threadIdx.x == 0) {
    // order by decreasing theta; directions dropped from S (sig = 0) go last
    for (int i = 0; i < s; ++i) {
      order[i] = i;
      th[i] = H[i][i];
    }
    for (int i = 1; i < s; ++i) {
      int key = order[i];
      int q = i - 1;
      while (q >= 0 && th[order[q]] < th[key]) {
        order[q + 1] = order[q];
        --q;
      }
      order[q + 1] = key;
    }
    for (int i = 0; i < s; ++i) theta[i] = th[order[i]];
  }
  __syncthreads();
  // Cm[:, i] = U diag(sig) V[:, order[i]]
  for (int q = threadIdx.x; q < s * s; q += blockDim.x) {
    int a = q / s, i = q % s;
    int oi = order[i];
    double acc = 0.0;
    for (int t = 0; t < s; ++t) acc += U[a][t] * sig[t] * V[t][oi];
    Cm[a * s + i] = acc;
  }
}

// X = Y Cm (Ritz vectors) and Y = A2 Cm = T X (the next basis, and what the residual check reads)
__global__ void k_next_basis(int l, int s, double* __restrict__ Y, const double* __restrict__ A2,
                             const double* __restrict__ Cm, double* __restrict__ X, const int* conv_it, int it) {
  if (*conv_it < it) return;
  __shared__ double cm[SMAX * SMAX];
  for (int q = threadIdx.x; q < s * s; q += blockDim.x) cm[q] = Cm[q];
  __syncthreads();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < l; r += gridDim.x * blockDim.x) {
    double y[SMAX], a2[SMAX];
    for (int t = 0; t < s; ++t) {
      y[t] = Y[static_cast<int64_t>(r) * s + t];
      a2[t] = A2[static_cast<int64_t>(r) * s + t];
    }
    for (int i = 0; i < s; ++i) {
      double xv = 0.0, yv = 0.0;
      for (int t = 0; t < s; ++t) {
        xv += y[t] * cm[t * s + i];
        yv += a2[t] * cm[t * s + i];
      }
      X[static_cast<int64_t>(r) * s + i] = xv;
      Y[static_cast<int64_t>(r) * s + i] = yv;
    }
  }
}

// cT[q] = sum_j c_j T_jq, with T = X[:, :k] diag(sqrt(max(theta, 0)))  (one CTA)
__global__ void k_ct(int l, int s, int k, const double* __restrict__ c, const double* __restrict__ X,
                     const double* __restrict__ theta, double* __restrict__ T, double* __restrict__ cT) {
  __shared__ double red[256];
  for (int q = 0; q < k; ++q) {
    double sq = sqrt(fmax(theta[q], 0.0));
    double acc = 0.0;
    for (int j = threadIdx.x; j < l; j += blockDim.x) {
      double t = X[static_cast<int64_t>(j) * s + q] * sq;
      T[static_cast<int64_t>(j) * k + q] = t;
      acc += c[j] * t;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) cT[q] = red[0];
    __syncthreads();
  }
}

// Z_i = sum_a P_ia T_(col a) - cT / n
__global__ void k_embed(int64_t n, int k, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                        const double* __restrict__ val, const double* __restrict__ T, const double* __restrict__ cT,
                        double inv_n, double* __restrict__ Z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int q = 0; q < k; ++q) {
      double acc = 0.0;
      for (int a = rowptr[i]; a < rowptr[i + 1]; ++a) acc += val[a] * T[static_cast<int64_t>(col[a]) * k + q];
      Z[i * k + q] = acc - cT[q] * inv_n;
    }
  }
}

// Per column of Z: index of the largest |Z_iq| (lowest index on ties) -> flip sign if negative.
__global__ void k_sign_fix(int64_t n, int k, double* __restrict__ Z) {
  __shared__ double bv[32];
  __shared__ long long bi[32];
  __shared__ double s_sign;
  int q = blockIdx.x;
  double best = -1.0;
  long long arg = LLONG_MAX;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double a = fabs(Z[i * k + q]);
    if (a > best || (a == best && i < arg)) {
      best = a;
      arg = i;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    long long oa = __shfl_xor_sync(0xffffffffu, arg, o);
    if (ob > best || (ob == best && oa < arg)) {
      best = ob;
      arg = oa;
    }
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    bv[warp] = best;
    bi[warp] = arg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x / 32); ++w)
      if (bv[w] > best || (bv[w] == best && bi[w] < arg)) {
        best = bv[w];
        arg = bi[w];
      }
    s_sign = (arg < n && Z[arg * k + q] < 0.0) ? -1.0 : 1.0;
  }
  __syncthreads();
  if (s_sign < 0.0)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Z[i * k + q] = -Z[i * k + q];
}

// Ritz residuals of the top-k pairs (one CTA, fixed summation order): with X = Y Cm and TX = T X
// (the next basis), res[i] = ||TX_i - theta_i X_i|| / (|theta_1| ||X_i||).  Sets conv_it = it when
// every res[i] <= tol.
__global__ void __launch_bounds__(256) k_ritz_check(int l, int s, int k, const double* __restrict__ X,
                                                    const double* __restrict__ TX, const double* __restrict__ theta,
                                                    double* __restrict__ res, int* conv_it, int it, double tol) {
  if (*conv_it < it) return;
  __shared__ double num[256], den[256];
  __shared__ double s_worst;
  if (threadIdx.x == 0) s_worst = 0.0;
  const double scale = fmax(fabs(theta[0]), 1e-300);
  for (int q = 0; q < k; ++q) {
    double a = 0.0, b = 0.0;
    for (int j = threadIdx.x; j < l; j += blockDim.x) {
      double x = X[static_cast<int64_t>(j) * s + q];
      double r = TX[static_cast<int64_t>(j) * s + q] - theta[q] * x;
      a += r * r;
      b += x * x;
    }
    num[threadIdx.x] = a;
    den[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        num[threadIdx.x] += num[threadIdx.x + w];
        den[threadIdx.x] += den[threadIdx.x + w];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double rq = sqrt(num[0] / fmax(den[0], 1e-300)) / scale;
      res[q] = rq;
      s_worst = fmax(s_worst, rq);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_worst <= tol) *conv_it = it;
}

// ---------------------------------------------------------------- sBMDS (Lanczos) ----
//
// The vertex-space route of Sec. 3.3: the top-k eigenpairs of B = -1/2 J P WE P^T J (n x n, WE = W (.) W)
// by Lanczos with full orthogonalisation and thick restarts, touching B only through
// products: P^T (J x) = P^T x - mean(x) c and J (P s) = P s - (c.s / n) 1 with c = P^T 1.  The
// basis (at most SMAX vectors of n) and the dense projected matrix H = Q^T B Q are kept; on a
// restart the top k + 8 Ritz vectors and the last remainder direction form the new basis.

__global__ void k_col_count(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            int32_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int a = rowptr[i]; a < rowptr[i + 1]; ++a) atomicAdd(cnt + col[a], 1);
}

__global__ void k_col_fill(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const int32_t* __restrict__ tptr, int32_t* __restrict__ fill,
                           int32_t* __restrict__ trow, double* __restrict__ tval) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int a = rowptr[i]; a < rowptr[i + 1]; ++a) {
      int q = tptr[col[a]] + atomicAdd(fill + col[a], 1);
      trow[q] = static_cast<int32_t>(i);
      tval[q] = val[a];
    }
}

// y_r = sum_a v_a x_(c_a) over the rows of a CSR matrix (warp per row); mode 1 subtracts shift * sub_r
// (sub nullable), then scales by alpha.
__global__ void k_spmv(int64_t rows, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                       const double* __restrict__ v, const double* __restrict__ x, const double* __restrict__ sub,
                       const double* __restrict__ shift, double alpha, double* __restrict__ y) {
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w; r < rows; r += nw) {
    double a = 0.0;
    for (int e = ptr[r] + lane; e < ptr[r + 1]; e += 32) a += v[e] * x[idx[e]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) y[r] = alpha * (a - (shift ? *shift * (sub ? sub[r] : 1.0) : 0.0));
  }
}

// y = WE t, WE = W (.) W (dense l x l, warp per row)
__global__ void k_gemv_we(int l, const double* __restrict__ W, const double* __restrict__ t, double* __restrict__ y) {
  int lane = threadIdx.x & 31;
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = w; r < l; r += nw) {
    double a = 0.0;
    for (int j = lane; j < l; j += 32) {
      double d = W[static_cast<int64_t>(r) * l + j];
      a += d * d * t[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) y[r] = a;
  }
}

// out[q] (zeroed by the caller) += sum_i A[q][i] B[i] for q < nq, A column-major n x nq (one CTA row chunk)
__global__ void k_dots(int64_t n, int nq, const double* __restrict__ A, const double* __restrict__ b,
                       double scale_n, double* __restrict__ out) {
  __shared__ double red[SMAX + 1][8];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double acc[SMAX + 1];
#pragma unroll
  for (int q = 0; q < SMAX + 1; ++q) acc[q] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double bi = b[i];
#pragma unroll
    for (int q = 0; q < SMAX + 1; ++q)
      if (q < nq) acc[q] += A[q * n + i] * bi;
  }
#pragma unroll
  for (int q = 0; q < SMAX + 1; ++q) {
    double a = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[q][warp] = a;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    double a = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) a += red[threadIdx.x][w];
    atomicAdd(out + threadIdx.x, a * scale_n);
  }
}

// w -= sum_q A[q] h[q] (q < nq)
__global__ void k_sub_span(int64_t n, int nq, const double* __restrict__ A, const double* __restrict__ h,
                           double* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = w[i];
    for (int q = 0; q < nq; ++q) a -= A[q * n + i] * h[q];
    w[i] = a;
  }
}

// H[:, j] and H[j, :] from the two orthogonalisation passes h = h1 + h2 (j + 1 entries); beta = ||w||,
// q_(j+1) = w / beta when there is room.
__global__ void k_lz_column(int j, const double* __restrict__ h1, const double* __restrict__ h2,
                            const double* __restrict__ nrm2, double* __restrict__ H, double* __restrict__ beta) {
  int t = threadIdx.x;
  if (t <= j) {
    double v = h1[t] + h2[t];
    H[t * SMAX + j] = v;
    H[j * SMAX + t] = v;
  }
  if (t == 0) *beta = sqrt(fmax(*nrm2, 0.0));
}

__global__ void k_scale_into(int64_t n, const double* __restrict__ w, const double* __restrict__ beta,
                             double* __restrict__ q, double* __restrict__ H, int j) {
  double b = *beta;
  double inv = b > 0.0 ? 1.0 / b : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    q[i] = w[i] * inv;
  if (H && blockIdx.x == 0 && threadIdx.x == 0) {
    H[(j + 1) * SMAX + j] = b;
    H[j * SMAX + j + 1] = b;
  }
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

// Eigenpairs of the m x m projected matrix (one CTA): theta decreasing, S columns; res[i] =
// beta |S[m-1][i]| (the Ritz residual of pair i).
__global__ void __launch_bounds__(256) k_lz_ritz(int m, const double* __restrict__ Hg, const double* __restrict__ beta,
                                                 double* __restrict__ theta, double* __restrict__ S,
                                                 double* __restrict__ res) {
  __shared__ double A[SMAX][SMAX], V[SMAX][SMAX];
  __shared__ double cs[SMAX], sn[SMAX];
  __shared__ int pp[SMAX], qq[SMAX], order[SMAX];
  for (int q = threadIdx.x; q < SMAX * SMAX; q += blockDim.x) {
    int i = q / SMAX, jj = q % SMAX;
    A[i][jj] = (i < m && jj < m) ? 0.5 * (Hg[i * SMAX + jj] + Hg[jj * SMAX + i]) : 0.0;
  }
  __syncthreads();
  block_jacobi(A, V, m, cs, sn, pp, qq, 60);
  if (threadIdx.x == 0) {
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 1; i < m; ++i) {  // insertion sort by decreasing eigenvalue
      int o = order[i];
      int q = i - 1;
      while (q >= 0 && A[order[q]][order[q]] < A[o][o]) {
        order[q + 1] = order[q];
        --q;
      }
      order[q + 1] = o;
    }
  }
  __syncthreads();
  double b = *beta;
  for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
    int i = q / m, c = q % m;
    S[i * SMAX + c] = V[i][order[c]];
  }
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    theta[c] = A[order[c]][order[c]];
    res[c] = b * fabs(V[m - 1][order[c]]);
  }
}

// Qn[:, c] = sum_i Q[:, i] S[i][c] for c < p (Q column-major n x m)
__global__ void k_rotate_basis(int64_t n, int m, int p, const double* __restrict__ Q, const double* __restrict__ S,
                               double* __restrict__ Qn) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < p; ++c) {
      double a = 0.0;
      for (int i = 0; i < m; ++i) a += Q[i * n + r] * S[i * SMAX + c];
      Qn[c * n + r] = a;
    }
}

// After a thick restart: H = diag(theta_0 .. theta_(p-1)), the rest cleared
__global__ void k_restart_h(int p, const double* __restrict__ theta, double* __restrict__ H) {
  for (int q = threadIdx.x; q < SMAX * SMAX; q += blockDim.x) {
    int i = q / SMAX, j = q % SMAX;
    H[q] = (i == j && i < p) ? theta[i] : 0.0;
  }
}

// Z[:, q] = Q S[:, q] sqrt(max(theta_q, 0)), row-major n x k
__global__ void k_lz_embed(int64_t n, int m, int k, const double* __restrict__ Q, const double* __restrict__ S,
                           const double* __restrict__ theta, double* __restrict__ Z) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < k; ++c) {
      double a = 0.0;
      for (int i = 0; i < m; ++i) a += Q[i * n + r] * S[i * SMAX + c];
      Z[r * k + c] = a * sqrt(fmax(theta[c], 0.0));
    }
}

__global__ void k_random_vec(int64_t n, uint64_t seed, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h = splitmix64(seed ^ (0x9e3779b97f4a7c15ull * static_cast<uint64_t>(i + 1)));
    x[i] = static_cast<double>(h >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

// ------------------------------------------------------------ P^T, c and G ----
//
// G = (J P)^T (J P) = P^T P - c c^T / n without atomics on values, so that G is the same bit
// pattern on every run: P^T is built as CSR (column counts, prefix sum, fill), each column's
// entries are sorted by row, c_a is summed in that order, and row a of G is accumulated by one
// CTA from column a's entries in row order, each warp over a fixed contiguous part into its own
// shared-memory copy of the row; the copies are added in warp order in the epilogue, which also
// subtracts c_a c_b / n (FP64 centring).

constexpr int kSortCap = 8192;  // column segments sorted in shared memory; longer ones are ranked in global memory
constexpr size_t kSortSmem = kSortCap * (sizeof(int32_t) + sizeof(double));
constexpr int kGramWarps = 8;
constexpr int kGramTile = 2048;   // columns of G per pass (kGramWarps x kGramTile doubles of shared memory)
constexpr int kGramBatchK = 16;   // entries per row staged with a batch of 32 rows (more: read directly)
constexpr size_t kGramBatchBytes = static_cast<size_t>(kGramWarps) * 32 * kGramBatchK * (sizeof(double) + sizeof(int));

// (srow, sval) = each column segment of (trow, tval) in ascending row order (the rows of a column are
// distinct); c_a = the column's sum in that order.  One CTA per column.
__global__ void __launch_bounds__(256) k_col_sort(int l, const int32_t* __restrict__ tptr,
                                                  const int32_t* __restrict__ trow, const double* __restrict__ tval,
                                                  int32_t* __restrict__ srow, double* __restrict__ sval,
                                                  double* __restrict__ c) {
  extern __shared__ double sort_smem[];  // v[kSortCap] then key[kSortCap]
  double* v = sort_smem;
  int32_t* key = reinterpret_cast<int32_t*>(sort_smem + kSortCap);
  __shared__ double red[256];
  for (int a = blockIdx.x; a < l; a += gridDim.x) {
    const int s0 = tptr[a], len = tptr[a + 1] - s0;
    if (len <= kSortCap) {
      int np2 = 1;
      while (np2 < len) np2 <<= 1;
      for (int q = threadIdx.x; q < np2; q += blockDim.x) {
        key[q] = q < len ? trow[s0 + q] : INT_MAX;
        v[q] = q < len ? tval[s0 + q] : 0.0;
      }
      __syncthreads();
      for (int k = 2; k <= np2; k <<= 1)  // bitonic sort by row
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int q = threadIdx.x; q < np2; q += blockDim.x) {
            int p = q ^ j;
            if (p > q && ((key[q] > key[p]) == ((q & k) == 0))) {
              int32_t tk = key[q];
              key[q] = key[p];
              key[p] = tk;
              double tv = v[q];
              v[q] = v[p];
              v[p] = tv;
            }
          }
          __syncthreads();
        }
      for (int q = threadIdx.x; q < len; q += blockDim.x) {
        srow[s0 + q] = key[q];
        sval[s0 + q] = v[q];
      }
    } else {
      for (int q = threadIdx.x; q < len; q += blockDim.x) {  // rank by counting
        const int32_t r = trow[s0 + q];
        int rank = 0;
        for (int t = 0; t < len; ++t) rank += trow[s0 + t] < r;
        srow[s0 + rank] = r;
        sval[s0 + rank] = tval[s0 + q];
      }
    }
    __syncthreads();
    double acc = 0.0;  // thread t sums sorted positions t, t + 256, ...; then a fixed tree
    for (int q = threadIdx.x; q < len; q += blockDim.x) acc += sval[s0 + q];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) c[a] = red[0];
    __syncthreads();
  }
}

// Row a of G for every a (one CTA per row, kGramWarps warps): G_ab = sum over the rows i of column a
// (row order) of P_ia P_ib, minus (c_a c_b) / n.  Columns b in passes of `tile`.  Each warp takes a
// fixed contiguous part of column a's entries, in batches of 32 rows: one lane per row loads the row's
// entries into the warp's shared-memory batch (all 32 rows' loads in flight at once), then the warp
// adds the rows one after another, in row order, into its own shared-memory copy of row a.
__global__ void __launch_bounds__(kGramWarps * 32) k_gram_rows(int64_t n, int l, const int32_t* __restrict__ rowptr,
                                                               const int32_t* __restrict__ col,
                                                               const double* __restrict__ val,
                                                               const int32_t* __restrict__ tptr,
                                                               const int32_t* __restrict__ srow,
                                                               const double* __restrict__ sval,
                                                               const double* __restrict__ c, int tile,
                                                               double* __restrict__ G) {
  extern __shared__ double gw[];  // [kGramWarps][tile] rows, then the batches: values, then columns
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double nd = static_cast<double>(n);
  double* mine = gw + static_cast<int64_t>(warp) * tile;
  double* bval = gw + static_cast<int64_t>(kGramWarps) * tile + warp * 32 * kGramBatchK;
  int* bcol = reinterpret_cast<int*>(gw + static_cast<int64_t>(kGramWarps) * tile + kGramWarps * 32 * kGramBatchK) +
              warp * 32 * kGramBatchK;
  for (int a = blockIdx.x; a < l; a += gridDim.x) {
    const int s0 = tptr[a], len = tptr[a + 1] - s0;
    const int w0 = s0 + static_cast<int>(static_cast<int64_t>(len) * warp / kGramWarps);
    const int w1 = s0 + static_cast<int>(static_cast<int64_t>(len) * (warp + 1) / kGramWarps);
    const double ca = c[a];
    for (int b0 = 0; b0 < l; b0 += tile) {
      const int tb = min(tile, l - b0);
      for (int q = lane; q < tb; q += 32) mine[q] = 0.0;
      __syncwarp();
      for (int t0 = w0; t0 < w1; t0 += 32) {
        const int cnt = min(32, w1 - t0);
        double v = 0.0;
        int e0 = 0, e1 = 0;
        if (lane < cnt) {  // this lane's row of the batch: its P_ia and its entries
          const int i = srow[t0 + lane];
          v = sval[t0 + lane];
          e0 = rowptr[i];
          e1 = rowptr[i + 1];
          for (int e = e0; e < min(e1, e0 + kGramBatchK); ++e) {
            bcol[lane * kGramBatchK + (e - e0)] = col[e];
            bval[lane * kGramBatchK + (e - e0)] = val[e];
          }
        }
        __syncwarp();
        for (int j = 0; j < cnt; ++j) {  // rows in order; the entries of one row have distinct columns
          const double vj = __shfl_sync(0xffffffffu, v, j);
          const int f0 = __shfl_sync(0xffffffffu, e0, j), f1 = __shfl_sync(0xffffffffu, e1, j);
          for (int e = lane; e < f1 - f0; e += 32) {
            const bool stg = e < kGramBatchK;
            const int b = (stg ? bcol[j * kGramBatchK + e] : col[f0 + e]) - b0;
            const double vb = stg ? bval[j * kGramBatchK + e] : val[f0 + e];
            if (b >= 0 && b < tb) mine[b] += vj * vb;
          }
          __syncwarp();
        }
      }
      __syncthreads();
      for (int q = threadIdx.x; q < tb; q += blockDim.x) {
        double sum = 0.0;
        for (int w = 0; w < kGramWarps; ++w) sum += gw[static_cast<int64_t>(w) * tile + q];
        G[static_cast<int64_t>(a) * l + b0 + q] = sum - (ca * c[b0 + q]) / nd;
      }
      __syncthreads();
    }
  }
}

}  // namespace

// P^T as CSR with every column's rows ascending, and c = P^T 1 summed in that order (deterministic).
struct Transposed {
  int32_t* ptr = nullptr;  // [l + 1]
  int32_t* row = nullptr;  // [nnz]
  double* val = nullptr;   // [nnz]
  double* c = nullptr;     // [l]
  int64_t nnz = 0;
};

Transposed transpose_sorted(Ctx& c, int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col,
                            const double* val) {
  Transposed t;
  int32_t* cnt = c.zeros<int32_t>(l);
  k_col_count<<<grid_for(n, 256), 256, 0, c.stream>>>(n, rowptr, col, cnt);
  c.launched("col_count");
  t.ptr = c.alloc<int32_t>(l + 1);
  t.nnz = exclusive_scan(c, cnt, t.ptr, l);
  int32_t* fill = c.zeros<int32_t>(l);
  int32_t* trow = c.alloc<int32_t>(std::max<int64_t>(t.nnz, 1));
  double* tval = c.alloc<double>(std::max<int64_t>(t.nnz, 1));
  k_col_fill<<<grid_for(n, 256), 256, 0, c.stream>>>(n, rowptr, col, val, t.ptr, fill, trow, tval);
  c.launched("col_fill");
  t.row = c.alloc<int32_t>(std::max<int64_t>(t.nnz, 1));
  t.val = c.alloc<double>(std::max<int64_t>(t.nnz, 1));
  t.c = c.alloc<double>(l);
  static bool attr = false;
  if (!attr) {
    SBHA_CUDA(cudaFuncSetAttribute(k_col_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(kSortSmem)));
    attr = true;
  }
  k_col_sort<<<std::min<int>(l, 16 * num_sms()), 256, kSortSmem, c.stream>>>(l, t.ptr, trow, tval, t.row, t.val,
                                                                               t.c);
  c.launched("col_sort");
  for (void* p : {static_cast<void*>(cnt), static_cast<void*>(fill), static_cast<void*>(trow),
                  static_cast<void*>(tval)})
    c.free(p);
  return t;
}

// G = P^T P - c c^T / n (l x l, row-major) from the sorted transpose.
void centred_gram(Ctx& c, int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col, const double* val,
                  const Transposed& t, double* G) {
  const int tile = std::min<int>(l, kGramTile);
  const size_t smem = sizeof(double) * kGramWarps * tile + kGramBatchBytes;
  static bool attr = false;
  if (!attr) {
    SBHA_CUDA(cudaFuncSetAttribute(k_gram_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(sizeof(double) * kGramWarps * kGramTile + kGramBatchBytes)));
    attr = true;
  }
  k_gram_rows<<<std::min<int>(l, 64 * num_sms()), kGramWarps * 32, smem, c.stream>>>(n, l, rowptr, col, val, t.ptr,
                                                                                      t.row, t.val, t.c, tile, G);
  c.launched("gram");
}

MdsReport classical_scaling(Ctx& c, int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col,
                            const double* val, const double* W, int32_t k, const sbha_opts& o, double* Z,
                            double* evals) {
  if (o.eig_route == SBHA_EIG_LANCZOS) return classical_scaling_lanczos(c, n, l, rowptr, col, val, W, k, o, Z, evals);
  MdsReport rep;
  int s = std::min<int>(k + std::max(0, o.oversample), std::min<int>(l, SMAX));
  if (k < 1 || k > s) SBHA_THROW(SBHA_EINVAL, "k must satisfy 1 <= k <= min(l, 32) - oversample");
  k_check_csr<<<grid_for(n, 256), 256, 0, c.stream>>>(n, l, rowptr, col, c.d_err);
  c.launched("check_csr");
  c.check_device("mds");
  cudaEvent_t ev[3] = {};
  if (c.timing)
    for (cudaEvent_t& e : ev) SBHA_CUDA(cudaEventCreate(&e));
  if (c.timing) SBHA_CUDA(cudaEventRecord(ev[0], c.stream));
  Transposed pt = transpose_sorted(c, n, l, rowptr, col, val);
  double* cs = pt.c;
  double* G = c.alloc<double>(static_cast<size_t>(l) * l);
  if (c.timing) SBHA_CUDA(cudaEventRecord(ev[1], c.stream));
  centred_gram(c, n, l, rowptr, col, val, pt, G);
  if (c.timing) {  // the sorted transpose with c = P^T 1, then the Gram kernel alone
    SBHA_CUDA(cudaEventRecord(ev[2], c.stream));
    SBHA_CUDA(cudaEventSynchronize(ev[2]));
    float t01 = 0.f, t12 = 0.f;
    SBHA_CUDA(cudaEventElapsedTime(&t01, ev[0], ev[1]));
    SBHA_CUDA(cudaEventElapsedTime(&t12, ev[1], ev[2]));
    thread_stats().ms_transpose = t01;
    thread_stats().ms_gram = t12;
    thread_stats().p_nnz = pt.nnz;
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  c.free(pt.row);
  c.free(pt.val);
  double* Y = c.alloc<double>(static_cast<size_t>(l) * s);
  double* A1 = c.alloc<double>(static_cast<size_t>(l) * s);
  double* A2 = c.alloc<double>(static_cast<size_t>(l) * s);
  double* X = c.alloc<double>(static_cast<size_t>(l) * s);
  int nparts = (l + kGramRows - 1) / kGramRows;
  double* part = c.alloc<double>(static_cast<size_t>(nparts) * 2 * s * s);
  double* Cm = c.alloc<double>(static_cast<size_t>(s) * s);
  double* theta = c.alloc<double>(s);
  double* res = c.zeros<double>(k);
  int* conv_it = c.alloc<int>(1);
  int big = INT32_MAX;
  SBHA_CUDA(cudaMemcpyAsync(conv_it, &big, sizeof(int), cudaMemcpyHostToDevice, c.stream));
  k_random_block<<<grid_for(static_cast<int64_t>(l) * s, 256), 256, 0, c.stream>>>(l, s, o.seed, Y);
  c.launched("random_block");
  unsigned gg = static_cast<unsigned>((l + kGemmRows - 1) / kGemmRows);
  // the l x l x s products G Y and -1/2 (W.W) (G Y): on the tensor cores by exact slicing (the digits of
  // the constant operands G and W.W cut once), or on the FP64 pipes.  The sliced product is exact to
  // about K 2^-46 of |A||B| per entry, which at l = 2000 holds the Ritz residual near 1e-11: the
  // iteration therefore moves to the FP64 pipes once the residual is below kTcSwitch, and only FP64
  // products decide convergence below that.  AUTO takes the tensor cores from kTcMinL landmarks on
  // (below it the FP64 products are a few hundred microseconds and the sliced ones are not faster).
  constexpr double kTcSwitch = 1e-9;
  constexpr int kTcMinL = 4096;
  bool tc = o.dense_mode == SBHA_DENSE_TC || (o.dense_mode == SBHA_DENSE_AUTO && l >= kTcMinL);
  std::unique_ptr<TcConstProduct> tcG, tcW;
  if (tc) {
    tcG.reset(new TcConstProduct(c, l, G, false, s));
    tcW.reset(new TcConstProduct(c, l, W, true, s));
  }
  std::vector<double> hres(k);
  int max_it = std::max(1, o.eig_max_iter);
  int it = 0;
  int h_conv = INT32_MAX;
  const int check_every = 4;
  while (it < max_it) {
    int batch = std::min(check_every, max_it - it);
    for (int b = 0; b < batch; ++b, ++it) {
      if (tc) {  // (runs also in the few iterations of a batch after convergence; nothing reads them)
        tcG->times(Y, 1.0, A1);
        tcW->times(A1, -0.5, A2);
      } else {
        k_gemm_ls<<<gg, 256, 0, c.stream>>>(l, s, G, 0, Y, A1, 1.0, conv_it, it);
        c.launched("gemm_G");
        k_gemm_ls<<<gg, 256, 0, c.stream>>>(l, s, W, 1, A1, A2, -0.5, conv_it, it);
        c.launched("gemm_WE");
      }
      k_small_gram<<<nparts, 256, 0, c.stream>>>(l, s, Y, A1, A2, part, conv_it, it);
      c.launched("small_gram");
      k_rayleigh_ritz<<<1, 256, 0, c.stream>>>(s, k, nparts, part, Cm, theta, conv_it, it, c.d_err);
      c.launched("rayleigh_ritz");
      k_next_basis<<<grid_for(l, 128), 128, 0, c.stream>>>(l, s, Y, A2, Cm, X, conv_it, it);
      c.launched("next_basis");
      k_ritz_check<<<1, 256, 0, c.stream>>>(l, s, k, X, Y, theta, res, conv_it, it, o.eig_tol);
      c.launched("ritz_check");
    }
    SBHA_CUDA(cudaMemcpyAsync(&h_conv, conv_it, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    if (tc) SBHA_CUDA(cudaMemcpyAsync(hres.data(), res, sizeof(double) * k, cudaMemcpyDeviceToHost, c.stream));
    SBHA_CUDA(cudaStreamSynchronize(c.stream));
    if (h_conv != INT32_MAX) break;
    if (tc && *std::max_element(hres.begin(), hres.end()) < kTcSwitch) tc = false;  // FP64 from here on
  }
  c.check_device("mds");
  rep.converged = h_conv != INT32_MAX;
  rep.iterations = rep.converged ? h_conv + 1 : it;
  {  // Ritz residuals of the returned pairs, from the last check
    std::vector<double> hr(k);
    SBHA_CUDA(cudaMemcpyAsync(hr.data(), res, sizeof(double) * k, cudaMemcpyDeviceToHost, c.stream));
    SBHA_CUDA(cudaStreamSynchronize(c.stream));
    for (double v : hr) rep.residual = std::max(rep.residual, v);
  }
  double* T = c.alloc<double>(static_cast<size_t>(l) * k);
  double* cT = c.alloc<double>(k);
  k_ct<<<1, 256, 0, c.stream>>>(l, s, k, cs, X, theta, T, cT);
  c.launched("ct");
  k_embed<<<grid_for(n, 128), 128, 0, c.stream>>>(n, k, rowptr, col, val, T, cT, 1.0 / static_cast<double>(n), Z);
  c.launched("embed");
  k_sign_fix<<<k, 256, 0, c.stream>>>(n, k, Z);
  c.launched("sign_fix");
  SBHA_CUDA(cudaMemcpyAsync(evals, theta, sizeof(double) * k, cudaMemcpyDeviceToDevice, c.stream));
  return rep;
}

}  // namespace sbha

namespace sbha {

MdsReport classical_scaling_lanczos(Ctx& c, int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col,
                                    const double* val, const double* W, int32_t k, const sbha_opts& o, double* Z,
                                    double* evals) {
  MdsReport rep;
  const int m = static_cast<int>(std::min<int64_t>(SMAX, n));
  if (k < 1 || k > m - 10) SBHA_THROW(SBHA_EINVAL, "Lanczos scaling needs 1 <= k <= min(n, 32) - 10");
  const int p = k + 8;  // kept Ritz vectors on a restart; at least two new Lanczos steps per restart
  k_check_csr<<<grid_for(n, 256), 256, 0, c.stream>>>(n, l, rowptr, col, c.d_err);
  c.launched("check_csr");
  c.check_device("mds");
  // P^T as CSR over the l landmark columns, rows ascending, and c = P^T 1
  Transposed pt = transpose_sorted(c, n, l, rowptr, col, val);
  const int32_t* tptr = pt.ptr;
  const int32_t* trow = pt.row;
  const double* tval = pt.val;
  double* cs = pt.c;
  double* ones = c.alloc<double>(n);
  k_fill<<<grid_for(n, 256), 256, 0, c.stream>>>(n, 1.0, ones);
  c.launched("lz_ones");
  const unsigned gn = grid_for(n, 256), gw = grid_for(n * 32, 256), gl = grid_for(static_cast<int64_t>(l) * 32, 256);
  const unsigned gd = std::min<unsigned>(gn, 4 * num_sms());
  double* Q = c.alloc<double>(static_cast<size_t>(SMAX) * n);  // basis, column-major
  double* Qn = c.alloc<double>(static_cast<size_t>(SMAX) * n);
  double* w = c.alloc<double>(n);
  double* t = c.alloc<double>(l);
  double* sv = c.alloc<double>(l);
  double* scal = c.alloc<double>(4);  // [0] mean, [1] c.s / n, [2] ||w||^2
  double* h1 = c.alloc<double>(SMAX + 1);
  double* h2 = c.alloc<double>(SMAX + 1);
  double* H = c.zeros<double>(SMAX * SMAX);
  double* beta = c.zeros<double>(1);
  double* theta = c.alloc<double>(SMAX);
  double* S = c.alloc<double>(SMAX * SMAX);
  double* res = c.alloc<double>(SMAX);
  // y = -1/2 J P WE P^T J x
  auto apply_B = [&](const double* x, double* y) {
    SBHA_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * 2, c.stream));
    k_dots<<<gd, 256, 0, c.stream>>>(n, 1, ones, x, 1.0 / static_cast<double>(n), scal);
    c.launched("lz_mean");
    k_spmv<<<gl, 256, 0, c.stream>>>(l, tptr, trow, tval, x, cs, scal, 1.0, t);  // P^T x - mean(x) c
    c.launched("lz_spmv_t");
    k_gemv_we<<<gl, 256, 0, c.stream>>>(l, W, t, sv);
    c.launched("lz_gemv");
    k_dots<<<1, 256, 0, c.stream>>>(l, 1, cs, sv, 1.0 / static_cast<double>(n), scal + 1);
    c.launched("lz_cs");
    k_spmv<<<gw, 256, 0, c.stream>>>(n, rowptr, col, val, sv, nullptr, scal + 1, -0.5, y);
    c.launched("lz_spmv");
  };
  // w <- w - Q h over the first nq columns, twice, with the coefficients h1 + h2
  auto orthogonalise = [&](int nq) {
    SBHA_CUDA(cudaMemsetAsync(h1, 0, sizeof(double) * (SMAX + 1), c.stream));
    SBHA_CUDA(cudaMemsetAsync(h2, 0, sizeof(double) * (SMAX + 1), c.stream));
    k_dots<<<gd, 256, 0, c.stream>>>(n, nq, Q, w, 1.0, h1);
    c.launched("lz_dots");
    k_sub_span<<<gn, 256, 0, c.stream>>>(n, nq, Q, h1, w);
    c.launched("lz_sub");
    k_dots<<<gd, 256, 0, c.stream>>>(n, nq, Q, w, 1.0, h2);
    c.launched("lz_dots");
    k_sub_span<<<gn, 256, 0, c.stream>>>(n, nq, Q, h2, w);
    c.launched("lz_sub");
    SBHA_CUDA(cudaMemsetAsync(scal + 2, 0, sizeof(double), c.stream));
    k_dots<<<gd, 256, 0, c.stream>>>(n, 1, w, w, 1.0, scal + 2);
    c.launched("lz_norm");
  };
  // start: q0 = J x / ||J x||, x seeded
  k_random_vec<<<gn, 256, 0, c.stream>>>(n, o.seed, w);
  c.launched("lz_start");
  SBHA_CUDA(cudaMemsetAsync(scal, 0, sizeof(double), c.stream));
  k_dots<<<gd, 256, 0, c.stream>>>(n, 1, ones, w, 1.0 / static_cast<double>(n), scal);
  c.launched("lz_mean");
  k_sub_span<<<gn, 256, 0, c.stream>>>(n, 1, ones, scal, w);
  c.launched("lz_sub");
  SBHA_CUDA(cudaMemsetAsync(scal + 2, 0, sizeof(double), c.stream));
  k_dots<<<gd, 256, 0, c.stream>>>(n, 1, w, w, 1.0, scal + 2);
  c.launched("lz_norm");
  k_lz_column<<<1, 32, 0, c.stream>>>(-1, h1, h2, scal + 2, H, beta);  // beta = ||J x||
  c.launched("lz_beta");
  k_scale_into<<<gn, 256, 0, c.stream>>>(n, w, beta, Q, nullptr, -1);
  c.launched("lz_scale");
  int nb = 1;
  const int max_steps = std::max(m, o.eig_max_iter);
  std::vector<double> hres(SMAX), hth(SMAX);
  for (;;) {
    while (nb <= m) {  // B q_(nb-1), orthogonalised against the nb basis vectors
      apply_B(Q + static_cast<int64_t>(nb - 1) * n, w);
      orthogonalise(nb);
      k_lz_column<<<1, SMAX, 0, c.stream>>>(nb - 1, h1, h2, scal + 2, H, beta);
      c.launched("lz_column");
      ++rep.iterations;
      if (nb == m) break;
      k_scale_into<<<gn, 256, 0, c.stream>>>(n, w, beta, Q + static_cast<int64_t>(nb) * n, H, nb - 1);
      c.launched("lz_scale");
      ++nb;
    }
    k_lz_ritz<<<1, 256, 0, c.stream>>>(m, H, beta, theta, S, res);
    c.launched("lz_ritz");
    c.check_device("mds");
    SBHA_CUDA(cudaMemcpyAsync(hres.data(), res, sizeof(double) * m, cudaMemcpyDeviceToHost, c.stream));
    SBHA_CUDA(cudaMemcpyAsync(hth.data(), theta, sizeof(double) * m, cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    double worst = 0.0, scale = std::max(std::fabs(hth[0]), 1e-300);
    for (int i = 0; i < k; ++i) worst = std::max(worst, hres[i] / scale);
    rep.residual = worst;
    if (worst <= o.eig_tol) break;
    if (rep.iterations >= max_steps) {
      rep.converged = false;
      break;
    }
    // thick restart: the top p Ritz vectors, then the remainder direction
    k_rotate_basis<<<gn, 256, 0, c.stream>>>(n, m, p, Q, S, Qn);
    c.launched("lz_rotate");
    SBHA_CUDA(cudaMemcpyAsync(Q, Qn, sizeof(double) * p * n, cudaMemcpyDeviceToDevice, c.stream));
    k_restart_h<<<1, 256, 0, c.stream>>>(p, theta, H);
    c.launched("lz_restart");
    k_scale_into<<<gn, 256, 0, c.stream>>>(n, w, beta, Q + static_cast<int64_t>(p) * n, nullptr, -1);
    c.launched("lz_scale");
    nb = p + 1;
  }
  k_lz_embed<<<gn, 256, 0, c.stream>>>(n, m, k, Q, S, theta, Z);
  c.launched("lz_embed");
  k_sign_fix<<<k, 256, 0, c.stream>>>(n, k, Z);
  c.launched("sign_fix");
  SBHA_CUDA(cudaMemcpyAsync(evals, theta, sizeof(double) * k, cudaMemcpyDeviceToDevice, c.stream));
  return rep;
}

}  // namespace sbha

// --------------------------------------------- allocation-free scaling ---
//
// sbha_mds_static: the same landmark-space scaling as sbha_mds, for callers that
// must not allocate device memory during the call.  Its workspace is the fixed
// file-scope array below (every GPU that loads the library holds it until the
// process exits).  Host code cannot use the array's name as a device address, so the
// address is looked up once per device with cudaGetSymbolAddress and cached.

namespace sbha {
namespace {

constexpr int32_t kStaticMaxL = 1024;  // largest landmark count the fixed workspace holds
constexpr int kStaticMaxParts = (kStaticMaxL + kGramRows - 1) / kGramRows;
// doubles: G, c, Y, A1, A2, X, small-Gram partials, Cm, theta, T, cT, Ritz residuals
constexpr size_t kStaticDoubles = static_cast<size_t>(kStaticMaxL) * kStaticMaxL + kStaticMaxL +
                                  4 * static_cast<size_t>(kStaticMaxL) * SMAX +
                                  static_cast<size_t>(kStaticMaxParts) * 2 * SMAX * SMAX + SMAX * SMAX + SMAX +
                                  static_cast<size_t>(kStaticMaxL) * SMAX + 2 * SMAX;
constexpr size_t kStaticBytes = kStaticDoubles * sizeof(double) + 256;  // + device error word and iteration flag

__device__ __align__(256) unsigned char g_mds_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};

unsigned char* scratch_for_current_device() {
  int dev = 0;
  SBHA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) SBHA_THROW(SBHA_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    SBHA_CUDA(cudaGetSymbolAddress(&p, g_mds_scratch));
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  return g_scratch_addr[dev];
}

}  // namespace
}  // namespace sbha

extern "C" int sbha_mds_static(int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col, const double* val,
                               const double* W, int32_t k, const sbha_opts* opts, double* Z_out, double* evals_out,
                               void* stream) {
  using namespace sbha;
  thread_error().clear();
  thread_stats() = sbha_stats{};
  int64_t launches = 0;
  try {
    sbha_opts o;
    sbha_opts_default(&o);
    if (opts) o = *opts;
    if (n < 1 || l < 1 || k < 1 || !rowptr || !col || !val || !W || !Z_out || !evals_out)
      SBHA_THROW(SBHA_EINVAL, "bad mds arguments");
    if (l > kStaticMaxL)
      SBHA_THROW(SBHA_EINVAL, "sbha_mds_static holds at most " + std::to_string(kStaticMaxL) +
                                  " landmarks in its fixed workspace; use sbha_mds for larger l");
    if (o.oversample < 0 || o.eig_max_iter < 1 || !(o.eig_tol > 0.0))
      SBHA_THROW(SBHA_EINVAL, "eigensolver limits must be positive");
    if (o.eig_route != SBHA_EIG_LANDMARK)
      SBHA_THROW(SBHA_EINVAL, "sbha_mds_static runs the landmark-space route only; use sbha_mds for Lanczos");
    int s = std::min<int>(k + o.oversample, std::min<int>(l, SMAX));
    if (k > s) SBHA_THROW(SBHA_EINVAL, "k must satisfy 1 <= k <= min(l, 32) - oversample");
    for (const void* p : {static_cast<const void*>(rowptr), static_cast<const void*>(col),
                          static_cast<const void*>(val), static_cast<const void*>(W), static_cast<const void*>(Z_out),
                          static_cast<const void*>(evals_out)})
      if (!is_device_ptr(p)) SBHA_THROW(SBHA_EINVAL, "sbha_mds_static needs every array in device memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto launched = [&](const char* what) {
      ++launches;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) SBHA_THROW(SBHA_ECUDA, std::string("launch of ") + what + ": " + cudaGetErrorString(e));
    };
    // carve the fixed workspace
    unsigned char* base = scratch_for_current_device();
    double* d = reinterpret_cast<double*>(base);
    double* G = d;
    d += static_cast<size_t>(l) * l;
    double* cs = d;
    d += l;
    double* Y = d;
    d += static_cast<size_t>(l) * s;
    double* A1 = d;
    d += static_cast<size_t>(l) * s;
    double* A2 = d;
    d += static_cast<size_t>(l) * s;
    double* X = d;
    d += static_cast<size_t>(l) * s;
    int nparts = (l + kGramRows - 1) / kGramRows;
    double* part = d;
    d += static_cast<size_t>(nparts) * 2 * s * s;
    double* Cm = d;
    d += static_cast<size_t>(s) * s;
    double* theta = d;
    d += s;
    double* T = d;
    d += static_cast<size_t>(l) * k;
    double* cT = d;
    d += k;
    double* res = d;
    d += k;
    int* flags = reinterpret_cast<int*>(base + kStaticDoubles * sizeof(double));
    int* err = flags;
    int* conv_it = flags + 1;
    // everything that accumulates starts from zero; the rest is written before it is read
    SBHA_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    SBHA_CUDA(cudaMemsetAsync(cs, 0, sizeof(double) * l, st));
    SBHA_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * l * l, st));
    int big = INT32_MAX;
    SBHA_CUDA(cudaMemcpyAsync(conv_it, &big, sizeof(int), cudaMemcpyHostToDevice, st));
    k_check_csr<<<grid_for(n, 256), 256, 0, st>>>(n, l, rowptr, col, err);
    launched("check_csr");
    int herr = 0;
    SBHA_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SBHA_CUDA(cudaStreamSynchronize(st));
    if (herr) SBHA_THROW(SBHA_EINVAL, "malformed CSR input (column out of range or row too long)");
    k_gram<<<grid_for(n * 32, 256), 256, 0, st>>>(n, l, rowptr, col, val, cs, G);
    launched("gram");
    k_center<<<grid_for(static_cast<int64_t>(l) * l, 256), 256, 0, st>>>(l, 1.0 / static_cast<double>(n), cs, G);
    launched("center");
    k_random_block<<<grid_for(static_cast<int64_t>(l) * s, 256), 256, 0, st>>>(l, s, o.seed, Y);
    launched("random_block");
    unsigned gg = static_cast<unsigned>((l + kGemmRows - 1) / kGemmRows);
    int it = 0, h_conv = INT32_MAX;
    while (it < o.eig_max_iter) {
      int batch = std::min(4, o.eig_max_iter - it);
      for (int b = 0; b < batch; ++b, ++it) {
        k_gemm_ls<<<gg, 256, 0, st>>>(l, s, G, 0, Y, A1, 1.0, conv_it, it);
        launched("gemm_G");
        k_gemm_ls<<<gg, 256, 0, st>>>(l, s, W, 1, A1, A2, -0.5, conv_it, it);
        launched("gemm_WE");
        k_small_gram<<<nparts, 256, 0, st>>>(l, s, Y, A1, A2, part, conv_it, it);
        launched("small_gram");
        k_rayleigh_ritz<<<1, 256, 0, st>>>(s, k, nparts, part, Cm, theta, conv_it, it, err);
        launched("rayleigh_ritz");
        k_next_basis<<<grid_for(l, 128), 128, 0, st>>>(l, s, Y, A2, Cm, X, conv_it, it);
        launched("next_basis");
        k_ritz_check<<<1, 256, 0, st>>>(l, s, k, X, Y, theta, res, conv_it, it, o.eig_tol);
        launched("ritz_check");
      }
      SBHA_CUDA(cudaMemcpyAsync(&h_conv, conv_it, sizeof(int), cudaMemcpyDeviceToHost, st));
      SBHA_CUDA(cudaStreamSynchronize(st));
      if (h_conv != INT32_MAX) break;
    }
    SBHA_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SBHA_CUDA(cudaStreamSynchronize(st));
    if (herr) SBHA_THROW(SBHA_ENOCONV, "a small Gram matrix lost positive definiteness");
    bool converged = h_conv != INT32_MAX;
    k_ct<<<1, 256, 0, st>>>(l, s, k, cs, X, theta, T, cT);
    launched("ct");
    k_embed<<<grid_for(n, 128), 128, 0, st>>>(n, k, rowptr, col, val, T, cT, 1.0 / static_cast<double>(n), Z_out);
    launched("embed");
    k_sign_fix<<<k, 256, 0, st>>>(n, k, Z_out);
    launched("sign_fix");
    SBHA_CUDA(cudaMemcpyAsync(evals_out, theta, sizeof(double) * k, cudaMemcpyDeviceToDevice, st));
    double hres[SMAX];
    SBHA_CUDA(cudaMemcpyAsync(hres, res, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    SBHA_CUDA(cudaStreamSynchronize(st));
    sbha_stats& stats = thread_stats();
    stats.eig_iterations = converged ? h_conv + 1 : it;
    for (int q = 0; q < k; ++q) stats.eig_residual = std::max(stats.eig_residual, hres[q]);
    stats.kernel_launches = launches;
    if (!converged) {
      thread_error() = "subspace iteration reached eig_max_iter before eig_tol";
      return SBHA_ENOCONV;
    }
    return SBHA_OK;
  } catch (const Error& e) {
    thread_error() = e.msg;
    cudaGetLastError();
    thread_stats().kernel_launches = launches;
    return e.status;
  } catch (const std::exception& e) {
    thread_error() = e.what();
    return SBHA_ECUDA;
  }
}
