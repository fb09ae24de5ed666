// The FMDS interpolation matrix from the biharmonic one (Sec. 3.4.2):
//   H = P (M_bb + mu I + M_bu P_u)^{-1} mu,
// which lets the landmark values deviate by an amount that mu controls.  The landmark rows of P are
// e_j, so the l x l matrix is S = (M P)_(b,:) + mu I: one CTA per landmark row gathers the rows of P
// that row b of M touches (its 2-ring).  S is SPD (a Schur complement of the SPD M, plus mu I), so
// mu S^{-1} comes from the library's blocked Cholesky, and H = P (mu S^{-1}) is an n x l x l FP64
// product on the landmark-space engine (tensor cores or FP64 pipes, as opts->dense_mode says).
#include "internal.cuh"

namespace sbha {

namespace {

// S[i][j] = sum_e M[b, c_e] P[c_e][j] + mu [i == j], b = idx[i]
__global__ void k_fmds_s(int32_t l, const int32_t* __restrict__ idx, const int32_t* __restrict__ rowptr,
                         const int32_t* __restrict__ col, const double* __restrict__ val,
                         const double* __restrict__ P, double mu, double* __restrict__ S) {
  const int i = blockIdx.x;
  const int b = idx[i];
  for (int j = threadIdx.x; j < l; j += blockDim.x) {
    double a = 0.0;
    for (int e = rowptr[b]; e < rowptr[b + 1]; ++e) a += val[e] * P[static_cast<int64_t>(col[e]) * l + j];
    S[static_cast<int64_t>(i) * l + j] = a + (i == j ? mu : 0.0);
  }
}

__global__ void k_scaled_identity(int32_t l, double mu, double* __restrict__ X) {
  const int64_t total = static_cast<int64_t>(l) * l;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
    X[q] = (q / l == q % l) ? mu : 0.0;
}

}  // namespace

void fmds_interpolation(Ctx& c, const DevCSR& M, const int32_t* idx, int32_t l, const double* P, double mu,
                        const sbha_opts& o, double* H) {
  double* S = c.alloc<double>(static_cast<size_t>(l) * l);
  k_fmds_s<<<l, 256, 0, c.stream>>>(l, idx, M.rowptr, M.col, M.val, P, mu, S);
  c.launched("fmds_s");
  double* Lc = cholesky(c, l, S);
  double* X = S;  // mu S^{-1}, in place of S
  k_scaled_identity<<<grid_for(static_cast<int64_t>(l) * l, 256), 256, 0, c.stream>>>(l, mu, X);
  c.launched("scaled_identity");
  cholesky_solve(c, l, Lc, X, l);
  if (o.dense_mode == SBHA_DENSE_FP64)
    dgemm_rowmajor(c, M.rows, l, l, P, X, H);
  else
    dgemm_tc_rowmajor(c, M.rows, l, l, P, X, H);
}

}  // namespace sbha
