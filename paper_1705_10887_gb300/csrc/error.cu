// Sampled relative error of the BHA approximation K~ = P W P^T (Eq. 9) as Sec. 4.1 measures it:
// eps = ||K~ - K||_F^2 / ||K||_F^2, estimated on a subset S of rows when K is too large to hold.
//
// Two passes, FP64 throughout:
//   1. T = P_S W' (|S| x l, row-major), W' = W or W (.) W: a CTA per sampled row, a thread per
//      column of W, the row's few nonzeros broadcast from the CSR;
//   2. a thread per vertex v keeps row v of P in registers and, for every sampled row s, forms
//      K~_sv = sum_e P_ve T[s][c_e] (the row of T is a few KB and stays in L1), reads the exact
//      K_sv (coalesced over v) and accumulates (K~_sv - K'_sv)^2 and K'_sv^2; a CTA reduction
//      and one FP64 atomic per CTA give the two sums.
// The work is |S| * nnz(P) multiply-adds; K_S is read once.
#include <algorithm>

#include "internal.cuh"

namespace sbha {

namespace {

constexpr int kErrThreads = 256;
constexpr int kRegEntries = 16;  // nonzeros of a row of P kept in registers (longer rows read memory)

// CSR columns in [0, l) with non-decreasing row pointers; sampled rows in [0, n).
__global__ void k_err_check(int64_t n, int32_t l, int32_t ns, const int32_t* __restrict__ rows,
                            const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            int* __restrict__ err) {
  const int64_t items = n > ns ? n : ns;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < items;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      if (rowptr[i + 1] < rowptr[i]) atomicExch(err, DERR_BAD_CSR);
      for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (col[e] < 0 || col[e] >= l) atomicExch(err, DERR_BAD_CSR);
    }
    if (i < ns && (rows[i] < 0 || rows[i] >= n)) atomicExch(err, DERR_BAD_INDEX);
  }
}

// T[s][c] = sum_e P[rows[s], e] W'[e][c]
__global__ void k_rows_times_w(int32_t l, const int32_t* __restrict__ rows, const int32_t* __restrict__ rowptr,
                               const int32_t* __restrict__ col, const double* __restrict__ val,
                               const double* __restrict__ W, int squared, double* __restrict__ T) {
  const int s = blockIdx.x;
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= l) return;
  const int r = rows[s];
  double a = 0.0;
  for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
    double w = W[static_cast<int64_t>(col[e]) * l + c];
    a += val[e] * (squared ? w * w : w);
  }
  T[static_cast<int64_t>(s) * l + c] = a;
}

__global__ void __launch_bounds__(kErrThreads) k_bha_err(int64_t n, int32_t ns, int32_t l,
                                                          const int32_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col,
                                                          const double* __restrict__ val,
                                                          const double* __restrict__ T,
                                                          const double* __restrict__ K, int squared,
                                                          double* __restrict__ acc) {
  __shared__ double red[2][kErrThreads / 32];
  double num = 0.0, den = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int e0 = rowptr[v], ne = rowptr[v + 1] - e0;
    int kc[kRegEntries];
    double kv[kRegEntries];
#pragma unroll
    for (int q = 0; q < kRegEntries; ++q) {
      kc[q] = q < ne ? col[e0 + q] : 0;
      kv[q] = q < ne ? val[e0 + q] : 0.0;
    }
    for (int s = 0; s < ns; ++s) {
      const double* Ts = T + static_cast<int64_t>(s) * l;
      double kt = 0.0;
#pragma unroll
      for (int q = 0; q < kRegEntries; ++q)
        if (q < ne) kt += kv[q] * Ts[kc[q]];
      for (int q = kRegEntries; q < ne; ++q) kt += val[e0 + q] * Ts[col[e0 + q]];
      double k = K[static_cast<int64_t>(s) * n + v];
      if (squared) k *= k;
      const double d = kt - k;
      num += d * d;
      den += k * k;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = num;
    red[1][warp] = den;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int w = 0; w < kErrThreads / 32; ++w) t += red[threadIdx.x][w];
    atomicAdd(acc + threadIdx.x, t);
  }
}

}  // namespace

void bha_error(Ctx& c, int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col, const double* val,
               const double* W, int32_t ns, const int32_t* rows, const double* K_rows, int squared, double* acc) {
  SBHA_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(double), c.stream));
  k_err_check<<<grid_for(std::max<int64_t>(n, ns), kErrThreads), kErrThreads, 0, c.stream>>>(n, l, ns, rows, rowptr,
                                                                                             col, c.d_err);
  c.launched("err_check");
  c.check_device("bha_error");
  if (ns == 0) return;
  // sampled rows in slices whose T (|S| x l) stays within 256 MB
  const int32_t slice = static_cast<int32_t>(std::max<int64_t>(1, std::min<int64_t>(ns, (32ll << 20) / l)));
  double* T = c.alloc<double>(static_cast<size_t>(slice) * l);
  for (int32_t s0 = 0; s0 < ns; s0 += slice) {
    const int32_t cnt = std::min(slice, ns - s0);
    dim3 g1(static_cast<unsigned>(cnt), static_cast<unsigned>((l + kErrThreads - 1) / kErrThreads));
    k_rows_times_w<<<g1, kErrThreads, 0, c.stream>>>(l, rows + s0, rowptr, col, val, W, squared, T);
    c.launched("rows_times_w");
    k_bha_err<<<grid_for(n, kErrThreads), kErrThreads, 0, c.stream>>>(n, cnt, l, rowptr, col, val, T,
                                                                      K_rows + static_cast<int64_t>(s0) * n, squared,
                                                                      acc);
    c.launched("bha_err");
  }
}

}  // namespace sbha
