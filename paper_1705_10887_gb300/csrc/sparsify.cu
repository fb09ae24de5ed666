// Thresholding of the interpolation operator (Sec. 3.1, Eq. 8).
//
// Row mode: every non-landmark row keeps its min(p_row, l) entries of largest
// magnitude (ties: smaller column).  The solve produces the columns a chunk at a
// time, so each row carries a running selection that is merged with the next
// chunk's values: a warp owns a row, each lane holds a few candidates in registers
// and the warp extracts the best candidate `keep` times (warp-wide argmax on
// (|v|, -column)).  No dense n x l operator is ever stored.
//
// Column mode (Eq. 8 read literally): column j keeps the p largest-magnitude entries
// over the non-landmark rows (ties: smaller row), p = round((n - l) p_row / l).  A CTA
// owns a column: an 8-bit-digit radix select on the magnitude bits finds the p-th
// largest magnitude, then an ordered block compaction emits the chosen rows in
// ascending row order.
//
// Magnitudes are compared as doubles (or as the bits of |v|, which order the same),
// so the selection is exact for the given values.
#include <cfloat>
#include <climits>

#include "internal.cuh"

namespace sbha {

namespace {

constexpr int BW = 32;
constexpr int kMaxBlocks = 16;  // 512 columns per chunk
constexpr int kMaxKeep = 128;  // p_row at most
constexpr int kMaxCand = kMaxBlocks + kMaxKeep / 32;  // candidates per lane: a chunk row and the kept share

// Selection order of the row mode: larger magnitude, then smaller column.  The magnitudes compare
// as integers (no FP64 compare on the few FP64 pipes): the bits of |v| order like |v|, a NaN keys
// below every number and kEmptyKey below everything.
constexpr long long kEmptyKey = LLONG_MIN;
__device__ __forceinline__ long long row_key(double v) {
  const long long a = __double_as_longlong(v) & 0x7fffffffffffffffLL;
  return a > 0x7ff0000000000000LL ? -1LL : a;
}
__device__ __forceinline__ bool beats_bits(long long ka, int ca, long long kb, int cb) {
  return ka > kb || (ka == kb && ca < cb);
}

__global__ void k_topk_rows(int64_t m, int nb, int j0, int ncols, const double* __restrict__ X, int keep,
                            double* __restrict__ topv, int32_t* __restrict__ topc, int first) {
  int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < m; u += nwarps) {
    // fixed slots, so that the candidates stay in registers: slots 0..3 the kept entries lane, lane + 32,
    // ...; slot 4 + cb the chunk's column block cb; `live` marks the slots holding a candidate not yet
    // taken
    double v[kMaxCand];
    int c[kMaxCand];
    unsigned live = 0;
#pragma unroll
    for (int t = 0; t < kMaxKeep / 32; ++t) {
      const int i = lane + 32 * t;
      const bool on = !first && i < keep;
      v[t] = on ? topv[u * keep + i] : 0.0;
      c[t] = on ? topc[u * keep + i] : INT_MAX;
      if (on) live |= 1u << t;
    }
#pragma unroll
    for (int cb = 0; cb < kMaxBlocks; ++cb) {
      const int t = kMaxKeep / 32 + cb;
      const int cc = cb * BW + lane;
      const bool on = cb < nb && cc < ncols;
      v[t] = on ? X[(static_cast<int64_t>(cb) * m + u) * BW + lane] : 0.0;
      c[t] = on ? j0 + cc : INT_MAX;
      if (on) live |= 1u << t;
    }
    for (int r = 0; r < keep; ++r) {
      long long bk = kEmptyKey;
      double bv = 0.0;
      int bc = INT_MAX, bi = -1;
#pragma unroll
      for (int i = 0; i < kMaxCand; ++i) {
        if (!((live >> i) & 1u)) continue;
        const long long k = row_key(v[i]);
        if (beats_bits(k, c[i], bk, bc)) {
          bk = k;
          bc = c[i];
          bv = v[i];
          bi = i;
        }
      }
      int wl = lane;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        int oc = __shfl_xor_sync(0xffffffffu, bc, o);
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int ol = __shfl_xor_sync(0xffffffffu, wl, o);
        if (beats_bits(ok, oc, bk, bc) || (ok == bk && oc == bc && ol < wl)) {
          bk = ok;
          bc = oc;
          bv = ov;
          wl = ol;
        }
      }
      if (wl == lane && bi >= 0) live &= ~(1u << bi);
      if (lane == 0) {
        topv[u * keep + r] = bv;
        topc[u * keep + r] = bc;
      }
    }
  }
}

__global__ void k_row_counts(int64_t n, const int32_t* __restrict__ lmcol, int keep, int32_t* __restrict__ cnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    cnt[v] = lmcol[v] >= 0 ? 1 : keep;
}

__global__ void k_rows_fill(int64_t n, const int32_t* __restrict__ lmcol, const int32_t* __restrict__ uidx, int keep,
                            const double* __restrict__ topv, const int32_t* __restrict__ topc,
                            const int32_t* __restrict__ rowptr, int32_t* __restrict__ col, double* __restrict__ val) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int base = rowptr[v];
    if (lmcol[v] >= 0) {
      col[base] = lmcol[v];
      val[base] = 1.0;
      continue;
    }
    int64_t u = uidx[v];
    int cs[kMaxKeep];
    double vs[kMaxKeep];
    for (int i = 0; i < keep; ++i) {
      int key = topc[u * keep + i];
      double kv = topv[u * keep + i];
      int q = i - 1;
      while (q >= 0 && cs[q] > key) {
        cs[q + 1] = cs[q];
        vs[q + 1] = vs[q];
        --q;
      }
      cs[q + 1] = key;
      vs[q + 1] = kv;
    }
    for (int i = 0; i < keep; ++i) {
      col[base + i] = cs[i];
      val[base + i] = vs[i];
    }
  }
}

// --------------------------------------------------------- column mode ----

constexpr int kSelThreads = 512;

__device__ __forceinline__ unsigned long long mag_bits(double v) {
  return isnan(v) ? 0ull : static_cast<unsigned long long>(__double_as_longlong(fabs(v)));
}

// Block-wide exclusive scan of one int per thread; returns the prefix, total in *tot.
__device__ int block_scan(int x, int* sh, int* tot) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < (int)(blockDim.x >> 5)) sh[lane] = w;
  }
  __syncthreads();
  int pre = inc - x + (warp > 0 ? sh[warp - 1] : 0);
  *tot = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return pre;
}

// One CTA per column of the chunk: the p largest |X| over rows (ties: the row visited first in
// the order ord, nullable: ascending), output in that order.
__global__ void __launch_bounds__(kSelThreads) k_topk_col(int64_t m, int j0, const double* __restrict__ X, int p,
                                                           const int32_t* __restrict__ ord, double* __restrict__ cval,
                                                           int32_t* __restrict__ crow) {
  __shared__ int hist[256];
  __shared__ int sh[32];
  __shared__ unsigned long long s_prefix;
  __shared__ int s_need;
  int c = blockIdx.x;
  int cb = c / BW, lane = c % BW;
  const double* xc = X + static_cast<int64_t>(cb) * m * BW + lane;
  unsigned long long prefix = 0, mask = 0;
  int need = p;  // how many of the entries matching `prefix` (in the current digit) we still need
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int64_t u = threadIdx.x; u < m; u += blockDim.x) {
      unsigned long long k = mag_bits(xc[u * BW]);
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 0xff], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0, d = 255;
      for (; d > 0; --d) {
        if (acc + hist[d] >= need) break;
        acc += hist[d];
      }
      s_prefix = prefix | (static_cast<unsigned long long>(d) << shift);
      s_need = need - acc;
    }
    __syncthreads();
    prefix = s_prefix;
    need = s_need;
    mask |= 0xffull << shift;
    __syncthreads();
  }
  // prefix = bits of the p-th largest magnitude; `need` entries equal to it are taken (lowest rows first)
  unsigned long long thr = prefix;
  int running = 0, eq_taken = 0;
  for (int64_t base = 0; base < m; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t u = i < m ? (ord ? ord[i] : i) : m;
    unsigned long long k = u < m ? mag_bits(xc[u * BW]) : 0ull;
    int is_eq = (u < m && k == thr) ? 1 : 0;
    int tot_eq;
    int eq_rank = block_scan(is_eq, sh, &tot_eq) + eq_taken;
    int sel = (u < m && (k > thr || (is_eq && eq_rank < need))) ? 1 : 0;
    int tot;
    int pos = block_scan(sel, sh, &tot) + running;
    if (sel) {
      crow[static_cast<int64_t>(j0 + c) * p + pos] = static_cast<int32_t>(u);
      cval[static_cast<int64_t>(j0 + c) * p + pos] = xc[u * BW];
    }
    running += tot;
    eq_taken += tot_eq;
  }
}

__global__ void k_col_counts(int l, int p, const int32_t* __restrict__ crow, const int32_t* __restrict__ uvert,
                             int32_t* __restrict__ cnt) {
  int64_t total = static_cast<int64_t>(l) * p;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[uvert[crow[q]]], 1);
}

__global__ void k_col_landmark_counts(int64_t n, const int32_t* __restrict__ lmcol, int32_t* __restrict__ cnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (lmcol[v] >= 0) cnt[v] = 1;
}

__global__ void k_col_scatter(int64_t n, int l, int p, const int32_t* __restrict__ crow,
                              const double* __restrict__ cval, const int32_t* __restrict__ uvert,
                              const int32_t* __restrict__ lmcol, const int32_t* __restrict__ rowptr,
                              int32_t* __restrict__ cursor, int32_t* __restrict__ col, double* __restrict__ val) {
  int64_t total = static_cast<int64_t>(l) * p;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int v = uvert[crow[q]];
    int pos = rowptr[v] + atomicAdd(&cursor[v], 1);
    col[pos] = static_cast<int32_t>(q / p);
    val[pos] = cval[q];
  }
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (lmcol[v] >= 0) {
      col[rowptr[v]] = lmcol[v];
      val[rowptr[v]] = 1.0;
    }
}

// Sort each row's entries by column (rows of the column-mode operator are short).
__global__ void k_sort_rows(int64_t n, const int32_t* __restrict__ rowptr, int32_t* __restrict__ col,
                            double* __restrict__ val) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int s = rowptr[v], e = rowptr[v + 1];
    for (int i = s + 1; i < e; ++i) {
      int key = col[i];
      double kv = val[i];
      int q = i - 1;
      while (q >= s && col[q] > key) {
        col[q + 1] = col[q];
        val[q + 1] = val[q];
        --q;
      }
      col[q + 1] = key;
      val[q + 1] = kv;
    }
  }
}

}  // namespace

void topk_rows_merge(Ctx& c, int64_t m, int C, int j0, int ncols, const double* X, int keep, double* topv,
                     int32_t* topc, int first_chunk) {
  if (keep > kMaxKeep) SBHA_THROW(SBHA_EINVAL, "p_row above 128 is not supported");
  k_topk_rows<<<grid_for(m * 32, 256), 256, 0, c.stream>>>(m, C / BW, j0, ncols, X, keep, topv, topc, first_chunk);
  c.launched("topk_rows");
}

void assemble_rows_csr(Ctx& c, int64_t n, int32_t l, const int32_t* lmcol, const int32_t* uidx, int keep,
                       const double* topv, const int32_t* topc, int32_t* rowptr, int32_t* col, double* val) {
  (void)l;
  int32_t* cnt = c.alloc<int32_t>(n);
  k_row_counts<<<grid_for(n, 256), 256, 0, c.stream>>>(n, lmcol, keep, cnt);
  c.launched("row_counts");
  exclusive_scan(c, cnt, rowptr, n);
  k_rows_fill<<<grid_for(n, 128), 128, 0, c.stream>>>(n, lmcol, uidx, keep, topv, topc, rowptr, col, val);
  c.launched("rows_fill");
  c.free(cnt);
}

void topk_cols(Ctx& c, int64_t m, int C, int j0, int ncols, const double* X, int p, const int32_t* ord, double* cval,
               int32_t* crow) {
  (void)C;
  k_topk_col<<<ncols, kSelThreads, 0, c.stream>>>(m, j0, X, p, ord, cval, crow);
  c.launched("topk_col");
}

int64_t assemble_cols_csr(Ctx& c, int64_t n, int32_t l, const int32_t* lmcol, const int32_t* uvert, int p,
                          const double* cval, const int32_t* crow, int32_t* rowptr, int32_t* col, double* val,
                          int64_t cap) {
  int32_t* cnt = c.zeros<int32_t>(n);
  k_col_landmark_counts<<<grid_for(n, 256), 256, 0, c.stream>>>(n, lmcol, cnt);
  c.launched("col_landmark_counts");
  if (crow) {
    k_col_counts<<<grid_for(static_cast<int64_t>(l) * p, 256), 256, 0, c.stream>>>(l, p, crow, uvert, cnt);
    c.launched("col_counts");
  }
  int64_t nnz = exclusive_scan(c, cnt, rowptr, n);
  if (nnz > cap) SBHA_THROW(SBHA_EINVAL, "operator capacity too small");
  SBHA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, c.stream));
  int64_t items = crow ? static_cast<int64_t>(l) * p : 0;
  k_col_scatter<<<grid_for(items > n ? items : n, 256), 256, 0, c.stream>>>(n, crow ? l : 0, p, crow, cval, uvert,
                                                                            lmcol, rowptr, cnt, col, val);
  c.launched("col_scatter");
  k_sort_rows<<<grid_for(n, 128), 128, 0, c.stream>>>(n, rowptr, col, val);
  c.launched("sort_rows");
  c.free(cnt);
  return nnz;
}

}  // namespace sbha
