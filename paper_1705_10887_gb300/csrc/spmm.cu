// Sparse matrix x block of vectors, staged through shared memory.
//
// The block-CG solves multiply a sparse SPD matrix (7 entries per row for L_uu, ~19 for
// M_uu) with m x C blocks of vectors stored as C/32 column blocks of m rows x 32 values.
// Reading neighbour rows straight from global memory gathers every row about (entries per
// row) times through L1/L2.  The unknowns are numbered along a Morton curve through the
// vertex positions (locality_order), so that kTileRows consecutive rows form a compact
// surface patch and its neighbours lie in a thin ring around it (the tile's halo, ~1.4x
// the tile for the one-ring pattern of L_uu).  For each pass over 256 bytes of columns (two
// FP32 or one FP64 column block) a CTA copies the halo rows into shared memory with
// asynchronous 16-byte copies, together with the tile's row pointers, local column indices
// and values, then every warp computes its rows from shared memory and writes them once,
// coalesced.  A tile whose halo exceeds kHaloCap rows reads its neighbours from global
// memory instead.
#include <algorithm>
#include <climits>

#include "internal.cuh"
#include "spmm.cuh"

namespace sbha {

namespace {

constexpr int R = kTileRows;
constexpr int CAP = kHaloCap;
constexpr int NT = kTileThreads;
constexpr int NW = NT / 32;
constexpr int kRowBytes = 256;  // staged bytes per row and pass
constexpr int kCand = 4096;     // entries per tile the halo builder can sort (more: unstaged tile)
constexpr int kSortChunk = 2048;

// ------------------------------------------------------------------ Morton order ----

__global__ void k_bbox(int64_t m, const int32_t* __restrict__ vert, const double* __restrict__ xyz,
                       double* __restrict__ box) {
  __shared__ double red[6][NT];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t u = threadIdx.x; u < m; u += NT) {
    int64_t v = vert ? vert[u] : u;
    for (int a = 0; a < 3; ++a) {
      double p = xyz[3 * v + a];
      lo[a] = fmin(lo[a], p);
      hi[a] = fmax(hi[a], p);
    }
  }
  for (int a = 0; a < 3; ++a) {
    red[a][threadIdx.x] = lo[a];
    red[3 + a][threadIdx.x] = hi[a];
  }
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int a = 0; a < 3; ++a) {
        red[a][threadIdx.x] = fmin(red[a][threadIdx.x], red[a][threadIdx.x + w]);
        red[3 + a][threadIdx.x] = fmax(red[3 + a][threadIdx.x], red[3 + a][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) box[threadIdx.x] = red[threadIdx.x][0];
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {  // bits 0..9 to every third bit
  v &= 1023u;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// key = (30-bit Morton code of the quantised position) << 32 | row; padding keys are all ones
__global__ void k_morton(int64_t m, int64_t N, const int32_t* __restrict__ vert, const double* __restrict__ xyz,
                         const double* __restrict__ box, uint64_t* __restrict__ keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    if (i >= m) {
      keys[i] = ~0ull;
      continue;
    }
    int64_t v = vert ? vert[i] : i;
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
      double ext = box[3 + a] - box[a];
      double t = ext > 0.0 ? (xyz[3 * v + a] - box[a]) / ext : 0.0;
      q[a] = static_cast<uint32_t>(fmin(fmax(t * 1024.0, 0.0), 1023.0));
    }
    uint32_t code = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    keys[i] = (static_cast<uint64_t>(code) << 32) | static_cast<uint64_t>(i);
  }
}

// Bitonic sort of N = 2^p keys (N >= kSortChunk): merge stages with partner distance j >=
// kSortChunk in global memory, the rest of each merge inside kSortChunk-key chunks in shared memory.
__global__ void k_bitonic_global(int64_t N, uint64_t* __restrict__ a, int64_t k, int64_t j) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = i ^ j;
    if (p <= i) continue;
    bool up = (i & k) == 0;
    uint64_t x = a[i], y = a[p];
    if ((x > y) == up) {
      a[i] = y;
      a[p] = x;
    }
  }
}

__global__ void __launch_bounds__(NT) k_bitonic_local(uint64_t* __restrict__ a, int64_t k, int64_t jmax) {
  __shared__ uint64_t s[kSortChunk];
  int64_t base = static_cast<int64_t>(blockIdx.x) * kSortChunk;
  for (int i = threadIdx.x; i < kSortChunk; i += NT) s[i] = a[base + i];
  __syncthreads();
  for (int64_t j = jmax; j > 0; j >>= 1) {
    for (int i = threadIdx.x; i < kSortChunk; i += NT) {
      int p = i ^ static_cast<int>(j);
      if (p > i) {
        bool up = ((base + i) & k) == 0;
        uint64_t x = s[i], y = s[p];
        if ((x > y) == up) {
          s[i] = y;
          s[p] = x;
        }
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kSortChunk; i += NT) a[base + i] = s[i];
}

void bitonic_sort(Ctx& c, uint64_t* keys, int64_t N) {
  unsigned chunks = static_cast<unsigned>(N / kSortChunk);
  for (int64_t k = 2; k <= N; k <<= 1) {
    int64_t j = k >> 1;
    for (; j >= kSortChunk; j >>= 1) {
      k_bitonic_global<<<grid_for(N, 256), 256, 0, c.stream>>>(N, keys, k, j);
      c.launched("bitonic_global");
    }
    k_bitonic_local<<<chunks, NT, 0, c.stream>>>(keys, k, j);
    c.launched("bitonic_local");
  }
}

// ------------------------------------------------------------------ tiles ----

__global__ void k_order(int64_t m, const uint64_t* __restrict__ keys, int32_t* __restrict__ perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    perm[i] = static_cast<int32_t>(keys[i] & 0xffffffffull);
}

// Exclusive scan of n <= kCand ints in shared memory by one CTA; returns the total.
__device__ int block_scan(int* d, int n) {
  __shared__ int part[NT];
  int per = (n + NT - 1) / NT;
  int lo = threadIdx.x * per, hi = min(n, lo + per);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += d[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < NT; off <<= 1) {
    int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int i = lo; i < hi; ++i) {
    int x = d[i];
    d[i] = run;
    run += x;
  }
  int total = part[NT - 1];
  __syncthreads();
  return total;
}

// One CTA per tile (rows [t R, t R + R)): the sorted unique rows that the tile's entries
// reference, together with the tile's own rows (its halo), each entry's index in it and each
// row's own index in it.
// The halo list is padded to a multiple of 4 rows with copies of its last row (the TMA product
// gathers rows four at a time).
template <int R, int CAP>
__global__ void __launch_bounds__(NT) k_tile_halo(int64_t m, const int32_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ col, int32_t* __restrict__ halo,
                                                  int32_t* __restrict__ nh, int32_t* __restrict__ lcol,
                                                  uint16_t* __restrict__ lself) {
  static_assert(CAP % 4 == 0, "halo lists are padded to multiples of 4 rows");
  __shared__ int cand[kCand];
  __shared__ int flag[kCand];
  int t = blockIdx.x;
  int64_t r0 = static_cast<int64_t>(t) * R, r1 = min(m, r0 + R);
  int e0 = rowptr[r0], e1 = rowptr[r1];
  int ne = e1 - e0, nr = static_cast<int>(r1 - r0);
  for (int q = e0 + threadIdx.x; q < e1; q += NT) lcol[q] = 0;
  for (int i = threadIdx.x; i < nr; i += NT) lself[r0 + i] = 0;
  if (ne + nr > kCand) {
    if (threadIdx.x == 0) nh[t] = INT_MAX;
    return;
  }
  int P = 1;
  while (P < ne + nr) P <<= 1;
  for (int i = threadIdx.x; i < P; i += NT)
    cand[i] = i < ne ? col[e0 + i] : (i < ne + nr ? static_cast<int>(r0) + (i - ne) : INT_MAX);
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += NT) {
        int p = i ^ j;
        if (p > i) {
          bool up = (i & k) == 0;
          int x = cand[i], y = cand[p];
          if ((x > y) == up) {
            cand[i] = y;
            cand[p] = x;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < P; i += NT) flag[i] = (cand[i] != INT_MAX && (i == 0 || cand[i] != cand[i - 1])) ? 1 : 0;
  __syncthreads();
  int total = block_scan(flag, P);
  if (threadIdx.x == 0) nh[t] = total;
  if (total > CAP) return;
  // unique columns to the tile's halo list (flag holds each first occurrence's slot)
  int* uniq = halo + static_cast<int64_t>(t) * CAP;
  for (int i = threadIdx.x; i < P; i += NT)
    if (cand[i] != INT_MAX && (i == 0 || cand[i] != cand[i - 1])) uniq[flag[i]] = cand[i];
  __syncthreads();
  for (int i = total + threadIdx.x; i < ((total + 3) & ~3); i += NT) uniq[i] = uniq[total - 1];
  for (int i = threadIdx.x; i < total; i += NT) cand[i] = uniq[i];
  __syncthreads();
  for (int q = e0 + threadIdx.x; q < e1 + nr; q += NT) {
    int cc = q < e1 ? col[q] : static_cast<int>(r0) + (q - e1);
    int lo = 0, hi = total - 1;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (cand[mid] < cc) lo = mid + 1;
      else hi = mid;
    }
    if (q < e1) lcol[q] = lo;
    else lself[r0 + (q - e1)] = static_cast<uint16_t>(lo);
  }
}

__global__ void k_tile_stats(int ntiles, int CAP, const int32_t* __restrict__ nh, int64_t* __restrict__ out) {
  __shared__ int64_t a[NT], b[NT];
  int64_t s = 0, h = 0;
  for (int t = threadIdx.x; t < ntiles; t += NT)
    if (nh[t] <= CAP) {
      ++s;
      h += nh[t];
    }
  a[threadIdx.x] = s;
  b[threadIdx.x] = h;
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      a[threadIdx.x] += a[threadIdx.x + w];
      b[threadIdx.x] += b[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = a[0];
    out[1] = b[0];
  }
}

// ------------------------------------------------------------------ product ----

constexpr int kMeta = 2560;  // entries per tile whose column index and value are staged
constexpr size_t kStageBytes = static_cast<size_t>(CAP) * kRowBytes;
constexpr size_t kSmemBytes = kStageBytes + kMeta * 8 + kMeta * 4 + (R + 1) * 4;
constexpr int kChunksPerThread = (CAP * (kRowBytes / 16) + NT - 1) / NT;

template <class T>
struct Lane8;  // the 8 bytes of a pass row one lane owns
template <>
struct Lane8<float> {
  static constexpr int N = 2;
};
template <>
struct Lane8<double> {
  static constexpr int N = 1;
};

__device__ __forceinline__ void ld8(float (&d)[2], const float* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  d[0] = v.x;
  d[1] = v.y;
}
__device__ __forceinline__ void ld8(double (&d)[1], const double* p) { d[0] = __ldg(p); }
__device__ __forceinline__ void lds8(float (&d)[2], const unsigned char* p) {
  float2 v = *reinterpret_cast<const float2*>(p);
  d[0] = v.x;
  d[1] = v.y;
}
__device__ __forceinline__ void lds8(double (&d)[1], const unsigned char* p) {
  d[0] = *reinterpret_cast<const double*>(p);
}
__device__ __forceinline__ void st8(float* p, const float (&d)[2]) {
  *reinterpret_cast<float2*>(p) = make_float2(d[0], d[1]);
}
__device__ __forceinline__ void st8(double* p, const double (&d)[1]) { *p = d[0]; }

// Asynchronous copies global -> shared: 16 bytes (zero-filled when bytes == 0), 8 and 4 bytes.
// Completion is awaited by cp_async_wait_all, which is also the compiler barrier.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
template <class T>
__device__ __forceinline__ void cp_async_val(T* smem, const T* gmem) {
  if constexpr (sizeof(T) == 8)
    cp_async8(smem, gmem);
  else
    cp_async4(smem, gmem);
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Work items are (tile, pass) pairs; a pass covers NBP = 8 / sizeof(T) column blocks, 256
// bytes of every row.  Lane l owns the 8 bytes at offset 8 l of a pass row: column block
// b0 + (8 l) / (32 sizeof(T)), columns from ((8 l) mod (32 sizeof(T))) / sizeof(T).
// Per item the CTA stages the halo rows (cp.async) and the tile's row pointers, local column
// indices and values, then computes every output row from shared memory.
template <class T>
__global__ void __launch_bounds__(NT, 2)
    k_spmm_tiled(int64_t m, int nb, int ntiles, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ lcol,
                 const uint16_t* __restrict__ lself, const int32_t* __restrict__ col,
                 const int32_t* __restrict__ halo, const int32_t* __restrict__ nh, const T* __restrict__ val,
                 const T* __restrict__ x, T* __restrict__ y, T alpha, double* __restrict__ acc,
                 const int32_t* __restrict__ blk_act, bool self_dot) {
  constexpr int NBP = 8 / sizeof(T);    // column blocks per pass
  constexpr int EPL = Lane8<T>::N;      // values per lane
  constexpr int BROW = 32 * sizeof(T);  // bytes of one block row
  constexpr int CPB = BROW / 16;        // 16-byte chunks per block row
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* stage = smem;                                            // CAP rows x kRowBytes
  T* s_val = reinterpret_cast<T*>(smem + kStageBytes);                     // kMeta
  int* s_col = reinterpret_cast<int*>(smem + kStageBytes + kMeta * 8);     // kMeta
  int* s_ptr = reinterpret_cast<int*>(smem + kStageBytes + kMeta * 12);    // R + 1 (absolute offsets)
  __shared__ double red[NW][NBP * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int my_blk = (8 * lane) / BROW;                // block within the pass
  const int my_col = ((8 * lane) % BROW) / sizeof(T);  // first column within that block
  const int ngroups = (nb + NBP - 1) / NBP;
  const int64_t items = static_cast<int64_t>(ntiles) * ngroups;
  for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
    const int t = static_cast<int>(w / ngroups);
    const int b0 = static_cast<int>(w % ngroups) * NBP;
    unsigned actm = 0;  // bit q: block b0 + q is active
#pragma unroll
    for (int q = 0; q < NBP; ++q)
      if (b0 + q < nb && (!blk_act || blk_act[b0 + q] != 0)) actm |= 1u << q;
    if (!actm) continue;  // uniform over the CTA
    const int cnt = nh[t];
    const bool staged = cnt <= CAP;
    const int64_t r0 = static_cast<int64_t>(t) * R;
    const int nr = static_cast<int>(min(m, r0 + R) - r0);
    const int e0 = rowptr[r0];
    const int ne = rowptr[r0 + nr] - e0;
    const bool meta = ne <= kMeta;
    if (staged) {
      // halo row ids first (one batch of independent loads), then every copy in flight at once
      const int32_t* hrow = halo + static_cast<int64_t>(t) * CAP;
      const int nchunk = cnt * (kRowBytes / 16);
      int hr[kChunksPerThread];
#pragma unroll
      for (int k = 0; k < kChunksPerThread; ++k) {
        int q = threadIdx.x + k * NT;
        hr[k] = q < nchunk ? hrow[q / (kRowBytes / 16)] : 0;
      }
#pragma unroll
      for (int k = 0; k < kChunksPerThread; ++k) {
        int q = threadIdx.x + k * NT;
        if (q < nchunk) {
          int i = q / (kRowBytes / 16), ch = q % (kRowBytes / 16);
          int bb = ch / CPB, off = ch % CPB;
          bool on = (actm >> bb) & 1u;
          const T* src = on ? x + (static_cast<int64_t>(b0 + bb) * m + hr[k]) * 32 : x;
          cp_async16(stage + i * kRowBytes + ch * 16, reinterpret_cast<const unsigned char*>(src) + off * 16,
                     on ? 16 : 0);
        }
      }
    }
    for (int i = threadIdx.x; i <= nr; i += NT) cp_async4(s_ptr + i, rowptr + r0 + i);
    if (meta) {
      for (int q = threadIdx.x; q < ne; q += NT) {
        cp_async_val<T>(s_val + q, val + e0 + q);
        if (staged) cp_async4(s_col + q, lcol + e0 + q);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    T dot[EPL];
#pragma unroll
    for (int i = 0; i < EPL; ++i) dot[i] = T(0);
    const bool mine = (actm >> my_blk) & 1u;
    for (int r = warp; r < nr; r += NW) {
      const int64_t u = r0 + r;
      const int q0 = s_ptr[r] - e0, q1 = s_ptr[r + 1] - e0;
      T a[EPL];
#pragma unroll
      for (int i = 0; i < EPL; ++i) a[i] = T(0);
      for (int base = q0; base < q1; base += 32) {
        int q = base + lane;
        int k = 0;
        T v = T(0);
        if (q < q1) {
          if (meta) {
            v = s_val[q];
            k = s_col[q];
          } else {
            v = val[e0 + q];
            k = lcol[e0 + q];
          }
          if (!staged) k = col[e0 + q];
        }
        int n = min(32, q1 - base);
        // four entries at a time: their operand loads are independent
        for (int j0 = 0; j0 < n; j0 += 4) {
          int kj[4];
          T vj[4], xv[4][EPL];
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            kj[d] = __shfl_sync(0xffffffffu, k, min(j0 + d, 31));
            vj[d] = __shfl_sync(0xffffffffu, v, min(j0 + d, 31));
          }
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            bool ok = j0 + d < n;
            if (ok && staged)
              lds8(xv[d], stage + kj[d] * kRowBytes + lane * 8);
            else if (ok && mine)
              ld8(xv[d], x + (static_cast<int64_t>(b0 + my_blk) * m + kj[d]) * 32 + my_col);
            else
#pragma unroll
              for (int i = 0; i < EPL; ++i) xv[d][i] = T(0);
          }
#pragma unroll
          for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int i = 0; i < EPL; ++i) a[i] += vj[d] * xv[d][i];
        }
      }
      if (mine) {
        T out[EPL];
#pragma unroll
        for (int i = 0; i < EPL; ++i) out[i] = alpha * a[i];
        int64_t o = (static_cast<int64_t>(b0 + my_blk) * m + u) * 32 + my_col;
        st8(y + o, out);
        if (acc) {
          T xu[EPL];
          if (self_dot) {
#pragma unroll
            for (int i = 0; i < EPL; ++i) xu[i] = out[i];
          } else if (staged) {
            lds8(xu, stage + static_cast<int>(lself[u]) * kRowBytes + lane * 8);
          } else {
            ld8(xu, x + o);
          }
#pragma unroll
          for (int i = 0; i < EPL; ++i) dot[i] += xu[i] * out[i];
        }
      }
    }
    if (acc) {
#pragma unroll
      for (int i = 0; i < EPL; ++i) red[warp][lane * EPL + i] = static_cast<double>(dot[i]);
      __syncthreads();
      for (int cc = threadIdx.x; cc < NBP * 32; cc += NT) {
        if (!((actm >> (cc / 32)) & 1u)) continue;
        double sum = 0.0;
        for (int q = 0; q < NW; ++q) sum += red[q][cc];
        atomicAdd(acc + b0 * 32 + cc, sum);
      }
    }
    __syncthreads();  // the next item overwrites the stage, the metadata and red
  }
}

__global__ void k_iota(int64_t m, int32_t* __restrict__ perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    perm[i] = static_cast<int32_t>(i);
}

}  // namespace

void locality_order(Ctx& c, int64_t m, const int32_t* vert, const double* xyz, int32_t* perm) {
  if (m <= 0) return;
  if (!xyz) {  // no positions (a caller's graph): keep the given order
    k_iota<<<grid_for(m, 256), 256, 0, c.stream>>>(m, perm);
    c.launched("order_identity");
    return;
  }
  int64_t N = kSortChunk;
  while (N < m) N <<= 1;
  double* box = c.alloc<double>(6);
  uint64_t* keys = c.alloc<uint64_t>(N);
  k_bbox<<<1, NT, 0, c.stream>>>(m, vert, xyz, box);
  c.launched("order_bbox");
  k_morton<<<grid_for(N, 256), 256, 0, c.stream>>>(m, N, vert, xyz, box, keys);
  c.launched("order_morton");
  bitonic_sort(c, keys, N);
  k_order<<<grid_for(m, 256), 256, 0, c.stream>>>(m, keys, perm);
  c.launched("order_perm");
  c.free(box);
  c.free(keys);
}

TiledPattern build_tiles(Ctx& c, int64_t m, int64_t nnz, const int32_t* rowptr, const int32_t* col, int rows) {
  TiledPattern tp;
  tp.m = m;
  tp.nnz = nnz;
  tp.rowptr = rowptr;
  tp.col = col;
  if (rows != kTileRows && rows != kGatherRows) SBHA_THROW(SBHA_EINVAL, "build_tiles: unsupported tile rows");
  tp.rows = rows;
  tp.cap = rows == kTileRows ? CAP : kGatherCap;
  if (m <= 0) return tp;
  tp.ntiles = static_cast<int>((m + rows - 1) / rows);
  tp.lcol = c.alloc<int32_t>(nnz);
  tp.lself = c.alloc<uint16_t>(static_cast<int64_t>(tp.ntiles) * rows);  // whole tiles (copied in 4-byte words)
  tp.halo = c.alloc<int32_t>(static_cast<int64_t>(tp.ntiles) * tp.cap);
  tp.nh = c.alloc<int32_t>(tp.ntiles);
  if (rows == kTileRows)
    k_tile_halo<R, CAP><<<tp.ntiles, NT, 0, c.stream>>>(m, rowptr, col, tp.halo, tp.nh, tp.lcol, tp.lself);
  else
    k_tile_halo<kGatherRows, kGatherCap>
        <<<tp.ntiles, NT, 0, c.stream>>>(m, rowptr, col, tp.halo, tp.nh, tp.lcol, tp.lself);
  c.launched("tile_halo");
  int64_t* st = c.alloc<int64_t>(2);
  k_tile_stats<<<1, NT, 0, c.stream>>>(tp.ntiles, tp.cap, tp.nh, st);
  c.launched("tile_stats");
  int64_t h[2] = {0, 0};
  SBHA_CUDA(cudaMemcpyAsync(h, st, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
  SBHA_CUDA(cudaStreamSynchronize(c.stream));
  tp.staged_tiles = static_cast<int>(h[0]);
  tp.halo_rows = h[1];
  c.free(st);
  return tp;
}

template <class T>
void spmm_tiled(Ctx& c, cudaStream_t s, const TiledPattern& tp, int nb, const T* val, const T* x, T* y, T alpha,
                double* acc, const int32_t* blk_act, bool self_dot) {
  if (tp.m <= 0 || nb <= 0) return;
  static bool attr_set = false;  // the shared-memory attribute is per function: set once per process
  if (!attr_set) {
    SBHA_CUDA(cudaFuncSetAttribute(k_spmm_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(kSmemBytes)));
    SBHA_CUDA(cudaFuncSetAttribute(k_spmm_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(kSmemBytes)));
    attr_set = true;
  }
  constexpr int NBP = 8 / sizeof(T);
  int64_t items = static_cast<int64_t>(tp.ntiles) * ((nb + NBP - 1) / NBP);
  unsigned grid = static_cast<unsigned>(std::min<int64_t>(items, 2 * num_sms()));
  k_spmm_tiled<T><<<grid, NT, kSmemBytes, s>>>(tp.m, nb, tp.ntiles, tp.rowptr, tp.lcol, tp.lself, tp.col, tp.halo,
                                               tp.nh, val, x, y, alpha, acc, blk_act, self_dot);
  c.launched("spmm_tiled");
}

template void spmm_tiled<float>(Ctx&, cudaStream_t, const TiledPattern&, int, const float*, const float*, float*,
                                float, double*, const int32_t*, bool);
template void spmm_tiled<double>(Ctx&, cudaStream_t, const TiledPattern&, int, const double*, const double*, double*,
                                 double, double*, const int32_t*, bool);

}  // namespace sbha
