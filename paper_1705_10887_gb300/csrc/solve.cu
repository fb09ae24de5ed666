// Interpolation solve (Sec. 2.1 Eq. 3, Sec. 3 Eq. 6): P_u = -M_uu^{-1} M_ub, one
// right-hand side per landmark, by Jacobi-preconditioned conjugate gradients run on
// many columns at once, followed by thresholding (Sec. 3.1, Eq. 8).
//
// Layout.  Unknowns are the non-landmark vertices numbered along a Morton curve through
// their positions (locality_order), so consecutive unknowns are compact surface patches;
// uord keeps the ascending-vertex order for the column-mode thresholding.  A chunk of
// C right-hand sides is stored column-block-major: block cb holds 32 columns as an
// m x 32 row-major slab.  The matrix products (k_spmm_grp) give each CTA chunks of
// about 32 consecutive rows spread over the grid (chunk b, b + G, b + 2G, ...), so the
// whole grid sweeps one contiguous stretch of the ordering at a time and a neighbour
// row two CTAs share is read by both at about the same time, from L2.
//
// Per iteration three kernels run (four with the learned preconditioner): Q = A P with
// the column dots P.Q; the x and r updates with r.z and r.r; the direction update
// p = z + beta p.  The column dots are summed per CTA and added to FP64 accumulators
// with one atomic per column and CTA, so the CG scalars can differ in their last bits
// between runs.  Columns are independent CG runs; a column stops when
// ||r|| <= rtol ||b|| and a block of 32 stopped columns is skipped by all kernels.
//
// Mixed precision: the same CG runs in FP32 on an FP32 copy of M_uu to a modest
// relative reduction; the FP64 residual b - M_uu x is then recomputed with the FP64
// operator and the loop repeats (iterative refinement) until the FP64 residual
// meets rtol.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <memory>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "internal.cuh"
#include "mlp.cuh"
#include "spmm.cuh"

namespace sbha {

namespace {

constexpr int BW = 32;           // columns per block (one per lane)
constexpr int kCgThreads = 256;  // 8 warps
constexpr int kCgWarps = kCgThreads / 32;
constexpr int kMaxChunk = 512;   // columns solved together

// ------------------------------------------------------ system extraction --

__global__ void k_mark_landmarks(const int32_t* __restrict__ idx, int l, int n, int32_t* lmcol, int* err) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < l; j += gridDim.x * blockDim.x) {
    int v = idx[j];
    if (v < 0 || v >= n) {
      set_error(err, DERR_BAD_INDEX);
      continue;
    }
    if (atomicCAS(lmcol + v, -1, j) != -1) set_error(err, DERR_DUPLICATE);
  }
}

__global__ void k_unknown_flags(int64_t n, const int32_t* __restrict__ lmcol, int32_t* __restrict__ flag) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = lmcol[v] < 0 ? 1 : 0;
}

__global__ void k_unknown_verts(int64_t n, const int32_t* __restrict__ lmcol, const int32_t* __restrict__ uidx,
                                int32_t* __restrict__ uvert) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (lmcol[v] < 0) uvert[uidx[v]] = static_cast<int32_t>(v);
}

// perm[j] = position (in ascending-vertex order) of the unknown numbered j
__global__ void k_renumber(int64_t m, const int32_t* __restrict__ perm, const int32_t* __restrict__ asc,
                           int32_t* __restrict__ uvert, int32_t* __restrict__ uidx, int32_t* __restrict__ uord) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    int i = perm[j];
    int v = asc[i];
    uvert[j] = v;
    uidx[v] = static_cast<int32_t>(j);
    uord[i] = static_cast<int32_t>(j);
  }
}

__global__ void k_muu_count(int64_t m, const int32_t* __restrict__ uvert, const int32_t* __restrict__ mrow,
                            const int32_t* __restrict__ mcol, const int32_t* __restrict__ lmcol,
                            int32_t* __restrict__ cnt) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < m; u += (int64_t)gridDim.x * blockDim.x) {
    int v = uvert[u], c = 0;
    for (int e = mrow[v]; e < mrow[v + 1]; ++e) c += lmcol[mcol[e]] < 0;
    cnt[u] = c;
  }
}

__global__ void k_muu_fill(int64_t m, const int32_t* __restrict__ uvert, const int32_t* __restrict__ mrow,
                           const int32_t* __restrict__ mcol, const double* __restrict__ mval,
                           const int32_t* __restrict__ lmcol, const int32_t* __restrict__ uidx,
                           const int32_t* __restrict__ urow, int32_t* __restrict__ ucol, double* __restrict__ uval,
                           float* __restrict__ uval32, double* __restrict__ dinv, float* __restrict__ dinv32) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < m; u += (int64_t)gridDim.x * blockDim.x) {
    int v = uvert[u], q0 = urow[u], q = q0;
    for (int e = mrow[v]; e < mrow[v + 1]; ++e) {
      int w = mcol[e];
      if (lmcol[w] >= 0) continue;
      // insertion into the row, kept sorted by unknown index
      int cw = uidx[w];
      int p = q;
      while (p > q0 && ucol[p - 1] > cw) {
        ucol[p] = ucol[p - 1];
        uval[p] = uval[p - 1];
        --p;
      }
      ucol[p] = cw;
      uval[p] = mval[e];
      if (w == v) {
        dinv[u] = 1.0 / mval[e];
        dinv32[u] = static_cast<float>(1.0 / mval[e]);
      }
      ++q;
    }
    for (int p = q0; p < q; ++p) uval32[p] = static_cast<float>(uval[p]);
  }
}

// Right-hand side of landmark j: -M_ub e_j, i.e. minus column b_j of M at the unknown rows.
__global__ void k_rhs_count(int l, const int32_t* __restrict__ idx, const int32_t* __restrict__ mrow,
                            const int32_t* __restrict__ mcol, const int32_t* __restrict__ lmcol,
                            int32_t* __restrict__ cnt) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < l; j += gridDim.x * blockDim.x) {
    int b = idx[j], c = 0;
    for (int e = mrow[b]; e < mrow[b + 1]; ++e) c += lmcol[mcol[e]] < 0;
    cnt[j] = c;
  }
}

__global__ void k_rhs_fill(int l, const int32_t* __restrict__ idx, const int32_t* __restrict__ mrow,
                           const int32_t* __restrict__ mcol, const double* __restrict__ mval,
                           const int32_t* __restrict__ lmcol, const int32_t* __restrict__ uidx,
                           const int32_t* __restrict__ rptr, int32_t* __restrict__ rrow, double* __restrict__ rval) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < l; j += gridDim.x * blockDim.x) {
    int b = idx[j], q = rptr[j];
    for (int e = mrow[b]; e < mrow[b + 1]; ++e) {
      int w = mcol[e];
      if (lmcol[w] >= 0) continue;
      // M[w][b] from row w (the pattern is symmetric)
      int lo = mrow[w], hi = mrow[w + 1];
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (mcol[mid] < b) lo = mid + 1; else hi = mid;
      }
      rrow[q] = uidx[w];
      rval[q] = -mval[lo];
      ++q;
    }
  }
}

// --------------------------------------------------------------- CG ------
//
// Row-vector mapping.  A warp owns one row u of a chunk and covers all of its column
// blocks: with W = 16 / sizeof(T) values per 16-byte vector, 32 / W lanes share a
// block row (128 B in FP32, 256 B in FP64) and a warp-wide vector access spans W
// consecutive blocks; NS = 16 / W such accesses cover the 512 columns of a full chunk.
// Every lane therefore keeps the same 16 columns for every row it touches, so the
// per-column dot products are accumulated in registers, summed over the CTA's warps in
// shared memory and added to a global FP64 accumulator with one atomic per column and
// CTA.  (The order of those atomic additions varies from run to run, so the CG scalars
// can differ in their last bits between runs.)

template <class T>
struct VT;
template <>
struct VT<float> {
  using V = float4;
  static constexpr int W = 4;
};
template <>
struct VT<double> {
  using V = double2;
  static constexpr int W = 2;
};

__device__ __forceinline__ void vld(float (&d)[4], const float* p) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  d[0] = v.x;
  d[1] = v.y;
  d[2] = v.z;
  d[3] = v.w;
}
__device__ __forceinline__ void vld(double (&d)[2], const double* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  d[0] = v.x;
  d[1] = v.y;
}
// plain (coherent) loads for arrays this kernel also writes
__device__ __forceinline__ void vldw(float (&d)[4], const float* p) {
  float4 v = *reinterpret_cast<const float4*>(p);
  d[0] = v.x;
  d[1] = v.y;
  d[2] = v.z;
  d[3] = v.w;
}
__device__ __forceinline__ void vldw(double (&d)[2], const double* p) {
  double2 v = *reinterpret_cast<const double2*>(p);
  d[0] = v.x;
  d[1] = v.y;
}
__device__ __forceinline__ void vst(float* p, const float (&d)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(d[0], d[1], d[2], d[3]);
}
__device__ __forceinline__ void vst(double* p, const double (&d)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(d[0], d[1]);
}

// Lane geometry of the row-vector mapping.
template <class T>
struct Lanes {
  static constexpr int W = VT<T>::W;
  static constexpr int LPB = 32 / W;  // lanes per block row
  static constexpr int NS = 16 / W;   // vector accesses per row (16 blocks max)
  int bo, wc;                         // block offset within an access, first column within the block
  __device__ __forceinline__ Lanes(int lane) : bo(lane / LPB), wc((lane % LPB) * W) {}
  __device__ __forceinline__ int block(int s) const { return s * W + bo; }
  // chunk-local column of element i of access s
  __device__ __forceinline__ int column(int s, int i) const { return block(s) * BW + wc + i; }
  __device__ __forceinline__ int64_t offset(int s, int64_t m, int64_t u) const {
    return (static_cast<int64_t>(block(s)) * m + u) * BW + wc;
  }
};

// Adds the CTA's per-column partials (part[s][i] of every lane) to acc[column] (FP64 atomics).
template <class T, int NS, int W>
__device__ __forceinline__ void cta_accumulate(T (*red)[kMaxChunk], const T (&part)[NS][W], const Lanes<T>& L,
                                               int nb, int C, double* acc) {
  int warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int i = 0; i < W; ++i)
      if (L.block(s) < nb) red[warp][L.column(s, i)] = part[s][i];
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    T sum = T(0);
    for (int w = 0; w < kCgWarps; ++w) sum += red[w][c];
    atomicAdd(acc + c, static_cast<double>(sum));
  }
  __syncthreads();
}

constexpr int kGrpRows = 128;   // rows per CTA at most
constexpr int kGrpMeta = 1536;  // staged entries per CTA (more: read from global memory)
constexpr int kGrpChunks = 8;   // chunks per CTA at most

// One staged nonzero: its column and value, read as one 8- or 16-byte shared-memory word.
template <class T>
struct alignas(2 * sizeof(T)) GrpEnt {
  int c;
  T v;
};

// Rows of one CTA in the block-group kernels.  The (locality-ordered) rows are cut into chunks
// of R consecutive rows; CTA b takes chunks b, b + G, ..., b + (nci - 1) G (G = gridDim.x), so
// that at any moment the grid sweeps one contiguous stretch of the ordering and a neighbour row
// that two CTAs share is read by both at about the same time (from L2, not twice from DRAM).
// Local row lr = i R + j is row (b + i G) R + j.  The chunks' CSR slices are copied into shared
// memory back to back in one coalesced batch: local row lr has entries [ptr[lr], ptr[lr + 1]),
// in the staged array when the CTA's entries fit (staged), else at col/val[q + gsh[i]].
struct GrpShared {
  int ptr[kGrpRows + 1];
  int off[kGrpChunks + 1];
  int gsh[kGrpChunks];
  bool staged;
};

// Global row of local row lr (m or more: past the end, no row).
__device__ __forceinline__ int64_t grp_row(int lr, int R) {
  return (blockIdx.x + static_cast<int64_t>(lr / R) * gridDim.x) * R + lr % R;
}

template <class T>
__device__ __forceinline__ void grp_stage(int64_t m, int R, int nci, const int32_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ col, const T* __restrict__ val, GrpShared& sh,
                                          GrpEnt<T>* s_ent) {
  const int64_t G = gridDim.x;
  if (threadIdx.x < nci) {
    int64_t row0 = (blockIdx.x + threadIdx.x * G) * R;
    int a = rowptr[min(row0, m)], e = rowptr[min(row0 + R, m)];
    sh.off[threadIdx.x + 1] = e - a;
    sh.gsh[threadIdx.x] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sh.off[0] = 0;
    for (int i = 0; i < nci; ++i) sh.off[i + 1] += sh.off[i];
    sh.staged = sh.off[nci] <= kGrpMeta;
  }
  __syncthreads();
  const bool staged = sh.staged;
  for (int lr = threadIdx.x; lr < nci * R; lr += blockDim.x) {
    int i = lr / R, j = lr % R;
    int64_t row0 = (blockIdx.x + i * G) * R;
    sh.ptr[lr] = sh.off[i] + rowptr[min(row0 + j, m)] - sh.gsh[i];
  }
  if (threadIdx.x == 0) sh.ptr[nci * R] = sh.off[nci];
  if (staged)
    for (int i = 0; i < nci; ++i) {
      const int a = sh.gsh[i], o = sh.off[i], len = sh.off[i + 1] - o;
      for (int q = threadIdx.x; q < len; q += blockDim.x) {
        GrpEnt<T> e;
        e.c = col[a + q];
        e.v = val[a + q];
        s_ent[o + q] = e;
      }
    }
  __syncthreads();
  if (!staged && threadIdx.x < nci) sh.gsh[threadIdx.x] -= sh.off[threadIdx.x];
  __syncthreads();
}

// a = sum_q v_q x[c_q] over local row lr's nonzeros for this lane's W columns (xb: the lane's
// columns of x), up to U neighbours gathered in one round of independent loads (the sum runs over
// the entries in CSR order whatever U is).
template <class T, int U, bool ST>
__device__ __forceinline__ void grp_row_sum(const GrpEnt<T>* s_ent, int q0, int q1, int gs,
                                            const int32_t* __restrict__ col, const T* __restrict__ val,
                                            const T* __restrict__ xb, T (&a)[VT<T>::W]);

template <class T, int U = 8>
__device__ __forceinline__ void grp_row_product(const GrpShared& sh, const GrpEnt<T>* s_ent, int lr, int R,
                                                const int32_t* __restrict__ col, const T* __restrict__ val,
                                                const T* __restrict__ xb, T (&a)[VT<T>::W]) {
  if (sh.staged)
    grp_row_sum<T, U, true>(s_ent, sh.ptr[lr], sh.ptr[lr + 1], 0, col, val, xb, a);
  else
    grp_row_sum<T, U, false>(s_ent, sh.ptr[lr], sh.ptr[lr + 1], sh.gsh[lr / R], col, val, xb, a);
}

// The same sum for entries [q0, q1) of the staged (or, staged == false, global at offset gs) CSR slice.
template <class T, int U, bool ST>
__device__ __forceinline__ void grp_row_sum(const GrpEnt<T>* s_ent, int q0, int q1, int gs,
                                            const int32_t* __restrict__ col, const T* __restrict__ val,
                                            const T* __restrict__ xb, T (&a)[VT<T>::W]) {
  constexpr int W = VT<T>::W;
#pragma unroll
  for (int i = 0; i < W; ++i) a[i] = T(0);
  for (int base = q0; base < q1; base += U) {
    int kk[U];
    T vv[U], xv[U][W];
#pragma unroll
    for (int d = 0; d < U; ++d) {
      const int q = base + d;
      const bool ok = q < q1;
      if constexpr (ST) {
        kk[d] = ok ? s_ent[q].c : 0;
        vv[d] = ok ? s_ent[q].v : T(0);
      } else {
        kk[d] = ok ? col[q + gs] : 0;
        vv[d] = ok ? val[q + gs] : T(0);
      }
    }
#pragma unroll
    for (int d = 0; d < U; ++d) {
      if (base + d < q1)
        vld(xv[d], xb + static_cast<int64_t>(kk[d]) * BW);
      else
#pragma unroll
        for (int i = 0; i < W; ++i) xv[d][i] = T(0);
    }
#pragma unroll
    for (int d = 0; d < U; ++d)
#pragma unroll
      for (int i = 0; i < W; ++i) a[i] += vv[d] * xv[d][i];
  }
}

// Warp-to-work map of the block-group kernels: each warp owns 512 bytes of a row (BPA blocks,
// one vector load per lane per neighbour); the CTA's warps split the 16 blocks (NG groups) and
// RW row sets.
template <class T>
struct GrpMap {
  static constexpr int W = VT<T>::W;        // values per vector load: 4 (FP32) or 2 (FP64)
  static constexpr int LPB = 32 / W;        // lanes per 32-column block row
  static constexpr int BPA = 32 / LPB;      // blocks per warp-wide access: 4 or 2
  static constexpr int NG = 16 / BPA;       // block groups per 16 blocks: 4 or 8
  static constexpr int RW = kCgWarps / NG;  // warps per group in a CTA: 2 or 1
  int g, rw, blk, c0;
  __device__ GrpMap() {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    g = warp % NG;
    rw = warp / NG;
    blk = g * BPA + lane / LPB;
    c0 = (lane % LPB) * W;
  }
};

// y = alpha * A x, the CTA's rows staged by grp_stage and swept by its warps (GrpMap).  Blocks with
// blk_act == 0 are skipped; with acc, acc[c] += sum_u x_uc y_uc (sum_u y_uc^2 when self_dot).  U
// neighbours in flight per row and MINB resident CTAs per SM: the register budget trades loads in
// flight per warp against resident warps (the autotuner picks).
template <class T, int U = 8, int MINB = 4>
__global__ void __launch_bounds__(kCgThreads, MINB) k_spmm_grp(int64_t m, int nb, const int32_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col, const T* __restrict__ val,
                                                          const T* __restrict__ x, T* __restrict__ y, T alpha,
                                                          double* __restrict__ acc, int C,
                                                          const int32_t* __restrict__ blk_act, bool self_dot,
                                                          int R, int nci) {
  using M = GrpMap<T>;
  constexpr int W = M::W;
  __shared__ T red[M::RW][kMaxChunk];  // the warps of one row set write disjoint column groups
  __shared__ GrpShared sh;
  __shared__ GrpEnt<T> s_ent[kGrpMeta];
  const M mp;
  const bool on = mp.blk < nb && (!blk_act || blk_act[mp.blk] != 0);
  grp_stage<T>(m, R, nci, rowptr, col, val, sh, s_ent);
  T dot[W];
#pragma unroll
  for (int i = 0; i < W; ++i) dot[i] = T(0);
  // chunk i of the CTA, rows j of the chunk (no divisions per row); the CSR slices from shared memory
  // or, when they did not fit, from global memory: two specialised loops
  auto sweep = [&](auto staged_tag) {
    constexpr bool ST = decltype(staged_tag)::value;
    const T* xb = x + static_cast<int64_t>(mp.blk) * m * BW + mp.c0;
    for (int i = 0; i < nci; ++i) {
      const int64_t row0 = (blockIdx.x + static_cast<int64_t>(i) * gridDim.x) * R;
      const int gs = ST ? 0 : sh.gsh[i];
      for (int j = mp.rw; j < R; j += M::RW) {
      const int64_t gr = row0 + j;
      if (gr >= m) break;
      const int lr = i * R + j;
      T a[W];
      grp_row_sum<T, U, ST>(s_ent, sh.ptr[lr], sh.ptr[lr + 1], gs, col, val, xb, a);
      T out[W];
#pragma unroll
      for (int i = 0; i < W; ++i) out[i] = alpha * a[i];
      int64_t o = (static_cast<int64_t>(mp.blk) * m + gr) * BW + mp.c0;
      vst(y + o, out);
      if (acc) {
        T xu[W];
        if (self_dot) {
#pragma unroll
          for (int i = 0; i < W; ++i) xu[i] = out[i];
        } else {
          vld(xu, x + o);
        }
#pragma unroll
        for (int i = 0; i < W; ++i) dot[i] += xu[i] * out[i];
      }
      }
    }
  };
  if (on) {
    if (sh.staged)
      sweep(std::true_type{});
    else
      sweep(std::false_type{});
  }
  if (acc) {
    if (mp.blk < nb)
#pragma unroll
      for (int i = 0; i < W; ++i) red[mp.rw][mp.blk * BW + mp.c0 + i] = dot[i];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      int cb = c / BW;
      if (cb >= nb) continue;
      T sum = T(0);
#pragma unroll
      for (int r = 0; r < M::RW; ++r) sum += red[r][c];
      atomicAdd(acc + c, static_cast<double>(sum));
    }
  }
}

// ------------------------------------------------------- pipelined gathers ----
//
// The gather of k_spmm_grp holds one row's neighbour loads in registers, which caps the bytes a
// warp has in flight at one row.  The pipelined variants copy, per lane, the lane's 16-byte slice
// of every neighbour row of the next D rows into a per-warp ring in shared memory (cp.async, also
// cached in L1), one commit group per row, and read back only the lane's own slices, so no warp
// barrier is needed and D rows' neighbours are in flight at no register cost.  A row keeps at
// most kPipeK neighbours in the ring; any further ones are loaded directly when the row is summed.
// Every row is summed in the order of its CSR entries, as in k_spmm_grp: the results are the same
// bit for bit whichever kernel runs.

constexpr int kPipeK = 8;
constexpr int kPipeSlot = 32 * 16;  // bytes of one staged neighbour row slice of a warp

__device__ __forceinline__ void cp_async_ca16(const void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int D>
constexpr size_t pipe_ring_bytes() {
  return static_cast<size_t>(kCgWarps) * D * kPipeK * kPipeSlot;
}

// The warp's rows of the CTA (local rows rw, rw + RW, ...) with D rows of neighbour slices in
// flight; epi(gr, a) receives each row's sum a = sum_q v_q x[c_q] for this lane's W columns
// (xb: the lane's columns of x).  ring: the warp's D x kPipeK x kPipeSlot bytes of shared memory.
template <class T, int D, class Epi>
__device__ __forceinline__ void pipe_rows(int64_t m, int R, int nci, int rw, int RW, const GrpShared& sh,
                                          const GrpEnt<T>* s_ent, const int32_t* __restrict__ col,
                                          const T* __restrict__ val, const T* __restrict__ xb, unsigned char* ring,
                                          Epi&& epi) {
  constexpr int W = VT<T>::W;
  const int lane = threadIdx.x & 31;
  const int nloc = nci * R;
  const bool staged = sh.staged;
  auto issue = [&](int j) {
    const int r = rw + j * RW;
    if (r < nloc && grp_row(r, R) < m) {
      const int q0 = sh.ptr[r], q1 = min(sh.ptr[r + 1], q0 + kPipeK);
      const int gs = staged ? 0 : sh.gsh[r / R];
      unsigned char* slot = ring + (j % D) * (kPipeK * kPipeSlot) + lane * 16;
      for (int q = q0; q < q1; ++q) {
        const int k = staged ? s_ent[q].c : col[q + gs];
        cp_async_ca16(slot + (q - q0) * kPipeSlot, xb + static_cast<int64_t>(k) * BW);
      }
    }
    cp_async_commit();  // one group per row (possibly empty), so wait_group<D - 1> finds row j's
  };
#pragma unroll
  for (int j = 0; j < D; ++j) issue(j);
  for (int j = 0; rw + j * RW < nloc; ++j) {
    cp_async_wait<D - 1>();
    const int r = rw + j * RW;
    const int64_t gr = grp_row(r, R);
    if (gr < m) {
      const int q0 = sh.ptr[r], q1 = sh.ptr[r + 1];
      const int gs = staged ? 0 : sh.gsh[r / R];
      const int qs = min(q1, q0 + kPipeK);
      const unsigned char* slot = ring + (j % D) * (kPipeK * kPipeSlot) + lane * 16;
      T a[W];
#pragma unroll
      for (int i = 0; i < W; ++i) a[i] = T(0);
      for (int q = q0; q < qs; ++q) {
        const T v = staged ? s_ent[q].v : val[q + gs];
        T xv[W];
        vldw(xv, reinterpret_cast<const T*>(slot + (q - q0) * kPipeSlot));
#pragma unroll
        for (int i = 0; i < W; ++i) a[i] += v * xv[i];
      }
      for (int q = qs; q < q1; ++q) {  // beyond the ring's capacity
        const int k = staged ? s_ent[q].c : col[q + gs];
        const T v = staged ? s_ent[q].v : val[q + gs];
        T xv[W];
        vld(xv, xb + static_cast<int64_t>(k) * BW);
#pragma unroll
        for (int i = 0; i < W; ++i) a[i] += v * xv[i];
      }
      epi(gr, a);
    }
    issue(j + D);  // refills the slot just read
  }
  cp_async_wait<0>();
}

// k_spmm_grp with the pipelined gather (same arguments and results).
template <class T, int D>
__global__ void __launch_bounds__(kCgThreads) k_spmm_pipe(int64_t m, int nb, const int32_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col, const T* __restrict__ val,
                                                          const T* __restrict__ x, T* __restrict__ y, T alpha,
                                                          double* __restrict__ acc, int C,
                                                          const int32_t* __restrict__ blk_act, bool self_dot, int R,
                                                          int nci) {
  using M = GrpMap<T>;
  constexpr int W = M::W;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ T red[kCgWarps][kMaxChunk];
  __shared__ GrpShared sh;
  __shared__ GrpEnt<T> s_ent[kGrpMeta];
  const M mp;
  const int warp = threadIdx.x >> 5;
  const bool on = mp.blk < nb && (!blk_act || blk_act[mp.blk] != 0);
  grp_stage<T>(m, R, nci, rowptr, col, val, sh, s_ent);
  T dot[W];
#pragma unroll
  for (int i = 0; i < W; ++i) dot[i] = T(0);
  if (on) {
    const T* xb = x + static_cast<int64_t>(mp.blk) * m * BW + mp.c0;
    unsigned char* ring = dyn_smem + static_cast<size_t>(warp) * D * kPipeK * kPipeSlot;
    pipe_rows<T, D>(m, R, nci, mp.rw, M::RW, sh, s_ent, col, val, xb, ring, [&](int64_t gr, const T(&a)[W]) {
      T out[W];
#pragma unroll
      for (int i = 0; i < W; ++i) out[i] = alpha * a[i];
      const int64_t o = (static_cast<int64_t>(mp.blk) * m + gr) * BW + mp.c0;
      vst(y + o, out);
      if (acc) {
        T xu[W];
        if (self_dot) {
#pragma unroll
          for (int i = 0; i < W; ++i) xu[i] = out[i];
        } else {
          vld(xu, x + o);
        }
#pragma unroll
        for (int i = 0; i < W; ++i) dot[i] += xu[i] * out[i];
      }
    });
  }
  if (acc) {
    if (mp.blk < nb)
#pragma unroll
      for (int i = 0; i < W; ++i) red[warp][mp.blk * BW + mp.c0 + i] = dot[i];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      int cb = c / BW;
      if (cb >= nb) continue;
      int gg = cb / M::BPA;
      T sum = T(0);
#pragma unroll
      for (int r = 0; r < M::RW; ++r) sum += red[gg + r * M::NG][c];
      atomicAdd(acc + c, static_cast<double>(sum));
    }
  }
}

// Per-column CG state.  rz and act are double-buffered by iteration parity (the kernel that
// publishes the next value runs while others still read the current one); the three
// accumulators are double-buffered the same way and cleared one iteration ahead.
struct CgState {
  double* rz;      // [2][C]  r.z of the current iterate
  int32_t* act;    // [2][C]  column still iterating
  int32_t* bact;   // [2][nb] block has an active column
  double* bb;      // [C]     ||b||^2 of the right-hand side
  double* rr;      // [C]     ||r||^2 at the last update
  int32_t* iters;  // [C]     iterations taken
  int32_t* n_active;
  int32_t* it;     // iteration counter
  int32_t* blog;   // [max_iter+1] active column blocks per iteration (kernel timing only; nullable)
  double* pq;      // [2][C]  accumulator of p.q
  double* rzn;     // [2][C]  accumulator of r.z after the update
  double* rra;     // [2][C]  accumulator of r.r after the update
  double* start;   // [2][C]  r.z and b.b of the starting residual
  int32_t* fail;   // set when a column's r.r or r.z stops being finite (that column then stops)
};

// Block-streaming mapping of the CG vector kernels: CTA (x, y) owns column block y and the x-th
// contiguous range of rows (grid stream_grid); thread t handles the 16-byte vector t % VPR of rows
// t / VPR, t / VPR + kCgThreads / VPR, ..., so a warp reads and writes 512 contiguous bytes per
// instruction and every thread keeps the state of only W columns.  The per-column dot products are
// summed over the lanes that share columns (shuffles), then over the warps in a fixed order, and added
// to the global FP64 accumulators with one atomic per column and CTA.
template <class T>
struct Stream {
  static constexpr int W = VT<T>::W;  // values per 16-byte vector
  static constexpr int VPR = BW / W;  // vectors per block row
};

__device__ __forceinline__ void cta_row_range(int64_t m, int64_t* r0, int64_t* r1) {
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  *r0 = min(m, per * blockIdx.x);
  *r1 = min(m, *r0 + per);
}

// Grid of the block-streaming kernels: nb column blocks (y) x row ranges (x), one wave of
// `per_sm` CTAs per SM when every block is active.
dim3 stream_grid(int64_t m, int nb, int per_sm = 4) {
  const int64_t target = std::max(per_sm, 1) * static_cast<int64_t>(num_sms());
  int64_t gx = std::max<int64_t>(1, target / std::max(nb, 1));
  gx = std::min<int64_t>(gx, std::max<int64_t>(1, (m + 63) / 64));  // at least 64 rows per CTA
  return dim3(static_cast<unsigned>(gx), static_cast<unsigned>(nb));
}

// Adds the CTA's partial sums of one block's columns (per-thread a[W] for columns cv*W + i) to acc.
template <class T>
__device__ __forceinline__ void cta_block_sum(const T (&a)[VT<T>::W], double (*red)[BW], double* acc) {
  constexpr int W = Stream<T>::W, VPR = Stream<T>::VPR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, cv = threadIdx.x % VPR;
  double v[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    v[i] = static_cast<double>(a[i]);
#pragma unroll
    for (int o = VPR; o < 32; o <<= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  if (lane < VPR)
#pragma unroll
    for (int i = 0; i < W; ++i) red[warp][cv * W + i] = v[i];
  __syncthreads();
  if (threadIdx.x < BW) {
    double sum = 0.0;
    for (int w = 0; w < kCgWarps; ++w) sum += red[w][threadIdx.x];
    atomicAdd(acc + threadIdx.x, sum);
  }
  __syncthreads();
}

// x += alpha p (X nullable: the direction update does it) ; r -= alpha q ; accumulate r.r, and r.z
// with z = D^{-1} r when dinv is given (alpha = rz / pq per column)
template <class T>
__global__ void __launch_bounds__(kCgThreads) k_cg_xr(int64_t m, int nb, int C, int cur, T* __restrict__ X,
                                                      T* __restrict__ R, const T* __restrict__ P,
                                                      const T* __restrict__ Q, const T* __restrict__ dinv,
                                                      CgState s) {
  constexpr int W = Stream<T>::W, VPR = Stream<T>::VPR;
  __shared__ double red[kCgWarps][BW];
  const int cv = threadIdx.x % VPR;
  int64_t r0, r1;
  cta_row_range(m, &r0, &r1);
  const int64_t items = (r1 - r0) * VPR;
  const int b = blockIdx.y;
  if (s.bact[cur * nb + b] != 0) {  // uniform over the CTA
    T al[W], rz[W], rr[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int c = b * BW + cv * W + i;
      const double pq = s.pq[cur * C + c];
      al[i] = (s.act[cur * C + c] && pq != 0.0) ? static_cast<T>(s.rz[cur * C + c] / pq) : T(0);
      rz[i] = rr[i] = T(0);
    }
    const int64_t base = (static_cast<int64_t>(b) * m + r0) * BW + cv * W;
    // U rows per thread per round: every load of the round is issued before any store (the
    // compiler cannot reorder a load of R above a store to R), so U rows' bytes are in flight
    auto sweep = [&](auto u_tag, auto x_tag) {
      constexpr int U = decltype(u_tag)::value;
      constexpr bool WX = decltype(x_tag)::value;
      for (int64_t q0 = threadIdx.x; q0 < items; q0 += U * kCgThreads) {
        T rv[U][W], qv[U][W], xv[WX ? U : 1][W], pv[WX ? U : 1][W], d[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t q = q0 + static_cast<int64_t>(u) * kCgThreads;
          if (q < items) {
            const int64_t o = base + (q / VPR) * BW;
            vldw(rv[u], R + o);
            vld(qv[u], Q + o);
            if constexpr (WX) {
              vldw(xv[u], X + o);
              vld(pv[u], P + o);
            }
            d[u] = dinv ? dinv[r0 + q / VPR] : T(0);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t q = q0 + static_cast<int64_t>(u) * kCgThreads;
          if (q < items) {
            const int64_t o = base + (q / VPR) * BW;
            if constexpr (WX) {
#pragma unroll
              for (int i = 0; i < W; ++i) xv[u][i] += al[i] * pv[u][i];
              vst(X + o, xv[u]);
            }
#pragma unroll
            for (int i = 0; i < W; ++i) {
              rv[u][i] -= al[i] * qv[u][i];
              rz[i] += rv[u][i] * rv[u][i] * d[u];
              rr[i] += rv[u][i] * rv[u][i];
            }
            vst(R + o, rv[u]);
          }
        }
      }
    };
    if (X)
      sweep(std::integral_constant<int, 2>{}, std::true_type{});
    else
      sweep(std::integral_constant<int, 4>{}, std::false_type{});
    if (dinv) cta_block_sum<T>(rz, red, s.rzn + cur * C + b * BW);
    cta_block_sum<T>(rr, red, s.rra + cur * C + b * BW);
  }
}

// beta_c = rz_new / rz and the activity of every column into shared memory; CTA 0 publishes the
// next iteration's state and clears the next accumulators.
template <class T>
__device__ void cg_next_state(int nb, int C, int cur, double tol2, CgState s, T* beta, int* actv) {
  __shared__ int s_nact, s_nblk;
  const bool lead = blockIdx.x == 0 && blockIdx.y == 0;
  int nxt = cur ^ 1;
  if (threadIdx.x == 0) {
    s_nact = 0;
    s_nblk = 0;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double rz = s.rz[cur * C + c];
    double rzn = s.rzn[cur * C + c];
    int a = s.act[cur * C + c];
    actv[c] = a;
    beta[c] = (a && rz != 0.0) ? static_cast<T>(rzn / rz) : T(0);
    if (lead) {
      double rr = s.rra[cur * C + c];
      bool finite = isfinite(rr) && isfinite(rzn);
      if (a && !finite) atomicOr(s.fail, 1);
      bool still = a && finite && !(rr <= tol2 * s.bb[c]);
      if (a) {
        s.rr[c] = rr;
        s.iters[c] = *s.it + 1;
      }
      s.rz[nxt * C + c] = rzn;
      s.act[nxt * C + c] = still ? 1 : 0;
      s.pq[nxt * C + c] = 0.0;
      s.rzn[nxt * C + c] = 0.0;
      s.rra[nxt * C + c] = 0.0;
      if (still) atomicAdd(&s_nact, 1);
    }
  }
  __syncthreads();
  if (lead) {
    for (int cb = threadIdx.x; cb < nb; cb += blockDim.x) {
      int any = 0;
      for (int c = cb * BW; c < cb * BW + BW && c < C; ++c) any |= s.act[nxt * C + c];
      s.bact[nxt * nb + cb] = any;
      if (any) atomicAdd(&s_nblk, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      *s.n_active = s_nact;
      if (s.blog) s.blog[*s.it + 1] = s_nblk;  // active blocks of the next iteration
      *s.it += 1;
    }
  }
}

// beta = rz_new / rz ; p = z + beta p for active columns, z = D^{-1} r or the given Z.  CTA 0
// publishes the next iteration's state and clears the next accumulators.  Block-streaming mapping
// (k_cg_xr).
template <class T>
__global__ void __launch_bounds__(kCgThreads) k_cg_p(int64_t m, int nb, int C, int cur, double tol2,
                                                     const T* __restrict__ R, T* __restrict__ P,
                                                     const T* __restrict__ dinv, const T* __restrict__ Z, CgState s) {
  constexpr int W = Stream<T>::W, VPR = Stream<T>::VPR;
  __shared__ T beta[kMaxChunk];
  __shared__ int actv[kMaxChunk];
  cg_next_state<T>(nb, C, cur, tol2, s, beta, actv);
  const int cv = threadIdx.x % VPR;
  int64_t r0, r1;
  cta_row_range(m, &r0, &r1);
  const int64_t items = (r1 - r0) * VPR;
  const T* src = Z ? Z : R;
  const int b = blockIdx.y;
  if (s.bact[cur * nb + b] != 0) {  // uniform over the CTA
    T bt[W];
    bool ca[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      bt[i] = beta[b * BW + cv * W + i];
      ca[i] = actv[b * BW + cv * W + i] != 0;
    }
    const int64_t base = (static_cast<int64_t>(b) * m + r0) * BW + cv * W;
    constexpr int U = 4;  // rows per thread per round, all loaded before any store (as in k_cg_xr)
    for (int64_t q0 = threadIdx.x; q0 < items; q0 += U * kCgThreads) {
      T rv[U][W], pv[U][W], d[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t q = q0 + static_cast<int64_t>(u) * kCgThreads;
        if (q < items) {
          const int64_t o = base + (q / VPR) * BW;
          vld(rv[u], src + o);
          vldw(pv[u], P + o);
          d[u] = Z ? T(1) : dinv[r0 + q / VPR];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t q = q0 + static_cast<int64_t>(u) * kCgThreads;
        if (q < items) {
#pragma unroll
          for (int i = 0; i < W; ++i)
            if (ca[i]) pv[u][i] = rv[u][i] * d[u] + bt[i] * pv[u][i];
          vst(P + base + (q / VPR) * BW, pv[u]);
        }
      }
    }
  }
}

// Direction update with the learned preconditioner, z = G^T t (t = G r) formed on the fly:
// x += alpha p (the old p, this iteration's alpha; X nullable) and p = z + beta p for active columns,
// the product in the mapping of k_spmm_grp (grp_stage, grp_row_product, GrpMap).  CTA 0 publishes
// the next iteration's state as k_cg_p does; it writes only the other parity's slots, so alpha =
// rz / pq of this iteration stays readable.
template <class T, int D = 0>
__global__ void __launch_bounds__(kCgThreads) k_cg_p_gt(int64_t m, int nb, int C, int cur, double tol2,
                                                         const int32_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ col, const T* __restrict__ gt,
                                                         const T* __restrict__ Tg, T* __restrict__ P,
                                                         T* __restrict__ X, CgState s, int R, int nci) {
  using M = GrpMap<T>;
  constexpr int W = M::W;
  __shared__ T beta[kMaxChunk];
  __shared__ T alpha[kMaxChunk];
  __shared__ int actv[kMaxChunk];
  if (X)
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      double pq = s.pq[cur * C + c];
      alpha[c] = (s.act[cur * C + c] && pq != 0.0) ? static_cast<T>(s.rz[cur * C + c] / pq) : T(0);
    }
  __shared__ GrpShared sh;
  __shared__ GrpEnt<T> s_ent[kGrpMeta];
  cg_next_state<T>(nb, C, cur, tol2, s, beta, actv);
  const M mp;
  const bool on = mp.blk < nb && s.bact[cur * nb + mp.blk] != 0;
  T bt[W], al[W];
  bool ca[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    bt[i] = on ? beta[mp.blk * BW + mp.c0 + i] : T(0);
    al[i] = on && X ? alpha[mp.blk * BW + mp.c0 + i] : T(0);
    ca[i] = on && actv[mp.blk * BW + mp.c0 + i] != 0;
  }
  grp_stage<T>(m, R, nci, rowptr, col, gt, sh, s_ent);
  if (!on) return;
  const T* tb = Tg + static_cast<int64_t>(mp.blk) * m * BW + mp.c0;
  auto update = [&](int64_t gr, const T(&z)[W]) {
    int64_t o = (static_cast<int64_t>(mp.blk) * m + gr) * BW + mp.c0;
    T pv[W];
    vldw(pv, P + o);
    if (X) {
      T xv[W];
      vldw(xv, X + o);
#pragma unroll
      for (int i = 0; i < W; ++i) xv[i] += al[i] * pv[i];
      vst(X + o, xv);
    }
#pragma unroll
    for (int i = 0; i < W; ++i)
      if (ca[i]) pv[i] = z[i] + bt[i] * pv[i];
    vst(P + o, pv);
  };
  if constexpr (D == 0) {
    auto sweep = [&](auto staged_tag) {  // chunk i, its rows j (no divisions per row)
      constexpr bool ST = decltype(staged_tag)::value;
      for (int i = 0; i < nci; ++i) {
        const int64_t row0 = (blockIdx.x + static_cast<int64_t>(i) * gridDim.x) * R;
        const int gs = ST ? 0 : sh.gsh[i];
        for (int j = mp.rw; j < R; j += M::RW) {
          const int64_t gr = row0 + j;
          if (gr >= m) break;
          const int lr = i * R + j;
          T z[W];
          grp_row_sum<T, 8, ST>(s_ent, sh.ptr[lr], sh.ptr[lr + 1], gs, col, gt, tb, z);
          update(gr, z);
        }
      }
    };
    if (sh.staged)
      sweep(std::true_type{});
    else
      sweep(std::false_type{});
  } else {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const int warp = threadIdx.x >> 5;
    unsigned char* ring = dyn_smem + static_cast<size_t>(warp) * D * kPipeK * kPipeSlot;
    pipe_rows<T, D>(m, R, nci, mp.rw, M::RW, sh, s_ent, col, gt, tb, ring, update);
  }
}

// Loop condition of the graph-captured CG solve: keep iterating while some column is active and the
// iteration count is below it_limit (one thread).
__global__ void k_cg_continue(cudaGraphConditionalHandle handle, CgState s, int it_limit) {
  cudaGraphSetConditional(handle, (*s.n_active > 0 && *s.it < it_limit) ? 1u : 0u);
}

// p = z = D^{-1} r ; accumulate r.z and b.b (r = b at start) into start[0..C) and start[C..2C).
// Without dinv only b.b (the caller forms p and r.z with its own preconditioner).
template <class T>
__global__ void __launch_bounds__(kCgThreads) k_cg_start(int64_t m, int nb, int C, const T* __restrict__ R,
                                                           T* __restrict__ P, const T* __restrict__ dinv,
                                                           double* __restrict__ start) {
  constexpr int W = VT<T>::W, NS = Lanes<T>::NS;
  __shared__ T red[kCgWarps][kMaxChunk];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Lanes<T> L(lane);
  T rz[NS][W], bb[NS][W];
#pragma unroll
  for (int sg = 0; sg < NS; ++sg)
#pragma unroll
    for (int i = 0; i < W; ++i) rz[sg][i] = bb[sg][i] = T(0);
  const int64_t wstride = static_cast<int64_t>(gridDim.x) * kCgWarps;  // rows interleaved over all warps
  for (int64_t u = static_cast<int64_t>(blockIdx.x) * kCgWarps + warp; u < m; u += wstride) {
    T d = dinv ? dinv[u] : T(0);
#pragma unroll
    for (int sg = 0; sg < NS; ++sg) {
      if (L.block(sg) >= nb) continue;
      int64_t o = L.offset(sg, m, u);
      T rv[W], pv[W];
      vld(rv, R + o);
#pragma unroll
      for (int i = 0; i < W; ++i) {
        pv[i] = rv[i] * d;
        rz[sg][i] += rv[i] * pv[i];
        bb[sg][i] += rv[i] * rv[i];
      }
      if (dinv) vst(P + o, pv);
    }
  }
  cta_accumulate<T, NS, W>(red, rz, L, nb, C, start);
  cta_accumulate<T, NS, W>(red, bb, L, nb, C, start + C);
}

__global__ void k_cg_state0(int nb, int C, int ncols, const int32_t* __restrict__ skip, CgState s) {
  __shared__ int s_nact, s_nblk;
  if (threadIdx.x == 0) {
    s_nact = 0;
    s_nblk = 0;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double rz = s.start[c], bb = s.start[C + c];
    bool a = c < ncols && bb > 0.0 && !(skip && skip[c]);
    s.rz[c] = rz;
    s.bb[c] = bb;
    s.rr[c] = bb;
    s.act[c] = a ? 1 : 0;
    s.iters[c] = 0;
    for (int p = 0; p < 2; ++p) {
      s.pq[p * C + c] = 0.0;
      s.rzn[p * C + c] = 0.0;
      s.rra[p * C + c] = 0.0;
    }
    if (a) atomicAdd(&s_nact, 1);
  }
  __syncthreads();
  for (int cb = threadIdx.x; cb < nb; cb += blockDim.x) {
    int any = 0;
    for (int c = cb * BW; c < cb * BW + BW && c < C; ++c) any |= s.act[c];
    s.bact[cb] = any;
    if (any) atomicAdd(&s_nblk, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *s.n_active = s_nact;
    *s.it = 0;
    if (s.blog) s.blog[0] = s_nblk;
  }
}

// Scatter the sparse right-hand sides of landmark columns j0..j0+ncols-1 into block layout.
__global__ void k_scatter_rhs(int64_t m, int j0, int ncols, const int32_t* __restrict__ rptr,
                              const int32_t* __restrict__ rrow, const double* __restrict__ rval, double* __restrict__ B,
                              double sign) {
  for (int c = blockIdx.x; c < ncols; c += gridDim.x) {
    int j = j0 + c;
    int cb = c / BW, lane = c % BW;
    for (int e = rptr[j] + threadIdx.x; e < rptr[j + 1]; e += blockDim.x)
      B[(static_cast<int64_t>(cb) * m + rrow[e]) * BW + lane] += sign * rval[e];
  }
}

// acc[c] += ||column c||^2 of a block-layout FP64 array (acc zeroed by the caller)
__global__ void __launch_bounds__(kCgThreads) k_colnorm(int64_t m, int nb, int C, const double* __restrict__ X,
                                                          double* __restrict__ acc) {
  constexpr int W = 2, NS = 8;
  __shared__ double red[kCgWarps][kMaxChunk];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Lanes<double> L(lane);
  double s2[NS][W];
#pragma unroll
  for (int sg = 0; sg < NS; ++sg) s2[sg][0] = s2[sg][1] = 0.0;
  const int64_t wstride = static_cast<int64_t>(gridDim.x) * kCgWarps;  // rows interleaved over all warps
  for (int64_t u = static_cast<int64_t>(blockIdx.x) * kCgWarps + warp; u < m; u += wstride) {
#pragma unroll
    for (int sg = 0; sg < NS; ++sg) {
      if (L.block(sg) >= nb) continue;
      double v[W];
      vld(v, X + L.offset(sg, m, u));
      s2[sg][0] += v[0] * v[0];
      s2[sg][1] += v[1] * v[1];
    }
  }
  cta_accumulate<double, NS, W>(red, s2, L, nb, C, acc);
}

// Per column of a refinement step: done (residual at tolerance, or a padding column), the scale
// ||r|| (0 when done) and its reciprocal; n_todo counts the columns still to solve.
__global__ void k_refine_scale(int C, int ncols, const double* __restrict__ rn2, const double* __restrict__ bb,
                               double tol2, double* __restrict__ scale, double* __restrict__ inv,
                               int32_t* __restrict__ done, int32_t* __restrict__ n_todo) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    const bool d = c >= ncols || rn2[c] <= tol2 * bb[c];
    const double sc = d ? 0.0 : sqrt(rn2[c]);
    done[c] = d ? 1 : 0;
    scale[c] = sc;
    inv[c] = d ? 0.0 : 1.0 / sc;
    if (!d) atomicAdd(n_todo, 1);
  }
}

// Rin = R64 / ||r|| per column (0 for done columns), by the column's reciprocal scale: CTA (x, y)
// streams column block y over the x-th share of the rows, a warp per row and a lane per column.
template <class TI>
__global__ void k_refine_prepare(int64_t m, const double* __restrict__ R64, const double* __restrict__ inv,
                                 TI* __restrict__ Rin) {
  const int lane = threadIdx.x & 31;
  const double iv = inv[blockIdx.y * BW + lane];
  const int64_t base = static_cast<int64_t>(blockIdx.y) * m * BW + lane;
  const int wpc = blockDim.x >> 5;
  for (int64_t u = static_cast<int64_t>(blockIdx.x) * wpc + (threadIdx.x >> 5); u < m;
       u += static_cast<int64_t>(gridDim.x) * wpc) {
    const int64_t o = base + u * BW;
    Rin[o] = iv == 0.0 ? TI(0) : static_cast<TI>(R64[o] * iv);
  }
}

// R = B - A X over nb column blocks (block layout), each entry's sum carried in double-double and
// rounded once: products split exactly by fma (Dekker/Knuth error-free transformations), sums by
// TwoSum.  The refinement residual is then exact to about one rounding however much a row's terms
// cancel (the biharmonic rows sum to zero), so refinement can reach the correctly rounded solution
// instead of stalling at the FP64 residual's floor.  Explicit _rn intrinsics keep the compiler from
// fusing the error terms.  A warp per (block, row), a lane per column.
__global__ void __launch_bounds__(256) k_resid_dd(int64_t m, int nb, const int32_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                                  const double* __restrict__ X, const double* __restrict__ B,
                                                  double* __restrict__ R) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const int64_t total = static_cast<int64_t>(nb) * m;
  for (int64_t q = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5; q < total; q += nw) {
    const int64_t cb = q / m, u = q % m;
    const int64_t o = (cb * m + u) * BW + lane;
    const double* xb = X + cb * m * BW + lane;
    double sh = B[o], sl = 0.0;
    for (int e = rowptr[u]; e < rowptr[u + 1]; ++e) {
      const double a = val[e], x = xb[static_cast<int64_t>(col[e]) * BW];
      const double p = __dmul_rn(a, x);
      const double pe = fma(a, x, -p);  // a x - p exactly
      const double t = __dsub_rn(sh, p);
      const double bb = __dsub_rn(t, sh);
      double err = __dadd_rn(__dsub_rn(sh, __dsub_rn(t, bb)), __dsub_rn(-p, bb));  // sh - p - t exactly
      err = __dadd_rn(err, __dsub_rn(sl, pe));
      sh = __dadd_rn(t, err);
      sl = __dsub_rn(err, __dsub_rn(sh, t));
    }
    R[o] = __dadd_rn(sh, sl);
  }
}

// At or below this cg_rtol the refinement residuals are formed in double-double.  Above it the FP64
// residual (one rounding per fused multiply-add) is far from its floor, and double-double would cost
// about ten FP64 operations per nonzero on a part whose FP64 pipes are the slow ones.
constexpr double kExactResidualRtol = 1e-12;

void resid_dd(Ctx& c, int64_t m, int nb, const int32_t* rowptr, const int32_t* col, const double* val,
              const double* X, const double* B, double* R) {
  k_resid_dd<<<grid_for(static_cast<int64_t>(nb) * m * 32, 256), 256, 0, c.stream>>>(m, nb, rowptr, col, val, X, B,
                                                                                      R);
  c.launched("resid_dd");
}

// X64 += scale_c * Xin
template <class TI>
__global__ void k_refine_accumulate(int64_t m, const TI* __restrict__ Xin, const double* __restrict__ scale,
                                    double* __restrict__ X64) {
  const int lane = threadIdx.x & 31;
  const double sc = scale[blockIdx.y * BW + lane];
  if (sc == 0.0) return;  // a done column (lanes of one warp may differ; no warp-wide operation follows)
  const int64_t base = static_cast<int64_t>(blockIdx.y) * m * BW + lane;
  const int wpc = blockDim.x >> 5;
  for (int64_t u = static_cast<int64_t>(blockIdx.x) * wpc + (threadIdx.x >> 5); u < m;
       u += static_cast<int64_t>(gridDim.x) * wpc) {
    const int64_t o = base + u * BW;
    X64[o] += sc * static_cast<double>(Xin[o]);
  }
}

}  // namespace

// ---------------------------------------------------------------- host ----
//
// Two ways to the same operator P_u = -M_uu^{-1} M_ub:
//
// * direct: block-CG on M_uu, one right-hand side per landmark;
// * factored (default): M = L D^{-1} L with L = V - A (Sec. 2.2).  Splitting the
//   vertices into unknowns u and landmarks b,
//     M_uu = L_uu D_u^{-1} L_uu + L_ub D_b^{-1} L_bu,   M_ub = L_uu D_u^{-1} L_ub + L_ub D_b^{-1} L_bb,
//   and the interpolant g with g_b given satisfies, with w = D^{-1} L g,
//     L_uu w_u + L_ub w_b = 0,  D_u w_u = L_uu g_u + L_ub g_b,  D_b w_b = L_bu g_u + L_bb g_b.
//   Eliminating w_u and g_u gives, with the harmonic extension E = L_uu^{-1} A_ub (A_ub = -L_ub),
//     T = D_b + E^T D_u E,   S = L_bb - A_bu E,   Y = T^{-1} S,   P_u = E + L_uu^{-1} (D_u E Y).
//   Two block-CG solves with the pinned Laplacian L_uu (7 nonzeros per row, condition number
//   ~ (landmark spacing / edge length)^2) replace one with M_uu (19 nonzeros per row,
//   condition number ~ spacing^4), and the rest is dense landmark-space algebra.  The
//   result is checked against the FP64 residual of the original system M_uu P_u + M_ub and
//   corrected with the same factorisation (M_uu^{-1} r = L_uu^{-1} D_u (a - E T^{-1} E^T D_u a),
//   a = L_uu^{-1} r) until it meets cg_rtol.

namespace {

__global__ void k_lap_count(int64_t n, const int32_t* __restrict__ rowptr, int32_t* __restrict__ cnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    cnt[v] = rowptr[v + 1] - rowptr[v] + 1;
}

// L = V - A as a vertex CSR with the diagonal in its sorted place
__global__ void k_lap_fill(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const double* __restrict__ A, const double* __restrict__ V, const int32_t* __restrict__ lrow,
                           int32_t* __restrict__ lcol, double* __restrict__ lval) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int q = lrow[v];
    bool placed = false;
    for (int e = rowptr[v]; e < rowptr[v + 1]; ++e) {
      if (!placed && col[e] > v) {
        lcol[q] = static_cast<int32_t>(v);
        lval[q++] = V[v];
        placed = true;
      }
      lcol[q] = col[e];
      lval[q++] = -A[e];
    }
    if (!placed) {
      lcol[q] = static_cast<int32_t>(v);
      lval[q] = V[v];
    }
  }
}

// dense l x l block of a vertex CSR on the landmarks: B[j][k] = X[b_j][b_k]
__global__ void k_landmark_block_of(int l, const int32_t* __restrict__ idx, const int32_t* __restrict__ rowptr,
                                    const int32_t* __restrict__ col, const double* __restrict__ val,
                                    const int32_t* __restrict__ lmcol, double* __restrict__ B) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < l; j += gridDim.x * blockDim.x) {
    int b = idx[j];
    for (int e = rowptr[b]; e < rowptr[b + 1]; ++e) {
      int k = lmcol[col[e]];
      if (k >= 0) B[static_cast<int64_t>(j) * l + k] = val[e];
    }
  }
}

__global__ void k_gather(int64_t count, const int32_t* __restrict__ ids, const double* __restrict__ src,
                         double* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[ids[i]];
}

// y += alpha x over `count` elements
__global__ void k_axpy(int64_t count, double alpha, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x)
    y[q] += alpha * x[q];
}

// block-layout rows scaled: y[u][.] = d[u] * x[u][.]
__global__ void k_scale_rows(int64_t m, int nb, const double* __restrict__ d, const double* __restrict__ x,
                             double* __restrict__ y) {
  int64_t total = static_cast<int64_t>(nb) * m * BW;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
    y[q] = d[(q / BW) % m] * x[q];
}

// A sparse SPD system on the unknowns (CSR), with an FP32 copy and the inverse diagonal.
struct Mat {
  int64_t m = 0, nnz = 0;
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
  double* dinv = nullptr;
  float* dinv32 = nullptr;
  TiledPattern tp;  // row tiles for the staged product (ntiles == 0: plain product)
  bool staged = false;  // products staged through shared memory (SBHA_SPMM_STAGED), else row gathers
  bool contig = false;  // row gathers over contiguous row ranges per CTA (the unknowns are in locality order)
  int chunk = 0;        // gather products' launch shape: 0 autotuned, 16/32/64 rows per chunk, -1 contiguous
  int gather = 0;       // 0 the tuner picks the register or the pipelined gather, 1 register only, 2 pipelined only
  int depth = 0;        // pipelined gather: rows in flight per warp, 0 tuned, 2 or 4
  TiledPattern gtp;     // 64-row tiles of the TMA gather product (ntiles == 0: none)
  int tma = 0;          // FP32 products: 0 never TMA, 1 a candidate of the tuner, 2 always
};

struct Rhs {  // one sparse column over the unknown rows per landmark
  int32_t* ptr = nullptr;
  int32_t* row = nullptr;
  double* val = nullptr;
};

struct Sys {
  int64_t n = 0, m = 0;
  int32_t l = 0;
  int32_t* lmcol = nullptr;
  int32_t* uidx = nullptr;   // vertex -> unknown (meaningful for unknown vertices only)
  int32_t* uvert = nullptr;  // unknown -> vertex
  int32_t* uord = nullptr;   // unknowns in ascending vertex order
  Mat M;                  // M_uu
  Rhs Mb;                 // -M_ub e_j
  Mat L;                  // L_uu
  Rhs Ab;                 // A_ub e_j = -L_ub e_j
  double* Lbb = nullptr;  // l x l
  double* Du = nullptr;
  double* Db = nullptr;
};

Mat restrict_to_unknowns(Ctx& c, const DevCSR& X, const Sys& s) {
  const int T = 256;
  Mat A;
  A.m = s.m;
  int32_t* cnt = c.alloc<int32_t>(s.m);
  k_muu_count<<<grid_for(s.m, T), T, 0, c.stream>>>(s.m, s.uvert, X.rowptr, X.col, s.lmcol, cnt);
  c.launched("restrict_count");
  A.rowptr = c.alloc<int32_t>(s.m + 1);
  A.nnz = exclusive_scan(c, cnt, A.rowptr, s.m);
  A.col = c.alloc<int32_t>(A.nnz);
  A.val = c.alloc<double>(A.nnz);
  A.val32 = c.alloc<float>(A.nnz);
  A.dinv = c.alloc<double>(s.m);
  A.dinv32 = c.alloc<float>(s.m);
  k_muu_fill<<<grid_for(s.m, T), T, 0, c.stream>>>(s.m, s.uvert, X.rowptr, X.col, X.val, s.lmcol, s.uidx, A.rowptr,
                                                    A.col, A.val, A.val32, A.dinv, A.dinv32);
  c.launched("restrict_fill");
  c.free(cnt);
  return A;
}

// Column b_j of X at the unknown rows, negated: out_j = -X_ub e_j.
Rhs landmark_columns(Ctx& c, const DevCSR& X, const int32_t* idx, const Sys& s) {
  const int T = 256;
  Rhs r;
  int32_t* cnt = c.alloc<int32_t>(s.l);
  k_rhs_count<<<grid_for(s.l, T), T, 0, c.stream>>>(s.l, idx, X.rowptr, X.col, s.lmcol, cnt);
  c.launched("rhs_count");
  r.ptr = c.alloc<int32_t>(s.l + 1);
  int64_t nnz = exclusive_scan(c, cnt, r.ptr, s.l);
  r.row = c.alloc<int32_t>(nnz);
  r.val = c.alloc<double>(nnz);
  k_rhs_fill<<<grid_for(s.l, T), T, 0, c.stream>>>(s.l, idx, X.rowptr, X.col, X.val, s.lmcol, s.uidx, r.ptr, r.row,
                                                    r.val);
  c.launched("rhs_fill");
  c.free(cnt);
  return r;
}

Sys build_system(Ctx& c, const DevGraph& g, const DevCSR& M, const int32_t* idx, int32_t l, bool factored,
                 bool staged) {
  const int T = 256;
  Sys s;
  s.n = M.rows;
  s.l = l;
  s.lmcol = c.alloc<int32_t>(s.n);
  SBHA_CUDA(cudaMemsetAsync(s.lmcol, 0xff, sizeof(int32_t) * s.n, c.stream));
  k_mark_landmarks<<<grid_for(l, T), T, 0, c.stream>>>(idx, l, static_cast<int>(s.n), s.lmcol, c.d_err);
  c.launched("mark_landmarks");
  c.check_device("operator");
  int32_t* flag = c.alloc<int32_t>(s.n);
  k_unknown_flags<<<grid_for(s.n, T), T, 0, c.stream>>>(s.n, s.lmcol, flag);
  c.launched("unknown_flags");
  s.uidx = c.alloc<int32_t>(s.n + 1);
  s.m = exclusive_scan(c, flag, s.uidx, s.n);
  int32_t* asc = c.alloc<int32_t>(std::max<int64_t>(s.m, 1));
  k_unknown_verts<<<grid_for(s.n, T), T, 0, c.stream>>>(s.n, s.lmcol, s.uidx, asc);
  c.launched("unknown_verts");
  // unknowns numbered along a Morton curve through their positions: consecutive rows are
  // surface patches (the staged products rely on it); uord keeps ascending-vertex order
  s.uvert = c.alloc<int32_t>(std::max<int64_t>(s.m, 1));
  s.uord = c.alloc<int32_t>(std::max<int64_t>(s.m, 1));
  if (s.m > 0) {
    int32_t* perm = c.alloc<int32_t>(s.m);
    locality_order(c, s.m, asc, g.xyz, perm);
    k_renumber<<<grid_for(s.m, T), T, 0, c.stream>>>(s.m, perm, asc, s.uvert, s.uidx, s.uord);
    c.launched("renumber");
    c.free(perm);
  }
  c.free(asc);
  c.free(flag);
  if (s.m == 0) return s;
  s.M = restrict_to_unknowns(c, M, s);
  s.Mb = landmark_columns(c, M, idx, s);
  if (!factored && staged) {
    s.M.tp = build_tiles(c, s.m, s.M.nnz, s.M.rowptr, s.M.col);
    s.M.staged = true;
  }
  if (factored) {
    DevCSR Lv;
    Lv.rows = Lv.cols = s.n;
    int32_t* cnt = c.alloc<int32_t>(s.n);
    k_lap_count<<<grid_for(s.n, T), T, 0, c.stream>>>(s.n, g.rowptr, cnt);
    c.launched("lap_count");
    Lv.rowptr = c.alloc<int32_t>(s.n + 1);
    Lv.nnz = exclusive_scan(c, cnt, Lv.rowptr, s.n);
    Lv.col = c.alloc<int32_t>(Lv.nnz);
    Lv.val = c.alloc<double>(Lv.nnz);
    k_lap_fill<<<grid_for(s.n, T), T, 0, c.stream>>>(s.n, g.rowptr, g.col, g.A, g.V, Lv.rowptr, Lv.col, Lv.val);
    c.launched("lap_fill");
    c.free(cnt);
    s.L = restrict_to_unknowns(c, Lv, s);
    if (staged) {
      s.L.tp = build_tiles(c, s.m, s.L.nnz, s.L.rowptr, s.L.col);
      s.L.staged = true;
    }
    s.Ab = landmark_columns(c, Lv, idx, s);
    s.Lbb = c.zeros<double>(static_cast<size_t>(l) * l);
    k_landmark_block_of<<<grid_for(l, 128), 128, 0, c.stream>>>(l, idx, Lv.rowptr, Lv.col, Lv.val, s.lmcol, s.Lbb);
    c.launched("landmark_block_of");
    s.Du = c.alloc<double>(s.m);
    s.Db = c.alloc<double>(l);
    k_gather<<<grid_for(s.m, T), T, 0, c.stream>>>(s.m, s.uvert, g.D, s.Du);
    c.launched("gather");
    k_gather<<<grid_for(l, T), T, 0, c.stream>>>(l, idx, g.D, s.Db);
    c.launched("gather");
  }
  return s;
}

// CTAs of the row-parallel CG kernels: four per SM, at least two rows per warp.
int cg_grid(int64_t m) {
  int64_t g = (m + kCgWarps * 2 - 1) / (kCgWarps * 2);
  if (g > 4 * num_sms()) g = 4 * num_sms();
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

// Row mapping of the block-group kernels (grp_stage): one wave of four CTAs per SM, at most
// kGrpRows rows per CTA, in chunks of about `target` rows spread over the grid (0: one contiguous
// range per CTA).
struct GrpPlan {
  int R = 16, nci = 1;
  unsigned grid = 1;
};
GrpPlan grp_plan(int64_t m, int target, int cps = 4) {
  GrpPlan p;
  const int64_t wave = static_cast<int64_t>(cps) * num_sms();  // one wave of cps CTAs per SM
  int64_t per = std::min<int64_t>(kGrpRows, std::max<int64_t>(16, (m + wave - 1) / wave));
  int nci = target > 0 ? static_cast<int>((per + target / 2) / target) : 1;
  nci = std::max(1, std::min(kGrpChunks, nci));
  int R = static_cast<int>((per + nci - 1) / nci);
  if (nci * R > kGrpRows) {
    nci = 1;
    R = static_cast<int>(per);
  }
  int64_t nchunks = (m + R - 1) / R;
  p.R = R;
  p.nci = nci;
  p.grid = static_cast<unsigned>(std::max<int64_t>(1, (nchunks + nci - 1) / nci));
  return p;
}

constexpr int kGrpChunkRows = 32;  // default: the fastest on the 50k-vertex torus
// candidate launch shapes: rows per chunk (0 = one contiguous range per CTA) and pipeline depth
// (0 = register gather)
struct GrpCand {
  int target, depth, occ;  // occ: resident CTAs per SM of the register gather (4: 8 neighbours in
                           // flight per row, 6 or 8: 4 in flight with fewer registers)
  bool tma = false;        // the TMA gather product (FP32, its own tiles)
};
constexpr GrpCand kGrpCandidates[] = {{16, 0, 4},  {32, 0, 4}, {64, 0, 4}, {0, 0, 4},  {32, 0, 6}, {64, 0, 6},
                                      {32, 0, 8},  {32, 2, 4}, {32, 4, 4}, {64, 2, 4}, {16, 4, 4},
                                      {32, 0, 4, true}};
struct GrpKey {
  int64_t m, nnz;
  int nb, bytes, gather, depth, chunk, tma;  // chunk, gather, depth, tma: the caller's restrictions
  bool operator<(const GrpKey& o) const {
    return std::tie(m, nnz, nb, bytes, gather, depth, chunk, tma) <
           std::tie(o.m, o.nnz, o.nb, o.bytes, o.gather, o.depth, o.chunk, o.tma);
  }
};
struct GrpChoice {
  int target = kGrpChunkRows;
  int depth = 0;
  int occ = 4;
  bool tma = false;  // the TMA gather product; target/depth/occ then give the shape of the kernels
                     // that share the register gather's mapping (the fused direction update)
  double us = 0.0;
};
std::mutex g_grp_mu;
std::map<GrpKey, GrpChoice> g_grp_tuned;

// The TMA product is open to FP32 products of a matrix with its tiles.
int grp_tma(const Mat& A, int bytes) { return bytes == 4 && A.gtp.ntiles > 0 ? A.tma : 0; }

GrpKey grp_key(const Mat& A, int nb, int bytes) {
  return GrpKey{A.m, A.nnz, nb, bytes, A.gather, A.depth, A.chunk, grp_tma(A, bytes)};
}

bool grp_lookup(const GrpKey& k, GrpChoice* out) {
  std::lock_guard<std::mutex> lk(g_grp_mu);
  auto it = g_grp_tuned.find(k);
  if (it == g_grp_tuned.end()) return false;
  *out = it->second;
  return true;
}

// Reported in sbha_stats: the FP32 products' shape when the call has them (the inner solves), else
// the FP64 one.
void grp_note(const GrpChoice& ch, bool fp32) {
  sbha_stats& st = thread_stats();
  static thread_local bool have_fp32 = false;
  if (st.spmm_tuned_shapes == 0) have_fp32 = false;  // a new call: the stats were cleared
  if (fp32 || !have_fp32) {
    st.spmm_chunk_rows = ch.target;
    st.spmm_pipeline_depth = ch.depth;
    st.spmm_ctas_per_sm = ch.occ;
    st.spmm_tuned_us = ch.us;
    st.spmm_tma = ch.tma ? 1 : 0;
    have_fp32 = have_fp32 || fp32;
  }
  std::lock_guard<std::mutex> lk(g_grp_mu);
  st.spmm_tuned_shapes = static_cast<int32_t>(g_grp_tuned.size());
}

// Dynamic shared memory of the pipelined kernels (their rings), set once per instantiation.
template <class T, int D>
void pipe_attrs() {
  static std::once_flag once;
  std::call_once(once, [] {
    SBHA_CUDA(cudaFuncSetAttribute(k_spmm_pipe<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(pipe_ring_bytes<D>())));
    SBHA_CUDA(cudaFuncSetAttribute(k_cg_p_gt<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(pipe_ring_bytes<D>())));
  });
}

template <class T>
void launch_spmm(Ctx& c, const Mat& A, int nb, int C, const T* val, const T* x, T* y, T alpha, double* acc,
                 const int32_t* blk_act, bool self_dot, const GrpPlan& gp, int depth, int occ, const char* what) {
  if (depth == 0 && occ == 4) {
    k_spmm_grp<T, 8, 4><<<gp.grid, kCgThreads, 0, c.stream>>>(A.m, nb, A.rowptr, A.col, val, x, y, alpha, acc, C,
                                                              blk_act, self_dot, gp.R, gp.nci);
  } else if (depth == 0 && occ == 6) {
    k_spmm_grp<T, 4, 6><<<gp.grid, kCgThreads, 0, c.stream>>>(A.m, nb, A.rowptr, A.col, val, x, y, alpha, acc, C,
                                                              blk_act, self_dot, gp.R, gp.nci);
  } else if (depth == 0) {
    k_spmm_grp<T, 4, 8><<<gp.grid, kCgThreads, 0, c.stream>>>(A.m, nb, A.rowptr, A.col, val, x, y, alpha, acc, C,
                                                              blk_act, self_dot, gp.R, gp.nci);
  } else if (depth == 2) {
    pipe_attrs<T, 2>();
    k_spmm_pipe<T, 2><<<gp.grid, kCgThreads, pipe_ring_bytes<2>(), c.stream>>>(A.m, nb, A.rowptr, A.col, val, x, y,
                                                                               alpha, acc, C, blk_act, self_dot,
                                                                               gp.R, gp.nci);
  } else {
    pipe_attrs<T, 4>();
    k_spmm_pipe<T, 4><<<gp.grid, kCgThreads, pipe_ring_bytes<4>(), c.stream>>>(A.m, nb, A.rowptr, A.col, val, x, y,
                                                                               alpha, acc, C, blk_act, self_dot,
                                                                               gp.R, gp.nci);
  }
  c.launched(what);
}

// Autotuner of the launch shape: the first product with a matrix shape (rows, nonzeros, column
// blocks, value type, the caller's restrictions) times every admissible candidate in five
// interleaved rounds with CUDA events and keeps the fastest median for the process.  Every candidate sums each row in the same
// order, so the product is bit-identical whichever wins; trial launches skip the dot-product
// accumulator.  Not tuned while the stream is being captured (the default then).
template <class T>
GrpChoice grp_tune(Ctx& c, const Mat& A, int nb, int C, const T* val, const T* x, T* y, T alpha) {
  GrpKey key = grp_key(A, nb, static_cast<int>(sizeof(T)));
  const int tma = key.tma;
  GrpChoice ch;
  if (A.gather == 2) ch.depth = A.depth > 0 ? A.depth : 2;
  if (A.chunk != 0) ch.target = A.chunk > 0 ? A.chunk : 0;
  ch.tma = tma == 2;
  if (grp_lookup(key, &ch)) return ch;
  if (tma == 2) {  // the TMA product asked for: nothing to time
    std::lock_guard<std::mutex> lk(g_grp_mu);
    g_grp_tuned.emplace(key, ch);
    return ch;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SBHA_CUDA(cudaStreamIsCapturing(c.stream, &cap));
  if (cap != cudaStreamCaptureStatusNone) return ch;
  cudaEvent_t e0, e1;
  SBHA_CUDA(cudaEventCreate(&e0));
  SBHA_CUDA(cudaEventCreate(&e1));
  // the admissible candidates, then kRounds rounds in which each runs once (interleaved, so that no
  // candidate always follows the same one or always meets a warm L2); the median of its rounds
  std::vector<GrpCand> cands;
  for (const GrpCand& cand : kGrpCandidates) {
    if (cand.tma) {  // under AUTO, for FP32 products with tiles, unless the caller fixed the gather's shape
      if (tma == 1 && A.chunk == 0 && A.gather == 0 && std::is_same<T, float>::value) cands.push_back(cand);
      continue;
    }
    if (A.chunk != 0 && cand.target != (A.chunk > 0 ? A.chunk : 0)) continue;  // shape fixed by the caller
    // one contiguous range per CTA only when asked for: it can win a trial of the product alone, but the
    // fused direction update shares the mapping and there it re-reads 1.56x its vector from DRAM
    if (A.chunk == 0 && cand.target == 0) continue;
    // the pipelined gather runs only when asked for: it measured 1.7-2.8x slower than the register
    // gather on the 50k-vertex torus (its shared-memory ring halves the resident warps)
    if (A.gather != 2 && cand.depth != 0) continue;
    if (A.gather == 2 && cand.depth == 0) continue;
    if (A.depth != 0 && cand.depth != 0 && cand.depth != A.depth) continue;
    cands.push_back(cand);
  }
  constexpr int kRounds = 5;
  std::vector<std::vector<float>> times(cands.size());
  std::vector<bool> ok(cands.size(), true);
  for (int r = 0; r < kRounds; ++r)
    for (size_t k = 0; k < cands.size(); ++k) {
      if (!ok[k]) continue;
      const GrpCand& cand = cands[k];
      SBHA_CUDA(cudaEventRecord(e0, c.stream));
      if (cand.tma) {
        if constexpr (std::is_same<T, float>::value)
          ok[k] = spmm_tma(c, A.gtp, nb, val, x, y, alpha, nullptr, nullptr, false);
      } else {
        launch_spmm<T>(c, A, nb, C, val, x, y, alpha, nullptr, nullptr, false, grp_plan(A.m, cand.target, cand.occ),
                       cand.depth, cand.occ, "spmm_tune");
      }
      SBHA_CUDA(cudaEventRecord(e1, c.stream));
      SBHA_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      SBHA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      times[k].push_back(ms);
    }
  double best = 0.0, best_tma = 0.0;
  for (size_t k = 0; k < cands.size(); ++k) {
    if (!ok[k] || times[k].empty()) continue;
    std::sort(times[k].begin(), times[k].end());
    const double us = 1e3 * times[k][times[k].size() / 2];
    if (cands[k].tma) {
      best_tma = us;
    } else if (best == 0.0 || us < best) {
      best = us;
      ch.target = cands[k].target;
      ch.depth = cands[k].depth;
      ch.occ = cands[k].occ;
      ch.us = us;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_tma > 0.0 && best_tma < best) {  // the register shape stays for the kernels sharing its mapping
    ch.tma = true;
    ch.us = best_tma;
  }
  std::lock_guard<std::mutex> lk(g_grp_mu);
  g_grp_tuned.emplace(key, ch);
  return ch;
}

// The tuned (or default) choice of a matrix shape, for the kernels that share the mapping.
GrpChoice grp_choice_for(const Mat& A, int nb, int bytes) {
  GrpChoice ch;
  if (!grp_lookup(grp_key(A, nb, bytes), &ch)) {
    if (A.chunk != 0) ch.target = A.chunk > 0 ? A.chunk : 0;
    if (A.gather == 2) ch.depth = A.depth > 0 ? A.depth : 2;
  }
  return ch;
}

// y = alpha A x (+ the column dot products of k_spmm_grp): staged through shared memory when A has tiles.
template <class T>
void spmm(Ctx& c, const Mat& A, int nb, int C, const T* val, const T* x, T* y, T alpha, double* acc,
          const int32_t* blk_act, bool self_dot, const char* what) {
  if (A.tp.ntiles > 0 && A.staged) {
    spmm_tiled<T>(c, c.stream, A.tp, nb, val, x, y, alpha, acc, blk_act, self_dot);
  } else {
    if (A.m <= 0) return;
    GrpChoice ch = grp_tune<T>(c, A, nb, C, val, x, y, alpha);
    grp_note(ch, sizeof(T) == 4);
    if constexpr (std::is_same<T, float>::value) {
      if (ch.tma && spmm_tma(c, A.gtp, nb, val, x, y, alpha, acc, blk_act, self_dot)) return;
    }
    launch_spmm<T>(c, A, nb, C, val, x, y, alpha, acc, blk_act, self_dot, grp_plan(A.m, ch.target, ch.occ), ch.depth,
                   ch.occ, what);
  }
}

template <class T>
struct CgWork {
  T *X, *R, *P, *Q;
  T* Z = nullptr;  // preconditioned residual when M^{-1} = G^T G (allocated on first use)
  CgState st;
  int32_t* h_nact;  // pinned, 2 slots: the active-column count and the iteration counter
};

// CUDA-event timing of the conjugate-gradient kernels (opts.timing == 2).  Events are
// recorded on the launching stream around each launch; their durations are read after
// the periodic synchronisation and summed per kernel with the launch's algorithmic bytes.
struct KernelClock {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> which;
  std::vector<int> iter;  // iteration of the launch (for active-block lookup), -1 = all blocks
  int used = 0;
  explicit KernelClock(bool enabled) : on(enabled) {}
  ~KernelClock() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  void begin(Ctx& c) {
    if (!on) return;
    if (static_cast<int>(ev.size()) < 2 * (used + 1)) {
      cudaEvent_t a, b;
      SBHA_CUDA(cudaEventCreate(&a));
      SBHA_CUDA(cudaEventCreate(&b));
      ev.push_back(a);
      ev.push_back(b);
      which.push_back(0);
      iter.push_back(0);
    }
    SBHA_CUDA(cudaEventRecord(ev[2 * used], c.stream));
  }
  void end(Ctx& c, int k, int it) {
    if (!on) return;
    SBHA_CUDA(cudaEventRecord(ev[2 * used + 1], c.stream));
    which[used] = k;
    iter[used] = it;
    ++used;
  }
  // After a stream synchronisation: fold the recorded launches into the thread statistics.
  template <class F>
  void harvest(const std::vector<int32_t>& blog, int nb, F bytes) {
    if (!on) return;
    sbha_stats& st = thread_stats();
    for (int i = 0; i < used; ++i) {
      float ms = 0.f;
      SBHA_CUDA(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
      int k = which[i];
      int a = (iter[i] >= 0 && iter[i] < static_cast<int>(blog.size())) ? blog[iter[i]] : nb;
      st.cg_kernel_launches[k] += 1;
      st.cg_kernel_ms[k] += ms;
      st.cg_kernel_bytes[k] += bytes(k, a);
    }
    used = 0;
  }
};

// Runs CG on the block-layout system A X = R (R holds the right-hand side, X is zeroed),
// preconditioned by D^{-1} (dinv) or, when g is given, by G^T G with G and G^T stored on
// A's pattern (g, gt).  Returns the largest per-column iteration count; columns flagged in
// `skip` do not run.
template <class T>
int cg_run(Ctx& c, const Mat& A, const T* val, const T* dinv, const T* g, const T* gt, int C, int ncols, double rtol,
           int max_iter, CgWork<T>& w, const int32_t* skip, bool* converged) {
  int64_t m = A.m;
  int nb = C / BW;
  int G = cg_grid(m);
  // learned preconditioner on the gather path: the G^T product is fused into the direction update
  const bool fuse_gt = g && !(A.tp.ntiles > 0 && A.staged);
  GrpPlan gp = grp_plan(m, kGrpChunkRows);  // set after the first product (which tunes the shape)
  GrpChoice gch;
  bool gch_set = false;
  const dim3 sg = stream_grid(m, nb);  // the block-streaming vector kernels
  // k_cg_xr holds four rows' loads per thread (more registers): its grid is one wave at its occupancy
  static const int xr_per_sm = [] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cg_xr<T>, kCgThreads, 0) != cudaSuccess) {
      cudaGetLastError();
      n = 4;
    }
    return std::max(n, 1);
  }();
  const dim3 sgx = stream_grid(m, nb, xr_per_sm);
  KernelClock clk(c.timing >= 2);
  int32_t* blog = nullptr;
  std::vector<int32_t> hblog;
  if (clk.on) blog = c.alloc<int32_t>(max_iter + 1);
  w.st.blog = blog;
  const double sT = sizeof(T);
  auto bytes = [&](int k, int a) -> double {
    double mc = static_cast<double>(m) * BW * a * sT;  // one vector over the active blocks
    if (k == 0) return 4.0 * (m + 1) + A.nnz * (4.0 + sT) + 2.0 * mc;
    if (k == 1) return fuse_gt ? 3.0 * mc : 6.0 * mc + m * sT;  // fused: r and q only
    if (fuse_gt) return 4.0 * (m + 1) + A.nnz * (4.0 + sT) + 5.0 * mc;  // gather t, read and write p and x
    return 3.0 * mc + m * sT;
  };
  SBHA_CUDA(cudaMemsetAsync(w.X, 0, sizeof(T) * m * C, c.stream));
  SBHA_CUDA(cudaMemsetAsync(w.st.start, 0, sizeof(double) * 2 * C, c.stream));
  SBHA_CUDA(cudaMemsetAsync(w.st.fail, 0, sizeof(int32_t), c.stream));
  k_cg_start<T><<<G, kCgThreads, 0, c.stream>>>(m, nb, C, w.R, w.P, g ? nullptr : dinv, w.st.start);
  c.launched("cg_start");
  if (g) {  // p = G^T (G r), r.z = ||G r||^2
    spmm<T>(c, A, nb, C, g, w.R, w.Q, T(1), w.st.start, nullptr, true, "cg_precond");
    spmm<T>(c, A, nb, C, gt, w.Q, w.P, T(1), nullptr, nullptr, false, "cg_precond");
  }
  k_cg_state0<<<1, 512, 0, c.stream>>>(nb, C, ncols, skip, w.st);
  c.launched("cg_state0");
  double tol2 = rtol * rtol;
  int it = 0;
  const int check_every = 8;
  *converged = false;
  // After the first batch (which also tunes the product shapes) the rest of the solve can run as one
  // CUDA graph: a WHILE node whose body is two iterations and k_cg_continue, so the loop is decided
  // on the device from the active-column count, without a host round trip per batch.  Not with
  // per-kernel timing, on the legacy default stream, or inside a caller's capture.
  bool graph_ok = !clk.on && c.stream != nullptr && c.graphs;
  if (graph_ok) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    SBHA_CUDA(cudaStreamIsCapturing(c.stream, &cap));
    graph_ok = cap == cudaStreamCaptureStatusNone;
  }
  bool graph_done = false;
  auto iteration = [&](int it_) {
      int cur = it_ & 1;
      clk.begin(c);
      spmm<T>(c, A, nb, C, val, w.P, w.Q, T(1), w.st.pq + cur * C, w.st.bact + cur * nb, false, "cg_spmm");
      clk.end(c, 0, it_);
      clk.begin(c);
      k_cg_xr<T><<<sgx, kCgThreads, 0, c.stream>>>(m, nb, C, cur, fuse_gt ? nullptr : w.X, w.R, w.P, w.Q,
                                                  g ? nullptr : dinv, w.st);
      c.launched("cg_xr");
      clk.end(c, 1, it_);
      if (g) {  // z = G^T (G r) over the active blocks; r.z = ||G r||^2 (Q is free after the update)
        clk.begin(c);
        spmm<T>(c, A, nb, C, g, w.R, w.Q, T(1), w.st.rzn + cur * C, w.st.bact + cur * nb, true, "cg_precond");
        clk.end(c, 0, it_);
        if (!fuse_gt) {
          clk.begin(c);
          spmm<T>(c, A, nb, C, gt, w.Q, w.Z, T(1), nullptr, w.st.bact + cur * nb, false, "cg_precond");
          clk.end(c, 0, it_);
        }
      }
      clk.begin(c);
      if (fuse_gt) {  // p = G^T t + beta p in one pass (t = G r in Q)
        if (!gch_set) {  // after the first product, which tuned the shape
          gch = grp_choice_for(A, nb, static_cast<int>(sizeof(T)));
          gp = grp_plan(m, gch.target);
          gch_set = true;
        }
        if (gch.depth == 0) {
          k_cg_p_gt<T, 0><<<gp.grid, kCgThreads, 0, c.stream>>>(m, nb, C, cur, tol2, A.rowptr, A.col, gt, w.Q, w.P,
                                                                 w.X, w.st, gp.R, gp.nci);
        } else if (gch.depth == 2) {
          pipe_attrs<T, 2>();
          k_cg_p_gt<T, 2><<<gp.grid, kCgThreads, pipe_ring_bytes<2>(), c.stream>>>(
              m, nb, C, cur, tol2, A.rowptr, A.col, gt, w.Q, w.P, w.X, w.st, gp.R, gp.nci);
        } else {
          pipe_attrs<T, 4>();
          k_cg_p_gt<T, 4><<<gp.grid, kCgThreads, pipe_ring_bytes<4>(), c.stream>>>(
              m, nb, C, cur, tol2, A.rowptr, A.col, gt, w.Q, w.P, w.X, w.st, gp.R, gp.nci);
        }
      } else {
        k_cg_p<T><<<sg, kCgThreads, 0, c.stream>>>(m, nb, C, cur, tol2, w.R, w.P, dinv, g ? w.Z : nullptr, w.st);
      }
      c.launched("cg_p");
      clk.end(c, 2, it_);
  };
  while (it < max_iter) {
    if (graph_done) break;
    if (graph_ok && it > 0 && it % 2 == 0 && max_iter - it >= 2) {
      // the remaining iterations on the device (the body keeps the parity sequence 0, 1)
      cudaGraph_t graph = nullptr, body = nullptr;
      cudaGraphExec_t exec = nullptr;
      cudaGraphConditionalHandle handle;
      SBHA_CUDA(cudaGraphCreate(&graph, 0));
      SBHA_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      SBHA_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
      body = cp.conditional.phGraph_out[0];
      SBHA_CUDA(cudaStreamBeginCaptureToGraph(c.stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      const int64_t before = c.launches;
      iteration(0);
      iteration(1);
      k_cg_continue<<<1, 1, 0, c.stream>>>(handle, w.st, max_iter);
      c.launched("cg_continue");
      const int64_t per_body = c.launches - before;  // kernel nodes of one body run
      cudaGraph_t captured = nullptr;
      SBHA_CUDA(cudaStreamEndCapture(c.stream, &captured));
      SBHA_CUDA(cudaGraphInstantiate(&exec, graph, 0));
      SBHA_CUDA(cudaGraphLaunch(exec, c.stream));
      SBHA_CUDA(cudaGraphExecDestroy(exec));
      SBHA_CUDA(cudaGraphDestroy(graph));
      graph_done = true;
      // the launch count covers every body run: the device counter says how many iterations ran
      int32_t* h_it = w.h_nact + 1;
      SBHA_CUDA(cudaMemcpyAsync(h_it, w.st.it, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
      SBHA_CUDA(cudaStreamSynchronize(c.stream));
      const int runs = std::max(1, (*h_it - it + 1) / 2);
      c.launches += (runs - 1) * per_body;
      it = *h_it;
    } else {
      int batch = std::min(check_every, max_iter - it);
      for (int k = 0; k < batch; ++k, ++it) iteration(it);
    }
    SBHA_CUDA(cudaMemcpyAsync(w.h_nact, w.st.n_active, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    if (clk.on) {
      hblog.resize(it + 1);
      SBHA_CUDA(cudaMemcpyAsync(hblog.data(), blog, sizeof(int32_t) * (it + 1), cudaMemcpyDeviceToHost, c.stream));
    }
    SBHA_CUDA(cudaStreamSynchronize(c.stream));
    clk.harvest(hblog, nb, bytes);
    if (*w.h_nact == 0) {
      *converged = true;
      break;
    }
  }
  w.st.blog = nullptr;
  std::vector<int32_t> iters(C);
  int32_t h_fail = 0;
  SBHA_CUDA(cudaMemcpyAsync(iters.data(), w.st.iters, sizeof(int32_t) * C, cudaMemcpyDeviceToHost, c.stream));
  SBHA_CUDA(cudaMemcpyAsync(&h_fail, w.st.fail, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  SBHA_CUDA(cudaStreamSynchronize(c.stream));
  c.check_device("block-CG");      // a product kernel's bounded wait that gave up is an error of its own
  if (h_fail) *converged = false;  // a column went non-finite: its result must not be used
  if (blog) c.free(blog);
  int mx = 0;
  for (int q = 0; q < ncols; ++q) mx = std::max(mx, iters[q]);
  return mx;
}

template <class T>
CgWork<T> cg_alloc(Ctx& c, int64_t m, int C, int32_t* h_pinned) {
  CgWork<T> w;
  int nb = C / BW;
  int G = cg_grid(m);
  w.X = c.alloc<T>(m * C);
  w.R = c.alloc<T>(m * C);
  w.P = c.alloc<T>(m * C);
  w.Q = c.alloc<T>(m * C);
  w.st.rz = c.alloc<double>(2 * C);
  w.st.act = c.alloc<int32_t>(2 * C);
  w.st.bact = c.alloc<int32_t>(2 * nb);
  w.st.bb = c.alloc<double>(C);
  w.st.rr = c.alloc<double>(C);
  w.st.iters = c.alloc<int32_t>(C);
  w.st.n_active = c.alloc<int32_t>(1);
  w.st.it = c.alloc<int32_t>(1);
  w.st.blog = nullptr;
  w.st.pq = c.alloc<double>(2 * C);
  w.st.rzn = c.alloc<double>(2 * C);
  w.st.rra = c.alloc<double>(2 * C);
  w.st.start = c.alloc<double>(2 * C);
  w.st.fail = c.alloc<int32_t>(1);
  (void)G;
  w.h_nact = h_pinned;
  return w;
}

// Column norms^2 of a block-layout FP64 array into out[C].
void column_norms(Ctx& c, int64_t m, int C, const double* X, double* out) {
  SBHA_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * C, c.stream));
  k_colnorm<<<cg_grid(m), kCgThreads, 0, c.stream>>>(m, C / BW, C, X, out);
  c.launched("colnorm");
}

struct Outcome {
  int iterations = 0;
  int refinements = 0;
  double max_rel = 0.0;
  bool converged = true;
};

// Block solves A X = B (C columns, block layout, B dense FP64) to an FP64 residual of
// rtol ||b_j|| per column: inner CG in FP64 or FP32, outer FP64 residual refinement.
struct BlockSolver {
  Ctx& c;
  const Mat& A;
  int C, nb, G;
  bool mixed;
  const sbha_opts& o;
  int32_t* h;
  double *R64, *scale, *inv_scale, *rn2, *bb;
  int32_t* done;
  CgWork<double> w64{};
  CgWork<float> w32{};
  const LearnedPrecond* lp = nullptr;  // M^{-1} = G^T G when set, else Jacobi
  bool fell_back = false;              // a preconditioned inner solve failed: Jacobi from then on
  bool exact;                          // refinement residuals in double-double (cg_rtol <= kExactResidualRtol)

  BlockSolver(Ctx& ctx, const Mat& mat, int cols, bool mx, const sbha_opts& opts, int32_t* pinned)
      : c(ctx), A(mat), C(cols), nb(cols / BW), G(cg_grid(mat.m)), mixed(mx), o(opts), h(pinned),
        exact(opts.cg_rtol <= kExactResidualRtol) {
    int64_t m = A.m;
    R64 = c.alloc<double>(m * C);
    scale = c.alloc<double>(C);
    inv_scale = c.alloc<double>(C);
    rn2 = c.alloc<double>(C);
    bb = c.alloc<double>(C);
    done = c.alloc<int32_t>(C);
    if (mixed)
      w32 = cg_alloc<float>(c, m, C, h);
    else
      w64 = cg_alloc<double>(c, m, C, h);
  }

  // Switches the inner solves to the learned preconditioner (nullptr: back to Jacobi).
  void use(const LearnedPrecond* p) {
    lp = p;
    if (!p) return;
    if (mixed && !w32.Z) w32.Z = c.alloc<float>(A.m * C);
    if (!mixed && !w64.Z) w64.Z = c.alloc<double>(A.m * C);
  }

  // X0 (nullable, may alias X64): starting block.
  Outcome solve(const double* B, double* X64, int ncols, double rtol, const double* X0 = nullptr) {
    Outcome out;
    int64_t m = A.m;
    column_norms(c, m, C, B, bb);
    if (X0) {
      if (X0 != X64)
        SBHA_CUDA(cudaMemcpyAsync(X64, X0, sizeof(double) * m * C, cudaMemcpyDeviceToDevice, c.stream));
      residual(B, X64);
    } else {
      SBHA_CUDA(cudaMemsetAsync(X64, 0, sizeof(double) * m * C, c.stream));
      SBHA_CUDA(cudaMemcpyAsync(R64, B, sizeof(double) * m * C, cudaMemcpyDeviceToDevice, c.stream));
    }
    bool conv = false;
    for (int ref = 0; ref <= o.refine_max; ++ref) {
      column_norms(c, m, C, R64, rn2);
      int32_t* n_todo = mixed ? w32.st.n_active : w64.st.n_active;
      SBHA_CUDA(cudaMemsetAsync(n_todo, 0, sizeof(int32_t), c.stream));
      k_refine_scale<<<grid_for(C, 256), 256, 0, c.stream>>>(C, ncols, rn2, bb, rtol * rtol, scale, inv_scale, done,
                                                              n_todo);
      c.launched("refine_scale");
      if (mixed)
        k_refine_prepare<float><<<stream_grid(m, nb), 256, 0, c.stream>>>(m, R64, inv_scale, w32.R);
      else
        k_refine_prepare<double><<<stream_grid(m, nb), 256, 0, c.stream>>>(m, R64, inv_scale, w64.R);
      c.launched("refine_prepare");
      SBHA_CUDA(cudaMemcpyAsync(h, n_todo, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
      SBHA_CUDA(cudaStreamSynchronize(c.stream));
      if (*h == 0) {
        conv = true;
        break;
      }
      if (ref == o.refine_max) break;
      bool inner_conv = false;
      int its;
      // rho = max ||r|| / ||b|| over the columns still above rtol; the inner solve reduces each
      // residual by rtol / rho (halved for margin) at most, enough to finish in this step
      std::vector<double> hr(C), hb(C);
      SBHA_CUDA(cudaMemcpyAsync(hr.data(), rn2, sizeof(double) * C, cudaMemcpyDeviceToHost, c.stream));
      SBHA_CUDA(cudaMemcpyAsync(hb.data(), bb, sizeof(double) * C, cudaMemcpyDeviceToHost, c.stream));
      SBHA_CUDA(cudaStreamSynchronize(c.stream));
      double rho = 0.0;
      for (int q = 0; q < ncols; ++q)
        if (hb[q] > 0 && hr[q] > rtol * rtol * hb[q]) rho = std::max(rho, std::sqrt(hr[q] / hb[q]));
      double need = rho > 0 ? std::min(0.5, 0.5 * rtol / rho) : 0.5;
      if (mixed) {
        // FP32 cannot usefully go below inner_rtol in one step
        double inner = std::max(o.inner_rtol, need);
        its = cg_run<float>(c, A, A.val32, A.dinv32, lp ? lp->g32 : nullptr, lp ? lp->gt32 : nullptr, C, ncols,
                            inner, o.cg_max_iter, w32, done, &inner_conv);
      } else {
        // FP64: one step normally suffices; later steps only correct the drift between the
        // recursive and the true residual
        its = cg_run<double>(c, A, A.val, A.dinv, lp ? lp->g64 : nullptr, lp ? lp->gt64 : nullptr, C, ncols, need,
                             o.cg_max_iter, w64, done, &inner_conv);
      }
      out.iterations += its;
      if (lp && !inner_conv) {
        // the learned preconditioner stalled (or its iterate stopped being finite): this step is
        // discarded and repeated from the same residual by CG with Jacobi, which stays from then on
        lp = nullptr;
        fell_back = true;
        continue;
      }
      if (mixed)
        k_refine_accumulate<float><<<stream_grid(m, nb), 256, 0, c.stream>>>(m, w32.X, scale, X64);
      else
        k_refine_accumulate<double><<<stream_grid(m, nb), 256, 0, c.stream>>>(m, w64.X, scale, X64);
      c.launched("refine_accumulate");
      out.refinements = ref + 1;
      residual(B, X64);
    }
    std::vector<double> hr(C), hb(C);
    SBHA_CUDA(cudaMemcpyAsync(hr.data(), rn2, sizeof(double) * C, cudaMemcpyDeviceToHost, c.stream));
    SBHA_CUDA(cudaMemcpyAsync(hb.data(), bb, sizeof(double) * C, cudaMemcpyDeviceToHost, c.stream));
    SBHA_CUDA(cudaStreamSynchronize(c.stream));
    for (int q = 0; q < ncols; ++q)
      if (hb[q] > 0) out.max_rel = std::max(out.max_rel, std::sqrt(hr[q] / hb[q]));
    out.converged = conv;
    return out;
  }

  // R64 = B - A X64 in FP64
  void residual(const double* B, const double* X64) {
    int64_t m = A.m;
    KernelClock rclk(c.timing >= 2);
    rclk.begin(c);
    if (exact) {
      resid_dd(c, m, nb, A.rowptr, A.col, A.val, X64, B, R64);
    } else {
      spmm<double>(c, A, nb, C, A.val, X64, R64, -1.0, nullptr, nullptr, false, "resid_spmm");
    }
    rclk.end(c, 3, -1);
    if (rclk.on) {
      SBHA_CUDA(cudaStreamSynchronize(c.stream));
      rclk.harvest({}, nb, [&](int, int) { return 4.0 * (m + 1) + A.nnz * 12.0 + 2.0 * m * C * 8.0; });
    }
    if (!exact) {
      k_axpy<<<grid_for(m * C, 256), 256, 0, c.stream>>>(m * C, 1.0, B, R64);
      c.launched("axpy");
    }
  }
};

void scatter_columns(Ctx& c, int64_t m, const Rhs& r, int j0, int ncols, int C, double* B) {
  SBHA_CUDA(cudaMemsetAsync(B, 0, sizeof(double) * m * C, c.stream));
  k_scatter_rhs<<<std::max(1, std::min(ncols, 1024)), 64, 0, c.stream>>>(m, j0, ncols, r.ptr, r.row, r.val, B, 1.0);
  c.launched("scatter_rhs");
}

}  // namespace

// Declared in sparsify.cu
void topk_rows_merge(Ctx& c, int64_t m, int C, int j0, int ncols, const double* X, int keep, double* topv,
                     int32_t* topc, int first_chunk);
void assemble_rows_csr(Ctx& c, int64_t n, int32_t l, const int32_t* lmcol, const int32_t* uidx, int keep,
                       const double* topv, const int32_t* topc, int32_t* rowptr, int32_t* col, double* val);
void topk_cols(Ctx& c, int64_t m, int C, int j0, int ncols, const double* X, int p, const int32_t* ord, double* cval,
               int32_t* crow);
int64_t assemble_cols_csr(Ctx& c, int64_t n, int32_t l, const int32_t* lmcol, const int32_t* uvert, int p,
                          const double* cval, const int32_t* crow, int32_t* rowptr, int32_t* col, double* val,
                          int64_t cap);
// Declared in dense.cu
void weighted_gram(Ctx& c, int64_t m, int32_t l, const double* E, const double* Du, const double* Db, double* T);
void weighted_gram_tc(Ctx& c, int64_t m, int32_t l, const double* E, const double* Du, const double* Db, double* T);
void gemm_EY_tc(Ctx& c, int64_t m, int32_t l, const double* E, const double* Y, int64_t ldy, int64_t col0, int64_t N,
                const double* Du, double* F);
void landmark_schur(Ctx& c, int64_t m, int32_t l, const double* Lbb, const int32_t* aptr, const int32_t* arow,
                    const double* aval, const double* E, double* S);
void gemm_EY(Ctx& c, int64_t m, int32_t l, const double* E, const double* Y, int64_t ldy, int64_t col0, int64_t N,
             const double* Du, double* F);
void gemm_EtDX(Ctx& c, int64_t m, int32_t l, const double* E, const double* Du, const double* X, int64_t N,
               double* V);

int64_t operator_nnz(int64_t n, int32_t l, int32_t p_row, int32_t mode) {
  if (mode == SBHA_SPARSIFY_COLS) {
    int64_t m = n - l;
    int64_t p = (m * p_row * 2 + l) / (2LL * l);
    p = std::max<int64_t>(1, std::min<int64_t>(m, p));
    return l + static_cast<int64_t>(l) * p;
  }
  return l + (n - l) * std::min<int64_t>(p_row, l);
}

namespace {

// The dense operator P (n x l row-major, vertex order): e_j on landmark rows, P_u (block layout of
// the unknowns, m x lpad) elsewhere.
__global__ void k_dense_P(int64_t n, int64_t m, int32_t l, const int32_t* __restrict__ lmcol,
                          const int32_t* __restrict__ uidx, const double* __restrict__ Pu, double* __restrict__ out) {
  const int64_t total = n * l;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = q / l;
    const int j = static_cast<int>(q % l);
    if (lmcol[v] >= 0) {
      out[q] = lmcol[v] == j ? 1.0 : 0.0;
    } else {
      out[q] = Pu[((static_cast<int64_t>(j / BW) * m) + uidx[v]) * BW + j % BW];
    }
  }
}

}  // namespace

SolveReport interpolation_operator(Ctx& c, const DevGraph& g, const DevCSR& M, const int32_t* idx, int32_t l,
                                   int32_t p_row, const sbha_opts& o, int32_t* rowptr, int32_t* col, double* val,
                                   double* dense_P) {
  SolveReport rep;
  bool factored = o.solver == SBHA_SOLVER_FACTORED;
  // block-CG product kernel: row gathers unless staging is asked for
  bool staged = o.spmm_variant == SBHA_SPMM_STAGED;
  Sys s = build_system(c, g, M, idx, l, factored, staged);
  s.L.contig = s.M.contig = true;
  s.L.chunk = s.M.chunk = o.spmm_chunk_rows;
  s.L.gather = s.M.gather = o.spmm_variant == SBHA_SPMM_GATHER ? 1 : o.spmm_variant == SBHA_SPMM_PIPELINED ? 2 : 0;
  s.L.depth = s.M.depth = o.spmm_pipeline_depth;
  {
    // the TMA gather product serves the FP32 inner solves: a candidate of the tuner under AUTO
    const int tma = o.spmm_variant == SBHA_SPMM_TMA ? 2 : o.spmm_variant == SBHA_SPMM_AUTO ? 1 : 0;
    Mat& A32 = factored ? s.L : s.M;
    if (tma && o.precision == SBHA_PREC_FP32_REFINE && s.m > 0) {
      A32.gtp = build_tiles(c, s.m, A32.nnz, A32.rowptr, A32.col, kGatherRows);
      A32.tma = tma;
    }
  }
  int64_t m = s.m;
  int keep = std::min<int>(p_row, l);
  bool colmode = o.sparsify_mode == SBHA_SPARSIFY_COLS;
  int64_t pcol = 0;
  if (colmode) {
    pcol = (m * p_row * 2 + l) / (2LL * l);
    pcol = std::max<int64_t>(1, std::min<int64_t>(m, pcol));
  }
  double* topv = nullptr;
  int32_t* topc = nullptr;
  double* cval = nullptr;
  int32_t* crow = nullptr;
  if (m > 0) {
    if (colmode) {
      cval = c.alloc<double>(static_cast<size_t>(l) * pcol);
      crow = c.alloc<int32_t>(static_cast<size_t>(l) * pcol);
    } else {
      topv = c.alloc<double>(static_cast<size_t>(m) * keep);
      topc = c.alloc<int32_t>(static_cast<size_t>(m) * keep);
    }
  }
  int chunk = o.chunk_cols > 0 ? o.chunk_cols : kMaxChunk;
  chunk = std::min(chunk, kMaxChunk);
  chunk = std::max(BW, (chunk + BW - 1) / BW * BW);
  int lp = (l + BW - 1) / BW * BW;
  int C = std::min<int>(chunk, lp);
  C = std::max(C, (keep + BW - 1) / BW * BW);  // the first chunk must offer at least `keep` candidates per row
  int nb = C / BW;
  // learned preconditioner: trained on a pilot of the first `pilot` columns (opts.mlp_pilot_cols,
  // default kPilotCols), which plain Jacobi-preconditioned CG solves first
  const int pilot = o.mlp_pilot_cols > 0 ? o.mlp_pilot_cols : kPilotCols;
  bool learn = factored && o.precond == SBHA_PRECOND_MLP && l > pilot && C >= pilot;
  int64_t lpad = static_cast<int64_t>((l + C - 1) / C) * C;  // every chunk owns C full columns
  int32_t* h_pinned = nullptr;
  SBHA_CUDA(cudaMallocHost(&h_pinned, sizeof(int32_t) * 4));
  struct PinnedGuard {
    int32_t* p;
    ~PinnedGuard() { cudaFreeHost(p); }
  } guard{h_pinned};
  bool mixed = o.precision == SBHA_PREC_FP32_REFINE;
  {
    sbha_stats& st = thread_stats();
    const TiledPattern& tp = factored ? s.L.tp : s.M.tp;
    st.spmm_tiles = tp.ntiles;
    st.spmm_tiles_staged = tp.staged_tiles;
    st.spmm_halo_rows = tp.halo_rows;
    const TiledPattern& gtp = factored ? s.L.gtp : s.M.gtp;
    st.spmm_gather_tiles_staged = gtp.staged_tiles;
    st.spmm_gather_halo_rows = gtp.halo_rows;
    st.unknowns = m;
    st.nnz_uu = factored ? s.L.nnz : s.M.nnz;
    st.chunk_cols = C;
    st.inner_bytes = mixed ? 4 : 8;
  }
  if (m > 0) {
    auto nchunk = [&](int j0) { return std::min(C, l - j0); };
    auto slab = [&](double* base, int j0) { return base + static_cast<int64_t>(j0 / BW) * m * BW; };
    double* B = c.alloc<double>(m * C);
    double* Pu = c.zeros<double>(m * lpad);
    if (!factored) {
      BlockSolver bs(c, s.M, C, mixed, o, h_pinned);
      for (int j0 = 0; j0 < l; j0 += C) {
        int nc = nchunk(j0);
        scatter_columns(c, m, s.Mb, j0, nc, C, B);
        Outcome oc = bs.solve(B, slab(Pu, j0), nc, o.cg_rtol);
        rep.iterations += oc.iterations;
        rep.refinements = std::max(rep.refinements, oc.refinements);
        rep.max_rel_residual = std::max(rep.max_rel_residual, oc.max_rel);
        if (!oc.converged) rep.converged = false;
      }
    } else {
      // Laplacian solves are taken to a fiftieth of the target so that the assembled operator
      // meets cg_rtol on the biharmonic residual without a correction in the common case.
      double rtol_l = std::max(o.cg_rtol * 0.02, 1e-14);
      BlockSolver bs(c, s.L, C, mixed, o, h_pinned);
      double* E = c.zeros<double>(m * lpad);
      int its_e = 0, its_k = 0;
      std::unique_ptr<LearnedPrecond> lp;
      sbha_stats& st = thread_stats();
      for (int j0 = 0; j0 < l; j0 += C) {
        int nc = nchunk(j0);
        scatter_columns(c, m, s.Ab, j0, nc, C, B);
        Outcome oc;
        if (learn && j0 == 0) {
          // pilot: the plain solver's first columns to a loose tolerance, then the network trained
          // on those (right-hand side, solution) pairs
          SBHA_CUDA(cudaStreamSynchronize(c.stream));
          auto t0 = std::chrono::steady_clock::now();
          // a solver as wide as the pilot: its column blocks are the first ones of the chunk's block
          // layout (B and the slab of E), so it reads and writes them in place, and its full-width FP64
          // steps (norms, residuals, copies) cover only the pilot's blocks
          Outcome op;
          {
            BlockSolver bsp(c, s.L, (pilot + BW - 1) / BW * BW, mixed, o, h_pinned);
            op = bsp.solve(B, slab(E, 0), pilot, std::max(rtol_l, kPilotRtol));
          }
          its_e += op.iterations;
          st.e_iterations_jacobi = op.iterations;
          SBHA_CUDA(cudaStreamSynchronize(c.stream));
          auto t1 = std::chrono::steady_clock::now();
          lp.reset(new LearnedPrecond(c, m, s.L.nnz, s.L.rowptr, s.L.col, s.L.val, s.L.val32));
          int epochs = o.mlp_epochs > 0 ? o.mlp_epochs : 60;
          bool ok = lp->train(B, slab(E, 0), pilot, epochs, 3e-3f, &st.mlp_loss_first, &st.mlp_loss_last);
          auto t2 = std::chrono::steady_clock::now();
          st.mlp_ms_pilot = std::chrono::duration<double, std::milli>(t1 - t0).count();
          st.mlp_ms_train = std::chrono::duration<double, std::milli>(t2 - t1).count();
          st.mlp_trained = ok ? 1 : 0;
          st.mlp_train_columns = pilot;
          st.mlp_train_entries = lp->train_entries;
          if (ok && o.fault_inject == SBHA_FAULT_MLP_NAN) lp->poison();  // host-side fault injection (tests)
          if (ok) bs.use(lp.get());
          // every column of the chunk to full tolerance; the pilot columns start from their solutions
          oc = bs.solve(B, slab(E, 0), nc, rtol_l, slab(E, 0));
        } else {
          oc = bs.solve(B, slab(E, j0), nc, rtol_l);
          if (j0 == 0) st.e_iterations_jacobi = oc.iterations;
        }
        its_e += oc.iterations;
        rep.refinements = std::max(rep.refinements, oc.refinements);
        if (!oc.converged) rep.converged = false;
        if (bs.lp) st.e_iterations_learned = std::max(st.e_iterations_learned, oc.iterations);
      }
      double* T = c.alloc<double>(static_cast<size_t>(l) * l);
      double* S = c.alloc<double>(static_cast<size_t>(l) * l);
      double* Y = c.alloc<double>(static_cast<size_t>(l) * l);
      // landmark-space FP64 products: tensor cores by exact slicing, or the FP64 pipes
      const bool tc = o.dense_mode != SBHA_DENSE_FP64;
      if (tc)
        weighted_gram_tc(c, m, l, E, s.Du, s.Db, T);
      else
        weighted_gram(c, m, l, E, s.Du, s.Db, T);
      landmark_schur(c, m, l, s.Lbb, s.Ab.ptr, s.Ab.row, s.Ab.val, E, S);
      double* Lc = cholesky(c, l, T);  // T = D_b + E^T D_u E is SPD
      SBHA_CUDA(cudaMemcpyAsync(Y, S, sizeof(double) * l * l, cudaMemcpyDeviceToDevice, c.stream));
      cholesky_solve(c, l, Lc, Y, l);
      for (int j0 = 0; j0 < l; j0 += C) {
        int nc = nchunk(j0);
        SBHA_CUDA(cudaMemsetAsync(B, 0, sizeof(double) * m * C, c.stream));
        if (tc)
          gemm_EY_tc(c, m, l, E, Y, l, j0, nc, s.Du, B);
        else
          gemm_EY(c, m, l, E, Y, l, j0, nc, s.Du, B);
        Outcome oc = bs.solve(B, slab(Pu, j0), nc, rtol_l);
        its_k += oc.iterations;
        if (!oc.converged) rep.converged = false;
        k_axpy<<<grid_for(m * C, 256), 256, 0, c.stream>>>(m * static_cast<int64_t>(nb) * BW, 1.0, slab(E, j0),
                                                           slab(Pu, j0));
        c.launched("axpy");
      }
      rep.iterations = its_e + its_k;
      st.e_iterations = its_e;
      st.k_iterations = its_k;
      // FP64 check on the biharmonic system, with corrections through the factorisation
      double* R = c.alloc<double>(m * C);
      double* bn = c.alloc<double>(C);
      double* rn = c.alloc<double>(C);
      double* V = c.alloc<double>(static_cast<size_t>(l) * C);
      double* Wt = c.alloc<double>(static_cast<size_t>(l) * C);
      double* Xc = c.alloc<double>(m * C);
      rep.max_rel_residual = 0.0;
      for (int j0 = 0; j0 < l; j0 += C) {
        int nc = nchunk(j0);
        double* Pc = slab(Pu, j0);
        scatter_columns(c, m, s.Mb, j0, nc, C, B);
        column_norms(c, m, C, B, bn);
        double worst = 0.0;
        for (int corr = 0; corr <= o.refine_max; ++corr) {
          // R = b - M_uu P
          if (bs.exact) {
            resid_dd(c, m, nb, s.M.rowptr, s.M.col, s.M.val, Pc, B, R);
          } else {
            spmm<double>(c, s.M, nb, C, s.M.val, Pc, R, -1.0, nullptr, nullptr, false, "resid_spmm");
            k_axpy<<<grid_for(m * C, 256), 256, 0, c.stream>>>(m * C, 1.0, B, R);
            c.launched("axpy");
          }
          column_norms(c, m, C, R, rn);
          std::vector<double> hr(C), hb(C);
          SBHA_CUDA(cudaMemcpyAsync(hr.data(), rn, sizeof(double) * C, cudaMemcpyDeviceToHost, c.stream));
          SBHA_CUDA(cudaMemcpyAsync(hb.data(), bn, sizeof(double) * C, cudaMemcpyDeviceToHost, c.stream));
          SBHA_CUDA(cudaStreamSynchronize(c.stream));
          worst = 0.0;
          for (int q = 0; q < nc; ++q)
            if (hb[q] > 0) worst = std::max(worst, std::sqrt(hr[q] / hb[q]));
          if (worst <= o.cg_rtol || corr == o.refine_max) break;
          // P += M_uu^{-1} R = L_uu^{-1} D_u (a - E T^{-1} E^T D_u a), a = L_uu^{-1} R
          Outcome oa = bs.solve(R, Xc, nc, rtol_l);
          gemm_EtDX(c, m, l, E, s.Du, Xc, C, V);
          SBHA_CUDA(cudaMemcpyAsync(Wt, V, sizeof(double) * l * C, cudaMemcpyDeviceToDevice, c.stream));
          cholesky_solve(c, l, Lc, Wt, C);
          SBHA_CUDA(cudaMemsetAsync(R, 0, sizeof(double) * m * C, c.stream));
          gemm_EY(c, m, l, E, Wt, C, 0, nc, nullptr, R);  // R <- E T^{-1} E^T D_u a
          k_axpy<<<grid_for(m * C, 256), 256, 0, c.stream>>>(m * C, -1.0, R, Xc);
          c.launched("axpy");
          k_scale_rows<<<grid_for(m * C, 256), 256, 0, c.stream>>>(m, nb, s.Du, Xc, R);
          c.launched("scale_rows");
          Outcome ob = bs.solve(R, Xc, nc, rtol_l);
          k_axpy<<<grid_for(m * C, 256), 256, 0, c.stream>>>(m * C, 1.0, Xc, Pc);
          c.launched("axpy");
          rep.iterations += oa.iterations + ob.iterations;
          st.correction_iterations += oa.iterations + ob.iterations;
          st.corrections += 1;
          rep.refinements = std::max(rep.refinements, corr + 1);
        }
        rep.max_rel_residual = std::max(rep.max_rel_residual, worst);
        if (worst > o.cg_rtol) rep.converged = false;
      }
      st.mlp_fallback = bs.fell_back ? 1 : 0;
      for (void* p : {static_cast<void*>(R), static_cast<void*>(bn), static_cast<void*>(rn),
                      static_cast<void*>(V), static_cast<void*>(Wt), static_cast<void*>(Xc), static_cast<void*>(T),
                      static_cast<void*>(S), static_cast<void*>(Y), static_cast<void*>(E), static_cast<void*>(Lc)})
        c.free(p);
    }
    if (dense_P) {
      k_dense_P<<<grid_for(s.n * l, 256), 256, 0, c.stream>>>(s.n, m, l, s.lmcol, s.uidx, Pu, dense_P);
      c.launched("dense_P");
    }
    if (rowptr)
      for (int j0 = 0; j0 < l; j0 += C) {
        int nc = nchunk(j0);
        if (colmode)
          topk_cols(c, m, C, j0, nc, slab(Pu, j0), static_cast<int>(pcol), s.uord, cval, crow);
        else
          topk_rows_merge(c, m, C, j0, nc, slab(Pu, j0), keep, topv, topc, j0 == 0);
      }
  } else if (dense_P) {  // every vertex a landmark: P is a permutation
    k_dense_P<<<grid_for(s.n * l, 256), 256, 0, c.stream>>>(s.n, 0, l, s.lmcol, s.uidx, nullptr, dense_P);
    c.launched("dense_P");
  }
  if (!rowptr) return rep;  // only the dense operator was asked for
  if (colmode)
    assemble_cols_csr(c, s.n, l, s.lmcol, s.uvert, static_cast<int>(pcol), cval, crow, rowptr, col, val,
                      operator_nnz(s.n, l, p_row, SBHA_SPARSIFY_COLS));
  else
    assemble_rows_csr(c, s.n, l, s.lmcol, s.uidx, keep, topv, topc, rowptr, col, val);
  return rep;
}

// ------------------------------------------------ block solves on a caller's matrix ---

namespace {

// FP32 copy of the values and the inverse diagonal (FP64 and FP32) of a CSR matrix that stores
// every diagonal entry.
__global__ void k_mat_prepare(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, float* __restrict__ val32, double* __restrict__ dinv,
                              float* __restrict__ dinv32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      val32[e] = static_cast<float>(val[e]);
      if (col[e] == i) d = val[e];
    }
    dinv[i] = d != 0.0 ? 1.0 / d : 0.0;
    dinv32[i] = static_cast<float>(dinv[i]);
  }
}

Mat caller_mat(Ctx& c, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col, const double* val,
               bool prepare) {
  Mat A;
  A.m = n;
  A.nnz = nnz;
  A.rowptr = const_cast<int32_t*>(rowptr);
  A.col = const_cast<int32_t*>(col);
  A.val = const_cast<double*>(val);
  if (prepare) {
    A.val32 = c.alloc<float>(std::max<int64_t>(nnz, 1));
    A.dinv = c.alloc<double>(n);
    A.dinv32 = c.alloc<float>(n);
    k_mat_prepare<<<grid_for(n, 256), 256, 0, c.stream>>>(n, rowptr, col, val, A.val32, A.dinv, A.dinv32);
    c.launched("mat_prepare");
  }
  return A;
}

}  // namespace

void csr_block_spmm(Ctx& c, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col, const double* val,
                    int C, const double* x, double* y, double alpha) {
  Mat A = caller_mat(c, n, nnz, rowptr, col, val, false);
  spmm<double>(c, A, C / BW, C, val, x, y, alpha, nullptr, nullptr, false, "csr_spmm");
}

void csr_block_spmm_f32(Ctx& c, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                        const float* val, int nb, const float* x, float* y) {
  Mat A = caller_mat(c, n, nnz, rowptr, col, nullptr, false);
  spmm<float>(c, A, nb, nb * BW, val, x, y, 1.f, nullptr, nullptr, false, "csr_spmm_f32");
}

SpdReport spd_block_solve(Ctx& c, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                          const double* val, int C, int ncols, const double* B, double* X, const sbha_opts& o) {
  SpdReport rep;
  if (n <= 0 || ncols <= 0) return rep;
  Mat A = caller_mat(c, n, nnz, rowptr, col, val, true);
  A.chunk = o.spmm_chunk_rows;
  int32_t* h_pinned = nullptr;
  SBHA_CUDA(cudaMallocHost(&h_pinned, sizeof(int32_t) * 4));
  struct PinnedGuard {
    int32_t* p;
    ~PinnedGuard() { cudaFreeHost(p); }
  } guard{h_pinned};
  BlockSolver bs(c, A, C, o.precision == SBHA_PREC_FP32_REFINE, o, h_pinned);
  Outcome out = bs.solve(B, X, ncols, o.cg_rtol);
  rep.iterations = out.iterations;
  rep.max_rel = out.max_rel;
  rep.converged = out.converged;
  return rep;
}

}  // namespace sbha
