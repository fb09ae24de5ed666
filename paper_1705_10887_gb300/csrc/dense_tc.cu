// FP64 matrix products on the tcgen05 tensor cores, by exact integer slicing.
//
// The landmark-space products of the factored solver (T = E^T D_u E, and E Y) are m x l x l
// FP64 contractions: 2 m l^2 flops each, about 1.3 s apiece at l = 2000 on the FP64 pipes.
// Here they run on the BF16 tensor cores instead.  Every row r of the operand A (and of
// B^T) is scaled by a power of two 2^-e_r so that its entries lie in [-1/2, 1/2], then
// written as six signed 8-bit digits,
//     a = 2^e_r sum_{s<6} d_s 256^-(s+1),   |d_s| <= 128,   |remainder| <= (2^-49 + 2^-62) 2^e_r,
// each digit an integer that BF16 holds exactly.  The digits are peeled off a 62-bit fixed-point
// image of a 2^-e_r on the integer pipes (nearest digit, ties to even), not by FP64 arithmetic.  A product of two digits is an integer
// of at most 2^14, so a sum of up to 256 of them (or up to 1024/(d+1) per diagonal) is an
// exact integer in FP32.  The 21 digit pairs with s + t <= 5 are grouped by d = s + t into
// six FP32 accumulators in tensor memory; every 256 K the four leading diagonals (still
// exact) are read out and added, shifted by 8 (3 - d) bits, into int64 registers holding the exact
// sum in units of 2^-40, and the last two (weighted 2^-48 and below) run through K in FP32 and are
// added at the end.  The result
// is the FP64 product to within a few units of 2^-48 of |A| |B| per term.
//
// One CTA computes a 128 x 64 tile of C over one range of K (split-K), with all six digit
// slices of a 128 x 64 (A) and 64 x 64 (B) granule staged in shared memory (144 KB) per
// step, the MMAs issued by one thread, completion signalled through an mbarrier.  Every wait
// is bounded.  Only the issuing thread polls the mbarrier; its verdict reaches the other threads
// through shared memory after a CTA barrier, so all of them leave the loop together.  A wait that
// gives up records SBHA_ETIMEOUT, and the issuing thread then waits once more, on the same phase
// and with the default limit, for the products still in flight before the CTA frees its tensor
// memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace sbha {

namespace {

constexpr int kSlices = 6;
constexpr int kTM = 128, kTN = 64, kKG = 64;  // C tile rows and columns; K granule
constexpr int kGranA = kTM * kKG;             // BF16 elements of one A slice granule (16 KB)
constexpr int kGranB = kTN * kKG;             // (8 KB)
constexpr int kKH = kKG / 2;                                  // K per pipeline stage (half a granule)
constexpr int kStageBytes = kSlices * (kGranA + kGranB) * 2 / 2;  // one stage: 72 KB
constexpr int kStages = 3;
constexpr int kSmemBytes = kStages * kStageBytes;                // 216 KB
constexpr int kExactEvery = 4;  // granules between readouts of the exact diagonals (256 K)
constexpr int kTmemCols = 512;
constexpr int kThreads = 128;
constexpr long long kWaitLimit = 1LL << 22;  // default polls of a bounded wait


// ------------------------------------------------------------------ operands ----

// Operand accessors X(r, k): row r of the operand (an output row of A, or an output column
// for B), K index k.
struct ColsOfBlock {  // column r of a block-layout m x ncols array, optional row scale: X(r, k) = s_k E(k, r)
  const double* p;
  int64_t m;
  const double* scale;
  __device__ __forceinline__ double operator()(int64_t r, int64_t k) const {
    double v = p[((r >> 5) * m + k) * 32 + (r & 31)];
    return scale ? v * scale[k] : v;
  }
};
struct RowsOfBlock {  // row r of a block-layout array: X(r, k) = E(r, k)
  const double* p;
  int64_t m;
  __device__ __forceinline__ double operator()(int64_t r, int64_t k) const {
    return p[((k >> 5) * m + r) * 32 + (k & 31)];
  }
};
struct ColsOfRowMajor {  // column r of a row-major array (leading dimension ld): X(r, k) = Y(k, r)
  const double* p;
  int64_t ld;
  __device__ __forceinline__ double operator()(int64_t r, int64_t k) const { return p[k * ld + r]; }
};
struct SquaresOfRowMajor {  // row r of the elementwise square of a row-major array: X(r, k) = A(r, k)^2
  const double* p;
  int64_t ld;
  __device__ __forceinline__ double operator()(int64_t r, int64_t k) const {
    const double a = p[r * ld + k];
    return a * a;
  }
};
struct RowsOfRowMajor {  // row r of a row-major array: X(r, k) = A(r, k)
  const double* p;
  int64_t ld;
  __device__ __forceinline__ double operator()(int64_t r, int64_t k) const { return p[r * ld + k]; }
};

// e_r = ilogb(max_k |X(r, k)|) + 2 (0 for a zero row): one warp per row.
template <class X>
__global__ void k_row_exp(int64_t R, int64_t K, X x, int32_t* __restrict__ e) {
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w; r < R; r += nw) {
    double mx = 0.0;
    for (int64_t k = lane; k < K; k += 32) mx = fmax(mx, fabs(x(r, k)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) e[r] = mx > 0.0 ? ilogb(mx) + 2 : 0;
  }
}

// trunc(|x| 2^(62 - ex)) with the sign of x, as an integer (|x| < 2^(ex - 1), so |result| < 2^61): read
// from the bits of x, so no FP64 arithmetic.  Bits below 2^-62 of x 2^-ex are dropped, which adds at most
// 2^-62 2^ex to the slicing remainder.
__device__ __forceinline__ int64_t fixed62(double x, int ex) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int expf = static_cast<int>((b >> 52) & 0x7ff);
  unsigned long long mant = b & ((1ULL << 52) - 1);
  int E = -1074;  // subnormal or zero
  if (expf != 0) {
    mant |= 1ULL << 52;
    E = expf - 1075;
  }
  const int sh = E + 62 - ex;
  unsigned long long v = 0;
  if (mant != 0) {
    if (sh >= 0)
      v = sh < 11 ? mant << sh : 0;  // |x 2^-ex| < 1/2 keeps sh below 9 here
    else if (sh > -64)
      v = mant >> (-sh);
  }
  return (b >> 63) ? -static_cast<int64_t>(v) : static_cast<int64_t>(v);
}

// Digit images: slice s, row tile rt (TR rows), K granule kg is one contiguous granule of
// TR x 64 BF16 in the tensor cores' K-major layout without swizzle: 8 x 8 core matrices
// (8 rows of 16 bytes, 128 contiguous bytes), core (ri, ki) at (ri * 8 + ki) * 64 elements.
// Rows beyond R and K beyond K are zero.  One thread per (row, 8 consecutive K).
template <class X>
__global__ void k_digits(int64_t R, int64_t K, int TR, int64_t RT, int64_t KG, X x, const int32_t* __restrict__ e,
                         __nv_bfloat16* __restrict__ out) {
  int64_t total = RT * TR * KG * 8;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = q / (KG * 8), k8 = q % (KG * 8);
    int64_t kg = k8 >> 3;
    int ki = static_cast<int>(k8 & 7);
    int64_t rt = r / TR;
    int rr = static_cast<int>(r % TR);
    // each value as a 62-bit fixed-point integer V = |x| 2^(62 - ex) (truncated, sign restored), |V| < 2^61;
    // the digits peel off by arithmetic shifts with round-half-even, all on the integer pipes
    int64_t V[8];
    unsigned bad = 0;  // non-finite inputs: their digits are NaN, so the product shows them
    int ex = r < R ? e[r] : 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int64_t k = k8 * 8 + i;
      const double xv = (r < R && k < K) ? x(r, k) : 0.0;
      if (!isfinite(xv)) bad |= 1u << i;
      V[i] = fixed62(xv, ex);
    }
    int64_t base = ((rt * KG + kg) * TR + 0) * kKG;  // granule start within the slice (elements)
    int64_t within = static_cast<int64_t>((rr >> 3) * 8 + ki) * 64 + (rr & 7) * 8;
    int64_t sstride = RT * KG * TR * kKG;
#pragma unroll
    for (int s = 0; s < kSlices; ++s) {
      const int sh = 54 - 8 * s;  // digit s weighs 2^-8(s+1) = 2^(sh - 62)
      __align__(16) __nv_bfloat16 d[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        int64_t q = V[i] >> sh;  // floor
        const int64_t rem = V[i] - (q << sh), half = 1LL << (sh - 1);
        if (rem > half || (rem == half && (q & 1))) ++q;  // nearest, ties to even
        V[i] -= q << sh;
        d[i] = ((bad >> i) & 1u) ? __float2bfloat16_rn(__int_as_float(0x7fc00000))
                                 : __float2bfloat16_rn(static_cast<float>(q));  // |q| <= 128: exact in BF16
      }
      *reinterpret_cast<uint4*>(out + s * sstride + base + within) = *reinterpret_cast<const uint4*>(d);
    }
  }
}

// ------------------------------------------------------------------ tcgen05 ----

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, no swizzle; LBO = byte distance of K-adjacent
// core matrices, SBO = of M/N-adjacent ones.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}

// out(i, j, v) for C's rows i < M, columns j < N.
struct PartOut {  // row-major partial of split z
  double* p;
  int64_t M, N;
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double v) const {
    p[(static_cast<int64_t>(blockIdx.z) * M + i) * N + j] = v;
  }
};
struct BlockRowsOut {  // block layout (rows u, columns col0 + j), optional row scale
  double* p;
  int64_t m;
  const double* scale;
  __device__ __forceinline__ void operator()(int64_t u, int64_t j, double v) const {
    p[((j >> 5) * m + u) * 32 + (j & 31)] = scale ? v * scale[u] : v;
  }
};

// C tile (blockIdx.y, blockIdx.x) over the K granules of split blockIdx.z.  lower: C is
// symmetric and only the tiles touching the lower triangle are computed.
//
// Pipeline: K is staged in halves of a 64-wide granule (kKH = 32 K: six A and six B digit slices,
// 72 KB) in kStages buffers.  Iteration h: the copies of half-granule h have landed (every thread
// waits for its own cp.async group, then a CTA barrier); thread 0 issues its 42 MMAs and commits
// them to the stage's mbarrier; it then waits for the previous half-granule's commit (the tensor
// cores run in order, so that stage is free while half-granule h computes), and every thread
// refills that stage with half-granule h + kStages - 1.  Only thread 0 polls mbarriers; its verdict
// reaches the others through shared memory after a barrier.  Every 256 K (and at the end) thread 0
// also waits for h's own commit before the four exact diagonals are read out of tensor memory.
template <class OF>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __nv_bfloat16* __restrict__ Ad, const __nv_bfloat16* __restrict__ Bd, int64_t RTa, int64_t RTb,
              int64_t KG, int64_t kg_per_split, const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
              int64_t M, int64_t N, bool lower, OF out, int* err, long long wait_limit) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[kStages];
  __shared__ uint32_t s_taddr;
  __shared__ int s_ok;
  const int tm = blockIdx.y, tn = blockIdx.x;
  if (lower && static_cast<int64_t>(tm) * kTM + kTM - 1 < static_cast<int64_t>(tn) * kTN) return;
  const int64_t g0 = blockIdx.z * kg_per_split, g1 = min(KG, g0 + kg_per_split);
  const int64_t h0 = 2 * g0, h1 = 2 * g1;  // half-granules of this split
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_taddr)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 0) {
    for (int x = 0; x < kStages; ++x) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[x])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t taddr = s_taddr;
  const uint32_t idesc = idesc_bf16(kTM, kTN);
  const int64_t sstrideA = RTa * KG * kGranA, sstrideB = RTb * KG * kGranB;
  // copies of half-granule h into stage x: per slice, row group ri (8 rows) of the tile holds 4
  // K-adjacent core matrices (512 contiguous bytes) of the global granule h / 2, half h % 2
  auto load = [&](int64_t h, int x) {
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(smem + static_cast<size_t>(x) * kStageBytes);
    __nv_bfloat16* sB = sA + kSlices * (kGranA / 2);
    const int64_t g = h >> 1;
    const int half = static_cast<int>(h & 1);
    // 16-byte chunks per slice: (rows / 8) row groups x 32; the A and B loops have compile-time
    // geometry (no divisions by a runtime value per chunk), and the slice bases are hoisted
    constexpr int kPerA = (kTM / 8) * 32, kPerB = (kTN / 8) * 32;
    static_assert(kPerA % kThreads == 0 && kPerB % kThreads == 0, "whole rounds per slice");
    const __nv_bfloat16* gA = Ad + (tm * KG + g) * kGranA + half * 4 * 64;
    const __nv_bfloat16* gB = Bd + (tn * KG + g) * kGranB + half * 4 * 64;
#pragma unroll 1
    for (int sl = 0; sl < kSlices; ++sl) {
#pragma unroll
      for (int r = 0; r < kPerA / kThreads; ++r) {
        const int q = r * kThreads + threadIdx.x;
        const int ri = q >> 5, c16 = q & 31;
        cp_async16(sA + sl * (kGranA / 2) + ri * 4 * 64 + c16 * 8, gA + sl * sstrideA + ri * 8 * 64 + c16 * 8);
      }
#pragma unroll
      for (int r = 0; r < kPerB / kThreads; ++r) {
        const int q = r * kThreads + threadIdx.x;
        const int ri = q >> 5, c16 = q & 31;
        cp_async16(sB + sl * (kGranB / 2) + ri * 4 * 64 + c16 * 8, gB + sl * sstrideB + ri * 8 * 64 + c16 * 8);
      }
    }
  };
  // The four exact diagonals as one integer in units of 2^-40 (diagonal d weighs 2^(-8 (d + 2)), so
  // d = 0..3 shift by 24, 16, 8, 0 bits): each readout adds values below 2^24 in magnitude, so the
  // sum stays exact in int64 for K up to about 2^22.  Integer adds run on the integer pipes; the FP64
  // pipes (a few per SM on GB300) take only the final combination.
  long long acc[kTN];
#pragma unroll
  for (int j = 0; j < kTN; ++j) acc[j] = 0;
  bool fresh[kSlices];
#pragma unroll
  for (int d = 0; d < kSlices; ++d) fresh[d] = true;
  uint32_t phase[kStages];
  bool pending[kStages];  // a commit on that stage not yet waited for (meaningful in thread 0)
#pragma unroll
  for (int x = 0; x < kStages; ++x) {
    phase[x] = 0;
    pending[x] = false;
  }
  // prologue: the first kStages - 1 half-granules in flight, one cp.async group each
  for (int x = 0; x < kStages - 1; ++x) {
    if (h0 + x < h1) load(h0 + x, x);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  bool ok = true;
  for (int64_t h = h0; h < h1 && ok; ++h) {
    const int st = static_cast<int>((h - h0) % kStages);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kStages - 2) : "memory");  // h's copies (this thread's)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const bool last = h + 1 == h1;
    const bool readout = ((h - h0 + 1) % (2 * kExactEvery) == 0) || last;
    if (threadIdx.x == 0) {
      const uint32_t a0 = smem_u32(smem + static_cast<size_t>(st) * kStageBytes);
      const uint32_t b0 = a0 + kSlices * (kGranA / 2) * 2;
#pragma unroll
      for (int d = 0; d < kSlices; ++d) {
        for (int sa = 0; sa <= d; ++sa) {
          const int sb = d - sa;
          for (int kk = 0; kk < kKH / 16; ++kk) {
            uint64_t a = smem_desc(a0 + sa * (kGranA / 2) * 2 + kk * 256, 128, 512);
            uint64_t b = smem_desc(b0 + sb * (kGranB / 2) * 2 + kk * 256, 128, 512);
            uint32_t accum = (fresh[d] && sa == 0 && kk == 0) ? 0u : 1u;
            mma_bf16(taddr + d * kTN, a, b, idesc, accum);
          }
        }
        fresh[d] = false;
      }
      mma_commit(smem_u32(&mbar[st]));
      pending[st] = true;
      bool good = true;
      const int prev = (st + kStages - 1) % kStages;
      if (pending[prev]) {  // the previous half-granule's products: their stage is refilled below
        good = mbar_wait(smem_u32(&mbar[prev]), phase[prev], wait_limit);
        if (good) {
          phase[prev] ^= 1u;
          pending[prev] = false;
        }
      }
      if (good && readout) {  // this half-granule's products, before tensor memory is read
        good = mbar_wait(smem_u32(&mbar[st]), phase[st], wait_limit);
        if (good) {
          phase[st] ^= 1u;
          pending[st] = false;
        }
      }
      s_ok = good ? 1 : 0;
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    ok = s_ok != 0;
    if (!ok) break;
    if (readout) {  // the exact diagonals (d <= 3) into the integer sums
#pragma unroll 1
      for (int d = 0; d < 4; ++d) {
        const int sh = 8 * (3 - d);
#pragma unroll
        for (int cb = 0; cb < kTN / 16; ++cb) {
          float v[16];
          tmem_ld16(taddr + (static_cast<uint32_t>(warp * 32) << 16) + d * kTN + cb * 16, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[cb * 16 + i] += static_cast<long long>(__float2int_rn(v[i])) << sh;
        }
        fresh[d] = true;
      }
    }
    // refill the stage of half-granule h - 1 (its products are done) with half-granule h + kStages - 1
    const int64_t hn = h + kStages - 1;
    if (hn < h1) load(hn, static_cast<int>((hn - h0) % kStages));
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");  // no copy may land after the CTA has gone
  if (!ok) {
    // Products still in flight may be reading shared memory and writing tensor memory: wait for every
    // outstanding commit (same phases, default limit) before the memory is released.
    if (threadIdx.x == 0) {
      atomicCAS(err, DERR_NONE, DERR_TIMEOUT);
      for (int x = 0; x < kStages; ++x)
        if (pending[x]) mbar_wait(smem_u32(&mbar[x]), phase[x], kWaitLimit);
    }
  } else {
    // value = 2^(e_i + e_j) (acc 2^-40 + d4 2^-48 + d5 2^-56); the last two diagonals ran through all
    // of K in FP32 (their weight keeps the rounding below 2^-48 of the terms) and are read only here
    const int64_t i = static_cast<int64_t>(tm) * kTM + warp * 32 + lane;
    const int e_i = i < M ? ea[i] : 0;
    const bool ran = h1 > h0;  // an empty K range wrote nothing to tensor memory: its partial is zero
#pragma unroll
    for (int cb = 0; cb < kTN / 16; ++cb) {
      float v4[16], v5[16];
      if (ran) {
        tmem_ld16(taddr + (static_cast<uint32_t>(warp * 32) << 16) + 4 * kTN + cb * 16, v4);
        tmem_ld16(taddr + (static_cast<uint32_t>(warp * 32) << 16) + 5 * kTN + cb * 16, v5);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v4[q] = v5[q] = 0.f;
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = cb * 16 + q;
        const int64_t gj = static_cast<int64_t>(tn) * kTN + j;
        if (i < M && gj < N) {
          const double low = ldexp(static_cast<double>(v4[q]), -48) + ldexp(static_cast<double>(v5[q]), -56);
          out(i, gj, ldexp(ldexp(static_cast<double>(acc[j]), -40) + low, e_i + eb[gj]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(kTmemCols));
}

// T = diag(db) + sum of the split partials; sym: upper elements of uncomputed tiles are read transposed.
__global__ void k_sum_parts(int64_t M, int64_t N, int Z, const double* __restrict__ part,
                            const double* __restrict__ diag, double* __restrict__ out, bool sym, double alpha = 1.0) {
  int64_t total = M * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = q / N, j = q % N;
    bool computed = (i / kTM) * kTM + kTM - 1 >= (j / kTN) * kTN;
    int64_t src = (sym && !computed) ? j * N + i : q;
    double s = 0.0;
    for (int z = 0; z < Z; ++z) s += part[z * total + src];
    if (diag && i == j) s += diag[i];
    out[q] = alpha * s;
  }
}

struct Digits {
  __nv_bfloat16* d = nullptr;
  int32_t* e = nullptr;
  int64_t RT = 0, KG = 0;
};

Digits alloc_digits(Ctx& c, int64_t R, int64_t K, int TR) {
  Digits o;
  o.RT = (R + TR - 1) / TR;
  o.KG = (K + kKG - 1) / kKG;
  o.e = c.alloc<int32_t>(std::max<int64_t>(R, 1));
  o.d = c.alloc<__nv_bfloat16>(static_cast<size_t>(kSlices) * o.RT * o.KG * TR * kKG);
  return o;
}

template <class X>
void fill_digits(Ctx& c, int64_t R, int64_t K, int TR, X x, const Digits& o) {
  k_row_exp<X><<<grid_for(R * 32, 256), 256, 0, c.stream>>>(R, K, x, o.e);
  c.launched("tc_row_exp");
  k_digits<X><<<grid_for(o.RT * TR * o.KG * 8, 256), 256, 0, c.stream>>>(R, K, TR, o.RT, o.KG, x, o.e, o.d);
  c.launched("tc_digits");
}

template <class X>
Digits make_digits(Ctx& c, int64_t R, int64_t K, int TR, X x) {
  Digits o = alloc_digits(c, R, K, TR);
  fill_digits(c, R, K, TR, x, o);
  return o;
}

template <class OF>
void run_gemm(Ctx& c, const Digits& A, const Digits& B, int64_t M, int64_t N, int splits, bool lower, OF out) {
  static bool attr = false;
  if (!attr) {
    SBHA_CUDA(cudaFuncSetAttribute(k_gemm_tc<OF>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    attr = true;
  }
  int64_t kps = (A.KG + splits - 1) / splits;
  dim3 grid(static_cast<unsigned>(B.RT), static_cast<unsigned>(A.RT), static_cast<unsigned>(splits));
  k_gemm_tc<OF><<<grid, kThreads, kSmemBytes, c.stream>>>(A.d, B.d, A.RT, B.RT, A.KG, kps, A.e, B.e, M, N, lower,
                                                           out, c.d_err, wait_limit());
  c.launched("gemm_tc");
}

int choose_splits(int64_t tiles, int64_t KG) {
  int64_t s = std::max<int64_t>(1, (2 * num_sms() + tiles - 1) / std::max<int64_t>(tiles, 1));
  s = std::min<int64_t>(s, std::max<int64_t>(1, KG / kExactEvery));
  const int64_t kps = (KG + s - 1) / s;  // granules per split: no split is left without K
  return static_cast<int>((KG + kps - 1) / kps);
}

}  // namespace

// Process-wide limit of the bounded waits (sbha_set_wait_limit).
std::atomic<long long> g_wait_limit{kWaitLimit};
long long wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

void weighted_gram_tc(Ctx& c, int64_t m, int32_t l, const double* E, const double* Du, const double* Db, double* T) {
  Digits A = make_digits(c, l, m, kTM, ColsOfBlock{E, m, nullptr});
  Digits B = make_digits(c, l, m, kTN, ColsOfBlock{E, m, Du});
  int64_t tiles = A.RT * B.RT;
  int Z = choose_splits(tiles / 2 + 1, A.KG);
  double* part = c.alloc<double>(static_cast<size_t>(Z) * l * l);
  run_gemm(c, A, B, l, l, Z, true, PartOut{part, l, l});
  k_sum_parts<<<grid_for(static_cast<int64_t>(l) * l, 256), 256, 0, c.stream>>>(l, l, Z, part, Db, T, true);
  c.launched("sum_parts");
  c.check_device("tensor-core gram");
  for (void* p : {static_cast<void*>(A.d), static_cast<void*>(A.e), static_cast<void*>(B.d), static_cast<void*>(B.e),
                  static_cast<void*>(part)})
    c.free(p);
}

void gemm_EY_tc(Ctx& c, int64_t m, int32_t l, const double* E, const double* Y, int64_t ldy, int64_t col0, int64_t N,
                const double* Du, double* F) {
  Digits A = make_digits(c, m, l, kTM, RowsOfBlock{E, m});
  Digits B = make_digits(c, N, l, kTN, ColsOfRowMajor{Y + col0, ldy});
  run_gemm(c, A, B, m, N, 1, false, BlockRowsOut{F, m, Du});
  c.check_device("tensor-core product");
  for (void* p : {static_cast<void*>(A.d), static_cast<void*>(A.e), static_cast<void*>(B.d), static_cast<void*>(B.e)})
    c.free(p);
}

void dgemm_tc_rowmajor(Ctx& c, int64_t M, int64_t N, int64_t K, const double* A, const double* B, double* C) {
  Digits Ad = make_digits(c, M, K, kTM, RowsOfRowMajor{A, K});
  Digits Bd = make_digits(c, N, K, kTN, ColsOfRowMajor{B, N});
  int Z = choose_splits(Ad.RT * Bd.RT, Ad.KG);
  double* part = c.alloc<double>(static_cast<size_t>(Z) * M * N);
  run_gemm(c, Ad, Bd, M, N, Z, false, PartOut{part, M, N});
  k_sum_parts<<<grid_for(M * N, 256), 256, 0, c.stream>>>(M, N, Z, part, nullptr, C, false);
  c.launched("sum_parts");
  c.check_device("tensor-core product");
  for (void* p : {static_cast<void*>(Ad.d), static_cast<void*>(Ad.e), static_cast<void*>(Bd.d),
                  static_cast<void*>(Bd.e), static_cast<void*>(part)})
    c.free(p);
}

}  // namespace sbha

namespace sbha {

// C = alpha op(A) B for a constant square operand op(A) (A or A.A elementwise, M x M row-major) and
// a changing block B (M x N row-major, N <= 64): op(A)'s digits are cut once by the constructor,
// B's on every call into workspace kept for the object's life.
struct TcConstProduct::Impl {
  Digits A, B;
  int64_t M = 0, N = 0;
  int Z = 1;
  double* part = nullptr;
};

TcConstProduct::TcConstProduct(Ctx& ctx, int64_t M, const double* A, bool square, int64_t N) : c(ctx), p(new Impl) {
  p->M = M;
  p->N = N;
  if (square)
    p->A = make_digits(c, M, M, kTM, SquaresOfRowMajor{A, M});
  else
    p->A = make_digits(c, M, M, kTM, RowsOfRowMajor{A, M});
  p->B = alloc_digits(c, N, M, kTN);
  p->Z = choose_splits(p->A.RT * p->B.RT, p->A.KG);
  p->part = c.alloc<double>(static_cast<size_t>(p->Z) * M * N);
}

TcConstProduct::~TcConstProduct() {
  for (void* q : {static_cast<void*>(p->A.d), static_cast<void*>(p->A.e), static_cast<void*>(p->B.d),
                  static_cast<void*>(p->B.e), static_cast<void*>(p->part)})
    c.free(q);
  delete p;
}

void TcConstProduct::times(const double* B, double alpha, double* C) {
  fill_digits(c, p->N, p->M, kTN, ColsOfRowMajor{B, p->N}, p->B);
  run_gemm(c, p->A, p->B, p->M, p->N, p->Z, false, PartOut{p->part, p->M, p->N});
  k_sum_parts<<<grid_for(p->M * p->N, 256), 256, 0, c.stream>>>(p->M, p->N, p->Z, p->part, nullptr, C, false, alpha);
  c.launched("sum_parts");
}

}  // namespace sbha

extern "C" int64_t sbha_set_wait_limit(int64_t spins) {
  long long v = spins < 0 ? sbha::kWaitLimit : static_cast<long long>(spins);
  return sbha::g_wait_limit.exchange(v);
}
