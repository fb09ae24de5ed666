// Sparse x block-of-vectors product with TMA four-row gathers (FP32), for the block-CG solves
// of the interpolation operator (Sec. 2.1 Eq. 3, Sec. 3 Eq. 6).
//
// The operand x is m x C, stored as C/32 column blocks of m rows x 32 values (128 bytes per
// block row).  Viewed as a 2-D tensor of (C/32) m rows x 32 values, any four block rows can be
// fetched into shared memory by one tensor-memory-accelerator gather (tile::gather4), which
// takes four arbitrary row coordinates.  The unknowns are numbered along a Morton curve, so a
// tile of kGatherRows consecutive rows references a compact set of rows (its halo: the tile's
// rows and their neighbours, about 2x the tile on a triangle mesh).
//
// Work items are (tile, column group) pairs, a group being four column blocks (512 bytes of a
// row), enumerated tile-major: CTA b takes items b, b + G, b + 2G, ..., so that at any moment
// the grid covers one contiguous stretch of the ordering and a halo row two tiles share is read
// from DRAM once and then from L2.  One CTA per SM, 16 warps:
//   - warps 12..15 (producers) load the item's extent and halo row quadruples before they wait for
//     the stage, then warp 12 copies the tile's row pointers, entry indices and values into the
//     stage's metadata (asynchronous 4-byte copies) and producer warp p issues the gathers of the
//     group's block p (each lane a share), all on the stage's "full" mbarrier, which completes when
//     every producer lane's copies and every gathered byte have landed.  A TMA operation costs its
//     issuing warp tens of cycles, so one producer warp could not keep the stage filled (measured:
//     about 12 GB/s per SM with one, the full DRAM rate needs about 45);
//   - warps 0..11 (consumers) wait for "full", compute the tile's rows from shared memory (lane
//     l: block l / 8 of the group, values 4 (l mod 8) .. 4 (l mod 8) + 3), write y and release
//     the stage through its "empty" mbarrier (one arrival per warp).
// Two stages of 96 KB alternate.  Every row is summed in the order of its CSR entries, as in the
// register-gather products of the solver, so y is bit-identical to theirs; the column dot
// products (acc) are added per CTA in shared memory and then once per column to the FP64
// accumulators, so their last bits vary between runs, as they do for the other products.
// Tiles whose halo exceeds kGatherCap rows, or whose entries exceed kEntCap, are computed from
// global memory by the consumers (the producer only marks the stage full).
//
// Every mbarrier wait is bounded (wait_limit polls).  A wait that gives up records
// DERR_TIMEOUT and raises the CTA's abort flag; every role stops at its next item.  The producer
// warps take the decision to fill a stage together (a named-barrier AND over their 128 threads,
// reached by all of them on every item), so a stage they fill always receives all of its
// arrivals, and producer warp 12 then waits, again bounded, for the last fill of every stage
// before the CTA exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.cuh"
#include "spmm.cuh"

namespace sbha {

namespace {

constexpr int R = kGatherRows;   // rows per tile
constexpr int CAP = kGatherCap;  // halo rows per tile
constexpr int kGroup = 4;        // column blocks per item
constexpr int kStages = 2;
constexpr int kConsumers = 12;  // computing warps
constexpr int kProducers = 4;   // filling warps, one per block of the group
constexpr int kThreads = 32 * (kConsumers + kProducers);
static_assert(kProducers == kGroup, "producer warp p gathers block p of the group");
constexpr int kEntCap = 1024;  // staged entries per tile
constexpr int kBlkBytes = 128;  // one row of one 32-column FP32 block
constexpr int kMaxBlocks = 16;  // column blocks per call (512 columns)
constexpr int kStageX = kGroup * CAP * kBlkBytes;  // 96 KB of gathered rows per stage
constexpr long long kDrainLimit = 1LL << 22;       // polls of the final wait for the CTA's own gathers

struct StageMeta {
  int2 ent[kEntCap];     // per entry: its halo index and its value's bits
  int ptr[R + 1];        // the tile's row pointers (offsets into the CSR arrays)
  uint16_t self[R];      // halo index of each row itself
  int nr;                // rows of the tile
  int e0;                // the tile's first entry
  int staged;            // 1: halo and entries staged; 0: the consumers read global memory
};

constexpr size_t kOffMeta = static_cast<size_t>(kStages) * kStageX;
constexpr size_t kOffDot = kOffMeta + kStages * sizeof(StageMeta);
constexpr size_t kOffBar = kOffDot + kMaxBlocks * 32 * sizeof(float);
constexpr size_t kOffFlag = kOffBar + 2 * kStages * sizeof(uint64_t);
constexpr size_t kSmemBytes = kOffFlag + 16;
static_assert(kOffBar % 8 == 0, "mbarriers are 8-byte aligned");
static_assert(kSmemBytes <= 227 * 1024, "one CTA per SM");

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

// Waits for the completion of the phase with the given parity; false after `limit` polls or when
// another role raised the abort flag.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, long long limit, const volatile int* abort) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*abort) return false;
  }
  return false;
}

// Asynchronous 4-byte copy global -> shared (completion tracked through cp_async_arrive).
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// An arrival on the mbarrier once every cp.async this thread has issued so far has completed; it
// counts as one of the arrivals the mbarrier expects.
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(bar) : "memory");
}

// AND of `ok` over the producer warps' threads (named barrier 1; every producer thread reaches it).
__device__ __forceinline__ bool producers_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"(ok ? 1u : 0u), "n"(32 * kProducers)
      : "memory");
  return r != 0;
}

// Four block rows (tensor rows y0..y3, all 32 values) into 512 contiguous bytes of shared memory.
__device__ __forceinline__ void gather4(uint32_t dst, const CUtensorMap* map, int y0, int y1, int y2, int y3,
                                        uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(bar)
      : "memory");
}

// The item's tile, column group and active-block mask (bit q: block 4 g + q); 0 = nothing to do.
struct Item {
  int t, b0, nblk;
  unsigned act;
};

__device__ __forceinline__ Item decode(int64_t i, int ngr, int nb, const int32_t* __restrict__ blk_act) {
  Item it;
  it.t = static_cast<int>(i / ngr);
  it.b0 = static_cast<int>(i % ngr) * kGroup;
  it.nblk = min(kGroup, nb - it.b0);
  it.act = 0;
  for (int q = 0; q < it.nblk; ++q)
    if (!blk_act || blk_act[it.b0 + q] != 0) it.act |= 1u << q;
  return it;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_spmm_tma(const __grid_constant__ CUtensorMap xmap, int64_t m, int nb, int ntiles,
               const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ lcol,
               const uint16_t* __restrict__ lself, const int32_t* __restrict__ halo, const int32_t* __restrict__ nh,
               const float* __restrict__ val, const float* __restrict__ x, float* __restrict__ y, float alpha,
               double* __restrict__ acc, const int32_t* __restrict__ blk_act, bool self_dot, int* err,
               long long limit) {
  extern __shared__ __align__(1024) unsigned char smem[];
  StageMeta* meta = reinterpret_cast<StageMeta*>(smem + kOffMeta);
  float* s_dot = reinterpret_cast<float*>(smem + kOffDot);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);  // full[kStages], then empty[kStages]
  volatile int* abort = reinterpret_cast<volatile int*>(smem + kOffFlag);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kMaxBlocks * 32; i += kThreads) s_dot[i] = 0.f;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(smem_addr(&bars[s]), 33 * kProducers);  // per producer warp: 32 copy arrivals, lane 0's expect_tx
      bar_init(smem_addr(&bars[kStages + s]), kConsumers);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto fail = [&]() {
    atomicCAS(err, DERR_NONE, DERR_TIMEOUT);
    *abort = 1;
  };
  const int ngr = (nb + kGroup - 1) / kGroup;
  const int64_t items = static_cast<int64_t>(ntiles) * ngr;

  if (warp >= kConsumers) {
    // ---------------------------------------------------------------- producers ----
    const int pw = warp - kConsumers;  // gathers block pw of each group
    int k = 0;
    int last[kStages];
    for (int s = 0; s < kStages; ++s) last[s] = -1;
    for (int64_t i = blockIdx.x; i < items; i += gridDim.x) {
      const Item it = decode(i, ngr, nb, blk_act);
      if (!it.act) continue;  // the same for every warp
      const int s = k % kStages, use = k / kStages;
      const uint32_t full = smem_addr(&bars[s]), empty = smem_addr(&bars[kStages + s]);
      // one round of independent loads, whose latency overlaps the wait for the stage: the tile's
      // extent and this lane's halo row quadruples (j = lane, lane + 32; the list holds CAP rows)
      const int64_t r0 = static_cast<int64_t>(it.t) * R;
      const int nr = static_cast<int>(min(m, r0 + R) - r0);
      const int4* h4 = reinterpret_cast<const int4*>(halo + static_cast<int64_t>(it.t) * CAP);
      const int4 hq0 = h4[lane];
      const int4 hq1 = lane + 32 < CAP / 4 ? h4[lane + 32] : make_int4(0, 0, 0, 0);
      const int e0 = rowptr[r0], e1 = rowptr[r0 + nr];
      const int cnt = nh[it.t];
      bool ok = *abort == 0;
      if (ok && use > 0) ok = bar_wait(empty, (use - 1) & 1, limit, abort);
      if (!producers_all(ok)) {  // all producer warps stop here, before filling anything
        if (!ok) fail();
        break;
      }
      StageMeta& md = meta[s];
      const int ne = e1 - e0;
      const bool staged = cnt <= CAP && ne <= kEntCap;
      const int nh4 = staged ? (cnt + 3) >> 2 : 0;
      if (staged && pw == 0) {  // the metadata by asynchronous 4-byte copies, tracked by the mbarrier
        for (int r = lane; r <= nr; r += 32) cp_async4(&md.ptr[r], rowptr + r0 + r);
        if (lane < R / 2) cp_async4(&md.self[2 * lane], lself + r0 + 2 * lane);  // lself padded to whole tiles
        for (int q = lane; q < ne; q += 32) {
          cp_async4(&md.ent[q].x, lcol + e0 + q);
          cp_async4(&md.ent[q].y, val + e0 + q);
        }
      }
      const bool mine = staged && ((it.act >> pw) & 1u);
      if (lane == 0) {
        if (pw == 0) {
          md.nr = nr;
          md.e0 = e0;
          md.staged = staged ? 1 : 0;
        }
        // lane 0's arrival posts this warp's expected bytes before any of its gathers is issued (with
        // release semantics: it also publishes nr, e0 and staged)
        const uint32_t tx = mine ? static_cast<uint32_t>(nh4 * 4 * kBlkBytes) : 0u;
        if (tx)
          bar_arrive_tx(full, tx);
        else
          bar_arrive(full);
      }
      __syncwarp();
      if (mine) {
        const uint32_t xs = smem_addr(smem + static_cast<size_t>(s) * kStageX) + pw * CAP * kBlkBytes;
        const int base = (it.b0 + pw) * static_cast<int>(m);  // below 2^31 (checked by the host)
        if (lane < nh4)
          gather4(xs + static_cast<uint32_t>(4 * lane * kBlkBytes), &xmap, base + hq0.x, base + hq0.y, base + hq0.z,
                  base + hq0.w, full);
        if (lane + 32 < nh4)
          gather4(xs + static_cast<uint32_t>(4 * (lane + 32) * kBlkBytes), &xmap, base + hq1.x, base + hq1.y,
                  base + hq1.z, base + hq1.w, full);
      }
      cp_async_arrive(full);  // every lane: arrives once its copies have landed
      last[s] = use;
      ++k;
    }
    // every gather issued has landed before the CTA's shared memory is released (a fixed bound,
    // whatever the process-wide limit: copies in flight always complete); the producer warps stop
    // at the same item, so warp 0's record covers all of them
    if (pw == 0 && lane == 0)
      for (int s = 0; s < kStages; ++s)
        if (last[s] >= 0) {
          const volatile int never = 0;
          if (!bar_wait(smem_addr(&bars[s]), last[s] & 1, kDrainLimit, &never))
            atomicCAS(err, DERR_NONE, DERR_TIMEOUT);
        }
  } else {
    // ---------------------------------------------------------------- consumers ----
    const int bb = lane >> 3, c0 = (lane & 7) * 4;
    int k = 0;
    for (int64_t i = blockIdx.x; i < items; i += gridDim.x) {
      if (__any_sync(0xffffffffu, *abort != 0)) break;
      const Item it = decode(i, ngr, nb, blk_act);
      if (!it.act) continue;
      const int s = k % kStages, use = k / kStages;
      const uint32_t full = smem_addr(&bars[s]), empty = smem_addr(&bars[kStages + s]);
      if (!__all_sync(0xffffffffu, bar_wait(full, use & 1, limit, abort))) {
        if (lane == 0) fail();
        break;
      }
      const StageMeta& md = meta[s];
      const bool on = (it.act >> bb) & 1u;
      const int blk = it.b0 + bb;
      const int64_t r0 = static_cast<int64_t>(it.t) * R;
      const int nr = md.nr;
      const bool staged = md.staged != 0;
      float dot[4] = {0.f, 0.f, 0.f, 0.f};
      if (on) {
        const float* xs = reinterpret_cast<const float*>(smem + static_cast<size_t>(s) * kStageX) +
                          bb * CAP * 32 + c0;
        const float* xg = x + static_cast<int64_t>(blk) * m * 32 + c0;
        for (int r = warp; r < nr; r += kConsumers) {
          const int64_t u = r0 + r;
          float a[4] = {0.f, 0.f, 0.f, 0.f};
          if (staged) {
            const int q1 = md.ptr[r + 1] - md.e0;
            for (int base = md.ptr[r] - md.e0; base < q1; base += 8) {
              int kk[8];
              float vv[8];
              float4 xv[8];
#pragma unroll
              for (int d = 0; d < 8; ++d) {
                const bool ok = base + d < q1;
                const int2 e = ok ? md.ent[base + d] : make_int2(0, 0);
                kk[d] = e.x;
                vv[d] = __int_as_float(e.y);
              }
#pragma unroll
              for (int d = 0; d < 8; ++d)
                xv[d] = base + d < q1 ? *reinterpret_cast<const float4*>(xs + kk[d] * 32)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int d = 0; d < 8; ++d) {
                a[0] += vv[d] * xv[d].x;
                a[1] += vv[d] * xv[d].y;
                a[2] += vv[d] * xv[d].z;
                a[3] += vv[d] * xv[d].w;
              }
            }
          } else {
            const int q1 = rowptr[u + 1];
            for (int base = rowptr[u]; base < q1; base += 8) {
              int kk[8];
              float vv[8];
              float4 xv[8];
#pragma unroll
              for (int d = 0; d < 8; ++d) {
                const bool ok = base + d < q1;
                kk[d] = ok ? col[base + d] : 0;
                vv[d] = ok ? val[base + d] : 0.f;
              }
#pragma unroll
              for (int d = 0; d < 8; ++d)
                xv[d] = base + d < q1 ? __ldg(reinterpret_cast<const float4*>(xg + static_cast<int64_t>(kk[d]) * 32))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int d = 0; d < 8; ++d) {
                a[0] += vv[d] * xv[d].x;
                a[1] += vv[d] * xv[d].y;
                a[2] += vv[d] * xv[d].z;
                a[3] += vv[d] * xv[d].w;
              }
            }
          }
          const float4 out = make_float4(alpha * a[0], alpha * a[1], alpha * a[2], alpha * a[3]);
          const int64_t o = (static_cast<int64_t>(blk) * m + u) * 32 + c0;
          *reinterpret_cast<float4*>(y + o) = out;
          if (acc) {
            float4 xu = out;
            if (!self_dot)
              xu = staged ? *reinterpret_cast<const float4*>(xs + md.self[r] * 32)
                          : __ldg(reinterpret_cast<const float4*>(x + o));
            dot[0] += xu.x * out.x;
            dot[1] += xu.y * out.y;
            dot[2] += xu.z * out.z;
            dot[3] += xu.w * out.w;
          }
        }
      }
      __syncwarp();
      if (lane == 0) bar_arrive(empty);
      if (acc && on)
#pragma unroll
        for (int q = 0; q < 4; ++q) atomicAdd(&s_dot[blk * 32 + c0 + q], dot[q]);
      ++k;
    }
  }
  __syncthreads();
  if (acc)
    for (int cc = threadIdx.x; cc < nb * 32; cc += kThreads)
      if (!blk_act || blk_act[cc / 32] != 0) atomicAdd(acc + cc, static_cast<double>(s_dot[cc]));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

}  // namespace

bool spmm_tma(Ctx& c, const TiledPattern& tp, int nb, const float* val, const float* x, float* y, float alpha,
              double* acc, const int32_t* blk_act, bool self_dot) {
  if (tp.rows != kGatherRows || tp.cap != kGatherCap || tp.ntiles <= 0) return false;
  if (nb <= 0 || nb > kMaxBlocks) return false;
  if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0 || (reinterpret_cast<uintptr_t>(y) & 15u) != 0) return false;
  if (static_cast<int64_t>(nb) * tp.m > static_cast<int64_t>(INT32_MAX)) return false;
  PFN_cuTensorMapEncodeTiled_v12000 encode = encode_fn();
  if (!encode) return false;
  CUtensorMap map;
  const cuuint64_t dims[2] = {32, static_cast<cuuint64_t>(nb) * static_cast<cuuint64_t>(tp.m)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(kBlkBytes)};
  const cuuint32_t box[2] = {32, 1};
  const cuuint32_t estr[2] = {1, 1};
  if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(x), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  static std::once_flag attr;
  std::call_once(attr, [] {
    SBHA_CUDA(cudaFuncSetAttribute(k_spmm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(kSmemBytes)));
  });
  const int64_t items = static_cast<int64_t>(tp.ntiles) * ((nb + kGroup - 1) / kGroup);
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(items, num_sms()));
  k_spmm_tma<<<grid, kThreads, kSmemBytes, c.stream>>>(map, tp.m, nb, tp.ntiles, tp.rowptr, tp.col, tp.lcol,
                                                       tp.lself, tp.halo, tp.nh, val, x, y, alpha, acc, blk_act,
                                                       self_dot, c.d_err, wait_limit());
  c.launched("spmm_tma");
  return true;
}

}  // namespace sbha
