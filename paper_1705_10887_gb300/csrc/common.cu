// Host infrastructure: per-thread status, workspace, pointer classification, prefix sums.
#include "common.cuh"

#include <atomic>

namespace sbha {

sbha_stats& thread_stats() {
  static thread_local sbha_stats s{};
  return s;
}

std::string& thread_error() {
  static thread_local std::string e;
  return e;
}

Ctx::Ctx(void* s) : stream(static_cast<cudaStream_t>(s)) {
  d_err = alloc<int>(1);
  SBHA_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), stream));
}

Ctx::~Ctx() {
  for (void* p : blocks)
    if (p) cudaFreeAsync(p, stream);
  cudaStreamSynchronize(stream);
}

void* Ctx::raw_alloc(size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    SBHA_THROW(SBHA_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                cudaGetErrorString(e));
  }
  blocks.push_back(p);
  return p;
}

void Ctx::free(void* p) {
  for (auto& b : blocks)
    if (b == p) {
      cudaFreeAsync(b, stream);
      b = nullptr;
      return;
    }
}

void Ctx::launched(const char* what) {
  ++launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) SBHA_THROW(SBHA_ECUDA, std::string("launch of ") + what + ": " + cudaGetErrorString(e));
}

void Ctx::sync() { SBHA_CUDA(cudaStreamSynchronize(stream)); }

void Ctx::check_device(const char* stage) {
  int h = 0;
  SBHA_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  SBHA_CUDA(cudaStreamSynchronize(stream));
  if (h == DERR_NONE) return;
  std::string where = std::string(stage) + ": ";
  switch (h) {
    case DERR_BAD_FACE: SBHA_THROW(SBHA_EINVAL, where + "a face has a vertex id out of range or repeated");
    case DERR_NON_MANIFOLD: SBHA_THROW(SBHA_EINVAL, where + "an edge belongs to more than two faces");
    case DERR_VALENCE: SBHA_THROW(SBHA_EINVAL, where + "a vertex has more incident faces than the assembly supports (64)");
    case DERR_TWO_RING: SBHA_THROW(SBHA_EINVAL, where + "a vertex 2-ring exceeds the operator capacity (192)");
    case DERR_DISCONNECTED: SBHA_THROW(SBHA_EDISCONNECTED, where + "the mesh is not connected along its edges");
    case DERR_BAD_INDEX: SBHA_THROW(SBHA_EINVAL, where + "a vertex id is out of range");
    case DERR_DUPLICATE: SBHA_THROW(SBHA_EINVAL, where + "a landmark is listed twice");
    case DERR_BAD_CSR: SBHA_THROW(SBHA_EINVAL, where + "malformed CSR input (column out of range or row too long)");
    case DERR_TIMEOUT: SBHA_THROW(SBHA_ETIMEOUT, where + "a bounded device-side wait (tensor-core or TMA pipeline) gave up");
    case DERR_ISOLATED: SBHA_THROW(SBHA_EINVAL, where + "a vertex belongs to no triangle");
    case DERR_NOT_SPD: SBHA_THROW(SBHA_ENOCONV, where + "a small Gram matrix lost positive definiteness");
    default: SBHA_THROW(SBHA_ECUDA, where + "device error " + std::to_string(h));
  }
}

int num_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    dev = -1;
  }
  if (dev >= 0) {
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev < 0 ? 0 : dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 152;  // GB300's count when the runtime cannot say (no device: host-only calls)
  }
  if (dev >= 0) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------ prefix sum ---

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one tile; writes the tile total to tile_sums[blockIdx.x].
__global__ void k_scan_tiles(const int32_t* __restrict__ in, int32_t* __restrict__ out, int32_t* __restrict__ tile_sums,
                             int64_t n) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;  // inclusive
  }
  __syncthreads();
  int32_t run = inc - s + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = run;
}

__global__ void k_scan_add(int32_t* __restrict__ out, const int32_t* __restrict__ tile_offsets, int64_t n) {
  int64_t i = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x;
  int32_t add = tile_offsets[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k, i += kScanThreads)
    if (i < n) out[i] += add;
}

void scan_rec(Ctx& c, const int32_t* in, int32_t* out, int64_t n) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles < 1) tiles = 1;
  int32_t* sums = c.alloc<int32_t>(tiles + 1);
  k_scan_tiles<<<static_cast<unsigned>(tiles), kScanThreads, 0, c.stream>>>(in, out, sums, n);
  c.launched("scan_tiles");
  if (tiles > 1) {
    int32_t* offs = c.alloc<int32_t>(tiles + 1);
    scan_rec(c, sums, offs, tiles);
    k_scan_add<<<static_cast<unsigned>(tiles), kScanThreads, 0, c.stream>>>(out, offs, n);
    c.launched("scan_add");
  }
}

}  // namespace

int64_t exclusive_scan(Ctx& c, const int32_t* in, int32_t* out, int64_t n) {
  // out[0..n-1] = exclusive scan; out[n] = total (computed as out[n-1] + in[n-1])
  if (n == 0) {
    SBHA_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), c.stream));
    return 0;
  }
  scan_rec(c, in, out, n);
  int32_t last_out = 0, last_in = 0;
  SBHA_CUDA(cudaMemcpyAsync(&last_out, out + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  SBHA_CUDA(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  SBHA_CUDA(cudaStreamSynchronize(c.stream));
  int64_t total = static_cast<int64_t>(last_out) + last_in;
  if (total > INT32_MAX) SBHA_THROW(SBHA_EINVAL, "prefix sum exceeds the int32 range of CSR offsets");
  int32_t t32 = static_cast<int32_t>(total);
  SBHA_CUDA(cudaMemcpyAsync(out + n, &t32, sizeof(int32_t), cudaMemcpyHostToDevice, c.stream));
  SBHA_CUDA(cudaStreamSynchronize(c.stream));
  return total;
}

}  // namespace sbha
