// Shared host/device infrastructure of the sBHA CUDA library: status handling,
// stream-ordered workspace, host/device argument staging, prefix sums and the
// small warp/block helpers the kernels use.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sbha.h"

namespace sbha {

// ---------------------------------------------------------------- status ---

struct Error {
  int status;
  std::string msg;
};

// Per-thread diagnostics (see sbha_last_stats / sbha_last_error).
sbha_stats& thread_stats();
std::string& thread_error();

#define SBHA_THROW(code, text)          \
  do {                                  \
    throw ::sbha::Error{(code), (text)}; \
  } while (0)

#define SBHA_CUDA(call)                                                                              \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      throw ::sbha::Error{e_ == cudaErrorMemoryAllocation ? SBHA_ENOMEM : SBHA_ECUDA,                \
                          std::string(#call) + ": " + cudaGetErrorString(e_) + " at " __FILE__ ":" + \
                              std::to_string(__LINE__)};                                             \
  } while (0)

// Device-side error codes written by kernels into Ctx::d_err (first one wins).
enum DeviceError : int {
  DERR_NONE = 0,
  DERR_BAD_FACE = 1,      // face vertex out of range or repeated
  DERR_NON_MANIFOLD = 2,  // an edge in more than two faces
  DERR_VALENCE = 3,       // a vertex exceeds the per-vertex capacity of the assembly kernels
  DERR_TWO_RING = 4,      // a 2-ring exceeds the capacity of the operator kernel
  DERR_DISCONNECTED = 5,  // unreachable vertex
  DERR_BAD_INDEX = 6,     // landmark / source / target id out of range
  DERR_DUPLICATE = 7,     // landmark listed twice
  DERR_BAD_CSR = 8,       // CSR column out of range or row too long
  DERR_NOT_SPD = 9,       // non-positive pivot / Gram in a small dense factorisation
  DERR_ISOLATED = 10,     // a vertex belongs to no face
  DERR_TIMEOUT = 11,      // a bounded device-side wait gave up
};

// ------------------------------------------------------------- workspace ---

// Everything one API call needs on the device.  Allocations are stream-ordered
// (cudaMallocAsync on the call's stream) and released by the destructor.
struct Ctx {
  cudaStream_t stream = nullptr;
  int* d_err = nullptr;
  int64_t launches = 0;
  int timing = 0;  // opts.timing of the call
  bool graphs = true;  // CG solves may finish as device-decided CUDA graphs (opts.cg_graph)
  std::vector<void*> blocks;

  explicit Ctx(void* s);
  ~Ctx();
  Ctx(const Ctx&) = delete;
  Ctx& operator=(const Ctx&) = delete;

  void* raw_alloc(size_t bytes);
  template <class T>
  T* alloc(size_t count) {
    return static_cast<T*>(raw_alloc(sizeof(T) * (count ? count : 1)));
  }
  template <class T>
  T* zeros(size_t count) {
    T* p = alloc<T>(count);
    SBHA_CUDA(cudaMemsetAsync(p, 0, sizeof(T) * (count ? count : 1), stream));
    return p;
  }
  void free(void* p);

  // Kernel launch bookkeeping: checks the launch and counts it.
  void launched(const char* what);
  // Reads d_err (synchronises the stream) and throws on a device-side error.
  void check_device(const char* stage);
  void sync();
};

// True if `p` is device (or managed) memory of the current device.
bool is_device_ptr(const void* p);

// Returns a device copy of a caller array (or the pointer itself if already on the device).
template <class T>
const T* stage_in(Ctx& c, const T* p, size_t count) {
  if (p == nullptr || is_device_ptr(p)) return p;
  T* d = c.alloc<T>(count);
  SBHA_CUDA(cudaMemcpyAsync(d, p, sizeof(T) * count, cudaMemcpyHostToDevice, c.stream));
  return d;
}

// Output staging: device buffer to write, copied back to the caller's host array by finish().
template <class T>
struct Out {
  T* user = nullptr;
  T* dev = nullptr;
  size_t count = 0;
  bool host = false;
  void init(Ctx& c, T* p, size_t n) {
    user = p;
    count = n;
    host = p != nullptr && !is_device_ptr(p);
    dev = host ? c.alloc<T>(n) : p;
  }
  void finish(Ctx& c) {
    if (host && count) SBHA_CUDA(cudaMemcpyAsync(user, dev, sizeof(T) * count, cudaMemcpyDeviceToHost, c.stream));
  }
};

// Exclusive prefix sum of n int32 counts into out[0..n] (out[n] = total); returns the total.
int64_t exclusive_scan(Ctx& c, const int32_t* in, int32_t* out, int64_t n);

// ------------------------------------------------------------- launches ----

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, cached per
// device ordinal; 152 on GB300).
int num_sms();

// Blocks for `items` work items at `per_block` each, capped at max_blocks (0: 16 per SM).
inline unsigned grid_for(int64_t items, int per_block, int max_blocks = 0) {
  if (max_blocks <= 0) max_blocks = 16 * num_sms();
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return static_cast<unsigned>(g);
}

// ---------------------------------------------------------- device utils ---

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

// Non-negative doubles order like their bit patterns read as unsigned integers.
__device__ __forceinline__ unsigned long long dbits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}

// atomic min on a non-negative double; returns the previous value's bits
__device__ __forceinline__ unsigned long long atomic_min_nonneg(double* addr, double v) {
  return atomicMin(reinterpret_cast<unsigned long long*>(addr), dbits(v));
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace sbha
