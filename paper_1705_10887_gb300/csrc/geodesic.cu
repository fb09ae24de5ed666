// Shortest paths along mesh edges (Eq. 1 on the edge graph) and farthest-point
// landmarks (Eq. 5).
//
// Both use frontier relaxation: a CTA keeps a queue of vertices whose distance just
// dropped, relaxes their edges with an atomic minimum (non-negative doubles order
// like their bit patterns), and queues every vertex it lowered, until the queue is
// empty.  Each distance written is the left-fold sum of the edge lengths of some
// path from the source, and fl(d + w) is monotone in d, so the relaxation ends at
// the unique fixed point d(v) = min_u fl(d(u) + w(u,v)) -- the same doubles any exact
// shortest-path algorithm produces with the same edge lengths, independent of the
// order in which the threads happen to run.
//
// Farthest-point selection relaxes the new landmark's wave directly into the running
// minimum-distance field and propagates only where that field drops: a vertex whose
// distance from the new landmark is not below its current minimum cannot lower any
// vertex behind it (the earlier landmark reaches those through it at least as
// cheaply), so each step touches only the new landmark's Voronoi cell.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <vector>

#include "internal.cuh"

namespace sbha {

namespace {

constexpr int kFpsThreads = 1024;
constexpr int kSegShift = 5;    // argmax segments of 32 vertices
constexpr int kTileShift = 10;  // argmax tiles of 32 segments
constexpr int kSsspThreads = 512;
constexpr int kEdgeLanes = 8;   // threads sharing one queued vertex's edges

// Relaxation rounds of one wave inside one CTA.  The field being lowered is dist[v - dbase]
// (stamps likewise) for the vertices v of one connected component; the first queue holds the
// seeds and s_cnt[0] their number.  Eight threads share the edges of each queued vertex, so all
// the round's atomic updates are in flight together.  The queue counters are double-buffered:
// two barriers per round.  With seg_dirty, every 32-vertex segment (numbered from vertex seg_v0,
// plus seg_base) holding a lowered vertex is listed once in seg_list (count in *s_nseg).
// Returns when no distance dropped in a round.
__device__ void wave(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                     const double* __restrict__ len, double* dist, int32_t* qa, int32_t* qb, int32_t* stamp,
                     int* s_cnt, int& stamp_id, int32_t* seg_dirty, int32_t* seg_list, int* s_nseg, int dbase = 0,
                     int seg_v0 = 0, int seg_base = 0) {
  int32_t* cur = qa;
  int32_t* nxt = qb;
  for (int r = 0;; ++r) {
    __syncthreads();
    const int cn = s_cnt[r & 1];
    if (cn == 0) break;
    ++stamp_id;
    if (threadIdx.x == 0) s_cnt[(r + 1) & 1] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < cn * kEdgeLanes; t += blockDim.x) {
      int u = cur[t / kEdgeLanes];
      double du = __ldcg(dist + (u - dbase));
      int e1 = rowptr[u + 1];
      for (int e = rowptr[u] + t % kEdgeLanes; e < e1; e += kEdgeLanes) {
        int w = col[e];
        double cand = __dadd_rn(du, len[e]);
        unsigned long long old = atomic_min_nonneg(dist + (w - dbase), cand);
        if (dbits(cand) < old) {
          if (seg_dirty) {
            int sg = seg_base + ((w - seg_v0) >> kSegShift);
            if (atomicExch(seg_dirty + sg, 1) == 0) seg_list[atomicAdd(s_nseg, 1)] = sg;
          }
          if (atomicExch(stamp + (w - dbase), stamp_id) != stamp_id) nxt[atomicAdd(&s_cnt[(r + 1) & 1], 1)] = w;
        }
      }
    }
    int32_t* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
}

// Larger value wins; equal values go to the smaller index.
__device__ __forceinline__ void argmax_merge(double& v, int& i, double ov, int oi) {
  if (ov > v || (ov == v && oi < i)) {
    v = ov;
    i = oi;
  }
}

__device__ __forceinline__ void warp_argmax(double& bv, int& bi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    argmax_merge(bv, bi, ov, oi);
  }
}

// Block-wide argmax (larger value, then smaller index), result broadcast to every thread.
__device__ void block_argmax(double& bv, int& bi, double* s_v, int* s_i) {
  warp_argmax(bv, bi);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    s_v[warp] = bv;
    s_i[warp] = bi;
  }
  __syncthreads();
  if (warp == 0) {
    bv = lane < (int)(blockDim.x / 32) ? s_v[lane] : -1.0;
    bi = lane < (int)(blockDim.x / 32) ? s_i[lane] : INT_MAX;
    warp_argmax(bv, bi);
    if (lane == 0) {
      s_v[0] = bv;
      s_i[0] = bi;
    }
  }
  __syncthreads();
  bv = s_v[0];
  bi = s_i[0];
}

// All l steps of one mesh in one CTA; with several jobs, one CTA per mesh (a connected component
// of the graph, vertices [v0, v0 + n)), all in one launch.  The argmax is kept in three levels: the
// running minimum distance of every vertex, the maximum of every 32-vertex segment (global
// memory), and the maximum of every tile of 32 segments (shared memory).  After each wave only
// the segments it lowered, and then their tiles, are recomputed (a warp each); the next landmark
// is the argmax over the tiles.  Segments and tiles start at +inf, so a vertex no wave reaches
// stays visible.  Landmark ids are written relative to v0.
__global__ void __launch_bounds__(kFpsThreads) k_fps(const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col, const double* __restrict__ len,
                                                      const FpsJob* __restrict__ jobs, double* mind,
                                                      int32_t* __restrict__ idx, int32_t* qa, int32_t* qb,
                                                      int32_t* stamp, double* seg_v, int32_t* seg_i, int32_t* seg_dirty,
                                                      int32_t* seg_list, int* err) {
  extern __shared__ double fps_smem[];
  __shared__ int s_cnt[2], s_nseg, s_ntile;
  __shared__ double s_v[kFpsThreads / 32];
  __shared__ int s_i[kFpsThreads / 32];
  const FpsJob job = jobs[blockIdx.x];
  const int v0 = job.v0, n = job.n, l = job.l, sb = job.seg_base;
  const int nseg = (n + (1 << kSegShift) - 1) >> kSegShift;
  const int ntiles = (n + (1 << kTileShift) - 1) >> kTileShift;
  double* tv = fps_smem;
  int* ti = reinterpret_cast<int*>(tv + ntiles);
  int* tdirty = ti + ntiles;
  int* tlist = tdirty + ntiles;
  int32_t* cq = qa + v0;  // this mesh's queues
  int32_t* nq = qb + v0;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  for (int v = v0 + threadIdx.x; v < v0 + n; v += blockDim.x) {
    mind[v] = inf;
    stamp[v] = -1;
  }
  for (int ls = threadIdx.x; ls < nseg; ls += blockDim.x) {
    seg_v[sb + ls] = inf;
    seg_i[sb + ls] = v0 + (ls << kSegShift);
    seg_dirty[sb + ls] = 0;
  }
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    tv[t] = inf;
    ti[t] = v0 + (t << kTileShift);
    tdirty[t] = 0;
  }
  if (threadIdx.x == 0) {
    s_nseg = 0;
    s_ntile = 0;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int stamp_id = 0;
  int b = v0 + job.first;
  for (int j = 0; j < l; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) {
      idx[job.idx_off + j] = b - v0;
      mind[b] = 0.0;
      int sg = sb + ((b - v0) >> kSegShift);
      if (atomicExch(seg_dirty + sg, 1) == 0) seg_list[sb + s_nseg++] = sg;
      cq[0] = b;
      s_cnt[0] = 1;
    }
    wave(rowptr, col, len, mind, cq, nq, stamp, s_cnt, stamp_id, seg_dirty, seg_list + sb, &s_nseg, 0, v0, sb);
    if (j + 1 == l) break;
    __syncthreads();
    const int nd = s_nseg;
    for (int k = warp; k < nd; k += kFpsThreads / 32) {  // lowered segments, a warp each
      int sg = seg_list[sb + k];
      int ls = sg - sb;
      int lv = (ls << kSegShift) + lane;
      double bv = lv < n ? __ldcg(mind + v0 + lv) : -1.0;
      int bi = lv < n ? v0 + lv : INT_MAX;
      warp_argmax(bv, bi);
      if (lane == 0) {
        seg_v[sg] = bv;
        seg_i[sg] = bi;
        seg_dirty[sg] = 0;
        int t = ls >> (kTileShift - kSegShift);
        if (atomicExch(tdirty + t, 1) == 0) tlist[atomicAdd(&s_ntile, 1)] = t;
      }
    }
    __syncthreads();
    const int nt = s_ntile;
    for (int k = warp; k < nt; k += kFpsThreads / 32) {  // their tiles, a warp each
      int t = tlist[k];
      int ls = (t << (kTileShift - kSegShift)) + lane;
      double bv = ls < nseg ? __ldcg(seg_v + sb + ls) : -1.0;
      int bi = ls < nseg ? __ldcg(seg_i + sb + ls) : INT_MAX;
      warp_argmax(bv, bi);
      if (lane == 0) {
        tv[t] = bv;
        ti[t] = bi;
        tdirty[t] = 0;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_nseg = 0;
      s_ntile = 0;
    }
    // b_{j+1} = argmax over the tile maxima (lowest index on ties)
    double bv = -1.0;
    int bi = INT_MAX;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) argmax_merge(bv, bi, tv[t], ti[t]);
    block_argmax(bv, bi, s_v, s_i);
    if (bv > DBL_MAX) {
      if (threadIdx.x == 0) set_error(err, DERR_DISCONNECTED);
      break;
    }
    b = bi;
  }
}

// Landmark distances of many meshes in one launch: one CTA per (mesh, source landmark); the
// wave stays in the mesh's component (vertices [v0, v0 + n)), whose work arrays it owns.
__global__ void __launch_bounds__(kSsspThreads) k_sssp_jobs(const int32_t* __restrict__ rowptr,
                                                             const int32_t* __restrict__ col,
                                                             const double* __restrict__ len,
                                                             const SsspJob* __restrict__ jobs, double* dist_ws,
                                                             int32_t* qa_ws, int32_t* qb_ws, int32_t* stamp_ws,
                                                             const int32_t* __restrict__ tgt, double* __restrict__ out) {
  __shared__ int s_cnt[2];
  const SsspJob job = jobs[blockIdx.x];
  double* dist = dist_ws + job.ws_off;
  int32_t* qa = qa_ws + job.ws_off;
  int32_t* qb = qb_ws + job.ws_off;
  int32_t* stamp = stamp_ws + job.ws_off;
  for (int v = threadIdx.x; v < job.n; v += blockDim.x) {
    dist[v] = __longlong_as_double(0x7ff0000000000000LL);
    stamp[v] = -1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    dist[job.src - job.v0] = 0.0;
    qa[0] = job.src;
    s_cnt[0] = 1;
  }
  int stamp_id = 0;
  wave(rowptr, col, len, dist, qa, qb, stamp, s_cnt, stamp_id, nullptr, nullptr, nullptr, job.v0, 0, 0);
  __syncthreads();
  double* row = out + job.out_off;
  for (int b = threadIdx.x; b < job.t; b += blockDim.x) row[b] = __ldcg(dist + (tgt[job.tgt_off + b] - job.v0));
}

// One CTA per source: full single-source wave, then gather the requested targets.
__global__ void __launch_bounds__(kSsspThreads) k_sssp(int n, const int32_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ len, const int32_t* __restrict__ src,
                                                        double* dist_ws, int32_t* qa_ws, int32_t* qb_ws,
                                                        int32_t* stamp_ws, const int32_t* __restrict__ tgt, int t,
                                                        double* __restrict__ out, int64_t out_stride) {
  __shared__ int s_cnt[2];
  int64_t off = static_cast<int64_t>(blockIdx.x) * n;
  double* dist = dist_ws + off;
  int32_t* qa = qa_ws + off;
  int32_t* qb = qb_ws + off;
  int32_t* stamp = stamp_ws + off;
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    dist[v] = __longlong_as_double(0x7ff0000000000000LL);
    stamp[v] = -1;
  }
  __syncthreads();
  int s = src[blockIdx.x];
  if (threadIdx.x == 0) {
    dist[s] = 0.0;
    qa[0] = s;
    s_cnt[0] = 1;
  }
  int stamp_id = 0;
  wave(rowptr, col, len, dist, qa, qb, stamp, s_cnt, stamp_id, nullptr, nullptr, nullptr);
  __syncthreads();
  double* row = out + static_cast<int64_t>(blockIdx.x) * out_stride;
  if (tgt) {
    for (int b = threadIdx.x; b < t; b += blockDim.x) row[b] = __ldcg(dist + tgt[b]);
  } else {
    for (int v = threadIdx.x; v < n; v += blockDim.x) row[v] = __ldcg(dist + v);
  }
}

__global__ void k_check_ids(const int32_t* __restrict__ ids, int count, int n, int* err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    if (ids[i] < 0 || ids[i] >= n) set_error(err, DERR_BAD_INDEX);
}

// W_ij = (D_ij + D_ji) / 2, W_ii = 0
__global__ void k_symmetrise(const double* __restrict__ D, double* __restrict__ W, int l) {
  int64_t total = static_cast<int64_t>(l) * l;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int i = static_cast<int>(q / l), j = static_cast<int>(q % l);
    W[q] = (i == j) ? 0.0 : __dmul_rn(__dadd_rn(D[q], D[static_cast<int64_t>(j) * l + i]), 0.5);
  }
}

}  // namespace

void fps_jobs(Ctx& c, const DevGraph& g, const std::vector<FpsJob>& jobs, int32_t* idx, double* mind) {
  if (jobs.empty()) return;
  int32_t* qa = c.alloc<int32_t>(g.n);
  int32_t* qb = c.alloc<int32_t>(g.n);
  int32_t* stamp = c.alloc<int32_t>(g.n);
  int64_t nseg = 0;
  int max_n = 0;
  for (const FpsJob& j : jobs) {
    nseg = std::max<int64_t>(nseg, j.seg_base + ((j.n + (1 << kSegShift) - 1) >> kSegShift));
    max_n = std::max(max_n, j.n);
  }
  double* seg_v = c.alloc<double>(nseg);
  int32_t* seg_i = c.alloc<int32_t>(nseg);
  int32_t* seg_dirty = c.alloc<int32_t>(nseg);
  int32_t* seg_list = c.alloc<int32_t>(nseg);
  FpsJob* djobs = c.alloc<FpsJob>(jobs.size());
  SBHA_CUDA(cudaMemcpyAsync(djobs, jobs.data(), sizeof(FpsJob) * jobs.size(), cudaMemcpyHostToDevice, c.stream));
  int ntiles = (max_n + (1 << kTileShift) - 1) >> kTileShift;
  size_t smem = static_cast<size_t>(ntiles) * (sizeof(double) + 3 * sizeof(int));
  if (smem > 200 * 1024) SBHA_THROW(SBHA_EINVAL, "mesh too large for the landmark kernel's tile table");
  if (smem > 48 * 1024)
    SBHA_CUDA(cudaFuncSetAttribute(k_fps, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  k_fps<<<static_cast<unsigned>(jobs.size()), kFpsThreads, smem, c.stream>>>(g.rowptr, g.col, g.len, djobs, mind, idx,
                                                                              qa, qb, stamp, seg_v, seg_i, seg_dirty,
                                                                              seg_list, c.d_err);
  c.launched("fps");
  c.check_device("landmarks");
  for (void* p : {static_cast<void*>(qa), static_cast<void*>(qb), static_cast<void*>(stamp), static_cast<void*>(seg_v),
                  static_cast<void*>(seg_i), static_cast<void*>(seg_dirty), static_cast<void*>(seg_list),
                  static_cast<void*>(djobs)})
    c.free(p);
}

void fps(Ctx& c, const DevGraph& g, int32_t l, int32_t first, int32_t* idx, double* mind) {
  fps_jobs(c, g, {FpsJob{0, static_cast<int32_t>(g.n), l, first, 0, 0}}, idx, mind);
}

void sssp_jobs(Ctx& c, const DevGraph& g, const std::vector<SsspJob>& jobs, const int32_t* tgt, double* out) {
  // jobs in launches whose work arrays (20 bytes per component vertex) stay under ~4 GB
  size_t i = 0;
  while (i < jobs.size()) {
    std::vector<SsspJob> batch;
    int64_t ws = 0;
    while (i < jobs.size() && batch.size() < 65535 &&
           (batch.empty() || (ws + jobs[i].n) * 20LL < (4LL << 30))) {
      SsspJob j = jobs[i++];
      j.ws_off = ws;
      ws += j.n;
      batch.push_back(j);
    }
    double* dist = c.alloc<double>(ws);
    int32_t* qa = c.alloc<int32_t>(ws);
    int32_t* qb = c.alloc<int32_t>(ws);
    int32_t* stamp = c.alloc<int32_t>(ws);
    SsspJob* dj = c.alloc<SsspJob>(batch.size());
    SBHA_CUDA(cudaMemcpyAsync(dj, batch.data(), sizeof(SsspJob) * batch.size(), cudaMemcpyHostToDevice, c.stream));
    k_sssp_jobs<<<static_cast<unsigned>(batch.size()), kSsspThreads, 0, c.stream>>>(g.rowptr, g.col, g.len, dj, dist,
                                                                                    qa, qb, stamp, tgt, out);
    c.launched("sssp_jobs");
    c.sync();  // the job table is host memory staged per launch
    for (void* p : {static_cast<void*>(dist), static_cast<void*>(qa), static_cast<void*>(qb),
                    static_cast<void*>(stamp), static_cast<void*>(dj)})
      c.free(p);
  }
}

void symmetrise(Ctx& c, const double* D, double* W, int32_t l) {
  k_symmetrise<<<grid_for(static_cast<int64_t>(l) * l, 256), 256, 0, c.stream>>>(D, W, l);
  c.launched("symmetrise");
}

void geodesics(Ctx& c, const DevGraph& g, const int32_t* src, int32_t s, const int32_t* tgt, int32_t t, double* D) {
  int n = static_cast<int>(g.n);
  k_check_ids<<<grid_for(s, 256), 256, 0, c.stream>>>(src, s, n, c.d_err);
  c.launched("check_ids");
  if (tgt) {
    k_check_ids<<<grid_for(t, 256), 256, 0, c.stream>>>(tgt, t, n, c.d_err);
    c.launched("check_ids");
  }
  c.check_device("geodesics");
  // sources per launch: keep the per-source work arrays (20 bytes per vertex) under ~4 GB
  int64_t per_src = 20LL * n;
  int64_t batch = (4LL << 30) / per_src;
  if (batch < 1) batch = 1;
  if (batch > s) batch = s;
  if (batch > 65535) batch = 65535;
  double* dist = c.alloc<double>(batch * n);
  int32_t* qa = c.alloc<int32_t>(batch * n);
  int32_t* qb = c.alloc<int32_t>(batch * n);
  int32_t* stamp = c.alloc<int32_t>(batch * n);
  int64_t stride = tgt ? t : n;
  for (int64_t s0 = 0; s0 < s; s0 += batch) {
    int64_t cnt = (s - s0 < batch) ? s - s0 : batch;
    k_sssp<<<static_cast<unsigned>(cnt), kSsspThreads, 0, c.stream>>>(n, g.rowptr, g.col, g.len, src + s0, dist, qa,
                                                                       qb, stamp, tgt, t, D + s0 * stride, stride);
    c.launched("sssp");
  }
  c.free(dist);
  c.free(qa);
  c.free(qb);
  c.free(stamp);
}

void landmark_block(Ctx& c, const DevGraph& g, const int32_t* idx, int32_t l, double* W) {
  double* D = c.alloc<double>(static_cast<size_t>(l) * l);
  geodesics(c, g, idx, l, idx, l, D);
  k_symmetrise<<<grid_for(static_cast<int64_t>(l) * l, 256), 256, 0, c.stream>>>(D, W, l);
  c.launched("symmetrise");
  c.free(D);
}

}  // namespace sbha
