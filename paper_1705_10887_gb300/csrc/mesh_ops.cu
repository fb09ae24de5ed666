// Mesh assembly on the GPU (Sec. 2.2): edge graph in CSR, Euclidean edge lengths,
// cotangent weights A_ij = (cot alpha_ij + cot beta_ij) / 2, lumped mass D_ii = a third of
// the incident triangle areas, V_ii = sum_j A_ij, and the biharmonic operator
// M = (V - A)^T D^{-1} (V - A) on its 2-ring pattern.
//
// Design: every output row is produced by the thread that owns the vertex, by
// gathering over the vertex's incident triangles (vertex -> face incidence is built
// with a counting pass, a prefix sum and a per-vertex sort).  No atomics touch
// floating-point data, so every value is formed in a fixed order: the edge
// lengths, cotangents, masses and operator entries are the same doubles on every
// run.  Operations that must match a reference bit for bit use explicit
// round-to-nearest intrinsics so that the compiler cannot fuse them.
#include "internal.cuh"

namespace sbha {

namespace {

__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }

// sqrt((dx*dx + dy*dy) + dz*dz), dx = x_j - x_i
__device__ __forceinline__ double edge_length(const double* __restrict__ xyz, int i, int j) {
  double dx = dsub(xyz[3 * j + 0], xyz[3 * i + 0]);
  double dy = dsub(xyz[3 * j + 1], xyz[3 * i + 1]);
  double dz = dsub(xyz[3 * j + 2], xyz[3 * i + 2]);
  return __dsqrt_rn(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)));
}

// cot of the angle at c in triangle (a, b, c): (e1 . e2) / |e1 x e2|, e1 = x_a - x_c, e2 = x_b - x_c
__device__ double cot_at(const double* __restrict__ xyz, int a, int b, int c) {
  double e1x = dsub(xyz[3 * a + 0], xyz[3 * c + 0]);
  double e1y = dsub(xyz[3 * a + 1], xyz[3 * c + 1]);
  double e1z = dsub(xyz[3 * a + 2], xyz[3 * c + 2]);
  double e2x = dsub(xyz[3 * b + 0], xyz[3 * c + 0]);
  double e2y = dsub(xyz[3 * b + 1], xyz[3 * c + 1]);
  double e2z = dsub(xyz[3 * b + 2], xyz[3 * c + 2]);
  double dot = dadd(dadd(dmul(e1x, e2x), dmul(e1y, e2y)), dmul(e1z, e2z));
  double cx = dsub(dmul(e1y, e2z), dmul(e1z, e2y));
  double cy = dsub(dmul(e1z, e2x), dmul(e1x, e2z));
  double cz = dsub(dmul(e1x, e2y), dmul(e1y, e2x));
  return __ddiv_rn(dot, __dsqrt_rn(dadd(dadd(dmul(cx, cx), dmul(cy, cy)), dmul(cz, cz))));
}

// A triangle's edges in its stored order: (a,b) opposite c, (b,c) opposite a, (c,a) opposite b.
// Returns the cotangent opposite the edge {v, w} of triangle (a, b, c).
__device__ double cot_opposite(const double* __restrict__ xyz, int a, int b, int c, int v, int w) {
  if ((v == a && w == b) || (v == b && w == a)) return cot_at(xyz, a, b, c);
  if ((v == b && w == c) || (v == c && w == b)) return cot_at(xyz, b, c, a);
  return cot_at(xyz, c, a, b);
}

// 0.5 * |(x_b - x_a) x (x_c - x_a)|
__device__ double triangle_area(const double* __restrict__ xyz, int a, int b, int c) {
  double ux = dsub(xyz[3 * b + 0], xyz[3 * a + 0]), uy = dsub(xyz[3 * b + 1], xyz[3 * a + 1]),
         uz = dsub(xyz[3 * b + 2], xyz[3 * a + 2]);
  double wx = dsub(xyz[3 * c + 0], xyz[3 * a + 0]), wy = dsub(xyz[3 * c + 1], xyz[3 * a + 1]),
         wz = dsub(xyz[3 * c + 2], xyz[3 * a + 2]);
  double nx = dsub(dmul(uy, wz), dmul(uz, wy));
  double ny = dsub(dmul(uz, wx), dmul(ux, wz));
  double nz = dsub(dmul(ux, wy), dmul(uy, wx));
  return dmul(0.5, __dsqrt_rn(dadd(dadd(dmul(nx, nx), dmul(ny, ny)), dmul(nz, nz))));
}

__global__ void k_face_count(int64_t f, int64_t n, const int32_t* __restrict__ faces, int32_t* __restrict__ cnt,
                             int* err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < f; t += (int64_t)gridDim.x * blockDim.x) {
    int a = faces[3 * t], b = faces[3 * t + 1], c = faces[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n || a == b || b == c || a == c) {
      set_error(err, DERR_BAD_FACE);
      continue;
    }
    atomicAdd(&cnt[a], 1);
    atomicAdd(&cnt[b], 1);
    atomicAdd(&cnt[c], 1);
  }
}

__global__ void k_face_fill(int64_t f, const int32_t* __restrict__ faces, const int32_t* __restrict__ vfptr,
                            int32_t* __restrict__ cursor, int32_t* __restrict__ vf) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < f; t += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int v = faces[3 * t + k];
      int pos = vfptr[v] + atomicAdd(&cursor[v], 1);
      vf[pos] = static_cast<int32_t>(t);
    }
  }
}

// Sort every vertex's incident-face list ascending (face order fixes the mass summation order).
__global__ void k_face_sort(int64_t n, const int32_t* __restrict__ vfptr, int32_t* __restrict__ vf, int* err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int s = vfptr[v], e = vfptr[v + 1];
    if (e == s) {
      set_error(err, DERR_ISOLATED);
      continue;
    }
    if (e - s > kMaxFaces) {
      set_error(err, DERR_VALENCE);
      continue;
    }
    for (int p = s + 1; p < e; ++p) {
      int key = vf[p], q = p - 1;
      while (q >= s && vf[q] > key) {
        vf[q + 1] = vf[q];
        --q;
      }
      vf[q + 1] = key;
    }
  }
}

// Sorted unique 1-ring of v with the number of faces on each edge.  Returns the count or -1.
__device__ int gather_ring(int v, const int32_t* __restrict__ faces, const int32_t* __restrict__ vfptr,
                           const int32_t* __restrict__ vf, int* nb, int* mult, int* err) {
  int cnt = 0;
  for (int q = vfptr[v]; q < vfptr[v + 1]; ++q) {
    int t = vf[q];
    int a = faces[3 * t], b = faces[3 * t + 1], c = faces[3 * t + 2];
    int others[2];
    if (a == v) { others[0] = b; others[1] = c; }
    else if (b == v) { others[0] = c; others[1] = a; }
    else { others[0] = a; others[1] = b; }
    for (int k = 0; k < 2; ++k) {
      int w = others[k];
      int pos = 0;
      while (pos < cnt && nb[pos] < w) ++pos;
      if (pos < cnt && nb[pos] == w) {
        if (++mult[pos] > 2) {
          set_error(err, DERR_NON_MANIFOLD);
          return -1;
        }
        continue;
      }
      if (cnt == kMaxNbrs) {
        set_error(err, DERR_VALENCE);
        return -1;
      }
      for (int r = cnt; r > pos; --r) {
        nb[r] = nb[r - 1];
        mult[r] = mult[r - 1];
      }
      nb[pos] = w;
      mult[pos] = 1;
      ++cnt;
    }
  }
  return cnt;
}

__global__ void k_ring_count(int64_t n, const int32_t* __restrict__ faces, const int32_t* __restrict__ vfptr,
                             const int32_t* __restrict__ vf, int32_t* __restrict__ deg, int* err) {
  int nb[kMaxNbrs], mult[kMaxNbrs];
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int c = gather_ring(static_cast<int>(v), faces, vfptr, vf, nb, mult, err);
    deg[v] = c < 0 ? 0 : c;
  }
}

// Row v of the edge graph: neighbours, lengths, cotangent weights; lumped mass and weight sum.
__global__ void k_ring_fill(int64_t n, const double* __restrict__ xyz, const int32_t* __restrict__ faces,
                            const int32_t* __restrict__ vfptr, const int32_t* __restrict__ vf,
                            const int32_t* __restrict__ rowptr, int32_t* __restrict__ col, double* __restrict__ len,
                            double* __restrict__ A, double* __restrict__ D, double* __restrict__ V, int with_weights,
                            int* err) {
  int nb[kMaxNbrs], mult[kMaxNbrs];
  for (int64_t vv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; vv < n; vv += (int64_t)gridDim.x * blockDim.x) {
    int v = static_cast<int>(vv);
    int cnt = gather_ring(v, faces, vfptr, vf, nb, mult, err);
    if (cnt < 0) continue;
    int base = rowptr[v];
    double vsum = 0.0;
    for (int k = 0; k < cnt; ++k) {
      int w = nb[k];
      col[base + k] = w;
      len[base + k] = edge_length(xyz, v, w);
      if (!with_weights) continue;
      double s = 0.0;
      for (int q = vfptr[v]; q < vfptr[v + 1]; ++q) {
        int t = vf[q];
        int a = faces[3 * t], b = faces[3 * t + 1], c = faces[3 * t + 2];
        if (a == w || b == w || c == w) s = dadd(s, cot_opposite(xyz, a, b, c, v, w));
      }
      double aw = __ddiv_rn(s, 2.0);
      A[base + k] = aw;
      vsum = dadd(vsum, aw);
    }
    if (!with_weights) continue;
    V[v] = vsum;
    double mass = 0.0;
    for (int q = vfptr[v]; q < vfptr[v + 1]; ++q) {
      int t = vf[q];
      mass = dadd(mass, __ddiv_rn(triangle_area(xyz, faces[3 * t], faces[3 * t + 1], faces[3 * t + 2]), 3.0));
    }
    D[v] = mass;
  }
}

// ------------------------------------------------------- biharmonic ------

// Sorted union of {j} U N(j) over j in {i} U N(i).  Returns the count or -1 on overflow.
__device__ int gather_two_ring(int i, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int* keys,
                               int* err) {
  int cnt = 0;
  for (int a = rowptr[i] - 1; a < rowptr[i + 1]; ++a) {
    int j = (a < rowptr[i]) ? i : col[a];
    for (int b = rowptr[j] - 1; b < rowptr[j + 1]; ++b) {
      int k = (b < rowptr[j]) ? j : col[b];
      int lo = 0, hi = cnt;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
      }
      if (lo < cnt && keys[lo] == k) continue;
      if (cnt == kMaxTwoRing) {
        set_error(err, DERR_TWO_RING);
        return -1;
      }
      for (int r = cnt; r > lo; --r) keys[r] = keys[r - 1];
      keys[lo] = k;
      ++cnt;
    }
  }
  return cnt;
}

__global__ void k_bih_count(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            int32_t* __restrict__ cnt, int* err) {
  int keys[kMaxTwoRing];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int c = gather_two_ring(static_cast<int>(i), rowptr, col, keys, err);
    cnt[i] = c < 0 ? 0 : c;
  }
}

// L_jk of L = V - A: V_j on the diagonal, -A_jk off it (0 if k is not adjacent to j).
__device__ __forceinline__ double lap_entry(int j, int k, const int32_t* __restrict__ rowptr,
                                            const int32_t* __restrict__ col, const double* __restrict__ A,
                                            const double* __restrict__ V) {
  if (j == k) return V[j];
  int lo = rowptr[j], hi = rowptr[j + 1];
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (col[mid] < k) lo = mid + 1; else hi = mid;
  }
  return (lo < rowptr[j + 1] && col[lo] == k) ? -A[lo] : 0.0;
}

// Row i of M: M_ik = sum over j of (L_ji L_jk) / D_jj, j ascending over row i of L (the
// diagonal in its sorted place), so that M_ik and M_ki receive the same terms in the same order.
__global__ void k_bih_fill(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const double* __restrict__ A, const double* __restrict__ V, const double* __restrict__ D,
                           const int32_t* __restrict__ mrowptr, int32_t* __restrict__ mcol, double* __restrict__ mval,
                           int* err) {
  int keys[kMaxTwoRing];
  double acc[kMaxTwoRing];
  for (int64_t ii = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ii < n; ii += (int64_t)gridDim.x * blockDim.x) {
    int i = static_cast<int>(ii);
    int cnt = gather_two_ring(i, rowptr, col, keys, err);
    if (cnt < 0) continue;
    for (int q = 0; q < cnt; ++q) acc[q] = 0.0;
    // walk row i of L in ascending column order with the diagonal inserted
    int a = rowptr[i], ae = rowptr[i + 1];
    bool diag_done = false;
    while (a < ae || !diag_done) {
      int j;
      if (!diag_done && (a >= ae || col[a] > i)) {
        j = i;
        diag_done = true;
      } else {
        j = col[a++];
      }
      double Lji = lap_entry(j, i, rowptr, col, A, V);
      double Dj = D[j];
      int b = rowptr[j], be = rowptr[j + 1];
      bool jd = false;
      while (b < be || !jd) {
        int k;
        if (!jd && (b >= be || col[b] > j)) {
          k = j;
          jd = true;
        } else {
          k = col[b++];
        }
        double Ljk = (k == j) ? V[j] : -A[b - 1];
        int lo = 0, hi = cnt;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (keys[mid] < k) lo = mid + 1; else hi = mid;
        }
        acc[lo] = __dadd_rn(acc[lo], __ddiv_rn(__dmul_rn(Lji, Ljk), Dj));
      }
    }
    int base = mrowptr[i];
    for (int q = 0; q < cnt; ++q) {
      mcol[base + q] = keys[q];
      mval[base + q] = acc[q];
    }
  }
}

// A caller's graph (Sec. 2.2, generic graphs): rows ascending without repeats or self loops, every
// edge present in both directions with the same length, lengths finite and positive, at most
// kMaxNbrs neighbours.
__global__ void k_graph_check(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const double* __restrict__ length, int* err) {
  for (int64_t ii = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ii < n; ii += (int64_t)gridDim.x * blockDim.x) {
    const int i = static_cast<int>(ii);
    const int a = rowptr[i], e = rowptr[i + 1];
    if (e < a) {
      atomicExch(err, DERR_BAD_CSR);
      continue;
    }
    if (e - a > kMaxNbrs) atomicExch(err, DERR_VALENCE);
    for (int q = a; q < e; ++q) {
      const int j = col[q];
      if (j < 0 || j >= n || j == i || (q > a && col[q - 1] >= j)) {
        atomicExch(err, DERR_BAD_CSR);
        break;
      }
      if (length && !(length[q] > 0.0 && length[q] < INFINITY)) atomicExch(err, DERR_BAD_CSR);
      int lo = rowptr[j], hi = rowptr[j + 1];  // the reverse edge j -> i, by bisection in row j
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (col[mid] < i) lo = mid + 1; else hi = mid;
      }
      if (lo >= rowptr[j + 1] || col[lo] != i || (length && length[lo] != length[q])) atomicExch(err, DERR_BAD_CSR);
    }
  }
}

// D = I, A = the 0/1 adjacency, V = the degrees, edge lengths as given (or 1).
__global__ void k_graph_fill(int64_t n, const int32_t* __restrict__ rowptr, const double* __restrict__ length,
                             double* __restrict__ len, double* __restrict__ A, double* __restrict__ D,
                             double* __restrict__ V) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      len[q] = length ? length[q] : 1.0;
      if (A) A[q] = 1.0;
    }
    if (D) {
      D[i] = 1.0;
      V[i] = static_cast<double>(rowptr[i + 1] - rowptr[i]);
    }
  }
}

}  // namespace

DevMesh stage_mesh(Ctx& c, const sbha_mesh* m) {
  if (!m || m->n_vertices < 1 || m->n_faces < 1 || !m->xyz || !m->faces)
    SBHA_THROW(SBHA_EINVAL, "mesh must have vertices, faces and non-null arrays");
  if (m->n_vertices > INT32_MAX / 2 || m->n_faces > INT32_MAX / 8)
    SBHA_THROW(SBHA_EINVAL, "mesh too large for int32 indices");
  DevMesh d;
  d.n = m->n_vertices;
  d.f = m->n_faces;
  d.xyz = stage_in(c, m->xyz, static_cast<size_t>(3 * d.n));
  d.faces = stage_in(c, m->faces, static_cast<size_t>(3 * d.f));
  return d;
}

static DevGraph build_common(Ctx& c, const DevMesh& m, bool weights) {
  const int T = 128;
  int32_t* cnt = c.zeros<int32_t>(m.n);
  k_face_count<<<grid_for(m.f, T), T, 0, c.stream>>>(m.f, m.n, m.faces, cnt, c.d_err);
  c.launched("face_count");
  c.check_device("mesh");
  int32_t* vfptr = c.alloc<int32_t>(m.n + 1);
  int64_t corners = exclusive_scan(c, cnt, vfptr, m.n);
  int32_t* vf = c.alloc<int32_t>(corners);
  SBHA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * m.n, c.stream));
  k_face_fill<<<grid_for(m.f, T), T, 0, c.stream>>>(m.f, m.faces, vfptr, cnt, vf);
  c.launched("face_fill");
  k_face_sort<<<grid_for(m.n, T), T, 0, c.stream>>>(m.n, vfptr, vf, c.d_err);
  c.launched("face_sort");
  int32_t* deg = cnt;
  k_ring_count<<<grid_for(m.n, T), T, 0, c.stream>>>(m.n, m.faces, vfptr, vf, deg, c.d_err);
  c.launched("ring_count");
  c.check_device("mesh");
  DevGraph g;
  g.n = m.n;
  g.xyz = m.xyz;
  g.rowptr = c.alloc<int32_t>(m.n + 1);
  g.nnz = exclusive_scan(c, deg, g.rowptr, m.n);
  g.col = c.alloc<int32_t>(g.nnz);
  g.len = c.alloc<double>(g.nnz);
  if (weights) {
    g.A = c.alloc<double>(g.nnz);
    g.D = c.alloc<double>(m.n);
    g.V = c.alloc<double>(m.n);
  }
  k_ring_fill<<<grid_for(m.n, T), T, 0, c.stream>>>(m.n, m.xyz, m.faces, vfptr, vf, g.rowptr, g.col, g.len, g.A,
                                                    g.D, g.V, weights ? 1 : 0, c.d_err);
  c.launched("ring_fill");
  c.check_device("mesh");
  c.free(vf);
  c.free(vfptr);
  return g;
}

DevGraph build_graph(Ctx& c, const DevMesh& m) { return build_common(c, m, true); }

DevGraph build_graph_csr(Ctx& c, const sbha_graph* gr, bool weights) {
  if (!gr || gr->n_vertices < 1 || !gr->rowptr || !gr->col) SBHA_THROW(SBHA_EINVAL, "bad graph");
  const int64_t n = gr->n_vertices;
  int32_t nnz32 = 0;
  if (is_device_ptr(gr->rowptr)) {
    SBHA_CUDA(cudaMemcpyAsync(&nnz32, gr->rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
  } else {
    nnz32 = gr->rowptr[n];
  }
  if (nnz32 < 0) SBHA_THROW(SBHA_EINVAL, "graph rowptr[n] is negative");
  DevGraph g;
  g.n = n;
  g.nnz = nnz32;
  g.rowptr = const_cast<int32_t*>(stage_in(c, gr->rowptr, n + 1));
  g.col = const_cast<int32_t*>(stage_in(c, gr->col, std::max<int32_t>(nnz32, 1)));
  const double* length = gr->length ? stage_in(c, gr->length, std::max<int32_t>(nnz32, 1)) : nullptr;
  const int T = 128;
  k_graph_check<<<grid_for(n, T), T, 0, c.stream>>>(n, g.rowptr, g.col, length, c.d_err);
  c.launched("graph_check");
  c.check_device("graph");
  g.len = c.alloc<double>(std::max<int32_t>(nnz32, 1));
  if (weights) {
    g.A = c.alloc<double>(std::max<int32_t>(nnz32, 1));
    g.D = c.alloc<double>(n);
    g.V = c.alloc<double>(n);
  }
  k_graph_fill<<<grid_for(n, T), T, 0, c.stream>>>(n, g.rowptr, length, g.len, g.A, g.D, g.V);
  c.launched("graph_fill");
  return g;
}
DevGraph build_edge_lengths(Ctx& c, const DevMesh& m) { return build_common(c, m, false); }

DevCSR build_biharmonic(Ctx& c, const DevGraph& g) {
  const int T = 128;
  int32_t* cnt = c.alloc<int32_t>(g.n);
  k_bih_count<<<grid_for(g.n, T), T, 0, c.stream>>>(g.n, g.rowptr, g.col, cnt, c.d_err);
  c.launched("bih_count");
  c.check_device("biharmonic");
  DevCSR M;
  M.rows = M.cols = g.n;
  M.rowptr = c.alloc<int32_t>(g.n + 1);
  M.nnz = exclusive_scan(c, cnt, M.rowptr, g.n);
  M.col = c.alloc<int32_t>(M.nnz);
  M.val = c.alloc<double>(M.nnz);
  k_bih_fill<<<grid_for(g.n, T), T, 0, c.stream>>>(g.n, g.rowptr, g.col, g.A, g.V, g.D, M.rowptr, M.col, M.val,
                                                   c.d_err);
  c.launched("bih_fill");
  c.check_device("biharmonic");
  c.free(cnt);
  return M;
}

}  // namespace sbha
