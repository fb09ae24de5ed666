/*
 * Plain FP64 CPU oracle for sparse biharmonic MDS (Turek & Huth,
 * "Efficient, sparse representation of manifold distance matrices for
 * classical scaling", arXiv:1705.10887).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header or constant with the CUDA library.
 *
 * Every routine is the slow, obvious form of its definition:
 *   - cotangent adjacency, lumped mass, edge lengths: one loop over faces and a
 *     sort of the half-edges (Sec. 2.2, cotangent-weight and lumped-mass
 *     definitions);
 *   - geodesics: binary-heap Dijkstra on the mesh edges (Eq. 1, with
 *     mesh-edge shortest paths standing in for the surface geodesic);
 *   - farthest-point landmarks: one full Dijkstra per landmark and a linear
 *     argmax (Eq. 5);
 *   - biharmonic operator M = (V - A)^T D^{-1} (V - A): sparse triple product
 *     by rows (Sec. 2.2);
 *   - interpolation operator P_u = -M_uu^{-1} M_ub: reverse Cuthill-McKee
 *     ordering plus an envelope Cholesky factorisation, one forward/backward
 *     solve per landmark column (Eq. 3, Eq. 6; Sec. 3.2 names the sparse
 *     Cholesky route);
 *   - Gram matrix of J P and the column sums of P (Sec. 3.3);
 *   - cyclic Jacobi eigensolver for dense symmetric matrices.
 *
 * Floating point: compile with -ffp-contract=off.  Edge lengths are formed as
 * sqrt((dx*dx + dy*dy) + dz*dz) with dx = x_j - x_i, and path lengths are
 * left folds from the source, so that any exact shortest-path algorithm that
 * uses the same edge lengths reaches the same doubles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENOTSPD 3
#define ORC_ENOCONV 4

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ------------------------------------------------------------------------ */
/* Mesh operators: edge graph, edge lengths, cotangent weights, lumped mass  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t i, j;
  double cot; /* cotangent of the angle opposite edge (i, j) in one face */
} half_edge;

static int cmp_half_edge(const void* pa, const void* pb) {
  const half_edge* a = (const half_edge*)pa;
  const half_edge* b = (const half_edge*)pb;
  if (a->i != b->i) return a->i < b->i ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  /* equal keys: order by value so that the sum below does not depend on qsort */
  if (a->cot != b->cot) return a->cot < b->cot ? -1 : 1;
  return 0;
}

/* cot of the angle at vertex c in triangle (a, b, c): (e1 . e2) / |e1 x e2| */
static double cot_at(const double* xyz, int a, int b, int c) {
  double e1x = xyz[3 * a + 0] - xyz[3 * c + 0];
  double e1y = xyz[3 * a + 1] - xyz[3 * c + 1];
  double e1z = xyz[3 * a + 2] - xyz[3 * c + 2];
  double e2x = xyz[3 * b + 0] - xyz[3 * c + 0];
  double e2y = xyz[3 * b + 1] - xyz[3 * c + 1];
  double e2z = xyz[3 * b + 2] - xyz[3 * c + 2];
  double dot = e1x * e2x + e1y * e2y + e1z * e2z;
  double cx = e1y * e2z - e1z * e2y;
  double cy = e1z * e2x - e1x * e2z;
  double cz = e1x * e2y - e1y * e2x;
  return dot / sqrt(cx * cx + cy * cy + cz * cz);
}

static double edge_length(const double* xyz, int i, int j) {
  double dx = xyz[3 * j + 0] - xyz[3 * i + 0];
  double dy = xyz[3 * j + 1] - xyz[3 * i + 1];
  double dz = xyz[3 * j + 2] - xyz[3 * i + 2];
  double s = dx * dx;
  s = s + dy * dy;
  s = s + dz * dz;
  return sqrt(s);
}

/*
 * Builds the symmetric edge graph in CSR form (columns ascending) with, per
 * directed edge, its Euclidean length and the cotangent weight
 * A_ij = (cot alpha_ij + cot beta_ij) / 2 (one cotangent on a boundary edge),
 * and the lumped mass D_ii = (1/3) * sum of incident triangle areas.
 * Arrays col/len/A must hold 6*f entries.  Returns ORC_EINVAL for an
 * out-of-range or repeated vertex in a face, or an edge shared by more than
 * two faces.
 */
int orc_mesh_operators(int64_t n, int64_t f, const double* xyz, const int32_t* faces, int32_t* rowptr,
                       int32_t* col, double* len, double* A, double* D, int64_t* nnz_out) {
  half_edge* he = (half_edge*)malloc(sizeof(half_edge) * (size_t)(6 * f + 1));
  if (!he) return ORC_ENOMEM;
  for (int64_t v = 0; v < n; ++v) D[v] = 0.0;
  int64_t m = 0;
  for (int64_t t = 0; t < f; ++t) {
    int a = faces[3 * t + 0], b = faces[3 * t + 1], c = faces[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n || a == b || b == c || a == c) {
      free(he);
      return ORC_EINVAL;
    }
    /* edge (a,b) is opposite c, (b,c) opposite a, (c,a) opposite b */
    double cc = cot_at(xyz, a, b, c), ca = cot_at(xyz, b, c, a), cb = cot_at(xyz, c, a, b);
    he[m++] = (half_edge){a, b, cc};
    he[m++] = (half_edge){b, a, cc};
    he[m++] = (half_edge){b, c, ca};
    he[m++] = (half_edge){c, b, ca};
    he[m++] = (half_edge){c, a, cb};
    he[m++] = (half_edge){a, c, cb};
    double ux = xyz[3 * b + 0] - xyz[3 * a + 0], uy = xyz[3 * b + 1] - xyz[3 * a + 1], uz = xyz[3 * b + 2] - xyz[3 * a + 2];
    double wx = xyz[3 * c + 0] - xyz[3 * a + 0], wy = xyz[3 * c + 1] - xyz[3 * a + 1], wz = xyz[3 * c + 2] - xyz[3 * a + 2];
    double nx = uy * wz - uz * wy, ny = uz * wx - ux * wz, nz = ux * wy - uy * wx;
    double area = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
    D[a] += area / 3.0;
    D[b] += area / 3.0;
    D[c] += area / 3.0;
  }
  qsort(he, (size_t)m, sizeof(half_edge), cmp_half_edge);
  int64_t e = 0;
  for (int64_t v = 0; v <= n; ++v) rowptr[v] = 0;
  for (int64_t s = 0; s < m;) {
    int64_t t = s;
    double sum = 0.0;
    while (t < m && he[t].i == he[s].i && he[t].j == he[s].j) {
      sum += he[t].cot;
      ++t;
    }
    if (t - s > 2) {
      free(he);
      return ORC_EINVAL; /* non-manifold edge */
    }
    col[e] = he[s].j;
    len[e] = edge_length(xyz, he[s].i, he[s].j);
    A[e] = sum / 2.0;
    rowptr[he[s].i + 1]++;
    ++e;
    s = t;
  }
  for (int64_t v = 0; v < n; ++v) rowptr[v + 1] += rowptr[v];
  *nnz_out = e;
  free(he);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Dijkstra (binary heap, lazy deletion)                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  double d;
  int32_t v;
} heap_item;

static void heap_push(heap_item* h, int64_t* size, heap_item x) {
  int64_t i = (*size)++;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].d <= x.d) break;
    h[i] = h[p];
    i = p;
  }
  h[i] = x;
}

static heap_item heap_pop(heap_item* h, int64_t* size) {
  heap_item top = h[0];
  heap_item x = h[--(*size)];
  int64_t i = 0;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= *size) break;
    if (c + 1 < *size && h[c + 1].d < h[c].d) ++c;
    if (x.d <= h[c].d) break;
    h[i] = h[c];
    i = c;
  }
  if (*size > 0) h[i] = x;
  return top;
}

/* single-source shortest path lengths along mesh edges; dist[n] out (INFINITY if unreachable) */
static int dijkstra(int64_t n, const int32_t* rowptr, const int32_t* col, const double* len, int32_t src,
                    double* dist, heap_item* heap) {
  for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
  int64_t size = 0;
  dist[src] = 0.0;
  heap_push(heap, &size, (heap_item){0.0, src});
  while (size > 0) {
    heap_item it = heap_pop(heap, &size);
    if (it.d > dist[it.v]) continue; /* stale entry */
    for (int32_t e = rowptr[it.v]; e < rowptr[it.v + 1]; ++e) {
      int32_t w = col[e];
      double nd = it.d + len[e];
      if (nd < dist[w]) {
        dist[w] = nd;
        heap_push(heap, &size, (heap_item){nd, w});
      }
    }
  }
  return ORC_OK;
}

int orc_dijkstra(int64_t n, const int32_t* rowptr, const int32_t* col, const double* len, int32_t src, double* dist) {
  if (src < 0 || src >= n) return ORC_EINVAL;
  heap_item* heap = (heap_item*)malloc(sizeof(heap_item) * (size_t)(rowptr[n] + 1));
  if (!heap) return ORC_ENOMEM;
  dijkstra(n, rowptr, col, len, src, dist, heap);
  free(heap);
  return ORC_OK;
}

/*
 * Distances from each of s sources to each of t targets (row-major s x t).
 * tgt == NULL means all n vertices.  Sources run in parallel.
 */
int orc_geodesics(int64_t n, const int32_t* rowptr, const int32_t* col, const double* len, const int32_t* src,
                  int32_t s, const int32_t* tgt, int32_t t, double* out) {
  for (int32_t a = 0; a < s; ++a)
    if (src[a] < 0 || src[a] >= n) return ORC_EINVAL;
  if (tgt)
    for (int32_t b = 0; b < t; ++b)
      if (tgt[b] < 0 || tgt[b] >= n) return ORC_EINVAL;
  int status = ORC_OK;
#pragma omp parallel
  {
    double* dist = (double*)malloc(sizeof(double) * (size_t)n);
    heap_item* heap = (heap_item*)malloc(sizeof(heap_item) * (size_t)(rowptr[n] + 1));
    if (!dist || !heap) {
#pragma omp atomic write
      status = ORC_ENOMEM;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int32_t a = 0; a < s; ++a) {
        dijkstra(n, rowptr, col, len, src[a], dist, heap);
        if (tgt)
          for (int32_t b = 0; b < t; ++b) out[(int64_t)a * t + b] = dist[tgt[b]];
        else
          for (int64_t b = 0; b < n; ++b) out[(int64_t)a * n + b] = dist[b];
      }
    }
    free(dist);
    free(heap);
  }
  return status;
}

/*
 * Farthest-point landmarks (Eq. 5): b_1 = first; b_j maximises the minimum
 * distance to b_1..b_{j-1}; ties go to the lowest vertex index.  mind[n] holds
 * the final minimum distance to the chosen set.  Returns ORC_EINVAL if some
 * vertex cannot be reached from b_1 (disconnected mesh).
 */
int orc_fps(int64_t n, const int32_t* rowptr, const int32_t* col, const double* len, int32_t l, int32_t first,
            int32_t* idx, double* mind) {
  if (l < 1 || l > n || first < 0 || first >= n) return ORC_EINVAL;
  double* dist = (double*)malloc(sizeof(double) * (size_t)n);
  heap_item* heap = (heap_item*)malloc(sizeof(heap_item) * (size_t)(rowptr[n] + 1));
  if (!dist || !heap) {
    free(dist);
    free(heap);
    return ORC_ENOMEM;
  }
  for (int64_t v = 0; v < n; ++v) mind[v] = INFINITY;
  int32_t b = first;
  int status = ORC_OK;
  for (int32_t j = 0; j < l; ++j) {
    idx[j] = b;
    dijkstra(n, rowptr, col, len, b, dist, heap);
    for (int64_t v = 0; v < n; ++v)
      if (dist[v] < mind[v]) mind[v] = dist[v];
    if (j == 0)
      for (int64_t v = 0; v < n; ++v)
        if (isinf(dist[v])) status = ORC_EINVAL;
    if (status != ORC_OK) break;
    double best = -1.0;
    int32_t arg = -1;
    for (int64_t v = 0; v < n; ++v)
      if (mind[v] > best) {
        best = mind[v];
        arg = (int32_t)v;
      }
    b = arg;
  }
  free(dist);
  free(heap);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Biharmonic operator M = (V - A)^T D^{-1} (V - A)                           */
/* ------------------------------------------------------------------------ */

/* L = V - A as CSR with the diagonal included, columns ascending.  Lrowptr[n+1], Lcol/Lval[nnzA + n]. */
static void build_laplacian(int64_t n, const int32_t* rowptr, const int32_t* col, const double* A, int32_t* Lrowptr,
                            int32_t* Lcol, double* Lval) {
  int64_t e = 0;
  Lrowptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    double Vii = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) Vii += A[k];
    int placed = 0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (!placed && col[k] > i) {
        Lcol[e] = (int32_t)i;
        Lval[e++] = Vii;
        placed = 1;
      }
      Lcol[e] = col[k];
      Lval[e++] = -A[k];
    }
    if (!placed) {
      Lcol[e] = (int32_t)i;
      Lval[e++] = Vii;
    }
    Lrowptr[i + 1] = (int32_t)e;
  }
}

/* V_ii = sum_j A_ij (Sec. 2.2), summed left to right over the row's columns in ascending order */
int orc_weight_sums(int64_t n, const int32_t* rowptr, const double* A, double* V) {
  for (int64_t i = 0; i < n; ++i) {
    double v = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) v += A[k];
    V[i] = v;
  }
  return ORC_OK;
}

/* number of structural nonzeros of M (the 2-ring pattern) */
int orc_biharmonic_nnz(int64_t n, const int32_t* rowptr, const int32_t* col, int64_t* nnz_out) {
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!mark) return ORC_ENOMEM;
  for (int64_t v = 0; v < n; ++v) mark[v] = -1;
  int64_t total = 0;
  for (int64_t i = 0; i < n; ++i) {
    /* row i of L has columns {i} U N(i); row j of L has {j} U N(j) */
    int32_t ji_first = (int32_t)i;
    for (int32_t a = -1; a < rowptr[i + 1] - rowptr[i]; ++a) {
      int32_t j = a < 0 ? ji_first : col[rowptr[i] + a];
      if (mark[j] != (int32_t)i) {
        mark[j] = (int32_t)i;
        ++total;
      }
      for (int32_t b = rowptr[j]; b < rowptr[j + 1]; ++b) {
        int32_t k = col[b];
        if (mark[k] != (int32_t)i) {
          mark[k] = (int32_t)i;
          ++total;
        }
      }
    }
  }
  free(mark);
  *nnz_out = total;
  return ORC_OK;
}

/*
 * M_ik = sum_j (L^T)_ij D_jj^{-1} L_jk, with L = V - A (V_ii = sum_j A_ij).
 * Output CSR (Mrowptr[n+1], Mcol/Mval[nnz from orc_biharmonic_nnz]), columns ascending.
 */
int orc_biharmonic(int64_t n, const int32_t* rowptr, const int32_t* col, const double* A, const double* D,
                   int32_t* Mrowptr, int32_t* Mcol, double* Mval) {
  int64_t nnzA = rowptr[n];
  int32_t* Lrowptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t* Lcol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnzA + n));
  double* Lval = (double*)malloc(sizeof(double) * (size_t)(nnzA + n));
  double* acc = (double*)malloc(sizeof(double) * (size_t)n);
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!Lrowptr || !Lcol || !Lval || !acc || !mark || !list) {
    free(Lrowptr); free(Lcol); free(Lval); free(acc); free(mark); free(list);
    return ORC_ENOMEM;
  }
  build_laplacian(n, rowptr, col, A, Lrowptr, Lcol, Lval);
  for (int64_t v = 0; v < n; ++v) mark[v] = -1;
  int64_t e = 0;
  Mrowptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t cnt = 0;
    /* (L^T)_ij = L_ji; L is symmetric, so walk column i of L as row i */
    for (int32_t a = Lrowptr[i]; a < Lrowptr[i + 1]; ++a) {
      int32_t j = Lcol[a];
      double Lji = 0.0;
      for (int32_t q = Lrowptr[j]; q < Lrowptr[j + 1]; ++q)
        if (Lcol[q] == (int32_t)i) Lji = Lval[q];
      for (int32_t b = Lrowptr[j]; b < Lrowptr[j + 1]; ++b) {
        int32_t k = Lcol[b];
        if (mark[k] != (int32_t)i) {
          mark[k] = (int32_t)i;
          acc[k] = 0.0;
          list[cnt++] = k;
        }
        /* (L_ji * L_jk) / D_jj, summed over j ascending: M_ik and M_ki get the same terms in the same order */
        acc[k] += (Lji * Lval[b]) / D[j];
      }
    }
    /* emit in ascending column order (insertion sort of a short list) */
    for (int32_t p = 1; p < cnt; ++p) {
      int32_t key = list[p];
      int32_t q = p - 1;
      while (q >= 0 && list[q] > key) {
        list[q + 1] = list[q];
        --q;
      }
      list[q + 1] = key;
    }
    for (int32_t p = 0; p < cnt; ++p) {
      Mcol[e] = list[p];
      Mval[e++] = acc[list[p]];
    }
    Mrowptr[i + 1] = (int32_t)e;
  }
  free(Lrowptr); free(Lcol); free(Lval); free(acc); free(mark); free(list);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Interpolation operator: P_u = -M_uu^{-1} M_ub by envelope Cholesky        */
/* ------------------------------------------------------------------------ */

/* reverse Cuthill-McKee ordering of a symmetric pattern; perm[new] = old */
static void rcm_order(int64_t m, const int32_t* rp, const int32_t* ci, int32_t* perm) {
  int32_t* deg = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  char* seen = (char*)calloc((size_t)m, 1);
  int32_t* level = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int32_t* nb = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  for (int64_t v = 0; v < m; ++v) deg[v] = rp[v + 1] - rp[v];
  int64_t head = 0;
  for (;;) {
    /* start a new component at the unvisited vertex of least degree */
    int64_t start = -1;
    for (int64_t v = 0; v < m; ++v)
      if (!seen[v] && (start < 0 || deg[v] < deg[start])) start = v;
    if (start < 0) break;
    /* pseudo-peripheral refinement: BFS, move to a least-degree vertex of the last level */
    for (int it = 0; it < 4; ++it) {
      for (int64_t v = 0; v < m; ++v) level[v] = -1;
      int64_t qh = 0, qt = 0;
      nb[qt++] = (int32_t)start;
      level[start] = 0;
      int32_t maxlev = 0;
      while (qh < qt) {
        int32_t u = nb[qh++];
        for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
          int32_t w = ci[e];
          if (level[w] < 0 && !seen[w]) {
            level[w] = level[u] + 1;
            if (level[w] > maxlev) maxlev = level[w];
            nb[qt++] = w;
          }
        }
      }
      int64_t cand = start;
      for (int64_t q = 0; q < qt; ++q) {
        int32_t w = nb[q];
        if (level[w] == maxlev && (level[cand] != maxlev || deg[w] < deg[cand])) cand = w;
      }
      if (cand == start) break;
      start = cand;
    }
    /* Cuthill-McKee BFS: neighbours by increasing degree (then index) */
    int64_t qh = head;
    perm[head++] = (int32_t)start;
    seen[start] = 1;
    while (qh < head) {
      int32_t u = perm[qh++];
      int32_t cnt = 0;
      for (int32_t e = rp[u]; e < rp[u + 1]; ++e)
        if (!seen[ci[e]]) {
          nb[cnt++] = ci[e];
          seen[ci[e]] = 1;
        }
      for (int32_t p = 1; p < cnt; ++p) {
        int32_t key = nb[p];
        int32_t q = p - 1;
        while (q >= 0 && (deg[nb[q]] > deg[key] || (deg[nb[q]] == deg[key] && nb[q] > key))) {
          nb[q + 1] = nb[q];
          --q;
        }
        nb[q + 1] = key;
      }
      for (int32_t p = 0; p < cnt; ++p) perm[head++] = nb[p];
    }
  }
  /* reverse */
  for (int64_t a = 0, b = m - 1; a < b; ++a, --b) {
    int32_t t = perm[a];
    perm[a] = perm[b];
    perm[b] = t;
  }
  free(deg); free(seen); free(level); free(nb);
}

/*
 * Columns `cols[0..ncols)` (indices into idx) of the dense interpolation
 * operator P in vertex order: out[v*ncols + c] = P[v, cols[c]].  Landmark rows
 * are the identity block; unknown rows solve M_uu x = -M_ub e_j exactly
 * (envelope Cholesky of M_uu in RCM order).  idx[l] lists the landmark
 * vertices; landmark b = idx[j] is column j.
 */
/* Error-free transformations (Knuth's TwoSum, Dekker's split product; exact in IEEE double
   without fused multiply-add, which -ffp-contract=off rules out). */
static void two_sum(double a, double b, double* s, double* e) {
  double t = a + b;
  double bb = t - a;
  *e = (a - (t - bb)) + (b - bb);
  *s = t;
}
static void split27(double a, double* hi, double* lo) {
  double c = 134217729.0 * a; /* 2^27 + 1 */
  double h = c - (c - a);
  *hi = h;
  *lo = a - h;
}
static void two_prod(double a, double b, double* p, double* e) {
  double ah, al, bh, bl;
  double x = a * b;
  split27(a, &ah, &al);
  split27(b, &bh, &bl);
  *e = ((ah * bh - x) + ah * bl + al * bh) + al * bl;
  *p = x;
}
/* (sh, sl) -= (ph, pl) in double-double */
static void dd_sub(double* sh, double* sl, double ph, double pl) {
  double t, e;
  two_sum(*sh, -ph, &t, &e);
  e += *sl - pl;
  two_sum(t, e, sh, sl);
}

/* x <- (L L^T)^{-1} x with the envelope factor (rows a hold columns first[a]..a) */
static void envelope_solve(int64_t m, const double* Lf, const int64_t* start, const int32_t* first, double* y) {
  for (int64_t a = 0; a < m; ++a) { /* forward: L y = b */
    const double* ra = Lf + start[a] - first[a];
    double s = y[a];
    for (int64_t k = first[a]; k < a; ++k) s -= ra[k] * y[k];
    y[a] = s / ra[a];
  }
  for (int64_t a = m - 1; a >= 0; --a) { /* backward: L^T x = y (column sweep) */
    const double* ra = Lf + start[a] - first[a];
    y[a] = y[a] / ra[a];
    for (int64_t k = first[a]; k < a; ++k) y[k] -= ra[k] * y[a];
  }
}

enum { kRefinePasses = 2 };

int orc_interpolation(int64_t n, const int32_t* Mrowptr, const int32_t* Mcol, const double* Mval, const int32_t* idx,
                      int32_t l, const int32_t* cols, int32_t ncols, double* out) {
  if (l < 1 || l > n) return ORC_EINVAL;
  int32_t* lm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n); /* vertex -> landmark column or -1 */
  int32_t* un = (int32_t*)malloc(sizeof(int32_t) * (size_t)n); /* vertex -> unknown index or -1 */
  if (!lm || !un) { free(lm); free(un); return ORC_ENOMEM; }
  for (int64_t v = 0; v < n; ++v) lm[v] = -1;
  for (int32_t j = 0; j < l; ++j) {
    if (idx[j] < 0 || idx[j] >= n || lm[idx[j]] >= 0) { free(lm); free(un); return ORC_EINVAL; }
    lm[idx[j]] = j;
  }
  for (int32_t c = 0; c < ncols; ++c)
    if (cols[c] < 0 || cols[c] >= l) { free(lm); free(un); return ORC_EINVAL; }
  int64_t m = 0;
  for (int64_t v = 0; v < n; ++v) un[v] = lm[v] < 0 ? (int32_t)(m++) : -1;
  int32_t* uvert = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  for (int64_t v = 0; v < n; ++v)
    if (un[v] >= 0) uvert[un[v]] = (int32_t)v;
  /* landmark rows */
  for (int64_t v = 0; v < n; ++v)
    if (lm[v] >= 0)
      for (int32_t c = 0; c < ncols; ++c) out[v * ncols + c] = (cols[c] == lm[v]) ? 1.0 : 0.0;
  if (m == 0) { free(lm); free(un); free(uvert); return ORC_OK; }
  /* pattern of M_uu (unknown numbering) for the ordering */
  int32_t* rp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  int64_t cnt = 0;
  rp[0] = 0;
  for (int64_t u = 0; u < m; ++u) {
    int32_t v = uvert[u];
    for (int32_t e = Mrowptr[v]; e < Mrowptr[v + 1]; ++e)
      if (un[Mcol[e]] >= 0 && un[Mcol[e]] != (int32_t)u) ++cnt;
    rp[u + 1] = (int32_t)cnt;
  }
  int32_t* ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt + 1));
  cnt = 0;
  for (int64_t u = 0; u < m; ++u) {
    int32_t v = uvert[u];
    for (int32_t e = Mrowptr[v]; e < Mrowptr[v + 1]; ++e)
      if (un[Mcol[e]] >= 0 && un[Mcol[e]] != (int32_t)u) ci[cnt++] = un[Mcol[e]];
  }
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)m); /* new -> unknown */
  int32_t* iperm = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  rcm_order(m, rp, ci, perm);
  for (int64_t a = 0; a < m; ++a) iperm[perm[a]] = (int32_t)a;
  /* envelope: first[i] = smallest new column in row i (lower triangle) */
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
  int32_t* first = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  for (int64_t a = 0; a < m; ++a) {
    int32_t fmin = (int32_t)a;
    int32_t u = perm[a];
    for (int32_t e = rp[u]; e < rp[u + 1]; ++e)
      if (iperm[ci[e]] < fmin) fmin = iperm[ci[e]];
    first[a] = fmin;
  }
  start[0] = 0;
  for (int64_t a = 0; a < m; ++a) start[a + 1] = start[a] + (a - first[a] + 1);
  double* Lf = (double*)calloc((size_t)start[m], sizeof(double));
  if (!Lf) {
    free(lm); free(un); free(uvert); free(rp); free(ci); free(perm); free(iperm); free(start); free(first);
    return ORC_ENOMEM;
  }
  /* scatter M_uu's lower triangle into the envelope: row a holds columns first[a]..a */
  for (int64_t a = 0; a < m; ++a) {
    int32_t v = uvert[perm[a]];
    for (int32_t e = Mrowptr[v]; e < Mrowptr[v + 1]; ++e) {
      int32_t w = Mcol[e];
      if (un[w] < 0) continue;
      int32_t b = iperm[un[w]];
      if (b <= a) Lf[start[a] + (b - first[a])] = Mval[e];
    }
  }
  /* envelope Cholesky, row by row: L_ab = (M_ab - sum_k L_ak L_bk) / L_bb, L_aa = sqrt(M_aa - sum_k L_ak^2) */
  int status = ORC_OK;
  for (int64_t a = 0; a < m && status == ORC_OK; ++a) {
    double* ra = Lf + start[a] - first[a]; /* ra[b] = L_ab for first[a] <= b <= a */
    for (int64_t b = first[a]; b < a; ++b) {
      const double* rb = Lf + start[b] - first[b];
      int64_t k0 = first[a] > first[b] ? first[a] : first[b];
      double s = ra[b];
      for (int64_t k = k0; k < b; ++k) s -= ra[k] * rb[k];
      ra[b] = s / rb[b];
    }
    double s = ra[a];
    for (int64_t k = first[a]; k < a; ++k) s -= ra[k] * ra[k];
    if (!(s > 0.0)) status = ORC_ENOTSPD;
    else ra[a] = sqrt(s);
  }
  if (status == ORC_OK) {
#pragma omp parallel
    {
      double* y = (double*)malloc(sizeof(double) * (size_t)m);
      double* b = (double*)malloc(sizeof(double) * (size_t)m);
      double* r = (double*)malloc(sizeof(double) * (size_t)m);
#pragma omp for schedule(dynamic, 1)
      for (int32_t c = 0; c < ncols; ++c) {
        int32_t j = cols[c];
        int32_t bj = idx[j];
        /* right-hand side -M_ub e_j: column bj of M at the unknown rows.  The
           pattern is symmetric, so the rows w holding column bj are the columns of row bj. */
        for (int64_t a = 0; a < m; ++a) y[a] = 0.0;
        for (int32_t e = Mrowptr[bj]; e < Mrowptr[bj + 1]; ++e) {
          int32_t w = Mcol[e];
          if (un[w] < 0) continue;
          for (int32_t q = Mrowptr[w]; q < Mrowptr[w + 1]; ++q)
            if (Mcol[q] == bj) y[iperm[un[w]]] = -Mval[q];
        }
        for (int64_t a = 0; a < m; ++a) b[a] = y[a];
        envelope_solve(m, Lf, start, first, y);
        /* iterative refinement (Wilkinson): r = b - M_uu x in double-double, M_uu d = r with the
           same factor, x += d.  The forward error falls from about cond(M_uu) eps to about eps. */
        for (int pass = 0; pass < kRefinePasses; ++pass) {
          for (int64_t a = 0; a < m; ++a) {
            int32_t v = uvert[perm[a]];
            double sh = b[a], sl = 0.0;
            for (int32_t e = Mrowptr[v]; e < Mrowptr[v + 1]; ++e) {
              int32_t w = Mcol[e];
              if (un[w] < 0) continue;
              double ph, pl;
              two_prod(Mval[e], y[iperm[un[w]]], &ph, &pl);
              dd_sub(&sh, &sl, ph, pl);
            }
            r[a] = sh + sl;
          }
          envelope_solve(m, Lf, start, first, r);
          for (int64_t a = 0; a < m; ++a) y[a] += r[a];
        }
        for (int64_t a = 0; a < m; ++a) out[(int64_t)uvert[perm[a]] * ncols + c] = y[a];
      }
      free(y);
      free(b);
      free(r);
    }
  }
  free(lm); free(un); free(uvert); free(rp); free(ci); free(perm); free(iperm); free(start); free(first); free(Lf);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Classical scaling pieces                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Column sums c = P^T 1 and the centred Gram G = (J P)^T (J P) = P^T P - c c^T / n
 * (dense l x l, row-major) for P given in CSR (n rows, l columns).
 */
int orc_gram(int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col, const double* val, double* c, double* G) {
  for (int32_t j = 0; j < l; ++j) c[j] = 0.0;
  for (int64_t q = 0; q < (int64_t)l * l; ++q) G[q] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int32_t a = rowptr[i]; a < rowptr[i + 1]; ++a) {
      if (col[a] < 0 || col[a] >= l) return ORC_EINVAL;
      c[col[a]] += val[a];
      for (int32_t b = rowptr[i]; b < rowptr[i + 1]; ++b) G[(int64_t)col[a] * l + col[b]] += val[a] * val[b];
    }
  for (int32_t j = 0; j < l; ++j)
    for (int32_t k = 0; k < l; ++k) G[(int64_t)j * l + k] -= c[j] * c[k] / (double)n;
  return ORC_OK;
}

/*
 * Cyclic Jacobi eigensolver for a dense symmetric m x m matrix (row-major,
 * overwritten).  On return evals[m] holds the eigenvalues (unsorted, the final
 * diagonal) and V (row-major m x m) the eigenvectors as columns.  Each sweep
 * zeroes every off-diagonal pair (p, q) once with the rotation that
 * annihilates it; sweeps stop when the off-diagonal Frobenius norm is below
 * tol times the matrix norm.
 */
int orc_jacobi_eig(int32_t m, double* Amat, double* evals, double* V, int32_t max_sweeps, double tol) {
  for (int32_t i = 0; i < m; ++i)
    for (int32_t j = 0; j < m; ++j) V[(int64_t)i * m + j] = (i == j) ? 1.0 : 0.0;
  double total = 0.0;
  for (int64_t q = 0; q < (int64_t)m * m; ++q) total += Amat[q] * Amat[q];
  int status = ORC_ENOCONV;
  for (int32_t sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int32_t p = 0; p < m; ++p)
      for (int32_t q = p + 1; q < m; ++q) off += 2.0 * Amat[(int64_t)p * m + q] * Amat[(int64_t)p * m + q];
    if (off <= tol * tol * total) {
      status = ORC_OK;
      break;
    }
    for (int32_t p = 0; p < m - 1; ++p)
      for (int32_t q = p + 1; q < m; ++q) {
        double apq = Amat[(int64_t)p * m + q];
        if (apq == 0.0) continue;
        double app = Amat[(int64_t)p * m + p], aqq = Amat[(int64_t)q * m + q];
        /* tan of the rotation angle: root of t^2 + 2 theta t - 1 = 0 of smaller magnitude */
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0);
        double sn = t * cs;
        /* A <- R^T A R with R = [[c, s], [-s, c]] acting on (p, q) */
        for (int32_t k = 0; k < m; ++k) {
          double akp = Amat[(int64_t)k * m + p], akq = Amat[(int64_t)k * m + q];
          Amat[(int64_t)k * m + p] = cs * akp - sn * akq;
          Amat[(int64_t)k * m + q] = sn * akp + cs * akq;
        }
        for (int32_t k = 0; k < m; ++k) {
          double apk = Amat[(int64_t)p * m + k], aqk = Amat[(int64_t)q * m + k];
          Amat[(int64_t)p * m + k] = cs * apk - sn * aqk;
          Amat[(int64_t)q * m + k] = sn * apk + cs * aqk;
        }
        Amat[(int64_t)p * m + q] = 0.0;
        Amat[(int64_t)q * m + p] = 0.0;
        for (int32_t k = 0; k < m; ++k) {
          double vkp = V[(int64_t)k * m + p], vkq = V[(int64_t)k * m + q];
          V[(int64_t)k * m + p] = cs * vkp - sn * vkq;
          V[(int64_t)k * m + q] = sn * vkp + cs * vkq;
        }
      }
  }
  for (int32_t i = 0; i < m; ++i) evals[i] = Amat[(int64_t)i * m + i];
  return status;
}
