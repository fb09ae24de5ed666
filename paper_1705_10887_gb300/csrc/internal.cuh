// Cross-file interfaces of the sBHA CUDA library (not part of the C ABI).
#pragma once

#include <vector>

#include "common.cuh"

namespace sbha {

// Capacities of the per-vertex assembly kernels (checked; exceeding them is SBHA_EINVAL).
constexpr int kMaxFaces = 64;   // incident triangles per vertex
constexpr int kMaxNbrs = 64;    // 1-ring size
constexpr int kMaxTwoRing = 192;  // 2-ring size = nonzeros per row of the biharmonic operator

// Edge graph of a triangle mesh with the quantities of Sec. 2.2, all on the device.
struct DevGraph {
  int64_t n = 0, nnz = 0;
  int32_t* rowptr = nullptr;  // [n+1]
  int32_t* col = nullptr;     // [nnz] ascending per row
  double* len = nullptr;      // [nnz] Euclidean edge length, sqrt((dx*dx + dy*dy) + dz*dz)
  double* A = nullptr;        // [nnz] cotangent weight (cot a + cot b) / 2
  double* D = nullptr;        // [n] lumped mass: a third of the incident triangle areas
  double* V = nullptr;        // [n] row sums of A
  const double* xyz = nullptr;  // [n][3] vertex positions (the mesh's, not owned)
};

struct DevCSR {
  int64_t rows = 0, cols = 0, nnz = 0;
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
};

// Validated device copies of a caller mesh.
struct DevMesh {
  int64_t n = 0, f = 0;
  const double* xyz = nullptr;
  const int32_t* faces = nullptr;
};
DevMesh stage_mesh(Ctx& c, const sbha_mesh* m);

// Edge graph, edge lengths, cotangent weights, lumped mass (Sec. 2.2).
DevGraph build_graph(Ctx& c, const DevMesh& m);
// Biharmonic operator M = (V - A)^T D^{-1} (V - A) on the 2-ring pattern (Sec. 2.2).
DevCSR build_biharmonic(Ctx& c, const DevGraph& g);
// A caller's graph (Sec. 2.2, generic graphs: D = I, A = the 0/1 adjacency; edge lengths as given,
// or 1, for the geodesics), validated; no positions (xyz = nullptr).  weights = false: lengths only.
DevGraph build_graph_csr(Ctx& c, const sbha_graph* gr, bool weights);
// Only the edge lengths (for the geodesic entry points): same graph without A, D, V.
DevGraph build_edge_lengths(Ctx& c, const DevMesh& m);

// Farthest-point landmarks (Eq. 5).  idx [l] and mind [n] are device arrays.
void fps(Ctx& c, const DevGraph& g, int32_t l, int32_t first, int32_t* idx, double* mind);

// Farthest-point selection of several meshes in one launch: each job is one connected component
// of g (vertices [v0, v0 + n)), with its l, its first landmark (relative to v0), where its ids go
// in idx (relative to v0), and the base of its 32-vertex segments.
struct FpsJob {
  int32_t v0, n, l, first, idx_off, seg_base;
};
void fps_jobs(Ctx& c, const DevGraph& g, const std::vector<FpsJob>& jobs, int32_t* idx, double* mind);

// Single-source waves of several components in one launch per ~4 GB of work arrays: job src
// (a vertex of g) in component [v0, v0 + n); out[out_off + b] = d(src, tgt[tgt_off + b]), b < t.
struct SsspJob {
  int32_t src, v0, n, tgt_off, t;
  int64_t out_off, ws_off;
};
void sssp_jobs(Ctx& c, const DevGraph& g, const std::vector<SsspJob>& jobs, const int32_t* tgt, double* out);
// C = A B, row-major FP64 (M x K times K x N): on the FP64 pipes, or on the tensor cores by exact slicing
void dgemm_rowmajor(Ctx& c, int64_t M, int64_t N, int64_t K, const double* A, const double* B, double* C);
void dgemm_tc_rowmajor(Ctx& c, int64_t M, int64_t N, int64_t K, const double* A, const double* B, double* C);

// C = alpha op(A) B on the tensor cores by exact slicing (the engine of dgemm_tc_rowmajor), for a
// square operand op(A) = A or A.A (elementwise square), M x M row-major, that stays the same over many
// products with changing B (M x N row-major, N <= 64): op(A)'s digits are cut once.  The result is the
// FP64 product to a few units of 2^-48 of |op(A)| |B| per term; C is M x N row-major.
struct TcConstProduct {
  TcConstProduct(Ctx& c, int64_t M, const double* A, bool square, int64_t N);
  ~TcConstProduct();
  TcConstProduct(const TcConstProduct&) = delete;
  TcConstProduct& operator=(const TcConstProduct&) = delete;
  void times(const double* B, double alpha, double* C);

 private:
  struct Impl;
  Ctx& c;
  Impl* p;
};

// W = (D + D^T) / 2 with a zero diagonal (l x l)
void symmetrise(Ctx& c, const double* D, double* W, int32_t l);
// Shortest edge-path distances from src[s] to tgt[t] (tgt == nullptr: all vertices); D row-major.
void geodesics(Ctx& c, const DevGraph& g, const int32_t* src, int32_t s, const int32_t* tgt, int32_t t, double* D);
// W = symmetrised landmark distances (Sec. 3), [l x l].
void landmark_block(Ctx& c, const DevGraph& g, const int32_t* idx, int32_t l, double* W);

struct SolveReport {
  int32_t iterations = 0;
  int32_t refinements = 0;
  double max_rel_residual = 0.0;
  bool converged = true;
};

// Interpolation operator (Eq. 6) solved and thresholded (Eq. 8); writes the CSR of the
// n x l operator into rowptr/col/val (device arrays; col/val sized by operator_nnz).  dense_P
// (nullable, n x l row-major): also the operator before thresholding; rowptr = nullptr: only that.
SolveReport interpolation_operator(Ctx& c, const DevGraph& g, const DevCSR& M, const int32_t* idx, int32_t l,
                                   int32_t p_row, const sbha_opts& o, int32_t* rowptr, int32_t* col, double* val,
                                   double* dense_P = nullptr);

// Lower Cholesky factor of an SPD l x l row-major matrix (a new device array), and B (l x N row-major)
// <- (L L^T)^{-1} B with it.
double* cholesky(Ctx& c, int32_t l, const double* T);
void cholesky_solve(Ctx& c, int32_t l, const double* Lc, double* B, int64_t N);

// The FMDS interpolation matrix (Sec. 3.4.2) from the dense operator P (n x l row-major, landmark
// rows e_j) and the biharmonic operator M: H = P (M_bb + mu I + M_bu P_u)^{-1} mu, n x l row-major.
void fmds_interpolation(Ctx& c, const DevCSR& M, const int32_t* idx, int32_t l, const double* P, double mu,
                        const sbha_opts& o, double* H);
int64_t operator_nnz(int64_t n, int32_t l, int32_t p_row, int32_t mode);

struct MdsReport {
  int32_t iterations = 0;
  double residual = 0.0;
  bool converged = true;
};

// Block layout of C columns (C a multiple of 32): column q of row u at ((q / 32) n + u) 32 + q % 32.
// y = alpha A x for an n x n CSR matrix A (FP64) in that layout.
void csr_block_spmm(Ctx& c, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col, const double* val,
                    int C, const double* x, double* y, double alpha);
// y = A x in FP32 over nb column blocks (block layout), through the same tuned gather product as the
// FP32 block-CG solves: every row summed in CSR order from zero (fused multiply-adds), so it equals a
// plain CSR row loop.  Capturable when the matrix shape has been tuned, or with the default shape.
void csr_block_spmm_f32(Ctx& c, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                        const float* val, int nb, const float* x, float* y);
// X = A^{-1} B for an SPD n x n CSR matrix A that stores every diagonal entry, for the first ncols
// of the C columns of B (block layout): Jacobi-preconditioned block-CG with FP64 residual
// refinement (FP32 inner solves when o.precision is SBHA_PREC_FP32_REFINE) to o.cg_rtol.
struct SpdReport {
  int iterations = 0;
  double max_rel = 0.0;
  bool converged = true;
};
SpdReport spd_block_solve(Ctx& c, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                          const double* val, int C, int ncols, const double* B, double* X, const sbha_opts& o);

// Approximate geodesic distances by the heat method (Crane et al. 2013, the distances of the paper's
// experiments) from ns sources: D [ns x n] row-major, t = mfac h^2 with h the mean edge length.
SpdReport heat_geodesics(Ctx& c, const DevMesh& m, const DevGraph& g, const int32_t* src, int32_t ns, double mfac,
                         const sbha_opts& o, double* D, int32_t* jacobi_iterations);

// Sampled relative error of K~ = P W P^T (Sec. 4.1): acc[0] = sum over the ns rows of
// ||K~_s - K'_s||^2, acc[1] = sum of ||K'_s||^2 (K' = K_rows, or its square with squared != 0,
// W' likewise).  Every array on the device; acc [2].
void bha_error(Ctx& c, int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col, const double* val,
               const double* W, int32_t ns, const int32_t* rows, const double* K_rows, int squared, double* acc);

// Classical scaling (Sec. 3.3): through the landmark space, or by Lanczos on the n x n operator
// when o.eig_route is SBHA_EIG_LANCZOS (classical_scaling dispatches).
MdsReport classical_scaling_lanczos(Ctx& c, int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col,
                                    const double* val, const double* W, int32_t k, const sbha_opts& o, double* Z,
                                    double* evals);
MdsReport classical_scaling(Ctx& c, int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col,
                            const double* val, const double* W, int32_t k, const sbha_opts& o, double* Z,
                            double* evals);

// Polls a bounded device-side wait makes before it gives up (process-wide, sbha_set_wait_limit).
long long wait_limit();

}  // namespace sbha
