/*
 * sbha.h -- C ABI of the GB300 (sm_103a) implementation of sparse biharmonic
 * matrix approximation and sparse biharmonic multidimensional scaling
 * (sBHA / sBMDS; Turek & Huth, "Efficient, sparse representation of manifold
 * distance matrices for classical scaling", arXiv:1705.10887).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory.   Every array argument may live in host memory or in device memory of
 *           the current CUDA device; the library asks the CUDA runtime which
 *           (cudaPointerGetAttributes) and copies host arrays through `stream`.
 *           The caller allocates and owns every input and output.  The library
 *           owns only its internal workspace, which is allocated stream-ordered
 *           on `stream` and released before the call returns.
 * Layout.   Matrices are dense row-major unless stated.  Vertex positions are
 *           float64 [n x 3]; triangles are int32 [f x 3] (vertex ids 0..n-1).
 *           Sparse matrices are CSR: int32 rowptr[rows+1], int32 col[nnz]
 *           (ascending within a row), float64 val[nnz].
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *           synchronous with respect to the host: outputs are complete on return.
 * Errors.   Every call returns an sbha_status.  On failure outputs are
 *           unspecified (except SBHA_ENOCONV, see sbha_operator), nothing aborts,
 *           and sbha_last_error() describes the failure (per host thread).
 * Threads.  Calls from different host threads are safe when they use different
 *           streams, except sbha_mds_static (below).  Besides the per-thread error
 *           message and statistics the library keeps three pieces of process-wide
 *           state: the launch shapes its autotuner has picked (a table guarded by a
 *           mutex, filled on the first product with each matrix shape and reused by
 *           every later call), the fixed workspace of sbha_mds_static (one array per
 *           device, shared by every call: overlapping calls race, so the caller
 *           serialises them), and the iteration limit of bounded device waits
 *           (sbha_set_wait_limit).
 *
 * Citations give the paper's section, equation or algorithm that defines each
 * operation.
 */
#ifndef SBHA_H
#define SBHA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SBHA_OK = 0,
  SBHA_EINVAL = 1,         /* bad argument: sizes, ids, duplicate landmarks, non-manifold mesh */
  SBHA_EDISCONNECTED = 2,  /* some vertex cannot be reached along mesh edges */
  SBHA_ENOCONV = 3,        /* an iterative solver stopped at its iteration limit */
  SBHA_ENOMEM = 4,         /* device allocation failed */
  SBHA_ECUDA = 5,          /* a CUDA runtime call failed */
  SBHA_ETIMEOUT = 6,       /* a bounded device-side wait gave up */
  SBHA_ENOTIMPL = 7        /* option combination not provided by this build */
} sbha_status;

/* A triangle mesh: xyz float64 [n_vertices x 3], faces int32 [n_faces x 3]. */
typedef struct {
  int64_t n_vertices;
  int64_t n_faces;
  const double* xyz;
  const int32_t* faces;
} sbha_mesh;

/*
 * A generic graph (Sec. 2.2): the paper sets D = I and A = the graph's 0/1 adjacency, so the
 * biharmonic operator is M = (V - A)^2 with V the degrees.  Geodesics run along its edges with the
 * given lengths (NULL: every edge has length 1, hop counts).
 * rowptr int32 [n_vertices + 1], col int32 [nnz]: every row ascending, without repeats or self
 * loops, each edge listed in both directions (with equal lengths); at most 64 neighbours per
 * vertex and a 2-ring of at most 192.  length float64 [nnz], finite and positive, or NULL.
 * Host or device memory.  The graph is taken in the caller's vertex order (no positions: the
 * solver keeps that order for its unknowns).
 */
typedef struct {
  int64_t n_vertices;
  const int32_t* rowptr;
  const int32_t* col;
  const double* length;
} sbha_graph;

/* Precision of the interpolation solve (Sec. 3.2, Eq. 3). */
enum {
  SBHA_PREC_FP64 = 0,       /* FP64 conjugate gradients throughout */
  SBHA_PREC_FP32_REFINE = 1 /* FP32 inner conjugate gradients, FP64 residual refinement */
};

/* Preconditioner of the interpolation solve. */
enum {
  SBHA_PRECOND_JACOBI = 0, /* diagonal of M_uu */
  SBHA_PRECOND_MLP = 1     /* factored solver: the pinned-Laplacian solves after a pilot of
                              opts.mlp_pilot_cols columns (32 by default)
                              (solved with Jacobi to 1e-3) use M^{-1} = G^T G, G on the pattern of
                              L_uu with entries predicted by a small network trained on the GPU on
                              the pilot's (right-hand side, solution) pairs; Jacobi throughout if
                              training does not halve the loss, and from the first stalled inner
                              solve on */
};

/* How P_u = -M_uu^{-1} M_ub is computed (both give the same operator to cg_rtol). */
enum {
  SBHA_SOLVER_FACTORED = 0, /* through M = L D^{-1} L: two block-CG solves with the pinned cotangent
                               Laplacian L_uu plus dense landmark-space algebra, checked and
                               corrected on the FP64 residual of M_uu P_u + M_ub */
  SBHA_SOLVER_DIRECT = 1    /* block-CG on M_uu itself */
};

/* Kernel of the block-CG sparse products (same result up to rounding order). */
enum {
  SBHA_SPMM_AUTO = 0,   /* the library's choice: the tuner times the register gather's launch shapes
                           and, for FP32 products, the TMA gather, and keeps the fastest */
  SBHA_SPMM_GATHER = 1, /* warps gather their rows' neighbour rows from global memory into registers;
                           each CTA sweeps chunks of the locality-ordered rows spread over the grid */
  SBHA_SPMM_STAGED = 2, /* 128-row tiles stage their neighbours' rows in shared memory */
  SBHA_SPMM_PIPELINED = 3, /* the gather's mapping, with each warp's neighbour rows for the next 2 or 4
                             rows copied asynchronously (cp.async) into a shared-memory ring; only when
                             asked for (AUTO tunes the register gather's shape) */
  SBHA_SPMM_TMA = 4       /* FP32 products (opts.precision SBHA_PREC_FP32_REFINE): 64-row tiles whose
                             halo rows are brought into shared memory by TMA four-row gathers under a
                             producer warp, double-buffered, while sixteen warps compute; the FP64
                             products use the register gather.  Under AUTO it is one of the tuner's
                             candidates for the FP32 products */
};

/* Engine of the dense FP64 products: the landmark-space products of the factored solver (E^T D_u E
   and E Y, m x l x l each) and the eigen-subspace products of the landmark route (G Y and
   (W.W)(G Y), l x l x s per iteration). */
enum {
  SBHA_DENSE_AUTO = 0, /* the library's choice: tensor cores for the m x l x l products, and for the
                          eigen-subspace products from 4096 landmarks on */
  SBHA_DENSE_FP64 = 1, /* FP64 pipes */
  SBHA_DENSE_TC = 2    /* BF16 tensor cores on exact 8-bit slices of the FP64 operands, the exact partial
                          sums accumulated as 64-bit integers: the FP64 product to about K 2^-46 of
                          |A||B| per entry.  The eigen-subspace iteration moves to the FP64 pipes once its Ritz
                          residual is below 1e-9, so that FP64 products decide convergence. */
};

/* How the top-k eigenpairs of -1/2 J P (W.W) P^T J are found (Sec. 3.3; same pairs to the tolerances). */
enum {
  SBHA_EIG_LANDMARK = 0, /* in the landmark space: subspace iteration on the l x l product form */
  SBHA_EIG_LANCZOS = 1   /* sBMDS: thick-restart Lanczos with full reorthogonalisation on the n x n
                            operator, applied only through products with P, P^T and W.W (a basis of
                            at most 32 vectors of length n, no l x l Gram matrix) */
};

/* Thresholding rule that sparsifies the interpolation operator (Sec. 3.1, Eq. 8). */
enum {
  SBHA_SPARSIFY_ROWS = 0, /* keep min(p_row, l) largest |P_ij| in every non-landmark row */
  SBHA_SPARSIFY_COLS = 1  /* keep p = round((n-l) p_row / l) largest |P_ij| in every column */
};

typedef struct {
  int32_t precision;       /* SBHA_PREC_*; default SBHA_PREC_FP64 */
  int32_t precond;         /* SBHA_PRECOND_*; default SBHA_PRECOND_JACOBI */
  int32_t sparsify_mode;   /* SBHA_SPARSIFY_*; default SBHA_SPARSIFY_ROWS */
  int32_t chunk_cols;      /* right-hand sides solved together, 0 = automatic */
  double cg_rtol;          /* stop a column when ||r|| <= cg_rtol ||b||; default 1e-11 */
  int32_t cg_max_iter;     /* per solve (per refinement step in mixed precision); default 20000 */
  int32_t refine_max;      /* mixed precision: maximum FP64 refinement steps; default 12 */
  double inner_rtol;       /* mixed precision: FP32 inner reduction per step; default 1e-5 */
  int32_t oversample;      /* extra subspace vectors in the eigensolver; default 13 */
  int32_t eig_max_iter;    /* subspace iterations; default 300 */
  double eig_tol;          /* stop when every top-k Ritz pair (theta_i, x_i) has a residual
                              ||B x_i - theta_i x_i|| <= eig_tol theta_1 ||x_i||, B the operator of
                              the chosen route (sbha_mds); default 1e-12 */
  uint64_t seed;           /* starting block of the eigensolver; default 0x5eed */
  int32_t timing;          /* 1: per-stage times in sbha_stats (adds synchronisation);
                              2: also CUDA-event times of every conjugate-gradient kernel */
  int32_t solver;          /* SBHA_SOLVER_*; default SBHA_SOLVER_FACTORED */
  int32_t mlp_epochs;      /* SBHA_PRECOND_MLP: full-batch Adam epochs of the network; default 60 */
  int32_t spmm_variant;    /* SBHA_SPMM_*; default SBHA_SPMM_AUTO */
  int32_t dense_mode;      /* SBHA_DENSE_*; default SBHA_DENSE_AUTO */
  int32_t eig_route;       /* SBHA_EIG_*; default SBHA_EIG_LANDMARK.  SBHA_EIG_LANCZOS runs at most
                              max(32, eig_max_iter) operator products and needs k <= min(n, 32) - 10 */
  int32_t spmm_chunk_rows; /* launch shape of the gather products: 0 = autotuned per matrix shape (default),
                              16 / 32 / 64 = rows per chunk spread over the grid, -1 = one contiguous
                              range of rows per CTA (the same results either way) */
  int32_t fault_inject;    /* host-side fault injection for tests of the failure paths, 0 = none
                              (default).  SBHA_FAULT_MLP_NAN: the trained network's factor G is
                              overwritten with NaN before the first learned solve, which then stalls;
                              Jacobi must take over (sbha_stats.mlp_fallback) and the operator stays
                              correct.  Nothing is injected on the device. */
  int32_t mlp_pilot_cols;  /* SBHA_PRECOND_MLP: columns of the Jacobi pilot the network trains on, in
                              [1, 512] and at most the first chunk; 0 = 32 (default) */
  int32_t spmm_pipeline_depth; /* rows in flight per warp of the pipelined gather: 0 = autotuned (default),
                                  2 or 4 */
  int32_t cg_graph;        /* 1 (default): after its first batch of 8 iterations, each block-CG solve runs
                              to convergence as one CUDA graph whose WHILE node is decided on the device
                              (two iterations per pass, then a kernel sets the condition from the count of
                              active columns), with no host round trip per batch; 0: batches of 8
                              iterations checked by the host.  Same results either way. */
  int32_t reserved;
} sbha_opts;

/* Values of sbha_opts.fault_inject. */
enum {
  SBHA_FAULT_NONE = 0,
  SBHA_FAULT_MLP_NAN = 1
};

/* Fills `opts` with the defaults listed above. */
void sbha_opts_default(sbha_opts* opts);

/* Diagnostics of the last call made by this host thread. */
typedef struct {
  int32_t cg_iterations;      /* block-CG iterations executed: per chunk the largest count over its columns,
                                 summed over chunks, refinement steps and solves */
  int32_t refinements;        /* FP64 refinement steps taken (mixed precision) */
  double cg_max_rel_residual; /* max over columns of ||b - M_uu x|| / ||b|| in FP64 at exit */
  int32_t eig_iterations;     /* subspace iterations */
  double eig_residual;        /* max relative Ritz residual of the returned eigenpairs */
  int64_t kernel_launches;    /* kernels this library launched during the call */
  double ms_landmarks, ms_geodesics, ms_assembly, ms_solve, ms_sparsify, ms_mds; /* when opts.timing */
  /* Conjugate-gradient kernels, when opts.timing == 2 (CUDA events around every launch, on the
   * launching stream): index 0 = M_uu times the direction block, 1 = x/r update, 2 = direction
   * update, 3 = FP64 residual product.  Bytes are algorithmic: every operand read or written
   * once per launch (matrix, plus m x 32 values per active column block per vector). */
  int64_t cg_kernel_launches[4];
  double cg_kernel_ms[4];
  double cg_kernel_bytes[4];
  int64_t unknowns;           /* n - l */
  int64_t nnz_uu;             /* nonzeros of the matrix the block-CG multiplies (L_uu or M_uu) */
  int32_t chunk_cols;         /* right-hand sides solved together */
  int32_t inner_bytes;        /* 4 (FP32 inner solve) or 8 (FP64) */
  /* Learned preconditioner (SBHA_PRECOND_MLP, factored solver) */
  int32_t mlp_trained;          /* 1 if the network halved its loss and preconditions the later solves */
  int32_t mlp_fallback;         /* 1 if a preconditioned inner solve stalled and Jacobi took over */
  int32_t mlp_train_columns;    /* pilot columns solved with Jacobi and trained on */
  int32_t e_iterations_jacobi;  /* block-CG iterations of the first harmonic-extension solve (Jacobi):
                                   the pilot (to 1e-3) with SBHA_PRECOND_MLP, the first chunk otherwise */
  int32_t e_iterations_learned; /* largest block-CG iteration count of a learned-preconditioned
                                   harmonic-extension chunk (0 if none) */
  int32_t heat_sweeps;        /* sbha_heat_geodesics: Jacobi sweeps of the heat step (largest chunk) */
  int64_t mlp_train_entries;    /* entries of G that training touched */
  double mlp_loss_first, mlp_loss_last; /* training loss at the Jacobi start and after training */
  double mlp_ms_pilot;          /* host wall time of the pilot solve */
  double mlp_ms_train;          /* host wall time of building and training the network */
  /* Shared-memory staged products of the block-CG matrix (rows in tiles of 128 along a Morton curve) */
  int32_t spmm_tiles;           /* row tiles */
  int32_t spmm_tiles_staged;    /* tiles whose halo (rows they reference) fits the shared-memory stage */
  int64_t spmm_halo_rows;       /* total halo rows of the staged tiles */
  /* Factored solver: block-CG iterations by phase (summed over chunks) */
  int32_t e_iterations;         /* E = L_uu^{-1} A_ub (pilot included) */
  int32_t k_iterations;         /* L_uu^{-1} (D_u E Y) */
  int32_t correction_iterations; /* the two solves of every correction of the biharmonic residual */
  int32_t corrections;          /* correction rounds, summed over chunks */
  /* launch shape of the sparse products, picked per matrix shape by timing on first use: rows per
     chunk spread over the grid (0: one contiguous range per CTA), and its time per product; for the
     FP32 inner products when the call has them, else the FP64 ones */
  int32_t spmm_chunk_rows;
  int32_t spmm_tuned_shapes;    /* matrix shapes tuned so far in this process */
  double spmm_tuned_us;
  int32_t spmm_pipeline_depth;  /* rows in flight per warp of the picked product (0: register gather) */
  int32_t spmm_ctas_per_sm;     /* register gather: resident CTAs per SM it was built for (4: eight
                                   neighbour loads in flight per row; 6 or 8: four, fewer registers) */
  /* Scaling step, landmark route, with opts.timing >= 1 (CUDA events on the call's stream): the
     sorted transpose of P with c = P^T 1, and the centred Gram G = P^T P - c c^T / n (Sec. 3.3) */
  double ms_transpose;
  double ms_gram;
  int64_t p_nnz;                /* nonzeros of P the Gram read */
  /* TMA gather product of the FP32 inner solves (SBHA_SPMM_TMA, or picked by the tuner under AUTO):
     rows in tiles of 64 along the Morton curve, each tile's halo gathered four rows at a time */
  int32_t spmm_tma;                /* 1: the picked FP32 product is the TMA gather */
  int32_t spmm_gather_tiles_staged; /* its tiles whose halo (at most 192 rows) fits the stage */
  int64_t spmm_gather_halo_rows;   /* total halo rows of those tiles (before the padding to fours) */
} sbha_stats;

/* Copies the statistics of this thread's last call into *out. */
int sbha_last_stats(sbha_stats* out);

/* Message describing this thread's last failure ("" if none).  Valid until the next call. */
const char* sbha_last_error(void);

/* Library version string. */
const char* sbha_version(void);

/*
 * Farthest-point landmarks (Sec. 3, Eq. 5).
 *   b_1 = first; b_j = argmax_i min_{t<j} d(b_t, i), where d is the shortest-path
 *   length along mesh edges with Euclidean edge lengths (the geodesic distance of
 *   Eq. 1 on the edge graph).  Ties go to the lowest vertex index.
 * idx_out  int32 [l]   chosen vertex ids, in selection order.
 * mind_out float64 [n] final min distance of every vertex to the set (may be NULL).
 * Errors: SBHA_EINVAL for l < 1, l > n, first out of range, bad faces;
 *         SBHA_EDISCONNECTED if some vertex is unreachable from `first`.
 * Distances are exact: the same doubles as a Dijkstra that adds edge lengths
 * sqrt((dx*dx + dy*dy) + dz*dz) left to right along the path.
 */
int sbha_landmarks(const sbha_mesh* mesh, int32_t l, int32_t first, int32_t* idx_out, double* mind_out,
                   void* stream);

/*
 * Geodesic distances along mesh edges (Eq. 1) from s sources to t targets.
 * src int32 [s]; tgt int32 [t] or NULL for all n vertices (t is then ignored);
 * D_out float64 [s x (t or n)] row-major: D_out[a][b] = d(src[a], tgt[b]).
 * Unreachable targets get +infinity.  Errors: SBHA_EINVAL for ids out of range.
 */
int sbha_geodesics(const sbha_mesh* mesh, const int32_t* src, int32_t s, const int32_t* tgt, int32_t t,
                   double* D_out, void* stream);

/*
 * Landmark block W (Sec. 3): W_ij = d(b_i, b_j), symmetrised as (D_ij + D_ji)/2
 * with a zero diagonal.  idx int32 [l]; W_out float64 [l x l].
 */
int sbha_landmark_distances(const sbha_mesh* mesh, const int32_t* idx, int32_t l, double* W_out, void* stream);

/*
 * The mesh quantities of Sec. 2.2 exactly as the operator uses them, for inspection and checking.
 *   Edge graph: row v lists v's mesh neighbours in ascending order; len = Euclidean edge length
 *   sqrt((dx*dx + dy*dy) + dz*dz); A = cotangent weight (cot alpha + cot beta) / 2 (one cotangent
 *   on a boundary edge); D = lumped mass, a third of the incident triangle areas summed over the
 *   triangles in vertex-face order; V = row sums of A, summed left to right in column order.
 * rowptr int32 [n+1]; col int32 [cap]; len, A float64 [cap]; D, V float64 [n].  Size query:
 * col == NULL; *nnz_out receives the number of directed edges and nothing else is written.
 * Host or device memory.  Errors: SBHA_EINVAL (bad faces, non-manifold edge, valence above 64,
 * a vertex in no triangle, cap too small).
 */
int sbha_mesh_graph(const sbha_mesh* mesh, int32_t* rowptr, int32_t* col, double* len, double* A, double* D,
                    double* V, int64_t cap, int64_t* nnz_out, void* stream);

/*
 * The biharmonic operator M = (V - A)^T D^{-1} (V - A) of Sec. 2.2 (the matrix of Eq. 2 and 3)
 * as the operator uses it: CSR over the 2-ring pattern, columns ascending, entry
 * M_ik = sum over j ascending of (L_ji L_jk) / D_jj with L = V - A.
 * rowptr int32 [n+1]; col int32 [cap]; val float64 [cap].  Size query: col == NULL.
 * Host or device memory.  Errors: as sbha_mesh_graph, plus a 2-ring above 192 vertices.
 */
int sbha_biharmonic(const sbha_mesh* mesh, int32_t* rowptr, int32_t* col, double* val, int64_t cap,
                    int64_t* nnz_out, void* stream);

/*
 * Sparse interpolation operator P_sparse (Sec. 2.1 Eq. 3, Sec. 3 Eq. 6, Sec. 3.1 Eq. 8).
 *   M = (V - A)^T D^{-1} (V - A) with cotangent weights A, V = diag(row sums of A)
 *   and lumped mass D (Sec. 2.2); P_u = -M_uu^{-1} M_ub is solved column by column
 *   with preconditioned conjugate gradients, then thresholded by opts->sparsify_mode.
 * Output: CSR of the n x l operator in vertex order.  Landmark row idx[j] is exactly
 *   e_j (one entry 1.0 in column j).  rowptr int32 [n+1]; col int32 [cap];
 *   val float64 [cap].  In row mode nnz = l + (n - l) * min(p_row, l).
 *   Size query: pass col == NULL and val == NULL; *nnz_out receives the exact nnz
 *   (row mode) or an upper bound (column mode) and nothing else is computed.
 * idx int32 [l] landmark vertex ids (distinct).  p_row in [1, 128].
 * Errors: SBHA_EINVAL (bad ids, duplicates, p_row, cap too small, bad faces),
 *         SBHA_ENOCONV (outputs written; some column did not reach cg_rtol).
 */
int sbha_operator(const sbha_mesh* mesh, const int32_t* idx, int32_t l, int32_t p_row, const sbha_opts* opts,
                  int32_t* rowptr, int32_t* col, double* val, int64_t cap, int64_t* nnz_out, void* stream);

/*
 * Low-rank classical scaling with the sparse approximation (Sec. 3.3):
 * the top-k eigenpairs of -1/2 J P (W.W) P^T J, computed in the landmark space.
 *   c = P^T 1, G = (J P)^T (J P) = P^T P - c c^T / n (FP64 centring),
 *   theta, y: -1/2 (W.W) G y = theta y with y^T G y = 1 (subspace iteration with
 *   FP64 Rayleigh-Ritz, stopped on the Ritz residual of the top-k pairs, opts->eig_tol),
 *   Z = J P [y_1..y_k] diag(sqrt(max(theta, 0))).
 *   The squared landmark distances W.W are interpolated (the squared distances E
 *   of Eq. 4).  Each column of Z is signed so that its largest-magnitude entry is
 *   positive.
 * P: CSR n x l (rowptr [n+1], col, val); W float64 [l x l] symmetric;
 * Z_out float64 [n x k]; evals_out float64 [k] (decreasing).
 * With opts->eig_route = SBHA_EIG_LANCZOS the same pairs come from Lanczos on the n x n
 * operator itself (the paper's sBMDS): w = -1/2 J P ((W.W) (P^T (J q))), with J applied as
 * P^T J q = P^T q - mean(q) c and J (P s) = P s - (c.s / n) 1; Z = Q S_k diag(sqrt(theta)).
 * Errors: SBHA_EINVAL (k < 1, k + oversample > l with the landmark route, k > min(n, 32) - 10
 * with Lanczos, bad CSR), SBHA_ENOCONV.
 */
int sbha_mds(int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col, const double* val, const double* W,
             int32_t k, const sbha_opts* opts, double* Z_out, double* evals_out, void* stream);

/*
 * Sampled relative error of the approximation K~ = P W P^T (Eq. 9), as Sec. 4.1 measures it:
 * eps = ||K~ - K||_F^2 / ||K||_F^2, estimated on a subset of rows when K is too large to hold.
 * For the ns sampled rows S (K_rows[i] = the exact row rows[i] of K),
 *   num = sum_{s in S} sum_v (K~_sv - K_sv)^2,   den = sum_{s in S} sum_v K_sv^2,
 * so eps ~= num / den, exactly when S holds every row.  squared != 0 compares K (.) K with
 * P (W (.) W) P^T, the squared distances that classical scaling factors.  FP64 throughout.
 * P: CSR n x l (rowptr [n+1], col, val); W float64 [l x l]; rows int32 [ns]; K_rows float64
 * [ns x n] row-major (e.g. rows of sbha_geodesics); num_out, den_out float64 [1].  Arrays may be
 * host or device memory.
 * Errors: SBHA_EINVAL (n < 1, l < 1, ns < 0, a missing array, a column outside [0, l), a sampled
 * row outside [0, n)).
 */
int sbha_bha_error(int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col, const double* val,
                   const double* W, int32_t ns, const int32_t* rows, const double* K_rows, int32_t squared,
                   double* num_out, double* den_out, void* stream);

/*
 * The FMDS interpolation matrix derived from the biharmonic operator (Sec. 3.4.2):
 *   H = P (M_bb + mu I + M_bu P_u)^{-1} mu,
 * with P the dense operator of Eq. 6 (solved as sbha_operator solves it, before any thresholding) and
 * M the biharmonic operator.  Unlike P, H lets the landmark values deviate, by an amount mu controls
 * (the paper's experiments take mu = 50); its rows sum to one, and H -> P as mu grows.  The l x l
 * matrix is factored by Cholesky and H = P (mu S^{-1}) is formed on the landmark-space product
 * engine (opts->dense_mode).
 * idx int32 [l] landmark vertex ids; H_out float64 [n x l] row-major, host or device.
 * Errors: SBHA_EINVAL (bad mesh, l outside [1, n], mu not finite and positive, bad landmarks),
 * SBHA_ENOCONV (the solve did not reach opts->cg_rtol; H is still written).
 */
int sbha_fmds_operator(const sbha_mesh* mesh, const int32_t* idx, int32_t l, double mu, const sbha_opts* opts,
                       double* H_out, void* stream);

/*
 * Approximate geodesic distances by the heat method (Crane et al. 2013), the distance source of the
 * paper's experiments (Sec. 4), from ns sources:
 *   1. u = (D + t L)^{-1} delta_s with t = m h^2, h the mean edge length (L = V - A, D as in Sec. 2.2);
 *   2. X = -grad u / |grad u| on every triangle;
 *   3. the integrated divergence of X at every vertex (cotangent formula);
 *   4. L phi = -div X, and D_out[s][v] = phi(v) - phi(s).
 * Step 1 runs Jacobi's iteration on D + t L in FP64 (damped by 2 / (2 + gamma) when obtuse triangles
 * push the Gershgorin radius gamma of its Jacobi-scaled form to 1 or more; with positive cotangent
 * weights every term of the series is non-negative and the far field keeps full relative precision)
 * until no entry changes by more than 1e-15 relatively; step 4 is block-CG to opts->cg_rtol (FP32
 * inner solves with opts->precision = SBHA_PREC_FP32_REFINE).  u decays geometrically with the edge
 * distance from s; where it falls below the FP64 range (about 300 decades, meshes several hundred
 * edges across at m = 1), raise m.
 * src int32 [ns] vertex ids; m > 0 (m <= 0: 1); D_out float64 [ns x n] row-major, host or device.
 * Errors: SBHA_EINVAL (bad mesh, ns < 1, a source out of range), SBHA_ENOCONV (the heat sweeps
 * diverged or ran past 200,000, or the Poisson solve did not converge).
 */
int sbha_heat_geodesics(const sbha_mesh* mesh, const int32_t* src, int32_t ns, double m, const sbha_opts* opts,
                        double* D_out, void* stream);

/* Parameters of the preconditioner network: W1[64][6], b1[64], W2[64][64], b2[64], w3[64], b3. */
#define SBHA_MLP_PARAMS 4673
#define SBHA_MLP_FEATURES 6

/*
 * Loss and gradient of the preconditioner network on plain regression, exposed so that its
 * forward and backward kernels can be checked on their own.  The network is
 * y(x) = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3 with its parameters rounded to BF16 and FP32
 * arithmetic; loss = mean over the N samples of (y(x_s) - t_s)^2.
 * X float32 [N x 6]; T float32 [N]; params float32 [SBHA_MLP_PARAMS] (the FP32 master copy);
 * grad_out float32 [SBHA_MLP_PARAMS] = d loss / d params (with respect to the BF16-rounded
 * values); loss_out float64 [1].  Arrays may be host or device memory.
 * Errors: SBHA_EINVAL (N < 0, missing array).
 * The paper has no counterpart (the learned preconditioner is an addition to its solver).
 */
int sbha_mlp_gradient(int64_t N, const float* X, const float* T, const float* params, float* grad_out,
                      double* loss_out, void* stream);

/*
 * Training loss of the learned preconditioner and its gradient, as evaluated in every epoch
 * inside sbha_operator (SBHA_PRECOND_MLP).  For an SPD matrix A (m x m CSR with sorted
 * columns, a symmetric pattern and a positive diagonal: the pinned Laplacian L_uu inside the
 * library) the preconditioner is M^{-1} = G^T G, G on A's pattern with
 *   G_ij = (delta_ij + y(f_ij)) / sqrt(A_ii),
 *   f_ij = [i == j, -A_ij / A_ii, -A_ij / A_jj, leak_i, leak_j, nnz(row i) / 7]  (FP32),
 *   leak_i = (A_ii - sum_{k != i} |A_ik|) / A_ii,
 * and y the network of sbha_mlp_gradient.  For pairs of right-hand sides b_c and solutions
 * x_c of A x_c = b_c (c = 1..ncols), the error of one preconditioned step in the A^2 norm,
 *   loss = sum_c ||A (G^T G b_c - x_c)||^2 / (ncols ||b_c||^2)   (columns with b_c = 0 count 0).
 * rowptr int32 [m+1], col int32 [nnz], val float64 [nnz]; B, X float64 [m x ncols] row-major
 * (X may be NULL: A x_c = b_c is then taken as exact, and A x_c is replaced by b_c);
 * params float32 [SBHA_MLP_PARAMS]; grad_out float32 [SBHA_MLP_PARAMS] = d loss / d params
 * (FP32 arithmetic on an FP32 copy of A and B); loss_out float64 [1].  Arrays may be host or
 * device memory.
 * Errors: SBHA_EINVAL (m < 1, ncols outside [1, 512], missing array, malformed CSR: column out
 * of range, unsorted row, missing diagonal or transposed entry, a diagonal entry <= 0).
 * The paper has no counterpart.
 */
int sbha_precond_gradient(int64_t m, const int32_t* rowptr, const int32_t* col, const double* val, int32_t ncols,
                          const double* B, const double* X, const float* params, float* grad_out, double* loss_out,
                          void* stream);

/*
 * C = A B for row-major FP64 A [M x K], B [K x N], C [M x N], by the engine the operator uses
 * for its landmark-space products (mode SBHA_DENSE_TC or SBHA_DENSE_FP64; AUTO = TC), exposed
 * so that it can be checked on its own.  With TC every row of A and column of B is scaled by a
 * power of two and cut into six signed 8-bit digits; the tensor cores multiply digit planes in
 * BF16 with FP32 sums that stay exact integers, and the partial sums are combined in FP64.
 * Arrays may be host or device memory.  Errors: SBHA_EINVAL (M, N, K < 1, missing array,
 * unknown mode), SBHA_ETIMEOUT (a bounded wait for the tensor cores gave up).
 * The paper has no counterpart.
 */
int sbha_dgemm(int64_t M, int64_t N, int64_t K, const double* A, const double* B, double* C, int32_t mode,
               void* stream);

/*
 * Iteration limit of the bounded device-side waits (the tensor-core kernels' waits for their
 * matrix products).  A wait that reaches the limit gives up, the kernel waits (with the default
 * limit) for the work it has in flight, frees its tensor memory and returns, and the call reports
 * SBHA_ETIMEOUT.  spins < 0 restores the default (2^22 polls); 0 makes every such wait give up
 * at once, which tests of the timeout path use.  Process-wide; returns the previous limit.
 * The paper has no counterpart.
 */
int64_t sbha_set_wait_limit(int64_t spins);

/*
 * Allocation-free variant of sbha_mds.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory while they run the
 * scaling step -- for example a host application that reserves all device memory up
 * front in its own pool and forbids allocator calls afterwards, or a latency-bound
 * loop in which an allocation could stall or fail part-way through a pipeline.
 * It computes exactly what sbha_mds computes, with the same arguments and results,
 * under these rules:
 *   - every array (rowptr, col, val, W, Z_out, evals_out) must be device memory of the
 *     current device (host arrays are rejected with SBHA_EINVAL, since copying them
 *     would need a device buffer);
 *   - l <= 1024 (larger l returns SBHA_EINVAL with a message; use sbha_mds);
 *   - the landmark-space route only (opts->eig_route = SBHA_EIG_LANCZOS returns SBHA_EINVAL);
 *   - its workspace is one fixed device array of about 10.3 MB, defined in the
 *     library, that every GPU loading the library holds until the process exits;
 *     no cudaMalloc, cudaFree or other allocating call is made;
 *   - the first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call on each device
 *     before any stream capture begins;
 *   - all calls share the array: the parts that must start at zero are cleared on
 *     every call, and calls that overlap on the GPU (other streams, other threads)
 *     race on it and must be serialised by the caller.
 */
int sbha_mds_static(int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col, const double* val,
                    const double* W, int32_t k, const sbha_opts* opts, double* Z_out, double* evals_out,
                    void* stream);

/*
 * The whole sBMDS pipeline in one call: farthest-point landmarks from `first`,
 * landmark block W, sparse operator P, scaling.  Z_out float64 [n x k];
 * evals_out float64 [k]; idx_out int32 [l] (may be NULL).
 */
int sbha_embed(const sbha_mesh* mesh, int32_t l, int32_t first, int32_t p_row, int32_t k, const sbha_opts* opts,
               double* Z_out, double* evals_out, int32_t* idx_out, void* stream);

/*
 * sbha_operator and sbha_embed on a generic graph instead of a mesh (Sec. 2.2: D = I, A = the 0/1
 * adjacency; geodesics along the graph's edges).  Same arguments, results and errors, plus
 * SBHA_EINVAL for a malformed graph (a row not ascending, a self loop, an edge without its
 * reverse or with a different reverse length, a length not finite and positive) and for a vertex
 * with more than 64 neighbours.
 */
int sbha_graph_operator(const sbha_graph* graph, const int32_t* idx, int32_t l, int32_t p_row,
                        const sbha_opts* opts, int32_t* rowptr, int32_t* col, double* val, int64_t cap,
                        int64_t* nnz_out, void* stream);
int sbha_graph_embed(const sbha_graph* graph, int32_t l, int32_t first, int32_t p_row, int32_t k,
                     const sbha_opts* opts, double* Z_out, double* evals_out, int32_t* idx_out, void* stream);

/*
 * The whole pipeline for a batch of meshes of uneven size.  The paper treats one shape at
 * a time; this call exists for throughput on many shapes.  Results equal sbha_embed's on
 * each mesh (landmarks and W bit for bit, operator and embedding to the solver tolerances).
 *   - Every mesh becomes one connected component of a union mesh; farthest-point
 *     selection of all meshes runs in one launch (one CTA per mesh), and the landmark
 *     distances of all meshes in one launch per ~4 GB of work arrays (one CTA per
 *     landmark).
 *   - Then each mesh's operator and scaling step run on `workers` host threads (<= 0:
 *     min(count, 8)), each with its own non-blocking CUDA stream, largest meshes first,
 *     so that small meshes share the GPU.
 * meshes[count]; l[count] landmarks per mesh; first[count] (NULL: vertex 0 of every mesh);
 * p_row, k, opts as for sbha_embed.  Z_out[i] float64 [n_i x k], evals_out[i] float64 [k],
 * idx_out[i] int32 [l_i] (idx_out or idx_out[i] may be NULL).  Arrays may be host or device
 * memory.  sbha_last_stats sums iteration counts and launches over the batch and takes the
 * maximum residuals.
 * Errors: as sbha_embed, with the failing mesh's index in sbha_last_error.
 */
int sbha_embed_batch(int32_t count, const sbha_mesh* meshes, const int32_t* l, const int32_t* first, int32_t p_row,
                     int32_t k, const sbha_opts* opts, double* const* Z_out, double* const* evals_out,
                     int32_t* const* idx_out, int32_t workers, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SBHA_H */
