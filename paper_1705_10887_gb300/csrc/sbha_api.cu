// C ABI of the library (declared in include/sbha.h): argument checks, host/device
// staging, per-stage timing and error translation around the stage drivers.
#include <algorithm>
#include <cmath>
#include <exception>

#include "internal.cuh"
#include "mlp.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <thread>
#include <utility>
#include <vector>

using namespace sbha;

namespace {

struct StageTimer {
  cudaStream_t s;
  bool on;
  cudaEvent_t a{}, b{};
  StageTimer(Ctx& c, bool enabled) : s(c.stream), on(enabled) {
    if (on) {
      SBHA_CUDA(cudaEventCreate(&a));
      SBHA_CUDA(cudaEventCreate(&b));
      SBHA_CUDA(cudaEventRecord(a, s));
    }
  }
  double stop() {
    if (!on) return 0.0;
    float ms = 0.f;
    SBHA_CUDA(cudaEventRecord(b, s));
    SBHA_CUDA(cudaEventSynchronize(b));
    SBHA_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
  }
  ~StageTimer() {
    if (on) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  }
};

__global__ void k_offset_faces(int64_t count, int32_t off, int32_t* __restrict__ f) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x)
    f[q] += off;
}

__global__ void k_to_global(int64_t count, int32_t off, const int32_t* __restrict__ a, int32_t* __restrict__ b) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x)
    b[q] = a[q] + off;
}

template <class F>
int guarded(F&& body) {
  thread_error().clear();
  thread_stats() = sbha_stats{};
  try {
    return body();
  } catch (const Error& e) {
    thread_error() = e.msg;
    cudaGetLastError();
    return e.status;
  } catch (const std::exception& e) {
    thread_error() = e.what();
    return SBHA_ECUDA;
  }
}

sbha_opts resolve(const sbha_opts* o) {
  sbha_opts r;
  sbha_opts_default(&r);
  if (o) r = *o;
  if (r.precision != SBHA_PREC_FP64 && r.precision != SBHA_PREC_FP32_REFINE)
    SBHA_THROW(SBHA_EINVAL, "unknown precision mode");
  if (r.precond != SBHA_PRECOND_JACOBI && r.precond != SBHA_PRECOND_MLP)
    SBHA_THROW(SBHA_EINVAL, "unknown preconditioner");
  if (r.sparsify_mode != SBHA_SPARSIFY_ROWS && r.sparsify_mode != SBHA_SPARSIFY_COLS)
    SBHA_THROW(SBHA_EINVAL, "unknown sparsify mode");
  if (r.solver != SBHA_SOLVER_FACTORED && r.solver != SBHA_SOLVER_DIRECT) SBHA_THROW(SBHA_EINVAL, "unknown solver");
  if (r.spmm_pipeline_depth != 0 && r.spmm_pipeline_depth != 2 && r.spmm_pipeline_depth != 4)
    SBHA_THROW(SBHA_EINVAL, "spmm_pipeline_depth must be 0, 2 or 4");
  if (r.spmm_variant < SBHA_SPMM_AUTO || r.spmm_variant > SBHA_SPMM_TMA)
    SBHA_THROW(SBHA_EINVAL, "unknown spmm variant");
  if (r.dense_mode < SBHA_DENSE_AUTO || r.dense_mode > SBHA_DENSE_TC) SBHA_THROW(SBHA_EINVAL, "unknown dense mode");
  if (r.eig_route != SBHA_EIG_LANDMARK && r.eig_route != SBHA_EIG_LANCZOS) SBHA_THROW(SBHA_EINVAL, "unknown eig route");
  if (r.spmm_chunk_rows != 0 && r.spmm_chunk_rows != -1 && r.spmm_chunk_rows != 16 && r.spmm_chunk_rows != 32 &&
      r.spmm_chunk_rows != 64)
    SBHA_THROW(SBHA_EINVAL, "spmm_chunk_rows must be 0, -1, 16, 32 or 64");
  if (r.cg_graph != 0 && r.cg_graph != 1) SBHA_THROW(SBHA_EINVAL, "cg_graph must be 0 or 1");
  if (r.mlp_pilot_cols < 0 || r.mlp_pilot_cols > 512) SBHA_THROW(SBHA_EINVAL, "mlp_pilot_cols must be in [0, 512]");
  if (r.fault_inject != SBHA_FAULT_NONE && r.fault_inject != SBHA_FAULT_MLP_NAN)
    SBHA_THROW(SBHA_EINVAL, "unknown fault_inject value");
  if (!(r.cg_rtol > 0.0) || r.cg_max_iter < 1 || r.refine_max < 0 || !(r.inner_rtol > 0.0) || r.oversample < 0 ||
      r.eig_max_iter < 1 || !(r.eig_tol > 0.0))
    SBHA_THROW(SBHA_EINVAL, "solver tolerances and limits must be positive");
  return r;
}

void check_mesh_args(const sbha_mesh* m) {
  if (!m) SBHA_THROW(SBHA_EINVAL, "mesh is NULL");
}

void finish_stats(Ctx& c) { thread_stats().kernel_launches = c.launches; }

// The operator of the graph that make_graph(c) builds (a mesh's edge graph or a caller's graph).
template <class MakeGraph>
int operator_common(int64_t n, MakeGraph&& make_graph, const int32_t* idx, int32_t l, int32_t p_row,
                    const sbha_opts* opts, int32_t* rowptr, int32_t* col, double* val, int64_t cap, int64_t* nnz_out,
                    void* stream) {
  sbha_opts o = resolve(opts);
  if (l < 1 || l > n) SBHA_THROW(SBHA_EINVAL, "l must be in [1, n]");
  if (p_row < 1 || p_row > 128) SBHA_THROW(SBHA_EINVAL, "p_row must be in [1, 128]");
  if (!idx) SBHA_THROW(SBHA_EINVAL, "idx is NULL");
  int64_t nnz = operator_nnz(n, l, p_row, o.sparsify_mode);
  if (nnz_out) *nnz_out = nnz;
  if (!col && !val) return SBHA_OK;
  if (!rowptr || !col || !val) SBHA_THROW(SBHA_EINVAL, "rowptr, col and val must all be given");
  if (cap < nnz) SBHA_THROW(SBHA_EINVAL, "cap is smaller than the operator's nonzero count");
  Ctx c(stream);
  c.timing = o.timing;
  c.graphs = o.cg_graph != 0;
  const int32_t* didx = stage_in(c, idx, l);
  Out<int32_t> rp, cl;
  Out<double> vl;
  rp.init(c, rowptr, n + 1);
  cl.init(c, col, nnz);
  vl.init(c, val, nnz);
  StageTimer ta(c, o.timing != 0);
  DevGraph g = make_graph(c);
  DevCSR M = build_biharmonic(c, g);
  thread_stats().ms_assembly = ta.stop();
  StageTimer ts(c, o.timing != 0);
  SolveReport r = interpolation_operator(c, g, M, didx, l, p_row, o, rp.dev, cl.dev, vl.dev);
  c.check_device("operator");
  thread_stats().ms_solve = ts.stop();
  rp.finish(c);
  cl.finish(c);
  vl.finish(c);
  c.sync();
  sbha_stats& st = thread_stats();
  st.cg_iterations = r.iterations;
  st.refinements = r.refinements;
  st.cg_max_rel_residual = r.max_rel_residual;
  finish_stats(c);
  if (!r.converged) {
    thread_error() = "conjugate gradients reached the iteration limit before cg_rtol";
    return SBHA_ENOCONV;
  }
  return SBHA_OK;
}

// The whole pipeline on the graph that make_graph(c) builds.
template <class MakeGraph>
int embed_common(int64_t n, MakeGraph&& make_graph, int32_t l, int32_t first, int32_t p_row, int32_t k,
                 const sbha_opts* opts, double* Z_out, double* evals_out, int32_t* idx_out, void* stream) {
  sbha_opts o = resolve(opts);
  if (l < 1 || l > n) SBHA_THROW(SBHA_EINVAL, "l must be in [1, n]");
  if (first < 0 || first >= n) SBHA_THROW(SBHA_EINVAL, "first landmark out of range");
  if (p_row < 1 || p_row > 128) SBHA_THROW(SBHA_EINVAL, "p_row must be in [1, 128]");
  if (k < 1 || !Z_out || !evals_out) SBHA_THROW(SBHA_EINVAL, "bad embed outputs");
  Ctx c(stream);
  c.timing = o.timing;
  c.graphs = o.cg_graph != 0;
  bool timing = o.timing != 0;
  Out<double> Z, ev;
  Z.init(c, Z_out, static_cast<size_t>(n) * k);
  ev.init(c, evals_out, k);
  Out<int32_t> idxo;
  int32_t* idx = nullptr;
  if (idx_out) {
    idxo.init(c, idx_out, l);
    idx = idxo.dev;
  } else {
    idx = c.alloc<int32_t>(l);
  }
  sbha_stats& st = thread_stats();
  StageTimer ta(c, timing);
  DevGraph g = make_graph(c);
  DevCSR M = build_biharmonic(c, g);
  st.ms_assembly = ta.stop();
  StageTimer tl(c, timing);
  double* mind = c.alloc<double>(n);
  fps(c, g, l, first, idx, mind);
  c.free(mind);
  st.ms_landmarks = tl.stop();
  StageTimer tg(c, timing);
  double* W = c.alloc<double>(static_cast<size_t>(l) * l);
  landmark_block(c, g, idx, l, W);
  c.check_device("landmark_distances");
  st.ms_geodesics = tg.stop();
  StageTimer ts(c, timing);
  int64_t nnz = operator_nnz(n, l, p_row, o.sparsify_mode);
  int32_t* rowptr = c.alloc<int32_t>(n + 1);
  int32_t* col = c.alloc<int32_t>(nnz);
  double* val = c.alloc<double>(nnz);
  SolveReport sr = interpolation_operator(c, g, M, idx, l, p_row, o, rowptr, col, val);
  c.check_device("operator");
  st.ms_solve = ts.stop();
  StageTimer tm(c, timing);
  MdsReport mr = classical_scaling(c, n, l, rowptr, col, val, W, k, o, Z.dev, ev.dev);
  st.ms_mds = tm.stop();
  Z.finish(c);
  ev.finish(c);
  if (idx_out) idxo.finish(c);
  c.sync();
  st.cg_iterations = sr.iterations;
  st.refinements = sr.refinements;
  st.cg_max_rel_residual = sr.max_rel_residual;
  st.eig_iterations = mr.iterations;
  st.eig_residual = mr.residual;
  finish_stats(c);
  if (!sr.converged) {
    thread_error() = "conjugate gradients reached the iteration limit before cg_rtol";
    return SBHA_ENOCONV;
  }
  if (!mr.converged) {
    thread_error() = "the eigensolver reached eig_max_iter before its tolerance";
    return SBHA_ENOCONV;
  }
  return SBHA_OK;
}


}  // namespace

extern "C" {

void sbha_opts_default(sbha_opts* o) {
  if (!o) return;
  *o = sbha_opts{};
  o->precision = SBHA_PREC_FP64;
  o->precond = SBHA_PRECOND_JACOBI;
  o->sparsify_mode = SBHA_SPARSIFY_ROWS;
  o->chunk_cols = 0;
  o->cg_rtol = 1e-11;
  o->cg_max_iter = 20000;
  o->refine_max = 12;
  o->inner_rtol = 1e-5;
  o->oversample = 13;
  o->eig_max_iter = 300;
  o->eig_tol = 1e-12;
  o->seed = 0x5eedull;
  o->timing = 0;
  o->solver = SBHA_SOLVER_FACTORED;
  o->mlp_epochs = 60;
  o->spmm_variant = SBHA_SPMM_AUTO;
  o->dense_mode = SBHA_DENSE_AUTO;
  o->eig_route = SBHA_EIG_LANDMARK;
  o->cg_graph = 1;
}

int sbha_last_stats(sbha_stats* out) {
  if (!out) return SBHA_EINVAL;
  *out = thread_stats();
  return SBHA_OK;
}

const char* sbha_last_error(void) { return thread_error().c_str(); }

const char* sbha_version(void) { return "sbha-gb300 0.1 (sm_103a)"; }

int sbha_landmarks(const sbha_mesh* mesh, int32_t l, int32_t first, int32_t* idx_out, double* mind_out,
                   void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    if (l < 1 || l > mesh->n_vertices) SBHA_THROW(SBHA_EINVAL, "l must be in [1, n]");
    if (first < 0 || first >= mesh->n_vertices) SBHA_THROW(SBHA_EINVAL, "first landmark out of range");
    if (!idx_out) SBHA_THROW(SBHA_EINVAL, "idx_out is NULL");
    Ctx c(stream);
    DevMesh m = stage_mesh(c, mesh);
    StageTimer t0(c, false);
    DevGraph g = build_edge_lengths(c, m);
    Out<int32_t> idx;
    idx.init(c, idx_out, l);
    Out<double> mind;
    double* mind_dev = nullptr;
    if (mind_out) {
      mind.init(c, mind_out, m.n);
      mind_dev = mind.dev;
    } else {
      mind_dev = c.alloc<double>(m.n);
    }
    fps(c, g, l, first, idx.dev, mind_dev);
    idx.finish(c);
    if (mind_out) mind.finish(c);
    c.sync();
    finish_stats(c);
    return SBHA_OK;
  });
}

int sbha_geodesics(const sbha_mesh* mesh, const int32_t* src, int32_t s, const int32_t* tgt, int32_t t,
                   double* D_out, void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    if (s < 0 || (tgt && t < 0) || !D_out || (s > 0 && !src)) SBHA_THROW(SBHA_EINVAL, "bad geodesics arguments");
    if (s == 0 || (tgt && t == 0)) return SBHA_OK;
    Ctx c(stream);
    DevMesh m = stage_mesh(c, mesh);
    DevGraph g = build_edge_lengths(c, m);
    const int32_t* dsrc = stage_in(c, src, s);
    const int32_t* dtgt = tgt ? stage_in(c, tgt, t) : nullptr;
    int64_t cols = tgt ? t : m.n;
    Out<double> D;
    D.init(c, D_out, static_cast<size_t>(s) * cols);
    geodesics(c, g, dsrc, s, dtgt, tgt ? t : 0, D.dev);
    c.check_device("geodesics");
    D.finish(c);
    c.sync();
    finish_stats(c);
    return SBHA_OK;
  });
}

int sbha_landmark_distances(const sbha_mesh* mesh, const int32_t* idx, int32_t l, double* W_out, void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    if (l < 1 || !idx || !W_out) SBHA_THROW(SBHA_EINVAL, "bad landmark_distances arguments");
    Ctx c(stream);
    DevMesh m = stage_mesh(c, mesh);
    DevGraph g = build_edge_lengths(c, m);
    const int32_t* didx = stage_in(c, idx, l);
    Out<double> W;
    W.init(c, W_out, static_cast<size_t>(l) * l);
    landmark_block(c, g, didx, l, W.dev);
    c.check_device("landmark_distances");
    W.finish(c);
    c.sync();
    finish_stats(c);
    return SBHA_OK;
  });
}

int sbha_mesh_graph(const sbha_mesh* mesh, int32_t* rowptr, int32_t* col, double* len, double* A, double* D,
                    double* V, int64_t cap, int64_t* nnz_out, void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    Ctx c(stream);
    DevMesh m = stage_mesh(c, mesh);
    DevGraph g = build_graph(c, m);
    c.check_device("mesh_graph");
    if (nnz_out) *nnz_out = g.nnz;
    if (!col) {
      finish_stats(c);
      return SBHA_OK;
    }
    if (!rowptr || !len || !A || !D || !V) SBHA_THROW(SBHA_EINVAL, "rowptr, col, len, A, D and V must all be given");
    if (cap < g.nnz) SBHA_THROW(SBHA_EINVAL, "cap is smaller than the number of directed edges");
    Out<int32_t> rp, cl;
    Out<double> ln, av, dv, vv;
    rp.init(c, rowptr, g.n + 1);
    cl.init(c, col, g.nnz);
    ln.init(c, len, g.nnz);
    av.init(c, A, g.nnz);
    dv.init(c, D, g.n);
    vv.init(c, V, g.n);
    SBHA_CUDA(cudaMemcpyAsync(rp.dev, g.rowptr, sizeof(int32_t) * (g.n + 1), cudaMemcpyDeviceToDevice, c.stream));
    SBHA_CUDA(cudaMemcpyAsync(cl.dev, g.col, sizeof(int32_t) * g.nnz, cudaMemcpyDeviceToDevice, c.stream));
    SBHA_CUDA(cudaMemcpyAsync(ln.dev, g.len, sizeof(double) * g.nnz, cudaMemcpyDeviceToDevice, c.stream));
    SBHA_CUDA(cudaMemcpyAsync(av.dev, g.A, sizeof(double) * g.nnz, cudaMemcpyDeviceToDevice, c.stream));
    SBHA_CUDA(cudaMemcpyAsync(dv.dev, g.D, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, c.stream));
    SBHA_CUDA(cudaMemcpyAsync(vv.dev, g.V, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, c.stream));
    rp.finish(c);
    cl.finish(c);
    ln.finish(c);
    av.finish(c);
    dv.finish(c);
    vv.finish(c);
    c.sync();
    finish_stats(c);
    return SBHA_OK;
  });
}

int sbha_biharmonic(const sbha_mesh* mesh, int32_t* rowptr, int32_t* col, double* val, int64_t cap,
                    int64_t* nnz_out, void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    Ctx c(stream);
    DevMesh m = stage_mesh(c, mesh);
    DevGraph g = build_graph(c, m);
    DevCSR M = build_biharmonic(c, g);
    c.check_device("biharmonic");
    if (nnz_out) *nnz_out = M.nnz;
    if (!col) {
      finish_stats(c);
      return SBHA_OK;
    }
    if (!rowptr || !val) SBHA_THROW(SBHA_EINVAL, "rowptr, col and val must all be given");
    if (cap < M.nnz) SBHA_THROW(SBHA_EINVAL, "cap is smaller than the operator's nonzero count");
    Out<int32_t> rp, cl;
    Out<double> vl;
    rp.init(c, rowptr, M.rows + 1);
    cl.init(c, col, M.nnz);
    vl.init(c, val, M.nnz);
    SBHA_CUDA(cudaMemcpyAsync(rp.dev, M.rowptr, sizeof(int32_t) * (M.rows + 1), cudaMemcpyDeviceToDevice, c.stream));
    SBHA_CUDA(cudaMemcpyAsync(cl.dev, M.col, sizeof(int32_t) * M.nnz, cudaMemcpyDeviceToDevice, c.stream));
    SBHA_CUDA(cudaMemcpyAsync(vl.dev, M.val, sizeof(double) * M.nnz, cudaMemcpyDeviceToDevice, c.stream));
    rp.finish(c);
    cl.finish(c);
    vl.finish(c);
    c.sync();
    finish_stats(c);
    return SBHA_OK;
  });
}

int sbha_operator(const sbha_mesh* mesh, const int32_t* idx, int32_t l, int32_t p_row, const sbha_opts* opts,
                  int32_t* rowptr, int32_t* col, double* val, int64_t cap, int64_t* nnz_out, void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    return operator_common(
        mesh->n_vertices,
        [&](Ctx& c) {
          DevMesh m = stage_mesh(c, mesh);
          return build_graph(c, m);
        },
        idx, l, p_row, opts, rowptr, col, val, cap, nnz_out, stream);
  });
}

int sbha_graph_operator(const sbha_graph* graph, const int32_t* idx, int32_t l, int32_t p_row, const sbha_opts* opts,
                        int32_t* rowptr, int32_t* col, double* val, int64_t cap, int64_t* nnz_out, void* stream) {
  return guarded([&]() -> int {
    if (!graph) SBHA_THROW(SBHA_EINVAL, "graph is NULL");
    return operator_common(
        graph->n_vertices, [&](Ctx& c) { return build_graph_csr(c, graph, true); }, idx, l, p_row, opts, rowptr, col,
        val, cap, nnz_out, stream);
  });
}

int sbha_mds(int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col, const double* val, const double* W,
             int32_t k, const sbha_opts* opts, double* Z_out, double* evals_out, void* stream) {
  return guarded([&]() -> int {
    sbha_opts o = resolve(opts);
    if (n < 1 || l < 1 || k < 1 || !rowptr || !col || !val || !W || !Z_out || !evals_out)
      SBHA_THROW(SBHA_EINVAL, "bad mds arguments");
    Ctx c(stream);
    c.timing = o.timing;
    c.graphs = o.cg_graph != 0;
    int32_t nnz32 = 0;
    if (is_device_ptr(rowptr)) {
      SBHA_CUDA(cudaMemcpyAsync(&nnz32, rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
      c.sync();
    } else {
      nnz32 = rowptr[n];
    }
    if (nnz32 < 0) SBHA_THROW(SBHA_EINVAL, "rowptr[n] is negative");
    const int32_t* drp = stage_in(c, rowptr, n + 1);
    const int32_t* dcol = stage_in(c, col, nnz32);
    const double* dval = stage_in(c, val, nnz32);
    const double* dW = stage_in(c, W, static_cast<size_t>(l) * l);
    Out<double> Z, ev;
    Z.init(c, Z_out, static_cast<size_t>(n) * k);
    ev.init(c, evals_out, k);
    StageTimer tm(c, o.timing != 0);
    MdsReport r = classical_scaling(c, n, l, drp, dcol, dval, dW, k, o, Z.dev, ev.dev);
    thread_stats().ms_mds = tm.stop();
    Z.finish(c);
    ev.finish(c);
    c.sync();
    thread_stats().eig_iterations = r.iterations;
    thread_stats().eig_residual = r.residual;
    finish_stats(c);
    if (!r.converged) {
      thread_error() = "the eigensolver reached eig_max_iter before its tolerance";
      return SBHA_ENOCONV;
    }
    return SBHA_OK;
  });
}

int sbha_embed(const sbha_mesh* mesh, int32_t l, int32_t first, int32_t p_row, int32_t k, const sbha_opts* opts,
               double* Z_out, double* evals_out, int32_t* idx_out, void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    return embed_common(
        mesh->n_vertices,
        [&](Ctx& c) {
          DevMesh m = stage_mesh(c, mesh);
          return build_graph(c, m);
        },
        l, first, p_row, k, opts, Z_out, evals_out, idx_out, stream);
  });
}

int sbha_graph_embed(const sbha_graph* graph, int32_t l, int32_t first, int32_t p_row, int32_t k,
                     const sbha_opts* opts, double* Z_out, double* evals_out, int32_t* idx_out, void* stream) {
  return guarded([&]() -> int {
    if (!graph) SBHA_THROW(SBHA_EINVAL, "graph is NULL");
    return embed_common(
        graph->n_vertices, [&](Ctx& c) { return build_graph_csr(c, graph, true); }, l, first, p_row, k, opts, Z_out,
        evals_out, idx_out, stream);
  });
}

int sbha_bha_error(int64_t n, int32_t l, const int32_t* rowptr, const int32_t* col, const double* val,
                   const double* W, int32_t ns, const int32_t* rows, const double* K_rows, int32_t squared,
                   double* num_out, double* den_out, void* stream) {
  return guarded([&]() -> int {
    if (n < 1 || l < 1 || ns < 0 || !rowptr || !col || !val || !W || !num_out || !den_out || (ns > 0 && (!rows || !K_rows)))
      SBHA_THROW(SBHA_EINVAL, "bad bha_error arguments");
    Ctx c(stream);
    int32_t nnz32 = 0;
    if (is_device_ptr(rowptr)) {
      SBHA_CUDA(cudaMemcpyAsync(&nnz32, rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
      c.sync();
    } else {
      nnz32 = rowptr[n];
    }
    if (nnz32 < 0) SBHA_THROW(SBHA_EINVAL, "rowptr[n] is negative");
    const int32_t* drp = stage_in(c, rowptr, n + 1);
    const int32_t* dcol = stage_in(c, col, nnz32);
    const double* dval = stage_in(c, val, nnz32);
    const double* dW = stage_in(c, W, static_cast<size_t>(l) * l);
    const int32_t* drows = ns > 0 ? stage_in(c, rows, ns) : nullptr;
    const double* dK = ns > 0 ? stage_in(c, K_rows, static_cast<size_t>(ns) * n) : nullptr;
    double* acc = c.alloc<double>(2);
    bha_error(c, n, l, drp, dcol, dval, dW, ns, drows, dK, squared != 0, acc);
    double h[2] = {0.0, 0.0};
    SBHA_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    for (auto [out, v] : {std::pair<double*, double>{num_out, h[0]}, std::pair<double*, double>{den_out, h[1]}}) {
      if (is_device_ptr(out))
        SBHA_CUDA(cudaMemcpyAsync(out, &v, sizeof(double), cudaMemcpyHostToDevice, c.stream));
      else
        *out = v;
    }
    c.sync();
    finish_stats(c);
    return SBHA_OK;
  });
}

int sbha_fmds_operator(const sbha_mesh* mesh, const int32_t* idx, int32_t l, double mu, const sbha_opts* opts,
                       double* H_out, void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    sbha_opts o = resolve(opts);
    const int64_t n = mesh->n_vertices;
    if (l < 1 || l > n) SBHA_THROW(SBHA_EINVAL, "l must be in [1, n]");
    if (!idx || !H_out) SBHA_THROW(SBHA_EINVAL, "idx and H_out must be given");
    if (!(mu > 0.0) || !std::isfinite(mu)) SBHA_THROW(SBHA_EINVAL, "mu must be finite and positive");
    Ctx c(stream);
    c.timing = o.timing;
    c.graphs = o.cg_graph != 0;
    DevMesh dm = stage_mesh(c, mesh);
    const int32_t* didx = stage_in(c, idx, l);
    Out<double> Hv;
    Hv.init(c, H_out, static_cast<size_t>(n) * l);
    DevGraph g = build_graph(c, dm);
    DevCSR M = build_biharmonic(c, g);
    double* P = c.alloc<double>(static_cast<size_t>(n) * l);
    SolveReport r = interpolation_operator(c, g, M, didx, l, 1, o, nullptr, nullptr, nullptr, P);
    c.check_device("operator");
    fmds_interpolation(c, M, didx, l, P, mu, o, Hv.dev);
    c.check_device("fmds");
    Hv.finish(c);
    c.sync();
    sbha_stats& st = thread_stats();
    st.cg_iterations = r.iterations;
    st.refinements = r.refinements;
    st.cg_max_rel_residual = r.max_rel_residual;
    finish_stats(c);
    if (!r.converged) {
      thread_error() = "conjugate gradients reached the iteration limit before cg_rtol";
      return SBHA_ENOCONV;
    }
    return SBHA_OK;
  });
}

int sbha_heat_geodesics(const sbha_mesh* mesh, const int32_t* src, int32_t ns, double m, const sbha_opts* opts,
                        double* D_out, void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    sbha_opts o = resolve(opts);
    if (ns < 1 || !src || !D_out) SBHA_THROW(SBHA_EINVAL, "bad heat_geodesics arguments");
    const double mfac = m > 0.0 ? m : 1.0;
    Ctx c(stream);
    c.timing = o.timing;
    c.graphs = o.cg_graph != 0;
    DevMesh dm = stage_mesh(c, mesh);
    const int32_t* dsrc = stage_in(c, src, ns);
    Out<double> Dv;
    Dv.init(c, D_out, static_cast<size_t>(ns) * dm.n);
    DevGraph g = build_graph(c, dm);
    int32_t sweeps = 0;
    SpdReport r = heat_geodesics(c, dm, g, dsrc, ns, mfac, o, Dv.dev, &sweeps);
    c.check_device("heat_geodesics");
    Dv.finish(c);
    c.sync();
    sbha_stats& st = thread_stats();
    st.cg_iterations = r.iterations;
    st.cg_max_rel_residual = r.max_rel;
    st.heat_sweeps = sweeps;
    finish_stats(c);
    if (!r.converged) {
      thread_error() = "the heat sweeps or the Poisson solve did not converge";
      return SBHA_ENOCONV;
    }
    return SBHA_OK;
  });
}

int sbha_mlp_gradient(int64_t N, const float* X, const float* T, const float* params, float* grad_out,
                      double* loss_out, void* stream) {
  return guarded([&]() -> int {
    if (N < 0 || (N > 0 && (!X || !T)) || !params || !grad_out || !loss_out)
      SBHA_THROW(SBHA_EINVAL, "bad mlp_gradient arguments");
    Ctx c(stream);
    const float* dX = N > 0 ? stage_in(c, X, static_cast<size_t>(N) * kMlpFeatures) : nullptr;
    const float* dT = N > 0 ? stage_in(c, T, static_cast<size_t>(N)) : nullptr;
    const float* dP = stage_in(c, params, kMlpParams);
    Out<float> g;
    Out<double> lo;
    g.init(c, grad_out, kMlpParams);
    lo.init(c, loss_out, 1);
    mlp_gradient(c, N, dX, dT, dP, g.dev, lo.dev);
    g.finish(c);
    lo.finish(c);
    c.sync();
    finish_stats(c);
    return SBHA_OK;
  });
}

int sbha_precond_gradient(int64_t m, const int32_t* rowptr, const int32_t* col, const double* val, int32_t ncols,
                          const double* B, const double* X, const float* params, float* grad_out, double* loss_out,
                          void* stream) {
  return guarded([&]() -> int {
    if (m < 1 || m > INT32_MAX || !rowptr || !col || !val || !B || !params || !grad_out || !loss_out)
      SBHA_THROW(SBHA_EINVAL, "bad precond_gradient arguments");
    if (ncols < 1 || ncols > kPrecondMaxTrainCols) SBHA_THROW(SBHA_EINVAL, "ncols must lie in [1, 512]");
    Ctx c(stream);
    const int32_t* dptr = stage_in(c, rowptr, static_cast<size_t>(m) + 1);
    int32_t ends[2] = {0, 0};
    SBHA_CUDA(cudaMemcpyAsync(ends, dptr, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    SBHA_CUDA(cudaMemcpyAsync(ends + 1, dptr + m, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    if (ends[0] != 0 || ends[1] < m) SBHA_THROW(SBHA_EINVAL, "malformed CSR row pointers");
    int64_t nnz = ends[1];
    check_rowptr(c, m, dptr);
    const int32_t* dcol = stage_in(c, col, static_cast<size_t>(nnz));
    const double* dval = stage_in(c, val, static_cast<size_t>(nnz));
    const double* dB = stage_in(c, B, static_cast<size_t>(m) * ncols);
    const float* dP = stage_in(c, params, kMlpParams);
    float* val32 = c.alloc<float>(nnz);
    to_float(c, nnz, dval, val32);
    int ncp = (ncols + 31) / 32 * 32;
    double* Bblk = c.alloc<double>(static_cast<size_t>(m) * ncp);
    rows_to_blocks(c, m, ncols, dB, Bblk);
    double* Xblk = nullptr;
    if (X) {
      const double* dX = stage_in(c, X, static_cast<size_t>(m) * ncols);
      Xblk = c.alloc<double>(static_cast<size_t>(m) * ncp);
      rows_to_blocks(c, m, ncols, dX, Xblk);
    }
    Out<float> g;
    Out<double> lo;
    g.init(c, grad_out, kMlpParams);
    lo.init(c, loss_out, 1);
    LearnedPrecond P(c, m, nnz, dptr, dcol, dval, val32);
    P.loss_grad(Bblk, Xblk, ncols, dP, g.dev, lo.dev);
    g.finish(c);
    lo.finish(c);
    c.sync();
    finish_stats(c);
    return SBHA_OK;
  });
}


int sbha_embed_batch(int32_t count, const sbha_mesh* meshes, const int32_t* l, const int32_t* first, int32_t p_row,
                     int32_t k, const sbha_opts* opts, double* const* Z_out, double* const* evals_out,
                     int32_t* const* idx_out, int32_t workers, void* stream) {
  return guarded([&]() -> int {
    if (count < 1 || !meshes || !l || !Z_out || !evals_out) SBHA_THROW(SBHA_EINVAL, "bad batch arguments");
    if (p_row < 1 || p_row > 128) SBHA_THROW(SBHA_EINVAL, "p_row must be in [1, 128]");
    if (k < 1) SBHA_THROW(SBHA_EINVAL, "k must be at least 1");
    sbha_opts o = resolve(opts);
    std::vector<int64_t> vo(count + 1, 0), fo(count + 1, 0), lo(count + 1, 0), wo(count + 1, 0);
    for (int i = 0; i < count; ++i) {
      check_mesh_args(&meshes[i]);
      int64_t n = meshes[i].n_vertices;
      if (l[i] < 1 || l[i] > n) SBHA_THROW(SBHA_EINVAL, "mesh " + std::to_string(i) + ": l must be in [1, n]");
      if (first && (first[i] < 0 || first[i] >= n))
        SBHA_THROW(SBHA_EINVAL, "mesh " + std::to_string(i) + ": first landmark out of range");
      if (!Z_out[i] || !evals_out[i]) SBHA_THROW(SBHA_EINVAL, "mesh " + std::to_string(i) + ": missing outputs");
      vo[i + 1] = vo[i] + n;
      fo[i + 1] = fo[i] + meshes[i].n_faces;
      lo[i + 1] = lo[i] + l[i];
      wo[i + 1] = wo[i] + static_cast<int64_t>(l[i]) * l[i];
    }
    if (vo[count] > INT32_MAX / 2) SBHA_THROW(SBHA_EINVAL, "batch too large for 32-bit vertex ids");
    Ctx c(stream);
    // 1. every mesh as one component of a union mesh; landmarks of all meshes in one launch
    double* uxyz = c.alloc<double>(3 * vo[count]);
    int32_t* ufaces = c.alloc<int32_t>(3 * fo[count]);
    for (int i = 0; i < count; ++i) {
      SBHA_CUDA(cudaMemcpyAsync(uxyz + 3 * vo[i], meshes[i].xyz, sizeof(double) * 3 * meshes[i].n_vertices,
                                cudaMemcpyDefault, c.stream));
      SBHA_CUDA(cudaMemcpyAsync(ufaces + 3 * fo[i], meshes[i].faces, sizeof(int32_t) * 3 * meshes[i].n_faces,
                                cudaMemcpyDefault, c.stream));
      if (vo[i] > 0) {
        k_offset_faces<<<grid_for(3 * meshes[i].n_faces, 256), 256, 0, c.stream>>>(
            3 * meshes[i].n_faces, static_cast<int32_t>(vo[i]), ufaces + 3 * fo[i]);
        c.launched("offset_faces");
      }
    }
    DevMesh um;
    um.n = vo[count];
    um.f = fo[count];
    um.xyz = uxyz;
    um.faces = ufaces;
    DevGraph ug = build_edge_lengths(c, um);
    std::vector<FpsJob> fj(count);
    int64_t seg = 0;
    for (int i = 0; i < count; ++i) {
      int32_t n = static_cast<int32_t>(meshes[i].n_vertices);
      fj[i] = FpsJob{static_cast<int32_t>(vo[i]), n, l[i], first ? first[i] : 0, static_cast<int32_t>(lo[i]),
                     static_cast<int32_t>(seg)};
      seg += (n + 31) / 32;
    }
    int32_t* didx = c.alloc<int32_t>(lo[count]);  // landmark ids relative to each mesh
    double* mind = c.alloc<double>(vo[count]);
    fps_jobs(c, ug, fj, didx, mind);
    c.free(mind);
    // 2. landmark distances of all meshes: one CTA per (mesh, landmark)
    int32_t* gidx = c.alloc<int32_t>(lo[count]);  // the same landmarks as union vertex ids
    for (int i = 0; i < count; ++i) {
      k_to_global<<<grid_for(l[i], 256), 256, 0, c.stream>>>(l[i], static_cast<int32_t>(vo[i]), didx + lo[i],
                                                            gidx + lo[i]);
      c.launched("to_global");
    }
    std::vector<int32_t> hg(lo[count]);
    SBHA_CUDA(cudaMemcpyAsync(hg.data(), gidx, sizeof(int32_t) * lo[count], cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    std::vector<SsspJob> sj;
    sj.reserve(lo[count]);
    for (int i = 0; i < count; ++i)
      for (int j = 0; j < l[i]; ++j)
        sj.push_back(SsspJob{hg[lo[i] + j], static_cast<int32_t>(vo[i]), static_cast<int32_t>(meshes[i].n_vertices),
                             static_cast<int32_t>(lo[i]), l[i], wo[i] + static_cast<int64_t>(j) * l[i], 0});
    double* D = c.alloc<double>(wo[count]);
    double* W = c.alloc<double>(wo[count]);
    sssp_jobs(c, ug, sj, gidx, D);
    for (int i = 0; i < count; ++i) symmetrise(c, D + wo[i], W + wo[i], l[i]);
    c.check_device("landmark_distances");
    int64_t launches = c.launches;
    // 3. every mesh's operator and scaling step, meshes largest first on worker streams
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return meshes[a].n_vertices > meshes[b].n_vertices; });
    int nw = workers > 0 ? std::min(workers, count) : std::min(count, 8);
    std::atomic<int> next{0};
    std::mutex mu;
    int err_status = SBHA_OK;
    std::string err_msg;
    sbha_stats agg = sbha_stats{};
    bool noconv = false;
    auto worker = [&]() {
      cudaStream_t ws = nullptr;
      if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
        std::lock_guard<std::mutex> g(mu);
        if (err_status == SBHA_OK) {
          err_status = SBHA_ECUDA;
          err_msg = "stream creation failed";
        }
        return;
      }
      for (;;) {
        int q = next.fetch_add(1);
        if (q >= count) break;
        {
          std::lock_guard<std::mutex> g(mu);
          if (err_status != SBHA_OK) break;
        }
        int i = order[q];
        try {
          thread_stats() = sbha_stats{};
          Ctx ci(ws);
          ci.graphs = o.cg_graph != 0;
          int64_t n = meshes[i].n_vertices;
          DevMesh mi = stage_mesh(ci, &meshes[i]);
          DevGraph gi = build_graph(ci, mi);
          DevCSR Mi = build_biharmonic(ci, gi);
          int64_t nnz = operator_nnz(n, l[i], p_row, o.sparsify_mode);
          int32_t* rowptr = ci.alloc<int32_t>(n + 1);
          int32_t* col = ci.alloc<int32_t>(nnz);
          double* val = ci.alloc<double>(nnz);
          Out<double> Z, ev;
          Z.init(ci, Z_out[i], static_cast<size_t>(n) * k);
          ev.init(ci, evals_out[i], k);
          SolveReport sr = interpolation_operator(ci, gi, Mi, didx + lo[i], l[i], p_row, o, rowptr, col, val);
          ci.check_device("operator");
          MdsReport mr = classical_scaling(ci, n, l[i], rowptr, col, val, W + wo[i], k, o, Z.dev, ev.dev);
          Z.finish(ci);
          ev.finish(ci);
          if (idx_out && idx_out[i])
            SBHA_CUDA(cudaMemcpyAsync(idx_out[i], didx + lo[i], sizeof(int32_t) * l[i], cudaMemcpyDefault, ws));
          ci.sync();
          sbha_stats st = thread_stats();
          std::lock_guard<std::mutex> g(mu);
          agg.cg_iterations += sr.iterations;
          agg.refinements = std::max(agg.refinements, sr.refinements);
          agg.cg_max_rel_residual = std::max(agg.cg_max_rel_residual, sr.max_rel_residual);
          agg.eig_iterations = std::max(agg.eig_iterations, mr.iterations);
          agg.eig_residual = std::max(agg.eig_residual, mr.residual);
          agg.kernel_launches += ci.launches;
          agg.mlp_trained += st.mlp_trained;
          agg.mlp_fallback += st.mlp_fallback;
          agg.e_iterations += st.e_iterations;
          agg.k_iterations += st.k_iterations;
          agg.correction_iterations += st.correction_iterations;
          if (!sr.converged || !mr.converged) noconv = true;
        } catch (const Error& e) {
          std::lock_guard<std::mutex> g(mu);
          if (err_status == SBHA_OK) {
            err_status = e.status;
            err_msg = "mesh " + std::to_string(i) + ": " + e.msg;
          }
        } catch (const std::exception& e) {
          std::lock_guard<std::mutex> g(mu);
          if (err_status == SBHA_OK) {
            err_status = SBHA_ECUDA;
            err_msg = "mesh " + std::to_string(i) + ": " + e.what();
          }
        }
      }
      cudaStreamSynchronize(ws);
      cudaStreamDestroy(ws);
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < nw; ++t) pool.emplace_back(worker);
    for (std::thread& t : pool) t.join();
    agg.kernel_launches += launches;
    thread_stats() = agg;
    if (err_status != SBHA_OK) {
      thread_error() = err_msg;
      return err_status;
    }
    if (noconv) {
      thread_error() = "an iterative solver reached its iteration limit on some mesh";
      return SBHA_ENOCONV;
    }
    return SBHA_OK;
  });
}


int sbha_dgemm(int64_t M, int64_t N, int64_t K, const double* A, const double* B, double* C, int32_t mode,
               void* stream) {
  return guarded([&]() -> int {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C) SBHA_THROW(SBHA_EINVAL, "bad dgemm arguments");
    if (mode < SBHA_DENSE_AUTO || mode > SBHA_DENSE_TC) SBHA_THROW(SBHA_EINVAL, "unknown dense mode");
    Ctx c(stream);
    const double* dA = stage_in(c, A, static_cast<size_t>(M) * K);
    const double* dB = stage_in(c, B, static_cast<size_t>(K) * N);
    Out<double> Co;
    Co.init(c, C, static_cast<size_t>(M) * N);
    if (mode == SBHA_DENSE_FP64)
      dgemm_rowmajor(c, M, N, K, dA, dB, Co.dev);
    else
      dgemm_tc_rowmajor(c, M, N, K, dA, dB, Co.dev);
    Co.finish(c);
    c.sync();
    finish_stats(c);
    return SBHA_OK;
  });
}

}  // extern "C"
