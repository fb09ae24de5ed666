// C ABI of the library (declared in include/sbha.h): argument checks, host/device
// staging, per-stage timing and error translation around the stage drivers.
#include <algorithm>
#include <cmath>
#include <exception>

#include "internal.cuh"
#include "mlp.cuh"

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
  if (r.spmm_variant < SBHA_SPMM_AUTO || r.spmm_variant > SBHA_SPMM_STAGED)
    SBHA_THROW(SBHA_EINVAL, "unknown spmm variant");
  if (!(r.cg_rtol > 0.0) || r.cg_max_iter < 1 || r.refine_max < 0 || !(r.inner_rtol > 0.0) || r.oversample < 0 ||
      r.eig_max_iter < 1 || !(r.eig_tol > 0.0))
    SBHA_THROW(SBHA_EINVAL, "solver tolerances and limits must be positive");
  return r;
}

void check_mesh_args(const sbha_mesh* m) {
  if (!m) SBHA_THROW(SBHA_EINVAL, "mesh is NULL");
}

void finish_stats(Ctx& c) { thread_stats().kernel_launches = c.launches; }

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
  o->eig_tol = 1e-13;
  o->seed = 0x5eedull;
  o->timing = 0;
  o->solver = SBHA_SOLVER_FACTORED;
  o->mlp_epochs = 60;
  o->spmm_variant = SBHA_SPMM_AUTO;
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

int sbha_operator(const sbha_mesh* mesh, const int32_t* idx, int32_t l, int32_t p_row, const sbha_opts* opts,
                  int32_t* rowptr, int32_t* col, double* val, int64_t cap, int64_t* nnz_out, void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    sbha_opts o = resolve(opts);
    int64_t n = mesh->n_vertices;
    if (l < 1 || l > n) SBHA_THROW(SBHA_EINVAL, "l must be in [1, n]");
    if (p_row < 1 || p_row > 64) SBHA_THROW(SBHA_EINVAL, "p_row must be in [1, 64]");
    if (!idx) SBHA_THROW(SBHA_EINVAL, "idx is NULL");
    int64_t nnz = operator_nnz(n, l, p_row, o.sparsify_mode);
    if (nnz_out) *nnz_out = nnz;
    if (!col && !val) return SBHA_OK;
    if (!rowptr || !col || !val) SBHA_THROW(SBHA_EINVAL, "rowptr, col and val must all be given");
    if (cap < nnz) SBHA_THROW(SBHA_EINVAL, "cap is smaller than the operator's nonzero count");
    Ctx c(stream);
    c.timing = o.timing;
    DevMesh m = stage_mesh(c, mesh);
    const int32_t* didx = stage_in(c, idx, l);
    Out<int32_t> rp, cl;
    Out<double> vl;
    rp.init(c, rowptr, n + 1);
    cl.init(c, col, nnz);
    vl.init(c, val, nnz);
    StageTimer ta(c, o.timing != 0);
    DevGraph g = build_graph(c, m);
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
      thread_error() = "subspace iteration reached eig_max_iter before eig_tol";
      return SBHA_ENOCONV;
    }
    return SBHA_OK;
  });
}

int sbha_embed(const sbha_mesh* mesh, int32_t l, int32_t first, int32_t p_row, int32_t k, const sbha_opts* opts,
               double* Z_out, double* evals_out, int32_t* idx_out, void* stream) {
  return guarded([&]() -> int {
    check_mesh_args(mesh);
    sbha_opts o = resolve(opts);
    int64_t n = mesh->n_vertices;
    if (l < 1 || l > n) SBHA_THROW(SBHA_EINVAL, "l must be in [1, n]");
    if (first < 0 || first >= n) SBHA_THROW(SBHA_EINVAL, "first landmark out of range");
    if (p_row < 1 || p_row > 64) SBHA_THROW(SBHA_EINVAL, "p_row must be in [1, 64]");
    if (k < 1 || !Z_out || !evals_out) SBHA_THROW(SBHA_EINVAL, "bad embed outputs");
    Ctx c(stream);
    c.timing = o.timing;
    bool timing = o.timing != 0;
    DevMesh m = stage_mesh(c, mesh);
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
    DevGraph g = build_graph(c, m);
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
      thread_error() = "subspace iteration reached eig_max_iter before eig_tol";
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

}  // extern "C"
