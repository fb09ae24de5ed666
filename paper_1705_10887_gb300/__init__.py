"""Python binding of the sBHA / sBMDS CUDA library (``libsbha.so``, C ABI in ``include/sbha.h``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
outputs are returned in the same kind of container as the mesh positions.  With
CUDA tensors the library works on the current torch stream.

Importing this package does not compile anything; ``build()`` (or
``__graft_entry__.build()``) produces ``libsbha.so``.  Every call fails loudly if the
library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH
from .build import build  # noqa: F401  (re-exported)

try:  # torch is optional for numpy callers
    import torch
except Exception:  # pragma: no cover
    torch = None

__all__ = [
    "SbhaError",
    "Opts",
    "Stats",
    "library",
    "opts_default",
    "landmarks",
    "geodesics",
    "landmark_distances",
    "operator",
    "operator_nnz",
    "mds",
    "embed",
    "last_stats",
    "version",
    "PREC_FP64",
    "PREC_FP32_REFINE",
    "PRECOND_JACOBI",
    "PRECOND_MLP",
    "SPARSIFY_ROWS",
    "SPARSIFY_COLS",
    "SOLVER_FACTORED",
    "SOLVER_DIRECT",
    "SPMM_AUTO",
    "SPMM_GATHER",
    "SPMM_STAGED",
    "SPMM_PIPELINED",
    "SPMM_TMA",
    "DENSE_AUTO",
    "DENSE_FP64",
    "DENSE_TC",
    "EIG_LANDMARK",
    "EIG_LANCZOS",
    "dgemm",
    "MLP_PARAMS",
    "MLP_FEATURES",
    "mlp_gradient",
    "precond_gradient",
    "embed_batch",
    "bha_error",
    "graph_operator",
    "graph_embed",
    "heat_geodesics",
    "fmds_operator",
    "mesh_graph",
    "biharmonic",
    "set_wait_limit",
    "FAULT_NONE",
    "FAULT_MLP_NAN",
]

PREC_FP64, PREC_FP32_REFINE = 0, 1
PRECOND_JACOBI, PRECOND_MLP = 0, 1
SPARSIFY_ROWS, SPARSIFY_COLS = 0, 1
SOLVER_FACTORED, SOLVER_DIRECT = 0, 1
SPMM_AUTO, SPMM_GATHER, SPMM_STAGED, SPMM_PIPELINED, SPMM_TMA = 0, 1, 2, 3, 4
DENSE_AUTO, DENSE_FP64, DENSE_TC = 0, 1, 2
EIG_LANDMARK, EIG_LANCZOS = 0, 1
FAULT_NONE, FAULT_MLP_NAN = 0, 1

STATUS = {0: "SBHA_OK", 1: "SBHA_EINVAL", 2: "SBHA_EDISCONNECTED", 3: "SBHA_ENOCONV", 4: "SBHA_ENOMEM",
          5: "SBHA_ECUDA", 6: "SBHA_ETIMEOUT", 7: "SBHA_ENOTIMPL"}


class SbhaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Mesh(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_faces", ctypes.c_int64), ("xyz", ctypes.c_void_p),
                ("faces", ctypes.c_void_p)]


class Graph(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("length", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("precond", ctypes.c_int32), ("sparsify_mode", ctypes.c_int32),
                ("chunk_cols", ctypes.c_int32), ("cg_rtol", ctypes.c_double), ("cg_max_iter", ctypes.c_int32),
                ("refine_max", ctypes.c_int32), ("inner_rtol", ctypes.c_double), ("oversample", ctypes.c_int32),
                ("eig_max_iter", ctypes.c_int32), ("eig_tol", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("timing", ctypes.c_int32), ("solver", ctypes.c_int32), ("mlp_epochs", ctypes.c_int32),
                ("spmm_variant", ctypes.c_int32), ("dense_mode", ctypes.c_int32), ("eig_route", ctypes.c_int32),
                ("spmm_chunk_rows", ctypes.c_int32), ("fault_inject", ctypes.c_int32),
                ("mlp_pilot_cols", ctypes.c_int32), ("spmm_pipeline_depth", ctypes.c_int32),
                ("cg_graph", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("cg_iterations", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("cg_max_rel_residual", ctypes.c_double), ("eig_iterations", ctypes.c_int32),
                ("eig_residual", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("ms_landmarks", ctypes.c_double), ("ms_geodesics", ctypes.c_double),
                ("ms_assembly", ctypes.c_double), ("ms_solve", ctypes.c_double), ("ms_sparsify", ctypes.c_double),
                ("ms_mds", ctypes.c_double), ("cg_kernel_launches", ctypes.c_int64 * 4),
                ("cg_kernel_ms", ctypes.c_double * 4), ("cg_kernel_bytes", ctypes.c_double * 4),
                ("unknowns", ctypes.c_int64), ("nnz_uu", ctypes.c_int64), ("chunk_cols", ctypes.c_int32),
                ("inner_bytes", ctypes.c_int32), ("mlp_trained", ctypes.c_int32), ("mlp_fallback", ctypes.c_int32),
                ("mlp_train_columns", ctypes.c_int32), ("e_iterations_jacobi", ctypes.c_int32),
                ("e_iterations_learned", ctypes.c_int32), ("heat_sweeps", ctypes.c_int32),
                ("mlp_train_entries", ctypes.c_int64), ("mlp_loss_first", ctypes.c_double),
                ("mlp_loss_last", ctypes.c_double), ("mlp_ms_pilot", ctypes.c_double),
                ("mlp_ms_train", ctypes.c_double), ("spmm_tiles", ctypes.c_int32), ("spmm_tiles_staged", ctypes.c_int32),
                ("spmm_halo_rows", ctypes.c_int64), ("e_iterations", ctypes.c_int32), ("k_iterations", ctypes.c_int32),
                ("correction_iterations", ctypes.c_int32), ("corrections", ctypes.c_int32),
                ("spmm_chunk_rows", ctypes.c_int32), ("spmm_tuned_shapes", ctypes.c_int32),
                ("spmm_tuned_us", ctypes.c_double), ("spmm_pipeline_depth", ctypes.c_int32),
                ("spmm_ctas_per_sm", ctypes.c_int32), ("ms_transpose", ctypes.c_double), ("ms_gram", ctypes.c_double),
                ("p_nnz", ctypes.c_int64), ("spmm_tma", ctypes.c_int32),
                ("spmm_gather_tiles_staged", ctypes.c_int32), ("spmm_gather_halo_rows", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


_lib = None

# (name, restype, argtypes) of every exported symbol declared in include/sbha.h
_I32, _I64, _VP, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
SIGNATURES = [
    ("sbha_opts_default", None, [ctypes.POINTER(Opts)]),
    ("sbha_last_stats", ctypes.c_int, [ctypes.POINTER(Stats)]),
    ("sbha_last_error", ctypes.c_char_p, []),
    ("sbha_version", ctypes.c_char_p, []),
    ("sbha_landmarks", ctypes.c_int, [ctypes.POINTER(Mesh), _I32, _I32, _VP, _VP, _VP]),
    ("sbha_geodesics", ctypes.c_int, [ctypes.POINTER(Mesh), _VP, _I32, _VP, _I32, _VP, _VP]),
    ("sbha_landmark_distances", ctypes.c_int, [ctypes.POINTER(Mesh), _VP, _I32, _VP, _VP]),
    ("sbha_mesh_graph", ctypes.c_int,
     [ctypes.POINTER(Mesh), _VP, _VP, _VP, _VP, _VP, _VP, _I64, ctypes.POINTER(_I64), _VP]),
    ("sbha_biharmonic", ctypes.c_int, [ctypes.POINTER(Mesh), _VP, _VP, _VP, _I64, ctypes.POINTER(_I64), _VP]),
    ("sbha_set_wait_limit", _I64, [_I64]),
    ("sbha_operator", ctypes.c_int,
     [ctypes.POINTER(Mesh), _VP, _I32, _I32, ctypes.POINTER(Opts), _VP, _VP, _VP, _I64, ctypes.POINTER(_I64), _VP]),
    ("sbha_mds", ctypes.c_int, [_I64, _I32, _VP, _VP, _VP, _VP, _I32, ctypes.POINTER(Opts), _VP, _VP, _VP]),
    ("sbha_mds_static", ctypes.c_int, [_I64, _I32, _VP, _VP, _VP, _VP, _I32, ctypes.POINTER(Opts), _VP, _VP, _VP]),
    ("sbha_mlp_gradient", ctypes.c_int, [_I64, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("sbha_precond_gradient", ctypes.c_int, [_I64, _VP, _VP, _VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("sbha_embed", ctypes.c_int,
     [ctypes.POINTER(Mesh), _I32, _I32, _I32, _I32, ctypes.POINTER(Opts), _VP, _VP, _VP, _VP]),
    ("sbha_dgemm", ctypes.c_int, [_I64, _I64, _I64, _VP, _VP, _VP, _I32, _VP]),
    ("sbha_embed_batch", ctypes.c_int,
     [_I32, ctypes.POINTER(Mesh), _VP, _VP, _I32, _I32, ctypes.POINTER(Opts), _VP, _VP, _VP, _I32, _VP]),
    ("sbha_bha_error", ctypes.c_int, [_I64, _I32, _VP, _VP, _VP, _VP, _I32, _VP, _VP, _I32, _VP, _VP, _VP]),
    ("sbha_fmds_operator", ctypes.c_int, [ctypes.POINTER(Mesh), _VP, _I32, ctypes.c_double, ctypes.POINTER(Opts),
                                           _VP, _VP]),
    ("sbha_heat_geodesics", ctypes.c_int, [ctypes.POINTER(Mesh), _VP, _I32, ctypes.c_double, ctypes.POINTER(Opts),
                                            _VP, _VP]),
    ("sbha_graph_operator", ctypes.c_int,
     [ctypes.POINTER(Graph), _VP, _I32, _I32, ctypes.POINTER(Opts), _VP, _VP, _VP, _I64, ctypes.POINTER(_I64), _VP]),
    ("sbha_graph_embed", ctypes.c_int,
     [ctypes.POINTER(Graph), _I32, _I32, _I32, _I32, ctypes.POINTER(Opts), _VP, _VP, _VP, _VP]),
]


def library():
    """The loaded ``libsbha.so`` (ctypes handle).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_1705_10887_gb300.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int):
    if status != 0:
        msg = library().sbha_last_error().decode()
        raise SbhaError(status, msg)


def version() -> str:
    return library().sbha_version().decode()


def opts_default(**overrides) -> Opts:
    o = Opts()
    library().sbha_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def last_stats() -> dict:
    s = Stats()
    library().sbha_last_stats(ctypes.byref(s))
    return s.as_dict()


# ------------------------------------------------------------ marshalling --

def _is_torch(a) -> bool:
    return torch is not None and isinstance(a, torch.Tensor)


class _Space:
    """Where outputs go: numpy (host) or torch on a given device."""

    def __init__(self, like):
        self.torch = _is_torch(like)
        self.device = like.device if self.torch else None

    def empty(self, shape, dtype):
        if self.torch:
            tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
            return torch.empty(shape, dtype=tdt, device=self.device)
        return np.empty(shape, dtype=dtype)

    def stream(self):
        if self.torch and self.device.type == "cuda":
            return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        return ctypes.c_void_p(0)


def _prep(a, dtype, space: _Space):
    """Contiguous array of the right dtype, in the caller's container kind; returns (keepalive, ptr)."""
    if a is None:
        return None, None
    if _is_torch(a):
        tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        t = a.to(dtype=tdt).contiguous()
        return t, ctypes.c_void_p(t.data_ptr())
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, ctypes.c_void_p(arr.ctypes.data)


def _ptr(a):
    if a is None:
        return None
    return ctypes.c_void_p(a.data_ptr() if _is_torch(a) else a.ctypes.data)


def _mesh(xyz, faces, space):
    kx, px = _prep(xyz, np.float64, space)
    kf, pf = _prep(faces, np.int32, space)
    n = kx.shape[0]
    f = kf.shape[0]
    return Mesh(n, f, px, pf), (kx, kf)


def _sync(space):
    # calls return with results complete; nothing to do, kept for clarity
    return None


# --------------------------------------------------------------- calls ----

def landmarks(xyz, faces, l: int, first: int = 0, return_mind: bool = False):
    """Farthest-point landmarks along mesh edges (Eq. 5).  Returns idx (and the min-distance field)."""
    space = _Space(xyz)
    m, keep = _mesh(xyz, faces, space)
    idx = space.empty((l,), np.int32)
    mind = space.empty((m.n_vertices,), np.float64) if return_mind else None
    _check(library().sbha_landmarks(ctypes.byref(m), l, first, _ptr(idx), _ptr(mind), space.stream()))
    return (idx, mind) if return_mind else idx


def geodesics(xyz, faces, src, tgt=None):
    """Mesh-edge shortest-path distances, shape (len(src), len(tgt) or n)."""
    space = _Space(xyz)
    m, keep = _mesh(xyz, faces, space)
    ks, ps = _prep(src, np.int32, space)
    kt, pt = _prep(tgt, np.int32, space)
    cols = kt.shape[0] if kt is not None else m.n_vertices
    D = space.empty((ks.shape[0], cols), np.float64)
    _check(library().sbha_geodesics(ctypes.byref(m), ps, ks.shape[0], pt, kt.shape[0] if kt is not None else 0,
                                    _ptr(D), space.stream()))
    return D


def landmark_distances(xyz, faces, idx):
    """Symmetrised landmark block W (Sec. 3), shape (l, l)."""
    space = _Space(xyz)
    m, keep = _mesh(xyz, faces, space)
    ki, pi = _prep(idx, np.int32, space)
    l = ki.shape[0]
    W = space.empty((l, l), np.float64)
    _check(library().sbha_landmark_distances(ctypes.byref(m), pi, l, _ptr(W), space.stream()))
    return W


def mesh_graph(xyz, faces):
    """Edge graph and the Sec. 2.2 quantities the operator uses: (rowptr, col, len, A, D, V)."""
    space = _Space(xyz)
    m, keep = _mesh(xyz, faces, space)
    nnz = ctypes.c_int64(0)
    _check(library().sbha_mesh_graph(ctypes.byref(m), None, None, None, None, None, None, 0, ctypes.byref(nnz),
                                     space.stream()))
    n, e = m.n_vertices, nnz.value
    rowptr, col = space.empty((n + 1,), np.int32), space.empty((e,), np.int32)
    ln, A = space.empty((e,), np.float64), space.empty((e,), np.float64)
    D, V = space.empty((n,), np.float64), space.empty((n,), np.float64)
    _check(library().sbha_mesh_graph(ctypes.byref(m), _ptr(rowptr), _ptr(col), _ptr(ln), _ptr(A), _ptr(D), _ptr(V), e,
                                     ctypes.byref(nnz), space.stream()))
    return rowptr, col, ln, A, D, V


def biharmonic(xyz, faces):
    """The biharmonic operator M = (V - A)^T D^{-1} (V - A) (Sec. 2.2) as CSR (rowptr, col, val)."""
    space = _Space(xyz)
    m, keep = _mesh(xyz, faces, space)
    nnz = ctypes.c_int64(0)
    _check(library().sbha_biharmonic(ctypes.byref(m), None, None, None, 0, ctypes.byref(nnz), space.stream()))
    e = nnz.value
    rowptr, col, val = space.empty((m.n_vertices + 1,), np.int32), space.empty((e,), np.int32), \
        space.empty((e,), np.float64)
    _check(library().sbha_biharmonic(ctypes.byref(m), _ptr(rowptr), _ptr(col), _ptr(val), e, ctypes.byref(nnz),
                                     space.stream()))
    return rowptr, col, val


def set_wait_limit(spins: int) -> int:
    """Iteration limit of the bounded device waits (< 0: default; 0: give up at once).  Returns the old one."""
    return int(library().sbha_set_wait_limit(int(spins)))


def operator_nnz(n: int, l: int, p_row: int, opts: Opts | None = None) -> int:
    o = opts if opts is not None else opts_default()
    nnz = ctypes.c_int64(0)
    m = Mesh(n, 1, None, None)
    _check(library().sbha_operator(ctypes.byref(m), ctypes.c_void_p(1), l, p_row, ctypes.byref(o), None, None, None,
                                   0, ctypes.byref(nnz), ctypes.c_void_p(0)))
    return nnz.value


def operator(xyz, faces, idx, p_row: int, opts: Opts | None = None, allow_noconv: bool = False):
    """Sparse interpolation operator (Eq. 6 thresholded by Eq. 8) as CSR (rowptr, col, val)."""
    space = _Space(xyz)
    m, keep = _mesh(xyz, faces, space)
    ki, pi = _prep(idx, np.int32, space)
    l = ki.shape[0]
    o = opts if opts is not None else opts_default()
    nnz = operator_nnz(m.n_vertices, l, p_row, o)
    rowptr = space.empty((m.n_vertices + 1,), np.int32)
    col = space.empty((nnz,), np.int32)
    val = space.empty((nnz,), np.float64)
    got = ctypes.c_int64(0)
    st = library().sbha_operator(ctypes.byref(m), pi, l, p_row, ctypes.byref(o), _ptr(rowptr), _ptr(col), _ptr(val),
                                 nnz, ctypes.byref(got), space.stream())
    if not (allow_noconv and st == 3):
        _check(st)
    return rowptr, col, val


def fmds_operator(xyz, faces, idx, mu: float = 50.0, opts: Opts | None = None):
    """The FMDS interpolation matrix H = P (M_bb + mu I + M_bu P_u)^{-1} mu (Sec. 3.4.2), shape (n, l)."""
    space = _Space(xyz)
    mesh, keep = _mesh(xyz, faces, space)
    ki, pi = _prep(idx, np.int32, space)
    o = opts if opts is not None else opts_default()
    H = space.empty((mesh.n_vertices, ki.shape[0]), np.float64)
    _check(library().sbha_fmds_operator(ctypes.byref(mesh), pi, ki.shape[0], float(mu), ctypes.byref(o), _ptr(H),
                                        space.stream()))
    return H


def heat_geodesics(xyz, faces, src, m: float = 1.0, opts: Opts | None = None):
    """Heat-method geodesic distances (Crane et al. 2013), shape (len(src), n)."""
    space = _Space(xyz)
    mesh, keep = _mesh(xyz, faces, space)
    ks, ps = _prep(src, np.int32, space)
    o = opts if opts is not None else opts_default()
    D = space.empty((ks.shape[0], mesh.n_vertices), np.float64)
    _check(library().sbha_heat_geodesics(ctypes.byref(mesh), ps, ks.shape[0], float(m), ctypes.byref(o), _ptr(D),
                                         space.stream()))
    return D


def _graph(rowptr, col, length, space):
    kr, pr = _prep(rowptr, np.int32, space)
    kc, pc = _prep(col, np.int32, space)
    kl, pl = _prep(length, np.float64, space)
    return Graph(kr.shape[0] - 1, pr, pc, pl), (kr, kc, kl)


def graph_operator(rowptr, col, idx, p_row: int, length=None, opts: Opts | None = None):
    """sbha_operator on a generic graph (D = I, 0/1 adjacency; CSR rowptr/col, optional edge lengths)."""
    space = _Space(rowptr)
    g, keep = _graph(rowptr, col, length, space)
    ki, pi = _prep(idx, np.int32, space)
    l = ki.shape[0]
    o = opts if opts is not None else opts_default()
    nnz = operator_nnz(g.n_vertices, l, p_row, o)
    rp = space.empty((g.n_vertices + 1,), np.int32)
    cl = space.empty((nnz,), np.int32)
    vl = space.empty((nnz,), np.float64)
    got = ctypes.c_int64(0)
    _check(library().sbha_graph_operator(ctypes.byref(g), pi, l, p_row, ctypes.byref(o), _ptr(rp), _ptr(cl), _ptr(vl),
                                         nnz, ctypes.byref(got), space.stream()))
    return rp, cl, vl


def graph_embed(rowptr, col, l: int, p_row: int, k: int = 3, first: int = 0, length=None, opts: Opts | None = None):
    """sbha_embed on a generic graph.  Returns (Z (n, k), evals (k,), idx (l,))."""
    space = _Space(rowptr)
    g, keep = _graph(rowptr, col, length, space)
    o = opts if opts is not None else opts_default()
    Z = space.empty((g.n_vertices, k), np.float64)
    ev = space.empty((k,), np.float64)
    idx = space.empty((l,), np.int32)
    _check(library().sbha_graph_embed(ctypes.byref(g), l, first, p_row, k, ctypes.byref(o), _ptr(Z), _ptr(ev),
                                      _ptr(idx), space.stream()))
    return Z, ev, idx


def bha_error(rowptr, col, val, W, rows, K_rows, squared: bool = False):
    """Sampled relative error of K~ = P W P^T (Sec. 4.1).  K_rows[i] is the exact row rows[i] of K.
    Returns (num, den) with eps ~= num / den (squared: compare K.K with P (W.W) P^T)."""
    space = _Space(W)
    kr, pr = _prep(rowptr, np.int32, space)
    kc, pc = _prep(col, np.int32, space)
    kv, pv = _prep(val, np.float64, space)
    kw, pw = _prep(W, np.float64, space)
    ks, ps = _prep(rows, np.int32, space)
    kk, pk = _prep(K_rows, np.float64, space)
    n, l, ns = kr.shape[0] - 1, kw.shape[0], ks.shape[0]
    num, den = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(library().sbha_bha_error(n, l, pr, pc, pv, pw, ns, ps, pk, int(bool(squared)), ctypes.byref(num),
                                    ctypes.byref(den), space.stream()))
    return num.value, den.value


def mds(n: int, rowptr, col, val, W, k: int, opts: Opts | None = None):
    """Low-rank classical scaling (Sec. 3.3).  Returns (Z (n, k), evals (k,))."""
    space = _Space(W)
    kr, pr = _prep(rowptr, np.int32, space)
    kc, pc = _prep(col, np.int32, space)
    kv, pv = _prep(val, np.float64, space)
    kw, pw = _prep(W, np.float64, space)
    l = kw.shape[0]
    o = opts if opts is not None else opts_default()
    Z = space.empty((n, k), np.float64)
    ev = space.empty((k,), np.float64)
    _check(library().sbha_mds(n, l, pr, pc, pv, pw, k, ctypes.byref(o), _ptr(Z), _ptr(ev), space.stream()))
    return Z, ev


MLP_PARAMS, MLP_FEATURES = 4673, 6


def mlp_gradient(X, T, params):
    """Loss and gradient of the warm-start network (FP32 arrays: X (N, 6), T (N,), params (4673,))."""
    space = _Space(X)
    kx, px = _prep_f32(X)
    kt, pt = _prep_f32(T)
    kp, pp = _prep_f32(params)
    if _is_torch(kx):
        grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=kx.device)
        loss = torch.empty(1, dtype=torch.float64, device=kx.device)
    else:
        grad = np.empty(MLP_PARAMS, np.float32)
        loss = np.empty(1, np.float64)
    _check(library().sbha_mlp_gradient(kx.shape[0], px, pt, pp, _ptr(grad), _ptr(loss), space.stream()))
    return float(loss[0]), grad


def precond_gradient(rowptr, col, val, B, params, X=None):
    """Training loss and gradient of the learned preconditioner (M^{-1} = G^T G on the pattern of
    the CSR matrix (rowptr, col, val)) for the right-hand sides B (m, ncols) and, optionally, the
    paired solutions X (m, ncols)."""
    space = _Space(B)
    kr, pr = _prep(rowptr, np.int32, space)
    kc, pc = _prep(col, np.int32, space)
    kv, pv = _prep(val, np.float64, space)
    kb, pb = _prep(B, np.float64, space)
    kx, px = _prep(X, np.float64, space)
    kp, pp = _prep_f32(params)
    m, ncols = kb.shape
    if _is_torch(kb):
        grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=kb.device)
        loss = torch.empty(1, dtype=torch.float64, device=kb.device)
    else:
        grad = np.empty(MLP_PARAMS, np.float32)
        loss = np.empty(1, np.float64)
    _check(library().sbha_precond_gradient(m, pr, pc, pv, ncols, pb, px, pp, _ptr(grad), _ptr(loss), space.stream()))
    return float(loss[0]), grad


def _prep_f32(a):
    if _is_torch(a):
        t = a.to(dtype=torch.float32).contiguous()
        return t, ctypes.c_void_p(t.data_ptr())
    arr = np.ascontiguousarray(a, dtype=np.float32)
    return arr, ctypes.c_void_p(arr.ctypes.data)


def dgemm(A, B, mode: int = 0):
    """C = A @ B (FP64) by the operator's landmark-space product engine (DENSE_TC or DENSE_FP64)."""
    space = _Space(A)
    ka, pa = _prep(A, np.float64, space)
    kb, pb = _prep(B, np.float64, space)
    M, K = ka.shape
    K2, N = kb.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    C = space.empty((M, N), np.float64)
    _check(library().sbha_dgemm(M, N, K, pa, pb, _ptr(C), mode, space.stream()))
    return C


def embed_batch(meshes, l, p_row: int, k: int = 3, first=None, opts: Opts | None = None, workers: int = 0):
    """The whole pipeline for a list of (xyz, faces) meshes.  Returns a list of (Z, evals, idx)."""
    count = len(meshes)
    if count == 0:
        return []
    space = _Space(meshes[0][0])
    keep, structs = [], (Mesh * count)()
    for i, (xyz, faces) in enumerate(meshes):
        m, kp = _mesh(xyz, faces, space)
        keep.append(kp)
        structs[i] = m
    ls = np.ascontiguousarray(l, dtype=np.int32)
    fs = None if first is None else np.ascontiguousarray(first, dtype=np.int32)
    outs = []
    zp, ep, ip = (ctypes.c_void_p * count)(), (ctypes.c_void_p * count)(), (ctypes.c_void_p * count)()
    for i, (xyz, _) in enumerate(meshes):
        n = int(xyz.shape[0])
        Z = space.empty((n, k), np.float64)
        ev = space.empty((k,), np.float64)
        idx = space.empty((int(ls[i]),), np.int32)
        outs.append((Z, ev, idx))
        zp[i], ep[i], ip[i] = _ptr(Z).value, _ptr(ev).value, _ptr(idx).value
    o = opts if opts is not None else opts_default()
    _check(library().sbha_embed_batch(count, structs, ctypes.c_void_p(ls.ctypes.data),
                                      None if fs is None else ctypes.c_void_p(fs.ctypes.data), p_row, k,
                                      ctypes.byref(o), zp, ep, ip, workers, space.stream()))
    return outs


def embed(xyz, faces, l: int, p_row: int, k: int = 3, first: int = 0, opts: Opts | None = None):
    """Whole sBMDS pipeline.  Returns (Z (n, k), evals (k,), idx (l,))."""
    space = _Space(xyz)
    m, keep = _mesh(xyz, faces, space)
    o = opts if opts is not None else opts_default()
    Z = space.empty((m.n_vertices, k), np.float64)
    ev = space.empty((k,), np.float64)
    idx = space.empty((l,), np.int32)
    _check(library().sbha_embed(ctypes.byref(m), l, first, p_row, k, ctypes.byref(o), _ptr(Z), _ptr(ev), _ptr(idx),
                                space.stream()))
    return Z, ev, idx
