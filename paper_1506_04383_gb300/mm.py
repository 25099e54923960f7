"""Thin Python binding of the libmm.so C-ABI (include/mm.h).

Argument marshalling only: every step of the layout runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current stream.  The
binding fails loudly when the library has not been built or no GPU is
visible; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmm.so")

MM_OK = 0
STATUS = {0: "MM_OK", 1: "MM_ERR_INVALID_ARG", 2: "MM_ERR_NOT_CONNECTED", 3: "MM_ERR_CUDA",
          4: "MM_ERR_OOM", 5: "MM_ERR_NONFINITE", 6: "MM_ERR_TIMEOUT", 7: "MM_ERR_UNSUPPORTED"}
MM_PARAMS_VERSION = 1
MM_MAX_LEVELS = 64

# every symbol include/mm.h declares
EXPORTS = ["mm_default_params", "mm_status_string", "mm_last_error", "mm_build_hierarchy",
           "mm_build_hierarchy_levels",
           "mm_free_hierarchy", "mm_hierarchy_levels", "mm_level_info", "mm_level_export",
           "mm_sweep", "mm_repulsion", "mm_layout", "mm_sweep_profile", "mm_objective",
           "mm_khop", "mm_cluster",
           "mm_contract", "mm_prolong", "mm_layout_host", "mm_repulsion_noalloc",
           "mm_autotune", "mm_gemm_bf16", "mm_net_create", "mm_net_free", "mm_net_params",
           "mm_net_forward", "mm_net_gradients", "mm_net_train_step", "mm_hierarchy_set_net",
           "mm_layout_levels", "mm_repulsion_h", "mm_full_stress",
           "mm_selftest_wait_timeout", "mm_measure_fp32_peak", "mm_gemm_bf16_tn",
           "mm_net_gemm_profile", "mm_objective_bh"]
MM_NET_PARAMS = 17860


class MMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("struct_version", ctypes.c_uint32), ("k", ctypes.c_int32), ("theta", ctypes.c_float),
        ("exact_repulsion", ctypes.c_int32), ("coarsest_n", ctypes.c_int32),
        ("f", ctypes.c_float), ("b", ctypes.c_float), ("lp_rounds", ctypes.c_int32),
        ("iters_per_alpha", ctypes.c_int32), ("alpha0", ctypes.c_double),
        ("alpha_factor", ctypes.c_double), ("alpha_min", ctypes.c_double),
        ("eps", ctypes.c_double), ("eps_final", ctypes.c_double),
        ("max_iters_at_min", ctypes.c_int32), ("early_exit", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("max_levels", ctypes.c_int32),
        ("max_stalls", ctypes.c_int32), ("gather_lanes", ctypes.c_int32),
        ("heavy_degree", ctypes.c_int32), ("traverse_warps", ctypes.c_int32),
        ("fused_max_n", ctypes.c_int32), ("learned_prolong", ctypes.c_int32),
        ("leaf_size", ctypes.c_int32), ("bh_group", ctypes.c_int32),
        ("approx_levels", ctypes.c_int32), ("level_order", ctypes.c_int32),
        ("exact_max_n", ctypes.c_int32),
    ]


class Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("edge_len", ctypes.c_void_p),
                ("num_graphs", ctypes.c_int32), ("graph_ptr", ctypes.c_void_p)]


class LevelDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("omega", ctypes.c_void_p), ("node_c", ctypes.c_void_p),
                ("map", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("gather_lanes", ctypes.c_int32 * MM_MAX_LEVELS),
                ("traverse_warps", ctypes.c_int32 * MM_MAX_LEVELS),
                ("theta", ctypes.c_float), ("objective_ref", ctypes.c_double),
                ("objective", ctypes.c_double), ("layout_ms_before", ctypes.c_double),
                ("layout_ms_after", ctypes.c_double)]


class ProlongSample(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("map", ctypes.c_void_p), ("n_coarse", ctypes.c_int32),
                ("crow_ptr", ctypes.c_void_p), ("ccol", ctypes.c_void_p),
                ("c_coarse", ctypes.c_void_p), ("x_coarse", ctypes.c_void_p),
                ("seed", ctypes.c_uint64), ("level", ctypes.c_int32),
                ("x_target", ctypes.c_void_p)]


class LayoutStats(ctypes.Structure):
    _fields_ = [("num_levels", ctypes.c_int32), ("total_sweeps", ctypes.c_int32),
                ("vertex_updates", ctypes.c_int64),
                ("level_n", ctypes.c_int32 * MM_MAX_LEVELS),
                ("level_sweeps", ctypes.c_int32 * MM_MAX_LEVELS),
                ("final_alpha", ctypes.c_double), ("final_rel_change", ctypes.c_double),
                ("final_stress", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("level_rel_change", ctypes.c_float * MM_MAX_LEVELS)]

    def as_dict(self):
        nl = self.num_levels
        return dict(num_levels=nl, total_sweeps=self.total_sweeps,
                    vertex_updates=int(self.vertex_updates),
                    level_n=list(self.level_n[:nl]), level_sweeps=list(self.level_sweeps[:nl]),
                    final_alpha=self.final_alpha, final_rel_change=self.final_rel_change,
                    final_stress=self.final_stress, kernel_launches=int(self.kernel_launches),
                    level_rel_change=[float(v) for v in self.level_rel_change[:nl]])


_lib = None


def load(path: str = LIB_PATH):
    """Loads libmm.so; raises if it is missing (build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1506_04383_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, i32, i64, u64, f32, f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_uint64, ctypes.c_float, ctypes.c_double)
    lib.mm_default_params.argtypes = [P]
    lib.mm_default_params.restype = None
    lib.mm_status_string.argtypes = [i32]
    lib.mm_status_string.restype = ctypes.c_char_p
    lib.mm_last_error.argtypes = []
    lib.mm_last_error.restype = ctypes.c_char_p
    lib.mm_build_hierarchy.argtypes = [P, P, P, P]
    lib.mm_build_hierarchy_levels.argtypes = [i32, P, P, P, P, P]
    lib.mm_free_hierarchy.argtypes = [P]
    lib.mm_free_hierarchy.restype = None
    lib.mm_hierarchy_levels.argtypes = [P, P]
    lib.mm_level_info.argtypes = [P, i32, P, P, P]
    lib.mm_level_export.argtypes = [P, i32, P, P, P, P, P, P, P, P, P, P]
    lib.mm_sweep.argtypes = [P, i32, f64, P, P, P, P]
    lib.mm_repulsion.argtypes = [P, i32, P, f32, P, P]
    lib.mm_layout.argtypes = [P, P, P, P, P, P]
    lib.mm_sweep_profile.argtypes = [P, i32, P, i32, P, P, P]
    lib.mm_objective.argtypes = [P, i32, P, f64, P, P, P, P]
    lib.mm_khop.argtypes = [i32, P, P, P, P, i32, P, P, P, P, P, P]
    lib.mm_cluster.argtypes = [i32, P, P, P, P, f32, i32, u64, i32, P, P]
    lib.mm_contract.argtypes = [i32, P, P, P, P, P, P, P, P, P, P, P, P, P]
    lib.mm_prolong.argtypes = [i32, P, P, P, u64, i32, P, P]
    lib.mm_layout_host.argtypes = [i32, P, P, P, P, P, P, P]
    lib.mm_repulsion_noalloc.argtypes = [i32, P, f32, P, P]
    lib.mm_autotune.argtypes = [P, P, i32, f64, P, P]
    lib.mm_gemm_bf16.argtypes = [i32, i32, i32, P, P, P, i32, P, P, P]
    lib.mm_net_create.argtypes = [P, P]
    lib.mm_net_free.argtypes = [P]
    lib.mm_net_free.restype = None
    lib.mm_net_params.argtypes = [P, P, P]
    lib.mm_net_forward.argtypes = [P, P, P, P, P]
    lib.mm_net_gradients.argtypes = [P, P, P, P, P]
    lib.mm_net_train_step.argtypes = [P, P, f32, P, P]
    lib.mm_hierarchy_set_net.argtypes = [P, P]
    lib.mm_layout_levels.argtypes = [P, P, P, P]
    lib.mm_repulsion_h.argtypes = [P, i32, P, P, P]
    lib.mm_full_stress.argtypes = [P, P, P, P]
    lib.mm_selftest_wait_timeout.argtypes = [i32, P]
    lib.mm_measure_fp32_peak.argtypes = [i32, P, P, P]
    lib.mm_gemm_bf16_tn.argtypes = [i32, i32, P, P, P, P]
    lib.mm_net_gemm_profile.argtypes = [i32, i32, P, P]
    lib.mm_objective_bh.argtypes = [P, i32, P, f64, f32, P, P, P, P]
    for name in EXPORTS:
        fn = getattr(lib, name)
        if name not in ("mm_default_params", "mm_free_hierarchy", "mm_status_string",
                        "mm_last_error", "mm_net_free"):
            fn.restype = i32
    _lib = lib
    return lib


def _check(status):
    if status != MM_OK:
        msg = load().mm_last_error().decode(errors="replace")
        raise MMError(status, msg)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def default_params(**kw) -> Params:
    p = Params()
    load().mm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device visible: libmm has no CPU fallback")


class Hierarchy:
    """Owns an mm_hierarchy (freed on deletion)."""

    def __init__(self, handle, n):
        self.handle = handle
        self.n = n

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mm_free_hierarchy(self.handle)
            self.handle = None

    def levels(self) -> int:
        v = ctypes.c_int32()
        _check(load().mm_hierarchy_levels(self.handle, ctypes.byref(v)))
        return v.value

    def level_info(self, level):
        n, e, s = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().mm_level_info(self.handle, level, ctypes.byref(n), ctypes.byref(e),
                                    ctypes.byref(s)))
        return n.value, e.value, s.value


def build_hierarchy(row_ptr, col, params: Params = None, edge_len=None, graph_ptr=None,
                    stream=None):
    """row_ptr int64 [n+1] and col int32 [nnz] CUDA tensors (symmetric CSR).

    graph_ptr (host int32 [G+1] vertex offsets) lays out a block-diagonal
    batch of G independent graphs; graph i uses seed + i."""
    _require_cuda()
    lib = load()
    row_ptr = _dev(row_ptr, torch.int64, "row_ptr")
    col = _dev(col, torch.int32, "col")
    edge_len = _dev(edge_len, torch.float32, "edge_len")
    p = params if params is not None else default_params()
    gp = None
    if graph_ptr is not None:
        gp = np.ascontiguousarray(graph_ptr, dtype=np.int32)
    g = Graph(n=row_ptr.numel() - 1, nnz=col.numel(), row_ptr=row_ptr.data_ptr(),
              col=col.data_ptr() if col.numel() else None,
              edge_len=edge_len.data_ptr() if edge_len is not None else None,
              num_graphs=1 if gp is None else len(gp) - 1,
              graph_ptr=gp.ctypes.data if gp is not None else None)
    h = ctypes.c_void_p()
    _check(lib.mm_build_hierarchy(ctypes.byref(g), ctypes.byref(p), _stream(stream),
                                  ctypes.byref(h)))
    return Hierarchy(h, g.n)


def build_hierarchy_levels(levels, params: Params = None, edge_len0=None, stream=None):
    """Hierarchy from caller-supplied levels: a list of dicts with CUDA
    tensors row_ptr (int64), col (int32), optional omega / c (float32) and
    map (int32, all but the last level)."""
    _require_cuda()
    keep = []
    descs = (LevelDesc * len(levels))()
    for i, L in enumerate(levels):
        rp = _dev(L["row_ptr"], torch.int64, "row_ptr")
        col = _dev(L["col"], torch.int32, "col")
        om = _dev(L.get("omega"), torch.float32, "omega")
        c = _dev(L.get("c"), torch.float32, "c")
        mp = _dev(L.get("map"), torch.int32, "map")
        keep += [rp, col, om, c, mp]
        descs[i] = LevelDesc(n=rp.numel() - 1, nnz=col.numel(), row_ptr=rp.data_ptr(),
                             col=col.data_ptr() if col.numel() else None,
                             omega=om.data_ptr() if om is not None else None,
                             node_c=c.data_ptr() if c is not None else None,
                             map=mp.data_ptr() if mp is not None else None)
    el = _dev(edge_len0, torch.float32, "edge_len0")
    p = params if params is not None else default_params()
    h = ctypes.c_void_p()
    _check(load().mm_build_hierarchy_levels(len(levels), descs, _ptr(el), ctypes.byref(p),
                                            _stream(stream), ctypes.byref(h)))
    return Hierarchy(h, descs[0].n)


def level_export(h: Hierarchy, level: int, stream=None):
    n, nnzE, nnzS = h.level_info(level)
    dev = torch.device("cuda")
    out = dict(
        row_ptr=torch.empty(n + 1, dtype=torch.int64, device=dev),
        col=torch.empty(nnzE, dtype=torch.int32, device=dev),
        omega=torch.empty(nnzE, dtype=torch.float32, device=dev),
        c=torch.empty(n, dtype=torch.float32, device=dev),
        map=torch.full((n,), -1, dtype=torch.int32, device=dev),
        s_ptr=torch.empty(n + 1, dtype=torch.int64, device=dev),
        s_col=torch.empty(nnzS, dtype=torch.int32, device=dev),
        s_d=torch.empty(nnzS, dtype=torch.float32, device=dev),
        rho=torch.empty(n, dtype=torch.float32, device=dev),
    )
    _check(load().mm_level_export(h.handle, level, *[_ptr(out[k]) if out[k].numel() else None
                                                     for k in ("row_ptr", "col", "omega", "c",
                                                               "map", "s_ptr", "s_col", "s_d",
                                                               "rho")], _stream(stream)))
    torch.cuda.current_stream().synchronize()
    return out


def sweep(h: Hierarchy, level: int, alpha: float, x_in, x_out=None, stats=True, stream=None):
    """One Eq. 2 iteration; returns (x_out, [sum|dx|^2, sum|x|^2, stress] or None)."""
    x_in = _dev(x_in, torch.float32, "x_in")
    if x_out is None:
        x_out = torch.empty_like(x_in)
    st = (ctypes.c_double * 3)() if stats else None
    _check(load().mm_sweep(h.handle, level, float(alpha), _ptr(x_in), _ptr(x_out), st,
                           _stream(stream)))
    return x_out, (list(st) if stats else None)


def repulsion(h: Hierarchy, level: int, x, theta: float, stream=None):
    """F_u = sum_{v != u} r(u,v): theta > 0 Barnes-Hut, 0 tree-exact, < 0 tiled exact."""
    x = _dev(x, torch.float32, "x")
    F = torch.empty_like(x)
    _check(load().mm_repulsion(h.handle, level, _ptr(x), float(theta), _ptr(F), _stream(stream)))
    return F


def repulsion_h(h: Hierarchy, level: int, x, stream=None):
    """The first two sums of Eq. 3 (MulMent_h) on `level` (hierarchy built
    with approx_levels > 0)."""
    x = _dev(x, torch.float32, "x")
    F = torch.empty_like(x)
    _check(load().mm_repulsion_h(h.handle, level, _ptr(x), _ptr(F), _stream(stream)))
    return F


def full_stress(h: Hierarchy, x, stream=None):
    """Full stress F(x), optimal scale s, F(s x) and the number of pairs for a
    layout of the input graph (Sec. 4)."""
    x = _dev(x, torch.float32, "x")
    out = (ctypes.c_double * 4)()
    _check(load().mm_full_stress(h.handle, _ptr(x), out, _stream(stream)))
    return float(out[0]), float(out[1]), float(out[2]), int(out[3])


def repulsion_noalloc(x, theta: float, F_out=None, stream=None):
    """Barnes-Hut F for up to 32768 points with the library's fixed static
    scratch (the call allocates no device memory itself; the output buffer
    is the caller's).  x is a contiguous float32 [n, 2] CUDA tensor; F_out,
    if given, a float32 [n, 2] CUDA tensor on the same device.  The call runs
    on x's device.  Calls that overlap on the GPU race on the shared
    scratch."""
    _require_cuda()
    x = _dev(x, torch.float32, "x")
    if x.dim() != 2 or x.shape[1] != 2:
        raise ValueError(f"x must have shape [n, 2], got {tuple(x.shape)}")
    if F_out is None:
        F_out = torch.empty_like(x)
    F_out = _dev(F_out, torch.float32, "F_out")
    if F_out.shape != x.shape:
        raise ValueError(f"F_out must have shape {tuple(x.shape)}, got {tuple(F_out.shape)}")
    if F_out.device != x.device:
        raise ValueError(f"F_out is on {F_out.device}, x on {x.device}")
    with torch.cuda.device(x.device):
        _check(load().mm_repulsion_noalloc(x.shape[0], _ptr(x), float(theta), _ptr(F_out),
                                           _stream(stream)))
    return F_out


def measure_fp32_peak(reps: int = 20, stream=None):
    """Measured FP32 FMA throughput of the current device: (TFLOP/s, ms per
    launch)."""
    _require_cuda()
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().mm_measure_fp32_peak(int(reps), ctypes.byref(t), ctypes.byref(ms),
                                       _stream(stream)))
    return t.value, ms.value


def selftest_wait_timeout(spin_limit: int = 4096, stream=None) -> int:
    """Runs the library's self-test of its bounded device waits: a look-back
    wait on a status word that nothing writes must give up after spin_limit
    polls.  Returns the raw status (MM_ERR_TIMEOUT = the wait gave up, as
    intended; MM_OK = it did not)."""
    _require_cuda()
    return int(load().mm_selftest_wait_timeout(int(spin_limit), _stream(stream)))


def layout(h: Hierarchy, params: Params = None, x_init=None, x_out=None, stream=None):
    """Multilevel layout (or single-level schedule from x_init); returns (x, stats)."""
    x_init = _dev(x_init, torch.float32, "x_init")
    if x_out is None:
        x_out = torch.empty((h.n, 2), dtype=torch.float32, device="cuda")
    st = LayoutStats()
    _check(load().mm_layout(h.handle, ctypes.byref(params) if params is not None else None,
                            _ptr(x_init), _ptr(x_out), ctypes.byref(st), _stream(stream)))
    return x_out, st.as_dict()


STAGES = ["bbox", "morton_hist", "sort", "radix_tree_scan", "records", "traverse", "gather",
          "controller"]


def sweep_profile(h: Hierarchy, level: int, x, reps: int = 10, stream=None):
    """Mean ms per sweep stage (CUDA events) and the walk's work counters."""
    x = _dev(x, torch.float32, "x")
    ms = (ctypes.c_double * 8)()
    work = (ctypes.c_int64 * 4)()
    _check(load().mm_sweep_profile(h.handle, level, _ptr(x), int(reps), ms, work,
                                   _stream(stream)))
    return dict(stage_names=list(STAGES), stage_ms=list(ms), visits=int(work[0]),
                interactions=int(work[1]), nnz_S=int(work[2]), n=int(work[3]))


def autotune(h: Hierarchy, thetas=None, max_rel_drift: float = 0.01, stream=None):
    """Tunes lanes per S row and walk block shape per level, then theta under
    an objective drift bound; returns the choices and before/after times."""
    r = TuneResult()
    th = None
    if thetas is not None:
        th = np.ascontiguousarray(thetas, dtype=np.float32)
    _check(load().mm_autotune(h.handle, th.ctypes.data if th is not None else None,
                              0 if th is None else len(th), float(max_rel_drift),
                              ctypes.byref(r), _stream(stream)))
    nl = h.levels()
    return dict(gather_lanes=list(r.gather_lanes[:nl]), traverse_warps=list(r.traverse_warps[:nl]),
                theta=r.theta, objective_ref=r.objective_ref, objective=r.objective,
                layout_ms_before=r.layout_ms_before, layout_ms_after=r.layout_ms_after)


def gemm_bf16(A, B, bias=None, relu=False, out_bf16=False, stream=None):
    """C = A @ B^T on the tcgen05 tensor cores (BF16 in, FP32 accumulate).

    A [M, K] and B [N, K] bfloat16 CUDA tensors; returns FP32 [M, N] (and the
    BF16 copy when out_bf16)."""
    A = _dev(A, torch.bfloat16, "A")
    B = _dev(B, torch.bfloat16, "B")
    bias = _dev(bias, torch.float32, "bias")
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    Cb = torch.empty((M, N), dtype=torch.bfloat16, device="cuda") if out_bf16 else None
    _check(load().mm_gemm_bf16(M, N, K, _ptr(A), _ptr(B), _ptr(bias), int(relu), _ptr(C),
                               _ptr(Cb), _stream(stream)))
    return (C, Cb) if out_bf16 else C


def objective_bh(h: Hierarchy, level: int, x, alpha: float, theta: float, stream=None):
    """Eq. 1 with the ln-sum from Barnes-Hut log potentials at theta;
    returns (stress, ln-sum outside S, M)."""
    x = _dev(x, torch.float32, "x")
    st, ln, M = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().mm_objective_bh(h.handle, level, _ptr(x), float(alpha), float(theta),
                                  ctypes.byref(st), ctypes.byref(ln), ctypes.byref(M),
                                  _stream(stream)))
    return st.value, ln.value, M.value


def gemm_bf16_tn(A, B, stream=None):
    """out = A^T B on the tensor cores: A BF16 [n x R] (R = 16 or 128), B BF16
    [n x 64]; returns FP32 [R x 64]."""
    A = _dev(A, torch.bfloat16, "A")
    B = _dev(B, torch.bfloat16, "B")
    if A.dim() != 2 or B.dim() != 2 or A.shape[0] != B.shape[0] or B.shape[1] != 64:
        raise ValueError("need A [n x R] and B [n x 64]")
    out = torch.empty((A.shape[1], 64), dtype=torch.float32, device=A.device)
    _check(load().mm_gemm_bf16_tn(A.shape[0], A.shape[1], _ptr(A), _ptr(B), _ptr(out),
                                  _stream(stream)))
    return out


def net_gemm_profile(n: int, reps: int = 20, stream=None):
    """ms per launch of the layer product [n x 128] x [128 x 64] and of the
    weight-gradient partials [n x 128]^T x [n x 64] on the tensor cores."""
    _require_cuda()
    ms = (ctypes.c_double * 2)()
    _check(load().mm_net_gemm_profile(int(n), int(reps), ms, _stream(stream)))
    return float(ms[0]), float(ms[1])


def objective(h: Hierarchy, level: int, x, alpha: float, stream=None):
    """Eq. 1 over S (exact, all pairs): returns (stress, lnsum, M)."""
    x = _dev(x, torch.float32, "x")
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().mm_objective(h.handle, level, _ptr(x), float(alpha), ctypes.byref(a),
                               ctypes.byref(b), ctypes.byref(c), _stream(stream)))
    return a.value, b.value, c.value


def khop(row_ptr, col, k: int, edge_len=None, node_c=None, stream=None):
    """Pair set S of any graph; returns (s_ptr int64, s_col int32, s_d f32, rho f32)."""
    _require_cuda()
    lib = load()
    row_ptr = _dev(row_ptr, torch.int64, "row_ptr")
    col = _dev(col, torch.int32, "col")
    edge_len = _dev(edge_len, torch.float32, "edge_len")
    node_c = _dev(node_c, torch.float32, "node_c")
    n = row_ptr.numel() - 1
    sp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    nnz = ctypes.c_int64()
    args = (n, _ptr(row_ptr), _ptr(col) if col.numel() else None, _ptr(edge_len), _ptr(node_c),
            int(k), _ptr(sp), ctypes.byref(nnz))
    _check(lib.mm_khop(*args, None, None, None, _stream(stream)))
    m = nnz.value
    scol = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
    sd = torch.empty(max(m, 1), dtype=torch.float32, device="cuda")
    rho = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(lib.mm_khop(*args, _ptr(scol), _ptr(sd), _ptr(rho), _stream(stream)))
    return sp, scol[:m], sd[:m], rho


def cluster(row_ptr, col, omega, node_c, U: float, rounds: int, seed: int, level: int,
            stream=None):
    _require_cuda()
    row_ptr = _dev(row_ptr, torch.int64, "row_ptr")
    col = _dev(col, torch.int32, "col")
    omega = _dev(omega, torch.float32, "omega")
    node_c = _dev(node_c, torch.float32, "node_c")
    n = row_ptr.numel() - 1
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(load().mm_cluster(n, _ptr(row_ptr), _ptr(col), _ptr(omega), _ptr(node_c), float(U),
                             int(rounds), int(seed), int(level), _ptr(labels), _stream(stream)))
    return labels


def contract(row_ptr, col, omega, node_c, labels, stream=None):
    """Returns (map, c', row_ptr', col', omega')."""
    _require_cuda()
    row_ptr = _dev(row_ptr, torch.int64, "row_ptr")
    col = _dev(col, torch.int32, "col")
    omega = _dev(omega, torch.float32, "omega")
    node_c = _dev(node_c, torch.float32, "node_c")
    labels = _dev(labels, torch.int32, "labels")
    n = row_ptr.numel() - 1
    nnz = col.numel()
    mp = torch.empty(n, dtype=torch.int32, device="cuda")
    cc = torch.empty(n, dtype=torch.float32, device="cuda")
    crp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    ccol = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    cw = torch.empty(max(nnz, 1), dtype=torch.float32, device="cuda")
    nc, m = ctypes.c_int32(), ctypes.c_int64()
    _check(load().mm_contract(n, _ptr(row_ptr), _ptr(col), _ptr(omega), _ptr(node_c),
                              _ptr(labels), _ptr(mp), _ptr(cc), _ptr(crp), _ptr(ccol), _ptr(cw),
                              ctypes.byref(nc), ctypes.byref(m), _stream(stream)))
    nc, m = nc.value, m.value
    return mp, cc[:nc], crp[:nc + 1], ccol[:m], cw[:m]


def prolong(mp, x_coarse, c_coarse, seed: int, level: int, stream=None):
    _require_cuda()
    mp = _dev(mp, torch.int32, "map")
    x_coarse = _dev(x_coarse, torch.float32, "x_coarse")
    c_coarse = _dev(c_coarse, torch.float32, "c_coarse")
    xf = torch.empty((mp.numel(), 2), dtype=torch.float32, device="cuda")
    _check(load().mm_prolong(mp.numel(), _ptr(mp), _ptr(x_coarse), _ptr(c_coarse), int(seed),
                             int(level), _ptr(xf), _stream(stream)))
    return xf


def layout_host(row_ptr, col, params: Params = None, edge_len=None, stream=None):
    """One-call API over host numpy buffers; returns (x numpy [n,2], stats)."""
    _require_cuda()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    el = None if edge_len is None else np.ascontiguousarray(edge_len, dtype=np.float32)
    n = len(rp) - 1
    x = np.empty((n, 2), dtype=np.float32)
    st = LayoutStats()
    p = params if params is not None else default_params()
    _check(load().mm_layout_host(n, rp.ctypes.data_as(ctypes.c_void_p),
                                 cl.ctypes.data_as(ctypes.c_void_p),
                                 el.ctypes.data_as(ctypes.c_void_p) if el is not None else None,
                                 ctypes.byref(p), x.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.byref(st), _stream(stream)))
    return x, st.as_dict()


# ---------------------------------------------------------------- learned
class Net:
    """Learned prolongation network (owns an mm_prolong_net)."""

    def __init__(self, params):
        _require_cuda()
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MM_NET_PARAMS:
            raise ValueError(f"expected {MM_NET_PARAMS} parameters, got {p.size}")
        h = ctypes.c_void_p()
        _check(load().mm_net_create(p.ctypes.data, ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mm_net_free(self.handle)
            self.handle = None

    def params(self):
        out = np.empty(MM_NET_PARAMS, dtype=np.float32)
        _check(load().mm_net_params(self.handle, out.ctypes.data, None))
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().mm_net_params(self.handle, None, p.ctypes.data))

    @staticmethod
    def sample(fine, coarse, x_coarse, seed, level, x_target=None):
        """fine: dict row_ptr/col/map (CUDA); coarse: dict row_ptr/col/c (CUDA)."""
        keep = [fine["row_ptr"], fine["col"], fine["map"], coarse["row_ptr"], coarse["col"],
                coarse["c"], x_coarse, x_target]
        smp = ProlongSample(
            n=fine["row_ptr"].numel() - 1, row_ptr=fine["row_ptr"].data_ptr(),
            col=fine["col"].data_ptr(), map=fine["map"].data_ptr(),
            n_coarse=coarse["row_ptr"].numel() - 1, crow_ptr=coarse["row_ptr"].data_ptr(),
            ccol=coarse["col"].data_ptr(), c_coarse=coarse["c"].data_ptr(),
            x_coarse=x_coarse.data_ptr(), seed=int(seed), level=int(level),
            x_target=x_target.data_ptr() if x_target is not None else None)
        return smp, keep

    def forward(self, smp, stream=None):
        n = smp.n
        x = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        loss = ctypes.c_double(0.0)
        _check(load().mm_net_forward(self.handle, ctypes.byref(smp), _ptr(x), ctypes.byref(loss),
                                     _stream(stream)))
        return x, loss.value

    def gradients(self, smp, stream=None):
        g = np.empty(MM_NET_PARAMS, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(load().mm_net_gradients(self.handle, ctypes.byref(smp), g.ctypes.data,
                                       ctypes.byref(loss), _stream(stream)))
        return g, loss.value

    def train_step(self, smp, lr, stream=None):
        loss = ctypes.c_double(0.0)
        _check(load().mm_net_train_step(self.handle, ctypes.byref(smp), float(lr),
                                        ctypes.byref(loss), _stream(stream)))
        return loss.value


def set_net(h: Hierarchy, net):
    _check(load().mm_hierarchy_set_net(h.handle, net.handle if net is not None else None))
    h._net = net  # keep the network alive while attached


def layout_levels(h: Hierarchy, params: Params = None, stream=None):
    """mm_layout that also returns every level's final layout (list of CUDA
    tensors, level 0 first)."""
    L = h.levels()
    outs = [torch.empty((h.level_info(l)[0], 2), dtype=torch.float32, device="cuda")
            for l in range(L)]
    arr = (ctypes.c_void_p * L)(*[o.data_ptr() for o in outs])
    _check(load().mm_layout_levels(h.handle, ctypes.byref(params) if params is not None else None,
                                   arr, _stream(stream)))
    return outs
