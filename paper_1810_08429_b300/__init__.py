"""Python binding of the B300 GCA-H^2 library (``include/gca.h``).

Argument marshalling only: every step of the construction and of the
products runs in the CUDA kernels of ``libgca.so``.  PyTorch supplies
device memory and streams.  The library must be built first
(``python -m paper_1810_08429_b300._build`` or ``__graft_entry__.build()``);
importing this package without it raises immediately.

    import paper_1810_08429_b300 as gca
    tree = gca.tree_build(vertices, triangles, leaf_size=32)
    h = gca.build(vertices, triangles, tree, gca.Params(leaf_size=32, ...))
    y = h.matvec(x)                     # x: CUDA tensor (n,) or (n, R)
    yt = h.matvec(x, transpose=True)
"""

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgca.so")

F64, F32, BF16 = 0, 1, 2
DROP_F64, DROP_F32, DROP_BF16, DROP_EXPORT, F64_ENTRIES = 1, 2, 4, 8, 16  # gca_params.flags
_PREC = {"f64": F64, "f32": F32, "bf16": BF16, F64: F64, F32: F32, BF16: BF16}

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


class _Mesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("vertices", _f64p), ("triangles", _i32p)]


class _Tree(ctypes.Structure):
    _fields_ = [("nclusters", ctypes.c_int32), ("perm", _i32p), ("begin", _i32p),
                ("end", _i32p), ("child0", _i32p), ("child1", _i32p), ("level", _i32p)]


class _Params(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("eta", ctypes.c_double),
                ("box_gauss_m", ctypes.c_int32), ("aca_tol", ctypes.c_double),
                ("tri_rule", ctypes.c_int32), ("sauter_q", ctypes.c_int32),
                ("omega_margin", ctypes.c_double), ("flags", ctypes.c_uint32)]


class _Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nclusters", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("k", ctypes.c_int32), ("nfar", ctypes.c_int32), ("nnear", ctypes.c_int32),
                ("max_rank", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rank_sum", ctypes.c_int64), ("v_entries", ctypes.c_int64),
                ("e_entries", ctypes.c_int64), ("s_entries", ctypes.c_int64),
                ("n_entries", ctypes.c_int64), ("n_singular", ctypes.c_int64 * 4),
                ("build_seconds", ctypes.c_double)]


class _Phase(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("ms", ctypes.c_double)]


class _ColStats(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("max_rank", ctypes.c_int32), ("rank_sum", ctypes.c_int64),
                ("w_entries", ctypes.c_int64), ("f_entries", ctypes.c_int64)]


class _Dump(ctypes.Structure):
    _fields_ = [("rank", _i32p), ("pivots", _i32p), ("far", _i32p), ("near", _i32p),
                ("V", _f64p), ("E", _f64p), ("S", _f64p), ("N", _f64p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python paper_1810_08429_b300/_build.py`")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    sig = {
        "gca_tree_build": (ctypes.c_int, [ctypes.POINTER(_Mesh), ctypes.c_int32, ctypes.c_int32,
                                          _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p]),
        "gca_build": (ctypes.c_int, [ctypes.POINTER(_Mesh), ctypes.POINTER(_Tree),
                                     ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]),
        "h2_matvec": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int32, vp, ctypes.c_int64, vp,
                                     ctypes.c_int64, vp]),
        "h2_matvec_transpose": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int32, vp,
                                               ctypes.c_int64, vp, ctypes.c_int64, vp]),
        "h2_matvec_noalloc": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int32, vp, ctypes.c_int64, vp,
                                             ctypes.c_int64, vp]),
        "gca_h2_stats": (ctypes.c_int, [vp, ctypes.POINTER(_Stats)]),
        "gca_h2_export": (ctypes.c_int, [vp, ctypes.POINTER(_Dump)]),
        "gca_h2_status": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32)]),
        "gca_free": (None, [vp]),
        "gca_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "gca_last_error": (ctypes.c_char_p, []),
        "gca_build_batch": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(_Mesh), ctypes.POINTER(_Tree),
                                           ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]),
        "gca_batch_size": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32)]),
        "gca_batch_handle": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.POINTER(vp)]),
        "h2_matvec_batch": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64), vp]),
        "h2_matvec_transpose_batch": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                                     ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64),
                                                     ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64),
                                                     vp]),
        "gca_batch_status": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32)]),
        "gca_free_batch": (None, [vp]),
        "gca_profile_enable": (ctypes.c_int, [ctypes.c_int]),
        "gca_profile_read": (ctypes.c_int, [ctypes.POINTER(_Phase), ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int32)]),
        "gca_peak_probe": (ctypes.c_int, [_f64p, _f64p]),
        "gca_tune_batch": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64), vp,
                                          ctypes.POINTER(ctypes.c_int32)]),
        "gca_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
        "gca_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
        "gca_tune_get": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]),
        "gca_tune_clear": (None, []),
        "gca_h2_check": (ctypes.c_int, [vp, vp]),
        "gca_h2_clear_status": (ctypes.c_int, [vp]),
        "gca_batch_check": (ctypes.c_int, [vp, vp]),
        "gca_batch_clear_status": (ctypes.c_int, [vp]),
        "gca_h2_import": (ctypes.c_int, [ctypes.POINTER(_Tree), ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.POINTER(_Dump), ctypes.c_uint32, vp,
                                         ctypes.POINTER(vp)]),
        "gca_test_hook": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int64]),
        "gca_h2_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "gca_h2_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_uint32, vp, ctypes.POINTER(vp)]),
        "gca_build_double_layer": (ctypes.c_int, [ctypes.POINTER(_Mesh), ctypes.POINTER(_Tree),
                                                  ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]),
        "gca_build_collocation": (ctypes.c_int, [ctypes.POINTER(_Mesh), ctypes.POINTER(_Tree),
                                                 ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]),
        "gca_build_single_level": (ctypes.c_int, [ctypes.POINTER(_Mesh), ctypes.POINTER(_Tree),
                                                  ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]),
        "gca_build_green_quadrature": (ctypes.c_int, [ctypes.POINTER(_Mesh), ctypes.POINTER(_Tree),
                                                      ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]),
        "gca_build_p1": (ctypes.c_int, [ctypes.POINTER(_Mesh), ctypes.POINTER(_Tree),
                                        ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]),
        "gca_build_p1_curved": (ctypes.c_int, [ctypes.POINTER(_Mesh), _f64p, ctypes.POINTER(_Tree),
                                               ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]),
        "gca_tree_build_points": (ctypes.c_int, [ctypes.c_int32, _f64p, ctypes.c_int32, ctypes.c_int32,
                                                 _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p]),
        "gca_support_union": (ctypes.c_int, [ctypes.POINTER(_Mesh), ctypes.c_int32, _i32p, _i32p, _i32p,
                                             ctypes.c_int64, _i32p, vp]),
        "gca_h2_column_stats": (ctypes.c_int, [vp, ctypes.POINTER(_ColStats)]),
        "gca_h2_export_columns": (ctypes.c_int, [vp, ctypes.POINTER(_Dump)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NUMERIC, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_IO = 0, -1, -2, -3, -4, -5, -6, -7


class GCAError(RuntimeError):
    """A failed library call; ``status`` is the gca_status code."""

    def __init__(self, msg, status=None):
        super().__init__(msg)
        self.status = status


def _check(status, what):
    if status != 0:
        msg = lib.gca_last_error().decode(errors="replace")
        raise GCAError(f"{what}: {lib.gca_strerror(status).decode()} ({status}): {msg}", status)


@dataclass
class Params:
    """Construction parameters (mirrors ``gca_params``)."""
    leaf_size: int = 32
    eta: float = 2.0
    box_gauss_m: int = 3
    aca_tol: float = 1e-6
    tri_rule: int = 7
    sauter_q: int = 5
    omega_margin: float = -1.0
    flags: int = 0

    def _c(self):
        return _Params(self.leaf_size, self.eta, self.box_gauss_m, self.aca_tol, self.tri_rule,
                       self.sauter_q, self.omega_margin, self.flags)


def _mesh(vertices, triangles):
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    t = np.ascontiguousarray(triangles, dtype=np.int32)
    if v.ndim != 2 or v.shape[1] != 3 or t.ndim != 2 or t.shape[1] != 3:
        raise ValueError("vertices must be (nv, 3) and triangles (nt, 3)")
    m = _Mesh(v.shape[0], t.shape[0], v.ctypes.data_as(_f64p), t.ctypes.data_as(_i32p))
    return m, (v, t)


def tree_build(vertices, triangles, leaf_size):
    """Cluster tree by recursive bisection (``gca_tree_build``), as numpy arrays."""
    m, keep = _mesh(vertices, triangles)
    n = m.nt
    cap = max(2 * n - 1, 1)
    out = {k: np.zeros(n if k == "perm" else cap, dtype=np.int32)
           for k in ("perm", "begin", "end", "child0", "child1", "level")}
    nc = ctypes.c_int32(0)
    st = lib.gca_tree_build(ctypes.byref(m), leaf_size, cap,
                            *[out[k].ctypes.data_as(_i32p)
                              for k in ("perm", "begin", "end", "child0", "child1", "level")],
                            ctypes.byref(nc))
    _check(st, "gca_tree_build")
    for k in ("begin", "end", "child0", "child1", "level"):
        out[k] = out[k][:nc.value].copy()
    return out


def tree_build_points(points, leaf_size):
    """Cluster tree by recursive bisection of given points
    (``gca_tree_build_points``, e.g. the vertices for ``build_p1``)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    if pts.ndim != 2 or pts.shape[1] != 3:
        raise ValueError("points must be (n, 3)")
    n = pts.shape[0]
    cap = max(2 * n - 1, 1)
    out = {k: np.zeros(n if k == "perm" else cap, dtype=np.int32)
           for k in ("perm", "begin", "end", "child0", "child1", "level")}
    nc = ctypes.c_int32(0)
    st = lib.gca_tree_build_points(n, pts.ctypes.data_as(_f64p), leaf_size, cap,
                                   *[out[k].ctypes.data_as(_i32p)
                                     for k in ("perm", "begin", "end", "child0", "child1", "level")],
                                   ctypes.byref(nc))
    _check(st, "gca_tree_build_points")
    for k in ("begin", "end", "child0", "child1", "level"):
        out[k] = out[k][:nc.value].copy()
    return out


def support_union(vertices, triangles, lists, stream=None):
    """The support unions of Sect. 5 computed on the device
    (``gca_support_union``): for each list of vertex ids a list of rows
    (triangle, (l0, l1, l2)) in ascending triangle id, l_c the position of
    the triangle's corner c in the list or -1."""
    m, keep_m = _mesh(vertices, triangles)
    lists = [np.ascontiguousarray(a, dtype=np.int32).reshape(-1) for a in lists]
    ptr = np.zeros(len(lists) + 1, dtype=np.int32)
    for i, a in enumerate(lists):
        ptr[i + 1] = ptr[i] + len(a)
    flat = np.ascontiguousarray(np.concatenate(lists + [np.zeros(1, np.int32)]), dtype=np.int32)
    nv = keep_m[0].shape[0]
    val = np.bincount(np.clip(keep_m[1].reshape(-1), 0, nv), minlength=nv + 1)
    # ids out of range are refused by the library; they count 0 here
    cap = int(sum(int(val[np.where((a >= 0) & (a < nv), a, nv)].sum()) for a in lists))
    rows = np.zeros((max(cap, 1), 4), dtype=np.int32)
    counts = np.zeros(max(len(lists), 1), dtype=np.int32)
    _check(lib.gca_support_union(ctypes.byref(m), len(lists), ptr.ctypes.data_as(_i32p), flat.ctypes.data_as(_i32p),
                                 rows.ctypes.data_as(_i32p), cap, counts.ctypes.data_as(_i32p),
                                 _stream_ptr(stream)), "gca_support_union")
    out, at = [], 0
    for i in range(len(lists)):
        r = rows[at:at + counts[i]]
        at += counts[i]
        out.append([(int(a[0]), (int(a[1]), int(a[2]), int(a[3]))) for a in r])
    return out


def _tree(tree):
    arrs = {k: np.ascontiguousarray(tree[k], dtype=np.int32)
            for k in ("perm", "begin", "end", "child0", "child1", "level")}
    t = _Tree(len(arrs["begin"]), *[arrs[k].ctypes.data_as(_i32p)
                                     for k in ("perm", "begin", "end", "child0", "child1", "level")])
    return t, arrs


def _stream_ptr(stream):
    import torch
    if stream is None:
        if not torch.cuda.is_available():
            return ctypes.c_void_p(None)  # host-side validation fails before any device work
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class H2:
    """A built GCA-H^2 matrix on the current CUDA device (a gca_h2 handle).

    Handles returned by ``build`` own their device memory; handles of a
    ``Batch`` are views that the batch owns."""

    def __init__(self, handle, owner=None):
        self._h = ctypes.c_void_p(handle)
        self._owner = owner

    def __del__(self):
        self.free()

    def free(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and getattr(self, "_owner", None) is None:
            lib.gca_free(h)
        self._h = ctypes.c_void_p(None)

    @property
    def handle(self):
        return self._h

    def stats(self):
        s = _Stats()
        _check(lib.gca_h2_stats(self._h, ctypes.byref(s)), "gca_h2_stats")
        out = {name: getattr(s, name) for name, _ in _Stats._fields_ if name != "n_singular"}
        out["n_singular"] = list(s.n_singular)
        return out

    def status(self):
        """Sticky error bits of the products so far (0: none); synchronises."""
        v = ctypes.c_int32(0)
        _check(lib.gca_h2_status(self._h, ctypes.byref(v)), "gca_h2_status")
        return v.value

    def check(self, stream=None):
        """Raise GCAError (GCA_ERR_TIMEOUT, ...) if a product on this handle
        recorded an error (gca_h2_check); synchronises the stream."""
        _check(lib.gca_h2_check(self._h, _stream_ptr(stream)), "gca_h2_check")

    def clear_status(self):
        """Clear the sticky error bits (gca_h2_clear_status)."""
        _check(lib.gca_h2_clear_status(self._h), "gca_h2_clear_status")

    def matvec_noalloc(self, x, prec="f64", out=None, stream=None):
        """y = G_H2 x through h2_matvec_noalloc (workspace from the library's
        fixed device array; same conventions as ``matvec``)."""
        import torch
        p = _PREC[prec]
        dt = torch.float64 if p == F64 else torch.float32
        x2, vec = _as_colmajor(x, dt)
        n, R = x2.shape
        if out is None:
            out = _empty_like_colmajor(x2, dt)
        y2 = out[:, None] if out.dim() == 1 else out
        _check(lib.h2_matvec_noalloc(self._h, p, R, ctypes.c_void_p(x2.data_ptr()),
                                     x2.stride(1) if R > 1 else n, ctypes.c_void_p(y2.data_ptr()),
                                     y2.stride(1) if R > 1 else n, _stream_ptr(stream)),
               "h2_matvec_noalloc")
        return out[:, 0] if vec and out.dim() == 2 else out

    def export(self, parts=None):
        """Host copy of the representation (layout documented in gca.h); with
        `parts` (e.g. ("rank",)) only those arrays are copied."""
        s = self.stats()
        sizes = {"rank": s["nclusters"], "pivots": s["rank_sum"], "far": 2 * s["nfar"],
                 "near": 2 * s["nnear"], "V": s["v_entries"], "E": s["e_entries"],
                 "S": s["s_entries"], "N": s["n_entries"]}
        keys = ("rank", "pivots", "far", "near", "V", "E", "S", "N")
        want = set(keys if parts is None else parts)
        d = {k: np.zeros(max(sizes[k], 1), dtype=np.int32 if k in ("rank", "pivots", "far", "near")
                         else np.float64) for k in keys if k in want}
        dump = _Dump(*[d[k].ctypes.data_as(_i32p if d[k].dtype == np.int32 else _f64p) if k in d
                       else None for k in keys])
        _check(lib.gca_h2_export(self._h, ctypes.byref(dump)), "gca_h2_export")
        for k in d:
            d[k] = d[k][:sizes[k]]
        if "far" in d:
            d["far"] = d["far"].reshape(-1, 2)
        if "near" in d:
            d["near"] = d["near"].reshape(-1, 2)
        return d

    def save(self, path):
        """Write a checkpoint of this handle to `path` (gca_h2_save); ``load``
        reads it back."""
        _check(lib.gca_h2_save(self._h, os.fsencode(path)), "gca_h2_save")

    def column_stats(self):
        """Sizes of the column side (gca_h2_column_stats)."""
        s = _ColStats()
        _check(lib.gca_h2_column_stats(self._h, ctypes.byref(s)), "gca_h2_column_stats")
        return {name: getattr(s, name) for name, _ in _ColStats._fields_}

    def export_columns(self):
        """Host copy of the column side: rank (r'), pivots, W (leaf column
        bases) and F (column transfers) (gca_h2_export_columns)."""
        s = self.stats()
        c = self.column_stats()
        d = {"rank": np.zeros(s["nclusters"], dtype=np.int32),
             "pivots": np.zeros(max(c["rank_sum"], 1), dtype=np.int32),
             "W": np.zeros(max(c["w_entries"], 1)), "F": np.zeros(max(c["f_entries"], 1))}
        dump = _Dump(d["rank"].ctypes.data_as(_i32p), d["pivots"].ctypes.data_as(_i32p), None, None,
                     d["W"].ctypes.data_as(_f64p), d["F"].ctypes.data_as(_f64p), None, None)
        _check(lib.gca_h2_export_columns(self._h, ctypes.byref(dump)), "gca_h2_export_columns")
        d["pivots"] = d["pivots"][:c["rank_sum"]]
        d["W"] = d["W"][:c["w_entries"]]
        d["F"] = d["F"][:c["f_entries"]]
        return d

    def matvec_raw(self, prec, nrhs, x_ptr, ldx, y_ptr, ldy, stream_ptr, transpose=False):
        fn = lib.h2_matvec_transpose if transpose else lib.h2_matvec
        _check(fn(self._h, _PREC.get(prec, prec), nrhs, x_ptr, ldx, y_ptr, ldy, stream_ptr),
               "h2_matvec_transpose" if transpose else "h2_matvec")

    @property
    def n(self):
        return self.stats()["n"]

    def matvec(self, x, prec="f64", transpose=False, out=None, stream=None):
        """y = G_H2 x (or G_H2^T x) for x of shape (n,) or (n, R), a tensor on the
        GPU or in page-locked host memory (read in place by the product); the
        result is allocated beside x unless `out` is given."""
        import torch
        p = _PREC[prec]
        dt = torch.float64 if p == F64 else torch.float32
        x2, vec = _as_colmajor(x, dt)
        n, R = x2.shape
        if out is None:
            out = _empty_like_colmajor(x2, dt)
        y2 = out[:, None] if out.dim() == 1 else out
        if y2.stride(0) != 1 or y2.shape != (n, R):
            raise ValueError("out must be column-major (n, R)")
        self.matvec_raw(p, R, ctypes.c_void_p(x2.data_ptr()), x2.stride(1) if R > 1 else n,
                        ctypes.c_void_p(y2.data_ptr()), y2.stride(1) if R > 1 else n,
                        _stream_ptr(stream), transpose)
        return out[:, 0] if vec and out.dim() == 2 else out


def profile_enable(on=True, detail=False):
    """Start / stop per-phase GPU event timing (gca_profile_enable); with
    `detail` the build's per-level phases are split by level and cluster size."""
    _check(lib.gca_profile_enable((2 if detail else 1) if on else 0), "gca_profile_enable")


def profile_read():
    """{phase: (launches, ms)} accumulated since the last read (gca_profile_read)."""
    cap = 256
    buf = (_Phase * cap)()
    cnt = ctypes.c_int32(0)
    _check(lib.gca_profile_read(buf, cap, ctypes.byref(cnt)), "gca_profile_read")
    return {buf[i].name.decode(): (buf[i].launches, buf[i].ms) for i in range(min(cnt.value, cap))}


def peak_probe():
    """(float64, float32) FMA throughput of the current device in FLOP/s."""
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib.gca_peak_probe(ctypes.byref(a), ctypes.byref(b)), "gca_peak_probe")
    return a.value, b.value


def build(vertices, triangles, tree, params, stream=None):
    """gca_build on the current CUDA device; returns an ``H2``."""
    m, keep_m = _mesh(vertices, triangles)
    t, keep_t = _tree(tree)
    p = params._c()
    h = ctypes.c_void_p(None)
    _check(lib.gca_build(ctypes.byref(m), ctypes.byref(t), ctypes.byref(p), _stream_ptr(stream),
                         ctypes.byref(h)), "gca_build")
    return H2(h.value)


def _dump_arrays(d):
    """gca_host_dump over the arrays of `d` (keys as ``H2.export`` returns)."""
    arrs = {
        "rank": np.ascontiguousarray(d["rank"], dtype=np.int32),
        "pivots": np.ascontiguousarray(d["pivots"], dtype=np.int32),
        "far": np.ascontiguousarray(np.asarray(d["far"], dtype=np.int32).reshape(-1)),
        "near": np.ascontiguousarray(np.asarray(d["near"], dtype=np.int32).reshape(-1)),
    }
    for k in ("V", "E", "S", "N"):
        arrs[k] = np.ascontiguousarray(d[k], dtype=np.float64)
    for k, a in arrs.items():
        if a.size == 0:
            arrs[k] = np.zeros(1, dtype=a.dtype)
    dump = _Dump(*[arrs[k].ctypes.data_as(_i32p if arrs[k].dtype == np.int32 else _f64p)
                   for k in ("rank", "pivots", "far", "near", "V", "E", "S", "N")])
    return dump, arrs


def import_h2(tree, n, rep, flags=0, stream=None):
    """gca_h2_import: a handle from a host representation `rep` (dict with
    rank, pivots, far [(tau, sigma)], near, V, E, S, N in the layout of
    ``H2.export``) over the cluster tree `tree` of n triangles."""
    t, keep_t = _tree(tree)
    dump, keep_d = _dump_arrays(rep)
    nfar = len(np.asarray(rep["far"]).reshape(-1)) // 2
    nnear = len(np.asarray(rep["near"]).reshape(-1)) // 2
    h = ctypes.c_void_p(None)
    _check(lib.gca_h2_import(ctypes.byref(t), n, nfar, nnear, ctypes.byref(dump), flags,
                             _stream_ptr(stream), ctypes.byref(h)), "gca_h2_import")
    return H2(h.value)


def load(path, flags=0, stream=None):
    """gca_h2_load: a handle on the current CUDA device from a checkpoint
    written by ``H2.save``."""
    h = ctypes.c_void_p(None)
    _check(lib.gca_h2_load(os.fsencode(path), flags, _stream_ptr(stream), ctypes.byref(h)), "gca_h2_load")
    return H2(h.value)


def test_hook(name, value):
    """Set a failure-path test hook (gca_test_hook)."""
    _check(lib.gca_test_hook(name.encode(), int(value)), "gca_test_hook")


def build_double_layer(vertices, triangles, tree, params, stream=None):
    """gca_build_double_layer on the current CUDA device; returns an ``H2``
    whose products apply the double-layer matrix K (and K^T)."""
    m, keep_m = _mesh(vertices, triangles)
    t, keep_t = _tree(tree)
    p = params._c()
    h = ctypes.c_void_p(None)
    _check(lib.gca_build_double_layer(ctypes.byref(m), ctypes.byref(t), ctypes.byref(p), _stream_ptr(stream),
                                      ctypes.byref(h)), "gca_build_double_layer")
    return H2(h.value)


def _build_with(fn, name, vertices, triangles, tree, params, stream):
    m, keep_m = _mesh(vertices, triangles)
    t, keep_t = _tree(tree)
    p = params._c()
    h = ctypes.c_void_p(None)
    _check(fn(ctypes.byref(m), ctypes.byref(t), ctypes.byref(p), _stream_ptr(stream), ctypes.byref(h)), name)
    return H2(h.value)


def build_single_level(vertices, triangles, tree, params, stream=None):
    """Single-level GCA of G (gca_build_single_level); returns an ``H2``."""
    return _build_with(lib.gca_build_single_level, "gca_build_single_level", vertices, triangles, tree, params,
                       stream)


def build_green_quadrature(vertices, triangles, tree, params, stream=None):
    """Pure Green quadrature of G (gca_build_green_quadrature); returns an ``H2``."""
    return _build_with(lib.gca_build_green_quadrature, "gca_build_green_quadrature", vertices, triangles, tree,
                       params, stream)


def build_p1(vertices, triangles, tree, params, stream=None):
    """gca_build_p1: the single-layer matrix in the continuous piecewise
    linear (nodal) basis of Sect. 5 over a tree of the VERTICES (e.g.
    ``tree_build_points(vertices, leaf)``); returns an ``H2`` whose products
    take x and y with one row per vertex."""
    return _build_with(lib.gca_build_p1, "gca_build_p1", vertices, triangles, tree, params, stream)


def build_p1_curved(vertices, triangles, midpoints, tree, params, stream=None):
    """gca_build_p1_curved: the nodal basis on curved triangles (Sect. 6);
    `midpoints` (nt, 3, 3) holds the surface points over the edges (0, 1),
    (1, 2), (2, 0) of every triangle."""
    m, keep_m = _mesh(vertices, triangles)
    mid = np.ascontiguousarray(midpoints, dtype=np.float64)
    if mid.shape != (m.nt, 3, 3):
        raise ValueError("midpoints must be (nt, 3, 3)")
    t, keep_t = _tree(tree)
    p = params._c()
    h = ctypes.c_void_p(None)
    _check(lib.gca_build_p1_curved(ctypes.byref(m), mid.ctypes.data_as(_f64p), ctypes.byref(t), ctypes.byref(p),
                                   _stream_ptr(stream), ctypes.byref(h)), "gca_build_p1_curved")
    return H2(h.value)


def build_collocation(vertices, triangles, tree, params, stream=None):
    """gca_build_collocation on the current CUDA device; returns an ``H2``
    whose products apply the collocation matrix C (and C^T)."""
    m, keep_m = _mesh(vertices, triangles)
    t, keep_t = _tree(tree)
    p = params._c()
    h = ctypes.c_void_p(None)
    _check(lib.gca_build_collocation(ctypes.byref(m), ctypes.byref(t), ctypes.byref(p), _stream_ptr(stream),
                                     ctypes.byref(h)), "gca_build_collocation")
    return H2(h.value)


def _as_colmajor(x, dt):
    vec = x.dim() == 1
    x2 = x[:, None] if vec else x
    if x2.dtype != dt or not (x2.is_cuda or x2.is_pinned()):
        raise TypeError(f"x must be a {dt} tensor on the GPU or in page-locked host memory")
    if x2.stride(0) != 1:
        x2 = x2.t().contiguous().t()
        if not x2.is_cuda:
            x2 = x2.pin_memory()
    return x2, vec


def _empty_like_colmajor(x2, dt):
    """A column-major (n, R) result beside x2: on its GPU, or page-locked."""
    import torch
    if x2.is_cuda:
        return torch.empty((x2.shape[1], x2.shape[0]), dtype=dt, device=x2.device).t()
    return torch.empty((x2.shape[1], x2.shape[0]), dtype=dt, pin_memory=True).t()


class Batch:
    """Several GCA-H^2 matrices applied in one persistent launch (gca_h2_batch)."""

    def __init__(self, ptr):
        self._b = ctypes.c_void_p(ptr)
        cnt = ctypes.c_int32(0)
        _check(lib.gca_batch_size(self._b, ctypes.byref(cnt)), "gca_batch_size")
        self.handles = []
        for i in range(cnt.value):
            h = ctypes.c_void_p(None)
            _check(lib.gca_batch_handle(self._b, i, ctypes.byref(h)), "gca_batch_handle")
            self.handles.append(H2(h.value, owner=self))

    def __len__(self):
        return len(self.handles)

    def __del__(self):
        self.free()

    def free(self):
        b = getattr(self, "_b", None)
        if b is not None and b.value:
            for h in self.handles:
                h._h = ctypes.c_void_p(None)
            lib.gca_free_batch(b)
            self._b = ctypes.c_void_p(None)

    def status(self):
        v = ctypes.c_int32(0)
        _check(lib.gca_batch_status(self._b, ctypes.byref(v)), "gca_batch_status")
        return v.value

    def check(self, stream=None):
        """Raise GCAError if a product on this batch recorded an error."""
        _check(lib.gca_batch_check(self._b, _stream_ptr(stream)), "gca_batch_check")

    def clear_status(self):
        _check(lib.gca_batch_clear_status(self._b), "gca_batch_clear_status")

    def tune(self, xs, prec="f32", transpose=False, outs=None, stream=None):
        """Autotune the tile width of this product (``gca_tune_batch``): runs it
        with each candidate width (outs are overwritten), records the fastest
        for later products with the same key and returns it."""
        return self._call(xs, prec, transpose, outs, stream, tune=True)

    def matvec(self, xs, prec="f32", transpose=False, outs=None, stream=None):
        """[G_i x_i] (or transposes) for tensors x_i of shape (n_i,) or (n_i, R_i) on
        the GPU or in page-locked host memory."""
        return self._call(xs, prec, transpose, outs, stream, tune=False)

    def _call(self, xs, prec, transpose, outs, stream, tune):
        import torch
        p = _PREC[prec]
        dt = torch.float64 if p == F64 else torch.float32
        k = len(self.handles)
        if len(xs) != k:
            raise ValueError("one right-hand side block per mesh")
        xs2, vecs = zip(*[_as_colmajor(x, dt) for x in xs])
        if outs is None:
            outs = [_empty_like_colmajor(x2, dt) for x2 in xs2]
        ys2 = [o[:, None] if o.dim() == 1 else o for o in outs]
        nrhs = (ctypes.c_int32 * k)(*[x2.shape[1] for x2 in xs2])
        xp = (ctypes.c_void_p * k)(*[x2.data_ptr() for x2 in xs2])
        yp = (ctypes.c_void_p * k)(*[y2.data_ptr() for y2 in ys2])
        ldx = (ctypes.c_int64 * k)(*[x2.stride(1) if x2.shape[1] > 1 else x2.shape[0] for x2 in xs2])
        ldy = (ctypes.c_int64 * k)(*[y2.stride(1) if y2.shape[1] > 1 else y2.shape[0] for y2 in ys2])
        if tune:
            w = ctypes.c_int32(0)
            _check(lib.gca_tune_batch(self._b, p, 1 if transpose else 0, nrhs, xp, ldx, yp, ldy,
                                      _stream_ptr(stream), ctypes.byref(w)), "gca_tune_batch")
            return w.value
        fn = lib.h2_matvec_transpose_batch if transpose else lib.h2_matvec_batch
        _check(fn(self._b, p, nrhs, xp, ldx, yp, ldy, _stream_ptr(stream)), "h2_matvec_batch")
        return [o[:, 0] if v and o.dim() == 2 else o for o, v in zip(outs, vecs)]


def tune_save(path):
    """Write the tile-width table to a text file (``gca_tune_save``)."""
    _check(lib.gca_tune_save(os.fsencode(path)), "gca_tune_save")


def tune_load(path):
    """Merge a table written by ``tune_save`` (``gca_tune_load``)."""
    _check(lib.gca_tune_load(os.fsencode(path)), "gca_tune_load")


def tune_get(device, prec, transpose, nrhs, rows):
    """Tile width recorded for a key, 0 if none (``gca_tune_get``)."""
    w = ctypes.c_int32(0)
    _check(lib.gca_tune_get(device.encode(), _PREC.get(prec, prec), 1 if transpose else 0, nrhs, rows,
                            ctypes.byref(w)), "gca_tune_get")
    return w.value


def tune_clear():
    """Empty the tile-width table (``gca_tune_clear``)."""
    lib.gca_tune_clear()


def build_batch(meshes, trees, params, stream=None):
    """gca_build_batch over [(vertices, triangles)] with matching trees; returns a ``Batch``."""
    k = len(meshes)
    ms, keep = [], []
    for v, t in meshes:
        m, kp = _mesh(v, t)
        ms.append(m)
        keep.append(kp)
    trs = []
    for tr in trees:
        t, kp = _tree(tr)
        trs.append(t)
        keep.append(kp)
    marr = (_Mesh * k)(*ms)
    tarr = (_Tree * k)(*trs)
    p = params._c()
    b = ctypes.c_void_p(None)
    _check(lib.gca_build_batch(k, marr, tarr, ctypes.byref(p), _stream_ptr(stream), ctypes.byref(b)),
           "gca_build_batch")
    return Batch(b.value)


_AUTOGRAD = None


def _autograd_class():
    global _AUTOGRAD
    if _AUTOGRAD is None:
        import torch

        class H2Matvec(torch.autograd.Function):
            """y = G_H2 u as a differentiable torch operation.

            ``H2Matvec.apply(h, u, prec)`` runs ``h2_matvec``; the backward
            is the transposed H^2 product, dL/du = G_H2^T dL/dy
            (``h2_matvec_transpose``), so gradients of losses such as
            ||P G_H2 u - f||^2 cost one more product.  u is a CUDA tensor of
            shape (n,) or (n, R): float64 for prec "f64", float32 otherwise.
            """

            @staticmethod
            def forward(ctx, h, u, prec="f32"):
                ctx.h = h
                ctx.prec = prec
                return h.matvec(u, prec)

            @staticmethod
            def backward(ctx, gy):
                return None, ctx.h.matvec(gy, ctx.prec, transpose=True), None

        _AUTOGRAD = H2Matvec
    return _AUTOGRAD


def __getattr__(name):
    if name == "H2Matvec":
        return _autograd_class()
    raise AttributeError(name)


def h2_matvec_autograd(h, u, prec="f32"):
    """Differentiable y = G_H2 u (backward: the transposed product)."""
    return _autograd_class().apply(h, u, prec)
