"""GB300-native compressed Coulomb-integral engine for planewave bases.

A thin ctypes binding of libcoulomb.so (include/coulomb.h): argument marshalling only.
Every step of the hot path runs in the library's CUDA kernels; there is no CPU or
PyTorch fallback, and every call fails loudly (ImportError / CoulombError) when the
library is missing or a call is rejected.  PyTorch tensors are accepted wherever the C
ABI takes a device pointer; the stream defaults to torch's current stream.

Method: Pederson, arXiv:1502.08043.  The Coulomb kernel is factorised by a Laplace
transform, the t = alpha^-1/2 tail substitution and Gauss quadrature (Sec. II, Eqs. 5-14)
into per-node 1D tables; integrals (IJ|KL) and exchange sums of the uniform electron gas
(Sec. III) are rebuilt from them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcoulomb.so")

KERNELS = {"periodic": 0, "box": 1}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16x3": 2, "fp16x3": 3}
LOOKUPS = {"separable": 0, "collapsed": 1, "general": 2}
FORMATS = {"ids": 0, "vec": 1, "ids16": 2}
STATUS = {0: "ok", 1: "invalid argument", 2: "size beyond limit", 3: "CUDA error",
          4: "allocation failed", 5: "device wait timed out", 6: "not supported",
          7: "I/O or format error"}


class CoulombError(RuntimeError):
    def __init__(self, fn, status, detail=""):
        self.status = status
        msg = f"{fn}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class TableParams(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("R", ctypes.c_int), ("L", ctypes.c_double),
                ("S", ctypes.c_int), ("n_sub", ctypes.c_int), ("q_tail", ctypes.c_int),
                ("alpha_c", ctypes.c_double), ("prune_tol", ctypes.c_double),
                ("ratio", ctypes.c_double)]


class TablesInfo(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("R", ctypes.c_int), ("S", ctypes.c_int),
                ("n_sub", ctypes.c_int), ("q_tail", ctypes.c_int), ("L", ctypes.c_double),
                ("alpha_c", ctypes.c_double), ("prune_tol", ctypes.c_double),
                ("S_eff", ctypes.c_int), ("Nb", ctypes.c_int), ("Mg", ctypes.c_int),
                ("m_max", ctypes.c_int), ("device_bytes", ctypes.c_size_t),
                ("table_bytes", ctypes.c_size_t), ("ratio", ctypes.c_double),
                ("general_codes", ctypes.c_int),
                ("general_table_bytes", ctypes.c_size_t)]


class Box(ctypes.Structure):
    _fields_ = [("p", TableParams), ("R_F", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
# every symbol declared in include/coulomb.h, with its C signature
SIGNATURES = {
    "cc_build_tables": (_I, [ctypes.POINTER(TableParams), _P, ctypes.POINTER(_P)]),
    "cc_tables_info": (_I, [_P, ctypes.POINTER(TablesInfo)]),
    "cc_tables_nodes": (_I, [_P, _P, _P, _P, _P]),
    "cc_tables_values": (_I, [_P, _P]),
    "cc_tables_general_values": (_I, [_P, _P]),
    "cc_tables_save": (_I, [_P, ctypes.c_char_p]),
    "cc_tables_load": (_I, [ctypes.c_char_p, _P, ctypes.POINTER(_P)]),
    "cc_tables_free": (_I, [_P]),
    "cc_basis": (_I, [_I, ctypes.POINTER(_I), _P]),
    "cc_default_mesh": (_I, [_I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "cc_mesh_for_error": (_I, [_I, ctypes.c_double, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                               ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]),
    "cc_mesh_tune": (_I, [_I, ctypes.c_double, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                          ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "cc_build_tables_for_error": (_I, [_I, _I, ctypes.c_double, ctypes.c_double, _I, _P,
                                       ctypes.POINTER(_P)]),
    "cc_reconstruct_integrals": (_I, [_P, _P, _I64, _I, _I, _I, _P, _P, _P]),
    "cc_pair_matrix": (_I, [_P, _I64, _I64, _I, _I, _P, _P]),
    "cc_exchange_sums": (_I, [_P, _I, _I, _P, _P, _P]),
    "cc_set_gemm_tiles": (_I, [_I, _I, _I, _I]),
    "cc_autotune_gemm": (_I, [_P, _I, _I, _I, _P, _P, _P]),
    "cc_gemm_tiles_tuned": (_I, [_I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "cc_mixed_status": (_I, [_P, _P, _I]),
    "cc_exchange_sums_noalloc": (_I, [_P, _I, _P, _P, _P]),
    "cc_test_stall_next_mixed": (_I, []),
    "cc_set_mixed_variant": (_I, [_I]),
    "cc_set_simt_variant": (_I, [_I]),
    "cc_set_id_decode": (_I, [_I]),
    "cc_set_mixed_terms": (_I, [_I]),
    "cc_batch_create": (_I, [ctypes.POINTER(Box), _I, _P, ctypes.POINTER(_P)]),
    "cc_batch_info": (_I, [_P, _P, _P, _P, _P]),
    "cc_batch_exchange": (_I, [_P, _I, _P, _P, _P]),
    "cc_batch_set_plan": (_I, [_P, _I, _I]),
    "cc_batch_tune": (_I, [_P, _I, _P, _P, _I, _P, _P, _P]),
    "cc_batch_free": (_I, [_P]),
    "cc_status_string": (ctypes.c_char_p, [_I]),
    "cc_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded libcoulomb.so (ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "libcoulomb.so is not built: run `python -c 'import __graft_entry__ as g; "
                "g.build()'` (nvcc, sm_103a); there is no fallback implementation")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(fn, status):
    if status != 0:
        detail = lib().cc_last_error().decode() if status == 3 else ""
        raise CoulombError(fn, status, detail)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _stream(stream, *tensors):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    dev = None
    for t in tensors:
        if hasattr(t, "device") and t.is_cuda:
            dev = t.device
            break
    return torch.cuda.current_stream(dev).cuda_stream


class Tables:
    """A table handle (owns device memory).  Build with build_tables() or load_tables()."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)
        inf = TablesInfo()
        _check("cc_tables_info", lib().cc_tables_info(self._h, ctypes.byref(inf)))
        self.info = {k: getattr(inf, k) for k, _ in TablesInfo._fields_}

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("tables were freed")
        return self._h

    def __getattr__(self, k):
        info = self.__dict__.get("info")
        if info is not None and k in info:
            return info[k]
        raise AttributeError(k)

    def nodes(self):
        S = self.info["S"]
        a = np.zeros(S)
        w = np.zeros(S)
        part = np.zeros(S, dtype=np.int32)
        kept = np.zeros(S, dtype=np.int32)
        _check("cc_tables_nodes", lib().cc_tables_nodes(
            self.handle, a.ctypes.data, w.ctypes.data, part.ctypes.data, kept.ctypes.data))
        return a, w, part, kept.astype(bool)

    def values(self):
        T = np.zeros((self.info["S_eff"], 2 * self.info["R"] + 1))
        _check("cc_tables_values", lib().cc_tables_values(self.handle, T.ctypes.data))
        return T

    def general_values(self):
        """Box tables: the FP64 two-index tables A(alpha_s, d1, d2) of the kept nodes,
        float64[S_eff, (2R + 1)^2] by canonical code d1^2 + d1 + d2 (d1 >= |d2|)."""
        G = np.zeros((self.info["S_eff"], self.info["general_codes"]))
        _check("cc_tables_general_values",
               lib().cc_tables_general_values(self.handle, G.ctypes.data))
        return G

    def save(self, path):
        _check("cc_tables_save", lib().cc_tables_save(self.handle, str(path).encode()))

    def free(self):
        if self._h is not None:
            _check("cc_tables_free", lib().cc_tables_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_tables(kernel="periodic", R=4, L=10.0, S=32, n_sub=-1, q_tail=-1, alpha_c=1.0,
                 prune_tol=-1.0, ratio=5.0, stream=None) -> Tables:
    """cc_build_tables: nodes, weights and tables on the current CUDA device (FP64)."""
    p = TableParams(KERNELS[kernel] if isinstance(kernel, str) else int(kernel), int(R),
                    float(L), int(S), int(n_sub), int(q_tail), float(alpha_c), float(prune_tol),
                    float(ratio))
    h = ctypes.c_void_p()
    _check("cc_build_tables", lib().cc_build_tables(ctypes.byref(p), _stream(stream),
                                                    ctypes.byref(h)))
    return Tables(h.value)


def load_tables(path, stream=None) -> Tables:
    h = ctypes.c_void_p()
    _check("cc_tables_load", lib().cc_tables_load(str(path).encode(), _stream(stream),
                                                  ctypes.byref(h)))
    return Tables(h.value)


def default_mesh(S: int, R: int):
    """cc_default_mesh: (n_sub, q_tail) chosen when both are left to the library."""
    n = ctypes.c_int()
    q = ctypes.c_int()
    _check("cc_default_mesh", lib().cc_default_mesh(int(S), int(R), ctypes.byref(n),
                                                    ctypes.byref(q)))
    return n.value, q.value


def mesh_for_error(R: int, target: float, S_max: int = 1024):
    """cc_mesh_for_error: (S, n_sub, q_tail, error) of the fewest nodes whose default mesh
    reaches the stated method error."""
    S = ctypes.c_int()
    n = ctypes.c_int()
    q = ctypes.c_int()
    e = ctypes.c_double()
    _check("cc_mesh_for_error", lib().cc_mesh_for_error(int(R), float(target), int(S_max),
                                                        ctypes.byref(S), ctypes.byref(n),
                                                        ctypes.byref(q), ctypes.byref(e)))
    return S.value, n.value, q.value, e.value


def mesh_tune(R: int, target: float, S_max: int = 1024):
    """cc_mesh_tune: (S, n_sub, q_tail, alpha_c, ratio, error) of the fewest nodes over the
    tuned mesh family that reach the stated method error."""
    S, n, q = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    a, r, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check("cc_mesh_tune", lib().cc_mesh_tune(int(R), float(target), int(S_max), ctypes.byref(S),
                                              ctypes.byref(n), ctypes.byref(q), ctypes.byref(a),
                                              ctypes.byref(r), ctypes.byref(e)))
    return S.value, n.value, q.value, a.value, r.value, e.value


def build_tables_for_error(kernel="periodic", R=4, L=10.0, target=1e-6, S_max=1024,
                           stream=None) -> Tables:
    """cc_build_tables_for_error: tables on the tuned mesh with the fewest nodes for a stated
    periodic-kernel method error."""
    h = ctypes.c_void_p()
    _check("cc_build_tables_for_error", lib().cc_build_tables_for_error(
        KERNELS[kernel] if isinstance(kernel, str) else int(kernel), int(R), float(L),
        float(target), int(S_max), _stream(stream), ctypes.byref(h)))
    return Tables(h.value)


def basis(R: int) -> np.ndarray:
    """cc_basis: int8[Nb, 4] vectors (n_x, n_y, n_z, 0) in canonical order."""
    nb = ctypes.c_int()
    _check("cc_basis", lib().cc_basis(int(R), ctypes.byref(nb), None))
    out = np.zeros((nb.value, 4), dtype=np.int8)
    _check("cc_basis", lib().cc_basis(int(R), ctypes.byref(nb), out.ctypes.data))
    return out


def _prec_of(t):
    import torch
    if t.dtype == torch.float32:
        return PRECISIONS["fp32"]
    if t.dtype == torch.float64:
        return PRECISIONS["fp64"]
    raise TypeError("output must be float32 or float64")


def reconstruct_integrals(tables: Tables, quads, out, lookup="separable", counters=None,
                          stream=None):
    """cc_reconstruct_integrals.  quads: int32[n, 4] ids, int16[n, 4] ids (bit patterns of
    uint16, basis <= 65536) or int8[n, 4, 4] vectors;
    out: float32 / float64 [n]; counters: None or int64[3] (added to)."""
    import torch
    if quads.dtype == torch.int32:
        fmt, n = FORMATS["ids"], quads.shape[0]
    elif quads.dtype == torch.int8:
        fmt, n = FORMATS["vec"], quads.shape[0]
    elif quads.dtype in (torch.int16, getattr(torch, "uint16", torch.int16)):
        fmt, n = FORMATS["ids16"], quads.shape[0]   # the 16 bits of each id, unsigned
    else:
        raise TypeError("quads must be int32 ids, int16/uint16 ids or int8 vectors")
    if n and (not quads.is_contiguous() or quads[0].numel() * quads.element_size() !=
              (8 if fmt == FORMATS["ids16"] else 16)):
        raise ValueError("quads must be contiguous rows of four ids (or four int8x4 vectors)")
    if out.numel() < n:
        raise ValueError("output too small")
    if counters is not None and (counters.dtype != torch.int64 or counters.numel() < 3):
        raise TypeError("counters must be int64[3]")
    _check("cc_reconstruct_integrals", lib().cc_reconstruct_integrals(
        tables.handle, _ptr(quads), n, fmt, LOOKUPS[lookup], _prec_of(out), _ptr(out),
        _ptr(counters), _stream(stream, out)))
    return out


def pair_matrix(tables: Tables, row0, nrows, out, lookup="separable", stream=None):
    """cc_pair_matrix: out[nrows, Nb] = V(n_j - n_i), i = row0 .. row0 + nrows - 1."""
    if out.numel() < nrows * tables.info["Nb"]:
        raise ValueError("output too small")
    _check("cc_pair_matrix", lib().cc_pair_matrix(
        tables.handle, int(row0), int(nrows), LOOKUPS[lookup], _prec_of(out), _ptr(out),
        _stream(stream, out)))
    return out


def exchange_sums(tables: Tables, R_F, eps, Ex, precision=None, stream=None):
    """cc_exchange_sums: eps[(2R+1)^3] and Ex[2] = (E_x^sigma, total), FP64 reduction."""
    import torch
    Mg = tables.info["Mg"]
    if eps.numel() < Mg ** 3 or Ex.dtype != torch.float64 or Ex.numel() < 2:
        raise ValueError("eps must hold (2R+1)^3 values and Ex two float64")
    if precision is None:
        prec = _prec_of(eps)
    else:
        prec = PRECISIONS[precision]
        need = torch.float64 if prec == 0 else torch.float32
        if eps.dtype != need:
            raise TypeError(f"eps must be {need} for {precision}")
    _check("cc_exchange_sums", lib().cc_exchange_sums(
        tables.handle, int(R_F), prec, _ptr(eps), _ptr(Ex), _stream(stream, eps)))
    return eps, Ex


def exchange_sums_noalloc(tables: Tables, R_F, eps, Ex, stream=None):
    """cc_exchange_sums_noalloc: the FP32 exchange sums with all scratch in the library's
    fixed device array (no allocation; R <= 31; calls must not overlap on the GPU)."""
    import torch
    Mg = tables.info["Mg"]
    if eps.dtype != torch.float32 or eps.numel() < Mg ** 3:
        raise ValueError("eps must be float32 with (2R+1)^3 values")
    if Ex.dtype != torch.float64 or Ex.numel() < 2:
        raise ValueError("Ex must hold two float64")
    _check("cc_exchange_sums_noalloc", lib().cc_exchange_sums_noalloc(
        tables.handle, int(R_F), _ptr(eps), _ptr(Ex), _stream(stream, eps)))
    return eps, Ex


def mixed_status(tables: Tables, clear=True) -> int:
    """Error word of the tensor-core path (0 = fine; see cc_mixed_status)."""
    code = ctypes.c_int(0)
    lib().cc_mixed_status(tables.handle, ctypes.byref(code), 1 if clear else 0)
    return code.value


TILES = {0: "64x64", 1: "32x32", 2: "64x32"}


def autotune_gemm(tables: Tables, R_F, precision="fp32", reps=3, stream=None):
    """cc_autotune_gemm: time the dense SIMT chain with every tile pair, keep the fastest
    for this grid side and precision; returns {"small": .., "large": .., "ms": ..}."""
    choice = np.zeros(2, dtype=np.int32)
    ms = ctypes.c_float(0.0)
    st = _stream(stream)
    _check("cc_autotune_gemm", lib().cc_autotune_gemm(
        tables.handle, PRECISIONS[precision], int(R_F), int(reps), choice.ctypes.data,
        ctypes.byref(ms), st))
    return {"small": TILES[int(choice[0])], "large": TILES[int(choice[1])], "ms": ms.value}


def gemm_tiles_tuned(precision, Mg):
    """The measured tile pair for a grid side (cc_gemm_tiles_tuned), or None."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check("cc_gemm_tiles_tuned", lib().cc_gemm_tiles_tuned(PRECISIONS[precision], int(Mg),
                                                            ctypes.byref(a), ctypes.byref(b)))
    return None if a.value < 0 else {"small": TILES[a.value], "large": TILES[b.value]}


def set_gemm_tiles(precision, small_tile, large_tile, threshold=-1):
    _check("cc_set_gemm_tiles", lib().cc_set_gemm_tiles(PRECISIONS[precision], small_tile,
                                                        large_tile, threshold))


class Batch:
    """Many independent boxes whose exchange sums run in one persistent, graph-captured
    launch (cc_batch_*).  boxes: dicts with R, L, R_F, S and optionally kernel, n_sub,
    q_tail, alpha_c, prune_tol."""

    def __init__(self, boxes, stream=None):
        arr = (Box * len(boxes))()
        for i, b in enumerate(boxes):
            k = b.get("kernel", "periodic")
            arr[i].p = TableParams(KERNELS[k] if isinstance(k, str) else int(k), int(b["R"]),
                                   float(b["L"]), int(b["S"]), int(b.get("n_sub", -1)),
                                   int(b.get("q_tail", -1)), float(b.get("alpha_c", 1.0)),
                                   float(b.get("prune_tol", -1.0)), float(b.get("ratio", 5.0)))
            arr[i].R_F = int(b["R_F"])
        h = ctypes.c_void_p()
        _check("cc_batch_create", lib().cc_batch_create(arr, len(boxes), _stream(stream),
                                                        ctypes.byref(h)))
        self._h = h
        n = ctypes.c_int()
        items = ctypes.c_int()
        nbytes = ctypes.c_size_t()
        offs = np.zeros(len(boxes) + 1, dtype=np.int64)
        _check("cc_batch_info", lib().cc_batch_info(h, ctypes.byref(n), offs.ctypes.data,
                                                    ctypes.byref(items), ctypes.byref(nbytes)))
        self.nbox = n.value
        self.offsets = offs
        self.n_items = items.value
        self.device_bytes = nbytes.value

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("batch was freed")
        return self._h

    def exchange(self, eps, Ex, precision=None, stream=None):
        """eps: float32 / float64 [offsets[-1]]; Ex: float64 [nbox, 2].  precision None
        follows eps's dtype; "bf16x3" runs the tensor-core form (eps float32)."""
        import torch
        if eps.numel() < int(self.offsets[-1]) or Ex.numel() < 2 * self.nbox:
            raise ValueError("output too small")
        if precision is None:
            prec = _prec_of(eps)
        else:
            prec = PRECISIONS[precision]
            if eps.dtype != (torch.float64 if prec == 0 else torch.float32):
                raise TypeError("eps dtype does not match the precision")
        _check("cc_batch_exchange", lib().cc_batch_exchange(
            self.handle, prec, _ptr(eps), _ptr(Ex), _stream(stream, eps)))
        return eps, Ex

    def set_plan(self, ctas_per_sm=4, oversub=2):
        _check("cc_batch_set_plan", lib().cc_batch_set_plan(self.handle, ctas_per_sm, oversub))

    def tune(self, eps, Ex, reps=5, precision=None, stream=None):
        """cc_batch_tune.  SIMT engine (FP32 / FP64 by the dtype of eps): launch shape;
        precision="bf16x3": the tensor-core engine's work decomposition."""
        prec = PRECISIONS[precision] if precision else _prec_of(eps)
        choice = np.zeros(2, dtype=np.int32)
        ms = ctypes.c_float()
        _check("cc_batch_tune", lib().cc_batch_tune(
            self.handle, prec, _ptr(eps), _ptr(Ex), int(reps), choice.ctypes.data,
            ctypes.byref(ms), _stream(stream, eps)))
        if prec == PRECISIONS["bf16x3"]:
            return {"order": ["as given", "by decreasing cost"][int(choice[0])],
                    "cut": ["equal units", "equal estimated cost"][int(choice[1])],
                    "ms": ms.value}
        n = ctypes.c_int()
        items = ctypes.c_int()
        lib().cc_batch_info(self.handle, ctypes.byref(n), None, ctypes.byref(items), None)
        self.n_items = items.value
        return {"ctas_per_sm": int(choice[0]), "oversub": int(choice[1]), "ms": ms.value}

    def free(self):
        if self._h is not None:
            _check("cc_batch_free", lib().cc_batch_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
