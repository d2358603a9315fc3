"""Thin ctypes binding of libvtm (include/vtm.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  PyTorch is used by callers for
device memory and streams; device tensors are passed as raw pointers (``tensor.data_ptr()``) and
streams as ``torch.cuda.Stream.cuda_stream``.  Importing this module loads the library and fails
loudly when it has not been built (``python -m paper_0807_1949_gb300.build``).

The names mirror the C ABI: ``partition_evs`` -> ``vtm_partition_evs``, ``Solver`` wraps
``vtm_setup`` / ``vtm_iterate`` / ``vtm_solve`` / ``vtm_get_state`` ... .
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libvtm.so")

VTM_OK = 0
STATUS = {0: "OK", 1: "INVALID", 2: "NOT_SYMMETRIC", 3: "NOT_CONFORMAL", 4: "NOT_SPD", 5: "NOT_CONVERGED",
          6: "DIVERGED", 7: "TIMEOUT", 8: "CUDA", 9: "OOM"}
PART_GRID, PART_OWNERS, PART_EXPLICIT, PART_ELEMENTS, PART_CONFORMAL = 1, 2, 3, 4, 5
Z_UNIFORM, Z_EXPLICIT, Z_MATCHED, Z_LEARNED = 0, 1, 2, 3
MLP_IN, MLP_HIDDEN, MLP_PARAMS = 8, 64, 4801
FP64, FP32 = 0, 1


class VTMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vtm error {code} ({STATUS.get(code, '?')}): {msg}")
        self.code = code


class _CSR(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class _Spec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dims", C.c_int32 * 3), ("block", C.c_int32 * 3), ("npieces", C.c_int32),
                ("owner_ptr", C.c_void_p), ("owner_piece", C.c_void_p), ("nlines", C.c_int64),
                ("line_vertex", C.c_void_p), ("line_piece_a", C.c_void_p), ("line_piece_b", C.c_void_p),
                ("piece_ptr", C.c_void_p), ("copy_vertex", C.c_void_p), ("copy_share", C.c_void_p),
                ("local_rowptr", C.c_void_p), ("local_col", C.c_void_p), ("local_val", C.c_void_p),
                ("ncopy_lines", C.c_int64), ("line_copy_a", C.c_void_p), ("line_copy_b", C.c_void_p),
                ("nelem", C.c_int64), ("nodes_per_elem", C.c_int32), ("nnodes", C.c_int64),
                ("elem_nodes", C.c_void_p), ("elem_mats", C.c_void_p), ("node_unknown", C.c_void_p),
                ("elem_piece", C.c_void_p), ("elem_coords", C.c_void_p), ("coord_dim", C.c_int32),
                ("home", C.c_void_p), ("lam", C.c_double)]


class PartitionInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("npieces", C.c_int32), ("ncopies", C.c_int64), ("nlines", C.c_int64),
                ("nboundary", C.c_int64), ("max_piece", C.c_int64)]


class _Opts(C.Structure):
    _fields_ = [("z_mode", C.c_int32), ("z_uniform", C.c_double), ("z_lines", C.c_void_p), ("precision", C.c_int32),
                ("nrhs", C.c_int32), ("check_every", C.c_int32), ("inner_reduction", C.c_double),
                ("model", C.c_void_p), ("wait_polls", C.c_int64), ("withhold_slab", C.c_int32),
                ("sweep_variant", C.c_int32), ("sweep_form", C.c_int32),
                ("port_storage", C.c_int32), ("ncouplings", C.c_int64), ("couplings", C.c_void_p),
                ("coupling_y", C.c_void_p)]


class SolverInfo(C.Structure):
    _fields_ = [("npieces", C.c_int32), ("ncopies", C.c_int64), ("nends", C.c_int64), ("nrhs", C.c_int32),
                ("precision", C.c_int32), ("block_rows", C.c_int32), ("factor_entries", C.c_int64),
                ("band_entries", C.c_int64), ("factor_bytes", C.c_int64), ("max_halfband", C.c_int64),
                ("setup_ms", C.c_double), ("factor_ms", C.c_double), ("sweep_stages", C.c_int32),
                ("sweep_ctas_per_sm", C.c_int32), ("sweep_ms", C.c_double), ("flagged_pieces", C.c_int32),
                ("sweep_variant", C.c_int32), ("sweep_form", C.c_int32), ("port_bytes", C.c_int64),
                ("port_setup_ms", C.c_double), ("port_sweep_ms", C.c_double),
                ("nports", C.c_int64), ("port_storage_bits", C.c_int32), ("factor_tc", C.c_int32),
                ("ncouplings", C.c_int64), ("band_tc", C.c_int32), ("band_tc_bytes", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("checks", C.c_int32), ("restarts", C.c_int32), ("rel_residual", C.c_double),
                ("solve_ms", C.c_double), ("launches", C.c_int32)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libvtm.so is not built ({_LIB_PATH}); run __graft_entry__.build() or "
                          "python -m paper_0807_1949_gb300.build")
    try:  # make torch's CUDA runtime the one the library binds to, when torch is present
        import torch  # noqa: F401
    except Exception:
        pass
    lib = C.CDLL(_LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "vtm_partition_evs": (C.c_int, [vp, vp, vp]),
        "vtm_partition_get_info": (C.c_int, [vp, vp]),
        "vtm_rcb": (C.c_int, [vp, i64, i32, i32, vp]),
        "vtm_partition_get_piece": (C.c_int, [vp, i32, vp, vp, vp, vp, vp, vp, vp]),
        "vtm_partition_get_lines": (C.c_int, [vp, vp]),
        "vtm_partition_line_pairs": (C.c_int, [vp, vp, vp, vp]),
        "vtm_partition_destroy": (None, [vp]),
        "vtm_setup": (C.c_int, [vp, vp, vp, vp]),
        "vtm_solver_get_info": (C.c_int, [vp, vp]),
        "vtm_solver_get_history": (C.c_int, [vp, vp, vp, vp, vp]),
        "vtm_solver_destroy": (None, [vp]),
        "vtm_set_rhs": (C.c_int, [vp, vp, i64]),
        "vtm_reset": (C.c_int, [vp]),
        "vtm_iterate": (C.c_int, [vp, i32]),
        "vtm_solve": (C.c_int, [vp, vp, vp, i64, dbl, i32, vp]),
        "vtm_get_state": (C.c_int, [vp, vp]),
        "vtm_input_impedances": (C.c_int, [vp, vp]),
        "vtm_solver_get_impedances": (C.c_int, [vp, vp]),
        "vtm_solver_get_piece_precision": (C.c_int, [vp, vp]),
        "vtm_line_features": (C.c_int, [vp, vp]),
        "vtm_mlp_create": (C.c_int, [C.c_uint64, vp]),
        "vtm_mlp_destroy": (None, [vp]),
        "vtm_mlp_get_params": (C.c_int, [vp, vp]),
        "vtm_mlp_set_params": (C.c_int, [vp, vp]),
        "vtm_mlp_get_grads": (C.c_int, [vp, vp]),
        "vtm_mlp_forward": (C.c_int, [vp, vp, vp, i64, vp]),
        "vtm_mlp_loss_grad": (C.c_int, [vp, vp, vp, i64, vp, vp]),
        "vtm_mlp_adam_step": (C.c_int, [vp, C.c_float, C.c_float, C.c_float, C.c_float, vp]),
        "vtm_set_state": (C.c_int, [vp, vp]),
        "vtm_get_copies": (C.c_int, [vp, vp]),
        "vtm_relative_residual_noalloc": (C.c_int, [i64, vp, vp, vp, i32, vp, i64, vp, i64, vp, vp]),
        "vtm_last_error": (C.c_char_p, []),
        "vtm_version": (C.c_int, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def library_path() -> str:
    return _LIB_PATH


def _check(code: int, allow=()):
    if code != VTM_OK and code not in allow:
        raise VTMError(code, _lib.vtm_last_error().decode())
    return code


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _arr(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


class Partition:
    """Handle of a split electric graph (vtm_partition)."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.vtm_partition_destroy(self._h)
            self._h = C.c_void_p(None)

    @property
    def handle(self):
        return self._h

    def info(self) -> PartitionInfo:
        i = PartitionInfo()
        _check(_lib.vtm_partition_get_info(self._h, C.byref(i)))
        return i

    def piece(self, j: int):
        """(vertices, shares, local CSR (rowptr, col, val)) of subgraph j."""
        nj, nnz = C.c_int64(), C.c_int64()
        _check(_lib.vtm_partition_get_piece(self._h, j, C.byref(nj), C.byref(nnz), None, None, None, None, None))
        v = np.empty(nj.value, np.int64)
        s = np.empty(nj.value, np.float64)
        rp = np.empty(nj.value + 1, np.int64)
        col = np.empty(nnz.value, np.int32)
        val = np.empty(nnz.value, np.float64)
        _check(_lib.vtm_partition_get_piece(self._h, j, None, None, _ptr(v), _ptr(s), _ptr(rp), _ptr(col), _ptr(val)))
        return v, s, (rp, col, val)

    def lines(self) -> np.ndarray:
        """(nlines, 4) int64: (piece_a, local_a, piece_b, local_b)."""
        q = np.empty((self.info().nlines, 4), np.int64)
        _check(_lib.vtm_partition_get_lines(self._h, _ptr(q)))
        return q

    def line_pairs(self) -> tuple[np.ndarray, np.ndarray]:
        """Candidate couplings of §7.2 (vtm_partition_line_pairs): (count, 2) int64 line pairs of
        one bundle whose copies are neighbours in both subgraphs, and |a_ik| of each pair."""
        cnt = C.c_int64()
        _check(_lib.vtm_partition_line_pairs(self._h, C.byref(cnt), None, None))
        pr = np.empty((cnt.value, 2), np.int64)
        w = np.empty(cnt.value, np.float64)
        _check(_lib.vtm_partition_line_pairs(self._h, C.byref(cnt), _ptr(pr), _ptr(w)))
        return pr, w

    def line_features(self) -> np.ndarray:
        """(nends, 8) float32 features of every line end (vtm_line_features)."""
        f = np.empty((2 * self.info().nlines, MLP_IN), np.float32)
        _check(_lib.vtm_line_features(self._h, _ptr(f)))
        return f


def _csr_struct(A):
    rowptr, col, val = _arr(A.rowptr, np.int64), _arr(A.col, np.int32), _arr(A.val, np.float64)
    s = _CSR(n=A.n, nnz=len(val), rowptr=rowptr.ctypes.data, col=col.ctypes.data, val=val.ctypes.data)
    return s, (rowptr, col, val)


def partition_evs(A, kind: str = "grid", *, dims=None, block=None, owners=None, lines=None, explicit=None,
                  elements=None, npieces=None, home=None, lam: float = 0.5) -> Partition:
    """vtm_partition_evs.  A: object with n, rowptr, col, val (inputs.CSR).

    kind="grid":     dims=(nx, ny[, nz]), block=(sx, sy[, sz]).
    kind="owners":   owners=list of sorted piece tuples per vertex, lines=[(vertex, pa, pb), ...].
    kind="explicit": explicit=dict(piece_ptr, copy_vertex, copy_share, local_rowptr, local_col, local_val,
                     line_copy_a, line_copy_b).
    kind="elements": elements=dict(elem_nodes (m, k), elem_mats (m, k, k), node_unknown, and either
                     elem_piece (m,) or elem_coords (m, dim) with npieces).
    kind="conformal": home=(n,) home subgraph of every vertex, lam in (0, 1): the general SPD split
                     of App. 1 (dense; n <= 8192).
    """
    csr, keep = _csr_struct(A)
    sp = _Spec()
    hold = [keep]
    if kind == "grid":
        d = list(dims) + [1] * (3 - len(dims))
        b = list(block) + [1] * (3 - len(block))
        sp.kind = PART_GRID
        sp.dims[:] = d
        sp.block[:] = b
    elif kind == "owners":
        ptr = np.zeros(len(owners) + 1, np.int64)
        ptr[1:] = np.cumsum([len(o) for o in owners])
        pieces = _arr(np.concatenate([np.asarray(o, np.int32) for o in owners]), np.int32)
        lv = _arr([t[0] for t in lines], np.int64)
        la = _arr([t[1] for t in lines], np.int32)
        lb = _arr([t[2] for t in lines], np.int32)
        hold += [ptr, pieces, lv, la, lb]
        sp.kind = PART_OWNERS
        sp.npieces = int(pieces.max()) + 1
        sp.owner_ptr, sp.owner_piece = ptr.ctypes.data, pieces.ctypes.data
        sp.nlines, sp.line_vertex, sp.line_piece_a, sp.line_piece_b = len(lv), lv.ctypes.data, la.ctypes.data, lb.ctypes.data
    elif kind == "explicit":
        e = {k: v for k, v in explicit.items()}
        arrs = dict(piece_ptr=_arr(e["piece_ptr"], np.int64), copy_vertex=_arr(e["copy_vertex"], np.int64),
                    copy_share=_arr(e["copy_share"], np.float64), local_rowptr=_arr(e["local_rowptr"], np.int64),
                    local_col=_arr(e["local_col"], np.int32), local_val=_arr(e["local_val"], np.float64),
                    line_copy_a=_arr(e["line_copy_a"], np.int64), line_copy_b=_arr(e["line_copy_b"], np.int64))
        hold.append(arrs)
        sp.kind = PART_EXPLICIT
        sp.npieces = len(arrs["piece_ptr"]) - 1
        for k in ("piece_ptr", "copy_vertex", "copy_share", "local_rowptr", "local_col", "local_val",
                  "line_copy_a", "line_copy_b"):
            setattr(sp, k, arrs[k].ctypes.data)
        sp.ncopy_lines = len(arrs["line_copy_a"])
    elif kind == "elements":
        e = elements
        en = _arr(e["elem_nodes"], np.int64)
        em = _arr(e["elem_mats"], np.float64)
        nu = _arr(e["node_unknown"], np.int64)
        hold += [en, em, nu]
        sp.kind = PART_ELEMENTS
        sp.nelem, sp.nodes_per_elem, sp.nnodes = en.shape[0], en.shape[1], len(nu)
        sp.elem_nodes, sp.elem_mats, sp.node_unknown = en.ctypes.data, em.ctypes.data, nu.ctypes.data
        if e.get("elem_piece") is not None:
            ep = _arr(e["elem_piece"], np.int32)
            hold.append(ep)
            sp.elem_piece = ep.ctypes.data
            sp.npieces = int(npieces or ep.max() + 1)
        else:
            ec = _arr(e["elem_coords"], np.float64)
            hold.append(ec)
            sp.elem_coords, sp.coord_dim = ec.ctypes.data, ec.shape[1]
            sp.npieces = int(npieces)
    elif kind == "conformal":
        hm = _arr(home, np.int32)
        hold.append(hm)
        sp.kind = PART_CONFORMAL
        sp.npieces = int(npieces or hm.max() + 1)
        sp.home, sp.lam = hm.ctypes.data, float(lam)
    else:
        raise ValueError(kind)
    h = C.c_void_p()
    _check(_lib.vtm_partition_evs(C.byref(csr), C.byref(sp), C.byref(h)))
    return Partition(h.value)


def rcb(coords, nparts: int) -> np.ndarray:
    """vtm_rcb: recursive coordinate bisection of points (n, dim) into nparts subgraph ids."""
    c = _arr(coords, np.float64)
    out = np.empty(len(c), np.int32)
    _check(_lib.vtm_rcb(_ptr(c), len(c), c.shape[1], int(nparts), _ptr(out)))
    return out


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _data_ptr(x):
    """(pointer, keepalive) of a torch tensor (host or device) or numpy array, float64 contiguous."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous() or str(x.dtype) != "torch.float64":
            raise ValueError("tensors must be contiguous float64")
        return C.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a.ctypes.data_as(C.c_void_p), a


class Solver:
    """vtm_setup / vtm_iterate / vtm_solve on one partition.

    z: scalar (uniform), per-line array (order of Partition.lines()), "matched" (§7.1 rule,
       starting from z_init on every line), or an ``MLP`` (learned impedances).
    precision: "fp64" or "fp32".  nrhs: 1, 2, 4, 8, 16 or 32.
    sweep_variant: "auto" or "single" (one CTA works each block step in turn; the setup-time
    autotuner picks the staging depth) or "pipelined" (warp 0 finishes block k while the other
    warps prepare block k+1; nrhs <= 2; opt-in only, it measured slower everywhere) or "simt"
    (FP32, nrhs 16 / 32: the multi-RHS band sweep without its tensor-core products).
    coupling: coupled lines of §7.2.  None (uncoupled), a number gamma (every candidate pair of
    Partition.line_pairs() gets the conductance gamma |a_ik|), or (pairs (m, 2), y (m,)).
    Right-hand sides / solutions: (nrhs, n) float64 arrays or tensors, host or device.
    """

    def __init__(self, part: Partition, z=1.0, precision: str = "fp64", nrhs: int = 1, stream=None,
                 check_every: int = 10, inner_reduction: float = 0.0, z_init: float = 1.0,
                 wait_polls: int = 0, withhold_slab: int = -1, sweep_variant: str = "auto",
                 form: str = "auto", port_storage: str = "native", coupling=None):
        o = _Opts()
        ckeep = None
        if coupling is not None:
            if isinstance(coupling, (int, float, np.integer, np.floating)):
                pairs, w = part.line_pairs()
                y = float(coupling) * w
            else:
                pairs, y = coupling
            pairs, y = _arr(pairs, np.int64).reshape(-1, 2), _arr(y, np.float64).reshape(-1)
            if len(pairs) != len(y):
                raise ValueError("coupling: one conductance per pair")
            o.ncouplings, o.couplings, o.coupling_y = len(y), pairs.ctypes.data, y.ctypes.data
            ckeep = (pairs, y)
        o.port_storage = {"native": 0, "fp16": 1, "fp16-auto": 2}[port_storage]
        o.sweep_variant = {"auto": 0, "single": 1, "pipelined": 2, "simt": 3}[sweep_variant]
        o.sweep_form = {"auto": 0, "band": 1, "port": 2}[form]
        zarr = None
        if isinstance(z, MLP):
            o.z_mode, o.model = Z_LEARNED, z.handle.value
        elif isinstance(z, str):
            if z != "matched":
                raise ValueError(z)
            o.z_mode, o.z_uniform = Z_MATCHED, float(z_init)
        elif np.ndim(z) == 0:
            o.z_mode, o.z_uniform = Z_UNIFORM, float(z)
        else:
            zarr = _arr(z, np.float64)
            o.z_mode, o.z_lines = Z_EXPLICIT, zarr.ctypes.data
        o.precision = {"fp64": FP64, "fp32": FP32}[precision]
        o.nrhs = nrhs
        o.check_every = check_every
        o.inner_reduction = inner_reduction
        o.wait_polls = int(wait_polls)
        o.withhold_slab = int(withhold_slab) + 1 if withhold_slab >= 0 else 0
        self.nrhs = nrhs
        self.n = part.info().n
        h = C.c_void_p()
        _check(_lib.vtm_setup(part.handle, C.byref(o), _stream_handle(stream), C.byref(h)))
        self._h = h
        self._zkeep = (zarr, ckeep)

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.vtm_solver_destroy(self._h)
            self._h = C.c_void_p(None)

    def info(self) -> SolverInfo:
        i = SolverInfo()
        _check(_lib.vtm_solver_get_info(self._h, C.byref(i)))
        return i

    def set_rhs(self, b):
        p, keep = _data_ptr(b)
        _check(_lib.vtm_set_rhs(self._h, p, self.n))

    def reset(self):
        _check(_lib.vtm_reset(self._h))

    def iterate(self, sweeps: int):
        _check(_lib.vtm_iterate(self._h, int(sweeps)))

    def solve(self, b, x, rtol: float = 1e-10, maxit: int = 10000, raise_on_fail: bool = True) -> Stats:
        pb, kb = _data_ptr(b)
        px, kx = _data_ptr(x)
        st = Stats()
        code = _lib.vtm_solve(self._h, pb, px, self.n, float(rtol), int(maxit), C.byref(st))
        if raise_on_fail:
            _check(code)
        st.status = code
        return st

    def history(self) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Residual checks of the last solve (vtm_solver_get_history): sweeps at each check, max
        relative residual, max inner (defect-correction phase) residual."""
        cnt = C.c_int32()
        _check(_lib.vtm_solver_get_history(self._h, C.byref(cnt), None, None, None))
        sw = np.empty(cnt.value, np.int32)
        rel = np.empty(cnt.value, np.float64)
        inner = np.empty(cnt.value, np.float64)
        _check(_lib.vtm_solver_get_history(self._h, C.byref(cnt), _ptr(sw), _ptr(rel), _ptr(inner)))
        return sw, rel, inner

    def impedances(self) -> np.ndarray:
        """Line impedances in use, (nlines,)."""
        z = np.empty(self.info().nends // 2, np.float64)
        _check(_lib.vtm_solver_get_impedances(self._h, _ptr(z)))
        return z

    def piece_precision(self) -> np.ndarray:
        """32 or 64 per subgraph (FP32 solvers refactor flagged subgraphs in FP64)."""
        b = np.empty(self.info().npieces, np.int32)
        _check(_lib.vtm_solver_get_piece_precision(self._h, _ptr(b)))
        return b

    def input_impedances(self) -> np.ndarray:
        """Input impedance of every line end (Def. 7.1, other lines terminated), (nends,)."""
        r = np.empty(self.info().nends, np.float64)
        _check(_lib.vtm_input_impedances(self._h, _ptr(r)))
        return r

    def get_state(self) -> np.ndarray:
        """Outgoing waves of the last sweep, (nrhs, nends), end 2t / 2t+1 = sides a / b of line t."""
        ne = self.info().nends
        w = np.empty((self.nrhs, ne), np.float64)
        _check(_lib.vtm_get_state(self._h, _ptr(w)))
        return w

    def set_state(self, waves):
        w = _arr(waves, np.float64)
        _check(_lib.vtm_set_state(self._h, _ptr(w)))

    def copies(self) -> np.ndarray:
        """Last local solutions, (nrhs, ncopies), copies piece by piece in local order."""
        nc = self.info().ncopies
        x = np.empty((self.nrhs, nc), np.float64)
        _check(_lib.vtm_get_copies(self._h, _ptr(x)))
        return x


class MLP:
    """Learned impedance model (vtm_mlp_*): 8 -> 64 -> 64 -> 1, BF16 weights, FP32 accumulate."""

    def __init__(self, seed: int = 0):
        h = C.c_void_p()
        _check(_lib.vtm_mlp_create(C.c_uint64(seed), C.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.vtm_mlp_destroy(self._h)
            self._h = C.c_void_p(None)

    @property
    def handle(self):
        return self._h

    def get_params(self) -> np.ndarray:
        p = np.empty(MLP_PARAMS, np.float32)
        _check(_lib.vtm_mlp_get_params(self._h, _ptr(p)))
        return p

    def set_params(self, p):
        a = _arr(p, np.float32)
        assert a.size == MLP_PARAMS
        _check(_lib.vtm_mlp_set_params(self._h, _ptr(a)))

    def get_grads(self) -> np.ndarray:
        g = np.empty(MLP_PARAMS, np.float32)
        _check(_lib.vtm_mlp_get_grads(self._h, _ptr(g)))
        return g

    def forward(self, X, y, stream=None):
        """X: CUDA float32 (n, 8); y: CUDA float32 (n,)."""
        _check(_lib.vtm_mlp_forward(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()), int(X.shape[0]),
                                    _stream_handle(stream)))

    def loss_grad(self, X, t, stream=None) -> float:
        l = C.c_float()
        _check(_lib.vtm_mlp_loss_grad(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(t.data_ptr()), int(X.shape[0]),
                                      C.byref(l), _stream_handle(stream)))
        return l.value

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(_lib.vtm_mlp_adam_step(self._h, lr, beta1, beta2, eps, _stream_handle(stream)))


def relative_residual_noalloc(rowptr, col, val, b, x, rel, stream=None):
    """vtm_relative_residual_noalloc on device tensors: rel[r] = ||b_r - A x_r|| / ||b_r||.

    For callers that must not allocate device memory at call time; the library uses a fixed
    128-byte device array as its only scratch.  rowptr (int64, n + 1), col (int32), val (float64),
    b and x (float64, shape (nrhs, n) or (n,), contiguous, same shape) and rel (float64, at least
    nrhs entries) are CUDA tensors on one device; the call runs on that device, asynchronously on
    ``stream``.  Arguments are checked here so that no kernel reads or writes past a tensor.
    """
    want = (("rowptr", rowptr, "torch.int64"), ("col", col, "torch.int32"), ("val", val, "torch.float64"),
            ("b", b, "torch.float64"), ("x", x, "torch.float64"), ("rel", rel, "torch.float64"))
    for name, t, dt in want:
        if not hasattr(t, "data_ptr") or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if str(t.dtype) != dt or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dt.split('.')[1]} tensor")
        if t.device != b.device:
            raise ValueError(f"{name} is on {t.device}, b on {b.device}: all tensors must share one device")
    if rowptr.dim() != 1 or rowptr.numel() < 2:
        raise ValueError("rowptr must hold n + 1 >= 2 entries")
    n = int(rowptr.numel()) - 1
    if col.numel() != val.numel():
        raise ValueError("col and val must have one entry per stored element")
    if tuple(x.shape) != tuple(b.shape) or b.dim() not in (1, 2) or b.shape[-1] != n:
        raise ValueError(f"b and x must both have shape (nrhs, {n}) or ({n},)")
    nrhs = int(b.shape[0]) if b.dim() == 2 else 1
    if rel.numel() < nrhs:
        raise ValueError(f"rel holds {rel.numel()} entries, {nrhs} needed")
    import torch

    with torch.cuda.device(b.device):
        _check(_lib.vtm_relative_residual_noalloc(n, C.c_void_p(rowptr.data_ptr()), C.c_void_p(col.data_ptr()),
                                                  C.c_void_p(val.data_ptr()), nrhs, C.c_void_p(b.data_ptr()), n,
                                                  C.c_void_p(x.data_ptr()), n, C.c_void_p(rel.data_ptr()),
                                                  _stream_handle(stream)))


def version() -> int:
    return _lib.vtm_version()
