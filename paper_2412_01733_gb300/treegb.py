"""Thin Python binding of libtreegb.so (include/treegb.h), argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
only checks tensor shapes/dtypes/devices and passes raw device pointers and
the current CUDA stream through ctypes.  PyTorch supplies device memory and
streams.  If the library has not been built, importing works but the first
call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtreegb.so")

TREE_OK, TREE_ERR_ARG, TREE_ERR_CUDA, TREE_ERR_ALLOC, TREE_ERR_CAPACITY, TREE_ERR_STATE, TREE_ERR_DEVICE = range(7)
DEV_NONFINITE, DEV_STACK, DEV_NODES, DEV_TIMEOUT, DEV_LIST = 0x01, 0x02, 0x04, 0x08, 0x10
F32, F64 = 0, 1
FLAG_EMIT_LISTS = 0x1
FLAG_LISTS_ONLY = 0x2
PHASES = ("box", "keys", "sort", "octree", "gather", "moments", "walk", "lists", "diag", "direct", "adjoint",
          "h2d", "d2h")


class TreeParams(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("eps", ctypes.c_double), ("theta", ctypes.c_double),
                ("order", ctypes.c_int32), ("leaf_cap", ctypes.c_int32), ("group_size", ctypes.c_int32),
                ("stack_depth", ctypes.c_int32), ("precision", ctypes.c_int32), ("kahan", ctypes.c_int32),
                ("group_split", ctypes.c_int32), ("node_cap", ctypes.c_int64)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("depth", ctypes.c_int32),
                ("box_k", ctypes.c_int32), ("box_lo", ctypes.c_double * 3),
                ("level_offset", ctypes.c_int64 * 23), ("pp_pairs", ctypes.c_int64),
                ("pc_pairs", ctypes.c_int64), ("max_stack", ctypes.c_int64), ("n_groups", ctypes.c_int64),
                ("list_pc", ctypes.c_int64), ("list_pp", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("n_segments", ctypes.c_int64)]


class TreeError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn}: {status_string(code)} ({code})")
        self.code = code


_lib = None
_vp, _i64, _i32, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double

_SIGNATURES = {
    "tree_params_default": [ctypes.POINTER(TreeParams)],
    "tree_workspace_create": [_i64, ctypes.POINTER(TreeParams), ctypes.POINTER(_vp)],
    "tree_workspace_destroy": [_vp],
    "tree_set_params": [_vp, ctypes.POINTER(TreeParams)],
    "tree_get_params": [_vp, ctypes.POINTER(TreeParams)],
    "tree_build": [_vp, _vp, _i64, _i32, _vp],
    "tree_moments": [_vp, _vp, _vp, _vp],
    "tree_forces": [_vp, _vp, _vp, _i32, _vp],
    "tree_accel": [_vp, _vp, _vp, _i64, _vp, _vp, _vp],
    "tree_forces_adjoint": [_vp, _vp, _vp, _vp, _vp, _vp],
    "tree_energy_vjp": [_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp],
    "leapfrog_adjoint_step": [_vp, _vp, _vp, _vp, _vp, _vp, _dbl, _vp],
    "leapfrog_step": [_vp, _vp, _vp, _vp, _vp, _vp, _dbl, _i64, _vp],
    "leapfrog_step_host": [_vp, _vp, _vp, _vp, _vp, _vp, _dbl, _i64, _vp, _vp],
    "tree_diagnostics": [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp],
    "tree_direct_forces": [_vp, _vp, _vp, _i64, _i32, _vp, _i64, _vp, _vp, _vp],
    "tree_get_status": [_vp, ctypes.POINTER(_i32), _i32],
    "tree_set_waits": [_vp, _i64, _i32, _i64],
    "tree_get_info": [_vp, ctypes.POINTER(TreeInfo)],
    "tree_export_tree": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "tree_export_moments": [_vp, _vp, _vp, _vp, _vp],
    "tree_export_lists": [_vp, _vp, _vp, _vp, _vp, _vp],
    "tree_export_lists_groups": [_vp, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64), _vp,
                                 ctypes.POINTER(_i64), _vp, _vp],
    "tree_export_group_stats": [_vp, _vp, _vp],
    "tree_export_groups": [_vp, _vp, _vp],
    "tree_mac_table": [_dbl, ctypes.POINTER(_i64)],
    "tree_direct_forces_noalloc": [_vp, _vp, _i64, _i32, _dbl, _dbl, _vp, _i64, _vp, _vp, _vp],
    "tree_timing_enable": [_vp, _i32],
    "tree_timing_read": [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
    "tree_set_segments": [_vp, _i64, ctypes.POINTER(_i64)],
    "tree_get_segments": [_vp, ctypes.POINTER(_i64)],
    "tree_diagnostics_segments": [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp],
    "leapfrog_graph_capture": [_vp, _vp, _vp, _vp, _vp, _vp, _dbl, _i64, _vp],
    "leapfrog_graph_launch": [_vp, _vp],
    "tree_autotune": [ctypes.POINTER(TreeParams), _i64, ctypes.POINTER(_i64), _vp, _vp, _i64, _i32, _dbl,
                      ctypes.POINTER(TreeParams), ctypes.POINTER(_dbl), ctypes.POINTER(_i32), _vp],
    "tree_export_boxes": [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_i32)],
    "tree_fp32_peak": [ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)],
    "tree_status_string": [_i32],
    "tree_version": [],
}


def lib():
    """Load libtreegb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2412_01733_gb300.build.build() "
                               "(or __graft_entry__.build()); there is no fallback implementation")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name in ("tree_status_string", "tree_version") else ctypes.c_int
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().tree_status_string(int(code)).decode()


def version() -> str:
    return lib().tree_version().decode()


def _check(fn, code):
    if code != TREE_OK:
        raise TreeError(fn, code)


def mac_table(theta: float):
    """Integer thresholds D_l (l = 0..21): a level-l cell is far iff d2 >= D_l."""
    D = (_i64 * 22)()
    _check("tree_mac_table", lib().tree_mac_table(float(theta), D))
    return [int(v) for v in D]


def fp32_peak():
    """Measured FP32 FMA throughput of the current GPU, (scalar, packed) in TFLOP/s."""
    a, b = _dbl(0.0), _dbl(0.0)
    _check("tree_fp32_peak", lib().tree_fp32_peak(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def default_params(**kw) -> TreeParams:
    p = TreeParams()
    _check("tree_params_default", lib().tree_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"f32": F32, "f64": F64}[v]
        setattr(p, k, v)
    return p


def _offsets(offsets):
    offs = [int(o) for o in offsets]
    arr = (_i64 * len(offs))(*offs)
    return len(offs) - 1, arr


def autotune(x, m, offsets=None, reps=3, max_err=1e-3, **params):
    """Fastest (leaf_cap, group_size, stack_depth) for one force evaluation of (x, m)
    (ensemble: offsets as in Workspace.set_segments) among the candidates whose median
    relative force error against the FP64 direct sum on a fixed sample is <= max_err
    (None or <= 0: no bound).  Returns (TreeParams, table) with table rows
    (leaf_cap, group_size, stack_depth, ms, median error)."""
    base = default_params(**params)
    dt = torch.float64 if base.precision == F64 else torch.float32
    n = x.shape[1]
    if not x.is_cuda or x.dtype != dt or tuple(x.shape) != (3, n) or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA tensor (3, n) of the parameters' precision")
    if not m.is_cuda or m.dtype != dt or tuple(m.shape) != (n,) or not m.is_contiguous():
        raise ValueError("m must be a contiguous CUDA tensor (n,) of the parameters' precision")
    nseg, arr = _offsets(offsets) if offsets is not None else (0, None)
    best = TreeParams()
    rows = 32
    table = (_dbl * (5 * rows))()
    nc = _i32(rows)
    bound = 0.0 if max_err is None else float(max_err)
    _check("tree_autotune", lib().tree_autotune(ctypes.byref(base), nseg, arr, _ptr(x), _ptr(m), n, int(reps),
                                                bound, ctypes.byref(best), table, ctypes.byref(nc), _stream()))
    tab = [tuple(table[5 * i + k] for k in range(5)) for i in range(min(nc.value, rows))]
    return best, tab


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Workspace:
    """A tree workspace for up to n_max particles on the current CUDA device.

    Parameters are the fields of TreeParams (G, eps, theta, order, leaf_cap,
    group_size, stack_depth, precision, kahan, node_cap).  Arrays are torch
    CUDA tensors: x, v, a of shape (3, n); m, phi of shape (n,); dtype float32
    for precision "f32", float64 for "f64".
    """

    def __init__(self, n_max: int, **params):
        self._h = None
        self.params = default_params(**params)
        h = ctypes.c_void_p()
        _check("tree_workspace_create",
               lib().tree_workspace_create(int(n_max), ctypes.byref(self.params), ctypes.byref(h)))
        self._h = h
        self.n_max = int(n_max)
        self.n = 0
        self.dtype = torch.float64 if self.params.precision == F64 else torch.float32

    def close(self):
        if self._h is not None and _lib is not None:
            lib().tree_workspace_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- checks -----------------------------------------------------------
    def _vec(self, t, n, name):
        if t is None:
            raise ValueError(f"{name} is required")
        if not t.is_cuda or t.dtype != self.dtype or tuple(t.shape) != (3, n) or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {self.dtype} tensor of shape (3, {n})")
        return t

    def _scal(self, t, n, name, optional=False):
        if t is None:
            if optional:
                return None
            raise ValueError(f"{name} is required")
        if not t.is_cuda or t.dtype != self.dtype or tuple(t.shape) != (n,) or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {self.dtype} tensor of shape ({n},)")
        return t

    # -- the path -----------------------------------------------------------
    def set_params(self, **kw):
        p = TreeParams()
        _check("tree_get_params", lib().tree_get_params(self._h, ctypes.byref(p)))
        for k, v in kw.items():
            setattr(p, k, v)
        _check("tree_set_params", lib().tree_set_params(self._h, ctypes.byref(p)))
        self.params = p

    def set_segments(self, offsets=None):
        """Independent systems: system b = particles [offsets[b], offsets[b+1]) (see
        tree_set_segments); None returns to a single system."""
        if offsets is None:
            _check("tree_set_segments", lib().tree_set_segments(self._h, 0, None))
            return
        nseg, arr = _offsets(offsets)
        _check("tree_set_segments", lib().tree_set_segments(self._h, nseg, arr))

    def segments(self) -> int:
        v = _i64(0)
        _check("tree_get_segments", lib().tree_get_segments(self._h, ctypes.byref(v)))
        return int(v.value)

    def diagnostics_segments(self, x, v, m, phi=None, out=None):
        """Per-system FP64 diagnostics, float64 CUDA tensor (nseg, 8)."""
        n = x.shape[1]
        self._vec(x, n, "x"); self._vec(v, n, "v"); self._scal(m, n, "m")
        self._scal(phi, n, "phi", optional=True)
        if out is None:
            out = torch.empty((self.segments(), 8), dtype=torch.float64, device="cuda")
        _check("tree_diagnostics_segments", lib().tree_diagnostics_segments(self._h, _ptr(x), _ptr(v), _ptr(m),
                                                                            _ptr(phi), n, _ptr(out), _stream()))
        return out

    def graph_capture(self, x, v, m, a, tau, phi=None, diag=None):
        """Capture one leapfrog step (plus diagnostics into diag, a float64 CUDA tensor of 8,
        if given) as a CUDA graph; graph_launch() replays it on the current stream."""
        n = x.shape[1]
        self._vec(x, n, "x"); self._vec(v, n, "v"); self._scal(m, n, "m"); self._vec(a, n, "a")
        self._scal(phi, n, "phi", optional=True)
        if diag is not None and (not diag.is_cuda or diag.dtype != torch.float64 or diag.numel() < 8):
            raise ValueError("diag must be a CUDA float64 tensor of 8")
        _check("leapfrog_graph_capture", lib().leapfrog_graph_capture(self._h, _ptr(x), _ptr(v), _ptr(m), _ptr(a),
                                                                      _ptr(phi), float(tau), n, _ptr(diag)))
        self._graph_keep = (x, v, m, a, phi, diag)  # the graph holds these pointers
        self._graph_n = n

    def graph_launch(self):
        _check("leapfrog_graph_launch", lib().leapfrog_graph_launch(self._h, _stream()))
        self.n = self._graph_n

    def export_boxes(self):
        """Per-system box of the last build: (lo float64 (nseg, 3), k int32 (nseg,)) on the host."""
        ns = self.segments()
        lo = (_dbl * (3 * ns))()
        k = (_i32 * ns)()
        _check("tree_export_boxes", lib().tree_export_boxes(self._h, lo, k))
        return (torch.tensor(list(lo), dtype=torch.float64).reshape(ns, 3),
                torch.tensor(list(k), dtype=torch.int32))

    def build(self, x):
        n = x.shape[1]
        self._vec(x, n, "x")
        _check("tree_build", lib().tree_build(self._h, _ptr(x), n, self.params.precision, _stream()))
        self.n = n

    def moments(self, x, m):
        n = x.shape[1]
        self._vec(x, n, "x"); self._scal(m, n, "m")
        _check("tree_moments", lib().tree_moments(self._h, _ptr(x), _ptr(m), _stream()))

    def forces(self, a=None, phi=None, emit_lists=False, want_phi=True, lists_only=False):
        """Tree forces of the last build (a (3, n), phi (n,)); emit_lists also stores the
        interaction lists; lists_only stores them without evaluating forces (returns None, None)."""
        n = self.n
        if lists_only:
            _check("tree_forces", lib().tree_forces(self._h, None, None, FLAG_EMIT_LISTS | FLAG_LISTS_ONLY,
                                                    _stream()))
            return None, None
        if a is None:
            a = torch.empty((3, n), dtype=self.dtype, device="cuda")
        if phi is None and want_phi:
            phi = torch.empty((n,), dtype=self.dtype, device="cuda")
        self._vec(a, n, "a"); self._scal(phi, n, "phi", optional=True)
        _check("tree_forces", lib().tree_forces(self._h, _ptr(a), _ptr(phi),
                                                FLAG_EMIT_LISTS if emit_lists else 0, _stream()))
        return a, phi

    def forces_adjoint(self, a_bar, phi_bar=None, x_bar=None, m_bar=None):
        """Adds the VJP of the last tree_forces (lists stored with emit_lists=True) with cotangents
        (a_bar, phi_bar) to x_bar (3, n) and m_bar (n,); returns them (allocated as zeros if None)."""
        n = self.n
        self._vec(a_bar, n, "a_bar"); self._scal(phi_bar, n, "phi_bar", optional=True)
        if x_bar is None:
            x_bar = torch.zeros((3, n), dtype=self.dtype, device="cuda")
        if m_bar is None:
            m_bar = torch.zeros((n,), dtype=self.dtype, device="cuda")
        self._vec(x_bar, n, "x_bar"); self._scal(m_bar, n, "m_bar")
        _check("tree_forces_adjoint", lib().tree_forces_adjoint(self._h, _ptr(a_bar), _ptr(phi_bar), _ptr(x_bar),
                                                                _ptr(m_bar), _stream()))
        return x_bar, m_bar

    def energy_vjp(self, m, phi, w_bar, phi_bar=None, m_bar=None):
        """Cotangents of W = 1/2 sum m phi (tree_energy_vjp): w_bar a CUDA float64 tensor of one
        element; returns phi_bar (w_bar m / 2, allocated if None) after adding w_bar phi / 2 to m_bar."""
        n = m.shape[0]
        self._scal(m, n, "m"); self._scal(phi, n, "phi")
        if not w_bar.is_cuda or w_bar.dtype != torch.float64 or w_bar.numel() != 1:
            raise ValueError("w_bar must be a CUDA float64 tensor of one element")
        if phi_bar is None:
            phi_bar = torch.empty_like(m)
        self._scal(phi_bar, n, "phi_bar"); self._scal(m_bar, n, "m_bar", optional=True)
        _check("tree_energy_vjp", lib().tree_energy_vjp(self._h, _ptr(m), _ptr(phi), _ptr(w_bar.contiguous()), n,
                                                        _ptr(phi_bar), _ptr(m_bar), _stream()))
        return phi_bar

    def leapfrog_adjoint_step(self, x_bar, v_bar, a_bar, m_bar, tau, phi_bar=None):
        """One reverse leapfrog step through the tree stored at x_{n+1} (see treegb.h); in place."""
        n = self.n
        for t, nm in ((x_bar, "x_bar"), (v_bar, "v_bar"), (a_bar, "a_bar")):
            self._vec(t, n, nm)
        self._scal(m_bar, n, "m_bar"); self._scal(phi_bar, n, "phi_bar", optional=True)
        _check("leapfrog_adjoint_step", lib().leapfrog_adjoint_step(self._h, _ptr(x_bar), _ptr(v_bar), _ptr(a_bar),
                                                                    _ptr(m_bar), _ptr(phi_bar), float(tau),
                                                                    _stream()))

    def accel(self, x, m, a=None, phi=None, want_phi=True):
        """Accelerations and potentials of (x, m) by the tree (build + moments + forces)."""
        n = x.shape[1]
        self._vec(x, n, "x"); self._scal(m, n, "m")
        if a is None:
            a = torch.empty((3, n), dtype=self.dtype, device="cuda")
        if phi is None and want_phi:
            phi = torch.empty((n,), dtype=self.dtype, device="cuda")
        self._vec(a, n, "a"); self._scal(phi, n, "phi", optional=True)
        _check("tree_accel", lib().tree_accel(self._h, _ptr(x), _ptr(m), n, _ptr(a), _ptr(phi), _stream()))
        self.n = n
        return a, phi

    def leapfrog_step(self, x, v, m, a, tau, phi=None):
        """One KDK step in place (Eqs. 2-5); a: a^n in, a^{n+1} out."""
        n = x.shape[1]
        self._vec(x, n, "x"); self._vec(v, n, "v"); self._scal(m, n, "m"); self._vec(a, n, "a")
        self._scal(phi, n, "phi", optional=True)
        _check("leapfrog_step", lib().leapfrog_step(self._h, _ptr(x), _ptr(v), _ptr(m), _ptr(a), _ptr(phi),
                                                    float(tau), n, _stream()))
        self.n = n

    def leapfrog_step_host(self, x, v, m, a, tau, phi=None, diag=None):
        """One KDK step on a host-resident state (leapfrog_step_host): x, v, a (3, n), m, phi (n,) and
        diag (8,) float64 are pinned CPU tensors, updated when the current stream has run."""
        n = x.shape[1]
        for t, nm, shape in ((x, "x", (3, n)), (v, "v", (3, n)), (a, "a", (3, n)), (m, "m", (n,)),
                             (phi, "phi", (n,))):
            if t is None and nm == "phi":
                continue
            if t.is_cuda or t.dtype != self.dtype or tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous host {self.dtype} tensor of shape {shape}")
        if diag is not None and (diag.is_cuda or diag.dtype != torch.float64 or diag.numel() < 8):
            raise ValueError("diag must be a host float64 tensor of 8")
        _check("leapfrog_step_host", lib().leapfrog_step_host(self._h, _ptr(x), _ptr(v), _ptr(m), _ptr(a), _ptr(phi),
                                                              float(tau), n, _ptr(diag), _stream()))
        self.n = n

    def diagnostics(self, x, v, m, phi=None, out=None):
        """FP64 (E_kin, W, Px, Py, Pz, Lx, Ly, Lz) as a CUDA float64 tensor of 8."""
        n = x.shape[1]
        self._vec(x, n, "x"); self._vec(v, n, "v"); self._scal(m, n, "m")
        self._scal(phi, n, "phi", optional=True)
        if out is None:
            out = torch.empty(8, dtype=torch.float64, device="cuda")
        _check("tree_diagnostics", lib().tree_diagnostics(self._h, _ptr(x), _ptr(v), _ptr(m), _ptr(phi), n,
                                                          _ptr(out), _stream()))
        return out

    def direct(self, x, m, targets, precision=None):
        """GPU direct sum of Eq. 1 for the target indices: a (3, nt), phi (nt), float64."""
        n = x.shape[1]
        dt = self.params.precision if precision is None else {"f32": F32, "f64": F64}.get(precision, precision)
        want = torch.float64 if dt == F64 else torch.float32
        if x.dtype != want or m.dtype != want or not x.is_cuda or not m.is_cuda:
            raise ValueError("x, m must be CUDA tensors of the requested precision")
        if tuple(x.shape) != (3, n) or tuple(m.shape) != (n,):
            raise ValueError("bad shapes")
        targets = targets.to(device="cuda", dtype=torch.int64).contiguous()
        nt = targets.numel()
        a = torch.empty((3, nt), dtype=torch.float64, device="cuda")
        phi = torch.empty((nt,), dtype=torch.float64, device="cuda")
        _check("tree_direct_forces", lib().tree_direct_forces(self._h, _ptr(x.contiguous()), _ptr(m.contiguous()),
                                                              n, dt, _ptr(targets), nt, _ptr(a), _ptr(phi),
                                                              _stream()))
        return a, phi

    def set_waits(self, wait_cycles=0, withhold=None):
        """Limit of the device-side waits in clock cycles (0: keep), and the test injection
        withhold = (sort pass, tile) whose look-back words stay unpublished (None: off)."""
        wp, wt = (-1, -1) if withhold is None else (int(withhold[0]), int(withhold[1]))
        _check("tree_set_waits", lib().tree_set_waits(self._h, int(wait_cycles), wp, wt))

    # -- state, statistics, exports -----------------------------------------
    def status(self, clear=True) -> int:
        st = _i32(0)
        code = lib().tree_get_status(self._h, ctypes.byref(st), 1 if clear else 0)
        if code not in (TREE_OK, TREE_ERR_DEVICE):
            raise TreeError("tree_get_status", code)
        return int(st.value)

    def info(self) -> dict:
        i = TreeInfo()
        _check("tree_get_info", lib().tree_get_info(self._h, ctypes.byref(i)))
        return dict(n=i.n, n_nodes=i.n_nodes, depth=i.depth, box_k=i.box_k, box_lo=list(i.box_lo),
                    level_offset=list(i.level_offset), pp_pairs=i.pp_pairs, pc_pairs=i.pc_pairs,
                    max_stack=i.max_stack, n_groups=i.n_groups, list_pc=i.list_pc, list_pp=i.list_pp,
                    launches=i.launches, n_segments=i.n_segments)

    def timing(self, enable=True):
        """Start (enable=True) or stop per-phase GPU event timing."""
        _check("tree_timing_enable", lib().tree_timing_enable(self._h, 1 if enable else 0))

    def timing_read(self):
        """({phase: (total ms, calls)}, kernels launched in the timed phases)
        accumulated since timing(True); synchronises."""
        ms = (_dbl * len(PHASES))()
        calls = (_i64 * len(PHASES))()
        nl = _i64(0)
        _check("tree_timing_read", lib().tree_timing_read(self._h, ms, calls, ctypes.byref(nl)))
        return {ph: (float(ms[i]), int(calls[i])) for i, ph in enumerate(PHASES)}, int(nl.value)

    def launches(self) -> int:
        """Kernels launched by this workspace so far (host counter, no sync)."""
        return self.info()["launches"]

    def export_tree(self):
        inf = self.info()
        n, nn = inf["n"], inf["n_nodes"]
        dev = "cuda"
        keys = torch.empty(n, dtype=torch.int64, device=dev)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        level = torch.empty(nn, dtype=torch.int32, device=dev)
        corner = torch.empty((3, nn), dtype=torch.int32, device=dev)
        first = torch.empty(nn, dtype=torch.int32, device=dev)
        count = torch.empty(nn, dtype=torch.int32, device=dev)
        child = torch.empty(nn, dtype=torch.int32, device=dev)
        nchild = torch.empty(nn, dtype=torch.int32, device=dev)
        _check("tree_export_tree", lib().tree_export_tree(self._h, _ptr(keys), _ptr(perm), _ptr(level), _ptr(corner),
                                                          _ptr(first), _ptr(count), _ptr(child), _ptr(nchild),
                                                          _stream()))
        return dict(keys=keys, perm=perm, level=level, corner=corner, first=first, count=count, child=child,
                    nchild=nchild, info=inf)

    def export_moments(self):
        nn = self.info()["n_nodes"]
        M = torch.empty(nn, dtype=torch.float64, device="cuda")
        R = torch.empty((3, nn), dtype=torch.float64, device="cuda")
        Q = torch.empty((6, nn), dtype=torch.float64, device="cuda")
        _check("tree_export_moments", lib().tree_export_moments(self._h, _ptr(M), _ptr(R), _ptr(Q), _stream()))
        return M, R, Q

    def export_group_stats(self):
        """Per-group records of the last walk: int64 CUDA tensor (4, n_groups) =
        (far cells, near particles, deepest stack, near leaves)."""
        ng = self.info()["n_groups"]
        out = torch.empty((4, max(ng, 1)), dtype=torch.int32, device="cuda")
        _check("tree_export_group_stats", lib().tree_export_group_stats(self._h, _ptr(out), _stream()))
        return out[:, :ng].long()

    def export_groups(self):
        """Walk groups of the last build: int64 CUDA tensor of n_groups + 1 first indices."""
        ng = self.info()["n_groups"]
        out = torch.empty(ng + 1, dtype=torch.int32, device="cuda")
        _check("tree_export_groups", lib().tree_export_groups(self._h, _ptr(out), _stream()))
        return out.long()

    def export_lists(self):
        inf = self.info()
        ng = inf["n_groups"]
        pc_off = torch.empty(ng + 1, dtype=torch.int64, device="cuda")
        pp_off = torch.empty(ng + 1, dtype=torch.int64, device="cuda")
        pc = torch.empty(max(1, inf["list_pc"]), dtype=torch.int32, device="cuda")
        pp = torch.empty(max(1, inf["list_pp"]), dtype=torch.int32, device="cuda")
        _check("tree_export_lists", lib().tree_export_lists(self._h, _ptr(pc_off), _ptr(pc), _ptr(pp_off),
                                                            _ptr(pp), _stream()))
        return pc_off, pc[: inf["list_pc"]], pp_off, pp[: inf["list_pp"]]

    def export_lists_groups(self, gsel):
        """Lists of the selected groups (tree_export_lists_groups): (pc_off, pc, pp_off, pp) with the
        offsets as host int64 lists of len(gsel) + 1 and the entries as int32 CUDA tensors."""
        gs = [int(g) for g in gsel]
        k = len(gs)
        sel = (_i64 * max(k, 1))(*gs)
        pco = (_i64 * (k + 1))()
        ppo = (_i64 * (k + 1))()
        _check("tree_export_lists_groups", lib().tree_export_lists_groups(self._h, k, sel, pco, None, ppo, None,
                                                                          _stream()))
        pc = torch.empty(max(1, pco[k]), dtype=torch.int32, device="cuda")
        pp = torch.empty(max(1, ppo[k]), dtype=torch.int32, device="cuda")
        _check("tree_export_lists_groups", lib().tree_export_lists_groups(self._h, k, sel, pco, _ptr(pc), ppo,
                                                                          _ptr(pp), _stream()))
        return list(pco), pc[: pco[k]], list(ppo), pp[: ppo[k]]
