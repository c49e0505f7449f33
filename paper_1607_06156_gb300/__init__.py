"""GB300 connected-components engine: thin ctypes binding over libcc_gb300.so.

Every step of the hybrid route (Algorithm 2 of Jain et al., "An Adaptive
Parallel Algorithm for Computing Connected Components": degree
distribution, power-law/K-S route prediction, direction-optimizing BFS,
Shiloach-Vishkin iterations) runs in the library's CUDA kernels; this module
only marshals arguments. PyTorch supplies device memory and streams.

There is no CPU fallback: if the shared library has not been built the
import succeeds but every call raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcc_gb300.so")

CC_OK = 0
STATUS = {
    0: "CC_OK", 1: "CC_ERR_INVALID_ARG", 2: "CC_ERR_INVALID_EDGE", 3: "CC_ERR_OOM",
    4: "CC_ERR_NO_CONVERGENCE", 5: "CC_ERR_TIMEOUT", 6: "CC_ERR_CUDA", 7: "CC_ERR_UNSUPPORTED",
}
ROUTES = {"auto": 0, "learned": 1, "bfs": 2, "sv": 3}
FAULT_ALLOC, FAULT_ITER_CAP = 1, 2
MAX_SV_ITERS_RECORDED = 64
K_COUNT = 16
# kernel classes of cc_stats.kernel_ms (CC_K_* in the header)
KERNELS = ["degree", "hist", "ks", "scan", "csr", "bfs_topdown", "bfs_bottomup", "bfs_aux", "parent_init",
           "sv_first", "sv_gather_input", "sv_gather_list", "sv_shortcut", "finalize", "predict", "tuple_sort"]
MLP_IN, MLP_HIDDEN, MLP_OUT = 69, 128, 3
MLP_PARAMS = 128 * 69 + 128 + 128 * 128 + 128 + 3 * 128 + 3


class CCError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class Options(ctypes.Structure):
    _fields_ = [
        ("id_bytes", ctypes.c_int), ("route_policy", ctypes.c_int), ("ks_tau", ctypes.c_double),
        ("ks_min_tail", ctypes.c_int), ("ks_min_distinct", ctypes.c_int), ("max_iters", ctypes.c_int),
        ("bfs_cutoff_levels", ctypes.c_int), ("debug_checks", ctypes.c_int), ("fault_inject", ctypes.c_int),
        ("ks_min_span", ctypes.c_double), ("profile", ctypes.c_int), ("bfs_mode", ctypes.c_int),
        ("sv_sample_stride", ctypes.c_int), ("bfs_starts", ctypes.c_int),
        ("batch_hook_regions", ctypes.c_int), ("reserved", ctypes.c_int),
    ]


_OPTION_FIELDS = frozenset(f for f, _ in Options._fields_ if f != "reserved")


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("route", ctypes.c_int), ("route_source", ctypes.c_int),
        ("bfs_levels", ctypes.c_int), ("sv_iters", ctypes.c_int), ("degree_form", ctypes.c_int),
        ("ks_d", ctypes.c_double), ("ks_alpha", ctypes.c_double), ("ks_xmin", ctypes.c_int64),
        ("ks_ntail", ctypes.c_int64), ("ks_ncand", ctypes.c_int64), ("n", ctypes.c_int64), ("m", ctypes.c_int64),
        ("max_degree", ctypes.c_int64), ("seed_vertex", ctypes.c_int64), ("bfs_visited", ctypes.c_int64),
        ("comp_min", ctypes.c_int64), ("bfs_edges_inspected", ctypes.c_int64),
        ("m_active", ctypes.c_int64 * MAX_SV_ITERS_RECORDED),
        ("ms_degree", ctypes.c_float), ("ms_predict", ctypes.c_float), ("ms_csr", ctypes.c_float),
        ("ms_bfs", ctypes.c_float), ("ms_sv", ctypes.c_float), ("ms_finalize", ctypes.c_float),
        ("ms_total", ctypes.c_float), ("pad1", ctypes.c_float), ("launches", ctypes.c_int64),
        ("kernel_ms", ctypes.c_float * K_COUNT), ("kernel_launches", ctypes.c_int32 * K_COUNT),
        ("sv_hooks", ctypes.c_int64 * MAX_SV_ITERS_RECORDED),
        ("pred_confidence", ctypes.c_float), ("pred_route", ctypes.c_int), ("pred_cutoff", ctypes.c_int),
        ("ms_features", ctypes.c_float),
        ("batch_unroll", ctypes.c_int32),
        ("batch_grid_mult", ctypes.c_int32),
        ("sv_sample_stride", ctypes.c_int32), ("batch_deg_regions", ctypes.c_int32),
        ("bfs_starts", ctypes.c_int32), ("batch_sv_regions", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}
        it = max(0, min(self.sv_iters, MAX_SV_ITERS_RECORDED))
        d["m_active"] = [int(x) for x in self.m_active[:it]]
        d["sv_hooks"] = [int(x) for x in self.sv_hooks[:it]]
        d["kernel_ms"] = {KERNELS[i]: float(self.kernel_ms[i]) for i in range(len(KERNELS))}
        d["kernel_launches"] = {KERNELS[i]: int(self.kernel_launches[i]) for i in range(len(KERNELS))}
        return d


_lib = None
_vp, _i64, _int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int


class L2Rates(ctypes.Structure):
    """cc_l2_rates: measured L2 random-access rates (operations per second)."""
    _fields_ = [("gather", ctypes.c_double), ("red_add", ctypes.c_double), ("red_min", ctypes.c_double),
                ("atom_min", ctypes.c_double), ("table_words", ctypes.c_int64), ("ops", ctypes.c_int64),
                ("reps", ctypes.c_int32), ("grid", ctypes.c_int32)]


def lib() -> ctypes.CDLL:
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the engine has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        L.cc_default_options.argtypes = [ctypes.POINTER(Options)]
        L.cc_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(Options), _int]
        L.cc_set_options.argtypes = [_vp, ctypes.POINTER(Options)]
        L.cc_destroy.argtypes = [_vp]
        L.cc_labels.argtypes = [_vp, _vp, _i64, _i64, _vp, _vp]
        L.cc_labels_host.argtypes = [_vp, _vp, _i64, _i64, _vp, _vp]
        L.cc_labels_tuple_sv.argtypes = [_vp, _vp, _i64, _i64, _vp, _vp]
        L.cc_ks_statistic_batched.argtypes = [_vp, _vp, _vp, _vp, _int, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.cc_labels_batched.argtypes = [_vp, _vp, _vp, _vp, _int, _i64, _i64, _vp, _vp]
        L.cc_degree_distribution.argtypes = [_vp, _vp, _i64, _i64, _vp, _vp, _i64, _vp]
        L.cc_ks_statistic.argtypes = [_vp, _vp, _i64, _vp, _vp]
        L.cc_get_stats.argtypes = [_vp, ctypes.POINTER(Stats)]
        L.cc_labels_static.argtypes = [_vp, _int, _i64, _i64, _vp, _vp]
        L.cc_route_features.argtypes = [_vp, _vp, _i64, _i64, _vp, _vp]
        L.cc_set_predictor.argtypes = [_vp, _vp, ctypes.c_double]
        L.cc_mlp_forward.argtypes = [_vp, _vp, _int, _vp, _vp]
        L.cc_mlp_backward.argtypes = [_vp, _vp, _vp, _vp, _vp, _int, ctypes.c_float, _vp, _vp, _vp, _vp, _vp]
        L.cc_mlp_adam.argtypes = [_vp, _vp, _vp, _vp, _int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, _int, _vp]
        L.cc_measure_l2_rates.argtypes = [_vp, ctypes.POINTER(L2Rates), _vp]
        L.cc_strerror.argtypes = [_int]
        L.cc_strerror.restype = ctypes.c_char_p
        for f in ("cc_default_options", "cc_create", "cc_set_options", "cc_destroy", "cc_labels",
                  "cc_labels_batched", "cc_degree_distribution", "cc_ks_statistic", "cc_get_stats",
                  "cc_labels_static", "cc_route_features", "cc_set_predictor", "cc_mlp_forward",
                  "cc_mlp_backward", "cc_mlp_adam", "cc_measure_l2_rates", "cc_labels_host",
                  "cc_ks_statistic_batched", "cc_labels_tuple_sv"):
            getattr(L, f).restype = _int
        _lib = L
    return _lib


def default_options() -> Options:
    o = Options()
    lib().cc_default_options(ctypes.byref(o))
    return o


def _check(rc: int, where: str):
    if rc != CC_OK:
        raise CCError(rc, where)


def _stream_handle(stream, device) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream(device)
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _device_tensor(t, name: str, itemsize: int, floating: bool = False, numel: int = 0, device=None) -> None:
    """What the library cannot see behind a pointer: a contiguous CUDA tensor
    of the right element width and kind, holding at least `numel` elements,
    on the engine's device. A mismatch raises ValueError before the call
    instead of letting a kernel read or write past the tensor."""
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (it is on {t.device})")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on {t.device}, the engine on cuda:{device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.element_size() != itemsize or t.dtype.is_floating_point != floating or t.dtype.is_complex:
        kind = "floating-point" if floating else "integer"
        raise ValueError(f"{name} must hold {itemsize}-byte {kind} elements (it holds {t.dtype})")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, {numel} are needed")


def _pairs(edges, itemsize: int, device=None) -> int:
    """m of a device [m, 2] pair tensor, checked as above."""
    _device_tensor(edges, "edges", itemsize, device=device)
    if edges.numel() == 0:
        return 0
    if edges.dim() != 2 or edges.shape[1] != 2:
        raise ValueError(f"edges must have shape [m, 2] (it has {tuple(edges.shape)})")
    return edges.shape[0]


def _offsets(edge_offsets, vertex_offsets, m: int):
    """Host int64 copies of a batch's offsets ([G + 1] each); the last edge
    offset may not pass the pairs the edge tensor holds."""
    import torch

    eo = torch.as_tensor(edge_offsets).cpu().to(torch.int64).contiguous()
    vo = torch.as_tensor(vertex_offsets).cpu().to(torch.int64).contiguous()
    if eo.dim() != 1 or vo.dim() != 1 or eo.numel() < 1 or eo.numel() != vo.numel():
        raise ValueError("edge_offsets and vertex_offsets must be 1-D with G + 1 entries each")
    if int(eo[-1]) > m:
        raise ValueError(f"edge_offsets end at pair {int(eo[-1])}, the edges hold {m} pairs")
    return eo, vo


def _set_options(o: Options, opts: dict) -> None:
    """Copy keyword options into a cc_options; a name that is not a field
    raises instead of landing on a Python attribute the library never sees."""
    for k, v in opts.items():
        if k not in _OPTION_FIELDS:
            raise TypeError(f"unknown option {k!r} (cc_options fields: {', '.join(sorted(_OPTION_FIELDS))})")
        setattr(o, k, v)


class Engine:
    """One cc_ctx: a device workspace plus options (Algorithm 2 route policy)."""

    def __init__(self, id_bytes: int = 4, route: str = "auto", device: int = 0, **opts):
        o = default_options()
        o.id_bytes = id_bytes
        o.route_policy = ROUTES[route]
        _set_options(o, opts)
        self.device = device
        self._opt = o
        h = _vp()
        _check(lib().cc_create(ctypes.byref(h), ctypes.byref(o), device), "cc_create")
        self._h = h

    def set_options(self, route: str | None = None, **opts):
        o = self._opt
        if route is not None:
            o.route_policy = ROUTES[route]
        _set_options(o, opts)
        _check(lib().cc_set_options(self._h, ctypes.byref(o)), "cc_set_options")

    @property
    def options(self) -> Options:
        return self._opt

    def close(self):
        if getattr(self, "_h", None):
            lib().cc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----- raw-pointer calls (the C ABI as is) -----
    def labels_ptr(self, edges_ptr: int, n: int, m: int, labels_ptr: int, stream: int = 0) -> int:
        return lib().cc_labels(self._h, edges_ptr, n, m, labels_ptr, stream)

    # ----- torch conveniences -----
    def labels(self, edges, n: int, out=None, stream=None):
        """Component labels (min vertex id per component) of a device edge tensor [m, 2].

        Stream-ordered: returns once the work is enqueued on `stream` (the
        current stream by default). Errors found on the device are reported
        by check() / stats(), or by this call with debug_checks=1."""
        import torch

        m = _pairs(edges, self._opt.id_bytes, self.device)
        if out is None:
            out = torch.empty(n, dtype=edges.dtype, device=edges.device)
        _device_tensor(out, "out", self._opt.id_bytes, numel=n, device=self.device)
        rc = lib().cc_labels(self._h, edges.data_ptr() if m else None, n, m, out.data_ptr() if n else None,
                             _stream_handle(stream, edges.device))
        _check(rc, "cc_labels")
        return out

    def labels_tuple_sv(self, edges, n: int, out=None, stream=None):
        """Labels by the paper's sort-based SV (Algorithm 1) on the device
        (cc_labels_tuple_sv): the same labels as `labels`, for comparison."""
        import torch

        m = _pairs(edges, self._opt.id_bytes, self.device)
        if out is None:
            out = torch.empty(n, dtype=edges.dtype, device=edges.device)
        _device_tensor(out, "out", self._opt.id_bytes, numel=n, device=self.device)
        rc = lib().cc_labels_tuple_sv(self._h, edges.data_ptr() if m else None, n, m,
                                      out.data_ptr() if n else None, _stream_handle(stream, edges.device))
        _check(rc, "cc_labels_tuple_sv")
        return out

    def labels_host(self, edges, n: int, out=None, stream=None):
        """Labels of a host (CPU) [m, 2] edge tensor into a host tensor (cc_labels_host).
        Pin both tensors (`.pin_memory()`) for the copies to overlap the passes."""
        import torch

        if edges.device.type != "cpu" or not edges.is_contiguous():
            raise ValueError("edges must be a contiguous CPU tensor")
        if edges.element_size() != self._opt.id_bytes or edges.dtype.is_floating_point or edges.dtype.is_complex:
            raise ValueError(f"edges must hold {self._opt.id_bytes}-byte integer ids (it holds {edges.dtype})")
        if edges.numel() and (edges.dim() != 2 or edges.shape[1] != 2):
            raise ValueError(f"edges must have shape [m, 2] (it has {tuple(edges.shape)})")
        m = edges.shape[0] if edges.numel() else 0
        dt = torch.int32 if self._opt.id_bytes == 4 else torch.int64
        if out is None:
            out = torch.empty(n, dtype=dt)
        if out.device.type != "cpu" or out.dtype != dt or out.numel() != n or not out.is_contiguous():
            raise ValueError("out must be a contiguous CPU tensor of n ids")
        rc = lib().cc_labels_host(self._h, edges.data_ptr() if m else None, n, m, out.data_ptr(),
                                  _stream_handle(stream, self.device))
        _check(rc, "cc_labels_host")
        return out

    def labels_batched(self, edges, edge_offsets, vertex_offsets, out=None, stream=None):
        """Local labels of G independent graphs (int32 ids local to each graph); the
        offsets are given on the host and copied to the device."""
        import torch

        eo_h, vo_h = _offsets(edge_offsets, vertex_offsets, _pairs(edges, 4, self.device))
        if out is None:
            out = torch.empty(int(vo_h[-1]), dtype=torch.int32, device=edges.device)
        _device_tensor(out, "out", 4, numel=int(vo_h[-1]), device=self.device)
        return self.labels_batched_dev(edges, eo_h.to(edges.device), vo_h.to(edges.device), int(eo_h[-1]),
                                       int(vo_h[-1]), out, stream)

    def ks_statistic_batched(self, edges, edge_offsets, vertex_offsets, stream=None) -> dict:
        """Per-graph route prediction of a batch (cc_ks_statistic_batched): numpy arrays
        D, alpha, xmin, ncand, route, seed of G entries each."""
        import numpy as np

        m = _pairs(edges, 4, self.device)
        eo, vo = _offsets(np.ascontiguousarray(edge_offsets, dtype=np.int64),
                          np.ascontiguousarray(vertex_offsets, dtype=np.int64), m)
        G = eo.numel() - 1
        eo_d, vo_d = eo.to(edges.device), vo.to(edges.device)
        out = {k: np.zeros(G, dtype=dt) for k, dt in (("D", np.float64), ("alpha", np.float64), ("xmin", np.int64),
                                                     ("ncand", np.int64), ("route", np.int32), ("seed", np.int64))}
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        rc = lib().cc_ks_statistic_batched(self._h, edges.data_ptr() if m else None, eo_d.data_ptr(), vo_d.data_ptr(),
                                           G, int(eo[-1]), int(vo[-1]), ptr(out["D"]), ptr(out["alpha"]),
                                           ptr(out["xmin"]), ptr(out["ncand"]), ptr(out["route"]), ptr(out["seed"]),
                                           _stream_handle(stream, edges.device))
        _check(rc, "cc_ks_statistic_batched")
        return out

    def labels_batched_dev(self, edges, eo_dev, vo_dev, m_total: int, n_total: int, out, stream=None):
        """cc_labels_batched with the offsets on the device ([G + 1] int64 each) and their
        last entries given as m_total and n_total; stream-ordered like labels()."""
        m = _pairs(edges, 4, self.device)
        G = eo_dev.numel() - 1
        if G < 0 or vo_dev.numel() != G + 1:
            raise ValueError("eo_dev and vo_dev must hold G + 1 offsets each")
        if not 0 <= m_total <= m or n_total < 0:
            raise ValueError(f"m_total must be within the {m} pairs of edges and n_total >= 0")
        _device_tensor(eo_dev, "eo_dev", 8, numel=G + 1, device=self.device)
        _device_tensor(vo_dev, "vo_dev", 8, numel=G + 1, device=self.device)
        _device_tensor(out, "out", 4, numel=n_total, device=self.device)
        rc = lib().cc_labels_batched(self._h, edges.data_ptr() if edges.numel() else None, eo_dev.data_ptr(),
                                     vo_dev.data_ptr(), G, m_total, n_total, out.data_ptr() if out.numel() else None,
                                     _stream_handle(stream, edges.device))
        _check(rc, "cc_labels_batched")
        return out

    def degree_distribution(self, edges, n: int, hist_len: int = 0, stream=None):
        """(deg[n] uint32 as int32 tensor, hist[hist_len] uint64 as int64 tensor or None)."""
        import torch

        m = _pairs(edges, self._opt.id_bytes, self.device)
        deg = torch.empty(n, dtype=torch.int32, device=edges.device)
        hist = torch.empty(hist_len, dtype=torch.int64, device=edges.device) if hist_len > 0 else None
        rc = lib().cc_degree_distribution(self._h, edges.data_ptr() if m else None, n, m,
                                          deg.data_ptr() if n else None, hist.data_ptr() if hist is not None else None,
                                          hist_len, _stream_handle(stream, edges.device))
        _check(rc, "cc_degree_distribution")
        return deg, hist

    def ks_statistic(self, hist, stream=None) -> dict:
        """Power-law fit + K-S statistic of a device uint64 (int64 tensor) degree histogram."""
        _device_tensor(hist, "hist", 8, numel=1, device=self.device)
        out = (ctypes.c_double * 5)()
        rc = lib().cc_ks_statistic(self._h, hist.data_ptr(), hist.numel(), out, _stream_handle(stream, hist.device))
        _check(rc, "cc_ks_statistic")
        return {"D": out[0], "alpha": out[1], "xmin": int(out[2]), "ntail": int(out[3]), "ncand": int(out[4])}

    def route_features(self, edges, n: int, stream=None):
        """The predictor's CC_MLP_IN features of a device edge tensor (float32 tensor on its device)."""
        import torch

        m = _pairs(edges, self._opt.id_bytes, self.device)
        x = torch.empty(MLP_IN, dtype=torch.float32, device=edges.device)
        rc = lib().cc_route_features(self._h, edges.data_ptr() if m else None, n, m, x.data_ptr(),
                                     _stream_handle(stream, edges.device))
        _check(rc, "cc_route_features")
        return x

    def set_predictor(self, params, min_confidence: float = 0.75):
        """Installs fp32 predictor parameters (MLP_PARAMS floats) for route='learned'; None removes it."""
        import numpy as np

        if params is None:
            _check(lib().cc_set_predictor(self._h, None, min_confidence), "cc_set_predictor")
            return
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_PARAMS:
            raise ValueError(f"expected {MLP_PARAMS} parameters, got {p.size}")
        _check(lib().cc_set_predictor(self._h, p.ctypes.data_as(ctypes.c_void_p), min_confidence),
               "cc_set_predictor")

    def l2_rates(self, stream=None) -> dict:
        """Measured L2 random-access rates of this engine's device (cc_measure_l2_rates), in operations/s."""
        r = L2Rates()
        _check(lib().cc_measure_l2_rates(self._h, ctypes.byref(r), _stream_handle(stream, self.device)),
               "cc_measure_l2_rates")
        return {f: getattr(r, f) for f, _ in L2Rates._fields_}

    def stats(self) -> dict:
        """Statistics of the last call (waits for its stream)."""
        s = Stats()
        lib().cc_get_stats(self._h, ctypes.byref(s))
        return s.as_dict()

    def check(self) -> None:
        """Waits for the last call and raises its device-detected error, if any
        (cc_labels is stream-ordered: an id outside [0, n) or a run past the
        iteration cap is reported here, by the next call, or by the call
        itself with the debug_checks option)."""
        s = Stats()
        _check(lib().cc_get_stats(self._h, ctypes.byref(s)), "cc_labels (device status)")


def _mlp_batch(params, X) -> int:
    """B of a [B, MLP_IN] float32 feature tensor, with the flat parameters checked."""
    _device_tensor(params, "params", 4, floating=True, numel=MLP_PARAMS)
    _device_tensor(X, "X", 4, floating=True, device=params.device.index)
    if X.dim() != 2 or X.shape[1] != MLP_IN:
        raise ValueError(f"X must have shape [B, {MLP_IN}] (it has {tuple(X.shape)})")
    return X.shape[0]


def mlp_forward(params, X, act, stream=None):
    """cc_mlp_forward on device float32 tensors; act holds B * (2*128 + 3) floats."""
    B = _mlp_batch(params, X)
    _device_tensor(act, "act", 4, floating=True, numel=B * (2 * MLP_HIDDEN + MLP_OUT), device=X.device.index)
    _check(lib().cc_mlp_forward(params.data_ptr(), X.data_ptr(), X.shape[0], act.data_ptr(),
                                _stream_handle(stream, X.device)), "cc_mlp_forward")


def mlp_backward(params, X, y, t, w, lam, act, grad, scratch, loss, stream=None):
    """cc_mlp_backward on device tensors (y int32, others float32); adds the batch loss into loss[0]."""
    B = _mlp_batch(params, X)
    d = X.device.index
    _device_tensor(y, "y", 4, numel=B, device=d)
    for name, t_, k in (("t", t, B), ("w", w, B), ("act", act, B * (2 * MLP_HIDDEN + MLP_OUT)),
                        ("grad", grad, MLP_PARAMS), ("scratch", scratch, B * (3 + 2 * MLP_HIDDEN)), ("loss", loss, 1)):
        _device_tensor(t_, name, 4, floating=True, numel=k, device=d)
    _check(lib().cc_mlp_backward(params.data_ptr(), X.data_ptr(), y.data_ptr(), t.data_ptr(), w.data_ptr(),
                                 X.shape[0], lam, act.data_ptr(), grad.data_ptr(), scratch.data_ptr(),
                                 loss.data_ptr(), _stream_handle(stream, X.device)), "cc_mlp_backward")


def mlp_adam(params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """cc_mlp_adam on device float32 tensors (step >= 1)."""
    d = params.device.index
    for name, t_ in (("params", params), ("grad", grad), ("m", m), ("v", v)):
        _device_tensor(t_, name, 4, floating=True, numel=params.numel(), device=d)
    _check(lib().cc_mlp_adam(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), params.numel(), lr,
                             beta1, beta2, eps, step, _stream_handle(stream, params.device)), "cc_mlp_adam")


STATIC_MAX_VERTICES = 1 << 20
STATIC_MAX_PAIRS = 1 << 21


def labels_static(edges, n: int, out=None, stream=None):
    """cc_labels_static: labels with the library's built-in scratch (no device allocation by the library)."""
    import torch

    m = _pairs(edges, edges.element_size())
    if out is None:
        out = torch.empty(n, dtype=edges.dtype, device=edges.device)
    _device_tensor(out, "out", edges.element_size(), numel=n, device=edges.device.index)
    rc = lib().cc_labels_static(edges.data_ptr() if m else None, edges.element_size(), n, m,
                                out.data_ptr() if n else None, _stream_handle(stream, edges.device))
    _check(rc, "cc_labels_static")
    return out


def strerror(status: int) -> str:
    return lib().cc_strerror(status).decode()
