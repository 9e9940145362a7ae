"""ctypes binding of libbsp (include/bsp.h): argument marshalling only.

Every step of the estimator runs in the library's CUDA kernels; this module
converts torch tensors to pointers and status codes to exceptions.  If the
library is missing the import fails loudly -- there is no CPU fallback.

The functions keep the C names (``bsp_plan_create`` ...).  ``Bispectrum`` is
a convenience owner of a plan and its workspace.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbsp.so")

BSP_OK, BSP_EINVAL, BSP_ENOMEM, BSP_ECUDA, BSP_EUNSUPPORTED, BSP_ETIMEOUT, BSP_ESTATE = 0, -1, -2, -3, -4, -5, -6
BSP_FP32, BSP_SPLIT_BF16, BSP_BF16, BSP_SPLIT_F16 = 0, 1, 2, 3
BSP_SHOT_NOISE = 1
BSP_FULL_TENSOR = 2
PRECISIONS = {"fp32": BSP_FP32, "split_bf16": BSP_SPLIT_BF16, "bf16": BSP_BF16, "split_f16": BSP_SPLIT_F16}

# (name, restype, argtypes) of every exported entry point declared in include/bsp.h
_P = ctypes.c_void_p
_SIGS = [
    ("bsp_plan_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_uint]),
    ("bsp_plan_destroy", None, [_P]),
    ("bsp_plan_create_modal", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_double, ctypes.c_int, _P,
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                             ctypes.c_uint]),
    ("bsp_modal_size", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("bsp_modal_compute", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("bsp_modal_radial_powerlaw", ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                 _P]),
    ("bsp_modal_modes", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P]),
    ("bsp_modal_gamma", ctypes.c_int, [ctypes.c_int, _P, ctypes.c_double, ctypes.c_double, ctypes.c_int, _P]),
    ("bsp_modal_project", ctypes.c_int, [ctypes.c_int, _P, ctypes.c_int, _P, _P]),
    ("bsp_workspace_size", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    ("bsp_host_staging_size", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    ("bsp_counts", ctypes.c_int, [_P, _P, _P]),
    ("bsp_plan_bins", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), _P, _P]),
    ("bsp_set_wait_limit", ctypes.c_int, [_P, ctypes.c_longlong]),
    ("bsp_plan_tune_tc", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    ("bsp_batch_tuning", ctypes.c_int, [_P, _P, _P]),
    ("bsp_fp32_fma_peak", ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P]),
    ("bsp_bins_aliased", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P]),
    ("bsp_plan_share_counts", ctypes.c_int, [_P, _P]),
    ("bsp_compute", ctypes.c_int, [_P, _P, ctypes.c_double, _P, _P, _P]),
    ("bsp_compute_host", ctypes.c_int, [_P, _P, ctypes.c_double, _P, _P, _P]),
    ("bsp_last_raw", ctypes.c_int, [_P, _P, _P, _P]),
    ("bsp_power_compute", ctypes.c_int, [_P, _P, ctypes.c_double, _P, _P, _P, _P]),
    ("bsp_density_workspace_size", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    ("bsp_skew_workspace_size", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    ("bsp_skew_compute", ctypes.c_int, [_P, _P, _P, ctypes.c_size_t, _P, _P, _P]),
    ("bsp_ib_workspace_size", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    ("bsp_ib_compute", ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_size_t, _P, _P, _P]),
    ("bsp_density_cic", ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_longlong, _P, _P, ctypes.c_size_t, _P,
                                       _P, ctypes.POINTER(ctypes.c_double)]),
    ("bsp_device_status", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    ("bsp_set_accumulation_chunk", ctypes.c_int, [_P, ctypes.c_int]),
    ("bsp_plan_tune", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    ("bsp_batch_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.c_double, ctypes.c_int, _P,
                                        ctypes.c_int, _P, ctypes.c_int, ctypes.c_uint]),
    ("bsp_batch_destroy", None, [_P]),
    ("bsp_batch_workspace_size", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    ("bsp_batch_prepare", ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    ("bsp_batch_info", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), _P, _P, _P]),
    ("bsp_batch_bins", ctypes.c_int, [_P, _P, _P]),
    ("bsp_batch_run", ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P]),
    ("bsp_covariance", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    ("bsp_plan_stats", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    ("bsp_set_profiling", ctypes.c_int, [_P, ctypes.c_int]),
    ("bsp_phase_times", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]),
    ("bsp_triple_sums_static", ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_int, _P, ctypes.c_int, _P, _P]),
    ("bsp_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("bsp_last_error", ctypes.c_char_p, []),
    ("bsp_version", ctypes.c_int, []),
]
EXPORTS = [s[0] for s in _SIGS]

_lib = None


class BspError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.bsp_status_string(status).decode()
        detail = lib.bsp_last_error().decode()
        super().__init__("%s: %s (%d)%s" % (where, msg, status, (" -- " + detail) if detail else ""))
        self.status = status


def load(path: str | None = None):
    """Load libbsp.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise OSError("libbsp.so not built at %s (run paper_1708_05303_gb300.build.build())" % p)
        lib = ctypes.CDLL(p)
        for name, res, args in _SIGS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != BSP_OK:
        raise BspError(status, where)


def _dptr(t) -> int:
    """Device pointer of a CUDA torch tensor (or an int)."""
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return t.data_ptr()


def _stream_handle(stream) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def bsp_plan_create(n: int, box: float, edges, ells=(0, 2, 4), prec: int = BSP_FP32, flags: int = 0) -> int:
    lib = load()
    e = np.ascontiguousarray(edges, dtype=np.float64)
    l_ = np.ascontiguousarray(ells, dtype=np.int32)
    h = _P()
    st = lib.bsp_plan_create(ctypes.byref(h), int(n), float(box), int(e.size - 1),
                             e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(l_.size),
                             l_.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(prec), int(flags))
    _check(st, "bsp_plan_create")
    return h.value


def bsp_plan_create_modal(n: int, box: float, radial: np.ndarray, ells=(0, 2, 4), prec: int = BSP_FP32,
                          flags: int = 0) -> int:
    lib = load()
    tab = np.ascontiguousarray(radial, dtype=np.float64)
    l_ = np.ascontiguousarray(ells, dtype=np.int32)
    h = _P()
    st = lib.bsp_plan_create_modal(ctypes.byref(h), int(n), float(box), int(tab.shape[0]), tab.ctypes.data,
                                   int(l_.size), l_.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(prec),
                                   int(flags))
    _check(st, "bsp_plan_create_modal")
    return h.value


def bsp_modal_size(plan: int):
    nf, nt = ctypes.c_int(), ctypes.c_int()
    _check(load().bsp_modal_size(plan, ctypes.byref(nf), ctypes.byref(nt)), "bsp_modal_size")
    return nf.value, nt.value


def bsp_modal_compute(plan: int, delta_k, ws, S, stream=None):
    _check(load().bsp_modal_compute(plan, _dptr(delta_k), _dptr(ws), _stream_handle(stream), _dptr(S)),
           "bsp_modal_compute")


def bsp_modal_radial_powerlaw(n: int, box: float, n_modes: int, kmin: float, kmax: float, amp: float, n_s: float,
                              sqrt_k: bool = True) -> np.ndarray:
    tab = np.zeros((n_modes, 3 * (n // 2) ** 2 + 1))
    _check(load().bsp_modal_radial_powerlaw(int(n), float(box), int(n_modes), float(kmin), float(kmax), float(amp),
                                            float(n_s), int(bool(sqrt_k)), tab.ctypes.data),
           "bsp_modal_radial_powerlaw")
    return tab


def bsp_modal_modes(n_modes_1d: int, n_keep: int) -> np.ndarray:
    m = np.zeros((n_keep, 3), dtype=np.int32)
    _check(load().bsp_modal_modes(int(n_modes_1d), int(n_keep), m.ctypes.data), "bsp_modal_modes")
    return m


def bsp_modal_gamma(modes: np.ndarray, kmin: float, kmax: float, npts: int = 24) -> np.ndarray:
    m = np.ascontiguousarray(modes, dtype=np.int32).reshape(-1, 3)
    g = np.zeros((m.shape[0], m.shape[0]))
    _check(load().bsp_modal_gamma(int(m.shape[0]), m.ctypes.data, float(kmin), float(kmax), int(npts),
                                  g.ctypes.data), "bsp_modal_gamma")
    return g


def bsp_modal_project(gamma: np.ndarray, S: np.ndarray) -> np.ndarray:
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    s = np.ascontiguousarray(np.atleast_2d(S), dtype=np.float64)
    beta = np.zeros_like(s)
    _check(load().bsp_modal_project(int(g.shape[0]), g.ctypes.data, int(s.shape[0]), s.ctypes.data,
                                    beta.ctypes.data), "bsp_modal_project")
    return beta


def bsp_plan_destroy(plan: int):
    load().bsp_plan_destroy(plan)


def bsp_workspace_size(plan: int) -> int:
    v = ctypes.c_size_t()
    _check(load().bsp_workspace_size(plan, ctypes.byref(v)), "bsp_workspace_size")
    return v.value


def bsp_host_staging_size(plan: int) -> int:
    v = ctypes.c_size_t()
    _check(load().bsp_host_staging_size(plan, ctypes.byref(v)), "bsp_host_staging_size")
    return v.value


def bsp_counts(plan: int, ws, stream=None):
    _check(load().bsp_counts(plan, _dptr(ws), _stream_handle(stream)), "bsp_counts")


def bsp_plan_share_counts(dst: int, src: int):
    _check(load().bsp_plan_share_counts(dst, src), "bsp_plan_share_counts")


def bsp_plan_bins(plan: int):
    lib = load()
    nb = ctypes.c_int()
    _check(lib.bsp_plan_bins(plan, ctypes.byref(nb), None, None), "bsp_plan_bins")
    abc = np.zeros((nb.value, 3), dtype=np.int32)
    cnt = np.zeros(nb.value, dtype=np.float64)
    _check(lib.bsp_plan_bins(plan, ctypes.byref(nb), abc.ctypes.data, cnt.ctypes.data), "bsp_plan_bins")
    return abc, cnt


def bsp_bins_aliased(n: int, edges, bins) -> np.ndarray:
    """Per bin (a, b, c): True where the grid's mod-n triangle sum may hold
    wrapped triangles (the library's flag, hi_a + hi_b + hi_c > n); host
    only."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    b = np.ascontiguousarray(bins, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(b.shape[0], dtype=np.int32)
    _check(load().bsp_bins_aliased(int(n), len(e) - 1, e.ctypes.data, int(b.shape[0]), b.ctypes.data,
                                   out.ctypes.data), "bsp_bins_aliased")
    return out.astype(bool)


def bsp_compute(plan: int, delta_k, B, ws, nbar: float = 0.0, stream=None):
    _check(load().bsp_compute(plan, _dptr(delta_k), float(nbar), _dptr(ws), _stream_handle(stream), _dptr(B)),
           "bsp_compute")


def bsp_compute_host(plan: int, delta_k_host: np.ndarray, B_host: np.ndarray, ws, nbar: float = 0.0,
                     stream=None):
    """delta_k_host / B_host: numpy arrays (ideally in pinned memory) or host pointers."""
    dptr = delta_k_host if isinstance(delta_k_host, int) else delta_k_host.ctypes.data
    bptr = B_host if isinstance(B_host, int) else B_host.ctypes.data
    _check(load().bsp_compute_host(plan, dptr, float(nbar), _dptr(ws), _stream_handle(stream), bptr),
           "bsp_compute_host")


def bsp_power_compute(plan: int, delta_k, P, ws, nbar: float = 0.0, stream=None, Nk=None):
    _check(load().bsp_power_compute(plan, _dptr(delta_k), float(nbar), _dptr(ws), _stream_handle(stream), _dptr(P),
                                    _dptr(Nk) if Nk is not None else None), "bsp_power_compute")


def density_from_particles(pos, n: int, box: float, ws=None, stream=None):
    """delta(k) (complex64 [n][n][n/2+1], device) and nbar from particle
    positions (float32 [N_p][3] CUDA tensor, box units) by CIC with
    interlacing (bsp_density_cic).  ``ws`` may be a reusable uint8 CUDA
    tensor of bsp_density_workspace_size(n) bytes."""
    import torch

    nb = ctypes.c_size_t()
    _check(load().bsp_density_workspace_size(int(n), ctypes.byref(nb)), "bsp_density_workspace_size")
    if ws is None or ws.numel() < nb.value:
        ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device="cuda")
    out = torch.empty((n, n, n // 2 + 1), dtype=torch.complex64, device="cuda")
    nbar = ctypes.c_double()
    pos = pos.contiguous()
    _check(load().bsp_density_cic(int(n), float(box), int(pos.shape[0]), _dptr(pos), _dptr(ws), int(ws.numel()),
                                  _stream_handle(stream), _dptr(out), ctypes.byref(nbar)), "bsp_density_cic")
    return out, nbar.value


def bsp_last_raw(plan: int, ws, T, stream=None):
    _check(load().bsp_last_raw(plan, _dptr(ws), _stream_handle(stream), _dptr(T)), "bsp_last_raw")


def bsp_device_status(plan: int) -> int:
    """The plan's device error word (0 = no kernel reported a problem)."""
    v = ctypes.c_int()
    st = load().bsp_device_status(plan, ctypes.byref(v))
    if st not in (BSP_OK, BSP_ETIMEOUT):
        _check(st, "bsp_device_status")
    return v.value


def bsp_plan_stats(plan: int) -> dict:
    st = (ctypes.c_double * 4)()
    _check(load().bsp_plan_stats(plan, st), "bsp_plan_stats")
    return {"issued_macs_per_point": st[0], "useful_macs_per_point": st[1], "works": int(st[2]),
            "nsplit": int(st[3])}


def bsp_set_accumulation_chunk(plan: int, points: int):
    _check(load().bsp_set_accumulation_chunk(plan, int(points)), "bsp_set_accumulation_chunk")


def bsp_plan_tune_tc(plan: int, max_rows: int = 0, chunk_points: int = 0):
    _check(load().bsp_plan_tune_tc(plan, int(max_rows), int(chunk_points)), "bsp_plan_tune_tc")


def bsp_set_wait_limit(plan: int, cycles: int):
    _check(load().bsp_set_wait_limit(plan, int(cycles)), "bsp_set_wait_limit")


def bsp_fp32_fma_peak(iters: int = 1 << 21, stream=None):
    """(TFLOP/s, ms) of the library's FP32 FMA throughput kernel on the current GPU."""
    import torch

    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    scratch = torch.empty(nsm * 1024, dtype=torch.float32, device="cuda")
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().bsp_fp32_fma_peak(int(iters), _stream_handle(stream), _dptr(scratch), ctypes.byref(tf),
                                    ctypes.byref(ms)), "bsp_fp32_fma_peak")
    return tf.value, ms.value


def bsp_set_profiling(plan: int, on: bool):
    _check(load().bsp_set_profiling(plan, int(bool(on))), "bsp_set_profiling")


def bsp_phase_times(plan: int):
    """(ms[3] = filter+FFT, contraction, reduction summed over calls; ncalls; launches per call)."""
    ms = (ctypes.c_double * 3)()
    nc, nl = ctypes.c_int(), ctypes.c_int()
    _check(load().bsp_phase_times(plan, ms, ctypes.byref(nc), ctypes.byref(nl)), "bsp_phase_times")
    return list(ms), nc.value, nl.value


def bsp_triple_sums_static(fields, npts: int, nfields: int, triplets: np.ndarray, T, stream=None):
    """T[t] = sum_x F_i F_j F_k with no device allocation (fields, T: CUDA
    tensors or device pointers; triplets: host int32 [ntrip][3])."""
    tr = np.ascontiguousarray(triplets, dtype=np.int32).reshape(-1, 3)
    _check(load().bsp_triple_sums_static(_dptr(fields), int(npts), int(nfields), tr.ctypes.data, int(tr.shape[0]),
                                         _dptr(T), _stream_handle(stream)), "bsp_triple_sums_static")


def bsp_version() -> int:
    return int(load().bsp_version())


class Batch:
    """Mock ensemble on uneven grids through bsp_batch_*: ``run(deltas,
    size_index)`` returns the device FP64 rows [n_mocks][n_ell*n_bins];
    ``covariance(rows)`` returns (mean, cov) on the device."""

    def __init__(self, sizes, box, edges, ells=(0, 2, 4), prec="fp32", autotune=True, stream=None):
        import torch

        lib = load()
        self.sizes = [int(v) for v in sizes]
        self.ells = tuple(ells)
        sz = np.ascontiguousarray(self.sizes, dtype=np.int32)
        e = np.ascontiguousarray(edges, dtype=np.float64)
        l_ = np.ascontiguousarray(ells, dtype=np.int32)
        h = _P()
        _check(lib.bsp_batch_create(ctypes.byref(h), len(self.sizes), sz.ctypes.data, float(box), int(e.size - 1),
                                    e.ctypes.data, int(l_.size), l_.ctypes.data, PRECISIONS.get(prec, prec), 0),
               "bsp_batch_create")
        self.h = h.value
        n = ctypes.c_size_t()
        _check(lib.bsp_batch_workspace_size(self.h, ctypes.byref(n)), "bsp_batch_workspace_size")
        self.ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device="cuda")
        _check(lib.bsp_batch_prepare(self.h, _dptr(self.ws), _stream_handle(stream), int(bool(autotune))),
               "bsp_batch_prepare")
        nb = ctypes.c_int()
        ctas = np.zeros(len(self.sizes), dtype=np.int32)
        fb = np.zeros(len(self.sizes), dtype=np.int32)
        ms = np.zeros(len(self.sizes))
        _check(lib.bsp_batch_info(self.h, ctypes.byref(nb), ctas.ctypes.data, fb.ctypes.data, ms.ctypes.data),
               "bsp_batch_info")
        self.nbins = nb.value
        rows_t = np.zeros(len(self.sizes), dtype=np.int32)
        chunk_t = np.zeros(len(self.sizes), dtype=np.int32)
        _check(lib.bsp_batch_tuning(self.h, rows_t.ctypes.data, chunk_t.ctypes.data), "bsp_batch_tuning")
        self.tuning = {"target_ctas": ctas.tolist(), "fft_batch": fb.tolist(), "tc_max_rows": rows_t.tolist(),
                       "tc_chunk_points": chunk_t.tolist(), "ms": ms.tolist()}
        self.bins = np.zeros((self.nbins, 3), dtype=np.int32)
        self.counts = np.zeros(self.nbins)
        _check(lib.bsp_batch_bins(self.h, self.bins.ctypes.data, self.counts.ctypes.data), "bsp_batch_bins")

    def run(self, deltas, size_index, rows=None, stream=None):
        """deltas: host complex64 arrays (pinned torch tensors or numpy)."""
        import torch

        m = len(deltas)
        d = len(self.ells) * self.nbins
        if rows is None:
            rows = torch.empty((m, d), dtype=torch.float64, device="cuda")
        ptrs = (ctypes.c_void_p * m)(*[(x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data) for x in deltas])
        si = np.ascontiguousarray(size_index, dtype=np.int32)
        _check(load().bsp_batch_run(self.h, m, si.ctypes.data, ptrs, _dptr(self.ws), _stream_handle(stream),
                                    _dptr(rows)), "bsp_batch_run")
        return rows

    @staticmethod
    def covariance(rows, stream=None):
        import torch

        m, d = rows.shape
        mean = torch.empty(d, dtype=torch.float64, device="cuda")
        cov = torch.empty((d, d), dtype=torch.float64, device="cuda")
        _check(load().bsp_covariance(int(m), int(d), _dptr(rows), _dptr(mean), _dptr(cov), _stream_handle(stream)),
               "bsp_covariance")
        return mean, cov

    def close(self):
        if getattr(self, "h", None):
            load().bsp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Modal:
    """A modal plan plus its workspace: ``compute(delta_k)`` returns the raw
    projections <<B_l|Q_pqr>> [n_ell][n_trip] (FP64, device)."""

    def __init__(self, n, box, radial, ells=(0, 2, 4), prec="fp32"):
        import torch

        self.n, self.box, self.ells = int(n), float(box), tuple(ells)
        self.plan = bsp_plan_create_modal(n, box, radial, ells, PRECISIONS.get(prec, prec))
        self.nf, self.ntrip = bsp_modal_size(self.plan)
        self.ws = torch.empty(max(bsp_workspace_size(self.plan), 256), dtype=torch.uint8, device="cuda")
        self.S = torch.empty((len(self.ells), self.ntrip), dtype=torch.float64, device="cuda")

    def compute(self, delta_k, stream=None):
        bsp_modal_compute(self.plan, delta_k, self.ws, self.S, stream)
        return self.S

    def close(self):
        if getattr(self, "plan", None):
            bsp_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Spectra:
    """A plan's shell tables without the bispectrum workspace or counts: the
    skew spectrum and the integrated bispectrum, each with a workspace of its
    own, on the plan's shells and multipoles."""

    def __init__(self, n, box, edges, ells=(0, 2, 4)):
        self.n, self.box, self.ells = int(n), float(box), tuple(ells)
        self.edges = [float(e) for e in edges]
        self.plan = bsp_plan_create(n, box, edges, ells, BSP_FP32, 0)

    def skew(self, delta_k, ws=None, stream=None):
        """Skew-spectrum multipoles S [n_ell][n_shells] and mode counts Nk (FP64,
        device) on the plan's shells; ``ws`` an optional reusable uint8 CUDA
        tensor of bsp_skew_workspace_size bytes."""
        import torch

        nb = ctypes.c_size_t()
        _check(load().bsp_skew_workspace_size(self.plan, ctypes.byref(nb)), "bsp_skew_workspace_size")
        if ws is None or ws.numel() < nb.value:
            ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device="cuda")
        S = torch.empty((len(self.ells), len(self.edges) - 1), dtype=torch.float64, device="cuda")
        Nk = torch.empty(len(self.edges) - 1, dtype=torch.float64, device="cuda")
        _check(load().bsp_skew_compute(self.plan, _dptr(delta_k), _dptr(ws), int(ws.numel()), _stream_handle(stream),
                                       _dptr(S), _dptr(Nk)), "bsp_skew_compute")
        return S, Nk

    def integrated(self, delta_k, m, ws=None, stream=None):
        """Integrated-bispectrum multipoles iB [n_ell][n_shells] over m^3
        sub-cubes and the per-cube mode counts Nk (FP64, device) on the plan's
        shells; ``ws`` an optional reusable uint8 CUDA tensor of
        bsp_ib_workspace_size bytes."""
        import torch

        nb = ctypes.c_size_t()
        _check(load().bsp_ib_workspace_size(self.plan, int(m), ctypes.byref(nb)), "bsp_ib_workspace_size")
        if ws is None or ws.numel() < nb.value:
            ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device="cuda")
        iB = torch.empty((len(self.ells), len(self.edges) - 1), dtype=torch.float64, device="cuda")
        Nk = torch.empty(len(self.edges) - 1, dtype=torch.float64, device="cuda")
        _check(load().bsp_ib_compute(self.plan, _dptr(delta_k), int(m), _dptr(ws), int(ws.numel()),
                                     _stream_handle(stream), _dptr(iB), _dptr(Nk)), "bsp_ib_compute")
        return iB, Nk

    def close(self):
        if getattr(self, "plan", None):
            bsp_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Bispectrum(Spectra):
    """A plan plus its device workspace (PyTorch-allocated), counts done on
    construction.  ``compute(delta_k)`` returns B [n_ell][n_bins] (FP64,
    device) for a complex64 [n][n][n/2+1] CUDA tensor."""

    def __init__(self, n, box, edges, ells=(0, 2, 4), prec="fp32", host_staging=False, stream=None,
                 counts_from=None, ws=None, shot_noise=False, full_tensor=False):
        import torch

        self.n, self.box, self.ells = int(n), float(box), tuple(ells)
        self.edges = [float(e) for e in edges]
        self.plan = bsp_plan_create(n, box, edges, ells, PRECISIONS.get(prec, prec),
                                    (BSP_SHOT_NOISE if shot_noise else 0) | (BSP_FULL_TENSOR if full_tensor else 0))
        nbytes = bsp_workspace_size(self.plan)
        if host_staging:
            nbytes += bsp_host_staging_size(self.plan)
        if ws is not None and ws.numel() >= nbytes:
            self.ws = ws
        else:
            self.ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
        if counts_from is not None:
            bsp_plan_share_counts(self.plan, counts_from.plan)
        else:
            bsp_counts(self.plan, self.ws, stream)
        self.bins, self.counts = bsp_plan_bins(self.plan)
        # bins whose mod-n sum may hold wrapped triangles (the library's flag)
        self.aliased = bsp_bins_aliased(self.n, self.edges, self.bins)
        self.B = torch.empty((len(self.ells), len(self.bins)), dtype=torch.float64, device="cuda")

    def compute(self, delta_k, nbar: float = 0.0, stream=None):
        bsp_compute(self.plan, delta_k, self.B, self.ws, nbar, stream)
        return self.B

    def compute_host(self, delta_k_host, B_host, nbar: float = 0.0, stream=None):
        bsp_compute_host(self.plan, delta_k_host, B_host, self.ws, nbar, stream)
        return B_host

    def power(self, delta_k, nbar: float = 0.0, stream=None):
        """Power-spectrum multipoles P [n_ell][n_shells] and mode counts Nk
        [n_shells] (FP64, device) of delta_k on the plan's shells; uses the
        start of the plan's workspace."""
        import torch

        P = torch.empty((len(self.ells), len(self.edges) - 1), dtype=torch.float64, device="cuda")
        Nk = torch.empty(len(self.edges) - 1, dtype=torch.float64, device="cuda")
        bsp_power_compute(self.plan, delta_k, P, self.ws, nbar, stream, Nk)
        return P, Nk

    def raw(self, stream=None):
        import torch

        T = torch.empty_like(self.B)
        bsp_last_raw(self.plan, self.ws, T, stream)
        return T

    def close(self):
        if getattr(self, "plan", None):
            bsp_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
