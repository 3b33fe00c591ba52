"""Python binding of libgwfish, the GB300 Fisher-forecast library.

Argument marshalling only: every step of SNR, Fisher, inversion and the VJPs
runs in the CUDA kernels of ``libgwfish.so`` (C ABI in ``include/gwfish.h``).
PyTorch provides device memory and streams.  The functions keep the C names:
``gw_prepare_catalog``, ``gw_snr``, ``gw_fisher``, ``gw_fisher_inverse``,
``gw_snr_vjp``, ``gw_logdet_vjp_detangles``.  ``SNR`` wraps ``gw_snr`` and
``gw_snr_vjp`` as a ``torch.autograd.Function``.

The library must be built (``paper_2207_06910_gb300.build.build()`` or
``__graft_entry__.build()``); importing this module fails loudly otherwise,
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

GW_FP64, GW_MIXED, GW_DFLOAT = 0, 1, 2
ST_NOT_PD, ST_COND_GT_MAX, ST_NONFINITE, ST_EMPTY_GRID, ST_BAD_PARAM, ST_ILL_COND = 1, 2, 4, 8, 16, 32
ST_OVERFLOW = 64
ITEM_POINTS = 256          # grid points per work item (GW_ITEM_POINTS)
TC_ITEM_POINTS = 128       # the tensor-core Fisher pass (GW_TC_ITEM_POINTS)
FISHER_PARAMS_9 = ("Mc", "eta", "dL", "theta", "phi", "iota", "psi", "tc", "Phic")

_P = ctypes.c_void_p


class gw_catalog(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(k, _P) for k in (
        "Mc", "eta", "dL", "theta", "phi", "iota", "psi", "tc", "Phic",
        "chi1z", "chi2z", "LamT", "dLamT", "pset", "fmin", "fmax", "npts", "arm_mask", "sel")]


class gw_detector(ctypes.Structure):
    _fields_ = [("lat", ctypes.c_double), ("lon", ctypes.c_double), ("gamma", ctypes.c_double),
                ("zeta", ctypes.c_double), ("shape", ctypes.c_int32), ("psd", ctypes.c_int32)]


class gw_psd(ctypes.Structure):
    _fields_ = [("f0", ctypes.c_double), ("scale", ctypes.c_double), ("nterm", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("coef", ctypes.c_double * 4),
                ("pw", ctypes.c_double * 4), ("table_f", _P), ("table_s", _P),
                ("n_table", ctypes.c_int32), ("is_asd", ctypes.c_int32)]


GW_PSD_POWER_SUM, GW_PSD_TABLE = 0, 1


class gw_network(ctypes.Structure):
    _fields_ = [("n_det", ctypes.c_int32), ("earth_rotation", ctypes.c_int32),
                ("det", ctypes.POINTER(gw_detector)), ("n_psd", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("psd", ctypes.POINTER(gw_psd))]


EXPORTS = ("gw_create", "gw_destroy", "gw_last_error", "gw_abi_version", "gw_prepare_catalog",
           "gw_snr", "gw_fisher", "gw_fisher_inverse", "gw_snr_vjp", "gw_logdet_vjp_detangles",
           "gw_set_profiling", "gw_point_kernel_ms", "gw_fisher_noalloc", "gw_reserve",
           "gw_select_snr", "gw_fisher_eig", "gw_covariance", "gw_packed_submatrix",
           "gw_sky_area", "gw_strain", "gw_perturb_fisher", "gw_logdet_vjp_detangles_masked",
           "gw_fma_rate", "gw_fisher_refine", "gw_set_tile", "gw_autotune", "gw_set_fp64_gram",
           "gw_kernel_faults", "gw_fisher_routed")

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(path: str | None = None):
    """Load libgwfish.so and declare its signatures (no GPU needed)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libgwfish.so is not built ({p}); run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    i32, i64, d = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    C, N = ctypes.POINTER(gw_catalog), ctypes.POINTER(gw_network)
    lib.gw_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int]
    lib.gw_destroy.argtypes = [_P]
    lib.gw_last_error.argtypes = [_P]
    lib.gw_last_error.restype = ctypes.c_char_p
    lib.gw_abi_version.restype = ctypes.c_int
    lib.gw_prepare_catalog.argtypes = [_P, i64] + [_P] * 11 + [i32, d, i32, i32] + [_P] * 10 + [_P]
    lib.gw_snr.argtypes = [_P, C, N, ctypes.c_int, _P, _P, _P, _P]
    lib.gw_fisher.argtypes = [_P, C, N, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P]
    lib.gw_fisher_inverse.argtypes = [_P, _P, i64, ctypes.c_int, d, _P, _P, _P, _P, _P]
    lib.gw_snr_vjp.argtypes = [_P, C, N, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]
    lib.gw_logdet_vjp_detangles.argtypes = [_P, C, N, ctypes.c_int, ctypes.c_int, _P, _P, _P]
    lib.gw_logdet_vjp_detangles_masked.argtypes = [_P, C, N, ctypes.c_int, ctypes.c_int, _P,
                                                   ctypes.c_uint32, _P, _P]
    for name in EXPORTS:
        if name not in ("gw_last_error", "gw_abi_version", "gw_destroy", "gw_point_kernel_ms"):
            getattr(lib, name).restype = ctypes.c_int
    lib.gw_destroy.restype = ctypes.c_int
    lib.gw_reserve.argtypes = [_P, i64, i64, ctypes.c_int]
    lib.gw_fisher_noalloc.argtypes = [C, N, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]
    lib.gw_select_snr.argtypes = [_P, _P, i64, d, _P, ctypes.POINTER(i64), _P]
    lib.gw_strain.argtypes = [_P, C, N, ctypes.c_int, i64, _P, _P, _P, _P, _P, _P]
    lib.gw_fisher_eig.argtypes = [_P, _P, i64, ctypes.c_int, ctypes.c_int, _P, _P, _P]
    lib.gw_covariance.argtypes = [_P, _P, i64, ctypes.c_int, ctypes.c_uint32, _P, ctypes.c_int, d,
                                  d, _P, _P, _P, _P, _P]
    lib.gw_packed_submatrix.argtypes = [_P, _P, i64, ctypes.c_int, ctypes.c_uint32, _P, _P]
    lib.gw_perturb_fisher.argtypes = [_P, _P, i64, ctypes.c_int, d, _P, _P, _P]
    lib.gw_sky_area.argtypes = [_P, _P, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, d,
                                ctypes.c_int, _P, _P]
    lib.gw_fisher_refine.argtypes = [_P, C, N, ctypes.c_int, d, d] + [_P] * 10 + [
        ctypes.POINTER(i64), _P]
    lib.gw_fisher_routed.argtypes = [_P, C, N, ctypes.c_int, ctypes.c_uint32, d, d] + [_P] * 9 + [
        ctypes.POINTER(i64), ctypes.POINTER(i64), _P]
    lib.gw_set_tile.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.gw_set_fp64_gram.argtypes = [_P, ctypes.c_int]
    lib.gw_kernel_faults.argtypes = [_P, ctypes.POINTER(i32), ctypes.c_int]
    lib.gw_autotune.argtypes = [_P, C, N, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                ctypes.POINTER(d), _P]
    lib.gw_fma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(d), ctypes.POINTER(d),
                                ctypes.POINTER(d), _P]
    lib.gw_set_profiling.argtypes = [_P, ctypes.c_int]
    lib.gw_point_kernel_ms.argtypes = [_P]
    lib.gw_point_kernel_ms.restype = ctypes.c_double
    if path is None:
        _lib = lib
    return lib


class GWError(RuntimeError):
    pass


_ctx_by_dev: dict[int, _P] = {}


def context(device: int | None = None) -> _P:
    """The library context of a CUDA device (created on first use)."""
    if device is None:
        device = torch.cuda.current_device()
    if device not in _ctx_by_dev:
        lib = load_library()
        h = _P()
        st = lib.gw_create(ctypes.byref(h), int(device))
        if st != 0:
            raise GWError(f"gw_create failed with status {st}")
        _ctx_by_dev[device] = h
    return _ctx_by_dev[device]


def gw_reserve(max_events: int, max_items: int, max_sites: int = 1) -> None:
    """Pre-size the workspace and switch to asynchronous (graph-capturable) mode;
    max_items = 0 returns to the synchronous default."""
    ctx = context()
    _check(load_library().gw_reserve(ctx, int(max_events), int(max_items), int(max_sites)), ctx)


def work_items(npts, points_per_item: int | None = None) -> int:
    """Number of work items of a catalog with these grid lengths (items of
    ITEM_POINTS points, or TC_ITEM_POINTS for the tensor-core Fisher pass)."""
    p = ITEM_POINTS if points_per_item is None else int(points_per_item)
    n = torch.as_tensor(npts).to(torch.int64)
    return int(((n + p - 1) // p).sum().item())


def gw_set_profiling(enable: bool = True) -> None:
    """Record CUDA events around every point-loop kernel launch."""
    ctx = context()
    _check(load_library().gw_set_profiling(ctx, int(enable)), ctx)


def gw_point_kernel_ms() -> float:
    """Duration of the last point-loop kernel (ms), -1 if none recorded."""
    return load_library().gw_point_kernel_ms(context())


LENGTH_CLASSES = ("short", "medium", "long")     # <= ~380, <= ~3000, longer grids
TILES = [(g, b) for g in (4, 8, 16) for b in (1, 2)]


def gw_set_tile(prec: int, length_class: int, group: int, blocks_per_sm: int) -> None:
    """Fisher-pass tile (lanes per work item, CTAs per SM) of a precision and
    grid-length class (0 short, 1 medium, 2 long) on the current device."""
    ctx = context()
    _check(load_library().gw_set_tile(ctx, int(prec), int(length_class), int(group),
                                      int(blocks_per_sm)), ctx)


def gw_set_fp64_gram(tensor: bool) -> None:
    """FP64 Fisher pass: Gram matrix of the tangents on the tensor cores (exact
    digit products) or every product on the FP64 pipe (the default)."""
    ctx = context()
    _check(load_library().gw_set_fp64_gram(ctx, int(bool(tensor))), ctx)


def gw_kernel_faults(reset: bool = True) -> int:
    """1 if a kernel's bounded wait ran out since the last reset (its items'
    sums are NaN), else 0; synchronises the device."""
    ctx = context()
    f = ctypes.c_int32(0)
    _check(load_library().gw_kernel_faults(ctx, ctypes.byref(f), int(bool(reset))), ctx)
    return int(f.value)


def gw_autotune(cat: "Catalog", net: "Network", n_par: int, prec=GW_MIXED, reps: int = 3,
                stream=None) -> dict:
    """Time every tile of the Fisher pass on this catalog, install the fastest
    for its grid-length class: {'length_class', 'group', 'blocks_per_sm',
    'ms': {(group, blocks): ms}}."""
    ctx = context()
    c = cat.struct()
    cls, g, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ms = (ctypes.c_double * 6)()
    _check(load_library().gw_autotune(ctx, ctypes.byref(c), ctypes.byref(net.net), int(prec),
                                      int(n_par), int(reps), ctypes.byref(cls), ctypes.byref(g),
                                      ctypes.byref(b), ms, _stream(stream)), ctx)
    return {"length_class": cls.value, "group": g.value, "blocks_per_sm": b.value,
            "ms": {t: ms[i] for i, t in enumerate(TILES)}}


def gw_fma_rate(fp64: bool, iters: int | None = None, stream=None) -> dict:
    """Measured FMA throughput of the FP64 or FP32 pipe of the current device:
    {'fma_per_clk_sm', 'fma_per_s', 'sm_mhz', 'sms'}."""
    if iters is None:
        iters = 4096 if fp64 else 65536
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = load_library().gw_fma_rate(int(bool(fp64)), int(iters), ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c), _stream(stream))
    if st != 0:
        raise GWError(f"gw_fma_rate failed with status {st}")
    return {"fma_per_clk_sm": a.value, "fma_per_s": b.value, "sm_mhz": c.value,
            "sms": torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count}


def _check(st: int, ctx) -> None:
    if st != 0:
        msg = load_library().gw_last_error(ctx).decode(errors="replace")
        raise GWError(f"libgwfish status {st}: {msg}")


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError("device arrays must be contiguous CUDA tensors")
    return _P(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _P(s.cuda_stream)


class Catalog:
    """Device-resident catalog (structure of arrays, float64 / int8 / int32), with
    optional duty-factor arm masks (uint32 stored as int32, one per row) and an
    optional selection of rows (int64 indices; the catalog then holds
    ``len(sel)`` events)."""

    FIELDS = ("Mc", "eta", "dL", "theta", "phi", "iota", "psi", "tc", "Phic",
              "chi1z", "chi2z", "LamT", "dLamT")

    def __init__(self, tensors: dict, pset, fmin, fmax, npts, arm_mask=None, sel=None):
        self.t = {k: tensors.get(k) for k in self.FIELDS}
        self.pset, self.fmin, self.fmax, self.npts = pset, fmin, fmax, npts
        self.arm_mask, self.sel = arm_mask, sel
        self.n = int(sel.numel()) if sel is not None else int(self.t["Mc"].numel())

    @classmethod
    def from_numpy(cls, ev: np.ndarray, pset, fmin, fmax, npts, device="cuda", arm_mask=None):
        """From oracle-style event rows [n, 13] (order of ``FIELDS``)."""
        ev = np.asarray(ev, dtype=np.float64).reshape(-1, 13)
        n = ev.shape[0]
        t = {k: torch.as_tensor(np.ascontiguousarray(ev[:, i]), device=device)
             for i, k in enumerate(cls.FIELDS)}
        col = lambda a, dt: torch.as_tensor(np.array(np.broadcast_to(a, (n,)), dtype=dt), device=device)
        mask = None
        if arm_mask is not None:
            mask = col(np.asarray(arm_mask, dtype=np.uint32).view(np.int32), np.int32)
        return cls(t, col(pset, np.int8), col(fmin, np.float64), col(fmax, np.float64),
                   col(npts, np.int32), mask)

    def struct(self) -> gw_catalog:
        c = gw_catalog()
        c.n = self.n
        for k in self.FIELDS:
            setattr(c, k, _ptr(self.t[k]))
        c.pset, c.fmin, c.fmax, c.npts = (_ptr(self.pset), _ptr(self.fmin), _ptr(self.fmax),
                                          _ptr(self.npts))
        if self.arm_mask is not None and self.arm_mask.dtype != torch.int32:
            raise TypeError("arm_mask must be an int32 (bit pattern of uint32) tensor")
        if self.sel is not None and self.sel.dtype != torch.int64:
            raise TypeError("sel must be an int64 tensor")
        c.arm_mask, c.sel = _ptr(self.arm_mask), _ptr(self.sel)
        return c

    def with_field(self, name, tensor):
        t = dict(self.t)
        t[name] = tensor
        return Catalog(t, self.pset, self.fmin, self.fmax, self.npts, self.arm_mask, self.sel)

    def with_arm_mask(self, arm_mask):
        """Same rows with duty-factor arm masks (int32 tensor, one per row; None = all on)."""
        return Catalog(self.t, self.pset, self.fmin, self.fmax, self.npts, arm_mask, self.sel)

    def select(self, sel):
        """The events at rows ``sel`` (int64 tensor) of this catalog's columns."""
        if self.sel is not None:
            sel = self.sel[sel]
        return Catalog(self.t, self.pset, self.fmin, self.fmax, self.npts, self.arm_mask, sel)


class Network:
    """Host-side detector network (see gw_network in include/gwfish.h).

    PSD rows are ``f0, scale, nterm, c0..c3, p0..p3`` (a power sum); a row with
    nterm = -(k+1) is tabulated noise curve k of ``tables``, a list of
    (f, values, is_asd) with f and values 1-D float64 arrays (numpy or CUDA
    tensors, copied to the device), times the row's scale."""

    def __init__(self, det, psd, rotation: int, tables=None, device="cuda"):
        det = np.asarray(det, dtype=np.float64).reshape(-1, 6)
        psd = np.asarray(psd, dtype=np.float64).reshape(-1, 11)
        self.det_rows, self.psd_rows, self.rotation = det, psd, int(rotation)
        self.tables = []
        for f, v, asd in (tables or []):
            f = torch.as_tensor(f, dtype=torch.float64, device=device).contiguous()
            v = torch.as_tensor(v, dtype=torch.float64, device=device).contiguous()
            if f.dim() != 1 or f.shape != v.shape:
                raise ValueError("a PSD table needs 1-D frequency and value arrays of one length")
            self.tables.append((f, v, bool(asd)))
        self._dets = (gw_detector * len(det))()
        for i, r in enumerate(det):
            self._dets[i] = gw_detector(r[0], r[1], r[2], r[3], int(r[4]), int(r[5]))
        self._psds = (gw_psd * len(psd))()
        for i, r in enumerate(psd):
            p = gw_psd()
            p.f0, p.scale, p.nterm = r[0], r[1], int(r[2])
            if p.nterm < 0:
                k = -p.nterm - 1
                if k >= len(self.tables):
                    raise ValueError(f"psd row {i} reads table {k}; {len(self.tables)} given")
                f, v, asd = self.tables[k]
                p.kind, p.nterm = GW_PSD_TABLE, 0
                p.table_f, p.table_s = _P(f.data_ptr()), _P(v.data_ptr())
                p.n_table, p.is_asd = int(f.numel()), int(asd)
            for j in range(4):
                p.coef[j] = r[3 + j]
                p.pw[j] = r[7 + j]
            self._psds[i] = p
        self.net = gw_network(len(det), self.rotation, self._dets, len(psd), 0, self._psds)

    @property
    def n_det(self) -> int:
        return len(self.det_rows)

    def with_gamma(self, d: int, gamma: float) -> "Network":
        det = self.det_rows.copy()
        det[d, 2] = gamma
        return Network(det, self.psd_rows, self.rotation, self.tables)


def n_packed(n_par: int) -> int:
    return n_par * (n_par + 1) // 2


def unpack(packed: torch.Tensor, n_par: int) -> torch.Tensor:
    """[P(P+1)/2, n] packed upper, event-minor  ->  [n, P, P] (a view copy)."""
    n = packed.shape[1]
    out = torch.empty((n, n_par, n_par), dtype=packed.dtype, device=packed.device)
    k = 0
    for i in range(n_par):
        for j in range(i, n_par):
            out[:, i, j] = packed[k]
            out[:, j, i] = packed[k]
            k += 1
    return out


# ---------------------------------------------------------------- entry points
def gw_prepare_catalog(raw: dict, npts_rule, device="cuda", stream=None) -> Catalog:
    """Raw seeded draws (m1, m2, chi1, chi2, lam1, lam2, dL_Mpc, zflag, tcoal,
    theta, phi, iota, psi, Phic, pset, fmin, optional npts) -> device Catalog."""
    ctx = context()
    f64 = lambda k: torch.as_tensor(np.ascontiguousarray(raw[k], np.float64), device=device)
    n = len(raw["m1"])
    ins = {k: f64(k) for k in ("m1", "m2", "chi1", "chi2", "lam1", "lam2", "dL_Mpc", "tcoal", "fmin")}
    zflag = torch.as_tensor(np.ascontiguousarray(raw["zflag"], np.uint8), device=device)
    given = None
    fixed, per, lo, hi = 0, 0.0, 0, 0
    if npts_rule[0] == "fixed":
        fixed = int(npts_rule[1])
    elif npts_rule[0] == "efold":
        per, lo, hi = float(npts_rule[1]), int(npts_rule[2]), int(npts_rule[3])
    else:
        given = torch.as_tensor(np.ascontiguousarray(raw["npts"], np.int32), device=device)
    out = {k: torch.empty(n, dtype=torch.float64, device=device) for k in
           ("Mc", "eta", "dL", "chi1z", "chi2z", "LamT", "dLamT", "tc", "fmax")}
    npts = torch.empty(n, dtype=torch.int32, device=device)
    st = load_library().gw_prepare_catalog(
        ctx, n, _ptr(ins["m1"]), _ptr(ins["m2"]), _ptr(ins["chi1"]), _ptr(ins["chi2"]),
        _ptr(ins["lam1"]), _ptr(ins["lam2"]), _ptr(ins["dL_Mpc"]), _ptr(zflag), _ptr(ins["tcoal"]),
        _ptr(ins["fmin"]), _ptr(given), fixed, per, lo, hi,
        _ptr(out["Mc"]), _ptr(out["eta"]), _ptr(out["dL"]), _ptr(out["chi1z"]), _ptr(out["chi2z"]),
        _ptr(out["LamT"]), _ptr(out["dLamT"]), _ptr(out["tc"]), _ptr(out["fmax"]), _ptr(npts),
        _stream(stream))
    _check(st, ctx)
    t = dict(out)
    for k in ("theta", "phi", "iota", "psi", "Phic"):
        t[k] = f64(k)
    pset = torch.as_tensor(np.ascontiguousarray(raw["pset"], np.int8), device=device)
    return Catalog(t, pset, ins["fmin"], out["fmax"], npts)


def gw_snr(cat: Catalog, net: Network, prec=GW_FP64, per_detector=False, stream=None):
    ctx = context()
    dev = cat.t["Mc"].device
    snr = torch.empty(cat.n, dtype=torch.float64, device=dev)
    sdet = torch.empty((net.n_det, cat.n), dtype=torch.float64, device=dev) if per_detector else None
    status = torch.empty(cat.n, dtype=torch.int32, device=dev)
    c = cat.struct()
    st = load_library().gw_snr(ctx, ctypes.byref(c), ctypes.byref(net.net), int(prec), _ptr(snr),
                               _ptr(sdet), _ptr(status), _stream(stream))
    _check(st, ctx)
    return (snr, sdet, status) if per_detector else (snr, status)


def gw_select_snr(snr: torch.Tensor, threshold: float, stream=None) -> torch.Tensor:
    """Detection gate (the snr_th option of Sec. 5): int64 indices of the events
    with SNR above ``threshold``, in increasing order (synchronises the stream)."""
    ctx = context()
    n = int(snr.numel())
    sel = torch.empty(n, dtype=torch.int64, device=snr.device)
    cnt = ctypes.c_int64(0)
    _check(load_library().gw_select_snr(ctx, _ptr(snr), n, float(threshold), _ptr(sel),
                                        ctypes.byref(cnt), _stream(stream)), ctx)
    return sel[:cnt.value]


def gw_fisher(cat: Catalog, net: Network, n_par: int, prec=GW_FP64, stream=None, out=None,
              grad_snr: torch.Tensor | None = None):
    """Returns (fisher [P(P+1)/2, n] packed upper event-minor, snr [n], status [n]);
    with ``grad_snr`` [n] also the fused SNR VJP grad_params [P, n] (4th item)."""
    ctx = context()
    dev = cat.t["Mc"].device
    if out is None:
        fisher = torch.empty((n_packed(n_par), cat.n), dtype=torch.float64, device=dev)
        snr = torch.empty(cat.n, dtype=torch.float64, device=dev)
        status = torch.empty(cat.n, dtype=torch.int32, device=dev)
        gp = (torch.empty((n_par, cat.n), dtype=torch.float64, device=dev)
              if grad_snr is not None else None)
    else:
        fisher, snr, status = out[:3]
        gp = out[3] if len(out) > 3 else None
    c = cat.struct()
    st = load_library().gw_fisher(ctx, ctypes.byref(c), ctypes.byref(net.net), int(prec), n_par,
                                  _ptr(fisher), _ptr(snr), _ptr(status),
                                  _ptr(grad_snr.contiguous() if grad_snr is not None else None),
                                  _ptr(gp), _stream(stream))
    _check(st, ctx)
    return (fisher, snr, status, gp) if grad_snr is not None else (fisher, snr, status)


GW_ETOOLARGE = 5


def gw_fisher_noalloc(cat: Catalog, net: Network, n_par: int, fisher: torch.Tensor,
                      snr: torch.Tensor | None, status: torch.Tensor, prec=GW_FP64,
                      stream=None) -> int:
    """Allocation-free Fisher pass into caller-provided tensors; returns the C
    status (0 ok, GW_ETOOLARGE when the request exceeds the static workspace)."""
    c = cat.struct()
    return load_library().gw_fisher_noalloc(ctypes.byref(c), ctypes.byref(net.net), int(prec),
                                            n_par, _ptr(fisher), _ptr(snr), _ptr(status),
                                            _stream(stream))


def gw_fisher_inverse(fisher: torch.Tensor, n_par: int, cond_max=1e50, stream=None, out=None):
    """Returns (cov packed like fisher, cond [n], inv_err [n], status [n])."""
    ctx = context()
    n = fisher.shape[1]
    if out is None:
        cov = torch.empty_like(fisher)
        cond = torch.empty(n, dtype=torch.float64, device=fisher.device)
        err = torch.empty(n, dtype=torch.float64, device=fisher.device)
        status = torch.empty(n, dtype=torch.int32, device=fisher.device)
    else:
        cov, cond, err, status = out
    st = load_library().gw_fisher_inverse(ctx, _ptr(fisher), n, n_par, float(cond_max), _ptr(cov),
                                          _ptr(cond), _ptr(err), _ptr(status), _stream(stream))
    _check(st, ctx)
    return cov, cond, err, status


REFINE_COND = 1e7      # default condition-number threshold of gw_fisher_refine


def gw_fisher_refine(cat: Catalog, net: Network, n_par: int, fisher, snr, status, inv,
                     grad_snr=None, grad_params=None, cond_th=REFINE_COND, cond_max=1e50,
                     refined=None, stream=None) -> int:
    """Recompute in FP64, in place, the events of a mixed pass whose inversion
    failed or whose condition number exceeds ``cond_th``.  ``inv`` is the
    (cov, cond, inv_err, status) tuple of gw_fisher_inverse; ``refined`` an
    optional uint8 [n] output.  Returns the number of refined events."""
    ctx = context()
    cov, cond, err, sti = inv
    c = cat.struct()
    cnt = ctypes.c_int64(0)
    st = load_library().gw_fisher_refine(
        ctx, ctypes.byref(c), ctypes.byref(net.net), n_par, float(cond_th), float(cond_max),
        _ptr(fisher), _ptr(snr), _ptr(status),
        _ptr(grad_snr.contiguous() if grad_snr is not None else None), _ptr(grad_params),
        _ptr(cov), _ptr(cond), _ptr(err), _ptr(sti), _ptr(refined), ctypes.byref(cnt),
        _stream(stream))
    _check(st, ctx)
    return int(cnt.value)


def gw_fisher_routed(cat: Catalog, net: Network, n_par: int, dfloat_psets: int = 1 << 1,
                     grad_snr: torch.Tensor | None = None, cond_th=REFINE_COND, cond_max=1e50,
                     stream=None, out=None):
    """Fisher pass and inversion with the precision chosen per event: parameter
    sets with their bit in ``dfloat_psets`` in double-float, the others mixed,
    those of them with a failed inversion or a condition number above
    ``cond_th`` recomputed in double-float.  Returns (fisher, snr, status, cov,
    cond, inv_err, inv_status[, grad_params], n_dfloat, n_refined), n_refined
    the mixed events recomputed."""
    ctx = context()
    dev = cat.t["Mc"].device
    n, npk = cat.n, n_packed(n_par)
    if out is None:
        f64 = dict(dtype=torch.float64, device=dev)
        fisher, snr = torch.empty((npk, n), **f64), torch.empty(n, **f64)
        status = torch.empty(n, dtype=torch.int32, device=dev)
        cov, cond, err = torch.empty((npk, n), **f64), torch.empty(n, **f64), torch.empty(n, **f64)
        sti = torch.empty(n, dtype=torch.int32, device=dev)
        gp = torch.empty((n_par, n), **f64) if grad_snr is not None else None
    else:
        fisher, snr, status, cov, cond, err, sti = out[:7]
        gp = out[7] if len(out) > 7 else None
    c = cat.struct()
    n_df, n_ref = ctypes.c_int64(0), ctypes.c_int64(0)
    st = load_library().gw_fisher_routed(
        ctx, ctypes.byref(c), ctypes.byref(net.net), n_par, int(dfloat_psets), float(cond_th),
        float(cond_max), _ptr(fisher), _ptr(snr), _ptr(status),
        _ptr(grad_snr.contiguous() if grad_snr is not None else None), _ptr(gp), _ptr(cov),
        _ptr(cond), _ptr(err), _ptr(sti), ctypes.byref(n_df), ctypes.byref(n_ref), _stream(stream))
    _check(st, ctx)
    res = (fisher, snr, status, cov, cond, err, sti) + ((gp,) if grad_snr is not None else ())
    return res + (int(n_df.value), int(n_ref.value))


def gw_snr_vjp(cat: Catalog, net: Network, n_par: int, grad_snr: torch.Tensor, prec=GW_FP64,
               stream=None, out=None, det_gamma=False):
    """grad_params [n_par, n] = grad_snr * d SNR / d theta; with ``det_gamma``
    also (grad_params, grad_gamma [n_det]) with grad_gamma[d] =
    sum_e grad_snr[e] d SNR_e / d gamma_d (detector orientations)."""
    ctx = context()
    g = out if out is not None else torch.empty((n_par, cat.n), dtype=torch.float64,
                                                device=grad_snr.device)
    gg = torch.empty(net.n_det, dtype=torch.float64, device=grad_snr.device) if det_gamma else None
    c = cat.struct()
    st = load_library().gw_snr_vjp(ctx, ctypes.byref(c), ctypes.byref(net.net), int(prec), n_par,
                                   _ptr(grad_snr.contiguous()), _ptr(g), _ptr(gg), _stream(stream))
    _check(st, ctx)
    return (g, gg) if det_gamma else g


def gw_logdet_vjp_detangles(cat: Catalog, net: Network, n_par: int, cov: torch.Tensor,
                            prec=GW_FP64, stream=None, out=None, det_mask=None):
    """d(sum_e log det Gamma_e)/d gamma_d for every detector d -> [n_det];
    with ``det_mask`` (bit d: detector d) only for those detectors, the others
    NaN (``gw_logdet_vjp_detangles_masked``)."""
    ctx = context()
    g = out if out is not None else torch.empty(net.n_det, dtype=torch.float64, device=cov.device)
    c = cat.struct()
    lib = load_library()
    if det_mask is None:
        st = lib.gw_logdet_vjp_detangles(ctx, ctypes.byref(c), ctypes.byref(net.net), int(prec),
                                         n_par, _ptr(cov), _ptr(g), _stream(stream))
    else:
        st = lib.gw_logdet_vjp_detangles_masked(ctx, ctypes.byref(c), ctypes.byref(net.net),
                                                int(prec), n_par, _ptr(cov), int(det_mask),
                                                _ptr(g), _stream(stream))
    _check(st, ctx)
    return g


class SNR(torch.autograd.Function):
    """Network SNR as a differentiable function of the catalog's Fisher
    parameters: forward = gw_snr, backward = gw_snr_vjp."""

    @staticmethod
    def forward(ctx_, params: torch.Tensor, base: Catalog, net: Network, n_par: int, prec: int):
        # params [n_par, n] float64 on the device, order of the Fisher slots;
        # slots 9, 10 are (chi1z, chi2z) for pset 1 events, (LamT, dLamT) for pset 2
        cat = base
        for i, k in enumerate(FISHER_PARAMS_9):
            cat = cat.with_field(k, params[i].contiguous())
        if n_par == 11:
            spin = base.pset == 1
            tide = base.pset == 2
            for i, (ks, kt) in enumerate((("chi1z", "LamT"), ("chi2z", "dLamT"))):
                row = params[9 + i]
                zs = base.t[ks] if base.t[ks] is not None else torch.zeros_like(row)
                zt = base.t[kt] if base.t[kt] is not None else torch.zeros_like(row)
                cat = cat.with_field(ks, torch.where(spin, row, zs).contiguous())
                cat = cat.with_field(kt, torch.where(tide, row, zt).contiguous())
        ctx_.cat, ctx_.net, ctx_.n_par, ctx_.prec = cat, net, n_par, prec
        snr, status = gw_snr(cat, net, prec)
        return snr

    @staticmethod
    def backward(ctx_, grad):
        g = gw_snr_vjp(ctx_.cat, ctx_.net, ctx_.n_par, grad.to(torch.float64).contiguous(),
                       ctx_.prec)
        return g, None, None, None, None


# ---- covariance tools (Secs. 4.1-4.2)
GW_INV_CHO, GW_INV_CHO_SVD, GW_INV_SVD, GW_INV_SVD_TRUNC, GW_INV_SVD_REG, GW_INV_LU = range(6)
GW_ST_SVD_FALLBACK = 128


def _keep_mask(keep, n_par: int) -> tuple[int, int]:
    if keep is None:
        return 0, n_par
    m = 0
    for i in keep:
        if not 0 <= int(i) < n_par:
            raise ValueError(f"parameter slot {i} outside [0, {n_par})")
        m |= 1 << int(i)
    return m, bin(m).count("1")


def gw_fisher_eig(fisher: torch.Tensor, n_par: int, normalize=True, vectors=True, stream=None):
    """Eigenvalues [n_par, n] (ascending) and eigenvectors [n_par * n_par, n] of
    packed Fisher matrices (CheckFisher)."""
    ctx = context()
    n = fisher.shape[1]
    w = torch.empty((n_par, n), dtype=torch.float64, device=fisher.device)
    V = torch.empty((n_par * n_par, n), dtype=torch.float64, device=fisher.device) if vectors else None
    _check(load_library().gw_fisher_eig(ctx, _ptr(fisher), n, n_par, int(bool(normalize)), _ptr(w),
                                        _ptr(V), _stream(stream)), ctx)
    return w, V


def gw_covariance(fisher: torch.Tensor, n_par: int, keep=None, prior=None, method=GW_INV_CHO_SVD,
                  thresh=1e-15, cond_max=1e50, stream=None):
    """Covariance after fixParams (``keep``: kept slots) and addPrior (``prior``:
    [n_par] host values) with a CovMatr inversion method.  Returns (cov packed
    over the kept parameters, cond [n], inv_err [n], status [n])."""
    ctx = context()
    n = fisher.shape[1]
    mask, k = _keep_mask(keep, n_par)
    cov = torch.empty((k * (k + 1) // 2, n), dtype=torch.float64, device=fisher.device)
    cond = torch.empty(n, dtype=torch.float64, device=fisher.device)
    err = torch.empty(n, dtype=torch.float64, device=fisher.device)
    status = torch.empty(n, dtype=torch.int32, device=fisher.device)
    pr = None
    if prior is not None:
        pr = (ctypes.c_double * n_par)(*[float(x) for x in np.broadcast_to(prior, (n_par,))])
    _check(load_library().gw_covariance(ctx, _ptr(fisher), n, n_par, mask, pr, int(method),
                                        float(thresh), float(cond_max), _ptr(cov), _ptr(cond),
                                        _ptr(err), _ptr(status), _stream(stream)), ctx)
    return cov, cond, err, status


def gw_packed_submatrix(mat: torch.Tensor, n_par: int, keep, stream=None) -> torch.Tensor:
    """Kept rows and columns of packed matrices (fix on Fisher, marginalise on C)."""
    ctx = context()
    n = mat.shape[1]
    mask, k = _keep_mask(keep, n_par)
    out = torch.empty((k * (k + 1) // 2, n), dtype=torch.float64, device=mat.device)
    _check(load_library().gw_packed_submatrix(ctx, _ptr(mat), n, n_par, mask, _ptr(out),
                                              _stream(stream)), ctx)
    return out


def gw_sky_area(cov: torch.Tensor, n_par: int, theta: torch.Tensor, i_theta=3, i_phi=4,
                perc=90.0, units="SqDeg", stream=None) -> torch.Tensor:
    """Delta Omega_perc% per event (Sec. 4.1), 'SqDeg' or 'Sterad'."""
    ctx = context()
    n = cov.shape[1]
    area = torch.empty(n, dtype=torch.float64, device=cov.device)
    _check(load_library().gw_sky_area(ctx, _ptr(cov), n, n_par, int(i_theta), int(i_phi),
                                      _ptr(theta.contiguous()), float(perc),
                                      1 if units == "SqDeg" else 0, _ptr(area), _stream(stream)), ctx)
    return area


def gw_strain(cat: Catalog, net: Network, prec=GW_FP64, stream=None):
    """Strain of every arm on every event's grid: returns (re, im [n_arm, total],
    freq [total], point_off [n + 1], status [n])."""
    ctx = context()
    dev = cat.npts.device
    npts = cat.npts if cat.sel is None else cat.npts[cat.sel]
    total = int(npts.clamp(min=0).to(torch.int64).sum().item())
    n_arm = sum(1 if int(r[4]) == 0 else 3 for r in net.det_rows)
    re = torch.empty((n_arm, total), dtype=torch.float64, device=dev)
    im = torch.empty((n_arm, total), dtype=torch.float64, device=dev)
    freq = torch.empty(total, dtype=torch.float64, device=dev)
    off = torch.empty(cat.n + 1, dtype=torch.int64, device=dev)
    status = torch.empty(cat.n, dtype=torch.int32, device=dev)
    c = cat.struct()
    _check(load_library().gw_strain(ctx, ctypes.byref(c), ctypes.byref(net.net), int(prec), total,
                                    _ptr(re), _ptr(im), _ptr(freq), _ptr(off), _ptr(status),
                                    _stream(stream)), ctx)
    return re, im, freq, off, status


def gw_perturb_fisher(fisher: torch.Tensor, n_par: int, r: torch.Tensor, eps=1e-10,
                      stream=None) -> torch.Tensor:
    """perturb_Fisher (Sec. 4.1): fisher * (1 + eps r) on the packed triangle."""
    ctx = context()
    out = torch.empty_like(fisher)
    _check(load_library().gw_perturb_fisher(ctx, _ptr(fisher), fisher.shape[1], n_par, float(eps),
                                            _ptr(r.contiguous()), _ptr(out), _stream(stream)), ctx)
    return out

