"""Thin ctypes binding of libtpcf (include/tpcf.h), same names as the C ABI.

Argument marshalling only: every step of the estimator runs in the library's
CUDA kernels.  PyTorch supplies device memory (tensor.data_ptr()) and streams.
Importing this module does not need a GPU; calling into the library does, and
a missing library raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtpcf.so")

TPCF_OK = 0
STATUS = {0: "TPCF_OK", -1: "TPCF_ERR_ARG", -2: "TPCF_ERR_OOM", -3: "TPCF_ERR_CUDA",
          -4: "TPCF_ERR_TIMEOUT", -5: "TPCF_ERR_UNSUPPORTED", -6: "TPCF_ERR_DATA"}
PREC = {"fp32": 0, "bf16x3": 1, "tf32x3": 2}
LOS = {"z": 0, "observer": 1}
CONV = {"S_COEFF": 0, "PAPER_EQ": 1}

# Names of every entry point include/tpcf.h declares (checked by the tests).
EXPORTS = ["tpcf_last_error", "tpcf_version", "tpcf_set_wait_limit", "tpcf_kernel_launches", "tpcf_quantize_host", "tpcf_multipole_count", "tpcf_multipole_index",
           "tpcf_bin_edges", "tpcf_build_grid", "tpcf_grid_destroy", "tpcf_grid_info", "tpcf_grid_points",
           "tpcf_accumulate_alm", "tpcf_pair_counts", "tpcf_partial_sizes", "tpcf_estimate_3pcf_partial",
           "tpcf_estimate_3pcf_finish", "tpcf_couple_multipoles", "tpcf_project", "tpcf_estimate_3pcf",
           "tpcf_estimate_3pcf_xi", "tpcf_estimate_3pcf_full_edge",
           "tpcf_estimate_3pcf_host", "tpcf_stream_status", "tpcf_trim_memory", "tpcf_couple_multipoles_static",
           "tpcf_batch_create", "tpcf_batch_info", "tpcf_batch_run", "tpcf_batch_run_graph", "tpcf_batch_destroy",
           "tpcf_batch_status",
           "tpcf_estimate_3pcf_batched", "tpcf_autotune",
           "tpcf_covariance", "tpcf_covariance_factors", "tpcf_data_vector_index", "tpcf_check_rsqrt", "tpcf_measure_fp32_peak",
           "tpcf_emu_create", "tpcf_emu_destroy", "tpcf_emu_param_count", "tpcf_emu_set_input_box",
           "tpcf_emu_fit_output_scaling", "tpcf_emu_train_step", "tpcf_emu_gradients", "tpcf_emu_predict",
           "tpcf_emu_get_params", "tpcf_emu_set_params", "tpcf_emu_get_output_scaling",
           "tpcf_emu_set_output_scaling", "tpcf_emu_get_input_box", "tpcf_emu_get_optimizer",
           "tpcf_emu_set_optimizer"]


class TpcfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class tpcf_config(ctypes.Structure):
    _fields_ = [("r_min", ctypes.c_double), ("r_max", ctypes.c_double),
                ("n_bins", ctypes.c_int32), ("l_max", ctypes.c_int32),
                ("n_L", ctypes.c_int32), ("L", ctypes.c_int32 * 8),
                ("periodic", ctypes.c_int32), ("box", ctypes.c_double),
                ("precision", ctypes.c_int32), ("remove_self", ctypes.c_int32),
                ("convention", ctypes.c_int32), ("cell_div", ctypes.c_int32),
                ("tile_primaries", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("los", ctypes.c_int32), ("observer", ctypes.c_double * 3)]


@dataclass
class Config:
    """Estimator configuration (mirrors tpcf_config)."""
    r_min: float
    r_max: float
    n_bins: int
    l_max: int
    Ls: tuple = (0, 2, 4)
    periodic: bool = True
    box: float = 500.0
    precision: str = "fp32"
    remove_self: bool = True
    convention: str = "S_COEFF"
    cell_div: int = 0
    tile_primaries: int = 0
    chunk: int = 0
    los: str = "z"                      # "z" (fixed) or "observer" (observer to each primary)
    observer: tuple = (0.0, 0.0, 0.0)   # observer position (box coordinates) for los="observer"

    def c(self) -> tpcf_config:
        arr = (ctypes.c_int32 * 8)(*(list(self.Ls) + [0] * (8 - len(self.Ls))))
        obs = (ctypes.c_double * 3)(*[float(v) for v in self.observer])
        return tpcf_config(self.r_min, self.r_max, self.n_bins, self.l_max, len(self.Ls), arr,
                           int(self.periodic), self.box, PREC[self.precision], int(self.remove_self),
                           CONV[self.convention], self.cell_div, self.tile_primaries, self.chunk,
                           LOS[self.los], obs)


_lib = None
P = ctypes.c_void_p
I64 = ctypes.c_int64
CFG = ctypes.POINTER(tpcf_config)


def lib():
    """Loads libtpcf.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtpcf.so is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "tpcf_last_error": ([], ctypes.c_char_p),
            "tpcf_version": ([], ctypes.c_int),
            "tpcf_set_wait_limit": ([I64, ctypes.c_int32], ctypes.c_int),
            "tpcf_kernel_launches": ([], ctypes.c_int64),
            "tpcf_multipole_count": ([CFG, P], ctypes.c_int),
            "tpcf_multipole_index": ([CFG, P, ctypes.c_int32], ctypes.c_int),
            "tpcf_bin_edges": ([CFG, P], ctypes.c_int),
            "tpcf_build_grid": ([P, P, I64, CFG, P, P], ctypes.c_int),
            "tpcf_grid_destroy": ([P], ctypes.c_int),
            "tpcf_grid_info": ([P, P, P], ctypes.c_int),
            "tpcf_grid_points": ([P, P, P, P, P], ctypes.c_int),
            "tpcf_accumulate_alm": ([P, P, P, I64, CFG, ctypes.c_double, P, P, P, P, P, P], ctypes.c_int),
            "tpcf_pair_counts": ([P, P, I64, CFG, P, P, P], ctypes.c_int),
            "tpcf_partial_sizes": ([CFG, P, P], ctypes.c_int),
            "tpcf_estimate_3pcf_partial": ([CFG, P, P, I64, P, P, I64, P, P, I64, P, P, I64, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int32, P, P, P], ctypes.c_int),
            "tpcf_estimate_3pcf_finish": ([CFG, ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                           P, P, P, P, P, P, P, P, P], ctypes.c_int),
            "tpcf_couple_multipoles": ([P, P, P, I64, CFG, P, P, P, P, P], ctypes.c_int),
            "tpcf_project": ([CFG, P, P, P, P], ctypes.c_int),
            "tpcf_estimate_3pcf": ([CFG, P, P, I64, P, P, I64, P, P, P, P, P, P], ctypes.c_int),
            "tpcf_estimate_3pcf_xi": ([CFG, P, P, I64, P, P, I64, P, P, P, P, P, P, P], ctypes.c_int),
            "tpcf_estimate_3pcf_full_edge": ([CFG, P, P, I64, P, P, I64, P, P, P, P, P], ctypes.c_int),
            "tpcf_estimate_3pcf_host": ([CFG, P, P, I64, P, P, I64, P, P, P, P, P, P], ctypes.c_int),
            "tpcf_stream_status": ([P], ctypes.c_int),
            "tpcf_trim_memory": ([], ctypes.c_int),
            "tpcf_couple_multipoles_static": ([P, P, P, I64, CFG, P, P, P, P, P], ctypes.c_int),
            "tpcf_batch_create": ([CFG, P, ctypes.c_int32, I64, P], ctypes.c_int),
            "tpcf_batch_info": ([P, P, P], ctypes.c_int),
            "tpcf_batch_run": ([P, P, P, P, P, P], ctypes.c_int),
            "tpcf_batch_run_graph": ([P, P, P, P, P, P], ctypes.c_int),
            "tpcf_batch_destroy": ([P], ctypes.c_int),
            "tpcf_estimate_3pcf_batched": ([CFG, P, P, P, ctypes.c_int32, P, P, P, P], ctypes.c_int),
            "tpcf_batch_status": ([P, P, P], ctypes.c_int),
            "tpcf_autotune": ([CFG, P, P, I64, P, CFG], ctypes.c_int),
            "tpcf_covariance": ([P, I64, I64, P, I64, P, P, P], ctypes.c_int),
            "tpcf_check_rsqrt": ([I64, ctypes.c_uint64, P, P], ctypes.c_int),
            "tpcf_measure_fp32_peak": ([P, P], ctypes.c_int),
            "tpcf_covariance_factors": ([I64, I64, I64, P, P], ctypes.c_int),
            "tpcf_data_vector_index": ([CFG, P, ctypes.c_int32, ctypes.c_int32, P, I64, P], ctypes.c_int),
            "tpcf_emu_create": ([P, ctypes.c_int32, ctypes.c_uint64, P], ctypes.c_int),
            "tpcf_emu_destroy": ([P], ctypes.c_int),
            "tpcf_emu_param_count": ([P, P], ctypes.c_int),
            "tpcf_emu_set_input_box": ([P, P, P], ctypes.c_int),
            "tpcf_emu_fit_output_scaling": ([P, P, I64, P], ctypes.c_int),
            "tpcf_emu_train_step": ([P, P, P, I64, ctypes.c_float, P, P], ctypes.c_int),
            "tpcf_emu_gradients": ([P, P, P, I64, P, P, P], ctypes.c_int),
            "tpcf_emu_predict": ([P, P, I64, P, P], ctypes.c_int),
            "tpcf_emu_get_params": ([P, P, P], ctypes.c_int),
            "tpcf_emu_set_params": ([P, P, P], ctypes.c_int),
            "tpcf_emu_get_output_scaling": ([P, P, P], ctypes.c_int),
            "tpcf_quantize_host": ([P, I64, ctypes.c_double, P], ctypes.c_int),
            "tpcf_emu_set_output_scaling": ([P, P, P], ctypes.c_int),
            "tpcf_emu_get_input_box": ([P, P, P], ctypes.c_int),
            "tpcf_emu_get_optimizer": ([P, P, P, P, P], ctypes.c_int),
            "tpcf_emu_set_optimizer": ([P, P, P, I64, P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int):
    if rc != TPCF_OK:
        raise TpcfError(rc, lib().tpcf_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensors passed to libtpcf must be contiguous")
        return t.data_ptr()
    return t.ctypes.data  # numpy (host) array


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def multipole_index(cfg: Config):
    c = cfg.c()
    n = ctypes.c_int32(0)
    _check(lib().tpcf_multipole_count(ctypes.byref(c), ctypes.addressof(n)))
    arr = (ctypes.c_int32 * (3 * n.value))()
    _check(lib().tpcf_multipole_index(ctypes.byref(c), ctypes.addressof(arr), n.value))
    return [tuple(arr[3 * k:3 * k + 3]) for k in range(n.value)]


def data_vector_index(cfg: Config, selected, eta: int):
    """tpcf_data_vector_index: flat indices (numpy int64) into a [n_mult][nb][nb] zeta
    array for the selected (l1, l2, L) multipoles over triangles b2 - b1 >= eta."""
    import numpy as np
    c = cfg.c()
    sel = np.ascontiguousarray(np.asarray(selected, dtype=np.int32).reshape(-1, 3))
    n = ctypes.c_int64(0)
    _check(lib().tpcf_data_vector_index(ctypes.byref(c), _ptr(sel), sel.shape[0], int(eta), None, 0,
                                        ctypes.addressof(n)))
    idx = np.empty(n.value, dtype=np.int64)
    _check(lib().tpcf_data_vector_index(ctypes.byref(c), _ptr(sel), sel.shape[0], int(eta), _ptr(idx), idx.size,
                                        ctypes.addressof(n)))
    return idx


def covariance(src, idx=None, n_dv=None, stream=None):
    """tpcf_covariance over the leading (mock) axis of the device tensor src
    (FP64, contiguous); idx (int64, host or device) selects entries of each
    mock's flattened row.  Returns (mean [n_dv], cov [n_dv, n_dv])."""
    if src.dtype != torch.float64 or not src.is_contiguous():
        raise ValueError("src must be a contiguous float64 tensor")
    n_mocks = src.shape[0]
    stride = src[0].numel()
    di = None
    if idx is not None:
        di = torch.as_tensor(idx, dtype=torch.int64).to(src.device).contiguous()
        n_dv = di.numel()
    elif n_dv is None:
        n_dv = stride
    mean = torch.empty(n_dv, dtype=torch.float64, device=src.device)
    cov = torch.empty((n_dv, n_dv), dtype=torch.float64, device=src.device)
    _check(lib().tpcf_covariance(_ptr(src), n_mocks, stride, _ptr(di), n_dv, _ptr(mean), _ptr(cov),
                                 _stream(stream)))
    return mean, cov


def check_rsqrt(n: int, seed: int = 1, stream=None) -> dict:
    """tpcf_check_rsqrt: the pair stage's reciprocal square root against __frsqrt_rn."""
    st = (ctypes.c_double * 5)()
    _check(lib().tpcf_check_rsqrt(n, seed, ctypes.addressof(st), _stream(stream)))
    return {"max_ulp": st[0], "mean_rel_diff": st[1], "mean_norm_err": st[2], "mean_norm_err_rn": st[3],
            "frac_differ": st[4]}


def covariance_factors(n_mocks: int, n_dv: int, n_params: int):
    """tpcf_covariance_factors: (Hartlap factor, Percival m1)."""
    h, m = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().tpcf_covariance_factors(n_mocks, n_dv, n_params, ctypes.addressof(h), ctypes.addressof(m)))
    return h.value, m.value


def bin_edges(cfg: Config):
    c = cfg.c()
    arr = (ctypes.c_uint64 * (cfg.n_bins + 1))()
    _check(lib().tpcf_bin_edges(ctypes.byref(c), ctypes.addressof(arr)))
    return [int(v) for v in arr]


def _as_dev_xyz(xyz, device):
    """uint32 numpy [n,3] or int32 tensor [n,3] -> contiguous int32 device tensor."""
    if isinstance(xyz, torch.Tensor):
        return xyz.to(device=device, dtype=torch.int32).contiguous()
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.uint32).view(np.int32)).to(device)


def _as_dev_w(w, device):
    if w is None:
        return None
    if isinstance(w, torch.Tensor):
        return w.to(device=device, dtype=torch.float32).contiguous()
    return torch.as_tensor(w, dtype=torch.float32).to(device).contiguous()


@dataclass
class Result:
    zeta: torch.Tensor
    mults: list
    nnn: torch.Tensor | None = None
    rrr: torch.Tensor | None = None
    pair_counts: torch.Tensor | None = None
    triplet_counts: torch.Tensor | None = None
    xi: torch.Tensor | None = None      # even 2PCF multipoles [l_max // 2 + 1, n_bins]
    extra: dict = field(default_factory=dict)


def estimate_3pcf(cfg: Config, d_xyz, d_w=None, r_xyz=None, r_w=None, stream=None, want_all=True,
                  device="cuda", want_xi=False) -> Result:
    """tpcf_estimate_3pcf on device tensors (numpy inputs are copied to the device first);
    with want_xi, tpcf_estimate_3pcf_xi, which adds the even 2PCF multipoles."""
    dx = _as_dev_xyz(d_xyz, device)
    dw = _as_dev_w(d_w, device)
    rx = _as_dev_xyz(r_xyz, device) if r_xyz is not None else None
    rw = _as_dev_w(r_w, device) if r_xyz is not None else None
    nd = dx.shape[0]
    nr = rx.shape[0] if rx is not None else 0
    mults = multipole_index(cfg)
    nb, L1 = cfg.n_bins, cfg.l_max + 1
    z = torch.empty((len(mults), nb, nb), dtype=torch.float64, device=device)
    nnn = rrr = pc = tc = None
    if want_all:
        nnn = torch.empty((L1, L1, L1, nb, nb), dtype=torch.float64, device=device)
        rrr = torch.empty((nb, nb), dtype=torch.float64, device=device)
        pc = torch.empty(nb, dtype=torch.int64, device=device)
        tc = torch.empty((nb, nb), dtype=torch.int64, device=device)
    c = cfg.c()
    if want_xi:
        xi = torch.empty((cfg.l_max // 2 + 1, nb), dtype=torch.float64, device=device)
        _check(lib().tpcf_estimate_3pcf_xi(ctypes.byref(c), _ptr(dx), _ptr(dw), nd, _ptr(rx), _ptr(rw), nr,
                                           _ptr(z), _ptr(nnn), _ptr(rrr), _ptr(pc), _ptr(tc), _ptr(xi),
                                           _stream(stream)))
        return Result(z, mults, nnn, rrr, pc, tc, xi)
    _check(lib().tpcf_estimate_3pcf(ctypes.byref(c), _ptr(dx), _ptr(dw), nd, _ptr(rx), _ptr(rw), nr,
                                    _ptr(z), _ptr(nnn), _ptr(rrr), _ptr(pc), _ptr(tc), _stream(stream)))
    return Result(z, mults, nnn, rrr, pc, tc)


def estimate_3pcf_full_edge(cfg: Config, d_xyz, d_w, r_xyz, r_w=None, stream=None, device="cuda",
                            want_xi=False) -> Result:
    """tpcf_estimate_3pcf_full_edge on device tensors: zeta with the full anisotropic
    edge correction; Result.rrr holds RRR^m_{l1 l2} [L1, L1, L1, nb, nb]."""
    dx = _as_dev_xyz(d_xyz, device)
    dw = _as_dev_w(d_w, device)
    rx = _as_dev_xyz(r_xyz, device)
    rw = _as_dev_w(r_w, device)
    mults = multipole_index(cfg)
    nb, L1 = cfg.n_bins, cfg.l_max + 1
    z = torch.empty((len(mults), nb, nb), dtype=torch.float64, device=device)
    nnn = torch.empty((L1, L1, L1, nb, nb), dtype=torch.float64, device=device)
    rrr = torch.empty((L1, L1, L1, nb, nb), dtype=torch.float64, device=device)
    xi = torch.empty((cfg.l_max // 2 + 1, nb), dtype=torch.float64, device=device) if want_xi else None
    c = cfg.c()
    _check(lib().tpcf_estimate_3pcf_full_edge(ctypes.byref(c), _ptr(dx), _ptr(dw), dx.shape[0], _ptr(rx), _ptr(rw),
                                              rx.shape[0], _ptr(z), _ptr(nnn), _ptr(rrr), _ptr(xi),
                                              _stream(stream)))
    return Result(z, mults, nnn, rrr, xi=xi)


def estimate_3pcf_host(cfg: Config, d_xyz, d_w=None, r_xyz=None, r_w=None, stream=None):
    """tpcf_estimate_3pcf_host: host (numpy, ideally pinned) buffers in and out."""
    import numpy as np
    mults = multipole_index(cfg)
    nb, L1 = cfg.n_bins, cfg.l_max + 1
    dx = np.ascontiguousarray(d_xyz, dtype=np.uint32)
    dw = None if d_w is None else np.ascontiguousarray(d_w, dtype=np.float32)
    rx = None if r_xyz is None else np.ascontiguousarray(r_xyz, dtype=np.uint32)
    rw = None if r_w is None else np.ascontiguousarray(r_w, dtype=np.float32)
    z = np.empty((len(mults), nb, nb))
    nnn = np.empty((L1, L1, L1, nb, nb))
    rrr = np.empty((nb, nb))
    pc = np.empty(nb, dtype=np.int64)
    tc = np.empty((nb, nb), dtype=np.int64)
    c = cfg.c()
    _check(lib().tpcf_estimate_3pcf_host(ctypes.byref(c), _ptr(dx), _ptr(dw), dx.shape[0], _ptr(rx), _ptr(rw),
                                         0 if rx is None else rx.shape[0], _ptr(z), _ptr(nnn), _ptr(rrr),
                                         _ptr(pc), _ptr(tc), _stream(stream)))
    return Result(z, mults, nnn, rrr, pc, tc)


class Grid:
    """tpcf_build_grid / tpcf_grid_destroy."""

    def __init__(self, cfg: Config, xyz, w=None, stream=None, device="cuda"):
        self.cfg = cfg
        self.xyz = _as_dev_xyz(xyz, device)
        self.w = _as_dev_w(w, device)
        self.handle = ctypes.c_void_p()
        c = cfg.c()
        _check(lib().tpcf_build_grid(_ptr(self.xyz), _ptr(self.w), self.xyz.shape[0], ctypes.byref(c),
                                     ctypes.addressof(self.handle), _stream(stream)))

    def info(self):
        n = ctypes.c_int64(0)
        nc = ctypes.c_int32(0)
        _check(lib().tpcf_grid_info(self.handle, ctypes.addressof(n), ctypes.addressof(nc)))
        return n.value, nc.value

    def points(self, stream=None):
        n, _ = self.info()
        dev = self.xyz.device
        xyz = torch.empty((n, 3), dtype=torch.int32, device=dev)
        w = torch.empty(n, dtype=torch.float32, device=dev)
        order = torch.empty(n, dtype=torch.int64, device=dev)
        _check(lib().tpcf_grid_points(self.handle, _ptr(xyz), _ptr(w), _ptr(order), _stream(stream)))
        return xyz, w, order

    def close(self):
        if self.handle:
            _check(lib().tpcf_grid_destroy(self.handle))
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def accumulate_alm(grid: Grid, cfg: Config, prim_xyz=None, prim_w=None, monopole_weight=-1.0, stream=None):
    """tpcf_accumulate_alm; returns (alm, counts, diag, wsp, pair_counts) device tensors."""
    dev = grid.xyz.device
    if prim_xyz is None:
        n = grid.info()[0]
        px = pw = None
    else:
        px = _as_dev_xyz(prim_xyz, dev)
        pw = _as_dev_w(prim_w, dev)
        n = px.shape[0]
    nb, L1 = cfg.n_bins, cfg.l_max + 1
    alm = torch.empty((n, nb, L1 * L1), dtype=torch.float32, device=dev)
    counts = torch.empty((n, nb), dtype=torch.int32, device=dev)
    diag = torch.zeros((L1 * (L1 + 1) // 2, nb), dtype=torch.float64, device=dev)
    wsp = torch.zeros((L1, nb), dtype=torch.float64, device=dev)
    pc = torch.zeros(nb, dtype=torch.int64, device=dev)
    c = cfg.c()
    _check(lib().tpcf_accumulate_alm(grid.handle, _ptr(px), _ptr(pw), n, ctypes.byref(c), float(monopole_weight),
                                     _ptr(alm), _ptr(counts), _ptr(diag), _ptr(wsp), _ptr(pc), _stream(stream)))
    return alm, counts, diag, wsp, pc


def pair_counts(grid: Grid, cfg: Config, prim_xyz=None, stream=None):
    """tpcf_pair_counts; returns (counts [n_prim][n_bins] int32, pair_counts [n_bins] int64)."""
    dev = grid.xyz.device
    if prim_xyz is None:
        n = grid.info()[0]
        px = None
    else:
        px = _as_dev_xyz(prim_xyz, dev)
        n = px.shape[0]
    counts = torch.empty((n, cfg.n_bins), dtype=torch.int32, device=dev)
    pc = torch.zeros(cfg.n_bins, dtype=torch.int64, device=dev)
    c = cfg.c()
    _check(lib().tpcf_pair_counts(grid.handle, _ptr(px), n, ctypes.byref(c), _ptr(counts), _ptr(pc), _stream(stream)))
    return counts, pc


def partial_sizes(cfg: Config):
    """tpcf_partial_sizes: (doubles, int64 counts) of one shard's partial results."""
    nf, ni = ctypes.c_int64(), ctypes.c_int64()
    c = cfg.c()
    _check(lib().tpcf_partial_sizes(ctypes.byref(c), ctypes.byref(nf), ctypes.byref(ni)))
    return nf.value, ni.value


def estimate_3pcf_partial(cfg: Config, d_xyz, d_w, r_xyz, r_w, dp_xyz, dp_w, rp_xyz, rp_w, w_d_total: float,
                          w_r_total: float, weighted_randoms: bool, stream=None, device="cuda"):
    """tpcf_estimate_3pcf_partial: one shard's additive partials (part_f FP64, part_i int64)
    as device tensors.  r_xyz / rp_xyz None: periodic analytic randoms."""
    def dx(a):
        return None if a is None else _as_dev_xyz(a, device)

    def dw(a):
        return None if a is None else _as_dev_w(a, device)
    d, dwt, r, rwt = dx(d_xyz), dw(d_w), dx(r_xyz), dw(r_w)
    dp, dpw, rp, rpw = dx(dp_xyz), dw(dp_w), dx(rp_xyz), dw(rp_w)
    nf, ni = partial_sizes(cfg)
    pf = torch.empty(nf, dtype=torch.float64, device=device)
    pi = torch.empty(ni, dtype=torch.int64, device=device)
    n = lambda a: 0 if a is None else a.shape[0]
    c = cfg.c()
    _check(lib().tpcf_estimate_3pcf_partial(ctypes.byref(c), _ptr(d), _ptr(dwt), n(d), _ptr(r), _ptr(rwt), n(r),
                                            _ptr(dp), _ptr(dpw), n(dp), _ptr(rp), _ptr(rpw), n(rp),
                                            float(w_d_total), float(w_r_total), int(bool(weighted_randoms)),
                                            _ptr(pf), _ptr(pi), _stream(stream)))
    return pf, pi


def estimate_3pcf_finish(cfg: Config, part_f, part_i, w_d_total: float, w_r_total: float, explicit_randoms: bool,
                         weighted_randoms: bool, want_xi=False, stream=None):
    """tpcf_estimate_3pcf_finish: the estimate (a Result) from the summed partials."""
    dev = part_f.device
    nb, L1 = cfg.n_bins, cfg.l_max + 1
    mults = multipole_index(cfg)
    zeta = torch.empty((len(mults), nb, nb), dtype=torch.float64, device=dev)
    nnn = torch.empty((L1, L1, L1, nb, nb), dtype=torch.float64, device=dev)
    rrr = torch.empty((nb, nb), dtype=torch.float64, device=dev)
    pc = torch.empty(nb, dtype=torch.int64, device=dev)
    tc = torch.empty((nb, nb), dtype=torch.int64, device=dev)
    xi = torch.empty((cfg.l_max // 2 + 1, nb), dtype=torch.float64, device=dev) if want_xi else None
    c = cfg.c()
    _check(lib().tpcf_estimate_3pcf_finish(ctypes.byref(c), float(w_d_total), float(w_r_total),
                                           int(bool(explicit_randoms)), int(bool(weighted_randoms)), _ptr(part_f),
                                           _ptr(part_i), _ptr(zeta), _ptr(nnn), _ptr(rrr), _ptr(pc), _ptr(tc),
                                           _ptr(xi), _stream(stream)))
    return Result(zeta, mults, nnn, rrr, pc, tc, xi)


def couple_multipoles(cfg: Config, alm, prim_w, counts, diag, wsp, stream=None):
    """tpcf_couple_multipoles; returns (nnn, triplet_counts)."""
    dev = alm.device
    nb, L1 = cfg.n_bins, cfg.l_max + 1
    nnn = torch.empty((L1, L1, L1, nb, nb), dtype=torch.float64, device=dev)
    tc = torch.empty((nb, nb), dtype=torch.int64, device=dev) if counts is not None else None
    c = cfg.c()
    _check(lib().tpcf_couple_multipoles(_ptr(alm), _ptr(prim_w), _ptr(counts), alm.shape[0], ctypes.byref(c),
                                        _ptr(diag), _ptr(wsp), _ptr(nnn), _ptr(tc), _stream(stream)))
    return nnn, tc


def couple_multipoles_static(cfg: Config, alm, prim_w, counts, diag, wsp, stream=None):
    """tpcf_couple_multipoles_static: the coupling step with no device allocation
    (fixed library scratch; see include/tpcf.h for the size limit and sharing rules)."""
    dev = alm.device
    nb, L1 = cfg.n_bins, cfg.l_max + 1
    nnn = torch.empty((L1, L1, L1, nb, nb), dtype=torch.float64, device=dev)
    tc = torch.empty((nb, nb), dtype=torch.int64, device=dev) if counts is not None else None
    c = cfg.c()
    _check(lib().tpcf_couple_multipoles_static(_ptr(alm), _ptr(prim_w), _ptr(counts), alm.shape[0],
                                               ctypes.byref(c), _ptr(diag), _ptr(wsp), _ptr(nnn), _ptr(tc),
                                               _stream(stream)))
    return nnn, tc


def project(cfg: Config, nnn, rrr, stream=None):
    mults = multipole_index(cfg)
    z = torch.empty((len(mults), cfg.n_bins, cfg.n_bins), dtype=torch.float64, device=nnn.device)
    c = cfg.c()
    _check(lib().tpcf_project(ctypes.byref(c), _ptr(nnn), _ptr(rrr), _ptr(z), _stream(stream)))
    return z


class Batch:
    """tpcf_batch_create / run / destroy: many periodic catalogues of uneven sizes,
    concatenated; mock k is rows offsets[k]:offsets[k+1] of the point arrays."""

    def __init__(self, cfg: Config, offsets, group_points: int = 0):
        import numpy as np
        self.cfg = cfg
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.n_mocks = len(self.offsets) - 1
        self.mults = multipole_index(cfg)
        self.handle = ctypes.c_void_p()
        c = cfg.c()
        _check(lib().tpcf_batch_create(ctypes.byref(c), _ptr(self.offsets), self.n_mocks, int(group_points),
                                       ctypes.addressof(self.handle)))

    def info(self):
        ng = ctypes.c_int32(0)
        nc = ctypes.c_int32(0)
        _check(lib().tpcf_batch_info(self.handle, ctypes.addressof(ng), ctypes.addressof(nc)))
        return ng.value, nc.value

    def zeta_buffer(self, device="cuda"):
        nb = self.cfg.n_bins
        return torch.empty((self.n_mocks, len(self.mults), nb, nb), dtype=torch.float64, device=device)

    def run(self, xyz, w, zeta, triplet_counts=None, stream=None):
        """Enqueues the whole batch on the stream (no host synchronisation)."""
        _check(lib().tpcf_batch_run(self.handle, _ptr(xyz), _ptr(w), _ptr(zeta), _ptr(triplet_counts),
                                    _stream(stream)))

    def run_graph(self, xyz, w, zeta, triplet_counts=None, stream=None):
        """tpcf_batch_run_graph: eager run + capture on first use of these buffers,
        one graph launch afterwards."""
        _check(lib().tpcf_batch_run_graph(self.handle, _ptr(xyz), _ptr(w), _ptr(zeta), _ptr(triplet_counts),
                                          _stream(stream)))

    def status(self, stream=None):
        """tpcf_batch_status: per-mock status codes of the last run (int32 numpy array)."""
        import numpy as np
        st = np.zeros(self.n_mocks, dtype=np.int32)
        _check(lib().tpcf_batch_status(self.handle, _ptr(st), _stream(stream)))
        return st

    def close(self):
        if self.handle:
            _check(lib().tpcf_batch_destroy(self.handle))
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate_3pcf_batched(cfg: Config, xyz, w, offsets, stream=None, device="cuda", want_counts=True,
                          want_status=False):
    """tpcf_estimate_3pcf_batched; returns (zeta [n_mocks, n_mult, nb, nb], triplet counts or None),
    and with want_status also the per-mock status codes (int32 numpy array)."""
    import numpy as np
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    dx = _as_dev_xyz(xyz, device)
    dw = _as_dev_w(w, device)
    nm = len(off) - 1
    nb = cfg.n_bins
    z = torch.empty((nm, len(multipole_index(cfg)), nb, nb), dtype=torch.float64, device=device)
    tc = torch.empty((nm, nb, nb), dtype=torch.int64, device=device) if want_counts else None
    st = np.zeros(nm, dtype=np.int32)
    c = cfg.c()
    _check(lib().tpcf_estimate_3pcf_batched(ctypes.byref(c), _ptr(dx), _ptr(dw), _ptr(off), nm, _ptr(z),
                                            _ptr(tc), _ptr(st), _stream(stream)))
    return (z, tc, st) if want_status else (z, tc)


def autotune(cfg: Config, xyz, w=None, stream=None, device="cuda") -> Config:
    """tpcf_autotune: the fastest (cell_div, tile_primaries, chunk) for catalogues like this one."""
    import dataclasses
    dx = _as_dev_xyz(xyz, device)
    dw = _as_dev_w(w, device)
    c = cfg.c()
    out = tpcf_config()
    _check(lib().tpcf_autotune(ctypes.byref(c), _ptr(dx), _ptr(dw), dx.shape[0], _stream(stream),
                               ctypes.byref(out)))
    return dataclasses.replace(cfg, cell_div=out.cell_div, tile_primaries=out.tile_primaries, chunk=out.chunk)


class Emulator:
    """tpcf_emu_*: the MLP emulator of the tree-level 3PCF multipoles
    (BF16 weights, FP32 accumulation, own forward / backward / Adam kernels)."""

    def __init__(self, widths, seed=0, device="cuda"):
        import numpy as np
        self.widths = [int(w) for w in widths]
        self.device = device
        arr = np.ascontiguousarray(self.widths, dtype=np.int32)
        self.handle = ctypes.c_void_p()
        _check(lib().tpcf_emu_create(_ptr(arr), len(self.widths) - 1, ctypes.c_uint64(seed),
                                     ctypes.addressof(self.handle)))
        n = ctypes.c_int64(0)
        _check(lib().tpcf_emu_param_count(self.handle, ctypes.addressof(n)))
        self.n_params = n.value
        self.loss_buf = torch.zeros(1, dtype=torch.float64, device=device)

    def set_input_box(self, lo, hi):
        import numpy as np
        lo = np.ascontiguousarray(lo, dtype=np.float32)
        hi = np.ascontiguousarray(hi, dtype=np.float32)
        _check(lib().tpcf_emu_set_input_box(self.handle, _ptr(lo), _ptr(hi)))

    def fit_output_scaling(self, y, stream=None):
        _check(lib().tpcf_emu_fit_output_scaling(self.handle, _ptr(y), y.shape[0], _stream(stream)))

    def output_scaling(self):
        import numpy as np
        mu = np.empty(self.widths[-1], dtype=np.float32)
        sd = np.empty(self.widths[-1], dtype=np.float32)
        _check(lib().tpcf_emu_get_output_scaling(self.handle, _ptr(mu), _ptr(sd)))
        return mu, sd

    def train_step(self, x, y, lr, loss=None, stream=None):
        """One Adam step; the batch loss (before the update) goes to `loss` (a
        one-element float64 device tensor) when given."""
        _check(lib().tpcf_emu_train_step(self.handle, _ptr(x), _ptr(y), x.shape[0], ctypes.c_float(lr),
                                         _ptr(loss), _stream(stream)))

    def gradients(self, x, y, stream=None):
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        _check(lib().tpcf_emu_gradients(self.handle, _ptr(x), _ptr(y), x.shape[0], _ptr(g), _ptr(self.loss_buf),
                                        _stream(stream)))
        return g, self.loss_buf

    def predict(self, x, out=None, stream=None):
        if out is None:
            out = torch.empty((x.shape[0], self.widths[-1]), dtype=torch.float32, device=self.device)
        _check(lib().tpcf_emu_predict(self.handle, _ptr(x), x.shape[0], _ptr(out), _stream(stream)))
        return out

    def get_params(self, stream=None):
        p = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        _check(lib().tpcf_emu_get_params(self.handle, _ptr(p), _stream(stream)))
        return p

    def set_params(self, p, stream=None):
        _check(lib().tpcf_emu_set_params(self.handle, _ptr(p), _stream(stream)))

    def input_box(self):
        import numpy as np
        lo = np.empty(self.widths[0], dtype=np.float32)
        hi = np.empty(self.widths[0], dtype=np.float32)
        _check(lib().tpcf_emu_get_input_box(self.handle, _ptr(lo), _ptr(hi)))
        return lo, hi

    def set_output_scaling(self, mean, sd):
        import numpy as np
        mean = np.ascontiguousarray(mean, dtype=np.float32)
        sd = np.ascontiguousarray(sd, dtype=np.float32)
        _check(lib().tpcf_emu_set_output_scaling(self.handle, _ptr(mean), _ptr(sd)))

    def optimizer_state(self, stream=None):
        """(m, v, step): the Adam moments (device tensors) and the step count."""
        m = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        v = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        step = ctypes.c_int64(0)
        _check(lib().tpcf_emu_get_optimizer(self.handle, _ptr(m), _ptr(v), ctypes.addressof(step), _stream(stream)))
        return m, v, step.value

    def set_optimizer_state(self, m, v, step, stream=None):
        _check(lib().tpcf_emu_set_optimizer(self.handle, _ptr(m), _ptr(v), int(step), _stream(stream)))

    def save(self, path, stream=None):
        """Checkpoint (weights, Adam state and step, input box, output scaling) to
        `path` (.npz), written to a temporary file and renamed into place."""
        import os
        import numpy as np
        p = self.get_params(stream)
        m, v, step = self.optimizer_state(stream)
        torch.cuda.synchronize(self.device)
        lo, hi = self.input_box()
        mu, sd = self.output_scaling()
        tmp = str(path) + ".tmp.npz"
        np.savez(tmp, widths=np.asarray(self.widths, dtype=np.int64), params=p.cpu().numpy(), m=m.cpu().numpy(),
                 v=v.cpu().numpy(), step=np.int64(step), in_lo=lo, in_hi=hi, out_mean=mu, out_sd=sd)
        os.replace(tmp, path)

    @classmethod
    def load(cls, path, device="cuda", stream=None):
        """A new handle restored from a checkpoint written by save()."""
        import numpy as np
        with np.load(path) as f:
            emu = cls([int(x) for x in f["widths"]], seed=0, device=device)
            emu.set_input_box(f["in_lo"], f["in_hi"])
            emu.set_output_scaling(f["out_mean"], f["out_sd"])
            emu.set_params(torch.from_numpy(f["params"]).to(device), stream)
            emu.set_optimizer_state(torch.from_numpy(f["m"]).to(device), torch.from_numpy(f["v"]).to(device),
                                    int(f["step"]), stream)
            torch.cuda.synchronize(device)
        return emu

    def close(self):
        if self.handle:
            _check(lib().tpcf_emu_destroy(self.handle))
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def quantize_host(x, box: float):
    """tpcf_quantize_host: host float positions in [0, box) -> uint32 fixed point
    (floor(x / box * 2^32) in FP64), same shape."""
    import numpy as np
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = np.empty(a.shape, dtype=np.uint32)
    _check(lib().tpcf_quantize_host(a.ctypes.data_as(ctypes.c_void_p), a.size, ctypes.c_double(box),
                                    u.ctypes.data_as(ctypes.c_void_p)))
    return u


def measure_fp32_peak(stream=None):
    """tpcf_measure_fp32_peak: (scalar FMA, paired FFMA2) throughput in TFLOP/s."""
    out = (ctypes.c_double * 2)()
    _check(lib().tpcf_measure_fp32_peak(ctypes.addressof(out), _stream(stream)))
    return float(out[0]), float(out[1])


def kernel_launches() -> int:
    """Kernels launched by libtpcf in this process so far."""
    return int(lib().tpcf_kernel_launches())


def stream_status(stream=None):
    _check(lib().tpcf_stream_status(_stream(stream)))


def trim_memory():
    """tpcf_trim_memory: hands the library's cached device scratch of the current
    device back to the driver (blocks whose stream-ordered release has completed)."""
    _check(lib().tpcf_trim_memory())
