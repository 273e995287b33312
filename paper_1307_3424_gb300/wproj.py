"""Thin Python binding of libwproj (include/wproj.h).

Argument marshalling only: every step runs in the CUDA library.  PyTorch
supplies device memory (tensors passed by data pointer) and the stream
(torch.cuda.current_stream()).  There is no CPU fallback: importing works
without a GPU, but every call needs libwproj.so and a CUDA device and raises
WprojError otherwise.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwproj.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_BUILT, ERR_UNSUPPORTED = range(7)
CHIRP = {"exact": 0, "linear": 1}
EXTENSION = {"full": 0, "clamp": 1}
VALUE_DTYPE = {"f32": 0, "bf16": 1, "f16": 2}
INDEX_FORMAT = {"auto": 0, "columns": 1, "mask": 2, "runs": 3}

EXPORTED = [
    "wproj_plan_create", "wproj_plan_destroy", "wproj_build_kernels", "wproj_get_csr",
    "wproj_phi", "wproj_phi_adj", "wproj_phi_cplx", "wproj_solve_bpdn", "wproj_power_norm2",
    "wproj_fft2d", "wproj_set_timing", "wproj_get_stats", "wproj_reset_stats",
    "wproj_dr_defaults", "wproj_last_error", "wproj_version", "wproj_dr_state_get",
    "wproj_dr_state_set", "wproj_phi_noalloc", "wproj_csr_rows",
    "wproj_batch_create", "wproj_batch_destroy", "wproj_batch_build", "wproj_batch_tune",
    "wproj_batch_set_schedule", "wproj_batch_phi", "wproj_batch_phi_adj", "wproj_batch_solve_bpdn",
    "wproj_batch_get_info", "wproj_gemm_bf16", "wproj_gemm_test_hook", "wproj_mlp_num_params", "wproj_mlp_create",
    "wproj_mlp_destroy", "wproj_mlp_set_params", "wproj_mlp_get_params", "wproj_mlp_targets",
    "wproj_mlp_forward", "wproj_mlp_gradients", "wproj_mlp_train", "wproj_build_kernels_learned",
    "wproj_daubechies_taps", "wproj_dwt2", "wproj_idwt2", "wproj_set_screens", "wproj_build_kernels_dde",
]


class WprojError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"wproj status {status}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("kb_support", ctypes.c_int32), ("fov", ctypes.c_double),
                ("chirp", ctypes.c_int32), ("extension", ctypes.c_int32), ("box", ctypes.c_int32),
                ("value_dtype", ctypes.c_int32), ("index_format", ctypes.c_int32), ("upsampling", ctypes.c_int32)]


class CSR(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_cols", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("row_scale", ctypes.c_void_p), ("value_dtype", ctypes.c_int32),
                ("index_format", ctypes.c_int32), ("n_seg", ctypes.c_int64), ("stream", ctypes.c_void_p),
                ("stream_bytes", ctypes.c_int64)]


class DRParams(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
                ("gamma_frac", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("phi_norm2", ctypes.c_double), ("power_iters", ctypes.c_int32),
                ("resume", ctypes.c_int32), ("psi", ctypes.c_int32), ("psi_levels", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int32), ("phi_norm2", ctypes.c_double),
                ("gamma", ctypes.c_double), ("final_resid", ctypes.c_double),
                ("final_l1", ctypes.c_double)]


class BatchSchedule(ctypes.Structure):
    _fields_ = [("piece", ctypes.c_int64), ("chunk", ctypes.c_int64), ("degrid_ms", ctypes.c_double),
                ("grid_ms", ctypes.c_double), ("lanes_per_piece", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_problems", ctypes.c_int32), ("m", ctypes.c_int64), ("pixels", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("n_pieces", ctypes.c_int64), ("n_chunks", ctypes.c_int64),
                ("piece", ctypes.c_int64), ("chunk", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("iter_launches", ctypes.c_int64), ("lanes_per_piece", ctypes.c_int32)]


class LearnedInfo(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("learned", ctypes.c_int64), ("rel_l2_mean", ctypes.c_double),
                ("plain_ms", ctypes.c_double), ("learned_ms", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("nnz", ctypes.c_int64), ("box_min", ctypes.c_int32),
                ("box_max", ctypes.c_int32), ("segments", ctypes.c_int64),
                ("degrid_pieces", ctypes.c_int64), ("grid_chunks", ctypes.c_int64),
                ("build_ms", ctypes.c_double), ("t_fft_ms", ctypes.c_double),
                ("t_degrid_ms", ctypes.c_double), ("t_grid_ms", ctypes.c_double),
                ("t_reduce_ms", ctypes.c_double), ("t_solver_ms", ctypes.c_double),
                ("n_fft", ctypes.c_int64), ("n_degrid", ctypes.c_int64), ("n_grid", ctypes.c_int64),
                ("n_reduce", ctypes.c_int64), ("n_solver", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("runs_bytes", ctypes.c_int64), ("t_build_fft_ms", ctypes.c_double),
                ("t_build_select_ms", ctypes.c_double), ("t_build_emit_ms", ctypes.c_double),
                ("n_build_fft", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    """Load libwproj.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise WprojError(ERR_UNSUPPORTED, f"{LIB_PATH} missing: build it with "
                         "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "wproj_plan_create": [P(vp), P(GridDesc)],
        "wproj_plan_destroy": [vp],
        "wproj_build_kernels": [vp, vp, i64, dbl, vp, P(CSR)],
        "wproj_get_csr": [vp, P(CSR)],
        "wproj_phi": [vp, vp, vp, vp],
        "wproj_phi_adj": [vp, vp, vp, vp, vp],
        "wproj_phi_cplx": [vp, vp, vp, vp],
        "wproj_phi_noalloc": [vp, vp, vp, vp],
        "wproj_csr_rows": [vp, i64, i64, vp, vp, vp],
        "wproj_solve_bpdn": [vp, vp, dbl, P(DRParams), vp, P(SolveInfo), vp],
        "wproj_power_norm2": [vp, i32, P(dbl), vp],
        "wproj_fft2d": [vp, vp, i32, i32, i32, vp],
        "wproj_set_timing": [vp, i32],
        "wproj_get_stats": [vp, P(Stats)],
        "wproj_reset_stats": [vp],
        "wproj_dr_state_get": [vp, vp, vp, P(dbl), P(dbl), vp],
        "wproj_dr_state_set": [vp, vp, vp, dbl, dbl, vp],
        "wproj_batch_create": [P(vp), i32, P(GridDesc)],
        "wproj_batch_destroy": [vp],
        "wproj_batch_build": [vp, vp, P(i64), dbl, vp],
        "wproj_batch_tune": [vp, P(BatchSchedule), vp],
        "wproj_batch_set_schedule": [vp, i64, i64, ctypes.c_int32, vp],
        "wproj_batch_phi": [vp, vp, vp, vp],
        "wproj_batch_phi_adj": [vp, vp, vp, vp],
        "wproj_batch_solve_bpdn": [vp, vp, P(dbl), P(DRParams), vp, vp],
        "wproj_batch_get_info": [vp, P(BatchInfo)],
        "wproj_gemm_bf16": [i32, i32, i32, vp, vp, vp, vp, i32, vp],
        "wproj_gemm_test_hook": [i32, ctypes.c_uint64],
        "wproj_daubechies_taps": [i32, P(dbl)],
        "wproj_set_screens": [vp, vp, i32, vp],
        "wproj_build_kernels_dde": [vp, vp, i64, vp, dbl, vp],
        "wproj_dwt2": [i32, i32, i32, vp, vp, vp, vp],
        "wproj_idwt2": [i32, i32, i32, vp, vp, vp, vp],
        "wproj_mlp_create": [P(vp)],
        "wproj_mlp_destroy": [vp],
        "wproj_mlp_set_params": [vp, vp, vp],
        "wproj_mlp_get_params": [vp, vp, vp],
        "wproj_mlp_targets": [vp, vp, vp, vp, vp, vp],
        "wproj_mlp_forward": [vp, vp, i64, vp, vp],
        "wproj_mlp_gradients": [vp, vp, vp, vp, i64, dbl, P(dbl), vp, vp],
        "wproj_mlp_train": [vp, vp, vp, vp, i64, i32, i32, dbl, dbl, vp, vp],
        "wproj_build_kernels_learned": [vp, vp, vp, i64, dbl, dbl, vp, P(LearnedInfo), vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.wproj_mlp_num_params.argtypes = []
    L.wproj_mlp_num_params.restype = ctypes.c_int64
    L.wproj_dr_defaults.argtypes = [P(DRParams)]
    L.wproj_dr_defaults.restype = None
    L.wproj_last_error.restype = ctypes.c_char_p
    L.wproj_version.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(st: int):
    if st != OK:
        raise WprojError(st, lib().wproj_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise WprojError(ERR_INVALID_ARG, "tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise WprojError(ERR_INVALID_ARG, "tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class _CAI:
    """Zero-copy view of plan-owned device memory (__cuda_array_interface__)."""

    def __init__(self, ptr: int, shape: tuple, typestr: str):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": shape,
                                         "typestr": typestr, "version": 2, "strides": None}


def dr_defaults() -> DRParams:
    p = DRParams()
    lib().wproj_dr_defaults(ctypes.byref(p))
    return p


class CSRView:
    """G in CSR terms (valid until the next build or close of its plan).

    row_ptr is a zero-copy view.  COLUMNS format: `col` / `val` are zero-copy
    views of the plan's arrays.  TILE_MASK format (tile stream): `rows(k0, k1)`
    exports rows on demand; `col` / `val` export every row on first access.
    Values are complex64 (f32) or (nnz, 2) bf16 / f16 scaled by `row_scale`.
    """

    def __init__(self, plan: "Plan", c: CSR):
        self._plan = plan
        self.m, self.nnz, self.n_cols, self.n_seg = int(c.m), int(c.nnz), int(c.n_cols), int(c.n_seg)
        self.value_dtype = {0: "f32", 1: "bf16", 2: "f16"}[c.value_dtype]
        self.index_format = {1: "columns", 2: "mask", 3: "runs"}[c.index_format]
        self.stream_bytes = int(c.stream_bytes)
        self._dev = torch.device("cuda", torch.cuda.current_device())
        self.row_ptr = torch.as_tensor(_CAI(c.row_ptr, (self.m + 1,), "<i8"), device=self._dev)
        self.row_scale = None
        if c.value_dtype != 0:
            self.row_scale = torch.as_tensor(_CAI(c.row_scale, (self.m,), "<f4"), device=self._dev)
        self._col = self._val = None
        if self.index_format == "columns":
            self._col = torch.as_tensor(_CAI(c.col, (self.nnz,), "<i4"), device=self._dev)
            self._val = self._val_view(torch.as_tensor(_CAI(c.val, (self.nnz, 2), "<f4" if c.value_dtype == 0
                                                            else "<i2"), device=self._dev))

    def _val_view(self, raw: torch.Tensor) -> torch.Tensor:
        if self.value_dtype == "f32":
            return torch.view_as_complex(raw)
        return raw.view(torch.bfloat16 if self.value_dtype == "bf16" else torch.float16)

    def rows(self, k0: int, k1: int):
        """(col, val) of rows [k0, k1) in CSR order, fresh device tensors."""
        rp = self.row_ptr
        n = int(rp[k1].item() - rp[k0].item()) if k1 > k0 else 0
        col = torch.empty(max(n, 1), dtype=torch.int32, device=self._dev)[:n]
        raw = torch.empty((max(n, 1), 2), dtype=torch.float32 if self.value_dtype == "f32" else torch.int16,
                          device=self._dev)[:n]
        _check(lib().wproj_csr_rows(self._plan._h, int(k0), int(k1), ctypes.c_void_p(col.data_ptr()),
                                    ctypes.c_void_p(raw.data_ptr()), _stream(None)))
        return col, self._val_view(raw)

    def _export_all(self):
        if self._col is None:
            self._col, self._val = self.rows(0, self.m)

    @property
    def col(self) -> torch.Tensor:
        self._export_all()
        return self._col

    @property
    def val(self) -> torch.Tensor:
        self._export_all()
        return self._val


class Plan:
    """A libwproj plan: geometry, the built G and its work buffers."""

    def __init__(self, n: int, fov: float, kb_support: int = 4, chirp: str = "exact",
                 extension: str = "full", box="G", value_dtype: str = "f32", index_format: str = "auto",
                 upsampling: bool = False):
        """box: "G" (default) the exact S = 2N box, "rule" the S(w) rule, or a
        fixed power of two.  upsampling=True: the paper's operator C-hat F U
        (visibilities on the grid, kb_support=1, grid cells 1/fov)."""
        self._h = ctypes.c_void_p()
        self.n = n
        self.G = 2 * n
        self.value_dtype = value_dtype
        box_i = 2 * n if box in ("G", None) else (0 if box == "rule" else int(box))
        d = GridDesc(n, kb_support, float(fov), CHIRP[chirp], EXTENSION[extension], box_i,
                     VALUE_DTYPE[value_dtype], INDEX_FORMAT[index_format], 1 if upsampling else 0)
        self.desc = d
        self.m = 0
        _check(lib().wproj_plan_create(ctypes.byref(self._h), ctypes.byref(d)))

    def close(self):
        if self._h:
            lib().wproj_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ---- Part I
    def build_kernels(self, uvw: torch.Tensor, e: float, screen_id: torch.Tensor | None = None,
                      stream=None) -> CSR:
        """G for the visibilities uvw (M, 3); screen_id (M int32 on the device)
        attaches the screen set by set_screens to every row."""
        if uvw.dtype != torch.float64 or uvw.dim() != 2 or uvw.shape[1] != 3:
            raise WprojError(ERR_INVALID_ARG, "uvw must be an (M, 3) float64 tensor")
        out = CSR()
        if screen_id is None:
            _check(lib().wproj_build_kernels(self._h, _ptr(uvw), uvw.shape[0], float(e), _stream(stream),
                                             ctypes.byref(out)))
        else:
            if screen_id.dtype != torch.int32 or screen_id.numel() != uvw.shape[0] or not screen_id.is_cuda:
                raise WprojError(ERR_INVALID_ARG, "screen_id must be an int32 device tensor of M ids")
            _check(lib().wproj_build_kernels_dde(self._h, _ptr(uvw), uvw.shape[0], _ptr(screen_id.contiguous()),
                                                 float(e), _stream(stream)))
            _check(lib().wproj_get_csr(self._h, ctypes.byref(out)))
        self.m = int(out.m)
        return out

    def set_screens(self, screens: torch.Tensor | None, stream=None):
        """Direction-dependent screens, complex64 (n, G, G), centred (index a at
        offset a - G/2); None drops them."""
        if screens is None:
            _check(lib().wproj_set_screens(self._h, None, 0, _stream(stream)))
            return
        G = 2 * self.n
        if screens.dtype != torch.complex64 or screens.dim() != 3 or tuple(screens.shape[1:]) != (G, G):
            raise WprojError(ERR_INVALID_ARG, f"screens must be complex64 (n, {G}, {G})")
        screens = screens.contiguous()
        _check(lib().wproj_set_screens(self._h, _ptr(screens), screens.shape[0], _stream(stream)))

    def build_kernels_learned(self, net: "MLP", uvw: torch.Tensor, e: float, rel_l2_max: float = 1e-3,
                              stream=None):
        """Plain build, then rows whose predicted kernel passes the checks take it
        (include/wproj.h).  Returns (info dict, per-row relative L2 errors)."""
        if uvw.dtype != torch.float64 or uvw.dim() != 2 or uvw.shape[1] != 3:
            raise WprojError(ERR_INVALID_ARG, "uvw must be an (M, 3) float64 tensor")
        uvw = uvw.contiguous()
        err = torch.empty(uvw.shape[0], dtype=torch.float32, device=uvw.device)
        info = LearnedInfo()
        _check(lib().wproj_build_kernels_learned(self._h, net._h, _ptr(uvw), uvw.shape[0], float(e),
                                                 float(rel_l2_max), _ptr(err), ctypes.byref(info), _stream(stream)))
        self.m = uvw.shape[0]
        return {f: getattr(info, f) for f, _ in info._fields_}, err

    def csr(self) -> CSRView:
        """View of G (see CSRView)."""
        c = CSR()
        _check(lib().wproj_get_csr(self._h, ctypes.byref(c)))
        return CSRView(self, c)

    # ---- Part II
    def phi(self, x: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if x.dtype == torch.complex64:
            return self.phi_cplx(x, y, stream)
        if x.dtype != torch.float32 or tuple(x.shape) != (self.n, self.n):
            raise WprojError(ERR_INVALID_ARG, f"x must be a ({self.n}, {self.n}) float32 tensor")
        if y is None:
            y = torch.empty(self.m, dtype=torch.complex64, device=x.device)
        _check(lib().wproj_phi(self._h, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def phi_cplx(self, x: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if x.dtype != torch.complex64 or tuple(x.shape) != (self.n, self.n):
            raise WprojError(ERR_INVALID_ARG, f"x must be a ({self.n}, {self.n}) complex64 tensor")
        if y is None:
            y = torch.empty(self.m, dtype=torch.complex64, device=x.device)
        _check(lib().wproj_phi_cplx(self._h, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def phi_adj(self, y: torch.Tensor, x_re: torch.Tensor | None = None, complex_out: bool = False,
                stream=None):
        if y.dtype != torch.complex64 or y.numel() != self.m:
            raise WprojError(ERR_INVALID_ARG, f"y must be a complex64 tensor of {self.m} visibilities")
        if complex_out:
            xc = torch.empty((self.n, self.n), dtype=torch.complex64, device=y.device)
            _check(lib().wproj_phi_adj(self._h, _ptr(y), None, _ptr(xc), _stream(stream)))
            return xc
        if x_re is None:
            x_re = torch.empty((self.n, self.n), dtype=torch.float32, device=y.device)
        _check(lib().wproj_phi_adj(self._h, _ptr(y), _ptr(x_re), None, _stream(stream)))
        return x_re

    # ---- Part III
    def solve_bpdn(self, y: torch.Tensor, eps: float, iters: int = 50, inner_iters: int = 10,
                   gamma_frac: float = 1e-2, lam: float = 1.0, phi_norm2: float = 0.0,
                   power_iters: int = 100, x_out: torch.Tensor | None = None, sync: bool = True,
                   resume: bool = False, psi: int = 0, psi_levels: int = 4, stream=None):
        """Douglas-Rachford BPDN (Eq. 7).  psi = 0: Dirac basis; psi = p: Daubechies
        wavelets with p vanishing moments (8 = Db8) over psi_levels levels; the
        returned image is x = Psi alpha.  resume=True continues from the plan's
        state (the previous solve or dr_state_set) instead of z = Psi^T Re Phi^H y, u = 0."""
        if y.dtype != torch.complex64 or y.numel() != self.m:
            raise WprojError(ERR_INVALID_ARG, f"y must be a complex64 tensor of {self.m} visibilities")
        prm = DRParams(iters, inner_iters, gamma_frac, lam, phi_norm2, power_iters, 1 if resume else 0,
                       psi, psi_levels)
        if x_out is None:
            x_out = torch.empty((self.n, self.n), dtype=torch.float32, device=y.device)
        info = SolveInfo() if sync else None
        _check(lib().wproj_solve_bpdn(self._h, _ptr(y), float(eps), ctypes.byref(prm), _ptr(x_out),
                                      ctypes.byref(info) if info is not None else None, _stream(stream)))
        return x_out, info

    def dr_state(self, stream=None):
        """Checkpoint of the DR state: (z, u, gamma, phi_norm2), z and u on the device."""
        dev = torch.device("cuda", torch.cuda.current_device())
        z = torch.empty((self.n, self.n), dtype=torch.float32, device=dev)
        u = torch.empty(self.m, dtype=torch.complex64, device=dev)
        g, n2 = ctypes.c_double(), ctypes.c_double()
        _check(lib().wproj_dr_state_get(self._h, _ptr(z), _ptr(u), ctypes.byref(g), ctypes.byref(n2),
                                        _stream(stream)))
        return z, u, g.value, n2.value

    def set_dr_state(self, z: torch.Tensor, u: torch.Tensor, gamma: float, phi_norm2: float, stream=None):
        """Restore a checkpoint; z and u may live on the host or the device."""
        if tuple(z.shape) != (self.n, self.n) or z.dtype != torch.float32:
            raise WprojError(ERR_INVALID_ARG, "z must be an (N, N) float32 tensor")
        if u.numel() != self.m or u.dtype != torch.complex64:
            raise WprojError(ERR_INVALID_ARG, "u must be a complex64 tensor of M entries")
        z, u = z.contiguous(), u.contiguous()
        _check(lib().wproj_dr_state_set(self._h, ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                        float(gamma), float(phi_norm2), _stream(stream)))

    def power_norm2(self, iters: int = 100, stream=None) -> float:
        out = ctypes.c_double()
        _check(lib().wproj_power_norm2(self._h, iters, ctypes.byref(out), _stream(stream)))
        return out.value

    # ---- reporting
    def set_timing(self, on: bool):
        _check(lib().wproj_set_timing(self._h, 1 if on else 0))

    def stats(self) -> dict:
        s = Stats()
        _check(lib().wproj_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def reset_stats(self):
        _check(lib().wproj_reset_stats(self._h))


def fft2d(x: torch.Tensor, inverse: bool = False, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Unnormalised 2-D DFT of a (batch, n, n) or (n, n) complex64 tensor."""
    if x.dtype != torch.complex64 or x.shape[-1] != x.shape[-2]:
        raise WprojError(ERR_INVALID_ARG, "x must be complex64 with square trailing dims")
    n = x.shape[-1]
    batch = x.numel() // (n * n)
    if out is None:
        out = torch.empty_like(x)
    _check(lib().wproj_fft2d(_ptr(x), _ptr(out), n, batch, 1 if inverse else 0, _stream(stream)))
    return out


def daubechies_taps(p: int) -> list[float]:
    """Low-pass analysis taps (2p) of the extremal-phase Daubechies wavelet with p
    vanishing moments."""
    out = (ctypes.c_double * (2 * p))() if p > 0 else (ctypes.c_double * 1)()
    _check(lib().wproj_daubechies_taps(p, out))
    return list(out)


def _wavelet(fn, src: torch.Tensor, levels: int, p: int, out, stream):
    if src.dtype != torch.float32 or src.dim() != 2 or src.shape[0] != src.shape[1] or not src.is_contiguous():
        raise WprojError(ERR_INVALID_ARG, "expected a contiguous (n, n) float32 tensor")
    n = src.shape[0]
    if out is None:
        out = torch.empty_like(src)
    work = torch.empty(max(1, n * n // 2), dtype=torch.float32, device=src.device)
    _check(fn(n, levels, p, _ptr(src), _ptr(out), _ptr(work), _stream(stream)))
    return out


def dwt2(x: torch.Tensor, levels: int = 4, p: int = 8, out: torch.Tensor | None = None, stream=None):
    """alpha = Psi^T x: periodic 2-D Daubechies-p analysis in the Mallat layout."""
    return _wavelet(lib().wproj_dwt2, x, levels, p, out, stream)


def idwt2(alpha: torch.Tensor, levels: int = 4, p: int = 8, out: torch.Tensor | None = None, stream=None):
    """x = Psi alpha: the synthesis (inverse and transpose of dwt2)."""
    return _wavelet(lib().wproj_idwt2, alpha, levels, p, out, stream)


class Batch:
    """Many independent problems (image sides ns, shared field of view) whose
    operators and Douglas-Rachford iterations run as shared launches
    (include/wproj.h, wproj_batch_*).  Images, visibilities and uvw are
    concatenated in problem order; `split_images` / `split_vis` cut them apart."""

    def __init__(self, ns, fov: float, kb_support: int = 4, chirp: str = "exact", extension: str = "full",
                 box="rule"):
        self._h = ctypes.c_void_p()
        self.ns = [int(n) for n in ns]
        descs = (GridDesc * len(self.ns))()
        for i, n in enumerate(self.ns):
            box_i = 2 * n if box in ("G", None) else (0 if box == "rule" else int(box))
            descs[i] = GridDesc(n, kb_support, float(fov), CHIRP[chirp], EXTENSION[extension], box_i,
                                VALUE_DTYPE["f32"], INDEX_FORMAT["columns"])
        self.img_off = [0]
        for n in self.ns:
            self.img_off.append(self.img_off[-1] + n * n)
        self.ms, self.vis_off = [], [0]
        _check(lib().wproj_batch_create(ctypes.byref(self._h), len(self.ns), descs))

    def close(self):
        if self._h:
            lib().wproj_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def pixels(self) -> int:
        return self.img_off[-1]

    @property
    def m(self) -> int:
        return self.vis_off[-1]

    def build_kernels(self, uvw: torch.Tensor, ms, e: float, stream=None):
        """uvw: (sum ms, 3) float64 on the device, problems in order."""
        self.ms = [int(m) for m in ms]
        self.vis_off = [0]
        for m in self.ms:
            self.vis_off.append(self.vis_off[-1] + m)
        if uvw.dtype != torch.float64 or tuple(uvw.shape) != (self.m, 3):
            raise WprojError(ERR_INVALID_ARG, f"uvw must be a ({self.m}, 3) float64 tensor")
        arr = (ctypes.c_int64 * len(self.ms))(*self.ms)
        _check(lib().wproj_batch_build(self._h, _ptr(uvw.contiguous()), arr, float(e), _stream(stream)))

    def tune(self, stream=None) -> dict:
        out = BatchSchedule()
        _check(lib().wproj_batch_tune(self._h, ctypes.byref(out), _stream(stream)))
        return {f: getattr(out, f) for f, _ in out._fields_}

    def set_schedule(self, piece: int, chunk: int, lanes_per_piece: int = 0, stream=None):
        _check(lib().wproj_batch_set_schedule(self._h, int(piece), int(chunk), int(lanes_per_piece),
                                              _stream(stream)))

    def info(self) -> dict:
        out = BatchInfo()
        _check(lib().wproj_batch_get_info(self._h, ctypes.byref(out)))
        return {f: getattr(out, f) for f, _ in out._fields_}

    def phi(self, x: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if x.dtype != torch.float32 or x.numel() != self.pixels:
            raise WprojError(ERR_INVALID_ARG, f"x must hold {self.pixels} float32 pixels")
        if y is None:
            y = torch.empty(self.m, dtype=torch.complex64, device=x.device)
        _check(lib().wproj_batch_phi(self._h, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def phi_adj(self, y: torch.Tensor, x: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if y.dtype != torch.complex64 or y.numel() != self.m:
            raise WprojError(ERR_INVALID_ARG, f"y must hold {self.m} complex64 visibilities")
        if x is None:
            x = torch.empty(self.pixels, dtype=torch.float32, device=y.device)
        _check(lib().wproj_batch_phi_adj(self._h, _ptr(y), _ptr(x), _stream(stream)))
        return x

    def solve_bpdn(self, y: torch.Tensor, eps, iters: int = 50, inner_iters: int = 10, gamma_frac: float = 1e-2,
                   lam: float = 1.0, power_iters: int = 100, x_out: torch.Tensor | None = None,
                   resume: bool = False, psi: int = 0, psi_levels: int = 4, stream=None) -> torch.Tensor:
        if y.dtype != torch.complex64 or y.numel() != self.m:
            raise WprojError(ERR_INVALID_ARG, f"y must hold {self.m} complex64 visibilities")
        eps = [float(v) for v in eps]
        if len(eps) != len(self.ns):
            raise WprojError(ERR_INVALID_ARG, "one eps per problem")
        prm = DRParams(iters, inner_iters, gamma_frac, lam, 0.0, power_iters, 1 if resume else 0, psi, psi_levels)
        if x_out is None:
            x_out = torch.empty(self.pixels, dtype=torch.float32, device=y.device)
        arr = (ctypes.c_double * len(eps))(*eps)
        _check(lib().wproj_batch_solve_bpdn(self._h, _ptr(y), arr, ctypes.byref(prm), _ptr(x_out),
                                            _stream(stream)))
        return x_out

    def split_images(self, x: torch.Tensor):
        return [x[a:b].view(n, n) for a, b, n in zip(self.img_off[:-1], self.img_off[1:], self.ns)]

    def split_vis(self, y: torch.Tensor):
        return [y[a:b] for a, b in zip(self.vis_off[:-1], self.vis_off[1:])]


def gemm_bf16(a: torch.Tensor, b: torch.Tensor, bias: torch.Tensor | None = None, out_bf16: bool = False,
              stream=None) -> torch.Tensor:
    """a (m, k) and b (n, k) BF16 on the device: a @ b.T (+ bias) on the tensor cores."""
    if a.dtype != torch.bfloat16 or b.dtype != torch.bfloat16 or a.shape[1] != b.shape[1]:
        raise WprojError(ERR_INVALID_ARG, "a (m, k) and b (n, k) must be bfloat16")
    m, k = a.shape
    n = b.shape[0]
    c = torch.empty((m, n), dtype=torch.bfloat16 if out_bf16 else torch.float32, device=a.device)
    _check(lib().wproj_gemm_bf16(m, n, k, _ptr(a.contiguous()), _ptr(b.contiguous()),
                                 _ptr(bias) if bias is not None else None, _ptr(c), 1 if out_bf16 else 0,
                                 _stream(stream)))
    return c


class MLP:
    """The learned-kernel network (include/wproj.h, wproj_mlp_*): (w, offset) ->
    32 x 32 kernel window (2048 values) + support logits (1024)."""

    N_IN, N_HID, N_VAL, N_MASK = 3, 256, 2048, 1024

    def __init__(self, params: torch.Tensor | None = None):
        self._h = ctypes.c_void_p()
        _check(lib().wproj_mlp_create(ctypes.byref(self._h)))
        self.n_params = int(lib().wproj_mlp_num_params())
        if params is not None:
            self.set_params(params)

    def close(self):
        if self._h:
            lib().wproj_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p: torch.Tensor, stream=None):
        if p.dtype != torch.float32 or p.numel() != self.n_params:
            raise WprojError(ERR_INVALID_ARG, f"params must be {self.n_params} float32 values")
        p = p.contiguous()
        _check(lib().wproj_mlp_set_params(self._h, ctypes.c_void_p(p.data_ptr()), _stream(stream)))

    def params(self, stream=None) -> torch.Tensor:
        p = torch.empty(self.n_params, dtype=torch.float32)
        _check(lib().wproj_mlp_get_params(self._h, ctypes.c_void_p(p.data_ptr()), _stream(stream)))
        return p

    @staticmethod
    def targets(plan: "Plan", uvw: torch.Tensor, stream=None):
        dev = uvw.device
        m = uvw.shape[0]
        x0 = torch.empty((m, 3), dtype=torch.float32, device=dev)
        tv = torch.empty((m, 2048), dtype=torch.float32, device=dev)
        tm = torch.empty((m, 1024), dtype=torch.float32, device=dev)
        _check(lib().wproj_mlp_targets(plan._h, _ptr(uvw.contiguous()), _ptr(x0), _ptr(tv), _ptr(tm),
                                       _stream(stream)))
        return x0, tv, tm

    def forward(self, x0: torch.Tensor, stream=None) -> torch.Tensor:
        m = x0.shape[0]
        y = torch.empty((m, 3072), dtype=torch.float32, device=x0.device)
        _check(lib().wproj_mlp_forward(self._h, _ptr(x0.contiguous()), m, _ptr(y), _stream(stream)))
        return y

    def gradients(self, x0, tv, tm, mask_weight: float = 0.1, stream=None):
        loss = ctypes.c_double()
        g = torch.empty(self.n_params, dtype=torch.float32, device=x0.device)
        _check(lib().wproj_mlp_gradients(self._h, _ptr(x0.contiguous()), _ptr(tv.contiguous()),
                                         _ptr(tm.contiguous()), x0.shape[0], float(mask_weight),
                                         ctypes.byref(loss), _ptr(g), _stream(stream)))
        return loss.value, g

    def train(self, x0, tv, tm, batch: int, steps: int, lr: float, mask_weight: float = 0.1, stream=None):
        losses = (ctypes.c_float * max(1, steps))()
        _check(lib().wproj_mlp_train(self._h, _ptr(x0.contiguous()), _ptr(tv.contiguous()), _ptr(tm.contiguous()),
                                     x0.shape[0], int(batch), int(steps), float(lr), float(mask_weight), losses,
                                     _stream(stream)))
        return list(losses)[:steps]
