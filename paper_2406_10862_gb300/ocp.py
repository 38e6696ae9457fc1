"""Thin Python binding of the C interface in ``include/ocp.h``.

Only argument marshalling happens here: every computation runs in the CUDA
kernels of ``_build/libocp.so``.  There is no fallback -- if the library has
not been built, or no CUDA device is present, using it raises.  Device memory
and streams come from PyTorch: arrays are ``torch.Tensor`` objects on the
grid's device, and calls are enqueued on the current PyTorch stream of that
device unless a stream is given.

The functions keep the C names (``ocp_linearize`` ...); ``Grid`` wraps them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

OCP_OK, OCP_ERR_INVALID_ARG, OCP_ERR_CUDA, OCP_ERR_OOM = 0, 1, 2, 3
OCP_ERR_NONFINITE, OCP_ERR_TIMEOUT, OCP_ERR_UNSUPPORTED = 4, 5, 6
STATUS_NAMES = {0: "OCP_OK", 1: "OCP_ERR_INVALID_ARG", 2: "OCP_ERR_CUDA", 3: "OCP_ERR_OOM",
                4: "OCP_ERR_NONFINITE", 5: "OCP_ERR_TIMEOUT", 6: "OCP_ERR_UNSUPPORTED"}

# Every symbol the header declares; the CPU tests check the library exports them.
EXPORTS = ["ocp_grid_create", "ocp_grid_destroy", "ocp_grid_info", "ocp_bsr_pattern", "ocp_linearize",
           "ocp_linearize_noalloc", "ocp_probe_fp64", "ocp_batch_create", "ocp_batch_destroy",
           "ocp_batch_set_io", "ocp_batch_linearize", "ocp_batch_graph_launch", "ocp_batch_tune",
           "ocp_batch_set_shape", "ocp_batch_get_shape", "ocp_batch_get_status", "ocp_grid_set_shape",
           "ocp_grid_get_shape", "ocp_grid_cluster_tiles",
           "ocp_solver_work_doubles", "ocp_bicgstab", "ocp_newton_update", "ocp_well_rates_vjp",
           "ocp_grid_update_perm", "ocp_coupling_work_ints", "ocp_coupling_components", "ocp_linearize_wells",
           "ocp_bicgstab_wells", "ocp_well_update", "ocp_residual_norms", "ocp_linearize_pn", "ocp_pn_update",
           "ocp_pn_norms", "ocp_pn_from_natural", "ocp_impec_pressure", "ocp_impec_update", "ocp_bicgstab_scalar", "ocp_bsr_spmv", "ocp_adjoint_vjp",
           "ocp_well_rates", "ocp_get_status", "ocp_last_error"]

# ocp_well_ctrl: int32 mode, int32 phase, double target, double limit (24 bytes)
CTRL_DTYPE = np.dtype([("mode", "<i4"), ("phase", "<i4"), ("target", "<f8"), ("limit", "<f8")])


def well_controls(controls, limits, device):
    """Device array of ocp_well_ctrl from (mode, phase, target) tuples and limits."""
    a = np.zeros(len(controls), dtype=CTRL_DTYPE)
    for i, ((mode, phase, target), lim) in enumerate(zip(controls, limits)):
        a[i] = (int(mode), int(phase), float(target), float(lim))
    raw = np.frombuffer(a.tobytes(), dtype=np.uint8) if len(a) else np.zeros(0, dtype=np.uint8)
    return torch.as_tensor(raw.copy(), device=device)


def read_controls(ctrl):
    """(mode, phase, target, limit) tuples of a device ocp_well_ctrl array."""
    a = np.frombuffer(ctrl.cpu().numpy().tobytes(), dtype=CTRL_DTYPE)
    return [(int(r["mode"]), int(r["phase"]), float(r["target"]), float(r["limit"])) for r in a]


class OcpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class _Well(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("phase", ctypes.c_int), ("p_bh", ctypes.c_double),
                ("rw", ctypes.c_double), ("skin", ctypes.c_double), ("nperf", ctypes.c_int),
                ("cells", ctypes.POINTER(ctypes.c_int64))]


_D = ctypes.POINTER(ctypes.c_double)


class _Desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("top_depth", ctypes.c_double), ("nphase", ctypes.c_int),
                ("lnk", _D), ("phi", _D),
                ("kz_over_kx", ctypes.c_double), ("cr", ctypes.c_double), ("p_ref", ctypes.c_double),
                ("nrow", ctypes.c_int),
                ("tab_p", _D), ("tab_Bo", _D), ("tab_Bg", _D), ("tab_Rs", _D), ("tab_muo", _D), ("tab_mug", _D)]
    _fields_ += [(n, ctypes.c_double) for n in
                 ("bw_ref", "cw", "muw", "rho_osc", "rho_gsc", "rho_wsc", "co_under", "cmu_under",
                  "swc", "sorw", "sorg", "sgc", "nw", "now", "ng", "nog", "krw_max", "krg_max", "kro_cw",
                  "pcow_max", "pcgo_max")]
    _fields_ += [("nwell", ctypes.c_int), ("wells", ctypes.POINTER(_Well))]


class _BatchIO(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("u_new", "flag_new", "u_old", "flag_old", "residual",
                                                "bsr_val", "face_flux")]


class _Shape(ctypes.Structure):
    _fields_ = [("cells_per_tile", ctypes.c_int * 3), ("ctas_per_sm", ctypes.c_int * 3), ("ordered", ctypes.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libocp.so (building it first only when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libocp.so is not built (%s); run __graft_entry__.build()" % path)
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i64, i32p = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
    lib.ocp_grid_create.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int, ctypes.POINTER(vp)]
    lib.ocp_grid_destroy.argtypes = [vp]
    lib.ocp_grid_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64)]
    lib.ocp_bsr_pattern.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.ocp_linearize.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, vp, vp, vp, vp]
    lib.ocp_linearize_noalloc.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, vp, vp, vp, vp]
    lib.ocp_bsr_spmv.argtypes = [vp, vp, ctypes.c_double, vp, ctypes.c_double, vp, ctypes.c_int, vp]
    lib.ocp_adjoint_vjp.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.ocp_well_rates.argtypes = [vp, vp, vp, vp, vp]
    lib.ocp_get_status.argtypes = [vp, vp]
    lib.ocp_probe_fp64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.ocp_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
    lib.ocp_batch_destroy.argtypes = [vp]
    lib.ocp_batch_set_io.argtypes = [vp, ctypes.POINTER(_BatchIO)]
    lib.ocp_batch_linearize.argtypes = [vp, ctypes.c_double, vp]
    lib.ocp_batch_graph_launch.argtypes = [vp, ctypes.c_double, vp]
    lib.ocp_batch_tune.argtypes = [vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_Shape), vp]
    lib.ocp_batch_set_shape.argtypes = [vp, ctypes.POINTER(_Shape)]
    lib.ocp_batch_get_shape.argtypes = [vp, ctypes.POINTER(_Shape)]
    lib.ocp_batch_get_status.argtypes = [vp, vp]
    lib.ocp_grid_set_shape.argtypes = [vp, ctypes.POINTER(_Shape)]
    lib.ocp_grid_get_shape.argtypes = [vp, ctypes.POINTER(_Shape)]
    lib.ocp_grid_cluster_tiles.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.ocp_solver_work_doubles.argtypes = [vp]
    lib.ocp_solver_work_doubles.restype = ctypes.c_int64
    lib.ocp_bicgstab.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp,
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), vp]
    lib.ocp_newton_update.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, vp, vp, vp]
    lib.ocp_well_rates_vjp.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.ocp_linearize_wells.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.ocp_bicgstab_wells.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_double), vp]
    lib.ocp_well_update.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp, vp, vp]
    lib.ocp_residual_norms.argtypes = [vp, vp, ctypes.c_double, vp, vp, vp, vp]
    lib.ocp_linearize_pn.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp, vp, vp, vp, vp, vp]
    lib.ocp_pn_update.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp, vp]
    lib.ocp_pn_norms.argtypes = [vp, vp, ctypes.c_double, vp, vp]
    lib.ocp_pn_from_natural.argtypes = [vp, vp, vp, vp, vp]
    lib.ocp_impec_pressure.argtypes = [vp, vp, ctypes.c_double, vp, vp, vp]
    lib.ocp_impec_update.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp]
    lib.ocp_bicgstab_scalar.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_int, vp,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), vp]
    lib.ocp_grid_update_perm.argtypes = [vp, vp, vp]
    lib.ocp_coupling_work_ints.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.ocp_coupling_work_ints.restype = ctypes.c_int64
    lib.ocp_coupling_components.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, vp, vp, vp]
    lib.ocp_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("ocp_last_error", "ocp_solver_work_doubles", "ocp_coupling_work_ints"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(st):
    if st != OCP_OK:
        raise OcpError(st, _lib.ocp_last_error().decode(errors="replace"))


def _ptr(t):
    return t.data_ptr() if t is not None else None


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(device, stream):
    """The CUDA stream handle for a call: the given torch stream, else the
    device's current one (read without building a Stream object)."""
    if stream is None:
        if _raw_stream is not None:
            return _raw_stream(device.index if device.index is not None else torch.cuda.current_device())
        stream = torch.cuda.current_stream(device)
    return stream.cuda_stream


class _DevView:
    """Zero-copy view of device memory owned by the library."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3}


def make_desc(desc):
    """The C descriptor of a ``workloads.GridDesc``-like object, and the host
    arrays it points into (keep them alive while the descriptor is used)."""
    keep = []

    def arr(a, dtype=np.float64):
        a = np.ascontiguousarray(a, dtype=dtype)
        keep.append(a)
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double if dtype == np.float64 else ctypes.c_int64))

    d = _Desc()
    for name in ("nx", "ny", "nz", "nphase"):
        setattr(d, name, int(getattr(desc, name)))
    for name in ("dx", "dy", "dz", "top_depth", "kz_over_kx", "cr", "p_ref", "bw_ref", "cw", "muw",
                 "rho_osc", "rho_gsc", "rho_wsc", "co_under", "cmu_under", "swc", "sorw", "sorg", "sgc",
                 "nw", "now", "ng", "nog", "krw_max", "krg_max", "kro_cw", "pcow_max", "pcgo_max"):
        setattr(d, name, float(getattr(desc, name)))
    d.lnk = arr(desc.lnk)
    d.phi = arr(desc.phi)
    d.nrow = len(desc.tab_p)
    for name in ("tab_p", "tab_Bo", "tab_Bg", "tab_Rs", "tab_muo", "tab_mug"):
        setattr(d, name, arr(getattr(desc, name)))
    wells = (_Well * max(1, len(desc.wells)))()
    keep.append(wells)
    for k, w in enumerate(desc.wells):
        wells[k].kind = int(w.kind)
        wells[k].phase = int(w.phase)
        wells[k].p_bh = float(w.p_bh)
        wells[k].rw = float(w.rw)
        wells[k].skin = float(w.skin)
        wells[k].nperf = len(w.cells)
        wells[k].cells = arr(w.cells, np.int64)
    d.nwell = len(desc.wells)
    d.wells = wells
    return d, keep


class Grid:
    """A grid on one CUDA device (``ocp_grid_create``); owns its device data."""

    def __init__(self, desc, device=0):
        lib = load()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        d, keep = make_desc(desc)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.ocp_grid_create(ctypes.byref(d), self.device.index or 0, ctypes.byref(h)))
        self._h = h
        del keep
        n, nb, nnzb = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
        _check(lib.ocp_grid_info(h, ctypes.byref(n), ctypes.byref(nb), ctypes.byref(nnzb)))
        self.N, self.nb, self.nnzb = n.value, nb.value, nnzb.value
        self.nwell = len(desc.wells)
        self.nperf = int(sum(len(w.cells) for w in desc.wells))

    def close(self):
        if getattr(self, "_h", None):
            load().ocp_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def _t(self, t, numel, dtype, name, allow_none=False):
        if t is None:
            if allow_none:
                return None
            raise ValueError("%s is required" % name)
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dtype:
            raise ValueError("%s must be a %s tensor on %s" % (name, dtype, self.device))
        if not t.is_contiguous() or t.numel() != numel:
            raise ValueError("%s must be contiguous with %d elements (got %d)" % (name, numel, t.numel()))
        return t

    def empty(self, n, dtype=torch.float64):
        return torch.empty(n, dtype=dtype, device=self.device)

    def pattern(self):
        """(row_ptr, col_idx): int32 device tensors holding copies of the grid's pattern."""
        rp, ci = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load().ocp_bsr_pattern(self._h, ctypes.byref(rp), ctypes.byref(ci)))
        row_ptr = torch.as_tensor(_DevView(rp.value, self.N + 1, "<i4"), device=self.device).clone()
        col_idx = torch.as_tensor(_DevView(ci.value, self.nnzb, "<i4"), device=self.device).clone()
        return row_ptr, col_idx

    # ------------------------------------------------------------ calls
    def _flags(self, flag_new, flag_old):
        """Phase-state flags: required with three phases; with two phases
        optional (unused by the library), each checked when given."""
        required = self.nb == 3
        self._t(flag_new, self.N, torch.int8, "flag_new", allow_none=not required)
        self._t(flag_old, self.N, torch.int8, "flag_old", allow_none=not required)

    def linearize(self, u_new, flag_new, u_old, flag_old, dt, residual=None, bsr_val=None,
                  face_flux=None, want_face_flux=False, stream=None):
        N, nb = self.N, self.nb
        self._t(u_new, nb * N, torch.float64, "u_new")
        self._t(u_old, nb * N, torch.float64, "u_old")
        self._flags(flag_new, flag_old)
        residual = residual if residual is not None else self.empty(nb * N)
        bsr_val = bsr_val if bsr_val is not None else self.empty(self.nnzb * nb * nb)
        if face_flux is None and want_face_flux:
            face_flux = self.empty(3 * nb * N)
        self._t(residual, nb * N, torch.float64, "residual")
        self._t(bsr_val, self.nnzb * nb * nb, torch.float64, "bsr_val")
        self._t(face_flux, 3 * nb * N, torch.float64, "face_flux", allow_none=True)
        _check(load().ocp_linearize(self._h, _ptr(u_new), _ptr(flag_new), _ptr(u_old), _ptr(flag_old),
                                    float(dt), _ptr(residual), _ptr(bsr_val), _ptr(face_flux),
                                    _stream(self.device, stream)))
        return residual, bsr_val, face_flux

    def linearize_noalloc(self, u_new, flag_new, u_old, flag_old, dt, residual, bsr_val, face_flux=None,
                          stream=None):
        """``ocp_linearize_noalloc``: the caller passes every output; the
        library's fixed scratch array is used (grids of at most 41 943 cells)."""
        N, nb = self.N, self.nb
        self._t(u_new, nb * N, torch.float64, "u_new")
        self._t(u_old, nb * N, torch.float64, "u_old")
        self._flags(flag_new, flag_old)
        self._t(residual, nb * N, torch.float64, "residual")
        self._t(bsr_val, self.nnzb * nb * nb, torch.float64, "bsr_val")
        self._t(face_flux, 3 * nb * N, torch.float64, "face_flux", allow_none=True)
        _check(load().ocp_linearize_noalloc(self._h, _ptr(u_new), _ptr(flag_new), _ptr(u_old), _ptr(flag_old),
                                            float(dt), _ptr(residual), _ptr(bsr_val), _ptr(face_flux),
                                            _stream(self.device, stream)))
        return residual, bsr_val, face_flux

    def spmv(self, bsr_val, x, alpha=1.0, beta=0.0, y=None, transpose=False, stream=None):
        n = self.nb * self.N
        self._t(bsr_val, self.nnzb * self.nb * self.nb, torch.float64, "bsr_val")
        self._t(x, n, torch.float64, "x")
        y = y if y is not None else self.empty(n)
        self._t(y, n, torch.float64, "y")
        _check(load().ocp_bsr_spmv(self._h, _ptr(bsr_val), float(alpha), _ptr(x), float(beta), _ptr(y),
                                   int(bool(transpose)), _stream(self.device, stream)))
        return y

    def adjoint_vjp(self, u_new, flag_new, u_old, flag_old, dt, bsr_val, face_flux, lam,
                    want=("unew", "uold", "lnk", "phi"), out=None, stream=None):
        N, nb = self.N, self.nb
        self._t(u_new, nb * N, torch.float64, "u_new")
        self._t(u_old, nb * N, torch.float64, "u_old")
        self._flags(flag_new, flag_old)
        self._t(lam, nb * N, torch.float64, "lambda")
        out = dict(out or {})
        sizes = {"unew": nb * N, "uold": nb * N, "lnk": N, "phi": N}
        for k in want:
            if k not in out:
                out[k] = self.empty(sizes[k])
            self._t(out[k], sizes[k], torch.float64, "g_" + k)
        _check(load().ocp_adjoint_vjp(self._h, _ptr(u_new), _ptr(flag_new), _ptr(u_old), _ptr(flag_old),
                                      float(dt), _ptr(bsr_val), _ptr(face_flux), _ptr(lam),
                                      _ptr(out.get("unew")), _ptr(out.get("uold")), _ptr(out.get("lnk")),
                                      _ptr(out.get("phi")), _stream(self.device, stream)))
        return out

    def well_rates(self, u, flag, q=None, stream=None):
        q = q if q is not None else self.empty(max(1, self.nwell) * self.nb)
        _check(load().ocp_well_rates(self._h, _ptr(u), _ptr(flag), _ptr(q), _stream(self.device, stream)))
        return q[: self.nwell * self.nb]

    def status(self, stream=None):
        """Synchronise and return the sticky device status (an int, 0 = OK)."""
        return load().ocp_get_status(self._h, _stream(self.device, stream))

    # ------------------------------------------------------------ Newton support
    def solver_work(self):
        return self.empty(int(load().ocp_solver_work_doubles(self._h)))

    def bicgstab(self, bsr_val, b, x, rtol, maxit, transpose=False, work=None, stream=None, check=True):
        """Solve A x = b (A^T x = b); x is the initial guess, updated in place.
        Returns (status, iterations, relative residual)."""
        work = work if work is not None else self.solver_work()
        it, rr = ctypes.c_int(), ctypes.c_double()
        st = load().ocp_bicgstab(self._h, _ptr(bsr_val), _ptr(b), _ptr(x), float(rtol), int(maxit),
                                 int(bool(transpose)), _ptr(work), ctypes.byref(it), ctypes.byref(rr),
                                 _stream(self.device, stream))
        if check:
            _check(st)
        return st, it.value, rr.value

    def newton_update(self, u, flag, du, scale, ds_max, du_max, nswitch, stream=None):
        _check(load().ocp_newton_update(self._h, _ptr(u), _ptr(flag), _ptr(du), float(scale), float(ds_max),
                                        _ptr(du_max), _ptr(nswitch), _stream(self.device, stream)))

    def well_rates_vjp(self, u, flag, q_bar, g_u=None, g_lnk=None, stream=None):
        _check(load().ocp_well_rates_vjp(self._h, _ptr(u), _ptr(flag), _ptr(q_bar), _ptr(g_u), _ptr(g_lnk),
                                         _stream(self.device, stream)))

    def update_perm(self, lnk, stream=None):
        self._t(lnk, self.N, torch.float64, "lnk")
        _check(load().ocp_grid_update_perm(self._h, _ptr(lnk), _stream(self.device, stream)))

    # ------------------------------------------------------------ wells as unknowns
    def linearize_wells(self, u_new, flag_new, u_old, flag_old, dt, p_bh, ctrl, out=None, want_face_flux=False,
                        stream=None):
        """``ocp_linearize_wells``.  Returns a dict with residual, bsr_val,
        face_flux (or None), well_res, well_b, well_c, well_d."""
        N, nb, nw, npf = self.N, self.nb, self.nwell, self.nperf
        self._t(u_new, nb * N, torch.float64, "u_new")
        self._t(u_old, nb * N, torch.float64, "u_old")
        self._flags(flag_new, flag_old)
        self._t(p_bh, nw, torch.float64, "p_bh")
        self._t(ctrl, 24 * nw, torch.uint8, "ctrl")
        o = dict(out or {})
        sizes = {"residual": nb * N, "bsr_val": self.nnzb * nb * nb, "well_res": max(nw, 1),
                 "well_b": max(npf, 1) * nb, "well_c": max(npf, 1) * nb, "well_d": max(nw, 1)}
        for k, n in sizes.items():
            if k not in o:
                o[k] = self.empty(n)
            self._t(o[k], n, torch.float64, k)
        if want_face_flux and o.get("face_flux") is None:
            o["face_flux"] = self.empty(3 * nb * N)
        ff = o.get("face_flux")
        self._t(ff, 3 * nb * N, torch.float64, "face_flux", allow_none=True)
        _check(load().ocp_linearize_wells(self._h, _ptr(u_new), _ptr(flag_new), _ptr(u_old), _ptr(flag_old),
                                          float(dt), _ptr(p_bh), _ptr(ctrl), _ptr(o["residual"]),
                                          _ptr(o["bsr_val"]), _ptr(ff), _ptr(o["well_res"]), _ptr(o["well_b"]),
                                          _ptr(o["well_c"]), _ptr(o["well_d"]), _stream(self.device, stream)))
        o["face_flux"] = ff
        return o

    def bicgstab_wells(self, bsr_val, well_b, well_c, well_d, b, b_w, x, x_w, rtol, maxit, transpose=False,
                       work=None, stream=None, check=True):
        """Solve [A B; C D][x; x_w] = [b; b_w] (transposed with ``transpose``)
        through the Schur complement of the well unknowns; x is the initial
        guess.  Returns (status, iterations, relative residual)."""
        work = work if work is not None else self.solver_work()
        it, rr = ctypes.c_int(), ctypes.c_double()
        st = load().ocp_bicgstab_wells(self._h, _ptr(bsr_val), _ptr(well_b), _ptr(well_c), _ptr(well_d), _ptr(b),
                                       _ptr(b_w), _ptr(x), _ptr(x_w), float(rtol), int(maxit),
                                       int(bool(transpose)), _ptr(work), ctypes.byref(it), ctypes.byref(rr),
                                       _stream(self.device, stream))
        if check:
            _check(st)
        return st, it.value, rr.value

    def well_update(self, p_bh, dp, scale, ctrl, dp_max, nswitch, stream=None):
        _check(load().ocp_well_update(self._h, _ptr(p_bh), _ptr(dp), float(scale), _ptr(ctrl), _ptr(dp_max),
                                      _ptr(nswitch), _stream(self.device, stream)))

    def residual_norms(self, residual, dt, well_res, ctrl, norms=None, stream=None):
        norms = norms if norms is not None else self.empty(4)
        _check(load().ocp_residual_norms(self._h, _ptr(residual), float(dt), _ptr(well_res), _ptr(ctrl),
                                         _ptr(norms), _stream(self.device, stream)))
        return norms

    # ------------------------------------------------------------ pressure and amounts
    def linearize_pn(self, pn_new, pn_old, dt, out=None, full=False, stream=None):
        """``ocp_linearize_pn``: the reduced system over (P, N_o[, N_g]) and
        the elimination coefficients; with ``full`` also the system with the
        volume rows.  Returns a dict (residual, bsr_val, elim, flag[,
        residual_full, bsr_val_full])."""
        N, nb, L = self.N, self.nb, self.nb + 1
        self._t(pn_new, L * N, torch.float64, "pn_new")
        self._t(pn_old, L * N, torch.float64, "pn_old")
        o = dict(out or {})
        sizes = {"residual": nb * N, "bsr_val": self.nnzb * nb * nb, "elim": L * N}
        if full:
            sizes.update(residual_full=L * N, bsr_val_full=self.nnzb * L * L)
        for k, n in sizes.items():
            if o.get(k) is None:
                o[k] = self.empty(n)
            self._t(o[k], n, torch.float64, k)
        if o.get("flag") is None:
            o["flag"] = torch.empty(N, dtype=torch.int8, device=self.device)
        self._t(o["flag"], N, torch.int8, "flag")
        _check(load().ocp_linearize_pn(self._h, _ptr(pn_new), _ptr(pn_old), float(dt), _ptr(o["residual"]),
                                       _ptr(o["bsr_val"]), _ptr(o["elim"]), _ptr(o.get("residual_full")),
                                       _ptr(o.get("bsr_val_full")), _ptr(o["flag"]), _stream(self.device, stream)))
        return o

    def pn_update(self, pn, dx, scale, elim, dx_max, stream=None):
        _check(load().ocp_pn_update(self._h, _ptr(pn), _ptr(dx), float(scale), _ptr(elim), _ptr(dx_max),
                                    _stream(self.device, stream)))

    def pn_from_natural(self, u, flag, pn=None, stream=None):
        """(P, N) of a natural state (``ocp_pn_from_natural``)."""
        pn = pn if pn is not None else self.empty((self.nb + 1) * self.N)
        self._t(u, self.nb * self.N, torch.float64, "u")
        _check(load().ocp_pn_from_natural(self._h, _ptr(u), _ptr(flag), _ptr(pn), _stream(self.device, stream)))
        return pn

    # ------------------------------------------------------------ IMPEC
    def impec_pressure(self, pn, dt, val=None, rhs=None, stream=None):
        """``ocp_impec_pressure``: (val [nnzb], rhs [N]) of the pressure system."""
        self._t(pn, (self.nb + 1) * self.N, torch.float64, "pn")
        val = val if val is not None else self.empty(self.nnzb)
        rhs = rhs if rhs is not None else self.empty(self.N)
        self._t(val, self.nnzb, torch.float64, "val")
        self._t(rhs, self.N, torch.float64, "rhs")
        _check(load().ocp_impec_pressure(self._h, _ptr(pn), float(dt), _ptr(val), _ptr(rhs),
                                         _stream(self.device, stream)))
        return val, rhs

    def impec_update(self, pn_old, dp, dt, pn_new=None, stream=None):
        pn_new = pn_new if pn_new is not None else self.empty((self.nb + 1) * self.N)
        self._t(dp, self.N, torch.float64, "dp")
        _check(load().ocp_impec_update(self._h, _ptr(pn_old), _ptr(dp), float(dt), _ptr(pn_new),
                                       _stream(self.device, stream)))
        return pn_new

    def bicgstab_scalar(self, val, b, x, rtol, maxit, work=None, stream=None, check=True):
        work = work if work is not None else self.solver_work()
        it, rr = ctypes.c_int(), ctypes.c_double()
        st = load().ocp_bicgstab_scalar(self._h, _ptr(val), _ptr(b), _ptr(x), float(rtol), int(maxit), _ptr(work),
                                        ctypes.byref(it), ctypes.byref(rr), _stream(self.device, stream))
        if check:
            _check(st)
        return st, it.value, rr.value

    def pn_norms(self, residual_full, dt, norms=None, stream=None):
        norms = norms if norms is not None else self.empty(4)
        _check(load().ocp_pn_norms(self._h, _ptr(residual_full), float(dt), _ptr(norms), _stream(self.device, stream)))
        return norms

    def coupling_components(self, u_new, flag_new, u_old, flag_old, threshold, px, py, pz, labels=None,
                            work=None, stream=None):
        """``ocp_coupling_components``: adaptive coupling of the px x py x pz
        subdomains (Sec. 4).  Returns (labels, work) device tensors: labels[s]
        is the smallest subdomain index of s's component, work[2 S] the number
        of marked cells, work[2 S + 1] the union-find retries and work[2 S + 2]
        an error flag (1 if a loop bound was reached; never expected)."""
        lib = load()
        N, nb = self.N, self.nb
        self._t(u_new, nb * N, torch.float64, "u_new")
        self._t(u_old, nb * N, torch.float64, "u_old")
        self._flags(flag_new, flag_old)
        S = int(px) * int(py) * int(pz)
        nwork = int(lib.ocp_coupling_work_ints(int(px), int(py), int(pz)))
        if S < 1 or nwork < 1:
            raise ValueError("subdomain counts must be positive")
        labels = labels if labels is not None else torch.empty(S, dtype=torch.int32, device=self.device)
        work = work if work is not None else torch.empty(nwork, dtype=torch.int32, device=self.device)
        self._t(labels, S, torch.int32, "labels")
        self._t(work, nwork, torch.int32, "work")
        _check(lib.ocp_coupling_components(self._h, _ptr(u_new), _ptr(flag_new), _ptr(u_old), _ptr(flag_old),
                                           float(threshold), int(px), int(py), int(pz), _ptr(labels), _ptr(work),
                                           _stream(self.device, stream)))
        return labels, work

    def set_shape(self, d):
        """Launch shape of ocp_linearize on this grid (``ocp_grid_set_shape``)."""
        _check(load().ocp_grid_set_shape(self._h, ctypes.byref(shape_from_dict(d))))

    def get_shape(self):
        sh = _Shape()
        _check(load().ocp_grid_get_shape(self._h, ctypes.byref(sh)))
        return shape_to_dict(sh)

    def cluster_tiles(self):
        """Largest grid, in 32-cell tiles, that the one-cluster launch
        (``ordered = 4``) takes on this grid's device; 0 if none."""
        n = ctypes.c_int()
        _check(load().ocp_grid_cluster_tiles(self._h, ctypes.byref(n)))
        return n.value


def shape_to_dict(sh):
    return {"cells_per_tile": list(sh.cells_per_tile), "ctas_per_sm": list(sh.ctas_per_sm), "ordered": sh.ordered}


def shape_from_dict(d):
    sh = _Shape()
    for q in range(3):
        sh.cells_per_tile[q] = int(d["cells_per_tile"][q])
        sh.ctas_per_sm[q] = int(d["ctas_per_sm"][q])
    sh.ordered = int(d.get("ordered", 0))
    return sh


class Batch:
    """An ensemble of grids linearised together (``ocp_batch_*``)."""

    def __init__(self, grids):
        lib = load()
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g._h.value for g in self.grids])
        h = ctypes.c_void_p()
        _check(lib.ocp_batch_create(arr, len(self.grids), ctypes.byref(h)))
        self._h = h
        self.device = self.grids[0].device

    def close(self):
        if getattr(self, "_h", None):
            load().ocp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_io(self, ios):
        """ios: one dict per grid with u_new, flag_new, u_old, flag_old,
        residual, bsr_val[, face_flux] device tensors."""
        arr = (_BatchIO * len(self.grids))()
        self._io = ios
        for k, (g, io) in enumerate(zip(self.grids, ios)):
            nb, N = g.nb, g.N
            g._t(io["u_new"], nb * N, torch.float64, "u_new")
            g._t(io["u_old"], nb * N, torch.float64, "u_old")
            g._t(io["residual"], nb * N, torch.float64, "residual")
            g._t(io["bsr_val"], g.nnzb * nb * nb, torch.float64, "bsr_val")
            g._t(io.get("face_flux"), 3 * nb * N, torch.float64, "face_flux", allow_none=True)
            for name in _BatchIO._fields_:
                t = io.get(name[0])
                setattr(arr[k], name[0], t.data_ptr() if t is not None else None)
        _check(load().ocp_batch_set_io(self._h, arr))

    def linearize(self, dt, graph=False, stream=None):
        f = load().ocp_batch_graph_launch if graph else load().ocp_batch_linearize
        _check(f(self._h, float(dt), _stream(self.device, stream)))

    def tune(self, dt, reps=3, stream=None):
        sh = _Shape()
        _check(load().ocp_batch_tune(self._h, float(dt), int(reps), ctypes.byref(sh), _stream(self.device, stream)))
        return shape_to_dict(sh)

    def set_shape(self, d):
        _check(load().ocp_batch_set_shape(self._h, ctypes.byref(shape_from_dict(d))))

    def get_shape(self):
        sh = _Shape()
        _check(load().ocp_batch_get_shape(self._h, ctypes.byref(sh)))
        return shape_to_dict(sh)

    def status(self, stream=None):
        return load().ocp_batch_get_status(self._h, _stream(self.device, stream))


def probe_fp64(device=0, reps=3):
    """Sustained FP64 FMA rate of the device in GFLOP/s (``ocp_probe_fp64``)."""
    lib = load()
    r = ctypes.c_double()
    _check(lib.ocp_probe_fp64(int(device), int(reps), ctypes.byref(r)))
    return 2.0 * r.value / 1e9

