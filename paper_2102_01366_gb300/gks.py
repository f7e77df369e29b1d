"""Thin ctypes binding of libgks (include/gks.h), same names as the C ABI.

Argument marshalling only: every step of the scheme runs in libgks.  PyTorch
supplies device memory (the workspace and the state tensors) and the CUDA
stream.  There is no fallback: if libgks.so is missing or fails to load, every
entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgks.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gks.h")

GKS_OK = 0
STATUS = {0: "GKS_OK", -1: "GKS_E_ARG", -2: "GKS_E_MESH", -3: "GKS_E_STENCIL", -4: "GKS_E_STATE",
          -5: "GKS_E_CUDA", -6: "GKS_E_TIMEOUT", -7: "GKS_E_NOMEM", -8: "GKS_E_UNSUPPORTED"}


class GksError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__("%s -> %s: %s" % (fn, STATUS.get(status, status), msg))
        self.status = status


class gks_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("mu", C.c_double),
                ("eps_weno", C.c_double), ("tau_eps", C.c_double), ("tau_c", C.c_double),
                ("prandtl", C.c_double), ("wall_temperature", C.c_double), ("wall_velocity", C.c_double * 3),
                ("weno", C.c_int32), ("order", C.c_int32), ("smooth_flux", C.c_int32),
                ("viscous", C.c_int32), ("precision", C.c_int32), ("wall_constraint", C.c_int32)]


_lib = None
_vp = C.c_void_p
_i64p = C.POINTER(C.c_int64)


def header_functions():
    """Names of the functions declared in include/gks.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gks_[a-z0-9_]+)\s*\(", src)))


def lib():
    """Load libgks.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libgks.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    sig = {
        "gks_params_default": (None, [C.POINTER(gks_params)]),
        "gks_last_error": (C.c_char_p, []),
        "gks_mesh_create": (C.c_int32, [_vp, C.c_int64, _vp, _vp, C.c_int64, _vp, C.POINTER(_vp)]),
        "gks_mesh_create_cases": (C.c_int32, [_vp, C.c_int64, _vp, _vp, C.c_int64, _vp, C.c_int32, _vp,
                                              C.POINTER(_vp)]),
        "gks_mesh_cases": (C.c_int32, [_vp, C.POINTER(C.c_int32), _vp]),
        "gks_mesh_set_boundary": (C.c_int32, [_vp, _vp]),
        "gks_case_times": (C.c_int32, [_vp, _vp, _vp]),
        "gks_mesh_destroy": (None, [_vp]),
        "gks_mesh_info": (C.c_int32, [_vp, _i64p, _i64p, _i64p]),
        "gks_mesh_topology": (C.c_int32, [_vp] * 6),
        "gks_mesh_geometry": (C.c_int32, [_vp] * 9),
        "gks_stencil_build": (C.c_int32, [_vp, _i64p]),
        "gks_mesh_stencils": (C.c_int32, [_vp, _vp, _vp]),
        "gks_mesh_wall_stencils": (C.c_int32, [_vp, _vp, _vp, _vp, _vp]),
        "gks_workspace_bytes": (C.c_size_t, [_vp, C.POINTER(gks_params)]),
        "gks_state_create": (C.c_int32, [_vp, C.POINTER(gks_params), _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
        "gks_state_destroy": (None, [_vp]),
        "gks_init_state": (C.c_int32, [_vp, _vp, _vp]),
        "gks_step": (C.c_int32, [_vp, C.c_int32, C.c_double, C.c_double]),
        "gks_sync": (C.c_int32, [_vp]),
        "gks_get_state": (C.c_int32, [_vp, _vp, _vp]),
        "gks_get_time": (C.c_int32, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "gks_step_host": (C.c_int32, [_vp, _vp, _vp, C.c_int32, C.c_double, _vp, _vp]),
        "gks_timestep": (C.c_int32, [_vp, C.POINTER(C.c_double)]),
        "gks_step_timed": (C.c_int32, [_vp, C.c_int32, C.c_double, C.c_double, _vp, _vp]),
        "gks_timestep_noalloc": (C.c_int32, [C.POINTER(gks_params), _vp, _vp, C.c_int64, _vp, _vp]),
        "gks_residual": (C.c_int32, [_vp, _vp]),
        "gks_adjoint_workspace_bytes": (C.c_size_t, [_vp]),
        "gks_set_fixed_state": (C.c_int32, [_vp, _vp, _vp]),
        "gks_adjoint_step": (C.c_int32, [_vp, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t]),
        "gks_adjoint_step_staged": (C.c_int32, [_vp, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                                C.c_size_t]),
        "gks_get_stage_state": (C.c_int32, [_vp, _vp, _vp]),
        "gks_debug_reconstruct": (C.c_int32, [_vp, _vp, _vp, _vp]),
        "gks_debug_face_records": (C.c_int32, [_vp, C.c_double, C.c_int32, _vp]),
        "gks_debug_wait_timeout": (C.c_int32, [_vp, C.c_int32]),
        "gks_debug_grid_barrier_timeout": (C.c_int32, [_vp, C.c_int32]),
        "gks_state_set_variant": (C.c_int32, [_vp, C.c_int32, C.c_int32, C.c_int32]),
        "gks_state_set_fused": (C.c_int32, [_vp, C.c_int32]),
        "gks_state_get_fused": (C.c_int32, [_vp, _vp]),
        "gks_autotune": (C.c_int32, [_vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32), _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _call(name, *args):
    st = getattr(lib(), name)(*args)
    if st != GKS_OK:
        raise GksError(name, st, lib().gks_last_error().decode())
    return st


def _np_ptr(a):
    return a.ctypes.data_as(_vp) if a is not None else None


def params(gamma=1.4, cfl=1.0, mu=0.0, eps_weno=1e-8, tau_eps=0.01, tau_c=1.0, weno=1, order=3,
           smooth_flux=0, viscous=0, precision=0, prandtl=1.0, wall_temperature=1.0, wall_velocity=(0.0, 0.0, 0.0),
           wall_constraint=0):
    p = gks_params()
    lib().gks_params_default(C.byref(p))
    p.gamma, p.cfl, p.mu, p.eps_weno, p.tau_eps, p.tau_c = gamma, cfl, mu, eps_weno, tau_eps, tau_c
    p.prandtl = prandtl
    p.wall_temperature = wall_temperature
    for i in range(3):
        p.wall_velocity[i] = float(wall_velocity[i])
    p.weno, p.order, p.smooth_flux, p.viscous, p.precision = weno, order, smooth_flux, viscous, precision
    p.wall_constraint = wall_constraint
    return p


class Mesh:
    """gks_mesh: connectivity, FP64 geometry and stencils (host object)."""

    def __init__(self, mesh, build_stencils=True):
        self._h = _vp()
        xyz = np.ascontiguousarray(mesh["xyz"], dtype=np.float64)
        tet = np.ascontiguousarray(mesh["tet"], dtype=np.int64)
        shift = np.ascontiguousarray(mesh["shift"], dtype=np.int8)
        period = np.ascontiguousarray(mesh["period"], dtype=np.float64)
        if "case" in mesh:
            case = np.ascontiguousarray(mesh["case"], dtype=np.int32)
            _call("gks_mesh_create_cases", _np_ptr(xyz), xyz.shape[0], _np_ptr(tet), _np_ptr(shift),
                  tet.shape[0], _np_ptr(case), int(mesh["ncase"]), _np_ptr(period), C.byref(self._h))
        else:
            _call("gks_mesh_create", _np_ptr(xyz), xyz.shape[0], _np_ptr(tet), _np_ptr(shift),
                  tet.shape[0], _np_ptr(period), C.byref(self._h))
        nc, nf, nb = C.c_int64(), C.c_int64(), C.c_int64()
        _call("gks_mesh_info", self._h, C.byref(nc), C.byref(nf), C.byref(nb))
        self.nc, self.nf, self.n_boundary = nc.value, nf.value, nb.value
        ncase = C.c_int32()
        _call("gks_mesh_cases", self._h, C.byref(ncase), None)
        self.ncase = ncase.value
        self.case_first = np.zeros(self.ncase + 1, np.int64)
        _call("gks_mesh_cases", self._h, C.byref(ncase), _np_ptr(self.case_first))
        self.n_singular = None
        if mesh.get("bkind") is not None:
            self.set_boundary(mesh["bkind"])
        if build_stencils:
            ns = C.c_int64()
            _call("gks_stencil_build", self._h, C.byref(ns))
            self.n_singular = ns.value

    def set_boundary(self, kind):
        """kind[nc][4] per local face (GKS_BC_OPEN 0, GKS_BC_SLIP_WALL 1,
        GKS_BC_FIXED 2, GKS_BC_NOSLIP_WALL 3); read on boundary faces only;
        applies to states created afterwards."""
        kind = np.ascontiguousarray(kind, dtype=np.int8).reshape(self.nc, 4)
        _call("gks_mesh_set_boundary", self._h, _np_ptr(kind))

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.gks_mesh_destroy(self._h)
            self._h = _vp()

    def topology(self):
        nc, nf = self.nc, self.nf
        out = dict(face_v=np.zeros((nf, 3), np.int64), face_lr=np.zeros((nf, 2), np.int64),
                   nbr=np.zeros((nc, 4), np.int64), csr_face=np.zeros((nc, 4), np.int64),
                   csr_sign=np.zeros((nc, 4), np.int8))
        _call("gks_mesh_topology", self._h, *[_np_ptr(out[k]) for k in
                                              ("face_v", "face_lr", "nbr", "csr_face", "csr_sign")])
        return out

    def geometry(self):
        nc, nf = self.nc, self.nf
        out = dict(vol=np.zeros(nc), cen=np.zeros((nc, 3)), mom2=np.zeros((nc, 6)), dr=np.zeros(nc),
                   farea=np.zeros(nf), fnorm=np.zeros((nf, 3)), gp_l=np.zeros((nf, 3, 3)),
                   gp_r=np.zeros((nf, 3, 3)))
        _call("gks_mesh_geometry", self._h, *[_np_ptr(out[k]) for k in
                                              ("vol", "cen", "mom2", "dr", "farea", "fnorm", "gp_l", "gp_r")])
        return out

    def stencils(self):
        M1 = np.zeros((self.nc, 3, 4))
        M2 = np.zeros((self.nc, 9, 16))
        _call("gks_mesh_stencils", self._h, _np_ptr(M1), _np_ptr(M2))
        return M1, M2

    def wall_stencils(self):
        """Sec. 4.4 constrained operators of the non-slip wall cells:
        (W1[nc][3][5], W2[nc][9][17], built[nc]) (gks_mesh_wall_stencils)."""
        W1 = np.zeros((self.nc, 3, 5))
        W2 = np.zeros((self.nc, 9, 17))
        built = np.zeros(self.nc, np.int8)
        n = C.c_int64()
        _call("gks_mesh_wall_stencils", self._h, _np_ptr(W1), _np_ptr(W2), _np_ptr(built), C.byref(n))
        return W1, W2, built


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class State:
    """gks_state over a torch-allocated device workspace and a torch stream."""

    def __init__(self, mesh: Mesh, p: gks_params, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.mesh = mesh
        self.params = p
        self.variant = (0, 3, 0)  # the library default: canonical faces, 3 flux blocks per SM, fused slopes
        self.cell_order = 0  # the caller's cell order
        self.device = torch.device(device)
        nbytes = lib().gks_workspace_bytes(mesh._h, C.byref(p))
        if nbytes == 0:
            raise GksError("gks_workspace_bytes", -1, lib().gks_last_error().decode())
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws_ptr = self.workspace.data_ptr() + off
        self.workspace_bytes = nbytes
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self._h = _vp()
        with torch.cuda.device(self.device):
            _call("gks_state_create", mesh._h, C.byref(p), C.c_void_p(self._ws_ptr), nbytes,
                  C.c_void_p(self.stream.cuda_stream), C.byref(self._h))

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.gks_state_destroy(self._h)
            self._h = _vp()

    # -- state --------------------------------------------------------------
    def init(self, W, dW):
        """W [5, nc], dW [15, nc] float64 (numpy or torch)."""
        t = self.torch
        W = t.as_tensor(np.ascontiguousarray(W) if isinstance(W, np.ndarray) else W,
                        dtype=t.float64, device=self.device).contiguous()
        dW = t.as_tensor(np.ascontiguousarray(dW) if isinstance(dW, np.ndarray) else dW,
                         dtype=t.float64, device=self.device).contiguous()
        assert W.shape == (5, self.mesh.nc) and dW.shape == (15, self.mesh.nc)
        self.stream.wait_stream(t.cuda.current_stream(self.device))
        _call("gks_init_state", self._h, _dptr(W), _dptr(dW))
        self._keep = (W, dW)  # alive until the stream has consumed them
        self.sync()
        self._keep = None

    def step(self, nsteps=1, dt_fixed=0.0, t_end=0.0):
        _call("gks_step", self._h, int(nsteps), float(dt_fixed), float(t_end))

    def sync(self):
        _call("gks_sync", self._h)

    def get(self):
        """(W [5, nc], dW [15, nc]) as float64 torch tensors."""
        t = self.torch
        W = t.empty((5, self.mesh.nc), dtype=t.float64, device=self.device)
        dW = t.empty((15, self.mesh.nc), dtype=t.float64, device=self.device)
        _call("gks_get_state", self._h, _dptr(W), _dptr(dW))
        self.sync()
        return W, dW

    def time(self):
        tt, dt = C.c_double(), C.c_double()
        _call("gks_get_time", self._h, C.byref(tt), C.byref(dt))
        return tt.value, dt.value

    KERNELS = ("dt", "slopes", "recon", "flux1", "update1", "flux2", "update2", "stage1", "stage2")

    def step_timed(self, nsteps=1, dt_fixed=0.0, t_end=0.0):
        """Kernel-by-kernel steps with CUDA events between launches; returns
        {kernel class: (total ms, launches)}."""
        ms = np.zeros(len(self.KERNELS))
        cnt = np.zeros(len(self.KERNELS), np.int64)
        _call("gks_step_timed", self._h, int(nsteps), float(dt_fixed), float(t_end), _np_ptr(ms), _np_ptr(cnt))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.KERNELS)}

    def case_times(self):
        """(t[ncase], dt_last[ncase]) of every case."""
        t = np.zeros(self.mesh.ncase)
        dt = np.zeros(self.mesh.ncase)
        _call("gks_case_times", self._h, _np_ptr(t), _np_ptr(dt))
        return t, dt

    def timestep(self):
        dt = C.c_double()
        _call("gks_timestep", self._h, C.byref(dt))
        return dt.value

    def residual(self):
        out = np.zeros(5)
        _call("gks_residual", self._h, _np_ptr(out))
        return out

    def set_fixed_state(self, W, dW):
        """The state fixed boundary faces hold from now on, [5|15, nc] FP64
        (gks_set_fixed_state); later init() calls keep it."""
        t = self.torch
        args = [t.as_tensor(x, dtype=t.float64, device=self.device).contiguous() for x in (W, dW)]
        self.stream.wait_stream(t.cuda.current_stream(self.device))
        _call("gks_set_fixed_state", self._h, *[_dptr(x) for x in args])

    def stage_state(self):
        """(W*, grad W*) of the last step's first stage (gks_get_stage_state;
        FP64 states)."""
        t = self.torch
        Ws = t.empty((5, self.mesh.nc), dtype=t.float64, device=self.device)
        dWs = t.empty((15, self.mesh.nc), dtype=t.float64, device=self.device)
        self.stream.wait_stream(t.cuda.current_stream(self.device))
        _call("gks_get_stage_state", self._h, _dptr(Ws), _dptr(dWs))
        return Ws, dWs

    def adjoint_step(self, W, dW, lamW, lamdW, dt, stage=None):
        """Adjoint of one step at (W, dW) with the frozen step dt
        (gks_adjoint_step): returns d J / d (W, dW) given d J / d (W', dW') of
        the step's result.  All [5|15, nc] float64 CUDA tensors; the state is
        left initialised at (W, dW).  stage: the step's (W*, grad W*) from
        stage_state() after that step (gks_adjoint_step_staged: the same
        result without recomputing the first stage's flux and update)."""
        t = self.torch
        args = [t.as_tensor(x, dtype=t.float64, device=self.device).contiguous() for x in (W, dW, lamW, lamdW)]
        if stage is not None:
            args = args[:2] + [t.as_tensor(x, dtype=t.float64, device=self.device).contiguous()
                               for x in stage] + args[2:]
        oW = t.empty((5, self.mesh.nc), dtype=t.float64, device=self.device)
        odW = t.empty((15, self.mesh.nc), dtype=t.float64, device=self.device)
        nbytes = lib().gks_adjoint_workspace_bytes(self._h)
        if getattr(self, "_adj_ws", None) is None or self._adj_ws.numel() < nbytes:
            self._adj_ws = t.empty(nbytes, dtype=t.uint8, device=self.device)
        self.stream.wait_stream(t.cuda.current_stream(self.device))
        _call("gks_adjoint_step" if stage is None else "gks_adjoint_step_staged", self._h, float(dt),
              *[_dptr(x) for x in args], _dptr(oW), _dptr(odW), _dptr(self._adj_ws), nbytes)
        return oW, odW

    def step_host(self, W_host, dW_host, nsteps=1, dt_fixed=0.0, W_out=None, dW_out=None):
        """Host buffers in and out (torch CPU tensors, pinned for async copies)."""
        W_out = W_host if W_out is None else W_out
        dW_out = dW_host if dW_out is None else dW_out
        _call("gks_step_host", self._h, C.c_void_p(W_host.data_ptr()), C.c_void_p(dW_host.data_ptr()),
              int(nsteps), float(dt_fixed), C.c_void_p(W_out.data_ptr()), C.c_void_p(dW_out.data_ptr()))
        return W_out, dW_out

    def run(self, nsteps=None, t_end=None, dt_fixed=0.0, chunk=64):
        """Advance nsteps, or until t_end (polling the device time per chunk)."""
        if t_end is None:
            self.step(nsteps, dt_fixed, 0.0)
            self.sync()
            return self.time()[0]
        while True:
            self.step(chunk, dt_fixed, t_end)
            self.sync()
            tt, dt = self.case_times()
            if (tt >= t_end * (1 - 1e-14)).all() or (dt <= 0.0).all():
                return float(tt.min())

    # -- tuning ----------------------------------------------------------------
    def set_variant(self, face_order, flux_blocks, slopes_pass=0):
        _call("gks_state_set_variant", self._h, int(face_order), int(flux_blocks), int(slopes_pass))
        self.variant = (int(face_order), int(flux_blocks), int(slopes_pass))

    NVARIANTS = 10  # variants gks_autotune times: 8 with separate kernels, 2 with one launch per stage

    def set_fused(self, fused=True):
        """Each stage as one persistent launch (precision 1 only; results are
        bit-identical to the separate kernels; gks_state_set_fused)."""
        _call("gks_state_set_fused", self._h, int(bool(fused)))

    def fused(self):
        v = C.c_int32()
        _call("gks_state_get_fused", self._h, C.byref(v))
        return int(v.value)

    def set_cell_order(self, order):
        """Device cell ordering (FP32 bulk): 0 the caller's, 1 reverse
        Cuthill-McKee, 2 Morton; results are unchanged (gks_state_set_cell_order)."""
        _call("gks_state_set_cell_order", self._h, int(order))
        self.cell_order = int(order)

    def _tune_key(self):
        p = self.params
        name = self.torch.cuda.get_device_name(self.device)
        return "%s|nc=%d|nf=%d|ncase=%d|prec=%d|weno=%d|order=%d|smooth=%d|visc=%d" % (
            name, self.mesh.nc, self.mesh.nf, self.mesh.ncase, p.precision, p.weno, p.order,
            p.smooth_flux, p.viscous)

    def autotune(self, steps=10, cache=None, orders=False):
        """Choose the fastest execution variant for this mesh and options by
        timing them (gks_autotune; with ``orders`` also over the cell
        orderings, gks_autotune_orders); results are cached in a JSON file
        keyed by GPU name, mesh size and options (``cache``: path, None for
        the default ~/.cache/paper_2102_01366_gb300/autotune.json, False for
        no cache)."""
        import json
        if cache is None:
            cache = os.environ.get("GKS_AUTOTUNE_CACHE", os.path.join(
                os.path.expanduser("~"), ".cache", "paper_2102_01366_gb300", "autotune.json"))
        key = self._tune_key() + ("|orders" if orders else "")
        table = {}
        if cache and os.path.exists(cache):
            try:
                table = json.load(open(cache))
            except (OSError, ValueError):
                table = {}
        if key in table and len(table[key].get("variant", ())) == 3 and "fused" in table[key]:
            if orders and "cell_order" in table[key]:
                self.set_cell_order(table[key]["cell_order"])
            self.set_variant(*table[key]["variant"])
            if self.params.precision == 1 or table[key]["fused"]:
                self.set_fused(table[key]["fused"])
            return dict(table[key], cached=True)
        fo, fb, sp = C.c_int32(), C.c_int32(), C.c_int32()
        if orders:
            co = C.c_int32()
            ms = np.zeros(3)
            _call("gks_autotune_orders", self._h, int(steps), C.byref(co), C.byref(fo), C.byref(fb), C.byref(sp),
                  _np_ptr(ms))
            self.cell_order = co.value
            self.variant = (fo.value, fb.value, sp.value)
            res = {"variant": list(self.variant), "cell_order": co.value, "fused": self.fused(),
                   "ms_per_order": ms[:3 if self.params.precision != 0 else 1].tolist()}
        else:
            ms = np.zeros(self.NVARIANTS)
            _call("gks_autotune", self._h, int(steps), C.byref(fo), C.byref(fb), C.byref(sp), _np_ptr(ms))
            self.variant = (fo.value, fb.value, sp.value)
            res = {"variant": list(self.variant), "fused": self.fused(),
                   "ms_per_step": [None if np.isnan(x) else float(x) for x in ms]}
        if cache:
            try:
                os.makedirs(os.path.dirname(cache), exist_ok=True)
                table[key] = res
                tmp = cache + ".tmp%d" % os.getpid()
                json.dump(table, open(tmp, "w"), indent=1)
                os.replace(tmp, cache)
            except OSError:
                pass
        return dict(res, cached=False)

    # -- diagnostics ----------------------------------------------------------
    def debug_reconstruct(self):
        t = self.torch
        nc = self.mesh.nc
        poly = t.empty((nc, 5, 10), dtype=t.float64, device=self.device)
        slopes = t.empty((nc, 5, 3), dtype=t.float64, device=self.device)
        fb = t.empty((nc,), dtype=t.int32, device=self.device)
        _call("gks_debug_reconstruct", self._h, _dptr(poly), _dptr(slopes), _dptr(fb))
        self.sync()
        return poly, slopes, fb

    def debug_wait_timeout(self, tries=8):
        """Status of a bounded device wait that gives up (gks_debug_wait_timeout)."""
        return lib().gks_debug_wait_timeout(self._h, int(tries))

    def debug_grid_barrier_timeout(self, tries=8):
        """Status of the one-launch stage's grid barrier giving up
        (gks_debug_grid_barrier_timeout)."""
        return lib().gks_debug_grid_barrier_timeout(self._h, int(tries))

    def debug_face_records(self, dt, stage):
        t = self.torch
        rec = t.empty((self.mesh.nf, 40 if stage == 1 else 20), dtype=t.float64, device=self.device)
        _call("gks_debug_face_records", self._h, float(dt), int(stage), _dptr(rec))
        self.sync()
        return rec


def make_step_function(state, dt):
    """A torch.autograd.Function for one step of ``state`` with the frozen
    step dt: forward runs gks_step from (W, dW), backward gks_adjoint_step
    (the forward state is recomputed, so only each step's input is kept).
    Chaining N applications differentiates an N-step run."""
    torch = state.torch

    class _Step(torch.autograd.Function):
        @staticmethod
        def forward(ctx, W, dW):
            state.init(W.detach(), dW.detach())
            state.step(1, float(dt), 0.0)
            Wn, dWn = state.get()
            ctx.start = (W.detach().clone(), dW.detach().clone())
            return Wn, dWn

        @staticmethod
        def backward(ctx, gW, gdW):
            W, dW = ctx.start
            gW = torch.zeros_like(W) if gW is None else gW
            gdW = torch.zeros_like(dW) if gdW is None else gdW
            return state.adjoint_step(W, dW, gW, gdW, dt)

    return _Step.apply


def wall_pressure_force(mesh, kinds, gamma=1.4, wall=(1, 3), device="cuda"):
    """A differentiable output for gradients: the pressure force on the wall
    faces, sum over faces of p A n, with p the pressure of the adjacent
    cell's average and n the face's unit normal pointing out of the fluid
    (first order in the cell size).  mesh: a Mesh; kinds[nc][4] the boundary
    kinds per local face (wall = slip 1 and non-slip 3 by default).  Returns
    a torch function of W [5, nc] (FP64) giving the 3-vector."""
    import torch
    top, geo = mesh.topology(), mesh.geometry()
    kinds = np.asarray(kinds).reshape(mesh.nc, 4)
    on = (top["nbr"] < 0) & np.isin(kinds, wall)
    cells, lf = np.nonzero(on)
    faces = top["csr_face"][cells, lf]
    sign = top["csr_sign"][cells, lf].astype(np.float64)
    an = geo["farea"][faces, None] * geo["fnorm"][faces] * sign[:, None]
    cells_t = torch.as_tensor(cells, device=device)
    an_t = torch.as_tensor(an, device=device)

    def force(W):
        Wc = W[:, cells_t]
        p = (gamma - 1.0) * (Wc[4] - 0.5 * (Wc[1:4] ** 2).sum(0) / Wc[0])
        return (p[:, None] * an_t).sum(0)
    return force


def checkpoint_interval(nc, nsteps, device="cuda", fraction=0.5, per_cell=160):
    """The checkpoint spacing checkpointed_gradient uses by default: 1 (keep
    every state, no recomputation) when the nsteps saved states (per_cell
    bytes a cell each: 160 for an FP64 state, 320 with its stage state) fit
    in `fraction` of the device's free memory, else the smallest spacing
    whose checkpoints plus one segment do."""
    import torch
    per_state = int(per_cell) * int(nc)
    free = torch.cuda.mem_get_info(torch.device(device))[0] if str(device).startswith("cuda") else 1 << 40
    budget = fraction * free
    for every in range(1, max(1, nsteps) + 1):
        if (nsteps // every + every) * per_state <= budget:
            return every
    return max(1, nsteps)


def checkpointed_gradient(mesh, params, W0, dW0, nsteps, dt, loss, checkpoint_every=None, primal_precision=0,
                          device="cuda"):
    """Gradient of loss(W_N) after N steps of frozen step dt with respect to
    the initial (W0, dW0), by the adjoint with checkpointing: the primal run
    keeps every `checkpoint_every`-th state (in FP64, on the device), the
    reverse sweep recomputes each segment from its checkpoint in FP64 and
    applies gks_adjoint_step backwards through it, so the memory is one
    segment plus the checkpoints.  checkpoint_every None: the spacing of
    checkpoint_interval (every step where the states fit in memory, so that
    nothing is recomputed beyond what each adjoint step recomputes itself).
    With every step kept and an FP64 primal, each step's stage state (W*,
    grad W*) is kept as well and handed to the adjoint step, which then
    skips the first stage's flux and update (the gradient is unchanged).

    loss: a torch function of the final W [5, nc] (FP64 tensor) returning a
    scalar.  primal_precision 1 runs the primal in FP32 bulk (the checkpoints
    are its FP64 master states); the reverse sweep is FP64 either way, so the
    gradient then belongs to FP64 segments restarted from FP32-run
    checkpoints.  device: where the inputs, checkpoints and adjoints are
    kept (the library's states live on the GPU).  Returns (loss value,
    dJ/dW0, dJ/d dW0)."""
    import torch
    if not isinstance(mesh, Mesh):
        mesh = Mesh(mesh)
    p64 = gks_params()
    C.memmove(C.byref(p64), C.byref(params), C.sizeof(gks_params))
    p64.precision = 0
    s64 = State(mesh, p64)
    primal = s64
    if primal_precision:
        pp = gks_params()
        C.memmove(C.byref(pp), C.byref(params), C.sizeof(gks_params))
        pp.precision = 1
        primal = State(mesh, pp)
    W = torch.as_tensor(np.ascontiguousarray(W0) if isinstance(W0, np.ndarray) else W0,
                        dtype=torch.float64, device=device)
    dW = torch.as_tensor(np.ascontiguousarray(dW0) if isinstance(dW0, np.ndarray) else dW0,
                         dtype=torch.float64, device=device)
    if checkpoint_every is None:
        checkpoint_every = checkpoint_interval(mesh.nc, nsteps, device, per_cell=160 if primal_precision else 320)
    staged = checkpoint_every == 1 and not primal_precision
    stages = {}
    checkpoints = {0: (W.clone(), dW.clone())}
    primal.init(W, dW)
    for n in range(1, nsteps + 1):
        primal.step(1, float(dt), 0.0)
        if staged:
            stages[n - 1] = primal.stage_state()
        if n % checkpoint_every == 0 and n < nsteps:
            checkpoints[n] = primal.get()
    primal.sync()
    Wn, _ = primal.get()
    Wn = Wn.clone().requires_grad_(True)
    J = loss(Wn)
    J.backward()
    lam_W = Wn.grad.detach().clone()
    lam_dW = torch.zeros((15, mesh.nc), dtype=torch.float64, device=device)
    starts = sorted(checkpoints)
    for k in reversed(range(len(starts))):
        n0 = starts[k]
        n1 = starts[k + 1] if k + 1 < len(starts) else nsteps
        Wc, dWc = checkpoints[n0]
        segment = [(Wc, dWc)]
        if n1 - n0 > 1:  # (each adjoint step initialises the state itself)
            s64.init(Wc, dWc)
            for _ in range(n0 + 1, n1):
                s64.step(1, float(dt), 0.0)
                segment.append(s64.get())
        for Ws, dWs in reversed(segment):
            if staged:
                lam_W, lam_dW = s64.adjoint_step(Ws, dWs, lam_W, lam_dW, dt, stage=stages.pop(n0))
            else:
                lam_W, lam_dW = s64.adjoint_step(Ws, dWs, lam_W, lam_dW, dt)
    return float(J.detach()), lam_W, lam_dW
