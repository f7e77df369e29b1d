"""ctypes driver of the plain FP64 CPU oracle (gks_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are its only users; the CUDA library never calls
it.  ``build()`` compiles the C source with gcc next to this file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gks_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle (plain C11, FP64, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "gks_oracle.h"))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("mu", C.c_double),
                ("eps_weno", C.c_double), ("tau_eps", C.c_double), ("tau_c", C.c_double),
                ("weno", C.c_int32), ("order", C.c_int32), ("smooth_flux", C.c_int32),
                ("viscous", C.c_int32), ("prandtl", C.c_double), ("wall_temperature", C.c_double),
                ("wall_velocity", C.c_double * 3), ("wall_constraint", C.c_int32)]


def params(gamma=1.4, cfl=0.5, mu=0.0, eps_weno=1e-8, tau_eps=0.01, tau_c=1.0, weno=0,
           order=3, smooth_flux=0, viscous=0, prandtl=1.0, wall_temperature=1.0, wall_velocity=(0.0, 0.0, 0.0),
           wall_constraint=0):
    return Params(gamma, cfl, mu, eps_weno, tau_eps, tau_c, weno, order, smooth_flux, viscous, prandtl,
                  wall_temperature, (C.c_double * 3)(*[float(u) for u in wall_velocity]), int(wall_constraint))


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_bp = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.ora_mesh_build.restype = C.c_void_p
        L.ora_mesh_build.argtypes = [_dp, C.c_int64, _ip, _bp, C.c_int64, _dp, C.c_char_p, C.c_int]
        L.ora_mesh_free.argtypes = [C.c_void_p]
        L.ora_mesh_set_boundary.restype = C.c_int
        L.ora_mesh_set_boundary.argtypes = [C.c_void_p, _bp]
        L.ora_mesh_set_fixed_state.argtypes = [C.c_void_p, _dp, _dp]
        for fn in ("ora_mesh_nc", "ora_mesh_nf", "ora_mesh_n_singular"):
            getattr(L, fn).restype = C.c_int64
            getattr(L, fn).argtypes = [C.c_void_p]
        L.ora_mesh_topology.argtypes = [C.c_void_p, _ip, _ip, _ip, _ip, _bp]
        L.ora_mesh_geometry.argtypes = [C.c_void_p] + [_dp] * 8
        L.ora_mesh_stencils.argtypes = [C.c_void_p, _dp, _dp]
        L.ora_mesh_wall_stencils.restype = C.c_int64
        L.ora_mesh_wall_stencils.argtypes = [C.c_void_p, _dp, _dp, _bp]
        L.ora_reconstruct.argtypes = [C.c_void_p, C.POINTER(Params), _dp, _dp, _dp, _dp, _i32p]
        L.ora_gp_flux.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp, C.c_double,
                                  _dp, _dp, _dp, _dp]
        L.ora_face_records.argtypes = [C.c_void_p, C.POINTER(Params), _dp, _dp, C.c_double,
                                       C.c_int, _dp]
        L.ora_timestep.restype = C.c_double
        L.ora_timestep.argtypes = [C.c_void_p, C.POINTER(Params), _dp]
        L.ora_step.argtypes = [C.c_void_p, C.POINTER(Params), _dp, _dp, C.c_double,
                               C.POINTER(C.c_double)]
        L.ora_s2o4_linear_ode.restype = C.c_double
        L.ora_s2o4_linear_ode.argtypes = [C.c_double]
        L.ora_smoothness.restype = C.c_double
        L.ora_smoothness.argtypes = [C.c_void_p, C.c_int64, _dp, C.c_int]
        L.ora_weno_beta0.restype = C.c_double
        L.ora_weno_beta0.argtypes = [C.c_double, _dp, C.c_int, C.c_double, C.POINTER(C.c_double), _dp]
        L.ora_weno_weights.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, _dp]
        _lib = L
    return _lib


class Mesh:
    """Oracle mesh (topology, geometry, stencils) built from generator arrays."""

    def __init__(self, mesh):
        L = lib()
        err = C.create_string_buffer(256)
        xyz = np.ascontiguousarray(mesh["xyz"], dtype=np.float64)
        tet = np.ascontiguousarray(mesh["tet"], dtype=np.int64)
        shift = np.ascontiguousarray(mesh["shift"], dtype=np.int8)
        period = np.ascontiguousarray(mesh["period"], dtype=np.float64)
        self._h = L.ora_mesh_build(xyz, xyz.shape[0], tet, shift, tet.shape[0], period, err, 256)
        if not self._h:
            raise ValueError("oracle mesh: " + err.value.decode())
        self.nc = L.ora_mesh_nc(self._h)
        self.nf = L.ora_mesh_nf(self._h)
        self.n_singular = L.ora_mesh_n_singular(self._h)
        if mesh.get("bkind") is not None:
            self.set_boundary(mesh["bkind"])
        if mesh.get("fixed_state") is not None:
            self.set_fixed_state(*mesh["fixed_state"])

    def set_boundary(self, kind):
        """kind[nc][4]: 0 open, 1 slip wall, per local face (read on boundary
        faces only)."""
        kind = np.ascontiguousarray(kind, dtype=np.int8).reshape(self.nc, 4)
        if lib().ora_mesh_set_boundary(self._h, kind) != 0:
            raise ValueError("oracle mesh: invalid boundary kind")

    def set_fixed_state(self, W, dW):
        """The state fixed boundaries (kind 2) hold: W[5][nc], dW[15][nc]."""
        lib().ora_mesh_set_fixed_state(self._h, np.ascontiguousarray(W, dtype=np.float64),
                                       np.ascontiguousarray(dW, dtype=np.float64))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ora_mesh_free(self._h)
            self._h = None

    def topology(self):
        nc, nf = self.nc, self.nf
        out = dict(face_v=np.zeros((nf, 3), np.int64), face_lr=np.zeros((nf, 2), np.int64),
                   nbr=np.zeros((nc, 4), np.int64), csr_face=np.zeros((nc, 4), np.int64),
                   csr_sign=np.zeros((nc, 4), np.int8))
        lib().ora_mesh_topology(self._h, out["face_v"], out["face_lr"], out["nbr"],
                                out["csr_face"], out["csr_sign"])
        return out

    def geometry(self):
        nc, nf = self.nc, self.nf
        out = dict(vol=np.zeros(nc), cen=np.zeros((nc, 3)), mom2=np.zeros((nc, 6)),
                   dr=np.zeros(nc), farea=np.zeros(nf), fnorm=np.zeros((nf, 3)),
                   gp_l=np.zeros((nf, 3, 3)), gp_r=np.zeros((nf, 3, 3)))
        lib().ora_mesh_geometry(self._h, out["vol"], out["cen"], out["mom2"], out["dr"],
                                out["farea"], out["fnorm"], out["gp_l"], out["gp_r"])
        return out

    def stencils(self):
        M1 = np.zeros((self.nc, 3, 4))
        M2 = np.zeros((self.nc, 9, 16))
        lib().ora_mesh_stencils(self._h, M1, M2)
        return M1, M2

    def wall_stencils(self):
        """Sec. 4.4 constrained stencils of the non-slip wall cells:
        (MW1[nc][3][5], MW2[nc][9][17], wallc[nc])."""
        MW1 = np.zeros((self.nc, 3, 5))
        MW2 = np.zeros((self.nc, 9, 17))
        wc = np.zeros(self.nc, np.int8)
        lib().ora_mesh_wall_stencils(self._h, MW1, MW2, wc)
        return MW1, MW2, wc

    def reconstruct(self, p, W, dW):
        poly = np.zeros((self.nc, 5, 10))
        slopes = np.zeros((self.nc, 5, 3))
        fb = np.zeros(self.nc, np.int32)
        lib().ora_reconstruct(self._h, C.byref(p), np.ascontiguousarray(W, dtype=np.float64),
                              np.ascontiguousarray(dW, dtype=np.float64), poly, slopes, fb)
        return poly, slopes, fb

    def smoothness(self, c, v, r):
        """Smoothness indicator (Sec. 4.2) of cell c for the basis-form
        polynomial v[10]; r = 1 or 2."""
        return lib().ora_smoothness(self._h, int(c), np.ascontiguousarray(v, dtype=np.float64), int(r))

    def face_records(self, p, W, dW, dt, stage):
        rec = np.zeros((self.nf, 40 if stage == 1 else 20))
        if lib().ora_face_records(self._h, C.byref(p), np.ascontiguousarray(W, dtype=np.float64),
                                  np.ascontiguousarray(dW, dtype=np.float64), dt, stage, rec) != 0:
            raise ValueError("oracle: a fixed boundary face has no state")
        return rec

    def timestep(self, p, W):
        return lib().ora_timestep(self._h, C.byref(p), np.ascontiguousarray(W, dtype=np.float64))

    def step(self, p, W, dW, dt=0.0):
        """One two-stage step; returns (W, dW, dt_used) as new arrays."""
        W = np.array(W, dtype=np.float64, order="C", copy=True)
        dW = np.array(dW, dtype=np.float64, order="C", copy=True)
        used = C.c_double(0.0)
        if lib().ora_step(self._h, C.byref(p), W, dW, float(dt), C.byref(used)) != 0:
            raise ValueError("oracle: a fixed boundary face has no state")
        return W, dW, used.value

    def run(self, p, W, dW, nsteps=None, t_end=None, dt=0.0):
        """Several steps; with t_end the last step is clipped to reach it."""
        t = 0.0
        n = 0
        while True:
            if nsteps is not None and n >= nsteps:
                break
            if t_end is not None and t >= t_end * (1 - 1e-14):
                break
            d = dt if dt > 0 else self.timestep(p, W)
            if t_end is not None and t + d > t_end:
                d = t_end - t
            W, dW, used = self.step(p, W, dW, d)
            t += used
            n += 1
        return W, dW, t, n


def gp_flux(p, Wl, dWl, Wr, dWr, dt):
    """Kinetic solution at one Gauss point in the local frame; dW[i][q]."""
    out = [np.zeros(5) for _ in range(4)]
    lib().ora_gp_flux(C.byref(p), np.ascontiguousarray(Wl, dtype=np.float64),
                      np.ascontiguousarray(dWl, dtype=np.float64),
                      np.ascontiguousarray(Wr, dtype=np.float64),
                      np.ascontiguousarray(dWr, dtype=np.float64), float(dt), *out)
    return tuple(out)


def weno_beta0(vol, b, eps=1e-8):
    """beta_0 of the two-step reconstruction (Sec. 4.3) from the neighbours'
    step-1 slopes b[nn][3]; returns (beta_0, sigma^1st, wbar^1st[nn])."""
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1, 3)
    s1 = C.c_double(0.0)
    w1 = np.zeros(max(len(b), 1))
    beta0 = lib().ora_weno_beta0(float(vol), b.reshape(-1) if len(b) else np.zeros(3), len(b), float(eps),
                                 C.byref(s1), w1)
    return beta0, s1.value, w1[:len(b)]


def weno_weights(order, beta0, beta1, beta2=0.0, eps=1e-8):
    """Normalised nonlinear weights (Sec. 4.2) [wbar_0, wbar_1, wbar_2]."""
    w = np.zeros(3)
    lib().ora_weno_weights(int(order), float(eps), float(beta0), float(beta1), float(beta2), w)
    return w


def s2o4_linear_ode(z):
    return lib().ora_s2o4_linear_ode(float(z))
