"""Seeded synthetic inputs: tetrahedral box meshes, initial fields, exact solutions.

This module is the one place that both the CUDA library's callers and the CPU
oracle take their inputs from.  It holds none of the scheme's arithmetic (no
reconstruction, no kinetic flux, no time stepping): it only generates vertex
coordinates and connectivity, cell averages of analytic fields by quadrature,
and exact reference solutions used to measure errors.

Mesh recipe (the paper's tests use hexahedral grids split into tetrahedra,
Sec. 5.1, "6 x N^3 cells"; the split pattern is not given there):

* an nx x ny x nz grid of hexahedra of a box [0,Lx]x[0,Ly]x[0,Lz];
* every hexahedron is cut into the 6 Kuhn (Freudenthal) tetrahedra
  v0 -> v0+e_a -> v0+e_a+e_b -> v0+e_a+e_b+e_c for each permutation (a,b,c) of
  the axes; all six share the main diagonal v0-v7.  The split is translation
  invariant, so it is conforming across periodic boundaries;
* every unique vertex is moved by a uniform random jitter in [-j*h, j*h] per
  axis drawn from numpy's PCG64 with the given seed; on a non-periodic axis
  the vertices of the two end planes are moved only tangentially.

A periodic axis keeps n unique vertex planes; a tetrahedron that wraps refers
to the base vertex and carries an integer image shift, so its geometric vertex
is ``xyz[v] + shift * period``.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

KUHN_PERMS = list(itertools.permutations(range(3)))


def box_mesh(n, length=(1.0, 1.0, 1.0), periodic=(True, True, True), jitter=0.1,
             seed=0, diagonal=(1, 1, 1)):
    """Jittered Kuhn-split box mesh.

    ``diagonal`` picks which main diagonal of each hexahedron the six
    tetrahedra share: (1,1,1) joins (0,0,0)-(1,1,1); a -1 mirrors that axis,
    e.g. (1,1,-1) joins (0,0,1)-(1,1,0).

    Returns a dict with
      xyz    float64 [nv, 3]   unique vertex coordinates
      tet    int64   [nc, 4]   vertex ids of each tetrahedron (positive volume)
      shift  int8    [nc, 4, 3] periodic image shift of each tet vertex
      period float64 [3]       period per axis, 0 on a non-periodic axis
    """
    n = tuple(int(v) for v in n)
    length = tuple(float(v) for v in length)
    periodic = tuple(bool(v) for v in periodic)
    nv_ax = [n[a] if periodic[a] else n[a] + 1 for a in range(3)]
    h = [length[a] / n[a] for a in range(3)]
    rng = np.random.Generator(np.random.PCG64(seed))

    ii, jj, kk = np.meshgrid(np.arange(nv_ax[0]), np.arange(nv_ax[1]),
                             np.arange(nv_ax[2]), indexing="ij")
    # vertex id = i + nvx*(j + nvy*k): flatten with x fastest
    grid = [ii.transpose(2, 1, 0).ravel(), jj.transpose(2, 1, 0).ravel(),
            kk.transpose(2, 1, 0).ravel()]
    nv = grid[0].size
    xyz = np.empty((nv, 3))
    jit = rng.uniform(-1.0, 1.0, size=(nv, 3))
    for a in range(3):
        xyz[:, a] = grid[a] * h[a]
        amp = jitter * h[a] * jit[:, a]
        if not periodic[a]:
            amp = np.where((grid[a] == 0) | (grid[a] == n[a]), 0.0, amp)
        xyz[:, a] += amp

    hi, hj, hk = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]),
                             indexing="ij")
    hexes = np.stack([hi.transpose(2, 1, 0).ravel(), hj.transpose(2, 1, 0).ravel(),
                      hk.transpose(2, 1, 0).ravel()], axis=1)  # x fastest
    nh = hexes.shape[0]
    tets = np.empty((nh, 6, 4), dtype=np.int64)
    shifts = np.zeros((nh, 6, 4, 3), dtype=np.int8)
    mirror = [a for a in range(3) if diagonal[a] < 0]
    for t, perm in enumerate(KUHN_PERMS):
        offs = [np.zeros(3, dtype=np.int64)]
        for a in perm:
            o = offs[-1].copy()
            o[a] += 1
            offs.append(o)
        for o in offs:
            for a in mirror:
                o[a] = 1 - o[a]
        odd = sum(1 for x in range(3) for y in range(x + 1, 3) if perm[x] > perm[y]) % 2
        odd = (odd + len(mirror)) % 2
        if odd:  # negative orientation: swap vertices 1 and 2
            offs[1], offs[2] = offs[2], offs[1]
        for v, o in enumerate(offs):
            c = hexes + o[None, :]
            idx = np.zeros(nh, dtype=np.int64)
            stride = 1
            for a in range(3):
                ca = c[:, a]
                if periodic[a]:
                    wrap = ca >= n[a]
                    shifts[:, t, v, a] = wrap.astype(np.int8)
                    ca = np.where(wrap, ca - n[a], ca)
                idx += ca * stride
                stride *= nv_ax[a]
            tets[:, t, v] = idx
    period = np.array([length[a] if periodic[a] else 0.0 for a in range(3)])
    return {
        "xyz": xyz,
        "tet": tets.reshape(nh * 6, 4),
        "shift": shifts.reshape(nh * 6, 4, 3),
        "period": period,
        "n": n,
        "length": length,
        "periodic": periodic,
    }


def tet_vertices(mesh):
    """Geometric vertex positions [nc, 4, 3] with periodic shifts applied."""
    return mesh["xyz"][mesh["tet"]] + mesh["shift"].astype(np.float64) * mesh["period"]


# --------------------------------------------------------------------------
# quadrature used only to synthesise cell averages of analytic fields
# --------------------------------------------------------------------------

def _collapsed_gauss(order):
    """Points (barycentric xi, eta, zeta) and weights (sum 1) of a collapsed
    tensor Gauss-Legendre rule on the unit tetrahedron (Duffy map)."""
    g, w = np.polynomial.legendre.leggauss(order)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    pts, wts = [], []
    for a, wa in zip(g, w):
        for b, wb in zip(g, w):
            for c, wc in zip(g, w):
                xi = a
                eta = b * (1.0 - a)
                zeta = c * (1.0 - a) * (1.0 - b)
                pts.append((xi, eta, zeta))
                wts.append(wa * wb * wc * (1.0 - a) ** 2 * (1.0 - b))
    pts = np.array(pts)
    wts = np.array(wts)
    return pts, wts / wts.sum()


def cell_average(mesh, func, order=5, chunk=200_000):
    """Cell averages of ``func(x[..., 3]) -> [..., m]`` over every tetrahedron."""
    pts, wts = _collapsed_gauss(order)
    lam = np.stack([1.0 - pts.sum(1), pts[:, 0], pts[:, 1], pts[:, 2]], axis=1)  # [q,4]
    verts = tet_vertices(mesh)
    out = []
    for s in range(0, verts.shape[0], chunk):
        v = verts[s:s + chunk]
        x = np.einsum("qa,cad->cqd", lam, v)
        f = func(x)  # [c, q, m]
        out.append(np.einsum("q,cqm->cm", wts, f))
    return np.concatenate(out, axis=0)


# --------------------------------------------------------------------------
# initial / exact fields.  State layout: W [5, nc] conservative variables
# (rho, rho U1, rho U2, rho U3, rho E); dW [15, nc] = d W_q / d x_i stored at
# row 3*q + i (component-major).
# --------------------------------------------------------------------------

def _prim_to_cons(rho, u, p, gamma):
    ke = 0.5 * rho * (u[..., 0] ** 2 + u[..., 1] ** 2 + u[..., 2] ** 2)
    return np.stack([rho, rho * u[..., 0], rho * u[..., 1], rho * u[..., 2],
                     p / (gamma - 1.0) + ke], axis=-1)


def sine_wave_fields(x, t=0.0, amp=0.2, k=2.0 * math.pi, u=(1.0, 1.0, 1.0),
                     p=1.0, gamma=1.4):
    """Point values and gradients of the advected density wave
    rho = 1 + amp sin(k (x+y+z - (u1+u2+u3) t)), constant velocity and pressure
    (Sec. 5.1; the phase speed along x+y+z is u1+u2+u3).
    Returns W [..., 5] and dW [..., 15]."""
    s = x[..., 0] + x[..., 1] + x[..., 2] - (u[0] + u[1] + u[2]) * t
    rho = 1.0 + amp * np.sin(k * s)
    drho = amp * k * np.cos(k * s)
    uu = np.broadcast_to(np.asarray(u, dtype=np.float64), x.shape)
    W = _prim_to_cons(rho, uu, np.full_like(rho, p), gamma)
    # every conservative component is affine in rho here
    dqdrho = np.array([1.0, u[0], u[1], u[2], 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)])
    dW = np.empty(x.shape[:-1] + (15,))
    for q in range(5):
        for i in range(3):
            dW[..., 3 * q + i] = dqdrho[q] * drho
    return W, dW


def sine_wave_state(mesh, t=0.0, order=5, amp=0.2, k=2.0 * math.pi, u=(1.0, 1.0, 1.0), p=1.0,
                    gamma=1.4):
    """Cell averages of W and of grad W for the density wave at time t.  Every
    conservative variable is affine in rho, so only the averages of
    sin(k s) and cos(k s), s = x + y + z - (u1+u2+u3) t, are integrated."""
    c = u[0] + u[1] + u[2]

    def f(x):
        sarg = k * (x[..., 0] + x[..., 1] + x[..., 2] - c * t)
        return np.stack([np.sin(sarg), np.cos(sarg)], axis=-1)

    avg = cell_average(mesh, f, order=order)
    rho = 1.0 + amp * avg[:, 0]
    drho = amp * k * avg[:, 1]
    dqdrho = np.array([1.0, u[0], u[1], u[2], 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)])
    W = dqdrho[:, None] * rho[None, :]
    W[4] += p / (gamma - 1.0)
    dW = np.repeat((dqdrho[:, None] * drho[None, :]), 3, axis=0)
    return np.ascontiguousarray(W), np.ascontiguousarray(dW)


def _neg_fraction(d):
    """Fraction of each tetrahedron on which the linear function with vertex
    values d [nc, 4] is negative (divided difference of x_+^3)."""
    d = d.astype(np.float64).copy()
    out = np.zeros(d.shape[0])
    allneg = (d < 0).all(1)
    out[allneg] = 1.0
    cut = ~allneg & (d < 0).any(1)
    dc = d[cut]
    # separate coincident values slightly; the effect is ~1e-9 in the fraction
    scale = np.abs(dc).max(1, keepdims=True) + 1e-300
    for a in range(4):
        for b in range(a + 1, 4):
            tie = np.abs(dc[:, a] - dc[:, b]) < 1e-9 * scale[:, 0]
            dc[tie, b] += 2e-9 * scale[tie, 0] * (b + 1)
    pos = np.zeros(dc.shape[0])
    for i in range(4):
        den = np.ones(dc.shape[0])
        for j in range(4):
            if j != i:
                den *= dc[:, i] - dc[:, j]
        pos += np.maximum(dc[:, i], 0.0) ** 3 / den
    out[cut] = 1.0 - pos
    return out


def riemann_x_state(mesh, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x0=0.5,
                    gamma=1.4):
    """Planar Riemann data along x: (rho, u1, p) on x < x0 and x > x0, exact
    volume fractions of the plane split per cell, zero gradients (Sod's data
    by default)."""
    verts = tet_vertices(mesh)
    frac_l = _neg_fraction(verts[:, :, 0] - x0)
    def cons(st):
        rho, u, p = st
        return _prim_to_cons(np.array(rho), np.array([u, 0.0, 0.0]), np.array(p), gamma)
    wl, wr = cons(left), cons(right)
    W = frac_l[None, :] * wl[:, None] + (1.0 - frac_l)[None, :] * wr[:, None]
    return np.ascontiguousarray(W), np.zeros((15, W.shape[1]))


# --------------------------------------------------------------------------
# exact Riemann solution (ideal gas), for error measurement
# --------------------------------------------------------------------------

def exact_riemann(left, right, gamma=1.4):
    """Star state (p*, u*) of the 1-D Riemann problem, by Newton's method on
    the pressure function f_L(p) + f_R(p) + du = 0 (shock branch from the
    Rankine-Hugoniot relations, rarefaction branch from the isentropic ones)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)

    def fk(p, rk, pk, ck):
        if p > pk:
            a = 2.0 / ((gamma + 1.0) * rk)
            b = (gamma - 1.0) / (gamma + 1.0) * pk
            q = math.sqrt(a / (p + b))
            return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + b))
        e = (gamma - 1.0) / (2.0 * gamma)
        r = (p / pk) ** e
        return (2.0 * ck / (gamma - 1.0) * (r - 1.0),
                (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rk * ck))

    def f(p):
        a, da = fk(p, rl, pl, cl)
        b, db = fk(p, rr, pr, cr)
        return a + b + (ur - ul), da + db

    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        val, der = f(p)
        pn = max(1e-12, p - val / der)
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    a, _ = fk(p, rl, pl, cl)
    b, _ = fk(p, rr, pr, cr)
    u = 0.5 * (ul + ur) + 0.5 * (b - a)
    return p, u


def sample_riemann(xi, left, right, gamma=1.4):
    """Self-similar exact solution (rho, u, p) at xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = exact_riemann(left, right, gamma)
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    # left side of contact
    if ps > pl:  # left shock
        rsl = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0)
        sl = ul - cl * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
        left_zone = xi < sl
        star_l = (xi >= sl) & (xi < us)
        fan_l = np.zeros_like(xi, dtype=bool)
    else:  # left rarefaction
        rsl = rl * (ps / pl) ** (1.0 / gamma)
        csl = cl * (ps / pl) ** ((gamma - 1) / (2 * gamma))
        head, tail = ul - cl, us - csl
        left_zone = xi < head
        fan_l = (xi >= head) & (xi < tail)
        star_l = (xi >= tail) & (xi < us)
    if ps > pr:  # right shock
        rsr = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0)
        sr = ur + cr * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
        right_zone = xi >= sr
        star_r = (xi >= us) & (xi < sr)
        fan_r = np.zeros_like(xi, dtype=bool)
    else:
        rsr = rr * (ps / pr) ** (1.0 / gamma)
        csr = cr * (ps / pr) ** ((gamma - 1) / (2 * gamma))
        head, tail = ur + cr, us + csr
        right_zone = xi >= head
        fan_r = (xi >= tail) & (xi < head)
        star_r = (xi >= us) & (xi < tail)
    rho[left_zone], u[left_zone], p[left_zone] = rl, ul, pl
    rho[right_zone], u[right_zone], p[right_zone] = rr, ur, pr
    rho[star_l], u[star_l], p[star_l] = rsl, us, ps
    rho[star_r], u[star_r], p[star_r] = rsr, us, ps
    if fan_l.any():
        x = xi[fan_l]
        c = 2.0 / (gamma + 1) * (cl + 0.5 * (gamma - 1) * (ul - x))
        uf = 2.0 / (gamma + 1) * (cl + 0.5 * (gamma - 1) * ul + x)
        rho[fan_l] = rl * (c / cl) ** (2.0 / (gamma - 1))
        u[fan_l] = uf
        p[fan_l] = pl * (c / cl) ** (2.0 * gamma / (gamma - 1))
    if fan_r.any():
        x = xi[fan_r]
        c = 2.0 / (gamma + 1) * (cr - 0.5 * (gamma - 1) * (ur - x))
        uf = 2.0 / (gamma + 1) * (-cr + 0.5 * (gamma - 1) * ur + x)
        rho[fan_r] = rr * (c / cr) ** (2.0 / (gamma - 1))
        u[fan_r] = uf
        p[fan_r] = pr * (c / cr) ** (2.0 * gamma / (gamma - 1))
    return rho, u, p


def riemann_x_exact_density(mesh, t, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1),
                            x0=0.5, gamma=1.4, order=6):
    """Cell averages of the exact density at time t > 0 (quadrature of the
    piecewise-smooth exact solution)."""
    def f(x):
        r, _, _ = sample_riemann((x[..., 0] - x0) / t, left, right, gamma)
        return r[..., None]
    return cell_average(mesh, f, order=order)[:, 0]


BC_OPEN, BC_SLIP_WALL, BC_FIXED, BC_NOSLIP_WALL, BC_ISOTHERMAL_WALL, BC_MOVING_WALL = 0, 1, 2, 3, 4, 5


def boundary_kinds(mesh, spec):
    """Boundary kind per local face, int8 [nc, 4] (face f is opposite tet
    vertex f).  ``spec`` maps (axis, "lo" | "hi") to a kind for the faces on
    that end plane of a non-periodic axis (the planes are the extreme vertex
    coordinates; the generator jitters end-plane vertices only tangentially);
    every other face gets BC_OPEN."""
    xyz = mesh["xyz"]
    tet = mesh["tet"]
    kind = np.zeros(tet.shape, dtype=np.int8)
    for (a, end), k in spec.items():
        if mesh["period"][..., a].any():
            raise ValueError("axis %d is periodic" % a)
        plane = xyz[:, a].min() if end == "lo" else xyz[:, a].max()
        on = xyz[tet, a] == plane  # [nc, 4]
        for f in range(4):
            others = [v for v in range(4) if v != f]
            kind[on[:, others].all(axis=1), f] = k
    return kind


def wall_kinds(mesh, axes):
    """Slip walls (BC_SLIP_WALL) on both end planes of the given axes."""
    return boundary_kinds(mesh, {(a, e): BC_SLIP_WALL for a in axes for e in ("lo", "hi")})


def wall_reflection_exact_density(mesh, t, state=(1.0, 1.0, 1.0), length=1.0, gamma=1.4,
                                  order=6):
    """Uniform gas (rho, u, p) moving along x between slip walls at x = 0 and
    x = length: at the right wall a shock reflects, at the left wall a
    rarefaction opens.  Each is the Riemann problem between the gas and its
    mirror image; the two fans are separated while the rarefaction head
    (u + c) t and the shock have not met.  Cell averages of the exact density
    at time t."""
    rho, u, p = state
    gas, mirror = (rho, u, p), (rho, -u, p)
    ps, _ = exact_riemann(gas, mirror, gamma)
    c = math.sqrt(gamma * p / rho)
    shock = u - c * math.sqrt((gamma + 1) / (2 * gamma) * ps / p + (gamma - 1) / (2 * gamma))
    if (u + c) * t >= length + shock * t:
        raise ValueError("the two wall waves have met before t")

    def f(x):
        xx = x[..., 0]
        r_left, _, _ = sample_riemann(xx / t, mirror, gas, gamma)
        r_right, _, _ = sample_riemann((xx - length) / t, gas, mirror, gamma)
        return np.where(xx < 0.5 * length, r_left, r_right)[..., None]
    return cell_average(mesh, f, order=order)[:, 0]


def shu_osher_state(mesh, gamma=1.4, order=3):
    """Shu-Osher data along x on [0, 10] (Sec. 5.2): (3.857134, 2.629369,
    10.33333) for x <= 1, (1 + 0.2 sin 5x, 0, 1) beyond; cell averages by
    quadrature (collapsed Gauss of the given order), gradients of the smooth
    part by the same quadrature, zero in cells the jump cuts."""
    left = np.array([3.857134, 2.629369, 10.33333])

    def prim(x):
        xx = x[..., 0]
        rho = np.where(xx <= 1.0, left[0], 1.0 + 0.2 * np.sin(5.0 * xx))
        u = np.where(xx <= 1.0, left[1], 0.0)
        p = np.where(xx <= 1.0, left[2], 1.0)
        return rho, u, p

    def cons(x):
        rho, u, p = prim(x)
        z = np.zeros_like(rho)
        return np.stack([rho, rho * u, z, z, p / (gamma - 1.0) + 0.5 * rho * u * u], axis=-1)
    W = cell_average(mesh, cons, order=order).T.copy()
    # gradients: only rho and rho E vary in the smooth part (d/dx of the
    # sine), and U = 0 there
    def grad(x):
        xx = x[..., 0]
        out = np.zeros(xx.shape + (15,))
        out[..., 0] = np.where(xx <= 1.0, 0.0, 0.2 * 5.0 * np.cos(5.0 * xx))  # d rho / dx
        return out
    dW = cell_average(mesh, grad, order=order).T.copy()
    verts = tet_vertices(mesh)
    cut = (verts[:, :, 0].min(axis=1) < 1.0) & (verts[:, :, 0].max(axis=1) > 1.0)
    dW[:, cut] = 0.0
    return np.ascontiguousarray(W), np.ascontiguousarray(dW)


def blast_wave_state(mesh, gamma=1.4):
    """Woodward-Colella blast wave on [0, 1] (Sec. 5.2): rho = 1, u = 0 and
    p = 1000 | 0.01 | 100 split at x = 0.1 and 0.9; exact volume fractions of
    the two planes per cell, zero gradients."""
    verts = tet_vertices(mesh)
    f_left = _neg_fraction(verts[:, :, 0] - 0.1)
    f_right = 1.0 - _neg_fraction(verts[:, :, 0] - 0.9)
    f_mid = 1.0 - f_left - f_right
    E = (1000.0 * f_left + 0.01 * f_mid + 100.0 * f_right) / (gamma - 1.0)
    W = np.zeros((5, verts.shape[0]))
    W[0] = 1.0
    W[4] = E
    return W, np.zeros((15, W.shape[1]))


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def sine_wave_case(n=8, jitter=0.1, seed=1, diagonal=(1, 1, -1)):
    """Periodic unit cube, n^3 hexes x 6 tets, rho = 1 + 0.2 sin 2pi(x+y+z),
    U = (1,1,1), p = 1, gamma = 1.4.  The tetrahedra share the hexahedron
    diagonal (0,0,1)-(1,1,0), across the direction of propagation: the split
    is not given in the paper, and this one reproduces the magnitude of its
    accuracy table on the same setup."""
    mesh = box_mesh((n, n, n), (1.0, 1.0, 1.0), (True, True, True), jitter, seed, diagonal)
    W, dW = sine_wave_state(mesh)
    return mesh, W, dW


def sod_case(nx=64, nyz=8, jitter=0.1, seed=2):
    """Sod tube along x on [0,1]x[0,0.1]^2 (y, z periodic, x ends open),
    nx x nyz x nyz hexes x 6 tets."""
    mesh = box_mesh((nx, nyz, nyz), (1.0, 0.1, 0.1), (False, True, True), jitter, seed)
    W, dW = riemann_x_state(mesh)
    return mesh, W, dW


# --------------------------------------------------------------------------
# batches of independent cases (one mesh, disjoint components)
# --------------------------------------------------------------------------

def shear_decay_state(mesh, amp=0.05, rho=1.0, p=1.0, length=1.0, gamma=1.4, order=4):
    """Tangential shear v = amp sin(pi x / length) (along y) in a gas of
    uniform density and pressure: cell averages of W and of grad W."""
    k = math.pi / length

    def cons(x):
        s = np.sin(k * x[..., 0])
        v = amp * s
        z = np.zeros_like(v)
        return np.stack([np.full_like(v, rho), z, rho * v, z, p / (gamma - 1.0) + 0.5 * rho * v * v], axis=-1)

    def grad(x):
        s, c = np.sin(k * x[..., 0]), np.cos(k * x[..., 0])
        out = np.zeros(x.shape[:-1] + (15,))
        out[..., 3 * 2 + 0] = rho * amp * k * c              # d(rho v)/dx
        out[..., 3 * 4 + 0] = rho * amp * amp * k * s * c    # d(rho E)/dx
        return out
    W = cell_average(mesh, cons, order=order).T.copy()
    dW = cell_average(mesh, grad, order=order).T.copy()
    return np.ascontiguousarray(W), np.ascontiguousarray(dW)


def shear_decay_amplitude(mesh, W, length=1.0, vol=None):
    """Least-squares amplitude of rho v against sin(pi x / length) over the
    cells (volume weighted, cell averages of the sine by quadrature)."""
    s = cell_average(mesh, lambda x: np.sin(math.pi / length * x[..., 0])[..., None], order=4)[:, 0]
    if vol is None:
        vol = np.ones_like(s)
    return float((vol * W[2] * s).sum() / (vol * s * s).sum())


def shear_decay_case(nx=16, nyz=2, amp=0.05, jitter=0.1, seed=7):
    """Decaying shear between no-slip adiabatic walls at x = 0 and 1 (y, z
    periodic, cubic hexahedra, nx x nyz x nyz hexes x 6 tets).  For a viscous
    gas at low Mach number v = amp sin(pi x) exp(-nu pi^2 t), nu = mu / rho."""
    w = nyz / nx
    mesh = box_mesh((nx, nyz, nyz), (1.0, w, w), (False, True, True), jitter, seed)
    mesh["bkind"] = boundary_kinds(mesh, {(0, "lo"): BC_NOSLIP_WALL, (0, "hi"): BC_NOSLIP_WALL})
    W, dW = shear_decay_state(mesh, amp=amp)
    return mesh, W, dW


def isentropic_vortex_fields(x, length=10.0, strength=5.0, mach=0.5, gamma=1.4):
    """Conservative variables of an isentropic vortex (axis along z through
    the box centre, core radius 1) on a free stream of Mach number `mach`
    along (1,1,1)/sqrt(3), rho_inf = 1, p_inf = 1/gamma (c_inf = 1): the
    swirl u_theta = strength/(2 pi) r exp((1 - r^2)/2) and the temperature
    T = p/rho = 1/gamma - (gamma-1)/gamma strength^2/(8 pi^2) exp(1 - r^2) of
    the radial momentum balance, with rho = (gamma T)^(1/(gamma-1))."""
    c = 0.5 * length
    dx, dy = x[..., 0] - c, x[..., 1] - c
    r2 = dx * dx + dy * dy
    k = strength / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    ui = mach / math.sqrt(3.0)
    u = ui - k * dy
    v = ui + k * dx
    w = np.full_like(u, ui)
    T = 1.0 / gamma - (gamma - 1.0) / gamma * strength ** 2 / (8.0 * math.pi ** 2) * np.exp(1.0 - r2)
    rho = (gamma * T) ** (1.0 / (gamma - 1.0))
    p = rho * T
    return np.stack([rho, rho * u, rho * v, rho * w, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)],
                    axis=-1)


def isentropic_vortex_case(n=64, length=10.0, strength=5.0, mach=0.5, jitter=0.1, seed=8, order=3):
    """The isentropic vortex on the periodic box [0, length]^3, n^3 hexes x 6
    tets: cell averages of W by quadrature, cell-averaged gradients by
    quadrature of central differences of the field (step 1e-5 length)."""
    mesh = box_mesh((n, n, n), (length,) * 3, (True, True, True), jitter, seed)
    f = lambda x: isentropic_vortex_fields(x, length, strength, mach)
    W = cell_average(mesh, f, order=order).T.copy()
    h = 1e-5 * length

    def grad(x):
        out = np.empty(x.shape[:-1] + (15,))
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            d = (f(x + e) - f(x - e)) / (2.0 * h)
            out[..., i::3] = d
        return out
    dW = cell_average(mesh, grad, order=order).T.copy()
    return mesh, np.ascontiguousarray(W), np.ascontiguousarray(dW)


def wall_reflection_case(nx=64, nyz=4, state=(1.0, 1.0, 1.0), jitter=0.1, seed=3):
    """Uniform gas moving along x in [0,1] x [0,nyz/nx]^2 (cubic hexahedra)
    between slip walls at x = 0 and 1, y and z periodic; nx x nyz x nyz
    hexes x 6 tets."""
    w = nyz / nx
    mesh = box_mesh((nx, nyz, nyz), (1.0, w, w), (False, True, True), jitter, seed)
    mesh["bkind"] = wall_kinds(mesh, (0,))
    W, dW = riemann_x_state(mesh, left=state, right=state)
    return mesh, W, dW


def shu_osher_case(nx=200, nyz=2, jitter=0.0, seed=4):
    """Shu-Osher problem (Sec. 5.2) on [0,10]x[0,0.1]^2, nx x nyz x nyz hexes
    x 6 tets, y, z periodic.  Both x ends fixed to the initial state: on the
    left the supersonic inflow (every characteristic enters, so holding the
    inflow state is the non-reflecting condition), on the right the wave
    profile carried past the boundary; ``fixed_state`` is that state."""
    mesh = box_mesh((nx, nyz, nyz), (10.0, 0.1, 0.1), (False, True, True), jitter, seed)
    mesh["bkind"] = boundary_kinds(mesh, {(0, "lo"): BC_FIXED, (0, "hi"): BC_FIXED})
    W, dW = shu_osher_state(mesh)
    mesh["fixed_state"] = (W, dW)
    return mesh, W, dW


def blast_wave_case(nx=200, nyz=2, jitter=0.0, seed=6):
    """Woodward-Colella blast wave (Sec. 5.2) on [0,1]x[0,0.01]^2 with
    reflecting (slip-wall) ends, nx x nyz x nyz hexes x 6 tets, y, z
    periodic."""
    mesh = box_mesh((nx, nyz, nyz), (1.0, 0.01, 0.01), (False, True, True), jitter, seed)
    mesh["bkind"] = wall_kinds(mesh, (0,))
    W, dW = blast_wave_state(mesh)
    return mesh, W, dW


def batch_mesh(meshes):
    """Disjoint union of meshes: vertex ids offset, cells grouped by case.
    Adds ``case`` (int32 per tet) and per-case ``period`` [ncase, 3]."""
    xyz, tet, shift, case, period = [], [], [], [], []
    off = 0
    for k, m in enumerate(meshes):
        xyz.append(m["xyz"])
        tet.append(m["tet"] + off)
        shift.append(m["shift"])
        case.append(np.full(m["tet"].shape[0], k, dtype=np.int32))
        period.append(m["period"])
        off += m["xyz"].shape[0]
    out = {"xyz": np.concatenate(xyz), "tet": np.concatenate(tet), "shift": np.concatenate(shift),
           "case": np.concatenate(case), "period": np.stack(period), "ncase": len(meshes),
           "case_cells": np.array([m["tet"].shape[0] for m in meshes])}
    if any(m.get("bkind") is not None for m in meshes):
        out["bkind"] = np.concatenate([m["bkind"] if m.get("bkind") is not None
                                       else np.zeros(m["tet"].shape, np.int8) for m in meshes])
    return out


def riemann_slab_state(mesh, inner=(1.0, 1.0), outer=(0.125, 0.1), mach=1.0, x0=0.25, x1=0.75,
                       gamma=1.4):
    """Periodic planar Riemann data: (rho, p) = inner on x0 <= x < x1 and outer
    elsewhere, both moving along x at Ma times the inner sound speed; exact
    volume fractions of the two planes per cell, zero gradients."""
    verts = tet_vertices(mesh)
    frac_in = _neg_fraction(verts[:, :, 0] - x1) - _neg_fraction(verts[:, :, 0] - x0)
    u = mach * math.sqrt(gamma * inner[1] / inner[0])
    def cons(rho, p):
        return _prim_to_cons(np.array(rho), np.array([u, 0.0, 0.0]), np.array(p), gamma)
    wi, wo = cons(*inner), cons(*outer)
    W = frac_in[None, :] * wi[:, None] + (1.0 - frac_in)[None, :] * wo[:, None]
    return np.ascontiguousarray(W), np.zeros((15, W.shape[1]))


def batch_cases(n_cases=48, n_range=(8, 40), seed=5, jitter=0.1, quad_order=3,
                riemann=((1.0, 1.0), (0.5, 0.6))):
    """Independent periodic unit cubes of n^3 hexes x 6 tets, n uniform in
    n_range (seeded); each case a density wave or a planar Riemann problem
    ((rho, p) = riemann[0] inside the slab, riemann[1] outside) moving at a
    Mach number uniform in [0.5, 3].  The default jump is milder than Sod's:
    the scheme has no positivity limiter on cell averages, and a Sod-strength
    jump moving at Mach 1.4 over a jittered 36^3 mesh already produces a
    negative pressure in its first step (the CPU oracle gives the same).
    Returns (batch mesh, W, dW, case descriptions, the cases' meshes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    meshes, Ws, dWs, desc = [], [], [], []
    for k in range(n_cases):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        kind = "sine" if rng.random() < 0.5 else "riemann"
        mach = float(rng.uniform(0.5, 3.0))
        m = box_mesh((n, n, n), (1.0, 1.0, 1.0), (True, True, True), jitter, seed * 1000 + k,
                     diagonal=(1, 1, -1))
        if kind == "sine":
            W, dW = sine_wave_state(m, order=quad_order)
        else:
            W, dW = riemann_slab_state(m, inner=riemann[0], outer=riemann[1], mach=mach)
        meshes.append(m)
        Ws.append(W)
        dWs.append(dW)
        desc.append({"n": n, "kind": kind, "mach": mach if kind == "riemann" else None})
    return batch_mesh(meshes), np.concatenate(Ws, axis=1), np.concatenate(dWs, axis=1), desc, meshes


def sphere_shell_mesh(nr=64, ntheta=96, nphi=192, r0=0.5, r1=20.0, ratio=1.08):
    """O-type mesh of the shell r0 <= r <= r1 around a sphere of diameter
    2 r0 (the viscous sphere of Sec. 5.3): nr radial layers with radii in
    geometric progression (ratio between successive spacings), ntheta polar
    and nphi azimuthal divisions, every (r, theta, phi) hexahedron cut into
    the 6 Kuhn tetrahedra in index space.  On the two rows of hexahedra
    touching a pole the azimuthal edge on the axis collapses to a point;
    the 3 Kuhn tetrahedra that contain such an edge are degenerate and are
    left out, so those rows carry 3 tetrahedra per hexahedron:
    nc = 6 nr (ntheta - 2) nphi + 3 nr 2 nphi.  Faces are flat (the
    sphere is represented by its inscribed polyhedron); the split is
    mirrored in theta on the southern half so that both poles are alike
    (the split of each theta = const face is unchanged by the mirror, so
    the two halves stay conforming); no periodic axis
    (the seam at phi = 2 pi reuses the vertices at phi = 0).  bkind marks
    the faces on r = r0 as non-slip walls and those on r = r1 as fixed
    (far-field) faces.  Cells are ordered with phi fastest, then theta,
    then r."""
    q = float(ratio)
    s = np.arange(nr + 1, dtype=np.float64)
    frac = s / nr if q == 1.0 else (q ** s - 1.0) / (q ** nr - 1.0)
    rad = r0 + (r1 - r0) * frac
    th = math.pi * np.arange(ntheta + 1) / ntheta
    ph = 2.0 * math.pi * np.arange(nphi) / nphi
    npole = nr + 1
    # vertex ids: north poles, south poles, then (i, j = 1..ntheta-1, k)
    nv = 2 * npole + npole * (ntheta - 1) * nphi
    xyz = np.empty((nv, 3))
    xyz[:npole] = np.stack([np.zeros(npole), np.zeros(npole), rad], axis=1)
    xyz[npole:2 * npole] = np.stack([np.zeros(npole), np.zeros(npole), -rad], axis=1)
    I, J, K = np.meshgrid(np.arange(npole), np.arange(1, ntheta), np.arange(nphi), indexing="ij")
    R, T, P = rad[I], th[J], ph[K]
    xyz[2 * npole:] = np.stack([R * np.sin(T) * np.cos(P), R * np.sin(T) * np.sin(P), R * np.cos(T)],
                               axis=-1).reshape(-1, 3)
    vrad = np.empty(nv, dtype=np.int64)
    vrad[:npole] = np.arange(npole)
    vrad[npole:2 * npole] = np.arange(npole)
    vrad[2 * npole:] = I.ravel()

    def vid(i, j, k):
        k = k % nphi
        mid = 2 * npole + (i * (ntheta - 1) + (j - 1)) * nphi + k
        return np.where(j == 0, i, np.where(j == ntheta, npole + i, mid))

    hi, hj, hk = np.meshgrid(np.arange(nr), np.arange(ntheta), np.arange(nphi), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()  # phi fastest
    nh = hi.size
    # southern half: the split mirrored in theta, so that both poles carry
    # the same pattern (the unmirrored split leaves the south-pole cells
    # with nearly dependent stencils)
    south = hj >= (ntheta + 1) // 2
    tets = np.empty((nh, 6, 4), dtype=np.int64)
    for t, perm in enumerate(KUHN_PERMS):
        o = [0, 0, 0]
        offs = [list(o)]
        for a in perm:
            o[a] += 1
            offs.append(list(o))
        for v, (oi, oj, ok) in enumerate(offs):
            tets[:, t, v] = vid(hi + oi, hj + np.where(south, 1 - oj, oj), hk + ok)
    tets = tets.reshape(-1, 4)
    srt = np.sort(tets, axis=1)
    keep = (srt[:, 1:] != srt[:, :-1]).all(axis=1)
    tets = tets[keep]
    # positive orientation
    x = xyz[tets]
    vol = np.einsum("ij,ij->i", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))
    neg = vol < 0.0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    nc = tets.shape[0]
    kind = np.zeros((nc, 4), dtype=np.int8)
    tr = vrad[tets]
    for f in range(4):
        others = [v for v in range(4) if v != f]
        kind[(tr[:, others] == 0).all(axis=1), f] = BC_NOSLIP_WALL
        kind[(tr[:, others] == nr).all(axis=1), f] = BC_FIXED
    return {
        "xyz": xyz,
        "tet": tets,
        "shift": np.zeros((nc, 4, 3), dtype=np.int8),
        "period": np.zeros(3),
        "bkind": kind,
        "n": (nr, ntheta, nphi),
        "radii": (float(r0), float(r1)),
    }


def sphere_case(nr=64, ntheta=96, nphi=192, r0=0.5, r1=20.0, ratio=1.08, mach=0.2, reynolds=100.0,
                gamma=1.4):
    """Viscous flow past a sphere of diameter D = 2 r0 (Sec. 5.3): the shell
    mesh of sphere_shell_mesh started impulsively from the free stream
    (rho = 1, p = 1/gamma so that c = 1, U = (mach, 0, 0)), zero gradients;
    the far-field faces hold that state.  Returns (mesh, W, dW, mu) with the
    constant viscosity mu = rho U D / Re."""
    mesh = sphere_shell_mesh(nr, ntheta, nphi, r0, r1, ratio)
    nc = mesh["tet"].shape[0]
    p = 1.0 / gamma
    w = np.array([1.0, mach, 0.0, 0.0, p / (gamma - 1.0) + 0.5 * mach * mach])
    W = np.ascontiguousarray(np.repeat(w[:, None], nc, axis=1))
    dW = np.zeros((15, nc))
    mesh["fixed_state"] = (W, dW)
    return mesh, W, dW, mach * 2.0 * r0 / reynolds
