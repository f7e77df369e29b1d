"""Pins of the oracle's gas-kinetic flux at one Gauss point (Sec. 2.2 and the
equilibrium-state construction of Sec. 4.5).

The brute-force reference integrates the time-dependent distribution of
Eq. 2nd-flux numerically: velocity space by Gauss-Hermite (full space),
Gauss-Legendre on a truncated half line (half space) and Gauss-Laguerre in
xi^2 (K = 2 internal degrees of freedom at gamma = 1.4), time by composite
Gauss-Legendre.  Moments, micro-slopes and the kinetic weighting are thus
computed without the oracle's erfc/recursion moment tables or its sparse
polynomial algebra.  Invariants (uniform flow gives the Euler flux, mirror
antisymmetry) close the remaining gaps."""
import math

import numpy as np
import pytest

GAMMA = 1.4
K = 2  # (5 - 3 gamma) / (gamma - 1) at gamma = 1.4


def _prim(W):
    rho = W[0]
    U = W[1:4] / rho
    p = (GAMMA - 1.0) * (W[4] - 0.5 * rho * U @ U)
    return rho, U, p, rho / (2.0 * p)


def _nodes(U, lam, half):
    """Nodes (u1,u2,u3,s=xi^2) and weights of the normalised Maxwellian
    measure, u1 restricted to u1>0 (half=+1), u1<0 (-1) or unrestricted."""
    zh, wh = np.polynomial.hermite.hermgauss(24)
    sl = 1.0 / math.sqrt(lam)
    u2 = U[1] + zh * sl
    u3 = U[2] + zh * sl
    w2 = wh / math.sqrt(math.pi)
    if half == 0:
        u1 = U[0] + zh * sl
        w1 = wh / math.sqrt(math.pi)
    else:
        # integrate exp(-lam (u-U)^2) sqrt(lam/pi) on the half line, truncated
        # where the Gaussian is below 1e-30 of its peak
        a, b = (0.0, max(U[0], 0.0) + 9.0 * sl) if half > 0 else (min(U[0], 0.0) - 9.0 * sl, 0.0)
        zg, wg = np.polynomial.legendre.leggauss(160)
        u1 = 0.5 * (b - a) * zg + 0.5 * (a + b)
        w1 = 0.5 * (b - a) * wg * math.sqrt(lam / math.pi) * np.exp(-lam * (u1 - U[0]) ** 2)
    zl, wl = np.polynomial.laguerre.laggauss(8)
    s = zl / lam  # weight lam exp(-lam s) ds: exact for K = 2
    ws = wl
    g = np.meshgrid(u1, u2, u3, s, indexing="ij")
    w = np.einsum("a,b,c,d->abcd", w1, w2, w2, ws)
    return [x.ravel() for x in g], w.ravel()


def _psi(nodes):
    u1, u2, u3, s = nodes
    return np.stack([np.ones_like(u1), u1, u2, u3, 0.5 * (u1 * u1 + u2 * u2 + u3 * u3 + s)])


def _slope_values(a, nodes):
    return a @ _psi(nodes)


def _micro(full_nodes, full_w, rhs):
    P = _psi(full_nodes)
    M = (P * full_w) @ P.T
    return np.linalg.solve(M, rhs)


def _slopes(W, dW):
    rho, U, p, lam = _prim(W)
    nodes, w = _nodes(U, lam, 0)
    a = [_micro(nodes, w, dW[i] / rho) for i in range(3)]
    P = _psi(nodes)
    au = sum(_slope_values(a[i], nodes) * nodes[i] for i in range(3))
    A = _micro(nodes, w, -(P * w) @ au)
    return a, A


def _time_integrals(f, d, tau_n):
    """int_0^d f(t) dt by composite Gauss-Legendre, refined near t = 0
    where exp(-t/tau_n) varies fastest."""
    z, wz = np.polynomial.legendre.leggauss(40)
    cuts = [0.0]
    x = tau_n
    while x < d:
        cuts.append(x)
        x *= 3.0
    cuts.append(d)
    tot = 0.0
    for a, b in zip(cuts[:-1], cuts[1:]):
        t = 0.5 * (b - a) * z + 0.5 * (a + b)
        tot = tot + 0.5 * (b - a) * sum(wi * f(ti) for wi, ti in zip(wz, t))
    return tot


def brute_force(Wl, dWl, Wr, dWr, dt, viscous=False, mu=0.0, tau_eps=0.01, tau_c=1.0, prandtl=1.0):
    rl, Ul, pl, laml = _prim(Wl)
    rr, Ur, pr, lamr = _prim(Wr)
    al, Al = _slopes(Wl, dWl)
    ar, Ar = _slopes(Wr, dWr)
    nl, wl = _nodes(Ul, laml, +1)
    nr, wr = _nodes(Ur, lamr, -1)
    Pl, Pr = _psi(nl), _psi(nr)
    Wc = rl * (Pl @ wl) + rr * (Pr @ wr)
    dWc = np.array([rl * (Pl * wl) @ _slope_values(al[i], nl) + rr * (Pr * wr) @ _slope_values(ar[i], nr)
                    for i in range(3)])
    rc, Uc, pc, lamc = _prim(Wc)
    ac, Ac = _slopes(Wc, dWc)
    nc_, wc = _nodes(Uc, lamc, 0)
    Pc = _psi(nc_)
    tau = mu / pc if viscous else 0.0
    jump = abs((pl - pr) / (pl + pr)) * dt
    tau_n = (mu / pc if viscous else tau_eps * dt) + tau_c * jump

    # velocity moments of each piece of Eq. 2nd-flux (with and without u1)
    def pieces(nodes, w, P, a, A):
        au = sum(_slope_values(a[i], nodes) * nodes[i] for i in range(3))
        Av = _slope_values(A, nodes)
        out = {}
        for name, extra in (("F", nodes[0]), ("W", np.ones_like(nodes[0]))):
            out[name] = ((P * w) @ extra, (P * w) @ (au * extra), (P * w) @ (Av * extra))
        # heat flux density (u1 - U1) (|u - U|^2 + xi^2) / 2 about the
        # interface equilibrium velocity (a scalar moment)
        c = [nodes[i] - Uc[i] for i in range(3)]
        qv = c[0] * 0.5 * (c[0] * c[0] + c[1] * c[1] + c[2] * c[2] + nodes[3])
        out["Q"] = (w @ qv, w @ (au * qv), w @ (Av * qv))
        return out

    mc = pieces(nc_, wc, Pc, ac, Ac)
    ml = pieces(nl, wl, Pl, al, Al)
    mr = pieces(nr, wr, Pr, ar, Ar)

    def f_moments(kind, t):
        e = math.exp(-t / tau_n)
        C1, C2, C3 = 1.0 - e, (t + tau) * e - tau, t - tau + tau * e
        c0, c1, c2 = mc[kind]
        l0, l1, l2 = ml[kind]
        r0, r1, r2 = mr[kind]
        return (rc * (C1 * c0 + C2 * c1 + C3 * c2)
                + rl * e * (l0 - (tau + t) * l1 - tau * l2)
                + rr * e * (r0 - (tau + t) * r1 - tau * r2))

    Fh = _time_integrals(lambda t: f_moments("F", t), 0.5 * dt, tau_n)
    F = _time_integrals(lambda t: f_moments("F", t), dt, tau_n)
    if viscous and prandtl != 1.0:
        # the energy flux gains (1/Pr - 1) times the time integral of the heat flux
        Fh = Fh.copy()
        F = F.copy()
        Fh[4] += (1.0 / prandtl - 1.0) * _time_integrals(lambda t: f_moments("Q", t), 0.5 * dt, tau_n)
        F[4] += (1.0 / prandtl - 1.0) * _time_integrals(lambda t: f_moments("Q", t), dt, tau_n)
    return Fh, F, f_moments("W", 0.0), f_moments("W", dt)


def _random_state(rng, scale_grad=0.3):
    rho = rng.uniform(0.5, 2.0)
    U = rng.uniform(-1.0, 1.0, size=3)
    p = rng.uniform(0.5, 2.0)
    W = np.array([rho, rho * U[0], rho * U[1], rho * U[2], p / (GAMMA - 1) + 0.5 * rho * U @ U])
    dW = rng.normal(size=(3, 5)) * scale_grad
    return W, dW


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("viscous", [False, True])
def test_flux_matches_brute_force_quadrature(oracle_mod, seed, viscous):
    rng = np.random.default_rng(seed)
    Wl, dWl = _random_state(rng)
    Wr, dWr = _random_state(rng)
    dt = 0.02
    mu = 2e-3 if viscous else 0.0
    p = oracle_mod.params(viscous=int(viscous), mu=mu)
    got = oracle_mod.gp_flux(p, Wl, dWl, Wr, dWr, dt)
    ref = brute_force(Wl, dWl, Wr, dWr, dt, viscous=viscous, mu=mu)
    for g, r, name in zip(got, ref, ("Fh", "F", "W0", "Wdt")):
        scale = np.abs(r).max()
        assert np.abs(g - r).max() < 1e-11 * scale, (name, g, r)


@pytest.mark.parametrize("seed", [3, 4])
def test_prandtl_fix_matches_brute_force_quadrature(oracle_mod, seed):
    """Pr = 0.72: the energy flux gains (1/Pr - 1) times the time integral of
    the heat flux of the interface distribution, here integrated directly
    from its definition over velocity space and time."""
    rng = np.random.default_rng(seed)
    Wl, dWl = _random_state(rng)
    Wr, dWr = _random_state(rng)
    dt, mu = 0.02, 2e-3
    got = oracle_mod.gp_flux(oracle_mod.params(viscous=1, mu=mu, prandtl=0.72), Wl, dWl, Wr, dWr, dt)
    base = oracle_mod.gp_flux(oracle_mod.params(viscous=1, mu=mu), Wl, dWl, Wr, dWr, dt)
    ref = brute_force(Wl, dWl, Wr, dWr, dt, viscous=True, mu=mu, prandtl=0.72)
    for g, r, name in zip(got, ref, ("Fh", "F", "W0", "Wdt")):
        scale = np.abs(r).max()
        assert np.abs(g - r).max() < 1e-11 * scale, (name, g, r)
    # only the energy flux moves, and by a visible amount
    for i in (0, 1):
        np.testing.assert_array_equal(got[i][:4], base[i][:4])
        assert abs(got[i][4] - base[i][4]) > 1e-6 * abs(base[i][4])
    np.testing.assert_array_equal(got[2], base[2])
    np.testing.assert_array_equal(got[3], base[3])


@pytest.mark.parametrize("U", [(0.0, 0.0, 0.0), (0.4, -0.3, 0.2)])
def test_prandtl_fix_scales_the_fourier_heat_flux(oracle_mod, U):
    """Gas with uniform pressure and velocity and a linear temperature
    T = p / rho = T0 + s x1 (R = 1), smooth solver: the energy flux over
    [0, d] is the convected energy plus the Fourier heat flux
    -kappa s d with kappa = mu c_p / Pr, c_p = gamma / (gamma - 1) (the BGK
    model alone gives Pr = 1).  Holds for a moving gas too (the correction
    measures the heat flux about the gas velocity)."""
    p0, T0, s_, mu, dt = 1.0, 1.2, 0.3, 2e-3, 0.01
    U = np.array(U)
    rho = p0 / T0
    drho = -p0 * s_ / T0 ** 2
    W = np.array([rho, rho * U[0], rho * U[1], rho * U[2], p0 / (GAMMA - 1) + 0.5 * rho * U @ U])
    dW = np.zeros((3, 5))
    dW[0] = [drho, drho * U[0], drho * U[1], drho * U[2], 0.5 * drho * U @ U]
    cp = GAMMA / (GAMMA - 1.0)
    F = {}
    for pr in (1.0, 0.72):
        F[pr] = oracle_mod.gp_flux(oracle_mod.params(viscous=1, mu=mu, smooth_flux=1, prandtl=pr),
                                   W, dW, W, dW, dt)
    for i, d in ((0, 0.5 * dt), (1, dt)):
        if not U.any():
            np.testing.assert_allclose(F[1.0][i][4], -mu * cp * s_ * d, rtol=1e-12)
            np.testing.assert_allclose(F[0.72][i][4], -mu * cp * s_ * d / 0.72, rtol=1e-12)
        np.testing.assert_allclose(F[0.72][i][4] - F[1.0][i][4], (1 / 0.72 - 1) * (-mu * cp * s_ * d),
                                   rtol=1e-10)


def test_uniform_flow_gives_euler_flux(oracle_mod):
    rng = np.random.default_rng(5)
    W, _ = _random_state(rng)
    z = np.zeros((3, 5))
    rho, U, p, _ = _prim(W)
    euler = np.array([rho * U[0], rho * U[0] ** 2 + p, rho * U[0] * U[1], rho * U[0] * U[2],
                      U[0] * (W[4] + p)])
    for smooth in (0, 1):
        Fh, F, W0, Wdt = oracle_mod.gp_flux(oracle_mod.params(smooth_flux=smooth), W, z, W, z, 0.05)
        np.testing.assert_allclose(Fh, 0.025 * euler, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(F, 0.05 * euler, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(W0, W, rtol=1e-13)
        np.testing.assert_allclose(Wdt, W, rtol=1e-13)


def test_mirror_antisymmetry(oracle_mod):
    """Swapping the sides and reversing the normal (u1 -> -u1, x1 -> -x1)
    reverses the flux and mirrors the interface state."""
    rng = np.random.default_rng(9)
    Wl, dWl = _random_state(rng)
    Wr, dWr = _random_state(rng)
    P = np.diag([1.0, -1.0, 1.0, 1.0, 1.0])

    def mirror_grad(dW):
        out = dW @ P.T
        out[0] = -out[0]
        return out

    p = oracle_mod.params()
    a = oracle_mod.gp_flux(p, Wl, dWl, Wr, dWr, 0.03)
    b = oracle_mod.gp_flux(p, P @ Wr, mirror_grad(dWr), P @ Wl, mirror_grad(dWl), 0.03)
    np.testing.assert_allclose(b[0], -(P @ a[0]), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b[1], -(P @ a[1]), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b[2], P @ a[2], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b[3], P @ a[3], rtol=1e-12, atol=1e-15)


def test_smooth_flux_linear_data_limit(oracle_mod):
    """Smooth solver with tau = 0 and identical smooth sides: the interface
    state evolves as W(t) = W - t dF/dx1 (Euler equations, to first order in
    t since f = g(1 + A t) is linear in time), checked against the Euler
    flux Jacobian applied to the normal gradient."""
    rng = np.random.default_rng(12)
    W, dW = _random_state(rng, 0.2)
    dt = 1e-3
    _, _, W0, Wdt = oracle_mod.gp_flux(oracle_mod.params(smooth_flux=1), W, dW, W, dW, dt)

    def euler_flux(Wv, axis):
        rho, U, p, _ = _prim(Wv)
        f = np.array([rho * U[axis], rho * U[0] * U[axis], rho * U[1] * U[axis], rho * U[2] * U[axis],
                      U[axis] * (Wv[4] + p)])
        f[1 + axis] += p
        return f

    div = np.zeros(5)
    h = 1e-6
    for axis in range(3):
        J = np.stack([(euler_flux(W + h * e, axis) - euler_flux(W - h * e, axis)) / (2 * h)
                      for e in np.eye(5)], axis=1)
        div += J @ dW[axis]
    np.testing.assert_allclose(W0, W, rtol=1e-13)
    np.testing.assert_allclose((Wdt - W0) / dt, -div, rtol=1e-7, atol=1e-9)
