"""FP64 CPU restatement of one two-stage step in plain PyTorch operations, so
that torch.autograd gives the step's exact reverse sweep on the CPU.

TEST INFRASTRUCTURE ONLY: the tests use it as a second, independent check of
the library's adjoint (gks_adjoint_step); nothing in the product imports it.

Scope: third-order reconstruction with linear weights (R = P^2 = M2 d, Sec.
4.1) or the multi-resolution WENO weights of Sec. 4.2-4.3 (beta_0 by the
two-step construction from the neighbours' P1 slopes), or the second-order
one (Eq. final_weno_expression-2nd), with the Gauss-point positivity check
that falls back to the cell average (reading R9), the full gas-kinetic solver (Eq. 2nd-flux with the equilibrium state of
Eq. new-equ-part) or the smooth one (Eq. 2nd-smooth-flux), Euler (tau = 0) or
Navier-Stokes (tau = mu / p_c, Sec. 2.2) with the heat-flux correction for a
Prandtl number other than 1 (the reading of the oracle), periodic meshes or
boundary faces that are open, slip or non-slip walls or fixed (Sec. 4.4 and
the oracle's readings: one-sided stencils, the linear-weight boundary cells'
least-squares first-order fit, the ghosts at the Gauss points),
the S2O4 step of Sec. 3 with the linear flux fit (Eqs. linear-system, s2o4)
and the cell-averaged gradients from the divergence theorem (Eq.
gauss-formula).  Geometry, connectivity and the stencil operators M2 come
from the C oracle (they do not depend on the state); everything that does
is written here afresh: the face frame, the Maxwellian moments as products
of one-dimensional moments (sparse polynomials in u, v, w, xi^2), the
micro-slopes by a 5x5 linear solve, the time integrals of the distribution,
the stage sums."""
import math

import numpy as np
import torch

PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


# ----------------------------------------------------------- polynomials --
# a polynomial in (u, v, w, s = xi^2) is a dict {(a, b, c, d): coefficient}

def _pmul(p, q):
    out = {}
    for ka, ca in p.items():
        for kb, cb in q.items():
            k = (ka[0] + kb[0], ka[1] + kb[1], ka[2] + kb[2], ka[3] + kb[3])
            out[k] = out[k] + ca * cb if k in out else ca * cb
    return out


def _padd(p, q):
    out = dict(p)
    for k, c in q.items():
        out[k] = out[k] + c if k in out else c
    return out


_PSI = [{(0, 0, 0, 0): 1.0}, {(1, 0, 0, 0): 1.0}, {(0, 1, 0, 0): 1.0}, {(0, 0, 1, 0): 1.0},
        {(2, 0, 0, 0): 0.5, (0, 2, 0, 0): 0.5, (0, 0, 2, 0): 0.5, (0, 0, 0, 1): 0.5}]
_U = [{(1, 0, 0, 0): 1.0}, {(0, 1, 0, 0): 1.0}, {(0, 0, 1, 0): 1.0}]


def _slope_poly(a):
    """a . psi for a [N, 5]"""
    out = {}
    for k in range(5):
        out = _padd(out, {key: c * a[:, k] for key, c in _PSI[k].items()})
    return out


# ------------------------------------------------------ Maxwellian moments --
class _Moments:
    """Normalised moments <u^a v^b w^c xi^2d> of a Maxwellian (U, lam), with
    u restricted to u > 0 (half = +1), u < 0 (-1) or free (0)."""

    def __init__(self, U, lam, K, half, order=8):
        h = 0.5 / lam
        self.tab = []
        for axis in range(3):
            m = [None] * (order + 1)
            Ua = U[:, axis]
            if axis == 0 and half != 0:
                sg = float(half)
                m[0] = 0.5 * torch.special.erfc(-sg * torch.sqrt(lam) * Ua)
                m[1] = Ua * m[0] + sg * torch.exp(-lam * Ua * Ua) / (2.0 * torch.sqrt(math.pi * lam))
            else:
                m[0] = torch.ones_like(Ua)
                m[1] = Ua
            for n in range(order - 1):
                m[n + 2] = Ua * m[n + 1] + (n + 1) * h * m[n]
            self.tab.append(m)
        self.xi = [torch.ones_like(lam), K * h, (K * K + 2.0 * K) * h * h, K * (K + 2.0) * (K + 4.0) * h ** 3]

    def of(self, poly):
        tot = 0.0
        for (a, b, c, d), coef in poly.items():
            tot = tot + coef * self.tab[0][a] * self.tab[1][b] * self.tab[2][c] * self.xi[d]
        return tot

    def psi(self, poly):
        """the 5-vector <poly psi_k>, [N, 5]"""
        return torch.stack([self.of(_pmul(poly, _PSI[k])) for k in range(5)], dim=1)

    def gram(self):
        """<psi_k psi_j>, [N, 5, 5]"""
        rows = [self.psi(_PSI[k]) for k in range(5)]
        return torch.stack(rows, dim=1)


def _prim(W, gamma):
    rho = W[:, 0]
    U = W[:, 1:4] / rho[:, None]
    p = (gamma - 1.0) * (W[:, 4] - 0.5 * rho * (U * U).sum(1))
    return rho, U, p, rho / (2.0 * p)


def _slopes(full, rho, dW):
    """micro-slopes a_i (<(a_i . psi) psi> = dW_i / rho) and A
    (<(A + sum_i a_i u_i) . psi> = 0) by direct solves; dW [N, 3, 5]"""
    G = full.gram()
    a = [torch.linalg.solve(G, dW[:, i] / rho[:, None]) for i in range(3)]
    rhs = 0.0
    for i in range(3):
        rhs = rhs + full.psi(_pmul(_U[i], _slope_poly(a[i])))
    A = torch.linalg.solve(G, -rhs)
    return a, A


def point_flux(Wl, gl, Wr, gr, dt, gamma=1.4, tau_eps=0.01, tau_c=1.0, mu=0.0, viscous=False, smooth=False,
               prandtl=1.0):
    """Kinetic solution at N points in the face frame (x1 along the normal):
    states [N, 5], gradients [N, 3, 5] (d/dx_i).  Returns the flux integrals
    over [0, dt/2] and [0, dt] and the states at t = 0 and dt."""
    K = (5.0 - 3.0 * gamma) / (gamma - 1.0)
    rl, Ul, pl, laml = _prim(Wl, gamma)
    rr, Ur, pr, lamr = _prim(Wr, gamma)
    fl, fr = _Moments(Ul, laml, K, 0), _Moments(Ur, lamr, K, 0)
    hl, hr = _Moments(Ul, laml, K, +1), _Moments(Ur, lamr, K, -1)
    al, Al = _slopes(fl, rl, gl)
    ar, Ar = _slopes(fr, rr, gr)
    one = {(0, 0, 0, 0): 1.0}
    Wc = rl[:, None] * hl.psi(one) + rr[:, None] * hr.psi(one)
    dWc = torch.stack([rl[:, None] * hl.psi(_slope_poly(al[i])) + rr[:, None] * hr.psi(_slope_poly(ar[i]))
                       for i in range(3)], dim=1)
    rc, Uc, pc, lamc = _prim(Wc, gamma)
    fc = _Moments(Uc, lamc, K, 0)
    ac, Ac = _slopes(fc, rc, dWc)
    jump = tau_c * torch.abs((pl - pr) / (pl + pr)) * dt
    tau = mu / pc if viscous else torch.zeros_like(pc)
    tau_n = tau + jump if viscous else tau_eps * dt + jump
    tau = tau[:, None]

    def au(a):  # sum_i (a_i . psi) u_i
        out = {}
        for i in range(3):
            out = _padd(out, _pmul(_U[i], _slope_poly(a[i])))
        return out
    u1 = _U[0]
    c_f, c_fa, c_fA = fc.psi(u1), fc.psi(_pmul(u1, au(ac))), fc.psi(_pmul(u1, _slope_poly(Ac)))
    c_wa, c_wA = fc.psi(au(ac)), fc.psi(_slope_poly(Ac))
    c_w = fc.psi(one)
    sides = [(rl, hl, al, Al), (rr, hr, ar, Ar)]
    kin = [(r[:, None], h.psi(u1), h.psi(_pmul(u1, au(a))), h.psi(_pmul(u1, _slope_poly(A))), h.psi(one),
            h.psi(au(a)), h.psi(_slope_poly(A))) for r, h, a, A in sides]
    rcc = rc[:, None]

    def flux(d):
        """int_0^d of the flux and of the state (the latter for the Pr fix)"""
        if smooth:
            F = rcc * (d * c_f - tau * d * (c_fa + c_fA) + 0.5 * d * d * c_fA)
            IW = rcc * (d * c_w - tau * d * (c_wa + c_wA) + 0.5 * d * d * c_wA)
            return F, IW
        E = torch.exp(-d / tau_n)[:, None]
        tn = tau_n[:, None]
        k0 = tn * (1.0 - E)
        k1 = tn * tn * (1.0 - E) - tn * d * E
        q1, q2, q3 = d - k0, k1 + tau * k0 - tau * d, 0.5 * d * d - tau * d + tau * k0
        F = rcc * (q1 * c_f + q2 * c_fa + q3 * c_fA)
        IW = rcc * (q1 * c_w + q2 * c_wa + q3 * c_wA)
        for r, f0, f1, f2, w0, w1, w2 in kin:
            F = F + r * (k0 * f0 - (tau * k0 + k1) * f1 - tau * k0 * f2)
            IW = IW + r * (k0 * w0 - (tau * k0 + k1) * w1 - tau * k0 * w2)
        return F, IW

    def fixed(F, IW):
        if not (viscous and prandtl != 1.0):
            return F
        # F_E += (1/Pr - 1) q, q the heat flux about U^c (expanded into F and IW)
        uu = 0.5 * (Uc * Uc).sum(1)
        qf = F[:, 4] - (Uc * F[:, 1:4]).sum(1) + uu * F[:, 0]
        qw = IW[:, 4] - (Uc * IW[:, 1:4]).sum(1) + uu * IW[:, 0]
        return torch.cat([F[:, :4], (F[:, 4] + (1.0 / prandtl - 1.0) * (qf - Uc[:, 0] * qw))[:, None]], dim=1)

    def state(t):
        if smooth:
            return rcc * (c_w - tau * (c_wa + c_wA) + t * c_wA)
        e = torch.exp(-t / tau_n)[:, None]
        out = rcc * ((1.0 - e) * c_w + ((t + tau) * e - tau) * c_wa + (t - tau + tau * e) * c_wA)
        for r, _, _, _, w0, w1, w2 in kin:
            out = out + r * (e * w0 - (tau + t) * e * w1 - tau * e * w2)
        return out
    return fixed(*flux(0.5 * dt)), fixed(*flux(dt)), state(0.0), state(dt)


# -------------------------------------------------------------- the step --
def _frame(n):
    """rows (n, t1, t2), a right-handed orthonormal frame per face, [nf, 3, 3]"""
    e = torch.zeros_like(n)
    use_x = n[:, 0].abs() < 0.9
    e[use_x, 0] = 1.0
    e[~use_x, 1] = 1.0
    t1 = e - (e * n).sum(1, keepdim=True) * n
    t1 = t1 / torch.linalg.norm(t1, dim=1, keepdim=True)
    t2 = torch.cross(n, t1, dim=1)
    return torch.stack([n, t1, t2], dim=1)


OPEN, SLIP, FIXED, NOSLIP, ISOTHERMAL, MOVING = 0, 1, 2, 3, 4, 5


def _moving_ghost(W, g, gamma, Uw):
    """non-slip adiabatic wall moving with Uw [F, 3] (face frame): the
    at-rest ghost taken in the wall's frame, m -> 2 rho Uw - m,
    E -> E - 2 Uw.m + 2 rho |Uw|^2; derivatives d rho -> -d rho,
    dm -> dm - 2 Uw d rho, dE -> -dE + 2 Uw.dm - 2 |Uw|^2 d rho"""
    rho, m, E = W[:, 0], W[:, 1:4], W[:, 4]
    uu = (Uw * Uw).sum(1)
    Wl = torch.cat([rho[:, None], 2.0 * rho[:, None] * Uw - m,
                    (E - 2.0 * (Uw * m).sum(1) + 2.0 * rho * uu)[:, None]], dim=1)
    dr, dm, dE = g[:, :, 0], g[:, :, 1:4], g[:, :, 4]
    gl = torch.cat([-dr[:, :, None], dm - 2.0 * Uw[:, None, :] * dr[:, :, None],
                    (-dE + 2.0 * (Uw[:, None, :] * dm).sum(2) - 2.0 * uu[:, None] * dr)[:, :, None]], dim=2)
    return Wl, gl


def _isothermal_ghost(W, g, gamma, Tw):
    """Sec. 4.4 non-slip isothermal wall (face frame, T = p / rho): pressure
    kept, velocity reversed, T -> 2 Tw - T; dU, dT kept, dp reversed, back to
    conservative derivatives; W [F, 5], g [F, 3, 5]"""
    gm1 = gamma - 1.0
    rho = W[:, 0]
    U = W[:, 1:4] / rho[:, None]
    Q = 0.5 * (U * U).sum(1)
    p = gm1 * (W[:, 4] - rho * Q)
    Tr = p / rho
    Tl = 2.0 * Tw - Tr
    rl = p / Tl
    Wl = torch.cat([rl[:, None], -rl[:, None] * U, (p / gm1 + rl * Q)[:, None]], dim=1)
    dU = (g[:, :, 1:4] - g[:, :, :1] * U[:, None, :]) / rho[:, None, None]          # [F, 3, 3]
    dQ = (U[:, None, :] * dU).sum(2)                                                 # [F, 3]
    dp = gm1 * (g[:, :, 4] - g[:, :, 0] * Q[:, None] - rho[:, None] * dQ)
    dT = (dp - g[:, :, 0] * Tr[:, None]) / rho[:, None]
    dpl = -dp
    drl = (dpl - dT * rl[:, None]) / Tl[:, None]
    gm = drl[:, :, None] * (-U[:, None, :]) + dU * rl[:, None, None]
    ge = drl * Q[:, None] - rl[:, None] * dQ + dpl / gm1
    return Wl, torch.cat([drl[:, :, None], gm, ge[:, :, None]], dim=2)


class Step:
    """One step on an oracle mesh.  kinds[nc][4]: boundary kind per local face
    (read on boundary faces); fixed = (W [5, nc], dW [15, nc]) the state that
    fixed faces hold."""

    def __init__(self, om, gamma=1.4, tau_eps=0.01, tau_c=1.0, mu=0.0, viscous=False, smooth=False, prandtl=1.0,
                 weno=False, eps=1e-8, kinds=None, fixed=None, order=3, wall_temperature=1.0,
                 wall_velocity=(0.0, 0.0, 0.0)):
        geo, top = om.geometry(), om.topology()
        M1, M2 = om.stencils()
        self.weno, self.eps, self.order, self.twall = weno, eps, order, wall_temperature
        self.uwall = torch.tensor(wall_velocity, dtype=torch.float64)
        t = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64)
        self.vol, self.mom = t(geo["vol"]), t(geo["mom2"])
        self.area, self.n = t(geo["farea"]), t(geo["fnorm"])
        self.gpl, self.gpr = t(geo["gp_l"]), t(geo["gp_r"])
        self.lr = torch.as_tensor(top["face_lr"])
        self.nbr = torch.as_tensor(top["nbr"])
        self.M2 = t(M2)
        self.M1 = t(M1)
        nc, nf = self.vol.shape[0], self.n.shape[0]
        # boundary faces: the kind of each (from the interior cell's local face)
        self.fkind = torch.full((nf,), -1, dtype=torch.int64)
        csr_face, csr_sign = top["csr_face"], top["csr_sign"]
        nbr = top["nbr"]
        if (nbr < 0).any():
            kinds = np.zeros((nc, 4), np.int64) if kinds is None else np.asarray(kinds).reshape(nc, 4)
            cells, lf = np.nonzero(nbr < 0)
            self.fkind[torch.as_tensor(csr_face[cells, lf])] = torch.as_tensor(kinds[cells, lf].astype(np.int64))
        self.bcell = torch.as_tensor((nbr < 0).any(axis=1))
        self.nmask = torch.as_tensor(nbr >= 0, dtype=torch.float64)        # [nc, 4]
        self.nbr_safe = torch.where(self.nbr >= 0, self.nbr, torch.arange(nc)[:, None])
        # centroid offsets to the neighbours (periodic images from the face geometry)
        off = np.zeros((nc, 4, 3))
        gl, gr = geo["gp_l"][:, 0], geo["gp_r"][:, 0]
        for f in range(4):
            fi = csr_face[:, f]
            d = np.where((csr_sign[:, f] > 0)[:, None], gl[fi] - gr[fi], gr[fi] - gl[fi])
            off[:, f] = np.where((nbr[:, f] >= 0)[:, None], d, 0.0)
        self.off = t(off)
        # each cell's own Gauss points (offsets from its centroid), [nc, 12, 3]
        own = np.zeros((nc, 4, 3, 3))
        for f in range(4):
            fi = csr_face[:, f]
            own[:, f] = np.where((csr_sign[:, f] > 0)[:, None, None], geo["gp_l"][fi], geo["gp_r"][fi])
        self.gp_own = t(own.reshape(nc, 12, 3))
        self.fixed = None if fixed is None else (t(fixed[0]).T, t(fixed[1]).T.reshape(-1, 5, 3))
        self.R = _frame(self.n)
        self.kw = dict(gamma=gamma, tau_eps=tau_eps, tau_c=tau_c, mu=mu, viscous=viscous, smooth=smooth,
                       prandtl=prandtl)

    def _recon(self, W, dW):
        """R's coefficients a in the zero-mean basis per cell and component,
        [nc, 5, 9]: P2 = M2 d (linear weights), or the WENO combination"""
        Q0 = W.T                                   # [nc, 5]
        m = self.nmask
        Qn = W.T[self.nbr_safe]                    # [nc, 4, 5] (a missing neighbour reads the cell itself)
        G = dW.T.reshape(-1, 5, 3)[self.nbr_safe] * m[:, :, None, None]                 # [nc, 4, 5, 3]
        dq = ((Qn - Q0[:, None, :]) * m[:, :, None]).permute(0, 2, 1)                   # [nc, 5, 4]
        d = torch.cat([dq, G.permute(0, 2, 1, 3).reshape(-1, 5, 12)], dim=2)          # [nc, 5, 16]
        a = torch.einsum("ckj,cqj->cqk", self.M2, d)
        if self.weno:
            a = self._weno(a, dq)
        elif self.order == 2:  # R = P1
            b = torch.einsum("cij,cqj->cqi", self.M1, dq)
            a = torch.cat([b, torch.zeros_like(a[:, :, 3:])], dim=2)
        elif self.bcell.any():
            a = torch.where(self.bcell[:, None, None], self._linear_fit(dq, G), a)
        return self._positivity(a, Q0), Q0

    def _positivity(self, a, Q0):
        """R at the cell's 12 face Gauss points; a negative density or
        pressure at any of them makes the cell constant (R = P0, all
        components; a decision, not differentiated)"""
        with torch.no_grad():
            X = self.gp_own                                                    # [nc, 12, 3]
            val = Q0[:, None, :] + torch.einsum("cqk,cgk->cgq", a[:, :, :3], X)
            for q, (i, j) in enumerate(PAIRS):
                val = val + a[:, None, :, 3 + q] * (X[:, :, i] * X[:, :, j] - self.mom[:, q][:, None])[:, :, None]
            rho = val[:, :, 0]
            pres = (self.kw["gamma"] - 1.0) * (val[:, :, 4] - 0.5 * (val[:, :, 1:4] ** 2).sum(2) / rho)
            bad = ((rho <= 0.0) | (pres <= 0.0)).any(dim=1)
        self.fallbacks.append(bad)
        return torch.where(bad[:, None, None], torch.zeros_like(a), a)

    def _linear_fit(self, dq, G):
        """Sec. 4.4 with linear weights: a boundary cell's first-order
        least-squares fit to its neighbours' averages (d_r . b = dQ_r) and
        averaged gradients (h0 b = h0 grad Q_r), [nc, 5, 9]"""
        h2 = self.vol ** (2.0 / 3.0)
        m, off = self.nmask, self.off
        A = torch.einsum("cr,cri,crj->cij", m, off, off) + (m.sum(1) * h2)[:, None, None] * torch.eye(3)
        rhs = torch.einsum("cri,cqr->cqi", off, dq) + h2[:, None, None] * G.sum(1)      # [nc, 5, 3]
        b = torch.linalg.solve(A[:, None], rhs[..., None])[..., 0]
        return torch.cat([b, torch.zeros(b.shape[0], 5, 6, dtype=b.dtype)], dim=2)

    def _weno(self, a, dq):
        """Sec. 4.2-4.3: smoothness indicators of P1 (slopes b = M1 dQ), P2 and
        the two-step beta_0 (the neighbours' P1 slopes weighted by 1 +
        sigma1 / (eps + beta_0j)), nonlinear weights gamma (1 + (sigma /
        (eps + beta))^2), R = w2 p2 + w1 p1 + w0 p0 (readings R3-R6, R13)"""
        eps = self.eps
        v = self.vol[:, None]
        b = torch.einsum("cij,cqj->cqi", self.M1, dq)                                   # [nc, 5, 3]
        beta1 = v ** (2.0 / 3.0) * (b * b).sum(2)
        bn = b[self.nbr_safe]
        m = self.nmask[:, None, :]                                                     # [nc, 1, 4]
        b0j = v[:, :, None] ** (2.0 / 3.0) * (bn * bn).sum(3).permute(0, 2, 1)          # [nc, 5, 4]
        pair, npair = 0.0, 0.0
        for j in range(4):
            for k in range(j):
                pair = pair + m[:, :, j] * m[:, :, k] * torch.abs(b0j[:, :, j] - b0j[:, :, k])
                npair = npair + m[:, :, j] * m[:, :, k]
        s1 = (pair / npair) ** (4.0 / 3.0)
        w1 = m * (1.0 + s1[:, :, None] / (eps + b0j))
        beta0 = (w1 * b0j).sum(2) / w1.sum(2)
        g11, g01 = 10.0 / 11.0, 1.0 / 11.0
        if self.order == 2:
            # R^2nd = w1 p1 + w0 p0, sigma = |beta_1 - beta_0|^{4/3}
            sigma = torch.abs(beta1 - beta0) ** (4.0 / 3.0)
            w0 = g01 * (1.0 + (sigma / (eps + beta0)) ** 2)
            w1_ = g11 * (1.0 + (sigma / (eps + beta1)) ** 2)
            p1 = torch.cat([b / g11, torch.zeros_like(a[:, :, 3:])], dim=2)
            return (w1_ / (w0 + w1_))[:, :, None] * p1
        # beta_2 from the exact integrals of the quadratic over the cell
        lin = a[:, :, :3]
        H = torch.zeros(a.shape[0], 5, 3, 3, dtype=a.dtype)
        for q, (i, j) in enumerate(PAIRS):
            H[:, :, i, j] = H[:, :, i, j] + a[:, :, 3 + q]
            H[:, :, j, i] = H[:, :, j, i] + a[:, :, 3 + q]
        Mm = torch.zeros(a.shape[0], 3, 3, dtype=a.dtype)
        for q, (i, j) in enumerate(PAIRS):
            Mm[:, i, j] = self.mom[:, q]
            Mm[:, j, i] = self.mom[:, q]
        first = (lin * lin).sum(2) + torch.einsum("cqij,cjk,cqik->cq", H, Mm, H)
        second = sum(H[:, :, i, j] ** 2 for i in range(3) for j in range(i, 3))
        beta2 = v ** (2.0 / 3.0) * first + v ** (4.0 / 3.0) * second
        sigma = (0.5 * (torch.abs(beta2 - beta1) + torch.abs(beta2 - beta0))) ** (4.0 / 3.0)
        g2, g1, g0 = 100.0 / 111.0, 10.0 / 111.0, 1.0 / 111.0
        w = [g * (1.0 + (sigma / (eps + beta)) ** 2) for g, beta in ((g0, beta0), (g1, beta1), (g2, beta2))]
        ws = w[0] + w[1] + w[2]
        # p0 = Q0, p1 = (P1 - g01 P0) / g11, p2 = (P2 - g1 p1 - g0 p0) / g2; the constants all Q0
        p1 = torch.cat([b / g11, torch.zeros_like(a[:, :, 3:])], dim=2)
        p2 = (a - g1 * p1) / g2
        return (w[2] / ws)[:, :, None] * p2 + (w[1] / ws)[:, :, None] * p1

    def _eval(self, a, Q0, cells, X):
        """value [F, 5] and gradient [F, 3, 5] of R of `cells` at offsets X [F, 3]"""
        a, Q0, M = a[cells], Q0[cells], self.mom[cells]
        val = Q0 + torch.einsum("fqk,fk->fq", a[:, :, :3], X)
        grad = a[:, :, :3].permute(0, 2, 1).clone()
        for q, (i, j) in enumerate(PAIRS):
            val = val + a[:, :, 3 + q] * (X[:, i] * X[:, j] - M[:, q])[:, None]
            grad[:, i, :] = grad[:, i, :] + a[:, :, 3 + q] * X[:, j][:, None]
            grad[:, j, :] = grad[:, j, :] + a[:, :, 3 + q] * X[:, i][:, None]
        return val, grad

    def _to_local(self, R, W, g):
        m = torch.einsum("fij,fj->fi", R, W[:, 1:4])
        Wl = torch.cat([W[:, :1], m, W[:, 4:]], dim=1)
        gx = torch.einsum("fij,fjq->fiq", R, g)                       # derivative index
        gm = torch.einsum("fij,fkj->fki", R, gx[:, :, 1:4])            # momentum components
        gl = torch.cat([gx[:, :, :1], gm, gx[:, :, 4:]], dim=2)
        return Wl, gl

    def _to_global(self, R, F):
        m = torch.einsum("fji,fj->fi", R, F[:, 1:4])
        return torch.cat([F[:, :1], m, F[:, 4:]], dim=1)

    def _faces(self, W, dW, dt):
        """per face: sum_k w_k of Fh, F, W(0) n, W(dt) n (global frame)"""
        a, Q0 = self._recon(W, dW)
        L, Rr = self.lr[:, 0], self.lr[:, 1]
        Ls, Rs = torch.where(L >= 0, L, Rr), torch.where(Rr >= 0, Rr, L)   # a missing side starts as the other
        kind = self.fkind
        w = self.area / 3.0
        out = [0.0, 0.0, 0.0, 0.0]
        for k in range(3):
            XL = torch.where((L >= 0)[:, None], self.gpl[:, k], self.gpr[:, k])
            XR = torch.where((Rr >= 0)[:, None], self.gpr[:, k], self.gpl[:, k])
            vl, gl = self._eval(a, Q0, Ls, XL)
            vr, gr = self._eval(a, Q0, Rs, XR)
            Wl, gll = self._to_local(self.R, vl, gl)
            Wr, grl = self._to_local(self.R, vr, gr)
            sides = [[Wl, gll], [Wr, grl]]
            for side, missing in ((0, L < 0), (1, Rr < 0)):
                if not missing.any():
                    continue
                inner = Rs if side == 0 else Ls
                Xi = XR if side == 0 else XL
                Wg, gg = sides[side]
                # open: the interior cell's average with zero gradient
                ow, og = self._to_local(self.R, Q0[inner], torch.zeros_like(gg))
                sel = (missing & (kind == OPEN))[:, None]
                Wg = torch.where(sel, ow, Wg)
                gg = torch.where(sel[:, :, None], og, gg)
                if self.fixed is not None:
                    fW, fg = self.fixed[0][inner], self.fixed[1][inner].permute(0, 2, 1)   # [F, 5], [F, 3, 5]
                    fw, fgl = self._to_local(self.R, fW + torch.einsum("fiq,fi->fq", fg, Xi), fg)
                    sel = (missing & (kind == FIXED))[:, None]
                    Wg = torch.where(sel, fw, Wg)
                    gg = torch.where(sel[:, :, None], fgl, gg)
                # slip wall (face frame): rho U1 reversed; x1-derivatives reversed
                # except that of rho U1; x2-, x3-derivatives of rho U1 reversed
                sw = torch.tensor([1.0, -1.0, 1.0, 1.0, 1.0], dtype=Wg.dtype)
                sg = torch.tensor([[-1.0, 1.0, -1.0, -1.0, -1.0], [1.0, -1.0, 1.0, 1.0, 1.0],
                                   [1.0, -1.0, 1.0, 1.0, 1.0]], dtype=Wg.dtype)
                sel = (missing & (kind == SLIP))[:, None]
                Wg = torch.where(sel, Wg * sw, Wg)
                gg = torch.where(sel[:, :, None], gg * sg, gg)
                # non-slip wall at rest: momenta reversed, their derivatives kept;
                # every derivative of rho and rho E reversed
                nw = torch.tensor([1.0, -1.0, -1.0, -1.0, 1.0], dtype=Wg.dtype)
                ng = torch.tensor([-1.0, 1.0, 1.0, 1.0, -1.0], dtype=Wg.dtype)
                sel = (missing & (kind == NOSLIP))[:, None]
                Wg = torch.where(sel, Wg * nw, Wg)
                gg = torch.where(sel[:, :, None], gg * ng, gg)
                sel = missing & (kind == MOVING)
                if sel.any():
                    Uw = torch.einsum("fij,j->fi", self.R, self.uwall)
                    mw, mg = _moving_ghost(Wg, gg, self.kw["gamma"], Uw)
                    Wg = torch.where(sel[:, None], mw, Wg)
                    gg = torch.where(sel[:, None, None], mg, gg)
                sel = missing & (kind == ISOTHERMAL)
                if sel.any():
                    iw, ig = _isothermal_ghost(Wg, gg, self.kw["gamma"], self.twall)
                    Wg = torch.where(sel[:, None], iw, Wg)
                    gg = torch.where(sel[:, None, None], ig, gg)
                sides[side] = [Wg, gg]
            (Wl, gll), (Wr, grl) = sides
            Fh, F, W0, Wt = point_flux(Wl, gll, Wr, grl, dt, **self.kw)
            res = [self._to_global(self.R, x) for x in (Fh, F, W0, Wt)]
            for j in range(4):
                out[j] = out[j] + w[:, None] * res[j]
        return out

    def _cell_sum(self, per_face):
        """sum over each cell's faces with s = +1 as left cell, -1 as right; [nc, ...]"""
        nc = self.vol.shape[0]
        shape = (nc,) + tuple(per_face.shape[1:])
        out = torch.zeros(shape, dtype=per_face.dtype)
        L, R = self.lr[:, 0], self.lr[:, 1]
        out = out.index_add(0, L[L >= 0], per_face[L >= 0])
        return out.index_add(0, R[R >= 0], -per_face[R >= 0])

    def __call__(self, W, dW, dt):
        """(W [5, nc], dW [15, nc]) -> (W^{n+1}, grad W^{n+1}) with the step dt"""
        n = self.n
        vol = self.vol[:, None]
        self.fallbacks = []  # the positivity decisions of the two stages
        Fh, F, W0, Wt = self._faces(W, dW, dt)
        Ws = W.T - self._cell_sum(Fh) / vol
        half = 0.5 * (W0 + Wt)
        gs = self._cell_sum(half[:, :, None] * n[:, None, :]) / vol[:, :, None]
        S = self._cell_sum(8.0 / 3.0 * Fh - 1.0 / 3.0 * F)
        G = self._cell_sum(W0[:, :, None] * n[:, None, :])
        dWs = gs.reshape(-1, 15).T
        Fh2, F2, W02, Wt2 = self._faces(Ws.T, dWs, dt)
        Wn = W.T - (S + self._cell_sum(4.0 / 3.0 * (F2 - 2.0 * Fh2))) / vol
        gn = (G + self._cell_sum((Wt2 - W02)[:, :, None] * n[:, None, :])) / vol[:, :, None]
        return Wn.T, gn.reshape(-1, 15).T
