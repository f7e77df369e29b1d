"""Adjoint of the step (gks_adjoint_step) on the GPU, FP64, against central
finite differences (step 1e-6) of the forward map, both the GPU's and the
CPU oracle's, with the time step frozen:

    < lambda, (F(x + h v) - F(x - h v)) / 2h >  =  < J^T lambda, v >

for random adjoints lambda and directions v over all 20 values of every
cell; then a gradient through three chained steps (torch autograd over the
step function) of the total kinetic energy with respect to the initial
density field (velocity and pressure held), against finite differences of
the three-step run.  Unsupported configurations are rejected."""
import numpy as np
import pytest

from paper_2102_01366_gb300 import gks
from paper_2102_01366_gb300 import inputs as I

pytestmark = pytest.mark.gpu

H = 1e-6


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    from paper_2102_01366_gb300 import _build
    _build.build()
    gks.lib()
    return torch


def _case(seed=61, state="sine"):
    if state in ("open", "slip", "noslip", "fixed", "isothermal", "moving"):
        # open, wall or fixed-state ends on x, y and z periodic; a smooth moving state
        mesh = I.box_mesh((4, 3, 3), (1.0, 0.75, 0.75), (False, True, True), jitter=0.1, seed=seed)
        if state != "open":
            kind = {"slip": I.BC_SLIP_WALL, "noslip": I.BC_NOSLIP_WALL, "fixed": I.BC_FIXED,
                    "isothermal": I.BC_ISOTHERMAL_WALL, "moving": I.BC_MOVING_WALL}[state]
            mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): kind, (0, "hi"): kind})
        W, dW = I.sine_wave_state(mesh, k=8.0 * np.pi / 3.0, u=(0.6, 0.5, -0.3))
    elif state == "sine":
        mesh = I.box_mesh((3, 3, 3), jitter=0.1, seed=seed)
        W, dW = I.sine_wave_state(mesh, u=(0.8, 0.5, -0.3))
    else:  # a moving density and pressure slab: far-from-linear WENO weights
        mesh = I.box_mesh((4, 3, 3), jitter=0.1, seed=seed)
        W, dW = I.riemann_slab_state(mesh, inner=(1.0, 1.0), outer=(0.5, 0.6), mach=0.8)
    rng = np.random.Generator(np.random.PCG64(seed))
    W = W * (1.0 + 0.01 * rng.standard_normal(W.shape))
    dW = dW + 0.05 * rng.standard_normal(dW.shape)
    return mesh, W, dW, rng


def _dot(a, b):
    return float(sum((np.asarray(x) * np.asarray(y)).sum() for x, y in zip(a, b)))


@pytest.mark.parametrize("weno,smooth,viscous,state", [(0, 0, 0, "sine"), (0, 1, 0, "sine"), (0, 0, 1, "sine"),
                                                       (0, 1, 1, "sine"), (1, 0, 0, "sine"), (1, 0, 0, "slab"),
                                                       (1, 0, 1, "slab"), (1, 0, 0, "open"), (1, 0, 1, "open"),
                                                       (1, 0, 0, "slip"), (0, 0, 1, "noslip"), (1, 0, 0, "fixed"),
                                                       (0, 0, 1, "fixed"), (0, 0, 1, "isothermal"), (1, 0, 1, "moving")])
def test_adjoint_matches_finite_differences(cuda, oracle_mod, weno, smooth, viscous, state):
    """Viscous runs carry tau = mu / p_c and each side's time slope A
    through the reverse-mode point adjoint; weno = 1 differentiates the
    nonlinear weights (on the slab they move the gradient by ~10 % from the
    linear-weight one); open
    ends and slip and non-slip walls take their ghosts' adjoints; fixed ends
    hold a state set once (gks_set_fixed_state), a constant of the step.  The
    slab's many |x| terms (pairs of smoothness indicators, pressure jumps)
    sit close to their kinks, and so do some of the viscous WENO runs'
    (on the open box the difference quotient moves by 1.5e-6 between
    h = 1e-6 and 1e-7, converging on the adjoint), so those differences use
    a smaller step."""
    torch = cuda
    mesh, W, dW, rng = _case(state=state)
    H = 1e-7 if state == "slab" or (weno and viscous) else 1e-6
    g = gks.Mesh(mesh)
    kw = dict(weno=weno, cfl=0.5, smooth_flux=smooth, viscous=viscous, mu=0.01 * viscous,
              wall_velocity=(0.0, 0.4, -0.2) if state == "moving" else (0.0, 0.0, 0.0))
    s = gks.State(g, gks.params(precision=0, **kw))
    if state == "fixed":
        # the boundary state, set apart from the (perturbed) initialisations
        Wf, dWf = W * (1.0 + 0.02 * rng.standard_normal(W.shape)), 0.5 * dW
        s.set_fixed_state(Wf, dWf)
        mesh["fixed_state"] = (Wf, dWf)
    o = oracle_mod.Mesh(mesh)
    p = oracle_mod.params(**kw)
    dt = 0.5 * o.timestep(p, W)
    lam = (rng.standard_normal(W.shape), rng.standard_normal(dW.shape))
    v = (rng.standard_normal(W.shape) * np.abs(W).max(axis=1, keepdims=True),
         rng.standard_normal(dW.shape) * np.abs(dW).max())

    def gpu_step(Wx, dWx):
        s.init(Wx, dWx)
        s.step(1, dt, 0.0)
        return [x.cpu().numpy() for x in s.get()]

    jv_gpu = [(a - b) / (2 * H) for a, b in zip(gpu_step(W + H * v[0], dW + H * v[1]),
                                                 gpu_step(W - H * v[0], dW - H * v[1]))]
    op, om = o.step(p, W + H * v[0], dW + H * v[1], dt), o.step(p, W - H * v[0], dW - H * v[1], dt)
    jv_ora = [(op[0] - om[0]) / (2 * H), (op[1] - om[1]) / (2 * H)]
    lW, ldW = s.adjoint_step(torch.tensor(W), torch.tensor(dW), torch.tensor(lam[0]), torch.tensor(lam[1]), dt)
    jtl = (lW.cpu().numpy(), ldW.cpu().numpy())
    lhs_gpu, lhs_ora, rhs = _dot(lam, jv_gpu), _dot(lam, jv_ora), _dot(jtl, v)
    assert abs(lhs_gpu - rhs) < 1e-6 * abs(rhs), (lhs_gpu, rhs)
    assert abs(lhs_ora - rhs) < 1e-6 * abs(rhs), (lhs_ora, rhs)
    # a second call in a row on the same state gives the same result
    lW2, ldW2 = s.adjoint_step(torch.tensor(W), torch.tensor(dW), torch.tensor(lam[0]), torch.tensor(lam[1]), dt)
    assert torch.equal(lW, lW2) and torch.equal(ldW, ldW2)


@pytest.mark.parametrize("weno,smooth,state", [(0, 0, "sine"), (0, 1, "sine"), (1, 0, "noslip")])
def test_prandtl_fix_adjoint(cuda, oracle_mod, weno, smooth, state):
    """Pr = 0.72: the heat-flux correction's transpose (the uncorrected flux,
    the state integrals and the interface velocity it depends on) against
    central differences of the GPU and oracle forward maps."""
    torch = cuda
    mesh, W, dW, rng = _case(state=state)
    H = 1e-7 if weno else 1e-6
    g = gks.Mesh(mesh)
    kw = dict(weno=weno, cfl=0.5, smooth_flux=smooth, viscous=1, mu=0.01, prandtl=0.72)
    s = gks.State(g, gks.params(precision=0, **kw))
    o = oracle_mod.Mesh(mesh)
    p = oracle_mod.params(**kw)
    dt = 0.5 * o.timestep(p, W)
    lam = (rng.standard_normal(W.shape), rng.standard_normal(dW.shape))
    v = (rng.standard_normal(W.shape) * np.abs(W).max(axis=1, keepdims=True),
         rng.standard_normal(dW.shape) * np.abs(dW).max())

    def gpu_step(Wx, dWx):
        s.init(Wx, dWx)
        s.step(1, dt, 0.0)
        return [x.cpu().numpy() for x in s.get()]

    jv_gpu = [(a - b) / (2 * H) for a, b in zip(gpu_step(W + H * v[0], dW + H * v[1]),
                                                 gpu_step(W - H * v[0], dW - H * v[1]))]
    op, om = o.step(p, W + H * v[0], dW + H * v[1], dt), o.step(p, W - H * v[0], dW - H * v[1], dt)
    jv_ora = [(op[0] - om[0]) / (2 * H), (op[1] - om[1]) / (2 * H)]
    lW, ldW = s.adjoint_step(torch.tensor(W), torch.tensor(dW), torch.tensor(lam[0]), torch.tensor(lam[1]), dt)
    rhs = _dot((lW.cpu().numpy(), ldW.cpu().numpy()), v)
    assert abs(_dot(lam, jv_gpu) - rhs) < 1e-6 * abs(rhs), (_dot(lam, jv_gpu), rhs)
    assert abs(_dot(lam, jv_ora) - rhs) < 1e-6 * abs(rhs), (_dot(lam, jv_ora), rhs)


@pytest.mark.parametrize("weno", [0, 1])
def test_sphere_shell_adjoint(cuda, oracle_mod, weno):
    """The viscous sphere's configuration on a 1,080-cell shell: non-slip
    wall (with the linear weights' first-order wall cells or WENO), far
    field held at a set state, Pr = 0.72, pole wedges; one step's adjoint
    against central differences of the GPU and oracle forward maps."""
    torch = cuda
    mesh = I.sphere_shell_mesh(3, 6, 12, 0.5, 1.5, 1.08)
    W, dW = I.sine_wave_state(mesh, amp=0.2, k=2.0, u=(0.35, 0.15, 0.0), p=1 / 1.4)
    rng = np.random.Generator(np.random.PCG64(71))
    W = W * (1.0 + 0.01 * rng.standard_normal(W.shape))
    dW = dW + 0.05 * rng.standard_normal(dW.shape)
    mesh["fixed_state"] = (W, dW)
    H = 1e-7 if weno else 1e-6
    g = gks.Mesh(mesh)
    kw = dict(weno=weno, cfl=0.5, viscous=1, mu=0.01, prandtl=0.72)
    s = gks.State(g, gks.params(precision=0, **kw))
    s.set_fixed_state(W, dW)
    o = oracle_mod.Mesh(mesh)
    p = oracle_mod.params(**kw)
    dt = 0.5 * o.timestep(p, W)
    lam = (rng.standard_normal(W.shape), rng.standard_normal(dW.shape))
    v = (rng.standard_normal(W.shape) * np.abs(W).max(axis=1, keepdims=True),
         rng.standard_normal(dW.shape) * np.abs(dW).max())

    def gpu_step(Wx, dWx):
        s.init(Wx, dWx)
        s.step(1, dt, 0.0)
        return [x.cpu().numpy() for x in s.get()]

    jv_gpu = [(a - b) / (2 * H) for a, b in zip(gpu_step(W + H * v[0], dW + H * v[1]),
                                                 gpu_step(W - H * v[0], dW - H * v[1]))]
    op, om = o.step(p, W + H * v[0], dW + H * v[1], dt), o.step(p, W - H * v[0], dW - H * v[1], dt)
    jv_ora = [(op[0] - om[0]) / (2 * H), (op[1] - om[1]) / (2 * H)]
    lW, ldW = s.adjoint_step(torch.tensor(W), torch.tensor(dW), torch.tensor(lam[0]), torch.tensor(lam[1]), dt)
    rhs = _dot((lW.cpu().numpy(), ldW.cpu().numpy()), v)
    assert abs(_dot(lam, jv_gpu) - rhs) < 1e-6 * abs(rhs), (_dot(lam, jv_gpu), rhs)
    assert abs(_dot(lam, jv_ora) - rhs) < 1e-6 * abs(rhs), (_dot(lam, jv_ora), rhs)


def test_wall_force_gradient_on_the_sphere_shell(cuda):
    """J = x-component of the pressure force on the sphere (gks.wall_pressure_force)
    after 3 steps of the viscous shell (WENO, Pr 0.72, far field held at a
    set state); dJ/d rho_0 along a random direction (velocity and pressure
    held) by the chained adjoint, against a central difference of the
    forward runs."""
    torch = cuda
    mesh = I.sphere_shell_mesh(3, 6, 12, 0.5, 1.5, 1.08)
    W, dW = I.sine_wave_state(mesh, amp=0.2, k=2.0, u=(0.35, 0.15, 0.0), p=1 / 1.4)
    rng = np.random.Generator(np.random.PCG64(73))
    W = W * (1.0 + 0.01 * rng.standard_normal(W.shape))
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(precision=0, weno=1, cfl=0.5, viscous=1, mu=0.01, prandtl=0.72))
    s.set_fixed_state(W, dW)
    s.init(W, dW)
    dt = 0.5 * s.timestep()
    force = gks.wall_pressure_force(g, mesh["bkind"])

    def run(W0):
        Wc, dWc = torch.tensor(W0, device="cuda"), torch.tensor(dW, device="cuda")
        states = []
        for _ in range(3):
            states.append((Wc, dWc))
            s.init(Wc, dWc)
            s.step(1, dt, 0.0)
            Wc, dWc = s.get()
        return Wc, states

    Wn, states = run(W)
    Wn = Wn.clone().requires_grad_(True)
    J = force(Wn)[0]
    J.backward()
    lam_W = Wn.grad.detach().clone()
    lam_dW = torch.zeros((15, g.nc), dtype=torch.float64, device="cuda")
    for Wc, dWc in reversed(states):
        lam_W, lam_dW = s.adjoint_step(Wc, dWc, lam_W, lam_dW, dt)
    d = rng.standard_normal(g.nc)
    U = W[1:4] / W[0]
    dW0 = np.concatenate([d[None], d[None] * U, 0.5 * d[None] * (U ** 2).sum(0)[None]])
    ad = float((lam_W.cpu().numpy() * dW0).sum())
    h = 1e-7
    with torch.no_grad():
        fd = (float(force(run(W + h * dW0)[0])[0]) - float(force(run(W - h * dW0)[0])[0])) / (2 * h)
    assert abs(ad - fd) < 1e-6 * abs(fd), (ad, fd)


@pytest.mark.parametrize("weno,state", [(0, "sine"), (1, "sine"), (1, "slab")])
def test_second_order_reconstruction_adjoint(cuda, oracle_mod, weno, state):
    """R^2nd (Eq. final_weno_expression-2nd): linear weights give R = P1, the
    nonlinear ones weigh p1 against p0 with beta_1 and the two-step beta_0;
    both against central differences of the GPU and oracle forward maps."""
    torch = cuda
    mesh, W, dW, rng = _case(state=state)
    H = 1e-7 if state == "slab" else 1e-6
    g = gks.Mesh(mesh)
    kw = dict(weno=weno, order=2, cfl=0.5)
    s = gks.State(g, gks.params(precision=0, **kw))
    o = oracle_mod.Mesh(mesh)
    p = oracle_mod.params(**kw)
    dt = 0.5 * o.timestep(p, W)
    lam = (rng.standard_normal(W.shape), rng.standard_normal(dW.shape))
    v = (rng.standard_normal(W.shape) * np.abs(W).max(axis=1, keepdims=True),
         rng.standard_normal(dW.shape) * np.abs(dW).max())

    def gpu_step(Wx, dWx):
        s.init(Wx, dWx)
        s.step(1, dt, 0.0)
        return [x.cpu().numpy() for x in s.get()]

    jv_gpu = [(a - b) / (2 * H) for a, b in zip(gpu_step(W + H * v[0], dW + H * v[1]),
                                                 gpu_step(W - H * v[0], dW - H * v[1]))]
    op, om = o.step(p, W + H * v[0], dW + H * v[1], dt), o.step(p, W - H * v[0], dW - H * v[1], dt)
    jv_ora = [(op[0] - om[0]) / (2 * H), (op[1] - om[1]) / (2 * H)]
    lW, ldW = s.adjoint_step(torch.tensor(W), torch.tensor(dW), torch.tensor(lam[0]), torch.tensor(lam[1]), dt)
    rhs = _dot((lW.cpu().numpy(), ldW.cpu().numpy()), v)
    assert abs(_dot(lam, jv_gpu) - rhs) < 1e-6 * abs(rhs), (_dot(lam, jv_gpu), rhs)
    assert abs(_dot(lam, jv_ora) - rhs) < 1e-6 * abs(rhs), (_dot(lam, jv_ora), rhs)


@pytest.mark.parametrize("state,weno,viscous,smooth,prandtl", [
    ("sine", 0, 0, 0, 1.0), ("sine", 0, 1, 0, 1.0), ("sine", 0, 1, 1, 1.0), ("sine", 0, 1, 0, 0.72),
    ("sine", 0, 0, 1, 1.0), ("sine", 1, 0, 0, 1.0), ("sine", 1, 1, 0, 0.72), ("slab", 1, 0, 0, 1.0),
    ("open", 0, 0, 0, 1.0), ("open", 1, 0, 0, 1.0), ("slip", 1, 0, 0, 1.0), ("noslip", 0, 1, 0, 1.0),
    ("noslip", 1, 1, 0, 0.72), ("fixed", 1, 0, 0, 1.0), ("fixed", 0, 1, 0, 1.0), ("sine-o2", 0, 0, 0, 1.0),
    ("sine-o2", 1, 0, 0, 1.0), ("slab-o2", 1, 0, 0, 1.0), ("sine-lowp", 0, 0, 0, 1.0),
    ("sine-lowp", 1, 0, 0, 1.0), ("isothermal", 0, 1, 0, 1.0), ("isothermal", 1, 1, 0, 0.72),
    ("moving", 0, 1, 0, 1.0), ("moving", 1, 1, 0, 1.0)])
def test_adjoint_matches_cpu_reverse_sweep(cuda, oracle_mod, state, weno, viscous, smooth, prandtl):
    """The adjoint against an FP64 CPU reverse sweep: torch.autograd through
    the plain-PyTorch restatement of the step (oracle/torch_step.py, itself
    pinned to the C oracle's step), linear or WENO weights, full or smooth
    flux, Euler or Navier-Stokes with the Pr fix, periodic meshes (the
    density wave and the moving slab) and boxes with open, wall or fixed
    ends (the fixed state set apart); the second-order R ("-o2") and a cell
    that falls back to its average ("-lowp").  Both are exact derivatives,
    so they agree to rounding, every entry of d J / d (W, grad W)."""
    import torch
    from oracle import torch_step as TS
    base, _, variant = state.partition("-")
    mesh, W, dW, rng = _case(state=base)
    order = 2 if variant == "o2" else 3
    if variant == "lowp":
        W = W.copy()
        W[4, 0] = 0.5 * (W[1, 0] ** 2 + W[2, 0] ** 2 + W[3, 0] ** 2) / W[0, 0] + 0.05 / 0.4
    g = gks.Mesh(mesh)
    kw = dict(mu=0.01 * viscous, viscous=viscous, smooth_flux=smooth, prandtl=prandtl, weno=weno, order=order,
              wall_temperature=0.9, wall_velocity=(0.0, 0.4, -0.2))
    s = gks.State(g, gks.params(precision=0, cfl=0.5, **kw))
    fixed = None
    if state == "fixed":
        fixed = (W * (1.0 + 0.02 * rng.standard_normal(W.shape)), 0.5 * dW)
        s.set_fixed_state(*fixed)
        mesh["fixed_state"] = fixed
    o = oracle_mod.Mesh(mesh)
    dt = 0.5 * o.timestep(oracle_mod.params(cfl=0.5, **kw), W)
    lam = (rng.standard_normal(W.shape), rng.standard_normal(dW.shape))
    lW, ldW = s.adjoint_step(torch.tensor(W), torch.tensor(dW), torch.tensor(lam[0]), torch.tensor(lam[1]), dt)
    Wt = torch.tensor(W, requires_grad=True)
    dWt = torch.tensor(dW, requires_grad=True)
    st = TS.Step(o, mu=kw["mu"], viscous=bool(viscous), smooth=bool(smooth), prandtl=prandtl,
                 weno=bool(weno), kinds=mesh.get("bkind"), fixed=fixed, order=order, wall_temperature=0.9,
                 wall_velocity=(0.0, 0.4, -0.2))
    Wn, dWn = st(Wt, dWt, dt)
    if variant == "lowp":
        assert st.fallbacks[0][0]
    ((Wn * torch.tensor(lam[0])).sum() + (dWn * torch.tensor(lam[1])).sum()).backward()
    # (the second-order R reads no gradients: the step then does not depend on grad W at all)
    cpu_dW = dWt.grad.numpy() if dWt.grad is not None else np.zeros_like(dW)
    for gpu, cpu in ((lW.cpu().numpy(), Wt.grad.numpy()), (ldW.cpu().numpy(), cpu_dW)):
        scale = np.abs(cpu).max() if np.abs(cpu).any() else np.abs(lW.cpu().numpy()).max()
        assert np.abs(gpu - cpu).max() < 1e-11 * scale, np.abs(gpu - cpu).max() / scale


def test_kinetic_energy_gradient_through_three_steps(cuda, oracle_mod):
    """J = sum |Omega| |rho U|^2 / (2 rho) after 3 steps; dJ/d rho_0 (initial
    cell-average density, U and p held) by autograd over the chained step
    function, checked along a random direction of the density field."""
    torch = cuda
    mesh, W, dW, rng = _case(seed=62)
    g = gks.Mesh(mesh)
    vol = torch.tensor(g.geometry()["vol"], device="cuda")
    s = gks.State(g, gks.params(precision=0, weno=0, cfl=0.5))
    o = oracle_mod.Mesh(mesh)
    dt = 0.5 * o.timestep(oracle_mod.params(weno=0, cfl=0.5), W)
    gamma = 1.4
    Wt = torch.tensor(W, device="cuda")
    U = Wt[1:4] / Wt[0]
    p = (gamma - 1.0) * (Wt[4] - 0.5 * (Wt[1:4] ** 2).sum(0) / Wt[0])
    dW0 = torch.tensor(dW, device="cuda")

    def energy(rho, step):
        W0 = torch.cat([rho[None], rho[None] * U, (p / (gamma - 1.0) + 0.5 * rho * (U ** 2).sum(0))[None]])
        Wc, dWc = W0, dW0
        for _ in range(3):
            Wc, dWc = step(Wc, dWc)
        return (vol * (Wc[1:4] ** 2).sum(0) / (2.0 * Wc[0])).sum()

    step = gks.make_step_function(s, dt)
    rho = Wt[0].clone().requires_grad_(True)
    J = energy(rho, step)
    J.backward()
    grad = rho.grad.detach()

    def plain(Wx, dWx):
        s.init(Wx, dWx)
        s.step(1, dt, 0.0)
        return s.get()

    d = torch.tensor(rng.standard_normal(W.shape[1]), device="cuda") * 0.1
    with torch.no_grad():
        fd = (energy(Wt[0] + H * d, plain) - energy(Wt[0] - H * d, plain)) / (2 * H)
    ad = float((grad * d).sum())
    assert abs(ad - float(fd)) < 1e-6 * abs(ad), (ad, float(fd))


def test_unsupported_configurations_are_rejected(cuda):
    torch = cuda
    mesh, W, dW, _ = _case()
    g = gks.Mesh(mesh)
    args = [torch.tensor(x, device="cuda") for x in (W, dW, np.zeros_like(W), np.zeros_like(dW))]
    for kw in (dict(weno=0, precision=1),):
        s = gks.State(g, gks.params(cfl=0.5, **kw))
        with pytest.raises(gks.GksError) as e:
            s.adjoint_step(*args, 1e-3)
        assert e.value.status == -8  # GKS_E_UNSUPPORTED
    fixed_mesh, Wo, dWo = I.shu_osher_case(nx=8, nyz=2)  # fixed-state ends
    s = gks.State(gks.Mesh(fixed_mesh), gks.params(weno=0, cfl=0.5))
    argso = [torch.tensor(x, device="cuda") for x in (Wo, dWo, np.zeros_like(Wo), np.zeros_like(dWo))]
    with pytest.raises(gks.GksError) as e:
        s.adjoint_step(*argso, 1e-3)
    assert e.value.status == -8


@pytest.mark.parametrize("weno", [0, 1])
def test_positivity_fallback_cell(cuda, oracle_mod, weno):
    """A low-pressure cell (p = 0.05 among p ~ 1) whose reconstruction falls
    back to its average in the first stage (the positivity branch): its
    adjoint passes the constant's adjoint to its own average only.  The
    fallback decision holds under the differences' perturbations (checked),
    so central differences of the GPU and of the oracle forward map pin the
    piecewise derivative."""
    torch = cuda
    mesh, W, dW, rng = _case()
    W = W.copy()
    W[4, 0] = 0.5 * (W[1, 0] ** 2 + W[2, 0] ** 2 + W[3, 0] ** 2) / W[0, 0] + 0.05 / 0.4
    H = 1e-7
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(precision=0, weno=weno, cfl=0.5))
    o = oracle_mod.Mesh(mesh)
    p = oracle_mod.params(weno=weno, cfl=0.5)
    dt = 0.5 * o.timestep(p, W)
    lam = (rng.standard_normal(W.shape), rng.standard_normal(dW.shape))
    v = (rng.standard_normal(W.shape) * np.abs(W).max(axis=1, keepdims=True),
         rng.standard_normal(dW.shape) * np.abs(dW).max())
    for sgn in (1.0, -1.0, 0.0):
        s.init(W + sgn * H * v[0], dW + sgn * H * v[1])
        assert s.debug_reconstruct()[2].cpu().numpy()[0] == 1

    def gpu_step(Wx, dWx):
        s.init(Wx, dWx)
        s.step(1, dt, 0.0)
        return [x.cpu().numpy() for x in s.get()]

    jv_gpu = [(a - b) / (2 * H) for a, b in zip(gpu_step(W + H * v[0], dW + H * v[1]),
                                                 gpu_step(W - H * v[0], dW - H * v[1]))]
    op, om = o.step(p, W + H * v[0], dW + H * v[1], dt), o.step(p, W - H * v[0], dW - H * v[1], dt)
    jv_ora = [(op[0] - om[0]) / (2 * H), (op[1] - om[1]) / (2 * H)]
    lW, ldW = s.adjoint_step(torch.tensor(W), torch.tensor(dW), torch.tensor(lam[0]), torch.tensor(lam[1]), dt)
    rhs = _dot((lW.cpu().numpy(), ldW.cpu().numpy()), v)
    assert abs(_dot(lam, jv_gpu) - rhs) < 1e-6 * abs(rhs), (_dot(lam, jv_gpu), rhs)
    assert abs(_dot(lam, jv_ora) - rhs) < 1e-6 * abs(rhs), (_dot(lam, jv_ora), rhs)


def test_mach_number_gradient_of_the_vortex(cuda):
    """dJ/dMa for J = total kinetic energy after 4 steps of the isentropic
    vortex (periodic 6^3 x 6 box): the chained adjoint gives dJ/d(W0, dW0),
    the derivative of the initial state with respect to the free-stream Mach
    number comes from the input generator (central difference of the cell
    averages, which are linear in the free-stream velocity), and the product
    matches a central difference of J(Ma) through the forward runs."""
    torch = cuda
    n, ma, hm = 6, 0.5, 1e-5

    def case(m):
        return I.isentropic_vortex_case(n=n, mach=m, order=3)
    mesh, W, dW = case(ma)
    g = gks.Mesh(mesh)
    vol = torch.tensor(g.geometry()["vol"], device="cuda")
    s = gks.State(g, gks.params(precision=0, weno=0, cfl=0.5))
    s.init(W, dW)
    dt = s.timestep()

    def energy_of(Wc):
        return (vol * (Wc[1:4] ** 2).sum(0) / (2.0 * Wc[0])).sum()

    def run(W0, dW0):
        Wc, dWc = torch.tensor(W0, device="cuda"), torch.tensor(dW0, device="cuda")
        states = []
        for _ in range(4):
            states.append((Wc, dWc))
            s.init(Wc, dWc)
            s.step(1, dt, 0.0)
            Wc, dWc = s.get()
        return Wc, states

    Wn, states = run(W, dW)
    lam_W = torch.zeros_like(Wn)
    lam_W[1:4] = vol * Wn[1:4] / Wn[0]
    lam_W[0] = -0.5 * vol * (Wn[1:4] ** 2).sum(0) / Wn[0] ** 2
    lam_dW = torch.zeros((15, g.nc), dtype=torch.float64, device="cuda")
    for Wc, dWc in reversed(states):
        lam_W, lam_dW = s.adjoint_step(Wc, dWc, lam_W, lam_dW, dt)
    _, Wp, dWp = case(ma + hm)
    _, Wm, dWm = case(ma - hm)
    dW0 = (Wp - Wm) / (2 * hm)
    ddW0 = (dWp - dWm) / (2 * hm)
    ad = float((lam_W.cpu().numpy() * dW0).sum() + (lam_dW.cpu().numpy() * ddW0).sum())
    fd = (float(energy_of(run(Wp, dWp)[0])) - float(energy_of(run(Wm, dWm)[0]))) / (2 * hm)
    assert abs(ad - fd) < 1e-6 * abs(fd), (ad, fd)


def test_checkpointed_gradient(cuda):
    """Six steps with a checkpoint every 2 give the same gradient as a
    checkpoint every step (the recomputation is exact in FP64); an FP32-bulk
    primal run with FP64 checkpoints gives a gradient within 1e-3 of it."""
    torch = cuda
    mesh, W, dW, _ = _case(seed=64)
    g = gks.Mesh(mesh)
    p = gks.params(weno=1, cfl=0.5)
    s = gks.State(g, p)
    s.init(W, dW)
    dt = s.timestep()
    vol = torch.tensor(g.geometry()["vol"], device="cuda")

    def loss(Wn):
        return (vol * (Wn[1:4] ** 2).sum(0) / (2.0 * Wn[0])).sum()

    J1, gW1, gdW1 = gks.checkpointed_gradient(g, p, W, dW, 6, dt, loss, checkpoint_every=1)
    J2, gW2, gdW2 = gks.checkpointed_gradient(g, p, W, dW, 6, dt, loss, checkpoint_every=2)
    assert J1 == J2
    assert torch.equal(gW1, gW2) and torch.equal(gdW1, gdW2)
    J3, gW3, _ = gks.checkpointed_gradient(g, p, W, dW, 6, dt, loss, checkpoint_every=2, primal_precision=1)
    assert abs(J3 - J1) < 1e-5 * abs(J1)
    assert float((gW3 - gW1).abs().max() / gW1.abs().max()) < 1e-3


@pytest.mark.parametrize("kw", [dict(weno=1), dict(weno=0, order=2),
                                dict(weno=1, viscous=1, mu=0.01, prandtl=0.72)])
def test_staged_adjoint_step_equals_the_recomputing_one(cuda, kw):
    """The adjoint step given its step's stage state (W*, grad W*) from the
    primal skips the first stage's flux and update and returns the same
    adjoint to the bit; stage_state() is defined only after a step of an
    FP64 state."""
    torch = cuda
    mesh, W, dW, _ = _case(seed=66, state="noslip")
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(cfl=0.5, **kw))
    s.init(W, dW)
    with pytest.raises(gks.GksError) as e:
        s.stage_state()  # no step yet
    assert e.value.status == -4  # GKS_E_STATE
    dt = s.timestep()
    s.step(1, dt, 0.0)
    stage = s.stage_state()
    Wt, dWt = torch.tensor(W, device="cuda"), torch.tensor(dW, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(5)
    lW = torch.randn((5, g.nc), generator=gen, device="cuda", dtype=torch.float64)
    ldW = torch.randn((15, g.nc), generator=gen, device="cuda", dtype=torch.float64)
    a = s.adjoint_step(Wt, dWt, lW, ldW, dt)
    b = s.adjoint_step(Wt, dWt, lW, ldW, dt, stage=stage)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    s32 = gks.State(g, gks.params(cfl=0.5, precision=1, **kw))
    s32.init(W, dW)
    s32.step(1)
    with pytest.raises(gks.GksError) as e:
        s32.stage_state()
    assert e.value.status == -8  # GKS_E_UNSUPPORTED
