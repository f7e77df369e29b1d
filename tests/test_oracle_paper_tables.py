"""The oracle against the paper's printed accuracy tables (Sec. 5.1,
Tables 1-3), read from tests/golden/sine_wave_tables.txt.

The paper does not say how each hexahedron is split into six tetrahedra.
The Kuhn split used here shares one main diagonal per hexahedron; with that
diagonal across the direction of propagation ((0,0,1)-(1,1,0) for a wave
along (1,1,1)) the linear third-order errors match Table 1 to a few
percent, so the scheme itself is pinned to the paper's numbers.  The
nonlinear-weight rows depend on details the paper leaves open (the
normalisation of beta_0, the pair average) and are held to a factor of 2."""
import math
import os

import numpy as np
import pytest

from paper_2102_01366_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sine_wave_tables.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        tab, kind, n, l1, l2, li = line.split()
        rows[(kind, int(n))] = (float(l1), float(l2), float(li))
    return rows


def _errors(oracle_mod, n, weno, order):
    mesh = I.box_mesh((n, n, n), (2.0, 2.0, 2.0), (True, True, True), jitter=0.0, seed=0,
                      diagonal=(1, 1, -1))
    W, dW = I.sine_wave_state(mesh, k=math.pi)
    om = oracle_mod.Mesh(mesh)
    W1, _, t, _ = om.run(oracle_mod.params(cfl=1.0, weno=weno, order=order), W, dW, t_end=2.0)
    assert abs(t - 2.0) < 1e-12
    We, _ = I.sine_wave_state(mesh, t=t, k=math.pi)
    vol = om.geometry()["vol"]
    d = W1[0] - We[0]
    return ((vol * np.abs(d)).sum() / vol.sum(), math.sqrt((vol * d * d).sum() / vol.sum()),
            np.abs(d).max())


def test_table1_linear_third_order_n5(oracle_mod):
    ref = _golden()[("linear-3rd", 5)]
    got = _errors(oracle_mod, 5, 0, 3)
    for g, r in zip(got, ref):
        assert abs(g / r - 1.0) < 0.05, (got, ref)


@pytest.mark.parametrize("kind,weno,order", [("weno-3rd", 1, 3), ("weno-2nd", 1, 2)])
def test_tables2_3_nonlinear_weights_n5(oracle_mod, kind, weno, order):
    ref = _golden()[(kind, 5)]
    got = _errors(oracle_mod, 5, weno, order)
    for g, r in zip(got, ref):
        assert 0.5 < g / r < 2.0, (got, ref)
