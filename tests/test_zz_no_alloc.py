"""gks_timestep_noalloc: the time-step reduction for callers that may not
allocate device memory (its scratch is a fixed array inside the library).

It must give the same value as gks_timestep, which reduces through the
caller's workspace, on two calls in a row over different meshes (the second
call reuses the shared scratch the first one wrote).  Collected last so that
a stop-at-first-failure run has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2102_01366_gb300 import gks
from paper_2102_01366_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU")
    from paper_2102_01366_gb300 import _build
    _build.build()
    gks.lib()
    return torch


def _reference_and_inputs(torch, mesh, W, dW):
    g = gks.Mesh(mesh)
    p = gks.params(weno=1, cfl=0.5)
    s = gks.State(g, p)
    s.init(W, dW)
    dt_ref = s.timestep()
    d_W = torch.tensor(W, dtype=torch.float64, device="cuda")
    d_dr = torch.tensor(g.geometry()["dr"], dtype=torch.float64, device="cuda")
    return g, p, dt_ref, d_W, d_dr


def test_noalloc_timestep_matches_workspace_version(torch_cuda):
    torch = torch_cuda
    cases = [I.sod_case(), I.sine_wave_case(n=3)]  # 24,576 then 162 cells
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for i, (mesh, W, dW) in enumerate(cases):
        g, p, dt_ref, d_W, d_dr = _reference_and_inputs(torch, mesh, W, dW)
        st = gks.lib().gks_timestep_noalloc(C.byref(p), C.c_void_p(d_W.data_ptr()),
                                            C.c_void_p(d_dr.data_ptr()), g.nc,
                                            C.c_void_p(out[i:].data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == 0, gks.lib().gks_last_error().decode()
        torch.cuda.synchronize()
        got = float(out[i].item())
        assert abs(got - dt_ref) <= 1e-14 * dt_ref, (i, got, dt_ref)


def test_noalloc_rejects_too_many_cells(torch_cuda):
    torch = torch_cuda
    p = gks.params()
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = C.c_void_p(d.data_ptr())
    too_many = 8192 * 256 + 1
    st = gks.lib().gks_timestep_noalloc(C.byref(p), ptr, ptr, too_many, ptr, None)
    assert st == -1
    assert "n_cell" in gks.lib().gks_last_error().decode()
