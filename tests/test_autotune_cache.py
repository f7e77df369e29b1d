"""The autotuner's result cache in the Python binding (host logic, no GPU).

State.autotune times the execution variants through gks_autotune and keeps
the winner in a JSON file keyed by GPU name, mesh size and scheme options.
Here the library calls are replaced by a fake that records them, so the
keying, reuse, recovery from a damaged file and the no-cache mode are
checked on the CPU."""
import ctypes as C
import json
import types

import numpy as np
import pytest

from paper_2102_01366_gb300 import gks


class _FakeCuda:
    @staticmethod
    def get_device_name(dev):
        return "test GPU"


def _state(precision=1, nc=100):
    s = gks.State.__new__(gks.State)  # no device, no library handle
    s.params = gks.params(precision=precision, weno=1)
    s.mesh = types.SimpleNamespace(nc=nc, nf=2 * nc, ncase=1)
    s.torch = types.SimpleNamespace(cuda=_FakeCuda)
    s.device = "cuda:0"
    s._h = None
    return s


@pytest.fixture
def calls(monkeypatch):
    log = []

    def fake_call(name, *args):
        log.append((name, args[1:]))
        if name == "gks_autotune":
            _, steps, fo, fb, sp, ms = args
            fo._obj.value, fb._obj.value, sp._obj.value = 1, 2, 1
            out = np.ctypeslib.as_array(C.cast(ms, C.POINTER(C.c_double)), shape=(gks.State.NVARIANTS,))
            out[:] = np.arange(10.0, 0.0, -1.0)
            out[8] = np.nan  # a variant the library did not time
        elif name == "gks_state_get_fused":
            args[1]._obj.value = 1
        return 0

    monkeypatch.setattr(gks, "_call", fake_call)
    return log


def _names(log):
    return [n for n, _ in log]


def test_first_call_tunes_and_stores(calls, tmp_path):
    cache = str(tmp_path / "sub" / "autotune.json")
    res = _state().autotune(steps=3, cache=cache)
    assert res["cached"] is False and res["variant"] == [1, 2, 1]
    # 10 variants: 8 with separate kernels, 2 with one launch per stage; NaN (untimed) reads None
    assert res["ms_per_step"] == [10.0, 9.0, 8.0, 7.0, 6.0, 5.0, 4.0, 3.0, None, 1.0]
    assert res["fused"] == 1
    assert _names(calls) == ["gks_autotune", "gks_state_get_fused"] and calls[0][1][0] == 3
    table = json.load(open(cache))
    (key, entry), = table.items()
    assert key.startswith("test GPU|nc=100|nf=200|ncase=1|prec=1|weno=1")
    assert entry["variant"] == [1, 2, 1] and entry["fused"] == 1


def test_second_call_reuses_the_stored_variant(calls, tmp_path):
    cache = str(tmp_path / "autotune.json")
    _state().autotune(cache=cache)
    calls.clear()
    s = _state()
    res = s.autotune(cache=cache)
    assert res["cached"] is True and res["variant"] == [1, 2, 1]
    assert _names(calls) == ["gks_state_set_variant", "gks_state_set_fused"]
    assert calls[0][1] == (1, 2, 1) and calls[1][1] == (1,)
    assert s.variant == (1, 2, 1)


def test_options_and_sizes_get_their_own_entries(calls, tmp_path):
    cache = str(tmp_path / "autotune.json")
    _state(precision=1).autotune(cache=cache)
    res = _state(precision=0).autotune(cache=cache)
    assert res["cached"] is False and len(res["ms_per_step"]) == gks.State.NVARIANTS
    _state(nc=101).autotune(cache=cache)
    assert len(json.load(open(cache))) == 3
    assert _names(calls).count("gks_autotune") == 3


def test_damaged_cache_is_retuned_and_rewritten(calls, tmp_path):
    cache = tmp_path / "autotune.json"
    cache.write_text("{ not json")
    res = _state().autotune(cache=str(cache))
    assert res["cached"] is False and _names(calls) == ["gks_autotune", "gks_state_get_fused"]
    assert len(json.load(open(cache))) == 1
    # an entry without a complete variant is not trusted either
    key = next(iter(json.load(open(cache))))
    cache.write_text(json.dumps({key: {"variant": [1, 2]}}))
    calls.clear()
    assert _state().autotune(cache=str(cache))["cached"] is False
    assert _names(calls) == ["gks_autotune", "gks_state_get_fused"]
    # nor one from before the one-launch stage (no "fused" entry)
    cache.write_text(json.dumps({key: {"variant": [1, 2, 1]}}))
    calls.clear()
    assert _state().autotune(cache=str(cache))["cached"] is False


def test_no_cache_mode_writes_nothing(calls, tmp_path, monkeypatch):
    monkeypatch.setenv("HOME", str(tmp_path))
    monkeypatch.delenv("GKS_AUTOTUNE_CACHE", raising=False)
    res = _state().autotune(cache=False)
    assert res["cached"] is False
    assert list(tmp_path.iterdir()) == []


def test_environment_variable_names_the_default_cache(calls, tmp_path, monkeypatch):
    cache = tmp_path / "env.json"
    monkeypatch.setenv("GKS_AUTOTUNE_CACHE", str(cache))
    _state().autotune()
    assert cache.exists() and len(json.load(open(cache))) == 1
