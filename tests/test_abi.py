"""The C-ABI library loads and exports every function the headers under
include/ declare (no device work: runs without a GPU)."""
import ctypes
import os
import re
import types

import pytest

from paper_1904_06680_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(npp_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_exports_all_declared_symbols():
    from paper_1904_06680_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 10, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    from paper_1904_06680_gb300 import npp
    assert sorted(npp.EXPORTS) == _declared()
    npp.lib()


def test_n_theta_and_config_validation_without_device():
    from paper_1904_06680_gb300 import inputs, npp
    for w, n in [(16, 450), (32, 1410), (64, 4866)]:
        assert npp.npp_n_theta(npp.make_config(inputs.planner(w), 1, 1, 1)) == n
    assert npp.npp_n_theta(npp.make_config(dict(inputs.planner(16), widths=(8, 24, 24, 2)), 1, 1, 1)) == -1
    assert npp.npp_n_theta(npp.make_config(inputs.PAPER, 1, 1, 1)) == -1


def test_binding_fails_loudly_without_library(monkeypatch):
    """No CPU fallback: without the built library every entry point raises."""
    from paper_1904_06680_gb300 import npp
    monkeypatch.setattr(npp, "_lib", None)
    monkeypatch.setattr(npp, "LIB_PATH", os.path.join(os.path.dirname(npp.LIB_PATH), "missing", "libnpp.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        npp.lib()
    with pytest.raises(RuntimeError):
        npp.npp_n_theta(npp.make_config(inputs.planner(16), 1, 1, 1))


def test_config_checks_shared_by_create_and_noalloc():
    """npp_create and the allocation-free plan step reject the same
    configurations (the checks run before any device call)."""
    from paper_1904_06680_gb300 import npp
    bad = [dict(lr=-0.5), dict(Ts=0.0), dict(half_wid=float("nan")), dict(u_min=3.0, u_max=-3.0),
           dict(feature_frame=2)]
    out = npp.npp_outputs()
    out.best = 16                      # never dereferenced: the configuration is rejected first
    for b in bad:
        cfg = npp.make_config(dict(inputs.planner(16), **b), 8, 4, 4)
        with pytest.raises(npp.NppError) as e1:
            npp.npp_create(cfg, 0)
        with pytest.raises(npp.NppError) as e2:
            npp.npp_plan_step_noalloc(cfg, [0, 0, 0, 0, 0, 0], [5, 0, 0, 0], None, 0, 8, 4, 1, 0, None, out,
                                      stream=types.SimpleNamespace(cuda_stream=0))
        assert e1.value.status == e2.value.status == npp.NPP_INVALID_ARG, b
