"""CPU checks of the C ABI boundary: the library builds, loads without a GPU,
exports every entry point declared in include/qtb.h, rejects bad arguments on
the host, and the binding fails loudly when the library is missing."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qtb():
    from paper_1905_02521_gb300 import build
    build.build()
    from paper_1905_02521_gb300 import qtb as q
    return q


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "qtb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qtb_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(qtb):
    names = declared_entry_points()
    assert "qtb_init" in names and "qtb_step_n" in names and "qtb_set_filter" in names
    assert "qtb_observables" in names
    L = qtb.lib()
    for n in names:
        assert hasattr(L, n), n


def test_host_validation_rejects_bad_arguments(qtb):
    # validation happens before any CUDA call, so it runs without a GPU
    from paper_1905_02521_gb300 import workloads as W
    s, pot = W.mgo_system(2, 300.0)
    base = dict(mass=pot["mass"], charge=pot["charge"], buck_A=pot["buck_A"], buck_rho=pot["buck_rho"],
                buck_C=pot["buck_C"], dsf_alpha=0.2, r_cut=8.0, dt=1.0, torch_alloc=False, torch_stream=False)
    with pytest.raises(qtb.QtbError) as e:
        qtb.qtb_init([], base)
    assert e.value.code == qtb.ERR_ARG
    bad = dict(s, T=-1.0)
    with pytest.raises(qtb.QtbError) as e:
        qtb.qtb_init([bad], base)
    assert e.value.code == qtb.ERR_ARG and "T > 0" in str(e.value)
    small = dict(s, box=np.array([7.0, 8.42, 8.42]))
    with pytest.raises(qtb.QtbError) as e:
        qtb.qtb_init([small], base)
    assert "r_cut" in str(e.value)
    beads = dict(s, pos=np.repeat(s["pos"], 7, axis=0), vel=None)
    with pytest.raises(qtb.QtbError) as e:
        qtb.qtb_init([beads], base)
    assert "n_beads" in str(e.value)
    with pytest.raises(qtb.QtbError):
        qtb.qtb_init([s], dict(base, dt=0.0))
    with pytest.raises(qtb.QtbError):
        qtb.qtb_kappa_solve(0)
    for call in (qtb.qtb_rebuild_lists, qtb.qtb_list_rebuilds, qtb.qtb_sync):   # null context
        with pytest.raises(qtb.QtbError) as e:
            call(None)
        assert e.value.code == qtb.ERR_ARG


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_1905_02521_gb300 import build, qtb as q
    monkeypatch.setattr(q, "_lib", None)
    monkeypatch.setattr(build, "LIB", "/nonexistent/libqtb.so")
    with pytest.raises(RuntimeError, match="not built"):
        q.lib()
