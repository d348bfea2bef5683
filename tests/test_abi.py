"""Host-side checks of the C ABI: the library loads without a GPU, exports every
entry point that include/kg.h declares, and rejects bad calls before touching CUDA."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def kg():
    import __graft_entry__ as g
    g.build_library()
    from paper_1501_04552_gb300 import kg as K
    return K


def test_every_declared_symbol_is_exported(kg):
    names = kg.header_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(kg.lib, n), n


def test_calls_before_init_are_state_errors(kg):
    kg.lib.kg_finalize()
    assert kg.lib.kg_step(1) == kg.KG_ESTATE
    E = C.c_double()
    assert kg.lib.kg_energy(C.byref(E)) == kg.KG_ESTATE
    assert kg.lib.kg_fetch(None) == kg.KG_ESTATE
    assert "kg_fetch" in kg.last_error()


def test_bad_arguments_rejected_on_the_host(kg):
    u = np.zeros((16, 16, 16))
    assert kg.lib.kg_init(17, 32.0, 0.01, u.ctypes.data, None) == kg.KG_ENOTSUP
    assert kg.lib.kg_init(1024, 32.0, 0.01, u.ctypes.data, None) == kg.KG_ENOTSUP
    assert kg.lib.kg_init(16, -1.0, 0.01, u.ctypes.data, None) == kg.KG_EINVAL
    assert kg.lib.kg_init(16, 32.0, 0.0, u.ctypes.data, None) == kg.KG_EINVAL
    assert kg.lib.kg_init(16, 32.0, float("nan"), u.ctypes.data, None) == kg.KG_EINVAL
    assert kg.lib.kg_init(16, 32.0, 0.01, None, None) == kg.KG_EINVAL
    bad = u.copy()
    bad[3, 4, 5] = np.inf
    assert kg.lib.kg_init(16, 32.0, 0.01, bad.ctypes.data, None) == kg.KG_EINVAL
    assert "u0" in kg.last_error()
    v = u.copy()
    v[0, 0, 0] = np.nan
    assert kg.lib.kg_init(16, 32.0, 0.01, u.ctypes.data, v.ctypes.data) == kg.KG_EINVAL


def test_options_round_trip_and_validation(kg):
    kg.kg_set_options(precision="mixed", energy_every=10, nonlinearity=0.5, blowup_threshold=1e3, drift_tol=1e-3)
    o = kg.kg_get_options()
    assert o == {"precision": kg.KG_MIXED, "energy_every": 10, "nonlinearity": 0.5,
                 "blowup_threshold": 1e3, "drift_tol": 1e-3}
    bad = kg.kg_options(7, 0, 1.0, 0.0, 0.0)
    assert kg.lib.kg_set_options(C.byref(bad)) == kg.KG_EINVAL
    bad = kg.kg_options(0, -1, 1.0, 0.0, 0.0)
    assert kg.lib.kg_set_options(C.byref(bad)) == kg.KG_EINVAL
    bad = kg.kg_options(0, 0, float("inf"), 0.0, 0.0)
    assert kg.lib.kg_set_options(C.byref(bad)) == kg.KG_EINVAL
    kg.kg_set_options()
    assert kg.kg_get_options()["precision"] == kg.KG_DF64
