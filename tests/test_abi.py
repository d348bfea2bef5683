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
    # and the binding gives every entry point an explicit signature (ctypes defaults would
    # pass doubles and sizes wrongly)
    assert sorted(kg._sig) == names


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
                 "blowup_threshold": 1e3, "drift_tol": 1e-3, "tune_cache": None}
    bad = kg.kg_options(7, 0, 1.0, 0.0, 0.0)
    assert kg.lib.kg_set_options(C.byref(bad)) == kg.KG_EINVAL
    bad = kg.kg_options(0, -1, 1.0, 0.0, 0.0)
    assert kg.lib.kg_set_options(C.byref(bad)) == kg.KG_EINVAL
    bad = kg.kg_options(0, 0, float("inf"), 0.0, 0.0)
    assert kg.lib.kg_set_options(C.byref(bad)) == kg.KG_EINVAL
    kg.kg_set_options()
    assert kg.kg_get_options()["precision"] == kg.KG_DF64


def test_tune_cache_path_through_options(kg, tmp_path):
    """the ensemble autotuner's cache file can be named through kg_set_options: the library
    keeps its own copy, NULL leaves it as set, "" clears it, and kg_ens_set_tune_cache is the
    same setting"""
    path = str(tmp_path / "tune.txt")
    kg.kg_set_options(tune_cache=path)
    assert kg.kg_get_options()["tune_cache"] == path
    kg.kg_set_options(energy_every=5)                  # NULL: the file stays
    assert kg.kg_get_options()["tune_cache"] == path
    assert kg.lib.kg_ens_set_tune_cache(b"other.txt") == kg.KG_OK
    assert kg.kg_get_options()["tune_cache"] == "other.txt"
    kg.kg_set_options(tune_cache="")                   # "": no file
    assert kg.kg_get_options()["tune_cache"] is None
    kg.kg_set_options()


def test_scheme_round_trip_and_validation(kg):
    """the scheme applies at the next init; combinations the composed scheme does not
    define are refused on the host"""
    kg.lib.kg_finalize()
    assert kg.kg_get_scheme() == kg.KG_SCHEME_EQ2
    assert kg.lib.kg_set_scheme(7) == kg.KG_EINVAL
    assert kg.lib.kg_get_scheme(None) == kg.KG_EINVAL
    kg.kg_set_scheme("composed4")
    assert kg.kg_get_scheme() == kg.KG_SCHEME_COMPOSED4
    u = np.zeros((16, 16, 16))
    kg.kg_set_options(energy_every=5)
    assert kg.lib.kg_init(16, 32.0, 0.01, u.ctypes.data, None) == kg.KG_EINVAL
    assert "composed" in kg.last_error()
    kg.kg_set_options(drift_tol=1e-6)
    assert kg.lib.kg_init(16, 32.0, 0.01, u.ctypes.data, None) == kg.KG_EINVAL
    kg.kg_set_options()
    uc = np.zeros((16, 16, 16), dtype=np.complex128)
    assert kg.lib.kg_init_complex(16, 32.0, 0.01, uc.ctypes.data, None) == kg.KG_ENOTSUP
    kg.kg_set_scheme()
    assert kg.kg_get_scheme() == kg.KG_SCHEME_EQ2


def _rotl_sum(payload):
    """the checkpoint checksum as kg.h defines it: sum mod 2^64 of word i rotated left by i mod 64"""
    w = np.frombuffer(payload.tobytes(), dtype="<u8")
    r = (np.arange(w.size) % 64).astype(np.uint64)
    rot = np.where(r == 0, w, (w << r) | (w >> ((np.uint64(64) - r) % np.uint64(64))))
    return int(sum(int(x) for x in rot) % (1 << 64))


def test_state_checksum_definition(kg):
    rng = np.random.default_rng(9)
    for n in (0, 8, 8 * 63, 8 * 64, 8 * 65, 8 * 1000):
        p = rng.integers(0, 256, size=n, dtype=np.uint8)
        assert kg.kg_state_checksum(p) == _rotl_sum(p)
    # order matters: swapping two distinct words changes the sum
    p = np.arange(16, dtype=np.uint64).view(np.uint8)
    q = p.copy().view(np.uint64)
    q[[2, 3]] = q[[3, 2]]
    assert kg.kg_state_checksum(p) != kg.kg_state_checksum(q.view(np.uint8))


def _checkpoint(kg, N=16, **over):
    h = kg.kg_state_header()
    h.magic = kg.KG_STATE_MAGIC
    h.version = kg.KG_STATE_VERSION
    h.header_bytes = kg.STATE_HEADER_BYTES
    h.N, h.precision, h.energy_every, h.frozen = N, kg.KG_DF64, 0, 0
    h.L, h.dt, h.nonlinearity = 32.0, 0.01, 1.0
    h.blowup_level = -1
    arr = 16 * N * N * (N // 2 + 1)
    payload = np.random.default_rng(1).integers(0, 256, size=2 * arr, dtype=np.uint8)
    h.payload_bytes = 2 * arr
    h.checksum = kg.kg_state_checksum(payload)
    for k, v in over.items():
        setattr(h, k, v)
    return np.concatenate([np.frombuffer(bytes(h), dtype=np.uint8), payload])


def test_checkpoint_rejected_on_the_host(kg):
    """every malformed checkpoint is refused before any CUDA call, with KG_EINVAL or KG_ENOTSUP"""
    kg.lib.kg_finalize()
    used = C.c_size_t(0)
    assert kg.lib.kg_save_state(None, 0, C.byref(used)) == kg.KG_ESTATE
    assert kg.lib.kg_load_state(None, 0) == kg.KG_EINVAL
    good = _checkpoint(kg)
    assert kg.lib.kg_load_state(good.ctypes.data, 100) == kg.KG_EINVAL
    cases = [
        (dict(magic=b"KGSTATE2"), kg.KG_EINVAL, "magic"),
        (dict(version=2), kg.KG_EINVAL, "version"),
        (dict(header_bytes=255), kg.KG_EINVAL, "header"),
        (dict(N=17), kg.KG_ENOTSUP, "N"),
        (dict(precision=9), kg.KG_EINVAL, "precision"),
        (dict(dt=0.0), kg.KG_EINVAL, "range"),
        (dict(L=float("nan")), kg.KG_EINVAL, "range"),
        (dict(energy_every=-1), kg.KG_EINVAL, "range"),
        (dict(level=-3), kg.KG_EINVAL, "range"),
        (dict(frozen=2), kg.KG_EINVAL, "range"),
        (dict(payload_bytes=8), kg.KG_EINVAL, "payload"),
        (dict(scheme=5), kg.KG_EINVAL, "range"),
        (dict(scheme=kg.KG_SCHEME_COMPOSED4, energy_every=3), kg.KG_EINVAL, "range"),
    ]
    for over, code, word in cases:
        b = _checkpoint(kg, **over)
        assert kg.lib.kg_load_state(b.ctypes.data, b.size) == code, over
        assert word in kg.last_error(), (over, kg.last_error())
    assert kg.lib.kg_load_state(good.ctypes.data, good.size - 1) == kg.KG_EINVAL
    assert "truncated" in kg.last_error()
    bad = good.copy()
    bad[kg.STATE_HEADER_BYTES + 1000] ^= 1
    assert kg.lib.kg_load_state(bad.ctypes.data, bad.size) == kg.KG_EINVAL
    assert "checksum" in kg.last_error()
    # a refused checkpoint leaves the options alone
    kg.kg_set_options(precision="mixed", energy_every=3)
    b = _checkpoint(kg, frozen=5)
    assert kg.lib.kg_load_state(b.ctypes.data, b.size) == kg.KG_EINVAL
    assert kg.kg_get_options()["precision"] == kg.KG_MIXED
    assert kg.kg_get_options()["energy_every"] == 3
    kg.kg_set_options()


def test_complex_entry_points_reject_bad_arguments_on_the_host(kg):
    kg.lib.kg_finalize()
    N = 16
    u = np.zeros((N, N, N), dtype=np.complex128)
    assert kg.lib.kg_init_complex(17, 32.0, 0.01, u.ctypes.data, None) == kg.KG_ENOTSUP
    assert kg.lib.kg_init_complex(N, 32.0, -0.01, u.ctypes.data, None) == kg.KG_EINVAL
    assert kg.lib.kg_init_complex(N, 32.0, 0.01, None, None) == kg.KG_EINVAL
    bad = u.copy()
    bad[2, 3, 4] = complex(np.inf, 0.0)
    assert kg.lib.kg_init_complex(N, 32.0, 0.01, bad.ctypes.data, None) == kg.KG_EINVAL
    v = u.copy()
    v[0, 0, 1] = complex(0.0, np.nan)          # the imaginary parts are checked too
    assert kg.lib.kg_init_complex(N, 32.0, 0.01, u.ctypes.data, v.ctypes.data) == kg.KG_EINVAL
    out = np.empty((N, N, N), dtype=np.complex128)
    assert kg.lib.kg_fetch_complex(out.ctypes.data) == kg.KG_ESTATE
    assert kg.lib.kg_fetch_complex_device(None) == kg.KG_ESTATE


def test_large_field_finiteness_check_on_the_host(kg):
    """fields above 4M values are checked by several host threads: a bad value in any
    chunk, the last one included, is still found before anything touches the GPU"""
    N = 256
    u = np.zeros((N, N, N))
    for pos in [(0, 0, 0), (128, 7, 3), (N - 1, N - 1, N - 1)]:
        u[pos] = np.nan
        assert kg.lib.kg_init(N, 32.0, 0.01, u.ctypes.data, None) == kg.KG_EINVAL
        u[pos] = -np.inf
        assert kg.lib.kg_init(N, 32.0, 0.01, u.ctypes.data, None) == kg.KG_EINVAL
        u[pos] = 0.0


def test_ensemble_and_network_arguments_rejected_on_the_host(kg):
    ok_N = np.array([64, 128], dtype=np.int32)
    A = np.array([1.0, 2.0])
    s = np.array([1.0, 1.5])
    lib = kg.lib
    assert lib.kg_ens_init(0, ok_N.ctypes.data, 32.0, 0.005, A.ctypes.data, s.ctypes.data) == kg.KG_EINVAL
    assert lib.kg_ens_init(1025, ok_N.ctypes.data, 32.0, 0.005, A.ctypes.data, s.ctypes.data) == kg.KG_EINVAL
    assert lib.kg_ens_init(2, None, 32.0, 0.005, A.ctypes.data, s.ctypes.data) == kg.KG_EINVAL
    assert lib.kg_ens_init(2, ok_N.ctypes.data, 32.0, -1.0, A.ctypes.data, s.ctypes.data) == kg.KG_EINVAL
    bad_N = np.array([64, 96], dtype=np.int32)
    assert lib.kg_ens_init(2, bad_N.ctypes.data, 32.0, 0.005, A.ctypes.data, s.ctypes.data) == kg.KG_ENOTSUP
    bad_A = np.array([1.0, np.nan])
    assert lib.kg_ens_init(2, ok_N.ctypes.data, 32.0, 0.005, bad_A.ctypes.data, s.ctypes.data) == kg.KG_EINVAL
    bad_s = np.array([1.0, 0.0])
    assert lib.kg_ens_init(2, ok_N.ctypes.data, 32.0, 0.005, A.ctypes.data, bad_s.ctypes.data) == kg.KG_EINVAL
    # calls that need an ensemble or a network before one exists
    done = C.c_longlong()
    ms = C.c_double()
    lib.kg_ens_finalize()
    assert lib.kg_ens_run(10, 0.0, C.byref(done), C.byref(ms)) == kg.KG_ESTATE
