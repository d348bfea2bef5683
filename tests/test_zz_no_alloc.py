"""kg_energy_q_noalloc: the quadratic energy of a caller-held state pair, computed with
no device allocation (partial sums in the library's static device scratch).

It serves callers that cannot call cudaMalloc (device memory owned by another
allocator or a fixed pool, or loops that cannot take cudaMalloc's synchronisation).
Checked through the C ABI against the context path: with lam = 0 the energy
kg_energy returns is exactly Q^{n-1/2}, computed there with allocated scratch.
Two calls in a row, so the second sees the scratch the first one left behind.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 32.0


@pytest.fixture(scope="module")
def kg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build_library()
    from paper_1501_04552_gb300 import kg as K
    yield K
    K.kg_finalize()
    K.kg_set_options()


def test_noalloc_q_matches_context_energy_twice(kg):
    import torch
    N, dt = 64, 0.02
    u0 = I.gaussian(N, L, 1.3, 2.0) + 0.05 * I.plane_wave(N, L, (3, -1, N // 2), "cos")
    v0 = 0.3 * I.gaussian(N, L, 1.0, 2.5)
    kg.kg_set_options(precision="df64", nonlinearity=0.0)
    kg.kg_init(N, L, dt, u0, v0)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        kg.kg_step(7)
        E = kg.kg_energy()                       # lam = 0: E^{n-1/2} = Q^{n-1/2}
        a, b = kg.kg_fetch_spectral(N)
        d_a = torch.from_numpy(a.view(np.float64)).cuda()
        d_b = torch.from_numpy(b.view(np.float64)).cuda()
        rc = kg.lib.kg_energy_q_noalloc(N, L, dt, d_a.data_ptr(), d_b.data_ptr(), out.data_ptr(), None)
        assert rc == kg.KG_OK, kg.last_error()
        torch.cuda.synchronize()
        q = float(out.item())
        assert abs(q - E) <= 1e-13 * abs(E), (call, q, E)
    kg.kg_set_options()


def test_noalloc_q_at_512_many_partials(kg):
    """512^3: 4112 partial sums, so the final sum's threads each add several of them"""
    import torch
    N, dt = 512, 0.005
    kg.kg_set_options(precision="df64", nonlinearity=0.0)
    kg.kg_init(N, L, dt, I.gaussian(N, L, 1.0, 2.0), 0.2 * I.gaussian(N, L, 1.0, 3.0))
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        kg.kg_step(3)
        E = kg.kg_energy()
        a, b = kg.kg_fetch_spectral(N)
        d_a = torch.from_numpy(a.view(np.float64)).cuda()
        d_b = torch.from_numpy(b.view(np.float64)).cuda()
        del a, b
        rc = kg.lib.kg_energy_q_noalloc(N, L, dt, d_a.data_ptr(), d_b.data_ptr(), out.data_ptr(), None)
        assert rc == kg.KG_OK, kg.last_error()
        torch.cuda.synchronize()
        q = float(out.item())
        assert abs(q - E) <= 1e-13 * abs(E), (call, q, E)
        del d_a, d_b
    kg.kg_finalize()
    kg.kg_set_options()


def test_noalloc_rejects_sizes_beyond_the_static_scratch(kg):
    import torch
    d = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = d.data_ptr()
    assert kg.lib.kg_energy_q_noalloc(646, L, 0.01, p, p, p, None) == kg.KG_ENOTSUP
    assert "static scratch maximum" in kg.last_error()
    assert kg.lib.kg_energy_q_noalloc(15, L, 0.01, p, p, p, None) == kg.KG_ENOTSUP
    assert kg.lib.kg_energy_q_noalloc(16, L, 0.01, None, p, p, None) == kg.KG_EINVAL
