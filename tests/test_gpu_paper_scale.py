"""Paper-scale parity after the stated step count.

The 512^3 workload (u0 = 0.1 exp(-|x|^2) plus low-passed noise, seed 1501, L = 32,
dt = 0.005, u_t(0) = 0) is stepped 200 times by the scheme of Eq. (2) with the energy
of section 1.1 (the discrete form E^{n-1/2} of the library header) read every 10 steps,
through kg_init / kg_step / kg_energy / kg_fetch, in the launch configuration the
benchmark times, and compared element by element with the FP64 CPU oracle stepped the
same way on the same u0:

  * double-float and IEEE-FP64 passes: relative L2 of u^200 <= 1e-12, each of the 21
    energies within 1e-12 (relative) of the oracle's;
  * FP32 passes (the FP32/FP64 split): relative L2 of u^200 <= 1e-5, energies within 1e-6.

The oracle takes several minutes at this size on the host cores; it runs in a thread
(the C oracle releases the interpreter lock) while the three GPU runs proceed.
"""
import concurrent.futures as cf

import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N, L, DT, STEPS, EVERY = 512, 32.0, 0.005, 200, 10
TOL = {"df64": (1e-12, 1e-12), "fp64": (1e-12, 1e-12), "mixed": (1e-5, 1e-6)}


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


@pytest.fixture(scope="module")
def workload():
    return I.bump_noise(N)


def _oracle_run(u0):
    from oracle import oracle as O
    s = O.Solver(N, L, DT, u0, None)
    energies = [s.energy()]
    for _ in range(STEPS // EVERY):
        s.step(EVERY)
        energies.append(s.energy())
    u = s.fetch()
    s.close()
    return u, np.array(energies)


@pytest.fixture(scope="module")
def oracle_future(workload):
    ex = cf.ThreadPoolExecutor(max_workers=1)
    fut = ex.submit(_oracle_run, workload["u0"])
    yield fut
    ex.shutdown(wait=True)


@pytest.fixture(scope="module")
def gpu_runs(kg, workload, oracle_future):
    out = {}
    for prec in TOL:
        kg.kg_set_options(precision=prec, energy_every=EVERY)
        kg.kg_init(N, L, DT, workload["u0"], None)
        es = [kg.kg_energy()]
        for _ in range(STEPS // EVERY):
            kg.kg_step(EVERY)
            es.append(kg.kg_energy())
        out[prec] = (kg.kg_fetch(N), np.array(es))
        kg.kg_finalize()
    kg.kg_set_options()
    return out


@pytest.mark.parametrize("prec", list(TOL))
def test_200_steps_match_oracle(gpu_runs, oracle_future, prec):
    u_ref, e_ref = oracle_future.result()
    u, e = gpu_runs[prec]
    tol_u, tol_e = TOL[prec]
    err = float(np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref))
    assert err <= tol_u, (prec, err)
    assert e.shape == e_ref.shape == (STEPS // EVERY + 1,)
    rel_e = np.abs(e - e_ref) / np.abs(e_ref)
    print("paper-scale %s: relative L2 of u^200 %.3e, largest relative energy difference %.3e"
          % (prec, err, rel_e.max()))
    assert rel_e.max() <= tol_e, (prec, rel_e.max(), int(rel_e.argmax()))
