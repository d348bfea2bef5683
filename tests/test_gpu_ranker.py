"""A reduced ranker study end to end on the GPU: solver labels, training, sweep
ranking, judging and the gain measurements (short horizon T = 1.5 so it runs fast)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build_library()
    from paper_1501_04552_gb300 import kg as K
    yield K
    K.kg_mlp_finalize()
    K.kg_ens_finalize()


def test_reduced_study(kg):
    from paper_1501_04552_gb300 import ranker as R
    res = R.run(n_train=768, n_sweep=4096, n_judge=128, T=1.5, epochs=120, n_s=8, width=0.08, guess=0.15,
                band=0.15, precision="mixed")
    assert 0.05 < res["blowup_fraction"] < 0.95
    assert res["heldout_auc"] > 0.95
    assert res["judged_label_accuracy_uniform"] > 0.9
    # points the network ranks near p = 1/2 sit near the solver's boundary far more often
    assert res["near_boundary_gain"] > 2.0
    assert res["boundary_max_disagreement"] <= 0.08 + 1e-12
