"""Launch configurations of the direct epipolar kernel (tile, CTAs per SM)
and the autotuner that picks one: every configuration gives the oracle's
loss and gradient; configurations that differ only in the number of CTAs
process the same warp runs and give identical bits."""
import numpy as np
import pytest

from synthetic.scenes import make_scene
from tests import _gpu as G
from tests._util import perturbed_params_ea

pytestmark = pytest.mark.gpu


def _eval(pr, p):
    import torch
    from paper_2505_04612_b300 import fastmap as F
    L, g = pr.loss_grad(F.FM_STAGE_EPIPOLAR, torch.from_numpy(np.asarray(p, np.float32).reshape(-1)).cuda())
    return L, g.cpu().numpy()


@pytest.mark.parametrize("U", [11, 15, 21])
def test_every_configuration_matches_the_oracle(U):
    from paper_2505_04612_b300 import fastmap as F
    sc = make_scene("c2", 3, n_cams=40, n_points=8000)
    xs = G.oracle_xs(sc)
    p = perturbed_params_ea(sc, 1)
    Lo, go = G.ea_oracle(sc, p, "l2", xs=xs)
    with G.make_problem(sc) as pr:
        pr.set_ea_loss(F.FM_EA_L2)
        ref = None
        for ctas in (1, 2, 3, 0):
            pr.set_tuning(U, ctas)
            assert pr.get_tuning() == dict(pairs_per_lane=U, ctas_per_sm=ctas)
            L, g = _eval(pr, p)
            assert abs(L - Lo) <= 1e-5 * Lo
            assert G.rel_err(g.reshape(go.shape), go) < 1e-4
            if ctas == 1:
                ref = g
            else:
                np.testing.assert_array_equal(g, ref)   # same warp runs, other CTAs


def test_autotune_picks_a_valid_configuration():
    from paper_2505_04612_b300 import fastmap as F
    sc = make_scene("c1", 2)
    xs = G.oracle_xs(sc)
    p = perturbed_params_ea(sc, 3)
    with G.make_problem(sc) as pr:
        pr.set_ea_loss(F.FM_EA_L2)   # the autotuner times L1 evaluations and leaves the loss as it was
        t = pr.autotune(repeats=3)
        assert t["pairs_per_lane"] in (11, 15, 21) and t["ctas_per_sm"] >= 1
        assert t["us_per_eval"] > 0
        assert pr.get_tuning() == {k: t[k] for k in ("pairs_per_lane", "ctas_per_sm")}
        L, g = _eval(pr, p)
    Lo, go = G.ea_oracle(sc, p, "l2", xs=xs)
    assert abs(L - Lo) <= 1e-5 * Lo
    assert G.rel_err(g.reshape(go.shape), go) < 1e-4


def test_invalid_tuning_is_rejected():
    from paper_2505_04612_b300 import fastmap as F
    sc = make_scene("c1", 2)
    with G.make_problem(sc) as pr:
        for bad in [(13, 0), (15, -1), (7, 2), (31, 2)]:
            with pytest.raises(F.FastMapError) as e:
                pr.set_tuning(*bad)
            assert e.value.status == F.FM_ERR_INVALID_ARG
        assert pr.get_tuning()["pairs_per_lane"] == 15
