"""Edge cases of the path's variants against the oracle, through the C ABI:
patch equal to the array, singleton axes, search window 1 (the reference
alone), group size 1, for the Poisson matching distances and policies, soft
thresholding, windowed weights and the shared-source variance, one at a
time and all together, with and without mass conservation."""
import numpy as np
import pytest

from paper_2609_34622_b300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu

SHAPES = [((8, 8), (8, 8), (3, 3), (19, 19), (16, 32)),
          ((1, 300), (1, 16), (1, 4), (1, 33), (16, 32)),
          ((300, 1), (16, 1), (4, 1), (33, 1), (16, 32)),
          ((30, 30), (4, 4), (2, 2), (1, 1), (16, 32)),
          ((30, 30), (4, 4), (2, 2), (5, 5), (1, 1)),
          ((17,), (17,), (1,), (3,), (2, 2)),
          ((9, 8, 7), (3, 3, 3), (2, 2, 2), (3, 3, 3), (8, 8))]

VARIANTS = {
    "deviance-reference": dict(match_metric="poisson_deviance", match_policy="reference_finite_count"),
    "pearson-standardized": dict(match_metric="pearson", match_policy="candidate_standardized", match_t=1.0),
    "anscombe-fixed": dict(match_metric="anscombe_ssd", match_policy="fixed", match_t=1.0),
    "soft": dict(ht_rule="soft"),
    "windowed": dict(weight_domain="windowed_synthesis"),
    "shared-source": dict(cov_planes=4),
    "all": dict(match_metric="poisson_deviance", match_policy="reference_finite_count", ht_rule="soft",
                weight_domain="windowed_synthesis", cov_planes=2),
}


@pytest.fixture(scope="module")
def ctx():
    import paper_2609_34622_b300.bmnd as bm
    from paper_2609_34622_b300 import build as B
    B.build()
    c = bm.Context(0)
    yield c
    c.close()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to("cuda:0")


@pytest.mark.parametrize("variant", list(VARIANTS), ids=list(VARIANTS))
@pytest.mark.parametrize("mc", [0, 3])
def test_variant_edge_shapes(ctx, oracle, variant, mc):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    kw = VARIANTS[variant]
    rng = np.random.default_rng(71)
    for shape, patch, step, search, gs in SHAPES:
        x = rng.uniform(0.2, 1.0, size=shape)
        y, sp = synth.poisson_observe(x, 20.0, rng)
        noise = ("poisson", sp)
        p = oracle.params(shape, patch, step, search, noise, gs, 2, mc, **kw)
        ref = PT.oracle_two_stages_f32_pilot(oracle, p, y)
        out = torch.empty(shape, dtype=torch.float32, device="cuda:0")
        ctx.bmnd_denoise(_cuda(y), out, noise, patch, step, search, gs, 2, mc, bm.params(**kw))
        got = out.cpu().numpy()
        PT.assert_voxels(got, ref, 1.0, what="%s %s" % (variant, shape))
        if mc == 3:
            assert float(got.astype(np.float64).sum()) == pytest.approx(float(y.astype(np.float64).sum()),
                                                                        rel=1e-4)
