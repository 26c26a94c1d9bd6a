"""Parity of the reference-coverage analysis (Sec. 9.3) of the CUDA path with
the oracle, through the C ABI: the coverage map bit for bit, the reference
count exactly and the CV to rounding, over schedules, shift densities,
passes and 1-D to 4-D shapes with singleton axes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [((8,), (3,), (2,), "off", 2.0, 1), ((481, 321), (8, 8), (3, 3), "generated", 2.0, 2),
         ((256, 256), (8, 8), (3, 3), "balanced", 2.0, 2), ((41, 37), (8, 8), (3, 3), "generated", 4.0, 1),
         ((37, 29), (5, 4), (3, 2), "balanced", 4.0, 2), ((1, 40, 17), (1, 6, 5), (1, 4, 3), "sparse", 2.0, 2),
         ((20, 18, 16), (4, 4, 4), (2, 2, 2), "generated", 2.0, 2), ((9, 7, 5, 6), (3, 2, 2, 3), (2, 1, 2, 2),
                                                                     "generated", 1.0, 2),
         ((262144,), (32,), (4,), "generated", 2.0, 2), ((23, 31), (6, 6), (4, 5), "off", 2.0, 1)]


@pytest.fixture(scope="module")
def ctx():
    import paper_2609_34622_b300.bmnd as bm
    from paper_2609_34622_b300 import build as B
    B.build()
    c = bm.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("shape,patch,step,sched,rho,K", CASES,
                         ids=["x".join(map(str, c[0])) + "-" + c[3] + "-%g-%d" % (c[4], c[5]) for c in CASES])
def test_coverage_bit_exact(ctx, oracle, shape, patch, step, sched, rho, K):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    cov = torch.full(shape, -1, dtype=torch.int32, device="cuda:0")
    n, cv = ctx.bmnd_coverage(shape, patch, step, bm.params(schedule=sched, shift_density=rho, passes=K),
                              coverage=cov)
    ref, rn, rcv = oracle.coverage(oracle.params(shape, patch, step, (1,) * len(shape), schedule=sched,
                                                 shift_density=rho, passes=K))
    np.testing.assert_array_equal(cov.cpu().numpy(), ref)
    assert n == rn
    assert cv == pytest.approx(rcv, rel=1e-12, abs=1e-15)
    n2, cv2 = ctx.bmnd_coverage(shape, patch, step, bm.params(schedule=sched, shift_density=rho, passes=K))
    assert (n2, cv2) == (n, cv)


def test_coverage_rejections(ctx):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    with pytest.raises(ValueError):
        ctx.bmnd_coverage((16, 16), (4, 4), (2, 2), coverage=torch.zeros((16, 16), device="cuda:0"))
    with pytest.raises(ValueError):
        ctx.bmnd_coverage((16, 16), (4, 4), (2, 2), coverage=torch.zeros((15, 16), dtype=torch.int32, device="cuda:0"))
    with pytest.raises(bm.BmndError):
        ctx.bmnd_coverage((16, 16), (4, 4), (5, 2))
