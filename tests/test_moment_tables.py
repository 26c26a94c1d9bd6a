"""Host logic of the Poisson matching calibration: the finite-count moment
tables that the library computes on the host (Pascal-rule Binomial weights)
equal the oracle's (log-gamma weights) after rounding to float32, entry for
entry, for every pooled count 0..4096 (Prop. "Universal finite-count
moments").  Host computation only: no device is touched."""
import numpy as np
import pytest

from paper_2609_34622_b300 import bmnd

METRICS = ("poisson_deviance", "pearson", "anscombe_ssd")


@pytest.mark.parametrize("metric", METRICS)
def test_library_tables_equal_oracle(oracle, metric):
    mu, v = bmnd.bmnd_match_moments(metric)
    omu, ov = oracle.moment_table_f32(metric, bmnd.MOMENT_NMAX + 1)
    assert mu.shape == (4097,)
    bad_mu = np.flatnonzero(mu != omu)
    bad_v = np.flatnonzero(v != ov)
    assert bad_mu.size == 0, (bad_mu[:10], mu[bad_mu[:10]], omu[bad_mu[:10]])
    assert bad_v.size == 0, (bad_v[:10], v[bad_v[:10]], ov[bad_v[:10]])


def test_pearson_table_closed_form():
    """Prop. "Exact Pearson moments" in the library's table."""
    mu, v = bmnd.bmnd_match_moments("pearson", 64)
    n = np.arange(1, 64)
    assert mu[0] == 0 and v[0] == 0
    np.testing.assert_array_equal(mu[1:], np.float32(1.0))
    np.testing.assert_allclose(v[1:], 2 - 2 / n, rtol=1e-7)


def test_invalid_arguments():
    lib = bmnd.load()
    fp = np.zeros(8, np.float32).ctypes.data_as(bmnd.ctypes.POINTER(bmnd.ctypes.c_float))
    assert lib.bmnd_match_moments(0, 4, fp, fp) == 1
    assert lib.bmnd_match_moments(4, 4, fp, fp) == 1
    assert lib.bmnd_match_moments(1, 0, fp, fp) == 1
    assert lib.bmnd_match_moments(1, 4098, fp, fp) == 1
    assert lib.bmnd_match_moments(1, 4, None, fp) == 1
