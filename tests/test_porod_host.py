"""pf_porod_fit is host arithmetic in the library (no device work), so it is checked here
against the oracle's Porod fit (Sec. 3) on any machine."""
import numpy as np
import pytest

import oracle
from paper_2109_02598_gb300 import _lib
from paper_2109_02598_gb300.build import build


@pytest.fixture(scope="module")
def pf():
    build()
    import paper_2109_02598_gb300 as pf
    return pf


@pytest.mark.parametrize("seed", range(4))
def test_matches_oracle(pf, seed):
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(8, 200))
    c = (np.arange(nb) + 0.5) * (np.pi * np.sqrt(2) / nb)
    m = np.exp(rng.normal(0, 0.5, nb)) * c ** rng.uniform(-4.5, -1.5)
    n = rng.integers(0, 40, nb)
    m[rng.integers(0, nb, 3)] = 0.0
    lo, hi = sorted(rng.uniform(0.1, 3.0, 2))
    if ((c >= lo) & (c <= hi) & (n > 0) & (m > 0)).sum() < 2:
        lo, hi = 0.0, 5.0
    ref = oracle.porod_fit(c, m, n, lo, hi)
    got = pf.porod_fit(c, m, n, lo, hi)
    assert got[2] == ref[2]
    assert abs(got[0] - ref[0]) <= 1e-12 * max(1.0, abs(ref[0]))
    assert abs(got[1] - ref[1]) <= 1e-12 * max(1.0, abs(ref[1]))


def test_rejects_bad_windows(pf):
    c = np.array([0.5, 1.0, 1.5])
    m = np.array([1.0, 0.5, 0.2])
    n = np.array([1, 1, 1])
    with pytest.raises(pf.PfError, match="k_lo < k_hi"):
        pf.porod_fit(c, m, n, 1.0, 1.0)
    with pytest.raises(pf.PfError, match="fewer than two"):
        pf.porod_fit(c, m, n, 1.2, 2.0)
    with pytest.raises(pf.PfError, match="fewer than two"):
        pf.porod_fit(c, m, np.array([0, 1, 0]), 0.0, 2.0)
    assert _lib.load().pf_porod_fit(3, None, None, None, 0.0, 1.0, None, None, None) == \
        _lib.PF_ERR_INVALID_ARG
