"""Pins of the oracle's Porod-law fit (Sec. 3): an exact power law is recovered exactly, the
fit agrees with an independent least-squares routine, the window and the empty bins are
honoured, and a coarsened Model A state from the oracle's spectral solver shows the
k^-(d+1) tail the paper uses to validate its solutions."""
import numpy as np
import pytest

import oracle
import synthetic


def test_exact_power_law_is_recovered():
    c = np.linspace(0.05, 3.0, 40)
    m = 2.5 * c ** -3.0
    slope, icpt, n = oracle.porod_fit(c, m, np.ones(40, dtype=np.int64), 0.2, 2.0)
    assert abs(slope + 3.0) < 1e-12 and abs(icpt - np.log(2.5)) < 1e-12
    assert n == int(((c >= 0.2) & (c <= 2.0)).sum())


def test_agrees_with_library_least_squares_and_skips_unusable_bins():
    rng = np.random.default_rng(3)
    c = np.linspace(0.1, 2.0, 30)
    m = np.exp(rng.normal(0, 0.3, 30)) * c ** -2.2
    cnt = np.ones(30, dtype=np.int64)
    cnt[5] = 0      # empty bin
    m[9] = 0.0      # S = 0 has no logarithm
    slope, icpt, n = oracle.porod_fit(c, m, cnt, 0.3, 1.8)
    sel = (c >= 0.3) & (c <= 1.8) & (cnt > 0) & (m > 0)
    ref = np.polyfit(np.log(c[sel]), np.log(m[sel]), 1)
    assert n == sel.sum()
    assert abs(slope - ref[0]) < 1e-10 and abs(icpt - ref[1]) < 1e-10


def test_too_few_bins_is_an_error():
    with pytest.raises(ValueError):
        oracle.porod_fit([1.0, 2.0], [1.0, 1.0], [1, 1], 1.5, 3.0)


@pytest.mark.slow
def test_coarsened_model_a_follows_porods_law():
    # Model A quenched from U(-1, 1), 2D 256^2, t = 100, S(k) averaged over two seeds:
    # the slope of the tail between twice the peak wavenumber and k = 1.5 is -(d + 1) = -3
    Ss = []
    for seed in range(2):
        x0 = synthetic.paper_timing_init("ac", (256, 256), seed=seed)
        x, = oracle.spectral_run("ac", x0, (1.0, 1.0), 0.2, 500)
        c, m, cnt = oracle.structure_factor(x, 1.0, 64)
        Ss.append(m)
    slope, _, n = oracle.porod_fit(c, np.mean(Ss, axis=0), cnt, 0.4, 1.5)
    assert n >= 10
    assert -3.3 < slope < -2.7
