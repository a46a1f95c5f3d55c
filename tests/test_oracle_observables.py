"""Pins of the oracle's adjacent gap ratio (Sec. 2.2) against values fixed independently of
it: a worked example by hand, the two closed-form means of random-matrix theory, its
invariances, and the localization trend of the model itself at small L."""
import math

import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import observables as obs


def test_worked_example():
    # levels 0, 1, 3, 4, 8 (given out of order): gaps 1, 2, 1, 4 -> ratios 1/2, 1/2, 1/4
    r = obs.gap_ratios([3.0, 0.0, 8.0, 1.0, 4.0])
    assert np.allclose(r, [0.5, 0.5, 0.25], rtol=0, atol=0)
    mean, n = obs.gap_ratio_mean([3.0, 0.0, 8.0, 1.0, 4.0])
    assert n == 3 and mean == pytest.approx(5.0 / 12.0, abs=1e-15)


def test_degenerate_and_short_inputs():
    # a level with both gaps zero has no ratio; one zero gap gives r = 0
    assert np.array_equal(obs.gap_ratios([1.0, 1.0, 1.0, 2.0]), [0.0])
    assert obs.gap_ratios([2.0, 5.0]).size == 0
    mean, n = obs.gap_ratio_mean([7.0])
    assert n == 0 and math.isnan(mean)
    with pytest.raises(ValueError):
        obs.gap_ratios([0.0, np.nan, 1.0])


def test_invariant_under_shift_scale_and_order():
    rng = np.random.default_rng(1)
    E = rng.normal(size=200)
    base = obs.gap_ratio_mean(E)[0]
    assert obs.gap_ratio_mean(3.5 * E - 7.0)[0] == pytest.approx(base, rel=1e-12)
    assert obs.gap_ratio_mean(rng.permutation(E))[0] == pytest.approx(base, rel=1e-15)
    assert obs.gap_ratio_mean(-E)[0] == pytest.approx(base, rel=1e-12)


def test_poisson_mean_is_2ln2_minus_1():
    # independent uniform levels: the gaps of a Poisson process, <r> = 2 ln 2 - 1
    rng = np.random.default_rng(2)
    reals = [rng.uniform(0.0, 1.0, 2000) for _ in range(50)]
    got = obs.gap_ratio_average(reals)
    # ~100,000 ratios, standard deviation of r ~ 0.29: 5 sigma = 0.005
    assert abs(got - (2 * math.log(2) - 1)) < 0.005


def test_goe_3x3_surmise_mean_is_4_minus_2sqrt3():
    # the middle level of 3 x 3 GOE matrices: <r> = 4 - 2 sqrt(3) exactly (Atas et al. 2013)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(60000, 3, 3))
    A = (A + np.swapaxes(A, 1, 2)) / 2.0
    got = obs.gap_ratio_average(list(np.linalg.eigvalsh(A)))
    assert abs(got - (4 - 2 * math.sqrt(3))) < 0.005


def test_model_trend_weak_vs_strong_disorder():
    # mid-spectrum levels of the open L = 12 chain: level repulsion at weak disorder,
    # Poisson-like statistics deep in the localized phase
    def mean_r(W, seeds):
        reals = []
        for sd in seeds:
            h = np.random.default_rng(sd).uniform(-W, W, 12)
            ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(12, h)))
            reals.append(ev[len(ev) // 4: 3 * len(ev) // 4])
        return obs.gap_ratio_average(reals)
    weak, strong = mean_r(0.5, range(6)), mean_r(12.0, range(6))
    assert weak > 0.48 and strong < 0.43 and weak - strong > 0.08
