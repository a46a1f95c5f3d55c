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


# ---------------------------------------------------------------- entanglement entropy
def _word(up_sites):
    return sum(1 << i for i in up_sites)


def _vec(states, amp):
    v = np.zeros(states.size)
    for word, a in amp.items():
        v[int(np.searchsorted(states, word))] = a
    return v


def test_entropy_of_product_states_is_zero():
    st = ham.basis(10, 5)
    for r in (0, 17, st.size - 1):
        v = np.zeros(st.size)
        v[r] = 1.0
        for l_a in (1, 4, 5, 9):
            assert obs.entanglement_entropy(st, v, l_a) == 0.0


def test_entropy_of_singlets_across_the_cut():
    st = ham.basis(10, 5)
    base = _word([0, 1, 6, 7])
    # one singlet on the bond (4, 5) that the cut after 5 sites crosses: ln 2
    v = _vec(st, {base | _word([4]): 1.0, base | _word([5]): -1.0})
    assert obs.entanglement_entropy(st, v, 5) == pytest.approx(math.log(2), abs=1e-14)
    # the same vector cut after 3 sites: the singlet is on the right, S = 0
    assert obs.entanglement_entropy(st, v, 3) == pytest.approx(0.0, abs=1e-14)
    # two singlets (4, 5) and (3, 6) crossing the cut: 2 ln 2 (sign and norm do not matter)
    b2 = _word([0, 1, 7])
    amp = {}
    for a, sa in (((4,), 1.0), ((5,), -1.0)):
        for b, sb in (((3,), 1.0), ((6,), -1.0)):
            amp[b2 | _word(a + b)] = 3.0 * sa * sb
    v2 = _vec(st, amp)
    assert obs.entanglement_entropy(st, -v2, 5) == pytest.approx(2 * math.log(2), abs=1e-13)


@pytest.mark.parametrize("L,l_a", [(10, 5), (10, 3), (12, 6), (12, 7)])
def test_entropy_matches_free_fermion_closed_form(L, l_a):
    # delta = 0, open chain: eigenstates are Slater determinants; the dense eigenvector of
    # the matching energy must carry the correlation-matrix entropy of its modes
    from oracle import closed_form as cf
    rng = np.random.default_rng(L + 10 * l_a)
    h = rng.uniform(-2.0, 2.0, L)
    n_up = L // 2
    st = ham.basis(L, n_up)
    ev, V = np.linalg.eigh(ham.dense_sector(ham.Chain(L, h, delta=0.0)))
    checked = 0
    for trial in range(12):
        occ = sorted(rng.choice(L, n_up, replace=False)) if trial else list(range(n_up))
        E, S = cf.free_fermion_entropy(L, h, occ, l_a)
        j = int(np.argmin(np.abs(ev - E)))
        gaps = np.abs(np.delete(ev, j) - ev[j])
        if abs(ev[j] - E) > 1e-10 or gaps.min() < 1e-6:
            continue  # degenerate within the tolerance: no unique eigenvector to compare
        assert obs.entanglement_entropy(st, V[:, j], l_a) == pytest.approx(S, abs=1e-9)
        checked += 1
    assert checked >= 6


def test_entropy_bounded_by_the_reduced_rank():
    from math import comb
    rng = np.random.default_rng(5)
    L, l_a = 12, 6
    st = ham.basis(L, 6)
    rank = sum(min(comb(l_a, p), comb(L - l_a, 6 - p)) for p in range(0, 7))
    for _ in range(3):
        S = obs.entanglement_entropy(st, rng.normal(size=st.size), l_a)
        assert 0.0 < S <= math.log(rank) + 1e-12
