"""GPU parity of the adjacent gap ratio (Sec. 2.2) with the oracle: per-realization means
within FP64 summation-order rounding, ratio counts exact, on unsorted levels, ties,
non-finite levels, every short length, the largest length, and dense eigenvalues of the
model."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import hamiltonian as ham
from oracle import observables as obs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mbl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_00217_gb300 as m
    m.binding.lib()
    return m


def _check(mbl, levels, m=None):
    """levels: nprob x ld array; the first m entries of each row are a realization."""
    E = torch.from_numpy(np.ascontiguousarray(levels)).to(DEV)
    m = levels.shape[1] if m is None else m
    r, c = mbl.gap_ratio(E, m)
    r, c = r.cpu().numpy(), c.cpu().numpy()
    for i in range(levels.shape[0]):
        row = levels[i, :m]
        if not np.all(np.isfinite(row)):
            assert c[i] == 0 and math.isnan(r[i])
            continue
        want, n = obs.gap_ratio_mean(row)
        assert c[i] == n, (i, c[i], n)
        if n == 0:
            assert math.isnan(r[i])
        else:
            assert abs(r[i] - want) <= 1e-13 * max(1.0, abs(want)), (i, r[i], want)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 17, 64, 255, 256, 1000, 4096])
def test_random_levels_every_length(mbl, m):
    rng = np.random.default_rng(m)
    levels = rng.normal(size=(9, m)) * 10.0 ** rng.integers(-3, 4, size=(9, 1))
    _check(mbl, levels)


def test_ties_padding_and_bad_rows(mbl):
    rng = np.random.default_rng(7)
    levels = np.round(rng.uniform(0, 20, size=(12, 40)))  # many exact ties
    levels[3, :] = 5.0                                    # every gap zero: no ratio
    levels[4, 7] = np.nan                                 # non-finite level
    levels[5, 0] = np.inf
    levels[6, :20] = np.sort(levels[6, :20])[::-1]        # descending input
    _check(mbl, levels)
    # rows longer than m: only the first m entries count (ld > m)
    _check(mbl, rng.normal(size=(5, 50)), m=33)


def test_dense_model_levels(mbl):
    # mid-spectrum levels of L = 10 open chains at weak and strong disorder
    rows = []
    for W in (0.5, 8.0):
        for seed in range(4):
            h = wl.fields(10, W, seed)
            ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(10, h)))
            rows.append(ev[63:189])
    _check(mbl, np.array(rows))


def test_empty_batch_is_a_no_op(mbl):
    E = torch.empty((0, 8), dtype=torch.float64, device=DEV)
    r, c = mbl.gap_ratio(E)
    assert r.numel() == 0 and c.numel() == 0
