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


# ---------------------------------------------------------------- entanglement entropy
@pytest.mark.parametrize("L,n_up,l_a", [(8, 4, 4), (10, 5, 5), (10, 5, 1), (10, 5, 9), (11, 4, 6), (12, 6, 6),
                                        (14, 7, 7), (16, 8, 8), (13, 6, 3)])
def test_entropy_random_vectors(mbl, L, n_up, l_a):
    rng = np.random.default_rng(L * 100 + l_a)
    st = ham.basis(L, n_up)
    V = rng.normal(size=(st.size, 5)) * np.array([1.0, 2.5, 1e-3, 1.0, 7.0])
    V[:, 3] = 0.0
    V[7 % st.size, 3] = 1.0  # a basis state: S = 0
    chain = mbl.make_chain(L, np.zeros(L), 1.0, False, n_up)
    S = mbl.entanglement_entropy(chain, l_a, torch.from_numpy(V).to(DEV)).cpu().numpy()
    for e in range(V.shape[1]):
        want = obs.entanglement_entropy(st, V[:, e], l_a)
        assert abs(S[e] - want) <= 1e-10, (e, S[e], want)


def test_entropy_of_eigenvectors_and_strided_input(mbl):
    # eigenvectors of the L = 12 chain at weak and strong disorder (dense), read from a
    # wider row-major block (ld > nvec); a zero column gives NaN
    L = 12
    st = ham.basis(L, 6)
    cols = []
    for W in (0.5, 8.0):
        h = wl.fields(L, W, 3)
        ev, Vd = np.linalg.eigh(ham.dense_sector(ham.Chain(L, h)))
        cols += [Vd[:, 400], Vd[:, 462]]
    V = np.zeros((st.size, 8))
    V[:, :4] = np.array(cols).T
    Vg = torch.from_numpy(V).to(DEV)[:, :5]  # ld = 8, nvec = 5; column 4 is zero
    chain = mbl.make_chain(L, np.zeros(L))
    S = mbl.entanglement_entropy(chain, 6, Vg).cpu().numpy()
    for e in range(4):
        assert abs(S[e] - obs.entanglement_entropy(st, cols[e], 6)) <= 1e-10
    assert math.isnan(S[4])
    # volume-law vs area-law: weak-disorder eigenstates are far more entangled
    assert min(S[0], S[1]) > max(S[2], S[3])


def test_entropy_half_cut_l20_sampled(mbl):
    # the bench size (L = 20, half cut: Gram blocks up to 252 x 252), two random columns
    L = 20
    st = ham.basis(L, 10)
    rng = np.random.default_rng(20)
    V = rng.normal(size=(st.size, 2))
    chain = mbl.make_chain(L, np.zeros(L))
    S = mbl.entanglement_entropy(chain, 10, torch.from_numpy(V).to(DEV)).cpu().numpy()
    for e in range(2):
        assert abs(S[e] - obs.entanglement_entropy(st, V[:, e], 10)) <= 1e-9
