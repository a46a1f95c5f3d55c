"""GPU parity: the CUDA library (through the C ABI) against the oracle.

Integer work (basis, ranks) must match bit for bit.  Products must match the FP64
oracle within a bound derived from the arithmetic: each output element is a sum of
at most |B| + 1 rounded terms, so its error is at most c * u * (|d - sigma| |x_r| +
1/2 sum |x_r'|) with u the unit roundoff of the kernel's type, plus (FP32 only) the
rounding of d - sigma itself, |d_err| <= 6 u32 (sum|h| + |sigma| + delta |B| / 2).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import hamiltonian as ham

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


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


# ---------------------------------------------------------------- basis
@pytest.mark.parametrize("L,n_up", [(2, 1), (5, 2), (12, 6), (12, 0), (12, 12), (13, 4), (16, 8),
                                    (20, 10), (24, 12), (25, 9)])
def test_basis_build_bit_exact(mbl, L, n_up):
    ref = ham.basis(L, n_up)
    n = mbl.basis_size(L, n_up)
    assert n == ref.size
    st = torch.empty(n, dtype=torch.int32, device=DEV)
    mbl.basis_build(L, n_up, st)
    got = st.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("L,n_up", [(12, 6), (18, 9), (26, 13), (28, 14), (32, 16)])
def test_basis_rank_bit_exact(mbl, L, n_up):
    rng = np.random.default_rng(L)
    # valid words from random rank positions (built on the GPU, ranked back) and
    # random words (mostly invalid)
    n = mbl.basis_size(L, n_up)
    q = 200000 if L <= 28 else 20000
    pos = rng.integers(0, n, q)
    words_valid = np.empty(q, dtype=np.uint32)
    # unrank on the CPU by the definition for L <= 24, else via the GPU basis for L <= 28
    if L <= 28:
        st = torch.empty(n, dtype=torch.int32, device=DEV)
        mbl.basis_build(L, n_up, st)
        words_valid = st.cpu().numpy().view(np.uint32)[pos]
    else:
        # popcount-n_up words drawn directly
        for i in range(q):
            bits = rng.choice(L, n_up, replace=False)
            words_valid[i] = np.sum(np.uint64(1) << bits.astype(np.uint64)).astype(np.uint32)
    words_rand = rng.integers(0, 2 ** 32, q, dtype=np.uint64).astype(np.uint32)
    words = np.concatenate([words_valid, words_rand])
    ranks = torch.empty(words.size, dtype=torch.int64, device=DEV)
    mbl.basis_rank(L, n_up, _gpu(words.view(np.int32)), ranks)
    got = ranks.cpu().numpy()
    if L <= 28:
        assert np.array_equal(got[:q], pos)
    # reference for every word: popcount / range check, then the combinatorial sum
    from math import comb
    pc = np.array([bin(int(w)).count("1") for w in words])
    inr = (words.astype(np.uint64) >> np.uint64(L)) == 0 if L < 32 else np.ones(words.size, bool)
    valid = (pc == n_up) & inr
    assert np.all(got[~valid] == -1)
    sample = np.nonzero(valid)[0][:2000]
    for i in sample:
        w, r, j = int(words[i]), 0, 0
        for p in range(32):
            if (w >> p) & 1:
                j += 1
                r += comb(p, j)
        assert got[i] == r


# ---------------------------------------------------------------- product
def _offdiag_abs(chain, X):
    """1/2 sum over neighbours of |x_r'|, via the oracle with zero diagonal."""
    c0 = ham.Chain(chain.L, np.zeros(chain.L), delta=0.0, periodic=chain.periodic, n_up=chain.n_up)
    return ham.apply(c0, 0.0, np.abs(X).astype(np.float64))


def _bound(chain, sigma, X, dtype):
    d = ham.diag(chain) - sigma
    scale = np.abs(d)[:, None] * np.abs(X.astype(np.float64)) + _offdiag_abs(chain, X)
    nb = chain.num_bonds()
    u = np.finfo(dtype).eps
    derr = 6 * u * (np.sum(np.abs(chain.h)) + abs(sigma) + chain.delta * nb / 2 + 1)
    return 4 * (nb + 2) * u * scale + derr * np.abs(X.astype(np.float64)) + 1e-300


CASES = [(10, False, 1.0), (13, True, 0.7), (16, True, 1.0), (18, False, 0.0), (14, False, 1.0)]


@pytest.mark.parametrize("L,periodic,delta", CASES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_apply_matches_oracle(mbl, L, periodic, delta, k, dtype):
    h = wl.fields(L, 8.0, L + k)
    chain = ham.Chain(L, h, delta=delta, periodic=periodic)
    n = ham.sector_dim(L, L // 2)
    X = wl.block(n, k, 100 + k, dtype)
    sigma = 0.37
    ref = ham.apply(chain, sigma, X.astype(np.float64))
    Y = torch.empty((n, k), dtype=torch.float32 if dtype == np.float32 else torch.float64, device=DEV)
    mbl.hamiltonian_apply(mbl.make_chain(L, h, delta, periodic), sigma, _gpu(X), Y)
    got = Y.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    assert np.all(err <= _bound(chain, sigma, X, dtype)), err.max()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_apply_strided_and_odd_sectors(mbl, dtype):
    """Leading dimensions > k, a sector away from half filling, and a ragged k."""
    for (L, n_up, periodic, k, ld) in [(13, 5, True, 8, 12), (12, 3, False, 5, 7), (11, 6, True, 32, 40),
                                       (2, 1, False, 4, 4), (9, 0, True, 3, 3), (8, 8, False, 2, 2)]:
        h = wl.fields(L, 4.0, L * 7 + n_up)
        chain = ham.Chain(L, h, delta=0.9, periodic=periodic, n_up=n_up)
        n = ham.sector_dim(L, n_up)
        Xb = wl.block(n, ld, 7, dtype)
        ref = ham.apply(chain, -0.2, Xb[:, :k].astype(np.float64))
        Yb = torch.full((n, ld), 123.0, dtype=torch.float32 if dtype == np.float32 else torch.float64, device=DEV)
        Xt = _gpu(Xb)
        mbl.hamiltonian_apply(mbl.make_chain(L, h, 0.9, periodic, n_up), -0.2, Xt[:, :k], Yb[:, :k])
        got = Yb.cpu().numpy()
        assert np.all(got[:, k:] == 123.0)  # untouched padding
        err = np.abs(got[:, :k].astype(np.float64) - ref)
        assert np.all(err <= _bound(chain, -0.2, Xb[:, :k], dtype))


def test_apply_deterministic(mbl):
    L, k = 18, 32
    h = wl.fields(L, 8.0, 3)
    n = ham.sector_dim(L, L // 2)
    X = _gpu(wl.block(n, k, 9, np.float32))
    c = mbl.make_chain(L, h, 1.0, True)
    Y1 = torch.empty_like(X)
    Y2 = torch.empty_like(X)
    mbl.hamiltonian_apply(c, 0.1, X, Y1)
    mbl.hamiltonian_apply(c, 0.1, X, Y2)
    assert torch.equal(Y1, Y2)


def test_apply_rejects_bad_arguments(mbl):
    L = 10
    h = wl.fields(L, 1.0, 0)
    n = ham.sector_dim(L, 5)
    X = torch.zeros((n, 4), dtype=torch.float64, device=DEV)
    Y = torch.zeros_like(X)
    with pytest.raises(mbl.MBLError):  # wrong n
        mbl.hamiltonian_apply(mbl.make_chain(L, h, 1.0, False, 4), 0.0, X, Y)
    with pytest.raises(mbl.MBLError):  # in-place
        mbl.hamiltonian_apply(mbl.make_chain(L, h), 0.0, X, X)
    hn = h.copy()
    hn[3] = np.nan
    with pytest.raises(mbl.MBLError):
        mbl.hamiltonian_apply(mbl.make_chain(L, hn), 0.0, X, Y)


@pytest.mark.parametrize("L,k,dtype", [(26, 8, np.float32), (26, 64, np.float32), (24, 32, np.float64),
                                       (28, 16, np.float32)])
def test_apply_full_size_sampled(mbl, L, k, dtype):
    """Full-size sweep shapes: sampled rows against the oracle row product."""
    h = wl.fields(L, 8.0, 0)
    chain = ham.Chain(L, h, periodic=False)
    n = ham.sector_dim(L, L // 2)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    g = torch.Generator(device=DEV)
    g.manual_seed(L * 100 + k)
    X = torch.randn((n, k), generator=g, device=DEV, dtype=tdt)
    Y = torch.empty_like(X)
    mbl.hamiltonian_apply(mbl.make_chain(L, h), 0.5, X, Y)
    rng = np.random.default_rng(k)
    rows = np.unique(np.concatenate([rng.integers(0, n, 300), [0, 1, n // 2, n - 2, n - 1]]))
    # the oracle needs every neighbour row of the sampled rows: copy X back once
    Xh = X.cpu().numpy()
    ref = ham.apply_rows(chain, 0.5, Xh.astype(np.float64), rows)
    got = Y[torch.from_numpy(rows).to(DEV)].cpu().numpy().astype(np.float64)
    d = ham.diag(chain)[rows] - 0.5
    u = np.finfo(dtype).eps
    scale = (np.abs(d)[:, None] + 0.5 * L) * np.abs(Xh).max()
    derr = 6 * u * (np.sum(np.abs(h)) + 0.5 + L)
    assert np.all(np.abs(got - ref) <= 4 * (L + 2) * u * scale + derr * np.abs(Xh).max())


@pytest.mark.parametrize("bits", [-1, 2, 3, 5, 8, 16])
@pytest.mark.parametrize("L,periodic,k,dtype", [(14, True, 8, np.float32), (13, False, 32, np.float64),
                                                (16, True, 64, np.float32), (12, True, 1, np.float32),
                                                (15, False, 4, np.float64)])
def test_apply_every_tile_width(mbl, bits, L, periodic, k, dtype):
    """The tiled kernel for every tile width (and the untiled one) against the oracle."""
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    h = wl.fields(L, 6.0, L * 3 + k)
    chain = ham.Chain(L, h, delta=1.0, periodic=periodic)
    n = ham.sector_dim(L, L // 2)
    X = wl.block(n, k, 7 + bits, dtype)
    ref = ham.apply(chain, -0.3, X.astype(np.float64))
    Y = torch.empty((n, k), dtype=tdt, device=DEV)
    mbl.binding.set_product_tile_bits(k, tdt, bits)
    try:
        mbl.hamiltonian_apply(mbl.make_chain(L, h, 1.0, periodic), -0.3, _gpu(X), Y)
    finally:
        mbl.binding.set_product_tile_bits(k, tdt, 0)
    err = np.abs(Y.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= _bound(chain, -0.3, X, dtype)), err.max()


def _staged_bits(L, k, itemsize):
    """Tile width the staged schedule uses: the widest B <= min(13, L - 2) whose largest
    tile C(B, B/2) * k * itemsize fits in 48 KB."""
    from math import comb
    B = min(13, L - 2)
    while B >= 2 and comb(B, B // 2) * k * itemsize > 48 * 1024:
        B -= 1
    return B


@pytest.mark.parametrize("L,periodic,n_up,k,dtype", [
    (16, True, 8, 32, np.float32), (18, False, 9, 64, np.float32), (14, True, 7, 8, np.float32),
    (13, False, 5, 16, np.float32), (15, True, 7, 4, np.float32), (14, False, 7, 32, np.float64),
    (16, True, 8, 64, np.float64), (12, True, 6, 2, np.float64), (17, True, 8, 16, np.float64)])
def test_staged_schedule_matches_oracle_and_tiled(mbl, L, periodic, n_up, k, dtype):
    """Schedule 3 (whole tiles staged in shared memory by bulk copies) against the
    oracle, and bit for bit against the persistent tiled kernel at the same tile width."""
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    h = wl.fields(L, 7.0, 100 + L + k)
    chain = ham.Chain(L, h, delta=0.9, periodic=periodic, n_up=n_up)
    n = ham.sector_dim(L, n_up)
    X = wl.block(n, k, 11 + k, dtype)
    ref = ham.apply(chain, 0.4, X.astype(np.float64))
    c = mbl.make_chain(L, h, 0.9, periodic, n_up)
    Xg = _gpu(X)
    Ys = torch.full((n, k), float("nan"), dtype=tdt, device=DEV)
    Yt = torch.full((n, k), float("nan"), dtype=tdt, device=DEV)
    B = _staged_bits(L, k, np.dtype(dtype).itemsize)
    try:
        mbl.binding.set_product_schedule(k, tdt, 3)
        mbl.hamiltonian_apply(c, 0.4, Xg, Ys)
        mbl.binding.set_product_schedule(k, tdt, 1)
        mbl.binding.set_product_tile_bits(k, tdt, B)
        mbl.hamiltonian_apply(c, 0.4, Xg, Yt)
    finally:
        mbl.binding.set_product_schedule(k, tdt, 0)
        mbl.binding.set_product_tile_bits(k, tdt, 0)
    ys = Ys.cpu().numpy()
    err = np.abs(ys.astype(np.float64) - ref)
    assert np.all(err <= _bound(chain, 0.4, X, dtype)), err.max()
    assert np.array_equal(ys, Yt.cpu().numpy())


def test_staged_schedule_full_size_sampled(mbl):
    """Schedule 3 at L = 26 (k = 32, FP32): sampled rows against the oracle."""
    L, k = 26, 32
    h = wl.fields(L, 8.0, 7)
    chain = ham.Chain(L, h, periodic=True)
    n = ham.sector_dim(L, L // 2)
    g = torch.Generator(device=DEV)
    g.manual_seed(5)
    X = torch.randn((n, k), generator=g, device=DEV, dtype=torch.float32)
    Y = torch.empty_like(X)
    try:
        mbl.binding.set_product_schedule(k, torch.float32, 3)
        mbl.hamiltonian_apply(mbl.make_chain(L, h, 1.0, True), 0.5, X, Y)
    finally:
        mbl.binding.set_product_schedule(k, torch.float32, 0)
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.integers(0, n, 300), [0, 1, n // 2, n - 2, n - 1]]))
    Xh = X.cpu().numpy()
    ref = ham.apply_rows(chain, 0.5, Xh.astype(np.float64), rows)
    got = Y[torch.from_numpy(rows).to(DEV)].cpu().numpy().astype(np.float64)
    d = ham.diag(chain)[rows] - 0.5
    u = np.finfo(np.float32).eps
    scale = (np.abs(d)[:, None] + 0.5 * L) * np.abs(Xh).max()
    derr = 6 * u * (np.sum(np.abs(h)) + 0.5 + L)
    assert np.all(np.abs(got - ref) <= 4 * (L + 2) * u * scale + derr * np.abs(Xh).max())


@pytest.mark.parametrize("L,periodic,n_up,k,dtype", [
    (16, True, 8, 32, np.float32), (18, False, 9, 64, np.float32), (14, True, 7, 8, np.float32),
    (13, False, 5, 16, np.float32), (15, True, 4, 32, np.float32), (20, True, 10, 32, np.float32),
    (14, False, 7, 32, np.float64), (16, True, 8, 64, np.float64), (12, True, 6, 4, np.float64),
    (17, True, 8, 16, np.float64), (11, True, 9, 8, np.float64)])
@pytest.mark.parametrize("schedule", [4, 5])
def test_ring_schedules_match_oracle_and_tiled(mbl, L, periodic, n_up, k, dtype, schedule):
    """Schedules 4 (streamed) and 5 (slab): a producer warp copies every row block of a
    tile's product into a ring of shared-memory slots.  Against the oracle, and bit for bit
    against the persistent tiled kernel at the same tile width."""
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    B = mbl.binding.product_tile_width(L, tdt, k, schedule)
    if schedule == 5 and not (32 <= k * np.dtype(dtype).itemsize <= 256):
        assert B == 0  # rows outside the slab kernel's range: persistent instead
        B = mbl.binding.product_tile_width(L, tdt, k, 1)
    assert B >= 2
    h = wl.fields(L, 7.0, 200 + L + k)
    chain = ham.Chain(L, h, delta=1.1, periodic=periodic, n_up=n_up)
    n = ham.sector_dim(L, n_up)
    X = wl.block(n, k, 13 + k, dtype)
    ref = ham.apply(chain, -0.7, X.astype(np.float64))
    c = mbl.make_chain(L, h, 1.1, periodic, n_up)
    Xg = _gpu(X)
    Ys = torch.full((n, k), float("nan"), dtype=tdt, device=DEV)
    Yt = torch.full((n, k), float("nan"), dtype=tdt, device=DEV)
    try:
        mbl.binding.set_product_schedule(k, tdt, schedule)
        mbl.hamiltonian_apply(c, -0.7, Xg, Ys)
        mbl.binding.set_product_schedule(k, tdt, 1)
        mbl.binding.set_product_tile_bits(k, tdt, B)
        mbl.hamiltonian_apply(c, -0.7, Xg, Yt)
    finally:
        mbl.binding.set_product_schedule(k, tdt, 0)
        mbl.binding.set_product_tile_bits(k, tdt, 0)
    ys = Ys.cpu().numpy()
    err = np.abs(ys.astype(np.float64) - ref)
    assert np.all(err <= _bound(chain, -0.7, X, dtype)), err.max()
    assert np.array_equal(ys, Yt.cpu().numpy())


@pytest.mark.parametrize("schedule", [4, 5])
def test_ring_schedules_full_size_sampled(mbl, schedule):
    """Schedules 4 and 5 at L = 26 (k = 32, FP32, periodic): sampled rows against the
    oracle."""
    L, k = 26, 32
    h = wl.fields(L, 8.0, 17)
    chain = ham.Chain(L, h, periodic=True)
    n = ham.sector_dim(L, L // 2)
    g = torch.Generator(device=DEV)
    g.manual_seed(6)
    X = torch.randn((n, k), generator=g, device=DEV, dtype=torch.float32)
    Y = torch.empty_like(X)
    try:
        mbl.binding.set_product_schedule(k, torch.float32, schedule)
        mbl.hamiltonian_apply(mbl.make_chain(L, h, 1.0, True), 0.5, X, Y)
    finally:
        mbl.binding.set_product_schedule(k, torch.float32, 0)
    rng = np.random.default_rng(4)
    rows = np.unique(np.concatenate([rng.integers(0, n, 300), [0, 1, n // 2, n - 2, n - 1]]))
    Xh = X.cpu().numpy()
    ref = ham.apply_rows(chain, 0.5, Xh.astype(np.float64), rows)
    got = Y[torch.from_numpy(rows).to(DEV)].cpu().numpy().astype(np.float64)
    d = ham.diag(chain)[rows] - 0.5
    u = np.finfo(np.float32).eps
    scale = (np.abs(d)[:, None] + 0.5 * L) * np.abs(Xh).max()
    derr = 6 * u * (np.sum(np.abs(h)) + 0.5 + L)
    assert np.all(np.abs(got - ref) <= 4 * (L + 2) * u * scale + derr * np.abs(Xh).max())
    assert torch.isfinite(Y).all()


@pytest.mark.parametrize("L,periodic,k,dtype", [(16, True, 32, np.float32), (15, False, 16, np.float64),
                                                (14, True, 3, np.float32)])
def test_autotune_keeps_a_correct_choice(mbl, L, periodic, k, dtype):
    """The autotuner times its candidates on the caller's buffers, keeps one, and the
    products that follow (under the kept choice) still match the oracle."""
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    h = wl.fields(L, 6.0, 40 + L)
    chain = ham.Chain(L, h, periodic=periodic)
    n = ham.sector_dim(L, L // 2)
    c = mbl.make_chain(L, h, 1.0, periodic)
    X = _gpu(wl.block(n, k, 9, dtype))
    Y = torch.empty_like(X)
    choice = mbl.binding.autotune_product(c, X, Y, reps=3)
    if k == 3:  # no tiled kernel for this width: nothing to choose
        assert choice["schedule"] == 0
    else:
        assert choice["schedule"] in (1, 2, 3, 4, 5) and choice["lane_bytes"] in (32, 64)
        assert choice["tile_bits"] >= 2 and choice["microseconds"] > 0
    Xh = X.cpu().numpy()
    mbl.hamiltonian_apply(c, 0.25, X, Y)
    ref = ham.apply(chain, 0.25, Xh.astype(np.float64))
    err = np.abs(Y.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= _bound(chain, 0.25, Xh, dtype)), err.max()


# ---------------------------------------------------------------- Gram (Rayleigh-Ritz)
@pytest.mark.parametrize("n,p,q", [(1000, 8, 8), (4099, 32, 32), (20000, 96, 96), (184756, 96, 96),
                                   (30001, 192, 192), (5000, 64, 160), (777, 256, 16)])
@pytest.mark.parametrize("engine", [1, 2])
def test_gram_engines_match_fp64(mbl, n, p, q, engine):
    """C = A^T B in FP32 on the CUDA cores and on the tensor cores (tcgen05, TF32 split)
    against numpy FP64: |C - C64| <= c * 2^-21 * (|A|^T |B|) elementwise."""
    rng = np.random.default_rng(n + p + q)
    A = rng.standard_normal((n, p))
    B = rng.standard_normal((n, q)) * np.linspace(0.5, 3.0, q)
    C = mbl.binding.gram(_gpu(A), _gpu(B), "f32", engine).cpu().numpy()
    ref = A.T @ B
    scale = np.abs(A).T @ np.abs(B)
    err = np.abs(C - ref)
    assert np.all(err <= 8 * 2.0 ** -21 * scale), (err / scale).max()
    if engine == 2:
        # the split recovers FP32 accuracy: single-pass TF32 would leave errors near 2^-11
        assert (err / scale).max() < 2.0 ** -18
    C64 = mbl.binding.gram(_gpu(A), _gpu(B), "f64", 1).cpu().numpy()
    assert np.abs(C64 - ref).max() <= 1e-12 * scale.max()


@pytest.mark.gpu
@pytest.mark.parametrize("n,p", [(1000, 8), (4099, 32), (20000, 96), (184756, 96), (30001, 192), (777, 256),
                                 (17, 5), (33, 130)])
def test_gram_of_a_block_with_itself(mbl, n, p):
    """S^T S (one operand read once, the same tensor-core tile serving both sides) on both
    engines against numpy FP64, within 8 * 2^-21 of |S|^T |S|; the result is symmetric to
    the same accuracy."""
    rng = np.random.default_rng(3 * n + p)
    S = rng.standard_normal((n, p)) * np.linspace(0.25, 4.0, p)
    ref = S.T @ S
    scale = np.abs(S).T @ np.abs(S)
    for engine in (1, 2):
        G = mbl.binding.gram(_gpu(S), _gpu(S), "f32", engine).cpu().numpy()
        assert np.all(np.abs(G - ref) <= 8 * 2.0 ** -21 * scale), (engine, (np.abs(G - ref) / scale).max())
        assert np.all(np.abs(G - G.T) <= 16 * 2.0 ** -21 * scale)


@pytest.mark.gpu
@pytest.mark.parametrize("n,p,q", [(1000, 8, 8), (4099, 32, 32), (184756, 96, 32), (184756, 64, 32),
                                   (30001, 192, 64), (777, 64, 16), (129, 17, 5), (1, 3, 1)])
@pytest.mark.parametrize("engine", [1, 2])
def test_update_engines_match_fp64(mbl, n, p, q, engine):
    """D = beta C + alpha A M (the block update of the LOBPCG step) in FP32 on the CUDA cores
    and on the tensor cores (tcgen05, TF32 split) against numpy FP64: inputs rounded to FP32,
    FP32 arithmetic, so |D - D64| <= c * 2^-21 * (|alpha| |A| |M| + |beta C|) elementwise."""
    rng = np.random.default_rng(7 * n + p + q)
    A = rng.standard_normal((n, p))
    M = rng.standard_normal((p, q)) * np.linspace(0.5, 3.0, q)
    C = rng.standard_normal((n, q))
    alpha, beta = -0.75, 1.25
    ref = beta * C + alpha * (A @ M)
    scale = abs(alpha) * (np.abs(A) @ np.abs(M))
    D = mbl.binding.update(_gpu(A), _gpu(M), _gpu(C), alpha, beta, "f32", engine).cpu().numpy()
    err = np.abs(D - ref)
    bound = scale + np.abs(beta * C)
    assert np.all(err <= 8 * 2.0 ** -21 * bound), (err / bound).max()
    if engine == 2:
        # the split recovers FP32 accuracy: single-pass TF32 would leave errors near 2^-11
        assert (err / bound).max() < 2.0 ** -18
    # beta = 0 without C
    D0 = mbl.binding.update(_gpu(A), _gpu(M), None, alpha, 0.0, "f32", engine).cpu().numpy()
    assert np.all(np.abs(D0 - alpha * (A @ M)) <= 8 * 2.0 ** -21 * scale)
    D64 = mbl.binding.update(_gpu(A), _gpu(M), _gpu(C), alpha, beta, "f64", 1).cpu().numpy()
    assert np.abs(D64 - ref).max() <= 1e-12 * (scale.max() + np.abs(beta * C).max())


@pytest.mark.gpu
@pytest.mark.parametrize("alpha,beta", [(-1.0, 1.0), (1.0, 0.0), (1.0, 1.0), (-1.0, 0.0), (2.5, 1.0), (1.0, -0.5)])
def test_update_scalars_and_special_values(mbl, alpha, beta):
    """The update for the solver's scalar pairs (alpha = +-1, beta in {0, 1}) and general
    ones, with A holding zeros, FP32-subnormal, FP64-subnormal and near-FP32-overflow
    magnitudes next to ordinary values: every element within the FP32 bound of the FP64
    result, on both engines."""
    rng = np.random.default_rng(int(100 * alpha + 10 * beta) % 1000)
    n, p, q = 128 * 40 + 3, 64, 32
    A = rng.standard_normal((n, p))
    A[::7, 3] = 0.0
    A[5::11, 9] = -0.0
    A[2::13, 17] = 1e-39 * rng.standard_normal(A[2::13, 17].shape)
    A[3::17, 21] = 1e-310
    A[1::19, 30] = 1e37
    M = rng.standard_normal((p, q))
    C = rng.standard_normal((n, q))
    ref = beta * C + alpha * (A @ M)
    scale = abs(alpha) * (np.abs(A) @ np.abs(M))
    for engine in (1, 2):
        D = mbl.binding.update(_gpu(A), _gpu(M), _gpu(C), alpha, beta, "f32", engine).cpu().numpy()
        err = np.abs(D - ref)
        bound = scale + np.abs(beta * C)
        assert np.all(np.isfinite(D))
        assert np.all(err <= 8 * 2.0 ** -21 * bound + 1e-300), (engine, (err / bound).max())


@pytest.mark.gpu
def test_tensor_core_dispatch_and_fallback(mbl):
    """Engine 2 takes the TMA-fed tensor-core kernels for aligned blocks with even leading
    dimensions (their TF32-split result differs from the CUDA cores' FP32 FMA in the low
    bits) and falls back to the CUDA cores, with the same accuracy, for a block that starts
    8 bytes past a 16-byte boundary or has an odd leading dimension."""
    rng = np.random.default_rng(21)
    n, p, q = 128 * 40 + 5, 64, 32
    A = rng.standard_normal((n, p))
    M = rng.standard_normal((p, q))
    ref_u = A @ M
    ref_g = A.T @ A
    su = np.abs(A) @ np.abs(M)
    sg = np.abs(A).T @ np.abs(A)
    d1 = mbl.binding.update(_gpu(A), _gpu(M), None, 1.0, 0.0, "f32", 1).cpu().numpy()
    d2 = mbl.binding.update(_gpu(A), _gpu(M), None, 1.0, 0.0, "f32", 2).cpu().numpy()
    g1 = mbl.binding.gram(_gpu(A), _gpu(A), "f32", 1).cpu().numpy()
    g2 = mbl.binding.gram(_gpu(A), _gpu(A), "f32", 2).cpu().numpy()
    assert not np.array_equal(d1, d2) and not np.array_equal(g1, g2)
    # an n x p view one double past the start of a padded buffer: 8-byte aligned only
    big = _gpu(np.concatenate([np.zeros(1), A.ravel()]))
    Av = big[1:].view(n, p)
    assert Av.data_ptr() % 16 == 8
    du = mbl.binding.update(Av, _gpu(M), None, 1.0, 0.0, "f32", 2).cpu().numpy()
    assert np.array_equal(du, d1)  # the CUDA-core kernel, bit for bit
    gu = mbl.binding.gram(Av, Av, "f32", 2).cpu().numpy()
    assert np.all(np.abs(gu - ref_g) <= 8 * 2.0 ** -21 * sg)
    assert np.all(np.abs(du - ref_u) <= 8 * 2.0 ** -21 * su)
    # odd leading dimension (p = 63): CUDA cores under engine 2 too
    A3 = A[:, :63].copy()
    e1 = mbl.binding.update(_gpu(A3), _gpu(M[:63]), None, 1.0, 0.0, "f32", 1).cpu().numpy()
    e2 = mbl.binding.update(_gpu(A3), _gpu(M[:63]), None, 1.0, 0.0, "f32", 2).cpu().numpy()
    assert np.array_equal(e1, e2)


@pytest.mark.gpu
def test_update_engines_agree_on_padded_tiles(mbl):
    """Ragged tails: n not a multiple of the 128-row tile, p not a multiple of the 32-wide K
    chunk or of the 16-column box, q not a multiple of 16 -- the tensor-core result equals
    the CUDA-core one to FP32 accuracy in every row, including the last partial tile (no
    stale rows or columns).  Even p and q keep the rows 16-byte aligned, the condition for
    the TMA-fed kernel; odd ones take the CUDA cores under every engine."""
    rng = np.random.default_rng(11)
    for n, p, q in [(128 * 152 + 1, 34, 18), (128 * 304 - 5, 190, 62), (127, 2, 2), (128 * 5, 16, 64),
                    (128 * 152 * 3 + 77, 96, 32), (128 * 152 + 1, 33, 17), (127, 1, 1)]:
        A = rng.standard_normal((n, p))
        M = rng.standard_normal((p, q))
        d1 = mbl.binding.update(_gpu(A), _gpu(M), None, 1.0, 0.0, "f32", 1).cpu().numpy()
        d2 = mbl.binding.update(_gpu(A), _gpu(M), None, 1.0, 0.0, "f32", 2).cpu().numpy()
        scale = np.abs(A) @ np.abs(M)
        assert np.all(np.isfinite(d2))
        assert np.all(np.abs(d1 - d2) <= 2.0 ** -18 * scale), (n, p, q)
