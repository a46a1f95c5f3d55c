"""The C ABI without a GPU: the library loads, exports every function include/mbl.h
declares, its structs have the header's layout, and the entry points that do no GPU
work (sizes, argument checks, tuning switches, status text) behave as documented."""
import ctypes
import math
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mbl.h")


@pytest.fixture(scope="module")
def so():
    from paper_2012_00217_gb300 import build as pbuild
    if pbuild.needs_build():
        if shutil.which(pbuild.NVCC) is None and not os.path.exists(pbuild.NVCC):
            pytest.skip("nvcc not available to build the library")
        pbuild.build()
    from paper_2012_00217_gb300 import binding
    binding.lib.cache_clear()
    return binding.lib()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mbl_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("mbl_basis_build", "mbl_basis_rank", "mbl_hamiltonian_apply", "mbl_lobpcg_solve",
                 "mbl_lobpcg_solve_batched", "mbl_spectrum_bounds"):
        assert need in names


def test_every_declared_function_is_exported(so):
    missing = [nm for nm in _declared() if not hasattr(so, nm)]
    assert not missing, missing


def test_binding_covers_the_header(so):
    from paper_2012_00217_gb300 import binding
    assert sorted(binding.EXPORTED) == _declared()


def test_noalloc_entry_point_and_its_limit(so):
    """The allocation-free solve is exported, and the binding's copy of its scratch size
    equals the header's MBL_NOALLOC_SCRATCH_BYTES (the refusal test relies on it)."""
    from paper_2012_00217_gb300 import binding
    assert hasattr(so, "mbl_lobpcg_solve_noalloc")
    m = re.search(r"#define\s+MBL_NOALLOC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", open(HEADER).read())
    assert m, "MBL_NOALLOC_SCRATCH_BYTES not found in the header"
    assert binding.NOALLOC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2))


def _c_layout(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "layout.c"
    fields = {
        "mbl_chain": ["L", "n_up", "periodic", "delta", "h_host"],
        "mbl_lobpcg_opts": ["nev", "k", "max_iter", "pcg_iters", "tol", "pcg_tol", "norm_h", "mode",
                            "use_graph", "timing"],
        "mbl_lobpcg_stats": ["iters", "converged", "matvecs", "seconds", "max_rel_resid", "norm_h",
                             "t_setup", "t_resid", "t_pcg", "t_wp", "t_gram", "t_small", "t_update",
                             "t_refresh", "t_hrr"],
        "mbl_product_choice": ["schedule", "lane_bytes", "tile_bits", "microseconds"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mbl.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (st, st))
        for f in fs:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (st, f, st, f))
    lines += ["return 0; }"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        st, f, v = line.split()
        got[(st, f)] = int(v)
    return got


def test_struct_layouts_match_the_header(tmp_path):
    from paper_2012_00217_gb300 import binding
    c = _c_layout(tmp_path)
    for st, cls in (("mbl_chain", binding.Chain), ("mbl_lobpcg_opts", binding.LobpcgOpts),
                    ("mbl_lobpcg_stats", binding.LobpcgStats), ("mbl_product_choice", binding.ProductChoice)):
        assert c[(st, "sizeof")] == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert c[(st, f)] == getattr(cls, f).offset, (st, f)


def test_basis_size_is_the_binomial(so):
    for L in range(1, 33):
        for m in range(0, L + 1):
            assert so.mbl_basis_size(L, m) == math.comb(L, m)
    for L, m in ((0, 0), (33, 16), (10, 11), (10, -1), (-4, 2)):
        assert so.mbl_basis_size(L, m) < 0


def test_status_strings(so):
    from paper_2012_00217_gb300 import binding
    seen = set()
    for code in (binding.MBL_OK, binding.MBL_ERR_ARG, binding.MBL_ERR_WORKSPACE, binding.MBL_ERR_CUDA,
                 binding.MBL_ERR_NOT_CONVERGED, binding.MBL_ERR_BREAKDOWN, binding.MBL_ERR_NUMERIC):
        s = binding.status_string(code)
        assert s and s not in seen
        seen.add(s)
    assert binding.status_string(12345)


def test_launch_counter_is_host_state(so):
    a = so.mbl_kernel_launch_count()
    assert a >= 0
    assert so.mbl_kernel_launch_count() == a  # nothing launched in between


def _ws(so, chain, opts):
    from paper_2012_00217_gb300 import binding
    sz = ctypes.c_size_t(0)
    rc = so.mbl_lobpcg_workspace_size(ctypes.byref(chain), ctypes.byref(opts), ctypes.byref(sz))
    return rc, sz.value


def test_workspace_size_grows_with_block_and_checks_options(so):
    import paper_2012_00217_gb300 as mbl
    from paper_2012_00217_gb300 import binding
    ch = mbl.make_chain(16, np.linspace(-1, 1, 16))
    prev = 0
    for k in (8, 16, 32, 64):
        rc, b = _ws(so, ch, mbl.make_opts(4, k))
        assert rc == binding.MBL_OK and b > prev
        prev = b
    # mixed mode keeps the PCG vectors in FP32: a smaller workspace than FP64
    _, b64 = _ws(so, ch, mbl.make_opts(8, 16, mode=mbl.MODE_FP64))
    _, bmx = _ws(so, ch, mbl.make_opts(8, 16, mode=mbl.MODE_MIXED))
    assert 0 < bmx < b64
    for bad in (mbl.make_opts(0, 8), mbl.make_opts(9, 8), mbl.make_opts(4, 65), mbl.make_opts(4, 8, mode=7),
                mbl.make_opts(4, 8, tol=0.0), mbl.make_opts(4, 8, pcg_iters=-1)):
        assert _ws(so, ch, bad)[0] == binding.MBL_ERR_ARG
    # 3k > n: the block does not fit the sector
    small = mbl.make_chain(6, np.zeros(6))  # n = 20
    assert _ws(so, small, mbl.make_opts(4, 8))[0] == binding.MBL_ERR_ARG
    # bad chains
    keep = []
    for L, n_up in ((40, 20), (12, 13), (1, 0)):
        h = np.zeros(max(L, 1))
        keep.append(h)
        c = binding.Chain(L, n_up, 0, 1.0, h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert _ws(so, c, mbl.make_opts(1, 1))[0] == binding.MBL_ERR_ARG
    # odd L and other sectors are allowed
    assert _ws(so, mbl.make_chain(13, np.zeros(13), n_up=4), mbl.make_opts(2, 4))[0] == binding.MBL_OK


def test_batched_workspace_is_slots_times_largest(so):
    import paper_2012_00217_gb300 as mbl
    from paper_2012_00217_gb300 import binding
    chains = [mbl.make_chain(L, np.zeros(L)) for L in (12, 14, 16)]
    opts = mbl.make_opts(8, 16)
    one = _ws(so, chains[-1], opts)[1]
    b1 = binding.batched_workspace_size(chains, opts, 1)
    b3 = binding.batched_workspace_size(chains, opts, 3)
    assert b1 >= one and b3 >= 3 * one
    assert b3 < 3 * one + 3 * 4096  # slot alignment and the table of lanes only


def test_tuning_switches_validate(so):
    from paper_2012_00217_gb300 import binding
    ok, bad = binding.MBL_OK, binding.MBL_ERR_ARG
    for k, dt, bits, want in ((32, 0, 5, ok), (32, 1, -1, ok), (32, 0, 0, ok), (1, 0, 16, ok),
                              (32, 0, 1, bad), (32, 0, 17, bad), (0, 0, 4, bad), (257, 0, 4, bad),
                              (32, 2, 4, bad)):
        assert so.mbl_set_product_tile_bits(k, dt, bits) == want
    for k, dt, nb, want in ((32, 0, 16, ok), (32, 1, 32, ok), (8, 0, 0, ok), (32, 0, 64, ok), (32, 0, 8, bad),
                            (32, 0, 128, bad), (0, 0, 16, bad)):
        assert so.mbl_set_product_lane_bytes(k, dt, nb) == want
    # restore the defaults
    for k in (1, 32):
        for dt in (0, 1):
            so.mbl_set_product_tile_bits(k, dt, 0)
    for k in (8, 32):
        for dt in (0, 1):
            so.mbl_set_product_lane_bytes(k, dt, 0)
    for sch, want in ((0, ok), (1, ok), (2, ok), (3, ok), (4, ok), (5, ok), (6, bad), (-1, bad)):
        assert so.mbl_set_product_schedule(64, 0, sch) == want
    so.mbl_set_product_schedule(64, 0, 0)
    for eng, want in ((0, ok), (1, ok), (2, ok), (3, bad), (-1, bad)):
        assert so.mbl_set_gram_engine(eng) == want
    so.mbl_set_gram_engine(0)


def test_tile_width_query_host_schedules(so):
    """mbl_product_tile_width for the host-decided orders: the tile-bits switch for 1 and 2,
    the widest B <= min(13, L - 2) whose largest tile C(B, B/2) rows fits 48 KB for 3 and
    32 KB for 5,
    0 where no tiled kernel exists, MBL_ERR_ARG for bad arguments (no device needed)."""
    from math import comb
    from paper_2012_00217_gb300 import binding
    bad = binding.MBL_ERR_ARG
    for L, dt, k in ((20, 0, 32), (16, 1, 16), (26, 0, 64), (9, 0, 4)):
        es = 4 if dt == 0 else 8
        B = min(13, L - 2)
        while B >= 2 and comb(B, B // 2) * k * es > 48 * 1024:
            B -= 1
        assert so.mbl_product_tile_width(L, dt, k, 3) == B
        # slab order: the widest B whose largest tile fits one 32 KB ring slot (rows of 32..256 bytes)
        Bs = min(13, L - 2)
        while Bs >= 2 and comb(Bs, Bs // 2) * k * es > 32 * 1024:
            Bs -= 1
        want = Bs if 32 <= k * es <= 256 else 0
        assert so.mbl_product_tile_width(L, dt, k, 5) == want
        for bits in (5, 9):
            assert so.mbl_set_product_tile_bits(k, dt, bits) == binding.MBL_OK
            try:
                assert so.mbl_product_tile_width(L, dt, k, 1) == min(bits, L - 2)
                assert so.mbl_product_tile_width(L, dt, k, 2) == min(bits, L - 2)
            finally:
                so.mbl_set_product_tile_bits(k, dt, 0)
        assert so.mbl_product_tile_width(L, dt, k, 1) >= 2
    assert so.mbl_product_tile_width(20, 0, 3, 1) == 0  # no tiled kernel for k = 3
    assert so.mbl_product_tile_width(20, 0, 2, 3) == 0  # 8-byte rows: no bulk copies
    so.mbl_set_product_tile_bits(32, 0, -1)
    try:
        assert so.mbl_product_tile_width(20, 0, 32, 3) == 0  # untiled kernel forced
    finally:
        so.mbl_set_product_tile_bits(32, 0, 0)
    for L, dt, k, sch in ((3, 0, 8, 1), (33, 0, 8, 1), (20, 2, 8, 1), (20, 0, 0, 1), (20, 0, 257, 1),
                          (20, 0, 8, 0), (20, 0, 8, 6)):
        assert so.mbl_product_tile_width(L, dt, k, sch) == bad


def test_autotune_checks_arguments_before_any_launch(so):
    import paper_2012_00217_gb300 as mbl
    from paper_2012_00217_gb300 import binding
    ch = mbl.make_chain(12, np.zeros(12))
    n = math.comb(12, 6)
    c = binding.ProductChoice()
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every case below fails its checks first
    for dtype, X, Y, nn, k, reps in ((2, fake, fake, n, 8, 3), (0, None, fake, n, 8, 3), (0, fake, fake, n - 1, 8, 3),
                                     (0, fake, fake, n, 0, 3), (0, fake, fake, n, 8, 0), (0, fake, fake, n, 8, 3)):
        rc = so.mbl_autotune_product(ctypes.byref(ch), dtype, X, Y, nn, k, reps, ctypes.byref(c), None)
        assert rc == binding.MBL_ERR_ARG  # the last case: X and Y overlap


def test_non_finite_chain_or_shift_is_refused_on_the_host(so):
    """Host-side fault injection: NaN or Inf in a field, in delta or in sigma is an
    argument error, found before any device work (the pointers below are never used)."""
    import paper_2012_00217_gb300 as mbl
    from paper_2012_00217_gb300 import binding
    bad = binding.MBL_ERR_ARG
    n = math.comb(12, 6)
    fake = ctypes.c_void_p(1 << 20)
    for field, delta, sigma in ((np.nan, 1.0, 0.0), (np.inf, 1.0, 0.0), (0.5, np.nan, 0.0), (0.5, 1.0, np.inf)):
        h = np.zeros(12)
        h[3] = field
        ch = mbl.make_chain(12, h, delta)
        assert so.mbl_hamiltonian_apply(ctypes.byref(ch), ctypes.c_double(sigma), 1, fake, 8, fake, 8, n, 8,
                                        None) == bad
        opts = mbl.make_opts(4, 8)
        ev, res = np.zeros(4), np.zeros(4)
        st = binding.LobpcgStats()
        assert so.mbl_lobpcg_solve(ctypes.byref(ch), ctypes.c_double(sigma), ctypes.byref(opts), fake, fake,
                                   ctypes.c_size_t(1 << 40), ev.ctypes.data_as(ctypes.c_void_p), None,
                                   res.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st), None) == bad


def test_gap_ratio_checks_arguments_before_any_launch(so):
    from paper_2012_00217_gb300 import binding
    ok, bad = binding.MBL_OK, binding.MBL_ERR_ARG
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every case fails its checks or launches nothing
    for nprob, m, ld, ptrs, want in ((-1, 8, 8, (fake, fake, fake), bad), (4, 0, 8, (fake, fake, fake), bad),
                                     (4, 4097, 4097, (fake, fake, fake), bad), (4, 8, 7, (fake, fake, fake), bad),
                                     (4, 8, 8, (None, fake, fake), bad), (4, 8, 8, (fake, None, fake), bad),
                                     (4, 8, 8, (fake, fake, None), bad), (0, 8, 8, (None, None, None), ok)):
        assert so.mbl_gap_ratio(nprob, m, ptrs[0], ld, ptrs[1], ptrs[2], None) == want


def test_update_checks_arguments_before_any_launch(so):
    """mbl_update refuses bad shapes, leading dimensions, precision/engine pairs and a
    missing C with beta != 0 on the host; n = 0 launches nothing."""
    from paper_2012_00217_gb300 import binding
    ok, bad = binding.MBL_OK, binding.MBL_ERR_ARG
    f = ctypes.c_void_p(1 << 20)  # never dereferenced: every case fails its checks or launches nothing
    F32, F64 = binding.MBL_F32, binding.MBL_F64
    cases = (  # A, lda, p, M, ldm, q, C, ldc, D, ldd, n, alpha, beta, precision, engine, want
        (f, 8, 8, f, 8, 8, f, 8, f, 8, 0, 1.0, 1.0, F32, 2, ok),
        (f, 8, 8, f, 8, 8, f, 8, f, 8, 0, 1.0, 1.0, F64, 2, bad),
        (f, 193, 193, f, 8, 8, f, 8, f, 8, 10, 1.0, 0.0, F32, 2, bad),
        (f, 8, 8, f, 65, 65, f, 65, f, 65, 10, 1.0, 0.0, F32, 2, bad),
        (f, 7, 8, f, 8, 8, f, 8, f, 8, 10, 1.0, 0.0, F32, 1, bad),
        (f, 8, 8, f, 8, 8, None, 8, f, 8, 10, 1.0, 0.5, F32, 1, bad),
        (f, 8, 8, f, 8, 8, f, 8, f, 8, 10, float("nan"), 0.0, F32, 1, bad),
        (f, 8, 8, f, 8, 8, f, 8, f, 8, 10, 1.0, 0.0, 3, 1, bad),
        (f, 8, 8, f, 8, 8, f, 8, f, 8, 10, 1.0, 0.0, F32, 3, bad),
        (None, 8, 8, f, 8, 8, f, 8, f, 8, 10, 1.0, 0.0, F32, 1, bad),
        (f, 8, 8, f, 8, 8, f, 8, f, 8, -1, 1.0, 0.0, F32, 1, bad),
    )
    for *args, want in cases:
        assert so.mbl_update(*args, None) == want, args


def test_entanglement_workspace_and_argument_checks(so):
    import paper_2012_00217_gb300 as mbl
    from paper_2012_00217_gb300 import binding
    bad = binding.MBL_ERR_ARG
    ch = mbl.make_chain(20, np.zeros(20))
    prev = 0
    for nvec in (1, 4, 16):
        b = binding.entanglement_workspace_size(ch, 10, nvec)
        assert b > prev
        prev = b
    # the half cut at L = 20: 11 blocks of (252 x 252 gather, 252 x 253 Gram) per column
    assert 11 * 16 * 8 * 2 * 252 * 252 < binding.entanglement_workspace_size(ch, 10, 16) < 2 ** 28
    sz = ctypes.c_size_t(0)
    for L, n_up, l_a, nvec in ((20, 10, 0, 1), (20, 10, 20, 1), (20, 10, 5, -1), (24, 12, 12, 1), (33, 16, 8, 1)):
        h = np.zeros(max(L, 1))
        c = binding.Chain(L, n_up, 0, 1.0, h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert so.mbl_entanglement_workspace_size(ctypes.byref(c), l_a, nvec, ctypes.byref(sz)) == bad
    # a cut whose Gram sides stay small is fine at L = 24 (one site on the left)
    c24 = mbl.make_chain(24, np.zeros(24))
    assert binding.entanglement_workspace_size(c24, 1, 2) > 0
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every case below fails its checks or launches nothing
    assert so.mbl_entanglement_entropy(ctypes.byref(ch), 10, 4, fake, 3, fake, fake, 1 << 30, None) == bad
    assert so.mbl_entanglement_entropy(ctypes.byref(ch), 10, 4, None, 4, fake, fake, 1 << 30, None) == bad
    assert so.mbl_entanglement_entropy(ctypes.byref(ch), 10, 4, fake, 4, fake, fake, 16,
                                       None) == binding.MBL_ERR_WORKSPACE
    assert so.mbl_entanglement_entropy(ctypes.byref(ch), 10, 0, None, 0, None, None, 0, None) == binding.MBL_OK


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2012_00217_gb300 import binding
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "absent.so"))
    binding.lib.cache_clear()
    try:
        with pytest.raises(RuntimeError, match="not built"):
            binding.lib()
    finally:
        monkeypatch.undo()
        binding.lib.cache_clear()
