"""Library selection builders (host C++) against the oracle's independent
Python builders: identical types, pair lists and windows (bit-exact)."""
import numpy as np
import pytest

from oracle import select as osel


@pytest.fixture(scope="module")
def gcmod():
    from paper_2005_03060_gb300 import _build
    _build.build()
    from paper_2005_03060_gb300 import gridcorr
    return gridcorr


def _same(a, b):
    assert [tuple(t) for t in a.types.tolist()] == [tuple(t) for t in b.types]
    assert np.array_equal(a.type_ptr, b.type_ptr)
    assert np.array_equal(a.pair_i, b.pair_i)
    assert np.array_equal(a.pair_j, b.pair_j)
    assert np.array_equal(a.win_t0, b.win_t0)
    assert np.array_equal(a.win_t1, b.win_t1)
    assert a.P == b.P and a.n_cycle == b.n_cycle and a.t_int == b.t_int


@pytest.mark.parametrize("L,T,p", [(3, 10, 1.0), (4, 64, 1.0), (5, 100, 0.5), (6, 33, 0.05),
                                   (8, 256, 1.0), (12, 2048, 1.0), (16, 100, 2.0), (32, 4096, 1.0),
                                   (4, 64, 0.5859375)])   # budget 37.5: a tie between 33 and 42 pairs
def test_subset_matches_oracle(gcmod, L, T, p):
    _same(gcmod.Selection("subset", L, T, p), osel.subset(L, T, p))


def test_subset_paper_sizes(gcmod):
    """Pair counts of the configured arrays (p = 1, log base 2)."""
    for L, P, k in [(8, 390, 8), (32, 10446, 11), (64, 47250, 12), (128, 224786, 14)]:
        s = gcmod.Selection("subset", L, 1024)
        assert (s.P, s.n_ubl, s.null_dim) == (P, k, 4)
    _same(gcmod.Selection("subset", 64, 8192), osel.subset(64, 8192))


@pytest.mark.parametrize("L,T", [(3, 50), (4, 100), (8, 256), (12, 2048), (32, 4096)])
def test_lowcad_matches_oracle(gcmod, L, T):
    _same(gcmod.Selection("lowcad", L, T), osel.lowcad(L, T))


def test_natural_log_budget(gcmod):
    _same(gcmod.Selection("subset", 16, 100, 1.0, 0.0), osel.subset(16, 100, 1.0, 0.0))


def test_selection_errors(gcmod):
    with pytest.raises(gcmod.GridcorrError) as e:
        gcmod.Selection("subset", 2, 10)
    assert e.value.status == gcmod.GC_EDEGEN
    with pytest.raises(gcmod.GridcorrError):
        gcmod.Selection("subset", 1, 10)
    with pytest.raises(gcmod.GridcorrError):
        gcmod.Selection("lowcad", 8, 0)


def test_lowcad_beyond_the_pair_cap_is_refused(gcmod):
    """A low-cadence selection takes every pair, N (N - 1) / 2; past 2^28 pairs
    (about 23 000 antennas) the builder refuses with GC_EUNSUPPORTED before
    allocating them, instead of running out of host memory."""
    import time
    t0 = time.perf_counter()
    with pytest.raises(gcmod.GridcorrError) as e:
        gcmod.Selection("lowcad", 256, 1 << 20)
    assert e.value.status == gcmod.GC_EUNSUPPORTED
    assert time.perf_counter() - t0 < 60.0
    sel = gcmod.Selection("lowcad", 24, 4096)        # well inside the cap: every pair
    assert sel.P == 576 * 575 // 2


@pytest.mark.parametrize("s", [3, 4, 6, 8, 11])
def test_hex_subset_matches_oracle(gcmod, s):
    """Masked-lattice subset selection of a hexagonal array equals the oracle's
    (types, order, pairs), and both hexagon layouts agree."""
    from paper_2005_03060_gb300 import synth
    L, m = osel.hex_mask(s)
    L2, m2 = synth.hex_mask(s)
    assert L2 == L and np.array_equal(m, m2)
    ref = osel.subset_layout(L, m, "triangular", 512)
    sel = gcmod.Selection("subset", L, 512, mask=m, lattice="triangular")
    assert sel.masked == 1 and sel.lattice == "triangular" and sel.n_ant == int(m.sum())
    assert [tuple(t) for t in sel.types.tolist()] == ref.types
    assert np.array_equal(sel.type_ptr, ref.type_ptr)
    assert np.array_equal(sel.pair_i, ref.pair_i) and np.array_equal(sel.pair_j, ref.pair_j)
    assert sel.null_dim == 4


def test_full_mask_equals_unmasked(gcmod):
    L = 8
    a = gcmod.Selection("subset", L, 256)
    b = gcmod.Selection("subset", L, 256, mask=np.ones(L * L, np.uint8))
    assert np.array_equal(a.types, b.types) and np.array_equal(a.pair_i, b.pair_i)
    assert np.array_equal(a.pair_j, b.pair_j)


def test_masked_selection_errors(gcmod):
    L = 6
    m = np.zeros(L * L, np.uint8)
    m[:2] = 1                                  # two antennas
    with pytest.raises(gcmod.GridcorrError):
        gcmod.Selection("subset", L, 64, mask=m)
    m = np.zeros(L * L, np.uint8)
    m[0::2] = 1                                # columns 0, 2, 4: the (1,0) type has no pair
    with pytest.raises(gcmod.GridcorrError) as e:
        gcmod.Selection("subset", L, 64, mask=m)
    assert e.value.status == gcmod.GC_EDEGEN


@pytest.mark.parametrize("s,T", [(4, 256), (8, 1024), (11, 4096)])
def test_hex_lowcad_matches_oracle(gcmod, s, T):
    L, m = osel.hex_mask(s)
    ref = osel.lowcad_layout(L, m, "triangular", T)
    sel = gcmod.Selection("lowcad", L, T, mask=m, lattice="triangular")
    assert [tuple(t) for t in sel.types.tolist()] == ref.types
    assert np.array_equal(sel.type_ptr, ref.type_ptr)
    assert np.array_equal(sel.pair_i, ref.pair_i) and np.array_equal(sel.pair_j, ref.pair_j)
    assert np.array_equal(sel.win_t0, ref.win_t0) and np.array_equal(sel.win_t1, ref.win_t1)
    assert sel.n_cycle == ref.n_cycle and sel.t_int == ref.t_int
    n = int(m.sum())
    assert sel.P == n * (n - 1) // 2            # every pair exactly once


@pytest.mark.parametrize("L,s", [(3, None), (8, None), (5, 3), (9, 5)])
def test_edge_mask_matches_oracle(gcmod, L, s):
    """gc_sel_edge (host) against the oracle's edge antennas (Sec. 5.4):
    square grids, and hexagonal arrays of side s on the triangular lattice."""
    from oracle import visvar as ov
    if s is None:
        sel, m, lat = gcmod.Selection("subset", L, 64), None, "square"
    else:
        L2, m = osel.hex_mask(s)
        assert L2 == L
        sel, lat = gcmod.Selection("subset", L, 64, mask=m, lattice="triangular"), "triangular"
    assert np.array_equal(sel.edge_mask().astype(bool), ov.edge_antennas(L, m, lat))
