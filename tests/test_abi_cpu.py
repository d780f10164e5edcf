"""CPU tests of the C ABI: the library loads, exports every declared entry
point, and its host-side layout and planning logic matches the oracle
bit-exactly (host-only context, no device work)."""
import numpy as np
import pytest

bst = pytest.importorskip("paper_1808_10804_gb300.bst")

from oracle import u1  # noqa: E402
from workloads import u1_config  # noqa: E402
from bst_helpers import to_oracle_leg  # noqa: E402


@pytest.fixture(scope="module")
def hctx():
    try:
        bst.lib()
    except RuntimeError as e:
        pytest.skip(str(e))
    c = bst.Context(device=-1)
    yield c
    c.close()


def test_every_declared_symbol_is_exported(hctx):
    L = bst.lib()
    names = bst.exported_names()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []


@pytest.mark.parametrize("name", ["tiny", "d4chi16", "d6chi72", "d8chi256"])
def test_site_layout_matches_oracle(hctx, name):
    cfg = u1_config(name)
    for key in ("A", "R"):
        L = hctx.layout(cfg[key])
        olegs = [u1.leg_from_spec(s) for s in cfg[key]]
        assert [to_oracle_leg(l) for l in L.legs] == olegs
        assert L.nnz == u1.nnz(olegs)
        blocks = L.blocks()
        assert [b[0] for b in blocks] == u1.blocks(olegs)
        offs = np.cumsum([0] + [int(np.prod(b[2])) for b in blocks])[:-1]
        assert [b[1] for b in blocks] == list(offs)


def test_contract_layout_and_symmetry_errors(hctx):
    a = hctx.layout([bst.Leg(1, (-1, 1), (1, 2)), bst.Leg(-1, (-2, 0, 2), (1, 2, 1)), bst.Leg(1, (-1, 1), (2, 1))])
    b = hctx.layout([bst.Leg(1, (-2, 0, 2), (1, 2, 1)), bst.Leg(-1, (-1, 1), (1, 1)), bst.Leg(-1, (0, 2), (2, 1))])
    c = hctx.contract_layout(a, b, [1], [0])
    assert [to_oracle_leg(l) for l in c.legs] == [to_oracle_leg(x) for x in (a.legs[0], a.legs[2], b.legs[1], b.legs[2])]
    with pytest.raises(bst.BstError) as e:
        hctx.contract_layout(a, b, [0], [1])          # same flow on both sides
    assert e.value.code == 2
    with pytest.raises(bst.BstError) as e:
        hctx.contract_layout(a, a, [1], [1])
    assert e.value.code == 2
    with pytest.raises(bst.BstError) as e:
        hctx.contract_layout(a, b, [7], [0])
    assert e.value.code == 1


def test_layout_interning_and_bad_legs(hctx):
    l1 = hctx.layout([bst.Leg(1, (-1, 1), (2, 2)), bst.Leg(-1, (-1, 1), (2, 2))])
    l2 = hctx.layout([bst.Leg(1, (-1, 1), (2, 2)), bst.Leg(-1, (-1, 1), (2, 2))])
    assert l1 == l2
    with pytest.raises(bst.BstError):
        hctx.layout([bst.Leg(1, (1, -1), (2, 2))])     # unsorted charges
    with pytest.raises(bst.BstError):
        hctx.layout([bst.Leg(1, (-1, 1), (0, 2))])     # zero degeneracy
    with pytest.raises(bst.BstError):
        hctx.layout([bst.Leg(2, (-1, 1), (1, 2))])     # bad flow


def test_batched_call_checks_and_tuning_switch(hctx):
    """Argument checks of the batched contraction and the autotuner switch
    run on the host: a host-only context rejects device work with BST_E_ARG
    before touching any pointer; the tuning log starts empty."""
    import ctypes as C
    L = hctx.layout([bst.Leg(1, (-1, 1), (2, 2)), bst.Leg(-1, (-1, 1), (2, 2))])
    arr = C.c_void_p * 1
    legs = (C.c_int32 * 1)(1)
    legs0 = (C.c_int32 * 1)(0)
    st = bst.lib().bst_contract_batched(hctx.h, 0, arr(L.h), arr(None), arr(L.h), arr(None), 1, legs, legs0,
                                        0, 1.0, 0.0, arr(L.h), arr(None), None)
    assert st == 1   # nbatch < 1
    st = bst.lib().bst_contract_batched(hctx.h, 1, arr(L.h), arr(None), arr(L.h), arr(None), 1, legs, legs0,
                                        0, 1.0, 0.0, arr(L.h), arr(None), None)
    assert st == 1   # host-only context
    hctx.set_autotune(False)
    hctx.set_autotune(True)
    assert hctx.tuning_log() == ""


@pytest.mark.parametrize("seed", range(4))
def test_contract_flops_counts_matched_block_pairs(hctx, seed):
    """bst_contract_flops plans on the host (no device) and reports 2 M K N
    over the matched block pairs, enumerated independently from the
    oracle's block lists."""
    from bst_helpers import matched_pair_flops
    rng = np.random.default_rng(900 + seed)

    def leg(flow):
        qs = sorted(rng.choice(np.arange(-3, 4), size=int(rng.integers(1, 4)), replace=False))
        return u1.Leg(flow, tuple(int(q) for q in qs), tuple(int(d) for d in rng.integers(1, 6, size=len(qs))))
    s0, s1 = leg(1), leg(-1)
    a_legs = [leg(1), s0, leg(-1), s1]
    b_legs = [s1.dual(), leg(1), s0.dual()]
    A = hctx.layout([bst.Leg(l.flow, l.charges, l.degs) for l in a_legs])
    B = hctx.layout([bst.Leg(l.flow, l.charges, l.degs) for l in b_legs])
    f = hctx.contract_flops(A, B, [1, 3], [2, 0])
    assert f == matched_pair_flops(a_legs, [1, 3], b_legs, [2, 0])
