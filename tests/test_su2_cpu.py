"""CPU tests of the library's SU(2) host logic against the oracle: the
Clebsch-Gordan coefficients it uses and its canonical block layouts (sector
tuples, fusion-tree labels, offsets) must match bit-exactly in structure and
to rounding in value.  Host-only context, no device work."""
import itertools

import numpy as np
import pytest

bst = pytest.importorskip("paper_1808_10804_gb300.bst")

from oracle import su2  # noqa: E402
from workloads import su2_config  # noqa: E402


@pytest.fixture(scope="module")
def hctx():
    try:
        bst.lib()
    except RuntimeError as e:
        pytest.skip(str(e))
    c = bst.Context(device=-1)
    yield c
    c.close()


def test_cg_matches_oracle(hctx):
    worst = 0.0
    for tj1, tj2 in itertools.product(range(0, 11), range(0, 11)):
        for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2):
            for tm1 in range(-tj1, tj1 + 1, 2):
                for tm2 in range(-tj2, tj2 + 1, 2):
                    tM = tm1 + tm2
                    if abs(tM) > tJ:
                        continue
                    worst = max(worst, abs(bst.su2_cg(tj1, tm1, tj2, tm2, tJ, tM) - su2.cg(tj1, tm1, tj2, tm2, tJ, tM)))
    assert worst < 2e-15, worst
    # forbidden arguments give exactly zero
    assert bst.su2_cg(1, 1, 1, 1, 0, 0) == 0.0
    assert bst.su2_cg(2, 0, 2, 0, 2, 0) == 0.0 or abs(bst.su2_cg(2, 0, 2, 0, 2, 0)) < 1e-16


def bst_legs(legs):
    return [bst.Leg(l.flow, tuple(l.spins), tuple(l.degs)) for l in legs]


def layout_matches(hctx, legs):
    L = hctx.layout(bst_legs(legs), group="su2")
    want = su2.blocks(legs)
    got_blocks = L.blocks()
    got_trees = L.trees()
    assert len(got_blocks) == len(want)
    off = 0
    for (idx, tree), (s, o, sh), t in zip(want, got_blocks, got_trees):
        assert tuple(s) == tuple(idx)
        assert tuple(t) == tuple(tree)
        assert o == off
        assert tuple(sh) == su2.block_shape(legs, idx)
        off += int(np.prod(sh))
    assert L.nnz == su2.nnz(legs) == off
    return L


FLOWS = [(1,), (-1,), (1, -1), (1, 1, -1), (1, -1, -1), (-1, -1, -1), (1, 1, -1, -1), (-1, -1, -1, -1),
         (1, 1, 1, -1), (1, -1, 1, -1), (1, 1, 1, 1, -1), (-1, 1, -1, 1, -1, 1)]


@pytest.mark.parametrize("flows", FLOWS)
@pytest.mark.parametrize("seed", range(3))
def test_layout_matches_oracle(hctx, flows, seed):
    rng = np.random.default_rng(1000 * seed + len(flows))
    legs = []
    for f in flows:
        ns = int(rng.integers(1, 4))
        sp = tuple(sorted(rng.choice(np.arange(0, 7), size=ns, replace=False).tolist()))
        legs.append(su2.Leg(f, sp, tuple(int(x) for x in rng.integers(1, 4, size=ns))))
    layout_matches(hctx, legs)


def test_cfg3_layouts_and_contract_layout(hctx):
    cfg = su2_config("D10chi150")
    k = su2.Leg(1, *cfg["k"])
    x = su2.Leg(1, *cfg["x"])
    X2 = [k.dual(), x.dual(), k.dual(), x.dual()]
    a = [k, k, k.dual(), k.dual()]
    LX = layout_matches(hctx, X2)
    La = layout_matches(hctx, a)
    LC = hctx.contract_layout(LX, La, (0, 2), (1, 0))
    want = [x.dual(), x.dual(), k.dual(), k.dual()]
    assert [(l.flow, tuple(l.charges), tuple(l.degs)) for l in LC.legs] == \
        [(l.flow, l.spins, l.degs) for l in want]
    layout_matches(hctx, want)


def test_su2_rejects_u1_only_ops(hctx):
    L = hctx.layout([bst.Leg(1, (0, 1), (1, 1)), bst.Leg(-1, (0, 1), (1, 1))], group="su2")
    U = hctx.layout([bst.Leg(1, (-1, 1), (1, 1)), bst.Leg(-1, (-1, 1), (1, 1))])
    with pytest.raises(bst.BstError) as e:
        hctx.contract_layout(L, U, (1,), (0,))
    assert e.value.code == 1
    with pytest.raises(bst.BstError):
        hctx.layout([bst.Leg(1, (-1, 1), (1, 1))], group="su2")   # negative spin
