"""Pins of the oracle's unit-cell CTM move (an Lx x Ly cell, each site with
its own environment; Sec. 3.1 unit cells, Sec. 4.1's 2 x 2 cell): a 1 x 1
cell is the one-site move; a cell of identical copies moves every site as
the one-site move does; without truncation, every renewed site's 3 x 3
network equals the 3 x 4 network of its row before the move (the
projectors of the cuts above and below the row pair up as identities), for
distinct random sites and environments; the rotation of a cell by four
quarter turns is the identity."""
import numpy as np
import pytest

from oracle import ctm, u1
from workloads import u1_config, values


def tiny_cell(Lx, Ly, seed=0, same=False):
    cfg = u1_config("tiny")
    base = ctm.u1_network(cfg)
    rng = np.random.default_rng(seed)
    site = {}
    for x in range(Lx):
        for y in range(Ly):
            net = {}
            for r, (lg, arr) in base.items():
                if same:
                    net[r] = (lg, arr.copy())
                else:
                    net[r] = (lg, u1.to_dense(lg, rng.standard_normal(u1.nnz(lg))))
            site[(x, y)] = net
    return {"Lx": Lx, "Ly": Ly, "site": site}


def test_one_site_cell_is_the_one_site_move():
    cell = tiny_cell(1, 1, same=True)
    net = cell["site"][(0, 0)]
    for d in "LURD":
        got = ctm.cell_move(cell, d, 6)["site"][(0, 0)]
        want = ctm.move(net, d, 6)
        for r in ctm.ROLES:
            assert got[r][0] == want[r][0]
            assert np.array_equal(got[r][1], want[r][1]), (d, r)


def test_cell_of_copies_moves_like_one_site():
    """Identical sites and environments: the LEFT cell move absorbs column 0
    into column 1 (one one-site move) and then column 1 into column 0 (a
    second one); every row alike."""
    cell = tiny_cell(2, 2, same=True)
    net = cell["site"][(0, 0)]
    got = ctm.cell_move(cell, "L", 6)
    once = ctm.move(net, "L", 6)
    twice = ctm.move(once, "L", 6)
    for (x, y), s in got["site"].items():
        want = once if x == 1 else twice
        for r in ctm.ROLES:
            assert s[r][0] == want[r][0]
            assert np.allclose(s[r][1], want[r][1], rtol=0, atol=1e-12), ((x, y), r)


def dense_cell(Lx, Ly, seed, D=2, X=3, Xs=None):
    """No symmetry, distinct positive random tensors per site; the
    environment bonds of the cut above row y have dimension Xs[y] (every
    cut a different dimension), the horizontal ones X.  The half systems of
    the cut between rows y and y+1 are then square (Xs[y+1] D) and full
    rank."""
    rng = np.random.default_rng(seed)
    Xs = Xs or [X] * Ly
    z = lambda f, d: u1.Leg(f, (0,), (d,))
    a_legs = [z(1, D), z(1, D), z(-1, D), z(-1, D)]
    site = {}
    for x in range(Lx):
        for y in range(Ly):
            up, dn = Xs[y], Xs[(y + 1) % Ly]
            legs = {"C1": [z(-1, X), z(-1, up)], "C2": [z(1, X), z(-1, up)], "C3": [z(1, dn), z(1, X)],
                    "C4": [z(1, dn), z(-1, X)], "T1": [z(1, X), a_legs[1].dual(), z(-1, X)],
                    "T2": [z(1, up), a_legs[2].dual(), z(-1, dn)], "T3": [z(1, X), a_legs[3].dual(), z(-1, X)],
                    "T4": [z(1, up), a_legs[0].dual(), z(-1, dn)]}
            net = {r: (lg, rng.random([l.dim for l in lg])) for r, lg in legs.items()}
            net["a"] = (a_legs, rng.random((D,) * 4))
            site[(x, y)] = net
    return {"Lx": Lx, "Ly": Ly, "site": site}


def test_untruncated_cell_move_keeps_row_values():
    """Square full-rank half systems and every singular value kept: the
    projectors of each cut satisfy P P~ = 1, so the renewed 3 x 3 network of
    site (1, y) times the three norms equals the 3 x 4 row network of
    columns 0, 1 before the move; it fails if a row takes the projectors of
    the wrong cut (above and below differ for distinct sites)."""
    for Lx, Ly, Xs in ((2, 2, [2, 3]), (2, 3, [3, 2, 4]), (3, 2, [3, 3])):
        cell = dense_cell(Lx, Ly, seed=Lx * 10 + Ly, Xs=Xs)
        full = 10 ** 6
        before = {(x, y): ctm.row_value(cell, x, y) for x in range(Lx) for y in range(Ly)}
        out, infos = ctm.cell_left_move(cell, full, rel_cutoff=0.0, return_info=True)
        # column 0 renewed column 1's left environment from the original
        # cell (later columns see renewed tensors)
        for rec in infos:
            if rec["x"] != 0:
                continue
            y = rec["y"]
            n = rec["norms"]
            assert rec["info"]["kept"] == Xs[(y + 1) % Ly] * 2
            new = out["site"][(1, y)]
            s1 = cell["site"][(1, y)]
            val = ctm.network_value({r: (new[r] if r in ("C1", "T4", "C4") else s1[r]) for r in ctm.ROLES})
            # P (Rt^T Rb)^-1 P~ amplifies rounding by the half systems'
            # condition numbers (~1e4 here)
            assert abs(val * n[0] * n[1] * n[2] / before[(0, y)] - 1) < 1e-6, (Lx, Ly, y)


def test_wrong_cut_fails_the_row_identity(monkeypatch):
    """A planted mistake (every row renormalised with the projectors of the
    cut below it only) cannot satisfy the identity of the test above: with
    cuts of different dimensions its renewed tensors do not even fit."""
    orig = ctm.renormalise

    def wrong(net, X1, P3a, Pt3a, la, P3b, Pt3b, lb):
        return orig(net, X1, P3b, Pt3b, lb, P3b, Pt3b, lb)

    cell = dense_cell(2, 2, seed=22, Xs=[2, 3])
    monkeypatch.setattr(ctm, "renormalise", wrong)
    with pytest.raises(ValueError):
        ctm.cell_left_move(cell, 10 ** 6, rel_cutoff=0.0)


def test_cell_rotation_by_four_quarter_turns_is_identity():
    cell = tiny_cell(3, 2, seed=4)
    back = ctm.rotate_cell(cell, 4)
    assert back["Lx"] == 3 and back["Ly"] == 2
    for k, net in cell["site"].items():
        for r in ctm.ROLES:
            assert np.array_equal(back["site"][k][r][1], net[r][1])


@pytest.mark.parametrize("d", list("LURD"))
def test_cell_of_copies_every_direction(d):
    """Identical sites in a 2 x 3 cell: a move in any direction leaves every
    site with either one or two absorptions of the one-site move (the
    rotation puts the cell's columns or rows in line)."""
    cell = tiny_cell(2, 3, same=True)
    net = cell["site"][(0, 0)]
    once = ctm.move(net, d, 6)
    twice = ctm.move(once, d, 6)
    thrice = ctm.move(twice, d, 6)
    got = ctm.cell_move(cell, d, 6)
    seen = set()
    for s in got["site"].values():
        match = None
        for n_abs, want in ((1, once), (2, twice), (3, thrice)):
            if all(s[r][0] == want[r][0] and np.allclose(s[r][1], want[r][1], rtol=0, atol=1e-12)
                   for r in ctm.ROLES):
                match = n_abs
        assert match is not None
        seen.add(match)
    # L, R absorb the two columns; U, D the three rows
    assert seen == ({1, 2} if d in "LR" else {1, 2, 3})
