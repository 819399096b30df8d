"""Pins of the oracle's hybrid tree mode, the tool behind the GPU tree parity
test: a flag decision whose xi lies within the value tolerance of xi_crit is
"undecided" and is taken from the other side's values; every other decision
is the oracle's own.

Planted mistakes (on the CPU, in the table that stands for the other side):
a value changed far beyond the tolerance at a pixel whose decision is clear
must NOT change the hybrid tree, while a plain replay of the same table does
change its tree -- so a GPU that flipped a decided pixel would fail the GPU
test. Values equal to the oracle's own give its own tree back.
"""
import numpy as np
import pytest

import oracle
import scenes


@pytest.fixture(scope="module")
def cone():
    sc = scenes.cone_shock_amr(2, n_base=32, brick=8, levels=2)
    return sc, oracle.Oracle(sc)


def _table(t, scale=None):
    p_int = t["p_int"].copy()
    if scale is not None:
        p_int = p_int * scale
    return dict(level=t["level"], i=t["i"], j=t["j"], p_int=p_int, p_col=t["col"])


def _same_tree(a, b):
    return a["n_nodes"] == b["n_nodes"] and all((a[k] == b[k]).all() for k in ("level", "i", "j", "leaf"))


def test_own_values_give_own_tree(cone):
    sc, o = cone
    v = scenes.axis_view("+z")
    t = o.air(v, 32, 3, 0.5)
    h = o.air(v, 32, 3, 0.5, other=_table(t))
    assert _same_tree(t, h)
    hy = h["hybrid"]
    assert hy["decisions"] > 1000
    assert hy["taken_from_other"] == 0 and hy["unresolved"] == 0
    assert 0 <= hy["undecided"] < 0.01 * hy["decisions"]


def test_decided_flip_in_other_is_ignored(cone):
    """Plant the image maximum at one unrefined pixel of a zero-valued region
    in the other table: a plain replay of that table refines around it, the
    hybrid tree does not (the oracle's own xi there is exactly 0, decided)."""
    sc, o = cone
    v = scenes.axis_view("+z")
    t = o.air(v, 32, 3, 0.5)
    leaf, p = t["leaf"], t["p_int"]
    cand = [k for k in range(32 * 32) if leaf[k] and p[k] == 0.0 and 2 <= t["i"][k] < 30 and
            2 <= t["j"][k] < 30]
    assert cand
    k = cand[len(cand) // 2]
    add = np.zeros_like(p)
    add[k] = p.max()
    tab = _table(t)
    tab["p_int"] = tab["p_int"] + add
    try:
        r = o.air(v, 32, 3, 0.5, replay=tab)
        replay_changed = not _same_tree(r, t)
    except oracle.OracleError:
        replay_changed = True  # the replay needed pixels the table does not hold
    assert replay_changed
    h = o.air(v, 32, 3, 0.5, other=tab)
    assert _same_tree(h, t)
    assert h["hybrid"]["taken_from_other"] == 0


def test_margin_zero_counts_only_exact_ties(cone):
    sc, o = cone
    v = scenes.axis_view("+z")
    t = o.air(v, 32, 3, 0.5)
    h = o.air(v, 32, 3, 0.5, other=_table(t), rtol=0.0, margin=0.0)
    assert _same_tree(h, t) and h["hybrid"]["undecided"] == 0


def test_margin_switches_between_own_and_other(cone):
    """Other table: a constant value everywhere (xi = 0, nothing refines). With
    the usual margin the hybrid tree is the oracle's own but for the few
    undecided decisions. With an enormous
    margin every decision whose xi moves at all under the value tolerance
    follows the other table and stays unflagged; decisions where xi cannot
    move (all-zero stencils, or an isolated peak, where the scale-free xi
    stays 1) keep the oracle's own answer. The tree then lies strictly
    between the base image and the oracle's own tree."""
    sc, o = cone
    v = scenes.axis_view("+z")
    t = o.air(v, 32, 3, 0.5)
    tab = _table(t)
    tab["p_int"] = np.ones_like(tab["p_int"])
    r = o.air(v, 32, 3, 0.5, replay=tab)
    assert r["n_nodes"] == 32 * 32
    h = o.air(v, 32, 3, 0.5, other=tab)
    hy = h["hybrid"]
    # only the few undecided decisions may follow the other table
    assert hy["taken_from_other"] <= hy["undecided"] < 0.01 * hy["decisions"]
    assert _same_tree(h, t) or hy["taken_from_other"] > 0
    assert h["n_nodes"] >= t["n_nodes"] - 16 * hy["taken_from_other"]
    w = o.air(v, 32, 3, 0.5, other=tab, margin=1e30)
    assert 32 * 32 < w["n_nodes"] < t["n_nodes"]
    hy = w["hybrid"]
    assert hy["taken_from_other"] > 0 and hy["unresolved"] == 0
