"""Pins for the FP64 oracle: closed forms, hand-worked values, brute force and
invariants that fix what the oracle must compute independently of its own code.

Parkin (2010): Section 1/2 step (ii) (ray sums), Section 3 Eq. 1 and Eq. 2
(truncation error), Section 2 steps (iii)-(v) (scan, balance, refine, loop),
Table 1 (pixel counts)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Eq. 1 / 2
def test_xi_hand_values():
    d = json.load(open(os.path.join(GOLD, "eq2_hand_values.json")))
    for c in d["cases"]:
        s = np.array(c["stencil"], float)
        assert oracle.xi(s, 0) == pytest.approx(c["xi_axis"], abs=1e-15), c["name"]
        assert oracle.xi(s, 1) == pytest.approx(c["xi_literal"], abs=1e-15), c["name"]


def test_eq2_reduces_to_eq1_on_1d_images():
    """An image varying along one axis only: Eq. 2 (axis-sum reading) = Eq. 1."""
    rng = np.random.default_rng(1)
    for _ in range(500):
        a, b, c = rng.normal(size=3) * rng.choice([1e-3, 1, 1e4])
        eq1 = abs(c - 2 * b + a) / (abs(c - b) + abs(b - a))
        st_u = np.array([[a, b, c]] * 3)           # varies with u (di) only
        st_v = st_u.T.copy()                        # varies with v (dj) only
        assert oracle.xi(st_u, 0) == pytest.approx(eq1, rel=1e-12)
        assert oracle.xi(st_v, 0) == pytest.approx(eq1, rel=1e-12)
        # literal reading doubles the denominator
        assert oracle.xi(st_u, 1) == pytest.approx(eq1 / math.sqrt(2), rel=1e-12)


def test_xi_bounded_symmetric_dimensionless():
    """Section 3: the estimate is bounded (0 <= xi <= 1 after the clamp) and
    dimensionless (invariant under p -> a p + b); Eq. 2 is symmetric under
    reflections and exchange of the two image axes."""
    rng = np.random.default_rng(2)
    for _ in range(2000):
        s = rng.normal(size=(3, 3)) * rng.choice([1e-6, 1.0, 1e6])
        x = oracle.xi(s, 0)
        assert 0.0 <= x <= 1.0
        for t in (s.T, s[::-1], s[:, ::-1], s[::-1, ::-1].T):
            assert oracle.xi(np.ascontiguousarray(t), 0) == pytest.approx(x, rel=1e-12, abs=1e-15)
        a, b = rng.uniform(0.1, 10) * rng.choice([-1, 1]), rng.normal() * 100
        assert oracle.xi(a * s + b, 0) == pytest.approx(x, rel=1e-7, abs=1e-12)


# ------------------------------------------------------------- ray sums
def _ray(view, n0, L, i, j):
    """Camera convention: u = normalize(up x d), v = d x u; pixel centre
    -H + (i + 1/2) 2H / (n0 2^L)."""
    d = np.array(view.dir, float); d /= np.linalg.norm(d)
    u = np.cross(view.up, d); u /= np.linalg.norm(u)
    v = np.cross(d, u)
    H = view.half_extent
    pix = 2 * H / (n0 * 2 ** L)
    o = np.array(view.center) + (-H + (i + 0.5) * pix) * u + (-H + (j + 0.5) * pix) * v
    return o, d


def _clip(o, d, lo, hi):
    t0, t1 = -np.inf, np.inf
    for a in range(3):
        if d[a] == 0:
            if not (lo[a] <= o[a] < hi[a]):
                return None
        else:
            ta, tb = sorted(((lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]))
            t0, t1 = max(t0, ta), min(t1, tb)
    return (t0, t1) if t0 < t1 else None


def _dense_fields(scene):
    """Finest-level dense arrays of rho (and T) built directly from the brick list."""
    if scene.kind == "uniform":
        return scene.rho, scene.temp
    nx, ny, nz = scene.finest_n
    rho = np.full((nz, ny, nx), np.nan)
    T = np.full((nz, ny, nx), np.nan) if scene.temp is not None else None
    B, Lm = scene.brick, scene.max_level
    for b in range(len(scene.brick_level)):
        s = 1 << (Lm - scene.brick_level[b])
        ox, oy, oz = scene.brick_origin[b]
        blk = np.repeat(np.repeat(np.repeat(scene.rho[b], s, 0), s, 1), s, 2)
        rho[oz:oz + B * s, oy:oy + B * s, ox:ox + B * s] = blk
        if T is not None:
            tb = np.repeat(np.repeat(np.repeat(scene.temp[b], s, 0), s, 1), s, 2)
            T[oz:oz + B * s, oy:oy + B * s, ox:ox + B * s] = tb
    assert not np.isnan(rho).any()
    return rho, T


def _brute_force(scene, view, n0, L, i, j, M=400_000):
    """Sample the ray at M midpoints; I = sum over samples of the exact
    constant-medium solution, accumulated front to back."""
    o, d = _ray(view, n0, L, i, j)
    seg = _clip(o, d, scene.lo, scene.hi)
    nb = scene.n_bands
    if seg is None:
        return 0.0, np.zeros(nb)
    rho3, T3 = _dense_fields(scene)
    nz, ny, nx = rho3.shape
    t0, t1 = seg
    dt = (t1 - t0) / M
    t = t0 + (np.arange(M) + 0.5) * dt
    P = o[None, :] + t[:, None] * d[None, :]
    idx = []
    for a, n in enumerate((nx, ny, nz)):
        h = (scene.hi[a] - scene.lo[a]) / n
        idx.append(np.clip(np.floor((P[:, a] - scene.lo[a]) / h).astype(np.int64), 0, n - 1))
    rho = rho3[idx[2], idx[1], idx[0]]
    N = rho.sum() * dt
    I = np.zeros(nb)
    for b in range(nb):
        if scene.emis_mode == 1:
            lam = np.array([_lam_ref(scene, b, x) for x in T3[idx[2], idx[1], idx[0]]]) \
                if M <= 20000 else _lam_vec(scene, b, T3[idx[2], idx[1], idx[0]])
            j_ = rho * rho * lam
        else:
            j_ = rho * rho
        alpha = scene.kappa[b] * rho
        dtau = alpha * dt
        tau_before = np.concatenate([[0.0], np.cumsum(dtau)[:-1]])
        with np.errstate(divide="ignore", invalid="ignore"):
            term = np.where(alpha > 0, j_ / np.where(alpha > 0, alpha, 1) * -np.expm1(-dtau),
                            j_ * dt)
        I[b] = (term * np.exp(-tau_before)).sum()
    return N, I


def _lam_vec(scene, b, T):
    nt = scene.lambda_table.shape[1]
    x = (np.log10(T) - scene.logT_lo) / (scene.logT_hi - scene.logT_lo) * (nt - 1)
    x = np.clip(x, 0, nt - 1)
    k = np.minimum(np.floor(x).astype(int), nt - 2)
    w = x - k
    tab = scene.lambda_table[b].astype(np.float64)
    return (1 - w) * tab[k] + w * tab[k + 1]


def _lam_ref(scene, b, T):
    return _lam_vec(scene, b, np.array([T]))[0]


def test_uniform_slab_closed_form():
    """Constant medium of depth D: N = rho D, I = S (1 - exp(-tau)), S = j/alpha."""
    n = 16
    rho = np.zeros((n, n, n))
    rho[4:12] = 2.5                            # z-cells 4..11: depth 8 cells = 1.0
    for kappa in (0.0, 0.05, 0.7, 4.0):
        sc = scenes.uniform_from_array(rho, kappa=kappa)
        o = oracle.Oracle(sc)
        col, inten, steps = o.trace(scenes.axis_view("+z"), 16, [0, 0], [3, 9], [5, 15])
        D = 1.0
        assert col == pytest.approx([2.5 * D] * 2, rel=1e-14)
        if kappa == 0:
            expect = 2.5 ** 2 * D
        else:
            S = 2.5 ** 2 / (kappa * 2.5)
            expect = S * -math.expm1(-kappa * 2.5 * D)
        assert inten[:, 0] == pytest.approx([expect] * 2, rel=1e-13)
        assert list(steps) == [n, n]


def test_two_slab_front_to_back():
    """Front slab A then back slab B: I = S_A(1-e^-tA) + e^-tA S_B(1-e^-tB);
    the opposite view swaps the roles."""
    n = 8
    rho = np.zeros((n, n, n))
    rho[0:4] = 1.0     # z in [-1, 0)
    rho[4:8] = 3.0     # z in [0, 1)
    kappa = 0.4
    sc = scenes.uniform_from_array(rho, kappa=kappa)
    o = oracle.Oracle(sc)
    D = 1.0

    def slab(r):
        return r / kappa * -math.expm1(-kappa * r * D), kappa * r * D

    SA, tA = slab(1.0)
    SB, tB = slab(3.0)
    _, Ip, _ = o.trace(scenes.axis_view("+z"), 8, [0], [2], [2])   # rays travel +z: low z first
    _, Im, _ = o.trace(scenes.axis_view("-z"), 8, [0], [2], [2])
    assert Ip[0, 0] == pytest.approx(SA + math.exp(-tA) * SB, rel=1e-13)
    assert Im[0, 0] == pytest.approx(SB + math.exp(-tB) * SA, rel=1e-13)
    assert Ip[0, 0] != pytest.approx(Im[0, 0], rel=1e-3)


def test_sphere_column_density_converges():
    """Uniform sphere: N(b) -> 2 rho0 sqrt(R^2 - b^2) as the grid is refined."""
    R = 0.6
    errs = []
    bs = np.array([0.0, 0.1, 0.25, 0.4, 0.5])
    for n in (32, 64, 128):
        o = oracle.Oracle(scenes.uniform_sphere(n, R))
        v = scenes.axis_view("+z")
        # pixel whose centre is at (u, v) = (b + small offset, 0.0123)
        cols = []
        for b in bs:
            o_, d = np.array([b + 1e-3, 0.0123, 0.0]), np.array([0.0, 0.0, 1.0])
            res = 4096
            i = int(round((o_[0] + 1) / (2 / res) - 0.5))
            j = int(round((o_[1] + 1) / (2 / res) - 0.5))
            c, _, _ = o.trace(v, res, [0], [i], [j])
            u_c, v_c = -1 + (i + 0.5) * 2 / res, -1 + (j + 0.5) * 2 / res
            exact = 2 * math.sqrt(max(R * R - u_c * u_c - v_c * v_c, 0.0))
            cols.append(abs(c[0] - exact))
        errs.append(max(cols))
    assert errs[-1] < 2.5 * (2 / 128)          # within ~one cell of chord per end
    assert errs[2] < errs[0]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_sampling_uniform(seed):
    sc = scenes.random_uniform(seed, n=(6, 7, 8), kappa=0.6)
    o = oracle.Oracle(sc)
    rng = np.random.default_rng(seed)
    views = scenes.random_views(seed, 3)
    for v in views:
        for _ in range(2):
            i, j = rng.integers(0, 32, size=2)
            c, I, _ = o.trace(v, 32, [0], [i], [j])
            Nb, Ib = _brute_force(sc, v, 32, 0, i, j)
            if Nb == 0.0:
                assert c[0] == 0.0
                continue
            assert c[0] == pytest.approx(Nb, rel=2e-4)
            assert I[0, 0] == pytest.approx(Ib[0], rel=2e-4)


def test_brute_force_sampling_amr_multiband():
    """Mixed-level brick grid with temperatures and 4 bands."""
    sc = scenes.cone_shock_amr(3, n_base=16, brick=4, levels=2, n_bands=4, e_lo=0.5,
                               e_hi=10.0, kappa0=0.5, thickness=0.15)
    assert len(set(sc.brick_level.tolist())) == 3
    o = oracle.Oracle(sc)
    rng = np.random.default_rng(7)
    views = scenes.random_views(11, 2) + [scenes.axis_view("+x", 1.0)]
    checked = 0
    for v in views:
        for _ in range(3):
            i, j = rng.integers(4, 28, size=2)
            c, I, _ = o.trace(v, 32, [0], [i], [j])
            Nb, Ib = _brute_force(sc, v, 32, 0, i, j, M=600_000)
            if Nb == 0.0:
                continue
            checked += 1
            assert c[0] == pytest.approx(Nb, rel=3e-4)
            for b in range(4):
                assert I[0, b] == pytest.approx(Ib[b], rel=3e-4, abs=1e-12 * max(1, Ib.max()))
    assert checked >= 6


def test_optically_thin_flux_equals_grid_sum():
    """kappa = 0, axis view, pixels aligned with and no larger than the finest
    cells: sum_pixels I A = sum_cells j V (the paper's 'fixed' error ~0)."""
    sc = scenes.wind_shell_uniform(0, n=32, kappa=0.0)
    o = oracle.Oracle(sc)
    for res in (32, 64):
        img = o.fixed(scenes.axis_view("+z"), res)
        flux = img["inten"][:, 0].sum() * (2.0 / res) ** 2
        grid = (sc.rho ** 2).sum() * (2.0 / 32) ** 3
        assert flux == pytest.approx(grid, rel=1e-13)
    # AMR with temperatures: pixels at the finest cell size
    am = scenes.cone_shock_amr(1, n_base=16, brick=4, levels=2, kappa0=0.0, thickness=0.15)
    oa = oracle.Oracle(am)
    img = oa.fixed(scenes.axis_view("+z"), 64)
    flux = img["inten"][:, 0].sum() * (2.0 / 64) ** 2
    grid = 0.0
    hf = 2.0 / 64
    for b in range(len(am.brick_level)):
        vol = (hf * (1 << (2 - am.brick_level[b]))) ** 3
        lam = _lam_vec(am, 0, am.temp[b].astype(np.float64).ravel())
        grid += (am.rho[b].astype(np.float64).ravel() ** 2 * lam).sum() * vol
    assert flux == pytest.approx(grid, rel=1e-12)


def _dense_cell_ids(scene):
    """Finest-level dense array of cell identifiers (brick, local cell), built
    directly from the brick list: equal ids mark one (possibly coarse) cell."""
    nx, ny, nz = scene.finest_n
    ids = np.full((nz, ny, nx), -1, np.int64)
    B, Lm = scene.brick, scene.max_level
    for b in range(len(scene.brick_level)):
        s = 1 << (Lm - scene.brick_level[b])
        ox, oy, oz = scene.brick_origin[b]
        loc = b * B ** 3 + np.arange(B ** 3).reshape(B, B, B)
        ids[oz:oz + B * s, oy:oy + B * s, ox:ox + B * s] = \
            np.repeat(np.repeat(np.repeat(loc, s, 0), s, 1), s, 2)
    assert (ids >= 0).all()
    return ids


@pytest.mark.parametrize("axis", ["+x", "-x", "+y", "-y", "+z", "-z"])
def test_amr_axis_columns_by_definition(axis):
    """Rays along a grid axis through a three-level brick grid, one per finest
    column: N = sum of rho ds down the column, the step count = the number of
    distinct cells it crosses, and (kappa = 0) I = sum of j ds, each read off
    dense finest-level arrays. Pins the brick lookup, the column each pixel's
    ray runs down and the merging of a coarse cell's finest pieces into one
    chord (the order of travel is pinned by the two-slab test)."""
    sc = scenes.cone_shock_amr(3, n_base=16, brick=4, levels=2, kappa0=0.0, thickness=0.15)
    assert len(set(sc.brick_level.tolist())) == 3
    rho3, T3 = _dense_fields(sc)
    ids = _dense_cell_ids(sc)
    lam3 = _lam_vec(sc, 0, T3.ravel()).reshape(T3.shape)
    res = sc.finest_n[0]
    h = [(sc.hi[a] - sc.lo[a]) / sc.finest_n[a] for a in range(3)]
    v = scenes.axis_view(axis)
    img = oracle.Oracle(sc).fixed(v, res)
    multi = 0
    for k in range(res * res):
        org, d = _ray(v, res, 0, img["i"][k], img["j"][k])
        a = int(np.argmax(np.abs(d)))
        sel = [int(np.floor((org[c] - sc.lo[c]) / h[c])) for c in range(3)]
        sel[a] = slice(None)
        key = (sel[2], sel[1], sel[0])
        r, cid, lam = rho3[key], ids[key], lam3[key]
        if d[a] < 0:
            r, cid, lam = r[::-1], cid[::-1], lam[::-1]
        steps = 1 + int(np.count_nonzero(np.diff(cid)))
        multi += steps < len(cid)
        assert img["steps"][k] == steps
        assert img["col"][k] == pytest.approx(r.sum() * h[a], rel=1e-12)
        assert img["inten"][k, 0] == pytest.approx((r * r * lam).sum() * h[a], rel=1e-12)
    assert multi > res  # many columns cross coarse cells


def test_amr_single_level_equals_uniform():
    sc = scenes.random_uniform(5, n=(8, 8, 8), kappa=0.3)
    am = scenes.as_amr_single_level(sc, 4)
    ou, oa = oracle.Oracle(sc), oracle.Oracle(am)
    for v in scenes.random_views(3, 3) + [scenes.axis_view("+y")]:
        a = ou.fixed(v, 16)
        b = oa.fixed(v, 16)
        np.testing.assert_allclose(a["col"], b["col"], rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(a["inten"], b["inten"], rtol=1e-13, atol=1e-14)
        assert (a["steps"] == b["steps"]).all()


def test_lambda_table_interpolation():
    sc = scenes.cone_shock_amr(0, n_base=8, brick=4, levels=0, n_bands=3, e_lo=0.5)
    o = oracle.Oracle(sc)
    tab = sc.lambda_table.astype(np.float64)
    nt = tab.shape[1]
    for b in range(3):
        for k in (0, 5, 31, nt - 1):
            T = 10 ** (4 + 5 * k / (nt - 1))
            assert o.lam(b, T) == pytest.approx(tab[b, k], rel=1e-12, abs=1e-300)
        T = 10 ** (4 + 5 * 10.25 / (nt - 1))
        assert o.lam(b, T) == pytest.approx(0.75 * tab[b, 10] + 0.25 * tab[b, 11], rel=1e-9)
        assert o.lam(b, 10.0) == tab[b, 0]
        assert o.lam(b, 1e12) == tab[b, -1]


# --------------------------------------------------------- refinement loop
def _pyramid_replay(fn, n0, Lm):
    lv, ii, jj, p = [], [], [], []
    for L in range(Lm + 1):
        n = n0 << L
        J, I = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        u = -1 + (I + 0.5) * 2 / n
        v = -1 + (J + 0.5) * 2 / n
        lv.append(np.full(n * n, L)); ii.append(I.ravel()); jj.append(J.ravel())
        p.append(fn(u, v).ravel())
    p = np.concatenate(p).astype(np.float64)
    return dict(level=np.concatenate(lv), i=np.concatenate(ii), j=np.concatenate(jj),
                p_int=p, p_col=p)


def test_step_edge_tree_golden():
    g = json.load(open(os.path.join(GOLD, "step_edge_tree.json")))
    sc = scenes.random_uniform(0, n=(4, 4, 4))
    o = oracle.Oracle(sc)
    rp = _pyramid_replay(lambda u, v: (u > 0).astype(float), g["base_res"], g["max_level"])
    t = o.air(scenes.axis_view("+z"), g["base_res"], g["max_level"], g["xi_crit"], replay=rp)
    for k in ("n_refined", "n_nodes", "n_leaves", "n_sweeps"):
        assert t[k] == g[k], k
    leaf = t["leaf"] == 1
    for L, cols in g["leaf_columns"].items():
        sel = leaf & (t["level"] == int(L))
        assert sorted(set(t["i"][sel].tolist())) == cols
        assert sel.sum() == len(cols) * (g["base_res"] << int(L))


def _raster_levels(t, n0, Lm):
    nf = n0 << Lm
    R = np.full((nf, nf), -1)
    leaf = t["leaf"] == 1
    for L, i, j in zip(t["level"][leaf], t["i"][leaf], t["j"][leaf]):
        s = 1 << (Lm - L)
        assert (R[j * s:(j + 1) * s, i * s:(i + 1) * s] == -1).all()
        R[j * s:(j + 1) * s, i * s:(i + 1) * s] = L
    return R


def _check_tree(t, n0, Lm):
    assert t["n_nodes"] == n0 * n0 + 4 * t["n_refined"]           # Table 1 counting
    assert t["n_leaves"] == n0 * n0 + 3 * t["n_refined"]
    R = _raster_levels(t, n0, Lm)
    assert (R >= 0).all()                                          # leaves tile the image
    # 2:1 balance across the 8 neighbours
    for dj, di in ((0, 1), (1, 0), (1, 1), (1, -1)):
        a = R[max(dj, 0):R.shape[0] + min(dj, 0), max(di, 0):R.shape[1] + min(di, 0)]
        b = R[max(-dj, 0):R.shape[0] + min(-dj, 0), max(-di, 0):R.shape[1] + min(-di, 0)]
        assert np.abs(a - b).max() <= 1
    # every node's parent is an interior node one level up
    par = t["parent"]
    k = np.nonzero(par >= 0)[0]
    assert (t["level"][par[k]] == t["level"][k] - 1).all()
    assert (t["leaf"][par[k]] == 0).all()
    assert (t["i"][k] // 2 == t["i"][par[k]]).all() and (t["j"][k] // 2 == t["j"][par[k]]).all()


def test_tree_invariants_wind_shell():
    sc = scenes.wind_shell_uniform(0)
    o = oracle.Oracle(sc)
    v = scenes.axis_view("+z")
    rays = []
    for xc in (0.8, 0.5, 0.2):
        t = o.air(v, 16, 3, xc)
        _check_tree(t, 16, 3)
        rays.append(t["n_nodes"])
        # nothing left unflagged above threshold: every leaf below the top level has xi < xi_crit
    assert rays[0] <= rays[1] <= rays[2]
    # xi_crit > 1: base image only
    t = o.air(v, 16, 3, 1.01)
    assert t["n_nodes"] == 256 and t["n_refined"] == 0
    # xi_crit = 0: every leaf at the maximum level, equal to the fixed finest image
    t = o.air(v, 16, 3, 0.0)
    _check_tree(t, 16, 3)
    leaf = t["leaf"] == 1
    assert (t["level"][leaf] == 3).all() and leaf.sum() == 128 * 128
    f = o.fixed(v, 128)
    key = t["j"][leaf] * 128 + t["i"][leaf]
    order = np.argsort(key)
    assert (t["col"][leaf][order] == f["col"]).all()
    assert (t["inten"][leaf][order] == f["inten"]).all()


def test_tree_invariants_amr_and_refine_on():
    sc = scenes.cone_shock_amr(0, n_base=32, brick=8, levels=2)
    o = oracle.Oracle(sc)
    v = scenes.axis_view("+z")
    for ro in (0, 1, 2):
        for xn in (0, 1):
            t = o.air(v, 16, 3, 0.5, xi_norm=xn, refine_on=ro)
            _check_tree(t, 16, 3)
    a = o.air(v, 16, 3, 0.5, refine_on=0)["n_nodes"]
    b = o.air(v, 16, 3, 0.5, refine_on=1)["n_nodes"]
    c = o.air(v, 16, 3, 0.5, refine_on=2)["n_nodes"]
    assert c >= max(a, b)


def test_scan_is_complete():
    """After the loop every leaf below the top level has xi < xi_crit with the
    final neighbour values (step v: loop until nothing is flagged). The stencil
    lookup here is a dictionary walk up the levels, not the oracle's maps."""
    sc = scenes.wind_shell_uniform(2)
    o = oracle.Oracle(sc)
    v = scenes.axis_view("+z")
    n0, Lm, xc = 16, 3, 0.5
    t = o.air(v, n0, Lm, xc)
    maps = {}
    for k in range(t["n_nodes"]):
        maps[(t["level"][k], t["i"][k], t["j"][k])] = k

    def value(L, i, j):
        n = n0 << L
        i, j = min(max(i, 0), n - 1), min(max(j, 0), n - 1)
        for l in range(L, -1, -1):
            k = maps.get((l, i >> (L - l), j >> (L - l)))
            if k is not None:
                return t["p_int"][k]
        raise AssertionError

    for k in np.nonzero((t["leaf"] == 1) & (t["level"] < Lm))[0]:
        L, i, j = t["level"][k], t["i"][k], t["j"][k]
        s = [[value(L, i + di, j + dj) for di in (-1, 0, 1)] for dj in (-1, 0, 1)]
        assert oracle.xi(np.array(s), 0) < xc


def test_table1_counting_identity():
    """Table 1: every AIR row's pixel count is 32^2 + 4 x (number of refined
    pixels), so 'Pixels' counts traced rays (all tree nodes). The oracle counts
    n_nodes the same way (checked in _check_tree)."""
    g = json.load(open(os.path.join(GOLD, "table1_counts.json")))
    n0 = g["base_res"]
    assert g["fixed_pixels"] == (n0 << g["levels"]) ** 2
    for row in g["air"]:
        assert (row["pixels"] - n0 * n0) % 4 == 0
        assert (row["pixels"] - n0 * n0) % 3 != 0
    # lower threshold -> more pixels and more time, as in the table
    px = [r["pixels"] for r in sorted(g["air"], key=lambda r: r["xi_crit"])]
    assert px == sorted(px, reverse=True)


def test_replay_reproduces_own_tree():
    """Feeding the oracle its own traced values gives back the same tree."""
    sc = scenes.wind_shell_uniform(1)
    o = oracle.Oracle(sc)
    v = scenes.axis_view("+z")
    t = o.air(v, 16, 3, 0.3)
    rp = dict(level=t["level"], i=t["i"], j=t["j"], p_int=t["p_int"], p_col=t["col"])
    r = o.air(v, 16, 3, 0.3, replay=rp)
    for k in ("level", "i", "j", "leaf", "parent"):
        assert (r[k] == t[k]).all()


def test_replay_missing_node_is_an_error():
    sc = scenes.wind_shell_uniform(1)
    o = oracle.Oracle(sc)
    v = scenes.axis_view("+z")
    t = o.air(v, 16, 3, 0.3)
    keep = t["level"] < 2
    rp = dict(level=t["level"][keep], i=t["i"][keep], j=t["j"][keep],
              p_int=t["p_int"][keep], p_col=t["col"][keep])
    with pytest.raises(oracle.OracleError):
        o.air(v, 16, 3, 0.3, replay=rp)
