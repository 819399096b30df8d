"""Seeded synthetic scenes and views for adaptive image ray-tracing (AIR).

These generators build the *inputs* that both the CUDA path and the FP64 oracle
consume: simulation grids (uniform Cartesian or block-structured AMR), the
emission table, opacities and camera views. They contain none of the method's
arithmetic (no ray marching, no radiative transfer, no refinement criterion);
they only sample analytic density/temperature fields at cell centres.

The paper's own test problem (Section 3: a hot ring on a FLASH/PARAMESH AMR grid
with MEKAL emissivities) cannot be rebuilt here: the simulation output and the
MEKAL tables are not available. These scenes stand in for it with the shapes of
the paper's workloads: an AMR grid of cubic bricks refined around a thin, hot,
emitting feature that fills a fraction of the image, and a smooth uniform-grid
wind with a perturbed shell.

Every random number is drawn from numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

K_B_KEV = 8.617333262e-8  # Boltzmann constant in keV / K


# --------------------------------------------------------------------------
# Views (orthographic camera, observer at a distance much larger than the box)
# --------------------------------------------------------------------------
@dataclass
class View:
    """Orthographic view: rays travel along `dir`; the image plane is spanned by
    u = normalize(up x dir) and v = dir x u, centred on `center`, covering
    [-half_extent, half_extent]^2."""
    dir: tuple
    up: tuple = (0.0, 1.0, 0.0)
    center: tuple = (0.0, 0.0, 0.0)
    half_extent: float = 1.0


def axis_view(axis: str = "+z", half_extent: float = 1.0) -> View:
    sign = -1.0 if axis[0] == "-" else 1.0
    k = "xyz".index(axis[-1])
    d = [0.0, 0.0, 0.0]
    d[k] = sign
    up = (0.0, 1.0, 0.0) if k != 1 else (1.0, 0.0, 0.0)
    return View(dir=tuple(d), up=up, half_extent=half_extent)


def random_views(seed: int, n: int, half_extent: float = math.sqrt(3.0)) -> list:
    """n directions uniform on the sphere (normalised Gaussian triples)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        g = rng.standard_normal(3)
        d = g / np.linalg.norm(g)
        up = (0.0, 1.0, 0.0) if abs(d[1]) < 0.999 else (1.0, 0.0, 0.0)
        out.append(View(dir=tuple(float(x) for x in d), up=up, half_extent=half_extent))
    return out


# --------------------------------------------------------------------------
# Emission table (synthetic stand-in for the MEKAL look-up tables)
# --------------------------------------------------------------------------
def band_edges(n_bands: int, e_lo: float = 0.5, e_hi: float = 10.0) -> np.ndarray:
    """Log-spaced band edges in keV."""
    return e_lo * (e_hi / e_lo) ** (np.arange(n_bands + 1) / n_bands)


def cooling_table(edges_kev: np.ndarray, n_tbins: int = 64, logT_lo: float = 4.0,
                  logT_hi: float = 9.0) -> np.ndarray:
    """Band emissivity per unit rho^2, Lambda_b(T), tabulated at n_tbins points
    uniform in log10 T. Thermal-bremsstrahlung shape: the band integral of
    T^-1/2 exp(-E/kT) dE, i.e. T^1/2 (exp(-E_lo/kT) - exp(-E_hi/kT)), with T in
    units of 1e7 K. Returned as float32 [n_bands, n_tbins]; the table values are
    data shared by both sides."""
    logT = logT_lo + (logT_hi - logT_lo) * np.arange(n_tbins) / (n_tbins - 1)
    T = 10.0 ** logT
    kT = K_B_KEV * T
    lo = edges_kev[:-1, None]
    hi = edges_kev[1:, None]
    tab = np.sqrt(T / 1e7)[None, :] * (np.exp(-lo / kT[None, :]) - np.exp(-hi / kT[None, :]))
    return tab.astype(np.float32)


def band_kappa(edges_kev: np.ndarray, kappa0: float) -> np.ndarray:
    """Photo-absorption-like opacity per unit density: kappa0 (E_mid / 1 keV)^(-8/3)."""
    emid = np.sqrt(edges_kev[:-1] * edges_kev[1:])
    return (kappa0 * emid ** (-8.0 / 3.0)).astype(np.float64)


# --------------------------------------------------------------------------
# Scene container
# --------------------------------------------------------------------------
@dataclass
class Scene:
    kind: str                      # "uniform" or "amr"
    lo: tuple
    hi: tuple
    n: tuple                       # uniform: cells per axis; amr: base cells per axis
    rho: np.ndarray                # uniform [nz,ny,nx]; amr [nb,B,B,B] (x fastest)
    temp: np.ndarray | None = None
    brick: int = 0
    max_level: int = 0
    brick_level: np.ndarray | None = None    # int32 [nb]
    brick_origin: np.ndarray | None = None   # int32 [nb,3] (x,y,z) in finest-cell units
    emis_mode: int = 0             # 0: j = rho^2 ; 1: j = rho^2 Lambda_b(T)
    lambda_table: np.ndarray | None = None   # float32 [n_bands, n_tbins]
    logT_lo: float = 4.0
    logT_hi: float = 9.0
    kappa: np.ndarray = field(default_factory=lambda: np.zeros(1))
    name: str = ""

    @property
    def n_bands(self) -> int:
        return int(len(self.kappa))

    @property
    def n_cells(self) -> int:
        return int(self.rho.size)

    @property
    def finest_n(self) -> tuple:
        s = 1 << self.max_level if self.kind == "amr" else 1
        return tuple(int(x) * s for x in self.n)


# --------------------------------------------------------------------------
# Uniform grid: r^-2 wind plus a perturbed Gaussian shell
# --------------------------------------------------------------------------
WIND_SHELL_KAPPA = 3.0 / 87.0
"""Opacity per unit density for the wind+shell scene. 87 is the analytic column
density of the noise-free profile along the central sight line
(2*(0.05*400 + 19) for the floored r^-2 wind, plus 9*sigma*sqrt(2 pi)/0.25*2 for
the shell), so the central optical depth is close to 3."""


def wind_shell_uniform(seed: int = 0, n: int = 64, kappa: float = WIND_SHELL_KAPPA,
                       sigma: float = 0.05, sigma_n: float = 0.05) -> Scene:
    """64^3 Cartesian grid over [-1,1]^3 with FP64 density
    rho = max(r,0.05)^-2 (1 + 9 g exp(sigma_n z - sigma_n^2/2)),
    g = exp(-(r-0.5)^2 / (2 sigma^2)), z ~ N(0,1) per cell (5% lognormal noise on a
    10x overdense shell). Emissivity j = rho^2, opacity kappa*rho, one band."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    g = np.exp(-((r - 0.5) ** 2) / (2 * sigma * sigma))
    noise = rng.standard_normal((n, n, n))
    rho = np.maximum(r, 0.05) ** -2 * (1.0 + 9.0 * g * np.exp(sigma_n * noise - 0.5 * sigma_n ** 2))
    return Scene(kind="uniform", lo=(-1.0,) * 3, hi=(1.0,) * 3, n=(n, n, n),
                 rho=rho.astype(np.float64), emis_mode=0,
                 kappa=np.array([kappa], dtype=np.float64), name=f"wind_shell_{n}^3_s{seed}")


# --------------------------------------------------------------------------
# Block-structured AMR: conical colliding-wind shock
# --------------------------------------------------------------------------
def _cone_distance(px, py, pz, apex, half_angle):
    """Signed distance to the lateral surface of a cone (axis +x) in the (a, r)
    half-plane, and a mask of points whose projection lands on the a>=0 sheet."""
    a = px - apex[0]
    r = np.sqrt((py - apex[1]) ** 2 + (pz - apex[2]) ** 2)
    ct, st = math.cos(half_angle), math.sin(half_angle)
    d = r * ct - a * st
    on_sheet = a * ct + r * st >= 0.0
    d = np.where(on_sheet, d, np.sqrt(a * a + r * r))
    return d, on_sheet


def _lattice_noise(lattice, lo, scale, PX, PY, PZ):
    """Unit-variance field: trilinear interpolation of lattice normals, divided
    pointwise by the root of the summed squared weights."""
    n = lattice.shape[0]
    acc = np.zeros(PX.shape)
    w2 = np.zeros(PX.shape)
    g = [(P - lo) / scale for P in (PX, PY, PZ)]
    i = [np.clip(np.floor(x).astype(np.int64), 0, n - 2) for x in g]
    f = [x - k for x, k in zip(g, i)]
    for dz in (0, 1):
        wz = f[2] if dz else 1.0 - f[2]
        for dy in (0, 1):
            wy = f[1] if dy else 1.0 - f[1]
            for dx in (0, 1):
                wx = f[0] if dx else 1.0 - f[0]
                w = wx * wy * wz
                acc += w * lattice[i[2] + dz, i[1] + dy, i[0] + dx]
                w2 += w * w
    return acc / np.sqrt(w2)


def cone_shock_amr(seed: int = 0, n_base: int = 128, brick: int = 16, levels: int = 3,
                   n_bands: int = 1, e_lo: float = 1.0, e_hi: float = 10.0,
                   kappa0: float = 0.3, half_angle_deg: float = 30.0,
                   thickness: float = 0.04, apex=(-0.5, 0.0, 0.0),
                   star=(-0.8, 0.0, 0.0), clump_sigma: float = 0.3,
                   clump_scale: float = 0.0, n_tbins: int = 64,
                   refine_margin: float = 1.0, keep_smooth: bool = False) -> Scene:
    """Block-AMR grid over [-1,1]^3: n_base^3 base cells in brick^3 bricks,
    `levels` refinement levels (factor 2) on bricks near a conical shock
    (apex `apex`, axis +x, half-angle 30 deg, shell thickness 0.04 = 0.02 of the
    box). A brick is refined while the cone surface passes within
    refine_margin * (brick half-diagonal) + thickness/2 of its centre.

    Fields (FP32, sampled at cell centres of each leaf brick at its own level):
      rho = rho_w * (4 in the shocked shell, 0.25 inside the cone, 1 outside)
            * exp(0.3 z - 0.045)  (lognormal clumping, z ~ N(0,1))
      z is drawn independently per cell (clump_scale = 0, the default), or is a
      clump field of correlation length clump_scale > 0: unit normals on a
      lattice of that spacing, trilinearly interpolated and renormalised to
      unit variance at every point, so z is a function of position, the same in
      coarse and fine bricks.
      rho_w = max(|x - star|, 0.05)^-2
      T = 10^7.5 K in the shell, 10^4 K elsewhere.
    Emission: j_b = rho^2 Lambda_b(T) (64-bin table), absorption kappa_b rho with
    kappa_b = kappa0 (E_mid/keV)^-8/3 over n_bands log-spaced bands in [e_lo, e_hi].
    """
    assert n_base % brick == 0
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = -1.0, 1.0
    nf = n_base << levels
    hf = (hi - lo) / nf
    half_angle = math.radians(half_angle_deg)
    nb0 = n_base // brick

    # level-0 bricks, then refine level by level
    g = np.arange(nb0)
    bz, by, bx = np.meshgrid(g, g, g, indexing="ij")
    S0 = brick << levels
    cur = np.stack([bx.ravel(), by.ravel(), bz.ravel()], axis=1).astype(np.int64) * S0
    leaf_levels, leaf_origins = [], []
    for lev in range(levels + 1):
        S = brick << (levels - lev)
        ctr = lo + (cur + S / 2.0) * hf
        d, _ = _cone_distance(ctr[:, 0], ctr[:, 1], ctr[:, 2], apex, half_angle)
        half_diag = math.sqrt(3.0) * 0.5 * S * hf
        refine = (np.abs(d) <= refine_margin * half_diag + thickness / 2) if lev < levels \
            else np.zeros(len(cur), dtype=bool)
        keep = cur[~refine]
        leaf_levels.append(np.full(len(keep), lev, dtype=np.int32))
        leaf_origins.append(keep)
        ref = cur[refine]
        h = S // 2
        kids = []
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    kids.append(ref + np.array([dx * h, dy * h, dz * h], dtype=np.int64))
        cur = np.concatenate(kids, axis=0) if kids else np.zeros((0, 3), np.int64)
        if len(cur):
            cur = cur[np.lexsort((cur[:, 0], cur[:, 1], cur[:, 2]))]
    levels_arr = np.concatenate(leaf_levels)
    origins = np.concatenate(leaf_origins, axis=0)
    nb = len(levels_arr)

    # fields at cell centres, brick by brick (vectorised over chunks of bricks)
    rho = np.empty((nb, brick, brick, brick), dtype=np.float32)
    temp = np.empty((nb, brick, brick, brick), dtype=np.float32)
    off = np.arange(brick) + 0.5
    smooth = np.empty(rho.shape, dtype=np.float64) if keep_smooth else None
    if clump_scale > 0:
        nl = int(math.ceil((hi - lo) / clump_scale)) + 2
        lattice = rng.standard_normal((nl, nl, nl))
    else:
        cell_noise = rng.standard_normal(nb * brick ** 3).reshape(nb, brick, brick, brick)
    chunk = max(1, (1 << 22) // brick ** 3)
    for lev in range(levels + 1):
        sel_all = np.nonzero(levels_arr == lev)[0]
        step = 1 << (levels - lev)
        for c0 in range(0, len(sel_all), chunk):
            sel = sel_all[c0:c0 + chunk]
            o = origins[sel].astype(np.float64)
            cx = lo + (o[:, 0:1] + off[None, :] * step) * hf
            cy = lo + (o[:, 1:2] + off[None, :] * step) * hf
            cz = lo + (o[:, 2:3] + off[None, :] * step) * hf
            shp = (len(sel), brick, brick, brick)
            PX = np.broadcast_to(cx[:, None, None, :], shp)
            PY = np.broadcast_to(cy[:, None, :, None], shp)
            PZ = np.broadcast_to(cz[:, :, None, None], shp)
            rw = np.sqrt((PX - star[0]) ** 2 + (PY - star[1]) ** 2 + (PZ - star[2]) ** 2)
            rho_w = np.maximum(rw, 0.05) ** -2
            d, on_sheet = _cone_distance(PX, PY, PZ, apex, half_angle)
            shell = (np.abs(d) <= thickness / 2) & on_sheet
            inside = (d < -thickness / 2) & on_sheet
            fac = np.where(shell, 4.0, np.where(inside, 0.25, 1.0))
            if clump_scale > 0:
                z = _lattice_noise(lattice, lo, clump_scale, PX, PY, PZ)
            else:
                z = cell_noise[sel]
            clump = np.exp(clump_sigma * z - 0.5 * clump_sigma ** 2)
            rho[sel] = (rho_w * fac * clump).astype(np.float32)
            if keep_smooth:
                smooth[sel] = rho_w * fac
            temp[sel] = np.where(shell, 10.0 ** 7.5, 1e4).astype(np.float32)

    edges = band_edges(n_bands, e_lo, e_hi)
    sc = Scene(kind="amr", lo=(lo,) * 3, hi=(hi,) * 3, n=(n_base,) * 3, rho=rho, temp=temp,
                 brick=brick, max_level=levels, brick_level=levels_arr,
                 brick_origin=origins.astype(np.int32), emis_mode=1,
                 lambda_table=cooling_table(edges, n_tbins), logT_lo=4.0, logT_hi=9.0,
                 kappa=band_kappa(edges, kappa0),
                 name=f"cone_amr_{n_base}^3_b{brick}_L{levels}_{n_bands}band_c{clump_scale}_s{seed}")
    if keep_smooth:
        sc.rho_smooth = smooth
        sc.clump_sigma = clump_sigma
    return sc


def clumps_cones_amr(seed: int = 0, n_base: int = 512, brick: int = 32, levels: int = 5,
                     n_clumps: int = 200, r_range=(0.005, 0.02), contrast=(10.0, 1000.0),
                     clump_factor: float = 1.0, cone_levels: int = 0, n_bands: int = 32,
                     e_lo: float = 0.5, e_hi: float = 10.0, kappa0: float = 0.3,
                     half_angle_deg: float = 30.0, thickness: float = 0.04,
                     clump_sigma: float = 0.3, n_tbins: int = 64) -> Scene:
    """Large block-AMR scene over [-1,1]^3: two colliding-wind shock cones and
    n_clumps dense clumps.

    Winds: rho_w = |x - s1|^-2 + |x - s2|^-2 (floored at 0.05), stars
    s1 = (-0.8, 0, 0), s2 = (0.8, 0.1, 0). Cones: apex (-0.5, 0, 0) axis +x and
    apex (0.5, 0.1, 0) axis -x, half-angle 30 deg; shell of thickness 0.04 at
    4x density and T = 10^7.5 K, interior 0.25x; elsewhere T = 10^4 K.
    Clumps: centres uniform in [-0.8, 0.8]^3, radii log-uniform in r_range,
    density contrast log-uniform in `contrast`, T = 10^5 K inside. Every cell
    carries lognormal clumping exp(0.3 z - 0.045), z ~ N(0,1) per cell.

    Refinement (factor 2 per level, `levels` levels): a brick is refined while
    it intersects a clump of radius r and its edge exceeds clump_factor * r;
    bricks within a half-diagonal + thickness/2 of a cone surface are refined
    below level cone_levels (0: the cones stay at the base resolution, where
    the shell is 10 base cells thick at n_base 512). Fields are FP32, sampled
    at the cell centres of each leaf brick at its own level; the per-cell
    normals come from one PCG64 stream per chunk of 2^21 cells, spawned from
    SeedSequence([seed, 1]), so the fields do not depend on how the chunks are
    scheduled over threads."""
    assert n_base % brick == 0
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = -1.0, 1.0
    nf = n_base << levels
    hf = (hi - lo) / nf
    half_angle = math.radians(half_angle_deg)
    cr = np.exp(rng.uniform(math.log(r_range[0]), math.log(r_range[1]), n_clumps))
    cc = rng.uniform(-0.8, 0.8, size=(n_clumps, 3))
    cf = np.exp(rng.uniform(math.log(contrast[0]), math.log(contrast[1]), n_clumps))
    stars = ((-0.8, 0.0, 0.0), (0.8, 0.1, 0.0))
    cones = (((-0.5, 0.0, 0.0), 1.0), ((0.5, 0.1, 0.0), -1.0))

    def cone_d(px, py, pz, apex, sgn):
        a = sgn * (px - apex[0])
        r = np.sqrt((py - apex[1]) ** 2 + (pz - apex[2]) ** 2)
        ct, st = math.cos(half_angle), math.sin(half_angle)
        on = a * ct + r * st >= 0.0
        d = np.where(on, r * ct - a * st, np.sqrt(a * a + r * r))
        return d, on

    nb0 = n_base // brick
    g = np.arange(nb0)
    bz, by, bx = np.meshgrid(g, g, g, indexing="ij")
    cur = np.stack([bx.ravel(), by.ravel(), bz.ravel()], axis=1).astype(np.int64) * (brick << levels)
    leaf_levels, leaf_origins = [], []
    for lev in range(levels + 1):
        S = brick << (levels - lev)
        size = S * hf
        ref = np.zeros(len(cur), dtype=bool)
        if lev < levels and len(cur):
            blo = lo + cur * hf
            bhi = blo + size
            for k in range(n_clumps):
                if size > clump_factor * cr[k]:
                    q = np.clip(cc[k], blo, bhi)
                    ref |= ((q - cc[k]) ** 2).sum(axis=1) <= cr[k] ** 2
            if lev < cone_levels:
                ctr = blo + size / 2
                for apex, sgn in cones:
                    d, _ = cone_d(ctr[:, 0], ctr[:, 1], ctr[:, 2], apex, sgn)
                    ref |= np.abs(d) <= math.sqrt(3.0) * size / 2 + thickness / 2
        keep = cur[~ref]
        leaf_levels.append(np.full(len(keep), lev, dtype=np.int32))
        leaf_origins.append(keep)
        rr = cur[ref]
        h = S // 2
        kids = [rr + np.array([dx * h, dy * h, dz * h], dtype=np.int64)
                for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
        cur = np.concatenate(kids, axis=0) if len(rr) else np.zeros((0, 3), np.int64)
        if len(cur):
            cur = cur[np.lexsort((cur[:, 0], cur[:, 1], cur[:, 2]))]
    levels_arr = np.concatenate(leaf_levels)
    origins = np.concatenate(leaf_origins, axis=0)
    nb = len(levels_arr)

    rho = np.empty((nb, brick, brick, brick), dtype=np.float32)
    temp = np.empty((nb, brick, brick, brick), dtype=np.float32)
    off = (np.arange(brick) + 0.5).astype(np.float64)
    ct, st = math.cos(half_angle), math.sin(half_angle)
    f32 = np.float32
    chunk = max(1, (1 << 21) // brick ** 3)
    starts = list(range(0, nb, chunk))
    streams = np.random.SeedSequence([seed, 1]).spawn(len(starts))

    def fill(ci):
        c0 = starts[ci]
        sel = np.arange(c0, min(nb, c0 + chunk))
        m = len(sel)
        step = (1 << (levels - levels_arr[sel])).astype(np.float64)
        o = origins[sel].astype(np.float64)
        # cell-centre coordinates per axis, [m, B] (float32 after the FP64 sum)
        cx = (lo + (o[:, 0:1] + off[None, :] * step[:, None]) * hf).astype(f32)
        cy = (lo + (o[:, 1:2] + off[None, :] * step[:, None]) * hf).astype(f32)
        cz = (lo + (o[:, 2:3] + off[None, :] * step[:, None]) * hf).astype(f32)
        X = cx[:, None, None, :]
        Y = cy[:, None, :, None]
        Z = cz[:, :, None, None]
        rho_w = np.zeros((m, brick, brick, brick), dtype=f32)
        for s_ in stars:
            ryz2 = (Y - f32(s_[1])) ** 2 + (Z - f32(s_[2])) ** 2            # [m, B, B, 1]
            rw = np.sqrt((X - f32(s_[0])) ** 2 + ryz2)
            rho_w += np.maximum(rw, f32(0.05)) ** -2
        fac = np.ones_like(rho_w)
        tv = np.full(rho_w.shape, f32(1e4))
        for apex, sgn in cones:
            a = f32(sgn) * (X - f32(apex[0]))                                # [m, 1, 1, B]
            r = np.sqrt((Y - f32(apex[1])) ** 2 + (Z - f32(apex[2])) ** 2)  # [m, B, B, 1]
            on = a * f32(ct) + r * f32(st) >= 0
            d = np.where(on, r * f32(ct) - a * f32(st), np.sqrt(a * a + r * r))
            shell = (np.abs(d) <= f32(thickness / 2)) & on
            inside = (d < f32(-thickness / 2)) & on
            fac = np.where(shell, fac * f32(4.0), np.where(inside, fac * f32(0.25), fac))
            tv = np.where(shell, f32(10.0 ** 7.5), tv)
        # clumps: only those whose sphere meets a brick of this chunk
        h = 0.5 * step[:, None] * hf
        blo = np.stack([cx[:, 0], cy[:, 0], cz[:, 0]], axis=1) - h
        bhi = blo + brick * step[:, None] * hf
        for k in range(n_clumps):
            q = np.clip(cc[k], blo, bhi)
            hit = np.nonzero(((q - cc[k]) ** 2).sum(axis=1) <= cr[k] ** 2)[0]
            if len(hit) == 0:
                continue
            ck = cc[k].astype(f32)
            r2 = (X[hit] - ck[0]) ** 2 + (Y[hit] - ck[1]) ** 2 + (Z[hit] - ck[2]) ** 2
            inn = r2 <= f32(cr[k] ** 2)
            fac[hit] = np.where(inn, fac[hit] * f32(cf[k]), fac[hit])
            tv[hit] = np.where(inn, f32(1e5), tv[hit])
        zr = np.random.Generator(np.random.PCG64(streams[ci]))
        z = zr.standard_normal(m * brick ** 3, dtype=np.float32).reshape(rho_w.shape)
        clump = np.exp(f32(clump_sigma) * z - f32(0.5 * clump_sigma ** 2))
        rho[sel] = rho_w * fac * clump
        temp[sel] = tv

    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(fill, range(len(starts))))

    edges = band_edges(n_bands, e_lo, e_hi)
    return Scene(kind="amr", lo=(lo,) * 3, hi=(hi,) * 3, n=(n_base,) * 3, rho=rho, temp=temp,
                 brick=brick, max_level=levels, brick_level=levels_arr,
                 brick_origin=origins.astype(np.int32), emis_mode=1,
                 lambda_table=cooling_table(edges, n_tbins), logT_lo=4.0, logT_hi=9.0,
                 kappa=band_kappa(edges, kappa0),
                 name=f"clumps_cones_{n_base}^3_b{brick}_L{levels}_{n_clumps}cl_{n_bands}band_s{seed}")


def reseed(scene: Scene, seed: int) -> Scene:
    """The same cone-shock grid with the per-cell clumping redrawn from `seed`
    (equal to cone_shock_amr(seed, ...) with the same other arguments, whose
    brick layout draws no random numbers). Needs a scene made with
    keep_smooth=True and clump_scale=0."""
    import copy
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal(scene.rho_smooth.size).reshape(scene.rho_smooth.shape)
    sig = scene.clump_sigma
    out = copy.copy(scene)
    out.rho = (scene.rho_smooth * np.exp(sig * z - 0.5 * sig ** 2)).astype(np.float32)
    out.name = scene.name.rsplit("_s", 1)[0] + f"_s{seed}"
    return out


# --------------------------------------------------------------------------
# Small analytic scenes used by the closed-form pins
# --------------------------------------------------------------------------
def uniform_from_array(rho: np.ndarray, lo=(-1.0,) * 3, hi=(1.0,) * 3, kappa=0.0,
                       temp: np.ndarray | None = None, lambda_table=None,
                       logT_lo: float = 4.0, logT_hi: float = 9.0) -> Scene:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    kap = np.atleast_1d(np.asarray(kappa, dtype=np.float64))
    return Scene(kind="uniform", lo=tuple(lo), hi=tuple(hi), n=(nx, ny, nz), rho=rho,
                 temp=None if temp is None else np.ascontiguousarray(temp, np.float64),
                 emis_mode=0 if lambda_table is None else 1,
                 lambda_table=lambda_table, logT_lo=logT_lo, logT_hi=logT_hi, kappa=kap,
                 name="array")


def uniform_sphere(n: int, radius: float = 0.6, rho0: float = 1.0) -> Scene:
    """rho0 inside |x| < radius (cell-centre test), 0 outside, on [-1,1]^3."""
    c = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    rho = np.where(x * x + y * y + z * z < radius * radius, rho0, 0.0)
    return uniform_from_array(rho)


def random_uniform(seed: int, n=(8, 8, 8), kappa=0.5, with_temp: bool = False,
                   n_bands: int = 1) -> Scene:
    """Lognormal random field on a small uniform grid (brute-force pins)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = n
    rho = np.exp(0.5 * rng.standard_normal((nz, ny, nx)))
    if not with_temp:
        return uniform_from_array(rho, kappa=kappa)
    temp = 10.0 ** rng.uniform(6.0, 8.5, size=(nz, ny, nx))
    edges = band_edges(n_bands, 0.5, 10.0)
    return uniform_from_array(rho, kappa=band_kappa(edges, kappa), temp=temp,
                              lambda_table=cooling_table(edges))


def as_amr_single_level(scene: Scene, brick: int) -> Scene:
    """Re-express a uniform scene as a block-AMR grid with one level of bricks
    (pure re-layout of the same cell values)."""
    nx, ny, nz = scene.n
    assert nx % brick == 0 and ny % brick == 0 and nz % brick == 0
    bx, by, bz = nx // brick, ny // brick, nz // brick
    r = scene.rho.reshape(bz, brick, by, brick, bx, brick).transpose(0, 2, 4, 1, 3, 5)
    rho = np.ascontiguousarray(r.reshape(-1, brick, brick, brick))
    temp = None
    if scene.temp is not None:
        t = scene.temp.reshape(bz, brick, by, brick, bx, brick).transpose(0, 2, 4, 1, 3, 5)
        temp = np.ascontiguousarray(t.reshape(-1, brick, brick, brick))
    gz, gy, gx = np.meshgrid(np.arange(bz), np.arange(by), np.arange(bx), indexing="ij")
    origins = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1).astype(np.int32) * brick
    return Scene(kind="amr", lo=scene.lo, hi=scene.hi, n=scene.n, rho=rho, temp=temp,
                 brick=brick, max_level=0, brick_level=np.zeros(len(origins), np.int32),
                 brick_origin=origins, emis_mode=scene.emis_mode,
                 lambda_table=scene.lambda_table, logT_lo=scene.logT_lo,
                 logT_hi=scene.logT_hi, kappa=scene.kappa, name=scene.name + "_as_amr")


def refine_uniform_to_amr(scene: Scene, brick: int, refine_mask_fn, seed: int = 0) -> Scene:
    """One extra level: bricks for which refine_mask_fn(brick_centre) is true are
    split into 8 children whose cells copy the parent cell value (piecewise
    constant prolongation) times an independent lognormal factor, so the finer
    cells carry new information. Used for small mixed-level pins."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = as_amr_single_level(scene, brick)
    hf = (scene.hi[0] - scene.lo[0]) / (scene.n[0] * 2)
    levels, origins, rhos = [], [], []
    for b in range(len(base.brick_level)):
        o = base.brick_origin[b].astype(np.int64) * 2  # finest units (1 extra level)
        ctr = np.array(scene.lo) + (o + brick) * hf
        if refine_mask_fn(ctr):
            parent = base.rho[b]
            fine = np.repeat(np.repeat(np.repeat(parent, 2, 0), 2, 1), 2, 2)
            fine = fine * np.exp(0.2 * rng.standard_normal(fine.shape))
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        levels.append(1)
                        origins.append(o + np.array([dx, dy, dz]) * brick)
                        rhos.append(fine[dz * brick:(dz + 1) * brick, dy * brick:(dy + 1) * brick,
                                         dx * brick:(dx + 1) * brick])
        else:
            levels.append(0)
            origins.append(o)
            rhos.append(base.rho[b])
    return Scene(kind="amr", lo=scene.lo, hi=scene.hi, n=scene.n,
                 rho=np.ascontiguousarray(np.stack(rhos)), brick=brick, max_level=1,
                 brick_level=np.array(levels, np.int32),
                 brick_origin=np.array(origins, np.int32), emis_mode=0, kappa=scene.kappa,
                 name=scene.name + "_amr2")


# --------------------------------------------------------------------------
# The paper's test problem (Section 3, Eq. 3): a hot ring on a block-AMR grid
# --------------------------------------------------------------------------
RING_LENGTH_UNIT_CM = 1e17
RING_DENSITY_UNIT = 1e-26  # g cm^-3


def _ring_boundary_distance(x, r, half_w, r_in, r_out):
    """Distance from points (|x|, r) to the boundary of the ring's cross-section
    rectangle [-half_w, half_w] x [r_in, r_out] in the (x, r) half-plane."""
    ax = np.abs(x)
    inside = (ax <= half_w) & (r >= r_in) & (r <= r_out)
    dx_out = np.maximum(ax - half_w, 0.0)
    dr_out = np.maximum(np.maximum(r_in - r, r - r_out), 0.0)
    d_out = np.hypot(dx_out, dr_out)
    d_in = np.minimum(np.minimum(half_w - ax, r - r_in), r_out - r)
    return np.where(inside, d_in, d_out), inside


def ring_amr(n_base: int = 32, brick: int = 8, levels: int = 4, beta_g_per_cm: float = 2.5e9,
             rho_out_gcc: float = 1e-25, T_in: float = 1e8, T_out: float = 1e4,
             e_lo: float = 1.0, e_hi: float = 10.0, n_tbins: int = 64) -> Scene:
    """Section 3's test problem on a PARAMESH-like grid: a ring in the yz-plane
    (thickness 1e17 cm, |x| < w/2; inner and outer radii 3.5e17 and 4e17 cm) in
    a box of +-5e17 cm; rho = beta r_yz^-2 in the ring (Eq. 3) and 1e-25 g cm^-3
    elsewhere; T = 1e8 K in the ring, 1e4 K elsewhere. 4^3 base bricks of 8^3
    cells, 4 nested levels (512^3 effective) on bricks the ring's surface passes
    through, as a density/temperature refinement would place them. Emission in
    the 1-10 keV band from the bremsstrahlung-shaped table; optically thin.

    Units: lengths in 1e17 cm, density in 1e-26 g cm^-3 (so FP32 rho^2 stays
    normal). beta = 2.5e9 g cm^-1 (the printed 2.5e-9 would make the ring 1e19
    times less dense than its surroundings and its flux ~1e-55 instead of the
    quoted 1.4e-19 erg s^-1 cm^-2)."""
    L = RING_LENGTH_UNIT_CM
    half_w, r_in, r_out = 0.5e17 / L, 3.5e17 / L, 4e17 / L
    lo, hi = -5e17 / L, 5e17 / L
    nf = n_base << levels
    hf = (hi - lo) / nf
    nb0 = n_base // brick
    g = np.arange(nb0)
    bz, by, bx = np.meshgrid(g, g, g, indexing="ij")
    S0 = brick << levels
    cur = np.stack([bx.ravel(), by.ravel(), bz.ravel()], axis=1).astype(np.int64) * S0
    leaf_levels, leaf_origins = [], []
    for lev in range(levels + 1):
        S = brick << (levels - lev)
        ctr = lo + (cur + S / 2.0) * hf
        rr = np.hypot(ctr[:, 1], ctr[:, 2])
        d, _ = _ring_boundary_distance(ctr[:, 0], rr, half_w, r_in, r_out)
        refine = (d <= math.sqrt(3.0) * 0.5 * S * hf) if lev < levels else np.zeros(len(cur), bool)
        leaf_levels.append(np.full(int((~refine).sum()), lev, dtype=np.int32))
        leaf_origins.append(cur[~refine])
        ref = cur[refine]
        h = S // 2
        kids = [ref + np.array([dx * h, dy * h, dz * h]) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
        cur = np.concatenate(kids) if len(ref) else np.zeros((0, 3), np.int64)
    levels_arr = np.concatenate(leaf_levels)
    origins = np.concatenate(leaf_origins, axis=0)
    nb = len(levels_arr)
    off = np.arange(brick) + 0.5
    rho = np.empty((nb, brick, brick, brick), np.float32)
    temp = np.empty((nb, brick, brick, brick), np.float32)
    for lev in range(levels + 1):
        sel = np.nonzero(levels_arr == lev)[0]
        if not len(sel):
            continue
        step = 1 << (levels - lev)
        o = origins[sel].astype(np.float64)
        cx = lo + (o[:, 0:1] + off[None, :] * step) * hf
        cy = lo + (o[:, 1:2] + off[None, :] * step) * hf
        cz = lo + (o[:, 2:3] + off[None, :] * step) * hf
        shp = (len(sel), brick, brick, brick)
        PX = np.broadcast_to(cx[:, None, None, :], shp)
        PY = np.broadcast_to(cy[:, None, :, None], shp)
        PZ = np.broadcast_to(cz[:, :, None, None], shp)
        r = np.hypot(PY, PZ)
        inside = (np.abs(PX) < half_w) & (r >= r_in) & (r <= r_out)
        rho_in = beta_g_per_cm / (r * L) ** 2 / RING_DENSITY_UNIT
        rho[sel] = np.where(inside, rho_in, rho_out_gcc / RING_DENSITY_UNIT).astype(np.float32)
        temp[sel] = np.where(inside, T_in, T_out).astype(np.float32)
    edges = band_edges(1, e_lo, e_hi)
    return Scene(kind="amr", lo=(lo,) * 3, hi=(hi,) * 3, n=(n_base,) * 3, rho=rho, temp=temp,
                 brick=brick, max_level=levels, brick_level=levels_arr,
                 brick_origin=origins.astype(np.int32), emis_mode=1,
                 lambda_table=cooling_table(edges, n_tbins), logT_lo=4.0, logT_hi=9.0,
                 kappa=np.zeros(1), name=f"ring_{n_base}^3_b{brick}_L{levels}")


def ring_view() -> View:
    """Face-on view along +x with (u, v) = (y, z) (the paper's Fig. 1)."""
    return View(dir=(1.0, 0.0, 0.0), up=(0.0, 0.0, 1.0), half_extent=5e17 / RING_LENGTH_UNIT_CM)


# ---------------------------------------------------------------------------
# Initial weights of the refinement-depth network (an input to both the GPU
# library and the FP64 network reference; no arithmetic of the method)
MLP_SHAPES = [("W1", (16, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
              ("W3", (64, 5)), ("b3", (5,))]


def mlp_init(seed: int, scale: float = 1.0) -> np.ndarray:
    """He-style random initial parameters (weights N(0, 2 / fan_in) x scale,
    biases zero) as one flat FP64 vector in the library's parameter order
    W1[16][64], b1, W2[64][64], b2, W3[64][5], b3 (input index first)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for name, shp in MLP_SHAPES:
        if name.startswith("W"):
            parts.append((rng.standard_normal(shp) * scale * np.sqrt(2.0 / shp[0])).ravel())
        else:
            parts.append(np.zeros(int(np.prod(shp))))
    return np.concatenate(parts)
