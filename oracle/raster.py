"""Finest-level raster of an adaptive image: plain numpy, FP64.

Test infrastructure, like the rest of oracle/: only tests/, the smoke check
and bench.py's CPU baseline use it; the library does not.

Section 2 step vi lets the output image be sharpened by interpolating between
adjacent pixels of differing resolution (a super-resolution step, citing Chu
2009, with no method fixed). The reading used here, for an image of base
n0^2 pixels refined to max_level Lm, on the raster of (n0 2^Lm)^2 finest
pixels:

* nearest: each finest pixel takes the value of the leaf that covers it;
* bilinear: with L the level of that leaf, the finest pixel's centre is
  placed on the level-L pixel grid, u = (x + 1/2) 2^(L - Lm) - 1/2 (and v
  likewise), and the value is the bilinear interpolation between the four
  level-L pixels (floor(u) + {0, 1}, floor(v) + {0, 1}), indices clamped to
  the image. The value of a level-L pixel is that of the deepest existing
  node at level <= L covering it, the neighbour rule of the refinement scan
  (every traced node keeps its value, interior ones included). A finest-level
  leaf therefore keeps its own value exactly, and the raster is continuous
  across coarse leaves of one level."""
import numpy as np


def level_maps(level, i, j, value, n0, Lm):
    """Per level L, the value of the deepest existing node at level <= L over
    every level-L pixel ([n0 2^L, n0 2^L], index [j, i]), and the level of
    that node."""
    level = np.asarray(level)
    i = np.asarray(i)
    j = np.asarray(j)
    value = np.asarray(value, dtype=np.float64)
    filled, deep = [], []
    for L in range(Lm + 1):
        nl = n0 << L
        m = np.full((nl, nl), np.nan)
        d = np.full((nl, nl), -1, dtype=np.int64)
        sel = level == L
        m[j[sel], i[sel]] = value[sel]
        d[j[sel], i[sel]] = L
        if L > 0:
            up = np.repeat(np.repeat(filled[L - 1], 2, axis=0), 2, axis=1)
            upd = np.repeat(np.repeat(deep[L - 1], 2, axis=0), 2, axis=1)
            miss = np.isnan(m)
            m[miss] = up[miss]
            d[miss] = upd[miss]
        assert not np.isnan(m).any(), "the base image must be complete"
        filled.append(m)
        deep.append(d)
    return filled, deep


def raster(level, i, j, value, n0, Lm, mode="bilinear"):
    """Raster [n0 2^Lm, n0 2^Lm] (index [y, x]) of one quantity; `level, i, j,
    value` list every traced node of the image in any order."""
    filled, deep = level_maps(level, i, j, value, n0, Lm)
    nf = n0 << Lm
    if mode == "nearest":
        return filled[Lm].copy()
    assert mode == "bilinear"
    leaf_level = deep[Lm]                       # level of the leaf over each finest pixel
    y, x = np.meshgrid(np.arange(nf), np.arange(nf), indexing="ij")
    out = np.empty((nf, nf))
    for L in range(Lm + 1):
        sel = leaf_level == L
        if not sel.any():
            continue
        nl = n0 << L
        s = 2.0 ** (L - Lm)
        u = (x[sel] + 0.5) * s - 0.5
        v = (y[sel] + 0.5) * s - 0.5
        i0 = np.floor(u).astype(np.int64)
        j0 = np.floor(v).astype(np.int64)
        fu = u - i0
        fv = v - j0
        m = filled[L]
        ia, ib = np.clip(i0, 0, nl - 1), np.clip(i0 + 1, 0, nl - 1)
        ja, jb = np.clip(j0, 0, nl - 1), np.clip(j0 + 1, 0, nl - 1)
        out[sel] = ((1 - fu) * (1 - fv) * m[ja, ia] + fu * (1 - fv) * m[ja, ib]
                    + (1 - fu) * fv * m[jb, ia] + fu * fv * m[jb, ib])
    return out
