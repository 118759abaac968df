"""Host-side checks of the index bounds the Radon kernels rely on, restated
in numpy from the parallel-beam Joseph geometry (float64 split tables,
float32 device arithmetic emulated with numpy float32):

* the adjoint stages AWIN = 32 bins per angle and tile, starting at a window
  computed from the tile corners; every bin whose sample lands on a line of
  the tile (positions p0 - 1 .. p0 + 15) must lie in the per-line range the
  kernel walks, and that range inside the staged window -- a bin outside it
  would be dropped silently;
* the forward loops, per warp of 96 bins, only over the lines between two
  bounds; every sample on a line outside them must be out of range.
"""
import math

import numpy as np
import pytest

F = np.float32
ATS, AWIN = 16, 32


def split(v):
    fl = np.floor(v)
    f = (v - fl).astype(F)
    up = f >= F(1)
    f = np.where(up, F(0), f)
    return (fl + up).astype(np.int64), f


def tables(n1, n2, A, B, span=math.pi):
    c1, c2, cb = (n1 - 1) / 2.0, (n2 - 1) / 2.0, (B - 1) / 2.0
    out = []
    for k in range(A):
        th = k * (span / A)
        cs, sn = math.cos(th), math.sin(th)
        rs = abs(cs) + 1e-9 >= abs(sn)
        c_line, c_pos = (c1, c2) if rs else (c2, c1)
        den, oth = (cs, sn) if rs else (sn, cs)
        qi, qf = split(c_pos + (np.arange(B) - cb) / den)
        nl = n1 if rs else n2
        ri, rf = split(-(np.arange(nl) - c_line) * oth / den)
        out.append(dict(rs=rs, sl=F(den), ot=F(oth), tl=F(oth) / F(den), qi=qi, qf=qf, ri=ri, rf=rf, nl=nl,
                        na=n2 if rs else n1, c_line=F(0.5) * F(nl - 1)))
    return out, F(c1), F(c2), F(cb)


def sample_lo(qi, qf, ri, rf):
    f = (qf + rf).astype(F)
    carry = (f >= F(1)).astype(np.int64)
    return qi + ri + carry


def window(t, i0, j0, c1, c2, cb):
    pa = F(j0 if t["rs"] else i0) - (c2 if t["rs"] else c1)
    la = F(i0 if t["rs"] else j0) - (c1 if t["rs"] else c2)
    sl, ot = t["sl"], t["ot"]
    mp = min(sl * (pa - F(1)), sl * (pa + F(ATS)))
    ml = min(ot * la, ot * (la + F(ATS - 1)))
    return int(np.floor(cb + mp + ml)) - 4


@pytest.mark.parametrize("n,A,B,tiles", [(64, 90, 100, None), (37, 7, 61, None), (512, 720, 736, 48)])
def test_adjoint_bins_inside_staged_window(n, A, B, tiles):
    tab, c1, c2, cb = tables(n, n, A, B)
    nt = (n + ATS - 1) // ATS
    rng = np.random.default_rng(0)
    all_tiles = [(ty, tx) for ty in range(nt) for tx in range(nt)]
    if tiles is not None:
        pick = rng.choice(len(all_tiles), tiles, replace=False)
        all_tiles = [all_tiles[p] for p in pick] + [(0, 0), (nt - 1, nt - 1), (0, nt - 1)]
    m_all = np.arange(B)
    worst = 0
    for ty, tx in all_tiles:
        i0, j0 = ty * ATS, tx * ATS
        for t in tab:
            wlo = window(t, i0, j0, c1, c2, cb)
            p0 = j0 if t["rs"] else i0
            cpos = c2 if t["rs"] else c1
            for r in range(ATS):
                l = (i0 if t["rs"] else j0) + r
                if l >= t["nl"]:
                    continue
                ri, rf = t["ri"][l], t["rf"][l]
                base = cb - t["sl"] * (cpos + (F(ri) + rf))
                ma, mb = base + t["sl"] * F(p0 - 1), base + t["sl"] * F(p0 + ATS)
                mlo = max(0, int(np.floor(min(ma, mb))) - 1)
                mhi = min(B - 1, int(np.ceil(max(ma, mb))) + 1)
                lo = sample_lo(t["qi"], t["qf"], ri, rf)
                hit = m_all[(lo - p0 >= -1) & (lo - p0 < ATS)]
                if hit.size:
                    assert hit.min() >= mlo and hit.max() <= mhi, (ty, tx, l)
                    assert mlo >= wlo and hit.max() < wlo + AWIN, (ty, tx, l, mlo, wlo)
                    worst = max(worst, mhi - wlo)
    assert worst < AWIN


@pytest.mark.parametrize("n,A,B", [(64, 90, 100), (512, 720, 736), (37, 7, 61)])
def test_forward_line_range_covers_every_sample(n, A, B):
    tab, c1, c2, cb = tables(n, n, A, B)
    for t in tab:
        nl, na = t["nl"], t["na"]
        Q = (t["qi"].astype(F) + t["qf"]).astype(F)
        lo = sample_lo(t["qi"][:, None], t["qf"][:, None], t["ri"][None, :], t["rf"][None, :])
        inside = (lo >= -1) & (lo <= na - 1)          # some weight lands on the line
        for base in range(0, B, 96):
            mf, ml = base, min(base + 95, B - 1)
            qmin, qmax = min(Q[mf], Q[ml]), max(Q[mf], Q[ml])
            l_beg, l_end = 0, nl
            if abs(t["tl"]) > F(1e-6):
                e1 = t["c_line"] + (qmin - F(na)) / t["tl"]
                e2 = t["c_line"] + (qmax + F(1)) / t["tl"]
                l_beg = max(0, int(np.floor(min(e1, e2))) - 2)
                l_end = min(nl, int(np.ceil(max(e1, e2))) + 3)
            elif qmax < F(-3) or qmin > F(na + 2):
                l_end = 0
            rows = inside[mf:ml + 1]
            outside = np.ones(nl, bool)
            outside[l_beg:l_end] = False
            assert not rows[:, outside].any(), (base, l_beg, l_end)
