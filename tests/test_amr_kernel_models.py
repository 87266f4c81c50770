"""Host models of the index arithmetic of two AMR kernels (1D-3D, leaves of 8 and 16 cells):

* `ghost_fill_kernel` (one CTA per slab): every load of a restriction or prolongation slab
  stays inside its source leaf, vector loads and stores start at aligned offsets, and every
  ghost value of the slab is written exactly once;
* `reflux_kernel` (one thread per record, variable and tangential cell): for any set of faces
  of one coarse leaf with level jumps, every (face, cell) correction is applied exactly once,
  each cell by one thread, in the order x, y, z;
* the float32 march kernel's last-stage totals: the per-warp float-float butterfly leaves every
  lane with the same bits, and the CTA's total is the exact sum to float-float accuracy.
"""
import itertools

import numpy as np
import pytest


def face_dims(nd, d):
    e1 = -1 if nd < 2 else (1 if d == 0 else 0)
    e2 = -1 if nd < 3 else (1 if d == 2 else 2)
    return e1, e2


def face_cell(nd, B, d, n, a1, a2):
    e1, e2 = face_dims(nd, d)
    x = [0, 0, 0]
    x[d] = n
    if e1 >= 0:
        x[e1] = a1
    if e2 >= 0:
        x[e2] = a2
    assert all(0 <= x[e] < B for e in range(3)), x
    return x[0] + B * (x[1] + B * x[2])


@pytest.mark.parametrize("nd,B", [(1, 8), (1, 16), (2, 8), (2, 16), (3, 8), (3, 16)])
def test_ghost_fill_indices(nd, B):
    NV, HB = nd + 2, B // 2
    NT = 1 if nd == 1 else (B if nd == 2 else B * B)
    NCC = 1 if nd == 1 else (HB if nd == 2 else HB * HB)
    NTH = (NCC * NV + 31) // 32 * 32
    for d in range(nd):
        e1, e2 = face_dims(nd, d)
        NA, NB = (2 if e1 >= 0 else 1), (2 if e2 >= 0 else 1)
        for side in (0, 1):
            written = set()  # restriction slab
            for tid in range(NTH):
                for i in range((NT * NV + NTH - 1) // NTH):
                    q = tid + i * NTH
                    if q >= NT * NV:
                        continue
                    t, v = q % NT, q // NT
                    t1, t2 = (t % B if e1 >= 0 else 0), (t // B if e2 >= 0 else 0)
                    q1, q2 = t1 // HB, t2 // HB
                    f1, f2 = 2 * t1 - q1 * B, 2 * t2 - q2 * B
                    n0 = B - 4 if side == 0 else 0
                    if d == 0:
                        for b_ in range(NB):
                            for a in range(NA):
                                assert face_cell(nd, B, d, n0, f1 + a, f2 + b_) % 4 == 0
                    else:
                        for k in range(4):
                            for b_ in range(NB):
                                assert face_cell(nd, B, d, n0 + k, f1, f2 + b_) % 2 == 0
                                face_cell(nd, B, d, n0 + k, f1 + 1, f2 + b_)
                    for m in (0, 1):
                        o = (v * 2 + m) * NT + t
                        assert o not in written
                        written.add(o)
            assert len(written) == NV * 2 * NT
            offs = itertools.product(range(0, B, HB) if e1 >= 0 else [0], range(0, B, HB) if e2 >= 0 else [0])
            for off in offs:  # prolongation slab at every tangential offset in the coarse face
                written = set()
                for q in range(min(NTH, NCC * NV)):
                    qc, v = q % NCC, q // NCC
                    c1, c2 = (qc % HB if e1 >= 0 else 0), (qc // HB if e2 >= 0 else 0)
                    p1, p2, pn = off[0] + c1, off[1] + c2, (B - 1 if side == 0 else 0)
                    face_cell(nd, B, d, pn, p1, p2)
                    face_cell(nd, B, d, pn - 1 if side == 0 else pn + 1, p1, p2)
                    fn = 0 if side == 0 else B - 2
                    for k in range(2 if d else 1):
                        for b_ in range(NB):
                            for a in range(NA if d == 0 else 1):
                                cell = face_cell(nd, B, d, fn + k, 2 * c1 + a, 2 * c2 + b_)
                                assert cell % 2 == 0
                    if e1 >= 0 and 1 <= p1 < B - 1:
                        face_cell(nd, B, d, pn, p1 - 1, p2), face_cell(nd, B, d, pn, p1 + 1, p2)
                    if e2 >= 0 and 1 <= p2 < B - 1:
                        face_cell(nd, B, d, pn, p1, p2 - 1), face_cell(nd, B, d, pn, p1, p2 + 1)
                    for m in (0, 1):
                        for b_ in range(NB):
                            for a in range(NA):
                                t = (2 * c1 + a) + B * (2 * c2 + b_) if nd >= 2 else 0
                                assert 0 <= t < NT and (NA == 1 or a == 1 or t % 2 == 0)
                                o = (v * 2 + m) * NT + t
                                assert o not in written
                                written.add(o)
                assert len(written) == NV * 2 * NT


def compose_cell(nd, B, d, n, t):
    if nd == 1:
        return n
    if nd == 2:
        return n + B * t if d == 0 else t + B * n
    t1, t2 = t % B, t // B
    return [n + B * (t1 + B * t2), t1 + B * (n + B * t2), t1 + B * (t2 + B * n)][d]


@pytest.mark.parametrize("nd,B", [(1, 8), (2, 8), (2, 16), (3, 8), (3, 16)])
def test_reflux_single_writer_in_face_order(nd, B):
    NT = 1 if nd == 1 else (B if nd == 2 else B * B)
    for mask in range(1, 1 << (2 * nd)):
        faces = [f for f in range(2 * nd) if mask >> f & 1]  # the group's records, faces ascending
        writers, applied = {}, {}
        for r, f in enumerate(faces):
            for t in range(NT):
                cell = compose_cell(nd, B, f >> 1, B - 1 if f & 1 else 0, t)
                x = [cell % B, (cell // B) % B if nd > 1 else 0, cell // (B * B) if nd > 2 else 0]

                def touches(g):
                    return x[g >> 1] == (B - 1 if g & 1 else 0)

                if any(touches(faces[k]) for k in range(r)):
                    continue
                assert cell not in writers
                writers[cell] = r
                seq = []
                for k in range(r, len(faces)):
                    g = faces[k]
                    if k > r and not touches(g):
                        continue
                    dk = g >> 1
                    tk = 0 if nd == 1 else (x[1 if dk == 0 else 0] if nd == 2 else
                                            [x[1] + B * x[2], x[0] + B * x[2], x[0] + B * x[1]][dk])
                    assert compose_cell(nd, B, dk, B - 1 if g & 1 else 0, tk) == cell
                    seq.append(g)
                applied[cell] = seq
        pairs = set()
        for cell, seq in applied.items():
            assert seq == sorted(seq)
            for g in seq:
                assert (g, cell) not in pairs
                pairs.add((g, cell))
        assert len(pairs) == len(faces) * NT


def ff_add(hi, lo, h2, l2):
    """float-float add of the kernel (TwoSum of the high parts, low parts added), in float32."""
    f = np.float32
    s = f(hi + h2)
    bb = f(s - hi)
    e = f(f(hi - f(s - bb)) + f(h2 - bb))
    return s, f(f(lo + l2) + e)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_last_stage_totals_butterfly(seed):
    rng = np.random.default_rng(seed)
    f = np.float32
    nwarps, cells = 4, 13  # 4 warps of the last stage's CTA; ~13 cells per thread (8 per leaf, 1.68 leaves)
    # per thread: TwoSum accumulation of its cells (scaled conserved values of mixed sign)
    vals = (rng.normal(size=(nwarps * 32, cells)) * 10.0 ** rng.integers(-2, 3, size=(nwarps * 32, cells))).astype(f)
    hi = np.zeros(nwarps * 32, dtype=f)
    lo = np.zeros(nwarps * 32, dtype=f)
    for t in range(nwarps * 32):
        for x in vals[t]:
            hi[t], lo[t] = ff_add(hi[t], lo[t], x, f(0))
    # per warp: butterfly over lane ^ o, o = 16 .. 1; both partners of an exchange compute it
    wh, wl = [], []
    for w in range(nwarps):
        h = hi[32 * w:32 * w + 32].copy()
        l = lo[32 * w:32 * w + 32].copy()
        for o in (16, 8, 4, 2, 1):
            nh, nl = h.copy(), l.copy()
            for lane in range(32):
                nh[lane], nl[lane] = ff_add(h[lane], l[lane], h[lane ^ o], l[lane ^ o])
            h, l = nh, nl
        assert np.all(h == h[0]) and np.all(l == l[0])  # every lane holds the same bits
        wh.append(h[0])
        wl.append(l[0])
    hh, ll = wh[0], wl[0]
    for w in range(1, nwarps):  # the warps in order
        hh, ll = ff_add(hh, ll, wh[w], wl[w])
    exact = float(np.sum(vals.astype(np.float64), dtype=np.float64))
    scale = float(np.sum(np.abs(vals.astype(np.float64))))
    assert abs((float(hh) + float(ll)) - exact) <= 2.0 ** -40 * scale
