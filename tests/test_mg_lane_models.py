"""Host models of the lane programs of three 2D multigrid kernels, checked against the plain
definitions they replace (numpy, float32 arithmetic in the kernels' order):

* the red-black strip sweep with a column pair per lane (`sweep2d_kernel`): lanes 0 and 31 are
  halo, each lane holds one red and one black cell per row, the horizontal neighbour of each
  colour comes from the lane beside; it must equal two in-place colour sweeps bit for bit
  (periodic and zero-flux, ragged strips, with and without the zero start);
* the residual-restriction from a 4 x 4 patch (`restrict_cell2d`): equal to the per-child
  form with the neighbour sums of `nbsum`;
* the neighbour selection of the defect update over four consecutive cells (`update64_kernel`):
  the same neighbour values, in the same order, as the strided form.
"""
import numpy as np
import pytest

f32 = np.float32
W = 60  # columns per strip


def colour_sweeps(x, b, n, ih2, idg, neu, idgtab):
    x = x.copy()
    for colour in (0, 1):
        for r in range(n):
            for c in range(n):
                if (c + r) & 1 != colour:
                    continue

                def g(rr, cc):
                    if neu and not (0 <= rr < n and 0 <= cc < n):
                        return f32(0)
                    return x[rr % n, cc % n]

                s = f32(f32(f32(g(r, c - 1) + g(r, c + 1)) + g(r - 1, c)) + g(r + 1, c))
                d = idg if not neu else idgtab[(c == 0) + (c == n - 1) + (r == 0) + (r == n - 1)]
                x[r, c] = f32(f32(b[r, c] + f32(s * ih2)) * d)
    return x


def pair_strip_sweep(x, b, n, H, ih2, idg, neu, idgtab, xzero=False):
    out = np.full((n, n), np.nan, dtype=np.float32)
    lanes = np.arange(32)
    for sy in range((n + H - 1) // H):
        for sx in range((n + W - 1) // W):
            x0, y0 = sx * W, sy * H
            y1 = min(y0 + H, n)
            ca = x0 - 2 + 2 * lanes
            cw = ca % n
            colin = (ca >= 0) & (ca < n)
            out_lane = (lanes >= 1) & (lanes <= 30) & (ca < n)

            def inside(r):
                return np.ones(32, bool) if not neu else (colin & (0 <= r < n))

            def ldx(r):
                if xzero:
                    return np.zeros((32, 2), np.float32)
                v = np.stack([x[r % n, cw], x[r % n, cw + 1]], 1).astype(np.float32)
                v[~inside(r)] = 0
                return v

            def ldb(r):
                return np.stack([b[r % n, cw], b[r % n, cw + 1]], 1).astype(np.float32)

            def idg_at(e, r):
                if not neu:
                    return np.full(32, idg, np.float32)
                c = ca + e
                return idgtab[(c == 0).astype(int) + (c == n - 1) + (r == 0) + (r == n - 1)]

            def up(v):  # lane k gets lane k-1's value
                o = v.copy()
                o[1:] = v[:-1]
                return o

            def down(v):
                o = v.copy()
                o[:-1] = v[1:]
                return o

            def upd(bb, l, rr, m, p, d):
                s = ((l + rr).astype(f32) + m).astype(f32) + p
                return ((bb + (s.astype(f32) * ih2).astype(f32)).astype(f32) * d).astype(f32)

            def red(om, o0, op, bb, r):
                o = o0.copy()
                if (r & 1) == 0:
                    o[:, 0] = upd(bb[:, 0], up(o0[:, 1]), o0[:, 1], om[:, 0], op[:, 0], idg_at(0, r))
                else:
                    o[:, 1] = upd(bb[:, 1], o0[:, 0], down(o0[:, 0]), om[:, 1], op[:, 1], idg_at(1, r))
                o[~inside(r)] = 0
                return o

            oa, ob, oc, od = ldx(y0 - 2), ldx(y0 - 1), ldx(y0), ldx(y0 + 1)
            rm, r0 = red(oa, ob, oc, ldb(y0 - 1), y0 - 1), red(ob, oc, od, ldb(y0), y0)
            b0, os_, os1 = ldb(y0), oc, od
            for s in range(y0, y1):
                os2 = ldx(s + 2)
                bs1 = ldb(s + 1)
                rp = red(os_, os1, os2, bs1, s + 1)
                ov = r0.copy()
                if (s & 1) == 0:
                    ov[:, 1] = upd(b0[:, 1], r0[:, 0], down(r0[:, 0]), rm[:, 1], rp[:, 1], idg_at(1, s))
                else:
                    ov[:, 0] = upd(b0[:, 0], up(r0[:, 1]), r0[:, 1], rm[:, 0], rp[:, 0], idg_at(0, s))
                for k in np.nonzero(out_lane)[0]:
                    assert np.isnan(out[s, ca[k]]) and np.isnan(out[s, ca[k] + 1])
                    out[s, ca[k]], out[s, ca[k] + 1] = ov[k]
                rm, r0, b0, os_, os1 = r0, rp, bs1, os1, os2
    assert not np.isnan(out).any()
    return out


@pytest.mark.parametrize("n,H", [(2, 8), (6, 4), (16, 4), (62, 8), (122, 64), (130, 16)])
@pytest.mark.parametrize("neu", [False, True])
def test_pair_strip_sweep_is_two_colour_sweeps(n, H, neu):
    rng = np.random.default_rng(n + 7 * H)
    ih2, idg = f32(3.7), f32(0.21)
    idgtab = np.array([0.21, 0.23, 0.27, 0.31, 0.37], np.float32)
    for xz in (False, True):
        x = np.zeros((n, n), np.float32) if xz else rng.standard_normal((n, n)).astype(np.float32)
        b = rng.standard_normal((n, n)).astype(np.float32)
        ref = colour_sweeps(x, b, n, ih2, idg, neu, idgtab)
        assert np.array_equal(pair_strip_sweep(x, b, n, H, ih2, idg, neu, idgtab, xzero=xz), ref)


def restrict_generic(x, b, nf, neu, lam, ih2):
    nc = nf // 2
    out = np.zeros((nc, nc))
    for cj in range(nc):
        for ci in range(nc):
            s = 0.0
            for o in range(4):
                fx, fy = 2 * ci + (o & 1), 2 * cj + (o >> 1)
                sn, miss, first = 0.0, 0, True
                for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                    qx, qy = fx + dx, fy + dy
                    if not (0 <= qx < nf and 0 <= qy < nf):
                        if neu:
                            miss += 1
                            continue
                        qx, qy = qx % nf, qy % nf
                    sn = x[qy, qx] if (first and not neu) else sn + x[qy, qx]
                    first = False
                lap = (sn - (4 - miss) * x[fy, fx]) * ih2
                s = s + (b[fy, fx] - (lam * x[fy, fx] - lap))
            out[cj, ci] = s * 0.25
    return out


def restrict_patch(x, b, nf, neu, lam, ih2):
    nc = nf // 2
    out = np.zeros((nc, nc))
    for cj in range(nc):
        for ci in range(nc):
            x0, y0 = 2 * ci, 2 * cj
            col = [x0 - 1 if x0 > 0 else (-1 if neu else nf - 1), x0, x0 + 1, x0 + 2 if x0 + 2 < nf else (-1 if neu else 0)]
            row = [y0 - 1 if y0 > 0 else (-1 if neu else nf - 1), y0, y0 + 1, y0 + 2 if y0 + 2 < nf else (-1 if neu else 0)]
            P = np.zeros((4, 4))
            for r in range(4):
                for c in range(4):
                    if not (r in (0, 3) and c in (0, 3)) and row[r] >= 0 and col[c] >= 0:
                        P[r, c] = x[row[r], col[c]]
            s = 0.0
            for o in range(4):
                r, c = 1 + (o >> 1), 1 + (o & 1)
                miss = 0
                if not neu:
                    sn = P[r, c - 1]
                    sn = sn + P[r, c + 1]
                    sn = sn + P[r - 1, c]
                    sn = sn + P[r + 1, c]
                else:
                    sn = 0.0
                    for ok, v in ((col[c - 1] >= 0, P[r, c - 1]), (col[c + 1] >= 0, P[r, c + 1]),
                                  (row[r - 1] >= 0, P[r - 1, c]), (row[r + 1] >= 0, P[r + 1, c])):
                        if ok:
                            sn = sn + v
                        else:
                            miss += 1
                lap = (sn - (4 - miss) * P[r, c]) * ih2
                s = s + (b[row[r], col[c]] - (lam * P[r, c] - lap))
            out[cj, ci] = s * 0.25
    return out


@pytest.mark.parametrize("nf", [2, 4, 10, 16])
@pytest.mark.parametrize("neu", [False, True])
def test_restriction_patch_matches_per_child_form(nf, neu):
    rng = np.random.default_rng(nf)
    x, b = rng.standard_normal((nf, nf)), rng.standard_normal((nf, nf))
    assert np.array_equal(restrict_patch(x, b, nf, neu, 1.7, 3.3), restrict_generic(x, b, nf, neu, 1.7, 3.3))


def update_neighbours_strided(E, n, neu):
    out = {}
    for t in range(n * n):
        c = [t % n, t // n]
        stride = [1, n]
        nb = []
        for d in range(2):
            for side in (-1, 1):
                if (side < 0 and c[d] == 0) or (side > 0 and c[d] == n - 1):
                    if neu:
                        continue
                    q = t + (n - 1) * stride[d] if side < 0 else t - (n - 1) * stride[d]
                else:
                    q = t + side * stride[d]
                nb.append(E[q])
        out[t] = (E[t], nb)
    return out


def update_neighbours_rows_of_four(E, n, neu):
    out = {}
    for t0 in range(0, n * n, 4):
        r, c0 = t0 // n, t0 % n
        hasdn, hasup, hasl, hasr = r > 0, r + 1 < n, c0 > 0, c0 + 4 < n
        d4 = [0] * 4 if (neu and not hasdn) else list(E[(t0 - n if hasdn else t0 + (n - 1) * n) + np.arange(4)])
        u4 = [0] * 4 if (neu and not hasup) else list(E[(t0 + n if hasup else t0 - (n - 1) * n) + np.arange(4)])
        lft = 0 if (neu and not hasl) else E[t0 - 1 if hasl else t0 + n - 1]
        rgt = 0 if (neu and not hasr) else E[t0 + 4 if hasr else t0 + 4 - n]
        ev = [lft] + list(E[t0:t0 + 4]) + [rgt]
        for q in range(4):
            nb = []
            if not (neu and q == 0 and not hasl):
                nb.append(ev[q])
            if not (neu and q == 3 and not hasr):
                nb.append(ev[q + 2])
            if not (neu and not hasdn):
                nb.append(d4[q])
            if not (neu and not hasup):
                nb.append(u4[q])
            out[t0 + q] = (ev[q + 1], nb)
    return out


@pytest.mark.parametrize("n", [4, 8, 12, 20])
@pytest.mark.parametrize("neu", [False, True])
def test_update_rows_of_four_select_the_strided_neighbours(n, neu):
    E = np.random.default_rng(n).standard_normal(n * n)
    assert update_neighbours_rows_of_four(E, n, neu) == update_neighbours_strided(E, n, neu)
