"""Host logic of the shared-memory grid path: the interpolation table that the
plan builds on the host (exported as ffb_interp_units; no GPU needed).

The table drives the last step of the type-2 NUFFT of Eq. nufft (Sec. III):
every polar node reads the 8 x 8 window of the oversampled half grid at its
origin with ES-kernel weights.  Checked here against the geometry restated
from that definition:
  * every node of each half lies in exactly one unit of one block;
  * interpolating a random half grid through the records, the way the kernel
    reads them (one 9 x 9 union per unit, 9 row and 9 column weights per
    node), equals the direct 8 x 8 sum of phi(f2 - r) phi(f1 - q) over the
    node's window, and the node's window lies inside its unit's union;
  * blocks stay within their unit and node budgets, and each half warp of a
    block holds one unit of every bank slot (origin mod 16) that still has
    units when it is formed."""
import math

import numpy as np
import pytest

W = 8
H = (W + 1) // 2
BETA = 2.30 * W


@pytest.fixture(scope="module")
def ffb():
    from paper_1412_0781_gb300 import build
    build.build()
    from paper_1412_0781_gb300 import ffb as mod
    return mod


def phi(x):
    z = 2.0 * x / W
    u = 1.0 - z * z
    return np.where(u > 0.0, np.exp(BETA * (np.sqrt(np.maximum(u, 0.0)) - 1.0)), 0.0)


def radii(n_xi, c):
    t, _ = np.polynomial.legendre.leggauss(n_xi)
    return 0.5 * c * (t + 1.0)


def decode(rec, blk, nb, n_xi, n_theta, N):
    """Per half: list of (node t, union row ru, union column cu, row weights
    (9,), column weights (9,)) over the unit's 9 x 9 union."""
    nq0 = n_theta // 4 + 1
    out = [[], []]
    gu = rec.shape[2]
    for b in range(rec.shape[0]):
        half = 0 if b < nb[0] else 1
        t0, cnt = int(blk[b, 0]), int(blk[b, 1])
        meta = rec[b, 18]
        origin = meta[:, 0].copy().view(np.int32)
        s01 = meta[:, 1].copy().view(np.uint32)
        s23 = meta[:, 2].copy().view(np.uint32)
        for u in range(gu):
            slots = [int(s01[u]) & 0xFFFF, int(s01[u]) >> 16, int(s23[u]) & 0xFFFF, int(s23[u]) >> 16]
            if slots[0] == 0xFFFF:
                continue
            ru, cu = int(origin[u]) & 0xFFFF, int(origin[u]) >> 16
            for i, sl in enumerate(slots):
                if sl == 0xFFFF:
                    assert not rec[b, :18, u, i].any()          # an empty slot carries zero weights
                    continue
                assert sl < cnt
                out[half].append((t0 + sl, ru, cu, rec[b, 9:18, u, i].copy(), rec[b, 0:9, u, i].copy()))
    return out, nq0


CASES = [(64, 0.5, 32.0), (128, 0.5, 64.0), (128, 0.4, 50.0)]


@pytest.mark.parametrize("L,c,R", CASES)
def test_units_cover_every_node_and_interpolate_like_the_direct_sum(ffb, L, c, R):
    N = 2 * L
    n_xi = int(math.ceil(4 * c * R - 1e-9))
    n_theta = int(math.ceil(16 * c * R - 1e-9))
    n_theta += n_theta & 1
    xi = radii(n_xi, c)
    rec, blk, nb, MH, SLD, nu = ffb.interp_units(N, W, BETA, n_theta, xi)
    assert rec.shape[0] == nb[0] + nb[1] == blk.shape[0] and nu <= 4
    units, nq0 = decode(rec, blk, nb, n_xi, n_theta, N)
    rng = np.random.default_rng(L + int(10 * c))
    for half in (0, 1):
        l0 = 0 if half == 0 else nq0
        nl = nq0 if half == 0 else n_theta // 2 - nq0
        ts = sorted(u[0] for u in units[half])
        assert ts == list(range(n_xi * nl))                 # each node exactly once
        S = rng.standard_normal((MH + 1, SLD)) + 1j * rng.standard_normal((MH + 1, SLD))
        S[:, MH:] = 0.0                                     # the two zero pad columns
        S[MH, :] = 0.0                                      # and the zero pad row
        m1lo = -H if half == 0 else -(N // 2) - H
        err, scale = 0.0, 0.0
        for (t, r0, cu, rows, cols) in units[half]:
            j, l = t // nl, l0 + t % nl
            th = 2.0 * math.pi * l / n_theta
            p1, p2 = N * xi[j] * math.cos(th), N * xi[j] * math.sin(th)
            m1, m2 = math.ceil(p1 - 0.5 * W), math.ceil(p2 - 0.5 * W)
            c0, r0e = m1 - m1lo, m2 + H
            assert 0 <= r0e - r0 <= 1 and 0 <= c0 - cu <= 1     # the window inside the 9 x 9 union
            assert 0 <= r0e and r0e + W <= MH and 0 <= c0 and c0 + W <= MH
            assert r0 + 9 <= MH + 1 and cu + 9 <= SLD
            wy, wx = phi((p2 - m2) - np.arange(W)), phi((p1 - m1) - np.arange(W))
            direct = wy @ S[r0e:r0e + W, c0:c0 + W] @ wx
            table = rows.astype(np.float64) @ S[r0:r0 + 9, cu:cu + 9] @ cols.astype(np.float64)
            err = max(err, abs(table - direct))
            scale = max(scale, float(np.abs(wy).sum() * np.abs(wx).sum()))
        assert err <= 1e-6 * scale, (half, err, scale)


@pytest.mark.parametrize("L,c,R", CASES[:2])
def test_blocks_budgets_and_bank_slots(ffb, L, c, R):
    N = 2 * L
    n_xi, n_theta = int(4 * c * R), int(16 * c * R)
    rec, blk, nb, MH, SLD, nu_max = ffb.interp_units(N, W, BETA, n_theta, radii(n_xi, c))
    gu = rec.shape[2]                                  # one unit per thread of the CTA
    gn = (gu // 32) * N // 2                           # nodes per block: one staging entry each (N/2 per warp)
    total_units = total_nodes = 0
    for b in range(rec.shape[0]):
        assert 1 <= blk[b, 1] <= gn
        s01 = rec[b, 18, :, 1].copy().view(np.uint32)
        s23 = rec[b, 18, :, 2].copy().view(np.uint32)
        slot0 = s01 & 0xFFFF
        used = np.nonzero(slot0 != 0xFFFF)[0]
        nu = len(used)
        assert nu <= gu and np.array_equal(used, np.arange(nu))   # empty units only at the end
        filled = [(s01[:nu] & 0xFFFF) != 0xFFFF, (s01[:nu] >> 16) != 0xFFFF,
                  (s23[:nu] & 0xFFFF) != 0xFFFF, (s23[:nu] >> 16) != 0xFFFF]
        nodes = int(sum(np.count_nonzero(f) for f in filled[:nu_max]))
        assert not any(np.count_nonzero(f) for f in filled[nu_max:])
        assert nodes == blk[b, 1]
        total_units += nu
        total_nodes += nodes
        origin = rec[b, 18, :nu, 0].copy().view(np.int32)
        bank = ((origin & 0xFFFF) * SLD + (origin >> 16)) % 16
        # half warp h reads units 16 h .. 16 h + 15: it holds one unit of
        # every slot that still has units left when it is formed (at most 16)
        left = np.bincount(bank, minlength=16)
        for h0 in range(0, nu, 16):
            grp = bank[h0:h0 + 16]
            assert len(set(grp.tolist())) >= min(int(np.count_nonzero(left)), len(grp))
            left -= np.bincount(grp, minlength=16)
        assert not left.any()
    # the grouping pays: well above two nodes per unit on these polar grids
    assert total_nodes / total_units > 2.2


def test_rejects_unsupported_geometry(ffb):
    with pytest.raises(ffb.FFBError):
        ffb.interp_units(512, W, BETA, 256, radii(64, 0.5))        # N outside {128, 256}
    with pytest.raises(ffb.FFBError):
        ffb.interp_units(256, 7, 2.30 * 7, 512, radii(128, 0.5))   # w != 8
