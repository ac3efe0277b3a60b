"""Host logic of the separate-kernel path's tiled interpolation: the table the
plan builds on the host (exported as ffb_tile_units; no GPU needed).

The table drives the last step of the type-2 NUFFT of Eq. nufft (Sec. III)
for the plans whose oversampled half grid does not fit in one SM's shared
memory: every polar node reads the 8 x 8 window of the half grid G at its
origin with ES-kernel weights.  Checked against the geometry restated from
that definition:
  * every node t = j n_theta/2 + l appears in exactly one block's node list;
  * each node's window origin lies in its block's tile, and its window inside
    its unit's 9 x 9 union inside the tile held in shared memory;
  * interpolating a random half grid (columns wrapped mod N) through the
    records, the way the kernel reads them, equals the direct 8 x 8 sum of
    phi(f2 - r) phi(f1 - q) over the node's window;
  * blocks hold at most GU units, empty units only at the end, and each half
    warp holds one unit of every bank slot that still has units when it is
    formed."""
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


def sizes(L, c, R):
    n_xi = int(math.ceil(4 * c * R - 1e-9))
    n_theta = int(math.ceil(16 * c * R - 1e-9))
    n_theta += n_theta & 1
    t, _ = np.polynomial.legendre.leggauss(n_xi)
    return n_xi, n_theta, 0.5 * c * (t + 1.0)


@pytest.mark.parametrize("L,c,R", [(32, 0.5, 16.0), (45, 0.5, 22.5), (96, 0.5, 48.0), (100, 0.4, 40.0)])
def test_tiles_cover_every_node_and_interpolate_like_the_direct_sum(ffb, L, c, R):
    N = 2 * L
    n_xi, n_theta, xi = sizes(L, c, R)
    nh = n_theta // 2
    Mh = N // 2 + 1 + 2 * H
    rec, blk, nodes, geo = ffb.tile_units(N, W, BETA, n_theta, xi)
    TR, TC, RS, CS, pitch = geo["TR"], geo["TC"], geo["RS"], geo["CS"], geo["pitch"]
    assert sorted(nodes.tolist()) == list(range(n_xi * nh))          # every node exactly once
    rng = np.random.default_rng(L)
    G = rng.standard_normal((Mh, N)) + 1j * rng.standard_normal((Mh, N))
    err, scale = 0.0, 0.0
    for b in range(blk.shape[0]):
        e0, u0, first, cnt = (int(v) for v in blk[b])
        assert e0 % TR == 0 and u0 % TC == 0
        # the tile as the kernel stages it: row i = G row e0 + i (zero past
        # the half grid), column k = m1 = u0 + k - N/2 - H taken mod N
        T = np.zeros((RS, CS), complex)
        for i in range(RS):
            if e0 + i < Mh:
                T[i] = G[e0 + i, (u0 + np.arange(CS) - N // 2 - H) % N]
        meta = rec[b, 18]
        origin = meta[:, 0].copy().view(np.int32)
        s01 = meta[:, 1].copy().view(np.uint32)
        s23 = meta[:, 2].copy().view(np.uint32)
        slot0 = s01 & 0xFFFF
        used = np.nonzero(slot0 != 0xFFFF)[0]
        assert np.array_equal(used, np.arange(len(used)))           # empty units only at the end
        seen = set()
        for u in used:
            ru, cu = int(origin[u]) & 0xFFFF, int(origin[u]) >> 16
            assert ru + 9 <= RS and cu + 9 <= CS
            slots = [int(s01[u]) & 0xFFFF, int(s01[u]) >> 16, int(s23[u]) & 0xFFFF, int(s23[u]) >> 16]
            for i, sl in enumerate(slots):
                if sl == 0xFFFF:
                    assert not rec[b, :18, u, i].any()
                    continue
                assert sl < cnt and sl not in seen
                seen.add(sl)
                t = int(nodes[first + sl])
                j, l = divmod(t, nh)
                th = 2.0 * math.pi * l / n_theta
                p1, p2 = N * xi[j] * math.cos(th), N * xi[j] * math.sin(th)
                m1, m2 = math.ceil(p1 - 0.5 * W), math.ceil(p2 - 0.5 * W)
                r0, uu = m2 + H, m1 + N // 2 + H
                assert e0 <= r0 < e0 + TR and u0 <= uu < u0 + TC          # origin in the tile
                dr, dc = r0 - e0 - ru, uu - u0 - cu
                assert dr in (0, 1) and dc in (0, 1)                      # window inside the union
                wy, wx = phi((p2 - m2) - np.arange(W)), phi((p1 - m1) - np.arange(W))
                direct = wy @ G[r0:r0 + W][:, (m1 + np.arange(W)) % N] @ wx
                rows = rec[b, 9:18, u, i].astype(np.float64)
                cols = rec[b, 0:9, u, i].astype(np.float64)
                table = rows @ T[ru:ru + 9, cu:cu + 9] @ cols
                err = max(err, abs(table - direct))
                scale = max(scale, float(np.abs(wy).sum() * np.abs(wx).sum()))
        assert len(seen) == cnt
    assert err <= 1e-6 * scale


@pytest.mark.parametrize("L", [96, 256])
def test_tile_blocks_budgets_and_bank_slots(ffb, L):
    N = 2 * L
    n_xi, n_theta, xi = sizes(L, 0.5, L / 2)
    rec, blk, nodes, geo = ffb.tile_units(N, W, BETA, n_theta, xi)
    gu, pitch = rec.shape[2], geo["pitch"]
    units = 0
    for b in range(blk.shape[0]):
        slot0 = rec[b, 18, :, 1].copy().view(np.uint32) & 0xFFFF
        nu = int(np.count_nonzero(slot0 != 0xFFFF))
        assert 1 <= nu <= gu and 1 <= blk[b, 3] <= 4 * nu
        units += nu
        origin = rec[b, 18, :nu, 0].copy().view(np.int32)
        bank = ((origin & 0xFFFF) * pitch + (origin >> 16)) % 16
        left = np.bincount(bank, minlength=16)
        for h0 in range(0, nu, 16):
            grp = bank[h0:h0 + 16]
            assert len(set(grp.tolist())) >= min(int(np.count_nonzero(left)), len(grp))
            left -= np.bincount(grp, minlength=16)
        assert not left.any()
    # the grouping pays on the polar grid: well above two nodes per unit
    assert len(nodes) / units > 2.2


def test_tile_table_rejects_unsupported_width(ffb):
    n_xi, n_theta, xi = sizes(64, 0.5, 32.0)
    with pytest.raises(ffb.FFBError):
        ffb.tile_units(128, 7, 2.30 * 7, n_theta, xi)
