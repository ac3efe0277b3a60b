"""Batching: several stacks of uneven L and n through a1-a7 in one call
(ffb_group_*: per-stack branches, one grouped covariance launch over the
uneven per-k blocks of every stack, CUDA-graph replay, autotuned item shape).

Checks: the grouped SYRK against the FP64 oracle's covariance of seeded
coefficients (Eqs. ck, ck_0); the expansion of sampled images of every stack
against the oracle; the group's coefficients equal to ffb_expand's bit for
bit, on the eager call and on the graph replays; the covariance equal to the
single-plan path within float32 accumulation error."""
import math

import numpy as np
import pytest
import torch

from oracle import fb
from paper_1412_0781_gb300 import FFBError, Group, Plan, data

pytestmark = pytest.mark.gpu

# (L, n): the L values of the batching workload, ragged n, one empty stack
STACKS = [(64, 300), (96, 130), (128, 200), (180, 61), (256, 24), (64, 0), (128, 37)]


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _images(L, n, s):
    rng = np.random.default_rng(1000 + s)
    snr = float(rng.uniform(1 / 50, 1 / 5))
    spec = data.StackSpec(max(n, 1), L, L / 2, 12, (2.0 * L / 128, 8.0 * L / 128), snr, 20141206 + 1000 * s)
    imgs, _, _ = data.blob_stack(spec)
    return imgs[:n]


@pytest.fixture(scope="module")
def stacks(dev):
    return [_images(L, n, s).to(dev) for s, (L, n) in enumerate(STACKS)]


def _plans(prec):
    return [Plan(L, 0.5, L / 2, eps=1e-6, precision=prec) for L, _ in STACKS]


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_group_equals_single_plans_and_replays(dev, stacks, prec):
    plans = _plans(prec)
    g = Group(plans)
    coefs = [torch.empty((n, p.P, 2), device=dev) if n else None for p, (_, n) in zip(plans, STACKS)]
    imgs = [x if x.shape[0] else None for x in stacks]
    g.expand_cov(imgs, coefs, reset=True)
    first = [c.clone() if c is not None else None for c in coefs]
    cov_first = [p.cov_get()[1].clone() if n else None for p, (_, n) in zip(plans, STACKS)]
    for _ in range(3):                    # capture, then replays of the same graph
        for c in coefs:
            if c is not None:
                c.fill_(float("nan"))
        g.expand_cov(imgs, coefs, reset=True)
    g.sync()
    info = g.info()
    assert info["eager"] == 1 and info["graphs"] == 1 and info["replays"] == 3
    assert info["launches"] > 0 and info["candidates"] > 0
    if prec == "fp32":
        assert info["quad_rounds"] == 0
    else:
        # one grouped quadrature launch per round, its launch shape tuned once
        assert info["quad_rounds"] >= 1 and info["quad_candidates"] >= 1
        qc = g.quad_tuning()
        assert any(c["per_sm"] == info["quad_per_sm"] and c["stages"] == info["quad_stages"] for c in qc)
        assert all(c["ms"] > 0 for c in qc)
    cands = g.tuning()
    assert any(c["per"] == info["per"] and c["tile"] == info["tile"] and c["grid"] == info["grid"] for c in cands)
    refs = _plans(prec)
    for s, (p, r, (L, n)) in enumerate(zip(plans, refs, STACKS)):
        if n == 0:
            continue
        a = r.expand(stacks[s])
        assert torch.equal(first[s], a), "stack %d: group != ffb_expand" % s
        assert torch.equal(coefs[s], a), "stack %d: graph replay != eager" % s
        r.covariance(a, reset=True)
        _, Cr = r.cov_get()
        _, Cg = p.cov_get()
        rel = float((Cg - Cr).norm() / Cr.norm())
        assert rel < 1e-5, "stack %d covariance vs single plan: %.3e" % (s, rel)
        assert float((Cg - cov_first[s]).norm() / Cr.norm()) < 1e-6   # same item shape: rounding order only
    g.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-5), ("tf32x3", 1e-5), ("bf16", 3e-2)])
def test_group_covariance_matches_oracle(dev, prec, tol):
    """Seeded complex coefficients per stack (rounded to float32), accumulated
    in two grouped calls (reset, then accumulate), against the oracle's
    two-pass float64 covariance of each stack."""
    plans = _plans(prec)
    g = Group(plans)
    rng = np.random.default_rng(77)
    coefs, ref = [], []
    for p, (L, n) in zip(plans, STACKS):
        if n == 0:
            coefs.append(None)
            ref.append(None)
            continue
        op = fb.make_plan(L, 0.5, L / 2)
        a = rng.standard_normal((n, op.P)) + 1j * rng.standard_normal((n, op.P)) + 1.5
        a[:, :op.p[0]] = a[:, :op.p[0]].real
        a = a.astype(np.complex64).astype(np.complex128)
        m0, blocks = fb.covariance(op, a)
        ref.append((m0, np.concatenate([b.ravel() for b in blocks])))
        coefs.append(torch.view_as_real(torch.from_numpy(a.astype(np.complex64))).contiguous().to(dev))
    half = [None if c is None else c[: c.shape[0] // 2].contiguous() for c in coefs]
    rest = [None if c is None else c[c.shape[0] // 2:].contiguous() for c in coefs]
    g.covariance(half, reset=True)
    g.covariance(rest, reset=False)
    g.sync()
    for s, (p, r) in enumerate(zip(plans, ref)):
        if r is None:
            continue
        m, C = p.cov_get()
        err = np.linalg.norm(C.cpu().numpy() - r[1]) / np.linalg.norm(r[1])
        print("stack %d L=%d %s grouped covariance rel L2: %.3e" % (s, STACKS[s][0], prec, err))
        assert err <= tol
        assert np.linalg.norm(m.cpu().numpy() - r[0]) / np.linalg.norm(r[0]) <= 1e-6
    g.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_group_expansion_matches_oracle_on_samples(dev, stacks, prec):
    plans = _plans(prec)
    g = Group(plans)
    coefs = [torch.empty((n, p.P, 2), device=dev) if n else None for p, (_, n) in zip(plans, STACKS)]
    g.expand_cov([x if x.shape[0] else None for x in stacks], coefs, reset=True)
    g.sync()
    for s, (L, n) in enumerate(STACKS):
        if n == 0:
            continue
        idx = [0, n - 1] if L < 256 else [n - 1]     # the last image sits in a ragged chunk
        op = fb.make_plan(L, 0.5, L / 2)
        ref = fb.expand(op, stacks[s][idx].double().cpu().numpy())
        got = torch.view_as_complex(coefs[s][idx].cpu()).numpy().astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print("stack %d L=%d %s sampled coefficients rel L2: %.3e" % (s, L, prec, err))
        assert err <= 1e-5
    g.close()


def test_group_rejects_bad_membership(dev):
    a = Plan(64, 0.5, 32.0, precision="fp32")
    b = Plan(96, 0.5, 48.0, precision="bf16x3")
    with pytest.raises(FFBError):
        Group([a, a])                      # one plan twice
    with pytest.raises(FFBError):
        Group([a, b])                      # mixed precision
    g = Group([a, Plan(96, 0.5, 48.0, precision="fp32")])
    a.set_precision("bf16x3")
    x = torch.zeros((4, 64, 64), device=dev)
    c = torch.empty((4, a.P, 2), device=dev)
    with pytest.raises(FFBError) as ei:
        g.expand_cov([x, None], [c, None])
    assert ei.value.status == -7          # FFB_ERR_STATE
    g.close()


def test_batching_workload_48_stacks_against_oracle(dev):
    """The batching workload's 48 stacks (seeded recipe: L drawn from
    {64, 96, 128, 180, 256}, R = L/2, SNR uniform in [1/50, 1/5]) with every
    stack's n cut to 1/100 of the recipe's (5 to 200 images), BF16x3 (float32
    path with compensated tensor-core GEMMs): one group call eager, one
    capturing, one replayed.  Every stack's first and last image against the
    FP64 oracle's expansion; every coefficient of the replay bit-equal to
    ffb_expand's; the grouped covariance against the oracle's covariance of
    the group's own coefficients (Eqs. ck, ck_0)."""
    from dataclasses import replace
    specs = [replace(sp, n=max(5, sp.n // 100)) for sp in data.batching_stacks()]
    assert len(specs) == 48 and {sp.L for sp in specs} == {64, 96, 128, 180, 256}
    imgs = [data.blob_stack(sp, device=dev)[0] for sp in specs]
    plans = [Plan(sp.L, sp.c, sp.R, eps=1e-6, precision="bf16x3") for sp in specs]
    coefs = [torch.empty((sp.n, p.P, 2), device=dev) for sp, p in zip(specs, plans)]
    g = Group(plans)
    for _ in range(3):
        g.expand_cov(imgs, coefs, reset=True)
    g.sync()
    info = g.info()
    assert info["eager"] == 1 and info["graphs"] == 1 and info["replays"] == 2
    assert info["quad_rounds"] >= 1
    for s, (sp, p, x, c) in enumerate(zip(specs, plans, imgs, coefs)):
        ref = Plan(sp.L, sp.c, sp.R, eps=1e-6, precision="bf16x3")
        assert torch.equal(c, ref.expand(x)), "stack %d: group != ffb_expand" % s
        ref.close()
        op = fb.make_plan(sp.L, sp.c, sp.R)
        a = torch.view_as_complex(c.cpu()).numpy().astype(np.complex128)
        pick = [0, sp.n - 1]
        ao = fb.expand(op, x[pick].double().cpu().numpy())
        err = np.linalg.norm(a[pick] - ao) / np.linalg.norm(ao)
        assert err <= 1e-5, "stack %d (L = %d): coefficients vs oracle %.2e" % (s, sp.L, err)
        m_ref, blocks = fb.covariance(op, a)
        m, C = p.cov_get()
        Cb = [b.numpy() for b in p.unpack_blocks(C.cpu())]
        num = sum(np.linalg.norm(x1 - x2) ** 2 for x1, x2 in zip(Cb, blocks))
        den = sum(np.linalg.norm(x2) ** 2 for x2 in blocks)
        assert math.sqrt(num / den) <= 1e-5, "stack %d: covariance vs oracle" % s
        assert np.linalg.norm(m.cpu().numpy() - m_ref) <= 1e-5 * np.linalg.norm(m_ref)
    g.close()
    for p in plans:
        p.close()
