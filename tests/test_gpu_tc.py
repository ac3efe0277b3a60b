"""Tensor-core forms of the radial quadrature (Eq. a) against the FP64 oracle.

The compensated forms (TF32x3, BF16x3) carry the float32 gate (relative L2
<= 1e-5); plain TF32 / BF16 errors are reported with a loose sanity bound."""
import numpy as np
import pytest
import torch

from oracle import fb
from paper_1412_0781_gb300 import Plan, data

pytestmark = pytest.mark.gpu

GATES = {"tf32x3": 1e-5, "bf16x3": 1e-5, "tf32": 5e-3, "bf16": 3e-2}


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _stack(L, n):
    spec = data.StackSpec(n, L, L / 2, 12 if L >= 64 else 6, (2.0 * L / 128 if L >= 64 else 1.5,
                                                            8.0 * L / 128 if L >= 64 else 4.0), 0.1, 777 + L)
    imgs, _, _ = data.blob_stack(spec)
    return imgs


_REF = {}


def _oracle(L, imgs):
    key = (L, imgs.shape[0])
    if key not in _REF:
        op = fb.make_plan(L, 0.5, L / 2)
        _REF[key] = fb.expand(op, imgs.double().numpy())
    return _REF[key]


@pytest.mark.parametrize("L,n", [(32, 300), (128, 160), (180, 20), (256, 8)])
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "tf32", "bf16"])
def test_tc_quadrature_matches_oracle(dev, L, n, prec):
    """L = 180 (n_theta = 720, the separate-kernel NUFFT) and L = 256 (K = 256
    in four bf16 / eight tf32 chunks streamed through a three-stage pipeline)
    cover the K-pipelined contraction beyond one resident tile."""
    imgs = _stack(L, n)
    ref = _oracle(L, imgs)
    plan = Plan(L, 0.5, L / 2, eps=1e-6, precision=prec)
    a = torch.view_as_complex(plan.expand(imgs.to(dev)).cpu()).numpy().astype(np.complex128)
    err = np.linalg.norm(a - ref) / np.linalg.norm(ref)
    print("L=%d %s coefficient rel L2 vs FP64 oracle: %.3e" % (L, prec, err))
    assert np.all(a[:, :plan.p[0]].imag == 0.0)
    assert err <= GATES[prec]
    plan.close()


@pytest.mark.parametrize("L,prec", [(64, "bf16x3"), (128, "bf16x3"), (128, "tf32x3")])
def test_tc_grouped_quadrature_ragged_and_independent(dev, L, prec):
    """One quadrature launch takes the ring spectra of several chunks (up to
    four, as many as fit the plane budget): a stack of two full groups and a
    ragged one gives every image the coefficients it gets alone, and sampled
    images at the chunk and group seams match the oracle."""
    plan = Plan(L, 0.5, L / 2, eps=1e-6, precision=prec)
    per = 4 * plan.chunk                       # at least one group
    n = 2 * per + 37
    spec = data.StackSpec(n, L, L / 2, 12, (2.0 * L / 128, 8.0 * L / 128), 0.1, 4711 + L)
    imgs, _, _ = data.blob_stack(spec, device=dev)
    coef = plan.expand(imgs)
    sel = [0, plan.chunk - 1, plan.chunk, 2 * plan.chunk, per - 1, per, 2 * per - 1, 2 * per, n - 1]
    alone = plan.expand(imgs[sel].contiguous())
    assert torch.equal(coef[sel], alone)
    op = fb.make_plan(L, 0.5, L / 2)
    ref = fb.expand(op, imgs[sel].double().cpu().numpy())
    a = torch.view_as_complex(coef[sel].cpu()).numpy().astype(np.complex128)
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) <= GATES[prec]
    plan.close()


@pytest.mark.parametrize("L,n", [(32, 200), (128, 3000)])
def test_tc_covariance_matches_oracle(dev, L, n):
    """Covariance blocks (Eqs. ck, ck_0) from the tensor-core SYRK, fed the
    oracle's own coefficients (rounded to float32), against the oracle's
    two-pass float64 covariance."""
    op = fb.make_plan(L, 0.5, L / 2)
    rng = np.random.default_rng(L)
    a = (rng.standard_normal((n, op.P)) + 1j * rng.standard_normal((n, op.P))) + 2.0
    a[:, :op.p[0]] = a[:, :op.p[0]].real
    a = a.astype(np.complex64).astype(np.complex128)
    mean0, blocks = fb.covariance(op, a)
    Co = np.concatenate([b.ravel() for b in blocks])
    coef = torch.view_as_real(torch.from_numpy(a.astype(np.complex64))).contiguous().to(dev)
    for prec, tol in (("tf32x3", 1e-5), ("bf16x3", 1e-5), ("tf32", 5e-3), ("bf16", 3e-2)):
        plan = Plan(L, 0.5, L / 2, eps=1e-6, precision=prec)
        plan.covariance(coef[: n // 3].contiguous(), reset=True)
        plan.covariance(coef[n // 3:].contiguous(), reset=False)
        m, C = plan.cov_get()
        err = np.linalg.norm(C.cpu().numpy() - Co) / np.linalg.norm(Co)
        print("L=%d %s covariance rel L2: %.3e" % (L, prec, err))
        assert err <= tol
        assert np.linalg.norm(m.cpu().numpy() - mean0) / np.linalg.norm(mean0) <= 1e-6
        plan.close()


def test_tc_covariance_and_eigs_with_compensated_quadrature(dev):
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec)
    op = fb.make_plan(spec.L, spec.c, spec.R)
    _, blocks = fb.covariance(op, fb.expand(op, imgs.double().numpy()))
    lam = np.concatenate(fb.eig_blocks(blocks)[0])
    for prec in ("tf32x3", "bf16x3"):
        plan = Plan(spec.L, spec.c, spec.R, eps=1e-6, precision=prec)
        plan.covariance(plan.expand(imgs.to(dev)), reset=True)
        ev, _ = plan.eig()
        err = np.linalg.norm(ev.cpu().numpy() - lam) / np.linalg.norm(lam)
        print("%s eigenvalue rel L2: %.3e" % (prec, err))
        assert err <= 1e-5
        plan.close()


def test_set_precision_switches_path(dev):
    imgs = _stack(128, 20).to(dev)
    plan = Plan(128, 0.5, 64.0, eps=1e-6, precision="fp32")
    a32 = plan.expand(imgs).clone()
    plan.set_precision("tf32x3")
    a3 = plan.expand(imgs)
    plan.set_precision("fp32")
    b32 = plan.expand(imgs)
    assert torch.equal(a32, b32)
    rel = float((a3 - a32).norm() / a32.norm())
    assert 0 < rel <= 1e-5
