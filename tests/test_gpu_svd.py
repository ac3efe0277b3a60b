"""The SVD route (Sec. III, Alg. 2 step 4 second alternative) on the GPU
against the FP64 oracle's SVD of the coefficient matrices."""
import numpy as np
import pytest
import torch

from oracle import fb
from paper_1412_0781_gb300 import Plan, data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _coef(op, n, seed):
    rng = np.random.default_rng(seed)
    scale = np.exp(-np.linspace(0, 4, op.P))[None, :]          # a decaying spectrum
    a = (rng.standard_normal((n, op.P)) + 1j * rng.standard_normal((n, op.P))) * scale + 0.2
    a[:, :op.p[0]] = a[:, :op.p[0]].real
    return a.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("L,n", [(32, 500), (128, 3000), (256, 400)])
def test_svd_route_matches_oracle(dev, L, n):
    op = fb.make_plan(L, 0.5, L / 2)
    a = _coef(op, n, L)
    lams, vecs = fb.svd_route(op, a)
    plan = Plan(L, 0.5, L / 2, eps=1e-6)
    coef = torch.view_as_real(torch.from_numpy(a.astype(np.complex64))).contiguous().to(dev)
    ev, U = plan.svd(coef)
    ev = ev.cpu().numpy()
    blocks = plan.unpack_blocks(U.cpu())
    lam_all = np.concatenate(lams)
    err = np.linalg.norm(ev - lam_all) / np.linalg.norm(lam_all)
    # the covariance U diag(lambda) U^T per block against the oracle's
    num = den = 0.0
    for k in range(len(op.p)):
        o, pk = op.offset[k], op.p[k]
        Ug = blocks[k].numpy()
        Cg = Ug @ np.diag(ev[o:o + pk]) @ Ug.T
        Co = vecs[k] @ np.diag(lams[k]) @ vecs[k].T
        num += np.sum((Cg - Co) ** 2)
        den += np.sum(Co ** 2)
    ec = np.sqrt(num / den)
    print("L=%d n=%d SVD route: eigenvalues rel L2 %.2e, U diag(l) U^T rel L2 %.2e" % (L, n, err, ec))
    assert err <= 1e-5
    assert ec <= 1e-5
    # the k = 0 mean used by the filter
    plan.close()


def test_svd_route_agrees_with_covariance_route_on_blobs(dev):
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec)
    plan = Plan(spec.L, spec.c, spec.R, eps=1e-6)
    coef = plan.expand(imgs.to(dev))
    plan.covariance(coef, reset=True)
    ev_c, _ = plan.eig()
    ev_s, _ = plan.svd(coef)
    e = float((ev_s - ev_c).norm() / ev_c.norm())
    print("blob stack: SVD route vs covariance route eigenvalues rel L2 %.2e" % e)
    assert e <= 1e-5
