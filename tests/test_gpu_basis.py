"""Steerable principal components themselves (Alg. 2 step 5, Sec. V): radial
eigenfunctions (Eq. sPCArad) and eigenimages on the pixel grid (Eq. IFT_FB),
computed in float64 on the GPU, against the FP64 oracle and the
orthonormality of the Fourier-Bessel basis."""
import math

import numpy as np
import pytest
import torch

from oracle import fb
from paper_1412_0781_gb300 import FFBError, Plan, data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec)
    gp = Plan(spec.L, spec.c, spec.R, eps=1e-6)
    gp.covariance(gp.expand(imgs.to("cuda:0")), reset=True)
    ev, U = gp.eig()
    op = fb.make_plan(spec.L, spec.c, spec.R)
    vecs = [b.numpy() for b in gp.unpack_blocks(U.cpu())]
    return gp, op, ev.cpu().numpy(), vecs


def test_radial_eigenfunctions_match_oracle_and_are_orthonormal(setup):
    gp, op, _, vecs = setup
    f = gp.radial_eigenfunctions().cpu()
    ref = fb.radial_eigenfunctions(op, vecs)
    for k in range(gp.k_max + 1):
        fk = gp.radial_block(f, k).numpy()
        assert np.max(np.abs(fk - ref[k])) <= 1e-11 * max(1.0, np.max(np.abs(ref[k])))
        # 2 pi sum_j f^{k,l} f^{k,l'} xi_j w_j = U^T G_k U, with G_k the radial
        # Gram matrix of the basis under the same quadrature (identity up to
        # the quadrature error of Fig. 2a, which grows as R shrinks: ~3e-6 at
        # R = 16); U orthogonal makes the eigenfunctions orthonormal to the
        # same level.
        sw = (op.xi * op.w)[:, None]
        G = 2 * math.pi * (fk * sw).T @ fk
        phi = op.B[k].T / sw                       # N_{kq} J_k(R_{kq} xi_j / c), (n_xi, p_k)
        Gk = 2 * math.pi * (phi * sw).T @ phi
        Uk = vecs[k]
        assert np.max(np.abs(G - Uk.T @ Gk @ Uk)) < 1e-12
        gram_err = np.max(np.abs(Gk - np.eye(Gk.shape[0])))
        assert np.max(np.abs(G - np.eye(G.shape[0]))) <= Gk.shape[0] * gram_err + 1e-12


def test_eigenimages_match_analytic_synthesis(setup):
    gp, op, ev, vecs = setup
    order = np.argsort(-ev)[:6]
    pairs = []
    for t in order:
        k = int(np.searchsorted(np.array(gp.offset), t, side="right") - 1)
        pairs.append((k, int(t - gp.offset[k])))
    pairs.append((0, 0))
    g = gp.eigenimages(pairs).cpu().numpy()
    for i, (k, l) in enumerate(pairs):
        a = np.zeros((2, op.P), complex)
        a[0, op.offset[k]:op.offset[k] + op.p[k]] = vecs[k][:, l]
        a[1] = 1j * a[0]
        s = fb.synthesize_analytic(op, a, "derived") / (1.0 if k == 0 else 2.0)
        scale = np.max(np.abs(s[0])) + np.max(np.abs(s[1]))
        assert np.max(np.abs(g[i].real - s[0])) < 1e-10 * scale
        if k > 0:
            assert np.max(np.abs(g[i].imag + s[1])) < 1e-10 * scale
        else:
            assert np.max(np.abs(g[i].imag)) < 1e-12 * scale


def test_eigenimages_reject_bad_pairs(setup):
    gp, _, _, _ = setup
    with pytest.raises(FFBError):
        gp.eigenimages([(gp.k_max + 1, 0)])
    with pytest.raises(FFBError):
        gp.eigenimages([(0, gp.p[0])])


def _rotate90(x):
    """I'(i1, i2) = I(i2, -i1) on the grid i = a - L/2 (as in the oracle
    pins): row a1 >= 1 of the result is column L - a1 of the input, row 0
    (i1 = -L/2, whose image -i1 = L/2 is off the grid) is zero."""
    L = x.shape[-1]
    out = torch.zeros_like(x)
    cols = L - torch.arange(1, L, device=x.device)
    out[:, 1:, :] = x[:, :, cols].transpose(1, 2)
    return out


PAIRS = [(0, 0), (1, 0), (2, 0), (3, 0), (1, 1)]
TRIPLES = [(1, 0, 1, 0, 0), (1, 0, 2, 0, 0), (1, 0, 0, 0, 0), (2, 0, 1, 0, 0)]


def test_invariant_features_match_oracle(setup):
    gp, op, _, _ = setup
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec)
    coef = gp.expand(imgs.to("cuda:0"))
    pw, bs = gp.invariants(coef, PAIRS, TRIPLES)
    a = fb.expand(op, imgs.double().numpy())
    mean0, blocks = fb.covariance(op, a)
    _, vecs = fb.eig_blocks(blocks)
    rp, rb = fb.invariant_features(op, a, mean0, vecs, PAIRS, TRIPLES)
    gb = bs.cpu().double().numpy()
    gb = gb[..., 0] + 1j * gb[..., 1]
    ep = np.linalg.norm(pw.cpu().double().numpy() - rp) / np.linalg.norm(rp)
    eb = np.linalg.norm(gb - rb) / np.linalg.norm(rb)
    print("invariant features vs oracle: power %.2e, bispectrum %.2e" % (ep, eb))
    assert ep <= 1e-4 and eb <= 1e-4


def test_invariant_features_are_rotation_invariant_on_gpu(setup):
    gp, _, _, _ = setup
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec, n=64)
    # a 90-degree rotation is exact on the grid for images that vanish for
    # r >= R (Eqs. rot, refl); the stack's noise covers every pixel
    x = (imgs * data.support_mask(spec.L, spec.R)).to("cuda:0").contiguous()
    pw, bs = gp.invariants(gp.expand(x), PAIRS, TRIPLES)
    pr, br = gp.invariants(gp.expand(_rotate90(x)), PAIRS, TRIPLES)
    assert float((pr - pw).norm() / pw.norm()) <= 1e-5
    assert float((br - bs).norm() / bs.norm()) <= 1e-5


def test_invariant_features_reject_bad_indices(setup):
    gp, _, _, _ = setup
    coef = torch.zeros((2, gp.P, 2), device="cuda:0")
    with pytest.raises(FFBError):
        gp.invariants(coef, [(gp.k_max + 1, 0)])
    with pytest.raises(FFBError):
        gp.invariants(coef, [], [(gp.k_max, 0, 1, 0, 0)])
