"""The precision workload (L = 128, SNR = 1/10, blob stacks) on its first
1000 images: coefficients and the top-20 eigenpairs of the 1000 images, and
the top-20 denoised images of the first 300 (the oracle's synthesis is the
slow part), for each GPU precision against the FP64 oracle.  FP32 and the compensated
tensor-core forms (TF32x3, BF16x3) carry the 1e-5 relative L2 gate on
coefficients, eigenvalues and denoised images; eigenvectors (conditioned by
the eigenvalue gaps) are gated at 1e-4; plain TF32 / BF16 are reported."""
import numpy as np
import pytest
import torch

from oracle import fb
from paper_1412_0781_gb300 import Plan, data

pytestmark = pytest.mark.gpu

N_SUB = 1000
N_DEN = 300
K_TOP = 20
GATED = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-5}


@pytest.fixture(scope="module")
def ref():
    import __graft_entry__
    __graft_entry__.build()
    spec = data.PRECISION_L128
    imgs, _, _ = data.blob_stack(spec, n=N_SUB)
    op = fb.make_plan(spec.L, spec.c, spec.R)
    x = imgs.double().numpy()
    a = fb.expand(op, x)
    mean0, blocks = fb.covariance(op, a)
    lams, vecs = fb.eig_blocks(blocks)
    hs = fb.select_filter(op, lams, "topk", K=K_TOP)
    den = fb.synthesize(op, fb.filter_coefficients(op, a[:N_DEN], mean0, vecs, hs))
    top = sorted([(-lams[k][l], k, l) for k in range(len(lams)) for l in range(lams[k].size)])[:K_TOP]
    return imgs, op, a, lams, vecs, den, [(k, l) for _, k, l in top]


def _rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3", "tf32", "bf16"])
def test_precision_subset_against_oracle(ref, prec):
    imgs, op, a_ref, lams, vecs, den_ref, top = ref
    dev = torch.device("cuda:0")
    plan = Plan(op.L, op.c, op.R, eps=1e-6, precision=prec)
    x = imgs.to(dev)
    coef = plan.expand(x)
    a = torch.view_as_complex(coef.cpu()).numpy().astype(np.complex128)
    e_coef = _rel(a, a_ref)
    plan.covariance(coef, reset=True)
    ev, U = plan.eig()
    ev = ev.cpu().numpy()
    blocks = [b.numpy() for b in plan.unpack_blocks(U.cpu())]
    lam_g = np.array([ev[op.offset[k] + l] for k, l in top])
    lam_r = np.array([lams[k][l] for k, l in top])
    e_lam = _rel(lam_g, lam_r)
    # eigenvectors: sign-aligned difference of each of the top components
    e_vec = max(min(np.linalg.norm(blocks[k][:, l] - vecs[k][:, l]), np.linalg.norm(blocks[k][:, l] + vecs[k][:, l]))
                for k, l in top)
    # the tail of ffb_denoise (selection, filter with the synthesis weights,
    # adjoint) with the 1000 images' eigenpairs, on the first N_DEN images
    plan.select("topk", K=K_TOP)
    den_coef = plan.filter(coef[:N_DEN].contiguous(), weight=True)
    den = plan.expand_adjoint(den_coef).double().cpu().numpy()
    e_den = _rel(den, den_ref)
    print("%s: coefficients %.2e, top-%d eigenvalues %.2e, eigenvectors %.2e, denoised %.2e"
          % (prec, e_coef, K_TOP, e_lam, e_vec, e_den))
    if prec in GATED:
        tol = GATED[prec]
        assert e_coef <= tol and e_lam <= tol and e_den <= tol
        assert e_vec <= 1e-4
    else:
        assert e_coef <= 5e-3 and e_lam <= 5e-3   # reported; loose sanity bound
    plan.close()
