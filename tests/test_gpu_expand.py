"""GPU parity of the forward hot path (plan tables, polar NUFFT, ring DFT,
radial quadrature, covariance, eigenpairs) against the FP64 oracle, through
the C ABI.  Tolerances: relative L2 <= 1e-5 for float32 results (coefficients,
covariance, eigenvalues); the NUFFT at the requested eps against the direct
NDFT; float64 setup tables at 1e-12."""
import math

import numpy as np
import pytest
import torch

from oracle import fb
from paper_1412_0781_gb300 import Plan, FFBError, data

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


_PLANS = {}


def gplan(L, eps=1e-6, precision="fp32"):
    key = (L, eps, precision)
    if key not in _PLANS:
        _PLANS[key] = Plan(L, 0.5, L / 2, eps=eps, precision=precision)
    return _PLANS[key]


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def as_complex(coef):
    return torch.view_as_complex(coef.detach().cpu().contiguous()).numpy().astype(np.complex128)


# --- a0: setup tables --------------------------------------------------------
@pytest.mark.parametrize("L", [32, 64, 128])
def test_plan_tables_match_oracle(dev, L):
    gp, op = gplan(L), fb.make_plan(L, 0.5, L / 2)
    assert (gp.k_max, gp.P, gp.n_xi, gp.n_theta) == (op.k_max, op.P, op.n_xi, op.n_theta)
    assert gp.p == list(op.p) and gp.offset == list(op.offset)
    z, xi, w, B = gp.tables()
    assert np.max(np.abs(z - np.concatenate(op.zeros)) / np.concatenate(op.zeros)) < 1e-13
    assert np.max(np.abs(xi - op.xi)) < 1e-15
    assert np.max(np.abs(w - op.w) / op.w) < 1e-12
    Bo = np.concatenate(op.B, axis=0)
    assert np.max(np.abs(B - Bo)) < 1e-12 * np.max(np.abs(Bo))


# --- a1-a3: NUFFT vs direct NDFT -------------------------------------------
@pytest.mark.parametrize("L,n", [(32, 6), (64, 3), (128, 2)])
def test_polar_nufft_within_eps_of_direct_ndft(dev, L, n):
    gp, op = gplan(L), fb.make_plan(L, 0.5, L / 2)
    noise = data.white_noise(n, L, seed=100 + L)
    blobs, _, _ = data.blob_stack(data.StackSpec(n, L, L / 2, 8, (1.5, 6.0), 0.2, 200 + L))
    for imgs in (noise, blobs):
        F = gp.polar(imgs.to(dev))
        Fg = torch.view_as_complex(F.cpu()).numpy().astype(np.complex128)
        Fo = fb.ndft_polar(op, imgs.double().numpy())[:, :, :gp.n_theta // 2]
        assert rel(Fg, Fo) <= gp.eps


# --- a1-a5: coefficients -------------------------------------------------------
def test_expand_tiny_config_matches_oracle(dev):
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec)
    gp, op = gplan(spec.L), fb.make_plan(spec.L, spec.c, spec.R)
    a = as_complex(gp.expand(imgs.to(dev)))
    ao = fb.expand(op, imgs.double().numpy())
    assert rel(a, ao) <= TOL
    per_image = np.linalg.norm(a - ao, axis=1) / np.linalg.norm(ao, axis=1)
    assert per_image.max() <= 3 * TOL
    assert np.all(a[:, :gp.p[0]].imag == 0.0)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_odd_image_size_matches_oracle(dev, prec):
    """Odd L (45: pixel indices -22..22, N = 90 = 2 3^2 5, n_theta = 180, a
    mixed-radix FFT on both axes): the expansion and the adjoint against the
    oracle."""
    L, c, R = 45, 0.5, 22.5
    imgs, _, _ = data.blob_stack(data.StackSpec(6, L, R, 6, (1.5, 4.0), 0.2, 20141209))
    gp = Plan(L, c, R, eps=1e-6, precision=prec)
    try:
        op = fb.make_plan(L, c, R)
        assert (gp.P, gp.n_xi, gp.n_theta, gp.N) == (op.P, op.n_xi, op.n_theta, 90)
        a = as_complex(gp.expand(imgs.to(dev)))
        assert rel(a, fb.expand(op, imgs.double().numpy())) <= TOL
        rng = np.random.default_rng(45)
        y = rng.standard_normal((3, gp.P)) + 1j * rng.standard_normal((3, gp.P))
        y = y.astype(np.complex64).astype(np.complex128)
        yd = torch.view_as_real(torch.from_numpy(y.astype(np.complex64))).contiguous().to(dev)
        g = gp.expand_adjoint(yd).double().cpu().numpy()
        assert rel(g, fb.adjoint(op, y)) <= TOL
    finally:
        gp.close()


def test_expand_ragged_chunks_and_independence(dev):
    """n spans several internal chunks plus a ragged tail; each image's
    coefficients do not depend on which chunk it fell in."""
    L = 32
    gp, op = gplan(L), fb.make_plan(L, 0.5, L / 2)
    n = 2 * gp.chunk + 37
    imgs, _, _ = data.blob_stack(data.StackSpec(n, L, 16.0, 6, (1.5, 4.0), 0.2, 31337))
    d = imgs.to(dev)
    a_all = gp.expand(d)
    sel = [0, gp.chunk - 1, gp.chunk, 2 * gp.chunk - 1, 2 * gp.chunk, n - 1]
    sub = gp.expand(d[sel].contiguous())
    assert torch.equal(a_all[sel], sub)
    ao = fb.expand(op, imgs[sel].double().numpy())
    assert rel(as_complex(a_all[sel]), ao) <= TOL


def test_expand_zero_images_is_noop(dev):
    gp = gplan(32)
    out = torch.full((1, gp.P, 2), 7.0, device=dev)
    gp.expand(torch.empty((0, 32, 32), device=dev), out=out[:0])
    assert torch.all(out == 7.0)


def test_rotation_reflection_on_gpu(dev):
    """Eqs. rot/refl on the CUDA path alone: rotation by pi/2 multiplies
    a_{k,q} by e^{-i k pi/2}, reflection conjugates (images zero for r >= R)."""
    L = 64
    gp = gplan(L)
    imgs, _, _ = data.blob_stack(data.StackSpec(4, L, 32.0, 8, (2.0, 6.0), 0.5, 77))
    mask = data.support_mask(L, 32.0)
    imgs = imgs * mask
    x = imgs.to(dev)
    o = L // 2
    # I'(a1, a2) = I(a2 - o + o, -(a1 - o) + o): rotation; index -o maps outside -> zero there
    idx = torch.arange(L)
    rot = torch.zeros_like(imgs)
    src1 = idx[None, :].expand(L, L)                 # a2
    src2 = (2 * o - idx)[:, None].expand(L, L)       # -(a1 - o) + o
    ok = (src2 < L)
    rot[:, ok] = imgs[:, src1[ok], src2[ok]]
    ref = torch.zeros_like(imgs)
    s1 = 2 * o - idx
    okr = s1 < L
    ref[:, okr, :] = imgs[:, s1[okr], :]
    a = as_complex(gp.expand(x))
    ar = as_complex(gp.expand(rot.to(dev)))
    af = as_complex(gp.expand(ref.to(dev)))
    kof = np.concatenate([np.full(pk, k) for k, pk in enumerate(gp.p)])
    assert rel(ar, a * np.exp(-1j * kof * math.pi / 2)) <= TOL
    assert rel(af, a.conj()) <= TOL


@pytest.mark.parametrize("L", [64, 128])
def test_fused_cluster_variant_equals_plain(dev, L, monkeypatch):
    """The grid kernel's two variants (the CTA pair of an image in a cluster
    sharing the row and column FFTs through distributed shared memory, or each
    CTA computing them alone) run the same arithmetic on the same values: the
    polar samples and the coefficients agree bit for bit."""
    gp = gplan(L)
    monkeypatch.setenv("FFB_FUSED_CLUSTER", "0")
    plain = Plan(L, 0.5, L / 2, eps=1e-6)
    monkeypatch.delenv("FFB_FUSED_CLUSTER")
    assert plain.polar_variant == 1 and gp.polar_variant in (1, 2)
    n = 2 * gp.chunk + 5      # two full launches and a ragged one
    imgs, _, _ = data.blob_stack(data.StackSpec(n, L, L / 2, 8, (1.5, 6.0), 0.2, 4242), device=dev)
    assert torch.equal(gp.polar(imgs[:7]), plain.polar(imgs[:7]))
    assert torch.equal(gp.expand(imgs), plain.expand(imgs))
    plain.close()


@pytest.mark.parametrize("which,samples", [
    ("fp32", (0, 151, 152, 607, 608, 9999, 12345, 19847, 19999)),
    ("precision", (0, 151, 152, 607, 608, 1215, 1216, 50000, 77777, 99847, 99999))])
def test_expand_full_size_l128_sampled(dev, which, samples):
    """Full-size L = 128 stacks in the benchmark's launch configuration:
    n = 20000 in FP32 and n = 100000 in BF16x3 (the headline precision, whose
    ring DFT runs on the tensor cores), sampled images against the oracle,
    at the first and last image and across chunk (152 images) and
    quadrature-group (608 images) boundaries."""
    spec = data.FP32_L128 if which == "fp32" else data.PRECISION_L128
    imgs, _, _ = data.blob_stack(spec, device=dev)
    gp = gplan(128) if which == "fp32" else gplan(128, precision="bf16x3")
    op = fb.make_plan(128, 0.5, 64.0)
    coef = gp.expand(imgs)
    torch.cuda.synchronize()
    a = as_complex(coef[list(samples)])
    ao = fb.expand(op, imgs[list(samples)].double().cpu().numpy())
    assert rel(a, ao) <= TOL
    assert torch.isfinite(coef).all()
    del coef, imgs
    torch.cuda.empty_cache()


# --- a6-a8: covariance and eigenpairs ------------------------------------------
def _oracle_cov(L, imgs):
    op = fb.make_plan(L, 0.5, L / 2)
    ao = fb.expand(op, imgs.double().numpy())
    mean0, blocks = fb.covariance(op, ao)
    return op, ao, mean0, blocks


def test_covariance_matches_oracle(dev):
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec)
    gp = gplan(spec.L)
    coef = gp.expand(imgs.to(dev))
    gp.covariance(coef, reset=True)
    mean, C = gp.cov_get()
    op, ao, mean0, blocks = _oracle_cov(spec.L, imgs)
    assert rel(mean.cpu().numpy(), mean0) <= TOL
    Cg = np.concatenate([b.ravel() for b in gp.unpack_blocks(C.cpu())])
    Co = np.concatenate([b.ravel() for b in blocks])
    assert rel(Cg, Co) <= TOL
    for k, (bg, bo) in enumerate(zip(gp.unpack_blocks(C.cpu()), blocks)):
        assert np.allclose(bg.numpy(), bg.numpy().T, atol=0)  # exactly symmetric
        assert np.linalg.norm(bg.numpy() - bo) <= 1e-4 * np.linalg.norm(bo) + 1e-12


def test_covariance_streaming_equals_one_call(dev):
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec)
    gp = gplan(spec.L)
    coef = gp.expand(imgs.to(dev))
    gp.covariance(coef, reset=True)
    m1, C1 = gp.cov_get()
    gp.covariance(coef[:77].contiguous(), reset=True)
    gp.covariance(coef[77:150].contiguous(), reset=False)
    gp.covariance(coef[150:].contiguous(), reset=False)
    m2, C2 = gp.cov_get()
    assert rel(C2.cpu().numpy(), C1.cpu().numpy()) < 1e-6
    assert rel(m2.cpu().numpy(), m1.cpu().numpy()) < 1e-6


def test_jacobi_on_exact_blocks(dev):
    """The float64 Jacobi solver alone, on the oracle's exact covariance
    blocks: eigenvalues and (gap-separated) eigenvectors vs numpy.eigh."""
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec)
    gp = gplan(spec.L)
    _, _, _, blocks = _oracle_cov(spec.L, imgs)
    packed = torch.tensor(np.concatenate([b.ravel() for b in blocks]), device=dev)
    ev, U = gp.eig_blocks(packed)
    lams, vecs = fb.eig_blocks(blocks)
    evn = ev.cpu().numpy()
    for k, (lam, V, Ug) in enumerate(zip(lams, vecs, gp.unpack_blocks(U.cpu()))):
        o, pk = gp.offset[k], gp.p[k]
        scale = max(abs(lam).max(), 1e-300)
        assert np.max(np.abs(evn[o:o + pk] - lam)) <= 1e-12 * scale
        Ug = Ug.numpy()
        assert np.max(np.abs(Ug.T @ Ug - np.eye(pk))) < 1e-12
        gaps = np.abs(np.diff(lam))
        for l in range(pk):
            gap = min(gaps[l - 1] if l > 0 else np.inf, gaps[l] if l < pk - 1 else np.inf)
            if gap > 1e-6 * scale:
                assert np.max(np.abs(Ug[:, l] - V[:, l])) < 1e-8


def test_eig_matches_oracle(dev):
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec)
    gp = gplan(spec.L)
    coef = gp.expand(imgs.to(dev))
    gp.covariance(coef, reset=True)
    ev, U = gp.eig()
    _, _, _, blocks = _oracle_cov(spec.L, imgs)
    lams, vecs = fb.eig_blocks(blocks)
    lam_all = np.concatenate(lams)
    evn = ev.cpu().numpy()
    assert rel(evn, lam_all) <= TOL
    top = np.argsort(-lam_all)[:20]
    assert np.max(np.abs(evn[top] - lam_all[top]) / lam_all[top]) <= TOL
    # top-20 eigenvectors: |<u_gpu, u_ref>| close to 1 where separated
    Ublocks = gp.unpack_blocks(U.cpu())
    for t in top:
        k = int(np.searchsorted(np.array(gp.offset), t, side="right") - 1)
        l = t - gp.offset[k]
        lam = lams[k]
        gap = min(abs(lam[l] - lam[l - 1]) if l > 0 else np.inf,
                  abs(lam[l] - lam[l + 1]) if l + 1 < lam.size else np.inf)
        if gap > 1e-2 * lam[0]:
            assert abs(abs(Ublocks[k][:, l].numpy() @ vecs[k][:, l]) - 1) < 1e-4


# --- error paths ---------------------------------------------------------------
def test_nonfinite_input_is_reported(dev):
    gp = gplan(32)
    x = torch.zeros((3, 32, 32), device=dev)
    x[1, 5, 7] = float("nan")
    gp.expand(x)
    with pytest.raises(FFBError) as e:
        gp.sync()
    assert e.value.status == -4
    gp.sync()   # the latch is cleared


def test_eig_before_covariance_is_state_error(dev):
    gp = Plan(16, 0.5, 8.0)
    with pytest.raises(FFBError) as e:
        gp.eig()
    assert e.value.status == -7
    gp.close()


def test_launch_count_grows(dev):
    gp = gplan(32)
    before = gp.launch_count()
    gp.expand(torch.zeros((5, 32, 32), device=dev))
    assert gp.launch_count() >= before + 4


def test_profile_stride_counts_every_launch(dev):
    """Sampled kernel timing: with a stride s only every s-th launch of a
    class is bracketed by events, but the launch count is complete and the
    class total is the sampled mean times that count."""
    gp = gplan(64)
    imgs = torch.zeros((5 * gp.chunk + 3, 64, 64), device=dev)
    gp.expand(imgs)
    torch.cuda.synchronize()
    for stride in (1, 4):
        gp.profile(True, stride=stride)
        gp.expand(imgs)
        torch.cuda.synchronize()
        prof = gp.profile_read()
        gp.profile(False)
        ms, calls = prof["grid_interp"]
        assert calls == 6 and ms > 0.0
    with pytest.raises(FFBError):
        gp.profile(True, stride=-1)


def test_cov_export_merge_import_roundtrip(dev):
    """Statistics of two disjoint halves pooled with ffb_cov_merge equal the
    statistics of the whole stack; importing them reproduces its eigenpairs."""
    from paper_1412_0781_gb300.ffb import cov_merge
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec)
    gp = gplan(spec.L)
    coef = gp.expand(imgs.to(dev))
    gp.covariance(coef, reset=True)
    full = gp.cov_export()
    ev_full, _ = gp.eig()
    gp.covariance(coef[:120].contiguous(), reset=True)
    s1 = gp.cov_export()
    gp.covariance(coef[120:].contiguous(), reset=True)
    s2 = gp.cov_export()
    pooled = cov_merge(gp.p, np.stack([s1, s2]))
    assert pooled[0] == full[0] == spec.n
    assert rel(pooled[1:], full[1:]) < 1e-6
    gp.cov_import(pooled)
    ev, _ = gp.eig()
    assert rel(ev.cpu().numpy(), ev_full.cpu().numpy()) < 1e-6
