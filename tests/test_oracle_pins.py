"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these re-runs the oracle's own formula: each compares with a library
special case (scipy / numpy), a value printed in the paper (tests/golden), a
closed form or identity, a group action, or brute force on a tiny input.
"""
import math
import os

import numpy as np
import pytest
import scipy.special as sp

from oracle import fb, special

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for ln in open(os.path.join(GOLDEN, name)):
        if ln.strip() and not ln.startswith("#"):
            key, val = ln.split()
            out[key] = float(val)
    return out


def _masked_noise(L, R, n, seed):
    rng = np.random.default_rng(seed)
    I = rng.standard_normal((n, L, L))
    idx = np.arange(L) - L // 2
    r2 = idx[:, None] ** 2 + idx[None, :] ** 2
    I[:, r2 >= R * R] = 0.0
    return I


# --- special functions ------------------------------------------------------
@pytest.mark.parametrize("k", [0, 1, 2, 7, 50, 183, 379])
def test_besselj_matches_scipy(k):
    x = np.linspace(0.0, 410.0, 1500)
    assert np.max(np.abs(special.besselj(k, x) - sp.jv(k, x))) < 5e-14


def test_besselj_identities():
    """Three-term recurrence J_{k-1} + J_{k+1} = (2k/x) J_k and Neumann's
    addition identity J_0^2 + 2 sum_k J_k^2 = 1 (no library involved)."""
    for x in (0.7, 33.3, 151.0, 395.5):
        ks = np.arange(0, 700)
        J = special.besselj(ks, np.full(ks.shape, x))
        rec = J[:-2] + J[2:] - 2 * ks[1:-1] / x * J[1:-1]
        assert np.max(np.abs(rec)) < 1e-13 * max(1.0, 400.0 / x)
        assert abs(J[0] ** 2 + 2 * np.sum(J[1:] ** 2) - 1.0) < 1e-14


@pytest.mark.parametrize("k", [0, 1, 10, 120])
def test_bessel_zeros_match_scipy(k):
    z = special.bessel_zeros(k, 410.0)
    ref = sp.jn_zeros(k, z.size)
    assert np.all(ref[-1] <= 410.0) and sp.jn_zeros(k, z.size + 1)[-1] > 410.0
    assert np.max(np.abs(z - ref) / ref) < 1e-14


@pytest.mark.parametrize("n", [16, 64, 128, 256])
def test_gauss_legendre(n):
    x, w = special.gauss_legendre(n)
    xl, wl = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xl)) < 1e-14
    assert np.max(np.abs(w - wl) / wl) < 1e-10       # numpy's own weights carry ~1e-11
    c = 0.5
    xc, wc = special.gauss_legendre(n, 0.0, c)
    for m in (0, 1, 7, n, 2 * n - 2, 2 * n - 1):   # exact for degree <= 2n-1
        exact = c ** (m + 1) / (m + 1)
        assert abs(np.sum(wc * xc ** m) - exact) <= 5e-14 * exact


# --- plan: sampling criterion and sizes (Sec. II-A, Alg. 1 step 1) ----------
def test_plan_sizes_golden():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "sizes.txt")) if not ln.startswith("#")]
    for row in rows:
        L = int(row[0])
        if L > 64:
            continue                      # larger plans are exercised in GPU tests
        p = fb.make_plan(L, 0.5, L / 2)
        assert (p.k_max, p.P, int(p.p[0] + 2 * p.p[1:].sum()), int(np.sum(p.p ** 2)),
                p.n_xi, p.n_theta) == tuple(int(float(v)) for v in row[2:])


@pytest.mark.parametrize("L", [32, 64])
def test_breen_bounds(L):
    """Eqs. kmaxbs and the total-count bounds 8(cR)^2 <= p <= 4 pi (cR)^2;
    per-k bounds of Eq. pkbs hold to +-1 (the derivation uses '~')."""
    c, R = 0.5, L / 2
    p = fb.make_plan(L, c, R)
    assert 4 * c * R - 3.517 < p.k_max < 2 * math.pi * c * R - 2.042
    tot = int(p.p[0] + 2 * p.p[1:].sum())
    assert 8 * (c * R) ** 2 <= tot <= 4 * math.pi * (c * R) ** 2
    for k, pk in enumerate(p.p):
        assert 2 * c * R - k / 2 - 3.035 / 4 - 1 < pk < 2 * c * R - k / math.pi + 1.4 / 4 + 1


def test_criterion_variants_differ_by_one_zero_per_k():
    lit = fb.make_plan(32, 0.5, 16.0, "literal")
    inc = fb.make_plan(32, 0.5, 16.0, "inclusive")
    assert inc.k_max >= lit.k_max
    assert np.all(inc.p[:lit.k_max + 1] == lit.p + 1)


def _gram_errors(p):
    """|2 pi sum_j N J_k(R_q xi_j/c) N J_k(R_q' xi_j/c) xi_j w_j - delta_qq'|
    per k (the exact integral of Eq. gint gives delta after normalisation)."""
    out = []
    for k in range(p.k_max + 1):
        NJ = p.B[k] / (p.xi * p.w)[None, :]
        G = 2 * math.pi * (NJ * (p.xi * p.w)[None, :]) @ NJ.T
        out.append(np.abs(G - np.eye(G.shape[0])))
    return out


def test_gram_identity():
    """Sec. II-B / Fig. 2a: the largest radial quadrature error is at
    k = 0, q1 = q2 = p_0, and it falls steeply with n_xi; at n_xi =
    ceil(4cR) it is at rounding level once R is large (R = 64 here), while a
    few extra nodes bring a small R (R = 32) to rounding level too."""
    p = fb.make_plan(64, 0.5, 32.0)
    E = _gram_errors(p)
    worst = max(e.max() for e in E)
    assert E[0][-1, -1] == worst                 # G(0, p_0, p_0) is the worst
    assert worst < 1e-7
    p_more = fb.make_plan(64, 0.5, 32.0, n_xi=p.n_xi + 12)
    assert max(e.max() for e in _gram_errors(p_more)) < 1e-13
    assert max(e.max() for e in _gram_errors(fb.make_plan(128, 0.5, 64.0))) < 1e-12


def test_worked_example_psi_1_5():
    """Sec. II-B: F f = psi^{1,5}, c = 0.5, R = 30 gives a_{1,5} = 1, all
    others 0, to RMSE 1.2e-16 and max error 2.7e-15 (golden values)."""
    g = _golden("worked_example_psi_1_5.txt")
    L = int(2 * g["R"])
    p = fb.make_plan(L, g["c"], g["R"])
    k, qi = int(g["k"]), int(g["q"]) - 1
    x1, x2 = p.polar_points()
    th = np.arctan2(x2, x1)
    radial = 1.0 / (p.c * math.sqrt(math.pi) * abs(sp.jv(k + 1, p.zeros[k][qi]))) \
        * sp.jv(k, p.zeros[k][qi] * p.xi / p.c)
    F = (radial[:, None] * np.exp(1j * k * th))[None]
    a = fb.coefficients_from_polar(p, F)[0]
    target = np.zeros(p.P, complex)
    target[p.offset[k] + qi] = 1.0
    err = np.abs(a - target)
    assert math.sqrt(np.mean(err ** 2)) <= 2 * g["rmse"]
    assert err.max() <= 2 * g["max_abs_err"]


# --- polar Fourier transform (Eq. nufft) -------------------------------------
def test_ndft_brute_force():
    """Direct evaluation of the double sum of Eq. nufft with explicit loops."""
    p = fb.make_plan(6, 0.5, 3.0)
    rng = np.random.default_rng(3)
    I = rng.standard_normal((2, 6, 6))
    F = fb.ndft_polar(p, I)
    x1, x2 = p.polar_points()
    idx = p.pixel_index()
    for (j, l) in [(0, 0), (1, 5), (p.n_xi - 1, p.n_theta - 1), (2, 7)]:
        for i in range(2):
            s = 0j
            for a in range(6):
                for b in range(6):
                    s += I[i, a, b] * complex(math.cos(-2 * math.pi * (x1[j, l] * idx[a] + x2[j, l] * idx[b])),
                                              math.sin(-2 * math.pi * (x1[j, l] * idx[a] + x2[j, l] * idx[b])))
            assert abs(F[i, j, l] - s) < 1e-13


@pytest.mark.parametrize("L", [8, 9])
def test_ndft_points_on_the_dft_grid_is_fft2(L):
    """At x = m / L the sum of Eq. nufft is the 2D DFT of the image: with
    i = a - floor(L/2), F(m/L) = fft2(I)[m] exp(2 pi i (m1 + m2) floor(L/2) / L)
    (library special case, even and odd L)."""
    rng = np.random.default_rng(4)
    I = rng.standard_normal((2, L, L))
    m1 = rng.integers(0, L, 12)
    m2 = rng.integers(0, L, 12)
    F = fb.ndft_points(I, m1 / L, m2 / L)
    ref = np.fft.fft2(I)[:, m1, m2] * np.exp(2j * math.pi * (m1 + m2) * (L // 2) / L)[None, :]
    assert np.max(np.abs(F - ref)) < 1e-12 * np.max(np.abs(ref))


def test_ndft_points_of_a_delta_and_polar_grid():
    """A single unit pixel at i0 has F(x) = exp(-2 pi i x . i0) (closed form);
    the plan-free polar grid has the full plan's radii and angles."""
    L = 10
    I = np.zeros((1, L, L))
    I[0, 7, 2] = 1.0                                  # i0 = (7 - 5, 2 - 5)
    rng = np.random.default_rng(5)
    x1, x2 = rng.uniform(-0.5, 0.5, 9), rng.uniform(-0.5, 0.5, 9)
    F = fb.ndft_points(I, x1, x2)[0]
    assert np.max(np.abs(F - np.exp(-2j * math.pi * (x1 * 2 + x2 * -3)))) < 1e-13
    p = fb.make_plan(16, 0.5, 8.0)
    xi, th = fb.polar_grid(0.5, p.n_xi, p.n_theta)
    assert np.array_equal(xi, p.xi)
    a, b = p.polar_points()
    assert np.max(np.abs(xi[:, None] * np.cos(th)[None, :] - a)) == 0.0
    assert np.max(np.abs(xi[:, None] * np.sin(th)[None, :] - b)) == 0.0


def test_ndft_hermitian_half_ring():
    """Real images: F(xi, theta + pi) = conj F(xi, theta)."""
    p = fb.make_plan(16, 0.5, 8.0)
    F = fb.ndft_polar(p, _masked_noise(16, 8, 2, 4))
    h = p.n_theta // 2
    assert np.max(np.abs(F[:, :, h:] - F[:, :, :h].conj())) < 1e-12


# --- whole forward map T* ----------------------------------------------------
def _rotate90(I):
    """I'(i1, i2) = I(i2, -i1): counter-clockwise rotation by pi/2."""
    n, L, _ = I.shape
    o = L // 2
    out = np.zeros_like(I)
    for a1 in range(L):
        for a2 in range(L):
            s1, s2 = (a2 - o), -(a1 - o)
            if -o <= s1 < L - o and -o <= s2 < L - o:
                out[:, a1, a2] = I[:, s1 + o, s2 + o]
    return out


def _reflect(I):
    """I'(i1, i2) = I(-i1, i2)."""
    n, L, _ = I.shape
    o = L // 2
    out = np.zeros_like(I)
    for a1 in range(L):
        s1 = -(a1 - o)
        if -o <= s1 < L - o:
            out[:, a1, :] = I[:, s1 + o, :]
    return out


def test_rotation_and_reflection():
    """Eqs. rot / refl: rotation by pi/2 multiplies a_{k,q} by e^{-i k pi/2};
    reflection x -> -x conjugates.  Exact on the grid when n_theta = 0 mod 4
    and the image vanishes for r >= R."""
    p = fb.make_plan(16, 0.5, 8.0)
    I = _masked_noise(16, 8, 3, 5)
    a = fb.expand(p, I)
    ar = fb.expand(p, _rotate90(I))
    af = fb.expand(p, _reflect(I))
    scale = np.max(np.abs(a))
    assert np.max(np.abs(ar - a * np.exp(-1j * p.k_of * math.pi / 2))) < 1e-13 * scale
    assert np.max(np.abs(af - a.conj())) < 1e-13 * scale


def _real_operator(p):
    """Q (p x L^2): T* with the k > 0 coefficients split into sqrt(2) Re and
    sqrt(2) Im, so that |Q x|^2 = |a|_W^2 (both +-k terms counted)."""
    L = p.L
    A = fb.expand(p, np.eye(L * L).reshape(L * L, L, L))
    p0 = p.p[0]
    return np.concatenate([A[:, :p0].real, math.sqrt(2) * A[:, p0:].real,
                           math.sqrt(2) * A[:, p0:].imag], axis=1).T, A


def test_near_unitary_spectrum():
    """Fig. 3: eigenvalues of T*T are mostly 1, none above 1 beyond the
    quadrature error, the smallest still close to 1."""
    p = fb.make_plan(24, 0.5, 12.0)
    Q, _ = _real_operator(p)
    ev = np.linalg.eigvalsh(Q @ Q.T)
    assert ev.max() < 1.0 + 1e-3
    assert abs(np.median(ev) - 1.0) < 1e-4
    assert np.mean(ev > 0.99) > 0.75
    assert ev.min() > 0.85


def test_bessel_inequality():
    p = fb.make_plan(16, 0.5, 8.0)
    I = np.random.default_rng(6).standard_normal((4, 16, 16))
    a = fb.expand(p, I)
    normW = np.sum(np.abs(a) ** 2 * p.weights_W()[None, :], axis=1)
    assert np.all(normW <= (1 + 1e-3) * np.sum(I ** 2, axis=(1, 2)))


# --- adjoint and synthesis ---------------------------------------------------
def test_adjoint_is_transpose_of_brute_force_matrix():
    p = fb.make_plan(12, 0.5, 6.0)
    _, A = _real_operator(p)                 # A[i, :] = T* e_i
    rng = np.random.default_rng(7)
    y = rng.standard_normal((2, p.P)) + 1j * rng.standard_normal((2, p.P))
    ref = (A.conj() @ y.T).real.T.reshape(2, 12, 12)   # Re(M^H y)
    assert np.max(np.abs(fb.adjoint(p, y) - ref)) < 1e-13 * np.max(np.abs(ref))


def test_adjoint_dot_product():
    p = fb.make_plan(16, 0.5, 8.0)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((3, 16, 16))
    y = rng.standard_normal((3, p.P)) + 1j * rng.standard_normal((3, p.P))
    lhs = np.sum((fb.expand(p, x).conj() * y).real, axis=1)
    rhs = np.sum(x * fb.adjoint(p, y), axis=(1, 2))
    assert np.max(np.abs(lhs - rhs) / np.abs(lhs)) < 1e-12


def test_synthesis_matches_analytic_inverse_transform():
    """S a = T(W a) is the polar quadrature of sum_k,q a_{k,q} F^{-1}(psi^{k,q});
    Eq. IFT_FB gives the same sum in closed form.  With the phase i^k that the
    inverse transform of Eq. IPFT produces they agree to the quadrature error;
    the phase printed in Eq. IFT_FB (i^-k) gives a different image."""
    p = fb.make_plan(16, 0.5, 8.0)
    rng = np.random.default_rng(9)
    a = rng.standard_normal((2, p.P)) + 1j * rng.standard_normal((2, p.P))
    a[:, :p.p[0]] = a[:, :p.p[0]].real
    s_quad = fb.synthesize(p, a)
    idx = p.pixel_index()
    inner = (idx[:, None] ** 2 + idx[None, :] ** 2) < (p.R / 2) ** 2
    scale = np.max(np.abs(s_quad))
    d_der = np.max(np.abs((s_quad - fb.synthesize_analytic(p, a, "derived"))[:, inner]))
    d_pr = np.max(np.abs((s_quad - fb.synthesize_analytic(p, a, "printed"))[:, inner]))
    assert d_der < 1e-3 * scale
    assert d_pr > 0.1 * scale


# --- steerable covariance and PCA (Sec. III, Alg. 2) -------------------------
def test_covariance_against_rotation_average_definition():
    """Eq. cov: C_{(k,q),(k',q')} = (1/4 pi n) sum_i int_0^{2pi}
    (a_{k,q} conj a_{k',q'} + a_{-k,q} conj a_{-k',q'}) e^{-i(k-k')alpha} d alpha,
    evaluated by brute force over the full +-k coefficient vector with an
    exact trapezoid rule in alpha; it must be block diagonal with the blocks
    of Eqs. ck / ck_0 (after the k = 0 mean is removed, Alg. 2 step 1)."""
    p = fb.make_plan(12, 0.5, 6.0)
    rng = np.random.default_rng(10)
    I = rng.standard_normal((7, 12, 12)) + 0.5
    a = fb.expand(p, I)
    n = a.shape[0]
    mean0, blocks = fb.covariance(p, a)
    ac = a.copy()
    ac[:, :p.p[0]] -= mean0[None, :]
    # full vector over k = -kmax..kmax: a_{-k,q} = conj(a_{k,q})
    ks, cols = [], []
    for k in range(-p.k_max, p.k_max + 1):
        o, pk = p.offset[abs(k)], p.p[abs(k)]
        for qi in range(pk):
            ks.append(k)
            cols.append(ac[:, o + qi] if k >= 0 else ac[:, o + qi].conj())
    ks = np.array(ks)
    Afull = np.stack(cols, axis=1)                       # (n, p)
    # index of (-k, q) for each (k, q)
    start = {k: int(np.argmax(ks == k)) for k in range(-p.k_max, p.k_max + 1)}
    neg = np.array([start[-k] + (i - start[k]) for i, k in enumerate(ks)])
    nalpha = 4 * p.k_max + 4
    alphas = 2 * math.pi * np.arange(nalpha) / nalpha
    C = np.zeros((ks.size, ks.size), dtype=complex)
    for al in alphas:
        ph = np.exp(-1j * (ks[:, None] - ks[None, :]) * al)
        M1 = Afull.T @ Afull.conj()
        M2 = Afull[:, neg].T @ Afull[:, neg].conj()
        C += (M1 + M2) * ph
    C *= (2 * math.pi / nalpha) / (4 * math.pi * n)
    for k in range(0, p.k_max + 1):
        sel = np.nonzero(ks == k)[0]
        assert np.max(np.abs(C[np.ix_(sel, sel)] - blocks[k])) < 1e-12
        other = np.nonzero(ks != k)[0]
        assert np.max(np.abs(C[np.ix_(sel, other)])) < 1e-12


def test_eigendecomposition_definition():
    p = fb.make_plan(16, 0.5, 8.0)
    a = fb.expand(p, np.random.default_rng(11).standard_normal((40, 16, 16)))
    _, blocks = fb.covariance(p, a)
    lams, vecs = fb.eig_blocks(blocks)
    for C, lam, U in zip(blocks, lams, vecs):
        assert np.all(np.diff(lam) <= 1e-15)
        assert np.max(np.abs(C @ U - U * lam[None, :])) < 1e-12 * max(1.0, np.abs(lam).max())
        assert np.max(np.abs(U.T @ U - np.eye(U.shape[1]))) < 1e-12
        piv = np.argmax(np.abs(U), axis=0)
        assert np.all(U[piv, np.arange(U.shape[1])] > 0)


def test_white_noise_marchenko_pastur():
    """Sec. V: for pure white noise every eigenvalue of C^(k) lies in
    sigma^2 (1 +- sqrt(gamma_k))^2 (gamma_0 = p_0/n, gamma_k = p_k/2n), up to
    finite-n fluctuation and the spread of T*T below 1."""
    p = fb.make_plan(24, 0.5, 12.0)
    n, sigma2 = 1500, 2.0
    I = math.sqrt(sigma2) * np.random.default_rng(12).standard_normal((n, 24, 24))
    _, blocks = fb.covariance(p, fb.expand(p, I))
    lams, _ = fb.eig_blocks(blocks)
    for k, lam in enumerate(lams):
        g = p.p[k] / n if k == 0 else p.p[k] / (2 * n)
        assert lam.max() < 1.05 * sigma2 * (1 + math.sqrt(g)) ** 2
        assert lam.min() > 0.85 * sigma2 * (1 - math.sqrt(g)) ** 2


def test_planted_component_recovered():
    """A rank-one signal s_i u planted in the k = 3 block of white coefficient
    noise is the top eigenvector of C^(3), eigenvalue ~ var(s) + sigma^2."""
    p = fb.make_plan(16, 0.5, 8.0)
    rng = np.random.default_rng(13)
    n = 4000
    a = (rng.standard_normal((n, p.P)) + 1j * rng.standard_normal((n, p.P))) / math.sqrt(2)
    a[:, :p.p[0]] = a[:, :p.p[0]].real * math.sqrt(2)
    o, pk = p.offset[3], p.p[3]
    u = rng.standard_normal(pk)
    u /= np.linalg.norm(u)
    s = 3.0 * (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2)
    a[:, o:o + pk] += s[:, None] * u[None, :]
    _, blocks = fb.covariance(p, a)
    lams, vecs = fb.eig_blocks(blocks)
    assert abs(abs(vecs[3][:, 0] @ u) - 1.0) < 1e-2
    assert abs(lams[3][0] - (9.0 + 1.0)) < 0.6


def test_topk_and_mp_selection():
    p = fb.make_plan(16, 0.5, 8.0)
    lams = [np.sort(np.random.default_rng(k).uniform(0, 10, pk))[::-1] for k, pk in enumerate(p.p)]
    hs = fb.select_filter(p, lams, "topk", K=7)
    kept = sorted([(-lams[k][l], k, l) for k in range(len(lams)) for l in range(lams[k].size)])[:7]
    assert sum(int(h.sum()) for h in hs) == 7
    for _, k, l in kept:
        assert hs[k][l] == 1.0
    hs = fb.select_filter(p, lams, "mp_wiener", sigma2=4.0, n=100)
    for k, (lam, h) in enumerate(zip(lams, hs)):
        g = p.p[k] / 100 if k == 0 else p.p[k] / 200
        thr = 4.0 * (1 + math.sqrt(g)) ** 2
        assert np.all((h > 0) == (lam > thr))
        assert np.allclose(h[lam > thr], 1 - 4.0 / lam[lam > thr])


def test_denoise_all_components_is_projection():
    """With every component kept (h = 1) the filter is the identity on the
    coefficients (mean removed then added back), so denoise = S T*."""
    p = fb.make_plan(16, 0.5, 8.0)
    I = _masked_noise(16, 8, 30, 14) + 1.0
    out = fb.denoise(p, I, "all")
    ref = fb.synthesize(p, fb.expand(p, I))
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))


def test_svd_route_equals_covariance_eigenpairs():
    """Sec. III: the left singular vectors of A^(k) are the eigenvectors of
    C^(k) and s^2/n its eigenvalues.  The oracle's SVD route (LAPACK SVD of the
    stacked real matrix) against its covariance route (two-pass covariance,
    LAPACK symmetric eigensolver): two different algorithms on the same data."""
    plan = fb.make_plan(24, 0.5, 12.0)
    rng = np.random.default_rng(8)
    n = 90
    a = rng.standard_normal((n, plan.P)) + 1j * rng.standard_normal((n, plan.P))
    a *= np.linspace(2.0, 0.5, plan.P)[None, :]
    a[:, :plan.p[0]] = a[:, :plan.p[0]].real + 0.3
    _, blocks = fb.covariance(plan, a)
    lc, uc = fb.eig_blocks(blocks)
    ls, us = fb.svd_route(plan, a)
    for k in range(len(plan.p)):
        assert np.max(np.abs(lc[k] - ls[k])) <= 1e-12 * max(1.0, lc[k].max())
        # compare the spectral projectors (robust to near-degenerate pairs)
        Pc = uc[k] @ np.diag(lc[k]) @ uc[k].T
        Ps = us[k] @ np.diag(ls[k]) @ us[k].T
        assert np.max(np.abs(Pc - Ps)) <= 1e-12 * max(1.0, lc[k].max())


def test_invariant_features_under_rotation_and_reflection():
    """Exact 90-degree rotations and the reflection of the grid (Eqs. rot, refl)
    leave the power spectrum of the steerable coefficients unchanged and
    leave (rotation) or conjugate (reflection) the bispectrum -- checked on the
    images themselves, through the whole expansion."""
    L = 24
    plan = fb.make_plan(L, 0.5, L / 2)
    I = _masked_noise(L, L // 2, 40, 21)
    a = fb.expand(plan, I)
    mean0, blocks = fb.covariance(plan, a)
    _, vecs = fb.eig_blocks(blocks)
    pairs = [(0, 0), (1, 0), (2, 1), (5, 0)]
    triples = [(1, 0, 1, 0, 0), (1, 0, 2, 1, 0), (2, 0, 3, 0, 1), (0, 1, 4, 0, 0)]
    pw, bs = fb.invariant_features(plan, a, mean0, vecs, pairs, triples)
    ar = fb.expand(plan, _rotate90(I))                     # exact on the pixel grid
    pwr, bsr = fb.invariant_features(plan, ar, mean0, vecs, pairs, triples)
    assert np.max(np.abs(pwr - pw)) <= 1e-10 * np.max(np.abs(pw))
    assert np.max(np.abs(bsr - bs)) <= 1e-10 * np.max(np.abs(bs))
    af = fb.expand(plan, _reflect(I))
    pwf, bsf = fb.invariant_features(plan, af, mean0, vecs, pairs, triples)
    assert np.max(np.abs(pwf - pw)) <= 1e-10 * np.max(np.abs(pw))
    assert np.max(np.abs(bsf - np.conj(bs))) <= 1e-10 * np.max(np.abs(bs))


# --- radial eigenfunctions, selection and filtering (Eqs. sPCArad, sPCAcoeff,
# --- compselect; Sec. V): pins that do not pass through the oracle's formulas
def test_radial_eigenfunctions_of_identity_are_the_basis_radial_parts():
    """With U^(k) = I the radial eigenfunctions are the radial parts of the
    Fourier-Bessel basis itself, N_{k,q} J_k(R_{k,q} xi / c) with
    N_{k,q} = 1 / (c sqrt(pi) |J_{k+1}(R_{k,q})|) (Sec. II-A), evaluated here
    with SciPy's Bessel functions and zeros at the Gauss-Legendre nodes of
    numpy.  A quadrature factor xi_j w_j left in, or a wrong normalisation,
    fails this."""
    L, c, R = 32, 0.5, 16.0
    plan = fb.make_plan(L, c, R)
    xi, _ = np.polynomial.legendre.leggauss(plan.n_xi)
    xi = 0.5 * c * (xi + 1.0)
    f = fb.radial_eigenfunctions(plan, [np.eye(pk) for pk in plan.p])
    for k, pk in enumerate(plan.p):
        z = sp.jn_zeros(k, pk)
        ref = sp.jv(k, z[None, :] * xi[:, None] / c) / (c * math.sqrt(math.pi) * np.abs(sp.jv(k + 1, z)))[None, :]
        assert f[k].shape == (plan.n_xi, pk)
        assert np.max(np.abs(f[k] - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_radial_eigenfunctions_are_orthonormal_on_the_disk():
    """For any orthogonal U^(k) the functions f^{k,l}(xi) e^{ik theta} are
    orthonormal on the disk of radius c: 2 pi int_0^c f f' xi dxi = delta
    (orthonormality of the Fourier-Bessel basis, Fig. 2a).  The integral is
    taken with 64 extra Gauss-Legendre nodes on [0, c] (numpy's rule), where
    its error is at rounding level, so the check is against the mathematics,
    not against the plan's own quadrature."""
    L, c, R = 48, 0.5, 24.0
    base = fb.make_plan(L, c, R)
    fine = fb.Plan(L, c, R, n_xi=base.n_xi + 64)
    t, wt = np.polynomial.legendre.leggauss(fine.n_xi)
    xi, w = 0.5 * c * (t + 1.0), 0.5 * c * wt
    rng = np.random.default_rng(31)
    vecs = [np.linalg.qr(rng.standard_normal((pk, pk)))[0] for pk in fine.p]
    f = fb.radial_eigenfunctions(fine, vecs)
    for k in (0, 1, 5, len(fine.p) // 2, len(fine.p) - 1):
        G = 2.0 * math.pi * (f[k] * (xi * w)[:, None]).T @ f[k]
        assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-11


class _Sizes:
    """Stand-in for a plan where a rule needs only the block sizes p_k."""

    def __init__(self, p):
        self.p = np.asarray(p, dtype=np.int64)


def test_mp_selection_worked_example():
    """Eq. compselect worked by hand for p = (25, 16, 9), n = 100, sigma^2 = 1:
    gamma_0 = p_0/n = 0.25 gives the edge (1 + 0.5)^2 = 2.25; gamma_1 =
    p_1/(2n) = 0.08 gives (1 + 0.28284)^2 = 1.64569; gamma_2 = 0.045 gives
    (1 + 0.21213)^2 = 1.46926.  The eigenvalues below sit on both sides of
    each edge and also on both sides of the edges that a wrong gamma
    (p_0/(2n) for k = 0: 1.832; p_k/n for k > 0: 1.96 and 1.69) would give."""
    lams = [np.array([3.0, 2.3, 2.2] + [1.0] * 22),
            np.array([1.7, 1.6] + [0.9] * 14),
            np.array([1.5, 1.45] + [0.8] * 7)]
    hs = fb.select_filter(_Sizes([25, 16, 9]), lams, "mp_wiener", sigma2=1.0, n=100)
    expect = [{0: 2.0 / 3.0, 1: 1.3 / 2.3}, {0: 0.7 / 1.7}, {0: 0.5 / 1.5}]
    for k in range(3):
        for l in range(lams[k].size):
            assert hs[k][l] == pytest.approx(expect[k].get(l, 0.0), abs=1e-15)
    hs = fb.select_filter(_Sizes([25, 16, 9]), lams, "mp_hard", sigma2=1.0, n=100)
    for k in range(3):
        assert sorted(np.flatnonzero(hs[k])) == sorted(expect[k])
        assert np.all(hs[k][list(expect[k])] == 1.0)


def test_topk_selection_worked_example():
    """Ranking of (k, l) pairs by eigenvalue with ties to the smaller k, then
    the smaller l, worked by hand on three blocks."""
    lams = [np.array([5.0, 1.0]), np.array([7.0, 3.0, 3.0]), np.array([5.0, 0.5])]
    order = [(1, 0), (0, 0), (2, 0), (1, 1), (1, 2), (0, 1), (2, 1)]
    for K in range(len(order) + 1):
        hs = fb.select_filter(_Sizes([2, 3, 2]), lams, "topk", K=K)
        kept = {(k, l) for k in range(3) for l in range(lams[k].size) if hs[k][l] == 1.0}
        assert kept == set(order[:K])
        assert sum(int(np.count_nonzero(h)) for h in hs) == K


def test_mp_selection_keeps_exactly_the_planted_components():
    """Spiked white-noise model (Sec. V): coefficients of white noise of
    variance sigma^2 (real for k = 0, complex with E|a|^2 = sigma^2 for k > 0)
    plus rank-one signals planted in three blocks.  The noise eigenvalues stay
    below the Marchenko-Pastur edge and the spikes lie far above it, so the
    selection must keep exactly the planted (k, l), and the Wiener gain must be
    close to the population value s / (s + sigma^2)."""
    p = [9, 12, 7, 5]
    n, sigma2 = 6000, 1.5
    rng = np.random.default_rng(37)
    planted = {0: 2.0, 1: 3.0, 3: 1.5}
    lams = []
    for k, pk in enumerate(p):
        if k == 0:
            A = math.sqrt(sigma2) * rng.standard_normal((n, pk))
        else:
            A = math.sqrt(sigma2 / 2) * (rng.standard_normal((n, pk)) + 1j * rng.standard_normal((n, pk)))
        if k in planted:
            u = rng.standard_normal(pk)
            u /= np.linalg.norm(u)
            s = rng.standard_normal(n) if k == 0 else (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2)
            A = A + math.sqrt(planted[k]) * s[:, None] * u[None, :]
        C = (A.real.T @ A.real + A.imag.T @ A.imag) / n
        lams.append(np.sort(np.linalg.eigvalsh(C))[::-1])
    hs = fb.select_filter(_Sizes(p), lams, "mp_wiener", sigma2=sigma2, n=n)
    for k in range(len(p)):
        kept = list(np.flatnonzero(hs[k]))
        assert kept == ([0] if k in planted else [])
        if k in planted:
            assert hs[k][0] == pytest.approx(planted[k] / (planted[k] + sigma2), abs=0.05)


def _planted_coefficients(plan, n, rng, mean_scale=2.0):
    a = rng.standard_normal((n, plan.P)) + 1j * rng.standard_normal((n, plan.P))
    a[:, :plan.p[0]] = a[:, :plan.p[0]].real
    m = mean_scale * rng.standard_normal(plan.p[0])
    a[:, :plan.p[0]] += m[None, :]
    return a, m


def test_filter_with_signed_permutation_eigenvectors():
    """Closed form of Eq. sPCAcoeff and the filter when every U^(k) is a signed
    permutation (u_l = s_l e_{pi(l)}): the steerable coefficient c_{k,l} is
    s_l (a - m)_{pi(l)}, and the filtered coefficient q is
    h_{pi^-1(q)} (a - m)_q + m_q, whatever the signs.  The k = 0 mean m is
    nonzero and the gains are distinct and not 0 or 1."""
    plan = fb.make_plan(16, 0.5, 8.0)
    rng = np.random.default_rng(41)
    a, m = _planted_coefficients(plan, 7, rng)
    vecs, perms, signs, hs = [], [], [], []
    for pk in plan.p:
        pi = rng.permutation(pk)
        s = rng.choice([-1.0, 1.0], pk)
        U = np.zeros((pk, pk))
        U[pi, np.arange(pk)] = s
        vecs.append(U)
        perms.append(pi)
        signs.append(s)
        hs.append(rng.uniform(0.1, 0.9, pk))
    cs = fb.steerable_coefficients(plan, a, m, vecs)
    out = fb.filter_coefficients(plan, a, m, vecs, hs)
    for k, (o, pk) in enumerate(zip(plan.offset, plan.p)):
        x = a[:, o:o + pk] - (m[None, :] if k == 0 else 0.0)
        assert np.allclose(cs[k], signs[k][None, :] * x[:, perms[k]], rtol=0, atol=1e-14)
        inv = np.argsort(perms[k])
        ref = hs[k][inv][None, :] * x + (m[None, :] if k == 0 else 0.0)
        assert np.allclose(out[:, o:o + pk], ref, rtol=0, atol=1e-13)


def test_filter_against_dense_operator_on_the_full_coefficient_vector():
    """Brute force over the full coefficient vector a_{k,q}, k = -k_max..k_max
    (a_{-k,q} = conj a_{k,q} for a real image): one dense matrix
    F = blockdiag_k U^(|k|) diag(h^(|k|)) U^(|k|)T acting on a - m, plus m,
    where m is the k = 0 mean.  The +k part must equal the oracle's filtered
    coefficients and the -k part their conjugate (the filtered image stays
    real).  Eigenvectors are random orthogonal, gains random in (0, 1)."""
    import scipy.linalg as sla
    plan = fb.make_plan(16, 0.5, 8.0)
    rng = np.random.default_rng(43)
    a, m = _planted_coefficients(plan, 5, rng)
    vecs = [np.linalg.qr(rng.standard_normal((pk, pk)))[0] for pk in plan.p]
    hs = [rng.uniform(0.0, 1.0, pk) for pk in plan.p]
    K = len(plan.p) - 1
    ks = list(range(-K, K + 1))
    blocks = [vecs[abs(k)] @ np.diag(hs[abs(k)]) @ vecs[abs(k)].T for k in ks]
    F = sla.block_diag(*blocks)
    full = np.concatenate([np.conj(a[:, plan.offset[-k]:plan.offset[-k] + plan.p[-k]]) if k < 0
                           else a[:, plan.offset[k]:plan.offset[k] + plan.p[k]] for k in ks], axis=1)
    mfull = np.zeros(full.shape[1])
    z = int(sum(plan.p[abs(k)] for k in ks if k < 0))
    mfull[z:z + plan.p[0]] = m
    den = (full - mfull[None, :]) @ F.T + mfull[None, :]
    out = fb.filter_coefficients(plan, a, m, vecs, hs)
    pos, neg = den[:, z:], den[:, :z]
    assert np.max(np.abs(pos - out)) <= 1e-13 * np.max(np.abs(out))
    for k in range(1, K + 1):
        o = plan.offset[k]
        start = z - int(sum(plan.p[1:k + 1]))
        assert np.max(np.abs(neg[:, start:start + plan.p[k]] - np.conj(out[:, o:o + plan.p[k]]))) < 1e-13


def test_filter_zero_gain_returns_the_mean_and_unit_gain_the_input():
    """h = 0 removes every component: the result is the k = 0 mean and zero
    for k > 0.  h = 1 keeps all of them: the result is the input itself (the
    mean is removed and added back).  Both with a nonzero mean."""
    plan = fb.make_plan(16, 0.5, 8.0)
    rng = np.random.default_rng(47)
    a, m = _planted_coefficients(plan, 6, rng, mean_scale=5.0)
    vecs = [np.linalg.qr(rng.standard_normal((pk, pk)))[0] for pk in plan.p]
    zero = fb.filter_coefficients(plan, a, m, vecs, [np.zeros(pk) for pk in plan.p])
    assert np.max(np.abs(zero[:, :plan.p[0]] - m[None, :])) < 1e-14
    assert np.max(np.abs(zero[:, plan.p[0]:])) == 0.0
    one = fb.filter_coefficients(plan, a, m, vecs, [np.ones(pk) for pk in plan.p])
    assert np.max(np.abs(one - a)) < 1e-13 * np.max(np.abs(a))


def test_steerable_coefficients_recover_planted_components():
    """Images built as a = m + sum_l t_{i,l} u_l in each block (u_l orthonormal,
    m the k = 0 mean) have steerable coefficients exactly t (Eq. sPCAcoeff
    with the k = 0 centring of Alg. 2 step 1); the covariance of the same
    stack, built with the oracle's own mean, reproduces m."""
    plan = fb.make_plan(16, 0.5, 8.0)
    rng = np.random.default_rng(53)
    n = 40
    m = 3.0 * rng.standard_normal(plan.p[0])
    vecs = [np.linalg.qr(rng.standard_normal((pk, pk)))[0] for pk in plan.p]
    a = np.zeros((n, plan.P), complex)
    ts = []
    for k, (o, pk) in enumerate(zip(plan.offset, plan.p)):
        t = rng.standard_normal((n, pk))
        if k == 0:
            t -= t.mean(axis=0)            # the planted components have zero mean
        else:
            t = t + 1j * rng.standard_normal((n, pk))
        ts.append(t)
        a[:, o:o + pk] = t @ vecs[k].T + (m[None, :] if k == 0 else 0.0)
    mean0, _ = fb.covariance(plan, a)
    assert np.max(np.abs(mean0 - m)) < 1e-13 * np.max(np.abs(m))
    cs = fb.steerable_coefficients(plan, a, mean0, vecs)
    for k in range(len(plan.p)):
        assert np.max(np.abs(cs[k] - ts[k])) < 1e-12
