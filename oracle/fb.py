"""FP64 oracle of the fast Fourier-Bessel expansion and steerable PCA
(test infrastructure only; see ``oracle/__init__.py``).

Notation follows the paper: images I(i1, i2) on the pixel grid
i = -ceil((L-1)/2) .. floor((L-1)/2) (Sec. II), band limit c, support radius
R, Bessel zeros R_{k,q}, Gauss-Legendre nodes xi_j with weights w_j on [0, c],
angles theta_l = 2 pi l / n_theta, coefficients a_{k,q} for k >= 0.

Readings taken where the paper is silent or inconsistent (each is listed in
the design notes of the repository):
* the 1/(2R)^2 factor printed in Eq. nufft is dropped, so that T* is close to
  unitary as Fig. 3 and the noise model of Sec. V require;
* the sampling criterion is the literal R_{k,q+1} <= 2 pi c R (Eq. criterion1);
* Im a_{0,q} is set to zero after the quadrature (real images, Sec. II-B);
* covariances are normalised by 1/n (Eq. ck);
* coefficient inner product <u, v> = Re sum_{k>=0,q} conj(u) v; the adjoint of
  the expansion T* is T y = Re(M^H y) and the synthesis of a full real image is
  S a = T(W a) with W = 1 for k = 0 and 2 for k > 0.
"""
import math
from functools import lru_cache

import numpy as np

from .special import besselj, bessel_zeros, gauss_legendre


# ----------------------------------------------------------------------------
# Plan: sampling criterion, quadrature sizes, radial tables (Alg. 1 steps 1-2)
# ----------------------------------------------------------------------------
class Plan:
    """Precomputed quantities of Alg. 1 steps 1-2 for one (L, c, R)."""

    def __init__(self, L, c, R, criterion="literal", n_xi=None, n_theta=None):
        if not (L >= 4 and 0.0 < c <= 0.5 and 0.0 < R <= L / 2.0):
            raise ValueError("need L >= 4, 0 < c <= 1/2, 0 < R <= L/2")
        self.L, self.c, self.R = int(L), float(c), float(R)
        X = 2.0 * math.pi * c * R          # right-hand side of Eq. criterion1
        zeros, p = [], []
        k = 0
        while True:
            z = bessel_zeros(k, X)
            if criterion == "literal":      # R_{k,q+1} <= 2 pi c R
                pk = max(0, z.size - 1)
            elif criterion == "inclusive":  # R_{k,q} <= 2 pi c R
                pk = z.size
            else:
                raise ValueError(criterion)
            if pk == 0:
                break
            zeros.append(z[:pk])
            p.append(pk)
            k += 1
        self.k_max = len(p) - 1
        self.p = np.array(p, dtype=np.int64)
        self.offset = np.concatenate([[0], np.cumsum(self.p)[:-1]]).astype(np.int64)
        self.P = int(self.p.sum())
        self.zeros = zeros
        # Alg. 1 step 1: n_xi = ceil(4cR), n_theta = ceil(16cR); Fig. 2 varies
        # both, so they can be overridden
        self.n_xi = int(math.ceil(4.0 * c * R - 1e-9)) if n_xi is None else int(n_xi)
        self.n_theta = int(math.ceil(16.0 * c * R - 1e-9)) if n_theta is None else int(n_theta)
        # Alg. 1 step 2: Gauss-Legendre rule on [0, c] ...
        self.xi, self.w = gauss_legendre(self.n_xi, 0.0, c)
        # ... and B^(k)_{q,j} = N_{k,q} J_k(R_{k,q} xi_j / c) xi_j w_j  (Eq. a)
        kk = np.concatenate([np.full(pk, kq) for kq, pk in enumerate(p)])
        rr = np.concatenate(zeros)
        self.norm = 1.0 / (c * math.sqrt(math.pi) * np.abs(besselj(kk + 1, rr)))
        Jtab = besselj(kk[:, None], rr[:, None] * self.xi[None, :] / c)
        Ball = self.norm[:, None] * Jtab * (self.xi * self.w)[None, :]
        self.B = [Ball[o:o + pk] for o, pk in zip(self.offset, self.p)]
        self.k_of = kk                       # angular index of each coefficient
        self._nd = None

    # pixel index i = -ceil((L-1)/2) .. floor((L-1)/2)  (Sec. II)
    def pixel_index(self):
        return np.arange(self.L, dtype=np.float64) - (self.L // 2)

    def polar_points(self):
        """xi1 = xi_j cos(theta_l), xi2 = xi_j sin(theta_l), shape (n_xi, n_theta)."""
        th = 2.0 * math.pi * np.arange(self.n_theta) / self.n_theta
        return (self.xi[:, None] * np.cos(th)[None, :],
                self.xi[:, None] * np.sin(th)[None, :])

    def weights_W(self):
        """W = 1 on k = 0 coefficients, 2 on k > 0 (both +k and -k terms)."""
        return np.where(self.k_of == 0, 1.0, 2.0)

    def _ndft_factors(self):
        if self._nd is None:
            x1, x2 = self.polar_points()
            idx = self.pixel_index()
            U = np.exp(-2j * math.pi * x1.reshape(-1, 1) * idx[None, :])
            V = np.exp(-2j * math.pi * x2.reshape(-1, 1) * idx[None, :])
            self._nd = (U, V)
        return self._nd


@lru_cache(maxsize=8)
def make_plan(L, c, R, criterion="literal", n_xi=None, n_theta=None):
    return Plan(L, c, R, criterion, n_xi, n_theta)


# ----------------------------------------------------------------------------
# Forward map a = T* I   (Eqs. nufft, 1DFFT, a)
# ----------------------------------------------------------------------------
def ndft_polar(plan, images, batch=4):
    """F(I)(xi1, xi2) = sum_{i1,i2} I(i1,i2) exp(-2 pi i (xi1 i1 + xi2 i2))
    at every polar node (all n_theta angles), by the direct non-uniform DFT
    (Eq. nufft without the 1/(2R)^2 factor).  The exponential splits into
    u(i1) v(i2), so the double sum is sum_{i1} u(i1) sum_{i2} I(i1,i2) v(i2).
    Returns complex (n, n_xi, n_theta)."""
    images = np.asarray(images, dtype=np.float64)
    n, L = images.shape[0], plan.L
    U, V = plan._ndft_factors()
    out = np.empty((n, U.shape[0]), dtype=np.complex128)
    for s in range(0, n, batch):
        blk = images[s:s + batch]                       # (b, L, L)
        b = blk.shape[0]
        UI = U @ blk.transpose(1, 0, 2).reshape(L, b * L)   # (M, b*L)
        UI = UI.reshape(-1, b, L)
        out[s:s + b] = np.einsum("mbj,mj->bm", UI, V)
    return out.reshape(n, plan.n_xi, plan.n_theta)


def polar_grid(c, n_xi, n_theta):
    """The polar nodes without the Bessel tables of a full plan (for sizes
    whose plan takes too long here): Gauss-Legendre radii xi_j on [0, c]
    (Alg. 1 step 2) and angles theta_l = 2 pi l / n_theta (Sec. III).
    Returns (xi, theta), both float64."""
    xi, _ = gauss_legendre(int(n_xi), 0.0, float(c))
    return xi, 2.0 * math.pi * np.arange(int(n_theta)) / int(n_theta)


def ndft_points(images, x1, x2):
    """F(I)(x1, x2) = sum_{i1,i2} I(i1,i2) exp(-2 pi i (x1 i1 + x2 i2)) at
    arbitrary frequency points (the definition inside Eq. nufft, without the
    1/(2R)^2 factor), one point at a time as u^T I v with u(i1), v(i2) the
    two exponential factors.  images (n, L, L), x1, x2 (m,) -> complex (n, m)."""
    images = np.asarray(images, dtype=np.float64)
    L = images.shape[-1]
    idx = np.arange(L, dtype=np.float64) - (L // 2)     # i = -ceil((L-1)/2) .. (Sec. II)
    out = np.empty((images.shape[0], len(x1)), dtype=np.complex128)
    for t, (a, b) in enumerate(zip(x1, x2)):
        u = np.exp(-2j * math.pi * float(a) * idx)
        v = np.exp(-2j * math.pi * float(b) * idx)
        out[:, t] = np.einsum("i,nij,j->n", u, images, v)
    return out


def ring_dft_matrix(plan):
    """E[l, k] = (2 pi / n_theta) exp(-2 pi i k l / n_theta), k = 0..k_max."""
    l = np.arange(plan.n_theta)[:, None]
    k = np.arange(plan.k_max + 1)[None, :]
    return (2.0 * math.pi / plan.n_theta) * np.exp(-2j * math.pi * k * l / plan.n_theta)


def ring_dft(plan, F):
    """F^(xi_j, k) = (2pi/n_theta) sum_l F(xi_j, theta_l) e^{-2 pi i k l/n_theta}
    (Eq. 1DFFT) as the plain sum.  F: (n, n_xi, n_theta) -> (n, n_xi, k_max+1)."""
    return F @ ring_dft_matrix(plan)


def radial_quadrature(plan, Fhat):
    """a_{k,q} = sum_j N_{k,q} J_k(R_{k,q} xi_j/c) F^(xi_j, k) xi_j w_j
    (Eq. a).  Fhat: (n, n_xi, k_max+1) -> a: (n, P), k ascending, q ascending."""
    n = Fhat.shape[0]
    a = np.empty((n, plan.P), dtype=np.complex128)
    for k, (o, pk) in enumerate(zip(plan.offset, plan.p)):
        a[:, o:o + pk] = Fhat[:, :, k] @ plan.B[k].T
    a[:, :plan.p[0]] = a[:, :plan.p[0]].real       # a_{0,q} is real
    return a


def coefficients_from_polar(plan, F):
    """Alg. 1 step 4 given the polar samples F (n, n_xi, n_theta)."""
    return radial_quadrature(plan, ring_dft(plan, F))


def expand(plan, images):
    """a = T* I (Alg. 1 steps 3-4), images (n, L, L) -> a (n, P) complex."""
    return coefficients_from_polar(plan, ndft_polar(plan, images))


# ----------------------------------------------------------------------------
# Adjoint T and synthesis S = T W
# ----------------------------------------------------------------------------
def adjoint(plan, y, batch=4):
    """T y = Re(M^H y), the adjoint of ``expand`` for the inner products
    <u, v> = Re sum conj(u) v on coefficients and sum x y on images.  Steps:
    transposed quadrature, conjugate-transposed ring DFT, adjoint NDFT
    (exp(+2 pi i xi . i)), real part.  y: (n, P) complex -> (n, L, L)."""
    y = np.asarray(y, dtype=np.complex128)
    n, L = y.shape[0], plan.L
    Ghat = np.zeros((n, plan.n_xi, plan.k_max + 1), dtype=np.complex128)
    for k, (o, pk) in enumerate(zip(plan.offset, plan.p)):
        Ghat[:, :, k] = y[:, o:o + pk] @ plan.B[k]
    G = Ghat @ ring_dft_matrix(plan).conj().T          # (n, n_xi, n_theta)
    G = G.reshape(n, -1)
    U, V = plan._ndft_factors()
    Uc, Vc = U.conj(), V.conj()
    out = np.empty((n, L, L))
    for i in range(n):
        out[i] = ((Uc * G[i][:, None]).T @ Vc).real
    return out


def synthesize(plan, a):
    """Real image of the truncated expansion (Eq. contapprox), S a = T(W a)."""
    return adjoint(plan, np.asarray(a) * plan.weights_W()[None, :])


def ift_fb(plan, k, q_index, r, phase="derived"):
    """Inverse Fourier transform of psi_c^{k,q} at radius r (without the
    e^{i k phi} factor), Eq. IFT_FB:
        2 c sqrt(pi) (-1)^q R_{k,q} J_k(2 pi c r) s_k / ((2 pi c r)^2 - R_{k,q}^2)
    with s_k = i^k when derived from the inverse transform convention of
    Eq. IPFT (Jacobi-Anger), or s_k = i^{-k} as the equation is printed.
    ``q_index`` is 0-based (q = q_index + 1)."""
    c = plan.c
    Rkq = plan.zeros[k][q_index]
    q = q_index + 1
    z = 2.0 * math.pi * c * np.asarray(r, dtype=np.float64)
    Jk = besselj(k, z)
    den = z * z - Rkq * Rkq
    near = np.abs(z - Rkq) < 1e-7
    # removable singularity: R J_k(z)/(z^2-R^2) -> J_k'(R)/2 = -J_{k+1}(R)/2
    ratio = np.where(near, -besselj(k + 1, Rkq) / 2.0,
                     Rkq * Jk / np.where(near, 1.0, den))
    s = (1j) ** k if phase == "derived" else (1j) ** (-k)
    return 2.0 * c * math.sqrt(math.pi) * (-1.0) ** q * s * ratio


def synthesize_analytic(plan, a, phase="derived"):
    """f(i) = sum_{k=-kmax}^{kmax} sum_q a_{k,q} F^{-1}(psi^{k,q})(r, phi) on the
    pixel grid (Eq. IFT_FB, the route of Sec. V for eigenimages), using
    a_{-k,q} = conj(a_{k,q}) so the +-k pair contributes 2 Re(.)."""
    a = np.asarray(a, dtype=np.complex128)
    idx = plan.pixel_index()
    X1, X2 = np.meshgrid(idx, idx, indexing="ij")
    r = np.hypot(X1, X2)
    phi = np.arctan2(X2, X1)
    out = np.zeros((a.shape[0], plan.L, plan.L))
    for k, (o, pk) in enumerate(zip(plan.offset, plan.p)):
        wk = 1.0 if k == 0 else 2.0
        ang = np.exp(1j * k * phi)
        for qi in range(pk):
            g = ift_fb(plan, k, qi, r, phase) * ang
            out += wk * (a[:, o + qi, None, None] * g[None]).real
    return out


# ----------------------------------------------------------------------------
# Steerable PCA (Alg. 2)
# ----------------------------------------------------------------------------
def covariance(plan, a):
    """Mean of the k = 0 coefficients (Alg. 2 step 1, Eq. mean2) and the
    blocks C^(k) = (1/n) Re{A^(k) A^(k)*} (Eq. ck), C^(0) = (1/n) A0 A0^*
    after subtracting the mean (Eq. ck_0).  Two-pass, float64."""
    a = np.asarray(a, dtype=np.complex128)
    n = a.shape[0]
    p0 = int(plan.p[0])
    mean0 = a[:, :p0].real.mean(axis=0)
    blocks = []
    for k, (o, pk) in enumerate(zip(plan.offset, plan.p)):
        A = a[:, o:o + pk]
        if k == 0:
            X = A.real - mean0[None, :]
            blocks.append(X.T @ X / n)
        else:
            blocks.append((A.real.T @ A.real + A.imag.T @ A.imag) / n)
    return mean0, blocks


def eig_blocks(blocks):
    """Eigenpairs of each block, eigenvalues descending (Alg. 2 step 4).
    Each eigenvector is signed so that its entry of largest magnitude (first
    one on ties) is positive."""
    lams, vecs = [], []
    for C in blocks:
        lam, U = np.linalg.eigh(C)
        order = np.argsort(-lam, kind="stable")
        lam, U = lam[order], U[:, order]
        piv = np.argmax(np.abs(U), axis=0)
        sgn = np.sign(U[piv, np.arange(U.shape[1])])
        sgn[sgn == 0] = 1.0
        lams.append(lam)
        vecs.append(U * sgn[None, :])
    return lams, vecs


def select_filter(plan, lams, mode, K=None, sigma2=None, n=None):
    """Per-block filter h^(k)_l applied to the steerable coefficients.

    ``topk``: keep the K pairs (k, l) of largest eigenvalue (ties: smaller k,
    then smaller l), h = 1.  ``mp_wiener``: keep components above the
    Marchenko-Pastur edge lambda > sigma^2 (1 + sqrt(gamma_k))^2 with
    gamma_0 = p_0/n, gamma_k = p_k/(2n) (Eq. compselect), h = (lambda -
    sigma^2)/lambda (the soft threshold (lambda - sigma^2)_+ of Sec. V as a
    per-coefficient Wiener gain); ``mp_hard``: the same selection with h = 1.
    ``all``: h = 1 everywhere."""
    hs = [np.zeros_like(l) for l in lams]
    if mode == "all":
        return [np.ones_like(l) for l in lams]
    if mode == "topk":
        cand = [(-lam[l], k, l) for k, lam in enumerate(lams) for l in range(lam.size)]
        cand.sort()
        for _, k, l in cand[:K]:
            hs[k][l] = 1.0
        return hs
    if mode in ("mp_wiener", "mp_hard"):
        for k, lam in enumerate(lams):
            gamma = plan.p[k] / n if k == 0 else plan.p[k] / (2.0 * n)
            thr = sigma2 * (1.0 + math.sqrt(gamma)) ** 2
            keep = lam > thr
            hs[k][keep] = 1.0 if mode == "mp_hard" else (lam[keep] - sigma2) / lam[keep]
        return hs
    raise ValueError(mode)


def steerable_coefficients(plan, a, mean0, vecs):
    """c^i_{k,l} = sum_q a^i_{k,q} u^(k)_l(q)  (Eq. sPCAcoeff), with the
    k = 0 coefficients centred first (Alg. 2 step 1)."""
    out = []
    for k, (o, pk) in enumerate(zip(plan.offset, plan.p)):
        A = a[:, o:o + pk].copy()
        if k == 0:
            A = A - mean0[None, :]
        out.append(A @ vecs[k])
    return out


def filter_coefficients(plan, a, mean0, vecs, hs):
    """a_den^(k) = U^(k) diag(h^(k)) U^(k)T (a^(k) - mean), mean added back."""
    cs = steerable_coefficients(plan, a, mean0, vecs)
    out = np.zeros_like(np.asarray(a, dtype=np.complex128))
    for k, (o, pk) in enumerate(zip(plan.offset, plan.p)):
        out[:, o:o + pk] = (cs[k] * hs[k][None, :]) @ vecs[k].T
        if k == 0:
            out[:, o:o + pk] += mean0[None, :]
    return out


def denoise(plan, images, mode, K=None, sigma2=None):
    """Expand, build the steerable covariance, eigendecompose, filter and
    synthesise back (Alg. 1 + Alg. 2 + Sec. V)."""
    a = expand(plan, images)
    mean0, blocks = covariance(plan, a)
    lams, vecs = eig_blocks(blocks)
    hs = select_filter(plan, lams, mode, K=K, sigma2=sigma2, n=a.shape[0])
    return synthesize(plan, filter_coefficients(plan, a, mean0, vecs, hs))


def radial_eigenfunctions(plan, vecs):
    """f^{k,l}(xi_j) = sum_q N_{k,q} J_k(R_{k,q} xi_j/c) u^(k)_l(q) (Eq.
    sPCArad, Alg. 2 step 5), returned per k as (n_xi, p_k)."""
    out = []
    for k, (o, pk) in enumerate(zip(plan.offset, plan.p)):
        tab = plan.B[k] / (plan.xi * plan.w)[None, :]     # N J_k(R xi_j/c)
        out.append(tab.T @ vecs[k])
    return out


# ----------------------------------------------------------------------------
# SVD route (Sec. III after Eqs. ck, ck_0; Alg. 2 step 4, second alternative)
# ----------------------------------------------------------------------------
def svd_route(plan, a):
    """Eigenpairs of every C^(k) from the SVD of the coefficient matrix:
    X_k has the rows (Re a_{i,k,.}, Im a_{i,k,.}) for k > 0 and
    Re a_{i,0,.} - mean for k = 0, so C^(k) = X_k^T X_k / n; its right
    singular vectors (the left singular vectors of A^(k) as a p_k x n matrix)
    and s^2 / n are the eigenpairs, descending, signed as in eig_blocks."""
    a = np.asarray(a)
    n = a.shape[0]
    lams, vecs = [], []
    for k, (o, pk) in enumerate(zip(plan.offset, plan.p)):
        blk = a[:, o:o + pk]
        if k == 0:
            X = blk.real - blk.real.mean(axis=0)
        else:
            X = np.concatenate([blk.real, blk.imag], axis=0)
        _, s, Vt = np.linalg.svd(X, full_matrices=False)
        lam = s ** 2 / n
        V = Vt.T
        if V.shape[1] < pk:              # fewer rows than p_k: the rest has eigenvalue 0
            Q, _ = np.linalg.qr(np.concatenate([V, np.eye(pk)], axis=1))
            V = np.concatenate([V, Q[:, V.shape[1]:pk]], axis=1)
            lam = np.concatenate([lam, np.zeros(pk - len(lam))])
        piv = np.argmax(np.abs(V), axis=0)
        sgn = np.sign(V[piv, np.arange(V.shape[1])])
        sgn[sgn == 0] = 1.0
        lams.append(lam)
        vecs.append(V * sgn[None, :])
    return lams, vecs


# ----------------------------------------------------------------------------
# Rotation-invariant features (Sec. I: bispectrum-like features of the
# steerable PCA coefficients)
# ----------------------------------------------------------------------------
def invariant_features(plan, a, mean0, vecs, pairs, triples):
    """Power spectrum |c_{k,l}|^2 for the (k, l) in ``pairs`` and bispectrum
    c_{k1,l1} c_{k2,l2} conj(c_{k1+k2,l3}) for the (k1, l1, k2, l2, l3) in
    ``triples``, with c the steerable PCA coefficients (Eq. sPCAcoeff).  An
    in-plane rotation multiplies c_{k,l} by e^{-ik alpha}, which cancels in
    both; a reflection conjugates c, which leaves the power and conjugates the
    bispectrum."""
    c = steerable_coefficients(plan, a, mean0, vecs)
    pw = np.stack([np.abs(c[k][:, l]) ** 2 for k, l in pairs], axis=1) if pairs else np.zeros((a.shape[0], 0))
    bs = (np.stack([c[k1][:, l1] * c[k2][:, l2] * np.conj(c[k1 + k2][:, l3]) for k1, l1, k2, l2, l3 in triples],
                   axis=1) if triples else np.zeros((a.shape[0], 0), complex))
    return pw, bs
