"""Special functions for the FP64 oracle (test infrastructure only).

* ``besselj``      J_k(x), integer k >= 0, by Bessel's integral.
* ``bessel_zeros`` positive zeros of J_k below a bound, by sign-change
                   bracketing on a fine grid followed by bisection.
* ``gauss_legendre`` n-point Gauss-Legendre nodes/weights on [a, b]
                   (Golub-Welsch eigenvalues, polished by Newton steps on
                   the Legendre three-term recurrence).

Parity: pinned against ``scipy.special.jv`` / ``jn_zeros`` and
``numpy.polynomial.legendre.leggauss`` plus polynomial exactness in
``tests/test_oracle_pins.py``.
"""
import numpy as np

_CHUNK = 1 << 14


def besselj(k, x):
    """J_k(x) for integer k >= 0 and real x >= 0 (arrays broadcast).

    Bessel's integral  J_k(x) = (1/2pi) * int_{-pi}^{pi} cos(k t - x sin t) dt.
    The integrand is 2pi-periodic and entire, so the M-point trapezoid rule on
    one period is exact except for the aliased terms J_{k +- pM}(x), p >= 1.
    J_n(x) with n = x + d decays like the Airy function of d (n/2)^(-1/3), so
    M = x + k + 16 ((x + k)/2)^(1/3) + 10 pushes them below 1e-18.  The phase
    k t_m = 2 pi (k m mod M) / M is reduced exactly in integers.
    """
    k, x = np.broadcast_arrays(np.asarray(k, dtype=np.int64),
                               np.asarray(x, dtype=np.float64))
    shape = k.shape
    ki = k.ravel()
    xf = x.ravel()
    out = np.empty(xf.size, dtype=np.float64)
    if xf.size == 0:
        return out.reshape(shape)
    top = float(np.max(np.abs(xf)) + np.max(ki))
    M = 2 * (int(top + 16.0 * (top / 2.0) ** (1.0 / 3.0) + 10) // 2 + 1)
    # the integrand is even in t, so the M-point rule on [-pi, pi) equals the
    # rule on [0, pi] with nodes m = 0..M/2 and half weight at both ends
    m = np.arange(M // 2 + 1, dtype=np.int64)
    wt = np.full(m.size, 2.0 / M)
    wt[0] = wt[-1] = 1.0 / M
    sin_t = np.sin(2.0 * np.pi * m / M)
    for s in range(0, xf.size, _CHUNK):
        kk = ki[s:s + _CHUNK, None]
        xx = xf[s:s + _CHUNK, None]
        phase = 2.0 * np.pi * ((kk * m[None, :]) % M) / M
        out[s:s + _CHUNK] = np.cos(phase - xx * sin_t[None, :]) @ wt
    return out.reshape(shape)


def bessel_zeros(k, xmax, step=0.2, iters=56):
    """All positive zeros of J_k that are <= xmax, ascending (float64 array).

    Consecutive positive zeros of J_k are more than 2.4 apart, so a grid of
    spacing ``step`` brackets each zero in its own cell; every bracket is then
    halved ``iters`` times (bisection needs no derivative and cannot jump to a
    neighbouring zero).  Zeros of J_k (k >= 1) all exceed k.
    """
    lo = float(k) if k > 0 else 0.0
    if xmax <= lo:
        return np.zeros(0)
    n = int(np.ceil((xmax + 2.0 * step - lo) / step)) + 1
    grid = lo + step * np.arange(n)
    grid[0] = max(grid[0], 1e-3)
    v = besselj(k, grid)
    s = np.nonzero(np.sign(v[:-1]) * np.sign(v[1:]) < 0)[0]
    a, b = grid[s].copy(), grid[s + 1].copy()
    fa = v[s].copy()
    for _ in range(iters):
        m = 0.5 * (a + b)
        fm = besselj(k, m)
        left = np.sign(fm) == np.sign(fa)
        a = np.where(left, m, a)
        fa = np.where(left, fm, fa)
        b = np.where(left, b, m)
    z = 0.5 * (a + b)
    return z[z <= xmax]


def _legendre_and_derivative(n, x):
    """P_n(x) and P_n'(x) by the three-term recurrence
    (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1}."""
    p0 = np.ones_like(x)
    p1 = x.copy()
    for m in range(1, n):
        p0, p1 = p1, ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
    # derivative from (1 - x^2) P_n' = n (P_{n-1} - x P_n)
    dp = n * (p0 - x * p1) / (1.0 - x * x)
    return p1, dp


def gauss_legendre(n, a=-1.0, b=1.0):
    """n-point Gauss-Legendre rule on [a, b], nodes ascending.

    Nodes: eigenvalues of the symmetric tridiagonal Jacobi matrix of the
    Legendre recurrence (off-diagonal m / sqrt(4 m^2 - 1)), then two Newton
    steps on P_n.  Weights: w = 2 / ((1 - x^2) P_n'(x)^2), scaled to [a, b].
    """
    m = np.arange(1, n, dtype=np.float64)
    beta = m / np.sqrt(4.0 * m * m - 1.0)
    J = np.diag(beta, 1) + np.diag(beta, -1)
    x = np.sort(np.linalg.eigvalsh(J))
    for _ in range(2):
        p, dp = _legendre_and_derivative(n, x)
        x = x - p / dp
    _, dp = _legendre_and_derivative(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    half = 0.5 * (b - a)
    return a + half * (x + 1.0), half * w
