"""Writes tests/golden/sizes.txt from scipy.special.jn_zeros.

The counts follow the literal sampling criterion R_{k,q+1} <= 2 pi c R
(Eq. criterion1) with c = 1/2, R = L/2; n_xi = ceil(4cR), n_theta =
ceil(16cR) (Alg. 1 step 1).  Run: python tests/golden/make_sizes.py
"""
import math
import os

import numpy as np
import scipy.special as sp


def sizes(L, c=0.5):
    R = L / 2.0
    X = 2.0 * math.pi * c * R
    P = p = sq = 0
    k = 0
    kmax = -1
    while True:
        z = sp.jn_zeros(k, int(X / math.pi) + 5)
        pk = max(0, int(np.sum(z <= X)) - 1)
        if pk == 0:
            break
        P += pk
        p += pk if k == 0 else 2 * pk
        sq += pk * pk
        kmax = k
        k += 1
    return (L, R, kmax, P, p, sq, math.ceil(4 * c * R - 1e-9), math.ceil(16 * c * R - 1e-9))


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(__file__), "sizes.txt")
    head = [ln for ln in open(path) if ln.startswith("#")]
    with open(path, "w") as f:
        f.writelines(head)
        for L in (16, 32, 64, 96, 128, 180, 256):
            f.write(" ".join(str(v) for v in sizes(L)) + "\n")
