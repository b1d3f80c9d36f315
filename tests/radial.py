"""Independent 1-D references for spherically symmetric sources.

For a radial source rho(s), the Yukawa convolution with G_k = e^{-k r}/(4 pi r)
is u(r) = 1/(2 k r) int_0^inf s rho(s) (e^{-k|r-s|} - e^{-k(r+s)}) ds (shell
theorem for the modified Helmholtz kernel), and the Coulomb convolution with 1/r
is V(r) = (4 pi / r) int_0^inf s rho(s) min(r, s) ds.  These are evaluated with
scipy's adaptive quadrature, which shares nothing with the 3-D sums under test.
"""
import math

import numpy as np
from scipy import integrate


def yukawa_radial(rho, k, r):
    out = np.empty(len(r))
    for i, ri in enumerate(r):
        g = lambda s: s * rho(s) * (math.exp(-k * abs(ri - s)) - math.exp(-k * (ri + s)))
        a, _ = integrate.quad(g, 0.0, ri, limit=200, epsabs=1e-13, epsrel=1e-11)
        b, _ = integrate.quad(g, ri, np.inf, limit=200, epsabs=1e-13, epsrel=1e-11)
        out[i] = (a + b) / (2.0 * k * ri)
    return out


def coulomb_radial(rho, r):
    out = np.empty(len(r))
    for i, ri in enumerate(r):
        a, _ = integrate.quad(lambda s: s * s * rho(s), 0.0, ri, limit=200, epsabs=1e-13)
        b, _ = integrate.quad(lambda s: s * rho(s), ri, np.inf, limit=200, epsabs=1e-13)
        out[i] = 4.0 * math.pi * (a / ri + b)
    return out
