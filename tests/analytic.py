"""Closed-form solutions and error norms used to pin the oracle (no oracle code here).

* constant kernel, f0 = exp(-x): eq. (fcoagsolution), Sec. 4.2
* additive kernel K = x + y, f0 = exp(-x): the textbook Golovin solution
  f = (1 - T) / (x sqrt T) exp(-(1 + T) x) I_1(2 x sqrt T), T = 1 - exp(-t)
* multiplicative fragmentation with uniform binary breakage, f0 = exp(-x):
  eq. (fragsolution), Sec. 4.4
* e_c norm with R = 16 Gauss points per bin (Sec. 4.1), evaluated with numpy's
  Legendre routines, independent of the oracle.
"""
import numpy as np
from numpy.polynomial import legendre as npl
from scipy import special


def g_constant(x, t):
    return x * 4.0 / (2.0 + t) ** 2 * np.exp(-2.0 * x / (2.0 + t))


def g_golovin(x, t):
    T = 1.0 - np.exp(-t)
    sT = np.sqrt(T)
    z = 2.0 * x * sT
    # x f = (1-T)/sqrt(T) exp(-(1+T)x) I_1(z) = (1-T)/sqrt(T) exp(-x(1-sqrtT)^2) ive(1, z)
    return (1.0 - T) / sT * np.exp(-x * (1.0 - sT) ** 2) * special.ive(1, z)


def g_pure_frag(x, t):
    return x * (1.0 + t) ** 2 * np.exp(-x * (1.0 + t))


def dg_eval(coef, edges, k, x):
    """Evaluate the DG polynomial (eq. 2.3) at points x with numpy.polynomial.legendre."""
    coef = np.asarray(coef).reshape(len(edges) - 1, k + 1)
    j = np.clip(np.searchsorted(edges, x, side="right") - 1, 0, len(edges) - 2)
    h = edges[j + 1] - edges[j]
    xc = 0.5 * (edges[j] + edges[j + 1])
    xi = 2.0 * (x - xc) / h
    out = np.empty_like(x, dtype=float)
    for n in range(x.size):
        out.flat[n] = npl.legval(xi.flat[n], coef[j.flat[n]])
    return out


def e_c(coef, edges, k, g_exact, R=16):
    """Continuous L1 error of Sec. 4.1 with R Gauss points per bin."""
    s, w = npl.leggauss(R)
    coef = np.asarray(coef).reshape(len(edges) - 1, k + 1)
    err = 0.0
    for j in range(len(edges) - 1):
        h = edges[j + 1] - edges[j]
        xc = 0.5 * (edges[j] + edges[j + 1])
        x = xc + 0.5 * h * s
        err += 0.5 * h * np.sum(w * np.abs(npl.legval(s, coef[j]) - g_exact(x)))
    return err


def log_edges(x_min, x_max, n):
    e = x_min * (x_max / x_min) ** (np.arange(n + 1) / n)
    e[0], e[-1] = x_min, x_max
    return e
