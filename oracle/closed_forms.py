"""Textbook closed forms used only to pin the grid quantities.

* 1D Gaussian-polynomial integrals (Gaussian product theorem + moments
  int y^n exp(-p y^2) dy = Gamma((n+1)/2) / p^((n+1)/2) for even n), which give
  the continuum overlap and kinetic integrals of the separable s/p GTOs.
* s-s nuclear attraction with the Boys function F0(T) = (1/2) sqrt(pi/T) erf(sqrt T).
* The exact integral of 1/|x| over a rectangular cell (Newtonian potential of
  a prism, eight-corner formula).
* Hydrogen with one normalised s-Gaussian: E(a) = 3a/2 - 2 sqrt(2a/pi),
  minimum -4/(3 pi) at a = 8/(9 pi).
"""
import math

import numpy as np
from scipy.special import erf, gamma


def _moment(n, p):
    if n % 2:
        return 0.0
    return gamma((n + 1) / 2.0) / p ** ((n + 1) / 2.0)


def _poly_shift(coefs, shift):
    """(y + shift)^n expansions: coefs[n] of (x-A)^n with x - A = y + shift."""
    out = np.zeros(len(coefs))
    for n, c in enumerate(coefs):
        for k in range(n + 1):
            out[k] += c * math.comb(n, k) * shift ** (n - k)
    return out


def overlap_1d(pa, A, alpha, pb, B, beta):
    """int (sum pa[n] (x-A)^n) e^{-alpha (x-A)^2} (sum pb[n] (x-B)^n) e^{-beta (x-B)^2} dx."""
    p = alpha + beta
    P = (alpha * A + beta * B) / p
    mu = alpha * beta / p
    pre = math.exp(-mu * (A - B) ** 2)
    qa = _poly_shift(pa, P - A)
    qb = _poly_shift(pb, P - B)
    prod = np.convolve(qa, qb)
    return pre * sum(c * _moment(n, p) for n, c in enumerate(prod))


def _deriv(poly, alpha):
    """d/dx of (sum c_n (x-A)^n) e^{-alpha (x-A)^2} -> polynomial times the same Gaussian."""
    out = np.zeros(len(poly) + 1)
    for n, c in enumerate(poly):
        if n:
            out[n - 1] += n * c
        out[n + 1] += -2.0 * alpha * c
    return out


def gto_1d(alpha, is_p):
    nrm = (2.0 * alpha / math.pi) ** 0.25 * (2.0 * math.sqrt(alpha) if is_p else 1.0)
    return np.array([0.0, nrm]) if is_p else np.array([nrm])


def overlap_and_stiffness_1d(alpha, A, pa_is_p, beta, B, pb_is_p):
    """(int g_a g_b, int g_a' g_b') for normalised 1D factors."""
    pa = gto_1d(alpha, pa_is_p)
    pb = gto_1d(beta, pb_is_p)
    s = overlap_1d(pa, A, alpha, pb, B, beta)
    t = overlap_1d(_deriv(pa, alpha), A, alpha, _deriv(pb, beta), B, beta)
    return s, t


def boys0(T):
    if T < 1e-12:
        return 1.0 - T / 3.0
    return 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))


def nuclear_ss(alpha, A, beta, B, C, Z=1.0):
    """int g_a g_b Z/|x - C| for normalised s-Gaussians (3D)."""
    A, B, C = map(np.asarray, (A, B, C))
    p = alpha + beta
    mu = alpha * beta / p
    P = (alpha * A + beta * B) / p
    na = (2 * alpha / math.pi) ** 0.75
    nb = (2 * beta / math.pi) ** 0.75
    return Z * na * nb * (2 * math.pi / p) * math.exp(-mu * np.sum((A - B) ** 2)) * \
        boys0(p * np.sum((P - C) ** 2))


def _prism_F(x, y, z):
    r = math.sqrt(x * x + y * y + z * z)
    f = 0.0
    if r == 0.0:
        return 0.0
    if x != 0 and y != 0:
        f += x * y * math.log(z + r) if z + r > 0 else 0.0
    if y != 0 and z != 0:
        f += y * z * math.log(x + r) if x + r > 0 else 0.0
    if z != 0 and x != 0:
        f += z * x * math.log(y + r) if y + r > 0 else 0.0
    if x != 0:
        f -= 0.5 * x * x * math.atan(y * z / (x * r))
    if y != 0:
        f -= 0.5 * y * y * math.atan(x * z / (y * r))
    if z != 0:
        f -= 0.5 * z * z * math.atan(x * y / (z * r))
    return f


def cell_integral_inv_r(lo, hi):
    """int over the box [lo0,hi0]x[lo1,hi1]x[lo2,hi2] of 1/|x| (exact)."""
    tot = 0.0
    for i, x in enumerate((lo[0], hi[0])):
        for j, y in enumerate((lo[1], hi[1])):
            for k, z in enumerate((lo[2], hi[2])):
                sgn = (-1) ** (i + j + k + 1)
                tot += sgn * _prism_F(x, y, z)
    return tot


def hydrogen_single_gaussian(alpha):
    return 1.5 * alpha - 2.0 * math.sqrt(2.0 * alpha / math.pi)
