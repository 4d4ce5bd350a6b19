"""R-term Gaussian-sum (sinc quadrature) rule for the Newton kernel 1/z.

Sec. 2.2, Eqs. 2.6-2.7: 1/z = (2/sqrt(pi)) int_0^inf exp(-z^2 t^2) dt, and a
sinc quadrature of this Laplace-Gauss integral gives an R-term separable
approximation 1/z ~ sum_q c_q exp(-t_q^2 z^2).  The paper does not print
the nodes, weights or range.  Reading used here (both implementations
follow it; the table is an input of every solve, so parity never depends
on it):

* substitute t = e^u:  1/z = (2/sqrt(pi)) int_R exp(u - z^2 e^{2u}) du;
* scale z to [1, rho], rho = zmax / zmin;
* R - 1 trapezoid nodes u_lo + q*hs, q = 0..R-2, on [u_lo, u_hi] with half
  weight at both ends, plus one node for the tail (-inf, u_lo), where the
  integrand is e^u exp(-z^2 e^{2u}): weight (2/sqrt(pi)) e^{u_lo} and
  t = e^{u_lo}/sqrt(3) (matching its first two moments in z^2);
* (u_lo, u_hi) minimise the maximum relative error on 301 log-spaced
  points of [1, rho], by a fixed coarse-to-fine grid search.
"""
import numpy as np

NZ = 301


def rule(R, u_lo, u_hi):
    n = R - 1
    hs = (u_hi - u_lo) / (n - 1)
    u = u_lo + hs * np.arange(n)
    t = np.exp(u)
    c = (2.0 / np.sqrt(np.pi)) * hs * t
    c[0] *= 0.5
    c[-1] *= 0.5
    tt = np.exp(u_lo) / np.sqrt(3.0)
    ct = (2.0 / np.sqrt(np.pi)) * np.exp(u_lo)
    return np.r_[tt, t], np.r_[ct, c]


def max_rel_err(t, c, rho, nz=NZ):
    zs = np.exp(np.linspace(0.0, np.log(rho), nz))
    return float(np.max(np.abs(np.exp(-(zs[:, None] * t[None, :]) ** 2) @ c * zs - 1.0)))


def _search(R, rho):
    best = None
    lo_c, hi_c = -15.0, 1.0
    for step_lo, step_hi, span in ((1.0, 0.25, None), (0.2, 0.05, 5), (0.04, 0.01, 5)):
        if span is None:
            los = np.arange(-30.0, -1.99, step_lo)
            his = np.arange(0.0, 3.001, step_hi)
        else:
            los = lo_c + step_lo * np.arange(-span, span + 1)
            his = hi_c + step_hi * np.arange(-span, span + 1)
        for u_lo in los:
            for u_hi in his:
                if u_hi <= u_lo:
                    continue
                t, c = rule(R, u_lo, u_hi)
                e = max_rel_err(t, c, rho)
                if best is None or e < best[0]:
                    best = (e, u_lo, u_hi)
        lo_c, hi_c = best[1], best[2]
    return best


def sinc_table(R: int, zmin: float, zmax: float):
    """Return (t, c, err): 1/z ~ sum_q c_q exp(-t_q^2 z^2) for z in
    [zmin, zmax]; err = the maximum relative error on the test points."""
    if R < 3:
        raise ValueError("R >= 3")
    rho = zmax / zmin
    err, u_lo, u_hi = _search(R, rho)
    t, c = rule(R, u_lo, u_hi)
    return t / zmin, c / zmin, err


def default_range(p):
    """z-range of a problem: from h/100 (inside the singular cell) to twice a
    bound on the largest nucleus-node distance over the lattice window."""
    h = p.h
    ext = 0.0
    for a in range(3):
        ext += (p.N[a] * h + (p.L[a] // 2 + 1) * p.b0) ** 2
    return h * 1e-2, 2.0 * np.sqrt(ext)


def table_for(p):
    zmin, zmax = default_range(p)
    return sinc_table(p.R, zmin, zmax)
