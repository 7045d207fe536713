"""Closed forms and brute-force definitions used to pin the oracle (and, at full size, the GPU
results). Nothing here calls the oracle or the CUDA path.

* Kaufman's partition function of the m x n periodic square lattice (B. Kaufman, Phys. Rev. 76,
  1232 (1949)), J = 1, h = 0; and from it, in exact arithmetic, the number of configurations
  with every energy (the coefficients of Z as a polynomial in exp(-2K), as P. D. Beale, Phys.
  Rev. Lett. 76, 78 (1996), obtained them).
* The periodic chain in a field, from the 2 x 2 transfer matrix (Ising 1925).
* Non-interacting spins in a field.
* Run counting on a ring: the number of cyclic binary strings with U ones and 2r runs.
* A pure-Python brute force (a second language), for graphs of up to ~14 spins.
"""
from __future__ import annotations

import math
from itertools import product


def _log2cosh(x: float) -> float:
    ax = abs(x)
    return ax + math.log1p(math.exp(-2.0 * ax))


def _log_abs_2sinh(x: float):
    """(sign, log|2 sinh x|)."""
    if x == 0.0:
        return 0, -math.inf
    ax = abs(x)
    return (1 if x > 0 else -1), ax + math.log(-math.expm1(-2.0 * ax))


def kaufman_logz(m: int, n: int, T: float, J: float = 1.0) -> float:
    """ln Z of the m x n torus (J > 0, h = 0) by Kaufman's four-product formula:
    Z = 1/2 (2 sinh 2K)^(mn/2) [P1 + P2 + P3 + P4], K = J/T, with
    P1 = prod_r 2cosh(m g_(2r+1)/2), P2 = prod_r 2sinh(m g_(2r+1)/2),
    P3 = prod_r 2cosh(m g_(2r)/2),   P4 = prod_r 2sinh(m g_(2r)/2),  r = 0..n-1,
    cosh g_l = cosh 2K coth 2K - cos(pi l / n) for l >= 1 and g_0 = 2K + ln tanh K (signed)."""
    K = J / T
    c = math.cosh(2 * K) / math.tanh(2 * K)

    def gamma(l: int) -> float:
        if l == 0:
            return 2 * K + math.log(math.tanh(K))
        return math.acosh(c - math.cos(math.pi * l / n))

    terms = []  # (sign, log|P|)
    odd = [gamma(2 * r + 1) for r in range(n)]
    even = [gamma(2 * r) for r in range(n)]
    for gs in (odd, even):
        terms.append((1, sum(_log2cosh(m * g / 2) for g in gs)))
        sign, lg = 1, 0.0
        for g in gs:
            s, l = _log_abs_2sinh(m * g / 2)
            sign *= s
            lg += l
        terms.append((sign, lg))
    lmax = max(l for s, l in terms if s != 0)
    tot = math.fsum(s * math.exp(l - lmax) for s, l in terms if s != 0)
    return math.log(0.5) + (m * n / 2) * math.log(2 * math.sinh(2 * K)) + lmax + math.log(tot)


def _kaufman_z_mp(m: int, n: int, K):
    """Kaufman's Z of the m x n torus at coupling K (J = 1, h = 0) in mpmath at the working precision."""
    import mpmath as mp
    c = mp.cosh(2 * K) / mp.tanh(2 * K)

    def gamma(l: int):
        if l == 0:
            return 2 * K + mp.log(mp.tanh(K))
        return mp.acosh(c - mp.cos(mp.pi * l / n))

    odd = [gamma(2 * r + 1) for r in range(n)]
    even = [gamma(2 * r) for r in range(n)]
    p = mp.mpf(0)
    for gs in (odd, even):
        p += mp.fprod(2 * mp.cosh(m * g / 2) for g in gs)
        p += mp.fprod(2 * mp.sinh(m * g / 2) for g in gs)
    return mp.mpf(1) / 2 * (2 * mp.sinh(2 * K)) ** (mp.mpf(m * n) / 2) * p


def kaufman_energy_counts(m: int, n: int, digits: int = 0) -> list:
    """Exact number of configurations of the m x n torus (J = 1) with k unsatisfied bonds, k = 0..2mn
    (E = -2mn + 2k), from Kaufman's closed form alone: Z e^(-2mnK) = sum_k g_k x^k with x = e^(-2K)
    is a polynomial of degree 2mn; it is evaluated at 2mn + 1 points of (0, 1) in high precision,
    interpolated (Newton's divided differences, then the monomial coefficients) and rounded to
    integers. Each coefficient is checked to be within 0.01 of its integer."""
    import mpmath as mp
    d = 2 * m * n
    with mp.workdps(digits or 4 * d + 60):
        xs = [mp.mpf(j + 1) / (d + 2) for j in range(d + 1)]
        ys = [_kaufman_z_mp(m, n, -mp.log(x) / 2) * x ** (m * n) for x in xs]   # e^(-2mnK) = x^(mn)
        coef = list(ys)                        # divided differences, in place
        for lvl in range(1, d + 1):
            for i in range(d, lvl - 1, -1):
                coef[i] = (coef[i] - coef[i - 1]) / (xs[i] - xs[i - lvl])
        poly = [mp.mpf(0)] * (d + 1)           # Newton form -> monomials, Horner from the top
        for i in range(d, -1, -1):
            for k in range(d, 0, -1):
                poly[k] = poly[k - 1] - xs[i] * poly[k]
            poly[0] = coef[i] - xs[i] * poly[0]
        out = []
        for c in poly:
            r = int(mp.nint(c))
            if abs(c - r) > mp.mpf("0.01"):
                raise ArithmeticError("interpolated coefficient is not an integer: precision too low")
            out.append(r)
    return out


def ring_logz(n: int, T: float, h: float = 0.0, J: float = 1.0) -> float:
    """ln Z of the periodic chain of n spins: Z = l+^n + l-^n with
    l+- = e^K cosh(h/T) +- sqrt(e^(2K) sinh^2(h/T) + e^(-2K)), K = J/T.
    At h = 0 this is (2 cosh K)^n + (2 sinh K)^n."""
    K, b = J / T, h / T
    root = math.sqrt(math.exp(2 * K) * math.sinh(b) ** 2 + math.exp(-2 * K))
    lp = math.exp(K) * math.cosh(b) + root
    lm = math.exp(K) * math.cosh(b) - root
    r = lm / lp
    return n * math.log(lp) + math.log1p(r ** n) if r ** n > -1 else float("nan")


def free_spins(n: int, T: float, h: float):
    """(lnZ, <M>, chi) of n non-interacting spins: Z = (2 cosh(h/T))^n, <M> = n tanh(h/T),
    chi = (n/T) sech^2(h/T)."""
    b = h / T
    return n * _log2cosh(b), n * math.tanh(b), n / T / math.cosh(b) ** 2


def ring_joint_count(n: int, up: int, runs_pairs: int) -> int:
    """Number of ring configurations (labelled sites) with `up` up spins and 2r runs, i.e. 2r
    unsatisfied bonds: (n/r) C(up-1, r-1) C(n-up-1, r-1) for r >= 1; for r = 0 one all-up and
    one all-down configuration."""
    r = runs_pairs
    if r == 0:
        return 1 if up in (0, n) else 0
    if up < r or n - up < r:
        return 0
    return n * math.comb(up - 1, r - 1) * math.comb(n - up - 1, r - 1) // r


def brute_force_g(n: int, edges):
    """g as a dict {(E, M): count}: every configuration, spins from bits (bit 1 = up), E = -sum
    J s_i s_j over the listed edges (duplicates counted as listed, i.e. summed), M = sum s_i."""
    out = {}
    for bits in product((0, 1), repeat=n):
        s = [1 if b else -1 for b in reversed(bits)]
        E = -sum(J * s[i] * s[j] for i, j, J in edges)
        M = sum(s)
        out[(E, M)] = out.get((E, M), 0) + 1
    return out


def brute_force_g_range(n: int, edges, lo: int, hi: int):
    """Like brute_force_g, over configuration words s in [lo, hi) only; spin i is bit i of s."""
    out = {}
    for s in range(lo, hi):
        sp = [1 if (s >> i) & 1 else -1 for i in range(n)]
        E = -sum(J * sp[i] * sp[j] for i, j, J in edges)
        M = sum(sp)
        out[(E, M)] = out.get((E, M), 0) + 1
    return out


def kaufman_C(m: int, n: int, T: float, J: float = 1.0) -> float:
    """Specific heat of the m x n torus from Kaufman's ln Z by central differences:
    C = T^2 d^2lnZ/dT^2 + 2 T dlnZ/dT (accurate to ~1e-7 relative)."""
    d = 1e-4 * T
    f0, fp, fm = kaufman_logz(m, n, T, J), kaufman_logz(m, n, T + d, J), kaufman_logz(m, n, T - d, J)
    return T * T * (fp - 2 * f0 + fm) / (d * d) + 2 * T * (fp - fm) / (2 * d)


def golden_max(f, lo: float, hi: float, tol: float = 1e-10) -> float:
    """Argument of the maximum of a unimodal f on [lo, hi] by golden-section search."""
    r = (math.sqrt(5) - 1) / 2
    a, b = lo, hi
    c, d = b - r * (b - a), a + r * (b - a)
    fc, fd = f(c), f(d)
    while b - a > tol * max(1.0, abs(a)):
        if fc > fd:
            b, d, fd = d, c, fc
            c = b - r * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + r * (b - a)
            fd = f(d)
    return 0.5 * (a + b)


def kaufman_C_peak(m: int, n: int, near: float, step: float = 0.001) -> float:
    """Peak of Kaufman's C(T) near `near`: vertex of the least-squares parabola through C at
    near + k*step, k = -3..3 (the curvature there dwarfs the finite-difference noise of C, and
    the fitted vertex is biased by the asymmetry of the peak only at order step^2, ~2e-6 here)."""
    import numpy as np
    ts = near + step * np.arange(-3, 4)
    a, b, _ = np.polyfit(ts - near, [kaufman_C(m, n, t) for t in ts], 2)
    return near - b / (2 * a)


def free_spin_moments(n: int, T: float, h: float):
    """(<|M|>, <M^2>, <M^4>) of n non-interacting spins in a field: each spin is +1 with
    probability p = (1 + tanh(h/T)) / 2, so the number of up spins is binomial(n, p). <|M|> is
    the binomial sum; the even moments come from the cumulants of one spin (mean t, variance
    1 - t^2, third -2t(1 - t^2), fourth -2(1 - t^2)(1 - 3t^2)), which add over the n spins."""
    t = math.tanh(h / T)
    p = (1 + t) / 2
    absm = math.fsum(math.comb(n, k) * p ** k * (1 - p) ** (n - k) * abs(2 * k - n) for k in range(n + 1))
    k1, k2 = n * t, n * (1 - t * t)
    k3, k4 = n * -2 * t * (1 - t * t), n * -2 * (1 - t * t) * (1 - 3 * t * t)
    m2 = k2 + k1 * k1
    m4 = k4 + 4 * k3 * k1 + 3 * k2 * k2 + 6 * k2 * k1 * k1 + k1 ** 4
    return absm, m2, m4


def ring_M2(n: int, T: float, J: float = 1.0) -> float:
    """<M^2> of the periodic chain at h = 0: n times the sum over distances r of the correlation
    <s_0 s_r> = (t^r + t^(n-r)) / (1 + t^n), t = tanh(J/T) (the 2 x 2 transfer matrix)."""
    t = math.tanh(J / T)
    return n * math.fsum((t ** r + t ** (n - r)) / (1 + t ** n) for r in range(n))


def brute_force_magnetisation(n: int, edges, T: float, h: float):
    """(<|M|>, <M^2>, <M^4>) by summing over every configuration with its Boltzmann weight
    exp(-(E - h M)/T), E = -sum J s_i s_j (no table in between)."""
    terms = []
    for s in range(1 << n):
        sp = [1 if (s >> i) & 1 else -1 for i in range(n)]
        E = -sum(J * sp[i] * sp[j] for i, j, J in edges)
        M = sum(sp)
        terms.append((-(E - h * M) / T, M))
    lmax = max(l for l, _ in terms)
    w = [(math.exp(l - lmax), M) for l, M in terms]
    Z = math.fsum(x for x, _ in w)
    return tuple(math.fsum(x * f(M) for x, M in w) / Z for f in (abs, lambda M: M * M, lambda M: M ** 4))
