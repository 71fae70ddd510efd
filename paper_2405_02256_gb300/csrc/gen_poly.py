"""Derive the short polynomial kernels used by the FP32 hybrid-transform paths.

Each function f is approximated on [0, X] by its degree-d Chebyshev interpolant (the
classical Chebyshev-economisation route: interpolate at the d + 1 Chebyshev nodes of
[0, X], then convert to the power basis).  f is evaluated from its own power series in
exact rational arithmetic, so no library routine enters the constants:

* J0(2 sqrt(y)) = sum_k (-y)^k / (k!)^2            (Abramowitz & Stegun 9.1.10)
* cos(sqrt(w))  = sum_k (-w)^k / (2k)!
* sin(sqrt(w)) / sqrt(w) = sum_k (-w)^k / (2k+1)!   (sin z = z q(z^2))
* J1(2 sqrt(y)) / sqrt(y) = sum_k (-y)^k / (k! (k+1)!)  (A&S 9.1.10; J1(z) = (z/2) q((z/2)^2))
* (1 - J0(2 sqrt(y))) / y = sum_k (-y)^k / ((k+1)!)^2  (J0 - 1 = -y q(y): no constant term)
* (1 - cos(sqrt(w))) / w = sum_k (-w)^k / (2k+2)!      (cos z - 1 = -w q(w), w = z^2)

The last two serve the hybrid transforms, which sum kbar(s) - kbar(0) instead of kbar(s)
(the constant drops out of the closed form of Lemma 3.1 because sum_v Delta_eps(v) = 0):
evaluated this way the small terms keep their relative accuracy.

The script prints the FP32 constants (copied into ht.cu) and the worst absolute error of
an FP32 Horner evaluation with fused multiply-adds on a fine grid.

Run:  python paper_2405_02256_gb300/csrc/gen_poly.py
"""
from fractions import Fraction
from math import comb, cos, factorial, pi

import numpy as np


def series(kind: str, x: Fraction, terms: int = 40) -> Fraction:
    s = Fraction(0)
    p = Fraction(1)
    for k in range(terms):
        den = {"j0": factorial(k) ** 2, "cos": factorial(2 * k), "sinc": factorial(2 * k + 1),
               "j1q": factorial(k) * factorial(k + 1), "j0m1q": factorial(k + 1) ** 2,
               "cosm1q": factorial(2 * k + 2)}[kind]
        s += p / den
        p *= -x
    return s


def cheb_power_coeffs(kind: str, X: float, deg: int):
    """Power-basis coefficients (in x) of the Chebyshev interpolant on [0, X]."""
    n = deg + 1
    nodes = [0.5 * X * (1 + cos(pi * (2 * j + 1) / (2 * n))) for j in range(n)]
    vals = [float(series(kind, Fraction(t))) for t in nodes]
    # Vandermonde solve in exact-ish float64 on the scaled variable t = x / X
    V = np.array([[(t / X) ** k for k in range(n)] for t in nodes], dtype=np.float64)
    a = np.linalg.solve(V, np.array(vals))
    return [a[k] / X ** k for k in range(n)]


def horner_f32(c, x):
    x = np.float32(x)
    p = np.float32(c[-1])
    for ck in reversed(c[:-1]):
        p = np.float32(np.float64(p) * np.float64(x) + np.float64(np.float32(ck)))   # fma, one rounding
    return p


def report(kind: str, X: float, deg: int):
    c = cheb_power_coeffs(kind, X, deg)
    c32 = [np.float32(v) for v in c]
    xs = np.linspace(0.0, X, 20001)
    err = max(abs(float(horner_f32(c32, x)) - float(series(kind, Fraction(float(np.float32(x)))))) for x in xs[::20])
    print(f"{kind} on [0, {X}] degree {deg}: max |error| of FP32 Horner = {err:.3e}")
    if kind in ("j0m1q", "cosm1q"):
        # the kernels use x q(x): report its absolute and relative error (one more rounding)
        ea = er = 0.0
        for x in xs[::20]:
            xf = float(np.float32(x))
            got = float(np.float32(np.float64(np.float32(xf)) * np.float64(horner_f32(c32, xf))))
            want = xf * float(series(kind, Fraction(xf)))
            ea = max(ea, abs(got - want))
            if want:
                er = max(er, abs(got - want) / abs(want))
        print(f"   x q(x): max |error| {ea:.3e}, max relative error {er:.3e}")
    print("   {" + ", ".join(f"{float(v):.9e}f" for v in c32) + "}")


if __name__ == "__main__":
    report("j0", 0.25, 3)       # |z| <= 1
    report("j0", 1.0, 5)        # |z| <= 2
    report("cos", 0.5625, 3)    # |z| <= 0.75
    report("cos", 3.0625, 5)    # |z| <= 1.75
    report("sinc", 0.5625, 3)   # |z| <= 0.75
    report("sinc", 3.0625, 5)   # |z| <= 1.75
    report("j1q", 0.25, 3)      # |z| <= 1
    report("j1q", 1.0, 5)       # |z| <= 2
    report("j0m1q", 0.0625, 2)  # |z| <= 0.5
    report("j0m1q", 0.25, 3)    # |z| <= 1
    report("j0m1q", 1.0, 4)     # |z| <= 2
    report("sinc", 0.25, 2)     # |z| <= 0.5
    report("cosm1q", 0.25, 2)    # |z| <= 0.5
    report("cosm1q", 0.5625, 2)  # |z| <= 0.75
    report("cosm1q", 3.0625, 4)  # |z| <= 1.75
