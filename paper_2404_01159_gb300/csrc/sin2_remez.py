#!/usr/bin/env python
"""Coefficients of the DTLZ1/DTLZ3 g-term polynomial used in eval_steps.cuh.

The multimodal g-term is y^2 + 2 sin^2(10 pi y).  After 10 y is reduced by
its nearest integer to r (|r| <= 1/2), the kernels evaluate
2 sin^2(pi r) = 1 - cos(2 pi r) = u q(u), u = r^2, with q a degree-5
polynomial.  q is the minimax (equioscillating) fit of u q(u) to
1 - cos(2 pi sqrt(u)) on u in [0, 1/4], found by the Remez exchange
algorithm (E. Ya. Remez, 1934): solve for the coefficients and the levelled
error on a reference set, move the reference to the extrema of the error,
repeat.  The maximum error of the fit is about 1.2e-8; evaluated in float32
(Horner, fused multiply-adds) the term is within 4e-7 of the exact value.

    python sin2_remez.py      # prints the float32 coefficients c1..c6
"""
import numpy as np

DEG = 5   # degree of q


def target(u):
    u = np.asarray(u, dtype=np.float64)
    return 1.0 - np.cos(2.0 * np.pi * np.sqrt(u))


def remez(deg=DEG, a=0.0, b=0.25, iters=40, grid=400001):
    n = deg + 2                       # deg + 1 coefficients and the levelled error
    k = np.arange(n)
    x = (a + b) / 2 - (b - a) / 2 * np.cos(np.pi * k / (n - 1))
    g = np.linspace(a, b, grid)
    for _ in range(iters):
        A = np.empty((n, n))
        for i in range(deg + 1):
            A[:, i] = x ** (i + 1)    # u * u^i
        A[:, deg + 1] = (-1.0) ** k
        sol = np.linalg.solve(A, target(x))
        c = sol[: deg + 1]
        err = sum(c[i] * g ** (i + 1) for i in range(deg + 1)) - target(g)
        # one extremum per run of constant sign
        ext, i0, s = [], 0, np.sign(err)
        for i in range(1, grid):
            if s[i] != s[i0]:
                ext.append(i0 + int(np.argmax(np.abs(err[i0:i]))))
                i0 = i
        ext.append(i0 + int(np.argmax(np.abs(err[i0:]))))
        while len(ext) > n:           # keep n alternating extrema
            ext = ext[1:] if abs(err[ext[0]]) < abs(err[ext[-1]]) else ext[:-1]
        if len(ext) < n:
            break
        x = g[ext]
    return c, float(np.max(np.abs(err)))


if __name__ == "__main__":
    c, e = remez()
    print(f"// minimax error {e:.3e}")
    for i, v in enumerate(c):
        print(f"constexpr float kQ{i + 1} = {np.float32(v)!r}f;".replace("np.float32(", "").replace(")f", "f"))
