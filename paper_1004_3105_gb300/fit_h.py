"""Fits the polynomial h of Methods B3 and P2 (paper Sec. 3 and Sec. 4) and
writes its coefficients to csrc/h_poly.inc.

The paper approximates g(u) = sqrt(-ln(1 - u) / u) on 0 <= u <= tau = 8/9
(rho = 1) after the change of variable v = (6u - 4) / (4 - 3u), which maps
[0, 8/9] onto [-1, 1] and puts the singularities of h(v) = g(u(v)) at
v = +-2; a polynomial in v that is close to minimax is obtained by truncating
a Chebyshev series.  The paper prints no coefficients (its degree-15 fit is
for double precision), so this script computes them: Chebyshev interpolation
of h at the degree-D Chebyshev points in double precision, conversion to the
monomial basis, and the smallest degree whose float32 Horner evaluation stays
within 2e-7 relative of h on a dense grid.  Run it to regenerate the file:

    python -m paper_1004_3105_gb300.fit_h
"""
from __future__ import annotations

import os

import numpy as np
from numpy.polynomial import chebyshev as C

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "h_poly.inc")


def u_of_v(v):
    """Inverse of v = (6u - 4) / (4 - 3u)."""
    return 4.0 * (1.0 + v) / (6.0 + 3.0 * v)


def h(v):
    u = u_of_v(np.asarray(v, dtype=np.float64))
    out = np.ones_like(u)
    nz = u > 0
    out[nz] = np.sqrt(-np.log1p(-u[nz]) / u[nz])
    return out


def horner32(coef, v):
    """Evaluates sum coef[i] v^i in float32 with fused multiply-adds."""
    c = np.asarray(coef, dtype=np.float32)
    v = np.asarray(v, dtype=np.float32)
    acc = np.full_like(v, c[-1])
    for a in c[-2::-1]:
        acc = (acc.astype(np.float64) * v.astype(np.float64) + np.float64(a)).astype(np.float32)
    return acc


def fit(max_rel=2e-7, max_degree=20):
    grid = np.linspace(-1.0, 1.0, 200001)
    ref = h(grid)
    for deg in range(4, max_degree + 1):
        cheb = C.chebinterpolate(h, deg)
        mono = C.cheb2poly(cheb)
        err = np.max(np.abs(horner32(mono, grid).astype(np.float64) - ref) / ref)
        if err < max_rel:
            return deg, mono, err
    raise RuntimeError("no degree meets the bound")


def main():
    deg, mono, err = fit()
    lines = [
        "// Generated by paper_1004_3105_gb300/fit_h.py -- do not edit.",
        "// h(v) = sqrt(-ln(1 - u) / u) with u = 4(1 + v) / (6 + 3v), v in [-1, 1]",
        "// (Methods B3 and P2, paper Sec. 3 and Sec. 4; rho = 1, tau = 8/9): truncated",
        f"// Chebyshev interpolation of degree {deg} in double precision, monomial form;",
        f"// float32 Horner evaluation within {err:.2e} relative of h on [-1, 1].",
        f"constexpr int kHDegree = {deg};",
        "__device__ __constant__ float kHCoef[kHDegree + 1] = {",
    ]
    for a in mono:
        lines.append(f"    {np.float32(a)!r}f,".replace("np.float32(", "").replace(")f", "f"))
    lines.append("};")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"degree {deg}, max relative error {err:.3e} -> {OUT}")


if __name__ == "__main__":
    main()
