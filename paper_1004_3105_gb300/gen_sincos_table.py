"""Writes csrc/sincos_table.inc: sin and cos of the 256 angles 2 pi i / 256
(i = 0 .. 255), each computed in double precision and rounded to float32,
for the accurate Box-Muller path (Algorithm B1, paper Sec. 2, step 3).  The
kernel evaluates sin/cos(2 pi t) by angle addition from the nearest table
angle, with short Taylor polynomials of the remainder (|delta| <= pi/256).
Run it to regenerate the file:

    python -m paper_1004_3105_gb300.gen_sincos_table
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "sincos_table.inc")
N = 256


def table():
    """The first quarter turn in double precision (sin and cos of pi/2 set to
    their exact 1 and 0), the others by the exact quarter-turn symmetries, so
    that the table is exactly symmetric and exact at multiples of pi/2."""
    q = N // 4
    a = 2.0 * np.pi * np.arange(q + 1, dtype=np.float64) / N
    sb, cb = np.sin(a), np.cos(a)
    sb[q], cb[q] = 1.0, 0.0
    s, c = np.empty(N), np.empty(N)
    for i in range(N):
        k, quarter = i % q, i // q
        s[i], c[i] = [(sb[k], cb[k]), (cb[k], -sb[k]), (-sb[k], -cb[k]), (-cb[k], sb[k])][quarter]
    return s.astype(np.float32), c.astype(np.float32)


def literal(v) -> str:
    """A C hex-float literal equal to the float32 value v."""
    return float(np.float32(v)).hex() + "f"


def main():
    s, c = table()
    lines = ["// Generated by paper_1004_3105_gb300/gen_sincos_table.py -- do not edit.",
             f"// {{sin, cos}}(2 pi i / {N}), i = 0 .. {N - 1}, in double precision rounded to float32."]
    for i in range(N):
        lines.append(f"{{{literal(s[i])}, {literal(c[i])}}},")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(OUT)


if __name__ == "__main__":
    main()
