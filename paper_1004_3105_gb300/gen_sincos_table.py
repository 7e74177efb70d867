"""Writes csrc/sincos_table.inc: for the 1024 angles a_i = 2 pi i / 1024
(i = 0 .. 1023) the four float32 values

    sin a_i,  cos a_i,  -sin a_i / 2,  -cos a_i / 2,

sin and cos computed in double precision and rounded to float32 (the halves
are exact halvings of the rounded values).  The accurate Box-Muller path
(Algorithm B1, paper Sec. 2, step 3) evaluates sin/cos(2 pi v) by angle
addition from a_i with i the top ten bits of the angle word and the exact
remainder delta in [0, 2 pi / 1024):

    sin(a + delta) ~ sin a + delta (cos a + delta (-sin a / 2))
    cos(a + delta) ~ cos a + delta (-sin a + delta (-cos a / 2))

(sin delta ~ delta, cos delta ~ 1 - delta^2 / 2; the dropped terms are below
delta^3 / 6 < 4e-8).  Run it to regenerate the file:

    python -m paper_1004_3105_gb300.gen_sincos_table
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "sincos_table.inc")
N = 1024


def table():
    """(sin, cos, -sin/2, -cos/2) as float32 arrays.  The first quarter turn
    in double precision (sin and cos of pi/2 set to their exact 1 and 0), the
    others by the exact quarter-turn symmetries, so that the table is exactly
    symmetric and exact at multiples of pi/2."""
    q = N // 4
    a = 2.0 * np.pi * np.arange(q + 1, dtype=np.float64) / N
    sb, cb = np.sin(a), np.cos(a)
    sb[q], cb[q] = 1.0, 0.0
    s, c = np.empty(N), np.empty(N)
    for i in range(N):
        k, quarter = i % q, i // q
        s[i], c[i] = [(sb[k], cb[k]), (cb[k], -sb[k]), (-sb[k], -cb[k]), (-cb[k], sb[k])][quarter]
    s32, c32 = s.astype(np.float32), c.astype(np.float32)
    return s32, c32, (-s32 / np.float32(2)).astype(np.float32), (-c32 / np.float32(2)).astype(np.float32)


def literal(v) -> str:
    """A C hex-float literal equal to the float32 value v."""
    return float(np.float32(v)).hex() + "f"


def main():
    s, c, hs, hc = table()
    lines = ["// Generated by paper_1004_3105_gb300/gen_sincos_table.py -- do not edit.",
             f"// {{sin, cos, -sin/2, -cos/2}}(2 pi i / {N}), i = 0 .. {N - 1}; sin and cos in double",
             "// precision rounded to float32, the halves exact."]
    for i in range(N):
        lines.append(f"{{{literal(s[i])}, {literal(c[i])}, {literal(hs[i])}, {literal(hc[i])}}},")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(OUT)


if __name__ == "__main__":
    main()
