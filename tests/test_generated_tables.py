"""The constant tables the CUDA path compiles in, each generated by a script
beside it: csrc/sincos_table.inc (gen_sincos_table.py; the accurate B1
sin/cos, Algorithm B1, Sec. 2) and csrc/h_poly.inc (fit_h.py; the polynomial
h of Methods B3 and P2, Sec. 3 and Sec. 4).  Each committed file is what its
script writes, and each meets the accuracy its kernels rely on, checked
against FP64 evaluations of the definitions written out here."""
import math
import os
import re

import numpy as np

from paper_1004_3105_gb300 import fit_h, gen_sincos_table

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1004_3105_gb300", "csrc")


def read(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def test_sincos_table_is_generated_and_accurate():
    num = r"(-?0x[0-9a-f.]+p[+-]\d+)f"
    rows = re.findall(r"\{" + ", ".join([num] * 4) + r"\}", read("sincos_table.inc"))
    n = gen_sincos_table.N
    assert len(rows) == n == 1024
    t = np.array([[float.fromhex(x) for x in r] for r in rows])
    s, c, hs, hc = t[:, 0], t[:, 1], t[:, 2], t[:, 3]
    gs, gc, ghs, ghc = gen_sincos_table.table()
    for got, want in ((s, gs), (c, gc), (hs, ghs), (hc, ghc)):
        np.testing.assert_array_equal(got, want.astype(np.float64))
    # every sin/cos entry is the float32 nearest to the true value: within half a float ulp
    a = 2.0 * np.pi * np.arange(n) / n
    for got, ref in ((s, np.sin(a)), (c, np.cos(a))):
        half_ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64) / 2
        assert np.all(np.abs(got - ref) <= half_ulp + 1e-15)
        assert np.all(got.astype(np.float32) == got)
    # the third and fourth columns are exact halvings, negated
    np.testing.assert_array_equal(hs, -s / 2)
    np.testing.assert_array_equal(hc, -c / 2)
    # exact at the quarter turns, and exactly quarter-turn symmetric
    q = n // 4
    assert (s[0], c[0], s[q], c[q], s[2 * q], c[2 * q], s[3 * q], c[3 * q]) == (0, 1, 1, 0, 0, -1, -1, 0)
    np.testing.assert_array_equal(s[q:], c[:3 * q])
    np.testing.assert_array_equal(c[q:], -s[:3 * q])


def test_sincos_angle_addition_error_bound():
    # the quadratic angle addition the accurate B1 path evaluates, in float64
    # from the float32 table over remainders delta in [0, 2 pi / 1024): its
    # truncation (delta^3 / 6 and below) plus the table's rounding stays below
    # 1e-7 of the true sin and cos, at every table angle
    gs, gc, ghs, ghc = (x.astype(np.float64) for x in gen_sincos_table.table())
    n = gen_sincos_table.N
    d = np.linspace(0.0, 2.0 * np.pi / n, 257)[:-1]
    i = np.arange(n)[:, None]
    a = 2.0 * np.pi * i / n
    s = gs[i] + d * (gc[i] + d * ghs[i])
    c = gc[i] + d * (-gs[i] + d * ghc[i])
    assert np.max(np.abs(s - np.sin(a + d))) < 1e-7
    assert np.max(np.abs(c - np.cos(a + d))) < 1e-7


def horner_f32(coef, v):
    """sum coef[i] v^i by float32 Horner steps with fused multiply-add (the
    product of two float32 values is exact in float64)."""
    acc = np.full(v.shape, np.float32(coef[-1]))
    for a in coef[-2::-1]:
        acc = (acc.astype(np.float64) * v.astype(np.float64) + np.float64(np.float32(a))).astype(np.float32)
    return acc


def test_h_poly_is_generated_and_accurate():
    text = read("h_poly.inc")
    deg = int(re.search(r"kHDegree = (\d+);", text).group(1))
    body = text[text.index("kHCoef"):]
    coef = np.array([float(x) for x in re.findall(r"(-?[0-9][0-9.e+-]*)f,", body)], dtype=np.float32)
    assert coef.size == deg + 1
    fdeg, mono, err = fit_h.fit()
    assert fdeg == deg
    np.testing.assert_array_equal(np.asarray(mono, dtype=np.float32), coef)
    # the definition: v = (6u - 4)/(4 - 3u) maps u in [0, 8/9] onto v in [-1, 1]
    # and h(v) = sqrt(-ln(1 - u)/u) (-> 1 as u -> 0)
    v = np.linspace(-1.0, 1.0, 400001)
    u = 4.0 * (1.0 + v) / (6.0 + 3.0 * v)
    assert u[0] == 0.0 and abs(u[-1] - 8.0 / 9.0) < 1e-15
    ref = np.ones_like(u)
    ref[1:] = np.sqrt(-np.log1p(-u[1:]) / u[1:])
    got = horner_f32(coef, v.astype(np.float32)).astype(np.float64)
    rel = np.abs(got - ref) / ref
    assert rel.max() < 2e-7
    stated = float(re.search(r"within ([0-9.e+-]+) relative", text).group(1))
    assert stated < 2e-7 and abs(stated - err) < 1e-9
    # the two ends: h(-1) = 1 (u = 0) and h(1) = sqrt(9 ln 9 / 8)
    assert abs(horner_f32(coef, np.array([-1.0], np.float32))[0] - 1.0) < 2e-7
    assert abs(horner_f32(coef, np.array([1.0], np.float32))[0] - math.sqrt(9.0 * math.log(9.0) / 8.0)) < 3e-7
