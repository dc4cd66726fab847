"""Replay of the MT_FP64 weights' binary64 exp(-t) (csrc/mt_pair.cuh,
exp_neg): its constants read from the kernel source and its operations
replayed one by one, each rounded once to binary64 (exact rational
arithmetic, then one rounding), so that the GPU's results can be compared
with it bit for bit and the recipe with the exact exponential."""
import math
import re
from fractions import Fraction
from pathlib import Path

SRC = Path(__file__).resolve().parents[1] / "paper_1811_05474_gb300" / "csrc" / "mt_pair.cuh"


def _constants():
    text = SRC.read_text()
    body = text[text.index("double exp_neg(double t)"):]
    body = body[:body.index("\n}\n")]
    table = text[text.index("kExp2j32[32] = {"):]
    table = table[:table.index("};")]
    tab = [float.fromhex(h) for h in re.findall(r"0x[0-9a-f.]+p[+-]?\d+", table)]
    return tab, body


def _hex_after(body, marker):
    line = next(ln for ln in body.splitlines() if marker in ln)
    return [float.fromhex(h) for h in re.findall(r"0x[0-9a-f.]+p[+-]?\d+", line)]


def _round(v: Fraction) -> float:
    return float(v)  # Fraction -> float rounds to nearest, ties to even


def fma(a, b, c):
    return _round(Fraction(a) * Fraction(b) + Fraction(c))


def replay(t: float, tab, c) -> float:
    """exp_neg(t) as the kernel computes it, every operation rounded once."""
    if not t <= 745.5:
        return 0.0 if t > 745.5 else t + t
    x = -t
    magic = 6755399441055744.0  # 1.5 * 2^52
    kd = fma(x, c["inv"], magic)
    kf = _round(Fraction(kd) - Fraction(magic))
    k = int(kf)
    r = fma(-kf, c["head"], x)
    r = fma(-kf, c["tail"], r)
    q = fma(r, c["c6"], c["c5"])
    q = fma(r, q, c["c4"])
    q = fma(r, q, c["c3"])
    q = fma(r, q, 0.5)
    em1 = fma(_round(Fraction(r) * Fraction(r)), q, r)
    T = tab[k & 31]
    res = fma(T, em1, T)
    return math.ldexp(res, k >> 5)


def consts():
    """(table, named constants) as they stand in the kernel source."""
    tab, body = _constants()
    kd_line = _hex_after(body, "x 32 / ln2")
    head = _hex_after(body, "head of ln2 / 32")
    tail = _hex_after(body, "// tail")
    q0 = _hex_after(body, "1/720, 1/120")
    return tab, {"inv": kd_line[0], "head": head[0], "tail": tail[0], "c6": q0[0], "c5": q0[1],
                 "c4": _hex_after(body, "// 1/24")[0], "c3": _hex_after(body, "// 1/6")[0]}
