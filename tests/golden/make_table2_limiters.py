"""Writes table2_limiters.txt: the flux limiters of Table 2 evaluated in
60-digit arithmetic (mpmath) straight from the tabulated closed forms,

    sum         F = 1 / (3 + R)
    max         F = 1 / max(3, R)
    Kershaw     F = 2 / (3 + sqrt(9 + 4 R^2))
    Larsen-n    F = (3^n + R^n)^(-1/n)
    LP          F = (coth R - 1/R) / R        (R = 0: the limit 1/3 of Eq. 19)
    CDA         F = 1/3                       (Sec. 6.1)

at arguments chosen around the oracle's branch points (the LP series below
R = 0.2, the max kink at 3) and far into both limits of Eq. 19.  Nothing here
calls the oracle or the GPU library; run it with `python make_table2_limiters.py`
to rewrite the table (it needs mpmath, which sympy installs).
"""
from __future__ import annotations

import os

R_VALUES = ["0", "1e-10", "1e-6", "1e-3", "0.05", "0.1999", "0.2", "0.5", "0.999", "1", "1.001", "2",
            "2.999", "3", "3.001", "5", "8.99", "9", "9.01", "17", "100", "1e3", "1e6", "1e9", "1e15"]
LARSEN_N = ["1", "2", "3", "4.5"]


def table(mp):
    mp.mp.dps = 60
    three = mp.mpf(3)

    def lp(R):
        return mp.mpf(1) / 3 if R == 0 else (mp.coth(R) - 1 / R) / R

    rows = []
    for rs in R_VALUES:
        # the argument as the binary double the test passes, so both sides see the same R
        R = mp.mpf(float(rs))
        rows.append(("cda", "0", rs, mp.mpf(1) / 3))
        rows.append(("sum", "0", rs, 1 / (three + R)))
        rows.append(("max", "0", rs, 1 / max(three, R)))
        rows.append(("kershaw", "0", rs, 2 / (three + mp.sqrt(9 + 4 * R * R))))
        for ns in LARSEN_N:
            n = mp.mpf(ns)
            rows.append(("larsen", ns, rs, (three ** n + R ** n) ** (-1 / n)))
        rows.append(("lp", "0", rs, lp(R)))
    return rows


def main() -> None:
    import mpmath as mp

    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "table2_limiters.txt"), "w") as fh:
        fh.write("# Flux limiters F(R) of Table 2 (and CDA, Sec. 6.1), 60-digit evaluations of the\n")
        fh.write("# closed forms, written by make_table2_limiters.py.  R is the double nearest the\n")
        fh.write("# decimal in column 3.  LP at R = 0 is its limit 1/3 (Eq. 19).\n")
        fh.write("# kind larsen_n R F\n")
        for kind, n, rs, F in table(mp):
            fh.write(f"{kind} {n} {rs} {mp.nstr(F, 30, min_fixed=1, max_fixed=0)}\n")


if __name__ == "__main__":
    main()
