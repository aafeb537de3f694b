"""Writes the exact-rational ERX fixtures in this folder.

Calls only the oracle's exact rational implementation (oracle/erx_exact.py),
which follows Sec. III-C/III-D of the paper in ``fractions.Fraction``
arithmetic.  Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
from fractions import Fraction as F

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.erx_exact import erx_exact  # noqa: E402


def _lcg_cube(seed, lines, width, bands, hi):
    # small deterministic integer cube (a plain LCG, no library RNG)
    s = seed
    out = []
    for _ in range(lines):
        line = []
        for _ in range(width):
            px = []
            for _ in range(bands):
                s = (1103515245 * s + 12345) % (1 << 31)
                px.append(s % hi)
            line.append(px)
        out.append(line)
    return out


CASES = [
    # name, seed, lines, width, bands, hi, alpha, ridge, proj, order
    ("w3_b2_t4", 1, 4, 3, 2, 50, F(1, 10), F(1, 100000), None, "update_then_score"),
    ("w4_b3_t5", 2, 5, 4, 3, 4096, F(1, 10), F(1, 100000), None, "update_then_score"),
    ("w5_b3_t4_stu", 3, 4, 5, 3, 4096, F(1, 10), F(1, 100000), None, "score_then_update"),
    ("w4_b2_t3_a1", 4, 3, 4, 2, 20, F(1), F(1, 100000), None, "update_then_score"),
    ("w6_b4_t3_proj2", 5, 3, 6, 4, 100, F(1, 4), F(1, 1000),
     [[F(1), F(0)], [F(-1), F(1)], [F(0), F(0)], [F(1), F(-1)]], "update_then_score"),
    ("w4_b3_t4_ridge0", 6, 4, 4, 3, 1000, F(3, 10), F(0), None, "update_then_score"),
]


def main():
    out = []
    for name, seed, t, w, b, hi, alpha, ridge, proj, order in CASES:
        cube = _lcg_cube(seed, t, w, b, hi)
        d2, (mu, k) = erx_exact(cube, alpha=alpha, ridge=ridge, w=proj, order=order)
        out.append({
            "name": name, "cube": cube, "alpha": str(alpha), "ridge": str(ridge),
            "proj": None if proj is None else [[str(v) for v in row] for row in proj],
            "order": order,
            "delta2": [[str(v) for v in line] for line in d2],
            "final_mu": [str(v) for v in mu],
            "final_K": [[str(v) for v in row] for row in k],
        })
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "erx_exact_tiny.json")
    with open(path, "w") as f:
        json.dump({"source": "exact rational ERX (Sec. III-C, III-D) from oracle/erx_exact.py",
                   "cases": out}, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
