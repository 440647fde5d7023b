"""Reader of the hand-worked fixtures in tests/golden/ (text only, no
arithmetic of the method): each case is an image, optional S and Q tables,
and windows with their expected sums, means and variances (exact fractions).
"""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_cases(name="hand_worked.txt"):
    cases = []
    lines = [ln.split("#", 1)[0].strip() for ln in open(os.path.join(GOLDEN, name))]
    lines = [ln for ln in lines if ln]
    i = 0
    cur = None
    while i < len(lines):
        tok = lines[i].split()
        if tok[0] == "case":
            cur = {"name": tok[1], "windows": []}
            cases.append(cur)
            i += 1
        elif tok[0] == "image":
            r, c = int(tok[1]), int(tok[2])
            cur["image"] = np.array([[int(v) for v in lines[i + 1 + k].split()] for k in range(r)])
            assert cur["image"].shape == (r, c)
            i += 1 + r
        elif tok[0] in ("S", "Q"):
            r = cur["image"].shape[0]
            cur[tok[0]] = np.array([[int(v) for v in lines[i + 1 + k].split()] for k in range(r)],
                                   dtype=np.uint64)
            i += 1 + r
        elif tok[0] == "window":
            w = {"shape": tuple(int(v) for v in tok[1:5])}
            for k, key in enumerate(("sum", "mean", "var")):
                t = lines[i + 1 + k].split()
                assert t[0] == key, (cur["name"], t)
                w[key] = [Fraction(v) for v in t[1:]]
            cur["windows"].append(w)
            i += 4
        else:
            raise ValueError("bad golden line: %r" % lines[i])
    return cases


def expected(w, R, C):
    """(sum as uint64, mean as the correctly rounded double, std as the
    correctly rounded double of sqrt(var)) arrays of shape R x C."""
    import math
    from decimal import Decimal, getcontext
    getcontext().prec = 80
    s = np.array([int(v) for v in w["sum"]], dtype=np.uint64).reshape(R, C)
    m = np.array([float(v) for v in w["mean"]]).reshape(R, C)   # Fraction -> double rounds correctly
    d = []
    for v in w["var"]:
        x = (Decimal(v.numerator) / Decimal(v.denominator)).sqrt()
        d.append(float(x))          # 80-digit root rounded once to double
    assert all(math.isfinite(v) for v in d)
    return s, m, np.array(d).reshape(R, C)
