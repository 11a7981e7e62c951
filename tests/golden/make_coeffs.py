"""Writes coeffs.json: the kernel coefficients every test renders with.

f1 is the paper's (Sec. 3.1; the printed c0/c1 labels are swapped and c1 is
taken as -0.773/4.386 so that the root is the printed 4.386). f'_2 and f3 are
not printed in the paper; they come from the oracle's restatement of the
Sec. 3.1 fit (oracle/fit.py). Calls only oracle/.

    python tests/golden/make_coeffs.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fit  # noqa: E402


def main():
    c2 = fit.fit(2)
    c3 = fit.fit(3)
    # App. A: f2 fitted over the range a tile-culled renderer evaluates
    c2r = {str(t): [float(v) for v in fit.fit_f2_range(t)] + [0.0] for t in (8, 16)}
    out = {
        "_source": "f1: Sec. 3.1 printed values (labels swapped, root 4.386). "
                   "f2 (cut, Eq. 6) and f3: oracle/fit.py, L1 fit of Sec. 3.1, 2^14 midpoint samples, "
                   "Adam 20000 steps. Values for f2/f3 are not printed in the paper (parity unpinned). "
                   "poly2_range: App. A, f2 = max(poly, 0) fitted over [0, x_max(tile)] for 8 and 16 pixel "
                   "tiles (oracle/fit.py fit_f2_range; parity unpinned).",
        "poly1": [0.773, -0.773 / 4.386, 0.0, 0.0],
        "poly2": [float(v) for v in c2] + [0.0],
        "poly3": [float(v) for v in c3],
        "poly2_range": c2r,
        "poly2_range_x_max": {t: fit.x_max_tile(int(t)) for t in c2r},
        "l1_loss": {"poly1": fit.l1_loss([0.773, -0.773 / 4.386], 1),
                    "poly2": fit.l1_loss(c2, 2), "poly3": fit.l1_loss(c3, 3),
                    **{f"poly2_range_{t}": fit.l1_loss(c, 2) for t, c in c2r.items()}},
    }
    with open(os.path.join(HERE, "coeffs.json"), "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")
    print(json.dumps(out, indent=2))


if __name__ == "__main__":
    main()
