"""Write the oracle regression fixtures of tests/golden/ (run from the repo root).

The paper prints no worked example values for the FBP path (Sec. 4-5 give the
formulas and Table perf gives timings only), so these fixtures are the FP64
oracle's own outputs on small seeded inputs. This script calls only oracle/ and
the seeded input generators; tests/test_golden.py recomputes the same values and
compares them with the stored ones, so any later change of the oracle's
arithmetic shows up (and must then be justified from the paper).
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lamino_oracle as O  # noqa: E402
from paper_2401_11101_gb300 import inputs as I  # noqa: E402

GEOM = I.Geometry(8, 8, 8, 8, 8, 12, math.radians(20.0))
SEED = 50
# (x3, x2, x1) indices of the sampled voxels
SAMPLES = [(z, y, x) for z in (0, 3, 7) for y in (1, 4, 6) for x in (0, 2, 5, 7)]


def compute():
    d = I.random_projections(GEOM, SEED)
    out = {}
    for kind in ("ramp", "shepp", "parzen"):
        vd = O.fbp_direct(d, GEOM, kind)
        vf = O.fbp_fourier(d, GEOM, kind)
        out[f"direct_{kind}"] = [vd[s] for s in SAMPLES] + [float(vd.sum()), float(np.abs(vd).sum())]
        out[f"fourier_{kind}"] = [vf[s] for s in SAMPLES] + [float(vf.sum()), float(np.abs(vf).sum())]
    return out


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_fbp_8cube.txt")
    vals = compute()
    with open(path, "w") as f:
        f.write("# FP64 oracle FBP on the 8^3 geometry (8 angles, detector 8x12, tilt 20 deg),\n")
        f.write(f"# projections inputs.random_projections(seed={SEED}); written by make_golden.py.\n")
        f.write("# Each line: name, then the voxels at SAMPLES (make_golden.py), the sum and the\n")
        f.write("# sum of absolute values.\n")
        for k, v in vals.items():
            f.write(k + " " + " ".join(repr(float(x)) for x in v) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
