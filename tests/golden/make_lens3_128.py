"""Writes lens3_128_angles.json: the opening angles of the four lenses of
the three-layer lens field at 128 x 128 (radius 12.5, Neumann angle 20
degrees) after 10000 steps of the FP64 oracle, measured with the arc fit
of tests/droplets.py. Calls only the oracle and the input generators.

    python tests/golden/make_lens3_128.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402
from tests import droplets  # noqa: E402

STEPS = 10000
SIDE, RADIUS = 128, 12.5


def main():
    p = workloads.lens3_params(SIDE, SIDE, RADIUS)
    h0 = workloads.lens3_heights(SIDE, SIDE, RADIUS)
    f = oracle.run(p, oracle.init(p, h0.ravel()), STEPS)
    h = oracle.heights(p, f).reshape(h0.shape)
    centres = workloads.lens3_centres(SIDE, SIDE, RADIUS)
    ang = droplets.lens3_angles(h, centres, RADIUS)
    out = {
        "what": "opening angles (degrees) and arc-fit errors E of the four lenses, "
                "upper surface z3 and lower surface z2, FP64 oracle",
        "workload": "lens3 %dx%d radius %.1f Neumann angle 20 deg" % (SIDE, SIDE, RADIUS),
        "steps": STEPS,
        "upper": [[a[0][0], a[0][1]] for a in ang],
        "lower": [[a[1][0], a[1][1]] for a in ang],
        "mass": [float(m) for m in h.sum(axis=(1, 2))],
    }
    with open(os.path.join(HERE, "lens3_128_angles.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
