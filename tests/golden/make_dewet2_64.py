"""Writes dewet2_64_stats.json: statistics of a long two-layer dewetting
run (D2Q9 64 x 64, workloads.dewet2_*) from the FP64 oracle, which the GPU
run is compared with: the rupture step (first multiple of 100 with some
layer below 1.5 h*), the per-layer mass, the radial spectra of both layers
at 3/4 of the rupture step, and the dewetted fraction and the histogram of
the upper layer at three times the rupture step. Calls only the oracle and
the input generators.

    python tests/golden/make_dewet2_64.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402
from tests import droplets  # noqa: E402

SIDE, EVERY, LIMIT = 64, 100, 20000
BINS = np.linspace(0.0, 1.2, 25)


def main():
    p = workloads.dewet2_params(SIDE)
    h0 = workloads.dewet2_heights(SIDE)
    state = {"t": 0, "f": oracle.init(p, h0.ravel())}

    def at(t):
        state["f"] = oracle.run(p, state["f"], t - state["t"])
        state["t"] = t
        return oracle.heights(p, state["f"]).reshape(2, SIDE, SIDE)

    tr, _ = droplets.rupture_step(at, p["hstar"], EVERY, LIMIT)
    # restart for the samples at 3/4 and 3 times the rupture step
    state.update(t=0, f=oracle.init(p, h0.ravel()))
    h_pre = at(3 * tr // 4)
    h_post = at(3 * tr)
    hist, _ = np.histogram(h_post[1], bins=BINS)
    out = {
        "what": "oracle statistics of the two-layer dewetting run, D2Q9 64x64",
        "every": EVERY, "rupture_step": tr,
        "mass": [float(m) for m in h_post.sum(axis=(1, 2))],
        "spectrum_step": 3 * tr // 4,
        "spectra": [droplets.radial_spectrum(h_pre[i]).tolist() for i in range(2)],
        "post_step": 3 * tr,
        "dewetted_fraction": float((h_post[1] < 2 * p["hstar"]).mean()),
        "hist_bins": BINS.tolist(),
        "hist_upper": (hist / hist.sum()).tolist(),
    }
    with open(os.path.join(HERE, "dewet2_64_stats.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
