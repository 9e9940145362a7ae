"""Write fullsize_512_64shells.json: the FP64 oracle's raw sums T^l and counts
for a fixed sample of bins of the 512^3 / 64-shell workload (field seed 1710,
sigma_g = 0.3 quadratic + Kaiser model, shells of width 2 k_f from k_f,
l = 0, 2, 4), so that the full-size GPU tests and the benchmark's precision
comparison can check those bins without running the oracle at 512^3 each
time.  Calls only the oracle and the seeded input generator.

The sample: every valid bin with a <= 4 (the low-k bins, where the sum over x
cancels most and the tensor-core paths depart most from FP32), and six bins
spread over the rest of the range.

    python tests/golden/make_fullsize_512.py      (a few minutes on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1708_05303_gb300.synth import FieldModel, linear_edges, make_field  # noqa: E402

N, BOX, SEED, SHELLS = 512, 1000.0, 1708 + 2, 64
SPREAD = [(20, 12, 10), (40, 21, 20), (63, 62, 61), (63, 40, 21), (40, 20, 20), (63, 32, 31)]


def main():
    oracle.build()
    t0 = time.time()
    edges = linear_edges(SHELLS)
    dk, _ = make_field(FieldModel(n=N, box=BOX, sigma_g=0.3), SEED)
    # valid low-k bins from the counts of every candidate with a <= 4 (small shells: cheap)
    low = [(a, b, c) for a in range(5) for b in range(a + 1) for c in range(b + 1)]
    cnt = oracle.counts(N, edges, low)
    bins = [t for t, c in zip(low, cnt) if c >= 1] + SPREAD
    r = oracle.bispectrum(dk.astype(np.complex128), N, BOX, edges, (0, 2, 4), bins=bins)
    out = {
        "what": "FP64 oracle raw sums T^l = sum_x F^l_a F_b F_c and counts N_abc at 512^3, 64 shells of "
                "width 2 k_f from k_f, l = 0, 2, 4, field seed 1710 (sigma_g = 0.3), for a sample of bins",
        "script": "tests/golden/make_fullsize_512.py",
        "n": N, "box": BOX, "seed": SEED, "edges": edges, "ells": [0, 2, 4],
        "bins": [list(map(int, t)) for t in r["bins"]],
        "counts": [float(c) for c in r["counts"]],
        "T": [[float(v) for v in row] for row in r["T"]],
        "sumsq": [[float(v) for v in row] for row in r["sumsq"]],
        "oracle_seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(HERE, "fullsize_512_64shells.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("wrote %d bins in %.0f s" % (len(bins), time.time() - t0))


if __name__ == "__main__":
    main()
