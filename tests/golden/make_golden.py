"""Write the stored oracle values under tests/golden/.

Calls only ``oracle/`` and the seeded input generators; no value here comes
from the CUDA library.  Re-run after any change to the oracle's arithmetic:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import qwb_oracle as O  # noqa: E402
from paper_2506_00976_gb300 import synth  # noqa: E402


def blobs3_32():
    """Single pair of 32 x 32 three-blob measures, kappa = 4, p = 2, with the
    exact W_2 of the full 1024 x 1024 problem."""
    N, kappa, p = 32, 4, 2.0
    mu, nu = synth.make_measure(N, "blobs3", 0, 0), synth.make_measure(N, "blobs3", 0, 1)
    b = O.bounds(mu, nu, N, kappa, p)
    out = {"N": N, "kappa": kappa, "p": p, "classes": "blobs3 images 0 and 1, workload 0",
           "w_exact": O.wasserstein_exact(mu, nu, N, p),
           "lb": b["lb"], "lb_p": b["lb_p"], "ub_weighted": b["ub_weighted"],
           "ub_primal": b["ub_primal"], "w_hat_p": b["w_hat_p"],
           "lb_mincost": O.lb_mincost(mu, nu, N, kappa, p)}
    with open(os.path.join(HERE, "blobs3_32_k4_p2.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(out)


if __name__ == "__main__":
    blobs3_32()
