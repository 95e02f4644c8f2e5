"""Write the stored oracle outputs used as regression fixtures.

Calls only the oracle and the seeded input generators:
    python tests/golden/make_golden.py
Fixture scurve_n2048.json: the 2048-point s-curve (seed 0) with the bandwidth
eps = median squared pairwise distance, and the top-10 eigenvalues of the
symmetric diffusion matrix S (Algorithm 1 with alpha = 1, S the symmetric
conjugate of the Markov matrix) from the oracle's full-reorthogonalisation
Lanczos (Algorithm 2, symmetric case).
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import synth  # noqa: E402


def main():
    X = synth.as_f32(synth.s_curve(2048, 0))
    eps = O.median_sqdist(X)
    q, dg, s = O.degrees(X, eps, 1.0)
    ev, _, it, st = O.lanczos_S(X, eps, s, 10, conv_tol=1e-10)
    assert st == 0
    out = {"workload": "s-curve N=2048 d=3 seed 0, alpha=1, eps=median squared distance",
           "eps": eps, "evals_top10": [float(v) for v in ev], "lanczos_iterations": it}
    with open(os.path.join(HERE, "scurve_n2048.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
