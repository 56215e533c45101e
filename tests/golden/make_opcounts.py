"""Writes opcount_mech53.json: the FP64 operation counts of one rate evaluation, one analytical
Jacobian (with its own rate evaluation), one LU factorization and one LU solve, counted by the
CPU oracle's operation-counting scalar type on the 53-species / 325-reaction synthetic mechanism.
The benchmark turns them into the algorithmic FLOPs of its roofline.  Run:
    python tests/golden/make_opcounts.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2105_12070_gb300 import synth  # noqa: E402  (input generator only)


def main():
    w = synth.workload_shear_layer(16)
    ora = oracle.OracleMechanism(w["mech"].write_temp())
    counts = ora.opcount(w["p_Pa"], float(w["T"][100]), w["Y"][:, 100])
    out = {"mechanism": "synthetic, seed 2, 53 species, 325 reactions (30 third-body, 25 Troe)", "N": ora.N,
           "counts": counts, "generated_by": "tests/golden/make_opcounts.py (oracle operation count)"}
    with open(os.path.join(HERE, "opcount_mech53.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
