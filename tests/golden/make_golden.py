"""Writes the stored expected values under tests/golden/.

Calls only the seeded generator (``synthetic``) and the CPU oracle; never the
CUDA library.  Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic  # noqa: E402
from oracle import strings  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def generator_digests():
    out = {}
    for name, w in synthetic.WORKLOADS.items():
        I = synthetic.integrals(w["norb"], w["nalpha"], w["nbeta"], w["seed"])
        out[name] = {
            "seed": w["seed"],
            "h1": synthetic.array_digest(I.h1),
            "eri": synthetic.array_digest(I.eri),
            "dipole": synthetic.array_digest(I.dipole),
        }
    return out


def table_digests():
    """SHA-256 of the brute-force excitation tables (int32 tgt, uint16 pq, int8 sgn)."""
    out = {}
    for n, m in [(8, 4), (10, 5), (12, 6), (14, 7)]:
        masks, tgt, pq, sgn = strings.excitation_table(n, m)
        out[f"{n}_{m}"] = {
            "nstrings": int(len(masks)),
            "masks": synthetic.array_digest(masks.astype(np.int64)),
            "tgt": synthetic.array_digest(tgt),
            "pq": synthetic.array_digest(pq),
            "sgn": synthetic.array_digest(sgn),
        }
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "generator_sha256.json"), "w") as f:
        json.dump(generator_digests(), f, indent=1, sort_keys=True)
    with open(os.path.join(HERE, "tables_sha256.json"), "w") as f:
        json.dump(table_digests(), f, indent=1, sort_keys=True)
    print("wrote", os.listdir(HERE))
