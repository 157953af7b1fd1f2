"""Writes oracle_tiny_ngs_32.json: regression values of the FP64 oracle on the
32x32 three-NGS workload.  Calls only oracle/ and the seeded input generator."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2510_19542_gb300 import synth  # noqa: E402


def main():
    g = synth.config(1)
    out = oracle.OraclePlan(g).reconstruct(synth.frame(g))
    rng = np.random.default_rng(12345)
    lpq = np.stack([rng.integers(0, out.shape[0], 16), rng.integers(0, 32, 16),
                    rng.integers(0, 32, 16)], axis=1)
    gold = {
        "_source": "oracle.OraclePlan(synth.config(1)).reconstruct(synth.frame(synth.config(1)))",
        "layer_rms": np.sqrt(np.mean(out ** 2, axis=(1, 2))).tolist(),
        "sample_lpq": lpq.tolist(),
        "sample_values": out[lpq[:, 0], lpq[:, 1], lpq[:, 2]].tolist(),
    }
    with open(os.path.join(HERE, "oracle_tiny_ngs_32.json"), "w") as f:
        json.dump(gold, f, indent=1)


if __name__ == "__main__":
    main()
