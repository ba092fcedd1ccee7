"""Write the stored expected values under tests/golden/.

Calls only the input generator (``inputs``) and the oracle (``oracle``):
no stored value comes from the CUDA library.

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import inputs  # noqa: E402
import oracle  # noqa: E402


def input_hashes():
    out = {}
    for dtype in ("uint32", "uint64"):
        for dist in inputs.DISTS:
            k = inputs.keys(np.dtype(dtype), dist, 2**20)
            out[f"{dtype}:{dist}"] = hashlib.sha256(k.tobytes()).hexdigest()
    return out


def oracle_hashes():
    """SHA-256 of the oracle's sorted keys and values for a few small cases."""
    out = {}
    for dtype in ("uint32", "uint64"):
        for dist in inputs.DISTS:
            n = 3 * 2**15  # 2^16 + 2^15, a non-power-of-two length (Sec. 3)
            k = inputs.keys(np.dtype(dtype), dist, n)
            v = inputs.values(np.dtype(dtype), n)
            sk, sv = oracle.lsd_sort(k, v)
            out[f"{dtype}:{dist}:{n}"] = {
                "keys": hashlib.sha256(sk.tobytes()).hexdigest(),
                "vals": hashlib.sha256(sv.tobytes()).hexdigest(),
            }
    return out


def main():
    with open(os.path.join(HERE, "inputs_sha256.json"), "w") as f:
        json.dump(input_hashes(), f, indent=1, sort_keys=True)
        f.write("\n")
    with open(os.path.join(HERE, "oracle_sha256.json"), "w") as f:
        json.dump(oracle_hashes(), f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
