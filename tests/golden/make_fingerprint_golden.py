"""Writes fingerprint_alg1.txt: Algorithm 1 (Sec. V) worked step by step on a few determinants.

The orbital map values come from the oracle's Philox4x32-10 (itself pinned to the published
known-answer vectors) with the map key ("FCIQ", "MAP1") and counter (k, 0, 0, 0); every step of the
recurrence hash <- p hash + map(orbital_i) i (p = 1099511628211, i counted from 1 over the occupied
spin orbitals in ascending order, arithmetic modulo 2^64) is written out so that each line can be
checked by hand. Run from the repository root: python tests/golden/make_fingerprint_golden.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import oracle as O  # noqa: E402

P = 1099511628211
KEY = (0x46434951, 0x4D415031)  # "FCIQ", "MAP1" as 32-bit words
CASES = [[5], [0, 1], [3, 7, 10], [1, 4, 9, 30], [0, 2, 65, 100], [63, 64, 126, 127]]


def map_value(k: int) -> int:
    o = O.philox([k, 0, 0, 0], list(KEY))
    return o[0] | (o[1] << 32)


def main():
    lines = ["# Algorithm 1 (Sec. V) worked by hand: hash = 0; for i = 1..N: hash <- p*hash + map(det(i))*i,",
             "# p = 1099511628211, arithmetic modulo 2^64 (the paper's final abs/mod over a range is not applied).",
             "# map(k) = out0 | out1 << 32 of Philox4x32-10 with key (0x46434951, 0x4D415031), counter (k, 0, 0, 0).",
             "# Written by tests/golden/make_fingerprint_golden.py.",
             "# map <spin orbital> <map value, hex>"]
    orbs = sorted({k for c in CASES for k in c})
    for k in orbs:
        lines.append(f"map {k} {map_value(k):016x}")
    lines.append("# case <occupied spin orbitals, ascending, comma-separated> <hash after i = 1 .. N, hex>")
    for c in CASES:
        h, steps = 0, []
        for i, k in enumerate(c, start=1):
            h = (P * h + map_value(k) * i) % (1 << 64)
            steps.append(f"{h:016x}")
        lines.append("case " + ",".join(map(str, c)) + " " + " ".join(steps))
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "fingerprint_alg1.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
