"""Writes the regression fixtures in this folder from the FP64 oracle only.

These are not pins (the oracle's pins are in test_oracle_pins.py); they
freeze the oracle's exact integer outputs so that an accidental change to
its sampler or random stream shows up as a diff:
  * philox_blocks.txt: Philox4x32-10 blocks for a few counters and keys;
  * binomial_inversion.txt: exact-branch survivor counts (CDF inversion of
    the Sec. 3.1 reading) for fixed (N, p) and 32-bit words.
Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

PHILOX_CASES = [((0, 0, 0, 0), (0, 0)), ((1, 2, 3, 4), (5, 6)), ((0xFFFFFFFF, 7, 0x1234, 9), (0xDEADBEEF, 0x12345)),
                ((0, 3000 * 6000 + 17, 99999, (5 << 4) | 2), (0x89ABCDEF, 0x01234567))]
INV_CASES = [(1, 0.7), (5, 0.7), (20, 0.7), (32, 0.3), (64, 0.5), (13, 0.999), (9, 0.01)]


def words() -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(20220305))
    w = rng.integers(0, 2 ** 32, 48, dtype=np.uint64).astype(np.uint32)
    return np.concatenate([np.array([0, 0xFFFFFFFF, 0x80000000, 0x4CCCCCCC], np.uint32), w])


def main():
    with open(os.path.join(HERE, "philox_blocks.txt"), "w") as f:
        f.write("# counter(4) key(2) -> block(4), hex; oracle.philox (Philox4x32-10, SC'11)\n")
        for c, k in PHILOX_CASES:
            b = oracle.philox(c, k)
            f.write(" ".join(f"{v:08x}" for v in (*c, *k, *b)) + "\n")
    w = words()
    with open(os.path.join(HERE, "binomial_inversion.txt"), "w") as f:
        f.write("# N p : counts for the words below (oracle.binomial_invert, exact branch of the Sec. 3.1 reading)\n")
        f.write("words " + " ".join(f"{v:08x}" for v in w) + "\n")
        for N, p in INV_CASES:
            k = oracle.binomial_invert(N, p, w)
            f.write(f"{N} {p!r} : " + " ".join(str(int(v)) for v in k) + "\n")


if __name__ == "__main__":
    main()
