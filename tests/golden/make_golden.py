"""Writes the regression fixtures in this folder from the FP64 oracle only.

These are not pins (the oracle's pins are in test_oracle_pins.py); they
freeze the oracle's exact integer outputs so that an accidental change to
its sampler or random stream shows up as a diff:
  * philox_blocks.txt: Philox4x32-10 blocks for a few counters and keys;
  * binomial_inversion.txt: exact-branch survivor counts (CDF inversion of
    the Sec. 3.1 reading) for fixed (N, p) and 32-bit words;
  * binomial_bins.txt: per-bin survivor counts of both branches for fixed
    (seed, event, plane, depo, wire, tick) on the quad random stream.
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
# (N, p, seed, wire, tick, depo, event, plane, nticks): exact and normal branches, all four words of a quad
BIN_CASES = [(20, 0.7, 0xDEADBEEF12345, 17, 4000 + t, 99, 5, 2, 6000) for t in range(4)] + \
            [(5000, 0.7, 0xDEADBEEF12345, 17, 4000 + t, 99, 5, 2, 6000) for t in range(4)] + \
            [(33, 0.3, 1001, 0, 0, 0, 0, 0, 6000), (3, 0.5, 7, 959, 5999, 123456, 63, 1, 6000),
             (40000, 0.5, 1, 2, 3, 4, 0, 0, 6250), (60, 0.62, 9, 3, 6249, 1, 0, 0, 6250)]


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
    with open(os.path.join(HERE, "binomial_bins.txt"), "w") as f:
        f.write("# N p seed wire tick depo event plane nticks -> count (oracle.binomial, exact_max 32)\n")
        for N, p, seed, w, t, d, ev, pl, nt in BIN_CASES:
            k = oracle.binomial(N, p, seed, w, t, d, event_id=ev, plane_id=pl, nticks=nt)
            f.write(f"{N} {p!r} {seed} {w} {t} {d} {ev} {pl} {nt} {k}\n")


if __name__ == "__main__":
    main()
