"""Write tests/golden/oracle_tiny.txt from the oracle alone.

The paper prints no worked example with numbers (its Table 1 compares against
MNE-python, which is not available), so this fixture is a regression lock on
the oracle: a tiny CWT computed by oracle/ and nothing else.  Regenerate it
only together with a change to the oracle's arithmetic, and name in that
commit the passage of the paper that justifies the change.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402

TINY = dict(n=24, N=32, fs=64.0, freqs=(3.0, 9.5, 20.0), n_cycles=(3.0, 5.0, 7.0), seed=20250607)


def compute(n, N, fs, freqs, n_cycles, seed):
    """Rows: for each scale, [Re c(t) for t < n] then [Im c(t) for t < n]."""
    x = np.random.default_rng(seed).standard_normal(n)
    c = oracle.cwt(x, N, fs, list(freqs), list(n_cycles), threads=1)[0]
    return np.concatenate([c.real, c.imag], axis=0)


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny.txt")
    rows = compute(**TINY)
    header = ("Oracle regression fixture, written by tests/golden/make_golden.py from oracle/ only.\n"
              f"Parameters: {TINY}.  Rows 0..S-1: Re c_s(t); rows S..2S-1: Im c_s(t).\n"
              "Definition: cyclic convolution with the unit-energy periodised Morlet wavelet "
              "(Eq. 2, Eq. 3).")
    np.savetxt(out, rows, fmt="%.17e", header=header)
    print(out)


if __name__ == "__main__":
    main()
