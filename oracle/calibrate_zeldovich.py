"""Amplitude of the Zel'dovich displacement for the CIC workload (128^3
particles on a 128^3 grid, displacement seed 2000).

The workload asks for a per-cell contrast of about 100.  A one-particle-per-
cell Zel'dovich field with P(k) ~ k^-1.5 does not get there: past shell
crossing its CIC density saturates in sheets at a few tens.  The amplitude
used is therefore the one (on a grid of amplitudes, in box units times the
grid size) that maximises max(rho - 1) of the oracle's CIC density.  Test
infrastructure: calls only the oracle and the seeded generators; its printed
value is stored in paper_1110_1379_gb300/synth.py (ZELDOVICH_AMPLITUDE_128).

    python -m oracle.calibrate_zeldovich
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1110_1379_gb300 import synth  # noqa: E402


def peak(amp, n=128, seed=2000):
    pos = synth.zeldovich_positions(n, seed, amplitude=amp)
    return float(O.cic(pos, (n, n, n)).max() - 1.0)


def calibrate(lo=20.0, hi=80.0, step=2.5):
    best = (None, -1.0)
    a = lo
    while a <= hi + 1e-9:
        p = peak(a)
        if p > best[1]:
            best = (a, p)
        a += step
    return best


if __name__ == "__main__":
    a, p = calibrate()
    print(f"{a:.2f} max(rho-1) = {p:.2f}")
