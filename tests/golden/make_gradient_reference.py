"""Writes gradient_2p20_20000.npz: the FP64 oracle's state of the moving-gradient
workload (stable variant: linear eps ramp 1 -> 2 over 2^18 of 2^20 cells,
v = 0.7c, S = 0.5, source and probe as in workloads.config4) after 20000 steps,
for the precision-tier test of the GPU path.  Calls only the oracle.

The fields are exactly zero outside the cells the source's pulse has reached,
so the file keeps the window [lo, hi) that holds every nonzero value of B and
D, plus the probe's DFT.  Run from the repository root:
    python tests/golden/make_gradient_reference.py      (about half an hour)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2304_06586_gb300 import workloads as w  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gradient_2p20_20000.npz")


def main(n_steps=20000):
    wl = w.config4("stable", n_steps=n_steps)
    I = wl.instances[0]
    o = oracle.Instance(I.nz, wl.S, I.beta, kind=I.kind, interp=I.interp, z=I.z, eps=I.eps, mu=I.mu)
    for s in I.sources:
        o.add_source(*s)
    for p in I.probes:
        o.add_probe(p[0], p[1])
    t0 = time.time()
    o.run(n_steps)
    nzb = np.nonzero((o.B != 0) | (o.D != 0))[0]
    lo, hi = int(nzb[0]), int(nzb[-1]) + 1
    np.savez_compressed(OUT, lo=lo, hi=hi, nz=I.nz, n_steps=n_steps, B=o.B[lo:hi], D=o.D[lo:hi],
                        spectrum=o.spectrum(0), bins=I.probes[0][1])
    print("wrote %s: window [%d, %d), %.0f s" % (OUT, lo, hi, time.time() - t0))


if __name__ == "__main__":
    main()
