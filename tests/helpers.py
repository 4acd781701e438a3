"""Shared test helpers: configure the CUDA path and the oracle from one workload spec."""
import numpy as np


def make_sim(wl, prec=None, tuning=None, allow_unstable=True):
    from paper_2304_06586_gb300 import binding as gb
    sim = gb.Simulation([i.nz for i in wl.instances], wl.S, gb.F32 if prec is None else prec)
    for k, I in enumerate(wl.instances):
        sim.set_medium(k, I.kind, I.beta, I.interp, I.z, I.eps, I.mu, allow_unstable)
        for s in I.sources:
            sim.add_source(k, *s)
        for p in I.probes:
            sim.add_probe(k, p[0], p[1])
    if tuning:
        sim.set_tuning(*tuning)
    return sim


def make_oracle(wl):
    import oracle
    out = []
    for I in wl.instances:
        o = oracle.Instance(I.nz, wl.S, I.beta, kind=I.kind, interp=I.interp, z=I.z, eps=I.eps, mu=I.mu)
        for s in I.sources:
            o.add_source(*s)
        for p in I.probes:
            o.add_probe(p[0], p[1])
        out.append(o)
    return out


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
