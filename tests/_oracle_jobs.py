"""Oracle work items for a process pool (spawn context), so that the many
independent lattices of a parity test can run on all host cores.  Each item
is a plain call into ``oracle``; nothing here touches the GPU."""
import numpy as np


def run(dims, L, beta, seed, start, nsweeps, every, s=None, t0=0, heatbath=False):
    import oracle
    s_out, E, M = oracle.run(dims, L, beta, seed, nsweeps, measure_every=every, start=start,
                             s=s, t0=t0, heatbath=heatbath)
    return s_out, E, M


def one_sweep(dims, L, beta, seed, s, t):
    import oracle
    s = np.ascontiguousarray(s, dtype=np.int8).copy()
    oracle.sweep(dims, L, s, seed, oracle.thresholds(dims, beta), t)
    return s, oracle.energy(dims, L, s), oracle.magnetization(dims, L, s)


def observables(dims, L, s):
    import oracle
    return oracle.energy(dims, L, s), oracle.magnetization(dims, L, s)
