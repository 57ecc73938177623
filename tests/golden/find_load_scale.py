"""Offline choice of each workload's load level (calls only the generator and the oracle).

For each workload, the loadability limit lambda* is the largest multiple of
0.05 reached by load continuation (all loads and the generators' shares
scaled together, Newton-Raphson warm-started from the previous point).  The
workload runs at load_scale = 0.75 * lambda*, rounded down to 0.05, which
leaves a 25% loading margin for the load trajectories (capped at 1: loads
are never raised above the specified distribution).  The chosen values
are stored in ``WORKLOADS`` of the synthetic-input module; the test
``test_workload_feasible`` checks that Newton-Raphson from the flat start
converges at them.

Usage:  python tests/golden/find_load_scale.py [workload ...]
"""
import sys
import os
import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
from paper_2110_02590_b300 import synth  # noqa: E402
import oracle  # noqa: E402


def loadability(name: str) -> float:
    kw = dict(synth.WORKLOADS[name])
    kw.pop("load_scale", None)
    net = synth.make_network(name=name, load_scale=1.0, **kw)
    on = oracle.OracleNet(net)
    u0 = synth.flat_control(net)
    x = None
    best = 0.0
    for a in np.arange(0.05, 2.0001, 0.05):
        u = u0.copy()
        u[1 + on.npv:] *= a
        xx, info = on.powerflow(u, pd=net.pd * a, qd=net.qd * a, x0=x)
        if info["rc"] != 0:
            break
        x, best = xx, round(float(a), 2)
    return best


if __name__ == "__main__":
    names = sys.argv[1:] or list(synth.WORKLOADS)
    for name in names:
        lam = loadability(name)
        scale = min(1.0, np.floor(0.75 * lam / 0.05 + 1e-9) * 0.05)
        print(f"{name}: loadability {lam:.2f} -> load_scale {scale:.2f}", flush=True)
