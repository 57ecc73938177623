"""Small hand-built networks for the tests (inputs only, no method arithmetic)."""
import dataclasses

import numpy as np

from paper_2110_02590_b300 import synth


def custom_network(n_bus, branches, gen_bus, pd, qd, rate=None, c2=None, c1=None):
    """branches: list of (f, t, r, x, b, tap)."""
    br = np.array(branches, dtype=np.float64)
    nl = len(branches)
    ng = len(gen_bus)
    c2 = np.full(ng, 100.0) if c2 is None else np.asarray(c2, float)
    c1 = np.full(ng, 2000.0) if c1 is None else np.asarray(c1, float)
    share = np.full(ng, np.sum(pd) / ng)
    return synth.Network(
        n_bus=n_bus, n_branch=nl, n_gen=ng, ref_bus=int(gen_bus[0]),
        pd=np.asarray(pd, float), qd=np.asarray(qd, float),
        vmin=np.full(n_bus, 0.9), vmax=np.full(n_bus, 1.1),
        br_from=br[:, 0].astype(np.int32), br_to=br[:, 1].astype(np.int32),
        br_r=br[:, 2].copy(), br_x=br[:, 3].copy(), br_b=br[:, 4].copy(), br_tap=br[:, 5].copy(),
        br_rate=np.full(nl, 1.0) if rate is None else np.asarray(rate, float),
        gen_bus=np.asarray(gen_bus, np.int32), gen_c2=c2, gen_c1=c1, gen_c0=np.zeros(ng),
        gen_pmin=np.zeros(ng), gen_pmax=np.full(ng, 10.0), gen_qmin=np.full(ng, -10.0),
        gen_qmax=np.full(ng, 10.0), gen_share=share, name="custom")


def with_branch_r(net, r):
    return dataclasses.replace(net, br_r=np.asarray(r, float))


def with_costs(net, c2, c1):
    return dataclasses.replace(net, gen_c2=np.asarray(c2, float), gen_c1=np.asarray(c1, float))
