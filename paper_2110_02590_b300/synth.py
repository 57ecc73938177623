"""Seeded synthetic transmission grids and load trajectories.

This module only draws inputs: bus/branch/generator tables, load
trajectories and augmented-Lagrangian parameter vectors.  It holds none of
the method's arithmetic (no AC power flow, no derivatives), so both the
CUDA path and the CPU oracle consume exactly the same arrays.

Random numbers come from xoshiro256** seeded through SplitMix64
(Blackman & Vigna, "Scrambled linear pseudorandom number generators",
2018), implemented here from the published definitions so a seed gives the
same network on every machine and numpy version.

Network shape (stand-in for the PGLIB PEGASE cases of Table 1):
  * buses placed uniformly in the unit square;
  * a random recursive spanning tree: bus i >= 1 links to one of the (up to)
    three nearest buses among 0..i-1, chosen uniformly;
  * chords until n_branch: a uniform bus a and a uniform choice among its
    eight nearest neighbours (``chords="local"``, the default, which keeps
    the near-planar structure and low LU fill of real grids) or among all
    buses (``chords="uniform"``, an expander-like stress case);
  * r ~ U(0.002, 0.02), x = r * U(3, 10), line charging b ~ U(0, 0.05);
    a fraction of branches are transformers with tap ~ U(0.95, 1.05);
  * loads on 60% of buses: P ~ U(0.1, 1.0) p.u., Q = P * U(0.1, 0.4);
  * generators on bus 0 (the slack) and n_gen - 1 distinct uniform buses;
    quadratic cost c2 ~ U(0.005, 0.02) $/MW^2h, c1 ~ U(10, 40) $/MWh,
    converted to per-unit power on baseMVA = 100;
  * each generator's share of load: every bus's load split equally among
    the generators nearest to it in hops (breadth-first search); the
    base-case dispatch is that share, P limits [0, 1.5 * max(share, mean/5)],
    Q limits [-pmax, pmax]; voltage bounds [0.94, 1.06];
  * flow limits: 1.2 x the base-case flows, the base case taken as the
    linearised (DC) flow of the share dispatch, floored at 0.1 p.u.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

MASK64 = (1 << 64) - 1


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & MASK64


class Xoshiro256ss:
    """xoshiro256** 1.0 with SplitMix64 seeding (both from their published definitions)."""

    def __init__(self, seed: int):
        z = seed & MASK64
        s = []
        for _ in range(4):
            z = (z + 0x9E3779B97F4A7C15) & MASK64
            w = z
            w = ((w ^ (w >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
            w = ((w ^ (w >> 27)) * 0x94D049BB133111EB) & MASK64
            s.append(w ^ (w >> 31))
        self.s = s

    def next(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & MASK64, 7) * 9) & MASK64
        t = (s[1] << 17) & MASK64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next() >> 11) * (1.0 / 9007199254740992.0))

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        if n <= 0:
            raise ValueError("below(n) needs n > 0")
        lim = (1 << 64) - ((1 << 64) % n)
        while True:
            r = self.next()
            if r < lim:
                return r % n

    def uniform_array(self, n: int, lo: float, hi: float) -> np.ndarray:
        return np.array([self.uniform(lo, hi) for _ in range(n)], dtype=np.float64)

    def sample(self, population: int, k: int) -> np.ndarray:
        """k distinct integers from range(population), partial Fisher-Yates."""
        idx = list(range(population))
        for i in range(k):
            j = i + self.below(population - i)
            idx[i], idx[j] = idx[j], idx[i]
        return np.array(idx[:k], dtype=np.int64)

    def normal(self) -> float:
        """Standard normal by the Box-Muller transform."""
        u1 = self.uniform()
        while u1 <= 0.0:
            u1 = self.uniform()
        u2 = self.uniform()
        return float(np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2))


@dataclass
class Network:
    """Raw network tables (per-unit on base_mva).  Generator g sits on gen_bus[g]."""
    n_bus: int
    n_branch: int
    n_gen: int
    ref_bus: int
    pd: np.ndarray
    qd: np.ndarray
    vmin: np.ndarray
    vmax: np.ndarray
    br_from: np.ndarray
    br_to: np.ndarray
    br_r: np.ndarray
    br_x: np.ndarray
    br_b: np.ndarray
    br_tap: np.ndarray
    br_rate: np.ndarray
    gen_bus: np.ndarray
    gen_c2: np.ndarray
    gen_c1: np.ndarray
    gen_c0: np.ndarray
    gen_pmin: np.ndarray
    gen_pmax: np.ndarray
    gen_qmin: np.ndarray
    gen_qmax: np.ndarray
    base_mva: float = 100.0
    seed: int = 0
    name: str = ""
    xy: np.ndarray = field(default=None, repr=False)
    gen_share: np.ndarray = field(default=None, repr=False)

    def copy_with_loads(self, pd: np.ndarray, qd: np.ndarray) -> "Network":
        import dataclasses
        return dataclasses.replace(self, pd=np.ascontiguousarray(pd, dtype=np.float64),
                                   qd=np.ascontiguousarray(qd, dtype=np.float64))


def _nearest(xy: np.ndarray, i: int, cand_hi: int, k: int) -> np.ndarray:
    d = np.hypot(xy[:cand_hi, 0] - xy[i, 0], xy[:cand_hi, 1] - xy[i, 1])
    k = min(k, cand_hi)
    order = np.lexsort((np.arange(cand_hi), d))  # distance, then index
    return order[:k]


def _tree_candidates(xy: np.ndarray):
    """For every bus i >= 1, the (up to) three nearest buses among 0..i-1 by (distance, index)."""
    from scipy.spatial import cKDTree
    n = xy.shape[0]
    k = min(n, 48)
    dist, idx = cKDTree(xy).query(xy, k)
    out = [None]
    for i in range(1, n):
        row = sorted((dist[i, j], idx[i, j]) for j in range(k) if idx[i, j] < i)
        if len(row) >= min(3, i):
            out.append(np.array([b for _, b in row[:3]], dtype=np.int64))
        else:
            out.append(_nearest(xy, i, i, 3))
    return out


def _knn_all(xy: np.ndarray, k: int) -> np.ndarray:
    """k nearest other buses of every bus, by distance then index."""
    from scipy.spatial import cKDTree
    n = xy.shape[0]
    kk = min(k + 1, n)
    dist, idx = cKDTree(xy).query(xy, kk)
    out = np.empty((n, kk - 1), dtype=np.int64)
    for i in range(n):
        row = [(dist[i, j], idx[i, j]) for j in range(kk) if idx[i, j] != i][: kk - 1]
        row.sort()
        out[i] = [b for _, b in row]
    return out


def _dc_flows(n_bus, ref, f, t, x, tap, pinj):
    """Linearised (DC) branch flows for a net injection vector; input shaping only."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    bser = 1.0 / (x * tap)
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([bser, bser, -bser, -bser])
    B = sp.csr_matrix((vals, (rows, cols)), shape=(n_bus, n_bus))
    keep = np.array([i for i in range(n_bus) if i != ref])
    th = np.zeros(n_bus)
    th[keep] = spl.spsolve(B[keep][:, keep].tocsc(), pinj[keep])
    return (th[f] - th[t]) * bser


def _regional_shares(n_bus, f, t, gen_bus, pd):
    """Each bus's load split equally among the generators nearest to it in hops."""
    import collections
    adj = [[] for _ in range(n_bus)]
    for a, b in zip(f.tolist(), t.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    share = np.zeros(len(gen_bus))
    # hop distance from every generator bus (multi-source BFS keeping all nearest owners)
    dist = np.full(n_bus, -1, dtype=np.int64)
    owners = [set() for _ in range(n_bus)]
    q = collections.deque()
    for g, b in enumerate(gen_bus.tolist()):
        dist[b] = 0
        owners[b].add(g)
        q.append(b)
    while q:
        b = q.popleft()
        for o in adj[b]:
            if dist[o] < 0:
                dist[o] = dist[b] + 1
                owners[o] |= owners[b]
                q.append(o)
            elif dist[o] == dist[b] + 1:
                owners[o] |= owners[b]
    for i in range(n_bus):
        if pd[i] != 0.0:
            own = sorted(owners[i])
            for g in own:
                share[g] += pd[i] / len(own)
    return share


def make_network(n_bus: int, n_gen: int, n_branch: int, seed: int,
                 transformer_frac: float = 0.1, chords: str = "local",
                 name: str = "", load_scale: float = 1.0) -> Network:
    if n_bus < 2 or n_gen < 1 or n_gen > n_bus:
        raise ValueError("need n_bus >= 2 and 1 <= n_gen <= n_bus")
    if n_branch < n_bus - 1 or n_branch > n_bus * (n_bus - 1) // 2:
        raise ValueError("n_branch must be between n_bus-1 and n_bus*(n_bus-1)/2")
    rng = Xoshiro256ss(seed)
    xy = np.array([[rng.uniform(), rng.uniform()] for _ in range(n_bus)])
    edges = set()
    f_list, t_list = [], []
    tree_parent = _tree_candidates(xy)
    for i in range(1, n_bus):
        cand = tree_parent[i]
        j = int(cand[rng.below(len(cand))])
        f_list.append(j)
        t_list.append(i)
        edges.add((min(i, j), max(i, j)))
    if chords == "local":
        knn = _knn_all(xy, 8)
    elif chords != "uniform":
        raise ValueError("chords must be 'local' or 'uniform'")
    while len(f_list) < n_branch:
        a = rng.below(n_bus)
        if chords == "local":
            b = int(knn[a][rng.below(knn.shape[1])])
        else:
            b = rng.below(n_bus)
        if a == b:
            continue
        key = (min(a, b), max(a, b))
        if key in edges:
            continue
        edges.add(key)
        f_list.append(a)
        t_list.append(b)
    nl = n_branch
    f = np.array(f_list, dtype=np.int32)
    t = np.array(t_list, dtype=np.int32)
    r = rng.uniform_array(nl, 0.002, 0.02)
    x = r * rng.uniform_array(nl, 3.0, 10.0)
    b = rng.uniform_array(nl, 0.0, 0.05)
    tap = np.ones(nl)
    n_tr = int(round(transformer_frac * nl))
    for k in rng.sample(nl, n_tr):
        tap[k] = rng.uniform(0.95, 1.05)
    # loads
    n_load = int(round(0.6 * n_bus))
    pd = np.zeros(n_bus)
    qd = np.zeros(n_bus)
    for i in rng.sample(n_bus, n_load):
        p = rng.uniform(0.1, 1.0)
        pd[i] = load_scale * p
        qd[i] = load_scale * p * rng.uniform(0.1, 0.4)
    # generators: bus 0 is the slack, the rest on distinct buses
    others = rng.sample(n_bus - 1, n_gen - 1) + 1
    gen_bus = np.concatenate([[0], np.sort(others)]).astype(np.int32)
    base = 100.0
    c2 = rng.uniform_array(n_gen, 0.005, 0.02) * base * base
    c1 = rng.uniform_array(n_gen, 10.0, 40.0) * base
    c0 = np.zeros(n_gen)
    share = _regional_shares(n_bus, f, t, gen_bus, pd)
    pmin = np.zeros(n_gen)
    pmax = 1.5 * np.maximum(share, 0.2 * share.mean())
    qmin = -pmax.copy()
    qmax = pmax.copy()
    vmin = np.full(n_bus, 0.94)
    vmax = np.full(n_bus, 1.06)
    # flow limits from the DC flows of the equal-share dispatch
    pinj = -pd.copy()
    pinj[gen_bus] += share
    flows = _dc_flows(n_bus, 0, f, t, x, tap, pinj)
    rate = np.maximum(1.2 * np.abs(flows), 0.1)
    return Network(n_bus=n_bus, n_branch=nl, n_gen=n_gen, ref_bus=0,
                   pd=pd, qd=qd, vmin=vmin, vmax=vmax,
                   br_from=f, br_to=t, br_r=r, br_x=x, br_b=b, br_tap=tap, br_rate=rate,
                   gen_bus=gen_bus, gen_c2=c2, gen_c1=c1, gen_c0=c0,
                   gen_pmin=pmin, gen_pmax=pmax, gen_qmin=qmin, gen_qmax=qmax,
                   base_mva=base, seed=seed, name=name, xy=xy, gen_share=share)


# Workloads (sizes of the synthetic stand-ins; seeds fixed per workload).
# load_scale: the specified loads make some pockets of these grids collapse
# (no AC solution at full load); each workload runs at 75% of its
# loadability limit found by load continuation, capped at 1 (values
# reproduced by tests/golden/find_load_scale.py).
WORKLOADS = {
    "tiny30": dict(n_bus=30, n_gen=6, n_branch=41, seed=0, transformer_frac=0.1, load_scale=1.0),
    "medium1400": dict(n_bus=1400, n_gen=260, n_branch=2000, seed=1, transformer_frac=0.1,
                       load_scale=0.45),
    "large9200": dict(n_bus=9200, n_gen=1450, n_branch=16000, seed=2, transformer_frac=0.2,
                      load_scale=0.75),
    "batchA500": dict(n_bus=500, n_gen=90, n_branch=715, seed=3, transformer_frac=0.1,
                      load_scale=0.90),
    "batchB2000": dict(n_bus=2000, n_gen=300, n_branch=2860, seed=4, transformer_frac=0.1,
                       load_scale=0.45),
    "big20000": dict(n_bus=20000, n_gen=3000, n_branch=34000, seed=5, transformer_frac=0.1,
                     load_scale=0.60),
}

_CACHE: dict = {}


def workload(name: str, chords: str = "local") -> Network:
    key = (name, chords)
    if key not in _CACHE:
        _CACHE[key] = make_network(chords=chords, name=name, **WORKLOADS[name])
    return _CACHE[key]


def flat_control(net: Network) -> np.ndarray:
    """Controls u = (v_ref, v_pv, p_pv) of the base case: |V| = 1, each generator at its share.

    PV buses are the generator buses other than the slack, in ascending bus order.
    """
    gen_of = {int(b): g for g, b in enumerate(net.gen_bus)}
    pv = sorted(int(b) for b in net.gen_bus if int(b) != net.ref_bus)
    return np.concatenate([[1.0], np.ones(len(pv)), net.gen_share[[gen_of[b] for b in pv]]])


def flat_state(net: Network) -> np.ndarray:
    """Flat start x = (theta_pv, theta_pq, v_pq) = (0, 0, 1)."""
    n_pv = net.n_gen - 1
    n_pq = net.n_bus - net.n_gen
    return np.concatenate([np.zeros(n_pv + n_pq), np.ones(n_pq)])


def ar1_loads(net: Network, n_steps: int, seed: int, phi: float = 0.99, sd: float = 0.01):
    """Load trajectories p_t = p_nom (1 + a_t), a_t = phi a_{t-1} + sd * eps_t, per bus.

    Reactive loads scale by the same factor.  Returns (pd[n_steps, n_bus], qd[n_steps, n_bus]).
    """
    rng = Xoshiro256ss(seed)
    a = np.zeros(net.n_bus)
    pds = np.empty((n_steps, net.n_bus))
    qds = np.empty((n_steps, net.n_bus))
    for s in range(n_steps):
        eps = np.array([rng.normal() for _ in range(net.n_bus)])
        a = phi * a + sd * eps
        pds[s] = net.pd * (1.0 + a)
        qds[s] = net.qd * (1.0 + a)
    return pds, qds


def constraint_count(net: Network) -> int:
    return 2 * net.n_branch + (net.n_bus - net.n_gen) + (net.n_gen - 1) + 2


def al_inputs(net: Network, seed: int, rho: float = 10.0, sigma_f: float = 1e-4,
              y_scale: float = 0.1) -> dict:
    """Seeded augmented-Lagrangian inputs (sigma_c, y, s, rho, sigma_f), independent of any solve.

    Constraint order: (|S_f|^2 per branch, |S_t|^2 per branch, v_pq, p_ref, q_ref, q_pv).
    sigma_c = 1/rate^2 on line flows and 1 elsewhere; s is drawn strictly inside its bounds.
    """
    rng = Xoshiro256ss(seed)
    m = constraint_count(net)
    nl = net.n_branch
    pv = sorted(int(b) for b in net.gen_bus if int(b) != net.ref_bus)
    pq = sorted(set(range(net.n_bus)) - set(int(b) for b in net.gen_bus))
    gen_of = {int(b): g for g, b in enumerate(net.gen_bus)}
    g_ref = gen_of[net.ref_bus]
    lo = np.concatenate([np.zeros(2 * nl), net.vmin[pq], [net.gen_pmin[g_ref], net.gen_qmin[g_ref]],
                         net.gen_qmin[[gen_of[b] for b in pv]]])
    hi = np.concatenate([net.br_rate ** 2, net.br_rate ** 2, net.vmax[pq],
                         [net.gen_pmax[g_ref], net.gen_qmax[g_ref]],
                         net.gen_qmax[[gen_of[b] for b in pv]]])
    sigma_c = np.concatenate([1.0 / net.br_rate ** 2, 1.0 / net.br_rate ** 2, np.ones(m - 2 * nl)])
    frac = rng.uniform_array(m, 0.2, 0.8)
    s = lo + frac * (hi - lo)
    y = rng.uniform_array(m, -y_scale, y_scale)
    return dict(sigma_f=float(sigma_f), sigma_c=sigma_c, y=y, s=s, rho=float(rho), s_lo=lo, s_hi=hi)


def static_instance(net: Network, al: dict, c_base: np.ndarray, margin: float = 1.2,
                    v_margin: float = 0.02) -> dict:
    """Bounds of a static OPF instance whose AC base case is feasible (a copy of `al` with new s_lo,
    s_hi and sigma_c).  c_base: the constraint values at the base case (the flat control's power
    flow at nominal loads, computed by the caller).

    - line flows: limit r^2 = max(rate, margin |S|)^2, |S| the larger end's base-case flow; the
      squared flows have only this upper limit, so their lower bound is the inactive -r^2 (a bound
      of 0 is degenerate on a zero-flow branch); sigma_c = 1 / r^2;
    - reactive generation (q_ref, q_pv): limits widened to cover margin |q| of the base case;
    - PQ voltages: bounds widened to cover (1 -/+ v_margin) times the base-case voltage.
    """
    nl = net.n_branch
    npv = len([b for b in net.gen_bus if int(b) != net.ref_bus])
    m = constraint_count(net)
    npq = m - 2 * nl - 2 - npv
    c_base = np.asarray(c_base, dtype=np.float64)
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in al.items()}
    lo, hi, sig = out["s_lo"], out["s_hi"], out["sigma_c"]
    r2 = np.maximum(net.br_rate ** 2, margin ** 2 * np.maximum(c_base[:nl], c_base[nl:2 * nl]))
    hi[:2 * nl] = np.concatenate([r2, r2])
    lo[:2 * nl] = -hi[:2 * nl]
    sig[:2 * nl] = 1.0 / hi[:2 * nl]
    v = slice(2 * nl, 2 * nl + npq)
    lo[v] = np.minimum(lo[v], (1.0 - v_margin) * c_base[v])
    hi[v] = np.maximum(hi[v], (1.0 + v_margin) * c_base[v])
    q = slice(2 * nl + npq + 1, m)
    qb = margin * np.abs(c_base[q])
    lo[q] = np.minimum(lo[q], -qb)
    hi[q] = np.maximum(hi[q], qb)
    return out


def control_bounds(net: Network):
    """Bounds of u = (v_ref, v_pv, p_pv)."""
    pv = sorted(int(b) for b in net.gen_bus if int(b) != net.ref_bus)
    gen_of = {int(b): g for g, b in enumerate(net.gen_bus)}
    lo = np.concatenate([[net.vmin[net.ref_bus]], net.vmin[pv], net.gen_pmin[[gen_of[b] for b in pv]]])
    hi = np.concatenate([[net.vmax[net.ref_bus]], net.vmax[pv], net.gen_pmax[[gen_of[b] for b in pv]]])
    return lo, hi
