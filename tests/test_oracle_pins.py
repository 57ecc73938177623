"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: values
printed in the paper (Table 1), textbook closed forms, conservation laws,
finite differences of independently re-solved power flows, a brute force
built from hyper-dual numbers on the complex-voltage form of the power-flow
equations, and the graph-theoretic characterisation of LU fill.
"""
import collections
import dataclasses
import json
import os

import numpy as np
import pytest

import oracle
from paper_2110_02590_b300 import synth
from tests.netutil import custom_network, with_branch_r, with_costs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _solve(name_or_net):
    net = synth.workload(name_or_net) if isinstance(name_or_net, str) else name_or_net
    on = oracle.OracleNet(net)
    u = synth.flat_control(net)
    x, info = on.powerflow(u, tol=1e-12, max_it=30)
    assert info["rc"] == 0, info
    return net, on, u, x


# ---------------------------------------------------------------- dimensions

def test_dimensions_match_table1():
    """n_x = n_pv + 2 n_pq, n_u = 2 n_pv + 1, m = 2 n_l + n_pq + n_pv + 2 reproduce Table 1."""
    with open(os.path.join(GOLDEN, "table1_dims.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        n_pv = (case["n_u"] - 1) // 2
        net = synth.make_network(case["n_v"], n_pv + 1, case["n_e"], seed=11)
        on = oracle.OracleNet(net)
        assert (on.nx, on.nu, on.m) == (case["n_x"], case["n_u"], case["m"]), case["case"]


@pytest.mark.parametrize("name,dims", [("tiny30", (53, 11, 113)), ("medium1400", (2539, 519, 5401)),
                                       ("large9200", (16949, 2899, 41201)),
                                       ("batchA500", (909, 179, 1931)), ("batchB2000", (3699, 599, 7721))])
def test_workload_dimensions(name, dims):
    on = oracle.OracleNet(synth.workload(name))
    assert (on.nx, on.nu, on.m) == dims


# ---------------------------------------------------------------- power flow

def test_powerflow_two_bus_closed_form():
    """Slack V1 = 1, PQ load S = P + jQ through z = r + jx (no shunt): textbook |V2| and loss."""
    r, x, P, Q = 0.02, 0.08, 0.8, 0.3
    net = custom_network(2, [(0, 1, r, x, 0.0, 1.0)], gen_bus=[0], pd=[0.0, P], qd=[0.0, Q])
    on = oracle.OracleNet(net)
    assert (on.nx, on.nu) == (2, 1)
    u = np.array([1.0])
    xs, info = on.powerflow(u, tol=1e-13)
    assert info["rc"] == 0
    a = 1.0 - 2.0 * (r * P + x * Q)
    v2sq = 0.5 * (a + np.sqrt(a * a - 4.0 * (r * r + x * x) * (P * P + Q * Q)))
    assert abs(xs[1] - np.sqrt(v2sq)) < 1e-12
    ev = on.eval(xs, u)
    loss = r * (P * P + Q * Q) / v2sq
    assert abs(ev["P"][0] - (P + loss)) < 1e-12  # slack covers load plus series loss


@pytest.mark.parametrize("name", ["tiny30", "medium1400", "batchA500", "batchB2000"])
def test_powerflow_residual_and_loss_balance(name):
    """||g||_2 < 1e-10 (stop test of the paper) and generation - load = sum of series losses."""
    net = synth.workload(name)
    on = oracle.OracleNet(net)
    u = synth.flat_control(net)
    x, info = on.powerflow(u)
    assert info["rc"] == 0 and info["res2"] < 1e-10
    ev = on.eval(x, u)
    assert np.linalg.norm(ev["g"]) < 1e-10
    # complex voltages, independent series-loss formula r |y|^2 |V_f / tau - V_t|^2
    pv = sorted(int(b) for b in net.gen_bus if b != net.ref_bus)
    pq = sorted(set(range(net.n_bus)) - set(int(b) for b in net.gen_bus))
    n_pv, n_pq = len(pv), len(pq)
    vm = np.empty(net.n_bus)
    va = np.zeros(net.n_bus)
    vm[net.ref_bus] = u[0]
    vm[pv] = u[1:1 + n_pv]
    vm[pq] = x[n_pv + n_pq:]
    va[pv] = x[:n_pv]
    va[pq] = x[n_pv:n_pv + n_pq]
    V = vm * np.exp(1j * va)
    f, t = net.br_from, net.br_to
    y = 1.0 / (net.br_r + 1j * net.br_x)
    loss = np.sum(net.br_r * np.abs(y) ** 2 * np.abs(V[f] / net.br_tap - V[t]) ** 2)
    gen = u[1 + n_pv:].sum() + ev["c"][2 * net.n_branch + n_pq]  # PV outputs + slack output
    assert abs((gen - net.pd.sum()) - loss) < 1e-9 * max(1.0, loss)
    assert abs(ev["P"].sum() - loss) < 1e-9 * max(1.0, loss)
    assert loss > 0.0


def test_powerflow_lossless_network():
    net = with_branch_r(synth.workload("tiny30"), np.zeros(41))
    on = oracle.OracleNet(net)
    u = synth.flat_control(net)
    x, info = on.powerflow(u)
    assert info["rc"] == 0
    assert abs(on.eval(x, u)["P"].sum()) < 1e-10


@pytest.mark.slow
@pytest.mark.parametrize("name", ["large9200", "big20000"])
def test_workload_feasible(name):
    """Newton-Raphson from the flat start converges at the stored load level, |V| in [0.8, 1.2]."""
    net = synth.workload(name)
    on = oracle.OracleNet(net)
    u = synth.flat_control(net)
    x, info = on.powerflow(u)
    assert info["rc"] == 0 and info["res2"] < 1e-10
    n_pq = on.npq
    assert 0.8 <= x[-n_pq:].min() and x[-n_pq:].max() <= 1.2


# ---------------------------------------------------------------- gradient

def _fd_grad(on, u, x, al, cols, h=1e-6):
    out = []
    for j in cols:
        e = np.zeros(on.nu)
        e[j] = h
        vals = []
        for sgn in (1.0, -1.0):
            xx, info = on.powerflow(u + sgn * e, x0=x, tol=1e-12, max_it=30)
            assert info["rc"] == 0
            vals.append(on.reduced_gradient(xx, u + sgn * e, al)["F"])
        out.append((vals[0] - vals[1]) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("name,cols,h,tol", [("tiny30", None, 1e-6, 2e-7),
                                            ("medium1400", [0, 1, 7, 260, 300, 518], 1e-5, 1e-6)])
def test_gradient_central_fd(name, cols, h, tol):
    """Prop. 1 gradient equals central differences of F(x(u), u) with the power flow re-solved."""
    net, on, u, x = _solve(name)
    al = synth.al_inputs(net, seed=7)
    gr = on.reduced_gradient(x, u, al)
    cols = list(range(on.nu)) if cols is None else cols
    fd = _fd_grad(on, u, x, al, cols, h=h)
    scale = np.abs(gr["grad_u"]).max()
    assert np.abs(fd - gr["grad_u"][cols]).max() <= tol * scale
    assert np.allclose(gr["grad_s"], -(al["y"] * al["sigma_c"] + al["rho"] * al["sigma_c"] ** 2
                                        * (gr["c"] - al["s"])), rtol=1e-13, atol=0)


def test_gradient_and_hessian_special_case():
    """No slack cost, no penalties: lambda = 0, grad = sigma_f (2 a p + b), H = diag(2 sigma_f a) on p_pv."""
    base = synth.workload("tiny30")
    c2 = base.gen_c2.copy()
    c1 = base.gen_c1.copy()
    c2[0] = 0.0
    c1[0] = 0.0
    net = with_costs(base, c2, c1)
    net, on, u, x = _solve(net)
    al = synth.al_inputs(net, seed=3)
    al.update(y=np.zeros(on.m), rho=0.0)
    gr = on.reduced_gradient(x, u, al)
    assert np.abs(gr["lam"]).max() == 0.0
    npv = on.npv
    pv = sorted(int(b) for b in net.gen_bus if b != net.ref_bus)
    gidx = [int(np.where(net.gen_bus == b)[0][0]) for b in pv]
    expect = np.zeros(on.nu)
    expect[1 + npv:] = al["sigma_f"] * (2 * net.gen_c2[gidx] * u[1 + npv:] + net.gen_c1[gidx])
    assert np.allclose(gr["grad_u"], expect, rtol=1e-14, atol=1e-14)
    H = on.reduced_hessian(x, u, al)
    Hexp = np.zeros((on.nu, on.nu))
    Hexp[1 + npv:, 1 + npv:] = np.diag(2 * al["sigma_f"] * net.gen_c2[gidx])
    assert np.abs(H - Hexp).max() <= 1e-14 * np.abs(Hexp).max()


# ---------------------------------------------------------------- Hessian

def _mesh_net(nb=12, seed=5):
    """A small meshed net whose flows are far from the tiny workload's (second brute-force case)."""
    return synth.make_network(nb, 4, nb + 6, seed=seed, transformer_frac=0.3)


@pytest.mark.parametrize("which", ["tiny30", "mesh12"])
def test_hessian_matches_hyperdual_bruteforce(which):
    """Prop. 2 HVPs equal the dense l_uu + l_ux S + S^T l_xu + S^T l_xx S built from hyper-dual numbers."""
    net = synth.workload("tiny30") if which == "tiny30" else _mesh_net()
    net, on, u, x = _solve(net)
    al = synth.al_inputs(net, seed=9)
    H = on.reduced_hessian(x, u, al)
    bf = on.bruteforce(x, u, al)
    assert np.linalg.norm(H - bf["H"]) <= 1e-11 * np.linalg.norm(bf["H"])
    gr = on.reduced_gradient(x, u, al)
    assert np.abs(gr["grad_u"] - bf["grad_u"]).max() <= 1e-11 * np.abs(bf["grad_u"]).max()
    # custom second-order weights go through the same path
    om = np.linspace(0.5, 3.0, on.m)
    assert np.linalg.norm(on.reduced_hessian(x, u, al, omega=om) - on.bruteforce(x, u, al, omega=om)["H"]) \
        <= 1e-11 * np.linalg.norm(bf["H"])


def test_hessian_symmetry_and_fd():
    """Symmetry, and columns equal central differences of the reduced gradient (power flow re-solved)."""
    net, on, u, x = _solve("medium1400")
    al = synth.al_inputs(net, seed=4)
    cols = [0, 3, 261, 400, 518]
    Hc = on.reduced_hessian(x, u, al, cols=cols)
    H = on.reduced_hessian(x, u, al)
    assert np.linalg.norm(H - H.T) <= 1e-11 * np.linalg.norm(H)
    assert np.allclose(H[:, cols], Hc, rtol=0, atol=1e-12 * np.abs(H).max())
    h = 2e-6
    for k, j in enumerate(cols):
        e = np.zeros(on.nu)
        e[j] = h
        gs = []
        for sgn in (1.0, -1.0):
            xx, info = on.powerflow(u + sgn * e, x0=x, tol=1e-12, max_it=30)
            assert info["rc"] == 0
            gs.append(on.reduced_gradient(xx, u + sgn * e, al)["grad_u"])
        fd = (gs[0] - gs[1]) / (2 * h)
        assert np.abs(fd - Hc[:, k]).max() <= 2e-6 * np.abs(Hc[:, k]).max()


def test_hessian_gauss_newton_weights():
    """H(omega) - H(0) = J^T diag(omega) J with the reduced Jacobian J of the brute force."""
    net, on, u, x = _solve("tiny30")
    al = synth.al_inputs(net, seed=12)
    om = np.exp(np.linspace(-1.0, 1.0, on.m))
    H1 = on.reduced_hessian(x, u, al, omega=om)
    H0 = on.reduced_hessian(x, u, al, omega=np.zeros(on.m))
    J = on.bruteforce(x, u, al)["J"]
    ref = J.T @ (om[:, None] * J)
    assert np.linalg.norm((H1 - H0) - ref) <= 1e-11 * np.linalg.norm(ref)
    # the reduced Jacobian products agree with the brute-force J
    v = np.linspace(-1, 1, on.nu)
    w = np.linspace(1, -2, on.m)
    Jv, Jtw = on.jac_prod(x, u, v=v, w=w)
    assert np.abs(Jv - J @ v).max() <= 1e-11 * np.abs(J @ v).max()
    assert np.abs(Jtw - J.T @ w).max() <= 1e-11 * np.abs(J.T @ w).max()


def test_gauss_newton_part_is_psd():
    """With phi' = 0 (sigma_f = 0, y = 0, s = c) the reduced Hessian is rho J^T D^2 J >= 0."""
    net, on, u, x = _solve("tiny30")
    al = synth.al_inputs(net, seed=2)
    c = on.eval(x, u)["c"]
    al.update(sigma_f=0.0, y=np.zeros(on.m), s=c.copy())
    H = on.reduced_hessian(x, u, al)
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert ev.min() >= -1e-10 * ev.max()


# ---------------------------------------------------------------- symbolic

def _bus_graph(net):
    state = [i for i in range(net.n_bus) if i != net.ref_bus]
    adj = {i: set() for i in state}
    for a, b in zip(net.br_from.tolist(), net.br_to.tolist()):
        if a != net.ref_bus and b != net.ref_bus:
            adj[a].add(b)
            adj[b].add(a)
    gens = set(int(b) for b in net.gen_bus)
    w = {i: (1 if i in gens else 2) for i in state}
    return adj, w


@pytest.mark.parametrize("name", ["tiny30", "batchA500"])
def test_ordering_is_exact_minimum_degree(name):
    """Replay the elimination: each chosen bus has minimum weighted degree, smallest id on ties."""
    net = synth.workload(name)
    sym = oracle.OracleNet(net).symbolic()
    adj, w = _bus_graph(net)
    alive = set(adj)
    for p in sym["bus_order"].tolist():
        deg = {i: sum(w[j] for j in adj[i]) for i in alive}
        best = min(alive, key=lambda i: (deg[i], i))
        assert p == best
        alive.remove(p)
        nb = adj.pop(p)
        for q in nb:
            adj[q].discard(p)
            adj[q] |= nb - {q}
    assert not alive


@pytest.mark.parametrize("name", ["tiny30", "batchA500"])
def test_fill_pattern_path_theorem(name):
    """L_ij != 0 (i > j) iff a path joins i and j through vertices numbered below j (Rose-Tarjan)."""
    net = synth.workload(name)
    on = oracle.OracleNet(net)
    sym = on.symbolic()
    perm, rp, ci = sym["perm"], sym["rowptr"], sym["colidx"]
    nx = on.nx
    iperm = np.empty(nx, np.int64)
    iperm[perm] = np.arange(nx)
    # structural pattern of G_x: variables of adjacent (or equal) state buses are coupled
    pv = sorted(int(b) for b in net.gen_bus if b != net.ref_bus)
    pq = sorted(set(range(net.n_bus)) - set(int(b) for b in net.gen_bus))
    bvars = collections.defaultdict(list)
    for k, b in enumerate(pv):
        bvars[b].append(k)
    for k, b in enumerate(pq):
        bvars[b] += [len(pv) + k, len(pv) + len(pq) + k]
    adj, _ = _bus_graph(net)
    g = [set() for _ in range(nx)]
    for b in adj:
        for o in list(adj[b]) + [b]:
            for i in bvars[b]:
                for j in bvars[o]:
                    if i != j:
                        g[iperm[i]].add(int(iperm[j]))
    expect = [set() for _ in range(nx)]
    for j in range(nx):
        seen = {j}
        stack = [j]
        while stack:
            a = stack.pop()
            for b in g[a]:
                if b in seen:
                    continue
                seen.add(b)
                if b < j:
                    stack.append(b)
                else:
                    expect[b].add(j)
    for i in range(nx):
        row = ci[rp[i]:rp[i + 1]].tolist()
        assert row == sorted(row) and i in row
        assert set(c for c in row if c < i) == expect[i]
        assert set(c for c in row if c > i) == {k for k in range(i + 1, nx) if i in expect[k]}


def test_level_sets_definition():
    net = synth.workload("medium1400")
    on = oracle.OracleNet(net)
    s = on.symbolic()
    rp, ci, lf, lb = s["rowptr"], s["colidx"], s["lev_f"], s["lev_b"]
    assert sorted(s["perm"].tolist()) == list(range(on.nx))
    for i in range(on.nx):
        row = ci[rp[i]:rp[i + 1]]
        lo, hi = row[row < i], row[row > i]
        assert lf[i] == (lf[lo].max() + 1 if lo.size else 0)
        assert lb[i] == (lb[hi].max() + 1 if hi.size else 0)
