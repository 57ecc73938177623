"""Pins of the oracle's reduced Jacobian and gradient-based scaling (Sec. III-B, Sec. IV-A "Scaling"; no GPU).

The scaling rule is pinned on hand-computed cases; the explicit reduced
Jacobian and the cost gradient it scales are pinned against central finite
differences of independently re-solved power flows.
"""
import numpy as np
import pytest

import oracle
from oracle import scaling
from paper_2110_02590_b300 import synth


def _solve(name):
    net = synth.workload(name)
    on = oracle.OracleNet(net)
    u = synth.flat_control(net)
    x, info = on.powerflow(u, tol=1e-12, max_it=30)
    assert info["rc"] == 0
    return net, on, u, x


def test_scaling_rule_by_hand():
    """Rows within g_max keep 1; larger rows get g_max / norm; tiny scales are floored at s_min;
    an all-zero row keeps 1; signs do not matter."""
    J = np.array([[250.0, -3.0],
                  [0.0, 0.0],
                  [-0.5, 99.9],
                  [1e12, 1.0],
                  [-100.0, 100.0],
                  [0.0, -400.0]])
    sig, sf = scaling.gradient_scaling(J, np.array([-400.0, 2.0]))
    assert sig.tolist() == [0.4, 1.0, 1.0, 1e-8, 1.0, 0.25]
    assert sf == 0.25
    sig2, sf2 = scaling.gradient_scaling(J, np.array([0.0, 0.0]), g_max=10.0, s_min=1e-3)
    assert sig2.tolist() == [0.04, 1.0, 10.0 / 99.9, 1e-3, 0.1, 0.025]
    assert sf2 == 1.0
    # with the caller's own scales the rule applies to the rows as written, p_i dc_i/du
    prior = np.array([2.0, 5.0, 0.1, 1e-9, 0.5, 0.25])
    sig3, _ = scaling.gradient_scaling(J, np.array([1.0]), prior=prior)
    assert sig3[[0, 1, 2, 4, 5]].tolist() == [2.0 * (100.0 / 500.0), 5.0, 0.1, 0.5, 0.25]
    assert sig3[3] == pytest.approx(1e-10, rel=1e-15)  # 1e-9 * 1e12 = 1000 > 100: scaled by 0.1


def test_explicit_jacobian_matches_finite_differences():
    """J e_j = d c(x(u), u) / du_j by central differences of re-solved power flows (tiny30, all
    controls): the |S|^2 rows, the PQ voltages and the generator P/Q rows."""
    net, on, u, x = _solve("tiny30")
    J = scaling.explicit_jacobian(on, x, u)
    h = 1e-6
    for j in range(on.nu):
        e = np.zeros(on.nu)
        e[j] = h
        xp, ip = on.powerflow(u + e, x0=x, tol=1e-12, max_it=30)
        xm, im = on.powerflow(u - e, x0=x, tol=1e-12, max_it=30)
        assert ip["rc"] == 0 and im["rc"] == 0
        fd = (on.eval(xp, u + e)["c"] - on.eval(xm, u - e)["c"]) / (2 * h)
        assert np.abs(fd - J[:, j]).max() <= 1e-6 * max(1.0, np.abs(J[:, j]).max())


def test_cost_gradient_matches_finite_differences():
    """The reduced gradient of the generation cost (the AL functional with sigma_f = 1 and no
    multiplier or penalty term) equals central differences of the cost through re-solved power
    flows."""
    net, on, u, x = _solve("tiny30")
    g = scaling.cost_gradient(on, x, u)
    z = np.zeros(on.m)
    al = dict(sigma_f=1.0, rho=0.0, sigma_c=z, y=z, s=z)
    h = 1e-6
    for j in range(on.nu):
        e = np.zeros(on.nu)
        e[j] = h
        xp, _ = on.powerflow(u + e, x0=x, tol=1e-12, max_it=30)
        xm, _ = on.powerflow(u - e, x0=x, tol=1e-12, max_it=30)
        fp = on.reduced_gradient(xp, u + e, al)["F"]
        fm = on.reduced_gradient(xm, u - e, al)["F"]
        assert abs((fp - fm) / (2 * h) - g[j]) <= 1e-6 * max(1.0, np.abs(g).max())


@pytest.mark.parametrize("g_max", [1.0, 100.0])
def test_scaled_rows_within_g_max(g_max):
    """After scaling every row's largest reduced derivative is at most g_max, and a row that
    needed no scaling keeps its size (medium1400)."""
    net, on, u, x = _solve("medium1400")
    cols = list(range(0, on.nu, 7))
    J = scaling.explicit_jacobian(on, x, u, cols=cols)
    sig, sf = scaling.gradient_scaling(J, scaling.cost_gradient(on, x, u)[cols], g_max=g_max)
    rows = np.abs(J).max(axis=1)
    assert np.all(sig * rows <= g_max * (1 + 1e-15))
    assert np.all(sig[rows <= g_max] == 1.0)
    assert np.all((sig > 0) & (sig <= 1))
    assert 0 < sf <= 1
