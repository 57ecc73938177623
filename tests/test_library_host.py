"""Host-side checks of libopf (no GPU): exported symbols, bit-exact symbolic
analysis against the oracle, and argument validation."""
import ctypes
import dataclasses

import numpy as np
import pytest

import oracle
import paper_2110_02590_b300 as P
from paper_2110_02590_b300 import synth
from tests.netutil import custom_network


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_02590_b300 import build
    build.build()


def test_library_exports_every_declared_symbol():
    names = P.exported_symbols()
    assert "opf_reduced_hessian" in names and "opf_powerflow" in names and len(names) >= 15
    so = ctypes.CDLL(P.LIB_PATH)
    for name in names:
        assert hasattr(so, name), name


KEYS = ("bus_order", "perm", "rowptr", "colidx", "lev_f", "lev_b")


@pytest.mark.parametrize("name,chords", [("tiny30", "local"), ("medium1400", "local"), ("batchA500", "local"),
                                         ("batchB2000", "local"), ("large9200", "local"),
                                         ("medium1400", "uniform")])
def test_symbolic_bit_exact_vs_oracle(name, chords):
    net = synth.workload(name, chords=chords)
    lib_sym = P.symbolic_analyze(net)
    orc_sym = oracle.OracleNet(net).symbolic()
    for k in KEYS:
        assert np.array_equal(lib_sym[k], orc_sym[k]), k
    assert lib_sym["nlev_f"] == lib_sym["lev_f"].max() + 1


def test_symbolic_parallel_branches_and_two_bus():
    # parallel branches 1-2 and a two-bus net (no PV bus)
    net = custom_network(4, [(0, 1, 0.01, 0.05, 0.01, 1.0), (1, 2, 0.01, 0.04, 0.0, 1.0),
                             (1, 2, 0.02, 0.06, 0.0, 1.0), (2, 3, 0.01, 0.05, 0.02, 0.98)],
                         gen_bus=[0, 3], pd=[0, 0.5, 0.4, 0.1], qd=[0, 0.1, 0.1, 0.0])
    for n in (net, custom_network(2, [(0, 1, 0.02, 0.08, 0.0, 1.0)], gen_bus=[0], pd=[0, 0.8], qd=[0, 0.3])):
        a = P.symbolic_analyze(n)
        b = oracle.OracleNet(n).symbolic()
        for k in KEYS:
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("mutate,msg", [
    (lambda n: dataclasses.replace(n, br_to=np.where(np.arange(n.n_branch) == 0, n.br_from, n.br_to)), "self-loop"),
    (lambda n: dataclasses.replace(n, br_r=np.zeros(n.n_branch), br_x=np.zeros(n.n_branch)), "r = x = 0"),
    (lambda n: dataclasses.replace(n, gen_bus=np.where(np.arange(n.n_gen) == 1, n.gen_bus[2], n.gen_bus)),
     "two generators"),
    (lambda n: dataclasses.replace(n, ref_bus=int(np.setdiff1d(np.arange(n.n_bus), n.gen_bus)[0])),
     "no generator"),
])
def test_invalid_networks_rejected(mutate, msg):
    net = mutate(synth.workload("tiny30"))
    with pytest.raises(P.OPFError) as ei:
        P.symbolic_analyze(net)
    assert ei.value.status == 1 and msg in str(ei.value)


def test_disconnected_bus_rejected():
    net = custom_network(3, [(0, 1, 0.01, 0.05, 0.0, 1.0), (0, 1, 0.02, 0.05, 0.0, 1.0)],
                         gen_bus=[0], pd=[0, 0.1, 0.1], qd=[0, 0, 0])
    with pytest.raises(P.OPFError) as ei:
        P.symbolic_analyze(net)
    assert "not connected" in str(ei.value)
