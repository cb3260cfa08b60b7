"""The purification chain captured in one CUDA graph (no host
synchronisation inside), against its eager run and the CPU oracle."""
import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import bsm, chain
    return bsm, chain, torch


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_graph_replay_equals_eager_and_oracle(mods, oracle, prec):
    bsm, chain, torch = mods
    w = I.purification_start(nb=200)
    X0 = bsm.Matrix.from_host(w["X0"])
    g = chain.McWeenyGraph(X0, 10, w["eps"], prec=prec)
    eager = g.result.data_host().copy()
    pat = g.result.pattern()
    # wipe the intermediate values, then recompute everything from the graph
    for h in g.X[1:] + g.X2 + g.X3:
        h.set_data(np.zeros(h.info().data_len))
    g.replay()
    torch.cuda.synchronize()
    assert g.status() == 0
    np.testing.assert_array_equal(g.result.data_host(), eager)
    for a, b in zip(g.result.pattern(), pat):
        np.testing.assert_array_equal(a, b)
    if prec == "fp64":
        ref = oracle.mcweeny(w["X0"], 10, w["eps"])[-1]
        np.testing.assert_array_equal(pat[0], ref.row_ptr)
        np.testing.assert_array_equal(pat[1], ref.col_idx)
        assert rel_fro(eager, ref.data) <= 1e-12


def test_ozaki_chain_graph_replay(mods, oracle):
    """The chain on mixed 5 / 13 blocks (tensor-core items on the Ozaki path:
    line exponents, slices and the numeric kernel all inside the graph):
    replay equals the eager pass bit for bit, and both follow the oracle."""
    bsm, chain, torch = mods
    w = I.purification_start(nb=120, occ=0.05, sizes=(5, 13), probs=(0.6, 0.4))
    X0 = bsm.Matrix.from_host(w["X0"])
    g = chain.McWeenyGraph(X0, 4, w["eps"], prec="ozaki")
    eager = g.result.data_host().copy()
    for h in g.X[1:] + g.X2 + g.X3:
        h.set_data(np.zeros(h.info().data_len))
    g.replay()
    torch.cuda.synchronize()
    assert g.status() == 0
    np.testing.assert_array_equal(g.result.data_host(), eager)
    ref = oracle.mcweeny(w["X0"], 4, w["eps"])[-1]
    pat = g.result.pattern()
    np.testing.assert_array_equal(pat[0], ref.row_ptr)
    np.testing.assert_array_equal(pat[1], ref.col_idx)
    assert rel_fro(eager, ref.data) <= 1e-12


def test_graph_replay_flags_changed_patterns(mods):
    """New X0 values that change the filtered patterns: the replay must not
    write past any handle's storage; the status words report it."""
    bsm, chain, torch = mods
    w = I.purification_start(nb=150)
    X0 = bsm.Matrix.from_host(w["X0"])
    g = chain.McWeenyGraph(X0, 4, w["eps"])
    before = g.result.data_host().copy()
    # same pattern, all values zero: every product is filtered away, so the
    # recomputed sizes differ from the eager pass
    X0.set_data(np.zeros_like(w["X0"].data))
    g.replay()
    torch.cuda.synchronize()
    assert g.status() != 0
    # restore and replay: back to the eager result
    X0.set_data(w["X0"].data)
    g.replay()
    torch.cuda.synchronize()
    assert g.status() == 0
    np.testing.assert_array_equal(g.result.data_host(), before)
