"""use_graph = 1: the captured kernel sequence replayed for later calls of the same plan gives
the products of the direct launches (new inputs with the same bonds included), and a change of
bonds captures again."""

import numpy as np
import pytest
import torch

import ttgen
from oracle import tt as ott

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import paper_2410_19747_gb300 as pkg
    pkg.build()
    hd = pkg.Handle(0)
    yield hd
    hd.close()


def run(h, A, B, **kw):
    import paper_2410_19747_gb300 as pkg
    out, rep = pkg.ttm_multiply(h, [torch.from_numpy(c).cuda() for c in A], [torch.from_numpy(c).cuda() for c in B], **kw)
    torch.cuda.synchronize()
    return [c.cpu().numpy() for c in out], rep


def rel(O, P):
    return ott.diff_norm(O, P) / ott.norm(P)


@pytest.mark.parametrize("prec", ["fp64", "bf16_split"])
def test_graph_replay_matches_direct_launches(h, prec):
    kw = dict(eps=1e-14, chi_max=8, chi_out=8, prec=prec)
    A1, B1 = ttgen.rand_tt(10, 2, 8, 1000, canon="left"), ttgen.rand_tt(10, 2, 8, 1100, canon="left")
    A2, B2 = ttgen.rand_tt(10, 2, 8, 1001, canon="left"), ttgen.rand_tt(10, 2, 8, 1101, canon="left")
    D1, r1 = run(h, A1, B1, **kw)
    D2, _ = run(h, A2, B2, **kw)
    G1, g1 = run(h, A1, B1, use_graph=1, **kw)      # capture, then replay
    G1b, _ = run(h, A1, B1, use_graph=1, **kw)      # replay
    G2, g2 = run(h, A2, B2, use_graph=1, **kw)      # replay with new inputs of the same bonds
    for G, D in ((G1, D1), (G1b, D1), (G2, D2)):
        assert ott.bonds_of(G) == ott.bonds_of(D)
        assert rel(G, D) <= 1e-12
    assert g1["n_swaps"] == r1["n_swaps"] and g1["n_kernel_launches"] == r1["n_kernel_launches"]
    P2 = ott.dense(A2) * ott.dense(B2)   # chi_max = 8 truncates: within the reported bound
    assert np.linalg.norm(ott.dense(G2) - P2) <= g2["err_bound"] * (1 + 1e-9) + 1e-12 * np.linalg.norm(P2)
    # other bonds: a new capture
    A3, B3 = ttgen.rand_tt(10, 2, 6, 1002, canon="left"), ttgen.rand_tt(10, 2, 5, 1102, canon="left")
    D3, _ = run(h, A3, B3, **kw)
    G3, _ = run(h, A3, B3, use_graph=1, **kw)
    assert ott.bonds_of(G3) == ott.bonds_of(D3) and rel(G3, D3) <= 1e-12
