"""The state machine of Fig. 4, traced on the GPU.

The statistics instances of the pass count every state transition they make
-- ACC->RSVD (Alg. 1 line 11), ACC->MCHD (line 14), RSVD->MCHD (line 15),
RSVD->ACC (line 18) -- and check the two the reservation holder makes on the
word its atomic returns (the field must be RSVD).  After a pass:
  * no illegal transition happened;
  * every reservation ended in a commit or a release (ACC->RSVD = RSVD->MCHD
    + RSVD->ACC), so the census of the state array shows no RSVD vertex;
  * claims, commits and matches agree with the checker's pair count, and the
    census shows exactly 2 x pairs MCHD vertices (MCHD is absorbing).
"""
import numpy as np
import pytest
import torch

import graphgen as gg
from tests.conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def skp():
    import paper_2507_04420_gb300 as m
    torch.cuda.set_device(0)
    return m


GRAPHS = {
    "rmat14": lambda: gg.rmat(14, 16, seed=4),
    "uniform": lambda: gg.uniform(20000, 120000, seed=5),
    "star": lambda: gg.star(20000),
    "k64_64": lambda: gg.complete_bipartite(64, 64),
    "grid": lambda: gg.grid(100, 120),
}


def _check_trace(st, census, n, pairs):
    tr = st["transitions"]
    assert st["illegal_transitions"] == 0
    assert tr[0] == tr[2] + tr[3]                 # every reservation ended
    assert tr[1] == tr[2] == st["matches"] == pairs
    assert census == {"acc": n - 2 * pairs, "rsvd": 0, "mchd": 2 * pairs, "other": 0}


@pytest.mark.parametrize("bits", [2, 8, 32])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_csr_pass_transitions(skp, name, bits):
    g = GRAPHS[name]()
    d = g.to("cuda")
    with skp.Graph(d.offsets, d.nbrs) as h:
        for sym in (0, 1):
            mate = h.skipper(status_bits=bits, stats=1, grain=256, symmetric=sym)
            v = h.validate(mate)
            assert v.flags == 0
            _check_trace(h.stats(), h.state_census(), g.n, v.n_pairs)


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_edge_list_pass_transitions(skp, bits):
    g = gg.rmat(13, 16, seed=6)
    s, t = gg.edge_list(g, "shuffle", seed=6)
    with skp.EdgeList(g.n, s.cuda(), t.cuda()) as h:
        mate = h.skipper(status_bits=bits, stats=1, grain=256)
        v = h.validate(mate)
        assert v.flags == 0
        _check_trace(h.stats(), h.state_census(), g.n, v.n_pairs)


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_poisoned_vertex_stays_reserved_and_nothing_else_does(skp, bits):
    """A vertex left RSVD by no thread (fault injection) is the only RSVD one
    after the pass times out; every reservation a thread made still ended."""
    g = gg.rmat(12, 8, seed=6)
    hub = int(torch.argmax(g.offsets[1:] - g.offsets[:-1]))
    d = g.to("cuda")
    with skp.Graph(d.offsets, d.nbrs) as h:
        with pytest.raises(skp.SkipperError):
            h.skipper(status_bits=bits, stats=1, poison_vertex=hub + 1, spin_limit=2000)
        st = h.stats()
        tr = st["transitions"]
        assert st["illegal_transitions"] == 0 and tr[0] == tr[2] + tr[3]
        c = h.state_census()
        assert c["rsvd"] == 1 and c["other"] == 0 and c["mchd"] == 2 * tr[2]
