"""CUDA-graph replay of whole step blocks gives bit-identical walks."""
import numpy as np
import pytest

import workloads
from oracle import scf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_02242_gb300 as p

    return p


@pytest.mark.parametrize("prec,pc", [(0, 0), (0, 4), (2, 0)])
def test_graph_replay_is_bit_identical(pkg, prec, pc):
    w = workloads.config("c0")
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    runs = []
    for g in (0, 1):
        p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed,
                               qr_period=5, energy_period=2, pc_period=pc, precision=prec,
                               use_graph=g)
        r = pkg.AfqmcRun(h1, L, C, p)
        # 3 steps unaligned, then whole blocks, then a tail
        for n in (3, 17, 20, 4):
            r.propagate(n)
        runs.append(r)
    a, b = runs
    pa, wa, la = a.get_walkers()
    pb, wb, lb = b.get_walkers()
    assert np.array_equal(pa, pb) and np.array_equal(wa, wb) and np.array_equal(la, lb)
    assert np.array_equal(a.energy_log(), b.energy_log())
    assert a.info().step == b.info().step == 44
