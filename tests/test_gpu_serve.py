"""Serving loop: runs admitted by footprint from one device pool, advanced
together tick by tick; each result equals the same run stepped alone."""
import numpy as np
import pytest

import workloads

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


def requests(n=5):
    from paper_1711_02242_gb300.serve import Request

    out = []
    sizes = [(12, 3, 48, 32), (30, 3, 150, 64), (20, 2, 100, 128), (40, 5, 200, 48), (16, 2, 80, 16)]
    for i, (M, N, G, W) in enumerate(sizes[:n]):
        h1, L, _ = workloads.hamiltonian(M, G, 4000 + i)
        L = 0.3 * L  # milder vectors keep walkers alive through the run
        trial = np.linalg.eigh(h1)[1][:, :N]
        out.append(Request(rid=i, arrival=0.02 * i, h1=h1, L=L, trial=trial, nwalkers=W,
                           nsteps=40, seed=77 + i, energy_period=10))
    return out


@pytest.mark.parametrize("prec", [0, 2])
def test_results_alone_equal_results_in_the_mix(pkg, prec):
    from paper_1711_02242_gb300.serve import Server

    reqs = requests()
    probe = Server(1 << 20, precision=prec)
    sizes = [probe.footprint(r) for r in reqs]
    # a pool that holds about two runs at a time, so admission has to wait
    srv = Server(int(2.2 * max(sizes)), precision=prec, chunk_steps=10)
    done = srv.run(reqs, realtime=True)
    assert sorted(r.rid for r in done) == list(range(len(reqs)))
    assert all(r.admit >= r.arrival for r in done)
    # the same requests one at a time
    for r in requests():
        alone = Server(int(1.1 * srv.footprint(r)), precision=prec).run([r], realtime=False)[0]
        mixed = next(d for d in done if d.rid == r.rid)
        assert np.array_equal(alone.energies, mixed.energies, equal_nan=True)
        assert np.isfinite(alone.energies[:, 1]).all()
        assert alone.energies.shape[0] == 4


def test_pool_first_fit_reuses_memory(pkg):
    from paper_1711_02242_gb300.serve import DevicePool

    p = DevicePool(1 << 20)
    a = p.alloc(1000)
    b = p.alloc(5000)
    c = p.alloc(300)
    assert a[0] % 256 == 0 and b[0] % 256 == 0 and c[0] % 256 == 0
    p.release(*b)
    d = p.alloc(4000)
    assert d[0] == b[0]  # first fit reuses the hole
    p.release(*a)
    p.release(*c)
    p.release(*d)
    assert p.free_bytes() == p.size and len(p.free) == 1
    assert p.alloc(p.size + 1) is None
