"""The sharded population's comb through the C ABI (afqmc_export_weights,
afqmc_comb_plan, afqmc_pack_walkers, afqmc_unpack_walkers,
afqmc_energy_sums) on one GPU: a population held by one state and combed by
the host driver equals the state's own comb (pc_period) bit for bit --
walkers, weights, overlaps and energies -- on the float64 and BF16 paths.
The multi-rank exchange around these calls is tested on the CPU with gloo
(tests/test_sharded.py)."""
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


@pytest.mark.parametrize("prec", [0, 2])
def test_driver_comb_equals_the_states_own_comb(pkg, prec):
    from paper_1711_02242_gb300.dist import ShardedPopulation, StateShard

    w = workloads.config("c0")
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    kw = dict(dt=w.dt, seed=5, qr_period=5, precision=prec)
    own = pkg.AfqmcRun(h1, L, C, pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, pc_period=5,
                                                    energy_period=2, **kw))
    drv = pkg.AfqmcRun(h1, L, C, pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, pc_period=0,
                                                    energy_period=0, **kw))
    pop = ShardedPopulation(StateShard(drv), pc_period=5, energy_period=2).run(30)
    own.propagate(30)
    pa, wa, la = own.get_walkers()
    pb, wb, lb = drv.get_walkers()
    assert np.array_equal(pa, pb) and np.array_equal(wa, wb) and np.array_equal(la, lb)
    log = own.energy_log()
    assert [int(r[0]) for r in log] == [s for s, _, _ in pop.records]
    assert np.array_equal(log[:, 1], np.array([e for _, e, _ in pop.records]))
    assert np.array_equal(log[:, 2], np.array([d for _, _, d in pop.records]))
    # the combs copied walkers
    assert any(len(set(p.tolist())) < len(p) for _, p in pop.parents)
    assert own.info().status == 0 and drv.info().status == 0


def test_population_calls_refuse_unsupported_states(pkg):
    import ctypes

    w = workloads.config("c0")
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    run = pkg.AfqmcRun(h1, L, C, pkg.default_params(w.M, w.N, w.nchol, 4, mode=pkg.AFQMC_FREE))
    rows = ctypes.c_void_p(0)
    assert pkg.lib().afqmc_pack_walkers(run.s, None, 0, rows) == -7  # EUNSUPPORTED
    ph = pkg.AfqmcRun(h1, L, C, pkg.default_params(w.M, w.N, w.nchol, 4))
    assert pkg.lib().afqmc_unpack_walkers(ph.s, None, 0, None) == -6  # ESTATE: no plan yet
