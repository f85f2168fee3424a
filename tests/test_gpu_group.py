"""Uneven systems advanced by one graph launch per block (afqmc_group_*):
each run is bit-identical to the same run stepped alone, whether the block is
captured as every run's own kernels or - mixed precision - with each of the
step's four tensor-core contractions of all runs as one grouped persistent
launch (tile widths timed on the runs' buffers), or switched between the two
by the group's timed choice."""
import numpy as np
import pytest

import workloads
from oracle import scf

pytestmark = pytest.mark.gpu

SYSTEMS = [
    workloads.Workload("a", M=12, N=3, nchol=48, nwalkers=32, seed=5, ham_seed=1000),
    workloads.Workload("b", M=24, N=3, nchol=120, nwalkers=64, seed=6, ham_seed=3001),
    workloads.Workload("c", M=40, N=5, nchol=200, nwalkers=16, seed=7, ham_seed=3002),
]


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_02242_gb300 as p

    return p


def make(pkg, w, prec):
    import torch

    h1, L, _ = w.hamiltonian()
    L = 0.3 * L  # milder vectors keep walkers alive through the run
    C, _, _, _ = scf.rhf(h1, L, w.N)
    p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed, qr_period=5,
                           energy_period=5, precision=prec, use_graph=1)
    return pkg.AfqmcRun(h1, L, C, p, stream=torch.cuda.Stream())


@pytest.mark.parametrize("prec,grouped", [(0, True), (2, True), (2, False), (1, True),
                                          (2, "auto")])
def test_group_matches_runs_stepped_alone(pkg, prec, grouped):
    alone = [make(pkg, w, prec) for w in SYSTEMS]
    for r in alone:
        r.propagate(20)
    grouped_runs = [make(pkg, w, prec) for w in SYSTEMS]
    g = pkg.AfqmcGroup(grouped_runs)
    g.set_grouped(grouped)
    g.propagate(10)
    on, bn = g.tiles()
    # the grouped contractions serve mixed runs only (in the timed choice the
    # first blocks use them)
    assert on == (bool(grouped) and prec != 0)
    if on:
        assert bn[0] in (64, 128, 256) and bn[1] in (128, 256) and bn[2] in (160, 256) and bn[3] == bn[2]
    g.propagate(10)
    g.synchronize()
    for a, b in zip(alone, grouped_runs):
        pa, wa, la = a.get_walkers()
        pb, wb, lb = b.get_walkers()
        assert np.array_equal(pa, pb) and np.array_equal(wa, wb) and np.array_equal(la, lb)
        assert np.array_equal(a.energy_log(), b.energy_log(), equal_nan=True)
        assert np.isfinite(a.energy_log()[:, 1]).all()
        assert b.info().step == 20
    g.close()


def test_group_rejects_mismatched_blocks(pkg):
    import torch

    w = SYSTEMS[0]
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    p1 = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, qr_period=5, energy_period=5,
                            use_graph=1)
    p2 = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, qr_period=4, energy_period=4,
                            use_graph=1)
    r1 = pkg.AfqmcRun(h1, L, C, p1, stream=torch.cuda.Stream())
    r2 = pkg.AfqmcRun(h1, L, C, p2, stream=torch.cuda.Stream())
    with pytest.raises(pkg.AfqmcError, match="EINVAL"):
        pkg.AfqmcGroup([r1, r2])
