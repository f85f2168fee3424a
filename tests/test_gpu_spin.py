"""Two spin blocks on the GPU (float64 path) against the oracle.

A walker with N_up spin-up and N_dn spin-down orbitals and a trial whose
spin-down orbitals are not among the spin-up ones (Theorem 1.1: the overlap
is the product over spins).  Walkers, weights, overlaps and energies agree
with the oracle to 1e-10 relative at every step over 50 steps (population
control off), and with the comb on the parents and walkers agree too.
"""
import numpy as np
import pytest

import workloads
from oracle import afqmc, scf
from test_gpu_parity import TOL, compare_state, pkg  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def spin_pair(pkg, M, nup, ndn, G, W, ham_seed, lscale=1.0, **kw):
    h1, L, _ = workloads.hamiltonian(M, G, ham_seed, l_scale=workloads.l_amplitude(M, G))
    L = L * lscale
    C, _, conv, _ = scf.rhf(h1, L, nup)
    rng = np.random.default_rng(ham_seed)
    # spin-down orbitals: a rotation of the RHF orbitals mixed with virtuals
    Cf = np.linalg.eigh(h1)[1]
    Vd = np.linalg.qr(Cf[:, :ndn] + 0.3 * rng.standard_normal((M, ndn)))[0]
    op = dict(dt=0.005, seed=ham_seed % 97 + 1, qr_period=kw.pop("qr_period", 5),
              energy_period=kw.pop("energy_period", 1), taylor_order=6,
              pc_period=kw.pop("pc_period", 0), mode=kw.pop("mode", "phaseless"))
    orc = afqmc.Oracle(h1, L, C, W, afqmc.Params(**op), trial_dn=Vd)
    gp = dict(op)
    gp["mode"] = pkg.AFQMC_FREE if op["mode"] == "free" else pkg.AFQMC_PHASELESS
    p = pkg.default_params(M, nup, G, W, Ndn=ndn, **gp)
    run = pkg.AfqmcRun(h1, L, (C, Vd), p)
    return orc, run


def test_two_spin_blocks_fifty_steps_match_oracle(pkg):
    """12 orbitals, 3 spin-up and 2 spin-down electrons, 48 vectors, 32
    walkers, QR every 5 steps, energies every step: 50 steps at 1e-10."""
    orc, run = spin_pair(pkg, 12, 3, 2, 48, 32, 1000)
    info = run.info()
    assert abs(info.E_T - orc.setup.E_T) < 1e-12 * abs(orc.setup.E_T)
    assert abs(info.H0p - orc.setup.H0p) < 1e-11 * abs(orc.setup.H0p)
    el = run.local_energies()
    eo = orc.local_energies()
    assert np.max(np.abs(el - eo) / np.abs(eo)) < TOL
    for _ in range(50):
        run.propagate(1)
        orc.step()
        assert compare_state(run, orc) > 0
    e_gpu = run.energy_log()[:, 1]
    e_orc = np.array([r[1] / r[2] for r in orc.records])
    assert np.max(np.abs(e_gpu - e_orc) / np.abs(e_orc)) < TOL


@pytest.mark.parametrize("nup,ndn", [(5, 3), (2, 6), (1, 1)])
def test_two_spin_blocks_ragged_with_comb(pkg, nup, ndn):
    """M=20, odd vector and walker counts, QR every 3 steps, the comb every 4
    steps: identical parents, walkers and energies."""
    orc, run = spin_pair(pkg, 20, nup, ndn, 33, 17, 2000 + nup, qr_period=3, pc_period=4,
                         energy_period=2)
    for _ in range(12):
        run.propagate(1)
        orc.step()
        compare_state(run, orc)
    e_gpu = run.energy_log()[:, 1]
    e_orc = np.array([r[1] / r[2] for r in orc.records])
    assert np.max(np.abs(e_gpu - e_orc) / np.abs(e_orc)) < TOL


def test_two_spin_blocks_free_projection(pkg):
    """Free projection with two blocks: complex weights (Eq. weight_update)."""
    orc, run = spin_pair(pkg, 12, 4, 2, 24, 16, 3000, mode="free", lscale=0.5)
    for _ in range(10):
        run.propagate(1)
        orc.step()
    phi, wt, _ = run.get_walkers()
    assert np.max(np.abs(wt - orc.weight) / np.abs(orc.weight)) < TOL
    W = phi.shape[0]
    d = np.linalg.norm((phi - orc.phi).reshape(W, -1), axis=1)
    assert np.max(d / np.linalg.norm(orc.phi.reshape(W, -1), axis=1)) < TOL


def test_identical_blocks_reproduce_the_closed_shell_walk(pkg):
    """A two-block run with the spin-down trial equal to the spin-up one
    (N_dn = N_up) walks like the closed-shell run on the same fields."""
    w = workloads.config("c0")
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    kw = dict(dt=w.dt, seed=w.seed, qr_period=5, energy_period=1)
    a = pkg.AfqmcRun(h1, L, C, pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, **kw))
    b = pkg.AfqmcRun(h1, L, (C, C), pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, Ndn=w.N,
                                                       **kw))
    a.propagate(20)
    b.propagate(20)
    pa, wa, la = a.get_walkers()
    pb, wb, lb = b.get_walkers()
    alive = np.nonzero(wa != 0)[0]
    assert np.array_equal(np.nonzero(wb != 0)[0], alive) and alive.size > 0
    assert np.max(np.abs(wb[alive] - wa[alive]) / np.abs(wa[alive])) < 1e-10
    assert np.max(np.abs(pb[alive][:, :, :w.N] - pa[alive])) < 1e-10
    assert np.max(np.abs(pb[alive][:, :, w.N:] - pa[alive])) < 1e-10
    ea, eb = a.energy_log()[:, 1], b.energy_log()[:, 1]
    assert np.max(np.abs(eb - ea) / np.abs(ea)) < 1e-10
