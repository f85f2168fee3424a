"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 path: walker matrices, weights, overlaps and energies agree with the
oracle to 1e-10 relative at every step (population control off); the
generator's integers are bit-exact.  Inputs are the seeded synthetic
Hamiltonians of ``workloads`` and the oracle's RHF trial.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import afqmc, philox, scf

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_02242_gb300 as p

    return p


def rel_phi(a, b):
    W = a.shape[0]
    d = np.linalg.norm((a - b).reshape(W, -1), axis=1)
    n = np.linalg.norm(b.reshape(W, -1), axis=1)
    return np.max(d / n)


def make_pair(pkg, w: workloads.Workload, nwalkers=None, H0=0.0, mode="phaseless", lscale=1.0,
              **kw):
    h1, L, _ = w.hamiltonian()
    L = L * lscale
    C, _, conv, _ = scf.rhf(h1, L, w.N)
    W = nwalkers or w.nwalkers
    op = dict(dt=w.dt, seed=w.seed, qr_period=w.qr_period, energy_period=kw.pop("energy_period", 1),
              taylor_order=w.taylor_order, pc_period=kw.pop("pc_period", 0), mode=mode)
    op.update(kw)
    orc = afqmc.Oracle(h1, L, C, W, afqmc.Params(**op), H0=H0)
    gp = dict(op)
    gp["mode"] = pkg.AFQMC_FREE if mode == "free" else pkg.AFQMC_PHASELESS
    p = pkg.default_params(w.M, w.N, w.nchol, W, H0=H0, **gp)
    run = pkg.AfqmcRun(h1, L, C, p)
    return orc, run


def compare_state(run, orc, tol=TOL):
    phi, wt, lo = run.get_walkers()
    alive = np.nonzero(orc.weight != 0)[0]
    assert np.array_equal(np.nonzero(wt != 0)[0], alive), "different walkers alive"
    if alive.size:
        assert rel_phi(phi[alive], orc.phi[alive]) < tol
        ow = orc.weight[alive]
        assert np.max(np.abs(wt[alive] - ow) / np.abs(ow)) < tol
        # log <Psi_T|Psi> = 2 log det S: real part and phase carry the same
        # absolute rounding error, ~ eps * cond(S), so both are bounded
        # relative to 1 + |log det|
        scale = 1 + np.abs(orc.logdet[alive].real)
        assert np.max(np.abs(lo[alive].real - orc.logdet[alive].real) / scale) < tol
        dph = np.angle(np.exp(1j * (lo[alive].imag - orc.logdet[alive].imag)))
        assert np.max(np.abs(dph) / scale) < tol
    return alive.size


# ------------------------------------------------------------- generator ----
def test_philox_words_bit_exact(pkg):
    import torch

    rng = np.random.default_rng(0)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = 0x0123456789ABCDEF
    d = torch.from_numpy(ctr.view(np.int32)).cuda()
    out = pkg.afqmc_philox4x32_10(key, d).cpu().numpy().view(np.uint32)
    ref = philox.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], key & 0xFFFFFFFF, key >> 32)
    for c in range(4):
        assert np.array_equal(out[:, c], ref[c].astype(np.uint32))


@pytest.mark.parametrize("nchol", [1, 48, 501])
def test_gaussian_fields_match_oracle(pkg, nchol):
    got = pkg.afqmc_gaussian_fields(7, 123456, 5, 64, nchol).cpu().numpy()
    ref = philox.gaussian_fields(7, 123456, np.arange(5, 69), nchol)
    assert np.max(np.abs(got - ref)) < 1e-13


# ------------------------------------------------ step-by-step FP64 parity --
def test_c0_fifty_steps_match_oracle(pkg):
    """The 12-orbital workload: 32 walkers, 50 steps, QR every 5 steps,
    energy every step; everything within 1e-10 relative at every step."""
    w = workloads.config("c0")
    orc, run = make_pair(pkg, w)
    info = run.info()
    assert abs(info.E_T - orc.setup.E_T) < 1e-12 * abs(orc.setup.E_T)
    assert abs(info.H0p - orc.setup.H0p) < 1e-11 * abs(orc.setup.H0p)
    for _ in range(50):
        run.propagate(1)
        orc.step()
        compare_state(run, orc)
    log = run.energy_log()
    e_orc = np.array([r[1] / r[2] for r in orc.records])
    assert log.shape[0] == 50
    assert np.array_equal(log[:, 0], np.arange(1, 51))
    assert np.max(np.abs(log[:, 1] - e_orc) / np.abs(e_orc)) < TOL
    assert np.max(np.abs(log[:, 2] - np.array([r[2] for r in orc.records]))
                  / np.array([r[2] for r in orc.records])) < TOL


def test_local_energies_random_walkers(pkg):
    """Eqs. localenergy2/3 for random complex walkers (not near the trial)."""
    w = workloads.Workload("rand", M=37, N=5, nchol=61, nwalkers=7, seed=3, ham_seed=77)
    orc, run = make_pair(pkg, w)
    rng = np.random.default_rng(1)
    phi = rng.standard_normal((7, 37, 5)) + 1j * rng.standard_normal((7, 37, 5))
    wt = np.ones(7)
    run.set_walkers(phi, wt)
    ld, th = afqmc.overlap(orc.setup, phi)
    e_ref = afqmc.local_energy(orc.setup, th)
    e = run.local_energies()
    assert np.max(np.abs(e - e_ref) / np.abs(e_ref)) < TOL
    _, _, lo = run.get_walkers()
    assert np.max(np.abs(lo.real - ld.real)) < 1e-10 * np.max(np.abs(ld.real))


@pytest.mark.parametrize("shape", [
    dict(M=7, N=1, nchol=5, nwalkers=1),      # single walker, one electron
    dict(M=6, N=6, nchol=3, nwalkers=3),      # every orbital occupied
    dict(M=70, N=9, nchol=131, nwalkers=5),   # ragged tiles, odd nchol
    dict(M=65, N=33, nchol=40, nwalkers=2),   # N above one warp
])
def test_ragged_shapes_match_oracle(pkg, shape):
    w = workloads.Workload("edge", seed=11, ham_seed=500 + shape["M"], qr_period=2, **shape)
    orc, run = make_pair(pkg, w)
    for _ in range(6):
        run.propagate(1)
        orc.step()
        compare_state(run, orc)


def test_free_projection_matches_oracle(pkg):
    """Eq. weight_update with complex weights (no force bias, no caps)."""
    w = workloads.config("c0")
    orc, run = make_pair(pkg, w, mode="free", nwalkers=16, energy_period=2)
    for _ in range(10):
        run.propagate(1)
        orc.step()
        compare_state(run, orc)
    log = run.energy_log()
    e_orc = np.array([(r[1] / r[2]).real for r in orc.records])
    assert np.max(np.abs(log[:, 1] - e_orc) / np.abs(e_orc)) < TOL


def test_population_control_matches_oracle(pkg):
    """Comb every 5 steps: identical parents when the weights agree."""
    w = workloads.config("c0")
    orc, run = make_pair(pkg, w, pc_period=5, energy_period=5)
    for _ in range(20):
        run.propagate(1)
        orc.step()
        compare_state(run, orc)


def test_dead_walkers_stay_frozen(pkg):
    w = workloads.config("c0")
    orc, run = make_pair(pkg, w, nwalkers=8)
    run.propagate(2)
    orc.run(2)
    phi, wt, _ = run.get_walkers()
    wt = wt.copy()
    wt[[1, 4]] = 0.0
    run.set_walkers(phi, wt)
    orc.weight[[1, 4]] = 0.0
    before = run.get_walkers()[0][[1, 4]]
    run.propagate(3)
    orc.run(3)
    after, wt2, _ = run.get_walkers()
    assert np.array_equal(after[[1, 4]], before)
    assert np.all(wt2[[1, 4]] == 0)
    compare_state(run, orc)


def test_c1_two_steps_full_population(pkg):
    """M=100, N=10, 500 Cholesky vectors, 1024 walkers: two steps, every walker."""
    w = workloads.config("c1")
    orc, run = make_pair(pkg, w, energy_period=2)
    run.propagate(2)
    orc.run(2)
    compare_state(run, orc)
    e = run.energy_log()[-1, 1]
    e_ref = orc.records[-1][1] / orc.records[-1][2]
    assert abs(e - e_ref) < TOL * abs(e_ref)


def test_c2_full_size_sampled_walkers(pkg):
    """M=300, N=25, 1800 vectors, 512 walkers on the GPU, as launched by the
    benchmark; the oracle follows 4 sampled walkers (the others carry zero
    weight in the oracle so it skips them) for one step."""
    w = workloads.config("c2")
    h1, L, _ = w.hamiltonian()
    # any orthonormal determinant is a valid trial; both sides get the same
    # one (the core-Hamiltonian orbitals: SCF does not converge at this scale)
    C = np.linalg.eigh(h1)[1][:, :w.N]
    sample = np.array([0, 97, 300, 511])
    p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed,
                           qr_period=w.qr_period, energy_period=1)
    run = pkg.AfqmcRun(h1, L, C, p)
    orc = afqmc.Oracle(h1, L, C, w.nwalkers, afqmc.Params(dt=w.dt, seed=w.seed, energy_period=0))
    mask = np.zeros(w.nwalkers, bool)
    mask[sample] = True
    orc.weight[~mask] = 0.0
    run.propagate(1)
    orc.step()
    phi, wt, lo = run.get_walkers()
    assert rel_phi(phi[sample], orc.phi[sample]) < TOL
    ok = orc.weight[sample] != 0
    assert np.array_equal(wt[sample] != 0, ok)
    assert np.max(np.abs(wt[sample][ok] - orc.weight[sample][ok]) / orc.weight[sample][ok]) < TOL
    e = run.local_energies()[sample]
    e_ref = afqmc.local_energy(orc.setup, orc.theta[sample])
    assert np.max(np.abs(e - e_ref) / np.abs(e_ref)) < TOL


# ------------------------------------------------------------ host logic ----
def test_checkpoint_resume_is_bit_identical(pkg):
    w = workloads.config("c0")
    _, a = make_pair(pkg, w, nwalkers=8, pc_period=4)
    _, b = make_pair(pkg, w, nwalkers=8, pc_period=4)
    a.propagate(7)
    blob = a.save()
    a.propagate(9)
    b.load(blob)
    b.propagate(9)
    pa, wa, la = a.get_walkers()
    pb, wb, lb = b.get_walkers()
    assert np.array_equal(pa, pb) and np.array_equal(wa, wb) and np.array_equal(la, lb)
    assert np.array_equal(a.energy_log(), b.energy_log())


def test_errors_are_reported_not_raised_on_device(pkg):
    import torch

    w = workloads.config("c0")
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    p = pkg.default_params(w.M, w.N, w.nchol, 4)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.AfqmcError, match="ENOSPC"):
        pkg.AfqmcRun(h1, L, C, p, workspace=small)
    bad = h1.copy()
    bad[2, 3] = math.nan
    with pytest.raises(pkg.AfqmcError, match="ENONFINITE"):
        pkg.AfqmcRun(bad, L, C, p)
    q = pkg.default_params(w.M, w.N, w.nchol, 4, precision=7)
    with pytest.raises(pkg.AfqmcError):
        pkg.AfqmcRun(h1, L, C, q)
