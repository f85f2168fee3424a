"""Multi-determinant trial on the GPU (afqmc_init_multidet; Sec. 3.4, Eqs.
usesherman, precomputing2, localenergy2/3) against the oracle's
multi-determinant walk (oracle.multidet).

Float64 path: walkers, weights, log-overlaps and energy records agree with the
oracle to 1e-10 relative at every checked step; the mixed path agrees with
the float64 path within the operand rounding.  Trials: three non-orthogonal
determinants (each spin of each determinant a different rotation of the RHF
orbitals, so spin-up and spin-down orbitals differ) with complex
coefficients; a ragged shape with two determinants; a one-determinant trial
given through the multi-determinant entry point, which must reproduce the
single-determinant walk of afqmc_init; and the unsupported combinations and
bad inputs.  With three orbitals per spin every determinant differs from the
leading one in at most four columns, so the library evaluates that trial
relative to determinant 0 (the low-rank route of tests/test_gpu_smw.py) and
the per-determinant oracle checks it; five orbitals per spin take the
per-determinant route.  (CI expansions about the walker's own determinant,
where each w_d E_d of the per-determinant evaluation is a 0/0 limit, are
covered by tests/test_gpu_smw.py.)
"""
import numpy as np
import pytest

import workloads
from oracle import afqmc, multidet, scf

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


def noci_trial(M, N, G, seed, nd):
    """A multi-determinant trial of non-orthogonal determinants around the RHF
    determinant of the first Hamiltonian seed (from `seed` on) whose RHF
    iteration converges: determinant d, spin s has the orbitals of the RHF
    basis rotated by exp(K_ds), K_ds a random antisymmetric matrix (small
    occupied-virtual mixing, different for the two spins); determinant 0
    spin up is the RHF determinant itself."""
    import scipy.linalg as sla

    for sd in range(seed, seed + 40):
        h1, L, _ = workloads.hamiltonian(M, G, sd, l_scale=workloads.l_amplitude(M, G))
        C, _, conv, _ = scf.rhf(h1, L, N)
        if conv:
            break
    assert conv
    rng = np.random.default_rng(sd)
    q, _ = np.linalg.qr(np.hstack([C, rng.standard_normal((M, M - N))]))
    basis = np.hstack([C, q[:, N:]])
    up, dn = [], []
    for d in range(nd):
        for lst, s in ((up, 0), (dn, 1)):
            if d == 0 and s == 0:
                lst.append(C)
                continue
            K = 0.08 * rng.standard_normal((M, M))
            K = K - K.T
            lst.append(basis @ sla.expm(K)[:, :N])
    coef = np.array([0.95, 0.2 - 0.1j, -0.15])[:nd]
    return h1, L, coef, np.array(up), np.array(dn)


def compare(run, orc):
    phi, wt, lo = run.get_walkers()
    alive = np.nonzero(orc.weight != 0)[0]
    assert np.array_equal(np.nonzero(wt != 0)[0], alive)
    W = phi.shape[0]
    d = np.linalg.norm((phi - orc.phi).reshape(W, -1), axis=1)
    n = np.linalg.norm(orc.phi.reshape(W, -1), axis=1)
    assert np.max(d[alive] / n[alive]) < TOL
    assert np.max(np.abs(wt[alive] - orc.weight[alive]) / orc.weight[alive]) < TOL
    scale = 1 + np.abs(orc.logdet[alive].real)
    assert np.max(np.abs(lo[alive].real - orc.logdet[alive].real) / scale) < TOL
    dph = np.angle(np.exp(1j * (lo[alive].imag - orc.logdet[alive].imag)))
    assert np.max(np.abs(dph) / scale) < TOL
    return alive.size


@pytest.mark.parametrize("M,N,G,W,nd,qr,ep", [(12, 3, 48, 32, 3, 5, 1), (20, 5, 33, 17, 2, 3, 2)])
def test_walk_matches_oracle(pkg, M, N, G, W, nd, qr, ep):
    h1, L, coef, up, dn = noci_trial(M, N, G, 7000 + M, nd)
    p_o = afqmc.Params(dt=0.01, seed=5, qr_period=qr, energy_period=ep)
    orc = multidet.MultiDetOracle(h1, L, coef, up, dn, W, p_o)
    p = pkg.default_params(M, N, G, W, dt=0.01, seed=5, qr_period=qr, energy_period=ep, ndet=nd)
    run = pkg.AfqmcRun(h1, L, (coef, up, dn), p)
    assert abs(run.info().E_T - orc.setup.E_T) < TOL * abs(orc.setup.E_T)
    e0 = run.local_energies()
    assert np.max(np.abs(e0 - orc.local_energies())) < TOL * np.max(np.abs(e0))
    for chunk in (4, 6):
        orc.run(chunk)
        run.propagate(chunk)
        assert compare(run, orc) > W // 2
    log = run.energy_log()
    want = np.array([r[1] / r[2] for r in orc.records])
    assert np.max(np.abs(log[:, 1] - want) / np.abs(want)) < TOL
    e = run.local_energies()
    alive = orc.weight != 0
    eo = orc.local_energies()
    assert np.max(np.abs(e[alive] - eo[alive]) / np.abs(eo[alive])) < TOL
    run.close()


def test_one_determinant_is_the_single_determinant_walk(pkg):
    M, N, G, W = 12, 3, 48, 16
    h1, L, coef, up, dn = noci_trial(M, N, G, 7100, 1)
    a = pkg.AfqmcRun(h1, L, (np.array([1.0]), up[:1], up[:1]),  # the RHF determinant, both spins
                     pkg.default_params(M, N, G, W, dt=0.01, seed=2, ndet=1))
    b = pkg.AfqmcRun(h1, L, up[0], pkg.default_params(M, N, G, W, dt=0.01, seed=2))
    a.propagate(8)
    b.propagate(8)
    pa, wa, la = a.get_walkers()
    pb, wb, lb = b.get_walkers()
    assert np.max(np.abs(pa - pb)) < 1e-11 and np.max(np.abs(wa - wb)) < 1e-11 * np.max(wb.real)
    assert np.max(np.abs(a.energy_log()[:, 1] - b.energy_log()[:, 1])) < 1e-10
    a.close()
    b.close()


@pytest.mark.parametrize("prec,tol_e,tol_phi", [(2, 3e-3, 1.5e-2), (1, 4e-4, 2e-3)])
def test_mixed_path_close_to_float64(pkg, prec, tol_e, tol_phi):
    """The mixed path (the force-bias traces and the exchange of every
    determinant and spin on the tensor cores from BF16/TF32 copies of Lh_ds and
    Theta_ds; overlaps, weights and combinations in float64) against the
    float64 path on the same trial, seed and steps: they differ by the operand
    rounding only (BF16 2^-9, TF32 2^-11 relative per operand)."""
    M, N, G, W, nd = 24, 5, 120, 64, 3  # five columns per spin differ: per-determinant route
    h1, L, coef, up, dn = noci_trial(M, N, G, 7300, nd)
    out = []
    for precision in (0, prec):
        p = pkg.default_params(M, N, G, W, dt=0.01, seed=4, qr_period=5, energy_period=1,
                               ndet=nd, precision=precision)
        run = pkg.AfqmcRun(h1, L, (coef, up, dn), p)
        e0 = run.local_energies()
        run.propagate(7)
        out.append((run.info().E_T, e0, run.get_walkers(), run.energy_log()))
        assert run.info().status == 0
        run.close()
    (et0, e00, (phi0, w0, _), log0), (et1, e01, (phi1, w1, _), log1) = out
    assert abs(et1 - et0) < tol_e * abs(et0)
    assert np.max(np.abs(e01 - e00) / np.abs(e00)) < tol_e
    alive = np.nonzero(w0 != 0)[0]
    assert np.array_equal(np.nonzero(w1 != 0)[0], alive) and alive.size > W // 2
    d = np.linalg.norm((phi1 - phi0)[alive].reshape(alive.size, -1), axis=1)
    n = np.linalg.norm(phi0[alive].reshape(alive.size, -1), axis=1)
    assert np.max(d / n) < tol_phi
    assert np.max(np.abs(w1[alive] - w0[alive]) / w0[alive]) < tol_phi
    assert log1.shape == log0.shape
    assert np.max(np.abs(log1[:, 1] - log0[:, 1]) / np.abs(log0[:, 1])) < tol_e


def test_errors(pkg):
    M, N, G, W = 12, 3, 48, 8
    h1, L, coef, up, dn = noci_trial(M, N, G, 7200, 2)
    for kw in (dict(pc_period=5), dict(bp_steps=4), dict(mode=pkg.AFQMC_FREE),
               dict(pc_period=5, precision=pkg.AFQMC_MIXED_BF16)):
        with pytest.raises(pkg.AfqmcError, match="EUNSUPPORTED"):
            pkg.afqmc_workspace_size(pkg.default_params(M, N, G, W, ndet=2, **kw))
    import ctypes

    # afqmc_init takes the single RHF trial only (ndet = 0)
    p = pkg.default_params(M, N, G, W, ndet=2)
    st = ctypes.c_void_p()
    assert pkg.lib().afqmc_init(ctypes.byref(p), None, None, None, None, None, 0, None,
                                ctypes.byref(st)) == -1
    bad = up.copy()
    bad[1] *= 1.5
    with pytest.raises(pkg.AfqmcError, match="EINVAL"):
        pkg.AfqmcRun(h1, L, (coef, bad, dn), pkg.default_params(M, N, G, W, ndet=2))
