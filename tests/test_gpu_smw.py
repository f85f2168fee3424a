"""Multi-determinant trial evaluated relative to its leading determinant on the
GPU (Sec. 3.4, Eqs. usesherman, precomputing2, localenergy2/3, the
Sherman-Morrison-Woodbury remark) against the oracle's walk (oracle.smw).

Trials are CI expansions about the RHF determinant: each determinant replaces
up to four RHF orbitals per spin, in place, by virtual orbitals (single to
quadruple excitations, complex coefficients).  The walkers start at the RHF
determinant, where every excited determinant has zero overlap with them while
H and the v_g still connect it: the case the per-determinant evaluation
cannot take.  Float64 path: E_T, local energies, walkers, weights,
log-overlaps and energy records agree with the oracle to 1e-10 relative at
every checked step.  The mixed precisions keep this float64 evaluation and
propagate in BF16/TF32: they agree with the float64 walk within the operand
rounding.
"""
import numpy as np
import pytest

import workloads
from oracle import afqmc, scf, smw

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


def ci_trial(M, N, G, seed, excitations, coef):
    """RHF orbitals of the first converging Hamiltonian seed from `seed`, and
    the determinants of the excitation list: (up, dn), each a list of
    (hole i, virtual a) with a counted from N."""
    for sd in range(seed, seed + 40):
        h1, L, _ = workloads.hamiltonian(M, G, sd, l_scale=workloads.l_amplitude(M, G))
        C, _, conv, _ = scf.rhf(h1, L, N)
        if conv:
            break
    assert conv
    rng = np.random.default_rng(sd)
    q, _ = np.linalg.qr(np.hstack([C, rng.standard_normal((M, M - N))]))
    virt = q[:, N:]
    up, dn = [], []
    for eu, ed in excitations:
        Vu, Vd = C.copy(), C.copy()
        for i, a in eu:
            Vu[:, i] = virt[:, a]
        for i, a in ed:
            Vd[:, i] = virt[:, a]
        up.append(Vu)
        dn.append(Vd)
    return h1, L, np.asarray(coef), np.array(up), np.array(dn)


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


CASES = {
    # 12 orbitals, 3 electrons per spin: singles and doubles in either spin
    "cisd": (12, 3, 48, 32, 5, 1,
             [([], []), ([(2, 0)], []), ([], [(1, 2)]), ([(2, 0)], [(2, 0)]),
              ([(1, 1), (2, 3)], []), ([(0, 4)], [(2, 1)]), ([], [(0, 0), (1, 5)])],
             [0.92, 0.18 - 0.07j, -0.11, 0.25j, 0.08 + 0.04j, -0.05 + 0.12j, 0.06]),
    # ragged: M=20, N=5, 33 vectors, 17 walkers; a quadruple excitation and a
    # determinant equal to the reference in one spin
    "ragged": (20, 5, 33, 17, 3, 2,
               [([], []), ([(4, 0)], [(3, 2)]), ([(0, 1), (1, 2), (3, 3), (4, 5)], []),
                ([], [(2, 7), (4, 1)])],
               [1.0, -0.2 + 0.15j, 0.07, 0.1j]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_ci_walk_matches_oracle(pkg, case):
    M, N, G, W, qr, ep, exc, coef = CASES[case]
    h1, L, coef, up, dn = ci_trial(M, N, G, 7100 + M, exc, coef)
    nd = len(coef)
    p_o = afqmc.Params(dt=0.01, seed=3, qr_period=qr, energy_period=ep)
    orc = smw.SMWOracle(h1, L, coef, up, dn, W, p_o)
    p = pkg.default_params(M, N, G, W, dt=0.01, seed=3, qr_period=qr, energy_period=ep, ndet=nd)
    run = pkg.AfqmcRun(h1, L, (coef, up, dn), p)
    assert abs(run.info().E_T - orc.setup.E_T) < TOL * abs(orc.setup.E_T)
    e0 = run.local_energies()
    assert np.max(np.abs(e0 - orc.local_energies())) < TOL * np.max(np.abs(e0))
    for chunk in (4, 8):
        orc.run(chunk)
        run.propagate(chunk)
        assert compare(run, orc) > W // 2
        e = run.local_energies()
        eo = orc.local_energies()
        alive = np.nonzero(orc.weight != 0)[0]
        assert np.max(np.abs(e[alive] - eo[alive])) < TOL * np.max(np.abs(eo[alive]))
    log = run.energy_log()
    e_orc = np.array([r[1] / r[2] for r in orc.records])
    assert np.max(np.abs(log[:, 1] - e_orc) / np.abs(e_orc)) < TOL
    assert run.info().status == 0


def test_ci_trial_differs_from_the_reference_alone(pkg):
    """The excited determinants move E_T (their H-coupling to the reference)."""
    M, N, G, W, qr, ep, exc, coef = CASES["cisd"]
    h1, L, coef, up, dn = ci_trial(M, N, G, 7100 + M, exc, coef)
    p = pkg.default_params(M, N, G, W, ndet=len(coef))
    run = pkg.AfqmcRun(h1, L, (coef, up, dn), p)
    p1 = pkg.default_params(M, N, G, W, ndet=1)
    run1 = pkg.AfqmcRun(h1, L, (coef[:1], up[:1], dn[:1]), p1)
    assert abs(run.info().E_T - run1.info().E_T) > 1e-4


@pytest.mark.parametrize("prec,tol_e,tol_phi", [(2, 3e-3, 1.5e-2), (1, 4e-4, 4e-3)])
def test_ci_mixed_path_close_to_float64(pkg, prec, tol_e, tol_phi):
    """The CI trial on the mixed path (BF16/TF32 propagation, the float64
    evaluation relative to the reference) against the float64 path on the same
    seed and steps: they differ by the propagation's operand rounding only.
    Orbitals and weights within 8 units of the operand rounding (8 x 2^-9 =
    1.6e-2 BF16, 8 x 2^-11 = 3.9e-3 TF32) after seven steps."""
    M, N, G, W, qr, ep, exc, coef = CASES["cisd"]
    h1, L, coef, up, dn = ci_trial(M, N, G, 7100 + M, exc, coef)
    out = []
    for precision in (0, prec):
        p = pkg.default_params(M, N, G, W, dt=0.01, seed=4, qr_period=5, energy_period=1,
                               ndet=len(coef), precision=precision)
        run = pkg.AfqmcRun(h1, L, (coef, up, dn), p)
        e0 = run.local_energies()
        run.propagate(7)
        out.append((run.info().E_T, e0, run.get_walkers(), run.energy_log()))
        assert run.info().status == 0
        run.close()
    (et0, e00, (phi0, w0, _), log0), (et1, e01, (phi1, w1, _), log1) = out
    # the set-up (E_T, local energies at the reference) is float64 on both paths
    assert abs(et1 - et0) < 1e-12 * abs(et0)
    assert np.max(np.abs(e01 - e00) / np.abs(e00)) < 1e-12
    alive = np.nonzero(w0 != 0)[0]
    assert np.array_equal(np.nonzero(w1 != 0)[0], alive) and alive.size > W // 2
    d = np.linalg.norm((phi1 - phi0)[alive].reshape(alive.size, -1), axis=1)
    n = np.linalg.norm(phi0[alive].reshape(alive.size, -1), axis=1)
    assert np.max(d / n) < tol_phi
    assert np.max(np.abs(w1[alive] - w0[alive]) / w0[alive]) < tol_phi
    assert np.max(np.abs(log1[:, 1] - log0[:, 1]) / np.abs(log0[:, 1])) < tol_e
