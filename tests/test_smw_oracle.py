"""Pins of the reference-relative multi-determinant oracle (Sec. 3.4, Eqs.
usesherman, precomputing2, localenergy2, localenergy3; oracle.smw).

The case the per-determinant evaluation cannot resolve: a CI trial about a
reference determinant (single and double excitations in either spin, complex
coefficients) at the reference itself, where every excited determinant has
zero overlap with the walker while H still connects it.  Overlap, force-bias
traces and local energy are checked against brute-force Fock space there, at
walkers a hair away from it (overlaps of 1e-9) and at generic walkers.  For
generic non-orthogonal determinants the oracle equals the per-determinant
oracle (oracle.multidet), whose own pins are Fock space as well; a
one-determinant trial walks like the single-determinant oracle.
"""
import numpy as np
import pytest

import workloads
from fock import Fock, eri_from_cholesky
from oracle import afqmc, multidet, scf, smw


def system(M=4, G=6, seed=31):
    h1, L, _ = workloads.hamiltonian(M, G, seed)
    return h1, 0.6 * L


def ci_trial(C, N, excitations):
    """Determinants of the reference C[:, :N] with columns replaced in place:
    excitations is a list of (up, dn), each a list of (hole i, particle a)."""
    up, dn = [], []
    for eu, ed in excitations:
        Vu, Vd = C[:, :N].copy(), C[:, :N].copy()
        for i, a in eu:
            Vu[:, i] = C[:, a]
        for i, a in ed:
            Vd[:, i] = C[:, a]
        up.append(Vu)
        dn.append(Vd)
    return up, dn


EXC = [([], []), ([(1, 2)], []), ([], [(0, 3)]), ([(0, 2)], [(0, 2)]), ([(0, 2), (1, 3)], []),
       ([(1, 3)], [(0, 2)])]
COEF = np.array([0.9, 0.2 - 0.1j, -0.15, 0.3j, 0.12 + 0.05j, -0.07 + 0.2j])


def fock_reference(h1, L, H0, A, up, dn, phi):
    F = Fock(h1.shape[0])
    H = F.hamiltonian(h1, eri_from_cholesky(L), H0=H0)
    psiT = sum(A[d] * F.determinant(up[d], dn[d]) for d in range(len(A)))
    out = []
    for w in range(phi.shape[0]):
        psi = F.determinant(phi[w], phi[w])
        ov = psiT.conj() @ psi
        e = (psiT.conj() @ (H @ psi)) / ov
        t = np.array([(psiT.conj() @ (F.one_body(L[g]) @ psi)) / ov for g in range(L.shape[0])])
        out.append((ov, e, t))
    return out


@pytest.mark.parametrize("where", ["reference", "near", "generic"])
def test_ci_trial_matches_fock_space(where):
    M, N, G = 4, 2, 6
    h1, L = system(M, G)
    C = np.linalg.eigh(h1)[1]
    up, dn = ci_trial(C, N, EXC)
    st = smw.SMWSetup(h1, L, COEF, up, dn, H0=0.4)
    rng = np.random.default_rng(12)
    if where == "reference":
        phi = (C[:, :N] + 0j)[None]
    elif where == "near":
        # excited determinants' overlaps of order 1e-9
        phi = (C[:, :N] + 1e-9 * (rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))))[None]
    else:
        phi = rng.standard_normal((3, M, N)) + 1j * rng.standard_normal((3, M, N))
    ev = smw.evaluate(st, phi, energy=True)
    for w, (ov, e, t) in enumerate(fock_reference(h1, L, 0.4, COEF, up, dn, phi)):
        assert abs(np.exp(ev["logov"][w]) - ov) < 1e-12 * abs(ov)
        assert abs(ev["E"][w] - e) < 1e-11 * max(1.0, abs(e))
        assert np.max(np.abs(ev["t"][w] - t)) < 1e-11 * max(1.0, np.max(np.abs(t)))
    if where == "reference":
        # every excited determinant is orthogonal to the walker
        assert np.all(np.abs(ev["r"][0, 1:, 0] * ev["r"][0, 1:, 1]) < 1e-14)


def test_ci_trial_energy_differs_from_the_leading_determinant_alone():
    """At the reference the excited determinants change the mixed energy by
    their H-coupling (this is what the per-determinant evaluation loses)."""
    M, N, G = 4, 2, 6
    h1, L = system(M, G)
    C = np.linalg.eigh(h1)[1]
    up, dn = ci_trial(C, N, EXC)
    phi = (C[:, :N] + 0j)[None]
    e_ci = smw.evaluate(smw.SMWSetup(h1, L, COEF, up, dn), phi, energy=True)["E"][0]
    e_0 = smw.evaluate(smw.SMWSetup(h1, L, COEF[:1], up[:1], dn[:1]), phi, energy=True)["E"][0]
    assert abs(e_ci - e_0) > 1e-3


def test_generic_determinants_equal_the_per_determinant_oracle():
    M, N, G = 6, 3, 9
    h1, L = system(M, G, seed=5)
    rng = np.random.default_rng(3)
    nd = 4
    q = lambda: np.linalg.qr(rng.standard_normal((M, N)))[0]
    Vu = [q() for _ in range(nd)]
    Vd = [q() for _ in range(nd)]
    A = np.array([1.0, -0.4 + 0.3j, 0.25j, 0.6])
    phi = rng.standard_normal((5, M, N)) + 1j * rng.standard_normal((5, M, N))
    s_md = multidet.MultiDetSetup(h1, L, A, Vu, Vd, H0=-0.3)
    s_smw = smw.SMWSetup(h1, L, A, Vu, Vd, H0=-0.3)
    lo, th, w = multidet.overlap(s_md, phi)
    ev = smw.evaluate(s_smw, phi, energy=True)
    assert np.max(np.abs(np.exp(ev["logov"] - lo) - 1)) < 1e-11
    t = multidet.force_bias_trace(s_md, th, w)
    assert np.max(np.abs(ev["t"] - t)) < 1e-10 * np.max(np.abs(t))
    e = multidet.local_energy(s_md, th, w)
    assert np.max(np.abs(ev["E"] - e)) < 1e-10 * np.max(np.abs(e))
    assert abs(s_smw.E_T - s_md.E_T) < 1e-11 * abs(s_md.E_T)


def test_single_determinant_trial_walks_like_the_single_determinant_oracle():
    h1, L = system()
    C, _, conv, _ = scf.rhf(h1, L, 2)
    assert conv
    p = afqmc.Params(dt=0.02, seed=9, qr_period=3, energy_period=1)
    o1 = afqmc.Oracle(h1, L, C, 8, p).run(7)
    os_ = smw.SMWOracle(h1, L, [1.0], [C], [C], 8, p).run(7)
    assert abs(os_.setup.E_T - o1.setup.E_T) < 1e-12 * abs(o1.setup.E_T)
    assert np.max(np.abs(os_.phi - o1.phi)) < 1e-12
    assert np.max(np.abs(os_.weight - o1.weight)) < 1e-12
    assert np.allclose([r[1] for r in os_.records], [r[1] for r in o1.records], rtol=1e-12)


def test_walk_equals_the_per_determinant_walk_for_non_orthogonal_determinants():
    M, N, G = 5, 2, 8
    h1, L = system(M, G, seed=11)
    rng = np.random.default_rng(8)
    C, _, _, _ = scf.rhf(h1, L, N)
    Vu = [C, np.linalg.qr(C + 0.3 * rng.standard_normal((M, N)))[0]]
    Vd = [C, np.linalg.qr(C + 0.3 * rng.standard_normal((M, N)))[0]]
    A = [1.0, 0.35 - 0.2j]
    p = afqmc.Params(dt=0.02, seed=4, qr_period=3, energy_period=1)
    om = multidet.MultiDetOracle(h1, L, A, Vu, Vd, 6, p).run(8)
    os_ = smw.SMWOracle(h1, L, A, Vu, Vd, 6, p).run(8)
    assert abs(os_.setup.E_T - om.setup.E_T) < 1e-11 * abs(om.setup.E_T)
    assert np.max(np.abs(os_.phi - om.phi)) < 1e-10
    assert np.max(np.abs(os_.weight - om.weight)) < 1e-10
    assert np.allclose([r[1] for r in os_.records], [r[1] for r in om.records], rtol=1e-10)


def test_ci_trial_walk_stays_finite_and_uses_the_couplings():
    """A CI trial walk from the reference: finite weights and energies, and
    the first energy record differs from the leading-determinant walk's."""
    M, N, G = 4, 2, 6
    h1, L = system(M, G)
    C = np.linalg.eigh(h1)[1]
    up, dn = ci_trial(C, N, EXC)
    p = afqmc.Params(dt=0.01, seed=2, qr_period=2, energy_period=1)
    o = smw.SMWOracle(h1, L, COEF, up, dn, 8, p).run(6)
    o0 = smw.SMWOracle(h1, L, COEF[:1], up[:1], dn[:1], 8, p).run(6)
    assert o.nonfinite == 0 and np.all(np.isfinite(o.weight)) and np.count_nonzero(o.weight) == 8
    e = np.array([r[1] / r[2] for r in o.records])
    e0 = np.array([r[1] / r[2] for r in o0.records])
    assert np.all(np.isfinite(e)) and abs(e[0] - e0[0]) > 1e-4
