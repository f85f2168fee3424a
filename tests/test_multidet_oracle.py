"""Pins of the multi-determinant oracle (Sec. 3.4, Eqs. usesherman,
precomputing2, localenergy2, localenergy3).

The overlap, the force-bias traces and the local energy of a three-determinant
trial with different spin-up and spin-down orbitals and complex coefficients
are checked against brute-force Fock space; a one-determinant trial reproduces
the single-determinant oracle (set-up, estimators and a short walk) exactly;
scaling every coefficient by one complex number leaves the estimators alone; a
determinant orthogonal to the walker drops out without non-finite values (it
differs from the walker in two orbitals of each spin, so H does not connect
them either and the single-determinant energy is the exact mixed one).
"""
import numpy as np

import workloads
from fock import Fock, eri_from_cholesky
from oracle import afqmc, multidet, scf


def orthonormal(rng, M, N):
    q, _ = np.linalg.qr(rng.standard_normal((M, N)))
    return q


def system(M=4, G=6, seed=31):
    h1, L, _ = workloads.hamiltonian(M, G, seed)
    return h1, 0.6 * L


def test_single_determinant_trial_is_the_single_determinant_oracle():
    h1, L = system()
    C, _, conv, _ = scf.rhf(h1, L, 2)
    assert conv
    p = afqmc.Params(dt=0.02, seed=9, qr_period=3, energy_period=1)
    o1 = afqmc.Oracle(h1, L, C, 8, p).run(7)
    om = multidet.MultiDetOracle(h1, L, [1.0], [C], [C], 8, p).run(7)
    assert abs(om.setup.E_T - o1.setup.E_T) < 1e-12 * abs(o1.setup.E_T)
    assert np.max(np.abs(om.setup.c - o1.setup.c)) < 1e-13
    assert np.max(np.abs(om.phi - o1.phi)) < 1e-12
    assert np.max(np.abs(om.weight - o1.weight)) < 1e-12
    d = np.angle(np.exp(1j * (om.logdet.imag - o1.logdet.imag)))
    assert np.max(np.abs(om.logdet.real - o1.logdet.real)) < 1e-12 and np.max(np.abs(d)) < 1e-12
    assert np.allclose([r[1] for r in om.records], [r[1] for r in o1.records], rtol=1e-12)


def test_overlap_force_bias_and_energy_match_fock_space():
    M, N, G = 4, 2, 6
    h1, L = system(M, G)
    rng = np.random.default_rng(4)
    nd = 3
    Vu = [orthonormal(rng, M, N) for _ in range(nd)]
    Vd = [orthonormal(rng, M, N) for _ in range(nd)]
    A = np.array([0.9, -0.3 + 0.2j, 0.15j])
    st = multidet.MultiDetSetup(h1, L, A, Vu, Vd, H0=0.4)
    W = 3
    phi = rng.standard_normal((W, M, N)) + 1j * rng.standard_normal((W, M, N))
    logov, theta, w = multidet.overlap(st, phi)
    t = multidet.force_bias_trace(st, theta, w)
    e = multidet.local_energy(st, theta, w)
    F = Fock(M)
    H = F.hamiltonian(h1, eri_from_cholesky(L), H0=0.4)
    psiT = sum(A[d] * F.determinant(Vu[d], Vd[d]) for d in range(nd))
    for wi in range(W):
        psi = F.determinant(phi[wi], phi[wi])
        ov = psiT.conj() @ psi
        assert abs(np.exp(logov[wi]) - ov) < 1e-12 * abs(ov)
        eref = (psiT.conj() @ (H @ psi)) / ov
        assert abs(e[wi] - eref) < 1e-11 * max(1.0, abs(eref))
        for g in range(G):
            tref = (psiT.conj() @ (F.one_body(L[g]) @ psi)) / ov
            assert abs(t[wi, g] - tref) < 1e-11 * max(1.0, abs(tref))
    assert np.allclose(np.sum(w, axis=1), 1.0)


def test_estimators_do_not_depend_on_a_common_coefficient_factor():
    M, N, G = 5, 2, 7
    h1, L = system(M, G, seed=8)
    rng = np.random.default_rng(6)
    Vu = [orthonormal(rng, M, N) for _ in range(2)]
    Vd = [orthonormal(rng, M, N) for _ in range(2)]
    A = np.array([1.0, 0.4 - 0.1j])
    phi = rng.standard_normal((4, M, N)) + 1j * rng.standard_normal((4, M, N))
    s1 = multidet.MultiDetSetup(h1, L, A, Vu, Vd)
    s2 = multidet.MultiDetSetup(h1, L, (2.0 - 1.5j) * A, Vu, Vd)
    l1, th1, w1 = multidet.overlap(s1, phi)
    l2, th2, w2 = multidet.overlap(s2, phi)
    assert np.allclose(np.exp(l2 - l1), np.conj(2.0 - 1.5j))
    assert np.allclose(w1, w2) and np.allclose(th1, th2)
    assert np.allclose(multidet.local_energy(s1, th1, w1), multidet.local_energy(s2, th2, w2))


def test_determinant_orthogonal_to_the_walker_drops_out():
    M, N, G = 4, 2, 5
    h1, L = system(M, G, seed=3)
    e = np.eye(M)
    V0, V1 = e[:, :2], e[:, 2:]
    st = multidet.MultiDetSetup(h1, L, [1.0, 0.5], [V0, V1], [V0, V1])
    phi = (e[:, :2] + 0j)[None]  # <Psi_1|Psi> = 0
    logov, theta, w = multidet.overlap(st, phi)
    assert w[0, 1] == 0 and abs(w[0, 0] - 1) < 1e-15
    assert np.all(np.isfinite(theta))
    e_md = multidet.local_energy(st, theta, w)
    st1 = afqmc.Setup(h1, L, V0)
    _, th = afqmc.overlap(st1, phi)
    assert abs(e_md[0] - afqmc.local_energy(st1, th)[0]) < 1e-12
