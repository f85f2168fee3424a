"""Pins of the oracle's two-spin-block walkers (N_up != N_dn, different
spin-up and spin-down trial orbitals) against brute-force Fock space.

Theorem 1.1 takes the overlap of two Slater determinants as the product over
spins of det(V_sigma^H phi_sigma); the propagator B(x) of Eq. hs2 is spin
independent, so it acts on the spin-up and spin-down orbitals alike.  Every
quantity the oracle forms per block (overlap, Theta, force bias, local
energy, the step's overlap ratio and importance function, Gram-Schmidt) is
checked against explicit Jordan-Wigner vectors and operators, which know
nothing of blocks.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from fock import Fock, eri_from_cholesky
from oracle import afqmc, philox

M, NU, ND, G = 4, 3, 2, 6


@pytest.fixture(scope="module")
def spin_case():
    h1, L, _ = workloads.hamiltonian(M, G, 91)
    L = 0.6 * L
    rng = np.random.default_rng(13)
    # a trial whose spin-down orbitals are not a subset of the spin-up ones
    Vu = np.linalg.qr(rng.standard_normal((M, NU)))[0]
    Vd = np.linalg.qr(rng.standard_normal((M, ND)))[0]
    pu = Vu + 0.3 * rng.standard_normal((M, NU)) + 0.3j * rng.standard_normal((M, NU))
    pd = Vd + 0.3 * rng.standard_normal((M, ND)) + 0.3j * rng.standard_normal((M, ND))
    F = Fock(M)
    H0 = 0.4
    H = F.hamiltonian(h1, eri_from_cholesky(L), H0)
    vg = [1j * F.one_body(L[g]).toarray() for g in range(G)]
    return dict(h1=h1, L=L, Vu=Vu, Vd=Vd, pu=pu, pd=pd, F=F, H=H, H0=H0, vg=vg,
                phi=np.concatenate([pu, pd], axis=1))


def _psiT(c):
    return c["F"].determinant(c["Vu"], c["Vd"])


def _psi(c, phi):
    return c["F"].determinant(phi[:, :NU], phi[:, NU:])


def test_setup_trial_energy_and_background(spin_case):
    """E_T = <Psi_T|H|Psi_T> (UHF energy) and c_g with vbar_g = i c_g =
    <Psi_T|v_g|Psi_T> (Sec. 2.4) for a two-block trial."""
    c = spin_case
    st = afqmc.Setup(c["h1"], c["L"], c["Vu"], c["H0"], trial_dn=c["Vd"])
    psiT = _psiT(c)
    nrm = psiT.conj() @ psiT
    e_t = (psiT.conj() @ (c["H"] @ psiT)) / nrm
    assert abs(st.E_T - e_t.real) < 1e-12 * abs(e_t)
    for g in range(G):
        assert abs(1j * st.c[g] - (psiT.conj() @ c["vg"][g] @ psiT) / nrm) < 1e-13


def test_overlap_force_bias_and_local_energy(spin_case):
    """Theorem 1.1 (product over spins), Eq. precomputing2 and Eqs.
    localenergy2/3 with the exchange over same-spin pairs only."""
    c = spin_case
    st = afqmc.Setup(c["h1"], c["L"], c["Vu"], c["H0"], trial_dn=c["Vd"])
    logdet, theta = afqmc.overlap(st, c["phi"][None])
    psiT, psi = _psiT(c), _psi(c, c["phi"])
    ov = psiT.conj() @ psi
    assert abs(np.exp(logdet[0]) - ov) < 1e-13 * abs(ov)
    eloc = (psiT.conj() @ (c["H"] @ psi)) / ov
    assert abs(afqmc.local_energy(st, theta)[0] - eloc) < 1e-12 * abs(eloc)
    t = afqmc.force_bias_trace(st, theta)[0]
    for g in range(G):
        vm = psiT.conj() @ c["vg"][g] @ psi / ov
        assert abs(vm - 1j * t[g]) < 1e-13


def test_mean_field_rewrite(spin_case):
    """Sec. 2.4 with the two-block trial's background: H = H0' + v0' -
    1/2 sum_g (v_g - vbar_g)^2."""
    c = spin_case
    F = c["F"]
    st = afqmc.Setup(c["h1"], c["L"], c["Vu"], c["H0"], trial_dn=c["Vd"])
    I = np.eye(F.dim)
    H = st.H0p * I + F.one_body(st.v0p).toarray()
    for g in range(G):
        d = c["vg"][g] - 1j * st.c[g] * I
        H = H - 0.5 * d @ d
    assert np.max(np.abs(H - c["H"].toarray())) < 1e-12


def _propagator(c, st, x, dt):
    """B(x) with the mean-field operators and scalar (Eqs. hs2, primitive) as
    Fock-space exponentials."""
    F = c["F"]
    psiT = _psiT(c)
    nrm = psiT.conj() @ psiT
    I = np.eye(F.dim)
    v = eri_from_cholesky(c["L"])
    v0 = F.one_body(c["h1"] - 0.5 * np.einsum("prrq->pq", v)).toarray()
    A = np.zeros((F.dim, F.dim), complex)
    vbars = []
    for g in range(G):
        vbar = psiT.conj() @ c["vg"][g] @ psiT / nrm
        vbars.append(vbar)
        v0 = v0 - vbar * c["vg"][g]
        A = A + math.sqrt(dt) * x[g] * (c["vg"][g] - vbar * I)
    H0p = c["H0"] + 0.5 * np.sum(np.array(vbars) ** 2)
    half = sla.expm(-0.5 * dt * v0)
    return np.exp(-dt * (H0p - st.E_T)) * half @ sla.expm(A) @ half


def test_free_projection_step(spin_case):
    """Eq. weight_update: one free-projection step multiplies the weight by
    <Psi_T|B(x)|Psi>/<Psi_T|Psi>, and the new spin blocks span B(x)|Psi>."""
    c = spin_case
    dt = 0.02
    p = afqmc.Params(dt=dt, taylor_order=40, qr_period=0, energy_period=0, mode="free", seed=5)
    o = afqmc.Oracle(c["h1"], c["L"], c["Vu"], 1, p, H0=c["H0"], phi0=c["phi"], trial_dn=c["Vd"])
    xi = philox.gaussian_fields(5, 0, [0], G)[0]
    o.step()
    psiT, psi = _psiT(c), _psi(c, c["phi"])
    psi1 = _propagator(c, o.setup, xi, dt) @ psi
    assert abs(o.weight[0] - (psiT.conj() @ psi1) / (psiT.conj() @ psi)) < 1e-12
    psi1o = _psi(c, o.phi[0])
    k = np.argmax(np.abs(psi1o))
    assert np.max(np.abs(psi1 - psi1[k] / psi1o[k] * psi1o)) < 1e-12 * np.max(np.abs(psi1))


def _fock_xbar(c, dt, phi):
    psiT, psi = _psiT(c), _psi(c, phi)
    ov, nrm = psiT.conj() @ psi, psiT.conj() @ psiT
    return np.array([-math.sqrt(dt) * (psiT.conj() @ v @ psi / ov - psiT.conj() @ v @ psiT / nrm)
                     for v in c["vg"]])


@pytest.mark.parametrize("mode", ["complex_is", "phaseless"])
def test_importance_function_and_phaseless_weight(spin_case, mode):
    """Eq. hybrid-wt with the optimal force bias of Eq. fb (complex weight)
    and the phaseless weight |I| max(0, cos Arg R) of Eq. weight_update_2,
    from Fock-space R and I."""
    c = spin_case
    dt = 0.3
    p = afqmc.Params(dt=dt, taylor_order=50, qr_period=0, energy_period=0, mode=mode, seed=3,
                     fb_cap=-1.0, wmax=1e300)
    o = afqmc.Oracle(c["h1"], c["L"], c["Vu"], 1, p, H0=c["H0"], phi0=c["phi"], trial_dn=c["Vd"])
    xi = philox.gaussian_fields(3, 0, [0], G)[0]
    xbar = _fock_xbar(c, dt, c["phi"])
    psiT, psi = _psiT(c), _psi(c, c["phi"])
    R = (psiT.conj() @ (_propagator(c, o.setup, xi - xbar, dt) @ psi)) / (psiT.conj() @ psi)
    I = R * np.exp(np.sum(xi * xbar) - 0.5 * np.sum(xbar * xbar))
    o.step()
    if mode == "complex_is":
        assert abs(o.weight[0] - I) < 1e-12 * abs(I)
    else:
        expected = abs(I) * max(0.0, math.cos(np.angle(R)))
        assert abs(o.weight[0] - expected) < 1e-12 * max(1.0, expected)


def test_gram_schmidt_per_spin_block(spin_case):
    """Sec. 3.4.5 / Theorem 1.5 per spin: each block becomes the Q of its own
    QR factorisation (a spin-down orbital is never projected on a spin-up
    one); force bias and local energy are unchanged and the overlap scales by
    det(R_up) det(R_dn)."""
    c = spin_case
    st = afqmc.Setup(c["h1"], c["L"], c["Vu"], c["H0"], trial_dn=c["Vd"])
    phi = 2.5 * c["phi"][None]
    q = afqmc.mgs(phi, st.blocks)
    logr = 0.0
    for a, b in ((0, NU), (NU, NU + ND)):
        Q, R = np.linalg.qr(phi[0][:, a:b])
        ph = np.diag(R) / np.abs(np.diag(R))
        assert np.max(np.abs(q[0][:, a:b] - Q * ph)) < 1e-13
        logr += np.sum(np.log(np.abs(np.diag(R))))
    ld0, th0 = afqmc.overlap(st, phi)
    ld1, th1 = afqmc.overlap(st, q)
    assert np.max(np.abs(afqmc.force_bias_trace(st, th0) - afqmc.force_bias_trace(st, th1))) < 1e-11
    e0, e1 = afqmc.local_energy(st, th0), afqmc.local_energy(st, th1)
    assert abs(e0[0] - e1[0]) < 1e-11 * abs(e0[0])
    assert abs((ld0[0].real - ld1[0].real) - logr) < 1e-12


def test_two_identical_blocks_are_the_closed_shell_walk():
    """A two-block run whose spin-down trial equals the spin-up one (N_up =
    N_dn) is the restricted closed-shell walk: same weights, overlaps and
    energies over steps with Gram-Schmidt."""
    w = workloads.config("c0")
    h1, L, _ = w.hamiltonian()
    C = np.linalg.eigh(h1)[1][:, :w.N]
    p = afqmc.Params(dt=w.dt, seed=2, qr_period=3, energy_period=2)
    a = afqmc.Oracle(h1, L, C, 8, p).run(7)
    b = afqmc.Oracle(h1, L, C, 8, p, trial_dn=C).run(7)
    assert np.max(np.abs(b.weight - a.weight) / np.abs(a.weight)) < 1e-11
    assert np.max(np.abs(b.logdet - a.logdet)) < 1e-10
    assert np.max(np.abs(b.phi[:, :, :w.N] - a.phi)) < 1e-11
    assert np.max(np.abs(b.phi[:, :, w.N:] - a.phi)) < 1e-11
    ea = np.array([r[1] / r[2] for r in a.records])
    eb = np.array([r[1] / r[2] for r in b.records])
    assert np.max(np.abs(eb - ea) / np.abs(ea)) < 1e-12
