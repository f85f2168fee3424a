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


def test_real_propagator_projection_is_the_constrained_path():
    """P9 (Sec. 3.3, the constrained-path limit): with a real propagator the
    overlap ratio R is real, so max(0, cos Arg R) is 1 or 0 and the phaseless
    weight update becomes the constrained path: a walker whose overlap with
    the trial changes sign is removed, the others are multiplied by R.  No
    two-body term (L = 0: no fields, no force bias, B = exp(-dt h)), real
    two-block walkers near a node of the spin-up overlap (with a closed-shell
    walker det(S)^2 could never change sign).  R from scipy's expm of h."""
    M, dt = 4, 0.1
    rng = np.random.default_rng(3)
    h = rng.standard_normal((M, M))
    h = 0.5 * (h + h.T)
    h[0, 1] = h[1, 0] = 2.0
    L = np.zeros((1, M, M))
    Vu, Vd = np.eye(M)[:, :1], np.eye(M)[:, 1:2]
    B = sla.expm(-dt * h)
    eps = np.array([0.05, 1.0, -0.02, 0.6])  # spin-up overlaps near and far from the node
    phi = np.zeros((eps.size, M, 2))
    phi[:, 0, 0] = eps
    phi[:, 1, 0] = 1.0
    phi[:, 2, 1] = 1.0
    phi[:, 1, 1] = 0.3
    p = afqmc.Params(dt=dt, taylor_order=4, qr_period=0, energy_period=0, fb_cap=-1.0,
                     wmax=1e300, seed=1)
    o = afqmc.Oracle(h, L, Vu, eps.size, p, phi0=phi.astype(complex), trial_dn=Vd)
    e_shift = o.e_shift
    o.step()
    flips = 0
    for w in range(eps.size):
        up, dn = B @ phi[w][:, :1], B @ phi[w][:, 1:]
        R = (np.linalg.det(Vu.T @ up) * np.linalg.det(Vd.T @ dn)
             / (np.linalg.det(Vu.T @ phi[w][:, :1]) * np.linalg.det(Vd.T @ phi[w][:, 1:])))
        R *= math.exp(-dt * (0.0 - e_shift))
        if R < 0:
            flips += 1
            assert o.weight[w] == 0.0
        else:
            assert abs(o.weight[w] - R) < 1e-12 * R
    assert 0 < flips < eps.size


def test_trotter_error_of_the_energy_falls_as_dt_squared():
    """P12 (Sec. 3.3: the Trotter error is O(dt^2)): the oracle's step averaged
    exactly over its field (one Cholesky vector, Gauss-Hermite quadrature)
    is a Fock-space operator T(dt); the energy <Psi_T|H T^n|Psi_T> /
    <Psi_T|T^n|Psi_T> at beta = n dt = 1 approaches the exact
    <Psi_T|H e^(-beta H)|Psi_T> / <Psi_T|e^(-beta H)|Psi_T> with an error that
    falls 4x per halving of dt.  Two spin blocks (N_up = 2, N_dn = 1), so T
    is built on every determinant of the sector, spin-up and spin-down
    orbitals differing."""
    M_, nu, nd, G_ = 4, 2, 1, 1
    h1, L, _ = workloads.hamiltonian(M_, G_, 31)
    L = 1.5 * L
    rng = np.random.default_rng(31)
    Vu = np.linalg.qr(rng.standard_normal((M_, nu)))[0]
    Vd = np.linalg.qr(rng.standard_normal((M_, nd)))[0]
    F = Fock(M_)
    H = F.hamiltonian(h1, eri_from_cholesky(L), 0.0).toarray()
    sec = F.number_sector(nu, nd)
    Hs = H[np.ix_(sec, sec)]
    psiT = F.determinant(Vu, Vd)[sec]
    xk, wk = np.polynomial.hermite_e.hermegauss(30)
    wk = wk / math.sqrt(2 * math.pi)
    dets = [(np.eye(M_)[:, list(u)], np.eye(M_)[:, list(d)])
            for u in itertools.combinations(range(M_), nu)
            for d in itertools.combinations(range(M_), nd)]

    def field_averaged_step(dt):
        st = afqmc.Setup(h1, L, Vu, 0.0, dt=dt, trial_dn=Vd)
        U = np.zeros((sec.size, len(dets)), complex)
        TU = np.zeros_like(U)
        for b, (Pu, Pd) in enumerate(dets):
            phi = np.concatenate([Pu, Pd], 1).astype(complex)
            U[:, b] = F.determinant(Pu, Pd)[sec]
            for x, wx in zip(xk, wk):
                xv = np.array([x], complex)
                V = afqmc.assemble_V(st, xv[None])
                phi1 = st.Bhalf @ afqmc.taylor(V, (st.Bhalf @ phi)[None], 40)[0]
                scal = math.exp(-dt * st.H0p) * np.exp(-1j * math.sqrt(dt) * (xv @ st.c))
                TU[:, b] += wx * scal * F.determinant(phi1[:, :nu], phi1[:, nu:])[sec]
        return TU @ np.linalg.inv(U)

    ev, Us = np.linalg.eigh(Hs)
    pb = Us @ (np.exp(-(ev - ev[0])) * (Us.conj().T @ psiT))
    exact = ((psiT.conj() @ Hs @ pb) / (psiT.conj() @ pb)).real
    errs = []
    for dt in (0.1, 0.05, 0.025):
        v = np.linalg.matrix_power(field_averaged_step(dt), int(round(1.0 / dt))) @ psiT
        errs.append(abs(((psiT.conj() @ Hs @ v) / (psiT.conj() @ v)).real - exact))
    assert 3.5 < errs[0] / errs[1] < 4.8 and 3.5 < errs[1] / errs[2] < 4.8
    assert errs[2] < 1e-3
