"""Pins of the oracle's back-propagation (Sec. "Computing ground-state
properties: the backpropagation algorithm", Eqs. bp1, bp, bp_dets).

The one-body density between two determinants is checked in the full Fock
space; the back-propagated determinant against the adjoint identity
<Phi_m|Psi_n> = <Psi_T|B(x_{n+m-1}) ... B(x_n)|Psi_n>, which fails for a wrong
order, a missing conjugation or a wrong sign of the fields; a window of no steps
against the mixed estimator; and free-projection back-propagation (no
constraint, Eq. bp exact up to the Trotter error) against the exact
<Psi_T|e^{-m dt H} rho e^{-n dt H}|Psi_T> / <Psi_T|e^{-(m+n) dt H}|Psi_T> from
exact diagonalisation.
"""
import math

import numpy as np
import pytest

import workloads
from fock import Fock, eri_from_cholesky
from oracle import afqmc, scf


def small_system(M=4, G=8, seed=77, scale=0.6, N=2):
    h1, L, _ = workloads.hamiltonian(M, G, seed)
    L = L * scale
    C, e, conv, _ = scf.rhf(h1, L, N)
    assert conv
    return h1, L, C


def test_one_body_density_matches_fock_space():
    M, N = 4, 2
    rng = np.random.default_rng(5)
    phi = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    psi = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    F = Fock(M)
    bra, ket = F.determinant(phi), F.determinant(psi)
    rho = afqmc.one_body_density(phi[None], psi[None])[0]
    for p in range(M):
        for q in range(M):
            E = np.zeros((M, M))
            E[p, q] = 1.0
            want = (bra.conj() @ (F.one_body(E) @ ket)) / (bra.conj() @ ket)
            assert abs(rho[p, q] - want) < 1e-12 * max(1.0, abs(want)), (p, q)


def test_back_propagated_determinant_is_the_adjoint():
    h1, L, C = small_system()
    o = afqmc.Oracle(h1, L, C, 8, afqmc.Params(dt=0.02, seed=11, qr_period=5))
    o.run(3)
    o.bp_begin()
    rec = o.bp
    o.run(7)  # crosses a Gram-Schmidt step
    *_, phi_m = o.bp_end()
    st = o.setup
    fwd = rec["psi_n"].copy()
    for x in rec["fields"]:
        fwd = st.Bhalf @ afqmc.taylor(afqmc.assemble_V(st, x), st.Bhalf @ fwd, 6)
    lhs = np.linalg.det(np.conj(np.swapaxes(phi_m, 1, 2)) @ rec["psi_n"])
    rhs = np.linalg.det(np.einsum("pi,wpj->wij", st.VT, fwd))
    assert np.max(np.abs(lhs - rhs) / np.abs(rhs)) < 1e-11
    # the same with the fields' sign or conjugation wrong does not hold
    bad = np.array(np.broadcast_to(st.VT, phi_m.shape), np.complex128)
    for x in reversed(rec["fields"]):
        bad = st.Bhalf @ afqmc.taylor(afqmc.assemble_V(st, np.conj(x)), st.Bhalf @ bad, 6)
    lbad = np.linalg.det(np.conj(np.swapaxes(bad, 1, 2)) @ rec["psi_n"])
    assert np.min(np.abs(lbad - rhs) / np.abs(rhs)) > 1e-4


def test_empty_window_is_the_mixed_estimator():
    h1, L, C = small_system()
    o = afqmc.Oracle(h1, L, C, 16, afqmc.Params(dt=0.02, seed=2))
    o.run(4)
    o.bp_begin()
    rho_pres, rho_phl, wp, w, _ = o.bp_end()
    VT = o.setup.VT
    mixed = 2.0 * np.swapaxes(o.theta @ VT.T, 1, 2)  # <Psi_T|a+_p a_q|Psi>/<Psi_T|Psi>
    want = np.einsum("w,wpq->pq", o.weight, mixed) / np.sum(o.weight)
    assert np.max(np.abs(rho_phl - want)) < 1e-12
    assert np.max(np.abs(rho_pres - want)) < 1e-12 and abs(wp - w) < 1e-13 * abs(w)
    # trace = number of electrons, for any pair of determinants
    assert abs(np.trace(rho_phl) - 2 * C.shape[1]) < 1e-12


def test_path_restoration_factor_of_one_step():
    """Over a one-step window the BP-PRes weight is W_{n+1} exp(-i dt Im E_loc)
    / cos(dtheta): it restores the phase and undoes the projection of that step."""
    h1, L, C = small_system()
    p = afqmc.Params(dt=0.02, seed=8, qr_period=0)
    o = afqmc.Oracle(h1, L, C, 6, p)
    o.run(2)
    ld0 = o.logdet.copy()
    o.bp_begin()
    rec = o.bp
    o.step()
    _, _, wp, w, _ = o.bp_end()
    st = o.setup
    x = rec["fields"][0]
    sdt = math.sqrt(p.dt)
    logR = o.logdet - ld0 - p.dt * (st.H0p - o.e_shift) - 1j * sdt * (x @ st.c)
    cosd = np.cos(afqmc.wrap_phase(logR.imag))
    e = afqmc.local_energy(st, o.theta)
    keep = o.weight > 0
    want = np.sum((o.weight * np.exp(-1j * p.dt * e.imag) / np.where(keep, cosd, 1.0))[keep])
    assert abs(wp - want) < 1e-12 * abs(want)


@pytest.fixture(scope="module")
def fci_bp():
    h1, L, C = small_system(M=4, G=8, N=2)
    F = Fock(4)
    H = F.hamiltonian(h1, eri_from_cholesky(L)).toarray()
    sec = F.number_sector(2, 2)
    Hs = H[np.ix_(sec, sec)]
    psiT = F.determinant(C)[sec]
    ev, U = np.linalg.eigh(Hs)

    def prop(beta, v):
        return (U * np.exp(-beta * (ev - ev[0]))) @ (U.conj().T @ v)

    def rho_bp(beta_n, beta_m):
        right = prop(beta_n, psiT)
        left = prop(beta_m, psiT)
        den = left.conj() @ right
        out = np.zeros((4, 4), np.complex128)
        for p in range(4):
            for q in range(4):
                E = np.zeros((4, 4))
                E[p, q] = 1.0
                op = F.one_body(E).toarray()[np.ix_(sec, sec)]
                out[p, q] = (left.conj() @ (op @ right)) / den
        return out

    return h1, L, C, rho_bp


def test_free_projection_back_propagation_is_exact(fci_bp):
    """Without a constraint, Eq. bp estimates the exact finite-(n, m) ratio."""
    h1, L, C, rho_bp = fci_bp
    W, dt, n, m = 4000, 0.01, 60, 40
    p = afqmc.Params(dt=dt, seed=5, mode="free", qr_period=5, energy_period=0,
                     ecap_C=-1, fb_cap=-1, wmax=1e300)
    o = afqmc.Oracle(h1, L, C, W, p).run(n)
    o.bp_begin()
    rec = o.bp
    o.run(m)
    psi_n = rec["psi_n"]
    *_, phi_m = o.bp_end()
    rho_w = afqmc.one_body_density(phi_m, psi_n)
    w = o.weight
    est = np.einsum("w,wpq->pq", w, rho_w) / np.sum(w)
    groups = np.array_split(np.arange(W), 20)
    sub = np.array([np.einsum("w,wpq->pq", w[g], rho_w[g]) / np.sum(w[g]) for g in groups])
    err = np.std(sub.real, axis=0) / math.sqrt(len(groups))
    exact = rho_bp(n * dt, m * dt)
    assert np.max(np.abs(exact.imag)) < 1e-10
    z = np.abs(est.real - exact.real) / (err + 1e-4)
    assert z.max() < 4.0, (z.max(), est.real, exact.real)
    # the back-propagated density is not the mixed one: the test can tell
    mixed = rho_bp(n * dt + m * dt, 0.0)
    assert np.max(np.abs(mixed.real - exact.real) / (err + 1e-4)) > 8.0


def test_comb_inside_the_window_keeps_each_path_whole():
    """With population control inside the window every copy carries its
    parent's Psi_n and fields: propagating the recorded Psi_n with the recorded
    fields gives the walker's current orbitals (same Theta = Phi S^-1, which
    the Gram-Schmidt steps leave unchanged)."""
    h1, L, C = small_system()
    o = afqmc.Oracle(h1, L, C, 16, afqmc.Params(dt=0.02, seed=12, qr_period=4, pc_period=3))
    o.run(2)
    o.bp_begin()
    rec = o.bp
    o.run(8)  # two combs (steps 3, 6, 9) inside the window
    st = o.setup
    fwd = rec["psi_n"].copy()
    for x in rec["fields"]:
        fwd = st.Bhalf @ afqmc.taylor(afqmc.assemble_V(st, x), st.Bhalf @ fwd, 6)
    _, th_fwd = afqmc.overlap(st, fwd)
    assert np.max(np.abs(th_fwd - o.theta)) < 1e-10 * np.max(np.abs(o.theta))
    rho, phl, wp, w, _ = o.bp_end()
    assert abs(np.trace(phl) - 2 * C.shape[1]) < 1e-10
