"""Phaseless AFQMC with a multi-determinant trial (the CPU oracle).

TEST INFRASTRUCTURE: the reference the GPU library's multi-determinant walk is
checked against.  Only tests, the smoke check and the CPU-baseline leg of the
benchmark may import it; the GPU library never calls it.

Sec. 3.4 ("Importance sampling with a multi-determinant trial", Eqs.
usesherman, precomputing, precomputing2, localenergy2, localenergy3): the trial
is Psi_T = sum_d A_d Psi_d, each Psi_d a determinant with its own spin-up and
spin-down orbitals V_du, V_dd (M x N, real, orthonormal columns).  Walkers stay
closed shell (both spin blocks the same M x N matrix phi): B(x) acts on both
spins alike, so the walk keeps them equal and the projection is unchanged; the
trial enters through

  * the overlap <Psi_T|Psi> = sum_d A_d^* det(V_du^T phi) det(V_dd^T phi),
  * the per-determinant Theta_ds = phi (V_ds^T phi)^-1 and weights
    w_d = A_d^* <Psi_d|Psi> / <Psi_T|Psi>,
  * the force bias trace t_g = sum_d w_d sum_s Tr(Lh_dsg Theta_ds)
    (Eq. precomputing2, Lh_dsg = V_ds^T L_g),
  * the local energy sum_d w_d E_d with, per determinant (Eq. localenergy3 with
    the 1/2 of Eq. bo_ham2),
      E_d = H0 + sum_s Tr(hh_ds Theta_ds)
            + 1/2 sum_g [(sum_s Tr(Lh_dsg Theta_ds))^2 - sum_s Tr(Lh_dsg Theta_ds Lh_dsg Theta_ds)],
    hh_ds = V_ds^T h.

Readings (the paper leaves them open):

  * the mean-field background uses the leading determinant d = 0:
    c_g = Tr(L_g (P_0u + P_0d)), P_0s = V_0s V_0s^T (any c_g keeps the
    Hamiltonian exact; Sec. 2.4).
  * the walkers start at phi = V_0u, and E_T is the mixed local energy there.
  * a determinant with det(V_ds^T phi) = 0 has weight 0 and no Theta.  This
    is the right limit only when H does not connect Psi_d to the walker; for a
    determinant orthogonal (or nearly so) to a walker, w_d E_d and w_d Tr(...)
    are 0/0 limits that this per-determinant evaluation does not resolve, so
    the method is meant for non-orthogonal determinants (e.g. different
    rotations of a reference), not for CI expansions about the walkers' own
    determinant.
  * every determinant is handled in full here; the evaluation relative to
    a reference determinant, which resolves those limits, is oracle.smw.

The walk itself (fields, propagation, phaseless weights, Gram-Schmidt, energy
records) follows oracle.afqmc.Oracle step for step.
"""
from __future__ import annotations

import math

import numpy as np

from . import afqmc, philox


class MultiDetSetup:
    """Once-per-run quantities for a multi-determinant trial (Secs. 2.3, 2.4, 3.4)."""

    def __init__(self, h1, L, coeffs, Vu, Vd, H0=0.0, dt=0.005):
        self.h1 = np.asarray(h1, np.float64)
        self.L = np.asarray(L, np.float64)
        self.A = np.asarray(coeffs, np.complex128)
        self.V = np.stack([np.asarray(Vu, np.float64), np.asarray(Vd, np.float64)], axis=1)
        self.nd = self.V.shape[0]  # (nd, 2, M, N)
        self.nchol, self.M, _ = self.L.shape
        self.N = self.V.shape[3]
        self.H0, self.dt = float(H0), float(dt)
        P = self.V[0, 0] @ self.V[0, 0].T + self.V[0, 1] @ self.V[0, 1].T
        self.c = np.einsum("gpq,qp->g", self.L, P)
        v0 = self.h1 - 0.5 * np.einsum("gpr,grq->pq", self.L, self.L)
        self.v0p = v0 + np.einsum("g,gpq->pq", self.c, self.L)
        self.H0p = self.H0 - 0.5 * float(np.sum(self.c ** 2))
        ev, U = np.linalg.eigh(-0.5 * self.dt * self.v0p)
        self.Bhalf = (U * np.exp(ev)) @ U.T
        # half-rotated vectors and one-body matrix per determinant and spin
        self.Lh = np.einsum("dspi,gpq->dsgiq", self.V, self.L)  # (nd, 2, G, N, M)
        self.hh = np.einsum("dspi,pq->dsiq", self.V, self.h1)  # (nd, 2, N, M)
        self.phi0 = self.V[0, 0]
        ld, th, w = overlap(self, self.phi0[None].astype(np.complex128))
        self.E_T = float(local_energy(self, th, w).real[0])


def overlap(st: MultiDetSetup, phi):
    """(log <Psi_T|Psi> (W,) complex with Im in (-pi, pi], Theta (W, nd, 2, M, N),
    determinant weights w_d = A_d^* <Psi_d|Psi> / <Psi_T|Psi> (W, nd))."""
    W = phi.shape[0]
    S = np.einsum("dspi,wpj->wdsij", st.V, phi)  # (W, nd, 2, N, N)
    sign, logabs = np.linalg.slogdet(S)  # (W, nd, 2)
    ok = np.all(sign != 0, axis=2)  # (W, nd)
    # log(A_d^* <Psi_d|Psi>) for the determinants with a non-zero overlap
    lo = np.where(ok, np.sum(logabs, axis=2), -np.inf) + 0j
    lo = lo + 1j * np.where(ok, np.angle(np.prod(np.where(ok[..., None], sign, 1.0), axis=2)), 0.0)
    lo = lo + np.log(np.conj(st.A))[None, :]
    ref = np.max(lo.real, axis=1)  # log-sum-exp in a fixed order of d
    terms = np.where(ok, np.exp(lo - ref[:, None]), 0.0)
    tot = np.sum(terms, axis=1)
    logov = ref + np.log(tot)
    logov = logov.real + 1j * afqmc.wrap_phase(logov.imag)
    w = terms / tot[:, None]
    theta = np.zeros((W, st.nd, 2, st.M, st.N), np.complex128)
    for wi in range(W):
        for d in range(st.nd):
            if ok[wi, d]:
                for s in range(2):
                    theta[wi, d, s] = phi[wi] @ np.linalg.inv(S[wi, d, s])
    return logov, theta, w


def force_bias_trace(st: MultiDetSetup, theta, w):
    """t_g = sum_d w_d sum_s Tr(Lh_dsg Theta_ds) (Eq. precomputing2), (W, nchol)."""
    tr = np.einsum("dsgiq,wdsqi->wdg", st.Lh, theta)
    return np.einsum("wd,wdg->wg", w, tr)


def local_energy(st: MultiDetSetup, theta, w):
    """<Psi_T|H|Psi>/<Psi_T|Psi> per walker: sum_d w_d E_d (Eqs. localenergy2/3)."""
    W = theta.shape[0]
    N, M, G = st.N, st.M, st.nchol
    e1 = np.einsum("dsiq,wdsqi->wd", st.hh, theta)
    tr = np.einsum("dsgiq,wdsqi->wdsg", st.Lh, theta)
    coul = 0.5 * np.sum(np.sum(tr, axis=2) ** 2, axis=2)
    exch = np.zeros((W, st.nd), np.complex128)
    for wi in range(W):
        for d in range(st.nd):
            if w[wi, d] == 0:
                continue
            for s in range(2):
                Lh2 = st.Lh[d, s].reshape(G * N, M)
                T = (Lh2 @ theta[wi, d, s]).reshape(G, N, N)
                exch[wi, d] += np.einsum("gij,gji->", T, T)
    Ed = st.H0 + e1 + coul - 0.5 * exch
    return np.sum(w * Ed, axis=1)


class MultiDetOracle:
    """A population of closed-shell walkers importance-sampled with a
    multi-determinant trial (phaseless; the steps of oracle.afqmc.Oracle)."""

    def __init__(self, h1, L, coeffs, Vu, Vd, nwalkers, params: afqmc.Params | None = None,
                 H0=0.0):
        self.p = p = params or afqmc.Params()
        if p.mode != "phaseless" or p.pc_period:
            raise ValueError("the multi-determinant oracle walks phaseless, without the comb")
        self.setup = st = MultiDetSetup(h1, L, coeffs, Vu, Vd, H0, p.dt)
        self.W = int(nwalkers)
        self.phi = np.array(np.broadcast_to(st.phi0, (self.W, st.M, st.N)), np.complex128)
        self.logdet, self.theta, self.wd = overlap(st, self.phi)
        self.weight = np.ones(self.W)
        self.step_count = 0
        self.e_shift = st.E_T if math.isnan(p.e_shift) else float(p.e_shift)
        self.wmax = max(100.0, self.W / 10.0) if math.isnan(p.wmax) else float(p.wmax)
        self.records = []
        self.nonfinite = 0

    def step(self):
        st, p = self.setup, self.p
        k = self.step_count
        sdt = math.sqrt(p.dt)
        alive = np.nonzero(self.weight != 0)[0]
        if alive.size:
            phi = self.phi[alive]
            xi = philox.gaussian_fields(p.seed, k, alive, st.nchol)
            t = force_bias_trace(st, self.theta[alive], self.wd[alive])
            xbar = -1j * sdt * (t - st.c)
            if p.fb_cap > 0:
                mag = np.abs(xbar)
                big = mag > p.fb_cap
                xbar = np.where(big, xbar * (p.fb_cap / np.where(big, mag, 1.0)), xbar)
            x = xi - xbar
            V = afqmc.assemble_V(st, x)
            phi_new = st.Bhalf @ afqmc.taylor(V, st.Bhalf @ phi, p.taylor_order)
            logdet_new, theta_new, wd_new = overlap(st, phi_new)
            logR = (logdet_new - self.logdet[alive] - p.dt * (st.H0p - self.e_shift)
                    - 1j * sdt * (x @ st.c))
            logI = logR + np.sum(xi * xbar, axis=1) - 0.5 * np.sum(xbar * xbar, axis=1)
            dtheta = afqmc.wrap_phase(logR.imag)
            w_new = self.weight[alive] * np.exp(logI.real) * np.maximum(0.0, np.cos(dtheta))
            w_new = np.minimum(w_new, self.wmax)
            bad = ~np.isfinite(w_new)
            self.nonfinite += int(np.count_nonzero(bad))
            w_new = np.where(bad, 0.0, w_new)
            self.phi[alive] = phi_new
            self.logdet[alive] = logdet_new
            self.theta[alive] = theta_new
            self.wd[alive] = wd_new
            self.weight[alive] = w_new
        self.step_count += 1
        n = self.step_count
        if p.qr_period and n % p.qr_period == 0:
            alive = np.nonzero(self.weight != 0)[0]
            if alive.size:
                self.phi[alive] = afqmc.mgs(self.phi[alive])
                ld, th, wd = overlap(st, self.phi[alive])
                self.logdet[alive] = ld
                self.theta[alive] = th
                self.wd[alive] = wd
        if p.energy_period and n % p.energy_period == 0:
            self.records.append((n,) + self.energy_sums())

    def run(self, nsteps):
        for _ in range(nsteps):
            self.step()
        return self

    def local_energies(self):
        return local_energy(self.setup, self.theta, self.wd)

    def energy_sums(self):
        alive = np.nonzero(self.weight != 0)[0]
        if alive.size == 0:
            return 0.0, 0.0
        e = local_energy(self.setup, self.theta[alive], self.wd[alive]).real
        if self.p.ecap_C > 0:
            half = math.sqrt(self.p.ecap_C / self.p.dt)
            e = np.clip(e, self.setup.E_T - half, self.setup.E_T + half)
        w = self.weight[alive]
        return float(np.sum(w * e)), float(np.sum(w))
