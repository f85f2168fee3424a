"""Multi-determinant trial evaluated relative to a reference determinant (the CPU oracle).

TEST INFRASTRUCTURE: the reference the GPU library's low-rank multi-determinant
walk is checked against.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark may import it; the GPU library never calls it.

Sec. 3.4 (Eqs. usesherman, precomputing, precomputing2, localenergy2,
localenergy3), with every determinant taken relative to the reference d = 0 as
the Sherman-Morrison-Woodbury remark there suggests for expansions about a
reference.  Psi_T = sum_d A_d Psi_d, Psi_d with spin-up and spin-down orbitals
V_du, V_dd (M x N, real); walkers closed shell (both spin blocks phi).

For spin s: S_0s = V_0s^T phi (invertible: the walkers keep a non-zero
overlap with the reference), Theta_0s = phi S_0s^-1, and for determinant d

    M_ds = V_ds^T Theta_0s,   so  det(V_ds^T phi) = det M_ds det S_0s.

For a one-body operator X (h or L_g) let Y_ds(X) = V_ds^T X Theta_0s and

    det(M_ds + eps Y_ds(X)) = r_ds + eps c1_ds(X) + eps^2 c2_ds(X) + O(eps^3),

r_ds = det M_ds.  With G_ds = phi (V_ds^T phi)^-1 V_ds^T the one-body Green's
function of determinant d (where it exists):

    r_ds Tr(X G_ds) = c1_ds(X),
    r_ds [Tr(X G_ds)^2 - Tr(X G_ds X G_ds)] = 2 c2_ds(X)

(the Taylor coefficients of det(I + eps M^-1 Y) times det M), and both sides
are polynomials in the entries of M and Y: no division by r_ds, so a
determinant with zero overlap contributes its finite limit.  The coefficients
are written out by multilinearity of the determinant in its rows:

    c1 = sum_i det(M with row i taken from Y),
    c2 = sum_{i<j} det(M with rows i and j taken from Y).

With z_d = A_d^* r_du r_dd and Z = sum_d z_d:

    <Psi_T|Psi> = det S_0u det S_0d Z,
    t_g = sum_d A_d^* [c1_du(L_g) r_dd + r_du c1_dd(L_g)] / Z          (Eq. precomputing2),
    E_loc = sum_d A_d^* [H0 r_du r_dd + c1_du(h) r_dd + r_du c1_dd(h)
            + sum_g (c2_du(L_g) r_dd + r_du c2_dd(L_g) + c1_du(L_g) c1_dd(L_g))] / Z,

the per-determinant expressions of oracle.multidet (Eqs. localenergy2/3 with
the 1/2 of Eq. bo_ham2) multiplied through by <Psi_d|Psi> / <Psi_0|Psi>.

Readings as in oracle.multidet: the mean-field background and the initial
walkers come from determinant 0 (c_g = Tr(L_g (P_0u + P_0d)), phi = V_0u),
E_T is the mixed local energy of the initial walkers; phaseless walk, no comb.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import afqmc, philox


class SMWSetup:
    """Once-per-run quantities (Secs. 2.3, 2.4, 3.4) for a trial taken relative to determinant 0."""

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
        self.phi0 = self.V[0, 0]
        ev0 = evaluate(self, self.phi0[None].astype(np.complex128), energy=True)
        self.E_T = float(ev0["E"].real[0])


def poly_coeffs(Mm, Y):
    """(r, c1, c2) of det(Mm + eps Y) by multilinearity in the rows; Mm, Y (..., N, N)."""
    N = Mm.shape[-1]
    r = np.linalg.det(Mm)
    c1 = np.zeros_like(r)
    for i in range(N):
        A = Mm.copy()
        A[..., i, :] = Y[..., i, :]
        c1 = c1 + np.linalg.det(A)
    c2 = np.zeros_like(r)
    for i, j in itertools.combinations(range(N), 2):
        A = Mm.copy()
        A[..., i, :] = Y[..., i, :]
        A[..., j, :] = Y[..., j, :]
        c2 = c2 + np.linalg.det(A)
    return r, c1, c2


def evaluate(st: SMWSetup, phi, energy=False):
    """Per walker: log <Psi_T|Psi> (complex, Im in (-pi, pi]), the force-bias
    traces t (W, nchol) and, if asked, the local energy E (W,)."""
    W = phi.shape[0]
    S0 = np.einsum("spi,wpj->wsij", st.V[0], phi)  # (W, 2, N, N)
    sgn, lab = np.linalg.slogdet(S0)
    th0 = np.einsum("wpj,wsjk->wspk", phi, np.linalg.inv(S0))  # Theta_0s (W, 2, M, N)
    Mm = np.einsum("dspi,wspk->wdsik", st.V, th0)  # M_ds (W, nd, 2, N, N)
    r = np.linalg.det(Mm)  # (W, nd, 2)
    Ac = np.conj(st.A)[None, :]
    Z = np.sum(Ac * r[:, :, 0] * r[:, :, 1], axis=1)  # (W,)
    logov = np.sum(lab + np.log(sgn.astype(np.complex128)), axis=1) + np.log(Z)
    logov = logov.real + 1j * afqmc.wrap_phase(logov.imag)
    # Y_ds(L_g) = V_ds^T L_g Theta_0s: (W, nd, 2, G, N, N)
    YL = np.einsum("dspi,gpq,wsqk->wdsgik", st.V, st.L, th0)
    Mg = np.broadcast_to(Mm[:, :, :, None], YL.shape)
    rL, c1L, c2L = poly_coeffs(Mg, YL)
    ru, rd = r[:, :, 0][..., None], r[:, :, 1][..., None]  # (W, nd, 1)
    t = np.sum(Ac[..., None] * (c1L[:, :, 0] * rd + ru * c1L[:, :, 1]), axis=1) / Z[:, None]
    out = {"logov": logov, "t": t, "r": r, "Z": Z}
    if energy:
        Yh = np.einsum("dspi,pq,wsqk->wdsik", st.V, st.h1, th0)
        _, c1h, _ = poly_coeffs(Mm, Yh)
        num = (st.H0 * r[:, :, 0] * r[:, :, 1] + c1h[:, :, 0] * r[:, :, 1] + r[:, :, 0] * c1h[:, :, 1]
               + np.sum(c2L[:, :, 0] * rd + ru * c2L[:, :, 1] + c1L[:, :, 0] * c1L[:, :, 1], axis=2))
        out["E"] = np.sum(Ac * num, axis=1) / Z
    return out


class SMWOracle:
    """A population of closed-shell walkers importance-sampled with a
    multi-determinant trial evaluated relative to determinant 0 (phaseless;
    the steps of oracle.afqmc.Oracle)."""

    def __init__(self, h1, L, coeffs, Vu, Vd, nwalkers, params: afqmc.Params | None = None,
                 H0=0.0):
        self.p = p = params or afqmc.Params()
        if p.mode != "phaseless" or p.pc_period:
            raise ValueError("the multi-determinant oracle walks phaseless, without the comb")
        self.setup = st = SMWSetup(h1, L, coeffs, Vu, Vd, H0, p.dt)
        self.W = int(nwalkers)
        self.phi = np.array(np.broadcast_to(st.phi0, (self.W, st.M, st.N)), np.complex128)
        ev = evaluate(st, self.phi)
        self.logdet, self.t = ev["logov"], ev["t"]
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
            xbar = -1j * sdt * (self.t[alive] - st.c)
            if p.fb_cap > 0:
                mag = np.abs(xbar)
                big = mag > p.fb_cap
                xbar = np.where(big, xbar * (p.fb_cap / np.where(big, mag, 1.0)), xbar)
            x = xi - xbar
            V = afqmc.assemble_V(st, x)
            phi_new = st.Bhalf @ afqmc.taylor(V, st.Bhalf @ phi, p.taylor_order)
            ev = evaluate(st, phi_new)
            logR = (ev["logov"] - self.logdet[alive] - p.dt * (st.H0p - self.e_shift)
                    - 1j * sdt * (x @ st.c))
            logI = logR + np.sum(xi * xbar, axis=1) - 0.5 * np.sum(xbar * xbar, axis=1)
            dtheta = afqmc.wrap_phase(logR.imag)
            w_new = self.weight[alive] * np.exp(logI.real) * np.maximum(0.0, np.cos(dtheta))
            w_new = np.minimum(w_new, self.wmax)
            bad = ~np.isfinite(w_new)
            self.nonfinite += int(np.count_nonzero(bad))
            w_new = np.where(bad, 0.0, w_new)
            self.phi[alive] = phi_new
            self.logdet[alive] = ev["logov"]
            self.t[alive] = ev["t"]
            self.weight[alive] = w_new
        self.step_count += 1
        n = self.step_count
        if p.qr_period and n % p.qr_period == 0:
            alive = np.nonzero(self.weight != 0)[0]
            if alive.size:
                self.phi[alive] = afqmc.mgs(self.phi[alive])
                ev = evaluate(st, self.phi[alive])
                self.logdet[alive] = ev["logov"]
                self.t[alive] = ev["t"]
        if p.energy_period and n % p.energy_period == 0:
            self.records.append((n,) + self.energy_sums())

    def run(self, nsteps):
        for _ in range(nsteps):
            self.step()
        return self

    def local_energies(self):
        return evaluate(self.setup, self.phi, energy=True)["E"]

    def energy_sums(self):
        alive = np.nonzero(self.weight != 0)[0]
        if alive.size == 0:
            return 0.0, 0.0
        e = evaluate(self.setup, self.phi[alive], energy=True)["E"].real
        if self.p.ecap_C > 0:
            half = math.sqrt(self.p.ecap_C / self.p.dt)
            e = np.clip(e, self.setup.E_T - half, self.setup.E_T + half)
        w = self.weight[alive]
        return float(np.sum(w * e)), float(np.sum(w))
