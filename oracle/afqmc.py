"""Plain FP64 phaseless AFQMC for a closed-shell molecule (the CPU oracle).

TEST INFRASTRUCTURE: this module is the reference the GPU library is checked
against.  Only tests, the smoke check and the CPU-baseline leg of the
benchmark may import it; the GPU library never calls it.

Everything is float64 / complex128 numpy, batched over walkers only where the
walkers are independent (Sec. 3.5, step 7 of the algorithm outline), and
follows the paper's order of operations.  Notation (Motta & Zhang 2017):

  M orbitals, N electrons per spin (closed shell, N_up = N_dn = N).
  Walker |Psi> is a Slater determinant; both spin blocks are the same M x N
  matrix phi because the trial is RHF and B(x) is spin independent (the
  one-body operators v_g of Sec. 2.3 act identically on both spins), so one
  block is propagated and every spin sum is a factor 2.
  Two spin blocks (a trial with different spin-up and spin-down orbitals,
  N_up != N_dn allowed; Theorem 1.1 takes the product over sigma): phi holds
  the N_up spin-up columns followed by the N_dn spin-down ones, B(x) acts on
  all of them alike, and every determinant, inverse, Gram-Schmidt sweep and
  exchange trace is taken per block; each spin sum then has its two terms
  instead of a factor 2.
  Trial V_T (M x N, real, orthonormal columns); P = V_T V_T^T.
  S = V_T^T phi, Theta = phi S^-1 (Sec. 3.4, Eq. precomputing), the overlap
  <Psi_T|Psi> = det(S)^2 (Theorem 1.1).
  Half-rotated Cholesky vectors Lh_g = V_T^T L_g (N x M, Eq. precomputing2),
  hh = V_T^T h.

Readings of the paper taken here (each also listed in the design notes):

  * mean-field background (Sec. 2.4): vbar_g = <v_g>_T = i c_g with
    c_g = 2 Tr(L_g P); v0' = h - 1/2 sum_g L_g^2 + sum_g c_g L_g (Eq. mcd1
    plus the shift); H0' = H0 - 1/2 sum_g c_g^2.
  * force bias (Eq. fb with v' = v - vbar):
    xbar_g = -sqrt(dt) <v'_g>_m = -i sqrt(dt) (t_g - c_g),
    t_g = 2 Tr(Lh_g Theta) (Eq. precomputing2 for one determinant);
    capped in magnitude, |xbar_g| <= fb_cap, phase kept (Appendix B).
  * propagation (Eqs. primitive, hs2, weight_update_2): with xi ~ N(0,1) and
    x = xi - xbar, phi <- B_half T_n(V) B_half phi, B_half = exp(-dt v0'/2),
    V = i sqrt(dt) sum_g x_g L_g, T_n the Taylor series truncated at order n
    (Sec. 3.4.2).  The remaining scalar of B(x - xbar) is
    exp(-dt (H0' - E_T) - i sqrt(dt) sum_g x_g c_g).
  * hybrid importance function (Eq. hybrid-wt):
    I = R exp(sum_g xi_g xbar_g - 1/2 sum_g xbar_g^2), with the overlap ratio
    R = <Psi_T|Psi'>/<Psi_T|Psi> including that scalar.
  * phaseless projection (Eq. if_rle, weight_update_2):
    W <- W |I| max(0, cos dtheta), dtheta = Arg R; then W <- min(W, W_max)
    (Appendix B).  theta is kept at 0.
  * local energy (Eqs. localenergy2/localenergy3, with the 1/2 of H_2 in
    Eq. bo_ham2 restored):
    E_loc = H0 + 2 Tr(hh Theta) + 1/2 sum_g t_g^2 - sum_g Tr(Lh_g Theta Lh_g Theta),
    Re E_loc clamped to E_T +- sqrt(C/dt) in the estimator (Eq. cap).
  * modified Gram-Schmidt (Sec. 3.4.5) every qr_period steps, then the
    overlap, log det and Theta are recomputed from the new orbitals.
  * population control (Sec. 3.4.4, scheme not given in the paper): a
    fixed-size comb, see ``comb``.
  * dead walkers (W = 0) are skipped (algorithm outline, step 2).
  * back-propagation (Sec. "Computing ground-state properties", Eqs. bp1,
    Bprod-bp, bp, bp_dets): a window opened at step n keeps Psi_n and the
    shifted fields x = xi - xbar of every later step; at step n + m,
    Phi_m = B^+(x_n) ... B^+(x_{n+m-1}) Psi_T with B(x)^+ = B(-conj(x)); the
    denominator <Psi_{m,w}|Psi_{n,w}> printed in Eq. bp reads
    <Phi_{m,w}|Psi_{n,w}>.  BP-PRes multiplies W_{n+m} by, per step k of the
    window, exp(-i dt Im E_loc(Psi_k)) / max(0, cos dtheta_k) (0 where the
    projection zeroed the walker; the weight cap is not undone).  The comb
    gives each copy its parent's path (Psi_n, fields, factor).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import philox

_NAN = float("nan")


@dataclasses.dataclass
class Params:
    dt: float = 0.005
    taylor_order: int = 6
    qr_period: int = 5
    pc_period: int = 0
    energy_period: int = 1
    seed: int = 1
    e_shift: float = _NAN  # NaN -> E_T
    ecap_C: float = 2.0  # <= 0 disables the local-energy cap
    fb_cap: float = 1.0  # <= 0 disables the force-bias cap
    wmax: float = _NAN  # NaN -> max(100, nwalkers/10)
    # "phaseless": Eq. weight_update_2 (the method).
    # "free": free projection, Eq. weight_update (complex weights, no bias).
    # "complex_is": importance sampling with the force bias and complex
    #               weights W <- W I, no phaseless projection (exact).
    mode: str = "phaseless"
    # global index of walker 0: walker w draws the fields of walker walker0 + w
    # (a population split over several oracles)
    walker0: int = 0


def wrap_phase(a):
    """Map angles to (-pi, pi]."""
    a = np.asarray(a, dtype=np.float64)
    w = np.mod(a + math.pi, 2.0 * math.pi) - math.pi
    return np.where(w == -math.pi, math.pi, w)


class Setup:
    """Once-per-run quantities built from (h, L, V_T) (Secs. 2.3, 2.4, 3.4).

    trial: the RHF orbitals (both spins), or with trial_dn given the spin-up
    orbitals, trial_dn the spin-down ones (two spin blocks).  `blocks` lists
    (first column, end column, trial orbitals) per block and `sf` is the
    number of spins each block stands for (2 closed shell, 1 otherwise)."""

    def __init__(self, h1, L, trial, H0=0.0, dt=0.005, trial_dn=None):
        h1 = np.asarray(h1, np.float64)
        L = np.asarray(L, np.float64)
        Vu = np.asarray(trial, np.float64)
        if trial_dn is None:
            VT = Vu
            self.blocks = [(0, Vu.shape[1], Vu)]
            self.sf = 2.0
        else:
            Vd = np.asarray(trial_dn, np.float64)
            VT = np.concatenate([Vu, Vd], axis=1)
            self.blocks = [(0, Vu.shape[1], Vu), (Vu.shape[1], VT.shape[1], Vd)]
            self.sf = 1.0
        self.h1, self.L, self.VT, self.H0, self.dt = h1, L, VT, float(H0), float(dt)
        self.nchol, self.M, _ = L.shape
        self.N = VT.shape[1]
        # P = sum over spins of the trial's density V_sigma V_sigma^T
        P = self.sf * (VT @ VT.T)
        # c_g = Tr(L_g P): the trial expectation of v_g is i c_g (Sec. 2.4).
        self.c = np.einsum("gpq,qp->g", L, P)
        # v0 = h - 1/2 sum_g L_g L_g (Eq. mcd1 with v_prrq = sum_g (L_g L_g)_pq)
        v0 = h1 - 0.5 * np.einsum("gpr,grq->pq", L, L)
        # v0' = v0 - sum_g vbar_g v_g = v0 + sum_g c_g L_g (mean-field shift)
        self.v0p = v0 + np.einsum("g,gpq->pq", self.c, L)
        # H0' = H0 + 1/2 sum_g vbar_g^2 = H0 - 1/2 sum_g c_g^2
        self.H0p = self.H0 - 0.5 * float(np.sum(self.c ** 2))
        # B_half = exp(-dt v0'/2) by the symmetric eigendecomposition
        ev, U = np.linalg.eigh(-0.5 * self.dt * self.v0p)
        self.Bhalf = (U * np.exp(ev)) @ U.T
        # half-rotated Cholesky vectors and one-body matrix (Eq. precomputing2)
        self.Lh = np.einsum("pi,gpq->giq", VT, L)  # (nchol, N, M)
        self.hh = VT.T @ h1  # (N, M)
        self.E_T = float(local_energy(self, VT[None].astype(np.complex128)).real[0])


def overlap(setup: Setup, phi):
    """Per spin block S = V_T^T phi, Theta = phi S^-1, and
    log <Psi_T|Psi> = sum_sigma log det S_sigma (Theorem 1.1): 2 log det S
    for the closed-shell block.

    Returns (logdet (W,) complex with Im wrapped to (-pi, pi], Theta (W,M,N)).
    """
    theta = np.empty(phi.shape, np.complex128)
    la = 0.0
    ph = 0.0
    for a, b, V in setup.blocks:
        S = np.einsum("pi,wpj->wij", V, phi[:, :, a:b])
        sign, logabs = np.linalg.slogdet(S)
        la = la + setup.sf * logabs
        ph = ph + setup.sf * np.angle(sign)
        theta[:, :, a:b] = phi[:, :, a:b] @ np.linalg.inv(S)
    logdet = la + 1j * wrap_phase(ph)
    return logdet, theta


def force_bias_trace(setup: Setup, theta):
    """t_g = sum_sigma Tr(Lh_g,sigma Theta_sigma), shape (W, nchol): 2 Tr(Lh_g Theta)
    for the closed-shell block, the sum of the two blocks' traces otherwise."""
    return setup.sf * np.einsum("giq,wqi->wg", setup.Lh, theta)


def local_energy(setup: Setup, theta):
    """Mixed local energy <Psi_T|H|Psi>/<Psi_T|Psi> per walker (complex):
    H0 + sum_sigma Tr(hh_sigma Theta_sigma)
       + 1/2 sum_g [t_g^2 - sum_sigma Tr(T_g,sigma T_g,sigma)],
    T_g,sigma = Lh_g,sigma Theta_sigma (same-spin blocks only)."""
    W = theta.shape[0]
    e1 = setup.sf * np.einsum("iq,wqi->w", setup.hh, theta)
    t = force_bias_trace(setup, theta)
    exch = np.zeros(W, np.complex128)
    for a, b, _ in setup.blocks:
        n = b - a
        Lh2 = setup.Lh[:, a:b, :].reshape(setup.nchol * n, setup.M)
        for w in range(W):
            T = (Lh2 @ theta[w][:, a:b]).reshape(setup.nchol, n, n)  # T_g = Lh_g Theta
            exch[w] += 0.5 * setup.sf * np.einsum("gij,gji->", T, T)
    return setup.H0 + e1 + 0.5 * np.sum(t * t, axis=1) - exch


def assemble_V(setup: Setup, x):
    """V = i sqrt(dt) sum_g x_g L_g per walker, complex symmetric (W, M, M)."""
    Lf = setup.L.reshape(setup.nchol, -1)
    s = math.sqrt(setup.dt)
    re = x.real @ Lf
    im = x.imag @ Lf
    V = (1j * s) * (re + 1j * im)
    return V.reshape(-1, setup.M, setup.M)


def taylor(V, phi, order):
    """sum_{k=0}^{order} V^k phi / k! (Sec. 3.4.2, truncated Taylor series)."""
    term = phi.copy()
    acc = phi.copy()
    for k in range(1, order + 1):
        term = (V @ term) / k
        acc = acc + term
    return acc


def mgs(phi, blocks=None):
    """Modified Gram-Schmidt over the orbital columns (Sec. 3.4.5).

    Column k is orthogonalised against the already-finished columns one at a
    time (each projection uses the partially updated vector), then scaled to
    unit norm: u_k <- u_k - <u'_j|u_k> u'_j for j < k; u'_k = u_k/|u_k|.
    With spin blocks (a list of (first, end, ...) column ranges) each block is
    swept on its own: a spin-down orbital is never projected on a spin-up one.
    """
    q = phi.copy()
    N = q.shape[2]
    starts = [0] * N
    for blk in blocks or [(0, N)]:
        for k in range(blk[0], blk[1]):
            starts[k] = blk[0]
    for k in range(N):
        v = q[:, :, k]
        for j in range(starts[k], k):
            proj = np.einsum("wp,wp->w", q[:, :, j].conj(), v)
            v = v - proj[:, None] * q[:, :, j]
        nrm = np.sqrt(np.einsum("wp,wp->w", v.conj(), v).real)
        q[:, :, k] = v / nrm[:, None]
    return q


def comb(weights, u):
    """Fixed-size comb population control (Sec. 3.4.4; the scheme is ours).

    W_tot and the cumulative weights C_j are sequential float64 sums in
    walker order.  Tooth k (k = 0..N_w-1) sits at ((k + u) * W_tot) / N_w and
    is owned by the walker j with C_{j-1} <= tooth < C_j.  New slot k takes a
    copy of walker j (copies therefore appear in walker-index order) and every
    new weight is W_tot / N_w.  A tooth at or beyond C_{N_w-1} (rounding)
    goes to the last walker with positive weight.

    Returns (parent index per new slot, new weight) or (None, 0) when the
    population has no weight left.
    """
    w = np.asarray(weights, np.float64)
    n = w.size
    cum = np.add.accumulate(w)  # sequential prefix sums
    wtot = float(cum[-1])
    if not (wtot > 0.0) or not math.isfinite(wtot):
        return None, 0.0
    k = np.arange(n, dtype=np.float64)
    teeth = ((k + u) * wtot) / n
    parent = np.searchsorted(cum, teeth, side="right")
    last_alive = int(np.nonzero(w > 0.0)[0][-1])
    parent = np.where(parent >= n, last_alive, parent)
    return parent, wtot / n


def one_body_density(phi_bra, psi, setup: Setup | None = None):
    """Spin-summed one-body density <Phi|a+_p a_q|Psi>/<Phi|Psi> between
    determinants, per walker: rho_pq = sum_sigma [Psi_s (Phi_s^H Psi_s)^-1
    Phi_s^H]_qp, shape (W, M, M); for closed-shell determinants (both spin
    blocks the same M x N matrix) 2 [Psi (Phi^H Psi)^-1 Phi^H]_qp."""
    blocks = setup.blocks if setup is not None else [(0, psi.shape[2], None)]
    sf = setup.sf if setup is not None else 2.0
    rho = 0.0
    for a, b, _ in blocks:
        bra = np.conj(np.swapaxes(phi_bra[:, :, a:b], 1, 2))
        S = bra @ psi[:, :, a:b]  # Phi^H Psi, (W, n, n)
        G = psi[:, :, a:b] @ np.linalg.inv(S) @ bra  # (W, M, M)
        rho = rho + sf * np.swapaxes(G, 1, 2)
    return rho


class Oracle:
    """A population of walkers stepped by the phaseless AFQMC algorithm."""

    def __init__(self, h1, L, trial, nwalkers, params: Params | None = None,
                 H0=0.0, phi0=None, trial_dn=None):
        self.p = p = params or Params()
        self.setup = Setup(h1, L, trial, H0, p.dt, trial_dn=trial_dn)
        st = self.setup
        self.W = int(nwalkers)
        if phi0 is None:
            phi0 = st.VT
        phi0 = np.asarray(phi0, np.complex128)
        if phi0.ndim == 2:
            phi0 = np.broadcast_to(phi0, (self.W, st.M, st.N))
        self.phi = np.array(phi0, np.complex128)
        self.logdet, self.theta = overlap(st, self.phi)
        complex_w = p.mode in ("free", "complex_is")
        self.weight = np.ones(self.W, np.complex128 if complex_w else np.float64)
        self.step_count = 0
        self.e_shift = st.E_T if math.isnan(p.e_shift) else float(p.e_shift)
        self.wmax = max(100.0, self.W / 10.0) if math.isnan(p.wmax) else float(p.wmax)
        self.records = []  # (step, sum W Re E_loc, sum W)
        self.nonfinite = 0
        self.bp = None  # back-propagation window (bp_begin .. bp_end)

    # --- one step of the random walk (algorithm outline, steps 2-7) -------
    def step(self):
        st, p = self.setup, self.p
        k = self.step_count
        sdt = math.sqrt(p.dt)
        alive = np.nonzero(self.weight != 0)[0]
        if alive.size:
            phi = self.phi[alive]
            theta = self.theta[alive]
            xi = philox.gaussian_fields(p.seed, k, alive + p.walker0, st.nchol)
            if p.mode == "free":
                xbar = np.zeros((alive.size, st.nchol), np.complex128)
            else:
                t = force_bias_trace(st, theta)
                xbar = -1j * sdt * (t - st.c)
                if p.fb_cap > 0 and p.mode == "phaseless":
                    mag = np.abs(xbar)
                    big = mag > p.fb_cap
                    xbar = np.where(big, xbar * (p.fb_cap / np.where(big, mag, 1.0)), xbar)
            x = xi - xbar
            V = assemble_V(st, x)
            phi_new = st.Bhalf @ taylor(V, st.Bhalf @ phi, p.taylor_order)
            logdet_new, theta_new = overlap(st, phi_new)
            logR = (logdet_new - self.logdet[alive] - p.dt * (st.H0p - self.e_shift)
                    - 1j * sdt * (x @ st.c))
            logI = logR + np.sum(xi * xbar, axis=1) - 0.5 * np.sum(xbar * xbar, axis=1)
            w_old = self.weight[alive]
            if p.mode == "phaseless":
                dtheta = wrap_phase(logR.imag)
                w_new = w_old * np.exp(logI.real) * np.maximum(0.0, np.cos(dtheta))
                w_new = np.minimum(w_new, self.wmax)
            elif p.mode == "free":
                w_new = w_old * np.exp(logR)
            else:
                w_new = w_old * np.exp(logI)
            bad = ~np.isfinite(w_new)
            self.nonfinite += int(np.count_nonzero(bad))
            w_new = np.where(bad, 0.0, w_new)
            self.phi[alive] = phi_new
            self.logdet[alive] = logdet_new
            self.theta[alive] = theta_new
            self.weight[alive] = w_new
            if self.bp is not None:
                xs = np.zeros((self.W, st.nchol), np.complex128)
                xs[alive] = x
                self.bp["fields"].append(xs)
                if p.mode == "phaseless":
                    # path restoration (BP-PRes): give back the phase of the
                    # importance function, exp(-i dt Im E_loc(Psi_k)), and undo
                    # the cosine projection of this step
                    e_new = local_energy(st, theta_new)
                    cosd = np.cos(dtheta)
                    keep = (cosd > 0.0) & ~bad
                    f = np.where(keep, np.exp(-1j * p.dt * e_new.imag)
                                 / np.where(keep, cosd, 1.0), 0.0)
                    self.bp["factor"][alive] *= f
        elif self.bp is not None:
            self.bp["fields"].append(np.zeros((self.W, st.nchol), np.complex128))
        self.step_count += 1
        n = self.step_count
        if p.qr_period and n % p.qr_period == 0:
            self.orthonormalize()
        if p.pc_period and n % p.pc_period == 0:
            self.population_control(k)
        if p.energy_period and n % p.energy_period == 0:
            self.records.append((n,) + self.energy_sums())

    def run(self, nsteps):
        for _ in range(nsteps):
            self.step()
        return self

    def orthonormalize(self):
        alive = np.nonzero(self.weight != 0)[0]
        if alive.size:
            self.phi[alive] = mgs(self.phi[alive], self.setup.blocks)
            ld, th = overlap(self.setup, self.phi[alive])
            self.logdet[alive] = ld
            self.theta[alive] = th

    def population_control(self, step):
        if self.p.mode != "phaseless":
            raise ValueError("the comb acts on real weights")
        u = philox.comb_uniform(self.p.seed, step)
        parent, wnew = comb(self.weight, u)
        if parent is None:
            return
        self.phi = self.phi[parent].copy()
        self.logdet = self.logdet[parent].copy()
        self.theta = self.theta[parent].copy()
        self.weight = np.full(self.W, wnew)
        if self.bp is not None:
            # a copy carries its parent's path: Psi_n, fields and restoration factor
            self.bp["psi_n"] = self.bp["psi_n"][parent].copy()
            self.bp["factor"] = self.bp["factor"][parent].copy()
            self.bp["fields"] = [f[parent].copy() for f in self.bp["fields"]]

    # --- back-propagation (Sec. "Computing ground-state properties") --------
    def bp_begin(self):
        """Open a back-propagation window at the current step n: keep Psi_n of
        every walker and, at every later step, the shifted fields x - xbar that
        built B (Eq. bp_dets) and the BP-PRes factor of the weight; a comb
        inside the window copies these with the walkers."""
        self.bp = {"psi_n": self.phi.copy(), "fields": [],
                   "factor": np.ones(self.W, np.complex128)}

    def bp_end(self):
        """Close the window after m steps: Phi_m = B^+(x_n) ... B^+(x_{n+m-1}) Psi_T
        (Eq. bp_dets, with B(x)^+ = B(-conj(x)): L_g real symmetric and the Taylor
        polynomial has real coefficients), and the weighted averages of Eq. bp of
        the spin-summed one-body density <Phi_m|a+_p a_q|Psi_n>/<Phi_m|Psi_n>:
        returns (rho BP-PRes with weights W_{n+m} prod_k factor_k, rho BP-PhL
        with W_{n+m}, the two weight sums, Phi_m)."""
        st, p = self.setup, self.p
        bp, self.bp = self.bp, None
        phi = np.array(np.broadcast_to(st.VT, (self.W, st.M, st.N)), np.complex128)
        for x in reversed(bp["fields"]):
            V = assemble_V(st, -np.conj(x))
            phi = st.Bhalf @ taylor(V, st.Bhalf @ phi, p.taylor_order)
        alive = np.nonzero(self.weight != 0)[0]
        rho = one_body_density(phi[alive], bp["psi_n"][alive], st)
        w = self.weight[alive]
        wp = w * bp["factor"][alive]
        rho_pres = np.einsum("w,wpq->pq", wp, rho) / np.sum(wp)
        rho_phl = np.einsum("w,wpq->pq", w, rho) / np.sum(w)
        return rho_pres, rho_phl, complex(np.sum(wp)), complex(np.sum(w)), phi

    # --- estimators (Eq. localenergy, Eq. cap) ------------------------------
    def local_energies(self):
        return local_energy(self.setup, self.theta)

    def energy_sums(self):
        """(sum_w W Re E_loc, sum_w W) over live walkers; E_loc capped."""
        alive = np.nonzero(self.weight != 0)[0]
        if alive.size == 0:
            return 0.0, 0.0
        e = local_energy(self.setup, self.theta[alive])
        w = self.weight[alive]
        if self.p.mode == "phaseless":
            er = e.real
            if self.p.ecap_C > 0:
                half = math.sqrt(self.p.ecap_C / self.p.dt)
                er = np.clip(er, self.setup.E_T - half, self.setup.E_T + half)
            return float(np.sum(w * er)), float(np.sum(w))
        return complex(np.sum(w * e)), complex(np.sum(w))

    def energy(self):
        num, den = self.energy_sums()
        return num / den if den != 0 else _NAN
