"""Restricted Hartree-Fock for the single-determinant trial (Sec. 3.4.1).

TEST INFRASTRUCTURE: part of the CPU oracle.  Only tests, the smoke check and
the CPU-baseline leg of the benchmark may import it.

The two-body interaction is given by its Cholesky vectors,
v_pqrs = sum_g L[g]_pr L[g]_qs (Sec. 2.3, Eq. chol).  For a closed-shell
density P = C_occ C_occ^T (per spin) the Fock matrix is

    F = h + 2 sum_g Tr(L_g P) L_g - sum_g L_g P L_g

and the RHF energy (the Slater-Condon energy of the determinant) is

    E = 2 Tr(h P) + 2 sum_g Tr(L_g P)^2 - sum_g Tr(L_g P L_g P) + H0.

Roothaan iterations with Pulay's DIIS on the commutator FP - PF; the
orbitals are orthonormal (the basis is an orthonormal MO basis, Sec. 2).
"""
from __future__ import annotations

import numpy as np


def fock(h1, L, C):
    N = C.shape[1]
    P = C @ C.T
    nchol, M, _ = L.shape
    Lf = L.reshape(nchol, M * M)
    coul = Lf @ P.reshape(M * M)  # Tr(L_g P) for symmetric L_g
    J = 2.0 * (coul @ Lf).reshape(M, M)
    LC = L @ C  # (nchol, M, N)
    K = np.tensordot(LC, LC, axes=([0, 2], [0, 2]))  # sum_g L_g P L_g
    del N
    return h1 + J - K, P, coul


def rhf_energy(h1, L, C, H0=0.0):
    P = C @ C.T
    nchol, M, _ = L.shape
    coul = L.reshape(nchol, M * M) @ P.reshape(M * M)
    LC = L @ C
    CLC = np.einsum("pi,gpj->gij", C, LC)  # C^T L_g C
    exch = np.einsum("gij,gji->", CLC, CLC)
    return H0 + 2.0 * np.sum(h1 * P) + 2.0 * np.sum(coul ** 2) - exch


def rhf(h1, L, N, H0=0.0, tol=1e-10, max_iter=500, diis_size=8,
        level_shift=0.0):
    """Return (C_occ (M, N), E_RHF, converged, residual)."""
    M = h1.shape[0]
    e, C = np.linalg.eigh(h1)
    C = C[:, :N]
    errs, focks = [], []
    resid = np.inf
    for _ in range(max_iter):
        F, P, _ = fock(h1, L, C)
        err = F @ P - P @ F
        resid = float(np.max(np.abs(err)))
        if resid < tol:
            return C, rhf_energy(h1, L, C, H0), True, resid
        errs.append(err)
        focks.append(F)
        if len(errs) > diis_size:
            errs.pop(0)
            focks.pop(0)
        n = len(errs)
        if n >= 2:
            B = -np.ones((n + 1, n + 1))
            B[n, n] = 0.0
            for i in range(n):
                for j in range(n):
                    B[i, j] = np.sum(errs[i] * errs[j])
            rhs = np.zeros(n + 1)
            rhs[n] = -1.0
            try:
                coef = np.linalg.solve(B, rhs)[:n]
                F = sum(c * f for c, f in zip(coef, focks))
            except np.linalg.LinAlgError:
                pass
        if level_shift:
            F = F + level_shift * (np.eye(M) - P)
        e, Cn = np.linalg.eigh(F)
        C = Cn[:, :N]
    return C, rhf_energy(h1, L, C, H0), False, resid
