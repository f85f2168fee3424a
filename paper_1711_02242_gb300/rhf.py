"""Closed-shell Hartree-Fock trial for afqmc_init (host-side input preparation).

The trial |Psi_T> of Sec. 3.4.1 is an input of the library, not a step of the
walk.  This helper builds it from (h, L) for callers that have no quantum
chemistry code: Roothaan iterations on the Fock matrix
F = h + 2 sum_g Tr(L_g D) L_g - sum_g (L_g C)(L_g C)^T, D = C C^T, accelerated
by Pulay's DIIS on the orbital gradient F D - D F.
"""
from __future__ import annotations

import numpy as np


def rhf_trial(h1, L, N, tol=1e-10, max_iter=300, nvec=8):
    """Return (C_occ (M, N), converged, max |FD - DF|)."""
    h1 = np.asarray(h1, np.float64)
    G, M, _ = L.shape
    Lf = L.reshape(G, M * M)
    _, C = np.linalg.eigh(h1)
    C = C[:, :N]
    hist_F, hist_e = [], []
    grad = np.inf
    for _ in range(max_iter):
        D = C @ C.T
        J = 2.0 * ((Lf @ D.ravel()) @ Lf).reshape(M, M)
        LC = np.matmul(L, C)
        K = np.tensordot(LC, LC, axes=([0, 2], [0, 2]))
        F = h1 + J - K
        e = F @ D - D @ F
        grad = float(np.abs(e).max())
        if grad < tol:
            return C, True, grad
        hist_F.append(F)
        hist_e.append(e.ravel())
        hist_F, hist_e = hist_F[-nvec:], hist_e[-nvec:]
        n = len(hist_F)
        if n > 1:
            E = np.array(hist_e)
            A = np.zeros((n + 1, n + 1))
            A[:n, :n] = E @ E.T
            A[n, :n] = A[:n, n] = -1.0
            b = np.zeros(n + 1)
            b[n] = -1.0
            try:
                w = np.linalg.lstsq(A, b, rcond=None)[0][:n]
                F = np.tensordot(w, np.array(hist_F), axes=1)
            except np.linalg.LinAlgError:
                pass
        _, V = np.linalg.eigh(F)
        C = V[:, :N]
    return C, False, grad
