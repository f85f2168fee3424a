"""Modified Cholesky decomposition of the two-electron interaction (the CPU oracle).

TEST INFRASTRUCTURE: the reference the GPU decomposition is checked against.
Only tests, the smoke check and the CPU-baseline leg of the benchmark may
import it; the GPU library never calls it.

Sec. 2.3 ("Modified Cholesky decomposition", Eqs. mcd1, chol, chol2): with
real orbitals the interaction v_pqrs is the symmetric positive semi-definite
matrix V_{mu nu} with mu = (p, r), nu = (q, s); here mu = p M + r and
nu = q M + s, so V = v.transpose(0, 2, 1, 3).reshape(M*M, M*M).  After k
vectors the residual is Delta = V - sum_g L^g (L^g)^T (Eq. chol).  One
iteration, in the paper's order:

  1. nu0 = the index of the largest residual diagonal, Delta_max = Delta_{nu0 nu0};
     stop when Delta_max < delta (then |Delta_{mu nu}| < delta everywhere by
     Cauchy-Schwarz).
  2. damped prescreening: every mu with sqrt(|Delta_{mu mu}| Delta_max) <=
     min(1e-9, delta) is set to zero.
  3. the next vector is the residual column through the pivot over its square
     root, L_mu = Delta_{mu nu0} / sqrt(Delta_max) (Eq. chol2).
  4. the residual is updated by that vector.

Readings (the paper leaves these open):

  * the residual column is formed from V and the vectors found so far,
    Delta_{mu nu0} = V_{mu nu0} - sum_g L^g_mu L^g_nu0, and only its diagonal
    is kept between iterations (Delta_{mu mu} -= (L_mu)^2), so the M^2 x M^2
    residual is never stored.
  * "set equal to zero" in step 2 zeroes the row and column mu of the
    residual: Delta_{mu mu} = 0 and L_mu = 0 in the new vector.  A zeroed
    diagonal passes the test again at every later iteration, so a screened
    index stays at zero in every later vector.
  * among equal largest diagonals the smallest index is the pivot.
  * the stopping test "Delta < delta" is on the largest residual diagonal.
"""
from __future__ import annotations

import numpy as np

# prescreening floor of step 2: sqrt(|Delta_mm| Delta_max) <= min(SCREEN, delta)
SCREEN = 1e-9


def eri_matrix(v: np.ndarray) -> np.ndarray:
    """V_{(pr),(qs)} = v_pqrs as an (M*M) x (M*M) matrix, mu = p M + r (Sec. 2.3)."""
    M = v.shape[0]
    return np.ascontiguousarray(v.transpose(0, 2, 1, 3).reshape(M * M, M * M))


def modified_cholesky(V: np.ndarray, delta: float, max_vectors: int | None = None):
    """Vectors L [n][dim], pivots [n], the Delta_max of each iteration [n] and the
    largest residual diagonal left, for the symmetric PSD matrix V (Eqs. chol,
    chol2).  Stops when the largest residual diagonal is below delta, or after
    max_vectors vectors (then ``converged`` is False)."""
    V = np.asarray(V, dtype=np.float64)
    dim = V.shape[0]
    if max_vectors is None:
        max_vectors = dim
    tau = min(SCREEN, delta)
    d = np.diag(V).copy()  # residual diagonal Delta_{mu mu}
    vecs = np.zeros((max_vectors, dim))
    pivots, dmaxs = [], []
    n = 0
    converged = False
    while True:
        nu0 = int(np.argmax(d))  # first of equal maxima
        dmax = d[nu0]
        if not np.isfinite(dmax):
            raise FloatingPointError("non-finite residual diagonal")
        if dmax < delta:
            converged = True
            break
        if n == max_vectors:
            break
        screened = np.sqrt(np.abs(d) * dmax) <= tau  # step 2
        d[screened] = 0.0
        col = V[:, nu0] - vecs[:n].T @ vecs[:n, nu0]  # residual column Delta_{mu nu0}
        col[screened] = 0.0
        vec = col / np.sqrt(dmax)  # Eq. chol2
        d -= vec * vec  # residual update, diagonal only
        vecs[n] = vec
        pivots.append(nu0)
        dmaxs.append(dmax)
        n += 1
    return vecs[:n].copy(), np.array(pivots, dtype=np.int64), np.array(dmaxs), float(np.max(d)), converged
