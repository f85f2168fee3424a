"""Pins of the modified Cholesky oracle (Sec. 2.3, Eqs. chol and chol2).

None of these re-type the oracle's loop.  They check it against closed forms
(2x2 and diagonal matrices), LAPACK's pivoted Cholesky (dpstrf, the same
largest-diagonal pivot rule), the rank of an interaction built from known
vectors, the threshold bound the paper derives from Cauchy-Schwarz, the
symmetry of vectors of a real interaction and the one-body term of Eq. mcd1,
and the damped prescreening on a matrix with one tiny diagonal.
"""
import numpy as np
import pytest
import scipy.linalg.lapack as lapack

import workloads
from fock import eri_from_cholesky
from oracle import mcd


def random_psd(n, rank, seed, decay=None):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((rank, n))
    if decay is not None:
        A *= (decay ** np.arange(rank))[:, None]
    V = A.T @ A
    return (V + V.T) / 2


def test_two_by_two_closed_form():
    a, b, c = 2.0, 0.6, 3.0
    L, piv, dmax, resid, conv = mcd.modified_cholesky(np.array([[a, b], [b, c]]), 1e-12)
    # the larger diagonal (index 1) first: L1 = (b, c) / sqrt(c); then the Schur
    # complement a - b^2 / c on index 0
    assert list(piv) == [1, 0] and conv
    assert np.allclose(L[0], [b / np.sqrt(c), np.sqrt(c)], rtol=0, atol=1e-15)
    assert np.allclose(L[1], [np.sqrt(a - b * b / c), 0.0], rtol=0, atol=1e-15)
    assert np.allclose(dmax, [c, a - b * b / c], rtol=0, atol=1e-15)
    assert abs(resid) < 1e-15


def test_diagonal_matrix_sorted_square_roots():
    a = np.array([0.5, 3.0, 1e-3, 2.0, 1e-7])
    L, piv, dmax, resid, conv = mcd.modified_cholesky(np.diag(a), 1e-5)
    assert list(piv) == [1, 3, 0, 2] and conv
    want = np.zeros((4, 5))
    for k, p in enumerate([1, 3, 0, 2]):
        want[k, p] = np.sqrt(a[p])
    assert np.max(np.abs(L - want)) < 1e-15 * np.sqrt(3.0)  # a / sqrt(a), rounded
    assert resid == 1e-7  # the diagonal left below delta


def test_matches_lapack_pivoted_cholesky():
    """dpstrf pivots on the largest remaining diagonal and stops when it is
    at or below tol: the same vectors, in the same order, as Eq. chol2."""
    n, rank = 40, 25
    V = random_psd(n, rank, 5)
    L, piv, dmax, resid, conv = mcd.modified_cholesky(V, 1e-10)
    c, lpiv, lrank, info = lapack.dpstrf(V.copy(), tol=1e-10, lower=1)
    assert lrank == rank and len(piv) == rank and conv
    lpiv = lpiv - 1
    assert list(piv) == list(lpiv[:rank])
    # P^T V P = C C^T with (P^T V P)[k, j] = V[lpiv[k], lpiv[j]]: vector g has
    # C[k, g] at index lpiv[k]
    want = np.zeros((rank, n))
    want[:, lpiv] = np.tril(c)[:, :rank].T
    assert np.max(np.abs(L - want)) < 1e-12 * np.max(np.abs(want))


def test_threshold_bounds_every_residual_element():
    """Stopping at Delta_max < delta bounds every element of the residual by
    delta (Cauchy-Schwarz); every pivot taken was at least delta, and the
    pivots never grow (the diagonal only decreases)."""
    V = random_psd(60, 60, 9, decay=0.8)
    counts = []
    for delta in (1e-3, 1e-5, 1e-8):
        L, piv, dmax, resid, conv = mcd.modified_cholesky(V, delta)
        R = V - L.T @ L
        assert conv and resid < delta
        assert np.max(np.abs(R)) < delta
        assert np.max(np.diag(R)) < delta + 1e-15
        assert np.all(dmax >= delta)
        assert np.all(np.diff(dmax) <= 1e-15)
        assert len(set(piv)) == len(piv)
        counts.append(len(piv))
    assert counts[0] < counts[1] < counts[2] < 60


def test_interaction_from_known_vectors():
    """v_pqrs = sum_g L_g[p,r] L_g[q,s] with G symmetric vectors: the matrix
    of Sec. 2.3 has rank G, so the decomposition returns G vectors; they are
    symmetric in (p, r) like every real interaction's, and they rebuild the
    one-body term sum_r v_prrq of Eq. mcd1."""
    M, G = 6, 10
    _, Lg, _ = workloads.hamiltonian(M, G, 321)
    v = eri_from_cholesky(Lg)
    V = mcd.eri_matrix(v)
    assert V[2 * M + 4, 1 * M + 5] == v[2, 1, 4, 5]  # mu = p M + r, nu = q M + s
    delta = 1e-10
    L, piv, dmax, resid, conv = mcd.modified_cholesky(V, delta)
    assert len(piv) == G and conv
    Lm = L.reshape(G, M, M)
    assert np.max(np.abs(Lm - Lm.transpose(0, 2, 1))) < 1e-12
    assert np.max(np.abs(V - L.T @ L)) < delta
    one_body = np.einsum("prrq->pq", v)
    assert np.max(np.abs(one_body - np.einsum("gpr,grq->pq", Lm, Lm))) < M * delta


def test_damped_prescreening_zeroes_a_tiny_diagonal():
    """Row and column 7 scaled by 1e-11: sqrt(|Delta_77| Delta_max) is below
    1e-9 from the first iteration, so index 7 is zero in every vector and never
    a pivot, although the unscreened first vector would be nonzero there; the
    residual bound still holds."""
    V = random_psd(20, 20, 13)
    s = np.ones(20)
    s[7] = 1e-11
    V = V * s[:, None] * s[None, :]
    delta = 1e-6
    L, piv, dmax, resid, conv = mcd.modified_cholesky(V, delta)
    assert conv and 7 not in piv and len(piv) == 19
    assert np.all(L[:, 7] == 0.0)
    nu0 = piv[0]
    assert V[7, nu0] / np.sqrt(V[nu0, nu0]) != 0.0
    assert np.max(np.abs(V - L.T @ L)) < delta
    # without the scaling, nothing is screened: all 20 indices are pivots
    L2, piv2, *_ = mcd.modified_cholesky(random_psd(20, 20, 13), delta)
    assert sorted(piv2) == list(range(20))


def test_vector_cap_returns_the_leading_vectors():
    V = random_psd(30, 30, 21)
    L, piv, dmax, resid, conv = mcd.modified_cholesky(V, 1e-12)
    L3, piv3, dmax3, resid3, conv3 = mcd.modified_cholesky(V, 1e-12, max_vectors=3)
    assert conv and not conv3 and len(piv3) == 3
    assert np.array_equal(L3, L[:3]) and list(piv3) == list(piv[:3])
    assert resid3 >= 1e-12


def test_zero_matrix_gives_no_vectors():
    L, piv, dmax, resid, conv = mcd.modified_cholesky(np.zeros((5, 5)), 1e-6)
    assert L.shape == (0, 5) and conv and resid == 0.0
    with pytest.raises(FloatingPointError):
        mcd.modified_cholesky(np.array([[1.0, 0.0], [0.0, np.nan]]), 1e-6)
