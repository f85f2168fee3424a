"""Brute-force second quantisation in the full Fock space (test helper).

Builds fermion operators by the Jordan-Wigner construction on 2M spin
orbitals (mode p + sigma*M), so that Slater determinants, the Hamiltonian of
Eq. bo_ham2 and exponentials of one-body operators are explicit vectors and
matrices.  Used only to pin the oracle for M <= 6; it shares nothing with the
oracle beyond the mathematics it checks.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


class Fock:
    def __init__(self, M: int):
        self.M = M
        n = 2 * M
        self.n = n
        self.dim = 1 << n
        I2 = sp.identity(2, format="csr", dtype=np.complex128)
        Z = sp.csr_matrix(np.diag([1.0, -1.0]).astype(np.complex128))
        # annihilator on one mode: |1> -> |0>, basis (|0>, |1>)
        a1 = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]], np.complex128))
        self.a = []
        for j in range(n):
            ops = [Z] * j + [a1] + [I2] * (n - j - 1)
            m = ops[0]
            for o in ops[1:]:
                m = sp.kron(m, o, format="csr")
            self.a.append(m)
        self.ad = [m.conj().T.tocsr() for m in self.a]
        vac = np.zeros(self.dim, np.complex128)
        vac[0] = 1.0
        self.vac = vac

    def mode(self, p, s):
        return p + s * self.M

    def one_body(self, A):
        """sum_sigma sum_pq A_pq a+_{p sigma} a_{q sigma} (spin independent)."""
        M = self.M
        out = sp.csr_matrix((self.dim, self.dim), dtype=np.complex128)
        for s in (0, 1):
            for p in range(M):
                for q in range(M):
                    if A[p, q] != 0:
                        out = out + A[p, q] * (self.ad[self.mode(p, s)] @ self.a[self.mode(q, s)])
        return out.tocsr()

    def hamiltonian(self, h1, v, H0=0.0):
        """H0 + sum h_pq a+a + 1/2 sum v_pqrs a+_p a+_q a_s a_r (Eq. bo_ham2)."""
        M = self.M
        H = H0 * sp.identity(self.dim, dtype=np.complex128, format="csr") + self.one_body(h1)
        for s, t in itertools.product((0, 1), repeat=2):
            for p, q, r, u in itertools.product(range(M), repeat=4):
                val = v[p, q, r, u]
                if abs(val) < 1e-15:
                    continue
                op = (self.ad[self.mode(p, s)] @ self.ad[self.mode(q, t)]
                      @ self.a[self.mode(u, t)] @ self.a[self.mode(r, s)])
                H = H + 0.5 * val * op
        return H.tocsr()

    def determinant(self, U_up, U_dn=None):
        """|Psi> = prod_i c+_{u_i up} prod_i c+_{v_i dn} |0> (Eq. SDdef)."""
        if U_dn is None:
            U_dn = U_up
        M = self.M
        psi = self.vac.copy()
        # apply creators right to left: the last orbital acts first
        cols = [(U_up[:, i], 0) for i in range(U_up.shape[1])] + \
               [(U_dn[:, i], 1) for i in range(U_dn.shape[1])]
        for u, s in reversed(cols):
            op = sum(u[p] * self.ad[self.mode(p, s)] for p in range(M))
            psi = op @ psi
        return psi

    def number_sector(self, n_up, n_dn):
        idx = []
        M = self.M
        for b in range(self.dim):
            # mode j is bit (n-1-j) in the kron ordering
            bits = [(b >> (self.n - 1 - j)) & 1 for j in range(self.n)]
            if sum(bits[:M]) == n_up and sum(bits[M:]) == n_dn:
                idx.append(b)
        return np.array(idx)


def eri_from_cholesky(L):
    """v_pqrs = sum_g L_g[p, r] L_g[q, s] (Eq. chol with V_(pr),(qs) = v_pqrs)."""
    return np.einsum("gpr,gqs->pqrs", L, L)


def expm_sparse_apply(Aop, vec):
    return sla.expm(Aop.toarray()) @ vec
