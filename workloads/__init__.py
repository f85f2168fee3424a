"""Seeded synthetic inputs for phaseless AFQMC runs.

This module only draws random numbers and describes workload shapes. It holds
none of the AFQMC arithmetic: no SCF, no propagation, no energies. Both the
CPU oracle (``oracle/``) and the GPU library's callers (``bench.py``, tests)
take their Hamiltonians from here, so the two sides always see the same input.

Hamiltonian recipe (the synthetic stand-in for the molecular integrals of the
paper, Sec. 2 "The AFQMC method", Eqs. bo_ham2 / bo_ham_matel):

* ``h1`` is real symmetric, ``M x M``: diagonal ``linspace(-2, 2, M)`` Ha,
  strictly-upper entries drawn ``N(0, 0.05)`` (0.05 is the standard
  deviation) in row-major order, then mirrored.
* each Cholesky vector ``L[g]`` (``g = 0 .. nchol-1``) is real symmetric
  ``M x M``: upper-triangle entries including the diagonal drawn
  ``N(0, a * exp(-g / M))`` in row-major order, then mirrored.  The
  two-electron tensor ``v_pqrs = sum_g L[g]_pr L[g]_qs`` (Sec. 2.3, Eq. chol)
  is then positive semi-definite by construction.
* the amplitude ``a`` is 0.5 for the 12-orbital, 48-vector workload and, for
  the others, 0.5 scaled so that ``sum_g ||L[g]||_F^2`` -- the variance of
  the one-body operator ``sum_g x_g L[g]`` under unit Gaussian fields -- is
  the same as there (``l_amplitude``).  Drawn with 0.5 at every size, the
  300-orbital operator has ``||sqrt(dt) sum_g x_g L[g]|| ~ 15``: its
  sixth-order Taylor series is far from converged, every walker overflows
  within a few steps, and the energies reach 2e5 Ha.
* draws come from numpy's PCG64 generator seeded ``1000 + config_index``;
  ``h1`` is drawn first, then ``L[0]``, ``L[1]``, ...
* the nuclear repulsion ``H0`` is 0.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload",
    "CONFIGS",
    "config",
    "hamiltonian",
    "l_amplitude",
    "batched_systems",
    "request_stream",
    "interaction_matrix",
    "interaction_matrix_device",
    "interaction_pairs",
    "interaction_pairs_device",
    "pair_expansion",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape and run parameters of one synthetic phaseless-AFQMC run."""

    name: str
    M: int  # orbitals
    N: int  # electrons per spin (N_up = N_dn, closed shell)
    nchol: int  # Cholesky vectors N_gamma
    nwalkers: int
    dt: float = 0.005
    nsteps: int = 200
    qr_period: int = 5
    pc_period: int = 0
    energy_period: int = 1
    taylor_order: int = 6
    seed: int = 1  # Philox key for the auxiliary fields
    ham_seed: int = 1000  # PCG64 seed of the Hamiltonian draw

    def hamiltonian(self):
        return hamiltonian(self.M, self.nchol, self.ham_seed,
                           l_scale=l_amplitude(self.M, self.nchol))


def l_amplitude(M: int, nchol: int, decay: float | None = None) -> float:
    """Amplitude of ``L[0]`` that gives ``sum_g ||L[g]||_F^2`` (expected) the
    value it has for M = 12, nchol = 48, decay 12, amplitude 0.5."""
    def spread(m, n, d):
        return m * m * sum(math.exp(-2.0 * g / d) for g in range(n))

    return 0.5 * math.sqrt(spread(12, 48, 12.0) / spread(M, nchol, float(decay or M)))


# The five workloads of the phaseless-AFQMC hot path.  Index i uses PCG64
# seed 1000 + i for its Hamiltonian and Philox seed 1 + i for its fields.
CONFIGS = {
    # M=12 closed shell, 3+3 electrons, 48 Cholesky vectors, 32 walkers.
    "c0": Workload("c0", M=12, N=3, nchol=48, nwalkers=32, nsteps=200,
                   qr_period=5, energy_period=1, seed=1, ham_seed=1000),
    # M=100, 10+10 electrons, 500 vectors, 1024 walkers, 1000 steps.
    "c1": Workload("c1", M=100, N=10, nchol=500, nwalkers=1024, nsteps=1000,
                   qr_period=5, energy_period=10, seed=2, ham_seed=1001),
    # M=300, 25+25 electrons, 1800 vectors, 512 walkers, energy every 10 steps.
    "c2": Workload("c2", M=300, N=25, nchol=1800, nwalkers=512, nsteps=100,
                   qr_period=5, energy_period=10, seed=3, ham_seed=1002),
}


def config(name: str) -> Workload:
    return CONFIGS[name]


def _sym_from_upper(rng: np.random.Generator, M: int, scale: float,
                    include_diag: bool) -> np.ndarray:
    iu = np.triu_indices(M, 0 if include_diag else 1)
    a = np.zeros((M, M))
    a[iu] = rng.normal(0.0, scale, size=iu[0].size)
    a = a + np.triu(a, 1).T
    return a


def hamiltonian(M: int, nchol: int, ham_seed: int, decay: float | None = None,
                l_scale: float = 0.5):
    """Return ``(h1, L, H0)``: ``h1`` (M, M), ``L`` (nchol, M, M), float64.

    ``decay`` is the decay length of the Cholesky-vector amplitudes
    (default ``M``); ``l_scale`` the amplitude of ``L[0]`` (default 0.5).
    """
    if decay is None:
        decay = float(M)
    rng = np.random.Generator(np.random.PCG64(ham_seed))
    h1 = _sym_from_upper(rng, M, 0.05, include_diag=False)
    h1[np.diag_indices(M)] = np.linspace(-2.0, 2.0, M)
    L = np.empty((nchol, M, M))
    for g in range(nchol):
        L[g] = _sym_from_upper(rng, M, l_scale * math.exp(-g / decay), True)
    return h1, L, 0.0


def interaction_matrix(L: np.ndarray) -> np.ndarray:
    """The two-electron matrix V[(p, r)][(q, s)] = v_pqrs = sum_g L[g]_pr L[g]_qs
    of Cholesky vectors ``L`` (nchol, M, M), as an (M*M) x (M*M) float64 array
    with row index p*M + r; symmetrised so that V == V.T exactly.  The input of
    the modified Cholesky decomposition (Sec. 2.3)."""
    G, M, _ = L.shape
    Lm = np.ascontiguousarray(L.reshape(G, M * M))
    V = Lm.T @ Lm
    V += V.T
    V *= 0.5
    return V


def pair_expansion(M: int) -> np.ndarray:
    """Index map (M*M,) from (p, r), row p*M + r, to its pair p' <= r' (row-major
    order of the upper triangle), so that V = Vpair[idx][:, idx]."""
    iu = np.triu_indices(M)
    pair = np.zeros((M, M), np.int64)
    pair[iu] = np.arange(iu[0].size)
    pair = pair + np.triu(pair, 1).T
    return pair.reshape(-1)


def interaction_pairs(L: np.ndarray) -> np.ndarray:
    """The two-electron matrix over index pairs p <= r (row-major upper
    triangle): Vpair[(p, r)][(q, s)] = sum_g L[g]_pr L[g]_qs, symmetrised so
    that Vpair == Vpair.T exactly.  Vpair[idx][:, idx] with idx =
    pair_expansion(M) is the full matrix, rows (p, r) and (r, p) equal."""
    M = L.shape[1]
    iu = np.triu_indices(M)
    Lp = np.ascontiguousarray(L[:, iu[0], iu[1]])
    W = Lp.T @ Lp
    W += W.T
    W *= 0.5
    return W


def interaction_pairs_device(L: np.ndarray, device="cuda:0"):
    """``interaction_pairs(L)`` built on a CUDA device with PyTorch (16 GB at
    M = 300)."""
    import torch

    M = L.shape[1]
    iu = np.triu_indices(M)
    Lp = torch.from_numpy(np.ascontiguousarray(L[:, iu[0], iu[1]])).to(device)
    W = Lp.T @ Lp
    del Lp
    W += W.T.clone()
    W *= 0.5
    return W


def interaction_matrix_device(L: np.ndarray, device="cuda:0"):
    """``interaction_matrix(L)`` built on a CUDA device with PyTorch (for
    interactions too large to form on the host, e.g. M = 300: 65 GB).  The
    products run over the M(M+1)/2 index pairs p <= r, whose rows and columns
    are then repeated for (r, p), so rows (p, r) and (r, p) are identical;
    the result is symmetric to rounding, then symmetrised exactly."""
    import torch

    G, M, _ = L.shape
    iu = np.triu_indices(M)
    Lp = torch.from_numpy(np.ascontiguousarray(L[:, iu[0], iu[1]])).to(device)
    W = Lp.T @ Lp
    del Lp
    W = (W + W.T) * 0.5
    idx = torch.from_numpy(pair_expansion(M)).to(device)
    V = W.index_select(0, idx)
    del W
    return V.index_select(1, idx)


def batched_systems(seed: int = 3000, count: int = 16):
    """Uneven systems for one grouped launch: M in {40, 60, ..., 200},
    N = M/8, nchol = 5M, walkers in {64, 128, ..., 1024}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        M = int(rng.choice(np.arange(40, 201, 20)))
        W = int(rng.choice(np.arange(64, 1025, 64)))
        out.append(Workload(f"sys{i}", M=M, N=M // 8, nchol=5 * M, nwalkers=W,
                            nsteps=500, qr_period=5, energy_period=10,
                            seed=100 + i, ham_seed=seed + 1 + i))
    return out


def request_stream(seed: int = 4000, count: int = 200, rate: float = 20.0,
                   blocks: int = 20, steps_per_block: int = 50):
    """Poisson stream of run requests: arrival times (s) and workloads.

    M uniform in [20, 300], N uniform in [2, M/8], nchol = 5M, walkers
    uniform in [128, 2048], ``blocks`` blocks of ``steps_per_block`` steps.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        M = int(rng.integers(20, 301))
        N = int(rng.integers(2, max(2, M // 8) + 1))
        W = int(rng.integers(128, 2049))
        reqs.append((t, Workload(f"req{i}", M=M, N=N, nchol=5 * M, nwalkers=W,
                                 nsteps=blocks * steps_per_block, qr_period=5,
                                 energy_period=steps_per_block,
                                 seed=10_000 + i, ham_seed=seed + 1 + i)))
    return reqs
