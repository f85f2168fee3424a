"""Local energies of the mixed path (tcgen05 exchange with the fused
sum_ij T_ij T_ji epilogue, Eq. localenergy3) on walkers that all differ.

Expected values come from the oracle only: the float64 energies of
oracle.afqmc.local_energy, and the same formula evaluated with the operands
the mixed path feeds the tensor cores (the half-rotated vectors and Theta
rounded to BF16 or TF32, products and sums exact).  The library works in the
orthonormal basis whose first N vectors are the trial orbitals and whose
others complete them by the Householder QR of the trial; the operands are
rounded in that basis (Lh_g Q and Q^T Theta), which complete_basis below
rebuilds the same way.  The float64 path must
match the first to 1e-9 and the mixed path the second to 2e-5 of the size of
the energy's terms (|one-body| + |Coulomb| + |exchange|): what is left is FP32
accumulation.  A (g, w) block taken from the wrong walker or vector moves
E_loc by the spread of the exchange energies across walkers, above that
bound on every shape (checked).  How far the rounded operands themselves move
the energy (the mixed path's bias) is reported by the benchmark, not bounded
here.  Shapes cover every column padding of the exchange tile (2N padded to
16, 32, 64, 128: 16, 8, 4, 2 walkers per tile), a single electron pair,
ragged vector and walker counts, and N = 64 (the largest N a state takes).
"""
import numpy as np
import pytest

import workloads
from oracle import afqmc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_02242_gb300 as p

    return p


def round_bf16(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_tf32(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def complete_basis(trial):
    """Orthogonal Q with Q[:, :N] = trial: Householder QR of the trial
    (reflectors H_1 .. H_N), Q = H_1 ... H_N with its first N columns set to
    the trial."""
    M, N = trial.shape
    a = trial.copy()
    vs = []
    for k in range(N):
        x = a[k:, k]
        alpha = -np.linalg.norm(x) if x[0] >= 0 else np.linalg.norm(x)
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv > 0:
            v /= nv
        a[k:, k:] -= 2.0 * np.outer(v, v @ a[k:, k:])
        vs.append(v)
    q = np.eye(M)
    for k in range(N - 1, -1, -1):
        q[k:, :] -= 2.0 * np.outer(vs[k], vs[k] @ q[k:, :])
    q[:, :N] = trial
    return q


def energy_terms(setup, theta, rnd=None, Q=None):
    """(E_loc, |one-body| + |Coulomb| + |exchange|, exchange) per walker; with
    rnd, the two-body terms use Lh Q and Q^T Theta rounded."""
    e1 = 2.0 * np.einsum("iq,wqi->w", setup.hh, theta)
    Lh, th = setup.Lh, theta
    if rnd is not None:
        Lh = rnd(Lh @ Q)
        th = np.einsum("pq,wpi->wqi", Q, theta)
        th = rnd(th.real) + 1j * rnd(th.imag)
    t = 2.0 * np.einsum("giq,wqi->wg", Lh, th)
    G, N, M = Lh.shape
    Lh2 = Lh.reshape(G * N, M)
    ex = np.empty(theta.shape[0], np.complex128)
    for w in range(theta.shape[0]):
        T = (Lh2 @ th[w]).reshape(G, N, N)
        ex[w] = np.einsum("gij,gji->", T, T)
    coul = 0.5 * np.sum(t * t, axis=1)
    return setup.H0 + e1 + coul - ex, np.abs(e1) + np.abs(coul) + np.abs(ex), ex


SHAPES = [  # M, N, nchol, nwalkers
    (16, 1, 40, 37),
    (24, 7, 60, 50),
    (40, 16, 80, 40),
    (80, 33, 100, 20),
    (140, 64, 60, 9),
]


@pytest.mark.parametrize("M,N,G,W", SHAPES)
def test_mixed_local_energies_match_rounded_oracle(pkg, M, N, G, W):
    h1, L, _ = workloads.hamiltonian(M, G, 4000 + M + N)
    trial = np.linalg.eigh(h1)[1][:, :N]
    rng = np.random.default_rng(M * 100 + N)
    phi = trial[None] + (0.5 / np.sqrt(M)) * (rng.standard_normal((W, M, N))
                                              + 1j * rng.standard_normal((W, M, N)))
    setup = afqmc.Setup(h1, L, trial)
    Q = complete_basis(trial)
    _, theta = afqmc.overlap(setup, phi)
    e_ref = afqmc.local_energy(setup, theta)
    _, scale, ex = energy_terms(setup, theta)
    # a misplaced exchange block would show: the walkers' exchange energies differ
    assert np.std(ex.real) > 25 * 2e-5 * scale.max()
    for prec, rnd, tol in ((0, None, 1e-9), (2, round_bf16, 2e-5), (1, round_tf32, 2e-5)):
        p = pkg.default_params(M, N, G, W, precision=prec, energy_period=0)
        run = pkg.AfqmcRun(h1, L, trial, p)
        run.set_walkers(phi, np.ones(W))
        e = run.local_energies()
        assert run.info().status == 0
        want = e_ref if rnd is None else energy_terms(setup, theta, rnd, Q)[0]
        err = np.abs(e - want) / scale
        assert err.max() < tol, (prec, int(err.argmax()), err.max())
