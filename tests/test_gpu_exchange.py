"""Local energies of the mixed path (tcgen05 exchange with the fused
sum_ij T_ij T_ji epilogue, Eq. localenergy3) against the float64 path on
the same walkers.

The walkers are the trial plus a random complex perturbation of 0.3, so every
walker has its own exchange energy; a (g, w) block taken from the wrong walker
or vector moves E_loc by far more than the bound.  Shapes cover every column
padding of the exchange tile (2N padded to 16, 32, 64, 128: 16, 8, 4, 2
walkers per tile), a single electron pair, ragged vector and walker counts,
and N = 64 (128 rows of Theta^T per walker).  The float64 path is held to
the oracle at 1e-10 elsewhere, so the bound is the operand rounding alone:
BF16 inputs (2^-9) 3e-3 relative, TF32 inputs (2^-11) 5e-4.
"""
import numpy as np
import pytest

import workloads

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


SHAPES = [  # M, N, nchol, nwalkers
    (16, 1, 40, 37),
    (24, 7, 60, 50),
    (40, 16, 80, 40),
    (80, 33, 100, 20),
    (140, 64, 60, 9),
]


@pytest.mark.parametrize("M,N,G,W", SHAPES)
def test_mixed_local_energies_match_fp64(pkg, M, N, G, W):
    h1, L, _ = workloads.hamiltonian(M, G, 4000 + M + N)
    trial = np.linalg.eigh(h1)[1][:, :N]
    rng = np.random.default_rng(M * 100 + N)
    phi = trial[None] + 0.3 * (rng.standard_normal((W, M, N)) + 1j * rng.standard_normal((W, M, N)))
    wts = np.ones(W)
    energies = {}
    for prec in (0, 2, 1):
        p = pkg.default_params(M, N, G, W, precision=prec, energy_period=0)
        run = pkg.AfqmcRun(h1, L, trial, p)
        run.set_walkers(phi, wts)
        energies[prec] = run.local_energies()
        assert run.info().status == 0
    e64 = energies[0]
    # the walkers really differ
    assert np.std(e64.real) > 0.05 * np.abs(e64.real).mean()
    for prec, tol in ((2, 3e-3), (1, 5e-4)):
        err = np.abs(energies[prec] - e64) / np.abs(e64)
        assert err.max() < tol, (prec, int(err.argmax()), err.max())
