"""Modified Cholesky decomposition on the GPU (afqmc_modified_cholesky, Sec. 2.3,
Eqs. chol and chol2) against the oracle (oracle.mcd) on the same matrices.

The two sides sum the earlier vectors in different orders, so the vectors agree
to rounding: 1e-10 of the largest element.  The pivots must be the same
sequence; on an interaction matrix the rows (p, r) and (r, p) are equal, so a
pivot is compared as the unordered pair {p, r} (either row gives the same
vector).  Cases: random positive semi-definite matrices of full and deficient
rank, the interaction of the 100-orbital, 500-vector workload (dimension 1e4,
several indices per warp, the launch shape of the benchmark), damped
prescreening of a tiny diagonal, the vector cap, one-element and zero
matrices, a non-finite diagonal and argument errors; and the decomposition
over index pairs p <= r (afqmc_modified_cholesky_pairs) against the oracle
on the full matrix, with odd and even pair counts.
"""
import numpy as np
import pytest

import workloads
from oracle import mcd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_02242_gb300 as pkg

    return torch, pkg


def random_psd(n, rank, seed, decay=None):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((rank, n))
    if decay is not None:
        A *= (decay ** np.arange(rank))[:, None]
    V = A.T @ A
    return (V + V.T) / 2


def gpu_mcd(torch, pkg, V, delta, max_vectors):
    L, piv, resid = pkg.afqmc_modified_cholesky(torch.from_numpy(V).cuda(), delta, max_vectors)
    torch.cuda.synchronize()
    return L.cpu().numpy(), piv.cpu().numpy().astype(np.int64), resid


def compare(got, want, M=None):
    L, piv, resid = got
    Lo, pivo, dmaxo, reso, convo = want
    assert L.shape == Lo.shape, (L.shape, Lo.shape)
    if M is None:
        assert np.array_equal(piv, pivo)
    else:
        canon = lambda p: np.minimum(p // M, p % M) * M + np.maximum(p // M, p % M)  # noqa: E731
        assert np.array_equal(canon(piv), canon(pivo))
    scale = max(np.max(np.abs(Lo)), 1e-300) if Lo.size else 1.0
    if Lo.size:
        err = np.max(np.abs(L - Lo)) / scale
        assert err < 1e-10, err
    assert abs(resid - reso) <= 1e-10 * max(abs(reso), scale * scale)


@pytest.mark.parametrize("n,rank,decay,delta", [
    (1, 1, None, 1e-8),
    (7, 7, None, 1e-12),
    (300, 300, 0.97, 1e-6),   # full rank, decaying spectrum: stops on delta
    (333, 120, None, 1e-8),   # rank deficient: stops after the rank
    (2000, 700, 0.99, 1e-5),
])
def test_random_psd_matches_oracle(env, n, rank, decay, delta):
    torch, pkg = env
    V = random_psd(n, rank, 100 + n, decay)
    want = mcd.modified_cholesky(V, delta)
    got = gpu_mcd(torch, pkg, V, delta, n)
    compare(got, want)
    assert want[4] and got[2] < delta


@pytest.mark.parametrize("M,G,delta", [(10, 30, 1e-8), (24, 120, 1e-6), (100, 500, 1e-6)])
def test_interaction_matches_oracle(env, M, G, delta):
    torch, pkg = env
    _, L, _ = workloads.hamiltonian(M, G, 2000 + M, l_scale=workloads.l_amplitude(M, G))
    V = workloads.interaction_matrix(L)
    want = mcd.modified_cholesky(V, delta)
    got = gpu_mcd(torch, pkg, V, delta, G + 16)
    compare(got, want, M=M)
    # the vectors rebuild the interaction within delta (spot rows)
    Lg = got[0]
    rows = np.random.default_rng(M).choice(M * M, 16, replace=False)
    assert np.max(np.abs(V[rows] - Lg[:, rows].T @ Lg)) < delta


def test_prescreening_zeroes_tiny_diagonal(env):
    torch, pkg = env
    V = random_psd(64, 64, 7)
    s = np.ones(64)
    s[5] = 1e-11
    s[40] = 3e-12
    V = V * s[:, None] * s[None, :]
    want = mcd.modified_cholesky(V, 1e-6)
    got = gpu_mcd(torch, pkg, V, 1e-6, 64)
    compare(got, want)
    assert np.all(got[0][:, [5, 40]] == 0.0) and 5 not in got[1] and 40 not in got[1]


def test_vector_cap(env):
    torch, pkg = env
    V = random_psd(500, 500, 3, 0.98)
    full = mcd.modified_cholesky(V, 1e-9)
    L, piv, resid = gpu_mcd(torch, pkg, V, 1e-9, 37)
    assert L.shape == (37, 500) and resid >= 1e-9
    assert np.array_equal(piv, full[1][:37])
    assert np.max(np.abs(L - full[0][:37])) < 1e-10 * np.max(np.abs(full[0]))
    assert abs(resid - full[2][37]) < 1e-10 * full[2][0]  # the next pivot's Delta_max


def test_zero_and_nonfinite(env):
    torch, pkg = env
    L, piv, resid = gpu_mcd(torch, pkg, np.zeros((50, 50)), 1e-6, 10)
    assert L.shape == (0, 50) and resid == 0.0
    V = random_psd(40, 40, 1)
    V[17, 17] = np.nan
    with pytest.raises(pkg.AfqmcError, match="ENONFINITE"):
        gpu_mcd(torch, pkg, V, 1e-6, 40)


def test_argument_errors(env):
    torch, pkg = env
    import ctypes

    lib = pkg.lib()
    V = torch.eye(8, dtype=torch.float64, device="cuda:0")
    out = torch.empty((8, 8), dtype=torch.float64, device="cuda:0")
    n = ctypes.c_size_t(0)
    assert lib.afqmc_mcd_workspace_size(8, 8, ctypes.byref(n)) == 0
    ws = torch.empty(n.value, dtype=torch.uint8, device="cuda:0")
    nv = ctypes.c_int32(-1)
    r = ctypes.c_double(0)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    args = lambda dim, delta, mv, nbytes: (dim, vp(V), delta, mv, vp(out), None,  # noqa: E731
                                           ctypes.byref(nv), ctypes.byref(r), vp(ws), nbytes, st)
    assert lib.afqmc_modified_cholesky(*args(8, 1e-6, 8, n.value - 1)) == -2  # ENOSPC
    assert lib.afqmc_modified_cholesky(*args(8, 0.0, 8, n.value)) == -1
    assert lib.afqmc_modified_cholesky(*args(8, float("nan"), 8, n.value)) == -1
    assert lib.afqmc_modified_cholesky(*args(0, 1e-6, 8, n.value)) == -1
    assert lib.afqmc_modified_cholesky(*args(8, 1e-6, 0, n.value)) == -1
    assert lib.afqmc_modified_cholesky(*args(8, 1e-6, 8, n.value)) == 0
    torch.cuda.synchronize()
    assert nv.value == 8 and np.allclose(out.cpu().numpy(), np.eye(8)[[0, 1, 2, 3, 4, 5, 6, 7]])


@pytest.mark.parametrize("M,G,delta", [(10, 30, 1e-8), (24, 120, 1e-6), (100, 500, 1e-6)])
def test_pair_space_matches_full_oracle(env, M, G, delta):
    """afqmc_modified_cholesky_pairs on the pair matrix gives the vectors and
    pivots the oracle finds on the full M^2 x M^2 matrix (rows (p, r) and
    (r, p) equal), the vectors exactly symmetric."""
    torch, pkg = env
    _, L, _ = workloads.hamiltonian(M, G, 3000 + M, l_scale=workloads.l_amplitude(M, G))
    W = workloads.interaction_pairs(L)
    idx = workloads.pair_expansion(M)
    want = mcd.modified_cholesky(W[idx][:, idx], delta)
    Lg, piv, resid = pkg.afqmc_modified_cholesky_pairs(torch.from_numpy(W).cuda(), M, delta,
                                                       G + 16)
    torch.cuda.synchronize()
    Lg = Lg.cpu().numpy()
    assert np.array_equal(Lg, Lg.transpose(0, 2, 1))
    piv = piv.cpu().numpy().astype(np.int64)
    assert np.all(piv // M <= piv % M)  # the lower index p*M + r of each pair
    compare((Lg.reshape(len(piv), M * M), piv, resid), want, M=M)
