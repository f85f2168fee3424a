"""afqmc_local_energies_noalloc: local energies with no device allocation.

Some callers cannot allocate device memory (their framework owns all of it
through its own pool, or an allocation would synchronise the device in the
middle of their stream work), so this entry point keeps its intermediate
results in a fixed array inside the library.  Its output must equal that of
afqmc_local_energies() on the same walkers, on two calls in a row (the second
call reuses the array the first one left behind).  This file is collected
last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import scf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_02242_gb300 as pkg

    f = pkg.lib().afqmc_local_energies_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32] * 4 + [ctypes.c_void_p] * 3 + [ctypes.c_double,
                                                                   ctypes.c_void_p, ctypes.c_void_p]
    return torch, pkg, f


def _operands(torch, w, h1, L, C, phi):
    """Lh, hh and Theta^T as the entry point takes them, from the caller's
    walkers (plain PyTorch float64 on the GPU)."""
    dev = torch.device("cuda")
    VT = torch.tensor(C, dtype=torch.float64, device=dev)
    Lh = torch.einsum("pi,gpq->giq", VT, torch.tensor(L, device=dev)).contiguous()
    hh = (VT.T @ torch.tensor(h1, device=dev)).contiguous()
    Phi = torch.tensor(phi, device=dev)
    theta = Phi @ torch.linalg.inv(VT.T.to(Phi.dtype) @ Phi)  # (W, M, N)
    thetaT = torch.stack([theta.real, theta.imag], 1).transpose(2, 3).contiguous()  # [W][2][N][M]
    return Lh, hh, thetaT


def _call(torch, f, w, nwalkers, Lh, hh, thetaT, H0, out):
    return f(w.M, w.N, w.nchol, nwalkers, Lh.data_ptr(), hh.data_ptr(), thetaT.data_ptr(), H0,
             out.data_ptr(), torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("name,nsteps", [("c0", 7), ("c1", 2)])
def test_noalloc_matches_workspace_entry_point(env, name, nsteps):
    torch, pkg, f = env
    w = workloads.config(name)
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed, H0=0.25,
                           energy_period=0)
    run = pkg.AfqmcRun(h1, L, C, p)
    run.propagate(nsteps)
    expected = run.local_energies()
    phi, _, _ = run.get_walkers()
    run.close()
    Lh, hh, thetaT = _operands(torch, w, h1, L, C, phi)
    outs = []
    for _ in range(2):
        out = torch.full((w.nwalkers, 2), float("nan"), dtype=torch.float64, device="cuda")
        pkg._check(_call(torch, f, w, w.nwalkers, Lh, hh, thetaT, 0.25, out))
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    for o in outs:
        got = o[:, 0] + 1j * o[:, 1]
        assert np.max(np.abs(got - expected) / np.abs(expected)) < 1e-10
    assert np.array_equal(outs[0], outs[1])


def _scratch_per_walker(N, nchol):
    """float64 of the fixed array one walker takes: the force-bias traces
    (2 nchol) and one complex exchange partial per block of Cholesky vectors,
    whose size follows the float64 exchange kernel's tiling (256 threads x 32
    outputs per block, 160 KB of shared memory holding a block's vectors in
    32-column panels plus two Theta panels)."""
    gc = (256 * 32) // (2 * N * N)
    cap = (160 * 1024 // 8 - 2 * N * (32 + 1)) // (N * 32)
    gc = max(1, min(gc, cap, nchol))
    return 2 * nchol + 2 * (-(-nchol // gc))


def test_noalloc_boundary_of_the_array(env):
    """The largest walker count the 2^21-float64 array holds runs and matches
    afqmc_local_energies; one walker more returns ENOSPC and launches
    nothing."""
    torch, pkg, f = env
    w = workloads.config("c0")
    wmax = (1 << 21) // _scratch_per_walker(w.N, w.nchol)
    assert wmax * _scratch_per_walker(w.N, w.nchol) <= 1 << 21
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    p = pkg.default_params(w.M, w.N, w.nchol, wmax, dt=w.dt, seed=w.seed, energy_period=0)
    run = pkg.AfqmcRun(h1, L, C, p)
    run.propagate(2)
    expected = run.local_energies()
    phi, _, _ = run.get_walkers()
    run.close()
    Lh, hh, thetaT = _operands(torch, w, h1, L, C, phi)
    out = torch.full((wmax, 2), float("nan"), dtype=torch.float64, device="cuda")
    pkg._check(_call(torch, f, w, wmax, Lh, hh, thetaT, 0.0, out))
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    got = o[:, 0] + 1j * o[:, 1]
    assert np.max(np.abs(got - expected) / np.abs(expected)) < 1e-10
    # one more walker (operands sized for it) is refused before any launch
    big = torch.zeros((wmax + 1) * 2 * w.N * w.M, dtype=torch.float64, device="cuda")
    out1 = torch.zeros((wmax + 1) * 2, dtype=torch.float64, device="cuda")
    n0 = pkg.afqmc_launch_count()
    rc = _call(torch, f, w, wmax + 1, Lh, hh, big, 0.0, out1)
    assert rc == -2  # AFQMC_ENOSPC
    assert pkg.afqmc_launch_count() == n0


def test_noalloc_rejects_sizes_beyond_the_array(env):
    torch, pkg, f = env
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    n0 = pkg.afqmc_launch_count()
    rc = f(300, 25, 1800, 4096, x.data_ptr(), x.data_ptr(), x.data_ptr(), 0.0, x.data_ptr(), st)
    assert rc == -2  # AFQMC_ENOSPC, nothing launched
    assert b"fixed array" in pkg.lib().afqmc_last_error()
    # more walkers than the exchange grid takes: refused, nothing launched
    rc = f(12, 1, 1, 70000, x.data_ptr(), x.data_ptr(), x.data_ptr(), 0.0, x.data_ptr(), st)
    assert rc == -1  # AFQMC_EINVAL
    assert pkg.afqmc_launch_count() == n0
