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

    dev = torch.device("cuda")
    VT = torch.tensor(C, dtype=torch.float64, device=dev)
    Lh = torch.einsum("pi,gpq->giq", VT, torch.tensor(L, device=dev)).contiguous()
    hh = (VT.T @ torch.tensor(h1, device=dev)).contiguous()
    Phi = torch.tensor(phi, device=dev)
    theta = Phi @ torch.linalg.inv(VT.T.to(Phi.dtype) @ Phi)  # (W, M, N)
    thetaT = torch.stack([theta.real, theta.imag], 1).transpose(2, 3).contiguous()  # [W][2][N][M]
    st = torch.cuda.current_stream()
    outs = []
    for _ in range(2):
        out = torch.full((w.nwalkers, 2), float("nan"), dtype=torch.float64, device=dev)
        rc = f(w.M, w.N, w.nchol, w.nwalkers, Lh.data_ptr(), hh.data_ptr(), thetaT.data_ptr(),
               0.25, out.data_ptr(), st.cuda_stream)
        pkg._check(rc)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    for o in outs:
        got = o[:, 0] + 1j * o[:, 1]
        assert np.max(np.abs(got - expected) / np.abs(expected)) < 1e-10
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_sizes_beyond_the_array(env):
    torch, pkg, f = env
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = f(300, 25, 1800, 4096, x.data_ptr(), x.data_ptr(), x.data_ptr(), 0.0, x.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert rc == -2  # AFQMC_ENOSPC, nothing launched
    assert b"fixed array" in pkg.lib().afqmc_last_error()
