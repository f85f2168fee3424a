"""Failure detection without a GPU fault.

Device side: a bounded wait on a flag that nothing sets gives up, writes
AFQMC_ETIMEOUT to a status word and returns; the context stays usable.
Host side: non-finite inputs, a short workspace and bad parameters are
rejected before the state is created (the Cholesky vectors by one pass on
the device after their upload, the smaller inputs on the host); walkers
whose weights overflow are zeroed and counted, never propagated as NaN into
the estimator.
"""
import ctypes
import math

import numpy as np
import pytest

import workloads

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


def test_bounded_wait_times_out_and_context_survives(env):
    torch, pkg = env
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    pkg._check(pkg.lib().afqmc_wait_flag(ctypes.c_void_p(flag.data_ptr()), 2000,
                                         ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(st)))
    torch.cuda.synchronize()
    assert int(status.item()) == -5  # AFQMC_ETIMEOUT
    # a set flag ends the wait at once and leaves the status alone
    flag.fill_(1)
    status.zero_()
    pkg._check(pkg.lib().afqmc_wait_flag(ctypes.c_void_p(flag.data_ptr()), 1 << 20,
                                         ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(st)))
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    # the context still works
    assert float((torch.ones(4, device="cuda") * 2).sum().item()) == 8.0


def test_overflowing_weights_are_zeroed_and_counted(env):
    torch, pkg = env
    w = workloads.config("c0")
    h1, L, _ = w.hamiltonian()
    L = 6.0 * L  # violent fields: weights overflow within a few steps
    C = np.linalg.eigh(h1)[1][:, :w.N]
    p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=0.05, seed=3, energy_period=1,
                           ecap_C=-1.0, wmax=math.inf)
    run = pkg.AfqmcRun(h1, L, C, p)
    run.propagate(20)
    info = run.info()
    _, wt, _ = run.get_walkers()
    assert np.all(np.isfinite(wt))
    assert info.nonfinite + np.count_nonzero(wt == 0) > 0
    assert info.status == 0
    log = run.energy_log()
    live = log[:, 3] > 0
    assert np.all(np.isfinite(log[live, 1]))


@pytest.mark.parametrize("where", ["L", "h1"])
def test_nonfinite_inputs_are_rejected_with_their_index(env, where):
    torch, pkg = env
    w = workloads.config("c0")
    h1, L, _ = w.hamiltonian()
    C = np.linalg.eigh(h1)[1][:, :w.N]
    p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers)
    for value in (np.nan, np.inf, -np.inf):
        h, l = h1.copy(), L.copy()
        if where == "L":
            idx = (w.nchol - 3) * w.M * w.M + 5 * w.M + 7  # a late vector
            l.reshape(-1)[idx] = value
            l.reshape(-1)[idx + 11] = value  # the first bad index is named
        else:
            idx = 2 * w.M + 1
            h.reshape(-1)[idx] = value
        with pytest.raises(pkg.AfqmcError, match=rf"{where}\[{idx}\] is not finite"):
            pkg.AfqmcRun(h, l, C, p)
    # the device is usable afterwards, and the clean inputs set up
    run = pkg.AfqmcRun(h1, L, C, p)
    assert run.info().status == 0
    run.close()
