"""Back-propagation estimators on the GPU (afqmc_bp_begin / afqmc_bp_end; Sec.
"Computing ground-state properties: the backpropagation algorithm", Eqs. bp,
bp_dets, BP-PRes weights) against the oracle's window on the same walk.

The float64 walk matches the oracle to 1e-10 step by step, so the recorded
fields and weights are the same; the back-propagated density matrices (BP-PRes
and BP-PhL), their weight sums and the window length must then agree to
1e-9 of the largest element.  Cases: the 12-orbital workload over a window
that crosses two Gram-Schmidt steps, a ragged shape (odd N, nchol, walker
count, QR every 3 steps, energies every 2 so the window evaluates local
energies on its own), an empty window (the mixed estimator), a window with
population control inside it (copies carry their parents' paths), free projection
(no restoration factor), a walk that keeps going after the window (unchanged
by it, with and without graph replay), and the argument and state errors.
The mixed path's window (BF16/TF32 fields and tensor-core backward sweep) is
held to the float64 path's on the same system within the operand rounding
(measured 8e-4 BF16, 2e-4 TF32 of the largest element; bound 4e-3 / 1e-3).
"""
import numpy as np
import pytest

import workloads
from oracle import afqmc, scf

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_02242_gb300 as p

    return p


def make_pair(pkg, M, N, G, W, seed=4, mode="phaseless", qr=5, ep=1, dt=0.01, bp_steps=32,
              use_graph=0, stream=None, pc=0):
    h1, L, _ = workloads.hamiltonian(M, G, 6000 + M + N, l_scale=workloads.l_amplitude(M, G))
    C, _, conv, _ = scf.rhf(h1, L, N)
    assert conv
    op = dict(dt=dt, seed=seed, qr_period=qr, energy_period=ep, mode=mode, pc_period=pc)
    orc = afqmc.Oracle(h1, L, C, W, afqmc.Params(**op))
    gp = dict(op)
    gp["mode"] = pkg.AFQMC_FREE if mode == "free" else pkg.AFQMC_PHASELESS
    p = pkg.default_params(M, N, G, W, bp_steps=bp_steps, use_graph=use_graph, **gp)
    run = pkg.AfqmcRun(h1, L, C, p, stream=stream)
    return orc, run


def check(got, want):
    rho, phl, wp, w, m = got
    orho, ophl, owp, ow, _ = want
    scale = max(np.max(np.abs(orho)), 1.0)
    assert np.max(np.abs(rho - orho)) < TOL * scale, np.max(np.abs(rho - orho))
    assert np.max(np.abs(phl - ophl)) < TOL * scale, np.max(np.abs(phl - ophl))
    assert abs(wp - owp) < TOL * abs(owp) and abs(w - ow) < TOL * abs(ow)
    # and the estimator is a density: Hermitian up to noise, trace 2N
    return m


@pytest.mark.parametrize("M,N,G,W,n,m,qr,ep,pc", [
    (12, 3, 48, 32, 4, 10, 5, 1, 0),
    (20, 7, 33, 50, 3, 7, 3, 2, 0),
    (16, 4, 40, 24, 2, 0, 5, 1, 0),   # empty window: the mixed estimator
    (12, 3, 48, 32, 2, 9, 4, 1, 3),   # combs inside the window carry the paths
])
def test_window_matches_oracle(pkg, M, N, G, W, n, m, qr, ep, pc):
    orc, run = make_pair(pkg, M, N, G, W, qr=qr, ep=ep, pc=pc)
    orc.run(n)
    run.propagate(n)
    orc.bp_begin()
    run.bp_begin()
    orc.run(m)
    run.propagate(m)
    want = orc.bp_end()
    got = run.bp_end()
    assert got[4] == m
    check(got, want)
    assert abs(np.trace(got[1]).real - 2 * N) < 1e-8
    assert np.count_nonzero(orc.weight) > W // 2  # most walkers alive: a real test
    run.close()


def test_free_projection_window(pkg):
    orc, run = make_pair(pkg, 12, 3, 48, 16, mode="free", qr=5, ep=0)
    orc.run(3)
    run.propagate(3)
    orc.bp_begin()
    run.bp_begin()
    orc.run(8)
    run.propagate(8)
    got = run.bp_end()
    check(got, orc.bp_end())
    assert np.max(np.abs(got[0] - got[1])) < 1e-12  # no restoration factor
    run.close()


def test_walk_continues_unchanged(pkg):
    """A window does not change the walk (graph replay is suspended while it is
    open): walkers and energies after it equal a run without one."""
    import torch

    st = torch.cuda.Stream()
    _, a = make_pair(pkg, 12, 3, 48, 32, ep=5, use_graph=1, stream=st)
    _, b = make_pair(pkg, 12, 3, 48, 32, ep=5, use_graph=1, stream=st)
    a.propagate(5)
    b.propagate(5)
    a.bp_begin()
    a.propagate(10)
    a.bp_end()
    b.propagate(10)
    a.propagate(5)
    b.propagate(5)
    pa, wa, la = a.get_walkers()
    pb, wb, lb = b.get_walkers()
    assert np.array_equal(pa, pb) and np.array_equal(wa, wb) and np.array_equal(la, lb)
    assert np.array_equal(a.energy_log(), b.energy_log())
    a.close()
    b.close()


def test_errors(pkg):
    h1, L, _ = workloads.hamiltonian(12, 48, 7, l_scale=0.5)
    C, _, _, _ = scf.rhf(h1, L, 3)
    run = pkg.AfqmcRun(h1, L, C, pkg.default_params(12, 3, 48, 8))
    with pytest.raises(pkg.AfqmcError, match="EINVAL"):
        run.bp_begin()  # no window buffers
    run.close()
    with pytest.raises(pkg.AfqmcError, match="EINVAL"):
        pkg.afqmc_workspace_size(pkg.default_params(12, 3, 48, 8, bp_steps=-1))
    run = pkg.AfqmcRun(h1, L, C, pkg.default_params(12, 3, 48, 8, bp_steps=4))
    with pytest.raises(pkg.AfqmcError, match="ESTATE"):
        run.bp_end()
    run.bp_begin()
    with pytest.raises(pkg.AfqmcError, match="ESTATE"):
        run.bp_begin()
    run.propagate(3)
    with pytest.raises(pkg.AfqmcError, match="ENOSPC"):
        run.propagate(2)  # 3 + 2 > 4
    run.propagate(1)
    assert run.bp_end()[4] == 4
    run.close()


@pytest.mark.parametrize("prec,tol", [(2, 4e-3), (1, 1e-3)])
def test_mixed_path_window_close_to_float64(pkg, prec, tol):
    """The mixed path's window (fields recorded as BF16/TF32 operands, backward
    sweep on the tensor cores, densities in float64) against the float64
    path's on the same system, seed and steps: the two walks differ by the
    operand rounding only, and so do the densities."""
    out = []
    for precision in (0, prec):
        h1, L, _ = workloads.hamiltonian(24, 120, 6100, l_scale=workloads.l_amplitude(24, 120))
        C, _, _, _ = scf.rhf(h1, L, 4)
        p = pkg.default_params(24, 4, 120, 64, dt=0.01, seed=3, qr_period=5, energy_period=1,
                               bp_steps=8, precision=precision)
        run = pkg.AfqmcRun(h1, L, C, p)
        run.propagate(3)
        run.bp_begin()
        run.propagate(6)
        out.append(run.bp_end())
        if precision == 0:
            run.bp_begin()  # empty window at the same step: the mixed estimator
            mixed_est = run.bp_end()[1]
        assert run.info().status == 0
        run.close()
    (r0, p0, w0, v0, _), (r1, p1, w1, v1, _) = out
    scale = np.max(np.abs(r0))
    d_pres = np.max(np.abs(r1 - r0)) / scale
    d_phl = np.max(np.abs(p1 - p0)) / scale
    d_bp = np.max(np.abs(p0 - mixed_est)) / scale
    print(f"mixed precision {prec}: BP-PRes {d_pres:.2e} BP-PhL {d_phl:.2e}; "
          f"back-propagated vs mixed estimator {d_bp:.2e}")
    assert d_pres < tol and d_phl < tol
    assert abs(np.trace(p1).real - 8) < 1e-8
    # six steps of back-propagation move the density by more than the rounding
    assert d_bp > 3 * max(d_pres, d_phl)
