"""Mixed-precision path (tcgen05 BF16/TF32 contractions, FP32 propagation,
FP64 overlaps/weights/QR) against the FP64 path on identical fields.

The FP64 path is itself held to the oracle at 1e-10 (test_gpu_parity), so
these tolerances measure the rounding of the mixed path only: BF16 inputs
carry a relative error of 2^-9, TF32 inputs 2^-11, FP32 propagation 2^-24.
"""
import numpy as np
import pytest

import workloads
from oracle import scf

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


def runs(pkg, w, precisions, nwalkers=None, **kw):
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    out = {}
    for prec in precisions:
        p = pkg.default_params(w.M, w.N, w.nchol, nwalkers or w.nwalkers, dt=w.dt, seed=w.seed,
                               qr_period=w.qr_period, precision=prec, **kw)
        out[prec] = pkg.AfqmcRun(h1, L, C, p)
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,tol", [(2, 3e-3), (1, 4e-4)])
def test_trial_energy_mixed_vs_fp64(pkg, prec, tol):
    """E_loc at the trial (Eqs. localenergy2/3): force bias and exchange
    contractions on the tensor cores, ragged tiles (N=10: 12 vectors and 12
    walkers per tile; 500 vectors, 1024 walkers)."""
    w = workloads.config("c1")
    r = runs(pkg, w, [0, prec], energy_period=0)
    e64 = r[0].local_energies()
    emx = r[prec].local_energies()
    assert np.max(np.abs(emx - e64) / np.abs(e64)) < tol
    assert r[prec].info().status == 0


@pytest.mark.parametrize("prec,tol_phi,tol_e", [(2, 3e-2, 5e-3), (1, 5e-3, 5e-4)])
@pytest.mark.parametrize("nwalkers", [32, 200, 400, 520])
def test_one_step_mixed_vs_fp64(pkg, prec, tol_phi, tol_e, nwalkers):
    """One full step of the 12-orbital workload on identical Philox fields;
    200 walkers put field rows in both halves of a 256-row V tile and in a
    ragged last tile.  With an even number of 256-row V tiles (200, 400
    walkers) the V contraction runs on CTA pairs sharing the Cholesky tile by
    multicast, with an odd number (32, 520) on single CTAs."""
    w = workloads.config("c0")
    r = runs(pkg, w, [0, prec], nwalkers=nwalkers, energy_period=1)
    for x in r.values():
        x.propagate(1)
    p64, w64, _ = r[0].get_walkers()
    pmx, wmx, _ = r[prec].get_walkers()
    alive = np.nonzero(w64 != 0)[0]
    assert alive.size > nwalkers // 2
    assert rel(pmx[alive], p64[alive]) < tol_phi
    e64 = r[0].energy_log()[-1, 1]
    emx = r[prec].energy_log()[-1, 1]
    assert abs(emx - e64) < tol_e * abs(e64)
    assert r[prec].info().status == 0


def test_mixed_full_size_runs_clean(pkg):
    """M=300, N=25, 1800 vectors, 512 walkers: set-up and two steps in BF16
    with an energy evaluation; the tensor-core status word stays 0 and the
    trial energy matches the FP64 set-up to BF16 accuracy."""
    w = workloads.config("c2")
    h1, L, _ = w.hamiltonian()
    C = np.linalg.eigh(h1)[1][:, :w.N]
    p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed, precision=2,
                           energy_period=2)
    run = pkg.AfqmcRun(h1, L, C, p)
    e_mixed_trial = run.local_energies()[0]
    run.propagate(2)
    info = run.info()
    assert info.status == 0 and info.step == 2
    assert run.energy_log().shape[0] == 1
    p64 = pkg.default_params(w.M, w.N, w.nchol, 4, dt=w.dt, seed=w.seed, energy_period=0)
    r64 = pkg.AfqmcRun(h1, L, C, p64)
    e64 = r64.local_energies()[0]
    assert abs(e_mixed_trial - e64) < 5e-3 * abs(e64)


@pytest.mark.parametrize("prec,tol_bias,tol_phi", [(2, 4e-3, 8e-3), (1, 2e-3, 2e-3)])
def test_mixed_weights_carry_no_common_drift(pkg, prec, tol_bias, tol_phi):
    """Seven steps of the mixed and float64 paths on the same fields: the
    ratio of each walker's weight to its float64 value stays 1 on average.
    B_half = exp(-dt v0'/2) has a diagonal close to 1; rounded to BF16/TF32 it
    would scale every walker's orbitals by the same factor each step (a
    common weight drift of about -1 %/step in BF16), so the half steps apply
    it as I + (B_half - I) with the identity part exact."""
    h1, L, _ = workloads.hamiltonian(24, 120, 6100, l_scale=workloads.l_amplitude(24, 120))
    C, _, _, _ = scf.rhf(h1, L, 4)
    out = []
    for precision in (0, prec):
        p = pkg.default_params(24, 4, 120, 64, dt=0.01, seed=4, qr_period=5, energy_period=1,
                               precision=precision)
        run = pkg.AfqmcRun(h1, L, C, p)
        run.propagate(7)
        out.append(run.get_walkers())
        assert run.info().status == 0
        run.close()
    (phi0, w0, _), (phi1, w1, _) = out
    alive = np.nonzero((w0 != 0) & (w1 != 0))[0]
    assert alive.size > 32
    ratio = (w1[alive] / w0[alive]).real
    assert abs(np.mean(ratio) - 1) < tol_bias
    d = np.linalg.norm((phi1 - phi0)[alive].reshape(alive.size, -1), axis=1)
    n = np.linalg.norm(phi0[alive].reshape(alive.size, -1), axis=1)
    assert np.max(d / n) < tol_phi


def _seven_steps(pkg, precisions):
    h1, L, _ = workloads.hamiltonian(24, 120, 6100, l_scale=workloads.l_amplitude(24, 120))
    C, _, _, _ = scf.rhf(h1, L, 4)
    out = []
    for precision in precisions:
        p = pkg.default_params(24, 4, 120, 64, dt=0.01, seed=4, qr_period=5, energy_period=1,
                               precision=precision)
        run = pkg.AfqmcRun(h1, L, C, p)
        e0 = run.local_energies()
        run.propagate(7)
        out.append((e0, run.get_walkers(), run.energy_log()))
        assert run.info().status == 0
        run.close()
    return out


@pytest.mark.parametrize("base,prec32,tol_phi", [(6, 4, 1e-2), (5, 3, 3e-3)])
def test_f32lu_precisions_close_to_float64_lu(pkg, base, prec32, tol_phi):
    """The opt-in _F32LU precisions (the elimination, Theta and Gram-Schmidt
    in FP32; log det sums, overlap ratios and weights in float64) against the
    same mixed precision with those steps in float64: seven steps on
    identical fields differ by FP32 rounding fed through the BF16/TF32
    contractions, with no common weight drift."""
    (e0a, (pa, wa, _), la), (e0b, (pb, wb, _), lb) = _seven_steps(pkg, (base, prec32))
    assert np.max(np.abs(e0b - e0a) / np.abs(e0a)) < 1e-5
    alive = np.nonzero((wa != 0) & (wb != 0))[0]
    assert alive.size > 32
    d = np.linalg.norm((pb - pa)[alive].reshape(alive.size, -1), axis=1)
    n = np.linalg.norm(pa[alive].reshape(alive.size, -1), axis=1)
    assert np.max(d / n) < tol_phi
    assert abs(np.mean((wb[alive] / wa[alive]).real) - 1) < 2e-3
    assert np.max(np.abs(lb[:, 1] - la[:, 1]) / np.abs(la[:, 1])) < 2e-4


@pytest.mark.parametrize("base,prec,tol_phi", [(6, 2, 2e-3), (5, 1, 5e-4)])
def test_fp32_theta_close_to_float64_theta(pkg, base, prec, tol_phi):
    """The default mixed precisions form Theta = Phi S^-1 in FP32 from the
    float64 S^-1 (the elimination, log det, overlap ratios, weights and
    Gram-Schmidt stay float64): seven steps on identical fields against the
    same precision with Theta formed in float64.  Theta only reaches the
    BF16/TF32 operands and the one-body trace, so the walks agree to far
    below the operand rounding, the weights carry no common drift, and the
    overlaps (float64 on both sides) agree to the walkers' difference."""
    (e0a, (pa, wa, la_ov), la), (e0b, (pb, wb, lb_ov), lb) = _seven_steps(pkg, (base, prec))
    assert np.max(np.abs(e0b - e0a) / np.abs(e0a)) < 1e-7
    alive = np.nonzero((wa != 0) & (wb != 0))[0]
    assert alive.size > 32
    d = np.linalg.norm((pb - pa)[alive].reshape(alive.size, -1), axis=1)
    n = np.linalg.norm(pa[alive].reshape(alive.size, -1), axis=1)
    assert np.max(d / n) < tol_phi
    assert abs(np.mean((wb[alive] / wa[alive]).real) - 1) < 1e-3
    assert np.max(np.abs(lb[:, 1] - la[:, 1]) / np.abs(la[:, 1])) < 5e-5


@pytest.mark.parametrize("prec", [2, 1])
def test_mixed_energies_after_comb_and_restore_match_fresh_evaluation(pkg, prec):
    """The comb moves walkers (orbitals, Theta, overlaps) between slots and a
    checkpoint restore replaces them: the local energies the state then
    evaluates (force bias and exchange from the BF16/TF32 operand copies)
    equal those of a state given the same walkers by set_walkers, which
    recomputes every operand from the orbitals (to the last bits of the
    basis rotation set_walkers applies: an operand whose BF16/TF32 rounding
    flips moves an energy by far less than 2e-5 relative, a stale operand of
    a copied walker by orders of magnitude more); after the restore the
    energies are bitwise those before the save."""
    w = workloads.config("c0")
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    kw = dict(dt=w.dt, seed=w.seed, qr_period=0, energy_period=0, precision=prec)
    run = pkg.AfqmcRun(h1, L, C, pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, pc_period=3,
                                                    **kw))
    fresh = pkg.AfqmcRun(h1, L, C, pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, **kw))
    run.propagate(3)  # ends with a comb
    phi, wt, _ = run.get_walkers()
    assert len(set(np.round(np.abs(phi[:, 0, 0]), 12))) < w.nwalkers  # copies were made
    e_run = run.local_energies()
    fresh.set_walkers(phi, wt)
    e_fresh = fresh.local_energies()
    assert np.max(np.abs(e_run - e_fresh) / np.abs(e_fresh)) < 2e-5
    blob = run.save()
    run.propagate(2)
    run.load(blob)
    assert np.array_equal(run.local_energies(), e_run)
