"""A single contraction of the M=300 step, for kernel profiling.

    python -m paper_1711_02242_gb300.profile_case [--case v|fb|taylor|mcd|bp|md] [--dtype bf16|tf32|fp64]
                                                  [--reps 3] [--walkers 512] [--orbitals 300]
                                                  [--window 20]

Case "v": V = sum_g x_g L_g as afqmc_contract with the M=300 shapes
(A = 1024 x 1800 fields, B = 45150 x 1800 packed Cholesky vectors, C FP32):
about 350 MB on the device, B alone (162 MB BF16) larger than the 129 MB L2.
Case "fb": the force-bias contraction (A = 1024 x 7600, B = 1800 x 7600).
Case "taylor": the sixth-order Taylor series of exp(V) on 512 walkers with
M = 300, N = 25 (afqmc_taylor_series; V is 187 MB in BF16).
Case "mcd": the modified Cholesky decomposition over index pairs
(afqmc_modified_cholesky_pairs, delta = 1e-6) of the interaction of the seeded
Hamiltonian with `--orbitals` M orbitals and 6M vectors (the pair matrix is
16.3 GB at M = 300, 1.3 GB at M = 160); one launch per vector.
Case "md": the walk of the M=100 workload (10+10 electrons, 500 vectors, 1024
walkers) in the `--dtype` precision with a trial of 1, 2 and 4 non-orthogonal
determinants (rotations of the RHF determinant): time per step and per energy
evaluation.
Case "bp": the M=300 walk (512 walkers, 1800 vectors, RHF trial) with a
back-propagation window of `--window` steps: time per step without and with
the window open, and the time of afqmc_bp_end (backward sweep and densities).
Random operands; prints the mean time per launch from CUDA events.
"""
from __future__ import annotations

import argparse
import ctypes

import numpy as np

import paper_1711_02242_gb300 as pkg


def main():
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="v", choices=["v", "fb", "taylor", "mcd", "bp", "md"])
    ap.add_argument("--window", type=int, default=20)
    ap.add_argument("--orbitals", type=int, default=300)
    ap.add_argument("--walkers", type=int, default=512)
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "tf32", "fp64"])
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    from paper_1711_02242_gb300 import build as b

    b.build()
    if a.case == "taylor":
        return taylor(a)
    if a.case == "mcd":
        return mcd(a)
    if a.case == "bp":
        return bp(a)
    if a.case == "md":
        return md(a)
    if a.case == "v":
        m, n, k, pitch = 1024, 45150, 1800, 1800
    else:
        m, n, k, pitch = 1024, 1800, 25 * 304, 25 * 304
    dt = torch.bfloat16 if a.dtype == "bf16" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((m, pitch), generator=g, device="cuda").to(dt)
    B = torch.randn((n, pitch), generator=g, device="cuda").to(dt)
    ldc = (n + 3) // 4 * 4
    C = torch.empty((m, ldc), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    lib = pkg.lib()

    def call():
        pkg._check(lib.afqmc_contract(0 if a.dtype == "bf16" else 1, m, n, k,
                                      ctypes.c_void_p(A.data_ptr()), pitch,
                                      ctypes.c_void_p(B.data_ptr()), pitch, ctypes.c_float(1.0),
                                      ctypes.c_void_p(C.data_ptr()), ldc,
                                      ctypes.c_void_p(st.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream)))

    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    flops = 2.0 * m * n * k
    print(f"case {a.case} {a.dtype}: m={m} n={n} k={k}: {ms:.4f} ms/launch, "
          f"{flops / ms / 1e9:.1f} TFLOP/s, status {int(st.item())}")
    assert int(st.item()) == 0


def taylor(a):
    import torch

    W, N, M, Mp, order = a.walkers, 25, 300, 304, 6
    dt = torch.bfloat16 if a.dtype == "bf16" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(0)
    V = torch.zeros((W, M, 2 * Mp), device="cuda")
    V[:, :, :M] = torch.randn((W, M, M), generator=g, device="cuda") * (0.05 / M ** 0.5)
    V[:, :, Mp:Mp + M] = torch.randn((W, M, M), generator=g, device="cuda") * (0.05 / M ** 0.5)
    V = V.to(dt)
    T0 = torch.zeros((W, 2 * N, 2 * Mp), device="cuda")
    T0[:, :, :M] = torch.randn((W, 2 * N, M), generator=g, device="cuda")
    T0 = T0.to(dt)
    T1 = torch.empty_like(T0)
    S = torch.empty((W, 2 * N, Mp), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    lib = pkg.lib()

    def call():
        pkg._check(lib.afqmc_taylor_series(0 if a.dtype == "bf16" else 1, W, N, M, Mp, order,
                                           ctypes.c_void_p(V.data_ptr()),
                                           ctypes.c_void_p(T0.data_ptr()),
                                           ctypes.c_void_p(T1.data_ptr()),
                                           ctypes.c_void_p(S.data_ptr()), Mp, 0,
                                           ctypes.c_void_p(st.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream)))

    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    vbytes = V.numel() * V.element_size()
    print(f"case taylor {a.dtype}: W={W} N={N} M={M} order={order}: {ms:.4f} ms/launch, "
          f"V {vbytes / 1e6:.0f} MB once from HBM: {vbytes / ms / 1e6:.0f} GB/s, "
          f"V per term (L2): {order * vbytes / ms / 1e6:.0f} GB/s, status {int(st.item())}")
    assert int(st.item()) == 0


def mcd(a):
    import torch

    import workloads

    M = a.orbitals
    G = 6 * M
    _, L, _ = workloads.hamiltonian(M, G, 5000 + M, l_scale=workloads.l_amplitude(M, G))
    W = workloads.interaction_pairs_device(L)
    del L
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Lv, piv, resid = pkg.afqmc_modified_cholesky_pairs(W, M, 1e-6, G + 16)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    n = Lv.shape[0]
    print(f"case mcd M={M} pairs={W.shape[0]} vectors={n} residual={resid:.3e} "
          f"ms={min(times):.3f} per-vector-us={1e3 * min(times) / n:.2f}")


def bp(a):
    import time

    import torch

    import workloads
    from paper_1711_02242_gb300.rhf import rhf_trial

    w = workloads.config("c2")
    h1, L, H0 = w.hamiltonian()
    C, _, _ = rhf_trial(h1, L, w.N, max_iter=25)
    prec = {"fp64": 0, "tf32": 1, "bf16": 2}[a.dtype]
    m = a.window
    p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed, H0=H0,
                           qr_period=w.qr_period, energy_period=w.energy_period, precision=prec,
                           bp_steps=m)
    st = torch.cuda.Stream()
    run = pkg.AfqmcRun(h1, L, C, p, stream=st)
    run.propagate(10)
    st.synchronize()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        st.synchronize()
        return e0.elapsed_time(e1)

    t_plain = timed(lambda: run.propagate(m))
    run.bp_begin()
    t_window = timed(lambda: run.propagate(m))
    t0 = time.perf_counter()
    rho, phl, wp, wsum, n = run.bp_end()
    t_end = 1e3 * (time.perf_counter() - t0)
    print(f"case bp {a.dtype} M={w.M} walkers={w.nwalkers} window={n}: "
          f"ms/step plain={t_plain / m:.3f} window-open={t_window / m:.3f}; "
          f"bp_end ms={t_end:.2f}; trace(rho_PRes)={np.trace(rho).real:.6f} "
          f"|sum W F|/sum W={abs(wp) / abs(wsum):.4f}; status={run.info().status}")
    run.close()


def md(a):
    import scipy.linalg as sla
    import torch

    import workloads
    from paper_1711_02242_gb300.rhf import rhf_trial

    w = workloads.config("c1")
    h1, L, H0 = w.hamiltonian()
    C, _, _ = rhf_trial(h1, L, w.N, max_iter=25)
    rng = np.random.default_rng(11)
    q, _ = np.linalg.qr(np.hstack([C, rng.standard_normal((w.M, w.M - w.N))]))
    basis = np.hstack([C, q[:, w.N:]])

    def rotated():
        K = 0.02 * rng.standard_normal((w.M, w.M))
        return basis @ sla.expm(K - K.T)[:, :w.N]

    st = torch.cuda.Stream()
    steps = 10
    for nd in (1, 2, 4):
        up = np.array([C] + [rotated() for _ in range(nd - 1)])
        dn = np.array([C] + [rotated() for _ in range(nd - 1)])
        coef = np.array([1.0] + [0.3 / nd] * (nd - 1), np.complex128)
        p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed, H0=H0,
                               qr_period=w.qr_period, energy_period=0, ndet=nd,
                               precision={"fp64": 0, "tf32": 1, "bf16": 2}[a.dtype])
        run = pkg.AfqmcRun(h1, L, (coef, up, dn), p, stream=st)
        run.propagate(2)
        st.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        run.propagate(steps)
        e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1) / steps
        import time

        t0 = time.perf_counter()
        run.local_energies()
        te = 1e3 * (time.perf_counter() - t0)
        print(f"case md {a.dtype} M={w.M} N={w.N} nchol={w.nchol} walkers={w.nwalkers} ndet={nd}: "
              f"ms/step={ms:.2f} walker-steps/s={w.nwalkers / ms * 1e3:.0f} energy-eval ms={te:.2f} "
              f"status={run.info().status} alive={run.info().alive}")
        run.close()


if __name__ == "__main__":
    main()

