"""Taylor expansion of exp(V) on the tensor cores (afqmc_taylor_series).

The reference repeats what the kernel is specified to do (Sec. 3.4.2 with the
operands in BF16/TF32): T_k = V T_{k-1} / k formed from the rounded operands
in float64, rounded to FP32 and then to the operand type before the next
product, and summed into S = T_1 + ... + T_n.  What is left between the two is FP32
accumulation order and the operand-rounding flips it causes: a term element
that lands on the other side of a BF16 (TF32) rounding boundary moves by one
unit of 2^-8 (2^-11) and carries that into the later terms.  Replaying the
reference with 3e-6 relative noise on every product (about FP32 accumulation
over K = 2 Mp) moves S by up to 1.1e-3 (BF16) and 1.5e-4 (TF32) per walker at
these sizes, so the bound is 3e-3 (BF16) and 6e-4 (TF32) relative per walker;
with |V| ~ 3 the last term alone is over 2e-2 of S (checked), so a dropped or
mis-signed term cannot pass.  Both routes (one launch for the whole series, one launch per
term) are checked, including walker counts above one CTA per SM, so CTAs
take several walkers in turn.
"""
import ctypes

import numpy as np
import pytest

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


def round_bf16(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def round_tf32(x):
    # round to nearest, ties away from zero, 10 explicit mantissa bits
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


def operands(rng, W, N, M, Mp, rnd):
    s = 1.5 / np.sqrt(M)
    V = s * (rng.standard_normal((W, M, M)) + 1j * rng.standard_normal((W, M, M)))
    T0 = (rng.standard_normal((W, M, N)) + 1j * rng.standard_normal((W, M, N))) / np.sqrt(M)
    Vr, Vi = rnd(V.real), rnd(V.imag)
    Tr, Ti = rnd(T0.real), rnd(T0.imag)
    dV = np.zeros((W, M, 2 * Mp), np.float32)
    dV[:, :, :M] = Vr
    dV[:, :, Mp:Mp + M] = Vi
    dT = np.zeros((W, 2 * N, 2 * Mp), np.float32)
    trT, tiT = np.swapaxes(Tr, 1, 2), np.swapaxes(Ti, 1, 2)  # [W][N][M]
    dT[:, :N, :M] = trT
    dT[:, :N, Mp:Mp + M] = -tiT
    dT[:, N:, :M] = tiT
    dT[:, N:, Mp:Mp + M] = trT
    Vlo = Vr.astype(np.float64) + 1j * Vi.astype(np.float64)
    Tlo = Tr.astype(np.float64) + 1j * Ti.astype(np.float64)
    return dV, dT, Vlo, Tlo


def reference(Vlo, Tlo, N, M, Mp, order, rnd):
    """S = T_1 + ... + T_n as [W][2N][Mp], and the last term's size relative to S."""
    acc = np.zeros((Vlo.shape[0], 2 * N, Mp))
    T = Tlo
    last = None
    for k in range(1, order + 1):
        D = Vlo @ T  # [W][M][N]
        sc = np.float32(1.0 / np.float32(k))
        tr = D.real.astype(np.float32) * sc
        ti = D.imag.astype(np.float32) * sc
        acc[:, :N, :M] += np.swapaxes(tr, 1, 2)
        acc[:, N:2 * N, :M] += np.swapaxes(ti, 1, 2)
        T = rnd(tr).astype(np.float64) + 1j * rnd(ti).astype(np.float64)
        last = np.sqrt((tr.astype(np.float64) ** 2 + ti.astype(np.float64) ** 2).sum(axis=(1, 2)))
    return acc, last / np.linalg.norm(acc.reshape(acc.shape[0], -1), axis=1)


def run(torch, pkg, dtype, dV, dT, W, N, M, Mp, lds, order, per_term):
    dev = torch.device("cuda:0")
    if dtype == 0:
        tV = torch.from_numpy(dV).to(dev).to(torch.bfloat16).contiguous()
        tT0 = torch.from_numpy(dT).to(dev).to(torch.bfloat16).contiguous()
    else:
        tV = torch.from_numpy(dV).to(dev)
        tT0 = torch.from_numpy(dT).to(dev)
    tT1 = torch.zeros_like(tT0)
    tS = torch.full((W, 2 * N, lds), 7.0, dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream(dev)
    rc = pkg.lib().afqmc_taylor_series(
        dtype, W, N, M, Mp, order, ctypes.c_void_p(tV.data_ptr()), ctypes.c_void_p(tT0.data_ptr()),
        ctypes.c_void_p(tT1.data_ptr()), ctypes.c_void_p(tS.data_ptr()), lds, per_term,
        ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(st.cuda_stream))
    assert rc == 0, pkg.lib().afqmc_last_error()
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return tS.cpu().numpy().astype(np.float64)


SHAPES = [  # dtype, W, N, M
    (0, 3, 3, 12),
    (0, 7, 10, 100),
    (0, 5, 25, 300),    # three 128-row tiles of p, ragged K block
    (1, 5, 25, 300),
    (0, 3, 64, 200),    # 128 operand rows
    (1, 3, 48, 300),    # TF32 term too large for shared memory: per-term route only
    (0, 400, 5, 60),    # more walkers than SMs: CTAs take walkers in turn
    (1, 333, 8, 130),
]


@pytest.mark.parametrize("dtype,W,N,M", SHAPES)
def test_taylor_series_matches_reference(env, dtype, W, N, M):
    torch, pkg = env
    rnd = round_bf16 if dtype == 0 else round_tf32
    Mp = (M + 15) // 16 * 16
    order = 6
    rng = np.random.default_rng(1000 + 7 * W + N + M + dtype)
    dV, dT, Vlo, Tlo = operands(rng, W, N, M, Mp, rnd)
    ref, last = reference(Vlo, Tlo, N, M, Mp, order, rnd)
    tol = 3e-3 if dtype == 0 else 6e-4
    lds = Mp + 16 * (W % 2)  # a padded pitch on some shapes
    # even the last term is well above the tolerance, so a lost term shows
    assert np.all(last > 5 * tol), last.min()
    for per_term in (0, 1):
        got = run(torch, pkg, dtype, dV, dT, W, N, M, Mp, lds, order, per_term)
        err = [np.linalg.norm(got[w, :, :M] - ref[w, :, :M]) / np.linalg.norm(ref[w])
               for w in range(W)]
        assert max(err) < tol, (per_term, int(np.argmax(err)), max(err))
        # columns p >= M are never written
        assert np.all(got[:, :, M:] == 7.0)


def test_taylor_series_rejects_bad_sizes(env):
    torch, pkg = env
    lib = pkg.lib()
    buf = torch.zeros(1 << 16, dtype=torch.float32, device="cuda:0")
    p = ctypes.c_void_p(buf.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # Mp not a multiple of 16, Mp < M, 2N > 128, bad dtype, order 0
    for args in [(0, 1, 2, 20, 20, 6), (0, 1, 2, 40, 32, 6), (0, 1, 65, 20, 32, 6),
                 (3, 1, 2, 20, 32, 6), (0, 1, 2, 20, 32, 0)]:
        assert lib.afqmc_taylor_series(*args, p, p, p, p, 32, 0, p, st) == -1  # AFQMC_EINVAL
    # sum pitch below Mp or not a multiple of 4
    for lds in (16, 34):
        assert lib.afqmc_taylor_series(0, 1, 2, 20, 32, 6, p, p, p, p, lds, 0, p, st) == -1
