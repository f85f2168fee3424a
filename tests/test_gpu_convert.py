"""The float64 <-> float32 conversions of the mixed path's FP32 kernels
(Theta rows, Gram-Schmidt, the half-step epilogues), written in integer
arithmetic after IEEE 754-2008 (round to nearest, ties to even; exact
widening), against the hardware conversions bit for bit: random values over
the whole exponent range, exact ties with even and odd results, the edges of
the float range (largest finite, rounding up to infinity, the smallest normal
and subnormal results), signed zeros, infinities and NaN."""
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
    import paper_1711_02242_gb300 as p

    return p, torch


def doubles():
    rng = np.random.default_rng(17)
    # random bit patterns with exponents spread over [-200, 200] around the float range
    sign = rng.integers(0, 2, 200000, dtype=np.uint64) << np.uint64(63)
    exp = rng.integers(1023 - 200, 1023 + 200, 200000).astype(np.uint64) << np.uint64(52)
    man = rng.integers(0, 1 << 52, 200000, dtype=np.uint64)
    x = (sign | exp | man).view(np.float64)
    # exact ties: low 29 mantissa bits = 1 << 28, kept bit 0 even or odd
    t_man = (rng.integers(0, 1 << 23, 4000, dtype=np.uint64) << np.uint64(29)) | np.uint64(1 << 28)
    t_exp = rng.integers(1023 - 120, 1023 + 120, 4000).astype(np.uint64) << np.uint64(52)
    ties = (t_exp | t_man).view(np.float64)
    f32 = np.finfo(np.float32)
    edges = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, float(f32.max),
                      float(f32.max) * (1 + 2.0 ** -25), float(f32.max) * (1 + 2.0 ** -24),
                      float(f32.tiny), float(f32.tiny) * (1 - 2.0 ** -30), 2.0 ** -149, 2.0 ** -150,
                      2.0 ** -151, 3.0 * 2.0 ** -151, 1e-300, -1e300, 2.0 ** 128, np.pi, -np.e])
    return np.concatenate([x, ties, -ties, edges])


def test_round_f32_matches_hardware(env):
    p, torch = env
    x = torch.from_numpy(doubles()).cuda()
    got = p.afqmc_round_f32(x).cpu().numpy()
    want = x.to(torch.float32).cpu().numpy()
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint32), want[~nan].view(np.uint32))
    # and the IEEE definition as numpy implements it
    ref = doubles().astype(np.float32)
    ok = ~np.isnan(ref)
    assert np.array_equal(got[ok].view(np.uint32), ref[ok].view(np.uint32))


def test_widen_f32_matches_hardware(env):
    p, torch = env
    rng = np.random.default_rng(5)
    bits = np.concatenate([rng.integers(0, 1 << 32, 300000, dtype=np.uint64).astype(np.uint32),
                           np.array([0, 0x80000000, 1, 0x807fffff, 0x00800000, 0x7f7fffff,
                                     0x7f800000, 0xff800000, 0x7fc00000], np.uint32)])
    x = torch.from_numpy(bits.view(np.float32)).cuda()
    got = p.afqmc_widen_f32(x).cpu().numpy()
    want = bits.view(np.float32).astype(np.float64)
    ok = ~np.isnan(want)
    assert np.array_equal(np.isnan(got), ~ok)
    assert np.array_equal(got[ok].view(np.uint64), want[ok].view(np.uint64))


def test_empty_and_bad_arguments(env):
    p, torch = env
    assert p.afqmc_round_f32(torch.empty(0, dtype=torch.float64, device="cuda")).numel() == 0
    import ctypes

    assert p.lib().afqmc_round_f32(None, None, 5, None) == -1
    assert p.lib().afqmc_widen_f32(None, None, -1, None) == -1
