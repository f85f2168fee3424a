"""Python binding of libafqmc.so, the GB300 phaseless-AFQMC library.

Argument marshalling only: every step of the walk runs in the library's CUDA
kernels.  PyTorch provides the device workspace (a uint8 tensor) and the CUDA
stream.  The functions keep the C names of ``include/afqmc.h``; ``AfqmcRun``
wraps one state.

There is no CPU fallback: if the library has not been built (``build()``),
``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libafqmc.so")

AFQMC_OK = 0
# the mixed paths keep S^-1, log det, overlap ratios, weights and
# Gram-Schmidt in float64 and form Theta = Phi S^-1 in FP32
AFQMC_FP64, AFQMC_MIXED_TF32, AFQMC_MIXED_BF16 = 0, 1, 2
# the mixed paths with S^-1, Theta and Gram-Schmidt in FP32 (opt-in)
AFQMC_MIXED_TF32_F32LU, AFQMC_MIXED_BF16_F32LU = 3, 4
# the mixed paths with Theta = Phi S^-1 also in float64
AFQMC_MIXED_TF32_F64THETA, AFQMC_MIXED_BF16_F64THETA = 5, 6
AFQMC_PHASELESS, AFQMC_FREE = 0, 1
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOSPC", -3: "ENONFINITE", -4: "ECUDA",
          -5: "ETIMEOUT", -6: "ESTATE", -7: "EUNSUPPORTED"}

EXPORTED = ["afqmc_default_params", "afqmc_workspace_size", "afqmc_init", "afqmc_propagate",
            "afqmc_energy", "afqmc_local_energies", "afqmc_get_walkers", "afqmc_set_walkers",
            "afqmc_get_energy_log", "afqmc_get_info", "afqmc_save", "afqmc_load",
            "afqmc_destroy", "afqmc_last_error", "afqmc_launch_count",
            "afqmc_philox4x32_10", "afqmc_gaussian_fields", "afqmc_contract",
            "afqmc_profile_start", "afqmc_profile_stop", "afqmc_local_energies_noalloc",
            "afqmc_group_create", "afqmc_group_propagate", "afqmc_group_destroy",
            "afqmc_group_set_grouped", "afqmc_group_tiles",
            "afqmc_wait_flag", "afqmc_taylor_series", "afqmc_mcd_workspace_size",
            "afqmc_modified_cholesky", "afqmc_mcd_pairs_workspace_size",
            "afqmc_modified_cholesky_pairs", "afqmc_bp_begin", "afqmc_bp_end",
            "afqmc_init_multidet", "afqmc_round_f32", "afqmc_widen_f32",
            "afqmc_walker_row_bytes", "afqmc_export_weights", "afqmc_comb_plan",
            "afqmc_pack_walkers", "afqmc_unpack_walkers", "afqmc_energy_sums"]


class Params(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("N", ctypes.c_int32), ("nchol", ctypes.c_int32),
                ("nwalkers", ctypes.c_int32), ("dt", ctypes.c_double),
                ("e_shift", ctypes.c_double), ("H0", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("taylor_order", ctypes.c_int32),
                ("qr_period", ctypes.c_int32), ("pc_period", ctypes.c_int32),
                ("energy_period", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("ecap_C", ctypes.c_double),
                ("fb_cap", ctypes.c_double), ("wmax", ctypes.c_double),
                ("max_records", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("bp_steps", ctypes.c_int32), ("ndet", ctypes.c_int32),
                ("Ndn", ctypes.c_int32), ("walker0", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("E_T", ctypes.c_double), ("H0p", ctypes.c_double),
                ("e_shift", ctypes.c_double), ("wmax", ctypes.c_double),
                ("step", ctypes.c_int64), ("nonfinite", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("alive", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class AfqmcError(RuntimeError):
    pass


_lib = None


def lib():
    """Load libafqmc.so (built by ``build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise AfqmcError(f"{LIB_PATH} is not built; run paper_1711_02242_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    vp = ctypes.c_void_p
    sig = {
        "afqmc_default_params": (None, [P(Params)]),
        "afqmc_workspace_size": (ctypes.c_int, [P(Params), P(ctypes.c_size_t)]),
        "afqmc_init": (ctypes.c_int, [P(Params), dp, dp, dp, dp, vp, ctypes.c_size_t, vp,
                                      P(vp)]),
        "afqmc_propagate": (ctypes.c_int, [vp, ctypes.c_int32]),
        "afqmc_energy": (ctypes.c_int, [vp, dp, dp]),
        "afqmc_local_energies": (ctypes.c_int, [vp, dp]),
        "afqmc_get_walkers": (ctypes.c_int, [vp, dp, dp, dp]),
        "afqmc_set_walkers": (ctypes.c_int, [vp, dp, dp]),
        "afqmc_get_energy_log": (ctypes.c_int, [vp, dp, ctypes.c_int32, P(ctypes.c_int32)]),
        "afqmc_get_info": (ctypes.c_int, [vp, P(Info)]),
        "afqmc_save": (ctypes.c_int, [vp, vp, P(ctypes.c_size_t)]),
        "afqmc_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
        "afqmc_destroy": (ctypes.c_int, [vp]),
        "afqmc_last_error": (ctypes.c_char_p, []),
        "afqmc_launch_count": (ctypes.c_int64, []),
        "afqmc_philox4x32_10": (ctypes.c_int, [ctypes.c_uint64, vp, ctypes.c_int64, vp, vp]),
        "afqmc_round_f32": (ctypes.c_int, [vp, vp, ctypes.c_int64, vp]),
        "afqmc_widen_f32": (ctypes.c_int, [vp, vp, ctypes.c_int64, vp]),
        "afqmc_gaussian_fields": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_int32, vp, vp]),
        "afqmc_contract": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                          ctypes.c_float, vp, ctypes.c_int64, vp, vp]),
        "afqmc_profile_start": (ctypes.c_int, [vp, ctypes.c_int32]),
        "afqmc_profile_stop": (ctypes.c_int, [vp, vp, vp, vp]),
        "afqmc_local_energies_noalloc": (ctypes.c_int, [ctypes.c_int32] * 4 + [vp] * 3 +
                                         [ctypes.c_double, vp, vp]),
        "afqmc_group_create": (ctypes.c_int, [P(vp), ctypes.c_int32, vp, P(vp)]),
        "afqmc_group_propagate": (ctypes.c_int, [vp, ctypes.c_int32]),
        "afqmc_group_destroy": (ctypes.c_int, [vp]),
        "afqmc_group_set_grouped": (ctypes.c_int, [vp, ctypes.c_int32]),
        "afqmc_group_tiles": (ctypes.c_int, [vp, P(ctypes.c_int32)]),
        "afqmc_wait_flag": (ctypes.c_int, [vp, ctypes.c_int64, vp, vp]),
        "afqmc_taylor_series": (ctypes.c_int, [ctypes.c_int32] + [ctypes.c_int64] * 4 +
                                [ctypes.c_int32, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int32,
                                 vp, vp]),
        "afqmc_mcd_workspace_size": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32,
                                                    P(ctypes.c_size_t)]),
        "afqmc_modified_cholesky": (ctypes.c_int, [ctypes.c_int64, vp, ctypes.c_double,
                                                   ctypes.c_int32, vp, vp, P(ctypes.c_int32),
                                                   dp, vp, ctypes.c_size_t, vp]),
        "afqmc_init_multidet": (ctypes.c_int, [P(Params), dp, dp, ctypes.c_int32, dp, dp, dp, vp,
                                               ctypes.c_size_t, vp, P(vp)]),
        "afqmc_walker_row_bytes": (ctypes.c_int, [vp, P(ctypes.c_size_t)]),
        "afqmc_export_weights": (ctypes.c_int, [vp, vp]),
        "afqmc_comb_plan": (ctypes.c_int, [vp, vp, ctypes.c_int64, vp, vp]),
        "afqmc_pack_walkers": (ctypes.c_int, [vp, vp, ctypes.c_int32, vp]),
        "afqmc_unpack_walkers": (ctypes.c_int, [vp, vp, ctypes.c_int32, vp]),
        "afqmc_energy_sums": (ctypes.c_int, [vp, vp]),
        "afqmc_bp_begin": (ctypes.c_int, [vp]),
        "afqmc_bp_end": (ctypes.c_int, [vp, dp, dp, dp, P(ctypes.c_int32)]),
        "afqmc_mcd_pairs_workspace_size": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                                          P(ctypes.c_size_t)]),
        "afqmc_modified_cholesky_pairs": (ctypes.c_int, [ctypes.c_int32, vp, ctypes.c_double,
                                                         ctypes.c_int32, vp, vp, P(ctypes.c_int32),
                                                         dp, vp, ctypes.c_size_t, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != AFQMC_OK:
        msg = lib().afqmc_last_error().decode(errors="replace")
        raise AfqmcError(f"{STATUS.get(rc, rc)}: {msg}")


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_params(M=0, N=0, nchol=0, nwalkers=0, **kw) -> Params:
    p = Params()
    lib().afqmc_default_params(ctypes.byref(p))
    p.M, p.N, p.nchol, p.nwalkers = M, N, nchol, nwalkers
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def afqmc_workspace_size(p: Params) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().afqmc_workspace_size(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def afqmc_philox4x32_10(key: int, ctr):
    """Philox4x32-10 words for a (n, 4) int32/uint32 CUDA tensor of counters."""
    import torch

    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    st = torch.cuda.current_stream(ctr.device)
    _check(lib().afqmc_philox4x32_10(key, ctypes.c_void_p(ctr.data_ptr()), ctr.shape[0],
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream)))
    return out


def afqmc_round_f32(x):
    """float64 CUDA tensor -> float32 by the integer-arithmetic conversion the
    mixed path's kernels use (round to nearest, ties to even)."""
    import torch

    x = x.contiguous()
    out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    st = torch.cuda.current_stream(x.device)
    _check(lib().afqmc_round_f32(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 x.numel(), ctypes.c_void_p(st.cuda_stream)))
    return out


def afqmc_widen_f32(x):
    """float32 CUDA tensor -> float64 (exact) by the mixed path's conversion."""
    import torch

    x = x.contiguous()
    out = torch.empty(x.shape, dtype=torch.float64, device=x.device)
    st = torch.cuda.current_stream(x.device)
    _check(lib().afqmc_widen_f32(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 x.numel(), ctypes.c_void_p(st.cuda_stream)))
    return out


def afqmc_gaussian_fields(seed: int, step: int, w0: int, nw: int, nchol: int, device="cuda:0"):
    """The fields afqmc_propagate draws for walkers [w0, w0+nw) at one step."""
    import torch

    out = torch.empty((nw, nchol), dtype=torch.float64, device=device)
    st = torch.cuda.current_stream(out.device)
    _check(lib().afqmc_gaussian_fields(seed, step, w0, nw, nchol, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(st.cuda_stream)))
    return out


def afqmc_modified_cholesky(V, delta: float, max_vectors: int, workspace=None):
    """Modified Cholesky vectors of the symmetric PSD CUDA float64 matrix V
    (Sec. 2.3, Eqs. chol/chol2): returns (L [nvec][dim], pivots [nvec], the
    largest residual diagonal left).  Converged iff that residual < delta."""
    import torch

    V = V.contiguous()
    dim = V.shape[0]
    nbytes = ctypes.c_size_t(0)
    _check(lib().afqmc_mcd_workspace_size(dim, max_vectors, ctypes.byref(nbytes)))
    if workspace is None or workspace.numel() < nbytes.value:
        workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=V.device)
    L = torch.empty((max_vectors, dim), dtype=torch.float64, device=V.device)
    piv = torch.empty(max_vectors, dtype=torch.int32, device=V.device)
    nvec = ctypes.c_int32(0)
    resid = ctypes.c_double(0.0)
    st = torch.cuda.current_stream(V.device)
    _check(lib().afqmc_modified_cholesky(
        dim, ctypes.c_void_p(V.data_ptr()), float(delta), max_vectors,
        ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(piv.data_ptr()), ctypes.byref(nvec),
        ctypes.byref(resid), ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
        ctypes.c_void_p(st.cuda_stream)))
    n = nvec.value
    return L[:n], piv[:n], resid.value


def afqmc_modified_cholesky_pairs(Vpair, M: int, delta: float, max_vectors: int,
                                  workspace=None):
    """The decomposition over index pairs p <= r of a real-orbital interaction
    (CUDA float64 Vpair, npair x npair): returns (L [nvec][M][M], pivots as
    p*M + r, the largest residual diagonal left)."""
    import torch

    Vpair = Vpair.contiguous()
    nbytes = ctypes.c_size_t(0)
    _check(lib().afqmc_mcd_pairs_workspace_size(M, max_vectors, ctypes.byref(nbytes)))
    if workspace is None or workspace.numel() < nbytes.value:
        workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=Vpair.device)
    L = torch.empty((max_vectors, M, M), dtype=torch.float64, device=Vpair.device)
    piv = torch.empty(max_vectors, dtype=torch.int32, device=Vpair.device)
    nvec = ctypes.c_int32(0)
    resid = ctypes.c_double(0.0)
    st = torch.cuda.current_stream(Vpair.device)
    _check(lib().afqmc_modified_cholesky_pairs(
        M, ctypes.c_void_p(Vpair.data_ptr()), float(delta), max_vectors,
        ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(piv.data_ptr()), ctypes.byref(nvec),
        ctypes.byref(resid), ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
        ctypes.c_void_p(st.cuda_stream)))
    n = nvec.value
    return L[:n], piv[:n], resid.value


def afqmc_launch_count() -> int:
    return int(lib().afqmc_launch_count())


class AfqmcRun:
    """One AFQMC state on a CUDA device: workspace, stream, walkers."""

    def __init__(self, h1, L, trial, params: Params, device="cuda:0", stream=None,
                 workspace=None):
        """trial: the RHF orbitals [M][N]; with two spin blocks (params.Ndn >= 1)
        a tuple (spin-up orbitals [M][N], spin-down orbitals [M][Ndn]); for a
        multi-determinant trial (params.ndet >= 1) a tuple (coefficients
        [ndet] complex, spin-up orbitals [ndet][M][N], spin-down orbitals
        [ndet][M][N])."""
        import torch

        self.p = params
        self.device = torch.device(device)
        nbytes = afqmc_workspace_size(params)
        if workspace is None:
            workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ws = workspace
        base = workspace.data_ptr()
        off = (-base) % 256
        if stream is None:
            # graph capture needs a created stream (the default stream cannot be captured)
            stream = (torch.cuda.Stream(device=self.device) if params.use_graph
                      else torch.cuda.current_stream(self.device))
        self.stream = stream
        h1 = np.ascontiguousarray(h1, np.float64)
        L = np.ascontiguousarray(L, np.float64)
        if h1.shape != (params.M, params.M) or L.shape != (params.nchol, params.M, params.M):
            raise AfqmcError("input shapes do not match the parameters")
        st = ctypes.c_void_p()
        ws_ptr = ctypes.c_void_p(base + off)
        ws_len = ctypes.c_size_t(workspace.numel() - off)
        sptr = ctypes.c_void_p(self.stream.cuda_stream)
        if params.ndet > 0:
            coef, up, dn = trial
            nd = params.ndet
            coef = np.asarray(coef, np.complex128).reshape(nd)
            cf = np.ascontiguousarray(np.stack([coef.real, coef.imag], -1))
            up = np.ascontiguousarray(up, np.float64)
            dn = np.ascontiguousarray(dn, np.float64)
            if up.shape != (nd, params.M, params.N) or dn.shape != up.shape:
                raise AfqmcError("trial orbitals must be [ndet][M][N]")
            with torch.cuda.device(self.device):
                rc = lib().afqmc_init_multidet(ctypes.byref(params), _dptr(h1), _dptr(L), nd,
                                               _dptr(cf), _dptr(up), _dptr(dn), ws_ptr, ws_len,
                                               sptr, ctypes.byref(st))
        else:
            if params.Ndn > 0:
                up, dn = trial
                dn = np.ascontiguousarray(dn, np.float64)
                if dn.shape != (params.M, params.Ndn):
                    raise AfqmcError("spin-down trial must be [M][Ndn]")
            else:
                up, dn = trial, None
            up = np.ascontiguousarray(up, np.float64)
            if up.shape != (params.M, params.N):
                raise AfqmcError("input shapes do not match the parameters")
            with torch.cuda.device(self.device):
                rc = lib().afqmc_init(ctypes.byref(params), _dptr(h1), _dptr(L), _dptr(up),
                                      _dptr(dn) if dn is not None else None, ws_ptr, ws_len,
                                      sptr, ctypes.byref(st))
        _check(rc)
        self.s = st

    # -- the walk ---------------------------------------------------------------
    def propagate(self, nsteps: int):
        _check(lib().afqmc_propagate(self.s, int(nsteps)))

    def energy(self):
        E, w = ctypes.c_double(), ctypes.c_double()
        _check(lib().afqmc_energy(self.s, ctypes.byref(E), ctypes.byref(w)))
        return E.value, w.value

    def local_energies(self):
        out = np.empty((self.p.nwalkers, 2))
        _check(lib().afqmc_local_energies(self.s, _dptr(out)))
        return out[:, 0] + 1j * out[:, 1]

    def bp_begin(self):
        """Open a back-propagation window at the current step."""
        _check(lib().afqmc_bp_begin(self.s))

    def bp_end(self):
        """Close the window: (rho BP-PRes, rho BP-PhL) as complex M x M arrays,
        (sum W F, sum W) and the window's length in steps."""
        M = self.p.M
        rho = np.empty((2, M, M))
        phl = np.empty((2, M, M))
        ws = np.empty(4)
        n = ctypes.c_int32(0)
        _check(lib().afqmc_bp_end(self.s, _dptr(rho), _dptr(phl), _dptr(ws), ctypes.byref(n)))
        return (rho[0] + 1j * rho[1], phl[0] + 1j * phl[1], complex(ws[0], ws[1]),
                complex(ws[2], ws[3]), n.value)

    @property
    def ncols(self) -> int:
        """Orbital columns per walker: N, or N_up + N_dn with two spin blocks."""
        return self.p.N + (self.p.Ndn if self.p.Ndn > 0 else 0)

    def get_walkers(self):
        W, M, N = self.p.nwalkers, self.p.M, self.ncols
        phi = np.empty((W, M, N, 2))
        wt = np.empty((W, 2))
        lo = np.empty((W, 2))
        _check(lib().afqmc_get_walkers(self.s, _dptr(phi), _dptr(wt), _dptr(lo)))
        return phi[..., 0] + 1j * phi[..., 1], wt[:, 0] + 1j * wt[:, 1], lo[:, 0] + 1j * lo[:, 1]

    def weights(self):
        """Walker weights W e^{i theta} (complex), without copying the orbitals."""
        wt = np.empty((self.p.nwalkers, 2))
        _check(lib().afqmc_get_walkers(self.s, None, _dptr(wt), None))
        return wt[:, 0] + 1j * wt[:, 1]

    def set_walkers(self, phi, weight):
        W, M, N = self.p.nwalkers, self.p.M, self.ncols
        phi = np.asarray(phi, np.complex128).reshape(W, M, N)
        ph = np.ascontiguousarray(np.stack([phi.real, phi.imag], -1))
        w = np.asarray(weight, np.complex128).reshape(W)
        wt = np.ascontiguousarray(np.stack([w.real, w.imag], -1))
        _check(lib().afqmc_set_walkers(self.s, _dptr(ph), _dptr(wt)))

    def energy_log(self):
        cap = self.p.max_records
        rec = np.empty((cap, 4))
        n = ctypes.c_int32()
        _check(lib().afqmc_get_energy_log(self.s, _dptr(rec), cap, ctypes.byref(n)))
        return rec[: n.value].copy()

    def info(self) -> Info:
        i = Info()
        _check(lib().afqmc_get_info(self.s, ctypes.byref(i)))
        return i

    def save(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(lib().afqmc_save(self.s, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().afqmc_save(self.s, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().afqmc_load(self.s, buf, len(blob)))

    def close(self):
        if getattr(self, "s", None):
            lib().afqmc_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AfqmcGroup:
    """Independent runs advanced together by one CUDA graph launch per block
    of steps (afqmc_group_*).  Every run needs use_graph=1, its own stream and
    the same graph block length."""

    def __init__(self, runs, stream=None):
        import torch

        self.runs = list(runs)
        dev = self.runs[0].device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        arr = (ctypes.c_void_p * len(self.runs))(*[r.s.value for r in self.runs])
        g = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _check(lib().afqmc_group_create(arr, len(self.runs),
                                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(g)))
        self.g = g

    def propagate(self, nsteps: int):
        _check(lib().afqmc_group_propagate(self.g, int(nsteps)))

    def set_grouped(self, on):
        """True: grouped tensor-core contractions (one persistent launch per
        phase for all runs) where the runs allow; False: each run's own
        kernels; "auto" (the default): the faster of the two, by timing."""
        _check(lib().afqmc_group_set_grouped(self.g, 2 if on == "auto" else (1 if on else 0)))

    def tiles(self):
        """(grouped?, tile widths of the force-bias, V, first and last half-step
        launches) as chosen on the first propagate."""
        bn = (ctypes.c_int32 * 4)()
        r = lib().afqmc_group_tiles(self.g, bn)
        if r < 0:
            _check(r)
        return bool(r), list(bn)

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "g", None):
            lib().afqmc_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wmax_default(nwalkers: int) -> float:
    return max(100.0, nwalkers / 10.0)


__all__ = ["AfqmcRun", "Params", "Info", "AfqmcError", "default_params", "lib",
           "afqmc_workspace_size", "afqmc_launch_count", "EXPORTED", "math"]
