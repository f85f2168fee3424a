"""The C-ABI library builds for sm_103a, loads, and exports every symbol its
header declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "afqmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"AFQMC_API\s+[\w\s\*]+?\b(afqmc_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_02242_gb300 as pkg

    return pkg


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("afqmc_init", "afqmc_propagate", "afqmc_energy", "afqmc_workspace_size"):
        assert required in names
    assert len(names) >= 17


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(built.EXPORTED) == declared_functions()


def test_params_struct_matches_header_defaults(built):
    p = built.default_params(12, 3, 48, 32)
    assert (p.dt, p.taylor_order, p.qr_period, p.pc_period) == (0.005, 6, 5, 0)
    assert p.ecap_C == 2.0 and p.fb_cap == 1.0 and p.max_records == 4096
    assert p.e_shift != p.e_shift and p.wmax != p.wmax  # NaN defaults
    assert ctypes.sizeof(built.Params) == 120
    assert p.bp_steps == 0 and p.ndet == 0 and p.Ndn == 0 and p.walker0 == 0


def test_workspace_size_and_validation_without_gpu(built):
    p = built.default_params(300, 25, 1800, 512)
    n = built.afqmc_workspace_size(p)
    # packed Cholesky vectors alone are 1800 * 45150 doubles
    assert n > 1800 * 45150 * 8
    assert n % 256 == 0
    with pytest.raises(built.AfqmcError, match="EINVAL"):
        built.afqmc_workspace_size(built.default_params(10, 11, 5, 4))
    with pytest.raises(built.AfqmcError, match="EINVAL"):
        built.afqmc_workspace_size(built.default_params(10, 2, 5, 4, dt=-1.0))


def test_spin_block_parameters_without_gpu(built):
    """Two spin blocks (Ndn >= 1): the workspace holds N_up + N_dn orbital
    columns per walker; they run on the float64 path only, with at most 64
    columns; walker0 is a non-negative field counter offset."""
    n1 = built.afqmc_workspace_size(built.default_params(12, 3, 48, 32))
    n2 = built.afqmc_workspace_size(built.default_params(12, 3, 48, 32, Ndn=2))
    n3 = built.afqmc_workspace_size(built.default_params(12, 5, 48, 32))
    assert n1 < n2 <= n3
    for kw, err in ((dict(Ndn=2, precision=2), "EUNSUPPORTED"), (dict(Ndn=2, bp_steps=4), "EUNSUPPORTED"),
                    (dict(Ndn=13), "EINVAL"), (dict(Ndn=-1), "EINVAL"), (dict(walker0=-1), "EINVAL")):
        with pytest.raises(built.AfqmcError, match=err):
            built.afqmc_workspace_size(built.default_params(12, 3, 48, 32, **kw))
    with pytest.raises(built.AfqmcError, match="EUNSUPPORTED"):
        built.afqmc_workspace_size(built.default_params(100, 40, 48, 32, Ndn=30))
    # the spin-down trial is required exactly when Ndn >= 1 (refused before any device call)
    st = ctypes.c_void_p()
    lib = built.lib()
    h = (ctypes.c_double * 144)()
    p = built.default_params(12, 3, 48, 32, Ndn=2)
    assert lib.afqmc_init(ctypes.byref(p), h, h, h, None, ctypes.c_void_p(256), 1 << 30, None,
                          ctypes.byref(st)) == -1
    assert b"trial_dn" in lib.afqmc_last_error()


def test_library_has_no_oracle_dependency():
    """The product path never imports or links the oracle."""
    pkgdir = os.path.join(ROOT, "paper_1711_02242_gb300")
    for dirpath, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_mcd_workspace_size_and_validation_without_gpu(built):
    """The decomposition's workspace holds the residual diagonal, the pivot's
    components and the reduction tree (one result per 32 indices; the vectors
    themselves live in the caller's output); bad sizes are refused before any
    device call."""
    lib = built.lib()
    n = ctypes.c_size_t(0)
    assert lib.afqmc_mcd_workspace_size(90000, 1800, ctypes.byref(n)) == 0
    want = 90000 * 8 + 1800 * 8 + 2813 * 24
    assert want <= n.value < want + 4096 and n.value % 256 == 0
    for dim, mv in ((0, 10), (10, 0), (10, 16385), (1 << 31, 10)):
        assert lib.afqmc_mcd_workspace_size(dim, mv, ctypes.byref(n)) == -1
    nv = ctypes.c_int32(0)
    assert lib.afqmc_modified_cholesky(10, None, 1e-6, 10, None, None, ctypes.byref(nv), None,
                                       None, 0, None) == -1


def test_mcd_pairs_workspace_size_without_gpu(built):
    lib = built.lib()
    n = ctypes.c_size_t(0)
    assert lib.afqmc_mcd_pairs_workspace_size(300, 1800, ctypes.byref(n)) == 0
    npair = 300 * 301 // 2
    assert n.value >= npair * 8 * (1800 + 1) and n.value % 256 == 0
    assert n.value < npair * 8 * (1800 + 1) + 17 * npair + (4 << 20)
    for M, mv in ((0, 10), (2049, 10), (10, 0)):
        assert lib.afqmc_mcd_pairs_workspace_size(M, mv, ctypes.byref(n)) == -1
