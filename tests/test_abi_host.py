"""The C-ABI library loads, exports every declared symbol, and its host-side O_h tables
equal the oracle's bit for bit (CPU only; no device work)."""

import ctypes

import numpy as np

from oracle import lattice as L


def test_library_exports_every_header_symbol(lib):
    from paper_2412_08229_gb300 import _abi
    names = _abi.header_functions()
    assert "lbm_create" in names and "nco_set_weights" in names and "lbm_energy_spectrum" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in _abi._SIGNATURES, f"{name} has no ctypes declaration"


def test_version_string(lib):
    import paper_2412_08229_gb300 as P
    assert "sm_103a" in P.lbm_version()


def test_null_context_is_rejected_without_device_work(lib):
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_destroy(None) == 0
    assert b"invalid" in lib.lbm_last_error(None)


def test_group_tables_bit_exact_against_oracle(lib):
    import paper_2412_08229_gb300 as P
    R, vperm, mperm, msign = P.lbm_group_tables()
    o_perm, o_sign = L.moment_action_tables()
    oracle_R = {L.G_MATRICES[g].tobytes(): g for g in range(48)}
    seen = set()
    for g in range(48):
        key = R[g].astype(np.int64).tobytes()
        assert key in oracle_R, f"library element {g} is not a cube symmetry"
        go = oracle_R[key]
        seen.add(go)
        assert (vperm[g] == L.G_VPERM[go]).all()
        assert (mperm[g] == o_perm[go]).all()
        assert (msign[g] == o_sign[go]).all()
    assert len(seen) == 48


def test_invalid_configurations_are_refused_before_device_work(lib):
    """lbm_create checks every argument before it touches the GPU: empty grids, grids whose
    27 x cells state does not fit 32-bit indices (the largest accepted cube is 430^3),
    non-positive viscosity, unknown enums, a non-cube reduced Taylor-Green domain and
    forcing off the periodic box all return LBM_ERR_ARG with no context."""
    import paper_2412_08229_gb300 as P
    from paper_2412_08229_gb300 import _abi

    def refused(**kw):
        base = dict(nx=4, ny=4, nz=4, nu=0.01)
        base.update(kw)
        cfg = P._config(base.pop("nx"), base.pop("ny"), base.pop("nz"), base.pop("nu"), **base)
        out = ctypes.c_void_p(123)
        st = lib.lbm_create(ctypes.byref(cfg), None, ctypes.byref(out))
        return st == _abi.LBM_ERR_ARG and out.value is None

    assert refused(nx=0)
    assert refused(nz=-3)
    assert refused(nx=431, ny=431, nz=431)        # 27 * 431^3 >= 2^31
    assert refused(nx=2 ** 16, ny=2 ** 16, nz=2)  # the product overflows 32 bits
    assert 27 * 430 ** 3 < 2 ** 31                # so 430^3 passes this check
    assert refused(nu=0.0)
    assert refused(nu=float("nan"))
    assert refused(boundary="tgv_reduced", nx=4, ny=4, nz=5)
    assert refused(forcing=dict(power=1e-6), boundary="mirror")
    cfg = P._config(4, 4, 4, 0.01)
    cfg.op = 9
    out = ctypes.c_void_p(123)
    assert lib.lbm_create(ctypes.byref(cfg), None, ctypes.byref(out)) == _abi.LBM_ERR_ARG and out.value is None
    cfg = P._config(4, 4, 4, 0.01)
    cfg.net_precision = 7
    assert lib.lbm_create(ctypes.byref(cfg), None, ctypes.byref(out)) == _abi.LBM_ERR_ARG
