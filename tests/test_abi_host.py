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
