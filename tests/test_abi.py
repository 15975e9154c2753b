"""The C ABI library loads and exports every symbol include/bsmps.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bsmps.h")).read()
    return sorted(set(re.findall(r"BSMPS_API\s+[\w\s\*]+?\b(bsmps_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["bsmps_mps_create", "bsmps_mpo_from_integrals", "bsmps_apply_H", "bsmps_truncate",
                     "bsmps_precondition", "bsmps_eigensolve_step", "bsmps_dot"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2604_16118_gb300 import build as B
    lib_path = B.build()
    import ctypes
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    from paper_2604_16118_gb300 import native
    assert set(native.DECLARED) == set(declared_symbols())
    native.load(lib_path)


def test_status_strings_without_device():
    from paper_2604_16118_gb300 import native
    lib = native.lib()
    assert lib.bsmps_status_string(0) == b"ok"
    assert b"CUDA" in lib.bsmps_status_string(8)


def test_random_size_matches_oracle_without_device():
    # host-only entry point: the block index rule is bit-exact with the oracle's
    from paper_2604_16118_gb300 import native
    from synth import hubbard_chain, spinless_random_chain
    from tests._common import n_random
    for wl, r in [(spinless_random_chain(K=12, N=6), 32), (hubbard_chain(L=8), 40),
                  (hubbard_chain(L=32), 256)]:
        assert native.mps_random_size(wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r) == n_random(wl, r)
    with pytest.raises(native.BsmpsError):
        native.mps_random_size(4, 0, 5, 0, 8)
