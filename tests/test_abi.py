"""CPU-side checks of the C ABI library: it builds, loads, and exports every
function include/ltpc.h declares.  No compute call is made here."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2508_06771_gb300 import build as B
    from paper_2508_06771_gb300 import ltpc
    B.build()
    return ltpc.load_library()


def test_exports_every_declared_symbol(lib):
    from paper_2508_06771_gb300 import ltpc
    names = ltpc.header_symbols()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_required_bytes_is_host_only(lib):
    import numpy as np
    from paper_2508_06771_gb300 import ltpc
    inv = np.ones(10)
    cfg = ltpc.Config()
    cfg.precision, cfg.n_cells, cfg.capacity = ltpc.F32, 10, 1000
    cfg.mass, cfg.charge, cfg.eps0, cfg.weight = 9.1e-31, 1.6e-19, 8.85e-12, 1.0
    cfg.inv_volume = inv.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.ltpc_required_bytes(ctypes.byref(cfg), ctypes.byref(sb), ctypes.byref(wb)) == 0
    assert sb.value >= 1000 * 16 and wb.value > 1000 * 4
    cfg.capacity = 0
    assert lib.ltpc_required_bytes(ctypes.byref(cfg), ctypes.byref(sb), ctypes.byref(wb)) == ltpc.EINVAL
    cfg.capacity, cfg.precision = 1000, 7
    assert lib.ltpc_required_bytes(ctypes.byref(cfg), ctypes.byref(sb), ctypes.byref(wb)) == ltpc.EINVAL


def test_bijection_mode_adds_one_exchange_record_per_particle(lib):
    """The bijection mode's work buffer holds the clusters' exchange records: one per particle
    of capacity, 16 bytes in binary32 and 32 in binary64 (plus alignment)."""
    import numpy as np
    from paper_2508_06771_gb300 import ltpc
    inv = np.ones(10)
    for prec, rec in ((ltpc.F32, 16), (ltpc.F64, 32)):
        sizes = {}
        for mode in (ltpc.PAIR_KEY, ltpc.PAIR_BIJECTION):
            cfg = ltpc.Config()
            cfg.precision, cfg.n_cells, cfg.capacity, cfg.pairing_mode = prec, 10, 1000, mode
            cfg.mass, cfg.charge, cfg.eps0, cfg.weight = 9.1e-31, 1.6e-19, 8.85e-12, 1.0
            cfg.inv_volume = inv.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
            assert lib.ltpc_required_bytes(ctypes.byref(cfg), ctypes.byref(sb), ctypes.byref(wb)) == 0
            sizes[mode] = (sb.value, wb.value)
        assert sizes[ltpc.PAIR_KEY][0] == sizes[ltpc.PAIR_BIJECTION][0]
        extra = sizes[ltpc.PAIR_BIJECTION][1] - sizes[ltpc.PAIR_KEY][1]
        assert 1000 * rec <= extra < 1000 * rec + 256, (prec, extra)


def test_strerror(lib):
    from paper_2508_06771_gb300 import ltpc
    for code in (ltpc.OK, ltpc.EINVAL, ltpc.ECAPACITY, ltpc.ECUDA, ltpc.ETIMEOUT, ltpc.ENONFINITE,
                 ltpc.EUNSUPPORTED, ltpc.EINTERNAL):
        assert ltpc.strerror(code)
    assert ltpc.strerror(-99) == "unknown status"
