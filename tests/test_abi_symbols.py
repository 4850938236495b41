"""The C ABI library loads without a GPU and exports every symbol that
include/gputb.h declares; the binding's signature table covers them all."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gputb.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"TB_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2509_06525_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    syms = declared_symbols()
    for name in ("kpm_moments", "kpm_dos", "tb_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    handle = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(handle, s)]
    assert not missing, missing


def test_binding_signatures_cover_header(libpath):
    from paper_2509_06525_gb300 import gputb
    assert sorted(gputb.SIGNATURES) == declared_symbols()
    assert gputb.lib().tb_abi_version() == gputb.ABI_VERSION == 9


def test_workspace_query_needs_no_gpu_for_invalid_sizes(libpath):
    from paper_2509_06525_gb300 import gputb
    assert gputb.lib().kpm_moments_workspace_size(0, 16, 1, 0) == 0
    assert gputb.lib().kpm_moments_workspace_size(100, 1, 1, 0) == 0


def test_step_shape_table_host_logic(libpath):
    """The shape list of every (R, precision) and the lookup order of the
    shape table (forced entry, then the size class floor(log2 n), then 0)
    are host logic: no GPU needed."""
    from paper_2509_06525_gb300 import gputb as g
    for prec in (g.F32, g.F64):
        for R in (1, 2, 4, 8, 16, 32):
            count = g.kpm_shape_count(R, prec)
            assert count >= 1
            for k in range(count):
                info = g.kpm_shape_info(R, prec, k)
                cpt = info["complex_per_thread"]
                assert R % cpt == 0
                assert info["rows_per_tile"] == 256 // (R // cpt) * info["rows_per_thread"]
                assert info["min_blocks"] >= 1
                assert (info["stages"] >= 2) == bool(info["pipelined"])
                assert info["rows_per_tile"] == 256 // (R // cpt) * info["rows_per_thread"] or \
                    info["pipelined"] != 2
            with pytest.raises(g.GputbError):
                g.kpm_shape_info(R, prec, count)
        assert g.kpm_shape_count(3, prec) == 0
    g.kpm_clear_shapes()
    try:
        assert g.kpm_get_shape(1000, 8, g.F32, True) == 0
        g.kpm_set_shape(1024, 8, g.F32, 1, 2)            # size class 10: n in [1024, 2047]
        assert g.kpm_get_shape(1024, 8, g.F32, True) == 2
        assert g.kpm_get_shape(2047, 8, g.F32, True) == 2
        assert g.kpm_get_shape(1023, 8, g.F32, True) == 0
        assert g.kpm_get_shape(2048, 8, g.F32, True) == 0
        assert g.kpm_get_shape(1500, 8, g.F32, False) == 0  # other mode untouched
        g.kpm_force_shape(8, g.F32, 1)                      # forced: every size, both modes
        assert g.kpm_get_shape(1500, 8, g.F32, True) == 1
        assert g.kpm_get_shape(7, 8, g.F32, False) == 1
        assert g.kpm_get_shape(7, 8, g.F64, False) == 0     # other precision untouched
        g.kpm_force_shape(8, g.F32, -1)
        assert g.kpm_get_shape(1500, 8, g.F32, True) == 2
        with pytest.raises(g.GputbError):
            g.kpm_set_shape(1024, 8, g.F32, 1, g.kpm_shape_count(8, g.F32))
    finally:
        g.kpm_clear_shapes()
    assert g.kpm_get_shape(1500, 8, g.F32, True) == 0
