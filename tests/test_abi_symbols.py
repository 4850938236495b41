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
    assert gputb.lib().tb_abi_version() == gputb.ABI_VERSION == 6


def test_workspace_query_needs_no_gpu_for_invalid_sizes(libpath):
    from paper_2509_06525_gb300 import gputb
    assert gputb.lib().kpm_moments_workspace_size(0, 16, 1, 0) == 0
    assert gputb.lib().kpm_moments_workspace_size(100, 1, 1, 0) == 0
