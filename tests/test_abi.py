"""The C ABI library builds, loads and exports every entry point declared in
include/*.h (no compute calls, no GPU needed)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(lra_[a-z_0-9]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lra_cross_create", "lra_cross_destroy", "lra_cross_submit",
                     "lra_cross_poll", "lra_cross_fetch_cur", "lra_cross_cancel"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_01391_gb300 as L
    lib = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(L.EXPORTED) <= _declared()


def test_status_strings_without_gpu():
    import paper_1611_01391_gb300 as L
    assert L.lra_status_str(0) == "ok"
    assert "singular" in L.lra_status_str(L.LRA_ESINGULAR)


def test_create_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    import paper_1611_01391_gb300 as L
    try:
        L.lra_cross_create(0)
    except L.LraError as e:
        assert e.code in (L.LRA_ECUDA, L.LRA_EINVAL)
    else:
        raise AssertionError("context created without a GPU")


def test_footprint_and_validation_on_host():
    import numpy as np
    import paper_1611_01391_gb300 as L
    src = L.lra_source(L.LRA_GEN_CAUCHY, 1, 65536, 65536, None, 0, 1, 1, 0.0)
    params, keep = L.make_params(16, 24, 4, np.arange(24), resid_rows=np.arange(1000),
                                 resid_cols=np.arange(1000))
    b = L.lra_cross_footprint(src, params)
    assert 2 * 65536 * 24 * 4 <= b < 2 * 65536 * 24 * 4 + (4 << 20)
    params.k = 30
    try:
        L.lra_cross_footprint(src, params)
    except L.LraError as e:
        assert e.code == L.LRA_EINVAL
    else:
        raise AssertionError("k > l accepted")
