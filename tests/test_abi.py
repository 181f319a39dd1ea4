"""The C ABI library builds, loads and exports every entry point declared in
include/*.h (no compute calls, no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

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


def _c_fields(struct):
    """Field names of a typedef'd struct in include/lra_cross.h, in order."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "lra_cross.h")).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + struct + r"\s*;", text).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "type a, b" or "type* a" -> the declarators after the type
        parts = decl.replace("*", " ").split()
        rest = " ".join(parts[1:]) if parts[0] != "const" else " ".join(parts[2:])
        names += [n.strip() for n in rest.split(",")]
    return names


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the ABI structs have the size and field offsets
    the C compiler gives the header's declarations."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        import pytest
        pytest.skip("no C compiler")
    import paper_1611_01391_gb300 as L
    structs = ["lra_ctx_params", "lra_source", "lra_params", "lra_info", "lra_cur_out", "lra_block",
               "lra_batch_params", "lra_batch_out", "lra_cynical_params", "lra_cynical_out", "lra_refine_params",
               "lra_refine_out", "lra_rf_params", "lra_rf_out", "lra_lsr_params", "lra_lsr_out"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lra_cross.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f in _c_fields(s):
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.splitlines():
        s, f, v = line.split()
        cls = getattr(L, s)
        if f == "size":
            assert ctypes.sizeof(cls) == int(v), (s, ctypes.sizeof(cls), v)
        else:
            assert getattr(cls, f).offset == int(v), (s, f, getattr(cls, f).offset, v)


def _valid_pair():
    import numpy as np
    import paper_1611_01391_gb300 as L
    src = L.lra_source(L.LRA_GEN_GAUSS, 3, 5000, 4000, None, 0, 16, 16, 0.5)
    params, keep = L.make_params(8, 12, 2, np.arange(12), resid_rows=np.arange(100),
                                 resid_cols=np.arange(100))
    return src, params, keep


# every rejection rule of the host validation, one at a time, each from a
# valid pair; lra_cross_footprint runs the same validation as submit
_BREAKERS = {
    "unknown kind": lambda L, s, p: setattr(s, "kind", 7),
    "m < 1": lambda L, s, p: setattr(s, "m", 0),
    "n too large": lambda L, s, p: setattr(s, "n", (1 << 30) + 1),
    "dense without a": lambda L, s, p: (setattr(s, "kind", L.LRA_DENSE_F32), setattr(s, "a", None)),
    "dense lda < n": lambda L, s, p: (setattr(s, "kind", L.LRA_DENSE_F32), setattr(s, "a", 256),
                                      setattr(s, "lda", 3999)),
    "generator without y": lambda L, s, p: setattr(s, "y", None),
    "dim 4": lambda L, s, p: setattr(s, "dim", 4),
    "gauss h = 0": lambda L, s, p: setattr(s, "h", 0.0),
    "l = 97": lambda L, s, p: (setattr(p, "l", 97)),
    "k = 0": lambda L, s, p: setattr(p, "k", 0),
    "l > n": lambda L, s, p: setattr(s, "n", 11),
    "sweeps = 0": lambda L, s, p: setattr(p, "sweeps", 0),
    "delta = 0": lambda L, s, p: setattr(p, "delta", 0.0),
    "rank_tol < 0": lambda L, s, p: setattr(p, "rank_tol", -1.0),
    "q without s": lambda L, s, p: setattr(p, "resid_s", 0),
    "sample > m": lambda L, s, p: setattr(p, "resid_q", 5001),
    "tol without sample": lambda L, s, p: (setattr(p, "tol", 1e-3), setattr(p, "resid_q", 0),
                                           setattr(p, "resid_s", 0)),
    "trace_cap < 0": lambda L, s, p: setattr(p, "trace_cap", -1),
    "full residual on a generator": lambda L, s, p: setattr(p, "flags", 2),
    "full residual, unaligned base": lambda L, s, p: (setattr(s, "kind", L.LRA_DENSE_F32),
                                                      setattr(s, "a", 4100), setattr(s, "lda", 4000),
                                                      setattr(p, "flags", 2)),
}


@pytest.mark.parametrize("rule", sorted(_BREAKERS))
def test_host_validation_rejects(rule):
    import paper_1611_01391_gb300 as L
    src, params, keep = _valid_pair()
    assert L.lra_cross_footprint(src, params) > 0
    _BREAKERS[rule](L, src, params)
    with pytest.raises(L.LraError) as e:
        L.lra_cross_footprint(src, params)
    assert e.value.code == L.LRA_EINVAL


def test_footprint_grows_with_the_strips():
    """The job's allocation holds both strips (4 (m + n) l bytes) plus
    per-job pieces independent of m and n."""
    import paper_1611_01391_gb300 as L
    src, params, keep = _valid_pair()
    b0 = L.lra_cross_footprint(src, params)
    src.m, src.n = 2 * 5000, 2 * 4000
    b1 = L.lra_cross_footprint(src, params)
    grow = 4 * (5000 + 4000) * 12
    assert abs((b1 - b0) - grow) <= 2 * 256   # two 256-byte-aligned pieces


def test_library_seed_draw_equals_the_oracle_draw():
    """lra_draw_columns (host code of the library) and the oracle's own
    SplitMix64 + Floyd sampling, written separately, draw the same J0."""
    import oracle as O
    import paper_1611_01391_gb300 as L
    for seed, n, l in ((0, 10, 10), (1, 100, 8), (161101391, 65536, 24), (2**63 + 5, 32768, 96),
                       (42, 1 << 30, 3)):
        assert list(L.lra_draw_columns(seed, n, l)) == O.draw_columns(seed, n, l)
    with pytest.raises(L.LraError):
        L.lra_draw_columns(1, 5, 6)


def test_noalloc_rejects_aliasing_strides_on_host():
    """Stride rules of lra_maxvol_noalloc are checked before any CUDA call:
    both >= 1, and the N x l elements must not share addresses."""
    import paper_1611_01391_gb300 as L
    fake = 256    # never dereferenced: every case below fails validation first
    N, l = 100, 8
    for rs, cs in ((0, 1), (8, 0), (-8, 1), (4, 1), (1, 50), (3, 2)):
        rc = L.lra_maxvol_noalloc(fake, N, l, rs, cs, fake, None, 1e-2, 0, fake, None)
        assert rc == L.LRA_EINVAL, (rs, cs, rc)


def test_gather_entries_validates_on_host():
    import paper_1611_01391_gb300 as L
    bad = L.lra_source(L.LRA_GEN_GAUSS, 3, 100, 100, None, 0, 1, 1, 0.0)   # h = 0
    rc = L._gather_entries(ctypes.byref(bad), 256, 4, 256, 4, 256, None)
    assert rc == L.LRA_EINVAL
    ok = L.lra_source(L.LRA_GEN_CAUCHY, 1, 100, 100, None, 0, 1, 1, 0.0)
    assert L._gather_entries(ctypes.byref(ok), 256, 0, 256, 4, 256, None) == L.LRA_OK   # empty: no launch
    assert L._gather_entries(ctypes.byref(ok), 256, -1, 256, 4, 256, None) == L.LRA_EINVAL


def _bucket_key(gpu, kind, l_max, k_max, blocks):
    """The batch tuner's bucket, written from its documented rule."""
    import numpy as np

    def p2(v):
        p = 1
        while p < v:
            p *= 2
        return p
    side = np.sort(np.maximum(blocks[:, 1], blocks[:, 3]))
    return (f"{gpu}|kind={kind}|lmax={l_max}|kmax={k_max}|blocks={p2(len(blocks))}"
            f"|median={p2(int(side[len(side) // 2]))}|max={p2(int(side[-1]))}")


def test_batch_tuning_cache_lookup_on_host(tmp_path):
    """The tuner's cache (JSON, one entry per GPU and workload bucket) is
    found for the same GPU and bucket, including a workload of other sizes
    in the same bucket, and not for another GPU or another bucket."""
    import numpy as np
    import paper_1611_01391_gb300 as L
    from paper_1611_01391_gb300.api import make_batch_params
    blocks = np.array([[0, 300, 0, 260], [0, 2000, 0, 1500], [0, 250, 0, 280]], np.int64)
    jc = np.tile(np.arange(96, dtype=np.int32), (3, 1))
    p, keep = make_batch_params(12, 96, 64, 2, 1e-6, jc)
    src = L.lra_source(L.LRA_GEN_INVDIST, 3, 1 << 20, 1 << 20, None, 0, 1, 1, 0.0)
    key = _bucket_key("NVIDIA GB300", L.LRA_GEN_INVDIST, 96, 64, blocks)
    path = tmp_path / "tuning.json"
    path.write_text('{\n  "lra_batch_tuning": 1,\n  "entries": {\n'
                    f'    "other|kind=4": {{"cluster_mask": 9, "cutover_side": 512, "order": 0, "ms_default": 1, "ms_tuned": 1}},\n'
                    f'    "{key}": {{"cluster_mask": 11, "cutover_side": 1024, "order": 1, "ms_default": 61.0, "ms_tuned": 55.0}}\n'
                    '  }\n}\n')
    t = L.lra_batch_tuning_lookup(path, "NVIDIA GB300", src, blocks, p)
    assert t is not None and (t.cluster_mask, t.cutover_side, t.order) == (11, 1024, 1)
    assert (t.l_max, t.k_max, t.sweeps) == (96, 64, 2)          # the rest copied from params
    same_bucket = blocks.copy()
    same_bucket[1, 1] = 1900                                     # max side still in (1024, 2048]
    assert L.lra_batch_tuning_lookup(path, "NVIDIA GB300", src, same_bucket, p) is not None
    assert L.lra_batch_tuning_lookup(path, "NVIDIA B200", src, blocks, p) is None
    other = blocks.copy()
    other[1, 1] = other[1, 3] = 900                              # max side now in (512, 1024]
    assert L.lra_batch_tuning_lookup(path, "NVIDIA GB300", src, other, p) is None
    assert L.lra_batch_tuning_lookup(tmp_path / "absent.json", "NVIDIA GB300", src, blocks, p) is None
