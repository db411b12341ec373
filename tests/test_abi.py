"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/mprk.h declares, and rejects
invalid configurations before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from paper_2202_11890_gb300 import build as B


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mprk_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mprk_create", "mprk_step", "mprk_destroy", "mprk_get_state",
                     "mprk_set_state", "mprk_diagnostics", "mprk_last_error", "mprk_rhs"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_configs_are_rejected_without_a_device(lib):
    from paper_2202_11890_gb300 import mprk as M
    q = np.ones((4, 12, 8))
    cases = [dict(nz_B=3), dict(nz_B=2), dict(m=0), dict(nx=3), dict(precision=7),
             dict(scheme=9), dict(wall=5), dict(dt=-1.0), dict(mu1=0.0), dict(x_walls=2), dict(base=3),
             dict(base=2, precision=1), dict(base=1, ny=4), dict(m=65), dict(nz_S=1), dict(nz_F=1),
             dict(ny=2), dict(ny=4, precision=1), dict(ny=4, x_walls=1), dict(ny=4, dy=0.0), dict(cfl=11.0),
             dict(gamma=1.0), dict(G=-1.0), dict(diag_every=-1),
             # the largest grid the ABI takes has 2^31 cells
             dict(nx=65536, nz_S=16384, nz_F=16384)]
    for over in cases:
        base = dict(nx=8, nz_S=4, nz_B=4, nz_F=4, m=2)
        geo = {k: over.pop(k) for k in list(over) if k in base}
        base.update(geo)
        cfg = M.mprk_config_default(**base)
        for k, v in over.items():
            setattr(cfg, k, v)
        h = C.c_void_p()
        rc = M.lib().mprk_create(C.byref(cfg), q.ctypes.data_as(C.c_void_p), M.MPRK_HOST, None,
                                 C.byref(h))
        assert rc == M.MPRK_EINVAL, (base, over, rc)
        assert M.mprk_last_error()


def test_config_default_matches_the_paper_constants(lib):
    from paper_2202_11890_gb300 import mprk as M
    cfg = M.mprk_config_default(64, 30, 4, 30, 4)
    assert cfg.gamma == 1.4 and cfg.Pr == 0.72
    assert cfg.mu1 == 1.0 / 20000 and cfg.mu2 == 1.0 / 5000
    assert cfg.G == 0.008140864714 and cfg.dx == 10.0 / 64


def test_python_config_layout_matches_the_header(tmp_path):
    """Every field of the ctypes mirror sits at the offset the C compiler
    gives the header's struct, and the sizes agree."""
    import subprocess
    from paper_2202_11890_gb300 import mprk as M
    names = [f[0] for f in M.mprk_config._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%s %zu\\n", "{n}", offsetof(mprk_config, {n}));\n' for n in names)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "mprk.h"\nint main(void) {\n' + body +
                   '  printf("sizeof %zu\\n", sizeof(mprk_config));\n  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for n in names:
        assert int(got[n]) == getattr(M.mprk_config, n).offset, n
    assert int(got["sizeof"]) == C.sizeof(M.mprk_config)


def test_tuning_table_round_trip_without_a_device(lib, tmp_path):
    """The launch-tuning table loads from JSON, answers lookups by size
    bucket (floor log2 of the mean cells), saves the same entries back, and
    rejects out-of-range values; none of it needs a GPU."""
    from paper_2202_11890_gb300 import mprk as M
    M.mprk_tune_clear()
    # FP32 flux defaults to the per-stage form (tiles per item 0)
    assert M.mprk_tune_lookup(1, 5000.0) == {"tiles_per_item": 0, "ctas_per_sm": 0, "tile_rows": 16,
                                             "tuned": False}
    assert M.mprk_tune_lookup(0, 5000.0)["tiles_per_item"] == 2
    assert M.mprk_tune_lookup(0, 5000.0)["tile_rows"] == 8
    assert M.mprk_tile_lookup(5000.0) is None
    src = tmp_path / "t.json"
    src.write_text('{"gpu": "", "entries": [\n'
                   ' {"precision": 1, "bucket": 12, "group": 4, "ctas_per_sm": 2, "ms": 1.5},\n'
                   ' {"precision": 0, "bucket": 16, "group": 1, "ctas_per_sm": 3, "tile_rows": 4, "ms": 9},\n'
                   ' {"precision": 1, "bucket": 14, "group": 0, "ctas_per_sm": 0, "ms": 2.5},\n'
                   ' {"stage_launch": 1, "bucket": 21, "tile_rows": 2, "threads_per_cell": 2, "ms": 0.1}\n]}\n')
    M.mprk_tune_load(str(src))
    assert M.mprk_tune_lookup(1, 5000.0) == {"tiles_per_item": 4, "ctas_per_sm": 2, "tile_rows": 16,
                                             "tuned": True}  # 2^12 <= 5000
    assert M.mprk_tune_lookup(1, 9000.0)["tuned"] is False                                            # bucket 13
    assert M.mprk_tune_lookup(1, 20000.0) == {"tiles_per_item": 0, "ctas_per_sm": 0, "tile_rows": 16,
                                              "tuned": True}  # the per-stage form, bucket 14
    assert M.mprk_tune_lookup(0, 70000.0) == {"tiles_per_item": 1, "ctas_per_sm": 3, "tile_rows": 4,
                                              "tuned": True}
    assert M.mprk_tile_lookup(2.5e6) == {"tile_rows": 2, "threads_per_cell": 2}  # 2^21 <= 2.5e6 < 2^22
    assert M.mprk_tile_lookup(5e6) is None
    out = tmp_path / "u.json"
    M.mprk_tune_save(str(out))
    M.mprk_tune_clear()
    assert M.mprk_tile_lookup(2.5e6) is None
    M.mprk_tune_load(str(out))
    assert M.mprk_tune_lookup(0, 70000.0)["tiles_per_item"] == 1
    assert M.mprk_tune_lookup(0, 70000.0)["tile_rows"] == 4
    assert M.mprk_tile_lookup(2.5e6) == {"tile_rows": 2, "threads_per_cell": 2}
    for bad_entry in ('{"precision": 1, "bucket": 12, "group": -1, "ctas_per_sm": 2}',
                      '{"precision": 0, "bucket": 12, "group": 0, "ctas_per_sm": 2}',
                      '{"precision": 0, "bucket": 12, "group": 2, "ctas_per_sm": 2, "tile_rows": 2}',
                      '{"stage_launch": 1, "bucket": 21, "tile_rows": 3, "threads_per_cell": 1}',
                      '{"stage_launch": 1, "bucket": 21, "tile_rows": 8, "threads_per_cell": 4}',
                      '{"stage_launch": 1, "bucket": 21, "tile_rows": 8}'):
        bad = tmp_path / "bad.json"
        bad.write_text('{"gpu": "", "entries": [' + bad_entry + ']}')
        with pytest.raises(M.MprkError):
            M.mprk_tune_load(str(bad))
    M.mprk_tune_clear()


def test_binding_rejects_buffers_it_cannot_pass_as_pointers():
    """The binding hands raw pointers to the library, so it takes only
    C-contiguous float64 arrays and tensors and raises TypeError otherwise
    (also under python -O)."""
    from paper_2202_11890_gb300 import mprk as M
    a = np.zeros((4, 3, 5))
    assert M._ptr(a) == (a.ctypes.data, M.MPRK_HOST)
    for bad in (np.zeros((4, 3, 5), dtype=np.float32), np.zeros((4, 3, 10))[:, :, ::2], [0.0] * 4):
        with pytest.raises(TypeError):
            M._ptr(bad)
    torch = pytest.importorskip("torch")
    t = torch.zeros(4, 3, 5, dtype=torch.float64)
    assert M._ptr(t) == (t.data_ptr(), M.MPRK_HOST)
    for bad in (torch.zeros(4, 3, 5), torch.zeros(4, 5, 3, dtype=torch.float64).transpose(1, 2)):
        with pytest.raises(TypeError):
            M._ptr(bad)


def test_static_entry_point_checks_the_fp32flux_layout_without_a_device(lib):
    """mprk_step_static's FP32-flux mode moves whole 256-byte row segments
    of the caller's unpadded state, so it takes only nx a multiple of 32 and
    a 256-byte aligned state; it says so before any CUDA call. (The pointer
    values are never dereferenced: the call returns first.)"""
    from paper_2202_11890_gb300 import mprk as M
    cases = [(45, 4096), (64, 4096 + 8), (96, 4096 + 128)]
    for nx, addr in cases:
        cfg = M.mprk_config_default(nx, 8, 4, 8, 2, dt=1e-3)
        cfg.precision = M.MPRK_FP32FLUX
        rc = M.lib().mprk_step_static(C.byref(cfg), C.c_void_p(addr), 1, None)
        assert rc == M.MPRK_EINVAL, (nx, addr, rc)
        assert "multiple of 32" in M.mprk_last_error()
