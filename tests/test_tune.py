"""Host-side checks of the autotuner cache (no GPU needed): the shape bucket,
the text form, lookups, and that workspace queries account for a tuned
configuration."""
import ctypes as ct
import math

import pytest

from paper_2608_06536_b300 import build as pkg_build
from paper_2608_06536_b300 import jk


@pytest.fixture()
def lib():
    pkg_build.build()
    L = jk.load_library()
    L.jk_tune_clear()
    yield L
    L.jk_tune_clear()


def _problem(n, naux, ks):
    f = (jk.jk_factor * 1)(jk.jk_factor(n, naux, 0x1000))
    d = (jk.jk_density * len(ks))()
    for s, k in enumerate(ks):
        d[s].k, d[s].symmetric, d[s].X, d[s].Y = k, 0, 0x2000, 0x3000
    return f, d


def _line(op, prec, sms, nmol, n, naux, nd, ksum, cfg, ms=1.5):
    # bucket: nbf in steps of 32, naux in steps of 256, width in steps of 16
    tile = cfg[3] if len(cfg) > 3 else 0
    return (f"jk-tune 4 {op} {prec} {sms} {nmol} {math.ceil(n / 32)} {math.ceil(naux / 256)} {nd} "
            f"{math.ceil(ksum / 16)} {cfg[0]} {cfg[1]} {cfg[2]} {tile} {ms:.6f}\n")


def _lookup(lib, n, naux, ks, prec=jk.JK_SPLIT_BF16, sms=148):
    f, d = _problem(n, naux, ks)
    cfg = jk.jk_tune_config()
    st = lib.jk_tune_lookup(jk.JK_OP_BUILD, 1, f, None, len(ks), d, prec, sms, ct.byref(cfg))
    return st, cfg.as_dict()


def test_empty_cache(lib):
    assert jk.tune_export() == ""
    st, _ = _lookup(lib, 400, 2400, [40] * 8)
    assert st == jk.JK_ERR_UNSUPPORTED


def test_import_lookup_and_bucket(lib):
    jk.tune_import(_line(0, 1, 148, 1, 400, 2400, 8, 320, (600, 1, 0)))
    st, cfg = _lookup(lib, 400, 2400, [40] * 8)
    assert st == jk.JK_OK and cfg == {"aux_chunk": 600, "schedule": 1, "raster": 0, "tile": 0}
    # same bucket: nbf 385..416, naux 2305..2560, same count, width 305..320
    assert _lookup(lib, 390, 2500, [39] * 8)[0] == jk.JK_OK
    # other buckets, other SM count, other precision
    assert _lookup(lib, 420, 2400, [40] * 8)[0] == jk.JK_ERR_UNSUPPORTED
    assert _lookup(lib, 400, 2600, [40] * 8)[0] == jk.JK_ERR_UNSUPPORTED
    assert _lookup(lib, 400, 2400, [40] * 7)[0] == jk.JK_ERR_UNSUPPORTED
    assert _lookup(lib, 400, 2400, [40] * 8, sms=132)[0] == jk.JK_ERR_UNSUPPORTED
    assert _lookup(lib, 400, 2400, [40] * 8, prec=jk.JK_FP64)[0] == jk.JK_ERR_UNSUPPORTED


def test_export_round_trip_and_later_entries_win(lib):
    a = _line(0, 1, 148, 1, 400, 2400, 8, 320, (600, 1, 0))
    b = _line(0, 0, 148, 1, 1000, 5000, 16, 1600, (40, 0, 0))
    jk.tune_import("# saved cache\n\n" + a + b)
    text = jk.tune_export()
    assert len(text.splitlines()) == 2
    jk.tune_clear()
    jk.tune_import(text)
    assert jk.tune_export() == text
    jk.tune_import(_line(0, 1, 148, 1, 400, 2400, 8, 320, (300, 0, 1, 1)))
    assert _lookup(lib, 400, 2400, [40] * 8)[1] == {"aux_chunk": 300, "schedule": 0, "raster": 1, "tile": 1}
    # export into a short buffer: truncated, NUL-terminated, full length reported
    n = ct.c_size_t()
    buf = ct.create_string_buffer(10)
    assert lib.jk_tune_export(buf, 10, ct.byref(n)) == jk.JK_OK
    assert n.value == len(jk.tune_export()) and len(buf.value) == 9


@pytest.mark.parametrize("bad", [
    "jk-tune 3 0 1 148 1 13 10 8 20 600 1 0 1.0",         # an older version (no tile width)
    "jk-tune 4 0 1 148 1 13 10 8 20 600 2 0 0 1.0",       # schedule out of range
    "jk-tune 4 0 1 148 1 13 10 8 20 600 0 2 0 1.0",       # raster out of range
    "jk-tune 4 0 1 148 1 13 10 8 20 600 0 0 2 1.0",       # tile out of range
    "jk-tune 4 0 1 148 1 13 10 8 20 -5 0 0 0 1.0",        # negative chunk
    "jk-tune 4 0 1 148 1 13 10 8 20 600 0 0 0",           # missing field
    "jk-tune 4 0 1 148 1 13 10 8 20 600 0 0 0 1.0 extra", # trailing text
    "tune 4 0 1 148 1 13 10 8 20 600 0 0 0 1.0",          # wrong tag
])
def test_malformed_lines_rejected(lib, bad):
    good = _line(0, 1, 148, 1, 400, 2400, 8, 320, (600, 1, 0))
    with pytest.raises(jk.JKError):
        jk.tune_import(good + bad + "\n")
    # entries before the bad line are kept
    assert _lookup(lib, 400, 2400, [40] * 8)[0] == jk.JK_OK


def test_query_covers_tuned_configuration(lib):
    """A handle-free query answers for the larger of the default and the
    tuned configuration (the SM count is 0 where no device is visible)."""
    f, d = _problem(400, 2400, [40] * 8)
    nb = ct.c_size_t()
    assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, f, None, 8, d, jk.JK_SPLIT_BF16, ct.byref(nb)) == jk.JK_OK
    base = nb.value
    sms = 0
    import torch
    if torch.cuda.is_available():
        sms = torch.cuda.get_device_properties(0).multi_processor_count
    # a tuned chunk of all 2400 aux indices needs more than the automatic one
    jk.tune_import(_line(0, 1, sms, 1, 400, 2400, 8, 320, (2400, 0, 0)))
    assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, f, None, 8, d, jk.JK_SPLIT_BF16, ct.byref(nb)) == jk.JK_OK
    assert nb.value > base
    # a small tuned chunk never lowers the answer below the default's
    jk.tune_import(_line(0, 1, sms, 1, 400, 2400, 8, 320, (100, 0, 0)))
    assert lib.jk_workspace_query(jk.JK_OP_BUILD, 1, f, None, 8, d, jk.JK_SPLIT_BF16, ct.byref(nb)) == jk.JK_OK
    assert nb.value == base
