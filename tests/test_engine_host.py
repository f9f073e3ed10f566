"""Host-side logic of the batch executor, the autotuner table and the request
server: argument checks and the tuning file, all before any device work (no
GPU needed)."""
import ctypes
import json

import pytest

from paper_2512_04317_gb300 import build, mxfft


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mxfft.load()


def test_engine_and_server_argument_checks(lib):
    h = ctypes.c_void_p()
    for tau, target, flags in [(0.0, 0.5, 0), (1.0, 0.5, 0), (1e-3, -1.0, 0), (1e-3, 0.5, 32)]:
        assert lib.mxfft_engine_create(tau, target, flags, ctypes.byref(h)) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_engine_create(1e-3, 0.3, 0, ctypes.byref(h)) == mxfft.MXFFT_ERR_UNSUPPORTED
    assert lib.mxfft_engine_create(1e-3, 0.5, 0, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_engine_run(None, None, 0, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_engine_get_status(None, None, None, 0) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_engine_destroy(None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_tune(None, 1, None, None) == mxfft.MXFFT_ERR_INVALID
    for slots, mbs in [(0, 16), (65, 16), (2, 0)]:
        cfg = mxfft.ServerConfig(slots, mbs, 0, 1e-3, 0.5, 0, 0)
        assert lib.mxfft_server_create(ctypes.byref(cfg), ctypes.byref(h)) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_server_submit(None, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_server_poll(None, None, 0, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_server_wait(None, 1.0) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_server_stats(None, None, None, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_server_destroy(None) == mxfft.MXFFT_ERR_INVALID


def test_item_and_request_layouts_match_the_header():
    # field offsets of the C structs (x86-64 and aarch64 LP64)
    assert ctypes.sizeof(mxfft.Item) == 56 and mxfft.Item.in_.offset == 24
    assert mxfft.Item.rss.offset == 48
    assert ctypes.sizeof(mxfft.Request) == 64 and mxfft.Request.tag.offset == 40
    assert mxfft.Request.host_rss.offset == 56
    assert ctypes.sizeof(mxfft.Completion) == 40 and mxfft.Completion.t_done_us.offset == 32
    assert ctypes.sizeof(mxfft.ServerConfig) == 40 and mxfft.ServerConfig.tau.offset == 16
    assert mxfft.ServerConfig.max_batch_bytes.offset == 32


def test_tuning_file_round_trip(lib, tmp_path):
    mxfft.mxfft_tune_clear()
    empty = tmp_path / "empty.json"
    mxfft.mxfft_tune_save(str(empty))
    assert json.loads(empty.read_text()) == {"mxfft_tune": 1, "entries": []}
    # n = 256 rows of a 256 x 256 slice: groups of 16 transforms x 8 threads,
    # so 1, 2 or 4 groups per CTA
    entry = {"n": 256, "other": 256, "dim": 1, "fmt": 0, "m": 16, "batch_class": 6, "ng": 2,
             "us": 1.0}
    f = tmp_path / "one.json"
    f.write_text(json.dumps({"mxfft_tune": 1, "entries": [entry]}))
    mxfft.mxfft_tune_load(str(f))
    out = tmp_path / "out.json"
    mxfft.mxfft_tune_save(str(out))
    got = json.loads(out.read_text())["entries"]
    assert len(got) == 1
    assert {k: got[0][k] for k in entry if k != "us"} == {k: entry[k] for k in entry if k != "us"}
    # a tensor-core entry (resident CTAs per SM of its persistent grid) beside it
    tc = {"kind": 1, "n": 512, "other": 512, "dim": 0, "fmt": 0, "m": 1, "batch_class": 9,
          "tile": 2048, "ctas_per_sm": 4, "us": 2.0}
    f.write_text(json.dumps({"mxfft_tune": 1, "entries": [tc]}))
    mxfft.mxfft_tune_load(str(f))
    mxfft.mxfft_tune_save(str(out))
    got = json.loads(out.read_text())["entries"]
    assert len(got) == 2
    kinds = {g.get("kind", 0): g for g in got}
    assert {k: kinds[1][k] for k in tc if k != "us"} == {k: tc[k] for k in tc if k != "us"}
    assert "ctas_per_sm" not in kinds[0] and kinds[0]["ng"] == 2
    mxfft.mxfft_tune_clear()
    mxfft.mxfft_tune_save(str(out))
    assert json.loads(out.read_text())["entries"] == []


@pytest.mark.parametrize("bad", [
    "not json",
    '{"entries": []}',                                                     # no magic key
    '{"mxfft_tune": 1, "entries": [{"n": 256, "other": 256}]}',            # missing fields
    '{"mxfft_tune": 1, "entries": [{"n": 256, "other": 256, "dim": 1, "fmt": 0, "m": 16,'
    ' "batch_class": 6, "ng": 3}]}',                                       # not a candidate
    '{"mxfft_tune": 1, "entries": [{"n": 256, "other": 256, "dim": 1, "fmt": 0, "m": 16,'
    ' "batch_class": 6, "ng": 8}]}',                                       # 1024 threads
    '{"mxfft_tune": 1, "entries": [{"kind": 1, "n": 512, "other": 512, "dim": 1, "fmt": 0,'
    ' "m": 1, "batch_class": 6, "ctas_per_sm": 9}]}',                      # above 8 per SM
    '{"mxfft_tune": 1, "entries": [{"kind": 1, "n": 2048, "other": 512, "dim": 1, "fmt": 0,'
    ' "m": 1, "batch_class": 6, "tile": 2048, "ctas_per_sm": 4}]}',        # 128 threads, n > 1024
    '{"mxfft_tune": 1, "entries": [{"kind": 1, "n": 512, "other": 512, "dim": 1, "fmt": 0,'
    ' "m": 1, "batch_class": 6, "tile": 1024, "ctas_per_sm": 4}]}',        # no such tile
    '{"mxfft_tune": 1, "entries": [{"kind": 1, "n": 64, "other": 512, "dim": 1, "fmt": 0,'
    ' "m": 1, "batch_class": 6, "ctas_per_sm": 1}]}',                      # no tensor-core pass
    '{"mxfft_tune": 1, "entries": [{"kind": 1, "n": 512, "other": 512, "dim": 1, "fmt": 2,'
    ' "m": 1, "batch_class": 6, "ctas_per_sm": 1}]}',                      # 6-bit format
    '{"mxfft_tune": 1, "entries": [{"kind": 2, "n": 256, "other": 256, "dim": 1, "fmt": 0,'
    ' "m": 16, "batch_class": 6, "ng": 2}]}',                              # unknown kind
    '{"mxfft_tune": 1, "entries": [{"kind": 1, "n": 512, "other": 512, "dim": 1, "fmt": 0,'
    ' "m": 1, "batch_class": 6, "ng": 1}]}',                               # field of the other kind
])
def test_tuning_file_rejects_malformed(lib, tmp_path, bad):
    f = tmp_path / "bad.json"
    f.write_text(bad)
    with pytest.raises(mxfft.MxfftError) as ei:
        mxfft.mxfft_tune_load(str(f))
    assert ei.value.status == mxfft.MXFFT_ERR_INVALID
    with pytest.raises(mxfft.MxfftError):
        mxfft.mxfft_tune_load(str(tmp_path / "missing.json"))


def test_rss_argument_checks(lib):
    bad = [(-1, 1, 4, 4), (1, 0, 4, 4), (1, 1, 0, 4)]
    for images, coils, n0, n1 in bad:
        assert lib.mxfft_rss(None, None, images, coils, n0, n1, None) == mxfft.MXFFT_ERR_INVALID
    assert lib.mxfft_rss(None, None, 1, 1, 4, 4, None) == mxfft.MXFFT_ERR_INVALID   # null
    # z occupies [16, 144), out [64, 128): overlapping
    assert lib.mxfft_rss(16, 64, 1, 1, 4, 4, None) == mxfft.MXFFT_ERR_INVALID       # overlap
    assert lib.mxfft_rss(8, 65536, 1, 1, 4, 4, None) == mxfft.MXFFT_ERR_INVALID     # alignment
    assert lib.mxfft_rss(None, None, 0, 1, 4, 4, None) == mxfft.MXFFT_OK            # nothing
