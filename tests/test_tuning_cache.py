"""The autotuner's JSON cache (host logic of the binding): keys, atomic
writes, format versions, and the cached path of api.autotune with the
library calls replaced by fakes (no GPU)."""
import json
import os

import pytest

from paper_2103_09943_gb300 import api


def test_key_names_gpu_sizes_and_scene_flag():
    k = api.tuning_cache_key("GB300", 8, 2048, 2048, 4, 7, 1, False)
    assert k == "GB300|N=8|H=2048|W=2048|ratio=4|R=7|r=1|scene=0"
    assert api.tuning_cache_key("GB300", 8, 2048, 2048, 4, 7, 1, True) != k
    assert api.tuning_cache_key("B200", 8, 2048, 2048, 4, 7, 1, False) != k


def test_write_read_roundtrip_and_version(tmp_path):
    path = str(tmp_path / "tuning.json")
    assert api.read_tuning_cache(path) == {}
    entries = {"a": {"choices": {"prec_rows": 4}}}
    api.write_tuning_cache(path, entries)
    assert api.read_tuning_cache(path) == entries
    assert os.listdir(tmp_path) == ["tuning.json"]          # no temporary left behind
    with open(path, "w") as fh:
        json.dump({"version": 0, "entries": entries}, fh)
    assert api.read_tuning_cache(path) == {}                # another format: ignored


def test_autotune_uses_and_fills_the_cache(tmp_path, monkeypatch):
    path = str(tmp_path / "tuning.json")
    monkeypatch.setattr(api.torch.cuda, "get_device_name", lambda dev=None: "FakeGPU")
    calls = {"set": [], "timed": 0}
    choices = {k: 1 for k in api.TUNING_CHOICES}
    key = api.tuning_cache_key("FakeGPU", 4, 256, 256, 4, 5, 1, False)
    api.write_tuning_cache(path, {key: {"choices": choices}})
    monkeypatch.setattr(api, "set_tuning",
                        lambda *a, **kw: calls["set"].append((a, kw)))
    out = api.autotune(4, 256, 256, 4, 5, 1, device="cpu", cache=path)
    assert out["cached"] is True and calls["set"] == [((4, 256, 256, 4, 1), choices)]

    # a miss times (here: a fake library) and adds the record
    class FakeLib:
        def ps_autotune(self, *args):
            calls["timed"] += 1
            t = args[-1]._obj
            t.prec_rows, t.llp_rows, t.llp_pf, t.split = 2, 66, 3, 0
            t.llp_bands, t.prec_impl, t.db_impl, t.llp_form = 1, 2, 1, 2
            return 0
    monkeypatch.setattr(api._lib, "load", lambda *a: FakeLib())
    monkeypatch.setattr(api, "workspace", lambda *a, **kw: _FakeWs())
    monkeypatch.setattr(api, "_stream", lambda: None)
    out = api.autotune(8, 512, 512, 4, 6, 1, device="cpu", cache=path)
    assert calls["timed"] == 1 and out["llp_form"] == 2
    entries = api.read_tuning_cache(path)
    rec = entries[api.tuning_cache_key("FakeGPU", 8, 512, 512, 4, 6, 1, False)]
    assert rec["choices"] == {"prec_rows": 2, "llp_rows": 66, "llp_pf": 3, "split": 0,
                              "llp_bands": 1, "prec_impl": 2, "db_impl": 1, "llp_form": 2}
    assert key in entries                                   # earlier records kept


class _FakeWs:
    def data_ptr(self):
        return 0

    def numel(self):
        return 0
