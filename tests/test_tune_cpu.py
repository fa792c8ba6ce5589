"""The autotuner's cache logic on the CPU, with the library calls replaced by a
fake: a search runs only for sides the cache lacks, its results are written
atomically under a key that names the GPU, driver, library version, dtype and
filter side, and malformed records count as absent."""
import json

import pytest

from paper_1302_5586_gb300 import tune


class FakeLib:
    PENCIL_F32, PENCIL_F16, PENCIL_BATCH_VARIANTS = 0, 1, 2

    def __init__(self, measured=1, version=100):
        self.set_calls, self.tune_calls = [], []
        self.measured, self.version = measured, version

    def pencil_device_info(self):
        return ("Fake GB300", 152, 13000)

    def pencil_version(self):
        return self.version

    def pencil_batch_set_variant(self, plan, ks, v):
        self.set_calls.append((ks, v))

    def make_images(self, items):
        return list(items)

    def pencil_tune(self, plan, imgs, reps, stream):
        self.tune_calls.append((sorted({it[5] for it in imgs}), reps, stream))
        return {ks: self.measured for ks in sorted({it[5] for it in imgs})}


def items(*sides):
    return [(None, None, None, 8, 8, ks) for ks in sides]


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(tune, "b", f)
    return f


def test_search_then_cache(fake, tmp_path):
    path = str(tmp_path / "sub" / "t.json")
    first = tune.autotune("plan", 0, items(3, 15, 3), reps=4, path=path, stream="s")
    assert first == {3: (1, "measured"), 15: (1, "measured")}
    assert fake.tune_calls == [([3, 15], 4, "s")]
    with open(path) as f:
        rec = json.load(f)
    assert sorted(rec) == ["Fake GB300|sm152|drv13000|lib100|f32|k15", "Fake GB300|sm152|drv13000|lib100|f32|k3"]
    again = tune.autotune("plan", 0, items(3, 15, 7), path=path, stream="s")
    assert again == {3: (1, "cache"), 15: (1, "cache"), 7: (1, "measured")}
    assert fake.tune_calls[-1] == ([7], 5, "s")  # only the side the cache lacked
    assert (3, 1) in fake.set_calls and (15, 1) in fake.set_calls
    assert tune.cached_variants(0, path) == {3: 1, 7: 1, 15: 1}
    assert tune.cached_variants(1, path) == {}  # binary16 never tuned
    assert not [p for p in (tmp_path / "sub").iterdir() if p.name.endswith(".tmp")]


def test_key_names_the_library_version(fake, tmp_path):
    path = str(tmp_path / "t.json")
    tune.autotune("plan", 0, items(5), path=path, stream="s")
    fake.version = 101  # a rebuilt library: old records do not apply
    assert tune.cached_variants(0, path) == {}
    assert tune.autotune("plan", 0, items(5), path=path, stream="s") == {5: (1, "measured")}


@pytest.mark.parametrize("bad", [{"variant": 7}, {"variant": -1}, {"variant": "x"}, {}, 3, None])
def test_malformed_record_is_a_miss(fake, tmp_path, bad):
    path = str(tmp_path / "t.json")
    key = "Fake GB300|sm152|drv13000|lib100|f32|k9"
    with open(path, "w") as f:
        json.dump({key: bad}, f)
    assert tune.cached_variants(0, path) == {}
    assert tune.autotune("plan", 0, items(9), path=path, stream="s") == {9: (1, "measured")}
    with open(path) as f:
        assert json.load(f)[key]["variant"] == 1  # replaced by the measurement


@pytest.mark.parametrize("text", ["not json", "[1, 2]", ""])
def test_unreadable_cache_file_is_empty(fake, tmp_path, text):
    path = tmp_path / "t.json"
    path.write_text(text)
    assert tune.cached_variants(0, str(path)) == {}
    assert tune.autotune("plan", 0, items(3), path=str(path), stream="s") == {3: (1, "measured")}


def test_no_cache_leaves_no_file(fake, tmp_path):
    path = tmp_path / "t.json"
    assert tune.autotune("plan", 1, items(3), use_cache=False, path=str(path), stream="s") == {3: (1, "measured")}
    assert not path.exists()


def test_bare_file_name_and_env_path(fake, tmp_path, monkeypatch):
    monkeypatch.chdir(tmp_path)
    tune.autotune("plan", 0, items(3), path="t.json", stream="s")
    assert (tmp_path / "t.json").exists()
    monkeypatch.setenv("PENCIL_TUNE_CACHE", str(tmp_path / "env.json"))
    assert tune.cache_path() == str(tmp_path / "env.json")
    tune.autotune("plan", 0, items(3), stream="s")
    assert (tmp_path / "env.json").exists()
