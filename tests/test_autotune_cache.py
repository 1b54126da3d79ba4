"""The JSON cache of launch shapes (api.autotune_cached): a miss tunes and
stores the choice under (device, ring degree, chain), a hit sets it without
tuning, other chains or devices miss, and a corrupt file is treated as empty.
The tuner and the device query are replaced by fakes (no GPU needed)."""
import json

from paper_2408_07304_gb300 import api


class _Ctx:
    def __init__(self, log_n, primes, device=0):
        self.log_n, self.primes, self.device = log_n, primes, device
        self.variant = None


def test_autotune_cache(tmp_path, monkeypatch):
    calls = []
    monkeypatch.setattr(api, "_device_name", lambda d: f"GPU{d}")
    monkeypatch.setattr(api, "zn_autotune", lambda ctx, pk, zc, b: (calls.append(b) or (5, [1.0] * 8)))
    monkeypatch.setattr(api, "zn_set_variant", lambda ctx, v: setattr(ctx, "variant", v))
    path = str(tmp_path / "tune.json")
    a = _Ctx(14, [11, 13])
    assert api.autotune_cached(a, None, None, 64, path) == (5, False) and calls == [64]
    assert json.load(open(path)) == {"GPU0|14|11,13": 5}
    b = _Ctx(14, [11, 13])
    assert api.autotune_cached(b, None, None, 64, path) == (5, True) and b.variant == 5 and calls == [64]
    c = _Ctx(14, [11, 17])
    assert api.autotune_cached(c, None, None, 64, path) == (5, False) and len(calls) == 2
    d = _Ctx(14, [11, 13], device=1)
    assert api.autotune_cached(d, None, None, 64, path)[1] is False and len(calls) == 3
    assert len(json.load(open(path))) == 3
    open(path, "w").write("{not json")
    assert api.autotune_cached(a, None, None, 64, path) == (5, False) and len(calls) == 4
