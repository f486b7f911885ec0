"""Host logic (no GPU) of the autograd form: the rasterizer pool and the key
capacity kept in line with the counts, with the library's device calls
replaced by host fakes."""
import pytest
import torch

from synth import scenes as S


class _FakeRast:
    def __init__(self, capacity):
        self.capacity = capacity
        self.device = torch.device("cpu")
        self.keys = torch.empty(capacity, dtype=torch.int64)
        self.vals = torch.empty(capacity, dtype=torch.int32)
        self._ws_sort = self._ws_pb = self._bm = object()
        self.n_keys = torch.zeros(1, dtype=torch.int64)


def test_capacity_follows_the_counts(monkeypatch):
    """The backward's one synchronisation: under 90 % of the capacity nothing
    changes; above it the capacity grows to 1.25 n + 4096 for the next call
    (new key buffers, the capacity-sized scratch dropped); an overflow resets
    the device status, grows the capacity and raises; another device error
    is raised as it is."""
    from paper_2510_06644_gb300 import autograd as A, gs
    status = {"code": gs.GS_OK}
    resets = []
    monkeypatch.setattr(gs, "gs_status_poll", lambda blocking=True, stream=None: (status["code"], 0))
    monkeypatch.setattr(gs, "gs_status_reset", lambda stream=None: resets.append(1))
    r = _FakeRast(10000)
    r.n_keys.fill_(8500)
    A._settle(r)
    assert r.capacity == 10000 and r._bm is not None
    keys = r.keys
    A._grow(r, 10000)   # not larger: the buffers stay
    assert r.keys is keys and r._bm is not None
    # exactly the capacity still fits (then grows for the next call)
    r.n_keys.fill_(10000)
    A._settle(r)
    assert r.capacity == int(10000 * 1.25) + 4096
    r = _FakeRast(10000)
    r.n_keys.fill_(9500)
    A._settle(r)
    assert r.capacity == int(9500 * 1.25) + 4096 == r.keys.numel() == r.vals.numel()
    assert r._ws_sort is None and r._ws_pb is None and r._bm is None
    status["code"] = gs.GS_ERR_CAPACITY
    r.n_keys.fill_(50000)
    with pytest.raises(gs.GsError) as e:
        A._settle(r)
    assert e.value.code == gs.GS_ERR_CAPACITY and resets == [1]
    assert r.capacity == int(50000 * 1.25) + 4096
    status["code"] = gs.GS_ERR_INVALID_ARG
    r.n_keys.fill_(10)
    with pytest.raises(gs.GsError) as e:
        A._settle(r)
    assert e.value.code == gs.GS_ERR_INVALID_ARG and resets == [1]
    # a count above the capacity without the device flag is an overflow too
    status["code"] = gs.GS_OK
    r.n_keys.fill_(r.capacity + 1)
    with pytest.raises(gs.GsError):
        A._settle(r)


def test_pool_lends_one_rasterizer_per_grid_and_record_type(monkeypatch):
    """A rasterizer is built (its keys counted once) only when none of the
    same (n, sampled grid, strides, record type, device) is free; given back,
    it is lent again with the caller's config."""
    from paper_2510_06644_gb300 import autograd as A, gs
    built, counts = [], []

    class FakeRasterizer(_FakeRast):
        def __init__(self, n, cam, cfg, rec_dtype, capacity, device):
            super().__init__(capacity)
            self.cfg = cfg
            built.append((n, cam["W"], cam.get("sx", 1), rec_dtype, capacity))

    monkeypatch.setattr(A, "Rasterizer", FakeRasterizer)
    monkeypatch.setattr(gs, "gs_project", lambda cfg, cs, g, rec_dtype=gs.GS_F32: None)

    def fake_count(cs, probe, n, rec_dtype=gs.GS_F32, cfg=None):
        counts.append(n)
        return torch.tensor([3000])

    monkeypatch.setattr(gs, "gs_bin_count", fake_count)
    pool = A._Pool()
    cam = S.camera(96, 72, 80.0)
    a = pool.take(100, cam, "cfgA", gs.GS_F32, "cpu", None)
    assert a.capacity == int(3000 * 1.25) + 4096 and counts == [100]
    b = pool.take(100, cam, "cfgA", gs.GS_F32, "cpu", None)   # a is still lent out
    assert b is not a and len(built) == 2
    pool.give(a)
    c = pool.take(100, cam, "cfgB", gs.GS_F32, "cpu", None)
    assert c is a and c.cfg == "cfgB" and len(built) == 2
    for other in (dict(cam, sx=2, sy=2), dict(cam, W=97)):
        pool.give(c)
        d = pool.take(100, other, "cfgB", gs.GS_F32, "cpu", None)
        assert d is not a
        pool.take(100, cam, "cfgB", gs.GS_F32, "cpu", None)   # takes a back
    pool.give(a)
    assert pool.take(100, cam, "cfgB", gs.GS_BF16, "cpu", None) is not a
    assert pool.take(101, cam, "cfgB", gs.GS_F32, "cpu", None) is not a
    assert pool.take(100, cam, "cfgB", gs.GS_F32, "cpu", None) is a
