"""Host logic of the stream-collide variant cache (no GPU): the winner of a
timing run is stored per (device, storage, lattice), reused on the next run,
and timed again when the library refuses the stored variant."""
from paper_1110_0995_gb300 import autotune, lbibm


class FakeSim:
    def __init__(self, dims, offered=None, best=(2, 256, 0.05)):
        self.dims = dims
        self.offered = offered
        self.best = best
        self.timed = 0
        self.config = None

    def autotune(self, repeats):
        self.timed += 1
        self.config = self.best[:2]
        return self.best

    def set_kernel_config(self, npt, bs):
        if self.offered is not None and (npt, bs) not in self.offered:
            raise lbibm.LbError(lbibm.LB_ERR_ARG, "no such variant")
        self.config = (npt, bs)

    pf = 0

    def set_prefetch(self, d):
        self.pf = d

    def prefetch(self):
        return self.pf


def test_cache_stores_reuses_and_retunes(tmp_path, monkeypatch):
    monkeypatch.setenv("LBIBM_CACHE", str(tmp_path / "at.json"))
    a = FakeSim([(256, 128, 64)])
    a.pf = 65536                      # the distance the library's autotuner kept
    r = autotune.tune(a, "GB300", "f32")
    assert not r["cached"] and a.timed == 1 and (r["npt"], r["bs"], r["pf"]) == (2, 256, 65536)
    b = FakeSim([(256, 128, 64)])
    r = autotune.tune(b, "GB300", "f32")
    assert r["cached"] and b.timed == 0 and b.config == (2, 256) and b.pf == 65536
    # another lattice, storage or device is a separate entry
    for sim, dev, st in ((FakeSim([(128, 64, 64)]), "GB300", "f32"), (FakeSim([(256, 128, 64)]), "GB300", "f16"),
                         (FakeSim([(256, 128, 64)]), "other", "f32")):
        assert not autotune.tune(sim, dev, st)["cached"] and sim.timed == 1
    # the library no longer offers the stored variant: time again, store the new winner
    c = FakeSim([(256, 128, 64)], offered={(1, 1152)}, best=(1, 1152, 0.04))
    r = autotune.tune(c, "GB300", "f32")
    assert not r["cached"] and c.timed == 1 and c.config == (1, 1152)
    d = FakeSim([(256, 128, 64)], offered={(1, 1152)})
    assert autotune.tune(d, "GB300", "f32")["cached"] and d.config == (1, 1152)


def test_unwritable_cache_still_tunes(tmp_path, monkeypatch):
    blocker = tmp_path / "file"
    blocker.write_text("")
    monkeypatch.setenv("LBIBM_CACHE", str(blocker / "sub" / "at.json"))   # parent is a file
    s = FakeSim([(64, 32, 32)])
    r = autotune.tune(s, "GB300", "f32")
    assert not r["cached"] and s.timed == 1
