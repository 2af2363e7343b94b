"""Host logic of the autotuner (no GPU): candidate lists, the choice of the
fastest candidate per kernel, and the JSON cache, with a fake simulation that
reports made-up kernel times."""
import pytest

from paper_1612_03310_gb300 import autotune, inputs


class FakeSim:
    made = 0

    def __init__(self, grid, und, bunch, precision=1, stream=None):
        FakeSim.made += 1
        self.t = dict(stencil_variant=1, lz=0, push_variant=1, push_ctas_per_sm=0,
                      push_sparse_below=0)
        self.closed = False

    def step(self, n):
        pass

    def set_tuning(self, **kw):
        self.t.update(kw)

    def profile(self, on):
        pass

    def kernel_times(self):
        t = self.t
        # stencil: marching with lz = 32 fastest; push: tiled with 2 CTAs/SM
        # and sparse tiles below 64
        st = 1.0 if t["stencil_variant"] == 0 else 0.5 + abs(t["lz"] - 32) / 100.0
        pu = 2.0 if t["push_variant"] == 0 else 0.4 + abs(t["push_ctas_per_sm"] - 2) / 10.0
        if t["push_variant"] == 1 and t["push_sparse_below"]:
            pu -= 0.1 - abs(t["push_sparse_below"] - 64) / 1000.0
        return {"potential_step": (st * 4, 4), "push": (pu * 4, 4)}

    def close(self):
        self.closed = True


@pytest.fixture
def fake(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "CACHE_DIR", str(tmp_path))
    monkeypatch.setattr(autotune.mithra, "Simulation", FakeSim)
    monkeypatch.setattr(autotune, "device_name", lambda: "fake")
    FakeSim.made = 0
    return FakeSim


def test_candidates_cover_both_forms():
    g = inputs.workload("c2")["grid"]
    st = autotune.stencil_candidates(g)
    assert dict(stencil_variant=0, lz=0) in st
    assert all(c["lz"] <= g["nz"] for c in st)
    assert any(c["stencil_variant"] == 1 for c in st)
    pu = autotune.push_candidates(3)
    assert dict(push_variant=0, push_ctas_per_sm=0, push_sparse_below=0) in pu
    assert [c["push_ctas_per_sm"] for c in pu if c["push_variant"] == 1] == [1, 2, 3]
    assert autotune.sparse_candidates(pu[0]) == []
    sp = autotune.sparse_candidates(pu[2])
    assert [c["push_sparse_below"] for c in sp] == list(autotune.SPARSE_THRESHOLDS)
    assert all(c["push_ctas_per_sm"] == pu[2]["push_ctas_per_sm"] for c in sp)


def test_picks_fastest_and_caches(fake):
    g = inputs.random_grid(0, 64, 64, 256)
    b = inputs.random_particles(1, g, 1000)
    best = autotune.tune(g, None, b, 1)
    assert best == dict(stencil_variant=1, lz=32, push_variant=1, push_ctas_per_sm=2,
                        push_sparse_below=64)
    assert fake.made == 1
    again = autotune.tune(g, None, b, 1)
    assert again == best and fake.made == 1  # served from the cache
    other = autotune.tune(dict(g, nz=128), None, b, 1)
    assert fake.made == 2 and other["lz"] == 32


def test_key_buckets_particle_counts():
    g = inputs.random_grid(0, 16, 16, 16)
    assert autotune.key_of(g, 1000, 1) == autotune.key_of(g, 1023, 1)
    assert autotune.key_of(g, 1000, 1) != autotune.key_of(g, 5000, 1)
    assert autotune.key_of(g, 1000, 1) != autotune.key_of(g, 1000, 0)
