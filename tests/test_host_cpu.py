"""Host-side logic that needs no GPU: the autotuner's candidate tilings, the
benchmark's traffic record lookup and option parsing, and the workload
generators' structure."""
import hashlib
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tuner_candidates_respect_pipeline_constraints():
    pytest.importorskip("torch")
    from paper_2509_15744_gb300 import tune
    c3 = tune.candidates(3, 512)
    assert {c[3] for c in c3} == {3}                     # one field per launch: register queue
    cb = tune.candidates(3, 512, batched=True)
    assert {c[3] for c in cb} == {3, 4, 5}
    assert all(c[1] == 16 for c in cb if c[3] in (4, 5))   # 16 rows per CTA
    assert all(c[0] == 8 for c in cb if c[3] == 5)         # TMA-streamed kernel: z-block of 8
    assert all(c[2] in (2, 3) and c[0] in (8, 16, 32, 64, 128) for c in cb)
    # z-blocks that keep the accumulator in tensor memory (32; 16 with Kahan)
    assert {(16, 16, 2, 4), (32, 16, 2, 4)} <= set(cb)
    c2 = tune.candidates(2, 300)
    assert all(c[3] == 0 and c[1] == 8 for c in c2)
    # small grids do not get z-blocks deeper than the grid
    assert all(c[0] <= 32 for c in tune.candidates(3, 12))


def test_tuner_cache_key_separates_kahan():
    pytest.importorskip("torch")
    from paper_2509_15744_gb300 import tune

    class M:
        shape, order, physics, storage = (64, 64, 64), 8, "velocity", "f32"

    a, b = M(), M()
    a.kahan, b.kahan = False, True
    assert tune._key(a, 16) != tune._key(b, 16)


def test_traffic_record_is_used_only_for_the_current_kernel_source(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    csrc = tmp_path / "paper_2509_15744_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_bytes(b"kernel v1")
    prof = tmp_path / "profiles"
    prof.mkdir()
    digest = hashlib.sha256(b"kernel v1").hexdigest()[:16]
    (prof / "k_w_traffic.txt").write_text(
        "# comment: with a colon\n"
        f"kernel_source_sha256_16: {digest}\nworkload: w\ndram_bytes_per_launch_full_size: 12345\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("k.cu", "w") == 12345.0
    assert bench.kernel_traffic("k.cu", "other workload") is None
    (prof / "k_w2_traffic.txt").write_text(
        f"kernel_source_sha256_16: {digest}\nworkload: w2\ntiling: 32,16,2,4\n"
        "dram_bytes_per_launch_full_size: 777\n")
    assert bench.kernel_traffic("k.cu", "w2", (32, 16, 2, 4)) == 777.0
    assert bench.kernel_traffic("k.cu", "w2", [64, 16, 2, 4]) is None   # taken with another tiling
    (csrc / "k.cu").write_bytes(b"kernel v2")           # the kernel changed since the capture
    assert bench.kernel_traffic("k.cu", "w") is None


def test_bench_options():
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    try:
        sys.argv = ["bench.py", "--tiling", "64:16:2:4", "--grad-mode", "reverse", "--forward-curve"]
        a = bench.parse()
        assert a.tiling == "64:16:2:4" and a.grad_mode == "reverse" and a.forward_curve
        sys.argv = ["bench.py"]
        a = bench.parse()
        assert a.gpus == 1 and a.warmup >= 3 and a.workload == "w2" and a.impl == "ours"
        assert a.cta_order is None   # the tuner's pick
        sys.argv = ["bench.py", "--cta-order", "0"]
        assert bench.parse().cta_order == 0
        sys.argv = ["bench.py", "--cta-order", "2"]
        with pytest.raises(SystemExit):
            bench.parse()
    finally:
        sys.argv = old


def test_smooth_field_is_a_sum_of_separable_modes():
    from paper_2509_15744_gb300 import workloads as WL
    f = WL.smooth_field_3d(np.random.default_rng(4), (20, 24, 28), 50.0, lo=1500.0, hi=4500.0, nmodes=6)
    assert f.dtype == np.float32 and f.flags["C_CONTIGUOUS"] and f.shape == (20, 24, 28)
    assert f.min() == pytest.approx(1500.0) and f.max() == pytest.approx(4500.0, rel=1e-6)
    # the same modes evaluated cell by cell (before the affine map to [lo, hi])
    rng = np.random.default_rng(4)
    z, y, x = (np.arange(n, dtype=np.float64) for n in (20, 24, 28))
    ref = np.zeros((20, 24, 28))
    for _ in range(6):
        kz, ky, kx = rng.normal(0.0, 1.0 / 50.0, 3)
        ph = rng.uniform(0, 2 * np.pi, 3)
        amp = rng.normal()
        ref += amp * np.cos(kz * z + ph[0])[:, None, None] * np.cos(ky * y + ph[1])[None, :, None] \
            * np.cos(kx * x + ph[2])[None, None, :]
    ref = 1500.0 + (ref - ref.min()) * 3000.0 / (ref.max() - ref.min())
    np.testing.assert_allclose(f, ref, rtol=2e-5)
    w4 = WL.workload4(n=32, nt=10)
    assert w4.nshots == 4 and len(set(w4.sources)) == 4 and w4.receivers[0].size == 32 * 32


class _FakeModel:
    """Stands in for wave.Model in the tuner: records the tiling and launch
    order it is given and the gradient calls made with them."""

    def __init__(self, shape, kahan=False):
        import torch
        self.shape, self.order, self.physics, self.storage, self.kahan = shape, 8, "velocity", "f32", kahan
        self.param = torch.zeros(1)
        self.tiling, self.cta_order, self.calls = None, 1, []

    def set_tiling(self, *t):
        self.tiling = tuple(t)

    def set_schedule(self, order):
        self.cta_order = int(order)

    def gradient(self, shots, **kw):
        self.calls.append((self.tiling, self.cta_order))


def _fake_tuner(monkeypatch, tmp_path, times):
    """The tuner with its timing read from `times[(tiling, order)]` (ms per launch)."""
    import torch
    from paper_2509_15744_gb300 import tune
    state = {}
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tune_cache.json"))
    monkeypatch.setattr(tune.torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(tune.W, "timing_enable", lambda on: None)
    monkeypatch.setattr(tune.W, "timing_read",
                        lambda: (times.get((state["m"].tiling, state["m"].cta_order), 100.0), 1, 0.0))
    shot = tune.W.Shot(0, torch.zeros(31), torch.zeros(4, dtype=torch.int64), None)
    return tune, state, [shot, shot]


def test_tuner_keeps_the_faster_launch_order_of_its_best_tiling(monkeypatch, tmp_path):
    pytest.importorskip("torch")
    best = (32, 16, 2, 4)
    times = {(best, 1): 7.70, (best, 0): 7.60, ((16, 16, 2, 4), 1): 8.0}
    tune, state, shots = _fake_tuner(monkeypatch, tmp_path, times)
    m = state["m"] = _FakeModel((64, 64, 64))
    assert tune.tune(m, shots, batched=True) == best
    assert m.tiling == best and m.cta_order == 0
    # every candidate was timed in the default (plane-major) order, the best one also in the other
    assert {o for t, o in m.calls if t != best} == {1}
    assert (best, 0) in m.calls
    # the cache holds the order; a second call applies it without timing anything
    import json
    assert json.load(open(tune.CACHE))[tune._key(m, 2)] == list(best) + [0]
    m2 = state["m"] = _FakeModel((64, 64, 64))
    assert tune.tune(m2, shots, batched=True) == best
    assert m2.calls == [] and m2.cta_order == 0 and m2.tiling == best


def test_tuner_stays_plane_major_when_it_is_faster(monkeypatch, tmp_path):
    pytest.importorskip("torch")
    best = (16, 16, 2, 4)
    times = {(best, 1): 6.0, (best, 0): 6.5}
    tune, state, shots = _fake_tuner(monkeypatch, tmp_path, times)
    m = state["m"] = _FakeModel((64, 64, 64), kahan=True)
    assert tune.tune(m, shots, batched=True) == best
    assert m.cta_order == 1


def test_tuner_reads_cache_entries_without_an_order(monkeypatch, tmp_path):
    pytest.importorskip("torch")
    import json
    tune, state, shots = _fake_tuner(monkeypatch, tmp_path, {})
    m = state["m"] = _FakeModel((64, 64, 64))
    m.cta_order = 0
    json.dump({tune._key(m, 2): [64, 16, 2, 4]}, open(tune.CACHE, "w"))
    assert tune.tune(m, shots, batched=True) == (64, 16, 2, 4)
    assert m.cta_order == 1 and m.calls == []


def test_tuner_tries_no_launch_order_in_2d(monkeypatch, tmp_path):
    pytest.importorskip("torch")
    tune, state, shots = _fake_tuner(monkeypatch, tmp_path, {((16, 8, 3, 0), 1): 1.0})
    m = state["m"] = _FakeModel((64, 64))
    assert tune.tune(m, shots) == (16, 8, 3, 0)
    assert all(o == 1 for _, o in m.calls)
