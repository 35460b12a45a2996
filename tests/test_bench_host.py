"""Host-side logic of bench.py that needs no GPU: the hash that ties the
committed ncu counters to the stencil sources, the per-site scaling of those
counters, and the algorithmic flop count of one apply."""
import json
import os
import shutil

import bench


def _copy_sources(tmp_path):
    for f in bench.KERNEL_SOURCES:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, f), dst)


def test_kernel_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    src = tmp_path / bench.KERNEL_SOURCES[0]
    text = src.read_text()
    src.write_text(text.replace("\n", "\n// a comment added\n", 1) + "\n/* block\n comment */\n")
    assert bench.kernel_hash() == h0
    src.write_text(text.replace("const int nblk", "const int nblk2", 1))
    assert bench.kernel_hash() != h0


def test_measured_traffic_scales_by_sites_and_checks_the_hash(tmp_path, monkeypatch):
    _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    cap = {"mode": "f32-full", "nrhs": 1, "launch_shape": 10368, "lattice": [16, 16, 16, 32],
           "dram_bytes_per_launch": 1000.0}
    doc = {"kernel_hash": bench.kernel_hash(), "captures": [cap]}
    (tmp_path / "profiles" / "dslash_traffic.json").write_text(json.dumps(doc))
    assert bench.measured_traffic("f32-full", 1, 10368, [32, 32, 32, 64]) == 1000.0 * 16
    assert bench.measured_traffic("f32-full", 1, 2176, [32, 32, 32, 64]) is None  # other launch shape
    assert bench.measured_traffic("f16-2row", 1, 10368, [32, 32, 32, 64]) is None  # other storage
    doc["kernel_hash"] = "0" * 16
    (tmp_path / "profiles" / "dslash_traffic.json").write_text(json.dumps(doc))
    assert bench.measured_traffic("f32-full", 1, 10368, [32, 32, 32, 64]) is None  # stale counters


def test_flop_count_of_one_apply():
    """The method's count (one mat-vec per hop and spin, accumulation into the
    class accumulators, class scaling, gamma combine, diagonal) from the offsets
    of the 3^4 hypercube, and the implementation's pair-form count."""
    import itertools

    classes = [sum(1 for c in d if c) for d in itertools.product((-1, 0, 1), repeat=4) if any(d)]
    assert sorted(set(classes)) == [1, 2, 3, 4] and len(classes) == 80
    matvec = 80 * 4 * (9 * 6 + 6 * 2)                         # 3x3 complex mat-vec per spin
    accumulate = sum(24 * (1 + n) for n in classes)           # lambda + n gamma accumulators
    scale, combine, gamma, diag = 4 * 5 * 24, 5 * 3 * 24, 4 * 24, 2 * 24
    assert matvec + accumulate + scale + combine + gamma + diag == bench.FLOPS_PER_SITE == 29208
    assert bench.method_flops("f32-2row") == 29208 + 80 * 42
    # implementation: class sizes 8/24/32/16 hops = 4/12/16/8 (d, -d) pairs
    pairs = {1: 4, 2: 12, 3: 16, 4: 8}
    colour = 80 * 4 * 9 * 8                                  # complex MACs, 8 flops each
    spin = sum(k * 2 * (2 * 24 + 24 + 24 * n) for n, k in pairs.items())  # sum/difference, lambda, gamma
    assert colour + spin + 2 * 24 == bench.IMPL_FLOPS_PER_SITE == 34032
