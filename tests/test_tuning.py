"""The shape cache (paper_1310_6978_b300/tuning.py) on the CPU: keys, the
JSON round trip, and the committed shapes of the three n = 36 workloads the
benchmark times -- present, within the options' ranges, and applied to the
layout the kernels are built with."""
import json

import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import tuning
from paper_1310_6978_b300 import workloads as W

N36 = [W.TRANSITIVE6, W.TRIFREE9, W.AUT6]


def test_keys_separate_text_domain_and_mode():
    a = tuning.key("var a\na\n", 1, 0)
    assert a == tuning.key("var a\na\n", 1, 0)
    assert len({a, tuning.key("var a\na\n", 2, 0), tuning.key("var a\na\n", 1, 1), tuning.key("var b\nb\n", 1, 0)}) == 4


def test_save_and_load_round_trip(tmp_path):
    path = str(tmp_path / "shapes.json")
    assert tuning.load(path) == {}
    cache = {"x:k1:m0": {"regs_log2": 2, "unit_bits": 13}}
    tuning.save(cache, path)
    assert tuning.load(path) == cache
    with open(path, "w") as f:
        f.write("not json")
    assert tuning.load(path) == {}


def test_committed_shapes_cover_the_benchmark_and_build_their_layouts():
    cache = tuning.load()
    for wl in N36:
        shape = cache[tuning.key(wl.text, wl.k, 0)]
        assert 1 <= shape["regs_log2"] <= 3 and 0 <= shape["warps_log2"] <= 5
        assert 1 <= shape["min_blocks"] <= 32 and 1 <= shape["loop_level_bits"] <= 16
        assert 0 <= shape["unit_bits"] <= 24 and 0 <= shape.get("inner_bits", 0) <= 5
        p = F.compile(wl.text, wl.k)
        assert tuning.ensure(p, 0, cache) == shape
        lay = p.debug_dump(0)["layout"]
        assert lay["r"] == shape["regs_log2"] and lay["warp_bits"] == shape["warps_log2"]
        assert lay["unit_bits"] == shape["unit_bits"]
        assert 5 + lay["r"] + lay["lane_bits"] + lay["warp_bits"] + sum(lay["loop_bits"]) + lay["unit_bits"] == wl.n
        inner = shape.get("inner_bits", 0)
        outer = lay["loop_bits"][:-1] if inner else lay["loop_bits"]
        assert all(b <= shape["loop_level_bits"] for b in outer)
        if inner:
            assert lay["loop_bits"][-1] == inner


def test_ensure_leaves_unknown_programs_at_the_default_shape():
    p = F.compile("var a, b, c\na & (b | c)\n")
    before = json.dumps(p.debug_dump(0)["layout"], sort_keys=True)
    assert tuning.ensure(p, 0, {}, tune=False) is None
    assert json.dumps(p.debug_dump(0)["layout"], sort_keys=True) == before
