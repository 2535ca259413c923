"""The C ABI boundary without a GPU: libfbg.so loads, exports every function
include/fbg.h declares, compiles on the host, and refuses to evaluate without
a device (no CPU path).  The product does not load the oracle."""
import os
import re
import subprocess
import sys

import pytest

import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fbg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(fbg_[a-z_0-9]+)\s*\(", text, flags=re.M)))


def test_every_declared_function_is_exported():
    names = declared_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(L.lib, n)]
    assert missing == []


def test_library_is_built_for_sm_103a_and_links_no_oracle():
    out = subprocess.run(["ldd", L.LIB_PATH], capture_output=True, text=True).stdout
    assert "oracle" not in out
    assert "libcuda.so" not in out          # the driver is loaded at run time by the CUDA runtime


def test_package_does_not_import_the_oracle():
    code = ("import sys; sys.path.insert(0, %r); import paper_1310_6978_b300 as F; "
            "from paper_1310_6978_b300 import _lib, workloads, tuning; "
            "F.compile('var a\\na\\n'); print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert r.stdout.strip() == "False", r.stderr


def test_host_only_calls_work_without_a_gpu():
    p = F.compile("var r(S,S)\nA[i:S] r(i,i)\n", 3)
    assert p.n == 9 and p.var_name(4) == "r(1,1)"
    s = p.stats()
    assert s.n == 9 and s.luts >= 0
    assert "fbg_jit_count" in p.source(0) and "fbg_jit_table" in p.source(1)
    d = p.debug_dump(2)
    assert d["layout"]["n"] == 9


@pytest.mark.parametrize("engine", [L.ENGINE_AUTO, L.ENGINE_JIT, L.ENGINE_INTERP])
def test_evaluation_fails_loudly_without_a_device(engine):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    p = F.compile("var a, b\na & b\n").set_option(L.OPT_ENGINE, engine)
    with pytest.raises(L.FbgError) as ei:
        p.count(stream=0)
    assert ei.value.status in (L.FBG_ECUDA, L.FBG_EJIT)


def test_option_validation():
    p = F.compile("var a\na\n")
    for opt, bad in [(L.OPT_ENGINE, 7), (L.OPT_REGS_LOG2, 0), (L.OPT_REGS_LOG2, 4), (L.OPT_WARPS_LOG2, 6),
                     (L.OPT_LOOP_LEVEL_BITS, -1), (L.OPT_LOOP_LEVEL_BITS, 17), (999, 1)]:
        with pytest.raises(L.FbgError) as ei:
            p.set_option(opt, bad)
        assert ei.value.status == L.FBG_EINVAL
    # item pieces are a scheduling choice: accepted as on/off, no rebuild
    for v in (1, 0, 5):
        p.set_option(L.OPT_SPLIT_ITEMS, v)


@pytest.mark.parametrize("opts", [
    {}, {L.OPT_UNIT_BITS: 2}, {L.OPT_UNIT_BITS: 0, L.OPT_LOOP_LEVEL_BITS: 3},
    {L.OPT_UNIT_BITS: 2, L.OPT_LOOP_LEVEL_BITS: 5}, {L.OPT_UNIT_BITS: 2, L.OPT_LOOP_LEVEL_BITS: 16},
    {L.OPT_UNIT_BITS: 6}, {L.OPT_UNIT_BITS: 4, L.OPT_LOOP_LEVEL_BITS: 2, L.OPT_INNER_BITS: 1}])
def test_piece_bits_follow_the_loop_levels(opts):
    """An item can be split over the first loop level only when that level
    is a runtime loop: there is one, and it is not the unrolled innermost
    level (at most 5 bits, emitted as straight-line copies); pieces go up to
    16 (4 bits)."""
    from paper_1310_6978_b300 import workloads as W
    p = F.compile(W.posets(5).text, 5)
    for k, v in opts.items():
        p.set_option(k, v)
    lay = p.debug_dump(0)["layout"]
    lb = lay["loop_bits"]
    runtime_first = len(lb) >= 2 or (len(lb) == 1 and lb[0] > 5)
    assert lay["split_bits"] == (min(lb[0], 4) if runtime_first else 0), lay
    src = p.source(0)
    assert ("for (fbg_u32 i2 = lo2; i2 < hi2; ++i2)" in src) == runtime_first


def test_batch_specialised_kernels_compile_without_a_device():
    from paper_1310_6978_b300 import workloads as W
    mix = [W.transitive(5), W.equivalences(5), W.cnf3(22, 4), W.cnf3(21, 5)] * 2 + [W.cnf3(12, 1), W.POSET3]
    progs = [F.compile(w.text, w.k) for w in mix]
    ok, spec, log = F.batch_build_check(progs)
    assert ok, log
    assert spec == 4          # one kernel per distinct program with n >= 20
    src = F.batch_source(progs)
    assert src.count("fbg_jit_count(FbgLaunch P)") == 4 and "fbg_finish_count" in src
