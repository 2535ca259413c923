"""Function symbols on the GPU (Sec. 3.1): counts, tables and model lists
against the oracle, and larger counts against closed forms and brute-force
numbers that hold without any formula text."""
import numpy as np
import pytest
import torch

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import unlabelled as U
from paper_1310_6978_b300 import workloads as W

pytestmark = pytest.mark.gpu

SMALL = [W.semigroups(2), W.semigroups(3), W.latin_squares(3), W.latin_squares(3, first_row=True),
         W.reduced_latin_squares(4), W.groups(3), W.groups_identity0(3),
         W.Workload("image", 3, "var r(S)\nfun f(S)\nA[x:S] r(f(x))\n", 3, 12)]


@pytest.mark.parametrize("wl", SMALL, ids=lambda w: f"{w.family}{w.param}")
@pytest.mark.parametrize("engine", [L.ENGINE_JIT, L.ENGINE_INTERP])
def test_counts_tables_models_match_oracle(wl, engine):
    th = oracle.Theory(wl.text, wl.k)
    p = F.compile(wl.text, wl.k)
    p.set_option(L.OPT_ENGINE, engine)
    assert p.n == th.n
    assert p.count() == th.count()
    words = torch.zeros(p.table_words(), dtype=torch.int64, device="cuda")
    p.truth_table(words)
    assert np.array_equal(words.cpu().numpy().view(np.uint64), th.table())
    models, total = th.models(1 << 16)
    buf = torch.zeros(1 << 16, dtype=torch.int64, device="cuda")
    gtotal, written = p.enumerate_models(buf)
    assert gtotal == total and written == len(models)
    assert np.array_equal(buf[:written].cpu().numpy().view(np.uint64), models)


def test_larger_counts_against_closed_forms():
    # groups of order 4 with identity 0: Z4 has 3 labellings fixing 0 (3!/|Aut Z4| = 3), V4 one
    assert F.compile(W.groups_identity0(4).text, 4).count() == 4
    # Latin squares of order 4 with the first row fixed: 576 / 4! = 24
    p = F.compile(W.latin_squares(4, first_row=True).text, 4)
    assert p.n == 48 and p.count() == 24
    # reduced Latin squares of order 5: 56
    p = F.compile(W.reduced_latin_squares(5).text, 5)
    assert p.n == 52 and p.count() == 56


def test_unlabelled_semigroups_from_gpu_models():
    p = F.compile(W.semigroups(3).text, 3)
    r = U.unlabelled_count(p, 3, cap=1 << 12)
    assert r["labelled"] == 113 and r["unlabelled"] == 24 and r["burnside_sum"] == 113
