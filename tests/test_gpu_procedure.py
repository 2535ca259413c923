"""GPU: killing variables and the counting procedure of Sec. 3.4 evaluated as
one batch of reduced theories (exact integers)."""
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import procedure as P
from paper_1310_6978_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_killed_families_on_gpu(k):
    for wl, want in [(W.posets_reflexivity_killed(k), [0, 1, 3, 19, 219, 4231, 130023][k]),
                     (W.bounded_posets_killed(k), None)]:
        p = F.compile(wl.text, wl.k)
        c = p.count()
        if want is not None:
            assert c == want
        else:
            th = oracle.Theory(wl.text, wl.k)
            assert c == (th.count() if th.n <= 22 else th.count_par(0, 1 << th.n))


@pytest.mark.parametrize("n", [5, 7, 8])
def test_layer_procedure_on_gpu_batch(n):
    l_proc, detail = P.count_bounded_posets_by_layers(n, P.gpu_batch_counter)
    K = F.compile(W.bounded_posets_killed(n).text, n).count()
    assert l_proc == n * (n - 1) * K
    assert len(detail) == 2 ** (n - 3)


@pytest.mark.parametrize("k", [5, 6])
def test_special_element_posets_on_gpu(k):
    """SO.txt (Sec. 4.2): partial orders with a special element, k^2 - k free
    letters, counted directly on the GPU and by the counting procedure of
    Sec. 3.4 (minimal / non-minimal partition, the reduced theories in one
    batch); both equal the backtracking counter.  The procedure also
    reproduces the number of partial orders (reflexivity killed)."""
    from oracle import counters as C
    w = W.posets_special(k)
    want = C.count_posets_special_c(k)
    assert F.compile(w.text, w.k).count() == want
    l, detail = P.count_by_partition(w.text, k, 2, lambda c, x: P.minimal_theta(c, x, "p"), P.MINIMAL_S,
                                     P.gpu_batch_counter, rel="p")
    assert l == want and len(detail) == k + 1
    q = W.posets_reflexivity_killed(k)
    l2, _ = P.count_by_partition(q.text, k, 2, lambda c, x: P.minimal_theta(c, x, "r"), P.MINIMAL_S,
                                 P.gpu_batch_counter, rel="r")
    assert l2 == C.count_posets_c(k) == [4231, 130023][k - 5]
