"""Writes tests/golden/cnf32_seed<S>.txt: the full truth table of the seeded
3-CNF formula with n = 32 letters and m = 136 clauses (seed S), computed by
the oracle alone -- bit j of the table is the formula evaluated at the
valuation mu_j (Prop. 2.2, Sec. 2.3), j in [0, 2^32) -- stored as its model
count and the SHA-256 of the table's 2^26 little-endian u64 words.

Run: python tests/golden/make_cnf32.py S [RATIO]   (about 7 minutes on 8 cores)
Seed 1 (the benchmark's formula) is unsatisfiable, so its table is all zero;
seed 2 is satisfiable and gives a table with ones to compare.  With a clause
ratio other than 4.25 (m = floor(RATIO * 32 + 1/2) clauses) the file is
cnf32_r<RATIO>_seed<S>.txt: ratio 2 (m = 64, seed 3) is the dense table,
with millions of models and level conjunctions that prune far less.
The 2^32 assignments are split into equal aligned ranges; each thread has
the oracle fill its own slice of the table (oracle_range, single-threaded C,
one call per range)."""
import concurrent.futures as cf
import ctypes
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1310_6978_b300 import workloads as W  # noqa: E402  (seeded inputs only)

def golden_name(seed: int, ratio: float = 4.25) -> str:
    return f"cnf32_seed{seed}.txt" if ratio == 4.25 else f"cnf32_r{ratio:g}_seed{seed}.txt"


def main(seed: int, ratio: float = 4.25):
    out_path = os.path.join(os.path.dirname(os.path.abspath(__file__)), golden_name(seed, ratio))
    wl = W.cnf3(32, seed, ratio)
    m = len(wl.text.splitlines()) - 1
    th = oracle.Theory(wl.text, wl.k)
    assert th.n == 32
    words = np.zeros(1 << 26, dtype=np.uint64)
    lib = oracle._load()
    chunks = 256
    span = (1 << 32) // chunks

    def run(c):
        lo = c * span
        out = ctypes.c_uint64()
        sl = words[lo >> 6:(lo + span) >> 6]
        lib.oracle_range(th._h, lo, lo + span, ctypes.byref(out), sl.ctypes.data_as(ctypes.c_void_p), None, 0, None)
        return out.value

    with cf.ThreadPoolExecutor(max_workers=oracle.max_threads()) as ex:
        count = sum(ex.map(run, range(chunks)))
    assert count == int(np.bitwise_count(words).sum())
    digest = hashlib.sha256(words.astype("<u8").tobytes()).hexdigest()
    with open(out_path, "w") as f:
        f.write(f"# 3-CNF n=32 m={m} seed {seed} (workloads.cnf3(32, {seed}, {ratio:g})): full truth table by the oracle,\n")
        f.write("# bit j = formula at mu_j (Prop. 2.2), written by tests/golden/make_cnf32.py\n")
        f.write(f"count {count}\n")
        f.write(f"sha256 {digest}\n")
    print(count, digest)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1, float(sys.argv[2]) if len(sys.argv) > 2 else 4.25)
