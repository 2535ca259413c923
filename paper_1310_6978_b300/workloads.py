"""Seeded synthetic workloads: formula TEXT only.

This module is the one input source shared by the CUDA path and the CPU
oracle.  It writes theories in the library's formula language and holds none
of the method's arithmetic (no evaluation, no grounding, no counting).  The
families are the ones used as worked examples of the method: partial orders
(Sec. 4.2 and Sec. 5.2), equivalence and transitive relations, graphs as
symmetric irreflexive relations, triangle-free graphs, automorphisms of a
structure as permutation matrices (Sec. 1 and Sec. 5.3 mention automorphism
counting), the Boolean system BAequ4 (Sec. 5.1) and random 3-CNF.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so every workload is
reproducible from its seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

MASK64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, m: int) -> int:
        """Uniform integer in [0, m) by the multiply-high map of the top 32 bits."""
        return ((self.next() >> 32) * m) >> 32

    def uniform01(self) -> float:
        return ((self.next() >> 11) + 0.5) / float(1 << 53)


@dataclass(frozen=True)
class Workload:
    family: str
    param: int          # k for structures, n for 3-CNF
    text: str
    k: int              # domain size passed to compile
    n: int              # number of propositional variables

    def __repr__(self):
        return f"Workload({self.family}, {self.param}, n={self.n})"


# -- relation families over a k-element domain (letters r(i,j), n = k^2) --

REFLEXIVE = "A[i:S] r(i,i)"
ANTISYMMETRIC = "A[i,j:S2] ~(r(i,j) & r(j,i))"
SYMMETRIC = "A[i,j:S2] (r(i,j) -> r(j,i))"
TRANSITIVE = "A[i,j,l:S] (r(i,j) & r(j,l) -> r(i,l))"


def posets(k: int) -> Workload:
    text = "\n".join(["var r(S,S)", REFLEXIVE, ANTISYMMETRIC, TRANSITIVE]) + "\n"
    return Workload("poset", k, text, k, k * k)


def equivalences(k: int) -> Workload:
    text = "\n".join(["var r(S,S)", REFLEXIVE, SYMMETRIC, TRANSITIVE]) + "\n"
    return Workload("equiv", k, text, k, k * k)


def transitive(k: int) -> Workload:
    text = "\n".join(["var r(S,S)", TRANSITIVE]) + "\n"
    return Workload("transitive", k, text, k, k * k)


def graphs(k: int) -> Workload:
    """Labelled simple graphs as irreflexive symmetric relations (n = k^2)."""
    text = "\n".join(["var r(S,S)", "A[i:S] ~r(i,i)", "A[i,j:S2] (r(i,j) <-> r(j,i))"]) + "\n"
    return Workload("graph", k, text, k, k * k)


def triangle_free(k: int) -> Workload:
    """Labelled triangle-free graphs on k vertices: one letter per pair a<b."""
    text = "var e(S<S)\nA[a,b,c:S | a<b, b<c] ~(e(a,b) & e(b,c) & e(a,c))\n"
    return Workload("trifree", k, text, k, k * (k - 1) // 2)


def random_graph_bits(k: int, seed: int) -> str:
    """G(k, 1/2): edge {a<b}, pairs in lexicographic order, present iff the
    top bit of the next draw is 1.  Returned as the k*k adjacency bits (row
    major, symmetric, zero diagonal)."""
    rng = SplitMix64(seed)
    adj = [[0] * k for _ in range(k)]
    for a in range(k):
        for b in range(a + 1, k):
            if rng.next() >> 63:
                adj[a][b] = adj[b][a] = 1
    return "".join(str(adj[i][j]) for i in range(k) for j in range(k))


def automorphisms(k: int, seed: int) -> Workload:
    """Automorphisms of G(k,1/2) as k x k permutation matrices p(i,a)
    ('i is mapped to a'): exactly one true per row and per column, and
    edges preserved: p(i,a) & p(j,b) -> (E(i,j) <-> E(a,b))."""
    bits = random_graph_bits(k, seed)
    text = "\n".join([
        "var p(S,S)",
        f"const E(S,S) = {bits}",
        "A[i:S] E[a:S] p(i,a)",
        "A[i:S] A[a,b:S | a<b] ~(p(i,a) & p(i,b))",
        "A[a:S] E[i:S] p(i,a)",
        "A[a:S] A[i,j:S | i<j] ~(p(i,a) & p(j,a))",
        "A[i,j:S2] A[a,b:S2] (p(i,a) & p(j,b) -> (E(i,j) <-> E(a,b)))",
    ]) + "\n"
    return Workload("aut", k, text, k, k * k)


def cnf3(n: int, seed: int, ratio: float = 4.25) -> Workload:
    """Random 3-CNF: m = floor(ratio*n + 1/2) clauses; each clause picks 3
    distinct variables (rejection) and negates each with probability 1/2."""
    rng = SplitMix64(seed)
    m = int(math.floor(ratio * n + 0.5))
    lines = ["var x(S)"]
    for _ in range(m):
        vs = []
        while len(vs) < 3:
            v = rng.below(n)
            if v not in vs:
                vs.append(v)
        lits = []
        for v in vs:
            neg = rng.next() >> 63
            lits.append(("~" if neg else "") + f"x({v})")
        lines.append(" | ".join(lits))
    return Workload("cnf3", n, "\n".join(lines) + "\n", n, n)


# The Boolean system of Sec. 5.1 (BAequ4): x + y + ~z + u = 1 and x v yz = u,
# the second written as ~((x | y & z) ^ u).
BAEQU4 = Workload("baequ4", 4, "var x, y, z, u\ne1 = x ^ y ^ ~z ^ u\ne2 = ~((x | y & z) ^ u)\n", 1, 4)


def minterm(n: int, alpha: int) -> Workload:
    """x_0^{a_0} & ... & x_{n-1}^{a_{n-1}} over propositional letters."""
    names = [f"v{i}" for i in range(n)]
    lits = [(names[i] if (alpha >> i) & 1 else "~" + names[i]) for i in range(n)]
    return Workload("minterm", n, "var " + ", ".join(names) + "\n" + " & ".join(lits) + "\n", 1, n)


def single_var(n: int, i: int) -> Workload:
    """The formula x_i over n declared letters: its table is generator x_i."""
    names = [f"v{t}" for t in range(n)]
    return Workload("var", n, "var " + ", ".join(names) + "\n" + names[i] + "\n", 1, n)


# -- named configurations ---------------------------------------------------

POSET3 = posets(3)                         # n = 9, 512 assignments, 19 models
CNF32 = cnf3(32, seed=1)                   # n = 32, m = 136
TRANSITIVE6 = transitive(6)                # n = 36
TRIFREE9 = triangle_free(9)                # n = 36
AUT6 = automorphisms(6, seed=3)            # n = 36


def batch_mix(count: int = 4096, seed: int = 2) -> "list[Workload]":
    """Mixed batch: family uniform over {equivalences k=2..6, posets k=2..5,
    triangle-free k=3..8, 3-CNF n=16..30}; parameter uniform in its range."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        fam = rng.below(4)
        if fam == 0:
            out.append(equivalences(2 + rng.below(5)))
        elif fam == 1:
            out.append(posets(2 + rng.below(4)))
        elif fam == 2:
            out.append(triangle_free(3 + rng.below(6)))
        else:
            n = 16 + rng.below(15)
            out.append(cnf3(n, seed=rng.next()))
    return out


@dataclass(frozen=True)
class Request:
    rid: int
    arrival_s: float
    workload: Workload
    mode: str            # "count" or "enumerate"
    cap: int


def _family_for_n(rng: SplitMix64, n: int) -> Workload:
    opts = []
    for k in (4, 5, 6):
        if k * k == n:
            opts += [equivalences(k), posets(k), transitive(k)]
    for k in (7, 8, 9):
        if k * (k - 1) // 2 == n:
            opts.append(triangle_free(k))
    if n == 36:
        opts.append(automorphisms(6, seed=rng.next()))
    if not opts:
        return cnf3(n, seed=rng.next())
    return opts[rng.below(len(opts))]


def request_stream(count: int, rate_per_s: float, seed: int = 5,
                   n_lo: int = 16, n_hi: int = 38, enum_frac: float = 0.10,
                   cap: int = 1_000_000) -> "list[Request]":
    """Poisson arrivals (exponential gaps at ``rate_per_s``); n uniform in
    [n_lo, n_hi]; a family among those with exactly n letters, else 3-CNF;
    ``enum_frac`` of the requests enumerate models (capped), the rest count."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += -math.log(rng.uniform01()) / rate_per_s
        n = n_lo + rng.below(n_hi - n_lo + 1)
        wl = _family_for_n(rng, n)
        mode = "enumerate" if rng.uniform01() < enum_frac else "count"
        out.append(Request(rid, t, wl, mode, cap))
    return out


# -- killing variables (Sec. 3.3) and the bounded posets of Sec. 5.2 ---------

POSET_AXIOMS = [REFLEXIVE, ANTISYMMETRIC, TRANSITIVE]


def posets_reflexivity_killed(k: int) -> Workload:
    """Partial orders with the letters r(i,i) killed to 1 (the assumptions of
    the SO.txt example, Sec. 4.2): k^2 - k free letters."""
    text = "\n".join(["var r(S,S)", "assume A[i:S] r(i,i)", ANTISYMMETRIC, TRANSITIVE]) + "\n"
    return Workload("poset_killed", k, text, k, k * k - k)


def posets_special(k: int) -> Workload:
    """Partial orders with a special element, the SO.txt script of Sec. 4.2:
    p(i,j) reads i <= j; reflexivity is assumed (the letters p(i,i) killed to
    1, k^2 - k free letters); antisymmetry and transitivity over distinct
    pairs and triples; some element is comparable with every element."""
    text = "\n".join(["var p(S,S)", "assume A[i:S] p(i,i)",
                      "A[i,j:S2] (~p(i,j) | ~p(j,i))",
                      "A[i,j,l:S3] (~(p(i,j) & p(j,l)) | p(i,l))",
                      "E[i:S].A[j:S] (p(i,j) | p(j,i))"]) + "\n"
    return Workload("poset_special", k, text, k, k * k - k)


def bounded_posets(k: int) -> Workload:
    """Partial orders with a least and a greatest element (Sec. 5.2), k >= 2."""
    text = "\n".join(["var r(S,S)", *POSET_AXIOMS, "E[x:S].A[y:S] r(x,y)", "E[x:S].A[y:S] r(y,x)"]) + "\n"
    return Workload("bounded_poset", k, text, k, k * k)


def bounded_posets_killed(k: int) -> Workload:
    """The adequate family K of Sec. 5.2: 0 is the least and k-1 the greatest
    element; eq. (conspa) kills 5k-6 letters (read with the greatest element
    k-1: r(0,i)=1, r(j,0)=0 for j>=1, r(i,k-1)=1, r(k-1,l)=0 for l<=k-2,
    r(i,i)=1), leaving (k-2)(k-3) free letters."""
    kill = [f"assume A[i:S] r(0,i)", f"assume A[j:S | j>0] ~r(j,0)", f"assume A[i:S] r(i,{k - 1})",
            f"assume A[l:S | l<{k - 1}] ~r({k - 1},l)", "assume A[i:S] r(i,i)"]
    text = "\n".join(["var r(S,S)", *kill, ANTISYMMETRIC, TRANSITIVE]) + "\n"
    return Workload("bounded_poset_killed", k, text, k, (k - 2) * (k - 3))


# -- function symbols (Sec. 3.1: letters p_{F a_1..a_k b}) --------------------

ASSOCIATIVE = "A[x,y,z:S] m(m(x,y),z) = m(x,m(y,z))"
LEFT_CANCEL = "A[x,y,z:S] (m(x,y) = m(x,z) -> y = z)"
RIGHT_CANCEL = "A[x,y,z:S] (m(y,x) = m(z,x) -> y = z)"


def semigroups(k: int) -> Workload:
    """Associative binary operations on k elements (letters m(a,b,u), k^3)."""
    text = "\n".join(["fun m(S,S)", ASSOCIATIVE]) + "\n"
    return Workload("semigroup", k, text, k, k ** 3)


def latin_squares(k: int, first_row: bool = False) -> Workload:
    """Quasigroups = Latin squares of order k (both cancellation laws); with
    ``first_row`` the row m(0,j) = j is assumed, which kills k^2 letters."""
    lines = ["fun m(S,S)"]
    if first_row:
        lines.append("assume A[j:S] m(0,j) = j")
    lines += [LEFT_CANCEL, RIGHT_CANCEL]
    return Workload("latin_row" if first_row else "latin", k, "\n".join(lines) + "\n", k,
                    k ** 3 - (k * k if first_row else 0))


def reduced_latin_squares(k: int) -> Workload:
    """Latin squares with first row and column 0..k-1; letters that the
    border rules out (m(i,j) = i or = j inside) are killed as well."""
    lines = ["fun m(S,S)", "assume A[j:S] m(0,j) = j", "assume A[i:S] m(i,0) = i",
             "assume A[i,j:S | i>0, j>0] (~(m(i,j) = i) & ~(m(i,j) = j))",
             LEFT_CANCEL, RIGHT_CANCEL]
    m = k - 1
    free = m * (m - 1) * (k - 2) + m * (k - 1)
    return Workload("latin_reduced", k, "\n".join(lines) + "\n", k, free)


def groups_identity0(k: int) -> Workload:
    """Groups on k elements with identity 0 (identity row and column killed):
    associativity and a right inverse for every element."""
    lines = ["fun m(S,S)", "assume A[x:S] (m(0,x) = x & m(x,0) = x)", ASSOCIATIVE,
             "A[x:S] E[y:S] m(x,y) = 0"]
    return Workload("group_e0", k, "\n".join(lines) + "\n", k, (k - 1) ** 2 * k)


def groups(k: int) -> Workload:
    """Groups on k elements: associativity, an identity and inverses."""
    lines = ["fun m(S,S)", ASSOCIATIVE,
             "E[e:S] (A[x:S] (m(e,x) = x & m(x,e) = x) & A[x:S] E[y:S] m(x,y) = e)"]
    return Workload("group", k, "\n".join(lines) + "\n", k, k ** 3)
