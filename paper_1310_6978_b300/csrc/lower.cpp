// lower.cpp -- variable grouping, level-aware lowering and LOP3 mapping.
//
// Sec. 2.3 splits each generator b_i into blocks of 2^k bits and evaluates
// d_j = t(b_1j..b_nj) on a 2^k-bit processor; 2^r processors act as one
// 2^(k+r)-bit processor.  Here the assignment integer j is split into the
// groups of Layout: the low 5 (+r) bits are bit positions inside a thread's
// 32-bit registers (their generator words are the constants 0xAAAAAAAA,
// 0xCCCCCCCC, ...), then lane/warp bits, loop levels and block-uniform unit
// bits.  A subterm is computed at the outermost level where all of its
// variables are fixed (hoisting); n-ary conjunctions and disjunctions are
// reassociated so that the part over outer variables is hoisted, and the
// top-level conjunction is split per level so that a level whose partial
// conjunction is zero for a whole warp can skip its inner levels.
// Mapping covers the 2-input gate DAG with 3-input LUTs (one lop3.b32 per
// 32-bit register), minimising LUT count by dynamic programming over
// 3-feasible cuts of fanout-free cones.
#include <algorithm>
#include <cstring>
#include <map>
#include <unordered_map>

#include "fbg_internal.hpp"

namespace fbg {

static const uint32_t kInReg[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};

int Layout::loop_pos(int i) const {
  int p = 5 + r + lane_bits + warp_bits;
  for (int j = (int)loop_bits.size() - 1; j > i; j--) p += loop_bits[(size_t)j];
  return p;
}

int Layout::level_of_pos(int p) const {
  if (n <= 5 || p < 5 + r) return LV_CONST;
  if (p < 5 + r + lane_bits + warp_bits) return LV_THREAD;
  if (p >= n - unit_bits) return LV_UNIT;
  for (int i = 0; i < (int)loop_bits.size(); i++) {
    int b = loop_pos(i);
    if (p >= b && p < b + loop_bits[(size_t)i]) return 2 + i;
  }
  return LV_UNIT;
}

Layout make_layout(int n, const LayoutParams& prm, const std::vector<int>& order) {
  Layout L;
  L.n = n;
  if (n > 5) {
    L.r = std::min(prm.r_max, n - 5);
    int rem = n - 5 - L.r;
    L.lane_bits = std::min(5, rem);
    rem -= L.lane_bits;
    L.warp_bits = std::min(prm.warps_log2, rem);
    rem -= L.warp_bits;
    int loops = std::min(rem, prm.loop_bits_max);
    // units take what the loop budget leaves, and at least unit_bits_max when possible
    int units = std::min(rem, prm.unit_bits_max);
    loops = std::min(loops, rem - units);
    if (rem - units - loops > 0) units = rem - loops;   // everything else becomes units
    L.unit_bits = units;
    int lb = std::max(1, prm.loop_level_bits);
    // the innermost level may have its own width; the others split the rest
    // from the top, with no more levels than the engine holds
    int inner = prm.inner_bits > 0 ? std::min(prm.inner_bits, loops) : 0;
    loops -= inner;
    const int room = std::max(1, prm.max_loop_levels - (inner > 0 ? 1 : 0));
    lb = std::max(lb, (loops + room - 1) / room);
    while (loops > 0) {
      int b = std::min(lb, loops);
      L.loop_bits.push_back(b);
      loops -= b;
    }
    if (inner > 0) L.loop_bits.push_back(inner);
  }
  L.pos_of_var.assign((size_t)n, 0);
  L.var_of_pos.assign((size_t)n, 0);
  for (int t = 0; t < n; t++) {
    int v = order[(size_t)t];
    L.pos_of_var[(size_t)v] = n - 1 - t;
    L.var_of_pos[(size_t)(n - 1 - t)] = v;
  }
  return L;
}

std::vector<int> identity_order(int n) {
  std::vector<int> o((size_t)n);
  for (int t = 0; t < n; t++) o[(size_t)t] = n - 1 - t;
  return o;
}

// Enumerate-mode order: the layout of make_layout(n, prm, .) with the
// letters placed so that the work item (unit u, warp slice w) holds the
// assignment integers with top bits u, w (a contiguous, ascending interval)
// and its loop nest runs through them in ascending order: unit positions
// take the top letters, warp positions the letters just below them, the
// loop positions the next ones, and lanes, registers and in-word bits keep
// their own letters.
std::vector<int> enum_order(int n, const LayoutParams& prm) {
  const Layout S = make_layout(n, prm, identity_order(n));
  const int wb = S.warp_bits, ub = S.unit_bits;
  const int w0 = S.first_warp_pos();           // first warp position
  const int l0 = w0 + wb;                      // first loop position
  std::vector<int> var_at((size_t)n);
  for (int p = 0; p < n; p++) {
    int v = p;
    if (p >= w0 && p < l0) v = n - ub - wb + (p - w0);   // warp slice: just below the units
    else if (p >= l0 && p < n - ub) v = p - wb;           // loops: below the warp slice
    var_at[(size_t)p] = v;
  }
  std::vector<int> order((size_t)n);
  for (int t = 0; t < n; t++) order[(size_t)t] = var_at[(size_t)(n - 1 - t)];
  return order;
}

// support of every DAG node as a 64-bit variable set
static std::vector<uint64_t> supports(const FormDag& d) {
  std::vector<uint64_t> s((size_t)d.size(), 0);
  for (int i = 0; i < d.size(); i++) {
    const FNode& f = d.node(i);
    if (f.op == FVAR) s[(size_t)i] = 1ull << f.var;
    for (int c : f.kids) s[(size_t)i] |= s[(size_t)c];
  }
  return s;
}

// Count-mode order: the variable placed next (from the top position down) is
// the one that completes the most top-level conjuncts together with the
// variables already placed, then the one most connected to them, then the
// most frequent.  Conjuncts decided high up let whole warps skip inner
// levels; the order does not change any count.
// tie-break of search_order variant `seed` (splitmix64 of seed, step, letter)
static uint64_t order_tie(uint64_t seed, int step, int v) {
  uint64_t z = seed * 0x9E3779B97F4A7C15ull + (uint64_t)step * 0xBF58476D1CE4E5B9ull + (uint64_t)v * 0x94D049BB133111EBull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

std::vector<int> search_order(const Grounded& g, uint64_t seed) {
  const FormDag& d = g.dag;
  std::vector<uint64_t> sup = supports(d);
  std::vector<uint64_t> conj;
  const FNode& root = d.node(g.root);
  if (root.op == FAND)
    for (int c : root.kids) conj.push_back(sup[(size_t)c]);
  else
    conj.push_back(sup[(size_t)g.root]);
  int n = g.nvars;
  std::vector<int> occ((size_t)n, 0);
  for (uint64_t s : conj)
    for (int v = 0; v < n; v++)
      if ((s >> v) & 1) occ[(size_t)v]++;
  std::vector<int> order;
  uint64_t chosen = 0;
  std::vector<long long> done_of((size_t)n), conn_of((size_t)n);
  for (int step = 0; step < n; step++) {
    // per candidate letter v: the conjuncts that v completes (v is their
    // last letter not yet placed) and the letters already placed that share
    // a conjunct with v, in one pass over the conjuncts
    std::fill(done_of.begin(), done_of.end(), 0);
    std::fill(conn_of.begin(), conn_of.end(), 0);
    for (uint64_t s : conj) {
      const uint64_t rest = s & ~chosen;
      if (!rest) continue;
      const long long placed = __builtin_popcountll(s & chosen);
      if ((rest & (rest - 1)) == 0) done_of[(size_t)__builtin_ctzll(rest)]++;
      for (uint64_t r = rest; r; r &= r - 1) conn_of[(size_t)__builtin_ctzll(r)] += placed;
    }
    int best = -1;
    long long bk[3] = {-1, -1, -1};
    for (int v = 0; v < n; v++) {
      if ((chosen >> v) & 1) continue;
      long long key[3] = {done_of[(size_t)v], conn_of[(size_t)v], occ[(size_t)v]};
      const bool tie = best >= 0 && !std::lexicographical_compare(bk, bk + 3, key, key + 3) &&
                       !std::lexicographical_compare(key, key + 3, bk, bk + 3);
      if (best < 0 || std::lexicographical_compare(bk, bk + 3, key, key + 3) ||
          (tie && seed && order_tie(seed, step, v) < order_tie(seed, step, best))) {
        best = v;
        std::memcpy(bk, key, sizeof bk);
      }
    }
    order.push_back(best);
    chosen |= 1ull << best;
  }
  return order;
}

// The conjuncts over unit and warp letters are evaluated bitwise over all
// 2^(unit bits + warp bits) items: item bit b is a free generator over the
// item index (bit t of its word vector is bit b of t, Sec. 2.2-2.3).  Each
// kept conjunct is compiled into a short program over a small register file
// (or a table over its word-index letters) and applied once per block of
// words on which it is fixed, blocks visited as a tree over the word-index
// bits; a block whose AND is zero is skipped whole.  Nothing of the size of
// the item vector is held but the result.
namespace {
struct CIns {
  uint8_t op;        // 0 const 0, 1 const 1, 2 var, 3 not, 4 and, 5 or, 6 xor, 7 copy
  uint8_t bit;       // var: item bit
  uint32_t dst, a, b;
};
}  // namespace

std::vector<uint64_t> alive_words(const Grounded& g, const Layout& L) {
  const int wb = L.warp_bits, ub = L.unit_bits + wb;
  if (L.unit_bits <= 0 || ub > 22) return {};
  const FormDag& d = g.dag;
  std::vector<uint64_t> sup = supports(d);
  uint64_t umask = 0;
  std::vector<int> ubit(64, -1);
  for (int b = 0; b < ub; b++) {
    const int pos = b < wb ? L.first_lane_pos() + L.lane_bits + b : L.first_unit_pos() + (b - wb);
    const int v = L.var_of_pos[(size_t)pos];
    umask |= 1ull << v;
    ubit[(size_t)v] = b;
  }
  std::vector<int> keep;
  const FNode& root = d.node(g.root);
  if (root.op == FAND) {
    for (int c : root.kids)
      if ((sup[(size_t)c] & ~umask) == 0) keep.push_back(c);
  } else if ((sup[(size_t)g.root] & ~umask) == 0) {
    keep.push_back(g.root);
  }
  if (keep.empty()) return {};
  // one program per kept conjunct: the nodes under it, children first (a
  // child's id is smaller), each in its own register
  std::vector<std::vector<CIns>> progs;
  std::vector<uint32_t> out_reg;
  size_t nregs = 1;
  std::vector<int> slot((size_t)d.size(), -1);
  for (int c : keep) {
    std::vector<int> nodes, stack{c};
    while (!stack.empty()) {
      int x = stack.back();
      stack.pop_back();
      if (slot[(size_t)x] != -1) continue;
      slot[(size_t)x] = 0;
      nodes.push_back(x);
      for (int k : d.node(x).kids) stack.push_back(k);
    }
    std::sort(nodes.begin(), nodes.end());
    for (size_t i = 0; i < nodes.size(); i++) slot[(size_t)nodes[i]] = (int)i;
    std::vector<CIns> pr;
    for (int x : nodes) {
      const FNode& f = d.node(x);
      const uint32_t r = (uint32_t)slot[(size_t)x];
      switch (f.op) {
        case F0: pr.push_back({0, 0, r, 0, 0}); break;
        case F1: pr.push_back({1, 0, r, 0, 0}); break;
        case FVAR: pr.push_back({2, (uint8_t)ubit[(size_t)f.var], r, 0, 0}); break;
        case FNOT: pr.push_back({3, 0, r, (uint32_t)slot[(size_t)f.kids[0]], 0}); break;
        case FXOR:
          pr.push_back({6, 0, r, (uint32_t)slot[(size_t)f.kids[0]], (uint32_t)slot[(size_t)f.kids[1]]});
          break;
        case FAND:
        case FOR: {
          const uint8_t op = f.op == FAND ? 4 : 5;
          if (f.kids.empty()) {
            pr.push_back({(uint8_t)(f.op == FAND ? 1 : 0), 0, r, 0, 0});
            break;
          }
          pr.push_back({7, 0, r, (uint32_t)slot[(size_t)f.kids[0]], 0});
          for (size_t i = 1; i < f.kids.size(); i++) pr.push_back({op, 0, r, r, (uint32_t)slot[(size_t)f.kids[i]]});
          break;
        }
      }
    }
    nregs = std::max(nregs, nodes.size());
    out_reg.push_back((uint32_t)slot[(size_t)c]);
    progs.push_back(std::move(pr));
    for (int x : nodes) slot[(size_t)x] = -1;
  }
  const uint64_t U = 1ull << ub;
  const size_t W = U >= 64 ? (size_t)(U / 64) : 1;
  const uint64_t tail = U >= 64 ? ~0ull : ((1ull << U) - 1ull);
  static const uint64_t pat[6] = {0xAAAAAAAAAAAAAAAAull, 0xCCCCCCCCCCCCCCCCull, 0xF0F0F0F0F0F0F0F0ull,
                                  0xFF00FF00FF00FF00ull, 0xFFFF0000FFFF0000ull, 0xFFFFFFFF00000000ull};
  std::vector<uint64_t> reg(nregs, 0);
  auto run = [&](size_t c, uint64_t w) {
    for (const CIns& in : progs[c]) {
      uint64_t v = 0;
      switch (in.op) {
        case 0: v = 0; break;
        case 1: v = ~0ull; break;
        case 2: v = in.bit < 6 ? pat[in.bit] : (((w >> (in.bit - 6)) & 1) ? ~0ull : 0ull); break;
        case 3: v = ~reg[in.a]; break;
        case 4: v = reg[in.a] & reg[in.b]; break;
        case 5: v = reg[in.a] | reg[in.b]; break;
        case 6: v = reg[in.a] ^ reg[in.b]; break;
        default: v = reg[in.a]; break;
      }
      reg[in.dst] = v;
    }
    return reg[out_reg[c]];
  };
  // a conjunct over few word-index letters (item bits >= 6) becomes a table:
  // its 64-bit value for each setting of those letters (the in-word letters
  // are the patterns), so a word costs a gather of those bits and a lookup
  struct Table {
    std::vector<int> hbits;        // item bits >= 6 in the support, as word-index bits
    std::vector<uint64_t> words;   // value per setting of hbits
  };
  std::vector<Table> tables(progs.size());
  std::vector<char> tabled(progs.size(), 0);
  for (size_t c = 0; c < progs.size(); c++) {
    std::vector<int> hb;
    for (const CIns& in : progs[c])
      if (in.op == 2 && in.bit >= 6 && std::find(hb.begin(), hb.end(), in.bit - 6) == hb.end()) hb.push_back(in.bit - 6);
    if (hb.size() > 10) continue;
    Table t;
    t.hbits = hb;
    t.words.resize(1ull << hb.size());
    for (uint64_t m = 0; m < t.words.size(); m++) {
      uint64_t w = 0;
      for (size_t i = 0; i < hb.size(); i++)
        if ((m >> i) & 1) w |= 1ull << hb[i];
      t.words[m] = run(c, w);
    }
    tables[c] = std::move(t);
    tabled[c] = 1;
  }
  // The words are visited as a binary tree over the word-index bits, top
  // bit first: a conjunct whose lowest word-index letter is bit m is fixed
  // on every block of 2^m consecutive words, so it is applied once per such
  // block; a block whose AND is already zero holds no live item and is
  // skipped whole (the level pruning of the kernels, on the host).  Conjuncts
  // without a table are evaluated per word.
  int nb = 0;
  while (((size_t)1 << nb) < W) nb++;
  std::vector<std::vector<size_t>> at_level((size_t)nb + 1);
  for (size_t c = 0; c < progs.size(); c++) {
    int lvl = 0;
    if (tabled[c]) {
      lvl = nb;
      for (int h : tables[c].hbits) lvl = std::min(lvl, h);
    }
    at_level[(size_t)lvl].push_back(c);
  }
  auto apply = [&](int lvl, uint64_t w, uint64_t acc) {
    for (size_t c : at_level[(size_t)lvl]) {
      if (!acc) break;
      if (tabled[c]) {
        const Table& t = tables[c];
        uint64_t m = 0;
        for (size_t i = 0; i < t.hbits.size(); i++) m |= ((w >> t.hbits[i]) & 1ull) << i;
        acc &= t.words[m];
      } else {
        acc &= run(c, w);
      }
    }
    return acc;
  };
  std::vector<uint64_t> all(W, 0);
  struct Node {
    int lvl;        // the block holds words [w, w + 2^lvl)
    uint64_t w;
    uint64_t acc;   // AND of the conjuncts fixed on the block
  };
  std::vector<Node> stack{{nb, 0, apply(nb, 0, tail)}};
  while (!stack.empty()) {
    Node nd = stack.back();
    stack.pop_back();
    if (!nd.acc) continue;
    if (nd.lvl == 0) {
      all[(size_t)nd.w] = nd.acc;
      continue;
    }
    const int child = nd.lvl - 1;
    for (uint64_t half : {(uint64_t)1, (uint64_t)0}) {
      const uint64_t w = nd.w | (half << child);
      const uint64_t acc = apply(child, w, nd.acc);
      if (acc) stack.push_back({child, w, acc});
    }
  }
  return all;
}

std::vector<uint8_t> alive_items(const Grounded& g, const Layout& L) {
  std::vector<uint64_t> all = alive_words(g, L);
  if (all.empty()) return {};
  const uint64_t U = 1ull << (L.unit_bits + L.warp_bits);
  std::vector<uint8_t> alive((size_t)U, 0);
  for (uint64_t u = 0; u < U; u++) alive[(size_t)u] = (uint8_t)((all[(size_t)(u >> 6)] >> (u & 63)) & 1);
  return alive;
}

uint32_t rmask_of(const LutProgram& p, const Val& v) {
  if (v.kind == V_LUT) return p.luts[(size_t)v.id].rmask;
  if (v.kind == V_VAR) return 0;
  const ConstVec& c = p.consts[(size_t)v.id];
  uint32_t m = 0;
  for (size_t s = 0; s < c.w.size(); s++)
    for (int b = 0; (1u << b) < c.w.size(); b++)
      if (c.w[s] != c.w[s ^ (1u << b)]) m |= 1u << b;
  return m;
}

namespace {

enum GOp : uint8_t { G_AND, G_OR, G_XOR };
enum GKind : uint8_t { K_CONST, K_VAR, K_GATE };

struct GNode {
  GKind kind;
  GOp op = G_AND;
  int cid = -1, pos = -1;
  int in[2] = {0, 0};    // literals: node*2 + negation
  int level = LV_CONST;
  uint32_t rmask = 0;
};

inline int lit(int node, bool neg) { return node * 2 + (neg ? 1 : 0); }
inline int lnode(int l) { return l >> 1; }
inline bool lneg(int l) { return l & 1; }

struct Cut {
  int leaf[3];
  int nleaf;
  long long cost;
};

class Lowerer {
 public:
  Lowerer(const Grounded& g, const Layout& L) : g_(g), L_(L), nreg_(1u << L.r) {
    prog_.layout = L;
  }

  LutProgram run() {
    const FormDag& d = g_.dag;
    flevel_.assign((size_t)d.size(), LV_CONST);
    for (int i = 0; i < d.size(); i++) {
      const FNode& f = d.node(i);
      if (f.op == FVAR) flevel_[(size_t)i] = L_.level_of_pos(L_.pos_of_var[(size_t)f.var]);
      for (int c : f.kids) flevel_[(size_t)i] = std::max(flevel_[(size_t)i], flevel_[(size_t)c]);
    }
    memo_.assign((size_t)d.size(), -1);
    int nl = L_.nlevels();
    std::vector<int> acc_lit((size_t)nl, -1);
    int out = lower_root(acc_lit);
    map_and_emit(out, acc_lit);
    return std::move(prog_);
  }

 private:
  // ---------------------------------------------------------- constants --
  int const_node(const std::vector<uint32_t>& w) {
    auto it = const_ids_.find(w);
    if (it != const_ids_.end()) return it->second;
    ConstVec cv;
    cv.w = w;
    prog_.consts.push_back(cv);
    GNode gn;
    gn.kind = K_CONST;
    gn.cid = (int)prog_.consts.size() - 1;
    gn.level = LV_CONST;
    nodes_.push_back(gn);
    int id = (int)nodes_.size() - 1;
    nodes_.back().rmask = rmask_of(prog_, Val{V_CONST, gn.cid});
    const_ids_.emplace(w, id);
    return id;
  }
  const std::vector<uint32_t>& cval(int node) const { return prog_.consts[(size_t)nodes_[(size_t)node].cid].w; }
  std::vector<uint32_t> lit_const(int l) const {
    std::vector<uint32_t> w = cval(lnode(l));
    if (lneg(l))
      for (auto& x : w) x = ~x;
    return w;
  }
  static bool all_is(const std::vector<uint32_t>& w, uint32_t v) {
    for (uint32_t x : w)
      if (x != v) return false;
    return true;
  }
  bool is_const(int l) const { return nodes_[(size_t)lnode(l)].kind == K_CONST; }
  int const_lit(const std::vector<uint32_t>& w) { return lit(const_node(w), false); }

  // word value of a constant-level DAG node, per register index
  std::vector<uint32_t> eval_const(int f) {
    auto it = cmemo_.find(f);
    if (it != cmemo_.end()) return it->second;
    const FNode& n = g_.dag.node(f);
    std::vector<uint32_t> w(nreg_, 0);
    switch (n.op) {
      case F0: break;
      case F1: std::fill(w.begin(), w.end(), ~0u); break;
      case FVAR: {
        int p = L_.pos_of_var[(size_t)n.var];
        for (uint32_t s = 0; s < nreg_; s++)
          w[s] = p < 5 ? kInReg[p] : (((s >> (p - 5)) & 1u) ? ~0u : 0u);
        break;
      }
      case FNOT: {
        w = eval_const(n.kids[0]);
        for (auto& x : w) x = ~x;
        break;
      }
      case FAND: {
        std::fill(w.begin(), w.end(), ~0u);
        for (int c : n.kids) {
          auto v = eval_const(c);
          for (uint32_t s = 0; s < nreg_; s++) w[s] &= v[s];
        }
        break;
      }
      case FOR: {
        for (int c : n.kids) {
          auto v = eval_const(c);
          for (uint32_t s = 0; s < nreg_; s++) w[s] |= v[s];
        }
        break;
      }
      case FXOR: {
        auto a = eval_const(n.kids[0]), b = eval_const(n.kids[1]);
        for (uint32_t s = 0; s < nreg_; s++) w[s] = a[s] ^ b[s];
        break;
      }
    }
    cmemo_.emplace(f, w);
    return w;
  }

  // -------------------------------------------------------------- gates --
  int gate(GOp op, int a, int b) {
    if (is_const(a) && is_const(b)) {
      auto x = lit_const(a), y = lit_const(b);
      for (uint32_t s = 0; s < nreg_; s++) x[s] = op == G_AND ? (x[s] & y[s]) : op == G_OR ? (x[s] | y[s]) : (x[s] ^ y[s]);
      return const_lit(x);
    }
    if (is_const(a)) std::swap(a, b);
    if (is_const(b)) {
      auto c = lit_const(b);
      if (op == G_AND) {
        if (all_is(c, 0)) return const_lit(c);
        if (all_is(c, ~0u)) return a;
      } else if (op == G_OR) {
        if (all_is(c, ~0u)) return const_lit(c);
        if (all_is(c, 0)) return a;
      } else {
        if (all_is(c, 0)) return a;
        if (all_is(c, ~0u)) return a ^ 1;
      }
      b = const_lit(c);   // keep constant operands positive
    }
    if (a == b) return op == G_XOR ? const_lit(std::vector<uint32_t>(nreg_, 0)) : a;
    if (a == (b ^ 1)) return const_lit(std::vector<uint32_t>(nreg_, op == G_AND ? 0u : ~0u));
    bool outneg = false;
    if (op == G_XOR) {
      if (lneg(a) && !is_const(a)) { a ^= 1; outneg = !outneg; }
      if (lneg(b) && !is_const(b)) { b ^= 1; outneg = !outneg; }
    }
    if (a > b) std::swap(a, b);
    uint64_t key = ((uint64_t)op << 62) ^ ((uint64_t)(uint32_t)a << 31) ^ (uint64_t)(uint32_t)b;
    auto it = gate_ids_.find(key);
    int id;
    if (it != gate_ids_.end()) {
      id = it->second;
    } else {
      GNode gn;
      gn.kind = K_GATE;
      gn.op = op;
      gn.in[0] = a;
      gn.in[1] = b;
      gn.level = std::max(nodes_[(size_t)lnode(a)].level, nodes_[(size_t)lnode(b)].level);
      gn.rmask = nodes_[(size_t)lnode(a)].rmask | nodes_[(size_t)lnode(b)].rmask;
      nodes_.push_back(gn);
      id = (int)nodes_.size() - 1;
      gate_ids_.emplace(key, id);
      prog_.gates++;
    }
    return lit(id, outneg);
  }

  int var_node(int pos) {
    auto it = var_ids_.find(pos);
    if (it != var_ids_.end()) return it->second;
    GNode gn;
    gn.kind = K_VAR;
    gn.pos = pos;
    gn.level = L_.level_of_pos(pos);
    nodes_.push_back(gn);
    int id = (int)nodes_.size() - 1;
    var_ids_.emplace(pos, id);
    return id;
  }

  int level_of_lit(int l) const { return nodes_[(size_t)lnode(l)].level; }

  // n-ary AND/OR: operands grouped by level, each group folded into a chain,
  // groups joined from the outermost level inwards so every prefix is hoisted.
  // If `accs` is given (top-level conjunction), the running value after each
  // level's group is recorded there.
  int nary(GOp op, const std::vector<int>& kids, std::vector<int>* accs) {
    std::vector<std::pair<int, int>> items;   // (level, literal)
    std::vector<std::vector<int>> keys;
    for (size_t i = 0; i < kids.size(); i++) {
      int l = lower(kids[i]);
      items.push_back({level_of_lit(l), l});
      // operands that share sub-operands (clauses with common literals) are
      // placed next to each other, which keeps shared partial values short-lived
      const FNode& f = g_.dag.node(kids[i]);
      keys.push_back(f.op == FAND || f.op == FOR ? f.kids : std::vector<int>{kids[i]});
    }
    std::vector<size_t> ord(items.size());
    for (size_t i = 0; i < ord.size(); i++) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) {
      if (items[a].first != items[b].first) return items[a].first < items[b].first;
      return keys[a] < keys[b];
    });
    {
      std::vector<std::pair<int, int>> sorted;
      for (size_t i : ord) sorted.push_back(items[i]);
      items.swap(sorted);
    }
    int x = -1;
    size_t i = 0;
    while (i < items.size()) {
      size_t j = i;
      int lev = items[i].first;
      int grp = -1;
      while (j < items.size() && items[j].first == lev) {
        grp = grp < 0 ? items[j].second : gate(op, grp, items[j].second);
        j++;
      }
      x = x < 0 ? grp : gate(op, x, grp);
      if (accs && lev >= 0) (*accs)[(size_t)lev] = x;
      if (accs && lev < 0) const_acc_lit_ = x;
      i = j;
    }
    if (x < 0) x = const_lit(std::vector<uint32_t>(nreg_, op == G_AND ? ~0u : 0u));
    return x;
  }

  int lower(int f) {
    if (memo_[(size_t)f] >= 0) return memo_[(size_t)f];
    const FNode& n = g_.dag.node(f);
    int r;
    if (flevel_[(size_t)f] == LV_CONST) {
      r = const_lit(eval_const(f));
    } else {
      switch (n.op) {
        case FVAR: r = lit(var_node(L_.pos_of_var[(size_t)n.var]), false); break;
        case FNOT: r = lower(n.kids[0]) ^ 1; break;
        case FXOR: r = gate(G_XOR, lower(n.kids[0]), lower(n.kids[1])); break;
        case FAND: r = nary(G_AND, n.kids, nullptr); break;
        case FOR: r = nary(G_OR, n.kids, nullptr); break;
        default: r = const_lit(eval_const(f)); break;
      }
    }
    memo_[(size_t)f] = r;
    return r;
  }

  int lower_root(std::vector<int>& acc_lit) {
    const FNode& root = g_.dag.node(g_.root);
    if (root.op == FAND && flevel_[(size_t)g_.root] != LV_CONST) return nary(G_AND, root.kids, &acc_lit);
    int l = lower(g_.root);
    int lev = level_of_lit(l);
    if (lev >= 0) acc_lit[(size_t)lev] = l;
    else const_acc_lit_ = l;
    return l;
  }

  // ------------------------------------------------------------ mapping --
  long long weight(int node) const { return 1LL << __builtin_popcount(nodes_[(size_t)node].rmask); }

  bool exclusive(int x) const {
    const GNode& gx = nodes_[(size_t)x];
    return gx.kind == K_GATE && fanout_[(size_t)x] == 1 && !required_[(size_t)x] && gx.level == user_level_[(size_t)x];
  }

  static bool merge_leaves(const int* a, int na, const int* b, int nb, int* out, int& no) {
    no = 0;
    for (int i = 0; i < na; i++) out[no++] = a[i];
    for (int i = 0; i < nb; i++) {
      bool dup = false;
      for (int j = 0; j < no; j++) dup |= out[j] == b[i];
      if (!dup) {
        if (no == 3) return false;
        out[no++] = b[i];
      }
    }
    std::sort(out, out + no);
    return true;
  }

  void enumerate_cuts(int g) {
    const GNode& gn = nodes_[(size_t)g];
    struct Opt { int leaf[3]; int n; long long extra; };
    // a child is either a leaf of the cut, or its own cut is absorbed: always
    // for a child used only here; for a shared child (same level) when its
    // cut's leaves are already computed values -- the shared logic is then
    // duplicated inside this LUT for free instead of kept live in a register
    auto options = [&](int x, std::vector<Opt>& o) {
      const bool ex = exclusive(x);
      Opt leaf{{x, 0, 0}, 1, ex ? best_[(size_t)x] : 0};
      o.push_back(leaf);
      const GNode& gx = nodes_[(size_t)x];
      if (gx.kind != K_GATE || gx.level != gn.level) return;
      for (const Cut& c : cuts_[(size_t)x]) {
        if (ex) {
          o.push_back(Opt{{c.leaf[0], c.leaf[1], c.leaf[2]}, c.nleaf, c.cost - weight(x)});
        } else {
          bool free_leaves = true;
          for (int i = 0; i < c.nleaf; i++) free_leaves &= !exclusive(c.leaf[i]);
          if (free_leaves) o.push_back(Opt{{c.leaf[0], c.leaf[1], c.leaf[2]}, c.nleaf, 0});
        }
      }
    };
    std::vector<Opt> oa, ob;
    options(lnode(gn.in[0]), oa);
    options(lnode(gn.in[1]), ob);
    std::vector<Cut>& out = cuts_[(size_t)g];
    for (auto& a : oa)
      for (auto& b : ob) {
        Cut c;
        if (!merge_leaves(a.leaf, a.n, b.leaf, b.n, c.leaf, c.nleaf)) continue;
        c.cost = weight(g) + a.extra + b.extra;
        bool dup = false;
        for (auto& e : out)
          if (e.nleaf == c.nleaf && std::equal(e.leaf, e.leaf + e.nleaf, c.leaf)) {
            e.cost = std::min(e.cost, c.cost);
            dup = true;
          }
        if (!dup) out.push_back(c);
      }
    std::sort(out.begin(), out.end(), [](const Cut& x, const Cut& y) { return x.cost < y.cost || (x.cost == y.cost && x.nleaf < y.nleaf); });
    if (out.size() > 12) out.resize(12);
    best_[(size_t)g] = out.empty() ? (1LL << 40) : out[0].cost;
  }

  // truth table of node x over the leaves (patterns 0xF0, 0xCC, 0xAA)
  uint8_t cone_tt(int x, const int* leaf, int nleaf, std::unordered_map<int, uint8_t>& memo) {
    static const uint8_t pat[3] = {0xF0, 0xCC, 0xAA};
    for (int i = 0; i < nleaf; i++)
      if (leaf[i] == x) return pat[i];
    auto it = memo.find(x);
    if (it != memo.end()) return it->second;
    const GNode& gx = nodes_[(size_t)x];
    uint8_t v = 0;
    if (gx.kind == K_GATE) {
      uint8_t a = cone_tt(lnode(gx.in[0]), leaf, nleaf, memo), b = cone_tt(lnode(gx.in[1]), leaf, nleaf, memo);
      if (lneg(gx.in[0])) a = (uint8_t)~a;
      if (lneg(gx.in[1])) b = (uint8_t)~b;
      v = gx.op == G_AND ? (uint8_t)(a & b) : gx.op == G_OR ? (uint8_t)(a | b) : (uint8_t)(a ^ b);
    } else {
      throw CompileError{"internal: cut does not cover its cone"};
    }
    memo.emplace(x, v);
    return v;
  }

  Val leaf_val(int x) {
    const GNode& gx = nodes_[(size_t)x];
    if (gx.kind == K_CONST) return Val{V_CONST, gx.cid};
    if (gx.kind == K_VAR) return Val{V_VAR, gx.pos};
    return Val{V_LUT, emit(x)};
  }

  // the operands of a LUT: the most recently built (deepest, e.g. a running
  // conjunction) first, so that short side values are computed right before
  // their use and do not stay live across a long chain
  void emit_leaves(const Cut& c, Lut& lu) {
    int order[3] = {0, 1, 2};
    std::sort(order, order + c.nleaf, [&](int a, int b) { return c.leaf[a] > c.leaf[b]; });
    for (int q = 0; q < c.nleaf; q++) lu.in[order[q]] = leaf_val(c.leaf[order[q]]);
    for (int i = c.nleaf; i < 3; i++) lu.in[i] = lu.in[0];
  }

  // emit node x (a gate) as a LUT with its best cut; returns the LUT index
  int emit(int x) {
    auto it = emitted_.find(x);
    if (it != emitted_.end()) return it->second;
    const Cut& c = cuts_[(size_t)x][0];
    Lut lu;
    emit_leaves(c, lu);
    std::unordered_map<int, uint8_t> memo;
    lu.tt = cone_tt(x, c.leaf, c.nleaf, memo);
    lu.level = nodes_[(size_t)x].level;
    lu.rmask = nodes_[(size_t)x].rmask;
    raw_.push_back(lu);
    int id = (int)raw_.size() - 1;
    emitted_.emplace(x, id);
    return id;
  }

  // a required output literal as a positive value
  Val output_val(int l) {
    int x = lnode(l);
    const GNode& gx = nodes_[(size_t)x];
    if (gx.kind == K_CONST) {
      auto w = lit_const(l);
      return Val{V_CONST, nodes_[(size_t)lnode(const_lit(w))].cid};
    }
    if (!lneg(l)) return leaf_val(x);
    auto it = neg_emitted_.find(x);
    if (it != neg_emitted_.end()) return Val{V_LUT, it->second};
    Lut lu;
    if (gx.kind == K_VAR) {
      lu.in[0] = lu.in[1] = lu.in[2] = Val{V_VAR, gx.pos};
      lu.tt = (uint8_t)~0xF0;
    } else {
      const Cut& c = cuts_[(size_t)x][0];
      emit_leaves(c, lu);
      std::unordered_map<int, uint8_t> memo;
      lu.tt = (uint8_t)~cone_tt(x, c.leaf, c.nleaf, memo);
    }
    lu.level = gx.level;
    lu.rmask = gx.rmask;
    raw_.push_back(lu);
    int id = (int)raw_.size() - 1;
    neg_emitted_.emplace(x, id);
    return Val{V_LUT, id};
  }

  void map_and_emit(int out, std::vector<int>& acc_lit) {
    int N = (int)nodes_.size();
    fanout_.assign((size_t)N, 0);
    required_.assign((size_t)N, false);
    user_level_.assign((size_t)N, -2);
    // reachability from the outputs
    std::vector<int> roots;
    roots.push_back(out);
    for (int l : acc_lit)
      if (l >= 0) roots.push_back(l);
    std::vector<bool> live((size_t)N, false);
    std::vector<int> stack;
    for (int l : roots) {
      required_[(size_t)lnode(l)] = true;
      stack.push_back(lnode(l));
    }
    while (!stack.empty()) {
      int x = stack.back();
      stack.pop_back();
      if (live[(size_t)x]) continue;
      live[(size_t)x] = true;
      const GNode& gx = nodes_[(size_t)x];
      if (gx.kind == K_GATE)
        for (int l : gx.in) stack.push_back(lnode(l));
    }
    for (int x = 0; x < N; x++) {
      if (!live[(size_t)x] || nodes_[(size_t)x].kind != K_GATE) continue;
      for (int l : nodes_[(size_t)x].in) {
        int c = lnode(l);
        fanout_[(size_t)c]++;
        if (user_level_[(size_t)c] == -2) user_level_[(size_t)c] = nodes_[(size_t)x].level;
        else if (user_level_[(size_t)c] != nodes_[(size_t)x].level) user_level_[(size_t)c] = -3;
      }
    }
    cuts_.assign((size_t)N, {});
    best_.assign((size_t)N, 0);
    for (int x = 0; x < N; x++)
      if (live[(size_t)x] && nodes_[(size_t)x].kind == K_GATE) enumerate_cuts(x);

    // outputs first (positive values), then order by level
    Val outv = output_val(out);
    std::vector<Val> accv(acc_lit.size());
    for (size_t i = 0; i < acc_lit.size(); i++)
      if (acc_lit[i] >= 0) accv[i] = output_val(acc_lit[i]);

    // stable sort of the LUTs by level keeps topological order inside a level
    std::vector<int> idx(raw_.size());
    for (size_t i = 0; i < idx.size(); i++) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return raw_[(size_t)a].level < raw_[(size_t)b].level; });
    std::vector<int> newid(raw_.size());
    for (size_t i = 0; i < idx.size(); i++) newid[(size_t)idx[i]] = (int)i;
    auto remap = [&](Val v) {
      if (v.kind == V_LUT) v.id = newid[(size_t)v.id];
      return v;
    };
    for (int i : idx) {
      Lut lu = raw_[(size_t)i];
      for (auto& v : lu.in) v = remap(v);
      prog_.luts.push_back(lu);
    }
    prog_.out = remap(outv);
    int nl = L_.nlevels();
    prog_.levels.assign((size_t)nl, LevelInfo{});
    for (int lv = 0; lv < nl; lv++) {
      LevelInfo& li = prog_.levels[(size_t)lv];
      li.lut_begin = (int)(std::lower_bound(prog_.luts.begin(), prog_.luts.end(), lv,
                                            [](const Lut& a, int l) { return a.level < l; }) - prog_.luts.begin());
      li.lut_end = (int)(std::lower_bound(prog_.luts.begin(), prog_.luts.end(), lv + 1,
                                          [](const Lut& a, int l) { return a.level < l; }) - prog_.luts.begin());
      if (acc_lit[(size_t)lv] >= 0) {
        li.has_acc = true;
        li.acc = remap(accv[(size_t)lv]);
      }
      long long ops = 0;
      for (int i = li.lut_begin; i < li.lut_end; i++) ops += 1LL << __builtin_popcount(prog_.luts[(size_t)i].rmask);
      if (lv < 16) prog_.lop3_per_level[lv] = ops;
    }
    if (const_acc_lit_ >= 0) prog_.const_acc.w = lit_const(const_acc_lit_);
    else prog_.const_acc.w.assign(nreg_, ~0u);
  }

  const Grounded& g_;
  const Layout& L_;
  uint32_t nreg_;
  LutProgram prog_;
  std::vector<int> flevel_;
  std::vector<int> memo_;
  std::map<int, std::vector<uint32_t>> cmemo_;
  std::vector<GNode> nodes_;
  std::map<std::vector<uint32_t>, int> const_ids_;
  std::unordered_map<uint64_t, int> gate_ids_;
  std::unordered_map<int, int> var_ids_;
  int const_acc_lit_ = -1;
  std::vector<int> fanout_;
  std::vector<bool> required_;
  std::vector<int> user_level_;
  std::vector<std::vector<Cut>> cuts_;
  std::vector<long long> best_;
  std::vector<Lut> raw_;
  std::unordered_map<int, int> emitted_, neg_emitted_;
};

}  // namespace

LutProgram lower_and_map(const Grounded& g, const Layout& L) {
  Lowerer lw(g, L);
  return lw.run();
}

}  // namespace fbg
