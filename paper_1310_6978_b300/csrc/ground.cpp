// ground.cpp -- the translation * of Sec. 3.1 into a hash-consed Boolean DAG.
//
// R(a_1..a_k)* is the letter q_{R a_1..a_k}; forall x phi is the conjunction
// of phi(a) over the domain, exists the disjunction; ~ & | commute with *.
// '^' is the symmetric difference of Sec. 4.2.  The DAG removes the
// constants 0 and 1 as it is built (the Reduction submodule of Sec. 4.1) and
// shares equal subterms (common-subexpression elimination).
#include <algorithm>

#include "fbg_internal.hpp"

namespace fbg {

FormDag::FormDag() {
  nodes_.push_back(FNode{F0, -1, {}});
  nodes_.push_back(FNode{F1, -1, {}});
}

int FormDag::intern(FNode&& n) {
  std::string key;
  key.reserve(8 + 8 * n.kids.size());
  key.push_back((char)n.op);
  key.append(reinterpret_cast<const char*>(&n.var), sizeof(int));
  for (int c : n.kids) key.append(reinterpret_cast<const char*>(&c), sizeof(int));
  auto it = table_.find(key);
  if (it != table_.end()) return it->second;
  int id = (int)nodes_.size();
  nodes_.push_back(std::move(n));
  table_.emplace(std::move(key), id);
  return id;
}

int FormDag::var(int v) { return intern(FNode{FVAR, v, {}}); }

int FormDag::mk_not(int a) {
  if (a == 0) return 1;
  if (a == 1) return 0;
  if (nodes_[a].op == FNOT) return nodes_[a].kids[0];
  return intern(FNode{FNOT, -1, {a}});
}

int FormDag::mk_nary(FOp op, const std::vector<int>& in) {
  const int absorbing = op == FAND ? 0 : 1, neutral = op == FAND ? 1 : 0;
  std::vector<int> kids;
  kids.reserve(in.size());
  for (int c : in) {
    if (nodes_[c].op == op) {
      for (int g : nodes_[c].kids) kids.push_back(g);
    } else {
      kids.push_back(c);
    }
  }
  std::vector<int> keep;
  keep.reserve(kids.size());
  for (int c : kids) {
    if (c == absorbing) return absorbing;
    if (c != neutral) keep.push_back(c);
  }
  std::sort(keep.begin(), keep.end());
  keep.erase(std::unique(keep.begin(), keep.end()), keep.end());
  for (int c : keep)
    if (nodes_[c].op == FNOT && std::binary_search(keep.begin(), keep.end(), nodes_[c].kids[0])) return absorbing;
  if (keep.empty()) return neutral;
  if (keep.size() == 1) return keep[0];
  return intern(FNode{op, -1, std::move(keep)});
}

int FormDag::mk_and(const std::vector<int>& kids) { return mk_nary(FAND, kids); }
int FormDag::mk_or(const std::vector<int>& kids) { return mk_nary(FOR, kids); }

int FormDag::mk_xor(int a, int b) {
  if (a == 0) return b;
  if (b == 0) return a;
  if (a == 1) return mk_not(b);
  if (b == 1) return mk_not(a);
  bool neg = false;
  if (nodes_[a].op == FNOT) { a = nodes_[a].kids[0]; neg = !neg; }
  if (nodes_[b].op == FNOT) { b = nodes_[b].kids[0]; neg = !neg; }
  if (a == b) return neg ? 1 : 0;
  if (a > b) std::swap(a, b);
  int x = intern(FNode{FXOR, -1, {a, b}});
  return neg ? mk_not(x) : x;
}

namespace {

struct Grounder {
  const Theory& th;
  FormDag& dag;
  std::vector<int> env;
  const std::vector<int>* killed = nullptr;      // per declared letter
  const std::vector<int>* free_index = nullptr;  // per declared letter

  int idx(const IndexTerm& t) const { return t.slot < 0 ? t.value : env[(size_t)t.slot]; }

  bool guards_hold(const Ast& q) const {
    for (const Guard& g : q.guards) {
      int l = idx(g.l), r = idx(g.r);
      bool ok = false;
      switch (g.op) {
        case 0: ok = l < r; break;
        case 1: ok = l <= r; break;
        case 2: ok = l > r; break;
        case 3: ok = l >= r; break;
        case 4: ok = l == r; break;
        default: ok = l != r; break;
      }
      if (!ok) return false;
    }
    if (q.distinct)
      for (int a = 0; a < q.nbound; a++)
        for (int b = a + 1; b < q.nbound; b++)
          if (env[(size_t)(q.first_slot + a)] == env[(size_t)(q.first_slot + b)]) return false;
    return true;
  }

  int atom(const Ast& e) {
    const Family& f = th.fams[(size_t)e.family];
    long lin = 0;
    for (auto& t : e.idx) {
      int v = idx(t);
      if (v < 0 || v >= th.k) throw CompileError{"index out of the domain in '" + f.name + "'"};
      lin = lin * th.k + v;
    }
    if (f.is_const) return f.bits[(size_t)lin] ? 1 : 0;
    int rk = f.rank[(size_t)lin];
    if (rk < 0) throw CompileError{"'" + f.name + "' applied to a tuple outside its declaration"};
    int id = f.first_id + rk;
    if (killed && (*killed)[(size_t)id] >= 0) return (*killed)[(size_t)id] ? 1 : 0;
    return dag.var(free_index ? (*free_index)[(size_t)id] : id);
  }

  // an assume line: a conjunction of literals, possibly under universal
  // quantifiers; each literal fixes its letter, later ones replacing earlier
  void assume(const Ast& e, bool value, std::vector<int>& fixed) {
    switch (e.kind) {
      case Ast::Const:
        if (e.value == 1 && value) return;
        break;
      case Ast::Atom: {
        const Family& f = th.fams[(size_t)e.family];
        if (f.is_const) break;
        long lin = 0;
        for (auto& t : e.idx) {
          int v = idx(t);
          if (v < 0 || v >= th.k) throw CompileError{"index out of the domain in an assume line"};
          lin = lin * th.k + v;
        }
        int rk = f.rank[(size_t)lin];
        if (rk < 0) break;
        fixed[(size_t)(f.first_id + rk)] = value ? 1 : 0;
        return;
      }
      case Ast::Not:
        if (e.a->kind != Ast::Atom) break;
        assume(*e.a, !value, fixed);
        return;
      case Ast::And:
        if (!value) break;
        assume(*e.a, true, fixed);
        assume(*e.b, true, fixed);
        return;
      case Ast::Forall: {
        if (!value) break;
        if ((int)env.size() < e.first_slot + e.nbound) env.resize((size_t)(e.first_slot + e.nbound));
        std::vector<int> t((size_t)e.nbound, 0);
        for (;;) {
          for (int i = 0; i < e.nbound; i++) env[(size_t)(e.first_slot + i)] = t[(size_t)i];
          if (guards_hold(e)) assume(*e.a, true, fixed);
          int p = e.nbound - 1;
          while (p >= 0 && ++t[(size_t)p] == th.k) t[(size_t)p--] = 0;
          if (p < 0) break;
        }
        return;
      }
      default:
        break;
    }
    throw CompileError{"an assume line must be a conjunction of literals over declared letters"};
  }

  int go(const Ast& e) {
    switch (e.kind) {
      case Ast::Const: return e.value ? 1 : 0;
      case Ast::Atom: return atom(e);
      case Ast::Not: return dag.mk_not(go(*e.a));
      case Ast::And: return dag.mk_and({go(*e.a), go(*e.b)});
      case Ast::Or: return dag.mk_or({go(*e.a), go(*e.b)});
      case Ast::Xor: return dag.mk_xor(go(*e.a), go(*e.b));
      case Ast::Imp: return dag.mk_or({dag.mk_not(go(*e.a)), go(*e.b)});
      case Ast::Iff: return dag.mk_not(dag.mk_xor(go(*e.a), go(*e.b)));
      case Ast::Forall:
      case Ast::Exists: {
        if ((int)env.size() < e.first_slot + e.nbound) env.resize((size_t)(e.first_slot + e.nbound));
        std::vector<int> parts;
        std::vector<int> t((size_t)e.nbound, 0);
        for (;;) {
          for (int i = 0; i < e.nbound; i++) env[(size_t)(e.first_slot + i)] = t[(size_t)i];
          if (guards_hold(e)) parts.push_back(go(*e.a));
          int p = e.nbound - 1;
          while (p >= 0 && ++t[(size_t)p] == th.k) t[(size_t)p--] = 0;
          if (p < 0) break;
        }
        return e.kind == Ast::Forall ? dag.mk_and(parts) : dag.mk_or(parts);
      }
    }
    return 0;
  }
};

}  // namespace

Grounded ground(const Theory& th) {
  Grounded g;
  Grounder gr{th, g.dag, {}};
  // killing variables (Sec. 3.3): assumed letters become constants and the
  // free letters are renumbered in declaration order
  g.killed.assign((size_t)th.nvars, -1);
  for (auto& a : th.assumes) gr.assume(*a, true, g.killed);
  std::vector<int> free_index((size_t)th.nvars, -1);
  for (int v = 0; v < th.nvars; v++)
    if (g.killed[(size_t)v] < 0) {
      free_index[(size_t)v] = (int)g.letter_of_var.size();
      g.letter_of_var.push_back(v);
    }
  g.nvars = (int)g.letter_of_var.size();
  gr.killed = &g.killed;
  gr.free_index = &free_index;
  std::vector<int> ax;
  for (auto& a : th.axioms) ax.push_back(gr.go(*a));
  g.root = g.dag.mk_and(ax);
  return g;
}

}  // namespace fbg
