// ground.cpp -- the translation * of Sec. 3.1 into a hash-consed Boolean DAG.
//
// R(a_1..a_k)* is the letter q_{R a_1..a_k}; forall x phi is the conjunction
// of phi(a) over the domain, exists the disjunction; ~ & | commute with *.
// '^' is the symmetric difference of Sec. 4.2.  The DAG removes the
// constants 0 and 1 as it is built (the Reduction submodule of Sec. 4.1) and
// shares equal subterms (common-subexpression elimination).
//
// Function symbols follow the rules of * for terms: (F(a..) = b)* is the
// letter p_{Fa..b}; (F(t_1..t_m) = b)* is the conjunction over value tuples
// (b_1..b_m) of ((t_1 = b_1)* & .. -> p_{Fb_1..b_m b}); R(t_1..t_m)* is the
// same with q_{Rb_1..b_m} as consequent; (t = u)* is the conjunction over b
// of ((t = b)* -> (u = b)*).  These are exact on valuations where every
// function symbol has exactly one value per argument tuple, so that
// condition is added as conjuncts: at least one value, and no two.
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

  int in_domain(int v, const std::string& where) const {
    if (v < 0 || v >= th.k) throw CompileError{"index out of the domain in '" + where + "'"};
    return v;
  }

  // the letter of family f at the tuple of domain elements tup
  int letter(const Family& f, const std::vector<int>& tup) {
    long lin = 0;
    for (int v : tup) lin = lin * th.k + in_domain(v, f.name);
    if (f.is_const) return f.bits[(size_t)lin] ? 1 : 0;
    int rk = f.rank[(size_t)lin];
    if (rk < 0) throw CompileError{"'" + f.name + "' applied to a tuple outside its declaration"};
    int id = f.first_id + rk;
    if (killed && (*killed)[(size_t)id] >= 0) return (*killed)[(size_t)id] ? 1 : 0;
    return dag.var(free_index ? (*free_index)[(size_t)id] : id);
  }

  int atom(const Ast& e) {
    const Family& f = th.fams[(size_t)e.family];
    if (e.targs.empty()) {
      std::vector<int> tup;
      for (auto& t : e.idx) tup.push_back(idx(t));
      return letter(f, tup);
    }
    return applied(f, e.targs, -1);
  }

  // Sum over the values of the function-term arguments of F(args..) (plain
  // arguments keep their one value): the conjunction of
  // ((t_i = b_i)* & .. -> letter(F, b.., [b])).  b < 0: a relation atom.
  int applied(const Family& f, const std::vector<Term>& args, int b) {
    std::vector<int> tup(args.size() + (b >= 0 ? 1 : 0), 0);
    std::vector<int> fun_pos;
    for (size_t i = 0; i < args.size(); i++) {
      if (args[i].family < 0) tup[i] = in_domain(idx(args[i].ix), f.name);
      else fun_pos.push_back((int)i);
    }
    if (b >= 0) tup.back() = b;
    std::vector<int> parts;
    std::vector<int> vals(fun_pos.size(), 0);
    for (;;) {
      std::vector<int> ante;
      for (size_t q = 0; q < fun_pos.size(); q++) {
        tup[(size_t)fun_pos[q]] = vals[q];
        ante.push_back(eq_value(args[(size_t)fun_pos[q]], vals[q]));
      }
      parts.push_back(dag.mk_or({dag.mk_not(dag.mk_and(ante)), letter(f, tup)}));
      int p = (int)vals.size() - 1;
      while (p >= 0 && ++vals[(size_t)p] == th.k) vals[(size_t)p--] = 0;
      if (p < 0) break;
    }
    return dag.mk_and(parts);
  }

  // (t = b)* for the domain element b
  int eq_value(const Term& t, int b) {
    if (t.family < 0) return in_domain(idx(t.ix), "=") == b ? 1 : 0;
    return applied(th.fams[(size_t)t.family], t.args, b);
  }

  int equation(const Ast& e) {
    const Term &l = e.lhs, &r = e.rhs;
    if (l.family < 0 && r.family < 0) return in_domain(idx(l.ix), "=") == in_domain(idx(r.ix), "=") ? 1 : 0;
    if (l.family < 0) return eq_value(r, in_domain(idx(l.ix), "="));
    if (r.family < 0) return eq_value(l, in_domain(idx(r.ix), "="));
    std::vector<int> parts;
    for (int b = 0; b < th.k; b++) parts.push_back(dag.mk_or({dag.mk_not(eq_value(l, b)), eq_value(r, b)}));
    return dag.mk_and(parts);
  }

  // every function symbol takes exactly one value at every argument tuple
  void functional(std::vector<int>& out) {
    for (const Family& f : th.fams) {
      if (!f.is_fun) continue;
      const int m = f.arity - 1;
      std::vector<int> tup((size_t)f.arity, 0);
      for (;;) {
        std::vector<int> vals;
        for (int b = 0; b < th.k; b++) {
          tup[(size_t)m] = b;
          vals.push_back(letter(f, tup));
        }
        out.push_back(dag.mk_or(vals));
        for (int b = 0; b < th.k; b++)
          for (int c = b + 1; c < th.k; c++) out.push_back(dag.mk_not(dag.mk_and({vals[(size_t)b], vals[(size_t)c]})));
        int p = m - 1;
        while (p >= 0 && ++tup[(size_t)p] == th.k) tup[(size_t)p--] = 0;
        if (p < 0) break;
      }
    }
  }

  // an assume line: a conjunction of literals, possibly under universal
  // quantifiers; each literal fixes its letter, later ones replacing earlier
  void assume(const Ast& e, bool value, std::vector<int>& fixed) {
    switch (e.kind) {
      case Ast::Const:
        if (e.value == 1 && value) return;
        break;
      case Ast::Eq: {
        // F(a..) = b with plain a.., b: p_{Fa..b} := value; when true, the
        // other values of F at a.. are 0
        const Term& app = e.lhs.family >= 0 ? e.lhs : e.rhs;
        const Term& val = e.lhs.family >= 0 ? e.rhs : e.lhs;
        if (app.family < 0 || val.family >= 0) break;
        const Family& f = th.fams[(size_t)app.family];
        long lin = 0;
        bool plain = true;
        for (auto& t : app.args) {
          if (t.family >= 0) { plain = false; break; }
          int v = idx(t.ix);
          if (v < 0 || v >= th.k) throw CompileError{"index out of the domain in an assume line"};
          lin = lin * th.k + v;
        }
        if (!plain) break;
        int b = idx(val.ix);
        if (b < 0 || b >= th.k) throw CompileError{"index out of the domain in an assume line"};
        int base = f.first_id + (int)(lin * th.k);
        if (value)
          for (int u = 0; u < th.k; u++) fixed[(size_t)(base + u)] = u == b ? 1 : 0;
        else
          fixed[(size_t)(base + b)] = 0;
        return;
      }
      case Ast::Atom: {
        const Family& f = th.fams[(size_t)e.family];
        if (f.is_const || !e.targs.empty()) break;
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
        if (e.a->kind != Ast::Atom && e.a->kind != Ast::Eq) break;
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
      case Ast::Eq: return equation(e);
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
  if (g.nvars > 64) throw CompileError{"more than 64 free variables"};
  gr.killed = &g.killed;
  gr.free_index = &free_index;
  std::vector<int> ax;
  gr.functional(ax);
  for (auto& a : th.axioms) ax.push_back(gr.go(*a));
  g.root = g.dag.mk_and(ax);
  return g;
}

}  // namespace fbg
