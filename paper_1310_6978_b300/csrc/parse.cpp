// parse.cpp -- formula text -> Theory (declarations + axiom syntax trees).
//
// The language follows the script language of Sec. 4.2: Python operators
// ~ & ^ | for negation, conjunction, symmetric difference and disjunction,
// bounded quantifiers A[..] / E[..] over the sets S = range(k),
// S2 = perm(range(k),2) and S3 = perm(range(k),3), quantifiers separated by
// '.', labels "e1 = ..." as in the BAequ4 example of Sec. 5.1.  Added here:
// '->' and '<->', guards "A[a,b:S | a<b]", and 'var' / 'const' declarations
// that fix the letters of the set P of Sec. 3.1 and their numbering, and
// 'fun' declarations of function symbols (letters p_{Fa..b}, named F(a..,b))
// with terms F(t,..) and equations t = u / t != u as atomic formulas.
#include <cctype>
#include <cstring>

#include "fbg_internal.hpp"

namespace fbg {
namespace {

enum Tok { T_END, T_NAME, T_NUM, T_SYM };

struct Token {
  Tok kind;
  std::string text;
};

std::vector<Token> tokenize(const std::string& line, int lineno) {
  static const char* syms[] = {"<->", "->", "<=", ">=", "==", "!=", "(", ")", "[", "]", ",", ":", ".",
                               "|", "&", "^", "~", "<", ">", "="};
  std::vector<Token> out;
  size_t i = 0;
  while (i < line.size()) {
    char c = line[i];
    if (c == '#') break;
    if (c == ' ' || c == '\t' || c == '\r') { i++; continue; }
    if (std::isalpha((unsigned char)c) || c == '_') {
      size_t j = i;
      while (j < line.size() && (std::isalnum((unsigned char)line[j]) || line[j] == '_')) j++;
      out.push_back({T_NAME, line.substr(i, j - i)});
      i = j;
      continue;
    }
    if (std::isdigit((unsigned char)c)) {
      size_t j = i;
      while (j < line.size() && std::isdigit((unsigned char)line[j])) j++;
      out.push_back({T_NUM, line.substr(i, j - i)});
      i = j;
      continue;
    }
    bool hit = false;
    for (const char* s : syms) {
      size_t n = std::strlen(s);
      if (line.compare(i, n, s) == 0) {
        out.push_back({T_SYM, s});
        i += n;
        hit = true;
        break;
      }
    }
    if (!hit) throw CompileError{"line " + std::to_string(lineno) + ": unexpected character '" + std::string(1, c) + "'"};
  }
  out.push_back({T_END, ""});
  return out;
}

class LineParser {
 public:
  LineParser(Theory& th, std::vector<Token> toks, int lineno) : th_(th), t_(std::move(toks)), line_(lineno) {}

  [[noreturn]] void fail(const std::string& m) { throw CompileError{"line " + std::to_string(line_) + ": " + m}; }
  const Token& cur() const { return t_[p_]; }
  bool is_sym(const char* s) const { return cur().kind == T_SYM && cur().text == s; }
  bool take(const char* s) {
    if (is_sym(s)) { p_++; return true; }
    return false;
  }
  void need(const char* s) {
    if (!take(s)) fail(std::string("expected '") + s + "'");
  }
  std::string name() {
    if (cur().kind != T_NAME) fail("expected a name");
    return t_[p_++].text;
  }
  bool at_end() const { return cur().kind == T_END; }

  void declaration(bool is_const, bool is_fun = false) {
    Family f;
    f.name = name();
    for (auto& g : th_.fams)
      if (g.name == f.name) fail("name declared twice: " + f.name);
    if (take("(")) {
      for (;;) {
        if (name() != "S") fail("declared positions range over S");
        f.arity++;
        f.lt.push_back(false);
        if (take(",")) continue;
        if (!is_fun && take("<")) { f.lt.back() = true; continue; }
        break;
      }
      need(")");
    }
    if (is_fun) {   // the value position
      f.arity++;
      f.lt.push_back(false);
      f.is_fun = true;
    }
    if (f.arity > 4) fail("arity above 4");
    long total = 1;
    for (int i = 0; i < f.arity; i++) total *= th_.k;
    if (total > (1L << 20)) fail("family too large");
    f.rank.assign((size_t)total, -1);
    int rk = 0;
    for (long lin = 0; lin < total; lin++) {
      // decode lin into a tuple, most significant position first
      std::vector<int> tup(f.arity);
      long x = lin;
      for (int q = f.arity - 1; q >= 0; q--) { tup[q] = (int)(x % th_.k); x /= th_.k; }
      bool ok = true;
      for (int q = 0; q + 1 < f.arity; q++)
        if (f.lt[q] && !(tup[q] < tup[q + 1])) ok = false;
      if (ok) f.rank[(size_t)lin] = rk++;
    }
    f.count = rk;
    f.is_const = is_const;
    if (is_const) {
      for (int q = 0; q + 1 < f.arity; q++)
        if (f.lt[q]) fail("constants use full tuples");
      need("=");
      std::string bits;
      while (cur().kind == T_NUM) bits += t_[p_++].text;
      if ((long)bits.size() != total) fail("constant '" + f.name + "' needs " + std::to_string(total) + " bits");
      for (char c : bits) {
        if (c != '0' && c != '1') fail("constant bits are 0 or 1");
        f.bits.push_back((uint8_t)(c - '0'));
      }
    } else {
      f.first_id = th_.nvars;
      if (th_.nvars + f.count > 4096) fail("more than 4096 declared letters");
      th_.nvars += f.count;
      for (long lin = 0; lin < total; lin++) {
        if (f.rank[(size_t)lin] < 0) continue;
        std::string nm = f.name;
        if (f.arity) {
          nm += "(";
          long x = lin;
          std::vector<int> tup(f.arity);
          for (int q = f.arity - 1; q >= 0; q--) { tup[q] = (int)(x % th_.k); x /= th_.k; }
          for (int q = 0; q < f.arity; q++) nm += (q ? "," : "") + std::to_string(tup[q]);
          nm += ")";
        }
        th_.var_names.push_back(nm);
      }
    }
    th_.fams.push_back(std::move(f));
  }

  IndexTerm index_term() {
    IndexTerm t;
    if (cur().kind == T_NUM) {
      t.slot = -1;
      t.value = std::stoi(t_[p_++].text);
      return t;
    }
    std::string nm = name();
    for (int i = (int)bound_.size() - 1; i >= 0; i--)
      if (bound_[i] == nm) { t.slot = i; return t; }
    fail("unbound index '" + nm + "'");
  }

  int bound_slot(const std::string& nm) const {
    for (int i = (int)bound_.size() - 1; i >= 0; i--)
      if (bound_[i] == nm) return i;
    return -1;
  }
  int family_of(const std::string& nm) const {
    for (int i = 0; i < (int)th_.fams.size(); i++)
      if (th_.fams[i].name == nm) return i;
    return -1;
  }

  // numeral | bound name | F(term, ..) for a function symbol F
  Term term() {
    Term t;
    if (cur().kind == T_NAME && bound_slot(cur().text) < 0) {
      int f = family_of(cur().text);
      if (f >= 0) {
        const Family& F = th_.fams[(size_t)f];
        if (!F.is_fun) fail("a relation symbol is not a term");
        p_++;
        t.family = f;
        if (F.arity > 1) {
          need("(");
          do t.args.push_back(term()); while (take(","));
          need(")");
        }
        if ((int)t.args.size() != F.arity - 1) fail("'" + F.name + "' takes " + std::to_string(F.arity - 1) + " arguments");
        return t;
      }
    }
    t.ix = index_term();
    return t;
  }

  std::unique_ptr<Ast> equation() {
    auto e = std::make_unique<Ast>();
    e->kind = Ast::Eq;
    e->lhs = term();
    bool neg = false;
    if (take("!=")) neg = true;
    else need("=");
    e->rhs = term();
    if (!neg) return e;
    auto n = std::make_unique<Ast>();
    n->kind = Ast::Not;
    n->a = std::move(e);
    return n;
  }

  bool at_equation_sign(size_t q) const {
    return t_[q].kind == T_SYM && (t_[q].text == "=" || t_[q].text == "!=");
  }

  std::unique_ptr<Ast> quantifier(bool forall) {
    auto q = std::make_unique<Ast>();
    q->kind = forall ? Ast::Forall : Ast::Exists;
    std::vector<std::string> names;
    do names.push_back(name()); while (take(","));
    need(":");
    std::string set = name();
    if (set == "S") q->distinct = false;
    else if (set == "S2" || set == "S3") {
      q->distinct = true;
      if ((int)names.size() != set[1] - '0') fail(set + " binds exactly " + set.substr(1) + " names");
    } else fail("unknown set '" + set + "'");
    if (names.size() > 8) fail("too many bound names");
    q->first_slot = (int)bound_.size();
    q->nbound = (int)names.size();
    for (auto& s : names) bound_.push_back(s);
    if (take("|")) {
      do {
        Guard g;
        g.l = index_term();
        static const char* ops[] = {"<", "<=", ">", ">=", "==", "!="};
        int op = -1;
        for (int i = 0; i < 6; i++)
          if (is_sym(ops[i])) op = i;
        if (op < 0) fail("expected a comparison");
        p_++;
        g.op = op;
        g.r = index_term();
        q->guards.push_back(g);
      } while (take(",") || take("&"));
    }
    need("]");
    take(".");
    q->a = unary();
    bound_.resize((size_t)q->first_slot);
    return q;
  }

  std::unique_ptr<Ast> primary() {
    if (take("(")) {
      auto e = formula();
      need(")");
      return e;
    }
    if (cur().kind == T_NUM) {
      if (at_equation_sign(p_ + 1)) return equation();
      std::string s = t_[p_++].text;
      if (s != "0" && s != "1") fail("constants are 0 or 1");
      auto e = std::make_unique<Ast>();
      e->kind = Ast::Const;
      e->value = s[0] - '0';
      return e;
    }
    if (cur().kind == T_NAME) {
      const std::string& nm0 = cur().text;
      if ((nm0 == "A" || nm0 == "E") && t_[p_ + 1].kind == T_SYM && t_[p_ + 1].text == "[") {
        p_ += 2;
        return quantifier(nm0 == "A");
      }
      int f0 = family_of(nm0);
      if (bound_slot(nm0) >= 0 || (f0 >= 0 && th_.fams[(size_t)f0].is_fun)) return equation();
    }
    std::string nm = name();
    int fam = family_of(nm);
    if (fam < 0) fail("undeclared name '" + nm + "'");
    auto e = std::make_unique<Ast>();
    e->kind = Ast::Atom;
    e->family = fam;
    const Family& F = th_.fams[(size_t)fam];
    bool any_fun = false;
    std::vector<Term> args;
    if (take("(")) {
      do {
        args.push_back(term());
        if (args.back().family >= 0) any_fun = true;
        e->idx.push_back(args.back().ix);
      } while (take(","));
      need(")");
    }
    if ((int)args.size() != F.arity) fail("'" + nm + "' takes " + std::to_string(F.arity) + " indices");
    if (any_fun) {
      for (bool l : F.lt)
        if (l) fail("function terms in a family declared with '<'");
      e->targs = std::move(args);
    }
    return e;
  }

  std::unique_ptr<Ast> unary() {
    if (take("~")) {
      auto e = std::make_unique<Ast>();
      e->kind = Ast::Not;
      e->a = unary();
      return e;
    }
    return primary();
  }

  static std::unique_ptr<Ast> join(Ast::Kind k, std::unique_ptr<Ast> a, std::unique_ptr<Ast> b) {
    auto e = std::make_unique<Ast>();
    e->kind = k;
    e->a = std::move(a);
    e->b = std::move(b);
    return e;
  }

  // precedence climbing, loosest first: <->, -> (right), |, ^, &
  std::unique_ptr<Ast> level_and() {
    auto l = unary();
    while (take("&")) l = join(Ast::And, std::move(l), unary());
    return l;
  }
  std::unique_ptr<Ast> level_xor() {
    auto l = level_and();
    while (take("^")) l = join(Ast::Xor, std::move(l), level_and());
    return l;
  }
  std::unique_ptr<Ast> level_or() {
    auto l = level_xor();
    while (take("|")) l = join(Ast::Or, std::move(l), level_xor());
    return l;
  }
  std::unique_ptr<Ast> level_imp() {
    auto l = level_or();
    if (take("->")) return join(Ast::Imp, std::move(l), level_imp());
    return l;
  }
  std::unique_ptr<Ast> formula() {
    auto l = level_imp();
    while (take("<->")) l = join(Ast::Iff, std::move(l), level_imp());
    return l;
  }

  void line() {
    if (at_end()) return;
    if (cur().kind == T_NAME && (cur().text == "var" || cur().text == "const" || cur().text == "fun") &&
        t_[p_ + 1].kind == T_NAME) {
      bool c = cur().text == "const", fn = cur().text == "fun";
      p_++;
      if (c) declaration(true);
      else {
        do declaration(false, fn); while (take(","));
      }
    } else if (cur().kind == T_NAME && cur().text == "assume" && t_[p_ + 1].kind != T_END &&
               !(t_[p_ + 1].kind == T_SYM && t_[p_ + 1].text != "(" && t_[p_ + 1].text != "~")) {
      p_++;
      th_.assumes.push_back(formula());
    } else {
      // a label, unless the name is a declared symbol (then it is an equation)
      if (cur().kind == T_NAME && t_[p_ + 1].kind == T_SYM && t_[p_ + 1].text == "=" && family_of(cur().text) < 0)
        p_ += 2;
      th_.axioms.push_back(formula());
    }
    if (!at_end()) fail("unexpected '" + cur().text + "'");
  }

 private:
  Theory& th_;
  std::vector<Token> t_;
  size_t p_ = 0;
  int line_;
  std::vector<std::string> bound_;
};

}  // namespace

Theory parse_theory(const std::string& text, int k) {
  if (k < 1 || k > 64) throw CompileError{"domain size must be 1..64"};
  Theory th;
  th.k = k;
  size_t start = 0;
  int lineno = 1;
  while (start <= text.size()) {
    size_t nl = text.find('\n', start);
    std::string ln = text.substr(start, nl == std::string::npos ? std::string::npos : nl - start);
    LineParser lp(th, tokenize(ln, lineno), lineno);
    lp.line();
    if (nl == std::string::npos) break;
    start = nl + 1;
    lineno++;
  }
  return th;
}

}  // namespace fbg
