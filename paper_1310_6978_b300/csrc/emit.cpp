// emit.cpp -- code generation from a LUT program:
//   * CUDA source of a straight-line kernel specialised to one formula
//     (compiled by NVRTC for sm_103a), count or truth-table mode;
//   * bytecode, constant table and slot allocation for the interpreter.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <sstream>
#include <unordered_map>
#include <unordered_set>

#include "emit.hpp"

namespace fbg {

// ---------------------------------------------------------------- NVRTC --

namespace {

std::string hex32(uint32_t v) {
  char b[16];
  std::snprintf(b, sizeof b, "0x%08xu", v);
  return b;
}

// One 32-bit register of a LUT value after folding: a constant, or a
// reference to an emitted register / generator word, possibly negated
// (negations are absorbed into the consumers' truth tables).
struct Sym {
  bool is_const = true;
  uint32_t c = 0;
  std::string name;
  bool neg = false;
  // provably the same in every lane: built only from constants, unit letters
  // and loop counters (the compiler may run such lop3 on the uniform datapath)
  bool uni = true;
  bool operator==(const Sym& o) const {
    return is_const == o.is_const && (is_const ? c == o.c : (name == o.name && neg == o.neg));
  }
};

// The innermost loop level is emitted unrolled when it has at most 5 bits.
static bool innermost_unrolled(const Layout& L) { return L.nlevels() > 2 && L.loop_bits.back() <= 5; }

}  // namespace

int top_loop_split_bits(const Layout& L) {
  if (L.nlevels() <= 2) return 0;
  if (L.nlevels() == 3 && innermost_unrolled(L)) return 0;   // the first loop level is the unrolled one
  return std::min(L.loop_bits[0], 4);
}

namespace {

// Source generator.  Every LUT register is folded: all-zero/all-one inputs
// fix their bit, negated inputs flip, repeated inputs merge; a function of at
// most one input becomes a constant or an alias, identical operations inside
// one scope share a register, and what remains is one lop3.b32.  The
// innermost loop level is unrolled: in each of its 2^b copies the level's
// generator words are constants, so the copy is folded further.
class SrcGen {
 public:
  // counters: count level executions (lvl[]) for fbg_exec_stats; a kernel
  // built without them spends no instructions or registers on them
  explicit SrcGen(const LutProgram& prog, bool counters = true, int popc_cost = 4)
      : split_bits(top_loop_split_bits(prog.layout)), p(prog), L(prog.layout), nreg(1 << prog.layout.r),
        nl(prog.layout.nlevels()), counters_(counters) {
    popc_cost_ = popc_cost;
    if (innermost_unrolled(L)) {
      unroll_lv = nl - 1;
      unroll_bits = L.loop_bits.back();
      unroll_base = L.loop_pos(nl - 3);
    }
    ops.assign((size_t)nl, 0);
    uops.assign((size_t)nl, 0);
    fold_base();
    if (unroll_lv >= 0) fold_unrolled();
  }

  std::vector<long long> ops;   // lop3.b32 per thread per execution of each level (lane-varying)
  std::vector<long long> uops;  // warp-uniform lop3 per warp per execution of each level
  int unroll_lv = -1;
  const int split_bits;   // pieces of an item: up to 2^split_bits over the first loop level

  std::string generate(int mode, int block, int minb);
  std::string unit_fn_count(const std::string& fname);
  std::string unit_fn_table(const std::string& fname);
  std::string unit_fn_enum(const std::string& fname);

 private:
  const LutProgram& p;
  const Layout& L;
  int nreg, nl;
  bool counters_;
  int unroll_bits = 0, unroll_base = 0;
  std::vector<std::vector<Sym>> sym;                  // [lut][s], levels other than unroll_lv
  std::vector<std::vector<std::string>> code;         // real lop3 calls of those
  std::vector<Sym> usym;   // [(copy * luts of the level + lut - first) * nreg + s]
  size_t ulevel_luts = 0;
  std::vector<std::vector<std::string>> ustmt;        // [copy] statements
  std::vector<std::vector<std::string>> ustmt_name;   // [copy] the value each statement defines
  // every lop3 call emitted by folding: its name, the values it reads, its
  // level and whether it is warp-uniform; live_ holds those the kernel needs
  struct CallInfo {
    std::vector<std::string> deps;
    int level = 0;
    bool uni = false;
    int copy = -1;                 // copy of the unrolled level, or -1
    int tt = 0;                    // lop3 immLut over args (arg 0 = bit 2 of the index)
    std::string args[3];           // operand expressions: names or 32-bit immediates
  };
  static std::string call_text(const CallInfo& ci) {
    return "fbg_lop3<" + std::to_string(ci.tt) + ">(" + ci.args[0] + ", " + ci.args[1] + ", " + ci.args[2] + ")";
  }
  bool merged_ = false;
  std::unordered_map<std::string, CallInfo> calls_;
  std::unordered_set<std::string> live_;
  bool is_live(const std::string& name) const { return live_.count(name) != 0; }
  std::ostringstream o;

  bool in_unrolled(int lut) const { return unroll_lv >= 0 && p.luts[(size_t)lut].level == unroll_lv; }

  // Counting the result words of one innermost execution.  POPC issues on
  // the XU pipe at a quarter of the rate of lop3 on the ALU pipe; a full
  // adder (xor3 and majority: two lop3) turns three words of one weight into
  // one word of that weight and one of twice the weight, which trades one
  // POPC for two lop3.  The accumulators ucnt, ucnt2, ucnt4, ucnt8 hold the
  // popcounts of words of weight 1, 2, 4, 8.
  struct CountState {
    std::vector<std::string> pend[4];
    int fa_left = 0;
  };
  int fa_id_ = 0;

  // lanes beyond the valid range of a small program must not count; with
  // all 32 lanes in use and n >= 5 every bit of every word is an assignment
  bool need_thread_mask() const { return L.lane_bits < 5 || valid_mask() != 0xFFFFFFFFu; }

  static std::string acc_name(int k) { return k == 0 ? "ucnt" : "ucnt" + std::to_string(1 << k); }

  // full adders per innermost execution: balance the ALU work (A lop3 and
  // adds, plus two lop3 per full adder) against the POPC work of the W
  // words, a POPC costing `cost` lop3 slots (4: the XU pipe at a quarter of
  // the lop3 rate); each full adder saves one POPC
  int popc_cost_ = 4;
  int full_adder_budget(int W, long long A) const {
    const long long c = popc_cost_;
    long long f = (c * W - A + (c + 2) / 2) / (c + 2);
    if (f < 0) f = 0;
    if (f > W / 2) f = W / 2;
    return (int)f;
  }

  void count_reduce(CountState& cs, const std::string& ind, bool last) {
    for (;;) {
      int k = -1;
      if (cs.fa_left > 0)
        for (int t = 0; t < 3 && k < 0; t++)
          if (cs.pend[t].size() >= 3) k = t;
      if (k < 0) break;
      auto& v = cs.pend[k];
      std::string a = v[v.size() - 3], b = v[v.size() - 2], c = v[v.size() - 1];
      v.resize(v.size() - 3);
      std::string sn = "fs" + std::to_string(fa_id_), cn = "fc" + std::to_string(fa_id_);
      fa_id_++;
      o << ind << "const fbg_u32 " << sn << " = fbg_lop3<0x96>(" << a << ", " << b << ", " << c << ");\n";
      o << ind << "const fbg_u32 " << cn << " = fbg_lop3<0xe8>(" << a << ", " << b << ", " << c << ");\n";
      v.push_back(sn);
      cs.pend[k + 1].push_back(cn);
      cs.fa_left--;
    }
    if (last || cs.fa_left == 0) {
      for (int k = 0; k < 4; k++) {
        for (auto& e : cs.pend[k])
          o << ind << acc_name(k) << " = fbg_madd(" << acc_name(k) << ", __popc(" << e << "), one);\n";
        cs.pend[k].clear();
      }
    }
  }

  // the count of one innermost execution: words[c] are the result words of
  // copy c (one copy when the innermost level is not unrolled), emitted after
  // that copy's statements
  void emit_counts(const std::vector<std::vector<std::string>>* stmts, const std::vector<std::vector<Sym>>& words,
                   long long alu_ops, const std::string& ind) {
    const bool masked = need_thread_mask();
    int W = 0;
    for (auto& ws : words)
      for (const Sym& w : ws) W += w.is_const ? 0 : 1;
    CountState cs;
    cs.fa_left = masked ? 0 : full_adder_budget(W, alu_ops + W / 2 + 4);
    for (size_t c = 0; c < words.size(); c++) {
      if (stmts)
        for (auto& st : (*stmts)[c]) o << ind << st << "\n";
      for (const Sym& w : words[c]) {
        if (masked) {
          o << ind << "ucnt += __popc(" << expr(w) << " & tm);\n";
        } else if (w.is_const) {
          if (w.c) o << ind << "ucnt += " << __builtin_popcount(w.c) << "u;\n";
        } else {
          cs.pend[0].push_back(expr(w));
        }
      }
      count_reduce(cs, ind, c + 1 == words.size());
    }
  }

  Sym operand_sym(const Val& v, int s, int copy) const {
    Sym x;
    if (v.kind == V_CONST) {
      x.c = p.consts[(size_t)v.id].w[(size_t)s];
    } else if (v.kind == V_VAR) {
      if (copy >= 0 && L.level_of_pos(v.id) == unroll_lv) {
        x.c = ((copy >> (v.id - unroll_base)) & 1) ? 0xFFFFFFFFu : 0u;
      } else {
        x.is_const = false;
        x.name = "V" + std::to_string(v.id);
        // unit and loop letters are the same in every lane of a warp (an
        // item is one unit of one warp; the compiler can keep them in uniform
        // registers); the lane, register and warp bits of a thread are not
        x.uni = L.level_of_pos(v.id) >= 1;
      }
    } else {
      size_t r = (size_t)((uint32_t)s & p.luts[(size_t)v.id].rmask);
      if (copy >= 0 && in_unrolled(v.id))
        x = usym[((size_t)copy * ulevel_luts + (size_t)(v.id - p.levels[(size_t)unroll_lv].lut_begin)) * (size_t)nreg + r];
      else
        x = sym[(size_t)v.id][r];
    }
    return x;
  }

  static std::string expr(const Sym& x) {
    if (x.is_const) return hex32(x.c);
    return x.neg ? "(~" + x.name + ")" : x.name;
  }

  std::string operand(const Val& v, int s, int copy = -1) const { return expr(operand_sym(v, s, copy)); }

  // fold one LUT register; *call receives the lop3 call when one is needed
  using CseMap = std::unordered_map<std::string, std::string>;

  // the register name of LUT i, register s (copy c of the unrolled level, or c < 0)
  static std::string fold_name(int i, int s, int c) {
    std::string nm = "L" + std::to_string(i) + "_" + std::to_string(s);
    if (c >= 0) nm += "_u" + std::to_string(c);
    return nm;
  }

  // fold register s of LUT i; the name is made only when a new lop3 is needed
  Sym fold_one(int i, int s, int copy, CseMap& cse, std::string* call) {
    const Lut& lu = p.luts[(size_t)i];
    call->clear();
    Sym in[3];
    for (int k = 0; k < 3; k++) in[k] = operand_sym(lu.in[k], s, copy);
    uint8_t f[8];
    for (int m = 0; m < 8; m++) f[m] = (uint8_t)((lu.tt >> m) & 1);
    int fixed[3] = {-1, -1, -1};
    for (int k = 0; k < 3; k++) {
      if (in[k].is_const && (in[k].c == 0u || in[k].c == 0xFFFFFFFFu)) fixed[k] = in[k].c ? 1 : 0;
      if (!in[k].is_const && in[k].neg) {
        uint8_t g[8];
        for (int m = 0; m < 8; m++) g[m] = f[m ^ (4 >> k)];
        std::memcpy(f, g, 8);
        in[k].neg = false;
      }
    }
    Sym fs[3];
    unsigned kf = 0;
    int map[3] = {-1, -1, -1};
    for (int k = 0; k < 3; k++) {
      if (fixed[k] >= 0) continue;
      for (unsigned t = 0; t < kf; t++)
        if (fs[t] == in[k]) map[k] = (int)t;
      if (map[k] < 0) {
        map[k] = (int)kf;
        fs[kf++] = in[k];
      }
    }
    uint8_t g[8];
    for (unsigned a = 0; a < (1u << kf); a++) {
      int bit[3];
      for (int k = 0; k < 3; k++) bit[k] = fixed[k] >= 0 ? fixed[k] : (int)((a >> map[k]) & 1u);
      g[a] = f[(bit[0] << 2) | (bit[1] << 1) | bit[2]];
    }
    for (int t = (int)kf - 1; t >= 0; t--) {   // drop inputs the function ignores
      bool dep = false;
      for (unsigned a = 0; a < (1u << kf); a++)
        if (g[a] != g[a ^ (1u << t)]) dep = true;
      if (dep) continue;
      uint8_t h[8];
      for (unsigned a = 0; a < (1u << (kf - 1)); a++) {
        unsigned lo = a & ((1u << t) - 1u), hi = a >> t;
        h[a] = g[lo | (hi << (t + 1))];
      }
      for (unsigned q = (unsigned)t; q + 1 < kf; q++) fs[q] = std::move(fs[q + 1]);
      std::memcpy(g, h, sizeof h);
      kf--;
    }
    Sym out;
    bool all_imm = true, uni = true;
    for (unsigned q = 0; q < kf; q++) {
      all_imm &= fs[q].is_const;
      uni &= fs[q].uni;
    }
    if (kf == 0) {
      out.c = g[0] ? 0xFFFFFFFFu : 0u;
    } else if (all_imm) {
      uint32_t v = 0;
      for (int b = 0; b < 32; b++) {
        unsigned a = 0;
        for (unsigned q = 0; q < kf; q++) a |= ((fs[q].c >> b) & 1u) << q;
        v |= (uint32_t)g[a] << b;
      }
      out.c = v;
    } else if (kf == 1 && !fs[0].is_const) {
      out = fs[0];
      out.neg = g[0] == 1;
    } else {
      int tt = 0;
      for (int m = 0; m < 8; m++) {
        unsigned ab[3] = {(unsigned)(m >> 2) & 1u, (unsigned)(m >> 1) & 1u, (unsigned)m & 1u};
        unsigned a = 0;
        for (unsigned q = 0; q < kf; q++) a |= ab[q] << q;
        tt |= g[a] << m;
      }
      std::string c3;
      c3.reserve(64);
      c3 += "fbg_lop3<";
      c3 += std::to_string(tt);
      c3 += ">(";
      c3 += expr(fs[0]);
      c3 += ", ";
      c3 += expr(fs[kf > 1 ? 1 : 0]);
      c3 += ", ";
      c3 += expr(fs[kf > 2 ? 2 : 0]);
      c3 += ")";
      out.is_const = false;
      out.uni = uni;
      auto it = cse.find(c3);
      if (it != cse.end()) {
        out.name = it->second;
      } else {
        const std::string name = fold_name(i, s, copy);
        cse.emplace(c3, name);
        out.name = name;
        *call = c3;
        CallInfo ci;
        for (unsigned q = 0; q < kf; q++)
          if (!fs[q].is_const) ci.deps.push_back(fs[q].name);
        ci.level = copy >= 0 ? unroll_lv : lu.level;
        ci.uni = uni;
        ci.copy = copy;
        ci.tt = tt;
        ci.args[0] = expr(fs[0]);
        ci.args[1] = expr(fs[kf > 1 ? 1 : 0]);
        ci.args[2] = expr(fs[kf > 2 ? 2 : 0]);
        calls_[name] = std::move(ci);
      }
    }
    return out;
  }

  void fold_base() {
    const size_t n = p.luts.size();
    sym.assign(n, {});
    code.assign(n, {});
    CseMap cse;
    int cur = -100;
    for (size_t i = 0; i < n; i++) {
      const Lut& lu = p.luts[i];
      sym[i].assign((size_t)nreg, Sym{});
      code[i].assign((size_t)nreg, "");
      if (lu.level == unroll_lv) continue;
      if (lu.level != cur) {
        cse.clear();
        cur = lu.level;
      }
      for (int s = 0; s < nreg; s++) {
        if (((uint32_t)s & lu.rmask) != (uint32_t)s) continue;
        std::string call;
        sym[i][(size_t)s] = fold_one((int)i, s, -1, cse, &call);
        if (!call.empty()) code[i][(size_t)s] = call;
      }
    }
  }

  void fold_unrolled() {
    const LevelInfo& li = p.levels[(size_t)unroll_lv];
    const int copies = 1 << unroll_bits;
    ulevel_luts = (size_t)(li.lut_end - li.lut_begin);
    usym.assign((size_t)copies * ulevel_luts * (size_t)nreg, Sym{});
    ustmt.assign((size_t)copies, {});
    ustmt_name.assign((size_t)copies, {});
    CseMap cse;   // shared: the copies are one straight-line block
    for (int c = 0; c < copies; c++) {
      for (int i = li.lut_begin; i < li.lut_end; i++) {
        const Lut& lu = p.luts[(size_t)i];
        for (int s = 0; s < nreg; s++) {
          if (((uint32_t)s & lu.rmask) != (uint32_t)s) continue;
          std::string call;
          Sym v = fold_one(i, s, c, cse, &call);
          usym[((size_t)c * ulevel_luts + (size_t)(i - li.lut_begin)) * (size_t)nreg + (size_t)s] = v;
          if (!call.empty()) {
            ustmt[(size_t)c].push_back("const fbg_u32 " + v.name + " = " + call + ";");
            ustmt_name[(size_t)c].push_back(v.name);
          }
        }
      }
    }
  }

  // positions of non-constant variables used by the program, by level
  std::vector<std::vector<int>> used_vars() const {
    std::vector<bool> used((size_t)L.n, false);
    for (const Lut& lu : p.luts)
      for (const Val& v : lu.in)
        if (v.kind == V_VAR) used[(size_t)v.id] = true;
    if (p.out.kind == V_VAR) used[(size_t)p.out.id] = true;
    for (const auto& li : p.levels)
      if (li.has_acc && li.acc.kind == V_VAR) used[(size_t)li.acc.id] = true;
    std::vector<std::vector<int>> byl((size_t)nl);
    for (int pos = 0; pos < L.n; pos++)
      if (used[(size_t)pos]) {
        int lv = L.level_of_pos(pos);
        if (lv >= 0 && lv != unroll_lv) byl[(size_t)lv].push_back(pos);
      }
    return byl;
  }

  static std::string lut_name(int i, int s) { return "L" + std::to_string(i) + "_" + std::to_string(s); }

  // The values the kernel needs: the result words of every copy and the
  // partial conjunctions of the levels whose warp vote is emitted (mode 0:
  // count, 1: table), and all they read.  Calls nothing reads are dead (with
  // pruning off, the level conjunctions feed no vote); they are neither
  // emitted nor counted in ops / uops.
  void mark_live(int mode) {
    mark_live_from_roots(mode);
    merge_chains(mode);
  }

  void mark_live_from_roots(int mode) {
    std::vector<std::string> stack = root_names(mode);
    live_.clear();
    while (!stack.empty()) {
      std::string nm = stack.back();
      stack.pop_back();
      auto it = calls_.find(nm);
      if (it == calls_.end() || live_.count(nm)) continue;
      live_.insert(nm);
      for (auto& d : it->second.deps) stack.push_back(d);
    }
    ops.assign((size_t)nl, 0);
    uops.assign((size_t)nl, 0);
    for (auto& nm : live_) {
      const CallInfo& ci = calls_[nm];
      (ci.uni ? uops : ops)[(size_t)ci.level]++;
    }
  }

  // the statements of the unrolled copies that define live values
  std::vector<std::vector<std::string>> live_ustmt() const {
    std::vector<std::vector<std::string>> out(ustmt.size());
    for (size_t c = 0; c < ustmt.size(); c++)
      for (size_t t = 0; t < ustmt[c].size(); t++)
        if (is_live(ustmt_name[c][t]))
          out[c].push_back("const fbg_u32 " + ustmt_name[c][t] + " = " + call_text(calls_.at(ustmt_name[c][t])) + ";");
    return out;
  }

  // The value names the kernel reads outside lop3 calls: the result words of
  // every copy and the partial conjunctions of the levels whose votes the
  // kernel of `mode` emits (the roots of mark_live).
  std::vector<std::string> root_names(int mode) const {
    const int last = nl - 1;
    std::vector<std::string> r;
    auto root = [&](const Val& v, int copy) {
      for (int s = 0; s < nreg; s++) {
        Sym x = operand_sym(v, s, copy);
        if (!x.is_const) r.push_back(x.name);
      }
    };
    if (unroll_lv >= 0)
      for (int c = 0; c < (1 << unroll_bits); c++) root(p.out, c);
    else
      root(p.out, -1);
    if (p.levels[0].has_acc && (mode == 0 || last > 0)) root(p.levels[0].acc, -1);
    if (nl > 1 && p.levels[1].has_acc && last > 1) root(p.levels[1].acc, -1);
    for (int lv = 2; lv < last; lv++)
      if (lv != unroll_lv && p.levels[(size_t)lv].has_acc) root(p.levels[(size_t)lv].acc, -1);
    return r;
  }

  // Constant folding leaves many lop3 calls with one or two distinct
  // operands (a loop letter of an unrolled copy, a register's constant, a
  // repeated input), so a chain of such calls may fit fewer 3-input LUTs
  // than the mapping before folding found.  A live call Y that is not read
  // outside lop3 calls, whose every reader X is a live call of the same
  // level (and copy), is merged into all its readers when, for each, the
  // operands of X and Y together are at most three: X's truth table is
  // recomputed over them and Y disappears (one lop3 fewer; a reader never
  // grows).  Repeated until no merge applies.  Results are unchanged (each
  // reader computes the same function of the operands).
  static int merged_tt(const CallInfo& X, const CallInfo& Y, const std::string& yn, const std::vector<std::string>& ops) {
    auto val = [&](const std::vector<int>& v, const std::string& a) {
      return v[(size_t)(std::find(ops.begin(), ops.end(), a) - ops.begin())];
    };
    const size_t m = ops.size();
    // slot q < m of the new call holds operand q; slots q >= m repeat
    // operand 0, so only the first m slot bits select the value
    int tt = 0;
    for (int idx = 0; idx < 8; idx++) {
      std::vector<int> v(m, 0);
      for (size_t q = 0; q < m; q++) v[q] = (idx >> (2 - (int)q)) & 1;
      const int ybit = (Y.tt >> ((val(v, Y.args[0]) << 2) | (val(v, Y.args[1]) << 1) | val(v, Y.args[2]))) & 1;
      auto xin = [&](const std::string& a) { return a == yn ? ybit : val(v, a); };
      const int xbit = (X.tt >> ((xin(X.args[0]) << 2) | (xin(X.args[1]) << 1) | xin(X.args[2]))) & 1;
      tt |= xbit << idx;
    }
    return tt;
  }

  static std::vector<std::string> merged_ops(const CallInfo& X, const CallInfo& Y, const std::string& yn) {
    std::vector<std::string> ops;
    auto add = [&](const std::string& a) {
      if (std::find(ops.begin(), ops.end(), a) == ops.end()) ops.push_back(a);
    };
    for (const std::string& a : X.args)
      if (a != yn) add(a);
    for (const std::string& a : Y.args) add(a);
    return ops;
  }

  void merge_chains(int mode) {
    if (merged_) return;
    merged_ = true;
    for (;;) {
      std::unordered_set<std::string> roots;
      for (const std::string& r : root_names(mode)) roots.insert(r);
      // readers of every live call (each reader once)
      std::unordered_map<std::string, std::vector<std::string>> readers;
      std::vector<std::string> order(live_.begin(), live_.end());
      std::sort(order.begin(), order.end());   // a fixed order: the same source on every build
      for (const std::string& nm : order) {
        const CallInfo& ci = calls_.at(nm);
        for (int q = 0; q < 3; q++) {
          const std::string& a = ci.args[q];
          if (calls_.count(a) && (q == 0 || (a != ci.args[0] && (q == 1 || a != ci.args[1]))))
            readers[a].push_back(nm);
        }
      }
      std::unordered_set<std::string> touched, gone;
      bool changed = false;
      for (const std::string& yn : order) {
        if (roots.count(yn) || touched.count(yn)) continue;
        auto rit = readers.find(yn);
        if (rit == readers.end() || rit->second.empty()) continue;
        const CallInfo& Y = calls_.at(yn);
        bool ok = true;
        for (const std::string& xn : rit->second) {
          const CallInfo& X = calls_.at(xn);
          ok = ok && !touched.count(xn) && !gone.count(xn) && X.level == Y.level && X.copy == Y.copy &&
               merged_ops(X, Y, yn).size() <= 3;
        }
        if (!ok) continue;
        for (const std::string& xn : rit->second) {
          CallInfo& X = calls_.at(xn);
          const std::vector<std::string> ops = merged_ops(X, Y, yn);
          CallInfo nx = X;
          nx.tt = merged_tt(X, Y, yn, ops);
          for (int q = 0; q < 3; q++) nx.args[q] = ops[(size_t)q < ops.size() ? (size_t)q : 0];
          nx.deps.clear();
          for (const std::string& a : ops)
            if (a.compare(0, 2, "0x") != 0) nx.deps.push_back(a);
          nx.uni = X.uni && Y.uni;
          X = nx;
          touched.insert(xn);
        }
        touched.insert(yn);
        gone.insert(yn);
        changed = true;
      }
      if (!changed) break;
      // liveness again from the roots: merged-away calls are no longer read
      mark_live_from_roots(mode);
    }
  }

  void declare_level(int lv, const std::string& ind) {
    const LevelInfo& li = p.levels[(size_t)lv];
    for (int i = li.lut_begin; i < li.lut_end; i++)
      for (int s = 0; s < nreg; s++)
        if (!code[(size_t)i][(size_t)s].empty() && is_live(lut_name(i, s)))
          o << ind << "fbg_u32 " << lut_name(i, s) << ";\n";
  }

  void luts(int lv, const std::string& ind) {
    const LevelInfo& li = p.levels[(size_t)lv];
    for (int i = li.lut_begin; i < li.lut_end; i++)
      for (int s = 0; s < nreg; s++)
        if (!code[(size_t)i][(size_t)s].empty() && is_live(lut_name(i, s)))
          o << ind << lut_name(i, s) << " = " << call_text(calls_.at(lut_name(i, s))) << ";\n";
  }

  std::string any_nonzero(const Val& v) const {
    std::string e;
    for (int s = 0; s < nreg; s++) {
      if (!e.empty()) e += " | ";
      e += operand(v, s);
    }
    return "((" + e + ") != 0u)";
  }

  void var_words(const std::vector<int>& vars, const std::string& src, int base, const std::string& ind, bool wide) {
    for (int pos : vars) {
      int b = pos - base;
      if (wide)
        o << ind << "const fbg_u32 V" << pos << " = 0u - (fbg_u32)((" << src << " >> " << b << ") & 1ull);\n";
      else
        o << ind << "const fbg_u32 V" << pos << " = 0u - ((" << src << " >> " << b << ") & 1u);\n";
    }
  }

  uint32_t valid_mask() const {
    if (L.n >= 5) return 0xFFFFFFFFu;
    return (uint32_t)((1ull << (1u << L.n)) - 1ull);
  }

  void store(const std::string& ind, const std::string& T, const std::vector<std::string>& w) {
    if (L.r == 0) {
      o << ind << "reinterpret_cast<fbg_u64*>(table)[0] = (fbg_u64)" << w[0] << ";\n";
    } else if (L.r == 1) {
      o << ind << "reinterpret_cast<uint2*>(table)[(" << T << ") - tile0] = make_uint2(" << w[0] << ", " << w[1] << ");\n";
    } else if (L.r == 2) {
      o << ind << "reinterpret_cast<uint4*>(table)[(" << T << ") - tile0] = make_uint4(" << w[0] << ", " << w[1] << ", "
        << w[2] << ", " << w[3] << ");\n";
    } else {
      for (int q = 0; q < nreg / 4; q++)
        o << ind << "reinterpret_cast<uint4*>(table)[((" << T << ") - tile0) * " << nreg / 4 << " + " << q << "] = make_uint4("
          << w[4 * q] << ", " << w[4 * q + 1] << ", " << w[4 * q + 2] << ", " << w[4 * q + 3] << ");\n";
    }
  }
};

// Per-unit device function of count mode: this thread's number of models over
// the units [u0, u1), the thread taking the lane and warp bits tb; lvl[l]
// counts the executions of level l; when the first loop level is a runtime
// loop (top_loop_split_bits > 0) it runs over [lo2, hi2) only, so that one
// heavy item can be handed out as several pieces.  Keeping the work fetch
// outside this function keeps the control flow the compiler sees simple.
std::string SrcGen::unit_fn_count(const std::string& fname) {
  mark_live(0);
  auto vars = used_vars();
  const int tvalid = 1 << (L.lane_bits + L.warp_bits);
  const int last = nl - 1;
  o << "__device__ __noinline__ fbg_u64 " << fname
    << "(fbg_u64 u0, fbg_u64 u1, fbg_u32 tb, fbg_u64* lvl, fbg_u32 lo2, fbg_u32 hi2) {\n";
  o << "  const fbg_u32 tm = (tb < " << tvalid << "u) ? " << hex32(valid_mask()) << " : 0u;\n";
  // a 1 the compiler cannot see (tb < 2^31 always): count adds become IMAD
  o << "  const fbg_u32 one = (tb >> 31) | 1u;\n";
  if (counters_) {
    o << "  lvl[0]++;\n";
    // level execution counters live in registers during the call
    for (int lv = 1; lv < nl; lv++) o << "  fbg_u32 it" << lv << " = 0;\n";
  }
  var_words(vars[0], "tb", L.first_lane_pos(), "  ", false);
  declare_level(0, "  ");
  luts(0, "  ");
  if (p.levels[0].has_acc)
    o << "  if (!__any_sync(FBG_FULL, " << any_nonzero(p.levels[0].acc) << ")) return 0;\n";
  o << "  fbg_u64 total = 0;\n";
  o << "  for (fbg_u64 u = u0; u < u1; ++u) {\n";
  if (counters_) o << "    it1++;\n";
  var_words(vars[1], "u", L.first_unit_pos(), "    ", true);
  declare_level(1, "    ");
  luts(1, "    ");
  if (p.levels[1].has_acc && last > 1)
    o << "    if (!__any_sync(FBG_FULL, " << any_nonzero(p.levels[1].acc) << ")) continue;\n";
  o << "    fbg_u32 ucnt = 0, ucnt2 = 0, ucnt4 = 0, ucnt8 = 0;\n";
  std::string ind = "    ";
  for (int lv = 2; lv < nl; lv++) {
    if (lv == unroll_lv) break;
    std::string iv = "i" + std::to_string(lv);
    if (lv == 2)
      o << ind << "for (fbg_u32 " << iv << " = lo2; " << iv << " < hi2; ++" << iv << ") {\n";
    else
      o << ind << "for (fbg_u32 " << iv << " = 0; " << iv << " < " << (1u << L.loop_bits[(size_t)(lv - 2)]) << "u; ++" << iv << ") {\n";
    ind += "  ";
    if (counters_) o << ind << "it" << lv << "++;\n";
    var_words(vars[(size_t)lv], iv, L.loop_pos(lv - 2), ind, false);
    declare_level(lv, ind);
    luts(lv, ind);
    if (p.levels[(size_t)lv].has_acc && lv < last)
      o << ind << "if (!__any_sync(FBG_FULL, " << any_nonzero(p.levels[(size_t)lv].acc) << ")) continue;\n";
  }
  if (unroll_lv >= 0) {
    if (counters_) o << ind << "it" << unroll_lv << "++;\n";
    std::vector<std::vector<Sym>> words((size_t)(1 << unroll_bits));
    for (int c = 0; c < (1 << unroll_bits); c++)
      for (int s = 0; s < nreg; s++) words[(size_t)c].push_back(operand_sym(p.out, s, c));
    const std::vector<std::vector<std::string>> lst = live_ustmt();
    emit_counts(&lst, words, ops[(size_t)unroll_lv], ind);
  } else {
    std::vector<std::vector<Sym>> words(1);
    for (int s = 0; s < nreg; s++) words[0].push_back(operand_sym(p.out, s, -1));
    emit_counts(nullptr, words, ops[(size_t)last], ind);
  }
  for (int lv = (unroll_lv >= 0 ? unroll_lv - 1 : last); lv >= 2; lv--) {
    ind.resize(ind.size() - 2);
    o << ind << "}\n";
  }
  o << "    total += (fbg_u64)ucnt + 2ull * ucnt2 + 4ull * ucnt4 + 8ull * ucnt8;\n";
  o << "  }\n";
  if (counters_)
    for (int lv = 1; lv < nl; lv++) o << "  lvl[" << lv << "] += it" << lv << ";\n";
  o << "  return total;\n";
  o << "}\n";
  return o.str();
}

// Per-item device function of enumerate mode (layout of enum_order: the item
// (unit u, warp slice w) is the interval of assignment integers
// [(u << wb | w) << (n - ub - wb), +2^(n - ub - wb)), its loop letters come
// next below the warp slice in the order of the loop nest, then the lane,
// register and in-word bits).  The warp writes the models of the item in
// ascending order from models[base]: per innermost execution (per copy of an
// unrolled level) the lanes' popcounts are scanned across the warp, and each
// lane writes its models at its offset; nothing at or beyond `cap` is
// written, and the item stops once the running offset reaches it.
std::string SrcGen::unit_fn_enum(const std::string& fname) {
  auto vars = used_vars();
  const int tvalid = 1 << (L.lane_bits + L.warp_bits);
  const int last = nl - 1;
  const int wb = L.warp_bits;
  const int lane_mask = (1 << L.lane_bits) - 1;
  o << "__device__ __noinline__ void " << fname
    << "(fbg_u64 u, fbg_u32 tb, fbg_u64 base, fbg_u64* models, fbg_u64 cap, fbg_u64* lvl) {\n";
  o << "  const fbg_u32 tm = (tb < " << tvalid << "u) ? " << hex32(valid_mask()) << " : 0u;\n";
  o << "  const fbg_u32 lane = threadIdx.x & 31u;\n";
  // the assignment integer of this lane's tile at loop coordinates 0
  std::string jt = "((fbg_u64)(tb & " + std::to_string(lane_mask) + "u) << " + std::to_string(5 + L.r) + ")";
  if (wb > 0) jt += " | ((fbg_u64)(tb >> 5) << " + std::to_string(L.n - L.unit_bits - wb) + ")";
  if (L.unit_bits > 0) jt += " | (u << " + std::to_string(L.first_unit_pos()) + ")";
  o << "  const fbg_u64 J0 = " << jt << ";\n";
  o << "  fbg_u64 off = base;\n";
  if (counters_) o << "  lvl[0]++;\n";
  var_words(vars[0], "tb", L.first_lane_pos(), "  ", false);
  declare_level(0, "  ");
  luts(0, "  ");
  if (p.levels[0].has_acc)
    o << "  if (!__any_sync(FBG_FULL, " << any_nonzero(p.levels[0].acc) << ")) return;\n";
  if (counters_) o << "  lvl[1]++;\n";
  var_words(vars[1], "u", L.first_unit_pos(), "  ", true);
  declare_level(1, "  ");
  luts(1, "  ");
  if (p.levels[1].has_acc && last > 1)
    o << "  if (!__any_sync(FBG_FULL, " << any_nonzero(p.levels[1].acc) << ")) return;\n";
  std::string ind = "  ";
  std::string jexpr = "J0";
  for (int lv = 2; lv < nl; lv++) {
    if (lv == unroll_lv) break;
    std::string iv = "i" + std::to_string(lv);
    o << ind << "for (fbg_u32 " << iv << " = 0; " << iv << " < " << (1u << L.loop_bits[(size_t)(lv - 2)]) << "u; ++" << iv << ") {\n";
    ind += "  ";
    if (counters_) o << ind << "lvl[" << lv << "]++;\n";
    var_words(vars[(size_t)lv], iv, L.loop_pos(lv - 2), ind, false);
    declare_level(lv, ind);
    luts(lv, ind);
    if (p.levels[(size_t)lv].has_acc && lv < last)
      o << ind << "if (!__any_sync(FBG_FULL, " << any_nonzero(p.levels[(size_t)lv].acc) << ")) continue;\n";
    jexpr += " | ((fbg_u64)" + iv + " << " + std::to_string(L.loop_pos(lv - 2) - wb) + ")";
  }
  // compaction of one innermost execution (one copy): words w[s] of this lane
  auto compact = [&](const std::vector<std::string>& w, const std::string& jbase, const std::string& in) {
    o << in << "{\n";
    o << in << "  const fbg_u32 ew[" << nreg << "] = {";
    for (int s2 = 0; s2 < nreg; s2++) o << (s2 ? ", " : "") << "(" << w[(size_t)s2] << ") & tm";
    o << "};\n";
    o << in << "  fbg_u32 c = 0;\n";
    o << in << "  #pragma unroll\n";
    o << in << "  for (int s = 0; s < " << nreg << "; s++) c += (fbg_u32)__popc(ew[s]);\n";
    o << in << "  fbg_u32 incl = c;\n";
    o << in << "  #pragma unroll\n";
    o << in << "  for (int d = 1; d < 32; d <<= 1) {\n";
    o << in << "    const fbg_u32 y = __shfl_up_sync(FBG_FULL, incl, d);\n";
    o << in << "    if (lane >= (fbg_u32)d) incl += y;\n";
    o << in << "  }\n";
    o << in << "  const fbg_u32 wtot = __shfl_sync(FBG_FULL, incl, 31);\n";
    o << in << "  fbg_u64 at = off + (incl - c);\n";
    o << in << "  const fbg_u64 J = " << jbase << ";\n";
    o << in << "  for (int s = 0; s < " << nreg << " && at < cap; s++) {\n";
    o << in << "    fbg_u32 x = ew[s];\n";
    o << in << "    while (x && at < cap) {\n";
    o << in << "      const int b = __ffs((int)x) - 1;\n";
    o << in << "      x &= x - 1u;\n";
    o << in << "      models[at++] = J | ((fbg_u64)s << 5) | (fbg_u64)b;\n";
    o << in << "    }\n";
    o << in << "  }\n";
    o << in << "  off += wtot;\n";
    o << in << "}\n";
    o << in << "if (off >= cap) return;\n";
  };
  if (unroll_lv >= 0) {
    if (counters_) o << ind << "lvl[" << unroll_lv << "]++;\n";
    const std::vector<std::vector<std::string>> lst = live_ustmt();
    for (int c = 0; c < (1 << unroll_bits); c++) {
      for (auto& st : lst[(size_t)c]) o << ind << st << "\n";
      std::vector<std::string> w;
      for (int s2 = 0; s2 < nreg; s2++) w.push_back(operand(p.out, s2, c));
      compact(w, jexpr + " | ((fbg_u64)" + std::to_string(c) + "u << " + std::to_string(unroll_base - wb) + ")", ind);
    }
  } else {
    std::vector<std::string> w;
    for (int s2 = 0; s2 < nreg; s2++) w.push_back(operand(p.out, s2));
    compact(w, jexpr, ind);
  }
  for (int lv = (unroll_lv >= 0 ? unroll_lv - 1 : last); lv >= 2; lv--) {
    ind.resize(ind.size() - 2);
    o << ind << "}\n";
  }
  o << "}\n";
  return o.str();
}

// Per-unit device function of truth-table mode: stores every tile of unit u;
// tiles under a level whose partial conjunction is zero store zeros.
std::string SrcGen::unit_fn_table(const std::string& fname) {
  mark_live(1);
  auto vars = used_vars();
  const int tvalid = 1 << (L.lane_bits + L.warp_bits);
  const int last = nl - 1;
  o << "__device__ __noinline__ void " << fname << "(fbg_u64 u, fbg_u32* table, fbg_u64 tile0, fbg_u64* lvl) {\n";
  o << "  const fbg_u32 tb = threadIdx.x;\n";
  o << "  const fbg_u32 tm = (tb < " << tvalid << "u) ? " << hex32(valid_mask()) << " : 0u;\n";
  var_words(vars[0], "tb", L.first_lane_pos(), "  ", false);
  declare_level(0, "  ");
  luts(0, "  ");
  o << "  bool a1 = true;\n";
  if (p.levels[0].has_acc && last > 0) o << "  a1 = __any_sync(FBG_FULL, " << any_nonzero(p.levels[0].acc) << ");\n";
  declare_level(1, "  ");
  var_words(vars[1], "u", L.first_unit_pos(), "  ", true);
  o << "  if (a1) {\n";
  o << "    lvl[1]++;\n";
  luts(1, "    ");
  if (p.levels[1].has_acc && last > 1) o << "    a1 = __any_sync(FBG_FULL, " << any_nonzero(p.levels[1].acc) << ");\n";
  o << "  }\n";
  auto tile_base = [&](int upto) {
    std::string t = "(fbg_u64)tb";
    for (int lv = 2; lv < upto; lv++) t += " | ((fbg_u64)i" + std::to_string(lv) + " << " + std::to_string(L.loop_pos(lv - 2) - 5 - L.r) + ")";
    if (L.unit_bits) t += " | (u << " + std::to_string(L.first_unit_pos() - 5 - L.r) + ")";
    return t;
  };
  std::string ind = "  ";
  int prev = 1;
  for (int lv = 2; lv < nl; lv++) {
    if (lv == unroll_lv) break;
    std::string iv = "i" + std::to_string(lv);
    o << ind << "for (fbg_u32 " << iv << " = 0; " << iv << " < " << (1u << L.loop_bits[(size_t)(lv - 2)]) << "u; ++" << iv << ") {\n";
    ind += "  ";
    o << ind << "bool a" << lv << " = a" << (lv - 1) << ";\n";
    declare_level(lv, ind);
    var_words(vars[(size_t)lv], iv, L.loop_pos(lv - 2), ind, false);
    o << ind << "if (a" << lv << ") {\n";
    o << ind << "  lvl[" << lv << "]++;\n";
    luts(lv, ind + "  ");
    if (p.levels[(size_t)lv].has_acc && lv < last)
      o << ind << "  a" << lv << " = __any_sync(FBG_FULL, " << any_nonzero(p.levels[(size_t)lv].acc) << ");\n";
    o << ind << "}\n";
    prev = lv;
  }
  if (unroll_lv >= 0) {
    const int sh = L.loop_pos(unroll_lv - 2) - 5 - L.r;
    o << ind << "{\n";
    o << ind << "  const fbg_u64 T = " << tile_base(unroll_lv) << ";\n";
    o << ind << "  if (a" << prev << " && tm) {\n";
    o << ind << "    lvl[" << unroll_lv << "]++;\n";
    const std::vector<std::vector<std::string>> lst = live_ustmt();
    for (int c = 0; c < (1 << unroll_bits); c++) {
      for (auto& st : lst[(size_t)c]) o << ind << "    " << st << "\n";
      std::vector<std::string> w;
      for (int s = 0; s < nreg; s++) w.push_back("(" + operand(p.out, s, c) + " & tm)");
      store(ind + "    ", "T | ((fbg_u64)" + std::to_string(c) + "u << " + std::to_string(sh) + ")", w);
    }
    o << ind << "  } else if (tm) {\n";
    o << ind << "    for (fbg_u32 z = 0; z < " << (1u << unroll_bits) << "u; ++z) {\n";
    std::vector<std::string> zw((size_t)nreg, "0u");
    store(ind + "      ", "T | ((fbg_u64)z << " + std::to_string(sh) + ")", zw);
    o << ind << "    }\n";
    o << ind << "  }\n";
    o << ind << "}\n";
  } else {
    o << ind << "const fbg_u32 keep = a" << prev << " ? tm : 0u;\n";
    o << ind << "const fbg_u64 T = " << tile_base(nl) << ";\n";
    std::vector<std::string> w;
    for (int s = 0; s < nreg; s++) w.push_back("(" + operand(p.out, s) + " & keep)");
    o << ind << "if (tm) {\n";
    store(ind + "  ", "T", w);
    o << ind << "}\n";
  }
  for (int lv = (unroll_lv >= 0 ? unroll_lv - 1 : last); lv >= 2; lv--) {
    ind.resize(ind.size() - 2);
    o << ind << "}\n";
  }
  o << "}\n";
  return o.str();
}

// The kernels.  Count mode: the work items are (warp slice w, unit v) pairs
// that a warp pulls by itself, never waiting for the other warps of its
// block; the warp evaluates an item with the warp bits of w.  Without an
// order the items go out w-major (item t of the R = unit_end - unit_begin
// units is w = t / R, v = t % R) in chunks of consecutive units, which one
// call evaluates with its thread-level values computed once; with an order
// (P.unit_perm, longest measured items first) item t is P.unit_perm[t].
// Table mode: a block pulls whole units (its stores are dense and the work
// per unit is even).
std::string SrcGen::generate(int mode, int block, int minb) {
  const char* kname = mode == 0 ? "fbg_jit_count" : mode == 1 ? "fbg_jit_table" : "fbg_jit_enum";
  if (mode == 0 || mode == 2) unit_fn_count("fbg_unit_count");
  else unit_fn_table("fbg_unit_table");
  if (mode == 2) {
    // Enumerate mode, two passes of one kernel over the items t = u << wb | w
    // (ascending t = ascending assignment integers): with P.models null each
    // item's number of models goes to P.unit_counts[t]; with P.models set
    // (P.unit_offsets = the exclusive prefix of those counts) each item
    // writes its models from its offset, skipping items at or past P.cap.
    unit_fn_enum("fbg_unit_enum");
    const int wb = L.warp_bits;
    o << "extern \"C\" __global__ void __launch_bounds__(" << block << ", " << minb << ") " << kname << "(FbgLaunch P) {\n";
    o << "  fbg_u64 lvl[" << nl << "] = {0};\n";
    o << "  const fbg_u32 lane = threadIdx.x & 31u;\n";
    o << "  const fbg_u64 chunk = P.chunk ? P.chunk : 1ull;\n";
    o << "  const fbg_u64 items = (P.unit_end - P.unit_begin) << " << wb << ";\n";
    o << "  const fbg_u32 full2 = " << (split_bits > 0 ? (1u << L.loop_bits[0]) : 0u) << "u;\n";
    o << "  for (;;) {\n";
    o << "    fbg_u64 t = fbg_next_items_warp(P, chunk);\n";
    o << "    if (t >= items) break;\n";
    o << "    const fbg_u64 e = t + chunk < items ? t + chunk : items;\n";
    o << "    for (; t < e; ++t) {\n";
    o << "      const fbg_u64 v = t >> " << wb << ";\n";
    o << "      const fbg_u32 tb = lane | ((fbg_u32)(t & " << ((1u << wb) - 1u) << "u) << 5);\n";
    o << "      if (!P.models) {\n";
    o << "        const fbg_u64 c = fbg_warp_sum(fbg_unit_count(P.unit_begin + v, P.unit_begin + v + 1, tb, lvl, 0u, full2));\n";
    o << "        if (lane == 0u) P.unit_counts[t] = c;\n";
    o << "      } else {\n";
    o << "        const fbg_u64 b = P.unit_offsets[t];\n";
    o << "        if (b < P.cap) fbg_unit_enum(P.unit_begin + v, tb, b, P.models, P.cap, lvl);\n";
    o << "      }\n";
    o << "    }\n";
    o << "  }\n";
    o << "  if (P.iters && lane == 0u) {\n";
    o << "    for (int l = 0; l < " << nl << "; l++) if (lvl[l]) atomicAdd(P.iters + l, lvl[l]);\n";
    o << "  }\n";
    o << "}\n";
    return o.str();
  }
  o << "extern \"C\" __global__ void __launch_bounds__(" << block << ", " << minb << ") " << kname << "(FbgLaunch P) {\n";
  if (mode == 0) {
    o << "  fbg_u64 lvl[" << nl << "] = {0};\n";
    o << "  fbg_u64 total = 0;\n";
    o << "  const fbg_u32 lane = threadIdx.x & 31u;\n";
    o << "  const fbg_u64 chunk = P.chunk ? P.chunk : 1ull;\n";
    o << "  const fbg_u64 R = P.unit_end - P.unit_begin;\n";
    o << "  const fbg_u64 items = P.unit_perm ? P.nperm : (R << " << L.warp_bits << ");\n";
    // the whole first loop level (unused when it is not a runtime loop)
    o << "  const fbg_u32 full2 = " << (split_bits > 0 ? (1u << L.loop_bits[0]) : 0u) << "u;\n";
    o << "  for (;;) {\n";
    o << "    fbg_u64 t = fbg_next_items_warp(P, chunk);\n";
    o << "    if (t >= items) break;\n";
    o << "    const fbg_u64 e = t + chunk < items ? t + chunk : items;\n";
    o << "    if (P.unit_perm) {\n";
    o << "      for (; t < e; ++t) {\n";
    o << "        const fbg_u32 it = P.unit_perm[t];\n";
    o << "        const fbg_u32 base = it & 0xFFFFFFu;\n";
    o << "        const fbg_u64 v = base >> " << L.warp_bits << ";\n";
    o << "        const fbg_u32 tb = lane | ((base & " << ((1u << L.warp_bits) - 1u) << "u) << 5);\n";
    if (split_bits > 0) {
      // piece q of 2^s of the first loop level (s <= split_bits)
      o << "        const fbg_u32 s = (it >> 28) < " << split_bits << "u ? (it >> 28) : " << split_bits << "u;\n";
      o << "        const fbg_u32 q = (it >> 24) & ((1u << s) - 1u);\n";
      o << "        const fbg_u32 w2 = full2 >> s;\n";
      o << "        total += fbg_unit_count(P.unit_begin + v, P.unit_begin + v + 1, tb, lvl, q * w2, q * w2 + w2);\n";
    } else {
      o << "        total += fbg_unit_count(P.unit_begin + v, P.unit_begin + v + 1, tb, lvl, 0u, full2);\n";
    }
    o << "      }\n";
    o << "      continue;\n";
    o << "    }\n";
    o << "    while (t < e) {\n";
    o << "      const fbg_u64 w = t / R, v0 = t - w * R;\n";
    o << "      const fbg_u64 span = (e - t) < (R - v0) ? (e - t) : (R - v0);\n";
    o << "      const fbg_u32 tb = lane | ((fbg_u32)w << 5);\n";
    o << "      if (P.unit_counts || P.unit_trace || P.item_trace) {\n";
    o << "        for (fbg_u64 v = v0; v < v0 + span; ++v) {\n";
    o << "          const fbg_u64 t0 = (P.unit_trace || P.item_trace) ? fbg_globaltimer() : 0ull;\n";
    o << "          const fbg_u64 c = fbg_unit_count(P.unit_begin + v, P.unit_begin + v + 1, tb, lvl, 0u, full2);\n";
    o << "          total += c;\n";
    o << "          const fbg_u64 ws = fbg_warp_sum(c);\n";
    o << "          if (lane == 0u && ws && P.unit_counts) atomicAdd(P.unit_counts + v, ws);\n";
    o << "          if (lane == 0u && P.unit_trace) {\n";
    o << "            atomicAdd(P.unit_trace + 2 * v, fbg_globaltimer() - t0);\n";
    o << "            atomicMin(P.unit_trace + 2 * v + 1, t0);\n";
    o << "          }\n";
    o << "          if (lane == 0u && P.item_trace) P.item_trace[(v << " << L.warp_bits << ") | w] = fbg_globaltimer() - t0;\n";
    o << "        }\n";
    o << "      } else {\n";
    o << "        total += fbg_unit_count(P.unit_begin + v0, P.unit_begin + v0 + span, tb, lvl, 0u, full2);\n";
    o << "      }\n";
    o << "      t += span;\n";
    o << "    }\n";
    o << "  }\n";
    o << "  total = fbg_warp_sum(total);\n";
    o << "  if (P.done) {\n";
    o << "    if (lane == 0u) fbg_finish_count(P, total);\n";
    o << "  } else if (lane == 0u && total) {\n";
    o << "    atomicAdd(P.count, total);\n";
    o << "  }\n";
    o << "  if (P.iters && lane == 0u) {\n";
    o << "    for (int l = 0; l < " << nl << "; l++) if (lvl[l]) atomicAdd(P.iters + l, lvl[l]);\n";
    o << "  }\n";
    o << "}\n";
    return o.str();
  }
  o << "  fbg_u64 lvl[" << nl << "] = {0};\n";
  o << "  __shared__ fbg_u64 s_unit;\n";
  o << "  const fbg_u64 chunk = P.chunk ? P.chunk : 1ull;\n";
  o << "  for (;;) {\n";
  o << "    const fbg_u64 u = fbg_next_units(P, &s_unit, chunk);\n";
  o << "    if (u >= P.unit_end) break;\n";
  o << "    const fbg_u64 e = u + chunk < P.unit_end ? u + chunk : P.unit_end;\n";
  // a slice of the table starts at 64-bit word P.table_word0: tiles of 2^r
  // 32-bit words before it are not stored
  o << "    for (fbg_u64 v = u; v < e; ++v) fbg_unit_table(v, P.table, (P.table_word0 * 2ull) >> " << L.r << ", lvl);\n";
  o << "  }\n";
  o << "  if (P.iters && (threadIdx.x & 31u) == 0u) {\n";
  o << "    for (int l = 0; l < " << nl << "; l++) if (lvl[l]) atomicAdd(P.iters + l, lvl[l]);\n";
  o << "  }\n";
  o << "}\n";
  return o.str();
}

}  // namespace

std::string emit_cuda_source(const LutProgram& p, int mode, int block, int minblocks,
                             std::vector<long long>* ops_per_level, int* unrolled_level, bool counters,
                             std::vector<long long>* uniform_ops_per_level, int popc_cost) {
  SrcGen g(p, counters, popc_cost);
  std::string src = g.generate(mode, block, minblocks);
  if (ops_per_level) *ops_per_level = g.ops;
  if (uniform_ops_per_level) *uniform_ops_per_level = g.uops;
  if (unrolled_level) *unrolled_level = g.unroll_lv;
  return src;
}

// ---------------------------------------------------------- interpreter --

InterpCode emit_bytecode(const LutProgram& p) {
  const Layout& L = p.layout;
  if (L.r > 1) throw CompileError{"internal: the interpreter uses 64-bit tiles (r <= 1)"};
  InterpCode c;
  c.prog = FbgInterpProg{};
  const int nluts = (int)p.luts.size();
  // constants as 64-bit words (register 0 low, register 1 high)
  for (const ConstVec& cv : p.consts) {
    uint64_t lo = cv.w[0], hi = cv.w.size() > 1 ? cv.w[1] : cv.w[0];
    c.consts.push_back(lo | (hi << 32));
  }
  if (c.consts.size() > FBG_INTERP_MAX_CONSTS) throw CompileError{"too many distinct constants for the interpreter"};
  // last use of every LUT value; values used by a deeper level, by a prune
  // check of a deeper level or by the epilogue stay live to the end
  std::vector<int> last_use((size_t)nluts, -1);
  std::vector<int> users((size_t)nluts, 0);
  std::vector<int> only_user((size_t)nluts, -1);
  std::vector<bool> to_end((size_t)nluts, false), pinned((size_t)nluts, false);
  for (int i = 0; i < nluts; i++) {
    const Lut& lu = p.luts[(size_t)i];
    int prev = -1;
    for (const Val& v : lu.in) {
      if (v.kind != V_LUT || v.id == prev) continue;
      bool dup = false;
      for (const Val& w : lu.in)
        if (&w < &v && w.kind == V_LUT && w.id == v.id) dup = true;
      if (dup) continue;
      int j = v.id;
      last_use[(size_t)j] = std::max(last_use[(size_t)j], i);
      users[(size_t)j]++;
      only_user[(size_t)j] = i;
      if (p.luts[(size_t)j].level < lu.level) to_end[(size_t)j] = true;
    }
  }
  for (int lv = 0; lv < (int)p.levels.size(); lv++) {
    const LevelInfo& li = p.levels[(size_t)lv];
    if (!li.has_acc || li.acc.kind != V_LUT) continue;
    int j = li.acc.id;
    pinned[(size_t)j] = true;
    if (p.luts[(size_t)j].level < lv) to_end[(size_t)j] = true;
    else last_use[(size_t)j] = std::max(last_use[(size_t)j], std::max(li.lut_end - 1, j));
  }
  if (p.out.kind == V_LUT) {
    to_end[(size_t)p.out.id] = true;
    pinned[(size_t)p.out.id] = true;
  }
  // Which values are equal in every tile of a block: those whose letters
  // avoid the lane and warp positions (a tile is the 64 assignments of the
  // in-word and register positions, and the tiles of a block differ only in
  // their lane and warp bits).  Such a value needs one word per block (a
  // block slot) instead of one per tile: the slot file, which sets how many
  // one-warp blocks fit an SM, holds only the values that differ per tile.
  const uint64_t tile_bits = (((1ull << (L.lane_bits + L.warp_bits)) - 1ull) << L.first_lane_pos());
  std::vector<uint64_t> support((size_t)nluts, 0);
  for (int i = 0; i < nluts; i++)
    for (const Val& v : p.luts[(size_t)i].in) {
      if (v.kind == V_VAR) support[(size_t)i] |= 1ull << v.id;
      if (v.kind == V_LUT) support[(size_t)i] |= support[(size_t)v.id];
    }
  auto per_tile = [&](int i) { return (support[(size_t)i] & tile_bits) != 0; };
  // slots: accumulator for a value read only by the next instruction of its
  // level; otherwise a block slot when the value is equal in every tile and
  // one is free, else a tile slot
  std::vector<int> slot((size_t)nluts, -1);
  std::vector<bool> shared_slot((size_t)nluts, false);
  std::vector<int> free_tile, free_shared;
  std::vector<std::pair<int, int>> busy;   // (last use, value)
  int nslots = 0, nshared = 0;
  for (int i = 0; i < nluts; i++) {
    // release values whose last use is this instruction or earlier
    for (size_t q = 0; q < busy.size();) {
      if (busy[q].first <= i) {
        const int v = busy[q].second;
        (shared_slot[(size_t)v] ? free_shared : free_tile).push_back(slot[(size_t)v]);
        busy[q] = busy.back();
        busy.pop_back();
      } else {
        q++;
      }
    }
    bool acc = !to_end[(size_t)i] && !pinned[(size_t)i] && users[(size_t)i] == 1 && only_user[(size_t)i] == i + 1 &&
               p.luts[(size_t)(i + 1)].level == p.luts[(size_t)i].level;
    if (acc) continue;
    auto take = [](std::vector<int>& fl, int& count) {
      if (!fl.empty()) {
        auto it = std::min_element(fl.begin(), fl.end());
        const int s = *it;
        fl.erase(it);
        return s;
      }
      return count++;
    };
    const bool sh = !per_tile(i) && (!free_shared.empty() || nshared < FBG_INTERP_MAX_SHARED);
    shared_slot[(size_t)i] = sh;
    slot[(size_t)i] = sh ? take(free_shared, nshared) : take(free_tile, nslots);
    if (!to_end[(size_t)i]) busy.push_back({std::max(last_use[(size_t)i], i), i});
  }
  if (nslots > FBG_INTERP_MAX_SLOTS) throw CompileError{"program needs " + std::to_string(nslots) + " live values (max " + std::to_string(FBG_INTERP_MAX_SLOTS) + ")"};
  auto code = [&](const Val& v) -> uint32_t {
    if (v.kind == V_CONST) return FBG_OP_CONST | (uint32_t)v.id;
    if (v.kind == V_VAR) return FBG_OP_VAR | (uint32_t)v.id;
    if (slot[(size_t)v.id] < 0) return FBG_OP_ACC;
    return shared_slot[(size_t)v.id] ? (FBG_OP_SHARED | (uint32_t)slot[(size_t)v.id]) : (uint32_t)slot[(size_t)v.id];
  };
  for (int i = 0; i < nluts; i++) {
    const Lut& lu = p.luts[(size_t)i];
    uint64_t dst = slot[(size_t)i] < 0 ? FBG_DST_ACC
                   : shared_slot[(size_t)i] ? (uint64_t)(FBG_DST_SHARED + (unsigned)slot[(size_t)i])
                                            : (uint64_t)slot[(size_t)i];
    uint64_t w = (uint64_t)lu.tt | (dst << 8) | ((uint64_t)code(lu.in[0]) << 16) | ((uint64_t)code(lu.in[1]) << 32) |
                 ((uint64_t)code(lu.in[2]) << 48);
    c.ins.push_back(w);
  }
  FbgInterpProg& G = c.prog;
  G.n = (unsigned)L.n;
  G.nlevels = (unsigned)L.nlevels();
  if (G.nlevels > FBG_INTERP_MAX_LEVELS) throw CompileError{"too many loop levels"};
  G.nslots = (unsigned)std::max(1, nslots);
  G.nshared = (unsigned)nshared;
  G.nconst = (unsigned)c.consts.size();
  G.tvalid = 1u << (L.lane_bits + L.warp_bits);
  G.first_unit_pos = (unsigned)L.first_unit_pos();
  G.unit_bits = (unsigned)L.unit_bits;
  G.out_op = code(p.out);
  G.vmask = L.n >= 6 ? ~0ull : ((1ull << (1u << L.n)) - 1ull);
  G.nunits = 1ull << L.unit_bits;
  for (int lv = 0; lv < (int)G.nlevels; lv++) {
    const LevelInfo& li = p.levels[(size_t)lv];
    FbgInterpLevel& X = G.lev[lv];
    X.ins_begin = (unsigned)li.lut_begin;
    X.ins_end = (unsigned)li.lut_end;
    X.has_acc = li.has_acc ? 1u : 0u;
    X.acc_op = li.has_acc ? code(li.acc) : 0u;
    if (lv >= 2) {
      X.bits = (unsigned)L.loop_bits[(size_t)(lv - 2)];
      X.pos = (unsigned)L.loop_pos(lv - 2);
    }
  }
  c.nslots = G.nslots;
  return c;
}

}  // namespace fbg
