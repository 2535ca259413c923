// fbg_internal.hpp -- host-side data structures of the formula compiler.
//
// Pipeline (all host code, no GPU work):
//   text --parse--> Ast --ground (Sec. 3.1, map *)--> Form DAG (hash-consed,
//   constants removed: the "Reduction" of Sec. 4.1) --choose Layout-->
//   --lower (level-aware reassociation, 2-input gates)--> --map (3-feasible
//   cuts, min-area cover)--> LUT program split into loop levels.
// The LUT program is consumed by the NVRTC emitter and by the bytecode
// emitter for the interpreter kernel.
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

namespace fbg {

struct CompileError {
  std::string msg;
};

// ---------------------------------------------------------------- syntax --

struct IndexTerm {
  int slot = -1;   // bound-name slot, or -1 for a literal
  int value = 0;
};

struct Guard {
  IndexTerm l, r;
  int op = 0;      // 0 <, 1 <=, 2 >, 3 >=, 4 ==, 5 !=
};

// a term: an index (family < 0) or a function symbol applied to terms
struct Term {
  int family = -1;
  IndexTerm ix;
  std::vector<Term> args;
};

struct Ast {
  enum Kind { Const, Atom, Not, And, Or, Xor, Imp, Iff, Forall, Exists, Eq } kind = Const;
  int value = 0;                      // Const
  int family = -1;                    // Atom
  std::vector<IndexTerm> idx;         // Atom: plain arguments
  std::vector<Term> targs;            // Atom: all arguments as terms, when one is a function term
  Term lhs, rhs;                      // Eq
  std::unique_ptr<Ast> a, b;
  int first_slot = 0, nbound = 0;     // quantifiers
  bool distinct = false;              // S2 / S3
  std::vector<Guard> guards;
};

struct Family {
  std::string name;
  int arity = 0;
  std::vector<bool> lt;               // lt[p]: position p < position p+1
  bool is_const = false;
  bool is_fun = false;                // function symbol: the last position is the value
  int first_id = 0;                   // variables: id of the first tuple
  int count = 0;                      // number of admissible tuples
  std::vector<int> rank;              // linear tuple index -> rank or -1
  std::vector<uint8_t> bits;          // constants: value per linear tuple
};

struct Theory {
  int k = 1;
  int nvars = 0;                       // declared letters
  std::vector<Family> fams;
  std::vector<std::unique_ptr<Ast>> axioms;
  std::vector<std::unique_ptr<Ast>> assumes;   // 'assume' lines (killing, Sec. 3.3)
  std::vector<std::string> var_names;  // "r(1,2)" per declared letter
};

Theory parse_theory(const std::string& text, int k);  // throws CompileError

// ------------------------------------------------------------- Form DAG --
// n-ary AND/OR, binary XOR, NOT, variables and the two constants; hash-consed
// with the identities x&1=x, x&0=0, x&x=x, x&~x=0 (and duals), ~~x=x,
// x^x=0, x^~x=1, x^0=x, x^1=~x.

enum FOp : uint8_t { F0, F1, FVAR, FNOT, FAND, FOR, FXOR };

struct FNode {
  FOp op;
  int var = -1;
  std::vector<int> kids;
};

class FormDag {
 public:
  FormDag();
  int zero() const { return 0; }
  int one() const { return 1; }
  int var(int v);
  int mk_not(int a);
  int mk_and(const std::vector<int>& kids);
  int mk_or(const std::vector<int>& kids);
  int mk_xor(int a, int b);
  const FNode& node(int i) const { return nodes_[i]; }
  int size() const { return (int)nodes_.size(); }

 private:
  int intern(FNode&& n);
  int mk_nary(FOp op, const std::vector<int>& kids);
  std::vector<FNode> nodes_;
  std::unordered_map<std::string, int> table_;
};

struct Grounded {
  FormDag dag;
  int root = 1;
  int nvars = 0;                   // free letters (declared minus killed)
  std::vector<int> letter_of_var;  // free letter -> declared letter id
  std::vector<int> killed;         // per declared letter: -1 free, 0/1 killed value
};

Grounded ground(const Theory& th);   // the map * of Sec. 3.1

// --------------------------------------------------------------- layout --
// Bits of the assignment integer j, from the least significant:
//   [0,5)            in-register bit (32 assignments per 32-bit word)
//   [5,5+r)          register index inside a thread's tile of 2^r words
//   lane bits (<=5), warp bits, then loop levels innermost-first, then the
//   unit bits (one unit = one block-uniform prefix, fetched dynamically).
// A permutation maps formula variables to bit positions (identity for
// truth tables and model lists, a search-order heuristic for counts).

enum Level : int { LV_CONST = -1, LV_THREAD = 0, LV_UNIT = 1 };   // loops: 2..

struct Layout {
  int n = 0;
  int r = 0, lane_bits = 0, warp_bits = 0, unit_bits = 0;
  std::vector<int> loop_bits;        // outermost first
  std::vector<int> pos_of_var, var_of_pos;

  int nlevels() const { return 2 + (int)loop_bits.size(); }
  int tile_bits() const { return n <= 5 ? 0 : n - 5 - r; }
  int first_lane_pos() const { return 5 + r; }
  int first_warp_pos() const { return 5 + r + lane_bits; }
  // loop level i (0 = outermost) occupies positions [loop_pos(i), +loop_bits[i])
  int loop_pos(int i) const;
  int first_unit_pos() const { return n - unit_bits; }
  int level_of_pos(int p) const;
};

struct LayoutParams {
  int r_max = 2;
  int warps_log2 = 3;
  int unit_bits_max = 13;
  int loop_level_bits = 4;
  int loop_bits_max = 16;
  int inner_bits = 0;        // innermost loop level's bits (0 = loop_level_bits)
  int max_loop_levels = 64;  // wider levels when the loop bits would need more
};

Layout make_layout(int n, const LayoutParams& prm, const std::vector<int>& order_top_first);
std::vector<int> identity_order(int n);                          // top position first
// count-mode heuristic; seed != 0 breaks ties between equally good letters
// by a seeded hash instead of the lowest index (a variant the autotuner tries)
std::vector<int> search_order(const Grounded& g, uint64_t seed = 0);
std::vector<int> enum_order(int n, const LayoutParams& prm);     // enumerate mode: items are intervals
// Per work item (unit u, warp slice w) of layout L, index u << warp_bits | w
// (1 byte each): 0 when a top-level conjunct whose letters all sit in unit
// and warp positions is false on that item, so the item has no models;
// empty when there is no such conjunct or more than 20 unit + warp bits.
std::vector<uint8_t> alive_items(const Grounded& g, const Layout& L);
// the same as a bit vector: bit t of word t / 64 set when item t may hold
// models (empty: no conjunct over unit and warp letters, or too many items)
std::vector<uint64_t> alive_words(const Grounded& g, const Layout& L);

// ------------------------------------------------------------ LUT program --

enum ValKind : uint8_t { V_CONST, V_VAR, V_LUT };

struct Val {
  ValKind kind = V_CONST;
  int id = 0;          // const index / bit position / LUT index
  bool operator==(const Val& o) const { return kind == o.kind && id == o.id; }
};

struct ConstVec {
  std::vector<uint32_t> w;   // one 32-bit word per register index (2^r)
};

struct Lut {
  uint8_t tt = 0;            // lop3 immLut: f(0xF0, 0xCC, 0xAA)
  Val in[3];
  int level = 0;
  uint32_t rmask = 0;        // register-index bits the value depends on
};

struct LevelInfo {
  int lut_begin = 0, lut_end = 0;   // LUTs of this level, topologically ordered
  bool has_acc = false;             // new top-level conjuncts at this level
  Val acc;                          // conjunction of all conjuncts at levels <= this
};

struct LutProgram {
  Layout layout;
  std::vector<ConstVec> consts;
  std::vector<Lut> luts;
  std::vector<LevelInfo> levels;    // index = level (0 thread, 1 unit, 2.. loops)
  Val out;                          // the formula value (positive literal)
  ConstVec const_acc;               // conjunction of constant-level conjuncts
  // statistics
  int gates = 0;                    // 2-input gates before mapping
  long long lop3_per_level[16] = {0};   // 32-bit lop3 per execution of each level
};

LutProgram lower_and_map(const Grounded& g, const Layout& L);

uint32_t rmask_of(const LutProgram& p, const Val& v);

}  // namespace fbg
