/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.  Plain, slow CPU oracle for the
 * free-Boolean-generator evaluation.  Only tests, the smoke check and the
 * bench's CPU-baseline leg may load it; the product never does.
 *
 * What it computes is the plain definition (Prop. 2.2, Sec. 2.3): the vector
 * t(b_1..b_n) over the free generators has, at position j, the value of the
 * formula under the valuation mu_j.  The valuation follows the generator
 * matrix M of Sec. 2.2 with the index order flipped: variable x_i takes
 * bit i of j (x_0 is the paper's b_n).  So the oracle does NOT evaluate
 * bitwise at all: for every assignment integer j it decodes mu_j and
 * model-checks the quantified formula on the finite structure h(mu_j) of
 * Sec. 3.2 (R(a..) holds iff mu_j(q_{Ra..}) = 1), walking the syntax tree
 * with C booleans.  Quantifiers are loops over the domain (the map * of
 * Sec. 3.1 read semantically: forall = conjunction over A, exists =
 * disjunction over A); and/or short-circuit.  There is no grounding, no
 * DAG, no LOP3 and nothing shared with the CUDA path.
 *
 * Text format (one axiom per line, the theory is their conjunction):
 *   var x, y, r(S,S), e(S<S)     declare variables; ids in declaration order,
 *                                tuples in lexicographic order ('<' = strictly
 *                                increasing positions)
 *   const E(S,S) = 0110...       constant relation, bits over all tuples in
 *                                lexicographic order
 *   fun m(S,S)                   function symbol with values in the domain
 *                                (Sec. 3.1): letters m(a,b,u) = "m(a,b) = u",
 *                                tuples (a,b,u) in lexicographic order; 'fun c'
 *                                declares a constant symbol, letters c(u)
 *   [label =] formula            operators ~ & ^ | -> <-> with Python
 *                                precedence (~ > & > ^ > |) then -> (right
 *                                assoc) then <->; constants 0 1; quantifiers
 *                                A[i,j:S | i<j] / E[i:S2] scope over the next
 *                                unary term; an optional '.' may follow ']'.
 *   assume formula              kill letters: a conjunction of literals,
 *                                possibly quantified, fixes each letter
 *                                (later lines override earlier ones); the
 *                                remaining letters keep declaration order.
 *                                A literal m(a) = b fixes m(a,b) to 1 and
 *                                m(a,b') to 0 for every b' != b; its negation
 *                                fixes m(a,b) to 0.
 * Terms: a numeral, a bound name, or m(t,..) for a declared function symbol.
 * An equation t1 = t2 (or t1 != t2) is an atomic formula; relation atoms
 * take terms as arguments (not in families declared with '<').
 * Semantics of function symbols: mu_j defines a structure of the language
 * only when every m(a..) has exactly one value u with m(a..,u) true (h of
 * Sec. 3.2 reads F(a..) = b off mu(p_{Fa..b})); any other mu_j is not a model.
 * Terms are then evaluated by looking up that value.
 *   '#' starts a comment.
 * Sets: S = range(k) per bound name; S2/S3 = ordered tuples of 2/3 distinct
 * elements (the paper's perm(range(n),2) and perm(range(n),3), Sec. 4.2).
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <ctype.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_ARITY 4
#define OR_MAX_BOUND 32
#define OR_MAX_FAM 64
#define OR_MAX_LETTERS 4096         /* declared letters; at most 64 stay free */

enum { N_CONST, N_ATOM, N_NOT, N_AND, N_OR, N_XOR, N_IMP, N_IFF, N_FORALL, N_EXISTS, N_EQ };
enum { CMP_LT, CMP_LE, CMP_GT, CMP_GE, CMP_EQ, CMP_NE };

typedef struct {
  char name[64];
  int arity;
  int lt[OR_MAX_ARITY];       /* lt[p] = 1: position p < position p+1 */
  int is_const;
  int is_fun;                 /* function symbol: arity = arguments + 1 (the value) */
  int first_id;               /* variables: id of the first tuple */
  int count;                  /* number of tuples in the family */
  unsigned char *bits;        /* constants: value per tuple, k^arity entries */
} Family;

/* an index term: bound-variable slot (>=0) or literal value (slot = -1) */
typedef struct { int slot; int value; } Idx;

typedef struct { Idx l, r; int op; } Cmp;

/* a term: an index (fam < 0) or a function symbol applied to terms */
typedef struct Term {
  int fam;
  Idx idx;
  int nargs;
  struct Term *args[OR_MAX_ARITY];
} Term;

typedef struct Node {
  int kind;
  int value;                  /* N_CONST */
  int fam;                    /* N_ATOM */
  int nidx;
  Idx idx[OR_MAX_ARITY];
  Term *targ[OR_MAX_ARITY];   /* N_ATOM: argument i is this term when non-NULL */
  Term *lhs, *rhs;            /* N_EQ */
  struct Node *a, *b;         /* children */
  /* quantifiers */
  int nbound, first_slot;     /* bound names occupy slots first_slot.. */
  int distinct;               /* 1 for S2 / S3 */
  int ncmp;
  Cmp cmp[8];
} Node;

typedef struct oracle_prog {
  int k;
  int nvars;                  /* free letters (declared minus killed) */
  int nletters;               /* declared letters */
  int nfam;
  Family fam[OR_MAX_FAM];
  int naxioms;
  Node **axioms;
  int nassume;
  Node **assumes;             /* 'assume' lines, in order */
  signed char fixed[OR_MAX_LETTERS];  /* per declared letter: -1 free, else its killed value */
  int bit_of[OR_MAX_LETTERS];         /* per free letter: its bit in the assignment integer */
} oracle_prog;

/* ------------------------------------------------------------------ */
/* parsing                                                              */

typedef struct {
  const char *s;
  int pos;
  int line;
  char err[256];
  oracle_prog *p;
  char bound[OR_MAX_BOUND][64];
  int nbound;
} Parser;

static void set_err(Parser *ps, const char *msg) {
  if (!ps->err[0]) snprintf(ps->err, sizeof ps->err, "line %d: %s", ps->line, msg);
}

static void skip_ws(Parser *ps) {
  for (;;) {
    char c = ps->s[ps->pos];
    if (c == ' ' || c == '\t' || c == '\r') { ps->pos++; continue; }
    if (c == '#') { while (ps->s[ps->pos] && ps->s[ps->pos] != '\n') ps->pos++; continue; }
    return;
  }
}

static int peek(Parser *ps) { skip_ws(ps); return ps->s[ps->pos]; }

static int accept(Parser *ps, const char *tok) {
  skip_ws(ps);
  size_t n = strlen(tok);
  if (strncmp(ps->s + ps->pos, tok, n) == 0) { ps->pos += (int)n; return 1; }
  return 0;
}

static int expect(Parser *ps, const char *tok) {
  if (accept(ps, tok)) return 1;
  char m[96]; snprintf(m, sizeof m, "expected '%s'", tok); set_err(ps, m);
  return 0;
}

static int read_name(Parser *ps, char *out) {
  skip_ws(ps);
  int c = ps->s[ps->pos];
  if (!(isalpha(c) || c == '_')) return 0;
  int n = 0;
  while (isalnum((unsigned char)ps->s[ps->pos]) || ps->s[ps->pos] == '_') {
    if (n < 63) out[n++] = ps->s[ps->pos];
    ps->pos++;
  }
  out[n] = 0;
  return 1;
}

static int read_int(Parser *ps, int *out) {
  skip_ws(ps);
  if (!isdigit((unsigned char)ps->s[ps->pos])) return 0;
  long v = 0;
  while (isdigit((unsigned char)ps->s[ps->pos])) { v = v * 10 + (ps->s[ps->pos] - '0'); ps->pos++; if (v > 1000000) v = 1000000; }
  *out = (int)v;
  return 1;
}

static Node *new_node(int kind) {
  Node *n = (Node *)calloc(1, sizeof(Node));
  n->kind = kind;
  return n;
}

static void free_term(Term *t) {
  if (!t) return;
  for (int i = 0; i < t->nargs; i++) free_term(t->args[i]);
  free(t);
}

static void free_node(Node *n) {
  if (!n) return;
  free_node(n->a);
  free_node(n->b);
  for (int i = 0; i < OR_MAX_ARITY; i++) free_term(n->targ[i]);
  free_term(n->lhs);
  free_term(n->rhs);
  free(n);
}

static int find_family(oracle_prog *p, const char *name) {
  for (int i = 0; i < p->nfam; i++)
    if (strcmp(p->fam[i].name, name) == 0) return i;
  return -1;
}

static int find_bound(Parser *ps, const char *name) {
  for (int i = ps->nbound - 1; i >= 0; i--)
    if (strcmp(ps->bound[i], name) == 0) return i;
  return -1;
}

static Node *parse_formula(Parser *ps);
static Node *parse_unary(Parser *ps);

static int parse_idx(Parser *ps, Idx *out) {
  char nm[64];
  int v;
  if (read_int(ps, &v)) { out->slot = -1; out->value = v; return 1; }
  if (read_name(ps, nm)) {
    int s = find_bound(ps, nm);
    if (s < 0) { char m[128]; snprintf(m, sizeof m, "unbound index '%s'", nm); set_err(ps, m); return 0; }
    out->slot = s; out->value = 0;
    return 1;
  }
  set_err(ps, "expected index");
  return 0;
}

/* term: numeral | bound name | f(term, ..) for a function symbol f */
static Term *parse_term(Parser *ps) {
  Term *t = (Term *)calloc(1, sizeof(Term));
  t->fam = -1;
  char nm[64];
  skip_ws(ps);
  int save = ps->pos;
  if (read_name(ps, nm)) {
    int f = find_family(ps->p, nm);
    if (find_bound(ps, nm) < 0 && f >= 0) {
      const Family *F = &ps->p->fam[f];
      if (!F->is_fun) { set_err(ps, "a relation symbol is not a term"); free(t); return NULL; }
      t->fam = f;
      if (F->arity > 1) {
        if (!expect(ps, "(")) { free(t); return NULL; }
        do {
          if (t->nargs >= F->arity - 1) { set_err(ps, "too many arguments"); free_term(t); return NULL; }
          Term *a = parse_term(ps);
          if (!a) { free_term(t); return NULL; }
          t->args[t->nargs++] = a;
        } while (accept(ps, ","));
        if (!expect(ps, ")")) { free_term(t); return NULL; }
      }
      if (t->nargs != F->arity - 1) { set_err(ps, "wrong number of arguments"); free_term(t); return NULL; }
      return t;
    }
    ps->pos = save;
  }
  if (!parse_idx(ps, &t->idx)) { free(t); return NULL; }
  return t;
}

/* '=' that is not '==' */
static int accept_eq(Parser *ps) {
  skip_ws(ps);
  if (ps->s[ps->pos] == '=' && ps->s[ps->pos + 1] != '=') { ps->pos++; return 1; }
  return 0;
}

/* the rest of an equation 't = u' / 't != u' after its left side */
static Node *parse_equation(Parser *ps, Term *lhs) {
  int neg = 0;
  if (accept(ps, "!=")) neg = 1;
  else if (!accept_eq(ps)) { set_err(ps, "expected '=' or '!=' after a term"); free_term(lhs); return NULL; }
  Term *rhs = parse_term(ps);
  if (!rhs) { free_term(lhs); return NULL; }
  Node *e = new_node(N_EQ);
  e->lhs = lhs;
  e->rhs = rhs;
  if (!neg) return e;
  Node *n = new_node(N_NOT);
  n->a = e;
  return n;
}

static Node *parse_quant(Parser *ps, int forall) {
  /* '[' already consumed */
  Node *q = new_node(forall ? N_FORALL : N_EXISTS);
  char names[OR_MAX_BOUND][64];
  int nn = 0;
  do {
    if (nn >= 8 || !read_name(ps, names[nn])) { set_err(ps, "bad bound name list"); free_node(q); return NULL; }
    nn++;
  } while (accept(ps, ","));
  if (!expect(ps, ":")) { free_node(q); return NULL; }
  char set[64];
  if (!read_name(ps, set)) { set_err(ps, "expected set name"); free_node(q); return NULL; }
  if (strcmp(set, "S") == 0) q->distinct = 0;
  else if (strcmp(set, "S2") == 0) { q->distinct = 1; if (nn != 2) { set_err(ps, "S2 binds exactly 2 names"); free_node(q); return NULL; } }
  else if (strcmp(set, "S3") == 0) { q->distinct = 1; if (nn != 3) { set_err(ps, "S3 binds exactly 3 names"); free_node(q); return NULL; } }
  else { set_err(ps, "unknown set (S, S2, S3)"); free_node(q); return NULL; }
  if (ps->nbound + nn > OR_MAX_BOUND) { set_err(ps, "too many nested bound names"); free_node(q); return NULL; }
  q->first_slot = ps->nbound;
  q->nbound = nn;
  for (int i = 0; i < nn; i++) strcpy(ps->bound[ps->nbound++], names[i]);
  if (accept(ps, "|")) {
    do {
      if (q->ncmp >= 8) { set_err(ps, "too many guard comparisons"); goto fail; }
      Cmp *c = &q->cmp[q->ncmp++];
      if (!parse_idx(ps, &c->l)) goto fail;
      if (accept(ps, "<=")) c->op = CMP_LE;
      else if (accept(ps, ">=")) c->op = CMP_GE;
      else if (accept(ps, "==")) c->op = CMP_EQ;
      else if (accept(ps, "!=")) c->op = CMP_NE;
      else if (accept(ps, "<")) c->op = CMP_LT;
      else if (accept(ps, ">")) c->op = CMP_GT;
      else { set_err(ps, "expected comparison"); goto fail; }
      if (!parse_idx(ps, &c->r)) goto fail;
    } while (accept(ps, ",") || accept(ps, "&"));
  }
  if (!expect(ps, "]")) goto fail;
  accept(ps, ".");
  q->a = parse_unary(ps);
  if (!q->a) goto fail;
  ps->nbound -= nn;
  return q;
fail:
  ps->nbound = q->first_slot;
  free_node(q);
  return NULL;
}

static Node *parse_primary(Parser *ps) {
  int c = peek(ps);
  if (c == '(') {
    ps->pos++;
    Node *n = parse_formula(ps);
    if (!n) return NULL;
    if (!expect(ps, ")")) { free_node(n); return NULL; }
    return n;
  }
  int v;
  if (isdigit(c)) {
    int save = ps->pos;
    if (!read_int(ps, &v)) { set_err(ps, "bad numeral"); return NULL; }
    skip_ws(ps);
    if ((ps->s[ps->pos] == '=' && ps->s[ps->pos + 1] != '=') || (ps->s[ps->pos] == '!' && ps->s[ps->pos + 1] == '=')) {
      ps->pos = save;
      Term *t = parse_term(ps);
      return t ? parse_equation(ps, t) : NULL;
    }
    if (v > 1) { set_err(ps, "constants are 0 or 1"); return NULL; }
    Node *n = new_node(N_CONST);
    n->value = v;
    return n;
  }
  char nm[64];
  int start = ps->pos;
  if (!read_name(ps, nm)) { set_err(ps, "expected a term"); return NULL; }
  /* quantifier keyword: A or E directly followed by '[' */
  if ((strcmp(nm, "A") == 0 || strcmp(nm, "E") == 0) && peek(ps) == '[') {
    ps->pos++;
    return parse_quant(ps, nm[0] == 'A');
  }
  int f = find_family(ps->p, nm);
  if (find_bound(ps, nm) >= 0 || (f >= 0 && ps->p->fam[f].is_fun)) {
    ps->pos = start;
    Term *t = parse_term(ps);
    return t ? parse_equation(ps, t) : NULL;
  }
  if (f < 0) { char m[128]; snprintf(m, sizeof m, "undeclared name '%s'", nm); set_err(ps, m); return NULL; }
  Node *n = new_node(N_ATOM);
  n->fam = f;
  if (peek(ps) == '(') {
    ps->pos++;
    do {
      if (n->nidx >= OR_MAX_ARITY) { set_err(ps, "too many indices"); free_node(n); return NULL; }
      Term *t = parse_term(ps);
      if (!t) { free_node(n); return NULL; }
      if (t->fam < 0) { n->idx[n->nidx] = t->idx; free(t); }
      else n->targ[n->nidx] = t;
      n->nidx++;
    } while (accept(ps, ","));
    if (!expect(ps, ")")) { free_node(n); return NULL; }
  }
  if (n->nidx != ps->p->fam[f].arity) { set_err(ps, "wrong number of indices"); free_node(n); return NULL; }
  for (int i = 0; i < n->nidx; i++)
    if (n->targ[i])
      for (int q = 0; q + 1 < ps->p->fam[f].arity; q++)
        if (ps->p->fam[f].lt[q]) { set_err(ps, "function terms in a family declared with '<'"); free_node(n); return NULL; }
  return n;
}

static Node *parse_unary(Parser *ps) {
  if (peek(ps) == '~') {
    ps->pos++;
    Node *a = parse_unary(ps);
    if (!a) return NULL;
    Node *n = new_node(N_NOT);
    n->a = a;
    return n;
  }
  return parse_primary(ps);
}

static Node *bin(int kind, Node *a, Node *b) {
  Node *n = new_node(kind);
  n->a = a;
  n->b = b;
  return n;
}

static Node *parse_and(Parser *ps) {
  Node *l = parse_unary(ps);
  while (l && peek(ps) == '&') {
    ps->pos++;
    Node *r = parse_unary(ps);
    if (!r) { free_node(l); return NULL; }
    l = bin(N_AND, l, r);
  }
  return l;
}

static Node *parse_xor(Parser *ps) {
  Node *l = parse_and(ps);
  while (l && peek(ps) == '^') {
    ps->pos++;
    Node *r = parse_and(ps);
    if (!r) { free_node(l); return NULL; }
    l = bin(N_XOR, l, r);
  }
  return l;
}

static Node *parse_or(Parser *ps) {
  Node *l = parse_xor(ps);
  /* '|' alone; a guard '|' never reaches here (guards are inside [..]) */
  while (l && peek(ps) == '|') {
    ps->pos++;
    Node *r = parse_xor(ps);
    if (!r) { free_node(l); return NULL; }
    l = bin(N_OR, l, r);
  }
  return l;
}

static Node *parse_imp(Parser *ps) {
  Node *l = parse_or(ps);
  if (l && accept(ps, "->")) {
    Node *r = parse_imp(ps);
    if (!r) { free_node(l); return NULL; }
    l = bin(N_IMP, l, r);
  }
  return l;
}

static Node *parse_formula(Parser *ps) {
  Node *l = parse_imp(ps);
  while (l && accept(ps, "<->")) {
    Node *r = parse_imp(ps);
    if (!r) { free_node(l); return NULL; }
    l = bin(N_IFF, l, r);
  }
  return l;
}

/* number of tuples of a family over range(k) respecting '<' constraints */
static long family_size(const Family *f, int k) {
  if (f->arity == 0) return 1;
  long total = 0;
  int t[OR_MAX_ARITY] = {0};
  for (;;) {
    int ok = 1;
    for (int p = 0; p + 1 < f->arity; p++)
      if (f->lt[p] && !(t[p] < t[p + 1])) ok = 0;
    total += ok;
    int p = f->arity - 1;
    while (p >= 0 && ++t[p] == k) { t[p] = 0; p--; }
    if (p < 0) break;
  }
  return total;
}

/* rank of a tuple among the family's tuples in lexicographic order, -1 if outside */
static long tuple_rank(const Family *f, int k, const int *tup) {
  for (int p = 0; p < f->arity; p++)
    if (tup[p] < 0 || tup[p] >= k) return -1;
  for (int p = 0; p + 1 < f->arity; p++)
    if (f->lt[p] && !(tup[p] < tup[p + 1])) return -1;
  /* count admissible tuples lexicographically smaller, by plain enumeration */
  long rank = 0;
  int t[OR_MAX_ARITY] = {0};
  if (f->arity == 0) return 0;
  for (;;) {
    int same = 1;
    for (int p = 0; p < f->arity; p++) if (t[p] != tup[p]) same = 0;
    if (same) return rank;
    int ok = 1;
    for (int p = 0; p + 1 < f->arity; p++)
      if (f->lt[p] && !(t[p] < t[p + 1])) ok = 0;
    rank += ok;
    int p = f->arity - 1;
    while (p >= 0 && ++t[p] == k) { t[p] = 0; p--; }
    if (p < 0) break;
  }
  return -1;
}

static int parse_decl(Parser *ps, int is_const, int is_fun) {
  oracle_prog *p = ps->p;
  if (p->nfam >= OR_MAX_FAM) { set_err(ps, "too many declarations"); return 0; }
  Family *f = &p->fam[p->nfam];
  memset(f, 0, sizeof *f);
  if (!read_name(ps, f->name)) { set_err(ps, "expected a name"); return 0; }
  if ((strcmp(f->name, "A") == 0 || strcmp(f->name, "E") == 0) && !is_const) { /* allowed, disambiguated by '[' */ }
  if (find_family(p, f->name) >= 0) { set_err(ps, "name declared twice"); return 0; }
  if (accept(ps, "(")) {
    for (;;) {
      char d[64];
      if (!read_name(ps, d) || strcmp(d, "S") != 0) { set_err(ps, "declared positions range over S"); return 0; }
      if (f->arity >= OR_MAX_ARITY - (is_fun ? 1 : 0)) { set_err(ps, "arity too large"); return 0; }
      f->arity++;
      if (accept(ps, ",")) continue;
      if (!is_fun && accept(ps, "<")) { f->lt[f->arity - 1] = 1; continue; }
      break;
    }
    if (!expect(ps, ")")) return 0;
  }
  if (is_fun) f->arity++;    /* the value position */
  f->is_fun = is_fun;
  f->is_const = is_const;
  f->count = (int)family_size(f, p->k);
  if (is_const) {
    for (int q = 0; q + 1 < f->arity; q++)
      if (f->lt[q]) { set_err(ps, "constants use full tuples (no '<')"); return 0; }
    if (!expect(ps, "=")) return 0;
    skip_ws(ps);
    long want = f->count;
    f->bits = (unsigned char *)calloc((size_t)(want > 0 ? want : 1), 1);
    long got = 0;
    while (ps->s[ps->pos] == '0' || ps->s[ps->pos] == '1') {
      if (got < want) f->bits[got] = (unsigned char)(ps->s[ps->pos] - '0');
      got++;
      ps->pos++;
    }
    if (got != want) { set_err(ps, "constant has the wrong number of bits"); free(f->bits); f->bits = NULL; return 0; }
  } else {
    f->first_id = p->nvars;
    if ((long)p->nvars + f->count > OR_MAX_LETTERS) { set_err(ps, "more than 4096 declared letters"); return 0; }
    p->nvars += f->count;
  }
  p->nfam++;
  return 1;
}

static void free_prog(oracle_prog *p) {
  if (!p) return;
  for (int i = 0; i < p->naxioms; i++) free_node(p->axioms[i]);
  free(p->axioms);
  for (int i = 0; i < p->nassume; i++) free_node(p->assumes[i]);
  free(p->assumes);
  for (int i = 0; i < p->nfam; i++) free(p->fam[i].bits);
  free(p);
}

/* ------------------------------------------------------------------ */
/* evaluation: model checking on the structure decoded from j            */

typedef struct { const oracle_prog *p; uint64_t j; int env[OR_MAX_BOUND]; int bad; } Ctx;

static int idx_value(const Ctx *c, Idx x) { return x.slot < 0 ? x.value : c->env[x.slot]; }

/* h(mu_j): the free letter numbered v holds iff bit v of j is 1; a killed
   letter (Sec. 3.3) has its assumed value */
static int letter_value(const oracle_prog *p, uint64_t j, int id) {
  if (p->fixed[id] >= 0) return p->fixed[id];
  return (int)((j >> p->bit_of[id]) & 1u);
}

/* linear index of an argument tuple of a function symbol (values in range) */
static long fun_base(const oracle_prog *p, const Family *f, const int *args) {
  long lin = 0;
  for (int i = 0; i + 1 < f->arity; i++) lin = lin * p->k + args[i];
  return f->first_id + lin * p->k;
}

/* F^A(a..) = the b with mu_j(p_{Fa..b}) = 1; mu_j is known to be functional */
static int term_value(Ctx *c, const Term *t) {
  if (t->fam < 0) return idx_value(c, t->idx);
  const Family *f = &c->p->fam[t->fam];
  int args[OR_MAX_ARITY];
  for (int i = 0; i < t->nargs; i++) args[i] = term_value(c, t->args[i]);
  for (int i = 0; i < t->nargs; i++)
    if (args[i] < 0 || args[i] >= c->p->k) { c->bad = 1; return 0; }
  long base = fun_base(c->p, f, args);
  for (int b = 0; b < c->p->k; b++)
    if (letter_value(c->p, c->j, (int)(base + b))) return b;
  c->bad = 1;
  return 0;
}

/* mu_j defines a structure of the language: every function symbol has
   exactly one value at every argument tuple */
static int functional(const oracle_prog *p, uint64_t j) {
  for (int fi = 0; fi < p->nfam; fi++) {
    const Family *f = &p->fam[fi];
    if (!f->is_fun) continue;
    long tuples = f->count / p->k;
    for (long t = 0; t < tuples; t++) {
      int ones = 0;
      for (int b = 0; b < p->k; b++) ones += letter_value(p, j, (int)(f->first_id + t * p->k + b));
      if (ones != 1) return 0;
    }
  }
  return 1;
}

static int eval(Ctx *c, const Node *n);

static int guard_ok(const Ctx *c, const Node *q) {
  for (int i = 0; i < q->ncmp; i++) {
    int l = idx_value(c, q->cmp[i].l), r = idx_value(c, q->cmp[i].r), ok = 0;
    switch (q->cmp[i].op) {
      case CMP_LT: ok = l < r; break;
      case CMP_LE: ok = l <= r; break;
      case CMP_GT: ok = l > r; break;
      case CMP_GE: ok = l >= r; break;
      case CMP_EQ: ok = l == r; break;
      case CMP_NE: ok = l != r; break;
    }
    if (!ok) return 0;
  }
  if (q->distinct)
    for (int a = 0; a < q->nbound; a++)
      for (int b = a + 1; b < q->nbound; b++)
        if (c->env[q->first_slot + a] == c->env[q->first_slot + b]) return 0;
  return 1;
}

/* forall: conjunction over the tuples; exists: disjunction (Sec. 3.1) */
static int eval_quant(Ctx *c, const Node *q, int pos) {
  int forall = q->kind == N_FORALL;
  if (pos == q->nbound) {
    if (!guard_ok(c, q)) return forall ? 1 : 0;
    return eval(c, q->a);
  }
  for (int v = 0; v < c->p->k; v++) {
    c->env[q->first_slot + pos] = v;
    int r = eval_quant(c, q, pos + 1);
    if (forall && !r) return 0;
    if (!forall && r) return 1;
  }
  return forall ? 1 : 0;
}

static int eval(Ctx *c, const Node *n) {
  switch (n->kind) {
    case N_CONST: return n->value;
    case N_ATOM: {
      const Family *f = &c->p->fam[n->fam];
      int tup[OR_MAX_ARITY];
      for (int i = 0; i < n->nidx; i++) tup[i] = n->targ[i] ? term_value(c, n->targ[i]) : idx_value(c, n->idx[i]);
      long r = tuple_rank(f, c->p->k, tup);
      if (r < 0) { c->bad = 1; return 0; }
      if (f->is_const) {
        long lin = 0;
        for (int i = 0; i < f->arity; i++) lin = lin * c->p->k + tup[i];
        return f->bits[lin];
      }
      return letter_value(c->p, c->j, f->first_id + (int)r);
    }
    case N_EQ: return term_value(c, n->lhs) == term_value(c, n->rhs);
    case N_NOT: return !eval(c, n->a);
    case N_AND: return eval(c, n->a) && eval(c, n->b);
    case N_OR: return eval(c, n->a) || eval(c, n->b);
    case N_XOR: return eval(c, n->a) != eval(c, n->b);
    case N_IMP: return !eval(c, n->a) || eval(c, n->b);
    case N_IFF: return eval(c, n->a) == eval(c, n->b);
    case N_FORALL:
    case N_EXISTS: return eval_quant(c, n, 0);
  }
  return 0;
}

/* every index inside a term names a domain element */
static int check_term(Ctx *c, const Term *t) {
  if (t->fam < 0) {
    int v = idx_value(c, t->idx);
    return v >= 0 && v < c->p->k;
  }
  for (int i = 0; i < t->nargs; i++)
    if (!check_term(c, t->args[i])) return 0;
  return 1;
}

/* every atom instance must name a declared tuple: checked by a full walk
   (no short-circuit) so that errors do not depend on j */
static int check_atoms(Ctx *c, const Node *n) {
  switch (n->kind) {
    case N_CONST: return 1;
    case N_EQ: return check_term(c, n->lhs) && check_term(c, n->rhs);
    case N_ATOM: {
      const Family *f = &c->p->fam[n->fam];
      int tup[OR_MAX_ARITY];
      for (int i = 0; i < n->nidx; i++) {
        if (n->targ[i]) {
          if (!check_term(c, n->targ[i])) return 0;
          tup[i] = 0;   /* any element: '<' families take no function terms */
        } else {
          tup[i] = idx_value(c, n->idx[i]);
        }
      }
      return tuple_rank(f, c->p->k, tup) >= 0;
    }
    case N_NOT: return check_atoms(c, n->a);
    case N_FORALL:
    case N_EXISTS: {
      int total = 1;
      int nb = n->nbound;
      long combos = 1;
      for (int i = 0; i < nb; i++) combos *= c->p->k;
      for (long t = 0; t < combos; t++) {
        long r = t;
        for (int i = nb - 1; i >= 0; i--) { c->env[n->first_slot + i] = (int)(r % c->p->k); r /= c->p->k; }
        if (guard_ok(c, n)) total &= check_atoms(c, n->a);
      }
      return total;
    }
    default: return check_atoms(c, n->a) && check_atoms(c, n->b);
  }
}

/* An assume line kills letters (Sec. 3.3; the assumptions dictionary of
   Sec. 4.2): it must be a conjunction of literals, possibly under universal
   quantifiers; each literal fixes its letter (atom: 1, negated atom: 0), and
   a later assignment of the same letter replaces an earlier one. */
static int apply_assume(Ctx *c, const Node *n, int value) {
  switch (n->kind) {
    case N_CONST: return n->value == 1 && value == 1;
    case N_ATOM: {
      const Family *f = &c->p->fam[n->fam];
      if (f->is_const) return 0;
      int tup[OR_MAX_ARITY];
      for (int i = 0; i < n->nidx; i++) {
        if (n->targ[i]) return 0;
        tup[i] = idx_value(c, n->idx[i]);
      }
      long r = tuple_rank(f, c->p->k, tup);
      if (r < 0) return 0;
      ((oracle_prog *)c->p)->fixed[f->first_id + r] = (signed char)value;
      return 1;
    }
    case N_EQ: {
      /* m(a..) = b with plain a.., b (either side): the value of m at a.. */
      const Term *app = n->lhs->fam >= 0 ? n->lhs : n->rhs, *val = n->lhs->fam >= 0 ? n->rhs : n->lhs;
      if (app->fam < 0 || val->fam >= 0) return 0;
      const Family *f = &c->p->fam[app->fam];
      int args[OR_MAX_ARITY];
      for (int i = 0; i < app->nargs; i++) {
        if (app->args[i]->fam >= 0) return 0;
        args[i] = idx_value(c, app->args[i]->idx);
        if (args[i] < 0 || args[i] >= c->p->k) return 0;
      }
      int b = idx_value(c, val->idx);
      if (b < 0 || b >= c->p->k) return 0;
      long base = fun_base(c->p, f, args);
      oracle_prog *w = (oracle_prog *)c->p;
      if (value)
        for (int u = 0; u < c->p->k; u++) w->fixed[base + u] = (signed char)(u == b);
      else
        w->fixed[base + b] = 0;
      return 1;
    }
    case N_NOT:
      if (n->a->kind != N_ATOM && n->a->kind != N_EQ) return 0;
      return apply_assume(c, n->a, !value);
    case N_AND:
      if (!value) return 0;
      return apply_assume(c, n->a, 1) && apply_assume(c, n->b, 1);
    case N_FORALL: {
      if (!value) return 0;
      int nb = n->nbound, ok = 1;
      long combos = 1;
      for (int i = 0; i < nb; i++) combos *= c->p->k;
      for (long t = 0; t < combos && ok; t++) {
        long r = t;
        for (int i = nb - 1; i >= 0; i--) { c->env[n->first_slot + i] = (int)(r % c->p->k); r /= c->p->k; }
        if (guard_ok(c, n)) ok = apply_assume(c, n->a, 1);
      }
      return ok;
    }
    default: return 0;
  }
}

/* ------------------------------------------------------------------ */
/* public interface (ctypes)                                            */

int oracle_parse(const char *text, int k, oracle_prog **out, char *err, int errlen) {
  *out = NULL;
  if (k < 1 || k > 64) { snprintf(err, (size_t)errlen, "domain size must be 1..64"); return 1; }
  oracle_prog *p = (oracle_prog *)calloc(1, sizeof(oracle_prog));
  p->k = k;
  Parser ps;
  memset(&ps, 0, sizeof ps);
  ps.s = text;
  ps.p = p;
  ps.line = 1;
  int cap = 16;
  p->axioms = (Node **)calloc((size_t)cap, sizeof(Node *));
  while (ps.s[ps.pos] && !ps.err[0]) {
    skip_ws(&ps);
    char c = ps.s[ps.pos];
    if (c == '\n') { ps.pos++; ps.line++; continue; }
    if (c == 0) break;
    int save = ps.pos;
    char word[64];
    int have = read_name(&ps, word);
    if (have && strcmp(word, "var") == 0 && (ps.s[ps.pos] == ' ' || ps.s[ps.pos] == '\t')) {
      do { if (!parse_decl(&ps, 0, 0)) break; } while (accept(&ps, ","));
    } else if (have && strcmp(word, "fun") == 0 && (ps.s[ps.pos] == ' ' || ps.s[ps.pos] == '\t')) {
      do { if (!parse_decl(&ps, 0, 1)) break; } while (accept(&ps, ","));
    } else if (have && strcmp(word, "const") == 0 && (ps.s[ps.pos] == ' ' || ps.s[ps.pos] == '\t')) {
      parse_decl(&ps, 1, 0);
    } else if (have && strcmp(word, "assume") == 0 && (ps.s[ps.pos] == ' ' || ps.s[ps.pos] == '\t')) {
      Node *f = parse_formula(&ps);
      if (f) {
        p->assumes = (Node **)realloc(p->assumes, sizeof(Node *) * (size_t)(p->nassume + 1));
        p->assumes[p->nassume++] = f;
      }
    } else {
      /* optional label:  name '=' formula   (but not '==', and not an
         equation whose left side is a declared function symbol) */
      if (have) {
        skip_ws(&ps);
        if (!(ps.s[ps.pos] == '=' && ps.s[ps.pos + 1] != '=') || find_family(p, word) >= 0) ps.pos = save;
        else ps.pos++;
      } else {
        ps.pos = save;
      }
      Node *f = parse_formula(&ps);
      if (f) {
        if (p->naxioms == cap) { cap *= 2; p->axioms = (Node **)realloc(p->axioms, sizeof(Node *) * (size_t)cap); }
        p->axioms[p->naxioms++] = f;
      }
    }
    if (ps.err[0]) break;
    skip_ws(&ps);
    if (ps.s[ps.pos] && ps.s[ps.pos] != '\n') set_err(&ps, "unexpected text after the end of a line");
  }
  p->nletters = p->nvars;
  for (int v = 0; v < OR_MAX_LETTERS; v++) p->fixed[v] = -1;
  if (!ps.err[0]) {
    Ctx c;
    memset(&c, 0, sizeof c);
    c.p = p;
    for (int i = 0; i < p->nassume && !ps.err[0]; i++)
      if (!apply_assume(&c, p->assumes[i], 1))
        snprintf(ps.err, sizeof ps.err, "assume line %d is not a conjunction of literals over declared letters", i + 1);
    /* free letters keep their declaration order */
    int nf = 0;
    for (int v = 0; v < p->nletters; v++)
      if (p->fixed[v] < 0) p->bit_of[v] = nf++;
    p->nvars = nf;
    if (nf > 64 && !ps.err[0]) snprintf(ps.err, sizeof ps.err, "more than 64 free variables");
    for (int i = 0; i < p->naxioms && !ps.err[0]; i++)
      if (!check_atoms(&c, p->axioms[i])) { snprintf(ps.err, sizeof ps.err, "axiom %d names an undeclared tuple", i + 1); break; }
  }
  if (ps.err[0]) {
    snprintf(err, (size_t)errlen, "%s", ps.err);
    free_prog(p);
    return 1;
  }
  *out = p;
  return 0;
}

void oracle_free(oracle_prog *p) { free_prog(p); }
int oracle_num_vars(const oracle_prog *p) { return p->nvars; }
int oracle_num_letters(const oracle_prog *p) { return p->nletters; }

/* the value of the theory (conjunction of axioms) under mu_j */
int oracle_eval(const oracle_prog *p, uint64_t j) {
  if (!functional(p, j)) return 0;
  Ctx c;
  memset(&c, 0, sizeof c);
  c.p = p;
  c.j = j;
  for (int i = 0; i < p->naxioms; i++)
    if (!eval(&c, p->axioms[i])) return 0;
  return 1;
}

/* Assignments j in [lo, hi): count of models; optional table bits (word
   (j-lo)>>6 of table, bit (j-lo)&63; the caller zeroes it); optional list of
   the first `cap` models in ascending order, with the total in *nmodels. */
void oracle_range(const oracle_prog *p, uint64_t lo, uint64_t hi, uint64_t *count,
                  uint64_t *table, uint64_t *models, uint64_t cap, uint64_t *nmodels) {
  uint64_t cnt = 0;
  for (uint64_t j = lo; j < hi; j++) {
    if (oracle_eval(p, j)) {
      if (table) table[(j - lo) >> 6] |= 1ull << ((j - lo) & 63);
      if (models && cnt < cap) models[cnt] = j;
      cnt++;
    }
  }
  *count = cnt;
  if (nmodels) *nmodels = cnt;
}

/* Subcube of 2^n: the variables in `mask` fixed to the bits of `vals`, the
   others free.  The free variables, lowest first, go to freev; the return
   value is their number nf.  The subcube has 2^nf assignments; a count over
   it fits a u64 only for nf <= 63, so the counters below refuse nf = 64. */
static int cube_free_vars(const oracle_prog *p, uint64_t mask, int freev[64]) {
  int nf = 0;
  for (int i = 0; i < p->nvars; i++)
    if (!((mask >> i) & 1)) freev[nf++] = i;
  return nf;
}

/* the assignment integer of point t (bit b of t = the b-th free variable) */
static uint64_t cube_point(uint64_t mask, uint64_t vals, const int *freev, int nf, uint64_t t) {
  uint64_t j = vals & mask;
  for (int b = 0; b < nf; b++) j |= ((t >> b) & 1ull) << freev[b];
  return j;
}

/* Number of assignments of a subcube with nf free variables, or
   ORACLE_CUBE_TOO_BIG (all ones) for nf = 64, whose count need not fit. */
uint64_t oracle_cube_size(int nf) {
  if (nf < 0 || nf > 63) return ~0ull;
  return 1ull << nf;
}

/* models with the variables in `mask` fixed to the bits of `vals`: the
   definition (Prop. 2.2) restricted to a subcube, by a loop over the free
   variables' values.  Returns all ones when 64 variables are free. */
uint64_t oracle_count_cube(const oracle_prog *p, uint64_t mask, uint64_t vals) {
  int freev[64];
  const int nf = cube_free_vars(p, mask, freev);
  const uint64_t total = oracle_cube_size(nf);
  if (total == ~0ull) return ~0ull;
  uint64_t cnt = 0;
  for (uint64_t t = 0; t < total; t++) cnt += (uint64_t)oracle_eval(p, cube_point(mask, vals, freev, nf, t));
  return cnt;
}

/* count_cube with the free assignments split statically across threads:
   the same subcube, the same points, the same refusal at 64 free variables */
uint64_t oracle_count_cube_par(const oracle_prog *p, uint64_t mask, uint64_t vals, int nthreads) {
  int freev[64];
  const int nf = cube_free_vars(p, mask, freev);
  const uint64_t total = oracle_cube_size(nf);
  if (total == ~0ull) return ~0ull;
  uint64_t cnt = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for reduction(+ : cnt) schedule(static)
#endif
  for (uint64_t t = 0; t < total; t++) cnt += (uint64_t)oracle_eval(p, cube_point(mask, vals, freev, nf, t));
  (void)nthreads;
  return cnt;
}

/* the same count over [lo, hi) with the range split statically across
   threads (timing of the CPU baseline only; identical arithmetic) */
uint64_t oracle_count_par(const oracle_prog *p, uint64_t lo, uint64_t hi, int nthreads) {
  uint64_t cnt = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for reduction(+ : cnt) schedule(static)
#endif
  for (long long j = (long long)lo; j < (long long)hi; j++) cnt += (uint64_t)oracle_eval(p, (uint64_t)j);
  (void)nthreads;
  return cnt;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
