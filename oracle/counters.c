/*
 * counters.c -- TEST INFRASTRUCTURE ONLY.  Independent backtracking counters
 * of labelled structures, written without any formula: they pin the oracle
 * and give exact values at sizes the oracle cannot finish (n = 36).
 */
#include <stdint.h>
#include <string.h>

/* transitive relations on k points: decide the pairs (i,j) in row-major order;
   after each decision check every transitivity instance a->b, b->c => a->c
   whose three pairs are decided and that involves the new pair */
static int TK;
static unsigned char R[8][8], D[8][8];

static int trans_ok(int i, int j) {
  for (int x = 0; x < TK; x++) {
    /* (i,j) as the first pair: i->j, j->x => i->x */
    if (D[j][x] && D[i][x] && R[i][j] && R[j][x] && !R[i][x]) return 0;
    /* (i,j) as the second pair: x->i, i->j => x->j */
    if (D[x][i] && D[x][j] && R[x][i] && R[i][j] && !R[x][j]) return 0;
    /* (i,j) as the implied pair: i->x, x->j => i->j */
    if (D[i][x] && D[x][j] && R[i][x] && R[x][j] && !R[i][j]) return 0;
  }
  return 1;
}

static uint64_t trans_rec(int p) {
  if (p == TK * TK) return 1;
  int i = p / TK, j = p % TK;
  uint64_t total = 0;
  D[i][j] = 1;
  for (int v = 0; v < 2; v++) {
    R[i][j] = (unsigned char)v;
    if (trans_ok(i, j)) total += trans_rec(p + 1);
  }
  D[i][j] = 0;
  R[i][j] = 0;
  return total;
}

uint64_t counter_transitive(int k) {
  if (k < 0 || k > 8) return 0;
  TK = k;
  memset(R, 0, sizeof R);
  memset(D, 0, sizeof D);
  return trans_rec(0);
}

/* triangle-free graphs on k vertices: decide the edges (a,b), a<b, in
   lexicographic order; an edge may be present only if no decided vertex c
   is adjacent to both ends */
static int GK, NE, EA[64], EB[64];
static unsigned char ADJ[16][16];

static uint64_t tri_rec(int e) {
  if (e == NE) return 1;
  int a = EA[e], b = EB[e];
  uint64_t total = tri_rec(e + 1);   /* edge absent */
  int ok = 1;
  for (int c = 0; c < GK && ok; c++)
    if (ADJ[a][c] && ADJ[b][c]) ok = 0;
  if (ok) {
    ADJ[a][b] = ADJ[b][a] = 1;
    total += tri_rec(e + 1);
    ADJ[a][b] = ADJ[b][a] = 0;
  }
  return total;
}

uint64_t counter_triangle_free(int k) {
  if (k < 0 || k > 11) return 0;
  GK = k;
  NE = 0;
  memset(ADJ, 0, sizeof ADJ);
  for (int a = 0; a < k; a++)
    for (int b = a + 1; b < k; b++) {
      EA[NE] = a;
      EB[NE] = b;
      NE++;
    }
  return tri_rec(0);
}

/* partial orders on k points: decide the pairs (i,j), i != j, in row-major
   order (the diagonal is forced); reject a new pair that breaks
   antisymmetry or transitivity among decided pairs */
static int PK;
static unsigned char PR[10][10], PD[10][10];

static int poset_ok(int i, int j) {
  if (PR[i][j] && PD[j][i] && PR[j][i]) return 0;
  for (int x = 0; x < PK; x++) {
    if (PD[j][x] && PD[i][x] && PR[i][j] && PR[j][x] && !PR[i][x]) return 0;
    if (PD[x][i] && PD[x][j] && PR[x][i] && PR[i][j] && !PR[x][j]) return 0;
    if (PD[i][x] && PD[x][j] && PR[i][x] && PR[x][j] && !PR[i][j]) return 0;
  }
  return 1;
}

/* at a leaf (every pair decided): 1, or with PSPECIAL set, 1 only when some
   element is comparable with every element */
static int PSPECIAL;

static uint64_t poset_leaf(void) {
  if (!PSPECIAL) return 1;
  for (int a = 0; a < PK; a++) {
    int all = 1;
    for (int b = 0; b < PK && all; b++) all = PR[a][b] || PR[b][a];
    if (all) return 1;
  }
  return 0;
}

static uint64_t poset_rec(int p) {
  if (p == PK * PK) return poset_leaf();
  int i = p / PK, j = p % PK;
  if (i == j) return poset_rec(p + 1);
  uint64_t total = 0;
  PD[i][j] = 1;
  for (int v = 0; v < 2; v++) {
    PR[i][j] = (unsigned char)v;
    if (poset_ok(i, j)) total += poset_rec(p + 1);
  }
  PD[i][j] = 0;
  PR[i][j] = 0;
  return total;
}

uint64_t counter_posets(int k) {
  if (k < 0 || k > 9) return 0;
  PSPECIAL = 0;
  PK = k;
  memset(PR, 0, sizeof PR);
  memset(PD, 0, sizeof PD);
  for (int i = 0; i < k; i++) PR[i][i] = PD[i][i] = 1;
  return poset_rec(0);
}

/* partial orders on k points with a special element: one comparable with
   every element (the SO.txt example of Sec. 4.2), by the same search */
uint64_t counter_posets_special(int k) {
  if (k < 0 || k > 9) return 0;
  PSPECIAL = 1;
  PK = k;
  memset(PR, 0, sizeof PR);
  memset(PD, 0, sizeof PD);
  for (int i = 0; i < k; i++) PR[i][i] = PD[i][i] = 1;
  uint64_t r = poset_rec(0);
  PSPECIAL = 0;
  return r;
}
