/*
 * fbg.h -- C ABI of the free-Boolean-generator evaluator (libfbg.so).
 *
 * Method (Mijajlovic & Pejovic, "Computing finite models using free Boolean
 * generators"): a first-order theory T over a k-element domain is translated
 * into a propositional formula t(x_0..x_{n-1}) (the map * of Sec. 3.1); t is
 * evaluated bitwise over the free generators b_i of the free Boolean algebra
 * with n generators (Sec. 2.2), which gives the vector d whose position j is
 * t(mu_j) -- the full DNF of t (Prop. 2.2, Sec. 2.3).  Its number of ones is
 * the number l_{T,n} of labelled models (Sec. 3.2).
 *
 * Conventions fixed by this library:
 *   - assignment integer j in [0, 2^n): variable x_i takes bit i of j (the
 *     generator matrix of Sec. 2.2 with the index order flipped: x_i is the
 *     paper's b_{n-i});
 *   - truth table bit j lives in 64-bit word j>>6, bit j&63; for n < 6 the
 *     single word's bits >= 2^n are 0;
 *   - variables are numbered in declaration order, each declared family in
 *     lexicographic tuple order (r(i,j) of a k x k relation is i*k+j);
 *   - model lists are ascending in j.
 *
 * Formula text (the script language of Sec. 4.2, subset plus declarations):
 *   var x, y, r(S,S), e(S<S)      declarations ('<' = strictly increasing)
 *   const E(S,S) = 0110...        constant relation, k^arity bits
 *   [label =] formula             one axiom per line; the theory is their
 *                                 conjunction.  Operators ~ & ^ | with Python
 *                                 precedence, then -> (right assoc) and <->;
 *                                 constants 0 1; bounded quantifiers
 *                                 A[i,j:S | i<j] and E[i:S2] (S = range(k),
 *                                 S2/S3 = ordered tuples of distinct
 *                                 elements) scoping over the next unary term,
 *                                 optionally followed by '.'; '#' comments.
 *   assume formula                killing variables (Sec. 3.3; the assumptions
 *                                 of Sec. 4.2): a conjunction of literals,
 *                                 possibly under A[..], fixes each letter
 *                                 (atom 1, negated atom 0); later lines
 *                                 override earlier ones.  Killed letters are
 *                                 not variables: the free letters keep their
 *                                 declaration order and n counts only them.
 *
 * Ownership and threads: the caller owns every device buffer and every CUDA
 * stream passed in (streams as cudaStream_t cast to void*, NULL = the legacy
 * default stream).  A program owns its compiled kernels' scratch (a few
 * counters and per-unit partial counts, allocated on first use, freed by
 * fbg_program_free).  Calls on one program must not overlap; distinct
 * programs may be used from different threads.  No call falls back to the
 * CPU: without a CUDA device every evaluation returns FBG_ECUDA.
 * Errors: every call returns an fbg_status; fbg_last_error() gives the
 * calling thread's last message.
 */
#ifndef FBG_H
#define FBG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fbg_program fbg_program;
typedef struct fbg_batch fbg_batch;
typedef struct fbg_server fbg_server;

typedef enum {
  FBG_OK = 0,
  FBG_EINVAL = 1,      /* bad argument (null pointer, wrong buffer size, bad option) */
  FBG_EPARSE = 2,      /* formula text does not parse or names an undeclared tuple */
  FBG_ETOOBIG = 3,     /* n > 63 for counts, n > 40 for tables / model lists,
                          or a program too large for the interpreter */
  FBG_ENOMEM = 4,      /* device allocation failed */
  FBG_ECUDA = 5,       /* CUDA runtime error (including: no device) */
  FBG_EJIT = 6,        /* NVRTC compilation of the specialised kernel failed */
  FBG_ETIMEOUT = 7,    /* a wait exceeded its limit */
  FBG_ECANCELLED = 8,  /* request cancelled */
  FBG_EBUSY = 9        /* server: result not ready yet */
} fbg_status;

/* evaluation engines */
enum {
  FBG_ENGINE_AUTO = 0,   /* specialised kernel for single programs, else interpreter */
  FBG_ENGINE_JIT = 1,    /* NVRTC straight-line kernel (count and table) */
  FBG_ENGINE_INTERP = 2  /* generic bytecode interpreter kernel */
};

/* program options (fbg_set_option) */
enum {
  FBG_OPT_ENGINE = 1,          /* FBG_ENGINE_* */
  FBG_OPT_PRUNE = 2,           /* 1 (default): levels whose partial conjunction is
                                  zero skip their inner levels; 0: evaluate every word */
  FBG_OPT_REGS_LOG2 = 3,       /* JIT: 32-bit registers per thread tile, log2 (1..3, default 2) */
  FBG_OPT_WARPS_LOG2 = 4,      /* JIT: warps per block, log2 (0..5, default 3) */
  FBG_OPT_UNIT_BITS = 5,       /* max block-uniform unit bits (default 13) */
  FBG_OPT_LOOP_LEVEL_BITS = 6, /* bits per loop level (0, the default: 4 for the NVRTC kernels, 1 for
                                  the interpreter, which prunes after every letter; the interpreter
                                  widens levels to hold at most 8) */
  FBG_OPT_SEARCH_ORDER = 7,    /* counts: 1 (default) heuristic variable order, 0 identity */
  FBG_OPT_MIN_BLOCKS = 8,      /* JIT: __launch_bounds__ min blocks per SM (default 2) */
  FBG_OPT_STATS = 9,           /* 1: kernels carry level counters and record executed level
                                  iterations (fbg_exec_stats); changing it rebuilds the
                                  kernels and drops a unit order (fbg_schedule_units) */
  FBG_OPT_INNER_BITS = 10,     /* JIT: bits of the innermost loop level, which is emitted
                                  unrolled with its generator words folded as constants
                                  (0 = default: as the other levels; 1..5) */
  FBG_OPT_SPLIT_ITEMS = 11,    /* 1: fbg_schedule_units hands a long item out as up to 16
                                  pieces over the first loop level; 0 (default): whole items.
                                  Pieces shorten a lone launch whose longest items end it
                                  late; launches that share the GPU already fill that tail.
                                  Read by the next fbg_schedule_units; no rebuild */
  FBG_OPT_POPC_COST = 12,      /* JIT count kernels: the cost of one POPC in lop3 issue slots that
                                  decides how many full adders (two lop3 each, one POPC saved)
                                  compress an innermost execution's result words before POPC:
                                  about (c*W - A) / (c + 2) for W words and A lop3; 0 = none,
                                  default 4 (POPC on the XU pipe at a quarter of the lop3 rate);
                                  0..16 */
  FBG_OPT_ORDER_SEED = 13,     /* counts: variant of the heuristic variable order (0 = default: ties
                                  go to the lowest letter; 1..255: ties broken by a seeded hash).
                                  The order decides how much of the space the level conjunctions
                                  prune; counts are the same under every order */
};

typedef struct {
  int n;                    /* number of propositional letters */
  int domain_k;
  int64_t dag_nodes;        /* hash-consed DAG after grounding */
  int64_t gates;            /* 2-input gates after level-aware lowering (count layout) */
  int64_t luts;             /* 3-input LUTs after mapping (count layout) */
  int nlevels;              /* 2 + loop levels */
  int64_t lop3_per_level[16];  /* lane-varying lop3.b32 per thread per execution of each level of
                                  the count kernel the current options build */
  int regs_log2, lane_bits, warp_bits, unit_bits;
  int loop_bits[8];
  int interp_slots;         /* shared-memory slots of the interpreter program */
} fbg_stats;

typedef struct {
  uint64_t level_iters[16]; /* warp-level executions of each level in the last count */
  double lop3_executed;     /* lop3.b32 lane operations those executions issued whose inputs vary
                               across lanes (the vector ALU pipe's work) */
  double lop3_nominal;      /* lane operations without pruning: every word evaluated */
  int engine;               /* engine that ran */
  double lop3_uniform;      /* warp operations of lop3 whose inputs are all warp-uniform (constants,
                               unit letters and loop counters; the compiler may run them on the
                               uniform pipe) */
} fbg_exec_stats;

/*
 * Compile formula text over the domain range(domain_k) (Sec. 3.1 map *, then
 * the hash-consed DAG with constants removed: the Reduction of Sec. 4.1).
 * Host only, no GPU work.  *out is owned by the caller (fbg_program_free).
 * Returns FBG_EPARSE with a message for bad text, FBG_ETOOBIG above 64 letters.
 */
fbg_status fbg_compile(const char *formula, int domain_k, fbg_program **out);

/* number n of propositional letters (the set P of Sec. 3.1), -1 on null */
int fbg_num_vars(const fbg_program *prog);

/* name of letter i, e.g. "r(2,0)"; FBG_EINVAL if i is out of range or len too small */
fbg_status fbg_var_name(const fbg_program *prog, int i, char *buf, size_t len);

fbg_status fbg_set_option(fbg_program *prog, int option, int64_t value);

fbg_status fbg_program_stats(fbg_program *prog, fbg_stats *out);

/*
 * Exact number of models l_{T,n} = popcount of d (Sec. 3.2): evaluates every
 * assignment, never stores d.  Synchronises `stream`; *out_count is host
 * memory.  n <= 63.
 */
fbg_status fbg_count(fbg_program *prog, void *stream, uint64_t *out_count);

/* as fbg_count, but writes the count to device memory dev_out (8 bytes,
   caller-owned, overwritten) and returns without synchronising.  One launch,
   no memset: the kernel's last warp writes *dev_out and zeroes the program's
   counters.  Launches of one program share those counters, so they must not
   overlap: issue them on one stream (or order them with events); different
   programs may run concurrently on different streams. */
fbg_status fbg_count_async(fbg_program *prog, void *stream, uint64_t *dev_out);

/*
 * One count launch per program, back to back on `stream` (no counterpart in
 * the paper: the plain one-launch-per-formula evaluation that the batch of
 * fbg_batch_* is measured against): progs[i]'s count goes to dev_out[i]
 * (caller-owned device memory, nprogs 64-bit words), as fbg_count_async
 * would write it.  Kernels are built on first use (NVRTC or interpreter per
 * each program's engine option).  Asynchronous; stops at the first error.
 */
fbg_status fbg_count_each(fbg_program **progs, size_t nprogs, void *stream, uint64_t *dev_out);

/*
 * Per-unit partial counts of the count layout: unit u fixes the letters
 * returned by fbg_unit_vars to the bits of u (bit b of u = value of letter
 * vars[b]); the counts sum to fbg_count.  dev_counts: nunits device u64s.
 * Synchronises `stream`.
 */
fbg_status fbg_count_units(fbg_program *prog, void *stream, uint64_t *dev_counts, uint64_t nunits);
/*
 * Models among the units [unit_begin, unit_end) of the count layout (clipped
 * to the unit count of fbg_unit_vars): a long count split into chunks whose
 * sums give fbg_count, e.g. to checkpoint and resume it.  Synchronises.
 */
fbg_status fbg_count_range(fbg_program *prog, void *stream, uint64_t unit_begin, uint64_t unit_end,
                           uint64_t *out_count);
fbg_status fbg_unit_vars(fbg_program *prog, int *vars, int max_vars, int *nvars, uint64_t *nunits);

/*
 * Full truth table d = t(b_1..b_n) (Prop. 2.2, Sec. 2.3) into caller-owned
 * device memory dev_words of exactly nwords = max(1, 2^(n-6)) 64-bit words
 * (bit j at word j>>6, bit j&63).  Asynchronous on `stream`.  n <= 40.
 */
fbg_status fbg_truth_table(fbg_program *prog, void *stream, uint64_t *dev_words, size_t nwords);

/*
 * Models of T* in ascending j (the valuations of out.txt, Sec. 4.2; each
 * decodes to a labelled model by the map h of Sec. 3.2): the first
 * min(cap, total) are written to caller-owned device memory dev_models;
 * *total (host) receives the exact number of models, *written the number
 * stored.  Synchronises `stream`.  n <= 40.
 * Engine: the specialised (NVRTC) kernel by default -- its layout makes every
 * (unit, warp slice) work item an interval of j; one pass counts each item's
 * models, a scan gives each item its first position, and a second pass has
 * each warp write its items' models in order (warp prefix sums of the
 * lanes' popcounts), skipping items that start at or past cap -- or the
 * interpreter (FBG_OPT_ENGINE = FBG_ENGINE_INTERP, or when the specialised
 * build fails under FBG_ENGINE_AUTO).  FBG_ETOOBIG above 2^26 items.
 */
fbg_status fbg_enumerate_models(fbg_program *prog, void *stream, uint64_t *dev_models, size_t cap,
                                uint64_t *total, uint64_t *written);

/*
 * Unit ranges of truth tables and model lists (no counterpart in the paper;
 * the assignment space split by its top letters, one range per GPU).  The
 * specialised kernel's table layout (mode 1) and model-list layout (mode 2)
 * each have *nunits units; unit u holds the assignments j with j >> (n - log2 nunits) == u, a
 * contiguous range of *words_per_unit 64-bit table words.  Ranges need the
 * specialised engine (FBG_EINVAL when the program asks for the
 * interpreter); n <= 40.
 */
fbg_status fbg_table_units(fbg_program *prog, int mode, uint64_t *nunits, uint64_t *words_per_unit);

/*
 * The table words of units [unit_begin, unit_end): nwords must be
 * (unit_end - unit_begin) * words_per_unit; dev_words[i] is word
 * unit_begin * words_per_unit + i of the whole table (bit j at word j>>6,
 * bit j&63).  Asynchronous.  FBG_EINVAL for an empty or out-of-range range
 * or when a unit is smaller than one 64-bit word (then only the whole range
 * is allowed).
 */
fbg_status fbg_truth_table_range(fbg_program *prog, void *stream, uint64_t unit_begin, uint64_t unit_end,
                                 uint64_t *dev_words, size_t nwords);

/*
 * The models among units [unit_begin, unit_end) of the model-list layout, in
 * ascending j: the first min(cap, *total) are written to dev_models, *total
 * is the exact number of models in the range.  Concatenating the lists of
 * consecutive ranges in order gives the list of fbg_enumerate_models.
 * Synchronises `stream`.
 */
fbg_status fbg_enumerate_models_range(fbg_program *prog, void *stream, uint64_t unit_begin, uint64_t unit_end,
                                      uint64_t *dev_models, size_t cap, uint64_t *total, uint64_t *written);

/*
 * Count without any device allocation by the library.  The paper has no
 * counterpart of this entry point; it exists for callers that cannot let a
 * library call cudaMalloc -- a process whose caching allocator already owns
 * the free device memory, or code that must keep to a fixed, pre-reserved
 * budget -- while fbg_count allocates the program's device buffers and
 * scratch on first use.  Here the work counters, program descriptor,
 * bytecode, constants and work queue of the interpreter count kernel live in
 * one file-scope device array of FBG_NOALLOC_SCRATCH_BYTES, held by every GPU
 * that loads the library until the process exits; no cudaMalloc, cudaFree or
 * other allocating routine is called.  Programs whose bytecode and queue do
 * not fit return FBG_ETOOBIG with the size they need.
 * The caller passes the compiled program and dev_out, one caller-owned device
 * u64 that receives the count (overwritten).  The call synchronises `stream`.
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress, with the device current); make that first
 * call before any stream capture.  All calls share the one array, which
 * keeps the last call's contents (counters are cleared by each call): calls
 * that overlap on the GPU -- from several host threads or streams -- race and
 * must be serialised by the caller.
 */
#define FBG_NOALLOC_SCRATCH_BYTES (128u * 1024u)
fbg_status fbg_count_noalloc(fbg_program *prog, void *stream, uint64_t *dev_out);

/*
 * Autotuner of the specialised kernel (mode 0 count, 1 truth table, n <= 34):
 * searches the layout knobs -- FBG_OPT_LOOP_LEVEL_BITS (also the depth of
 * the unrolled innermost level), FBG_OPT_REGS_LOG2 (words per thread),
 * FBG_OPT_MIN_BLOCKS, FBG_OPT_WARPS_LOG2 (block shape), FBG_OPT_UNIT_BITS --
 * one at a time from the current setting, compiling each candidate with
 * NVRTC and timing `reps` launches with CUDA events on `stream`; the program
 * keeps the fastest shape.  Table tuning allocates one table temporarily.
 */
typedef struct {
  double best_ms;
  int trials;
  int regs_log2, warps_log2, min_blocks, loop_level_bits, unit_bits;
  int inner_bits;
  int popc_cost;
  int order_seed;
} fbg_tune_result;
fbg_status fbg_autotune(fbg_program *prog, void *stream, int mode, int reps, fbg_tune_result *out);

/* executed work of the last fbg_count with FBG_OPT_STATS = 1, or of the last
   fbg_truth_table of the specialised kernel with FBG_OPT_STATS = 1 (which then
   synchronises its stream to read the level counters) */
fbg_status fbg_last_exec_stats(fbg_program *prog, fbg_exec_stats *out);

/* Diagnostics (no counterpart in the paper): host wall time, in seconds,
 * that this program has spent so far building specialised kernels (layout,
 * lowering, item pruning, source emission, the kernel cache, uploads; an
 * NVRTC compile when the cache misses) and inside fbg_count outside those
 * builds (launch, copy of the count, synchronisation).  FBG_EINVAL on null. */
fbg_status fbg_debug_host_times(const fbg_program *prog, double *build_s, double *count_s);

/*
 * Host compile caches (no counterpart in the paper; the host half of the
 * Translate and Reduction submodules of Sec. 4.1 is repeated work when the
 * same text comes back).  fbg_compile keeps the parsed and grounded theory of
 * the last 512 (text, domain_k) pairs; kernel builds keep the layout, LUT
 * program, emitted source or bytecode and the build-time item pruning of the
 * last 256 specialised and 512 interpreter builds, keyed by text, domain_k,
 * mode and every shape option.  Entries are immutable and shared; device
 * buffers stay per program.  out[0..8] receives hits, misses and entries of
 * the compile, specialised-build and interpreter-build caches.  With
 * clear != 0 the caches are emptied first (the counters are kept).
 * FBG_EINVAL on null.
 */
fbg_status fbg_debug_host_caches(int clear, uint64_t out[9]);

/* CUDA source of the specialised kernel (mode 0 count, 1 table, 2 model
   list), exactly as the kernel build compiles it with the current options;
   *len receives the size; buf may be NULL to query it */
fbg_status fbg_program_source(fbg_program *prog, int mode, char *buf, size_t *len);

/*
 * Diagnostic: the compiled program as JSON text -- which = 0 / 1 / 4: LUT
 * program of the specialised count / table / model-list kernel (layout,
 * constants per register, LUTs with levels); 2 / 3: interpreter bytecode of
 * the count / identity layout.  Used to check the compiler on a machine without a GPU; it does
 * not evaluate anything.  *len receives the size; buf may be NULL.
 * For which = 0 the layout also gives "split_bits" (the largest s of the
 * item pieces the count kernel takes, 0 when none), and the object gives
 * "alive_items" (the (unit, warp slice) items that can hold models, when
 * the build-time pruning removes any) and, once the count kernel is built,
 * "item_list_entries" (entries of the item list full-range counts hand out).
 */
fbg_status fbg_debug_dump(fbg_program *prog, int which, char *buf, size_t *len);

/* Longest-first unit order (no counterpart in the paper).  The work of a
 * unit of fbg_unit_vars depends on how much of its subspace the level
 * conjunctions prune, and a few heavy units can keep a few SMs busy long
 * after the rest are idle.  This call runs one count launch that times every
 * item (unit, warp slice) on the GPU's nanosecond timer, with
 * FBG_OPT_SPLIT_ITEMS splits each item that takes longer than half the mean
 * load of a warp into 2, 4, 8 or 16 pieces over the values of the first loop
 * level (only when that level is a runtime loop), sorts the items and pieces by time,
 * longest first, and keeps that order on the device: later full-range
 * counts of the program through fbg_count and fbg_count_async hand out items
 * in it.  Results do not depend on the order or the pieces.  The
 * order is dropped when an option rebuilds the kernel.  Synchronises the
 * stream; allocates 8 bytes per item temporarily and keeps 4 bytes per item
 * or piece.  FBG_EINVAL when the program does not use the NVRTC engine,
 * FBG_ETOOBIG above 2^24 items. */
fbg_status fbg_schedule_units(fbg_program *prog, void *stream);

/* Diagnostics (no counterpart in the paper): one count launch of the NVRTC
 * engine that records, per unit u of fbg_unit_vars, dev_trace[2u] = the
 * nanoseconds all warps spent on u (summed over warp slices) and
 * dev_trace[2u+1] = the earliest start time of u on the GPU's nanosecond timer.
 * dev_trace: device memory of 2 * nunits u64 words, caller-owned, written
 * whole; nunits must equal the unit count.  Units are evaluated one at a time
 * while tracing, so the launch is slower than fbg_count.  Synchronises the
 * stream.  FBG_EINVAL when the program does not use the NVRTC engine. */
fbg_status fbg_debug_unit_trace(fbg_program *prog, void *stream, uint64_t *dev_trace, uint64_t nunits);

/* Diagnostics: the per-item times that fbg_schedule_units sorts.  dev_ns[u *
 * S + w] = nanoseconds the warp spent on unit u, warp slice w (S = 2^warp
 * bits of the layout, fbg_debug_dump); nitems must be nunits * S. */
fbg_status fbg_debug_item_trace(fbg_program *prog, void *stream, uint64_t *dev_ns, uint64_t nitems);

/*
 * Diagnostics without a device: the NVRTC sources of the specialised count
 * kernels a batch of these programs would build, one after another ("" when
 * none would be specialised), and an NVRTC
 * compile of a kernel body (the library's device headers are available to it)
 * with the library's options; log receives the NVRTC/ptxas messages.
 */
fbg_status fbg_debug_batch_source(fbg_program *const *progs, int nprogs, char *buf, size_t *len);
fbg_status fbg_debug_nvrtc_compile(const char *body, char *log, size_t loglen);
/* compile (without loading) the specialised kernels a batch of these programs
   would build; *specialized receives the number that compile */
fbg_status fbg_debug_batch_build(fbg_program *const *progs, int nprogs, int *specialized, char *log, size_t loglen);

/* The integer-logic roof, measured (no counterpart in the paper): one launch
 * of a kernel in which every thread runs 16 independent lop3.b32 chains, no
 * memory traffic; *tops = lop3.b32 lane-operations per second / 1e12.
 * Synchronises the stream. */
fbg_status fbg_probe_lop3_rate(void *stream, double *tops);

/* NVRTC/ptxas log of the last specialised-kernel build (registers, spills) */
const char *fbg_program_jit_log(fbg_program *prog);

void fbg_program_free(fbg_program *prog);

/* calling thread's last error message ("" if none) */
const char *fbg_last_error(void);

/*
 * Batch (the inner loop of the counting procedure of Sec. 3.4 runs over many
 * reduced formulas): count many programs together.  Interpreted programs share
 * one persistent interpreter launch fed by a device work queue of (program,
 * unit range) items, largest first.  Programs must outlive the batch.
 * max_item_units bounds the units per queue item (0 = automatic).  flags:
 * FBG_BATCH_GRAPH captures the whole run (memset, launches, result copy) in a
 * CUDA graph on the first run and replays it afterwards;
 * FBG_BATCH_SPECIALIZE compiles the distinct programs with n >= 20 that carry
 * the most nominal work (at most 512) into specialised count kernels (NVRTC,
 * in parallel, 180 s deadline); each instance of such a program is one
 * self-resetting launch of its kernel, the launches spread longest first (by
 * one timed launch per kernel at creation) over eight side streams, the
 * interpreter launch on a ninth; every other program is interpreted.
 */
enum { FBG_BATCH_GRAPH = 1, FBG_BATCH_SPECIALIZE = 2 };
fbg_status fbg_batch_create(fbg_program *const *progs, int nprogs, uint64_t max_item_units, int flags,
                            fbg_batch **out);
/* enqueue one evaluation of every program on `stream` (asynchronous) */
fbg_status fbg_batch_run(fbg_batch *batch, void *stream);
/* wait for the last run and copy the exact counts into host memory (nprogs u64) */
fbg_status fbg_batch_results(fbg_batch *batch, void *stream, uint64_t *host_counts);
/* queue geometry: items, total units, blocks launched, specialised programs */
fbg_status fbg_batch_info(fbg_batch *batch, uint64_t *items, uint64_t *units, int *grid, int *specialized);
/* per program (nprogs ints): 1 if the batch kernel runs it specialised, 0 if interpreted */
fbg_status fbg_batch_program_kinds(fbg_batch *batch, int *specialized);
void fbg_batch_free(fbg_batch *batch);

/*
 * Serving loop: requests (formula text, domain, count or enumerate) are
 * compiled on submission (count requests with up to 2^20 units, model lists
 * with up to 2^16, one letter per loop level), admitted while their device
 * memory fits the budget and a slot is free, and evaluated in ticks with the
 * interpreter kernel (no kernel compile on the tick loop); a request whose
 * units are all removed at build time finishes at admission with no models;
 * each tick runs one launch over a
 * share of the work of every admitted request (chunks of units), so requests
 * that arrive while others run join the next tick.  Partial counts stay on
 * the device across ticks.  A model list is tick work as well: its units are
 * counted in the same launch, each into its own counter; in the tick that
 * counts its last unit, a scan gives every unit its first position and one
 * more launch (shared by all model lists finishing in that tick) writes the
 * models in ascending j into a device buffer of `cap` words, from which the
 * first min(cap, total) reach the result.  Count requests whose text recurs
 * move to a specialised kernel once a background thread has compiled it
 * (jit_min_n, jit_after).  A host thread drives the ticks on
 * its own stream, two ticks in flight (it prepares and enqueues the next tick
 * while the GPU runs the current one); per-request device buffers come from
 * the stream-ordered allocator.
 */
typedef struct {
  uint64_t mem_budget_bytes;   /* device memory for admitted requests (0 = 1 GiB) */
  uint64_t tick_units;         /* max units evaluated per tick (0 = 65536) */
  int max_inflight;            /* max admitted requests (0 = 4096) */
  uint64_t tick_assignments;   /* assignments evaluated per tick, at least one unit per admitted
                                  request (0 = 2^36); requests with the least remaining work go
                                  first and finish in one tick when they fit a fair share */
  int jit_min_n;               /* recurring texts: a count request with at least this many letters
                                  (0 = 30; negative = never) whose (text, domain) has been submitted
                                  jit_after times gets a specialised count kernel, compiled by a
                                  background thread of the server (NVRTC), never by the tick loop;
                                  count requests of that text admitted once it is ready are counted
                                  by it (one launch over all their units, on a side stream that runs
                                  beside the tick's interpreter launch) */
  int jit_after;               /* submissions of one (text, domain) before its compile starts (0 = 2) */
  int jit_max_programs;        /* specialised programs a server keeps (0 = 64); texts beyond stay
                                  on the interpreter */
} fbg_server_options;

enum { FBG_MODE_COUNT = 0, FBG_MODE_ENUMERATE = 1 };

typedef struct {
  fbg_status status;
  uint64_t count;              /* exact number of models */
  uint64_t written;            /* enumerate: models stored */
  const uint64_t *models;      /* enumerate: host array of `written` models, owned by the server */
  double submit_s, admit_s, done_s;   /* server clock (seconds): entry to fbg_server_submit (before the
                                         request's compile), admission, result ready */
} fbg_result;

fbg_status fbg_server_create(const fbg_server_options *opt, fbg_server **out);
fbg_status fbg_server_submit(fbg_server *srv, const char *formula, int domain_k, int mode, uint64_t cap,
                             uint64_t *request_id);
/* FBG_OK with *out filled when done, FBG_EBUSY while pending */
fbg_status fbg_server_poll(fbg_server *srv, uint64_t request_id, fbg_result *out);
/* ids of requests finished since the last call, oldest first: up to max_ids
   go to ids[], *n receives how many (each finished request is handed out
   once; poll it for the result, then release it) */
fbg_status fbg_server_completed(fbg_server *srv, uint64_t *ids, size_t max_ids, size_t *n);
/* block until every submitted request is done (timeout_s <= 0: no limit) */
fbg_status fbg_server_drain(fbg_server *srv, double timeout_s);
/* release a finished request's result memory */
fbg_status fbg_server_release(fbg_server *srv, uint64_t request_id);
fbg_status fbg_server_stats(fbg_server *srv, uint64_t *ticks, uint64_t *launches, double *busy_s);
/* diagnostics: seconds the server thread spent admitting requests (building
   their interpreter programs), in ticks (launches to completion) and copying
   finished model lists to the host */
fbg_status fbg_server_profile(fbg_server *srv, double *admit_s, double *count_s, double *enum_s);
/* diagnostics: seconds of device time of the ticks' launches (CUDA events
   around each tick's launches), summed */
fbg_status fbg_server_gpu_time(fbg_server *srv, double *gpu_s);
/* recurring texts: specialised programs ready, count requests they have
   counted, and the background thread's seconds of compiling (NVRTC, module
   load, the ordering of the kernel's items, its first count) */
fbg_status fbg_server_jit_stats(fbg_server *srv, uint64_t *programs, uint64_t *requests, double *compile_s);
void fbg_server_free(fbg_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* FBG_H */
