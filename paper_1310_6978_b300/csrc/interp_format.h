// interp_format.h -- bytecode of the generic interpreter kernel.
//
// A program is a list of 64-bit instructions, each one 3-input LUT on 64-bit
// words (two lop3.b32: the thread's tile is 2 registers, r = 1), grouped by
// loop level.  Instruction word: lut[0:8) dst[8:16) a[16:32) b[32:48) c[48:64).
// Operand codes (16 bit): a tile slot 0..FBG_INTERP_MAX_SLOTS-1 (one 64-bit
// word per tile: a column of the block's slot file), FBG_OP_SHARED|i (block
// slot i: one word for the whole block, for values that do not depend on the
// lane and warp letters and so are equal in every tile), FBG_OP_CONST|i
// (entry i of the constant table), FBG_OP_VAR|p (generator word of bit
// position p, p >= 6), FBG_OP_ACC (the accumulator register).  dst: a tile
// slot, FBG_DST_SHARED + i for block slot i, or FBG_DST_ACC.
#pragma once

#define FBG_INTERP_MAX_LEVELS 10
// tiles per block: the layout's threads (5 lane bits, 1 warp bit).  Two
// tiles per thread halve the decode and dispatch work per bit; four were
// measured slower (the larger slot file in shared memory costs occupancy).
#define FBG_INTERP_BLOCK 64
#define FBG_INTERP_THREADS 32        // threads per block; each evaluates BLOCK / THREADS tiles
#define FBG_INTERP_WARPS_LOG2 1
#define FBG_INTERP_MAX_SLOTS 160      // tile slots
#define FBG_INTERP_MAX_SHARED 95      // block slots (dst codes 160..254)
#define FBG_INTERP_MAX_CONSTS 512   // constant table entries (global memory)

#define FBG_OP_SHARED 0x1000u
#define FBG_OP_CONST 0x4000u
#define FBG_OP_VAR 0x8000u
#define FBG_OP_ACC 0xFFFFu
#define FBG_DST_SHARED 160u
#define FBG_DST_ACC 255u

struct FbgInterpLevel {
  unsigned int ins_begin, ins_end;   // instructions of this level
  unsigned int bits, pos;            // loop levels: bit count and first bit position
  unsigned int has_acc, acc_op;      // prune check on this operand (warp vote)
};

struct FbgInterpProg {
  unsigned int n;                    // number of variables
  unsigned int nlevels;              // 2 + loop levels (level 0 thread, 1 unit)
  unsigned int nslots, nconst;       // tile slots, constants
  unsigned int nshared;              // block slots
  unsigned int tvalid;               // threads of a block that hold real tiles
  unsigned int first_unit_pos, unit_bits;
  unsigned int out_op;               // operand holding the formula value
  unsigned long long vmask;          // valid bits of a tile word (n < 6)
  unsigned long long nunits;
  const unsigned long long* ins;     // device pointer to instructions
  const unsigned long long* consts;  // device pointer to the constant table
  FbgInterpLevel lev[FBG_INTERP_MAX_LEVELS];
};

// one entry of the persistent batch queue: units [unit_begin, unit_end) of a program
struct FbgWorkItem {
  unsigned int prog;
  unsigned int flags;
  unsigned long long unit_begin, unit_end;
};

// FbgWorkItem.flags: count pass of an item of one unit whose count also goes
// to its program's per-unit counts (FbgSlotOut.unit_counts[unit])
#define FBG_ITEM_UNIT_COUNTS 1u

// Per-program outputs of a launch over several programs (the server's model
// lists): per-unit counts of the count pass, and for the write pass the
// exclusive prefix of those counts, the model buffer and its capacity.
struct FbgSlotOut {
  unsigned long long* unit_counts;
  const unsigned long long* unit_offsets;
  unsigned long long* models;
  unsigned long long cap;
};
