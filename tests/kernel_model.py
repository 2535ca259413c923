"""CPU models of the two evaluation kernels, driven by the compiler's JSON dump
(fbg_debug_dump).  Test infrastructure: they let the compiler (grounding,
lowering, LOP3 mapping, levels, bytecode and slot allocation) be checked
against the oracle on a machine without a GPU.  They are NOT an evaluation
path of the library and never run in the product.
"""
from __future__ import annotations

import numpy as np

M32 = np.uint32(0xFFFFFFFF)
M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
INREG = [0xAAAAAAAA, 0xCCCCCCCC, 0xF0F0F0F0, 0xFF00FF00, 0xFFFF0000]


def lut_apply(tt: int, a, b, c):
    """Bitwise 3-input function with lop3 truth table tt = f(0xF0, 0xCC, 0xAA)."""
    out = np.zeros_like(a)
    for m in range(8):
        if (tt >> m) & 1:
            x = a if (m >> 2) & 1 else ~a
            y = b if (m >> 1) & 1 else ~b
            z = c if m & 1 else ~c
            out |= x & y & z
    return out


# ------------------------------------------------------------ LUT programs --

def lut_program_values(d: dict):
    """Evaluate a LUT-program dump over every tile at once.  Returns
    (out[s] arrays over tiles, acc dict level -> list per register, layout)."""
    L = d["layout"]
    n, r = L["n"], L["r"]
    nreg = 1 << r
    tb = 0 if n <= 5 else n - 5 - r
    T = np.arange(1 << tb, dtype=np.uint64)

    def var_word(pos):
        return ((np.uint32(0) - ((T >> np.uint64(pos - 5 - r)) & np.uint64(1)).astype(np.uint32))).astype(np.uint32)

    vcache = {}

    def operand(v, s, vals):
        kind, i = v
        if kind == 0:
            return np.full(T.shape, d["consts"][i][s], dtype=np.uint32)
        if kind == 1:
            if i not in vcache:
                vcache[i] = var_word(i)
            return vcache[i]
        return vals[i][s & d["luts"][i][5]]

    vals = []
    for (tt, a, b, c, level, rmask) in d["luts"]:
        per = {}
        for s in range(nreg):
            if (s & rmask) != s:
                continue
            per[s] = lut_apply(tt, operand(a, s, vals), operand(b, s, vals), operand(c, s, vals))
        vals.append(per)
    out = [operand(d["out"], s, vals) for s in range(nreg)]
    accs = {}
    for lv, (b0, e0, has, acc) in enumerate(d["levels"]):
        if has:
            accs[lv] = [operand(acc, s, vals) for s in range(nreg)]
    return out, accs, L


def valid_mask32(n):
    return 0xFFFFFFFF if n >= 5 else (1 << (1 << n)) - 1


def lut_program_count(d: dict) -> int:
    out, accs, L = lut_program_values(d)
    vm = np.uint32(valid_mask32(L["n"]))
    total = 0
    for s, w in enumerate(out):
        total += int(np.unpackbits((w & vm).view(np.uint8)).sum())
    return total


def lut_program_table(d: dict) -> np.ndarray:
    """Truth table as u64 words (identity layout only)."""
    out, accs, L = lut_program_values(d)
    n, r = L["n"], L["r"]
    assert L["pos_of_var"] == list(range(n)), "table needs the identity layout"
    vm = np.uint32(valid_mask32(n))
    words32 = np.stack([w & vm for w in out], axis=1).reshape(-1)   # tile-major, register-minor
    if n <= 5:
        return np.array([int(words32[0])], dtype=np.uint64)
    return words32.view(np.uint64).copy()


def lut_program_prune_sound(d: dict) -> bool:
    """Every level's partial conjunction covers the formula value: a zero
    partial conjunction may skip inner levels without changing results."""
    out, accs, L = lut_program_values(d)
    const_acc = d["const_acc"]
    for s, w in enumerate(out):
        if np.any(w & ~np.uint32(const_acc[s])):
            return False
        for lv, a in accs.items():
            if np.any(w & ~a[s]):
                return False
    return True


# ------------------------------------------------------------- interpreter --

OP_SHARED, OP_CONST, OP_VAR, OP_ACC, DST_SHARED, DST_ACC = 0x1000, 0x4000, 0x8000, 0xFFFF, 160, 255
BLOCK = 64   # tiles of a block: one warp of 32 threads, two tiles each


class InterpModel:
    """Literal model of interp_kernel: one block (one warp holding all 64
    tiles) runs the units in order; loop levels as an odometer; the prune
    vote covers the whole warp, so every tile; slots and the accumulator as
    in the kernel."""

    def __init__(self, d: dict):
        self.d = d
        self.ins = [int(w) for w in d["ins"]]
        self.consts = [np.uint64(c) for c in d["consts"]]
        self.levels = d["levels"]
        self.nslots = d["nslots"]
        self.tb = np.arange(BLOCK, dtype=np.uint64)
        self.tvalid = self.tb < np.uint64(d["tvalid"])
        self.vmask = np.uint64(d["vmask"])

    def fetch(self, op):
        if op == OP_ACC:
            return self.acc
        if op & OP_VAR:
            bit = (self.coords >> np.uint64(op & 63)) & np.uint64(1)
            return np.where(bit == 1, M64, np.uint64(0))
        if op & OP_CONST:
            return np.full(BLOCK, self.consts[op & 0x3FFF], dtype=np.uint64)
        if op & OP_SHARED:
            # a block slot holds one word; the value must be equal in every tile
            return np.full(BLOCK, self.svals[op & 0xFFF], dtype=np.uint64)
        return self.slots[op]

    def exec_level(self, lv):
        b, e = self.levels[lv][0], self.levels[lv][1]
        for i in range(b, e):
            w = self.ins[i]
            lut, dst = w & 0xFF, (w >> 8) & 0xFF
            a = self.fetch((w >> 16) & 0xFFFF)
            bb = self.fetch((w >> 32) & 0xFFFF)
            c = self.fetch(w >> 48)
            v = lut_apply(lut, a, bb, c)
            if dst == DST_ACC:
                self.acc = v
            elif dst >= DST_SHARED:
                # only values equal in every (valid) tile may live in a block slot
                vv = v[self.tvalid]
                assert len(vv) == 0 or bool(np.all(vv == vv[0])), "block slot value differs between tiles"
                self.svals[dst - DST_SHARED] = v[0]
            else:
                self.slots[dst] = v

    def alive(self, lv, mode):
        has, op = self.levels[lv][4], self.levels[lv][5]
        mine = np.ones(BLOCK, dtype=bool) if not has else (self.fetch(op) != 0)
        return np.full(BLOCK, bool(mine.any()))   # one warp holds every tile

    def run(self, mode, cap=0, unit_offsets=None):
        d = self.d
        self.slots = np.zeros((max(1, self.nslots), BLOCK), dtype=np.uint64)
        self.svals = np.zeros(96, dtype=np.uint64)
        self.acc = np.zeros(BLOCK, dtype=np.uint64)
        self.coords = self.tb << np.uint64(6)
        nl = len(self.levels)
        self.exec_level(0)
        alive0 = self.alive(0, mode)
        count = np.zeros(BLOCK, dtype=np.uint64)
        unit_counts = []
        nwords = 1 if d["layout"]["n"] <= 6 else 1 << (d["layout"]["n"] - 6)
        table = np.zeros(nwords, dtype=np.uint64)
        models = []
        for u in range(d["nunits"]):
            before = int(count.sum())
            base = unit_offsets[u] if mode == 2 else 0
            active = alive0.copy()
            self.coords = (self.tb << np.uint64(6)) | (np.uint64(u << d["first_unit_pos"]) if d["unit_bits"] else np.uint64(0))
            self._unit_active = active
            if active.any():
                base = self.run_unit(mode, active, count, table, models, base, cap)
            unit_counts.append(int(count.sum()) - before)
        return int(count.sum()), table, models, unit_counts

    def run_unit(self, mode, active, count, table, models, base, cap):
        nl = len(self.levels)
        self.exec_level(1)
        a = active & self.alive(1, mode)
        if not a.any():
            return base
        # odometer; `mask[lv]` = lanes whose warp is still inside level lv
        it = [0] * nl
        stack_alive = {1: a}

        def leaf(act):
            nonlocal base
            word = np.where(self.tvalid & act, self.fetch(self.d["out_op"]) & self.vmask, np.uint64(0))
            if mode == 0:
                for t in range(BLOCK):
                    count[t] += np.uint64(bin(int(word[t])).count("1"))
            elif mode == 1:
                for t in range(BLOCK):
                    if self.tvalid[t] and act[t]:
                        table[int(self.coords[t]) >> 6] = word[t]
            else:
                for t in range(BLOCK):
                    wv = int(word[t])
                    b = 0
                    while wv:
                        if wv & 1:
                            if base < cap:
                                models.append(int(self.coords[t]) | b)
                            base += 1
                        wv >>= 1
                        b += 1

        if nl <= 2:
            leaf(a)
            return base

        def rec(lv, act):
            L = self.levels[lv]
            bits, pos = L[2], L[3]
            m = np.uint64(((1 << bits) - 1) << pos)
            for i in range(1 << bits):
                self.coords = (self.coords & ~m) | np.uint64(i << pos)
                self.exec_level(lv)
                al = act & self.alive(lv, mode)
                if not al.any():
                    continue
                if lv + 1 < nl:
                    rec(lv + 1, al)
                else:
                    leaf(al)

        rec(2, a)
        return base


def interp_count(d):
    return InterpModel(d).run(0)[0]


def interp_table(d):
    return InterpModel(d).run(1)[1]


def interp_models(d, cap):
    m = InterpModel(d)
    _, _, _, unit_counts = m.run(0)
    offs = np.concatenate([[0], np.cumsum(unit_counts)[:-1]]).astype(int).tolist()
    total = int(sum(unit_counts))
    _, _, models, _ = InterpModel(d).run(2, cap=cap, unit_offsets=offs)
    return models, total
