"""Register bytecode: the straight-line program the device interpreter runs.

Each instruction is one 32-bit word ``op | dst << 8 | a << 16 | b << 24`` over a
per-thread file of at most 255 slots, plus a per-program pool of binary64
constants (the coefficients of the polynomials and of the eps expansion).
This is the project's form of the paper's quadruple list (Sec. 2.1).

Opcodes (slot[i] is written s[i], c[k] a constant, x[j] a coordinate):

====  =====  =========================================
 1    LDX    s[d] = x[a]
 2    LDC    s[d] = c[a | b << 8]
 3    ADD    s[d] = s[a] + s[b]
 4    SUB    s[d] = s[a] - s[b]
 5    MUL    s[d] = s[a] * s[b]
 6    DIV    s[d] = s[a] / s[b]
 7    NEG    s[d] = -s[a]
 8    MAC    s[d] = s[a] * s[b] + s[d]
 9    ADDC   s[d] = s[a] + c[b]
10    MULC   s[d] = s[a] * c[b]
11    MACC   s[d] = s[a] * c[b] + s[d]
12    POWI   s[d] = s[a] ** n,  n = b as a signed byte
13    LOG    s[d] = log(s[a])
14    INV    s[d] = 1 / s[a]
15    MOV    s[d] = s[a]
16    ATAN2  s[d] = atan2(s[a], s[b])  (argument of a complex value)
====  =====  =========================================

An instruction reads its operands before it writes s[d], so d may equal a or b.
The result of the program is s[out_slot].
"""
from __future__ import annotations

import dataclasses

import numpy as np

OPS = {"LDX": 1, "LDC": 2, "ADD": 3, "SUB": 4, "MUL": 5, "DIV": 6, "NEG": 7, "MAC": 8,
       "ADDC": 9, "MULC": 10, "MACC": 11, "POWI": 12, "LOG": 13, "INV": 14, "MOV": 15, "ATAN2": 16}
NAMES = {v: k for k, v in OPS.items()}
MAX_SLOTS = 255
MAX_CONST = 65536


def encode(op, d=0, a=0, b=0):
    return (OPS[op] & 0xFF) | (d & 0xFF) << 8 | (a & 0xFF) << 16 | (b & 0xFF) << 24


def decode(word):
    return word & 0xFF, (word >> 8) & 0xFF, (word >> 16) & 0xFF, (word >> 24) & 0xFF


@dataclasses.dataclass
class Program:
    code: np.ndarray        # uint32
    consts: np.ndarray      # float64
    n_slots: int
    out_slot: int           # slot of the (first) result
    dim: int
    counts: dict            # opcode name -> number of instructions
    out_slots: tuple = ()   # slots of all results (several for a fused multi-order unit)

    def __post_init__(self):
        if not self.out_slots:
            self.out_slots = (self.out_slot,)

    def flops(self):
        """Arithmetic operations per point: ADD/SUB/MUL/NEG/ADDC/MULC = 1, MAC/MACC = 2,
        DIV/INV/LOG/POWI counted separately in ``counts``."""
        c = self.counts
        return sum(c.get(k, 0) for k in ("ADD", "SUB", "MUL", "NEG", "ADDC", "MULC")) + \
            2 * (c.get("MAC", 0) + c.get("MACC", 0))


def _args(n):
    if n[0] in ("add", "sub", "mul", "div", "atan2"):
        return (n[1], n[2])
    if n[0] == "fma":
        return (n[1], n[2], n[3])
    if n[0] in ("neg", "log", "inv", "powi"):
        return (n[1],)
    return ()


def _schedule(nodes, live, outs):
    """Order the live nodes for low register pressure: greedy list scheduling that
    always emits, among the nodes whose operands are available, one that frees the
    most slots (operands at their last use) net of the slot it occupies; ties go to
    the node created first.  Constants take no slot of their own here and are placed
    just before their first user."""
    import heapq
    outset = set(outs)
    preds, users = {}, {i: set() for i in live}
    for i in live:
        p = set(a for a in _args(nodes[i]) if nodes[a][0] != "c")
        preds[i] = p
        for a in p:
            users[a].add(i)
    remaining = {i: len(users[i]) for i in live}
    waiting = {i: len(preds[i]) for i in live}

    def score(i):
        freed = sum(1 for a in preds[i] if remaining[a] == 1 and a not in outset)
        occupies = 1 if (users[i] or i in outset) else 0
        return freed - occupies

    heap = []
    for i in live:
        if nodes[i][0] != "c" and waiting[i] == 0:
            heapq.heappush(heap, (-score(i), i))
    order = []
    done = set()
    while heap:
        s, i = heapq.heappop(heap)
        if i in done:
            continue
        cur = -score(i)
        if cur != s:                       # stale priority: re-queue with the current one
            heapq.heappush(heap, (cur, i))
            continue
        done.add(i)
        order.append(i)
        touched = set()
        for a in preds[i]:
            remaining[a] -= 1
            touched |= users[a]
        for u in users[i]:
            waiting[u] -= 1
            if waiting[u] == 0:
                heapq.heappush(heap, (-score(u), u))
        for u in touched:                  # their scores may have improved
            if u not in done and waiting[u] == 0:
                heapq.heappush(heap, (-score(u), u))
    return _place_constants(nodes, live, order)


def _place_constants(nodes, live, order):
    """Insert the constants of ``live`` just before their first user in ``order``."""
    first_use = {}
    for k, i in enumerate(order):
        for a in _args(nodes[i]):
            if nodes[a][0] == "c" and a not in first_use:
                first_use[a] = k
    by_pos = {}
    for cidx in (i for i in live if nodes[i][0] == "c"):
        by_pos.setdefault(first_use.get(cidx, len(order)), []).append(cidx)
    out = []
    for k, i in enumerate(order):
        out.extend(by_pos.get(k, []))
        out.append(i)
    out.extend(by_pos.get(len(order), []))
    return out


def _schedule_need_first(nodes, live, outs, ties_last_first=False):
    """Order the live nodes depth first from the results, visiting a node's operands in
    decreasing order of the slots their own evaluation needs (the Sethi-Ullman order
    for expression trees; on a shared operand the estimate counts it in every user, so
    it is an upper bound, and a node is emitted once, at its first visit).  Operands of
    equal need are visited in argument order, or last first."""
    args = {i: [a for a in _args(nodes[i]) if nodes[a][0] != "c"] for i in live}
    need = {}
    for root in live:                       # post-order need labels without recursion
        stack = [(root, False)]
        while stack:
            i, expanded = stack.pop()
            if i in need or nodes[i][0] == "c":
                continue
            if not expanded:
                stack.append((i, True))
                stack.extend((a, False) for a in args[i] if a not in need)
                continue
            ls = sorted((need[a] for a in args[i]), reverse=True)
            need[i] = max([1] + [l + k for k, l in enumerate(ls)])
    order, done = [], set()
    for root in sorted((o for o in dict.fromkeys(outs) if nodes[o][0] != "c"), key=lambda o: -need[o]):
        stack = [(root, False)]
        while stack:
            i, expanded = stack.pop()
            if i in done:
                continue
            if expanded:
                done.add(i)
                order.append(i)
                continue
            stack.append((i, True))
            # pushed in reverse visiting order: the neediest operand is popped first
            todo = [a for a in args[i] if a not in done]
            if not ties_last_first:
                todo.reverse()
            for a in sorted(todo, key=lambda a: need[a]):
                stack.append((a, False))
    return _place_constants(nodes, live, order)


def emit(graph, out, dim, fuse_fma=True):
    """Lower the nodes reachable from ``out`` (one node or a list of result nodes) to a
    Program (linear-scan slot allocation); results stay live to the end.  With
    ``fuse_fma`` a product used only by one sum is first contracted into a fused
    multiply-add (``ir.contract``).  The nodes are ordered three ways (greedy list
    scheduling, and depth first in need order with either tie order) and the order
    needing the fewest slots is kept, then the shortest: the slot file sets how many
    threads share an SM, and every order computes each value by the same operations."""
    outs = list(out) if isinstance(out, (list, tuple)) else [out]
    nodes = graph.nodes

    def live_set(roots):
        live = set()
        stack = list(roots)
        while stack:
            i = stack.pop()
            if i in live:
                continue
            live.add(i)
            stack += list(_args(nodes[i]))
        return live

    if fuse_fma:
        from .ir import contract
        outs = contract(graph, outs)
    live = live_set(outs)
    best, err = None, None
    schedules = (_schedule, _schedule_need_first,
                 lambda nodes, live, outs: _schedule_need_first(nodes, live, outs, ties_last_first=True))
    for schedule in schedules:
        try:
            prog = _lower(nodes, schedule(nodes, live, outs), outs, dim)
        except OverflowError as e:          # too many slots in this order: try the other
            err = e
            continue
        if best is None or (prog.n_slots, len(prog.code)) < (best.n_slots, len(best.code)):
            best = prog
    if best is None:
        raise err
    validate(best)
    return best


def _lower(nodes, order, outs, dim):
    """Linear-scan slot allocation and encoding of the scheduled nodes."""
    out = outs[0]

    consts = []
    cidx = {}

    def const_index(v):
        if v not in cidx:
            cidx[v] = len(consts)
            consts.append(v)
        return cidx[v]

    def is_small_const(i):
        n = nodes[i]
        if n[0] != "c":
            return False
        k = const_index(n[1])
        return k < 256

    # operands that are folded constants do not need slots
    folded = set()
    for i in order:
        n = nodes[i]
        if n[0] in ("add", "mul") and (is_small_const(n[1]) or is_small_const(n[2])):
            folded.add((i, n[1] if is_small_const(n[1]) else n[2]))
        elif n[0] == "fma" and is_small_const(n[2]):
            folded.add((i, n[2]))
    # which node ids are needed in a slot and where they are used last
    uses = {}
    for pos, i in enumerate(order):
        n = nodes[i]
        args = ()
        if n[0] in ("add", "sub", "mul", "div", "atan2"):
            args = (n[1], n[2])
        elif n[0] == "fma":
            args = (n[1], n[2], n[3])
        elif n[0] in ("neg", "log", "inv", "powi"):
            args = (n[1],)
        for a in args:
            if (i, a) in folded:
                continue
            uses.setdefault(a, []).append(pos)
    last = {a: max(p) for a, p in uses.items()}
    for o in outs:
        last[o] = len(order)

    code = []
    counts = {}
    slot = {}
    free = []
    n_slots = 0

    def put(op, d=0, a=0, b=0):
        code.append(encode(op, d, a, b))
        counts[op] = counts.get(op, 0) + 1

    def alloc():
        nonlocal n_slots
        if free:
            return free.pop()
        n_slots += 1
        if n_slots > MAX_SLOTS:
            raise OverflowError("program needs more than 255 slots")
        return n_slots - 1

    for pos, i in enumerate(order):
        n = nodes[i]
        kind = n[0]
        if kind == "c" and i not in uses and i not in outs:
            continue                      # only used folded
        # release operands whose last use is here (their slots may be reused by dst)
        args = ()
        if kind in ("add", "sub", "mul", "div", "atan2"):
            args = (n[1], n[2])
        elif kind == "fma":
            args = (n[1], n[2], n[3])
        elif kind in ("neg", "log", "inv", "powi"):
            args = (n[1],)
        dying = [a for a in dict.fromkeys(args) if a in slot and last.get(a) == pos]
        if kind == "fma":
            acc = n[3]
            if acc in dying:
                d = slot[acc]             # accumulate in place
                for a in dying:
                    if a != acc:
                        free.append(slot[a])
            else:
                # the copy of the accumulator is written before the multiply reads
                # its operands, so it must not land in an operand's slot
                d = alloc()
                put("MOV", d, slot[acc])
                for a in dying:
                    free.append(slot[a])
            if (i, n[2]) in folded:
                put("MACC", d, slot[n[1]], const_index(nodes[n[2]][1]))
            else:
                put("MAC", d, slot[n[1]], slot[n[2]])
            slot[i] = d
            continue
        for a in dying:
            free.append(slot[a])
        d = alloc()
        slot[i] = d
        if kind == "x":
            put("LDX", d, n[1])
        elif kind == "c":
            k = const_index(n[1])
            put("LDC", d, k & 0xFF, k >> 8)
        elif kind in ("add", "mul"):
            if (i, n[1]) in folded or (i, n[2]) in folded:
                cnode, other = (n[1], n[2]) if (i, n[1]) in folded else (n[2], n[1])
                put("ADDC" if kind == "add" else "MULC", d, slot[other], const_index(nodes[cnode][1]))
            else:
                put(kind.upper(), d, slot[n[1]], slot[n[2]])
        elif kind in ("sub", "div", "atan2"):
            put(kind.upper(), d, slot[n[1]], slot[n[2]])
        elif kind in ("neg", "log", "inv"):
            put(kind.upper(), d, slot[n[1]])
        elif kind == "powi":
            e = n[2]
            if not -128 <= e <= 127:
                raise OverflowError("integer power out of range")
            put("POWI", d, slot[n[1]], e & 0xFF)
        else:
            raise ValueError(kind)
    if len(consts) > MAX_CONST:
        raise OverflowError("too many constants")
    prog = Program(np.array(code, dtype=np.uint32), np.array(consts, dtype=np.float64),
                   max(n_slots, 1), slot[out], dim, counts, tuple(slot[o] for o in outs))
    return prog


def validate(prog):
    """Host-side check of a program: opcodes, slot, coordinate and constant indices,
    and that no slot is read before it is written."""
    written = set()
    R = prog.n_slots
    nc = len(prog.consts)
    if not 1 <= prog.dim <= 8:
        raise ValueError("dimension must be 1..8")
    if R > MAX_SLOTS:
        raise ValueError("too many slots")
    for pc, w in enumerate(prog.code.tolist()):
        op, d, a, b = decode(w)
        name = NAMES.get(op)
        if name is None:
            raise ValueError(f"bad opcode {op} at {pc}")
        reads = []
        if name == "LDX":
            if a >= prog.dim:
                raise ValueError(f"coordinate {a} out of range at {pc}")
        elif name == "LDC":
            if (a | b << 8) >= nc:
                raise ValueError(f"constant out of range at {pc}")
        elif name in ("ADD", "SUB", "MUL", "DIV", "ATAN2"):
            reads = [a, b]
        elif name == "MAC":
            reads = [a, b, d]
        elif name in ("ADDC", "MULC"):
            reads = [a]
            if b >= nc:
                raise ValueError(f"constant out of range at {pc}")
        elif name == "MACC":
            reads = [a, d]
            if b >= nc:
                raise ValueError(f"constant out of range at {pc}")
        elif name in ("NEG", "LOG", "INV", "MOV", "POWI"):
            reads = [a]
        for r in reads + [d]:
            if r >= R:
                raise ValueError(f"slot {r} out of range at {pc}")
        for r in reads:
            if r not in written:
                raise ValueError(f"slot {r} read before written at {pc}")
        written.add(d)
    for o in prog.out_slots:
        if o not in written:
            raise ValueError("output slot never written")
