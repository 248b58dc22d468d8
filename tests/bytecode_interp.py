"""A plain numpy interpreter of the register bytecode, for host-side tests only.

It is neither the oracle nor a fallback of the product: it checks, on the CPU,
that the emitted programs compute the oracle's integrands before any GPU run.
"""
import numpy as np

from paper_1511_03614_gb300.bytecode import decode, NAMES


def run(prog, X, dtype=np.float64):
    X = np.asarray(X, dtype=dtype)
    n = X.shape[0]
    s = np.zeros((prog.n_slots, n), dtype=dtype)
    c = prog.consts.astype(dtype)
    with np.errstate(all="ignore"):
        for w in prog.code.tolist():
            op, d, a, b = decode(w)
            name = NAMES[op]
            if name == "LDX":
                s[d] = X[:, a]
            elif name == "LDC":
                s[d] = c[a | b << 8]
            elif name == "ADD":
                s[d] = s[a] + s[b]
            elif name == "SUB":
                s[d] = s[a] - s[b]
            elif name == "MUL":
                s[d] = s[a] * s[b]
            elif name == "DIV":
                s[d] = s[a] / s[b]
            elif name == "NEG":
                s[d] = -s[a]
            elif name == "MAC":
                s[d] = s[a] * s[b] + s[d]
            elif name == "ADDC":
                s[d] = s[a] + c[b]
            elif name == "MULC":
                s[d] = s[a] * c[b]
            elif name == "MACC":
                s[d] = s[a] * c[b] + s[d]
            elif name == "POWI":
                e = b - 256 if b >= 128 else b
                s[d] = s[a] ** e
            elif name == "LOG":
                s[d] = np.log(s[a])
            elif name == "INV":
                s[d] = 1.0 / s[a]
            elif name == "MOV":
                s[d] = s[a]
            elif name == "ATAN2":
                s[d] = np.arctan2(s[a], s[b])
    if len(prog.out_slots) > 1:
        return np.stack([s[o].copy() for o in prog.out_slots], axis=1)
    return s[prog.out_slot].copy()
