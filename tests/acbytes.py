"""Serialise small hand-built arithmetic circuits in the compiled-AC byte format
(include/qkc.h) -- a test helper, so the evaluators can be checked on ACs whose
polynomial is known in closed form, independently of the compiler."""
import struct

import numpy as np

OPS = {"IND": 0, "PARAM": 1, "CONST": 2, "ADD": 3, "MUL": 4}


def pack(kind, n_qubits, n_angles, var_card, var_tag, nodes, root):
    """nodes: list of dicts in storage order: {"op", "children"} for ADD/MUL,
    {"op": "IND", "var", "val"}, {"op": "PARAM", "angle", "fn", "coef"},
    {"op": "CONST", "value"}; leaves first (IND, then PARAM, then CONST)."""
    N = len(nodes)
    level = [0] * N
    for i, nd in enumerate(nodes):
        if nd["op"] in ("ADD", "MUL"):
            level[i] = 1 + max(level[c] for c in nd["children"])
    order = sorted(range(N), key=lambda i: (level[i], i))
    assert order == list(range(N)), "nodes must be given in level order"
    D = max(level) + 1
    level_off = [0] * (D + 1)
    for l in level:
        level_off[l + 1] += 1
    for l in range(D):
        level_off[l + 1] += level_off[l]
    n_leaves = level_off[1]
    child_off = [0]
    child = []
    for nd in nodes:
        child += list(nd.get("children", []))
        child_off.append(len(child))
    la, lb, lc = [], [], []
    for nd in nodes[:n_leaves]:
        if nd["op"] == "IND":
            la.append(nd["var"]); lb.append(nd["val"]); lc += [1.0, 0.0]
        elif nd["op"] == "PARAM":
            la.append(nd["angle"]); lb.append(nd["fn"]); lc += [nd["coef"].real, nd["coef"].imag]
        else:
            la.append(-1); lb.append(0); lc += [nd["value"].real, nd["value"].imag]
    n_ind = sum(1 for nd in nodes if nd["op"] == "IND")
    out = bytearray(struct.pack("<16I", 0x43414B51, 1, kind, n_qubits, n_angles, len(var_card), N, len(child), D,
                                n_leaves, root, n_ind, 0, 0, 0, 0))

    def arr(a, dt):
        while len(out) % 8:
            out.append(0)
        out.extend(np.asarray(a, dtype=dt).tobytes())

    arr(var_card, "<u4"); arr(var_tag, "<i4"); arr(level_off, "<u4"); arr([OPS[n["op"]] for n in nodes], "u1")
    arr(child_off, "<u4"); arr(child, "<u4"); arr(la, "<i4"); arr(lb, "<i4"); arr(lc, "<f8")
    while len(out) % 8:
        out.append(0)
    return bytes(out)


def toy_ac():
    """f = l10 (l00 p + l01 q + c) + l11 c with p = (2 + i) cos(t0/2), q = exp(+i t1/2),
    c = 0.5 - 0.25 i, over two binary variables X0 (l00, l01) and X1 (l10, l11)."""
    c = 0.5 - 0.25j
    nodes = [
        {"op": "IND", "var": 0, "val": 0}, {"op": "IND", "var": 0, "val": 1},
        {"op": "IND", "var": 1, "val": 0}, {"op": "IND", "var": 1, "val": 1},
        {"op": "PARAM", "angle": 0, "fn": 0, "coef": 2 + 1j},
        {"op": "PARAM", "angle": 1, "fn": 3, "coef": 1 + 0j},
        {"op": "CONST", "value": c},
        {"op": "MUL", "children": [0, 4]},   # 7  l00 p
        {"op": "MUL", "children": [1, 5]},   # 8  l01 q
        {"op": "MUL", "children": [3, 6]},   # 9  l11 c
        {"op": "ADD", "children": [6, 7, 8]},  # 10
        {"op": "MUL", "children": [2, 10]},  # 11
        {"op": "ADD", "children": [9, 11]},  # 12 root
    ]
    return pack(1, 2, 2, [2, 2], [0, 1], nodes, 12)


def toy_value(angles, lam):
    """Closed form of toy_ac at indicator values lam = [[l00, l01], [l10, l11]]."""
    import cmath
    p = (2 + 1j) * cmath.cos(angles[0] / 2)
    q = cmath.exp(0.5j * angles[1])
    c = 0.5 - 0.25j
    return lam[1][0] * (lam[0][0] * p + lam[0][1] * q + c) + lam[1][1] * c


def toy_derivatives(angles, lam):
    """(d f / d lambda in (var, value) order, d f / d t0, d f / d t1)."""
    import cmath
    p = (2 + 1j) * cmath.cos(angles[0] / 2)
    q = cmath.exp(0.5j * angles[1])
    c = 0.5 - 0.25j
    dl = [lam[1][0] * p, lam[1][0] * q, lam[0][0] * p + lam[0][1] * q + c, c]
    dt0 = lam[1][0] * lam[0][0] * (2 + 1j) * (-0.5 * cmath.sin(angles[0] / 2))
    dt1 = lam[1][0] * lam[0][1] * 0.5j * q
    return dl, dt0, dt1
