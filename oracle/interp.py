"""Semantics of programs: the ComputeSemantics step (Sec. 2 and 2.2).

The semantics of tree T is the vector of its outputs over all fitness cases,
s_{T,j} = T(x_j) (Sec. 2).  The interpreter reads the linear genome left to
right with a LIFO stack (Sec. 2.2, "Interpreter"): a terminal pushes its value;
a function pops as many operands as its arity, applies itself and pushes the
result.  Random trees used by mutation are wrapped in the logistic function,
R = 1 / (1 + exp(-T)) (Sec. 2), so their outputs lie in [0, 1].

Everything here is float64.  Protected division returns 1 when the divisor's
magnitude is below protect_eps (the paper names the operator without its rule;
reading: strict |d| < eps, eps = float32(1e-3)).

Also provided: the paper's skip rule for malformed linear genomes (a function
whose operands are missing is skipped; the register Out keeps the last valid
function output), which well-formed postfix programs never trigger, and an
independent recursive evaluator over nested tuples used to pin the stack
interpreter.
"""
from __future__ import annotations

import numpy as np

from .trees import OP_ADD, OP_CONST, OP_DIV, OP_MUL, OP_SUB, OP_VAR, PAD


def _apply(op: int, a, b, eps: float):
    if op == OP_ADD:
        return a + b
    if op == OP_SUB:
        return a - b
    if op == OP_MUL:
        return a * b
    if op == OP_DIV:
        small = np.abs(b) < eps
        safe = np.where(small, 1.0, b)
        return np.where(small, 1.0, a / safe)
    raise ValueError(f"not a function gene: {op}")


def eval_postfix(genes, consts, X, protect_eps: float = 1e-3) -> np.ndarray:
    """Evaluate one postfix program on every case.

    X: float64 feature-major matrix (l, n).  Returns float64 (n,).
    """
    eps = float(np.float32(protect_eps))
    n = X.shape[1]
    stack = []
    for g, c in zip(genes, consts):
        g = int(g)
        if g == PAD:
            break
        op = g & 0xFF
        if op == OP_VAR:
            stack.append(X[g >> 8].astype(np.float64))
        elif op == OP_CONST:
            stack.append(np.full(n, float(c), dtype=np.float64))
        else:
            b = stack.pop()
            a = stack.pop()
            with np.errstate(all="ignore"):
                stack.append(_apply(op, a, b, eps))
    if len(stack) != 1:
        raise ValueError("program is not well-formed postfix")
    return stack[0]


def eval_linear_genome(genes, consts, X, protect_eps: float = 1e-3) -> np.ndarray:
    """The paper's rule for arbitrary linear genomes (Sec. 2.2, "Interpreter"):
    a function gene with fewer stacked operands than its arity is skipped; the
    register Out holds the output of the last function actually applied and
    is the program's value.  Reading for genomes that apply no function: the
    stack top, or 0 for an empty stack."""
    eps = float(np.float32(protect_eps))
    n = X.shape[1]
    stack = []
    out = None
    for g, c in zip(genes, consts):
        g = int(g)
        if g == PAD:
            break
        op = g & 0xFF
        if op == OP_VAR:
            stack.append(X[g >> 8].astype(np.float64))
        elif op == OP_CONST:
            stack.append(np.full(n, float(c), dtype=np.float64))
        else:
            if len(stack) < 2:
                continue
            b = stack.pop()
            a = stack.pop()
            with np.errstate(all="ignore"):
                out = _apply(op, a, b, eps)
            stack.append(out)
    if out is not None:
        return out
    if stack:
        return stack[-1]
    return np.zeros(n, dtype=np.float64)


def sigma(v) -> np.ndarray:
    """Logistic wrapping of a random tree, 1 / (1 + exp(-v)) (Sec. 2)."""
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(-np.asarray(v, dtype=np.float64)))


def bf16_round(v) -> np.ndarray:
    """Round float64 values to bfloat16 (round to nearest, ties to even),
    going through float32 first as a bf16 store of a float32 value does."""
    f = np.asarray(v, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    nan = np.isnan(f)
    r = np.where(nan, np.uint64(0x7FC00000), r)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def pool_semantics(genes, consts, lengths, X, protect_eps=1e-3, logistic=False,
                   bf16=False, linear=False) -> np.ndarray:
    """Semantic matrix of a pool: row i = semantics of program i (Alg. 1,
    S_T for the population, S_R for the random trees).  linear: the programs
    are the paper's linear genomes, read with the skip rule and Out."""
    rows = []
    evaluate = eval_linear_genome if linear else eval_postfix
    for i in range(genes.shape[0]):
        L = int(lengths[i])
        s = evaluate(genes[i, :L], consts[i, :L], X, protect_eps)
        if logistic:
            s = sigma(s)
            if bf16:
                s = bf16_round(s)
        rows.append(s)
    return np.stack(rows) if rows else np.zeros((0, X.shape[1]))


def eval_tree(node, x, protect_eps: float = 1e-3) -> float:
    """Recursive evaluation of a nested-tuple expression on one case.

    node: ('var', f) | ('const', c) | (op, left, right) with op in '+-*/'.
    x: sequence of feature values.  Plain Python floats (IEEE double).
    """
    eps = float(np.float32(protect_eps))
    kind = node[0]
    if kind == "var":
        return float(x[node[1]])
    if kind == "const":
        return float(node[1])
    a = eval_tree(node[1], x, protect_eps)
    b = eval_tree(node[2], x, protect_eps)
    if kind == "+":
        return a + b
    if kind == "-":
        return a - b
    if kind == "*":
        return a * b
    if kind == "/":
        return 1.0 if abs(b) < eps else a / b
    raise ValueError(kind)


def tree_to_postfix(node):
    """Serialise a nested-tuple expression to (genes, consts)."""
    genes, consts = [], []
    code = {"+": OP_ADD, "-": OP_SUB, "*": OP_MUL, "/": OP_DIV}

    def walk(nd):
        if nd[0] == "var":
            genes.append(OP_VAR | (nd[1] << 8))
            consts.append(np.float32(0.0))
        elif nd[0] == "const":
            genes.append(OP_CONST)
            consts.append(np.float32(nd[1]))
        else:
            walk(nd[1])
            walk(nd[2])
            genes.append(code[nd[0]])
            consts.append(np.float32(0.0))

    walk(node)
    return genes, consts


def postfix_to_tree(genes, consts):
    """Rebuild the nested-tuple expression a postfix program encodes."""
    names = {OP_ADD: "+", OP_SUB: "-", OP_MUL: "*", OP_DIV: "/"}
    st = []
    for g, c in zip(genes, consts):
        g = int(g)
        if g == PAD:
            break
        op = g & 0xFF
        if op == OP_VAR:
            st.append(("var", g >> 8))
        elif op == OP_CONST:
            st.append(("const", float(c)))
        else:
            b = st.pop()
            a = st.pop()
            st.append((names[op], a, b))
    assert len(st) == 1
    return st[0]


U32 = 2.0 ** -24          # unit roundoff of float32 round-to-nearest


def eval_postfix_fp32_bound(genes, consts, X, protect_eps: float = 1e-3, linear=False):
    """Exact (float64) value of a program and a first-order bound on the
    error of evaluating it in float32 arithmetic, every operation rounded
    once to nearest (running error analysis, Wilkinson).

    For operands a, b carrying errors ea, eb:
      a +- b : ea + eb
      a * b  : |a| eb + |b| ea + ea eb
      a / b  : (ea + |a/b| eb) / (|b| - eb)
    plus u (|r| + e) for the rounding of the result r.  The bound is
    infinite where float32 could take the other branch of protected division
    (|b| within its error of eps) or where a magnitude exceeds 1e38 (float32
    overflow), i.e. where the two precisions may legitimately disagree.
    linear: a linear genome, read with the skip rule and the Out register
    (eval_linear_genome).  Returns (value (n,), bound (n,)).
    """
    eps = float(np.float32(protect_eps))
    n = X.shape[1]
    stack = []
    out = None
    with np.errstate(all="ignore"):
        for g, c in zip(genes, consts):
            g = int(g)
            if g == PAD:
                break
            op = g & 0xFF
            if op == OP_VAR:
                stack.append((X[g >> 8].astype(np.float64), np.zeros(n)))
                continue
            if op == OP_CONST:
                stack.append((np.full(n, float(c)), np.zeros(n)))
                continue
            if linear and len(stack) < 2:
                continue
            b, eb = stack.pop()
            a, ea = stack.pop()
            if op == OP_ADD:
                r, e = a + b, ea + eb
            elif op == OP_SUB:
                r, e = a - b, ea + eb
            elif op == OP_MUL:
                r, e = a * b, np.abs(a) * eb + np.abs(b) * ea + ea * eb
            else:
                small = np.abs(b) < eps
                r = np.where(small, 1.0, a / np.where(small, 1.0, b))
                den = np.abs(b) - eb
                e = np.where(small, 0.0, (ea + np.abs(r) * eb) / np.where(den > 0, den, 1.0))
                ab = np.abs(b)
                flip = np.where(small, ab + eb >= eps, ab - eb < eps) | (~small & (den <= 0))
                e = np.where(flip, np.inf, e)
            e = e + U32 * (np.abs(r) + e)
            e = np.where(np.abs(r) > 1e38, np.inf, e)
            e = np.where(np.isfinite(r), e, np.inf)
            stack.append((r, e))
            out = (r, e)
    if linear:
        if out is not None:
            return out
        return stack[-1] if stack else (np.zeros(n), np.zeros(n))
    if len(stack) != 1:
        raise ValueError("program is not well-formed postfix")
    return stack[0]


def sigma_fp32_bound(v_bound):
    """Error bound of sigma computed in float32 from an argument with error
    v_bound: |sigma'| <= 1/4, plus a few roundings of a value in [0, 1]."""
    return np.asarray(v_bound) / 4.0 + 8 * U32
