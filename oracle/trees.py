"""Ramped half-and-half generation of postfix programs (initialisation).

The paper creates the population P and the pool of random trees R with its
CreatePopulation kernel (Algorithm 1) over the function set {+, -, x,
protected division} and terminals made of input features and ephemeral
random constants (Sec. 2.2, "Initialization"); programs are stored as linear
genomes that the interpreter reads left to right.  The paper does not fix a
tree-shape policy for this path, so the reading used here (shared contract) is
the classical ramped half-and-half scheme, emitted in postfix order:

  * individual i of a pool with depths [dmin, dmax], D = dmax - dmin + 1, gets
    depth_i = dmin + (i mod D) and the "full" method when floor(i / D) is even,
    "grow" otherwise;
  * nodes are decided in preorder (root depth 0), one Philox stream per tree
    (counter = (block, i, 0x80000000 | purpose, run)), words consumed in order:
      - at depth_i the node is a terminal (no word);
      - otherwise it is a function under "full" or at the root; under "grow"
        it is a function iff u24(word) < p_grow_function;
      - a function draws its operator as idx(word, 4) over (+, -, x, /);
      - a terminal is a feature iff u24(word) < p_feature_given_terminal, whose
        index is idx(word, l); otherwise a constant erc(word) in [lo, hi).
  * a function gene is emitted after both of its operand subtrees (postfix).

Gene encoding (shared contract): int32; 0 '+', 1 '-', 2 'x', 3 protected '/',
4 constant (value in the parallel float32 array), 5 | (f << 8) feature f,
-1 padding after the program's end.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np

from .philox import INIT_FLAG, WordStream, erc, idx, u24

OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_CONST, OP_VAR = 0, 1, 2, 3, 4, 5
PAD = -1


def max_genes(dmax: int) -> int:
    """Genes of a full binary tree of depth dmax: 2^(dmax+1) - 1."""
    return (1 << (dmax + 1)) - 1


def rhh_program(seed: int, run: int, purpose: int, i: int, dmin: int, dmax: int,
                n_features: int, p_grow: float, p_feature: float,
                const_lo: float, const_hi: float) -> Tuple[list, list]:
    """Postfix genes and constants of individual i (recursive preorder)."""
    D = dmax - dmin + 1
    depth = dmin + (i % D)
    full = ((i // D) % 2) == 0
    words = WordStream(seed, run, INIT_FLAG | purpose, i)
    p_grow32 = float(np.float32(p_grow))
    p_feat32 = float(np.float32(p_feature))
    genes: list = []
    consts: list = []

    def node(d: int) -> None:
        if d == depth:
            is_function = False
        elif full or d == 0:
            is_function = True
        else:
            is_function = u24(words.next()) < p_grow32
        if is_function:
            op = idx(words.next(), 4)
            node(d + 1)
            node(d + 1)
            genes.append(op)
            consts.append(np.float32(0.0))
        elif u24(words.next()) < p_feat32:
            f = idx(words.next(), n_features)
            genes.append(OP_VAR | (f << 8))
            consts.append(np.float32(0.0))
        else:
            genes.append(OP_CONST)
            consts.append(erc(words.next(), const_lo, const_hi))

    node(0)
    return genes, consts


def rhh_pool(seed: int, run: int, purpose: int, count: int, dmin: int, dmax: int,
             n_features: int, p_grow: float = 0.5, p_feature: float = 0.14 / 0.18,
             const_lo: float = -1.0, const_hi: float = 1.0):
    """Generate a pool; returns (genes int32 [count, K], consts f32 [count, K],
    lengths int32 [count]) with K = 2^(dmax+1) - 1 and padding genes = -1."""
    K = max_genes(dmax)
    genes = np.full((count, K), PAD, dtype=np.int32)
    consts = np.zeros((count, K), dtype=np.float32)
    lengths = np.zeros(count, dtype=np.int32)
    for i in range(count):
        g, c = rhh_program(seed, run, purpose, i, dmin, dmax, n_features,
                           p_grow, p_feature, const_lo, const_hi)
        lengths[i] = len(g)
        genes[i, :len(g)] = g
        consts[i, :len(c)] = c
    return genes, consts, lengths


# ---- the paper's fixed-length linear genome (init_mode 1) -------------------
#
# Every gene of a chromosome of K genes is drawn independently: a function
# with probability 0.8, a feature with probability 0.14, an ephemeral random
# constant with probability 0.04 (Sec. 2.2, "Initialization").  The printed
# probabilities add up to 0.98; they are read as relative weights, i.e.
# divided by 0.98.  Shared contract: gene j of individual i reads words 2j and
# 2j+1 of the stream (i, 0x80000000 | purpose, run); u24(word 2j) below
# float32(0.8 / 0.98) makes a function, whose operator is idx(word 2j+1, 4);
# below float32(0.94 / 0.98) a feature idx(word 2j+1, l); otherwise a
# constant erc(word 2j+1) in [lo, hi).
P_FUNCTION = 0.8 / 0.98
P_FUNCTION_OR_FEATURE = (0.8 + 0.14) / 0.98


def linear_genome(seed: int, run: int, purpose: int, i: int, K: int, n_features: int,
                  const_lo: float, const_hi: float):
    """Genes (int32 [K]) and constants (float32 [K]) of individual i."""
    from .philox import stream_words
    w = stream_words(seed, run, INIT_FLAG | purpose, i, 2 * K)
    u = u24(w[0::2])                      # gene class words (exact floats)
    c = w[1::2]                           # operator / feature / constant words
    is_fun = u < float(np.float32(P_FUNCTION))
    is_var = ~is_fun & (u < float(np.float32(P_FUNCTION_OR_FEATURE)))
    is_const = ~is_fun & ~is_var
    genes = np.where(is_fun, idx(c, 4),
                     np.where(is_var, OP_VAR | (idx(c, n_features) << 8), OP_CONST))
    consts = np.zeros(K, dtype=np.float32)
    for j in np.nonzero(is_const)[0]:
        consts[j] = erc(int(c[j]), const_lo, const_hi)
    return genes.astype(np.int32), consts


def linear_pool(seed: int, run: int, purpose: int, count: int, K: int, n_features: int,
                const_lo: float = -1.0, const_hi: float = 1.0):
    """A pool of linear genomes: (genes [count, K], consts [count, K],
    lengths [count] = K)."""
    genes = np.zeros((count, K), dtype=np.int32)
    consts = np.zeros((count, K), dtype=np.float32)
    for i in range(count):
        genes[i], consts[i] = linear_genome(seed, run, purpose, i, K, n_features,
                                            const_lo, const_hi)
    return genes, consts, np.full(count, K, dtype=np.int32)


def genome_max_stack(genes) -> int:
    """Deepest stack reached while interpreting a linear genome with the
    skip rule (a function short of operands leaves the stack as it is)."""
    sp = best = 0
    for g in genes:
        g = int(g)
        if g == PAD:
            break
        if (g & 0xFF) in (OP_CONST, OP_VAR):
            sp += 1
            best = max(best, sp)
        elif sp >= 2:
            sp -= 1
    return best


def postfix_depth(genes) -> int:
    """Depth of the tree a well-formed postfix program encodes (root = 0)."""
    st = []
    for g in genes:
        if g == PAD:
            break
        op = g & 0xFF
        if op in (OP_CONST, OP_VAR):
            st.append(0)
        else:
            b = st.pop()
            a = st.pop()
            st.append(1 + max(a, b))
    assert len(st) == 1
    return st[0]
