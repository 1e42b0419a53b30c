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
