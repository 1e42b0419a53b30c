"""The float32 running error bound used to judge the GPU interpreter really
bounds float32 evaluation (checked against numpy's IEEE single arithmetic)."""
import numpy as np

from oracle import interp as oi
from oracle import trees as ot


def _eval_f32(genes, consts, X32, eps):
    st = []
    e32 = np.float32(eps)
    with np.errstate(all="ignore"):
        for g, c in zip(genes, consts):
            if g == ot.PAD:
                break
            op = g & 0xFF
            if op == ot.OP_VAR:
                st.append(X32[g >> 8])
            elif op == ot.OP_CONST:
                st.append(np.full(X32.shape[1], c, dtype=np.float32))
            else:
                b = st.pop()
                a = st.pop()
                if op == 0:
                    r = a + b
                elif op == 1:
                    r = a - b
                elif op == 2:
                    r = a * b
                else:
                    small = np.abs(b) < e32
                    r = np.where(small, np.float32(1), a / np.where(small, np.float32(1), b))
                st.append(r.astype(np.float32))
    return st[0]


def test_bound_covers_float32_evaluation():
    rng = np.random.default_rng(3)
    X32 = rng.normal(size=(6, 4000)).astype(np.float32)
    X32[0, :50] = np.float32(1e-3) * (1 + rng.normal(size=50) * 1e-6).astype(np.float32)
    X64 = X32.astype(np.float64)
    G, C, L = ot.rhh_pool(7, 0, 1, 120, 2, 6, 6)
    finite_bounds = 0
    total = 0
    for i in range(120):
        g, c = G[i, :L[i]], C[i, :L[i]]
        v, e = oi.eval_postfix_fp32_bound(g, c, X64)
        f = _eval_f32(g, c, X32, 1e-3).astype(np.float64)
        fin = np.isfinite(e)
        assert np.all(np.abs(f[fin] - v[fin]) <= e[fin]), i
        finite_bounds += fin.sum()
        total += fin.size
        # not vacuous: the bound is tiny where the program stays well scaled
        tame = fin & (np.abs(v) < 10)
        if tame.any():
            assert np.median(e[tame]) < 1e-3
    assert finite_bounds / total > 0.99


def test_bound_marks_protected_division_threshold():
    e32 = float(np.float32(1e-3))
    # exact float32 operands carry no error: only the rounding of a / b counts
    X = np.array([[1.0, 1.0], [e32, 0.5]])
    v, e = oi.eval_postfix_fp32_bound([5, 5 | (1 << 8), ot.OP_DIV], [0, 0, 0], X)
    assert np.all(np.isfinite(e)) and np.all(e <= oi.U32 * np.abs(v) * 1.0001)
    # x0 / (x1 + x2) with x1 + x2 within its rounding error of eps: ambiguous
    X2 = np.array([[1.0, 1.0], [e32, e32], [1e-11, 0.25]])
    genes = [5, 5 | (1 << 8), 5 | (2 << 8), ot.OP_ADD, ot.OP_DIV]
    v2, e2 = oi.eval_postfix_fp32_bound(genes, [0] * 5, X2)
    assert not np.isfinite(e2[0])
    assert np.isfinite(e2[1])
