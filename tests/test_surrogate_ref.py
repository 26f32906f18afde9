"""Pins of the NumPy reference of the surrogate network (oracle/surrogate_ref.py): its
FP64 gradient agrees with central finite differences of its own forward pass, its neighbour
and edge sums agree with dense adjacency products, and its BF16 rounding is the IEEE
round-to-nearest-even one."""
import numpy as np
import pytest

from oracle import surrogate_ref as S


def small_graph(n=12, seed=0):
    rng = np.random.default_rng(seed)
    pairs = sorted({tuple(sorted(rng.choice(n, 2, replace=False))) for _ in range(3 * n)})
    row_ptr, col = S.csr(pairs, n)
    X = rng.normal(size=(n, S.FIN))
    E = rng.normal(size=(len(col), S.EIN))
    _, total = S.layout()
    p = rng.normal(scale=0.08, size=total)
    return pairs, row_ptr, col, X, E, p


def test_gradient_matches_finite_differences():
    pairs, row_ptr, col, X, E, p = small_graph()
    rng = np.random.default_rng(1)
    Y, c = S.forward(p, X, E, row_ptr, col, bf16=False)
    dY = rng.normal(size=Y.shape)
    g = S.backward(p, dY, c, row_ptr, col)
    off, total = S.layout()
    # probe every tensor: a few weights and a bias of each layer
    idx = []
    for ow, ob in off:
        idx += list(rng.integers(ow, ob, 6)) + [ob]
    h = 1e-6
    for k in idx:
        q = p.copy()
        q[k] += h
        yp, _ = S.forward(q, X, E, row_ptr, col, bf16=False)
        q[k] -= 2 * h
        ym, _ = S.forward(q, X, E, row_ptr, col, bf16=False)
        fd = np.sum(dY * (yp - ym)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_sums_equal_dense_adjacency_products():
    pairs, row_ptr, col, X, E, p = small_graph(n=9, seed=3)
    n = 9
    Adj = np.zeros((n, n))
    for a, b in pairs:
        Adj[a, b] = Adj[b, a] = 1.0
    recv = np.repeat(np.arange(n), np.diff(row_ptr))
    assert np.array_equal(np.sort(np.stack([recv, col], 1), axis=0), np.sort(np.argwhere(Adj > 0), axis=0))
    Y, c = S.forward(p, X, E, row_ptr, col, bf16=False)
    assert np.allclose(c["s1"], S.AGG * (Adj @ c["h1"]), rtol=1e-13, atol=1e-13)
    assert np.allclose(c["s2"], S.AGG * (Adj @ c["h2"]), rtol=1e-13, atol=1e-13)


def test_bf16_rounding_is_nearest_even():
    assert S.round_bf16(np.array([1.0]))[0] == 1.0
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert S.round_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert S.round_bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    x = np.random.default_rng(2).normal(size=1000)
    r = S.round_bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-300)
