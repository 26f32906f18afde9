"""Plain NumPy FP64 reference of the surrogate network (TEST INFRASTRUCTURE ONLY).

The GPU implementation (paper_2106_09576_gb300/csrc/surrogate.cu) is checked against this
file: forward outputs and parameter gradients on small graphs.  It shares no code with the
GPU path.  Written from the network's definition (include/surrogate.h):

  h0 = relu(X W0 + b0)
  m_e = relu([h0[recv(e)] | E_e] W1 + b1)          e = an edge j -> i, recv(e) = i
  a_i = c * (sum of m_e over the edges into i)      c = 0.125
  h1 = h0 + relu([h0 | a] W2 + b2)
  h2 = h1 + relu([h1 | s1] W3 + b3),  s1_i = c * (sum of h1_j over the neighbours j of i)
  h3 = h2 + relu([h2 | s2] W4 + b4),  s2_i = c * (sum of h2_j over the neighbours j of i)
  Y  = h3 W5 + b5

With `bf16=True` the values the GPU stores in BF16 (inputs, weights, activations, sums) are
rounded to BF16 (round to nearest, ties to even) at the same points; products and sums are
FP64.  The backward pass is the exact FP64 gradient of that computation, treating each
rounding as the identity (the GPU does the same).  With `bf16=False` everything is FP64, and
the gradient is pinned against central finite differences (tests/test_surrogate_ref.py).
"""
import numpy as np

H, FIN, EIN, NOUT = 128, 16, 16, 8
AGG = 0.125          # the scale of every neighbour or edge sum
SHAPES = [(FIN, H), (H + EIN, H), (2 * H, H), (2 * H, H), (2 * H, H), (H, NOUT)]


def layout():
    """(offset of W_l, offset of b_l) for l = 0..5 in the flat parameter array, and the total."""
    off, o = [], 0
    for (i, j) in SHAPES:
        off.append((o, o + i * j))
        o += i * j + j
    return off, o


def unpack(p):
    off, _ = layout()
    Ws, bs = [], []
    for (i, j), (ow, ob) in zip(SHAPES, off):
        Ws.append(p[ow:ow + i * j].reshape(i, j))
        bs.append(p[ob:ob + j])
    return Ws, bs


def round_bf16(a):
    """Round an array to BF16 precision (nearest, ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def csr(pairs, n):
    """Receiver-sorted CSR (rows in increasing sender order) of the undirected pairs."""
    rows = [[] for _ in range(n)]
    for a, b in pairs:
        rows[a].append(b)
        rows[b].append(a)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = []
    for i in range(n):
        row_ptr[i + 1] = row_ptr[i] + len(rows[i])
        col.extend(sorted(rows[i]))
    return row_ptr, np.array(col, dtype=np.int64)


def forward(p, X, E, row_ptr, col, bf16=True):
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Ws, bs = unpack(np.asarray(p, dtype=np.float64))
    Wr = [r(W) for W in Ws]
    n = len(row_ptr) - 1
    recv = np.repeat(np.arange(n), np.diff(row_ptr))
    c = {}
    c["X"] = r(X)
    c["E"] = r(E)
    z0 = c["X"] @ Wr[0] + bs[0]
    c["h0"] = r(np.maximum(z0, 0))
    A1 = np.concatenate([c["h0"][recv], c["E"]], axis=1)
    z1 = A1 @ Wr[1] + bs[1]
    c["u1"] = r(np.maximum(z1, 0))
    a = np.zeros((n, H))
    np.add.at(a, recv, c["u1"])
    c["a"] = r(AGG * a)
    z2 = np.concatenate([c["h0"], c["a"]], axis=1) @ Wr[2] + bs[2]
    u2 = np.maximum(z2, 0)
    c["u2"] = r(u2)
    c["h1"] = r(c["h0"] + u2)
    hs = c["h1"]
    for l, (sk, uk, hk) in zip((3, 4), (("s1", "u3", "h2"), ("s2", "u4", "h3"))):
        s = np.zeros((n, H))
        np.add.at(s, recv, hs[col])
        c[sk] = r(AGG * s)
        z = np.concatenate([hs, c[sk]], axis=1) @ Wr[l] + bs[l]
        u = np.maximum(z, 0)
        c[uk] = r(u)
        c[hk] = r(hs + u)
        hs = c[hk]
    Y = hs @ Wr[5] + bs[5]
    c["recv"], c["Wr"] = recv, Wr
    return Y, c


def backward(p, dY, c, row_ptr, col):
    """Gradient of sum(dY * Y) with respect to the flat parameters."""
    off, total = layout()
    Wr, recv = c["Wr"], c["recv"]
    n = len(row_ptr) - 1
    g = np.zeros(total)

    def put(l, dW, db):
        ow, ob = off[l]
        g[ow:ow + dW.size] = dW.ravel()
        g[ob:ob + db.size] = db

    put(5, c["h3"].T @ dY, dY.sum(0))
    dh = dY @ Wr[5].T
    for l, hin, sk, uk in ((4, "h2", "s2", "u4"), (3, "h1", "s1", "u3")):
        dz = dh * (c[uk] > 0)
        A = np.concatenate([c[hin], c[sk]], axis=1)
        put(l, A.T @ dz, dz.sum(0))
        dA = dz @ Wr[l].T
        ds = AGG * dA[:, H:]
        dns = np.zeros((n, H))
        np.add.at(dns, col, ds[recv])     # transpose of the neighbour sum
        dh = dh + dA[:, :H] + dns
    dz = dh * (c["u2"] > 0)
    A = np.concatenate([c["h0"], c["a"]], axis=1)
    put(2, A.T @ dz, dz.sum(0))
    dA = dz @ Wr[2].T
    dh0 = dh + dA[:, :H]
    da = dA[:, H:]
    dz1 = AGG * da[recv] * (c["u1"] > 0)
    A1 = np.concatenate([c["h0"][recv], c["E"]], axis=1)
    put(1, A1.T @ dz1, dz1.sum(0))
    dA1 = dz1 @ Wr[1].T
    np.add.at(dh0, recv, dA1[:, :H])
    dz0 = dh0 * (c["h0"] > 0)
    put(0, c["X"].T @ dz0, dz0.sum(0))
    return g
