"""The surrogate network's CUDA kernels against the NumPy FP64 reference
(oracle/surrogate_ref.py): the BF16 tensor-core product, the forward pass and every
parameter gradient on small seeded graphs, within bounds set by BF16 rounding; and a
training run that must reduce the loss."""
import numpy as np
import pytest

from oracle import surrogate_ref as S

pytestmark = pytest.mark.gpu


def bf16_array(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32), device="cuda").to(torch.bfloat16)


def test_bf16_tensor_core_product_matches_fp64():
    import torch
    from paper_2106_09576_gb300 import surrogate as SG
    rng = np.random.default_rng(0)
    for (M, K, N) in [(1000, 144, 128), (37, 16, 8), (513, 256, 128)]:
        A = S.round_bf16(rng.normal(size=(M, K)))
        B = S.round_bf16(rng.normal(size=(K, N)))
        Ct = torch.empty((M, N), dtype=torch.float32, device="cuda")
        At, Bt = bf16_array(A), bf16_array(B)          # kept alive until the product is read
        code = SG.lib().surr_gemm_bf16(SG._p(At), SG._p(Bt), SG._p(Ct), M, K, N, None)
        assert code == 0
        ref = A @ B
        err = np.abs(Ct.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < 1e-5, (M, K, N, err)


def test_tcgen05_product_matches_fp64():
    """The 5th-generation tensor-core product (tcgen05.mma, accumulator in tensor memory)
    the forward pass uses for its 128-wide layers: ragged row counts, every K the network
    uses, one and several tiles per CTA."""
    import ctypes
    import torch
    from paper_2106_09576_gb300 import surrogate as SG
    rng = np.random.default_rng(3)
    for (M, K) in [(1000, 144), (37, 16), (513, 256), (128, 128), (300, 64), (40000, 256)]:
        A = S.round_bf16(rng.normal(size=(M, K)))
        B = S.round_bf16(rng.normal(size=(K, 128)))
        Ct = torch.full((M, 128), float("nan"), dtype=torch.float32, device="cuda")
        At, Bt = bf16_array(A), bf16_array(B)          # kept alive until the product is read
        assert SG.lib().surr_gemm_bf16_tc(SG._p(At), SG._p(Bt), SG._p(Ct), M, K, None) == 0
        ref = A @ B
        got = Ct.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-5, (M, K, err)
    count = ctypes.c_int(-1)
    assert SG.lib().surr_tc_timeouts(ctypes.byref(count)) == 0 and count.value == 0


def test_tcgen05_rejects_shapes_outside_its_limits():
    import torch
    from paper_2106_09576_gb300 import surrogate as SG
    A = torch.zeros((64, 272), dtype=torch.bfloat16, device="cuda")
    B = torch.zeros((272, 128), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((64, 128), dtype=torch.float32, device="cuda")
    assert SG.lib().surr_gemm_bf16_tc(SG._p(A), SG._p(B), SG._p(C), 64, 272, None) == 1    # K > 256
    assert SG.lib().surr_gemm_bf16_tc(SG._p(A), SG._p(B), SG._p(C), 64, 40, None) == 1     # K % 16
    assert SG.lib().surr_gemm_bf16_tc(None, SG._p(B), SG._p(C), 64, 16, None) == 1


def test_tcgen05_waits_give_up_and_report():
    """The bound on the tensor-core kernel's mbarrier waits: a barrier that nothing arrives
    on must make every waiting thread give up, count one timeout and let the kernel return
    (no fault, no hang); the product kernel's own timeout counter is untouched."""
    import ctypes
    from paper_2106_09576_gb300 import surrogate as SG
    before = ctypes.c_int(-1)
    assert SG.lib().surr_tc_timeouts(ctypes.byref(before)) == 0
    gave_up, timed_out = ctypes.c_int(-1), ctypes.c_int(-1)
    assert SG.lib().surr_tc_wait_probe(ctypes.byref(gave_up), ctypes.byref(timed_out)) == 0
    assert gave_up.value == 128 and 1 <= timed_out.value <= 128
    after = ctypes.c_int(-1)
    assert SG.lib().surr_tc_timeouts(ctypes.byref(after)) == 0 and after.value == before.value


def random_case(n=300, seed=1):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0, 1, (n, 3))
    d = np.linalg.norm(pts[:, None, :] - pts[None, :, :], axis=-1)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if d[i, j] < 0.15]
    row_ptr, col = S.csr(pairs, n)
    X = rng.normal(size=(n, S.FIN))
    E = rng.normal(size=(len(col), S.EIN))
    _, total = S.layout()
    p = (rng.normal(scale=0.06, size=total)).astype(np.float32).astype(np.float64)
    return pairs, row_ptr, col, X, E, p


def gpu_graph(pairs, n, row_ptr, col):
    import torch
    from paper_2106_09576_gb300 import surrogate as SG
    g = SG.Graph.__new__(SG.Graph)
    g.n, g.n_edges = n, len(col)
    g.row_ptr = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    g.col = torch.empty(max(len(col), 1), dtype=torch.int32, device="cuda")
    g.recv = torch.empty(max(len(col), 1), dtype=torch.int32, device="cuda")
    P = torch.tensor(np.array(pairs, np.int32).reshape(-1, 2), device="cuda")
    scratch = torch.empty(2 * n + 1, dtype=torch.int32, device="cuda")
    assert SG.lib().surr_build_csr(SG._p(P), len(pairs), n, SG._p(g.row_ptr), SG._p(g.col), SG._p(scratch),
                                   None) == 0
    assert np.array_equal(g.row_ptr.cpu().numpy(), row_ptr)
    assert np.array_equal(g.col.cpu().numpy()[:len(col)], col)
    return g


def test_forward_and_gradients_match_the_reference():
    import torch
    from paper_2106_09576_gb300 import surrogate as SG
    pairs, row_ptr, col, X, E, p = random_case()
    n = len(row_ptr) - 1
    g = gpu_graph(pairs, n, row_ptr, col)
    net = SG.SurrogateNet()
    net.params.copy_(torch.tensor(p, dtype=torch.float32))
    net.sync_bf16()
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    Et = torch.tensor(E, dtype=torch.float32, device="cuda")
    Y = net.forward(Xt, Et, g).cpu().numpy().astype(np.float64)
    Yr, c = S.forward(p, X, E, row_ptr, col, bf16=True)
    rel = np.linalg.norm(Y - Yr) / np.linalg.norm(Yr)
    print(f"forward relative error {rel:.2e}")
    assert rel < 1e-2
    dY = np.random.default_rng(5).normal(size=Y.shape)
    dY[:, 6:] = 0.0
    grad = net.backward(torch.tensor(dY, dtype=torch.float32, device="cuda"), g).cpu().numpy().astype(np.float64)
    gr = S.backward(p, dY, c, row_ptr, col)
    off, total = S.layout()
    for l, (ow, ob) in enumerate(off):
        i, j = S.SHAPES[l]
        for name, lo, hi in (("W", ow, ow + i * j), ("b", ob, ob + j)):
            e = np.linalg.norm(grad[lo:hi] - gr[lo:hi]) / max(np.linalg.norm(gr[lo:hi]), 1e-30)
            print(f"layer {l} {name}: gradient relative error {e:.2e}")
            assert e < 3e-2, (l, name, e)


def test_forward_matches_the_reference_when_ctas_take_several_tiles():
    """12,000 nodes and ~120,000 edges: the edge layer has ~940 tiles of 128 rows for 304
    CTAs, so every CTA streams several tiles through its stage ring, alternates its two
    tensor-memory accumulators and gathers receiver rows fetched a tile ahead."""
    import torch
    spatial = pytest.importorskip("scipy.spatial")
    from paper_2106_09576_gb300 import surrogate as SG
    rng = np.random.default_rng(11)
    n = 12000
    pts = rng.uniform(0, 1, (n, 3))
    pairs = sorted(spatial.cKDTree(pts).query_pairs(0.0605))
    row_ptr, col = S.csr(pairs, n)
    assert len(col) > 3 * 304 * 128
    X = rng.normal(size=(n, S.FIN))
    E = rng.normal(size=(len(col), S.EIN))
    _, total = S.layout()
    p = (rng.normal(scale=0.06, size=total)).astype(np.float32).astype(np.float64)
    g = gpu_graph(pairs, n, row_ptr, col)
    net = SG.SurrogateNet()
    net.params.copy_(torch.tensor(p, dtype=torch.float32))
    net.sync_bf16()
    Y = net.forward(torch.tensor(X, dtype=torch.float32, device="cuda"),
                    torch.tensor(E, dtype=torch.float32, device="cuda"), g).cpu().numpy().astype(np.float64)
    Yr, _ = S.forward(p, X, E, row_ptr, col, bf16=True)
    rel = np.linalg.norm(Y - Yr) / np.linalg.norm(Yr)
    worst = np.abs(Y - Yr).max() / np.abs(Yr).max()
    print(f"forward relative error {rel:.2e}, worst element {worst:.2e}")
    assert rel < 1e-2 and worst < 5e-2


def test_training_reduces_the_loss_on_a_learnable_target():
    import torch
    from paper_2106_09576_gb300 import surrogate as SG
    pairs, row_ptr, col, X, E, _ = random_case(n=400, seed=3)
    n = len(row_ptr) - 1
    g = gpu_graph(pairs, n, row_ptr, col)
    net = SG.SurrogateNet()
    # target: a smooth function of the node's inputs and of its neighbours'
    Adj = np.zeros((n, n))
    recv = np.repeat(np.arange(n), np.diff(row_ptr))
    Adj[recv, col] = 1.0
    T = np.tanh(X[:, :6] + 0.2 * (Adj @ X[:, 6:12]))
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    Et = torch.tensor(E, dtype=torch.float32, device="cuda")
    Tt = torch.tensor(T, dtype=torch.float32, device="cuda")
    w = torch.ones(6, dtype=torch.float32, device="cuda")
    losses = [float(net.train_step(Xt, Et, g, Tt, w, 1e-3).item()) for _ in range(300)]
    print("loss", losses[0], "->", losses[-1])
    assert losses[-1] < 0.2 * losses[0]
