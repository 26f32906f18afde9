"""dem_find_pairs_static: the contact search for callers that cannot allocate device
memory (their memory belongs to their own pool allocator, or an allocation's implicit
synchronisation is unacceptable).  It must find exactly the pairs that a context's fine
search finds (dem_get_pairs), call after call, although every call reuses the same fixed
scratch array; honour the active mask, the caller's capacity and coarsened grids; refuse
totals above DEM_STATIC_MAX_PAIRS before writing anything; and leave the device's free
memory unchanged.  This file is collected last on purpose, and it also passes on its own
in a fresh process (the first call then performs the one-time address lookup)."""
import ctypes as C

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

MAX_PAIRS = 2 ** 31 - 1


def cloud(n, seed, L=0.03):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, (n, 3))
    R = rng.uniform(0.5e-3, 1e-3, n).astype(np.float32)
    rc = 1.3 * (2.0 * float(R.max()))           # the context's r_c = factor * d_max
    for k, f in enumerate([1.0, 1.0 - 2 ** -52, 1.0 + 2 ** -52]):
        x[2 * k + 1] = x[2 * k] + np.array([rc * f, 0.0, 0.0])
    cfg = dict(density=2500.0, particle=workloads.material(), wall=workloads.material(),
               gravity=(0, 0, 0), dt=1e-6, neighbor_factor=1.3, domain_lo=(0, 0, 0),
               domain_hi=(L, L, L))
    return workloads.Workload("cloud", cfg, [], x, np.zeros((n, 3)), np.zeros((n, 3)), R), rc


def sorted_pairs(p):
    p = np.asarray(p).reshape(-1, 2)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def brute_pairs(x, rc, active=None):
    """All i < j with dx*dx + dy*dy + dz*dz < rc*rc, summed left to right (the rounding of
    the context's fine search), among active particles."""
    out = []
    for i in range(len(x)):
        if active is not None and not active[i]:
            continue
        d = x[i + 1:] - x[i]
        s = d[:, 0] * d[:, 0]
        s = s + d[:, 1] * d[:, 1]
        s = s + d[:, 2] * d[:, 2]
        js = np.nonzero(s < rc * rc)[0] + i + 1
        if active is not None:
            js = js[active[js] != 0]
        out.extend((i, j) for j in js)
    return np.array(out, dtype=np.int32).reshape(-1, 2)


def raw_call(xd, n, rc, lo, hi, out=None, cap=0, active=None):
    import torch

    from paper_2106_09576_gb300.dem import load_library
    lib = load_library()
    cnt = C.c_int64(-1)
    lo_ = (C.c_double * 3)(*lo)
    hi_ = (C.c_double * 3)(*hi)
    code = lib.dem_find_pairs_static(C.c_void_p(xd.data_ptr()),
                                     None if active is None else C.c_void_p(active.data_ptr()), n, rc, lo_, hi_,
                                     None if out is None else C.c_void_p(out.data_ptr()), cap, C.byref(cnt),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, cnt.value


def test_static_scratch_pairs_match_context_pairs_twice_in_a_row():
    import torch

    from paper_2106_09576_gb300 import DEM
    from paper_2106_09576_gb300.dem import find_pairs_static

    for seed, n in ((11, 4000), (12, 2500)):      # two calls in a row, different sizes
        wl, rc = cloud(n, seed)
        ref = DEM(wl.cfg, wl.x, wl.v, wl.w, wl.radius, precision="fp64").pairs()
        xd = torch.tensor(wl.x, dtype=torch.float64, device="cuda")
        got = find_pairs_static(xd, rc, wl.cfg["domain_lo"], wl.cfg["domain_hi"]).cpu().numpy()
        assert len(ref) > 0
        assert np.array_equal(sorted_pairs(got), ref)

    # sizes beyond the documented maximum are refused with DEM_ERR_CAPACITY
    big = torch.zeros((262145, 3), dtype=torch.float64, device="cuda")
    code, _ = raw_call(big, 262145, 0.01, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    assert code == 3
    code, cnt = raw_call(big, 0, 0.01, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    assert code == 0 and cnt == 0


def test_active_mask_capacity_prefix_and_no_allocation():
    import torch

    from paper_2106_09576_gb300.dem import find_pairs_static

    wl, rc = cloud(3000, 21)
    rng = np.random.default_rng(5)
    act = (rng.random(wl.n) < 0.8).astype(np.uint8)
    ref = brute_pairs(wl.x, rc, act)
    xd = torch.tensor(wl.x, dtype=torch.float64, device="cuda")
    ad = torch.tensor(act, device="cuda")
    lo, hi = wl.cfg["domain_lo"], wl.cfg["domain_hi"]
    full = find_pairs_static(xd, rc, lo, hi, active=ad).cpu().numpy()
    assert len(ref) > 100 and np.array_equal(sorted_pairs(full), ref)
    # a caller buffer shorter than the total: count is the total, the buffer holds the
    # first `capacity` pairs of the (deterministic) full output, nothing beyond it moves
    cap = len(ref) // 3
    out = torch.full((cap + 8, 2), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    count = find_pairs_static(xd, rc, lo, hi, active=ad, out=out[:cap])
    free1 = torch.cuda.mem_get_info()[0]
    assert count == len(ref)
    o = out.cpu().numpy()
    assert np.array_equal(o[:cap], full[:cap]) and (o[cap:] == -7).all()
    assert free1 == free0, "the call with a caller buffer changed the device's free memory"
    # a second call with the same buffer: same answer
    assert find_pairs_static(xd, rc, lo, hi, active=ad, out=out[:cap]) == count
    assert np.array_equal(out.cpu().numpy()[:cap], full[:cap])


def test_coarsened_grid_and_one_crowded_cell():
    import torch

    from paper_2106_09576_gb300.dem import find_pairs_static

    # a cutoff of 1 mm in a 0.1 m box asks for 100^3 cells: coarsened below the limit
    rng = np.random.default_rng(8)
    x = rng.uniform(0.0, 0.1, (6000, 3))
    x[1] = x[0] + np.array([0.001, 0.0, 0.0])
    rc = 0.004
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    got = find_pairs_static(xd, rc, (0.0, 0.0, 0.0), (0.1, 0.1, 0.1)).cpu().numpy()
    assert np.array_equal(sorted_pairs(got), brute_pairs(x, rc))
    got = find_pairs_static(xd, 0.001 * (1 + 1e-9), (0.0, 0.0, 0.0), (0.1, 0.1, 0.1)).cpu().numpy()
    assert np.array_equal(sorted_pairs(got), brute_pairs(x, 0.001 * (1 + 1e-9)))
    # 2,000 particles in one cell, all within the cutoff of one another: every pair
    y = 0.5e-3 * rng.uniform(-1.0, 1.0, (2000, 3))
    yd = torch.tensor(y, dtype=torch.float64, device="cuda")
    got = find_pairs_static(yd, 0.01, (-0.01, -0.01, -0.01), (0.01, 0.01, 0.01)).cpu().numpy()
    i, j = np.triu_indices(2000, 1)
    assert np.array_equal(sorted_pairs(got), np.stack([i, j], 1).astype(np.int32))


def test_pair_total_above_the_limit_is_refused_before_writing():
    import torch

    # 70,000 particles within the cutoff of one another: 2,449,965,000 pairs > 2^31 - 1
    n = 70000
    rng = np.random.default_rng(9)
    xd = torch.tensor(1e-3 * rng.uniform(-1.0, 1.0, (n, 3)), dtype=torch.float64, device="cuda")
    out = torch.full((64, 2), -7, dtype=torch.int32, device="cuda")
    code, cnt = raw_call(xd, n, 0.01, (-0.01, -0.01, -0.01), (0.01, 0.01, 0.01), out=out, cap=64)
    assert code == 3 and cnt == n * (n - 1) // 2 > MAX_PAIRS
    assert (out.cpu().numpy() == -7).all()
    # the scratch is still usable afterwards
    wl, rc = cloud(1500, 31)
    from paper_2106_09576_gb300.dem import find_pairs_static
    got = find_pairs_static(torch.tensor(wl.x, dtype=torch.float64, device="cuda"), rc, wl.cfg["domain_lo"],
                            wl.cfg["domain_hi"]).cpu().numpy()
    assert np.array_equal(sorted_pairs(got), brute_pairs(wl.x, rc))
