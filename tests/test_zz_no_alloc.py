"""dem_find_pairs_static: the contact search for callers that cannot allocate device
memory (their memory belongs to their own pool allocator, or an allocation's implicit
synchronisation is unacceptable).  It must find exactly the pairs that a context's fine
search finds (dem_get_pairs), call after call, although every call reuses the same fixed
scratch array.  This file is collected last on purpose, and it also passes on its own in a
fresh process (the first call then performs the one-time address lookup)."""
import ctypes as C

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


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
    p = np.asarray(p)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def test_static_scratch_pairs_match_context_pairs_twice_in_a_row():
    import torch

    from paper_2106_09576_gb300 import DEM
    from paper_2106_09576_gb300.dem import find_pairs_static, load_library

    for seed, n in ((11, 4000), (12, 2500)):      # two calls in a row, different sizes
        wl, rc = cloud(n, seed)
        ref = DEM(wl.cfg, wl.x, wl.v, wl.w, wl.radius, precision="fp64").pairs()
        xd = torch.tensor(wl.x, dtype=torch.float64, device="cuda")
        got = find_pairs_static(xd, rc, wl.cfg["domain_lo"], wl.cfg["domain_hi"]).cpu().numpy()
        assert len(ref) > 0
        assert np.array_equal(sorted_pairs(got), ref)

    # sizes beyond the documented maximum are refused with DEM_ERR_CAPACITY
    lib = load_library()
    cnt = C.c_int64(0)
    lo = (C.c_double * 3)(0.0, 0.0, 0.0)
    hi = (C.c_double * 3)(1.0, 1.0, 1.0)
    big = torch.zeros((262145, 3), dtype=torch.float64, device="cuda")
    code = lib.dem_find_pairs_static(C.c_void_p(big.data_ptr()), None, 262145, 0.01, lo, hi, None, 0,
                                     C.byref(cnt), None)
    assert code == 3
