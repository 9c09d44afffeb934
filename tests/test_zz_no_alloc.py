"""The allocation-free cell sort (dsmc_sort_cells_static) against the regular
one (dsmc_sort_cells).

Some callers cannot allocate device memory when they sort -- a solver that
reserved the whole GPU for its particle arrays, or code that runs where a
cudaMalloc is not allowed -- so the library offers a sort whose scratch is a
fixed device array inside the library.  These tests check, through the C
ABI, that it returns exactly what the regular sort returns (the sort is
integer work: bit for bit), on two calls in a row (the shared scratch keeps
the previous call's contents and must be cleared), and that it refuses
sizes beyond its stated maximum.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2602_21244_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _regular(C, w, n_cells):
    import torch
    return C.sort_cells(torch.from_numpy(w[0]).cuda(), *[torch.from_numpy(x).cuda() for x in w[1:]],
                        n_cells)


def _static(D, w, n_cells, out):
    import torch
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    D.sort_cells_static(torch.from_numpy(w[0]).cuda(), *[torch.from_numpy(x).cuda() for x in w[1:]],
                        n_cells, out=out, status=status)
    return status


def test_static_sort_matches_regular_sort_twice():
    import torch
    from paper_2602_21244_gb300 import dsmc as D
    C = D.Context(0)
    a = W.hypersonic(scale=0.2, seed=3)          # ~370k particles, 6000 cells
    b = W.cavity(nx=60, ny=50, seed=4)            # different sizes, different cells
    for wl in (a, b):
        w = (wl["cell_id"], wl["vx"], wl["vy"], wl["vz"])
        n, nc = len(wl["cell_id"]), wl["n_cells"]
        out = dict(perm=torch.empty(n, dtype=torch.int32, device="cuda"),
                   cell_start=torch.empty(nc + 1, dtype=torch.int32, device="cuda"),
                   svx=torch.empty(n, dtype=torch.float64, device="cuda"),
                   svy=torch.empty(n, dtype=torch.float64, device="cuda"),
                   svz=torch.empty(n, dtype=torch.float64, device="cuda"))
        status = _static(D, w, nc, out)
        ref = _regular(C, w, nc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert C.sync_status() == 0
        for k in ("perm", "cell_start", "svx", "svy", "svz"):
            assert torch.equal(out[k], ref[k]), k
    C.close()


def _outputs(n, nc):
    import torch
    return dict(perm=torch.empty(n, dtype=torch.int32, device="cuda"),
                cell_start=torch.empty(nc + 1, dtype=torch.int32, device="cuda"),
                svx=torch.empty(n, dtype=torch.float64, device="cuda"),
                svy=torch.empty(n, dtype=torch.float64, device="cuda"),
                svz=torch.empty(n, dtype=torch.float64, device="cuda"))


def _large_cell_gas(n_big, nc=3000, n_rest=60000, seed=11):
    """A gas of small cells plus one cell of n_big particles spread through
    the input order (the block-wide path of the sort for cells above 1024)."""
    rng = np.random.default_rng(seed)
    cid = rng.integers(0, nc, n_rest + n_big).astype(np.int32)
    cid[rng.permutation(n_rest + n_big)[:n_big]] = 17
    v = [rng.standard_normal(n_rest + n_big) * 300.0 for _ in range(3)]
    return (cid, *v), nc


@pytest.mark.parametrize("n_big", [1025, 5000, 70000])
def test_static_sort_large_cell(n_big):
    import torch
    from paper_2602_21244_gb300 import dsmc as D
    C = D.Context(0)
    w, nc = _large_cell_gas(n_big)
    out = _outputs(len(w[0]), nc)
    for _ in range(2):   # the second call starts from the first call's scratch
        status = _static(D, w, nc, out)
        ref = _regular(C, w, nc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        for k in ("perm", "cell_start", "svx", "svy", "svz"):
            assert torch.equal(out[k], ref[k]), k
    C.close()


def test_static_sort_one_cell_of_maximum_size():
    """Every particle (2^20, the stated maximum) in one cell: the same order
    as the regular sort, in a bounded time."""
    import torch
    from paper_2602_21244_gb300 import dsmc as D
    C = D.Context(0)
    n, nc = D.STATIC_SORT_MAX_N, 4
    rng = np.random.default_rng(5)
    w = (np.full(n, 2, np.int32), *[rng.standard_normal(n) for _ in range(3)])
    out = _outputs(n, nc)
    dev = [torch.from_numpy(x).cuda() for x in w]
    D.sort_cells_static(*dev, nc, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    D.sort_cells_static(*dev, nc, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ref = _regular(C, w, nc)
    torch.cuda.synchronize()
    for k in ("perm", "cell_start", "svx", "svy", "svz"):
        assert torch.equal(out[k], ref[k]), k
    assert torch.equal(out["perm"], torch.arange(n, dtype=torch.int32, device="cuda"))
    print(f"one cell of {n} particles: {ms:.2f} ms")
    assert ms < 10.0, ms
    C.close()


def test_static_sort_bad_cell_id_and_no_particles():
    import torch
    from paper_2602_21244_gb300 import dsmc as D
    rng = np.random.default_rng(2)
    n, nc = 4000, 50
    cid = rng.integers(0, nc, n).astype(np.int32)
    cid[1234] = nc + 3
    w = (cid, *[rng.standard_normal(n) for _ in range(3)])
    out = _outputs(n, nc)
    status = _static(D, w, nc, out)
    torch.cuda.synchronize()
    assert int(status.item()) == D.DSMC_ERR_ARG
    cs = out["cell_start"].cpu().numpy()
    assert cs[-1] == n - 1
    ok = np.flatnonzero(cid < nc)
    want = ok[np.argsort(cid[ok], kind="stable")]
    assert np.array_equal(out["perm"].cpu().numpy()[:n - 1], want)
    # no particles: every cell empty, nothing else written
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    ef = torch.zeros(0, dtype=torch.float64, device="cuda")
    res = D.sort_cells_static(e, ef, ef, ef, nc)
    torch.cuda.synchronize()
    assert not res["cell_start"].any()


def test_static_sort_checks_output_lengths():
    import torch
    from paper_2602_21244_gb300 import dsmc as D
    w = (np.zeros(100, np.int32), *[np.zeros(100) for _ in range(3)])
    out = _outputs(100, 4)
    out["perm"] = out["perm"][:50]
    with pytest.raises(ValueError):
        _static(D, w, 4, out)


def test_static_sort_rejects_sizes_beyond_its_maximum():
    import torch
    from paper_2602_21244_gb300 import dsmc as D
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    ef = torch.zeros(0, dtype=torch.float64, device="cuda")
    with pytest.raises(D.DsmcError) as ex:
        D.sort_cells_static(e, ef, ef, ef, D.STATIC_SORT_MAX_CELLS + 1)
    assert ex.value.code == D.DSMC_ERR_UNSUPPORTED
