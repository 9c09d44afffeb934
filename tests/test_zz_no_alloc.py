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


def test_static_sort_rejects_sizes_beyond_its_maximum():
    import torch
    from paper_2602_21244_gb300 import dsmc as D
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    ef = torch.zeros(0, dtype=torch.float64, device="cuda")
    with pytest.raises(D.DsmcError) as ex:
        D.sort_cells_static(e, ef, ef, ef, D.STATIC_SORT_MAX_CELLS + 1)
    assert ex.value.code == D.DSMC_ERR_UNSUPPORTED
