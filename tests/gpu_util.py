"""Shared helpers of the GPU parity tests (CUDA path vs CPU oracle)."""
import math

import numpy as np

KB = 1.380649e-23
_CTX = None


def torch():
    import torch as T
    return T


def ctx():
    global _CTX
    from paper_2602_21244_gb300 import dsmc as D
    if _CTX is None:
        _CTX = D.Context(0)
    return _CTX


def cuda(a, dtype=None):
    T = torch()
    t = T.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def w_bits_tensor(bits):
    return cuda(bits.view(np.int16))


def gpu_step_pieces(wl, sgmax0, step=0, capacity=1 << 22, order=0):
    """Sort, moments and selection on the GPU for a workload dict (order:
    the pair list's buckets, rounds or claim levels)."""
    T = torch()
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    gas = D.make_gas(wl["gas"])
    cid = cuda(wl["cell_id"])
    vx, vy, vz = cuda(wl["vx"]), cuda(wl["vy"]), cuda(wl["vz"])
    srt = C.sort_cells(cid, vx, vy, vz, wl["n_cells"])
    mom = C.cell_moments(srt["cell_start"], srt["svx"], srt["svy"], srt["svz"])
    sg = cuda(sgmax0).clone()
    sel = C.select_pairs(gas, srt["cell_start"], srt["svx"], srt["svy"], srt["svz"], sg, step,
                         capacity, order=order)
    T.cuda.synchronize()
    return gas, srt, mom, sg, sel


def sel_host(sel):
    info = host(sel["info"])
    n = int(info[0])
    R = int(info[2] & 0xFFFFFFFF)
    ro = host(sel["round_offsets"])[:R + 1]
    pairs = host(sel["pairs"])[:n] if n else np.zeros((0, 4), np.int32)
    return dict(n_pairs=n, n_cand=int(info[1]), n_rounds=R, ro=ro, pairs=pairs)


def expected_buckets(ref, n_cells, order):
    """Bucket of each of the oracle's pairs (candidate order) in the GPU's
    list: its round, or its claim level = round + (n_rounds - 1 - the last
    round of its cell), derived here from the oracle's rounds."""
    r = np.asarray(ref["round"], np.int64)
    if order == 0 or len(r) == 0:
        return r
    last = np.full(n_cells, -1, np.int64)
    np.maximum.at(last, np.asarray(ref["cell"], np.int64), r)
    return r + (ref["n_rounds"] - 1) - last[np.asarray(ref["cell"], np.int64)]


def expected_deps(ref, bucket):
    """deps of the oracle's pairs: the 1-based buckets of the previous pairs of
    i and j in candidate order (0 = none), i | j << 16."""
    want = np.zeros(len(ref["i"]), np.uint32)
    last = {}
    for k, (i, j, b) in enumerate(zip(ref["i"].tolist(), ref["j"].tolist(), np.asarray(bucket).tolist())):
        want[k] = last.get(i, 0) | (last.get(j, 0) << 16)
        last[i] = last[j] = b + 1
    return want


def pairs_round_of(sh):
    """Bucket (round or level) of each pair of a bucket-major GPU pair list."""
    r = np.zeros(sh["n_pairs"], np.int32)
    for q in range(sh["n_rounds"]):
        r[sh["ro"][q]:sh["ro"][q + 1]] = q
    return r


def c_ref(mass=6.63e-26, T=273.0):
    return math.sqrt(2 * KB * T / mass)
