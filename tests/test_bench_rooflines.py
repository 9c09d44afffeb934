"""The bench's roofline arithmetic on CPU: bench.phase_bytes against the bytes
each phase must move, written out here from the data it reads and writes, and
bench.phase_rooflines' achieved rates, fractions and binding roof against the
same definitions (the neural MLP's FLOPs and special-function operations per
pair from its layer widths)."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

PIPE = {"mufu_tops": 10.0, "fp64_tflops": 1.0, "fp32_tflops": 70.0}


def _bytes(n, nc, pairs):
    v = 3 * 8   # one particle's FP64 velocity
    return {
        # cell id and velocity in; perm and sorted velocity out; cell_start
        "sort": (4 + v + 4 + v) * n + 4 * (nc + 1),
        # sorted velocities read; five FP64 moments written per cell
        "moments": v * n + 5 * 8 * nc,
        # sorted velocities read; (sigma g)_max read and written per cell;
        # per accepted pair an int4 record and a dependency word written
        "select": v * n + 2 * 8 * nc + (16 + 4) * pairs,
        # both particles' velocities read and written, and the two indices
        "collide": (2 * 2 * v + 2 * 4) * pairs,
        # velocities read and written; the pre-collision moments read
        "moment_match": 2 * v * n + 5 * 8 * nc,
    }


def test_phase_bytes_per_unit():
    for n, nc, pairs in [(0, 1, 0), (1000, 10, 300), (9144283, 150000, 6882379)]:
        assert bench.phase_bytes(n, nc, pairs) == _bytes(n, nc, pairs)


def test_phase_rooflines_rates_fractions_and_bound():
    pk = {"hbm_gbs": 5000.0, "bf16_tflops": 2000.0}
    n, nc, pairs = 1_000_000, 20_000, 500_000
    ms = {"sort": 0.1, "moments": 0.02, "select": 0.05, "collide": 0.2, "moment_match": 0.03}
    out = bench.phase_rooflines("neural", n, nc, pairs, ms, PIPE, pk)
    b = _bytes(n, nc, pairs)
    for ph, t in ms.items():
        roofs = out[ph]["roofs"]
        assert math.isclose(roofs["hbm"]["achieved"], b[ph] / (t * 1e-3) / 1e9)
        assert math.isclose(roofs["hbm"]["frac"], roofs["hbm"]["achieved"] / 5000.0)
        assert "issue" not in roofs   # instruction counts belong to the full-size gas only
        bound = max(roofs, key=lambda k: roofs[k]["frac"])
        assert out[ph]["bound"] == bound and out[ph]["frac"] == roofs[bound]["frac"]
    col = out["collide"]["roofs"]
    # input layer 8 -> 128, two 128 x 128 hidden layers, output 128 -> 3; 2 FLOP per MAC
    flop = 2 * (8 * 128 + 2 * 128 * 128 + 128 * 3)
    assert flop == 68352
    assert math.isclose(col["tensor"]["achieved"], pairs * flop / 0.2e-3 / 1e12)
    assert math.isclose(col["tensor"]["frac"], col["tensor"]["achieved"] / 2000.0)
    # three SiLU layers of 128 values, 1.25 special-function operations each
    assert math.isclose(col["mufu"]["achieved"], pairs * 3 * 128 * 1.25 / 0.2e-3 / 1e12)


def test_issue_roof_only_at_the_reference_size_and_fallback_peak():
    n = bench.ISSUE_REF_PARTICLES
    ms = {"sort": 0.4, "moments": 0.1, "select": 0.5, "collide": 1.7, "moment_match": 0.18}
    issue_peak = 152 * 4 * 2070e6
    out = bench.phase_rooflines("neural", n, 150000, 6882379, ms, PIPE, None, issue_peak=issue_peak)
    for ph in ("sort", "moments", "select", "moment_match"):
        iss = out[ph]["roofs"]["issue"]
        assert math.isclose(iss["achieved"], bench.PHASE_WARP_INSTR[1][ph] / (ms[ph] * 1e-3) / 1e9)
        assert math.isclose(iss["peak"], issue_peak / 1e9)
    assert "issue" not in out["collide"]["roofs"]
    assert out["sort"]["roofs"]["hbm"]["peak"] == 6800.0   # no measured peaks: the fallback
    # the VHS path's selection has its own count (far fewer candidates)
    vhs = bench.phase_rooflines("vhs", n, 150000, 317985, ms, PIPE, None, issue_peak=issue_peak)
    assert math.isclose(vhs["select"]["roofs"]["issue"]["achieved"],
                        bench.PHASE_WARP_INSTR[0]["select"] / (ms["select"] * 1e-3) / 1e9)
