"""Benchmark of the DSMC collision step on GB300.

One step = sort by cell, pre-step cell moments, NTC selection with the
round schedule, the pair updates of one path, cell moment matching: every
row of the method's hot path, over the hypersonic argon gas (500 x 300
cells around a disc, about 9.2 million particles, Mach-10 shock profile).

Timing: W untimed warm-up steps, then K timed steps.  Before every step
the pristine unsorted input (cell ids and velocities, 258 MB, larger than
L2) is copied back, outside the timed region, so each step sorts a
shuffled gas and starts with a cold L2.  The headline times the whole step
as one CUDA graph (dsmc_step_graph_launch) between CUDA events on its
stream; a second, un-graphed pass with events between the phases gives the
per-phase (per-kernel) times.

Output: one JSON line on rank 0.  The headline ``value`` is accepted pair
collisions per second of the whole step on the neural path; ``paths``
holds every update rule; for the VHS and look-up rules ``fused`` times the
same step fused into one pass over cell groups (dsmc_step_fused).  Multi-GPU runs are replicas (each rank its
own gas, no collective on the data path): ``value`` sums over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MLP_FLOP_PER_PAIR = 2 * (8 * 128 + 128 * 128 * 2 + 128 * 3)   # 68,352 (unpadded)
# chi-MLP 2 -> 512, 512, 512, 256, 128 -> 1: 1,378,560 FLOP per query (unpadded)
CHI_MLP_FLOP_PER_QUERY = 2 * (2 * 512 + 512 * 512 * 2 + 512 * 256 + 256 * 128 + 128)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per pair of
# k_collide_neural, from one ncu capture of a full-size launch on the
# hypersonic gas: 1000.1 + 941.5 MB for about 6.885 million pairs
# (the committed ncu summary of this kernel); the roofline's traffic is this
# times the pairs of the timed launch.
NEURAL_DRAM_BYTES_PER_PAIR = (1000.14e6 + 941.49e6) / 6.885e6
CANDIDATE_BYTES = 48                                             # two FP64 3-vectors read
PAIR_BYTES = 104                                                 # 2x24 read + 2x24 write + 8 index
# special-function operations per pair of the neural collide: 3 hidden layers
# x 128 SiLU values at 1.25 MUFU operations each (four exponentials and one
# reciprocal per four values)
MLP_MUFU_PER_PAIR = 3 * 128 * 1.25

# Per-pair instruction counts of the ALU-bound collide kernels, from one ncu
# capture each (the committed ncu summary of the collide kernels: sm__sass_thread_inst_executed_
# op_{dfma,dadd,dmul,ffma,ffma2,fadd,fmul,...}_pred_on.sum and
# sm__inst_executed_pipe_xu.sum x 32, divided by the launch's pairs); None
# until captured for the current kernels.  FP64 and FP32 in FLOPs (an FMA is
# two), MUFU in thread operations.
KERNEL_OPS = {
    "k_collide_vhs": {"fp64_flop": 99.2, "fp32_flop": 0.0, "mufu": 25.4},
    "k_collide_table": {"fp64_flop": 37.0, "fp32_flop": 180.0, "mufu": 18.0},
    "k_collide_jager": {"fp64_flop": 340.3, "fp32_flop": 7560.6, "mufu": 661.7},
    "k_jager_chi": {"fp64_flop": 179.3, "fp32_flop": 9008.9, "mufu": 1915.1},
}

# the kernels of each phase of the step (for the per-phase rooflines)
# Warp instructions issued per step by the shared phases on the full
# hypersonic gas (9,144,283 particles, 150,000 cells), from one ncu capture
# of smsp__inst_executed.sum over a bench run (median launch of each kernel
# times its launches per step); the selection's depend on the collision
# model (21.6M candidates for hard spheres, 3.2M for VHS).  They give the
# phases' instruction-issue roof (only at that size).
ISSUE_REF_PARTICLES = 9144283
PHASE_WARP_INSTR = {
    1: {"sort": 151.11e6, "moments": 60.94e6, "select": 249.49e6, "moment_match": 77.84e6},
    0: {"sort": 151.12e6, "moments": 60.95e6, "select": 77.67e6, "moment_match": 77.84e6},
}
PHASE_KERNELS = {
    "sort": ["k_rs_count", "k_rs_rowscan", "k_rs_scatter", "k_cell_start", "k_gather1"],
    "moments": ["k_cells<false>"],
    "select": ["k_sel_nwords", "k_scan_*", "k_sel_count", "k_sel_emit", "k_sel_rcount", "k_sel_rscan",
               "k_sel_scatter", "k_sel_finalize"],
    "moment_match": ["k_cells<true>"],
}
COLLIDE_KERNEL = {"vhs": "k_collide_vhs", "table": "k_collide_table", "jager": "k_collide_jager",
                  "neural": "k_collide_neural"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the gas (tests)")
    ap.add_argument("--paths", default="neural,jager,table,vhs")
    ap.add_argument("--n-nodes", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-standalone", dest="standalone", action="store_false")
    ap.add_argument("--standalone-items", default="chi_batch,sort,transport,chi_mlp,mlp,train,configs",
                    help="which standalone measurements to run (comma list)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the built-in launch shapes")
    return ap.parse_args()


def phase_bytes(n, nc, pairs):
    """Algorithmic HBM bytes of each phase of one step (inputs read once,
    outputs written once): sort 56 B/particle (cell id and velocities in, perm
    and sorted velocities out) + cell_start; moments 24 B/particle + 40 B/cell;
    selection 24 B/particle + 16 B/cell ((sigma g)_max in and out) + 20 B/pair
    (pair and dependency word); collide 104 B/pair; moment matching 48
    B/particle + 40 B/cell."""
    return {"sort": 56 * n + 4 * (nc + 1), "moments": 24 * n + 40 * nc, "select": 24 * n + 16 * nc + 20 * pairs,
            "collide": 104 * pairs, "moment_match": 48 * n + 40 * nc}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def measure_pipe_peaks(C, torch, dev):
    """FP32 FMA, paired FP32 FMA, FP64 FMA and MUFU ex2 rates of this GPU
    (dsmc_selftest_peak), each the best of three launches timed with CUDA
    events: FLOP/s for the FMA kinds, operations/s for ex2."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = sms * 8, 256
    out = {}
    stream = torch.cuda.current_stream(dev)
    sink = None
    for which, name in enumerate(C.PEAK_KINDS):
        # iterations sized for about 20 ms at the nominal rates
        iters = {0: 40000, 1: 20000, 2: 800, 3: 6000}[which]
        sink, ops = C.selftest_peak(which, blocks, threads, 100, sink)   # warm-up
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sink, ops = C.selftest_peak(which, blocks, threads, iters, sink)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            rate = ops / (ms * 1e-3)
            best = rate if best is None or rate > best else best
        out[name] = best
    if C.sync_status() != 0:
        raise RuntimeError("device status after the pipe-rate kernels")
    return {"fp32_tflops": max(out["fp32_fma"], out["fp32x2_fma"]) / 1e12,
            "fp32_scalar_fma_tflops": out["fp32_fma"] / 1e12, "fp32x2_fma_tflops": out["fp32x2_fma"] / 1e12,
            "fp64_tflops": out["fp64_fma"] / 1e12, "mufu_tops": out["mufu_ex2"] / 1e12,
            "how": f"dsmc_selftest_peak: {blocks} blocks x {threads} threads, 8 dependent chains per thread, "
                   "best of 3 launches, CUDA events"}


def roof_entry(achieved, peak, unit, peak_source):
    return {"achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak if peak else None,
            "peak_source": peak_source}


def phase_rooflines(path, n, nc, pairs, phase_ms, pipe, pk, issue_peak=None):
    """Per-phase (per-kernel for the collide) achieved rates against their
    roofs: HBM for sort, moments, selection and moment matching (algorithmic
    bytes of phase_bytes); for the collide HBM (104 B/pair) and, per path,
    the tensor pipe (neural: 68,352 FLOP/pair, bf16 burst peak: the kernel
    runs inside a 4 ms step), the MUFU (neural: 480 operations/pair), and the
    FP64 / FP32 / MUFU pipes from the kernel's per-pair instruction counts
    (KERNEL_OPS); for the shared phases on the full gas also instruction
    issue (PHASE_WARP_INSTR against issue_peak warp instructions/s: 4 per
    cycle per SM at the maximum SM clock).  "bound" is the roof with the
    largest fraction."""
    hbm = pk.get("hbm_gbs") if pk else 6800.0
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if pk else "fallback 6800 GB/s"
    bf16 = pk.get("bf16_tflops") if pk else 1900.0
    bf16_src = "MEASURED_PEAKS.json bf16_tflops, burst (of measured)" if pk else "fallback 1900 TFLOP/s"
    pb = phase_bytes(n, nc, pairs)
    out = {}
    for ph, ms in phase_ms.items():
        t = ms * 1e-3
        roofs = {"hbm": roof_entry(pb[ph] / t / 1e9, hbm, "GB/s", hbm_src)}
        instr = PHASE_WARP_INSTR[0 if path == "vhs" else 1].get(ph)
        if issue_peak and instr and n == ISSUE_REF_PARTICLES:
            roofs["issue"] = roof_entry(instr / t / 1e9, issue_peak / 1e9, "Ginst/s",
                                        "nominal issue rate: 4 warp instructions per cycle per SM at the "
                                        "maximum SM clock (ncu instruction counts)")
        kern = PHASE_KERNELS.get(ph)
        if ph == "collide":
            kname = COLLIDE_KERNEL[path]
            kern = [kname]
            if path == "neural":
                roofs["tensor"] = roof_entry(pairs * MLP_FLOP_PER_PAIR / t / 1e12, bf16, "TFLOP/s", bf16_src)
                roofs["mufu"] = roof_entry(pairs * MLP_MUFU_PER_PAIR / t / 1e12, pipe["mufu_tops"], "Top/s",
                                           "dsmc_selftest_peak ex2 (of measured)")
            ops = KERNEL_OPS.get(kname)
            if ops:
                if ops.get("fp64_flop"):
                    roofs["fp64"] = roof_entry(pairs * ops["fp64_flop"] / t / 1e12, pipe["fp64_tflops"],
                                               "TFLOP/s", "dsmc_selftest_peak FP64 FMA (of measured)")
                if ops.get("fp32_flop"):
                    roofs["fp32"] = roof_entry(pairs * ops["fp32_flop"] / t / 1e12, pipe["fp32_tflops"],
                                               "TFLOP/s", "dsmc_selftest_peak FP32 FMA (of measured)")
                if ops.get("mufu"):
                    roofs["mufu"] = roof_entry(pairs * ops["mufu"] / t / 1e12, pipe["mufu_tops"], "Top/s",
                                               "dsmc_selftest_peak ex2 (of measured)")
        bound = max(roofs, key=lambda k: roofs[k]["frac"] or 0.0)
        out[ph] = {"kernels": kern, "ms": ms, "bound": bound, "frac": roofs[bound]["frac"], "roofs": roofs}
    return out


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- GPU arm

def run_gb300(args, rank, world, dist):
    import torch
    from paper_2602_21244_gb300 import dsmc as D
    from paper_2602_21244_gb300 import workloads as W

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    C = D.Context(dev.index)
    wl = W.hypersonic(scale=args.scale, seed=rank)
    n, nc = len(wl["cell_id"]), wl["n_cells"]
    capacity = max(1 << 16, int(n * 1.5))
    st = D.StepState(C, n, nc, capacity, device=dev)
    pristine = [torch.from_numpy(a).to(dev) for a in (wl["cell_id"], wl["vx"], wl["vy"], wl["vz"])]
    T_cell = torch.from_numpy(wl["T_cell"]).to(dev)
    wts = W.mlp_weights()
    w_bits = torch.from_numpy(wts["W_bits"].view(np.int16)).to(dev)
    bias = torch.from_numpy(wts["bias"].astype(np.float32)).to(dev)
    mlp = D.make_mlp(8, 128, 3, 3, 0, W.sigma_v(), 273.0, 1e-12)
    pot = D.make_potential(W.JAGER_SYNTHETIC_AR)
    stream = torch.cuda.current_stream()
    sel = st.sel
    pipe = measure_pipe_peaks(C, torch, dev)

    def restore(src=None):
        src = pristine if src is None else src
        st.cell_id.copy_(src[0]); st.vx.copy_(src[1]); st.vy.copy_(src[2]); st.vz.copy_(src[3])

    # the same gas nearly sorted: cell order with 10 % of the particles moved
    # to a neighbouring cell, as after an advection step
    order = np.argsort(wl["cell_id"], kind="stable")
    cid_ns = wl["cell_id"][order].copy()
    rng_ns = np.random.default_rng(11)
    moved = rng_ns.random(n) < 0.1
    cid_ns[moved] = np.clip(cid_ns[moved] + rng_ns.choice([-1, 1], int(moved.sum())), 0, nc - 1)
    nearly_sorted = [torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                     for a in (cid_ns.astype(np.int32), wl["vx"][order], wl["vy"][order], wl["vz"][order])]

    results = {}
    neural_kernel = None
    # the look-up path's table (Sec. 3.4.4): 512 x 512 nodes over b/b_max and
    # ln(E_r/k_B) in [ln 5, ln 6e4], filled with the exact chi (128 nodes)
    table, table_info = None, None
    if "table" in args.paths.split(","):
        gas_t = D.make_gas(dict(wl["gas"], model=1))
        tab_args = dict(nb=512, nE=512, lnE_min=math.log(5.0), lnE_max=math.log(6.0e4), n_nodes=128)
        table = C.chi_table_build(gas_t, pot, **tab_args)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        table = C.chi_table_build(gas_t, pot, **tab_args)
        e1.record(stream)
        torch.cuda.synchronize()
        table_info = dict(nodes=[512, 512], n_nodes=128, ms=e0.elapsed_time(e1),
                          lnE_range=[tab_args["lnE_min"], tab_args["lnE_max"]])
    for path in [p for p in args.paths.split(",") if p]:
        gas = D.make_gas(dict(wl["gas"], model=0 if path == "vhs" else 1))
        path_d = D.make_path({"vhs": D.PATH_VHS, "jager": D.PATH_JAGER, "neural": D.PATH_NEURAL,
                              "table": D.PATH_TABLE}[path],
                             pot=pot, n_nodes=args.n_nodes, mlp=mlp, w_bits=w_bits, bias=bias,
                             table=table if path == "table" else None)
        tuned = None
        if args.autotune:
            # launch shapes of this path's tunable kernels, measured on this gas (untimed)
            restore()
            C.sigma_g_max_init(gas, T_cell, 5.0, out=st.sigma_g_max)
            t0 = time.time()
            trials = C.autotune_step(gas, path_d, st, step=0, reps=2)
            tuned = dict(seconds=round(time.time() - t0, 3), trials=len(trials),
                         shapes={D.TUNE_KERNELS[k]: list(C.tune_get(k))
                                 for k in sorted({D.TUNE_KERNELS.index(t["kernel"]) for t in trials})})
        C.sigma_g_max_init(gas, T_cell, 5.0, out=st.sigma_g_max)
        ev = lambda: torch.cuda.Event(enable_timing=True)
        phase_ms = {k: 0.0 for k in ("sort", "moments", "select", "collide", "moment_match")}
        step_ms, pairs, rounds = 0.0, 0, []
        launches0 = None
        for it in range(args.warmup + args.steps):
            restore()
            timed = it >= args.warmup
            if timed and launches0 is None:
                torch.cuda.synchronize()
                launches0 = C.launch_count()
            e = [ev() for _ in range(6)]
            e[0].record(stream)
            C.sort_cells(st.cell_id, st.vx, st.vy, st.vz, nc,
                         out=dict(perm=st.perm, cell_start=st.cell_start, svx=st.svx, svy=st.svy, svz=st.svz),
                         ws=st.ws)
            e[1].record(stream)
            C.cell_moments(st.cell_start, st.svx, st.svy, st.svz, mom=st.mom)
            e[2].record(stream)
            C.select_pairs(gas, st.cell_start, st.svx, st.svy, st.svz, st.sigma_g_max, it, capacity,
                           out=sel, ws=st.ws, order=D.ORDER_LEVELS if path == "neural" else D.ORDER_ROUNDS)
            e[3].record(stream)
            if path == "vhs":
                C.collide_vhs(gas, it, sel, st.svx, st.svy, st.svz)
            elif path == "jager":
                C.collide_jager(gas, pot, it, sel, st.svx, st.svy, st.svz, n_nodes=args.n_nodes)
            elif path == "table":
                C.collide_table(gas, table, it, sel, st.svx, st.svy, st.svz)
            else:
                C.collide_neural(gas, mlp, w_bits, bias, it, st.mom, sel, st.svx, st.svy, st.svz)
            e[4].record(stream)
            C.moment_match(st.cell_start, st.mom, st.svx, st.svy, st.svz)
            e[5].record(stream)
            if timed:
                torch.cuda.synchronize()
                rc = C.sync_status()
                if rc != 0:
                    raise RuntimeError(f"device status {rc} on path {path}")
                names = list(phase_ms)
                for q in range(5):
                    phase_ms[names[q]] += e[q].elapsed_time(e[q + 1])
                step_ms += e[0].elapsed_time(e[5])
                inf = st.info_host()
                pairs += inf["n_pairs"]
                rounds.append(inf["n_rounds"])
        launches = C.launch_count() - launches0
        K = args.steps
        # the same step as one CUDA graph (the production path): timed alone
        gstream = torch.cuda.Stream(device=dev)
        torch.cuda.synchronize()
        C.sigma_g_max_init(gas, T_cell, 5.0, out=st.sigma_g_max)
        C.step_graph_capture(gas, path_d, st, gstream)
        g_ms, g_pairs, lg0 = 0.0, 0, None
        for it in range(args.warmup + args.steps):
            if it == args.warmup:
                torch.cuda.synchronize()
                lg0 = C.launch_count()
            with torch.cuda.stream(gstream):
                restore()
                e0, e1 = ev(), ev()
                e0.record(gstream)
                C.step_graph_launch(it, gstream)
                e1.record(gstream)
            if it >= args.warmup:
                torch.cuda.synchronize()
                if C.sync_status(gstream) != 0:
                    raise RuntimeError(f"device status on graph path {path}")
                g_ms += e0.elapsed_time(e1)
                g_pairs += st.info_host()["n_pairs"]
        torch.cuda.synchronize()
        g_launches = C.launch_count() - lg0
        fused = None
        if path in ("vhs", "table"):
            # the same step fused into one pass over cell groups (dsmc_step_fused),
            # on the shuffled gas; then both forms on the nearly sorted one
            def timed(run, src, s=stream):
                C.sigma_g_max_init(gas, T_cell, 5.0, out=st.sigma_g_max)
                torch.cuda.synchronize()
                t_ms, t_pairs, l0 = 0.0, 0, None
                for it in range(args.warmup + args.steps):
                    if it == args.warmup:
                        torch.cuda.synchronize()
                        l0 = C.launch_count()
                    with torch.cuda.stream(s):
                        restore(src)
                        e0, e1 = ev(), ev()
                        e0.record(s)
                        run(it)
                        e1.record(s)
                    if it >= args.warmup:
                        torch.cuda.synchronize()
                        if C.sync_status(s) != 0:
                            raise RuntimeError(f"device status on {path}")
                        t_ms += e0.elapsed_time(e1)
                        t_pairs += st.info_host()["n_pairs"]
                torch.cuda.synchronize()
                return dict(collisions_per_s=t_pairs / (t_ms * 1e-3), ms_per_step=t_ms / K,
                            gpu_launches=C.launch_count() - l0)
            fused = timed(lambda it: C.step_fused(gas, path_d, st, it), None)
            # the unfused step as the graph captured above
            fused["nearly_sorted"] = dict(
                unfused=timed(lambda it: C.step_graph_launch(it, gstream), nearly_sorted, gstream),
                fused=timed(lambda it: C.step_fused(gas, path_d, st, it), nearly_sorted))
        pb = phase_bytes(n, nc, pairs / K)
        pk = peaks()
        hbm = pk.get("hbm_gbs") if pk else 6800.0
        phase_gbs = {k: pb[k] / (phase_ms[k] / K * 1e-3) / 1e9 for k in pb}
        sm_clk = (pk.get("sm_max_mhz") if pk else None) or 2070.0
        issue_peak = torch.cuda.get_device_properties(dev).multi_processor_count * 4 * sm_clk * 1e6
        roofs = phase_rooflines(path, n, nc, pairs / K, {k: v / K for k, v in phase_ms.items()}, pipe, pk,
                                issue_peak)
        results[path] = dict(
            rooflines=roofs,
            collisions_per_s=g_pairs / (g_ms * 1e-3), ms_per_step=g_ms / K,
            phase_gbs=phase_gbs, phase_hbm_frac={k: v / hbm for k, v in phase_gbs.items()},
            phased=dict(collisions_per_s=pairs / (step_ms * 1e-3), ms_per_step=step_ms / K),
            pairs_per_step=pairs / K, rounds_per_step=float(np.mean(rounds)),
            phase_ms={k: v / K for k, v in phase_ms.items()}, gpu_launches=g_launches,
            phased_gpu_launches=launches,
            step_ms_total=step_ms, pairs_total=pairs, autotune=tuned, fused=fused)
        if path == "neural":
            neural_kernel = dict(ms=phase_ms["collide"] / K, pairs=pairs / K)
    # ------------------------------------------------------------ standalone kernels
    # Jager deflection-angle batch (2^22 pairs) and the MLP alone (2^22 rows)
    extra = {}
    if table_info is not None:
        extra["chi_table"] = table_info
    items = set(args.standalone_items.split(",")) if args.standalone else set()
    if "chi_batch" in items:
        nb = 1 << 22
        b_np, g_np = W.chi_pairs(nb, seed=0)
        bt, gt = torch.from_numpy(b_np).to(dev), torch.from_numpy(g_np).to(dev)
        chi = torch.empty_like(bt)
        gas1 = D.make_gas(dict(wl["gas"], model=1))
        chi_tuned = None
        if args.autotune:
            C.autotune_chi(gas1, pot, bt, gt, n_nodes=args.n_nodes, chi=chi, reps=2)
            chi_tuned = list(C.tune_get(D.TUNE_KERNELS.index("jager_chi")))
        for _ in range(2):
            C.jager_chi(gas1, pot, bt, gt, n_nodes=args.n_nodes, chi=chi)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            C.jager_chi(gas1, pot, bt, gt, n_nodes=args.n_nodes, chi=chi)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        extra["chi_batch"] = dict(pairs=nb, ms=ms, chi_per_s=nb / (ms * 1e-3), n_nodes=args.n_nodes,
                                  shape=chi_tuned)
        ops = KERNEL_OPS.get("k_jager_chi")
        if ops:
            roofs = {k: roof_entry(nb * ops[o] / (ms * 1e-3) / 1e12, pipe[pk_], u, f"dsmc_selftest_peak (of measured)")
                     for k, o, pk_, u in (("fp64", "fp64_flop", "fp64_tflops", "TFLOP/s"),
                                          ("fp32", "fp32_flop", "fp32_tflops", "TFLOP/s"),
                                          ("mufu", "mufu", "mufu_tops", "Top/s")) if ops.get(o)}
            bound = max(roofs, key=lambda k: roofs[k]["frac"])
            extra["chi_batch"]["roofline"] = {"kernel": "k_jager_chi", "bound": bound, "frac": roofs[bound]["frac"],
                                              "roofs": roofs}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nb = 1 << 22
    gas1 = D.make_gas(dict(wl["gas"], model=1))
    if "sort" in items:
        # the sort alone on the shuffled gas of the step and on a nearly sorted one
        # (cell order with 10 % of the particles moved to a neighbouring cell, as
        # after an advection step)
        srt_out = dict(perm=st.perm, cell_start=st.cell_start, svx=st.svx, svy=st.svy, svz=st.svz)
        sort_ms = {}
        for name, inp in (("shuffled", pristine), ("nearly_sorted", nearly_sorted)):
            for _ in range(2):
                C.sort_cells(*inp, nc, out=srt_out, ws=st.ws)
            e0.record(stream)
            for _ in range(5):
                C.sort_cells(*inp, nc, out=srt_out, ws=st.ws)
            e1.record(stream)
            torch.cuda.synchronize()
            sort_ms[name] = e0.elapsed_time(e1) / 5
        extra["sort"] = dict(particles=n, ms=sort_ms,
                             gbs={k: phase_bytes(n, nc, 0)["sort"] / (v * 1e-3) / 1e9 for k, v in sort_ms.items()})
    if "transport" in items:
        # transport integrals: Omega(2,2)(T) and mu(T) at 64 temperatures (500 K to 20,000 K),
        # 32 b-panels x 8 x-panels of 16 nodes: 65,536 chi per temperature
        Tt = torch.from_numpy(np.geomspace(500.0, 2.0e4, 64)).to(dev)
        gas_m = D.make_gas(dict(wl["gas"], model=1))
        for _ in range(2):
            om, mu_t = C.transport_viscosity(gas_m, pot, Tt, n_nodes=args.n_nodes)
        e0.record(stream)
        om, mu_t = C.transport_viscosity(gas_m, pot, Tt, n_nodes=args.n_nodes)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        mu_h = mu_t.cpu().numpy()
        extra["transport"] = dict(temperatures=64, chi_evaluations=64 * 128 * 512, ms=ms,
                                  chi_per_s=64 * 128 * 512 / (ms * 1e-3), n_nodes=args.n_nodes,
                                  mu_Pa_s={"500K": float(mu_h[0]), "20000K": float(mu_h[-1])})
    if "chi_mlp" in items:
        # chi-MLP surrogate: the 512 x 512 look-up table synthesised on the tensor cores
        cw = W.chi_mlp_weights()
        cpk = C.chi_mlp_pack(torch.from_numpy(cw["W_bits"].view(np.int16)).to(dev))
        cb = torch.from_numpy(cw["bias"].astype(np.float32)).to(dev)
        ct = C.chi_mlp_table(cpk, cb, 512, 512)
        for _ in range(2):
            C.chi_mlp_table(cpk, cb, 512, 512, out=ct)
        e0.record(stream)
        for _ in range(5):
            C.chi_mlp_table(cpk, cb, 512, 512, out=ct)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        pk = peaks()
        peak = pk.get("bf16_tflops") if pk else 1900.0
        tf = 512 * 512 * CHI_MLP_FLOP_PER_QUERY / (ms * 1e-3) / 1e12
        extra["chi_mlp_table"] = dict(nodes=[512, 512], ms=ms, queries_per_s=512 * 512 / (ms * 1e-3), tflops=tf,
                                      frac_of_bf16_peak=tf / peak)
    if "mlp" in items:
        x = torch.randn((nb, 8), dtype=torch.float32, device=dev)
        y = torch.empty((nb, 3), dtype=torch.float32, device=dev)
        for _ in range(2):
            C.mlp_forward(mlp, w_bits, bias, x, y)
        e0.record(stream)
        for _ in range(3):
            C.mlp_forward(mlp, w_bits, bias, x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        pk = peaks()
        peak = pk.get("bf16_tflops") if pk else 1900.0
        tf = nb * MLP_FLOP_PER_PAIR / (ms * 1e-3) / 1e12
        extra["mlp_forward"] = dict(rows=nb, ms=ms, rows_per_s=nb / (ms * 1e-3), tflops=tf,
                                    frac_of_bf16_peak=tf / peak)
    if "train" in items:
        # training step on 2^20 pairs harvested by the Jager kernel (forward,
        # recomputing backward, Adam)
        nt = 1 << 20
        hv = W.harvest_inputs(nt, seed=0)
        hvi, hvj = torch.from_numpy(hv["vi"]).to(dev), torch.from_numpy(hv["vj"]).to(dev)
        hT = torch.from_numpy(hv["T"]).to(dev)
        vit, vjt = C.harvest_jager(gas1, pot, hvi, hvj, torch.from_numpy(hv["b"]).to(dev),
                                   torch.from_numpy(hv["eps"]).to(dev), n_nodes=args.n_nodes)
        theta = torch.from_numpy(np.concatenate([wts["W"], wts["bias"]]).astype(np.float32)).to(dev)
        m_, v_ = torch.zeros_like(theta), torch.zeros_like(theta)
        grad = torch.empty_like(theta)
        lossb = torch.zeros(1, dtype=torch.float64, device=dev)
        tws = C.train_workspace(dev)
        for stp in (1, 2):
            C.train_step(mlp, theta, m_, v_, stp, 1e-3, 0, hvi, hvj, hT, vit, vjt, grad, lossb, tws)
        e0.record(stream)
        for stp in range(3, 6):
            C.train_step(mlp, theta, m_, v_, stp, 1e-3, 0, hvi, hvj, hT, vit, vjt, grad, lossb, tws)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        # algorithmic MMA work: forward + recomputation + two backward GEMMs ~ 4 x the forward
        tf = 4 * nt * MLP_FLOP_PER_PAIR / (ms * 1e-3) / 1e12
        extra["train_step"] = dict(pairs=nt, ms=ms, steps_per_s=1e3 / ms, pairs_per_s=nt / (ms * 1e-3),
                                   tflops=tf, loss=float(lossb.item()))
    if C.sync_status() != 0:
        raise RuntimeError("device status after standalone kernels")
    # ------------------------------------------------------------ e2e (host buffers)
    e2e = None
    if not args.no_e2e and "neural" in results:
        import torch as T
        gas = D.make_gas(dict(wl["gas"], model=1))
        path = D.make_path(D.PATH_NEURAL, mlp=mlp, w_bits=w_bits, bias=bias)
        C.reserve(n, nc, capacity)
        pin = lambda a: T.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hin = [pin(wl["cell_id"]), pin(wl["vx"]), pin(wl["vy"]), pin(wl["vz"])]
        hT = pin(wl["T_cell"])
        outs = [T.empty(n, dtype=T.float64).pin_memory() for _ in range(3)]
        perm = T.empty(n, dtype=T.int32).pin_memory()
        for it in range(args.warmup):
            C.step_host(gas, path, *hin, hT, it, perm, *outs)
        t0 = time.perf_counter()
        tot = 0
        for it in range(args.steps):
            tot += C.step_host(gas, path, *hin, hT, it, perm, *outs)
        dt = time.perf_counter() - t0
        e2e = dict(value=tot / dt, unit="pair collisions/s",
                   h2d_bytes_per_step=n * (4 + 24), d2h_bytes_per_step=n * (4 + 24) + 24)
    # ------------------------------------------------------------ the two other gas configurations
    if "configs" in items:
        extra["configs"] = other_configs(C, D, W, torch, dev, args, mlp, w_bits, bias)
    extra["pipe_peaks"] = pipe
    return wl, n, nc, results, neural_kernel, e2e, extra


def other_configs(C, D, W, torch, dev, args, mlp, w_bits, bias):
    """The Couette gas (100 cells x 50 particles, VHS, 100 consecutive steps,
    each step's sorted output the next step's input; launch-bound at this
    size) and the cavity (200 x 200 cells, Poisson(20) particles per cell,
    neural path, pristine input restored before every step); every step one
    CUDA graph launch, timed with CUDA events."""
    out = {}
    stream = torch.cuda.current_stream()
    for name, wl, kind, steps in (("couette", W.couette(), D.PATH_VHS, 100),
                                  ("cavity", W.cavity(), D.PATH_NEURAL, max(args.steps, 5))):
        n, nc = len(wl["cell_id"]), wl["n_cells"]
        st = D.StepState(C, n, nc, max(1 << 16, 2 * n), device=dev)
        # both gases select with Bird's VHS cross-section (the cavity's ~80k
        # accepted pairs per step); the cavity's pairs collide by the network
        gas = D.make_gas(dict(wl["gas"], model=0))
        path = D.make_path(kind, mlp=mlp, w_bits=w_bits, bias=bias)
        src = [torch.from_numpy(a).to(dev) for a in (wl["cell_id"], wl["vx"], wl["vy"], wl["vz"])]
        C.sigma_g_max_init(gas, torch.from_numpy(wl["T_cell"]).to(dev), 5.0, out=st.sigma_g_max)
        gs = torch.cuda.Stream(device=dev)
        torch.cuda.synchronize()
        C.step_graph_capture(gas, path, st, gs)
        sorted_id = None
        ms, pairs, cand = 0.0, 0, 0
        for it in range(args.warmup + steps):
            with torch.cuda.stream(gs):
                if name == "couette":
                    if it == 0 or it == args.warmup:
                        st.cell_id.copy_(src[0]); st.vx.copy_(src[1]); st.vy.copy_(src[2]); st.vz.copy_(src[3])
                    else:   # carry the gas: sorted cell ids and post-collision velocities
                        st.cell_id.copy_(sorted_id); st.vx.copy_(st.svx); st.vy.copy_(st.svy); st.vz.copy_(st.svz)
                else:
                    st.cell_id.copy_(src[0]); st.vx.copy_(src[1]); st.vy.copy_(src[2]); st.vz.copy_(src[3])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(gs)
                C.step_graph_launch(it, gs)
                e1.record(gs)
            torch.cuda.synchronize()
            if name == "couette" and sorted_id is None:
                sorted_id = src[0][st.perm.long()].contiguous()
            if it >= args.warmup:
                if C.sync_status(gs) != 0:
                    raise RuntimeError(f"device status on {name}")
                ms += e0.elapsed_time(e1)
                inf = st.info_host()
                pairs += inf["n_pairs"]
                cand += inf["n_candidates"]
        out[name] = dict(workload=wl["name"], particles=n, cells=nc, path="vhs" if kind == D.PATH_VHS else "neural",
                         steps=steps, ms_per_step=ms / steps, collisions_per_s=pairs / (ms * 1e-3),
                         pairs_per_step=pairs / steps, candidates_per_step=cand / steps,
                         note="launch-bound at this size" if name == "couette" else None)
    return out


# ---------------------------------------------------------------------------- oracle arm

def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                name = line.split(":", 1)[1].strip()
                if name and not name.isdigit():
                    return name
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_sample(path="neural", steps=1, threads=None):
    """Time the CPU oracle (as it stands) on a bounded sample of the same gas:
    the hypersonic profile shrunk to 0.2 of the box (same shock shape), one
    whole step (sort, moments, selection, collide, moment matching) on
    `threads` host threads (None: all of them)."""
    import oracle as O
    from paper_2602_21244_gb300 import workloads as W
    n_all = O.num_threads()
    O.set_num_threads(threads if threads else n_all)
    used = O.num_threads()
    try:
        wl = W.hypersonic(scale=0.2)
        gas = O.make_gas(**dict(wl["gas"], model=1 if path != "vhs" else 0))
        sg = O.sigma_g_max_init(gas, wl["T_cell"], 5.0)
        wts = W.mlp_weights()
        mlp = O.make_mlp(8, 128, 3, 3, 0, W.sigma_v(), 273.0, 1e-12)
        pot = O.make_pot(W.JAGER_SYNTHETIC_AR)
        t0 = time.perf_counter()
        pairs = 0
        for st in range(steps):
            r = O.step(gas, wl["cell_id"], wl["vx"], wl["vy"], wl["vz"], wl["n_cells"], sg, st, path=path,
                       pot=pot, mlp=mlp, W=wts["W"], bias=wts["bias"], capacity=1 << 23)
            pairs += r["pairs"]["n_pairs"]
        dt = time.perf_counter() - t0
    finally:
        O.set_num_threads(n_all)
    return dict(value=pairs / dt, unit="pair collisions/s", cores=used, kind="oracle",
                sample=f"hypersonic gas at 0.2 scale ({len(wl['cell_id'])} particles, "
                       f"{wl['n_cells']} cells), {steps} full {path} step(s), {pairs} collisions, "
                       f"{dt:.1f} s on {used} thread(s)")


def cpu_baseline_both(path="neural"):
    """The oracle on all host threads (the reported value) and on one."""
    allc = oracle_sample(path=path)
    one = oracle_sample(path=path, threads=1)
    return dict(allc, cpu_model=cpu_model(), nproc=os.cpu_count(),
                single_thread={"value": one["value"], "cores": 1, "sample": one["sample"]})


def aggregate(ms, pairs, dist, device="cpu"):
    """Replicas: the job's time is the slowest rank's, its work the sum of the
    ranks' pairs; value = summed pairs / slowest time (pairs per second)."""
    if dist is None:
        return ms, pairs / (ms * 1e-3)
    import torch
    t = torch.tensor([ms, pairs], dtype=torch.float64, device=device)
    mx = t.clone(); dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone(); dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]) / (float(mx[0]) * 1e-3)


def headline_config(name, n, nc, path, world):
    """The workload the headline is quoted on (both arms report the same)."""
    return {"workload": f"hypersonic argon gas {name}, {n} particles, {nc} cells", "path": path,
            "l2": "pristine 258 MB input copied back before every step",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo" if args.impl == "reference" else "nccl")
    if args.impl == "reference":
        if rank == 0:
            from paper_2602_21244_gb300 import workloads as W
            full = W.hypersonic()   # the headline workload, for its config; the oracle times a sample
            cfg = headline_config(full["name"], len(full["cell_id"]), full["n_cells"], "neural", 1)
            del full
            for _ in range(args.warmup):
                oracle_sample(steps=1)   # untimed
            vals = []
            for _ in range(args.steps):
                vals.append(oracle_sample(steps=1))
            v = float(np.mean([x["value"] for x in vals]))
            cb = dict(vals[0], value=v, cpu_model=cpu_model(), nproc=os.cpu_count())
            line = {"impl": "reference", "metric": "pair collisions/s per update path (neural path, whole step)",
                    "value": v, "unit": "pair collisions/s", "n_gpus": args.gpus, "steps": args.steps,
                    "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                    "dtype": "f64", "data": "synthetic",
                    "config": cfg,
                    "cpu_baseline": cb,
                    "e2e": {"value": v, "unit": "pair collisions/s", "h2d_bytes_per_step": 0,
                            "d2h_bytes_per_step": 0}}
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    import torch
    clk = Clocks(int(os.environ.get("LOCAL_RANK", 0)))
    if dist is not None:
        dist.barrier()
    clk.start()
    wl, n, nc, results, nk, e2e, extra = run_gb300(args, rank, world, dist)
    clocks = clk.stop()
    head = results.get("neural") or next(iter(results.values()))
    head_path = "neural" if "neural" in results else next(iter(results))
    ms = head["ms_per_step"]
    value = head["collisions_per_s"]
    if dist is not None:
        ms, value = aggregate(ms, head["pairs_per_step"], dist, device="cuda")
    if rank == 0:
        pk = peaks()
        roof = None
        if nk is not None:
            # the kernel is timed inside a ~4 ms step, not a seconds-long loop: burst peak
            achieved = nk["pairs"] * MLP_FLOP_PER_PAIR / (nk["ms"] * 1e-3) / 1e12
            peak = pk.get("bf16_tflops") if pk else 1900.0
            roof = {"bound": "tensor", "kernel": "k_collide_neural", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": NEURAL_DRAM_BYTES_PER_PAIR * nk["pairs"] if NEURAL_DRAM_BYTES_PER_PAIR else None,
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, of measured)" if pk
                    else "fallback 1900 TFLOP/s"}
        cb = None
        if not args.no_cpu_baseline:
            cb = cpu_baseline_both()
        line = {"metric": "pair collisions/s per update path (neural path, whole step)",
                "value": value, "unit": "pair collisions/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": headline_config(wl["name"], n, nc, head_path, world),
                "paths": results, "standalone": extra, "roofline": roof, "cpu_baseline": cb, "e2e": e2e,
                "gpu_launches": int(sum(r["gpu_launches"] for r in results.values())),
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
